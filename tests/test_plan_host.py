"""Host planner (plan.h) without a GPU: padded FFT lengths, tile shapes, the work
lists of every pass and the term flags, through a host-only probe compiled with nvcc
(tests/plan_probe.cu)."""
import json
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
F_DEMAG, F_DMI, F_EX, F_EXT = 1, 2, 16, 128
E_CELL, E_STT, E_SOT = 1, 2, 4
MESHES = [(1, 1, 1), (2, 1, 1), (32, 32, 1), (33, 17, 2), (9, 6, 5), (6, 5, 8), (5, 4, 9), (70, 3, 1),
          (512, 512, 4), (256, 256, 256), (4096, 2, 1), (1, 6, 4), (5, 1, 6), (2048, 3, 1), (100, 100, 3)]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    return None


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = str(tmp_path_factory.mktemp("probe") / "plan_probe")
    subprocess.run([nvcc, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I", os.path.join(ROOT, "paper_2406_16064_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "plan_probe.cu"), "-o", exe], check=True, capture_output=True)
    lines = "".join(f"{nx} {ny} {nz} {f}\n" for (nx, ny, nz) in MESHES for f in (0, 1))
    out = subprocess.run([exe], input=lines, capture_output=True, text=True, check=True).stdout
    rows = [json.loads(l) for l in out.splitlines()]
    return [r for r in rows if "mesh" in r], [r for r in rows if "flags_case" in r]


def _pad(n, min2=False):
    if n <= 1:
        return 2 if min2 else 1
    p = 1
    while p < 2 * n - 1:
        p *= 2
    return p


def test_padded_sizes_and_tiles(probe):
    meshes, _ = probe
    assert len(meshes) == 2 * len(MESHES)
    for r in meshes:
        nx, ny, nz = r["mesh"]
        assert (r["Px"], r["Py"], r["Pz"]) == (_pad(nx, True), _pad(ny), _pad(nz)), r["mesh"]
        assert r["Kx"] == r["Px"] // 2 + 1 and r["ncomp"] == (6 if r["Pz"] > 1 else 4)
        Ty = r["Ty"]
        assert Ty & (Ty - 1) == 0 and 1 <= Ty <= 32
        assert r["Py"] * Ty <= max(4096 if r["f32"] else 2048, r["Py"])
        assert r["NBx"] * Ty >= r["Kx"] > (r["NBx"] - 1) * Ty
        assert r["spec"] == 3 * nz * r["NBx"] * r["Py"] * Ty
        # every mesh mm_add_sim accepts (padded lengths <= 8192 FP32, 4096 FP64) fits one CTA's
        # shared memory (x passes keep 4 KB for static arrays)
        lim = 8192 if r["f32"] else 4096
        if max(r["Px"], r["Py"], r["Pz"]) <= lim:
            sx, sxi, sy13, sz, sy2, syzc = r["smem"]
            cap = 227 * 1024
            assert max(sx, sxi) <= cap - 4096 and max(sy13, sz, sy2, syzc) <= cap, r["mesh"]


def test_x_tiles_cover_every_row_once_within_a_plane(probe):
    meshes, _ = probe
    for r in meshes:
        nx, ny, nz = r["mesh"]
        seen = []
        for sim, a, b, _ in r["x"]:
            assert sim == 0 and 1 <= b <= r["Rx"]
            assert a // ny == (a + b - 1) // ny, r["mesh"]      # never crosses a plane
            seen.extend(range(a, a + b))
        assert sorted(seen) == list(range(ny * nz)), r["mesh"]


def test_demag_column_lists(probe):
    """Films of 2..8 planes: one cluster item per kx block in the list of their plane count
    and group width; deeper meshes: y forward/inverse items per (plane, block, component) and
    z items per (ky, block); single planes: one y item per block."""
    meshes, _ = probe
    for r in meshes:
        nx, ny, nz = r["mesh"]
        Py, Pz, NBx, Ty = r["Py"], r["Pz"], r["NBx"], r["Ty"]
        blocks = list(range(NBx))
        if Pz > 1 and Py > 1 and nz <= 8:
            assert r["yzc"] == 1
            assert sorted(it[2] for it in r["yzc_items"]) == blocks
            wide = r["f32"] and Py in (32, 512, 8192)
            assert r["yzc_list"] == nz + 9 * wide
            qp = ((6 * nz + 3) // 4) * 4
            assert r["tens"] == NBx * (Py // 2 + 1) * Ty * qp
            assert not r["y13"] and not r["z"] and not r["y2"]
        elif Pz > 1:
            assert r["yzc"] == 0 and not r["yzc_items"] and not r["y2"]
            if Py > 1:
                assert sorted((a, b, c) for _, a, b, c in r["y13"]) == \
                    sorted((z, b, c) for z in range(nz) for b in blocks for c in range(3))
            else:
                assert not r["y13"]
            assert sorted((a, b) for _, a, b, _ in r["z"]) == sorted((ky, b) for ky in range(Py) for b in blocks)
            assert r["tens"] == r["ncomp"] * (Pz // 2 + 1) * (Py // 2 + 1) * r["Kx"]
        elif Py > 1:
            assert sorted(it[2] for it in r["y2"]) == blocks and not r["y13"] and not r["z"]
        else:
            assert not (r["y13"] or r["z"] or r["y2"] or r["yzc_items"])


def test_term_flags(probe):
    """F_DMI / F_EX from the constants; F_EXT for bulk or D_2d DMI, per-cell constants or
    spin torques, where per-cell values switch exchange and DMI on; E_* for each extension."""
    _, flags = probe
    for r in flags:
        kind, D, A, cells, a_any, d_any, ux, aJ = r["flags_case"]
        ext = kind >= 2 or cells or ux != 0 or aJ != 0
        ex = A != 0 or (ext and cells and a_any)
        dmi = (kind == 1 and D != 0) if not ext else (kind != 0 and (D != 0 or (cells and d_any)))
        want = (F_EXT if ext else 0) | (F_EX if ex else 0) | (F_DMI if dmi else 0)
        assert r["flags"] == want, r
        want_e = (E_CELL if cells else 0) | (E_STT if ux != 0 else 0) | (E_SOT if aJ != 0 else 0)
        assert r["eflags"] == want_e, r


def test_autotuner_candidates(probe):
    """Every candidate of every phase fits the kernels (power-of-two Ty <= 32 and at most
    the next power of two above Kx, 1 <= Rx <= ny, shared memory within a CTA's, CTA
    widths multiples of 32 up to the launch bound); the first candidate of each phase is
    its starting point (the rule in phase 0); the column group width only varies for FP32
    cluster-pass films, and selects the 32-point list when it is 2."""
    meshes, _ = probe
    cap = 227 * 1024
    for r in meshes:
        ph0, ph1, ph2 = r["cands"]
        if max(r["smem"][:2]) > cap - 4096:          # the mesh itself is refused (mm_add_sim)
            assert not ph0
            continue
        assert ph0 and ph1 and ph2
        assert (ph0[0]["pTy"], ph0[0]["pRx"]) == (r["Ty"], r["Rx"])
        maxth = 1024 if r["f32"] else 512
        kx2 = 1
        while kx2 < r["Kx"]:
            kx2 *= 2
        for c in ph0 + ph1 + ph2:
            Ty, Rx = c["pTy"], c["pRx"]
            assert Ty & (Ty - 1) == 0 and 1 <= Ty <= min(32, max(kx2, r["Ty"]))
            assert 1 <= Rx <= r["mesh"][1]
            sx, sxi, sy13, sz, sy2, syzc = c["smem"]
            assert max(sx, sxi) <= cap - 4096 and max(sy13, sz, sy2, syzc) <= cap
            assert c["st"] in (0, 1)
            for th in (c["xt"], c["ct"]):
                assert th == 0 or (th % 32 == 0 and 32 <= th <= maxth)
            if c["g"]:
                assert r["f32"] and r["yzc"]
                occ = {0: 0, 3: 1, 4: 2}[c["occ"]]
                assert c["list"] == r["mesh"][2] + 9 * (c["g"] - 1) + 18 * occ
            if c["occ"]:
                # three or four CTAs per SM: FP32, at most 4 planes, that many column tiles in 228 KB
                assert c["occ"] in (3, 4)
                assert r["f32"] and r["yzc"] and r["mesh"][2] <= 4 and c["occ"] * (syzc + 1024) <= 233472
        if not (r["f32"] and r["yzc"]):
            assert all(c["g"] == 0 for c in ph0)
        # phase 1 starts from phase 0's start, phase 2 from phase 1's
        assert (ph1[0]["Ty"], ph1[0]["g"]) == (ph0[0]["Ty"], ph0[0]["g"])
        assert (ph2[0]["Rx"], ph2[0]["xt"]) == (ph1[0]["Rx"], ph1[0]["xt"])
