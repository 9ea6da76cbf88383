"""Host planner of the single-launch attempts (attempt_small.h) without a GPU: which
meshes take the single launch, how rows and column units split over a cluster, and the
shared-memory layout of a CTA, through a host-only probe compiled with nvcc
(tests/small_probe.cu)."""
import json
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SHAPES = [(nx, ny) for nx in (1, 2, 3, 5, 16, 17, 31, 32, 33) for ny in (1, 2, 7, 16, 17, 32, 33)]


@pytest.fixture(scope="module")
def rows(tmp_path_factory):
    nvcc = next((c for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc"))
                 if c and os.path.exists(c)), None)
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = str(tmp_path_factory.mktemp("small") / "small_probe")
    subprocess.run([nvcc, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I", os.path.join(ROOT, "paper_2406_16064_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "small_probe.cu"), "-o", exe], check=True, capture_output=True)
    out = subprocess.run([exe], input="".join(f"{a} {b}\n" for a, b in SHAPES), capture_output=True, text=True,
                         check=True).stdout
    return [json.loads(l) for l in out.splitlines()]


def test_eligible_exactly_the_films_of_at_most_32x32_cells(rows):
    assert len(rows) == len(SHAPES)
    for r in rows:
        nx, ny = r["mesh"]
        assert r["eligible"] == (1 if nx <= 32 and ny <= 32 else 0), r["mesh"]
        assert r["halves"] == (2 if r["Py"] == 64 else 1)


def test_rows_and_units_cover_the_mesh_once(rows):
    for r in rows:
        if not r["eligible"]:
            continue
        nx, ny = r["mesh"]
        units = r["Kx"] * r["halves"]
        for nc, v in r["nc"].items():
            nc = int(nc)
            owned_rows = [y for b in range(nc) for y in range(b * v["rb"], min(ny, (b + 1) * v["rb"]))]
            owned_units = [u for b in range(nc) for u in range(b * v["cu"], min(units, (b + 1) * v["cu"]))]
            assert owned_rows == list(range(ny)) and owned_units == list(range(units)), (r["mesh"], nc)
            # the owner of a row / unit as the kernel computes it (index // block size) is in the cluster
            assert (ny - 1) // v["rb"] < nc and (units - 1) // v["cu"] < nc


def test_layout_fits_one_cta_and_keeps_the_buffers_apart(rows):
    for r in rows:
        if not r["eligible"]:
            continue
        nx, ny = r["mesh"]
        for nc, v in r["nc"].items():
            for prec, e in (("f32", 4), ("f64", 8)):
                halo, colin, spec, rowin, w64, tens, total = v[prec]
                rb, cu, H = v["rb"], v["cu"], r["halves"]
                z = 2 * e
                assert halo == 14 * 3 * rb * nx * e
                assert colin >= halo + 12 * nx * e and colin % 16 == 0
                assert spec == colin + 3 * cu * ny * z
                lyh = r["Py"] // H
                assert rowin == spec + 3 * cu * (lyh + lyh // 8 + 1) * z    # padded rows
                assert w64 == rowin + 3 * rb * r["Kx"] * H * z
                assert tens == w64 + 64 * z
                assert total >= tens + 4 * cu * (r["Py"] // H) * e and total % 16 == 0
                if int(nc) == 16:
                    # the cluster the library picks first fits one CTA's shared memory
                    assert total <= 227 * 1024, (r["mesh"], prec, total)
