"""The C-ABI library builds, loads and exports every symbol include/mm.h declares (no GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "mm.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mm_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2406_16064_gb300 import build, mm
    if not os.path.exists(mm.LIB_PATH):
        build.build()
    return mm.LIB_PATH


def test_every_declared_symbol_is_exported(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (mm_[a-z0-9_]+)\b", out))
    missing = [s for s in _declared() if s not in exported]
    assert not missing, missing
    assert len(_declared()) >= 20


def test_binding_covers_the_abi(libpath):
    from paper_2406_16064_gb300 import mm
    assert set(_declared()) == set(mm.SIGNATURES)
    L = mm.lib()
    for name in _declared():
        assert getattr(L, name) is not None


def test_create_without_gpu_fails_loudly(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2406_16064_gb300 import mm
    with pytest.raises(mm.MMError) as e:
        mm.Context("f64")
    assert e.value.code == mm.MM_ECUDA


def test_struct_layouts_match_the_header(libpath):
    import ctypes
    from paper_2406_16064_gb300 import mm
    assert ctypes.sizeof(mm.mm_mesh) == 3 * 4 + 4 + 3 * 8
    # Ms A D (24) + int+pad (8) + Ku u[3] Kc (40) + H[3] (24) + alpha gamma (16) + 2 ints (8)
    assert ctypes.sizeof(mm.mm_material) == 120
    assert ctypes.sizeof(mm.mm_status) == 4 * 8 + 2 * 8 + 2 * 4
    # t h t_end rtol max_dmdt (40) + two counters (16) + status, pad (8)
    assert ctypes.sizeof(mm.mm_checkpoint) == 5 * 8 + 2 * 8 + 2 * 4


def test_bounded_wait_rejects_spins_beyond_the_limit(libpath):
    """The range check runs before anything else, so it needs neither a context nor a GPU."""
    import ctypes
    from paper_2406_16064_gb300 import mm
    L = mm.lib()
    for spins in (-1, (1 << 22) + 1, 1 << 62):
        assert L.mm_debug_bounded_wait(None, ctypes.c_longlong(spins)) == mm.MM_EINVAL
        assert b"spins must be in [0, 4194304]" in L.mm_last_error(None)
