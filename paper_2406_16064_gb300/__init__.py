"""GB300-native finite-difference LLG solver core (libmm) -- Python side.

`paper_2406_16064_gb300.mm` is the ctypes binding of the C ABI declared in
include/mm.h; `paper_2406_16064_gb300.build` compiles the CUDA library
in-tree for sm_103a.  The arithmetic lives in csrc/*.cu only.
"""
from . import mm  # noqa: F401
