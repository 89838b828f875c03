"""CPU FP64 oracle for GSE-TDVP1 (Yang & White, arXiv:2005.06104), with the two-site TDVP
it is compared with (tdvp2.py) and the zip-up MPO application (apply_mpo_zipup).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
baseline leg of the benchmark may import this package; the product path (the
CUDA library and its binding) never does, and shares no code with it.
"""
from .gse_tdvp1 import *  # noqa: F401,F403
from .tdvp2 import heff2_apply, tdvp2_sweep  # noqa: F401
