"""GB300-native GSE-TDVP1 (global-subspace-expanded one-site TDVP, arXiv:2005.06104).

The compute path lives in the CUDA library `libgsetdvp.so` (sources in
`csrc/`, C-ABI in `include/gse_tdvp.h`); `gse_tdvp` is its Python binding and
`workloads` builds seeded synthetic inputs.  Importing the package loads
nothing; importing `gse_tdvp` loads the library and fails if it is missing.
"""
