"""The C-ABI library builds, loads and exports every entry point the header declares (no GPU)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_2005_06104_gb300", "libgsetdvp.so")
HEADER = os.path.join(ROOT, "include", "gse_tdvp.h")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_2005_06104_gb300 import build
        build.build()
    return C.CDLL(LIB)


def declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"TDVP_API\s+[\w\s\*]+?\b(tdvp_\w+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = declared()
    for must in ("tdvp_create", "tdvp_destroy", "tdvp_expand_basis", "tdvp_sweep", "tdvp_heff_apply",
                 "tdvp_energy", "tdvp_norm", "tdvp_expect_local", "tdvp_get_mps", "tdvp_heff_contract"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_side_argument_checks(lib):
    lib.tdvp_status_string.restype = C.c_char_p
    assert lib.tdvp_status_string(0) == b"ok"
    assert lib.tdvp_status_string(4) == b"Lanczos not converged"
    # null arguments are rejected before any device work
    assert lib.tdvp_create(None, None, None, None, None) == 1
    assert lib.tdvp_default_options(None) == 1
    assert lib.tdvp_destroy(None) == 1


def test_default_options_struct(lib):
    from paper_2005_06104_gb300 import gse_tdvp as g
    o = g.default_options(tau=-0.25j, chi_max=77)
    assert o.chi_max == 77 and o.tau_im == -0.25 and o.tau_re == 0.0
    assert o.lanczos_tol == 1e-12 and o.lanczos_max == 40 and o.precision == g.PREC_FP64
    assert g.declared_symbols() == declared()


def test_launch_counter_reads_without_a_gpu(lib):
    from paper_2005_06104_gb300 import gse_tdvp as g
    assert lib.tdvp_launch_count(None) == 1
    assert lib.tdvp_gemm_chunk_stats(None) == 1
    n0 = g.launch_count()
    assert isinstance(n0, int) and n0 >= 0
    assert g.launch_count() == n0  # nothing launched in between


def test_binding_constants_match_the_header():
    """The binding's enum values are the header's (time kind, precision form, Krylov method,
    status codes)."""
    from paper_2005_06104_gb300 import gse_tdvp as g
    txt = open(HEADER).read()
    enum = {k: int(v) for k, v in re.findall(r"\b(TDVP_[A-Z0-9_]+)\s*=\s*(\d+)", txt)}
    assert (g.REAL, g.IMAG) == (enum["TDVP_REAL"], enum["TDVP_IMAG"])
    for name in ("FP64", "TF32X3", "TF32X3_ENV", "BF16X10", "BF16X6"):
        assert getattr(g, "PREC_" + name) == enum["TDVP_PREC_" + name]
    assert g.KRYLOV_DENSITY_MATRIX == enum["TDVP_KRYLOV_DENSITY_MATRIX"]
    assert g.KRYLOV_ZIPUP == enum["TDVP_KRYLOV_ZIPUP"]
    codes = sorted(v for k, v in enum.items() if k == "TDVP_OK" or k.startswith("TDVP_ERR_"))
    assert codes == sorted(g.STATUS)


def test_contract_wrappers_check_operands_before_the_call():
    """The H_eff wrappers refuse operands that do not fit (shapes, dtype, placement) before any
    pointer reaches the library (a wrong W or x shape would make the C loops read past them)."""
    import numpy as np
    import torch
    from paper_2005_06104_gb300 import gse_tdvp as g
    from paper_2005_06104_gb300 import workloads as wl
    W = wl.heisenberg_mpo(wl.zigzag_ladder(4, 1.0, 1.0))[3]
    wl_, d, _, wr = W.shape
    L = torch.zeros((5, wl_, 5), dtype=torch.complex128)
    R = torch.zeros((6, wr, 6), dtype=torch.complex128)
    x = torch.zeros((5, d, 6), dtype=torch.complex128)
    y = torch.zeros_like(x)
    for fn in (g.heff_contract, g.heff_contract_noalloc):
        with pytest.raises(ValueError, match="CUDA"):
            fn(L, W, R, x, y)                          # host tensors
        with pytest.raises(ValueError, match="do not fit"):
            fn(L, np.zeros((wl_ + 1, d, d, wr), complex), R, x, y)
        with pytest.raises(ValueError, match="expected"):
            fn(L, W, R, torch.zeros((5, d, 7), dtype=torch.complex128), y)


def test_binding_refuses_bad_local_vectors_before_the_library():
    """The handle methods that take caller device vectors check placement, dtype, layout and
    the local-space size before any pointer reaches the library (a host tensor, a wrong dtype
    or a wrong size is refused here)."""
    torch = pytest.importorskip("torch")
    from paper_2005_06104_gb300 import gse_tdvp as g
    h = g.GseTdvp.__new__(g.GseTdvp)
    h.n, h.d = 3, 2
    h.bond_dims = lambda: [1, 2, 3, 1]
    assert h._site_size(0) == 4 and h._site_size(1) == 12 and h._site_size(2) == 6
    assert h._site_size(3) is None and h._site_size(-1) is None
    with pytest.raises(ValueError, match="CUDA complex128"):
        h.heff_apply(1, torch.zeros(12, dtype=torch.complex128), torch.zeros(12, dtype=torch.complex128))
    with pytest.raises(ValueError, match="CUDA complex128"):
        h.keff_apply(1, torch.zeros(4, dtype=torch.float64), torch.zeros(4, dtype=torch.float64))
    with pytest.raises(ValueError, match="CUDA complex128"):
        h.evolve_site(0, torch.zeros(4, dtype=torch.complex64), torch.zeros(4, dtype=torch.complex64), 0.1)
