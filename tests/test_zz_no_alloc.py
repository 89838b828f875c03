"""The allocation-free H_eff entry point (tdvp_heff_contract_noalloc).

Some callers cannot call cudaMalloc: a host framework that owns every device
allocation, or a loop that must never block on the allocator.  This entry point
keeps its intermediates in a fixed device array instead.  The test checks it
through the C ABI against the ordinary entry point (tdvp_heff_contract, FP64)
on two calls in a row with different shapes, within the FP64 tolerance the other
contraction tests use, and that sizes beyond the fixed array are refused.
This file is collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2005_06104_gb300 import workloads as wl

TOL64 = 1e-12


def _rand(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(shape[-1])


def _dev(*arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


def test_noalloc_heff_matches_allocating_entry():
    assert torch.cuda.is_available()
    from paper_2005_06104_gb300 import gse_tdvp as g
    W_cyl = wl.heisenberg_mpo(wl.cylinder_snake(6, 4))
    W_lad = wl.heisenberg_mpo(wl.zigzag_ladder(6, 1.0, 1.0))
    for call, (ml, mr, W) in enumerate([(96, 130, W_cyl[10]), (37, 45, W_lad[5])]):
        rng = np.random.default_rng(100 + call)
        L = _rand(rng, ml, W.shape[0], ml)
        R = _rand(rng, mr, W.shape[3], mr)
        x = _rand(rng, ml, W.shape[1], mr)
        Ld, Rd, xd = _dev(L, R, x)
        y_ref = torch.empty_like(xd)
        y_na = torch.full_like(xd, float("nan"))
        g.heff_contract(Ld, W, Rd, xd, y_ref, precision=g.PREC_FP64)
        g.heff_contract_noalloc(Ld, W, Rd, xd, y_na)
        err = (torch.linalg.norm(y_na - y_ref) / torch.linalg.norm(y_ref)).item()
        assert err < TOL64, (call, err)


def test_noalloc_rejects_oversize():
    from paper_2005_06104_gb300 import gse_tdvp as g
    W = wl.heisenberg_mpo(wl.cylinder_snake(6, 4))[10]
    m = 512  # (m w d m) * 2 * 16 bytes > 31 MiB
    L = torch.zeros((m, W.shape[0], m), dtype=torch.complex128, device="cuda")
    R = torch.zeros((m, W.shape[3], m), dtype=torch.complex128, device="cuda")
    x = torch.zeros((m, 2, m), dtype=torch.complex128, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(g.TDVPError) as e:
        g.heff_contract_noalloc(L, W, R, x, y)
    assert e.value.status == 1 and "31 MiB" in str(e.value)
