"""Parity of the device zip-up Krylov application (tdvp_set_krylov_method) with the oracle's
zip-up, and of a whole GSE-TDVP1 step built on it.  Gauge-invariant comparisons to 1e-10
(FP64).  The cutoffs here give the same bond dimensions under +-0.1 % changes, and the
oracle moves by under 2e-15 when its input is perturbed by 1e-12."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O
from paper_2005_06104_gb300 import workloads as wl


@pytest.fixture(scope="module")
def g():
    assert torch.cuda.is_available()
    from paper_2005_06104_gb300 import gse_tdvp
    return gse_tdvp


@pytest.mark.parametrize("tau,eps_k,cap", [(0.1, 1e-8, 64), (-0.25j, 1e-10, 64), (0.1, 1e-6, 12)])
def test_zipup_krylov_vector_matches_oracle(g, tau, eps_k, cap):
    lat = wl.zigzag_ladder(6, 1.0, 0.6)
    W = wl.heisenberg_mpo(lat)
    psi = O.left_canonicalize(wl.random_mps(lat.n, 6, 21))
    psi[-1] /= np.linalg.norm(psi[-1])
    st = g.GseTdvp(psi, W, tau=tau, eps_k=eps_k, chi_max=cap)
    st.krylov_method(g.KRYLOV_ZIPUP)
    st.apply_krylov()
    ref = O.krylov_vectors(psi, W, tau, 2, eps_k, cap, method="zipup")[0]
    mine = st.get_mps()
    assert st.bond_dims() == wl.mps_bond_dims(ref)
    assert abs(abs(O.mps_overlap(mine, ref)) - 1) < 1e-10
    assert abs(st.norm() - 1) < 1e-12
    for a in mine[:-1]:                                       # left-canonical, centre at N-1
        M = a.reshape(-1, a.shape[2])
        assert np.allclose(M.conj().T @ M, np.eye(M.shape[1]), atol=1e-12)
    st.close()


@pytest.mark.parametrize("kind", ["real", "imag"])
def test_zipup_gse_steps_match_oracle(g, kind):
    lat = wl.zigzag_ladder(5, 1.0, 1.0)
    W = wl.heisenberg_mpo(lat)
    if kind == "real":
        psi, tau, eps = wl.neel_state(lat, flip=(2, 0)), 0.1, 0.0
    else:
        psi, tau, eps = wl.random_product_state(lat.n, 1), -1j / wl.lambda_top(lat), 1e-10
    p = dict(tau=tau, k=3, eps_k=1e-8, eps_m=1e-8, chi_max=32, dt=0.1, kind=kind, eps=eps, krylov="zipup")
    st = g.GseTdvp(psi, W, tau=tau, eps_k=1e-8, eps_m=1e-8, eps=eps, chi_max=32)
    st.krylov_method(g.KRYLOV_ZIPUP)
    ref = psi
    for _ in range(3):
        st.step(0.1, g.REAL if kind == "real" else g.IMAG, 3)
        ref = O.gse_tdvp1_step(ref, W, p)
        assert st.bond_dims() == wl.mps_bond_dims(ref)
    assert abs(abs(O.mps_overlap(st.get_mps(), ref)) - 1) < 1e-10
    assert abs(st.energy() - O.mpo_expectation(ref, W).real) < 1e-10
    st.close()


def test_krylov_method_is_checked(g):
    lat = wl.chain(4)
    st = g.GseTdvp(wl.neel_state(lat), wl.heisenberg_mpo(lat))
    with pytest.raises(g.TDVPError) as e:
        st.krylov_method(7)
    assert e.value.status == 1
    st.close()
