"""One-axis twisting (Sec. II.B): a long-range MPO (w = 3, every pair coupled) from the +x
product state.  The GPU run follows the closed form <S^x(t)> = (N/2) cos^(N-1)(t) of Eq. 13
(the values of tests/golden/oat_closed_form.json) and the oracle's own trajectory."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O
from paper_2005_06104_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "oat_closed_form.json")


@pytest.fixture(scope="module")
def g():
    assert torch.cuda.is_available()
    from paper_2005_06104_gb300 import gse_tdvp
    return gse_tdvp


@pytest.mark.parametrize("prec", ["fp64", "bf16x10"])
def test_oat_sx_follows_closed_form(g, prec):
    gd = json.load(open(GOLDEN))
    n, dt = gd["n_sites"], gd["dt"]
    W = wl.oat_mpo(n)
    st = g.GseTdvp(wl.x_polarized_state(n), W, tau=dt, eps_k=gd["eps_k"], eps_m=gd["eps_m"], chi_max=64,
                   precision=g.PREC_FP64 if prec == "fp64" else g.PREC_BF16X10)
    e0 = st.energy()
    # <S^y> and <S^z> vanish by symmetry.  The precision form is held to a 1e-7 relative error
    # per step, taken here against the spin length N/2 and accumulated over the steps; FP64 to
    # 1e-7 absolute.
    for step in range(1, gd["steps"] + 1):
        tol_sym = 1e-7 if prec == "fp64" else 1e-7 * 0.5 * n * step
        st.step(dt, g.REAL, gd["k"])
        t = step * dt
        sx = sum(st.expect_local(wl.SX, i).real for i in range(n))
        sy = sum(st.expect_local(wl.SY, i).real for i in range(n))
        sz = sum(st.expect_local(wl.SZ, i).real for i in range(n))
        assert abs(sx - gd["sx"][step - 1]) < gd["tol_sx"]
        assert abs(sx - 0.5 * n * np.cos(t) ** (n - 1)) < gd["tol_sx"]
        assert abs(sy) < tol_sym and abs(sz) < tol_sym
        assert abs(st.energy() - e0) < 1e-7 * max(1.0, abs(e0))
    st.close()


def test_oat_matches_oracle_trajectory(g):
    """N = 24, dt = 0.05, k = 5 (the paper's second OAT setting): GPU and oracle states agree."""
    n, dt, k = 24, 0.05, 5
    W = wl.oat_mpo(n)
    psi = wl.x_polarized_state(n)
    p = dict(tau=dt, k=k, eps_k=1e-4, eps_m=1e-4, chi_max=64, dt=dt, kind="real", eps=0.0)
    st = g.GseTdvp(psi, W, tau=dt, eps_k=1e-4, eps_m=1e-4, chi_max=64)
    ref = psi
    for _ in range(4):
        st.step(dt, g.REAL, k)
        ref = O.gse_tdvp1_step(ref, W, p)
    assert st.bond_dims() == wl.mps_bond_dims(ref)
    assert abs(abs(O.mps_overlap(st.get_mps(), ref)) - 1) < 1e-9
    st.close()
