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
    # <S^y> and <S^z> vanish by symmetry.  FP64 holds them to 1e-7 absolute.  The precision
    # form breaks the symmetry by its contraction error, about 1.4e-7 of the spin length N/2
    # per step when the gauge moves keep every direction of numerical rank (R1); it is held to
    # 2e-7 of N/2 per step, accumulated over the steps.
    for step in range(1, gd["steps"] + 1):
        tol_sym = 1e-7 if prec == "fp64" else 2e-7 * 0.5 * n * step
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


def _squeezing(st, n, ops):
    """<S^x> and xi^2 (Eq. 15) of a device state from MPO expectations of total-spin products."""
    from oracle import oat_exact as X
    mom = {k: st.expect_mpo(v) for k, v in ops.items()}
    return mom["x"].real, X.squeezing_xi2(mom, n)


def _spin_ops(n):
    Mx, My, Mz = (wl.total_op_mpo(n, op) for op in (wl.SX, wl.SY, wl.SZ))
    return {"x": Mx, "yy": wl.mpo_product(My, My), "zz": wl.mpo_product(Mz, Mz),
            "yz": wl.mpo_product(My, Mz), "zy": wl.mpo_product(Mz, My)}


def test_expect_mpo_matches_oracle(g):
    n = 10
    psi = wl.random_mps(n, 8, 31)
    st = g.GseTdvp(psi, wl.heisenberg_mpo(wl.chain(n)))
    for W in list(_spin_ops(n).values()) + [wl.oat_mpo(n), wl.heisenberg_mpo(wl.chain(n))]:
        assert abs(st.expect_mpo(W) - O.mpo_expectation(psi, W)) < 1e-12 * max(1.0, abs(O.mpo_expectation(psi, W)))
    with pytest.raises(g.TDVPError):
        st.expect_mpo(wl.oat_mpo(n + 1))
    st.close()


@pytest.mark.parametrize("dt,k,eps_m,steps", [(0.025, 3, 1e-4, 4), (0.05, 5, 1e-8, 2)])
def test_oat_n100_paper_settings(g, dt, k, eps_m, steps):
    """N = 100 (Sec. II.B) in the paper's two settings (tau = dt, eps_K = 1e-4, eps = 0), capped
    at chi 64, to t = 0.1: the device follows the oracle (which sub-steps its local
    exponentials, R13: the spectral range is about N^2 / 4) in <S^x>, xi^2 and the energy, holds
    the energy to 1e-10 relative (the paper's bound for GSE-TDVP1), and stays within 1 % of the
    spin length of Eq. 13 and within a factor 1.6 of the exact xi^2 (Dicke subspace).

    With k = 5 and eps_M = 1e-8 the extension's cut on this permutation-symmetric state meets
    near-degenerate eigenvalues of Eq. 6, whose kept directions are fixed only to rounding over
    their gap: two correct implementations then enlarge the basis by different directions of
    equal count, and the steps that follow differ by about 6e-7 relative in <S^x> (a GPU sweep
    and an oracle sweep from one and the same enlarged state agree to 1e-15).  That setting is
    held to 1e-5 relative against the oracle; the other to 1e-8."""
    from oracle import oat_exact as X
    n = 100
    W = wl.oat_mpo(n)
    psi = wl.x_polarized_state(n)
    ops = _spin_ops(n)
    p = dict(tau=dt, k=k, eps_k=1e-4, eps_m=eps_m, chi_max=64, dt=dt, kind="real", eps=0.0)
    st = g.GseTdvp(psi, W, tau=dt, eps_k=1e-4, eps_m=eps_m, chi_max=64)
    e0 = st.energy()
    ref = psi
    for step in range(1, steps + 1):
        st.step(dt, g.REAL, k)
        ref = O.gse_tdvp1_step(ref, W, p)
        sx, xi2 = _squeezing(st, n, ops)
        mom_ref = {kk: O.mpo_expectation(ref, v) for kk, v in ops.items()}
        rel = 1e-8 if k == 3 else 1e-5
        assert st.bond_dims() == wl.mps_bond_dims(ref)
        assert abs(sx - mom_ref["x"].real) < rel * n
        assert abs(xi2 - X.squeezing_xi2(mom_ref, n)) < 10 * rel * xi2
        assert abs(st.energy() - e0) < 1e-10 * abs(e0)
        ex = X.oat_moments(n, step * dt)
        assert abs(sx - ex["x"].real) < 0.01 * 0.5 * n
        xi_ex = X.squeezing_xi2(ex, n)
        assert xi_ex / 1.6 < xi2 < 1.6 * xi_ex
    st.close()


def test_oat_n100_sweep_parity_from_one_enlarged_state(g):
    """The k = 5 setting of Sec. II.B at N = 100: the device's TDVP1 sweep and the oracle's, both
    from the state the device's extension produced, agree in <S^x> to 1e-9 relative (the
    sweep itself, QR gauge moves with the rank fallback and sub-stepped exponentials included,
    has no sensitivity of its own)."""
    n = 100
    W = wl.oat_mpo(n)
    Mx = wl.total_op_mpo(n, wl.SX)
    st = g.GseTdvp(wl.x_polarized_state(n), W, tau=0.05, eps_k=1e-4, eps_m=1e-8, chi_max=64)
    st.expand_basis(5)
    enlarged = st.get_mps()
    st.sweep(0.05, g.REAL)
    ref = O.tdvp1_sweep(enlarged, W, 0.05, "real", 0.0, 64)
    assert st.bond_dims() == wl.mps_bond_dims(ref)
    assert abs(st.expect_mpo(Mx).real - O.mpo_expectation(ref, Mx).real) < 1e-9 * 0.5 * n
    assert abs(abs(O.mps_overlap(st.get_mps(), ref)) - 1) < 1e-10
    st.close()
