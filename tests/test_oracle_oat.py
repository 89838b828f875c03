"""Pins of the exact OAT reference (Sec. II.B, Eqs. 12-15) and of the observable MPOs (CPU).

The Dicke-subspace solution is pinned to the closed form of Eq. 13, to <S^y> = <S^z> = 0, to
xi^2 = 1 for the initial coherent state, to exact diagonalisation of the full 2^N space at
N = 8, and to the optimal squeezing time the paper quotes (t_opt = 12^(1/6) (N/2)^(-2/3) / 2,
about 0.05 at N = 100).  The MPOs of total-spin sums and products equal the dense operators.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from oracle import oat_exact as X
from paper_2005_06104_gb300 import workloads as wl
from exact import mpo_to_dense, mps_to_dense, total_op


@pytest.mark.parametrize("n", [8, 40, 100])
def test_sx_closed_form_and_zero_moments(n):
    for t in (0.0, 0.01, 0.05, 0.13, 0.25):
        mom = X.oat_moments(n, t)
        assert abs(mom["x"] - 0.5 * n * np.cos(t) ** (n - 1)) < 1e-10 * n
        assert abs(mom["y"]) < 1e-10 * n and abs(mom["z"]) < 1e-10 * n
        # Casimir: <S^2> = S(S + 1) in the symmetric multiplet
        s2 = (mom["xx"] + mom["yy"] + mom["zz"]).real
        assert abs(s2 - 0.5 * n * (0.5 * n + 1)) < 1e-9 * n * n


def test_coherent_state_has_no_squeezing():
    for n in (8, 100):
        assert abs(X.squeezing_xi2(X.oat_moments(n, 0.0), n) - 1.0) < 1e-12


def test_dicke_solution_equals_full_ed():
    """N = 8: exp(-i t (S^z)^2) on the full 256-dimensional space, moments of total spins."""
    n = 8
    Sx, Sy, Sz = (total_op(op, n) for op in (wl.SX, wl.SY, wl.SZ))
    v0 = mps_to_dense(wl.x_polarized_state(n))
    for t in (0.07, 0.21, 0.6):
        v = sla.expm(-1j * t * (Sz @ Sz)) @ v0
        ops = {"x": Sx, "y": Sy, "z": Sz}
        mom = X.oat_moments(n, t)
        for a, A in ops.items():
            assert abs(np.vdot(v, A @ v) - mom[a]) < 1e-12
            for b, B in ops.items():
                assert abs(np.vdot(v, A @ (B @ v)) - mom[a + b]) < 1e-11


def test_optimal_squeezing_time_matches_the_quoted_scaling():
    n = 100
    ts = np.linspace(0.005, 0.25, 491)
    xi2 = [X.squeezing_xi2(X.oat_moments(n, t), n) for t in ts]
    t_min = ts[int(np.argmin(xi2))]
    t_opt = 12 ** (1 / 6) * (n / 2) ** (-2 / 3) / 2
    assert abs(t_opt - 0.05) < 0.01                   # the formula gives 0.0557, "about 0.05" (Sec. II.B)
    assert abs(t_min - 0.05) < 0.005                  # the exact optimum at N = 100
    assert abs(t_min - t_opt) < 0.25 * t_opt          # the large-N formula, to 25 % at N = 100
    assert min(xi2) < 0.2                             # strong squeezing at the optimum


def test_total_spin_mpos_equal_dense_operators():
    n = 6
    Sy, Sz = total_op(wl.SY, n), total_op(wl.SZ, n)
    My, Mz = wl.total_op_mpo(n, wl.SY), wl.total_op_mpo(n, wl.SZ)
    assert np.allclose(mpo_to_dense(My), Sy, atol=1e-14)
    assert np.allclose(mpo_to_dense(wl.mpo_product(My, Mz)), Sy @ Sz, atol=1e-13)
    assert np.allclose(mpo_to_dense(wl.mpo_product(Mz, My)), Sz @ Sy, atol=1e-13)   # order matters
    assert not np.allclose(Sy @ Sz, Sz @ Sy)
    # the oracle's MPO expectation of the product on a random state equals the dense one
    psi = wl.random_mps(n, 4, 9)
    v = mps_to_dense(psi)
    ref = np.vdot(v, Sy @ (Sz @ v)) / np.vdot(v, v)
    assert abs(O.mpo_expectation(psi, wl.mpo_product(My, Mz)) - ref) < 1e-12
