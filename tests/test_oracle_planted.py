"""Planted mistakes in the oracle (on the CPU): each plausible slip, put into one routine,
fails at least one of the pins that hold the oracle to exact diagonalisation and to the
paper's statements.  This checks that the pins can see the mistakes they are there to catch.

  * the Krylov operator of Eq. 10 built with the wrong sign of tau;
  * the backward bond step of the TDVP1 sweep (Sec. I.C step 3) with the wrong sign;
  * the full time step on each half-sweep instead of half of it (reading R4);
  * the weights of Eq. 5 ignored in the state-averaged density matrix;
  * the last Krylov vector left out of Eq. 5's sum;
  * the Lanczos stopping tolerance (R11) not honoured.
"""
import pytest

import oracle
import oracle.gse_tdvp1 as G
import test_oracle_method as M


def _fails(pin, *args):
    with pytest.raises(AssertionError):
        pin(*args)


def test_pins_pass_unplanted():
    M.test_krylov_vectors_exact_without_cutoff(0.1)
    M.test_tdvp1_exact_at_full_bond_dimension()
    M.test_extension_weights(1e-3)


def test_wrong_sign_of_tau_in_the_krylov_operator(monkeypatch):
    orig = G.mpo_one_minus_itau_h
    monkeypatch.setattr(G, "mpo_one_minus_itau_h", lambda W, tau: orig(W, -tau))
    _fails(M.test_krylov_vectors_exact_without_cutoff, 0.1)


def test_wrong_sign_of_the_backward_bond_step(monkeypatch):
    orig = G.keff_apply
    monkeypatch.setattr(G, "keff_apply", lambda L, R, C: -orig(L, R, C))
    _fails(M.test_tdvp1_exact_at_full_bond_dimension)


def test_full_time_step_on_each_half_sweep(monkeypatch):
    orig = G.tdvp1_sweep
    monkeypatch.setattr(oracle, "tdvp1_sweep", lambda psi, W, dt, kind, *a, **k: orig(psi, W, 2 * dt, kind, *a, **k))
    _fails(M.test_tdvp1_exact_at_full_bond_dimension)


def test_weights_of_eq5_ignored(monkeypatch):
    orig = G.basis_extension
    monkeypatch.setattr(oracle, "basis_extension",
                        lambda psi, phis, weights=None, *a, **k: orig(psi, phis, None, *a, **k))
    _fails(M.test_extension_weights, 1e-3)


def test_last_krylov_vector_left_out_of_the_extension(monkeypatch):
    """An off-by-one over l = 1..k-1 in Eq. 5 (the last vector dropped from rho~)."""
    orig = G.basis_extension
    monkeypatch.setattr(oracle, "basis_extension", lambda psi, phis, *a, **k: orig(psi, phis[:-1], *a, **k))
    _fails(M.test_extension_spans_krylov_vectors)


def test_lanczos_stopping_tolerance_not_honoured(monkeypatch):
    import test_oracle_pins as P
    orig = G.lanczos_expm
    monkeypatch.setattr(oracle, "lanczos_expm",
                        lambda f, x, delta, kind, tol=1e-12, nmax=40: orig(f, x, delta, kind, 1e-5, nmax))
    _fails(P.test_lanczos_matches_expm, "real")
