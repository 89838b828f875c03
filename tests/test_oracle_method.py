"""Pins of the oracle's algorithm-level routines (no GPU).

Krylov vectors (Sec. I.B, Eqs. 9-10), basis extension (Sec. I.A, Eqs. 3-7),
the TDVP1 sweep and whole GSE-TDVP1 steps (Sec. I.C) against exact
diagonalisation, closed forms (Sec. II.B, Eq. 13) and the properties the
paper states (Sec. I: unitarity in real time; a product state stays a product
state under plain TDVP1).
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from paper_2005_06104_gb300 import workloads as wl
from exact import (heisenberg_dense, mpo_to_dense, mps_to_dense, right_basis, site_op,
                   total_op, SZ, SX, SY, ground_energy_sz0)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _normalized(v):
    return v / np.linalg.norm(v)


@pytest.mark.parametrize("tau", [0.1, -1j / 4.0])
def test_krylov_vectors_exact_without_cutoff(tau):
    lat = wl.chain(8, 1.0, fields=np.linspace(-0.5, 0.7, 8))
    W = wl.heisenberg_mpo(lat)
    H = heisenberg_dense(lat.n, lat.bonds, lat.fields)
    psi = O.left_canonicalize(wl.random_mps(8, 3, 1))
    v = mps_to_dense(psi)
    phis = O.krylov_vectors(psi, W, tau, 4, 0.0, None)
    G = np.eye(2 ** 8) - 1j * tau * H
    ref = v
    for l, phi in enumerate(phis, start=1):
        ref = G @ ref
        u = mps_to_dense(phi)
        assert abs(np.linalg.norm(u) - 1) < 1e-13
        assert abs(abs(np.vdot(_normalized(ref), u)) - 1) < 1e-12
        assert np.allclose(u, _normalized(ref), atol=1e-11)        # same phase convention
        for a in phi[:-1]:                                          # left-canonical, centre at N
            M = a.reshape(-1, a.shape[2])
            assert np.allclose(M.conj().T @ M, np.eye(M.shape[1]), atol=1e-12)


def test_krylov_span_equals_power_span():
    """Eq. 10 spans the same space as Eq. 9 (statement at the end of Sec. I.B)."""
    lat = wl.chain(6)
    W = wl.heisenberg_mpo(lat)
    H = heisenberg_dense(6, lat.bonds)
    psi = O.left_canonicalize(wl.random_mps(6, 2, 3))
    v = mps_to_dense(psi)
    phis = O.krylov_vectors(psi, W, 0.2, 4, 0.0, None)
    K1 = np.stack([v] + [mps_to_dense(p) for p in phis], axis=1)
    K2 = np.stack([np.linalg.matrix_power(H, l) @ v for l in range(4)], axis=1)
    Q1, _ = np.linalg.qr(K1)
    Q2, _ = np.linalg.qr(K2)
    s = np.linalg.svd(Q1.conj().T @ Q2, compute_uv=False)
    assert np.allclose(s, 1.0, atol=1e-10)


def test_krylov_cutoff_controls_error():
    lat = wl.zigzag_ladder(5, 1.0, 1.0)
    W = wl.heisenberg_mpo(lat)
    H = heisenberg_dense(lat.n, lat.bonds)
    psi = O.left_canonicalize(wl.random_mps(lat.n, 4, 2))
    ref = _normalized((np.eye(2 ** lat.n) - 0.1j * H) @ mps_to_dense(psi))
    errs = []
    for eps in (1e-2, 1e-4, 1e-8):
        phi = O.krylov_vectors(psi, W, 0.1, 2, eps, None)[0]
        u = mps_to_dense(phi)
        errs.append(1 - abs(np.vdot(ref, u)) ** 2)
    assert errs[0] >= errs[1] >= errs[2] and errs[2] < 1e-7


def _extension_case(eps_m=0.0, chi_max=None, k=3, seed=4, n=8):
    lat = wl.zigzag_ladder(n // 2, 1.0, 1.0)
    W = wl.heisenberg_mpo(lat)
    psi = O.left_canonicalize(wl.random_mps(n, 2, seed))
    psi[-1] /= np.linalg.norm(psi[-1])
    phis = O.krylov_vectors(psi, W, 0.1, k, 0.0, None)
    out, added = O.basis_extension(psi, phis, None, eps_m, chi_max)
    return psi, phis, out, added


def test_extension_keeps_state_exactly():
    psi, phis, out, added = _extension_case()
    v0, v1 = mps_to_dense(psi), mps_to_dense(out)
    assert np.linalg.norm(v0 - v1) < 1e-13                      # Sec. I.A: psi retained exactly
    assert sum(added) > 0
    for a in out[1:]:                                            # B' right-orthonormal (Eq. 7)
        M = a.reshape(a.shape[0], -1)
        assert np.allclose(M @ M.conj().T, np.eye(M.shape[0]), atol=1e-12)
    # C_1 is not of full column rank once the bond is enlarged (text after Eq. 4)
    C1 = out[0].reshape(-1, out[0].shape[2])
    assert np.linalg.matrix_rank(C1, tol=1e-10) < C1.shape[1]


def test_extension_spans_krylov_vectors():
    """With eps_M = 0 and no cap, every psi~_l lies inside the enlarged right bases."""
    psi, phis, out, _ = _extension_case()
    n = len(out)
    for phi in phis:
        u = mps_to_dense(phi)
        for i in range(1, n):
            Phi = right_basis(out, i)                            # orthonormal columns
            M = u.reshape(2 ** i, -1)                            # (left, right)
            proj = (M @ Phi.conj()) @ Phi.T
            assert np.linalg.norm(M - proj) < 1e-10


@pytest.mark.parametrize("eps_m", [1e-3, 1e-5])
def test_extension_weights(eps_m):
    """Eq. 5's weights: rho~ = sum_l w_l C~_l^+ C~_l and eps_M is relative to tr rho~, so a
    common factor on the weights changes nothing, a zero weight removes that vector, and an
    unequal weighting changes the enlarged bases."""
    lat = wl.zigzag_ladder(4, 1.0, 1.0)
    W = wl.heisenberg_mpo(lat)
    psi = O.left_canonicalize(wl.random_mps(8, 2, 4))
    psi[-1] /= np.linalg.norm(psi[-1])
    phis = O.krylov_vectors(psi, W, 0.1, 3, 0.0, None)

    def projectors(out):
        return [right_basis(out, i) @ right_basis(out, i).conj().T for i in range(1, len(out))]

    base, n_base = O.basis_extension(psi, phis, None, eps_m, None)
    scaled, n_scaled = O.basis_extension(psi, phis, [4.0, 4.0], eps_m, None)
    assert n_scaled == n_base
    assert all(np.allclose(a, b, atol=1e-12) for a, b in zip(projectors(base), projectors(scaled)))
    zero, n_zero = O.basis_extension(psi, phis, [1.0, 0.0], eps_m, None)
    one, n_one = O.basis_extension(psi, phis[:1], None, eps_m, None)
    assert n_zero == n_one
    assert all(np.allclose(a, b, atol=1e-12) for a, b in zip(projectors(zero), projectors(one)))
    assert n_zero != n_base


def test_extension_bbar_orthogonal_to_b_and_svd_equivalence():
    """B_bar B^+ = 0 and eig(P rho~ P) = SVD of the direct sum of the P-projected C~_l (Eq. 6)."""
    lat = wl.chain(6)
    W = wl.heisenberg_mpo(lat)
    psi = O.left_canonicalize(wl.random_mps(6, 2, 8))
    phis = O.krylov_vectors(psi, W, 0.3, 3, 0.0, None)
    i = 5
    d, mr = 2, 1
    X = psi[i].reshape(psi[i].shape[0], d * mr)
    _, _, B, _ = O.svd_truncate(X)
    P = np.eye(d * mr) - B.conj().T @ B
    Xs = [p[i].reshape(p[i].shape[0], -1) for p in phis]
    rho = sum(x.conj().T @ x for x in Xs)
    ev = np.sort(np.linalg.eigvalsh(P @ rho @ P))[::-1]
    s = np.linalg.svd(np.concatenate([x @ P for x in Xs], axis=0), compute_uv=False)
    assert np.allclose(ev[: len(s)], s ** 2, atol=1e-13)
    out, added = O.basis_extension(psi, phis)
    Bp = out[i].reshape(out[i].shape[0], -1)
    r = B.shape[0]
    assert np.allclose(Bp[r:] @ Bp[:r].conj().T, 0, atol=1e-13)


def test_extension_caps_and_cutoff():
    _, _, out_full, added_full = _extension_case(0.0, None)
    _, _, out_cap, added_cap = _extension_case(0.0, 4)
    assert max(wl.mps_bond_dims(out_cap)) <= 4
    assert sum(added_cap) < sum(added_full)
    _, _, out_cut, added_cut = _extension_case(1e-3, None)
    assert sum(added_cut) <= sum(added_full)


def _ed_state(lat, psi):
    return mps_to_dense(psi)


def test_tdvp1_exact_at_full_bond_dimension():
    """With maximal bond dimensions the projector-splitting TDVP1 integrator is exact."""
    lat = wl.chain(8, 1.0, fields=np.linspace(-1, 1, 8))
    W = wl.heisenberg_mpo(lat)
    H = heisenberg_dense(lat.n, lat.bonds, lat.fields)
    psi = O.right_canonicalize(wl.random_mps(8, 16, 6))
    psi[0] /= np.linalg.norm(psi[0])
    v = mps_to_dense(psi)
    out = O.tdvp1_sweep(psi, W, 0.3, "real")
    ref = sla.expm(-0.3j * H) @ v
    assert np.linalg.norm(mps_to_dense(out) - ref) < 1e-9


def test_tdvp1_reversible_and_conserving():
    lat = wl.zigzag_ladder(4, 1.0, 1.0)
    W = wl.heisenberg_mpo(lat)
    psi = O.right_canonicalize(wl.random_mps(8, 3, 12))
    psi[0] /= np.linalg.norm(psi[0])
    e0 = O.mpo_expectation(psi, W).real
    fwd = O.tdvp1_sweep(psi, W, 0.2, "real")
    assert abs(O.mps_norm(fwd) - 1) < 1e-12
    assert abs(O.mpo_expectation(fwd, W).real - e0) < 1e-10        # energy conserved (Sec. II.B)
    back = O.tdvp1_sweep(fwd, W, -0.2, "real")
    assert abs(abs(O.mps_overlap(back, psi)) - 1) < 1e-10


def test_tdvp1_is_second_order_in_dt():
    """The symmetric splitting (dt/2 left to right, dt/2 right to left; reading R4) is of
    second order: against its own small-dt limit on a fixed-rank manifold the global error
    falls by 4 when dt halves (a first-order splitting would give 2)."""
    lat = wl.chain(8)
    W = wl.heisenberg_mpo(lat)
    psi0 = O.right_canonicalize(wl.random_mps(8, 3, 5))
    psi0[0] /= np.linalg.norm(psi0[0])
    T = 0.4

    def run(nsteps):
        psi = psi0
        for _ in range(nsteps):
            psi = O.tdvp1_sweep(psi, W, T / nsteps, "real")
        return mps_to_dense(psi)
    ref = run(128)
    errs = [np.linalg.norm(run(n) - ref) for n in (2, 4, 8)]
    for a, b in zip(errs, errs[1:]):
        assert 3.5 < a / b < 4.6


def test_tdvp1_product_state_stays_product():
    """Plain TDVP1 from a product state never grows the bond dimension (Introduction)."""
    lat = wl.zigzag_ladder(5, 1.0, 0.0)
    W = wl.heisenberg_mpo(lat)
    psi = wl.neel_state(lat)
    p = dict(tau=0.1, k=1, eps_k=1e-12, eps_m=1e-8, chi_max=32, dt=0.1, kind="imag", eps=1e-10)
    for _ in range(3):
        psi = O.gse_tdvp1_step(psi, W, p)
    assert max(wl.mps_bond_dims(psi)) == 1
    p["k"] = 3
    psi = O.gse_tdvp1_step(psi, W, p)
    assert max(wl.mps_bond_dims(psi)) > 1                           # the expansion fixes it


def test_gse_real_time_chain_vs_ed():
    """Heisenberg chain L=10 (Neel, dt=0.1, k=2, chi<=16, 10 steps) against ED."""
    p = wl.workload("heis_chain10")
    lat, W, psi = p["lattice"], p["mpo"], p["psi"]
    H = heisenberg_dense(lat.n, lat.bonds)
    v = mps_to_dense(psi)
    e0 = O.mpo_expectation(psi, W).real
    U = sla.expm(-1j * p["dt"] * H)
    Sz = [site_op(SZ, i, lat.n) for i in range(lat.n)]
    max_err = 0.0
    for _ in range(p["steps"]):
        psi = O.gse_tdvp1_step(psi, W, p)
        v = U @ v
        assert abs(O.mps_norm(psi) - 1) < 1e-12
        assert abs(O.mpo_expectation(psi, W).real - e0) < 1e-10    # unitarity preserved
        for i in range(lat.n):
            ex = np.real(np.vdot(v, Sz[i] @ v))
            max_err = max(max_err, abs(O.expect_local(psi, SZ, i).real - ex))
    assert max_err < 2e-3
    assert max(wl.mps_bond_dims(psi)) <= 16


def test_gse_chain_error_shrinks_with_bond_dimension_and_krylov_order():
    """Config 1 against ED: <S^z_i(t)> within 1e-4 at chi <= 16, k = 2, and the error falls
    towards 1e-8 with the full bond dimension (32) and a higher Krylov order (k = 4)."""
    lat = wl.chain(10)
    W = wl.heisenberg_mpo(lat)
    H = heisenberg_dense(lat.n, lat.bonds)
    U = sla.expm(-0.1j * H)
    Sz = [site_op(SZ, i, lat.n) for i in range(lat.n)]

    def run(chi, k, eps):
        psi = wl.neel_state(lat)
        v = mps_to_dense(psi)
        p = dict(tau=0.1, k=k, eps_k=eps, eps_m=eps, chi_max=chi, dt=0.1, kind="real", eps=0.0)
        err = 0.0
        for _ in range(10):
            psi = O.gse_tdvp1_step(psi, W, p)
            v = U @ v
            err = max(err, max(abs(O.expect_local(psi, SZ, i).real - np.real(np.vdot(v, Sz[i] @ v)))
                               for i in range(lat.n)))
        return err, 1 - abs(np.vdot(mps_to_dense(psi), v))

    coarse, _ = run(16, 2, 1e-8)
    fine, infid = run(32, 4, 1e-12)
    assert coarse < 1e-4
    assert fine < 1e-7 and fine < coarse / 50
    assert infid < 1e-10


def test_gse_dt_convergence_vs_ed():
    """Global error shrinks with the time step (second-order splitting)."""
    lat = wl.chain(8)
    W = wl.heisenberg_mpo(lat)
    H = heisenberg_dense(8, lat.bonds)
    psi0 = wl.neel_state(lat)
    v0 = mps_to_dense(psi0)
    T = 0.4
    errs = []
    for nsteps in (2, 4, 8):
        dt = T / nsteps
        p = dict(tau=dt, k=3, eps_k=1e-12, eps_m=1e-12, chi_max=64, dt=dt, kind="real", eps=0.0)
        psi = psi0
        for _ in range(nsteps):
            psi = O.gse_tdvp1_step(psi, W, p)
        ref = sla.expm(-1j * T * H) @ v0
        errs.append(np.linalg.norm(mps_to_dense(psi) - ref))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 2e-3


def test_gse_imaginary_time_decoupled_ladder_reaches_twice_chain_energy():
    """Rung-decoupled ladder (Sec. II.A): E -> 2 x single-chain ground energy."""
    lx = 6
    lat = wl.zigzag_ladder(lx, 1.0, 0.0)
    W = wl.heisenberg_mpo(lat)
    e_exact = 2 * ground_energy_sz0(lx, [(i, i + 1, 1.0) for i in range(lx - 1)])
    psi = wl.neel_state(lat)
    lam = wl.lambda_top(lat)
    p = dict(tau=-1j / lam, k=3, eps_k=1e-12, eps_m=1e-8, chi_max=64, dt=0.4, kind="imag",
             eps=1e-10)
    es = []
    for _ in range(40):
        psi = O.gse_tdvp1_step(psi, W, p)
        es.append(O.mpo_expectation(psi, W).real)
    assert all(b <= a + 1e-9 for a, b in zip(es, es[1:]))            # monotone decrease
    assert abs(es[-1] - e_exact) / abs(e_exact) < 2e-7


def test_oat_sx_closed_form():
    """OAT model (Sec. II.B): <S^x(t)> = (N/2) cos^(N-1)(t), <S^y> = <S^z> = 0 (Eq. 13)."""
    g = json.load(open(os.path.join(GOLDEN, "oat_closed_form.json")))
    n = g["n_sites"]
    W = wl.oat_mpo(n)
    psi = wl.x_polarized_state(n)
    p = dict(tau=g["dt"], k=g["k"], eps_k=g["eps_k"], eps_m=g["eps_m"], chi_max=64, dt=g["dt"],
             kind="real", eps=0.0)
    e0 = O.mpo_expectation(psi, W).real
    for step in range(1, g["steps"] + 1):
        psi = O.gse_tdvp1_step(psi, W, p)
        t = step * g["dt"]
        sx = sum(O.expect_local(psi, wl.SX, i).real for i in range(n))
        sy = sum(O.expect_local(psi, wl.SY, i).real for i in range(n))
        sz = sum(O.expect_local(psi, wl.SZ, i).real for i in range(n))
        assert abs(sx - g["sx"][step - 1]) < g["tol_sx"]
        assert abs(sx - 0.5 * n * np.cos(t) ** (n - 1)) < g["tol_sx"]
        assert abs(sy) < 1e-8 and abs(sz) < 1e-8
        assert abs(O.mpo_expectation(psi, W).real - e0) < 1e-10 * max(1.0, abs(e0))
