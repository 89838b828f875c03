"""Pins of the CPU oracle against exact results (no GPU).

Each test ties one oracle routine to something other than itself: Kronecker
product Hamiltonians, dense projected Hamiltonians, scipy's expm, exact
diagonalisation, and the identities the paper states (Sec. I.A: the state is
unchanged by the basis extension and B_bar B^+ = 0; Sec. I.B: the vectors of
Eq. 10 span the Krylov space of Eq. 9).
"""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from paper_2005_06104_gb300 import workloads as wl
from exact import (heisenberg_dense, mpo_to_dense, mps_to_dense, left_basis, right_basis,
                   site_op, total_op, SZ, SX, SY, ground_energy_sz0)


def _lat_cases():
    rng = np.random.default_rng(5)
    return [
        wl.chain(7, 1.0, fields=rng.uniform(-2, 2, 7)),
        wl.zigzag_ladder(4, 1.0, 0.0),
        wl.zigzag_ladder(4, 0.7, 1.3),
        wl.cylinder_snake(2, 4),
        wl.cylinder_snake(3, 3),
    ]


@pytest.mark.parametrize("lat", _lat_cases(), ids=lambda l: l.name)
def test_mpo_equals_kron_hamiltonian(lat):
    H = heisenberg_dense(lat.n, lat.bonds, lat.fields)
    W = wl.heisenberg_mpo(lat)
    assert np.allclose(mpo_to_dense(W), H, atol=1e-13)


def test_mpo_widths_match_channel_count():
    # w = 2 + 3 * (open sites at the cut): chain 5, zigzag ladder 8, 4-wide snake cylinder <= 14
    assert max(wl.mpo_bond_dims(wl.heisenberg_mpo(wl.chain(10)))) == 5
    assert max(wl.mpo_bond_dims(wl.heisenberg_mpo(wl.zigzag_ladder(20, 1, 0)))) == 8
    assert max(wl.mpo_bond_dims(wl.heisenberg_mpo(wl.zigzag_ladder(50, 1, 1)))) == 8
    dims = wl.mpo_bond_dims(wl.heisenberg_mpo(wl.cylinder_snake(16, 4)))
    assert max(dims) == 14 and set(dims[1:-1]) <= {5, 8, 11, 14}


def test_oat_mpo_is_total_sz_squared():
    n = 6
    Sz = total_op(SZ, n)
    assert np.allclose(mpo_to_dense(wl.oat_mpo(n)), Sz @ Sz, atol=1e-13)
    assert max(wl.mpo_bond_dims(wl.oat_mpo(n))) == 3


def test_ferromagnetic_top_of_spectrum():
    lat = wl.zigzag_ladder(4, 1.0, 1.0)
    ev = np.linalg.eigvalsh(heisenberg_dense(lat.n, lat.bonds))
    assert abs(ev[-1] - wl.lambda_top(lat)) < 1e-12


@pytest.mark.parametrize("tau", [0.1, -1j / 9.5, 0.03 - 0.02j])
def test_one_minus_itau_h_mpo(tau):
    lat = wl.zigzag_ladder(3, 1.0, 0.5)
    W = wl.heisenberg_mpo(lat)
    H = heisenberg_dense(lat.n, lat.bonds)
    Wk = O.mpo_one_minus_itau_h(W, tau)
    assert [w.shape for w in Wk] == [w.shape for w in W]     # same bond dimension (Sec. I.C)
    assert np.allclose(mpo_to_dense(Wk), np.eye(2 ** lat.n) - 1j * tau * H, atol=1e-13)


def _mixed_state(n, chi, seed, center):
    psi = wl.random_mps(n, chi, seed)
    psi = O.right_canonicalize(psi)
    for i in range(center):                      # move the centre right with SVDs
        ml, d, mr = psi[i].shape
        U, S, Vh, _ = O.svd_truncate(psi[i].reshape(ml * d, mr))
        psi[i] = U.reshape(ml, d, -1)
        psi[i + 1] = np.tensordot(S[:, None] * Vh, psi[i + 1], axes=([1], [0]))
    return psi


@pytest.mark.parametrize("center", [0, 2, 4, 6])
def test_heff_is_projected_hamiltonian(center):
    lat = wl.zigzag_ladder(4, 1.0, 0.8)
    n = lat.n
    W = wl.heisenberg_mpo(lat)
    H = heisenberg_dense(n, lat.bonds)
    psi = _mixed_state(n, 6, 11 + center, center)
    Ls, Rs = O.build_envs(psi, W, center)
    A = psi[center]
    ml, d, mr = A.shape
    PhiL, PhiR = left_basis(psi, center), right_basis(psi, center + 1)
    V = np.kron(np.kron(PhiL, np.eye(2)), PhiR)              # (2^n, ml*d*mr)
    Hproj = V.conj().T @ H @ V
    rng = np.random.default_rng(3)
    x = rng.standard_normal(A.shape) + 1j * rng.standard_normal(A.shape)
    y = O.heff_apply(Ls[center], W[center], Rs[center], x)
    assert np.allclose(y.reshape(-1), Hproj @ x.reshape(-1), atol=1e-12)
    # energy at the centre equals the dense expectation value
    v = mps_to_dense(psi)
    e = np.real(np.vdot(v, H @ v) / np.vdot(v, v))
    assert abs(O.energy_at_center(psi, W, center) - e) < 1e-12
    assert abs(O.mpo_expectation(psi, W) - e) < 1e-12


@pytest.mark.parametrize("bond", [1, 3, 6])
def test_keff_is_projected_hamiltonian(bond):
    lat = wl.chain(8, 1.0, fields=np.linspace(-1, 1, 8))
    n = lat.n
    W = wl.heisenberg_mpo(lat)
    H = heisenberg_dense(n, lat.bonds, lat.fields)
    psi = _mixed_state(n, 5, 21 + bond, bond)
    # bond between site bond-1 (left-canonical) and site bond (centre)
    Ls, Rs = O.build_envs(psi, W, bond)
    PhiL = left_basis(psi, bond)
    # right block including the centre site: fold the centre into R
    R_incl = O.env_right_step(Rs[bond], psi[bond], W[bond])
    PhiR_incl = right_basis(psi, bond)
    V = np.kron(PhiL, PhiR_incl)
    Hproj = V.conj().T @ H @ V
    rng = np.random.default_rng(4)
    m1, m2 = PhiL.shape[1], PhiR_incl.shape[1]
    C = rng.standard_normal((m1, m2)) + 1j * rng.standard_normal((m1, m2))
    y = O.keff_apply(Ls[bond], R_incl, C)
    assert np.allclose(y.reshape(-1), Hproj @ C.reshape(-1), atol=1e-12)


def test_environments_match_dense_gram():
    """L of the identity MPO = Gram matrix of the left block basis (plain definition)."""
    n = 6
    psi = wl.random_mps(n, 4, 9)
    Wid = [np.eye(2, dtype=complex).reshape(1, 2, 2, 1) for _ in range(n)]
    L = np.ones((1, 1, 1), complex)
    for i in range(3):
        L = O.env_left_step(L, psi[i], Wid[i])
    Phi = left_basis(psi, 3)
    assert np.allclose(L[:, 0, :], Phi.conj().T @ Phi, atol=1e-13)
    R = np.ones((1, 1, 1), complex)
    for i in range(n - 1, 2, -1):
        R = O.env_right_step(R, psi[i], Wid[i])
    Phi = right_basis(psi, 3)
    assert np.allclose(R[:, 0, :], Phi.conj().T @ Phi, atol=1e-13)


@pytest.mark.parametrize("kind", ["real", "imag"])
def test_lanczos_matches_expm(kind):
    rng = np.random.default_rng(7)
    n = 60
    M = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    H = 0.5 * (M + M.conj().T) / np.sqrt(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    delta = 0.37
    ref = sla.expm((-1j if kind == "real" else -1) * delta * H) @ x
    y, it = O.lanczos_expm(lambda v: H @ v, x, delta, kind, tol=1e-12, nmax=40)
    assert np.linalg.norm(y - ref) <= 1e-10 * np.linalg.norm(ref)
    assert it < 40
    if kind == "real":
        assert abs(np.linalg.norm(y) - np.linalg.norm(x)) < 1e-12 * np.linalg.norm(x)


def test_lanczos_small_space_and_nonconvergence():
    H = np.diag([1.0, -2.0, 0.5]).astype(complex)
    x = np.array([1.0, 1.0, 1.0], complex)
    y, it = O.lanczos_expm(lambda v: H @ v, x, 0.3, "real")
    assert np.allclose(y, np.exp(-0.3j * np.diag(H)) * x, atol=1e-13) and it <= 3
    rng = np.random.default_rng(1)
    M = rng.standard_normal((200, 200))
    H = (M + M.T) * 5
    with pytest.raises(O.LanczosNotConverged):
        O.lanczos_expm(lambda v: H @ v, rng.standard_normal(200) + 0j, 1.0, "real", 1e-12, 3)


def test_keep_count_rule():
    w = np.array([4.0, 2.0, 1.0, 0.5, 0.25])
    tot = w.sum()
    assert O.keep_count(w, tot, 0.0, 10, 0.0) == 5
    assert O.keep_count(w, tot, 0.25 / tot, 10, 0.0) == 4          # drop exactly the tail 0.25
    assert O.keep_count(w, tot, 0.8 / tot, 10, 0.0) == 3          # tail 0.75 fits
    assert O.keep_count(w, tot, 0.0, 2, 0.0) == 2
    assert O.keep_count(w, tot, 0.0, 10, 0.6) == 3                  # floor
    wc = np.array([3.0, 1.0, 1.0, 1.0, 0.1])                        # a 3-fold cluster
    assert O.keep_count(wc, wc.sum(), 1.05 / wc.sum(), 10, 0.0) == 4  # cut inside -> keep whole
    assert O.keep_count(wc, wc.sum(), 0.0, 3, 0.0) == 1             # cap inside -> drop whole
    assert O.keep_count(np.zeros(3), 0.0, 0.0, 3, 0.0) == 0


def test_gauge_moves_keep_state():
    psi = wl.random_mps(7, 8, 2)
    v = mps_to_dense(psi)
    for f in (O.left_canonicalize, O.right_canonicalize):
        out = f(psi)
        assert np.allclose(mps_to_dense(out), v, atol=1e-13)
    lc = O.left_canonicalize(psi)
    for a in lc[:-1]:
        M = a.reshape(-1, a.shape[2])
        assert np.allclose(M.conj().T @ M, np.eye(M.shape[1]), atol=1e-13)
    rc = O.right_canonicalize(psi)
    for a in rc[1:]:
        M = a.reshape(a.shape[0], -1)
        assert np.allclose(M @ M.conj().T, np.eye(M.shape[0]), atol=1e-13)


def test_expect_local_and_overlap_dense():
    psi = wl.random_mps(6, 4, 8)
    phi = wl.random_mps(6, 3, 9)
    v, u = mps_to_dense(psi), mps_to_dense(phi)
    assert abs(O.mps_overlap(phi, psi) - np.vdot(u, v)) < 1e-13
    for i in (0, 3, 5):
        ref = np.vdot(v, site_op(SZ, i, 6) @ v) / np.vdot(v, v)
        assert abs(O.expect_local(psi, SZ, i) - ref) < 1e-13


def test_local_expm_substeps_reach_expm():
    """R13: a step whose Lanczos space would need more than n_max vectors (spectral range 500,
    delta 0.1: phase range 50) is split into sub-steps and still matches expm to 1e-10; the
    single-run Lanczos with the same n_max refuses it."""
    rng = np.random.default_rng(12)
    n = 80
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    H = 0.5 * (A + A.conj().T)
    H *= 250.0 / np.max(np.abs(np.linalg.eigvalsh(H)))
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    with pytest.raises(O.LanczosNotConverged):
        O.lanczos_expm(lambda v: H @ v, x, 0.1, "real", 1e-12, 20)
    y, it = O.local_expm(lambda v: H @ v, x, 0.1, "real", 1e-12, 20)
    ref = sla.expm(-0.1j * H) @ x
    assert np.linalg.norm(y - ref) < 1e-10 * np.linalg.norm(x)
    assert it > 20
