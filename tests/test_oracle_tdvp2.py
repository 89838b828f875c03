"""Pins of the TDVP2 oracle (no GPU).

TDVP2 is the conventional two-site integrator the paper compares with (Introduction,
Sec. I.C, Fig. 1(c)).  Its oracle is tied to things other than itself: the dense
projected two-site Hamiltonian, exact propagation where the integrator is exact (two
sites; maximal bond dimensions), exact conservation laws, and the failure the paper
reports on the rung-decoupled ladder.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from paper_2005_06104_gb300 import workloads as wl
from exact import heisenberg_dense, mps_to_dense, left_basis, right_basis


def _centre_at(psi, c):
    psi = O.right_canonicalize(psi)
    for i in range(c):
        ml, d, mr = psi[i].shape
        U, S, Vh, _ = O.svd_truncate(psi[i].reshape(ml * d, mr))
        psi[i] = U.reshape(ml, d, -1)
        psi[i + 1] = np.tensordot(S[:, None] * Vh, psi[i + 1], axes=([1], [0]))
    return psi


def _normalised_right_canonical(psi):
    psi = O.right_canonicalize(psi)
    psi[0] = psi[0] / np.linalg.norm(psi[0])
    return psi


@pytest.mark.parametrize("pair", [0, 3, 6])
def test_heff2_is_projected_hamiltonian(pair):
    """H_eff^(2) on bond (i, i+1) equals V^+ H V, V = (left block) x 1_4 x (right block)."""
    lat = wl.zigzag_ladder(4, 1.0, 0.6)
    n = lat.n
    W = wl.heisenberg_mpo(lat)
    H = heisenberg_dense(n, lat.bonds)
    psi = _centre_at(wl.random_mps(n, 5, 31 + pair), pair)
    Ls, Rs = O.build_envs(psi, W, pair)
    PhiL, PhiR = left_basis(psi, pair), right_basis(psi, pair + 2)
    V = np.kron(np.kron(PhiL, np.eye(4)), PhiR)
    Hproj = V.conj().T @ H @ V
    ml, mr = PhiL.shape[1], PhiR.shape[1]
    rng = np.random.default_rng(pair)
    X = rng.standard_normal((ml, 2, 2, mr)) + 1j * rng.standard_normal((ml, 2, 2, mr))
    Y = O.heff2_apply(Ls[pair], W[pair], W[pair + 1], Rs[pair + 1], X)
    assert np.allclose(Y.reshape(-1), Hproj @ X.reshape(-1), atol=1e-12)


@pytest.mark.parametrize("kind", ["real", "imag"])
def test_tdvp2_two_sites_is_exact(kind):
    """On two sites the only bond holds the whole space: one step is exp(-i H dt)."""
    lat = wl.chain(2, 1.0, fields=[0.3, -0.7])
    W = wl.heisenberg_mpo(lat)
    H = heisenberg_dense(2, lat.bonds, lat.fields)
    psi = _normalised_right_canonical(wl.random_mps(2, 2, 3))
    v = mps_to_dense(psi)
    dt = 0.37
    out = O.tdvp2_sweep(psi, W, dt, kind)
    if kind == "real":
        ref = sla.expm(-1j * dt * H) @ v
    else:
        ref = sla.expm(-dt * H) @ v
        ref /= np.linalg.norm(ref)
    assert np.linalg.norm(mps_to_dense(out) - ref) < 1e-11


def test_tdvp2_exact_at_full_bond_dimension():
    """With maximal bond dimensions every projector is the identity and the splitting is exact."""
    lat = wl.chain(8, 1.0, fields=np.linspace(-1, 1, 8))
    W = wl.heisenberg_mpo(lat)
    H = heisenberg_dense(lat.n, lat.bonds, lat.fields)
    psi = _normalised_right_canonical(wl.random_mps(8, 16, 6))
    out = O.tdvp2_sweep(psi, W, 0.3, "real")
    ref = sla.expm(-0.3j * H) @ mps_to_dense(psi)
    assert np.linalg.norm(mps_to_dense(out) - ref) < 1e-9
    assert wl.mps_bond_dims(out) == wl.full_bond_dims(8, 16)


def test_tdvp2_real_time_conserves_norm_and_energy():
    """Without truncation each local step is unitary and keeps <H>: norm and energy hold."""
    lat = wl.zigzag_ladder(4, 1.0, 1.0)
    W = wl.heisenberg_mpo(lat)
    psi = _normalised_right_canonical(wl.random_mps(8, 3, 12))
    e0 = O.mpo_expectation(psi, W).real
    out = psi
    for _ in range(2):
        out = O.tdvp2_sweep(out, W, 0.2, "real")
    assert abs(O.mps_norm(out) - 1) < 1e-12
    assert abs(O.mpo_expectation(out, W).real - e0) < 1e-10
    assert max(wl.mps_bond_dims(out)) > 3                  # the two-site form grows the bonds


def test_tdvp2_truncation_cap_and_cutoff():
    lat = wl.chain(8, 1.0)
    W = wl.heisenberg_mpo(lat)
    psi = _normalised_right_canonical(wl.random_mps(8, 16, 8))
    st = {}
    out = O.tdvp2_sweep(psi, W, 0.2, "real", eps=0.0, chi_max=4, stats=st)
    assert max(wl.mps_bond_dims(out)) == 4
    assert max(st["discarded"]) > 0
    st_cut = {}
    out_cut = O.tdvp2_sweep(psi, W, 0.2, "real", eps=1e-3, stats=st_cut)
    assert all(x <= 1e-3 for x in st_cut["discarded"])
    assert max(wl.mps_bond_dims(out_cut)) < 16


def test_tdvp2_product_state_stays_on_rung_decoupled_ladder():
    """Fig. 1(c): on the rung-decoupled zigzag ladder the sites of every bond belong to
    different legs, so TDVP2 from Neel never builds entanglement and the energy stays put,
    while GSE-TDVP1 (same settings) lowers it."""
    lat = wl.zigzag_ladder(5, 1.0, 0.0)
    W = wl.heisenberg_mpo(lat)
    psi0 = wl.neel_state(lat)
    e0 = O.mpo_expectation(psi0, W).real
    psi = O.right_canonicalize(psi0)
    for _ in range(3):
        psi = O.tdvp2_sweep(psi, W, 0.1, "imag", eps=1e-10, chi_max=32)
    assert max(wl.mps_bond_dims(psi)) == 1
    assert abs(O.mpo_expectation(psi, W).real - e0) < 1e-12
    p = dict(tau=-1j / wl.lambda_top(lat), k=3, eps_k=1e-12, eps_m=1e-8, chi_max=32, dt=0.1,
             kind="imag", eps=1e-10)
    gse = O.gse_tdvp1_step(psi0, W, p)
    assert O.mpo_expectation(gse, W).real < e0 - 1e-3


def test_tdvp2_product_state_grows_on_chain():
    """On a nearest-neighbour chain every bond couples its two sites: TDVP2 leaves the
    product state in one step (TDVP1 cannot, Introduction) and lowers the energy."""
    lat = wl.chain(8)
    W = wl.heisenberg_mpo(lat)
    psi0 = wl.neel_state(lat)
    e0 = O.mpo_expectation(psi0, W).real
    out = O.tdvp2_sweep(O.right_canonicalize(psi0), W, 0.1, "imag", eps=1e-10, chi_max=32)
    assert max(wl.mps_bond_dims(out)) > 1
    assert O.mpo_expectation(out, W).real < e0 - 1e-3
    assert abs(O.mps_norm(out) - 1) < 1e-12
