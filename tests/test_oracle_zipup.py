"""Pins of the oracle's zip-up MPO application (no GPU).

Sec. I.B applies 1 - i tau H either by density matrices or variationally; the zip-up
algorithm is the application that needs no right density environments.  It is tied to
the dense product W|psi>, to the compression error bound of a canonical truncation sweep,
to exactness for an MPO without bonds, and to the density-matrix (exact + SVD) Krylov
vectors of Eq. 10.
"""
import numpy as np
import pytest

import oracle as O
from paper_2005_06104_gb300 import workloads as wl
from exact import mps_to_dense, mpo_to_dense


def _case(seed=4):
    lat = wl.zigzag_ladder(5, 1.0, 0.7)
    W = O.mpo_one_minus_itau_h(wl.heisenberg_mpo(lat), 0.1)
    psi = wl.random_mps(lat.n, 6, seed)
    return lat, W, psi


def _random_mpo(n, w, seed):
    """A random complex MPO with bond dimension w: not Hermitian, not symmetric."""
    rng = np.random.default_rng(seed)
    dims = [1] + [w] * (n - 1) + [1]
    return [(rng.standard_normal((dims[i], 2, 2, dims[i + 1])) + 1j * rng.standard_normal((dims[i], 2, 2, dims[i + 1])))
            / np.sqrt(2 * dims[i]) for i in range(n)]


@pytest.mark.parametrize("which", ["one_minus_itau_h", "random_w3"])
def test_zipup_without_cutoff_is_the_exact_product(which):
    lat, W, psi = _case()
    if which == "random_w3":
        W = _random_mpo(lat.n, 3, 5)
    ex = mpo_to_dense(W) @ mps_to_dense(psi)
    z = O.apply_mpo_zipup(W, psi, 0.0, None)
    assert np.linalg.norm(mps_to_dense(z) - ex) < 1e-12 * np.linalg.norm(ex)
    for a in z[:-1]:                                        # left-canonical, centre at N
        M = a.reshape(-1, a.shape[2])
        assert np.allclose(M.conj().T @ M, np.eye(M.shape[1]), atol=1e-12)


@pytest.mark.parametrize("eps", [1e-4, 1e-6, 1e-8])
def test_zipup_error_within_truncation_bound(eps):
    """Each of the 2(N-1) truncations drops at most eps of the weight (the zip pass
    0.1 eps): the relative error stays below sqrt(2 (N-1) eps)."""
    lat, W, psi = _case()
    ex = mpo_to_dense(W) @ mps_to_dense(psi)
    z = O.apply_mpo_zipup(W, psi, eps, None)
    err = np.linalg.norm(mps_to_dense(z) - ex) / np.linalg.norm(ex)
    assert 0 < err <= np.sqrt(2 * (lat.n - 1) * eps)


def test_zipup_commutes_with_site_unitaries():
    """Site unitaries leave every Schmidt spectrum unchanged, so the truncations make the
    same choices: zip-up of U|psi> (an MPO without bonds) equals U applied to the zip-up
    of |psi> under the identity MPO, at any cutoff."""
    n = 8
    rng = np.random.default_rng(2)
    U, I = [], []
    for _ in range(n):
        h = rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))
        q, _ = np.linalg.qr(h)
        U.append(q.reshape(1, 2, 2, 1))
        I.append(np.eye(2, dtype=complex).reshape(1, 2, 2, 1))
    psi = wl.random_mps(n, 4, 7)
    z = O.apply_mpo_zipup(U, psi, 1e-3, None)
    ref = O.apply_mpo_exact(U, O.apply_mpo_zipup(I, psi, 1e-3, None))
    assert wl.mps_bond_dims(z) == wl.mps_bond_dims(ref)
    assert np.linalg.norm(mps_to_dense(z) - mps_to_dense(ref)) < 1e-12 * np.linalg.norm(mps_to_dense(ref))
    assert np.linalg.norm(mps_to_dense(z) - mpo_to_dense(U) @ mps_to_dense(psi)) > 1e-6  # it did truncate


def test_zipup_krylov_vectors_match_the_density_matrix_ones():
    lat = wl.zigzag_ladder(5, 1.0, 1.0)
    W = wl.heisenberg_mpo(lat)
    psi = O.left_canonicalize(wl.random_mps(lat.n, 5, 9))
    psi[-1] /= np.linalg.norm(psi[-1])
    a = O.krylov_vectors(psi, W, 0.1, 3, 1e-10, 64, method="exact")
    b = O.krylov_vectors(psi, W, 0.1, 3, 1e-10, 64, method="zipup")
    for x, y in zip(a, b):
        assert abs(abs(O.mps_overlap(x, y)) - 1) < 1e-9
