"""Exact-diagonalisation and dense helpers used as pins for the oracle.

These are written independently of oracle/: Hamiltonians are assembled from
Kronecker products of spin matrices, MPS are contracted to dense vectors with
plain matrix products, and exponentials come from scipy.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

SZ = np.diag([0.5, -0.5]).astype(complex)
SP = np.array([[0, 1], [0, 0]], dtype=complex)
SM = np.array([[0, 0], [1, 0]], dtype=complex)
SX = 0.5 * (SP + SM)
SY = -0.5j * (SP - SM)


def site_op(op, i, n, sparse=False):
    """op acting on site i of n (site 0 is the most significant tensor factor)."""
    if sparse:
        return sp.kron(sp.kron(sp.identity(2 ** i, format="csr"), sp.csr_matrix(op)),
                       sp.identity(2 ** (n - i - 1), format="csr"), format="csr")
    return np.kron(np.kron(np.eye(2 ** i), op), np.eye(2 ** (n - i - 1)))


def heisenberg_dense(n, bonds, fields=None, sparse=False):
    """sum_b J (Sx Sx + Sy Sy + Sz Sz) + sum h Sz from explicit Kronecker products."""
    dim = 2 ** n
    H = sp.csr_matrix((dim, dim), dtype=complex) if sparse else np.zeros((dim, dim), complex)
    for i, j, J in bonds:
        for op in (SX, SY, SZ):
            H = H + J * (site_op(op, i, n, sparse) @ site_op(op, j, n, sparse))
    if fields is not None:
        for i, h in enumerate(fields):
            if h != 0:
                H = H + h * site_op(SZ, i, n, sparse)
    return H


def total_op(op, n):
    return sum(site_op(op, i, n) for i in range(n))


def mpo_to_dense(W):
    """Contract an MPO W_i[w,s,s',v] to a dense matrix with site 0 most significant."""
    M = W[0][0]                                   # [s, s', v]
    M = M.transpose(2, 0, 1)                      # [v, S, S']
    for w in W[1:]:
        v, S, Sp = M.shape
        T = np.tensordot(M, w, axes=([0], [0]))   # [S, S', s, s', v2]
        T = T.transpose(4, 0, 2, 1, 3)            # [v2, S, s, S', s']
        M = T.reshape(T.shape[0], S * 2, Sp * 2)
    return M[0]


def mps_to_dense(mps):
    v = mps[0].reshape(-1, mps[0].shape[2])       # [s1, b]
    for a in mps[1:]:
        v = (v @ a.reshape(a.shape[0], -1)).reshape(-1, a.shape[2])
    return v.reshape(-1)


def left_basis(mps, i):
    """Dense vectors of the left block states at bond i (columns): (2^i, m_i)."""
    if i == 0:
        return np.ones((1, 1), dtype=complex)
    v = mps[0].reshape(-1, mps[0].shape[2])
    for a in mps[1:i]:
        v = (v @ a.reshape(a.shape[0], -1)).reshape(-1, a.shape[2])
    return v


def right_basis(mps, i):
    """Dense vectors of the right block states at bond i (columns): (2^(n-i), m_i)."""
    n = len(mps)
    if i == n:
        return np.ones((1, 1), dtype=complex)
    v = mps[n - 1].reshape(mps[n - 1].shape[0], -1)      # [a, s_n]
    for a in reversed(mps[i:n - 1]):
        v = (a.reshape(-1, a.shape[2]) @ v).reshape(a.shape[0], -1)
    return v.T


def ground_energy_sz0(n, bonds):
    """Lowest eigenvalue of the Heisenberg Hamiltonian in the S^z_tot = 0 sector."""
    dim = 2 ** n
    states = [s for s in range(dim) if bin(s).count("1") == n // 2]
    H = heisenberg_dense(n, bonds, sparse=True)
    idx = np.array(states)
    Hs = H[idx][:, idx]
    if len(states) < 400:
        return float(np.linalg.eigvalsh(Hs.toarray())[0])
    return float(spla.eigsh(Hs, k=1, which="SA", tol=1e-12)[0][0])


def expm_apply(H, v, t):
    return sla.expm(-1j * t * H) @ v
