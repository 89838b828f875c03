"""Plain, slow, dense complex128 oracle for the two-site TDVP (TDVP2).

TEST INFRASTRUCTURE ONLY: imported by tests, never by the product path.

The paper does not restate TDVP2; it is the conventional integrator that GSE-TDVP1 is
measured against (Introduction: a one-site or two-site form of the projector-splitting
scheme; the two-site form truncates and so lets the bond dimension change; Sec. I.C: the
cost of a GSE-TDVP1 step against a TDVP2 step at the same bond dimension; Sec. II: the
failure on the rung-decoupled ladder, Fig. 1(c)).  This module follows the two-site form of
the integrator the paper cites (Haegeman et al., PRB 94, 165116), in the tensor conventions
of gse_tdvp1.py.

Per bond (i, i+1) of a left-to-right half-sweep:
  1. Theta = A_i A_{i+1}, the two-site centre;
  2. Theta <- exp(-i delta H_eff^(2)) Theta;
  3. Theta = U S Vh, truncated;  A_i <- U;  L_{i+1} from U;
  4. C = S Vh is the centre on site i+1; unless i+1 is the last site,
     C <- exp(+i delta H_eff^(1)) C (the backward step of the splitting);
  5. A_{i+1} <- C.
The right-to-left half-sweep is the mirror image.  Each half-sweep advances dt/2 (R4).

Readings (shared with the CUDA path by specification only):
  T1  the two-site SVD keeps the numerical rank (R1) and truncates with the cutoff eps
      and the cap chi_max (R2, R3) in real and in imaginary time alike: TDVP2 has no other
      way to bound its bond dimension, and the paper runs it in real time with eps = 1e-15
      and 1e-7 (Sec. II.B);
  T2  in imaginary time every local exponential is followed by renormalisation (R6).
"""
from __future__ import annotations

import numpy as np

from .gse_tdvp1 import build_envs, env_left_step, env_right_step, heff_apply, local_expm, svd_truncate


def heff2_apply(L, W1, W2, R, X):
    """Two-site effective Hamiltonian (the projected H on the two-site tangent space):
    Y[a,s,t,b] = sum L[a,w,a'] W1[w,s,s',u] W2[u,t,t',v] X[a',s',t',b'] R[b,v,b']."""
    T1 = np.tensordot(L, X, axes=([2], [0]))             # [a, w, s', t', b']
    T2 = np.tensordot(T1, W1, axes=([1, 2], [0, 2]))     # [a, t', b', s, u]
    T3 = np.tensordot(T2, W2, axes=([4, 1], [0, 2]))     # [a, b', s, t, v]
    return np.tensordot(T3, R, axes=([1, 4], [2, 1]))    # [a, s, t, b]


def tdvp2_sweep(mps, W, dt, kind, eps=0.0, chi_max=None, tol=1e-12, nmax=40, stats=None):
    """One symmetric TDVP2 step: left to right, then right to left, dt/2 each.
    Input: right-canonical, centre at site 1.  Output: the same gauge.
    `stats` (a dict) receives the Lanczos iteration counts and the discarded weights."""
    n = len(mps)
    if n < 2:
        raise ValueError("TDVP2 needs at least two sites")
    psi = [a.copy() for a in mps]
    delta = 0.5 * dt
    imag = kind == "imag"
    Ls, Rs = build_envs(psi, W, 0)
    iters, disc = [], []

    def evolve(matvec, x, dl):
        y, it = local_expm(matvec, x, dl, kind, tol, nmax)
        iters.append(it)
        return y / np.linalg.norm(y) if imag else y

    def split(theta):
        ml, d1, d2, mr = theta.shape
        U, S, Vh, dw = svd_truncate(theta.reshape(ml * d1, d2 * mr), eps, chi_max)
        disc.append(dw)
        return U, S, Vh

    for i in range(n - 1):
        theta = np.tensordot(psi[i], psi[i + 1], axes=([2], [0]))
        theta = evolve(lambda x: heff2_apply(Ls[i], W[i], W[i + 1], Rs[i + 1], x), theta, delta)
        ml, d1, d2, mr = theta.shape
        U, S, Vh = split(theta)
        psi[i] = U.reshape(ml, d1, -1)
        Ls[i + 1] = env_left_step(Ls[i], psi[i], W[i])
        C = (S[:, None] * Vh).reshape(-1, d2, mr)
        if i < n - 2:
            C = evolve(lambda x: heff_apply(Ls[i + 1], W[i + 1], Rs[i + 1], x), C, -delta)
        psi[i + 1] = C
    for i in range(n - 2, -1, -1):
        theta = np.tensordot(psi[i], psi[i + 1], axes=([2], [0]))
        theta = evolve(lambda x: heff2_apply(Ls[i], W[i], W[i + 1], Rs[i + 1], x), theta, delta)
        ml, d1, d2, mr = theta.shape
        U, S, Vh = split(theta)
        psi[i + 1] = Vh.reshape(-1, d2, mr)
        Rs[i] = env_right_step(Rs[i + 1], psi[i + 1], W[i + 1])
        C = (U * S[None, :]).reshape(ml, d1, -1)
        if i > 0:
            C = evolve(lambda x: heff_apply(Ls[i], W[i], Rs[i], x), C, -delta)
        psi[i] = C
    if stats is not None:
        stats["lanczos_iters"] = iters
        stats["discarded"] = disc
    return psi
