"""Plain, slow, dense complex128 oracle for GSE-TDVP1 (arXiv:2005.06104).

TEST INFRASTRUCTURE ONLY: imported by tests, the smoke check and the CPU
baseline leg of the benchmark; never by the product path.

Every function follows one passage of the paper (cited by section/equation)
or, where the paper relies on the standard one-site TDVP integrator it cites
(Sec. I.C step 3; Haegeman et al., PRB 94, 165116), that textbook definition.
Tensors are numpy complex128 arrays:

    MPS site   A[a, s, b]        (m_{i-1}, d, m_i)
    MPO site   W[w, s, s', v]    (w_{i-1}, d, d, w_i), <s|W|s'>
    left env   L[a, w, a']       bra index first, ket index last
    right env  R[b, v, b']       bra index first, ket index last

Readings of places where the paper is silent (all shared with the CUDA path
by specification only, never by code):

  R1  a gauge move that truncates nothing (the real-time sweep, where eps = 0 keeps the
      evolution exactly unitary, Sec. II.B; every canonicalisation) keeps the numerical
      rank: a thin QR (LQ right to left) taken block by block (R8) when every |R_jj|
      exceeds 1e-10 times the largest (full numerical rank: min(rows, cols) directions of
      each block), else the SVD with the numerical rank below.  A plain QR of a
      rank-deficient block (states with extra symmetry, such as the OAT state of Sec. II.B,
      have them) would keep directions set by rounding, which the next local updates then
      evolve into.  Every factorisation that selects (the SVD of the
      centre in the extension, Eq. 3; truncated moves in imaginary time; Krylov
      compression) is an SVD whose numerical rank keeps s > 1e-10 * s_max.  That
      threshold sits two decades above the Lanczos tolerance (1e-12), the size of the
      differences between two correct implementations, so both classify the same
      values; a pin shows that at 1e-14 the gauge-invariant results do not move;
  R2  truncation cutoffs are relative discarded weights: sum of dropped s^2
      (or eigenvalues) <= eps * total;
  R3  a cut never splits a cluster of values within relative 1e-8: the count
      grows to the end of the cluster, and if that breaks a cap it shrinks to
      the cluster's start;
  R4  each TDVP1 half-sweep uses half the time step;
  R5  Krylov vectors are (1 - i tau H)^l |psi>, each compressed and normalised
      (Eq. 10 plus "normalize each MPS separately");
  R6  in imaginary time every local exponential is followed by renormalisation;
  R7  the added rows B_bar are projected off range(B) twice and re-orthonormalised
      (by an SVD, keeping every row) so that B_bar B^+ = 0 holds to rounding;
  R13 a local exponential whose Lanczos space reaches n_max without meeting the tolerance is
      split into 2, 4, ... 64 equal sub-steps (long-range Hamiltonians such as Eq. 12 have a
      spectral range of order N^2 / 4, so one step of delta may need more than n_max vectors);
  R8  a matrix that is block diagonal up to a permutation (its rows and columns
      linked only through nonzero entries; conserved quantum numbers such as S^z
      make the forbidden entries exactly zero) is factorised block by block, and
      the spectra are merged in descending order.  A dense LAPACK call would mix
      singular vectors of near-degenerate values from different blocks and leak
      weight out of the conserved sector (1.6e-6 by step 5 on the 10-site chain).

  Z1  the zip-up application of an MPO truncates its right-to-left pass with 0.1 eps and
      the cap chi_max (the right block is not orthonormal there), then compresses left to
      right with eps and chi_max (R1-R3).

Functions whose parity is pinned by tests only through properties (not by a
closed form): none; every public routine here has a pin in tests/.
"""
from __future__ import annotations

import numpy as np
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components

RANK_RTOL = 1e-10       # R1
CLUSTER_RTOL = 1e-8     # R3
EIG_FLOOR_RTOL = 1e-12  # eigenvalues of Eq. 6 at or below this * tr(rho~) never count
LANCZOS_BREAKDOWN = 1e-13


class LanczosNotConverged(RuntimeError):
    pass


# ------------------------------------------------------------ truncation rule
def keep_count(weights, total, eps, cap, floor):
    """Number of leading (descending) weights to keep under R2/R3.

    weights: descending non-negative values (s^2 or eigenvalues); total: the
    reference weight for the relative cutoff; floor: values <= floor never count.
    """
    w = np.asarray(weights, dtype=np.float64)
    n_cand = int(np.count_nonzero(w > floor))
    if n_cand == 0 or cap <= 0:
        return 0
    w = w[:n_cand]
    # minimal n with sum(w[n:]) <= eps * total (values past n_cand are dropped anyway)
    tail = np.concatenate([np.cumsum(w[::-1])[::-1], [0.0]])
    n = n_cand
    limit = eps * total
    for j in range(n_cand + 1):
        if tail[j] <= limit:
            n = j
            break

    def inside_cluster(j):
        return 0 < j < n_cand and (w[j - 1] - w[j]) <= CLUSTER_RTOL * w[j - 1]

    while inside_cluster(n):
        n += 1
    if n > cap:
        n = cap
        while inside_cluster(n):
            n -= 1
    return n


def _components(nz):
    """Connected blocks of a rows x cols nonzero pattern: list of (row idx, col idx)."""
    rows, cols = nz.shape
    r, c = np.nonzero(nz)
    g = coo_matrix((np.ones(len(r)), (r, rows + c)), shape=(rows + cols, rows + cols))
    ncomp, lab = connected_components(g, directed=False)
    out = []
    for k in range(ncomp):
        ri = np.nonzero(lab[:rows] == k)[0]
        ci = np.nonzero(lab[rows:] == k)[0]
        if len(ri) and len(ci):
            out.append((ri, ci))
    return out


def svd_blocks(M):
    """Thin SVD of M taken block by block (R8): U, S (descending), Vh."""
    rows, cols = M.shape
    comps = _components(M != 0)
    if len(comps) <= 1:
        return np.linalg.svd(M, full_matrices=False)
    parts = []
    for ri, ci in comps:
        u, s, vh = np.linalg.svd(M[np.ix_(ri, ci)], full_matrices=False)
        for k in range(len(s)):
            parts.append((s[k], ri, u[:, k], ci, vh[k]))
    parts.sort(key=lambda t: -t[0])
    kmax = min(rows, cols)
    U = np.zeros((rows, kmax), dtype=M.dtype)
    Vh = np.zeros((kmax, cols), dtype=M.dtype)
    S = np.zeros(kmax)
    for k, (sv, ri, u, ci, vh) in enumerate(parts[:kmax]):
        S[k] = sv
        U[ri, k] = u
        Vh[k, ci] = vh
    return U, S, Vh


def eigh_blocks(H):
    """Eigen-decomposition of a Hermitian H block by block (R8), ascending like eigh."""
    n = H.shape[0]
    comps = _components((H != 0) | (H.conj().T != 0))
    if len(comps) <= 1:
        return np.linalg.eigh(H)
    vals, vecs = [], []
    seen = np.zeros(n, bool)
    for ri, _ in comps:
        w, v = np.linalg.eigh(H[np.ix_(ri, ri)])
        seen[ri] = True
        for k in range(len(w)):
            x = np.zeros(n, dtype=H.dtype)
            x[ri] = v[:, k]
            vals.append(w[k])
            vecs.append(x)
    for i in np.nonzero(~seen)[0]:               # all-zero rows: eigenvalue 0
        x = np.zeros(n, dtype=H.dtype)
        x[i] = 1.0
        vals.append(0.0)
        vecs.append(x)
    order = np.argsort(np.array(vals), kind="stable")
    return np.array(vals)[order], np.array(vecs).T[:, order]


def qr_blocks(M):
    """Thin QR of M block by block (R1, R8): M = Q R with Q^+ Q = 1.

    Each connected block (rows ri, cols ci) gets numpy's Householder QR, keeping
    min(len(ri), len(ci)) columns of Q; the new index runs over the blocks in turn.
    Rows and columns outside every block (all zero) get no direction."""
    rows, cols = M.shape
    comps = _components(M != 0)
    k = sum(min(len(ri), len(ci)) for ri, ci in comps)
    Q = np.zeros((rows, k), dtype=M.dtype)
    R = np.zeros((k, cols), dtype=M.dtype)
    off = 0
    for ri, ci in comps:
        q, r = np.linalg.qr(M[np.ix_(ri, ci)], mode="reduced")
        n = q.shape[1]
        Q[np.ix_(ri, np.arange(off, off + n))] = q
        R[np.ix_(np.arange(off, off + n), ci)] = r
        off += n
    return Q, R


def lq_blocks(M):
    """M = L Q with Q Q^+ = 1, block by block: the conjugate of qr_blocks(M^+)."""
    Qh, Rh = qr_blocks(M.conj().T)
    return Rh.conj().T, Qh.conj().T


def _qr_full_rank(M, R):
    """True when every block of the QR shows full numerical rank: all |R_jj| > RANK_RTOL times
    the largest |R_jj| of the matrix (a rank-deficient block has a column in the span of the
    ones before it, whose remainder R_jj vanishes)."""
    diag = []
    off = 0
    for ri, ci in _components(M != 0):
        n = min(len(ri), len(ci))
        diag.extend(abs(R[off + j, ci[j]]) for j in range(n))
        off += n
    if not diag:
        return False
    return min(diag) > RANK_RTOL * max(diag)


def gauge_split_right(M):
    """M = Q C with orthonormal columns Q, nothing cut (R1): the block QR when it shows full
    numerical rank, else the SVD with the numerical rank (Q = U, C = S Vh)."""
    Q, R = qr_blocks(M)
    if _qr_full_rank(M, R):
        return Q, R
    U, S, Vh, _ = svd_truncate(M)
    return U, S[:, None] * Vh


def gauge_split_left(M):
    """M = C Q with orthonormal rows Q, nothing cut: the mirror image of gauge_split_right."""
    Qh, Ch = gauge_split_right(M.conj().T)
    return Ch.conj().T, Qh.conj().T


def svd_truncate(M, eps=0.0, cap=None):
    """M = U S Vh, keeping columns by R1 + R2 + R3.  Returns U, S, Vh, discarded weight."""
    U, S, Vh = svd_blocks(M)
    if S.size == 0 or S[0] == 0.0:
        return U[:, :0], S[:0], Vh[:0], 0.0
    w = S * S
    total = float(np.sum(w))
    cap = len(S) if cap is None else cap
    n = keep_count(w, total, eps, cap, (RANK_RTOL * S[0]) ** 2)
    disc = float(np.sum(w[n:]) / total)
    return U[:, :n], S[:n], Vh[:n], disc


# ------------------------------------------------------------ MPS gauge moves
def left_canonicalize(mps, eps=0.0, cap=None):
    """Left-orthonormal A_1..A_{N-1}, centre at site N (Eq. 1), left to right: by block
    QRs when nothing is cut (R1), by truncated SVDs when eps or cap is given."""
    out = [a.copy() for a in mps]
    exact = eps == 0.0 and cap is None
    for i in range(len(out) - 1):
        ml, d, mr = out[i].shape
        M = out[i].reshape(ml * d, mr)
        if exact:
            Q, C = gauge_split_right(M)
        else:
            Q, S, Vh, _ = svd_truncate(M, eps, cap)
            C = S[:, None] * Vh
        out[i] = Q.reshape(ml, d, -1)
        out[i + 1] = np.tensordot(C, out[i + 1], axes=([1], [0]))
    return out


def right_canonicalize(mps, eps=0.0, cap=None):
    """Right-orthonormal B_2..B_N, centre at site 1 (Eq. 4), right to left: by block
    LQs when nothing is cut (R1), by truncated SVDs when eps or cap is given."""
    out = [a.copy() for a in mps]
    exact = eps == 0.0 and cap is None
    for i in range(len(out) - 1, 0, -1):
        ml, d, mr = out[i].shape
        M = out[i].reshape(ml, d * mr)
        if exact:
            C, Q = gauge_split_left(M)
        else:
            U, S, Q, _ = svd_truncate(M, eps, cap)
            C = U * S[None, :]
        out[i] = Q.reshape(-1, d, mr)
        out[i - 1] = np.tensordot(out[i - 1], C, axes=([2], [0]))
    return out


def mps_norm(mps):
    return np.sqrt(abs(mps_overlap(mps, mps)))


def mps_overlap(a, b):
    """<a|b> by transfer matrices, left to right."""
    E = np.ones((1, 1), dtype=np.complex128)
    for x, y in zip(a, b):
        T = np.tensordot(E, y, axes=([1], [0]))            # [a, s, b']
        E = np.tensordot(x.conj(), T, axes=([0, 1], [0, 1]))
    return complex(E[0, 0])


def expect_local(mps, op, site):
    """<psi|op_site|psi> / <psi|psi> by transfer matrices."""
    E = np.ones((1, 1), dtype=np.complex128)
    nrm = mps_overlap(mps, mps)
    for i, a in enumerate(mps):
        y = np.tensordot(op, a, axes=([1], [1])).transpose(1, 0, 2) if i == site else a
        T = np.tensordot(E, y, axes=([1], [0]))
        E = np.tensordot(a.conj(), T, axes=([0, 1], [0, 1]))
    return complex(E[0, 0]) / nrm


def mpo_expectation(mps, W):
    """<psi|H|psi> / <psi|psi> by a full left-to-right environment contraction."""
    L = np.ones((1, 1, 1), dtype=np.complex128)
    for a, w in zip(mps, W):
        L = env_left_step(L, a, w)
    return complex(L[0, 0, 0]) / mps_overlap(mps, mps)


# ------------------------------------------------------------ environments, H_eff, K_eff
def env_left_step(L, A, W):
    """L_{i+1}[b,v,b'] = sum conj(A[a,s,b]) L[a,w,a'] W[w,s,s',v] A[a',s',b']."""
    T1 = np.tensordot(L, A, axes=([2], [0]))             # [a, w, s', b']
    T2 = np.tensordot(T1, W, axes=([1, 2], [0, 2]))      # [a, b', s, v]
    out = np.tensordot(A.conj(), T2, axes=([0, 1], [0, 2]))  # [b, b', v]
    return out.transpose(0, 2, 1).copy()


def env_right_step(R, B, W):
    """R_{i-1}[a,w,a'] = sum conj(B[a,s,b]) W[w,s,s',v] R[b,v,b'] B[a',s',b']."""
    U1 = np.tensordot(B, R, axes=([2], [2]))             # [a', s', b, v]
    U2 = np.tensordot(U1, W, axes=([1, 3], [2, 3]))      # [a', b, w, s]
    out = np.tensordot(B.conj(), U2, axes=([1, 2], [3, 1]))  # [a, a', w]
    return out.transpose(0, 2, 1).copy()


def heff_apply(L, W, R, A):
    """One-site effective Hamiltonian (Sec. I.C, complexity O(m^3 w d)):
    Y[a,s,b] = sum L[a,w,a'] W[w,s,s',v] A[a',s',b'] R[b,v,b']."""
    T1 = np.tensordot(L, A, axes=([2], [0]))             # [a, w, s', b']
    T2 = np.tensordot(T1, W, axes=([1, 2], [0, 2]))      # [a, b', s, v]
    return np.tensordot(T2, R, axes=([1, 3], [2, 1]))    # [a, s, b]


def keff_apply(L, R, C):
    """Zero-site (bond) effective Hamiltonian of the TDVP1 backward step:
    Y[a,b] = sum L[a,w,a'] C[a',b'] R[b,w,b']."""
    T = np.tensordot(L, C, axes=([2], [0]))              # [a, w, b']
    return np.tensordot(T, R, axes=([1, 2], [1, 2]))


def build_envs(mps, W, center):
    """L_1..L_center (from sites < center) and R_center..R_N (from sites > center)."""
    n = len(mps)
    Ls = [None] * n
    Rs = [None] * n
    Ls[0] = np.ones((1, 1, 1), dtype=np.complex128)
    for i in range(center):
        Ls[i + 1] = env_left_step(Ls[i], mps[i], W[i])
    Rs[n - 1] = np.ones((1, 1, 1), dtype=np.complex128)
    for i in range(n - 1, center, -1):
        Rs[i - 1] = env_right_step(Rs[i], mps[i], W[i])
    return Ls, Rs


def energy_at_center(mps, W, center):
    """E = <C|H_eff C> / <C|C> at the orthogonality centre."""
    Ls, Rs = build_envs(mps, W, center)
    C = mps[center]
    Y = heff_apply(Ls[center], W[center], Rs[center], C)
    return float(np.real(np.vdot(C, Y) / np.vdot(C, C)))


# ------------------------------------------------------------ local exponential
def lanczos_expm(matvec, x, delta, kind, tol=1e-12, nmax=40):
    """exp(-i delta H) x (kind 'real') or exp(-delta H) x (kind 'imag') for Hermitian H
    given by `matvec`, by Lanczos with full re-orthogonalisation applied twice.

    Stops when beta_{j+1} |[exp(-i delta T_j) e_0]_j| <= tol, on breakdown
    (beta <= 1e-13) or when the Krylov space fills the whole space.
    Returns (y, iterations).
    """
    shape = x.shape
    v = x.reshape(-1)
    n = v.size
    beta0 = np.linalg.norm(v)
    if beta0 == 0.0:
        return x.copy(), 0
    V = [v / beta0]
    alphas, betas = [], []
    coef = (-1j * delta) if kind == "real" else (-delta)
    converged = False
    for j in range(nmax):
        w = matvec(V[j].reshape(shape)).reshape(-1)
        a = float(np.real(np.vdot(V[j], w)))
        w = w - a * V[j]
        if j > 0:
            w = w - betas[j - 1] * V[j - 1]
        Vm = np.array(V)
        for _ in range(2):
            w = w - Vm.T @ (Vm.conj() @ w)
        b = float(np.linalg.norm(w))
        alphas.append(a)
        betas.append(b)
        T = np.diag(alphas) + np.diag(betas[:-1], 1) + np.diag(betas[:-1], -1)
        ev, Q = np.linalg.eigh(T)
        y = Q @ (np.exp(coef * ev) * Q[0, :].conj())
        err = b * abs(y[-1])
        if err <= tol or b <= LANCZOS_BREAKDOWN or j + 1 == n:
            converged = True
            break
        V.append(w / b)
    if not converged:
        raise LanczosNotConverged(f"Lanczos: error {err:.3e} > {tol:.1e} after {nmax} steps")
    out = beta0 * (np.array(V[: len(y)]).T @ y)
    return out.reshape(shape), len(y)


def local_expm(matvec, x, delta, kind, tol=1e-12, nmax=40):
    """exp(-i delta H) x or exp(-delta H) x to the Lanczos tolerance (R11) with the sub-step rule
    R13: when nmax Krylov vectors do not reach tol, the step is split into s = 2, 4, ... 64 equal
    sub-steps, each a Lanczos exponential of delta / s.  Returns (y, total Krylov dimension)."""
    s = 1
    while True:
        try:
            y, total = x, 0
            for _ in range(s):
                y, it = lanczos_expm(matvec, y, delta / s, kind, tol, nmax)
                total += it
            return y, total
        except LanczosNotConverged:
            if 2 * s > 64:
                raise
            s *= 2


# ------------------------------------------------------------ TDVP1 sweep
def tdvp1_sweep(mps, W, dt, kind, eps=0.0, chi_max=None, tol=1e-12, nmax=40, stats=None):
    """One symmetric TDVP1 step (Sec. I.C step 3): left-to-right then right-to-left,
    each with time step dt/2 (R4).  Input: right-canonical, centre at site 1.
    Output: right-canonical, centre at site 1.

    Per site (L->R): A <- exp(-i delta H_eff) A; split A = Q C, by a block QR in real
    time (nothing is cut, eps = 0 keeps the step unitary: R1) and by an SVD with cutoff
    eps and cap in imaginary time (Q = U, C = S Vh); L_{i+1} from Q; C <- exp(+i delta
    K_eff) C; A_{i+1} <- C A_{i+1}.  Mirrored for R->L with LQ.
    """
    n = len(mps)
    psi = [a.copy() for a in mps]
    delta = 0.5 * dt
    imag = kind == "imag"
    cut_eps = eps
    cap = chi_max
    Ls, Rs = build_envs(psi, W, 0)
    iters = []

    def fwd(i, A):
        y, it = local_expm(lambda v: heff_apply(Ls[i], W[i], Rs[i], v), A, delta, kind, tol, nmax)
        iters.append(it)
        return y / np.linalg.norm(y) if imag else y

    def bwd(Lb, Rb, C):
        y, it = local_expm(lambda v: keff_apply(Lb, Rb, v), C, -delta, kind, tol, nmax)
        iters.append(it)
        return y / np.linalg.norm(y) if imag else y

    for i in range(n):
        psi[i] = fwd(i, psi[i])
        if i == n - 1:
            break
        ml, d, mr = psi[i].shape
        M = psi[i].reshape(ml * d, mr)
        if imag:
            Q, S, Vh, _ = svd_truncate(M, cut_eps, cap)
            C = S[:, None] * Vh
        else:
            Q, C = gauge_split_right(M)
        psi[i] = Q.reshape(ml, d, -1)
        Ls[i + 1] = env_left_step(Ls[i], psi[i], W[i])
        C = bwd(Ls[i + 1], Rs[i], C)
        psi[i + 1] = np.tensordot(C, psi[i + 1], axes=([1], [0]))
    for i in range(n - 1, -1, -1):
        psi[i] = fwd(i, psi[i])
        if i == 0:
            break
        ml, d, mr = psi[i].shape
        M = psi[i].reshape(ml, d * mr)
        if imag:
            U, S, Q, _ = svd_truncate(M, cut_eps, cap)
            C = U * S[None, :]
        else:
            C, Q = gauge_split_left(M)
        psi[i] = Q.reshape(-1, d, mr)
        Rs[i - 1] = env_right_step(Rs[i], psi[i], W[i])
        C = bwd(Ls[i], Rs[i - 1], C)
        psi[i - 1] = np.tensordot(psi[i - 1], C, axes=([2], [0]))
    if stats is not None:
        stats["lanczos_iters"] = iters
    return psi


# ------------------------------------------------------------ Krylov vectors (Sec. I.B)
def mpo_one_minus_itau_h(W, tau):
    """MPO of 1 - i tau H with the bond dimension of H's MPO (Sec. I.C step 1).

    In start/done form every term of H enters the "done" channel exactly once,
    so scaling all entries W[x, done] (x != done) by -i tau scales each term
    once; the identity is added as (1/N) 1 on every site's start->done entry.
    """
    n = len(W)
    c = -1j * tau
    out = []
    for i, w in enumerate(W):
        w2 = w.copy()
        wl, d, _, wr = w.shape
        done_r = wr - 1
        done_l = wl - 1 if i > 0 else None
        for x in range(wl):
            if x != done_l:
                w2[x, :, :, done_r] = c * w[x, :, :, done_r]
        w2[0, :, :, done_r] += np.eye(d) / n
        out.append(w2)
    return out


def apply_mpo_exact(W, mps):
    """Exact MPO x MPS: bond dimension m * w."""
    out = []
    for w, a in zip(W, mps):
        T = np.tensordot(w, a, axes=([2], [1]))          # [w, s, v, a, b]
        T = T.transpose(3, 0, 1, 4, 2)                   # [a, w, s, b, v]
        ml, wl, d, mr, wr = T.shape
        out.append(T.reshape(ml * wl, d, mr * wr))
    return out


ZIP_RELAX = 0.1  # Z1: the zip pass truncates with ZIP_RELAX * eps and the cap chi_max


def apply_mpo_zipup(W, mps, eps, chi_max=None):
    """W|mps> by the zip-up algorithm (Stoudenmire and White, NJP 12, 055026), the
    alternative to the density-matrix application that needs no right density environments
    (Sec. I.B names applying the MPO variationally or by density matrices).

    The state is brought to left-canonical form (exact, R1).  A right-to-left pass then
    contracts each site with the MPO and the carry from the right and splits the result
    by an SVD truncated with the relaxed cutoff ZIP_RELAX * eps and the cap chi_max
    (the right block of W|mps> is not orthonormal, so the local weights are only
    approximate there); the rows become right-orthonormal site tensors and U S moves
    left.  A left-to-right compression with eps and chi_max follows.
    Returns a left-canonical MPS with the centre at site N (not normalised)."""
    psi = left_canonicalize(mps)
    n = len(psi)
    carry = np.ones((1, 1, 1), dtype=np.complex128)      # [v, b, r]: MPO bond, state bond, new bond
    out = [None] * n
    for i in range(n - 1, -1, -1):
        T = np.tensordot(psi[i], W[i], axes=([1], [2]))  # [a, b, w, s, v]
        T = np.tensordot(T, carry, axes=([1, 4], [1, 0]))  # [a, w, s, r]
        ml, wl, d, rt = T.shape
        M = T.reshape(ml * wl, d * rt)
        if i == 0:
            out[0] = M.reshape(1, d, rt)
            break
        U, S, Vh, _ = svd_truncate(M, ZIP_RELAX * eps, chi_max)
        out[i] = Vh.reshape(-1, d, rt)
        carry = (U * S[None, :]).reshape(ml, wl, -1).transpose(1, 0, 2)
    return left_canonicalize(out, eps, chi_max)


def krylov_vectors(psi, W, tau, k, eps_k, chi_max, method="exact"):
    """|psi~_l> = (1 - i tau H)^l |psi>, l = 1..k-1 (Eq. 10), each compressed with
    cutoff eps_k and cap chi_max, normalised, left-canonical with centre at N.
    method "exact": exact application and SVD compression (the result of the density-matrix
    algorithm up to ties); "zipup": apply_mpo_zipup."""
    Wk = mpo_one_minus_itau_h(W, tau)
    phis = []
    phi = psi
    for _ in range(1, k):
        if method == "zipup":
            phi = apply_mpo_zipup(Wk, phi, eps_k, chi_max)
        else:
            phi = apply_mpo_exact(Wk, phi)
            phi = right_canonicalize(phi)
            phi = left_canonicalize(phi, eps_k, chi_max)
        phi[-1] = phi[-1] / np.linalg.norm(phi[-1])
        phis.append(phi)
    return phis


# ------------------------------------------------------------ basis extension (Sec. I.A)
def basis_extension(psi, phis, weights=None, eps_m=1e-8, chi_max=None):
    """Extend the bond bases of |psi> by the |psi~_l> (Eqs. 3, 5-7), right to left.

    Inputs: all states left-canonical with centres at site N.  At site i:
    C = U S B (no truncation, R1: only the row space B enters, taken by the block LQ when it
    shows full numerical rank, else by the rank-revealing SVD); P = 1 - B^+ B; rho~ = sum_l w_l C~_l^+ C~_l;
    rho_bar = P rho~ P diagonalised and truncated (eps_m relative to tr rho~,
    count <= min(chi_max - rank B, d m' - rank B)) -> B_bar; B' = [B; B_bar];
    centres move by Eq. 3.  Returns |psi> right-canonical with centre C_1
    (the C~_1 are dropped).
    """
    n = len(psi)
    psi = [a.copy() for a in psi]
    phis = [[a.copy() for a in p] for p in phis]
    wts = [1.0] * len(phis) if weights is None else list(weights)
    added = []
    for i in range(n - 1, 0, -1):
        ml, d, mr = psi[i].shape
        X = psi[i].reshape(ml, d * mr)
        _, B = gauge_split_left(X)                       # R1: the row space, numerical rank
        r = B.shape[0]
        nb = 0
        Bp = B
        if r < d * mr and phis:
            rho = np.zeros((d * mr, d * mr), dtype=np.complex128)
            for wl, p in zip(wts, phis):
                Xl = p[i].reshape(p[i].shape[0], d * mr)
                rho += wl * (Xl.conj().T @ Xl)
            P = np.eye(d * mr) - B.conj().T @ B
            rbar = P @ rho @ P
            rbar = 0.5 * (rbar + rbar.conj().T)
            ev, vec = eigh_blocks(rbar)
            ev, vec = ev[::-1], vec[:, ::-1]
            tr = float(np.real(np.trace(rho)))
            cap = d * mr - r
            if chi_max is not None:
                cap = min(cap, chi_max - r)
            nb = keep_count(np.maximum(ev, 0.0), tr, eps_m, cap, EIG_FLOOR_RTOL * tr)
            if nb > 0:
                # R7: enforce B_bar B^+ = 0 (stated after Eq. 6) to rounding: eigenvectors of
                # small eigenvalues may lean on range(B); project them out twice, re-orthonormalise
                Bbar = vec[:, :nb].conj().T
                for _ in range(2):
                    Bbar = Bbar - (Bbar @ B.conj().T) @ B
                _, _, Bbar = svd_blocks(Bbar)            # orthonormal rows, same span (R7, R8)
                Bp = np.concatenate([B, Bbar], axis=0)
        added.append(nb)
        psi[i] = Bp.reshape(-1, d, mr)
        G = X @ Bp.conj().T                                 # m_{i-1} x m'_{i-1}
        psi[i - 1] = np.tensordot(psi[i - 1], G, axes=([2], [0]))
        for p in phis:
            Xl = p[i].reshape(p[i].shape[0], d * mr)
            p[i - 1] = np.tensordot(p[i - 1], Xl @ Bp.conj().T, axes=([2], [0]))
            p[i] = None
    return psi, added[::-1]


# ------------------------------------------------------------ one GSE-TDVP1 step (Sec. I.C)
def expand_basis(psi, W, tau, k, eps_k, eps_m, chi_max, weights=None, method="exact"):
    """Steps 1 and 2: psi (any gauge) -> right-canonical, centre at site 1, bases enlarged.
    method: how the Krylov vectors apply the MPO (krylov_vectors)."""
    psi = left_canonicalize(psi)
    if k <= 1:
        return right_canonicalize(psi)
    phis = krylov_vectors(psi, W, tau, k, eps_k, chi_max, method)
    out, _ = basis_extension(psi, phis, weights, eps_m, chi_max)
    return out


def gse_tdvp1_step(psi, W, p, stats=None):
    """Steps 1-3 of GSE-TDVP1 with the parameters dict p (keys as in workloads)."""
    psi = expand_basis(psi, W, p["tau"], p["k"], p["eps_k"], p["eps_m"], p["chi_max"],
                       p.get("weights"), p.get("krylov", "exact"))
    return tdvp1_sweep(psi, W, p["dt"], p["kind"], p.get("eps", 0.0), p["chi_max"],
                       p.get("tol", 1e-12), p.get("nmax", 40), stats)


# ------------------------------------------------------------ sampled outputs at large sizes
def heff_apply_entries(L, W, R, A, entries):
    """Selected entries y[a,s,b] of the H_eff definition, one at a time:
    y[a,s,b] = sum_{w,s',v} W[w,s,s',v] (L[a,w,:] A[:,s',:] R[b,v,:]^T)."""
    out = []
    for a, s, b in entries:
        acc = 0.0j
        for t in range(A.shape[1]):
            M = L[a] @ A[:, t, :] @ R[b].T                  # (w_l, w_r)
            acc += np.sum(W[:, s, t, :] * M)
        out.append(acc)
    return np.array(out)
