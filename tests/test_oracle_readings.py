"""Pins of the oracle's readings R1 (gauge moves and numerical rank) and R8 (block-by-block
factorisation), on the CPU.

R1: a gauge move that cuts nothing is a thin QR per block (real-time sweeps keep eps = 0,
Sec. II.B; canonicalisations); the SVDs that select keep s > 1e-10 s_max.  The pins show
(i) the QR factors are exact, orthonormal and confined to their blocks, (ii) the result of
whole GSE-TDVP1 steps does not depend on which stable QR is used, and (iii) moving the rank
threshold from 1e-10 to 1e-14 leaves every gauge-invariant result unchanged to rounding.

R8: block-diagonal matrices (up to permutation) are factorised block by block.  The pins show
the merged spectra equal the dense ones, the vectors stay inside their blocks, and total S^z
(conserved by the Heisenberg dynamics, Sec. II) stays exact along GSE-TDVP1 steps, which a
dense factorisation of near-degenerate spectra does not guarantee.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from oracle import gse_tdvp1 as G
from paper_2005_06104_gb300 import workloads as wl

SZ = np.diag([0.5, -0.5]).astype(np.complex128)


def _block_matrix(rng, sizes, square=False):
    """A random complex matrix that is block diagonal after a random permutation of its rows
    and columns; returns it with the blocks' row and column index sets."""
    rows = sum(r for r, _ in sizes)
    cols = sum(c for _, c in sizes)
    M = np.zeros((rows, cols), dtype=np.complex128)
    pr, pc = rng.permutation(rows), rng.permutation(cols)
    if square:
        pc = pr
    blocks, r0, c0 = [], 0, 0
    for r, c in sizes:
        ri, ci = pr[r0:r0 + r], pc[c0:c0 + c]
        M[np.ix_(ri, ci)] = rng.standard_normal((r, c)) + 1j * rng.standard_normal((r, c))
        blocks.append((set(ri.tolist()), set(ci.tolist())))
        r0 += r
        c0 += c
    return M, blocks


def _block_of(blocks, idx, axis):
    for b, (ri, ci) in enumerate(blocks):
        if idx in (ri if axis == 0 else ci):
            return b
    return None


# ------------------------------------------------------------------ R1: QR gauge moves
@pytest.mark.parametrize("sizes", [[(6, 3), (2, 5), (4, 4)], [(9, 2), (1, 1), (3, 7)]])
def test_qr_blocks_exact_orthonormal_and_confined(sizes):
    rng = np.random.default_rng(5)
    M, blocks = _block_matrix(rng, sizes)
    Q, R = O.qr_blocks(M)
    k = sum(min(r, c) for r, c in sizes)
    assert Q.shape == (M.shape[0], k) and R.shape == (k, M.shape[1])
    assert np.allclose(Q.conj().T @ Q, np.eye(k), atol=1e-14)
    assert np.allclose(Q @ R, M, atol=1e-13)
    # every column of Q lives on the rows of one block and its row of R on that block's columns
    for j in range(k):
        rb = {_block_of(blocks, i, 0) for i in np.nonzero(Q[:, j])[0]}
        cb = {_block_of(blocks, i, 1) for i in np.nonzero(R[j])[0]}
        assert len(rb) == 1 and (cb <= rb)
    # a dense QR fills the forbidden entries with rounding noise (what R8 avoids)
    Qd, _ = np.linalg.qr(M)
    assert np.count_nonzero(Qd) > np.count_nonzero(Q)
    # LQ is the mirror image
    Lm, Qr = O.lq_blocks(M)
    assert np.allclose(Qr @ Qr.conj().T, np.eye(Qr.shape[0]), atol=1e-14)
    assert np.allclose(Lm @ Qr, M, atol=1e-13)


def test_qr_blocks_span_the_range():
    """For a full-column-rank block the QR directions span exactly its range: they equal the
    SVD's left singular vectors up to a unitary."""
    rng = np.random.default_rng(8)
    M, _ = _block_matrix(rng, [(7, 4), (5, 3)])
    Q, _ = O.qr_blocks(M)
    U = np.linalg.svd(M, full_matrices=False)[0]
    assert np.allclose(U @ (U.conj().T @ Q), Q, atol=1e-13)
    assert Q.shape[1] == np.linalg.matrix_rank(M)


def _pivoted_qr_blocks(M):
    """Another stable QR (Householder with column pivoting, blocks in reverse order)."""
    rows, cols = M.shape
    comps = G._components(M != 0)[::-1]
    k = sum(min(len(ri), len(ci)) for ri, ci in comps)
    Q = np.zeros((rows, k), dtype=np.complex128)
    R = np.zeros((k, cols), dtype=np.complex128)
    off = 0
    for ri, ci in comps:
        q, r, piv = sla.qr(M[np.ix_(ri, ci)], mode="economic", pivoting=True)
        rr = np.zeros_like(r)
        rr[:, piv] = r
        n = q.shape[1]
        Q[np.ix_(ri, np.arange(off, off + n))] = q
        R[np.ix_(np.arange(off, off + n), ci)] = rr
        off += n
    return Q, R


def _trajectory(psi, W, p, steps):
    out = []
    for _ in range(steps):
        psi = O.gse_tdvp1_step(psi, W, p)
        out.append((O.mpo_expectation(psi, W).real,
                    np.array([O.expect_local(psi, SZ, i).real for i in range(len(psi))]), psi))
    return out


def _max_difference(a, b):
    worst = 0.0
    for x, y in zip(a, b):
        assert [t.shape for t in x[2]] == [t.shape for t in y[2]]   # same bond dimensions
        worst = max(worst, abs(x[0] - y[0]), float(np.max(np.abs(x[1] - y[1]))),
                    abs(1.0 - abs(O.mps_overlap(x[2], y[2]))))
    return worst


def _cases():
    p1 = wl.workload("heis_chain10")
    lat = wl.zigzag_ladder(6, 1.0, 1.0)
    p2 = dict(tau=0.1, k=3, eps_k=1e-8, eps_m=1e-8, chi_max=64, dt=0.1, kind="real", eps=0.0)
    return [("chain10", p1["psi"], p1["mpo"], p1, 10),
            ("ladder2x6", wl.neel_state(lat, flip=(3, 0)), wl.heisenberg_mpo(lat), p2, 5)]


@pytest.mark.parametrize("case", [0, 1], ids=["chain10", "ladder2x6"])
def test_real_time_steps_do_not_depend_on_the_qr(case, monkeypatch):
    """The real-time result is a function of the state, not of the QR's rounding: a pivoted
    Householder QR taking the blocks in the other order reproduces every step to 1e-12."""
    _, psi, W, p, steps = _cases()[case]
    ref = _trajectory(psi, W, p, steps)
    monkeypatch.setattr(G, "qr_blocks", _pivoted_qr_blocks)
    alt = _trajectory(psi, W, p, steps)
    assert _max_difference(ref, alt) < 1e-12


@pytest.mark.parametrize("case", [0, 1], ids=["chain10", "ladder2x6"])
def test_rank_threshold_reading_does_not_move_results(case, monkeypatch):
    """R1's numerical-rank threshold 1e-10 s_max against 1e-14 s_max: with the gauge moves as
    QRs, E, <S^z_i> and the state (overlap) agree to 1e-12 and the bond dimensions are equal
    at every step of config 1 (10 steps) and of the 2 x 6 ladder (5 steps)."""
    _, psi, W, p, steps = _cases()[case]
    ref = _trajectory(psi, W, p, steps)
    monkeypatch.setattr(G, "RANK_RTOL", 1e-14)
    alt = _trajectory(psi, W, p, steps)
    assert _max_difference(ref, alt) < 1e-12


# ------------------------------------------------------------------ R8: block factorisations
def test_svd_blocks_equals_dense_spectrum_and_confines_vectors():
    rng = np.random.default_rng(3)
    M, blocks = _block_matrix(rng, [(6, 4), (3, 5), (5, 5), (2, 1)])
    U, S, Vh = O.svd_blocks(M)
    assert np.allclose(S, np.linalg.svd(M, compute_uv=False), rtol=1e-13, atol=1e-14)
    assert np.all(np.diff(S) <= 0)
    k = int(np.count_nonzero(S))           # the blocks' own values; the rest are zero padding
    assert k == 4 + 3 + 5 + 1
    U, Vh = U[:, :k], Vh[:k]
    assert np.allclose(U.conj().T @ U, np.eye(k), atol=1e-13)
    assert np.allclose(Vh @ Vh.conj().T, np.eye(k), atol=1e-13)
    assert np.allclose((U * S[:k]) @ Vh, M, atol=1e-13)
    for j in range(k):
        rb = {_block_of(blocks, i, 0) for i in np.nonzero(U[:, j])[0]}
        cb = {_block_of(blocks, i, 1) for i in np.nonzero(Vh[j])[0]}
        assert len(rb) == 1 and rb == cb


def test_eigh_blocks_equals_dense_spectrum_and_confines_vectors():
    rng = np.random.default_rng(4)
    X, blocks = _block_matrix(rng, [(5, 5), (3, 3), (4, 4)], square=True)
    H = X @ X.conj().T
    # two blocks share an eigenvalue: a dense solver may mix their vectors, the block one may not
    H2 = H.copy()
    ev, vec = O.eigh_blocks(H2)
    assert np.allclose(ev, np.linalg.eigvalsh(H2), rtol=1e-12, atol=1e-12)
    assert np.allclose(vec.conj().T @ vec, np.eye(len(ev)), atol=1e-13)
    assert np.allclose(H2 @ vec, vec * ev, atol=1e-11)
    for j in range(len(ev)):
        assert len({_block_of(blocks, i, 0) for i in np.nonzero(vec[:, j])[0]}) == 1


def test_eigh_blocks_degenerate_blocks_stay_separate():
    """Exactly degenerate eigenvalues in two different blocks: every eigenvector still lives in
    one block (a dense eigh returns arbitrary mixtures of the two)."""
    rng = np.random.default_rng(6)
    A = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
    A = A @ A.conj().T
    H = np.zeros((8, 8), dtype=np.complex128)
    perm = rng.permutation(8)
    H[np.ix_(perm[:4], perm[:4])] = A
    H[np.ix_(perm[4:], perm[4:])] = A          # the same spectrum twice
    _, vec = O.eigh_blocks(H)
    first = set(perm[:4].tolist())
    for j in range(8):
        nz = set(np.nonzero(vec[:, j])[0].tolist())
        assert nz <= first or not (nz & first)


def _total_sz_variance(psi):
    """<(S^z_tot)^2> - <S^z_tot>^2 of an MPS, by the dense vector (small chains)."""
    v = psi[0].reshape(-1, psi[0].shape[2])
    for a in psi[1:]:
        v = (v @ a.reshape(a.shape[0], -1)).reshape(-1, a.shape[2])
    v = v.reshape(-1)
    n = len(psi)
    sz = np.zeros(2 ** n)
    for i in range(n):
        bit = (np.arange(2 ** n) >> (n - 1 - i)) & 1
        sz += 0.5 - bit
    w = np.abs(v) ** 2 / np.vdot(v, v).real
    return float(w @ sz ** 2 - (w @ sz) ** 2), float(w @ sz)


def test_total_sz_stays_exact_along_gse_steps():
    """Ten GSE-TDVP1 steps of config 1 (Neel chain, S^z_tot = 0): the variance of S^z_tot stays
    at rounding (1e-14).  The block factorisations keep every basis vector inside one S^z
    sector, so no weight can leak between sectors."""
    p = wl.workload("heis_chain10")
    psi, W = p["psi"], p["mpo"]
    for _ in range(10):
        psi = O.gse_tdvp1_step(psi, W, p)
        var, mean = _total_sz_variance(psi)
        assert var < 1e-14 and abs(mean) < 1e-14
        # every bond vector carries one S^z charge: from the right end (charge 0), the
        # nonzero entries A[a, s, b] of each row a give one value sz(s) + q(b)
        q = np.zeros(1)
        for a in psi[::-1]:
            ml = a.shape[0]
            qn = np.full(ml, np.nan)
            for r in range(ml):
                s_idx, b_idx = np.nonzero(a[r])
                vals = set(np.round(np.array([0.5, -0.5])[s_idx] + q[b_idx], 6).tolist())
                assert len(vals) <= 1
                if vals:
                    qn[r] = vals.pop()
            q = qn


def _householder_qr_blocks(M):
    """Another unpivoted QR of each block, written out (beta = -e^{i arg x_0} |x|, reflectors
    applied column by column, Q accumulated backward): the same |R_jj| as numpy's up to rounding,
    other rounding everywhere."""
    rows, cols = M.shape
    comps = G._components(M != 0)
    k = sum(min(len(ri), len(ci)) for ri, ci in comps)
    Q = np.zeros((rows, k), dtype=np.complex128)
    R = np.zeros((k, cols), dtype=np.complex128)
    off = 0
    for ri, ci in comps:
        X = M[np.ix_(ri, ci)].copy()
        p_, q_ = X.shape
        kq = min(p_, q_)
        vs, taus = [], []
        for j in range(kq):
            x = X[j:, j].copy()
            nrm = np.linalg.norm(x)
            ph = x[0] / abs(x[0]) if abs(x[0]) > 0 else 1.0
            v = x.copy()
            v[0] = x[0] + ph * nrm
            vn = np.linalg.norm(v)
            if vn == 0:
                vs.append(None)
                continue
            v = v / vn
            X[j:, j:] -= 2.0 * np.outer(v, v.conj() @ X[j:, j:])
            vs.append(v)
        Qb = np.eye(p_, kq, dtype=np.complex128)
        for j in range(kq - 1, -1, -1):
            if vs[j] is not None:
                Qb[j:, :] -= 2.0 * np.outer(vs[j], vs[j].conj() @ Qb[j:, :])
        Q[np.ix_(ri, np.arange(off, off + kq))] = Qb
        R[np.ix_(np.arange(off, off + kq), ci)] = np.triu(X[:kq])
        off += kq
    return Q, R


def test_rank_deficient_moves_fall_back_to_the_rank_revealing_svd(monkeypatch):
    """R1 on a state with extra symmetry: one OAT step at N = 100 (Sec. II.B, dt = 0.05, k = 5)
    meets tall blocks of numerical rank below their width (s_min / s_max ~ 1e-17).  With the
    SVD fallback the step does not depend on the unpivoted QR used (3e-9 in <S^x>, the
    conditioning of the directions kept at s ~ 1e-9 s_max); a plain QR of the deficient blocks
    keeps rounding-set directions, and two QRs then disagree by 1.3e-4."""
    n = 100
    W = wl.oat_mpo(n)
    Mx = wl.total_op_mpo(n, wl.SX)
    p = dict(tau=0.05, k=5, eps_k=1e-4, eps_m=1e-8, chi_max=64, dt=0.05, kind="real", eps=0.0)

    def sx(qr, fallback):
        monkeypatch.setattr(G, "qr_blocks", qr)
        if not fallback:
            monkeypatch.setattr(G, "_qr_full_rank", lambda M, R: True)
        out = O.gse_tdvp1_step(wl.x_polarized_state(n), W, p)
        monkeypatch.undo()
        return O.mpo_expectation(out, Mx).real
    qr0 = G.qr_blocks
    Q, R = _householder_qr_blocks(np.arange(12.0).reshape(4, 3) + 1j)
    assert np.allclose(Q @ R, np.arange(12.0).reshape(4, 3) + 1j) and np.allclose(Q.conj().T @ Q, np.eye(3))
    assert abs(sx(qr0, True) - sx(_householder_qr_blocks, True)) < 1e-8
    assert abs(sx(qr0, False) - sx(_householder_qr_blocks, False)) > 1e-6
