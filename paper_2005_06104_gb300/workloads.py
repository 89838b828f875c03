"""Seeded synthetic inputs for GSE-TDVP1: lattices, Hamiltonian MPOs and MPS.

This module holds no step of the method itself.  It builds the *inputs* the
method takes (Sec. I: an MPS |psi> and the MPO of H), for the spin-1/2
Heisenberg lattices of the paper's benchmarks (Sec. II.A, Eq. 11; Fig. 1a) and
the one-axis-twisting model (Sec. II.B, Eq. 12).  Both the CUDA path (through
the C-ABI) and the CPU oracle consume these arrays, so neither side can bias
the other through its inputs.

Conventions shared by every consumer:

* spin basis index 0 = |up> (S^z=+1/2), 1 = |down>;
* an MPS is a list of complex128 arrays A_i[m_{i-1}, d, m_i] with m_0 = m_N = 1;
* an MPO is a list of complex128 arrays W_i[w_{i-1}, d, d, w_i] acting as
  <s|W|s'> (second index = output spin, third = input spin), w_0 = w_N = 1;
* the MPO is in finite-state ("start/done") form: at every inner bond channel 0
  means "no operator placed yet" and the last channel means "term complete".
  The left boundary selects "start" and the right boundary "done".
"""
from __future__ import annotations

import numpy as np

D = 2
SZ = np.array([[0.5, 0.0], [0.0, -0.5]], dtype=np.complex128)
SP = np.array([[0.0, 1.0], [0.0, 0.0]], dtype=np.complex128)  # |up><down|
SM = SP.T.copy()
SX = 0.5 * (SP + SM)
SY = -0.5j * (SP - SM)
ID2 = np.eye(2, dtype=np.complex128)


# ---------------------------------------------------------------- lattices
class Lattice:
    """A set of sites with coordinates, a 1D path order and weighted bonds."""

    def __init__(self, coords, bonds, fields=None, name=""):
        self.coords = list(coords)            # path index -> (x, y)
        self.n = len(self.coords)
        b = {}
        for i, j, J in bonds:
            if i == j:
                raise ValueError("self bond")
            key = (min(i, j), max(i, j))
            b[key] = b.get(key, 0.0) + float(J)
        self.bonds = [(i, j, J) for (i, j), J in sorted(b.items()) if J != 0.0]
        self.fields = np.zeros(self.n) if fields is None else np.asarray(fields, float)
        self.name = name

    def index_of(self, x, y):
        return self.coords.index((x, y))


def chain(n, J=1.0, fields=None):
    """Open chain of n sites, nearest-neighbour couplings J."""
    return Lattice([(x, 0) for x in range(n)],
                   [(x, x + 1, J) for x in range(n - 1)], fields, f"chain{n}")


def zigzag_ladder(lx, j_leg=1.0, j_rung=1.0):
    """2 x lx ladder on the zigzag path of Fig. 1a: path index = 2x + y.

    Leg bonds join path sites at distance 2, rung bonds at distance 1.
    """
    coords = [(i // 2, i % 2) for i in range(2 * lx)]
    bonds = []
    for x in range(lx):
        for y in range(2):
            if x + 1 < lx:
                bonds.append((2 * x + y, 2 * (x + 1) + y, j_leg))
        bonds.append((2 * x, 2 * x + 1, j_rung))
    return Lattice(coords, bonds, name=f"ladder2x{lx}")


def cylinder_snake(lx, ly=4, J=1.0):
    """ly x lx cylinder (periodic in y, open in x) on the snake path.

    Column x is walked y = 0..ly-1 when x is even and ly-1..0 when x is odd.
    """
    coords = []
    for x in range(lx):
        ys = range(ly) if x % 2 == 0 else range(ly - 1, -1, -1)
        coords += [(x, y) for y in ys]
    idx = {c: i for i, c in enumerate(coords)}
    bonds = []
    for x in range(lx):
        for y in range(ly):
            if x + 1 < lx:
                bonds.append((idx[(x, y)], idx[(x + 1, y)], J))
            if ly > 2 or y == 0:
                bonds.append((idx[(x, y)], idx[(x, (y + 1) % ly)], J))
    return Lattice(coords, bonds, name=f"cyl{ly}x{lx}")


# ---------------------------------------------------------------- MPOs
def _open_sites(lat):
    """open[c] = sorted sites j <= c-1 (0-based) with a bond partner >= c.

    c runs over cuts 0..n; cut c sits between path sites c-1 and c.
    """
    n = lat.n
    far = [-1] * n
    for i, j, _ in lat.bonds:
        far[i] = max(far[i], j)
    return [[j for j in range(c) if far[j] >= c] for c in range(n + 1)]


def heisenberg_mpo(lat):
    """MPO of H = sum_b J_b S_i.S_j + sum_i h_i S^z_i in start/done form.

    Channels at an inner cut: 0 = start, 1+3k+{0,1,2} = open site k carrying
    (S^z, S^+, S^-), last = done.  w = 2 + 3 * (number of open sites).
    """
    n = lat.n
    opn = _open_sites(lat)
    coup = {}
    for i, j, J in lat.bonds:
        coup[(i, j)] = J

    def width(c):
        if c == 0 or c == n:
            return 1
        return 2 + 3 * len(opn[c])

    W = []
    for i in range(n):
        wl, wr = width(i), width(i + 1)
        w = np.zeros((wl, D, D, wr), dtype=np.complex128)
        l_start = 0
        l_done = wl - 1 if i > 0 else None
        r_start = 0 if i < n - 1 else None
        r_done = wr - 1
        if r_start is not None:
            w[l_start, :, :, r_start] = ID2
        w[l_start, :, :, r_done] += lat.fields[i] * SZ
        if l_done is not None:
            w[l_done, :, :, r_done] = ID2
        if i < n - 1 and i in opn[i + 1]:
            k = opn[i + 1].index(i)
            for a, op in enumerate((SZ, SP, SM)):
                w[l_start, :, :, 1 + 3 * k + a] = op
        if i > 0:
            for kl, j in enumerate(opn[i]):
                if i < n - 1 and j in opn[i + 1]:
                    kr = opn[i + 1].index(j)
                    for a in range(3):
                        w[1 + 3 * kl + a, :, :, 1 + 3 * kr + a] = ID2
                J = coup.get((j, i), 0.0)
                if J != 0.0:
                    w[1 + 3 * kl + 0, :, :, r_done] += J * SZ
                    w[1 + 3 * kl + 1, :, :, r_done] += 0.5 * J * SM
                    w[1 + 3 * kl + 2, :, :, r_done] += 0.5 * J * SP
        W.append(w)
    return W


def oat_mpo(n, chi=1.0):
    """MPO of the one-axis-twisting Hamiltonian chi (S^z_tot)^2 (Eq. 12), w=3.

    (S^z)^2 = sum_i (S^z_i)^2 + 2 sum_{i<j} S^z_i S^z_j; channels start,
    "one S^z placed", done.
    """
    W = []
    for i in range(n):
        wl = 1 if i == 0 else 3
        wr = 1 if i == n - 1 else 3
        w = np.zeros((wl, D, D, wr), dtype=np.complex128)
        rd = wr - 1
        if i < n - 1:
            w[0, :, :, 0] = ID2
            w[0, :, :, 1] = 2.0 * chi * SZ
        w[0, :, :, rd] += chi * SZ @ SZ
        if i > 0:
            w[1, :, :, rd] += SZ
            w[2, :, :, rd] = ID2
            if i < n - 1:
                w[1, :, :, 1] = ID2
        W.append(w)
    return W


def total_op_mpo(n, op):
    """MPO of sum_i op_i (one-site operator on every site), w = 2: channels "before" and
    "after" the site that carries op."""
    W = []
    for i in range(n):
        wl = 1 if i == 0 else 2
        wr = 1 if i == n - 1 else 2
        w = np.zeros((wl, D, D, wr), dtype=np.complex128)
        last = wr - 1
        if i < n - 1:
            w[0, :, :, 0] = ID2
        w[0, :, :, last] += op
        if i > 0:
            w[wl - 1, :, :, last] += ID2
        W.append(w)
    return W


def mpo_product(A, B):
    """MPO of the operator product A B (A applied after B), bond dimensions multiplied:
    P[(w, u), s, s', (v, x)] = sum_t A[w, s, t, v] B[u, t, s', x]."""
    out = []
    for a, b in zip(A, B):
        p = np.einsum("wstv,utrx->wusrvx", a, b)
        wl, ul, d, _, vr, xr = p.shape
        out.append(p.reshape(wl * ul, d, d, vr * xr))
    return out


def mpo_bond_dims(W):
    return [W[0].shape[0]] + [w.shape[3] for w in W]


# ---------------------------------------------------------------- states
def product_state(vectors):
    """MPS of bond dimension 1 from per-site 2-vectors (normalised)."""
    out = []
    for v in vectors:
        v = np.asarray(v, dtype=np.complex128)
        out.append((v / np.linalg.norm(v)).reshape(1, D, 1))
    return out


def neel_state(lat, flip=None):
    """Neel product state: site (x, y) up iff x + y even; `flip` = (x, y) to flip."""
    vecs = []
    for (x, y) in lat.coords:
        up = (x + y) % 2 == 0
        if flip is not None and (x, y) == tuple(flip):
            up = not up
        vecs.append([1.0, 0.0] if up else [0.0, 1.0])
    return product_state(vecs)


def random_product_state(n, seed):
    """Each site cos(t/2)|up> + e^{i p} sin(t/2)|down>, (t, p) uniform on the sphere."""
    rng = np.random.default_rng(seed)
    vecs = []
    for _ in range(n):
        ct = rng.uniform(-1.0, 1.0)
        p = rng.uniform(0.0, 2.0 * np.pi)
        t = np.arccos(ct)
        vecs.append([np.cos(t / 2), np.exp(1j * p) * np.sin(t / 2)])
    return product_state(vecs)


def x_polarized_state(n):
    """All spins along +x (Sec. II.B initial state)."""
    return product_state([[1.0, 1.0]] * n)


def full_bond_dims(n, chi):
    return [min(chi, D ** i, D ** (n - i)) for i in range(n + 1)]


def random_mps(n, chi, seed, bond_dims=None):
    """Dense random complex MPS, entries N(0,1)+iN(0,1), bond dims min(chi, 2^i, 2^(n-i)).

    The tensors are not canonical; the consumer canonicalises.
    """
    rng = np.random.default_rng(seed)
    m = full_bond_dims(n, chi) if bond_dims is None else list(bond_dims)
    out = []
    for i in range(n):
        shape = (m[i], D, m[i + 1])
        a = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
        out.append((a / np.sqrt(np.prod(shape))).astype(np.complex128))
    return out


def random_isometric_mps(n, chi, seed):
    """Right-canonical random MPS, bond dims min(chi, 2^i, 2^(n-i)): every site but the first
    is the conjugate transpose of the orthonormal factor of a Gaussian complex matrix, the first
    a normalised Gaussian tensor.  Its Schmidt spectra are those of random isometries (spread
    over a few decades), unlike the products of Gaussian tensors of random_mps, whose spectra
    span many more."""
    rng = np.random.default_rng(seed)
    m = full_bond_dims(n, chi)
    out = [None] * n
    for i in range(n - 1, 0, -1):
        rows, cols = m[i], D * m[i + 1]
        g = rng.standard_normal((cols, rows)) + 1j * rng.standard_normal((cols, rows))
        q, _ = np.linalg.qr(g)                              # cols x rows, orthonormal columns
        out[i] = q.conj().T.reshape(rows, D, m[i + 1])
    a = rng.standard_normal((1, D, m[1])) + 1j * rng.standard_normal((1, D, m[1]))
    out[0] = (a / np.linalg.norm(a)).astype(np.complex128)
    return out


def mps_bond_dims(mps):
    return [mps[0].shape[0]] + [a.shape[2] for a in mps]


# ---------------------------------------------------------------- U(1) S^z sectors
SZ2 = (1, -1)   # 2 S^z of basis states 0 (up) and 1 (down): the conserved charge per site


def random_u1_mps(n, chi, seed, q_total=0, shuffle=True):
    """Right-canonical random MPS that conserves total 2 S^z = q_total: A_i[l, s, r] is nonzero
    only where q_r = q_l + SZ2[s] (bond charges from q = 0 at the left end to q_total at the
    right end).  Sector dimensions are built from the right: a left sector gets the smaller of
    the columns its block reaches and the left configurations of its charge, scaled down to
    chi in total; each block (a left sector's rows against the right sectors it reaches) is the
    conjugate transpose of the orthonormal factor of a Gaussian complex matrix.  shuffle applies
    a random permutation to every inner bond (both tensors), interleaving the sectors the way a
    factorisation that orders by singular value would."""
    from math import comb
    rng = np.random.default_rng(seed)
    dims = [None] * (n + 1)           # dims[i]: {charge: dimension} on the bond left of site i
    dims[n] = {q_total: 1}
    for i in range(n - 1, -1, -1):
        cand = {}
        for q in range(-i, i + 1, 2):
            reach = sum(dims[i + 1].get(q + dq, 0) for dq in SZ2)
            left = comb(i, (i + q) // 2)
            if reach and left:
                cand[q] = min(reach, left)
        tot = sum(cand.values())
        if tot > chi:
            cand = {q: max(1, (chi * c) // tot) for q, c in cand.items()}
            while sum(cand.values()) > chi:
                qmax = max(cand, key=lambda q: cand[q])
                cand[qmax] -= 1
        dims[i] = cand

    def offsets(dm):
        off, o = {}, 0
        for q in sorted(dm):
            off[q] = o
            o += dm[q]
        return off, o

    out = []
    for i in range(n):
        offl, ml = offsets(dims[i])
        offr, mr = offsets(dims[i + 1])
        A = np.zeros((ml, D, mr), dtype=np.complex128)
        for ql, dl in dims[i].items():
            cols = [(s, qr) for s, dq in enumerate(SZ2) for qr in [ql + dq] if qr in dims[i + 1]]
            width = sum(dims[i + 1][qr] for _, qr in cols)
            g = rng.standard_normal((width, dl)) + 1j * rng.standard_normal((width, dl))
            if i == 0:
                blk = (g / np.linalg.norm(g)).T
            else:
                q, _ = np.linalg.qr(g)                      # width x dl, orthonormal columns
                blk = q.conj().T                            # dl x width, orthonormal rows
            c = 0
            for s, qr in cols:
                w = dims[i + 1][qr]
                A[offl[ql]:offl[ql] + dl, s, offr[qr]:offr[qr] + w] = blk[:, c:c + w]
                c += w
        out.append(A)
    if shuffle:
        for i in range(1, n):
            p = rng.permutation(out[i].shape[0])
            out[i - 1] = out[i - 1][:, :, p]
            out[i] = out[i][p]
    return out


def bond_charges(mps, phys=SZ2, tol=0.0):
    """Charge of every index of every bond, read off the nonzero pattern: q = 0 on the left end,
    q_r = q_l + phys[s] for each entry |A[l, s, r]| > tol.  An index with no such entry (or
    reached only from indices without a charge) gets None.  Raises ValueError when two entries
    give one index different charges (the state does not conserve the charge)."""
    ph = np.asarray(phys, dtype=np.int64)
    qs = [[0] * mps[0].shape[0]]
    for A in mps:
        ql = qs[-1]
        known = np.array([q is not None for q in ql])
        qlv = np.array([q if q is not None else 0 for q in ql], dtype=np.int64)
        nz = (np.abs(A) > tol) & known[:, None, None]
        cand = (qlv[:, None] + ph[None, :])[:, :, None]             # charge each entry implies
        big = np.iinfo(np.int64).max
        lo = np.where(nz, cand, big).min(axis=(0, 1))
        hi = np.where(nz, cand, -big).max(axis=(0, 1))
        has = nz.any(axis=(0, 1))
        bad = has & (lo != hi)
        if bad.any():
            r = int(np.argmax(bad))
            raise ValueError(f"bond index {r} carries charges {lo[r]} and {hi[r]}")
        qs.append([int(lo[r]) if has[r] else None for r in range(A.shape[2])])
    return qs


def mpo_channel_charges(W, phys=SZ2):
    """Charge carried by every channel of every MPO bond: 0 on the left end, and
    c_v = c_w + phys[s] - phys[t] for each nonzero W_i[w, s, t, v] (s output, t input spin), so
    an environment L[a, w, a'] can be nonzero only where q_a - q_a' = c_w.  A channel that no
    chain of nonzero entries reaches from the left end gets None.  Raises ValueError when the
    MPO does not conserve the charge."""
    cs = [[0] * W[0].shape[0]]
    for Wi in W:
        cl = cs[-1]
        cr = [None] * Wi.shape[3]
        for w, s, t, v in np.argwhere(Wi != 0):
            if cl[w] is None:        # a channel no term reaches from the left end
                continue
            c = cl[w] + phys[s] - phys[t]
            if cr[v] is None:
                cr[v] = c
            elif cr[v] != c:
                raise ValueError(f"MPO channel {v} carries charges {cr[v]} and {c}")
        cs.append(cr)
    return cs


def heff_flops_u1(q_l, q_r, Wi, c_l, c_r, phys=SZ2):
    """Real flops of one H_eff apply counted over the nonzero blocks only (8 per complex
    multiply-add), for the three stages of the one-site contraction (Sec. I.C step 3):
      T1[(a,w),(t,b')] = sum_a' L[a,w,a'] x[a',t,b']      L nonzero iff q_a = q_a' + c_w
                                                          x nonzero iff q_b' = q_a' + phys[t]
      T2[(a,s),(v,b')] = sum_{w,t} W[w,s,t,v] T1[...]     T1 nonzero iff q_b' - q_a = phys[t] - c_w
      y[(a,s),b] = sum_{(v,b')} T2[(a,s),(v,b')] R[b,v,b']   R nonzero iff q_b = q_b' + c_v
    (a channel w no term reaches from the left end, c_w None, holds zero environments).
    q_l, q_r: charges of the left and right bond indices; c_l, c_r: channel charges of W's
    bonds.  The dense count of the same stages is 8 [m_l d m_r (m_l w_l + m_r w_r) + m_l m_r nnz W]."""
    from collections import Counter
    ql, qr = Counter(q_l), Counter(q_r)
    cl = Counter(c for c in c_l if c is not None)
    # stage 1: sum over a' of #(a, w) x #(t, b')
    f1 = 0
    for qa1, na1 in ql.items():
        n_aw = sum(nw * ql.get(qa1 + c, 0) for c, nw in cl.items())
        n_tb = sum(qr.get(qa1 + p, 0) for p in phys)
        f1 += na1 * n_aw * n_tb
    # stage 2: each nonzero W entry couples the (a, b') pairs of its charge difference
    f2 = 0
    for w, s, t, v in np.argwhere(Wi != 0):
        if c_l[w] is None:
            continue
        dq = phys[t] - c_l[w]
        f2 += sum(na * qr.get(qa + dq, 0) for qa, na in ql.items())
    # stage 3: sum over (v, b') of #(a, s) x #b; T2 has a block (s, v) only where some W entry
    # of a reachable channel w writes it, and there q_a = q_b' - phys[s] + c_v
    sv = {(int(s), int(v)) for w, s, t, v in np.argwhere(Wi != 0) if c_l[w] is not None}
    f3 = 0
    for s, v in sv:
        c = c_r[v]
        for qb1, nb1 in qr.items():
            f3 += nb1 * ql.get(qb1 - phys[s] + c, 0) * qr.get(qb1 + c, 0)
    return 8.0 * (f1 + f2 + f3)


def u1_heff_operands(q_l, q_r, c_l, c_r, seed, phys=SZ2):
    """Random operands of one U(1) H_eff apply with the zero pattern the charges fix:
    L[a, w, a'] where q_a = q_a' + c_w, R[b, v, b'] where q_b = q_b' + c_v and
    x[a, s, b] where q_b = q_a + phys[s] (Gaussian complex entries there, exact zeros elsewhere;
    channels with charge None are zero)."""
    rng = np.random.default_rng(seed)
    ql, qr = np.asarray(q_l), np.asarray(q_r)
    cl = np.array([np.nan if c is None else c for c in c_l])
    cr = np.array([np.nan if c is None else c for c in c_r])

    def rnd(mask):
        out = np.zeros(mask.shape, dtype=np.complex128)
        k = int(mask.sum())
        out[mask] = rng.standard_normal(k) + 1j * rng.standard_normal(k)
        return out
    L = rnd(ql[:, None, None] == ql[None, None, :] + cl[None, :, None])
    R = rnd(qr[:, None, None] == qr[None, None, :] + cr[None, :, None])
    x = rnd(qr[None, None, :] == ql[:, None, None] + np.asarray(phys)[None, :, None])
    return L, R, x


def sector_table(charges):
    """[(charge, dim, offset)] of one bond when every charge is one contiguous index range,
    else None."""
    table = []
    for k, q in enumerate(charges):
        if table and table[-1][0] == q:
            table[-1][1] += 1
        else:
            table.append([q, 1, k])
    if len({t[0] for t in table}) != len(table):
        return None
    return [tuple(t) for t in table]


# ---------------------------------------------------------------- workloads
def lambda_top(lat):
    """Sum_b J_b / 4: the ferromagnetic energy, the top of the Heisenberg spectrum
    for J_b >= 0 (used for i*tau = 1/lambda in imaginary time, Sec. I.B)."""
    return sum(J for _, _, J in lat.bonds) / 4.0


def workload(name, seed=None):
    """Named synthetic workloads (lattice, MPO, initial state, run parameters).

    heis_chain10   : Heisenberg chain L=10, Neel, real time dt=0.1, k=2, chi<=16
    ladder2x20_rd  : rung-decoupled 2x20 ladder (zigzag), random product state
                     (seed 1), imaginary time dtau=0.1, k=3, chi<=128
    ladder2x50     : rung-coupled 2x50 ladder (zigzag), Neel + flip at (25,0),
                     real time dt=0.1, k=3, chi<=512
    cyl4x16        : 4x16 cylinder (snake), Neel + flip at (8,0), real time
                     dt=0.1, k=3, chi<=1024
    """
    if name == "heis_chain10":
        lat = chain(10)
        return dict(name=name, lattice=lat, mpo=heisenberg_mpo(lat), psi=neel_state(lat),
                    kind="real", dt=0.1, k=2, tau=0.1, chi_max=16, steps=10,
                    eps_k=1e-8, eps_m=1e-8, eps=0.0, tol=1e-12)
    if name == "ladder2x20_rd":
        lat = zigzag_ladder(20, 1.0, 0.0)
        lam = lambda_top(lat)
        return dict(name=name, lattice=lat, mpo=heisenberg_mpo(lat),
                    psi=random_product_state(lat.n, 1 if seed is None else seed),
                    kind="imag", dt=0.1, k=3, tau=-1j / lam, chi_max=128, steps=50,
                    eps_k=1e-12, eps_m=1e-8, eps=1e-10, tol=1e-12)
    if name == "ladder2x50":
        lat = zigzag_ladder(50, 1.0, 1.0)
        return dict(name=name, lattice=lat, mpo=heisenberg_mpo(lat),
                    psi=neel_state(lat, flip=(25, 0)),
                    kind="real", dt=0.1, k=3, tau=0.1, chi_max=512, steps=40,
                    eps_k=1e-8, eps_m=1e-8, eps=0.0, tol=1e-12)
    if name == "cyl4x16":
        lat = cylinder_snake(16, 4)
        return dict(name=name, lattice=lat, mpo=heisenberg_mpo(lat),
                    psi=neel_state(lat, flip=(8, 0)),
                    kind="real", dt=0.1, k=3, tau=0.1, chi_max=1024, steps=20,
                    eps_k=1e-8, eps_m=1e-8, eps=0.0, tol=1e-12)
    raise KeyError(name)


def random_field_chains(n_chains=64, seed=0):
    """Batch of independent random-field Heisenberg chains (PCG64, seed 0):
    lengths U{20..60}, fields U[-2,2], chi_max U{32..128}; Neel start."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_chains):
        n = int(rng.integers(20, 61))
        h = rng.uniform(-2.0, 2.0, size=n)
        chi = int(rng.integers(32, 129))
        lat = chain(n, 1.0, fields=h)
        out.append(dict(lattice=lat, mpo=heisenberg_mpo(lat), psi=neel_state(lat),
                        chi_max=chi, kind="real", dt=0.05, k=2, tau=0.05))
    return out
