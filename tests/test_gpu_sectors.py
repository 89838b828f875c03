"""U(1) S^z sectors on the device (GPU vs oracle and vs the FP64 GPU form).

The Heisenberg Hamiltonian conserves total S^z, so every tensor of a state with definite S^z
is block-sparse in the bond charges (Sec. I.C: the cost statement counts only the nonzero
blocks).  The engine keeps dense storage but
  * orders the kept vectors of every new bond by block, so each charge sector is one
    contiguous index range (a gauge permutation of the bond), and
  * lets the BF16 tensor-core GEMMs skip every (output tile, 128-deep chunk) whose A or B
    tile is all zero: those add exact zeros.
The tests check the contiguity through charges read off the nonzero pattern, that the GEMMs
skip block work on such operands, and that results keep the oracle's values and the precision
form's bars.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O
from paper_2005_06104_gb300 import workloads as wl

TOL_BF16X10 = 5e-8
TOL_BF16X6 = 3e-6


@pytest.fixture(scope="module")
def g():
    assert torch.cuda.is_available()
    from paper_2005_06104_gb300 import gse_tdvp
    return gse_tdvp


def _contiguous(mps):
    qs = wl.bond_charges(mps)
    return all(wl.sector_table(q) is not None for q in qs)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("prec,tol", [("bf16x10", TOL_BF16X10), ("bf16x6", TOL_BF16X6)])
def test_heff_on_sector_ordered_environments_skips_zero_tiles(g, prec, tol):
    """H_eff at the middle site of a 20-site U(1) state at bond dimension 384 (sectors of up
    to about 100 indices; about 30 % of the (tile, chunk) pairs meet nonzero tiles of both
    operands): the BF16 forms match the oracle to their bars while multiplying well under all
    pairs."""
    n, c = 20, 10
    lat = wl.chain(n)
    W = wl.heisenberg_mpo(lat)
    psi = wl.random_u1_mps(n, 384, 5, shuffle=False)
    Ls, Rs = O.build_envs(psi, W, c)
    L, R, x = Ls[c], Rs[c], psi[c]
    assert min(x.shape[0], x.shape[2]) >= 300
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    Ld, Rd, xd = dev(L), dev(R), dev(x)
    yd = torch.empty_like(xd)
    p = g.PREC_BF16X10 if prec == "bf16x10" else g.PREC_BF16X6
    v0, m0 = g.gemm_chunk_stats()
    g.heff_contract(Ld, W[c], Rd, xd, yd, precision=p)
    v1, m1 = g.gemm_chunk_stats()
    ref = O.heff_apply(L, W[c], R, x)
    assert _rel(yd.cpu().numpy(), ref) < tol
    visited, multiplied = v1 - v0, m1 - m0
    assert visited > 0
    assert multiplied < 0.5 * visited, (visited, multiplied)
    # the zero pattern of y is the conserved one: exact zeros stay exact
    y = yd.cpu().numpy()
    assert np.all(y[ref == 0] == 0)


def test_dense_operands_skip_nothing(g):
    rng = np.random.default_rng(2)
    W = wl.heisenberg_mpo(wl.chain(6))[3]
    ml, mr = 200, 190
    r = lambda *s: rng.standard_normal(s) + 1j * rng.standard_normal(s)
    L, R, x = r(ml, W.shape[0], ml), r(mr, W.shape[3], mr), r(ml, 2, mr)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    Ld, Rd, xd = dev(L), dev(R), dev(x)
    yd = torch.empty_like(xd)
    v0, m0 = g.gemm_chunk_stats()
    g.heff_contract(Ld, W, Rd, xd, yd, precision=g.PREC_BF16X10)
    v1, m1 = g.gemm_chunk_stats()
    assert v1 - v0 > 0 and m1 - m0 == v1 - v0
    assert _rel(yd.cpu().numpy(), O.heff_apply(L, W, R, x)) < TOL_BF16X10


def test_engine_regroups_shuffled_sectors_and_matches_oracle(g):
    """A U(1) state whose bonds interleave the sectors: creating the handle (block QRs) and
    every GSE-TDVP1 step leave each sector contiguous, and the FP64 trajectory equals the
    oracle's."""
    n = 12
    lat = wl.chain(n)
    W = wl.heisenberg_mpo(lat)
    psi = wl.random_u1_mps(n, 48, 7)
    assert not _contiguous(psi)
    p = dict(tau=0.1, k=3, eps_k=1e-10, eps_m=1e-9, chi_max=64, dt=0.1, kind="real", eps=0.0)
    st = g.GseTdvp(psi, W, tau=0.1, eps_k=1e-10, eps_m=1e-9, chi_max=64)
    assert _contiguous(st.get_mps())
    ref = psi
    for _ in range(3):
        st.step(0.1, g.REAL, 3)
        ref = O.gse_tdvp1_step(ref, W, p)
        mine = st.get_mps()
        assert _contiguous(mine)
        assert st.bond_dims() == wl.mps_bond_dims(ref)
        assert abs(abs(O.mps_overlap(mine, ref)) - 1) < 1e-10
    assert abs(st.energy() - O.mpo_expectation(ref, W).real) < 1e-10
    st.close()


def test_bf16_steps_on_u1_state_skip_block_work_and_keep_the_bar(g):
    """Real-time GSE-TDVP1 on a 16-site U(1) state at chi 256: the BF16X10 form follows FP64 to
    relative 1e-7 in energy per step while its GEMMs skip the all-zero block work."""
    n = 16
    lat = wl.chain(n)
    W = wl.heisenberg_mpo(lat)
    psi = wl.random_u1_mps(n, 256, 9)
    kw = dict(tau=0.1, eps_k=1e-8, eps_m=1e-8, chi_max=256)
    a = g.GseTdvp(psi, W, precision=g.PREC_FP64, **kw)
    b = g.GseTdvp(psi, W, precision=g.PREC_BF16X10, **kw)
    v0, m0 = g.gemm_chunk_stats()
    for _ in range(2):
        a.step(0.1, g.REAL, 3)
        b.step(0.1, g.REAL, 3)
        assert abs(b.energy() - a.energy()) <= 1e-7 * abs(a.energy())
        assert abs(b.norm() - 1) < 1e-10
    v1, m1 = g.gemm_chunk_stats()
    assert _contiguous(b.get_mps())
    assert m1 - m0 < 0.7 * (v1 - v0), (v1 - v0, m1 - m0)
    a.close()
    b.close()


def test_bond_charges_and_sector_tables_through_the_abi(g):
    """tdvp_bond_charges and tdvp_bond_sectors (device read-out of the charges off the zero
    pattern) equal the host's reading of the state the handle returns, bit for bit, after
    tdvp_create on a shuffled U(1) state of total charge 2 and after GSE-TDVP1 steps (BF16X10);
    the right end carries the total charge and every sector is one contiguous range."""
    n = 16
    lat = wl.chain(n)
    W = wl.heisenberg_mpo(lat)
    psi = wl.random_u1_mps(n, 48, 3, q_total=2)
    h = g.GseTdvp(psi, W, tau=0.05, eps_k=1e-8, eps_m=1e-8, chi_max=64, precision=g.PREC_BF16X10)
    for step in range(3):
        if step:
            h.step(0.05, g.REAL, 3)
        q = h.bond_charges()
        ref = wl.bond_charges(h.get_mps())
        assert q == ref
        assert q[0] == [0] and q[n] == [2]
        for b in range(n + 1):
            tab, cont = h.bond_sectors(b)
            host = wl.sector_table(ref[b])
            assert cont and host is not None
            assert tab == host
    # spin flip: local charges (-1, +1) negate every bond charge
    assert h.bond_charges(phys=(-1, 1)) == [[-c for c in b] for b in ref]
    h.close()


def test_bond_charges_refuse_a_state_that_breaks_the_charge(g):
    """A dense random MPS conserves no charge: the read-out returns TDVP_ERR_SHAPE."""
    n = 8
    W = wl.heisenberg_mpo(wl.chain(n))
    h = g.GseTdvp(wl.random_mps(n, 6, 1), W, chi_max=16)
    with pytest.raises(g.TDVPError) as ei:
        h.bond_charges()
    assert ei.value.status == 2
    with pytest.raises(g.TDVPError):
        h.bond_sectors(3)
    h.close()
