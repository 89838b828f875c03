"""U(1) S^z sector helpers of the synthetic inputs (CPU): the random charge-conserving state,
the charges read off a nonzero pattern and the sector tables (charge, dim, offset)."""
import numpy as np
import pytest

import oracle as O
from paper_2005_06104_gb300 import workloads as wl


def _contiguous(mps):
    return all(wl.sector_table(q) is not None for q in wl.bond_charges(mps))


def test_random_u1_state_is_charge_conserving_and_canonical():
    psi = wl.random_u1_mps(12, 40, 3)
    assert not _contiguous(psi)                               # shuffled bonds interleave sectors
    assert _contiguous(wl.random_u1_mps(12, 40, 3, shuffle=False))
    for A in psi[1:]:
        M = A.reshape(A.shape[0], -1)
        assert np.allclose(M @ M.conj().T, np.eye(M.shape[0]), atol=1e-12)
    assert abs(O.mpo_expectation(psi, wl.total_op_mpo(12, wl.SZ))) < 1e-12


def test_bond_charges_of_neel_and_a_violating_state():
    lat = wl.chain(6)
    psi = wl.neel_state(lat)
    qs = wl.bond_charges(psi)
    assert [q[0] for q in qs] == [0, 1, 0, 1, 0, 1, 0]      # 2 S^z of the sites to the left
    bad = wl.random_mps(4, 2, 1)                              # dense: no conserved charge
    with pytest.raises(ValueError):
        wl.bond_charges(bad)


def test_sector_table_offsets():
    assert wl.sector_table([-1, -1, 1, 1, 1, 3]) == [(-1, 2, 0), (1, 3, 2), (3, 1, 5)]
    assert wl.sector_table([-1, 1, -1]) is None
    psi = wl.random_u1_mps(14, 60, 2, shuffle=False)
    for q, A in zip(wl.bond_charges(psi)[1:], psi):
        t = wl.sector_table(q)
        assert sum(dim for _, dim, _ in t) == A.shape[2]
        assert [c for c, _, _ in t] == sorted(c for c, _, _ in t)


@pytest.mark.parametrize("lat", ["cyl3x4", "chain12", "ladder6"])
def test_block_sparse_heff_flops_equal_the_structural_count(lat):
    """The sector formula of the H_eff flops equals a brute-force count over the actual nonzero
    patterns of the oracle's environments and site tensor, stage by stage."""
    lattice = {"cyl3x4": lambda: wl.cylinder_snake(3, 4), "chain12": lambda: wl.chain(12),
               "ladder6": lambda: wl.zigzag_ladder(6, 1.0, 0.5)}[lat]()
    n = lattice.n
    c = n // 2
    W = wl.heisenberg_mpo(lattice)
    psi = wl.random_u1_mps(n, 40, 1)
    Ls, Rs = O.build_envs(psi, W, c)
    Lnz, Rnz, xnz = np.abs(Ls[c]) > 0, np.abs(Rs[c]) > 0, np.abs(psi[c]) > 0
    Wnz = np.argwhere(W[c] != 0)
    f1 = sum(Lnz[:, :, a1].sum() * xnz[a1].sum() for a1 in range(Lnz.shape[2]))
    T1 = np.einsum("awx,xtb->awtb", Lnz.astype(float), xnz.astype(float)) > 0
    f2 = sum(T1[:, w, t, :].sum() for w, s, t, v in Wnz)
    T2 = np.zeros((Lnz.shape[0], 2, W[c].shape[3], xnz.shape[2]), bool)
    for w, s, t, v in Wnz:
        T2[:, s, v, :] |= T1[:, w, t, :]
    f3 = sum(T2[:, :, v, b1].sum() * Rnz[:, v, b1].sum() for v in range(T2.shape[2]) for b1 in range(T2.shape[3]))
    qs, cs = wl.bond_charges(psi), wl.mpo_channel_charges(W)
    got = wl.heff_flops_u1(qs[c], qs[c + 1], W[c], cs[c], cs[c + 1])
    assert got == 8 * (f1 + f2 + f3)
    ml, mr = psi[c].shape[0], psi[c].shape[2]
    dense = 8 * (ml * 2 * mr * (ml * W[c].shape[0] + mr * W[c].shape[3]) + ml * mr * len(Wnz))
    assert got < 0.3 * dense
