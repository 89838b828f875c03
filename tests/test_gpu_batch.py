"""Batches of independent chains (tdvp_batch_*): every chain evolves exactly as it would
alone, one chain matches the oracle, and a failing chain leaves the others untouched."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O
from paper_2005_06104_gb300 import workloads as wl


@pytest.fixture(scope="module")
def g():
    assert torch.cuda.is_available()
    from paper_2005_06104_gb300 import gse_tdvp
    return gse_tdvp


def _chains(seed=11):
    """Random-field Heisenberg chains of uneven length and bond cap (seeded), Neel start."""
    rng = np.random.default_rng(seed)
    out = []
    for n, chi in ((8, 12), (14, 24), (11, 16), (17, 32), (9, 8)):
        lat = wl.chain(n, 1.0, fields=rng.uniform(-2.0, 2.0, size=n))
        out.append((wl.neel_state(lat), wl.heisenberg_mpo(lat),
                    dict(tau=0.05, eps_k=1e-10, eps_m=1e-10, chi_max=chi)))
    return out


def test_batch_chains_match_single_runs(g):
    chains = _chains()
    b = g.GseTdvpBatch(chains, n_threads=4)
    for _ in range(2):
        assert b.step(0.05, g.REAL, 2) == [0] * len(chains)
    for i, (psi, W, kw) in enumerate(chains):
        a = g.GseTdvp(psi, W, **kw)
        for _ in range(2):
            a.step(0.05, g.REAL, 2)
        c = b.chain(i)
        assert c.bond_dims() == a.bond_dims()
        assert abs(abs(O.mps_overlap(c.get_mps(), a.get_mps())) - 1) < 1e-12
        assert abs(b.energies()[i] - a.energy()) < 1e-12 * abs(a.energy())
        a.close()
    assert all(abs(x - 1) < 1e-12 for x in b.norms())
    b.close()


def test_batch_chain_matches_oracle(g):
    psi, W, kw = _chains()[0]
    b = g.GseTdvpBatch([_chains()[4], (psi, W, kw)], n_threads=2)
    b.step(0.05, g.REAL, 2)
    p = dict(tau=0.05, k=2, eps_k=1e-10, eps_m=1e-10, chi_max=kw["chi_max"], dt=0.05, kind="real", eps=0.0)
    ref = O.gse_tdvp1_step(psi, W, p)
    mine = b.chain(1).get_mps()
    assert abs(abs(O.mps_overlap(mine, ref)) - 1) < 1e-9
    b.close()


def test_failing_chain_is_isolated(g):
    chains = _chains()[:3]
    bad = (chains[1][0], chains[1][1], dict(chains[1][2], lanczos_max=1))
    b = g.GseTdvpBatch([chains[0], bad, chains[2]], n_threads=3)
    e0 = b.energies()
    with pytest.raises(g.TDVPError) as e:
        b.step(0.05, g.REAL, 2)
    assert e.value.status == 4
    statuses = (g.C.c_int * 3)()
    s = g._lib.tdvp_batch_sweep(b.b, 0.05, g.REAL, statuses)
    assert s == 4 and list(statuses) == [0, 4, 0]
    e1 = b.energies()
    assert abs(e1[0] - e0[0]) < 1e-9 * abs(e0[0]) and abs(e1[2] - e0[2]) < 1e-9 * abs(e0[2])
    b.close()
