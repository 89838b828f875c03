"""Parity of the device-resident GSE-TDVP1 engine (through the C ABI) with the
oracle on identical seeded inputs.

Tensors differ by gauge between the two implementations, so states are
compared through gauge-invariant quantities: |<psi_gpu|psi_oracle>|, energies,
norms, local expectation values and bond dimensions.  FP64 agreement target
is 1e-10 (relative for energies, absolute for overlaps and <S^z>).  Both sides
factorise block-diagonal matrices block by block, so the conserved S^z stays
exact; the oracle against itself with Lanczos tol 1e-12 vs 1e-13 then differs
by ~1e-14 after 10 steps of the 10-site chain, well inside these bounds.
"""
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


def _opts(p):
    return dict(tau=p["tau"], eps_k=p["eps_k"], eps_m=p["eps_m"], eps=p.get("eps", 0.0), chi_max=p["chi_max"],
                lanczos_tol=p.get("tol", 1e-12))


def test_create_is_exact_gauge_move(g):
    lat = wl.zigzag_ladder(5, 1.0, 0.7)
    W = wl.heisenberg_mpo(lat)
    psi = wl.random_mps(lat.n, 12, 3)
    st = g.GseTdvp(psi, W)
    assert st.center() == lat.n - 1
    mine = st.get_mps()
    nrm = O.mps_norm(psi)
    assert abs(abs(O.mps_overlap(mine, psi)) / nrm ** 2 - 1) < 1e-12
    for a in mine[:-1]:                           # left-orthonormal
        M = a.reshape(-1, a.shape[2])
        assert np.allclose(M.conj().T @ M, np.eye(M.shape[1]), atol=1e-12)
    assert abs(st.energy() - O.mpo_expectation(psi, W).real) < 1e-10
    for c in (0, 3, 7):
        st.canonicalize(c)
        assert st.center() == c
        assert abs(st.energy() - O.mpo_expectation(psi, W).real) < 1e-10
    for i in (0, 4, 9):
        ref = O.expect_local(psi, wl.SZ, i)
        assert abs(st.expect_local(wl.SZ, i) - ref) < 1e-12
    st.close()


def test_sweep_krylov_dimensions_equal_the_oracle(g):
    """Each local exponential stops by the same test on both sides (R11), so the Krylov
    dimensions of a sweep, summed, and the number of exponentials equal the oracle's.  Small
    local problems launch several Lanczos iterations per host check, guided by the previous
    run's dimension: three sweeps in a row (the later ones with hints) keep the counts."""
    lat = wl.zigzag_ladder(5, 1.0, 1.0)
    W = wl.heisenberg_mpo(lat)
    psi = O.right_canonicalize(wl.random_mps(lat.n, 10, 8))
    psi[0] /= np.linalg.norm(psi[0])
    st = g.GseTdvp(psi, W, eps=0.0, chi_max=64)
    ref = psi
    for _ in range(3):
        stats = {}
        st.sweep(0.1, g.REAL)
        ref = O.tdvp1_sweep(ref, W, 0.1, "real", 0.0, 64, stats=stats)
        nfo = st.trunc_stats()
        assert nfo["lanczos_calls"] == len(stats["lanczos_iters"])
        assert nfo["lanczos_iters"] == sum(stats["lanczos_iters"])
    assert abs(abs(O.mps_overlap(st.get_mps(), ref)) - 1) < 1e-10
    st.close()


@pytest.mark.parametrize("kind", ["real", "imag"])
def test_tdvp1_sweep_matches_oracle(g, kind):
    lat = wl.zigzag_ladder(5, 1.0, 1.0)
    W = wl.heisenberg_mpo(lat)
    psi = O.right_canonicalize(wl.random_mps(lat.n, 10, 8))
    psi[0] /= np.linalg.norm(psi[0])
    eps = 1e-10 if kind == "imag" else 0.0
    st = g.GseTdvp(psi, W, eps=eps, chi_max=64)
    ref = psi
    for _ in range(3):
        st.sweep(0.1, g.REAL if kind == "real" else g.IMAG)
        ref = O.tdvp1_sweep(ref, W, 0.1, kind, eps, 64)
    mine = st.get_mps()
    assert st.bond_dims() == wl.mps_bond_dims(ref)
    assert abs(abs(O.mps_overlap(mine, ref)) - 1) < 1e-10
    assert abs(st.energy() - O.mpo_expectation(ref, W).real) < 1e-10
    assert abs(st.norm() - 1) < 1e-12
    st.close()


@pytest.mark.parametrize("tau,eps_k,cap", [(0.1, 1e-10, 64), (-0.25j, 1e-12, 64), (0.1, 1e-6, 12)])
def test_krylov_vector_matches_oracle(g, tau, eps_k, cap):
    """Density-matrix application of 1 - i tau H (GPU) == exact application + SVD compression (oracle)."""
    lat = wl.zigzag_ladder(6, 1.0, 0.6)
    W = wl.heisenberg_mpo(lat)
    psi = O.left_canonicalize(wl.random_mps(lat.n, 6, 21))
    psi[-1] /= np.linalg.norm(psi[-1])
    st = g.GseTdvp(psi, W, tau=tau, eps_k=eps_k, chi_max=cap)
    st.apply_krylov()
    ref = O.krylov_vectors(psi, W, tau, 2, eps_k, cap)[0]
    mine = st.get_mps()
    assert st.bond_dims() == wl.mps_bond_dims(ref)
    assert abs(abs(O.mps_overlap(mine, ref)) - 1) < 1e-10
    assert abs(st.norm() - 1) < 1e-12
    st.close()


def test_expand_basis_matches_oracle(g):
    lat = wl.zigzag_ladder(6, 1.0, 1.0)
    W = wl.heisenberg_mpo(lat)
    psi = wl.random_mps(lat.n, 3, 5)
    psi = O.left_canonicalize(psi)
    psi[-1] /= np.linalg.norm(psi[-1])
    st = g.GseTdvp(psi, W, tau=0.1, eps_k=1e-10, eps_m=1e-9, chi_max=40)
    st.expand_basis(3)
    ref = O.expand_basis(psi, W, 0.1, 3, 1e-10, 1e-9, 40)
    mine = st.get_mps()
    assert st.center() == 0
    assert st.bond_dims() == wl.mps_bond_dims(ref)
    assert abs(O.mps_overlap(mine, psi) - 1) < 1e-12         # the state is unchanged (Sec. I.A)
    for a in mine[1:]:                                        # B' right-orthonormal (Eq. 7)
        M = a.reshape(a.shape[0], -1)
        assert np.allclose(M @ M.conj().T, np.eye(M.shape[0]), atol=1e-12)
    assert st.trunc_stats()["added"] > 0
    # the enlarged bases are the same spaces: one sweep from each agrees
    st.sweep(0.1, g.REAL)
    ref = O.tdvp1_sweep(ref, W, 0.1, "real")
    assert abs(abs(O.mps_overlap(st.get_mps(), ref)) - 1) < 1e-10
    st.close()


def test_gse_real_time_heisenberg_chain(g):
    """Heisenberg chain L=10, Neel, dt=0.1, k=2, chi<=16, 10 steps: GPU == oracle."""
    p = wl.workload("heis_chain10")
    W, psi = p["mpo"], p["psi"]
    st = g.GseTdvp(psi, W, **_opts(p))
    ref = psi
    e0 = O.mpo_expectation(psi, W).real
    for _ in range(p["steps"]):
        st.step(p["dt"], g.REAL, p["k"])
        ref = O.gse_tdvp1_step(ref, W, p)
        assert st.bond_dims() == wl.mps_bond_dims(ref)
        assert abs(st.energy() - e0) < 1e-10                 # real time conserves energy
    mine = st.get_mps()
    assert abs(abs(O.mps_overlap(mine, ref)) - 1) < 1e-10
    for i in range(10):
        assert abs(st.expect_local(wl.SZ, i).real - O.expect_local(ref, wl.SZ, i).real) < 1e-10
    st.close()


def test_gse_imaginary_time_decoupled_ladder(g):
    """Rung-decoupled zigzag ladder, random product start (seed 1), imaginary time, k=3."""
    lat = wl.zigzag_ladder(6, 1.0, 0.0)
    W = wl.heisenberg_mpo(lat)
    psi = wl.random_product_state(lat.n, 1)
    lam = wl.lambda_top(lat)
    p = dict(tau=-1j / lam, k=3, eps_k=1e-12, eps_m=1e-8, chi_max=32, dt=0.1, kind="imag", eps=1e-10)
    st = g.GseTdvp(psi, W, **_opts(p))
    ref = psi
    for _ in range(5):
        st.step(p["dt"], g.IMAG, 3)
        ref = O.gse_tdvp1_step(ref, W, p)
    e_ref = O.mpo_expectation(ref, W).real
    assert abs(st.energy() - e_ref) < 1e-10 * abs(e_ref)
    assert st.bond_dims() == wl.mps_bond_dims(ref)
    st.close()


def test_precision_form_imaginary_time(g):
    """Imaginary time on the rung-coupled ladder (config 2's kind of run): the BF16X10 form
    follows the FP64 form to relative 1e-7 in energy at every step and both approach the
    ground state from above."""
    lat = wl.zigzag_ladder(6, 1.0, 1.0)
    W = wl.heisenberg_mpo(lat)
    psi = wl.random_product_state(lat.n, 1)
    lam = wl.lambda_top(lat)
    kw = dict(tau=-1j / lam, eps_k=1e-10, eps_m=1e-8, chi_max=48, eps=1e-10)
    a = g.GseTdvp(psi, W, precision=g.PREC_FP64, **kw)
    b = g.GseTdvp(psi, W, precision=g.PREC_BF16X10, **kw)
    e_prev = a.energy()
    for _ in range(6):
        a.step(0.2, g.IMAG, 3)
        b.step(0.2, g.IMAG, 3)
        ea, eb = a.energy(), b.energy()
        assert abs(eb - ea) <= 1e-7 * abs(ea)
        assert abs(b.norm() - 1) < 1e-10
        assert ea <= e_prev + 1e-12
        e_prev = ea
    a.close()
    b.close()


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x10"])
def test_precision_form_energy_and_norm(g, prec):
    """Tensor-core sweeps hold relative energy error <= 1e-7 and norm drift <= 1e-10 per step
    against the FP64 GPU form (real time, rung-coupled ladder, Neel with one flipped spin)."""
    lat = wl.zigzag_ladder(8, 1.0, 1.0)
    W = wl.heisenberg_mpo(lat)
    psi = wl.neel_state(lat, flip=(4, 0))
    kw = dict(tau=0.1, eps_k=1e-8, eps_m=1e-8, chi_max=48)
    a = g.GseTdvp(psi, W, precision=g.PREC_FP64, **kw)
    b = g.GseTdvp(psi, W, precision=g.PREC_TF32X3 if prec == "tf32x3" else g.PREC_BF16X10, **kw)
    e0 = a.energy()
    for _ in range(4):
        a.step(0.1, g.REAL, 3)
        b.step(0.1, g.REAL, 3)
        assert abs(b.norm() - 1) < 1e-10
        assert abs(b.energy() - a.energy()) <= 1e-7 * abs(a.energy())
    assert abs(a.energy() - e0) < 1e-10 * abs(e0)
    a.close()
    b.close()


def test_krylov_precision_bf16x6_keeps_the_energy_bar(g):
    """Krylov vectors in BF16X6 (3 slices) under a BF16X10 sweep: the state itself still holds
    relative energy error <= 1e-7 and norm drift <= 1e-10 per step against FP64 (the Krylov
    vectors only enrich the basis, Sec. I.B)."""
    lat = wl.zigzag_ladder(8, 1.0, 1.0)
    W = wl.heisenberg_mpo(lat)
    psi = wl.neel_state(lat, flip=(4, 0))
    kw = dict(tau=0.1, eps_k=1e-8, eps_m=1e-8, chi_max=48)
    a = g.GseTdvp(psi, W, precision=g.PREC_FP64, **kw)
    b = g.GseTdvp(psi, W, precision=g.PREC_BF16X10, **kw)
    b.krylov_precision(g.PREC_BF16X6)
    for _ in range(4):
        a.step(0.1, g.REAL, 3)
        b.step(0.1, g.REAL, 3)
        assert abs(b.norm() - 1) < 1e-10
        assert abs(b.energy() - a.energy()) <= 1e-7 * abs(a.energy())
    with pytest.raises(g.TDVPError):
        b.krylov_precision(9)
    a.close()
    b.close()


def test_errors_are_status_codes(g):
    lat = wl.chain(4)
    W = wl.heisenberg_mpo(lat)
    st = g.GseTdvp(wl.neel_state(lat), W)
    with pytest.raises(g.TDVPError) as e:
        st.canonicalize(7)
    assert e.value.status == 1
    with pytest.raises(g.TDVPError):
        st.expand_basis(0)
    st.set_options(lanczos_max=1)
    psi = wl.random_mps(4, 4, 1)
    st2 = g.GseTdvp(psi, W, lanczos_max=1)
    with pytest.raises(g.TDVPError) as e:
        st2.sweep(1.0, g.REAL)
    assert e.value.status == 4
    st.close()
    st2.close()


def test_save_and_load_resume_the_trajectory(g, tmp_path):
    """A checkpoint taken mid-trajectory resumes it: the loaded handle holds the same state
    (up to the exact gauge move of create) and the next step matches the uninterrupted run."""
    lat = wl.zigzag_ladder(5, 1.0, 1.0)
    W = wl.heisenberg_mpo(lat)
    kw = dict(tau=0.1, eps_k=1e-10, eps_m=1e-10, chi_max=32)
    a = g.GseTdvp(wl.neel_state(lat, flip=(2, 0)), W, **kw)
    a.step(0.1, g.REAL, 3)
    p = tmp_path / "mid.gse"
    a.save(p)
    b = g.GseTdvp.load(p, W, **kw)
    assert abs(abs(O.mps_overlap(a.get_mps(), b.get_mps())) - 1) < 1e-12
    assert b.bond_dims() == a.bond_dims()
    a.step(0.1, g.REAL, 3)
    b.step(0.1, g.REAL, 3)
    assert abs(abs(O.mps_overlap(a.get_mps(), b.get_mps())) - 1) < 1e-10
    assert abs(a.energy() - b.energy()) < 1e-10
    a.close()
    b.close()


@pytest.mark.parametrize("prec,chi", [("fp64", 8), ("bf16x10", 32)])
def test_checkpointed_density_environments_are_identical(g, prec, chi):
    """With a budget below the density environments' size only every K-th stays resident and
    the rest are rebuilt: the Krylov step and the following sweep are bit-identical."""
    lat = wl.zigzag_ladder(6, 1.0, 0.6)
    W = wl.heisenberg_mpo(lat)
    psi = O.left_canonicalize(wl.random_mps(lat.n, chi, 21))
    psi[-1] /= np.linalg.norm(psi[-1])
    kw = dict(tau=0.1, eps_k=1e-10, eps_m=1e-9, chi_max=64,
              precision=g.PREC_FP64 if prec == "fp64" else g.PREC_BF16X10)
    a = g.GseTdvp(psi, W, **kw)
    b = g.GseTdvp(psi, W, **kw)
    b.krylov_memory(1.0)
    a.apply_krylov()
    b.apply_krylov()
    assert a.krylov_memory() == 1
    assert b.krylov_memory() == int(np.ceil(np.sqrt(lat.n)))
    for x, y in zip(a.get_mps(), b.get_mps()):
        assert np.array_equal(x, y)
    a.step(0.1, g.REAL, 3)
    b.step(0.1, g.REAL, 3)
    assert a.bond_dims() == b.bond_dims()
    for x, y in zip(a.get_mps(), b.get_mps()):
        assert np.array_equal(x, y)
    a.close()
    b.close()
