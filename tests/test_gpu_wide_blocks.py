"""Parity of the blocked factorisations at the widths a chi = 1024 step runs (GPU vs oracle).

Dense random states carry no conserved charge, so every matrix the engine factorises is one
dense block: the widest schedules of the grouped kernels.
  * an imaginary-time sweep of a 24-site chain through bond dimension 512 splits each
    centre site by a truncated SVD of a dense (2 m) x m block, up to 1024 x 512 and
    512 x 1024 (k_jacobi_groups with a CTA per column pair; R->L moves take the
    conjugate-transposed orientation);
  * the real-time sweep of the same state moves the centre by dense block QRs of the same
    shapes (k_qr_groups, one group of CTAs per block);
  * a Krylov vector of a 14-site chain at cap 128 eigendecomposes dense density matrices of
    up to 256 rows (pivoted Cholesky by CTA groups, then the grouped Jacobi).
FP64 on the device against the oracle: equal bond dimensions, overlap and energy to 1e-10.
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


@pytest.fixture(scope="module")
def wide_state():
    """A right-canonical random state of 24 sites at bond dimension 512 (random isometries):
    every matrix its sweeps factorise keeps s_min / s_max >= 1.7e-9, clear of the 1e-10 rank
    threshold (products of Gaussian tensors give spectra that straddle it, which no threshold
    reading can compare between two implementations)."""
    lat = wl.chain(24)
    W = wl.heisenberg_mpo(lat)
    psi = wl.random_isometric_mps(24, 512, 41)
    assert max(wl.mps_bond_dims(psi)) == 512
    return W, psi


@pytest.mark.parametrize("kind", ["imag", "real"])
def test_sweep_through_dense_512_blocks_matches_oracle(g, wide_state, kind):
    W, psi = wide_state
    st = g.GseTdvp(psi, W, eps=0.0, chi_max=512)
    st.canonicalize(0)
    st.sweep(0.05, g.IMAG if kind == "imag" else g.REAL)
    ref = O.tdvp1_sweep(psi, W, 0.05, kind, 0.0, 512)
    assert st.bond_dims() == wl.mps_bond_dims(ref)
    assert abs(abs(O.mps_overlap(st.get_mps(), ref)) - 1) < 1e-10
    assert abs(st.energy() - O.mpo_expectation(ref, W).real) < 1e-10
    assert abs(st.norm() - 1) < 1e-12
    nfo = st.trunc_stats()
    if kind == "imag":
        assert nfo["svd_max_block"] >= 512           # the 512-column Jacobi schedule ran
    st.close()


def test_krylov_vector_dense_256_row_density_matrices(g):
    lat = wl.chain(14)
    W = wl.heisenberg_mpo(lat)
    psi = O.left_canonicalize(wl.random_mps(14, 64, 42))
    psi[-1] = psi[-1] / np.linalg.norm(psi[-1])
    st = g.GseTdvp(psi, W, tau=0.1, eps_k=1e-12, chi_max=128)
    st.apply_krylov()
    ref = O.krylov_vectors(psi, W, 0.1, 2, 1e-12, 128)[0]
    assert st.bond_dims() == wl.mps_bond_dims(ref)
    assert max(st.bond_dims()) >= 120                 # density matrices of about 2 x 120 rows
    assert abs(abs(O.mps_overlap(st.get_mps(), ref)) - 1) < 1e-10
    st.close()


def test_gse_steps_on_the_ladder_at_cap_128_match_oracle(g):
    """Three whole GSE-TDVP1 steps (Krylov vectors, extension, sweep; real time, k = 3) on the
    rung-coupled 2 x 8 zigzag ladder (w = 8) from a random-isometry state at bond dimension 64
    with chi_max = 128: the first extension doubles the middle bonds to the cap, so the cut of
    the projected density-matrix spectrum (Eq. 6) falls at the cap, and the Krylov vectors are
    compressed at it.  FP64 on the device against the oracle at every step: equal bond
    dimensions, overlap, energy and <S^z_i> to 1e-10."""
    lat = wl.zigzag_ladder(8, 1.0, 1.0)
    W = wl.heisenberg_mpo(lat)
    psi = wl.random_isometric_mps(16, 64, 5)
    p = dict(tau=0.1, k=3, eps_k=1e-8, eps_m=1e-8, chi_max=128, dt=0.1, kind="real", eps=0.0)
    st = g.GseTdvp(psi, W, tau=0.1, eps_k=1e-8, eps_m=1e-8, chi_max=128)
    sz = np.diag([0.5, -0.5]).astype(np.complex128)
    ref = psi
    for _ in range(3):
        st.step(0.1, g.REAL, 3)
        ref = O.gse_tdvp1_step(ref, W, p)
        assert st.bond_dims() == wl.mps_bond_dims(ref)
        assert abs(abs(O.mps_overlap(st.get_mps(), ref)) - 1) < 1e-10
        assert abs(st.energy() - O.mpo_expectation(ref, W).real) < 1e-10
    assert max(st.bond_dims()) == 128
    for i in (0, 5, 8, 15):
        assert abs(st.expect_local(sz, i).real - O.expect_local(ref, sz, i).real) < 1e-10
    st.close()
