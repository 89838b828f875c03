"""Kernel-level parity: one-site contractions on the GPU (through the C ABI)
against the oracle on identical seeded operands.

FP64 results agree to rounding (relative 1e-12, norm-wise).  The split-TF32
tensor-core form is held to relative 1e-5: each product keeps about 22
significant bits (hi + lo, the lo*lo term dropped, |x - hi - lo| <= 2^-22 |x|),
FP32 accumulation adds about 2^-24 sqrt(K) per output, and two GEMMs are
chained, which bounds the norm-wise error near 3e-6 for these shapes.

The BF16 exact-slice forms represent every operand entry to 2^-33 (4 slices)
or 2^-25 (3 slices) of its scaling group's largest magnitude and sum the
leading slice product exactly.  The other products (about 2^-7 of the leading
one) share one FP32 tensor-memory accumulator per 128-deep chunk: 72 (4 slices)
or 40 (3 slices) MMA accumulations, each rounding near 2^-23 of it, leave about
2^-24 of the chunk's magnitude.  Chunks add without loss, so for random operands
the norm-wise error stays near 2^-26..2^-24 (4 slices; measured 1.06e-8 at
m_l = 129, m_r = 127) and near 3e-7 (3 slices): the tests hold them to 5e-8
and 3e-6.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O
from paper_2005_06104_gb300 import workloads as wl

TOL64 = 1e-12
TOL_TC = 1e-5
TOL_BF16X10 = 5e-8
TOL_BF16X6 = 3e-6


@pytest.fixture(scope="module")
def g():
    assert torch.cuda.is_available()
    from paper_2005_06104_gb300 import gse_tdvp
    return gse_tdvp


def _rand(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(shape[-1])


def _dev(*arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


W_LADDER = wl.heisenberg_mpo(wl.zigzag_ladder(6, 1.0, 1.0))
W_CYL = wl.heisenberg_mpo(wl.cylinder_snake(6, 4))
SHAPES = [  # (ml, mr, W site) -- several tiles with ragged tails, the boundary sites, w = 1
    (1, 2, W_LADDER[0]), (2, 4, W_LADDER[1]), (37, 45, W_LADDER[5]), (100, 90, W_LADDER[6]),
    (129, 127, W_LADDER[7]), (96, 160, W_CYL[10]), (64, 1, W_LADDER[-1]),
]


@pytest.mark.parametrize("ml,mr,W", SHAPES, ids=lambda v: str(v) if np.isscalar(v) else "W")
@pytest.mark.parametrize("prec", ["fp64", "tf32x3", "bf16x10", "bf16x6"])
def test_heff_contract_matches_oracle(g, ml, mr, W, prec):
    rng = np.random.default_rng(ml * 1000 + mr)
    L = _rand(rng, ml, W.shape[0], ml)
    R = _rand(rng, mr, W.shape[3], mr)
    x = _rand(rng, ml, W.shape[1], mr)
    Ld, Rd, xd = _dev(L, R, x)
    yd = torch.empty_like(xd)
    g.heff_contract(Ld, W, Rd, xd, yd, precision=PREC[prec](g))
    ref = O.heff_apply(L, W, R, x)
    err = _rel(yd.cpu().numpy(), ref)
    assert err < TOL[prec], err


PREC = {"fp64": lambda g: g.PREC_FP64, "tf32x3": lambda g: g.PREC_TF32X3,
        "bf16x10": lambda g: g.PREC_BF16X10, "bf16x6": lambda g: g.PREC_BF16X6}
TOL = {"fp64": TOL64, "tf32x3": TOL_TC, "bf16x10": TOL_BF16X10, "bf16x6": TOL_BF16X6}


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x10"])
def test_heff_contract_cached_env_operands(g, prec):
    """Calls with one env tag reuse the tensor-core forms of L and R; a new tag rebuilds them."""
    rng = np.random.default_rng(23)
    W = W_CYL[9]
    ml, mr = 70, 90
    L1, L2 = _rand(rng, ml, W.shape[0], ml), _rand(rng, ml, W.shape[0], ml)
    R = _rand(rng, mr, W.shape[3], mr)
    x1, x2 = _rand(rng, ml, 2, mr), _rand(rng, ml, 2, mr)
    L1d, L2d, Rd, x1d, x2d = _dev(L1, L2, R, x1, x2)
    y = torch.empty_like(x1d)
    p = PREC[prec](g)
    g.heff_contract(L1d, W, Rd, x1d, y, p, env_tag=11)
    assert _rel(y.cpu().numpy(), O.heff_apply(L1, W, R, x1)) < TOL[prec]
    g.heff_contract(L1d, W, Rd, x2d, y, p, env_tag=11)  # cached L1, R
    assert _rel(y.cpu().numpy(), O.heff_apply(L1, W, R, x2)) < TOL[prec]
    g.heff_contract(L2d, W, Rd, x2d, y, p, env_tag=12)  # new content, new tag
    assert _rel(y.cpu().numpy(), O.heff_apply(L2, W, R, x2)) < TOL[prec]


@pytest.mark.parametrize("prec", ["bf16x10", "bf16x6"])
def test_heff_bf16_groups_with_wide_range(g, prec):
    """Rows whose entries span many orders of magnitude, a zero row and a zero
    chunk: the fixed-point slices keep every entry to 2^-33 (2^-25) of its
    group's largest magnitude, so the output error stays at that level of the
    output's scale."""
    rng = np.random.default_rng(17)
    W = W_LADDER[6]
    ml, mr = 160, 136
    L = _rand(rng, ml, W.shape[0], ml) * np.exp(rng.uniform(-12, 3, size=(ml, W.shape[0], 1)))
    R = _rand(rng, mr, W.shape[3], mr) * np.exp(rng.uniform(-12, 3, size=(1, W.shape[3], mr)))
    x = _rand(rng, ml, W.shape[1], mr) * np.exp(rng.uniform(-8, 0, size=(ml, 1, 1)))
    L[3] = 0.0
    x[:, :, 5] = 0.0
    L[:, :, 64:] *= 1e-9
    Ld, Rd, xd = _dev(L, R, x)
    yd = torch.empty_like(xd)
    g.heff_contract(Ld, W, Rd, xd, yd, precision=PREC[prec](g))
    ref = O.heff_apply(L, W, R, x)
    assert _rel(yd.cpu().numpy(), ref) < 10 * TOL[prec]
    assert np.all(yd.cpu().numpy()[3] == 0.0)


@pytest.mark.parametrize("ml,mr,w", [(1, 1, 1), (3, 5, 5), (70, 66, 8), (130, 129, 14)])
def test_keff_contract_matches_oracle(g, ml, mr, w):
    rng = np.random.default_rng(ml + 7 * mr)
    L = _rand(rng, ml, w, ml)
    R = _rand(rng, mr, w, mr)
    x = _rand(rng, ml, mr)
    Ld, Rd, xd = _dev(L, R, x)
    yd = torch.empty_like(xd)
    g.keff_contract(Ld, Rd, xd, yd)
    assert _rel(yd.cpu().numpy(), O.keff_apply(L, R, x)) < TOL64


@pytest.mark.parametrize("ml,mr,W", SHAPES, ids=lambda v: str(v) if np.isscalar(v) else "W")
def test_env_updates_match_oracle(g, ml, mr, W):
    rng = np.random.default_rng(3 * ml + mr)
    A = _rand(rng, ml, W.shape[1], mr)
    L = _rand(rng, ml, W.shape[0], ml)
    R = _rand(rng, mr, W.shape[3], mr)
    Ad, Ld, Rd = _dev(A, L, R)
    Lo = torch.empty((mr, W.shape[3], mr), dtype=torch.complex128, device="cuda")
    Ro = torch.empty((ml, W.shape[0], ml), dtype=torch.complex128, device="cuda")
    g.env_contract(0, Ld, W, Ad, Lo)
    g.env_contract(1, Rd, W, Ad, Ro)
    assert _rel(Lo.cpu().numpy(), O.env_left_step(L, A, W)) < TOL64
    assert _rel(Ro.cpu().numpy(), O.env_right_step(R, A, W)) < TOL64




@pytest.mark.parametrize("kind", ["real", "imag"])
@pytest.mark.parametrize("prec", ["fp64", "tf32x3", "bf16x10"])
def test_lanczos_exponential_matches_oracle(g, kind, prec):
    # environments of a random canonical MPS make H_eff Hermitian, as in the sweep
    lat = wl.zigzag_ladder(5, 1.0, 1.0)
    W = wl.heisenberg_mpo(lat)
    psi = O.right_canonicalize(wl.random_mps(lat.n, 24, 4))
    c = 4
    for i in range(c):
        ml, d, mr = psi[i].shape
        U, S, Vh, _ = O.svd_truncate(psi[i].reshape(ml * d, mr))
        psi[i] = U.reshape(ml, d, -1)
        psi[i + 1] = np.tensordot(S[:, None] * Vh, psi[i + 1], axes=([1], [0]))
    Ls, Rs = O.build_envs(psi, W, c)
    x = psi[c]
    delta = 0.05 if kind == "real" else 0.1
    ref, it_ref = O.lanczos_expm(lambda v: O.heff_apply(Ls[c], W[c], Rs[c], v), x, delta, kind)
    Ld, Rd, xd = _dev(Ls[c], Rs[c], x)
    yd = torch.empty_like(xd)
    it = g.expm_contract(Ld, W[c], Rd, xd, yd, delta, kind=g.REAL if kind == "real" else g.IMAG,
                         precision=PREC[prec](g))
    err = _rel(yd.cpu().numpy(), ref)
    if prec == "fp64":
        assert err < 1e-11 and it == it_ref
    elif prec == "bf16x10":
        assert err < TOL_BF16X10 and abs(it - it_ref) <= 1
    else:
        assert err < TOL_TC and abs(it - it_ref) <= 2


def test_lanczos_nonconvergence_is_reported(g):
    rng = np.random.default_rng(9)
    W = W_LADDER[5]
    L = _rand(rng, 30, W.shape[0], 30)
    L = L + L.conj().transpose(2, 1, 0)
    R = _rand(rng, 30, W.shape[3], 30)
    R = R + R.conj().transpose(2, 1, 0)
    x = _rand(rng, 30, 2, 30)
    Ld, Rd, xd = _dev(L, R, x)
    yd = torch.empty_like(xd)
    with pytest.raises(g.TDVPError) as e:
        g.expm_contract(Ld, W, Rd, xd, yd, 5.0, nmax=2)
    assert e.value.status == 4


def test_heff_full_size_sampled(g):
    """chi = 1024, w = 14 (the 4-wide cylinder's widest MPO site): sampled outputs of
    the tensor-core and FP64 applies against the oracle's entry-by-entry definition."""
    W = max(W_CYL, key=lambda w: w.shape[0] * w.shape[3])
    assert W.shape[0] == 14 and W.shape[3] == 14
    m = 1024
    gen = torch.Generator(device="cuda").manual_seed(5)

    def rnd(*shape):
        return torch.complex(torch.randn(*shape, generator=gen, device="cuda", dtype=torch.float64),
                             torch.randn(*shape, generator=gen, device="cuda", dtype=torch.float64)) / np.sqrt(shape[-1])
    Ld, Rd, xd = rnd(m, 14, m), rnd(m, 14, m), rnd(m, 2, m)
    y64 = torch.empty_like(xd)
    ytc = torch.empty_like(xd)
    ybf = torch.empty_like(xd)
    g.heff_contract(Ld, W, Rd, xd, y64, precision=g.PREC_FP64)
    g.heff_contract(Ld, W, Rd, xd, ytc, precision=g.PREC_TF32X3)
    g.heff_contract(Ld, W, Rd, xd, ybf, precision=g.PREC_BF16X10)
    L, R, x = Ld.cpu().numpy(), Rd.cpu().numpy(), xd.cpu().numpy()
    rng = np.random.default_rng(1)
    entries = [(int(rng.integers(m)), int(rng.integers(2)), int(rng.integers(m))) for _ in range(12)]
    entries += [(0, 0, 0), (m - 1, 1, m - 1), (127, 1, 128), (128, 0, 1023)]
    ref = O.heff_apply_entries(L, W, R, x, entries)
    got64 = np.array([y64[a, s, b].item() for a, s, b in entries])
    gottc = np.array([ytc[a, s, b].item() for a, s, b in entries])
    gotbf = np.array([ybf[a, s, b].item() for a, s, b in entries])
    scale = np.linalg.norm(ref) / np.sqrt(len(ref))
    assert np.max(np.abs(got64 - ref)) < 1e-11 * scale
    assert np.max(np.abs(gottc - ref)) < 3e-5 * scale
    assert np.max(np.abs(gotbf - ref)) < 2e-7 * scale
    # the whole output: the GPU forms agree norm-wise
    assert (torch.linalg.norm(ytc - y64) / torch.linalg.norm(y64)).item() < TOL_TC
    assert (torch.linalg.norm(ybf - y64) / torch.linalg.norm(y64)).item() < TOL_BF16X10


@pytest.mark.parametrize("prec", ["fp64", "tf32x3", "bf16x10", "bf16x6"])
def test_keff_apply_precision_forms_through_a_handle(g, prec):
    """tdvp_keff_apply in every precision form (the arithmetic of the sweep's backward bond
    steps) against the oracle's K_eff on the handle's own state: a 16-site rung-coupled zigzag
    ladder (w = 8) at bond dimension 144, centre moved to the middle bond, so both K_eff GEMMs
    (1152 x 144 x 144 and 144 x 144 x 1152) run on the tensor cores in the split forms."""
    lat = wl.zigzag_ladder(8, 1.0, 1.0)
    W = wl.heisenberg_mpo(lat)
    h = g.GseTdvp(wl.random_isometric_mps(16, 144, 4), W, chi_max=256)
    bond = 8
    h.canonicalize(bond)
    mps = h.get_mps()
    Ls, Rs = O.build_envs(mps, W, bond)
    R_incl = O.env_right_step(Rs[bond], mps[bond], W[bond])
    mb = mps[bond].shape[0]
    assert mb == 144
    rng = np.random.default_rng(11)
    x = _rand(rng, mb, mb)
    xd, = _dev(x)
    yd = torch.empty_like(xd)
    code = {"fp64": g.PREC_FP64, "tf32x3": g.PREC_TF32X3, "bf16x10": g.PREC_BF16X10, "bf16x6": g.PREC_BF16X6}[prec]
    tol = {"fp64": TOL64, "tf32x3": TOL_TC, "bf16x10": TOL_BF16X10, "bf16x6": TOL_BF16X6}[prec]
    h.keff_apply(bond, xd, yd, code)
    assert _rel(yd.cpu().numpy(), O.keff_apply(Ls[bond], R_incl, x)) < tol
    h.close()
