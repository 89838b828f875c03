// GSE-TDVP1 engine (Yang & White, arXiv:2005.06104, Sec. I): device-resident
// MPS, MPO and environments; H_eff / K_eff contractions; Lanczos local
// exponentials; the symmetric TDVP1 sweep (Sec. I.C step 3); Krylov vectors
// (1 - i tau H)^l |psi> (Eq. 10, Sec. I.C step 1) and the state-averaged basis
// extension (Eqs. 3, 5-7, Sec. I.C step 2).
#include <algorithm>
#include <cstring>

#include "engine.cuh"

namespace {
constexpr double kRankRtol = 1e-10;     // "SVD without truncation": keep s > 1e-10 s_max
constexpr double kClusterRtol = 1e-8;   // never split a cluster of near-equal weights
constexpr double kEigFloorRtol = 1e-12; // mixed density-matrix eigenvalues <= 1e-12 tr never count
const cplx kOne = {1.0, 0.0};
const cplx kZero = {0.0, 0.0};
const cplx kMinusOne = {-1.0, 0.0};
}  // namespace

// The Krylov density matrices of a precision form whose operands keep about FP32 accuracy
// (BF16X6: 2^-25; TF32X3: about 1e-6) are themselves formed to that accuracy, so their
// eigendecomposition rotates the FP64 Cholesky factor in FP32 (the Krylov vectors only enrich
// the basis, Sec. I.B).  FP64 and BF16X10 (about 1e-8) keep the FP64 rotations.
bool krylov_eig_fp32(int kp) {
  return kp == TDVP_PREC_BF16X6 || kp == TDVP_PREC_TF32X3 || kp == TDVP_PREC_TF32X3_ENV;
}

int keep_count(const std::vector<double>& w, double total, double eps, int cap, double floor_) {
  int n_cand = 0;
  while (n_cand < (int)w.size() && w[n_cand] > floor_) ++n_cand;
  if (n_cand == 0 || cap <= 0) return 0;
  // minimal n with sum(w[n:n_cand]) <= eps * total
  std::vector<double> tail(n_cand + 1, 0.0);
  for (int j = n_cand - 1; j >= 0; --j) tail[j] = tail[j + 1] + w[j];
  const double limit = eps * total;
  int n = n_cand;
  for (int j = 0; j <= n_cand; ++j)
    if (tail[j] <= limit) {
      n = j;
      break;
    }
  auto inside = [&](int j) { return j > 0 && j < n_cand && (w[j - 1] - w[j]) <= kClusterRtol * w[j - 1]; };
  while (inside(n)) ++n;
  if (n > cap) {
    n = cap;
    while (inside(n)) --n;
  }
  return n;
}

namespace {
// Selection functor for SVDs: numerical rank, then optional cutoff/cap on s^2.
struct SvdRule {
  double eps = 0.0;
  int cap = 1 << 30;
  double* discarded = nullptr;
  int operator()(const std::vector<double>& s) const {
    if (s.empty() || !(s[0] > 0.0)) return 0;
    std::vector<double> w(s.size());
    double tot = 0.0;
    for (size_t i = 0; i < s.size(); ++i) {
      w[i] = s[i] * s[i];
      tot += w[i];
    }
    const double fl = (kRankRtol * s[0]) * (kRankRtol * s[0]);
    const int n = keep_count(w, tot, eps, cap, fl);
    if (discarded) {
      double d = 0.0;
      for (size_t i = n; i < w.size(); ++i) d += w[i];
      *discarded += d / tot;
    }
    return n;
  }
};

__global__ void k_apply_op_site(const cplx* __restrict__ op, const cplx* __restrict__ A, int ml, int d,
                                int mr, cplx* __restrict__ out) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)ml * d * mr) return;
  const int b = e % mr;
  const int s = (e / mr) % d;
  const long long a = e / ((long long)mr * d);
  cplx acc = mkc(0.0, 0.0);
  for (int t = 0; t < d; ++t) cfma(acc, op[s * d + t], A[(a * d + t) * mr + b]);
  out[e] = acc;
}

__global__ void k_one(cplx* p) { p[0] = mkc(1.0, 0.0); }

// Right density environment, last stage:
// F[w][a][wb][ab] = sum_{(t,v,tb,vb)} Om[(w,wb),(t,v,tb,vb)] T2[v][a][t][vb][ab][tb],
// Om[(w,wb),(t,v,tb,vb)] = sum_s W[w,s,t,v] conj(W[wb,s,tb,vb]).
// T2 rows (a, t, v, vb), columns (ab, tb); F out as [a][w][wb][ab] (row index a outermost,
// the layout the next site's single GEMM reads)
__global__ void k_omega_stage(const cplx* __restrict__ T2, cplx* __restrict__ F, int ml, int d, int wl, int wr,
                              const int* __restrict__ off, const int* __restrict__ idx,
                              const cplx* __restrict__ val) {
  const int ab = blockIdx.x * blockDim.x + threadIdx.x;
  const int pr = blockIdx.y;  // w * wl + wb
  const long long a = blockIdx.z;
  if (ab >= ml) return;
  cplx acc = mkc(0.0, 0.0);
  for (int e = off[pr]; e < off[pr + 1]; ++e) {
    const int t = idx[4 * e], v = idx[4 * e + 1], tb = idx[4 * e + 2], vb = idx[4 * e + 3];
    const long long o = ((((a * d + t) * wr + v) * wr + vb) * ml + ab) * d + tb;
    cfma(acc, val[e], T2[o]);
  }
  const int w = pr / wl, wb = pr % wl;
  F[((a * wl + w) * wl + wb) * ml + ab] = acc;
}

// Zip-up MPO stage: out[a][w][s][c] = sum_{(v,t)} W[w,s,t,v] in[a][t][v][c]
// (the right grouping of the sparse MPO lists: row s * wl + w holds the (v, t) entries).
__global__ void k_wstage_zip(const cplx* __restrict__ in, cplx* __restrict__ out, int wl, int wr, int d, int C,
                             const int* __restrict__ off, const int* __restrict__ idx,
                             const cplx* __restrict__ val) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int sw = blockIdx.y;
  const long long a = blockIdx.z;
  if (c >= C) return;
  const int s = sw / wl, w = sw % wl;
  cplx acc = mkc(0.0, 0.0);
  for (int e = off[sw]; e < off[sw + 1]; ++e) {
    const int v = idx[2 * e], t = idx[2 * e + 1];
    cfma(acc, val[e], in[((a * d + t) * wr + v) * (long long)C + c]);
  }
  out[((a * wl + w) * d + s) * (long long)C + c] = acc;
}

// out[k][j] = conj(in[j][k]), in: rows x cols
__global__ void k_adjoint(const cplx* __restrict__ in, cplx* __restrict__ out, int rows, int cols) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)rows * cols) return;
  const long long k = e / rows, j = e % rows;  // e indexes out[k][j]
  out[e] = cconj(in[j * cols + k]);
}

// F[v][b][x] from Fp[b][v][x] (x: the wr * m contiguous trailing entries)
__global__ void k_swap_outer(const cplx* __restrict__ Fp, cplx* __restrict__ F, int m, int wr) {
  const long long inner = (long long)wr * m;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)m * wr * inner) return;
  const long long x = e % inner, vb = e / inner;  // vb = v * m + b (destination order)
  const long long v = vb / m, b = vb % m;
  F[e] = Fp[(b * wr + v) * inner + x];
}
}  // namespace

// ============================================================================
// set-up
// ============================================================================
void Engine::init(const tdvp_mps_desc* mps, const tdvp_mpo_desc* mpo, const tdvp_options* o,
                  cudaStream_t s) {
  tdvp_require(mps && mpo, TDVP_ERR_INVALID_ARG, "null descriptor");
  tdvp_require(mps->n_sites >= 1 && mps->n_sites == mpo->n_sites, TDVP_ERR_SHAPE,
               "MPS and MPO lengths differ or are < 1");
  tdvp_require(mps->d >= 1 && mps->d == mpo->d, TDVP_ERR_SHAPE, "physical dimensions differ");
  tdvp_require(mps->bond_dims && mps->sites && mpo->bond_dims && mpo->sites, TDVP_ERR_INVALID_ARG,
               "null arrays in descriptor");
  N = mps->n_sites;
  d = mps->d;
  st = static_cast<cudaStream_t>(s);
  tracer.st = st;
  if (o) opt = *o; else tdvp_default_options(&opt);
  int dev = 0;
  TDVP_CUDA(cudaGetDevice(&dev));
  TDVP_CUDA(cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev));
  blas.init(&pool, sm_count);
  psi.N = N;
  psi.d = d;
  psi.m.assign(mps->bond_dims, mps->bond_dims + N + 1);
  w.assign(mpo->bond_dims, mpo->bond_dims + N + 1);
  tdvp_require(psi.m[0] == 1 && psi.m[N] == 1, TDVP_ERR_SHAPE, "MPS boundary bond dims must be 1");
  tdvp_require(w[0] == 1 && w[N] == 1, TDVP_ERR_SHAPE, "MPO boundary bond dims must be 1");
  for (int i = 0; i <= N; ++i)
    tdvp_require(psi.m[i] >= 1 && w[i] >= 1, TDVP_ERR_SHAPE, "bond dims must be >= 1");
  psi.A.resize(N);
  for (int i = 0; i < N; ++i) {
    tdvp_require(mps->sites[i] != nullptr, TDVP_ERR_INVALID_ARG, "null MPS site pointer");
    const size_t n = (size_t)psi.m[i] * d * psi.m[i + 1];
    psi.A[i].reset(&pool, n);
    TDVP_CUDA(cudaMemcpyAsync(psi.A[i].data(), mps->sites[i], n * sizeof(cplx), cudaMemcpyHostToDevice, st));
  }
  W_host.resize(N);
  Wsp.resize(N);
  for (int i = 0; i < N; ++i) {
    tdvp_require(mpo->sites[i] != nullptr, TDVP_ERR_INVALID_ARG, "null MPO site pointer");
    const size_t n = (size_t)w[i] * d * d * w[i + 1];
    W_host[i].resize(n);
    std::memcpy(W_host[i].data(), mpo->sites[i], n * sizeof(cplx));
    for (const cplx& x : W_host[i])
      tdvp_require(std::isfinite(x.x) && std::isfinite(x.y), TDVP_ERR_NONFINITE, "non-finite MPO entry");
    Wsp[i].build(W_host[i].data(), w[i], w[i + 1], d);
    Wsp[i].upload();
  }
  L.resize(N);
  R.resize(N);
  Lok.assign(N, 0);
  Rok.assign(N, 0);
  scr.pool = &pool;
  lw.init(&pool);
  // left-canonical form with the centre at N-1 (Eq. 1)
  center = 0;
  for (int i = 0; i + 1 < N; ++i) move_right(i, 0.0, 1 << 30, false);
  center = N - 1;
  sync();
}

void Engine::release() {
  for (auto& ws : Wsp) ws.free_device();
  for (auto& ws : Wsp2) ws.free_device();
  lw.release();
  blas.release();
  for (auto& p : ev_pairs) {
    cudaEventDestroy(p.first);
    cudaEventDestroy(p.second);
  }
  for (auto& ev : ev_pool) cudaEventDestroy(ev);
  ev_pairs.clear();
  ev_pool.clear();
  tracer.release();
}

// ============================================================================
// environments
// ============================================================================
void Engine::invalidate_from_site(int i) {
  for (int j = i + 1; j < N; ++j) Lok[j] = 0;  // L[j] uses sites < j
  for (int j = 0; j < i && j < N; ++j) Rok[j] = 0;  // R[j] uses sites > j
  ++env_epoch;
}

void Engine::ensure_L(int i) {
  if (!Lok[0]) {
    L[0].reset(&pool, 1);
    k_one<<<1, 1, 0, st>>>(L[0].data());
    TDVP_CHECK_LAUNCH();
    Lok[0] = 1;
  }
  int j = i;
  while (!Lok[j]) --j;
  for (; j < i; ++j) env_left(j);
}

void Engine::ensure_R(int i) {
  if (!Rok[N - 1]) {
    R[N - 1].reset(&pool, 1);
    k_one<<<1, 1, 0, st>>>(R[N - 1].data());
    TDVP_CHECK_LAUNCH();
    Rok[N - 1] = 1;
  }
  int j = i;
  while (!Rok[j]) ++j;
  for (; j > i; --j) env_right(j);
}

// L[i+1] from L[i] and A[i]; R[i-1] from R[i] and A[i]
void Engine::env_left(int i) {
  PhaseScope ps(tracer, PH_ENV);
  const int ml = psi.m[i], mr = psi.m[i + 1];
  L[i + 1].ensure(&pool, (size_t)mr * w[i + 1] * mr);
  env_left_fp64(st, scr, L[i].data(), Wsp[i], psi.A[i].data(), ml, mr, d, L[i + 1].data(), env_prec);
  Lok[i + 1] = 1;
  ++env_epoch;
}

void Engine::env_right(int i) {
  PhaseScope ps(tracer, PH_ENV);
  const int ml = psi.m[i], mr = psi.m[i + 1];
  R[i - 1].ensure(&pool, (size_t)ml * w[i] * ml);
  env_right_fp64(st, scr, R[i].data(), Wsp[i], psi.A[i].data(), ml, mr, d, R[i - 1].data(), env_prec);
  Rok[i - 1] = 1;
  ++env_epoch;
}

SiteOp Engine::site_op(int i) {
  SiteOp op;
  op.L = L[i].data();
  op.R = R[i].data();
  op.W = &Wsp[i];
  op.ml = psi.m[i];
  op.mr = psi.m[i + 1];
  op.wl = w[i];
  op.wr = w[i + 1];
  op.d = d;
  op.env_key = ((long long)i << 40) ^ env_epoch;
  return op;
}

SiteOp Engine::pair_op(int i) {
  SiteOp op;
  op.L = L[i].data();
  op.R = R[i + 1].data();
  op.W = &Wsp2[i];
  op.ml = psi.m[i];
  op.mr = psi.m[i + 2];
  op.wl = w[i];
  op.wr = w[i + 2];
  op.d = d * d;
  op.env_key = ((long long)(N + i) << 40) ^ env_epoch;  // key space apart from the one-site operators
  return op;
}

// W2[w, (s t), (s' t'), u] = sum_v W_i[w, s, s', v] W_{i+1}[v, t, t', u]: the two-site
// effective Hamiltonian is the one-site one with physical dimension d^2, acting on
// Theta[a][(s t)][b] = sum_k A_i[a][s][k] A_{i+1}[k][t][b] in the one-site layout.
void Engine::build_pair_mpo() {
  if ((int)Wsp2.size() == N - 1) return;
  Wsp2.resize(std::max(N - 1, 0));
  const int D = d * d;
  for (int i = 0; i + 1 < N; ++i) {
    const int wl = w[i], wm = w[i + 1], wr = w[i + 2];
    std::vector<cplx> W2((size_t)wl * D * D * wr, kZero);
    const std::vector<cplx>& A = W_host[i];
    const std::vector<cplx>& B = W_host[i + 1];
    for (int a = 0; a < wl; ++a)
      for (int s = 0; s < d; ++s)
        for (int sp = 0; sp < d; ++sp)
          for (int v = 0; v < wm; ++v) {
            const cplx x = A[((a * d + s) * d + sp) * wm + v];
            if (x.x == 0.0 && x.y == 0.0) continue;
            for (int t = 0; t < d; ++t)
              for (int tp = 0; tp < d; ++tp)
                for (int u = 0; u < wr; ++u) {
                  const cplx y = B[((v * d + t) * d + tp) * wr + u];
                  if (y.x == 0.0 && y.y == 0.0) continue;
                  cplx& e = W2[((a * D + s * d + t) * D + sp * d + tp) * wr + u];
                  e = cadd(e, cmul(x, y));
                }
          }
    Wsp2[i].build(W2.data(), wl, wr, D);
    Wsp2[i].upload();
  }
}

void Engine::heff(int site, const cplx* x, cplx* y, int precision) { apply_op(site_op(site), x, y, precision); }

void Engine::apply_op(const SiteOp& op, const cplx* x, cplx* y, int precision) {
  if (!profile) {
    heff_apply_prec(st, scr, op, x, y, precision);
    return;
  }
  cudaEvent_t a, b;
  if (ev_pool.size() >= 2) {
    a = ev_pool.back();
    ev_pool.pop_back();
    b = ev_pool.back();
    ev_pool.pop_back();
  } else {
    TDVP_CUDA(cudaEventCreate(&a));
    TDVP_CUDA(cudaEventCreate(&b));
  }
  TDVP_CUDA(cudaEventRecord(a, st));
  heff_apply_prec(st, scr, op, x, y, precision);
  TDVP_CUDA(cudaEventRecord(b, st));
  ev_pairs.emplace_back(a, b);
  prof_flops += heff_flops(op);
  prof_count += 1;
}

// ============================================================================
// gauge moves: a block QR / LQ when nothing is cut (R1), else a truncated SVD
// (numerical rank 1e-10 s_max, cutoff eps, cap)
// ============================================================================
void Engine::move_right(int i, double eps, int cap, bool trunc) {
  const int ml = psi.m[i], mr = psi.m[i + 1], mr2 = psi.m[i + 2];
  QrOut qo;
  if (!trunc) qr_blocked(st, &pool, psi.A[i].data(), ml * d, mr, 0, qo);
  if (!trunc && qo.full_rank(kRankRtol)) {  // R1: the QR keeps the numerical rank
    const int r = qo.k;
    DArr nxt(&pool, (size_t)r * d * mr2);
    zgemm(st, OP_N, OP_N, r, d * mr2, mr, kOne, qo.C.data(), mr, psi.A[i + 1].data(), d * mr2, kZero, nxt.data(),
          d * mr2, 1, 0, 0, 0, &pool);
    psi.A[i] = std::move(qo.Q);
    psi.A[i + 1] = std::move(nxt);
    psi.m[i + 1] = r;
    invalidate_from_site(i);
    invalidate_from_site(i + 1);
    return;
  }
  SvdRule rule;
  if (trunc) {
    rule.eps = eps;
    rule.cap = cap;
    rule.discarded = &disc_eps;
  }
  SvdOut sv;
  svd_jacobi(st, &pool, psi.A[i].data(), ml * d, mr, rule, sv, true, false);
  const int r = sv.rank;
  tdvp_require(r >= 1, TDVP_ERR_NONFINITE, "move_right: zero tensor");
  // C = U^+ A = S Vh (r x mr), one FP64 GEMM instead of rotating V in every Jacobi round;
  // A[i+1] <- C A[i+1]
  DArr C(&pool, (size_t)r * mr);
  zgemm(st, OP_C, OP_N, r, mr, ml * d, kOne, sv.U.data(), r, psi.A[i].data(), mr, kZero, C.data(), mr, 1, 0, 0, 0,
        &pool);
  DArr nxt(&pool, (size_t)r * d * mr2);
  zgemm(st, OP_N, OP_N, r, d * mr2, mr, kOne, C.data(), mr, psi.A[i + 1].data(), d * mr2, kZero, nxt.data(),
        d * mr2, 1, 0, 0, 0, &pool);
  psi.A[i] = std::move(sv.U);
  psi.A[i + 1] = std::move(nxt);
  psi.m[i + 1] = r;
  invalidate_from_site(i);
  invalidate_from_site(i + 1);
}

void Engine::move_left(int i, double eps, int cap, bool trunc) {
  const int ml = psi.m[i], mr = psi.m[i + 1], ml0 = psi.m[i - 1];
  QrOut qo;
  if (!trunc) qr_blocked(st, &pool, psi.A[i].data(), ml, d * mr, 1, qo);
  if (!trunc && qo.full_rank(kRankRtol)) {  // R1: the LQ keeps the numerical rank
    const int r = qo.k;
    DArr prv(&pool, (size_t)ml0 * d * r);
    zgemm(st, OP_N, OP_N, ml0 * d, r, ml, kOne, psi.A[i - 1].data(), ml, qo.C.data(), r, kZero, prv.data(), r, 1, 0,
          0, 0, &pool);
    psi.A[i] = std::move(qo.Q);
    psi.A[i - 1] = std::move(prv);
    psi.m[i] = r;
    invalidate_from_site(i);
    invalidate_from_site(i - 1);
    return;
  }
  SvdRule rule;
  if (trunc) {
    rule.eps = eps;
    rule.cap = cap;
    rule.discarded = &disc_eps;
  }
  SvdOut sv;
  svd_jacobi(st, &pool, psi.A[i].data(), ml, d * mr, rule, sv, false, true);
  const int r = sv.rank;
  tdvp_require(r >= 1, TDVP_ERR_NONFINITE, "move_left: zero tensor");
  // C = A Vh^+ = U S (ml x r), one FP64 GEMM instead of rotating U in every Jacobi round
  DArr C(&pool, (size_t)ml * r);
  zgemm(st, OP_N, OP_C, ml, r, d * mr, kOne, psi.A[i].data(), d * mr, sv.Vh.data(), d * mr, kZero, C.data(), r, 1, 0,
        0, 0, &pool);
  DArr prv(&pool, (size_t)ml0 * d * r);
  zgemm(st, OP_N, OP_N, ml0 * d, r, ml, kOne, psi.A[i - 1].data(), ml, C.data(), r, kZero, prv.data(), r, 1, 0, 0, 0, &pool);
  psi.A[i] = std::move(sv.Vh);
  psi.A[i - 1] = std::move(prv);
  psi.m[i] = r;
  invalidate_from_site(i);
  invalidate_from_site(i - 1);
}

void Engine::canonicalize(int c) {
  tdvp_require(c >= 0 && c < N, TDVP_ERR_INVALID_ARG, "site out of range");
  PhaseScope ps(tracer, PH_CANON);
  while (center < c) {
    move_right(center, 0.0, 1 << 30, false);
    ++center;
  }
  while (center > c) {
    move_left(center, 0.0, 1 << 30, false);
    --center;
  }
  // environments are built on demand by their users (sweep, energy, heff): the Krylov
  // step, the extension and the local observables need none
}

// ============================================================================
// Lanczos exponential (full re-orthogonalisation, applied twice)
// ============================================================================
// A step whose Lanczos space reaches lanczos_max without meeting the tolerance is split into
// s = 2, 4, ... 64 equal sub-steps (long-range Hamiltonians have a spectral range of order N^2,
// so one step may need more Krylov vectors than lanczos_max); lanczos_expm reads x before it
// writes out, so the sub-steps run in place.
int Engine::lanczos(const std::function<void(const cplx*, cplx*)>& op, const cplx* x, cplx* out,
                    long long n, double delta, int kind, int slot) {
  int* hint = (slot >= 0 && slot < 4) ? &lanczos_hint[slot] : nullptr;
  int used = 0;
  try {
    for (int s = 1;; s *= 2) {
      try {
        used = 0;
        for (int k = 0; k < s; ++k)
          used += lanczos_expm(st, &pool, blas, lw, op, k == 0 ? x : out, out, n, delta / s, kind, opt.lanczos_tol,
                               opt.lanczos_max, hint);
        break;
      } catch (const TdvpError& e) {
        if (e.status != TDVP_ERR_LANCZOS_NOT_CONVERGED || 2 * s > 64) throw;
      }
    }
  } catch (...) {
    tc_check(st, scr);  // a device timeout explains a failure better than what followed it
    throw;
  }
  tc_check(st, scr);
  lanczos_iters += used;
  lanczos_calls += 1;
  return used;
}

// ============================================================================
// TDVP1 sweep (Sec. I.C step 3): L->R then R->L, each with dt/2
// ============================================================================
void Engine::sweep(double dt, int kind) {
  canonicalize(0);
  const double delta = 0.5 * dt;
  const bool imag = kind == TDVP_IMAG;
  const int prec = opt.precision;
  // the sweep's environments (the initial right ones included) in the precision form
  const int want_env = (prec == TDVP_PREC_TF32X3_ENV) ? TDVP_PREC_TF32X3 : prec_is_bf16(prec) ? prec : TDVP_PREC_FP64;
  if (want_env != TDVP_PREC_FP64)  // FP64 environments left by observables are rebuilt in that form
    for (int j = 0; j < N; ++j) Lok[j] = Rok[j] = 0;
  env_prec = want_env;
  for (int i = 0; i < N; ++i) ensure_R(i);
  ensure_L(0);
  lanczos_iters = lanczos_calls = 0;
  disc_eps = 0.0;
  DArr y;
  auto normalize = [&](cplx* v, long long n) {
    blas.norm2(st, v, n, lw.real + 140);
    scale_by_inv_sqrt(st, v, v, lw.real + 140, n);
  };
  auto evolve_site = [&](int i) {
    const long long n = (long long)psi.m[i] * d * psi.m[i + 1];
    y.ensure(&pool, n);
    PhaseScope ps(tracer, PH_LANCZOS_SITE);
    lanczos([&](const cplx* a, cplx* b) { heff(i, a, b, prec); }, psi.A[i].data(), y.data(), n, delta,
            kind, 0);
    if (imag) normalize(y.data(), n);
    TDVP_CUDA(cudaMemcpyAsync(psi.A[i].data(), y.data(), n * sizeof(cplx), cudaMemcpyDeviceToDevice, st));
  };
  for (int i = 0; i < N; ++i) {
    evolve_site(i);
    if (i == N - 1) break;
    const int ml = psi.m[i], mold = psi.m[i + 1], mr2 = psi.m[i + 2];
    DArr C;  // A = Q C
    int r = 0;
    {
      PhaseScope ps(tracer, PH_SVD);
      QrOut qo;
      if (!imag) qr_blocked(st, &pool, psi.A[i].data(), ml * d, mold, 0, qo);
      if (imag || !qo.full_rank(kRankRtol)) {  // SVD: Q = U, C = U^+ A = S Vh
        SvdRule rule;
        if (imag) {
          rule.eps = opt.eps;
          rule.cap = opt.chi_max;
          rule.discarded = &disc_eps;
        }
        SvdOut sv;
        svd_jacobi(st, &pool, psi.A[i].data(), ml * d, mold, rule, sv, true, false);
        r = sv.rank;
        tdvp_require(r >= 1, TDVP_ERR_NONFINITE, "sweep: zero site tensor");
        C.reset(&pool, (size_t)r * mold);
        zgemm(st, OP_C, OP_N, r, mold, ml * d, kOne, sv.U.data(), r, psi.A[i].data(), mold, kZero, C.data(), mold,
              1, 0, 0, 0, &pool);
        psi.A[i] = std::move(sv.U);
      } else {  // real time cuts nothing: block QR of full numerical rank (R1)
        r = qo.k;
        C = std::move(qo.C);
        psi.A[i] = std::move(qo.Q);
      }
    }
    psi.m[i + 1] = r;  // L[i+1] is r x w x r, R[i] still mold x w x mold
    env_left(i);
    DArr C2(&pool, (size_t)r * mold);
    const cplx* Lb = L[i + 1].data();
    const cplx* Rb = R[i].data();
    const int wb = w[i + 1];
    {
      PhaseScope ps(tracer, PH_LANCZOS_BOND);
      lanczos([&](const cplx* a, cplx* b) { keff_fp64(st, scr, Lb, r, Rb, mold, wb, a, b, prec); }, C.data(),
              C2.data(), (long long)r * mold, -delta, kind, 1);
    }
    if (imag) normalize(C2.data(), (long long)r * mold);
    DArr nxt(&pool, (size_t)r * d * mr2);
    zgemm(st, OP_N, OP_N, r, d * mr2, mold, kOne, C2.data(), mold, psi.A[i + 1].data(), d * mr2, kZero,
          nxt.data(), d * mr2, 1, 0, 0, 0, &pool);
    psi.A[i + 1] = std::move(nxt);
    center = i + 1;
    for (int j = i + 2; j < N; ++j) Lok[j] = 0;
  }
  for (int i = N - 1; i >= 0; --i) {
    evolve_site(i);
    if (i == 0) break;
    const int mold = psi.m[i], mr = psi.m[i + 1], ml0 = psi.m[i - 1];
    DArr C;  // A = C Q
    int r = 0;
    {
      PhaseScope ps(tracer, PH_SVD);
      QrOut qo;
      if (!imag) qr_blocked(st, &pool, psi.A[i].data(), mold, d * mr, 1, qo);
      if (imag || !qo.full_rank(kRankRtol)) {  // SVD: Q = Vh, C = A Vh^+ = U S
        SvdRule rule;
        if (imag) {
          rule.eps = opt.eps;
          rule.cap = opt.chi_max;
          rule.discarded = &disc_eps;
        }
        SvdOut sv;
        svd_jacobi(st, &pool, psi.A[i].data(), mold, d * mr, rule, sv, false, true);
        r = sv.rank;
        tdvp_require(r >= 1, TDVP_ERR_NONFINITE, "sweep: zero site tensor");
        C.reset(&pool, (size_t)mold * r);
        zgemm(st, OP_N, OP_C, mold, r, d * mr, kOne, psi.A[i].data(), d * mr, sv.Vh.data(), d * mr, kZero, C.data(),
              r, 1, 0, 0, 0, &pool);
        psi.A[i] = std::move(sv.Vh);
      } else {  // real time cuts nothing: block LQ of full numerical rank (R1)
        r = qo.k;
        C = std::move(qo.C);
        psi.A[i] = std::move(qo.Q);
      }
    }
    psi.m[i] = r;
    env_right(i);  // R[i-1]: r x w x r
    DArr C2(&pool, (size_t)mold * r);
    const cplx* Lb = L[i].data();
    const cplx* Rb = R[i - 1].data();
    const int wb = w[i];
    {
      PhaseScope ps(tracer, PH_LANCZOS_BOND);
      lanczos([&](const cplx* a, cplx* b) { keff_fp64(st, scr, Lb, mold, Rb, r, wb, a, b, prec); }, C.data(),
              C2.data(), (long long)mold * r, -delta, kind, 1);
    }
    if (imag) normalize(C2.data(), (long long)mold * r);
    DArr prv(&pool, (size_t)ml0 * d * r);
    zgemm(st, OP_N, OP_N, ml0 * d, r, mold, kOne, psi.A[i - 1].data(), mold, C2.data(), r, kZero, prv.data(),
          r, 1, 0, 0, 0, &pool);
    psi.A[i - 1] = std::move(prv);
    center = i - 1;
    for (int j = 0; j < i - 1; ++j) Rok[j] = 0;
    for (int j = i; j < N; ++j) Lok[j] = 0;
  }
  center = 0;
  for (int j = 1; j < N; ++j) Lok[j] = 0;
  if (env_prec != TDVP_PREC_FP64)  // observables always see FP64 environments
    for (int j = 0; j < N; ++j) Lok[j] = Rok[j] = 0;
  env_prec = TDVP_PREC_FP64;
  sync();
}

// ============================================================================
// Two-site TDVP (TDVP2): the conventional integrator GSE-TDVP1 is compared with
// (Introduction; Sec. I.C).  Per bond, the two-site centre Theta = A_i A_{i+1} is
// evolved by dt/2 under the two-site H_eff, split by a truncated SVD (cutoff eps and
// cap chi_max in real and imaginary time), and the new one-site centre is evolved
// back by dt/2 under the one-site H_eff, except at the last bond of a half-sweep.
// ============================================================================
void Engine::sweep2(double dt, int kind) {
  tdvp_require(N >= 2, TDVP_ERR_SHAPE, "TDVP2 needs at least two sites");
  build_pair_mpo();
  canonicalize(0);
  const double delta = 0.5 * dt;
  const bool imag = kind == TDVP_IMAG;
  const int prec = opt.precision;
  const int want_env = (prec == TDVP_PREC_TF32X3_ENV) ? TDVP_PREC_TF32X3 : prec_is_bf16(prec) ? prec : TDVP_PREC_FP64;
  if (want_env != TDVP_PREC_FP64)
    for (int j = 0; j < N; ++j) Lok[j] = Rok[j] = 0;
  env_prec = want_env;
  for (int i = 0; i < N; ++i) ensure_R(i);
  ensure_L(0);
  lanczos_iters = lanczos_calls = 0;
  disc_eps = 0.0;
  SvdRule rule;
  rule.eps = opt.eps;
  rule.cap = opt.chi_max;
  rule.discarded = &disc_eps;
  DArr theta, y;
  auto normalize = [&](cplx* v, long long n) {
    blas.norm2(st, v, n, lw.real + 140);
    scale_by_inv_sqrt(st, v, v, lw.real + 140, n);
  };
  // y <- exp(-i delta H_eff^(2)) A_i A_{i+1}, then its SVD as (m_i d) x (d m_{i+2}); only the
  // factor that becomes a site tensor (U left to right, Vh right to left) is formed, the
  // centre is then a GEMM with y
  auto evolve_split = [&](int i, SvdOut& sv, bool left_to_right) {
    const int ml = psi.m[i], m = psi.m[i + 1], mr = psi.m[i + 2];
    const long long n = (long long)ml * d * d * mr;
    theta.ensure(&pool, n);
    y.ensure(&pool, n);
    zgemm(st, OP_N, OP_N, ml * d, d * mr, m, kOne, psi.A[i].data(), m, psi.A[i + 1].data(), d * mr, kZero,
          theta.data(), d * mr, 1, 0, 0, 0, &pool);
    const SiteOp op = pair_op(i);
    {
      PhaseScope ps(tracer, PH_LANCZOS_SITE);
      lanczos([&](const cplx* a, cplx* b) { apply_op(op, a, b, prec); }, theta.data(), y.data(), n, delta, kind,
              2);
    }
    if (imag) normalize(y.data(), n);
    PhaseScope ps(tracer, PH_SVD);
    svd_jacobi(st, &pool, y.data(), ml * d, d * mr, rule, sv, left_to_right, !left_to_right);
    tdvp_require(sv.rank >= 1, TDVP_ERR_NONFINITE, "sweep2: zero two-site tensor");
  };
  // C <- exp(+i delta H_eff^(1)) C on site j (the backward step)
  auto evolve_back = [&](int j, DArr& C) {
    const long long n = (long long)psi.m[j] * d * psi.m[j + 1];
    DArr out(&pool, n);
    {
      PhaseScope ps(tracer, PH_LANCZOS_BOND);
      lanczos([&](const cplx* a, cplx* b) { heff(j, a, b, prec); }, C.data(), out.data(), n, -delta, kind, 3);
    }
    if (imag) normalize(out.data(), n);
    C = std::move(out);
  };
  for (int i = 0; i + 1 < N; ++i) {
    const int mr = psi.m[i + 2];
    SvdOut sv;
    evolve_split(i, sv, true);
    const int r = sv.rank;
    const int ml = psi.m[i];
    DArr C(&pool, (size_t)r * d * mr);  // U^+ Theta = S Vh: the centre on site i+1
    zgemm(st, OP_C, OP_N, r, d * mr, ml * d, kOne, sv.U.data(), r, y.data(), d * mr, kZero, C.data(), d * mr, 1, 0,
          0, 0, &pool);
    psi.A[i] = std::move(sv.U);
    psi.m[i + 1] = r;
    env_left(i);  // L[i+1]
    for (int j = 0; j <= i; ++j) Rok[j] = 0;  // R[j] read site i+1
    if (i + 2 < N) evolve_back(i + 1, C);
    psi.A[i + 1] = std::move(C);
    center = i + 1;
    for (int j = i + 2; j < N; ++j) Lok[j] = 0;
  }
  for (int i = N - 2; i >= 0; --i) {
    const int ml = psi.m[i];
    SvdOut sv;
    evolve_split(i, sv, false);
    const int r = sv.rank;
    const int mr = psi.m[i + 2];
    DArr C(&pool, (size_t)ml * d * r);  // Theta Vh^+ = U S: the centre on site i
    zgemm(st, OP_N, OP_C, ml * d, r, d * mr, kOne, y.data(), d * mr, sv.Vh.data(), d * mr, kZero, C.data(), r, 1, 0,
          0, 0, &pool);
    psi.A[i + 1] = std::move(sv.Vh);
    psi.m[i + 1] = r;
    env_right(i + 1);  // R[i]
    if (i > 0) evolve_back(i, C);
    psi.A[i] = std::move(C);
    center = i;
    for (int j = 0; j < i; ++j) Rok[j] = 0;
    for (int j = i + 1; j < N; ++j) Lok[j] = 0;
  }
  center = 0;
  for (int j = 1; j < N; ++j) Lok[j] = 0;
  if (env_prec != TDVP_PREC_FP64)
    for (int j = 0; j < N; ++j) Lok[j] = Rok[j] = 0;
  env_prec = TDVP_PREC_FP64;
  ++env_epoch;
  sync();
}

// ============================================================================
// Krylov vectors and basis extension (Sec. I.A-I.C, steps 1-2)
// ============================================================================
namespace {
// MPO of 1 - i tau H with the bond dimension of H's MPO.  In start/done form
// every term enters the "done" channel exactly once, so scaling the entries
// W[x, done] (x != done) by -i tau scales each term once; the identity enters
// as (1/N) 1 on each site's start -> done entry.
std::vector<cplx> one_minus_itau_h_site(const std::vector<cplx>& W, int i, int N, int wl, int wr, int d,
                                        double tau_re, double tau_im) {
  std::vector<cplx> out = W;
  const cplx c = mkc(tau_im, -tau_re);  // -i tau
  const int done_r = wr - 1;
  const int done_l = i > 0 ? wl - 1 : -1;
  for (int x = 0; x < wl; ++x) {
    if (x == done_l) continue;
    for (int s = 0; s < d; ++s)
      for (int t = 0; t < d; ++t) {
        cplx& e = out[((x * d + s) * d + t) * wr + done_r];
        e = cmul(c, e);
      }
  }
  for (int s = 0; s < d; ++s) out[((0 * d + s) * d + s) * wr + done_r].x += 1.0 / N;
  return out;
}
}  // namespace

void Engine::build_krylov_op(KrylovOp& kop) {
  kop.Wsp.resize(N);
  kop.om_off.resize(N);
  kop.om_idx.resize(N);
  kop.om_val.resize(N);
  for (int i = 0; i < N; ++i) {
    const int wl = w[i], wr = w[i + 1];
    auto h = one_minus_itau_h_site(W_host[i], i, N, wl, wr, d, opt.tau_re, opt.tau_im);
    kop.Wsp[i].build(h.data(), wl, wr, d);
    kop.Wsp[i].upload();
    // Om[(w,wb),(t,v,tb,vb)] = sum_s W[w,s,t,v] conj(W[wb,s,tb,vb]), kept where nonzero
    std::vector<int> off(wl * wl + 1, 0), idx;
    std::vector<cplx> val;
    auto at = [&](int ww, int s_, int t, int v) { return h[((ww * d + s_) * d + t) * wr + v]; };
    for (int ww = 0; ww < wl; ++ww)
      for (int wb = 0; wb < wl; ++wb) {
        for (int t = 0; t < d; ++t)
          for (int v = 0; v < wr; ++v)
            for (int tb = 0; tb < d; ++tb)
              for (int vb = 0; vb < wr; ++vb) {
                cplx acc = mkc(0.0, 0.0);
                for (int s_ = 0; s_ < d; ++s_) cfma_conj(acc, at(wb, s_, tb, vb), at(ww, s_, t, v));
                if (acc.x != 0.0 || acc.y != 0.0) {
                  idx.insert(idx.end(), {t, v, tb, vb});
                  val.push_back(acc);
                }
              }
        off[ww * wl + wb + 1] = (int)val.size();
      }
    auto up = [&](auto& vec, auto** dst) {
      using T = typename std::remove_reference<decltype(vec)>::type::value_type;
      TDVP_CUDA(cudaMalloc((void**)dst, std::max<size_t>(1, vec.size()) * sizeof(T)));
      if (!vec.empty())
        TDVP_CUDA(cudaMemcpy(*dst, vec.data(), vec.size() * sizeof(T), cudaMemcpyHostToDevice));
    };
    up(off, &kop.om_off[i]);
    up(idx, &kop.om_idx[i]);
    up(val, &kop.om_val[i]);
  }
}

void KrylovOp::release() {
  for (auto& ws : Wsp) ws.free_device();
  for (auto* p : om_off) cudaFree(p);
  for (auto* p : om_idx) cudaFree(p);
  for (auto* p : om_val) cudaFree(p);
  om_off.clear();
  om_idx.clear();
  om_val.clear();
  Wsp.clear();
}

// One Krylov vector by the density-matrix approach (Sec. I.B): out = (1 - i tau H) src
// compressed left to right with cutoff eps_k and cap chi_max, then normalised.
// R->L: right density environments F_i of (W src)(W src)^+ over sites > i, held as
// [b][v][vb][bb] (one GEMM per site reads them) and reordered to [v][b][vb][bb] when read.
// L->R: X[at][w][a] = <compressed left | exact left>; at site i
//   G[(at,s),(v,b)] = sum W[w,s,t,v] X[at,w,a] A[a,t,b],  rho = G F_i G^+ (size d m~),
//   its leading eigenvectors are the new left-orthonormal tensor, X <- U^+ G.
// This reaches, up to ties, the state of exact application followed by a
// right-canonical sweep and left-to-right SVD truncation.
void Engine::krylov_apply(const KrylovOp& kop, const MpsDev& src, MpsDev& out) {
  if (krylov_method == 1) {
    krylov_zipup(kop, src, out);
    return;
  }
  const cplx one = mkc(1.0, 0.0), zero = mkc(0.0, 0.0);
  // the Krylov vectors only enrich the basis (the state itself is kept exactly by the
  // extension), so the precision form may build them on the tensor cores
  const int kp = kprec();
  // Right density environments F[j] (sites > j), (w_{j+1} m_{j+1})^2 entries each, are built
  // right to left and read left to right, once each.  When all of them exceed the memory
  // budget only every K-th (K = ceil(sqrt(N))) stays resident; the others are rebuilt from
  // the next resident one when the left-to-right pass reaches their segment.  The rebuild
  // runs the same launches on the same inputs, so the results are identical.
  std::vector<DArr> F(N);
  F[N - 1].reset(&pool, 1);
  k_one<<<1, 1, 0, st>>>(F[N - 1].data());
  TDVP_CHECK_LAUNCH();
  double f_total = 0.0, f_max = 0.0, t_max = 0.0;
  for (int j = 0; j + 1 < N; ++j) {
    const double f = (double)DevicePool::size_class(sizeof(cplx) * (size_t)w[j + 1] * src.m[j + 1] * w[j + 1] *
                                                    src.m[j + 1]);
    f_total += f;
    f_max = std::max(f_max, f);
  }
  for (int i = 1; i < N; ++i) {  // the two GEMM intermediates of step_F
    const size_t t1 = sizeof(cplx) * (size_t)w[i + 1] * src.m[i] * d * w[i + 1] * src.m[i + 1];
    const size_t t2 = sizeof(cplx) * (size_t)w[i + 1] * src.m[i] * d * w[i + 1] * src.m[i] * d;
    t_max = std::max(t_max, (double)DevicePool::size_class(t1) + (double)DevicePool::size_class(t2));
  }
  double budget = krylov_mem_budget;
  if (!(budget > 0.0)) {
    // what the device has left (free plus this engine's cached blocks), less the GEMM
    // intermediates, the operand slices and the reordered copy of the largest environment, and
    // 16 GiB for everything else the pass allocates
    size_t fr = 0, tot = 0;
    TDVP_CUDA(cudaMemGetInfo(&fr, &tot));
    budget = (double)fr + (double)pool.cached_bytes() - t_max - 3.0 * f_max - 16.0 * (1ull << 30);
  }
  const int seg = f_total <= budget ? 1 : std::max(2, (int)std::ceil(std::sqrt((double)N)));
  krylov_env_segment = seg;
  auto resident = [&](int j) { return seg == 1 || j == N - 1 || j % seg == 0; };
  DArr T1, T2;
  // F[i-1] from F[i] and site i
  auto step_F = [&](int i) {
    PhaseScope ps(tracer, PH_KRYLOV_RENV);
    const int ml = src.m[i], m = src.m[i + 1], wl = w[i], wr = w[i + 1];
    const cplx* A = src.A[i].data();
    T1.ensure(&pool, (size_t)wr * ml * d * wr * m);
    // F[i] is held as [b][v][vb][bb]: one GEMM over all channels,
    // T1[(a,t)][(v,vb,bb)] = sum_b A[(a,t),b] F[b][(v,vb,bb)]
    zgemm_prec(st, scr, kp, OP_N, OP_N, ml * d, wr * wr * m, m, A, m, F[i].data(), (long long)wr * wr * m,
               T1.data(), (long long)wr * wr * m);
    // T2[(a,t,v,vb),(ab,tb)] = sum_bb T1[(a,t,v,vb),bb] conj(A[(ab,tb),bb])
    T2.ensure(&pool, (size_t)wr * ml * d * wr * ml * d);
    zgemm_prec(st, scr, kp, OP_N, OP_C, wr * ml * d * wr, ml * d, m, T1.data(), m, A, m, T2.data(), ml * d);
    F[i - 1].reset(&pool, (size_t)wl * ml * wl * ml);
    tdvp_require(ml <= 65535, TDVP_ERR_INVALID_ARG, "krylov: bond too large");
    dim3 g(ceil_div(ml, 128), wl * wl, ml);
    k_omega_stage<<<g, 128, 0, st>>>(T2.data(), F[i - 1].data(), ml, d, wl, wr, kop.om_off[i], kop.om_idx[i],
                                      kop.om_val[i]);
    TDVP_CHECK_LAUNCH();
  };
  for (int i = N - 1; i >= 1; --i) {
    step_F(i);
    if (!resident(i)) F[i].release();
  }
  T1.release();
  T2.release();
  // makes F[i] resident again: rebuilds the segment below the next resident environment
  auto need_F = [&](int i) {
    if (F[i].size() > 0) return;
    int c = i + 1;
    while (!resident(c)) ++c;
    for (int j = c; j > i; --j) step_F(j);
    T1.release();
    T2.release();
  };
  out.N = N;
  out.d = d;
  out.m.assign(N + 1, 1);
  out.A.clear();
  out.A.resize(N);
  DArr X(&pool, 1), Y1, G, H1, rho;
  k_one<<<1, 1, 0, st>>>(X.data());
  TDVP_CHECK_LAUNCH();
  int mt = 1;
  for (int i = 0; i < N; ++i) {
    const int ml = src.m[i], mr = src.m[i + 1], wl = w[i], wr = w[i + 1];
    Y1.ensure(&pool, (size_t)mt * wl * d * mr);
    zgemm_prec(st, scr, kp, OP_N, OP_N, mt * wl, d * mr, ml, X.data(), ml, src.A[i].data(), d * mr, Y1.data(), d * mr);
    G.ensure(&pool, (size_t)mt * d * wr * mr);
    wstage_left(st, kop.Wsp[i], Y1.data(), G.data(), mt, mr);  // G[at][s][v][b]
    if (i == N - 1) {
      out.A[i].reset(&pool, (size_t)mt * d);
      TDVP_CUDA(cudaMemcpyAsync(out.A[i].data(), G.data(), sizeof(cplx) * mt * d, cudaMemcpyDeviceToDevice, st));
      out.m[i] = mt;
      break;
    }
    const int n = mt * d, K = wr * mr;
    H1.ensure(&pool, (size_t)n * K);
    need_F(i);
    {
      // the right density environment in the row order of G's columns: [v][b][vb][bb]
      DArr Fv(&pool, (size_t)K * K);
      const long long ne = (long long)K * K;
      k_swap_outer<<<ceil_div(ne, 256), 256, 0, st>>>(F[i].data(), Fv.data(), mr, wr);
      TDVP_CHECK_LAUNCH();
      F[i] = std::move(Fv);
    }
    zgemm_prec(st, scr, kp, OP_N, OP_N, n, K, K, G.data(), K, F[i].data(), K, H1.data(), K);
    rho.ensure(&pool, (size_t)n * n);
    zgemm_prec(st, scr, kp, OP_N, OP_C, n, n, K, H1.data(), K, G.data(), K, rho.data(), n);
    F[i].release();
    // eigendecomposition of the Hermitian PSD rho: Jacobi SVD of its pivoted Cholesky factor
    const double eps_k = opt.eps_k;
    const int cap = opt.chi_max;
    double* disc = &disc_k;
    auto rule = [eps_k, cap, disc](const std::vector<double>& ev) -> int {
      double tot = 0.0;
      for (double v : ev) tot += v;
      if (!(tot > 0.0)) return 0;
      const int nk = keep_count(ev, tot, eps_k, cap, 1e-14 * ev[0]);
      double ds = 0.0;
      for (size_t q = nk; q < ev.size(); ++q) ds += ev[q];
      *disc += ds / tot;
      return nk;
    };
    SvdOut sv;
    {
      PhaseScope ps(tracer, PH_KRYLOV_EIG);
      eig_psd_jacobi(st, &pool, rho.data(), n, rule, sv, krylov_eig_fp32(kp));
    }
    const int keep = std::max(1, sv.rank);
    tdvp_require(sv.rank >= 1, TDVP_ERR_NONFINITE, "krylov: zero density matrix");
    // X <- U^+ G  : [keep][v][b]
    DArr Xn(&pool, (size_t)keep * K);
    zgemm_prec(st, scr, kp, OP_C, OP_N, keep, K, n, sv.U.data(), keep, G.data(), K, Xn.data(), K);
    out.A[i] = std::move(sv.U);  // (mt d) x keep  = [at][s][new]
    out.m[i] = mt;
    out.m[i + 1] = keep;
    X = std::move(Xn);
    mt = keep;
  }
  out.m[N] = 1;
  const long long n = (long long)out.m[N - 1] * d;
  blas.norm2(st, out.A[N - 1].data(), n, lw.real + 150);
  scale_by_inv_sqrt(st, out.A[N - 1].data(), out.A[N - 1].data(), lw.real + 150, n);
}

// Zip-up application of 1 - i tau H (the alternative to the density-matrix algorithm that
// needs no right density environments).  The source is left-canonical with its centre at
// N-1.  Right to left, each site is contracted with the MPO and the carry from the right,
// M[(a,w)][(s,r)]; its Gram matrix M^+ M gives the right singular vectors V (Hermitian PSD
// eigendecomposition) under the relaxed cutoff 0.1 eps_k and the cap chi_max.  The rows of
// V^+ become right-orthonormal site tensors and M V = U S is the next carry.  One
// left-to-right compression with eps_k and chi_max follows; the result is normalised,
// left-canonical with its centre at N-1.
void Engine::krylov_zipup(const KrylovOp& kop, const MpsDev& src, MpsDev& out) {
  const int kp = kprec();
  const double eps_k = opt.eps_k;
  const int cap = opt.chi_max;
  MpsDev t;
  t.N = N;
  t.d = d;
  t.m.assign(N + 1, 1);
  t.A.resize(N);
  DArr X(&pool, 1), T1, M, rho;
  k_one<<<1, 1, 0, st>>>(X.data());
  TDVP_CHECK_LAUNCH();
  int rt = 1;  // carry X[b][v][r]: src.m[i+1] x w[i+1] x rt
  for (int i = N - 1; i >= 0; --i) {
    const int ml = src.m[i], mr = src.m[i + 1], wl = w[i], wr = w[i + 1];
    // T1[(a,t)][(v,r)] = sum_b A[(a,t), b] X[b][(v,r)]
    T1.ensure(&pool, (size_t)ml * d * wr * rt);
    zgemm_prec(st, scr, kp, OP_N, OP_N, ml * d, wr * rt, mr, src.A[i].data(), mr, X.data(), (long long)wr * rt,
               T1.data(), (long long)wr * rt);
    // M[(a,w)][(s,r)] = sum_{(v,t)} W[w,s,t,v] T1[a][t][v][r]
    M.ensure(&pool, (size_t)ml * wl * d * rt);
    {
      const WSparse& ws = kop.Wsp[i];
      tdvp_require(ml <= 65535, TDVP_ERR_INVALID_ARG, "zip-up: bond too large");
      dim3 g(ceil_div(rt, 128), d * wl, ml);
      k_wstage_zip<<<g, 128, 0, st>>>(T1.data(), M.data(), wl, wr, d, rt, ws.d_r_off, ws.d_r_idx, ws.d_r_val);
      TDVP_CHECK_LAUNCH();
    }
    const int n = d * rt, K = ml * wl;
    if (i == 0) {  // K = 1: M is the centre tensor (1, d, rt)
      t.A[0].reset(&pool, (size_t)n);
      TDVP_CUDA(cudaMemcpyAsync(t.A[0].data(), M.data(), sizeof(cplx) * n, cudaMemcpyDeviceToDevice, st));
      t.m[1] = rt;
      break;
    }
    rho.ensure(&pool, (size_t)n * n);
    zgemm_prec(st, scr, kp, OP_C, OP_N, n, n, K, M.data(), n, M.data(), n, rho.data(), n);
    auto rule = [eps_k, cap](const std::vector<double>& ev) -> int {
      double tot = 0.0;
      for (double v : ev) tot += v;
      if (!(tot > 0.0)) return 0;
      return keep_count(ev, tot, 0.1 * eps_k, cap, 1e-14 * ev[0]);
    };
    SvdOut sv;
    {
      PhaseScope ps(tracer, PH_KRYLOV_EIG);
      eig_psd_jacobi(st, &pool, rho.data(), n, rule, sv, krylov_eig_fp32(kp));
    }
    const int keep = sv.rank;
    tdvp_require(keep >= 1, TDVP_ERR_NONFINITE, "zip-up: zero site");
    // site tensor V^+ (keep x (s, r)); next carry M V ((a, w) x keep) = [b][v][r] of site i-1
    t.A[i].reset(&pool, (size_t)keep * n);
    k_adjoint<<<ceil_div((long long)keep * n, 256), 256, 0, st>>>(sv.U.data(), t.A[i].data(), n, keep);
    TDVP_CHECK_LAUNCH();
    DArr Xn(&pool, (size_t)K * keep);
    zgemm_prec(st, scr, kp, OP_N, OP_N, K, keep, n, M.data(), n, sv.U.data(), keep, Xn.data(), keep);
    X = std::move(Xn);
    t.m[i] = keep;
    t.m[i + 1] = rt;
    rt = keep;
  }
  T1.release();
  M.release();
  rho.release();
  X.release();
  // left-to-right compression with eps_k and chi_max (the centre moves by U^+ A)
  SvdRule crule;
  crule.eps = eps_k;
  crule.cap = cap;
  crule.discarded = &disc_k;
  for (int i = 0; i + 1 < N; ++i) {
    const int ml = t.m[i], mr = t.m[i + 1], mr2 = t.m[i + 2];
    SvdOut sv;
    svd_jacobi(st, &pool, t.A[i].data(), ml * d, mr, crule, sv, true, false);
    const int r = sv.rank;
    tdvp_require(r >= 1, TDVP_ERR_NONFINITE, "zip-up: zero tensor in the compression");
    DArr C(&pool, (size_t)r * mr);
    zgemm(st, OP_C, OP_N, r, mr, ml * d, kOne, sv.U.data(), r, t.A[i].data(), mr, kZero, C.data(), mr, 1, 0, 0, 0,
          &pool);
    DArr nxt(&pool, (size_t)r * d * mr2);
    zgemm(st, OP_N, OP_N, r, d * mr2, mr, kOne, C.data(), mr, t.A[i + 1].data(), d * mr2, kZero, nxt.data(),
          d * mr2, 1, 0, 0, 0, &pool);
    t.A[i] = std::move(sv.U);
    t.A[i + 1] = std::move(nxt);
    t.m[i + 1] = r;
  }
  const long long n_last = (long long)t.m[N - 1] * d;
  blas.norm2(st, t.A[N - 1].data(), n_last, lw.real + 150);
  scale_by_inv_sqrt(st, t.A[N - 1].data(), t.A[N - 1].data(), lw.real + 150, n_last);
  out = std::move(t);
}

void Engine::expand_basis(int k, const double* weights) {
  tdvp_require(k >= 1 && k <= 16, TDVP_ERR_INVALID_ARG, "krylov order k must be in 1..16");
  disc_k = disc_m = 0.0;
  added_states = 0;
  canonicalize(N - 1);  // left-canonical, centre at N-1 (Eq. 1)
  if (k == 1) {
    canonicalize(0);
    return;
  }
  std::vector<double> wts(k - 1, 1.0);
  if (weights)
    for (int l = 0; l < k - 1; ++l) {
      tdvp_require(std::isfinite(weights[l]) && weights[l] >= 0.0, TDVP_ERR_INVALID_ARG,
                   "weights must be finite and >= 0");
      wts[l] = weights[l];
    }
  // ---- step 1: |psi~_l> = (1 - i tau H)^l |psi>, compressed (eps_k, chi_max), normalised
  KrylovOp kop;
  build_krylov_op(kop);
  std::vector<MpsDev> phis(k - 1);
  {
    PhaseScope ps(tracer, PH_KRYLOV);
    for (int l = 0; l < k - 1; ++l) krylov_apply(kop, l == 0 ? psi : phis[l - 1], phis[l]);
  }
  PhaseScope ps_ext(tracer, PH_EXTEND);
  // ---- step 2: basis extension, right to left (Eqs. 3, 5-7)
  const int nk = k - 1;
  for (int i = N - 1; i >= 1; --i) {
    const int ml = psi.m[i], mp = psi.m[i + 1], cols = d * mp, ml0 = psi.m[i - 1];
    const cplx* X = psi.A[i].data();
    // C = U S B without truncation: only the row space B enters (R1), taken by the block LQ
    // when it shows full numerical rank, else by the rank-revealing SVD
    DArr Bm;
    int r = 0;
    {
      PhaseScope ps(tracer, PH_EXTEND_SVD);
      QrOut qo;
      qr_blocked(st, &pool, X, ml, cols, 1, qo);
      if (qo.full_rank(kRankRtol)) {
        r = qo.k;
        Bm = std::move(qo.Q);
      } else {
        SvdOut sv;
        svd_jacobi(st, &pool, X, ml, cols, SvdRule{}, sv, false, true);
        r = sv.rank;
        Bm = std::move(sv.Vh);
      }
    }
    tdvp_require(r >= 1, TDVP_ERR_NONFINITE, "extension: zero centre tensor");
    int nb = 0;
    DArr Bbar;
    // at most min(chi_max, d m') - rank B states can be added (R12); a saturated bond adds none
    const int cap = std::min(cols, opt.chi_max) - r;
    if (cap > 0) {
      // Y = [sqrt(w_1) C~_1; ...]  (sum m~ x cols); tr rho~ = |Y|_F^2
      int rows = 0;
      for (int l = 0; l < nk; ++l) rows += phis[l].m[i];
      DArr Y(&pool, (size_t)rows * cols);
      int off = 0;
      for (int l = 0; l < nk; ++l) {
        const int ml_l = phis[l].m[i];
        scale_host(st, Y.data() + (long long)off * cols, phis[l].A[i].data(), mkc(std::sqrt(wts[l]), 0.0),
                   (long long)ml_l * cols);
        off += ml_l;
      }
      blas.norm2(st, Y.data(), (long long)rows * cols, lw.real + 151);
      double tr = 0.0;
      TDVP_CUDA(cudaMemcpyAsync(&tr, lw.real + 151, sizeof(double), cudaMemcpyDeviceToHost, st));
      TDVP_CUDA(cudaStreamSynchronize(st));
      // Y P = Y - (Y B^H) B : rho_bar = (Y P)^H (Y P) = P rho~ P  (Eq. 6)
      DArr G(&pool, (size_t)rows * r);
      for (int pass = 0; pass < 2; ++pass) {
        zgemm(st, OP_N, OP_C, rows, r, cols, kOne, Y.data(), cols, Bm.data(), cols, kZero, G.data(), r, 1, 0, 0, 0, &pool);
        zgemm(st, OP_N, OP_N, rows, cols, r, kMinusOne, G.data(), r, Bm.data(), cols, kOne, Y.data(), cols, 1, 0, 0, 0, &pool);
      }
      if (tr > 0.0) {
        const double eps_m = opt.eps_m;
        double* disc = &disc_m;
        auto rule = [tr, eps_m, cap, disc](const std::vector<double>& s) -> int {
          std::vector<double> ev(s.size());
          for (size_t q = 0; q < s.size(); ++q) ev[q] = s[q] * s[q];
          const int n = keep_count(ev, tr, eps_m, cap, kEigFloorRtol * tr);
          double dsum = 0.0;
          for (size_t q = n; q < ev.size(); ++q) dsum += ev[q];
          *disc += dsum / tr;
          return n;
        };
        SvdOut sy;
        {
          PhaseScope ps(tracer, PH_EXTEND_SVD);
          svd_jacobi(st, &pool, Y.data(), rows, cols, rule, sy, false, true);
        }
        nb = sy.rank;
        if (nb > 0) {
          // enforce B_bar B^H = 0 to rounding: project off range(B) twice, re-orthonormalise
          DArr Gb(&pool, (size_t)nb * r);
          for (int pass = 0; pass < 2; ++pass) {
            zgemm(st, OP_N, OP_C, nb, r, cols, kOne, sy.Vh.data(), cols, Bm.data(), cols, kZero, Gb.data(), r, 1, 0, 0, 0, &pool);
            zgemm(st, OP_N, OP_N, nb, cols, r, kMinusOne, Gb.data(), r, Bm.data(), cols, kOne, sy.Vh.data(),
                  cols, 1, 0, 0, 0, &pool);
          }
          SvdOut so;
          struct KeepAll {
            int operator()(const std::vector<double>& s) const { return (int)s.size(); }
          };
          svd_jacobi(st, &pool, sy.Vh.data(), nb, cols, KeepAll{}, so, false, true);
          Bbar = std::move(so.Vh);
          nb = so.rank;
        }
      }
    }
    added_states += nb;
    const int mnew = r + nb;
    DArr Bp(&pool, (size_t)mnew * cols);
    TDVP_CUDA(cudaMemcpyAsync(Bp.data(), Bm.data(), (size_t)r * cols * sizeof(cplx), cudaMemcpyDeviceToDevice,
                              st));
    if (nb > 0) {
      TDVP_CUDA(cudaMemcpyAsync(Bp.data() + (long long)r * cols, Bbar.data(), (size_t)nb * cols * sizeof(cplx),
                                cudaMemcpyDeviceToDevice, st));
      // B and B_bar each hold every sector of the new index: regroup the rows of B' so each
      // sector is contiguous (a gauge permutation of the bond; G and the centres below use B')
      const std::vector<int> perm = sector_row_order(st, &pool, Bp.data(), mnew, cols);
      if (!perm.empty()) {
        DArr B2(&pool, (size_t)mnew * cols);
        gather_rows(st, Bp.data(), mnew, cols, perm, B2.data());
        Bp = std::move(B2);
      }
    }
    // centres move by Eq. 3: C_{i-1} = A_{i-1} (C_i B'^H), likewise for every psi~_l
    DArr G(&pool, (size_t)ml * mnew);
    zgemm(st, OP_N, OP_C, ml, mnew, cols, kOne, X, cols, Bp.data(), cols, kZero, G.data(), mnew, 1, 0, 0, 0, &pool);
    DArr prv(&pool, (size_t)ml0 * d * mnew);
    zgemm(st, OP_N, OP_N, ml0 * d, mnew, ml, kOne, psi.A[i - 1].data(), ml, G.data(), mnew, kZero, prv.data(),
          mnew, 1, 0, 0, 0, &pool);
    for (int l = 0; l < nk; ++l) {
      MpsDev& ph = phis[l];
      const int mlp = ph.m[i], mlp0 = ph.m[i - 1];
      // the Krylov vectors only feed rho~ of the next bond (the basis they enrich, never
      // |psi> itself), so their centre moves run in the precision form
      DArr Gl(&pool, (size_t)mlp * mnew);
      zgemm_prec(st, scr, kprec(), OP_N, OP_C, mlp, mnew, cols, ph.A[i].data(), cols, Bp.data(), cols,
                 Gl.data(), mnew);
      DArr pp(&pool, (size_t)mlp0 * d * mnew);
      zgemm_prec(st, scr, kprec(), OP_N, OP_N, mlp0 * d, mnew, mlp, ph.A[i - 1].data(), mlp, Gl.data(), mnew,
                 pp.data(), mnew);
      ph.A[i - 1] = std::move(pp);
      ph.A[i].release();
      ph.m[i] = mnew;
    }
    psi.A[i] = std::move(Bp);
    psi.A[i - 1] = std::move(prv);
    psi.m[i] = mnew;
  }
  kop.release();
  center = 0;
  for (int j = 0; j < N; ++j) Lok[j] = Rok[j] = 0;
  sync();
}

void Engine::apply_krylov() {
  canonicalize(N - 1);
  KrylovOp kop;
  build_krylov_op(kop);
  MpsDev out;
  disc_k = 0.0;
  krylov_apply(kop, psi, out);
  kop.release();
  psi.m = out.m;
  for (int i = 0; i < N; ++i) psi.A[i] = std::move(out.A[i]);
  center = N - 1;
  for (int j = 0; j < N; ++j) Lok[j] = Rok[j] = 0;
  sync();
}

// ============================================================================
// observables
// ============================================================================
double Engine::energy() {
  const int c = center;
  ensure_L(c);
  ensure_R(c);
  const long long n = (long long)psi.m[c] * d * psi.m[c + 1];
  DArr y(&pool, n);
  heff(c, psi.A[c].data(), y.data(), TDVP_PREC_FP64);
  blas.multi_dot(st, psi.A[c].data(), n, 1, y.data(), n, lw.c.data());
  blas.norm2(st, psi.A[c].data(), n, lw.real + 152);
  cplx e;
  double nn;
  TDVP_CUDA(cudaMemcpyAsync(&e, lw.c.data(), sizeof(cplx), cudaMemcpyDeviceToHost, st));
  TDVP_CUDA(cudaMemcpyAsync(&nn, lw.real + 152, sizeof(double), cudaMemcpyDeviceToHost, st));
  sync();
  return e.x / nn;
}

double Engine::norm() {
  const int c = center;
  const long long n = (long long)psi.m[c] * d * psi.m[c + 1];
  blas.norm2(st, psi.A[c].data(), n, lw.real + 153);
  double nn;
  TDVP_CUDA(cudaMemcpyAsync(&nn, lw.real + 153, sizeof(double), cudaMemcpyDeviceToHost, st));
  sync();
  return std::sqrt(nn);
}

cplx Engine::expect_local(const double* op, int site) {
  canonicalize(site);
  const long long n = (long long)psi.m[site] * d * psi.m[site + 1];
  DArr o(&pool, (size_t)d * d), y(&pool, n);
  TDVP_CUDA(cudaMemcpyAsync(o.data(), op, sizeof(cplx) * d * d, cudaMemcpyHostToDevice, st));
  k_apply_op_site<<<ceil_div(n, 256), 256, 0, st>>>(o.data(), psi.A[site].data(), psi.m[site], d,
                                                      psi.m[site + 1], y.data());
  TDVP_CHECK_LAUNCH();
  blas.multi_dot(st, psi.A[site].data(), n, 1, y.data(), n, lw.c.data());
  blas.norm2(st, psi.A[site].data(), n, lw.real + 154);
  cplx e;
  double nn;
  TDVP_CUDA(cudaMemcpyAsync(&e, lw.c.data(), sizeof(cplx), cudaMemcpyDeviceToHost, st));
  TDVP_CUDA(cudaMemcpyAsync(&nn, lw.real + 154, sizeof(double), cudaMemcpyDeviceToHost, st));
  sync();
  return mkc(e.x / nn, e.y / nn);
}

// <psi|O|psi> / <psi|psi> for an MPO O: E_{i+1} = sum conj(A_i) E_i W_i A_i from E_0 = 1 over all
// sites (FP64, any gauge); <psi|psi> = |C|^2 at the orthogonality centre.
cplx Engine::expect_mpo(const tdvp_mpo_desc* op) {
  tdvp_require(op->n_sites == N && op->d == d, TDVP_ERR_SHAPE, "expect_mpo: MPO length or d differ from the state's");
  std::vector<int> wo(op->bond_dims, op->bond_dims + N + 1);
  tdvp_require(wo[0] == 1 && wo[N] == 1, TDVP_ERR_SHAPE, "expect_mpo: MPO boundary bond dims must be 1");
  for (int i = 0; i <= N; ++i) tdvp_require(wo[i] >= 1, TDVP_ERR_SHAPE, "expect_mpo: bond dims must be >= 1");
  DArr E(&pool, 1), En;
  k_one<<<1, 1, 0, st>>>(E.data());
  TDVP_CHECK_LAUNCH();
  for (int i = 0; i < N; ++i) {
    tdvp_require(op->sites[i] != nullptr, TDVP_ERR_INVALID_ARG, "expect_mpo: null MPO site");
    const cplx* Wi = reinterpret_cast<const cplx*>(op->sites[i]);
    for (size_t e = 0; e < (size_t)wo[i] * d * d * wo[i + 1]; ++e)
      tdvp_require(std::isfinite(Wi[e].x) && std::isfinite(Wi[e].y), TDVP_ERR_NONFINITE, "non-finite MPO entry");
    WSparse ws;
    ws.build(Wi, wo[i], wo[i + 1], d);
    ws.upload();
    const int ml = psi.m[i], mr = psi.m[i + 1];
    En.reset(&pool, (size_t)mr * wo[i + 1] * mr);
    env_left_fp64(st, scr, E.data(), ws, psi.A[i].data(), ml, mr, d, En.data(), TDVP_PREC_FP64);
    sync();
    ws.free_device();
    E = std::move(En);
  }
  cplx v;
  TDVP_CUDA(cudaMemcpyAsync(&v, E.data(), sizeof(cplx), cudaMemcpyDeviceToHost, st));
  const double n = norm();
  return mkc(v.x / (n * n), v.y / (n * n));
}
