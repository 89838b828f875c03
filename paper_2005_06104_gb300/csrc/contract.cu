// One-site contractions (FP64 on CUDA cores) and the Lanczos exponential.
#include <algorithm>

#include "contract.cuh"

namespace {
const cplx kOne = {1.0, 0.0};
const cplx kZero = {0.0, 0.0};
constexpr double kBreakdown = 1e-13;  // Lanczos invariant-subspace threshold
// local dimension up to which a Lanczos run may launch several iterations per host check
constexpr long long kSpeculateMaxN = 1LL << 18;
}  // namespace

double heff_flops(const SiteOp& op) {
  const double ml = op.ml, mr = op.mr, d = op.d;
  return 8.0 * (ml * d * mr * (ml * op.wl + mr * op.wr) + ml * mr * (double)op.W->nnz);
}

void heff_fp64(cudaStream_t st, Scratch& s, const SiteOp& op, const cplx* x, cplx* y) {
  const int ml = op.ml, mr = op.mr, wl = op.wl, wr = op.wr, d = op.d;
  s.t1.ensure(s.pool, (size_t)ml * wl * d * mr);
  s.t2.ensure(s.pool, (size_t)ml * d * wr * mr);
  // T1[(a,w),(s',b')] = L[(a,w),a'] x[a',(s',b')]
  zgemm(st, OP_N, OP_N, ml * wl, d * mr, ml, kOne, op.L, ml, x, d * mr, kZero, s.t1.data(), d * mr, 1, 0, 0, 0, s.pool);
  // T2[(a,s),(v,b')] = sum W[w,s,s',v] T1[(a,w),(s',b')]
  wstage_left(st, *op.W, s.t1.data(), s.t2.data(), ml, mr);
  // y[(a,s),b] = sum_{(v,b')} T2[(a,s),(v,b')] R[b,(v,b')]
  zgemm(st, OP_N, OP_T, ml * d, mr, wr * mr, kOne, s.t2.data(), (long long)wr * mr, op.R, (long long)wr * mr, kZero,
        y, mr, 1, 0, 0, 0, s.pool);
}

bool prec_is_bf16(int precision) { return precision == TDVP_PREC_BF16X10 || precision == TDVP_PREC_BF16X6; }

void heff_apply_prec(cudaStream_t st, Scratch& s, const SiteOp& op, const cplx* x, cplx* y, int precision) {
  if (prec_is_bf16(precision))
    heff_bf16s(st, s, op, x, y, bf16_slices(precision));
  else if (precision != TDVP_PREC_FP64)
    heff_tf32x3(st, s, op, x, y);
  else
    heff_fp64(st, s, op, x, y);
}

void zgemm_prec(cudaStream_t st, Scratch& s, int precision, int opA, int opB, int M, int N, int K, const cplx* A,
                long long lda, const cplx* B, long long ldb, cplx* C, long long ldc) {
  const bool big = (long long)M * N * K >= (1LL << 21) && M >= 64 && N >= 32;
  if (big && prec_is_bf16(precision))
    zgemm_bf16s(st, s, bf16_slices(precision), opA, opB, M, N, K, A, lda, B, ldb, C, ldc);
  else if (big && precision != TDVP_PREC_FP64)
    zgemm_tc(st, s, opA, opB, M, N, K, A, lda, B, ldb, C, ldc);
  else
    zgemm(st, opA, opB, M, N, K, kOne, A, lda, B, ldb, kZero, C, ldc, 1, 0, 0, 0, s.pool);
}

void keff_fp64(cudaStream_t st, Scratch& s, const cplx* L, int ml, const cplx* R, int mr, int w, const cplx* x,
               cplx* y, int precision) {
  s.t3.ensure(s.pool, (size_t)ml * w * mr);
  zgemm_prec(st, s, precision, OP_N, OP_N, ml * w, mr, ml, L, ml, x, mr, s.t3.data(), mr);
  zgemm_prec(st, s, precision, OP_N, OP_T, ml, mr, w * mr, s.t3.data(), (long long)w * mr, R, (long long)w * mr, y, mr);
}

void env_left_fp64(cudaStream_t st, Scratch& s, const cplx* L, const WSparse& W, const cplx* A, int ml, int mr, int d,
                   cplx* Lout, int precision) {
  const int wl = W.wl, wr = W.wr;
  s.t1.ensure(s.pool, (size_t)ml * wl * d * mr);
  s.t2.ensure(s.pool, (size_t)ml * d * wr * mr);
  zgemm_prec(st, s, precision, OP_N, OP_N, ml * wl, d * mr, ml, L, ml, A, d * mr, s.t1.data(), d * mr);
  wstage_left(st, W, s.t1.data(), s.t2.data(), ml, mr);
  // Lout[b,(v,b')] = sum_{(a,s)} conj(A[(a,s),b]) T2[(a,s),(v,b')]
  zgemm_prec(st, s, precision, OP_C, OP_N, mr, wr * mr, ml * d, A, mr, s.t2.data(), (long long)wr * mr, Lout,
             (long long)wr * mr);
}

void env_right_fp64(cudaStream_t st, Scratch& s, const cplx* R, const WSparse& W, const cplx* B, int ml, int mr, int d,
                    cplx* Rout, int precision) {
  const int wl = W.wl, wr = W.wr;
  s.t3.ensure(s.pool, (size_t)d * ml * mr);
  permute_asb_sab(st, B, s.t3.data(), ml, d, mr);  // Bp[s][a][b]
  s.t1.ensure(s.pool, (size_t)mr * wr * d * ml);
  // U1[(b,v),(s',a')] = sum_b' R[(b,v),b'] Bp[(s',a'),b']
  zgemm_prec(st, s, precision, OP_N, OP_T, mr * wr, d * ml, mr, R, mr, s.t3.data(), mr, s.t1.data(), d * ml);
  s.t2.ensure(s.pool, (size_t)d * mr * wl * ml);
  // U2[s][b][w][a'] = sum W[w,s,s',v] U1[b][v][s'][a']
  wstage_right(st, W, s.t1.data(), s.t2.data(), mr, ml);
  // Rout[a,(w,a')] = sum_{(s,b)} conj(B[a,(s,b)]) U2[(s,b),(w,a')]
  zgemm_prec(st, s, precision, OP_R, OP_N, ml, wl * ml, d * mr, B, d * mr, s.t2.data(), (long long)wl * ml, Rout,
             (long long)wl * ml);
}

void LanczosWork::init(DevicePool* pool) {
  c.reset(pool, 128);
  y.reset(pool, 64);
  if (!real) TDVP_CUDA(cudaMalloc(&real, sizeof(double) * 384));
}

void LanczosWork::release() {
  if (real) cudaFree(real);
  real = nullptr;
  V.release();
  w.release();
  c.release();
  y.release();
}

int lanczos_expm(cudaStream_t st, DevicePool* pool, Blas1& blas, LanczosWork& lw,
                 const std::function<void(const cplx*, cplx*)>& op, const cplx* x, cplx* out, long long n,
                 double delta, int kind, double tol, int nmax, int* hint) {
  nmax = std::min(std::max(1, nmax), 63);
  double* alpha = lw.real;
  double* beta = lw.real + 64;
  double* nrm2 = lw.real + 130;
  double* err = lw.real + 132;
  double* errs = lw.real + 256;  // 2 per iteration of a speculative batch
  lw.V.ensure(pool, (size_t)(nmax + 1) * n);
  lw.w.ensure(pool, (size_t)n);
  cplx* V = lw.V.data();
  cplx* wv = lw.w.data();
  blas.norm2(st, x, n, nrm2);
  double h_n2 = 0.0;
  TDVP_CUDA(cudaMemcpyAsync(&h_n2, nrm2, sizeof(double), cudaMemcpyDeviceToHost, st));
  TDVP_CUDA(cudaStreamSynchronize(st));
  tdvp_require(std::isfinite(h_n2), TDVP_ERR_NONFINITE, "Lanczos: non-finite start vector");
  const double beta0 = std::sqrt(h_n2);
  if (beta0 == 0.0) {
    TDVP_CUDA(cudaMemcpyAsync(out, x, n * sizeof(cplx), cudaMemcpyDeviceToDevice, st));
    return 0;
  }
  scale_by_inv_sqrt(st, V, x, nrm2, n);
  // A small local problem costs a host round trip per iteration more than its arithmetic.  With
  // a hint, the first hint - 1 iterations go out in one batch (each next vector scaled with a
  // guard, so an iteration after an invariant subspace only sees zeros) and their stopping
  // tests are read together.  A run that stops inside the batch recomputes the small
  // exponential at its stopping point (the same inputs and kernel, so the same result as
  // stopping there) and ignores the iterations after it.
  int batch = 1;
  if (hint && *hint > 2 && n <= kSpeculateMaxN)
    batch = (int)std::min<long long>({(long long)*hint - 1, (long long)nmax, n});
  int used = 0, last = -1;
  double last_err = 0.0;
  for (int j = 0; j < nmax;) {
    const int j0 = j;
    for (int b = 0; b < batch; ++b, ++j) {
      if (b > 0) scale_by_inv_sqrt_guarded(st, V + (long long)j * n, wv, nrm2, n);
      op(V + (long long)j * n, wv);
      // alpha_j = Re <v_j, w>; w -= V (V^H w), twice (full re-orthogonalisation); beta = |w|
      blas.lanczos_fused(st, 0, V, n, j + 1, wv, n, nullptr, lw.c.data(), alpha, j, nullptr, nullptr);
      blas.lanczos_fused(st, 1, V, n, j + 1, wv, n, lw.c.data(), lw.c.data() + 64, nullptr, j, nullptr, nullptr);
      blas.lanczos_fused(st, 2, V, n, j + 1, wv, n, lw.c.data() + 64, nullptr, nullptr, j, nrm2, beta + j + 1);
      tridiag_expv(st, alpha, beta, j + 1, delta, kind, nrm2, lw.y.data(), batch > 1 ? errs + 2 * b : err);
    }
    last = j - 1;
    double h_err[2 * 64];
    TDVP_CUDA(cudaMemcpyAsync(h_err, batch > 1 ? errs : err, sizeof(double) * 2 * batch, cudaMemcpyDeviceToHost,
                              st));
    TDVP_CUDA(cudaStreamSynchronize(st));
    for (int b = 0; b < batch; ++b) {
      const int jj = j0 + b;
      tdvp_require(std::isfinite(h_err[2 * b]) && std::isfinite(h_err[2 * b + 1]), TDVP_ERR_NONFINITE,
                   "Lanczos: non-finite coefficient");
      last_err = h_err[2 * b];
      if (h_err[2 * b] <= tol || h_err[2 * b + 1] <= kBreakdown || jj + 1 == n) {
        used = jj + 1;
        break;
      }
    }
    if (used > 0 || j == nmax) break;
    scale_by_inv_sqrt(st, V + (long long)j * n, wv, nrm2, n);
    batch = 1;
  }
  if (used == 0)
    throw TdvpError(TDVP_ERR_LANCZOS_NOT_CONVERGED,
                    "Lanczos error estimate " + std::to_string(last_err) + " above tolerance after " +
                        std::to_string(nmax) + " steps");
  if (used - 1 < last) tridiag_expv(st, alpha, beta, used, delta, kind, nrm2, lw.y.data(), err);
  multi_combine(st, out, V, n, used, lw.y.data(), beta0, n);
  if (hint) *hint = used;
  return used;
}
