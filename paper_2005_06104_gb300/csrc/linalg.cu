// FP64 complex kernels of the GSE-TDVP1 path: GEMM, MPO-tensor contraction
// stages, Krylov-vector BLAS-1, the small tridiagonal exponential of the
// Lanczos exponentiator and a one-sided Jacobi SVD.
#include <algorithm>
#include <cstring>
#include <memory>
#include <numeric>
#include <optional>
#include <unordered_map>

#include "linalg.cuh"

// ============================================================================
// ZGEMM (CUDA cores).  64x64 output tile, 8-deep K slices, 256 threads, each
// thread accumulates a 4x4 block (rows ty+16i, cols tx+16j).
// ============================================================================
namespace {
constexpr int GB_M = 64, GB_N = 64, GB_K = 8;

// nsplit > 1: blockIdx.z = batch * nsplit + split; split s sums K range
// [s*kchunk, min(K, (s+1)*kchunk)) into the partial buffer P[s][batch][M][N]
// (alpha applied, beta left to the reduction).
template <int OPA, int OPB>
__global__ void __launch_bounds__(256)
    k_zgemm(int M, int N, int K, cplx alpha, const cplx* __restrict__ A, long long lda,
            long long sA, const cplx* __restrict__ B, long long ldb, long long sB, cplx beta,
            cplx* __restrict__ C, long long ldc, long long sC, int nsplit, int kchunk, int nbatch,
            cplx* __restrict__ P) {
  __shared__ cplx As[GB_K][GB_M + 1];
  __shared__ cplx Bs[GB_K][GB_N + 1];
  const int split = blockIdx.z % nsplit;
  const long long bz = blockIdx.z / nsplit;
  A += bz * sA;
  B += bz * sB;
  if (nsplit > 1) {
    C = P + ((long long)split * nbatch + bz) * (long long)M * N;
    ldc = N;
    beta = mkc(0.0, 0.0);
  } else {
    C += bz * sC;
  }
  const int kbeg = split * kchunk;
  const int kend = min(K, kbeg + kchunk);
  const int m0 = blockIdx.y * GB_M, n0 = blockIdx.x * GB_N;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  cplx acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = mkc(0.0, 0.0);

  for (int k0 = kbeg; k0 < kend; k0 += GB_K) {
#pragma unroll
    for (int e = tid; e < GB_M * GB_K; e += 256) {
      int m, k;
      if (OPA == OP_N || OPA == OP_R) {
        m = e / GB_K;
        k = e % GB_K;
      } else {
        k = e / GB_M;
        m = e % GB_M;
      }
      const int gm = m0 + m, gk = k0 + k;
      cplx v = mkc(0.0, 0.0);
      if (gm < M && gk < kend) {
        v = (OPA == OP_N || OPA == OP_R) ? A[(long long)gm * lda + gk] : A[(long long)gk * lda + gm];
        if (OPA == OP_C || OPA == OP_R) v.y = -v.y;
      }
      As[k][m] = v;
    }
#pragma unroll
    for (int e = tid; e < GB_K * GB_N; e += 256) {
      int k, n;
      if (OPB == OP_N || OPB == OP_R) {
        k = e / GB_N;
        n = e % GB_N;
      } else {
        n = e / GB_K;
        k = e % GB_K;
      }
      const int gn = n0 + n, gk = k0 + k;
      cplx v = mkc(0.0, 0.0);
      if (gn < N && gk < kend) {
        v = (OPB == OP_N || OPB == OP_R) ? B[(long long)gk * ldb + gn] : B[(long long)gn * ldb + gk];
        if (OPB == OP_C || OPB == OP_R) v.y = -v.y;
      }
      Bs[k][n] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GB_K; ++kk) {
      cplx a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) cfma(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
  const bool use_beta = (beta.x != 0.0 || beta.y != 0.0);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      cplx r = cmul(alpha, acc[i][j]);
      cplx* c = C + (long long)gm * ldc + gn;
      if (use_beta) r = cadd(r, cmul(beta, *c));
      *c = r;
    }
  }
}

#define ZG_ARGS M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, ns, kc, nb, P
template <int OPA>
void zgemm_b(int opB, dim3 g, cudaStream_t st, int M, int N, int K, cplx alpha, const cplx* A,
             long long lda, long long sA, const cplx* B, long long ldb, long long sB, cplx beta,
             cplx* C, long long ldc, long long sC, int ns, int kc, int nb, cplx* P) {
  switch (opB) {
    case OP_N: k_zgemm<OPA, OP_N><<<g, 256, 0, st>>>(ZG_ARGS); break;
    case OP_T: k_zgemm<OPA, OP_T><<<g, 256, 0, st>>>(ZG_ARGS); break;
    case OP_C: k_zgemm<OPA, OP_C><<<g, 256, 0, st>>>(ZG_ARGS); break;
    default:   k_zgemm<OPA, OP_R><<<g, 256, 0, st>>>(ZG_ARGS); break;
  }
}
#undef ZG_ARGS

// C[b][m][n] = sum_s P[s][b][m][n] + beta C[b][m][n]  (fixed summation order)
__global__ void k_splitk_reduce(const cplx* __restrict__ P, int nsplit, int nbatch, int M, int N, cplx beta,
                                cplx* __restrict__ C, long long ldc, long long sC) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long per = (long long)M * N;
  if (e >= per * nbatch) return;
  const long long b = e / per, r = e % per;
  const int m = r / N, n = r % N;
  cplx acc = mkc(0.0, 0.0);
  for (int s = 0; s < nsplit; ++s) acc = cadd(acc, P[((long long)s * nbatch + b) * per + r]);
  cplx* c = C + b * sC + (long long)m * ldc + n;
  if (beta.x != 0.0 || beta.y != 0.0) acc = cadd(acc, cmul(beta, *c));
  *c = acc;
}
}  // namespace

void zgemm(cudaStream_t st, int opA, int opB, int M, int N, int K, cplx alpha, const cplx* A,
           long long lda, const cplx* B, long long ldb, cplx beta, cplx* C, long long ldc,
           int batch, long long sA, long long sB, long long sC, DevicePool* ws) {
  if (M <= 0 || N <= 0 || batch <= 0) return;
  tdvp_require(batch <= 65535, TDVP_ERR_INVALID_ARG, "zgemm: batch too large");
  tdvp_require(ceil_div(M, GB_M) <= 65535, TDVP_ERR_INVALID_ARG, "zgemm: M too large");
  if (K <= 0) {  // C = beta C
    tdvp_require(beta.x == 0.0 && beta.y == 0.0, TDVP_ERR_INVALID_ARG, "zgemm: K=0 with beta");
    for (int b = 0; b < batch; ++b)
      for (int r = 0; r < M; ++r)
        TDVP_CUDA(cudaMemsetAsync(C + b * sC + (long long)r * ldc, 0, sizeof(cplx) * N, st));
    return;
  }
  // FP64 throughput per SM is low on this part: a GEMM with few output tiles and a
  // long K is split along K over enough blocks to occupy the GPU (needs a pool).
  const long long tiles = (long long)ceil_div(N, GB_N) * ceil_div(M, GB_M) * batch;
  int ns = 1, kc = K;
  static const int sms = [] {  // thread-safe one-time initialisation
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 148;
  }();
  if (ws && tiles < 2LL * sms && K >= 32) {
    ns = (int)std::min<long long>((2LL * sms + tiles - 1) / tiles, (K + 15) / 16);
    ns = std::max(1, std::min(ns, 65535 / batch));
    kc = ((K + ns - 1) / ns + GB_K - 1) / GB_K * GB_K;
    ns = (K + kc - 1) / kc;
  }
  DArr part;
  if (ns > 1) part.reset(ws, (size_t)ns * batch * M * N);
  dim3 g(ceil_div(N, GB_N), ceil_div(M, GB_M), batch * ns);
  cplx* P = part.data();
  switch (opA) {
    case OP_N: zgemm_b<OP_N>(opB, g, st, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, ns, kc, batch, P); break;
    case OP_T: zgemm_b<OP_T>(opB, g, st, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, ns, kc, batch, P); break;
    case OP_C: zgemm_b<OP_C>(opB, g, st, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, ns, kc, batch, P); break;
    default:   zgemm_b<OP_R>(opB, g, st, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, ns, kc, batch, P); break;
  }
  TDVP_CHECK_LAUNCH();
  if (ns > 1) {
    const long long n = (long long)M * N * batch;
    k_splitk_reduce<<<ceil_div(n, 256), 256, 0, st>>>(P, ns, batch, M, N, beta, C, ldc, sC);
    TDVP_CHECK_LAUNCH();
  }
}

// ============================================================================
// MPO-tensor stages
// ============================================================================
void WSparse::build(const cplx* W, int wl_, int wr_, int d_) {
  wl = wl_;
  wr = wr_;
  d = d_;
  l_off.assign(d * wr + 1, 0);
  r_off.assign(d * wl + 1, 0);
  l_idx.clear();
  l_val.clear();
  r_idx.clear();
  r_val.clear();
  auto at = [&](int w, int s, int t, int v) { return W[((w * d + s) * d + t) * wr + v]; };
  nnz = 0;
  for (int s = 0; s < d; ++s)
    for (int v = 0; v < wr; ++v) {
      for (int w = 0; w < wl; ++w)
        for (int t = 0; t < d; ++t) {
          cplx x = at(w, s, t, v);
          if (x.x != 0.0 || x.y != 0.0) {
            l_idx.push_back(w);
            l_idx.push_back(t);
            l_val.push_back(x);
          }
        }
      l_off[s * wr + v + 1] = (int)l_val.size();
    }
  for (int s = 0; s < d; ++s)
    for (int w = 0; w < wl; ++w) {
      for (int v = 0; v < wr; ++v)
        for (int t = 0; t < d; ++t) {
          cplx x = at(w, s, t, v);
          if (x.x != 0.0 || x.y != 0.0) {
            r_idx.push_back(v);
            r_idx.push_back(t);
            r_val.push_back(x);
          }
        }
      r_off[s * wl + w + 1] = (int)r_val.size();
    }
  nnz = (int)l_val.size();
}

void WSparse::upload() {
  free_device();
  auto up = [](auto& vec, auto** dst) {
    using T = typename std::remove_reference<decltype(vec)>::type::value_type;
    size_t bytes = std::max<size_t>(1, vec.size()) * sizeof(T);
    TDVP_CUDA(cudaMalloc((void**)dst, bytes));
    if (!vec.empty()) TDVP_CUDA(cudaMemcpy(*dst, vec.data(), vec.size() * sizeof(T), cudaMemcpyHostToDevice));
  };
  up(l_off, &d_l_off);
  up(l_idx, &d_l_idx);
  up(l_val, &d_l_val);
  l_val_df.resize(l_val.size());
  for (size_t e = 0; e < l_val.size(); ++e) {
    const float rh = (float)l_val[e].x, ih = (float)l_val[e].y;
    l_val_df[e] = make_float4(rh, (float)(l_val[e].x - (double)rh), ih, (float)(l_val[e].y - (double)ih));
  }
  up(l_val_df, &d_l_val_df);
  up(r_off, &d_r_off);
  up(r_idx, &d_r_idx);
  up(r_val, &d_r_val);
}

void WSparse::free_device() {
  cudaFree(d_l_off);
  cudaFree(d_l_idx);
  cudaFree(d_l_val);
  cudaFree(d_l_val_df);
  d_l_val_df = nullptr;
  cudaFree(d_r_off);
  cudaFree(d_r_idx);
  cudaFree(d_r_val);
  d_l_off = d_l_idx = d_r_off = d_r_idx = nullptr;
  d_l_val = d_r_val = nullptr;
}

namespace {
__global__ void k_wstage_left(const cplx* __restrict__ in, cplx* __restrict__ out, int WL, int WR,
                              int D, int C, const int* __restrict__ off, const int* __restrict__ idx,
                              const cplx* __restrict__ val) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int sv = blockIdx.y;
  const long long a = blockIdx.z;
  if (c >= C) return;
  const int s = sv / WR, v = sv % WR;
  cplx acc = mkc(0.0, 0.0);
  for (int e = off[sv]; e < off[sv + 1]; ++e) {
    const int w = idx[2 * e], t = idx[2 * e + 1];
    cfma(acc, val[e], in[((a * WL + w) * D + t) * C + c]);
  }
  out[((a * D + s) * WR + v) * C + c] = acc;
}

__global__ void k_wstage_right(const cplx* __restrict__ in, cplx* __restrict__ out, int B, int WL,
                               int WR, int D, int C, const int* __restrict__ off,
                               const int* __restrict__ idx, const cplx* __restrict__ val) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int sw = blockIdx.y;
  const long long b = blockIdx.z;
  if (c >= C) return;
  const int s = sw / WL, w = sw % WL;
  cplx acc = mkc(0.0, 0.0);
  for (int e = off[sw]; e < off[sw + 1]; ++e) {
    const int v = idx[2 * e], t = idx[2 * e + 1];
    cfma(acc, val[e], in[((b * WR + v) * D + t) * C + c]);
  }
  out[(((long long)s * B + b) * WL + w) * C + c] = acc;
}

__global__ void k_permute_asb(const cplx* __restrict__ in, cplx* __restrict__ out, int A, int S, int B) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n = (long long)A * S * B;
  if (i >= n) return;
  const int b = i % B;
  const long long as = i / B;
  const int s = as % S;
  const long long a = as / S;
  out[((long long)s * A + a) * B + b] = in[i];
}
}  // namespace

void wstage_left(cudaStream_t st, const WSparse& w, const cplx* in, cplx* out, int A, int C) {
  tdvp_require(A <= 65535, TDVP_ERR_INVALID_ARG, "wstage_left: too many rows");
  dim3 g(ceil_div(C, 128), w.d * w.wr, A);
  k_wstage_left<<<g, 128, 0, st>>>(in, out, w.wl, w.wr, w.d, C, w.d_l_off, w.d_l_idx, w.d_l_val);
  TDVP_CHECK_LAUNCH();
}

void wstage_right(cudaStream_t st, const WSparse& w, const cplx* in, cplx* out, int B, int C) {
  tdvp_require(B <= 65535, TDVP_ERR_INVALID_ARG, "wstage_right: too many rows");
  dim3 g(ceil_div(C, 128), w.d * w.wl, B);
  k_wstage_right<<<g, 128, 0, st>>>(in, out, B, w.wl, w.wr, w.d, C, w.d_r_off, w.d_r_idx, w.d_r_val);
  TDVP_CHECK_LAUNCH();
}

void permute_asb_sab(cudaStream_t st, const cplx* in, cplx* out, int A, int S, int B) {
  const long long n = (long long)A * S * B;
  if (n == 0) return;
  k_permute_asb<<<ceil_div(n, 256), 256, 0, st>>>(in, out, A, S, B);
  TDVP_CHECK_LAUNCH();
}

// ============================================================================
// BLAS-1 (deterministic two-pass reductions)
// ============================================================================
namespace {
constexpr int RED_THREADS = 256;
constexpr int MD_CH = 8;

__device__ __forceinline__ cplx warp_sum(cplx v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, o);
    v.y += __shfl_down_sync(0xffffffffu, v.y, o);
  }
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(RED_THREADS)
    k_multidot_partial(const cplx* __restrict__ V, long long ldv, int nvec, const cplx* __restrict__ w,
                       long long n, cplx* __restrict__ partial) {
  __shared__ cplx red[MD_CH][RED_THREADS / 32];
  const int G = gridDim.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k0 = 0; k0 < nvec; k0 += MD_CH) {
    cplx acc[MD_CH];
#pragma unroll
    for (int q = 0; q < MD_CH; ++q) acc[q] = mkc(0.0, 0.0);
    for (long long i = (long long)blockIdx.x * RED_THREADS + threadIdx.x; i < n;
         i += (long long)G * RED_THREADS) {
      const cplx wi = w[i];
#pragma unroll
      for (int q = 0; q < MD_CH; ++q)
        if (k0 + q < nvec) cfma_conj(acc[q], V[(long long)(k0 + q) * ldv + i], wi);
    }
#pragma unroll
    for (int q = 0; q < MD_CH; ++q) {
      cplx s = warp_sum(acc[q]);
      if (lane == 0) red[q][warp] = s;
    }
    __syncthreads();
    if (threadIdx.x < MD_CH && k0 + (int)threadIdx.x < nvec) {
      cplx s = mkc(0.0, 0.0);
      for (int u = 0; u < RED_THREADS / 32; ++u) s = cadd(s, red[threadIdx.x][u]);
      partial[(long long)(k0 + threadIdx.x) * G + blockIdx.x] = s;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(RED_THREADS)
    k_reduce_partial_c(const cplx* __restrict__ partial, int G, cplx* __restrict__ out) {
  __shared__ cplx red[RED_THREADS / 32];
  const int k = blockIdx.x;
  cplx s = mkc(0.0, 0.0);
  for (int g = threadIdx.x; g < G; g += RED_THREADS) s = cadd(s, partial[(long long)k * G + g]);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    cplx t = mkc(0.0, 0.0);
    for (int u = 0; u < RED_THREADS / 32; ++u) t = cadd(t, red[u]);
    out[k] = t;
  }
}

__global__ void __launch_bounds__(RED_THREADS)
    k_norm2_partial(const cplx* __restrict__ x, long long n, double* __restrict__ partial) {
  __shared__ double red[RED_THREADS / 32];
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * RED_THREADS + threadIdx.x; i < n;
       i += (long long)gridDim.x * RED_THREADS)
    acc += cabs2(x[i]);
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int u = 0; u < RED_THREADS / 32; ++u) t += red[u];
    partial[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(RED_THREADS)
    k_reduce_partial_d(const double* __restrict__ partial, int G, double* __restrict__ out) {
  __shared__ double red[RED_THREADS / 32];
  double s = 0.0;
  for (int g = threadIdx.x; g < G; g += RED_THREADS) s += partial[g];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int u = 0; u < RED_THREADS / 32; ++u) t += red[u];
    *out = t;
  }
}

__global__ void k_multi_axpy_sub(cplx* __restrict__ w, const cplx* __restrict__ V, long long ldv,
                                 int nvec, const cplx* __restrict__ c, long long n) {
  __shared__ cplx cs[64];
  for (int k = threadIdx.x; k < nvec && k < 64; k += blockDim.x) cs[k] = c[k];
  __syncthreads();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  cplx acc = mkc(0.0, 0.0);
  for (int k = 0; k < nvec; ++k) cfma(acc, V[(long long)k * ldv + i], cs[k]);
  w[i] = csub(w[i], acc);
}

__global__ void k_multi_combine(cplx* __restrict__ y, const cplx* __restrict__ V, long long ldv,
                                int nvec, const cplx* __restrict__ c, double scale, long long n) {
  __shared__ cplx cs[64];
  for (int k = threadIdx.x; k < nvec && k < 64; k += blockDim.x) cs[k] = c[k];
  __syncthreads();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  cplx acc = mkc(0.0, 0.0);
  for (int k = 0; k < nvec; ++k) cfma(acc, V[(long long)k * ldv + i], cs[k]);
  y[i] = cscale(acc, scale);
}

__global__ void k_scale_inv_sqrt(cplx* __restrict__ dst, const cplx* __restrict__ src,
                                 const double* __restrict__ nrm2, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double s = 1.0 / sqrt(*nrm2);
  dst[i] = cscale(src[i], s);
}

// as k_scale_inv_sqrt, but a norm that is not a positive finite number above 1e-200 gives zeros
__global__ void k_scale_inv_sqrt_guarded(cplx* __restrict__ dst, const cplx* __restrict__ src,
                                         const double* __restrict__ nrm2, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double q = *nrm2;
  const double s = (q > 1e-200 && q <= 1.7e308) ? 1.0 / sqrt(q) : 0.0;
  dst[i] = cscale(src[i], s);
}

__global__ void k_scale_host(cplx* __restrict__ dst, const cplx* __restrict__ src, cplx s, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  dst[i] = cmul(src[i], s);
}

__global__ void k_copy_real(const cplx* c, int j, double* alpha) { alpha[j] = c[j].x; }
__global__ void k_store_beta(const double* nrm2, double* slot) { *slot = sqrt(*nrm2); }
}  // namespace

static int red_blocks(long long n, int max_blocks);

void Blas1::init(DevicePool* p, int sm_count) {
  pool = p;
  max_blocks = 2 * sm_count;
  partial.reset(pool, (size_t)max_blocks * 64);
  if (!counter) {
    TDVP_CUDA(cudaMalloc(&counter, sizeof(unsigned)));
    TDVP_CUDA(cudaMemset(counter, 0, sizeof(unsigned)));
  }
}

void Blas1::release() {
  if (counter) cudaFree(counter);
  counter = nullptr;
  partial.release();
}

// ---------------------------------------------------------------------------
// Fused Lanczos re-orthogonalisation steps.  Each kernel writes per-block
// partial sums; the last block to finish (atomic ticket, no waiting) reduces
// them in a fixed order, so results are deterministic and no block spins.
namespace {
__device__ __forceinline__ bool last_block(unsigned* counter) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned t = atomicAdd(counter, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  return is_last;
}

// mode 0: c = V^H w                        (alpha[j] = Re c[j])
// mode 1: w -= V cin;  c = V^H w
// mode 2: w -= V cin;  nrm2 = |w|^2, beta_slot = sqrt(nrm2)
__global__ void __launch_bounds__(RED_THREADS)
    k_lanczos_fused(int mode, const cplx* __restrict__ V, long long ldv, int nvec, cplx* __restrict__ w, long long n,
                    const cplx* __restrict__ cin, cplx* __restrict__ cout, double* __restrict__ alpha, int j,
                    double* __restrict__ nrm2, double* __restrict__ beta_slot, cplx* __restrict__ partial,
                    unsigned* __restrict__ counter) {
  __shared__ cplx cs[64];
  __shared__ cplx red[MD_CH][RED_THREADS / 32];
  __shared__ double dred[RED_THREADS / 32];
  const int G = gridDim.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (mode >= 1) {
    for (int k = threadIdx.x; k < nvec; k += blockDim.x) cs[k] = cin[k];
    __syncthreads();
    for (long long i = (long long)blockIdx.x * RED_THREADS + threadIdx.x; i < n; i += (long long)G * RED_THREADS) {
      cplx acc = mkc(0.0, 0.0);
      for (int k = 0; k < nvec; ++k) cfma(acc, V[(long long)k * ldv + i], cs[k]);
      w[i] = csub(w[i], acc);
    }
    // each thread re-reads only the w[i] it wrote: no block-wide barrier needed
  }
  if (mode <= 1) {
    for (int k0 = 0; k0 < nvec; k0 += MD_CH) {
      cplx acc[MD_CH];
#pragma unroll
      for (int q = 0; q < MD_CH; ++q) acc[q] = mkc(0.0, 0.0);
      for (long long i = (long long)blockIdx.x * RED_THREADS + threadIdx.x; i < n; i += (long long)G * RED_THREADS) {
        const cplx wi = w[i];
#pragma unroll
        for (int q = 0; q < MD_CH; ++q)
          if (k0 + q < nvec) cfma_conj(acc[q], V[(long long)(k0 + q) * ldv + i], wi);
      }
#pragma unroll
      for (int q = 0; q < MD_CH; ++q) {
        cplx t = warp_sum(acc[q]);
        if (lane == 0) red[q][warp] = t;
      }
      __syncthreads();
      if (threadIdx.x < MD_CH && k0 + (int)threadIdx.x < nvec) {
        cplx t = mkc(0.0, 0.0);
        for (int u = 0; u < RED_THREADS / 32; ++u) t = cadd(t, red[threadIdx.x][u]);
        partial[(long long)(k0 + threadIdx.x) * G + blockIdx.x] = t;
      }
      __syncthreads();
    }
    if (last_block(counter)) {
      for (int k = warp; k < nvec; k += RED_THREADS / 32) {
        cplx t = mkc(0.0, 0.0);
        for (int g = lane; g < G; g += 32) t = cadd(t, partial[(long long)k * G + g]);
        t = warp_sum(t);
        if (lane == 0) {
          cout[k] = t;
          if (mode == 0 && k == j) alpha[j] = t.x;
        }
      }
      if (threadIdx.x == 0) *counter = 0;
    }
  } else {
    double a = 0.0;
    for (long long i = (long long)blockIdx.x * RED_THREADS + threadIdx.x; i < n; i += (long long)G * RED_THREADS)
      a += cabs2(w[i]);
    a = warp_sum(a);
    if (lane == 0) dred[warp] = a;
    __syncthreads();
    double* dpart = reinterpret_cast<double*>(partial);
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int u = 0; u < RED_THREADS / 32; ++u) t += dred[u];
      dpart[blockIdx.x] = t;
    }
    if (last_block(counter)) {
      if (threadIdx.x == 0) {
        double t = 0.0;
        for (int g = 0; g < G; ++g) t += dpart[g];
        *nrm2 = t;
        *beta_slot = sqrt(t);
        *counter = 0;
      }
    }
  }
}
}  // namespace

void Blas1::lanczos_fused(cudaStream_t st, int mode, const cplx* V, long long ldv, int nvec, cplx* w, long long n,
                          const cplx* cin, cplx* cout, double* alpha, int j, double* nrm2, double* beta_slot) {
  tdvp_require(nvec >= 1 && nvec <= 64, TDVP_ERR_INVALID_ARG, "lanczos_fused: nvec out of range");
  const int G = red_blocks(n, max_blocks);
  k_lanczos_fused<<<G, RED_THREADS, 0, st>>>(mode, V, ldv, nvec, w, n, cin, cout, alpha, j, nrm2, beta_slot,
                                             partial.data(), counter);
  TDVP_CHECK_LAUNCH();
}

static int red_blocks(long long n, int max_blocks) {
  return std::max(1, std::min<int>(max_blocks, ceil_div(n, RED_THREADS * 4)));
}

void Blas1::multi_dot(cudaStream_t st, const cplx* V, long long ldv, int nvec, const cplx* w,
                      long long n, cplx* out) {
  tdvp_require(nvec <= 64, TDVP_ERR_INVALID_ARG, "multi_dot: nvec > 64");
  const int G = red_blocks(n, max_blocks);
  k_multidot_partial<<<G, RED_THREADS, 0, st>>>(V, ldv, nvec, w, n, partial.data());
  TDVP_CHECK_LAUNCH();
  k_reduce_partial_c<<<nvec, RED_THREADS, 0, st>>>(partial.data(), G, out);
  TDVP_CHECK_LAUNCH();
}

void Blas1::norm2(cudaStream_t st, const cplx* x, long long n, double* out) {
  const int G = red_blocks(n, max_blocks);
  double* part = reinterpret_cast<double*>(partial.data());
  k_norm2_partial<<<G, RED_THREADS, 0, st>>>(x, n, part);
  TDVP_CHECK_LAUNCH();
  k_reduce_partial_d<<<1, RED_THREADS, 0, st>>>(part, G, out);
  TDVP_CHECK_LAUNCH();
}

void multi_axpy_sub(cudaStream_t st, cplx* w, const cplx* V, long long ldv, int nvec, const cplx* c,
                    long long n) {
  tdvp_require(nvec <= 64, TDVP_ERR_INVALID_ARG, "multi_axpy: nvec > 64");
  if (n == 0 || nvec == 0) return;
  k_multi_axpy_sub<<<ceil_div(n, 256), 256, 0, st>>>(w, V, ldv, nvec, c, n);
  TDVP_CHECK_LAUNCH();
}

void multi_combine(cudaStream_t st, cplx* y, const cplx* V, long long ldv, int nvec, const cplx* c,
                   double scale, long long n) {
  tdvp_require(nvec <= 64, TDVP_ERR_INVALID_ARG, "multi_combine: nvec > 64");
  if (n == 0) return;
  k_multi_combine<<<ceil_div(n, 256), 256, 0, st>>>(y, V, ldv, nvec, c, scale, n);
  TDVP_CHECK_LAUNCH();
}

void scale_by_inv_sqrt(cudaStream_t st, cplx* dst, const cplx* src, const double* nrm2, long long n) {
  if (n == 0) return;
  k_scale_inv_sqrt<<<ceil_div(n, 256), 256, 0, st>>>(dst, src, nrm2, n);
  TDVP_CHECK_LAUNCH();
}

void scale_by_inv_sqrt_guarded(cudaStream_t st, cplx* dst, const cplx* src, const double* nrm2, long long n) {
  if (n == 0) return;
  k_scale_inv_sqrt_guarded<<<ceil_div(n, 256), 256, 0, st>>>(dst, src, nrm2, n);
  TDVP_CHECK_LAUNCH();
}

void scale_host(cudaStream_t st, cplx* dst, const cplx* src, cplx s, long long n) {
  if (n == 0) return;
  k_scale_host<<<ceil_div(n, 256), 256, 0, st>>>(dst, src, s, n);
  TDVP_CHECK_LAUNCH();
}

void fill_zero(cudaStream_t st, cplx* p, long long n) {
  if (n) TDVP_CUDA(cudaMemsetAsync(p, 0, n * sizeof(cplx), st));
}

void copy_real_part(cudaStream_t st, const cplx* c, int j, double* alpha) {
  k_copy_real<<<1, 1, 0, st>>>(c, j, alpha);
  TDVP_CHECK_LAUNCH();
}

void store_beta(cudaStream_t st, const double* nrm2, double* slot) {
  k_store_beta<<<1, 1, 0, st>>>(nrm2, slot);
  TDVP_CHECK_LAUNCH();
}

// ============================================================================
// exp(coef T) e_0 for a small symmetric tridiagonal T (Lanczos matrix).
//
// Chebyshev expansion on the Gershgorin interval [lo, hi] of T, T = c + h X
// with spec(X) in [-1, 1]:
//   real time  exp(-i delta T) = e^{-i delta c} sum_k eps_k (-i sgn delta)^k J_k(|delta| h) T_k(X)
//   imag time  exp(-delta T)   = e^{-delta lo} sum_k eps_k (-1)^k e^{-x} I_k(x) T_k(X),  delta > 0
//                              = e^{|delta| hi} sum_k eps_k e^{-x} I_k(x) T_k(X),        delta < 0
// with x = |delta| h, eps_0 = 1, eps_k = 2.  J_k and e^{-x} I_k come from Miller's
// backward recurrence normalised by J_0 + 2 sum J_2k = 1 and I_0 + 2 sum I_k = e^x.
// One block; thread i owns component i (n <= 64).
// ============================================================================
namespace {
constexpr int TRI_MAX = 64;
constexpr int CHEB_MAX = 1024;

__global__ void __launch_bounds__(TRI_MAX)
    k_tridiag_expv(const double* __restrict__ alpha, const double* __restrict__ beta, int n,
                   double delta, int kind, const double* __restrict__ nrm2_next,
                   cplx* __restrict__ y, double* __restrict__ err) {
  __shared__ double d[TRI_MAX], o[TRI_MAX + 1];
  __shared__ double tk[TRI_MAX];
  __shared__ double coef[CHEB_MAX + 1];
  __shared__ double sh_c, sh_h, sh_lo, sh_hi;
  __shared__ int sh_K, sh_bad;
  const int i = threadIdx.x;
  if (i < n) d[i] = alpha[i];
  if (i <= n) o[i] = (i >= 1 && i < n) ? beta[i] : 0.0;
  __syncthreads();
  if (i == 0) {
    double lo = 1e300, hi = -1e300;
    for (int r = 0; r < n; ++r) {
      const double rad = fabs(o[r]) + fabs(o[r + 1]);
      lo = fmin(lo, d[r] - rad);
      hi = fmax(hi, d[r] + rad);
    }
    const double c = 0.5 * (hi + lo), h = 0.5 * (hi - lo);
    sh_c = c;
    sh_h = h;
    sh_lo = lo;
    sh_hi = hi;
    const double x = fabs(delta) * h;
    int K = (int)(x + 10.0 * cbrt(x + 1.0) + 40.0);
    sh_bad = 0;
    if (K > CHEB_MAX) {
      K = CHEB_MAX;
      sh_bad = 1;
    }
    sh_K = K;
    // Miller backward recurrence, start well above K
    const int M = 2 * ((K + 40 + (int)x) / 2 + 1);
    for (int k = 0; k <= K; ++k) coef[k] = 0.0;
    if (x < 1e-300) {
      coef[0] = 1.0;
    } else {
      double jp1 = 0.0, jk = 1e-280, norm = 0.0;
      for (int k = M; k >= 1; --k) {
        // value at index k is jk, at k+1 is jp1; produce index k-1
        const double jm1 = (kind == 0) ? (2.0 * k / x) * jk - jp1 : (2.0 * k / x) * jk + jp1;
        if (k <= K) coef[k] = jk;
        if (kind == 0) {
          if ((k & 1) == 0) norm += 2.0 * jk;
        } else {
          norm += 2.0 * jk;
        }
        jp1 = jk;
        jk = jm1;
        if (fabs(jk) > 1e250) {  // rescale
          const double f = 1e-250;
          jk *= f;
          jp1 *= f;
          norm *= f;
          for (int q = k; q <= K; ++q) coef[q] *= f;
        }
      }
      coef[0] = jk;
      norm += jk;
      for (int k = 0; k <= K; ++k) coef[k] /= norm;
    }
  }
  __syncthreads();
  const int K = sh_K;
  const double c = sh_c, h = sh_h;
  const double inv_h = h > 0.0 ? 1.0 / h : 0.0;
  // scaled matrix X = (T - c) / h
  const double xd = (i < n) ? (d[i] - c) * inv_h : 0.0;
  const double xl = (i < n && i >= 1) ? o[i] * inv_h : 0.0;
  const double xr = (i + 1 < n) ? o[i + 1] * inv_h : 0.0;
  double acc_re = 0.0, acc_im = 0.0;
  // T_0 e0 = e0
  double cur = (i == 0) ? 1.0 : 0.0, prev = 0.0;
  for (int k = 0; k <= K; ++k) {
    // coefficient eps_k * phase_k * coef[k]
    const double ck = (k == 0 ? 1.0 : 2.0) * coef[k];
    double pre, pim;
    if (kind == 0) {
      // (-i sgn)^k
      const int m = k & 3;
      const double sgn = delta >= 0 ? 1.0 : -1.0;
      pre = (m == 0) ? 1.0 : (m == 2 ? -1.0 : 0.0);
      pim = (m == 1) ? -sgn : (m == 3 ? sgn : 0.0);
    } else {
      pre = (delta >= 0 && (k & 1)) ? -1.0 : 1.0;
      pim = 0.0;
    }
    acc_re += ck * pre * cur;
    acc_im += ck * pim * cur;
    if (k == K) break;
    if (i < n) tk[i] = cur;
    __syncthreads();
    double xv = 0.0;
    if (i < n) {
      xv = xd * cur;
      if (i >= 1) xv += xl * tk[i - 1];
      if (i + 1 < n) xv += xr * tk[i + 1];
    }
    const double nxt = (k == 0) ? xv : 2.0 * xv - prev;
    __syncthreads();
    prev = cur;
    cur = nxt;
  }
  if (i < n) {
    double fre, fim;
    if (kind == 0) {
      const double ph = -delta * c;
      fre = cos(ph);
      fim = sin(ph);
    } else {
      const double e = (delta >= 0) ? exp(-delta * sh_lo) : exp(-delta * sh_hi);
      fre = e;
      fim = 0.0;
    }
    y[i] = mkc(fre * acc_re - fim * acc_im, fre * acc_im + fim * acc_re);
    if (i == n - 1) {
      const double b = sqrt(*nrm2_next);
      const double ylast = sqrt(cabs2(y[i]));
      err[0] = sh_bad ? 1e300 : b * ylast;
      err[1] = b;
    }
  }
}
}  // namespace

void tridiag_expv(cudaStream_t st, const double* alpha, const double* beta, int n, double delta,
                  int kind, const double* nrm2_next, cplx* y, double* err) {
  tdvp_require(n >= 1 && n < TRI_MAX, TDVP_ERR_INVALID_ARG, "tridiag_expv: n out of range");
  k_tridiag_expv<<<1, TRI_MAX, 0, st>>>(alpha, beta, n, delta, kind, nrm2_next, y, err);
  TDVP_CHECK_LAUNCH();
}

// ============================================================================
// One-sided Jacobi SVD (Hestenes) in FP64.  The working matrix X (p x q,
// column-major) has its q columns orthogonalised by unitary plane rotations
// applied from the right, accumulated in Vx (q x q): X0 Vx = U S.
// Rows >= cols: X0 = M.  Rows < cols: X0 = M^H (so p >= q always).
// Columns are paired by the round-robin (circle) schedule; one sweep = qpad-1
// rounds of qpad/2 disjoint pairs.
// ============================================================================
namespace {
__device__ __forceinline__ void rr_pair(int round, int k, int qpad, int& P, int& Q) {
  const int m = qpad - 1;
  if (k == 0) {
    P = round;
    Q = m;
  } else {
    P = (round + k) % m;
    Q = (round - k + m) % m;
  }
  if (P > Q) {
    int t = P;
    P = Q;
    Q = t;
  }
}

// Rotation from a = |x_p|^2, b = |x_q|^2, c = x_p^H x_q:
//   x_p' = cs x_p - sn e^{-i phi} x_q,  x_q' = sn e^{i phi} x_p + cs x_q,  c = |c| e^{i phi}
// Pairs whose larger column is below floor2 (kJacobiFloor |M|_F^2) or whose smaller
// column is below kJacobiFloor times the larger (norms squared) are left alone.  Such
// columns hold singular values below 1e-15 of their neighbours, under every keep rule
// of the method (rank 1e-10 s_max, eigenvalue floor 1e-14 lambda_max), and rotating
// them against each other chases rounding noise for extra sweeps while moving the
// kept columns by at most 1e-15.
// Complex arithmetic and limits for the precision a Jacobi runs in: FP64 (double2) in general,
// FP32 (float2) for the eigendecompositions that the precision form allows in FP32.
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ float cabs2(float2 a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ void cfma_conj(float2& a, float2 b, float2 c) {
  a.x = fmaf(b.x, c.x, fmaf(b.y, c.y, a.x));
  a.y = fmaf(b.x, c.y, fmaf(-b.y, c.x, a.y));
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float2 warp_sum(float2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, o);
    v.y += __shfl_down_sync(0xffffffffu, v.y, o);
  }
  return v;
}
template <class T>
struct Jac;
template <>
struct Jac<double> {
  typedef double2 C;
  static __device__ __forceinline__ C make(double r, double i) { return make_double2(r, i); }
  static constexpr double eps = 2.2e-16, tol_min = 1e-15;
  // A sweep whose rotations all have |sin theta| <= 1e-8 ends the iteration (see below).
  static constexpr double small_angle2 = 1e-16;
};
template <>
struct Jac<float> {
  typedef float2 C;
  static __device__ __forceinline__ C make(float r, float i) { return make_float2(r, i); }
  static constexpr float eps = 1.2e-7f, tol_min = 1e-7f;
  // FP32 resolves couplings to about 1e-7: a sweep with |sin theta| <= 1e-6 ends it
  static constexpr float small_angle2 = 1e-12f;
};

constexpr double kJacobiFloor = 1e-30;
// A sweep whose rotations all have |sin theta| <= 1e-8 ends the iteration.  Each rotation
// annihilates its pair's coupling and only mixes the couplings of its two columns with the
// others, so after such a sweep every remaining coupling is of second order in the angles
// (about 1e-16 relative), which a further sweep would only confirm.  Near-degenerate
// columns with a tiny coupling give large angles and keep the iteration going.
constexpr double kJacobiSmallAngle2 = 1e-16;
template <class T, class C>
__device__ __forceinline__ bool jacobi_params(T a, T b, C c, T tol, T floor2, T& cs, C& sne) {
  const T big = fmax(a, b), small = fmin(a, b);
  if (big <= floor2 || small <= (T)kJacobiFloor * big) return false;
  const T ac2 = cabs2(c);
  // |c| > tol sqrt(a b), squared (no square root on the common no-rotation path)
  if (!(ac2 > tol * tol * a * b)) return false;
  const T inv_ac = rsqrt(ac2);
  const T zeta = (T)0.5 * (b - a) * inv_ac;
  const T t = (zeta >= (T)0 ? (T)1 : (T)-1) / (fabs(zeta) + sqrt((T)1 + zeta * zeta));
  cs = rsqrt((T)1 + t * t);
  const T sn_ac = cs * t * inv_ac;
  sne = Jac<T>::make(sn_ac * c.x, sn_ac * c.y);  // sn e^{i phi}
  return true;
}

template <class T, class C>
__device__ __forceinline__ void rotate_pair(C& xp, C& xq, T cs, C sne) {
  // xp' = cs xp - conj(sne) xq ; xq' = sne xp + cs xq
  const C np = csub(cscale(xp, cs), cmul(cconj(sne), xq));
  const C nq = cadd(cmul(sne, xp), cscale(xq, cs));
  xp = np;
  xq = nq;
}

__global__ void k_svd_prepare(const cplx* __restrict__ M, int rows, int cols, int orient,
                              cplx* __restrict__ X, cplx* __restrict__ V, int p, int q, int want_v) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nx = (long long)p * q;
  if (i < nx) {
    const int r = i % p;
    const int c = i / p;
    X[i] = (orient == 0) ? M[(long long)r * cols + c] : cconj(M[(long long)c * cols + r]);
  }
  if (want_v && i < (long long)q * q) {
    const int r = i % q, c = i / q;
    V[i] = mkc(r == c ? 1.0 : 0.0, 0.0);
  }
}

// One pair (P, Q) rotated by a whole block; returns true when a rotation with
// |sin theta| above 1e-8 was applied (kJacobiSmallAngle2).
template <class T>
__device__ bool jacobi_pair_block(typename Jac<T>::C* __restrict__ X, typename Jac<T>::C* __restrict__ V, int p, int q,
                                  int P, int Q, T tol, T floor2, int want_v) {
  typedef typename Jac<T>::C C;
  __shared__ T ra[8], rb[8];
  __shared__ C rc[8];
  __shared__ T s_cs;
  __shared__ C s_sne;
  __shared__ int s_do;
  C* xp = X + (long long)P * p;
  C* xq = X + (long long)Q * p;
  T a = 0, b = 0;
  C c = Jac<T>::make(0, 0);
  for (int r = threadIdx.x; r < p; r += blockDim.x) {
    const C u = xp[r], v = xq[r];
    a += cabs2(u);
    b += cabs2(v);
    cfma_conj(c, u, v);
  }
  const int warp = threadIdx.x >> 5;
  if (warp * 32 < p) {  // warps past the last row hold zeros: no FP64 reduction for them
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
  }
  if ((threadIdx.x & 31) == 0) {
    ra[warp] = a;
    rb[warp] = b;
    rc[warp] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    T A = 0, B = 0;
    C Cc = Jac<T>::make(0, 0);
    const int active = min((int)(blockDim.x >> 5), (p + 31) >> 5);  // the others hold exact zeros
    for (int u = 0; u < active; ++u) {
      A += ra[u];
      B += rb[u];
      Cc = cadd(Cc, rc[u]);
    }
    T cs;
    C sne;
    s_do = jacobi_params(A, B, Cc, tol, floor2, cs, sne) ? 1 : 0;
    s_cs = cs;
    s_sne = sne;
  }
  __syncthreads();
  const int doit = s_do;
  const T cs = s_cs;
  const C sne = s_sne;
  __syncthreads();  // the shared slots are reused by the next pair
  if (!doit) return false;
  for (int r = threadIdx.x; r < p; r += blockDim.x) {
    C u = xp[r], v = xq[r];
    rotate_pair(u, v, cs, sne);
    xp[r] = u;
    xq[r] = v;
  }
  const bool significant = cabs2(sne) > Jac<T>::small_angle2;
  if (want_v) {
    C* vp = V + (long long)P * q;
    C* vq = V + (long long)Q * q;
    for (int r = threadIdx.x; r < q; r += blockDim.x) {
      C u = vp[r], v = vq[r];
      rotate_pair(u, v, cs, sne);
      vp[r] = u;
      vq[r] = v;
    }
  }
  return significant;
}

// Grid-wide barrier for the cooperative path (all blocks co-resident by cooperative
// launch).  Every wait is bounded: after 2 s the barrier records an error and
// returns false, and the kernel unwinds.
struct GridBar {
  unsigned count;
  unsigned gen;
  int err;
  int rot[3];
};

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ bool grid_sync(GridBar* b, unsigned nblocks) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* vgen = &b->gen;
    volatile int* verr = &b->err;
    const unsigned g = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(&b->count, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(&b->count, 0u);
      __threadfence();
      atomicAdd(&b->gen, 1u);
    } else {
      const unsigned long long t0 = gtimer();
      while (*vgen == g) {
        if (*verr) {
          ok = 0;
          break;
        }
        if (gtimer() - t0 > 2000000000ull) {
          atomicExch(&b->err, 1);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// Medium path: one cooperative launch runs every sweep; blocks stride over the
// pairs of a round and meet at a grid barrier between rounds.
__global__ void __launch_bounds__(256)
    k_jacobi_coop(cplx* __restrict__ X, cplx* __restrict__ V, int p, int q, int qpad, double tol,
                  const double* __restrict__ fro2, int want_v, int max_sweeps, GridBar* bar,
                  int* __restrict__ sweeps_out) {
  const double floor2 = kJacobiFloor * (*fro2);
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (blockIdx.x == 0 && threadIdx.x == 0) bar->rot[(sweep + 1) % 3] = 0;
    for (int round = 0; round < qpad - 1; ++round) {
      for (int k = blockIdx.x; k < qpad / 2; k += gridDim.x) {
        int P, Q;
        rr_pair(round, k, qpad, P, Q);
        if (Q >= q) continue;
        if (jacobi_pair_block(X, V, p, q, P, Q, tol, floor2, want_v) && threadIdx.x == 0) bar->rot[sweep % 3] = 1;
      }
      if (!grid_sync(bar, gridDim.x)) return;
    }
    const int rot = ((volatile int*)bar->rot)[sweep % 3];
    if (!rot) {
      if (blockIdx.x == 0 && threadIdx.x == 0) *sweeps_out = sweep + 1;
      return;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *sweeps_out = max_sweeps + 1;
}

// Small path: the whole problem in shared memory, one block, warps own pairs.
__global__ void __launch_bounds__(256)
    k_jacobi_small(cplx* __restrict__ Xg, cplx* __restrict__ Vg, int p, int q, int qpad,
                   double tol, const double* __restrict__ fro2, int want_v, int max_sweeps,
                   int* __restrict__ sweeps_out) {
  const double floor2 = kJacobiFloor * (*fro2);
  extern __shared__ cplx sm[];
  cplx* X = sm;
  cplx* V = sm + (long long)p * q;
  __shared__ int s_rot;
  const int nx = p * q, nv = want_v ? q * q : 0;
  for (int e = threadIdx.x; e < nx; e += blockDim.x) X[e] = Xg[e];
  for (int e = threadIdx.x; e < nv; e += blockDim.x) V[e] = Vg[e];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    for (int round = 0; round < qpad - 1; ++round) {
      for (int k = warp; k < qpad / 2; k += nw) {
        int P, Q;
        rr_pair(round, k, qpad, P, Q);
        if (Q >= q) continue;
        cplx* xp = X + P * p;
        cplx* xq = X + Q * p;
        double a = 0.0, b = 0.0;
        cplx c = mkc(0.0, 0.0);
        for (int r = lane; r < p; r += 32) {
          const cplx u = xp[r], v = xq[r];
          a += cabs2(u);
          b += cabs2(v);
          cfma_conj(c, u, v);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          a += __shfl_xor_sync(0xffffffffu, a, o);
          b += __shfl_xor_sync(0xffffffffu, b, o);
          c.x += __shfl_xor_sync(0xffffffffu, c.x, o);
          c.y += __shfl_xor_sync(0xffffffffu, c.y, o);
        }
        double cs;
        cplx sne;
        if (!jacobi_params(a, b, c, tol, floor2, cs, sne)) continue;
        if (lane == 0 && cabs2(sne) > kJacobiSmallAngle2) s_rot = 1;
        for (int r = lane; r < p; r += 32) {
          cplx u = xp[r], v = xq[r];
          rotate_pair(u, v, cs, sne);
          xp[r] = u;
          xq[r] = v;
        }
        if (want_v) {
          cplx* vp = V + P * q;
          cplx* vq = V + Q * q;
          for (int r = lane; r < q; r += 32) {
            cplx u = vp[r], v = vq[r];
            rotate_pair(u, v, cs, sne);
            vp[r] = u;
            vq[r] = v;
          }
        }
      }
      __syncthreads();
    }
    const int rot = s_rot;
    __syncthreads();
    if (!rot) break;
  }
  for (int e = threadIdx.x; e < nx; e += blockDim.x) Xg[e] = X[e];
  for (int e = threadIdx.x; e < nv; e += blockDim.x) Vg[e] = V[e];
  if (threadIdx.x == 0) *sweeps_out = sweep + 1;
}

__global__ void k_fro2(const cplx* __restrict__ X, long long n, double* __restrict__ out) {
  __shared__ double red[8];
  double a = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) a += cabs2(X[i]);
  a = warp_sum(a);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int u = 0; u < (int)(blockDim.x >> 5); ++u) t += red[u];
    *out = t;
  }
}

__global__ void k_colnorms(const cplx* __restrict__ X, int p, int q, double* __restrict__ s) {
  const int j = blockIdx.x;
  double a = 0.0;
  for (int r = threadIdx.x; r < p; r += blockDim.x) a += cabs2(X[(long long)j * p + r]);
  __shared__ double red[8];
  a = warp_sum(a);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int u = 0; u < (int)(blockDim.x >> 5); ++u) t += red[u];
    s[j] = sqrt(t);
  }
}

// U[i*keep + r] from column perm[r] of a column-major (ld x *) matrix,
// divided by s_sorted[r] when `normalise`.
__global__ void k_gather_cols(const cplx* __restrict__ src, long long ld, int nrows,
                              const int* __restrict__ perm, const double* __restrict__ s_sorted,
                              int keep, int normalise, int conj_out, int transpose_out,
                              cplx* __restrict__ dst) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)nrows * keep) return;
  const int r = e % keep;
  const int i = e / keep;
  cplx v = src[(long long)perm[r] * ld + i];
  if (normalise) v = cscale(v, 1.0 / s_sorted[r]);
  if (conj_out) v = cconj(v);
  if (transpose_out)
    dst[(long long)r * nrows + i] = v;  // keep x nrows
  else
    dst[(long long)i * keep + r] = v;   // nrows x keep
}
}  // namespace

void svd_jacobi_keep(cudaStream_t st, DevicePool* pool, const cplx* M, int rows, int cols,
                     int (*select)(const std::vector<double>& s, void* ctx), void* ctx,
                     SvdOut& out, bool want_u, bool want_v) {
  out.rows = rows;
  out.cols = cols;
  out.s.clear();
  out.rank = 0;
  out.U.release();
  out.Vh.release();
  if (rows == 0 || cols == 0) return;
  const int orient = rows >= cols ? 0 : 1;
  const int p = orient == 0 ? rows : cols;
  const int q = orient == 0 ? cols : rows;
  const int qpad = q + (q & 1);
  atomic_max(g_svd_counters.max_q, q);
  // accumulated rotations are needed for V (orient 0) or U (orient 1)
  const bool need_acc = orient == 0 ? want_v : want_u;
  DArr X(pool, (size_t)p * q), Vx(pool, need_acc ? (size_t)q * q : 1);
  {
    const long long n = std::max<long long>((long long)p * q, need_acc ? (long long)q * q : 0);
    k_svd_prepare<<<ceil_div(n, 256), 256, 0, st>>>(M, rows, cols, orient, X.data(), Vx.data(), p, q,
                                                    need_acc ? 1 : 0);
    TDVP_CHECK_LAUNCH();
  }
  const double tol = std::max(1e-15, std::sqrt((double)p) * 2.2e-16);
  const int max_sweeps = 60;
  const size_t small_bytes = ((size_t)p * q + (need_acc ? (size_t)q * q : 0)) * sizeof(cplx);
  int* d_flag = nullptr;
  TDVP_CUDA(cudaMallocAsync(&d_flag, sizeof(int) + sizeof(double) * 2, st));
  double* d_fro2 = reinterpret_cast<double*>(d_flag + 2);
  k_fro2<<<1, 256, 0, st>>>(X.data(), (long long)p * q, d_fro2);
  TDVP_CHECK_LAUNCH();
  int sweeps = 0;
  if (q > 1) {
    if (small_bytes <= 96 * 1024) {
      static const bool attr_set = [] {
        TDVP_CUDA(cudaFuncSetAttribute(k_jacobi_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       96 * 1024));
        return true;
      }();
      (void)attr_set;
      k_jacobi_small<<<1, 256, small_bytes, st>>>(X.data(), Vx.data(), p, q, qpad, tol, d_fro2,
                                                   need_acc ? 1 : 0, max_sweeps, d_flag);
      TDVP_CHECK_LAUNCH();
      TDVP_CUDA(cudaMemcpyAsync(&sweeps, d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
      TDVP_CUDA(cudaStreamSynchronize(st));
      if (sweeps > max_sweeps) {
        cudaFreeAsync(d_flag, st);
        throw TdvpError(TDVP_ERR_SVD_NOT_CONVERGED, "Jacobi SVD did not converge");
      }
    } else {
      static const int coop_blocks = [] {
        int dev = 0, sms = 0, per_sm = 0;
        TDVP_CUDA(cudaGetDevice(&dev));
        TDVP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        TDVP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi_coop, 256, 0));
        return std::max(1, sms * std::max(1, per_sm));
      }();
      const int nblk = std::max(1, std::min(qpad / 2, coop_blocks));
      GridBar* bar = nullptr;
      TDVP_CUDA(cudaMallocAsync(&bar, sizeof(GridBar), st));
      TDVP_CUDA(cudaMemsetAsync(bar, 0, sizeof(GridBar), st));
      cplx* xp = X.data();
      cplx* vp = Vx.data();
      int pp = p, qq = q, qp = qpad, wv = need_acc ? 1 : 0, ms = max_sweeps;
      double tl = tol;
      const double* fr = d_fro2;
      void* args[] = {&xp, &vp, &pp, &qq, &qp, &tl, &fr, &wv, &ms, &bar, &d_flag};
      TDVP_CUDA(cudaLaunchCooperativeKernel((void*)k_jacobi_coop, dim3(nblk), dim3(256), args, 0, st));
      g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
      GridBar hb;
      TDVP_CUDA(cudaMemcpyAsync(&sweeps, d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
      TDVP_CUDA(cudaMemcpyAsync(&hb, bar, sizeof(GridBar), cudaMemcpyDeviceToHost, st));
      TDVP_CUDA(cudaStreamSynchronize(st));
      TDVP_CUDA(cudaFreeAsync(bar, st));
      if (hb.err) {
        cudaFreeAsync(d_flag, st);
        throw TdvpError(TDVP_ERR_TIMEOUT, "Jacobi SVD: a grid barrier wait ran out");
      }
      if (sweeps > max_sweeps) {
        cudaFreeAsync(d_flag, st);
        throw TdvpError(TDVP_ERR_SVD_NOT_CONVERGED, "Jacobi SVD did not converge");
      }
    }
  }
  TDVP_CUDA(cudaFreeAsync(d_flag, st));
  out.sweeps = sweeps;
  g_svd_counters.sweeps += sweeps;
  atomic_max(g_svd_counters.max_sweeps, sweeps);
  // singular values = column norms
  double* d_s = nullptr;
  TDVP_CUDA(cudaMallocAsync(&d_s, sizeof(double) * q, st));
  k_colnorms<<<q, 256, 0, st>>>(X.data(), p, q, d_s);
  TDVP_CHECK_LAUNCH();
  std::vector<double> s(q);
  TDVP_CUDA(cudaMemcpyAsync(s.data(), d_s, sizeof(double) * q, cudaMemcpyDeviceToHost, st));
  TDVP_CUDA(cudaStreamSynchronize(st));
  for (double v : s)
    tdvp_require(std::isfinite(v), TDVP_ERR_NONFINITE, "SVD: non-finite singular value");
  std::vector<int> perm(q);
  std::iota(perm.begin(), perm.end(), 0);
  std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return s[a] > s[b]; });
  out.s.resize(q);
  for (int r = 0; r < q; ++r) out.s[r] = s[perm[r]];
  const int keep = std::max(0, std::min(q, select(out.s, ctx)));
  out.rank = keep;
  if (keep == 0) {
    cudaFreeAsync(d_s, st);
    return;
  }
  int* d_perm = nullptr;
  double* d_ss = nullptr;
  TDVP_CUDA(cudaMallocAsync(&d_perm, sizeof(int) * keep, st));
  TDVP_CUDA(cudaMallocAsync(&d_ss, sizeof(double) * keep, st));
  TDVP_CUDA(cudaMemcpyAsync(d_perm, perm.data(), sizeof(int) * keep, cudaMemcpyHostToDevice, st));
  TDVP_CUDA(cudaMemcpyAsync(d_ss, out.s.data(), sizeof(double) * keep, cudaMemcpyHostToDevice, st));
  if (want_u) {
    out.U.reset(pool, (size_t)rows * keep);
    const long long n = (long long)rows * keep;
    if (orient == 0)  // U = X[:, perm] / s
      k_gather_cols<<<ceil_div(n, 256), 256, 0, st>>>(X.data(), p, rows, d_perm, d_ss, keep, 1, 0, 0,
                                                      out.U.data());
    else  // U = Vx[:, perm]
      k_gather_cols<<<ceil_div(n, 256), 256, 0, st>>>(Vx.data(), q, rows, d_perm, d_ss, keep, 0, 0, 0,
                                                      out.U.data());
    TDVP_CHECK_LAUNCH();
  }
  if (want_v) {
    out.Vh.reset(pool, (size_t)keep * cols);
    const long long n = (long long)cols * keep;
    if (orient == 0)  // Vh[r][j] = conj(Vx[j, perm r])
      k_gather_cols<<<ceil_div(n, 256), 256, 0, st>>>(Vx.data(), q, cols, d_perm, d_ss, keep, 0, 1, 1,
                                                      out.Vh.data());
    else  // Vh[r][j] = conj(X[j, perm r]) / s
      k_gather_cols<<<ceil_div(n, 256), 256, 0, st>>>(X.data(), p, cols, d_perm, d_ss, keep, 1, 1, 1,
                                                      out.Vh.data());
    TDVP_CHECK_LAUNCH();
  }
  TDVP_CUDA(cudaFreeAsync(d_perm, st));
  TDVP_CUDA(cudaFreeAsync(d_ss, st));
  TDVP_CUDA(cudaFreeAsync(d_s, st));
}

// ============================================================================
// small helpers
// ============================================================================
namespace {
__global__ void k_copy_block(cplx* __restrict__ dst, long long ldd, const cplx* __restrict__ src,
                             long long lds, int rows, int cols) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)rows * cols) return;
  const int r = e / cols, c = e % cols;
  dst[r * ldd + c] = src[r * lds + c];
}
}  // namespace

void copy_block(cudaStream_t st, cplx* dst, long long ldd, const cplx* src, long long lds, int rows,
                int cols) {
  const long long n = (long long)rows * cols;
  if (!n) return;
  k_copy_block<<<ceil_div(n, 256), 256, 0, st>>>(dst, ldd, src, lds, rows, cols);
  TDVP_CHECK_LAUNCH();
}

// ============================================================================
// Block-structured SVD.  Quantum numbers that the dynamics conserves (S^z for
// the Heisenberg models) make every matrix factorised by the method block
// diagonal up to a permutation, with the forbidden entries exactly zero in
// floating point (they are sums of products with a zero factor).  Rows and
// columns linked by nonzero entries form connected components; each component
// is an independent, much smaller SVD.  Singular values from all components are
// merged and sorted, so the selection rule sees the same spectrum as the dense
// SVD; U and Vh are scattered back in that global order.
// ============================================================================
namespace {
__global__ void k_nonzero_mask(const cplx* __restrict__ M, int rows, int cols, int words,
                               unsigned* __restrict__ mask) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)rows * words) return;
  const int w = e % words;
  const long long r = e / words;
  unsigned bits = 0;
  for (int b = 0; b < 32; ++b) {
    const int c = w * 32 + b;
    if (c < cols) {
      const cplx v = M[r * cols + c];
      if (v.x != 0.0 || v.y != 0.0) bits |= 1u << b;
    }
  }
  mask[e] = bits;
}



// Batched small blocks: descriptor per block.  Block b is gathered as the column-major
// working matrix X_b (p x q, p >= q; transposed and conjugated when orient = 1) and
// solved by one CTA with X_b, V_b in shared memory.
struct BlkDesc {
  int orient, p, q, nr, nc;  // nr/nc: rows/cols of the block in M
  long long x_off, v_off;
  int s_off, r_off, c_off;
  int need_v;  // the accumulated rotations are read (V for orient 0, U for orient 1)
};

__global__ void k_gather_batched(const cplx* __restrict__ M, int cols, const BlkDesc* __restrict__ desc,
                                 const int* __restrict__ ridx, const int* __restrict__ cidx, cplx* __restrict__ X,
                                 cplx* __restrict__ V) {
  const BlkDesc d = desc[blockIdx.x];
  cplx* Xb = X + d.x_off;
  cplx* Vb = V + d.v_off;
  for (int e = threadIdx.x; e < d.p * d.q; e += blockDim.x) {
    const int i = e % d.p, j = e / d.p;  // X_b[i + j p]
    cplx v;
    if (d.orient == 0)
      v = M[(long long)ridx[d.r_off + i] * cols + cidx[d.c_off + j]];
    else
      v = cconj(M[(long long)ridx[d.r_off + j] * cols + cidx[d.c_off + i]]);
    Xb[e] = v;
  }
  for (int e = threadIdx.x; e < d.q * d.q; e += blockDim.x) Vb[e] = mkc((e % d.q) == (e / d.q) ? 1.0 : 0.0, 0.0);
}

template <class T>
__global__ void __launch_bounds__(256)
    k_jacobi_batched(typename Jac<T>::C* __restrict__ X, typename Jac<T>::C* __restrict__ V,
                     const BlkDesc* __restrict__ desc, int max_sweeps, double* __restrict__ s_out,
                     int* __restrict__ bad) {
  typedef typename Jac<T>::C C;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C* sm = reinterpret_cast<C*>(sm_raw);
  __shared__ int s_rot;
  __shared__ T s_fro[8];
  const BlkDesc d = desc[blockIdx.x];
  const int p = d.p, q = d.q, qpad = q + (q & 1);
  C* Xs = sm;
  C* Vs = sm + (long long)p * q;
  C* Xg = X + d.x_off;
  C* Vg = V + d.v_off;
  T f = 0;
  for (int e = threadIdx.x; e < p * q; e += blockDim.x) {
    Xs[e] = Xg[e];
    f += cabs2(Xs[e]);
  }
  for (int e = threadIdx.x; e < q * q; e += blockDim.x) Vs[e] = Vg[e];
  f = warp_sum(f);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (lane == 0) s_fro[warp] = f;
  __syncthreads();
  T fro2 = 0;
  for (int u = 0; u < nw; ++u) fro2 += s_fro[u];
  const T floor2 = (T)kJacobiFloor * fro2;
  const T tol = fmax(Jac<T>::tol_min, sqrt((T)p) * Jac<T>::eps);
  int sweep = 0;
  for (; sweep < max_sweeps && q > 1; ++sweep) {
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    for (int round = 0; round < qpad - 1; ++round) {
      for (int k = warp; k < qpad / 2; k += nw) {
        int P, Q;
        rr_pair(round, k, qpad, P, Q);
        if (Q >= q) continue;
        C* xp = Xs + P * p;
        C* xq = Xs + Q * p;
        T a = 0, b = 0;
        C c = Jac<T>::make(0, 0);
        for (int r = lane; r < p; r += 32) {
          const C u = xp[r], v = xq[r];
          a += cabs2(u);
          b += cabs2(v);
          cfma_conj(c, u, v);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          a += __shfl_xor_sync(0xffffffffu, a, o);
          b += __shfl_xor_sync(0xffffffffu, b, o);
          c.x += __shfl_xor_sync(0xffffffffu, c.x, o);
          c.y += __shfl_xor_sync(0xffffffffu, c.y, o);
        }
        T cs;
        C sne;
        if (!jacobi_params(a, b, c, tol, floor2, cs, sne)) continue;
        if (lane == 0 && cabs2(sne) > Jac<T>::small_angle2) s_rot = 1;
        for (int r = lane; r < p; r += 32) {
          C u = xp[r], v = xq[r];
          rotate_pair(u, v, cs, sne);
          xp[r] = u;
          xq[r] = v;
        }
        if (d.need_v) {
          C* vp = Vs + P * q;
          C* vq = Vs + Q * q;
          for (int r = lane; r < q; r += 32) {
            C u = vp[r], v = vq[r];
            rotate_pair(u, v, cs, sne);
            vp[r] = u;
            vq[r] = v;
          }
        }
      }
      __syncthreads();
    }
    const int rot = s_rot;
    __syncthreads();
    if (!rot) break;
  }
  if (threadIdx.x == 0) {
    if (sweep >= max_sweeps) bad[0] = 1;
    atomicMax(&bad[1], sweep);  // sweep statistics: largest and total
    atomicAdd(&bad[2], sweep);
  }
  for (int e = threadIdx.x; e < p * q; e += blockDim.x) Xg[e] = Xs[e];
  for (int e = threadIdx.x; e < q * q; e += blockDim.x) Vg[e] = Vs[e];
  __syncthreads();
  for (int j = warp; j < q; j += nw) {
    T t = 0;
    for (int r = lane; r < p; r += 32) t += cabs2(Xs[j * p + r]);
    t = warp_sum(t);
    if (lane == 0) s_out[d.s_off + j] = sqrt((double)t);
  }
}

// Hermitian positive semidefinite blocks: pivoted Cholesky, in place, one CTA per
// block.  X_b (n x n, column-major) becomes L (n x rank) with A[piv][:, piv] = L L^H;
// elimination stops when the largest remaining diagonal entry is below
// rel_floor times the block's largest diagonal entry, and desc[b].q becomes the
// rank.  The one-sided Jacobi SVD of L then gives the eigenvectors (its left
// singular vectors) and eigenvalues (singular values squared) of the block.  L's
// singular values span half the decades of A's eigenvalues, so the sweeps that
// follow are far fewer than those of a Jacobi SVD of A itself.
__global__ void __launch_bounds__(256)
    k_pchol_batched(cplx* __restrict__ X, BlkDesc* __restrict__ desc, int* __restrict__ piv, double rel_floor) {
  __shared__ double s_val[8];
  __shared__ int s_idx[8];
  __shared__ double s_thr, s_piv;
  __shared__ int s_k;
  BlkDesc& dref = desc[blockIdx.x];
  const int n = dref.p;
  cplx* A = X + dref.x_off;
  int* pv = piv + dref.r_off;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int i = tid; i < n; i += blockDim.x) pv[i] = i;
  // largest diagonal entry from row `from` on: value and index (block-wide)
  auto argmax_diag = [&](int from, double& val, int& idx) {
    double v = -1.0;
    int k = from;
    for (int i = from + tid; i < n; i += blockDim.x) {
      const double t = A[(long long)i * n + i].x;
      if (t > v) {
        v = t;
        k = i;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, v, o);
      const int ok = __shfl_xor_sync(0xffffffffu, k, o);
      if (ov > v || (ov == v && ok < k)) {
        v = ov;
        k = ok;
      }
    }
    if (lane == 0) {
      s_val[warp] = v;
      s_idx[warp] = k;
    }
    __syncthreads();
    if (tid == 0) {
      double bv = s_val[0];
      int bk = s_idx[0];
      for (int u = 1; u < nw; ++u)
        if (s_val[u] > bv || (s_val[u] == bv && s_idx[u] < bk)) {
          bv = s_val[u];
          bk = s_idx[u];
        }
      s_piv = bv;
      s_k = bk;
    }
    __syncthreads();
    val = s_piv;
    idx = s_k;
    __syncthreads();
  };
  double dmax;
  int k0;
  argmax_diag(0, dmax, k0);
  if (tid == 0) s_thr = rel_floor * dmax;
  __syncthreads();
  const double thr = s_thr;
  int rank = 0;
  for (int j = 0; j < n; ++j) {
    double val;
    int k;
    argmax_diag(j, val, k);
    if (!(val > thr)) break;  // uniform: every thread read the same shared values
    if (k != j) {
      for (int l = tid; l < n; l += blockDim.x) {  // rows j and k, every column
        const cplx t = A[(long long)l * n + j];
        A[(long long)l * n + j] = A[(long long)l * n + k];
        A[(long long)l * n + k] = t;
      }
      __syncthreads();
      for (int i = tid; i < n; i += blockDim.x) {  // columns j and k, every row
        const cplx t = A[(long long)j * n + i];
        A[(long long)j * n + i] = A[(long long)k * n + i];
        A[(long long)k * n + i] = t;
      }
      if (tid == 0) {
        const int t = pv[j];
        pv[j] = pv[k];
        pv[k] = t;
      }
      __syncthreads();
    }
    const double ljj = sqrt(A[(long long)j * n + j].x);
    const double inv = 1.0 / ljj;
    __syncthreads();
    for (int i = tid; i < n; i += blockDim.x) {
      cplx& a = A[(long long)j * n + i];
      if (i > j)
        a = cscale(a, inv);
      else if (i < j)
        a = mkc(0.0, 0.0);
      else
        a = mkc(ljj, 0.0);
    }
    __syncthreads();
    const int m = n - j - 1;
    for (long long e = tid; e < (long long)m * m; e += blockDim.x) {
      const int i = j + 1 + (int)(e % m), l = j + 1 + (int)(e / m);
      const cplx li = A[(long long)j * n + i], ll = A[(long long)j * n + l];
      cplx& a = A[(long long)l * n + i];
      a = csub(a, cmul(li, cconj(ll)));
    }
    __syncthreads();
    rank = j + 1;
  }
  if (tid == 0) dref.q = rank;
}

// One kept singular triple per CTA: U[:, k] over the block's rows, Vh[k, :] over its columns.
struct SelEntry {
  int blk, j, k;
  double s;
};
__global__ void k_scatter_batched(const cplx* __restrict__ X, const cplx* __restrict__ V,
                                  const BlkDesc* __restrict__ desc, const SelEntry* __restrict__ sel,
                                  const int* __restrict__ ridx, const int* __restrict__ cidx, cplx* __restrict__ U,
                                  int keep, cplx* __restrict__ Vh, int cols, int want_u, int want_v,
                                  const int* __restrict__ piv) {
  const SelEntry e = sel[blockIdx.x];
  const BlkDesc d = desc[e.blk];
  const cplx* Xb = X + d.x_off + (long long)e.j * d.p;  // column j of X_b
  const cplx* Vb = V + d.v_off + (long long)e.j * d.q;  // column j of V_b
  const double inv = 1.0 / e.s;
  if (want_u)
    for (int i = threadIdx.x; i < d.nr; i += blockDim.x) {
      const cplx v = (d.orient == 0) ? cscale(Xb[i], inv) : Vb[i];
      const int li = piv ? piv[d.r_off + i] : i;  // row i of a pivoted factor is local row piv[i]
      U[(long long)ridx[d.r_off + li] * keep + e.k] = v;
    }
  if (want_v)
    for (int i = threadIdx.x; i < d.nc; i += blockDim.x) {
      const cplx v = (d.orient == 0) ? cconj(Vb[i]) : cscale(cconj(Xb[i]), inv);
      Vh[(long long)e.k * cols + cidx[d.c_off + i]] = v;
    }
}

struct DSU {
  std::vector<int> p;
  explicit DSU(int n) : p(n) { std::iota(p.begin(), p.end(), 0); }
  int find(int x) {
    while (p[x] != x) {
      p[x] = p[p[x]];
      x = p[x];
    }
    return x;
  }
  void unite(int a, int b) {
    a = find(a);
    b = find(b);
    if (a != b) p[std::max(a, b)] = std::min(a, b);
  }
};

}  // namespace

SvdCounters g_svd_counters;
thread_local Tracer* t_tracer = nullptr;
std::atomic<long long> g_kernel_launches{0};

// Barrier of the n CTAs that work on one block (all co-resident: cooperative launch).
// The arrival counter only grows: the e-th barrier of a group completes when it reaches
// e * n, so no CTA has to reset it and the waiters need no second signal.  Thread 0
// arrives with a release add (ordering the block's writes, which bar.sync has ordered
// before it) and polls with acquire loads (ordering the block's later reads, which the
// closing bar.sync passes on).  Bounded like grid_sync: every 64 polls the waiter checks
// the error word of the launch (gerr) and its 2 s limit; either makes it return false.
// `epoch` counts this CTA's barriers (the same sequence in every CTA of the group).
__device__ __forceinline__ void red_add_release_gpu(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ bool group_sync(GridBar* b, unsigned n, int* gerr, unsigned& epoch) {
  __shared__ int ok;
  __syncthreads();
  ++epoch;
  if (threadIdx.x == 0) {
    ok = 1;
    if (n > 1) {
      const unsigned target = epoch * n;
      red_add_release_gpu(&b->count, 1u);
      const unsigned long long t0 = gtimer();
      unsigned polls = 0;
      while ((int)(ld_acquire_gpu(&b->count) - target) < 0) {
        if ((++polls & 63u) == 0u) {
          if (*(volatile int*)gerr) {
            ok = 0;
            break;
          }
          if (gtimer() - t0 > 2000000000ull) {
            atomicExch(gerr, 1);
            ok = 0;
            break;
          }
        }
      }
    }
  }
  __syncthreads();
  return ok != 0;
}

// Many blocks at once over the whole GPU.  The FP64 pipe of one SM is a small
// fraction of the device's (about 8 GFLOP/s of 1.2 TFLOP/s on this part), so a block
// wider than a few dozen columns must not sit on one SM.  One cooperative launch
// runs the blocks of one call, each on its own group of CTAs.  Blocks are independent,
// so a group synchronises only its own CTAs between rounds (few participants, no
// waiting for wider blocks) and leaves as soon as its block has converged.  Group
// b holds CTAs [cta_off[b], cta_off[b+1]); its CTA lc takes the pairs lc, lc + n_b, ...
// of every round.  flags per block: rot[3] | sweeps; bars: one barrier per block;
// stat: bad, max sweeps, total sweeps (atomics); gerr: any barrier that ran out.
template <class T>
__global__ void __launch_bounds__(256)
    k_jacobi_groups(typename Jac<T>::C* __restrict__ X, typename Jac<T>::C* __restrict__ V,
                    const BlkDesc* __restrict__ desc, const int* __restrict__ cta_off, int nblk, int max_sweeps,
                    double* __restrict__ fro2, int* __restrict__ flags, GridBar* __restrict__ bars,
                    int* __restrict__ gerr, double* __restrict__ s_out, int* __restrict__ stat) {
  typedef typename Jac<T>::C C;
  __shared__ T red[8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int lo = 0, hi = nblk - 1;  // the block whose group holds this CTA
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (cta_off[mid] <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  const int b = lo;
  const int lc = blockIdx.x - cta_off[b];
  const unsigned n_b = (unsigned)(cta_off[b + 1] - cta_off[b]);
  const BlkDesc d = desc[b];
  int* rot = flags + 4 * b;
  GridBar* bar = bars + b;
  if (lc == 0) {
    const C* Xb = X + d.x_off;
    T f = 0;
    for (long long e = threadIdx.x; e < (long long)d.p * d.q; e += blockDim.x) f += cabs2(Xb[e]);
    f = warp_sum(f);
    if (lane == 0) red[warp] = f;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int u = 0; u < (int)(blockDim.x >> 5); ++u) t += red[u];
      fro2[b] = t;
      rot[0] = rot[1] = rot[2] = 0;
    }
    __syncthreads();
  }
  unsigned epoch = 0;
  if (!group_sync(bar, n_b, gerr, epoch)) return;
  const T floor2 = (T)(kJacobiFloor * fro2[b]);
  const T tol = fmax(Jac<T>::tol_min, sqrt((T)d.p) * Jac<T>::eps);
  const int qpad = d.q + (d.q & 1);
  int sweep = 0;
  bool converged = d.q <= 1;
  for (; sweep < max_sweeps && !converged; ++sweep) {
    if (lc == 0 && threadIdx.x == 0) rot[(sweep + 1) % 3] = 0;
    for (int round = 0; round < qpad - 1; ++round) {
      for (int k = lc; k < qpad / 2; k += n_b) {
        int P, Q;
        rr_pair(round, k, qpad, P, Q);
        if (Q >= d.q) continue;
        if (jacobi_pair_block(X + d.x_off, V + d.v_off, d.p, d.q, P, Q, tol, floor2, d.need_v) && threadIdx.x == 0)
          rot[sweep % 3] = 1;
      }
      if (!group_sync(bar, n_b, gerr, epoch)) return;
    }
    converged = ((volatile int*)rot)[sweep % 3] == 0;  // every CTA of the group reads it after the barrier
  }
  // singular values: column norms, spread over the group
  for (int j = lc; j < d.q; j += n_b) {
    const C* col = X + d.x_off + (long long)j * d.p;
    T t = 0;
    for (int r = threadIdx.x; r < d.p; r += blockDim.x) t += cabs2(col[r]);
    t = warp_sum(t);
    if (lane == 0) red[warp] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
      double u = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) u += red[w];
      s_out[d.s_off + j] = sqrt(u);
    }
    __syncthreads();
  }
  if (lc == 0 && threadIdx.x == 0) {
    const int used = converged ? sweep : max_sweeps;
    if (!converged) atomicExch(&stat[0], 1);
    atomicMax(&stat[1], used);
    atomicAdd(&stat[2], used);
  }
}

// Pivoted Cholesky of Hermitian PSD blocks with one group of CTAs per block (cooperative
// launch), for blocks too wide for one SM's FP64 pipe.  The block is column-major
// (entry (r, c) at c n + r); CTA lc of a group of G owns the columns c = lc (mod G).  Pivot
// step j: every CTA posts the largest diagonal entry of its own columns from row j on
// (ties to the smaller index); after a group barrier all read the same pivot k.  CTA 0
// swaps columns j and k whole, then rows j and k inside them, and forms column j of the
// factor; the other CTAs swap rows j and k in their own columns.  After a second barrier
// every CTA updates its own trailing columns with column j.  Each entry sees the
// arithmetic of k_pchol_batched, so the factor and the pivots are the same.
__global__ void __launch_bounds__(256)
    k_pchol_groups(cplx* __restrict__ X, BlkDesc* __restrict__ desc, int* __restrict__ piv,
                   const int* __restrict__ cta_off, int nblk, double rel_floor, double* __restrict__ pval,
                   int* __restrict__ pidx, GridBar* __restrict__ bars, int* __restrict__ gerr) {
  __shared__ double s_val[8];
  __shared__ int s_idx[8];
  int lo = 0, hi = nblk - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (cta_off[mid] <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  const int b = lo;
  const int c0 = cta_off[b];
  const int lc = blockIdx.x - c0;
  const int G = cta_off[b + 1] - c0;
  GridBar* bar = bars + b;
  const int n = desc[b].p;
  cplx* A = X + desc[b].x_off;
  int* pv = piv + desc[b].r_off;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  unsigned epoch = 0;
  if (lc == 0)
    for (int i = tid; i < n; i += blockDim.x) pv[i] = i;
  // first index >= from owned by this CTA
  auto first_own = [&](int from) { return from + ((lc - from % G) % G + G) % G; };
  // posts (largest diagonal entry of the own columns i >= from, its index); n = none
  auto post_argmax = [&](int from) {
    double v = -1.0;
    int k = n;
    for (int i = first_own(from) + tid * G; i < n; i += blockDim.x * G) {
      const double t = A[(long long)i * n + i].x;
      if (t > v || (t == v && i < k)) {
        v = t;
        k = i;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, v, o);
      const int ok = __shfl_xor_sync(0xffffffffu, k, o);
      if (ov > v || (ov == v && ok < k)) {
        v = ov;
        k = ok;
      }
    }
    if (lane == 0) {
      s_val[warp] = v;
      s_idx[warp] = k;
    }
    __syncthreads();
    if (tid == 0) {
      double bv = s_val[0];
      int bk = s_idx[0];
      for (int u = 1; u < nw; ++u)
        if (s_val[u] > bv || (s_val[u] == bv && s_idx[u] < bk)) {
          bv = s_val[u];
          bk = s_idx[u];
        }
      pval[blockIdx.x] = bv;
      pidx[blockIdx.x] = bk;
    }
  };
  // the group's pivot from the posted partials (every thread, same order, same result)
  auto read_argmax = [&](double& val, int& idx) {
    double bv = -1.0;
    int bk = n;
    for (int u = 0; u < G; ++u) {
      const double t = ((volatile double*)pval)[c0 + u];
      const int kk = ((volatile int*)pidx)[c0 + u];
      if (t > bv || (t == bv && kk < bk)) {
        bv = t;
        bk = kk;
      }
    }
    val = bv;
    idx = bk;
  };
  post_argmax(0);
  if (!group_sync(bar, (unsigned)G, gerr, epoch)) return;
  double dmax;
  int k0;
  read_argmax(dmax, k0);
  const double thr = rel_floor * dmax;
  int rank = 0;
  for (int j = 0; j < n; ++j) {
    double val = dmax;
    int k = k0;
    if (j > 0) {
      __syncthreads();  // the own trailing columns are complete
      post_argmax(j);
      if (!group_sync(bar, (unsigned)G, gerr, epoch)) return;
      read_argmax(val, k);
    }
    if (!(val > thr)) break;  // uniform over the group: every CTA read the same partials
    if (k != j)
      for (int c = lc + tid * G; c < n; c += blockDim.x * G) {  // rows j and k, own columns
        if (c == j || c == k) continue;
        const cplx t = A[(long long)c * n + j];
        A[(long long)c * n + j] = A[(long long)c * n + k];
        A[(long long)c * n + k] = t;
      }
    if (lc == 0) {
      if (k != j) {
        for (int r = tid; r < n; r += blockDim.x) {  // columns j and k, every row
          const cplx t = A[(long long)j * n + r];
          A[(long long)j * n + r] = A[(long long)k * n + r];
          A[(long long)k * n + r] = t;
        }
        __syncthreads();
        if (tid == 0) {  // rows j and k inside columns j and k
          cplx t = A[(long long)j * n + j];
          A[(long long)j * n + j] = A[(long long)j * n + k];
          A[(long long)j * n + k] = t;
          t = A[(long long)k * n + j];
          A[(long long)k * n + j] = A[(long long)k * n + k];
          A[(long long)k * n + k] = t;
          const int tp = pv[j];
          pv[j] = pv[k];
          pv[k] = tp;
        }
        __syncthreads();
      }
      const double ljj = sqrt(A[(long long)j * n + j].x);
      const double inv = 1.0 / ljj;
      __syncthreads();
      for (int i = tid; i < n; i += blockDim.x) {
        cplx& a = A[(long long)j * n + i];
        if (i > j)
          a = cscale(a, inv);
        else if (i < j)
          a = mkc(0.0, 0.0);
        else
          a = mkc(ljj, 0.0);
      }
    }
    if (!group_sync(bar, (unsigned)G, gerr, epoch)) return;  // column j is complete
    const int m = n - j - 1;
    const int l0 = first_own(j + 1);
    const int nc = l0 < n ? (n - 1 - l0) / G + 1 : 0;
    for (long long e = tid; e < (long long)m * nc; e += blockDim.x) {
      const int i = j + 1 + (int)(e % m), l = l0 + (int)(e / m) * G;
      const cplx li = A[(long long)j * n + i], ll = A[(long long)j * n + l];
      cplx& a = A[(long long)l * n + i];
      a = csub(a, cmul(li, cconj(ll)));
    }
    rank = j + 1;
  }
  if (lc == 0 && tid == 0) desc[b].q = rank;
}

namespace {
// Host side of k_jacobi_groups: CTA groups per block, one cooperative launch, bounded-wait check.
// d_stat receives {bad, max sweeps, total sweeps} like the batched kernel.
// Host side of k_pchol_groups: gsz[b] CTAs for block b (scaled down together when the
// groups do not all fit on the device at once), one cooperative launch, bounded-wait check.
__global__ void k_to_c64(const cplx* __restrict__ in, float2* __restrict__ out, long long n) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) out[e] = make_float2((float)in[e].x, (float)in[e].y);
}
__global__ void k_to_c128(const float2* __restrict__ in, cplx* __restrict__ out, long long n) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) out[e] = mkc((double)in[e].x, (double)in[e].y);
}

void run_pchol_groups(cudaStream_t st, cplx* Xs, BlkDesc* d_desc, int* d_piv, std::vector<int> gsz) {
  const int nblk = (int)gsz.size();
  static const int max_ctas = [] {
    int dev = 0, sms = 0, per_sm = 0;
    TDVP_CUDA(cudaGetDevice(&dev));
    TDVP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    TDVP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pchol_groups, 256, 0));
    return std::max(1, sms * std::min(4, std::max(1, per_sm)));
  }();
  long long total = 0;
  for (int g : gsz) total += g;
  const int budget = std::max(max_ctas, nblk);
  if (total > budget)
    for (int& g : gsz) g = std::max<long long>(1, (long long)g * budget / total);
  std::vector<int> cta_off(nblk + 1, 0);
  for (int b = 0; b < nblk; ++b) cta_off[b + 1] = cta_off[b] + gsz[b];
  const int nctas = cta_off[nblk];
  tdvp_require(nctas <= budget, TDVP_ERR_INVALID_ARG, "Cholesky groups exceed the co-resident CTAs");
  int* d_off = nullptr;
  int* d_idx = nullptr;
  double* d_val = nullptr;
  GridBar* bars = nullptr;
  TDVP_CUDA(cudaMallocAsync(&d_off, sizeof(int) * (nblk + 1), st));
  TDVP_CUDA(cudaMallocAsync(&d_idx, sizeof(int) * (nctas + 1), st));  // + the error word
  TDVP_CUDA(cudaMallocAsync(&d_val, sizeof(double) * nctas, st));
  TDVP_CUDA(cudaMallocAsync(&bars, sizeof(GridBar) * nblk, st));
  int* d_gerr = d_idx + nctas;
  TDVP_CUDA(cudaMemsetAsync(bars, 0, sizeof(GridBar) * nblk, st));
  TDVP_CUDA(cudaMemsetAsync(d_gerr, 0, sizeof(int), st));
  TDVP_CUDA(cudaMemcpyAsync(d_off, cta_off.data(), sizeof(int) * (nblk + 1), cudaMemcpyHostToDevice, st));
  int nb = nblk;
  double rel = 1e-15;
  const int* po = d_off;
  void* args[] = {&Xs, &d_desc, &d_piv, &po, &nb, &rel, &d_val, &d_idx, &bars, &d_gerr};
  TDVP_CUDA(cudaLaunchCooperativeKernel((void*)k_pchol_groups, dim3(nctas), dim3(256), args, 0, st));
  g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
  int herr = 0;
  TDVP_CUDA(cudaMemcpyAsync(&herr, d_gerr, sizeof(int), cudaMemcpyDeviceToHost, st));
  TDVP_CUDA(cudaStreamSynchronize(st));
  TDVP_CUDA(cudaFreeAsync(d_off, st));
  TDVP_CUDA(cudaFreeAsync(d_idx, st));
  TDVP_CUDA(cudaFreeAsync(d_val, st));
  TDVP_CUDA(cudaFreeAsync(bars, st));
  if (herr) throw TdvpError(TDVP_ERR_TIMEOUT, "pivoted Cholesky: a group barrier wait ran out");
}

template <class T>
void run_jacobi_multi(cudaStream_t st, typename Jac<T>::C* Xs, typename Jac<T>::C* Vs,
                      const std::vector<BlkDesc>& desc, const BlkDesc* d_desc, double* d_s, int* d_stat) {
  const int nblk = (int)desc.size();
  static const int max_ctas = [] {
    int dev = 0, sms = 0, per_sm = 0;
    TDVP_CUDA(cudaGetDevice(&dev));
    TDVP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    TDVP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi_groups<T>, 256, 0));
    return std::max(1, sms * std::min(4, std::max(1, per_sm)));
  }();
  // CTAs per block: one per pair of a round, scaled down together when they do not all fit
  std::vector<long long> pairs(nblk);
  long long total = 0;
  for (int b = 0; b < nblk; ++b) {
    pairs[b] = std::max(1, (desc[b].q + (desc[b].q & 1)) / 2);
    total += pairs[b];
  }
  std::vector<int> cta_off(nblk + 1, 0);
  const int budget = std::max(max_ctas, nblk);
  for (int b = 0; b < nblk; ++b) {
    long long nb = pairs[b];
    if (total > budget - nblk) nb = std::max<long long>(1, pairs[b] * (budget - nblk) / total);
    cta_off[b + 1] = cta_off[b] + (int)nb;
  }
  tdvp_require(cta_off[nblk] <= budget, TDVP_ERR_INVALID_ARG, "Jacobi groups exceed the co-resident CTAs");
  const int nctas = cta_off[nblk];
  int* d_off = nullptr;
  int* d_flags = nullptr;
  int* d_gerr = nullptr;
  double* d_fro2 = nullptr;
  GridBar* bars = nullptr;
  TDVP_CUDA(cudaMallocAsync(&d_off, sizeof(int) * (nblk + 1), st));
  TDVP_CUDA(cudaMallocAsync(&d_flags, sizeof(int) * 4 * nblk + sizeof(int), st));
  TDVP_CUDA(cudaMallocAsync(&d_fro2, sizeof(double) * nblk, st));
  TDVP_CUDA(cudaMallocAsync(&bars, sizeof(GridBar) * nblk, st));
  d_gerr = d_flags + 4 * nblk;
  TDVP_CUDA(cudaMemsetAsync(bars, 0, sizeof(GridBar) * nblk, st));
  TDVP_CUDA(cudaMemsetAsync(d_flags, 0, sizeof(int) * 4 * nblk + sizeof(int), st));
  TDVP_CUDA(cudaMemsetAsync(d_stat, 0, 3 * sizeof(int), st));
  TDVP_CUDA(cudaMemcpyAsync(d_off, cta_off.data(), sizeof(int) * (nblk + 1), cudaMemcpyHostToDevice, st));
  int nb = nblk, ms = 60;
  const BlkDesc* dd = d_desc;
  const int* po = d_off;
  void* args[] = {&Xs, &Vs, &dd, &po, &nb, &ms, &d_fro2, &d_flags, &bars, &d_gerr, &d_s, &d_stat};
  TDVP_CUDA(cudaLaunchCooperativeKernel((void*)k_jacobi_groups<T>, dim3(nctas), dim3(256), args, 0, st));
  g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
  int herr = 0;
  TDVP_CUDA(cudaMemcpyAsync(&herr, d_gerr, sizeof(int), cudaMemcpyDeviceToHost, st));
  TDVP_CUDA(cudaStreamSynchronize(st));
  TDVP_CUDA(cudaFreeAsync(d_off, st));
  TDVP_CUDA(cudaFreeAsync(d_flags, st));
  TDVP_CUDA(cudaFreeAsync(d_fro2, st));
  TDVP_CUDA(cudaFreeAsync(bars, st));
  if (herr) throw TdvpError(TDVP_ERR_TIMEOUT, "Jacobi SVD: a group barrier wait ran out");
}
}  // namespace

namespace {
// Connected blocks of the nonzero pattern of M (rows x cols, row-major): a device mask, then
// a host union-find over rows and columns.  Keyed by the smallest row of each block; rows and
// columns without a nonzero entry belong to no block.
std::map<int, std::pair<std::vector<int>, std::vector<int>>> block_components(cudaStream_t st, DevicePool* pool,
                                                                              const cplx* M, int rows, int cols) {
  const int words = (cols + 31) / 32;
  std::vector<unsigned> mask((size_t)rows * words);
  {
    RawBuf dm;
    dm.ensure(pool, sizeof(unsigned) * mask.size());
    const long long e = (long long)rows * words;
    k_nonzero_mask<<<ceil_div(e, 256), 256, 0, st>>>(M, rows, cols, words, dm.as<unsigned>());
    TDVP_CHECK_LAUNCH();
    TDVP_CUDA(cudaMemcpyAsync(mask.data(), dm.as<unsigned>(), sizeof(unsigned) * mask.size(),
                              cudaMemcpyDeviceToHost, st));
    TDVP_CUDA(cudaStreamSynchronize(st));
  }
  DSU dsu(rows + cols);
  std::vector<char> row_nz(rows, 0), col_nz(cols, 0);
  // Rows of one conserved-charge block usually share one nonzero pattern: a row whose pattern
  // equals an earlier row's is united with that row only, so the bit-by-bit unions run once
  // per distinct pattern.
  std::unordered_map<uint64_t, std::vector<int>> seen;
  for (int r = 0; r < rows; ++r) {
    const unsigned* rw = mask.data() + (size_t)r * words;
    uint64_t h = 1469598103934665603ull;
    bool any = false;
    for (int w = 0; w < words; ++w) {
      h = (h ^ rw[w]) * 1099511628211ull;
      any = any || rw[w] != 0u;
    }
    if (!any) continue;
    row_nz[r] = 1;
    auto& reps = seen[h];
    int twin = -1;
    for (int q : reps)
      if (std::memcmp(mask.data() + (size_t)q * words, rw, sizeof(unsigned) * words) == 0) {
        twin = q;
        break;
      }
    if (twin >= 0) {
      dsu.unite(r, twin);
      continue;
    }
    reps.push_back(r);
    for (int w = 0; w < words; ++w) {
      unsigned bits = rw[w];
      while (bits) {
        const int b = __builtin_ctz(bits);
        bits &= bits - 1;
        const int c = w * 32 + b;
        dsu.unite(r, rows + c);
        col_nz[c] = 1;
      }
    }
  }
  std::map<int, std::pair<std::vector<int>, std::vector<int>>> comp;
  for (int r = 0; r < rows; ++r)
    if (row_nz[r]) comp[dsu.find(r)].first.push_back(r);
  for (int c = 0; c < cols; ++c)
    if (col_nz[c]) comp[dsu.find(rows + c)].second.push_back(c);
  return comp;
}
__global__ void k_gather_rows(const cplx* __restrict__ M, long long cols, const int* __restrict__ perm, int rows,
                              cplx* __restrict__ out) {
  const long long n = (long long)rows * cols;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / cols, c = e % cols;
    out[e] = M[(long long)perm[r] * cols + c];
  }
}
}  // namespace

std::vector<int> sector_row_order(cudaStream_t st, DevicePool* pool, const cplx* M, int rows, int cols) {
  if (rows <= 1 || cols <= 0) return {};
  auto comp = block_components(st, pool, M, rows, cols);
  if (comp.size() <= 1) return {};
  std::vector<int> perm;
  perm.reserve(rows);
  std::vector<char> placed(rows, 0);
  for (auto& kv : comp)
    for (int r : kv.second.first) {
      perm.push_back(r);
      placed[r] = 1;
    }
  for (int r = 0; r < rows; ++r)
    if (!placed[r]) perm.push_back(r);  // zero rows, at the end
  bool identity = true;
  for (int r = 0; r < rows && identity; ++r) identity = perm[r] == r;
  if (identity) return {};
  return perm;
}

void gather_rows(cudaStream_t st, const cplx* M, int rows, int cols, const std::vector<int>& perm, cplx* out) {
  tdvp_require((int)perm.size() == rows, TDVP_ERR_INVALID_ARG, "gather_rows: permutation length");
  int* d_perm = nullptr;
  TDVP_CUDA(cudaMallocAsync(&d_perm, sizeof(int) * rows, st));
  TDVP_CUDA(cudaMemcpyAsync(d_perm, perm.data(), sizeof(int) * rows, cudaMemcpyHostToDevice, st));
  const long long n = (long long)rows * cols;
  k_gather_rows<<<(int)std::min<long long>(ceil_div(n, 256), 152 * 16), 256, 0, st>>>(M, cols, d_perm, rows, out);
  TDVP_CHECK_LAUNCH();
  TDVP_CUDA(cudaFreeAsync(d_perm, st));
}

void svd_blocked_keep(cudaStream_t st, DevicePool* pool, const cplx* M, int rows, int cols,
                      int (*select)(const std::vector<double>& s, void* ctx), void* ctx, SvdOut& out, bool want_u,
                      bool want_v, bool psd, bool jacobi_fp32) {
  g_svd_counters.calls++;
  const long long n = (long long)rows * cols;
  if (rows <= 1 || cols <= 1 || n > (1LL << 27)) {
    svd_jacobi_keep(st, pool, M, rows, cols, select, ctx, out, want_u, want_v);
    return;
  }
  auto prep = std::make_unique<ActivePhase>(PH_SVD_PREP);
  auto comp = block_components(st, pool, M, rows, cols);
  if (comp.empty()) {
    svd_jacobi_keep(st, pool, M, rows, cols, select, ctx, out, want_u, want_v);
    return;
  }
  if (comp.size() > 1) {
    g_svd_counters.blocked++;
    g_svd_counters.blocks += (long long)comp.size();
  }
  // Narrow blocks: one batched launch, one CTA per block with X_b, V_b in shared
  // memory.  As soon as one block is kMultiQ columns wide (or too large for shared
  // memory), every block goes to the cooperative launch that spreads each round's
  // pairs over the whole GPU.
  constexpr size_t kSmemCap = 200 * 1024;
  constexpr int kMultiQ = 24;
  bool multi = false;
  for (auto& kv : comp) {
    const int nr = (int)kv.second.first.size(), nc = (int)kv.second.second.size();
    const int p = std::max(nr, nc), q = std::min(nr, nc);
    if (q >= kMultiQ || ((size_t)p * q + (size_t)q * q) * sizeof(cplx) > kSmemCap) multi = true;
  }
  std::vector<BlkDesc> desc;
  std::vector<int> ridx, cidx;
  long long xo = 0, vo = 0;
  int so = 0;
  size_t smem_need = 0;
  for (auto& kv : comp) {
    auto& rr = kv.second.first;
    auto& cc = kv.second.second;
    const int nr = (int)rr.size(), nc = (int)cc.size();
    const int p = std::max(nr, nc), q = std::min(nr, nc);
    const size_t bytes = ((size_t)p * q + (size_t)q * q) * sizeof(cplx);
    atomic_max(g_svd_counters.max_q, q);
    if (multi && q >= kMultiQ) g_svd_counters.large_blocks++;
    BlkDesc d;
    d.orient = nr >= nc ? 0 : 1;
    d.need_v = d.orient == 0 ? (want_v ? 1 : 0) : (want_u ? 1 : 0);
    d.p = p;
    d.q = q;
    d.nr = nr;
    d.nc = nc;
    d.x_off = xo;
    d.v_off = vo;
    d.s_off = so;
    d.r_off = (int)ridx.size();
    d.c_off = (int)cidx.size();
    ridx.insert(ridx.end(), rr.begin(), rr.end());
    cidx.insert(cidx.end(), cc.begin(), cc.end());
    xo += (long long)p * q;
    vo += (long long)q * q;
    so += q;
    smem_need = std::max(smem_need, bytes);
    desc.push_back(d);
  }
  const int nsmall = (int)desc.size();
  struct Cand {
    double s;
    int blk, j;
  };
  std::vector<Cand> all;
  DArr Xs, Vs;
  BlkDesc* d_desc = nullptr;
  int *d_ridx = nullptr, *d_cidx = nullptr, *d_bad = nullptr, *d_piv = nullptr;
  double* d_s = nullptr;
  psd = psd && rows == cols && !want_v;
  // the factorisation reads each block as a square n x n matrix: a Hermitian pattern
  // gives square blocks; anything else takes the plain SVD (same eigen data for PSD)
  for (const BlkDesc& d : desc) psd = psd && d.nr == d.nc;
  if (nsmall) {
    Xs.reset(pool, (size_t)std::max<long long>(1, xo));
    Vs.reset(pool, (size_t)std::max<long long>(1, vo));
    TDVP_CUDA(cudaMallocAsync(&d_desc, sizeof(BlkDesc) * nsmall, st));
    TDVP_CUDA(cudaMallocAsync(&d_ridx, sizeof(int) * std::max<size_t>(1, ridx.size()), st));
    TDVP_CUDA(cudaMallocAsync(&d_cidx, sizeof(int) * std::max<size_t>(1, cidx.size()), st));
    TDVP_CUDA(cudaMallocAsync(&d_s, sizeof(double) * std::max(1, so) + 3 * sizeof(int), st));
    d_bad = reinterpret_cast<int*>(d_s + std::max(1, so));
    TDVP_CUDA(cudaMemcpyAsync(d_desc, desc.data(), sizeof(BlkDesc) * nsmall, cudaMemcpyHostToDevice, st));
    TDVP_CUDA(cudaMemcpyAsync(d_ridx, ridx.data(), sizeof(int) * ridx.size(), cudaMemcpyHostToDevice, st));
    TDVP_CUDA(cudaMemcpyAsync(d_cidx, cidx.data(), sizeof(int) * cidx.size(), cudaMemcpyHostToDevice, st));
    TDVP_CUDA(cudaMemsetAsync(d_bad, 0, 3 * sizeof(int), st));
    k_gather_batched<<<nsmall, 256, 0, st>>>(M, cols, d_desc, d_ridx, d_cidx, Xs.data(), Vs.data());
    TDVP_CHECK_LAUNCH();
    prep.reset();
    if (psd) {
      ActivePhase ph(PH_SVD_PCHOL);
      // eigendecomposition of a Hermitian PSD matrix: Jacobi SVD of its pivoted Cholesky
      // factor per block; eigenvalues below 1e-15 of the block's largest diagonal entry
      // (under every keep floor of the method) end the factorisation
      TDVP_CUDA(cudaMallocAsync(&d_piv, sizeof(int) * std::max<size_t>(1, ridx.size()), st));
      TDVP_CUDA(cudaMemsetAsync(d_s, 0, sizeof(double) * std::max(1, so), st));
      // blocks wider than one SM's FP64 pipe handles quickly get a group of CTAs each
      std::vector<int> gsz(nsmall);
      bool grouped = false;
      for (int b = 0; b < nsmall; ++b) {
        gsz[b] = std::min(16, std::max(1, desc[b].p / 48));
        grouped = grouped || gsz[b] > 1;
      }
      if (grouped) {
        run_pchol_groups(st, Xs.data(), d_desc, d_piv, gsz);
      } else {
        k_pchol_batched<<<nsmall, 256, 0, st>>>(Xs.data(), d_desc, d_piv, 1e-15);
        TDVP_CHECK_LAUNCH();
      }
    }
    std::optional<ActivePhase> jac(std::in_place, PH_SVD_JACOBI);
    static const bool attr = [] {
      TDVP_CUDA(cudaFuncSetAttribute(k_jacobi_batched<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kSmemCap));
      TDVP_CUDA(cudaFuncSetAttribute(k_jacobi_batched<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kSmemCap));
      return true;
    }();
    (void)attr;
    if (psd && jacobi_fp32) {
      // the factor (FP64 pivoted Cholesky) is rotated in FP32: its columns are graded, so the
      // one-sided Jacobi keeps about 1e-7 relative accuracy in every eigenvalue (s^2)
      RawBuf x32, v32;
      x32.ensure(pool, sizeof(float2) * (size_t)std::max<long long>(1, xo));
      v32.ensure(pool, sizeof(float2) * (size_t)std::max<long long>(1, vo));
      k_to_c64<<<ceil_div(std::max<long long>(1, xo), 256), 256, 0, st>>>(Xs.data(), x32.as<float2>(), xo);
      TDVP_CHECK_LAUNCH();
      k_to_c64<<<ceil_div(std::max<long long>(1, vo), 256), 256, 0, st>>>(Vs.data(), v32.as<float2>(), vo);
      TDVP_CHECK_LAUNCH();
      if (!multi) {
        k_jacobi_batched<float><<<nsmall, 256, smem_need / 2, st>>>(x32.as<float2>(), v32.as<float2>(), d_desc, 60,
                                                                   d_s, d_bad);
        TDVP_CHECK_LAUNCH();
      } else {
        run_jacobi_multi<float>(st, x32.as<float2>(), v32.as<float2>(), desc, d_desc, d_s, d_bad);
      }
      k_to_c128<<<ceil_div(std::max<long long>(1, xo), 256), 256, 0, st>>>(x32.as<float2>(), Xs.data(), xo);
      TDVP_CHECK_LAUNCH();
    } else if (!multi) {
      k_jacobi_batched<double><<<nsmall, 256, smem_need, st>>>(Xs.data(), Vs.data(), d_desc, 60, d_s, d_bad);
      TDVP_CHECK_LAUNCH();
    } else {
      run_jacobi_multi<double>(st, Xs.data(), Vs.data(), desc, d_desc, d_s, d_bad);
    }
    jac.reset();
    std::vector<double> hs(so);
    int hbad[3] = {0, 0, 0};
    TDVP_CUDA(cudaMemcpyAsync(hs.data(), d_s, sizeof(double) * so, cudaMemcpyDeviceToHost, st));
    TDVP_CUDA(cudaMemcpyAsync(hbad, d_bad, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
    TDVP_CUDA(cudaStreamSynchronize(st));
    tdvp_require(hbad[0] == 0, TDVP_ERR_SVD_NOT_CONVERGED, "batched Jacobi SVD did not converge");
    g_svd_counters.sweeps += hbad[2];
    atomic_max(g_svd_counters.max_sweeps, hbad[1]);
    for (int b = 0; b < nsmall; ++b)
      for (int j = 0; j < desc[b].q; ++j) {
        const double v = hs[desc[b].s_off + j];
        tdvp_require(std::isfinite(v), TDVP_ERR_NONFINITE, "SVD: non-finite singular value");
        if (psd) {
          if (v > 0.0) all.push_back({v * v, b, j});  // eigenvalue = (singular value of L)^2
        } else {
          all.push_back({v, b, j});
        }
      }
  }
  prep.reset();
  ActivePhase select_phase(PH_SVD_SELECT);
  std::stable_sort(all.begin(), all.end(), [](const Cand& a, const Cand& b) { return a.s > b.s; });
  out.rows = rows;
  out.cols = cols;
  out.s.assign(std::min(rows, cols), 0.0);
  for (size_t k = 0; k < all.size() && k < out.s.size(); ++k) out.s[k] = all[k].s;
  const int keep = std::max(0, std::min((int)all.size(), select(out.s, ctx)));
  out.rank = keep;
  out.sweeps = 0;
  out.U.release();
  out.Vh.release();
  if (keep > 0) {
    if (want_u) {
      out.U.reset(pool, (size_t)rows * keep);
      fill_zero(st, out.U.data(), (long long)rows * keep);
    }
    if (want_v) {
      out.Vh.reset(pool, (size_t)keep * cols);
      fill_zero(st, out.Vh.data(), (long long)keep * cols);
    }
    // kept vectors grouped by block (a conserved-charge sector), descending s inside each:
    // every sector of the new index is one contiguous range, so zero tiles of the tensors
    // built on it stay whole 128-row tiles the tensor-core GEMMs skip
    std::vector<int> ord(keep);
    for (int k = 0; k < keep; ++k) ord[k] = k;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return all[a].blk < all[b].blk; });
    std::vector<SelEntry> sel;
    for (int k = 0; k < keep; ++k) {
      const Cand& c = all[ord[k]];
      sel.push_back({c.blk, c.j, k, psd ? std::sqrt(c.s) : c.s});
    }
    if (!sel.empty()) {
      SelEntry* d_sel = nullptr;
      TDVP_CUDA(cudaMallocAsync(&d_sel, sizeof(SelEntry) * sel.size(), st));
      TDVP_CUDA(cudaMemcpyAsync(d_sel, sel.data(), sizeof(SelEntry) * sel.size(), cudaMemcpyHostToDevice, st));
      k_scatter_batched<<<(int)sel.size(), 128, 0, st>>>(Xs.data(), Vs.data(), d_desc, d_sel, d_ridx, d_cidx,
                                                          want_u ? out.U.data() : nullptr, keep,
                                                          want_v ? out.Vh.data() : nullptr, cols, want_u ? 1 : 0,
                                                          want_v ? 1 : 0, psd ? d_piv : nullptr);
      TDVP_CHECK_LAUNCH();
      TDVP_CUDA(cudaFreeAsync(d_sel, st));
    }
  }
  if (nsmall) {
    TDVP_CUDA(cudaFreeAsync(d_desc, st));
    TDVP_CUDA(cudaFreeAsync(d_ridx, st));
    TDVP_CUDA(cudaFreeAsync(d_cidx, st));
    TDVP_CUDA(cudaFreeAsync(d_s, st));
    if (d_piv) TDVP_CUDA(cudaFreeAsync(d_piv, st));
  }
}

// ============================================================================
// Block-structured thin QR / LQ: the gauge moves that cut nothing (real-time sweeps,
// canonicalisation).  Blocks come from the exact-zero pattern as for the SVD.  Block b
// is gathered as the column-major working matrix X_b (p x q): the block itself (orient 0,
// M = Q C) or its conjugate transpose (orient 1, M = C Q, an LQ).  Householder QR of X_b
// with kq = min(p, q) reflectors H_j = 1 - tau_j v_j v_j^H, v_j[j] = 1:
//   x = X_b[j:, j],  beta = -e^{i arg x_j} |x|,  v = (x - beta e_j) / (x_j - beta),
//   tau = 1 + |x_j| / |x|,  H_j x = beta e_j
// (tau = 0 for a zero column).  v_j's tail overwrites X_b below the diagonal, beta the
// diagonal; R is the upper trapezoid.  Q_b[:, c] = H_0 H_1 ... H_c e_c.
// ============================================================================
namespace {
struct QrDesc {
  int orient, p, q, kq;
  long long x_off, q_off;   // X_b (p x q) and Q_b (p x kq), column-major
  int r_off, c_off, k_off;  // the block's rows and columns in the index lists; its first new index
  int t_off;                // tau_b
};

__global__ void k_qr_gather(const cplx* __restrict__ M, int cols, const QrDesc* __restrict__ desc,
                            const int* __restrict__ ridx, const int* __restrict__ cidx, cplx* __restrict__ X) {
  const QrDesc d = desc[blockIdx.x];
  cplx* Xb = X + d.x_off;
  for (long long e = threadIdx.x; e < (long long)d.p * d.q; e += blockDim.x) {
    const int i = (int)(e % d.p), j = (int)(e / d.p);
    Xb[e] = d.orient == 0 ? M[(long long)ridx[d.r_off + i] * cols + cidx[d.c_off + j]]
                          : cconj(M[(long long)ridx[d.r_off + j] * cols + cidx[d.c_off + i]]);
  }
}

constexpr int kQrChunk = 8;  // columns whose dot products one block reduction serves

// Block-wide sums of n <= kQrChunk complex partials; the totals land in out[0..n).
__device__ __forceinline__ void qr_block_sums(cplx* acc, int n, cplx (*red)[kQrChunk], cplx* out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int t = 0; t < n; ++t) {
    const cplx v = warp_sum(acc[t]);
    if (lane == 0) red[warp][t] = v;
  }
  __syncthreads();
  if (threadIdx.x < n) {
    cplx s = mkc(0.0, 0.0);
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s = cadd(s, red[w][threadIdx.x]);
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// Reflector j from column j of X_b (rows j..p-1), by the whole block.
__device__ void qr_make_reflector(cplx* __restrict__ Xb, int p, int j, double* __restrict__ tau,
                                  cplx (*red)[kQrChunk], cplx* tot) {
  __shared__ cplx s_inv;
  __shared__ int s_zero;
  cplx* x = Xb + (long long)j * p;
  cplx acc[1] = {mkc(0.0, 0.0)};
  for (int r = j + threadIdx.x; r < p; r += blockDim.x) acc[0].x += cabs2(x[r]);
  qr_block_sums(acc, 1, red, tot);
  if (threadIdx.x == 0) {
    const double nrm = sqrt(tot[0].x);
    const cplx a = x[j];
    s_zero = !(nrm > 0.0);
    if (s_zero) {
      tau[j] = 0.0;
    } else {
      const double aa = sqrt(cabs2(a));
      const cplx ph = aa > 0.0 ? cscale(a, 1.0 / aa) : mkc(1.0, 0.0);
      const double den = aa + nrm;
      s_inv = cscale(cconj(ph), 1.0 / den);  // 1 / (x_j - beta) = e^{-i arg x_j} / (|x_j| + |x|)
      tau[j] = den / nrm;
      x[j] = cscale(ph, -nrm);  // beta
    }
  }
  __syncthreads();
  if (!s_zero) {
    const cplx inv = s_inv;
    for (int r = j + 1 + threadIdx.x; r < p; r += blockDim.x) x[r] = cmul(x[r], inv);
  }
  __syncthreads();
}

// Applies H_j (v staged in sv[0..p-j), sv[0] = 1) to the columns cols[0..n) of Y (rows j..p-1).
__device__ __forceinline__ void qr_apply(cplx* __restrict__ Y, int p, int j, const cplx* __restrict__ sv,
                                         double tj, const int* cols, int n, cplx (*red)[kQrChunk], cplx* tot) {
  cplx acc[kQrChunk];
#pragma unroll
  for (int t = 0; t < kQrChunk; ++t) acc[t] = mkc(0.0, 0.0);
  for (int r = j + threadIdx.x; r < p; r += blockDim.x) {
    const cplx v = sv[r - j];
#pragma unroll
    for (int t = 0; t < kQrChunk; ++t)
      if (t < n) cfma_conj(acc[t], v, Y[(long long)cols[t] * p + r]);
  }
  qr_block_sums(acc, n, red, tot);
  cplx w[kQrChunk];
#pragma unroll
  for (int t = 0; t < kQrChunk; ++t) w[t] = t < n ? cscale(tot[t], tj) : mkc(0.0, 0.0);
  for (int r = j + threadIdx.x; r < p; r += blockDim.x) {
    const cplx v = sv[r - j];
#pragma unroll
    for (int t = 0; t < kQrChunk; ++t)
      if (t < n) {
        cplx& y = Y[(long long)cols[t] * p + r];
        y = csub(y, cmul(w[t], v));
      }
  }
  __syncthreads();
}

// One cooperative launch: the CTAs [cta_off[b], cta_off[b+1]) factorise block b.  CTA lc of a
// group of G owns the columns c = lc (mod G).  Step j: every CTA stages v_j in shared memory
// and applies H_j to its own columns right of j; the owner of column j+1 then forms reflector
// j+1 from it; one bounded group barrier ends the step.  Q_b is then accumulated column by
// column (each CTA its own columns, H_j for j = c down to 0), with no further barrier.
__global__ void __launch_bounds__(256)
    k_qr_groups(cplx* __restrict__ X, cplx* __restrict__ Qb, double* __restrict__ tau,
                const QrDesc* __restrict__ desc, const int* __restrict__ cta_off, int nblk, GridBar* __restrict__ bars,
                int* __restrict__ gerr) {
  extern __shared__ cplx sv[];
  __shared__ cplx red[8][kQrChunk];
  __shared__ cplx tot[kQrChunk];
  int lo = 0, hi = nblk - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (cta_off[mid] <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  const int b = lo;
  const int lc = blockIdx.x - cta_off[b];
  const int G = cta_off[b + 1] - cta_off[b];
  const QrDesc d = desc[b];
  cplx* Xb = X + d.x_off;
  double* tb = tau + d.t_off;
  GridBar* bar = bars + b;
  unsigned epoch = 0;
  const int p = d.p, q = d.q, kq = d.kq;
  int cols[kQrChunk];
  if (kq > 0 && lc == 0) qr_make_reflector(Xb, p, 0, tb, red, tot);
  if (!group_sync(bar, (unsigned)G, gerr, epoch)) return;
  for (int j = 0; j < kq; ++j) {
    for (int r = j + threadIdx.x; r < p; r += blockDim.x) sv[r - j] = r == j ? mkc(1.0, 0.0) : Xb[(long long)j * p + r];
    __syncthreads();
    const double tj = tb[j];
    // own columns right of j (the smallest one first)
    int c0 = j + 1 + ((lc - (j + 1)) % G + G) % G;
    if (tj != 0.0)
      for (int c = c0; c < q;) {
        int n = 0;
        for (; n < kQrChunk && c < q; ++n, c += G) cols[n] = c;
        qr_apply(Xb, p, j, sv, tj, cols, n, red, tot);
      }
    if (j + 1 < kq) {
      if ((j + 1) % G == lc) qr_make_reflector(Xb, p, j + 1, tb, red, tot);
      if (!group_sync(bar, (unsigned)G, gerr, epoch)) return;
    }
  }
  // Q_b: own columns c < kq start as e_c; H_j applies to the columns c >= j
  cplx* Qc = Qb + d.q_off;
  for (int c = lc; c < kq; c += G)
    for (int r = threadIdx.x; r < p; r += blockDim.x) Qc[(long long)c * p + r] = mkc(r == c ? 1.0 : 0.0, 0.0);
  __syncthreads();
  const int last = lc < kq ? lc + ((kq - 1 - lc) / G) * G : -1;  // largest own column
  for (int j = last; j >= 0; --j) {
    const double tj = tb[j];
    if (tj == 0.0) continue;
    for (int r = j + threadIdx.x; r < p; r += blockDim.x) sv[r - j] = r == j ? mkc(1.0, 0.0) : Xb[(long long)j * p + r];
    __syncthreads();
    int c0 = j + ((lc - j) % G + G) % G;
    for (int c = c0; c < kq;) {
      int n = 0;
      for (; n < kQrChunk && c < kq; ++n, c += G) cols[n] = c;
      qr_apply(Qc, p, j, sv, tj, cols, n, red, tot);
    }
  }
}

// Entry (blk, j): column j of Q_b and row j of R_b into the outputs.
//   orient 0: Qout rows x K  (Qout[row, k_off + j] = Q_b[i, j]),
//             Cout K x cols  (Cout[k_off + j, col] = R_b[j, c], c >= j)
//   orient 1: Qout K x cols  (Qout[k_off + j, col] = conj Q_b[i, j]),
//             Cout rows x K  (Cout[row, k_off + j] = conj R_b[j, r], r >= j)
__global__ void k_qr_scatter(const cplx* __restrict__ X, const cplx* __restrict__ Qb, const QrDesc* __restrict__ desc,
                             const int2* __restrict__ ent, const int* __restrict__ ridx, const int* __restrict__ cidx,
                             cplx* __restrict__ Qout, cplx* __restrict__ Cout, int cols, int K,
                             double* __restrict__ diag) {
  const int2 e = ent[blockIdx.x];
  const QrDesc d = desc[e.x];
  const int j = e.y;
  const long long k = d.k_off + j;
  const cplx* qcol = Qb + d.q_off + (long long)j * d.p;
  const cplx* Xb = X + d.x_off;
  if (threadIdx.x == 0) diag[k] = sqrt(cabs2(Xb[(long long)j * d.p + j]));  // |R_jj| = |beta_j|
  if (d.orient == 0) {
    for (int i = threadIdx.x; i < d.p; i += blockDim.x) Qout[(long long)ridx[d.r_off + i] * K + k] = qcol[i];
    for (int c = j + threadIdx.x; c < d.q; c += blockDim.x)
      Cout[k * cols + cidx[d.c_off + c]] = Xb[(long long)c * d.p + j];
  } else {
    for (int i = threadIdx.x; i < d.p; i += blockDim.x) Qout[k * cols + cidx[d.c_off + i]] = cconj(qcol[i]);
    for (int r = j + threadIdx.x; r < d.q; r += blockDim.x)
      Cout[(long long)ridx[d.r_off + r] * K + k] = cconj(Xb[(long long)r * d.p + j]);
  }
}
}  // namespace

void qr_blocked(cudaStream_t st, DevicePool* pool, const cplx* M, int rows, int cols, int orient, QrOut& out) {
  ActivePhase phase(PH_QR);
  out.k = 0;
  out.Q.release();
  out.C.release();
  auto comp = block_components(st, pool, M, rows, cols);
  std::vector<QrDesc> desc;
  std::vector<int> ridx, cidx;
  long long xo = 0, qo = 0;
  int to = 0, K = 0, pmax = 1;
  for (auto& kv : comp) {
    auto& rr = kv.second.first;
    auto& cc = kv.second.second;
    const int nr = (int)rr.size(), nc = (int)cc.size();
    QrDesc d;
    d.orient = orient;
    d.p = orient == 0 ? nr : nc;
    d.q = orient == 0 ? nc : nr;
    d.kq = std::min(d.p, d.q);
    d.x_off = xo;
    d.q_off = qo;
    d.r_off = (int)ridx.size();
    d.c_off = (int)cidx.size();
    d.k_off = K;
    d.t_off = to;
    ridx.insert(ridx.end(), rr.begin(), rr.end());
    cidx.insert(cidx.end(), cc.begin(), cc.end());
    xo += (long long)d.p * d.q;
    qo += (long long)d.p * d.kq;
    to += d.kq;
    K += d.kq;
    pmax = std::max(pmax, d.p);
    desc.push_back(d);
  }
  if (K == 0) return;
  const int nblk = (int)desc.size();
  const size_t smem = (size_t)pmax * sizeof(cplx);
  tdvp_require(smem <= 200 * 1024, TDVP_ERR_INVALID_ARG, "QR: block too tall for the staged reflector");
  static const bool attr = [] {
    TDVP_CUDA(cudaFuncSetAttribute(k_qr_groups, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    return true;
  }();
  (void)attr;
  int dev = 0, sms = 0, per_sm = 0;
  TDVP_CUDA(cudaGetDevice(&dev));
  TDVP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  TDVP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_qr_groups, 256, smem));
  tdvp_require(per_sm >= 1, TDVP_ERR_INVALID_ARG, "QR: kernel does not fit on an SM");
  const int budget = std::max(nblk, sms * std::min(4, per_sm));
  // CTAs per block in proportion to its work (p q kq), at most one per two columns; a group of
  // one needs no barrier
  std::vector<double> work(nblk);
  double wsum = 0.0;
  for (int b = 0; b < nblk; ++b) {
    work[b] = (double)desc[b].p * desc[b].q * std::max(1, desc[b].kq);
    wsum += work[b];
  }
  std::vector<int> cta_off(nblk + 1, 0);
  for (int b = 0; b < nblk; ++b) {
    const int cap = std::max(1, (desc[b].q + 1) / 2);
    long long g = (long long)std::floor((double)(budget - nblk) * work[b] / wsum);
    g = std::max<long long>(1, std::min<long long>(cap, g));
    cta_off[b + 1] = cta_off[b] + (int)g;
  }
  const int nctas = cta_off[nblk];
  tdvp_require(nctas <= budget, TDVP_ERR_INVALID_ARG, "QR groups exceed the co-resident CTAs");
  DArr X(pool, (size_t)xo), Qb(pool, (size_t)std::max<long long>(1, qo));
  RawBuf meta;
  const size_t b_desc = sizeof(QrDesc) * nblk, b_r = sizeof(int) * ridx.size(), b_c = sizeof(int) * cidx.size();
  const size_t b_off = sizeof(int) * (nblk + 1), b_tau = sizeof(double) * to, b_bar = sizeof(GridBar) * nblk;
  std::vector<int2> ent;
  for (int b = 0; b < nblk; ++b)
    for (int j = 0; j < desc[b].kq; ++j) ent.push_back(make_int2(b, j));
  const size_t b_ent = sizeof(int2) * ent.size();
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t o_desc = 0, o_r = al(b_desc), o_c = o_r + al(b_r), o_off = o_c + al(b_c), o_tau = o_off + al(b_off),
               o_bar = o_tau + al(b_tau), o_ent = o_bar + al(b_bar), o_diag = o_ent + al(b_ent),
               o_err = o_diag + al(sizeof(double) * K);
  meta.ensure(pool, o_err + 256);
  char* base = meta.as<char>();
  auto* d_desc = reinterpret_cast<QrDesc*>(base + o_desc);
  auto* d_r = reinterpret_cast<int*>(base + o_r);
  auto* d_c = reinterpret_cast<int*>(base + o_c);
  auto* d_off = reinterpret_cast<int*>(base + o_off);
  auto* d_tau = reinterpret_cast<double*>(base + o_tau);
  auto* d_bar = reinterpret_cast<GridBar*>(base + o_bar);
  auto* d_ent = reinterpret_cast<int2*>(base + o_ent);
  auto* d_err = reinterpret_cast<int*>(base + o_err);
  auto* d_diag = reinterpret_cast<double*>(base + o_diag);
  TDVP_CUDA(cudaMemcpyAsync(d_desc, desc.data(), b_desc, cudaMemcpyHostToDevice, st));
  TDVP_CUDA(cudaMemcpyAsync(d_r, ridx.data(), b_r, cudaMemcpyHostToDevice, st));
  TDVP_CUDA(cudaMemcpyAsync(d_c, cidx.data(), b_c, cudaMemcpyHostToDevice, st));
  TDVP_CUDA(cudaMemcpyAsync(d_off, cta_off.data(), b_off, cudaMemcpyHostToDevice, st));
  TDVP_CUDA(cudaMemcpyAsync(d_ent, ent.data(), b_ent, cudaMemcpyHostToDevice, st));
  TDVP_CUDA(cudaMemsetAsync(d_bar, 0, b_bar, st));
  TDVP_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), st));
  k_qr_gather<<<nblk, 256, 0, st>>>(M, cols, d_desc, d_r, d_c, X.data());
  TDVP_CHECK_LAUNCH();
  {
    cplx* xp = X.data();
    cplx* qp = Qb.data();
    const QrDesc* dd = d_desc;
    const int* po = d_off;
    int nb = nblk;
    void* args[] = {&xp, &qp, &d_tau, &dd, &po, &nb, &d_bar, &d_err};
    TDVP_CUDA(cudaLaunchCooperativeKernel((void*)k_qr_groups, dim3(nctas), dim3(256), args, smem, st));
    g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
  }
  const size_t nq = orient == 0 ? (size_t)rows * K : (size_t)K * cols;
  const size_t nc = orient == 0 ? (size_t)K * cols : (size_t)rows * K;
  out.Q.reset(pool, nq);
  out.C.reset(pool, nc);
  fill_zero(st, out.Q.data(), (long long)nq);
  fill_zero(st, out.C.data(), (long long)nc);
  k_qr_scatter<<<(int)ent.size(), 128, 0, st>>>(X.data(), Qb.data(), d_desc, d_ent, d_r, d_c, out.Q.data(),
                                                  out.C.data(), cols, K, d_diag);
  TDVP_CHECK_LAUNCH();
  int herr = 0;
  std::vector<double> diag(K);
  TDVP_CUDA(cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  TDVP_CUDA(cudaMemcpyAsync(diag.data(), d_diag, sizeof(double) * K, cudaMemcpyDeviceToHost, st));
  TDVP_CUDA(cudaStreamSynchronize(st));
  if (herr) throw TdvpError(TDVP_ERR_TIMEOUT, "QR: a group barrier wait ran out");
  out.k = K;
  out.diag_min = *std::min_element(diag.begin(), diag.end());
  out.diag_max = *std::max_element(diag.begin(), diag.end());
  for (double v : diag) tdvp_require(std::isfinite(v), TDVP_ERR_NONFINITE, "QR: non-finite factor");
}
