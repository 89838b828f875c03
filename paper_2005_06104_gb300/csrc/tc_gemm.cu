// Tensor-core H_eff for sm_103a: complex contractions mapped to real
// tcgen05 GEMMs with TF32 operands split hi + lo (three products, FP32
// accumulation in tensor memory).
//
// Real embedding of a complex product C = A B (4M form): A stays interleaved
// (re, im) along K; B is expanded to the real (2N x 2K) operand
//   [ Re B  -Im B ]
//   [ Im B   Re B ]  (rows (n, re/im), K index (k, re/im))
// so that one real GEMM writes C interleaved.
//
// GEMM kernel: one CTA per 128 x 128 output tile, 6 warps:
//   warp 0      TMA producer (cp.async.bulk.tensor, 128B swizzle, 3 stages)
//   warp 1      TMEM allocator and single-thread tcgen05.mma issuer
//   warps 2..5  epilogue: tcgen05.ld from TMEM lanes 32*(warp%4) .. +31
// The tensor core's FP32 accumulation error grows linearly with the number of
// products summed in one accumulator (measured); K is therefore split into
// chunks of 32 that alternate between two TMEM accumulators, and the epilogue
// warps add each finished chunk into FP32 registers.
// Every mbarrier wait is bounded by a wall-clock limit; on expiry the CTA
// records an error word, drains its own copies and MMAs (bounded) and frees
// its tensor memory before returning.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>

#include "contract.cuh"
#include "tc_ptx.cuh"

namespace tc {
constexpr int BM = 128;

// Tile configurations.  BK fp32 per K-block: 32 uses the 128-byte swizzle, 16 the
// 64-byte swizzle.  BN = 256 halves the operand traffic per MAC (the kernel is
// fed from L2); its epilogue uses eight warps, two per TMEM lane quadrant.
template <int BN_, int BK_, int STAGES_>
struct Cfg {
  static constexpr int BN = BN_, BK = BK_, STAGES = STAGES_;
  static constexpr int A_TILE = BM * BK * 4;
  static constexpr int B_TILE = BN * BK * 4;
  static constexpr int STAGE_BYTES = 2 * A_TILE + 2 * B_TILE;
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
  static constexpr int TMEM_COLS = 2 * BN;           // two accumulators (ping-pong)
  static constexpr int CHUNK_KB = 32 / BK;           // K = 32 per accumulation chunk
  static constexpr int EPI_WARPS = 4 * (BN / 128);
  static constexpr int THREADS = 64 + 32 * EPI_WARPS;
  static constexpr int SWZ_BYTES = BK * 4;           // 128 or 64
};
using CfgN128 = Cfg<128, 32, 3>;
using CfgN256 = Cfg<256, 16, 4>;

// K is consumed in chunks of CHUNK_KB k-blocks.  Each chunk accumulates in one of
// two TMEM buffers (ping-pong) and the epilogue warps add it into FP32 registers
// with round-to-nearest adds, so the tensor core's own accumulator only ever
// sums CHUNK_KB * BK products.
template <class C>
__global__ void __launch_bounds__(C::THREADS, 1)
    k_gemm_tf32x3(const __grid_constant__ CUtensorMap tmAhi, const __grid_constant__ CUtensorMap tmAlo,
                  const __grid_constant__ CUtensorMap tmBhi, const __grid_constant__ CUtensorMap tmBlo, int M,
                  int N, int nkb, void* __restrict__ out, long long ldo, int out_f64, int* __restrict__ err) {
  constexpr int BN = C::BN, BK = C::BK, STAGES = C::STAGES, A_TILE = C::A_TILE, B_TILE = C::B_TILE;
  constexpr int STAGE_BYTES = C::STAGE_BYTES, TMEM_COLS = C::TMEM_COLS, CHUNK_KB = C::CHUNK_KB;
  constexpr int SWZ = C::SWZ_BYTES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* full = bars;
  uint64_t* empty = bars + STAGES;
  uint64_t* tfull = bars + 2 * STAGES;
  uint64_t* tempty = bars + 2 * STAGES + 2;
  uint64_t* done = bars + 2 * STAGES + 4;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int nchunks = (nkb + CHUNK_KB - 1) / CHUNK_KB;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&tfull[b]), 1);
      mbar_init(smem_u32(&tempty[b]), C::EPI_WARPS);
    }
    mbar_init(smem_u32(done), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    int issued = 0;
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb % STAGES, it = kb / STAGES;
      if (it > 0 && !mbar_wait(smem_u32(&empty[s]), (it - 1) & 1)) {
        *abort_flag = 1;
        break;
      }
      if (*abort_flag) break;
      uint8_t* st = smem + s * STAGE_BYTES;
      const uint32_t fb = smem_u32(&full[s]);
      mbar_expect_tx(fb, STAGE_BYTES);
      tma_load_2d(smem_u32(st), &tmAhi, fb, kb * BK, m0);
      tma_load_2d(smem_u32(st + A_TILE), &tmAlo, fb, kb * BK, m0);
      tma_load_2d(smem_u32(st + 2 * A_TILE), &tmBhi, fb, kb * BK, n0);
      tma_load_2d(smem_u32(st + 2 * A_TILE + B_TILE), &tmBlo, fb, kb * BK, n0);
      issued = kb + 1;
    }
    if (*abort_flag) {
      // drain our own copies still in flight (bounded)
      for (int kb = (issued > STAGES ? issued - STAGES : 0); kb < issued; ++kb)
        (void)mbar_wait(smem_u32(&full[kb % STAGES]), (kb / STAGES) & 1);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    const uint32_t idesc = idesc_tf32(BM, BN);
    for (int c = 0; c < nchunks && !*abort_flag; ++c) {
      const int b = c & 1, u = c >> 1;
      if (u > 0 && !mbar_wait(smem_u32(&tempty[b]), (u - 1) & 1)) {
        *abort_flag = 1;
        break;
      }
      fence_after();
      const uint32_t acc_tmem = tmem + (uint32_t)(b * BN);
      const int kb_end = min(nkb, (c + 1) * CHUNK_KB);
      for (int kb = c * CHUNK_KB; kb < kb_end; ++kb) {
        const int s = kb % STAGES, it = kb / STAGES;
        if (!mbar_wait(smem_u32(&full[s]), it & 1)) {
          *abort_flag = 1;
          break;
        }
        fence_after();
        const uint32_t a_hi = smem_u32(smem + s * STAGE_BYTES);
        const uint32_t a_lo = a_hi + A_TILE;
        const uint32_t b_hi = a_hi + 2 * A_TILE;
        const uint32_t b_lo = b_hi + B_TILE;
#pragma unroll
        for (int k = 0; k < BK / 8; ++k) {
          const uint32_t off = k * 32;  // 8 tf32 = 32 bytes along K inside the swizzle atom
          const uint32_t first = (kb == c * CHUNK_KB && k == 0) ? 0u : 1u;
          mma_tf32(acc_tmem, sdesc<SWZ>(a_hi + off), sdesc<SWZ>(b_hi + off), idesc, first);
          mma_tf32(acc_tmem, sdesc<SWZ>(a_hi + off), sdesc<SWZ>(b_lo + off), idesc, 1u);
          mma_tf32(acc_tmem, sdesc<SWZ>(a_lo + off), sdesc<SWZ>(b_hi + off), idesc, 1u);
        }
        mma_commit(smem_u32(&empty[s]));
      }
      if (*abort_flag) break;
      mma_commit(smem_u32(&tfull[b]));
    }
    mma_commit(smem_u32(done));  // fires when every issued MMA has completed
  } else if (warp >= 2) {
    // ---------------- epilogue: promote chunk partials into FP32 registers
    // warp w reads TMEM lanes 32*(w%4)..+31 and the column half (w-2)/4 (128 columns)
    const int q = warp & 3;
    const int half = (warp - 2) >> 2;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    constexpr int EC = 128;  // columns per epilogue warp
    float acc[EC];
#pragma unroll
    for (int j = 0; j < EC; ++j) acc[j] = 0.f;
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
      const int b = c & 1, u = c >> 1;
      bool got = mbar_wait(smem_u32(&tfull[b]), u & 1);
      if (!got) *abort_flag = 1;
      ok = __all_sync(0xffffffffu, got && !*abort_flag);  // keep the .aligned loads warp-uniform
      if (!ok) break;
      fence_after();
#pragma unroll
      for (int c0 = 0; c0 < EC; c0 += 16) {
        uint32_t v[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(tmem + lane_base + (uint32_t)(b * BN + half * EC + c0)));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[c0 + j] += __uint_as_float(v[j]);
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&tempty[b]));
    }
    const int gm = m0 + q * 32 + lane;
    const int nb = n0 + half * EC;
    if (ok && gm < M) {
      if (out_f64) {
        double* o = static_cast<double*>(out) + (long long)gm * ldo + nb;
        if (nb + EC <= N && (ldo & 1) == 0) {
#pragma unroll
          for (int j = 0; j < EC; j += 2)
            *reinterpret_cast<double2*>(o + j) = make_double2((double)acc[j], (double)acc[j + 1]);
        } else {
#pragma unroll
          for (int j = 0; j < EC; ++j)
            if (nb + j < N) o[j] = (double)acc[j];
        }
      } else {
        float* o = static_cast<float*>(out) + (long long)gm * ldo + nb;
        if (nb + EC <= N && (ldo & 3) == 0) {
#pragma unroll
          for (int j = 0; j < EC; j += 4)
            *reinterpret_cast<float4*>(o + j) = make_float4(acc[j], acc[j + 1], acc[j + 2], acc[j + 3]);
        } else {
#pragma unroll
          for (int j = 0; j < EC; ++j)
            if (nb + j < N) o[j] = acc[j];
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    // every MMA issued by this CTA has completed before its tensor memory is freed
    (void)mbar_wait(smem_u32(done), 0);
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
  if (threadIdx.x == 0 && *abort_flag) atomicExch(err, 1);
}

// ---------------------------------------------------------------- operand preparation
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
__device__ __forceinline__ void split2(double x, float& hi, float& lo) {
  hi = to_tf32((float)x);
  lo = to_tf32((float)(x - (double)hi));
}

// dst[r][k2] (ld) from complex src[r][c] interleaved; zero for k2 >= 2 cols and
// for the padding rows r >= rows (up to rows_pad)
__global__ void k_split_interleaved(const cplx* __restrict__ src, int rows, int rows_pad, int cols, int ld,
                                    float* __restrict__ hi, float* __restrict__ lo) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)rows_pad * ld) return;
  const int k2 = e % ld;
  const long long r = e / ld;
  float h = 0.f, l = 0.f;
  if (k2 < 2 * cols && r < rows) {
    const cplx v = src[r * cols + (k2 >> 1)];
    split2((k2 & 1) ? v.y : v.x, h, l);
  }
  hi[e] = h;
  lo[e] = l;
}

// Real expansion of a complex B operand.  Logical complex B[k][n] (k < K, n < Nc);
// src_kn: stored as src[k*Nc + n], else as src[n*K + k].  dst rows (n, c'), K index (k, c):
//   (re,re) = Re, (re,im) = -Im, (im,re) = Im, (im,im) = Re.  ld >= 2K, zero padded.
__global__ void k_expand_b(const cplx* __restrict__ src, int K, int Nc, int src_kn, int ld, int rows_pad,
                           float* __restrict__ hi, float* __restrict__ lo) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)rows_pad * ld) return;
  const int k2 = e % ld;
  const long long n2 = e / ld;
  float h = 0.f, l = 0.f;
  if (k2 < 2 * K && n2 < 2LL * Nc) {
    const int k = k2 >> 1, c = k2 & 1;
    const long long n = n2 >> 1;
    const int cp = (int)(n2 & 1);
    const cplx v = src_kn ? src[(long long)k * Nc + n] : src[n * K + k];
    double x;
    if (cp == 0)
      x = (c == 0) ? v.x : -v.y;
    else
      x = (c == 0) ? v.y : v.x;
    split2(x, h, l);
  }
  hi[e] = h;
  lo[e] = l;
}

// MPO stage on FP32 T1[a][w][t][b'] (complex) into the split stage-3 A operand
// T2[(a,s)][(v,b',c)] = sum_{(w,t)} W[w,s,t,v] T1[a,w,t,b'].
__global__ void k_stage2(const float2* __restrict__ T1, int WL, int WR, int D, int MR, const int* __restrict__ off,
                         const int* __restrict__ idx, const cplx* __restrict__ val, int ld, float* __restrict__ hi,
                         float* __restrict__ lo) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  const int sv = blockIdx.y;
  const long long a = blockIdx.z;
  if (b >= MR) return;
  const int s = sv / WR, v = sv % WR;
  double re = 0.0, im = 0.0;
  for (int e = off[sv]; e < off[sv + 1]; ++e) {
    const int w = idx[2 * e], t = idx[2 * e + 1];
    const float2 x = T1[((a * WL + w) * D + t) * MR + b];
    const cplx c = val[e];
    re += c.x * (double)x.x - c.y * (double)x.y;
    im += c.x * (double)x.y + c.y * (double)x.x;
  }
  const long long o = (a * D + s) * (long long)ld + 2LL * ((long long)v * MR + b);
  float h, l;
  split2(re, h, l);
  hi[o] = h;
  lo[o] = l;
  split2(im, h, l);
  hi[o + 1] = h;
  lo[o + 1] = l;
}

__global__ void k_zero_pad_cols(float* __restrict__ hi, float* __restrict__ lo, int rows, int ld, int from) {
  const int w = ld - from;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)rows * w) return;
  const long long r = e / w;
  const int c = from + (int)(e % w);
  hi[r * ld + c] = 0.f;
  lo[r * ld + c] = 0.f;
}

// ---------------------------------------------------------------- host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    TDVP_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    tdvp_require(q == cudaDriverEntryPointSuccess && p, TDVP_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

CUtensorMap make_map(const float* base, int rows, int ld, int box_rows, int bk) {
  tdvp_require((reinterpret_cast<uintptr_t>(base) & 15) == 0, TDVP_ERR_INVALID_ARG, "TMA base not 16B aligned");
  tdvp_require(ld % 32 == 0, TDVP_ERR_INVALID_ARG, "TMA row length must be a multiple of 32");
  tdvp_require(rows % box_rows == 0, TDVP_ERR_INVALID_ARG, "TMA operand rows must be padded to the box");
  tdvp_require(bk == 32 || bk == 16, TDVP_ERR_INVALID_ARG, "TMA K box must be 16 or 32");
  CUtensorMap m;
  std::memset(&m, 0, sizeof(m));
  cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
  cuuint32_t box[2] = {(cuuint32_t)bk, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE,
                           bk == 32 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  tdvp_require(r == CUDA_SUCCESS, TDVP_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  return m;
}

template <class C>
void launch_gemm(cudaStream_t st, const float* Ahi, const float* Alo, const float* Bhi, const float* Blo, int M, int N,
                 int ldk, void* out, long long ldo, bool out_f64, int* d_err) {
  static const bool attr = [] {
    TDVP_CUDA(cudaFuncSetAttribute(k_gemm_tf32x3<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM_BYTES));
    return true;
  }();
  (void)attr;
  // operands hold ceil(M/128)*128 and ceil(N/128)*128 rows (zero padded); a BN = 256
  // tile may reach 128 rows past the padded B operand only when N is not a multiple of
  // 256, and the host pads B to 256 rows in that case
  const int Mp = ceil_div(M, BM) * BM, Np = ceil_div(N, C::BN) * C::BN;
  const CUtensorMap ma = make_map(Ahi, Mp, ldk, BM, C::BK), mal = make_map(Alo, Mp, ldk, BM, C::BK);
  const CUtensorMap mb = make_map(Bhi, Np, ldk, C::BN, C::BK), mbl = make_map(Blo, Np, ldk, C::BN, C::BK);
  dim3 grid(ceil_div(N, C::BN), ceil_div(M, BM));
  tdvp_require(grid.y <= 65535, TDVP_ERR_INVALID_ARG, "gemm_tf32x3: M too large");
  k_gemm_tf32x3<C><<<grid, C::THREADS, C::SMEM_BYTES, st>>>(ma, mal, mb, mbl, M, N, ldk / C::BK, out, ldo,
                                                            out_f64 ? 1 : 0, d_err);
  TDVP_CHECK_LAUNCH();
}

// B operands are allocated with rows padded to a multiple of 256 (see bpad) so both
// tile shapes stay inside the buffer.
void gemm_tf32x3(cudaStream_t st, const float* Ahi, const float* Alo, const float* Bhi, const float* Blo, int M, int N,
                 int ldk, void* out, long long ldo, bool out_f64, int* d_err) {
  if (M <= 0 || N <= 0) return;
  tdvp_require(ldk % 32 == 0 && ldk > 0, TDVP_ERR_INVALID_ARG, "gemm_tf32x3: K must be padded to 32");
  if (N >= 256)
    launch_gemm<CfgN256>(st, Ahi, Alo, Bhi, Blo, M, N, ldk, out, ldo, out_f64, d_err);
  else
    launch_gemm<CfgN128>(st, Ahi, Alo, Bhi, Blo, M, N, ldk, out, ldo, out_f64, d_err);
}

inline int pad32(int k) { return (k + 31) / 32 * 32; }
inline int pad128(int k) { return (k + 127) / 128 * 128; }
inline int bpad(int n) { return (n + 255) / 256 * 256; }  // rows of a B operand (either tile shape)

// A operand of a general complex GEMM: hi/lo[m][k2] = split(opA(A)[m][k2/2] re|im),
// zero outside M x 2K (rows padded to Mp, row length ld)
__global__ void k_split_opa(const cplx* __restrict__ A, long long lda, int opA, int M, int K, int Mp, int ld,
                            float* __restrict__ hi, float* __restrict__ lo) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)Mp * ld) return;
  const int k2 = e % ld;
  const long long m = e / ld;
  float h = 0.f, l = 0.f;
  if (m < M && k2 < 2 * K) {
    const int k = k2 >> 1;
    cplx v = (opA == OP_N || opA == OP_R) ? A[m * lda + k] : A[(long long)k * lda + m];
    if (opA == OP_C || opA == OP_R) v.y = -v.y;
    split2((k2 & 1) ? v.y : v.x, h, l);
  }
  hi[e] = h;
  lo[e] = l;
}

// B operand expanded to the real (2N x 2K) form from opB(B)[k][n]
__global__ void k_expand_opb(const cplx* __restrict__ B, long long ldb, int opB, int K, int N, int rows_pad, int ld,
                             float* __restrict__ hi, float* __restrict__ lo) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)rows_pad * ld) return;
  const int k2 = e % ld;
  const long long n2 = e / ld;
  float h = 0.f, l = 0.f;
  if (k2 < 2 * K && n2 < 2LL * N) {
    const int k = k2 >> 1, c = k2 & 1;
    const long long n = n2 >> 1;
    const int cp = (int)(n2 & 1);
    cplx v = (opB == OP_N || opB == OP_R) ? B[(long long)k * ldb + n] : B[n * ldb + k];
    if (opB == OP_C || opB == OP_R) v.y = -v.y;
    const double x = (cp == 0) ? ((c == 0) ? v.x : -v.y) : ((c == 0) ? v.y : v.x);
    split2(x, h, l);
  }
  hi[e] = h;
  lo[e] = l;
}
}  // namespace tc

using namespace tc;

void heff_tf32x3(cudaStream_t st, Scratch& s, const SiteOp& op, const cplx* x, cplx* y) {
  const int ml = op.ml, mr = op.mr, wl = op.wl, wr = op.wr, d = op.d;
  TcEnvCache& c = s.tc;
  DevicePool* pool = s.pool;
  const int M1 = ml * wl, K1p = pad32(2 * ml), N1 = 2 * d * mr;
  const int M3 = ml * d, K3 = 2 * wr * mr, K3p = pad32(K3), N3 = 2 * mr;
  if (c.err.bytes() == 0) {
    c.err.ensure(pool, sizeof(int));
    TDVP_CUDA(cudaMemsetAsync(c.err.as<int>(), 0, sizeof(int), st));
  }
  const int M1p = pad128(M1), N1p = bpad(N1), M3p = pad128(M3), N3p = bpad(N3);
  if (op.env_key < 0 || c.key != op.env_key) {
    c.Lhi.ensure(pool, sizeof(float) * (size_t)M1p * K1p);
    c.Llo.ensure(pool, sizeof(float) * (size_t)M1p * K1p);
    long long n = (long long)M1p * K1p;
    k_split_interleaved<<<ceil_div(n, 256), 256, 0, st>>>(op.L, M1, M1p, ml, K1p, c.Lhi.as<float>(),
                                                          c.Llo.as<float>());
    TDVP_CHECK_LAUNCH();
    c.Rhi.ensure(pool, sizeof(float) * (size_t)N3p * K3p);
    c.Rlo.ensure(pool, sizeof(float) * (size_t)N3p * K3p);
    n = (long long)N3p * K3p;
    // R[b][(v,b')] is B[k=(v,b')][n=b] stored n-major
    k_expand_b<<<ceil_div(n, 256), 256, 0, st>>>(op.R, wr * mr, mr, 0, K3p, N3p, c.Rhi.as<float>(),
                                                 c.Rlo.as<float>());
    TDVP_CHECK_LAUNCH();
    c.key = op.env_key;
  }
  // stage 1: T1[(a,w)][(s',b',c)] = L x
  c.Bhi.ensure(pool, sizeof(float) * (size_t)N1p * K1p);
  c.Blo.ensure(pool, sizeof(float) * (size_t)N1p * K1p);
  {
    const long long n = (long long)N1p * K1p;
    k_expand_b<<<ceil_div(n, 256), 256, 0, st>>>(x, ml, d * mr, 1, K1p, N1p, c.Bhi.as<float>(), c.Blo.as<float>());
    TDVP_CHECK_LAUNCH();
  }
  c.T1.ensure(pool, sizeof(float) * (size_t)M1 * N1);
  gemm_tf32x3(st, c.Lhi.as<float>(), c.Llo.as<float>(), c.Bhi.as<float>(), c.Blo.as<float>(), M1, N1, K1p,
              c.T1.as<float>(), N1, false, c.err.as<int>());
  // stage 2: MPO tensor
  c.T2hi.ensure(pool, sizeof(float) * (size_t)M3p * K3p);
  c.T2lo.ensure(pool, sizeof(float) * (size_t)M3p * K3p);
  {
    const WSparse& ws = *op.W;
    tdvp_require(ml <= 65535, TDVP_ERR_INVALID_ARG, "heff_tc: bond too large");
    dim3 g(ceil_div(mr, 128), d * wr, ml);
    k_stage2<<<g, 128, 0, st>>>(c.T1.as<float2>(), wl, wr, d, mr, ws.d_l_off, ws.d_l_idx, ws.d_l_val, K3p,
                                c.T2hi.as<float>(), c.T2lo.as<float>());
    TDVP_CHECK_LAUNCH();
    if (K3p > K3) {
      const long long n = (long long)M3 * (K3p - K3);
      k_zero_pad_cols<<<ceil_div(n, 256), 256, 0, st>>>(c.T2hi.as<float>(), c.T2lo.as<float>(), M3, K3p, K3);
      TDVP_CHECK_LAUNCH();
    }
    if (M3p > M3) {
      const size_t off = (size_t)M3 * K3p, bytes = sizeof(float) * (size_t)(M3p - M3) * K3p;
      TDVP_CUDA(cudaMemsetAsync(c.T2hi.as<float>() + off, 0, bytes, st));
      TDVP_CUDA(cudaMemsetAsync(c.T2lo.as<float>() + off, 0, bytes, st));
    }
  }
  // stage 3: y[(a,s)][(b,c)] = T2 R^T  (FP64 output, interleaved complex)
  gemm_tf32x3(st, c.T2hi.as<float>(), c.T2lo.as<float>(), c.Rhi.as<float>(), c.Rlo.as<float>(), M3, N3, K3p,
              reinterpret_cast<double*>(y), N3, true, c.err.as<int>());
  c.pending = true;
}

void zgemm_tc(cudaStream_t st, Scratch& s, int opA, int opB, int M, int N, int K, const cplx* A, long long lda,
              const cplx* B, long long ldb, cplx* C, long long ldc) {
  if (M <= 0 || N <= 0) return;
  DevicePool* pool = s.pool;
  TcEnvCache& c = s.tc;
  if (c.err.bytes() == 0) {
    c.err.ensure(pool, sizeof(int));
    TDVP_CUDA(cudaMemsetAsync(c.err.as<int>(), 0, sizeof(int), st));
  }
  const int Kp = pad32(std::max(1, 2 * K)), Mp = pad128(M), Np = bpad(2 * N);
  RawBuf ahi, alo, bhi, blo;
  ahi.ensure(pool, sizeof(float) * (size_t)Mp * Kp);
  alo.ensure(pool, sizeof(float) * (size_t)Mp * Kp);
  bhi.ensure(pool, sizeof(float) * (size_t)Np * Kp);
  blo.ensure(pool, sizeof(float) * (size_t)Np * Kp);
  long long n = (long long)Mp * Kp;
  k_split_opa<<<ceil_div(n, 256), 256, 0, st>>>(A, lda, opA, M, K, Mp, Kp, ahi.as<float>(), alo.as<float>());
  TDVP_CHECK_LAUNCH();
  n = (long long)Np * Kp;
  k_expand_opb<<<ceil_div(n, 256), 256, 0, st>>>(B, ldb, opB, K, N, Np, Kp, bhi.as<float>(), blo.as<float>());
  TDVP_CHECK_LAUNCH();
  gemm_tf32x3(st, ahi.as<float>(), alo.as<float>(), bhi.as<float>(), blo.as<float>(), M, 2 * N, Kp,
              reinterpret_cast<double*>(C), 2 * ldc, true, c.err.as<int>());
  c.pending = true;
}

void tc_check(cudaStream_t st, Scratch& s) {
  TcEnvCache& c = s.tc;
  if (!c.pending || c.err.bytes() == 0) return;
  int h_err = 0;
  TDVP_CUDA(cudaMemcpyAsync(&h_err, c.err.as<int>(), sizeof(int), cudaMemcpyDeviceToHost, st));
  TDVP_CUDA(cudaStreamSynchronize(st));
  c.pending = false;
  if (h_err != 0) {
    TDVP_CUDA(cudaMemsetAsync(c.err.as<int>(), 0, sizeof(int), st));
    throw TdvpError(TDVP_ERR_TIMEOUT, "tensor-core GEMM: a bounded pipeline wait ran out");
  }
}
