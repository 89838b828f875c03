// Tensor-core complex GEMMs with BF16 "exact slices" (sm_103a, tcgen05 kind::f16).
//
// Each real operand (the 4M embedding of the complex one, as in the TF32 path)
// is cut into fixed-point slices.  For one scaling group, with 2^e the smallest
// power of two above its largest magnitude, every entry is written as
//   x = 2^e (a1 2^-8 + a2 2^-16 + a3 2^-24 + a4 2^-32) + r,   |r| <= 2^(e-33),
// with integers |a1| <= 256 and |a_s| <= 128 (s > 1), exact in BF16.  Slice s is
// stored as a_s 2^(-8(s-1)) (exact) and the group scale as the float 2^(e-8).
// A-operand groups are one row and one chunk of 128 along K; B-operand groups
// are whole rows, so the B scale is one factor per output column, applied once.
//
// The products of slices s, t (0-based) with s + t <= S - 1 are summed: the
// leading product a1 b1 in accumulator P, all others in accumulator Q.  Within a
// chunk P is a sum of at most 128 integers of magnitude <= 2^16, so every partial
// sum is an integer below 2^24 and the tensor core's FP32 accumulation of P is
// exact whatever its rounding.  Q is about 2^-7 of P; its 72 (S = 4) MMA
// accumulations per chunk, each rounding near 2^-23 of Q, leave about 2^-24 of P.  The epilogue scales each chunk by its A chunk scale
// (a power of two: exact) and adds it into a double-float (hi, lo) pair per output
// with Knuth's two-sum, so no error accrues across chunks.  GB300 runs FP64 at a
// small fraction of its FP32 rate, which is why the promotion uses FP32 pairs.
// S = 4 (10 products) represents the operands to 2^-33 of their group maxima and
// the products to about 2^-24 (the rounding of Q); S = 3 (6 products) to 2^-25.
//
// Kernel layout (one CTA per 128 x 128 output tile, three warpgroups):
//   warp 0       TMA producer: one 3-D box per operand and stage (all S slices)
//   warp 1       TMEM allocator and single-thread tcgen05.mma issuer
//   warps 2, 3   idle
//   warps 4..11  epilogue: warp w reads TMEM lanes 32*(w%4)..+31, columns 64*((w-4)/4)..+63
// The first warpgroup gives registers back (setmaxnreg 40) so that the epilogue
// warpgroups can hold 64 (hi, lo) pairs per thread (setmaxnreg 232):
// 128 * 40 + 256 * 232 = 384 * 168, the launch's own allocation.
// Tensor memory: two chunk buffers (ping-pong) x (P, Q) x 128 columns = 512 columns.
// Every mbarrier wait is bounded; on expiry the CTA records an error word, drains
// its copies and MMAs (bounded) and frees its tensor memory.
#include <cuda_bf16.h>

#include <cstring>

#include "contract.cuh"
#include "tc_ptx.cuh"

namespace tcb {
using namespace tc;

constexpr int BM = 128, BN = 128, BK = 32, STAGES = 3;
constexpr int KC = 128;                 // K elements per chunk (exactness bound of P: 128 * 2^16 < 2^24)
constexpr int kMaxChunks = 1024;        // chunks one CTA can walk (K up to 131072 real entries per split)
constexpr int KC_KB = KC / BK;          // k-blocks per chunk
constexpr int EPI_WARPS = 8;
constexpr int EPI_WARP0 = 4;            // first epilogue warp (second warpgroup)
constexpr int THREADS = 128 + 32 * EPI_WARPS;
constexpr int REGS_LAUNCH = 168, REGS_LOW = 40, REGS_HIGH = 232;
static_assert(128 * REGS_LOW + 32 * EPI_WARPS * REGS_HIGH <= THREADS * REGS_LAUNCH, "register split");
constexpr int TILE = BM * BK * 2;       // one slice of one operand tile (bytes); BM == BN
constexpr int TMEM_COLS = 512;
constexpr int EC = 64;                  // output columns per epilogue thread

template <int S>
struct SCfg {
  static constexpr int STAGE_BYTES = 2 * S * TILE;
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
};

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(acc)
      : "memory");
}

// hi + lo += v without loss (Knuth's two-sum into hi, its error into lo)
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float v) {
  const float s = __fadd_rn(hi, v);
  const float bb = __fadd_rn(s, -hi);
  const float e = __fadd_rn(__fadd_rn(hi, -__fadd_rn(s, -bb)), __fadd_rn(v, -bb));
  hi = s;
  lo = __fadd_rn(lo, e);
}

// (output tile, K chunk) pairs visited by k_gemm_bf16s since load: [0] all, [1] multiplied
__device__ unsigned long long g_chunk_pairs[2];

template <int S>
__global__ void __launch_bounds__(THREADS, 1)
    k_gemm_bf16s(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M, int N,
                 int nkb_total, int kb_split, const float* __restrict__ sA, long long lsA,
                 const float* __restrict__ sB, void* __restrict__ out, long long ldo, long long split_stride,
                 int out_df, int* __restrict__ err, const unsigned* __restrict__ maskA,
                 const unsigned* __restrict__ maskB, int mwords) {
  constexpr int STAGE_BYTES = SCfg<S>::STAGE_BYTES;
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
  // split K: this CTA takes k-blocks [kb0, kb0 + nkb) (kb0 a multiple of a chunk)
  const int kb0 = blockIdx.z * kb_split;
  const int nkb = min(nkb_total, kb0 + kb_split) - kb0;
  const int c0 = kb0 / KC_KB;
  const int nchunks = (nkb + KC_KB - 1) / KC_KB;
  // Chunks whose A tile (these BM rows) or B tile (these BN rows) holds only zeros add exact
  // zeros to this output tile: the list of the others, built once (the slicing kernels set a
  // bit per 128-row tile and chunk that holds a nonzero entry).  All three roles walk it.
  __shared__ int act[kMaxChunks];
  __shared__ int n_act;
  if (threadIdx.x == 0) {
    int n = 0;
    for (int c = 0; c < nchunks; ++c) {
      const int g = c0 + c;
      bool on = true;
      if (maskA) {
        on = (maskA[(long long)blockIdx.y * mwords + (g >> 5)] >> (g & 31)) & 1u;
        on = on && ((maskB[(long long)blockIdx.x * mwords + (g >> 5)] >> (g & 31)) & 1u);
      }
      if (on && n < kMaxChunks) act[n++] = c;
    }
    n_act = n;
    atomicAdd(&g_chunk_pairs[0], (unsigned long long)nchunks);
    atomicAdd(&g_chunk_pairs[1], (unsigned long long)n);
  }

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&tfull[b]), 1);
      mbar_init(smem_u32(&tempty[b]), EPI_WARPS);
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
  if (warp < EPI_WARP0) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(REGS_LOW));
  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer: all S slices of the A and B tiles of one k-block
    int issued = 0;  // running count of k-blocks loaded (stage = issued % STAGES)
    for (int ai = 0; ai < n_act && !*abort_flag; ++ai) {
      const int c = act[ai];
      const int kb_end = min(nkb, (c + 1) * KC_KB);
      for (int kb = c * KC_KB; kb < kb_end; ++kb) {
        const int s = issued % STAGES, it = issued / STAGES;
        if (it > 0 && !mbar_wait(smem_u32(&empty[s]), (it - 1) & 1)) {
          *abort_flag = 1;
          break;
        }
        if (*abort_flag) break;
        uint8_t* st = smem + s * STAGE_BYTES;
        const uint32_t fb = smem_u32(&full[s]);
        mbar_expect_tx(fb, STAGE_BYTES);
        tma_load_3d(smem_u32(st), &tmA, fb, (kb0 + kb) * BK, m0, 0);
        tma_load_3d(smem_u32(st + S * TILE), &tmB, fb, (kb0 + kb) * BK, n0, 0);
        ++issued;
      }
    }
    if (*abort_flag) {
      for (int q = (issued > STAGES ? issued - STAGES : 0); q < issued; ++q)
        (void)mbar_wait(smem_u32(&full[q % STAGES]), (q / STAGES) & 1);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    const uint32_t idesc = idesc_bf16(BM, BN);
    int used = 0;  // running count of k-blocks consumed, in the producer's order
    for (int ai = 0; ai < n_act && !*abort_flag; ++ai) {
      const int c = act[ai];
      const int b = ai & 1, u = ai >> 1;
      if (u > 0 && !mbar_wait(smem_u32(&tempty[b]), (u - 1) & 1)) {
        *abort_flag = 1;
        break;
      }
      fence_after();
      const uint32_t accP = tmem + (uint32_t)(b * 2 * BN);
      const uint32_t accQ = accP + BN;
      const int kb_end = min(nkb, (c + 1) * KC_KB);
      for (int kb = c * KC_KB; kb < kb_end; ++kb) {
        const int s = used % STAGES, it = used / STAGES;
        ++used;
        if (!mbar_wait(smem_u32(&full[s]), it & 1)) {
          *abort_flag = 1;
          break;
        }
        fence_after();
        const uint32_t a0 = smem_u32(smem + s * STAGE_BYTES);
        const uint32_t b0 = a0 + S * TILE;
#pragma unroll
        for (int k = 0; k < BK / 16; ++k) {
          const uint32_t off = k * 32;  // 16 bf16 = 32 bytes along K inside the 64-byte swizzle atom
          const uint32_t first = (kb == c * KC_KB && k == 0) ? 0u : 1u;
          mma_bf16(accP, sdesc<64>(a0 + off), sdesc<64>(b0 + off), idesc, first);
          uint32_t qacc = first;
#pragma unroll
          for (int sa = 0; sa < S; ++sa)
#pragma unroll
            for (int sb = 0; sb + sa < S; ++sb) {
              if (sa == 0 && sb == 0) continue;
              mma_bf16(accQ, sdesc<64>(a0 + sa * TILE + off), sdesc<64>(b0 + sb * TILE + off), idesc, qacc);
              qacc = 1u;
            }
        }
        mma_commit(smem_u32(&empty[s]));
      }
      if (*abort_flag) break;
      mma_commit(smem_u32(&tfull[b]));
    }
    mma_commit(smem_u32(done));
  }
  } else {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(REGS_HIGH));
    // ---------------- epilogue: scale each chunk and add it into (hi, lo) pairs
    const int q = warp & 3;
    const int half = (warp - EPI_WARP0) >> 2;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    const int gm = m0 + q * 32 + lane;
    const int nb = n0 + half * EC;
    float hi[EC], lo[EC];
#pragma unroll
    for (int j = 0; j < EC; ++j) hi[j] = lo[j] = 0.f;
    bool ok = true;
    for (int ai = 0; ai < n_act; ++ai) {
      const int c = act[ai];
      const int b = ai & 1, u = ai >> 1;
      bool got = mbar_wait(smem_u32(&tfull[b]), u & 1);
      if (!got) *abort_flag = 1;
      ok = __all_sync(0xffffffffu, got && !*abort_flag);
      if (!ok) break;
      fence_after();
      const float sa = sA[(long long)(c0 + c) * lsA + gm];
#pragma unroll
      for (int c0 = 0; c0 < EC; c0 += 8) {
        uint32_t vp[8], vq[8];
        const uint32_t col = tmem + lane_base + (uint32_t)(b * 2 * BN + half * EC + c0);
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(vp[0]), "=r"(vp[1]), "=r"(vp[2]), "=r"(vp[3]), "=r"(vp[4]), "=r"(vp[5]), "=r"(vp[6]),
                       "=r"(vp[7])
                     : "r"(col));
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(vq[0]), "=r"(vq[1]), "=r"(vq[2]), "=r"(vq[3]), "=r"(vq[4]), "=r"(vq[5]), "=r"(vq[6]),
                       "=r"(vq[7])
                     : "r"(col + BN));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          two_sum_acc(hi[c0 + j], lo[c0 + j], __fmul_rn(__uint_as_float(vp[j]), sa));
          two_sum_acc(hi[c0 + j], lo[c0 + j], __fmul_rn(__uint_as_float(vq[j]), sa));
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&tempty[b]));
    }
    if (ok) {  // warp-uniform
      // column scales: lane i holds those of columns nb + 2i, nb + 2i + 1 (inside the padded rows)
      const float2 sbv = __ldg(reinterpret_cast<const float2*>(sB + nb) + lane);
      const bool row_ok = gm < M;
      const bool vec = nb + EC <= N && (ldo & 1) == 0;
      if (out_df) {
        // double-float output: (hi, lo) FP32 pairs, scaled exactly by the power-of-two column scale
        float2* o = static_cast<float2*>(out) + blockIdx.z * split_stride + (long long)gm * ldo + nb;
#pragma unroll
        for (int j = 0; j < EC; j += 2) {
          const float s0 = __shfl_sync(0xffffffffu, sbv.x, j >> 1);
          const float s1 = __shfl_sync(0xffffffffu, sbv.y, j >> 1);
          const float4 v = make_float4(__fmul_rn(hi[j], s0), __fmul_rn(lo[j], s0), __fmul_rn(hi[j + 1], s1),
                                       __fmul_rn(lo[j + 1], s1));
          if (row_ok) {
            if (vec) {
              *reinterpret_cast<float4*>(o + j) = v;
            } else {
              if (nb + j < N) o[j] = make_float2(v.x, v.y);
              if (nb + j + 1 < N) o[j + 1] = make_float2(v.z, v.w);
            }
          }
        }
      } else {
        double* o = static_cast<double*>(out) + (long long)gm * ldo + nb;
#pragma unroll
        for (int j = 0; j < EC; j += 2) {
          const float s0 = __shfl_sync(0xffffffffu, sbv.x, j >> 1);
          const float s1 = __shfl_sync(0xffffffffu, sbv.y, j >> 1);
          const double d0 = ((double)hi[j] + (double)lo[j]) * (double)s0;
          const double d1 = ((double)hi[j + 1] + (double)lo[j + 1]) * (double)s1;
          if (row_ok) {
            if (vec) {
              *reinterpret_cast<double2*>(o + j) = make_double2(d0, d1);
            } else {
              if (nb + j < N) o[j] = d0;
              if (nb + j + 1 < N) o[j + 1] = d1;
            }
          }
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    (void)mbar_wait(smem_u32(done), 0);
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
  if (threadIdx.x == 0 && *abort_flag) atomicExch(err, 1);
}

// ---------------------------------------------------------------- operand slicing
// GB300 executes FP64 at a small fraction of its FP32 and integer rates, so the
// slicing runs without FP64 arithmetic: FP64 sources are cut into digits with
// integer operations on their bit patterns, double-float sources (FP32 hi, lo
// pairs) with exact FP32 operations.
//
// Sources give the real operand entries (k2, k2+1, k2+2, k2+3) of one row (k2 a
// multiple of 4), zero outside the logical matrix.  FP64 sources (kDF = false)
// fill double v[4]; double-float sources (kDF = true) fill float hi[4], lo[4].

// Rows m of opA(A) with K interleaved (re, im): the A operand of the 4M form.
struct SrcA {
  static constexpr bool kDF = false;
  const cplx* p;
  long long ld;
  int rows, K, op;
  __device__ void load4(long long m, int k2, double v[4]) const {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = (k2 >> 1) + h;
      double re = 0.0, im = 0.0;
      if (m < rows && k < K) {
        const cplx z = (op == OP_N || op == OP_R) ? p[m * ld + k] : p[(long long)k * ld + m];
        re = z.x;
        im = (op == OP_C || op == OP_R) ? -z.y : z.y;
      }
      v[2 * h] = re;
      v[2 * h + 1] = im;
    }
  }
};
// Rows (w, a) of the stage-1 A operand of H_eff, read from L[a][w][a'] channel by channel:
// a 128-row tile then holds one MPO channel w over a run of sector-ordered a, and under a
// conserved charge its nonzero columns a' lie in the one sector q_a - c_w.  In (a, w) order a
// tile mixes every channel and reaches the sectors of all channel charges at once.
struct SrcLwa {
  static constexpr bool kDF = false;
  const cplx* p;
  int ML, WL;
  __device__ void load4(long long m, int k2, double v[4]) const {
    const long long w = m / ML, a = m % ML;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = (k2 >> 1) + h;
      double re = 0.0, im = 0.0;
      if (w < WL && k < ML) {
        const cplx z = p[(a * WL + w) * ML + k];
        re = z.x;
        im = z.y;
      }
      v[2 * h] = re;
      v[2 * h + 1] = im;
    }
  }
};
// Rows (n, c') of the expanded real B operand built from opB(B)[k][n]:
//   row (n, re): (Re, -Im) over K index (k, re/im); row (n, im): (Im, Re).
struct SrcB {
  static constexpr bool kDF = false;
  const cplx* p;
  long long ld;
  int K, N, op;
  __device__ void load4(long long n2, int k2, double v[4]) const {
    const long long n = n2 >> 1;
    const int cp = (int)(n2 & 1);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = (k2 >> 1) + h;
      double re = 0.0, im = 0.0;
      if (n < N && k < K) {
        const cplx z = (op == OP_N || op == OP_R) ? p[(long long)k * ld + n] : p[n * ld + k];
        re = z.x;
        im = (op == OP_C || op == OP_R) ? -z.y : z.y;
      }
      v[2 * h] = cp == 0 ? re : im;
      v[2 * h + 1] = cp == 0 ? -im : re;
    }
  }
};

// s_hi + s_lo += (a_hi + a_lo)(b_hi + b_lo) in double-float arithmetic (about 2^-48)
__device__ __forceinline__ void df_mac(float& sh, float& sl, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  const float pe = __fmaf_rn(ah, bh, -p);  // exact rounding error of ah * bh
  const float cross = __fmaf_rn(ah, bl, __fmul_rn(al, bh));
  const float s = __fadd_rn(sh, p);
  const float bb = __fadd_rn(s, -sh);
  const float err = __fadd_rn(__fadd_rn(sh, -__fadd_rn(s, -bb)), __fadd_rn(p, -bb));
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(err, __fadd_rn(pe, cross)));
}

// Rows (a, s) of the stage-3 A operand of H_eff: K index (v, b', re/im),
//   T2[(a,s)][(v,b')] = sum_{(w,t)} W[w,s,t,v] T1[w][a][t][b']   (T1 rows in (w, a) order)
// with T1 and W as double-float complex (re hi, re lo, im hi, im lo).
struct SrcStage2 {
  static constexpr bool kDF = true;
  const float4* T1;
  const int* off;
  const int* idx;
  const float4* val;
  int ML, WL, WR, D, MR;
  __device__ void load4(long long row, int k2, float hi[4], float lo[4]) const {
    const long long a = row / D;
    const int s = (int)(row % D);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = (k2 >> 1) + h;
      const int vv = j / MR, b = j % MR;
      float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
      if (a < ML && vv < WR) {
        const int sv = s * WR + vv;
        for (int e = off[sv]; e < off[sv + 1]; ++e) {
          const int w = idx[2 * e], t = idx[2 * e + 1];
          const float4 x = T1[((w * ML + a) * D + t) * (long long)MR + b];
          const float4 c = val[e];
          df_mac(rh, rl, c.x, c.y, x.x, x.y);     // + Re c Re x
          df_mac(rh, rl, -c.z, -c.w, x.z, x.w);   // - Im c Im x
          df_mac(ih, il, c.x, c.y, x.z, x.w);     // + Re c Im x
          df_mac(ih, il, c.z, c.w, x.x, x.y);     // + Im c Re x
        }
      }
      // renormalise so that |lo| <= ulp(hi) / 2
      float t = __fadd_rn(rh, rl);
      rl = __fadd_rn(rl, -__fadd_rn(t, -rh));
      rh = t;
      t = __fadd_rn(ih, il);
      il = __fadd_rn(il, -__fadd_rn(t, -ih));
      ih = t;
      hi[2 * h] = rh;
      lo[2 * h] = rl;
      hi[2 * h + 1] = ih;
      lo[2 * h + 1] = il;
    }
  }
};

// Group exponent: the smallest e with (largest magnitude) < 2^e.  Groups whose largest
// magnitude is below 2^-100 (or zero) are taken as zero (live = false); a non-finite
// entry makes the scale NaN, so that it shows in the output.
struct GroupScale {
  int e = 0;
  bool live = false;
  float sc = 0.f;  // 2^(e-8)
};
__device__ __forceinline__ GroupScale scale_from_exponent(int unbiased, bool bad) {
  GroupScale g;
  if (bad) {
    g.sc = __int_as_float(0x7fc00000);
  } else if (unbiased >= -100) {
    g.live = true;
    g.e = unbiased + 1;
    g.sc = ldexpf(1.f, g.e - 8);
  }
  return g;
}
// |x| as an ordered integer key (larger magnitude, larger key; NaN/Inf above all finite)
__device__ __forceinline__ unsigned long long abs_key(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ GroupScale scale_from_key(unsigned long long key) {
  const int ex = (int)(key >> 52);
  if (ex == 0x7ff) return scale_from_exponent(0, true);
  if (ex == 0) return scale_from_exponent(-2000, false);  // zero or subnormal
  return scale_from_exponent(ex - 1023, false);
}
__device__ __forceinline__ GroupScale scale_from_float(float m, bool bad) {
  const int ex = (int)((__float_as_uint(m) >> 23) & 0xff);
  if (bad || ex == 0xff) return scale_from_exponent(0, true);
  if (ex == 0) return scale_from_exponent(-2000, false);
  return scale_from_exponent(ex - 127, false);
}

// integer value a (|a| < 2^22) as an exact float
__device__ __forceinline__ float int_to_float_exact(int a) {
  return __fadd_rn(__int_as_float(0x4B400000 + a), -12582912.0f);
}

// Digits of an FP64 entry: X = round(|x| 2^(32-e)) (|X| <= 2^32) from the bit pattern,
// then X = a1 2^24 + a2 2^16 + a3 2^8 + a4 with rounded signed digits; out[s] = a_{s+1} 2^(-8s).
template <int S>
__device__ __forceinline__ void digits_fp64(double x, const GroupScale& g, float out[S]) {
  long long X = 0;
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7ff);
  if (g.live && ex != 0) {
    const int shift = 20 + g.e - (ex - 1023);  // >= 21
    if (shift < 64) {
      const unsigned long long m53 = (b & 0xfffffffffffffull) | (1ull << 52);
      X = (long long)((m53 + (1ull << (shift - 1))) >> shift);
      if (b >> 63) X = -X;
    }
  }
  const int a1 = (int)((X + (1ll << 23)) >> 24);
  int r = (int)(X - ((long long)a1 << 24));  // [-2^23, 2^23)
  const int a2 = (r + (1 << 15)) >> 16;
  r -= a2 << 16;
  int a3, a4;
  if (S == 4) {
    a3 = (r + (1 << 7)) >> 8;
    a4 = r - (a3 << 8);
  } else {
    a3 = (r + (1 << 7)) >> 8;
    a4 = 0;
  }
  const int dg[4] = {a1, a2, a3, a4};
#pragma unroll
  for (int s = 0; s < S; ++s) out[s] = __fmul_rn(int_to_float_exact(dg[s]), __int_as_float((127 - 8 * s) << 23));
}

// Digits of a double-float entry hi + lo with exact FP32 steps: peel the rounded
// top digit off the head, fold the tail back in with a two-sum, repeat.
template <int S>
__device__ __forceinline__ void digits_df(float hi, float lo, const GroupScale& g, float out[S]) {
  if (!g.live) {
#pragma unroll
    for (int s = 0; s < S; ++s) out[s] = 0.f;
    return;
  }
  const float up = ldexpf(1.f, 32 - g.e);
  float H = __fmul_rn(hi, up), L = __fmul_rn(lo, up);  // |H + L| < 2^32
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int sh = 24 - 8 * s;                          // digit weight 2^sh
    const float w = __int_as_float((127 + sh) << 23), iw = __int_as_float((127 - sh) << 23);
    const float a = rintf(__fmul_rn(H, iw));
    out[s] = __fmul_rn(a, __int_as_float((127 - 8 * s) << 23));
    const float r = __fmaf_rn(-a, w, H);  // exact
    const float t = __fadd_rn(r, L);
    const float bb = __fadd_rn(t, -r);
    L = __fadd_rn(__fadd_rn(r, -__fadd_rn(t, -bb)), __fadd_rn(L, -bb));
    H = t;
  }
}

template <int S>
__device__ __forceinline__ void store_slices(const float d[4][S], __nv_bfloat16* out, long long slice_stride) {
#pragma unroll
  for (int s = 0; s < S; ++s) {
    // every digit has at most 8 significant bits: the top half of its FP32 pattern is its BF16
    uint2 pk;
    pk.x = (__float_as_uint(d[0][s]) >> 16) | (__float_as_uint(d[1][s]) & 0xffff0000u);
    pk.y = (__float_as_uint(d[2][s]) >> 16) | (__float_as_uint(d[3][s]) & 0xffff0000u);
    *reinterpret_cast<uint2*>(out + s * slice_stride) = pk;
  }
}

// The entries of one row segment: group-max contribution and the source values.
template <class Src>
struct Seg {
  double v[4];
  float hi[4], lo[4];
  __device__ void load(const Src& src, long long row, int k2) {
    if constexpr (Src::kDF) {
      src.load4(row, k2, hi, lo);
    } else {
      src.load4(row, k2, v);
    }
  }
  __device__ void zero() {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      v[i] = 0.0;
      hi[i] = lo[i] = 0.f;
    }
  }
  // any entry not exactly zero (a non-finite one counts)
  __device__ bool nonzero() const {
    bool nz = false;
#pragma unroll
    for (int i = 0; i < 4; ++i) nz = nz || v[i] != 0.0 || !(v[i] == v[i]) || hi[i] != 0.f || lo[i] != 0.f;
    return nz;
  }
  // max key (FP64) or max |hi| (double-float); bad = non-finite seen
  __device__ unsigned long long key() const {
    unsigned long long k = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) k = max(k, abs_key(v[i]));
    return k;
  }
  __device__ float fmaxabs(bool& bad) const {
    float m = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float a = fabsf(hi[i]);
      bad = bad || !(a <= 3.0e38f) || !(fabsf(lo[i]) <= 3.0e38f);
      m = fmaxf(m, a);
    }
    return m;
  }
  template <int S>
  __device__ void write(const GroupScale& g, __nv_bfloat16* out, long long slice_stride) const {
    float d[4][S];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if constexpr (Src::kDF)
        digits_df<S>(hi[i], lo[i], g, d[i]);
      else
        digits_fp64<S>(v[i], g, d[i]);
    }
    store_slices<S>(d, out, slice_stride);
  }
};

// warp-wide group scale of the segments held by the 32 lanes
template <class Src>
__device__ __forceinline__ GroupScale warp_scale(const Seg<Src>& sg) {
  if constexpr (Src::kDF) {
    bool bad = false;
    float m = sg.fmaxabs(bad);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    bad = __any_sync(0xffffffffu, bad);
    return scale_from_float(m, bad);
  } else {
    unsigned long long k = sg.key();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) k = max(k, __shfl_xor_sync(0xffffffffu, k, o));
    return scale_from_key(k);
  }
}

// A operands: one warp per (row, chunk of 128 K entries).
// out: [S][rows_pad][ldk] bf16; scale: [nch][rows_pad] float.
// mask (when non-null): bit ch of word (row / 128) * mw + ch / 32 is set when the group is not
// zero (its scale is nonzero or NaN), i.e. when the chunk holds a nonzero entry of the row tile.
template <int S, class Src>
__global__ void k_slice_chunks(Src src, int rows_pad, int ldk, int nch, __nv_bfloat16* __restrict__ out,
                               float* __restrict__ scale, unsigned* __restrict__ mask, int mw) {
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gw >= (long long)rows_pad * nch) return;  // warp-uniform
  const long long row = gw / nch;
  const int ch = (int)(gw % nch);
  const int k2 = ch * KC + 4 * lane;
  Seg<Src> sg;
  sg.zero();
  if (k2 < ldk) sg.load(src, row, k2);
  const GroupScale g = warp_scale(sg);
  if (k2 < ldk) sg.template write<S>(g, out + row * ldk + k2, (long long)rows_pad * ldk);
  if (lane == 0) {
    scale[(long long)ch * rows_pad + row] = g.sc;
    if (mask && g.sc != 0.f) atomicOr(&mask[(row >> 7) * mw + (ch >> 5)], 1u << (ch & 31));
  }
}

// B operands: one 128-thread block per row, one scale per row (two passes over
// the source: the largest magnitude, then the slices).  scale: [rows_pad] float.
template <int S, class Src>
__global__ void __launch_bounds__(128) k_slice_rows(Src src, int rows_pad, int ldk, __nv_bfloat16* __restrict__ out,
                                                    float* __restrict__ scale, unsigned* __restrict__ mask, int mw) {
  static_assert(!Src::kDF, "row-scaled operands come from FP64 sources");
  __shared__ unsigned long long red[4];
  const long long row = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  unsigned long long k = 0;
  Seg<Src> sg;
  for (int k2 = 4 * tid; k2 < ldk; k2 += 512) {
    sg.load(src, row, k2);
    k = max(k, sg.key());
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) k = max(k, __shfl_xor_sync(0xffffffffu, k, o));
  if (lane == 0) red[wid] = k;
  __syncthreads();
  k = max(max(red[0], red[1]), max(red[2], red[3]));
  const GroupScale g = scale_from_key(k);
  // warp wid covers the 128 entries [base, base + 128) of one chunk per pass (warp-uniform bound)
  for (int base = 128 * wid; base < ldk; base += 512) {
    const int k2 = base + 4 * lane;
    const bool in = k2 < ldk;
    if (in) sg.load(src, row, k2); else sg.zero();
    if (in) sg.template write<S>(g, out + row * ldk + k2, (long long)rows_pad * ldk);
    const bool nz = __any_sync(0xffffffffu, in && sg.nonzero());
    if (mask && nz && lane == 0) {
      const int ch = base >> 7;
      atomicOr(&mask[(row >> 7) * mw + (ch >> 5)], 1u << (ch & 31));
    }
  }
  if (tid == 0) scale[row] = g.sc;
}

// ---------------------------------------------------------------- host side
inline int pad32(int k) { return (k + 31) / 32 * 32; }
inline int pad128(int k) { return (k + 127) / 128 * 128; }

// A sliced operand: bf16 slices [S][rows_pad][ldk] and scales, per (chunk, row)
// ([nch][rows_pad], A operands) or per row ([rows_pad], B operands).
struct Sliced {
  RawBuf data, scale, mask;
  int rows_pad = 0, ldk = 0, nch = 0, S = 0, mw = 0;
  bool row_scale = false;
  void shape(DevicePool* pool, int S_, int rows, int K2, bool per_row) {
    S = S_;
    row_scale = per_row;
    rows_pad = pad128(std::max(rows, 1));
    ldk = pad32(std::max(K2, 1));
    nch = (ldk + KC - 1) / KC;
    mw = (nch + 31) / 32;
    data.ensure(pool, sizeof(__nv_bfloat16) * (size_t)S * rows_pad * ldk);
    scale.ensure(pool, sizeof(float) * (size_t)(per_row ? 1 : nch) * rows_pad);
    // one bit per (128-row tile, chunk) holding a nonzero entry (exact zeros of conserved charges)
    mask.ensure(pool, sizeof(unsigned) * (size_t)(rows_pad / 128) * mw);
  }
};

template <class Src>
void slice(cudaStream_t st, const Src& src, Sliced& o) {
  __nv_bfloat16* d = o.data.as<__nv_bfloat16>();
  float* sc = o.scale.as<float>();
  unsigned* mk = o.mask.as<unsigned>();
  TDVP_CUDA(cudaMemsetAsync(mk, 0, sizeof(unsigned) * (size_t)(o.rows_pad / 128) * o.mw, st));
  if (o.row_scale) {
    if constexpr (Src::kDF) {
      throw TdvpError(TDVP_ERR_INVALID_ARG, "slice: row-scaled operands come from FP64 sources");
    } else {
      if (o.S == 4)
        k_slice_rows<4, Src><<<o.rows_pad, 128, 0, st>>>(src, o.rows_pad, o.ldk, d, sc, mk, o.mw);
      else
        k_slice_rows<3, Src><<<o.rows_pad, 128, 0, st>>>(src, o.rows_pad, o.ldk, d, sc, mk, o.mw);
    }
  } else {
    const int blocks = ceil_div((long long)o.rows_pad * o.nch * 32, 256);
    if (o.S == 4)
      k_slice_chunks<4, Src><<<blocks, 256, 0, st>>>(src, o.rows_pad, o.ldk, o.nch, d, sc, mk, o.mw);
    else
      k_slice_chunks<3, Src><<<blocks, 256, 0, st>>>(src, o.rows_pad, o.ldk, o.nch, d, sc, mk, o.mw);
  }
  TDVP_CHECK_LAUNCH();
}

CUtensorMap make_map3(const Sliced& o, int box_rows) {
  const void* base = o.data.as<void>();
  tdvp_require((reinterpret_cast<uintptr_t>(base) & 15) == 0, TDVP_ERR_INVALID_ARG, "TMA base not 16B aligned");
  tdvp_require(o.ldk % 32 == 0 && o.rows_pad % box_rows == 0, TDVP_ERR_INVALID_ARG, "sliced operand not padded");
  CUtensorMap m;
  std::memset(&m, 0, sizeof(m));
  cuuint64_t dims[3] = {(cuuint64_t)o.ldk, (cuuint64_t)o.rows_pad, (cuuint64_t)o.S};
  cuuint64_t strides[2] = {(cuuint64_t)o.ldk * 2, (cuuint64_t)o.rows_pad * o.ldk * 2};
  cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, (cuuint32_t)o.S};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box,
                           estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  tdvp_require(r == CUDA_SUCCESS, TDVP_ERR_CUDA, "cuTensorMapEncodeTiled (bf16) failed: " + std::to_string((int)r));
  return m;
}

template <int S>
void launch_bf16s(cudaStream_t st, const CUtensorMap& ma, const CUtensorMap& mb, int M, int N, int nkb,
                  int kb_split, int splits, const float* sA, long long lsA, const float* sB, void* out,
                  long long ldo, long long split_stride, int out_df, int* d_err, const unsigned* maskA,
                  const unsigned* maskB, int mw) {
  static const bool attr = [] {
    // the register hand-over inside the kernel is sized for exactly this launch allocation
    cudaFuncAttributes fa;
    TDVP_CUDA(cudaFuncGetAttributes(&fa, k_gemm_bf16s<S>));
    tdvp_require(fa.numRegs == REGS_LAUNCH, TDVP_ERR_CUDA,
                 "gemm_bf16s: kernel built with " + std::to_string(fa.numRegs) + " registers, expected " +
                     std::to_string(REGS_LAUNCH));
    TDVP_CUDA(cudaFuncSetAttribute(k_gemm_bf16s<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   SCfg<S>::SMEM_BYTES));
    return true;
  }();
  (void)attr;
  dim3 grid(ceil_div(N, BN), ceil_div(M, BM), splits);
  tdvp_require(grid.y <= 65535 && splits <= 65535, TDVP_ERR_INVALID_ARG, "gemm_bf16s: grid too large");
  k_gemm_bf16s<S><<<grid, THREADS, SCfg<S>::SMEM_BYTES, st>>>(ma, mb, M, N, nkb, kb_split, sA, lsA, sB, out, ldo,
                                                              split_stride, out_df, d_err, maskA, maskB, mw);
  TDVP_CHECK_LAUNCH();
}

// Sum of the split-K partials (double-float pairs, one [M][N] slab per split) into
// the output: FP64, or double-float pairs when out_df.
__global__ void k_splitk_df(const float2* __restrict__ ws, int splits, int M, int N, void* __restrict__ out,
                            long long ldo, int out_df) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)M * N) return;
  const long long m = e / N, n = e % N;
  double sum = 0.0;
  for (int z = 0; z < splits; ++z) {
    const float2 v = ws[(long long)z * M * N + e];
    sum += (double)v.x + (double)v.y;
  }
  if (out_df) {
    const float hi = (float)sum;
    static_cast<float2*>(out)[m * ldo + n] = make_float2(hi, (float)(sum - (double)hi));
  } else {
    static_cast<double*>(out)[m * ldo + n] = sum;
  }
}

// Splits of K (whole 128-deep chunks) that minimise waves of CTAs x work per CTA:
// few output tiles (a narrow product or a long K) would otherwise leave most SMs idle.
int choose_splits(long long tiles, int nchunks) {
  static const int sms = [] {
    int dev = 0, n = 0;
    TDVP_CUDA(cudaGetDevice(&dev));
    TDVP_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
    return n > 0 ? n : 148;
  }();
  int best = 1;
  double best_t = (double)((tiles + sms - 1) / sms);
  for (int sp = 2; sp <= std::min(32, nchunks); ++sp) {
    const int cps = (nchunks + sp - 1) / sp;
    const int real = (nchunks + cps - 1) / cps;
    const double t = (double)((tiles * real + sms - 1) / sms) * cps / nchunks + 0.02;  // + reduction pass
    if (t < 0.9 * best_t) {
      best_t = t;
      best = real;
    }
  }
  return best;
}

// out[M x N] (row-major, ldo) = A B^T over the sliced real operands; FP64 entries, or
// double-float (hi, lo) FP32 pairs when out_df.  Products with few output tiles split
// K over more CTAs (partials in a pool workspace, summed by k_splitk_df).
void gemm_bf16s(cudaStream_t st, DevicePool* pool, const Sliced& A, const Sliced& B, int M, int N, void* out,
                long long ldo, bool out_df, int* d_err) {
  if (M <= 0 || N <= 0) return;
  tdvp_require(A.ldk == B.ldk && A.S == B.S, TDVP_ERR_INVALID_ARG, "gemm_bf16s: operand K or slices differ");
  tdvp_require(M <= A.rows_pad && N <= B.rows_pad, TDVP_ERR_INVALID_ARG, "gemm_bf16s: operand rows");
  tdvp_require(!A.row_scale && B.row_scale, TDVP_ERR_INVALID_ARG, "gemm_bf16s: operand scaling groups");
  const CUtensorMap ma = make_map3(A, BM), mb = make_map3(B, BN);
  const int nkb = A.ldk / BK;
  const int nchunks = (nkb + KC_KB - 1) / KC_KB;
  const long long tiles = (long long)ceil_div(N, BN) * ceil_div(M, BM);
  const int splits = pool ? choose_splits(tiles, nchunks) : 1;
  const int kb_split = splits > 1 ? ((nchunks + splits - 1) / splits) * KC_KB : nkb;
  RawBuf ws;
  void* dst = out;
  long long ld = ldo, stride = 0;
  int df = out_df ? 1 : 0;
  if (splits > 1) {
    ws.ensure(pool, sizeof(float2) * (size_t)splits * M * N);
    dst = ws.as<void>();
    ld = N;
    stride = (long long)M * N;
    df = 1;
  }
  tdvp_require(A.mw == B.mw && (kb_split + KC_KB - 1) / KC_KB <= kMaxChunks, TDVP_ERR_INVALID_ARG,
               "gemm_bf16s: chunk masks or chunks per split out of range");
  const unsigned* mA = A.mask.as<unsigned>();
  const unsigned* mB = B.mask.as<unsigned>();
  if (A.S == 4)
    launch_bf16s<4>(st, ma, mb, M, N, nkb, kb_split, splits, A.scale.as<float>(), A.rows_pad, B.scale.as<float>(),
                    dst, ld, stride, df, d_err, mA, mB, A.mw);
  else
    launch_bf16s<3>(st, ma, mb, M, N, nkb, kb_split, splits, A.scale.as<float>(), A.rows_pad, B.scale.as<float>(),
                    dst, ld, stride, df, d_err, mA, mB, A.mw);
  if (splits > 1) {
    const long long n = (long long)M * N;
    k_splitk_df<<<ceil_div(n, 256), 256, 0, st>>>(ws.as<float2>(), splits, M, N, out, ldo, out_df ? 1 : 0);
    TDVP_CHECK_LAUNCH();
  }
}
}  // namespace tcb

using namespace tcb;

struct TcSliceCache {
  long long key = -1;
  int S = 0;
  Sliced L, R, X, T2;
  RawBuf T1;
};

namespace {
TcSliceCache& slice_cache(Scratch& s) {
  if (!s.tcs) s.tcs = std::make_shared<TcSliceCache>();
  return *s.tcs;
}
int* tc_err(cudaStream_t st, Scratch& s) {
  TcEnvCache& c = s.tc;
  if (c.err.bytes() == 0) {
    c.err.ensure(s.pool, sizeof(int));
    TDVP_CUDA(cudaMemsetAsync(c.err.as<int>(), 0, sizeof(int), st));
  }
  c.pending = true;
  return c.err.as<int>();
}
}  // namespace

int bf16_slices(int precision) { return precision == TDVP_PREC_BF16X6 ? 3 : 4; }

void gemm_chunk_pairs(long long out[2]) {
  unsigned long long h[2] = {0, 0};
  TDVP_CUDA(cudaMemcpyFromSymbol(h, tcb::g_chunk_pairs, sizeof(h)));
  out[0] = (long long)h[0];
  out[1] = (long long)h[1];
}

void heff_bf16s(cudaStream_t st, Scratch& s, const SiteOp& op, const cplx* x, cplx* y, int S) {
  const int ml = op.ml, mr = op.mr, wl = op.wl, wr = op.wr, d = op.d;
  TcSliceCache& c = slice_cache(s);
  DevicePool* pool = s.pool;
  int* err = tc_err(st, s);
  if (op.env_key < 0 || c.key != op.env_key || c.S != S) {
    // L as the A operand: rows (w, a), K = (a', re/im)
    c.L.shape(pool, S, ml * wl, 2 * ml, false);
    slice(st, SrcLwa{op.L, ml, wl}, c.L);
    // R[b][(v,b')] is B[k=(v,b')][n=b] stored n-major (op T)
    c.R.shape(pool, S, 2 * mr, 2 * wr * mr, true);
    slice(st, SrcB{op.R, (long long)wr * mr, wr * mr, mr, OP_T}, c.R);
    c.key = op.env_key;
    c.S = S;
  }
  // stage 1: T1[(w,a)][(s',b',c)] = L x     (x[a'][(s',b')] is B[k=a'][n=(s',b')])
  c.X.shape(pool, S, 2 * d * mr, 2 * ml, true);
  slice(st, SrcB{x, (long long)d * mr, ml, d * mr, OP_N}, c.X);
  const int M1 = ml * wl, N1 = 2 * d * mr;
  c.T1.ensure(pool, sizeof(float2) * (size_t)M1 * N1);  // double-float
  gemm_bf16s(st, pool, c.L, c.X, M1, N1, c.T1.as<void>(), N1, true, err);
  // stage 2: MPO tensor, sliced straight into the stage-3 A operand
  const WSparse& ws = *op.W;
  c.T2.shape(pool, S, ml * d, 2 * wr * mr, false);
  tdvp_require(ws.d_l_val_df != nullptr, TDVP_ERR_INVALID_ARG, "heff_bf16s: MPO site without double-float values");
  slice(st, SrcStage2{c.T1.as<float4>(), ws.d_l_off, ws.d_l_idx, ws.d_l_val_df, ml, wl, wr, d, mr}, c.T2);
  // stage 3: y[(a,s)][(b,c)] = T2 R^T
  gemm_bf16s(st, pool, c.T2, c.R, ml * d, 2 * mr, y, 2 * mr, false, err);
}

void zgemm_bf16s(cudaStream_t st, Scratch& s, int S, int opA, int opB, int M, int N, int K, const cplx* A,
                 long long lda, const cplx* B, long long ldb, cplx* C, long long ldc) {
  if (M <= 0 || N <= 0) return;
  DevicePool* pool = s.pool;
  int* err = tc_err(st, s);
  Sliced a, b;
  a.shape(pool, S, M, 2 * std::max(K, 1), false);
  slice(st, SrcA{A, lda, M, K, opA}, a);
  b.shape(pool, S, 2 * N, 2 * std::max(K, 1), true);
  slice(st, SrcB{B, ldb, K, N, opB}, b);
  gemm_bf16s(st, pool, a, b, M, 2 * N, C, 2 * ldc, false, err);
}
