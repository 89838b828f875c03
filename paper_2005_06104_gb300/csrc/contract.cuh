// Tensor-network contractions of one site (H_eff, K_eff, environment updates)
// and the Lanczos local exponential, as free functions over device pointers.
// The engine and the handle-free C-ABI entry points share them.
#pragma once
#include <functional>
#include <memory>

#include "linalg.cuh"
#include "tc_gemm.cuh"

// Everything one-site contractions read: environments, MPO site, dimensions.
struct SiteOp {
  const cplx* L = nullptr;     // ml x wl x ml
  const cplx* R = nullptr;     // mr x wr x mr
  const WSparse* W = nullptr;  // MPO site (sparse lists on device)
  int ml = 0, mr = 0, wl = 0, wr = 0, d = 2;
  long long env_key = -1;      // identifies the (L, R) content for operand caching; -1 = never cache
};

struct TcSliceCache;  // sliced operands of the BF16 tensor-core path (tc_bf16.cu)

// Work buffers reused across calls (drawn from a pool).
struct Scratch {
  DevicePool* pool = nullptr;
  DArr t1, t2, t3;
  TcEnvCache tc;
  std::shared_ptr<TcSliceCache> tcs;
};

// Algorithmic flop count of one H_eff apply (8 real flops per complex multiply-add):
// 8 [ml d mr (ml wl + mr wr) + ml mr nnz(W)]
double heff_flops(const SiteOp& op);

// y[a,s,b] = sum L[a,w,a'] W[w,s,s',v] x[a',s',b'] R[b,v,b']
void heff_fp64(cudaStream_t st, Scratch& s, const SiteOp& op, const cplx* x, cplx* y);
void heff_tf32x3(cudaStream_t st, Scratch& s, const SiteOp& op, const cplx* x, cplx* y);
// The same on the BF16 exact-slice tensor-core GEMM with S = 3 or 4 slices per operand.
void heff_bf16s(cudaStream_t st, Scratch& s, const SiteOp& op, const cplx* x, cplx* y, int S);
// Slices per operand of a BF16 precision mode (BF16X6: 3, BF16X10: 4).
int bf16_slices(int precision);
// (output tile, 128-entry K chunk) pairs the BF16 tensor-core GEMMs visited on the current
// device since the library loaded: out[0] all of them, out[1] the ones multiplied (the rest
// had an all-zero A or B tile and were skipped).  Synchronises the device.
void gemm_chunk_pairs(long long out[2]);
bool prec_is_bf16(int precision);
void heff_apply_prec(cudaStream_t st, Scratch& s, const SiteOp& op, const cplx* x, cplx* y, int precision);
// C = opA(A) opB(B) (complex, alpha = 1, beta = 0) on the tensor cores (split TF32,
// FP32 accumulation, FP64 output).
void zgemm_tc(cudaStream_t st, Scratch& s, int opA, int opB, int M, int N, int K, const cplx* A, long long lda,
              const cplx* B, long long ldb, cplx* C, long long ldc);
// C = opA(A) opB(B) on the BF16 exact-slice tensor-core GEMM (S slices, FP64 output).
void zgemm_bf16s(cudaStream_t st, Scratch& s, int S, int opA, int opB, int M, int N, int K, const cplx* A,
                 long long lda, const cplx* B, long long ldb, cplx* C, long long ldc);
// The tensor-core GEMM of `precision` (zgemm_tc for the TF32 modes, zgemm_bf16s for
// the BF16 modes) when the product is large enough to fill its tiles, the FP64
// GEMM otherwise (alpha = 1, beta = 0).
void zgemm_prec(cudaStream_t st, Scratch& s, int precision, int opA, int opB, int M, int N, int K, const cplx* A,
                long long lda, const cplx* B, long long ldb, cplx* C, long long ldc);
// Reads the tensor-core error word of the launches since the last check (synchronises);
// throws TDVP_ERR_TIMEOUT when a bounded device wait ran out.
void tc_check(cudaStream_t st, Scratch& s);

// y[a,c] = sum L[a,w,a'] x[a',b'] R[c,w,b']   (x: ml x mr; L: ml x w x ml; R: mr x w x mr)
void keff_fp64(cudaStream_t st, Scratch& s, const cplx* L, int ml, const cplx* R, int mr, int w, const cplx* x,
               cplx* y, int precision = TDVP_PREC_FP64);

// Lout[b,v,b'] = sum conj(A[a,s,b]) L[a,w,a'] W[w,s,s',v] A[a',s',b']
void env_left_fp64(cudaStream_t st, Scratch& s, const cplx* L, const WSparse& W, const cplx* A, int ml, int mr,
                   int d, cplx* Lout, int precision = TDVP_PREC_FP64);
// Rout[a,w,a'] = sum conj(B[a,s,b]) W[w,s,s',v] R[b,v,b'] B[a',s',b']
void env_right_fp64(cudaStream_t st, Scratch& s, const cplx* R, const WSparse& W, const cplx* B, int ml, int mr,
                    int d, cplx* Rout, int precision = TDVP_PREC_FP64);

// Lanczos exponential with full re-orthogonalisation applied twice:
// out = exp(-i delta Op) x (kind 0) or exp(-delta Op) x (kind 1), Op Hermitian.
// Returns the Krylov dimension used; throws LANCZOS_NOT_CONVERGED when nmax
// steps do not bring the error estimate below tol.
struct LanczosWork {
  DArr V, w, c, y;
  double* real = nullptr;  // device: alpha[64], beta[65], nrm2, err[2], scratch norms; [256, 384):
                           // the error estimates of each iteration of a speculative run
  void init(DevicePool* pool);
  void release();
};
// hint (may be null): the Krylov dimension of the previous run of the same operator kind; read
// to launch the first iterations of a small local problem without a host round trip each,
// and updated to this run's dimension.  Results do not depend on it.
int lanczos_expm(cudaStream_t st, DevicePool* pool, Blas1& blas, LanczosWork& lw,
                 const std::function<void(const cplx*, cplx*)>& op, const cplx* x, cplx* out, long long n,
                 double delta, int kind, double tol, int nmax, int* hint = nullptr);
