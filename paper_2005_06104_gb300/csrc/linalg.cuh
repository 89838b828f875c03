// FP64 complex building blocks of the GSE-TDVP1 path (CUDA cores).
#pragma once
#include "common.cuh"

enum GemmOp { OP_N = 0, OP_T = 1, OP_C = 2, OP_R = 3 };  // R = conjugate, not transposed

// C[m,n] = alpha * sum_k opA(A)[m,k] opB(B)[k,n] + beta * C[m,n], all row-major.
// opA(A)[m,k] = A[m*lda+k] (N), A[k*lda+m] (T), conj(A[k*lda+m]) (C), conj(A[m*lda+k]) (R).
// batch > 1 uses strides sA, sB, sC (elements).  With a pool `ws`, GEMMs with few
// output tiles split K over more blocks (partials reduced in a fixed order);
// without one nothing is allocated.
void zgemm(cudaStream_t st, int opA, int opB, int M, int N, int K, cplx alpha, const cplx* A,
           long long lda, const cplx* B, long long ldb, cplx beta, cplx* C, long long ldc,
           int batch = 1, long long sA = 0, long long sB = 0, long long sC = 0, DevicePool* ws = nullptr);

// Sparse description of one MPO site tensor W[w][s][t][v] for the contraction
// stages: entries grouped by output (s, v) for left moves and by (s, w) for
// right moves.
struct WSparse {
  int wl = 0, wr = 0, d = 0;
  int nnz = 0;
  // left grouping: for out row (s, v): entries (w, t) with value
  std::vector<int> l_off;           // d*wr + 1
  std::vector<int> l_idx;           // 2*nnz: (w, t)
  std::vector<cplx> l_val;
  std::vector<float4> l_val_df;     // l_val as double-float pairs (re hi, re lo, im hi, im lo)
  // right grouping: for out row (s, w): entries (v, t)
  std::vector<int> r_off;           // d*wl + 1
  std::vector<int> r_idx;
  std::vector<cplx> r_val;
  // device copies
  int* d_l_off = nullptr;
  int* d_l_idx = nullptr;
  cplx* d_l_val = nullptr;
  float4* d_l_val_df = nullptr;
  int* d_r_off = nullptr;
  int* d_r_idx = nullptr;
  cplx* d_r_val = nullptr;
  void build(const cplx* W, int wl, int wr, int d);  // host W
  void upload();
  void free_device();
};

// out[a][s][v][c] = sum_{(w,t)} W[w,s,t,v] in[a][w][t][c]      (A = rows a, C = cols c)
void wstage_left(cudaStream_t st, const WSparse& w, const cplx* in, cplx* out, int A, int C);
// out[s][b][w][c] = sum_{(v,t)} W[w,s,t,v] in[b][v][t][c]
void wstage_right(cudaStream_t st, const WSparse& w, const cplx* in, cplx* out, int B, int C);

// out[s][a][b] = in[a][s][b] (and back with the inverse flag)
void permute_asb_sab(cudaStream_t st, const cplx* in, cplx* out, int A, int S, int B);

// Phases timed by the tracer (CUDA events on the engine stream).
enum TracePhase {
  PH_LANCZOS_SITE = 0, PH_LANCZOS_BOND, PH_SVD, PH_ENV, PH_KRYLOV, PH_EXTEND, PH_CANON,
  PH_KRYLOV_RENV, PH_KRYLOV_EIG, PH_EXTEND_SVD,
  // inside every blocked SVD / eigendecomposition: block detection (mask, host union-find,
  // gather), pivoted Cholesky, Jacobi sweeps, selection and scatter of the kept vectors
  PH_SVD_PREP, PH_SVD_PCHOL, PH_SVD_JACOBI, PH_SVD_SELECT,
  // every block QR / LQ of a gauge move that cuts nothing
  PH_QR, PH_COUNT
};

struct Tracer {
  bool on = false;
  cudaStream_t st = nullptr;
  std::vector<cudaEvent_t> pool;
  struct Mark {
    int phase;
    cudaEvent_t a, b;
  };
  std::vector<Mark> marks;
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    TDVP_CUDA(cudaEventCreate(&e));
    return e;
  }
  // sums per phase (ms) and recycles the events; the stream must be idle
  void read(double* out, int n) {
    for (int p = 0; p < n; ++p) out[p] = 0.0;
    for (auto& m : marks) {
      float t = 0.f;
      TDVP_CUDA(cudaEventElapsedTime(&t, m.a, m.b));
      if (m.phase < n) out[m.phase] += t;
      pool.push_back(m.a);
      pool.push_back(m.b);
    }
    marks.clear();
  }
  void release() {
    for (auto& m : marks) {
      cudaEventDestroy(m.a);
      cudaEventDestroy(m.b);
    }
    for (auto e : pool) cudaEventDestroy(e);
    marks.clear();
    pool.clear();
  }
};

// Records one interval of `phase` on the stream while it is in scope.
struct PhaseScope {
  Tracer& tr;
  int phase;
  cudaEvent_t a = nullptr;
  PhaseScope(Tracer& t, int p) : tr(t), phase(p) {
    if (tr.on) {
      a = tr.get();
      cudaEventRecord(a, tr.st);
    }
  }
  ~PhaseScope() {
    if (tr.on && a) {
      cudaEvent_t b = tr.get();
      cudaEventRecord(b, tr.st);
      tr.marks.push_back({phase, a, b});
    }
  }
};

// The tracer of the handle whose call runs on this thread (null when tracing is off);
// set by the C-ABI entry points, read by the factorisations.
extern thread_local Tracer* t_tracer;

// PhaseScope on the active tracer, when there is one.
struct ActivePhase {
  Tracer idle;
  PhaseScope ps;
  explicit ActivePhase(int p) : ps(t_tracer ? *t_tracer : idle, p) {}
};

// Reductions (deterministic, two-pass).  Results land in device memory.
struct Blas1 {
  DevicePool* pool = nullptr;
  DArr partial;          // scratch for block partials
  int max_blocks = 0;
  void init(DevicePool* p, int sm_count);
  // out[k] = sum_i conj(V[k*ldv + i]) w[i], k < nvec
  void multi_dot(cudaStream_t st, const cplx* V, long long ldv, int nvec, const cplx* w,
                 long long n, cplx* out);
  // *out = sum_i |x_i|^2 (double in device memory)
  void norm2(cudaStream_t st, const cplx* x, long long n, double* out);
  // One launch of a fused Lanczos step (partials reduced by the last block):
  //   mode 0: cout = V^H w, alpha[j] = Re cout[j]
  //   mode 1: w -= V cin, then cout = V^H w
  //   mode 2: w -= V cin, then *nrm2 = |w|^2, *beta_slot = sqrt(*nrm2)
  void lanczos_fused(cudaStream_t st, int mode, const cplx* V, long long ldv, int nvec, cplx* w, long long n,
                     const cplx* cin, cplx* cout, double* alpha, int j, double* nrm2, double* beta_slot);
  unsigned* counter = nullptr;  // ticket of the last-block reductions (reset by that block)
  void release();
};
// w[i] -= sum_k V[k*ldv+i] c[k]
void multi_axpy_sub(cudaStream_t st, cplx* w, const cplx* V, long long ldv, int nvec,
                    const cplx* c, long long n);
// y[i] = scale * sum_k V[k*ldv+i] c[k]  (scale read from host value)
void multi_combine(cudaStream_t st, cplx* y, const cplx* V, long long ldv, int nvec,
                   const cplx* c, double scale, long long n);
// dst = src * (1 / sqrt(*nrm2))   (nrm2 in device memory)
void scale_by_inv_sqrt(cudaStream_t st, cplx* dst, const cplx* src, const double* nrm2,
                       long long n);
// the same with zeros when *nrm2 is not a positive finite number above 1e-200
void scale_by_inv_sqrt_guarded(cudaStream_t st, cplx* dst, const cplx* src, const double* nrm2, long long n);
void scale_host(cudaStream_t st, cplx* dst, const cplx* src, cplx s, long long n);
void fill_zero(cudaStream_t st, cplx* p, long long n);
// Lanczos bookkeeping: alpha[j] = Re c[j]
void copy_real_part(cudaStream_t st, const cplx* c, int j, double* alpha);
// y[0..n) = exp(coef * T) e_0 for T tridiagonal (diag alpha, off beta[1..n-1]);
// kind 0: coef = -i delta, kind 1: coef = -delta.  err[0] = sqrt(nrm2_next) |y[n-1]|,
// err[1] = sqrt(nrm2_next) (beta_n), both written to device memory.
void tridiag_expv(cudaStream_t st, const double* alpha, const double* beta, int n,
                  double delta, int kind, const double* nrm2_next, cplx* y, double* err);
void store_beta(cudaStream_t st, const double* nrm2, double* beta_slot);

// One-sided Jacobi SVD of a complex FP64 matrix (row-major rows x cols).
struct SvdOut {
  int rows = 0, cols = 0, rank = 0;  // rank = number of computed singular values kept
  std::vector<double> s;             // sorted descending, all min(rows, cols)
  // U's columns and Vh's rows: the kept vectors grouped by block of the exact-zero pattern
  // (blocks in order of their smallest row, descending singular value inside a block), so
  // each conserved-charge sector of the new index is contiguous
  DArr U;                            // rows x keep   (row-major)
  DArr Vh;                           // keep x cols   (row-major)
  int sweeps = 0;
};
// Computes the SVD and sorts it; `select` picks how many to keep from the sorted s.
// want_u/want_v: which factors to materialise.
template <class Select>
void svd_jacobi(cudaStream_t st, DevicePool* pool, const cplx* M, int rows, int cols,
                Select select, SvdOut& out, bool want_u = true, bool want_v = true);
// implemented for this signature:
void svd_jacobi_keep(cudaStream_t st, DevicePool* pool, const cplx* M, int rows, int cols,
                     int (*select)(const std::vector<double>& s, void* ctx), void* ctx,
                     SvdOut& out, bool want_u, bool want_v);
// Process-wide counters of the SVD driver (calls, calls that split into blocks, blocks).
struct SvdCounters {
  std::atomic<long long> calls{0}, blocked{0}, blocks{0};
  std::atomic<long long> sweeps{0}, max_sweeps{0};  // Jacobi sweeps over all (blocks of) calls, and the most in one
  std::atomic<long long> large_blocks{0}, max_q{0};  // blocks too large for the batched path; widest block
};
inline void atomic_max(std::atomic<long long>& a, long long v) {
  long long cur = a.load(std::memory_order_relaxed);
  while (v > cur && !a.compare_exchange_weak(cur, v, std::memory_order_relaxed)) {
  }
}
extern SvdCounters g_svd_counters;

// The same contract, exploiting block structure (exact zeros from conserved
// quantum numbers): independent SVDs per connected block, merged spectrum.
// psd: M is Hermitian positive semidefinite and only U is wanted; the blocks are then
// factorised by pivoted Cholesky and the Jacobi SVD runs on the factor (fewer sweeps);
// out.s holds eigenvalues.
// jacobi_fp32 (psd only): the Jacobi rotations of the FP64 Cholesky factor run in FP32
// (eigenvalues to about 1e-7 relative, eigenvectors to about 1e-7 / relative gap); for the
// Krylov vectors of the precision forms, whose density matrices are formed to about that
// accuracy by the tensor-core GEMMs.
void svd_blocked_keep(cudaStream_t st, DevicePool* pool, const cplx* M, int rows, int cols,
                      int (*select)(const std::vector<double>& s, void* ctx), void* ctx,
                      SvdOut& out, bool want_u, bool want_v, bool psd = false, bool jacobi_fp32 = false);
template <class Select>
inline void svd_jacobi(cudaStream_t st, DevicePool* pool, const cplx* M, int rows, int cols,
                       Select select, SvdOut& out, bool want_u, bool want_v) {
  auto thunk = [](const std::vector<double>& s, void* ctx) -> int {
    return (*static_cast<Select*>(ctx))(s);
  };
  svd_blocked_keep(st, pool, M, rows, cols, thunk, &select, out, want_u, want_v);
}
// Eigendecomposition of a Hermitian positive semidefinite n x n matrix: out.s the
// eigenvalues (descending), out.U the kept eigenvectors (n x keep).
template <class Select>
inline void eig_psd_jacobi(cudaStream_t st, DevicePool* pool, const cplx* M, int n, Select select, SvdOut& out,
                           bool jacobi_fp32 = false) {
  auto thunk = [](const std::vector<double>& s, void* ctx) -> int {
    return (*static_cast<Select*>(ctx))(s);
  };
  svd_blocked_keep(st, pool, M, n, n, thunk, &select, out, true, false, true, jacobi_fp32);
}

// copy a (rows x cols) block into a (rows x ldo) destination at column offset
void copy_block(cudaStream_t st, cplx* dst, long long ldd, const cplx* src, long long lds,
                int rows, int cols);

// Thin QR (orient 0) or LQ (orient 1) of a row-major complex FP64 matrix, block by block
// (the exact-zero blocks of svd_blocked_keep), by Householder reflections in FP64.
// orient 0: M = Q C, Q rows x k with orthonormal columns, C k x cols.
// orient 1: M = C Q, Q k x cols with orthonormal rows, C rows x k.
// k = sum over blocks of min(block rows, block cols): no direction is dropped.  k = 0 (and
// no buffers) for a zero matrix.  Waits in the kernel are bounded (TDVP_ERR_TIMEOUT).
struct QrOut {
  int k = 0;
  DArr Q, C;
  double diag_min = 0.0, diag_max = 0.0;  // smallest and largest |R_jj| over all blocks
  // every block has full numerical rank: all |R_jj| > rtol max |R_jj| (a rank-deficient block
  // has a column in the span of the ones before it, whose remainder R_jj vanishes)
  bool full_rank(double rtol) const { return k > 0 && diag_min > rtol * diag_max; }
};
void qr_blocked(cudaStream_t st, DevicePool* pool, const cplx* M, int rows, int cols, int orient, QrOut& out);

// Row order that makes each block of M's exact-zero pattern (rows x cols, row-major) one
// contiguous range: blocks in order of their smallest row, rows ascending inside a block, zero
// rows last.  Empty when M is one block or already in that order.
std::vector<int> sector_row_order(cudaStream_t st, DevicePool* pool, const cplx* M, int rows, int cols);
// out[r, :] = M[perm[r], :]  (out and M must not overlap)
void gather_rows(cudaStream_t st, const cplx* M, int rows, int cols, const std::vector<int>& perm, cplx* out);
