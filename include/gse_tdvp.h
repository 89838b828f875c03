/*
 * gse_tdvp.h -- C ABI of libgsetdvp.so, a GB300 (sm_103a) implementation of the
 * global-subspace-expanded one-site TDVP (GSE-TDVP1) of Yang & White,
 * "Time Dependent Variational Principle with Ancillary Krylov Subspace"
 * (arXiv:2005.06104).
 *
 * Conventions (every call):
 *   - complex numbers are complex128 stored as interleaved (re, im) doubles;
 *   - an MPS site tensor A_i[m_{i-1}][d][m_i] is row-major, m_0 = m_N = 1
 *     (the form of Eq. 1);
 *   - an MPO site tensor W_i[w_{i-1}][d][d][w_i] is row-major and acts as
 *     <s|W|s'> (second index output spin, third input spin), w_0 = w_N = 1;
 *   - the MPO is in finite-state ("start/done") form: at every inner bond channel
 *     0 means "no operator placed yet" and channel w_i - 1 means "term complete";
 *     the left boundary is "start", the right boundary is "done".  This is what
 *     lets the library build the MPO of 1 - i tau H from the MPO of H (Sec. I.C
 *     step 1) with the same bond dimension;
 *   - sites are numbered 0..N-1; "bond b" joins sites b-1 and b (1 <= b <= N-1);
 *   - every call returns a tdvp_status; on error the handle keeps the last state
 *     that completed a call and tdvp_last_error() describes the failure.  No C++
 *     exception crosses this boundary;
 *   - "stream" is a cudaStream_t passed as void*; every call is synchronous with
 *     respect to the host on return (results that land in host memory are valid,
 *     device outputs are complete).
 */
#ifndef GSE_TDVP_H
#define GSE_TDVP_H

#if defined(__GNUC__)
#define TDVP_API __attribute__((visibility("default")))
#else
#define TDVP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TDVP_OK = 0,
  TDVP_ERR_INVALID_ARG = 1,       /* null pointer, bad site index, bad option   */
  TDVP_ERR_SHAPE = 2,             /* inconsistent bond / physical dimensions    */
  TDVP_ERR_OUT_OF_MEMORY = 3,     /* device allocation failed                   */
  TDVP_ERR_LANCZOS_NOT_CONVERGED = 4,
  TDVP_ERR_NONFINITE = 5,         /* NaN or Inf met in a norm or a coefficient  */
  TDVP_ERR_TIMEOUT = 6,           /* a bounded device wait ran out              */
  TDVP_ERR_CUDA = 7,              /* a CUDA runtime call failed                 */
  TDVP_ERR_SVD_NOT_CONVERGED = 8
} tdvp_status;

typedef enum { TDVP_REAL = 0, TDVP_IMAG = 1 } tdvp_time;

/* Arithmetic of the H_eff / environment contractions. */
typedef enum {
  TDVP_PREC_FP64 = 0,       /* FP64 on CUDA cores                                       */
  TDVP_PREC_TF32X3 = 1,     /* tcgen05 kind::tf32, operands split hi+lo, 3 products,
                               FP32 accumulation in 32-deep chunks: H_eff and the
                               Krylov-vector GEMMs; environments stay FP64             */
  TDVP_PREC_TF32X3_ENV = 2, /* as TF32X3, and the sweep's environment updates too      */
  TDVP_PREC_BF16X10 = 3,    /* tcgen05 kind::f16: each operand cut into 4 fixed-point
                               BF16 slices per row and 128-deep K chunk (power-of-two
                               chunk scale), 10 slice products, the leading one summed
                               exactly, the other 9 in one FP32 accumulator per
                               chunk, chunks promoted into FP32 (hi, lo) pairs:
                               operands to 2^-33 of their group maxima, products to
                               about 2^-24 (measured 1e-8 relative per H_eff apply).
                               H_eff, K_eff, environments and Krylov-vector GEMMs  */
  TDVP_PREC_BF16X6 = 4      /* as BF16X10 with 3 slices and 6 products (about 2^-25)   */
} tdvp_precision;

typedef struct tdvp_handle tdvp_handle;

typedef struct {
  int n_sites;                   /* N >= 1                                          */
  int d;                         /* physical dimension (2 for spin 1/2)             */
  const int* bond_dims;          /* N + 1 entries, first and last equal 1           */
  const double* const* sites;    /* N host pointers, site i holds
                                    2 * m_i * d * m_{i+1} doubles                   */
} tdvp_mps_desc;

typedef struct {
  int n_sites;
  int d;
  const int* bond_dims;          /* N + 1 MPO bond dims w_i, first and last equal 1 */
  const double* const* sites;    /* N host pointers, site i holds
                                    2 * w_i * d * d * w_{i+1} doubles               */
} tdvp_mpo_desc;

typedef struct {
  double tau_re, tau_im;   /* Krylov operator 1 - i tau H (Eq. 10).  Real time:
                              tau = dt; imaginary time: i tau = 1/lambda (Sec. I.B) */
  double eps_k;            /* cutoff applying 1 - i tau H (Sec. I.B, eps_K)         */
  double eps_m;            /* cutoff of the mixed density matrix, Eq. 6 (eps_M)     */
  double eps;              /* cutoff inside the TDVP1 sweep, imaginary time (eps);
                              also of the two-site SVDs of tdvp_sweep2, both kinds  */
  int chi_max;             /* cap on every bond dimension (state and Krylov vectors)*/
  double lanczos_tol;      /* local exponential error target                        */
  int lanczos_max;         /* maximum Krylov dimension of one Lanczos run; a local
                              exponential that does not converge within it is split
                              into 2, 4, ... 64 equal sub-steps                     */
  int precision;           /* tdvp_precision used inside tdvp_sweep                 */
} tdvp_options;

/* Fills `opt` with: tau = 0.1, eps_k = eps_m = 1e-8, eps = 0, chi_max = 1024,
 * lanczos_tol = 1e-12, lanczos_max = 40, precision = FP64. */
TDVP_API tdvp_status tdvp_default_options(tdvp_options* opt);

/* Creates a handle.  Copies the host MPS and MPO into device memory that the
 * library owns (the caller keeps its buffers), brings the MPS to left-canonical
 * form with its centre at site N-1 (Eq. 1) and uploads the MPO of H.
 * Errors: INVALID_ARG (null), SHAPE (dims inconsistent), OUT_OF_MEMORY, CUDA. */
TDVP_API tdvp_status tdvp_create(const tdvp_mps_desc* mps, const tdvp_mpo_desc* mpo,
                        const tdvp_options* opt, void* stream, tdvp_handle** out);

TDVP_API tdvp_status tdvp_destroy(tdvp_handle* h);
TDVP_API tdvp_status tdvp_set_options(tdvp_handle* h, const tdvp_options* opt);
TDVP_API const char* tdvp_last_error(const tdvp_handle* h);
TDVP_API const char* tdvp_status_string(tdvp_status s);

/* Moves the orthogonality centre to `site` by exact gauge moves (a QR / LQ per
 * conserved-charge block when every |R_jj| exceeds 1e-10 of the largest, else an
 * SVD keeping every singular value above 1e-10 s_max) and builds the
 * environments L_site and R_site.  The state is unchanged. */
TDVP_API tdvp_status tdvp_canonicalize(tdvp_handle* h, int site);

/* GSE steps 1 and 2 (Sec. I.C): builds |psi~_l> = (1 - i tau H)^l |psi>,
 * l = 1..k-1 (Eq. 10, cutoff eps_k, cap chi_max, each normalised) and extends
 * the bond bases of |psi> right to left with the state-averaged projected
 * density matrix of Eqs. 5-7 (cutoff eps_m).  Ends with the centre at site 0.
 * weights: k-1 host doubles (w_l in rho~ = sum_l w_l C~_l^+ C~_l) or NULL for
 * all ones.  k = 1 only moves the centre to site 0.  The state is unchanged. */
TDVP_API tdvp_status tdvp_expand_basis(tdvp_handle* h, int k, const double* weights);

/* Memory of the density-matrix Krylov step (Sec. I.B).  Its right density
 * environments F_j hold (w_{j+1} m_{j+1})^2 complex entries each (about 3.3 GB per
 * site at m = 1024, w = 14).  When their sum exceeds max_bytes, only every K-th
 * (K = ceil(sqrt(N))) stays on the device and the others are rebuilt, segment by
 * segment, when the left-to-right pass needs them: the same launches on the same
 * inputs, so the Krylov vectors are bit-identical, for at most one extra pass of
 * density-environment work.  max_bytes = 0 (the default) uses the free device
 * memory (plus the blocks this handle has cached) less the step's GEMM
 * intermediates, three times the largest F_j and 16 GiB; max_bytes < 0 leaves the
 * setting unchanged.  *last_segment
 * (optional) receives K of the last Krylov step, 1 when every F_j stayed. */
TDVP_API tdvp_status tdvp_krylov_memory(tdvp_handle* h, double max_bytes, int* last_segment);

/* How tdvp_expand_basis and tdvp_apply_krylov apply 1 - i tau H (Sec. I.B names
 * the density-matrix approach and applying the MPO variationally).
 *  TDVP_KRYLOV_DENSITY_MATRIX (default): right density environments, then one
 *    left-to-right pass of density-matrix eigendecompositions (optimal truncation;
 *    F_j memory, see tdvp_krylov_memory).
 *  TDVP_KRYLOV_ZIPUP: the zip-up algorithm, no density environments.  Right to left
 *    over the left-canonical source, each site contracted with the MPO and the carry
 *    is split by the eigendecomposition of its Gram matrix with the relaxed cutoff
 *    0.1 eps_k and the cap chi_max; then one left-to-right SVD compression with eps_k
 *    and chi_max.  The result is normalised, left-canonical, centre at N-1.
 * Other values give TDVP_ERR_INVALID_ARG. */
typedef enum { TDVP_KRYLOV_DENSITY_MATRIX = 0, TDVP_KRYLOV_ZIPUP = 1 } tdvp_krylov_method;
TDVP_API tdvp_status tdvp_set_krylov_method(tdvp_handle* h, int method);

/* Arithmetic of the Krylov vectors' contractions (Sec. I.B: the Krylov vectors of
 * Eq. 10 need less accuracy than |psi> itself, because they only enrich the basis
 * and the extension keeps |psi> exactly).  precision = -1 (the default) uses the
 * handle's tdvp_options.precision; a tdvp_precision value sets the form of the
 * density environments, the density matrices, the zip-up products and the
 * Krylov vectors' centre moves in the extension.  With a form of about FP32
 * accuracy (BF16X6, TF32X3), the eigendecompositions of the Krylov density
 * matrices also rotate their FP64 Cholesky factors in FP32.  |psi>'s own
 * contractions, the sweep and its factorisations are not affected.  Other values
 * give TDVP_ERR_INVALID_ARG. */
TDVP_API tdvp_status tdvp_set_krylov_precision(tdvp_handle* h, int precision);

/* One Krylov vector in place (Eq. 10 with l = 1, Sec. I.B): the state becomes
 * (1 - i tau H)|psi>, applied by the method tdvp_set_krylov_method selects (the
 * density-matrix approach by default) with cutoff eps_k and cap chi_max,
 * normalised, left-canonical with the centre at site N-1.  (tdvp_expand_basis
 * builds its Krylov vectors with the same routine.) */
TDVP_API tdvp_status tdvp_apply_krylov(tdvp_handle* h);

/* GSE step 3 (Sec. I.C): one symmetric one-site TDVP sweep, left to right then
 * right to left, each with time step dt/2.  kind = TDVP_REAL applies
 * exp(-i H dt); TDVP_IMAG applies exp(-H dt) and renormalises after every local
 * exponential, truncating with eps and chi_max.  Starts by moving the centre to
 * site 0 if needed; ends with the centre at site 0. */
TDVP_API tdvp_status tdvp_sweep(tdvp_handle* h, double dt, tdvp_time kind);

/* One symmetric two-site TDVP step (TDVP2): the conventional integrator that
 * GSE-TDVP1 is compared with (Introduction; Sec. I.C, cost at equal bond
 * dimension; Fig. 1(c)).  Left to right then right to left, each with dt/2.
 * Per bond (i, i+1): Theta = A_i A_{i+1} is evolved forward under the two-site
 * H_eff (the one-site contraction with the merged MPO of sites i and i+1,
 * physical dimension d^2), split by an SVD that keeps s > 1e-10 s_max and
 * truncates with eps and chi_max in real AND imaginary time, and the new
 * one-site centre is evolved backward under the one-site H_eff (omitted at the
 * last bond of each half-sweep).  TDVP_IMAG renormalises after every local
 * exponential.  Contractions use options.precision; SVDs, Lanczos and gauge
 * products stay FP64.  Needs N >= 2 (else TDVP_ERR_SHAPE).  Starts by moving
 * the centre to site 0; ends with the centre at site 0.  No basis extension is
 * involved; tdvp_trunc_stats reports the discarded weight under "eps". */
TDVP_API tdvp_status tdvp_sweep2(tdvp_handle* h, double dt, tdvp_time kind);

/* One-site effective Hamiltonian at `site` (the operator whose exponential the
 * TDVP1 sweep applies, Sec. I.C step 3; cost O(m^3 w d)):
 *   y[a,s,b] = sum L[a,w,a'] W[w,s,s',v] x[a',s',b'] R[b,v,b']
 * with the current environments L_site, R_site (call tdvp_canonicalize(site)
 * first).  x_dev, y_dev: caller-owned DEVICE buffers of m_site * d * m_{site+1}
 * complex128; they may not overlap.  precision: tdvp_precision. */
TDVP_API tdvp_status tdvp_heff_apply(tdvp_handle* h, int site, const void* x_dev, void* y_dev,
                            int precision);

/* Zero-site effective Hamiltonian on bond b (the backward step of TDVP1):
 *   y[a,b'] = sum L[a,w,a'] x[a',c] R[b',w,c]
 * with L = environment of sites < b and R = environment of sites >= b; needs
 * the centre at site b (tdvp_canonicalize(b)).  x_dev, y_dev: DEVICE buffers of
 * m_b * m_b complex128.  precision: tdvp_precision, as the sweep's backward
 * steps use it (the two GEMMs run on the tensor cores when they are large
 * enough: M N K >= 2^21, M >= 64, N >= 32; smaller ones stay FP64). */
TDVP_API tdvp_status tdvp_keff_apply(tdvp_handle* h, int bond, const void* x_dev, void* y_dev,
                            int precision);

/* Local exponential by Lanczos (FP64 vectors, full re-orthogonalisation
 * twice): y = exp(-i delta H_eff) x (REAL) or exp(-delta H_eff) x (IMAG) at
 * `site` with the current environments.  iters (host, may be NULL) receives the
 * Krylov dimension used (summed over sub-steps).  A run that does not reach
 * lanczos_tol within lanczos_max vectors is repeated as 2, 4, ... 64 equal
 * sub-steps of delta; LANCZOS_NOT_CONVERGED when 64 sub-steps do not converge. */
TDVP_API tdvp_status tdvp_evolve_site(tdvp_handle* h, int site, const void* x_dev, void* y_dev,
                             double delta, tdvp_time kind, int precision, int* iters);

/* Observables (host outputs). */
TDVP_API tdvp_status tdvp_energy(tdvp_handle* h, double* e);   /* <C|H_eff C>/<C|C> at the centre */
TDVP_API tdvp_status tdvp_norm(tdvp_handle* h, double* n);     /* |C| at the centre               */
/* <psi|op_site|psi>/<psi|psi>; op: host d*d complex128 row-major <s|op|s'>. */
TDVP_API tdvp_status tdvp_expect_local(tdvp_handle* h, const double* op, int site, double* re_im);
/* <psi|O|psi>/<psi|psi> for an operator given as an MPO (host descriptor in the layout of
 * tdvp_create's: N sites, the handle's d, boundary bond dimensions 1), by a left-to-right
 * FP64 environment contraction in any gauge (Sec. II.B uses two-point functions of the total
 * spin, Eqs. 14-15).  The state and its environments are left as they are.  re_im receives the
 * complex value; TDVP_ERR_SHAPE for an MPO of another length or d. */
TDVP_API tdvp_status tdvp_expect_mpo(tdvp_handle* h, const tdvp_mpo_desc* op, double* re_im);
TDVP_API tdvp_status tdvp_bond_dims(tdvp_handle* h, int* out);  /* N + 1 ints                   */
TDVP_API tdvp_status tdvp_center(tdvp_handle* h, int* site);

/* U(1) sector tables of the bond bases.  A Hamiltonian that conserves a U(1) charge
 * (total S^z of the Heisenberg and OAT models, Secs. II.A-B) keeps a state of
 * definite charge block sparse: A_i[l][s][r] can be nonzero only where
 * q_r = q_l + c_s.  The cost statement of Sec. I.C counts its contractions over
 * these blocks; the library stores tensors densely, orders every new bond index by
 * block, and lets its tensor-core GEMMs skip the all-zero tiles.
 *
 * tdvp_bond_charges reads the charge of every index of every bond (bond 0 to bond
 * N, N + 1 bonds, bond 0 first) off the exact-zero pattern of the current site
 * tensors: bond 0 carries charge 0 and index r of bond i+1 gets q_l + c_s from
 * every nonzero A_i[l][s][r].  phys_charges: d host ints c_s (2 S^z = +1, -1 for
 * spin 1/2).  charges: host buffer of sum_b m_b ints (tdvp_bond_dims gives m_b).
 * Errors: INVALID_ARG (null, |c_s| >= 2^20, N max|c_s| >= 2^30); SHAPE when an index gets two
 * different charges (the state does not conserve the charge) or none. */
TDVP_API tdvp_status tdvp_bond_charges(tdvp_handle* h, const int* phys_charges, int* charges);

/* The sector table of bond `bond` (0..N): the runs of equal charge along the bond
 * index as (charge[k], dim[k], offset[k]), k = 0.. in index order.  *n_sectors
 * receives the number of runs (at most max_sectors triples are written; host
 * buffers, may be NULL when max_sectors = 0); *contiguous is 1 when no charge
 * occurs in two runs (each sector one contiguous index range), else 0.  Errors as
 * tdvp_bond_charges, and INVALID_ARG for a bond out of range. */
TDVP_API tdvp_status tdvp_bond_sectors(tdvp_handle* h, const int* phys_charges, int bond, int max_sectors,
                                       int* charge, int* dim, int* offset, int* n_sectors, int* contiguous);
/* out[0..3]: discarded weight sums of the last call for eps_k, eps_m, eps, and the
 * number of basis states added by the last extension; out[4]: total Lanczos
 * iterations of the last sweep; out[5]: Lanczos calls of the last sweep;
 * out[6..8]: process-wide SVD calls, calls that split into independent blocks
 * (conserved quantum numbers), and blocks solved; out[9..10]: process-wide
 * Jacobi sweeps summed over all blocks, and the most sweeps one block took;
 * out[11..12]: blocks too large for the shared-memory batched path, and the
 * widest block (smaller dimension) seen. */
TDVP_API tdvp_status tdvp_trunc_stats(tdvp_handle* h, double* out13);

/* Copies the state to host buffers the caller allocated from tdvp_bond_dims
 * (site i: 2 * m_i * d * m_{i+1} doubles). */
TDVP_API tdvp_status tdvp_get_mps(tdvp_handle* h, double* const* sites_out);

/* ---------------------------------------------------------------------------
 * Batches of independent chains on one GPU (many chains of uneven length and
 * bond dimension, e.g. disorder realisations).  One engine per chain, each on
 * its own CUDA stream; a batch call runs the per-chain call for every chain on
 * n_threads host workers (<= 0: the number of host cores), longest chains
 * first, so the chains' kernels overlap on the device.  Arrays of n descriptors;
 * opts may be NULL (defaults for all) or n options.  Per-chain status codes go
 * to status[n] when non-null; the return value is the first non-OK status
 * (tdvp_batch_last_error names the chain).  A failing chain does not stop or
 * change the others.  tdvp_batch_handle lends the handle of chain i for any
 * per-chain call (observables, tdvp_get_mps); the batch keeps ownership. */
typedef struct tdvp_batch tdvp_batch;
TDVP_API tdvp_status tdvp_batch_create(int n, const tdvp_mps_desc* mps, const tdvp_mpo_desc* mpo,
                                       const tdvp_options* opts, int n_threads, tdvp_batch** out);
TDVP_API tdvp_status tdvp_batch_destroy(tdvp_batch* b);
TDVP_API tdvp_status tdvp_batch_size(const tdvp_batch* b, int* n);
TDVP_API tdvp_status tdvp_batch_handle(tdvp_batch* b, int i, tdvp_handle** h);
TDVP_API tdvp_status tdvp_batch_expand_basis(tdvp_batch* b, int krylov_order_k, const double* weights, int* status);
TDVP_API tdvp_status tdvp_batch_sweep(tdvp_batch* b, double dt, tdvp_time kind, int* status);
/* expand_basis then sweep on every chain: one GSE-TDVP1 step each */
TDVP_API tdvp_status tdvp_batch_step(tdvp_batch* b, int krylov_order_k, const double* weights, double dt,
                                     tdvp_time kind, int* status);
TDVP_API tdvp_status tdvp_batch_energy(tdvp_batch* b, double* out_n);
TDVP_API tdvp_status tdvp_batch_norm(tdvp_batch* b, double* out_n);
TDVP_API const char* tdvp_batch_last_error(const tdvp_batch* b);

/* ---------------------------------------------------------------------------
 * Checkpoints.  A file holds one MPS: magic "GSETDVP1", int32 {version 1, N, d,
 * 0}, int32 bond_dims[N + 1], the site tensors as complex128 [m_i][d][m_{i+1}]
 * row-major, and a 64-bit FNV-1a hash of all preceding bytes (little-endian).
 * Writers go through "<path>.tmp" and rename it over <path>.  Readers reject a
 * wrong magic or version, inconsistent dimensions, a truncated file or a hash
 * mismatch with TDVP_ERR_INVALID_ARG / TDVP_ERR_SHAPE; tdvp_checkpoint_last_error()
 * (per thread) gives the reason.  The checkpoint_* calls are host-only. */
/* Saves the current state of h (its gauge as it stands). */
TDVP_API tdvp_status tdvp_save(tdvp_handle* h, const char* path);
/* Creates a handle from a saved state, as tdvp_create does from host arrays. */
TDVP_API tdvp_status tdvp_load(const char* path, const tdvp_mpo_desc* mpo, const tdvp_options* opt, void* stream,
                               tdvp_handle** out);
TDVP_API tdvp_status tdvp_checkpoint_write(const char* path, const tdvp_mps_desc* mps);
/* N and d; and bond_dims (N + 1 ints) when bond_dims is non-null and capacity >= N + 1
 * (else TDVP_ERR_SHAPE, nothing written). */
TDVP_API tdvp_status tdvp_checkpoint_read_header(const char* path, int* n_sites, int* d, int* bond_dims,
                                                 int capacity);
/* Site tensors into caller buffers of the shapes the caller states (n_sites, d, bond_dims:
 * site i holds 2 m_i d m_{i+1} doubles).  The file is read once, checked against the size its
 * header implies and against its hash into memory of the library's own; the caller's buffers
 * are written only after that, and only when the file's N, d and bond dimensions equal the
 * stated ones (else TDVP_ERR_SHAPE).  tdvp_load reads the same way. */
TDVP_API tdvp_status tdvp_checkpoint_read(const char* path, int n_sites, int d, const int* bond_dims,
                                          double* const* sites_out);
TDVP_API const char* tdvp_checkpoint_last_error(void);

/* ---------------------------------------------------------------------------
 * Timing of the H_eff applies inside a handle (CUDA events on the handle's
 * stream).  tdvp_profile(h, 1) starts recording, 0 stops.  tdvp_profile_read
 * writes out3 = {applies, total milliseconds, total algorithmic flops} since
 * the last read (8 real flops per complex multiply-add,
 * 8 [m_l d m_r (m_l w_l + m_r w_r) + m_l m_r nnz(W)] per apply) and resets. */
TDVP_API tdvp_status tdvp_profile(tdvp_handle* h, int enable);
TDVP_API tdvp_status tdvp_profile_read(tdvp_handle* h, double* out3);

/* Per-phase timing (CUDA events on the handle's stream).  tdvp_trace(h, 1)
 * starts recording; tdvp_trace_read writes the milliseconds spent since the
 * last read into out[0..n) and resets.  Phases: 0 local exponentials of the
 * sweep (H_eff Lanczos), 1 backward bond exponentials (K_eff Lanczos), 2 gauge
 * moves of the sweep (block QR in real time, truncated SVD in imaginary time),
 * 3 environment updates, 4 Krylov vectors (step 1), 5 basis extension (step 2),
 * 6 gauge moves of tdvp_canonicalize, 7 right density environments of the
 * Krylov vectors, 8 their eigendecompositions, 9 SVDs of the extension; inside
 * every blocked SVD or eigendecomposition of 2, 6, 8, 9: 10 block detection
 * (nonzero mask, host union-find, gather), 11 pivoted Cholesky of density
 * matrices, 12 Jacobi sweeps, 13 selection and scatter of the kept vectors;
 * 14 every block QR / LQ (gauge moves that cut nothing, inside 2 and 6).
 * Intervals nest (3 runs inside 0..2, 7-8 inside 4, 9 inside 5, 10-14 inside
 * the factorisations), so the entries do not add up.  n may be smaller or
 * larger than 15; missing phases are left out, entries past the last phase
 * are zero. */
TDVP_API tdvp_status tdvp_trace(tdvp_handle* h, int enable);
TDVP_API tdvp_status tdvp_trace_read(tdvp_handle* h, double* out, int n);

/* Number of CUDA kernels this library has launched in this process, over all
 * handles and handle-free calls (a relaxed atomic counter bumped at every
 * launch site).  Differences of two reads count the launches in between.
 * Returns TDVP_ERR_INVALID_ARG for a null pointer. */
TDVP_API tdvp_status tdvp_launch_count(long long* out);

/* Block sparsity the BF16 tensor-core GEMMs exploit (Sec. I.C cost; conserved S^z charges
 * make most blocks of L, R, W and the site tensors exactly zero).  Each GEMM output tile of
 * 128 x 128 walks the K dimension in chunks of 128 real entries; the slicing kernels mark every
 * (128-row operand tile, chunk) that holds a nonzero entry, and a chunk whose A tile or B tile
 * is all zero adds an exact zero and is not multiplied.  The factorisations order the kept
 * vectors of every new bond by block, so each charge sector is one contiguous index range.
 * out2[0]: (output tile, chunk) pairs visited by the BF16 GEMMs on the current device since the
 * library loaded; out2[1]: the pairs multiplied.  Differences of two reads cover the calls in
 * between.  Synchronises the device; TDVP_ERR_INVALID_ARG for a null pointer. */
TDVP_API tdvp_status tdvp_gemm_chunk_stats(long long* out2);

/* ---------------------------------------------------------------------------
 * Handle-free contractions of one site on caller buffers (kernel-level entry
 * points; the same code the handle uses).  Device buffers are caller-owned
 * complex128 arrays; the MPO site W is a HOST array W[w_l][d][d][w_r].
 * Scratch comes from a library-wide pool.  Calls are serialised internally.
 * On error tdvp_contract_last_error() describes the failure. */
typedef struct { int ml, mr, wl, wr, d; } tdvp_site_dims;

/* y = H_eff x:  y[a,s,b] = sum L[a,w,a'] W[w,s,s',v] x[a',s',b'] R[b,v,b']
 * L: ml*wl*ml, R: mr*wr*mr, x, y: ml*d*mr (Sec. I.C step 3). */
TDVP_API tdvp_status tdvp_heff_contract(const tdvp_site_dims* dims, const void* L_dev, const double* W_host,
                                        const void* R_dev, const void* x_dev, void* y_dev, int precision,
                                        void* stream);
/* As tdvp_heff_contract, for repeated applies with the same environments (a
 * Lanczos run).  env_tag >= 0 names the content of (L, R, W, dims): when the
 * previous tensor-core call used the same tag, the tensor-core operand forms of
 * L and R built then are reused instead of being rebuilt from L_dev and R_dev.
 * The caller must give a new tag whenever L, R, W or dims change; -1 never
 * reuses (the behaviour of tdvp_heff_contract).  FP64 ignores the tag.
 * TDVP_ERR_INVALID_ARG for env_tag < -1. */
TDVP_API tdvp_status tdvp_heff_contract_cached(const tdvp_site_dims* dims, const void* L_dev,
                                               const double* W_host, const void* R_dev, const void* x_dev,
                                               void* y_dev, int precision, long long env_tag, void* stream);
/* y[a,c] = sum L[a,w,a'] x[a',b'] R[c,w,b']; L: ml*w*ml, R: mr*w*mr, x, y: ml*mr. */
TDVP_API tdvp_status tdvp_keff_contract(int ml, int mr, int w, const void* L_dev, const void* R_dev,
                                        const void* x_dev, void* y_dev, void* stream);
/* side 0: out[b,v,b'] = sum conj(A[a,s,b]) E[a,w,a'] W[w,s,s',v] A[a',s',b']   (E: ml*wl*ml, out: mr*wr*mr)
 * side 1: out[a,w,a'] = sum conj(A[a,s,b]) W[w,s,s',v] E[b,v,b'] A[a',s',b']   (E: mr*wr*mr, out: ml*wl*ml) */
TDVP_API tdvp_status tdvp_env_contract(const tdvp_site_dims* dims, int side, const void* E_dev,
                                       const double* W_host, const void* A_dev, void* out_dev, void* stream);
/* y = exp(-i delta H_eff) x (REAL) or exp(-delta H_eff) x (IMAG) by Lanczos with
 * full re-orthogonalisation twice, error target tol, at most nmax (<= 63) steps. */
TDVP_API tdvp_status tdvp_expm_contract(const tdvp_site_dims* dims, const void* L_dev, const double* W_host,
                                        const void* R_dev, const void* x_dev, void* y_dev, double delta,
                                        tdvp_time kind, int precision, double tol, int nmax, int* iters,
                                        void* stream);
/* The handle-free calls above share one library-wide context (device pool, operand
 * caches, Lanczos work space), set up on the device current at the first of them;
 * a later call with another device current returns TDVP_ERR_INVALID_ARG. */
TDVP_API const char* tdvp_contract_last_error(void);

/* y = H_eff x by the same FP64 contraction as tdvp_heff_contract(...,
 * TDVP_PREC_FP64, ...) (the summation order may differ: the results agree to
 * about 1e-12 relative), but without allocating device memory.  The paper has no counterpart: this entry
 * exists for callers that cannot call cudaMalloc (a host framework that owns
 * every device allocation, or a loop that must never block on the allocator).
 * Its intermediates live in a fixed 32 MiB file-scope device array that every
 * GPU loading the library keeps until the process exits; the limits are
 * (m_l w_l d m_r + m_l d w_r m_r) * 16 bytes <= 31 MiB and w_l d d w_r <= 16384,
 * and larger sizes return TDVP_ERR_INVALID_ARG.  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress) with the device
 * current, so make the first call on each device outside any stream capture.
 * All calls share the one array and keep its last contents (nothing in it
 * needs to start at zero); calls serialise on the host, but calls that overlap
 * on the GPU (different streams, or a caller that does not wait) race.  The
 * call synchronises `stream` before returning.  err (may be NULL) receives up
 * to err_len bytes of message on failure. */
TDVP_API tdvp_status tdvp_heff_contract_noalloc(const tdvp_site_dims* dims, const void* L_dev,
                                                const double* W_host, const void* R_dev, const void* x_dev,
                                                void* y_dev, void* stream, char* err, int err_len);

#ifdef __cplusplus
}
#endif
#endif /* GSE_TDVP_H */
