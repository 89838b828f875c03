// Device-resident GSE-TDVP1 engine: state, environments and the algorithm
// steps of Sec. I (basis extension, Krylov vectors, TDVP1 sweep).
#pragma once
#include <functional>

#include "contract.cuh"

// Number of leading (descending) weights kept under the truncation rule:
// relative discarded weight <= eps * total, values <= floor never kept, a cut
// never splits a cluster of values within relative 1e-8 (grow to the cluster's
// end; if that breaks the cap, shrink to its start).
int keep_count(const std::vector<double>& w_desc, double total, double eps, int cap, double floor_);

struct MpsDev {
  int N = 0, d = 2;
  std::vector<int> m;        // N + 1 bond dims
  std::vector<DArr> A;       // A[i]: m[i] x d x m[i+1]
};

// MPO of 1 - i tau H on the device (sparse lists for the site stage and the
// products Om = W conj(W) for the density environments).
struct KrylovOp {
  std::vector<WSparse> Wsp;
  std::vector<int*> om_off, om_idx;
  std::vector<cplx*> om_val;
  void release();
};

struct Engine {
  // declared first so it is destroyed last: every DArr below returns its block here
  DevicePool pool;
  // problem
  int N = 0, d = 2;
  std::vector<int> w;                    // MPO bond dims
  std::vector<std::vector<cplx>> W_host; // MPO of H (host copy)
  std::vector<WSparse> Wsp;              // MPO of H (device sparse)
  std::vector<WSparse> Wsp2;             // merged pair MPO of sites (i, i+1), physical dim d^2 (TDVP2)
  MpsDev psi;
  int center = 0;
  tdvp_options opt{};
  cudaStream_t st = nullptr;
  Blas1 blas;
  int sm_count = 148;
  // environments: L[i] = sites < i (m_i x w_i x m_i); R[i] = sites > i (m_{i+1} x w_{i+1} x m_{i+1})
  std::vector<DArr> L, R;
  std::vector<char> Lok, Rok;
  // contraction scratch and Lanczos work space
  Scratch scr;
  LanczosWork lw;
  long long env_epoch = 0;  // bumped whenever an environment is rebuilt or dropped
  int env_prec = TDVP_PREC_FP64;  // arithmetic of environment updates (the sweep's precision while it runs)
  // device bytes the Krylov step may hold in right density environments (0: half the free memory)
  double krylov_mem_budget = 0.0;
  int krylov_env_segment = 1;  // last Krylov step: 1 = all resident, else the checkpoint spacing
  int krylov_method = 0;       // 0: density-matrix application, 1: zip-up
  int krylov_prec = -1;        // arithmetic of the Krylov vectors' contractions (-1: opt.precision)
  int kprec() const { return krylov_prec < 0 ? opt.precision : krylov_prec; }
  // optional timing of the H_eff applies (CUDA events on the engine stream)
  bool profile = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pairs;
  double prof_flops = 0.0;
  long long prof_count = 0;
  Tracer tracer;
  // statistics of the last calls
  double disc_k = 0, disc_m = 0, disc_eps = 0;
  int added_states = 0;
  long long lanczos_iters = 0, lanczos_calls = 0;

  void init(const tdvp_mps_desc* mps, const tdvp_mpo_desc* mpo, const tdvp_options* o, cudaStream_t s);
  void release();

  // environments
  void ensure_L(int i);
  void ensure_R(int i);
  void invalidate_from_site(int i);  // A[i] changed
  // contractions (FP64 unless precision says otherwise)
  void heff(int site, const cplx* x, cplx* y, int precision);
  void apply_op(const SiteOp& op, const cplx* x, cplx* y, int precision);  // H_eff of op (timed when profiling)
  SiteOp site_op(int site);
  SiteOp pair_op(int i);  // two-site H_eff of (i, i+1): L[i], R[i+1], merged MPO, physical dim d^2
  void build_pair_mpo();
  void env_left(int i);   // L[i+1] from L[i], A[i]
  void env_right(int i);  // R[i-1] from R[i], A[i]
  // gauge moves
  void move_right(int i, double eps, int cap, bool imag_trunc);
  void move_left(int i, double eps, int cap, bool imag_trunc);
  void canonicalize(int c);
  // Lanczos exponential: out = exp(-i delta Op) x (kind 0) or exp(-delta Op) x (kind 1).  slot
  // (0..3, or -1 for none) names the operator kind whose previous Krylov dimension lets a small
  // run launch several iterations per host check (site, bond, two-site, backward site)
  int lanczos(const std::function<void(const cplx*, cplx*)>& op, const cplx* x, cplx* out,
              long long n, double delta, int kind, int slot = -1);
  int lanczos_hint[4] = {0, 0, 0, 0};
  // algorithm steps
  void sweep(double dt, int kind);
  void sweep2(double dt, int kind);  // two-site TDVP (the conventional integrator GSE-TDVP1 is compared with)
  void expand_basis(int k, const double* weights);
  void build_krylov_op(KrylovOp& kop);
  void krylov_apply(const KrylovOp& kop, const MpsDev& src, MpsDev& out);
  // the zip-up application of the same operator (no right density environments)
  void krylov_zipup(const KrylovOp& kop, const MpsDev& src, MpsDev& out);
  void apply_krylov();  // state <- normalised, compressed (1 - i tau H) state
  // observables
  double energy();
  double norm();
  cplx expect_local(const double* op, int site);
  cplx expect_mpo(const tdvp_mpo_desc* op);  // <psi|O|psi>/<psi|psi>, O an MPO of N sites
  void sync() { TDVP_CUDA(cudaStreamSynchronize(st)); }
};

// U(1) charges of every bond index (N + 1 bonds, bond 0 first), read off the exact-zero pattern
// of the current site tensors from charge 0 at the left end; phys_host holds the d local
// charges.  Throws TDVP_ERR_SHAPE when an index gets two charges or none.
std::vector<std::vector<int>> bond_charges(Engine& e, const int* phys_host);
// Runs of equal charge along one bond as (charge, dim, offset) triples; *contiguous is false
// when a charge occurs in more than one run.
std::vector<int> sector_runs(const std::vector<int>& q, bool* contiguous);

// The opaque handle of the C ABI: one engine and the text of its last error.
struct tdvp_handle {
  Engine eng;
  std::string err;
};
