// C-ABI entry points of libgsetdvp (declared in include/gse_tdvp.h).  Every
// entry point converts internal errors to a tdvp_status; no exception crosses
// the boundary.  On error the handle's message is kept for tdvp_last_error().
#include <algorithm>
#include <cstring>
#include <mutex>

#include "engine.cuh"


namespace {
template <class F>
tdvp_status guarded(tdvp_handle* h, F&& f) {
  if (!h) return TDVP_ERR_INVALID_ARG;
  // the factorisations of this call record their phases on the handle's tracer
  struct Bind {
    Tracer* prev;
    explicit Bind(Tracer* t) : prev(t_tracer) { t_tracer = t; }
    ~Bind() { t_tracer = prev; }
  } bind(h->eng.tracer.on ? &h->eng.tracer : nullptr);
  try {
    f();
    h->err.clear();
    return TDVP_OK;
  } catch (const TdvpError& e) {
    h->err = e.what();
    return e.status;
  } catch (const std::bad_alloc&) {
    h->err = "host allocation failed";
    return TDVP_ERR_OUT_OF_MEMORY;
  } catch (const std::exception& e) {
    h->err = e.what();
    return TDVP_ERR_CUDA;
  }
}

void check_options(const tdvp_options& o) {
  tdvp_require(std::isfinite(o.tau_re) && std::isfinite(o.tau_im), TDVP_ERR_INVALID_ARG, "tau not finite");
  tdvp_require(o.eps_k >= 0 && o.eps_m >= 0 && o.eps >= 0, TDVP_ERR_INVALID_ARG, "cutoffs must be >= 0");
  tdvp_require(o.chi_max >= 1, TDVP_ERR_INVALID_ARG, "chi_max must be >= 1");
  tdvp_require(o.lanczos_tol > 0 && o.lanczos_max >= 1 && o.lanczos_max <= 63, TDVP_ERR_INVALID_ARG,
               "lanczos_tol > 0 and 1 <= lanczos_max <= 63 required");
  tdvp_require(o.precision >= TDVP_PREC_FP64 && o.precision <= TDVP_PREC_BF16X6, TDVP_ERR_INVALID_ARG,
               "unknown precision");
}
}  // namespace

extern "C" {

tdvp_status tdvp_default_options(tdvp_options* o) {
  if (!o) return TDVP_ERR_INVALID_ARG;
  o->tau_re = 0.1;
  o->tau_im = 0.0;
  o->eps_k = 1e-8;
  o->eps_m = 1e-8;
  o->eps = 0.0;
  o->chi_max = 1024;
  o->lanczos_tol = 1e-12;
  o->lanczos_max = 40;
  o->precision = TDVP_PREC_FP64;
  return TDVP_OK;
}

const char* tdvp_status_string(tdvp_status s) {
  switch (s) {
    case TDVP_OK: return "ok";
    case TDVP_ERR_INVALID_ARG: return "invalid argument";
    case TDVP_ERR_SHAPE: return "shape mismatch";
    case TDVP_ERR_OUT_OF_MEMORY: return "out of memory";
    case TDVP_ERR_LANCZOS_NOT_CONVERGED: return "Lanczos not converged";
    case TDVP_ERR_NONFINITE: return "non-finite value";
    case TDVP_ERR_TIMEOUT: return "device wait timed out";
    case TDVP_ERR_CUDA: return "CUDA error";
    case TDVP_ERR_SVD_NOT_CONVERGED: return "SVD not converged";
  }
  return "unknown status";
}

tdvp_status tdvp_create(const tdvp_mps_desc* mps, const tdvp_mpo_desc* mpo, const tdvp_options* opt,
                        void* stream, tdvp_handle** out) {
  if (!out || !mps || !mpo) return TDVP_ERR_INVALID_ARG;
  *out = nullptr;
  tdvp_handle* h = nullptr;
  try {
    h = new tdvp_handle();
  } catch (...) {
    return TDVP_ERR_OUT_OF_MEMORY;
  }
  tdvp_status s = guarded(h, [&] {
    if (opt) check_options(*opt);
    h->eng.init(mps, mpo, opt, static_cast<cudaStream_t>(stream));
  });
  if (s != TDVP_OK) {
    fprintf(stderr, "tdvp_create: %s\n", h->err.c_str());
    h->eng.release();
    delete h;
    return s;
  }
  *out = h;
  return TDVP_OK;
}

tdvp_status tdvp_destroy(tdvp_handle* h) {
  if (!h) return TDVP_ERR_INVALID_ARG;
  cudaStreamSynchronize(h->eng.st);
  h->eng.release();
  delete h;
  return TDVP_OK;
}

tdvp_status tdvp_set_options(tdvp_handle* h, const tdvp_options* opt) {
  return guarded(h, [&] {
    tdvp_require(opt != nullptr, TDVP_ERR_INVALID_ARG, "null options");
    check_options(*opt);
    h->eng.opt = *opt;
  });
}

const char* tdvp_last_error(const tdvp_handle* h) { return h ? h->err.c_str() : "null handle"; }

tdvp_status tdvp_canonicalize(tdvp_handle* h, int site) {
  return guarded(h, [&] {
    h->eng.canonicalize(site);
    h->eng.sync();
  });
}

tdvp_status tdvp_expand_basis(tdvp_handle* h, int k, const double* weights) {
  return guarded(h, [&] { h->eng.expand_basis(k, weights); });
}

tdvp_status tdvp_apply_krylov(tdvp_handle* h) {
  return guarded(h, [&] { h->eng.apply_krylov(); });
}

tdvp_status tdvp_sweep(tdvp_handle* h, double dt, tdvp_time kind) {
  return guarded(h, [&] {
    tdvp_require(std::isfinite(dt), TDVP_ERR_INVALID_ARG, "dt not finite");
    tdvp_require(kind == TDVP_REAL || kind == TDVP_IMAG, TDVP_ERR_INVALID_ARG, "bad time kind");
    h->eng.sweep(dt, kind);
  });
}

tdvp_status tdvp_krylov_memory(tdvp_handle* h, double max_bytes, int* last_segment) {
  return guarded(h, [&] {
    tdvp_require(std::isfinite(max_bytes), TDVP_ERR_INVALID_ARG, "max_bytes not finite");
    if (max_bytes >= 0.0) h->eng.krylov_mem_budget = max_bytes;
    if (last_segment) *last_segment = h->eng.krylov_env_segment;
  });
}

tdvp_status tdvp_set_krylov_method(tdvp_handle* h, int method) {
  return guarded(h, [&] {
    tdvp_require(method == TDVP_KRYLOV_DENSITY_MATRIX || method == TDVP_KRYLOV_ZIPUP, TDVP_ERR_INVALID_ARG,
                 "unknown Krylov method");
    h->eng.krylov_method = method;
  });
}

tdvp_status tdvp_set_krylov_precision(tdvp_handle* h, int precision) {
  return guarded(h, [&] {
    tdvp_require(precision == -1 || (precision >= TDVP_PREC_FP64 && precision <= TDVP_PREC_BF16X6),
                 TDVP_ERR_INVALID_ARG, "unknown precision");
    h->eng.krylov_prec = precision;
  });
}

tdvp_status tdvp_sweep2(tdvp_handle* h, double dt, tdvp_time kind) {
  return guarded(h, [&] {
    tdvp_require(std::isfinite(dt), TDVP_ERR_INVALID_ARG, "dt not finite");
    tdvp_require(kind == TDVP_REAL || kind == TDVP_IMAG, TDVP_ERR_INVALID_ARG, "bad time kind");
    h->eng.sweep2(dt, kind);
  });
}

tdvp_status tdvp_heff_apply(tdvp_handle* h, int site, const void* x, void* y, int precision) {
  return guarded(h, [&] {
    Engine& e = h->eng;
    tdvp_require(x && y && x != y, TDVP_ERR_INVALID_ARG, "x, y must be distinct device buffers");
    tdvp_require(site >= 0 && site < e.N, TDVP_ERR_INVALID_ARG, "site out of range");
    tdvp_require(precision >= TDVP_PREC_FP64 && precision <= TDVP_PREC_BF16X6, TDVP_ERR_INVALID_ARG,
                 "unknown precision");
    e.ensure_L(site);
    e.ensure_R(site);
    e.heff(site, static_cast<const cplx*>(x), static_cast<cplx*>(y), precision);
    e.sync();
    tc_check(e.st, e.scr);
  });
}

tdvp_status tdvp_keff_apply(tdvp_handle* h, int bond, const void* x, void* y, int precision) {
  return guarded(h, [&] {
    Engine& e = h->eng;
    tdvp_require(x && y && x != y, TDVP_ERR_INVALID_ARG, "x, y must be distinct device buffers");
    tdvp_require(bond >= 1 && bond < e.N, TDVP_ERR_INVALID_ARG, "bond out of range");
    tdvp_require(precision >= TDVP_PREC_FP64 && precision <= TDVP_PREC_BF16X6, TDVP_ERR_INVALID_ARG,
                 "unknown precision");
    e.ensure_L(bond);
    e.ensure_R(bond - 1);
    const int mb = e.psi.m[bond];
    keff_fp64(e.st, e.scr, e.L[bond].data(), mb, e.R[bond - 1].data(), mb, e.w[bond], static_cast<const cplx*>(x),
              static_cast<cplx*>(y), precision);
    e.sync();
  });
}

tdvp_status tdvp_evolve_site(tdvp_handle* h, int site, const void* x, void* y, double delta, tdvp_time kind,
                             int precision, int* iters) {
  return guarded(h, [&] {
    Engine& e = h->eng;
    tdvp_require(x && y && x != y, TDVP_ERR_INVALID_ARG, "x, y must be distinct device buffers");
    tdvp_require(site >= 0 && site < e.N, TDVP_ERR_INVALID_ARG, "site out of range");
    tdvp_require(kind == TDVP_REAL || kind == TDVP_IMAG, TDVP_ERR_INVALID_ARG, "bad time kind");
    tdvp_require(std::isfinite(delta), TDVP_ERR_INVALID_ARG, "delta not finite");
    e.ensure_L(site);
    e.ensure_R(site);
    const long long n = (long long)e.psi.m[site] * e.d * e.psi.m[site + 1];
    const int it = e.lanczos([&](const cplx* a, cplx* b) { e.heff(site, a, b, precision); },
                             static_cast<const cplx*>(x), static_cast<cplx*>(y), n, delta, kind);
    e.sync();
    if (iters) *iters = it;
  });
}

tdvp_status tdvp_energy(tdvp_handle* h, double* out) {
  return guarded(h, [&] {
    tdvp_require(out != nullptr, TDVP_ERR_INVALID_ARG, "null output");
    *out = h->eng.energy();
  });
}

tdvp_status tdvp_norm(tdvp_handle* h, double* out) {
  return guarded(h, [&] {
    tdvp_require(out != nullptr, TDVP_ERR_INVALID_ARG, "null output");
    *out = h->eng.norm();
  });
}

tdvp_status tdvp_expect_local(tdvp_handle* h, const double* op, int site, double* re_im) {
  return guarded(h, [&] {
    tdvp_require(op && re_im, TDVP_ERR_INVALID_ARG, "null pointer");
    cplx v = h->eng.expect_local(op, site);
    re_im[0] = v.x;
    re_im[1] = v.y;
  });
}

tdvp_status tdvp_expect_mpo(tdvp_handle* h, const tdvp_mpo_desc* op, double* re_im) {
  return guarded(h, [&] {
    tdvp_require(op && re_im && op->bond_dims && op->sites, TDVP_ERR_INVALID_ARG, "null pointer");
    cplx v = h->eng.expect_mpo(op);
    re_im[0] = v.x;
    re_im[1] = v.y;
  });
}

tdvp_status tdvp_bond_dims(tdvp_handle* h, int* out) {
  return guarded(h, [&] {
    tdvp_require(out != nullptr, TDVP_ERR_INVALID_ARG, "null output");
    for (int i = 0; i <= h->eng.N; ++i) out[i] = h->eng.psi.m[i];
  });
}

tdvp_status tdvp_bond_charges(tdvp_handle* h, const int* phys_charges, int* charges) {
  return guarded(h, [&] {
    tdvp_require(phys_charges != nullptr && charges != nullptr, TDVP_ERR_INVALID_ARG, "null argument");
    const auto q = bond_charges(h->eng, phys_charges);
    for (const auto& b : q) charges = std::copy(b.begin(), b.end(), charges);
  });
}

tdvp_status tdvp_bond_sectors(tdvp_handle* h, const int* phys_charges, int bond, int max_sectors, int* charge,
                              int* dim, int* offset, int* n_sectors, int* contiguous) {
  return guarded(h, [&] {
    tdvp_require(phys_charges != nullptr && n_sectors != nullptr && contiguous != nullptr, TDVP_ERR_INVALID_ARG,
                 "null argument");
    tdvp_require(bond >= 0 && bond <= h->eng.N, TDVP_ERR_INVALID_ARG, "bond out of range");
    tdvp_require(max_sectors >= 0 && (max_sectors == 0 || (charge && dim && offset)), TDVP_ERR_INVALID_ARG,
                 "null table with max_sectors > 0");
    const auto q = bond_charges(h->eng, phys_charges);
    bool cont = true;
    const std::vector<int> t = sector_runs(q[bond], &cont);
    const int n = (int)t.size() / 3;
    for (int k = 0; k < std::min(n, max_sectors); ++k) {
      charge[k] = t[3 * k];
      dim[k] = t[3 * k + 1];
      offset[k] = t[3 * k + 2];
    }
    *n_sectors = n;
    *contiguous = cont ? 1 : 0;
  });
}

tdvp_status tdvp_center(tdvp_handle* h, int* site) {
  return guarded(h, [&] {
    tdvp_require(site != nullptr, TDVP_ERR_INVALID_ARG, "null output");
    *site = h->eng.center;
  });
}

tdvp_status tdvp_trunc_stats(tdvp_handle* h, double* out) {
  return guarded(h, [&] {
    tdvp_require(out != nullptr, TDVP_ERR_INVALID_ARG, "null output");
    Engine& e = h->eng;
    out[0] = e.disc_k;
    out[1] = e.disc_m;
    out[2] = e.disc_eps;
    out[3] = e.added_states;
    out[4] = (double)e.lanczos_iters;
    out[5] = (double)e.lanczos_calls;
    out[6] = (double)g_svd_counters.calls;
    out[7] = (double)g_svd_counters.blocked;
    out[8] = (double)g_svd_counters.blocks;
    out[9] = (double)g_svd_counters.sweeps;
    out[10] = (double)g_svd_counters.max_sweeps;
    out[11] = (double)g_svd_counters.large_blocks;
    out[12] = (double)g_svd_counters.max_q;
  });
}

tdvp_status tdvp_get_mps(tdvp_handle* h, double* const* sites_out) {
  return guarded(h, [&] {
    tdvp_require(sites_out != nullptr, TDVP_ERR_INVALID_ARG, "null output");
    Engine& e = h->eng;
    for (int i = 0; i < e.N; ++i) {
      tdvp_require(sites_out[i] != nullptr, TDVP_ERR_INVALID_ARG, "null site buffer");
      const size_t n = (size_t)e.psi.m[i] * e.d * e.psi.m[i + 1];
      TDVP_CUDA(cudaMemcpyAsync(sites_out[i], e.psi.A[i].data(), n * sizeof(cplx), cudaMemcpyDeviceToHost, e.st));
    }
    e.sync();
  });
}

tdvp_status tdvp_profile(tdvp_handle* h, int enable) {
  return guarded(h, [&] { h->eng.profile = enable != 0; });
}

tdvp_status tdvp_profile_read(tdvp_handle* h, double* out) {
  return guarded(h, [&] {
    tdvp_require(out != nullptr, TDVP_ERR_INVALID_ARG, "null output");
    Engine& e = h->eng;
    e.sync();
    double ms = 0.0;
    for (auto& p : e.ev_pairs) {
      float t = 0.f;
      TDVP_CUDA(cudaEventElapsedTime(&t, p.first, p.second));
      ms += t;
      e.ev_pool.push_back(p.first);
      e.ev_pool.push_back(p.second);
    }
    e.ev_pairs.clear();
    out[0] = (double)e.prof_count;
    out[1] = ms;
    out[2] = e.prof_flops;
    e.prof_count = 0;
    e.prof_flops = 0.0;
  });
}

tdvp_status tdvp_trace(tdvp_handle* h, int enable) {
  return guarded(h, [&] { h->eng.tracer.on = enable != 0; });
}

tdvp_status tdvp_trace_read(tdvp_handle* h, double* out, int n) {
  return guarded(h, [&] {
    tdvp_require(out != nullptr && n >= 0, TDVP_ERR_INVALID_ARG, "null output");
    h->eng.sync();
    h->eng.tracer.read(out, n);
  });
}

tdvp_status tdvp_launch_count(long long* out) {
  if (!out) return TDVP_ERR_INVALID_ARG;
  *out = g_kernel_launches.load(std::memory_order_relaxed);
  return TDVP_OK;
}

tdvp_status tdvp_gemm_chunk_stats(long long* out2) {
  if (!out2) return TDVP_ERR_INVALID_ARG;
  try {
    gemm_chunk_pairs(out2);
    return TDVP_OK;
  } catch (const TdvpError& e) {
    return e.status;
  } catch (...) {
    return TDVP_ERR_CUDA;
  }
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Handle-free contractions: one library-wide context (never destroyed, so no
// CUDA call runs from a static destructor after the runtime has shut down).
namespace {
struct RawCtx {
  std::mutex mu;
  DevicePool pool;
  Scratch scr;
  Blas1 blas;
  LanczosWork lw;
  bool ready = false;
  int device = -1;  // the device the pool, scratch and work space were set up on
  std::string err;
  long long key = 0;
};
RawCtx& raw() {
  static RawCtx* c = new RawCtx();
  return *c;
}

template <class F>
tdvp_status raw_guarded(F&& f) {
  RawCtx& c = raw();
  std::lock_guard<std::mutex> lk(c.mu);
  try {
    int dev = 0;
    TDVP_CUDA(cudaGetDevice(&dev));
    if (!c.ready) {
      int sms = 148;
      TDVP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
      c.scr.pool = &c.pool;
      c.blas.init(&c.pool, sms);
      c.lw.init(&c.pool);
      c.device = dev;
      c.ready = true;
    }
    // the context's device memory belongs to the device of the first call: another
    // current device would hand that device's kernels foreign pointers
    tdvp_require(dev == c.device, TDVP_ERR_INVALID_ARG,
                 "handle-free contractions run on the device current at their first call (" +
                     std::to_string(c.device) + "), not on device " + std::to_string(dev));
    f(c);
    c.err.clear();
    return TDVP_OK;
  } catch (const TdvpError& e) {
    c.err = e.what();
    return e.status;
  } catch (const std::exception& e) {
    c.err = e.what();
    return TDVP_ERR_CUDA;
  }
}

void check_dims(const tdvp_site_dims* d) {
  tdvp_require(d != nullptr, TDVP_ERR_INVALID_ARG, "null dims");
  tdvp_require(d->ml >= 1 && d->mr >= 1 && d->wl >= 1 && d->wr >= 1 && d->d >= 1, TDVP_ERR_SHAPE,
               "dims must be >= 1");
}

WSparse make_w(const tdvp_site_dims* d, const double* W_host) {
  tdvp_require(W_host != nullptr, TDVP_ERR_INVALID_ARG, "null W");
  WSparse w;
  w.build(reinterpret_cast<const cplx*>(W_host), d->wl, d->wr, d->d);
  w.upload();
  return w;
}
}  // namespace

extern "C" {

tdvp_status tdvp_heff_contract(const tdvp_site_dims* dims, const void* L, const double* W, const void* R,
                               const void* x, void* y, int precision, void* stream) {
  return tdvp_heff_contract_cached(dims, L, W, R, x, y, precision, -1, stream);
}

tdvp_status tdvp_heff_contract_cached(const tdvp_site_dims* dims, const void* L, const double* W, const void* R,
                                      const void* x, void* y, int precision, long long env_tag, void* stream) {
  return raw_guarded([&](RawCtx& c) {
    tdvp_require(env_tag >= -1, TDVP_ERR_INVALID_ARG, "env_tag must be >= -1");
    check_dims(dims);
    tdvp_require(L && R && x && y && x != y, TDVP_ERR_INVALID_ARG, "null or aliased buffers");
    tdvp_require(precision >= TDVP_PREC_FP64 && precision <= TDVP_PREC_BF16X6, TDVP_ERR_INVALID_ARG,
                 "unknown precision");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    WSparse w = make_w(dims, W);
    SiteOp op;
    op.L = static_cast<const cplx*>(L);
    op.R = static_cast<const cplx*>(R);
    op.W = &w;
    op.ml = dims->ml;
    op.mr = dims->mr;
    op.wl = dims->wl;
    op.wr = dims->wr;
    op.d = dims->d;
    // a tag names the (L, R) content for the operand caches of the tensor-core paths;
    // tags are kept apart from nothing else (this context serves only these calls)
    op.env_key = env_tag;
    heff_apply_prec(st, c.scr, op, static_cast<const cplx*>(x), static_cast<cplx*>(y), precision);
    TDVP_CUDA(cudaStreamSynchronize(st));
    w.free_device();
    tc_check(st, c.scr);
  });
}

tdvp_status tdvp_keff_contract(int ml, int mr, int wb, const void* L, const void* R, const void* x, void* y,
                               void* stream) {
  return raw_guarded([&](RawCtx& c) {
    tdvp_require(ml >= 1 && mr >= 1 && wb >= 1, TDVP_ERR_SHAPE, "dims must be >= 1");
    tdvp_require(L && R && x && y && x != y, TDVP_ERR_INVALID_ARG, "null or aliased buffers");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    keff_fp64(st, c.scr, static_cast<const cplx*>(L), ml, static_cast<const cplx*>(R), mr, wb,
              static_cast<const cplx*>(x), static_cast<cplx*>(y));
    TDVP_CUDA(cudaStreamSynchronize(st));
  });
}

tdvp_status tdvp_env_contract(const tdvp_site_dims* dims, int side, const void* E, const double* W, const void* A,
                              void* out, void* stream) {
  return raw_guarded([&](RawCtx& c) {
    check_dims(dims);
    tdvp_require(E && A && out && E != out, TDVP_ERR_INVALID_ARG, "null or aliased buffers");
    tdvp_require(side == 0 || side == 1, TDVP_ERR_INVALID_ARG, "side must be 0 or 1");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    WSparse w = make_w(dims, W);
    if (side == 0)
      env_left_fp64(st, c.scr, static_cast<const cplx*>(E), w, static_cast<const cplx*>(A), dims->ml, dims->mr,
                    dims->d, static_cast<cplx*>(out));
    else
      env_right_fp64(st, c.scr, static_cast<const cplx*>(E), w, static_cast<const cplx*>(A), dims->ml, dims->mr,
                     dims->d, static_cast<cplx*>(out));
    TDVP_CUDA(cudaStreamSynchronize(st));
    w.free_device();
  });
}

tdvp_status tdvp_expm_contract(const tdvp_site_dims* dims, const void* L, const double* W, const void* R,
                               const void* x, void* y, double delta, tdvp_time kind, int precision, double tol,
                               int nmax, int* iters, void* stream) {
  return raw_guarded([&](RawCtx& c) {
    check_dims(dims);
    tdvp_require(L && R && x && y && x != y, TDVP_ERR_INVALID_ARG, "null or aliased buffers");
    tdvp_require(kind == TDVP_REAL || kind == TDVP_IMAG, TDVP_ERR_INVALID_ARG, "bad time kind");
    tdvp_require(precision >= TDVP_PREC_FP64 && precision <= TDVP_PREC_BF16X6, TDVP_ERR_INVALID_ARG,
                 "unknown precision");
    tdvp_require(tol > 0 && nmax >= 1 && nmax <= 63 && std::isfinite(delta), TDVP_ERR_INVALID_ARG,
                 "bad Lanczos parameters");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    WSparse w = make_w(dims, W);
    SiteOp op;
    op.L = static_cast<const cplx*>(L);
    op.R = static_cast<const cplx*>(R);
    op.W = &w;
    op.ml = dims->ml;
    op.mr = dims->mr;
    op.wl = dims->wl;
    op.wr = dims->wr;
    op.d = dims->d;
    op.env_key = (1LL << 62) + (c.key++);  // cache operands within this call only
    const long long n = (long long)dims->ml * dims->d * dims->mr;
    int it = 0;
    try {
      it = lanczos_expm(
          st, &c.pool, c.blas, c.lw, [&](const cplx* a, cplx* b) { heff_apply_prec(st, c.scr, op, a, b, precision); },
          static_cast<const cplx*>(x), static_cast<cplx*>(y), n, delta, kind, tol, nmax);
    } catch (...) {
      w.free_device();
      tc_check(st, c.scr);
      throw;
    }
    TDVP_CUDA(cudaStreamSynchronize(st));
    w.free_device();
    tc_check(st, c.scr);
    if (iters) *iters = it;
  });
}

const char* tdvp_contract_last_error(void) { return raw().err.c_str(); }

}  // extern "C"
