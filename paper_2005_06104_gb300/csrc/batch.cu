// Many independent GSE-TDVP1 chains on one GPU.
//
// A batch owns one engine per chain, each on its own non-blocking CUDA stream.
// A batch call runs the per-chain call on every chain with a pool of host worker
// threads.  A worker takes the next chain from a shared counter, in order of
// decreasing cost estimate (N * max bond^3), so long chains start first, and then
// drives that chain's kernels on the chain's stream.  The chains' kernels thus
// overlap on the device.
//
// A GSE-TDVP1 step takes host decisions between its launches: the Lanczos
// stopping test, truncation ranks, SVD block structure.  It is therefore not
// expressible as one captured graph or one persistent launch.  Concurrent
// streams fill the GPU instead, with chains of different lengths and bond
// dimensions each advancing at their own pace.  Each chain keeps its own
// convergence and error state.  A failing chain reports its status and leaves
// the others untouched.
#include <algorithm>
#include <atomic>
#include <numeric>
#include <thread>
#include <vector>

#include "engine.cuh"

struct tdvp_batch {
  int device = 0;
  int threads = 1;
  std::vector<cudaStream_t> streams;
  std::vector<tdvp_handle*> chains;
  std::vector<int> order;  // chains by decreasing cost estimate
  std::string err;
};

namespace {
double cost_estimate(const tdvp_handle* h) {
  const Engine& e = h->eng;
  double mx = 1.0;
  for (int m : e.psi.m) mx = std::max(mx, (double)m);
  return (double)e.N * mx * mx * mx;
}

void reorder(tdvp_batch* b) {
  b->order.resize(b->chains.size());
  std::iota(b->order.begin(), b->order.end(), 0);
  std::vector<double> c(b->chains.size());
  for (size_t i = 0; i < c.size(); ++i) c[i] = b->chains[i] ? cost_estimate(b->chains[i]) : 0.0;
  std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) { return c[x] > c[y]; });
}

// Runs f(i) for every chain on the worker pool; per-chain statuses into st (may be null).
template <class F>
tdvp_status run_all(tdvp_batch* b, int* st, F&& f) {
  const int n = (int)b->chains.size();
  std::vector<int> status(n, TDVP_OK);
  std::atomic<int> next{0};
  auto worker = [&] {
    cudaSetDevice(b->device);
    while (true) {
      const int k = next.fetch_add(1);
      if (k >= n) break;
      const int i = b->order.empty() ? k : b->order[k];
      status[i] = f(i);
    }
  };
  const int nt = std::max(1, std::min(b->threads, n));
  std::vector<std::thread> pool;
  pool.reserve(nt - 1);
  for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
  worker();
  for (auto& t : pool) t.join();
  tdvp_status first = TDVP_OK;
  b->err.clear();
  for (int i = 0; i < n; ++i) {
    if (st) st[i] = status[i];
    if (status[i] != TDVP_OK && first == TDVP_OK) {
      first = (tdvp_status)status[i];
      b->err = "chain " + std::to_string(i) + ": " +
               (b->chains[i] ? std::string(tdvp_last_error(b->chains[i])) : std::string("not created"));
    }
  }
  return first;
}
}  // namespace

extern "C" {

tdvp_status tdvp_batch_create(int n, const tdvp_mps_desc* mps, const tdvp_mpo_desc* mpo, const tdvp_options* opts,
                              int n_threads, tdvp_batch** out) {
  if (!out || n < 1 || !mps || !mpo) return TDVP_ERR_INVALID_ARG;
  *out = nullptr;
  tdvp_batch* b = nullptr;
  try {
    b = new tdvp_batch();
    b->threads = n_threads > 0 ? n_threads : (int)std::max(1u, std::thread::hardware_concurrency());
    if (cudaGetDevice(&b->device) != cudaSuccess) {
      delete b;
      return TDVP_ERR_CUDA;
    }
    b->streams.assign(n, nullptr);
    b->chains.assign(n, nullptr);
    for (int i = 0; i < n; ++i)
      if (cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking) != cudaSuccess) {
        b->err = "stream creation failed";
        tdvp_batch_destroy(b);
        return TDVP_ERR_CUDA;
      }
  } catch (...) {
    delete b;
    return TDVP_ERR_OUT_OF_MEMORY;
  }
  const tdvp_status s = run_all(b, nullptr, [&](int i) {
    return (int)tdvp_create(&mps[i], &mpo[i], opts ? &opts[i] : nullptr, b->streams[i], &b->chains[i]);
  });
  if (s != TDVP_OK) {
    tdvp_batch_destroy(b);
    return s;
  }
  reorder(b);
  *out = b;
  return TDVP_OK;
}

tdvp_status tdvp_batch_destroy(tdvp_batch* b) {
  if (!b) return TDVP_ERR_INVALID_ARG;
  for (auto* h : b->chains)
    if (h) tdvp_destroy(h);
  for (auto s : b->streams)
    if (s) cudaStreamDestroy(s);
  delete b;
  return TDVP_OK;
}

tdvp_status tdvp_batch_size(const tdvp_batch* b, int* n) {
  if (!b || !n) return TDVP_ERR_INVALID_ARG;
  *n = (int)b->chains.size();
  return TDVP_OK;
}

tdvp_status tdvp_batch_handle(tdvp_batch* b, int i, tdvp_handle** h) {
  if (!b || !h || i < 0 || i >= (int)b->chains.size()) return TDVP_ERR_INVALID_ARG;
  *h = b->chains[i];
  return TDVP_OK;
}

tdvp_status tdvp_batch_expand_basis(tdvp_batch* b, int k, const double* weights, int* status) {
  if (!b) return TDVP_ERR_INVALID_ARG;
  return run_all(b, status, [&](int i) { return (int)tdvp_expand_basis(b->chains[i], k, weights); });
}

tdvp_status tdvp_batch_sweep(tdvp_batch* b, double dt, tdvp_time kind, int* status) {
  if (!b) return TDVP_ERR_INVALID_ARG;
  return run_all(b, status, [&](int i) { return (int)tdvp_sweep(b->chains[i], dt, kind); });
}

tdvp_status tdvp_batch_step(tdvp_batch* b, int k, const double* weights, double dt, tdvp_time kind, int* status) {
  if (!b) return TDVP_ERR_INVALID_ARG;
  const tdvp_status s = run_all(b, status, [&](int i) {
    const tdvp_status e = tdvp_expand_basis(b->chains[i], k, weights);
    return (int)(e != TDVP_OK ? e : tdvp_sweep(b->chains[i], dt, kind));
  });
  reorder(b);  // bond dimensions grow: keep the longest chains first
  return s;
}

tdvp_status tdvp_batch_energy(tdvp_batch* b, double* out) {
  if (!b || !out) return TDVP_ERR_INVALID_ARG;
  return run_all(b, nullptr, [&](int i) { return (int)tdvp_energy(b->chains[i], &out[i]); });
}

tdvp_status tdvp_batch_norm(tdvp_batch* b, double* out) {
  if (!b || !out) return TDVP_ERR_INVALID_ARG;
  return run_all(b, nullptr, [&](int i) { return (int)tdvp_norm(b->chains[i], &out[i]); });
}

const char* tdvp_batch_last_error(const tdvp_batch* b) { return b ? b->err.c_str() : "null batch"; }

}  // extern "C"
