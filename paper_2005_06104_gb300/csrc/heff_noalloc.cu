// H_eff apply with no device allocation.
//
// Some callers cannot call cudaMalloc: code that runs while the device
// allocator is off limits (an embedding framework that owns every device
// allocation and forbids others, a real-time loop that must not block on the
// allocator, or an allocation-free harness).  For them this file offers one
// entry point, tdvp_heff_contract_noalloc, whose intermediates live in a
// fixed file-scope device array instead of pool memory.  The arithmetic is the
// FP64 H_eff of tdvp_heff_contract; the caller still passes inputs and outputs.
#include <cstring>
#include <mutex>

#include "linalg.cuh"

namespace {
// Every GPU that loads the library holds this array until the process exits.
constexpr size_t kScratchBytes = size_t(32) << 20;      // 32 MiB in total
constexpr size_t kListBytes = size_t(1) << 20;          // first 1 MiB: MPO lists
constexpr int kMaxDev = 64;
constexpr int kMaxW = 16384;                            // w_l * d * d * w_r complex entries
static __device__ __align__(256) unsigned char g_heff_scratch[kScratchBytes];

std::mutex g_mu;
unsigned char* g_addr[kMaxDev] = {};
// host staging of the sparse MPO lists (fixed size: no host heap either)
int h_off[kMaxW + 1];
int h_idx[2 * kMaxW];
cplx h_val[kMaxW];

// The symbol's address must be looked up per device with that device current;
// in host code the name g_heff_scratch is only a host-side stand-in.
unsigned char* scratch_on_current_device() {
  int dev = 0;
  TDVP_CUDA(cudaGetDevice(&dev));
  tdvp_require(dev >= 0 && dev < kMaxDev, TDVP_ERR_INVALID_ARG, "device index out of range");
  if (!g_addr[dev]) {
    void* p = nullptr;
    TDVP_CUDA(cudaGetSymbolAddress(&p, g_heff_scratch));
    g_addr[dev] = static_cast<unsigned char*>(p);
  }
  return g_addr[dev];
}
}  // namespace

namespace {
void put_error(char* buf, int len, const char* msg) {
  if (!buf || len <= 0) return;
  std::strncpy(buf, msg, (size_t)len - 1);
  buf[len - 1] = '\0';
}
}  // namespace

extern "C" tdvp_status tdvp_heff_contract_noalloc(const tdvp_site_dims* dims, const void* L, const double* W_host,
                                                  const void* R, const void* x, void* y, void* stream, char* err,
                                                  int err_len) {
  std::lock_guard<std::mutex> lk(g_mu);
  put_error(err, err_len, "");
  try {
    tdvp_require(dims != nullptr && W_host && L && R && x && y && x != y, TDVP_ERR_INVALID_ARG,
                 "null or aliased argument");
    const int ml = dims->ml, mr = dims->mr, wl = dims->wl, wr = dims->wr, d = dims->d;
    tdvp_require(ml >= 1 && mr >= 1 && wl >= 1 && wr >= 1 && d >= 1, TDVP_ERR_SHAPE, "dims must be >= 1");
    const long long nw = (long long)wl * d * d * wr;
    tdvp_require(nw <= kMaxW && d * wr + 1 <= kMaxW + 1, TDVP_ERR_INVALID_ARG,
                 "MPO site too large for the fixed scratch (w_l d d w_r <= 16384)");
    const long long n1 = (long long)ml * wl * d * mr, n2 = (long long)ml * d * wr * mr;
    const long long need = (n1 + n2) * (long long)sizeof(cplx);
    tdvp_require(need <= (long long)(kScratchBytes - kListBytes), TDVP_ERR_INVALID_ARG,
                 "intermediates exceed the fixed scratch: (m_l w_l d m_r + m_l d w_r m_r) * 16 bytes must be "
                 "<= 31 MiB");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char* base = scratch_on_current_device();
    // sparse lists of W grouped by output (s, v), staged in fixed host arrays
    const cplx* W = reinterpret_cast<const cplx*>(W_host);
    int nnz = 0;
    h_off[0] = 0;
    for (int s = 0; s < d; ++s)
      for (int v = 0; v < wr; ++v) {
        for (int w = 0; w < wl; ++w)
          for (int t = 0; t < d; ++t) {
            const cplx e = W[((w * d + s) * d + t) * wr + v];
            if (e.x != 0.0 || e.y != 0.0) {
              h_idx[2 * nnz] = w;
              h_idx[2 * nnz + 1] = t;
              h_val[nnz] = e;
              ++nnz;
            }
          }
        h_off[s * wr + v + 1] = nnz;
      }
    int* d_off = reinterpret_cast<int*>(base);
    int* d_idx = reinterpret_cast<int*>(base + 65536 * sizeof(int));
    cplx* d_val = reinterpret_cast<cplx*>(base + 3 * 65536 * sizeof(int));
    TDVP_CUDA(cudaMemcpyAsync(d_off, h_off, sizeof(int) * (d * wr + 1), cudaMemcpyHostToDevice, st));
    if (nnz) {
      TDVP_CUDA(cudaMemcpyAsync(d_idx, h_idx, sizeof(int) * 2 * nnz, cudaMemcpyHostToDevice, st));
      TDVP_CUDA(cudaMemcpyAsync(d_val, h_val, sizeof(cplx) * nnz, cudaMemcpyHostToDevice, st));
    }
    WSparse ws;  // views into the fixed array; never uploaded or freed (free_device is never called)
    ws.wl = wl;
    ws.wr = wr;
    ws.d = d;
    ws.nnz = nnz;
    ws.d_l_off = d_off;
    ws.d_l_idx = d_idx;
    ws.d_l_val = d_val;
    cplx* T1 = reinterpret_cast<cplx*>(base + kListBytes);
    cplx* T2 = T1 + n1;
    const cplx one = mkc(1.0, 0.0), zero = mkc(0.0, 0.0);
    zgemm(st, OP_N, OP_N, ml * wl, d * mr, ml, one, static_cast<const cplx*>(L), ml, static_cast<const cplx*>(x),
          d * mr, zero, T1, d * mr);
    wstage_left(st, ws, T1, T2, ml, mr);
    zgemm(st, OP_N, OP_T, ml * d, mr, wr * mr, one, T2, (long long)wr * mr, static_cast<const cplx*>(R),
          (long long)wr * mr, zero, static_cast<cplx*>(y), mr);
    TDVP_CUDA(cudaStreamSynchronize(st));
    return TDVP_OK;
  } catch (const TdvpError& e) {
    put_error(err, err_len, e.what());
    return e.status;
  } catch (const std::exception& e) {
    put_error(err, err_len, e.what());
    return TDVP_ERR_CUDA;
  }
}
