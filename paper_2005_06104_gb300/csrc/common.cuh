// Shared device/host helpers of libgsetdvp: complex FP64 arithmetic, error
// handling, a caching device allocator and launch helpers.
#pragma once
#include <atomic>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <map>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/gse_tdvp.h"

typedef double2 cplx;

__host__ __device__ __forceinline__ cplx mkc(double r, double i) { return make_double2(r, i); }
__host__ __device__ __forceinline__ cplx cadd(cplx a, cplx b) { return mkc(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ cplx csub(cplx a, cplx b) { return mkc(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ cplx cmul(cplx a, cplx b) {
  return mkc(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ cplx cconj(cplx a) { return mkc(a.x, -a.y); }
__host__ __device__ __forceinline__ cplx cscale(cplx a, double s) { return mkc(a.x * s, a.y * s); }
// a += b * c
__host__ __device__ __forceinline__ void cfma(cplx& a, cplx b, cplx c) {
  a.x = fma(b.x, c.x, fma(-b.y, c.y, a.x));
  a.y = fma(b.x, c.y, fma(b.y, c.x, a.y));
}
// a += conj(b) * c
__host__ __device__ __forceinline__ void cfma_conj(cplx& a, cplx b, cplx c) {
  a.x = fma(b.x, c.x, fma(b.y, c.y, a.x));
  a.y = fma(b.x, c.y, fma(-b.y, c.x, a.y));
}
__host__ __device__ __forceinline__ double cabs2(cplx a) { return a.x * a.x + a.y * a.y; }

// Internal error type; converted to a tdvp_status at the C-ABI boundary.
struct TdvpError : public std::runtime_error {
  tdvp_status status;
  TdvpError(tdvp_status s, const std::string& m) : std::runtime_error(m), status(s) {}
};

#define TDVP_CUDA(call)                                                              \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      throw TdvpError(e_ == cudaErrorMemoryAllocation ? TDVP_ERR_OUT_OF_MEMORY        \
                                                      : TDVP_ERR_CUDA,               \
                      std::string(#call) + ": " + cudaGetErrorString(e_) + " at " +  \
                          __FILE__ + ":" + std::to_string(__LINE__));                \
    }                                                                                \
  } while (0)

// Process-wide count of kernel launches made by this library.  Every launch
// site is followed by exactly one TDVP_CHECK_LAUNCH, which bumps it.
extern std::atomic<long long> g_kernel_launches;
#define TDVP_CHECK_LAUNCH()                                             \
  do {                                                                  \
    g_kernel_launches.fetch_add(1, std::memory_order_relaxed);          \
    TDVP_CUDA(cudaGetLastError());                                      \
  } while (0)

inline void tdvp_require(bool ok, tdvp_status s, const std::string& msg) {
  if (!ok) throw TdvpError(s, msg);
}

// ---------------------------------------------------------------------------
// Caching device allocator: blocks are rounded up to a power of two (>= 4 KiB)
// and recycled per size class, so steady-state sweeps never call cudaMalloc.
class DevicePool {
 public:
  void* get(size_t bytes) {
    size_t cls = size_class(bytes);
    auto& fl = free_[cls];
    if (!fl.empty()) {
      void* p = fl.back();
      fl.pop_back();
      return p;
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, cls);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      trim();
      TDVP_CUDA(cudaMalloc(&p, cls));
    }
    live_bytes_ += cls;
    return p;
  }
  void put(void* p, size_t bytes) {
    if (p) free_[size_class(bytes)].push_back(p);
  }
  void trim() {
    for (auto& kv : free_)
      for (void* p : kv.second) {
        cudaFree(p);
        live_bytes_ -= kv.first;
      }
    free_.clear();
  }
  ~DevicePool() { trim(); }
  size_t live_bytes() const { return live_bytes_; }
  // bytes held in the free lists (allocated from the device, not in use)
  size_t cached_bytes() const {
    size_t b = 0;
    for (const auto& kv : free_) b += kv.first * kv.second.size();
    return b;
  }
  // powers of two up to 256 MiB; above, multiples of 1/16 of the next power of two (at most
  // 6.25 % unused), so that the large environments of a high bond dimension do not waste
  // up to half of their block
  static size_t size_class(size_t bytes) {
    size_t c = 4096;
    while (c < bytes) c <<= 1;
    if (c > (size_t(256) << 20)) {
      const size_t step = c >> 4;
      c = (bytes + step - 1) / step * step;
    }
    return c;
  }

 private:
  std::map<size_t, std::vector<void*>> free_;
  size_t live_bytes_ = 0;
};

// A device array of complex numbers drawn from a pool (RAII).
class DArr {
 public:
  DArr() = default;
  DArr(DevicePool* pool, size_t n) { reset(pool, n); }
  DArr(const DArr&) = delete;
  DArr& operator=(const DArr&) = delete;
  DArr(DArr&& o) noexcept { swap(o); }
  DArr& operator=(DArr&& o) noexcept {
    if (this != &o) {
      release();
      swap(o);
    }
    return *this;
  }
  ~DArr() { release(); }
  void reset(DevicePool* pool, size_t n) {
    release();
    pool_ = pool;
    n_ = n;
    if (n) p_ = static_cast<cplx*>(pool->get(n * sizeof(cplx)));
  }
  // keeps the buffer when it is large enough
  void ensure(DevicePool* pool, size_t n) {
    if (p_ && DevicePool::size_class(n * sizeof(cplx)) ==
                  DevicePool::size_class(n_ * sizeof(cplx))) {
      n_ = n;
      return;
    }
    reset(pool, n);
  }
  void release() {
    if (p_ && pool_) pool_->put(p_, n_ * sizeof(cplx));
    p_ = nullptr;
    n_ = 0;
  }
  void swap(DArr& o) {
    std::swap(p_, o.p_);
    std::swap(n_, o.n_);
    std::swap(pool_, o.pool_);
  }
  cplx* data() const { return p_; }
  size_t size() const { return n_; }

 private:
  cplx* p_ = nullptr;
  size_t n_ = 0;
  DevicePool* pool_ = nullptr;
};

// A raw device buffer (bytes) drawn from a pool (RAII).
class RawBuf {
 public:
  RawBuf() = default;
  RawBuf(const RawBuf&) = delete;
  RawBuf& operator=(const RawBuf&) = delete;
  ~RawBuf() { release(); }
  void ensure(DevicePool* pool, size_t bytes) {
    if (p_ && DevicePool::size_class(bytes) == DevicePool::size_class(bytes_)) {
      bytes_ = bytes;
      return;
    }
    release();
    pool_ = pool;
    bytes_ = bytes;
    if (bytes) p_ = pool->get(bytes);
  }
  void release() {
    if (p_ && pool_) pool_->put(p_, bytes_);
    p_ = nullptr;
    bytes_ = 0;
  }
  template <class T>
  T* as() const { return static_cast<T*>(p_); }
  size_t bytes() const { return bytes_; }

 private:
  void* p_ = nullptr;
  size_t bytes_ = 0;
  DevicePool* pool_ = nullptr;
};

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }
