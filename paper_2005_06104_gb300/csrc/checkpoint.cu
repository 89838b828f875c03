// Checkpoint files of an MPS: host-side writer and reader, and the handle
// entry points built on them (save the state of a handle, create a handle from
// a file).  Layout (little-endian):
//   "GSETDVP1"            8-byte magic
//   int32 version (1), N, d, reserved (0)
//   int32 bond_dims[N + 1]
//   per site i: complex128 A_i[m_i][d][m_{i+1}] (re, im interleaved)
//   uint64 FNV-1a hash of every preceding byte
// Files are written to "<path>.tmp" and renamed over <path>, so an interrupted
// save never leaves a partial file under the final name.
#include <cstdio>
#include <cstring>
#include <vector>

#include "engine.cuh"

namespace {
constexpr char kMagic[8] = {'G', 'S', 'E', 'T', 'D', 'V', 'P', '1'};
constexpr int kVersion = 1;
constexpr int kMaxSites = 1 << 20;

struct Fnv {
  uint64_t h = 1469598103934665603ull;
  void add(const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) {
      h ^= b[i];
      h *= 1099511628211ull;
    }
  }
};

struct File {
  FILE* f = nullptr;
  explicit File(FILE* p) : f(p) {}
  ~File() {
    if (f) fclose(f);
  }
};

void put(FILE* f, Fnv& h, const void* p, size_t n, const std::string& path) {
  tdvp_require(fwrite(p, 1, n, f) == n, TDVP_ERR_INVALID_ARG, "checkpoint: write failed: " + path);
  h.add(p, n);
}
void get(FILE* f, Fnv* h, void* p, size_t n, const std::string& path) {
  tdvp_require(fread(p, 1, n, f) == n, TDVP_ERR_INVALID_ARG, "checkpoint: file truncated: " + path);
  if (h) h->add(p, n);
}

struct Header {
  int n = 0, d = 0;
  std::vector<int> m;
};

void check_dims(int n, int d, const int* m) {
  tdvp_require(n >= 1 && n <= kMaxSites && d >= 1 && d <= 64, TDVP_ERR_SHAPE, "checkpoint: bad N or d");
  tdvp_require(m[0] == 1 && m[n] == 1, TDVP_ERR_SHAPE, "checkpoint: boundary bond dimensions must be 1");
  for (int i = 0; i <= n; ++i) tdvp_require(m[i] >= 1 && m[i] <= (1 << 20), TDVP_ERR_SHAPE, "checkpoint: bad bond");
}

Header read_header(FILE* f, Fnv& h, const std::string& path) {
  char magic[8];
  get(f, &h, magic, 8, path);
  tdvp_require(std::memcmp(magic, kMagic, 8) == 0, TDVP_ERR_INVALID_ARG, "checkpoint: not a GSE-TDVP file: " + path);
  int32_t hd[4];
  get(f, &h, hd, sizeof(hd), path);
  tdvp_require(hd[0] == kVersion, TDVP_ERR_INVALID_ARG, "checkpoint: unsupported version");
  Header r;
  r.n = hd[1];
  r.d = hd[2];
  tdvp_require(r.n >= 1 && r.n <= kMaxSites, TDVP_ERR_SHAPE, "checkpoint: bad N");
  r.m.resize(r.n + 1);
  get(f, &h, r.m.data(), sizeof(int32_t) * (r.n + 1), path);
  check_dims(r.n, r.d, r.m.data());
  return r;
}

// The whole file: header, sites (into caller buffers when `sites` is non-null), hash.
Header read_file(const std::string& path, double* const* sites) {
  File fl(fopen(path.c_str(), "rb"));
  tdvp_require(fl.f != nullptr, TDVP_ERR_INVALID_ARG, "checkpoint: cannot open " + path);
  Fnv h;
  Header r = read_header(fl.f, h, path);
  std::vector<double> tmp;
  for (int i = 0; i < r.n; ++i) {
    const size_t cnt = 2 * (size_t)r.m[i] * r.d * r.m[i + 1];
    double* dst = nullptr;
    if (sites) {
      tdvp_require(sites[i] != nullptr, TDVP_ERR_INVALID_ARG, "checkpoint: null site buffer");
      dst = sites[i];
    } else {
      tmp.resize(cnt);
      dst = tmp.data();
    }
    get(fl.f, &h, dst, sizeof(double) * cnt, path);
  }
  uint64_t want = 0;
  get(fl.f, nullptr, &want, sizeof(want), path);
  tdvp_require(want == h.h, TDVP_ERR_INVALID_ARG, "checkpoint: hash mismatch (corrupt file): " + path);
  return r;
}

void write_file(const std::string& path, int n, int d, const int* m, const double* const* sites) {
  check_dims(n, d, m);
  const std::string tmp = path + ".tmp";
  {
    File fl(fopen(tmp.c_str(), "wb"));
    tdvp_require(fl.f != nullptr, TDVP_ERR_INVALID_ARG, "checkpoint: cannot create " + tmp);
    Fnv h;
    put(fl.f, h, kMagic, 8, tmp);
    const int32_t hd[4] = {kVersion, n, d, 0};
    put(fl.f, h, hd, sizeof(hd), tmp);
    put(fl.f, h, m, sizeof(int32_t) * (n + 1), tmp);
    for (int i = 0; i < n; ++i) {
      tdvp_require(sites[i] != nullptr, TDVP_ERR_INVALID_ARG, "checkpoint: null site buffer");
      put(fl.f, h, sites[i], sizeof(double) * 2 * (size_t)m[i] * d * m[i + 1], tmp);
    }
    const uint64_t sum = h.h;
    tdvp_require(fwrite(&sum, 1, sizeof(sum), fl.f) == sizeof(sum), TDVP_ERR_INVALID_ARG,
                 "checkpoint: write failed: " + tmp);
    tdvp_require(fflush(fl.f) == 0, TDVP_ERR_INVALID_ARG, "checkpoint: flush failed: " + tmp);
  }
  tdvp_require(std::rename(tmp.c_str(), path.c_str()) == 0, TDVP_ERR_INVALID_ARG,
               "checkpoint: cannot rename " + tmp + " to " + path);
}

thread_local std::string g_ckpt_err;

template <class F>
tdvp_status ckpt_guarded(F&& f) {
  try {
    f();
    g_ckpt_err.clear();
    return TDVP_OK;
  } catch (const TdvpError& e) {
    g_ckpt_err = e.what();
    return e.status;
  } catch (const std::exception& e) {
    g_ckpt_err = e.what();
    return TDVP_ERR_INVALID_ARG;
  }
}
}  // namespace

extern "C" {

tdvp_status tdvp_checkpoint_write(const char* path, const tdvp_mps_desc* mps) {
  return ckpt_guarded([&] {
    tdvp_require(path && mps && mps->bond_dims && mps->sites, TDVP_ERR_INVALID_ARG, "null argument");
    write_file(path, mps->n_sites, mps->d, mps->bond_dims, mps->sites);
  });
}

tdvp_status tdvp_checkpoint_read_header(const char* path, int* n_sites, int* d, int* bond_dims) {
  return ckpt_guarded([&] {
    tdvp_require(path && n_sites && d, TDVP_ERR_INVALID_ARG, "null argument");
    File fl(fopen(path, "rb"));
    tdvp_require(fl.f != nullptr, TDVP_ERR_INVALID_ARG, std::string("checkpoint: cannot open ") + path);
    Fnv h;
    const Header r = read_header(fl.f, h, path);
    *n_sites = r.n;
    *d = r.d;
    if (bond_dims) std::memcpy(bond_dims, r.m.data(), sizeof(int) * (r.n + 1));
  });
}

tdvp_status tdvp_checkpoint_read(const char* path, double* const* sites_out) {
  return ckpt_guarded([&] {
    tdvp_require(path && sites_out, TDVP_ERR_INVALID_ARG, "null argument");
    read_file(path, sites_out);
  });
}

const char* tdvp_checkpoint_last_error(void) { return g_ckpt_err.c_str(); }

tdvp_status tdvp_save(tdvp_handle* h, const char* path) {
  if (!h) return TDVP_ERR_INVALID_ARG;
  const int n = h->eng.N, d = h->eng.d;
  std::vector<int> m(h->eng.psi.m.begin(), h->eng.psi.m.end());
  std::vector<std::vector<double>> host(n);
  std::vector<double*> ptr(n);
  for (int i = 0; i < n; ++i) {
    host[i].resize(2 * (size_t)m[i] * d * m[i + 1]);
    ptr[i] = host[i].data();
  }
  tdvp_status s = tdvp_get_mps(h, ptr.data());
  if (s != TDVP_OK) return s;
  tdvp_mps_desc desc;
  desc.n_sites = n;
  desc.d = d;
  desc.bond_dims = m.data();
  desc.sites = ptr.data();
  s = tdvp_checkpoint_write(path, &desc);
  if (s != TDVP_OK) h->err = g_ckpt_err;
  return s;
}

tdvp_status tdvp_load(const char* path, const tdvp_mpo_desc* mpo, const tdvp_options* opt, void* stream,
                      tdvp_handle** out) {
  if (!path || !mpo || !out) return TDVP_ERR_INVALID_ARG;
  int n = 0, d = 0;
  tdvp_status s = tdvp_checkpoint_read_header(path, &n, &d, nullptr);
  if (s != TDVP_OK) return s;
  std::vector<int> m(n + 1);
  s = tdvp_checkpoint_read_header(path, &n, &d, m.data());
  if (s != TDVP_OK) return s;
  std::vector<std::vector<double>> host(n);
  std::vector<double*> ptr(n);
  for (int i = 0; i < n; ++i) {
    host[i].resize(2 * (size_t)m[i] * d * m[i + 1]);
    ptr[i] = host[i].data();
  }
  s = tdvp_checkpoint_read(path, ptr.data());
  if (s != TDVP_OK) return s;
  tdvp_mps_desc desc;
  desc.n_sites = n;
  desc.d = d;
  desc.bond_dims = m.data();
  desc.sites = ptr.data();
  return tdvp_create(&desc, mpo, opt, stream, out);
}

}  // extern "C"
