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

// Bytes of a file with header r: magic, 4 ints, bond dims, sites, hash.
long double file_bytes(const Header& r) {
  long double b = 8.0L + 16.0L + 4.0L * (r.n + 1) + 8.0L;
  for (int i = 0; i < r.n; ++i) b += 16.0L * r.m[i] * r.d * r.m[i + 1];
  return b;
}

// A whole checkpoint read through one open file: the header, a check that the file has exactly
// the size the header implies (before anything large is allocated), every site into memory of
// its own, and the hash.  Nothing reaches a caller before the hash has been verified.
struct Loaded {
  Header hdr;
  std::vector<std::vector<double>> sites;
};

Loaded load_file(const std::string& path) {
  File fl(fopen(path.c_str(), "rb"));
  tdvp_require(fl.f != nullptr, TDVP_ERR_INVALID_ARG, "checkpoint: cannot open " + path);
  tdvp_require(std::fseek(fl.f, 0, SEEK_END) == 0, TDVP_ERR_INVALID_ARG, "checkpoint: cannot seek " + path);
  const long size = std::ftell(fl.f);
  tdvp_require(size >= 0 && std::fseek(fl.f, 0, SEEK_SET) == 0, TDVP_ERR_INVALID_ARG,
               "checkpoint: cannot seek " + path);
  Fnv h;
  Loaded out;
  out.hdr = read_header(fl.f, h, path);
  const long double want = file_bytes(out.hdr);
  tdvp_require(want == (long double)size, TDVP_ERR_INVALID_ARG,
               "checkpoint: file size does not match its header (truncated or corrupt): " + path);
  out.sites.resize(out.hdr.n);
  for (int i = 0; i < out.hdr.n; ++i) {
    out.sites[i].resize(2 * (size_t)out.hdr.m[i] * out.hdr.d * out.hdr.m[i + 1]);
    get(fl.f, &h, out.sites[i].data(), sizeof(double) * out.sites[i].size(), path);
  }
  uint64_t sum = 0;
  get(fl.f, nullptr, &sum, sizeof(sum), path);
  tdvp_require(sum == h.h, TDVP_ERR_INVALID_ARG, "checkpoint: hash mismatch (corrupt file): " + path);
  return out;
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

tdvp_status tdvp_checkpoint_read_header(const char* path, int* n_sites, int* d, int* bond_dims, int capacity) {
  return ckpt_guarded([&] {
    tdvp_require(path && n_sites && d, TDVP_ERR_INVALID_ARG, "null argument");
    File fl(fopen(path, "rb"));
    tdvp_require(fl.f != nullptr, TDVP_ERR_INVALID_ARG, std::string("checkpoint: cannot open ") + path);
    Fnv h;
    const Header r = read_header(fl.f, h, path);
    if (bond_dims)
      tdvp_require(capacity >= r.n + 1, TDVP_ERR_SHAPE, "checkpoint: bond_dims buffer holds fewer than N + 1 ints");
    *n_sites = r.n;
    *d = r.d;
    if (bond_dims) std::memcpy(bond_dims, r.m.data(), sizeof(int) * (r.n + 1));
  });
}

tdvp_status tdvp_checkpoint_read(const char* path, int n_sites, int d, const int* bond_dims,
                                 double* const* sites_out) {
  return ckpt_guarded([&] {
    tdvp_require(path && bond_dims && sites_out, TDVP_ERR_INVALID_ARG, "null argument");
    const Loaded f = load_file(path);
    tdvp_require(f.hdr.n == n_sites && f.hdr.d == d, TDVP_ERR_SHAPE, "checkpoint: N or d differ from the buffers'");
    for (int i = 0; i <= n_sites; ++i)
      tdvp_require(f.hdr.m[i] == bond_dims[i], TDVP_ERR_SHAPE, "checkpoint: bond dimensions differ from the buffers'");
    for (int i = 0; i < n_sites; ++i) {
      tdvp_require(sites_out[i] != nullptr, TDVP_ERR_INVALID_ARG, "checkpoint: null site buffer");
      std::memcpy(sites_out[i], f.sites[i].data(), sizeof(double) * f.sites[i].size());
    }
  });
}

const char* tdvp_checkpoint_last_error(void) { return g_ckpt_err.c_str(); }

tdvp_status tdvp_save(tdvp_handle* h, const char* path) {
  if (!h) return TDVP_ERR_INVALID_ARG;
  tdvp_status s = TDVP_OK;
  const tdvp_status g = ckpt_guarded([&] {
    tdvp_require(path != nullptr, TDVP_ERR_INVALID_ARG, "null path");
    const int n = h->eng.N, d = h->eng.d;
    std::vector<int> m(h->eng.psi.m.begin(), h->eng.psi.m.end());
    std::vector<std::vector<double>> host(n);
    std::vector<double*> ptr(n);
    for (int i = 0; i < n; ++i) {
      host[i].resize(2 * (size_t)m[i] * d * m[i + 1]);
      ptr[i] = host[i].data();
    }
    s = tdvp_get_mps(h, ptr.data());
    if (s != TDVP_OK) return;
    write_file(path, n, d, m.data(), ptr.data());
  });
  if (s != TDVP_OK) return s;  // tdvp_get_mps left its reason on the handle
  if (g != TDVP_OK) h->err = g_ckpt_err;
  return g;
}

tdvp_status tdvp_load(const char* path, const tdvp_mpo_desc* mpo, const tdvp_options* opt, void* stream,
                      tdvp_handle** out) {
  if (!path || !mpo || !out) return TDVP_ERR_INVALID_ARG;
  Loaded f;
  const tdvp_status s = ckpt_guarded([&] { f = load_file(path); });
  if (s != TDVP_OK) return s;
  std::vector<double*> ptr(f.hdr.n);
  for (int i = 0; i < f.hdr.n; ++i) ptr[i] = f.sites[i].data();
  tdvp_mps_desc desc;
  desc.n_sites = f.hdr.n;
  desc.d = f.hdr.d;
  desc.bond_dims = f.hdr.m.data();
  desc.sites = ptr.data();
  return tdvp_create(&desc, mpo, opt, stream, out);
}

}  // extern "C"
