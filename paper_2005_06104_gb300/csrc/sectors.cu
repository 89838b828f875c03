// U(1) sector tables of the bond bases.
//
// A Hamiltonian that conserves a U(1) charge (total S^z for the Heisenberg and OAT models)
// keeps a state of definite charge block sparse: an entry A_i[l, s, r] can be nonzero only
// where q_r = q_l + c_s, c_s the charge of local basis state s.  The cost statement of
// Sec. I.C counts contractions over these blocks.  The engine stores tensors densely and
// finds blocks from the exact-zero pattern (each factorisation orders the new bond index by
// block); this file reads the charges back off that pattern, bond by bond from the left end
// (charge 0), so that a caller can see the sector table (charge, dim, offset) of every bond.
#include <climits>
#include <cstdlib>

#include "engine.cuh"

namespace {
constexpr int kNoCharge = INT_MIN;

__global__ void k_charge_init(int* lo, int* hi, int n) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) {
    lo[r] = INT_MAX;
    hi[r] = INT_MIN;
  }
}

// Rows [y*rows, (y+1)*rows) of A viewed as (ml*d) x mr; one thread per column r.  Every exact
// nonzero A[l, s, r] with a known q_in[l] proposes q_in[l] + phys[s] for r.
__global__ void k_charge_minmax(const cplx* __restrict__ A, int ml, int d, int mr, const int* __restrict__ q_in,
                                const int* __restrict__ phys, int rows, int* lo, int* hi) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= mr) return;
  const long long r0 = (long long)blockIdx.y * rows;
  const long long r1 = min((long long)ml * d, r0 + rows);
  int a = INT_MAX, b = INT_MIN;
  for (long long ls = r0; ls < r1; ++ls) {
    const cplx v = A[ls * mr + r];
    if (v.x == 0.0 && v.y == 0.0) continue;
    const int ql = q_in[ls / d];
    if (ql == kNoCharge) continue;
    const int q = ql + phys[ls % d];
    a = min(a, q);
    b = max(b, q);
  }
  if (a <= b) {
    atomicMin(lo + r, a);
    atomicMax(hi + r, b);
  }
}

// flags bit 0: some index got two charges; bit 1: some index got none
__global__ void k_charge_final(const int* __restrict__ lo, const int* __restrict__ hi, int n, int* q_out,
                               int* flags) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  if (lo[r] > hi[r]) {
    q_out[r] = kNoCharge;
    atomicOr(flags, 2);
  } else if (lo[r] != hi[r]) {
    q_out[r] = kNoCharge;
    atomicOr(flags, 1);
  } else {
    q_out[r] = lo[r];
  }
}
}  // namespace

std::vector<std::vector<int>> bond_charges(Engine& e, const int* phys_host) {
  const int N = e.N, d = e.d;
  long long cmax = 0;
  for (int s = 0; s < d; ++s) {
    tdvp_require(phys_host[s] > -(1 << 20) && phys_host[s] < (1 << 20), TDVP_ERR_INVALID_ARG,
                 "bond_charges: local charges must lie within +-2^20");
    cmax = std::max(cmax, (long long)std::abs(phys_host[s]));
  }
  // every bond charge is a sum of at most N local charges: keep it inside int
  tdvp_require((long long)N * cmax < (1LL << 30), TDVP_ERR_INVALID_ARG,
               "bond_charges: N * max |local charge| must stay below 2^30");
  int mmax = 1;
  for (int m : e.psi.m) mmax = std::max(mmax, m);
  RawBuf phys, q_in, q_out, lo, hi, flags;
  phys.ensure(&e.pool, sizeof(int) * d);
  q_in.ensure(&e.pool, sizeof(int) * mmax);
  q_out.ensure(&e.pool, sizeof(int) * mmax);
  lo.ensure(&e.pool, sizeof(int) * mmax);
  hi.ensure(&e.pool, sizeof(int) * mmax);
  flags.ensure(&e.pool, sizeof(int));
  TDVP_CUDA(cudaMemcpyAsync(phys.as<int>(), phys_host, sizeof(int) * d, cudaMemcpyHostToDevice, e.st));
  TDVP_CUDA(cudaMemsetAsync(flags.as<int>(), 0, sizeof(int), e.st));
  std::vector<std::vector<int>> out(N + 1);
  out[0].assign(e.psi.m[0], 0);  // the left end carries charge 0
  TDVP_CUDA(cudaMemcpyAsync(q_in.as<int>(), out[0].data(), sizeof(int) * e.psi.m[0], cudaMemcpyHostToDevice, e.st));
  const int rows = 64;
  for (int i = 0; i < N; ++i) {
    const int ml = e.psi.m[i], mr = e.psi.m[i + 1];
    const int g1 = ceil_div(mr, 128);
    k_charge_init<<<g1, 128, 0, e.st>>>(lo.as<int>(), hi.as<int>(), mr);
    TDVP_CHECK_LAUNCH();
    dim3 g(g1, ceil_div((long long)ml * d, rows));
    tdvp_require(g.y <= 65535, TDVP_ERR_INVALID_ARG, "bond_charges: bond too large");
    k_charge_minmax<<<g, 128, 0, e.st>>>(e.psi.A[i].data(), ml, d, mr, q_in.as<int>(), phys.as<int>(), rows,
                                         lo.as<int>(), hi.as<int>());
    TDVP_CHECK_LAUNCH();
    k_charge_final<<<g1, 128, 0, e.st>>>(lo.as<int>(), hi.as<int>(), mr, q_out.as<int>(), flags.as<int>());
    TDVP_CHECK_LAUNCH();
    out[i + 1].resize(mr);
    TDVP_CUDA(cudaMemcpyAsync(out[i + 1].data(), q_out.as<int>(), sizeof(int) * mr, cudaMemcpyDeviceToHost, e.st));
    TDVP_CUDA(cudaMemcpyAsync(q_in.as<int>(), q_out.as<int>(), sizeof(int) * mr, cudaMemcpyDeviceToDevice, e.st));
  }
  int fl = 0;
  TDVP_CUDA(cudaMemcpyAsync(&fl, flags.as<int>(), sizeof(int), cudaMemcpyDeviceToHost, e.st));
  e.sync();
  for (int b = 0; b <= N; ++b) {
    for (size_t r = 0; r < out[b].size(); ++r) {
      tdvp_require(out[b][r] != kNoCharge, TDVP_ERR_SHAPE,
                   "bond_charges: index " + std::to_string(r) + " of bond " + std::to_string(b) +
                       ((fl & 1) ? " carries two charges or follows one that does: the state does not conserve them"
                                 : " has no nonzero entry"));
    }
  }
  return out;
}

std::vector<int> sector_runs(const std::vector<int>& q, bool* contiguous) {
  std::vector<int> t;  // (charge, dim, offset) triples
  for (size_t r = 0; r < q.size(); ++r) {
    if (!t.empty() && t[t.size() - 3] == q[r]) {
      ++t[t.size() - 2];
    } else {
      t.push_back(q[r]);
      t.push_back(1);
      t.push_back((int)r);
    }
  }
  bool ok = true;
  for (size_t a = 0; a < t.size() && ok; a += 3)
    for (size_t b = a + 3; b < t.size(); b += 3)
      if (t[a] == t[b]) {
        ok = false;
        break;
      }
  *contiguous = ok;
  return t;
}
