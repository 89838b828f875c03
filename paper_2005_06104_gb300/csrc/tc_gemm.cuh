// Tensor-core (tcgen05, sm_103a) split-TF32 contractions for H_eff.
#pragma once
#include "common.cuh"

// Operand caches of the environments of one site, in the layout the
// tensor-core GEMM reads (built once per site visit, reused by every Lanczos
// iteration).
struct TcEnvCache {
  long long key = -1;  // env_key of the cached (L, R); -1 = empty
  RawBuf Lhi, Llo;   // L as (m_l w_l) x (2 m_l) real, K contiguous, tf32 hi / lo parts
  RawBuf Rhi, Rlo;   // R expanded to a real (2 m_r) x (2 w_r m_r) operand, hi / lo
  RawBuf Bhi, Blo;   // per-apply operand of the vector (stage 1 B operand)
  RawBuf T1, T2hi, T2lo;  // stage outputs
  RawBuf err;        // device status word (non-zero: a bounded wait ran out)
  bool pending = false;  // launches since the last check of `err`
};

