// uf_finalize.h -- the stripe finalize (uf_finalize.cu).
#pragma once
#include "uf_internal.h"

namespace ufg {

// ---- finalize (uf_finalize.cu) ----
struct FinalArgs {
  int method;           // uf_method
  int n;
  int64_t s0, s1;       // stripes [s0, s1)
  int full;             // 1: condensed output, 0: stripe-major
  int mixed_forms;      // 1: the FP32 min kernel's abs-form stripes are present
  const unsigned long long *M, *M2, *Dg;  // fixed-point accumulators of this table
  double inv_scale;     // 2^-F
  void *out;
  int out_fp32;
  // sparse-row diagonal of this table (uf_sparse.cu), or null: R[k] = sum of
  // the sparse rows' x[k] (ACC_MIN) or l u[k]^alpha (ACC_GEN)
  const unsigned long long *Dsp;
};
cudaError_t launch_finalize(const FinalArgs &a, cudaStream_t st);

}  // namespace ufg
