// uf_finalize.h -- the stripe finalize (uf_finalize.cu).
#pragma once
#include "uf_internal.h"

namespace ufg {

// ---- finalize (uf_finalize.cu) ----
struct FinalArgs {
  int method;           // 0 unweighted, 1 / 2 weighted (min or abs form), 3 den and Q / N form
  int unnormalized;     // 1: the distance is the numerator alone, num * 2^-F
  int n;
  int64_t s0, s1;       // stripes [s0, s1)
  int full;             // 1: condensed output, 0: stripe-major
  unsigned abs_mask;    // ACC_MIN: stripes s with abs_row(abs_mask, s) hold the abs form
  int gen_abs;          // generalized: M2 holds N = num (FP64) instead of Q (FP32)
  unsigned long long *clamps;  // or null: counts cells whose min-form numerator rounded below 0
  // FP64 calls: the second words of M / M2 and of Dg / Dsp sit this many
  // elements after the first (two-word fixed point, uf_device.cuh); 0: one word
  int64_t m_lo_off, d_lo_off;
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
