// uf_finalize.cu -- stripe accumulators -> distances: the step that, in the
// paper, moves results out of the unified stripe buffer after the branch loop
// (Sec. 2), here with the num / den division in FP64.
//
// Per cell (stripe s, sample k, partner j = (k + s + 1) mod n), with
// M = sum_e min(x_e[k], x_e[j]) and D the same sum at offset 0:
//   weighted:    sum l |p_k - p_j| = D_k + D_j - 2M,  sum l (p_k + p_j) = D_k + D_j
//   unweighted:  sum l [xor] = W_k + W_j - 2G,         sum l [or] = W_k + W_j - G
//                (W = D, G = M on presence embeddings)
//   generalized: num = den - 2Q
// A ratio with den == 0 is 0; numerators are clamped at 0 against rounding.
#include "uf_internal.h"

namespace ufg {

__global__ void k_finalize(const FinalArgs a) {
  const int64_t rows = a.s1 - a.s0;
  const int64_t total = rows * a.n;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < total;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = c / a.n;
    const int k = (int)(c - r * a.n);
    const int64_t s = a.s0 + r;
    int64_t j = k + s + 1;
    if (j >= a.n) j -= a.n;
    if (a.full && 2 * (s + 1) == a.n && k >= a.n / 2) continue;  // duplicate half stripe
    const double m = a.M[c];
    double val;
    switch (a.method) {
    case 0: {  // unweighted
      const double w = a.Dg[k] + a.Dg[j];
      const double num = fmax(w - 2.0 * m, 0.0), den = w - m;
      val = den > 0.0 ? num / den : 0.0;
    } break;
    case 1:  // weighted unnormalized
      val = fmax(a.Dg[k] + a.Dg[j] - 2.0 * m, 0.0);
      break;
    case 2: {  // weighted normalized
      const double den = a.Dg[k] + a.Dg[j];
      const double num = fmax(den - 2.0 * m, 0.0);
      val = den > 0.0 ? num / den : 0.0;
    } break;
    default: {  // generalized: M = den, M2 = Q
      const double den = m;
      const double num = fmax(den - 2.0 * a.M2[c], 0.0);
      val = den > 0.0 ? num / den : 0.0;
    } break;
    }
    int64_t idx;
    if (a.full) {
      const int64_t i = k < j ? k : j, jj = k < j ? j : k;
      idx = (int64_t)a.n * i - i * (i + 1) / 2 + (jj - i - 1);
    } else {
      idx = c;
    }
    if (a.out_fp32) ((float *)a.out)[idx] = (float)val;
    else ((double *)a.out)[idx] = val;
  }
}

cudaError_t launch_finalize(const FinalArgs &a, cudaStream_t st) {
  const int64_t total = (a.s1 - a.s0) * (int64_t)a.n;
  if (total <= 0) return cudaSuccess;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_finalize<<<(int)blocks, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace ufg
