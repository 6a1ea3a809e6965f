// uf_finalize.cu -- stripe accumulators -> distances: the step that, in the
// paper, moves results out of the unified stripe buffer after the branch loop
// (Sec. 2), here with the num / den division in FP64.
//
// Accumulators are int64 fixed point (value * 2^F).  Per cell (stripe s,
// sample k, partner j = (k + s + 1) mod n), with D the diagonal sums and the
// cell holding M = sum min(x_k, x_j) (min form) or A = sum |x_k - x_j|
// (abs form):
//   weighted:    num = A  or  D_k + D_j - 2M,      den = D_k + D_j
//   unweighted:  num = A  or  W_k + W_j - 2G,      den = (W_k + W_j + A) / 2  or  W_k + W_j - G
//                (W = D, G = M on presence embeddings)
//   generalized: num = N (FP64)  or  den - 2Q (FP32)
//   variance-adjusted weighted: num = N, den as generalized (both precisions)
// The unnormalized methods return num * 2^-F.
// num and den are formed exactly in integers before the one FP64 division
// (the common 2^F cancels); weighted_unnormalized returns num * 2^-F.  FP64
// accumulators have two words (uf_device.cuh); they are combined here into
// one 128-bit integer in units of 2^-(F+32).
// A ratio with den == 0 is 0.  An abs-form numerator is a sum of
// nonnegative integers and never negative; a min-form numerator (FP32 only)
// can round a hair below 0 for two nearly identical samples and is then
// raised to 0 (and counted when the caller asks).
// Branches scattered by uf_sparse.cu add their per-sample terms R here: the
// diagonal is D + R, an abs-form cell gains R_k + R_j, and the generalized
// den and N gain R_k + R_j.
#include <algorithm>

#include "uf_internal.h"
#include "uf_finalize.h"

namespace ufg {

// One accumulator word pair as an integer in units of 2^-F (one word) or
// 2^-(F+32) (two words).
template <typename I>
__device__ __forceinline__ I acc_at(const unsigned long long *p, int64_t i, int64_t lo_off) {
  if constexpr (sizeof(I) == 8) {
    return (I)(long long)p[i];
  } else {
    return ((I)(long long)p[i] << 32) + (I)(long long)p[i + lo_off];
  }
}

template <typename I>
__device__ __forceinline__ double to_double(I x) { return (double)x; }

template <typename I>
__global__ void k_finalize(const FinalArgs a) {
  const int64_t rows = a.s1 - a.s0;
  const int64_t total = rows * a.n;
  const double inv_scale = sizeof(I) == 8 ? a.inv_scale : a.inv_scale / 4294967296.0;
  unsigned long long clamped = 0;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < total;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = c / a.n;
    const int k = (int)(c - r * a.n);
    const int64_t s = a.s0 + r;
    int64_t j = k + s + 1;
    if (j >= a.n) j -= a.n;
    if (a.full && 2 * (s + 1) == a.n && k >= a.n / 2) continue;  // duplicate half stripe
    I m = acc_at<I>(a.M, c, a.m_lo_off);
    const bool abs_form = a.method != 3 && abs_row(a.abs_mask, s);
    const I rk = a.Dsp ? acc_at<I>(a.Dsp, k, a.d_lo_off) : I(0), rj = a.Dsp ? acc_at<I>(a.Dsp, j, a.d_lo_off) : I(0);
    const I dk = (a.Dg ? acc_at<I>(a.Dg, k, a.d_lo_off) : I(0)) + rk;
    const I dj = (a.Dg ? acc_at<I>(a.Dg, j, a.d_lo_off) : I(0)) + rj;
    if (abs_form || a.method == 3) m += rk + rj;
    I num;
    double val;
    switch (a.method) {
    case 0: {  // unweighted
      const I w = dk + dj;
      I den2;  // den2 = 2 * den
      if (abs_form) {
        num = m;
        den2 = w + m;
      } else {
        num = w - 2 * m;
        den2 = 2 * (w - m);
      }
      if (num < 0) {
        clamped++;
        num = 0;
      }
      val = den2 > 0 ? 2.0 * to_double(num) / to_double(den2) : 0.0;
    } break;
    case 1: {  // weighted unnormalized
      num = abs_form ? m : dk + dj - 2 * m;
      if (num < 0) {
        clamped++;
        num = 0;
      }
      val = to_double(num) * inv_scale;
    } break;
    case 2: {  // weighted normalized
      const I den = dk + dj;
      num = abs_form ? m : den - 2 * m;
      if (num < 0) {
        clamped++;
        num = 0;
      }
      val = den > 0 ? to_double(num) / to_double(den) : 0.0;
    } break;
    default: {  // generalized: M = den, M2 = N or Q
      const I den = m;
      num = a.gen_abs ? acc_at<I>(a.M2, c, a.m_lo_off) + rk + rj : den - 2 * acc_at<I>(a.M2, c, a.m_lo_off);
      if (num < 0) {
        clamped++;
        num = 0;
      }
      val = den > 0 ? to_double(num) / to_double(den) : 0.0;
    } break;
    }
    if (a.unnormalized) val = to_double(num) * inv_scale;
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
  if (clamped && a.clamps) atomicAdd(a.clamps, clamped);
}

cudaError_t launch_finalize(const FinalArgs &a, cudaStream_t st) {
  const int64_t total = (a.s1 - a.s0) * (int64_t)a.n;
  if (total <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  int64_t blocks = (total + 255) / 256;
  blocks = std::min<int64_t>(blocks, (int64_t)std::max(sms, 1) * 64);  // a grid-stride loop beyond that
  if (a.m_lo_off != 0) k_finalize<__int128><<<(int)blocks, 256, 0, st>>>(a);
  else k_finalize<long long><<<(int)blocks, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace ufg
