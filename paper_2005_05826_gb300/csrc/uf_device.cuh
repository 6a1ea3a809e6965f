// uf_device.cuh -- device helpers shared by the dense stripe kernels
// (uf_stripe.cu) and the sparse-row pair kernels (uf_sparse.cu), so that both
// take the same per-branch values and the same fixed-point rounding.
#pragma once
#include <cuda_runtime.h>

#include "uf_internal.h"

namespace ufg {

template <typename T>
__device__ __forceinline__ T tmin(T a, T b);
template <>
__device__ __forceinline__ float tmin<float>(float a, float b) { return fminf(a, b); }
template <>
__device__ __forceinline__ double tmin<double>(double a, double b) { return fmin(a, b); }

// FP64 s^(alpha - 1) for s > 0 (s == 0 terms are zeroed by the caller)
template <typename T, int MODE>
__device__ __forceinline__ T gen_pow(T s, T am1);
template <>
__device__ __forceinline__ double gen_pow<double, 0>(double s, double) { return rsqrt(fmax(s, 1e-300)); }
template <>
__device__ __forceinline__ double gen_pow<double, 1>(double s, double am1) { return pow(fmax(s, 1e-300), am1); }

// s^(alpha - 1) on the SFU for FP32 s >= 1e-30 (never denormal):
// MODE 0 (alpha = 1/2) one reciprocal square root; MODE 1 exp2((alpha - 1) log2 s).
template <int MODE>
__device__ __forceinline__ float sfu_pow(float s, float am1) {
  float r;
  if (MODE == 0) {
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(s));
  } else {
    float lg;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(lg) : "f"(s));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(lg * am1));
  }
  return r;
}

// fixed point: round x * 2^F to the nearest integer
__device__ __forceinline__ long long to_fixed(float x, double scale) { return __float2ll_rn(x * (float)scale); }
__device__ __forceinline__ long long to_fixed(double x, double scale) { return __double2ll_rn(x * scale); }

// Embedding value of one sample at one branch from its count sum c under the
// branch, the branch length l and the sample total t (1 / t in FP32 as it).
template <typename T, int KIND>
__device__ __forceinline__ T emb_value(double c, double l, double total, float inv_total_f);

template <>
__device__ __forceinline__ double emb_value<double, EMB_SCALED>(double c, double l, double t, float) {
  return l * (c / t);
}
template <>
__device__ __forceinline__ double emb_value<double, EMB_PRESENCE>(double c, double l, double, float) {
  return c > 0.0 ? l : 0.0;
}
template <>
__device__ __forceinline__ double emb_value<double, EMB_PROP>(double c, double, double t, float) {
  return c / t;
}
template <>
__device__ __forceinline__ float emb_value<float, EMB_SCALED>(double c, double l, double, float it) {
  return (float)c * ((float)l * it);
}
template <>
__device__ __forceinline__ float emb_value<float, EMB_PRESENCE>(double c, double l, double, float) {
  return c > 0.0 ? (float)l : 0.0f;
}
// FP32 proportions carry a 1e-30 offset: it leaves every nonzero FP32
// proportion unchanged (all are far above 1e-30 * 2^24) and keeps the
// generalized kernel's s = u + v away from 0 without a guard per update.
template <>
__device__ __forceinline__ float emb_value<float, EMB_PROP>(double c, double, double, float it) {
  return (float)c * it + 1e-30f;
}

}  // namespace ufg
