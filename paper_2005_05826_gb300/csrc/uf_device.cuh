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

// The FP64 path's fixed point has two words: x * 2^F = hi + lo * 2^-32, hi the
// nearest integer and lo the rounded remainder (|lo| <= 2^31), so one term is
// kept to 2^-(F+32) and a sum of them is still exact integer arithmetic in
// each word (value = (hi + lo * 2^-32) * 2^-F; the words are combined only in
// the finalize).  The FP32 path keeps one word (lo = 0).
struct Fx2 {
  long long hi, lo;
};
constexpr double FX_LO_SCALE = 4294967296.0;  // 2^32
__device__ __forceinline__ Fx2 to_fixed2(double x, double scale) {
  const double y = x * scale;  // exact: scale is a power of two
  const double h = rint(y);
  return Fx2{(long long)h, __double2ll_rn((y - h) * FX_LO_SCALE)};  // y - h is exact
}
__device__ __forceinline__ Fx2 to_fixed2(float x, double scale) { return Fx2{to_fixed(x, scale), 0}; }
__device__ __forceinline__ Fx2 fx_add(Fx2 a, Fx2 b) { return Fx2{a.hi + b.hi, a.lo + b.lo}; }
__device__ __forceinline__ Fx2 fx_sub(Fx2 a, Fx2 b) { return Fx2{a.hi - b.hi, a.lo - b.lo}; }
__device__ __forceinline__ Fx2 fx_mul(Fx2 a, long long m) { return Fx2{a.hi * m, a.lo * m}; }
// the smaller value (|lo| <= 2^31 < 2^32, so hi decides unless equal)
__device__ __forceinline__ Fx2 fx_min(Fx2 a, Fx2 b) {
  return (a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo)) ? a : b;
}

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
