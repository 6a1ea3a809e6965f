// uf_stripe.cu -- the Striped UniFrac accumulation (paper Sec. 2-3, Figs. 1-3).
//
// For every branch e of a launch, stripe s and sample k the paper adds
// f(emb_e[k], emb_e[(k + s + 1) mod n]) * length_e into the stripe buffer.
// Here the per-branch term is rewritten so that one accumulator serves three
// methods (exact algebra, stated per method in the finalize kernel):
//   |u - v| = u + v - 2 min(u, v),  [a xor b] = a + b - 2 ab,  [a or b] = a + b - ab,
// so with x = l * u (l * presence for unweighted) every weighted / unweighted
// numerator and denominator follows from
//   M[s][k] = sum_e min(x_e[k], x_e[k + s + 1])   and   D[k] = sum_e x_e[k],
// the latter being the same sum at offset 0.  Generalized UniFrac keeps two
// accumulators, den = sum l s^a and Q = sum l min(u, v) s^(a-1), num = den - 2Q.
//
// Tiling: a CTA owns a TILE_S x TILE_K (stripe x sample) accumulator tile and
// streams all branch rows of the launch through it (the paper's input-buffer
// batching, Sec. 3 Fig. 2, taken to the whole launch): per stage, RB rows of
// the u window [k0, k0 + TILE_K) and the partner window [k0 + s0, k0 + s0 +
// TILE_K + TILE_S) are copied into shared memory with 16-byte cp.async, then
// each thread updates an RD x RK register micro-tile.  Shared rows carry 16
// bytes of padding per 128 bytes so the per-thread 16-byte reads are free of
// bank conflicts.
//
// Precision.  FP64: every update in FP64 into a register partial over B1 = 64
// branches, each partial added into the FP64 global accumulator.  FP32 (the
// paper's fp32 mode, Sec. 4):
// updates in FP32 into a register partial over B1 = 64 branches, partials
// summed into a second FP32 register level, and that level added into the
// FP64 global accumulator every 4096 branches and at the end.  Every cell runs
// the same sequence of operations, so two identical samples produce bitwise
// equal M and D and a distance of exactly 0.
#include <cfloat>

#include "uf_internal.h"

namespace ufg {

namespace {

constexpr int NT = 256;       // threads per CTA: 16 (stripe) x 16 (sample)
constexpr int RB = 8;         // branch rows per pipeline stage
constexpr int NSTAGE = 3;     // cp.async pipeline depth
constexpr int B1 = 64;        // FP32 inner partial length (branches)
constexpr int FLUSH = 4096;   // FP32 outer level length (branches) before the FP64 add

// 16 bytes of padding after every 128 bytes of a shared row
template <typename T>
__host__ __device__ constexpr int skew(int i) {
  return i + (int)(16 / sizeof(T)) * (i / (int)(128 / sizeof(T)));
}

template <typename T, int RD, int RK>
struct Geo {
  static constexpr int TS = 16 * RD;             // stripes per tile
  static constexpr int TK = 16 * RK;             // samples per tile
  static constexpr int VEC = 16 / sizeof(T);     // elements per 16-byte copy
  static constexpr int UW = TK;                  // u window
  static constexpr int VW = TK + TS;             // partner window (needs TK + TS - 1, shifted by one)
  static constexpr int US = skew<T>(UW);
  static constexpr int VS = skew<T>(VW);
  static constexpr int ROW = US + VS;
  static constexpr int STAGE = RB * ROW + RB;    // + the rows' lengths
  static constexpr int UCH = UW / VEC, VCH = VW / VEC, CH = UCH + VCH;
  static constexpr int NV = (RD + RK + VEC - 1) / VEC;  // partner vectors per thread
  static constexpr size_t SMEM = (size_t)NSTAGE * STAGE * sizeof(T);
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <typename T>
__device__ __forceinline__ T tmin(T a, T b);
template <>
__device__ __forceinline__ float tmin<float>(float a, float b) { return fminf(a, b); }
template <>
__device__ __forceinline__ double tmin<double>(double a, double b) { return fmin(a, b); }

// s^(alpha - 1) for s > 0 (the caller discards s == 0 terms)
template <typename T, int MODE>
__device__ __forceinline__ T gen_pow(T s, T am1);
template <>
__device__ __forceinline__ float gen_pow<float, 0>(float s, float) { return rsqrtf(fmaxf(s, 1e-30f)); }
template <>
__device__ __forceinline__ float gen_pow<float, 1>(float s, float am1) { return __powf(fmaxf(s, 1e-30f), am1); }
template <>
__device__ __forceinline__ double gen_pow<double, 0>(double s, double) { return rsqrt(fmax(s, 1e-300)); }
template <>
__device__ __forceinline__ double gen_pow<double, 1>(double s, double am1) { return pow(fmax(s, 1e-300), am1); }

// Stage loader: RB branch rows [e0, e0 + RB) of the u and partner windows.
template <typename T, int RD, int RK, bool LEN>
__device__ __forceinline__ void load_stage(T *stage, const StripeArgs &a, int e0, int k0, int s0) {
  using G = Geo<T, RD, RK>;
  const T *X = (const T *)a.X;
  for (int c = threadIdx.x; c < RB * G::CH; c += NT) {
    const int r = c / G::CH, q = c - r * G::CH;
    T *row = stage + r * G::ROW;
    const int e = e0 + r;
    T *dst;
    int64_t src;
    if (q < G::UCH) {
      dst = row + skew<T>(q * G::VEC);
      src = (int64_t)k0 + q * G::VEC;
    } else {
      const int qv = q - G::UCH;
      dst = row + G::US + skew<T>(qv * G::VEC);
      src = (int64_t)k0 + s0 + qv * G::VEC;
    }
    if (e < a.rows) {
      cp_async16(dst, X + (int64_t)e * a.pitch + src);
    } else {
#pragma unroll
      for (int i = 0; i < G::VEC; i++) dst[i] = T(0);
    }
  }
  if (LEN && threadIdx.x < RB) {
    const int e = e0 + threadIdx.x;
    stage[RB * G::ROW + threadIdx.x] = e < a.rows ? (T)a.len[e] : T(0);
  }
}

// Add a thread's FP32/FP64 cell values into the global FP64 stripe accumulator.
template <int RD, int RK, typename V>
__device__ __forceinline__ void flush_cells(double *M, const V (&val)[RD][RK], const StripeArgs &a,
                                            int s_base, int k_base) {
#pragma unroll
  for (int i = 0; i < RD; i++) {
    const int s = s_base + i;
    if (s < a.s_lo || s > a.s_hi) continue;
    double *row = M + (int64_t)(s - a.s_lo) * a.n;
#pragma unroll
    for (int j = 0; j < RK; j++) {
      const int k = k_base + j;
      if (k < a.n) row[k] += (double)val[i][j];
    }
  }
}

// ---- weighted / unweighted: M[s][k] += sum_e min(x_e[k], x_e[k + s + 1]) ----
template <typename T, int RD, int RK>
__global__ void __launch_bounds__(NT, 1) k_stripe_min(const StripeArgs a) {
  using G = Geo<T, RD, RK>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *smem = reinterpret_cast<T *>(smem_raw);
  const int k0 = blockIdx.x * G::TK;
  const int s0 = (a.m_lo + blockIdx.y) * G::TS;
  const int tk = threadIdx.x & 15, ts = threadIdx.x >> 4;
  const int uoff = skew<T>(RK * tk);
  const int w0 = RK * tk + RD * ts;  // partner window of this thread, used from w0 + 1

  constexpr bool F32 = sizeof(T) == 4;
  T acc[RD][RK];
  float mid[RD][RK];
#pragma unroll
  for (int i = 0; i < RD; i++)
#pragma unroll
    for (int j = 0; j < RK; j++) {
      acc[i][j] = T(0);
      mid[i][j] = 0.f;
    }

  const int nst = (a.rows + RB - 1) / RB;
#pragma unroll
  for (int p = 0; p < NSTAGE - 1; p++) {
    if (p < nst) load_stage<T, RD, RK, false>(smem + p * G::STAGE, a, p * RB, k0, s0);
    cp_async_commit();
  }
  int in_sub = 0, in_flush = 0;
  for (int it = 0; it < nst; it++) {
    cp_async_wait<NSTAGE - 2>();
    __syncthreads();
    {
      const int nx = it + NSTAGE - 1;
      if (nx < nst) load_stage<T, RD, RK, false>(smem + (nx % NSTAGE) * G::STAGE, a, nx * RB, k0, s0);
      cp_async_commit();
    }
    const T *stage = smem + (it % NSTAGE) * G::STAGE;
#pragma unroll 2
    for (int r = 0; r < RB; r++) {
      const T *urow = stage + r * G::ROW;
      const T *vrow = urow + G::US;
      T u[RK], v[G::NV * G::VEC];
#pragma unroll
      for (int q = 0; q < RK / G::VEC; q++)
        *reinterpret_cast<uint4 *>(&u[q * G::VEC]) =
            *reinterpret_cast<const uint4 *>(urow + uoff + q * G::VEC);
#pragma unroll
      for (int q = 0; q < G::NV; q++)
        *reinterpret_cast<uint4 *>(&v[q * G::VEC]) =
            *reinterpret_cast<const uint4 *>(vrow + skew<T>(w0 + q * G::VEC));
#pragma unroll
      for (int i = 0; i < RD; i++)
#pragma unroll
        for (int j = 0; j < RK; j++) acc[i][j] += tmin<T>(u[j], v[i + j + 1]);
    }
    in_sub += RB;
    in_flush += RB;
    if (F32) {
      if (in_sub == B1 || it == nst - 1) {
#pragma unroll
        for (int i = 0; i < RD; i++)
#pragma unroll
          for (int j = 0; j < RK; j++) {
            mid[i][j] += (float)acc[i][j];
            acc[i][j] = T(0);
          }
        in_sub = 0;
      }
      if (in_flush == FLUSH || it == nst - 1) {
        flush_cells<RD, RK>(a.M, mid, a, s0 + RD * ts, k0 + RK * tk);
#pragma unroll
        for (int i = 0; i < RD; i++)
#pragma unroll
          for (int j = 0; j < RK; j++) mid[i][j] = 0.f;
        in_flush = 0;
      }
    } else if (in_sub == B1 || it == nst - 1) {
      flush_cells<RD, RK>(a.M, acc, a, s0 + RD * ts, k0 + RK * tk);
#pragma unroll
      for (int i = 0; i < RD; i++)
#pragma unroll
        for (int j = 0; j < RK; j++) acc[i][j] = T(0);
      in_sub = 0;
    }
  }
  cp_async_wait<0>();
}

// ---- diagonal: D[k] += sum_e x_e[k], with the same operation sequence as
//      k_stripe_min applies to a cell whose two columns are equal ----
// Phase 1: one partial per (B1-row sub-block, sample), summed in row order.
template <typename T>
__global__ void k_diag_partial(const StripeArgs a, T *__restrict__ part) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.n) return;
  const int sb = blockIdx.y;
  const T *X = (const T *)a.X;
  const int e0 = sb * B1, e1 = min(a.rows, e0 + B1);
  T acc = T(0);
  for (int e = e0; e < e1; e++) {
    const T x = X[(int64_t)e * a.pitch + k];
    acc += tmin<T>(x, x);
  }
  part[(int64_t)sb * a.n + k] = acc;
}

// Phase 2: sub-block partials in order -- FP32: into an FP32 level added to
// the FP64 diagonal every FLUSH rows; FP64: each partial into the diagonal.
template <typename T>
__global__ void k_diag_reduce(const StripeArgs a, const T *__restrict__ part, int n_sb) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.n) return;
  constexpr bool F32 = sizeof(T) == 4;
  double d = a.Dg[k];
  float mid = 0.f;
  for (int sb = 0; sb < n_sb; sb++) {
    const T p = part[(int64_t)sb * a.n + k];
    if (F32) {
      mid += (float)p;
      if ((sb + 1) % (FLUSH / B1) == 0 || sb == n_sb - 1) {
        d += (double)mid;
        mid = 0.f;
      }
    } else {
      d += (double)p;
    }
  }
  a.Dg[k] = d;
}

// ---- generalized: den += l s w, Q += l min(u, v) w, w = s^(alpha - 1) ----
template <typename T, int RD, int RK, int MODE>
__global__ void __launch_bounds__(NT, 1) k_stripe_gen(const StripeArgs a) {
  using G = Geo<T, RD, RK>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *smem = reinterpret_cast<T *>(smem_raw);
  const int k0 = blockIdx.x * G::TK;
  const int s0 = (a.m_lo + blockIdx.y) * G::TS;
  const int tk = threadIdx.x & 15, ts = threadIdx.x >> 4;
  const int uoff = skew<T>(RK * tk);
  const int w0 = RK * tk + RD * ts;
  const T am1 = (T)(a.alpha - 1.0);

  constexpr bool F32 = sizeof(T) == 4;
  T accd[RD][RK], accq[RD][RK];
  float midd[RD][RK], midq[RD][RK];
#pragma unroll
  for (int i = 0; i < RD; i++)
#pragma unroll
    for (int j = 0; j < RK; j++) {
      accd[i][j] = accq[i][j] = T(0);
      midd[i][j] = midq[i][j] = 0.f;
    }
  const int nst = (a.rows + RB - 1) / RB;
#pragma unroll
  for (int p = 0; p < NSTAGE - 1; p++) {
    if (p < nst) load_stage<T, RD, RK, true>(smem + p * G::STAGE, a, p * RB, k0, s0);
    cp_async_commit();
  }
  int in_sub = 0, in_flush = 0;
  for (int it = 0; it < nst; it++) {
    cp_async_wait<NSTAGE - 2>();
    __syncthreads();
    {
      const int nx = it + NSTAGE - 1;
      if (nx < nst) load_stage<T, RD, RK, true>(smem + (nx % NSTAGE) * G::STAGE, a, nx * RB, k0, s0);
      cp_async_commit();
    }
    const T *stage = smem + (it % NSTAGE) * G::STAGE;
#pragma unroll 1
    for (int r = 0; r < RB; r++) {
      const T *urow = stage + r * G::ROW;
      const T *vrow = urow + G::US;
      const T l = stage[RB * G::ROW + r];
      T u[RK], v[G::NV * G::VEC];
#pragma unroll
      for (int q = 0; q < RK / G::VEC; q++)
        *reinterpret_cast<uint4 *>(&u[q * G::VEC]) =
            *reinterpret_cast<const uint4 *>(urow + uoff + q * G::VEC);
#pragma unroll
      for (int q = 0; q < G::NV; q++)
        *reinterpret_cast<uint4 *>(&v[q * G::VEC]) =
            *reinterpret_cast<const uint4 *>(vrow + skew<T>(w0 + q * G::VEC));
#pragma unroll
      for (int i = 0; i < RD; i++)
#pragma unroll
        for (int j = 0; j < RK; j++) {
          const T uu = u[j], vv = v[i + j + 1];
          const T s = uu + vv;
          T w = l * gen_pow<T, MODE>(s, am1);
          if (MODE == 1) w = s > T(0) ? w : T(0);
          accd[i][j] = fma(s, w, accd[i][j]);
          accq[i][j] = fma(tmin<T>(uu, vv), w, accq[i][j]);
        }
    }
    if (F32) {
      in_sub += RB;
      in_flush += RB;
      if (in_sub == B1 || it == nst - 1) {
#pragma unroll
        for (int i = 0; i < RD; i++)
#pragma unroll
          for (int j = 0; j < RK; j++) {
            midd[i][j] += (float)accd[i][j];
            midq[i][j] += (float)accq[i][j];
            accd[i][j] = accq[i][j] = T(0);
          }
        in_sub = 0;
      }
      if (in_flush == FLUSH || it == nst - 1) {
        flush_cells<RD, RK>(a.M, midd, a, s0 + RD * ts, k0 + RK * tk);
        flush_cells<RD, RK>(a.M2, midq, a, s0 + RD * ts, k0 + RK * tk);
#pragma unroll
        for (int i = 0; i < RD; i++)
#pragma unroll
          for (int j = 0; j < RK; j++) midd[i][j] = midq[i][j] = 0.f;
        in_flush = 0;
      }
    }
  }
  cp_async_wait<0>();
  if (!F32) {
    flush_cells<RD, RK>(a.M, accd, a, s0 + RD * ts, k0 + RK * tk);
    flush_cells<RD, RK>(a.M2, accq, a, s0 + RD * ts, k0 + RK * tk);
  }
}

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T, int RD, int RK>
cudaError_t run_min(const StripeArgs &a, cudaStream_t st) {
  using G = Geo<T, RD, RK>;
  cudaError_t e = set_smem(k_stripe_min<T, RD, RK>, G::SMEM);
  if (e != cudaSuccess) return e;
  dim3 grid((a.n + G::TK - 1) / G::TK, a.m_hi - a.m_lo + 1);
  k_stripe_min<T, RD, RK><<<grid, NT, G::SMEM, st>>>(a);
  return cudaGetLastError();
}

template <typename T, int RD, int RK, int MODE>
cudaError_t run_gen(const StripeArgs &a, cudaStream_t st) {
  using G = Geo<T, RD, RK>;
  cudaError_t e = set_smem(k_stripe_gen<T, RD, RK, MODE>, G::SMEM);
  if (e != cudaSuccess) return e;
  dim3 grid((a.n + G::TK - 1) / G::TK, a.m_hi - a.m_lo + 1);
  k_stripe_gen<T, RD, RK, MODE><<<grid, NT, G::SMEM, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

// micro-tiles: min kernels 8 x 8, generalized 4 x 8 (two accumulators)
void stripe_tile_shape(int acc, bool fp32, int *tile_s, int *tile_k) {
  (void)fp32;
  *tile_s = acc == ACC_GEN ? 16 * 4 : 16 * 8;
  *tile_k = 16 * 8;
}

cudaError_t launch_stripe_acc(int acc, bool fp32, const StripeArgs &a, cudaStream_t st) {
  if (a.rows <= 0 || a.m_hi < a.m_lo) return cudaSuccess;
  if (acc == ACC_MIN) return fp32 ? run_min<float, 8, 8>(a, st) : run_min<double, 8, 8>(a, st);
  const bool half = a.alpha == 0.5;
  if (fp32) return half ? run_gen<float, 4, 8, 0>(a, st) : run_gen<float, 4, 8, 1>(a, st);
  return half ? run_gen<double, 4, 8, 0>(a, st) : run_gen<double, 4, 8, 1>(a, st);
}

size_t diag_scratch_bytes(bool fp32, int rows, int n) {
  const int64_t n_sb = (rows + B1 - 1) / B1;
  return (size_t)n_sb * n * (fp32 ? 4 : 8);
}

cudaError_t launch_diag(bool fp32, const StripeArgs &a, void *scratch, cudaStream_t st) {
  if (a.rows <= 0) return cudaSuccess;
  const int n_sb = (a.rows + B1 - 1) / B1;
  dim3 g1((a.n + 127) / 128, n_sb);
  const int g2 = (a.n + 127) / 128;
  if (fp32) {
    k_diag_partial<float><<<g1, 128, 0, st>>>(a, (float *)scratch);
    k_diag_reduce<float><<<g2, 128, 0, st>>>(a, (const float *)scratch, n_sb);
  } else {
    k_diag_partial<double><<<g1, 128, 0, st>>>(a, (double *)scratch);
    k_diag_reduce<double><<<g2, 128, 0, st>>>(a, (const double *)scratch, n_sb);
  }
  return cudaGetLastError();
}

}  // namespace ufg
