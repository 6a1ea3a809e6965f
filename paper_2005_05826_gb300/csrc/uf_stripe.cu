// uf_stripe.cu -- the Striped UniFrac accumulation (paper Sec. 2-3, Figs. 1-3).
//
// For every branch e of a launch, stripe s and sample k the paper adds
// f(emb_e[k], emb_e[(k + s + 1) mod n]) * length_e into the stripe buffer.
// Here the per-branch term is rewritten (exact algebra; the finalize kernel
// states it per method):
//   |u - v| = u + v - 2 min(u, v),  [a xor b] = a + b - 2 ab,  [a or b] = a + b - ab,
// so with x = l * u (l * presence for unweighted) every weighted and
// unweighted numerator and denominator follows from the diagonal
// D[k] = sum_e x_e[k] and, per cell, either
//   M[s][k] = sum_e min(x_e[k], x_e[k + s + 1])        (min form) or
//   A[s][k] = sum_e |x_e[k] - x_e[k + s + 1]|          (abs form).
// One min-form update is one FMNMX (ALU pipe, half rate) plus half an FADD2;
// one abs-form update is half an FSUB2 plus one FADD (FMA pipe).  The FP32
// kernel gives stripes 1, 3, 5 and 7 of every 8 the abs form so the two pipes
// share the load (odd micro-tile rows read their partner pairs at even,
// register-pair aligned offsets).  The FP64 kernel uses the abs form on every
// stripe: its numerators are then sums of nonnegative terms, never a
// difference of two nearly equal sums, so their error stays relative to the
// distance however close two samples are.  Generalized UniFrac keeps two
// accumulators, den = sum l s^a and, FP32, Q = sum l min(u, v) s^(a-1) with
// num = den - 2Q or, FP64, N = sum l |u - v| s^(a-1) = num.
//
// Work is split into units (row chunk of up to a.chunk branches, tile of
// TILE_S stripes x TILE_K samples).  Persistent CTAs take units from a global
// counter, chunk-major, so the CTAs in flight read the same rows and those
// rows stay in L2.  Per unit, stages of rows (FP32: 16 rows, two stages;
// FP64: 8 rows, three stages) of the u window [k0, k0 + TILE_K) and the
// partner window [k0 + s0, k0 + s0 + TILE_K + TILE_S) go to shared memory by
// 16-byte cp.async while the previous stage is computed, and each thread
// updates an RD x RK register micro-tile.  Shared rows are XOR-swizzled in
// 16-byte units so the per-thread 16-byte reads are free of bank conflicts.
//
// Precision.  Register partials over B1 = 64 branches are summed into a
// second level kept in shared memory in the path's own precision (FP32 for
// the paper's fp32 mode, Sec. 4, FP64 otherwise); at the end of the unit that
// level is scaled by 2^F and rounded once to an int64 fixed-point value (FP64:
// two words, the second holding the remainder at 2^-32 of the first's step),
// which is added atomically into the int64 accumulator.  Integer addition is
// exact and order-free, so chunks may land in any order and the result is
// still deterministic; every cell (and the diagonal) runs the same FP32 /
// FP64 operation sequence within a unit, so two identical samples give
// bitwise equal accumulators and a distance of exactly 0 (an abs-form cell
// adds |x - x| = 0 exactly).
// F is chosen by the host from an upper bound B on any accumulated value so
// that 2 B 2^F <= 2^61.
#include <algorithm>
#include <cfloat>
#include <type_traits>

#include "uf_device.cuh"

namespace ufg {

namespace {

constexpr int NT = 256;       // threads per CTA: 16 (stripe) x 16 (sample)
constexpr int B1 = 64;        // inner partial length (branches)

// Shared rows are stored in 16-byte units with unit j placed at
// j ^ ((j >> 3) & MASK), MASK = (bytes a thread reads per 8-sample run) / 16 - 1.
// Eight threads that read the same unit offset q of consecutive 8-sample runs
// (any starting run) then hit eight distinct 16-byte bank groups.
template <typename T>
__host__ __device__ constexpr int swz(int elem) {
  constexpr int VEC = 16 / sizeof(T);
  constexpr int MASK = 8 * sizeof(T) / 16 - 1;
  const int j = elem / VEC;
  return (j ^ ((j >> 3) & MASK)) * VEC + elem % VEC;
}

template <typename T, int RD, int RK, int NACC>
struct Geo {
  // branch rows per pipeline stage and cp.async stages: FP32 16 rows in two
  // stages (half the block barriers of 8-row stages), FP64 8 rows in three
  static constexpr int RB = sizeof(T) == 4 ? 16 : 8;
  static constexpr int NSTAGE = sizeof(T) == 4 ? 2 : 3;
  static constexpr int TS = 16 * RD;             // stripes per tile
  static constexpr int TK = 16 * RK;             // samples per tile
  static constexpr int VEC = 16 / sizeof(T);     // elements per 16-byte copy
  static constexpr int UW = TK;                  // u window
  static constexpr int VW = TK + TS;             // partner window (needs TK + TS - 1, shifted by one)
  static constexpr int ROW = UW + VW;            // both parts are multiples of 128 bytes
  static constexpr int STAGE = RB * ROW + RB;    // + the rows' lengths (keeps 16-byte alignment)
  static constexpr int UCH = UW / VEC, VCH = VW / VEC, CH = UCH + VCH;
  static constexpr int NV = (RD + RK + VEC - 1) / VEC;  // partner vectors per thread
  // second level per thread and cell, in the path's precision
  using Mid = T;
  static constexpr size_t SMEM =
      (size_t)NSTAGE * STAGE * sizeof(T) + (size_t)NACC * RD * RK * NT * sizeof(Mid);
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// a - b on a register pair (one packed FP32 subtract)
__device__ __forceinline__ float2 fsub2(float2 a, float2 b) {
  unsigned long long ra, rb, rr;
  asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rr) : "l"(ra), "l"(rb));
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(rr));
  return r;
}

struct Unit {
  int r0, r1;       // branch rows
  int k0, s0;       // tile origin: first sample, first stripe
  int n, s_lo, s_hi;
  int64_t x_col;    // the table's first column in an embedding row
  int64_t m_off;    // the table's first accumulator cell
};

// Table holding tile number tt of the batch (tables in order of tile0).
__device__ __forceinline__ int table_of_tile(const TabDesc *tabs, int n_tabs, int tt) {
  int lo = 0, hi = n_tabs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tabs[mid].tile0 <= tt) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Next work unit for this CTA: chunk-major over (row chunk, tile of any table).
__device__ __forceinline__ bool next_unit(const StripeArgs &a, int tile_s, int tile_k, int *s_unit,
                                          Unit *u) {
  __syncthreads();  // everyone is done with the previous unit's shared data
  if (threadIdx.x == 0) *s_unit = atomicAdd(a.counter, 1);
  __syncthreads();
  const int id = *s_unit;
  const int n_chunks = (a.rows + a.chunk - 1) / a.chunk;
  if (id >= n_chunks * a.n_tiles) return false;
  const int c = id / a.n_tiles, tt = id - c * a.n_tiles;
  const TabDesc &tb = a.tabs[a.n_tabs == 1 ? 0 : table_of_tile(a.tabs, a.n_tabs, tt)];
  const int t = tt - tb.tile0;
  // bands of kband sample tiles: all stripe tiles of a band, then the next band
  const int n_st = tb.m_hi - tb.m_lo + 1;
  const int kb = max(1, min(tb.kband, tb.n_ktiles));
  const int band = t / (kb * n_st), within = t - band * (kb * n_st);
  const int width = min(kb, tb.n_ktiles - band * kb);
  const int kt = band * kb + within % width, st = within / width;
  u->r0 = c * a.chunk;
  u->r1 = min(a.rows, u->r0 + a.chunk);
  u->k0 = kt * tile_k;
  u->s0 = (tb.m_lo + st) * tile_s;
  u->n = tb.n;
  u->s_lo = tb.s_lo;
  u->s_hi = tb.s_hi;
  u->x_col = tb.x_col;
  u->m_off = tb.m_off;
  return true;
}

// Stage loader: G::RB branch rows [e0, e0 + G::RB) of the u window (columns from
// ucol) and the partner window (columns from vcol).
template <typename T, int RD, int RK, int NACC, bool LEN>
__device__ __forceinline__ void load_stage(T *stage, const StripeArgs &a, int e0, int e_end, int64_t ucol,
                                           int64_t vcol) {
  using G = Geo<T, RD, RK, NACC>;
  const T *X = (const T *)a.X;
  for (int c = threadIdx.x; c < G::RB * G::CH; c += NT) {
    const int r = c / G::CH, q = c - r * G::CH;
    T *row = stage + r * G::ROW;
    const int e = e0 + r;
    T *dst;
    int64_t src;
    if (q < G::UCH) {
      dst = row + swz<T>(q * G::VEC);
      src = ucol + q * G::VEC;
    } else {
      const int qv = q - G::UCH;
      dst = row + G::UW + swz<T>(qv * G::VEC);
      src = vcol + qv * G::VEC;
    }
    if (e < e_end) {
      cp_async16(dst, X + (int64_t)e * a.pitch + src);
    } else {
      // rows past the unit: zero, or for FP32 proportions the embedding's
      // 1e-30 floor (their length is 0, so they add nothing either way)
      const T pad = (LEN && sizeof(T) == 4) ? T(1e-30f) : T(0);
#pragma unroll
      for (int i = 0; i < G::VEC; i++) dst[i] = pad;
    }
  }
  if (LEN && threadIdx.x < G::RB) {
    const int e = e0 + threadIdx.x;
    stage[G::RB * G::ROW + threadIdx.x] = e < e_end ? (T)a.len[e] : T(0);
  }
}

// Add one thread's second-level cells (fixed point) into the accumulator.
template <typename T, int RD, int RK, typename Mid>
__device__ __forceinline__ void commit_cells(unsigned long long *M, const Mid *mid, const StripeArgs &a,
                                             const Unit &U, int s_base, int k_base) {
#pragma unroll
  for (int i = 0; i < RD; i++) {
    const int s = s_base + i;
    if (s < U.s_lo || s > U.s_hi) continue;
    unsigned long long *row = M + U.m_off + (int64_t)(s - U.s_lo) * U.n;
#pragma unroll
    for (int j = 0; j < RK; j++) {
      const int k = k_base + j;
      if (k < U.n) {
        const Fx2 q = to_fixed2(mid[(i * RK + j) * NT + threadIdx.x], a.scale);
        atomicAdd(row + k, (unsigned long long)q.hi);
        if constexpr (sizeof(T) == 8) atomicAdd(row + k + a.m_lo_off, (unsigned long long)q.lo);
      }
    }
  }
}

// ---- weighted / unweighted ----
// rows i of the micro-tile with bit i of ABSM clear: M += min(x_k, x_j);
// with it set: A += |x_k - x_j|
template <typename T, int RD, int RK, unsigned ABSM, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_stripe_min(const StripeArgs a) {
  using G = Geo<T, RD, RK, 1>;
  using Mid = typename G::Mid;
  constexpr bool F32 = sizeof(T) == 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *stg = reinterpret_cast<T *>(smem_raw);
  Mid *mid = reinterpret_cast<Mid *>(smem_raw + (size_t)G::NSTAGE * G::STAGE * sizeof(T));
  __shared__ int s_unit;
  const int tk = threadIdx.x & 15, ts = threadIdx.x >> 4;
  const int w0 = RK * tk + RD * ts;  // partner window of this thread, used from w0 + 1
  Unit U;
  while (next_unit(a, G::TS, G::TK, &s_unit, &U)) {
#pragma unroll
    for (int c = 0; c < RD * RK; c++) mid[c * NT + threadIdx.x] = Mid(0);
    const int nst = (U.r1 - U.r0 + G::RB - 1) / G::RB;
#pragma unroll
    for (int p = 0; p < G::NSTAGE - 1; p++) {
      if (p < nst) load_stage<T, RD, RK, 1, false>(stg + p * G::STAGE, a, U.r0 + p * G::RB, U.r1, U.x_col + U.k0,
                                        U.x_col + U.k0 + U.s0);
      cp_async_commit();
    }
    T acc[RD][RK];
#pragma unroll
    for (int i = 0; i < RD; i++)
#pragma unroll
      for (int j = 0; j < RK; j++) acc[i][j] = T(0);
    int in_sub = 0;
    for (int it = 0; it < nst; it++) {
      cp_async_wait<G::NSTAGE - 2>();
      __syncthreads();
      {
        const int nx = it + G::NSTAGE - 1;
        if (nx < nst)
          load_stage<T, RD, RK, 1, false>(stg + (nx % G::NSTAGE) * G::STAGE, a, U.r0 + nx * G::RB, U.r1,
                                          U.x_col + U.k0, U.x_col + U.k0 + U.s0);
        cp_async_commit();
      }
      const T *stage = stg + (it % G::NSTAGE) * G::STAGE;
      // the whole stage unrolled: 3 % faster than two rows per iteration in
      // a micro-benchmark of the FP32 kernel (fewer loop and address
      // instructions, more freedom to interleave the ALU and FMA pipes)
#pragma unroll
      for (int r = 0; r < G::RB; r++) {
        const T *urow = stage + r * G::ROW;
        const T *vrow = urow + G::UW;
        T u[RK], v[G::NV * G::VEC];
#pragma unroll
        for (int q = 0; q < RK / G::VEC; q++)
          *reinterpret_cast<uint4 *>(&u[q * G::VEC]) =
              *reinterpret_cast<const uint4 *>(urow + swz<T>(RK * tk + q * G::VEC));
#pragma unroll
        for (int q = 0; q < G::NV; q++)
          *reinterpret_cast<uint4 *>(&v[q * G::VEC]) =
              *reinterpret_cast<const uint4 *>(vrow + swz<T>(w0 + q * G::VEC));
        if constexpr (F32) {
#pragma unroll
          for (int i = 0; i < RD; i++)
#pragma unroll
            for (int j = 0; j < RK; j += 2) {
              if (!((ABSM >> i) & 1u)) {  // two mins, one paired add
                float2 a2 = make_float2(acc[i][j], acc[i][j + 1]);
                const float2 m2 = make_float2(fminf(u[j], v[i + j + 1]), fminf(u[j + 1], v[i + j + 2]));
                a2 = __fadd2_rn(a2, m2);
                acc[i][j] = a2.x;
                acc[i][j + 1] = a2.y;
              } else {  // one paired difference, one paired add of absolute values
                const float2 d2 = fsub2(make_float2(u[j], u[j + 1]), make_float2(v[i + j + 1], v[i + j + 2]));
                float2 a2 = make_float2(acc[i][j], acc[i][j + 1]);
                a2 = __fadd2_rn(a2, make_float2(fabsf(d2.x), fabsf(d2.y)));
                acc[i][j] = a2.x;
                acc[i][j + 1] = a2.y;
              }
            }
        } else {
#pragma unroll
          for (int i = 0; i < RD; i++)
#pragma unroll
            for (int j = 0; j < RK; j++) {
              if ((ABSM >> i) & 1u) acc[i][j] += fabs(u[j] - v[i + j + 1]);
              else acc[i][j] += tmin<T>(u[j], v[i + j + 1]);
            }
        }
      }
      in_sub += G::RB;
      if (in_sub == B1 || it == nst - 1) {
#pragma unroll
        for (int i = 0; i < RD; i++)
#pragma unroll
          for (int j = 0; j < RK; j++) {
            mid[(i * RK + j) * NT + threadIdx.x] += acc[i][j];
            acc[i][j] = T(0);
          }
        in_sub = 0;
      }
    }
    cp_async_wait<0>();
    commit_cells<T, RD, RK>(a.M, mid, a, U, U.s0 + RD * ts, U.k0 + RK * tk);
  }
}

// ---- generalized: den += l s w and, FP32, Q += l min(u, v) w or, FP64,
//      N += l |u - v| w, with w = s^(alpha - 1) ----
template <typename T, int RD, int RK, int MODE, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_stripe_gen(const StripeArgs a) {
  using G = Geo<T, RD, RK, 2>;
  using Mid = typename G::Mid;
  constexpr bool F32 = sizeof(T) == 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *stg = reinterpret_cast<T *>(smem_raw);
  Mid *midd = reinterpret_cast<Mid *>(smem_raw + (size_t)G::NSTAGE * G::STAGE * sizeof(T));
  Mid *midq = midd + RD * RK * NT;
  __shared__ int s_unit;
  const int tk = threadIdx.x & 15, ts = threadIdx.x >> 4;
  const int w0 = RK * tk + RD * ts;
  const T am1 = (T)(a.alpha - 1.0);
  Unit U;
  while (next_unit(a, G::TS, G::TK, &s_unit, &U)) {
#pragma unroll
    for (int c = 0; c < RD * RK; c++) midd[c * NT + threadIdx.x] = midq[c * NT + threadIdx.x] = Mid(0);
    const int nst = (U.r1 - U.r0 + G::RB - 1) / G::RB;
#pragma unroll
    for (int p = 0; p < G::NSTAGE - 1; p++) {
      if (p < nst) load_stage<T, RD, RK, 2, true>(stg + p * G::STAGE, a, U.r0 + p * G::RB, U.r1, U.x_col + U.k0,
                                       U.x_col + U.k0 + U.s0);
      cp_async_commit();
    }
    T accd[RD][RK], accq[RD][RK];
#pragma unroll
    for (int i = 0; i < RD; i++)
#pragma unroll
      for (int j = 0; j < RK; j++) accd[i][j] = accq[i][j] = T(0);
    int in_sub = 0;
    for (int it = 0; it < nst; it++) {
      cp_async_wait<G::NSTAGE - 2>();
      __syncthreads();
      {
        const int nx = it + G::NSTAGE - 1;
        if (nx < nst)
          load_stage<T, RD, RK, 2, true>(stg + (nx % G::NSTAGE) * G::STAGE, a, U.r0 + nx * G::RB, U.r1,
                                         U.x_col + U.k0, U.x_col + U.k0 + U.s0);
        cp_async_commit();
      }
      const T *stage = stg + (it % G::NSTAGE) * G::STAGE;
#pragma unroll 1
      for (int r = 0; r < G::RB; r++) {
        const T *urow = stage + r * G::ROW;
        const T *vrow = urow + G::UW;
        const T l = stage[G::RB * G::ROW + r];
        T u[RK], v[G::NV * G::VEC];
#pragma unroll
        for (int q = 0; q < RK / G::VEC; q++)
          *reinterpret_cast<uint4 *>(&u[q * G::VEC]) =
              *reinterpret_cast<const uint4 *>(urow + swz<T>(RK * tk + q * G::VEC));
#pragma unroll
        for (int q = 0; q < G::NV; q++)
          *reinterpret_cast<uint4 *>(&v[q * G::VEC]) =
              *reinterpret_cast<const uint4 *>(vrow + swz<T>(w0 + q * G::VEC));
        if constexpr (F32) {
          // pairs of cells per f32x2 instruction; the embedding keeps every
          // proportion >= 1e-30 (an offset no nonzero FP32 proportion can see),
          // so s > 0: for alpha = 1/2 an absent pair adds l sqrt(2e-30) to den
          // and exactly half of that to Q (net 0 to num), for other alpha its
          // term is zeroed explicitly
          const float2 l2 = make_float2(l, l);
#pragma unroll
          for (int i = 0; i < RD; i++)
#pragma unroll
            for (int j = 0; j < RK; j += 2) {
              const float2 uu = make_float2(u[j], u[j + 1]);
              const float2 vv = make_float2(v[i + j + 1], v[i + j + 2]);
              const float2 s2 = __fadd2_rn(uu, vv);
              float2 r2 = make_float2(sfu_pow<MODE>(s2.x, am1), sfu_pow<MODE>(s2.y, am1));
              if (MODE == 1) {  // s^(alpha-1) of an absent pair (s = 2e-30) must not count
                r2.x = s2.x > 4e-30f ? r2.x : 0.f;
                r2.y = s2.y > 4e-30f ? r2.y : 0.f;
              }
              const float2 w2 = __fmul2_rn(l2, r2);
              const float2 m2 = make_float2(fminf(uu.x, vv.x), fminf(uu.y, vv.y));
              float2 d2 = make_float2(accd[i][j], accd[i][j + 1]);
              float2 q2 = make_float2(accq[i][j], accq[i][j + 1]);
              d2 = __ffma2_rn(s2, w2, d2);
              q2 = __ffma2_rn(m2, w2, q2);
              accd[i][j] = d2.x;
              accd[i][j + 1] = d2.y;
              accq[i][j] = q2.x;
              accq[i][j + 1] = q2.y;
            }
        } else {
#pragma unroll
          for (int i = 0; i < RD; i++)
#pragma unroll
            for (int j = 0; j < RK; j++) {
              const T uu = u[j], vv = v[i + j + 1];
              const T s = uu + vv;
              T w = l * gen_pow<T, MODE>(s, am1);
              if (MODE == 1) w = s > T(0) ? w : T(0);
              accd[i][j] = fma(s, w, accd[i][j]);
              accq[i][j] = fma(fabs(uu - vv), w, accq[i][j]);
            }
        }
      }
      in_sub += G::RB;
      if (in_sub == B1 || it == nst - 1) {
#pragma unroll
        for (int i = 0; i < RD; i++)
#pragma unroll
          for (int j = 0; j < RK; j++) {
            const int c = (i * RK + j) * NT + threadIdx.x;
            midd[c] += accd[i][j];
            midq[c] += accq[i][j];
            accd[i][j] = accq[i][j] = T(0);
          }
        in_sub = 0;
      }
    }
    cp_async_wait<0>();
    commit_cells<T, RD, RK>(a.M, midd, a, U, U.s0 + RD * ts, U.k0 + RK * tk);
    commit_cells<T, RD, RK>(a.M2, midq, a, U, U.s0 + RD * ts, U.k0 + RK * tk);
  }
}

// ---- variance-adjusted weighted (Chang, Luan & Sun 2011):
//      den += w (u + v), N += w |u - v|, w = 1 / sqrt((c_k + c_j)(r_k + r_j))
//      with u = l p the length-scaled proportions, c the counts below the
//      branch and r = T - c, and w = 0 where either factor is 0 ----
// Rows hold three planes (u, c, r) of `pitch` elements each.  A stage carries
// RB rows of all three planes; the micro-tile is RD x RK with two
// accumulators per cell.
template <typename T, int RD, int RK>
struct GeoV {
  static constexpr int RB = sizeof(T) == 4 ? 8 : 4;  // rows per stage
  static constexpr int NSTAGE = 2;
  static constexpr int NPL = 3;                       // planes: u, c, r
  static constexpr int TS = 16 * RD, TK = 16 * RK;
  static constexpr int VEC = 16 / sizeof(T);
  static constexpr int UW = TK, VW = TK + TS, ROW = UW + VW;
  static constexpr int STAGE = RB * NPL * ROW;  // rows past the unit are zero (w = 0)
  static constexpr int UCH = UW / VEC, VCH = VW / VEC, CH = UCH + VCH;
  static constexpr int NV = (RD + RK + VEC - 1) / VEC;
  static constexpr size_t SMEM = (size_t)NSTAGE * STAGE * sizeof(T) + (size_t)2 * RD * RK * NT * sizeof(T);
  // Shared-memory position of row element `elem`.  A quarter-warp reads eight
  // 16-byte chunks: consecutive ones for FP32 (RK = 4 floats per chunk), which
  // hit eight distinct bank groups unswizzled (the swizzle of the 8 x 8 tile
  // would put two of them on one group whenever the run starts at an odd
  // chunk); every second one for FP64, which the swizzle spreads.
  static __device__ __forceinline__ int at(int elem) { return sizeof(T) == 4 ? elem : swz<T>(elem); }
};

template <typename T, int RD, int RK>
__device__ __forceinline__ void load_stage_vaw(T *stage, const StripeArgs &a, int e0, int e_end, int64_t ucol,
                                               int64_t vcol) {
  using G = GeoV<T, RD, RK>;
  const T *X = (const T *)a.X;
  for (int c = threadIdx.x; c < G::RB * G::NPL * G::CH; c += NT) {
    const int rp = c / G::CH, q = c - rp * G::CH;  // rp = row * NPL + plane
    const int r = rp / G::NPL, pl = rp - r * G::NPL;
    T *row = stage + rp * G::ROW;
    const int e = e0 + r;
    T *dst;
    int64_t src;
    if (q < G::UCH) {
      dst = row + G::at(q * G::VEC);
      src = ucol + q * G::VEC;
    } else {
      const int qv = q - G::UCH;
      dst = row + G::UW + G::at(qv * G::VEC);
      src = vcol + qv * G::VEC;
    }
    if (e < e_end) {
      cp_async16(dst, X + ((int64_t)e * G::NPL + pl) * a.pitch + src);
    } else {
#pragma unroll
      for (int i = 0; i < G::VEC; i++) dst[i] = T(0);
    }
  }
}

template <typename T>
__device__ __forceinline__ T vaw_weight(T prod);
template <>
__device__ __forceinline__ float vaw_weight<float>(float prod) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(prod));
  return prod > 0.f ? r : 0.f;
}
template <>
__device__ __forceinline__ double vaw_weight<double>(double prod) {
  return prod > 0.0 ? rsqrt(prod) : 0.0;
}

template <typename T, int RD, int RK, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_stripe_vaw(const StripeArgs a) {
  using G = GeoV<T, RD, RK>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *stg = reinterpret_cast<T *>(smem_raw);
  T *midd = reinterpret_cast<T *>(smem_raw + (size_t)G::NSTAGE * G::STAGE * sizeof(T));
  T *midn = midd + RD * RK * NT;
  __shared__ int s_unit;
  const int tk = threadIdx.x & 15, ts = threadIdx.x >> 4;
  const int w0 = RK * tk + RD * ts;
  Unit U;
  while (next_unit(a, G::TS, G::TK, &s_unit, &U)) {
#pragma unroll
    for (int c = 0; c < RD * RK; c++) midd[c * NT + threadIdx.x] = midn[c * NT + threadIdx.x] = T(0);
    const int nst = (U.r1 - U.r0 + G::RB - 1) / G::RB;
    if (nst > 0)
      load_stage_vaw<T, RD, RK>(stg, a, U.r0, U.r1, U.x_col + U.k0, U.x_col + U.k0 + U.s0);
    cp_async_commit();
    T accd[RD][RK], accn[RD][RK];
#pragma unroll
    for (int i = 0; i < RD; i++)
#pragma unroll
      for (int j = 0; j < RK; j++) accd[i][j] = accn[i][j] = T(0);
    int in_sub = 0;
    for (int it = 0; it < nst; it++) {
      cp_async_wait<0>();
      __syncthreads();
      if (it + 1 < nst)
        load_stage_vaw<T, RD, RK>(stg + ((it + 1) % G::NSTAGE) * G::STAGE, a, U.r0 + (it + 1) * G::RB, U.r1,
                                  U.x_col + U.k0, U.x_col + U.k0 + U.s0);
      cp_async_commit();
      const T *stage = stg + (it % G::NSTAGE) * G::STAGE;
#pragma unroll 1
      for (int r = 0; r < G::RB; r++) {
        T u[3][RK], v[3][G::NV * G::VEC];
#pragma unroll
        for (int pl = 0; pl < 3; pl++) {
          const T *urow = stage + (r * G::NPL + pl) * G::ROW;
          const T *vrow = urow + G::UW;
#pragma unroll
          for (int q = 0; q < RK / G::VEC; q++)
            *reinterpret_cast<uint4 *>(&u[pl][q * G::VEC]) =
                *reinterpret_cast<const uint4 *>(urow + G::at(RK * tk + q * G::VEC));
#pragma unroll
          for (int q = 0; q < G::NV; q++)
            *reinterpret_cast<uint4 *>(&v[pl][q * G::VEC]) =
                *reinterpret_cast<const uint4 *>(vrow + G::at(w0 + q * G::VEC));
        }
        if constexpr (sizeof(T) == 4) {
          // pairs of cells per f32x2 instruction (the weight's reciprocal
          // square roots stay scalar, on the SFU)
#pragma unroll
          for (int i = 0; i < RD; i++)
#pragma unroll
            for (int j = 0; j < RK; j += 2) {
              const float2 uu = make_float2(u[0][j], u[0][j + 1]);
              const float2 vv = make_float2(v[0][i + j + 1], v[0][i + j + 2]);
              // the two samples' counts below the branch, and the rest of their totals
              const float2 mv = __fadd2_rn(make_float2(u[1][j], u[1][j + 1]),
                                           make_float2(v[1][i + j + 1], v[1][i + j + 2]));
              const float2 rest = __fadd2_rn(make_float2(u[2][j], u[2][j + 1]),
                                             make_float2(v[2][i + j + 1], v[2][i + j + 2]));
              const float2 prod = __fmul2_rn(mv, rest);
              const float2 w = make_float2(vaw_weight<float>(prod.x), vaw_weight<float>(prod.y));
              const float2 s2 = __fadd2_rn(uu, vv);
              const float2 d2 = fsub2(uu, vv);
              float2 ad = make_float2(accd[i][j], accd[i][j + 1]);
              float2 an = make_float2(accn[i][j], accn[i][j + 1]);
              ad = __ffma2_rn(s2, w, ad);
              an = __ffma2_rn(make_float2(fabsf(d2.x), fabsf(d2.y)), w, an);
              accd[i][j] = ad.x;
              accd[i][j + 1] = ad.y;
              accn[i][j] = an.x;
              accn[i][j + 1] = an.y;
            }
        } else {
#pragma unroll
          for (int i = 0; i < RD; i++)
#pragma unroll
            for (int j = 0; j < RK; j++) {
              const T uu = u[0][j], vv = v[0][i + j + 1];
              const T mv = u[1][j] + v[1][i + j + 1];  // the two samples' counts below the branch
              const T rest = u[2][j] + v[2][i + j + 1];  // and the rest of their totals
              const T w = vaw_weight<T>(mv * rest);
              accd[i][j] = fma(uu + vv, w, accd[i][j]);
              accn[i][j] = fma(fabs(uu - vv), w, accn[i][j]);
            }
        }
      }
      in_sub += G::RB;
      if (in_sub >= B1 || it == nst - 1) {
#pragma unroll
        for (int i = 0; i < RD; i++)
#pragma unroll
          for (int j = 0; j < RK; j++) {
            const int c = (i * RK + j) * NT + threadIdx.x;
            midd[c] += accd[i][j];
            midn[c] += accn[i][j];
            accd[i][j] = accn[i][j] = T(0);
          }
        in_sub = 0;
      }
    }
    cp_async_wait<0>();
    commit_cells<T, RD, RK>(a.M, midd, a, U, U.s0 + RD * ts, U.k0 + RK * tk);
    commit_cells<T, RD, RK>(a.M2, midn, a, U, U.s0 + RD * ts, U.k0 + RK * tk);
  }
}

// ---- diagonal: D[k] += sum_e x_e[k], with the operation sequence a stripe
//      cell in min form runs when its two columns are equal ----
// Phase 1: one partial per (B1-row sub-block, sample), summed in row order;
// sub-blocks restart at every chunk boundary, as in the stripe kernels.
// Table holding combined sample column k (tables in order of off).
__device__ __forceinline__ int table_of_col(const TabDesc *tabs, int n_tabs, int k) {
  int lo = 0, hi = n_tabs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tabs[mid].off <= k) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <typename T>
__global__ void k_diag_partial(const StripeArgs a, T *__restrict__ part) {
  const int kg = blockIdx.x * blockDim.x + threadIdx.x;
  if (kg >= a.n_cols) return;
  const TabDesc &tb = a.tabs[a.n_tabs == 1 ? 0 : table_of_col(a.tabs, a.n_tabs, kg)];
  const int64_t k = tb.x_col + (kg - tb.off);  // the sample's column in its segment
  const int sb = blockIdx.y;
  const T *X = (const T *)a.X;
  const int per_chunk = (a.chunk + B1 - 1) / B1;
  const int c = sb / per_chunk;
  const int e0 = c * a.chunk + (sb - c * per_chunk) * B1;
  const int e1 = min(min(a.rows, (c + 1) * a.chunk), e0 + B1);
  T acc = T(0);
  for (int e = e0; e < e1; e++) {
    const T x = X[(int64_t)e * a.pitch + k];
    acc += tmin<T>(x, x);
  }
  part[(int64_t)sb * a.n_cols + kg] = acc;
}

// Phase 2: a chunk's sub-block partials summed in order in the path's
// precision, then rounded to fixed point (the stripe kernels' second level).
template <typename T>
__global__ void k_diag_reduce(const StripeArgs a, const T *__restrict__ part, int n_sb) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.n_cols) return;
  const int per_chunk = (a.chunk + B1 - 1) / B1;
  Fx2 d{0, 0};
  T mid = T(0);
  for (int sb = 0; sb < n_sb; sb++) {
    mid += part[(int64_t)sb * a.n_cols + k];
    if ((sb + 1) % per_chunk == 0 || sb == n_sb - 1) {
      d = fx_add(d, to_fixed2(mid, a.scale));
      mid = T(0);
    }
  }
  a.Dg[k] += (unsigned long long)d.hi;
  if constexpr (sizeof(T) == 8) a.Dg[k + a.d_lo_off] += (unsigned long long)d.lo;
}

template <typename K>
cudaError_t prepare(K kernel, size_t smem, int *grid, int units, int max_per_sm = 0) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0, dev = 0, sms = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, NT, smem);
  if (e != cudaSuccess) return e;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (max_per_sm > 0) per_sm = std::min(per_sm, max_per_sm);
  *grid = std::max(1, std::min(units, std::max(per_sm, 1) * sms));
  return cudaSuccess;
}

int units_of(const StripeArgs &a) {
  const int n_chunks = (a.rows + a.chunk - 1) / a.chunk;
  return n_chunks * a.n_tiles;
}

template <typename T, int RD, int RK, unsigned ABSM, int MINB>
cudaError_t run_min(const StripeArgs &a, cudaStream_t st) {
  using G = Geo<T, RD, RK, 1>;
  int grid = 0;
  cudaError_t e = prepare(k_stripe_min<T, RD, RK, ABSM, MINB>, G::SMEM, &grid, units_of(a));
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(a.counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  return launch_k(k_stripe_min<T, RD, RK, ABSM, MINB>, dim3(grid), dim3(NT), G::SMEM, st, a);
}

template <typename T, int RD, int RK, int MINB>
cudaError_t run_vaw(const StripeArgs &a, cudaStream_t st) {
  using G = GeoV<T, RD, RK>;
  int grid = 0;
  cudaError_t e = prepare(k_stripe_vaw<T, RD, RK, MINB>, G::SMEM, &grid, units_of(a));
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(a.counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  return launch_k(k_stripe_vaw<T, RD, RK, MINB>, dim3(grid), dim3(NT), G::SMEM, st, a);
}

template <typename T, int RD, int RK, int MODE, int MINB>
cudaError_t run_gen(const StripeArgs &a, cudaStream_t st, int max_per_sm = 0) {
  using G = Geo<T, RD, RK, 2>;
  int grid = 0;
  cudaError_t e = prepare(k_stripe_gen<T, RD, RK, MODE, MINB>, G::SMEM, &grid, units_of(a), max_per_sm);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(a.counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  return launch_k(k_stripe_gen<T, RD, RK, MODE, MINB>, dim3(grid), dim3(NT), G::SMEM, st, a);
}

}  // namespace

// micro-tiles: min kernels 8 x 8 (shape 1 of the FP32 min kernel: 4 x 8
// at three CTAs per SM, 64-stripe tiles that waste fewer stripes of small
// tables), generalized 4 x 8 (two accumulators), variance-adjusted 4 x 4
// (two accumulators, three planes)
void stripe_tile_shape(int acc, bool fp32, int *tile_s, int *tile_k, int shape) {
  *tile_s = acc == ACC_MIN && !(fp32 && shape == 1) ? 16 * 8 : 16 * 4;
  *tile_k = acc == ACC_VAW ? 16 * 4 : 16 * 8;
}

int stripe_shapes(int acc, bool fp32, unsigned abs_mask) {
  return acc == ACC_MIN && fp32 && abs_mask != 0xFFu ? 2 : 1;
}

int stripe_chunk_rows() { return 2048; }

cudaError_t launch_stripe_acc(int acc, bool fp32, const StripeArgs &a, cudaStream_t st) {
  if (a.rows <= 0 || a.n_tiles <= 0) return cudaSuccess;
  if (acc == ACC_MIN) {
    if (!fp32) return run_min<double, 8, 8, FP64_ABS_ROW_MASK, 1>(a, st);
    if (a.abs_mask == 0xFFu) return run_min<float, 8, 8, 0xFFu, 2>(a, st);
    return a.shape == 1 ? run_min<float, 4, 8, FP32_ABS_ROW_MASK, 3>(a, st)
                        : run_min<float, 8, 8, FP32_ABS_ROW_MASK, 2>(a, st);
  }
  if (acc == ACC_VAW) return fp32 ? run_vaw<float, 4, 4, 2>(a, st) : run_vaw<double, 4, 4, 1>(a, st);
  const bool half = a.alpha == 0.5;
  if (fp32) return half ? run_gen<float, 4, 8, 0, 2>(a, st) : run_gen<float, 4, 8, 1, 2>(a, st);
  return half ? run_gen<double, 4, 8, 0, 1>(a, st) : run_gen<double, 4, 8, 1, 1>(a, st);
}

size_t diag_scratch_bytes(bool fp32, int rows, int n_cols) {
  // sub-blocks of any chunk size >= 1,024 rows that is a multiple of B1
  const int64_t n_sb = (rows + B1 - 1) / B1 + (rows + 1023) / 1024;
  return (size_t)std::max<int64_t>(n_sb, 1) * n_cols * (fp32 ? 4 : 8);
}

cudaError_t launch_diag(bool fp32, const StripeArgs &a, void *scratch, cudaStream_t st) {
  if (a.rows <= 0) return cudaSuccess;
  const int per_chunk = (a.chunk + B1 - 1) / B1;
  const int n_chunks = (a.rows + a.chunk - 1) / a.chunk;
  const int n_sb = (n_chunks - 1) * per_chunk + ((a.rows - (n_chunks - 1) * a.chunk) + B1 - 1) / B1;
  dim3 g1((a.n_cols + 127) / 128, n_sb);
  const int g2 = (a.n_cols + 127) / 128;
  if (fp32) {
    const cudaError_t e = launch_k(k_diag_partial<float>, g1, dim3(128), 0, st, a, (float *)scratch);
    if (e != cudaSuccess) return e;
    return launch_k(k_diag_reduce<float>, dim3(g2), dim3(128), 0, st, a, (const float *)scratch, n_sb);
  }
  const cudaError_t e = launch_k(k_diag_partial<double>, g1, dim3(128), 0, st, a, (double *)scratch);
  if (e != cudaSuccess) return e;
  return launch_k(k_diag_reduce<double>, dim3(g2), dim3(128), 0, st, a, (const double *)scratch, n_sb);
}

}  // namespace ufg
