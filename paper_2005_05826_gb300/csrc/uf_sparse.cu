// uf_sparse.cu -- branches with few nonzero samples, as pair scatters.
//
// The stripe loop of the paper (Sec. 2-3, Figs. 1-3) visits every stripe
// cell of every branch.  In the reformulated accumulators (uf_stripe.cu) a
// branch e adds to cell (k, j)
//   min form:   min(x_e[k], x_e[j])               (0 unless both are nonzero)
//   abs form:   |x_e[k] - x_e[j]| = x_e[k] + x_e[j] - 2 min(x_e[k], x_e[j])
//   generalized den:  l s^a, s = u + v
//   generalized Q:    l min(u, v) s^(a-1)         (0 unless both are nonzero)
// and the diagonal gets x_e[k].  Near the tips most branches are nonzero in
// only a few samples, so all of a branch's nonzero terms come from its
// both-nonzero pairs plus one term per nonzero sample:
//   min form:  cell += min(X_k, X_j);  R[k] += X_k          (X = x rounded to fixed point)
//   abs form:  cell += -2 min(X_k, X_j) and the finalize adds R[k] + R[j]
//   generalized, with P_k = fixed(l u_k^a), w = l s^(a-1), q = fixed(w min(u, v)),
//   e = fixed(w |u - v|):
//              den += 2 q + e - P_k - P_j,  R[k] += P_k,  and
//              Q   += q          (FP32; num = den - 2 Q)   or
//              N   += e - P_k - P_j   (FP64; num = N),
//   so that den = sum l s^a and num = sum l s^(a-1) |u - v| over every
//   branch where u or v is nonzero (a one-sided branch gives l u^a to both),
//   and two identical samples still give num = 0 exactly.
// The finalize adds R[k] + R[j] where these terms need it (uf_finalize.cu);
// integer addition makes the order free and the result deterministic.  FP64
// terms carry the two-word fixed point of uf_device.cuh (every word summed on
// its own).  The tensor-core unweighted path scatters its sparse rows the
// same way, in the min form on presence rows (x = l): its finalize adds the
// cells to the gram matrix G and R to its diagonal.
//
// One CTA per (sparse branch, table).  The branch's tips are a contiguous
// range of tip numbers, so its nonzero counts are one contiguous run of the
// table's CSC entries: they are loaded into shared memory, sorted by sample
// (bitonic; a single tip's column is already sorted and is left alone), and
// equal samples are summed in entry order.  The z distinct samples give
// z (z - 1) / 2 pairs; each thread takes a contiguous range of the pair
// numbering and adds each pair to its stripe cell with one atomic per
// accumulator (two when the pair is the duplicated half stripe of an even n).
#include <cmath>
#include <type_traits>

#include "uf_device.cuh"
#include "uf_sparse.h"

namespace ufg {

namespace {

// Block-wide exclusive prefix of one int per thread (blockDim a multiple of 32).
__device__ int block_exclusive_scan(int v, int *sh, int *total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int w = lane < nw ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) sh[lane] = w;
  }
  __syncthreads();
  const int base = wid ? sh[wid - 1] : 0;
  *total = sh[nw - 1];
  __syncthreads();
  return base + x - v;
}

// u^alpha of a proportion u > 0
template <typename T, int MODE>
__device__ __forceinline__ T pow_alpha(T u, T alpha);
template <>
__device__ __forceinline__ double pow_alpha<double, 0>(double u, double) { return sqrt(u); }
template <>
__device__ __forceinline__ double pow_alpha<double, 1>(double u, double alpha) { return pow(u, alpha); }
template <>
__device__ __forceinline__ float pow_alpha<float, 0>(float u, float) { return u * sfu_pow<0>(u, -0.5f); }
template <>
__device__ __forceinline__ float pow_alpha<float, 1>(float u, float alpha) { return sfu_pow<1>(u, alpha); }

template <typename T, int MODE>
__device__ __forceinline__ T pow_am1(T s, T am1) {
  if constexpr (sizeof(T) == 4) return sfu_pow<MODE>(s, am1);
  else return gen_pow<T, MODE>(s, am1);
}

__device__ __forceinline__ void red_add(unsigned long long *p, long long v) {
  atomicAdd(p, (unsigned long long)v);
}
// both words of an FP64 term (the second lo_off elements after the first;
// lo_off == 0: one word, the first)
template <typename T>
__device__ __forceinline__ void red_add2(unsigned long long *p, int64_t lo_off, Fx2 v) {
  red_add(p, v.hi);
  if constexpr (sizeof(T) == 8)
    if (lo_off != 0) red_add(p + lo_off, v.lo);
}

// One distinct sample of a sparse row: its sample k, value x (or
// proportion u) and fixed-point term f, packed so that one 16-byte load
// (two for FP64) fetches all three in the pair loops.
template <typename T>
struct alignas(16) SpEnt;
template <>
struct alignas(16) SpEnt<float> {
  int k;
  float x;
  long long f;
};
template <>
struct alignas(16) SpEnt<double> {
  int k, pad;
  double x;
  long long f, f_lo;
};
__device__ __forceinline__ Fx2 ent_f(const SpEnt<float> &e) { return Fx2{e.f, 0}; }
__device__ __forceinline__ Fx2 ent_f(const SpEnt<double> &e) { return Fx2{e.f, e.f_lo}; }
__device__ __forceinline__ void set_f(SpEnt<float> &e, Fx2 v) { e.f = v.hi; }
__device__ __forceinline__ void set_f(SpEnt<double> &e, Fx2 v) {
  e.f = v.hi;
  e.f_lo = v.lo;
}

// One distinct sample of a fused list with F members (min form): the
// fixed-point terms of the listed row and of its members (0 where the sample
// is not below the member); its sample is in the list's separate key array.
template <typename T, int F>
struct FuEnt;
template <int F>
struct alignas(8) FuEnt<float, F> {
  long long f[1 + F];
};
template <int F>
struct alignas(16) FuEnt<double, F> {
  long long f[1 + F], f_lo[1 + F];
};
template <int F>
__device__ __forceinline__ Fx2 fu_f(const FuEnt<float, F> &e, int r) { return Fx2{e.f[r], 0}; }
template <int F>
__device__ __forceinline__ Fx2 fu_f(const FuEnt<double, F> &e, int r) { return Fx2{e.f[r], e.f_lo[r]}; }
template <int F>
__device__ __forceinline__ void fu_set(FuEnt<float, F> &e, int r, Fx2 v) { e.f[r] = v.hi; }
template <int F>
__device__ __forceinline__ void fu_set(FuEnt<double, F> &e, int r, Fx2 v) {
  e.f[r] = v.hi;
  e.f_lo[r] = v.lo;
}
// The same for the generalized method: each row's proportion u (0 where the
// sample is not below the row) and its term P = fixed(l u^alpha).
template <typename T, int F>
struct FuGEnt;
template <int F>
struct alignas(8) FuGEnt<float, F> {
  float x[1 + F];
  long long f[1 + F];
};
template <int F>
struct alignas(16) FuGEnt<double, F> {
  double x[1 + F];
  long long f[1 + F], f_lo[1 + F];
};
template <int F>
__device__ __forceinline__ Fx2 fu_f(const FuGEnt<float, F> &e, int r) { return Fx2{e.f[r], 0}; }
template <int F>
__device__ __forceinline__ Fx2 fu_f(const FuGEnt<double, F> &e, int r) { return Fx2{e.f[r], e.f_lo[r]}; }
template <int F>
__device__ __forceinline__ void fu_set(FuGEnt<float, F> &e, int r, Fx2 v) { e.f[r] = v.hi; }
template <int F>
__device__ __forceinline__ void fu_set(FuGEnt<double, F> &e, int r, Fx2 v) {
  e.f[r] = v.hi;
  e.f_lo[r] = v.lo;
}
// list entry type of a method's fused lists (F > 0) or of unfused lists
template <typename T, int ACC, int F>
using ListEnt = std::conditional_t<F == 0, SpEnt<T>,
                                   std::conditional_t<ACC == ACC_MIN, FuEnt<T, (F > 0 ? F : 1)>, FuGEnt<T, (F > 0 ? F : 1)>>>;

// What a pair update needs besides its two entries.
template <typename T>
struct PairCtx {
  int n, s_lo, s_hi;
  unsigned abs_mask;           // stripes in the abs form (abs_row)
  int gen_abs;                 // generalized: M2 holds N (1) or Q (0)
  int64_t m_lo_off;            // FP64: second words of M / M2 this many elements on
  unsigned long long *M, *M2;  // this table's cells (den and Q for the generalized method)
  T lt, am1;                   // branch length, alpha - 1
  double scale;
};

// Adds the pair (ea, eb), k_a < k_b, to its stripe cell when the stripe is
// stored: the min form min(X_a, X_b) (-2 times that in an abs-form stripe),
// or the generalized den and Q (or N) terms; twice for the duplicated half
// stripe.
template <typename T, int ACC, int MODE>
__device__ __forceinline__ void add_pair(const SpEnt<T> &ea, const SpEnt<T> &eb, const PairCtx<T> &c) {
  const int d = eb.k - ea.k;
  int s, kc;
  if (2 * d <= c.n) {
    s = d - 1;
    kc = ea.k;
  } else {
    s = c.n - d - 1;
    kc = eb.k;
  }
  if (s < c.s_lo || s > c.s_hi) return;
  const int64_t cell = (int64_t)(s - c.s_lo) * c.n + kc;
  const bool dup = 2 * d == c.n;  // also stored at k = k_b (= k_a + n/2)
  const Fx2 fa = ent_f(ea), fb = ent_f(eb);
  if (ACC == ACC_MIN) {
    Fx2 t = fx_min(fa, fb);
    if (abs_row(c.abs_mask, s)) t = fx_mul(t, -2);
    red_add2<T>(c.M + cell, c.m_lo_off, t);
    if (dup) red_add2<T>(c.M + cell + d, c.m_lo_off, t);
  } else {
    const T uu = ea.x, vv = eb.x;
    const T w = c.lt * pow_am1<T, MODE>(uu + vv, c.am1);
    const Fx2 q = to_fixed2(w * tmin<T>(uu, vv), c.scale);
    const Fx2 e = to_fixed2(w * (uu > vv ? uu - vv : vv - uu), c.scale);
    const Fx2 e_ab = fx_sub(fx_sub(e, fa), fb);
    const Fx2 den = fx_add(fx_mul(q, 2), e_ab);
    const Fx2 t2 = c.gen_abs ? e_ab : q;
    red_add2<T>(c.M + cell, c.m_lo_off, den);
    red_add2<T>(c.M2 + cell, c.m_lo_off, t2);
    if (dup) {
      red_add2<T>(c.M + cell + d, c.m_lo_off, den);
      red_add2<T>(c.M2 + cell + d, c.m_lo_off, t2);
    }
  }
}

// The pair (a, b), k_a < k_b, of a fused list: the sum over the listed row
// and its members of min(X_a, X_b) (a member without one of the samples
// adds 0), -2 times that in an abs-form stripe; the same integers as the
// rows' separate pair updates, in one atomic per word.
template <typename T, int F>
__device__ __forceinline__ void add_pair_fused(int ka, int kb, const FuEnt<T, F> &ea, const FuEnt<T, F> &eb,
                                               const PairCtx<T> &c) {
  const int d = kb - ka;
  int s, kc;
  if (2 * d <= c.n) {
    s = d - 1;
    kc = ka;
  } else {
    s = c.n - d - 1;
    kc = kb;
  }
  if (s < c.s_lo || s > c.s_hi) return;
  const int64_t cell = (int64_t)(s - c.s_lo) * c.n + kc;
  Fx2 t = fx_min(fu_f(ea, 0), fu_f(eb, 0));
#pragma unroll
  for (int r = 1; r <= F; r++) t = fx_add(t, fx_min(fu_f(ea, r), fu_f(eb, r)));
  if (abs_row(c.abs_mask, s)) t = fx_mul(t, -2);
  red_add2<T>(c.M + cell, c.m_lo_off, t);
  if (2 * d == c.n) red_add2<T>(c.M + cell + d, c.m_lo_off, t);
}

// The pair (a, b), k_a < k_b, of a fused generalized list: each row in which
// both samples are present (u > 0) gives the den and Q (or N) terms of its
// own update with its own length len[r]; their sums go with one atomic per
// accumulator and word, the same integers as the rows' separate updates.
template <typename T, int MODE, int F>
__device__ __forceinline__ void add_pair_fused_gen(int ka, int kb, const FuGEnt<T, F> &ea, const FuGEnt<T, F> &eb,
                                                   const PairCtx<T> &c, const T *len) {
  const int d = kb - ka;
  int s, kc;
  if (2 * d <= c.n) {
    s = d - 1;
    kc = ka;
  } else {
    s = c.n - d - 1;
    kc = kb;
  }
  if (s < c.s_lo || s > c.s_hi) return;
  const int64_t cell = (int64_t)(s - c.s_lo) * c.n + kc;
  Fx2 den{0, 0}, t2{0, 0};
#pragma unroll
  for (int r = 0; r <= F; r++) {
    const T uu = ea.x[r], vv = eb.x[r];
    if (!(uu > T(0) && vv > T(0))) continue;
    const T w = len[r] * pow_am1<T, MODE>(uu + vv, c.am1);
    const Fx2 q = to_fixed2(w * tmin<T>(uu, vv), c.scale);
    const Fx2 e = to_fixed2(w * (uu > vv ? uu - vv : vv - uu), c.scale);
    const Fx2 e_ab = fx_sub(fx_sub(e, fu_f(ea, r)), fu_f(eb, r));
    den = fx_add(den, fx_add(fx_mul(q, 2), e_ab));
    t2 = fx_add(t2, c.gen_abs ? e_ab : q);
  }
  red_add2<T>(c.M + cell, c.m_lo_off, den);
  red_add2<T>(c.M2 + cell, c.m_lo_off, t2);
  if (2 * d == c.n) {
    red_add2<T>(c.M + cell + d, c.m_lo_off, den);
    red_add2<T>(c.M2 + cell + d, c.m_lo_off, t2);
  }
}

template <typename T, int ACC, int MODE>
__global__ void __launch_bounds__(256) k_sparse_rows(const SparseArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int sh[33];
  const int P = a.cap;
  unsigned long long *key = reinterpret_cast<unsigned long long *>(smem_raw);  // (sample << 32) | entry
  double *cnt = reinterpret_cast<double *>(key + P);                          // entry -> count
  SpEnt<T> *E = reinterpret_cast<SpEnt<T> *>(cnt + P);                        // distinct samples

  const int v = a.nodes[blockIdx.x];
  const SpTab tb = a.tabs[blockIdx.y];
  const int64_t q0 = tb.col_ptr[a.tip_lo[v]];
  const int L = (int)(tb.col_ptr[a.tip_hi[v]] - q0);
  // the host sizes cap to every (row, table) run of the launch
  if (L <= 0 || L > P) return;
  const int tid = threadIdx.x, NT = blockDim.x;
  int P2 = 1;
  while (P2 < L) P2 <<= 1;
  for (int i = tid; i < P2; i += NT) {
    if (i < L) {
      key[i] = ((unsigned long long)(unsigned)tb.col_row[q0 + i] << 32) | (unsigned)i;
      cnt[i] = tb.col_val[q0 + i];
    } else {
      key[i] = ~0ull;
    }
  }
  __syncthreads();
  int unsorted = 0;
  for (int i = tid + 1; i < L; i += NT) unsorted |= (key[i] >> 32) <= (key[i - 1] >> 32);
  if (__syncthreads_or(unsorted)) {
    for (int k = 2; k <= P2; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = tid; i < P2; i += NT) {
          const int ixj = i ^ j;
          if (ixj > i) {
            const unsigned long long x = key[i], y = key[ixj];
            if ((x > y) == ((i & k) == 0)) {
              key[i] = y;
              key[ixj] = x;
            }
          }
        }
        __syncthreads();
      }
  }
  // distinct samples: the first entry of each run of equal samples
  const int EPT = (L + NT - 1) / NT, i0 = tid * EPT, i1 = min(L, i0 + EPT);
  int heads = 0;
  for (int i = i0; i < i1; i++) heads += (i == 0 || (key[i] >> 32) != (key[i - 1] >> 32));
  int z = 0;
  int u = block_exclusive_scan(heads, sh, &z);
  const double l = a.length[v];
  const T alpha = (T)a.alpha;
  for (int i = i0; i < i1; i++) {
    const unsigned smp = (unsigned)(key[i] >> 32);
    if (i > 0 && (unsigned)(key[i - 1] >> 32) == smp) continue;
    double c = 0.0;
    for (int m = i; m < L && (unsigned)(key[m] >> 32) == smp; m++) c += cnt[key[m] & 0xffffffffu];
    T x;
    if (a.kind == EMB_SCALED) x = emb_value<T, EMB_SCALED>(c, l, tb.total[smp], tb.inv_total_f[smp]);
    else if (a.kind == EMB_PRESENCE) x = emb_value<T, EMB_PRESENCE>(c, l, tb.total[smp], tb.inv_total_f[smp]);
    else x = emb_value<T, EMB_PROP>(c, l, tb.total[smp], tb.inv_total_f[smp]);
    Fx2 f;
    if (ACC == ACC_MIN) f = to_fixed2(x, a.scale);
    else f = to_fixed2((T)l * pow_alpha<T, MODE>(x, alpha), a.scale);
    SpEnt<T> en;
    en.k = (int)smp;
    en.x = x;
    set_f(en, f);
    E[u] = en;
    u++;
  }
  __syncthreads();
  for (int e = tid; e < z; e += NT) red_add2<T>(a.Dsp + tb.off + E[e].k, a.d_lo_off, ent_f(E[e]));

  // pairs (ia < ib) numbered row by row: row ia starts at ia (2z - ia - 1) / 2
  const int64_t npairs = (int64_t)z * (z - 1) / 2;
  if (npairs == 0) return;
  const int64_t per = (npairs + NT - 1) / NT;
  int64_t p = (int64_t)tid * per;
  const int64_t p1 = min(npairs, p + per);
  if (p >= p1) return;
  auto row_start = [z](int64_t r) { return r * (2 * (int64_t)z - r - 1) / 2; };
  const double bq = 2.0 * z - 1.0;
  int ia = (int)((bq - sqrt(fmax(bq * bq - 8.0 * (double)p, 0.0))) * 0.5);
  ia = max(0, min(ia, z - 2));
  while (ia > 0 && row_start(ia) > p) ia--;
  while (ia < z - 2 && row_start(ia + 1) <= p) ia++;
  int ib = ia + 1 + (int)(p - row_start(ia));
  SpEnt<T> ea = E[ia];
  PairCtx<T> c;
  c.n = tb.n;
  c.s_lo = tb.s_lo;
  c.s_hi = tb.s_hi;
  c.abs_mask = a.abs_mask;
  c.gen_abs = a.gen_abs;
  c.m_lo_off = a.m_lo_off;
  c.M = a.M + tb.m_off;
  c.M2 = ACC == ACC_GEN ? a.M2 + tb.m_off : nullptr;
  c.lt = (T)l;
  c.am1 = (T)(a.alpha - 1.0);
  c.scale = a.scale;
  for (; p < p1; p++) {
    add_pair<T, ACC, MODE>(ea, E[ib], c);
    if (++ib == z) {
      ia++;
      ib = ia + 1;
      ea = E[ia];
    }
  }
}

// List mode: the row's CSC run is sorted in shared memory as 8-byte keys
// only (so runs of up to SPARSE_LIST_MAX_ENTRIES fit), equal samples are
// summed in entry order reading the counts from global memory, and each
// distinct sample's k, x (or u) and fixed-point term go straight to the
// row's list; the per-sample terms R are added here once.
template <typename T, int ACC, int MODE, int F = 0>
__global__ void __launch_bounds__(256) k_sparse_lists(const SparseArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int sh[33];
  unsigned long long *key = reinterpret_cast<unsigned long long *>(smem_raw);  // (sample << 32) | entry
  const int v = a.nodes[blockIdx.x];
  const int row = a.row_base + blockIdx.x;
  const SpTab tb = a.tabs[0];
  const int64_t q0 = tb.col_ptr[a.tip_lo[v]];
  const int L = (int)(tb.col_ptr[a.tip_hi[v]] - q0);
  // the host sizes cap to every run of the launch and lz starts at 0
  if (L <= 0 || L > a.cap) return;
  const int tid = threadIdx.x, NT = blockDim.x;
  int P2 = 1;
  while (P2 < L) P2 <<= 1;
  for (int i = tid; i < P2; i += NT)
    key[i] = i < L ? ((unsigned long long)(unsigned)tb.col_row[q0 + i] << 32) | (unsigned)i : ~0ull;
  __syncthreads();
  int unsorted = 0;
  for (int i = tid + 1; i < L; i += NT) unsorted |= (key[i] >> 32) <= (key[i - 1] >> 32);
  if (__syncthreads_or(unsorted)) {
    for (int k = 2; k <= P2; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = tid; i < P2; i += NT) {
          const int ixj = i ^ j;
          if (ixj > i) {
            const unsigned long long x = key[i], y = key[ixj];
            if ((x > y) == ((i & k) == 0)) {
              key[i] = y;
              key[ixj] = x;
            }
          }
        }
        __syncthreads();
      }
  }
  const int EPT = (L + NT - 1) / NT, i0 = tid * EPT, i1 = min(L, i0 + EPT);
  int heads = 0;
  for (int i = i0; i < i1; i++) heads += (i == 0 || (key[i] >> 32) != (key[i - 1] >> 32));
  int z = 0;
  int u = block_exclusive_scan(heads, sh, &z);
  const double l = a.length[v];
  const T alpha = (T)a.alpha;
  const int64_t off = a.lofs[row];
  SpEnt<T> *le = reinterpret_cast<SpEnt<T> *>(a.le);
  if constexpr (F > 0) {
    // The members' tips are sub-ranges of this row's tips, so their count
    // entries are sub-runs [mlo, mhi) of its run: each distinct sample's
    // count under a member sums the same entries in the same order as the
    // member's own list would.
    int mlo[F], mhi[F];
    double ml[F];
#pragma unroll
    for (int j = 0; j < F; j++) {
      const int mv = a.members[(int64_t)F * row + j];
      mlo[j] = mv >= 0 ? (int)(tb.col_ptr[a.tip_lo[mv]] - q0) : 0;
      mhi[j] = mv >= 0 ? (int)(tb.col_ptr[a.tip_hi[mv]] - q0) : 0;
      ml[j] = mv >= 0 ? a.length[mv] : 0.0;
    }
    using FE = ListEnt<T, ACC, F>;
    FE *lf = reinterpret_cast<FE *>(a.le);
    for (int i = i0; i < i1; i++) {
      const unsigned smp = (unsigned)(key[i] >> 32);
      if (i > 0 && (unsigned)(key[i - 1] >> 32) == smp) continue;
      double c = 0.0, cm[F];
#pragma unroll
      for (int j = 0; j < F; j++) cm[j] = 0.0;
      for (int m = i; m < L && (unsigned)(key[m] >> 32) == smp; m++) {
        const int e = (int)(key[m] & 0xffffffffu);
        const double val = tb.col_val[q0 + e];
        c += val;
#pragma unroll
        for (int j = 0; j < F; j++)
          if (e >= mlo[j] && e < mhi[j]) cm[j] += val;
      }
      FE fe;
      // one row's term (and, generalized, its proportion; both 0 where the
      // sample is not below the row): as the row's own list computes them
      auto term = [&](int r, double cnt, double len) -> Fx2 {
        if constexpr (ACC == ACC_MIN) {
          const T x = a.kind == EMB_SCALED
                          ? emb_value<T, EMB_SCALED>(cnt, len, tb.total[smp], tb.inv_total_f[smp])
                          : emb_value<T, EMB_PRESENCE>(cnt, len, tb.total[smp], tb.inv_total_f[smp]);
          return to_fixed2(x, a.scale);
        } else {
          if (!(cnt > 0.0)) {
            fe.x[r] = T(0);
            return Fx2{0, 0};
          }
          const T x = emb_value<T, EMB_PROP>(cnt, len, tb.total[smp], tb.inv_total_f[smp]);
          fe.x[r] = x;
          return to_fixed2((T)len * pow_alpha<T, MODE>(x, alpha), a.scale);
        }
      };
      Fx2 f = term(0, c, l), dsum = f;
      fu_set(fe, 0, f);
#pragma unroll
      for (int j = 0; j < F; j++) {
        const Fx2 fm = term(1 + j, cm[j], ml[j]);
        fu_set(fe, 1 + j, fm);
        dsum = fx_add(dsum, fm);
      }
      lf[off + u] = fe;
      a.lk[off + u] = (int)smp;
      red_add2<T>(a.Dsp + tb.off + smp, a.d_lo_off, dsum);
      u++;
    }
    if (tid == 0) a.lz[row] = z;
    return;
  }
  for (int i = i0; i < i1; i++) {
    const unsigned smp = (unsigned)(key[i] >> 32);
    if (i > 0 && (unsigned)(key[i - 1] >> 32) == smp) continue;
    double c = 0.0;
    for (int m = i; m < L && (unsigned)(key[m] >> 32) == smp; m++) c += tb.col_val[q0 + (key[m] & 0xffffffffu)];
    T x;
    if (a.kind == EMB_SCALED) x = emb_value<T, EMB_SCALED>(c, l, tb.total[smp], tb.inv_total_f[smp]);
    else if (a.kind == EMB_PRESENCE) x = emb_value<T, EMB_PRESENCE>(c, l, tb.total[smp], tb.inv_total_f[smp]);
    else x = emb_value<T, EMB_PROP>(c, l, tb.total[smp], tb.inv_total_f[smp]);
    Fx2 f;
    if (ACC == ACC_MIN) f = to_fixed2(x, a.scale);
    else f = to_fixed2((T)l * pow_alpha<T, MODE>(x, alpha), a.scale);
    SpEnt<T> en;
    en.k = (int)smp;
    en.x = x;
    set_f(en, f);
    le[off + u] = en;
    a.lk[off + u] = (int)smp;
    red_add2<T>(a.Dsp + tb.off + smp, a.d_lo_off, f);
    u++;
  }
  if (tid == 0) a.lz[row] = z;
}

// first index in [lo, hi) of the ascending samples K with K[i] >= key
__device__ __forceinline__ int lower_index(const int *K, int lo, int hi, int key) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (K[mid] < key) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// COUNT: the instantiation for timed calls, which also counts the pair updates
// (kept apart: the count costs the counting-free kernel's 32 registers)
template <typename T, int ACC, int MODE, int F = 0, bool COUNT = false>
__global__ void __launch_bounds__(128) k_sparse_region(const SparseArgs a) {
  constexpr bool FUSED = F > 0;
  using Ent = ListEnt<T, ACC, F>;
  const int row = blockIdx.x;
  const SpTab tb = a.tabs[0];
  const int64_t off = a.lofs[row];
  // never past the row's list capacity
  const int z = (int)min((int64_t)a.lz[row], a.lofs[row + 1] - off);
  const Ent *E = reinterpret_cast<const Ent *>(a.le) + off;
  const int *K = a.lk + off;  // the same entries' samples, for the searches
  const int n = tb.n, half = n / 2;
  PairCtx<T> c;
  c.n = n;
  c.s_lo = tb.s_lo;
  c.s_hi = tb.s_hi;
  c.abs_mask = a.abs_mask;
  c.gen_abs = a.gen_abs;
  c.m_lo_off = a.m_lo_off;
  c.M = a.M + tb.m_off;
  c.M2 = ACC == ACC_GEN ? a.M2 + tb.m_off : nullptr;
  c.lt = ACC == ACC_GEN ? (T)a.length[a.nodes[row]] : T(0);
  // fused generalized lists: the lengths of the row and its members
  T len[1 + (F > 0 ? F : 1)];
  if constexpr (FUSED && ACC == ACC_GEN) {
    len[0] = c.lt;
#pragma unroll
    for (int j = 0; j < F; j++) {
      const int mv = a.members[(int64_t)F * row + j];
      len[1 + j] = mv >= 0 ? (T)a.length[mv] : T(0);
    }
  }
  c.am1 = (T)(a.alpha - 1.0);
  c.scale = a.scale;
  // Regions come in increasing stripe order (r0 of one is r1 of the one
  // before), so for a sample a the partners of window 1 move up and those of
  // window 2 move down from region to region: each entry keeps a cursor per
  // window where the previous region stopped, and only the first region of a
  // call searches for it.
  // 16-bit cursors: the region kernels stream every entry's state once per
  // region, so its bytes count (a list holds at most SPARSE_LIST_MAX_ENTRIES)
  uint16_t *cur1 = a.cur + off, *cur2 = a.cur + a.cur_stride + off;
  [[maybe_unused]] unsigned n_upd = 0;  // pair updates made by this thread: the cursors' moves
  auto add = [&](const Ent &ea, int ka, int b, int kb) {
    if constexpr (FUSED && ACC == ACC_MIN) add_pair_fused<T, F>(ka, kb, ea, E[b], c);
    else if constexpr (FUSED) add_pair_fused_gen<T, MODE, F>(ka, kb, ea, E[b], c, len);
    else add_pair<T, ACC, MODE>(ea, E[b], c);
  };
  for (int ia = threadIdx.x; ia < z - 1; ia += blockDim.x) {
    const Ent ea = E[ia];
    int ka;
    if constexpr (FUSED) ka = K[ia];
    else ka = ea.k;
    // window 1: d = k_b - k_a in [r0 + 1, min(r1, n/2)], stripe d - 1, cell column k_a
    {
      const int dlo = a.r0 + 1, dhi = min(a.r1, half);
      int b = a.first_region ? lower_index(K, ia + 1, z, ka + dlo) : (int)cur1[ia];
      [[maybe_unused]] const int b0 = b;
      if (dlo <= dhi)
        for (int kb; b < z && (kb = K[b]) <= ka + dhi; b++) add(ea, ka, b, kb);
      cur1[ia] = (uint16_t)b;
      if constexpr (COUNT) n_upd += (unsigned)(b - b0);
    }
    // window 2: d in [max(n - r1, n/2 + 1), n - r0 - 1], stripe n - d - 1, column k_b;
    // the cursor is one past the last partner not yet added
    {
      const int dlo = max(n - a.r1, half + 1), dhi = n - a.r0 - 1;
      int e = a.first_region ? lower_index(K, ia + 1, z, ka + dhi + 1) : (int)cur2[ia];
      [[maybe_unused]] const int e0 = e;
      if (dlo <= dhi)
        for (int kb; e > ia + 1 && (kb = K[e - 1]) >= ka + dlo; e--) add(ea, ka, e - 1, kb);
      cur2[ia] = (uint16_t)e;
      if constexpr (COUNT) n_upd += (unsigned)(e0 - e);
    }
  }
  if constexpr (COUNT) {  // every thread of the CTA is here
    __shared__ unsigned long long s_upd;
    if (threadIdx.x == 0) s_upd = 0;
    __syncthreads();
    unsigned long long w = n_upd;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if ((threadIdx.x & 31) == 0 && w) atomicAdd(&s_upd, w);
    __syncthreads();
    // spread over SPARSE_PAIR_SLOTS counters, so that no single address takes
    // one atomic per CTA of every region
    if (threadIdx.x == 0 && s_upd) atomicAdd(a.pair_count + (blockIdx.x & (SPARSE_PAIR_SLOTS - 1)), s_upd);
  }
}

template <typename T, int ACC, int MODE>
cudaError_t launch_one(const SparseArgs &a, size_t smem, cudaStream_t st) {
  auto kernel = k_sparse_rows<T, ACC, MODE>;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int nt = a.cap <= 512 ? 128 : 256;
  dim3 grid((unsigned)a.n_nodes, (unsigned)a.n_tabs);
  kernel<<<grid, nt, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

size_t sparse_smem_bytes(bool fp32, int cap) {
  return (size_t)cap * (8 + 8 + (fp32 ? sizeof(SpEnt<float>) : sizeof(SpEnt<double>)));
}

size_t sparse_entry_bytes(bool fp32, int fused, int acc) {
  if (fused == 2 && acc == ACC_GEN) return fp32 ? sizeof(FuGEnt<float, 2>) : sizeof(FuGEnt<double, 2>);
  if (fused != 0 && acc == ACC_GEN) return 0;
  if (fused == 2) return fp32 ? sizeof(FuEnt<float, 2>) : sizeof(FuEnt<double, 2>);
  if (fused == 6) return fp32 ? sizeof(FuEnt<float, 6>) : sizeof(FuEnt<double, 6>);
  return fp32 ? sizeof(SpEnt<float>) : sizeof(SpEnt<double>);
}

cudaError_t launch_sparse_rows(int acc, bool fp32, const SparseArgs &a, cudaStream_t st) {
  if (a.n_nodes <= 0 || a.n_tabs <= 0) return cudaSuccess;
  if (a.cap < 128 || (a.cap & (a.cap - 1)) || a.cap > SPARSE_MAX_ENTRIES || a.n_tabs > 65535)
    return cudaErrorInvalidValue;
  const size_t smem = sparse_smem_bytes(fp32, a.cap);
  const int mode = a.alpha == 0.5 ? 0 : 1;
  if (acc == ACC_MIN) return fp32 ? launch_one<float, ACC_MIN, 0>(a, smem, st) : launch_one<double, ACC_MIN, 0>(a, smem, st);
  if (fp32) return mode == 0 ? launch_one<float, ACC_GEN, 0>(a, smem, st) : launch_one<float, ACC_GEN, 1>(a, smem, st);
  return mode == 0 ? launch_one<double, ACC_GEN, 0>(a, smem, st) : launch_one<double, ACC_GEN, 1>(a, smem, st);
}

template <bool C>
cudaError_t launch_region(int acc, bool fp32, const SparseArgs &a, dim3 grid, cudaStream_t st) {
  const int mode = a.alpha == 0.5 ? 0 : 1;
  if (acc == ACC_MIN && a.fused != 0) {
    if (a.fused == 2) {
      if (fp32) k_sparse_region<float, ACC_MIN, 0, 2, C><<<grid, 128, 0, st>>>(a);
      else k_sparse_region<double, ACC_MIN, 0, 2, C><<<grid, 128, 0, st>>>(a);
    } else if (a.fused == 6) {
      if (fp32) k_sparse_region<float, ACC_MIN, 0, 6, C><<<grid, 128, 0, st>>>(a);
      else k_sparse_region<double, ACC_MIN, 0, 6, C><<<grid, 128, 0, st>>>(a);
    } else {
      return cudaErrorInvalidValue;
    }
  } else if (acc == ACC_MIN) {
    if (fp32) k_sparse_region<float, ACC_MIN, 0, 0, C><<<grid, 128, 0, st>>>(a);
    else k_sparse_region<double, ACC_MIN, 0, 0, C><<<grid, 128, 0, st>>>(a);
  } else if (a.fused == 2) {
    if (fp32) {
      if (mode == 0) k_sparse_region<float, ACC_GEN, 0, 2, C><<<grid, 128, 0, st>>>(a);
      else k_sparse_region<float, ACC_GEN, 1, 2, C><<<grid, 128, 0, st>>>(a);
    } else {
      if (mode == 0) k_sparse_region<double, ACC_GEN, 0, 2, C><<<grid, 128, 0, st>>>(a);
      else k_sparse_region<double, ACC_GEN, 1, 2, C><<<grid, 128, 0, st>>>(a);
    }
  } else if (a.fused != 0) {
    return cudaErrorInvalidValue;
  } else if (fp32) {
    if (mode == 0) k_sparse_region<float, ACC_GEN, 0, 0, C><<<grid, 128, 0, st>>>(a);
    else k_sparse_region<float, ACC_GEN, 1, 0, C><<<grid, 128, 0, st>>>(a);
  } else {
    if (mode == 0) k_sparse_region<double, ACC_GEN, 0, 0, C><<<grid, 128, 0, st>>>(a);
    else k_sparse_region<double, ACC_GEN, 1, 0, C><<<grid, 128, 0, st>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_sparse_region(int acc, bool fp32, const SparseArgs &a, cudaStream_t st) {
  if (a.n_nodes <= 0 || a.r0 >= a.r1) return cudaSuccess;
  const dim3 grid((unsigned)a.n_nodes);
  return a.pair_count ? launch_region<true>(acc, fp32, a, grid, st) : launch_region<false>(acc, fp32, a, grid, st);
}

size_t sparse_list_smem_bytes(int cap) { return (size_t)cap * 8; }

cudaError_t launch_sparse_lists(int acc, bool fp32, const SparseArgs &a, cudaStream_t st) {
  if (a.n_nodes <= 0) return cudaSuccess;
  if (a.cap < 128 || (a.cap & (a.cap - 1)) || a.cap > SPARSE_LIST_MAX_ENTRIES || a.n_tabs != 1)
    return cudaErrorInvalidValue;
  const size_t smem = sparse_list_smem_bytes(a.cap);
  const int mode = a.alpha == 0.5 ? 0 : 1;
  const int nt = a.cap <= 512 ? 128 : 256;
  const dim3 grid((unsigned)a.n_nodes);
  auto go = [&](auto kernel) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kernel<<<grid, nt, smem, st>>>(a);
    return cudaGetLastError();
  };
  if (acc == ACC_MIN && a.fused == 2)
    return fp32 ? go(k_sparse_lists<float, ACC_MIN, 0, 2>) : go(k_sparse_lists<double, ACC_MIN, 0, 2>);
  if (acc == ACC_MIN && a.fused == 6)
    return fp32 ? go(k_sparse_lists<float, ACC_MIN, 0, 6>) : go(k_sparse_lists<double, ACC_MIN, 0, 6>);
  if (acc == ACC_GEN && a.fused == 2) {
    if (fp32) return mode == 0 ? go(k_sparse_lists<float, ACC_GEN, 0, 2>) : go(k_sparse_lists<float, ACC_GEN, 1, 2>);
    return mode == 0 ? go(k_sparse_lists<double, ACC_GEN, 0, 2>) : go(k_sparse_lists<double, ACC_GEN, 1, 2>);
  }
  if (a.fused != 0) return cudaErrorInvalidValue;
  if (acc == ACC_MIN) return fp32 ? go(k_sparse_lists<float, ACC_MIN, 0>) : go(k_sparse_lists<double, ACC_MIN, 0>);
  if (fp32) return mode == 0 ? go(k_sparse_lists<float, ACC_GEN, 0>) : go(k_sparse_lists<float, ACC_GEN, 1>);
  return mode == 0 ? go(k_sparse_lists<double, ACC_GEN, 0>) : go(k_sparse_lists<double, ACC_GEN, 1>);
}

}  // namespace ufg
