// uf_gram.cu -- unweighted UniFrac as a tensor-core contraction on sm_103a.
//
// For 0/1 presence a, b: [a xor b] = a + b - 2ab and [a or b] = a + b - ab, so
// with P the sample x branch presence matrix and l the branch lengths
//   G = P diag(l) P^T,   W = diag(G),
//   num(i, j) = W_i + W_j - 2 G_ij,   den(i, j) = W_i + W_j - G_ij.
// G is computed with tcgen05.mma kind::f16 on BF16 operands: B = P (exact 0/1)
// and A_t = P diag(l_t) for the three BF16 terms of each length,
// l = l_hi + l_mid + l_lo (each product is exact; the sum of the three terms
// carries l to about 24 bits), accumulated in FP32 in tensor memory.
//
// Layout: Pl[4][npad_tot][K_pad] BF16, plane 0 = P, planes 1-3 = A_hi, A_mid,
// A_lo, branches contiguous (K-major for both MMA operands); the tables of a
// batch occupy consecutive row ranges of every plane.  A work unit is
// (K chunk of `kc` branches, tile of GM = 128 samples i x GN = 256 samples j of
// one table).  Only the tiles a call needs are scheduled and stored: those
// that hold a pair of the requested stripes (stripe s holds the pairs at
// distance j - i of s + 1 and n - s - 1, Fig. 1's stripes read off the gram
// matrix) or a diagonal cell; a full-range call needs every tile that meets
// the upper triangle i <= j.  Units run chunk-major over all tables of the
// batch.  Per unit the accumulator (128 lanes x 256 FP32 columns of TMEM, two
// buffers) is rounded to int64 fixed point (scale 2^F) and added atomically
// into the unit's tile of Gt, which holds only the stored tiles, each
// transposed (cell (i, j) at (j - j0) * GM + (i - i0)) so that the 32 lanes of
// a warp add into 32 consecutive words.  Integer addition is exact and
// order-free, so the result does not depend on the order chunks land in.
//
// Roles (192 threads): warp 0 issues TMA loads (128-byte swizzled boxes into a
// two-stage ring), warp 1 allocates tensor memory and issues the MMAs, warps
// 2-5 drain the accumulators.  Every wait on an mbarrier gives up after two
// seconds, raises an abort flag seen by all roles and reports through
// `err`; the kernel then waits (again bounded) for its own outstanding copies
// and MMAs, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "uf_internal.h"
#include "uf_gram.h"

namespace ufg {

namespace {

constexpr int GM = GRAM_TM;                          // samples i per tile (TMEM lanes)
constexpr int GN = GRAM_TN;                          // samples j per tile (TMEM columns)
constexpr int GK = 64;                               // branches per stage: 128 bytes of BF16
constexpr int NSPLIT = 3;
constexpr int GSTAGES = 2;
constexpr int A_BYTES = GM * GK * 2;                 // 16 KB
constexpr int B_BYTES = GN * GK * 2;                 // 32 KB
constexpr int STAGE_BYTES = NSPLIT * A_BYTES + B_BYTES;  // 80 KB
constexpr int G_THREADS = 192;
constexpr uint32_t TMEM_COLS = 512;                  // two accumulator buffers of GN columns
constexpr unsigned long long WAIT_NS = 2000000000ull;  // bounded waits: 2 s

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of `bar` with this parity; false on abort or timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort) {
  const unsigned long long t0 = global_ns();
  for (;;) {
    if (mbar_test(bar, parity)) return true;
    if (*abort) return false;
    if (global_ns() - t0 > WAIT_NS) {
      *abort = 1;
      return false;
    }
  }
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row
// groups 1024 bytes apart (SBO), descriptor version 1.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, both
// K-major, N = GN, M = GM.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(GN >> 3) << 17) |
                           ((uint32_t)(GM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct GUnit {
  int t;               // stored tile
  int bi, bj, k0, nk;  // its block coordinates, first branch and number of GK steps
  int n, row_base;
};

__device__ __forceinline__ GUnit gram_unit(const GramArgs &a, int u) {
  const int c = u / a.n_tiles, t = u - c * a.n_tiles;
  const GramTab &tb = a.tabs[a.tile_tab[t]];
  GUnit g;
  g.t = t;
  g.bi = a.tile_bi[t];
  g.bj = a.tile_bj[t];
  g.k0 = c * a.kc;
  g.nk = (min(a.kc, a.k_len - g.k0) + GK - 1) / GK;
  g.n = tb.n;
  g.row_base = tb.row_base;
  return g;
}

__global__ void __launch_bounds__(G_THREADS, 1)
    k_gram(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, const GramArgs a) {
  extern __shared__ unsigned char smem_dyn[];
  unsigned char *smem = (unsigned char *)(((uintptr_t)smem_dyn + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[GSTAGES], empty[GSTAGES], acc_full[2], acc_empty[2], mma_done, never;
  __shared__ uint32_t s_tmem;
  __shared__ volatile int s_abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < GSTAGES; s++) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; b++) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 4);
    }
    mbar_init(&mma_done, 1);
    mbar_init(&never, 1);  // no thread ever arrives on it
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;

  if (warp == 0 && lane == 0) {
    // ---- producer: TMA loads into the stage ring ----
    int stage = 0;
    uint32_t phase = 0;
    uint32_t armed[GSTAGES] = {0, 0};  // times each stage was armed
    for (int u = blockIdx.x; u < a.n_units && !s_abort; u += gridDim.x) {
      const GUnit g = gram_unit(a, u);
      for (int ks = 0; ks < g.nk; ks++) {
        if (!mbar_wait(&empty[stage], phase ^ 1, &s_abort)) break;
        mbar_expect_tx(&full[stage], STAGE_BYTES);
        armed[stage]++;
        unsigned char *base = smem + stage * STAGE_BYTES;
        const int kx = g.k0 + ks * GK;
        for (int t = 0; t < NSPLIT; t++)
          tma_load_2d(base + t * A_BYTES, &mapA, &full[stage], kx, (1 + t) * a.npad_tot + g.row_base + g.bi * GM);
        tma_load_2d(base + NSPLIT * A_BYTES, &mapB, &full[stage], kx, g.row_base + g.bj * GN);
        if (++stage == GSTAGES) {
          stage = 0;
          phase ^= 1;
        }
      }
    }
    // every armed load must have landed before the CTA may exit
    for (int s = 0; s < GSTAGES; s++)
      if (armed[s]) {
        const unsigned long long t0 = global_ns();
        while (!mbar_test(&full[s], (armed[s] - 1) & 1) && global_ns() - t0 < WAIT_NS) {
        }
      }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer ----
    int stage = 0;
    uint32_t phase = 0;
    int ul = 0;
    if (a.wait_test) mbar_wait(&never, 0, &s_abort);  // runs out after WAIT_NS and raises the abort
    for (int u = blockIdx.x; u < a.n_units && !s_abort; u += gridDim.x, ul++) {
      const GUnit g = gram_unit(a, u);
      const int b = ul & 1;
      if (!mbar_wait(&acc_empty[b], ((ul >> 1) & 1) ^ 1, &s_abort)) break;
      tc_fence_after();
      const uint32_t d = tmem + (uint32_t)(b * GN);
      bool ok = true;
      for (int ks = 0; ks < g.nk; ks++) {
        if (!mbar_wait(&full[stage], phase, &s_abort)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t base = smem_u32(smem + stage * STAGE_BYTES);
        for (int t = 0; t < NSPLIT; t++)
#pragma unroll
          for (int k = 0; k < GK / 16; k++)
            mma_bf16(d, desc_sw128(base + t * A_BYTES + k * 32), desc_sw128(base + NSPLIT * A_BYTES + k * 32),
                     (ks | t | k) != 0);
        mma_commit(&empty[stage]);
        if (++stage == GSTAGES) {
          stage = 0;
          phase ^= 1;
        }
      }
      if (!ok) break;
      mma_commit(&acc_full[b]);
    }
    // all MMAs issued by this thread complete before tensor memory is freed
    mma_commit(&mma_done);
    const unsigned long long t0 = global_ns();
    while (!mbar_test(&mma_done, 0) && global_ns() - t0 < WAIT_NS) {
    }
  } else if (warp >= 2) {
    // ---- epilogue: TMEM -> fixed point -> atomics into Gt ----
    const int quarter = warp & 3;  // the TMEM lane quarter this warp may access
    const int row = quarter * 32 + lane;
    const float scale = (float)a.scale;
    int ul = 0;
    for (int u = blockIdx.x; u < a.n_units && !s_abort; u += gridDim.x, ul++) {
      const GUnit g = gram_unit(a, u);
      const int b = ul & 1;
      if (!mbar_wait(&acc_full[b], (ul >> 1) & 1, &s_abort)) break;
      tc_fence_after();
      const int i = g.bi * GM + row;
      unsigned long long *tile = a.Gt + (int64_t)g.t * GRAM_TILE_CELLS + row;
      for (int c = 0; c < GN / 32; c++) {
        uint32_t r[32];
        tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * GN + c * 32), r);
#pragma unroll
        for (int q = 0; q < 32; q++) {
          const int j = g.bj * GN + c * 32 + q;
          if (i <= j && j < g.n) {
            const long long v = __float2ll_rn(__uint_as_float(r[q]) * scale);
            atomicAdd(tile + (c * 32 + q) * GM, (unsigned long long)v);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[b]);
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (threadIdx.x == 0 && s_abort) atomicExch(a.err, 1);
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

// Table whose plane rows include row k (tables in order of row_base).
__device__ __forceinline__ int gram_table_of_row(const GramTab *tabs, int n_tabs, int k) {
  int lo = 0, hi = n_tabs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tabs[mid].row_base <= k) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Presence and split-length planes of a branch block, transposed to
// sample-major: Pl[0][k][e] = presence flag, Pl[1 + t][k][e] = presence * l_t,
// for every plane row k (padding rows of a table are 0).  Branch e of the
// block is node nodes[e] (b0 + e without a list).
__global__ void k_gram_prep(int64_t b0, const int32_t *__restrict__ nodes, int rows, int k_len,
                            const int32_t *__restrict__ slot_of_node,
                            const uint8_t *__restrict__ flags, int64_t ld, const double *__restrict__ length,
                            const GramTab *__restrict__ tabs, int n_tabs, int npad_tot, int64_t K_pad,
                            __nv_bfloat16 *__restrict__ Pl) {
  __shared__ float tile[32][33];
  const int e_base = blockIdx.x * 32, k_base = blockIdx.y * 32;
  {
    const int k = k_base + threadIdx.x;  // plane row
    int col = -1;
    if (k < npad_tot) {
      const GramTab &tb = tabs[n_tabs == 1 ? 0 : gram_table_of_row(tabs, n_tabs, k)];
      const int kl = k - tb.row_base;
      if (kl < tb.n) col = tb.off + kl;
    }
    for (int el = threadIdx.y; el < 32; el += blockDim.y) {
      const int e = e_base + el;
      float p = 0.f;
      if (e < rows && col >= 0) {
        const int64_t v = nodes ? (int64_t)nodes[e] : b0 + e;
        p = flags[(int64_t)slot_of_node[v] * ld + col] ? 1.f : 0.f;
      }
      tile[el][threadIdx.x] = p;
    }
  }
  __syncthreads();
  const int e = e_base + threadIdx.x;
  double l = e < rows ? length[nodes ? (int64_t)nodes[e] : b0 + e] : 0.0;
  const __nv_bfloat16 hi = __double2bfloat16(l);
  const double r1 = l - (double)__bfloat162float(hi);
  const __nv_bfloat16 mid = __double2bfloat16(r1);
  const __nv_bfloat16 lo = __double2bfloat16(r1 - (double)__bfloat162float(mid));
  const __nv_bfloat16 zero = __float2bfloat16(0.f), one = __float2bfloat16(1.f);
  if (e >= k_len) return;
  const int64_t plane = (int64_t)npad_tot * K_pad;
  for (int kl = threadIdx.y; kl < 32; kl += blockDim.y) {
    const int k = k_base + kl;
    if (k >= npad_tot) continue;
    const bool on = tile[threadIdx.x][kl] != 0.f;
    const int64_t at = (int64_t)k * K_pad + e;
    Pl[at] = on ? one : zero;
    Pl[plane + at] = on ? hi : zero;
    Pl[2 * plane + at] = on ? mid : zero;
    Pl[3 * plane + at] = on ? lo : zero;
  }
}

// Cell (i, j), i <= j, of a table's gram matrix from the compact tiles, or -1
// (never for a cell of the call's stripes or the diagonal).
__device__ __forceinline__ long long gram_cell(const GramFinalArgs &a, int64_t i, int64_t j) {
  const int64_t bi = i / GM, bj = j / GN;
  const int t = a.tile_map[bi * (a.n_pad / GN) + bj];
  if (t < 0) return -1;
  return (long long)a.Gt[(int64_t)t * GRAM_TILE_CELLS + (j - bj * GN) * GM + (i - bi * GM)];
}

// Gram accumulators (plus the sparse rows' terms) -> distances for stripes [s0, s1).
__global__ void k_finalize_gram(const GramFinalArgs a) {
  const int64_t rows = a.s1 - a.s0;
  const int64_t total = rows * a.n;
  const bool aborted = a.err && *a.err != 0;  // a bounded wait gave up: no distance is valid
  unsigned long long clamped = 0;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < total;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = c / a.n;
    const int k = (int)(c - r * a.n);
    const int64_t s = a.s0 + r;
    int64_t j = k + s + 1;
    if (j >= a.n) j -= a.n;
    if (a.full && 2 * (s + 1) == a.n && k >= a.n / 2) continue;
    const int64_t lo = k < j ? k : j, hi = k < j ? j : k;
    long long g = gram_cell(a, lo, hi);
    long long wl = gram_cell(a, lo, lo), wh = gram_cell(a, hi, hi);
    const bool missing = g < 0 || wl < 0 || wh < 0;
    if (a.Msp) g += (long long)a.Msp[c];
    if (a.Dsp) {
      wl += (long long)a.Dsp[lo];
      wh += (long long)a.Dsp[hi];
    }
    const long long w = wl + wh;
    long long num = w - 2 * g;
    const long long den = w - g;
    if (num < 0) {
      clamped++;
      num = 0;
    }
    const double val = (aborted || missing) ? __longlong_as_double(0x7ff8000000000000ll)
                       : a.unnormalized    ? (double)num * a.inv_scale
                       : den > 0           ? (double)num / (double)den
                                           : 0.0;
    const int64_t idx = a.full ? (int64_t)a.n * lo - lo * (lo + 1) / 2 + (hi - lo - 1) : c;
    if (a.out_fp32) ((float *)a.out)[idx] = (float)val;
    else ((double *)a.out)[idx] = val;
  }
  if (clamped && a.clamps) atomicAdd(a.clamps, clamped);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The CUDA driver's tensor-map encoder (cuTensorMapEncodeTiled), looked up once (a function-local static
// initialises exactly once even when several threads call first).
EncodeTiledFn encode_fn() {
  static const EncodeTiledFn fn = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return (EncodeTiledFn)p;
    return (EncodeTiledFn) nullptr;
  }();
  return fn;
}

}  // namespace

int gram_pad(int n) { return (n + GN - 1) / GN * GN; }

int64_t gram_kpad(int rows) { return ((int64_t)std::max(rows, 1) + GK - 1) / GK * GK; }

void gram_tiles(int n, int64_t s0, int64_t s1, std::vector<int32_t> *bi, std::vector<int32_t> *bj) {
  const int n_pad = gram_pad(n);
  // distances j - i held by the stripes: [s0 + 1, s1] and [n - s1, n - s0 - 1]
  const int64_t d1a = s0 + 1, d1b = s1, d2a = (int64_t)n - s1, d2b = (int64_t)n - s0 - 1;
  for (int i = 0; i < n_pad / GM; i++)
    for (int j = 0; j < n_pad / GN; j++) {
      const int64_t i0 = (int64_t)i * GM, j0 = (int64_t)j * GN;
      if (i0 >= n || j0 >= n) continue;
      const int64_t imax = std::min<int64_t>(i0 + GM, n) - 1, jmax = std::min<int64_t>(j0 + GN, n) - 1;
      const int64_t dmin = std::max<int64_t>(0, j0 - imax), dmax = jmax - i0;
      if (dmax < 0) continue;  // no cell with i <= j
      const bool need = dmin == 0 || (dmin <= d1b && d1a <= dmax) || (dmin <= d2b && d2a <= dmax);
      if (need) {
        bi->push_back(i);
        bj->push_back(j);
      }
    }
}

size_t gram_smem_bytes() { return (size_t)GSTAGES * STAGE_BYTES + 1024; }

cudaError_t launch_gram_prep(int64_t b0, int rows, const int32_t *slot_of_node, const uint8_t *flags,
                             int64_t ld, const double *length, const GramTab *tabs, int n_tabs,
                             int npad_tot, int64_t K_pad, void *Pl, cudaStream_t st, const int32_t *nodes) {
  const int k_len = (int)((rows + GK - 1) / GK * GK);
  dim3 grid((k_len + 31) / 32, (npad_tot + 31) / 32), block(32, 8);
  return launch_k(k_gram_prep, grid, block, 0, st, b0, nodes, rows, k_len, slot_of_node, flags, ld, length, tabs,
                  n_tabs, npad_tot, K_pad, (__nv_bfloat16 *)Pl);
}

cudaError_t launch_gram(const GramArgs &a0, void *Pl, int64_t K_pad, cudaStream_t st) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap mapA, mapB;
  const cuuint64_t dims[2] = {(cuuint64_t)K_pad, (cuuint64_t)4 * a0.npad_tot};
  const cuuint64_t strides[1] = {(cuuint64_t)K_pad * 2};
  const cuuint32_t boxA[2] = {GK, GM}, boxB[2] = {GK, GN}, es[2] = {1, 1};
  if (enc(&mapA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, Pl, dims, strides, boxA, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  if (enc(&mapB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, Pl, dims, strides, boxB, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  GramArgs a = a0;
  a.n_units = ((a.k_len + a.kc - 1) / a.kc) * a.n_tiles;
  if (a.n_units <= 0) return cudaSuccess;
  const size_t smem = gram_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(k_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int grid = std::max(1, std::min(a.n_units, sms));
  return launch_k(k_gram, dim3(grid), dim3(G_THREADS), smem, st, mapA, mapB, a);
}

cudaError_t launch_finalize_gram(const GramFinalArgs &a, cudaStream_t st) {
  const int64_t total = (a.s1 - a.s0) * (int64_t)a.n;
  if (total <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  int64_t blocks = (total + 255) / 256;
  blocks = std::min<int64_t>(blocks, (int64_t)std::max(sms, 1) * 64);  // a grid-stride loop beyond that
  k_finalize_gram<<<(int)blocks, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace ufg
