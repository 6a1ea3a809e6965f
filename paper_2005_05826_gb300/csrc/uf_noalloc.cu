// uf_noalloc.cu -- uf_compute_noalloc: UniFrac on one GPU without allocating
// device memory.
//
// Who needs it: callers that may not call cudaMalloc -- an application whose
// own memory manager owns the device heap (a framework caching allocator, a
// service running under a fixed device-memory budget), or code that must not
// enter the allocator at all because its latency or its failure path is not
// allowed there.  uf_compute draws its working memory from the CUDA
// stream-ordered allocator and keeps device copies of the tree and table;
// this entry point does neither.  Its working memory is one fixed area,
// `g_scratch` below, a file-scope __device__ array of UF_NOALLOC_SCRATCH_BYTES
// that every GPU loading the library holds until the process exits.  Inputs
// are copied from the handles' host copies into that area on every call; the
// caller supplies the output buffer in device memory.
//
// The computation is the one uf_compute performs for the full stripe range
// with a single branch block: tip counts, internal levels, embedding rows,
// stripe accumulate, the diagonal (whose sub-block partials are this call's
// kernel scratch), and finalize -- the same kernels, launched with pointers
// into the fixed area.  A problem whose working set exceeds the area is
// rejected with UF_ENOMEM before anything is launched.
//
// Set-up: the first call on a device, with that device current, looks up the
// area's device address with cudaGetSymbolAddress (host code only sees a
// host-side stand-in under the array's name); the address is cached per device.
// Make that first call before any stream capture begins on the device.
//
// Sharing: every call on a device uses the same area and leaves its contents
// behind; the accumulators that must start at zero are cleared by each call.
// Calls whose work overlaps on the GPU (other streams, other host threads)
// race on the area; the call waits for its own work before returning, so
// calls from one thread in sequence are safe.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <exception>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/unifrac_gb300.h"
#include "uf_internal.h"
#include "uf_embed.h"
#include "uf_finalize.h"

namespace {

constexpr int UF_NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_scratch[UF_NOALLOC_SCRATCH_BYTES];

std::mutex g_setup_mu;
unsigned char *g_scratch_dev[UF_NOALLOC_MAX_DEVICES] = {nullptr};

// Device address of g_scratch on the current device (set-up on first use).
cudaError_t scratch_address(int device, unsigned char **out) {
  std::lock_guard<std::mutex> g(g_setup_mu);
  if (!g_scratch_dev[device]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_dev[device] = static_cast<unsigned char *>(p);
  }
  *out = g_scratch_dev[device];
  return cudaSuccess;
}

// Bump carver over the fixed area, 256-byte aligned.
struct Carve {
  unsigned char *base;
  size_t used = 0;
  template <typename T>
  T *take(size_t count) {
    used = (used + 255) / 256 * 256;
    T *p = reinterpret_cast<T *>(base ? base + used : nullptr);
    used += std::max<size_t>(count, 1) * sizeof(T);
    return p;
  }
};

int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

}  // namespace

namespace {
uf_status noalloc_fail(uf_status st, const char *msg) { return ufg::set_last_error(st, msg); }
}  // namespace

// (the CUDA sources build with hidden visibility; the ABI entry point is exported)
namespace {
uf_status compute_noalloc(const uf_tree *tree, const uf_table *table, uf_method method, double alpha,
                          uf_precision precision, double *out_device, void *cuda_stream) {
  using namespace ufg;
  TreeView tv;
  TableView xv;
  if (!tree_host_view(tree, &tv) || !table_host_view(table, &xv))
    return noalloc_fail(UF_EINVAL, "null tree or table");
  if (method < UF_UNWEIGHTED || method > UF_GENERALIZED)
    return noalloc_fail(UF_EINVAL, "the allocation-free entry point computes the methods UF_UNWEIGHTED .. "
                                   "UF_GENERALIZED");
  if (precision != UF_FP64 && precision != UF_MIXED) return noalloc_fail(UF_EINVAL, "unknown precision");
  if (method == UF_GENERALIZED && !(alpha >= 0.0 && alpha <= 1.0))
    return noalloc_fail(UF_EINVAL, "alpha must be in [0, 1]");
  if (xv.n_features != tv.n_tips) return noalloc_fail(UF_ETABLE, "table and tree tip counts differ");
  const int n = (int)xv.n;
  const int64_t S = n / 2;
  if (S == 0) return UF_OK;  // fewer than two samples: no pair
  if (!out_device) return noalloc_fail(UF_EINVAL, "null output buffer");

  if (method == UF_GENERALIZED && alpha == 1.0) method = UF_WEIGHTED_NORMALIZED;  // s^0 == 1
  const int acc = method == UF_GENERALIZED ? ACC_GEN : ACC_MIN;
  const int kind = method == UF_GENERALIZED ? EMB_PROP
                   : method == UF_UNWEIGHTED ? EMB_PRESENCE
                                             : EMB_SCALED;
  const bool fp32 = precision == UF_MIXED;
  const size_t es = fp32 ? 4 : 8;
  const size_t words = fp32 ? 1 : 2;
  int tile_s = 0, tile_k = 0;
  stripe_tile_shape(acc, fp32, &tile_s, &tile_k);
  const int m_hi = (int)((S - 1) / tile_s);
  const int64_t pitch = round_up(round_up(n, tile_k) + (int64_t)(m_hi + 1) * tile_s, 32);
  const int64_t N = tv.n_nodes, nb = N - 1;
  const double scale = accum_scale(tree, table, kind);

  // one branch block holding every branch; slot of node v = v
  std::vector<int32_t> level(N, 0), lists, slot(N);
  std::vector<std::pair<int64_t, int>> launches;
  {
    std::vector<std::vector<int32_t>> lv(1);
    for (int64_t v = 0; v < nb; v++) {
      if (tv.tip_of_node[v] >= 0) {
        lv[0].push_back((int32_t)v);
        continue;
      }
      int32_t L = 0;
      for (int32_t c = tv.child_ptr[v]; c < tv.child_ptr[v + 1]; c++) {
        const int32_t ch = tv.child_idx[c];
        if (tv.tip_of_node[ch] < 0) L = std::max(L, level[ch] + 1);
      }
      level[v] = L;
      if ((int)lv.size() < L + 2) lv.resize(L + 2);
      lv[L + 1].push_back((int32_t)v);
    }
    for (auto &l : lv) {
      launches.emplace_back((int64_t)lists.size(), (int)l.size());
      lists.insert(lists.end(), l.begin(), l.end());
    }
    for (int64_t v = 0; v < N; v++) slot[v] = (int32_t)v;
  }
  const int rows = (int)std::max<int64_t>(nb, 0);

  // layout of the fixed area (a dry run with a null base sizes it)
  auto layout = [&](Carve &c, void **p) {
    p[0] = c.take<double>(N);                       // length
    p[1] = c.take<int32_t>(N);                      // tip_of_node
    p[2] = c.take<int32_t>(N + 1);                  // child_ptr
    p[3] = c.take<int32_t>(std::max<int64_t>(nb, 1));  // child_idx
    p[4] = c.take<int32_t>(N);                      // slot_of_node
    p[5] = c.take<int32_t>(std::max<size_t>(lists.size(), 1));  // level lists
    p[6] = c.take<int64_t>(xv.n_features + 1);      // col_ptr
    p[7] = c.take<int32_t>(std::max<int64_t>(xv.nnz, 1));  // col_row
    p[8] = c.take<double>(std::max<int64_t>(xv.nnz, 1));   // col_val
    p[9] = c.take<double>(n);                       // total
    p[10] = c.take<float>(n);                       // inv_total_f
    p[11] = c.take<double>((size_t)std::max<int64_t>(nb, 1) * n);        // counts
    p[12] = c.take<unsigned char>((size_t)std::max(rows, 1) * pitch * es);  // X
    // fixed-point accumulators (FP64: two words each, the second after the first)
    p[13] = c.take<unsigned long long>((size_t)S * n * words);  // stripe accumulator
    p[14] = acc == ACC_GEN ? (void *)c.take<unsigned long long>((size_t)S * n * words) : nullptr;  // Q or N
    p[15] = acc == ACC_MIN ? (void *)c.take<unsigned long long>((size_t)n * words) : nullptr;      // diagonal
    p[16] = acc == ACC_MIN ? (void *)c.take<unsigned char>(diag_scratch_bytes(fp32, std::max(rows, 1), n))
                           : nullptr;                                        // diagonal partials
    p[17] = c.take<int>(1);                                                  // work-unit counter
    p[18] = c.take<TabDesc>(1);                                              // the table's description
  };
  void *p[19];
  Carve dry{nullptr};
  layout(dry, p);
  if (dry.used > UF_NOALLOC_SCRATCH_BYTES) {
    char msg[200];
    snprintf(msg, sizeof msg, "problem needs %zu bytes of working memory; the fixed area holds %zu",
             dry.used, UF_NOALLOC_SCRATCH_BYTES);
    return noalloc_fail(UF_ENOMEM, msg);
  }

  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess || device < 0 || device >= UF_NOALLOC_MAX_DEVICES) {
    cudaGetLastError();
    return noalloc_fail(UF_ECUDA, "no usable CUDA device");
  }
  const uf_status out_ok = check_device_output(out_device, "out_device");
  if (out_ok != UF_OK) return out_ok;
  unsigned char *base = nullptr;
  e = scratch_address(device, &base);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return noalloc_fail(UF_ECUDA, cudaGetErrorString(e));
  }
  Carve c{base};
  layout(c, p);
  cudaStream_t st = (cudaStream_t)cuda_stream;

#define UF_TRY(x)                                  \
  do {                                             \
    cudaError_t _e = (x);                          \
    if (_e != cudaSuccess) {                       \
      cudaGetLastError();                          \
      return noalloc_fail(UF_ECUDA, cudaGetErrorString(_e)); \
    }                                              \
  } while (0)
  auto h2d = [&](void *dst, const void *src, size_t bytes) {
    return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st) : cudaSuccess;
  };
  UF_TRY(h2d(p[0], tv.length, N * 8));
  UF_TRY(h2d(p[1], tv.tip_of_node, N * 4));
  UF_TRY(h2d(p[2], tv.child_ptr, (N + 1) * 4));
  UF_TRY(h2d(p[3], tv.child_idx, nb * 4));
  UF_TRY(h2d(p[4], slot.data(), N * 4));
  UF_TRY(h2d(p[5], lists.data(), lists.size() * 4));
  UF_TRY(h2d(p[6], xv.col_ptr, (xv.n_features + 1) * 8));
  UF_TRY(h2d(p[7], xv.col_row, xv.nnz * 4));
  UF_TRY(h2d(p[8], xv.col_val, xv.nnz * 8));
  UF_TRY(h2d(p[9], xv.total, (size_t)n * 8));
  UF_TRY(h2d(p[10], xv.inv_total_f, (size_t)n * 4));
  TabDesc tab{};
  tab.n = n;
  tab.off = 0;
  tab.s_lo = 0;
  tab.s_hi = (int)(S - 1);
  tab.m_lo = 0;
  tab.m_hi = m_hi;
  tab.n_ktiles = (n + tile_k - 1) / tile_k;
  tab.tile0 = 0;
  tab.kband = tab.n_ktiles;  // sample tile fastest over the whole table
  tab.x_col = 0;
  tab.m_off = 0;
  UF_TRY(h2d(p[18], &tab, sizeof tab));
  // accumulators start at zero; the rest of the area is overwritten before use
  UF_TRY(cudaMemsetAsync(p[13], 0, (size_t)S * n * 8 * words, st));
  if (p[14]) UF_TRY(cudaMemsetAsync(p[14], 0, (size_t)S * n * 8 * words, st));
  if (p[15]) UF_TRY(cudaMemsetAsync(p[15], 0, (size_t)n * 8 * words, st));

  const int32_t *d_lists = (const int32_t *)p[5], *d_slot = (const int32_t *)p[4];
  double *d_counts = (double *)p[11];
  if (rows > 0) {
    UF_TRY(launch_tip_counts(d_lists + launches[0].first, launches[0].second, d_slot,
                             (const int32_t *)p[1], (const int64_t *)p[6], (const int32_t *)p[7],
                             (const double *)p[8], d_counts, n, n, st));
    for (size_t l = 1; l < launches.size(); l++)
      UF_TRY(launch_node_counts(d_lists + launches[l].first, launches[l].second,
                                (const int32_t *)p[2], (const int32_t *)p[3], d_slot, d_counts, n, st));
    UF_TRY(launch_emb_rows(kind, fp32, 0, rows, d_slot, d_counts, n, (const double *)p[0],
                           (const double *)p[9], (const float *)p[10], p[12], pitch,
                           (const TabDesc *)p[18], 1, st));
    StripeArgs sa{};
    sa.X = p[12];
    sa.len = (const double *)p[0];
    sa.rows = rows;
    sa.pitch = pitch;
    sa.chunk = stripe_chunk_rows();
    sa.tabs = (const TabDesc *)p[18];
    sa.n_tabs = 1;
    sa.n_tiles = tab.n_ktiles * (m_hi + 1);
    sa.n_cols = n;
    sa.M = (unsigned long long *)p[13];
    sa.M2 = (unsigned long long *)p[14];
    sa.Dg = (unsigned long long *)p[15];
    sa.alpha = alpha;
    sa.scale = scale;
    sa.counter = (int *)p[17];
    sa.m_lo_off = fp32 ? 0 : (int64_t)S * n;
    sa.d_lo_off = fp32 ? 0 : n;
    UF_TRY(launch_stripe_acc(acc, fp32, sa, st));
    if (acc == ACC_MIN) UF_TRY(launch_diag(fp32, sa, p[16], st));
  }
  FinalArgs fa{};
  fa.method = method;
  fa.n = n;
  fa.s0 = 0;
  fa.s1 = S;
  fa.full = 1;
  fa.abs_mask = acc == ACC_MIN ? abs_row_mask(fp32) : 0u;
  fa.gen_abs = acc == ACC_GEN && !fp32;
  fa.M = (const unsigned long long *)p[13];
  fa.M2 = (const unsigned long long *)p[14];
  fa.Dg = (const unsigned long long *)p[15];
  fa.inv_scale = 1.0 / scale;
  fa.m_lo_off = fp32 ? 0 : (int64_t)S * n;
  fa.d_lo_off = fp32 ? 0 : n;
  fa.out = out_device;
  fa.out_fp32 = 0;
  UF_TRY(launch_finalize(fa, st));
  UF_TRY(cudaStreamSynchronize(st));
#undef UF_TRY
  return UF_OK;
}
}  // namespace

extern "C" __attribute__((visibility("default"))) uf_status uf_compute_noalloc(
                                         const uf_tree *tree, const uf_table *table,
                                         uf_method method, double alpha,
                                         uf_precision precision, double *out_device,
                                         void *cuda_stream) {
  ufg::set_last_error(UF_OK, "");
  try {
    return compute_noalloc(tree, table, method, alpha, precision, out_device, cuda_stream);
  } catch (const std::bad_alloc &) {
    return noalloc_fail(UF_ENOMEM, "host allocation failed");
  } catch (const std::exception &e) {
    char msg[300];
    snprintf(msg, sizeof msg, "host resources: %s", e.what());
    return noalloc_fail(UF_ENOMEM, msg);
  }
}
