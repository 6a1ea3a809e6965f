// uf_runtime.h -- host runtime internals shared by uf_host.cpp (tree and
// table handles, the C ABI), uf_split.cpp (the dense / sparse branch split)
// and uf_run.cpp (the launch sequence of one compute call).  Not part of the
// ABI; host code only.
#pragma once
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <system_error>
#include <thread>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/unifrac_gb300.h"
#include "uf_internal.h"
#include "uf_sparse.h"
#include "uf_embed.h"
#include "uf_finalize.h"
#include "uf_gram.h"

namespace ufg {
namespace rt {

// ---- errors and options (uf_host.cpp) ----
extern thread_local std::string g_err;   // uf_last_error() text of this thread
extern thread_local double g_h2d;        // bytes the current call uploaded
extern std::atomic<int64_t> g_branch_block, g_kernel_timing, g_tensor_path, g_graph, g_autotune, g_sparse, g_overlap,
    g_tensor_wait_test, g_tile_shape, g_sparse_fuse;

// Sets the thread's error text and returns st.
uf_status fail(uf_status st, const char *fmt, ...);

// Thrown by ck() on a CUDA error, after fail() recorded it.
struct CudaFail {
  uf_status st;
};
void ck(cudaError_t e, const char *what);

// Host threads for table preparation: the cores this process may run on, at most 16.
int host_threads();

// An NVTX range for the lifetime of the object: a call and its host phases
// appear by name on a profiler's timeline (a near no-op without a profiler).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

// Runs body(0 .. n-1) on the process's host worker pool (host_threads() - 1
// persistent threads, started on first use) and the calling thread, and
// returns when every index has run.  Indices are handed out one at a time, so
// calls from several threads (or from inside a body) share the pool without
// waiting on each other's indices.  In a forked child the pool is not
// inherited: the calling thread runs every index.  The first exception a
// body throws is rethrown in the caller once every index has run.
void run_parallel(int n, const std::function<void(int)> &body);
template <typename F>
void parallel_for(int n, F body) {
  run_parallel(n, std::function<void(int)>(std::move(body)));
}

// Allocator whose value-less construct leaves elements uninitialised: for
// buffers that are written in full right after they are sized.
template <typename T>
struct NoInit : std::allocator<T> {
  template <typename U>
  struct rebind {
    using other = NoInit<U>;
  };
  NoInit() = default;
  template <typename U>
  NoInit(const NoInit<U> &) {}
  template <typename U, typename... A>
  void construct(U *p, A &&...a) {
    if constexpr (sizeof...(A) == 0) ::new ((void *)p) U;
    else ::new ((void *)p) U(std::forward<A>(a)...);
  }
};

// Host -> device copy of pageable memory through a ring of pinned chunks:
// host threads fill one chunk while the copy engine drains the previous ones
// (a plain cudaMemcpy from pageable memory is staged by the driver at a
// fraction of the link's rate).  Synchronous: returns when dst holds the data.
void pinned_upload(void *dst, const void *src, size_t bytes);

// Several host arrays copied into one device allocation at 256-byte aligned
// offsets: one cudaMalloc per handle instead of one per array.
struct DevPack {
  std::vector<std::pair<const void *, size_t>> parts;
  std::vector<size_t> offs;
  size_t total = 0;
  template <typename T, typename Alloc>
  size_t add(const std::vector<T, Alloc> &h) {
    const size_t off = (total + 255) & ~(size_t)255;
    offs.push_back(off);
    parts.emplace_back(h.data(), h.size() * sizeof(T));
    total = off + std::max<size_t>(h.size() * sizeof(T), 16);
    return parts.size() - 1;
  }
  // the device copy; free with cudaFree
  char *upload(const char *what) {
    char *d = nullptr;
    ck(cudaMalloc(&d, std::max<size_t>(total, 16)), what);
    for (size_t i = 0; i < parts.size(); i++) {
      if (!parts[i].second) continue;
      try {
        pinned_upload(d + offs[i], parts[i].first, parts[i].second);
      } catch (...) {
        cudaFree(d);
        throw;
      }
      g_h2d += (double)parts[i].second;
    }
    return d;
  }
  template <typename T>
  static T *at(char *base, const DevPack &pk, size_t part) {
    return reinterpret_cast<T *>(base + pk.offs[part]);
  }
};


// ------------------------------------------------------------------- plan

// Postorder branch blocks [b0, b1) with their level lists and live slots.
struct Plan {
  int64_t block_rows = 0;
  std::vector<int64_t> b0, b1;
  // per block: offsets into `lists` of the tip list, then internal levels
  std::vector<std::vector<std::pair<int64_t, int>>> launches;  // (offset, count), first = tips
  std::vector<int32_t> lists;
  std::vector<int32_t> slot_of_node;
  int64_t n_slots = 0;
  // device copies (device id -> pointers)
  struct Dev {
    char *base = nullptr;  // one allocation holding both
    int32_t *lists = nullptr, *slot_of_node = nullptr;
  };
  std::map<int, Dev> dev;
};

struct RowSplit;
// (table ids, accumulator, FP32, sparse mode, block rows, region budget)
using SplitKey = std::tuple<std::vector<uint64_t>, int, int, int, int64_t, int64_t>;

}  // namespace rt
}  // namespace ufg

struct uf_tree {
  uint64_t id = 0;  // process-unique, never reused
  int64_t n_nodes = 0, n_tips = 0;
  std::vector<int64_t> parent;
  std::vector<double> length;
  std::vector<int32_t> tip_of_node;            // node -> tip number or -1
  std::vector<int32_t> child_ptr, child_idx;   // children in index order
  // tips under node v are the tip numbers [tip_lo[v], tip_hi[v]) when those
  // are contiguous (always so for a postorder numbering), else both -1
  std::vector<int32_t> tip_lo, tip_hi;
  std::mutex mu;
  struct Dev {
    char *base = nullptr;  // one allocation holding the arrays below
    double *length = nullptr;
    int32_t *tip_of_node = nullptr, *child_ptr = nullptr, *child_idx = nullptr;
    int32_t *tip_lo = nullptr, *tip_hi = nullptr;
  };
  std::map<int, Dev> dev;
  std::map<int64_t, std::unique_ptr<ufg::rt::Plan>> plans;  // by block rows
  std::map<ufg::rt::SplitKey, std::shared_ptr<const ufg::rt::RowSplit>> splits;  // dense / sparse branch splits
  // root distance of every node (root: 0), max over tips, total branch length
  std::vector<double> dist;
  std::vector<double> tip_dist;  // dist of tip number f
  double max_tip_dist = 0.0, total_length = 0.0;
  ~uf_tree() {
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto &kv : dev) {
      cudaSetDevice(kv.first);
      cudaFree(kv.second.base);
    }
    for (auto &p : plans)
      for (auto &kv : p.second->dev) {
        cudaSetDevice(kv.first);
        cudaFree(kv.second.base);
      }
    cudaSetDevice(cur);
  }
};

struct uf_table {
  uint64_t id = 0;                 // process-unique, never reused
  int64_t n = 0, n_features = 0, nnz = 0;
  std::vector<double> total;       // per-sample count totals (row order sums)
  std::vector<float> inv_total_f;  // 1 / total in FP32
  std::vector<int64_t> col_ptr;    // CSC view: tip f -> samples
  std::vector<int32_t, ufg::rt::NoInit<int32_t>> col_row;
  std::vector<double, ufg::rt::NoInit<double>> col_val;
  std::mutex mu;
  std::map<uint64_t, double> presence_bound;  // by tree id: max_k sum_{f in k} dist(tip f)
  double min_count = 1.0;                     // the smallest count of the table
  struct Dev {
    char *base = nullptr;  // one allocation holding the arrays below
    double *total = nullptr, *col_val = nullptr;
    float *inv_total_f = nullptr;
    int64_t *col_ptr = nullptr;
    int32_t *col_row = nullptr;
  };
  std::map<int, Dev> dev;
  ~uf_table() {
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto &kv : dev) {
      cudaSetDevice(kv.first);
      cudaFree(kv.second.base);
    }
    cudaSetDevice(cur);
  }
};

namespace ufg {
namespace rt {

// ---- device copies of the handles (uf_host.cpp); callers hold the handle's mutex ----
uf_tree::Dev &tree_dev(uf_tree *t, int device);
uf_table::Dev &table_dev(uf_table *t, int device);
Plan *get_plan(uf_tree *t, int64_t rows);
Plan::Dev &plan_dev(Plan *P, int device);

// ---- methods ----
// The accumulator and embedding a method runs on, and whether its distance
// is the numerator alone.
inline int acc_of(uf_method m) {
  return m == UF_GENERALIZED ? ACC_GEN
         : (m == UF_VAW_WEIGHTED_UNNORMALIZED || m == UF_VAW_WEIGHTED_NORMALIZED) ? ACC_VAW
                                                                                 : ACC_MIN;
}
inline int kind_of(uf_method m) {
  switch (m) {
  case UF_GENERALIZED: return EMB_PROP;
  case UF_UNWEIGHTED:
  case UF_UNWEIGHTED_UNNORMALIZED: return EMB_PRESENCE;
  case UF_VAW_WEIGHTED_UNNORMALIZED:
  case UF_VAW_WEIGHTED_NORMALIZED: return EMB_VAW;
  default: return EMB_SCALED;
  }
}
inline bool unnormalized(uf_method m) {
  return m == UF_WEIGHTED_UNNORMALIZED || m == UF_UNWEIGHTED_UNNORMALIZED || m == UF_VAW_WEIGHTED_UNNORMALIZED;
}

// ---- one compute call ----
// One table of a compute call: its stripe range and output.
struct TableJob {
  uf_table *table;
  int64_t start, stop;
  void *out;
  uf_report *rep;
};

// A compute call: one or more tables over one tree, one method and precision.
struct BatchJob {
  uf_method method;
  double alpha;
  bool fp32;
  int out_is_device, out_fp32;
  cudaStream_t st;
  std::vector<TableJob> tabs;
};

// Branches of a call split between the dense stripe kernels and the
// sparse-row pair kernel (uf_sparse.cu).
struct RowSplit {
  std::vector<int32_t> dense;       // dense branch nodes, block by block, ascending
  std::vector<int64_t> dense_ptr;   // per block: first index into dense (size blocks + 1)
  std::vector<double> dense_len;    // their branch lengths
  std::vector<std::vector<int32_t>> sparse;  // sparse branch nodes by capacity class
  std::vector<int> cap;             // shared-memory entries of each class
  bool lists = false;               // one table beyond L2: sample lists + stripe regions
  int64_t n_sparse = 0;
  double pairs = 0.0;               // both-nonzero pairs scattered, at most (sum over tables)
  int64_t max_dense = 0;            // most dense rows in one block
  // count rows the call needs: per block, a list of nodes built from their
  // tips' CSC columns (tips, and sparse branches under a dense parent), then
  // the dense internal nodes level by level; offsets into cnt_lists
  std::vector<int32_t> cnt_lists;
  std::vector<std::vector<std::pair<int64_t, int>>> cnt_launch;
};

// Stripe regions of a call's sparse scatter: one table whose accumulators
// exceed the L2 budget scatters region by region (launch_sparse_region) so
// that every region's cells stay in L2; otherwise one region.
constexpr double SPARSE_REGION_BYTES_DEFAULT = 48e6;
extern std::atomic<int64_t> g_region_bytes;
// split and region path: ACC_MIN or ACC_GEN (CUDA-core stripe kernels) or SPLIT_GRAM (tensor cores)
constexpr int SPLIT_GRAM = 2;
double sparse_regions(size_t n_tables, int acc, double acc_bytes);


// The split of a call, cached on the tree (uf_split.cpp).
std::shared_ptr<const RowSplit> get_split(uf_tree *tree, const BatchJob &J, const Plan *P, int acc, bool fp32);

// Runs one compute call on the current device (uf_run.cpp); throws CudaFail.
uf_status run_batch(uf_tree *tree, const BatchJob &J);
// Forgets the autotuned chunk sizes of this process (uf_run.cpp).
void forget_tuned_chunks();

}  // namespace rt
}  // namespace ufg
