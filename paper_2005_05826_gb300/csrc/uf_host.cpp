// uf_host.cpp -- host runtime behind the C ABI of include/unifrac_gb300.h.
//
// Validation of trees and tables, the postorder branch-block plan with
// level batching and live count slots, device residency of the inputs, and
// the orchestration of one uf_compute call:
//   per branch block: tip counts -> internal levels (children before parents)
//                     -> embedding rows -> stripe accumulate (+ diagonal)
//   then: finalize into the caller's output.
// Stripes are the paper's independent subproblems (Abstract; Sec. 2 Fig. 1).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <tuple>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <system_error>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/unifrac_gb300.h"
#include "uf_internal.h"

using namespace ufg;

namespace {

thread_local std::string g_err;

// Host threads for table preparation: the cores this process may run on, at most 16.
int host_threads() {
  const unsigned h = std::thread::hardware_concurrency();
  return (int)std::max(1u, std::min(h == 0 ? 1u : h, 16u));
}

// Runs body(0 .. n-1) on n threads (the calling thread takes the last) and joins.
template <typename F>
void parallel_for(int n, F body) {
  std::vector<std::thread> th;
  th.reserve(n > 1 ? n - 1 : 0);
  for (int c = 0; c + 1 < n; c++) th.emplace_back(body, c);
  body(n - 1);
  for (auto &x : th) x.join();
}

std::atomic<int64_t> g_branch_block{0};
std::atomic<int64_t> g_kernel_timing{0};
std::atomic<int64_t> g_tensor_path{1};
std::atomic<int64_t> g_graph{1};
std::atomic<int64_t> g_autotune{1};
std::atomic<int64_t> g_sparse{1};

uf_status fail(uf_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

struct CudaFail {
  uf_status st;
};

void ck(cudaError_t e, const char *what) {
  if (e != cudaSuccess) {
    cudaGetLastError();  // clear a sticky launch error where possible
    uf_status st = (e == cudaErrorMemoryAllocation) ? UF_ENOMEM : UF_ECUDA;
    fail(st, "%s: %s", what, cudaGetErrorString(e));
    throw CudaFail{st};
  }
}

thread_local double g_h2d = 0.0;  // bytes uploaded by the current call

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

template <typename T, typename Alloc>
T *dev_upload(const std::vector<T, Alloc> &h, const char *what) {
  g_h2d += (double)h.size() * sizeof(T);
  T *d = nullptr;
  size_t bytes = std::max<size_t>(h.size() * sizeof(T), 16);
  ck(cudaMalloc(&d, bytes), what);
  if (!h.empty()) {
    cudaError_t e = cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(d);
      ck(e, what);
    }
  }
  return d;
}

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
    int32_t *lists = nullptr, *slot_of_node = nullptr;
  };
  std::map<int, Dev> dev;
};

struct RowSplit;
// (table ids, accumulator, FP32, sparse mode, block rows, region budget)
using SplitKey = std::tuple<std::vector<uint64_t>, int, int, int, int64_t, int64_t>;

}  // namespace

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
    double *length = nullptr;
    int32_t *tip_of_node = nullptr, *child_ptr = nullptr, *child_idx = nullptr;
    int32_t *tip_lo = nullptr, *tip_hi = nullptr;
  };
  std::map<int, Dev> dev;
  std::map<int64_t, std::unique_ptr<Plan>> plans;  // by block rows
  std::map<SplitKey, std::shared_ptr<const RowSplit>> splits;  // dense / sparse branch splits
  // root distance of every node (root: 0), max over tips, total branch length
  std::vector<double> dist;
  double max_tip_dist = 0.0, total_length = 0.0;
  ~uf_tree() {
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto &kv : dev) {
      cudaSetDevice(kv.first);
      cudaFree(kv.second.length);
      cudaFree(kv.second.tip_of_node);
      cudaFree(kv.second.child_ptr);
      cudaFree(kv.second.child_idx);
      cudaFree(kv.second.tip_lo);
      cudaFree(kv.second.tip_hi);
    }
    for (auto &p : plans)
      for (auto &kv : p.second->dev) {
        cudaSetDevice(kv.first);
        cudaFree(kv.second.lists);
        cudaFree(kv.second.slot_of_node);
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
  std::vector<int32_t, NoInit<int32_t>> col_row;
  std::vector<double, NoInit<double>> col_val;
  std::mutex mu;
  std::map<uint64_t, double> presence_bound;  // by tree id: max_k sum_{f in k} dist(tip f)
  struct Dev {
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
      cudaFree(kv.second.total);
      cudaFree(kv.second.col_val);
      cudaFree(kv.second.inv_total_f);
      cudaFree(kv.second.col_ptr);
      cudaFree(kv.second.col_row);
    }
    cudaSetDevice(cur);
  }
};

namespace {

uf_tree::Dev &tree_dev(uf_tree *t, int device) {
  auto it = t->dev.find(device);
  if (it != t->dev.end()) return it->second;
  uf_tree::Dev d;
  try {
    d.length = dev_upload(t->length, "tree upload");
    d.tip_of_node = dev_upload(t->tip_of_node, "tree upload");
    d.child_ptr = dev_upload(t->child_ptr, "tree upload");
    d.child_idx = dev_upload(t->child_idx, "tree upload");
    d.tip_lo = dev_upload(t->tip_lo, "tree upload");
    d.tip_hi = dev_upload(t->tip_hi, "tree upload");
  } catch (...) {
    cudaFree(d.length);
    cudaFree(d.tip_of_node);
    cudaFree(d.child_ptr);
    cudaFree(d.child_idx);
    cudaFree(d.tip_lo);
    cudaFree(d.tip_hi);
    throw;
  }
  return t->dev[device] = d;
}

uf_table::Dev &table_dev(uf_table *t, int device) {
  auto it = t->dev.find(device);
  if (it != t->dev.end()) return it->second;
  uf_table::Dev d;
  try {
    d.total = dev_upload(t->total, "table upload");
    d.inv_total_f = dev_upload(t->inv_total_f, "table upload");
    d.col_ptr = dev_upload(t->col_ptr, "table upload");
    d.col_row = dev_upload(t->col_row, "table upload");
    d.col_val = dev_upload(t->col_val, "table upload");
  } catch (...) {
    cudaFree(d.total);
    cudaFree(d.inv_total_f);
    cudaFree(d.col_ptr);
    cudaFree(d.col_row);
    cudaFree(d.col_val);
    throw;
  }
  return t->dev[device] = d;
}

// Build the branch-block plan: blocks of `rows` consecutive postorder nodes;
// inside a block, tips first, then internal nodes by level (a node's level is
// one more than its deepest internal child in the same block); one count
// slot per node, freed at the end of the block that computes its parent.
Plan *get_plan(uf_tree *t, int64_t rows) {
  auto it = t->plans.find(rows);
  if (it != t->plans.end()) return it->second.get();
  auto P = std::make_unique<Plan>();
  P->block_rows = rows;
  const int64_t nb = t->n_nodes - 1;  // branches: every node but the root
  P->slot_of_node.assign(t->n_nodes, -1);
  std::vector<int32_t> level(t->n_nodes, 0);
  std::vector<int32_t> free_slots;
  int32_t next_slot = 0;
  std::vector<int64_t> release;  // nodes whose slot goes back at block end
  for (int64_t b0 = 0; b0 < nb; b0 += rows) {
    const int64_t b1 = std::min(nb, b0 + rows);
    P->b0.push_back(b0);
    P->b1.push_back(b1);
    std::vector<std::vector<int32_t>> lv(1);  // lv[0] = tips
    for (int64_t v = b0; v < b1; v++) {
      if (t->tip_of_node[v] >= 0) {
        lv[0].push_back((int32_t)v);
        continue;
      }
      int32_t L = 0;
      for (int32_t c = t->child_ptr[v]; c < t->child_ptr[v + 1]; c++) {
        const int32_t ch = t->child_idx[c];
        if (ch >= b0 && t->tip_of_node[ch] < 0) L = std::max(L, level[ch] + 1);
      }
      level[v] = L;
      if ((int)lv.size() < L + 2) lv.resize(L + 2);
      lv[L + 1].push_back((int32_t)v);
    }
    // slots for the block's nodes
    for (int64_t v = b0; v < b1; v++) {
      int32_t s;
      if (!free_slots.empty()) {
        s = free_slots.back();
        free_slots.pop_back();
      } else {
        s = next_slot++;
      }
      P->slot_of_node[v] = s;
    }
    std::vector<std::pair<int64_t, int>> ls;
    for (auto &l : lv) {
      ls.emplace_back((int64_t)P->lists.size(), (int)l.size());
      P->lists.insert(P->lists.end(), l.begin(), l.end());
    }
    P->launches.push_back(std::move(ls));
    // release: children of this block's internal nodes, and nodes whose
    // parent is the root (never read again)
    for (int64_t v = b0; v < b1; v++) {
      for (int32_t c = t->child_ptr[v]; c < t->child_ptr[v + 1]; c++)
        free_slots.push_back(P->slot_of_node[t->child_idx[c]]);
      if (t->parent[v] == t->n_nodes - 1) free_slots.push_back(P->slot_of_node[v]);
    }
  }
  P->n_slots = next_slot;
  Plan *raw = P.get();
  t->plans[rows] = std::move(P);
  return raw;
}

Plan::Dev &plan_dev(Plan *P, int device) {
  auto it = P->dev.find(device);
  if (it != P->dev.end()) return it->second;
  Plan::Dev d;
  try {
    d.lists = dev_upload(P->lists, "plan upload");
    d.slot_of_node = dev_upload(P->slot_of_node, "plan upload");
  } catch (...) {
    cudaFree(d.lists);
    throw;
  }
  return P->dev[device] = d;
}

struct DevBuf {
  void *p = nullptr;
  cudaStream_t st = nullptr;
  DevBuf() = default;
  DevBuf(size_t bytes, cudaStream_t s, const char *what) : st(s) {
    ck(cudaMallocAsync(&p, std::max<size_t>(bytes, 256), s), what);
  }
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  DevBuf(DevBuf &&o) noexcept : p(o.p), st(o.st) { o.p = nullptr; }
  DevBuf &operator=(DevBuf &&o) noexcept {
    std::swap(p, o.p);
    std::swap(st, o.st);
    return *this;
  }
  ~DevBuf() {
    if (p) cudaFreeAsync(p, st);
  }
  template <typename T>
  T *as() const { return (T *)p; }
};

// Pinned staging for the per-call metadata uploads (table descriptors, row
// lists): a cudaMemcpyAsync from pageable memory first waits for all earlier
// work on the stream, one from pinned memory does not, so consecutive calls
// on one stream overlap their host work with the previous call's kernels.
// One ring per process; a region is reused only after the event recorded
// behind its copy has completed.  The buffer lives until the process ends.
struct Staging {
  std::mutex mu;
  char *buf = nullptr;
  size_t cap = 0, head = 0;
  std::vector<std::tuple<size_t, size_t, cudaEvent_t>> live;  // [begin, end) copies in flight
};
Staging g_stage;

void staged_upload(void *dst, const void *src, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return;
  Staging &S = g_stage;
  std::lock_guard<std::mutex> g(S.mu);
  const size_t need = (bytes + 255) & ~(size_t)255;
  auto retire = [&](bool all, size_t b, size_t e) {
    for (size_t i = 0; i < S.live.size();) {
      const size_t lb = std::get<0>(S.live[i]), le = std::get<1>(S.live[i]);
      cudaEvent_t ev = std::get<2>(S.live[i]);
      const bool overlap = all || (lb < e && b < le);
      if (overlap) ck(cudaEventSynchronize(ev), "staging wait");
      if (overlap || cudaEventQuery(ev) == cudaSuccess) {
        cudaEventDestroy(ev);
        S.live[i] = S.live.back();
        S.live.pop_back();
      } else {
        cudaGetLastError();  // cudaErrorNotReady is not an error here
        i++;
      }
    }
  };
  if (need > S.cap) {
    retire(true, 0, 0);
    if (S.buf) cudaFreeHost(S.buf);
    S.buf = nullptr;
    S.cap = 0;
    const size_t cap = std::max<size_t>(need, (size_t)16 << 20);
    ck(cudaMallocHost((void **)&S.buf, cap), "alloc pinned staging");
    S.cap = cap;
    S.head = 0;
  }
  if (S.head + need > S.cap) S.head = 0;
  const size_t b = S.head, e = b + need;
  retire(false, b, e);
  memcpy(S.buf + b, src, bytes);
  ck(cudaMemcpyAsync(dst, S.buf + b, bytes, cudaMemcpyHostToDevice, st), "upload");
  cudaEvent_t ev;
  ck(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "cudaEventCreate");
  ck(cudaEventRecord(ev, st), "cudaEventRecord");
  S.live.emplace_back(b, e, ev);
  S.head = e;
}

// Per-call metadata packed into one device buffer with one staged upload.
struct Meta {
  std::vector<char> host;
  template <typename T>
  size_t add(const T *p, size_t n) {
    const size_t off = (host.size() + 255) & ~(size_t)255;
    host.resize(off + std::max<size_t>(n * sizeof(T), 1));
    if (n) memcpy(host.data() + off, p, n * sizeof(T));
    return off;
  }
  template <typename T>
  size_t add(const std::vector<T> &v) { return add(v.data(), v.size()); }
  DevBuf dev;
  void upload(cudaStream_t st) {
    dev = DevBuf(host.size(), st, "alloc call metadata");
    staged_upload(dev.p, host.data(), host.size(), st);
  }
  template <typename T>
  T *at(size_t off) const { return (T *)((char *)dev.p + off); }
};

void keep_pool_memory(int device) {
  static std::mutex mu;
  static std::map<int, bool> done;
  std::lock_guard<std::mutex> g(mu);
  if (done[device]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  done[device] = true;
}

int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// Phase timer: CUDA events recorded on the call's stream around each phase.
struct PhaseTimer {
  bool on;
  cudaStream_t st;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> marks;
  cudaEvent_t open_ev = nullptr;
  cudaStream_t open_st = nullptr;
  int open_phase = -1;
  PhaseTimer(bool enabled, cudaStream_t s) : on(enabled), st(s) {}
  // a phase is timed on the stream its launches go to (the call's stream by default)
  void begin(int phase, cudaStream_t on_stream = nullptr) {
    if (!on) return;
    open_st = on_stream ? on_stream : st;
    ck(cudaEventCreate(&open_ev), "cudaEventCreate");
    ck(cudaEventRecord(open_ev, open_st), "cudaEventRecord");
    open_phase = phase;
  }
  void end() {
    if (!on) return;
    cudaEvent_t e;
    ck(cudaEventCreate(&e), "cudaEventCreate");
    ck(cudaEventRecord(e, open_st), "cudaEventRecord");
    marks.push_back({open_phase, {open_ev, e}});
    open_ev = nullptr;
  }
  // after the stream is synchronized
  void collect(double *ms4) {
    for (auto &m : marks) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, m.second.first, m.second.second) == cudaSuccess) ms4[m.first] += t;
    }
  }
  ~PhaseTimer() {
    for (auto &m : marks) {
      cudaEventDestroy(m.second.first);
      cudaEventDestroy(m.second.second);
    }
    if (open_ev) cudaEventDestroy(open_ev);
  }
};

// Upper bound on every value an accumulator of this kind can reach:
//   l * p embeddings:         D_k = sum_f p_f dist(f) <= max tip distance
//   l * presence embeddings:  W_k <= min(total length, sum_{f in k} dist(f))
//   generalized (den, Q):     den <= sum l s^alpha <= 2 (W_k + W_j)
double accum_bound(uf_tree *tree, uf_table *table, int kind) {
  if (kind == EMB_SCALED) return tree->max_tip_dist;
  double pres;
  {
    std::lock_guard<std::mutex> g(table->mu);
    auto it = table->presence_bound.find(tree->id);
    if (it == table->presence_bound.end()) {
      std::vector<int32_t> tip_node(tree->n_tips);
      for (int64_t v = 0; v < tree->n_nodes; v++)
        if (tree->tip_of_node[v] >= 0) tip_node[tree->tip_of_node[v]] = (int32_t)v;
      // per-sample sums over feature ranges of about equal entries, one per thread
      const int T = (int)std::max<int64_t>(1, std::min<int64_t>(host_threads(), table->nnz / 200000));
      std::vector<int64_t> f_lo(T + 1, table->n_features);
      f_lo[0] = 0;
      for (int c = 1, f = 0; c < T; c++) {
        const int64_t want = table->nnz * c / T;
        while (f < table->n_features && table->col_ptr[f] < want) f++;
        f_lo[c] = f;
      }
      std::vector<std::vector<double>> part(T, std::vector<double>(table->n, 0.0));
      parallel_for(T, [&](int c) {
        double *per = part[c].data();
        for (int64_t f = f_lo[c]; f < f_lo[c + 1]; f++) {
          const double d = tree->dist[tip_node[f]];
          for (int64_t q = table->col_ptr[f]; q < table->col_ptr[f + 1]; q++) per[table->col_row[q]] += d;
        }
      });
      double mx = 0.0;
      for (int64_t k = 0; k < table->n; k++) {
        double x = 0.0;
        for (int c = 0; c < T; c++) x += part[c][k];
        mx = std::max(mx, x);
      }
      it = table->presence_bound.emplace(tree->id, mx).first;
    }
    pres = std::min(tree->total_length, it->second);
  }
  return kind == EMB_PRESENCE ? pres : 4.0 * pres;
}

}  // namespace

namespace ufg {
// Fixed-point scale 2^F of the accumulators: 2 * bound * 2^F <= 2^61.
double accum_scale(const uf_tree *tree, const uf_table *table, int kind) {
  const double B = accum_bound(const_cast<uf_tree *>(tree), const_cast<uf_table *>(table), kind);
  int F = 100;
  if (B > 0.0 && std::isfinite(B)) F = std::min(100, std::max(0, 60 - (int)std::ceil(std::log2(B))));
  return std::ldexp(1.0, F);
}
}  // namespace ufg

namespace {

// Private stream of the calling thread per device on which a call's launch
// sequence is captured into a CUDA graph.  Per thread, so that concurrent
// calls from several threads never share a capturing stream.
struct ThreadStreams {
  std::map<int, cudaStream_t> s;
  ~ThreadStreams() {
    for (auto &kv : s) cudaStreamDestroy(kv.second);
  }
};
thread_local ThreadStreams t_streams;

cudaStream_t capture_stream(int device) {
  auto it = t_streams.s.find(device);
  if (it != t_streams.s.end()) return it->second;
  cudaStream_t x = nullptr;
  ck(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking), "cudaStreamCreate");
  t_streams.s[device] = x;
  return x;
}

// Records the branch-block launch sequence of a call into a CUDA graph (on a
// private stream) and launches that graph on the caller's stream; when off,
// launches go to the caller's stream directly.
struct Capture {
  bool on;
  cudaStream_t user, cap = nullptr;
  bool open = false;
  Capture(bool enable, cudaStream_t st, int device) : on(enable), user(st) {
    if (!on) return;
    cap = capture_stream(device);
    ck(cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed), "cudaStreamBeginCapture");
    open = true;
  }
  cudaStream_t stream() const { return on ? cap : user; }
  // end the capture and launch the graph on the caller's stream
  void launch() {
    if (!on) return;
    cudaGraph_t g = nullptr;
    open = false;
    ck(cudaStreamEndCapture(cap, &g), "cudaStreamEndCapture");
    cudaGraphExec_t e = nullptr;
    cudaError_t err = cudaGraphInstantiate(&e, g, 0);
    if (err == cudaSuccess) err = cudaGraphLaunch(e, user);
    if (e) cudaGraphExecDestroy(e);  // freed once the launch completes
    cudaGraphDestroy(g);
    ck(err, "graph launch");
  }
  ~Capture() {
    if (open) {  // an error escaped mid-capture: drop the partial graph
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(cap, &g);
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
    }
  }
};

// Autotuned rows per work unit, by (accumulator, precision, size bucket).
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, int> g_tuned_chunk;

std::tuple<int, int, int, int> tune_key(int acc, bool fp32, int64_t n_tiles, int64_t rows) {
  auto lg = [](int64_t x) { return (int)std::floor(std::log2((double)std::max<int64_t>(x, 1))); };
  return {acc, fp32 ? 1 : 0, lg(n_tiles), lg(rows)};
}

// Time the accumulate launch of the first block with each candidate chunk
// size and keep the fastest (the accumulators are cleared afterwards).
int tune_chunk(int acc, bool fp32, StripeArgs sa, size_t cells, cudaStream_t st) {
  const int cand[4] = {1024, 2048, 4096, 8192};
  cudaEvent_t e0, e1;
  ck(cudaEventCreate(&e0), "cudaEventCreate");
  ck(cudaEventCreate(&e1), "cudaEventCreate");
  int best = stripe_chunk_rows();
  float best_ms = 1e30f;
  for (int c : cand) {
    if (c > 2 * std::max(sa.rows, 1024)) break;
    sa.chunk = c;
    ck(cudaEventRecord(e0, st), "cudaEventRecord");
    ck(launch_stripe_acc(acc, fp32, sa, st), "autotune");
    ck(cudaEventRecord(e1, st), "cudaEventRecord");
    ck(cudaEventSynchronize(e1), "cudaEventSynchronize");
    float ms = 0.f;
    ck(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ck(cudaMemsetAsync(sa.M, 0, cells * 8, st), "memset");
  if (sa.M2) ck(cudaMemsetAsync(sa.M2, 0, cells * 8, st), "memset");
  return best;
}

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

// Device copies of the inputs and the per-sample arrays on the combined axis.
struct Inputs {
  uf_tree::Dev *td = nullptr;
  Plan *P = nullptr;
  Plan::Dev *pd = nullptr;
  std::vector<uf_table::Dev *> xd;
};

Inputs bind_inputs(uf_tree *tree, const BatchJob &J, int device, int64_t rows) {
  Inputs in;
  {
    std::lock_guard<std::mutex> g(tree->mu);
    in.td = &tree_dev(tree, device);
    in.P = get_plan(tree, rows);
    in.pd = &plan_dev(in.P, device);
  }
  for (const TableJob &t : J.tabs) {
    std::lock_guard<std::mutex> g(t.table->mu);
    in.xd.push_back(&table_dev(t.table, device));
  }
  return in;
}

// Branch rows per embedding block for a working budget of per_row bytes a row
// plus fixed bytes.
int64_t block_rows(int64_t nb, double per_row, double fixed) {
  size_t free_b = 0, total_b = 0;
  ck(cudaMemGetInfo(&free_b, &total_b), "cudaMemGetInfo");
  const double budget = std::min(0.5 * (double)free_b - fixed, 24e9);
  int64_t rows = (int64_t)(budget / per_row / 1.1);
  rows = std::max<int64_t>(std::min<int64_t>(rows, nb), std::min<int64_t>(nb, 256));
  if (g_branch_block.load() > 0) rows = std::min<int64_t>(g_branch_block.load(), std::max<int64_t>(nb, 1));
  return std::max<int64_t>(rows, 1);
}

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

// Per branch v the count entries of table t under v are the CSC run of v's
// tips, ub_t(v) = col_ptr_t[tip_hi] - col_ptr_t[tip_lo] (an upper bound on the
// nonzero samples, exact when no two tips share a sample).  Mode 1 scatters
// v when the modelled time of its pairs is below that of a dense pass over
// its stripe cells; the rates are GB300 measurements of the two kernels and
// of global 64-bit atomics (L2-resident accumulators or not).  Mode 2
// scatters every branch that fits; mode 0 none.  The choice depends on the
// tree and the tables only, not on the stripe range, so that a range run
// gives bitwise the stripes of the full run.
// Stripe regions of a call's sparse scatter: one table whose accumulators
// exceed the L2 budget scatters region by region (launch_sparse_region) so
// that every region's cells stay in L2; otherwise one region.
constexpr double SPARSE_REGION_BYTES_DEFAULT = 48e6;
std::atomic<int64_t> g_region_bytes{(int64_t)SPARSE_REGION_BYTES_DEFAULT};
// split and region path: ACC_MIN or ACC_GEN (CUDA-core stripe kernels) or SPLIT_GRAM (tensor cores)
constexpr int SPLIT_GRAM = 2;
double sparse_regions(size_t n_tables, int acc, double acc_bytes) {
  const double budget = (double)g_region_bytes.load();
  if (n_tables != 1 || acc == SPLIT_GRAM || acc_bytes <= budget) return 1.0;
  return std::ceil(acc_bytes / budget);
}

RowSplit split_rows(const uf_tree *tree, const BatchJob &J, const Plan *P, int acc, bool fp32) {
  RowSplit R;
  const int mode = (int)g_sparse.load();
  const int64_t nb = tree->n_nodes - 1;
  const size_t nt = J.tabs.size();
  const int classes[5] = {128, 512, 2048, SPARSE_MAX_ENTRIES, SPARSE_LIST_MAX_ENTRIES};
  R.cap.assign(classes, classes + 5);
  R.sparse.resize(5);
  std::vector<char> is_sparse(std::max<int64_t>(nb, 1), 0);
  if (mode != 0) {
    const int n_acc = acc == ACC_GEN ? 2 : 1;
    double cells = 0.0, cols = 0.0;  // stripe cells of a full run of every table; samples
    for (size_t t = 0; t < nt; t++) {
      const double n = (double)J.tabs[t].table->n;
      cells += std::floor(n / 2.0) * n;
      cols += n;
    }
    // accumulators beyond L2: one table scatters region by region in L2
    // (sparse_regions), several tables scatter straight into HBM-resident cells
    const bool regions = sparse_regions(nt, acc, cells * 8.0 * n_acc) > 1;
    R.lists = regions;
    // list mode keeps only sort keys in shared memory: longer runs fit
    const int64_t max_entries = regions ? SPARSE_LIST_MAX_ENTRIES : SPARSE_MAX_ENTRIES;
    const double atom_rate = cells * 8.0 * n_acc <= 64e6 || regions ? 2.3e11 : 2.5e10;
    const double n_regions = regions ? sparse_regions(nt, acc, cells * 8.0 * n_acc) : 1.0;
    double dense_rate;  // cell updates per second of the dense kernel
    if (acc == SPLIT_GRAM) dense_rate = 2.5e14;
    else dense_rate = fp32 ? (acc == ACC_GEN ? 4e12 : 1.3e13) : (acc == ACC_GEN ? 5e10 : 2e11);
    const double visit_rate = fp32 ? 2e12 : (acc == ACC_GEN ? 3e10 : 1e12);
    const double job_cost = 5e-10;
    // a dense row also costs its count row and embedding (or planes) in HBM
    const double dense_t = cells / dense_rate + cols * 36.0 / 6e12;
    for (int64_t v = 0; v < nb; v++) {
      const int32_t lo = tree->tip_lo[v], hi = tree->tip_hi[v];
      if (lo < 0) continue;
      if (tree->length[v] == 0.0) {
        // a zero-length branch adds exactly 0 to every accumulator: skipped
        // (its count row is still built if a dense parent needs it)
        is_sparse[v] = 1;
        R.n_sparse++;
        continue;
      }
      double cost = 0.0, pairs = 0.0;
      int64_t mx = 0;
      for (size_t t = 0; t < nt; t++) {
        const auto &cp = J.tabs[t].table->col_ptr;
        const int64_t ub = cp[hi] - cp[lo];
        mx = std::max(mx, ub);
        if (ub == 0) continue;
        const double pr = (double)ub * (double)(ub - 1) / 2.0;
        pairs += pr;
        cost += job_cost + pr * (1.0 / visit_rate + n_acc / atom_rate) + (double)ub * 4.0 / atom_rate;
        if (regions) cost += n_regions * (job_cost + (double)ub * 4e-11);  // one visit per region
      }
      if (mx > max_entries) continue;
      if (mode == 2 || cost < dense_t) {
        is_sparse[v] = 1;
        int c = 0;
        while (classes[c] < mx) c++;
        R.sparse[c].push_back((int32_t)v);
        R.n_sparse++;
        R.pairs += pairs;
      }
    }
  }
  const int64_t root = tree->n_nodes - 1;
  auto parent_dense = [&](int64_t v) {
    const int64_t p = tree->parent[v];
    return p != root && !is_sparse[p];
  };
  for (size_t b = 0; b < P->b0.size(); b++) {
    const auto &ls = P->launches[b];
    std::vector<std::pair<int64_t, int>> lb;
    std::vector<int32_t> level;
    // nodes built from CSC columns
    level.clear();
    for (size_t l = 0; l < ls.size(); l++)
      for (int i = 0; i < ls[l].second; i++) {
        const int32_t v = P->lists[ls[l].first + i];
        const bool tip = l == 0;
        if (is_sparse[v] ? parent_dense(v) : tip) level.push_back(v);
      }
    lb.emplace_back((int64_t)R.cnt_lists.size(), (int)level.size());
    R.cnt_lists.insert(R.cnt_lists.end(), level.begin(), level.end());
    // dense internal nodes by level
    for (size_t l = 1; l < ls.size(); l++) {
      level.clear();
      for (int i = 0; i < ls[l].second; i++) {
        const int32_t v = P->lists[ls[l].first + i];
        if (!is_sparse[v]) level.push_back(v);
      }
      if (level.empty()) continue;
      lb.emplace_back((int64_t)R.cnt_lists.size(), (int)level.size());
      R.cnt_lists.insert(R.cnt_lists.end(), level.begin(), level.end());
    }
    R.cnt_launch.push_back(std::move(lb));
  }
  R.dense_ptr.push_back(0);
  for (size_t b = 0; b < P->b0.size(); b++) {
    for (int64_t v = P->b0[b]; v < P->b1[b]; v++)
      if (!is_sparse[v]) {
        R.dense.push_back((int32_t)v);
        R.dense_len.push_back(tree->length[v]);
      }
    R.dense_ptr.push_back((int64_t)R.dense.size());
    R.max_dense = std::max(R.max_dense, R.dense_ptr[b + 1] - R.dense_ptr[b]);
  }
  return R;
}

// The split of a call, cached on the tree by its tables and kind (tables are
// immutable and their ids are never reused).
std::shared_ptr<const RowSplit> get_split(uf_tree *tree, const BatchJob &J, const Plan *P, int acc, bool fp32) {
  SplitKey key;
  for (const TableJob &t : J.tabs) std::get<0>(key).push_back(t.table->id);
  std::get<1>(key) = acc;
  std::get<2>(key) = fp32 ? 1 : 0;
  std::get<3>(key) = (int)g_sparse.load();
  std::get<4>(key) = P->block_rows;
  std::get<5>(key) = g_region_bytes.load();
  std::lock_guard<std::mutex> g(tree->mu);
  auto it = tree->splits.find(key);
  if (it != tree->splits.end()) return it->second;
  if (tree->splits.size() >= 16) tree->splits.clear();
  auto sp = std::make_shared<const RowSplit>(split_rows(tree, J, P, acc, fp32));
  tree->splits.emplace(key, sp);
  return sp;
}

// Output buffers: the caller's device memory, or a device staging buffer
// copied to the caller's host memory at the end.
struct Outputs {
  std::vector<DevBuf> tmp;
  std::vector<void *> dev;
  std::vector<size_t> bytes;
};

Outputs bind_outputs(const BatchJob &J, cudaStream_t st) {
  Outputs o;
  for (const TableJob &t : J.tabs) {
    const int64_t n = t.table->n, S = n / 2;
    const bool full = t.start == 0 && t.stop == S;
    const size_t elems = full ? (size_t)n * (n - 1) / 2 : (size_t)(t.stop - t.start) * n;
    o.bytes.push_back(elems * (J.out_fp32 ? 4 : 8));
    if (J.out_is_device) {
      o.tmp.emplace_back();
      o.dev.push_back(t.out);
    } else {
      o.tmp.emplace_back(o.bytes.back(), st, "alloc output");
      o.dev.push_back(o.tmp.back().p);
    }
  }
  return o;
}

void fill_reports(uf_tree *tree, const BatchJob &J, const Outputs &o, double ms[4], int64_t kernels,
                  int64_t acc_launches, int path, int64_t rows, int64_t n_blocks, double exec_flops,
                  int tile_s, int tile_k, double seconds) {
  const int64_t nb = tree->n_nodes - 1;
  for (size_t t = 0; t < J.tabs.size(); t++) {
    if (!J.tabs[t].rep) continue;
    uf_report &r = *J.tabs[t].rep;
    memset(&r, 0, sizeof r);
    const int64_t n = J.tabs[t].table->n, S = n / 2;
    const bool full = J.tabs[t].start == 0 && J.tabs[t].stop == S;
    const int64_t rows_out = J.tabs[t].stop - J.tabs[t].start;
    const double pairs = full ? (double)n * (n - 1) / 2.0
                              : (double)rows_out * n - ((2 * J.tabs[t].stop == n) ? n / 2.0 : 0.0);
    r.updates = pairs * (double)nb;
    r.alg_flops = 2.0 * pairs * nb;
    r.exec_flops = exec_flops / (double)J.tabs.size();
    r.hbm_bytes_est = (double)nb * (double)n * 8 * 3 + (double)o.bytes[t];
    r.stripe_tile = tile_s;
    r.sample_tile = tile_k;
    r.branch_block = rows;
    r.n_blocks = n_blocks;
    r.kernels = kernels;
    r.path = path;
    r.h2d_bytes = g_h2d;
    r.d2h_bytes = J.out_is_device ? 0.0 : (double)o.bytes[t];
    r.t_embed_ms = ms[0];
    r.t_accumulate_ms = ms[1];
    r.t_diag_ms = ms[2];
    r.t_finalize_ms = ms[3];
    r.acc_launches = acc_launches;
    r.seconds = seconds;
  }
}

// Count rows of block b that the split needs: CSC-built nodes of every
// table, then the dense internal levels over the combined axis.
void enqueue_split_counts(const Inputs &in, const BatchJob &J, const std::vector<int> &off, const RowSplit &split,
                          size_t b, const int32_t *d_cnt, double *counts, int64_t ld, cudaStream_t st,
                          int64_t *kernels) {
  const auto &lb = split.cnt_launch[b];
  for (size_t t = 0; t < J.tabs.size(); t++) {
    ck(launch_slice_counts(d_cnt + lb[0].first, lb[0].second, in.td->tip_lo, in.td->tip_hi, in.pd->slot_of_node,
                           in.xd[t]->col_ptr, in.xd[t]->col_row, in.xd[t]->col_val, counts + off[t], ld,
                           (int)J.tabs[t].table->n, st),
       "count rows");
    *kernels += lb[0].second > 0;
  }
  for (size_t l = 1; l < lb.size(); l++) {
    ck(launch_node_counts(d_cnt + lb[l].first, lb[l].second, in.td->child_ptr, in.td->child_idx,
                          in.pd->slot_of_node, counts, ld, st),
       "node counts");
    (*kernels)++;
  }
}

// Unweighted, mixed precision, on the tensor cores: per branch block, counts
// -> presence / split-length planes of every table -> tcgen05 gram; then the
// gram finalize of every table.  Throws CudaFail on CUDA errors.
uf_status run_gram(uf_tree *tree, const BatchJob &J, int device, double scale, double t0_dummy) {
  (void)t0_dummy;
  const auto t_start = std::chrono::steady_clock::now();
  const size_t nt = J.tabs.size();
  std::vector<int> off(nt);
  std::vector<GramTab> gt(nt);
  std::vector<int32_t> tile_tab, tile_bi, tile_bj;
  int n_cols = 0, npad_tot = 0;
  int64_t gt_cells = 0;
  for (size_t t = 0; t < nt; t++) {
    const int n = (int)J.tabs[t].table->n;
    off[t] = n_cols;
    gt[t].n = n;
    gt[t].n_pad = gram_pad(n);
    gt[t].row_base = npad_tot;
    gt[t].off = n_cols;
    gt[t].gt_off = gt_cells;
    const size_t before = tile_bi.size();
    gram_tiles(gt[t].n_pad, &tile_bi, &tile_bj);
    tile_tab.insert(tile_tab.end(), tile_bi.size() - before, (int32_t)t);
    n_cols += n;
    npad_tot += gt[t].n_pad;
    gt_cells += (int64_t)gt[t].n_pad * gt[t].n_pad;
  }
  const int n_tiles = (int)tile_bi.size();
  const int64_t nb = tree->n_nodes - 1;
  const int64_t rows = block_rows(nb, (double)n_cols * 8.0 + 4.0 * npad_tot * 2.0 + 8.0, (double)gt_cells * 8.0);
  Inputs in = bind_inputs(tree, J, device, rows);
  const std::shared_ptr<const RowSplit> split_p = get_split(tree, J, in.P, SPLIT_GRAM, true);
  const RowSplit &split = *split_p;
  const int64_t K_pad = gram_kpad((int)std::max<int64_t>(split.max_dense, 1));
  cudaStream_t st = J.st;
  int64_t kernels = 0, acc_launches = 0;
  PhaseTimer timer(g_kernel_timing.load() != 0, st);
  std::vector<int32_t> tl(tile_tab);
  tl.insert(tl.end(), tile_bi.begin(), tile_bi.end());
  tl.insert(tl.end(), tile_bj.begin(), tile_bj.end());
  DevBuf counts((size_t)in.P->n_slots * n_cols * 8, st, "alloc counts");
  DevBuf Pl((size_t)4 * npad_tot * K_pad * 2, st, "alloc presence planes");
  DevBuf Gt((size_t)gt_cells * 8, st, "alloc gram");
  DevBuf err(sizeof(int), st, "alloc error flag");
  Meta meta;  // tile list, table descriptors and row lists: one staged upload
  const size_t o_tiles = meta.add(tl), o_tabs = meta.add(gt);
  const size_t o_cnt = meta.add(split.cnt_lists), o_dense = meta.add(split.dense);
  std::vector<int64_t> sp_off;
  size_t o_sparse = 0, o_sptabs = 0;
  if (split.n_sparse > 0) {
    std::vector<int32_t> all;
    for (const auto &c : split.sparse) {
      sp_off.push_back((int64_t)all.size());
      all.insert(all.end(), c.begin(), c.end());
    }
    std::vector<SpTab> sp(nt);
    for (size_t t = 0; t < nt; t++) {
      sp[t].col_ptr = in.xd[t]->col_ptr;
      sp[t].col_row = in.xd[t]->col_row;
      sp[t].col_val = in.xd[t]->col_val;
      sp[t].total = in.xd[t]->total;
      sp[t].inv_total_f = in.xd[t]->inv_total_f;
      sp[t].n = gt[t].n;
      sp[t].off = gt[t].off;
      sp[t].m_off = gt[t].gt_off;
      sp[t].n_pad = gt[t].n_pad;
    }
    o_sparse = meta.add(all);
    o_sptabs = meta.add(sp);
  }
  meta.upload(st);
  const int32_t *d_tiles = meta.at<int32_t>(o_tiles);
  const GramTab *d_tabs = meta.at<GramTab>(o_tabs);
  const int32_t *d_cnt = meta.at<int32_t>(o_cnt), *d_dense = meta.at<int32_t>(o_dense);
  ck(cudaMemsetAsync(Gt.p, 0, (size_t)gt_cells * 8, st), "memset");
  ck(cudaMemsetAsync(err.p, 0, sizeof(int), st), "memset");
  Outputs o = bind_outputs(J, st);
  double exec_flops = 0.0;
  Capture cap(g_graph.load() != 0 && !timer.on, st, device);
  const cudaStream_t ls = cap.stream();
  // the sparse-row scatters need no count rows or planes: first
  if (split.n_sparse > 0) {
    timer.begin(4);
    for (size_t c = 0; c < split.sparse.size(); c++) {
      if (split.sparse[c].empty()) continue;
      SparseArgs sp{};
      sp.nodes = meta.at<int32_t>(o_sparse) + sp_off[c];
      sp.n_nodes = (int)split.sparse[c].size();
      sp.cap = split.cap[c];
      sp.tip_lo = in.td->tip_lo;
      sp.tip_hi = in.td->tip_hi;
      sp.length = in.td->length;
      sp.tabs = meta.at<SpTab>(o_sptabs);
      sp.n_tabs = (int)nt;
      sp.kind = EMB_PRESENCE;
      sp.gram = 1;
      sp.M = Gt.as<unsigned long long>();
      sp.alpha = 1.0;
      sp.scale = scale;
      ck(launch_sparse_rows(ACC_MIN, false, sp, ls), "sparse rows");
      kernels++;
    }
    timer.end();
  }
  for (size_t b = 0; b < in.P->b0.size(); b++) {
    const int64_t b0 = in.P->b0[b];
    const int64_t d0 = split.dense_ptr[b], nd = split.dense_ptr[b + 1] - d0;
    timer.begin(0);
    enqueue_split_counts(in, J, off, split, b, d_cnt, counts.as<double>(), n_cols, ls, &kernels);
    if (nd > 0) {
      ck(launch_gram_prep(b0, (int)nd, in.pd->slot_of_node, counts.as<double>(), n_cols, in.td->length, d_tabs,
                          (int)nt, npad_tot, K_pad, Pl.p, ls, d_dense + d0),
         "presence planes");
      kernels++;
    }
    timer.end();
    if (nd == 0) continue;
    GramArgs ga{};
    ga.k_len = (int)round_up(nd, 64);
    ga.kc = 4096;
    ga.n_tiles = n_tiles;
    ga.npad_tot = npad_tot;
    ga.tile_tab = d_tiles;
    ga.tile_bi = d_tiles + n_tiles;
    ga.tile_bj = d_tiles + 2 * n_tiles;
    ga.tabs = d_tabs;
    ga.Gt = Gt.as<unsigned long long>();
    ga.scale = scale;
    ga.err = err.as<int>();
    timer.begin(1);
    ck(launch_gram(ga, Pl.p, K_pad, ls), "tensor-core gram");
    timer.end();
    kernels++;
    acc_launches++;
    exec_flops += 2.0 * 3 * 128.0 * 256.0 * ga.k_len * n_tiles;
  }
  timer.begin(3);
  for (size_t t = 0; t < nt; t++) {
    GramFinalArgs fa{};
    fa.n = gt[t].n;
    fa.n_pad = gt[t].n_pad;
    fa.s0 = J.tabs[t].start;
    fa.s1 = J.tabs[t].stop;
    fa.full = J.tabs[t].start == 0 && J.tabs[t].stop == gt[t].n / 2;
    fa.Gt = Gt.as<unsigned long long>() + gt[t].gt_off;
    fa.out = o.dev[t];
    fa.out_fp32 = J.out_fp32;
    ck(launch_finalize_gram(fa, ls), "finalize");
    kernels++;
  }
  timer.end();
  cap.launch();
  int h_err = 0;
  ck(cudaMemcpyAsync(&h_err, err.p, sizeof(int), cudaMemcpyDeviceToHost, st), "copy flag");
  if (!J.out_is_device)
    for (size_t t = 0; t < nt; t++)
      ck(cudaMemcpyAsync(J.tabs[t].out, o.dev[t], o.bytes[t], cudaMemcpyDeviceToHost, st), "copy out");
  counts = DevBuf();
  Pl = DevBuf();
  Gt = DevBuf();
  meta.dev = DevBuf();
  o.tmp.clear();
  ck(cudaStreamSynchronize(st), "synchronize");  // the error flag is read here
  err = DevBuf();
  if (h_err) return fail(UF_ETIMEOUT, "tensor-core kernel: a bounded wait gave up");
  double ms[5] = {0, 0, 0, 0, 0};
  timer.collect(ms);
  fill_reports(tree, J, o, ms, kernels, acc_launches, 1, rows, (int64_t)in.P->b0.size(), exec_flops, 256, 128,
               std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count());
  for (const TableJob &t : J.tabs)
    if (t.rep) {
      t.rep->chunk_rows = 4096;
      t.rep->graph = cap.on ? 1 : 0;
      t.rep->dense_rows = (int64_t)split.dense.size();
      t.rep->sparse_rows = split.n_sparse;
      t.rep->sparse_pairs = split.pairs;
      t.rep->t_sparse_ms = ms[4];
    }
  return UF_OK;
}

// Every other method / precision on the CUDA-core stripe kernels.  Throws
// CudaFail on CUDA errors.
uf_status run_stripes(uf_tree *tree, const BatchJob &J, int device, uf_method method, double scale) {
  const auto t_start = std::chrono::steady_clock::now();
  const size_t nt = J.tabs.size();
  const int acc = method == UF_GENERALIZED ? ACC_GEN : ACC_MIN;
  const int kind = method == UF_GENERALIZED ? EMB_PROP : method == UF_UNWEIGHTED ? EMB_PRESENCE : EMB_SCALED;
  const bool fp32 = J.fp32;
  const size_t es = fp32 ? 4 : 8;
  int tile_s = 0, tile_k = 0;
  stripe_tile_shape(acc, fp32, &tile_s, &tile_k);
  std::vector<TabDesc> tabs(nt);
  std::vector<int> off(nt);
  int n_cols = 0, n_tiles = 0;
  int64_t pitch = 0, cells = 0;
  for (size_t t = 0; t < nt; t++) {
    const int n = (int)J.tabs[t].table->n;
    TabDesc &d = tabs[t];
    d.n = n;
    d.off = n_cols;
    d.s_lo = (int)J.tabs[t].start;
    d.s_hi = (int)(J.tabs[t].stop - 1);
    d.m_lo = (int)(J.tabs[t].start / tile_s);
    d.m_hi = (int)((J.tabs[t].stop - 1) / tile_s);
    d.n_ktiles = (n + tile_k - 1) / tile_k;
    d.tile0 = n_tiles;
    d.x_col = pitch;
    d.m_off = cells;
    off[t] = n_cols;
    n_cols += n;
    n_tiles += d.n_ktiles * (d.m_hi - d.m_lo + 1);
    pitch += round_up(round_up(n, tile_k) + (int64_t)(d.m_hi + 1) * tile_s, 32);
    cells += (J.tabs[t].stop - J.tabs[t].start) * (int64_t)n;
  }
  const int64_t nb = tree->n_nodes - 1;
  const double acc_bytes = (double)cells * 8.0 * (acc == ACC_GEN ? 2 : 1) + n_cols * 8.0;
  const int64_t rows = block_rows(nb, (double)n_cols * 8.0 + (double)pitch * es + 8.0 + n_cols * es / 64.0, acc_bytes);
  Inputs in = bind_inputs(tree, J, device, rows);
  cudaStream_t st = J.st;
  const std::shared_ptr<const RowSplit> split_p = get_split(tree, J, in.P, acc, fp32);
  const RowSplit &split = *split_p;
  const int64_t xrows = std::max<int64_t>(split.max_dense, 1);
  int64_t kernels = 0, acc_launches = 0;
  PhaseTimer timer(g_kernel_timing.load() != 0, st);
  DevBuf counts((size_t)in.P->n_slots * n_cols * 8, st, "alloc counts");
  DevBuf X((size_t)xrows * pitch * es, st, "alloc embeddings");
  DevBuf M((size_t)cells * 8, st, "alloc stripes");
  DevBuf M2, Dg, Dsp, diag_tmp, counter(sizeof(int), st, "alloc counter");
  DevBuf total((size_t)n_cols * 8, st, "alloc totals"), inv_total((size_t)n_cols * 4, st, "alloc totals");
  // table descriptors and row lists: one staged upload
  Meta meta;
  const size_t o_tabs = meta.add(tabs);
  const size_t o_cnt = meta.add(split.cnt_lists);
  const size_t o_dense = meta.add(split.dense);
  const size_t o_dlen = meta.add(split.dense_len);
  size_t o_sparse = 0, o_sptabs = 0, o_lofs = 0;
  std::vector<int64_t> sp_off;  // first entry of each capacity class in the sparse list
  // one table whose accumulators exceed the L2 budget: the sparse rows write
  // their sample lists, then scatter their pairs stripe region by region
  const int n_acc = acc == ACC_GEN ? 2 : 1;
  const int64_t n_regions = (int64_t)sparse_regions(nt, acc, (double)cells * 8.0 * n_acc);
  const bool region_mode = split.n_sparse > 0 && (n_regions > 1 || split.lists);
  int64_t n_sparse_rows = 0;
  DevBuf lk, lx, lf, lz;
  if (split.n_sparse > 0) {
    std::vector<int32_t> all;
    for (const auto &c : split.sparse) {
      sp_off.push_back((int64_t)all.size());
      all.insert(all.end(), c.begin(), c.end());
    }
    n_sparse_rows = (int64_t)all.size();
    if (region_mode) {
      const auto &cp = J.tabs[0].table->col_ptr;
      std::vector<int64_t> lofs(all.size() + 1, 0);
      for (size_t r = 0; r < all.size(); r++)
        lofs[r + 1] = lofs[r] + (cp[tree->tip_hi[all[r]]] - cp[tree->tip_lo[all[r]]]);
      const size_t total_e = (size_t)std::max<int64_t>(lofs.back(), 1);
      lk = DevBuf(total_e * 4, st, "alloc sparse lists");
      lx = DevBuf(total_e * es, st, "alloc sparse lists");
      lf = DevBuf(total_e * 8, st, "alloc sparse lists");
      lz = DevBuf(std::max<size_t>(all.size(), 1) * 4, st, "alloc sparse lists");
      // rows without entries in the table return before writing their count
      ck(cudaMemsetAsync(lz.p, 0, std::max<size_t>(all.size(), 1) * 4, st), "memset");
      o_lofs = meta.add(lofs);
    }
    std::vector<SpTab> sp(nt);
    for (size_t t = 0; t < nt; t++) {
      sp[t].col_ptr = in.xd[t]->col_ptr;
      sp[t].col_row = in.xd[t]->col_row;
      sp[t].col_val = in.xd[t]->col_val;
      sp[t].total = in.xd[t]->total;
      sp[t].inv_total_f = in.xd[t]->inv_total_f;
      sp[t].n = tabs[t].n;
      sp[t].off = tabs[t].off;
      sp[t].s_lo = tabs[t].s_lo;
      sp[t].s_hi = tabs[t].s_hi;
      sp[t].m_off = tabs[t].m_off;
    }
    o_sparse = meta.add(all);
    o_sptabs = meta.add(sp);
    Dsp = DevBuf((size_t)n_cols * 8, st, "alloc diagonal");
    ck(cudaMemsetAsync(Dsp.p, 0, (size_t)n_cols * 8, st), "memset");
  }
  meta.upload(st);
  const TabDesc *d_tabs = meta.at<TabDesc>(o_tabs);
  const int32_t *d_cnt = meta.at<int32_t>(o_cnt);
  const int32_t *d_dense = meta.at<int32_t>(o_dense);
  const double *d_dlen = meta.at<double>(o_dlen);
  for (size_t t = 0; t < nt; t++) {
    const size_t n = (size_t)J.tabs[t].table->n;
    ck(cudaMemcpyAsync(total.as<double>() + off[t], in.xd[t]->total, n * 8, cudaMemcpyDeviceToDevice, st),
       "gather totals");
    ck(cudaMemcpyAsync(inv_total.as<float>() + off[t], in.xd[t]->inv_total_f, n * 4, cudaMemcpyDeviceToDevice,
                       st),
       "gather totals");
  }
  if (acc == ACC_GEN) {
    M2 = DevBuf((size_t)cells * 8, st, "alloc stripes");
    ck(cudaMemsetAsync(M2.p, 0, (size_t)cells * 8, st), "memset");
  } else {
    Dg = DevBuf((size_t)n_cols * 8, st, "alloc diagonal");
    diag_tmp = DevBuf(diag_scratch_bytes(fp32, (int)xrows, n_cols), st, "alloc diagonal scratch");
    ck(cudaMemsetAsync(Dg.p, 0, (size_t)n_cols * 8, st), "memset");
  }
  ck(cudaMemsetAsync(M.p, 0, (size_t)cells * 8, st), "memset");
  Outputs o = bind_outputs(J, st);
  double exec_flops = 0.0;
  // chunk size: tuned once per (accumulator, precision, size bucket)
  const auto key = tune_key(acc, fp32, n_tiles, xrows);
  int chunk = stripe_chunk_rows();
  bool tune = false;
  if (g_autotune.load() && !split.dense.empty()) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_tuned_chunk.find(key);
    if (it != g_tuned_chunk.end()) chunk = it->second;
    else tune = true;
  }
  // the launch sequence goes into a CUDA graph unless it is timed per phase
  Capture cap(g_graph.load() != 0 && !timer.on && !tune, st, device);
  const cudaStream_t ls = cap.stream();
  // the sparse-row scatters run after the dense blocks, whose chunk tuning clears M
  auto sparse_args = [&]() {
    SparseArgs sp{};
    sp.tip_lo = in.td->tip_lo;
    sp.tip_hi = in.td->tip_hi;
    sp.length = in.td->length;
    sp.tabs = meta.at<SpTab>(o_sptabs);
    sp.n_tabs = (int)nt;
    sp.kind = kind;
    sp.mixed_forms = fp32 && acc == ACC_MIN;
    sp.M = M.as<unsigned long long>();
    sp.M2 = M2.as<unsigned long long>();
    sp.Dsp = Dsp.as<unsigned long long>();
    sp.alpha = J.alpha;
    sp.scale = scale;
    if (region_mode) {
      sp.lk = lk.as<int32_t>();
      sp.lx = lx.p;
      sp.lf = lf.as<long long>();
      sp.lofs = meta.at<int64_t>(o_lofs);
      sp.lz = lz.as<int>();
    }
    return sp;
  };
  auto launch_sparse = [&](cudaStream_t on) {
    for (size_t c = 0; c < split.sparse.size(); c++) {
      if (split.sparse[c].empty()) continue;
      SparseArgs sp = sparse_args();
      sp.row_base = (int)sp_off[c];
      sp.nodes = meta.at<int32_t>(o_sparse) + sp_off[c];
      sp.n_nodes = (int)split.sparse[c].size();
      sp.cap = split.cap[c];
      if (region_mode) ck(launch_sparse_lists(acc, fp32, sp, on), "sparse lists");
      else ck(launch_sparse_rows(acc, fp32, sp, on), "sparse rows");
      kernels++;
    }
    if (!region_mode) return;
    const int64_t per = std::max<int64_t>(1, (int64_t)((double)g_region_bytes.load() / (8.0 * n_acc * tabs[0].n)));
    for (int64_t r0 = tabs[0].s_lo; r0 <= tabs[0].s_hi; r0 += per) {
      SparseArgs sp = sparse_args();
      sp.nodes = meta.at<int32_t>(o_sparse);
      sp.n_nodes = (int)n_sparse_rows;
      sp.r0 = (int)r0;
      sp.r1 = (int)std::min<int64_t>(r0 + per, (int64_t)tabs[0].s_hi + 1);
      ck(launch_sparse_region(acc, fp32, sp, on), "sparse regions");
      kernels++;
    }
  };
  bool tuned = false;
  for (size_t b = 0; b < in.P->b0.size(); b++) {
    const int64_t b0 = in.P->b0[b];
    const int64_t d0 = split.dense_ptr[b], nd = split.dense_ptr[b + 1] - d0;
    timer.begin(0);
    enqueue_split_counts(in, J, off, split, b, d_cnt, counts.as<double>(), n_cols, ls, &kernels);
    if (nd > 0) {
      ck(launch_emb_rows(kind, fp32, b0, (int)nd, in.pd->slot_of_node, counts.as<double>(), n_cols,
                         in.td->length, total.as<double>(), inv_total.as<float>(), X.p, pitch,
                         d_tabs, (int)nt, ls, d_dense + d0),
         "embedding rows");
      kernels++;
    }
    timer.end();
    if (nd == 0) continue;
    StripeArgs sa{};
    sa.X = X.p;
    sa.len = d_dlen + d0;
    sa.rows = (int)nd;
    sa.pitch = pitch;
    sa.chunk = chunk;
    sa.tabs = d_tabs;
    sa.n_tabs = (int)nt;
    sa.n_tiles = n_tiles;
    sa.n_cols = n_cols;
    sa.M = M.as<unsigned long long>();
    sa.M2 = M2.as<unsigned long long>();
    sa.Dg = Dg.as<unsigned long long>();
    sa.alpha = J.alpha;
    sa.scale = scale;
    sa.counter = counter.as<int>();
    if (tune && !tuned) {
      chunk = sa.chunk = tune_chunk(acc, fp32, sa, (size_t)cells, ls);
      tuned = true;
      std::lock_guard<std::mutex> g(g_tune_mu);
      g_tuned_chunk[key] = chunk;
    }
    timer.begin(1);
    ck(launch_stripe_acc(acc, fp32, sa, ls), "stripe accumulate");
    timer.end();
    kernels++;
    acc_launches++;
    exec_flops += 2.0 * (double)n_tiles * tile_s * tile_k * (double)nd;
    if (acc == ACC_MIN) {
      timer.begin(2);
      ck(launch_diag(fp32, sa, diag_tmp.p, ls), "diagonal accumulate");
      timer.end();
      kernels += 2;
    }
  }
  if (split.n_sparse > 0) {
    timer.begin(4);
    launch_sparse(ls);
    timer.end();
  }
  timer.begin(3);
  for (size_t t = 0; t < nt; t++) {
    FinalArgs fa{};
    fa.method = method;
    fa.n = tabs[t].n;
    fa.s0 = J.tabs[t].start;
    fa.s1 = J.tabs[t].stop;
    fa.full = J.tabs[t].start == 0 && J.tabs[t].stop == tabs[t].n / 2;
    fa.mixed_forms = fp32 && acc == ACC_MIN;
    fa.M = M.as<unsigned long long>() + tabs[t].m_off;
    fa.M2 = M2.p ? M2.as<unsigned long long>() + tabs[t].m_off : nullptr;
    fa.Dg = Dg.p ? Dg.as<unsigned long long>() + off[t] : nullptr;
    fa.Dsp = Dsp.p ? Dsp.as<unsigned long long>() + off[t] : nullptr;
    fa.inv_scale = 1.0 / scale;
    fa.out = o.dev[t];
    fa.out_fp32 = J.out_fp32;
    ck(launch_finalize(fa, ls), "finalize");
    kernels++;
  }
  timer.end();
  cap.launch();
  if (!J.out_is_device)
    for (size_t t = 0; t < nt; t++)
      ck(cudaMemcpyAsync(J.tabs[t].out, o.dev[t], o.bytes[t], cudaMemcpyDeviceToHost, st), "copy out");
  // buffers go back to the stream-ordered pool here
  counts = DevBuf();
  X = DevBuf();
  M = DevBuf();
  M2 = DevBuf();
  Dg = DevBuf();
  Dsp = DevBuf();
  diag_tmp = DevBuf();
  counter = DevBuf();
  meta.dev = DevBuf();
  total = DevBuf();
  inv_total = DevBuf();
  o.tmp.clear();
  if (!J.out_is_device || st == nullptr || timer.on) ck(cudaStreamSynchronize(st), "synchronize");
  else ck(cudaGetLastError(), "enqueue");
  double ms[5] = {0, 0, 0, 0, 0};
  timer.collect(ms);
  fill_reports(tree, J, o, ms, kernels, acc_launches, 0, rows, (int64_t)in.P->b0.size(), exec_flops, tile_s,
               tile_k, std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count());
  for (const TableJob &t : J.tabs)
    if (t.rep) {
      t.rep->chunk_rows = chunk;
      t.rep->graph = cap.on ? 1 : 0;
      t.rep->dense_rows = (int64_t)split.dense.size();
      t.rep->sparse_rows = split.n_sparse;
      t.rep->sparse_pairs = split.pairs;
      t.rep->t_sparse_ms = ms[4];
    }
  return UF_OK;
}

// One compute call on the current device; throws CudaFail on CUDA errors.
uf_status run_batch(uf_tree *tree, const BatchJob &J) {
  g_h2d = 0.0;
  int device = 0;
  ck(cudaGetDevice(&device), "cudaGetDevice");
  keep_pool_memory(device);
  uf_method method = J.method;
  if (method == UF_GENERALIZED && J.alpha == 1.0) method = UF_WEIGHTED_NORMALIZED;  // s^0 == 1
  const int kind = method == UF_GENERALIZED ? EMB_PROP : method == UF_UNWEIGHTED ? EMB_PRESENCE : EMB_SCALED;
  double scale = 0.0;  // one fixed-point scale valid for every table of the call
  for (const TableJob &t : J.tabs) {
    const double s = accum_scale(tree, t.table, kind);
    scale = scale == 0.0 ? s : std::min(scale, s);
  }
  if (method == UF_UNWEIGHTED && J.fp32 && g_tensor_path.load()) {
    // the tensor path keeps every table's whole n_pad x n_pad gram matrix (int64) on the
    // device whatever the stripe range; when that does not fit in half the free memory
    // the CUDA-core stripe kernels, which store only the requested stripes, take the call
    double gram_bytes = 0.0;
    for (const TableJob &t : J.tabs) {
      const double np = (double)gram_pad((int)t.table->n);
      gram_bytes += np * np * 8.0;
    }
    size_t free_b = 0, total_b = 0;
    ck(cudaMemGetInfo(&free_b, &total_b), "cudaMemGetInfo");
    if (gram_bytes <= 0.5 * (double)free_b) return run_gram(tree, J, device, scale, 0.0);
  }
  return run_stripes(tree, J, device, method, scale);
}

uf_status check_args(const uf_tree *tree, const uf_table *table, uf_method method, double alpha,
                     uf_precision precision) {
  if (!tree || !table) return fail(UF_EINVAL, "null tree or table");
  if (method < UF_UNWEIGHTED || method > UF_GENERALIZED) return fail(UF_EINVAL, "unknown method %d", (int)method);
  if (precision != UF_FP64 && precision != UF_MIXED) return fail(UF_EINVAL, "unknown precision %d", (int)precision);
  if (method == UF_GENERALIZED && !(alpha >= 0.0 && alpha <= 1.0))
    return fail(UF_EINVAL, "alpha must be in [0, 1] (got %g)", alpha);
  if (table->n_features != tree->n_tips)
    return fail(UF_ETABLE, "table has %lld features but the tree has %lld tips",
                (long long)table->n_features, (long long)tree->n_tips);
  return UF_OK;
}

}  // namespace

// ====================================================================== ABI

extern "C" {

uf_status uf_set_option(const char *name, int64_t value) {
  g_err.clear();
  if (!name) return fail(UF_EINVAL, "null option name");
  if (!strcmp(name, "branch_block")) {
    if (value < 0) return fail(UF_EINVAL, "branch_block must be >= 0");
    g_branch_block = value;
    return UF_OK;
  }
  if (!strcmp(name, "kernel_timing")) {
    if (value != 0 && value != 1) return fail(UF_EINVAL, "kernel_timing must be 0 or 1");
    g_kernel_timing = value;
    return UF_OK;
  }
  if (!strcmp(name, "tensor_path")) {
    if (value != 0 && value != 1) return fail(UF_EINVAL, "tensor_path must be 0 or 1");
    g_tensor_path = value;
    return UF_OK;
  }
  if (!strcmp(name, "graph")) {
    if (value != 0 && value != 1) return fail(UF_EINVAL, "graph must be 0 or 1");
    g_graph = value;
    return UF_OK;
  }
  if (!strcmp(name, "autotune")) {
    if (value < 0 || value > 2) return fail(UF_EINVAL, "autotune must be 0, 1 or 2");
    if (value == 2) {  // forget the tuned choices
      std::lock_guard<std::mutex> g(g_tune_mu);
      g_tuned_chunk.clear();
      value = 1;
    }
    g_autotune = value;
    return UF_OK;
  }
  if (!strcmp(name, "sparse")) {
    if (value < 0 || value > 2) return fail(UF_EINVAL, "sparse must be 0, 1 or 2");
    g_sparse = value;
    return UF_OK;
  }
  if (!strcmp(name, "sparse_region_bytes")) {
    if (value != 0 && value < 4096) return fail(UF_EINVAL, "sparse_region_bytes must be 0 or >= 4096");
    g_region_bytes = value ? value : (int64_t)SPARSE_REGION_BYTES_DEFAULT;
    return UF_OK;
  }
  return fail(UF_EINVAL, "unknown option '%s'", name);
}

int64_t uf_get_option(const char *name) {
  if (!name) return -1;
  if (!strcmp(name, "branch_block")) return g_branch_block.load();
  if (!strcmp(name, "kernel_timing")) return g_kernel_timing.load();
  if (!strcmp(name, "tensor_path")) return g_tensor_path.load();
  if (!strcmp(name, "graph")) return g_graph.load();
  if (!strcmp(name, "autotune")) return g_autotune.load();
  if (!strcmp(name, "sparse")) return g_sparse.load();
  if (!strcmp(name, "sparse_region_bytes")) return g_region_bytes.load();
  return -1;
}

const char *uf_last_error(void) { return g_err.c_str(); }

const char *uf_status_name(uf_status st) {
  switch (st) {
  case UF_OK: return "UF_OK";
  case UF_EINVAL: return "UF_EINVAL";
  case UF_ETREE: return "UF_ETREE";
  case UF_ETABLE: return "UF_ETABLE";
  case UF_ERANGE: return "UF_ERANGE";
  case UF_ENOMEM: return "UF_ENOMEM";
  case UF_ECUDA: return "UF_ECUDA";
  case UF_ETIMEOUT: return "UF_ETIMEOUT";
  case UF_ECANCELLED: return "UF_ECANCELLED";
  }
  return "UF_UNKNOWN";
}

int64_t uf_stripe_count(int64_t n_samples) { return n_samples < 2 ? 0 : n_samples / 2; }

uf_status uf_tree_create(int64_t n_nodes, const int64_t *parent, const double *length, uf_tree **out) {
  g_err.clear();
  if (!out) return fail(UF_EINVAL, "null output pointer");
  *out = nullptr;
  if (!parent || !length) return fail(UF_EINVAL, "null parent or length");
  if (n_nodes < 1) return fail(UF_EINVAL, "n_nodes must be >= 1 (got %lld)", (long long)n_nodes);
  if (n_nodes > INT32_MAX) return fail(UF_EINVAL, "n_nodes above 2^31 - 1");
  if (parent[n_nodes - 1] != -1) return fail(UF_ETREE, "the last node must be the root (parent -1)");
  for (int64_t i = 0; i + 1 < n_nodes; i++) {
    if (parent[i] <= i || parent[i] >= n_nodes)
      return fail(UF_ETREE, "node %lld: parent %lld must be in (%lld, %lld)", (long long)i,
                  (long long)parent[i], (long long)i, (long long)n_nodes);
    if (!std::isfinite(length[i]) || length[i] < 0.0)
      return fail(UF_ETREE, "node %lld: length %g must be finite and >= 0", (long long)i, length[i]);
  }
  try {
    auto t = std::make_unique<uf_tree>();
    static std::atomic<uint64_t> next_tree_id{1};
    t->id = next_tree_id++;
    t->n_nodes = n_nodes;
    t->parent.assign(parent, parent + n_nodes);
    t->length.assign(length, length + n_nodes);
    t->length[n_nodes - 1] = 0.0;  // no branch above the root
    std::vector<int32_t> nchild(n_nodes, 0);
    for (int64_t i = 0; i + 1 < n_nodes; i++) nchild[parent[i]]++;
    t->child_ptr.assign(n_nodes + 1, 0);
    for (int64_t i = 0; i < n_nodes; i++) t->child_ptr[i + 1] = t->child_ptr[i] + nchild[i];
    t->child_idx.assign(std::max<int64_t>(n_nodes - 1, 1), 0);
    std::vector<int32_t> fill(n_nodes, 0);
    for (int64_t i = 0; i + 1 < n_nodes; i++) {
      const int64_t p = parent[i];
      t->child_idx[t->child_ptr[p] + fill[p]++] = (int32_t)i;  // ascending child order
    }
    t->tip_of_node.assign(n_nodes, -1);
    int64_t tips = 0;
    for (int64_t i = 0; i < n_nodes; i++)
      if (nchild[i] == 0) t->tip_of_node[i] = (int32_t)tips++;
    t->n_tips = tips;
    {
      std::vector<int64_t> under(n_nodes, 0);
      t->tip_lo.assign(n_nodes, INT32_MAX);
      t->tip_hi.assign(n_nodes, -1);
      for (int64_t v = 0; v < n_nodes; v++) {  // children come before their parent
        if (t->tip_of_node[v] >= 0) {
          t->tip_lo[v] = t->tip_of_node[v];
          t->tip_hi[v] = t->tip_of_node[v] + 1;
          under[v] = 1;
        }
        if (v + 1 < n_nodes) {
          const int64_t p = parent[v];
          t->tip_lo[p] = std::min(t->tip_lo[p], t->tip_lo[v]);
          t->tip_hi[p] = std::max(t->tip_hi[p], t->tip_hi[v]);
          under[p] += under[v];
        }
      }
      for (int64_t v = 0; v < n_nodes; v++)
        if ((int64_t)t->tip_hi[v] - t->tip_lo[v] != under[v]) t->tip_lo[v] = t->tip_hi[v] = -1;
    }
    t->dist.assign(n_nodes, 0.0);
    for (int64_t v = n_nodes - 2; v >= 0; v--) {  // parents come later in the order
      t->dist[v] = t->length[v] + t->dist[parent[v]];
      t->total_length += t->length[v];
    }
    for (int64_t v = 0; v < n_nodes; v++)
      if (nchild[v] == 0) t->max_tip_dist = std::max(t->max_tip_dist, t->dist[v]);
    *out = t.release();
    return UF_OK;
  } catch (const std::bad_alloc &) {
    return fail(UF_ENOMEM, "host allocation failed");
  }
}

void uf_tree_destroy(uf_tree *tree) { delete tree; }
int64_t uf_tree_tips(const uf_tree *tree) { return tree ? tree->n_tips : -1; }

uf_status uf_table_create(int64_t n_samples, int64_t n_features, const int64_t *indptr,
                          const int32_t *indices, const double *data, const uf_tree *tree,
                          uf_table **out) {
  g_err.clear();
  if (!out) return fail(UF_EINVAL, "null output pointer");
  *out = nullptr;
  if (!indptr || !tree) return fail(UF_EINVAL, "null indptr or tree");
  if (n_samples < 1) return fail(UF_EINVAL, "n_samples must be >= 1");
  if (n_samples > INT32_MAX) return fail(UF_EINVAL, "n_samples above 2^31 - 1");
  if (n_features != tree->n_tips)
    return fail(UF_ETABLE, "n_features %lld != tree tips %lld", (long long)n_features,
                (long long)tree->n_tips);
  if (indptr[0] != 0) return fail(UF_ETABLE, "indptr[0] must be 0");
  for (int64_t k = 0; k < n_samples; k++)
    if (indptr[k + 1] <= indptr[k])
      return fail(UF_ETABLE, "sample %lld is empty or indptr decreases", (long long)k);
  const int64_t nnz = indptr[n_samples];
  if (nnz > 0 && (!indices || !data)) return fail(UF_EINVAL, "null indices or data");
  try {
    // sample ranges of about equal nonzeros, one per host thread
    const int T = (int)std::max<int64_t>(1, std::min<int64_t>(host_threads(), nnz / 100000));
    std::vector<int64_t> k_lo(T + 1, n_samples);
    k_lo[0] = 0;
    for (int c = 1, k = 0; c < T; c++) {
      const int64_t want = nnz * c / T;
      while (k < n_samples && indptr[k] < want) k++;
      k_lo[c] = k;
    }
    // validation (first failing sample wins, as a sequential scan would report)
    std::vector<int64_t> bad_k(T, -1);
    std::vector<std::string> bad_msg(T);
    parallel_for(T, [&](int c) {
      char buf[160];
      for (int64_t k = k_lo[c]; k < k_lo[c + 1]; k++)
        for (int64_t q = indptr[k]; q < indptr[k + 1]; q++) {
          if (indices[q] < 0 || indices[q] >= n_features)
            snprintf(buf, sizeof buf, "sample %lld: feature index %d out of range", (long long)k, indices[q]);
          else if (q > indptr[k] && indices[q] <= indices[q - 1])
            snprintf(buf, sizeof buf, "sample %lld: feature indices not strictly increasing", (long long)k);
          else if (!std::isfinite(data[q]) || data[q] <= 0.0)
            snprintf(buf, sizeof buf, "sample %lld: count %g must be finite and > 0", (long long)k, data[q]);
          else
            continue;
          bad_k[c] = k;
          bad_msg[c] = buf;
          return;
        }
    });
    for (int c = 0; c < T; c++)
      if (bad_k[c] >= 0) return fail(UF_ETABLE, "%s", bad_msg[c].c_str());
    auto t = std::make_unique<uf_table>();
    static std::atomic<uint64_t> next_id{1};
    t->id = next_id++;
    t->n = n_samples;
    t->n_features = n_features;
    t->nnz = nnz;
    t->total.assign(n_samples, 0.0);
    t->inv_total_f.assign(n_samples, 0.f);
    // CSC view by a counting sort: per-thread column counts, then each thread
    // scatters its samples (in increasing order) behind the earlier threads'
    std::vector<std::vector<int64_t>> cnt(T, std::vector<int64_t>(n_features, 0));
    parallel_for(T, [&](int c) {
      int64_t *cc = cnt[c].data();
      for (int64_t k = k_lo[c]; k < k_lo[c + 1]; k++) {
        double s = 0.0;
        for (int64_t q = indptr[k]; q < indptr[k + 1]; q++) {
          s += data[q];
          cc[indices[q]]++;
        }
        t->total[k] = s;
        t->inv_total_f[k] = (float)(1.0 / s);
      }
    });
    t->col_ptr.assign(n_features + 1, 0);
    for (int64_t f = 0; f < n_features; f++) {
      int64_t at = t->col_ptr[f];
      for (int c = 0; c < T; c++) {
        const int64_t x = cnt[c][f];
        cnt[c][f] = at;  // this thread's first slot in column f
        at += x;
      }
      t->col_ptr[f + 1] = at;
    }
    t->col_row.resize(std::max<int64_t>(nnz, 1));  // every entry written below (nnz >= 1)
    t->col_val.resize(std::max<int64_t>(nnz, 1));
    parallel_for(T, [&](int c) {
      int64_t *slot = cnt[c].data();
      for (int64_t k = k_lo[c]; k < k_lo[c + 1]; k++)
        for (int64_t q = indptr[k]; q < indptr[k + 1]; q++) {
          const int64_t at = slot[indices[q]]++;
          t->col_row[at] = (int32_t)k;
          t->col_val[at] = data[q];
        }
    });
    *out = t.release();
    return UF_OK;
  } catch (const std::bad_alloc &) {
    return fail(UF_ENOMEM, "host allocation failed");
  } catch (const std::system_error &) {
    return fail(UF_ENOMEM, "could not start host threads");
  }
}

void uf_table_destroy(uf_table *table) { delete table; }
int64_t uf_table_samples(const uf_table *table) { return table ? table->n : -1; }

uf_status uf_compute(const uf_tree *tree, const uf_table *table, uf_method method, double alpha,
                     uf_precision precision, int64_t stripe_start, int64_t stripe_stop, void *out,
                     int out_is_device, int out_fp32, uf_report *rep, void *cuda_stream) {
  g_err.clear();
  uf_status st = check_args(tree, table, method, alpha, precision);
  if (st) return st;
  const int64_t S = uf_stripe_count(table->n);
  if (stripe_start < 0 || stripe_stop < stripe_start || stripe_stop > S)
    return fail(UF_ERANGE, "stripe range [%lld, %lld) outside [0, %lld]", (long long)stripe_start,
                (long long)stripe_stop, (long long)S);
  if (rep) memset(rep, 0, sizeof *rep);
  if (stripe_start == stripe_stop) return UF_OK;
  if (!out) return fail(UF_EINVAL, "null output buffer");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return fail(UF_ECUDA, "no CUDA device available");
  }
  BatchJob J{method, alpha, precision == UF_MIXED, out_is_device, out_fp32, (cudaStream_t)cuda_stream, {}};
  J.tabs.push_back(TableJob{const_cast<uf_table *>(table), stripe_start, stripe_stop, out, rep});
  try {
    return run_batch(const_cast<uf_tree *>(tree), J);
  } catch (const CudaFail &f) {
    return f.st;
  } catch (const std::bad_alloc &) {
    return fail(UF_ENOMEM, "host allocation failed");
  }
}

uf_status uf_compute_batch(const uf_tree *tree, const uf_table *const *tables, int64_t n_tables,
                           uf_method method, double alpha, uf_precision precision,
                           void *const *outs, int out_is_device, uf_report *reps,
                           void *cuda_stream) {
  g_err.clear();
  if (!tables || !outs || n_tables < 0) return fail(UF_EINVAL, "null tables or outputs");
  BatchJob J{method, alpha, precision == UF_MIXED, out_is_device, 0, (cudaStream_t)cuda_stream, {}};
  for (int64_t t = 0; t < n_tables; t++) {
    uf_status st = check_args(tree, tables[t], method, alpha, precision);
    if (st) return st;
    if (reps) memset(&reps[t], 0, sizeof(uf_report));
    const int64_t S = uf_stripe_count(tables[t]->n);
    if (S == 0) continue;  // fewer than two samples: nothing to write
    if (!outs[t]) return fail(UF_EINVAL, "null output buffer for table %lld", (long long)t);
    J.tabs.push_back(TableJob{const_cast<uf_table *>(tables[t]), 0, S, outs[t], reps ? &reps[t] : nullptr});
  }
  if (J.tabs.empty()) return UF_OK;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return fail(UF_ECUDA, "no CUDA device available");
  }
  try {
    return run_batch(const_cast<uf_tree *>(tree), J);
  } catch (const CudaFail &f) {
    return f.st;
  } catch (const std::bad_alloc &) {
    return fail(UF_ENOMEM, "host allocation failed");
  }
}

}  // extern "C"

// ---------------------------------------------------------------- views
// Read-only access to the host copies held by a tree / table, for entry
// points implemented in other translation units.
namespace ufg {

bool tree_host_view(const uf_tree *t, TreeView *v) {
  if (!t || !v) return false;
  v->n_nodes = t->n_nodes;
  v->n_tips = t->n_tips;
  v->length = t->length.data();
  v->tip_of_node = t->tip_of_node.data();
  v->child_ptr = t->child_ptr.data();
  v->child_idx = t->child_idx.data();
  return true;
}

bool table_host_view(const uf_table *t, TableView *v) {
  if (!t || !v) return false;
  v->n = t->n;
  v->n_features = t->n_features;
  v->nnz = t->nnz;
  v->total = t->total.data();
  v->inv_total_f = t->inv_total_f.data();
  v->col_ptr = t->col_ptr.data();
  v->col_row = t->col_row.data();
  v->col_val = t->col_val.data();
  return true;
}

}  // namespace ufg

namespace ufg {
// Set the calling thread's uf_last_error() text (for entry points in other
// translation units) and return st.
uf_status set_last_error(uf_status st, const char *msg) {
  g_err = msg ? msg : "";
  return st;
}
}  // namespace ufg
