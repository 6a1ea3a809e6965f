// uf_run.cpp -- the launch sequence of one compute call: device buffers from
// the stream-ordered pool, metadata through a pinned staging ring, per branch
// block the count rows, embedding rows and the dense stripe accumulate (or
// the tensor-core gram), the sparse-row scatter, and the finalize, captured
// into one CUDA graph unless phases are timed.
#include <array>

#include "uf_runtime.h"

#include <deque>

namespace ufg {
namespace rt {

namespace {

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

// Device memory a call can use: free memory plus what the current device's
// stream-ordered pool holds reserved but unused (freed buffers of earlier
// calls stay reserved, keep_pool_memory, and are reused by the pool).
double available_bytes() {
  size_t free_b = 0, total_b = 0;
  ck(cudaMemGetInfo(&free_b, &total_b), "cudaMemGetInfo");
  double avail = (double)free_b;
  int device = 0;
  cudaMemPool_t pool;
  if (cudaGetDevice(&device) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    uint64_t reserved = 0, used = 0;
    if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) == cudaSuccess &&
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) == cudaSuccess && reserved > used)
      avail += (double)(reserved - used);
  }
  cudaGetLastError();
  return avail;
}

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

// Private streams of the calling thread per device: [0] records a call's
// launch sequence into a CUDA graph, [1] carries the sparse-row scatter
// beside the dense stripe kernel.  Per thread, so that concurrent calls from
// several threads never share a capturing stream.
struct ThreadStreams {
  std::map<int, std::array<cudaStream_t, 2>> s;
  ~ThreadStreams() {
    for (auto &kv : s)
      for (cudaStream_t x : kv.second) cudaStreamDestroy(x);
  }
};
thread_local ThreadStreams t_streams;

cudaStream_t private_stream(int device, int which) {
  auto it = t_streams.s.find(device);
  if (it == t_streams.s.end()) {
    std::array<cudaStream_t, 2> a{nullptr, nullptr};
    for (auto &x : a) ck(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking), "cudaStreamCreate");
    it = t_streams.s.emplace(device, a).first;
  }
  return it->second[which];
}
cudaStream_t capture_stream(int device) { return private_stream(device, 0); }

// A side branch of launches on the thread's side stream: fork() makes it wait
// for everything issued so far on the main stream, join() makes the main
// stream wait for the branch.  Inside a stream capture both streams belong to
// the same graph, which then holds two parallel branches.
struct SideBranch {
  cudaStream_t main, side;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool forked = false;
  SideBranch(cudaStream_t m, int device) : main(m), side(private_stream(device, 1)) {}
  cudaStream_t fork() {
    ck(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming), "cudaEventCreate");
    ck(cudaEventRecord(ev_fork, main), "cudaEventRecord");
    ck(cudaStreamWaitEvent(side, ev_fork, 0), "cudaStreamWaitEvent");
    forked = true;
    return side;
  }
  void join() {
    if (!forked) return;
    ck(cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming), "cudaEventCreate");
    ck(cudaEventRecord(ev_join, side), "cudaEventRecord");
    ck(cudaStreamWaitEvent(main, ev_join, 0), "cudaStreamWaitEvent");
    forked = false;
  }
  ~SideBranch() {
    if (forked) {  // an error escaped: still keep the main stream behind the branch
      cudaEvent_t e = nullptr;
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess &&
          cudaEventRecord(e, side) == cudaSuccess)
        cudaStreamWaitEvent(main, e, 0);
      if (e) cudaEventDestroy(e);
    }
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    cudaGetLastError();
  }
};

// Raises the calling thread's launch priority (launch_k) to the device's
// highest for its lifetime when on: the main path of a call whose sparse-row
// scatter runs beside it.
struct PriorityScope {
  int old;
  bool on;
  explicit PriorityScope(bool enable) : old(launch_priority()), on(enable) {
    if (!on) return;
    int least = 0, greatest = 0;
    ck(cudaDeviceGetStreamPriorityRange(&least, &greatest), "cudaDeviceGetStreamPriorityRange");
    set_launch_priority(greatest);
  }
  ~PriorityScope() { set_launch_priority(old); }
};

// Executable graphs already launched.  Destroying one makes the host wait for
// the work in flight on the device, even when that graph itself has finished
// (measured on GB300: destroying the previous call's finished graph while a
// 0.9 s tensor-core call ran held the host for 0.9 s).  So each is kept with
// an event recorded behind its launch, and they are destroyed together at
// the start of a later call once every one of them has completed (the
// caller has synchronised: nothing of ours is in flight), or, past 32
// queued, after a wait on the oldest.
struct LiveGraphs {
  std::mutex mu;
  std::deque<std::pair<cudaGraphExec_t, cudaEvent_t>> q;
};
LiveGraphs g_live_graphs;

void destroy_front(std::deque<std::pair<cudaGraphExec_t, cudaEvent_t>> &q) {
  cudaGraphExecDestroy(q.front().first);
  cudaEventDestroy(q.front().second);
  q.pop_front();
}

void retire_graph(cudaGraphExec_t e, cudaStream_t st) {
  cudaEvent_t ev = nullptr;
  if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess || cudaEventRecord(ev, st) != cudaSuccess) {
    if (ev) cudaEventDestroy(ev);
    cudaGetLastError();
    cudaStreamSynchronize(st);
    cudaGraphExecDestroy(e);
    return;
  }
  std::lock_guard<std::mutex> g(g_live_graphs.mu);
  auto &q = g_live_graphs.q;
  q.emplace_back(e, ev);
  while (q.size() > 32) {
    cudaEventSynchronize(q.front().second);
    destroy_front(q);
  }
  cudaGetLastError();
}

// At the start of a call: the queued graphs, if all of them have completed.
void reap_graphs() {
  std::lock_guard<std::mutex> g(g_live_graphs.mu);
  auto &q = g_live_graphs.q;
  for (const auto &x : q)
    if (cudaEventQuery(x.second) != cudaSuccess) {
      cudaGetLastError();  // cudaErrorNotReady is not an error here
      return;
    }
  while (!q.empty()) destroy_front(q);
}

// Records the branch-block launch sequence of a call into a CUDA graph (on a
// private stream) and launches that graph on the caller's stream; when off,
// launches go to the caller's stream directly.
struct Capture {
  bool on;
  cudaStream_t user, cap = nullptr;
  bool open = false;
  // the graph runs its kernels at their own launch priorities (launch_k)
  // rather than at the caller's stream priority
  bool node_priority = false;
  Capture(bool enable, cudaStream_t st, int device) : on(enable), user(st) {
    if (!on) return;
    reap_graphs();
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
    cudaError_t err =
        cudaGraphInstantiate(&e, g, node_priority ? (unsigned long long)cudaGraphInstantiateFlagUseNodePriority : 0ull);
    if (err == cudaSuccess) err = cudaGraphLaunch(e, user);
    if (e) {
      if (err == cudaSuccess) retire_graph(e, user);
      else cudaGraphExecDestroy(e);
    }
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

// Autotuned (tile shape, rows per work unit), by (accumulator, precision,
// size bucket).
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, std::pair<int, int>> g_tuned_chunk;

// kernel: 0 FP64, 1 FP32, 2 FP32 all-abs
std::tuple<int, int, int, int> tune_key(int acc, int kernel, int64_t n_tiles, int64_t rows) {
  auto lg = [](int64_t x) { return (int)std::floor(std::log2((double)std::max<int64_t>(x, 1))); };
  return {acc, kernel, lg(n_tiles), lg(rows)};
}

// A timing event destroyed with its scope, also when a CUDA error is thrown.
struct ScopedEvent {
  cudaEvent_t e = nullptr;
  ScopedEvent() { ck(cudaEventCreate(&e), "cudaEventCreate"); }
  ~ScopedEvent() {
    if (e) cudaEventDestroy(e);
  }
  ScopedEvent(const ScopedEvent &) = delete;
  ScopedEvent &operator=(const ScopedEvent &) = delete;
};

// Time the accumulate launch of the first block with each candidate tile
// shape and chunk size and keep the fastest (the accumulators are cleared
// afterwards).  tabs[s] / n_tiles[s]: the descriptors of shape s.
std::pair<int, int> tune_chunk(int acc, bool fp32, StripeArgs sa, const std::vector<const TabDesc *> &tabs,
                               const std::vector<int> &n_tiles, size_t m_bytes, cudaStream_t st) {
  const int cand[4] = {1024, 2048, 4096, 8192};
  const ScopedEvent ev0, ev1;
  cudaEvent_t e0 = ev0.e, e1 = ev1.e;
  std::pair<int, int> best{0, stripe_chunk_rows()};
  float best_ms = 1e30f;
  for (size_t shape = 0; shape < tabs.size(); shape++)
    for (int c : cand) {
      if (n_tiles[shape] < 0) break;  // not a candidate
      if (c > 2 * std::max(sa.rows, 1024)) break;
      sa.chunk = c;
      sa.shape = (int)shape;
      sa.tabs = tabs[shape];
      sa.n_tiles = n_tiles[shape];
      ck(cudaEventRecord(e0, st), "cudaEventRecord");
      ck(launch_stripe_acc(acc, fp32, sa, st), "autotune");
      ck(cudaEventRecord(e1, st), "cudaEventRecord");
      ck(cudaEventSynchronize(e1), "cudaEventSynchronize");
      float ms = 0.f;
      ck(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
      if (ms < best_ms) {
        best_ms = ms;
        best = {(int)shape, c};
      }
    }
  ck(cudaMemsetAsync(sa.M, 0, m_bytes, st), "memset");
  if (sa.M2) ck(cudaMemsetAsync(sa.M2, 0, m_bytes, st), "memset");
  return best;
}

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

// the region scatter's pair-update counters, summed
double pair_sum(const unsigned long long (&c)[SPARSE_PAIR_SLOTS]) {
  unsigned long long t = 0;
  for (unsigned long long v : c) t += v;
  return (double)t;
}

// Branch rows per embedding block for a working budget of per_row bytes a row
// plus fixed bytes.
int64_t block_rows(int64_t nb, double per_row, double fixed) {
  // 48 GB: about 31 blocks for a 1M-node tree and a 113,000-sample table
  // (fewer, longer dense launches: 2.6 % less time than 24 GB's 64 blocks)
  const double budget = std::min(0.5 * available_bytes() - fixed, 48e9);
  int64_t rows = (int64_t)(budget / per_row / 1.1);
  rows = std::max<int64_t>(std::min<int64_t>(rows, nb), std::min<int64_t>(nb, 256));
  if (g_branch_block.load() > 0) rows = std::min<int64_t>(g_branch_block.load(), std::max<int64_t>(nb, 1));
  return std::max<int64_t>(rows, 1);
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
                          size_t b, const int32_t *d_cnt, double *counts, int64_t ld, int64_t n_cols,
                          cudaStream_t st, int64_t *kernels) {
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
                          in.pd->slot_of_node, counts, ld, st, n_cols),
       "node counts");
    (*kernels)++;
  }
}

// The same rows as presence flags (the tensor-core unweighted path needs
// nothing else): one byte per sample instead of an FP64 count.
void enqueue_split_presence(const Inputs &in, const BatchJob &J, const std::vector<int> &off,
                            const RowSplit &split, size_t b, const int32_t *d_cnt, uint8_t *flags, int64_t ld,
                            int64_t n_cols, cudaStream_t st, int64_t *kernels) {
  const auto &lb = split.cnt_launch[b];
  for (size_t t = 0; t < J.tabs.size(); t++) {
    ck(launch_slice_presence(d_cnt + lb[0].first, lb[0].second, in.td->tip_lo, in.td->tip_hi, in.pd->slot_of_node,
                             in.xd[t]->col_ptr, in.xd[t]->col_row, flags + off[t], ld, (int)J.tabs[t].table->n,
                             st),
       "presence rows");
    *kernels += lb[0].second > 0;
  }
  for (size_t l = 1; l < lb.size(); l++) {
    ck(launch_node_presence(d_cnt + lb[l].first, lb[l].second, in.td->child_ptr, in.td->child_idx,
                            in.pd->slot_of_node, flags, ld, st, n_cols),
       "node presence");
    (*kernels)++;
  }
}

// Stripe-layout description of the tables of a call for the sparse-row
// scatter: samples, combined column, stored stripes and first cell of each.
struct SpLayout {
  int n, off, s_lo, s_hi;
  int64_t m_off;
};

// The sparse-row scatter of a call (uf_sparse.cu): its row lists by capacity
// class, the per-sample diagonal R, and for one table whose accumulators
// exceed the L2 budget the sample lists that are then scattered stripe region
// by region.  prepare() adds its metadata to the call's Meta before the
// upload; launch() enqueues the scatter.
struct SparseScatter {
  const RowSplit *split = nullptr;
  bool region_mode = false;
  int fuse_m = 0;         // members per min-form list row (launch_sparse_region); 0: unfused
  bool two_word = false;  // FP64 terms in two words (second words after the first)
  int n_acc = 1;
  int64_t n_sparse_rows = 0, cells = 0, n_cols = 0;
  std::vector<int64_t> sp_off;  // first entry of each capacity class in the sparse list
  std::vector<int64_t> cls_n;   // rows of each class that are launched
  size_t o_sparse = 0, o_sptabs = 0, o_lofs = 0, o_members = 0;
  DevBuf le, lk, lz, Dsp, cur;
  int64_t list_entries = 0;
  std::vector<SpLayout> lay;

  // acc: ACC_MIN / ACC_GEN; fp64_entries: terms computed in FP64
  void prepare(uf_tree *tree, const BatchJob &J, const Inputs &in, const RowSplit &sp,
               const std::vector<SpLayout> &layout, int acc, bool fp64_entries, bool two_words,
               int64_t call_cells, int64_t call_cols, Meta &meta, cudaStream_t st) {
    split = &sp;
    lay = layout;
    two_word = two_words;
    n_acc = acc == ACC_GEN ? 2 : 1;
    cells = call_cells;
    n_cols = call_cols;
    const size_t nt = J.tabs.size();
    if (sp.n_sparse == 0) return;
    const int64_t n_regions = (int64_t)sparse_regions(nt, acc, (double)cells * 8.0 * n_acc * (two_word ? 2 : 1));
    region_mode = n_regions > 1 || sp.lists;
    // the generalized method's entries carry each row's proportion as well:
    // two members at most
    fuse_m = !region_mode ? 0 : acc == ACC_MIN ? (int)g_sparse_fuse.load() : (int)std::min<int64_t>(g_sparse_fuse.load(), 2);
    std::vector<int32_t> all, members;
    if (fuse_m > 0) {
      // A sparse branch whose parent is a listed head rides in the parent's
      // list (its samples are among the parent's and its pairs among the
      // parent's pairs); with six members per head, so does a sparse child of
      // such a member (two levels below the head).  Parents come before
      // children in decreasing node order (parent[v] > v), so every head and
      // member is final when its children are visited.
      const int F = fuse_m, depth = F == 6 ? 2 : 1;
      const int64_t nn = tree->n_nodes;
      std::vector<int8_t> level(nn, -1), used(nn, 0);  // -1: not listed, 0: head, >0: member depth
      std::vector<int32_t> head_of(nn, -1), mem_of((size_t)nn * F, -1);
      for (const auto &c : sp.sparse)
        for (int32_t v : c) level[v] = 0;
      for (int64_t v = nn - 2; v >= 0; v--) {
        if (level[v] != 0) continue;
        const int64_t p = tree->parent[v];
        if (p < 0 || level[p] < 0 || level[p] >= depth) continue;
        const int32_t h = level[p] == 0 ? (int32_t)p : head_of[p];
        if (used[h] >= F) continue;
        mem_of[(size_t)h * F + used[h]++] = (int32_t)v;
        level[v] = (int8_t)(level[p] + 1);
        head_of[v] = h;
      }
      for (const auto &c : sp.sparse) {
        sp_off.push_back((int64_t)all.size());
        for (int32_t v : c)
          if (level[v] == 0) {
            all.push_back(v);
            members.insert(members.end(), mem_of.begin() + (size_t)v * F, mem_of.begin() + (size_t)v * F + F);
          }
        cls_n.push_back((int64_t)all.size() - sp_off.back());
      }
    } else {
      for (const auto &c : sp.sparse) {
        sp_off.push_back((int64_t)all.size());
        all.insert(all.end(), c.begin(), c.end());
        cls_n.push_back((int64_t)c.size());
      }
    }
    n_sparse_rows = (int64_t)all.size();
    if (region_mode) {
      const auto &cp = J.tabs[0].table->col_ptr;
      std::vector<int64_t> lofs(all.size() + 1, 0);
      for (size_t r = 0; r < all.size(); r++)
        lofs[r + 1] = lofs[r] + (cp[tree->tip_hi[all[r]]] - cp[tree->tip_lo[all[r]]]);
      const size_t total_e = (size_t)std::max<int64_t>(lofs.back(), 1);
      list_entries = (int64_t)total_e;
      le = DevBuf(total_e * sparse_entry_bytes(!fp64_entries, fuse_m, acc), st, "alloc sparse lists");
      lk = DevBuf(total_e * 4, st, "alloc sparse lists");
      cur = DevBuf(total_e * 2 * sizeof(uint16_t), st, "alloc sparse list cursors");
      lz = DevBuf(std::max<size_t>(all.size(), 1) * 4, st, "alloc sparse lists");
      // rows without entries in the table return before writing their count
      ck(cudaMemsetAsync(lz.p, 0, std::max<size_t>(all.size(), 1) * 4, st), "memset");
      o_lofs = meta.add(lofs);
      if (fuse_m > 0) o_members = meta.add(members);
    }
    std::vector<SpTab> tabs(nt);
    for (size_t t = 0; t < nt; t++) {
      tabs[t].col_ptr = in.xd[t]->col_ptr;
      tabs[t].col_row = in.xd[t]->col_row;
      tabs[t].col_val = in.xd[t]->col_val;
      tabs[t].total = in.xd[t]->total;
      tabs[t].inv_total_f = in.xd[t]->inv_total_f;
      tabs[t].n = lay[t].n;
      tabs[t].off = lay[t].off;
      tabs[t].s_lo = lay[t].s_lo;
      tabs[t].s_hi = lay[t].s_hi;
      tabs[t].m_off = lay[t].m_off;
    }
    o_sparse = meta.add(all);
    o_sptabs = meta.add(tabs);
    const size_t dsp_words = (size_t)n_cols * (two_word ? 2 : 1);
    Dsp = DevBuf(dsp_words * 8, st, "alloc diagonal");
    ck(cudaMemsetAsync(Dsp.p, 0, dsp_words * 8, st), "memset");
  }

  // base: kind, masks, M / M2, alpha and scale filled by the caller
  void launch(const Meta &meta, const Inputs &in, SparseArgs base, int acc, bool fp64_entries, int64_t region_bytes,
              cudaStream_t on, int64_t *kernels) const {
    if (!split || split->n_sparse == 0) return;
    const bool f32 = !fp64_entries;
    base.tip_lo = in.td->tip_lo;
    base.tip_hi = in.td->tip_hi;
    base.length = in.td->length;
    base.tabs = meta.at<SpTab>(o_sptabs);
    base.n_tabs = (int)lay.size();
    base.Dsp = Dsp.as<unsigned long long>();
    base.m_lo_off = two_word ? cells : 0;
    base.d_lo_off = two_word ? n_cols : 0;
    if (region_mode) {
      base.le = le.p;
      base.lk = lk.as<int>();
      base.lofs = meta.at<int64_t>(o_lofs);
      base.lz = lz.as<int>();
      base.cur = cur.as<uint16_t>();
      base.cur_stride = list_entries;
      base.fused = fuse_m;
      base.members = fuse_m > 0 ? meta.at<int32_t>(o_members) : nullptr;
    }
    for (size_t c = 0; c < split->sparse.size(); c++) {
      if (cls_n[c] == 0) continue;
      SparseArgs sp = base;
      sp.row_base = (int)sp_off[c];
      sp.nodes = meta.at<int32_t>(o_sparse) + sp_off[c];
      sp.n_nodes = (int)cls_n[c];
      sp.cap = split->cap[c];
      if (region_mode) ck(launch_sparse_lists(acc, f32, sp, on), "sparse lists");
      else ck(launch_sparse_rows(acc, f32, sp, on), "sparse rows");
      (*kernels)++;
    }
    if (!region_mode) return;
    const int64_t per =
        std::max<int64_t>(1, (int64_t)((double)region_bytes / (8.0 * n_acc * (two_word ? 2 : 1) * lay[0].n)));
    for (int64_t r0 = lay[0].s_lo; r0 <= lay[0].s_hi; r0 += per) {
      SparseArgs sp = base;
      sp.nodes = meta.at<int32_t>(o_sparse);
      sp.n_nodes = (int)n_sparse_rows;
      sp.r0 = (int)r0;
      sp.r1 = (int)std::min<int64_t>(r0 + per, (int64_t)lay[0].s_hi + 1);
      sp.first_region = r0 == lay[0].s_lo;
      ck(launch_sparse_region(acc, f32, sp, on), "sparse regions");
      (*kernels)++;
    }
  }
};

// Tiles the tensor path stores for one call: per table the tiles that hold
// a pair of its stripe range or a diagonal cell (gram_tiles), numbered across
// the tables, with each table's tile map.
struct GramPlan {
  std::vector<GramTab> gt;
  std::vector<int32_t> tile_tab, tile_bi, tile_bj, maps;
  int n_cols = 0, npad_tot = 0;
  int64_t n_tiles = 0;
};

GramPlan gram_plan(const BatchJob &J) {
  GramPlan G;
  const size_t nt = J.tabs.size();
  G.gt.resize(nt);
  for (size_t t = 0; t < nt; t++) {
    const int n = (int)J.tabs[t].table->n;
    GramTab &g = G.gt[t];
    g.n = n;
    g.n_pad = gram_pad(n);
    g.row_base = G.npad_tot;
    g.off = G.n_cols;
    g.map_off = (int64_t)G.maps.size();
    const int rows_b = g.n_pad / GRAM_TM, cols_b = g.n_pad / GRAM_TN;
    std::vector<int32_t> bi, bj;
    gram_tiles(n, J.tabs[t].start, J.tabs[t].stop, &bi, &bj);
    std::vector<int32_t> map((size_t)rows_b * cols_b, -1);
    for (size_t q = 0; q < bi.size(); q++) {
      map[(size_t)bi[q] * cols_b + bj[q]] = (int32_t)(G.tile_bi.size() + q);
    }
    G.maps.insert(G.maps.end(), map.begin(), map.end());
    G.tile_bi.insert(G.tile_bi.end(), bi.begin(), bi.end());
    G.tile_bj.insert(G.tile_bj.end(), bj.begin(), bj.end());
    G.tile_tab.insert(G.tile_tab.end(), bi.size(), (int32_t)t);
    G.n_cols += n;
    G.npad_tot += g.n_pad;
  }
  G.n_tiles = (int64_t)G.tile_bi.size();
  return G;
}

// Stripe cells of the call's tables: (stop - start) * n each.
int64_t stripe_cells(const BatchJob &J) {
  int64_t c = 0;
  for (const TableJob &t : J.tabs) c += (t.stop - t.start) * t.table->n;
  return c;
}

// Unweighted, mixed precision, on the tensor cores: per branch block, counts
// -> presence / split-length planes of every table -> tcgen05 gram into the
// stored tiles; the sparse rows scatter into stripe-layout cells; then the
// gram finalize of every table.  Throws CudaFail on CUDA errors.
uf_status run_gram(uf_tree *tree, const BatchJob &J, int device, double scale) {
  const auto t_start = std::chrono::steady_clock::now();
  const size_t nt = J.tabs.size();
  GramPlan G = gram_plan(J);
  std::vector<int> off(nt);
  std::vector<SpLayout> lay(nt);
  int64_t cells = 0;
  for (size_t t = 0; t < nt; t++) {
    off[t] = G.gt[t].off;
    lay[t] = SpLayout{G.gt[t].n, G.gt[t].off, (int)J.tabs[t].start, (int)(J.tabs[t].stop - 1), cells};
    cells += (J.tabs[t].stop - J.tabs[t].start) * G.gt[t].n;
  }
  const int n_cols = G.n_cols, npad_tot = G.npad_tot;
  const int n_tiles = (int)G.n_tiles;
  const int64_t nb = tree->n_nodes - 1;
  const double tile_bytes = (double)G.n_tiles * GRAM_TILE_CELLS * 8.0;
  const int64_t rows = block_rows(nb, (double)n_cols + 4.0 * npad_tot * 2.0 + 8.0, tile_bytes + cells * 8.0);
  Inputs in = [&] {
    NvtxRange r("uf: bind inputs");
    return bind_inputs(tree, J, device, rows);
  }();
  const std::shared_ptr<const RowSplit> split_p = [&] {
    NvtxRange r("uf: branch split");
    return get_split(tree, J, in.P, SPLIT_GRAM, true);
  }();
  const RowSplit &split = *split_p;
  const int64_t K_pad = gram_kpad((int)std::max<int64_t>(split.max_dense, 1));
  cudaStream_t st = J.st;
  int64_t kernels = 0, acc_launches = 0;
  PhaseTimer timer(g_kernel_timing.load() != 0, st);
  std::vector<int32_t> tl(G.tile_tab);
  tl.insert(tl.end(), G.tile_bi.begin(), G.tile_bi.end());
  tl.insert(tl.end(), G.tile_bj.begin(), G.tile_bj.end());
  // presence rows: stride rounded up to 16 bytes for the 16-byte level kernel
  const int64_t ld = round_up(n_cols, 16);
  DevBuf flags((size_t)in.P->n_slots * ld, st, "alloc presence rows");
  DevBuf Pl((size_t)4 * npad_tot * K_pad * 2, st, "alloc presence planes");
  DevBuf Gt((size_t)std::max<int64_t>(G.n_tiles, 1) * GRAM_TILE_CELLS * 8, st, "alloc gram tiles");
  DevBuf err(sizeof(int), st, "alloc error flag");
  DevBuf clamps(sizeof(unsigned long long), st, "alloc clamp counter");
  DevBuf Msp;
  Meta meta;  // tile list, table descriptors, tile maps and row lists: one staged upload
  const size_t o_tiles = meta.add(tl), o_tabs = meta.add(G.gt), o_maps = meta.add(G.maps);
  const size_t o_cnt = meta.add(split.cnt_lists), o_dense = meta.add(split.dense);
  // sparse rows: presence terms (x = l) in FP64, one word, min form, into
  // stripe-layout cells Msp and the per-sample R
  SparseScatter sc;
  sc.prepare(tree, J, in, split, lay, ACC_MIN, true, false, cells, n_cols, meta, st);
  if (split.n_sparse > 0) {
    Msp = DevBuf((size_t)cells * 8, st, "alloc sparse stripes");
    ck(cudaMemsetAsync(Msp.p, 0, (size_t)cells * 8, st), "memset");
  }
  meta.upload(st);
  const int32_t *d_tiles = meta.at<int32_t>(o_tiles);
  const GramTab *d_tabs = meta.at<GramTab>(o_tabs);
  const int32_t *d_cnt = meta.at<int32_t>(o_cnt), *d_dense = meta.at<int32_t>(o_dense);
  ck(cudaMemsetAsync(Gt.p, 0, (size_t)std::max<int64_t>(G.n_tiles, 1) * GRAM_TILE_CELLS * 8, st), "memset");
  ck(cudaMemsetAsync(err.p, 0, sizeof(int), st), "memset");
  ck(cudaMemsetAsync(clamps.p, 0, sizeof(unsigned long long), st), "memset");
  // the region scatter's pair updates, counted when the call is timed per phase
  DevBuf pair_ctr(SPARSE_PAIR_SLOTS * sizeof(unsigned long long), st, "alloc pair counter");
  ck(cudaMemsetAsync(pair_ctr.p, 0, SPARSE_PAIR_SLOTS * sizeof(unsigned long long), st), "memset");
  Outputs o = bind_outputs(J, st);
  double exec_flops = 0.0;
  Capture cap(g_graph.load() != 0 && !timer.on, st, device);
  const cudaStream_t ls = cap.stream();
  // the sparse-row scatters need no count rows or planes: first, on a side
  // branch beside the presence pass and the gram with option "sparse_overlap"
  SideBranch side(ls, device);
  const PriorityScope prio(split.n_sparse > 0 && g_overlap.load() != 0);
  cap.node_priority = prio.on;
  if (split.n_sparse > 0) {
    const cudaStream_t ss = g_overlap.load() != 0 ? side.fork() : ls;
    timer.begin(4, ss);
    SparseArgs sp{};
    sp.pair_count = timer.on ? pair_ctr.as<unsigned long long>() : nullptr;
    sp.kind = EMB_PRESENCE;
    sp.abs_mask = 0u;
    sp.M = Msp.as<unsigned long long>();
    sp.alpha = 1.0;
    sp.scale = scale;
    sc.launch(meta, in, sp, ACC_MIN, true, g_region_bytes.load(), ss, &kernels);
    timer.end();
  }
  for (size_t b = 0; b < in.P->b0.size(); b++) {
    const int64_t b0 = in.P->b0[b];
    const int64_t d0 = split.dense_ptr[b], nd = split.dense_ptr[b + 1] - d0;
    timer.begin(0);
    enqueue_split_presence(in, J, off, split, b, d_cnt, flags.as<uint8_t>(), ld, n_cols, ls, &kernels);
    if (nd > 0) {
      ck(launch_gram_prep(b0, (int)nd, in.pd->slot_of_node, flags.as<uint8_t>(), ld, in.td->length, d_tabs,
                          (int)nt, npad_tot, K_pad, Pl.p, ls, d_dense + d0),
         "presence planes");
      kernels++;
    }
    timer.end();
    if (nd == 0 || n_tiles == 0) continue;
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
    ga.wait_test = (int)g_tensor_wait_test.load();
    timer.begin(1);
    ck(launch_gram(ga, Pl.p, K_pad, ls), "tensor-core gram");
    timer.end();
    kernels++;
    acc_launches++;
    exec_flops += 2.0 * 3 * (double)GRAM_TILE_CELLS * ga.k_len * n_tiles;
  }
  side.join();
  timer.begin(3);
  for (size_t t = 0; t < nt; t++) {
    GramFinalArgs fa{};
    fa.n = G.gt[t].n;
    fa.n_pad = G.gt[t].n_pad;
    fa.s0 = J.tabs[t].start;
    fa.s1 = J.tabs[t].stop;
    fa.full = J.tabs[t].start == 0 && J.tabs[t].stop == G.gt[t].n / 2;
    fa.Gt = Gt.as<unsigned long long>();
    fa.tile_map = meta.at<int32_t>(o_maps) + G.gt[t].map_off;
    fa.Msp = Msp.p ? Msp.as<unsigned long long>() + lay[t].m_off : nullptr;
    fa.Dsp = sc.Dsp.p ? sc.Dsp.as<unsigned long long>() + off[t] : nullptr;
    fa.out = o.dev[t];
    fa.out_fp32 = J.out_fp32;
    fa.err = err.as<int>();
    fa.clamps = clamps.as<unsigned long long>();
    fa.unnormalized = unnormalized(J.method);
    fa.inv_scale = 1.0 / scale;
    ck(launch_finalize_gram(fa, ls), "finalize");
    kernels++;
  }
  timer.end();
  cap.launch();
  // a synchronous call reads the abort flag and returns UF_ETIMEOUT; an
  // asynchronous one (device outputs on a stream) is not held back for it:
  // the finalize has already written NaN to every output when it is set
  const bool sync = !J.out_is_device || st == nullptr || timer.on;
  const bool pairs_counted = timer.on && sc.region_mode;
  int h_err = 0;
  unsigned long long h_clamps = 0, h_pairs[SPARSE_PAIR_SLOTS] = {};
  if (sync) {
    ck(cudaMemcpyAsync(&h_err, err.p, sizeof(int), cudaMemcpyDeviceToHost, st), "copy flag");
    ck(cudaMemcpyAsync(&h_clamps, clamps.p, sizeof h_clamps, cudaMemcpyDeviceToHost, st), "copy count");
    ck(cudaMemcpyAsync(h_pairs, pair_ctr.p, sizeof h_pairs, cudaMemcpyDeviceToHost, st), "copy count");
  }
  if (!J.out_is_device)
    for (size_t t = 0; t < nt; t++)
      ck(cudaMemcpyAsync(J.tabs[t].out, o.dev[t], o.bytes[t], cudaMemcpyDeviceToHost, st), "copy out");
  flags = DevBuf();
  Pl = DevBuf();
  Gt = DevBuf();
  Msp = DevBuf();
  sc = SparseScatter();
  meta.dev = DevBuf();
  o.tmp.clear();
  err = DevBuf();
  clamps = DevBuf();
  pair_ctr = DevBuf();
  if (sync) ck(cudaStreamSynchronize(st), "synchronize");
  else ck(cudaGetLastError(), "enqueue");
  if (h_err) return fail(UF_ETIMEOUT, "tensor-core kernel: a bounded wait gave up");
  double ms[5] = {0, 0, 0, 0, 0};
  timer.collect(ms);
  fill_reports(tree, J, o, ms, kernels, acc_launches, 1, rows, (int64_t)in.P->b0.size(), exec_flops, GRAM_TN,
               GRAM_TM, std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count());
  for (const TableJob &t : J.tabs)
    if (t.rep) {
      t.rep->chunk_rows = 4096;
      t.rep->graph = cap.on ? 1 : 0;
      t.rep->dense_rows = (int64_t)split.dense.size();
      t.rep->sparse_rows = split.n_sparse;
      t.rep->sparse_pairs = split.pairs;
      t.rep->t_sparse_ms = ms[4];
      t.rep->sparse_pair_updates = pairs_counted ? pair_sum(h_pairs) : -1.0;
      t.rep->clamped = sync ? (int32_t)std::min<unsigned long long>(h_clamps, INT32_MAX) : -1;
    }
  return UF_OK;
}

// Every other method / precision on the CUDA-core stripe kernels.  Throws
// CudaFail on CUDA errors.
uf_status run_stripes(uf_tree *tree, const BatchJob &J, int device, uf_method method, double scale) {
  const auto t_start = std::chrono::steady_clock::now();
  const size_t nt = J.tabs.size();
  const int acc = acc_of(method), kind = kind_of(method);
  const bool fp32 = J.fp32;
  const size_t es = fp32 ? 4 : 8;
  const int planes = kind == EMB_VAW ? 3 : 1;  // embedding planes per branch row
  // stripes in the abs form: FP32 1, 3, 5, 7 of 8, FP64 all; the unweighted
  // numerator alone (unnormalized) all in FP32 too, since a min-form
  // numerator W_k + W_j - 2M carries FP32 rounding relative to W, not to num
  const unsigned amask = acc != ACC_MIN ? 0u
                         : (fp32 && method == UF_UNWEIGHTED_UNNORMALIZED) ? 0xFFu
                                                                          : abs_row_mask(fp32);
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
  // the descriptors of every tile shape the kernel offers (shape 0 above; the
  // others have shorter stripe tiles, so the rows' pitch of shape 0 fits them)
  const int n_shapes = stripe_shapes(acc, fp32, amask);
  // option "tile_shape": a forced shape when the kernel has it, else tuned (or 0)
  const int forced = g_tile_shape.load() >= 0 && g_tile_shape.load() < n_shapes ? (int)g_tile_shape.load() : -1;
  std::vector<std::vector<TabDesc>> shape_tabs(1, tabs);
  std::vector<int> shape_tiles(1, n_tiles), shape_ts(1, tile_s), shape_tk(1, tile_k);
  for (int sh = 1; sh < n_shapes; sh++) {
    int ts2 = 0, tk2 = 0, nt2 = 0;
    stripe_tile_shape(acc, fp32, &ts2, &tk2, sh);
    std::vector<TabDesc> tb2(tabs);
    for (TabDesc &d : tb2) {
      d.m_lo = d.s_lo / ts2;
      d.m_hi = d.s_hi / ts2;
      d.n_ktiles = (d.n + tk2 - 1) / tk2;
      d.tile0 = nt2;
      nt2 += d.n_ktiles * (d.m_hi - d.m_lo + 1);
    }
    shape_tabs.push_back(std::move(tb2));
    shape_tiles.push_back(nt2);
    shape_ts.push_back(ts2);
    shape_tk.push_back(tk2);
  }
  const int64_t nb = tree->n_nodes - 1;
  // FP64: every fixed-point accumulator has a second word (uf_device.cuh),
  // stored after the first: M and M2 at + cells, Dg and the sparse R at + n_cols
  const int words = fp32 ? 1 : 2;
  const double acc_bytes = ((double)cells * 8.0 * (acc == ACC_MIN ? 1 : 2) + n_cols * 8.0) * words;
  const int64_t rows =
      block_rows(nb, (double)n_cols * 8.0 + (double)pitch * es * planes + 8.0 + n_cols * es / 64.0, acc_bytes);
  Inputs in = [&] {
    NvtxRange r("uf: bind inputs");
    return bind_inputs(tree, J, device, rows);
  }();
  cudaStream_t st = J.st;
  const std::shared_ptr<const RowSplit> split_p = [&] {
    NvtxRange r("uf: branch split");
    return get_split(tree, J, in.P, acc, fp32);
  }();
  const RowSplit &split = *split_p;
  const int64_t xrows = std::max<int64_t>(split.max_dense, 1);
  int64_t kernels = 0, acc_launches = 0;
  PhaseTimer timer(g_kernel_timing.load() != 0, st);
  // count rows: stride rounded up to 16 elements for the 16-byte level kernel
  const int64_t ld = round_up(n_cols, 16);
  const size_t m_bytes = (size_t)cells * 8 * words, d_bytes = (size_t)n_cols * 8 * words;
  DevBuf counts((size_t)in.P->n_slots * ld * 8, st, "alloc counts");
  DevBuf X((size_t)xrows * pitch * es * planes, st, "alloc embeddings");
  DevBuf M(m_bytes, st, "alloc stripes");
  DevBuf M2, Dg, diag_tmp, counter(sizeof(int), st, "alloc counter");
  DevBuf clamps(sizeof(unsigned long long), st, "alloc clamp counter");
  DevBuf total((size_t)n_cols * 8, st, "alloc totals"), inv_total((size_t)n_cols * 4, st, "alloc totals");
  // unit order per table and shape: bands of sample tiles whose columns (their
  // u windows and every stripe tile's partner windows) for the rows of a work
  // unit fit in a third of L2, all stripe tiles of a band before the next;
  // without such a band, sample tile fastest over the whole table
  {
    const double l2_budget = 40e6, rows_u = (double)std::min<int64_t>(xrows, 8192) * (double)es * planes;
    for (size_t sh = 0; sh < shape_tabs.size(); sh++)
      for (TabDesc &d : shape_tabs[sh]) {
        const double cols = l2_budget / rows_u - (double)(d.m_hi - d.m_lo + 1) * shape_ts[sh];
        const int kb = (int)std::floor(cols / (2.0 * shape_tk[sh]));
        d.kband = kb >= 1 ? std::min(kb, d.n_ktiles) : d.n_ktiles;
      }
    tabs = shape_tabs[0];
  }
  // table descriptors and row lists: one staged upload
  Meta meta;
  const size_t o_tabs = meta.add(tabs);
  std::vector<size_t> o_shape_tabs(1, o_tabs);
  for (int sh = 1; sh < n_shapes; sh++) o_shape_tabs.push_back(meta.add(shape_tabs[sh]));
  const size_t o_cnt = meta.add(split.cnt_lists);
  const size_t o_dense = meta.add(split.dense);
  const size_t o_dlen = meta.add(split.dense_len);
  std::vector<SpLayout> lay(nt);
  for (size_t t = 0; t < nt; t++) lay[t] = SpLayout{tabs[t].n, tabs[t].off, tabs[t].s_lo, tabs[t].s_hi, tabs[t].m_off};
  SparseScatter sc;
  sc.prepare(tree, J, in, split, lay, acc, !fp32, !fp32, cells, n_cols, meta, st);
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
  if (acc != ACC_MIN) {
    M2 = DevBuf(m_bytes, st, "alloc stripes");
    ck(cudaMemsetAsync(M2.p, 0, m_bytes, st), "memset");
  } else {
    Dg = DevBuf(d_bytes, st, "alloc diagonal");
    diag_tmp = DevBuf(diag_scratch_bytes(fp32, (int)xrows, n_cols), st, "alloc diagonal scratch");
    ck(cudaMemsetAsync(Dg.p, 0, d_bytes, st), "memset");
  }
  ck(cudaMemsetAsync(M.p, 0, m_bytes, st), "memset");
  ck(cudaMemsetAsync(clamps.p, 0, sizeof(unsigned long long), st), "memset");
  // the region scatter's pair updates, counted when the call is timed per phase
  DevBuf pair_ctr(SPARSE_PAIR_SLOTS * sizeof(unsigned long long), st, "alloc pair counter");
  ck(cudaMemsetAsync(pair_ctr.p, 0, SPARSE_PAIR_SLOTS * sizeof(unsigned long long), st), "memset");
  Outputs o = bind_outputs(J, st);
  double exec_flops = 0.0;
  // tile shape and chunk size: tuned once per (accumulator, precision, size
  // bucket; the key's precision slot also tells the all-abs kernel apart)
  const auto key = tune_key(acc, (fp32 ? (amask == 0xFFu ? 2 : 1) : 0) + 4 * (forced + 1), n_tiles, xrows);
  int chunk = stripe_chunk_rows(), shape = forced > 0 ? forced : 0;
  bool tune = false;
  if (g_autotune.load() && !split.dense.empty()) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_tuned_chunk.find(key);
    if (it != g_tuned_chunk.end()) {
      shape = it->second.first;
      chunk = it->second.second;
    } else {
      tune = true;
    }
  }
  auto use_shape = [&](int sh) {
    shape = sh;
    tile_s = shape_ts[sh];
    tile_k = shape_tk[sh];
    n_tiles = shape_tiles[sh];
  };
  use_shape(shape);
  // the launch sequence goes into a CUDA graph unless it is timed per phase
  Capture cap(g_graph.load() != 0 && !timer.on && !tune, st, device);
  const cudaStream_t ls = cap.stream();
  // the sparse-row scatters run after the dense blocks, whose chunk tuning clears M
  auto launch_sparse = [&](cudaStream_t on) {
    SparseArgs sp{};
    sp.pair_count = timer.on ? pair_ctr.as<unsigned long long>() : nullptr;
    sp.kind = kind;
    sp.abs_mask = amask;
    sp.gen_abs = acc == ACC_GEN && !fp32;
    sp.M = M.as<unsigned long long>();
    sp.M2 = M2.as<unsigned long long>();
    sp.alpha = J.alpha;
    sp.scale = scale;
    sc.launch(meta, in, sp, acc, !fp32, g_region_bytes.load(), on, &kernels);
  };
  // with option "sparse_overlap" (default) the sparse-row scatter runs on a
  // side branch beside the count pass, the embeddings and the dense stripe
  // kernel (it needs none of them); otherwise (and while the chunk size is
  // being tuned, which clears M) it runs after the blocks
  SideBranch side(ls, device);
  const PriorityScope prio(split.n_sparse > 0 && !tune && g_overlap.load() != 0);
  cap.node_priority = prio.on;
  if (split.n_sparse > 0 && !tune && g_overlap.load() != 0) {
    const cudaStream_t ss = side.fork();
    timer.begin(4, ss);
    launch_sparse(ss);
    timer.end();
  }
  bool tuned = false;
  for (size_t b = 0; b < in.P->b0.size(); b++) {
    const int64_t b0 = in.P->b0[b];
    const int64_t d0 = split.dense_ptr[b], nd = split.dense_ptr[b + 1] - d0;
    timer.begin(0);
    enqueue_split_counts(in, J, off, split, b, d_cnt, counts.as<double>(), ld, n_cols, ls, &kernels);
    if (nd > 0) {
      ck(launch_emb_rows(kind, fp32, b0, (int)nd, in.pd->slot_of_node, counts.as<double>(), ld,
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
    sa.shape = shape;
    sa.tabs = meta.at<TabDesc>(o_shape_tabs[shape]);
    sa.n_tabs = (int)nt;
    sa.n_tiles = n_tiles;
    sa.n_cols = n_cols;
    sa.M = M.as<unsigned long long>();
    sa.M2 = M2.as<unsigned long long>();
    sa.Dg = Dg.as<unsigned long long>();
    sa.alpha = J.alpha;
    sa.scale = scale;
    sa.counter = counter.as<int>();
    sa.m_lo_off = fp32 ? 0 : cells;
    sa.d_lo_off = fp32 ? 0 : n_cols;
    sa.abs_mask = amask;
    if (tune && !tuned) {
      std::vector<const TabDesc *> tp;
      for (size_t o : o_shape_tabs) tp.push_back(meta.at<TabDesc>(o));
      std::vector<int> tiles(shape_tiles);
      if (forced >= 0) {  // only the forced shape is a candidate
        for (size_t sh = 0; sh < tp.size(); sh++)
          if ((int)sh != forced) tiles[sh] = -1;
      }
      const std::pair<int, int> best = tune_chunk(acc, fp32, sa, tp, tiles, m_bytes, ls);
      use_shape(best.first);
      chunk = best.second;
      sa.chunk = chunk;
      sa.shape = shape;
      sa.tabs = tp[shape];
      sa.n_tiles = n_tiles;
      tuned = true;
      std::lock_guard<std::mutex> g(g_tune_mu);
      g_tuned_chunk[key] = best;
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
  if (split.n_sparse > 0 && !side.ev_fork) {  // not launched beside a dense block
    timer.begin(4);
    launch_sparse(ls);
    timer.end();
  }
  side.join();
  timer.begin(3);
  for (size_t t = 0; t < nt; t++) {
    FinalArgs fa{};
    fa.method = acc == ACC_MIN ? (kind == EMB_PRESENCE ? 0 : 2) : 3;
    fa.unnormalized = unnormalized(method);
    fa.n = tabs[t].n;
    fa.s0 = J.tabs[t].start;
    fa.s1 = J.tabs[t].stop;
    fa.full = J.tabs[t].start == 0 && J.tabs[t].stop == tabs[t].n / 2;
    fa.abs_mask = amask;
    fa.gen_abs = acc == ACC_VAW || (acc == ACC_GEN && !fp32);
    fa.clamps = clamps.as<unsigned long long>();
    fa.M = M.as<unsigned long long>() + tabs[t].m_off;
    fa.M2 = M2.p ? M2.as<unsigned long long>() + tabs[t].m_off : nullptr;
    fa.Dg = Dg.p ? Dg.as<unsigned long long>() + off[t] : nullptr;
    fa.Dsp = sc.Dsp.p ? sc.Dsp.as<unsigned long long>() + off[t] : nullptr;
    fa.m_lo_off = fp32 ? 0 : cells;
    fa.d_lo_off = fp32 ? 0 : n_cols;
    fa.inv_scale = 1.0 / scale;
    fa.out = o.dev[t];
    fa.out_fp32 = J.out_fp32;
    ck(launch_finalize(fa, ls), "finalize");
    kernels++;
  }
  timer.end();
  cap.launch();
  // a synchronous call reads how many min-form numerators were raised to 0
  const bool sync = !J.out_is_device || st == nullptr || timer.on;
  const bool pairs_counted = timer.on && sc.region_mode;
  unsigned long long h_clamps = 0, h_pairs[SPARSE_PAIR_SLOTS] = {};
  if (sync) {
    ck(cudaMemcpyAsync(&h_clamps, clamps.p, sizeof h_clamps, cudaMemcpyDeviceToHost, st), "copy count");
    ck(cudaMemcpyAsync(h_pairs, pair_ctr.p, sizeof h_pairs, cudaMemcpyDeviceToHost, st), "copy count");
  }
  if (!J.out_is_device)
    for (size_t t = 0; t < nt; t++)
      ck(cudaMemcpyAsync(J.tabs[t].out, o.dev[t], o.bytes[t], cudaMemcpyDeviceToHost, st), "copy out");
  // buffers go back to the stream-ordered pool here
  counts = DevBuf();
  X = DevBuf();
  M = DevBuf();
  M2 = DevBuf();
  Dg = DevBuf();
  sc = SparseScatter();
  diag_tmp = DevBuf();
  counter = DevBuf();
  clamps = DevBuf();
  pair_ctr = DevBuf();
  meta.dev = DevBuf();
  total = DevBuf();
  inv_total = DevBuf();
  o.tmp.clear();
  if (sync) ck(cudaStreamSynchronize(st), "synchronize");
  else ck(cudaGetLastError(), "enqueue");
  double ms[5] = {0, 0, 0, 0, 0};
  timer.collect(ms);
  fill_reports(tree, J, o, ms, kernels, acc_launches, 0, rows, (int64_t)in.P->b0.size(), exec_flops, tile_s,
               tile_k, std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count());
  for (const TableJob &t : J.tabs)
    if (t.rep) {
      t.rep->chunk_rows = chunk;
      t.rep->graph = cap.on ? 1 : 0;
      t.rep->clamped = sync ? (int32_t)std::min<unsigned long long>(h_clamps, INT32_MAX) : -1;
      t.rep->dense_rows = (int64_t)split.dense.size();
      t.rep->sparse_rows = split.n_sparse;
      t.rep->sparse_pairs = split.pairs;
      t.rep->t_sparse_ms = ms[4];
      t.rep->sparse_pair_updates = pairs_counted ? pair_sum(h_pairs) : -1.0;
    }
  return UF_OK;
}

}  // namespace

// One compute call on the current device; throws CudaFail on CUDA errors.
uf_status run_batch(uf_tree *tree, const BatchJob &J) {
  static const char *const names[2][7] = {
      {"uf_compute unweighted fp64", "uf_compute weighted_unnormalized fp64", "uf_compute weighted_normalized fp64",
       "uf_compute generalized fp64", "uf_compute unweighted_unnormalized fp64",
       "uf_compute vaw_weighted_unnormalized fp64", "uf_compute vaw_weighted_normalized fp64"},
      {"uf_compute unweighted mixed", "uf_compute weighted_unnormalized mixed",
       "uf_compute weighted_normalized mixed", "uf_compute generalized mixed", "uf_compute unweighted_unnormalized mixed",
       "uf_compute vaw_weighted_unnormalized mixed", "uf_compute vaw_weighted_normalized mixed"}};
  NvtxRange call_range(names[J.fp32 ? 1 : 0][(int)J.method % 7]);
  g_h2d = 0.0;
  int device = 0;
  ck(cudaGetDevice(&device), "cudaGetDevice");
  keep_pool_memory(device);
  uf_method method = J.method;
  if (method == UF_GENERALIZED && J.alpha == 1.0) method = UF_WEIGHTED_NORMALIZED;  // s^0 == 1
  const int kind = kind_of(method);
  double scale = 0.0;  // one fixed-point scale valid for every table of the call
  for (const TableJob &t : J.tabs) {
    const double s = accum_scale(tree, t.table, kind);
    scale = scale == 0.0 ? s : std::min(scale, s);
  }
  // (the unweighted numerator alone stays on the CUDA-core kernels: the gram
  // gives it as W_i + W_j - 2G, rounded relative to W rather than to itself)
  if (method == UF_UNWEIGHTED && J.fp32 && g_tensor_path.load()) {
    // the tensor path stores the gram tiles the stripes need (and the
    // diagonal) plus the sparse rows' stripe cells; when those do not fit in
    // half the free memory the CUDA-core stripe kernels take the call
    const GramPlan G = gram_plan(J);
    const double need = (double)G.n_tiles * GRAM_TILE_CELLS * 8.0 + (double)stripe_cells(J) * 8.0;
    if (need <= 0.5 * available_bytes()) return run_gram(tree, J, device, scale);
  }
  return run_stripes(tree, J, device, method, scale);
}

void forget_tuned_chunks() {
  std::lock_guard<std::mutex> g(g_tune_mu);
  g_tuned_chunk.clear();
}

}  // namespace rt
}  // namespace ufg
