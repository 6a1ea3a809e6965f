// uf_host.cpp -- host runtime behind the C ABI of include/unifrac_gb300.h.
//
// Validation of trees and tables, their host preparation (children, tip
// ranges, CSC view), the postorder branch-block plan with level batching and
// live count slots, device residency of the inputs, the fixed-point scale,
// process options and the extern "C" entry points.  One call's launch
// sequence is in uf_run.cpp, the dense / sparse branch split in uf_split.cpp.
// Stripes are the paper's independent subproblems (Abstract; Sec. 2 Fig. 1).
#include "uf_runtime.h"

#include <unistd.h>

#include <condition_variable>
#include <deque>
#include <exception>

using namespace ufg;
using namespace ufg::rt;

namespace ufg {
namespace rt {

thread_local std::string g_err;
thread_local double g_h2d = 0.0;
std::atomic<int64_t> g_branch_block{0};
std::atomic<int64_t> g_sparse_fuse{2};
std::atomic<int64_t> g_kernel_timing{0};
std::atomic<int64_t> g_tensor_path{1};
std::atomic<int64_t> g_graph{1};
std::atomic<int64_t> g_autotune{1};
std::atomic<int64_t> g_sparse{1};
std::atomic<int64_t> g_overlap{1};
std::atomic<int64_t> g_tensor_wait_test{0};
std::atomic<int64_t> g_tile_shape{-1};
std::atomic<int64_t> g_region_bytes{(int64_t)SPARSE_REGION_BYTES_DEFAULT};

int host_threads() {
  const unsigned h = std::thread::hardware_concurrency();
  return (int)std::max(1u, std::min(h == 0 ? 1u : h, 16u));
}

namespace {

// The host worker pool behind parallel_for.  A call queues a job (its body,
// n, and counters on the caller's stack); idle workers attach to the front
// job and take indices until none is left, then detach.  The caller takes
// indices too, removes the job from the queue, and waits until every index
// has finished and no worker is attached, so the job never outlives its call.
struct PoolJob {
  const std::function<void(int)> *body;
  int n;
  std::atomic<int> next{0}, left{0};
  int users = 0;  // attached workers (guarded by the pool mutex)
  std::mutex emu;
  std::exception_ptr error;  // the first exception a body threw
};

struct Pool {
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<PoolJob *> q;
  std::vector<std::thread> workers;
  bool stop = false;
  pid_t pid = getpid();

  // Starts up to n_workers threads; if the system refuses one, the pool keeps
  // those it has (possibly none: run_parallel then runs on the caller alone).
  explicit Pool(int n_workers) {
    try {
      workers.reserve(n_workers);
      for (int i = 0; i < n_workers; i++) workers.emplace_back([this] { work(); });
    } catch (const std::exception &) {
    }
  }
  ~Pool() {
    {
      std::lock_guard<std::mutex> g(mu);
      stop = true;
    }
    cv_work.notify_all();
    for (auto &w : workers)
      if (w.joinable()) w.join();
  }
  static void take(PoolJob *j) {
    for (int i; (i = j->next.fetch_add(1)) < j->n;) {
      try {
        (*j->body)(i);
      } catch (...) {
        std::lock_guard<std::mutex> g(j->emu);
        if (!j->error) j->error = std::current_exception();
      }
      j->left.fetch_sub(1);
    }
  }
  void work() {
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
      cv_work.wait(lk, [&] { return stop || !q.empty(); });
      if (stop) return;
      PoolJob *j = q.front();
      j->users++;
      lk.unlock();
      take(j);
      lk.lock();
      if (!q.empty() && q.front() == j) q.pop_front();  // no index left to hand out
      j->users--;
      cv_done.notify_all();
    }
  }
};

Pool *host_pool() {
  // started on first use, never destroyed while other threads may use it
  static Pool *pool = new Pool(std::max(0, host_threads() - 1));
  return pool;
}

}  // namespace

void run_parallel(int n, const std::function<void(int)> &body) {
  if (n <= 0) return;
  Pool *pool = n > 1 ? host_pool() : nullptr;
  if (!pool || pool->workers.empty() || pool->pid != getpid()) {
    for (int i = 0; i < n; i++) body(i);  // an exception propagates from here directly
    return;
  }
  PoolJob j;
  j.body = &body;
  j.n = n;
  j.left = n;
  {
    std::lock_guard<std::mutex> g(pool->mu);
    pool->q.push_back(&j);
  }
  pool->cv_work.notify_all();
  Pool::take(&j);
  std::unique_lock<std::mutex> lk(pool->mu);
  for (auto it = pool->q.begin(); it != pool->q.end(); ++it)
    if (*it == &j) {
      pool->q.erase(it);
      break;
    }
  pool->cv_done.wait(lk, [&] { return j.left.load() == 0 && j.users == 0; });
  lk.unlock();
  if (j.error) std::rethrow_exception(j.error);  // e.g. std::bad_alloc becomes UF_ENOMEM
}

uf_status fail(uf_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

void ck(cudaError_t e, const char *what) {
  if (e != cudaSuccess) {
    cudaGetLastError();  // clear a sticky launch error where possible
    uf_status st = (e == cudaErrorMemoryAllocation) ? UF_ENOMEM : UF_ECUDA;
    fail(st, "%s: %s", what, cudaGetErrorString(e));
    throw CudaFail{st};
  }
}

// Pinned chunks for pinned_upload, one ring per device (the copy stream and
// events belong to it); the chunks themselves are portable pinned memory.
namespace {
struct UploadRing {
  static constexpr int NBUF = 4;
  static constexpr size_t CHUNK = (size_t)32 << 20;
  char *buf[NBUF] = {};
  cudaEvent_t ev[NBUF] = {};
  bool busy[NBUF] = {};
  cudaStream_t st = nullptr;
  bool ok = false;
};
std::mutex g_ring_mu;
std::map<int, UploadRing> g_rings;
}  // namespace

void pinned_upload(void *dst, const void *src, size_t bytes) {
  if (bytes == 0) return;
  int dev = 0;
  ck(cudaGetDevice(&dev), "upload");
  std::lock_guard<std::mutex> g(g_ring_mu);
  UploadRing &R = g_rings[dev];
  if (!R.ok) {
    bool good = cudaStreamCreateWithFlags(&R.st, cudaStreamNonBlocking) == cudaSuccess;
    for (int i = 0; good && i < UploadRing::NBUF; i++)
      good = cudaHostAlloc((void **)&R.buf[i], UploadRing::CHUNK, cudaHostAllocPortable) == cudaSuccess &&
             cudaEventCreateWithFlags(&R.ev[i], cudaEventDisableTiming) == cudaSuccess;
    if (!good) {  // no pinned memory: the driver's own staged copy
      cudaGetLastError();
      ck(cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice), "upload");
      return;
    }
    R.ok = true;
  }
  const char *s = static_cast<const char *>(src);
  char *d = static_cast<char *>(dst);
  const int nt = std::max(1, std::min(host_threads(), 8));
  int i = 0;
  for (size_t off = 0; off < bytes; off += UploadRing::CHUNK, i = (i + 1) % UploadRing::NBUF) {
    const size_t n = std::min(UploadRing::CHUNK, bytes - off);
    if (R.busy[i]) ck(cudaEventSynchronize(R.ev[i]), "upload");
    char *b = R.buf[i];
    parallel_for(nt, [&](int c) {
      const size_t a0 = n * c / nt, a1 = n * (c + 1) / nt;
      memcpy(b + a0, s + off + a0, a1 - a0);
    });
    ck(cudaMemcpyAsync(d + off, b, n, cudaMemcpyHostToDevice, R.st), "upload");
    ck(cudaEventRecord(R.ev[i], R.st), "upload");
    R.busy[i] = true;
  }
  ck(cudaStreamSynchronize(R.st), "upload");
  for (bool &x : R.busy) x = false;
}

uf_tree::Dev &tree_dev(uf_tree *t, int device) {
  auto it = t->dev.find(device);
  if (it != t->dev.end()) return it->second;
  DevPack pk;
  const size_t i_len = pk.add(t->length), i_ton = pk.add(t->tip_of_node), i_cp = pk.add(t->child_ptr),
               i_ci = pk.add(t->child_idx), i_lo = pk.add(t->tip_lo), i_hi = pk.add(t->tip_hi);
  uf_tree::Dev d;
  d.base = pk.upload("tree upload");
  d.length = DevPack::at<double>(d.base, pk, i_len);
  d.tip_of_node = DevPack::at<int32_t>(d.base, pk, i_ton);
  d.child_ptr = DevPack::at<int32_t>(d.base, pk, i_cp);
  d.child_idx = DevPack::at<int32_t>(d.base, pk, i_ci);
  d.tip_lo = DevPack::at<int32_t>(d.base, pk, i_lo);
  d.tip_hi = DevPack::at<int32_t>(d.base, pk, i_hi);
  return t->dev[device] = d;
}

uf_table::Dev &table_dev(uf_table *t, int device) {
  auto it = t->dev.find(device);
  if (it != t->dev.end()) return it->second;
  DevPack pk;
  const size_t i_tot = pk.add(t->total), i_inv = pk.add(t->inv_total_f), i_cp = pk.add(t->col_ptr),
               i_row = pk.add(t->col_row), i_val = pk.add(t->col_val);
  uf_table::Dev d;
  d.base = pk.upload("table upload");
  d.total = DevPack::at<double>(d.base, pk, i_tot);
  d.inv_total_f = DevPack::at<float>(d.base, pk, i_inv);
  d.col_ptr = DevPack::at<int64_t>(d.base, pk, i_cp);
  d.col_row = DevPack::at<int32_t>(d.base, pk, i_row);
  d.col_val = DevPack::at<double>(d.base, pk, i_val);
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
  P->lists.resize(std::max<int64_t>(nb, 0));
  std::vector<int32_t> level(t->n_nodes, 0);
  std::vector<int64_t> count;
  std::vector<int32_t> free_slots;
  int32_t next_slot = 0;
  for (int64_t b0 = 0; b0 < nb; b0 += rows) {
    const int64_t b1 = std::min(nb, b0 + rows);
    P->b0.push_back(b0);
    P->b1.push_back(b1);
    // list 0: the block's tips; list L + 1: its internal nodes of level L
    // (one more than the deepest internal child in the block); filled by a
    // counting sort, each list in node order
    count.assign(1, 0);
    for (int64_t v = b0; v < b1; v++) {
      if (t->tip_of_node[v] >= 0) {
        level[v] = -1;
        count[0]++;
        continue;
      }
      int32_t L = 0;
      for (int32_t c = t->child_ptr[v]; c < t->child_ptr[v + 1]; c++) {
        const int32_t ch = t->child_idx[c];
        if (ch >= b0 && t->tip_of_node[ch] < 0) L = std::max(L, level[ch] + 1);
      }
      level[v] = L;
      if ((int64_t)count.size() < L + 2) count.resize(L + 2, 0);
      count[L + 1]++;
    }
    std::vector<std::pair<int64_t, int>> ls(count.size());
    int64_t at = b0;
    for (size_t l = 0; l < count.size(); l++) {
      ls[l] = {at, (int)count[l]};
      count[l] = at;  // next position of list l
      at += ls[l].second;
    }
    for (int64_t v = b0; v < b1; v++) P->lists[count[level[v] + 1]++] = (int32_t)v;
    P->launches.push_back(std::move(ls));
    // slots for the block's nodes (the first block takes fresh slots in order)
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
    // release: children of this block's nodes, and nodes whose parent is the
    // root (never read again); nothing is reused after the last block
    if (b1 < nb)
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
  DevPack pk;
  const size_t i_l = pk.add(P->lists), i_s = pk.add(P->slot_of_node);
  Plan::Dev d;
  d.base = pk.upload("plan upload");
  d.lists = DevPack::at<int32_t>(d.base, pk, i_l);
  d.slot_of_node = DevPack::at<int32_t>(d.base, pk, i_s);
  return P->dev[device] = d;
}

}  // namespace rt
}  // namespace ufg

namespace {

// Upper bound on every value an accumulator of this kind can reach:
//   l * p embeddings:         D_k = sum_f p_f dist(f) <= max tip distance
//   l * presence embeddings:  W_k <= min(total length, sum_{f in k} dist(f))
//   generalized (den, Q):     den <= sum l s^alpha <= 2 (W_k + W_j)
//   variance-adjusted (den, N): den <= w_max (D_k + D_j), with the weight
//                             1 / sqrt(m_v (m - m_v)) <= w_max = max(1, 1 / c_min)
//                             (both factors are sums of counts >= c_min, or 0)
double accum_bound(uf_tree *tree, uf_table *table, int kind) {
  if (kind == EMB_SCALED) return tree->max_tip_dist;
  if (kind == EMB_VAW) return 2.0 * tree->max_tip_dist * std::max(1.0, 1.0 / table->min_count);
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

// Samples one compute call may hold on its combined sample axis (summed over
// a batch's tables): column numbers, a table's n + S and the axis length stay
// below 2^31 in the kernels' 32-bit index arithmetic.
constexpr int64_t MAX_CALL_SAMPLES = int64_t(1) << 30;

uf_status check_args(const uf_tree *tree, const uf_table *table, uf_method method, double alpha,
                     uf_precision precision) {
  if (!tree || !table) return fail(UF_EINVAL, "null tree or table");
  if (method < UF_UNWEIGHTED || method > UF_VAW_WEIGHTED_NORMALIZED)
    return fail(UF_EINVAL, "unknown method %d", (int)method);
  if (precision != UF_FP64 && precision != UF_MIXED) return fail(UF_EINVAL, "unknown precision %d", (int)precision);
  if (method == UF_GENERALIZED && !(alpha >= 0.0 && alpha <= 1.0))
    return fail(UF_EINVAL, "alpha must be in [0, 1] (got %g)", alpha);
  if (table->n_features != tree->n_tips)
    return fail(UF_ETABLE, "table has %lld features but the tree has %lld tips",
                (long long)table->n_features, (long long)tree->n_tips);
  return UF_OK;
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
      forget_tuned_chunks();
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
  if (!strcmp(name, "tensor_wait_test")) {
    if (value != 0 && value != 1) return fail(UF_EINVAL, "tensor_wait_test must be 0 or 1");
    g_tensor_wait_test = value;
    return UF_OK;
  }
  if (!strcmp(name, "sparse_overlap")) {
    if (value != 0 && value != 1) return fail(UF_EINVAL, "sparse_overlap must be 0 or 1");
    g_overlap = value;
    return UF_OK;
  }
  if (!strcmp(name, "sparse_fuse")) {
    if (value != 0 && value != 2 && value != 6) return fail(UF_EINVAL, "sparse_fuse must be 0, 2 or 6");
    g_sparse_fuse = value;
    return UF_OK;
  }
  if (!strcmp(name, "tile_shape")) {
    if (value < -1 || value > 1) return fail(UF_EINVAL, "tile_shape must be -1, 0 or 1");
    g_tile_shape = value;
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
  if (!strcmp(name, "sparse_overlap")) return g_overlap.load();
  if (!strcmp(name, "tensor_wait_test")) return g_tensor_wait_test.load();
  if (!strcmp(name, "tile_shape")) return g_tile_shape.load();
  if (!strcmp(name, "sparse_fuse")) return g_sparse_fuse.load();
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
  try {
    // validation over node ranges in parallel (the first failing node wins)
    const int T = (int)std::max<int64_t>(1, std::min<int64_t>(host_threads(), n_nodes / 65536));
    std::vector<int64_t> bad(T, -1);
    parallel_for(T, [&](int c) {
      const int64_t i0 = (n_nodes - 1) * c / T, i1 = (n_nodes - 1) * (c + 1) / T;
      for (int64_t i = i0; i < i1; i++)
        if (parent[i] <= i || parent[i] >= n_nodes || !std::isfinite(length[i]) || length[i] < 0.0) {
          bad[c] = i;
          return;
        }
    });
    for (int c = 0; c < T; c++)
      if (bad[c] >= 0) {
        const int64_t i = bad[c];
        if (parent[i] <= i || parent[i] >= n_nodes)
          return fail(UF_ETREE, "node %lld: parent %lld must be in (%lld, %lld)", (long long)i,
                      (long long)parent[i], (long long)i, (long long)n_nodes);
        return fail(UF_ETREE, "node %lld: length %g must be finite and >= 0", (long long)i, length[i]);
      }
    auto t = std::make_unique<uf_tree>();
    static std::atomic<uint64_t> next_tree_id{1};
    t->id = next_tree_id++;
    t->n_nodes = n_nodes;
    t->parent.assign(parent, parent + n_nodes);
    t->length.assign(length, length + n_nodes);
    t->length[n_nodes - 1] = 0.0;  // no branch above the root
    // one pass in index order (children come before their parent, so a
    // node's child count is final when it is reached): child counts, tip
    // numbers in index order, and each node's tip range [lo, hi) and tip count
    std::vector<int32_t> nchild(n_nodes, 0), under(n_nodes, 0);
    t->tip_of_node.assign(n_nodes, -1);
    t->tip_lo.assign(n_nodes, INT32_MAX);
    t->tip_hi.assign(n_nodes, -1);
    int32_t tips = 0;
    for (int64_t v = 0; v < n_nodes; v++) {
      if (nchild[v] == 0) {
        t->tip_of_node[v] = tips;
        t->tip_lo[v] = tips;
        t->tip_hi[v] = tips + 1;
        under[v] = 1;
        tips++;
      }
      if (v + 1 < n_nodes) {
        const int64_t p = parent[v];
        nchild[p]++;
        t->tip_lo[p] = std::min(t->tip_lo[p], t->tip_lo[v]);
        t->tip_hi[p] = std::max(t->tip_hi[p], t->tip_hi[v]);
        under[p] += under[v];
      }
    }
    t->n_tips = tips;
    t->child_ptr.assign(n_nodes + 1, 0);
    for (int64_t i = 0; i < n_nodes; i++) t->child_ptr[i + 1] = t->child_ptr[i] + nchild[i];
    t->child_idx.assign(std::max<int64_t>(n_nodes - 1, 1), 0);
    for (int64_t i = 0; i + 1 < n_nodes; i++) {
      const int64_t p = parent[i];
      t->child_idx[t->child_ptr[p + 1] - nchild[p]--] = (int32_t)i;  // ascending child order
    }
    // one pass in reverse order (parents first): root distances, the tips'
    // distances, and the tip ranges that are not contiguous (both set to -1)
    t->dist.assign(n_nodes, 0.0);
    t->tip_dist.resize(std::max<int32_t>(tips, 1));
    for (int64_t v = n_nodes - 1; v >= 0; v--) {
      if (v + 1 < n_nodes) {
        t->dist[v] = t->length[v] + t->dist[parent[v]];
        t->total_length += t->length[v];
      }
      if (t->tip_of_node[v] >= 0) {
        t->max_tip_dist = std::max(t->max_tip_dist, t->dist[v]);
        t->tip_dist[t->tip_of_node[v]] = t->dist[v];
      }
      if ((int64_t)t->tip_hi[v] - t->tip_lo[v] != under[v]) t->tip_lo[v] = t->tip_hi[v] = -1;
    }
    *out = t.release();
    return UF_OK;
  } catch (const std::bad_alloc &) {
    return fail(UF_ENOMEM, "host allocation failed");
  } catch (const std::exception &e) {
    return fail(UF_ENOMEM, "host resources: %s", e.what());
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
    auto t = std::make_unique<uf_table>();
    static std::atomic<uint64_t> next_id{1};
    t->n = n_samples;
    t->n_features = n_features;
    t->nnz = nnz;
    t->total.assign(n_samples, 0.0);
    t->inv_total_f.assign(n_samples, 0.f);
    // one pass per thread over its samples: validation (the first failing
    // sample wins, as a sequential scan would report), sample totals and the
    // thread's column counts for the CSC view (a counting sort)
    std::vector<int64_t> bad_k(T, -1);
    std::vector<std::string> bad_msg(T);
    std::vector<std::vector<int64_t>> cnt(T);
    // and the presence bound for this tree: max over samples of the summed
    // root distances of their tips (accum_bound)
    std::vector<double> pres(T, 0.0);
    std::vector<double> cmin(T, INFINITY);  // the smallest count (variance-adjusted bound)
    const double *tip_dist = tree->tip_dist.data();
    parallel_for(T, [&](int c) {
      char buf[160];
      for (int64_t k = k_lo[c]; k < k_lo[c + 1]; k++) {
        double s = 0.0, w = 0.0;
        for (int64_t q = indptr[k]; q < indptr[k + 1]; q++) {
          if (indices[q] < 0 || indices[q] >= n_features)
            snprintf(buf, sizeof buf, "sample %lld: feature index %d out of range", (long long)k, indices[q]);
          else if (q > indptr[k] && indices[q] <= indices[q - 1])
            snprintf(buf, sizeof buf, "sample %lld: feature indices not strictly increasing", (long long)k);
          else if (!std::isfinite(data[q]) || data[q] <= 0.0)
            snprintf(buf, sizeof buf, "sample %lld: count %g must be finite and > 0", (long long)k, data[q]);
          else {
            s += data[q];
            w += tip_dist[indices[q]];
            cmin[c] = std::min(cmin[c], data[q]);
            continue;
          }
          bad_k[c] = k;
          bad_msg[c] = buf;
          return;
        }
        t->total[k] = s;
        t->inv_total_f[k] = (float)(1.0 / s);
        pres[c] = std::max(pres[c], w);
      }
    });
    for (int c = 0; c < T; c++)
      if (bad_k[c] >= 0) return fail(UF_ETABLE, "%s", bad_msg[c].c_str());
    t->id = next_id++;
    t->presence_bound[tree->id] = *std::max_element(pres.begin(), pres.end());
    t->min_count = *std::min_element(cmin.begin(), cmin.end());
    // each thread's column counts (a counting sort) and, below, its scatter
    // run over feature blocks: a sample's entries are sorted by feature, so
    // each block's entries of a sample are the run after the previous
    // block's, and one block's counts and writes stay within its columns
    // (cache-resident) instead of spreading over every column
    const int NB = (int)std::max<int64_t>(1, std::min<int64_t>(64, n_features / 1024));
    auto by_blocks = [&](int c, auto &&visit) {
      const int64_t k0 = k_lo[c], nk = k_lo[c + 1] - k0;
      std::vector<int64_t> cur(indptr + k0, indptr + k0 + nk);
      for (int b = 0; b < NB; b++) {
        const int64_t fend = n_features * (b + 1) / NB;
        for (int64_t i = 0; i < nk; i++) {
          const int64_t qe = indptr[k0 + i + 1];
          int64_t q = cur[i];
          for (; q < qe && indices[q] < fend; q++) visit(k0 + i, q);
          cur[i] = q;
        }
      }
    };
    parallel_for(T, [&](int c) {
      cnt[c].assign(n_features, 0);
      int64_t *cc = cnt[c].data();
      by_blocks(c, [&](int64_t, int64_t q) { cc[indices[q]]++; });
    });
    // column starts, then each thread's first slot in every column (its
    // samples go behind the earlier threads'), over feature ranges in parallel
    t->col_ptr.assign(n_features + 1, 0);
    const int TF = (int)std::max<int64_t>(1, std::min<int64_t>(host_threads(), n_features / 4096));
    parallel_for(TF, [&](int c) {
      const int64_t f0 = n_features * c / TF, f1 = n_features * (c + 1) / TF;
      for (int64_t f = f0; f < f1; f++) {
        int64_t x = 0;
        for (int u = 0; u < T; u++) x += cnt[u][f];
        t->col_ptr[f + 1] = x;
      }
    });
    for (int64_t f = 0; f < n_features; f++) t->col_ptr[f + 1] += t->col_ptr[f];
    parallel_for(TF, [&](int c) {
      const int64_t f0 = n_features * c / TF, f1 = n_features * (c + 1) / TF;
      for (int64_t f = f0; f < f1; f++) {
        int64_t at = t->col_ptr[f];
        for (int u = 0; u < T; u++) {
          const int64_t x = cnt[u][f];
          cnt[u][f] = at;
          at += x;
        }
      }
    });
    t->col_row.resize(std::max<int64_t>(nnz, 1));  // every entry written below (nnz >= 1)
    t->col_val.resize(std::max<int64_t>(nnz, 1));
    parallel_for(T, [&](int c) {
      int64_t *slot = cnt[c].data();
      by_blocks(c, [&](int64_t k, int64_t q) {
        const int64_t at = slot[indices[q]]++;
        t->col_row[at] = (int32_t)k;
        t->col_val[at] = data[q];
      });
    });
    *out = t.release();
    return UF_OK;
  } catch (const std::bad_alloc &) {
    return fail(UF_ENOMEM, "host allocation failed");
  } catch (const std::exception &e) {
    return fail(UF_ENOMEM, "host resources: %s", e.what());
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
  if (table->n > MAX_CALL_SAMPLES)
    return fail(UF_EINVAL, "%lld samples: a compute call takes at most 2^30", (long long)table->n);
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
  if (out_is_device && (st = check_device_output(out, "out")) != UF_OK) return st;
  BatchJob J{method, alpha, precision == UF_MIXED, out_is_device, out_fp32, (cudaStream_t)cuda_stream, {}};
  J.tabs.push_back(TableJob{const_cast<uf_table *>(table), stripe_start, stripe_stop, out, rep});
  try {
    return run_batch(const_cast<uf_tree *>(tree), J);
  } catch (const CudaFail &f) {
    return f.st;
  } catch (const std::bad_alloc &) {
    return fail(UF_ENOMEM, "host allocation failed");
  } catch (const std::exception &e) {
    return fail(UF_ENOMEM, "host resources: %s", e.what());
  }
}

uf_status uf_compute_batch(const uf_tree *tree, const uf_table *const *tables, int64_t n_tables,
                           uf_method method, double alpha, uf_precision precision,
                           void *const *outs, int out_is_device, uf_report *reps,
                           void *cuda_stream) {
  g_err.clear();
  if (!tables || !outs || n_tables < 0) return fail(UF_EINVAL, "null tables or outputs");
  BatchJob J{method, alpha, precision == UF_MIXED, out_is_device, 0, (cudaStream_t)cuda_stream, {}};
  int64_t n_axis = 0;
  for (int64_t t = 0; t < n_tables; t++) {
    uf_status st = check_args(tree, tables[t], method, alpha, precision);
    if (st) return st;
    if (reps) memset(&reps[t], 0, sizeof(uf_report));
    const int64_t S = uf_stripe_count(tables[t]->n);
    if (S == 0) continue;  // fewer than two samples: nothing to write
    if (!outs[t]) return fail(UF_EINVAL, "null output buffer for table %lld", (long long)t);
    n_axis += tables[t]->n;
    if (n_axis > MAX_CALL_SAMPLES)
      return fail(UF_EINVAL, "tables 0..%lld hold %lld samples: a compute call takes at most 2^30",
                  (long long)t, (long long)n_axis);
    J.tabs.push_back(TableJob{const_cast<uf_table *>(tables[t]), 0, S, outs[t], reps ? &reps[t] : nullptr});
  }
  if (J.tabs.empty()) return UF_OK;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return fail(UF_ECUDA, "no CUDA device available");
  }
  if (out_is_device)
    for (const TableJob &t : J.tabs) {
      const uf_status st = check_device_output(t.out, "an output buffer");
      if (st != UF_OK) return st;
    }
  try {
    return run_batch(const_cast<uf_tree *>(tree), J);
  } catch (const CudaFail &f) {
    return f.st;
  } catch (const std::bad_alloc &) {
    return fail(UF_ENOMEM, "host allocation failed");
  } catch (const std::exception &e) {
    return fail(UF_ENOMEM, "host resources: %s", e.what());
  }
}

uf_status uf_compute_ranges(const uf_tree *tree, const uf_table *const *tables, const int64_t *starts,
                            const int64_t *stops, int64_t n_jobs, uf_method method, double alpha,
                            uf_precision precision, void *const *outs, int out_is_device, int out_fp32,
                            uf_report *reps, void *cuda_stream) {
  g_err.clear();
  if (!tables || !starts || !stops || !outs || n_jobs < 0) return fail(UF_EINVAL, "null job arrays");
  BatchJob J{method, alpha, precision == UF_MIXED, out_is_device, out_fp32, (cudaStream_t)cuda_stream, {}};
  int64_t n_axis = 0;
  for (int64_t t = 0; t < n_jobs; t++) {
    uf_status st = check_args(tree, tables[t], method, alpha, precision);
    if (st) return st;
    if (reps) memset(&reps[t], 0, sizeof(uf_report));
    const int64_t S = uf_stripe_count(tables[t]->n);
    if (starts[t] < 0 || stops[t] < starts[t] || stops[t] > S)
      return fail(UF_ERANGE, "job %lld: stripe range [%lld, %lld) outside [0, %lld]", (long long)t,
                  (long long)starts[t], (long long)stops[t], (long long)S);
    if (starts[t] == stops[t]) continue;  // nothing to write
    if (!outs[t]) return fail(UF_EINVAL, "null output buffer for job %lld", (long long)t);
    n_axis += tables[t]->n;
    if (n_axis > MAX_CALL_SAMPLES)
      return fail(UF_EINVAL, "jobs 0..%lld hold %lld samples: a compute call takes at most 2^30", (long long)t,
                  (long long)n_axis);
    J.tabs.push_back(
        TableJob{const_cast<uf_table *>(tables[t]), starts[t], stops[t], outs[t], reps ? &reps[t] : nullptr});
  }
  if (J.tabs.empty()) return UF_OK;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return fail(UF_ECUDA, "no CUDA device available");
  }
  if (out_is_device)
    for (const TableJob &t : J.tabs) {
      const uf_status st = check_device_output(t.out, "an output buffer");
      if (st != UF_OK) return st;
    }
  try {
    return run_batch(const_cast<uf_tree *>(tree), J);
  } catch (const CudaFail &f) {
    return f.st;
  } catch (const std::bad_alloc &) {
    return fail(UF_ENOMEM, "host allocation failed");
  } catch (const std::exception &e) {
    return fail(UF_ENOMEM, "host resources: %s", e.what());
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

uf_status check_device_output(const void *p, const char *what) {
  int cur = 0;
  cudaPointerAttributes at{};
  if (cudaGetDevice(&cur) != cudaSuccess || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return set_last_error(UF_ECUDA, "cannot query the output buffer's memory type");
  }
  char msg[200];
  if (at.type == cudaMemoryTypeDevice && at.device != cur) {
    snprintf(msg, sizeof msg, "%s is memory of device %d but device %d is current", what, at.device, cur);
    return set_last_error(UF_EINVAL, msg);
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) {
    snprintf(msg, sizeof msg, "%s is not device memory", what);
    return set_last_error(UF_EINVAL, msg);
  }
  return UF_OK;
}

namespace {
thread_local int tl_launch_priority = 0;
}
int launch_priority() { return tl_launch_priority; }
void set_launch_priority(int p) { tl_launch_priority = p; }
}  // namespace ufg
