// uf_split.cpp -- which branches of a call run through the dense stripe
// kernels and which are scattered pair by pair (uf_sparse.cu), by a cost
// model of the two paths on GB300; plus the count-row lists the split
// needs and a per-tree cache of splits.
#include "uf_runtime.h"

namespace ufg {
namespace rt {

double sparse_regions(size_t n_tables, int acc, double acc_bytes) {
  const double budget = (double)g_region_bytes.load();
  if (n_tables != 1 || acc_bytes <= budget) return 1.0;
  return std::ceil(acc_bytes / budget);
}

namespace {

// Per branch v the count entries of table t under v are the CSC run of v's
// tips, ub_t(v) = col_ptr_t[tip_hi] - col_ptr_t[tip_lo] (an upper bound on the
// nonzero samples, exact when no two tips share a sample).  Mode 1 scatters
// v when the modelled time of its pairs is below that of a dense pass over
// its stripe cells; the rates are GB300 measurements of the two kernels and
// of global 64-bit atomics (L2-resident accumulators or not).  Mode 2
// scatters every branch that fits; mode 0 none.  The choice depends on the
// tree and the tables only, not on the stripe range, so that a range run
// gives bitwise the stripes of the full run.
RowSplit split_rows(const uf_tree *tree, const BatchJob &J, const Plan *P, int acc, bool fp32) {
  RowSplit R;
  // the variance-adjusted method has no pair-scatter form: every branch dense
  const int mode = acc == ACC_VAW ? 0 : (int)g_sparse.load();
  const int64_t nb = tree->n_nodes - 1;
  const size_t nt = J.tabs.size();
  const int classes[5] = {128, 512, 2048, SPARSE_MAX_ENTRIES, SPARSE_LIST_MAX_ENTRIES};
  R.cap.assign(classes, classes + 5);
  R.sparse.resize(5);
  std::vector<char> is_sparse(std::max<int64_t>(nb, 1), 0);
  if (mode != 0) {
    // accumulator words per cell: FP64 terms are two-word fixed point
    // (uf_device.cuh) except on the tensor path, whose sparse rows keep one
    const int n_acc = (acc == ACC_GEN ? 2 : 1) * (fp32 || acc == SPLIT_GRAM ? 1 : 2);
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
    // the scatter runs table by table (its grid's y is the table), so each
    // table's atomics hit L2 when that table's accumulators fit there
    std::vector<double> pair_cost(nt), entry_cost(nt);
    const double n_regions = regions ? sparse_regions(nt, acc, cells * 8.0 * n_acc) : 1.0;
    double dense_rate;  // cell updates per second of the dense kernel
    if (acc == SPLIT_GRAM) dense_rate = 2.5e14;
    else dense_rate = fp32 ? (acc == ACC_GEN ? 4e12 : 1.3e13) : (acc == ACC_GEN ? 5e10 : 2e11);
    const double visit_rate = fp32 ? 2e12 : (acc == ACC_GEN ? 3e10 : 1e12);
    const double job_cost = 5e-10;
    // region lists are fused (a listed branch carries its sparse children,
    // and for the min form with option sparse_fuse 6 its grandchildren,
    // uf_run.cpp): on the 113k-sample table about 0.57 (0.43) of the pairs
    // and 0.54 (0.39) of the list entries remain, so a scattered branch costs
    // about that share of its own pairs and visits.  The tensor path's
    // scatter runs beside its gram and ends after it already: its split keeps
    // the unfused costs.
    const int64_t fm = acc == ACC_GEN ? std::min<int64_t>(g_sparse_fuse.load(), 2) : g_sparse_fuse.load();
    const double fuse = regions && acc != SPLIT_GRAM && fm > 0 ? (fm == 6 ? 0.45 : 0.6) : 1.0;
    for (size_t t = 0; t < nt; t++) {
      const double n = (double)J.tabs[t].table->n;
      const double atom_rate = std::floor(n / 2.0) * n * 8.0 * n_acc <= 64e6 || regions ? 2.3e11 : 2.5e10;
      pair_cost[t] = (1.0 / visit_rate + n_acc / atom_rate) * fuse;
      entry_cost[t] = 4.0 / atom_rate;
    }
    // a dense row also costs its count row and embedding (or planes) in HBM
    const double dense_t = cells / dense_rate + cols * 36.0 / 6e12;
    // node ranges in parallel; each class list is the ranges' lists in order,
    // so the result equals a sequential pass (pair counts are integers < 2^53:
    // their double sums are exact in any order)
    struct Part {
      std::vector<int32_t> cls[5];
      int64_t n_sparse = 0;
      double pairs = 0.0;
    };
    const int T = (int)std::max<int64_t>(1, std::min<int64_t>(host_threads(), nb / 16384));
    std::vector<Part> part(T);
    parallel_for(T, [&](int c) {
      Part &pt = part[c];
      const int64_t v0 = nb * c / T, v1 = nb * (c + 1) / T;
      for (int64_t v = v0; v < v1; v++) {
        const int32_t lo = tree->tip_lo[v], hi = tree->tip_hi[v];
        if (lo < 0) continue;
        if (tree->length[v] == 0.0) {
          // a zero-length branch adds exactly 0 to every accumulator: skipped
          // (its count row is still built if a dense parent needs it)
          is_sparse[v] = 1;
          pt.n_sparse++;
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
          cost += job_cost + pr * pair_cost[t] + (double)ub * entry_cost[t];
          // one visit per region: a CTA, and each entry's cursors walked to the
          // region (about 7e-12 s per entry and region measured on GB300 with a
          // 113,000-sample table; pairs at 4.3e-12 s)
          if (regions) cost += n_regions * (job_cost + (double)ub * 1e-11 * fuse);
        }
        if (mx > max_entries) continue;
        if (mode == 2 || cost < dense_t) {
          is_sparse[v] = 1;
          int k = 0;
          while (classes[k] < mx) k++;
          pt.cls[k].push_back((int32_t)v);
          pt.n_sparse++;
          pt.pairs += pairs;
        }
      }
    });
    for (int k = 0; k < 5; k++)
      for (const Part &pt : part) R.sparse[k].insert(R.sparse[k].end(), pt.cls[k].begin(), pt.cls[k].end());
    for (const Part &pt : part) {
      R.n_sparse += pt.n_sparse;
      R.pairs += pt.pairs;
    }
  }
  const int64_t root = tree->n_nodes - 1;
  auto parent_dense = [&](int64_t v) {
    const int64_t p = tree->parent[v];
    return p != root && !is_sparse[p];
  };
  // per list position: bit 0 = built from CSC columns (tips, and sparse
  // branches under a dense parent), bit 1 = a dense internal node; flagged in
  // parallel, then gathered in list order
  std::vector<uint8_t> flag(P->lists.size(), 0);
  {
    const int64_t np = (int64_t)P->lists.size();
    const int T = (int)std::max<int64_t>(1, std::min<int64_t>(host_threads(), np / 16384));
    parallel_for(T, [&](int c) {
      const int64_t p0 = np * c / T, p1 = np * (c + 1) / T;
      size_t b = 0;
      for (int64_t q = p0; q < p1; q++) {
        // block of position q: blocks cover consecutive ranges of the lists
        while (b + 1 < P->launches.size() && q >= P->launches[b + 1][0].first) b++;
        const auto &l0 = P->launches[b][0];
        const int32_t v = P->lists[q];
        const bool tip = q < l0.first + l0.second;
        flag[q] = (uint8_t)((is_sparse[v] ? parent_dense(v) : tip) | ((!tip && !is_sparse[v]) << 1));
      }
    });
  }
  for (size_t b = 0; b < P->b0.size(); b++) {
    const auto &ls = P->launches[b];
    std::vector<std::pair<int64_t, int>> lb;
    const int64_t q0 = ls[0].first, q1 = ls.back().first + ls.back().second;
    const int64_t at0 = (int64_t)R.cnt_lists.size();
    for (int64_t q = q0; q < q1; q++)
      if (flag[q] & 1) R.cnt_lists.push_back(P->lists[q]);
    lb.emplace_back(at0, (int)((int64_t)R.cnt_lists.size() - at0));
    for (size_t l = 1; l < ls.size(); l++) {
      const int64_t at = (int64_t)R.cnt_lists.size();
      for (int64_t q = ls[l].first; q < ls[l].first + ls[l].second; q++)
        if (flag[q] & 2) R.cnt_lists.push_back(P->lists[q]);
      if ((int64_t)R.cnt_lists.size() > at) lb.emplace_back(at, (int)((int64_t)R.cnt_lists.size() - at));
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

}  // namespace

// The split of a call, cached on the tree by its tables and kind (tables are
// immutable and their ids are never reused).
std::shared_ptr<const RowSplit> get_split(uf_tree *tree, const BatchJob &J, const Plan *P, int acc, bool fp32) {
  SplitKey key;
  for (const TableJob &t : J.tabs) std::get<0>(key).push_back(t.table->id);
  std::get<1>(key) = acc;
  std::get<2>(key) = fp32 ? 1 : 0;
  std::get<3>(key) = (int)(g_sparse.load() * 16 + g_sparse_fuse.load());
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

}  // namespace rt
}  // namespace ufg
