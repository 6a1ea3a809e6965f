// uf_sparse.h -- declarations of the sparse-row pair scatters (uf_sparse.cu)
// shared with the host runtime (kept apart from uf_internal.h so that the
// stripe kernels' sources do not change with them).
#pragma once
#include "uf_internal.h"

namespace ufg {

// ---- sparse rows (uf_sparse.cu) ----
// A branch whose subtree holds few nonzero counts adds to a stripe cell only
// when both samples of the cell are nonzero under it (min(x_k, x_j) = 0
// otherwise; the generalized den is split into per-sample terms plus a pair
// correction).  Such rows skip the dense kernels: one CTA per (row, table)
// gathers the subtree's nonzero samples from the table's CSC columns (the
// subtree's tips are a contiguous range of tip numbers) and scatters the
// both-nonzero pairs into the accumulators.
struct SpTab {
  const int64_t *col_ptr;   // CSC of the table: tip f -> entries [col_ptr[f], col_ptr[f + 1])
  const int32_t *col_row;   // sample of each entry (ascending within a tip)
  const double *col_val;    // count of each entry
  const double *total;      // per-sample count totals
  const float *inv_total_f; // 1 / total in FP32
  int n, off, s_lo, s_hi;   // samples, combined column, stored stripes
  int64_t m_off;            // first accumulator cell
};
struct SparseArgs {
  const int32_t *nodes;     // sparse branch nodes of this launch
  int n_nodes;
  int cap;                  // shared-memory capacity in entries (power of two, >= 128)
  const int32_t *tip_lo, *tip_hi;  // tips of node v: tip numbers [tip_lo[v], tip_hi[v])
  const double *length;     // branch length of every node
  const SpTab *tabs;
  int n_tabs;
  int kind;                 // EmbKind
  unsigned abs_mask;        // min kernels: stripes s with abs_row(abs_mask, s) in the abs form
  int gen_abs;              // generalized: M2 holds N (FP64 kernels) instead of Q (FP32)
  unsigned long long *M, *M2, *Dsp;  // cells (M / den), Q or N (generalized), per-sample diagonal R
  int64_t m_lo_off, d_lo_off;        // FP64: second words of M / M2 and of Dsp, this many elements on
  double alpha, scale;
  // list mode (one table, launch_sparse_lists): row blockIdx.x writes its
  // distinct samples, values and fixed-point terms at lofs[row_base +
  // blockIdx.x] (count in lz) for launch_sparse_region
  int row_base;
  void *le;                 // entries (sample, x or u, fixed-point X or P), ascending
                            // sample; sparse_entry_bytes() each
  int *lk;                  // the entries' samples alone (4 bytes each), for the
                            // region kernel's binary searches
  const int64_t *lofs;      // first entry of each row
  int *lz;                  // entries of each row
  // fused lists (list mode): a listed row also carries the terms of up to
  // `fused` member rows (2 or 6, generalized 2; 0: unfused), sparse branches
  // below it (so their samples are among its own and their pairs among its
  // pairs), and each of its pairs adds the sum of the rows' terms with one
  // atomic per accumulator; members[fused * (row_base + blockIdx.x) + i] is a
  // node or -1
  int fused;
  const int32_t *members;
  // region mode: only pairs whose stripe lies in [r0, r1) (launch_sparse_region)
  int r0, r1;
  unsigned long long *pair_count;  // non-null: the pair updates made are added to these
                                   // SPARSE_PAIR_SLOTS counters (summed by the host)
  int first_region;         // 1: the call's first region (cursors are searched, not read)
  uint16_t *cur;            // two cursors per list entry (indices into its row's list, which
                            // holds at most SPARSE_LIST_MAX_ENTRIES): window 1 at cur[e],
  int64_t cur_stride;       // window 2 at cur[cur_stride + e] (regions in increasing order)
};
// largest subtree entry count a sparse row may have: scattered directly from
// shared memory, or written as a list (one table, keys alone in shared memory)
constexpr int SPARSE_MAX_ENTRIES = 4096;
constexpr int SPARSE_LIST_MAX_ENTRIES = 16384;
static_assert(SPARSE_LIST_MAX_ENTRIES <= 65535, "list cursors are 16-bit");
constexpr int SPARSE_PAIR_SLOTS = 256;
size_t sparse_smem_bytes(bool fp32, int cap);
size_t sparse_entry_bytes(bool fp32, int fused = 0, int acc = ACC_MIN);
cudaError_t launch_sparse_rows(int acc, bool fp32, const SparseArgs &a, cudaStream_t st);
cudaError_t launch_sparse_lists(int acc, bool fp32, const SparseArgs &a, cudaStream_t st);
// Pairs of the listed rows (nodes[0 .. n_nodes), lists from a list-mode
// launch, table tabs[0]) whose stripe lies in [a.r0, a.r1): one CTA per row,
// each thread takes samples a and walks the partners b of the two windows of
// k_b - k_a that map into the region from per-entry cursors (set by binary
// search in the first region); fused lists add each pair's summed terms.
// Run region by region, in increasing stripe order, so that the accumulator
// cells a launch touches stay in L2.
cudaError_t launch_sparse_region(int acc, bool fp32, const SparseArgs &a, cudaStream_t st);

}  // namespace ufg
