// uf_gram.h -- unweighted UniFrac on the tensor cores (uf_gram.cu).
#pragma once
#include "uf_internal.h"

namespace ufg {

// ---- unweighted on tensor cores (uf_gram.cu) ----
// One table of a batch: its samples occupy rows [row_base, row_base + n_pad)
// of every presence plane; its gram matrix starts at gt_off.
struct GramTab {
  int n, n_pad;         // samples, padded to the 256-sample tile
  int row_base;         // first plane row
  int off;              // first column on the combined sample axis
  int64_t gt_off;       // first cell of its gram matrix (n_pad x n_pad)
};
struct GramArgs {
  int k_len;            // branches of this block, rounded up to 64
  int kc;               // branches per work unit (multiple of 64)
  int n_tiles;          // tiles of all tables
  int n_units;          // set by launch_gram
  int npad_tot;         // plane rows (sum of n_pad)
  const int32_t *tile_tab, *tile_bi, *tile_bj;
  const GramTab *tabs;
  unsigned long long *Gt;  // fixed point; cell (i, j), i <= j, of table t at gt_off + j * n_pad + i
  double scale;         // 2^F
  int *err;             // set to 1 when a bounded wait gave up
  int wait_test;        // 1: the MMA issuer first waits on a barrier nothing signals, so its
                        // bounded wait runs out (tests the abort path; option "tensor_wait_test")
};
struct GramFinalArgs {
  int n, n_pad;
  int64_t s0, s1;
  int full;
  const unsigned long long *Gt;  // this table's gram matrix
  void *out;
  int out_fp32;
  const int *err;                // the gram kernel's abort flag: when set, every output is NaN
};
int gram_pad(int n);                      // n rounded up to the tile
int64_t gram_kpad(int rows);              // branches rounded up to the stage
// upper-triangle tiles of one table: (bi, bj) pairs appended to bi / bj
void gram_tiles(int n_pad, std::vector<int32_t> *bi, std::vector<int32_t> *bj);
// planes of branches nodes[0 .. rows) (b0 .. b0 + rows - 1 when nodes is null)
// from their presence flags
cudaError_t launch_gram_prep(int64_t b0, int rows, const int32_t *slot_of_node, const uint8_t *flags,
                             int64_t ld, const double *length, const GramTab *tabs, int n_tabs,
                             int npad_tot, int64_t K_pad, void *Pl, cudaStream_t st,
                             const int32_t *nodes = nullptr);
cudaError_t launch_gram(const GramArgs &a, void *Pl, int64_t K_pad, cudaStream_t st);
cudaError_t launch_finalize_gram(const GramFinalArgs &a, cudaStream_t st);

}  // namespace ufg
