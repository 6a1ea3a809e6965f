// uf_gram.h -- unweighted UniFrac on the tensor cores (uf_gram.cu).
#pragma once
#include "uf_internal.h"

namespace ufg {

// ---- unweighted on tensor cores (uf_gram.cu) ----
// Tiles of a table's gram matrix: GRAM_TM samples i x GRAM_TN samples j.
constexpr int GRAM_TM = 128;
constexpr int GRAM_TN = 256;
constexpr int64_t GRAM_TILE_CELLS = (int64_t)GRAM_TM * GRAM_TN;
// One table of a batch: its samples occupy rows [row_base, row_base + n_pad)
// of every presence plane; its tile map (row-major over (i / GRAM_TM,
// j / GRAM_TN), n_pad / GRAM_TM rows of n_pad / GRAM_TN entries) starts at
// map_off and gives the stored tile of each block of cells, or -1.
struct GramTab {
  int n, n_pad;         // samples, padded to the 256-sample tile
  int row_base;         // first plane row
  int off;              // first column on the combined sample axis
  int64_t map_off;      // first entry of its tile map
};
struct GramArgs {
  int k_len;            // branches of this block, rounded up to 64
  int kc;               // branches per work unit (multiple of 64)
  int n_tiles;          // tiles of all tables
  int n_units;          // set by launch_gram
  int npad_tot;         // plane rows (sum of n_pad)
  const int32_t *tile_tab, *tile_bi, *tile_bj;  // stored tiles: table and block coordinates
  const GramTab *tabs;
  // fixed point, compact tiles: cell (i, j), i <= j, of stored tile t with
  // block coordinates (bi, bj) at t * GRAM_TILE_CELLS + (j - bj GRAM_TN) GRAM_TM + (i - bi GRAM_TM)
  unsigned long long *Gt;
  double scale;         // 2^F
  int *err;             // set to 1 when a bounded wait gave up
  int wait_test;        // 1: the MMA issuer first waits on a barrier nothing signals, so its
                        // bounded wait runs out (tests the abort path; option "tensor_wait_test")
};
struct GramFinalArgs {
  int n, n_pad;
  int64_t s0, s1;
  int full;
  const unsigned long long *Gt;  // the call's compact tiles
  const int32_t *tile_map;       // this table's tile map
  // sparse rows (uf_sparse.cu, min form on presence rows), or null: pair terms
  // in the stripe layout [(s1 - s0)][n] and per-sample terms [n]
  const unsigned long long *Msp, *Dsp;
  void *out;
  int out_fp32;
  const int *err;                // the gram kernel's abort flag: when set, every output is NaN
  unsigned long long *clamps;    // or null: counts numerators that rounded below 0
  int unnormalized;              // 1: the distance is the numerator alone, num * inv_scale
  double inv_scale;              // 2^-F
};
int gram_pad(int n);                      // n rounded up to the tile
int64_t gram_kpad(int rows);              // branches rounded up to the stage
// Tiles of one n-sample table that hold a pair of the stripes [s0, s1) or a
// diagonal cell, in row-major block order: (bi, bj) appended to bi / bj.
// Stripe s holds the pairs at distance d = j - i of s + 1 and n - s - 1.
void gram_tiles(int n, int64_t s0, int64_t s1, std::vector<int32_t> *bi, std::vector<int32_t> *bj);
// planes of branches nodes[0 .. rows) (b0 .. b0 + rows - 1 when nodes is null)
// from their presence flags
cudaError_t launch_gram_prep(int64_t b0, int rows, const int32_t *slot_of_node, const uint8_t *flags,
                             int64_t ld, const double *length, const GramTab *tabs, int n_tabs,
                             int npad_tot, int64_t K_pad, void *Pl, cudaStream_t st,
                             const int32_t *nodes = nullptr);
cudaError_t launch_gram(const GramArgs &a, void *Pl, int64_t K_pad, cudaStream_t st);
cudaError_t launch_finalize_gram(const GramFinalArgs &a, cudaStream_t st);

}  // namespace ufg
