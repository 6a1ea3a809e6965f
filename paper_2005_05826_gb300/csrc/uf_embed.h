// uf_embed.h -- count rows and embedding rows (uf_embed.cu).
#pragma once
#include "uf_internal.h"

namespace ufg {

// ---- embed (uf_embed.cu) ----
// Count rows live in slots of `ld` doubles (the combined sample axis).
cudaError_t launch_tip_counts(const int32_t *tip_nodes, int n_list, const int32_t *slot_of_node,
                              const int32_t *tip_of_node, const int64_t *col_ptr,
                              const int32_t *col_row, const double *col_val, double *counts,
                              int64_t ld, int n, cudaStream_t st);
// Count rows of listed nodes straight from the CSC columns of their tips
// (tip numbers [tip_lo[v], tip_hi[v]), in order).
cudaError_t launch_slice_counts(const int32_t *nodes, int n_list, const int32_t *tip_lo, const int32_t *tip_hi,
                                const int32_t *slot_of_node, const int64_t *col_ptr, const int32_t *col_row,
                                const double *col_val, double *counts, int64_t ld, int n, cudaStream_t st);
// Presence flags (uint8_t, 1 where the count is nonzero) instead of counts.
cudaError_t launch_slice_presence(const int32_t *nodes, int n_list, const int32_t *tip_lo, const int32_t *tip_hi,
                                  const int32_t *slot_of_node, const int64_t *col_ptr, const int32_t *col_row,
                                  uint8_t *flags, int64_t ld, int n, cudaStream_t st);
// Rows of one level's nodes from their children's rows, columns [0, n_used)
// of rows with stride ld (n_used < 0: all ld columns).
cudaError_t launch_node_presence(const int32_t *nodes, int n_list, const int32_t *child_ptr,
                                 const int32_t *child_idx, const int32_t *slot_of_node,
                                 uint8_t *flags, int64_t ld, cudaStream_t st, int64_t n_used = -1);
cudaError_t launch_node_counts(const int32_t *nodes, int n_list, const int32_t *child_ptr,
                               const int32_t *child_idx, const int32_t *slot_of_node,
                               double *counts, int64_t ld, cudaStream_t st, int64_t n_used = -1);
// Embedding rows of branches nodes[0 .. rows) (b0 .. b0 + rows - 1 when
// nodes is null) for every table segment; EMB_VAW rows hold three planes of
// `pitch` elements each, l p, c and T - c (a node list is required).
cudaError_t launch_emb_rows(int kind, bool fp32, int64_t b0, int rows,
                            const int32_t *slot_of_node, const double *counts, int64_t ld,
                            const double *length, const double *total, const float *inv_total_f,
                            void *X, int64_t pitch, const TabDesc *tabs, int n_tabs, cudaStream_t st,
                            const int32_t *nodes = nullptr);

}  // namespace ufg
