// uf_embed.cu -- per-branch embeddings (emb of Figs. 1-3; in the paper a CPU
// producer prepares them buffer by buffer, Sec. 3), built level by level on the GPU.
//
// A node's count row is the sum of its children's count rows (postorder:
// children first); a tip's row is its column of the count table.  The
// embedding row of a branch is then f(count[k] / total[k]) for every sample
// k, written over a padded width so that the stripe kernel can read the
// partner column k + d without a modulo.
#include "uf_device.cuh"
#include "uf_embed.h"

namespace ufg {

// One CTA per tip: zero the table's part of the tip's count slot, then
// scatter its CSC column (counts points at the table's first column).
__global__ void k_tip_counts(const int32_t *__restrict__ tip_nodes,
                             const int32_t *__restrict__ slot_of_node,
                             const int32_t *__restrict__ tip_of_node,
                             const int64_t *__restrict__ col_ptr,
                             const int32_t *__restrict__ col_row,
                             const double *__restrict__ col_val, double *__restrict__ counts,
                             int64_t ld, int n) {
  const int v = tip_nodes[blockIdx.x];
  double *row = counts + (int64_t)slot_of_node[v] * ld;
  for (int k = threadIdx.x; k < n; k += blockDim.x) row[k] = 0.0;
  __syncthreads();
  const int f = tip_of_node[v];
  const int64_t q1 = col_ptr[f + 1];
  for (int64_t q = col_ptr[f] + threadIdx.x; q < q1; q += blockDim.x) row[col_row[q]] = col_val[q];
}

// One CTA per node of a list: zero the table's part of the node's count
// slot, then add the CSC columns of its tips [tip_lo, tip_hi) one after the
// other (within one tip's column the samples are distinct, so its entries
// scatter without conflicts).  Serves tips and the nodes whose own subtree
// is not walked level by level (a branch scattered by the sparse-row path
// whose parent runs through the dense kernels).  With C = uint8_t the slot
// holds presence flags instead (1 where the count is nonzero).
template <typename C>
__global__ void k_slice_counts(const int32_t *__restrict__ nodes, const int32_t *__restrict__ tip_lo,
                               const int32_t *__restrict__ tip_hi, const int32_t *__restrict__ slot_of_node,
                               const int64_t *__restrict__ col_ptr, const int32_t *__restrict__ col_row,
                               const double *__restrict__ col_val, C *__restrict__ counts, int64_t ld, int n) {
  const int v = nodes[blockIdx.x];
  C *row = counts + (int64_t)slot_of_node[v] * ld;
  for (int k = threadIdx.x; k < n; k += blockDim.x) row[k] = C(0);
  __syncthreads();
  const int f1 = tip_hi[v];
  for (int f = tip_lo[v]; f < f1; f++) {
    const int64_t q1 = col_ptr[f + 1];
    for (int64_t q = col_ptr[f] + threadIdx.x; q < q1; q += blockDim.x) {
      if constexpr (sizeof(C) == 1) row[col_row[q]] = C(1);
      else row[col_row[q]] += col_val[q];
    }
    __syncthreads();
  }
}

// count[v][k] = sum of the children's count[c][k], children in index order
// (the order the postorder walk adds them in), over all ld columns; for
// presence flags (C = uint8_t) the OR of the children's flags.
// grid.x = nodes, grid.y = sample chunks.
template <typename C>
__global__ void k_node_counts(const int32_t *__restrict__ nodes,
                              const int32_t *__restrict__ child_ptr,
                              const int32_t *__restrict__ child_idx,
                              const int32_t *__restrict__ slot_of_node,
                              C *__restrict__ counts, int64_t ld) {
  const int v = nodes[blockIdx.x];
  const int64_t k = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
  if (k >= ld) return;
  C s = C(0);
  for (int c = child_ptr[v]; c < child_ptr[v + 1]; c++) {
    if constexpr (sizeof(C) == 1) s |= counts[(int64_t)slot_of_node[child_idx[c]] * ld + k];
    else s += counts[(int64_t)slot_of_node[child_idx[c]] * ld + k];
  }
  counts[(int64_t)slot_of_node[v] * ld + k] = s;
}

// The same with 16 bytes per thread (2 counts or 16 flags) for rows whose
// stride is a multiple of 16 bytes: each element is still the sum (OR) of
// the children's elements in index order, so the rows are bitwise those of
// k_node_counts.  Columns [0, n_used) are written; the ragged end of a row
// goes element by element.  grid.x = nodes, grid.y = column chunks.
template <typename C>
__global__ void k_node_counts_v16(const int32_t *__restrict__ nodes,
                                  const int32_t *__restrict__ child_ptr,
                                  const int32_t *__restrict__ child_idx,
                                  const int32_t *__restrict__ slot_of_node,
                                  C *__restrict__ counts, int64_t ld, int64_t n_used) {
  constexpr int V = 16 / (int)sizeof(C);
  const int v = nodes[blockIdx.x];
  const int64_t e0 = ((int64_t)blockIdx.y * blockDim.x + threadIdx.x) * V;
  if (e0 >= n_used) return;
  const int c0 = child_ptr[v], c1 = child_ptr[v + 1];
  C *dst = counts + (int64_t)slot_of_node[v] * ld + e0;
  if (e0 + V <= n_used) {
    if constexpr (sizeof(C) == 1) {
      uint4 s = make_uint4(0u, 0u, 0u, 0u);
      for (int c = c0; c < c1; c++) {
        const uint4 x = *reinterpret_cast<const uint4 *>(counts + (int64_t)slot_of_node[child_idx[c]] * ld + e0);
        s.x |= x.x;
        s.y |= x.y;
        s.z |= x.z;
        s.w |= x.w;
      }
      *reinterpret_cast<uint4 *>(dst) = s;
    } else {
      double2 s = make_double2(0.0, 0.0);
      for (int c = c0; c < c1; c++) {
        const double2 x =
            *reinterpret_cast<const double2 *>(counts + (int64_t)slot_of_node[child_idx[c]] * ld + e0);
        s.x += x.x;
        s.y += x.y;
      }
      *reinterpret_cast<double2 *>(dst) = s;
    }
    return;
  }
  for (int64_t e = e0; e < n_used; e++) {
    C s = C(0);
    for (int c = c0; c < c1; c++) {
      if constexpr (sizeof(C) == 1) s |= counts[(int64_t)slot_of_node[child_idx[c]] * ld + e];
      else s += counts[(int64_t)slot_of_node[child_idx[c]] * ld + e];
    }
    counts[(int64_t)slot_of_node[v] * ld + e] = s;
  }
}

// Node rows of one level: the 16-byte kernel when the stride and base allow
// it, else one element per thread.
template <typename C>
cudaError_t launch_node_rows(const int32_t *nodes, int n_list, const int32_t *child_ptr, const int32_t *child_idx,
                             const int32_t *slot_of_node, C *counts, int64_t ld, int64_t n_used,
                             cudaStream_t st) {
  if (n_list <= 0 || n_used <= 0) return cudaSuccess;
  if ((ld * (int64_t)sizeof(C)) % 16 == 0 && reinterpret_cast<uintptr_t>(counts) % 16 == 0) {
    constexpr int V = 16 / (int)sizeof(C);
    const int64_t chunks = (n_used + V - 1) / V;
    const int bt = chunks >= 256 ? 256 : 128;
    return launch_k(k_node_counts_v16<C>, dim3(n_list, (unsigned)((chunks + bt - 1) / bt)), dim3(bt), 0, st,
                    nodes, child_ptr, child_idx, slot_of_node, counts, ld, n_used);
  }
  return launch_k(k_node_counts<C>, dim3(n_list, (unsigned)((ld + 255) / 256)), dim3(256), 0, st, nodes,
                  child_ptr, child_idx, slot_of_node, counts, ld);
}

// Table whose row segment holds column j (segments are contiguous, in order).
__device__ __forceinline__ int segment_of(const TabDesc *tabs, int n_tabs, int64_t j) {
  int lo = 0, hi = n_tabs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tabs[mid].x_col <= j) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// One CTA per branch row r (node nodes[r], or b0 + r without a list): in
// table t's segment, X[r][x_col + j] = f(count[off + (j mod n)]) for j < the
// segment's width.
template <typename T, int KIND>
__global__ void k_emb_rows(int64_t b0, const int32_t *__restrict__ nodes,
                           const int32_t *__restrict__ slot_of_node,
                           const double *__restrict__ counts, int64_t ld,
                           const double *__restrict__ length, const double *__restrict__ total,
                           const float *__restrict__ inv_total_f, T *__restrict__ X, int64_t pitch,
                           const TabDesc *__restrict__ tabs, int n_tabs) {
  const int64_t v = nodes ? (int64_t)nodes[blockIdx.x] : b0 + blockIdx.x;
  const double *c = counts + (int64_t)slot_of_node[v] * ld;
  const double l = length[v];
  T *x = X + (int64_t)blockIdx.x * pitch;
  for (int64_t j = threadIdx.x; j < pitch; j += blockDim.x) {
    const TabDesc &tb = tabs[n_tabs == 1 ? 0 : segment_of(tabs, n_tabs, j)];
    int64_t k = j - tb.x_col;
    while (k >= tb.n) k -= tb.n;
    k += tb.off;
    x[j] = emb_value<T, KIND>(c[k], l, total[k], inv_total_f[k]);
  }
}

// Variance-adjusted rows: three planes per row r, each `pitch` elements:
// l p = l c / T (the branch length folded in, as it multiplies both sums),
// the count c below the branch and T - c, with the same wrap-padded columns
// as k_emb_rows.
template <typename T>
__global__ void k_emb_rows_vaw(const int32_t *__restrict__ nodes, const int32_t *__restrict__ slot_of_node,
                               const double *__restrict__ counts, int64_t ld, const double *__restrict__ length,
                               const double *__restrict__ total, const float *__restrict__ inv_total_f,
                               T *__restrict__ X, int64_t pitch, const TabDesc *__restrict__ tabs, int n_tabs) {
  const int64_t v = nodes[blockIdx.x];
  const double *c = counts + (int64_t)slot_of_node[v] * ld;
  const double l = length[v];
  T *x = X + (int64_t)blockIdx.x * 3 * pitch;
  for (int64_t j = threadIdx.x; j < pitch; j += blockDim.x) {
    const TabDesc &tb = tabs[n_tabs == 1 ? 0 : segment_of(tabs, n_tabs, j)];
    int64_t k = j - tb.x_col;
    while (k >= tb.n) k -= tb.n;
    k += tb.off;
    const double ck = c[k], tk = total[k];
    // FP32 rows use the FP32 reciprocal of the total (an FP64 division per
    // value costs more than the whole FP32 kernel saves)
    if constexpr (sizeof(T) == 4) x[j] = (float)l * ((float)ck * inv_total_f[k]);
    else x[j] = l * (ck / tk);
    x[pitch + j] = (T)ck;
    x[2 * pitch + j] = (T)(tk - ck);
  }
}

cudaError_t launch_tip_counts(const int32_t *tip_nodes, int n_list, const int32_t *slot_of_node,
                              const int32_t *tip_of_node, const int64_t *col_ptr,
                              const int32_t *col_row, const double *col_val, double *counts,
                              int64_t ld, int n, cudaStream_t st) {
  if (n_list <= 0) return cudaSuccess;
  k_tip_counts<<<n_list, 256, 0, st>>>(tip_nodes, slot_of_node, tip_of_node, col_ptr, col_row,
                                       col_val, counts, ld, n);
  return cudaGetLastError();
}

cudaError_t launch_slice_counts(const int32_t *nodes, int n_list, const int32_t *tip_lo, const int32_t *tip_hi,
                                const int32_t *slot_of_node, const int64_t *col_ptr, const int32_t *col_row,
                                const double *col_val, double *counts, int64_t ld, int n, cudaStream_t st) {
  if (n_list <= 0) return cudaSuccess;
  return launch_k(k_slice_counts<double>, dim3(n_list), dim3(256), 0, st, nodes, tip_lo, tip_hi, slot_of_node, col_ptr,
                  col_row, col_val, counts, ld, n);
}

cudaError_t launch_slice_presence(const int32_t *nodes, int n_list, const int32_t *tip_lo, const int32_t *tip_hi,
                                  const int32_t *slot_of_node, const int64_t *col_ptr, const int32_t *col_row,
                                  uint8_t *flags, int64_t ld, int n, cudaStream_t st) {
  if (n_list <= 0) return cudaSuccess;
  return launch_k(k_slice_counts<uint8_t>, dim3(n_list), dim3(256), 0, st, nodes, tip_lo, tip_hi, slot_of_node,
                  col_ptr, col_row, (const double *)nullptr, flags, ld, n);
}

cudaError_t launch_node_counts(const int32_t *nodes, int n_list, const int32_t *child_ptr,
                               const int32_t *child_idx, const int32_t *slot_of_node,
                               double *counts, int64_t ld, cudaStream_t st, int64_t n_used) {
  return launch_node_rows<double>(nodes, n_list, child_ptr, child_idx, slot_of_node, counts, ld,
                                  n_used < 0 ? ld : n_used, st);
}

cudaError_t launch_node_presence(const int32_t *nodes, int n_list, const int32_t *child_ptr,
                                 const int32_t *child_idx, const int32_t *slot_of_node,
                                 uint8_t *flags, int64_t ld, cudaStream_t st, int64_t n_used) {
  return launch_node_rows<uint8_t>(nodes, n_list, child_ptr, child_idx, slot_of_node, flags, ld,
                                   n_used < 0 ? ld : n_used, st);
}

cudaError_t launch_emb_rows(int kind, bool fp32, int64_t b0, int rows,
                            const int32_t *slot_of_node, const double *counts, int64_t ld,
                            const double *length, const double *total, const float *inv_total_f,
                            void *X, int64_t pitch, const TabDesc *tabs, int n_tabs, cudaStream_t st,
                            const int32_t *nodes) {
  if (rows <= 0) return cudaSuccess;
  if (kind == EMB_VAW) {
    if (!nodes) return cudaErrorInvalidValue;
    if (fp32)
      return launch_k(k_emb_rows_vaw<float>, dim3(rows), dim3(256), 0, st, nodes, slot_of_node, counts, ld, length,
                      total, inv_total_f, (float *)X, pitch, tabs, n_tabs);
    return launch_k(k_emb_rows_vaw<double>, dim3(rows), dim3(256), 0, st, nodes, slot_of_node, counts, ld, length,
                    total, inv_total_f, (double *)X, pitch, tabs, n_tabs);
  }
#define UF_EMB(T, K)                                                                                 \
  return launch_k(k_emb_rows<T, K>, dim3(rows), dim3(256), 0, st, b0, nodes, slot_of_node, counts, ld, length, \
                  total, inv_total_f, (T *)X, pitch, tabs, n_tabs)
  if (fp32) {
    if (kind == EMB_SCALED) UF_EMB(float, EMB_SCALED);
    if (kind == EMB_PRESENCE) UF_EMB(float, EMB_PRESENCE);
    UF_EMB(float, EMB_PROP);
  }
  if (kind == EMB_SCALED) UF_EMB(double, EMB_SCALED);
  if (kind == EMB_PRESENCE) UF_EMB(double, EMB_PRESENCE);
  UF_EMB(double, EMB_PROP);
#undef UF_EMB
}

}  // namespace ufg
