// uf_internal.h -- declarations shared by the host runtime and the kernels.
//
// Layouts (device memory):
//   counts  [n_slots][n]    FP64 count sums of live nodes (one slot per node
//                           from its computation until its block ends and
//                           its parent has been computed)
//   X       [rows][pitch]   one embedding row per branch of the current
//                           block; x[j] = f(counts[j mod n]) for every
//                           j < pitch, i.e. the row is extended with its own
//                           head so that the partner index k + d needs no
//                           modulo (the paper's unmodded emb[k + stripe + 1],
//                           Sec. 2 Fig. 1 and Sec. 3 Figs. 2-3)
//   M       [s_hi-s_lo+1][n] int64 fixed-point stripe accumulator, cell
//                           (s - s_lo) * n + k for the pair (k, (k + s + 1) mod n)
//                           (the unified buffer of Sec. 2, Fig. 1)
//   Dg      [n]             int64 fixed-point diagonal accumulator (partner offset 0)
// FP64 calls give every fixed-point accumulator a second word (uf_device.cuh,
// Fx2) in an array of the same shape at a stated element offset.
#pragma once
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/unifrac_gb300.h"

namespace ufg {

// what an embedding row holds
enum EmbKind : int {
  EMB_SCALED = 0,    // l_v * p(v): weighted methods
  EMB_PRESENCE = 1,  // l_v * [count > 0]: unweighted
  EMB_PROP = 2,      // p(v): generalized (the length is applied in the kernel)
  EMB_VAW = 3,       // variance-adjusted weighted: three planes per row, each `pitch`
                     // elements, l_v * p(v), the count c(v) below v and T - c(v)
};

// which quantity the accumulator holds
enum AccKind : int {
  ACC_MIN = 0,   // sum_e min(x_e[k], x_e[k + d])  (+ diagonal row d = 0)
  ACC_GEN = 1,   // generalized: den = sum l s^a and, FP32, Q = sum l min(u, v) s^(a-1)
                 // (num = den - 2Q) or, FP64, N = sum l |u - v| s^(a-1) (num = N)
  ACC_VAW = 3,   // variance-adjusted weighted: den = sum l w (u + v), N = sum l w |u - v|,
                 // w = 1 / sqrt((c_k + c_j)(r_k + r_j)) where both factors are > 0
};

// ---- batches ----
// One table of a batch as the stripe kernels see it.  The samples of all
// tables sit side by side on one combined sample axis (count slots, totals,
// the diagonal), and every embedding row holds one padded segment per table.
struct TabDesc {
  int n;              // samples
  int off;            // first column on the combined sample axis
  int s_lo, s_hi;     // stored stripes [s_lo, s_hi]
  int m_lo, m_hi;     // stripe tiles covering them
  int n_ktiles;       // sample tiles
  int tile0;          // first tile of this table in the batch's tile numbering
  int kband;          // unit order: bands of kband sample tiles, every stripe tile of a band
                      // before the next band (sample tile fastest within it), so that the
                      // rows' columns a band reads stay in L2
  int64_t x_col;      // first column of its segment in an embedding row
  int64_t m_off;      // first cell of its stripe accumulator
};

// ---- stripe accumulate (uf_stripe.cu) ----
// A stripe s whose bit (s mod 8) is set in the call's abs mask holds
// A = sum |x_k - x_j| (abs form) instead of M = sum min(x_k, x_j) (min form).
// FP32: stripes 1, 3, 5, 7 of every 8, so that the ALU and FMA pipes share
// the load (see uf_stripe.cu).  FP64: every stripe, so that no numerator is
// formed by cancellation (D_k + D_j - 2M) and its error stays relative to
// the distance itself, however close the two samples are.
constexpr unsigned FP32_ABS_ROW_MASK = 0xAAu;
constexpr unsigned FP64_ABS_ROW_MASK = 0xFFu;
__host__ __device__ constexpr unsigned abs_row_mask(bool fp32) { return fp32 ? FP32_ABS_ROW_MASK : FP64_ABS_ROW_MASK; }
__host__ __device__ constexpr bool abs_row(unsigned mask, int64_t s) { return (mask >> (s & 7)) & 1u; }

struct StripeArgs {
  const void *X;        // [rows][pitch] float or double, one segment per table
  const double *len;    // per-row branch length (generalized only), [rows]
  int rows;             // branches in this launch
  int64_t pitch;        // elements per row (all segments)
  int chunk;            // rows per work unit: a multiple of 64, >= 1,024
  const TabDesc *tabs;  // device array of n_tabs tables
  int n_tabs;
  int n_tiles;          // tiles of all tables (per row chunk)
  int n_cols;           // combined samples (diagonal length)
  unsigned long long *M;   // fixed point: M / A (ACC_MIN) or den (ACC_GEN), per table at m_off
  unsigned long long *M2;  // ACC_GEN: Q = sum l min(u, v) s^(a-1) (FP32) or
                           // N = sum l |u - v| s^(a-1) (FP64); else null
  unsigned long long *Dg;  // [n_cols] fixed-point diagonal (ACC_MIN, launch_diag), else null
  double alpha;         // generalized exponent
  double scale;         // 2^F: fixed-point scale of every accumulator
  int *counter;         // one int of device memory: the work-unit counter (reset per launch)
  // FP64 kernels: the second (low) word of every fixed-point accumulator sits
  // this many elements after its first word (M and M2 cells; Dg); the FP32
  // kernels keep one word
  int64_t m_lo_off, d_lo_off;
  // FP32 min kernel: 0xFF runs every stripe in the abs form (methods whose
  // numerator must not come from a difference of sums); anything else the
  // default FP32_ABS_ROW_MASK
  unsigned abs_mask;
  int shape;            // tile shape (stripe_tile_shape); the descriptors must match it
};
// stripes and samples per CTA tile of the accumulate kernel; `shape` picks
// one of stripe_shapes() tile shapes (0: the default)
void stripe_tile_shape(int acc, bool fp32, int *tile_s, int *tile_k, int shape = 0);
// tile shapes the accumulate kernel of (acc, precision, abs mask) offers
int stripe_shapes(int acc, bool fp32, unsigned abs_mask);
// default rows per work unit
int stripe_chunk_rows();
cudaError_t launch_stripe_acc(int acc, bool fp32, const StripeArgs &a, cudaStream_t st);
// D[k] += sum of the launch's rows at column k (ACC_MIN only), with the
// stripe kernel's operation order; scratch holds diag_scratch_bytes() (valid
// for every chunk size the StripeArgs may carry)
size_t diag_scratch_bytes(bool fp32, int rows, int n_cols);
cudaError_t launch_diag(bool fp32, const StripeArgs &a, void *scratch, cudaStream_t st);

}  // namespace ufg

// ---- host views of tree / table handles (uf_host.cpp) ----
struct uf_tree;
struct uf_table;
namespace ufg {
struct TreeView {
  int64_t n_nodes, n_tips;
  const double *length;
  const int32_t *tip_of_node, *child_ptr, *child_idx;
};
struct TableView {
  int64_t n, n_features, nnz;
  const double *total;
  const float *inv_total_f;
  const int64_t *col_ptr;
  const int32_t *col_row;
  const double *col_val;
};
bool tree_host_view(const ::uf_tree *t, TreeView *v);
bool table_host_view(const ::uf_table *t, TableView *v);
}  // namespace ufg

namespace ufg {
// Fixed-point scale 2^F for the accumulators of an embedding kind (uf_host.cpp).
double accum_scale(const ::uf_tree *tree, const ::uf_table *table, int kind);
// Set the calling thread's uf_last_error() text and return st (uf_host.cpp).
uf_status set_last_error(uf_status st, const char *msg);
// UF_OK when p is device (or managed) memory usable on the current device;
// else UF_EINVAL (memory of another device, host memory) or UF_ECUDA, with
// the thread's error text set (uf_host.cpp).
uf_status check_device_output(const void *p, const char *what);

// Scheduling priority that the calling thread's launches through launch_k
// carry (uf_host.cpp; 0: the stream's own).  A call raises it for the
// launches of its main path while its sparse-row scatter runs on a side
// stream at the default priority, so that the scatter takes only the SM
// slots the main path leaves free.
int launch_priority();
void set_launch_priority(int p);

// kernel<<<grid, block, smem, st>>>(args...) with the thread's launch
// priority as a launch attribute (kept when the launch is captured into a
// graph).
template <typename... KP, typename... A>
cudaError_t launch_k(void (*kernel)(KP...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, A &&...args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  const int p = launch_priority();
  if (p != 0) {
    at[0].id = cudaLaunchAttributePriority;
    at[0].val.priority = p;
    cfg.attrs = at;
    cfg.numAttrs = 1;
  }
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<A &&>(args)...);
}
}  // namespace ufg
