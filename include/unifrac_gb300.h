/*
 * unifrac_gb300.h -- C ABI of the GB300 Striped UniFrac engine.
 *
 * Computes all-pairs (or a stripe range of) UniFrac distances between the
 * samples of a count table over a rooted phylogenetic tree, on one GPU.
 *
 * Background.  Sfiligoi, McDonald & Knight, "Porting and optimizing UniFrac
 * for GPUs" (arXiv 2005.05826) ship the method as a C shared library that
 * any language can call (Abstract) and split the n x n
 * distance problem into independent stripes (Abstract, Sec. 1; Fig. 1):
 * stripe s, column k holds the pair (k, (k + s + 1) mod n), and the stripes
 * of a run live in one unified buffer indexed (s - start) * n + k (Sec. 2,
 * Fig. 1).  The paper prints no UniFrac formula; the four methods below are
 * the standard definitions of its refs [1] (unweighted, weighted) and the
 * generalized family, with p_A(v) the share of sample A's counts found
 * below node v and l_v the length of the branch above v:
 *
 *   UF_UNWEIGHTED             sum l_v [p_A>0 xor p_B>0] / sum l_v [p_A>0 or p_B>0]
 *   UF_WEIGHTED_UNNORMALIZED  sum l_v |p_A - p_B|
 *   UF_WEIGHTED_NORMALIZED    sum l_v |p_A - p_B| / sum l_v (p_A + p_B)
 *   UF_GENERALIZED (alpha)    sum l_v s^(alpha-1) |p_A - p_B| / sum l_v s^alpha,
 *                             s = p_A + p_B, terms with s == 0 contribute 0
 *
 * Further members of the Striped UniFrac family (Sec. 1 names the family),
 * with C_A(v) the count of sample A below v, T_A its total,
 * m_v = C_A(v) + C_B(v), m = T_A + T_B:
 *   UF_UNWEIGHTED_UNNORMALIZED    sum l_v [p_A>0 xor p_B>0]
 *   UF_VAW_WEIGHTED_UNNORMALIZED  sum l_v |p_A - p_B| / sqrt(m_v (m - m_v))
 *   UF_VAW_WEIGHTED_NORMALIZED    that sum / sum l_v (p_A + p_B) / sqrt(m_v (m - m_v))
 *   (variance-adjusted weighted UniFrac, Chang, Luan & Sun, BMC
 *   Bioinformatics 12:118, 2011; branches with m_v = 0 or m_v = m add 0;
 *   these run every branch through the dense stripe kernel: option
 *   "sparse" does not apply to them).  UF_UNWEIGHTED_UNNORMALIZED runs on
 *   the CUDA-core kernels in both precisions (its numerator is summed
 *   directly, never as a difference of sums)
 *
 * A ratio whose denominator is 0 is reported as 0.  The root's branch does
 * not exist: length[root] is ignored.
 *
 * Conventions for every call:
 *   - every entry point returns a uf_status (or a plain value where noted),
 *     never aborts and never throws; on failure uf_last_error() gives a
 *     message for the calling thread;
 *   - inputs are copied: the caller keeps ownership of every pointer it
 *     passes and may free it when the call returns;
 *   - sizes and indices are int64_t; node and sample counts are limited to
 *     2^31 - 1, and one compute call to 2^30 samples (summed over the
 *     tables of a batch; more is UF_EINVAL).
 */
#ifndef UNIFRAC_GB300_H
#define UNIFRAC_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    UF_OK = 0,
    UF_EINVAL = 1,     /* bad argument: null pointer, unknown enum, alpha outside [0, 1] */
    UF_ETREE = 2,      /* malformed tree (see uf_tree_create) */
    UF_ETABLE = 3,     /* malformed table or table / tree mismatch (see uf_table_create) */
    UF_ERANGE = 4,     /* stripe range outside [0, uf_stripe_count(n)] or start > stop */
    UF_ENOMEM = 5,     /* host or device allocation failed, or another host resource ran out */
    UF_ECUDA = 6,      /* a CUDA call failed (no device, launch error, ...) */
    UF_ETIMEOUT = 7,   /* a bounded device wait ran out */
    UF_ECANCELLED = 8  /* reserved: the call was cancelled */
} uf_status;

typedef enum {
    UF_UNWEIGHTED = 0,
    UF_WEIGHTED_UNNORMALIZED = 1,
    UF_WEIGHTED_NORMALIZED = 2,
    UF_GENERALIZED = 3,
    UF_UNWEIGHTED_UNNORMALIZED = 4,
    UF_VAW_WEIGHTED_UNNORMALIZED = 5,
    UF_VAW_WEIGHTED_NORMALIZED = 6
} uf_method;

/*
 * Both precisions keep every cross-branch-block accumulator in int64 fixed
 * point (value * 2^F, F chosen per call from an upper bound of the sums, so
 * that one grid step is about 1e-18 of a tree's root-to-tip distance) and
 * end with one FP64 num / den division.
 * UF_FP64   branch embeddings and per-branch updates in IEEE FP64 on CUDA
 *           cores, partial sums in FP64 before each fixed-point rounding;
 *           every numerator is a sum of nonnegative terms (no cancellation).
 *           Distances d within 1e-10 * |d| + 1e-15 of an FP64 per-pair
 *           evaluation: relative 1e-10 down to d = 1e-5, and the grid's
 *           absolute rounding below that (near-identical samples).
 * UF_MIXED  the paper's FP32 compute mode (Sec. 4): branch embeddings and
 *           per-branch updates in FP32 on CUDA cores -- or, for
 *           UF_UNWEIGHTED, exact 0/1 presence tiles times branch lengths
 *           split into three BF16 terms on the tcgen05 tensor cores with FP32
 *           accumulation -- with FP32 partial sums rounded into the
 *           fixed-point accumulators; distances within 1e-5 absolute
 *           (1e-5 * max(1, d) for UF_WEIGHTED_UNNORMALIZED).
 */
typedef enum { UF_FP64 = 0, UF_MIXED = 1 } uf_precision;

typedef struct uf_tree uf_tree;
typedef struct uf_table uf_table;

/* Filled by uf_compute when its rep argument is not NULL. */
typedef struct {
    double seconds;        /* host wall time of the call */
    double updates;        /* pair x branch updates: pairs covered x (n_nodes - 1) */
    double alg_flops;      /* algorithmic flops of the accumulation */
    double exec_flops;     /* flops executed (tensor path: all three split GEMMs, full tiles) */
    double hbm_bytes_est;  /* modelled HBM bytes of embed + accumulate + finalize */
    int64_t stripe_tile;   /* stripes per accumulator tile */
    int64_t sample_tile;   /* samples per accumulator tile */
    int64_t branch_block;  /* branches per embedding block */
    int64_t n_blocks;      /* embedding blocks (launch groups) used */
    int64_t kernels;       /* kernel launches issued by the call */
    int32_t path;          /* 0 = CUDA-core stripes, 1 = tcgen05 split-BF16 GEMM */
    int32_t clamped;       /* cells whose numerator, formed as a difference of sums
                              (min form, UF_MIXED only), rounded below 0 and was
                              raised to 0; -1 when not read (asynchronous call) */
    double h2d_bytes;      /* host -> device bytes copied by this call (first use of inputs) */
    double d2h_bytes;      /* device -> host bytes copied by this call (host output) */
    /* device time per phase in ms, measured with CUDA events on the call's
     * stream when the "kernel_timing" option is 1 (else 0) */
    double t_embed_ms;     /* tip counts, internal levels, embedding rows */
    double t_accumulate_ms;/* stripe accumulate (or tensor GEMM) launches */
    double t_diag_ms;      /* diagonal accumulate launches */
    double t_finalize_ms;  /* finalize */
    int64_t acc_launches;  /* accumulate launches timed in t_accumulate_ms */
    int64_t chunk_rows;    /* branches per accumulate work unit (autotuned) */
    int32_t graph;         /* 1: the launch sequence ran as one CUDA graph */
    int32_t reserved2;
    int64_t dense_rows;    /* branches run through the dense stripe kernels */
    int64_t sparse_rows;   /* branches kept out of the dense kernels (option "sparse"):
                              scattered pair by pair, or of length 0 and skipped */
    double sparse_pairs;   /* both-nonzero sample pairs of those branches, at most */
    double t_sparse_ms;    /* device time of the sparse-row launches ("kernel_timing") */
    double sparse_pair_updates;  /* pair updates the stripe-region scatter made (one
                              atomic per accumulator word each, two for the
                              duplicated half stripe), counted on the device when
                              "kernel_timing" is 1 and the call is synchronous;
                              -1 otherwise or without a region scatter */
} uf_report;

/*
 * Process-wide options (not tied to a tree or table):
 *   "branch_block"   0 = automatic (default); otherwise the number of
 *                    branches per embedding block (>= 1), e.g. to bound memory
 *   "kernel_timing"  0 (default) or 1: time each phase with CUDA events and
 *                    fill the t_*_ms fields of uf_report (adds a stream sync)
 *   "tensor_path"    1 (default): UF_UNWEIGHTED with UF_MIXED runs on the
 *                    tcgen05 tensor cores when the gram tiles its stripes need
 *                    (128 x 256 int64 cells each, the diagonal tiles included)
 *                    and the sparse rows' stripe cells fit in half the device
 *                    memory that is free or held unused by the stream-ordered
 *                    pool, else on the CUDA-core stripe kernels
 *                    (report path 0); 0: always on the CUDA-core kernels
 *   "graph"          1 (default): a call's branch-block launch sequence is
 *                    captured into a CUDA graph and launched as one graph
 *                    (not when "kernel_timing" is 1); 0: plain launches
 *   "autotune"       1 (default): the first call for an (accumulator,
 *                    precision, size) class times the accumulate kernel on
 *                    its first branch block with every tile shape it offers
 *                    (the FP32 min kernel: 128 x 128 or 64 x 128 stripes x
 *                    samples) and 1,024 / 2,048 / 4,096 / 8,192 branches per
 *                    work unit, and keeps the fastest for the process;
 *                    0: the first shape and 2,048; 2: forget the kept
 *                    choices, then 1
 *   "tile_shape"     -1 (default): the shape the autotuner picks; 0 or 1:
 *                    that shape, where the kernel offers it (for testing)
 *   "sparse"         1 (default): a branch whose subtree holds few count
 *                    entries skips the dense stripe kernels; its terms are
 *                    added pair by pair over the samples nonzero under it,
 *                    when a cost model of the two kernels says that is
 *                    faster; 0: every branch through the dense kernels;
 *                    2: every branch that can be scattered is (subtree with
 *                    at most 4,096 entries per table, 16,384 when one table's
 *                    accumulators are scattered region by region, and
 *                    contiguous tip numbers).  Applies to the CUDA-core stripe kernels and
 *                    to the tensor-core unweighted path; the results agree
 *                    within the precision's tolerance.
 *   "sparse_overlap" 1 (default): the sparse-row scatter runs on a second
 *                    stream beside the count pass, the embeddings and the
 *                    dense stripe kernel or tensor-core gram (it fills the SM
 *                    slots those leave); 0: in sequence with them.  The
 *                    results are the same bit for bit (integer accumulators)
 *   "tensor_wait_test"  0 (default); 1: the tensor-core kernel's MMA issuer
 *                    first waits on a barrier nothing signals, so the bounded
 *                    wait runs out after 2 s: a synchronous call returns
 *                    UF_ETIMEOUT and an asynchronous one writes NaN (for
 *                    testing the abort path; no fault, the context stays usable)
 *   "sparse_fuse"    2 (default), 6 or 0: in the region scatter of a min-form
 *                    method (the weighted methods and the tensor path's
 *                    unweighted) a listed branch also carries the terms of its
 *                    scattered children (2), or of its children and their
 *                    children (6), and adds each pair's summed terms with one
 *                    atomic; 0: every scattered branch on its own.  The
 *                    results are the same bit for bit (integer accumulators)
 *   "sparse_region_bytes"  48,000,000 (default; 0 restores it): a one-table
 *                    call whose stripe accumulators exceed this many bytes
 *                    writes the scattered branches' sample lists once and
 *                    adds their pairs stripe region by region, each region's
 *                    accumulators at most this size (so that they stay in L2);
 *                    at least 4,096
 * uf_set_option returns UF_EINVAL for an unknown name or a bad value;
 * uf_get_option returns -1 for an unknown name.
 */
uf_status uf_set_option(const char *name, int64_t value);
int64_t uf_get_option(const char *name);

/* Message describing the last failure on the calling thread ("" if none). */
const char *uf_last_error(void);

/* Name of a status code ("UF_OK", "UF_ETREE", ...). */
const char *uf_status_name(uf_status st);

/*
 * Number of stripes of an n-sample problem, floor(n / 2) (0 for n < 2).
 * Stripes 0 .. count-1 cover every unordered pair exactly once, except that
 * for even n the last stripe holds each of its n/2 pairs twice (columns k
 * and k + n/2), with equal values.  (Stripe definition: Sec. 2, Fig. 1.)
 */
int64_t uf_stripe_count(int64_t n_samples);

/*
 * Tree (the phylogeny the paper's embeddings are taken over, one branch per
 * non-root node, walked in postorder: Sec. 2, Fig. 1; the library form of
 * the method is a C shared library callable from any language, Abstract).
 * parent[i] is the parent of node i; every non-root node has
 * parent[i] > i (children before parents, as in a postorder); exactly one
 * root, the last node, with parent = -1.  length[i] >= 0 and finite is the
 * length of the branch above node i (length[root] is ignored).  Unary
 * nodes are allowed.  Tips are the nodes with no children; tip j is the
 * j-th tip in index order and carries feature j of every table.
 * Errors: UF_EINVAL (null pointer, n_nodes < 1), UF_ETREE (anything else).
 * The caller keeps ownership of parent / length; *out is owned by the
 * caller and released with uf_tree_destroy.
 */
uf_status uf_tree_create(int64_t n_nodes, const int64_t *parent, const double *length,
                         uf_tree **out);
void uf_tree_destroy(uf_tree *tree);
int64_t uf_tree_tips(const uf_tree *tree);

/*
 * Table (the per-sample feature counts from which the per-branch sample
 * embeddings of Sec. 2-3 are computed):
 * n_samples x n_features counts in CSR with samples as rows
 * (indptr[n_samples + 1], indices[nnz], data[nnz], nnz = indptr[n_samples]).
 * Requires n_features == tips of the tree, indptr[0] == 0, indices strictly
 * increasing within a row and in [0, n_features), data finite and > 0, and
 * at least one nonzero in every sample (else UF_ETABLE).  Counts are summed
 * below each node before the division by the sample total (exact for
 * integer counts).  The caller keeps ownership of the arrays; *out is
 * released with uf_table_destroy and is bound to this tree's tip count.
 */
uf_status uf_table_create(int64_t n_samples, int64_t n_features, const int64_t *indptr,
                          const int32_t *indices, const double *data, const uf_tree *tree,
                          uf_table **out);
void uf_table_destroy(uf_table *table);
int64_t uf_table_samples(const uf_table *table);

/*
 * Distances of the stripes [stripe_start, stripe_stop) (Sec. 2, Fig. 1;
 * stripes are independent subproblems, Abstract and Sec. 3 Table 2 runs).
 *   - [0, uf_stripe_count(n)) writes the full condensed matrix: n(n-1)/2
 *     values, pair (i, j), i < j, at n*i - i*(i+1)/2 + (j - i - 1);
 *   - any other range writes (stop - start) x n values in stripe-major
 *     order, value (s - start) * n + k = distance of the pair
 *     (k, (k + s + 1) mod n) -- the unified stripe buffer layout of Fig. 1;
 *   - start == stop writes nothing and returns UF_OK.
 * out: caller-owned buffer of that many doubles (or floats if out_fp32),
 *   in device memory of the current device if out_is_device (memory of
 *   another device, or host memory, is UF_EINVAL), else in host memory.  alpha is used by UF_GENERALIZED only and must be in [0, 1].
 * cuda_stream: a cudaStream_t (NULL = the legacy default stream).  The call
 *   returns after the results are in out, except when out_is_device is set
 *   and cuda_stream is not NULL: then it returns once the work is enqueued
 *   and out is ready when the stream reaches that point.
 * Working memory comes from the CUDA stream-ordered allocator of the current
 * device and is returned before the work completes on the stream.
 * Errors: UF_EINVAL, UF_ERANGE, UF_ETABLE (table of another tree),
 *   UF_ENOMEM, UF_ECUDA; UF_ETIMEOUT when a bounded wait of the tensor-core
 *   kernel (unweighted, mixed) ran out.  An asynchronous call does not wait
 *   to learn that: every value it writes is then NaN instead.
 */
uf_status uf_compute(const uf_tree *tree, const uf_table *table, uf_method method, double alpha,
                     uf_precision precision, int64_t stripe_start, int64_t stripe_stop, void *out,
                     int out_is_device, int out_fp32, uf_report *rep, void *cuda_stream);

/*
 * Many independent tables over one shared tree (the batching of several
 * input buffers into one kernel invocation, Sec. 3, taken across tables;
 * stripes as independent subproblems, Fig. 1), all full-range (condensed
 * output per table, layout as in uf_compute).  outs[t] receives table t's
 * n_t(n_t-1)/2 doubles (host or device per out_is_device); reps may be NULL
 * or an array of n_tables reports.  The tables' embedding and accumulate
 * work goes to the device as one batched schedule: one launch per embedding
 * level and one accumulate launch for all tables together.  Same stream
 * semantics and errors as uf_compute.
 */
uf_status uf_compute_batch(const uf_tree *tree, const uf_table *const *tables, int64_t n_tables,
                           uf_method method, double alpha, uf_precision precision,
                           void *const *outs, int out_is_device, uf_report *reps,
                           void *cuda_stream);

/*
 * Many stripe ranges in one call (stripes are independent subproblems,
 * Abstract and Fig. 1; several inputs batched into one kernel invocation,
 * Sec. 3): job t computes the stripes [starts[t], stops[t]) of tables[t]
 * into outs[t] -- the condensed matrix for the full range, stripe-major
 * values otherwise, as uf_compute -- in doubles, or floats if out_fp32.  A
 * table may appear in several jobs; all tables share the tree.  The jobs go
 * to the device as one batched schedule: one launch per embedding level and
 * one accumulate launch (or tensor-core gram) for all jobs together.  An
 * empty range writes nothing.  reps may be NULL or an array of n_jobs
 * reports.  Same stream semantics as uf_compute.
 * Errors: UF_EINVAL, UF_ERANGE (a range outside [0, uf_stripe_count(n)] or
 * start > stop), UF_ETABLE, UF_ENOMEM, UF_ECUDA, UF_ETIMEOUT.
 */
uf_status uf_compute_ranges(const uf_tree *tree, const uf_table *const *tables, const int64_t *starts,
                            const int64_t *stops, int64_t n_jobs, uf_method method, double alpha,
                            uf_precision precision, void *const *outs, int out_is_device, int out_fp32,
                            uf_report *reps, void *cuda_stream);

/*
 * uf_compute_noalloc -- the full-range computation of uf_compute (condensed
 * FP64 output) without allocating any device memory.  The paper has no
 * counterpart; it exists for callers that may not call cudaMalloc: an
 * application whose own memory manager owns the device heap (a framework's
 * caching allocator, a service held to a fixed device-memory budget), or code
 * that must not enter the allocator because its latency or its failure path
 * is not allowed at that point.
 *
 * Working memory is one fixed area of UF_NOALLOC_SCRATCH_BYTES (64 MiB) that
 * every GPU loading this library reserves until the process exits; tree and
 * table data are copied into it from the handles on every call.  A problem
 * whose working set (inputs, count sums, embedding rows, stripe accumulators)
 * does not fit is rejected with UF_ENOMEM and a message giving both sizes,
 * before any work is enqueued.
 * out_device: caller-owned device memory of n(n-1)/2 doubles on the current
 *   device (memory of another device, or host memory, is UF_EINVAL), layout
 *   as in uf_compute.  cuda_stream: cudaStream_t or NULL.  The call returns
 *   after the results are in out_device.
 * Methods UF_UNWEIGHTED .. UF_GENERALIZED (others are UF_EINVAL).
 * The first call on a device, with that device current, sets up the area's
 * device address (cudaGetSymbolAddress); make that first call before any
 * stream capture begins on the device.  All calls on a device share the area
 * and leave their data in it (accumulators are cleared by each call); calls
 * whose work overlaps on the GPU -- from other threads or other streams --
 * race on it.
 * Errors: UF_EINVAL, UF_ETABLE, UF_ENOMEM (too large for the area), UF_ECUDA.
 */
#define UF_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)
uf_status uf_compute_noalloc(const uf_tree *tree, const uf_table *table, uf_method method,
                             double alpha, uf_precision precision, double *out_device,
                             void *cuda_stream);

/*
 * uf_probe_l2_atomics -- diagnostic, not part of the method: the rate of
 * random 64-bit atomic adds into a device array of `bytes` bytes on the
 * current device (8 x a power of two, 8 KiB .. 16 GiB; 16 MiB stays in L2),
 * each thread adding 1 to pseudo-random words with no other memory traffic.
 * It is the ceiling that the stripe-region scatter's atomics (uf_compute's
 * sparse_pair_updates) are measured against.  Allocates and frees the array;
 * synchronous.  *adds_per_second receives the rate (0 on error).
 * Errors: UF_EINVAL (bad size or NULL), UF_ECUDA.
 */
uf_status uf_probe_l2_atomics(int64_t bytes, double *adds_per_second);

#ifdef __cplusplus
}
#endif

#endif /* UNIFRAC_GB300_H */
