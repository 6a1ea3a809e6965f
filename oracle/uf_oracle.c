/*
 * uf_oracle.c -- plain FP64 CPU oracle for UniFrac distances.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: only the tests, the smoke check and the benchmark's CPU
 * baseline use it.  It shares no code, header or table with the CUDA path.
 *
 * What it computes (per sample pair, straight from the definition):
 *   The paper (Sec. 1, refs [1] and [3]) names UniFrac and Striped UniFrac
 *   but prints no formula.  The definitions used are the standard ones of
 *   the metric literature the paper cites:
 *     c_{A,f}  = count of feature f in sample A,  T_A = sum_f c_{A,f}
 *     p_A(v)   = (sum of c_{A,f} over tips f below node v) / T_A
 *     a_A(v)   = [p_A(v) > 0]
 *     sum over every non-root node v, l_v = length of the branch above v
 *   unweighted             num = sum l_v (a_A xor a_B)   den = sum l_v (a_A or a_B)
 *   weighted unnormalized  d   = sum l_v |p_A - p_B|
 *   weighted normalized    num = sum l_v |p_A - p_B|     den = sum l_v (p_A + p_B)
 *   generalized(alpha)     over v with s = p_A + p_B > 0:
 *                          num = sum l_v s^alpha |p_A - p_B| / s
 *                          den = sum l_v s^alpha
 *   d = num / den, and d = 0 when den == 0.
 *
 * Further members of the Striped UniFrac family (the paper names the family,
 * Sec. 1, without formulas; the definitions are the published ones):
 *   unweighted unnormalized  d = sum l_v (a_A xor a_B): the unweighted
 *                          numerator without the division, as weighted
 *                          unnormalized is the weighted numerator alone.
 *   variance-adjusted weighted (Chang, Luan & Sun, BMC Bioinformatics 12:118,
 *   2011): every branch term is divided by sqrt(m_v (m - m_v)), with
 *     m_v = C_A(v) + C_B(v)  the two samples' counts below v,
 *     m   = T_A + T_B        their totals,
 *   over the branches with m_v > 0 and m - m_v > 0 (readings: a branch with
 *   m_v = 0 holds neither sample and adds 0; one with m_v = m holds all of
 *   both samples' counts, p_A = p_B = 1, and carries no information: it
 *   adds 0 to num and den):
 *     vaw unnormalized     d = sum l_v |p_A - p_B| / sqrt(m_v (m - m_v))
 *     vaw normalized       num = the same sum,
 *                          den = sum l_v (p_A + p_B) / sqrt(m_v (m - m_v)),
 *                          d = num / den (0 when den == 0).
 *
 * Algorithm, per pair (A, B), in the order the definition reads:
 *   1. scatter each sample's counts onto its tips,
 *   2. walk the nodes in postorder (children before parents) adding each
 *      node's count sum into its parent -- integer counts stay exact in FP64,
 *   3. divide each node sum by the sample total once,
 *   4. add the method's terms for every non-root node in postorder order,
 *   5. finalize num / den with the den == 0 -> 0 rule.
 *
 * A second routine, uo_striped, is the plain striped CPU loop of the paper's
 * Sec. 2-3 (Figs. 1-3): for every branch in postorder and every stripe s and
 * sample k it adds f(emb[k], emb[(k+s+1) mod n]) * length into a unified
 * stripe buffer indexed (s - start) * n + k.  It is a CPU baseline and a
 * second formulation checked against the per-pair walk in the tests.
 *
 * Validation mirrors the library's documented contract: the tree is a parent
 * array with parent[i] > i for every non-root node and exactly one root, the
 * last node; non-root lengths finite and >= 0; the table is CSR with samples
 * as rows, features mapped to tips in tip index order, indices strictly
 * increasing in a row, data finite and > 0, and no empty sample.
 */
#define _GNU_SOURCE
#include <math.h>
#include <pthread.h>
#include <sched.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

enum { UO_OK = 0, UO_EINVAL = 1, UO_ETREE = 2, UO_ETABLE = 3, UO_ERANGE = 4, UO_ENOMEM = 5 };
enum {
    UO_UNWEIGHTED = 0,
    UO_WEIGHTED_UNNORMALIZED = 1,
    UO_WEIGHTED_NORMALIZED = 2,
    UO_GENERALIZED = 3,
    UO_UNWEIGHTED_UNNORMALIZED = 4,
    UO_VAW_UNNORMALIZED = 5,
    UO_VAW_NORMALIZED = 6
};
#define UO_LAST_METHOD UO_VAW_NORMALIZED

/* methods whose distance is the numerator alone */
static int unnormalized(int method) {
    return method == UO_WEIGHTED_UNNORMALIZED || method == UO_UNWEIGHTED_UNNORMALIZED ||
           method == UO_VAW_UNNORMALIZED;
}

int uo_host_cores(void) {
    cpu_set_t set;
    CPU_ZERO(&set);
    if (sched_getaffinity(0, sizeof(set), &set) == 0) {
        int c = CPU_COUNT(&set);
        if (c > 0) return c;
    }
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    return c > 0 ? (int)c : 1;
}

/* ---- validation ------------------------------------------------------- */

int uo_check_tree(int64_t n_nodes, const int64_t *parent, const double *length) {
    if (n_nodes < 1 || !parent || !length) return UO_EINVAL;
    if (parent[n_nodes - 1] != -1) return UO_ETREE;
    for (int64_t i = 0; i + 1 < n_nodes; i++) {
        if (parent[i] <= i || parent[i] >= n_nodes) return UO_ETREE;
        if (!isfinite(length[i]) || length[i] < 0.0) return UO_ETREE;
    }
    return UO_OK;
}

/* tip_node[f] = node index of the f-th tip (tips = nodes with no children). */
static int64_t find_tips(int64_t n_nodes, const int64_t *parent, int64_t *tip_node) {
    char *has_child = calloc((size_t)n_nodes, 1);
    if (!has_child) return -1;
    for (int64_t i = 0; i + 1 < n_nodes; i++) has_child[parent[i]] = 1;
    int64_t t = 0;
    for (int64_t i = 0; i < n_nodes; i++)
        if (!has_child[i]) {
            if (tip_node) tip_node[t] = i;
            t++;
        }
    free(has_child);
    return t;
}

int64_t uo_tip_count(int64_t n_nodes, const int64_t *parent) {
    return find_tips(n_nodes, parent, NULL);
}

int uo_check_table(int64_t n_samples, int64_t n_features, const int64_t *indptr,
                   const int32_t *indices, const double *data, int64_t n_tips) {
    if (n_samples < 1 || n_features < 0 || !indptr) return UO_EINVAL;
    if (n_features != n_tips) return UO_ETABLE;
    if (indptr[0] != 0) return UO_ETABLE;
    for (int64_t k = 0; k < n_samples; k++) {
        int64_t b = indptr[k], e = indptr[k + 1];
        if (e <= b) return UO_ETABLE; /* decreasing pointer or empty sample */
        for (int64_t q = b; q < e; q++) {
            if (indices[q] < 0 || indices[q] >= n_features) return UO_ETABLE;
            if (q > b && indices[q] <= indices[q - 1]) return UO_ETABLE;
            if (!isfinite(data[q]) || data[q] <= 0.0) return UO_ETABLE;
        }
    }
    return UO_OK;
}

/* ---- the per-pair tree walk ------------------------------------------ */

typedef struct {
    int64_t n_nodes;
    const int64_t *parent;
    const double *length;
    const int64_t *tip_node;
    const int64_t *indptr;
    const int32_t *indices;
    const double *data;
    int method;
    double alpha;
    const int64_t *pi, *pj;
    double *out_d, *out_num, *out_den;
    int64_t n_pairs;
    int64_t next; /* shared work counter, guarded by mu */
    pthread_mutex_t mu;
    int failed;
} pair_job;

static double sample_total(const pair_job *J, int64_t a) {
    double t = 0.0;
    for (int64_t q = J->indptr[a]; q < J->indptr[a + 1]; q++) t += J->data[q];
    return t;
}

/* Steps 1-2: node count sums of sample a, written into C[0..n_nodes). */
static void node_sums(const pair_job *J, int64_t a, double *C) {
    memset(C, 0, sizeof(double) * (size_t)J->n_nodes);
    for (int64_t q = J->indptr[a]; q < J->indptr[a + 1]; q++)
        C[J->tip_node[J->indices[q]]] = J->data[q];
    for (int64_t v = 0; v + 1 < J->n_nodes; v++) C[J->parent[v]] += C[v];
}

static void one_pair(const pair_job *J, int64_t a, int64_t b, double *CA, double *CB,
                     double *d_out, double *num_out, double *den_out) {
    node_sums(J, a, CA);
    node_sums(J, b, CB);
    const double TA = sample_total(J, a), TB = sample_total(J, b);
    double num = 0.0, den = 0.0;
    for (int64_t v = 0; v + 1 < J->n_nodes; v++) {
        const double l = J->length[v];
        const double pA = CA[v] / TA, pB = CB[v] / TB; /* step 3 */
        switch (J->method) {
        case UO_UNWEIGHTED:
        case UO_UNWEIGHTED_UNNORMALIZED: {
            const int xa = pA > 0.0, xb = pB > 0.0;
            num += l * (double)(xa ^ xb);
            den += l * (double)(xa | xb);
        } break;
        case UO_WEIGHTED_UNNORMALIZED:
            num += l * fabs(pA - pB);
            break;
        case UO_VAW_UNNORMALIZED:
        case UO_VAW_NORMALIZED: {
            const double mv = CA[v] + CB[v], rest = (TA + TB) - mv;
            if (mv > 0.0 && rest > 0.0) {
                const double w = 1.0 / sqrt(mv * rest);
                num += l * w * fabs(pA - pB);
                den += l * w * (pA + pB);
            }
        } break;
        case UO_WEIGHTED_NORMALIZED:
            num += l * fabs(pA - pB);
            den += l * (pA + pB);
            break;
        case UO_GENERALIZED: {
            const double s = pA + pB;
            if (s > 0.0) {
                const double sa = pow(s, J->alpha);
                num += l * sa * fabs(pA - pB) / s;
                den += l * sa;
            }
        } break;
        }
    }
    double d;
    if (unnormalized(J->method)) d = num;
    else d = (den == 0.0) ? 0.0 : num / den;
    *d_out = d;
    if (num_out) *num_out = num;
    if (den_out) *den_out = den;
}

static void *pair_worker(void *arg) {
    pair_job *J = (pair_job *)arg;
    double *CA = malloc(sizeof(double) * (size_t)J->n_nodes);
    double *CB = malloc(sizeof(double) * (size_t)J->n_nodes);
    if (!CA || !CB) {
        pthread_mutex_lock(&J->mu);
        J->failed = 1;
        pthread_mutex_unlock(&J->mu);
        free(CA);
        free(CB);
        return NULL;
    }
    for (;;) {
        pthread_mutex_lock(&J->mu);
        int64_t i = J->next;
        J->next += 16;
        pthread_mutex_unlock(&J->mu);
        if (i >= J->n_pairs) break;
        int64_t e = i + 16 < J->n_pairs ? i + 16 : J->n_pairs;
        for (; i < e; i++)
            one_pair(J, J->pi[i], J->pj[i], CA, CB, &J->out_d[i],
                     J->out_num ? &J->out_num[i] : NULL, J->out_den ? &J->out_den[i] : NULL);
    }
    free(CA);
    free(CB);
    return NULL;
}

/*
 * Distances for n_pairs sample pairs (pi[q], pj[q]).  out_num / out_den may
 * be NULL.  n_threads <= 0 uses every core this process may run on.
 * Returns a status code; on success *threads_used is the thread count.
 */
int uo_pairs(int64_t n_nodes, const int64_t *parent, const double *length,
             int64_t n_samples, int64_t n_features, const int64_t *indptr,
             const int32_t *indices, const double *data, int method, double alpha,
             int64_t n_pairs, const int64_t *pi, const int64_t *pj, double *out_d,
             double *out_num, double *out_den, int n_threads, int *threads_used) {
    int st = uo_check_tree(n_nodes, parent, length);
    if (st) return st;
    if (method < UO_UNWEIGHTED || method > UO_LAST_METHOD) return UO_EINVAL;
    if (method == UO_GENERALIZED && !(alpha >= 0.0 && alpha <= 1.0)) return UO_EINVAL;
    int64_t *tip_node = malloc(sizeof(int64_t) * (size_t)n_nodes);
    if (!tip_node) return UO_ENOMEM;
    int64_t n_tips = find_tips(n_nodes, parent, tip_node);
    st = uo_check_table(n_samples, n_features, indptr, indices, data, n_tips);
    if (st) {
        free(tip_node);
        return st;
    }
    for (int64_t q = 0; q < n_pairs; q++)
        if (pi[q] < 0 || pi[q] >= n_samples || pj[q] < 0 || pj[q] >= n_samples) {
            free(tip_node);
            return UO_ERANGE;
        }
    pair_job J = {n_nodes, parent, length, tip_node, indptr, indices, data, method, alpha,
                  pi, pj, out_d, out_num, out_den, n_pairs, 0, PTHREAD_MUTEX_INITIALIZER, 0};
    int nt = n_threads > 0 ? n_threads : uo_host_cores();
    if (nt > 256) nt = 256;
    if ((int64_t)nt > (n_pairs + 15) / 16) nt = (int)((n_pairs + 15) / 16);
    if (nt < 1) nt = 1;
    pthread_t th[256];
    int started = 0;
    for (int t = 0; t < nt; t++)
        if (pthread_create(&th[t], NULL, pair_worker, &J) == 0) started++;
        else break;
    if (started == 0) pair_worker(&J);
    for (int t = 0; t < started; t++) pthread_join(th[t], NULL);
    free(tip_node);
    if (threads_used) *threads_used = started ? started : 1;
    return J.failed ? UO_ENOMEM : UO_OK;
}

/* ---- the plain striped loop (paper Sec. 2-3) ------------------------- */

typedef struct {
    int64_t n_nodes;
    const int64_t *parent;
    const double *length;
    const int64_t *tip_of_node; /* node -> tip number, -1 for internal nodes */
    const int64_t *col_ptr;     /* CSC view of the table: tip f's samples */
    const int64_t *col_row;
    const double *col_val;
    const double *total;        /* per-sample totals */
    int method;
    double alpha;
    int64_t n, start, stop;
    double *num, *den;          /* unified stripe buffers, (stop - start) * n */
    int64_t s_begin, s_end;     /* this worker's stripes */
    int failed;
} stripe_job;

/* Each worker walks every branch in postorder on its own and updates only its
 * own stripes, so workers never write the same cell. */
static void *stripe_worker(void *arg) {
    stripe_job *J = (stripe_job *)arg;
    const int64_t n = J->n, N = J->n_nodes;
    double *emb = malloc(sizeof(double) * (size_t)n);
    double **pending = calloc((size_t)N, sizeof(double *));
    if (!emb || !pending) { J->failed = 1; free(emb); free(pending); return NULL; }
    for (int64_t v = 0; v + 1 < N; v++) {
        /* the branch embedding: counts below v, divided by the sample totals */
        double *cnt = pending[v];
        pending[v] = NULL;
        if (!cnt) {
            cnt = calloc((size_t)n, sizeof(double));
            if (!cnt) { J->failed = 1; break; }
        }
        const int64_t f = J->tip_of_node[v];
        if (f >= 0)
            for (int64_t q = J->col_ptr[f]; q < J->col_ptr[f + 1]; q++) cnt[J->col_row[q]] = J->col_val[q];
        for (int64_t k = 0; k < n; k++) emb[k] = cnt[k] / J->total[k];
        const double l = J->length[v];
        for (int64_t s = J->s_begin; s < J->s_end; s++) {
            double *num = J->num + (s - J->start) * n;
            double *den = J->den + (s - J->start) * n;
            for (int64_t k = 0; k < n; k++) {
                const int64_t j = (k + s + 1) % n;
                const double u = emb[k];
                const double w = emb[j];
                switch (J->method) {
                case UO_UNWEIGHTED:
                case UO_UNWEIGHTED_UNNORMALIZED: {
                    const int xa = u > 0.0, xb = w > 0.0;
                    num[k] += l * (double)(xa ^ xb);
                    den[k] += l * (double)(xa | xb);
                } break;
                case UO_WEIGHTED_UNNORMALIZED:
                    num[k] += l * fabs(u - w);
                    break;
                case UO_VAW_UNNORMALIZED:
                case UO_VAW_NORMALIZED: {
                    const double mv = cnt[k] + cnt[j], rest = (J->total[k] + J->total[j]) - mv;
                    if (mv > 0.0 && rest > 0.0) {
                        const double wt = 1.0 / sqrt(mv * rest);
                        num[k] += l * wt * fabs(u - w);
                        den[k] += l * wt * (u + w);
                    }
                } break;
                case UO_WEIGHTED_NORMALIZED:
                    num[k] += l * fabs(u - w);
                    den[k] += l * (u + w);
                    break;
                case UO_GENERALIZED: {
                    const double sm = u + w;
                    if (sm > 0.0) {
                        const double sa = pow(sm, J->alpha);
                        num[k] += l * sa * fabs(u - w) / sm;
                        den[k] += l * sa;
                    }
                } break;
                }
            }
        }
        /* hand the count row to the parent (the root's sum is never used) */
        const int64_t p = J->parent[v];
        if (p != N - 1) {
            if (!pending[p]) { pending[p] = cnt; cnt = NULL; }
            else for (int64_t k = 0; k < n; k++) pending[p][k] += cnt[k];
        }
        free(cnt);
    }
    for (int64_t v = 0; v < N; v++) free(pending[v]);
    free(pending);
    free(emb);
    return NULL;
}

/*
 * Striped loop over stripes [start, stop): fills num / den stripe buffers
 * ((stop - start) * n each, zeroed here) and, if dist is not NULL, the
 * finalized distances in the same stripe-major layout.  Stripe s, column k
 * holds the pair (k, (k + s + 1) mod n).
 */
int uo_striped(int64_t n_nodes, const int64_t *parent, const double *length,
               int64_t n_samples, int64_t n_features, const int64_t *indptr,
               const int32_t *indices, const double *data, int method, double alpha,
               int64_t start, int64_t stop, double *num, double *den, double *dist,
               int n_threads, int *threads_used) {
    int st = uo_check_tree(n_nodes, parent, length);
    if (st) return st;
    if (method < UO_UNWEIGHTED || method > UO_LAST_METHOD) return UO_EINVAL;
    if (method == UO_GENERALIZED && !(alpha >= 0.0 && alpha <= 1.0)) return UO_EINVAL;
    const int64_t n = n_samples;
    if (start < 0 || stop < start || stop > n / 2) return UO_ERANGE;
    int64_t *tip_node = malloc(sizeof(int64_t) * (size_t)n_nodes);
    if (!tip_node) return UO_ENOMEM;
    const int64_t n_tips = find_tips(n_nodes, parent, tip_node);
    st = uo_check_table(n_samples, n_features, indptr, indices, data, n_tips);
    if (st) { free(tip_node); return st; }
    const int64_t rows = stop - start, nnz = indptr[n];
    int64_t *tip_of_node = malloc(sizeof(int64_t) * (size_t)n_nodes);
    int64_t *col_ptr = calloc((size_t)n_tips + 1, sizeof(int64_t));
    int64_t *col_row = malloc(sizeof(int64_t) * (size_t)(nnz + 1));
    double *col_val = malloc(sizeof(double) * (size_t)(nnz + 1));
    double *total = malloc(sizeof(double) * (size_t)n);
    int64_t *fill = calloc((size_t)n_tips + 1, sizeof(int64_t));
    if (!tip_of_node || !col_ptr || !col_row || !col_val || !total || !fill) {
        free(tip_node); free(tip_of_node); free(col_ptr); free(col_row); free(col_val);
        free(total); free(fill);
        return UO_ENOMEM;
    }
    for (int64_t v = 0; v < n_nodes; v++) tip_of_node[v] = -1;
    for (int64_t f = 0; f < n_tips; f++) tip_of_node[tip_node[f]] = f;
    for (int64_t q = 0; q < nnz; q++) col_ptr[indices[q] + 1]++;
    for (int64_t f = 0; f < n_tips; f++) col_ptr[f + 1] += col_ptr[f];
    for (int64_t k = 0; k < n; k++) {
        double t = 0.0;
        for (int64_t q = indptr[k]; q < indptr[k + 1]; q++) {
            const int64_t f = indices[q];
            col_row[col_ptr[f] + fill[f]] = k;
            col_val[col_ptr[f] + fill[f]] = data[q];
            fill[f]++;
            t += data[q];
        }
        total[k] = t;
    }
    memset(num, 0, sizeof(double) * (size_t)(rows * n));
    memset(den, 0, sizeof(double) * (size_t)(rows * n));
    int nt = n_threads > 0 ? n_threads : uo_host_cores();
    if (nt > 256) nt = 256;
    if (nt > rows) nt = rows > 0 ? (int)rows : 1;
    pthread_t th[256];
    stripe_job jobs[256];
    int started = 0, failed = 0;
    for (int t = 0; t < nt; t++) {
        jobs[t] = (stripe_job){n_nodes, parent, length, tip_of_node, col_ptr, col_row, col_val,
                               total, method, alpha, n, start, stop, num, den,
                               start + rows * t / nt, start + rows * (t + 1) / nt, 0};
    }
    for (int t = 0; t < nt; t++)
        if (pthread_create(&th[t], NULL, stripe_worker, &jobs[t]) == 0) started++;
        else break;
    for (int t = started; t < nt; t++) stripe_worker(&jobs[t]);
    for (int t = 0; t < started; t++) pthread_join(th[t], NULL);
    for (int t = 0; t < nt; t++) failed |= jobs[t].failed;
    if (!failed && dist) {
        for (int64_t r = 0; r < rows * n; r++) {
            if (unnormalized(method)) dist[r] = num[r];
            else dist[r] = den[r] == 0.0 ? 0.0 : num[r] / den[r];
        }
    }
    free(tip_node); free(tip_of_node); free(col_ptr); free(col_row); free(col_val);
    free(total); free(fill);
    if (threads_used) *threads_used = nt;
    return failed ? UO_ENOMEM : UO_OK;
}
