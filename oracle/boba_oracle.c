/*
 * BOBA oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded C restatement of what the BOBA hot path
 * computes (arXiv 2306.10410).  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load this file; the CUDA library never
 * includes, links or calls it, and it shares no code with the CUDA library.
 *
 * Every function cites the passage of the paper it follows.  Conventions:
 *   - COO(G) = (I, J), I, J in [n]^m, edge i is I(i) -> J(i)       (Sec. 2.1)
 *   - vertex IDs and positions are 0-based here (the paper's figures count
 *     from 1); the endpoint stream is I ++ J, position i < m holds I(i) and
 *     position m + e holds J(e)                                      (Sec. 4.3)
 *   - perm[k] = v means new label k holds old vertex v (p_k = v), and
 *     label = perm^-1                                                (Sec. 4.3)
 *
 * Return codes: 0 ok, 1 invalid argument, 2 a vertex ID outside [0, n).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_SENT 0xFFFFFFFFu

static int check_ids(const int32_t *a, int64_t m, int64_t n)
{
    for (int64_t i = 0; i < m; ++i)
        if (a[i] < 0 || (int64_t)a[i] >= n) return 2;
    return 0;
}

/*
 * First-occurrence keys, the r of Algorithm 2 (Sec. 4.4) when its update is an
 * AtomicMin: key[v] = min{ i in [0, 2m) : (I ++ J)(i) = v }, and the sentinel
 * 0xFFFFFFFF (the paper's "infinity") for a vertex in no edge.
 * Written as the definition: one ascending scan that keeps the first hit.
 */
int oracle_first_keys(const int32_t *I, const int32_t *J, int64_t m, int64_t n,
                      uint32_t *key)
{
    if (m < 0 || n < 0 || (m > 0 && n == 0)) return 1;
    if (check_ids(I, m, n) || check_ids(J, m, n)) return 2;
    for (int64_t v = 0; v < n; ++v) key[v] = ORACLE_SENT;
    for (int64_t i = 0; i < 2 * m; ++i) {
        int32_t v = (i < m) ? I[i] : J[i - m];
        if (key[v] == ORACLE_SENT) key[v] = (uint32_t)i;
    }
    return 0;
}

/*
 * Sequential BOBA, Algorithm 1 (Sec. 4.3): scan I, then J, with a seen-set S;
 * the first time a vertex is met it takes the next label.  The algorithm
 * requires every vertex to lie on an edge; a vertex on none is appended after
 * all others in ascending original ID, which is what Algorithm 2's initial
 * p = (1..n) followed by a stable ordering on keys r = infinity gives.
 * Alg. 1 stops early once all n vertices are seen; the result is the same
 * whether or not it does, so the loop simply runs to the end.
 * perm and label (both length n) receive p and p^-1.
 */
int oracle_boba_perm(const int32_t *I, const int32_t *J, int64_t m, int64_t n,
                     int32_t *perm, int32_t *label)
{
    if (m < 0 || n < 0 || (m > 0 && n == 0)) return 1;
    if (check_ids(I, m, n) || check_ids(J, m, n)) return 2;
    unsigned char *seen = (unsigned char *)calloc((size_t)(n > 0 ? n : 1), 1);
    if (!seen) return 1;
    int64_t k = 0;
    for (int64_t j = 0; j < m; ++j) {            /* the I half of I ++ J */
        int32_t v = I[j];
        if (!seen[v]) { seen[v] = 1; perm[k++] = v; }
    }
    if (k < n) {
        for (int64_t j = 0; j < m; ++j) {        /* the J half */
            int32_t v = J[j];
            if (!seen[v]) { seen[v] = 1; perm[k++] = v; }
        }
    }
    for (int64_t v = 0; v < n; ++v)              /* vertices on no edge */
        if (!seen[v]) perm[k++] = (int32_t)v;
    for (int64_t q = 0; q < n; ++q) label[perm[q]] = (int32_t)q;
    free(seen);
    return 0;
}

/*
 * The interleaved reading of Fig. 1: the flattened list I(0) J(0) I(1) J(1) ...
 * uniquified in stable order, then the isolated tail as above.  Used only to
 * reproduce the figure's printed "Uniquified" row; the method itself follows
 * I ++ J (Sec. 1.2, Alg. 1, Alg. 2).
 */
int oracle_boba_perm_interleaved(const int32_t *I, const int32_t *J, int64_t m,
                                 int64_t n, int32_t *perm, int32_t *label)
{
    if (m < 0 || n < 0 || (m > 0 && n == 0)) return 1;
    if (check_ids(I, m, n) || check_ids(J, m, n)) return 2;
    unsigned char *seen = (unsigned char *)calloc((size_t)(n > 0 ? n : 1), 1);
    if (!seen) return 1;
    int64_t k = 0;
    for (int64_t j = 0; j < m; ++j) {
        int32_t u = I[j], v = J[j];
        if (!seen[u]) { seen[u] = 1; perm[k++] = u; }
        if (!seen[v]) { seen[v] = 1; perm[k++] = v; }
    }
    for (int64_t v = 0; v < n; ++v)
        if (!seen[v]) perm[k++] = (int32_t)v;
    for (int64_t q = 0; q < n; ++q) label[perm[q]] = (int32_t)q;
    free(seen);
    return 0;
}

/*
 * Rewrite every edge through the permutation (Sec. 5.3 reorders the COO before
 * COO->CSR conversion): I'(e) = label[I(e)], J'(e) = label[J(e)], edge order
 * unchanged.
 */
int oracle_relabel(const int32_t *I, const int32_t *J, int64_t m, int64_t n,
                   const int32_t *label, int32_t *I_out, int32_t *J_out)
{
    if (m < 0 || n < 0) return 1;
    if (check_ids(I, m, n) || check_ids(J, m, n)) return 2;
    for (int64_t e = 0; e < m; ++e) {
        I_out[e] = label[I[e]];
        J_out[e] = label[J[e]];
    }
    return 0;
}

/*
 * COO -> CSR for the pull SpMV of Algorithm 3 (Sec. 1.2.2): row v lists the
 * in-neighbours u of v, i.e. the edges u -> v, so row = J (destination) and
 * column = I (source).  A stable counting sort: count rows, exclusive prefix
 * sum into row_ptr, then place edges in input order.  Duplicated edges stay
 * separate entries.  The entry for edge u -> v holds
 *   val = fp32( 1 / outdeg(u) ),  outdeg(u) = #{e : I(e) = u} (duplicates count),
 * the PageRank-style column normalisation (Sec. 5.1); fp32 rounding of the
 * fp64 quotient equals the correctly rounded fp32 quotient.
 * row_ptr has n+1 entries; col_out and val_out have m.
 */
int oracle_coo_to_csr(const int32_t *I, const int32_t *J, int64_t m, int64_t n,
                      int64_t *row_ptr, int32_t *col_out, float *val_out)
{
    if (m < 0 || n < 0 || (m > 0 && n == 0)) return 1;
    if (check_ids(I, m, n) || check_ids(J, m, n)) return 2;
    int64_t *outdeg = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    int64_t *cursor = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    if (!outdeg || !cursor) { free(outdeg); free(cursor); return 1; }
    for (int64_t v = 0; v <= n; ++v) row_ptr[v] = 0;
    for (int64_t e = 0; e < m; ++e) {
        row_ptr[J[e] + 1] += 1;
        outdeg[I[e]] += 1;
    }
    for (int64_t v = 0; v < n; ++v) row_ptr[v + 1] += row_ptr[v];
    for (int64_t v = 0; v < n; ++v) cursor[v] = row_ptr[v];
    for (int64_t e = 0; e < m; ++e) {
        int64_t p = cursor[J[e]]++;
        col_out[p] = I[e];
        val_out[p] = (float)(1.0 / (double)outdeg[I[e]]);
    }
    free(outdeg);
    free(cursor);
    return 0;
}

/*
 * Pull SpMV, Algorithm 3 (Sec. 1.2.2): y(v) = sum over the entries of row v of
 * A(v,u) * x(u), accumulated in fp64 in row order from the fp32 inputs.
 */
int oracle_spmv_f64(const int64_t *row_ptr, const int32_t *col, const float *val,
                    const float *x, int64_t n_rows, double *y)
{
    if (n_rows < 0) return 1;
    for (int64_t r = 0; r < n_rows; ++r) {
        double acc = 0.0;
        for (int64_t p = row_ptr[r]; p < row_ptr[r + 1]; ++p)
            acc += (double)val[p] * (double)x[col[p]];
        y[r] = acc;
    }
    return 0;
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/*
 * The NBR spatial-locality metric (Sec. 5.2):
 *   NBR(G) = (1/n') * sum over v with N(v) non-empty of lines(N(v)) / |N(v)|,
 * N(v) the set of distinct neighbours listed in CSR row v, lines(N(v)) the
 * number of distinct cache lines (u / ids_per_line) they fall in, and n' the
 * number of rows with a non-empty N(v) (rows with no neighbour have no ratio).
 * Returns the metric; writes the count n' to *n_counted.
 */
double oracle_nbr(const int64_t *row_ptr, const int32_t *col, int64_t n_rows,
                  int64_t ids_per_line, int64_t *n_counted)
{
    double sum = 0.0;
    int64_t counted = 0;
    int64_t cap = 0;
    int32_t *buf = NULL;
    for (int64_t r = 0; r < n_rows; ++r) {
        int64_t len = row_ptr[r + 1] - row_ptr[r];
        if (len == 0) continue;
        if (len > cap) {
            free(buf);
            cap = len;
            buf = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
            if (!buf) { if (n_counted) *n_counted = -1; return -1.0; }
        }
        memcpy(buf, col + row_ptr[r], (size_t)len * sizeof(int32_t));
        qsort(buf, (size_t)len, sizeof(int32_t), cmp_i32);
        int64_t distinct = 0, lines = 0;
        for (int64_t q = 0; q < len; ++q) {
            if (q == 0 || buf[q] != buf[q - 1]) {
                distinct++;
                if (q == 0 || buf[q] / ids_per_line != buf[q - 1] / ids_per_line)
                    lines++;
            }
        }
        sum += (double)lines / (double)distinct;
        counted++;
    }
    free(buf);
    if (n_counted) *n_counted = counted;
    return counted ? sum / (double)counted : 0.0;
}

/*
 * PageRank by power iteration over the edge list, the PR application of
 * Sec. 5.1 (it sweeps the whole graph repeatedly until convergence).  The paper
 * fixes none of its constants, so this is the standard definition (Page, Brin,
 * Motwani, Winograd 1999) in fp64, dangling mass spread uniformly:
 *   pr_0(v)     = 1/n
 *   D_t         = sum of pr_t(u) over the vertices u with outdeg(u) = 0
 *   pr_{t+1}(v) = (1 - d)/n + d * ( sum over edges u -> v of pr_t(u)/outdeg(u) + D_t/n )
 * outdeg counts duplicated edges; a self-loop is an ordinary edge.  Steps until
 * sum_v |pr_{t+1}(v) - pr_t(v)| < tol or max_iters steps have been taken.
 * pr (length n) receives the last iterate; *iters the steps taken and
 * *residual the last step's L1 change (0 if no step was taken).
 */
int oracle_pagerank(const int32_t *I, const int32_t *J, int64_t m, int64_t n, double d,
                    int64_t max_iters, double tol, double *pr, int64_t *iters, double *residual)
{
    if (m < 0 || n < 0 || (m > 0 && n == 0) || max_iters < 0 || !(d >= 0.0 && d < 1.0))
        return 1;
    if (check_ids(I, m, n) || check_ids(J, m, n)) return 2;
    *iters = 0;
    *residual = 0.0;
    if (n == 0) return 0;
    int64_t *outdeg = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    double *next = (double *)malloc((size_t)n * sizeof(double));
    if (!outdeg || !next) { free(outdeg); free(next); return 1; }
    for (int64_t e = 0; e < m; ++e) outdeg[I[e]] += 1;
    for (int64_t v = 0; v < n; ++v) pr[v] = 1.0 / (double)n;
    for (int64_t t = 0; t < max_iters; ++t) {
        double dangling = 0.0;
        for (int64_t u = 0; u < n; ++u)
            if (outdeg[u] == 0) dangling += pr[u];
        for (int64_t v = 0; v < n; ++v) next[v] = 0.0;
        for (int64_t e = 0; e < m; ++e) next[J[e]] += pr[I[e]] / (double)outdeg[I[e]];
        double change = 0.0;
        for (int64_t v = 0; v < n; ++v) {
            double nv = (1.0 - d) / (double)n + d * (next[v] + dangling / (double)n);
            change += fabs(nv - pr[v]);
            pr[v] = nv;
        }
        *iters = t + 1;
        *residual = change;
        if (change < tol) break;
    }
    free(outdeg);
    free(next);
    return 0;
}
