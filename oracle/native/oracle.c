/*
 * Plain FP64 CPU oracle for CSR-k sparse matrix-vector multiplication (test infrastructure).
 *
 * This file is the oracle that the CUDA path is checked against.  It is deliberately slow
 * and direct: one row at a time, one nonzero at a time, in stored order, with no blocking,
 * vectorisation or reordering of the arithmetic.  It must be compiled with
 * -ffp-contract=off so that every product is rounded before it is added (no FMA), which
 * makes it bit-identical to the Python oracle in oracle/spmv.py.
 *
 * It shares no code with the product library; only tests, the smoke check and the CPU
 * baseline leg of the benchmark load it.
 *
 * Functions:
 *   oracle_csr_spmv       y = alpha*A*x + beta*y, plain CSR        (Sec. 1 problem statement;
 *                                                                   Listing 1 inner loops)
 *   oracle_csr_spmv_rows  the same for a chosen subset of rows     (sampled checks at full size)
 *   oracle_csr3_spmv      the CSR-3 loop nest over super-super-rows, super-rows and rows
 *                                                                  (Listing 1, Sec. 2.2)
 *   oracle_csr3_spmv_omp  the same loop nest with Listing 1's OpenMP parallel loop over
 *                         super-super-rows (static schedule); CSR-2 is the case of one
 *                         super-row per super-super-row.  The timed CPU baseline.
 *                                                                  (Listing 1; Sec. 4.2, 6.1)
 *   oracle_csr_spmm       Y = alpha*A*X + beta*Y, k right-hand sides, X/Y row-major
 *   oracle_rcm            reverse Cuthill-McKee ordering (Sec. 2.1; reading spelled out below)
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* y_i = alpha * (sum over the row's stored entries, left to right, of a_ij * x_j)
 *       + beta * y_i.  With beta == 0 the old y is not read (BLAS convention), so
 *       NaN or garbage in y does not propagate. */
void oracle_csr_spmv(int32_t n, const int32_t* rowptr, const int32_t* colidx,
                     const double* vals, const double* x, double alpha, double beta,
                     double* y) {
    for (int32_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            double prod = vals[p] * x[colidx[p]];
            s = s + prod;
        }
        if (beta == 0.0) y[i] = alpha * s;
        else y[i] = alpha * s + beta * y[i];
    }
}

/* Same arithmetic as oracle_csr_spmv, for rows[0..m-1] only; out[t] is row rows[t].
 * yin may be NULL when beta == 0. */
void oracle_csr_spmv_rows(const int32_t* rowptr, const int32_t* colidx, const double* vals,
                          const double* x, double alpha, double beta, const double* yin,
                          const int64_t* rows, int64_t m, double* out) {
    for (int64_t t = 0; t < m; ++t) {
        int64_t i = rows[t];
        double s = 0.0;
        for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            double prod = vals[p] * x[colidx[p]];
            s = s + prod;
        }
        if (beta == 0.0) out[t] = alpha * s;
        else out[t] = alpha * s + beta * yin[i];
    }
}

/* Listing 1: loop over super-super-rows, then their super-rows, then their rows; each row's
 * dot product is the plain CSR one.  (The listing's OpenMP pragma is left out: the order of
 * rows does not change any single row's result.) */
void oracle_csr3_spmv(int32_t num_ssr, const int32_t* ssr_ptr, const int32_t* sr_ptr,
                      const int32_t* rowptr, const int32_t* colidx, const double* vals,
                      const double* x, double* y) {
    for (int32_t i = 0; i < num_ssr; ++i) {
        for (int32_t j = ssr_ptr[i]; j < ssr_ptr[i + 1]; ++j) {
            for (int32_t k = sr_ptr[j]; k < sr_ptr[j + 1]; ++k) {
                double temp = 0.0;
                for (int32_t l = rowptr[k]; l < rowptr[k + 1]; ++l) {
                    double prod = vals[l] * x[colidx[l]];
                    temp = temp + prod;
                }
                y[k] = temp;
            }
        }
    }
}

/* Listing 1 as printed, with its "parallel for" over super-super-rows: OpenMP threads
 * share the outermost loop in equal contiguous blocks (schedule(static)).  A row's result
 * is computed exactly as in oracle_csr3_spmv, so y is bit-identical to it for any thread
 * count.  nthreads <= 0 uses the OpenMP default.  Returns the number of threads that ran
 * the loop (1 when the file was built without OpenMP). */
#ifdef _OPENMP
#include <omp.h>
#endif
int oracle_csr3_spmv_omp(int32_t num_ssr, const int32_t* ssr_ptr, const int32_t* sr_ptr,
                         const int32_t* rowptr, const int32_t* colidx, const double* vals,
                         const double* x, double* y, int nthreads) {
    int used = 1;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
    {
#pragma omp single
        used = omp_get_num_threads();
#pragma omp for schedule(static)
        for (int32_t i = 0; i < num_ssr; ++i) {
            for (int32_t j = ssr_ptr[i]; j < ssr_ptr[i + 1]; ++j) {
                for (int32_t k = sr_ptr[j]; k < sr_ptr[j + 1]; ++k) {
                    double temp = 0.0;
                    for (int32_t l = rowptr[k]; l < rowptr[k + 1]; ++l) {
                        double prod = vals[l] * x[colidx[l]];
                        temp = temp + prod;
                    }
                    y[k] = temp;
                }
            }
        }
    }
#else
    (void)nthreads;
    oracle_csr3_spmv(num_ssr, ssr_ptr, sr_ptr, rowptr, colidx, vals, x, y);
#endif
    return used;
}

/* Y = alpha*A*X + beta*Y for k right-hand sides; X is n x k row-major with leading
 * dimension ldx, Y likewise with ldy.  Column c is exactly oracle_csr_spmv on X[:, c]. */
void oracle_csr_spmm(int32_t n, const int32_t* rowptr, const int32_t* colidx,
                     const double* vals, int32_t k, const double* X, int64_t ldx,
                     double alpha, double beta, double* Y, int64_t ldy) {
    for (int32_t c = 0; c < k; ++c) {
        for (int32_t i = 0; i < n; ++i) {
            double s = 0.0;
            for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
                double prod = vals[p] * X[(int64_t)colidx[p] * ldx + c];
                s = s + prod;
            }
            double* yi = &Y[(int64_t)i * ldy + c];
            if (beta == 0.0) *yi = alpha * s;
            else *yi = alpha * s + beta * *yi;
        }
    }
}

/* ------------------------------------------------------------------------------------
 * Reverse Cuthill-McKee (Sec. 2.1 names RCM as the bandwidth-limiting ordering; Sec. 5.3
 * applies it to the comparison libraries' inputs).  The paper does not define start node,
 * ties or disconnected graphs, so this oracle fixes the reading:
 *   1. Graph: vertices 0..n-1, edge {i,j} for i != j when A stores (i,j) or (j,i).
 *      deg(v) = number of distinct neighbours.
 *   2. While unvisited vertices remain: start s = unvisited vertex of least degree,
 *      smallest index on ties.
 *   3. Pseudo-peripheral search (George-Liu): level structure from s inside the unvisited
 *      part; c = least-degree vertex of the last level (smallest index on ties); if the
 *      level structure from c is deeper than the one from s, s = c and repeat; at most
 *      8 rounds.
 *   4. Cuthill-McKee: breadth-first from s; when a vertex is taken from the queue its
 *      unvisited neighbours are appended in order of (degree, index) ascending.
 *   5. Concatenate the components' sequences and reverse the whole: perm[new] = old.
 * ------------------------------------------------------------------------------------ */

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/* neighbour lists of the symmetrised pattern, sorted, self-loops and repeats removed */
static int build_graph(int32_t n, const int32_t* rowptr, const int32_t* colidx,
                       int64_t** xadj_out, int32_t** adj_out) {
    int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    if (!cnt) return -1;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            int32_t j = colidx[p];
            if (j == i) continue;
            cnt[i + 1]++;
            cnt[j + 1]++;
        }
    for (int32_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
    int32_t* tmp = (int32_t*)malloc(sizeof(int32_t) * (size_t)(cnt[n] > 0 ? cnt[n] : 1));
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!tmp || !fill) { free(cnt); free(tmp); free(fill); return -1; }
    for (int32_t i = 0; i < n; ++i) fill[i] = cnt[i];
    for (int32_t i = 0; i < n; ++i)
        for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            int32_t j = colidx[p];
            if (j == i) continue;
            tmp[fill[i]++] = j;
            tmp[fill[j]++] = i;
        }
    int64_t* xadj = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
    if (!xadj) { free(cnt); free(tmp); free(fill); return -1; }
    int64_t w = 0;
    xadj[0] = 0;
    for (int32_t i = 0; i < n; ++i) {
        int64_t a = cnt[i], b = cnt[i + 1];
        qsort(tmp + a, (size_t)(b - a), sizeof(int32_t), cmp_i32);
        for (int64_t q = a; q < b; ++q)
            if (q == a || tmp[q] != tmp[q - 1]) tmp[w++] = tmp[q];
        xadj[i + 1] = w;
    }
    free(cnt);
    free(fill);
    *xadj_out = xadj;
    *adj_out = tmp;
    return 0;
}

/* Breadth-first level structure from root over vertices with visited[v] == 0.  Returns
 * the number of levels; the last level's vertices are order[last_begin .. count-1]. */
static int32_t levels_from(int32_t root, const int64_t* xadj, const int32_t* adj,
                           const unsigned char* visited, int32_t* mark, int32_t stamp,
                           int32_t* order, int32_t* count, int32_t* last_begin) {
    int32_t head = 0, tail = 0, nlev = 0;
    order[tail++] = root;
    mark[root] = stamp;
    int32_t level_end = tail;
    int32_t begin = 0;
    while (head < tail) {
        begin = head;
        level_end = tail;
        nlev++;
        for (; head < level_end; ++head) {
            int32_t v = order[head];
            for (int64_t q = xadj[v]; q < xadj[v + 1]; ++q) {
                int32_t u = adj[q];
                if (!visited[u] && mark[u] != stamp) {
                    mark[u] = stamp;
                    order[tail++] = u;
                }
            }
        }
    }
    *count = tail;
    *last_begin = begin;
    return nlev;
}

typedef struct { int32_t deg, idx; } degkey;
static int cmp_degkey(const void* a, const void* b) {
    const degkey* x = (const degkey*)a;
    const degkey* y = (const degkey*)b;
    if (x->deg != y->deg) return (x->deg > y->deg) - (x->deg < y->deg);
    return (x->idx > y->idx) - (x->idx < y->idx);
}

/* perm[new] = old.  Returns 0 on success, -1 on allocation failure. */
int oracle_rcm(int32_t n, const int32_t* rowptr, const int32_t* colidx, int32_t* perm) {
    if (n <= 0) return 0;
    int64_t* xadj = NULL;
    int32_t* adj = NULL;
    if (build_graph(n, rowptr, colidx, &xadj, &adj)) return -1;
    unsigned char* visited = (unsigned char*)calloc((size_t)n, 1);
    int32_t* mark = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int32_t* scratch = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int32_t* seq = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int64_t maxdeg = 0;
    for (int32_t v = 0; v < n; ++v)
        if (xadj[v + 1] - xadj[v] > maxdeg) maxdeg = xadj[v + 1] - xadj[v];
    degkey* kids = (degkey*)malloc(sizeof(degkey) * (size_t)(maxdeg + 1));
    if (!visited || !mark || !scratch || !seq || !kids) {
        free(xadj); free(adj); free(visited); free(mark); free(scratch); free(seq); free(kids);
        return -1;
    }
    for (int32_t v = 0; v < n; ++v) mark[v] = -1;
    int32_t stamp = 0;
    int32_t nseq = 0;
    while (nseq < n) {
        /* step 2: least-degree unvisited vertex, smallest index on ties */
        int32_t s = -1;
        int64_t best = 0;
        for (int32_t v = 0; v < n; ++v) {
            if (visited[v]) continue;
            int64_t d = xadj[v + 1] - xadj[v];
            if (s < 0 || d < best) { s = v; best = d; }
        }
        /* step 3: pseudo-peripheral refinement */
        int32_t cnt, last_begin;
        int32_t depth = levels_from(s, xadj, adj, visited, mark, stamp++, scratch, &cnt, &last_begin);
        for (int round = 0; round < 8; ++round) {
            int32_t c = -1;
            int64_t cd = 0;
            for (int32_t q = last_begin; q < cnt; ++q) {
                int32_t v = scratch[q];
                int64_t d = xadj[v + 1] - xadj[v];
                if (c < 0 || d < cd || (d == cd && v < c)) { c = v; cd = d; }
            }
            int32_t cnt2, lb2;
            int32_t depth2 = levels_from(c, xadj, adj, visited, mark, stamp++, scratch, &cnt2, &lb2);
            if (depth2 > depth) {
                s = c;
                depth = depth2;
                cnt = cnt2;
                last_begin = lb2;
            } else {
                break;
            }
        }
        /* step 4: Cuthill-McKee breadth-first order from s */
        int32_t head = nseq;
        seq[nseq++] = s;
        visited[s] = 1;
        while (head < nseq) {
            int32_t v = seq[head++];
            int32_t m = 0;
            for (int64_t q = xadj[v]; q < xadj[v + 1]; ++q) {
                int32_t u = adj[q];
                if (!visited[u]) {
                    kids[m].deg = (int32_t)(xadj[u + 1] - xadj[u]);
                    kids[m].idx = u;
                    m++;
                }
            }
            qsort(kids, (size_t)m, sizeof(degkey), cmp_degkey);
            for (int32_t t = 0; t < m; ++t) {
                visited[kids[t].idx] = 1;
                seq[nseq++] = kids[t].idx;
            }
        }
    }
    /* step 5: reverse */
    for (int32_t i = 0; i < n; ++i) perm[i] = seq[n - 1 - i];
    free(xadj); free(adj); free(visited); free(mark); free(scratch); free(seq); free(kids);
    return 0;
}
