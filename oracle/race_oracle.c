/*
 * CPU ORACLE — TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously-correct reference for the SymmSpMV library.  Only
 * the test-suite, the smoke check and the benchmark's CPU-baseline leg may
 * load this file's shared object; the library itself never does, and shares
 * no code with it.
 *
 * Paper: Alappat et al., "A Recursive Algebraic Coloring Technique for
 * Hardware-Efficient Symmetric Sparse Matrix-Vector Multiplication"
 * (arXiv 1907.06487).  Section/algorithm/equation names below refer to it.
 *
 * Numeric part (FP64 throughout):
 *   orc_expand_full    symmetric expansion of upper CRS into full CRS
 *   orc_spmv_full      Alg. "SpMV using the CRS format" (b = A x), plus the
 *                      per-row scale s_i = sum_j |a_ij||x_j| used by the
 *                      parity bound |b_i - b_ref_i| <= tol * s_i
 *   orc_symm_spmv      Alg. "SymmSpMV" executed serially (b zeroed first)
 *   orc_spmv_sampled   b_i and s_i of the plain definition for chosen rows
 *                      only, in one pass over the upper CRS
 *   orc_symm_spmv_race Alg. "SymmSpMV" under a RACE schedule on CPU threads,
 *                      the paper's own execution model (OpenMP)
 *   orc_spmv_full_par  Alg. "SpMV using the CRS format" with its rows split
 *                      over CPU threads (OpenMP), no s
 *   orc_symm_gs        symmetric Gauss-Seidel sweeps under a schedule (R11)
 *   orc_symm_kacz      symmetric Kaczmarz sweeps under a schedule (R12)
 *   orc_coloring       MC / ABMC multicolouring schedules (R14)
 *   orc_matrix_powers  Y[:, q] = A^(q+1) x for q < p, the definition applied
 *                      p times, with |A|^(q+1) |x| for the bound (R13)
 *
 * Schedule part (integer + FP64 control arithmetic), Section 4:
 *   level construction (Alg. "Construction of levels", Eq. "level"),
 *   level-group pairing by the epsilon rule (Sec. 4.4.3 steps 1-3),
 *   red/blue split and load balancing with worker weights (Alg. "Load
 *   Balancing", Sec. 4.3 and 4.4.3 step 4), recursion into level groups with
 *   the distance-1 halo (Sec. 4.4.2), the RACE tree, effective row counts and
 *   parallel efficiency eta (Sec. 5), and a flattening of the tree into
 *   globally synchronised phases.
 *
 * Readings taken where the paper is silent or garbled (each one is listed
 * in the design notes of the repository):
 *   R1 root of a (sub)graph = its last vertex in the current order
 *      (Alg. "Construction of levels" sets root = n).  Opt-in: stage-0
 *      roots become a pseudo-peripheral vertex of their component
 *      (George and Liu, ACM TOMS 5, 1979), the start node of the RCM
 *      orderings the paper's inputs carry (Sec. 6.1).
 *   Opt-in RCM: the construction runs on the matrix relabelled by reverse
 *      Cuthill-McKee (components in the order of their lowest vertex, each
 *      from its pseudo-peripheral vertex; neighbours newly reached from a
 *      vertex taken by increasing degree, lowest index on ties; the whole
 *      sequence reversed), and its permutation is composed with that order.
 *   R2 BFS runs until the frontier is empty; unvisited vertices of the group
 *      restart from the last unvisited one at (max level so far) + 2
 *      (islands, Sec. 4.4.1).
 *   R3 inside a level vertices keep their current relative order.
 *   R4 weight a = (sum of sizes) * n_t(parent) / size(parent), one FP64
 *      division of exact integers; b = max(1, round-half-away(a));
 *      eps = 1 - |a - b|; acceptance eps > eps_s (strict).
 *   R5 a pair needs >= 2k levels and eps > eps_s; afterwards it grows only
 *      while a' <= b, keeping the strictly best eps (first wins ties).
 *      Remaining levels that cannot form a pair, fewer than 2k levels left,
 *      or threads used up: the rest joins the last pair, which gets all
 *      remaining threads.
 *   R6 red gets floor(n/2) levels of a pair, blue the rest.
 *   R7 load balancing: u_i = size_i / worker_i, mean_c = sum size / sum
 *      worker over colour c, var = sum diff^2 / len (left to right); the
 *      group index is absRankIdx[currRank]; shift(src->dst) moves one level
 *      from src to dst and slides the groups between them.
 *   R8 recursion into every group with > 1 thread while the stage limit
 *      allows; sub-graph = group plus its distance-1 halo (k = 2).
 *   R9 phases: P(leaf)=1, P(node) = max P over red children + max P over
 *      blue children; red children start at the node's offset, blue ones
 *      after the red block.  Empty leaves are not listed.
 *   R10 opt-in: stage-0 level groups need only one level (k = 1 in the
 *      pairing and balancing of the whole graph).  With upper storage in
 *      level order a row of level j updates b only in levels j and j + 1
 *      (lower storage: j - 1 and j), so same-colour groups one level apart
 *      stay write-disjoint, though not distance-2 independent; deeper
 *      stages keep k = 2 (halo neighbours are not confined to the next
 *      sub-level).
 *   R11 symmetric Gauss-Seidel on a schedule: the serial sweep in the
 *      schedule's execution order (forward: phases in order, rows of a leaf
 *      ascending; backward: phases reversed, rows descending), on the full
 *      matrix in the schedule's order.
 *   R12 symmetric Kaczmarz on a schedule: the same passes, each row
 *      projecting x onto its hyperplane (writes every column of the row).
 *   R14 multicolouring schedules (MC, ABMC): the paper compares with COLPACK
 *      and METIS; written here from its description, first-fit colouring in
 *      unit order, ABMC blocks = consecutive rows of the given order.
 *   R13 matrix powers: the paper names in-place matrix powers as future work
 *      only.  Read as the powers A x, A^2 x, ..., A^p x written as the p
 *      columns of one n x p array, each computed from the previous column
 *      (no vector storage besides the output); the values are those of the
 *      plain definition, whatever the order of evaluation.
 */
#ifdef _OPENMP
#include <omp.h>
#else
static int omp_get_max_threads(void) { return 1; }
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ====================================================================== */
/* Numeric oracle                                                          */
/* ====================================================================== */

/* Full symmetric CRS from upper CRS.  frp has n+1 entries; fci/fva must
 * hold 2*nnz_u - n_diag entries.  Columns of each full row come out sorted
 * (lower part first in increasing row order, then the upper part).       */
int64_t orc_expand_full(int32_t n, const int32_t *rp, const int32_t *ci, const double *va,
                        int64_t *frp, int32_t *fci, double *fva) {
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!cnt) return -1;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t t = rp[i]; t < rp[i + 1]; ++t) {
            cnt[i]++;
            if (ci[t] != i) cnt[ci[t]]++;
        }
    frp[0] = 0;
    for (int32_t i = 0; i < n; ++i) frp[i + 1] = frp[i] + cnt[i];
    for (int32_t i = 0; i < n; ++i) cnt[i] = frp[i];
    /* lower part: entry (i,j) of row i with j>i appears as (j,i) in row j;
       visiting i in increasing order appends in increasing column order. */
    for (int32_t i = 0; i < n; ++i)
        for (int32_t t = rp[i]; t < rp[i + 1]; ++t) {
            int32_t j = ci[t];
            if (j != i) { fci[cnt[j]] = i; fva[cnt[j]] = va[t]; cnt[j]++; }
        }
    for (int32_t i = 0; i < n; ++i)
        for (int32_t t = rp[i]; t < rp[i + 1]; ++t) {
            fci[cnt[i]] = ci[t]; fva[cnt[i]] = va[t]; cnt[i]++;
        }
    int64_t nnz = frp[n];
    free(cnt);
    return nnz;
}

/* Alg. "SpMV using the CRS format": b[row] = sum_idx A[idx]*x[col[idx]].
 * Also s[row] = sum |A[idx]|*|x[col[idx]]| (NULL to skip).                */
void orc_spmv_full(int32_t n, const int64_t *frp, const int32_t *fci, const double *fva,
                   const double *x, double *b, double *s) {
    for (int32_t row = 0; row < n; ++row) {
        double tmp = 0.0, a = 0.0;
        for (int64_t idx = frp[row]; idx < frp[row + 1]; ++idx) {
            tmp += fva[idx] * x[fci[idx]];
            a += fabs(fva[idx]) * fabs(x[fci[idx]]);
        }
        b[row] = tmp;
        if (s) s[row] = a;
    }
}

/* Matrix powers (R13: the paper's conclusion names in-place matrix powers
 * among the kernels a level-based formulation serves).  Y is n x p, column
 * q (entries q*n .. q*n+n-1) = A^(q+1) x: the plain definition applied p
 * times, each power to the previous one (Alg. "SpMV using the CRS format" on
 * the full matrix).  S (NULL to skip), same shape, = |A|^(q+1) |x|: every
 * rounding of power q is bounded in terms of it.  tmp: n doubles of
 * scratch when S is given.                                                */
void orc_matrix_powers(int32_t n, const int64_t *frp, const int32_t *fci, const double *fva, int32_t p,
                       const double *x, double *Y, double *S, double *tmp) {
    for (int32_t q = 0; q < p; ++q) {
        const double *src = q == 0 ? x : Y + (int64_t)(q - 1) * n;
        orc_spmv_full(n, frp, fci, fva, src, Y + (int64_t)q * n, q == 0 && S ? S : NULL);
        if (S && q > 0) /* |A| S_{q-1}: S_{q-1} >= 0, so the s output of the
                           definition applied to it is exactly that        */
            orc_spmv_full(n, frp, fci, fva, S + (int64_t)(q - 1) * n, tmp, S + (int64_t)q * n);
    }
}

/* SpMM with a row-major n x k block: B[:,c] = A X[:,c] column by column.  */
void orc_spmm_full(int32_t n, const int64_t *frp, const int32_t *fci, const double *fva,
                   int32_t k, const double *X, double *B, double *S) {
    for (int32_t row = 0; row < n; ++row)
        for (int32_t c = 0; c < k; ++c) {
            double tmp = 0.0, a = 0.0;
            for (int64_t idx = frp[row]; idx < frp[row + 1]; ++idx) {
                double xv = X[(int64_t)fci[idx] * k + c];
                tmp += fva[idx] * xv;
                a += fabs(fva[idx]) * fabs(xv);
            }
            B[(int64_t)row * k + c] = tmp;
            if (S) S[(int64_t)row * k + c] = a;
        }
}

/* Alg. "SymmSpMV" run serially; the algorithm accumulates with +=, so b
 * starts at zero.  The diagonal is the first entry of each row.           */
void orc_symm_spmv(int32_t n, const int32_t *rp, const int32_t *ci, const double *va,
                   const double *x, double *b) {
    for (int32_t i = 0; i < n; ++i) b[i] = 0.0;
    for (int32_t row = 0; row < n; ++row) {
        int32_t diag_idx = rp[row];
        b[row] += va[diag_idx] * x[row];
        double tmp = 0.0;
        for (int32_t idx = rp[row] + 1; idx < rp[row + 1]; ++idx) {
            tmp += va[idx] * x[ci[idx]];
            b[ci[idx]] += va[idx] * x[row];
        }
        b[row] += tmp;
    }
}

/* Alg. "SymmSpMV" under a RACE schedule, executed the way the paper runs it
 * on a multicore CPU (Sec. 4 and 6): the phases one after another with a
 * barrier between them; inside a phase the leaves run concurrently, one
 * leaf per thread at a time, each leaf's rows in order with plain updates
 * of b.  The leaves of a phase are distance-2 independent, so no two of them
 * touch one entry of b, and the result does not depend on the thread count
 * or the interleaving: every b entry receives its updates in phase order,
 * then row order.  Input: the permuted upper CRS and the flattened phases
 * (stage_ptr over leaf ranges [lo, hi)).  b is zeroed first.  nthreads <= 0
 * takes the OpenMP default; without OpenMP the loop runs serially.        */
void orc_symm_spmv_race(int32_t n, const int32_t *rp, const int32_t *ci, const double *va,
                        int32_t nphases, const int32_t *stage_ptr, const int32_t *lo, const int32_t *hi,
                        const double *x, double *b, int32_t nthreads) {
    (void)nthreads;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : omp_get_max_threads())
    {
#pragma omp for schedule(static)
        for (int32_t i = 0; i < n; ++i) b[i] = 0.0;
        for (int32_t p = 0; p < nphases; ++p) {
#pragma omp for schedule(dynamic, 1)
            for (int32_t l = stage_ptr[p]; l < stage_ptr[p + 1]; ++l) {
                for (int32_t row = lo[l]; row < hi[l]; ++row) {
                    b[row] += va[rp[row]] * x[row];
                    double tmp = 0.0;
                    for (int32_t idx = rp[row] + 1; idx < rp[row + 1]; ++idx) {
                        tmp += va[idx] * x[ci[idx]];
                        b[ci[idx]] += va[idx] * x[row];
                    }
                    b[row] += tmp;
                }
            }
        }
    }
}

/* Alg. "SpMV using the CRS format" with the rows split statically over CPU
 * threads (OpenMP; serial without it).                                    */
void orc_spmv_full_par(int32_t n, const int64_t *frp, const int32_t *fci, const double *fva,
                       const double *x, double *b, int32_t nthreads) {
    (void)nthreads;
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : omp_get_max_threads())
    for (int32_t row = 0; row < n; ++row) {
        double tmp = 0.0;
        for (int64_t idx = frp[row]; idx < frp[row + 1]; ++idx) tmp += fva[idx] * x[fci[idx]];
        b[row] = tmp;
    }
}

/* Threads the OpenMP runtime would use (1 without OpenMP).               */
int32_t orc_max_threads(void) { return omp_get_max_threads(); }

/* b_i = sum_j a_ij x_j and s_i = sum_j |a_ij||x_j| of the symmetric matrix
 * for the rows listed in rows[0..m), reading the upper CRS once.  Works on
 * a k-column row-major block (k=1 for a vector); outputs are m x k.       */
int orc_spmv_sampled(int32_t n, const int32_t *rp, const int32_t *ci, const double *va,
                     int32_t k, const double *X, int32_t m, const int32_t *rows,
                     double *B, double *S) {
    int32_t *slot = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!slot) return -1;
    for (int32_t i = 0; i < n; ++i) slot[i] = -1;
    for (int32_t q = 0; q < m; ++q) {
        if (rows[q] < 0 || rows[q] >= n || slot[rows[q]] != -1) { free(slot); return -2; }
        slot[rows[q]] = q;
    }
    for (int64_t q = 0; q < (int64_t)m * k; ++q) { B[q] = 0.0; S[q] = 0.0; }
    for (int32_t i = 0; i < n; ++i)
        for (int32_t t = rp[i]; t < rp[i + 1]; ++t) {
            int32_t j = ci[t];
            double a = va[t];
            if (slot[i] >= 0)       /* a_ij x_j contributes to row i */
                for (int32_t c = 0; c < k; ++c) {
                    double xv = X[(int64_t)j * k + c];
                    B[(int64_t)slot[i] * k + c] += a * xv;
                    S[(int64_t)slot[i] * k + c] += fabs(a) * fabs(xv);
                }
            if (j != i && slot[j] >= 0)   /* symmetric partner a_ji = a_ij */
                for (int32_t c = 0; c < k; ++c) {
                    double xv = X[(int64_t)i * k + c];
                    B[(int64_t)slot[j] * k + c] += a * xv;
                    S[(int64_t)slot[j] * k + c] += fabs(a) * fabs(xv);
                }
        }
    free(slot);
    return 0;
}

/* Canonical upper CRS from rows of (col,val) with col >= row in any order:
 * explicit 0.0 diagonal when missing, diagonal first, increasing columns.
 * Returns nnz of the output, -1 on an entry below the diagonal or a
 * duplicate.  Output arrays must hold nnz_in + n entries.                 */
static int cmp_pair(const void *a, const void *b) {
    const int64_t *x = (const int64_t *)a, *y = (const int64_t *)b;
    return (x[0] > y[0]) - (x[0] < y[0]);
}
int64_t orc_canonicalize(int32_t n, const int32_t *rp, const int32_t *ci, const double *va,
                         int32_t *orp, int32_t *oci, double *ova) {
    int64_t k = 0;
    int64_t maxrow = 0;
    for (int32_t i = 0; i < n; ++i)
        if (rp[i + 1] - rp[i] > maxrow) maxrow = rp[i + 1] - rp[i];
    int64_t *buf = (int64_t *)malloc(sizeof(int64_t) * 2 * (size_t)(maxrow + 1));
    if (!buf) return -2;
    for (int32_t i = 0; i < n; ++i) {
        orp[i] = (int32_t)k;
        int32_t len = rp[i + 1] - rp[i];
        int has_diag = 0;
        for (int32_t t = 0; t < len; ++t) {
            int32_t c = ci[rp[i] + t];
            if (c < i || c >= n) { free(buf); return -1; }
            if (c == i) has_diag = 1;
            buf[2 * t] = c; buf[2 * t + 1] = rp[i] + t;
        }
        qsort(buf, (size_t)len, 2 * sizeof(int64_t), cmp_pair);
        for (int32_t t = 1; t < len; ++t)
            if (buf[2 * t] == buf[2 * t - 2]) { free(buf); return -1; }
        if (!has_diag) { oci[k] = i; ova[k] = 0.0; ++k; }
        for (int32_t t = 0; t < len; ++t) { oci[k] = (int32_t)buf[2 * t]; ova[k] = va[buf[2 * t + 1]]; ++k; }
    }
    orp[n] = (int32_t)k;
    free(buf);
    return k;
}

/* ====================================================================== */
/* Schedule oracle                                                         */
/* ====================================================================== */

typedef struct {
    int32_t parent, stage, color, lo, hi, nthreads, thread_lo, nlev, nsub;
    int32_t first_child, nchildren, phase_count, phase_off;
    int64_t size, neff;
} onode;

typedef struct {
    int32_t n, nt, k, balance, max_depth, pp, one0;
    double eps[8];
    /* graph: full adjacency without self loops */
    int64_t *aptr; int32_t *adj;
    int64_t *vw;           /* vertex size in the balancing unit */
    /* current order */
    int32_t *order, *pos;
    /* BFS scratch */
    int32_t *dist, *tmark, *hmark, *dmark, *curr, *next;
    int32_t stamp;
    /* tree */
    onode *nodes; int32_t nnodes, capnodes;
    /* phases */
    int32_t nphases, nleaves;
    int32_t *stage_ptr, *leaf_lo, *leaf_hi, *leaf_node;
    double eta;
    int err;
} osched;

static int32_t new_node(osched *S) {
    if (S->nnodes == S->capnodes) {
        S->capnodes = S->capnodes ? 2 * S->capnodes : 64;
        S->nodes = (onode *)realloc(S->nodes, sizeof(onode) * (size_t)S->capnodes);
    }
    memset(&S->nodes[S->nnodes], 0, sizeof(onode));
    S->nodes[S->nnodes].first_child = -1;
    return S->nnodes++;
}

/* Breadth-first search over the whole graph from r: returns the
 * eccentricity of r and lists the vertices at that distance in far[0..*nfar).
 * dist must hold -1 everywhere on entry and does so again on return.     */
static int32_t ecc_from(const int64_t *aptr, const int32_t *adj, int32_t r, int32_t *dist, int32_t *queue,
                        int32_t *far, int32_t *nfar) {
    int32_t head = 0, tail = 0, ecc = 0;
    dist[r] = 0; queue[tail++] = r;
    while (head < tail) {
        int32_t u = queue[head++];
        if (dist[u] > ecc) ecc = dist[u];
        for (int64_t e = aptr[u]; e < aptr[u + 1]; ++e)
            if (dist[adj[e]] < 0) { dist[adj[e]] = dist[u] + 1; queue[tail++] = adj[e]; }
    }
    *nfar = 0;
    for (int32_t q = 0; q < tail; ++q) if (dist[queue[q]] == ecc) far[(*nfar)++] = queue[q];
    for (int32_t q = 0; q < tail; ++q) dist[queue[q]] = -1;
    return ecc;
}

/* George and Liu's pseudo-peripheral node finder: from the start r, pick
 * the vertex x of minimum degree (smallest index on ties) among the
 * vertices farthest from r; if x is farther from its own farthest vertices
 * than r is, continue from x, else r is the answer.                        */
static int32_t pseudo_peripheral(int32_t n, const int64_t *aptr, const int32_t *adj, int32_t r) {
    int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *far = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    for (int32_t i = 0; i < n; ++i) dist[i] = -1;
    int32_t nfar = 0;
    int32_t ecc_r = ecc_from(aptr, adj, r, dist, queue, far, &nfar);
    for (;;) {
        int32_t x = far[0];
        for (int32_t q = 1; q < nfar; ++q) {
            int32_t w = far[q];
            int64_t dw = aptr[w + 1] - aptr[w], dx = aptr[x + 1] - aptr[x];
            if (dw < dx || (dw == dx && w < x)) x = w;
        }
        int32_t ecc_x = ecc_from(aptr, adj, x, dist, queue, far, &nfar);
        if (ecc_x <= ecc_r) break;
        r = x; ecc_r = ecc_x;
    }
    free(dist); free(queue); free(far);
    return r;
}

/* Reverse Cuthill-McKee sequence (out[new] = old) of the graph aptr/adj.   */
static void rcm_sequence(int32_t n, const int64_t *aptr, const int32_t *adj, int32_t *out) {
    char *seen = (char *)calloc((size_t)n, 1);
    int32_t *kids = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t len = 0;
    for (int32_t v = 0; v < n; ++v) {
        if (seen[v]) continue;
        int32_t head = len;
        int32_t start = pseudo_peripheral(n, aptr, adj, v);
        out[len++] = start; seen[start] = 1;
        while (head < len) {
            int32_t u = out[head++], nk = 0;
            for (int64_t e = aptr[u]; e < aptr[u + 1]; ++e)
                if (!seen[adj[e]]) { seen[adj[e]] = 1; kids[nk++] = adj[e]; }
            /* insertion sort by (degree, index) */
            for (int32_t i = 1; i < nk; ++i) {
                int32_t w = kids[i], j = i;
                int64_t dw = aptr[w + 1] - aptr[w];
                while (j > 0) {
                    int32_t z = kids[j - 1];
                    int64_t dz = aptr[z + 1] - aptr[z];
                    if (dz < dw || (dz == dw && z < w)) break;
                    kids[j] = z; --j;
                }
                kids[j] = w;
            }
            for (int32_t i = 0; i < nk; ++i) out[len++] = kids[i];
        }
    }
    for (int32_t i = 0, j = n - 1; i < j; ++i, --j) { int32_t t = out[i]; out[i] = out[j]; out[j] = t; }
    free(kids); free(seen);
}

/* Level construction on the group order[lo..hi) (Alg. "Construction of
 * levels", Eq. "level"), restricted to the group plus its distance-1 halo
 * unless whole_graph.  Rewrites order[lo..hi) level by level (R3) and
 * returns the number of levels; *lsize receives per-level sizes in the
 * balancing unit and *lrows per-level row counts (caller frees).          */
static int32_t build_levels(osched *S, int32_t lo, int32_t hi, int whole_graph,
                            int64_t **lsize, int32_t **lrows) {
    int32_t st = ++S->stamp;
    for (int32_t p = lo; p < hi; ++p) S->tmark[S->order[p]] = st;
    if (!whole_graph)
        for (int32_t p = lo; p < hi; ++p) {
            int32_t v = S->order[p];
            S->hmark[v] = st;
            for (int64_t e = S->aptr[v]; e < S->aptr[v + 1]; ++e) S->hmark[S->adj[e]] = st;
        }
    int32_t remaining = hi - lo, scan = hi - 1, maxlvl = -1;
    while (remaining > 0) {
        while (S->dmark[S->order[scan]] == st) --scan;       /* R1/R2 */
        int32_t root = S->order[scan];
        if (whole_graph && S->pp) root = pseudo_peripheral(S->n, S->aptr, S->adj, root);
        int32_t lvl = (maxlvl < 0) ? 0 : maxlvl + 2;
        S->dmark[root] = st; S->dist[root] = lvl;
        if (S->tmark[root] == st) --remaining;
        if (lvl > maxlvl) maxlvl = lvl;
        int32_t nc = 1; S->curr[0] = root;
        while (nc > 0) {
            int32_t nn = 0;
            for (int32_t q = 0; q < nc; ++q) {
                int32_t u = S->curr[q];
                for (int64_t e = S->aptr[u]; e < S->aptr[u + 1]; ++e) {
                    int32_t w = S->adj[e];
                    if (!whole_graph && S->hmark[w] != st) continue;
                    if (S->dmark[w] == st) continue;
                    S->dmark[w] = st; S->dist[w] = lvl + 1;
                    if (S->tmark[w] == st) --remaining;
                    S->next[nn++] = w;
                }
            }
            if (nn > 0 && lvl + 1 > maxlvl) maxlvl = lvl + 1;
            int32_t *t = S->curr; S->curr = S->next; S->next = t;
            nc = nn; ++lvl;
        }
    }
    int32_t nlev = 0;
    for (int32_t p = lo; p < hi; ++p)
        if (S->dist[S->order[p]] + 1 > nlev) nlev = S->dist[S->order[p]] + 1;
    int64_t *sz = (int64_t *)calloc((size_t)nlev + 1, sizeof(int64_t));
    int32_t *rows = (int32_t *)calloc((size_t)nlev + 1, sizeof(int32_t));
    int32_t *start = (int32_t *)calloc((size_t)nlev + 1, sizeof(int32_t));
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(hi - lo + 1));
    for (int32_t p = lo; p < hi; ++p) {
        int32_t v = S->order[p], d = S->dist[v];
        rows[d]++; sz[d] += S->vw[v];
    }
    for (int32_t l = 1; l <= nlev; ++l) start[l] = start[l - 1] + rows[l - 1];
    for (int32_t p = lo; p < hi; ++p) {                       /* stable: R3 */
        int32_t v = S->order[p];
        tmp[start[S->dist[v]]++] = v;
    }
    for (int32_t p = lo; p < hi; ++p) { S->order[p] = tmp[p - lo]; S->pos[S->order[p]] = p; }
    free(tmp); free(start);
    *lsize = sz; *lrows = rows;
    return nlev;
}

/* Sec. 4.4.3 steps 1-3 (R4, R5): pairs of level groups with thread counts.
 * Writes pair boundaries pb[0..np] (level indices) and threads pt[0..np).  */
static int32_t make_pairs(const int64_t *sz, int32_t nlev, int32_t nt, double eps, int32_t k,
                          int32_t *pb, int32_t *pt) {
    int64_t tot = 0;
    for (int32_t l = 0; l < nlev; ++l) tot += sz[l];
    int32_t np = 0, start = 0, assigned = 0;
    pb[0] = 0;
    while (start < nlev) {
        int64_t s = 0;
        int32_t end = start, found = 0;
        double a = 0.0, b = 0.0, e = 0.0;
        while (end < nlev) {
            s += sz[end]; ++end;
            a = tot > 0 ? (double)(s * (int64_t)nt) / (double)tot : 0.0;
            b = round(a); if (b < 1.0) b = 1.0;
            e = 1.0 - fabs(a - b);
            if (end - start >= 2 * k && e > eps) { found = 1; break; }
        }
        if (!found) {                      /* rest joins the last pair (R5) */
            if (np > 0) { assigned -= pt[np - 1]; pt[np - 1] = nt - assigned; pb[np] = nlev; }
            else { pt[0] = nt; pb[1] = nlev; np = 1; }
            return np;
        }
        int32_t best_end = end; double best_e = e;
        while (end < nlev) {
            s += sz[end]; ++end;
            double a2 = (double)(s * (int64_t)nt) / (double)tot;
            if (a2 > b) break;
            double e2 = 1.0 - fabs(a2 - b);
            if (e2 > best_e) { best_e = e2; best_end = end; }
        }
        int32_t bi = (int32_t)b;
        if (nlev - best_end < 2 * k || assigned + bi >= nt) {
            pt[np] = nt - assigned; pb[np + 1] = nlev; ++np;
            return np;
        }
        pt[np] = bi; pb[np + 1] = best_end; ++np;
        assigned += bi; start = best_end;
    }
    return np;
}

typedef struct { double key; int32_t idx; } kv;
static int cmp_kv(const void *a, const void *b) {
    const kv *x = (const kv *)a, *y = (const kv *)b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

static double lb_variance(const int64_t *pre, const int32_t *tp, const int32_t *worker, int32_t len,
                          double *diff) {
    int64_t tot[2] = {0, 0}, wk[2] = {0, 0};
    for (int32_t i = 0; i < len; ++i) { tot[i & 1] += pre[tp[i + 1]] - pre[tp[i]]; wk[i & 1] += worker[i]; }
    double mean[2];
    for (int c = 0; c < 2; ++c) mean[c] = wk[c] > 0 ? (double)tot[c] / (double)wk[c] : 0.0;
    double var = 0.0;
    for (int32_t i = 0; i < len; ++i) {
        double u = (double)(pre[tp[i + 1]] - pre[tp[i]]) / (double)worker[i];
        diff[i] = u - mean[i & 1];
        var += diff[i] * diff[i];
    }
    return var / (double)len;
}

static void lb_shift(int32_t *tp, int32_t src, int32_t dst) {
    if (src > dst) for (int32_t j = dst + 1; j <= src; ++j) tp[j] += 1;
    else for (int32_t j = src + 1; j <= dst; ++j) tp[j] -= 1;
}

/* Alg. "Load Balancing" with worker weights (R7). tp has len+1 entries.   */
static void load_balance(const int64_t *sz, int32_t nlev, int32_t *tp, const int32_t *worker,
                         int32_t len, int32_t k) {
    int64_t *pre = (int64_t *)malloc(sizeof(int64_t) * ((size_t)nlev + 1));
    pre[0] = 0;
    for (int32_t l = 0; l < nlev; ++l) pre[l + 1] = pre[l] + sz[l];
    double *diff = (double *)malloc(sizeof(double) * (size_t)len);
    double *diff2 = (double *)malloc(sizeof(double) * (size_t)len);
    int32_t *absRank = (int32_t *)malloc(sizeof(int32_t) * (size_t)len);
    int32_t *rank = (int32_t *)malloc(sizeof(int32_t) * (size_t)len);
    int32_t *old = (int32_t *)malloc(sizeof(int32_t) * ((size_t)len + 1));
    kv *srt = (kv *)malloc(sizeof(kv) * (size_t)len);
    for (;;) {
        double var = lb_variance(pre, tp, worker, len, diff);
        for (int32_t i = 0; i < len; ++i) { srt[i].key = -fabs(diff[i]); srt[i].idx = i; }
        qsort(srt, (size_t)len, sizeof(kv), cmp_kv);
        for (int32_t i = 0; i < len; ++i) absRank[i] = srt[i].idx;
        for (int32_t i = 0; i < len; ++i) { srt[i].key = diff[i]; srt[i].idx = i; }
        qsort(srt, (size_t)len, sizeof(kv), cmp_kv);
        for (int32_t i = 0; i < len; ++i) rank[i] = srt[i].idx;
        memcpy(old, tp, sizeof(int32_t) * ((size_t)len + 1));
        int32_t currRank = 0;
        double newVar = var;
        int improved = 0;
        while (newVar >= var) {
            memcpy(tp, old, sizeof(int32_t) * ((size_t)len + 1));
            int fail = 1;
            int32_t t = absRank[currRank];
            if (diff[t] < 0.0) {
                for (int32_t q = len - 1; q >= 0; --q) {
                    int32_t el = rank[q];
                    if (el != t && tp[el + 1] - tp[el] > k) { lb_shift(tp, el, t); fail = 0; break; }
                }
            } else if (tp[t + 1] - tp[t] > k) {
                int32_t g = rank[0];
                if (g != t) { lb_shift(tp, t, g); fail = 0; }
            }
            if (!fail) newVar = lb_variance(pre, tp, worker, len, diff2);
            if (currRank == len - 1 && newVar >= var) {
                memcpy(tp, old, sizeof(int32_t) * ((size_t)len + 1));
                break;
            }
            if (newVar < var) { improved = 1; break; }
            ++currRank;
        }
        if (!improved) break;
    }
    free(pre); free(diff); free(diff2); free(absRank); free(rank); free(old); free(srt);
}

/* Split node id (Sec. 4.4.3) and recurse into children with > 1 thread.   */
static void split_node(osched *S, int32_t id) {
    onode nd = S->nodes[id];
    int whole = (nd.parent < 0);
    int64_t *sz; int32_t *rows;
    int32_t nlev = build_levels(S, nd.lo, nd.hi, whole, &sz, &rows);
    S->nodes[id].nsub = nlev;
    /* levels per group: k (= 2); one level at stage 0 when asked (R10) */
    int32_t k = (whole && S->one0) ? 1 : S->k;
    if (nlev < 2 * k) { free(sz); free(rows); return; }
    int32_t s = nd.stage + 1;
    double eps = S->eps[s < 8 ? s : 7];
    int32_t *pb = (int32_t *)malloc(sizeof(int32_t) * ((size_t)nlev + 2));
    int32_t *pt = (int32_t *)malloc(sizeof(int32_t) * ((size_t)nlev + 2));
    int32_t np = make_pairs(sz, nlev, nd.nthreads, eps, k, pb, pt);
    int32_t len = 2 * np;
    int32_t *tp = (int32_t *)malloc(sizeof(int32_t) * ((size_t)len + 1));
    int32_t *worker = (int32_t *)malloc(sizeof(int32_t) * (size_t)len);
    for (int32_t p = 0; p < np; ++p) {
        int32_t n_l = pb[p + 1] - pb[p];
        tp[2 * p] = pb[p]; tp[2 * p + 1] = pb[p] + n_l / 2;           /* R6 */
        worker[2 * p] = worker[2 * p + 1] = pt[p];
    }
    tp[len] = nlev;
    load_balance(sz, nlev, tp, worker, len, k);
    /* children, in level order */
    int32_t first = S->nnodes;
    int32_t row0 = nd.lo, thr = nd.thread_lo;
    for (int32_t g = 0; g < len; ++g) {
        int32_t c = new_node(S);
        onode *cn = &S->nodes[c];
        int32_t r = 0; int64_t w = 0;
        for (int32_t l = tp[g]; l < tp[g + 1]; ++l) { r += rows[l]; w += sz[l]; }
        cn->parent = id; cn->stage = s; cn->color = g & 1;
        cn->lo = row0; cn->hi = row0 + r; row0 += r;
        cn->nthreads = worker[g]; cn->thread_lo = thr;
        if (g & 1) thr += worker[g];
        cn->nlev = tp[g + 1] - tp[g]; cn->size = w;
    }
    S->nodes[id].first_child = first;
    S->nodes[id].nchildren = len;
    free(sz); free(rows); free(pb); free(pt); free(tp); free(worker);
    for (int32_t g = 0; g < len; ++g) {                                     /* R8 */
        onode cn = S->nodes[first + g];
        int allowed = (S->max_depth < 0) || (cn.stage + 1 < S->max_depth);
        if (cn.nthreads > 1 && allowed && cn.hi > cn.lo) split_node(S, first + g);
    }
}

/* Sec. 5: effective row count and phase counts (R9), bottom-up.           */
static void tree_metrics(osched *S, int32_t id) {
    onode *nd = &S->nodes[id];
    if (nd->nchildren == 0) { nd->neff = nd->size; nd->phase_count = 1; return; }
    int64_t mr = 0, mb = 0; int32_t pr = 0, pbk = 0;
    for (int32_t g = 0; g < nd->nchildren; ++g) {
        int32_t c = nd->first_child + g;
        tree_metrics(S, c);
        onode *cn = &S->nodes[c];
        if (cn->color == 0) { if (cn->neff > mr) mr = cn->neff; if (cn->phase_count > pr) pr = cn->phase_count; }
        else { if (cn->neff > mb) mb = cn->neff; if (cn->phase_count > pbk) pbk = cn->phase_count; }
    }
    nd = &S->nodes[id];
    nd->neff = mr + mb;
    nd->phase_count = pr + pbk;
}

static void assign_offsets(osched *S, int32_t id, int32_t off) {
    onode *nd = &S->nodes[id];
    nd->phase_off = off;
    if (nd->nchildren == 0) return;
    int32_t pr = 0;
    for (int32_t g = 0; g < nd->nchildren; ++g) {
        onode *cn = &S->nodes[nd->first_child + g];
        if (cn->color == 0 && cn->phase_count > pr) pr = cn->phase_count;
    }
    int32_t fc = nd->first_child, nc = nd->nchildren;
    for (int32_t g = 0; g < nc; ++g) {
        int32_t c = fc + g;
        assign_offsets(S, c, S->nodes[c].color == 0 ? off : off + pr);
    }
}

typedef struct { int32_t phase, lo, node; } leafkey;
static int cmp_leaf(const void *a, const void *b) {
    const leafkey *x = (const leafkey *)a, *y = (const leafkey *)b;
    if (x->phase != y->phase) return (x->phase > y->phase) - (x->phase < y->phase);
    return (x->lo > y->lo) - (x->lo < y->lo);
}

void orc_race_free(osched *S);

int orc_permute_upper(int32_t n, const int32_t *rp, const int32_t *ci, const double *va,
                      const int32_t *perm, int32_t *orp, int32_t *oci, double *ova);
int32_t orc_rcm_order(int32_t n, const int32_t *rp, const int32_t *ci, int32_t *order);

/* options: bit 0 = pseudo-peripheral stage-0 roots, bit 1 = RCM relabelling
 * first, bit 2 = stage-0 groups of one level (R10; see the readings).     */
osched *orc_race(int32_t n, const int32_t *rp, const int32_t *ci, int32_t nt, const double *eps8,
                 int32_t max_depth, int32_t balance, int32_t options) {
    if (n <= 0 || nt <= 0) return NULL;
    if (options & 2) {
        /* build on the RCM-relabelled matrix, then compose the permutations */
        int64_t nnz = rp[n];
        int32_t *ord = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
        int32_t *prp = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
        int32_t *pci = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
        double *zero = (double *)calloc((size_t)(nnz > 0 ? nnz : 1), sizeof(double));
        double *pva = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
        orc_rcm_order(n, rp, ci, ord);
        orc_permute_upper(n, rp, ci, zero, ord, prp, pci, pva);
        osched *S = orc_race(n, prp, pci, nt, eps8, max_depth, balance, options & ~2);
        if (S) {
            for (int32_t i = 0; i < n; ++i) S->order[i] = ord[S->order[i]];
            for (int32_t i = 0; i < n; ++i) S->pos[S->order[i]] = i;
        }
        free(ord); free(prp); free(pci); free(zero); free(pva);
        return S;
    }
    osched *S = (osched *)calloc(1, sizeof(osched));
    S->n = n; S->nt = nt; S->k = 2; S->balance = balance; S->max_depth = max_depth;
    S->pp = (options & 1) != 0;
    S->one0 = (options & 4) != 0;
    for (int i = 0; i < 8; ++i) S->eps[i] = eps8[i];
    /* symmetric adjacency (self loops dropped, Sec. 4 graph definitions) */
    S->aptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    for (int32_t i = 0; i < n; ++i)
        for (int32_t t = rp[i]; t < rp[i + 1]; ++t)
            if (ci[t] != i) { S->aptr[i + 1]++; S->aptr[ci[t] + 1]++; }
    for (int32_t i = 0; i < n; ++i) S->aptr[i + 1] += S->aptr[i];
    S->adj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(S->aptr[n] > 0 ? S->aptr[n] : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    memcpy(fill, S->aptr, sizeof(int64_t) * (size_t)n);
    for (int32_t i = 0; i < n; ++i)
        for (int32_t t = rp[i]; t < rp[i + 1]; ++t)
            if (ci[t] != i) { S->adj[fill[i]++] = ci[t]; S->adj[fill[ci[t]]++] = i; }
    free(fill);
    S->vw = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    for (int32_t i = 0; i < n; ++i)
        S->vw[i] = balance ? 1 + (S->aptr[i + 1] - S->aptr[i]) : 1;
    S->order = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    S->pos = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    for (int32_t i = 0; i < n; ++i) { S->order[i] = i; S->pos[i] = i; }
    S->dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    S->tmark = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    S->hmark = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    S->dmark = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    S->curr = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    S->next = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    /* root node T_{-1}(0): all vertices, all threads */
    int32_t r = new_node(S);
    S->nodes[r].parent = -1; S->nodes[r].stage = -1; S->nodes[r].color = 0;
    S->nodes[r].lo = 0; S->nodes[r].hi = n; S->nodes[r].nthreads = nt;
    int64_t tot = 0;
    for (int32_t i = 0; i < n; ++i) tot += S->vw[i];
    S->nodes[r].size = tot;
    if (max_depth != 0) split_node(S, r);
    tree_metrics(S, r);
    assign_offsets(S, r, 0);
    S->eta = (double)tot / ((double)S->nodes[r].neff * (double)nt);
    /* flatten: non-empty leaves sorted by (phase, first row) */
    int32_t nl = 0;
    for (int32_t i = 0; i < S->nnodes; ++i)
        if (S->nodes[i].nchildren == 0 && S->nodes[i].hi > S->nodes[i].lo) ++nl;
    leafkey *lk = (leafkey *)malloc(sizeof(leafkey) * (size_t)(nl > 0 ? nl : 1));
    nl = 0;
    for (int32_t i = 0; i < S->nnodes; ++i)
        if (S->nodes[i].nchildren == 0 && S->nodes[i].hi > S->nodes[i].lo) {
            lk[nl].phase = S->nodes[i].phase_off; lk[nl].lo = S->nodes[i].lo; lk[nl].node = i; ++nl;
        }
    qsort(lk, (size_t)nl, sizeof(leafkey), cmp_leaf);
    S->nphases = S->nodes[r].phase_count;
    S->nleaves = nl;
    S->stage_ptr = (int32_t *)calloc((size_t)S->nphases + 1, sizeof(int32_t));
    S->leaf_lo = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nl > 0 ? nl : 1));
    S->leaf_hi = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nl > 0 ? nl : 1));
    S->leaf_node = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nl > 0 ? nl : 1));
    for (int32_t q = 0; q < nl; ++q) {
        S->leaf_lo[q] = lk[q].lo; S->leaf_hi[q] = S->nodes[lk[q].node].hi; S->leaf_node[q] = lk[q].node;
        S->stage_ptr[lk[q].phase + 1]++;
    }
    for (int32_t p = 0; p < S->nphases; ++p) S->stage_ptr[p + 1] += S->stage_ptr[p];
    free(lk);
    /* scratch no longer needed */
    free(S->dist); free(S->tmark); free(S->hmark); free(S->dmark); free(S->curr); free(S->next);
    S->dist = S->tmark = S->hmark = S->dmark = S->curr = S->next = NULL;
    return S;
}

void orc_race_free(osched *S) {
    if (!S) return;
    free(S->aptr); free(S->adj); free(S->vw); free(S->order); free(S->pos);
    free(S->dist); free(S->tmark); free(S->hmark); free(S->dmark); free(S->curr); free(S->next);
    free(S->nodes); free(S->stage_ptr); free(S->leaf_lo); free(S->leaf_hi); free(S->leaf_node);
    free(S);
}

/* ---- accessors ---------------------------------------------------------- */
void orc_race_info(const osched *S, int32_t *info /* 6 */, double *eta) {
    info[0] = S->n; info[1] = S->nt; info[2] = S->nnodes; info[3] = S->nphases; info[4] = S->nleaves;
    int32_t depth = 0;
    for (int32_t i = 0; i < S->nnodes; ++i) if (S->nodes[i].stage + 1 > depth) depth = S->nodes[i].stage + 1;
    info[5] = depth;
    *eta = S->eta;
}
void orc_race_perm(const osched *S, int32_t *perm) { memcpy(perm, S->order, sizeof(int32_t) * (size_t)S->n); }
void orc_race_phases(const osched *S, int32_t *stage_ptr, int32_t *lo, int32_t *hi, int32_t *node) {
    memcpy(stage_ptr, S->stage_ptr, sizeof(int32_t) * ((size_t)S->nphases + 1));
    memcpy(lo, S->leaf_lo, sizeof(int32_t) * (size_t)S->nleaves);
    memcpy(hi, S->leaf_hi, sizeof(int32_t) * (size_t)S->nleaves);
    memcpy(node, S->leaf_node, sizeof(int32_t) * (size_t)S->nleaves);
}
/* node table, in creation order: 13 int32 + 2 int64 per node, unpacked   */
void orc_race_nodes(const osched *S, int32_t *i32 /* 13*nnodes */, int64_t *i64 /* 2*nnodes */) {
    for (int32_t i = 0; i < S->nnodes; ++i) {
        const onode *d = &S->nodes[i];
        int32_t *o = i32 + 13 * (size_t)i;
        o[0] = d->parent; o[1] = d->stage; o[2] = d->color; o[3] = d->lo; o[4] = d->hi;
        o[5] = d->nthreads; o[6] = d->thread_lo; o[7] = d->nlev; o[8] = d->nsub;
        o[9] = d->first_child; o[10] = d->nchildren; o[11] = d->phase_count; o[12] = d->phase_off;
        i64[2 * (size_t)i] = d->size; i64[2 * (size_t)i + 1] = d->neff;
    }
}

/* ---- canonical export (byte layout documented with race_export) -------- */
static void put32(uint8_t **p, int32_t v) { memcpy(*p, &v, 4); *p += 4; }
static void put64(uint8_t **p, int64_t v) { memcpy(*p, &v, 8); *p += 8; }
static void putd(uint8_t **p, double v) { memcpy(*p, &v, 8); *p += 8; }

static void export_node(const osched *S, int32_t id, uint8_t **p) {
    const onode *d = &S->nodes[id];
    put32(p, d->stage); put32(p, d->color); put32(p, d->lo); put32(p, d->hi);
    put32(p, d->nthreads); put32(p, d->thread_lo); put32(p, d->nlev); put32(p, d->nsub);
    put32(p, d->nchildren); put32(p, d->phase_count); put32(p, d->phase_off);
    put64(p, d->size); put64(p, d->neff);
    for (int32_t g = 0; g < d->nchildren; ++g) export_node(S, d->first_child + g, p);
}

int64_t orc_race_export(const osched *S, uint8_t *buf) {
    int64_t sz = 4 * 12 + 8 * 9 + 4 * (int64_t)S->n + 4 * ((int64_t)S->nphases + 1) +
                 8 * (int64_t)S->nleaves + (int64_t)S->nnodes * (11 * 4 + 2 * 8);
    if (!buf) return sz;
    uint8_t *p = buf;
    put32(&p, 0x45434152); put32(&p, 1);
    put32(&p, S->n); put32(&p, S->nt); put32(&p, S->k); put32(&p, S->balance);
    put32(&p, S->max_depth); put32(&p, S->nnodes); put32(&p, S->nphases); put32(&p, S->nleaves);
    put32(&p, 0); put32(&p, 0);
    for (int i = 0; i < 8; ++i) putd(&p, S->eps[i]);
    putd(&p, S->eta);
    for (int32_t i = 0; i < S->n; ++i) put32(&p, S->order[i]);
    for (int32_t i = 0; i <= S->nphases; ++i) put32(&p, S->stage_ptr[i]);
    for (int32_t i = 0; i < S->nleaves; ++i) { put32(&p, S->leaf_lo[i]); put32(&p, S->leaf_hi[i]); }
    export_node(S, 0, &p);
    return (int64_t)(p - buf);
}

/* Permuted upper CRS (Sec. 4.1: rows and columns permuted symmetrically):
 * entry (i,j,a) of the input lands in row min(P(i),P(j)), column max(...),
 * columns increasing (the diagonal therefore first).  Output arrays hold
 * nnz_u entries.                                                          */
int orc_permute_upper(int32_t n, const int32_t *rp, const int32_t *ci, const double *va,
                      const int32_t *perm, int32_t *orp, int32_t *oci, double *ova) {
    int32_t *newpos = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!newpos || !cnt) { free(newpos); free(cnt); return -1; }
    for (int32_t p = 0; p < n; ++p) newpos[perm[p]] = p;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t t = rp[i]; t < rp[i + 1]; ++t) {
            int32_t a = newpos[i], b = newpos[ci[t]];
            cnt[(a < b ? a : b) + 1]++;
        }
    for (int32_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
    for (int32_t i = 0; i <= n; ++i) orp[i] = (int32_t)cnt[i];
    for (int32_t i = 0; i < n; ++i)
        for (int32_t t = rp[i]; t < rp[i + 1]; ++t) {
            int32_t a = newpos[i], b = newpos[ci[t]];
            int32_t r = a < b ? a : b, c = a < b ? b : a;
            oci[cnt[r]] = c; ova[cnt[r]] = va[t]; cnt[r]++;
        }
    /* insertion sort per row (rows are short) */
    for (int32_t r = 0; r < n; ++r)
        for (int32_t t = orp[r] + 1; t < orp[r + 1]; ++t) {
            int32_t c = oci[t]; double v = ova[t]; int32_t u = t - 1;
            while (u >= orp[r] && oci[u] > c) { oci[u + 1] = oci[u]; ova[u + 1] = ova[u]; --u; }
            oci[u + 1] = c; ova[u + 1] = v;
        }
    free(newpos); free(cnt);
    return 0;
}

/* Conflict check of a flattened schedule on the permuted upper CRS: every
 * row in exactly one leaf, and within a phase the write sets
 * {rows of the leaf} U {upper columns of those rows} pairwise disjoint.
 * Returns 0 if valid, 1 = row coverage broken, 2 = write conflict.        */
int orc_check_phases(int32_t n, const int32_t *prp, const int32_t *pci, int32_t nphases,
                     const int32_t *stage_ptr, const int32_t *lo, const int32_t *hi) {
    int32_t *cover = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    int32_t *owner = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *ophase = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int rc = 0;
    for (int32_t i = 0; i < n; ++i) { owner[i] = -1; ophase[i] = -1; }
    for (int32_t ph = 0; ph < nphases && !rc; ++ph)
        for (int32_t q = stage_ptr[ph]; q < stage_ptr[ph + 1] && !rc; ++q)
            for (int32_t r = lo[q]; r < hi[q] && !rc; ++r) {
                if (r < 0 || r >= n) { rc = 1; break; }
                cover[r]++;
                for (int32_t t = prp[r]; t < prp[r + 1]; ++t) {
                    int32_t c = pci[t];
                    if (ophase[c] == ph && owner[c] != q) { rc = 2; break; }
                    ophase[c] = ph; owner[c] = q;
                }
            }
    for (int32_t i = 0; i < n && !rc; ++i) if (cover[i] != 1) rc = 1;
    free(cover); free(owner); free(ophase);
    return rc;
}

/* Symmetric Gauss-Seidel under a flattened schedule (R11: the paper names
 * Gauss-Seidel among the kernels with distance-k dependencies that RACE
 * schedules serve).  One sweep = a forward pass, phases in order, the rows of every leaf in
 * ascending order, then a backward pass, phases in reverse order, the rows
 * of every leaf in descending order; each row update
 *     x_i <- (b_i - sum_{j != i} a_ij x_j) / a_ii
 * reads the current x.  Leaves of a phase share no edge (the schedules are
 * distance-2 colourings, stronger than the distance 1 Gauss-Seidel needs),
 * so the leaf order inside a phase does not change the result.  Full CRS
 * (frp int64) of the matrix in the schedule's order; x updated in place.  */
void orc_symm_gs(int32_t n, const int64_t *frp, const int32_t *fci, const double *fva, int32_t nphases,
                 const int32_t *stage_ptr, const int32_t *lo, const int32_t *hi, const double *b, double *x,
                 int32_t sweeps) {
    (void)n;
    for (int32_t sw = 0; sw < sweeps; ++sw) {
        for (int32_t dir = 0; dir < 2; ++dir)
            for (int32_t pi = 0; pi < nphases; ++pi) {
                int32_t ph = dir == 0 ? pi : nphases - 1 - pi;
                for (int32_t q = stage_ptr[ph]; q < stage_ptr[ph + 1]; ++q)
                    for (int32_t k = 0; k < hi[q] - lo[q]; ++k) {
                        int32_t r = dir == 0 ? lo[q] + k : hi[q] - 1 - k;
                        double s = b[r], d = 0.0;
                        for (int64_t t = frp[r]; t < frp[r + 1]; ++t) {
                            if (fci[t] == r) d += fva[t];
                            else s -= fva[t] * x[fci[t]];
                        }
                        x[r] = s / d;
                    }
            }
    }
}

/* Symmetric Kaczmarz under a flattened schedule (R12: the paper names the
 * Kaczmarz solver among the kernels RACE serves).  Same passes as
 * orc_symm_gs; a row update projects x onto the row's hyperplane,
 *     f = (b_i - sum_j a_ij x_j) / sum_j a_ij^2,   x_j <- x_j + f a_ij  (all j),
 * so it writes x at every column of the row: rows of concurrent leaves must
 * share no column, which distance-2 independence gives.                   */
void orc_symm_kacz(int32_t n, const int64_t *frp, const int32_t *fci, const double *fva, int32_t nphases,
                   const int32_t *stage_ptr, const int32_t *lo, const int32_t *hi, const double *b, double *x,
                   int32_t sweeps) {
    (void)n;
    for (int32_t sw = 0; sw < sweeps; ++sw) {
        for (int32_t dir = 0; dir < 2; ++dir)
            for (int32_t pi = 0; pi < nphases; ++pi) {
                int32_t ph = dir == 0 ? pi : nphases - 1 - pi;
                for (int32_t q = stage_ptr[ph]; q < stage_ptr[ph + 1]; ++q)
                    for (int32_t k = 0; k < hi[q] - lo[q]; ++k) {
                        int32_t r = dir == 0 ? lo[q] + k : hi[q] - 1 - k;
                        double dot = 0.0, nrm = 0.0;
                        for (int64_t t = frp[r]; t < frp[r + 1]; ++t) {
                            dot += fva[t] * x[fci[t]];
                            nrm += fva[t] * fva[t];
                        }
                        double f = (b[r] - dot) / nrm;
                        for (int64_t t = frp[r]; t < frp[r + 1]; ++t) x[fci[t]] += f * fva[t];
                    }
            }
    }
}

/* Multicolouring schedules (R14: the paper's comparison methods, Sec. 3.3
 * and 6.3).  Units: rows (method 0, MC) or blocks of block_rows consecutive
 * rows (method 1, ABMC).  A unit takes the smallest colour not held by an
 * earlier unit that has a row within graph distance 2 of one of its rows
 * (distance in the symmetric graph, self-loops ignored).  Output: perm
 * (units colour by colour, units and their rows in order), stage_ptr (one
 * phase per colour, n_colours + 1 offsets into the leaves), leaf_lo/hi (one
 * leaf per unit, positions in the permuted order).  Returns the number of
 * colours; *n_leaves gets the number of units.                            */
int32_t orc_coloring(int32_t n, const int32_t *rp, const int32_t *ci, int32_t method, int32_t block_rows,
                     int32_t *perm, int32_t *stage_ptr, int32_t *leaf_lo, int32_t *leaf_hi, int32_t *n_leaves) {
    const int32_t bs = method == 0 ? 1 : block_rows;
    const int32_t units = (n + bs - 1) / bs;
    int64_t *aptr = calloc((size_t)n + 1, sizeof(int64_t));
    for (int32_t r = 0; r < n; ++r)
        for (int32_t t = rp[r]; t < rp[r + 1]; ++t)
            if (ci[t] != r) { aptr[r + 1]++; aptr[ci[t] + 1]++; }
    for (int32_t r = 0; r < n; ++r) aptr[r + 1] += aptr[r];
    int32_t *adj = malloc(sizeof(int32_t) * (size_t)(aptr[n] > 0 ? aptr[n] : 1));
    int64_t *pos = malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int32_t r = 0; r < n; ++r) pos[r] = aptr[r];
    for (int32_t r = 0; r < n; ++r)
        for (int32_t t = rp[r]; t < rp[r + 1]; ++t)
            if (ci[t] != r) { adj[pos[r]++] = ci[t]; adj[pos[ci[t]]++] = r; }
    int32_t *color = malloc(sizeof(int32_t) * (size_t)(units > 0 ? units : 1));
    /* used[c] != 0: colour c is held by an earlier unit near the current one */
    uint8_t *used = calloc((size_t)units + 1, 1);
    int32_t *seen = malloc(sizeof(int32_t) * (size_t)(units + 1));
    int32_t nseen, ncol = 0;
    for (int32_t u = 0; u < units; ++u) {
        nseen = 0;
        int32_t r1 = (u + 1) * bs < n ? (u + 1) * bs : n;
        for (int32_t r = u * bs; r < r1; ++r) {
            /* rows within distance 0, 1 and 2 of r */
            for (int64_t a = aptr[r] - 1; a < aptr[r + 1]; ++a) {
                int32_t w = a < aptr[r] ? r : adj[a];
                for (int64_t b = aptr[w] - 1; b < aptr[w + 1]; ++b) {
                    int32_t v = b < aptr[w] ? w : adj[b];
                    int32_t vu = v / bs;
                    if (vu < u && !used[color[vu]]) { used[color[vu]] = 1; seen[nseen++] = color[vu]; }
                }
            }
        }
        int32_t c = 0;
        while (used[c]) ++c;
        color[u] = c;
        if (c + 1 > ncol) ncol = c + 1;
        for (int32_t k = 0; k < nseen; ++k) used[seen[k]] = 0;
    }
    int32_t q = 0, row = 0;
    for (int32_t c = 0; c < ncol; ++c) {
        stage_ptr[c] = q;
        for (int32_t u = 0; u < units; ++u) {
            if (color[u] != c) continue;
            int32_t r1 = (u + 1) * bs < n ? (u + 1) * bs : n;
            leaf_lo[q] = row;
            for (int32_t r = u * bs; r < r1; ++r) perm[row++] = r;
            leaf_hi[q++] = row;
        }
    }
    stage_ptr[ncol] = q;
    *n_leaves = q;
    free(aptr); free(adj); free(pos); free(color); free(used); free(seen);
    return ncol;
}

/* The pseudo-peripheral vertex reached from `start` on the symmetric graph
 * of an upper CRS (self loops dropped).                                   */
int32_t orc_pseudo_peripheral(int32_t n, const int32_t *rp, const int32_t *ci, int32_t start) {
    int64_t *aptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    for (int32_t i = 0; i < n; ++i)
        for (int32_t t = rp[i]; t < rp[i + 1]; ++t)
            if (ci[t] != i) { aptr[i + 1]++; aptr[ci[t] + 1]++; }
    for (int32_t i = 0; i < n; ++i) aptr[i + 1] += aptr[i];
    int32_t *adj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(aptr[n] > 0 ? aptr[n] : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    memcpy(fill, aptr, sizeof(int64_t) * (size_t)n);
    for (int32_t i = 0; i < n; ++i)
        for (int32_t t = rp[i]; t < rp[i + 1]; ++t)
            if (ci[t] != i) { adj[fill[i]++] = ci[t]; adj[fill[ci[t]]++] = i; }
    int32_t r = pseudo_peripheral(n, aptr, adj, start);
    free(fill); free(adj); free(aptr);
    return r;
}

/* Reverse Cuthill-McKee order (order[new] = old) of the symmetric graph of
 * an upper CRS; returns n.                                                 */
int32_t orc_rcm_order(int32_t n, const int32_t *rp, const int32_t *ci, int32_t *order) {
    int64_t *aptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    for (int32_t i = 0; i < n; ++i)
        for (int32_t t = rp[i]; t < rp[i + 1]; ++t)
            if (ci[t] != i) { aptr[i + 1]++; aptr[ci[t] + 1]++; }
    for (int32_t i = 0; i < n; ++i) aptr[i + 1] += aptr[i];
    int32_t *adj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(aptr[n] > 0 ? aptr[n] : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    memcpy(fill, aptr, sizeof(int64_t) * (size_t)n);
    for (int32_t i = 0; i < n; ++i)
        for (int32_t t = rp[i]; t < rp[i + 1]; ++t)
            if (ci[t] != i) { adj[fill[i]++] = ci[t]; adj[fill[ci[t]]++] = i; }
    rcm_sequence(n, aptr, adj, order);
    free(fill); free(adj); free(aptr);
    return n;
}

/* Plain BFS distances on the whole graph from one root (Eq. "level").    */
int orc_bfs_dist(int32_t n, const int32_t *rp, const int32_t *ci, int32_t root, int32_t *dist) {
    int64_t *aptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    for (int32_t i = 0; i < n; ++i)
        for (int32_t t = rp[i]; t < rp[i + 1]; ++t)
            if (ci[t] != i) { aptr[i + 1]++; aptr[ci[t] + 1]++; }
    for (int32_t i = 0; i < n; ++i) aptr[i + 1] += aptr[i];
    int32_t *adj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(aptr[n] + 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    memcpy(fill, aptr, sizeof(int64_t) * (size_t)n);
    for (int32_t i = 0; i < n; ++i)
        for (int32_t t = rp[i]; t < rp[i + 1]; ++t)
            if (ci[t] != i) { adj[fill[i]++] = ci[t]; adj[fill[ci[t]]++] = i; }
    int32_t *q = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    for (int32_t i = 0; i < n; ++i) dist[i] = -1;
    int64_t h = 0, t = 0;
    dist[root] = 0; q[t++] = root;
    while (h < t) {
        int32_t u = q[h++];
        for (int64_t e = aptr[u]; e < aptr[u + 1]; ++e)
            if (dist[adj[e]] < 0) { dist[adj[e]] = dist[u] + 1; q[t++] = adj[e]; }
    }
    free(aptr); free(adj); free(fill); free(q);
    return 0;
}
