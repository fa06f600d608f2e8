/*
 * Seeded synthetic inputs for the SymmSpMV library and its oracle.
 *
 * This module only *generates* inputs: symmetric matrices in upper-triangle
 * CRS (diagonal stored first in each row, then strictly increasing columns)
 * and dense vectors.  It contains none of the method's arithmetic (no
 * products, no levels, no schedules), so both the CUDA path and the CPU
 * oracle may consume what it produces.
 *
 * Random numbers: splitmix64 (S. Vigna's public-domain generator, the
 * finaliser of Steele/Lea/Flood "Fast splittable pseudorandom number
 * generators", OOPSLA 2014).  A double in [0,1) is the top 53 bits / 2^53.
 *
 * Matrix families (stand-ins for the paper's SuiteSparse/ScaMaC inputs,
 * Table "Details of the benchmark matrices"):
 *   - 3D Anderson model, periodic 7-point stencil (paper's Anderson-16.5)
 *   - periodic Heisenberg XXZ chain, Sz=0 sector (paper's Spin-26)
 *   - 3D 27-point stencil, nonperiodic, SPD by diagonal dominance
 *   - 3D 7-point stencil, nonperiodic
 *   - random geometric graph Laplacian-like matrices (diag = sum w + 1)
 *   - random symmetric banded matrices
 *   - the 2D "artificial stencil" of the paper's RACE walk-through
 *     (Section 4, 5-point star plus the (+2,-2)/(-2,+2) anti-diagonal pair)
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef struct {
    int32_t n;
    int64_t nnz;        /* stored upper entries incl. diagonal */
    int32_t *row_ptr;   /* n+1 (int32: every generated nnz < 2^31) */
    int32_t *col;       /* nnz */
    double *val;        /* nnz */
} mg_csr;

static inline uint64_t sm64_next(uint64_t *s) {
    uint64_t z = (*s += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}
static inline double sm64_u01(uint64_t *s) { /* [0,1) */
    return (double)(sm64_next(s) >> 11) * 0x1.0p-53;
}

void mg_free(mg_csr *m) {
    if (!m) return;
    free(m->row_ptr); free(m->col); free(m->val);
    m->row_ptr = NULL; m->col = NULL; m->val = NULL;
}

static int mg_alloc(mg_csr *m, int32_t n, int64_t cap) {
    m->n = n; m->nnz = 0;
    m->row_ptr = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    m->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(cap > 0 ? cap : 1));
    m->val = (double *)malloc(sizeof(double) * (size_t)(cap > 0 ? cap : 1));
    if (!m->row_ptr || !m->col || !m->val) { mg_free(m); return -1; }
    return 0;
}

/* x[i] = lo + (hi-lo)*u, u in [0,1), drawn in index order. */
void mg_uniform(int64_t n, uint64_t seed, double lo, double hi, double *x) {
    uint64_t s = seed;
    for (int64_t i = 0; i < n; ++i) x[i] = lo + (hi - lo) * sm64_u01(&s);
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* ---------------------------------------------------------------------- */
/* 3D Anderson model: L^3 periodic, 7-point, lexicographic i=(x*L+y)*L+z.   */
/* Off-diagonals -1, diagonal uniform in [-W/2, W/2).  Requires L >= 3.     */
int mg_anderson(int32_t L, double W, uint64_t seed, mg_csr *m) {
    if (L < 3) return -1;
    int64_t n64 = (int64_t)L * L * L;
    if (n64 >= INT32_MAX) return -1;
    int32_t n = (int32_t)n64;
    if (mg_alloc(m, n, 4 * n64)) return -2;
    uint64_t s = seed;
    int64_t k = 0;
    for (int32_t x = 0; x < L; ++x)
        for (int32_t y = 0; y < L; ++y)
            for (int32_t z = 0; z < L; ++z) {
                int32_t i = (x * L + y) * L + z;
                m->row_ptr[i] = (int32_t)k;
                m->col[k] = i;
                m->val[k] = -0.5 * W + W * sm64_u01(&s);
                ++k;
                int32_t nb[6] = {
                    (((x + 1) % L) * L + y) * L + z, (((x + L - 1) % L) * L + y) * L + z,
                    (x * L + (y + 1) % L) * L + z,   (x * L + (y + L - 1) % L) * L + z,
                    (x * L + y) * L + (z + 1) % L,   (x * L + y) * L + (z + L - 1) % L};
                int32_t up[6]; int cnt = 0;
                for (int t = 0; t < 6; ++t) if (nb[t] > i) up[cnt++] = nb[t];
                qsort(up, (size_t)cnt, sizeof(int32_t), cmp_i32);
                for (int t = 0; t < cnt; ++t) {
                    if (t > 0 && up[t] == up[t - 1]) continue;
                    m->col[k] = up[t]; m->val[k] = -1.0; ++k;
                }
            }
    m->row_ptr[n] = (int32_t)k; m->nnz = k;
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Periodic XXZ chain, L sites, Sz=0 (popcount L/2).  Basis: ascending      */
/* L-bit integers with L/2 set bits, bit i = spin i up.  Index = rank in    */
/* the combinatorial number system (colex order == ascending integers).     */
/* H = J sum_i [ 1/2 (S+_i S-_{i+1} + h.c.) + Delta Sz_i Sz_{i+1} ]:        */
/*   off-diagonal J/2 for each bond whose two spins differ (swap them),     */
/*   diagonal J*Delta*(n_parallel - n_antiparallel)/4.                      */
static int64_t binom_tab[64][64];
static void binom_init(void) {
    static int done = 0;
    if (done) return;
    for (int a = 0; a < 64; ++a) {
        binom_tab[a][0] = 1;
        for (int b = 1; b < 64; ++b)
            binom_tab[a][b] = (a == 0) ? 0 : binom_tab[a - 1][b - 1] + binom_tab[a - 1][b];
    }
    done = 1;
}
static inline int64_t colex_rank(uint64_t s) {
    int64_t r = 0; int i = 1;
    while (s) {
        int p = __builtin_ctzll(s);
        r += binom_tab[p][i];
        ++i; s &= s - 1;
    }
    return r;
}

int mg_xxz(int32_t L, double J, double Delta, mg_csr *m) {
    if (L < 4 || L > 40 || (L & 1)) return -1;
    binom_init();
    int half = L / 2;
    int64_t n64 = binom_tab[L][half];
    if (n64 >= INT32_MAX) return -1;
    int32_t n = (int32_t)n64;
    if (mg_alloc(m, n, n64 * (int64_t)(L / 2 + 2))) return -2;
    /* first state: lowest L/2 bits set; next by Gosper's hack */
    uint64_t s = (1ULL << half) - 1ULL;
    uint64_t maskL = (L == 64) ? ~0ULL : ((1ULL << L) - 1ULL);
    int64_t k = 0;
    int32_t up[64];
    for (int32_t i = 0; i < n; ++i) {
        m->row_ptr[i] = (int32_t)k;
        int npar = 0, nanti = 0, cnt = 0;
        for (int b = 0; b < L; ++b) {
            int b2 = (b + 1) % L;
            int sb = (int)((s >> b) & 1ULL), sb2 = (int)((s >> b2) & 1ULL);
            if (sb == sb2) { ++npar; continue; }
            ++nanti;
            uint64_t t = s ^ ((1ULL << b) | (1ULL << b2));
            int64_t j = colex_rank(t);
            if (j > i) up[cnt++] = (int32_t)j;
        }
        m->col[k] = i; m->val[k] = J * Delta * 0.25 * (double)(npar - nanti); ++k;
        qsort(up, (size_t)cnt, sizeof(int32_t), cmp_i32);
        for (int t = 0; t < cnt; ++t) { m->col[k] = up[t]; m->val[k] = 0.5 * J; ++k; }
        /* Gosper: next integer with the same popcount */
        uint64_t c = s & (~s + 1ULL), r = s + c;
        s = (((r ^ s) >> 2) / c) | r;
        s &= maskL;
    }
    m->row_ptr[n] = (int32_t)k; m->nnz = k;
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Nonperiodic 3D stencil on nx*ny*nz points, lexicographic               */
/* i = (x*ny + y)*nz + z.  npt = 7 (face neighbours) or 27 (full cube).    */
/* Off-diagonals: -U for U uniform in (0,1] per undirected edge, drawn in   */
/* upper-CRS order (offdiag_mode 0), or exactly -1 (offdiag_mode 1).        */
/* Diagonal: sum over the full row of |a_ij| plus diag_shift.               */
int mg_stencil3d(int32_t nx, int32_t ny, int32_t nz, int npt, int offdiag_mode,
                 double diag_shift, uint64_t seed, mg_csr *m) {
    if (nx < 1 || ny < 1 || nz < 1 || (npt != 7 && npt != 27)) return -1;
    int64_t n64 = (int64_t)nx * ny * nz;
    if (n64 >= INT32_MAX) return -1;
    int32_t n = (int32_t)n64;
    int64_t cap = n64 * (npt == 7 ? 4 : 14);
    if (cap >= INT32_MAX) return -1;
    if (mg_alloc(m, n, cap)) return -2;
    double *absum = (double *)calloc((size_t)n, sizeof(double));
    if (!absum) { mg_free(m); return -2; }
    uint64_t s = seed;
    int64_t k = 0;
    for (int32_t x = 0; x < nx; ++x)
        for (int32_t y = 0; y < ny; ++y)
            for (int32_t z = 0; z < nz; ++z) {
                int32_t i = (x * ny + y) * nz + z;
                m->row_ptr[i] = (int32_t)k;
                int64_t dk = k++;
                m->col[dk] = i;
                /* upper neighbours in ascending index order: dx, dy, dz loops */
                for (int dx = 0; dx <= 1; ++dx)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dz = -1; dz <= 1; ++dz) {
                            int adx = dx, ady = dy < 0 ? -dy : dy, adz = dz < 0 ? -dz : dz;
                            if (adx + ady + adz == 0) continue;
                            if (npt == 7 && adx + ady + adz != 1) continue;
                            /* upper: offset must be lexicographically positive */
                            if (dx == 0 && (dy < 0 || (dy == 0 && dz < 0))) continue;
                            int32_t X = x + dx, Y = y + dy, Z = z + dz;
                            if (X >= nx || Y < 0 || Y >= ny || Z < 0 || Z >= nz) continue;
                            int32_t j = (X * ny + Y) * nz + Z;
                            double v = offdiag_mode ? -1.0 : -(1.0 - sm64_u01(&s));
                            m->col[k] = j; m->val[k] = v; ++k;
                            absum[i] += fabs(v); absum[j] += fabs(v);
                        }
            }
    m->row_ptr[n] = (int32_t)k; m->nnz = k;
    for (int32_t i = 0; i < n; ++i) m->val[m->row_ptr[i]] = absum[i] + diag_shift;
    free(absum);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Random geometric graph: npts points uniform in the unit cube (seeded),   */
/* edge when Euclidean distance < r.  Point index = generation order.       */
/* Off-diagonal -w with w uniform in (0,1] (drawn in upper-CRS order from a */
/* second stream seed+1), diagonal = sum of w over the full row + 1.        */
int mg_geometric(int32_t npts, double radius, uint64_t seed, mg_csr *m) {
    if (npts < 1 || !(radius > 0.0)) return -1;
    double *p = (double *)malloc(sizeof(double) * 3 * (size_t)npts);
    if (!p) return -2;
    uint64_t s = seed;
    for (int64_t i = 0; i < 3 * (int64_t)npts; ++i) p[i] = sm64_u01(&s);
    int32_t g = (int32_t)floor(1.0 / radius);
    if (g < 1) g = 1;
    if (g > 512) g = 512;
    int64_t ncell = (int64_t)g * g * g;
    int32_t *cstart = (int32_t *)calloc((size_t)ncell + 1, sizeof(int32_t));
    int32_t *cidx = (int32_t *)malloc(sizeof(int32_t) * (size_t)npts);
    int32_t *cell = (int32_t *)malloc(sizeof(int32_t) * (size_t)npts);
    if (!cstart || !cidx || !cell) { free(p); free(cstart); free(cidx); free(cell); return -2; }
    for (int32_t i = 0; i < npts; ++i) {
        int cx = (int)(p[3 * i] * g), cy = (int)(p[3 * i + 1] * g), cz = (int)(p[3 * i + 2] * g);
        if (cx >= g) cx = g - 1;
        if (cy >= g) cy = g - 1;
        if (cz >= g) cz = g - 1;
        cell[i] = (cx * g + cy) * g + cz;
        cstart[cell[i] + 1]++;
    }
    for (int64_t c = 0; c < ncell; ++c) cstart[c + 1] += cstart[c];
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (size_t)ncell);
    memcpy(fill, cstart, sizeof(int32_t) * (size_t)ncell);
    for (int32_t i = 0; i < npts; ++i) cidx[fill[cell[i]]++] = i;
    free(fill);
    /* count upper neighbours first */
    double r2 = radius * radius;
    int64_t cap = 0;
    int32_t *cnt = (int32_t *)calloc((size_t)npts, sizeof(int32_t));
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            cap = (int64_t)npts;
            for (int32_t i = 0; i < npts; ++i) cap += cnt[i];
            if (cap >= INT32_MAX || mg_alloc(m, npts, cap)) {
                free(p); free(cstart); free(cidx); free(cell); free(cnt); return -2;
            }
        }
        int64_t k = 0;
        int32_t *buf = NULL; int32_t bufcap = 0;
        for (int32_t i = 0; i < npts; ++i) {
            int c = cell[i];
            int cx = c / (g * g), cy = (c / g) % g, cz = c % g;
            int32_t nb = 0;
            if (pass == 1) { m->row_ptr[i] = (int32_t)k; m->col[k] = i; m->val[k] = 0.0; ++k; }
            for (int dx = -1; dx <= 1; ++dx)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dz = -1; dz <= 1; ++dz) {
                        int X = cx + dx, Y = cy + dy, Z = cz + dz;
                        if (X < 0 || Y < 0 || Z < 0 || X >= g || Y >= g || Z >= g) continue;
                        int cc = (X * g + Y) * g + Z;
                        for (int32_t t = cstart[cc]; t < cstart[cc + 1]; ++t) {
                            int32_t j = cidx[t];
                            if (j <= i) continue;
                            double ddx = p[3 * i] - p[3 * j], ddy = p[3 * i + 1] - p[3 * j + 1],
                                   ddz = p[3 * i + 2] - p[3 * j + 2];
                            if (ddx * ddx + ddy * ddy + ddz * ddz < r2) {
                                if (pass == 0) { cnt[i]++; continue; }
                                if (nb >= bufcap) {
                                    bufcap = bufcap ? 2 * bufcap : 64;
                                    buf = (int32_t *)realloc(buf, sizeof(int32_t) * (size_t)bufcap);
                                }
                                buf[nb++] = j;
                            }
                        }
                    }
            if (pass == 1) {
                qsort(buf, (size_t)nb, sizeof(int32_t), cmp_i32);
                for (int32_t t = 0; t < nb; ++t) { m->col[k] = buf[t]; ++k; }
            }
        }
        free(buf);
        if (pass == 1) { m->row_ptr[npts] = (int32_t)k; m->nnz = k; }
    }
    /* weights in upper-CRS order from stream seed+1 */
    double *wsum = (double *)calloc((size_t)npts, sizeof(double));
    uint64_t s2 = seed + 1ULL;
    for (int32_t i = 0; i < npts; ++i)
        for (int64_t t = m->row_ptr[i] + 1; t < m->row_ptr[i + 1]; ++t) {
            double w = 1.0 - sm64_u01(&s2);
            m->val[t] = -w;
            wsum[i] += w; wsum[m->col[t]] += w;
        }
    for (int32_t i = 0; i < npts; ++i) m->val[m->row_ptr[i]] = wsum[i] + 1.0;
    free(wsum); free(p); free(cstart); free(cidx); free(cell); free(cnt);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Random symmetric banded matrix: each upper off-diagonal (i,j),           */
/* 0 < j-i <= bw, present with probability p; weights as mg_geometric.      */
int mg_banded(int32_t n, int32_t bw, double p, uint64_t seed, mg_csr *m) {
    if (n < 1 || bw < 1) return -1;
    int64_t cap = (int64_t)n * (1 + (int64_t)(p * bw * 1.5 + 8));
    if (cap >= INT32_MAX) return -1;
    if (mg_alloc(m, n, cap)) return -2;
    uint64_t s = seed;
    double *wsum = (double *)calloc((size_t)n, sizeof(double));
    int64_t k = 0;
    for (int32_t i = 0; i < n; ++i) {
        m->row_ptr[i] = (int32_t)k;
        int64_t dk = k++;
        m->col[dk] = i;
        for (int32_t d = 1; d <= bw && (int64_t)i + d < n; ++d) {
            if (sm64_u01(&s) >= p) continue;
            if (k >= cap) { free(wsum); mg_free(m); return -3; }
            double w = 1.0 - sm64_u01(&s);
            m->col[k] = i + d; m->val[k] = -w; ++k;
            wsum[i] += w; wsum[i + d] += w;
        }
    }
    m->row_ptr[n] = (int32_t)k; m->nnz = k;
    for (int32_t i = 0; i < n; ++i) m->val[m->row_ptr[i]] = wsum[i] + 1.0;
    free(wsum);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* The 2D artificial stencil of the RACE walk-through (Section 4): on an     */
/* nx*ny grid with Dirichlet boundary, point (i,j) (index i*ny+j) couples   */
/* to (i+-1,j), (i,j+-1) and the anti-diagonal pair (i+2,j-2), (i-2,j+2).   */
/* Off-diagonals -1, diagonal 8.                                            */
int mg_paper_stencil2d(int32_t nx, int32_t ny, mg_csr *m) {
    if (nx < 1 || ny < 1) return -1;
    int32_t n = nx * ny;
    if (mg_alloc(m, n, (int64_t)n * 4)) return -2;
    int64_t k = 0;
    for (int32_t i = 0; i < nx; ++i)
        for (int32_t j = 0; j < ny; ++j) {
            int32_t v = i * ny + j;
            m->row_ptr[v] = (int32_t)k;
            m->col[k] = v; m->val[k] = 8.0; ++k;
            int32_t up[6]; int cnt = 0;
            const int off[6][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}, {2, -2}, {-2, 2}};
            for (int t = 0; t < 6; ++t) {
                int32_t a = i + off[t][0], b = j + off[t][1];
                if (a < 0 || a >= nx || b < 0 || b >= ny) continue;
                int32_t u = a * ny + b;
                if (u > v) up[cnt++] = u;
            }
            qsort(up, (size_t)cnt, sizeof(int32_t), cmp_i32);
            for (int t = 0; t < cnt; ++t) { m->col[k] = up[t]; m->val[k] = -1.0; ++k; }
        }
    m->row_ptr[n] = (int32_t)k; m->nnz = k;
    return 0;
}
