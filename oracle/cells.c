/*
 * CPU cell walks, FP64 (the "tier B" CPU baselines).  TEST INFRASTRUCTURE
 * ONLY: the tests and the benchmark's CPU-baseline leg load this file's
 * library; no product code path may call it.
 *
 * The radius query of Brodu, "Spherical Indexing for Neighborhood Queries",
 * over a lattice of cubic cells of side s (2^w cells per axis, Sec. II.B),
 * with the canonical predicate of brute.c (its definition is repeated here,
 * so that this file stands alone):
 *   - mode 0, the bin-lattice cube scan: every cell of the bounding cube of
 *     the query's sphere (Sec. I: "the cube of cells");
 *   - mode 1, the spherical index: the cell offsets within floor(d) + 1 of
 *     the query's cell, walked in order of their minimum bound
 *     b^2 = sum_a max(|o_a| - 1, 0)^2 (Sec. II.A, Fig. 2), cut at b > d, and
 *     each cell tested exactly against the query's position,
 *     t^2 = sum over o_a != 0 of (|o_a| - 1 + zeta_a)^2 <= d^2 (Sec. III.A,
 *     Eq. 1; zeta_a the distance from the query to its cell face toward o_a).
 * Both visit every cell that can hold a neighbor, so both give the plain
 * definition's lists (tested against brute.c); they differ in how many cells
 * and points they touch.  Cells are numbered z * Gx * Gy + y * Gx + x; an
 * offset that leaves the region on a non-cyclic axis goes to the one outside
 * cell (Sec. II.B), whose points are tested once per query; a query outside
 * the region tests every point.  The cell tests take d + 1e-9 cells, a
 * margin for the rounding of the FP64 binning.
 *
 * Build: gcc -O2 -fPIC -shared -ffp-contract=off -fno-fast-math -fopenmp
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static inline double gap1(double xi, double xj, double L, int cyclic) {
    double a = fabs(xj - xi);
    if (cyclic) {
        double w = L - a;
        if (w < a) a = w;
    }
    return a;
}

static inline double canon(const float *pi, const float *pj, const double *L, int cyc) {
    double ax = gap1((double)pi[0], (double)pj[0], L[0], cyc & 1);
    double ay = gap1((double)pi[1], (double)pj[1], L[1], (cyc >> 1) & 1);
    double az = gap1((double)pi[2], (double)pj[2], L[2], (cyc >> 2) & 1);
    double s = ax * ax;
    double t = ay * ay;
    s = s + t;
    t = az * az;
    s = s + t;
    return s;
}

typedef struct {
    int ox, oy, oz, b2;
} Offset;

static int cmp_offset(const void *a, const void *b) {
    const Offset *x = (const Offset *)a, *y = (const Offset *)b;
    return (x->b2 > y->b2) - (x->b2 < y->b2);
}

static int cmp_int(const void *a, const void *b) {
    const int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

typedef struct {
    int64_t G[3], C;        /* cells per axis, cell count (the outside cell is C) */
    int64_t *start;         /* C + 2 */
    int *order;             /* points in cell order, ascending index inside a cell */
    int64_t *cell;          /* cell of each point */
} Lattice;

static int bin(const float *pos, int64_t n, const double *origin, double s, const int *w, int cyc,
               Lattice *lt) {
    for (int a = 0; a < 3; ++a) lt->G[a] = (int64_t)1 << w[a];
    lt->C = lt->G[0] * lt->G[1] * lt->G[2];
    lt->start = (int64_t *)calloc((size_t)lt->C + 2, sizeof(int64_t));
    lt->order = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    lt->cell = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * ((size_t)lt->C + 1));
    if (!lt->start || !lt->order || !lt->cell || !fill) {
        free(fill);
        return -1;
    }
    for (int64_t i = 0; i < n; ++i) {
        int64_t c[3];
        int out = 0;
        for (int a = 0; a < 3; ++a) {
            int64_t k = (int64_t)floor(((double)pos[4 * i + a] - origin[a]) / s);
            if ((cyc >> a) & 1) {
                k %= lt->G[a];
                if (k < 0) k += lt->G[a];
            } else if (k < 0 || k >= lt->G[a]) {
                out = 1;
            }
            c[a] = k;
        }
        lt->cell[i] = out ? lt->C : (c[2] * lt->G[1] + c[1]) * lt->G[0] + c[0];
        ++lt->start[lt->cell[i] + 1];
    }
    for (int64_t c = 0; c <= lt->C; ++c) lt->start[c + 1] += lt->start[c];
    for (int64_t c = 0; c <= lt->C; ++c) fill[c] = lt->start[c];
    for (int64_t i = 0; i < n; ++i) lt->order[fill[lt->cell[i]]++] = (int)i;
    free(fill);
    return 0;
}

static void unbin(Lattice *lt) {
    free(lt->start);
    free(lt->order);
    free(lt->cell);
}

/* The walk's inputs shared by every query. */
typedef struct {
    const float *pos;
    int64_t n;
    const double *origin, *L;
    double s, d, r2;
    int cyc, mode;
    const Lattice *lt;
    const Offset *tab;
    int ntab;
} Ctx;

/* One query (point i): writes its neighbors, unsorted, to out (if not NULL)
 * and returns their number. */
static int64_t walk(const Ctx *x, int64_t i, int *out) {
    const float *pi = x->pos + 4 * i;
    const Lattice *lt = x->lt;
    int64_t k = 0;
    if (lt->cell[i] == lt->C) {   /* query outside the region: every point */
        for (int64_t j = 0; j < x->n; ++j)
            if (j != i && canon(pi, x->pos + 4 * j, x->L, x->cyc) <= x->r2) {
                if (out) out[k] = (int)j;
                ++k;
            }
        return k;
    }
    double u[3], zp[3], zn[3];
    int64_t c[3];
    for (int a = 0; a < 3; ++a) {
        u[a] = ((double)pi[a] - x->origin[a]) / x->s;
        c[a] = (int64_t)floor(u[a]);
        zp[a] = (double)(c[a] + 1) - u[a];
        zn[a] = u[a] - (double)c[a];
        if (zp[a] < 0.0) zp[a] = 0.0;
        if (zn[a] < 0.0) zn[a] = 0.0;
    }
    const double dm = x->d + 1e-9;
    int outside_seen = 0;
    int64_t lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    if (x->mode == 0) {
        for (int a = 0; a < 3; ++a) {
            lo[a] = (int64_t)floor(u[a] - dm) - c[a];
            hi[a] = (int64_t)floor(u[a] + dm) - c[a];
        }
    }
    const int ncells = x->mode == 0 ? (int)((hi[0] - lo[0] + 1) * (hi[1] - lo[1] + 1) * (hi[2] - lo[2] + 1))
                                    : x->ntab;
    for (int e = 0; e < ncells; ++e) {
        int o[3];
        if (x->mode == 0) {
            const int64_t nx = hi[0] - lo[0] + 1, ny = hi[1] - lo[1] + 1;
            o[0] = (int)(lo[0] + e % nx);
            o[1] = (int)(lo[1] + (e / nx) % ny);
            o[2] = (int)(lo[2] + e / (nx * ny));
        } else {
            const Offset *t = &x->tab[e];
            if ((double)t->b2 > dm * dm) break;   /* every later entry lies beyond d */
            double t2 = 0.0;
            o[0] = t->ox;
            o[1] = t->oy;
            o[2] = t->oz;
            for (int a = 0; a < 3; ++a) {
                if (o[a] > 0) {
                    const double g = (double)(o[a] - 1) + zp[a];
                    t2 += g * g;
                } else if (o[a] < 0) {
                    const double g = (double)(-o[a] - 1) + zn[a];
                    t2 += g * g;
                }
            }
            if (t2 > dm * dm) continue;           /* Eq. 1: no point of the cell within d */
        }
        int64_t tc[3];
        int leaves = 0;
        for (int a = 0; a < 3; ++a) {
            int64_t v = c[a] + o[a];
            if ((x->cyc >> a) & 1) {
                v %= lt->G[a];
                if (v < 0) v += lt->G[a];
            } else if (v < 0 || v >= lt->G[a]) {
                leaves = 1;
            }
            tc[a] = v;
        }
        int64_t cell;
        if (leaves) {
            if (outside_seen) continue;
            outside_seen = 1;
            cell = lt->C;
        } else {
            cell = (tc[2] * lt->G[1] + tc[1]) * lt->G[0] + tc[0];
        }
        for (int64_t p = lt->start[cell]; p < lt->start[cell + 1]; ++p) {
            const int j = lt->order[p];
            if (j != i && canon(pi, x->pos + 4 * j, x->L, x->cyc) <= x->r2) {
                if (out) out[k] = j;
                ++k;
            }
        }
    }
    return k;
}

static void set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

/*
 * Radius lists of the queries qidx[0..m) (all-agents: each query is a point
 * of pos and leaves itself out).  offsets NULL: write counts[m] only; else
 * write ids[offsets[q] ..] ascending.  mode 0: cube scan, 1: spherical index.
 * Returns 0; -1 when an allocation fails or a cyclic axis would wrap the
 * walk onto itself (2 (floor(d) + 1) + 1 > cells); -2 when a list's length
 * differs from its offsets.
 */
int or_cells_radius(const float *pos, int64_t n, const double *origin, double s, const int *w, int cyc,
                    double r, int mode, const int64_t *qidx, int64_t m, int64_t *counts,
                    const int64_t *offsets, int *ids, int nthreads) {
    const double d = r / s;
    const int R = (int)floor(d) + 1;
    for (int a = 0; a < 3; ++a)
        if (((cyc >> a) & 1) && 2 * R + 1 > (1 << w[a])) return -1;
    Lattice lt;
    if (bin(pos, n, origin, s, w, cyc, &lt) != 0) {
        unbin(&lt);
        return -1;
    }
    double L[3];
    for (int a = 0; a < 3; ++a) L[a] = s * (double)((int64_t)1 << w[a]);
    /* the offset table of Sec. II.A: every offset within R, by b^2 */
    const int side = 2 * R + 1;
    Offset *tab = (Offset *)malloc(sizeof(Offset) * (size_t)side * side * side);
    if (!tab) {
        unbin(&lt);
        return -1;
    }
    int nt = 0;
    for (int oz = -R; oz <= R; ++oz)
        for (int oy = -R; oy <= R; ++oy)
            for (int ox = -R; ox <= R; ++ox) {
                const int bx = abs(ox) > 0 ? abs(ox) - 1 : 0, by = abs(oy) > 0 ? abs(oy) - 1 : 0,
                          bz = abs(oz) > 0 ? abs(oz) - 1 : 0;
                tab[nt].ox = ox;
                tab[nt].oy = oy;
                tab[nt].oz = oz;
                tab[nt].b2 = bx * bx + by * by + bz * bz;
                ++nt;
            }
    qsort(tab, (size_t)nt, sizeof(Offset), cmp_offset);
    Ctx x = {pos, n, origin, L, s, d, (double)r * (double)r, cyc, mode, &lt, tab, nt};
    int bad = 0;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64) reduction(| : bad)
    for (int64_t q = 0; q < m; ++q) {
        const int64_t i = qidx[q];
        if (!offsets) {
            counts[q] = walk(&x, i, NULL);
        } else {
            int *dst = ids + offsets[q];
            const int64_t k = walk(&x, i, dst);
            if (k != offsets[q + 1] - offsets[q]) bad = 1;
            qsort(dst, (size_t)k, sizeof(int), cmp_int);
        }
    }
    free(tab);
    unbin(&lt);
    return bad ? -2 : 0;
}
