/*
 * CPU oracle, brute force, FP64.  TEST INFRASTRUCTURE ONLY: the tests, the
 * smoke check and the benchmark's CPU-baseline leg load this file's library;
 * no product code path may call it.
 *
 * What it computes is the plain definition of the neighborhood query of
 * Brodu, "Spherical Indexing for Neighborhood Queries":
 *   - Sec. I: the naive O(n) query (test every object against the center),
 *     repeated for every agent (O(n^2));
 *   - Sec. II.A: with center C, radius d and object distance x, an object is a
 *     neighbor when x <= d (inclusive);
 *   - Sec. II.A (K nearest): the K closest objects within the radius;
 *   - Sec. II.B / III.C: an axis may be cyclic (the region wraps), in which
 *     case the distance along that axis is the shorter way round.
 * The spherical index reaches exactly this set (it only skips cells that
 * cannot hold a neighbor), so the definition itself is the oracle.
 *
 * Canonical predicate (the paper fixes no rounding; this is the reading used
 * by every part of the project):
 *   a_k = |(double)xj_k - (double)xi_k|;   cyclic axis: a_k = min(a_k, L_k - a_k)
 *   D2  = (a_x*a_x + a_y*a_y) + a_z*a_z     every operation IEEE FP64, RN, no FMA
 *   r2  = (double)r * (double)r;            neighbor  <=>  D2 <= r2
 * K nearest are ordered by (D2, index).  The smooth neighbor reduction
 *   E = sum_i sum_{j != i, D2 < r2} (1 - D2/r2)^3
 * is the "functor applied to each neighbor" of Sec. IV.A made concrete; its
 * gradient is written out by hand below (closed form, FP64).
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

static inline double axis_gap(double xi, double xj, double L, int cyclic) {
    double a = fabs(xj - xi);
    if (cyclic) {
        double w = L - a;
        if (w < a) a = w;
    }
    return a;
}

/* Canonical FP64 squared distance between two float4 points. */
double or_canon_d2(const float *pi, const float *pj, const double *L, int cyc) {
    double ax = axis_gap((double)pi[0], (double)pj[0], L[0], cyc & 1);
    double ay = axis_gap((double)pi[1], (double)pj[1], L[1], (cyc >> 1) & 1);
    double az = axis_gap((double)pi[2], (double)pj[2], L[2], (cyc >> 2) & 1);
    double s = ax * ax;
    double t = ay * ay;
    s = s + t;
    t = az * az;
    s = s + t;
    return s;
}

/* Signed shortest displacement xi - xj along one axis (min image if cyclic). */
static inline double axis_disp(double xi, double xj, double L, int cyclic) {
    double dlt = xi - xj;
    if (cyclic) {
        if (dlt > 0.5 * L) dlt -= L;
        else if (dlt < -0.5 * L) dlt += L;
    }
    return dlt;
}

static void set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int or_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Radius query, counts.  pos: n float4 objects.  q: m float4 centers.
 * self[k] (nullable) is an object index excluded from query k's set (the
 * all-agents mode excludes the querying agent itself), or -1.
 */
int or_radius_counts(const float *pos, int64_t n, const float *q, int64_t m,
                     const int64_t *self, const double *L, int cyc, double r,
                     int64_t *counts, int nthreads) {
    const double r2 = r * r;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < m; ++k) {
        const int64_t me = self ? self[k] : -1;
        int64_t c = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == me) continue;
            if (or_canon_d2(q + 4 * k, pos + 4 * j, L, cyc) <= r2) ++c;
        }
        counts[k] = c;
    }
    return 0;
}

/* Radius query, lists: ids of query k go to ids[offsets[k] .. offsets[k+1]),
 * ascending (objects are scanned in index order). */
int or_radius_lists(const float *pos, int64_t n, const float *q, int64_t m,
                    const int64_t *self, const double *L, int cyc, double r,
                    const int64_t *offsets, int32_t *ids, int nthreads) {
    const double r2 = r * r;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < m; ++k) {
        const int64_t me = self ? self[k] : -1;
        int64_t w = offsets[k];
        const int64_t end = offsets[k + 1];
        for (int64_t j = 0; j < n && w < end; ++j) {
            if (j == me) continue;
            if (or_canon_d2(q + 4 * k, pos + 4 * j, L, cyc) <= r2) ids[w++] = (int32_t)j;
        }
    }
    return 0;
}

/*
 * K nearest within r_max (inclusive; r_max < 0 means unbounded), ordered by
 * (D2, index).  ids[m*k] padded with -1, d2[m*k] (FP64, padded with +inf),
 * counts[m] = number found (<= k).
 */
int or_knn(const float *pos, int64_t n, const float *q, int64_t m,
           const int64_t *self, const double *L, int cyc, double rmax, int k,
           int32_t *ids, double *d2, int32_t *counts, int nthreads) {
    const double r2 = rmax < 0 ? INFINITY : rmax * rmax;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t qi = 0; qi < m; ++qi) {
        int32_t *bi = ids + qi * (int64_t)k;
        double *bd = d2 + qi * (int64_t)k;
        for (int t = 0; t < k; ++t) { bi[t] = -1; bd[t] = INFINITY; }
        const int64_t me = self ? self[qi] : -1;
        int found = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == me) continue;
            const double dd = or_canon_d2(q + 4 * qi, pos + 4 * j, L, cyc);
            if (!(dd <= r2)) continue;
            /* (dd, j) with j increasing: an equal dd never displaces. */
            if (found == k && !(dd < bd[k - 1])) continue;
            int p = found < k ? found : k - 1;
            while (p > 0 && bd[p - 1] > dd) {
                bd[p] = bd[p - 1];
                bi[p] = bi[p - 1];
                --p;
            }
            bd[p] = dd;
            bi[p] = (int32_t)j;
            if (found < k) ++found;
        }
        counts[qi] = found;
    }
    return 0;
}

/*
 * Smooth neighbor reduction for the objects listed in idx[m]:
 *   e[t]  = sum_{j != i, D2 < r2} (1 - D2/r2)^3                       (i = idx[t])
 *   g[3t] = dE/dx_i = -(12/r2) sum_{j != i, D2 < r2} (1 - D2/r2)^2 (x_i - x_j)
 * E = sum_i e_i counts every unordered pair twice, so x_i appears in both
 * w(D_ij) and w(D_ji); d/dx_i of (1 - D2/r2)^3 is -3 (1 - D2/r2)^2 * 2 (x_i - x_j)/r2,
 * doubled for the two appearances: the factor 12.
 */
int or_reduce(const float *pos, int64_t n, const int64_t *idx, int64_t m,
              const double *L, int cyc, double r, double *e, double *g, int nthreads) {
    const double r2 = r * r;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < m; ++t) {
        const int64_t i = idx[t];
        const float *pi = pos + 4 * i;
        double es = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            const float *pj = pos + 4 * j;
            const double dd = or_canon_d2(pi, pj, L, cyc);
            if (!(dd < r2)) continue;
            const double u = 1.0 - dd / r2;
            es += u * u * u;
            const double c = u * u;
            gx += c * axis_disp((double)pi[0], (double)pj[0], L[0], cyc & 1);
            gy += c * axis_disp((double)pi[1], (double)pj[1], L[1], (cyc >> 1) & 1);
            gz += c * axis_disp((double)pi[2], (double)pj[2], L[2], (cyc >> 2) & 1);
        }
        e[t] = es;
        if (g) {
            g[3 * t + 0] = -12.0 / r2 * gx;
            g[3 * t + 1] = -12.0 / r2 * gy;
            g[3 * t + 2] = -12.0 / r2 * gz;
        }
    }
    return 0;
}

/*
 * The same reduction as or_reduce for every object at once, through the plain
 * bin lattice of Sec. I (the "cube" of cells around a query): objects are
 * binned into cells at least r wide on every axis, so every pair with
 * D2 < r2 lies in the same or adjacent cells (adjacent across the wrap on a
 * cyclic axis).  Each object scans the 3 x 3 x 3 cells around its own and
 * applies, per pair, the predicate and the terms of or_reduce; only the order
 * of the sum over j differs.  Cyclic axis a: G_a = floor(L_a / r) cells of
 * side L_a / G_a >= r, cell floor(x G_a / L_a) mod G_a (G_a >= 3, else the
 * call falls back to or_reduce); non-cyclic axis: cells of side r from the
 * smallest coordinate.  e[n], g[3n] (nullable) as or_reduce with idx = 0..n-1.
 */
int or_reduce_cells(const float *pos, int64_t n, const double *L, int cyc, double r, double *e,
                    double *g, int nthreads) {
    const double r2 = r * r;
    int64_t G[3];
    double lo[3], w[3];
    for (int a = 0; a < 3; ++a) {
        if ((cyc >> a) & 1) {
            G[a] = (int64_t)floor(L[a] / r);
            lo[a] = 0.0;
            w[a] = L[a] / (double)G[a];
            if (G[a] < 3) {
                int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
                for (int64_t i = 0; i < n; ++i) idx[i] = i;
                const int rc = or_reduce(pos, n, idx, n, L, cyc, r, e, g, nthreads);
                free(idx);
                return rc;
            }
        } else {
            double mn = INFINITY, mx = -INFINITY;
            for (int64_t i = 0; i < n; ++i) {
                const double x = (double)pos[4 * i + a];
                if (x < mn) mn = x;
                if (x > mx) mx = x;
            }
            if (n == 0) mn = mx = 0.0;
            lo[a] = mn;
            w[a] = r;
            G[a] = (int64_t)floor((mx - mn) / r) + 1;
        }
    }
    const int64_t C = G[0] * G[1] * G[2];
    int64_t *cell = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *start = (int64_t *)calloc((size_t)C + 1, sizeof(int64_t));
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)C);
    if (!cell || !start || !order || !fill) {
        free(cell); free(start); free(order); free(fill);
        return -1;
    }
    for (int64_t i = 0; i < n; ++i) {
        int64_t c[3];
        for (int a = 0; a < 3; ++a) {
            const double x = (double)pos[4 * i + a];
            int64_t k;
            if ((cyc >> a) & 1) {
                k = (int64_t)floor(x / L[a] * (double)G[a]);
                k %= G[a];
                if (k < 0) k += G[a];
            } else {
                k = (int64_t)floor((x - lo[a]) / w[a]);
                if (k < 0) k = 0;
                if (k >= G[a]) k = G[a] - 1;
            }
            c[a] = k;
        }
        cell[i] = (c[2] * G[1] + c[1]) * G[0] + c[0];
        ++start[cell[i] + 1];
    }
    for (int64_t c = 0; c < C; ++c) start[c + 1] += start[c];
    for (int64_t c = 0; c < C; ++c) fill[c] = start[c];
    for (int64_t i = 0; i < n; ++i) order[fill[cell[i]]++] = i;   /* ascending index inside a cell */
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        const float *pi = pos + 4 * i;
        const int64_t ci = cell[i];
        const int64_t cx = ci % G[0], cy = (ci / G[0]) % G[1], cz = ci / (G[0] * G[1]);
        double es = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
        for (int dz = -1; dz <= 1; ++dz) {
            int64_t z = cz + dz;
            if (cyc & 4) z = (z + G[2]) % G[2];
            else if (z < 0 || z >= G[2]) continue;
            for (int dy = -1; dy <= 1; ++dy) {
                int64_t y = cy + dy;
                if (cyc & 2) y = (y + G[1]) % G[1];
                else if (y < 0 || y >= G[1]) continue;
                for (int dx = -1; dx <= 1; ++dx) {
                    int64_t x = cx + dx;
                    if (cyc & 1) x = (x + G[0]) % G[0];
                    else if (x < 0 || x >= G[0]) continue;
                    const int64_t c = (z * G[1] + y) * G[0] + x;
                    for (int64_t t = start[c]; t < start[c + 1]; ++t) {
                        const int64_t j = order[t];
                        if (j == i) continue;
                        const float *pj = pos + 4 * j;
                        const double dd = or_canon_d2(pi, pj, L, cyc);
                        if (!(dd < r2)) continue;
                        const double u = 1.0 - dd / r2;
                        es += u * u * u;
                        const double cu = u * u;
                        gx += cu * axis_disp((double)pi[0], (double)pj[0], L[0], cyc & 1);
                        gy += cu * axis_disp((double)pi[1], (double)pj[1], L[1], (cyc >> 1) & 1);
                        gz += cu * axis_disp((double)pi[2], (double)pj[2], L[2], (cyc >> 2) & 1);
                    }
                }
            }
        }
        e[i] = es;
        if (g) {
            g[3 * i + 0] = -12.0 / r2 * gx;
            g[3 * i + 1] = -12.0 / r2 * gy;
            g[3 * i + 2] = -12.0 / r2 * gz;
        }
    }
    free(cell); free(start); free(order); free(fill);
    return 0;
}
