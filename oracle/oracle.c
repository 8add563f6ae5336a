/*
 * CPU oracle for the periodic neighbor query, RDF and Steinhardt order parameters of
 * freud (arXiv 1906.06317).  TEST INFRASTRUCTURE ONLY: the tests, the smoke check and
 * the bench's CPU-baseline leg call it; the product path never does.  It shares no
 * code with the CUDA library.
 *
 * Everything is plain FP64 written from the definitions, one query at a time.  The
 * cell list here is only a pruning device: every pair decision goes through the same
 * exact FP64 minimum-image sequence (min_image below), so the cell list can change
 * speed, never results (checked against O(N^2) enumeration in the tests).
 *
 * Box (Section "Implementation": triclinic box with three independent vectors, centred
 * at the origin): params (Lx, Ly, Lz, xy, xz, yz), a1 = (Lx,0,0), a2 = (xy Ly, Ly, 0),
 * a3 = (xz Lz, yz Lz, Lz).  Lz = 0 is a 2D box (Section "Implementation": boxes are
 * two- or three-dimensional): xz = yz = 0, points have z = 0, there is no periodicity
 * along z, and the widths are those of the parallelogram (w_z = infinity).
 *
 * Readings of the paper (it gives no formulas for these):
 *  - minimum image: reduce along a3, then a2, then a1 by rint of the Cartesian
 *    component over the box length (op order fixed below; valid for r < w_min/2);
 *  - a pair is a neighbor iff r = sqrt(r2) < r_max (strict), r2 = (dx dx + dy dy) + dz dz;
 *  - neighbor lists are ordered by (query index, point index);
 *  - kNN orders candidates by (r2, point index), keeps min(k, available);
 *  - RDF bin b holds R_b <= r < R_{b+1}, R_b = r_min + b*((r_max-r_min)/bins),
 *    R_bins = r_max;
 *  - q_l of a particle without neighbors is 0, and so is its gradient.
 * Compile with -O2 -ffp-contract=off so no multiply-add is fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_BOX_TOO_SMALL (-2)
#define ORC_ERR_OOM (-3)

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---------------------------------------------------------------------------- box */

static void box_vectors(const double *b, double a2x[1], double a3x[1], double a3y[1]) {
    a2x[0] = b[3] * b[1]; /* xy * Ly */
    a3x[0] = b[4] * b[2]; /* xz * Lz */
    a3y[0] = b[5] * b[2]; /* yz * Lz */
}

static int is_2d(const double *b) { return b[2] == 0.0; }

/* Perpendicular widths w_k = V / |a_i x a_j| (distance between opposite faces); in 2D
 * the parallelogram's heights A / |a_other| (A = Lx Ly) and w_z = infinity. */
int orc_box_widths(const double *b, double *w) {
    if (is_2d(b)) {
        double A = b[0] * b[1];
        w[0] = A / sqrt((b[3] * b[1]) * (b[3] * b[1]) + b[1] * b[1]);
        w[1] = A / b[0];
        w[2] = INFINITY;
        return ORC_OK;
    }
    double a1[3] = {b[0], 0.0, 0.0};
    double a2[3] = {b[3] * b[1], b[1], 0.0};
    double a3[3] = {b[4] * b[2], b[5] * b[2], b[2]};
    double V = b[0] * b[1] * b[2];
    const double *A[3] = {a1, a2, a3};
    for (int k = 0; k < 3; ++k) {
        const double *u = A[(k + 1) % 3], *v = A[(k + 2) % 3];
        double c0 = u[1] * v[2] - u[2] * v[1];
        double c1 = u[2] * v[0] - u[0] * v[2];
        double c2 = u[0] * v[1] - u[1] * v[0];
        w[k] = fabs(V) / sqrt(c0 * c0 + c1 * c1 + c2 * c2);
    }
    return ORC_OK;
}

static double min_width(const double *b) {
    double w[3];
    orc_box_widths(b, w);
    double m = w[0];
    if (w[1] < m) m = w[1];
    if (w[2] < m) m = w[2];
    return m;
}

/* Minimum-image displacement d = x_j - x_i, reduced along a3, a2, a1 in that order.
 * This exact sequence of IEEE double operations (no fused multiply-add) defines every
 * distance the library reports. */
static void min_image(const double *b, const double *xi, const double *xj, double *d) {
    double a2x, a3x, a3y;
    box_vectors(b, &a2x, &a3x, &a3y);
    double dx = xj[0] - xi[0];
    double dy = xj[1] - xi[1];
    double dz = xj[2] - xi[2];
    if (!is_2d(b)) { /* a 2D box has no z period */
        double nz = rint(dz / b[2]);
        dx = dx - nz * a3x;
        dy = dy - nz * a3y;
        dz = dz - nz * b[2];
    }
    double ny = rint(dy / b[1]);
    dx = dx - ny * a2x;
    dy = dy - ny * b[1];
    double nx = rint(dx / b[0]);
    dx = dx - nx * b[0];
    d[0] = dx;
    d[1] = dy;
    d[2] = dz;
}

static double r2_of(const double *d) { return (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]; }

int orc_min_image(const double *b, const double *xi, const double *xj, double *d_out, double *r_out) {
    min_image(b, xi, xj, d_out);
    *r_out = sqrt(r2_of(d_out));
    return ORC_OK;
}

/* Fractional coordinate in [0,1) of a point: s = M^{-1} x + 1/2, wrapped.  Used only to
 * pick cells (pruning), never to decide a pair. */
static void frac_wrapped(const double *b, const double *x, double *f) {
    double sz = is_2d(b) ? 0.0 : x[2] / b[2];
    double sy = (x[1] - sz * b[5] * b[2]) / b[1];
    double sx = (x[0] - sy * b[3] * b[1] - sz * b[4] * b[2]) / b[0];
    double s[3] = {sx + 0.5, sy + 0.5, sz + 0.5};
    for (int k = 0; k < 3; ++k) {
        f[k] = s[k] - floor(s[k]);
        if (f[k] >= 1.0) f[k] = 0.0;
        if (f[k] < 0.0) f[k] = 0.0;
    }
}

/* ------------------------------------------------------------------- cell list */

/* Cells per axis: floor(w_k / r_cell) with a relative margin; an axis with fewer than
 * 3 cells collapses to one cell (the stencil then spans the whole axis once). */
int orc_cells_dims(const double *b, double r_cell, int32_t *nc) {
    double w[3];
    if (!(r_cell > 0.0)) return ORC_ERR_ARG;
    orc_box_widths(b, w);
    int64_t tot = 1;
    for (int k = 0; k < 3; ++k) {
        double q = floor(w[k] / (r_cell * (1.0 + 1e-9)));
        int n = q > 512.0 ? 512 : (int)q;
        if (n < 3 || (k == 2 && is_2d(b))) n = 1;
        nc[k] = n;
        tot *= n;
    }
    return tot > (1 << 27) ? ORC_ERR_ARG : ORC_OK;
}

static int64_t cell_of(const double *b, const int32_t *nc, const double *x) {
    double f[3];
    frac_wrapped(b, x, f);
    int c[3];
    for (int k = 0; k < 3; ++k) {
        c[k] = (int)floor(f[k] * nc[k]);
        if (c[k] >= nc[k]) c[k] = nc[k] - 1;
        if (c[k] < 0) c[k] = 0;
    }
    return ((int64_t)c[2] * nc[1] + c[1]) * nc[0] + c[0];
}

/* Counting sort of points into cells: order[] lists point indices cell by cell in
 * increasing index order; cell_start has ncells+1 entries. */
int orc_cells_build(const double *b, const double *pts, int64_t n, const int32_t *nc,
                    int64_t *cell_start, int64_t *order) {
    int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    int64_t *cid = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    if (!cid) return ORC_ERR_OOM;
    memset(cell_start, 0, sizeof(int64_t) * (ncell + 1));
    for (int64_t i = 0; i < n; ++i) {
        cid[i] = cell_of(b, nc, pts + 3 * i);
        cell_start[cid[i] + 1]++;
    }
    for (int64_t c = 0; c < ncell; ++c) cell_start[c + 1] += cell_start[c];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (ncell > 0 ? ncell : 1));
    if (!fill) {
        free(cid);
        return ORC_ERR_OOM;
    }
    memcpy(fill, cell_start, sizeof(int64_t) * ncell);
    for (int64_t i = 0; i < n; ++i) order[fill[cid[i]]++] = i;
    free(fill);
    free(cid);
    return ORC_OK;
}

/* Candidate enumeration: all points in cells within +-s of the query's cell, each cell
 * once (an axis whose stencil would wrap onto itself is scanned whole). */
typedef struct {
    const double *b;
    const double *pts;
    const int32_t *nc;
    const int64_t *cell_start;
    const int64_t *order;
} cells_t;

typedef void (*visit_fn)(void *ctx, int64_t j);

static void for_candidates(const cells_t *C, const double *x, int s, visit_fn fn, void *ctx) {
    double f[3];
    frac_wrapped(C->b, x, f);
    int c[3], lo[3], hi[3];
    for (int k = 0; k < 3; ++k) {
        c[k] = (int)floor(f[k] * C->nc[k]);
        if (c[k] >= C->nc[k]) c[k] = C->nc[k] - 1;
        if (c[k] < 0) c[k] = 0;
        if (2 * s + 1 >= C->nc[k]) {
            lo[k] = 0;
            hi[k] = C->nc[k] - 1;
            c[k] = 0;
        } else {
            lo[k] = -s;
            hi[k] = s;
        }
    }
    for (int oz = lo[2]; oz <= hi[2]; ++oz)
        for (int oy = lo[1]; oy <= hi[1]; ++oy)
            for (int ox = lo[0]; ox <= hi[0]; ++ox) {
                int cz = ((c[2] + oz) % C->nc[2] + C->nc[2]) % C->nc[2];
                int cy = ((c[1] + oy) % C->nc[1] + C->nc[1]) % C->nc[1];
                int cx = ((c[0] + ox) % C->nc[0] + C->nc[0]) % C->nc[0];
                int64_t cell = ((int64_t)cz * C->nc[1] + cy) * C->nc[0] + cx;
                for (int64_t p = C->cell_start[cell]; p < C->cell_start[cell + 1]; ++p) fn(ctx, C->order[p]);
            }
}

static int all_cells_covered(const int32_t *nc, int s) {
    return (2 * s + 1 >= nc[0]) && (2 * s + 1 >= nc[1]) && (2 * s + 1 >= nc[2]);
}

/* ------------------------------------------------------------------ ball query */

typedef struct {
    int64_t j;
    double r2;
} hit_t;

typedef struct {
    const double *b;
    const double *pts;
    const double *xq;
    int64_t iq;
    int exclude_ii;
    double r_max;
    hit_t *buf;
    int64_t n, cap;
    int oom;
} ball_ctx;

static void ball_visit(void *vctx, int64_t j) {
    ball_ctx *B = (ball_ctx *)vctx;
    if (B->exclude_ii && j == B->iq) return;
    double d[3];
    min_image(B->b, B->xq, B->pts + 3 * j, d);
    double r2 = r2_of(d);
    if (sqrt(r2) < B->r_max) {
        if (B->n == B->cap) {
            int64_t nc = B->cap ? 2 * B->cap : 64;
            hit_t *nb = (hit_t *)realloc(B->buf, sizeof(hit_t) * nc);
            if (!nb) {
                B->oom = 1;
                return;
            }
            B->buf = nb;
            B->cap = nc;
        }
        B->buf[B->n].j = j;
        B->buf[B->n].r2 = r2;
        B->n++;
    }
}

static int cmp_hit_j(const void *a, const void *b) {
    int64_t x = ((const hit_t *)a)->j, y = ((const hit_t *)b)->j;
    return (x > y) - (x < y);
}

/*
 * Ball query for queries [q0, q1): every point j (j != query index when exclude_ii) with
 * r < r_max.  Mode count (pj == NULL): counts[q - q0] = number of neighbors.  Mode fill:
 * writes (j, r) sorted by j at out_offsets[q - q0] .. (offsets relative to q0's start).
 * nc == NULL selects O(N) brute force per query (every point is a candidate).
 */
int orc_ball_query(const double *b, const double *pts, int64_t n, const int32_t *nc,
                   const int64_t *cell_start, const int64_t *order, const double *qpts,
                   int64_t q0, int64_t q1, double r_max, int exclude_ii, int64_t *counts,
                   const int64_t *out_offsets, int64_t *pj, double *dist) {
    if (!(r_max > 0.0) || q1 < q0) return ORC_ERR_ARG;
    if (!(r_max < 0.5 * min_width(b))) return ORC_ERR_BOX_TOO_SMALL;
    cells_t C = {b, pts, nc, cell_start, order};
    ball_ctx B;
    memset(&B, 0, sizeof(B));
    B.b = b;
    B.pts = pts;
    B.exclude_ii = exclude_ii;
    B.r_max = r_max;
    for (int64_t q = q0; q < q1; ++q) {
        B.xq = qpts + 3 * q;
        B.iq = q;
        B.n = 0;
        if (nc) {
            for_candidates(&C, B.xq, 1, ball_visit, &B);
        } else {
            for (int64_t j = 0; j < n; ++j) ball_visit(&B, j);
        }
        if (B.oom) {
            free(B.buf);
            return ORC_ERR_OOM;
        }
        if (counts) counts[q - q0] = B.n;
        if (pj) {
            qsort(B.buf, (size_t)B.n, sizeof(hit_t), cmp_hit_j);
            int64_t o = out_offsets[q - q0];
            for (int64_t t = 0; t < B.n; ++t) {
                pj[o + t] = B.buf[t].j;
                dist[o + t] = sqrt(B.buf[t].r2);
            }
        }
    }
    free(B.buf);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ kNN */

static int cmp_hit_r2j(const void *a, const void *b) {
    const hit_t *x = (const hit_t *)a, *y = (const hit_t *)b;
    if (x->r2 < y->r2) return -1;
    if (x->r2 > y->r2) return 1;
    return (x->j > y->j) - (x->j < y->j);
}

typedef struct {
    const double *b;
    const double *pts;
    const double *xq;
    int64_t iq;
    int exclude_ii;
    hit_t *buf;
    int64_t n, cap;
    int oom;
} knn_ctx;

static void knn_visit(void *vctx, int64_t j) {
    knn_ctx *K = (knn_ctx *)vctx;
    if (K->exclude_ii && j == K->iq) return;
    double d[3];
    min_image(K->b, K->xq, K->pts + 3 * j, d);
    if (K->n == K->cap) {
        int64_t nc = K->cap ? 2 * K->cap : 256;
        hit_t *nb = (hit_t *)realloc(K->buf, sizeof(hit_t) * nc);
        if (!nb) {
            K->oom = 1;
            return;
        }
        K->buf = nb;
        K->cap = nc;
    }
    K->buf[K->n].j = j;
    K->buf[K->n].r2 = r2_of(d);
    K->n++;
}

/*
 * k nearest neighbors of queries [q0, q1), ordered by (r2, j); each query gets
 * min(k, available) entries written at out[(q - q0) * k + rank] (j, r); out_n holds the
 * per-query count.  A result whose farthest neighbor has r >= w_min/2 is not a reliable
 * minimum image: the call then returns ORC_ERR_BOX_TOO_SMALL.  With nc == NULL every
 * point is a candidate; with cells, the stencil grows until the k-th distance is below
 * the radius it is guaranteed to contain.
 */
int orc_knn(const double *b, const double *pts, int64_t n, const int32_t *nc, const int64_t *cell_start,
            const int64_t *order, const double *qpts, int64_t q0, int64_t q1, int k, int exclude_ii,
            int64_t *out_j, double *out_r, int64_t *out_n) {
    if (k <= 0 || q1 < q0) return ORC_ERR_ARG;
    double wmin = min_width(b);
    double w[3];
    orc_box_widths(b, w);
    cells_t C = {b, pts, nc, cell_start, order};
    knn_ctx K;
    memset(&K, 0, sizeof(K));
    K.b = b;
    K.pts = pts;
    K.exclude_ii = exclude_ii;
    int status = ORC_OK;
    for (int64_t q = q0; q < q1; ++q) {
        K.xq = qpts + 3 * q;
        K.iq = q;
        if (!nc) {
            K.n = 0;
            for (int64_t j = 0; j < n; ++j) knn_visit(&K, j);
        } else {
            double cw = w[0] / nc[0];
            if (w[1] / nc[1] < cw) cw = w[1] / nc[1];
            if (w[2] / nc[2] < cw) cw = w[2] / nc[2];
            for (int s = 1;; ++s) {
                K.n = 0;
                for_candidates(&C, K.xq, s, knn_visit, &K);
                if (K.oom) break;
                if (all_cells_covered(nc, s)) break;
                if (K.n >= k) {
                    qsort(K.buf, (size_t)K.n, sizeof(hit_t), cmp_hit_r2j);
                    if (sqrt(K.buf[k - 1].r2) < s * cw * (1.0 - 1e-12)) break;
                }
            }
        }
        if (K.oom) {
            free(K.buf);
            return ORC_ERR_OOM;
        }
        qsort(K.buf, (size_t)K.n, sizeof(hit_t), cmp_hit_r2j);
        int64_t m = K.n < k ? K.n : k;
        out_n[q - q0] = m;
        for (int64_t t = 0; t < m; ++t) {
            out_j[(q - q0) * k + t] = K.buf[t].j;
            out_r[(q - q0) * k + t] = sqrt(K.buf[t].r2);
        }
        if (m > 0 && !(sqrt(K.buf[m - 1].r2) < 0.5 * wmin)) status = ORC_ERR_BOX_TOO_SMALL;
    }
    free(K.buf);
    return status;
}

/* ------------------------------------------------------------------------ RDF */

/* Bin edges R_0..R_bins: R_b = r_min + b * ((r_max - r_min) / bins), R_bins = r_max. */
int orc_rdf_edges(int bins, double r_min, double r_max, double *edges) {
    if (bins <= 0 || !(r_max > r_min) || r_min < 0.0) return ORC_ERR_ARG;
    double delta = (r_max - r_min) / bins;
    for (int b = 0; b < bins; ++b) edges[b] = r_min + b * delta;
    edges[bins] = r_max;
    return ORC_OK;
}

typedef struct {
    const double *b;
    const double *pts;
    const double *xq;
    int64_t iq;
    int exclude_ii;
    const double *edges;
    int bins;
    uint64_t *counts;
} rdf_ctx;

static void rdf_visit(void *vctx, int64_t j) {
    rdf_ctx *R = (rdf_ctx *)vctx;
    if (R->exclude_ii && j == R->iq) return;
    double d[3];
    min_image(R->b, R->xq, R->pts + 3 * j, d);
    double r = sqrt(r2_of(d));
    if (!(r >= R->edges[0] && r < R->edges[R->bins])) return;
    /* the bin b with R_b <= r < R_{b+1}: a plain linear scan over the edges */
    int bin = 0;
    while (bin + 1 < R->bins && R->edges[bin + 1] <= r) ++bin;
    R->counts[bin]++;
}

/*
 * Adds, for every query q in [q0, q1), the number of points j (j != q when exclude_ii)
 * with R_b <= r < R_{b+1} to counts[b] (ordered pairs).  Cells must have been built with
 * r_cell >= r_max (or nc == NULL for brute force).
 */
int orc_rdf(const double *b, const double *pts, int64_t n, const int32_t *nc, const int64_t *cell_start,
            const int64_t *order, const double *qpts, int64_t q0, int64_t q1, int bins, double r_min,
            double r_max, int exclude_ii, uint64_t *counts) {
    if (bins <= 0 || !(r_max > r_min) || r_min < 0.0 || q1 < q0) return ORC_ERR_ARG;
    if (!(r_max < 0.5 * min_width(b))) return ORC_ERR_BOX_TOO_SMALL;
    double *edges = (double *)malloc(sizeof(double) * (bins + 1));
    if (!edges) return ORC_ERR_OOM;
    orc_rdf_edges(bins, r_min, r_max, edges);
    cells_t C = {b, pts, nc, cell_start, order};
    rdf_ctx R = {b, pts, NULL, 0, exclude_ii, edges, bins, counts};
    for (int64_t q = q0; q < q1; ++q) {
        R.xq = qpts + 3 * q;
        R.iq = q;
        if (nc)
            for_candidates(&C, R.xq, 1, rdf_visit, &R);
        else
            for (int64_t j = 0; j < n; ++j) rdf_visit(&R, j);
    }
    free(edges);
    return ORC_OK;
}

/* ----------------------------------------------------------------- Steinhardt */

static double factorial(int n) {
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

static double binom(int n, int k) { return factorial(n) / (factorial(k) * factorial(n - k)); }

/* Associated Legendre function P_l^m(x), 0 <= m <= l, with the Condon-Shortley phase,
 * from the explicit sum P_l(x) = 2^-l sum_k (-1)^k C(l,k) C(2l-2k,l) x^(l-2k) and
 * P_l^m = (-1)^m (1-x^2)^(m/2) d^m/dx^m P_l.  sin_theta = (1-x^2)^(1/2) is passed in. */
static double assoc_legendre(int l, int m, double x, double sin_theta) {
    double s = 0.0;
    for (int k = 0; 2 * k <= l - m; ++k) {
        int p = l - 2 * k;
        double c = ((k & 1) ? -1.0 : 1.0) * binom(l, k) * binom(2 * l - 2 * k, l) * factorial(p) / factorial(p - m);
        s += c * pow(x, p - m);
    }
    s /= pow(2.0, l);
    return ((m & 1) ? -1.0 : 1.0) * pow(sin_theta, m) * s;
}

static double legendre(int l, double x) { return assoc_legendre(l, 0, x, 0.0); }

/* dP_l/dx from the same explicit sum. */
static double legendre_deriv(int l, double x) {
    double s = 0.0;
    for (int k = 0; 2 * k < l; ++k) {
        int p = l - 2 * k;
        double c = ((k & 1) ? -1.0 : 1.0) * binom(l, k) * binom(2 * l - 2 * k, l);
        s += c * p * pow(x, p - 1);
    }
    return s / pow(2.0, l);
}

/* Orthonormal spherical harmonic Y_l^m at the direction of (x, y, z), any m in [-l, l]:
 * Y_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) P_l^m(cos theta) e^{i m phi},
 * Y_l^{-m} = (-1)^m conj(Y_l^m). */
int orc_ylm(int l, int m, double x, double y, double z, double *re, double *im) {
    if (l < 0 || m < -l || m > l) return ORC_ERR_ARG;
    int am = m < 0 ? -m : m;
    double r = sqrt(x * x + y * y + z * z);
    double ct = z / r;
    double st = sqrt(x * x + y * y) / r;
    double phi = atan2(y, x);
    double norm = sqrt((2 * l + 1) / (4.0 * M_PI) * factorial(l - am) / factorial(l + am));
    double p = norm * assoc_legendre(l, am, ct, st);
    double yr = p * cos(am * phi), yi = p * sin(am * phi);
    if (m < 0) {
        double sg = (am & 1) ? -1.0 : 1.0;
        yr = sg * yr;
        yi = -sg * yi;
    }
    *re = yr;
    *im = yi;
    return ORC_OK;
}

/*
 * Steinhardt q_l from its definition (Steinhardt, Nelson, Ronchetti 1983, cited in the
 * "Analysis Modules" section): Q_lm(i) = (1/n_i) sum_j Y_lm(u_ij),
 * q_l(i) = sqrt(4 pi/(2l+1) sum_{m=-l..l} |Q_lm(i)|^2), u_ij the minimum-image bond
 * direction.  Neighbors of particle i are nl_j[offsets[i] .. offsets[i+1]).
 * Particles listed in `which` (or all n when which == NULL, nwhich ignored) are
 * evaluated.  Qlm (optional) receives Q_lm for m = 0..l as (re, im) pairs per particle.
 */
int orc_steinhardt_ylm(const double *b, const double *pts, int64_t n, const int64_t *offsets,
                       const int64_t *nl_j, int l, const int64_t *which, int64_t nwhich, double *q,
                       double *Qlm) {
    if (l < 0 || l > 16) return ORC_ERR_ARG;
    int64_t cnt = which ? nwhich : n;
    for (int64_t t = 0; t < cnt; ++t) {
        int64_t i = which ? which[t] : t;
        int64_t nb = offsets[i + 1] - offsets[i];
        double sum = 0.0;
        for (int m = -l; m <= l; ++m) {
            double re = 0.0, im = 0.0;
            for (int64_t e = offsets[i]; e < offsets[i + 1]; ++e) {
                double d[3], yr, yi;
                min_image(b, pts + 3 * i, pts + 3 * nl_j[e], d);
                orc_ylm(l, m, d[0], d[1], d[2], &yr, &yi);
                re += yr;
                im += yi;
            }
            if (nb > 0) {
                re /= nb;
                im /= nb;
            }
            sum += re * re + im * im;
            if (Qlm && m >= 0) {
                Qlm[(t * (l + 1) + m) * 2 + 0] = re;
                Qlm[(t * (l + 1) + m) * 2 + 1] = im;
            }
        }
        q[t] = nb > 0 ? sqrt(4.0 * M_PI / (2 * l + 1) * sum) : 0.0;
    }
    return ORC_OK;
}

/* Same q_l through the addition theorem: q_l(i) = (1/n_i) sqrt(sum_j sum_k P_l(u_j . u_k)). */
int orc_steinhardt_legendre(const double *b, const double *pts, int64_t n, const int64_t *offsets,
                            const int64_t *nl_j, int l, const int64_t *which, int64_t nwhich, double *q) {
    if (l < 0 || l > 16) return ORC_ERR_ARG;
    int64_t cnt = which ? nwhich : n;
    for (int64_t t = 0; t < cnt; ++t) {
        int64_t i = which ? which[t] : t;
        int64_t nb = offsets[i + 1] - offsets[i];
        double S = 0.0;
        for (int64_t e = offsets[i]; e < offsets[i + 1]; ++e) {
            double dj[3];
            min_image(b, pts + 3 * i, pts + 3 * nl_j[e], dj);
            double rj = sqrt(r2_of(dj));
            for (int64_t f = offsets[i]; f < offsets[i + 1]; ++f) {
                double dk[3];
                min_image(b, pts + 3 * i, pts + 3 * nl_j[f], dk);
                double rk = sqrt(r2_of(dk));
                double c = (dj[0] * dk[0] + dj[1] * dk[1] + dj[2] * dk[2]) / (rj * rk);
                S += legendre(l, c);
            }
        }
        q[t] = (nb > 0 && S > 0.0) ? sqrt(S) / nb : 0.0;
    }
    return ORC_OK;
}

/*
 * Gradient of Q = (1/n) sum_i q_l(i) with respect to every coordinate, neighbor list
 * held fixed, from the addition-theorem form: with S_i = sum_jk P_l(c_jk),
 * dq_i/dd_ij = (1/(n_i sqrt(S_i))) (I - u_j u_j^T)/|d_ij| sum_k P_l'(c_jk) u_k,
 * d_ij = x_j - x_i, so x_j gains it and x_i loses it.  grad is (n, 3), overwritten.
 */
int orc_q_grad(const double *b, const double *pts, int64_t n, const int64_t *offsets, const int64_t *nl_j,
               int l, double *grad) {
    if (l < 0 || l > 16) return ORC_ERR_ARG;
    memset(grad, 0, sizeof(double) * 3 * n);
    double *u = NULL, *rr = NULL;
    int64_t cap = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t nb = offsets[i + 1] - offsets[i];
        if (nb == 0) continue;
        if (nb > cap) {
            cap = nb;
            free(u);
            free(rr);
            u = (double *)malloc(sizeof(double) * 3 * cap);
            rr = (double *)malloc(sizeof(double) * cap);
            if (!u || !rr) {
                free(u);
                free(rr);
                return ORC_ERR_OOM;
            }
        }
        for (int64_t e = 0; e < nb; ++e) {
            double d[3];
            min_image(b, pts + 3 * i, pts + 3 * nl_j[offsets[i] + e], d);
            rr[e] = sqrt(r2_of(d));
            for (int c = 0; c < 3; ++c) u[3 * e + c] = d[c] / rr[e];
        }
        double S = 0.0;
        for (int64_t e = 0; e < nb; ++e)
            for (int64_t f = 0; f < nb; ++f)
                S += legendre(l, u[3 * e] * u[3 * f] + u[3 * e + 1] * u[3 * f + 1] + u[3 * e + 2] * u[3 * f + 2]);
        if (!(S > 0.0)) continue;
        double pref = 1.0 / (nb * sqrt(S) * n);
        for (int64_t e = 0; e < nb; ++e) {
            double g[3] = {0.0, 0.0, 0.0};
            for (int64_t f = 0; f < nb; ++f) {
                double c = u[3 * e] * u[3 * f] + u[3 * e + 1] * u[3 * f + 1] + u[3 * e + 2] * u[3 * f + 2];
                double dp = legendre_deriv(l, c);
                for (int k = 0; k < 3; ++k) g[k] += dp * u[3 * f + k];
            }
            double ug = u[3 * e] * g[0] + u[3 * e + 1] * g[1] + u[3 * e + 2] * g[2];
            int64_t j = nl_j[offsets[i] + e];
            for (int k = 0; k < 3; ++k) {
                double gk = pref * (g[k] - ug * u[3 * e + k]) / rr[e];
                grad[3 * j + k] += gk;
                grad[3 * i + k] -= gk;
            }
        }
    }
    free(u);
    free(rr);
    return ORC_OK;
}

/* Per-bond spherical harmonics (LocalDescriptors, global orientation): for each pair e,
 * the minimum-image bond d = x_j - q_i and Y_lm(d) for l = 0..lmax with m = -l..l
 * (negative_m) or m = 0..l, in that order, written as (re, im) pairs; coincident points
 * give zeros. */
int orc_descriptors(const double *b, const double *pts, const double *qpts, int64_t m, const int64_t *qi,
                    const int64_t *pj, int lmax, int negative_m, double *out) {
    if (lmax < 0 || lmax > 16) return ORC_ERR_ARG;
    int nsph = negative_m ? (lmax + 1) * (lmax + 1) : (lmax + 1) * (lmax + 2) / 2;
    for (int64_t e = 0; e < m; ++e) {
        double d[3];
        min_image(b, qpts + 3 * qi[e], pts + 3 * pj[e], d);
        double r2 = r2_of(d);
        int o = 0;
        for (int l = 0; l <= lmax; ++l) {
            for (int mm = negative_m ? -l : 0; mm <= l; ++mm) {
                double yr = 0.0, yi = 0.0;
                if (r2 > 0.0) orc_ylm(l, mm, d[0], d[1], d[2], &yr, &yi);
                out[(e * nsph + o) * 2 + 0] = yr;
                out[(e * nsph + o) * 2 + 1] = yi;
                ++o;
            }
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ PMFT */

/* PMFT in the plane (Section "Potentials of Mean Force and Torque", Fig. 6): each bond
 * e = (i, j) is the minimum-image d = x_j - q_i written in the frame of query particle
 * i, whose orientation is the angle theta_i about z (the bond turned by -theta_i):
 *   x' = cos(theta_i) d_x + sin(theta_i) d_y,   y' = cos(theta_i) d_y - sin(theta_i) d_x,
 * counted in bin (floor((x' + x_max) / dx), floor((y' + y_max) / dy)) with
 * dx = 2 x_max / bx, dy = 2 y_max / by (an index of bx clamps to bx - 1) when
 * -x_max <= x' < x_max and -y_max <= y' < y_max.  counts (bx, by), x major, are added
 * to; xy_out (NULL or m pairs) receives (x', y'). */
int orc_pmftxy(const double *b, const double *pts, const double *qpts, const double *theta, int64_t m,
               const int64_t *qi, const int64_t *pj, double x_max, double y_max, int bx, int by, int64_t *counts,
               double *xy_out) {
    if (!(x_max > 0.0) || !(y_max > 0.0) || bx <= 0 || by <= 0) return ORC_ERR_ARG;
    const double dx = 2.0 * x_max / bx, dy = 2.0 * y_max / by;
    for (int64_t e = 0; e < m; ++e) {
        double d[3];
        min_image(b, qpts + 3 * qi[e], pts + 3 * pj[e], d);
        const double c = cos(theta[qi[e]]), s = sin(theta[qi[e]]);
        const double xr = c * d[0] + s * d[1];
        const double yr = c * d[1] - s * d[0];
        if (xy_out) {
            xy_out[2 * e] = xr;
            xy_out[2 * e + 1] = yr;
        }
        if (!(xr >= -x_max && xr < x_max && yr >= -y_max && yr < y_max)) continue;
        int ix = (int)floor((xr + x_max) / dx);
        int iy = (int)floor((yr + y_max) / dy);
        if (ix > bx - 1) ix = bx - 1;
        if (iy > by - 1) iy = by - 1;
        counts[(int64_t)ix * by + iy] += 1;
    }
    return ORC_OK;
}
