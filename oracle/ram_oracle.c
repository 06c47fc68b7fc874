/*
 * FP64 CPU oracle for the RAM (Rapid Advection Algorithm on Arbitrary Meshes)
 * bulk-velocity shift step and the residual upwind step (Benitez-Llambay et al.,
 * arXiv 2305.05362).
 *
 * THIS FILE IS TEST INFRASTRUCTURE. It is the slow, plain reference that the CUDA
 * library is checked against.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code with the CUDA
 * path (no headers, no helpers, no tables) and must never be used as a fallback.
 *
 * Everything is FP64, single row at a time, written in the order of the paper:
 *   Sec. 2          nodes x_{-1/2} < ... < x_{N-1/2}, widths, masses M_i = Q_i dx_i (Eq. 3)
 *   Sec. 3.1        reconstruction q_i: PLM with the van Leer limiter, PPM (App. A)
 *   Sec. 3.2        shifted edges (Eq. 16) and the remapped mass (Eq. 18)
 *   Sec. 3.3        Q = M / dx (Eq. 26)
 *   Eqs. 5-6        operator splitting: shift first, then the residual dv step
 * plus a hand-derived transpose of the linear (limiter-off, donor) step.
 *
 * Readings of points where the paper is silent or garbled:
 *   - content moves by +s (x~ = x - s, Sec. 3.2); s is reduced with a floor-mod.
 *   - an edge exactly on a node belongs to the cell on its right (the <= of Eq. 16).
 *   - App. A weights omega~_1..3 are read with SUMS of widths where the text prints
 *     products (the products are dimensionally inconsistent; Colella & Woodward 1984).
 *   - the delta<Q> limiter keeps the sign of delta<Q> (App. A.2).
 *   - the third PPM constraint reads (Q_R - Q_L)^2; the two overshoot fixes are
 *     exclusive and use the values left by the extremum test (App. A.2).
 *   - the PPM parabola variable is xi = (x - x_{i-1/2}) / dx_i in [0, 1] (Sec. 3.1).
 *   - order 4 is not in the paper: the in-cell cumulative is the mean of the two
 *     quartic interpolants of the cumulative mass through the node sets
 *     {i-5/2..i+3/2} and {i-3/2..i+5/2}.  With the limiter on it is scaled toward
 *     the cell mean (the maximum-principle scaling limiter of Zhang & Shu 2010):
 *     q~ = Q_i + theta (q - Q_i), theta the largest value in [0, 1] that keeps q~
 *     inside [min, max] of Q_{i-1}, Q_i, Q_{i+1} on the whole cell; the mean, and so
 *     the mass, is unchanged.
 *   - the fourth-order cell-average correction of Sec. 3.1 (A4): the stored values
 *     are point values Q_i; the remap works on <Q>_i = Q_i + (Q_{i+1} - 2Q_i +
 *     Q_{i-1}) / 24 (PPM) and the new point values solve the same relation for the
 *     remapped averages (a periodic tridiagonal system), so sum_i Q_i dx_i is
 *     conserved on a periodic uniform mesh; the residual step then acts on the point
 *     values.
 *   - limiter off: PLM takes the centred slope, PPM skips both limiter stages.
 *   - the residual step (only named in the paper, Sec. 4 and Eq. 6) is a flux-form
 *     upwind step at the interfaces: donor cell, or van Leer (PLM, van Leer slope,
 *     evaluated at the midpoint of the swept region), repeated nsub times with dt/nsub.
 *   - exact-cover copy rule: when both shifted edges of output cell i fall exactly
 *     on the two nodes of one source cell of the same width, Q'_i = Q_p exactly, so
 *     that a whole-cell shift is the cyclic permutation of Sec. 1 (Eq. 8).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_MESH 2
#define ORC_ERR_CFL 3
#define ORC_ERR_NOMEM 6

#define SCHEME_DONOR 0
#define SCHEME_VANLEER 1

/* ------------------------------------------------------------------------- */
/* mesh helpers (Sec. 2)                                                      */
/* ------------------------------------------------------------------------- */

/* periodic cell index */
static int cyc(long i, int n)
{
    long k = i % n;
    if (k < 0) k += n;
    return (int)k;
}

/* widths dx_i = x_{i+1/2} - x_{i-1/2}; returns nonzero if the nodes are not
 * strictly increasing (Sec. 2 requires a monotonic node sequence). */
static int widths(int n, const double *x, double *dx)
{
    for (int i = 0; i < n; ++i) {
        dx[i] = x[i + 1] - x[i];
        if (!(dx[i] > 0.0)) return ORC_ERR_MESH;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Step 1: reconstruction (Sec. 3.1, App. A)                                  */
/* ------------------------------------------------------------------------- */

/* PLM slope sigma_i (per unit length) for every cell.
 * Limiter on: van Leer harmonic slope, zero at extrema (Sec. 3.1).
 * Limiter off: centred slope through the neighbouring cell values. */
static void plm_slopes(int n, const double *dx, const double *q, int limiter,
                       double *sigma)
{
    for (int i = 0; i < n; ++i) {
        int im = cyc(i - 1, n), ip = cyc(i + 1, n);
        /* centre spacings x_i - x_{i-1} and x_{i+1} - x_i */
        double hl = 0.5 * (dx[im] + dx[i]);
        double hr = 0.5 * (dx[i] + dx[ip]);
        if (limiter) {
            double dl = (q[i] - q[im]) / hl;
            double dr = (q[ip] - q[i]) / hr;
            if (dl * dr <= 0.0)
                sigma[i] = 0.0;
            else
                sigma[i] = 2.0 * dl * dr / (dl + dr);
        } else {
            sigma[i] = (q[ip] - q[im]) / (hl + hr);
        }
    }
}

/* PPM coefficients (QL, QR, Q6) for every cell (Sec. 3.1 and App. A, with the
 * readings listed in the header). */
static void ppm_coefs(int n, const double *dx, const double *q, int limiter,
                      double *ql, double *qr, double *q6)
{
    double *dq = (double *)malloc(sizeof(double) * (size_t)n);
    double *face = (double *)malloc(sizeof(double) * (size_t)n); /* face[i] = <Q>_{i+1/2} */
    /* delta<Q>_i, App. A.1 */
    for (int i = 0; i < n; ++i) {
        int im = cyc(i - 1, n), ip = cyc(i + 1, n);
        double a = dx[im], b = dx[i], c = dx[ip];
        double d = b / (a + b + c) *
                   ((2.0 * a + b) / (b + c) * (q[ip] - q[i]) +
                    (b + 2.0 * c) / (a + b) * (q[i] - q[im]));
        if (limiter) {
            /* App. A.2, first stage */
            double up = q[ip] - q[i], dn = q[i] - q[im];
            if (up * dn > 0.0) {
                double m = fabs(d);
                if (2.0 * fabs(dn) < m) m = 2.0 * fabs(dn);
                if (2.0 * fabs(up) < m) m = 2.0 * fabs(up);
                d = (d >= 0.0) ? m : -m;
            } else {
                d = 0.0;
            }
        }
        dq[i] = d;
    }
    /* interface values <Q>_{i+1/2}, App. A.1 */
    for (int i = 0; i < n; ++i) {
        int im = cyc(i - 1, n), ip = cyc(i + 1, n), ip2 = cyc(i + 2, n);
        double hm = dx[im], h0 = dx[i], h1 = dx[ip], h2 = dx[ip2];
        double w1 = 2.0 * h1 * h0 / (h0 + h1) *
                    ((hm + h0) / (2.0 * h0 + h1) - (h2 + h1) / (2.0 * h1 + h0));
        double w2 = -h0 * (hm + h0) / (2.0 * h0 + h1);
        double w3 = h1 * (h1 + h2) / (h0 + 2.0 * h1);
        double sum4 = hm + h0 + h1 + h2;
        face[i] = q[i] + h0 / (h0 + h1) * (q[ip] - q[i]) +
                  (w1 * (q[ip] - q[i]) + w2 * dq[ip] + w3 * dq[i]) / sum4;
    }
    for (int i = 0; i < n; ++i) {
        double L = face[cyc(i - 1, n)], R = face[i], Q = q[i];
        if (limiter) {
            /* App. A.2, second stage */
            if ((R - Q) * (Q - L) <= 0.0) {
                L = Q;
                R = Q;
            } else {
                double dd = R - L;
                double qa = Q - 0.5 * (L + R);
                if (dd * qa > dd * dd / 6.0)
                    L = 3.0 * Q - 2.0 * R;
                else if (-dd * dd / 6.0 > dd * qa)
                    R = 3.0 * Q - 2.0 * L;
            }
        }
        ql[i] = L;
        qr[i] = R;
        q6[i] = 6.0 * Q - 3.0 * (L + R);
    }
    free(dq);
    free(face);
}

/* Reconstruction state of one row. */
typedef struct {
    int n, order;
    const double *q;
    double *dx;
    double *m;      /* masses M_i = Q_i dx_i (Eq. 3) */
    double *c0, *c1, *c2; /* PLM: (Q, sigma, -); PPM: (QL, QR, Q6); order 4: (theta, -, -) */
    int limited;          /* order 4 with the scaling limiter */
} recon_t;

static double quartic_theta(const recon_t *r, int i);

static int recon_build(recon_t *r, int n, const double *x, const double *q,
                       int order, int limiter)
{
    r->n = n;
    r->order = order;
    r->q = q;
    r->dx = (double *)malloc(sizeof(double) * (size_t)n);
    r->m = (double *)malloc(sizeof(double) * (size_t)n);
    r->c0 = (double *)calloc((size_t)n, sizeof(double));
    r->c1 = (double *)calloc((size_t)n, sizeof(double));
    r->c2 = (double *)calloc((size_t)n, sizeof(double));
    if (!r->dx || !r->m || !r->c0 || !r->c1 || !r->c2) return ORC_ERR_NOMEM;
    int st = widths(n, x, r->dx);
    if (st) return st;
    for (int i = 0; i < n; ++i) r->m[i] = q[i] * r->dx[i];
    r->limited = 0;
    if (order == 2) {
        for (int i = 0; i < n; ++i) r->c0[i] = q[i];
        plm_slopes(n, r->dx, q, limiter, r->c1);
    } else if (order == 3) {
        ppm_coefs(n, r->dx, q, limiter, r->c0, r->c1, r->c2);
    } else if (order == 4) {
        for (int i = 0; i < n; ++i) r->c0[i] = 1.0;
        if (limiter) {
            for (int i = 0; i < n; ++i) r->c0[i] = quartic_theta(r, i);
            r->limited = 1;
        }
    } else {
        return ORC_ERR_ARG;
    }
    return ORC_OK;
}

static void recon_free(recon_t *r)
{
    free(r->dx);
    free(r->m);
    free(r->c0);
    free(r->c1);
    free(r->c2);
}

/* Order-4 cumulative: Lagrange basis weights of the two quartics at local
 * offset d (d = x - x_{i-1/2}).  Nodes z[0..5] are the six nodes
 * x_{i-5/2} .. x_{i+5/2} relative to x_{i-1/2}; the left quartic uses z[0..4],
 * the right one z[1..5].  w[k] = (l_left_k(d) + l_right_k(d)) / 2. */
static void quartic_pair_weights(const double z[6], double d, double w[6])
{
    for (int k = 0; k < 6; ++k) w[k] = 0.0;
    for (int side = 0; side < 2; ++side) {
        int lo = side, hi = side + 4;
        for (int k = lo; k <= hi; ++k) {
            double l = 1.0;
            for (int j = lo; j <= hi; ++j) {
                if (j == k) continue;
                l *= (d - z[j]) / (z[k] - z[j]);
            }
            w[k] += 0.5 * l;
        }
    }
}

static void quartic_nodes(const recon_t *r, int i, double z[6])
{
    int n = r->n;
    double a = r->dx[cyc(i - 2, n)], b = r->dx[cyc(i - 1, n)], c = r->dx[i];
    double d = r->dx[cyc(i + 1, n)], e = r->dx[cyc(i + 2, n)];
    z[0] = -(a + b);
    z[1] = -b;
    z[2] = 0.0;
    z[3] = c;
    z[4] = c + d;
    z[5] = c + d + e;
}

/* cumulative-mass values at the six nodes, relative to C(x_{i-1/2}) */
static void quartic_values(const recon_t *r, int i, double v[6])
{
    int n = r->n;
    double ma = r->m[cyc(i - 2, n)], mb = r->m[cyc(i - 1, n)], mc = r->m[i];
    double md = r->m[cyc(i + 1, n)], me = r->m[cyc(i + 2, n)];
    v[0] = -(ma + mb);
    v[1] = -mb;
    v[2] = 0.0;
    v[3] = mc;
    v[4] = mc + md;
    v[5] = mc + md + me;
}

/* G_i(d) = integral of q_i from x_{i-1/2} to x_{i-1/2} + d, 0 <= d <= dx_i
 * (the partial integrals of Eq. 18). */
static double cell_G(const recon_t *r, int i, double d)
{
    double h = r->dx[i];
    if (r->order == 2) {
        /* q = Q + sigma (x - x_i), x_i = x_{i-1/2} + h/2 */
        return r->c0[i] * d + 0.5 * r->c1[i] * (d * d - d * h);
    } else if (r->order == 3) {
        double xi = d / h;
        double L = r->c0[i], R = r->c1[i], S = r->c2[i];
        return h * (L * xi + 0.5 * (R - L) * xi * xi +
                    S * (0.5 * xi * xi - xi * xi * xi / 3.0));
    } else {
        double z[6], v[6], w[6], g = 0.0;
        quartic_nodes(r, i, z);
        quartic_values(r, i, v);
        quartic_pair_weights(z, d, w);
        for (int k = 0; k < 6; ++k) g += w[k] * v[k];
        if (r->limited) {
            /* the profile scaled toward the mean: G~ = theta G + (1 - theta) Q d */
            double th = r->c0[i];
            g = th * g + (1.0 - th) * r->q[i] * d;
        }
        return g;
    }
}

/* Order-4 scaling limiter: theta in [0, 1] such that Q_i + theta (q_i(x) - Q_i)
 * stays within [min, max] of Q_{i-1}, Q_i, Q_{i+1} over the cell.  q_i = dG_i/dx is
 * a cubic; its power-basis coefficients come from G_i at xi = 1/4, 1/2, 3/4, 1 (a
 * 4 x 4 Vandermonde system, Gaussian elimination), and its extremes are at the
 * cell's ends or at the real roots of q' inside the cell. */
static double quartic_theta(const recon_t *r, int i)
{
    int n = r->n;
    double h = r->dx[i], Q = r->q[i];
    double qm = r->q[cyc(i - 1, n)], qp = r->q[cyc(i + 1, n)];
    double lo = Q, hi = Q;
    if (qm < lo) lo = qm;
    if (qp < lo) lo = qp;
    if (qm > hi) hi = qm;
    if (qp > hi) hi = qp;
    /* G(xi h) / h = a1 xi + a2 xi^2 + a3 xi^3 + a4 xi^4 */
    double A[4][5];
    recon_t u = *r;
    u.limited = 0;
    for (int k = 0; k < 4; ++k) {
        double xi = 0.25 * (k + 1), p = xi;
        for (int j = 0; j < 4; ++j) {
            A[k][j] = p;
            p *= xi;
        }
        A[k][4] = cell_G(&u, i, xi * h) / h;
    }
    for (int c = 0; c < 4; ++c) {
        int piv = c;
        for (int k = c + 1; k < 4; ++k)
            if (fabs(A[k][c]) > fabs(A[piv][c])) piv = k;
        for (int j = 0; j < 5; ++j) {
            double t = A[c][j];
            A[c][j] = A[piv][j];
            A[piv][j] = t;
        }
        for (int k = c + 1; k < 4; ++k) {
            double f = A[k][c] / A[c][c];
            for (int j = c; j < 5; ++j) A[k][j] -= f * A[c][j];
        }
    }
    double a[4];
    for (int c = 3; c >= 0; --c) {
        double t = A[c][4];
        for (int j = c + 1; j < 4; ++j) t -= A[c][j] * a[j];
        a[c] = t / A[c][c];
    }
    /* q(xi) = a1 + 2 a2 xi + 3 a3 xi^2 + 4 a4 xi^3; q'(xi) = 2 a2 + 6 a3 xi + 12 a4 xi^2 */
    double cand[4];
    int nc = 0;
    cand[nc++] = 0.0;
    cand[nc++] = 1.0;
    double qa = 12.0 * a[3], qb = 6.0 * a[2], qc = 2.0 * a[1];
    if (fabs(qa) > 1e-300) {
        double disc = qb * qb - 4.0 * qa * qc;
        if (disc >= 0.0) {
            double sq = sqrt(disc);
            double r1 = (-qb - sq) / (2.0 * qa), r2 = (-qb + sq) / (2.0 * qa);
            if (r1 > 0.0 && r1 < 1.0) cand[nc++] = r1;
            if (r2 > 0.0 && r2 < 1.0) cand[nc++] = r2;
        }
    } else if (fabs(qb) > 1e-300) {
        double r1 = -qc / qb;
        if (r1 > 0.0 && r1 < 1.0) cand[nc++] = r1;
    }
    double qmax = -INFINITY, qmin = INFINITY;
    for (int k = 0; k < nc; ++k) {
        double xi = cand[k];
        double v = a[0] + xi * (2.0 * a[1] + xi * (3.0 * a[2] + xi * 4.0 * a[3]));
        if (v > qmax) qmax = v;
        if (v < qmin) qmin = v;
    }
    double th = 1.0;
    if (qmax > hi && qmax - Q > 0.0) {
        double t = (hi - Q) / (qmax - Q);
        if (t < th) th = t;
    }
    if (qmin < lo && qmin - Q < 0.0) {
        double t = (lo - Q) / (qmin - Q);
        if (t < th) th = t;
    }
    if (th < 0.0) th = 0.0;
    return th;
}

/* ------------------------------------------------------------------------- */
/* Step 2: locate the shifted edges (Eq. 16)                                  */
/* ------------------------------------------------------------------------- */

/* reduce a shift to [0, L) */
static double reduce_shift(double s, double L)
{
    double r = s - L * floor(s / L);
    if (r >= L) r -= L;
    if (r < 0.0) r += L;
    if (r >= L) r = 0.0;
    return r;
}

/* binary search: the p with x[p] <= y < x[p+1], y in [x[0], x[n]) */
static int locate(int n, const double *x, double y)
{
    int lo = 0, hi = n; /* invariant: x[lo] <= y < x[hi] */
    while (hi - lo > 1) {
        int mid = lo + (hi - lo) / 2;
        if (x[mid] <= y)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

/* All shifted edges of a row.  Edge j (node x_{j-1/2}, j = 0..n-1) moves to
 * y_j = x_{j-1/2} - s reduced into [x_{-1/2}, x_{N-1/2}); p_j is the source cell
 * holding it and d_j = y_j - x_{p_j - 1/2} its offset (Eq. 16).  The last node is
 * the first one moved by a period, so p(N) = p(0) (Eq. 18). */
static void shifted_edges(int n, const double *x, double sred, int *p, double *y,
                          double *d)
{
    double L = x[n] - x[0];
    for (int j = 0; j < n; ++j) {
        double yy = x[j] - sred;
        if (yy < x[0]) yy += L;
        if (yy >= x[n]) yy -= L;
        if (yy < x[0]) yy = x[0];
        int pp = locate(n, x, yy);
        p[j] = pp;
        y[j] = yy;
        d[j] = yy - x[pp];
    }
}

/* Output-cell description shared by the forward map and its transpose. */
typedef struct {
    int pl, pr;       /* source cells holding the left and right shifted edges */
    double dl, dr;    /* offsets of the edges inside those cells */
    int same;         /* both edges in one cell, no seam crossing */
    int nwhole;       /* number of whole source cells strictly between pl and pr */
    int copy;         /* exact-cover copy rule */
} cover_t;

static void cover_cell(int n, const double *dx, const int *p, const double *y,
                       const double *d, int i, cover_t *c)
{
    int jr = cyc(i + 1, n);
    int pl = p[i], pr = p[jr];
    double dl = d[i], dr = d[jr];
    /* the output interval crosses the periodic seam when its right end lies left
     * of its left end after the reduction (a single cell always spans the period) */
    int wrap = (y[jr] <= y[i]) || (n == 1);
    c->pl = pl;
    c->pr = pr;
    c->dl = dl;
    c->dr = dr;
    c->same = (!wrap && pl == pr);
    if (c->same)
        c->nwhole = 0;
    else if (wrap)
        c->nwhole = pr - pl - 1 + n;
    else
        c->nwhole = pr - pl - 1;
    c->copy = (dl == 0.0 && dr == 0.0 && c->nwhole == 0 && !c->same &&
               pr == cyc(pl + 1, n) && dx[pl] == dx[i]);
}

/* edge arrays of one row */
typedef struct {
    int *p;
    double *y, *d;
} edges_t;

static void edges_build(edges_t *e, int n, const double *x, double sred)
{
    e->p = (int *)malloc(sizeof(int) * (size_t)n);
    e->y = (double *)malloc(sizeof(double) * (size_t)n);
    e->d = (double *)malloc(sizeof(double) * (size_t)n);
    shifted_edges(n, x, sred, e->p, e->y, e->d);
}

static void edges_free(edges_t *e)
{
    free(e->p);
    free(e->y);
    free(e->d);
}

/* ------------------------------------------------------------------------- */
/* The shift: Eqs. 15-18 and 26                                               */
/* ------------------------------------------------------------------------- */

int oracle_shift(int n, const double *x, const double *q_in, int order, int limiter,
                 double s, double *q_out)
{
    if (n < 1 || !x || !q_in || !q_out) return ORC_ERR_ARG;
    if (!isfinite(s)) return ORC_ERR_ARG;
    recon_t r;
    int st = recon_build(&r, n, x, q_in, order, limiter);
    if (st) {
        recon_free(&r);
        return st;
    }
    double L = x[n] - x[0];
    double sred = reduce_shift(s, L);
    edges_t e;
    edges_build(&e, n, x, sred);
    for (int i = 0; i < n; ++i) {
        cover_t c;
        cover_cell(n, r.dx, e.p, e.y, e.d, i, &c);
        if (c.copy) {
            q_out[i] = q_in[c.pl];
            continue;
        }
        double mass;
        if (c.same) {
            mass = cell_G(&r, c.pl, c.dr) - cell_G(&r, c.pl, c.dl);
        } else {
            /* right part of the left cell, whole cells in between, left part of
             * the right cell (Eq. 18, with p(N) = p(0)) */
            mass = r.m[c.pl] - cell_G(&r, c.pl, c.dl);
            for (int k = 1; k <= c.nwhole; ++k) mass += r.m[cyc(c.pl + k, n)];
            mass += cell_G(&r, c.pr, c.dr);
        }
        q_out[i] = mass / r.dx[i]; /* Eq. 26 */
    }
    edges_free(&e);
    recon_free(&r);
    return ORC_OK;
}

/* Reconstruction coefficients, exposed so that tests can integrate q_i by an
 * independent quadrature.  out has 3 doubles per cell:
 * order 2 -> (Q_i, sigma_i, 0); order 3 -> (QL_i, QR_i, Q6_i). */
int oracle_reconstruct(int n, const double *x, const double *q, int order, int limiter,
                       double *out)
{
    if (n < 1 || (order != 2 && order != 3)) return ORC_ERR_ARG;
    recon_t r;
    int st = recon_build(&r, n, x, q, order, limiter);
    if (!st)
        for (int i = 0; i < n; ++i) {
            out[3 * i] = r.c0[i];
            out[3 * i + 1] = r.c1[i];
            out[3 * i + 2] = r.c2[i];
        }
    recon_free(&r);
    return st;
}

/* In-cell cumulative G_i(d) for a list of (cell, offset) pairs. */
int oracle_cell_cumulative(int n, const double *x, const double *q, int order,
                           int limiter, int npts, const int *cell, const double *d,
                           double *out)
{
    recon_t r;
    int st = recon_build(&r, n, x, q, order, limiter);
    if (!st)
        for (int k = 0; k < npts; ++k) out[k] = cell_G(&r, cyc(cell[k], n), d[k]);
    recon_free(&r);
    return st;
}

/* ------------------------------------------------------------------------- */
/* Residual step (Eq. 6): flux-form upwind with velocity dv at the interfaces   */
/* ------------------------------------------------------------------------- */

/* One sub-step.  dv[j] sits at node x_{j-1/2}; h is the sub-step length.
 * Returns ORC_ERR_CFL (after completing the update) if |dv h| exceeds the width
 * of the upwind cell anywhere. */
static int residual_substep(int n, const double *dx, const double *q, const double *dv,
                            double h, int scheme, double *q_next)
{
    int st = ORC_OK;
    double *sigma = NULL;
    double *flux = (double *)malloc(sizeof(double) * (size_t)n);
    if (scheme == SCHEME_VANLEER) {
        sigma = (double *)malloc(sizeof(double) * (size_t)n);
        plm_slopes(n, dx, q, 1, sigma);
    }
    for (int j = 0; j < n; ++j) {
        double c = dv[j] * h; /* signed swept length */
        int jm = cyc(j - 1, n);
        double qhat;
        if (c > 0.0) {
            qhat = q[jm];
            if (sigma) qhat += sigma[jm] * 0.5 * (dx[jm] - c);
            if (c > dx[jm]) st = ORC_ERR_CFL;
        } else if (c < 0.0) {
            qhat = q[j];
            if (sigma) qhat -= sigma[j] * 0.5 * (dx[j] + c);
            if (-c > dx[j]) st = ORC_ERR_CFL;
        } else {
            qhat = 0.0;
        }
        flux[j] = c * qhat;
    }
    for (int i = 0; i < n; ++i) q_next[i] = q[i] - (flux[cyc(i + 1, n)] - flux[i]) / dx[i];
    free(flux);
    free(sigma);
    return st;
}

int oracle_residual(int n, const double *x, const double *q_in, const double *dv,
                    double dt, int scheme, int nsub, double *q_out)
{
    if (n < 1 || nsub < 1 || (scheme != SCHEME_DONOR && scheme != SCHEME_VANLEER))
        return ORC_ERR_ARG;
    double *dx = (double *)malloc(sizeof(double) * (size_t)n);
    double *cur = (double *)malloc(sizeof(double) * (size_t)n);
    double *nxt = (double *)malloc(sizeof(double) * (size_t)n);
    int st = widths(n, x, dx);
    int cfl = ORC_OK;
    if (!st) {
        memcpy(cur, q_in, sizeof(double) * (size_t)n);
        double h = dt / nsub;
        for (int k = 0; k < nsub; ++k) {
            if (residual_substep(n, dx, cur, dv, h, scheme, nxt)) cfl = ORC_ERR_CFL;
            double *t = cur;
            cur = nxt;
            nxt = t;
        }
        memcpy(q_out, cur, sizeof(double) * (size_t)n);
    }
    free(dx);
    free(cur);
    free(nxt);
    return st ? st : cfl;
}

/* One RAM step: the shift by s, then the residual step (Eqs. 5-6).  dv may be NULL
 * (dv = 0, the residual is the identity). */
int oracle_step(int n, const double *x, const double *q_in, int order, int limiter,
                double s, const double *dv, double dt, int scheme, int nsub,
                double *q_out)
{
    double *tmp = (double *)malloc(sizeof(double) * (size_t)n);
    int st = oracle_shift(n, x, q_in, order, limiter, s, tmp);
    if (!st) {
        if (dv)
            st = oracle_residual(n, x, tmp, dv, dt, scheme, nsub, q_out);
        else
            memcpy(q_out, tmp, sizeof(double) * (size_t)n);
    }
    free(tmp);
    return st;
}

/* shift of one step from the bulk velocity, and the accumulated phase v0 t mod L */
double oracle_shift_from_velocity(double v0, double dt) { return v0 * dt; }

double oracle_phase_update(double phase, double v0, double dt, double L)
{
    return reduce_shift(phase + v0 * dt, L);
}

/* Batched driver over packed rows: row r owns cells [row_offset[r], row_offset[r+1])
 * and nodes nodes[row_offset[r] + r .. row_offset[r+1] + r] (or the first row's
 * nodes for every row when shared_mesh is set).  Rows are independent
 * (dimensional splitting, Sec. 3.5); OpenMP spreads them over host threads when
 * the library was built with it. */
int oracle_step_rows(int n_rows, const long long *row_offset, const double *nodes,
                     int shared_mesh, const signed char *order, int limiter,
                     const double *shift, const double *dv, double dt, int scheme,
                     const int *nsub, const double *q_in, double *q_out)
{
    int st_all = ORC_OK;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int r = 0; r < n_rows; ++r) {
        long long b = row_offset[r];
        int n = (int)(row_offset[r + 1] - b);
        const double *x = shared_mesh ? nodes : nodes + b + r;
        int st = oracle_step(n, x, q_in + b, order[r], limiter, shift[r],
                             dv ? dv + b : NULL, dt, scheme, nsub ? nsub[r] : 1,
                             q_out + b);
        if (st) {
#ifdef _OPENMP
#pragma omp critical
#endif
            if (!st_all || st_all == ORC_ERR_CFL) st_all = st;
        }
    }
    return st_all;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    int t = 1;
#pragma omp parallel
    {
#pragma omp master
        t = omp_get_num_threads();
    }
    return t;
#else
    return 1;
#endif
}

double oracle_shift_from_velocity(double v0, double dt);

/* ------------------------------------------------------------------------- */
/* Two dimensions by dimensional splitting (Sec. 3.5): the radial sweep          */
/* ------------------------------------------------------------------------- */

/* Flux-form upwind advection in r on a polar mesh (cylindrical geometry), one
 * sweep of length dt over every azimuthal column: rings j = 0..nr-1 between the
 * radii rf[j] < rf[j+1]; q[j * nphi + i] is cell (ring j, azimuthal cell i);
 * vr[j * nphi + i] is the radial velocity on face j (radius rf[j], between rings
 * j-1 and j), faces 0 and nr are closed (no flux).  Per unit angle, the face has
 * length rf[j] and ring j has area (rf[j+1]^2 - rf[j]^2) / 2:
 *   q'_j = q_j - dt (rf[j+1] F_{j+1} - rf[j] F_j) / area_j,
 * with F = vr q_up (donor) or vr times the upwind ring's van Leer profile (the
 * harmonic slope over the ring centres' spacings, Sec. 3.1) at the midpoint of
 * the swept interval.  Returns ORC_ERR_CFL (after the update) where |vr| dt
 * exceeds the upwind ring's width. */
int oracle_radial_upwind(int nr, int nphi, const double *rf, const double *q,
                         const double *vr, double dt, int scheme, double *q_out)
{
    if (nr < 1 || nphi < 1 || (scheme != SCHEME_DONOR && scheme != SCHEME_VANLEER))
        return ORC_ERR_ARG;
    for (int j = 0; j < nr; ++j)
        if (!(rf[j + 1] > rf[j]) || !(rf[j] >= 0.0)) return ORC_ERR_MESH;
    int st = ORC_OK;
    double *dr = (double *)malloc(sizeof(double) * (size_t)nr);
    double *col = (double *)malloc(sizeof(double) * (size_t)nr);
    double *sig = (double *)malloc(sizeof(double) * (size_t)nr);
    double *F = (double *)malloc(sizeof(double) * (size_t)(nr + 1));
    for (int j = 0; j < nr; ++j) dr[j] = rf[j + 1] - rf[j];
    for (int i = 0; i < nphi; ++i) {
        for (int j = 0; j < nr; ++j) col[j] = q[(size_t)j * nphi + i];
        /* van Leer slopes per unit length; zero at the closed ends */
        for (int j = 0; j < nr; ++j) {
            sig[j] = 0.0;
            if (scheme == SCHEME_VANLEER && j > 0 && j < nr - 1) {
                double dl = (col[j] - col[j - 1]) / (0.5 * (dr[j - 1] + dr[j]));
                double dq = (col[j + 1] - col[j]) / (0.5 * (dr[j] + dr[j + 1]));
                sig[j] = (dl * dq > 0.0) ? 2.0 * dl * dq / (dl + dq) : 0.0;
            }
        }
        F[0] = 0.0;
        F[nr] = 0.0;
        for (int j = 1; j < nr; ++j) {
            double v = vr[(size_t)j * nphi + i];
            double c = v * dt; /* signed swept length */
            double qh = 0.0;
            if (c > 0.0) {
                qh = col[j - 1] + sig[j - 1] * 0.5 * (dr[j - 1] - c);
                if (c > dr[j - 1]) st = ORC_ERR_CFL;
            } else if (c < 0.0) {
                qh = col[j] - sig[j] * 0.5 * (dr[j] + c);
                if (-c > dr[j]) st = ORC_ERR_CFL;
            }
            F[j] = v * qh;
        }
        for (int j = 0; j < nr; ++j) {
            double area = 0.5 * (rf[j + 1] * rf[j + 1] - rf[j] * rf[j]);
            q_out[(size_t)j * nphi + i] = col[j] - dt * (rf[j + 1] * F[j + 1] - rf[j] * F[j]) / area;
        }
    }
    free(dr);
    free(col);
    free(sig);
    free(F);
    return st;
}

/* The largest step for which neighbouring rings, turning at the angular rates
 * omega[j], shear by at most beta times the smallest azimuthal cell dphi_min
 * (the shear limit of dimensional splitting, Sec. 3.5):
 *   dt = beta dphi_min / max_j |omega[j+1] - omega[j]|  (infinite for a rigid rotation). */
double oracle_shear_dt(int nr, const double *omega, double dphi_min, double beta)
{
    double m = 0.0;
    for (int j = 0; j + 1 < nr; ++j) {
        double d = fabs(omega[j + 1] - omega[j]);
        if (d > m) m = d;
    }
    return m > 0.0 ? beta * dphi_min / m : INFINITY;
}

/* One split step of a polar disk: the RAM step of every ring (azimuthal shift by
 * omega[j] dt on the shared mesh phi, residual dvphi), then the radial sweep. */
int oracle_step_2d(int nr, int nphi, const double *phi, const double *rf, const double *omega,
                   const double *q_in, int order, int limiter, const double *dvphi, int scheme,
                   const int *nsub, const double *vr, double dt, double *q_out)
{
    double *mid = (double *)malloc(sizeof(double) * (size_t)nr * nphi);
    int st = ORC_OK;
    for (int j = 0; j < nr && st != ORC_ERR_ARG && st != ORC_ERR_MESH; ++j) {
        int sj = oracle_step(nphi, phi, q_in + (size_t)j * nphi, order, limiter,
                             oracle_shift_from_velocity(omega[j], dt),
                             dvphi ? dvphi + (size_t)j * nphi : NULL, dt, scheme,
                             nsub ? nsub[j] : 1, mid + (size_t)j * nphi);
        if (sj) st = sj;
    }
    if (st == ORC_OK || st == ORC_ERR_CFL) {
        int sr = oracle_radial_upwind(nr, nphi, rf, mid, vr, dt, scheme, q_out);
        if (sr) st = sr;
    }
    free(mid);
    return st;
}

/* ------------------------------------------------------------------------- */
/* Fourth-order cell-average correction (Sec. 3.1)                              */
/* ------------------------------------------------------------------------- */

/* <Q>_i = Q_i + (Q_{i+1} - 2 Q_i + Q_{i-1}) / 24, periodic. */
int oracle_a4_average(int n, const double *q, double *avg)
{
    if (n < 1) return ORC_ERR_ARG;
    for (int i = 0; i < n; ++i)
        avg[i] = q[i] + (q[cyc(i + 1, n)] - 2.0 * q[i] + q[cyc(i - 1, n)]) / 24.0;
    return ORC_OK;
}

/* The point values whose corrected averages are `avg`: the periodic tridiagonal
 * system Q_{i-1} + 22 Q_i + Q_{i+1} = 24 <Q>_i, solved by the Thomas algorithm
 * with the Sherman-Morrison correction for the two corner entries. */
int oracle_a4_point(int n, const double *avg, double *q)
{
    if (n < 1) return ORC_ERR_ARG;
    if (n == 1) {
        q[0] = avg[0];
        return ORC_OK;
    }
    if (n == 2) {
        /* 22 q0 + 2 q1 = 24 a0, 2 q0 + 22 q1 = 24 a1 */
        double det = 22.0 * 22.0 - 4.0;
        q[0] = (22.0 * 24.0 * avg[0] - 2.0 * 24.0 * avg[1]) / det;
        q[1] = (22.0 * 24.0 * avg[1] - 2.0 * 24.0 * avg[0]) / det;
        return ORC_OK;
    }
    double *b = (double *)malloc(sizeof(double) * (size_t)n);
    double *y = (double *)malloc(sizeof(double) * (size_t)n);
    double *z = (double *)malloc(sizeof(double) * (size_t)n);
    double *u = (double *)calloc((size_t)n, sizeof(double));
    double *cp = (double *)malloc(sizeof(double) * (size_t)n);
    double gamma = -22.0, alpha = 1.0, beta = 1.0; /* corners A[n-1][0], A[0][n-1] */
    for (int i = 0; i < n; ++i) b[i] = 22.0;
    b[0] -= gamma;
    b[n - 1] -= alpha * beta / gamma;
    u[0] = gamma;
    u[n - 1] = alpha;
    /* solve T y = 24 avg and T z = u (T tridiagonal with unit off-diagonals) */
    for (int pass = 0; pass < 2; ++pass) {
        double *out = pass == 0 ? y : z;
        for (int i = 0; i < n; ++i) out[i] = pass == 0 ? 24.0 * avg[i] : u[i];
        cp[0] = 1.0 / b[0];
        out[0] = out[0] / b[0];
        for (int i = 1; i < n; ++i) {
            double m = b[i] - cp[i - 1];
            cp[i] = 1.0 / m;
            out[i] = (out[i] - out[i - 1]) / m;
        }
        for (int i = n - 2; i >= 0; --i) out[i] -= cp[i] * out[i + 1];
    }
    double f = (y[0] + beta * y[n - 1] / gamma) / (1.0 + z[0] + beta * z[n - 1] / gamma);
    for (int i = 0; i < n; ++i) q[i] = y[i] - f * z[i];
    free(b);
    free(y);
    free(z);
    free(u);
    free(cp);
    return ORC_OK;
}

/* One RAM step with the A4 correction: PPM remap of the corrected averages, the
 * point values recovered from the remapped averages, then the residual step. */
int oracle_step_a4(int n, const double *x, const double *q_in, int limiter, double s,
                   const double *dv, double dt, int scheme, int nsub, double *q_out)
{
    double *avg = (double *)malloc(sizeof(double) * (size_t)n);
    double *sh = (double *)malloc(sizeof(double) * (size_t)n);
    double *pt = (double *)malloc(sizeof(double) * (size_t)n);
    int st = oracle_a4_average(n, q_in, avg);
    if (!st) st = oracle_shift(n, x, avg, 3, limiter, s, sh);
    if (!st) st = oracle_a4_point(n, sh, pt);
    if (!st) {
        if (dv)
            st = oracle_residual(n, x, pt, dv, dt, scheme, nsub, q_out);
        else
            memcpy(q_out, pt, sizeof(double) * (size_t)n);
    }
    free(avg);
    free(sh);
    free(pt);
    return st;
}

/* ------------------------------------------------------------------------- */
/* Transpose of the linear step (limiter off, donor residual)                  */
/* ------------------------------------------------------------------------- */

/* adjoint of G_i(d) scaled by w, accumulated into the coefficient adjoints
 * (l0, l1, l2) of cell i or, for order 4, directly into the mass adjoints gm */
static void cell_G_adjoint(const recon_t *r, int i, double d, double w, double *l0,
                           double *l1, double *l2, double *gm)
{
    int n = r->n;
    double h = r->dx[i];
    if (r->order == 2) {
        l0[i] += w * d;
        l1[i] += w * 0.5 * (d * d - d * h);
    } else if (r->order == 3) {
        double xi = d / h;
        l0[i] += w * h * (xi - 0.5 * xi * xi);
        l1[i] += w * h * 0.5 * xi * xi;
        l2[i] += w * h * (0.5 * xi * xi - xi * xi * xi / 3.0);
    } else {
        double z[6], b[6];
        quartic_nodes(r, i, z);
        quartic_pair_weights(z, d, b);
        /* node values in terms of masses: v0 = -(m_{i-2}+m_{i-1}), v1 = -m_{i-1},
         * v3 = m_i, v4 = m_i + m_{i+1}, v5 = m_i + m_{i+1} + m_{i+2} */
        gm[cyc(i - 2, n)] += w * (-b[0]);
        gm[cyc(i - 1, n)] += w * (-b[0] - b[1]);
        gm[i] += w * (b[3] + b[4] + b[5]);
        gm[cyc(i + 1, n)] += w * (b[4] + b[5]);
        gm[cyc(i + 2, n)] += w * b[5];
    }
}

/* g_in = A^T g_out for the limiter-off shift A. */
int oracle_shift_adjoint(int n, const double *x, int order, double s,
                         const double *g_out, double *g_in)
{
    if (n < 1 || !isfinite(s)) return ORC_ERR_ARG;
    double *zero = (double *)calloc((size_t)n, sizeof(double));
    recon_t r;
    int st = recon_build(&r, n, x, zero, order, 0); /* only the widths are used */
    if (st) {
        recon_free(&r);
        free(zero);
        return st;
    }
    double *gm = (double *)calloc((size_t)n, sizeof(double));
    double *l0 = (double *)calloc((size_t)n, sizeof(double));
    double *l1 = (double *)calloc((size_t)n, sizeof(double));
    double *l2 = (double *)calloc((size_t)n, sizeof(double));
    double L = x[n] - x[0];
    double sred = reduce_shift(s, L);
    edges_t e;
    edges_build(&e, n, x, sred);
    for (int i = 0; i < n; ++i) {
        cover_t c;
        cover_cell(n, r.dx, e.p, e.y, e.d, i, &c);
        double u = g_out[i] / r.dx[i]; /* adjoint of Eq. 26 */
        if (c.copy) {
            gm[c.pl] += g_out[i] / r.dx[c.pl];
            continue;
        }
        if (c.same) {
            cell_G_adjoint(&r, c.pl, c.dr, u, l0, l1, l2, gm);
            cell_G_adjoint(&r, c.pl, c.dl, -u, l0, l1, l2, gm);
        } else {
            gm[c.pl] += u;
            cell_G_adjoint(&r, c.pl, c.dl, -u, l0, l1, l2, gm);
            for (int k = 1; k <= c.nwhole; ++k) gm[cyc(c.pl + k, n)] += u;
            cell_G_adjoint(&r, c.pr, c.dr, u, l0, l1, l2, gm);
        }
    }
    edges_free(&e);
    /* masses M = Q dx */
    for (int i = 0; i < n; ++i) g_in[i] = gm[i] * r.dx[i];
    /* transpose of the limiter-off reconstruction */
    if (order == 2) {
        for (int i = 0; i < n; ++i) {
            int im = cyc(i - 1, n), ip = cyc(i + 1, n);
            double span = 0.5 * (r.dx[im] + r.dx[i]) + 0.5 * (r.dx[i] + r.dx[ip]);
            g_in[i] += l0[i];
            g_in[ip] += l1[i] / span;
            g_in[im] -= l1[i] / span;
        }
    } else if (order == 3) {
        double *lface = (double *)calloc((size_t)n, sizeof(double));
        double *ldq = (double *)calloc((size_t)n, sizeof(double));
        for (int i = 0; i < n; ++i) {
            /* Q6 = 6Q - 3(QL + QR); QL_i = face_{i-1}, QR_i = face_i */
            g_in[i] += 6.0 * l2[i];
            lface[cyc(i - 1, n)] += l0[i] - 3.0 * l2[i];
            lface[i] += l1[i] - 3.0 * l2[i];
        }
        for (int i = 0; i < n; ++i) {
            int im = cyc(i - 1, n), ip = cyc(i + 1, n), ip2 = cyc(i + 2, n);
            double hm = r.dx[im], h0 = r.dx[i], h1 = r.dx[ip], h2 = r.dx[ip2];
            double w1 = 2.0 * h1 * h0 / (h0 + h1) *
                        ((hm + h0) / (2.0 * h0 + h1) - (h2 + h1) / (2.0 * h1 + h0));
            double w2 = -h0 * (hm + h0) / (2.0 * h0 + h1);
            double w3 = h1 * (h1 + h2) / (h0 + 2.0 * h1);
            double sum4 = hm + h0 + h1 + h2;
            double a = h0 / (h0 + h1) + w1 / sum4; /* coefficient of (q[ip] - q[i]) */
            double lf = lface[i];
            g_in[i] += lf * (1.0 - a);
            g_in[ip] += lf * a;
            ldq[ip] += lf * w2 / sum4;
            ldq[i] += lf * w3 / sum4;
        }
        for (int i = 0; i < n; ++i) {
            int im = cyc(i - 1, n), ip = cyc(i + 1, n);
            double a = r.dx[im], b = r.dx[i], c = r.dx[ip];
            double alpha = b / (a + b + c) * (2.0 * a + b) / (b + c);
            double beta = b / (a + b + c) * (b + 2.0 * c) / (a + b);
            /* dq_i = alpha (q_{i+1} - q_i) + beta (q_i - q_{i-1}) */
            g_in[ip] += ldq[i] * alpha;
            g_in[i] += ldq[i] * (beta - alpha);
            g_in[im] -= ldq[i] * beta;
        }
        free(lface);
        free(ldq);
    }
    recon_free(&r);
    free(zero);
    free(gm);
    free(l0);
    free(l1);
    free(l2);
    return ORC_OK;
}

/* Transpose of the donor-cell residual step (nsub sub-steps).  q_in is the input
 * of the residual step (the shifted field); g_dv (may be NULL) receives
 * d loss / d dv added to its current contents.  At dv_j == 0 the upwind side
 * is taken as the left cell (the derivative of the flux from dv > 0). */
int oracle_residual_adjoint_donor(int n, const double *x, const double *q_in,
                                  const double *dv, double dt, int nsub,
                                  const double *g_out, double *g_in, double *g_dv)
{
    if (n < 1 || nsub < 1) return ORC_ERR_ARG;
    double *dx = (double *)malloc(sizeof(double) * (size_t)n);
    int st = widths(n, x, dx);
    if (st) {
        free(dx);
        return st;
    }
    double h = dt / nsub;
    /* forward states of every sub-step */
    double *states = (double *)malloc(sizeof(double) * (size_t)n * (size_t)(nsub + 1));
    memcpy(states, q_in, sizeof(double) * (size_t)n);
    for (int k = 0; k < nsub; ++k)
        residual_substep(n, dx, states + (size_t)k * n, dv, h, SCHEME_DONOR,
                         states + (size_t)(k + 1) * n);
    double *g = (double *)malloc(sizeof(double) * (size_t)n);
    double *gn = (double *)malloc(sizeof(double) * (size_t)n);
    double *lf = (double *)malloc(sizeof(double) * (size_t)n);
    memcpy(g, g_out, sizeof(double) * (size_t)n);
    for (int k = nsub - 1; k >= 0; --k) {
        const double *qk = states + (size_t)k * n;
        /* q_next_i = q_i - (F_{i+1} - F_i) / dx_i  ->  dL/dF_j */
        for (int j = 0; j < n; ++j) lf[j] = g[j] / dx[j] - g[cyc(j - 1, n)] / dx[cyc(j - 1, n)];
        for (int i = 0; i < n; ++i) gn[i] = g[i];
        for (int j = 0; j < n; ++j) {
            double c = dv[j] * h;
            int up = (c >= 0.0) ? cyc(j - 1, n) : j;
            /* F_j = c q_up */
            gn[up] += lf[j] * c;
            if (g_dv) g_dv[j] += lf[j] * h * qk[up];
        }
        double *t = g;
        g = gn;
        gn = t;
    }
    memcpy(g_in, g, sizeof(double) * (size_t)n);
    free(dx);
    free(states);
    free(g);
    free(gn);
    free(lf);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Linearisation of the limited step at a forward state                         */
/* ------------------------------------------------------------------------- */

/* The tangent (directional derivative) of the shift at q0 along v, for PLM and PPM
 * with or without the limiter: every quantity of the reconstruction is carried as
 * a value and its derivative, and every branch of the limiters (App. A.2, the van
 * Leer slope) is taken as the value decides it -- the linearisation at the
 * forward state.  The remap (Eq. 18) is linear in the reconstruction for fixed
 * edges, so its tangent is the same formula on the derivatives. */
typedef struct {
    double v, d;
} dual_t;

static dual_t dmk(double v, double d)
{
    dual_t r = {v, d};
    return r;
}
static dual_t dadd(dual_t a, dual_t b) { return dmk(a.v + b.v, a.d + b.d); }
static dual_t dsub(dual_t a, dual_t b) { return dmk(a.v - b.v, a.d - b.d); }
static dual_t dmul(dual_t a, dual_t b) { return dmk(a.v * b.v, a.d * b.v + a.v * b.d); }
static dual_t dscale(dual_t a, double s) { return dmk(a.v * s, a.d * s); }
static dual_t ddiv(dual_t a, dual_t b)
{
    return dmk(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}

int oracle_shift_jvp(int n, const double *x, const double *q0, int order, int limiter,
                     double s, const double *vdir, double *out)
{
    if (n < 1 || (order != 2 && order != 3)) return ORC_ERR_ARG;
    recon_t r;
    int st = recon_build(&r, n, x, q0, order, limiter); /* widths and the edge geometry */
    if (st) {
        recon_free(&r);
        return st;
    }
    const double *dx = r.dx;
    dual_t *q = (dual_t *)malloc(sizeof(dual_t) * (size_t)n);
    dual_t *c0 = (dual_t *)malloc(sizeof(dual_t) * (size_t)n);
    dual_t *c1 = (dual_t *)malloc(sizeof(dual_t) * (size_t)n);
    dual_t *c2 = (dual_t *)malloc(sizeof(dual_t) * (size_t)n);
    for (int i = 0; i < n; ++i) q[i] = dmk(q0[i], vdir[i]);
    if (order == 2) {
        for (int i = 0; i < n; ++i) {
            int im = cyc(i - 1, n), ip = cyc(i + 1, n);
            double hl = 0.5 * (dx[im] + dx[i]), hr = 0.5 * (dx[i] + dx[ip]);
            dual_t sig;
            if (limiter) {
                dual_t dl = dscale(dsub(q[i], q[im]), 1.0 / hl);
                dual_t dr = dscale(dsub(q[ip], q[i]), 1.0 / hr);
                if (dl.v * dr.v <= 0.0)
                    sig = dmk(0.0, 0.0);
                else
                    sig = ddiv(dscale(dmul(dl, dr), 2.0), dadd(dl, dr));
            } else {
                sig = dscale(dsub(q[ip], q[im]), 1.0 / (hl + hr));
            }
            c0[i] = q[i];
            c1[i] = sig;
        }
    } else {
        dual_t *dq = (dual_t *)malloc(sizeof(dual_t) * (size_t)n);
        dual_t *face = (dual_t *)malloc(sizeof(dual_t) * (size_t)n);
        for (int i = 0; i < n; ++i) {
            int im = cyc(i - 1, n), ip = cyc(i + 1, n);
            double a = dx[im], b = dx[i], c = dx[ip];
            dual_t up = dsub(q[ip], q[i]), dn = dsub(q[i], q[im]);
            dual_t d = dadd(dscale(up, b / (a + b + c) * (2.0 * a + b) / (b + c)),
                            dscale(dn, b / (a + b + c) * (b + 2.0 * c) / (a + b)));
            if (limiter) {
                if (up.v * dn.v > 0.0) {
                    /* sign(d) min(|d|, 2|dn|, 2|up|), the smallest taken by value */
                    dual_t m = d.v >= 0.0 ? d : dscale(d, -1.0);
                    dual_t an = dscale(dn.v >= 0.0 ? dn : dscale(dn, -1.0), 2.0);
                    dual_t au = dscale(up.v >= 0.0 ? up : dscale(up, -1.0), 2.0);
                    if (an.v < m.v) m = an;
                    if (au.v < m.v) m = au;
                    d = d.v >= 0.0 ? m : dscale(m, -1.0);
                } else {
                    d = dmk(0.0, 0.0);
                }
            }
            dq[i] = d;
        }
        for (int i = 0; i < n; ++i) {
            int im = cyc(i - 1, n), ip = cyc(i + 1, n), ip2 = cyc(i + 2, n);
            double hm = dx[im], h0 = dx[i], h1 = dx[ip], h2 = dx[ip2];
            double w1 = 2.0 * h1 * h0 / (h0 + h1) *
                        ((hm + h0) / (2.0 * h0 + h1) - (h2 + h1) / (2.0 * h1 + h0));
            double w2 = -h0 * (hm + h0) / (2.0 * h0 + h1);
            double w3 = h1 * (h1 + h2) / (h0 + 2.0 * h1);
            double sum4 = hm + h0 + h1 + h2;
            dual_t del = dsub(q[ip], q[i]);
            face[i] = dadd(dadd(q[i], dscale(del, h0 / (h0 + h1))),
                           dscale(dadd(dadd(dscale(del, w1), dscale(dq[ip], w2)), dscale(dq[i], w3)),
                                  1.0 / sum4));
        }
        for (int i = 0; i < n; ++i) {
            dual_t L = face[cyc(i - 1, n)], R = face[i], Q = q[i];
            if (limiter) {
                if ((R.v - Q.v) * (Q.v - L.v) <= 0.0) {
                    L = Q;
                    R = Q;
                } else {
                    double dd = R.v - L.v, qa = Q.v - 0.5 * (L.v + R.v);
                    if (dd * qa > dd * dd / 6.0)
                        L = dsub(dscale(Q, 3.0), dscale(R, 2.0));
                    else if (-dd * dd / 6.0 > dd * qa)
                        R = dsub(dscale(Q, 3.0), dscale(L, 2.0));
                }
            }
            c0[i] = L;
            c1[i] = R;
            c2[i] = dsub(dscale(Q, 6.0), dscale(dadd(L, R), 3.0));
        }
        free(dq);
        free(face);
    }
    /* the remap of the derivatives: the forward formulas with d in place of v */
    recon_t t = r;
    double *d0 = (double *)malloc(sizeof(double) * (size_t)n);
    double *d1 = (double *)malloc(sizeof(double) * (size_t)n);
    double *d2 = (double *)calloc((size_t)n, sizeof(double));
    double *dm = (double *)malloc(sizeof(double) * (size_t)n);
    double *dqv = (double *)malloc(sizeof(double) * (size_t)n);
    for (int i = 0; i < n; ++i) {
        d0[i] = c0[i].d;
        d1[i] = c1[i].d;
        if (order == 3) d2[i] = c2[i].d;
        dqv[i] = vdir[i];
        dm[i] = vdir[i] * dx[i];
    }
    t.c0 = d0;
    t.c1 = d1;
    t.c2 = d2;
    t.m = dm;
    t.q = dqv;
    t.limited = 0;
    double L = x[n] - x[0];
    edges_t e;
    edges_build(&e, n, x, reduce_shift(s, L));
    for (int i = 0; i < n; ++i) {
        cover_t c;
        cover_cell(n, dx, e.p, e.y, e.d, i, &c);
        if (c.copy) {
            out[i] = vdir[c.pl];
            continue;
        }
        double mass;
        if (c.same) {
            mass = cell_G(&t, c.pl, c.dr) - cell_G(&t, c.pl, c.dl);
        } else {
            mass = t.m[c.pl] - cell_G(&t, c.pl, c.dl);
            for (int k = 1; k <= c.nwhole; ++k) mass += t.m[cyc(c.pl + k, n)];
            mass += cell_G(&t, c.pr, c.dr);
        }
        out[i] = mass / dx[i];
    }
    edges_free(&e);
    free(d0);
    free(d1);
    free(d2);
    free(dm);
    free(dqv);
    free(q);
    free(c0);
    free(c1);
    free(c2);
    recon_free(&r);
    return ORC_OK;
}

/* The transpose of that tangent, by its definition: (J^T g)_k = <J e_k, g>, one
 * tangent per cell (small rows only: quadratic cost). */
int oracle_shift_vjp(int n, const double *x, const double *q0, int order, int limiter,
                     double s, const double *g, double *out)
{
    double *e = (double *)calloc((size_t)n, sizeof(double));
    double *col = (double *)malloc(sizeof(double) * (size_t)n);
    int st = ORC_OK;
    for (int k = 0; k < n && !st; ++k) {
        e[k] = 1.0;
        st = oracle_shift_jvp(n, x, q0, order, limiter, s, e, col);
        e[k] = 0.0;
        double acc = 0.0;
        for (int i = 0; i < n; ++i) acc += col[i] * g[i];
        out[k] = acc;
    }
    free(e);
    free(col);
    return st;
}

/* Transpose of the step linearised at q_in: the shift (PLM / PPM, the limiter as
 * the plan has it) linearised at q_in, then the donor residual (linear).  g_dv as
 * in oracle_step_adjoint. */
int oracle_step_adjoint_limited(int n, const double *x, const double *q_in, int order,
                                int limiter, double s, const double *dv, double dt, int nsub,
                                const double *g_out, double *g_in, double *g_dv)
{
    double *qs = (double *)malloc(sizeof(double) * (size_t)n);
    double *gs = (double *)malloc(sizeof(double) * (size_t)n);
    int st = oracle_shift(n, x, q_in, order, limiter, s, qs);
    if (!st) {
        if (dv)
            st = oracle_residual_adjoint_donor(n, x, qs, dv, dt, nsub, g_out, gs, g_dv);
        else
            memcpy(gs, g_out, sizeof(double) * (size_t)n);
    }
    if (!st) st = oracle_shift_vjp(n, x, q_in, order, limiter, s, gs, g_in);
    free(qs);
    free(gs);
    return st;
}

/* Transpose of one linear RAM step (limiter-off shift, donor residual): given
 * the step input q_in and the cotangent of the output, produce the cotangent of
 * the input and add d loss / d dv into g_dv (may be NULL). dv may be NULL. */
int oracle_step_adjoint(int n, const double *x, const double *q_in, int order, double s,
                        const double *dv, double dt, int nsub, const double *g_out,
                        double *g_in, double *g_dv)
{
    double *qs = (double *)malloc(sizeof(double) * (size_t)n);
    double *gs = (double *)malloc(sizeof(double) * (size_t)n);
    int st = oracle_shift(n, x, q_in, order, 0, s, qs);
    if (!st) {
        if (dv)
            st = oracle_residual_adjoint_donor(n, x, qs, dv, dt, nsub, g_out, gs, g_dv);
        else
            memcpy(gs, g_out, sizeof(double) * (size_t)n);
    }
    if (!st) st = oracle_shift_adjoint(n, x, order, s, gs, g_in);
    free(qs);
    free(gs);
    return st;
}
