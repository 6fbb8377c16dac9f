/*
 * cnsf_oracle.c -- plain, slow, FP64 CPU oracle of the convolutional
 * non-separable footprint (CNSF) fan-beam projector.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the bench's CPU
 * baseline leg load this file.  It shares no code, header, table or constant
 * with the CUDA library: it has its own geometry struct, its own ray set-up,
 * its own box-spline evaluation and its own support enumeration.
 *
 * What it computes (Zhang & Entezari, "A Convolutional Forward and
 * Back-Projection Model for Fan-Beam Geometry"):
 *
 *   geometry  Sec. II.A: source p = D_po u, detector line perpendicular to u at
 *             distance D_ps from the source, detector coordinate s along w.
 *   entry     Eq. (18): a(view, cell, pixel) = h^2 M_[zeta1, zeta2, tau'](s'),
 *             zeta_i = R_{v(s)perp} (h e_i) (Eq. 16), s' the coordinate of the
 *             pixel centre on v(s)perp, tau' the effective blur of Eq. (17),
 *             all taken on the ray through the centre of the detector cell.
 *   box spline Sec. III.A: M_Xi = M_xi1 * ... * M_xiN, each M_xi a centred box
 *             of width |xi| and unit integral.  The three-direction spline is
 *             evaluated as the window average (width tau') of the trapezoid
 *             box_zeta1 * box_zeta2, integrated piece by piece (every piece is
 *             non-negative, so there is no cancellation).
 *   forward   Eq. (6): y = A c, one ray-driven loop per (view, cell).
 *   back      A^T y, one pixel-driven loop per pixel.
 *   Ref       Eq. (1)-(2): the bin average (1/tau) int chord(s) ds of the exact
 *             line integral of the pixel indicator, by Gauss-Legendre on the
 *             smooth pieces between pixel-corner rays (the paper's "reference
 *             projector", Sec. IV).
 *
 * Readings of the paper taken here (it is silent on them): the ray for cell j is
 * the line from p through the cell centre q_j = d + s_j w with d = -D_so u; a
 * bin value is the mean (not the integral) of line integrals over the cell; the
 * effective blur is measured on v(s)perp at the depth of the pixel centre along
 * the central ray; the blur window is centred on the central ray.
 *
 * Parallel-beam mode (geometry flag `parallel`): every ray of a view runs along
 * -u, the detector coordinate is s = x . w and tau' = tau (Theorem 1, exact).
 *
 * Arc-detector mode (geometry flag `arc`, the equiangular fan of Sec. I): the
 * cells lie on the circle of radius D_ps about the source; the detector
 * coordinate s is the arc length from the point p - D_ps u, so the ray of
 * coordinate s leaves the source at the angle s/D_ps from -u (towards w).  The
 * entry follows the same steps as the flat case: the central ray through the
 * cell centre, the two cell edges perspective-divided in its frame (Eq. 17),
 * and Ref is the bin average over s of the exact chords.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int nx, ny;          /* image columns, rows; image stored [ny][nx]          */
    double h;            /* pixel side (mm)                                      */
    double cx, cy;       /* image centre (mm)                                    */
    int nviews;
    const double *angles;/* view angles theta_k (rad), length nviews             */
    int ndet;
    double ds;           /* detector pitch (mm)                                  */
    double tau;          /* detector cell width (mm)                             */
    double det_off;      /* detector centre offset along s (mm)                  */
    double dpo;          /* source to rotation centre (mm)                       */
    double dps;          /* source to detector line (mm)                         */
    int parallel;        /* 1: parallel-beam rays (Theorem 1)                    */
    int arc;             /* 1: cells on the arc of radius D_ps about the source  */
} og_geom;

/* ------------------------------------------------------------------ frames */
typedef struct {
    double ux, uy;   /* viewing direction u = (cos t, sin t)       */
    double wx, wy;   /* detector axis, perpendicular to u          */
    double px, py;   /* source p = D_po u                          */
    double dx, dy;   /* detector centre d = -(D_ps - D_po) u       */
} og_view;

static og_view og_make_view(const og_geom *g, int k)
{
    og_view v;
    double th = g->angles[k];
    v.ux = cos(th);
    v.uy = sin(th);
    v.wx = -v.uy;
    v.wy = v.ux;
    v.px = g->dpo * v.ux;
    v.py = g->dpo * v.uy;
    v.dx = -(g->dps - g->dpo) * v.ux;
    v.dy = -(g->dps - g->dpo) * v.uy;
    return v;
}

static double og_cell_centre(const og_geom *g, int j)
{
    return (j - 0.5 * (g->ndet - 1)) * g->ds + g->det_off;
}

static void og_pixel_centre(const og_geom *g, int i, int r, double *kx, double *ky)
{
    *kx = g->cx + (i - 0.5 * (g->nx - 1)) * g->h;
    *ky = g->cy + (r - 0.5 * (g->ny - 1)) * g->h;
}

/* The point of the detector at coordinate s (fan beam): on the flat line d + s w,
 * or on the arc p + D_ps (-cos(s/D_ps) u + sin(s/D_ps) w). */
static void og_detector_point(const og_geom *g, const og_view *w, double s, double *qx, double *qy)
{
    if (g->arc) {
        double gam = s / g->dps, cg = cos(gam), sg = sin(gam);
        *qx = w->px + g->dps * (-cg * w->ux + sg * w->wx);
        *qy = w->py + g->dps * (-cg * w->uy + sg * w->wy);
    } else {
        *qx = w->dx + s * w->wx;
        *qy = w->dy + s * w->wy;
    }
}

/* A ray of the view for detector coordinate s: a point o on it, unit direction
 * v, unit normal n (the basis of v(s)perp), and whether it is a half-line from
 * the source (fan) or a full line (parallel). */
typedef struct {
    double ox, oy, vx, vy, nx, ny;
    int halfline;
} og_ray;

static og_ray og_make_ray(const og_geom *g, const og_view *w, double s)
{
    og_ray r;
    if (g->parallel) {
        r.ox = s * w->wx;
        r.oy = s * w->wy;
        r.vx = -w->ux;
        r.vy = -w->uy;
        r.halfline = 0;
    } else {
        double qx, qy;                                          /* point on detector */
        og_detector_point(g, w, s, &qx, &qy);
        double ex = qx - w->px, ey = qy - w->py;
        double len = sqrt(ex * ex + ey * ey);
        r.ox = w->px;
        r.oy = w->py;
        r.vx = ex / len;
        r.vy = ey / len;
        r.halfline = 1;
    }
    r.nx = -r.vy;
    r.ny = r.vx;
    return r;
}

/* ------------------------------------------------------------ box splines */
/* Trapezoid g = box_a * box_b (a >= b >= 0, a > 0): centred, unit integral. */
static double og_trap(double a, double b, double x)
{
    double ax = fabs(x);
    double plateau = 0.5 * (a - b), outer = 0.5 * (a + b);
    if (ax >= outer) return 0.0;
    if (ax <= plateau) return 1.0 / a;
    return (outer - ax) / (a * b);
}

/* Exact integral of the trapezoid box_a * box_b over [lo, hi], summed over its
 * three linear pieces (rising ramp, plateau, falling ramp).  Each piece
 * contributes (length) x (mean of the two end values) >= 0. */
static double og_trap_integral(double a, double b, double lo, double hi)
{
    double k0 = -0.5 * (a + b), k1 = -0.5 * (a - b), k2 = 0.5 * (a - b), k3 = 0.5 * (a + b);
    double sum = 0.0, l, r;
    l = fmax(lo, k0); r = fmin(hi, k1);            /* rising ramp, width b   */
    if (r > l) sum += (r - l) * 0.5 * ((l - k0) + (r - k0)) / (a * b);
    l = fmax(lo, k1); r = fmin(hi, k2);            /* plateau 1/a            */
    if (r > l) sum += (r - l) / a;
    l = fmax(lo, k2); r = fmin(hi, k3);            /* falling ramp, width b  */
    if (r > l) sum += (r - l) * 0.5 * ((k3 - l) + (k3 - r)) / (a * b);
    return sum;
}

/* M_[z1, z2, z3](x): centred three-direction univariate box spline, i.e. the
 * convolution of three centred unit-integral boxes of widths |z1|, |z2|, |z3|
 * (Sec. III.A).  z3 is the window; z3 = 0 gives the two-direction spline of
 * Eq. (16).  A zero zeta drops out (M_0 = delta). */
double og_box3(double z1, double z2, double z3, double x)
{
    double a = fmax(fabs(z1), fabs(z2)), b = fmin(fabs(z1), fabs(z2)), c = fabs(z3);
    if (a == 0.0) {               /* both footprint directions vanish: box_c alone */
        if (c == 0.0) return 0.0;
        return fabs(x) < 0.5 * c ? 1.0 / c : 0.0;
    }
    if (c == 0.0) return og_trap(a, b, x);
    return og_trap_integral(a, b, x - 0.5 * c, x + 0.5 * c) / c;
}

/* The literal closed form of Eq. (18): Delta_z1 Delta_z2 Delta_z3 (y)_+^2 / 2!,
 * divided by z1 z2 z3 (the divided differences of the unit-integral
 * elementary boxes), shifted by (|z1|+|z2|+|z3|)/2 to centre it.  Long double;
 * it cancels badly when a z is small, so it serves only as a cross-check. */
double og_box3_divdiff(double z1, double z2, double z3, double x)
{
    long double a = fabsl((long double)z1), b = fabsl((long double)z2), c = fabsl((long double)z3);
    long double y = (long double)x + 0.5L * (a + b + c);
    long double sum = 0.0L;
    for (int m = 0; m < 8; ++m) {
        long double t = y;
        int sign = 1;
        if (m & 1) { t -= a; sign = -sign; }
        if (m & 2) { t -= b; sign = -sign; }
        if (m & 4) { t -= c; sign = -sign; }
        if (t > 0.0L) sum += sign * 0.5L * t * t;
    }
    return (double)(sum / (a * b * c));
}

/* ------------------------------------------------------------ CNSF entry */
/* Effective blur of Eq. (17): the two edges of cell j are written in the frame
 * [v(s)perp, v(s)] of the central ray (origin at the source), perspective
 * divided, and the difference is scaled to the depth t of the pixel centre. */
static double og_tau_prime_at(const og_geom *g, const og_view *w, const og_ray *ray, double sj,
                              double t)
{
    if (g->parallel) return g->tau;
    double ratio[2];
    for (int e = 0; e < 2; ++e) {
        double se = sj + (e ? 0.5 : -0.5) * g->tau, qx, qy;
        og_detector_point(g, w, se, &qx, &qy);
        qx -= w->px;
        qy -= w->py;
        double x1 = ray->nx * qx + ray->ny * qy;   /* coordinate on v(s)perp */
        double x2 = ray->vx * qx + ray->vy * qy;   /* coordinate along v(s)  */
        ratio[e] = x1 / x2;                        /* perspective division   */
    }
    return fabs(t * (ratio[1] - ratio[0]));
}

typedef struct { double zeta1, zeta2, sprime, tprime, depth; } og_parts;

static og_parts og_entry_parts(const og_geom *g, int k, int j, int i, int r)
{
    og_view w = og_make_view(g, k);
    double sj = og_cell_centre(g, j);
    og_ray ray = og_make_ray(g, &w, sj);
    double kx, ky;
    og_pixel_centre(g, i, r, &kx, &ky);
    og_parts P;
    P.zeta1 = g->h * ray.nx;                                    /* R_{v perp} h e1 */
    P.zeta2 = g->h * ray.ny;                                    /* R_{v perp} h e2 */
    P.sprime = ray.nx * (kx - ray.ox) + ray.ny * (ky - ray.oy); /* R_{v perp}(k - p) */
    P.depth = ray.vx * (kx - ray.ox) + ray.vy * (ky - ray.oy);
    P.tprime = og_tau_prime_at(g, &w, &ray, sj, P.depth);
    return P;
}

double og_entry(const og_geom *g, int k, int j, int i, int r)
{
    og_parts P = og_entry_parts(g, k, j, i, r);
    return g->h * g->h * og_box3(P.zeta1, P.zeta2, P.tprime, P.sprime);
}

void og_entry_parts_out(const og_geom *g, int k, int j, int i, int r, double *out5)
{
    og_parts P = og_entry_parts(g, k, j, i, r);
    out5[0] = P.zeta1; out5[1] = P.zeta2; out5[2] = P.sprime; out5[3] = P.tprime; out5[4] = P.depth;
}

/* ------------------------------------------------------- exact line integral */
/* Chord length of a ray with the axis-aligned square of side h centred at
 * (kx, ky): slab clipping (Liang-Barsky).  This is Eq. (1) for the pixel
 * indicator. */
static double og_chord_ray(const og_ray *ray, double kx, double ky, double h)
{
    double t0 = ray->halfline ? 0.0 : -INFINITY, t1 = INFINITY;
    double lo[2] = {kx - 0.5 * h, ky - 0.5 * h}, hi[2] = {kx + 0.5 * h, ky + 0.5 * h};
    double o[2] = {ray->ox, ray->oy}, v[2] = {ray->vx, ray->vy};
    for (int a = 0; a < 2; ++a) {
        if (v[a] == 0.0) {
            if (o[a] < lo[a] || o[a] > hi[a]) return 0.0;
        } else {
            double ta = (lo[a] - o[a]) / v[a], tb = (hi[a] - o[a]) / v[a];
            if (ta > tb) { double tmp = ta; ta = tb; tb = tmp; }
            if (ta > t0) t0 = ta;
            if (tb < t1) t1 = tb;
        }
    }
    return t1 > t0 ? t1 - t0 : 0.0;
}

double og_chord(const og_geom *g, int k, double s, int i, int r)
{
    og_view w = og_make_view(g, k);
    og_ray ray = og_make_ray(g, &w, s);
    double kx, ky;
    og_pixel_centre(g, i, r, &kx, &ky);
    return og_chord_ray(&ray, kx, ky, g->h);
}

/* Detector coordinate of the ray through an image point (perspective
 * projection, the operator P of Eq. (4)). */
static double og_project_point(const og_geom *g, const og_view *w, double x, double y)
{
    double xw = x * w->wx + y * w->wy;
    if (g->parallel) return xw;
    double xu = x * w->ux + y * w->uy;
    if (g->arc) return g->dps * atan2(xw, g->dpo - xu);
    return g->dps * xw / (g->dpo - xu);
}

/* Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on P_n. */
static void og_gauss_legendre(int n, double *x, double *wt)
{
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5)), pp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p1 = 1.0, p2 = 0.0;
            for (int k = 1; k <= n; ++k) {
                double p3 = p2;
                p2 = p1;
                p1 = ((2.0 * k - 1.0) * z * p2 - (k - 1.0) * p3) / k;
            }
            pp = n * (z * p1 - p2) / (z * z - 1.0);
            double z1 = z;
            z = z1 - p1 / pp;
            if (fabs(z - z1) < 1e-16) break;
        }
        x[i] = -z;
        x[n - 1 - i] = z;
        wt[i] = wt[n - 1 - i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
}

/* Ref entry: (1/tau) int_{s_j - tau/2}^{s_j + tau/2} chord(s) ds, split at the
 * detector positions of the four pixel corners (where chord(s) has kinks) and
 * integrated by ng-point Gauss-Legendre on each smooth piece. */
double og_ref_entry(const og_geom *g, int k, int j, int i, int r, int ng)
{
    og_view w = og_make_view(g, k);
    double sj = og_cell_centre(g, j);
    double kx, ky;
    og_pixel_centre(g, i, r, &kx, &ky);
    double lo = sj - 0.5 * g->tau, hi = sj + 0.5 * g->tau;
    if (g->tau == 0.0) {
        og_ray ray = og_make_ray(g, &w, sj);
        return og_chord_ray(&ray, kx, ky, g->h);
    }
    double cuts[6];
    int nc = 0;
    cuts[nc++] = lo;
    for (int c = 0; c < 4; ++c) {
        double x = kx + ((c & 1) ? 0.5 : -0.5) * g->h, y = ky + ((c & 2) ? 0.5 : -0.5) * g->h;
        double sc = og_project_point(g, &w, x, y);
        if (sc > lo && sc < hi) cuts[nc++] = sc;
    }
    cuts[nc++] = hi;
    for (int a = 1; a < nc; ++a)          /* insertion sort */
        for (int b = a; b > 0 && cuts[b] < cuts[b - 1]; --b) {
            double t = cuts[b]; cuts[b] = cuts[b - 1]; cuts[b - 1] = t;
        }
    double xg[64], wg[64];
    if (ng > 64) ng = 64;
    og_gauss_legendre(ng, xg, wg);
    double sum = 0.0;
    for (int p = 0; p + 1 < nc; ++p) {
        double a = cuts[p], b = cuts[p + 1];
        if (b <= a) continue;
        double mid = 0.5 * (a + b), half = 0.5 * (b - a), part = 0.0;
        for (int q = 0; q < ng; ++q) {
            og_ray ray = og_make_ray(g, &w, mid + half * xg[q]);
            part += wg[q] * og_chord_ray(&ray, kx, ky, g->h);
        }
        sum += part * half;
    }
    return sum / g->tau;
}

/* Ref entry by the midpoint rule with m rays across the cell (supersampled ray
 * integration). */
double og_ref_entry_midpoint(const og_geom *g, int k, int j, int i, int r, long m)
{
    og_view w = og_make_view(g, k);
    double sj = og_cell_centre(g, j);
    double kx, ky;
    og_pixel_centre(g, i, r, &kx, &ky);
    double sum = 0.0;
    for (long q = 0; q < m; ++q) {
        double s = sj - 0.5 * g->tau + (q + 0.5) * g->tau / (double)m;
        og_ray ray = og_make_ray(g, &w, s);
        sum += og_chord_ray(&ray, kx, ky, g->h);
    }
    return sum / (double)m;
}

/* --------------------------------------------------- support enumerations */
/* Upper bound of tau' over the image (depth <= D_po + image radius). */
static double og_tau_prime_bound(const og_geom *g)
{
    if (g->parallel) return g->tau;
    double rx = fabs(g->cx) + 0.5 * g->nx * g->h, ry = fabs(g->cy) + 0.5 * g->ny * g->h;
    double tmax = g->dpo + sqrt(rx * rx + ry * ry);
    if (g->arc) return tmax * 2.0 * tan(0.5 * g->tau / g->dps);   /* edges at +-tau/(2 D_ps) rad */
    double smax = fabs(g->det_off) + 0.5 * g->ndet * g->ds + g->tau;
    /* the bin subtends at most tau*D_ps/(D_ps^2 + s^2 - s*tau) per unit depth */
    double denom = g->dps * g->dps - smax * g->tau;
    if (denom < 0.5 * g->dps * g->dps) denom = 0.5 * g->dps * g->dps;
    return tmax * g->tau * g->dps / denom;
}

/* Half-width (in s') outside which every entry is zero, plus one pixel of
 * margin: the support of M_[z1,z2,tau'] is (|z1|+|z2|+tau')/2. */
static double og_reach(const og_geom *g)
{
    return 0.5 * (sqrt(2.0) * g->h + og_tau_prime_bound(g)) + g->h;
}

typedef double (*og_entry_fn)(const og_geom *, int, int, int, int, int);

static double og_entry_cnsf_cb(const og_geom *g, int k, int j, int i, int r, int ng)
{
    (void)ng;
    return og_entry(g, k, j, i, r);
}

static double og_entry_ref_cb(const og_geom *g, int k, int j, int i, int r, int ng)
{
    return og_ref_entry(g, k, j, i, r, ng);
}

/* y_j = sum_n c_n a_jn for one (view, cell): walk the dominant axis of the ray
 * and take, on each row (or column), the pixels within `reach` of the ray. */
static double og_ray_sum(const og_geom *g, const double *c, int k, int j, og_entry_fn fn, int ng,
                         double extra, long *nnz)
{
    og_view w = og_make_view(g, k);
    og_ray ray = og_make_ray(g, &w, og_cell_centre(g, j));
    double reach = og_reach(g) + extra;
    double acc = 0.0;
    if (fabs(ray.vy) >= fabs(ray.vx)) {
        for (int r = 0; r < g->ny; ++r) {
            double kx, ky;
            og_pixel_centre(g, 0, r, &kx, &ky);
            double xc = ray.ox + (ky - ray.oy) / ray.vy * ray.vx;   /* crossing of row r */
            double half = reach / fabs(ray.nx);
            int ilo = (int)ceil((xc - half - g->cx) / g->h + 0.5 * (g->nx - 1));
            int ihi = (int)floor((xc + half - g->cx) / g->h + 0.5 * (g->nx - 1));
            if (ilo < 0) ilo = 0;
            if (ihi > g->nx - 1) ihi = g->nx - 1;
            for (int i = ilo; i <= ihi; ++i) {
                double a = fn(g, k, j, i, r, ng);
                if (nnz && a > 0.0) ++*nnz;
                if (c) acc += c[(long)r * g->nx + i] * a;
            }
        }
    } else {
        for (int i = 0; i < g->nx; ++i) {
            double kx, ky;
            og_pixel_centre(g, i, 0, &kx, &ky);
            double yc = ray.oy + (kx - ray.ox) / ray.vx * ray.vy;   /* crossing of column i */
            double half = reach / fabs(ray.ny);
            int rlo = (int)ceil((yc - half - g->cy) / g->h + 0.5 * (g->ny - 1));
            int rhi = (int)floor((yc + half - g->cy) / g->h + 0.5 * (g->ny - 1));
            if (rlo < 0) rlo = 0;
            if (rhi > g->ny - 1) rhi = g->ny - 1;
            for (int r = rlo; r <= rhi; ++r) {
                double a = fn(g, k, j, i, r, ng);
                if (nnz && a > 0.0) ++*nnz;
                if (c) acc += c[(long)r * g->nx + i] * a;
            }
        }
    }
    return acc;
}

/* Forward projection y = A c (Eq. 6); y is [nviews][ndet]. */
void og_forward(const og_geom *g, const double *c, double *y)
{
    long nr = (long)g->nviews * g->ndet;
#pragma omp parallel for schedule(dynamic, 8)
    for (long kj = 0; kj < nr; ++kj)
        y[kj] = og_ray_sum(g, c, (int)(kj / g->ndet), (int)(kj % g->ndet), og_entry_cnsf_cb, 0, 0.0,
                           NULL);
}

/* Forward projection with the Ref entries (bin-integrated exact chords). */
void og_forward_ref(const og_geom *g, const double *c, double *y, int ng)
{
    long nr = (long)g->nviews * g->ndet;
#pragma omp parallel for schedule(dynamic, 8)
    for (long kj = 0; kj < nr; ++kj)
        y[kj] = og_ray_sum(g, c, (int)(kj / g->ndet), (int)(kj % g->ndet), og_entry_ref_cb, ng,
                           g->h, NULL);
}

/* y for a list of (view, cell) pairs only. */
void og_forward_rays(const og_geom *g, const double *c, long nsamp, const int *views,
                     const int *cells, double *out)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (long q = 0; q < nsamp; ++q)
        out[q] = og_ray_sum(g, c, views[q], cells[q], og_entry_cnsf_cb, 0, 0.0, NULL);
}

/* Number of non-zero entries of A (found by the ray-driven enumeration). */
long og_count_nnz(const og_geom *g)
{
    long total = 0, nr = (long)g->nviews * g->ndet;
#pragma omp parallel for schedule(dynamic, 8) reduction(+ : total)
    for (long kj = 0; kj < nr; ++kj) {
        long cnt = 0;
        og_ray_sum(g, NULL, (int)(kj / g->ndet), (int)(kj % g->ndet), og_entry_cnsf_cb, 0, 0.0, &cnt);
        total += cnt;
    }
    return total;
}

/* (A^T y)_n for one pixel: for each view, project the pixel centre onto the
 * detector and take the cells within reach (widened by `extra`). */
static double og_pixel_sum_fn(const og_geom *g, const double *y, int i, int r, og_entry_fn fn, int ng,
                              double extra)
{
    double kx, ky;
    og_pixel_centre(g, i, r, &kx, &ky);
    double reach = og_reach(g) + extra;
    double smax = fabs(g->det_off) + 0.5 * g->ndet * g->ds + g->ds;
    double lmax = sqrt(g->dps * g->dps + smax * smax);
    double acc = 0.0;
    for (int k = 0; k < g->nviews; ++k) {
        og_view w = og_make_view(g, k);
        double sn = og_project_point(g, &w, kx, ky);
        double wdet = reach;
        double depth = g->dpo - (kx * w.ux + ky * w.uy);
        if (g->arc) wdet = g->dps * asin(fmin(1.0, reach / depth));
        else if (!g->parallel) wdet = reach * lmax / depth;
        double s0 = og_cell_centre(g, 0);
        int jlo = (int)ceil((sn - wdet - s0) / g->ds);
        int jhi = (int)floor((sn + wdet - s0) / g->ds);
        if (jlo < 0) jlo = 0;
        if (jhi > g->ndet - 1) jhi = g->ndet - 1;
        for (int j = jlo; j <= jhi; ++j)
            acc += y[(long)k * g->ndet + j] * fn(g, k, j, i, r, ng);
    }
    return acc;
}

static double og_pixel_sum(const og_geom *g, const double *y, int i, int r)
{
    return og_pixel_sum_fn(g, y, i, r, og_entry_cnsf_cb, 0, 0.0);
}

/* Back projection c = A^T y; c is [ny][nx]. */
void og_back(const og_geom *g, const double *y, double *c)
{
    long np = (long)g->nx * g->ny;
#pragma omp parallel for schedule(dynamic, 16)
    for (long n = 0; n < np; ++n)
        c[n] = og_pixel_sum(g, y, (int)(n % g->nx), (int)(n / g->nx));
}

/* A^T y for a list of pixels (flat indices r*nx + i) only. */
void og_back_pixels(const og_geom *g, const double *y, long nsamp, const long *pix, double *out)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (long q = 0; q < nsamp; ++q)
        out[q] = og_pixel_sum(g, y, (int)(pix[q] % g->nx), (int)(pix[q] / g->nx));
}

/* Ref operators: the same enumerations with the Ref entries (bin-averaged exact
 * chords), the reach widened by one pixel (the support of a bin's wedge is not
 * centred on the central ray). */
void og_back_ref(const og_geom *g, const double *y, double *c, int ng)
{
    long np = (long)g->nx * g->ny;
#pragma omp parallel for schedule(dynamic, 16)
    for (long n = 0; n < np; ++n)
        c[n] = og_pixel_sum_fn(g, y, (int)(n % g->nx), (int)(n / g->nx), og_entry_ref_cb, ng, g->h);
}

void og_forward_ref_rays(const og_geom *g, const double *c, long nsamp, const int *views,
                         const int *cells, double *out, int ng)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (long q = 0; q < nsamp; ++q)
        out[q] = og_ray_sum(g, c, views[q], cells[q], og_entry_ref_cb, ng, g->h, NULL);
}

void og_back_ref_pixels(const og_geom *g, const double *y, long nsamp, const long *pix, double *out, int ng)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (long q = 0; q < nsamp; ++q)
        out[q] = og_pixel_sum_fn(g, y, (int)(pix[q] % g->nx), (int)(pix[q] / g->nx), og_entry_ref_cb, ng, g->h);
}

/* Dense Ref matrix (every triple, no culling), row (view*ndet + cell), column (r*nx + i). */
void og_matrix_ref(const og_geom *g, double *a, int ng)
{
    long nr = (long)g->nviews * g->ndet, np = (long)g->nx * g->ny;
#pragma omp parallel for schedule(dynamic, 8)
    for (long kj = 0; kj < nr; ++kj)
        for (long n = 0; n < np; ++n)
            a[kj * np + n] = og_ref_entry(g, (int)(kj / g->ndet), (int)(kj % g->ndet), (int)(n % g->nx),
                                          (int)(n / g->nx), ng);
}

/* Brute force: every (view, cell, pixel) triple, no support culling. */
void og_forward_dense(const og_geom *g, const double *c, double *y)
{
    long nr = (long)g->nviews * g->ndet;
#pragma omp parallel for schedule(dynamic, 8)
    for (long kj = 0; kj < nr; ++kj) {
        double acc = 0.0;
        for (int r = 0; r < g->ny; ++r)
            for (int i = 0; i < g->nx; ++i)
                acc += c[(long)r * g->nx + i] * og_entry(g, (int)(kj / g->ndet), (int)(kj % g->ndet), i, r);
        y[kj] = acc;
    }
}

void og_back_dense(const og_geom *g, const double *y, double *c)
{
    long np = (long)g->nx * g->ny;
#pragma omp parallel for schedule(dynamic, 16)
    for (long n = 0; n < np; ++n) {
        double acc = 0.0;
        for (int k = 0; k < g->nviews; ++k)
            for (int j = 0; j < g->ndet; ++j)
                acc += y[(long)k * g->ndet + j] * og_entry(g, k, j, (int)(n % g->nx), (int)(n / g->nx));
        c[n] = acc;
    }
}

/* The dense matrix A, row (view*ndet + cell), column (r*nx + i). */
void og_matrix(const og_geom *g, double *a)
{
    long nr = (long)g->nviews * g->ndet, np = (long)g->nx * g->ny;
#pragma omp parallel for schedule(dynamic, 8)
    for (long kj = 0; kj < nr; ++kj)
        for (long n = 0; n < np; ++n)
            a[kj * np + n] = og_entry(g, (int)(kj / g->ndet), (int)(kj % g->ndet), (int)(n % g->nx),
                                      (int)(n / g->nx));
}

int og_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void og_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
