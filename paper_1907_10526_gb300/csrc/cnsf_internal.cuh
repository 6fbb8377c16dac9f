// cnsf_internal.cuh -- geometry constants, table layouts and the per-ray /
// per-tile parameter derivations shared by the host table builder and the
// device kernels of the CNSF projector.
//
// Notation (Zhang & Entezari, Sec. II.A, III.B-C):
//   u = (cos t, sin t), w = (-sin t, cos t); source p = D_po u;
//   cell j centre s_j on the detector line at distance D_ps from the source;
//   central ray direction v_j = (-D_ps u + s_j w)/L_j, L_j = sqrt(D_ps^2 + s_j^2);
//   its unit normal n_j = (s_j u + D_ps w)/L_j spans v(s)perp;
//   zeta_1 = h n_x, zeta_2 = h n_y (Eq. 16); s' = n_j . (k - p);
//   t = v_j . (k - p) the depth of pixel centre k along the central ray;
//   tau' = t * dtan_j (Eq. 17, reading: perspective-divided edge coordinates
//   scaled to the pixel depth), dtan_j = tan(phi+) - tan(phi-), phi+- the angles
//   of the two cell edges from the central ray.
#pragma once

#include <cstdint>
#include <cmath>

#ifndef __CUDACC__
#define __host__
#define __device__
#define __forceinline__ inline
#endif

namespace cnsf {

// Plain numbers of a geometry, passed by value to every kernel.
struct GeomConsts {
    int nx, ny, nv, nd;
    double h, cx, cy;
    double ds, tau, doff;
    double dpo, dps;
    double rimg;      // distance from the rotation centre to the farthest image corner
    double s0;        // centre of cell 0
    int par;          // 1: parallel beam (Theorem 1): rays along -u, s = x . w, tau' = tau
    int arc;          // 1: fan beam onto the arc of radius D_ps about the source (s = arc length)
};

// Per-cell quantities that do not depend on the view.
__host__ __device__ inline double cell_centre(const GeomConsts &g, int j)
{
    return (j - 0.5 * (g.nd - 1)) * g.ds + g.doff;
}

// tan(phi+) - tan(phi-) for cell j: the two cell edges seen from the source in the frame of
// the central ray (the perspective division of Eq. 17 at unit depth).
__host__ __device__ inline double cell_dtan(const GeomConsts &g, double sj)
{
    double d2 = g.dps * g.dps + sj * sj, ht = 0.5 * g.tau;
    return ht * g.dps * (1.0 / (d2 + sj * ht) + 1.0 / (d2 - sj * ht));
}

// Direction of the central ray of cell j in the rotating frame: v_j = -cos(g_j) u + sin(g_j) w,
// normal n_j = sin(g_j) u + cos(g_j) w, and the blur slope dtan_j (tau' = depth * dtan_j).
// Flat detector: sin = s_j/L_j, cos = D_ps/L_j, dtan from the cell edges (cell_dtan).
// Arc detector: g_j = s_j/D_ps and both edges sit at +-tau/(2 D_ps) from the central ray, so
// dtan_j = 2 tan(tau/(2 D_ps)) for every cell.
__host__ __device__ inline void cell_dir(const GeomConsts &g, double sj, double *sg, double *cg, double *dtan)
{
    if (g.arc) {
        double ga = sj / g.dps;
        *sg = sin(ga);
        *cg = cos(ga);
        *dtan = 2.0 * tan(0.5 * g.tau / g.dps);
    } else {
        double L = sqrt(g.dps * g.dps + sj * sj);
        *sg = sj / L;
        *cg = g.dps / L;
        *dtan = cell_dtan(g, sj);
    }
}

// Ray parameters of one (view, cell) in the walk frame.  The walk runs over the image
// axis "b" that the ray crosses most steeply (rows when |v_y| >= |v_x|, otherwise columns of
// the transposed image); along each crossed line the candidate pixels are indexed by the
// other axis "a".  For a pixel at a-index ia on the line b = rb, with crossing f(rb):
//   s'  = sign * B * (ia - f(rb))            (B = h |n_a| >= h/sqrt 2)
//   t   = lambda(rb) + va h (ia - f(rb))      (depth along the central ray)
//   e   = tau'/2 = e(rb) + kap (ia - f(rb)),  e(rb) = e0 + rb de
template <typename T>
struct RayParams {
    T f0, g;          // f(rb) = f0 + rb g, a-index of the crossing of line rb
    T e0, de, kap;    // half effective blur along the walk (mm)
    T B, C;           // h|n_a| >= h|n_b|: the two footprint widths (Eq. 16)
    T dtan;           // tan(phi+) - tan(phi-)
    int transposed;   // 0: walk rows (b = y); 1: walk columns (b = x)
    int na, nb;       // image extent across / along the walk
};

// Parallel beam: the ray of cell j is the line through s_j w along v = -u, its normal is w, and
// the blur is tau at every depth (e = tau/2, de = kap = 0, dtan = 0).
template <typename T>
__host__ __device__ inline RayParams<T> make_ray_params(const GeomConsts &g, double c, double s, int j)
{
    double sj = cell_centre(g, j);
    double vx, vy, nxv, nyv, px, py, dtan;
    if (g.par) {
        vx = -c; vy = -s; nxv = -s; nyv = c;
        px = -sj * s; py = sj * c;
        dtan = 0.0;
    } else {
        double sg, cg;
        cell_dir(g, sj, &sg, &cg, &dtan);
        vx = -cg * c - sg * s; vy = -cg * s + sg * c;
        nxv = sg * c - cg * s; nyv = sg * s + cg * c;
        px = g.dpo * c; py = g.dpo * s;
    }
    RayParams<T> R;
    int tr = fabs(vy) >= fabs(vx) ? 0 : 1;
    double va, vb, na_, nb_, pa, pb, ca, cb;
    int Na, Nb;
    if (!tr) {
        va = vx; vb = vy; na_ = nxv; nb_ = nyv; pa = px; pb = py; ca = g.cx; cb = g.cy; Na = g.nx; Nb = g.ny;
    } else {
        va = vy; vb = vx; na_ = nyv; nb_ = nxv; pa = py; pb = px; ca = g.cy; cb = g.cx; Na = g.ny; Nb = g.nx;
    }
    // source in index units of the walk frame
    double PA = (pa - ca) / g.h + 0.5 * (Na - 1);
    double PB = (pb - cb) / g.h + 0.5 * (Nb - 1);
    double gg = va / vb;
    R.f0 = (T)(PA - PB * gg);
    R.g = (T)gg;
    // lambda(rb) = (rb - PB) h / vb
    R.e0 = (T)(g.par ? 0.5 * g.tau : (-PB * g.h / vb) * 0.5 * dtan);
    R.de = (T)((g.h / vb) * 0.5 * dtan);
    R.kap = (T)(va * g.h * 0.5 * dtan);
    R.B = (T)(g.h * fabs(na_));
    R.C = (T)(g.h * fabs(nb_));
    R.dtan = (T)dtan;
    R.transposed = tr;
    R.na = Na;
    R.nb = Nb;
    return R;
}

// Box-spline constants of one ray: trapezoid box_B * box_C with plateau half-width p and
// outer half-width q, the reciprocal of C (clamped so that C = 0 stays finite) and the
// normalisation h^2 / (2B) of the blurred footprint (Eq. 18 with the pixel area).
template <typename T>
struct BoxConsts {
    T p, q, iC, nrm;
};

template <typename T>
__host__ __device__ inline BoxConsts<T> make_box_consts(double B, double C, double h)
{
    BoxConsts<T> b;
    b.p = (T)(0.5 * (B - C));
    b.q = (T)(0.5 * (B + C));
    double Cc = C > 1e-30 * h ? C : 1e-30 * h;
    b.iC = (T)(1.0 / Cc);
    b.nrm = (T)(h * h / (2.0 * B));
    return b;
}

// Per (pixel tile, view) coefficients of the back projector.  For the pixel at offset
// (di, dr) from the tile's reference point:
//   D_n   = Dt + aD di + bD dr            (depth of the pixel centre along u from the source)
//   y'    = yt + ay di + by dr            (coordinate along w)
//   sigma = J + phi + (rho + a1 di + b1 dr) / D_n
// where sigma is the continuous cell coordinate of the pixel centre's perspective
// projection (Eq. 4), split into an integer J and a small remainder so that FP32 keeps it
// to ~1e-6 cells.
template <typename T>
struct TileView {
    T Dt, yt, a1, b1, rho, phi;
    int J;
};

// (it, rt) is the reference point of the tile in pixel-index units (the centre of the
// tile's part inside the image, so that the per-pixel offsets stay small and the point lies
// in front of the source).  (hc, hs) = h (cos, sin) is the per-pixel step of the depth.
// Parallel beam: the projection is affine, sigma = (y' - s_0)/ds; the depth is held at
// D_n = 1 (hc = hs = 0) so that the same per-pixel arithmetic applies.
// Arc detector: sigma = (D_ps atan2(y', D_n) - s_0)/ds.  Relative to the reference point,
//   sigma = J + phi + (D_ps/ds) atan((a1 di + b1 dr) / (D_n Dt + y' yt)),
// where a1 di + b1 dr = y' Dt - yt D_n exactly (no constant term, so no cancellation), and
// rho = 0.
__host__ __device__ inline void tile_view_double(const GeomConsts &g, double c, double s, double it, double rt,
                                                 double *Dt, double *yt, double *a1, double *b1,
                                                 double *rho, double *phi, int *J, double *hc, double *hs)
{
    double kx = g.cx + (it - 0.5 * (g.nx - 1)) * g.h;
    double ky = g.cy + (rt - 0.5 * (g.ny - 1)) * g.h;
    double xu = kx * c + ky * s, yw = -kx * s + ky * c;
    double ay = -g.h * s, by = g.h * c;
    double D, aD, bD, Nt, aN, bN;
    if (g.par) {
        D = 1.0; aD = 0.0; bD = 0.0;
        Nt = (yw - g.s0) / g.ds; aN = ay / g.ds; bN = by / g.ds;
        *hc = 0.0; *hs = 0.0;
    } else {
        D = g.dpo - xu; aD = -g.h * c; bD = -g.h * s;
        Nt = (g.dps * yw - g.s0 * D) / g.ds;
        aN = (g.dps * ay - g.s0 * aD) / g.ds;
        bN = (g.dps * by - g.s0 * bD) / g.ds;
        *hc = g.h * c; *hs = g.h * s;
    }
    double sig = Nt / D;
    if (g.arc) sig = (g.dps * atan2(yw, D) - g.s0) / g.ds;
    double Jd = floor(sig);
    *Dt = D;
    *yt = yw;
    if (g.arc) {
        *a1 = ay * D - yw * aD;
        *b1 = by * D - yw * bD;
        *rho = 0.0;
    } else {
        *a1 = aN - sig * aD;
        *b1 = bN - sig * bD;
        *rho = Nt - sig * D;
    }
    *phi = sig - Jd;
    *J = (int)Jd;
}

// Fixed-point (32.32) form of the forward walk used by the FP32 kernel.
struct RayF {
    long long A0;     // fixed point of f(r0) - hw at the first walked line
    long long G;      // fixed point of the per-line slope g
    float e0, de;     // half blur at the first walked line and per line
    float kap;        // half blur per unit a-offset within a line
    float hw;         // candidate half-window (a-index units)
    int r0, nrows;    // first walked line and number of lines
    int kc;           // candidates per line
    int flags;        // bit 0: transposed walk
};
static_assert(sizeof(RayF) == 48, "RayF layout");

// The table's candidate window covers the blur at the deepest point of the whole image.
// For the lines this thread walks, the blur is at most e_max = max(e at the first and the
// last line) plus |kap| per unit offset, so every non-zero entry satisfies
// |u| < ((B + C)/2 + e_max)/(B - |kap|): shrink the window to that (when narrower), moving
// its fixed-point start by the same amount, and walk fewer candidates per line.
#ifdef __CUDACC__
__device__ __forceinline__ void tighten_window(RayF &R, float q, float B)
{
    const float emax = fmaxf(R.e0, fmaf((float)(R.nrows - 1), R.de, R.e0));
    const float hw = (q + emax) / (B - fabsf(R.kap)) + 1e-3f;
    if (hw < R.hw) {
        const long long D = __float2ll_rz((R.hw - hw) * 4294967296.0f);   // >= 0, in 32.32 units
        R.A0 += D;
        R.hw -= __ll2float_rn(D) * (1.0f / 4294967296.0f);
        R.kc = min(R.kc, (int)floorf(2.f * R.hw) + 1);
    }
}
#endif

// Per-(view, cell) trapezoid constants of the FP32 kernels: box_B * box_C (Eq. 16 widths)
// as its outer half-width q = (B + C)/2, p/C with p = (B - C)/2 the plateau half-width,
// 1/C (clamped for C = 0) and C/2.  B = 2(q - C/2); the normalisation of Eq. (18) with the
// pixel area is h^2/(2B).
struct alignas(16) BoxF {
    float q, piC, iC, hC;
};

// Per-cell constants of the FP32 back projector: s' = D_n g1 (sigma - j) and
// tau'/2 = D_n c1 + y' c2 for a pixel at depth D_n and coordinate y' along w.
struct alignas(16) CellF {
    float g1, c1, c2, pad;   // ds/L_j, cos(g_j) dtan_j/2, sin(g_j) dtan_j/2 (flat: cos = D_ps/L_j)
};

// Pair constants of the FP32 back projector: entry m of parity o holds cells 2m + o and
// 2m + o + 1 side by side, so the two cells' values come as FP32 pairs for the packed
// (FFMA2) arithmetic, and a window can start its pairs at any cell.  A cell past n_det
// repeats the last cell's constants (its sinogram value is 0).  Each entry is 32 bytes,
// read with one 256-bit load: per (parity, view, pair) the trapezoid constants (q, p/C,
// 1/C, -C/2 of both cells), per (parity, pair) the view-independent cell slopes (ds/L_j,
// cos(g_j) dtan_j/2, sin(g_j) dtan_j/2 of both cells), a table of a few KB that stays in
// L1 across views.  The normalisation 2/B of each (view, cell) is applied to the sinogram
// value when the call builds its cell pairs.

// Back-projector cell window (cells) of a pixel at depth D_n, coordinate y' along w:
//   hwc = kz * h(|y' c - D_n s| + |y' s + D_n c|) / D_n^2 * (1.02 + 2 h / D_n) + ke
// The first term is (zeta1 + zeta2)/2 * L / (D_n ds) for the ray through the pixel centre
// (the widths of Eq. 16 on that ray, with slack for the neighbouring cell rays), the second
// bounds tau'/2 * L / (D_n ds) = (D_ps + s_j s_n / D_ps) dtan_j / (2 ds).
struct BpWindow {
    double kz, ke;
};

}  // namespace cnsf

// Host-side geometry object behind the opaque handle.
// Blocks of the eight-value forward walk: FP8_VT consecutive base views x FP8_CT consecutive
// cells (128 threads).  Rays of neighbouring views and cells cross nearly the same pixels, so
// a block of a few views over fewer cells walks a narrower band of the image than 128 cells of
// one view, and more of its loads hit L1.
constexpr int FP8_VT = 4;
constexpr int FP8_CT = 128 / FP8_VT;
#ifdef __CUDACC__
#define CNSF_HD __host__ __device__
#else
#define CNSF_HD
#endif
CNSF_HD inline int fp8_cell_tiles(int nd) { return (nd + FP8_CT - 1) / FP8_CT; }
CNSF_HD inline int fp8_blocks(int nv, int nd) { return ((nv / 8 + 1 + FP8_VT - 1) / FP8_VT) * fp8_cell_tiles(nd); }

struct cnsf_geometry {
    cnsf::GeomConsts gc;
    int device;
    int pad;                  // zero columns on each side of the padded image copies
    int kc_max;               // largest candidate count per walked line
    size_t device_bytes;      // device memory held by the tables below
    int sym;                  // 1: FP32 single-image projections reuse entries over the quarter turn
    int sym8;                 // 1: and over the reflection (views 0 .. nv/8 evaluated)
    int exact;                // 1: FP32 kernels form window differences piece by piece
    cnsf::BpWindow bw;        // back projector cell window
    // device tables
    double *d_view_cs;        // [nv][2] cos, sin (FP64)
    double *d_cell_d;         // [nd][4] sin(g_j), cos(g_j), dtan_j, s_j (FP64; parallel: 0, 1, 0, s_j)
    cnsf::BoxF *d_box;        // [nv][nd]
    cnsf::CellF *d_cellf;     // [nd]
    float *d_box2;            // [2][nv][ceil(n_det/2)][8]: q, p/C, 1/C, -C/2 of cells 2m + o, 2m + o + 1
    float *d_cell2;           // [2][ceil(n_det/2)][8]: ds/L, c1, c2 of cells 2m + o, 2m + o + 1, 0, 0
    // launch orders, heaviest blocks first (so that the tail of the grid is short work)
    int *d_fp_order;          // [ceil(nv*nd/128)] forward blocks of 128 rays
    int *d_fp_order4;         // [ceil(nv/4*nd/128)] the same over the rays of views < nv/4 (sym only)
    int *d_fp_order8;         // [ceil((nv/8+1)*nd/128)] the same over views 0 .. nv/8 (sym8 only)
    float *d_ac;              // [2][nv/4][ceil(n_det/2)][8]: q/C, p/C, ds/(L C), c1/C of cells 2m + o, 2m + o + 1 (sym only)
    int *d_bp_order;          // [ceil(nx/16)*ceil(ny/16)] back-projection tiles
    float4 *d_tv;             // [tiles][nv][2] FP32 back-projection tile coefficients (when <= 1 GiB), or null
    int *d_tj;                // [tiles][nv] their integer cell offsets
    cnsf::RayF *d_ray;        // [nv][nd]
};
