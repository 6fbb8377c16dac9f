// reference.cu -- the reference projector (Ref) of Sec. IV on the GPU.
//
// Every entry is the bin average of the exact line integrals of the pixel indicator (Eq. 1,
// 2 with the detector blur of a cell of width tau):
//   a_ref(view, cell j, pixel) = (1/tau) int_{s_j - tau/2}^{s_j + tau/2} chord(s) ds,
// with chord(s) the length of the ray of detector coordinate s inside the pixel square.
// chord(s) is smooth between the detector coordinates of the four pixel corners (where the
// ray enters or leaves through another edge), so the integral is split there and each smooth
// piece is integrated by 6-point Gauss-Legendre, which is exact to rounding for these
// pieces (the nearest singularity of a piece lies many piece-widths away).  FP64 throughout,
// whatever the dtype of the images and sinograms.
//
// Forward: one warp per (view, cell) walks every line of the image along the axis its
// central ray crosses most steeply (lane l the lines l, l + 32, ...) and takes the pixels
// that the cell's wedge (the two rays through the cell edges) reaches on that line.  Back:
// one thread per pixel takes, for each view, the cells whose bin meets the pixel's shadow
// [min corner, max corner].  Both use the same entry function, so the two operators are
// adjoint to rounding.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "cnsf_internal.cuh"
#include "cnsf_runtime.h"

namespace cnsf {

// Gauss-Legendre, 6 points on [-1, 1]: the positive roots of P_6 and their weights.
__constant__ double c_gl6_x[3] = {0.2386191860831969086305017, 0.6612093864662645136613996,
                                  0.9324695142031520278123016};
__constant__ double c_gl6_w[3] = {0.4679139345726910473898703, 0.3607615730481386075698335,
                                  0.1713244923791703450402961};

// The ray of detector coordinate sd in the view (c, s) = (cos, sin) of theta: a point o on
// it and a direction v (not normalised), |v| returned.  Flat: from the source p = D_po u
// towards d + sd w; arc: from p at the angle sd/D_ps from -u; parallel: through sd w along -u.
struct RefRay {
    double ox, oy, vx, vy, len;
};

__device__ __forceinline__ RefRay ref_ray(const GeomConsts &g, double c, double s, double sd)
{
    RefRay R;
    if (g.par) {
        R.ox = -sd * s; R.oy = sd * c;
        R.vx = -c; R.vy = -s;
        R.len = 1.0;
        return R;
    }
    double a, b;   // v = -a u + b w
    if (g.arc) {
        sincos(sd / g.dps, &b, &a);
        R.len = 1.0;
    } else {
        a = g.dps;
        b = sd;
        R.len = sqrt(a * a + b * b);
    }
    R.ox = g.dpo * c; R.oy = g.dpo * s;
    R.vx = -a * c - b * s; R.vy = -a * s + b * c;
    return R;
}

// Length of the ray inside the square of half-side hh centred at (kx, ky) (slab clipping of
// the full line; every pixel lies in front of the source, so the part behind it misses).
__device__ __forceinline__ double ref_chord(const RefRay &R, double kx, double ky, double hh)
{
    double t0 = -INFINITY, t1 = INFINITY;
    if (R.vx != 0.0) {
        const double iv = 1.0 / R.vx;
        const double ta = (kx - hh - R.ox) * iv, tb = (kx + hh - R.ox) * iv;
        t0 = fmax(t0, fmin(ta, tb));
        t1 = fmin(t1, fmax(ta, tb));
    } else if (fabs(R.ox - kx) > hh) {
        return 0.0;
    }
    if (R.vy != 0.0) {
        const double iv = 1.0 / R.vy;
        const double ta = (ky - hh - R.oy) * iv, tb = (ky + hh - R.oy) * iv;
        t0 = fmax(t0, fmin(ta, tb));
        t1 = fmin(t1, fmax(ta, tb));
    } else if (fabs(R.oy - ky) > hh) {
        return 0.0;
    }
    return t1 > t0 ? (t1 - t0) * R.len : 0.0;
}

// Detector coordinate of the point (x, y) (the projection P of Eq. 4, or its arc and
// parallel counterparts).
__device__ __forceinline__ double ref_project(const GeomConsts &g, double c, double s, double x, double y)
{
    const double yw = -x * s + y * c;
    if (g.par) return yw;
    const double D = g.dpo - (x * c + y * s);
    return g.arc ? g.dps * atan2(yw, D) : g.dps * yw / D;
}

__device__ __forceinline__ void cswap(double &a, double &b)
{
    const double lo = fmin(a, b), hi = fmax(a, b);
    a = lo;
    b = hi;
}

// The pixel's four corner coordinates on the detector, sorted.
__device__ __forceinline__ void ref_corners(const GeomConsts &g, double c, double s, double kx, double ky, double hh,
                                            double q[4])
{
    q[0] = ref_project(g, c, s, kx - hh, ky - hh);
    q[1] = ref_project(g, c, s, kx + hh, ky - hh);
    q[2] = ref_project(g, c, s, kx - hh, ky + hh);
    q[3] = ref_project(g, c, s, kx + hh, ky + hh);
    cswap(q[0], q[1]);
    cswap(q[2], q[3]);
    cswap(q[0], q[2]);
    cswap(q[1], q[3]);
    cswap(q[1], q[2]);
}

// (1/tau) int over [lo, hi] of the chord, split at the sorted corner coordinates q.
__device__ double ref_entry(const GeomConsts &g, double c, double s, double kx, double ky, const double q[4],
                            double lo, double hi)
{
    const double a = fmax(lo, q[0]), b = fmin(hi, q[3]);
    if (!(b > a)) return 0.0;
    const double hh = 0.5 * g.h;
    const double br[4] = {a, fmin(fmax(q[1], a), b), fmin(fmax(q[2], a), b), b};
    double sum = 0.0;
    for (int p = 0; p < 3; ++p) {
        const double l = br[p], r = br[p + 1];
        if (!(r > l)) continue;
        const double m = 0.5 * (l + r), hw = 0.5 * (r - l);
        double part = 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double d = hw * c_gl6_x[k];
            part += c_gl6_w[k] * (ref_chord(ref_ray(g, c, s, m - d), kx, ky, hh) +
                                  ref_chord(ref_ray(g, c, s, m + d), kx, ky, hh));
        }
        sum += part * hw;
    }
    return sum / g.tau;
}

// One warp per ray: lane l takes the lines l, l + 32, ...; the lanes' sums are combined by
// a fixed shuffle tree (the result does not depend on scheduling).
template <typename T>
__global__ void __launch_bounds__(128) ref_fp_kernel(GeomConsts g, const double *__restrict__ view_cs,
                                                     const T *__restrict__ img, T *__restrict__ sino)
{
    const int nr = g.nv * g.nd;
    const int lane = threadIdx.x & 31;
    const int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (q >= nr) return;   // whole warps leave together
    const long long b = blockIdx.y;
    const int k = q / g.nd, j = q - k * g.nd;
    const double c = view_cs[2 * k], s = view_cs[2 * k + 1];
    const double sj = cell_centre(g, j), lo = sj - 0.5 * g.tau, hi = sj + 0.5 * g.tau, hh = 0.5 * g.h;
    const T *im = img + b * (long long)g.nx * g.ny;
    // walk axis of the central ray: rows (b = y) when it is steeper in y
    const RefRay Rc = ref_ray(g, c, s, sj);
    const bool tr = fabs(Rc.vy) < fabs(Rc.vx);
    const RefRay E[2] = {ref_ray(g, c, s, lo), ref_ray(g, c, s, hi)};
    const int na = tr ? g.ny : g.nx, nb = tr ? g.nx : g.ny;
    const double ca = tr ? g.cy : g.cx, cb = tr ? g.cx : g.cy;
    double acc = 0.0;
    for (int rb = lane; rb < nb; rb += 32) {
        const double yb = cb + (rb - 0.5 * (nb - 1)) * g.h;
        // a-extent of the wedge within the band |b - yb| <= h/2: its vertices are the edge
        // crossings of the band's two sides, plus the ray origin when it lies in the band
        double amin = INFINITY, amax = -INFINITY;
        bool all = false;
        for (int e = 0; e < 2; ++e) {
            const double oa = tr ? E[e].oy : E[e].ox, ob = tr ? E[e].ox : E[e].oy;
            const double va = tr ? E[e].vy : E[e].vx, vb = tr ? E[e].vx : E[e].vy;
            if (fabs(vb) < 1e-12 * (fabs(va) + fabs(vb))) { all = true; break; }
            for (int side = 0; side < 2; ++side) {
                const double a = oa + (yb + (side ? hh : -hh) - ob) * (va / vb);
                amin = fmin(amin, a);
                amax = fmax(amax, a);
            }
            if (!g.par && fabs(ob - yb) <= hh) {
                amin = fmin(amin, oa);
                amax = fmax(amax, oa);
            }
        }
        int ilo = 0, ihi = na - 1;
        if (!all) {
            const double flo = ceil((amin - hh - ca) / g.h + 0.5 * (na - 1));
            const double fhi = floor((amax + hh - ca) / g.h + 0.5 * (na - 1));
            if (!(flo <= fhi) || fhi < 0.0 || flo > na - 1.0) continue;
            ilo = (int)fmax(flo, 0.0);
            ihi = (int)fmin(fhi, na - 1.0);
        }
        for (int ia = ilo; ia <= ihi; ++ia) {
            const int i = tr ? rb : ia, r = tr ? ia : rb;
            const double kx = g.cx + (i - 0.5 * (g.nx - 1)) * g.h, ky = g.cy + (r - 0.5 * (g.ny - 1)) * g.h;
            double qc[4];
            ref_corners(g, c, s, kx, ky, hh, qc);
            const double w = ref_entry(g, c, s, kx, ky, qc, lo, hi);
            if (w != 0.0) acc += (double)im[(long long)r * g.nx + i] * w;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) sino[b * nr + q] = (T)acc;
}

template <typename T>
__global__ void __launch_bounds__(128) ref_bp_kernel(GeomConsts g, const double *__restrict__ view_cs,
                                                     const T *__restrict__ sino, T *__restrict__ img)
{
    const int np = g.nx * g.ny;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= np) return;
    const long long b = blockIdx.y;
    const int i = n % g.nx, r = n / g.nx;
    const double kx = g.cx + (i - 0.5 * (g.nx - 1)) * g.h, ky = g.cy + (r - 0.5 * (g.ny - 1)) * g.h;
    const double hh = 0.5 * g.h, ht = 0.5 * g.tau;
    const T *y = sino + b * (long long)g.nv * g.nd;
    double acc = 0.0;
    for (int k = 0; k < g.nv; ++k) {
        const double c = view_cs[2 * k], s = view_cs[2 * k + 1];
        double qc[4];
        ref_corners(g, c, s, kx, ky, hh, qc);
        // bins [s_j - tau/2, s_j + tau/2] that meet [q0, q3]
        const double flo = floor((qc[0] - ht - g.s0) / g.ds), fhi = ceil((qc[3] + ht - g.s0) / g.ds);
        if (fhi < 0.0 || flo > g.nd - 1.0) continue;
        const int jlo = (int)fmax(flo, 0.0), jhi = (int)fmin(fhi, g.nd - 1.0);
        double part = 0.0;
        for (int j = jlo; j <= jhi; ++j) {
            const double sj = cell_centre(g, j);
            const double w = ref_entry(g, c, s, kx, ky, qc, sj - ht, sj + ht);
            if (w != 0.0) part += (double)y[(long long)k * g.nd + j] * w;
        }
        acc += part;
    }
    img[b * (long long)np + n] = (T)acc;
}

int launch_forward_ref(const cnsf_geometry *geo, const void *img, void *sino, int batch, int dtype, cudaStream_t st)
{
    if (batch == 0) return CNSF_OK;
    const GeomConsts &g = geo->gc;
    const int nr = g.nv * g.nd;
    dim3 blk(128), grd((nr + 3) / 4, batch);   // four rays (warps) per block
    if (dtype == CNSF_F32)
        ref_fp_kernel<float><<<grd, blk, 0, st>>>(g, geo->d_view_cs, (const float *)img, (float *)sino);
    else
        ref_fp_kernel<double><<<grd, blk, 0, st>>>(g, geo->d_view_cs, (const double *)img, (double *)sino);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? CNSF_OK : record_cuda_error(e);
}

int launch_back_ref(const cnsf_geometry *geo, const void *sino, void *img, int batch, int dtype, cudaStream_t st)
{
    if (batch == 0) return CNSF_OK;
    const GeomConsts &g = geo->gc;
    const int np = g.nx * g.ny;
    dim3 blk(128), grd((np + 127) / 128, batch);
    if (dtype == CNSF_F32)
        ref_bp_kernel<float><<<grd, blk, 0, st>>>(g, geo->d_view_cs, (const float *)sino, (float *)img);
    else
        ref_bp_kernel<double><<<grd, blk, 0, st>>>(g, geo->d_view_cs, (const double *)sino, (double *)img);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? CNSF_OK : record_cuda_error(e);
}

}  // namespace cnsf
