// back.cu -- back projection c = A^T y with the entries of Eq. (18).
//
// Pixel-driven gather, no atomics.  A block owns a 16 x 16 pixel tile; for each view the
// pixel centre is projected onto the detector (perspective division, Eq. 4) and the few
// cells its footprint reaches are gathered.  The projection of the whole tile is computed
// once per view in FP64 (tile_view_double) and split into an integer cell index plus a
// small remainder, so that FP32 carries the sub-cell position of every pixel to ~1e-6
// cells; the per-pixel work is then a handful of FP32 FMAs and one reciprocal.
#include <cuda_runtime.h>

#include "cnsf_internal.cuh"
#include "cnsf_runtime.h"
#include "footprint.cuh"

namespace cnsf {

constexpr int BP_T = 16;        // tile side (pixels)
constexpr int BP_CHUNK = 256;   // views whose tile coefficients are staged at once

template <typename T>
struct alignas(16) TileViewS {
    T Dt, yt, a1, b1, rho, phi, hc, hs;
};

// Per-cell constants of the pair (view, cell) in FP32: from the tables built on the host.
struct CellsF32 {
    const float4 *cell;   // ds/L, D_ps dtan/(2L), s_j dtan/(2L)
    const float4 *box;    // p, q, 1/C, h^2/(2B)  per (view, cell)
};

// One view of the pixel's gather in FP32.
__device__ __forceinline__ float bp_view_f32(const TileViewS<float> &T, int J, float di, float dr, float kr,
                                             int nd, const float *__restrict__ yrow,
                                             const float4 *__restrict__ boxrow, const float4 *__restrict__ cell)
{
    float Dn = fmaf(-T.hc, di, fmaf(-T.hs, dr, T.Dt));   // depth along u
    float yp = fmaf(-T.hs, di, fmaf(T.hc, dr, T.yt));    // coordinate along w
    float rD = __fdividef(1.0f, Dn);
    float sig = fmaf(fmaf(T.a1, di, fmaf(T.b1, dr, T.rho)), rD, T.phi);   // cell coordinate - J
    float hwc = kr * rD;
    int jlo = max((int)ceilf(sig - hwc), -J);
    int jhi = min((int)floorf(sig + hwc), nd - 1 - J);
    float part = 0.f;
    for (int jl = jlo; jl <= jhi; ++jl) {
        float4 cf = __ldg(cell + J + jl);
        float4 bx = __ldg(boxrow + J + jl);
        float d = sig - (float)jl;
        float x = fabsf(Dn * cf.x * d);                 // |s'|
        float e = fmaf(Dn, cf.y, yp * cf.z);            // tau'/2 at the pixel depth
        float hC = 0.5f * (bx.y - bx.x);
        float w = window_diff(x, e, bx.x, bx.y * bx.z, bx.z, hC);
        part = fmaf(__ldg(yrow + J + jl) * bx.w, __fdividef(w, e), part);
    }
    return part;
}

__global__ void __launch_bounds__(256) bp_f32_kernel(GeomConsts g, const double *__restrict__ view_cs,
                                                     const float4 *__restrict__ cell,
                                                     const float4 *__restrict__ box,
                                                     const float *__restrict__ sino, float *__restrict__ img,
                                                     float kr)
{
    __shared__ TileViewS<float> tv[BP_CHUNK];
    __shared__ int tj[BP_CHUNK];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BP_T + tx;
    const int it = blockIdx.x * BP_T, rt = blockIdx.y * BP_T;
    const long long b = blockIdx.z;
    const int i = it + tx, r = rt + ty;
    const bool inside = i < g.nx && r < g.ny;
    const float *y = sino + b * (long long)g.nv * g.nd;
    const float di = (float)tx, dr = (float)ty;
    float acc = 0.f;
    for (int v0 = 0; v0 < g.nv; v0 += BP_CHUNK) {
        const int nvc = min(BP_CHUNK, g.nv - v0);
        __syncthreads();
        if (tid < nvc) {
            double c = view_cs[2 * (v0 + tid)], s = view_cs[2 * (v0 + tid) + 1];
            double Dt, yt, a1, b1, rho, phi;
            int J;
            tile_view_double(g, c, s, it, rt, &Dt, &yt, &a1, &b1, &rho, &phi, &J);
            TileViewS<float> T;
            T.Dt = (float)Dt; T.yt = (float)yt; T.a1 = (float)a1; T.b1 = (float)b1;
            T.rho = (float)rho; T.phi = (float)phi; T.hc = (float)(g.h * c); T.hs = (float)(g.h * s);
            tv[tid] = T;
            tj[tid] = J;
        }
        __syncthreads();
        if (inside) {
            float part = 0.f;
            for (int vv = 0; vv < nvc; ++vv) {
                const int v = v0 + vv;
                part += bp_view_f32(tv[vv], tj[vv], di, dr, kr, g.nd, y + (long long)v * g.nd,
                                    box + (long long)v * g.nd, cell);
                if ((vv & 15) == 15) {   // blocked summation over groups of 16 views
                    acc += part;
                    part = 0.f;
                }
            }
            acc += part;
        }
    }
    if (inside) img[(b * g.ny + r) * g.nx + i] = acc;
}

// FP64: same tiling and enumeration; every per-pair constant is recomputed in FP64 from
// the view and cell angles.
__global__ void __launch_bounds__(256) bp_f64_kernel(GeomConsts g, const double *__restrict__ view_cs,
                                                     const double *__restrict__ celld,
                                                     const double *__restrict__ sino, double *__restrict__ img,
                                                     double kr)
{
    __shared__ TileViewS<double> tv[BP_CHUNK / 2];
    __shared__ int tj[BP_CHUNK / 2];
    __shared__ double tcs[BP_CHUNK / 2][2];
    const int chunk = BP_CHUNK / 2;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BP_T + tx;
    const int it = blockIdx.x * BP_T, rt = blockIdx.y * BP_T;
    const long long b = blockIdx.z;
    const int i = it + tx, r = rt + ty;
    const bool inside = i < g.nx && r < g.ny;
    const double *y = sino + b * (long long)g.nv * g.nd;
    const double di = tx, dr = ty;
    double acc = 0.0;
    for (int v0 = 0; v0 < g.nv; v0 += chunk) {
        const int nvc = min(chunk, g.nv - v0);
        __syncthreads();
        if (tid < nvc) {
            double c = view_cs[2 * (v0 + tid)], s = view_cs[2 * (v0 + tid) + 1];
            TileViewS<double> T;
            int J;
            tile_view_double(g, c, s, it, rt, &T.Dt, &T.yt, &T.a1, &T.b1, &T.rho, &T.phi, &J);
            T.hc = g.h * c;
            T.hs = g.h * s;
            tv[tid] = T;
            tj[tid] = J;
            tcs[tid][0] = c;
            tcs[tid][1] = s;
        }
        __syncthreads();
        if (!inside) continue;
        for (int vv = 0; vv < nvc; ++vv) {
            const TileViewS<double> T = tv[vv];
            const int J = tj[vv];
            const double c = tcs[vv][0], s = tcs[vv][1];
            const double *yrow = y + (long long)(v0 + vv) * g.nd;
            double Dn = T.Dt - T.hc * di - T.hs * dr;
            double yp = T.yt - T.hs * di + T.hc * dr;
            double sig = T.phi + (T.rho + T.a1 * di + T.b1 * dr) / Dn;
            double hwc = kr / Dn;
            int jlo = max((int)ceil(sig - hwc), -J);
            int jhi = min((int)floor(sig + hwc), g.nd - 1 - J);
            double part = 0.0;
            for (int jl = jlo; jl <= jhi; ++jl) {
                const int j = J + jl;
                double sj = celld[4 * j], L = celld[4 * j + 1], dt = celld[4 * j + 2];
                double nxv = (sj * c - g.dps * s) / L, nyv = (sj * s + g.dps * c) / L;
                double B = g.h * fmax(fabs(nxv), fabs(nyv)), C = g.h * fmin(fabs(nxv), fabs(nyv));
                BoxConsts<double> bc = make_box_consts<double>(B, C, g.h);
                double x = fabs(Dn * (g.ds / L) * (sig - jl));
                double e = (g.dps * Dn + sj * yp) / L * 0.5 * dt;
                double w = window_diff(x, e, bc.p, bc.q * bc.iC, bc.iC, 0.5 * C);
                part += yrow[j] * bc.nrm * (w / e);
            }
            acc += part;
        }
    }
    if (inside) img[(b * g.ny + r) * g.nx + i] = acc;
}

int launch_back(const cnsf_geometry *geo, const void *sino, void *img, int batch, int dtype, cudaStream_t st)
{
    if (batch == 0) return CNSF_OK;
    const GeomConsts &g = geo->gc;
    dim3 blk(BP_T, BP_T), grd((g.nx + BP_T - 1) / BP_T, (g.ny + BP_T - 1) / BP_T, batch);
    if (dtype == CNSF_F32)
        bp_f32_kernel<<<grd, blk, 0, st>>>(g, geo->d_view_cs, (const float4 *)geo->d_cell_f,
                                           (const float4 *)geo->d_box, (const float *)sino, (float *)img,
                                           (float)geo->kr);
    else
        bp_f64_kernel<<<grd, blk, 0, st>>>(g, geo->d_view_cs, geo->d_cell_d, (const double *)sino, (double *)img,
                                           geo->kr);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? CNSF_OK : record_cuda_error(e);
}

}  // namespace cnsf
