// back.cu -- back projection c = A^T y with the entries of Eq. (18).
//
// Pixel-driven gather, no atomics.  A block owns a 16 x 16 pixel tile; for each view the
// pixel centre is projected onto the detector (perspective division, Eq. 4) and the cells
// its footprint reaches are gathered.  The projection of the tile centre is computed once
// per view in FP64 (tile_view_double) and split into an integer cell index plus a small
// remainder, so that FP32 carries the sub-cell position of every pixel to ~1e-6 cells;
// the per-pixel work is then a handful of FP32 FMAs and one reciprocal.  The cell window
// is bounded per pixel from the footprint widths of the ray through the pixel centre
// (BpWindow), so few cells outside the support are visited.
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

struct BpArgs {
    float kz, ke, h2;   // window constants; h2 = 2h
    float h2q;          // h^2 / 4
};

// One view of the pixel's gather in FP32.  Per candidate cell it reads the trapezoid
// constants of the (view, cell) pair, the cell's s' and tau' slopes and the sinogram value;
// the normalisation h^2/(2B) = h^2/(4(p + C/2)) is folded into the division by tau'.
__device__ __forceinline__ float bp_view_f32(const TileViewS<float> &T, int J, float di, float dr,
                                             const BpArgs &a, int nd, const float *__restrict__ yrow,
                                             const float4 *__restrict__ boxrow, const float4 *__restrict__ cell)
{
    const float Dn = fmaf(-T.hc, di, fmaf(-T.hs, dr, T.Dt));   // depth along u
    const float yp = fmaf(-T.hs, di, fmaf(T.hc, dr, T.yt));    // coordinate along w
    const float rD = rcp_approx(Dn);
    const float sig = fmaf(fmaf(T.a1, di, fmaf(T.b1, dr, T.rho)), rD, T.phi);   // cell coordinate - J
    // footprint widths of the ray through the pixel centre: h(|n_x| + |n_y|) * rho
    const float za = fmaf(yp, T.hc, -Dn * T.hs), zb = fmaf(yp, T.hs, Dn * T.hc);
    const float zs = fabsf(za) + fabsf(zb);
    const float hwc = fmaf(a.kz * zs * rD * rD, fmaf(a.h2, rD, 1.02f), a.ke);
    const int jlo = max((int)ceilf(sig - hwc), -J);
    const int jhi = min((int)floorf(sig + hwc), nd - 1 - J);
    const float4 *bp = boxrow + J + jlo;
    const float4 *cp = cell + J + jlo;
    const float *yq = yrow + J + jlo;
    float d = sig - (float)jlo;
    float part = 0.f;
    for (int jl = jlo; jl <= jhi; ++jl) {
        const float4 A = __ldg(bp++);    // p, q/C, 1/C, C/2
        const float4 C = __ldg(cp++);    // ds/L, D_ps dtan/(2L), s_j dtan/(2L)
        const float yv = __ldg(yq++);
        const float x = fabsf(Dn * C.x * d);          // |s'|
        const float e = fmaf(Dn, C.y, yp * C.z);      // tau'/2 at the pixel depth
        const float w = window_diff(x, e, A.x, A.y, A.z, A.w);
        part = fmaf(yv * w, rcp_approx((A.x + A.w) * e), part);
        d -= 1.f;
    }
    return part;
}

__global__ void __launch_bounds__(256) bp_f32_kernel(GeomConsts g, const double *__restrict__ view_cs,
                                                     const float4 *__restrict__ box,
                                                     const float4 *__restrict__ cell,
                                                     const float *__restrict__ sino, float *__restrict__ img,
                                                     BpArgs a, const int *__restrict__ order, int ntx, int nsplit,
                                                     float *__restrict__ partial)
{
    __shared__ TileViewS<float> tv[BP_CHUNK];
    __shared__ int tj[BP_CHUNK];
    // 8 warps, each an 8 x 4 patch of the 16 x 16 tile: compact patches project onto few
    // cells, so a warp's loads of the cell tables touch few cache lines.
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tx = (warp & 1) * 8 + (lane & 7), ty = (warp >> 1) * 4 + (lane >> 3);
    const int tile = order[blockIdx.x];   // tiles with the most work first
    const int it = (tile % ntx) * BP_T, rt = (tile / ntx) * BP_T;
    // blockIdx.y: which part of the views this block gathers (the parts of a tile are summed
    // afterwards in a fixed order, so the result does not depend on scheduling)
    const long long b = blockIdx.z;
    const int vbeg = (int)((long long)g.nv * blockIdx.y / nsplit), vend = (int)((long long)g.nv * (blockIdx.y + 1) / nsplit);
    const int i = it + tx, r = rt + ty;
    const bool inside = i < g.nx && r < g.ny;
    const float *y = sino + b * (long long)g.nv * g.nd;
    const float ctr = 0.5f * (BP_T - 1);
    const float di = (float)tx - ctr, dr = (float)ty - ctr;
    float acc = 0.f;
    for (int v0 = vbeg; v0 < vend; v0 += BP_CHUNK) {
        const int nvc = min(BP_CHUNK, vend - v0);
        __syncthreads();
        if (tid < nvc) {
            double c = view_cs[2 * (v0 + tid)], s = view_cs[2 * (v0 + tid) + 1];
            double Dt, yt, a1, b1, rho, phi;
            int J;
            tile_view_double(g, c, s, it + (double)ctr, rt + (double)ctr, &Dt, &yt, &a1, &b1, &rho, &phi, &J);
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
                part += bp_view_f32(tv[vv], tj[vv], di, dr, a, g.nd, y + (long long)v * g.nd,
                                    box + (long long)v * g.nd, cell);
                if ((vv & 15) == 15) {   // blocked summation over groups of 16 views
                    acc += part;
                    part = 0.f;
                }
            }
            acc += part;
        }
    }
    if (inside) {
        if (nsplit == 1)
            img[(b * g.ny + r) * g.nx + i] = acc * a.h2q;
        else
            partial[((blockIdx.y * (long long)gridDim.z + b) * g.ny + r) * g.nx + i] = acc * a.h2q;
    }
}

// img = sum over the view parts, in part order
__global__ void bp_sum_parts_kernel(const float *__restrict__ partial, float *__restrict__ img, long long n, int nsplit)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        float s = partial[t];
        for (int k = 1; k < nsplit; ++k) s += partial[k * n + t];
        img[t] = s;
    }
}

// FP64: same tiling and window; every per-pair constant is recomputed in FP64 from the view
// and cell angles.
__global__ void __launch_bounds__(256) bp_f64_kernel(GeomConsts g, const double *__restrict__ view_cs,
                                                     const double *__restrict__ celld,
                                                     const double *__restrict__ sino, double *__restrict__ img,
                                                     double kz, double ke)
{
    constexpr int chunk = BP_CHUNK / 2;
    __shared__ TileViewS<double> tv[chunk];
    __shared__ int tj[chunk];
    __shared__ double tcs[chunk][2];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BP_T + tx;
    const int it = blockIdx.x * BP_T, rt = blockIdx.y * BP_T;
    const long long b = blockIdx.z;
    const int i = it + tx, r = rt + ty;
    const bool inside = i < g.nx && r < g.ny;
    const double *y = sino + b * (long long)g.nv * g.nd;
    const double ctr = 0.5 * (BP_T - 1);
    const double di = tx - ctr, dr = ty - ctr;
    double acc = 0.0;
    for (int v0 = 0; v0 < g.nv; v0 += chunk) {
        const int nvc = min(chunk, g.nv - v0);
        __syncthreads();
        if (tid < nvc) {
            double c = view_cs[2 * (v0 + tid)], s = view_cs[2 * (v0 + tid) + 1];
            TileViewS<double> T;
            int J;
            tile_view_double(g, c, s, it + ctr, rt + ctr, &T.Dt, &T.yt, &T.a1, &T.b1, &T.rho, &T.phi, &J);
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
            const double Dn = T.Dt - T.hc * di - T.hs * dr;
            const double yp = T.yt - T.hs * di + T.hc * dr;
            const double sig = T.phi + (T.rho + T.a1 * di + T.b1 * dr) / Dn;
            const double zs = fabs(yp * T.hc - Dn * T.hs) + fabs(yp * T.hs + Dn * T.hc);
            const double hwc = kz * zs / (Dn * Dn) * (1.02 + 2.0 * g.h / Dn) + ke;
            const int jlo = max((int)ceil(sig - hwc), -J);
            const int jhi = min((int)floor(sig + hwc), g.nd - 1 - J);
            double part = 0.0;
            for (int jl = jlo; jl <= jhi; ++jl) {
                const int j = J + jl;
                const double sj = celld[4 * j], L = celld[4 * j + 1], dt = celld[4 * j + 2];
                const double nxv = (sj * c - g.dps * s) / L, nyv = (sj * s + g.dps * c) / L;
                const double B = g.h * fmax(fabs(nxv), fabs(nyv)), C = g.h * fmin(fabs(nxv), fabs(nyv));
                const BoxConsts<double> bc = make_box_consts<double>(B, C, g.h);
                const double x = fabs(Dn * (g.ds / L) * (sig - jl));
                const double e = (g.dps * Dn + sj * yp) / L * 0.5 * dt;
                const double w = window_diff(x, e, bc.p, bc.q * bc.iC, bc.iC, 0.5 * C);
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
    if (dtype == CNSF_F32 && batch >= 2) return launch_back_batch(geo, (const float *)sino, (float *)img, batch, st);
    const GeomConsts &g = geo->gc;
    dim3 blk(BP_T, BP_T), grd((g.nx + BP_T - 1) / BP_T, (g.ny + BP_T - 1) / BP_T, batch);
    if (dtype == CNSF_F32) {
        BpArgs a{(float)geo->bw.kz, (float)geo->bw.ke, (float)(2.0 * g.h), (float)(0.25 * g.h * g.h)};
        // Enough blocks for several waves: split each tile's views when the tiles alone give
        // fewer than ~32 blocks per SM (partial images, then a fixed-order sum).
        int sms = 0, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const long long blocks = (long long)grd.x * grd.y * batch;
        int nsplit = 1;
        while (nsplit < 8 && blocks * nsplit < 32LL * std::max(sms, 1) && g.nv / (2 * nsplit) >= 32) nsplit *= 2;
        float *partial = nullptr;
        const long long nimg = (long long)batch * g.nx * g.ny;
        if (nsplit > 1) {
            cudaError_t e = cudaMallocAsync((void **)&partial, (size_t)nsplit * nimg * sizeof(float), st);
            if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? (record_cuda_error(e), CNSF_ERR_NOMEM) : record_cuda_error(e);
        }
        bp_f32_kernel<<<dim3(grd.x * grd.y, nsplit, grd.z), dim3(BP_T * BP_T), 0, st>>>(
            g, geo->d_view_cs, reinterpret_cast<const float4 *>(geo->d_box),
            reinterpret_cast<const float4 *>(geo->d_cellf), (const float *)sino, (float *)img, a, geo->d_bp_order,
            (int)grd.x, nsplit, partial);
        if (nsplit > 1) {
            bp_sum_parts_kernel<<<(unsigned)std::min<long long>((nimg + 255) / 256, 4096), 256, 0, st>>>(
                partial, (float *)img, nimg, nsplit);
            cudaFreeAsync(partial, st);
        }
    } else {
        bp_f64_kernel<<<grd, blk, 0, st>>>(g, geo->d_view_cs, geo->d_cell_d, (const double *)sino, (double *)img,
                                           geo->bw.kz, geo->bw.ke);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? CNSF_OK : record_cuda_error(e);
}

}  // namespace cnsf
