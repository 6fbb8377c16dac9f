// back.cu -- back projection c = A^T y with the entries of Eq. (18).
//
// Pixel-driven gather, no atomics.  A block owns a 16 x 16 pixel tile; for each view the
// pixel centre is projected onto the detector (perspective division, Eq. 4) and the cells
// its footprint reaches are gathered.  The projection of the tile's reference point (the
// centre of the tile's part inside the image) is computed once per view in FP64
// (tile_view_double) and split into an integer cell index plus a small remainder, so that
// FP32 carries the sub-cell position of every pixel to ~1e-6 cells;
// the per-pixel work is then a handful of FP32 FMAs and one reciprocal.  The cell window
// is bounded per pixel from the footprint widths of the ray through the pixel centre
// (BpWindow), so few cells outside the support are visited.  In FP32 a thread owns a 2 x 2
// pixel quad and gathers it as two pixel pairs, each pair sharing its cell-table loads.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "cnsf_internal.cuh"
#include "cnsf_runtime.h"
#include "footprint.cuh"

namespace cnsf {

constexpr int BP_T = 16;        // tile side (pixels)
constexpr int BP_CHUNK = 256;   // views whose tile coefficients are staged at once
constexpr int BP_QUAD_THREADS = BP_T * BP_T / 4;   // FP32 kernel: one thread per 2 x 2 pixel quad

template <typename T>
struct alignas(16) TileViewS {
    T Dt, yt, a1, b1, rho, phi, hc, hs;
};

struct BpArgs {
    float kz, ke, h2;   // window constants; h2 = 2h
    float h2sq;         // 2 h^2
    float h2q;          // h^2 / 4
    float kscale;       // arc detector: cells per radian, D_ps / ds
    float dg;           // arc detector: radians per cell, ds / D_ps
    float nk6;          // arc detector: -dg^2 / 6 (sine series)
    long long box_odd;  // offsets (floats) of the odd-aligned pair tables: 8 nv ceil(n_det/2)
    int cell_odd;       // and 8 ceil(n_det/2)
    float s0, ds;       // centre of cell 0 and cell pitch (mm)
    float idps;         // 1/D_ps (0 for parallel rays)
    float ked;          // arc detector: tau'/2 per unit G (dtan / (2 dg))
    float nk2;          // arc detector: -dg^2 / 2 (cosine series)
};

// The FP32 per-(tile, view) coefficients from the FP64 projection of the tile's reference point.
__device__ __forceinline__ void tile_view_f32(const GeomConsts &g, double c, double s, double it, double rt,
                                              TileViewS<float> &T, int &J)
{
    double Dt, yt, a1, b1, rho, phi, hc, hs;
    tile_view_double(g, c, s, it, rt, &Dt, &yt, &a1, &b1, &rho, &phi, &J, &hc, &hs);
    T.Dt = (float)Dt; T.yt = (float)yt; T.a1 = (float)a1; T.b1 = (float)b1;
    T.rho = (float)rho; T.phi = (float)phi; T.hc = (float)hc; T.hs = (float)hs;
}

// Reference point of a tile's coefficients, as offsets from its first pixel: the centre of
// the part of the tile that lies in the image.  A tile that overhangs the image edge keeps
// its reference on image pixels, in front of the source (validated for the image only).
__host__ __device__ inline double tile_ref(int t0, int n) { return 0.5 * ((n - t0 < BP_T ? n - t0 : BP_T) - 1); }

// Geometry-time table of those coefficients for every (tile, view): two float4 and J.
__global__ void tile_view_table_kernel(GeomConsts g, const double *__restrict__ view_cs, int ntx, int ntiles,
                                       float4 *__restrict__ tab, int *__restrict__ jtab)
{
    const long long n = (long long)ntiles * g.nv;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int tile = (int)(t / g.nv), v = (int)(t - (long long)tile * g.nv);
        const int it = (tile % ntx) * BP_T, rt = (tile / ntx) * BP_T;
        TileViewS<float> T;
        int J;
        tile_view_f32(g, view_cs[2 * v], view_cs[2 * v + 1], it + tile_ref(it, g.nx), rt + tile_ref(rt, g.ny), T, J);
        tab[2 * t] = make_float4(T.Dt, T.yt, T.a1, T.b1);
        tab[2 * t + 1] = make_float4(T.rho, T.phi, T.hc, T.hs);
        jtab[t] = J;
    }
}

int build_tile_view_table(cnsf_geometry *geo)
{
    const GeomConsts &g = geo->gc;
    const int ntx = (g.nx + BP_T - 1) / BP_T, nty = (g.ny + BP_T - 1) / BP_T;
    const long long n = (long long)ntx * nty * g.nv;
    if (n * 36 > (1LL << 30)) return CNSF_OK;   // larger geometries compute it in the kernel
    cudaError_t e = cudaMalloc((void **)&geo->d_tv, (size_t)n * 2 * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc((void **)&geo->d_tj, (size_t)n * sizeof(int));
    if (e != cudaSuccess) {
        if (geo->d_tv) cudaFree(geo->d_tv);
        geo->d_tv = nullptr;
        geo->d_tj = nullptr;
        return e == cudaErrorMemoryAllocation ? (record_cuda_error(e), CNSF_ERR_NOMEM) : record_cuda_error(e);
    }
    geo->device_bytes += (size_t)n * (2 * sizeof(float4) + sizeof(int));
    tile_view_table_kernel<<<(unsigned)std::min<long long>((n + 255) / 256, 8192), 256>>>(g, geo->d_view_cs, ntx,
                                                                                          ntx * nty, geo->d_tv,
                                                                                          geo->d_tj);
    e = cudaDeviceSynchronize();
    return e == cudaSuccess ? CNSF_OK : record_cuda_error(e);
}

// Per-(pixel, view) set-up of the gather from the pixel's depth D_n, detector coordinate y'
// and the numerator of its cell coordinate (affine in the pixel offset, so a neighbour's
// values are one addition away): the cell coordinate sigma (minus J) and, for the arc
// detector, the sine-series factor G.  Flat or parallel detector: sigma is the ratio of
// two affine functions of the pixel offset (perspective division, Eq. 4).  Arc detector:
// the angle from the ray through the tile's reference point, atan of
// (y' Dt - yt D_n)/(D_n Dt + y' yt) (a numerator without constant term), in cells.
struct BpPixel {
    float Dn, yp, sig, G, iDn;   // iDn = 1/D_n (flat, parallel), reused by the blur factors
};

template <bool ARC>
__device__ __forceinline__ BpPixel bp_pixel_f32(const TileViewS<float> &T, float Dn, float yp, float num,
                                                const BpArgs &a)
{
    BpPixel P;
    P.Dn = Dn;
    P.yp = yp;
    P.iDn = ARC ? 0.f : rcp_approx(Dn);
    P.sig = ARC ? fmaf(atan_small(num * rcp_approx(fmaf(Dn, T.Dt, yp * T.yt))), a.kscale, T.phi)
                : fmaf(num, P.iDn, T.phi);
    P.G = ARC ? sqrtf(fmaf(Dn, Dn, yp * yp)) * a.dg : 0.f;
    return P;
}

// Half-width (cells) of a cell window that holds the footprint of every pixel of a 2 x 2
// quad, from pixel 0's depth D_n and detector coordinate y'.  For one pixel the window is
// kz zs / D_n^2 (1.02 + 2h / D_n) + ke with zs = |y' hc - D_n hs| + |y' hs + D_n hc| (the
// footprint widths of the ray through its centre, with margin for the perspective across
// the pixel); it grows with zs and 1/D_n.  A step along a row changes the second term of zs
// by -h^2 and leaves the first; a step down a column changes the first by h^2 and leaves the
// second: over the quad zs is at most zs_0 + 2h^2, and D_n at least D_n,0 - max(hc, 0) -
// max(hs, 0).
__device__ __forceinline__ float bp_quad_hwc(const TileViewS<float> &T, float Dn0, float yp0, const BpArgs &a)
{
    const float za = fmaf(yp0, T.hc, -Dn0 * T.hs), zb = fmaf(yp0, T.hs, Dn0 * T.hc);
    const float zs = fabsf(za) + fabsf(zb) + a.h2sq;
    const float rD = rcp_approx(Dn0 - fmaxf(T.hc, 0.f) - fmaxf(T.hs, 0.f));
    return fmaf(a.kz * zs * rD * rD, fmaf(a.h2, rD, 1.02f), a.ke);
}

// The two entries of one cell pair (cells 2m + o, 2m + o + 1 of the tables of parity o)
// for one pixel in packed FP32x2 arithmetic, without the factor 2/B of the normalisation
// h^2/(2B) (the sinogram pairs carry it) and without h^2/4 (applied to the sum): the
// window difference divided by tau'.  d holds the two cells' offsets from the pixel's
// projection, in cells.  Arc detector: |s'| = R sin(dg d), R the pixel's
// distance from the source; with dg d below ~0.05 rad, R dg d (1 - (dg d)^2/6) is that sine
// to ~1e-9 relative (the next term of the series).
template <bool ARC, bool EXACT>
__device__ __forceinline__ float2 bp_pair_f32(const BpPixel &P, float2 d, const float (&A)[8], const float (&C)[8],
                                              float nk6)
{
    const float2 ne1 = make_float2(-1.f, -1.f);
    float2 xs;
    if (ARC)
        xs = __fmul2_rn(__fmul2_rn(make_float2(P.G, P.G), d),
                        __ffma2_rn(__fmul2_rn(d, d), make_float2(nk6, nk6), make_float2(1.f, 1.f)));
    else
        xs = __fmul2_rn(__fmul2_rn(make_float2(P.Dn, P.Dn), make_float2(C[0], C[1])), d);
    const float2 x = make_float2(fabsf(xs.x), fabsf(xs.y));                                 // |s'|
    const float2 e = __ffma2_rn(make_float2(P.Dn, P.Dn), make_float2(C[2], C[3]),
                                __fmul2_rn(make_float2(P.yp, P.yp), make_float2(C[4], C[5])));
    const float2 w = wdiff2p<EXACT>(x, e, ne1, make_float2(A[0], A[1]), make_float2(A[2], A[3]),
                                   make_float2(A[4], A[5]), make_float2(A[6], A[7]));
    return __fmul2_rn(w, make_float2(rcp_approx(e.x), rcp_approx(e.y)));
}

// One view of the gather for two pixels a and b of a thread, over the union [g0, g1] of
// their cell windows [sigma - hwc, sigma + hwc] (hwc bounding both pixels' half-widths)
// clipped to the detector, two cells per step.  The steps start at g0 whatever its parity
// (pair tables and sinogram pairs exist in both alignments), so a window of L cells takes
// ceil(L/2) steps.  Each cell pair's constants and sinogram values are loaded once and serve
// both pixels (the L1 path carries every loaded byte to each lane, so sharing the loads
// halves that traffic).  A cell of the union outside one pixel's own window, or the cell
// past g1 of an odd-length window, lies outside that pixel's support (the window bounds the
// support with margin), so its entry for that pixel is exactly 0; a cell past n_det has
// sinogram value 0.  Returns the two pixels' sums.
template <bool ARC, bool EXACT>
__device__ __forceinline__ float2 bp_view2_f32(const BpPixel &Pa, const BpPixel &Pb, float hwc, int J, const BpArgs &a,
                                               int nd, const float2 *__restrict__ y2row,
                                               const float2 *__restrict__ y2orow, const float *__restrict__ boxrow,
                                               const float *__restrict__ cell2)
{
    const float lo = fminf(Pa.sig, Pb.sig) - hwc, hi = fmaxf(Pa.sig, Pb.sig) + hwc;
    const int g0 = J + max((int)ceilf(lo), -J), g1 = J + min((int)floorf(hi), nd - 1 - J);
    const int odd = g0 & 1;
    const int m0 = g0 >> 1, m1 = (g1 - odd) >> 1;   // m0 > m1 when the window misses the detector
    if (odd) {   // pairs (2m + 1, 2m + 2)
        boxrow += a.box_odd;
        cell2 += a.cell_odd;
        y2row = y2orow;
    }
    const float off = (float)(2 * m0 + odd - J);
    float2 da = make_float2(Pa.sig - off, Pa.sig - off - 1.f), db = make_float2(Pb.sig - off, Pb.sig - off - 1.f);
    const float2 m2 = make_float2(-2.f, -2.f);
    float2 acca = make_float2(0.f, 0.f), accb = make_float2(0.f, 0.f);
    for (int m = m0; m <= m1; ++m) {
        float A[8], C[8];
        ldg256(boxrow + 8 * m, A);    // q | p/C | 1/C | -C/2, pairs
        ldg256(cell2 + 8 * m, C);     // ds/L | c1 | c2, pairs
        const float2 yb = __ldg(y2row + m);                                                  // y 2/B
        acca = __ffma2_rn(yb, bp_pair_f32<ARC, EXACT>(Pa, da, A, C, a.nk6), acca);
        accb = __ffma2_rn(yb, bp_pair_f32<ARC, EXACT>(Pb, db, A, C, a.nk6), accb);
        da = __fadd2_rn(da, m2);
        db = __fadd2_rn(db, m2);
    }
    return make_float2(acca.x + acca.y, accb.x + accb.y);
}

// FP32 back projection with a 2 x 2 pixel quad per thread (64 threads per 16 x 16 tile, a
// warp covering 16 x 8 pixels), views in chunks of BP_CHUNK whose tile coefficients are
// staged in shared memory.  For each (tile, view) the quad is gathered as two pixel pairs
// along the image axis whose unit step moves the projection least (columns when
// |d sigma/d row| <= |d sigma/d column|), so the two pixels of a pair reach nearly the same
// cells and their union window adds little.
template <bool ARC, bool EXACT>
__global__ void __launch_bounds__(BP_QUAD_THREADS, 10) bp_f32_kernel(GeomConsts g, const double *__restrict__ view_cs,
                                                                 const float *__restrict__ box2,
                                                                 const float *__restrict__ cell2,
                                                                 const float2 *__restrict__ y2,
                                                                 const float2 *__restrict__ y2o,
                                                                 float *__restrict__ img, BpArgs a,
                                                                 const int *__restrict__ order, int ntx, int nsplit,
                                                                 float *__restrict__ partial,
                                                                 const float4 *__restrict__ tvtab,
                                                                 const int *__restrict__ tjtab)
{
    __shared__ TileViewS<float> tv[BP_CHUNK];
    __shared__ int tj[BP_CHUNK];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // lanes 4k .. 4k + 3 take a 2 x 2 block of quads: their cell windows lie close, so a
    // warp's loads touch fewer 128-byte lines per group of four lanes
    const int tx = 2 * ((lane & 1) | ((lane >> 1) & 6)), ty = 8 * warp + 2 * (((lane >> 1) & 1) | ((lane >> 3) & 2));
    const int tile = order[blockIdx.x];   // tiles with the most work first
    const int it = (tile % ntx) * BP_T, rt = (tile / ntx) * BP_T;
    const long long b = blockIdx.z;
    const int vbeg = (int)((long long)g.nv * blockIdx.y / nsplit), vend = (int)((long long)g.nv * (blockIdx.y + 1) / nsplit);
    const int i = it + tx, r = rt + ty;
    // quad pixels: 0 (i, r), 1 (i + 1, r), 2 (i, r + 1), 3 (i + 1, r + 1)
    const bool in0 = i < g.nx && r < g.ny, in1 = i + 1 < g.nx && r < g.ny;
    const bool in2 = i < g.nx && r + 1 < g.ny, in3 = i + 1 < g.nx && r + 1 < g.ny;
    const int ndh = (g.nd + 1) >> 1;
    const float2 *y = y2 + b * (long long)g.nv * ndh, *yo = y2o + b * (long long)g.nv * ndh;
    const double refx = tile_ref(it, g.nx), refy = tile_ref(rt, g.ny);
    const float di = (float)(tx - refx), dr = (float)(ty - refy);
    float part[4] = {0.f, 0.f, 0.f, 0.f}, acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int v0 = vbeg; v0 < vend; v0 += BP_CHUNK) {
        const int nvc = min(BP_CHUNK, vend - v0);
        __syncthreads();
        for (int k = tid; k < nvc; k += BP_QUAD_THREADS) {
            if (tvtab) {   // precomputed with the geometry
                const long long t = (long long)tile * g.nv + v0 + k;
                const float4 u0 = __ldg(tvtab + 2 * t), u1 = __ldg(tvtab + 2 * t + 1);
                TileViewS<float> T;
                T.Dt = u0.x; T.yt = u0.y; T.a1 = u0.z; T.b1 = u0.w; T.rho = u1.x; T.phi = u1.y; T.hc = u1.z; T.hs = u1.w;
                tv[k] = T;
                tj[k] = __ldg(tjtab + t);
            } else {
                tile_view_f32(g, view_cs[2 * (v0 + k)], view_cs[2 * (v0 + k) + 1], it + refx, rt + refy, tv[k],
                              tj[k]);
            }
        }
        __syncthreads();
        if (in0) {
            for (int vv = 0; vv < nvc; ++vv) {
                const int v = v0 + vv;
                const TileViewS<float> T = tv[vv];
                const int J = tj[vv];
                const bool col = fabsf(T.b1) <= fabsf(T.a1);   // pairs along a column
                const float2 *yrow = y + (long long)v * ndh;
                const float *brow = box2 + 8 * (long long)v * ndh;
                // pixel 0, then its neighbours by the per-pixel steps of D_n, y' and the
                // numerator: down a column (-hs, hc, b1), along a row (-hc, -hs, a1)
                const float Dn0 = fmaf(-T.hc, di, fmaf(-T.hs, dr, T.Dt));
                const float yp0 = fmaf(-T.hs, di, fmaf(T.hc, dr, T.yt));
                const float nu0 = ARC ? fmaf(T.a1, di, T.b1 * dr) : fmaf(T.a1, di, fmaf(T.b1, dr, T.rho));
                const float sDn = col ? -T.hs : -T.hc, syp = col ? T.hc : -T.hs, snu = col ? T.b1 : T.a1;   // pair step
                const float oDn = col ? -T.hc : -T.hs, oyp = col ? -T.hs : T.hc, onu = col ? T.a1 : T.b1;   // other step
                const BpPixel P0 = bp_pixel_f32<ARC>(T, Dn0, yp0, nu0, a);
                BpPixel P1 = bp_pixel_f32<ARC>(T, Dn0 + sDn, yp0 + syp, nu0 + snu, a);
                BpPixel P2 = bp_pixel_f32<ARC>(T, Dn0 + oDn, yp0 + oyp, nu0 + onu, a);
                BpPixel P3 = bp_pixel_f32<ARC>(T, Dn0 + oDn + sDn, yp0 + oyp + syp, nu0 + onu + snu, a);
                // a pixel outside the image takes pixel 0's window (its sums are not stored)
                const bool inP1 = col ? in2 : in1, inP2 = col ? in1 : in2;
                if (!inP1) P1.sig = P0.sig;
                if (!inP2) P2.sig = P0.sig;
                if (!in3) P3.sig = P0.sig;
                const float hwc = bp_quad_hwc(T, Dn0, yp0, a);
                const float2 *yorow = yo + (long long)v * ndh;
                const float2 s1 = bp_view2_f32<ARC, EXACT>(P0, P1, hwc, J, a, g.nd, yrow, yorow, brow, cell2);
                const float2 s2 = bp_view2_f32<ARC, EXACT>(P2, P3, hwc, J, a, g.nd, yrow, yorow, brow, cell2);
                part[0] += s1.x;
                part[1] += col ? s2.x : s1.y;
                part[2] += col ? s1.y : s2.x;
                part[3] += s2.y;
                if ((vv & 15) == 15) {   // blocked summation over groups of 16 views
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        acc[q] += part[q];
                        part[q] = 0.f;
                    }
                }
            }
        }
    }
    if (in0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int iq = i + (q & 1), rq = r + (q >> 1);
            if (iq >= g.nx || rq >= g.ny) continue;
            const float val = (acc[q] + part[q]) * a.h2q;
            if (nsplit == 1)
                img[(b * g.ny + rq) * g.nx + iq] = val;
            else
                partial[((blockIdx.y * (long long)gridDim.z + b) * g.ny + rq) * g.nx + iq] = val;
        }
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

// ------------------------------------------------------------------ four rotations
// With the quarter-turn symmetry of fp_rot4_f32_kernel, a(v + kV/4, j, n) = a(v, j, R^-k n)
// (R the quarter turn of the pixel lattice, (i, r) -> (N-1-r, i)), so
//     (A^T y)[n] = sum_k T_k(R^-k n),   T_k(p) = sum_{v < V/4} sum_j y[v + kV/4][j] a(v, j, p).
// Every pixel p gathers T_0 .. T_3 over the first quarter of the views: each entry a(v, j, p)
// is evaluated once and weighs the four sinogram values y[v + kV/4][j], which a per-call table
// holds together (one 32-byte entry per cell pair and view).  The orbit sum then adds
// T_k(R^-k n) over k for every pixel n.

// Y4[o][v][m] holds, for k = 0..3, the pair (w y[v + kV/4][2m + o], w' y[v + kV/4][2m + o + 1])
// with w = 2/B of (v, cell) (the same for the four views: a quarter turn swaps the two widths
// of Eq. 16), 0 past n_det; v < V/4.
__global__ void sino_pairs_rot4_kernel(const float *__restrict__ y, const BoxF *__restrict__ box,
                                       float4 *__restrict__ y4, int nv, int nd)
{
    const int ndh = (nd + 1) >> 1, nv4 = nv >> 2;
    const long long n = 2LL * nv4 * ndh;
    y += (long long)blockIdx.y * nv * nd;   // image y of a batch
    y4 += 2 * n * blockIdx.y;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int o = (int)(t / ((long long)nv4 * ndh));
        const long long rem = t - (long long)o * nv4 * ndh;
        const int v = (int)(rem / ndh), m = (int)(rem - (long long)v * ndh);
        const int j = 2 * m + o;
        const BoxF *br = box + (long long)v * nd;
        float out[8];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float *yr = y + (long long)(v + k * nv4) * nd;
            out[2 * k] = j < nd ? yr[j] / (br[j].q - br[j].hC) : 0.f;
            out[2 * k + 1] = j + 1 < nd ? yr[j + 1] / (br[j + 1].q - br[j + 1].hC) : 0.f;
        }
        y4[2 * t] = make_float4(out[0], out[1], out[2], out[3]);
        y4[2 * t + 1] = make_float4(out[4], out[5], out[6], out[7]);
    }
}

// The per-(quad, view) set-up shared by the four-rotation kernels and their span table:
// pixel 0 from the tile coefficients and its neighbours by the per-pixel steps of D_n, y'
// and the numerator (down a column (-hs, hc, b1), along a row (-hc, -hs, a1)); P1 is the
// neighbour along the axis that moves the projection least (col: down the column), P2 the
// other one, P3 both; a pixel outside the image takes pixel 0's window.
struct QuadView {
    BpPixel P0, P1, P2, P3;
    float hwc;
    bool col;
};

template <bool ARC>
__device__ __forceinline__ QuadView quad_view_setup(const TileViewS<float> &T, float di, float dr, bool in1, bool in2,
                                                    bool in3, const BpArgs &a)
{
    QuadView Q;
    Q.col = fabsf(T.b1) <= fabsf(T.a1);   // pairs along a column
    const bool col = Q.col;
    const float Dn0 = fmaf(-T.hc, di, fmaf(-T.hs, dr, T.Dt));
    const float yp0 = fmaf(-T.hs, di, fmaf(T.hc, dr, T.yt));
    const float nu0 = ARC ? fmaf(T.a1, di, T.b1 * dr) : fmaf(T.a1, di, fmaf(T.b1, dr, T.rho));
    const float sDn = col ? -T.hs : -T.hc, syp = col ? T.hc : -T.hs, snu = col ? T.b1 : T.a1;   // pair step
    const float oDn = col ? -T.hc : -T.hs, oyp = col ? -T.hs : T.hc, onu = col ? T.a1 : T.b1;   // other step
    Q.P0 = bp_pixel_f32<ARC>(T, Dn0, yp0, nu0, a);
    Q.P1 = bp_pixel_f32<ARC>(T, Dn0 + sDn, yp0 + syp, nu0 + snu, a);
    Q.P2 = bp_pixel_f32<ARC>(T, Dn0 + oDn, yp0 + oyp, nu0 + onu, a);
    Q.P3 = bp_pixel_f32<ARC>(T, Dn0 + oDn + sDn, yp0 + oyp + syp, nu0 + onu + snu, a);
    const bool inP1 = col ? in2 : in1, inP2 = col ? in1 : in2;
    if (!inP1) Q.P1.sig = Q.P0.sig;
    if (!inP2) Q.P2.sig = Q.P0.sig;
    if (!in3) Q.P3.sig = Q.P0.sig;
    Q.hwc = bp_quad_hwc(T, Dn0, yp0, a);
    return Q;
}

// Absolute cells [g0, g1] of the union of two pixels' windows, clipped to the detector
// (g0 > g1 when the window misses it).
__device__ __forceinline__ void pair_window(const BpPixel &Pa, const BpPixel &Pb, float hwc, int J, int nd, int &g0,
                                            int &g1)
{
    const float lo = fminf(Pa.sig, Pb.sig) - hwc, hi = fmaxf(Pa.sig, Pb.sig) + hwc;
    g0 = J + max((int)ceilf(lo), -J);
    g1 = J + min((int)floorf(hi), nd - 1 - J);
}

// Per-pixel factors of the quarter-turn gather's merged pair table.  The blur of cell j at a
// pixel of depth D_n and detector-axis coordinate y' is tau'_j/2 = D_n c1_j + y' c2_j with
// c2_j = c1_j s_j / D_ps (flat detector, s_j = s_sigma - d ds for the cell d cells below the
// pixel's projection s_sigma), so tau'_j/2 = c1_j (K - d L), K = D_n + y' s_sigma / D_ps,
// L = y' ds / D_ps; parallel rays: K = 1, L = 0 (c1 = tau/2).  The flat and parallel gathers
// carry d' = D_n d (s' = (ds/L_j) d') and L' = L / D_n.  Arc detector: tau'_j/2 =
// (dtan/2) R cos(dg d), R the pixel's distance from the source, by its two-term series
// E (1 - (dg d)^2 / 2), E = (dtan/2) R (the next term is below 1e-9 relative for dg d < 0.05).
struct BpPixel4 {
    BpPixel P;
    float K, L;   // flat, parallel: K and L'; arc: E and unused
};

template <bool ARC>
__device__ __forceinline__ BpPixel4 bp_pixel4(const BpPixel &P, int J, const BpArgs &a)
{
    BpPixel4 Q;
    Q.P = P;
    if (ARC) {
        Q.K = P.G * a.ked;
        Q.L = 0.f;
    } else {
        const float ssig = fmaf((float)J + P.sig, a.ds, a.s0);
        Q.K = fmaf(P.yp * ssig, a.idps, P.Dn);
        Q.L = P.yp * a.ds * a.idps * P.iDn;
    }
    return Q;
}

// The two entries of one cell pair for one pixel from the merged entry A (pairs), all in
// units of the cell's C (the narrower trapezoid width of Eq. 16, clamped away from 0 as
// 1/C is): q/C | p/C | ds/(L C) | c1/C, arc detector q/C | p/C | 1/C | unused.  In these
// units the window difference of footprint.cuh takes 1/C = 1 and -C/2 = -1/2, and the
// entry, a ratio of the difference to the half blur, is unchanged; d: flat and parallel
// d' = D_n d, arc d (cells).  Without 2/B and h^2/4, as bp_pair_f32.
template <bool ARC, bool EXACT>
__device__ __forceinline__ float2 bp_pair_rot4(const BpPixel4 &Q, float2 d, const float (&A)[8], const BpArgs &a)
{
    const float2 ne1 = make_float2(-1.f, -1.f);
    float2 xs, e;
    if (ARC) {
        const float2 d2 = __fmul2_rn(d, d), iC = make_float2(A[4], A[5]);
        xs = __fmul2_rn(__fmul2_rn(make_float2(Q.P.G, Q.P.G), d),
                        __ffma2_rn(d2, make_float2(a.nk6, a.nk6), make_float2(1.f, 1.f)));
        e = __fmul2_rn(make_float2(Q.K, Q.K), __ffma2_rn(d2, make_float2(a.nk2, a.nk2), make_float2(1.f, 1.f)));
        xs = __fmul2_rn(xs, iC);
        e = __fmul2_rn(e, iC);
    } else {
        xs = __fmul2_rn(make_float2(A[4], A[5]), d);
        e = __fmul2_rn(make_float2(A[6], A[7]), __ffma2_rn(d, make_float2(-Q.L, -Q.L), make_float2(Q.K, Q.K)));
    }
    const float2 x = make_float2(fabsf(xs.x), fabsf(xs.y));   // |s'| / C
    const float2 w = wdiff2p<EXACT>(x, e, ne1, make_float2(A[0], A[1]), make_float2(A[2], A[3]),
                                    make_float2(1.f, 1.f), make_float2(-0.5f, -0.5f));
    return __fmul2_rn(w, make_float2(rcp_approx(e.x), rcp_approx(e.y)));
}

// bp_view2_f32 for the four rotations: the same window and cell pairs, the pair's constants
// in one merged 32-byte entry (ac) and its four rotations' weighted sinogram values in
// another (y4); each pair's entries for pixels a and b are applied to the four rotations
// and added to ta[k], tb[k] (lanes: the two cells of the pair).
template <bool ARC, bool EXACT>
__device__ __forceinline__ void bp_view2_rot4(const BpPixel4 &Qa, const BpPixel4 &Qb, float hwc, int J,
                                              const BpArgs &a, int nd, const float *__restrict__ y4row,
                                              const float *__restrict__ y4orow, const float *__restrict__ acrow,
                                              long long ac_odd, float2 (&ta)[4], float2 (&tb)[4])
{
    int g0, g1;
    pair_window(Qa.P, Qb.P, hwc, J, nd, g0, g1);
    const int odd = g0 & 1;
    const int m0 = g0 >> 1, m1 = (g1 - odd) >> 1;   // m0 > m1 when the window misses the detector
    if (odd) {   // pairs (2m + 1, 2m + 2)
        acrow += ac_odd;
        y4row = y4orow;
    }
    const float off = (float)(2 * m0 + odd - J);
    // cell offsets of the two pixels; flat and parallel carry D_n d
    const float sa = ARC ? 1.f : Qa.P.Dn, sb = ARC ? 1.f : Qb.P.Dn;
    float2 da = make_float2(sa * (Qa.P.sig - off), sa * (Qa.P.sig - off - 1.f));
    float2 db = make_float2(sb * (Qb.P.sig - off), sb * (Qb.P.sig - off - 1.f));
    const float2 sta = make_float2(-2.f * sa, -2.f * sa), stb = make_float2(-2.f * sb, -2.f * sb);
    for (int m = m0; m <= m1; ++m) {
        float A[8], Y[8];
        ldg256(acrow + 8 * m, A);     // q/C | p/C | ds/(L C) | c1/C, pairs
        ldg256(y4row + 8 * m, Y);     // y 2/B of the four rotations, pairs
        const float2 wa = bp_pair_rot4<ARC, EXACT>(Qa, da, A, a);
        const float2 wb = bp_pair_rot4<ARC, EXACT>(Qb, db, A, a);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 yk = make_float2(Y[2 * k], Y[2 * k + 1]);
            ta[k] = __ffma2_rn(yk, wa, ta[k]);
            tb[k] = __ffma2_rn(yk, wb, tb[k]);
        }
        da = __fadd2_rn(da, sta);
        db = __fadd2_rn(db, stb);
    }
}

// bp_f32_kernel over the first quarter of the views with four accumulators per pixel: the
// partial images T_k (view part s: partial[(4 s + k)][N][N]).  The quad's pixel pairs are
// gathered along the axis that moves the projection least, the two pairings in two
// branches (uniform over the block) so that every accumulator keeps its register.
template <bool ARC, bool EXACT, bool BATCH>
__global__ void __launch_bounds__(BP_QUAD_THREADS, 8) bp_rot4_f32_kernel(GeomConsts g, const float *__restrict__ ac,
                                                                     const float *__restrict__ y4, BpArgs a,
                                                                     const int *__restrict__ order, int ntx, int nsplit,
                                                                     float *__restrict__ partial,
                                                                     const double *__restrict__ view_cs,
                                                                     const float4 *__restrict__ tvtab,
                                                                     const int *__restrict__ tjtab)
{
    __shared__ TileViewS<float> tv[BP_CHUNK];
    __shared__ int tj[BP_CHUNK];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // lanes 4k .. 4k + 3 take a 2 x 2 block of quads: their cell windows lie close, so a
    // warp's loads touch fewer 128-byte lines per group of four lanes
    const int tx = 2 * ((lane & 1) | ((lane >> 1) & 6)), ty = 8 * warp + 2 * (((lane >> 1) & 1) | ((lane >> 3) & 2));
    const int tile = order[blockIdx.x];   // tiles with the most work first
    const int it = (tile % ntx) * BP_T, rt = (tile / ntx) * BP_T;
    const int nv4 = g.nv >> 2;
    const int vbeg = (int)((long long)nv4 * blockIdx.y / nsplit), vend = (int)((long long)nv4 * (blockIdx.y + 1) / nsplit);
    if (BATCH) {   // image z of a batch (the single-image instantiation has no offsets)
        y4 += 16LL * blockIdx.z * nv4 * ((g.nd + 1) >> 1);
        partial += 4LL * blockIdx.z * nsplit * g.nx * g.ny;
    }
    const int i = it + tx, r = rt + ty;
    const bool in0 = i < g.nx && r < g.ny, in1 = i + 1 < g.nx && r < g.ny;
    const bool in2 = i < g.nx && r + 1 < g.ny, in3 = i + 1 < g.nx && r + 1 < g.ny;
    const int ndh = (g.nd + 1) >> 1;
    const double refx = tile_ref(it, g.nx), refy = tile_ref(rt, g.ny);
    const float di = (float)(tx - refx), dr = (float)(ty - refy);
    float2 t[4][4];   // [quad pixel][rotation]
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int k = 0; k < 4; ++k) t[q][k] = make_float2(0.f, 0.f);
    for (int v0 = vbeg; v0 < vend; v0 += BP_CHUNK) {
        const int nvc = min(BP_CHUNK, vend - v0);
        __syncthreads();
        for (int k = tid; k < nvc; k += BP_QUAD_THREADS) {
            if (tvtab) {   // precomputed with the geometry
                const long long tt = (long long)tile * g.nv + v0 + k;
                const float4 u0 = __ldg(tvtab + 2 * tt), u1 = __ldg(tvtab + 2 * tt + 1);
                TileViewS<float> T;
                T.Dt = u0.x; T.yt = u0.y; T.a1 = u0.z; T.b1 = u0.w; T.rho = u1.x; T.phi = u1.y; T.hc = u1.z; T.hs = u1.w;
                tv[k] = T;
                tj[k] = __ldg(tjtab + tt);
            } else {
                tile_view_f32(g, view_cs[2 * (v0 + k)], view_cs[2 * (v0 + k) + 1], it + refx, rt + refy, tv[k],
                              tj[k]);
            }
        }
        __syncthreads();
        if (!in0) continue;
        for (int vv = 0; vv < nvc; ++vv) {
            const int v = v0 + vv;
            const TileViewS<float> T = tv[vv];
            const int J = tj[vv];
            const float *arow = ac + 8 * (long long)v * ndh;
            const float *yrow = y4 + 8 * (long long)v * ndh, *yorow = y4 + 8 * (long long)(nv4 + v) * ndh;
            const long long ac_odd = 8LL * nv4 * ndh;
            const QuadView Q = quad_view_setup<ARC>(T, di, dr, in1, in2, in3, a);
            const BpPixel4 P0 = bp_pixel4<ARC>(Q.P0, J, a), P1 = bp_pixel4<ARC>(Q.P1, J, a);
            const BpPixel4 P2 = bp_pixel4<ARC>(Q.P2, J, a), P3 = bp_pixel4<ARC>(Q.P3, J, a);
            if (Q.col) {   // P1 is quad pixel 2, P2 quad pixel 1
                bp_view2_rot4<ARC, EXACT>(P0, P1, Q.hwc, J, a, g.nd, yrow, yorow, arow, ac_odd, t[0], t[2]);
                bp_view2_rot4<ARC, EXACT>(P2, P3, Q.hwc, J, a, g.nd, yrow, yorow, arow, ac_odd, t[1], t[3]);
            } else {
                bp_view2_rot4<ARC, EXACT>(P0, P1, Q.hwc, J, a, g.nd, yrow, yorow, arow, ac_odd, t[0], t[1]);
                bp_view2_rot4<ARC, EXACT>(P2, P3, Q.hwc, J, a, g.nd, yrow, yorow, arow, ac_odd, t[2], t[3]);
            }
        }
    }
    if (in0) {
        const long long nn = (long long)g.nx * g.ny;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int iq = i + (q & 1), rq = r + (q >> 1);
            if (iq >= g.nx || rq >= g.ny) continue;
#pragma unroll
            for (int k = 0; k < 4; ++k)
                partial[(4LL * blockIdx.y + k) * nn + (long long)rq * g.nx + iq] = (t[q][k].x + t[q][k].y) * a.h2q;
        }
    }
}

// ------------------------------------------------------------------ rotations and reflections
// With the reflection symmetry as well (see fp_rot8_f32_kernel), the views -k + mV/4 add, per
// pixel p, U_m(p) = sum_k sum_j y[-k + mV/4][n_det - 1 - j] a(k, j, p) over the views
// k = 0 .. V/8 that are not their own mirror images, and
//     (A^T y)[n] = sum_m T_m(R^-m n) + sum_m U_m(M R^-m n),   M (i, r) = (i, N-1-r).
// Two per-call tables hold the 16 weighted values of a cell pair (2m, 2m + 1): T8[k][m],
// 32 bytes, y[k + rV/4][j] w_j (r = 0..3), and after it U8[k][m], 32 bytes,
// y[-k + rV/4][n_det - 1 - j] w_j (zero for the self-mirror views k = 0 and 8k = V), each
// the first cell's four values, then the second's; w_j = 2/B of (k, j), 0 past n_det.  Two
// 32-byte tables rather than one of 64-byte records, and even-aligned pairs only: the
// neighbouring lanes of a warp, about two pairs apart, then share 128-byte lines, and the
// L1 data pipe, the back projector's bound, moves fewer wavefronts.
__global__ void sino_pairs_rot8_kernel(const float *__restrict__ y, const BoxF *__restrict__ box,
                                       float4 *__restrict__ y8, int nv, int nd)
{
    const int ndh = (nd + 1) >> 1, nk = nv / 8 + 1, v4 = nv >> 2;
    const long long n = (long long)nk * ndh;
    y += (long long)blockIdx.y * nv * nd;   // image y of a batch
    y8 += 4 * n * blockIdx.y;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(t / ndh), m = (int)(t - (long long)k * ndh);
        const bool self = k == 0 || 8 * k == nv;
        const BoxF *br = box + (long long)k * nd;
        float out[16];
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            const int j = 2 * m + hh;
            const float w = j < nd ? 1.f / (br[j].q - br[j].hC) : 0.f;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const float *yt = y + (long long)(k + r * v4) * nd;
                const float *yu = y + (long long)((nv - k + r * v4) % nv) * nd;
                out[4 * hh + r] = j < nd ? yt[j] * w : 0.f;
                out[8 + 4 * hh + r] = (j < nd && !self) ? yu[nd - 1 - j] * w : 0.f;
            }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c)   // T8 at float4 2t, U8 at 2n + 2t
            y8[(c < 2 ? 0 : 2 * n) + 2 * t + (c & 1)] = make_float4(out[4 * c], out[4 * c + 1], out[4 * c + 2], out[4 * c + 3]);
    }
}

// bp_view2_rot4 with the eight values per cell pair (the merged constants and 2 x 32 bytes
// of weighted sinogram, uoff floats apart), over even-aligned pairs only: the pairs
// (2m, 2m + 1) that cover the window, so a cell just outside it may be evaluated too (its
// entry is zero, or rounding-level at the support's edge).  Each pixel's two entries are
// applied to the pair's sixteen values as packed pairs of neighbouring values (adjacent
// registers of the 256-bit loads): ta[i], tb[i] accumulate the values 2i and 2i + 1 of
// T_0..3, U_0..3.  (Warp-uniform alignment halves the lines a warp's loads touch, for about
// a fifth more pair steps: 0.231 -> 0.226 ms at 512^2 x 720; the quarter-turn kernel, with
// two loads per step, is faster with both alignments.)
template <bool ARC, bool EXACT>
__device__ __forceinline__ void bp_view2_rot8(const BpPixel4 &Qa, const BpPixel4 &Qb, float hwc, int J,
                                              const BpArgs &a, int nd, const float *__restrict__ y8row,
                                              const float *__restrict__ acrow, long long uoff, float2 (&ta)[4],
                                              float2 (&tb)[4])
{
    int g0, g1;
    pair_window(Qa.P, Qb.P, hwc, J, nd, g0, g1);
    const int m0 = g0 >> 1, m1 = g1 >> 1;   // m0 > m1 when the window misses the detector
    const float off = (float)(2 * m0 - J);
    const float sa = ARC ? 1.f : Qa.P.Dn, sb = ARC ? 1.f : Qb.P.Dn;
    float2 da = make_float2(sa * (Qa.P.sig - off), sa * (Qa.P.sig - off - 1.f));
    float2 db = make_float2(sb * (Qb.P.sig - off), sb * (Qb.P.sig - off - 1.f));
    const float2 sta = make_float2(-2.f * sa, -2.f * sa), stb = make_float2(-2.f * sb, -2.f * sb);
    for (int m = m0; m <= m1; ++m) {
        float A[8], Y[8], Z[8];
        ldg256(acrow + 8 * m, A);          // q/C | p/C | ds/(L C) | c1/C, pairs
        ldg256(y8row + 8 * m, Y);          // T8: pairs of the four rotations
        ldg256(y8row + 8 * m + uoff, Z);   // U8: pairs of the four mirrored views
        const float2 wa = bp_pair_rot4<ARC, EXACT>(Qa, da, A, a);
        const float2 wb = bp_pair_rot4<ARC, EXACT>(Qb, db, A, a);
        const float2 wa0 = make_float2(wa.x, wa.x), wa1 = make_float2(wa.y, wa.y);
        const float2 wb0 = make_float2(wb.x, wb.x), wb1 = make_float2(wb.y, wb.y);
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const float2 y0 = make_float2(Y[2 * i], Y[2 * i + 1]), y1 = make_float2(Y[4 + 2 * i], Y[5 + 2 * i]);
            const float2 z0 = make_float2(Z[2 * i], Z[2 * i + 1]), z1 = make_float2(Z[4 + 2 * i], Z[5 + 2 * i]);
            ta[i] = __ffma2_rn(y1, wa1, __ffma2_rn(y0, wa0, ta[i]));
            tb[i] = __ffma2_rn(y1, wb1, __ffma2_rn(y0, wb0, tb[i]));
            ta[2 + i] = __ffma2_rn(z1, wa1, __ffma2_rn(z0, wa0, ta[2 + i]));
            tb[2 + i] = __ffma2_rn(z1, wb1, __ffma2_rn(z0, wb0, tb[2 + i]));
        }
        da = __fadd2_rn(da, sta);
        db = __fadd2_rn(db, stb);
    }
}

// bp_rot4_f32_kernel over the views k = 0 .. V/8 with the eight accumulators T_0..3, U_0..3
// per pixel: the partial images partial[8 s + c] of view part s.
template <bool ARC, bool EXACT, bool BATCH>
__global__ void __launch_bounds__(BP_QUAD_THREADS, 8) bp_rot8_f32_kernel(GeomConsts g, const float *__restrict__ ac,
                                                                     const float *__restrict__ y8, BpArgs a,
                                                                     const int *__restrict__ order, int ntx, int nsplit,
                                                                     float *__restrict__ partial,
                                                                     const double *__restrict__ view_cs,
                                                                     const float4 *__restrict__ tvtab,
                                                                     const int *__restrict__ tjtab)
{
    __shared__ TileViewS<float> tv[BP_CHUNK];
    __shared__ int tj[BP_CHUNK];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // lanes 4k .. 4k + 3 take a 2 x 2 block of quads: their cell windows lie close, so a
    // warp's loads touch fewer 128-byte lines per group of four lanes
    const int tx = 2 * ((lane & 1) | ((lane >> 1) & 6)), ty = 8 * warp + 2 * (((lane >> 1) & 1) | ((lane >> 3) & 2));
    const int tile = order[blockIdx.x];   // tiles with the most work first
    const int it = (tile % ntx) * BP_T, rt = (tile / ntx) * BP_T;
    const int nk = g.nv / 8 + 1;
    const int vbeg = (int)((long long)nk * blockIdx.y / nsplit), vend = (int)((long long)nk * (blockIdx.y + 1) / nsplit);
    if (BATCH) {   // image z of a batch (the single-image instantiation has no offsets)
        y8 += 16LL * blockIdx.z * nk * ((g.nd + 1) >> 1);
        partial += 8LL * blockIdx.z * nsplit * g.nx * g.ny;
    }
    const int i = it + tx, r = rt + ty;
    const bool in0 = i < g.nx && r < g.ny, in1 = i + 1 < g.nx && r < g.ny;
    const bool in2 = i < g.nx && r + 1 < g.ny, in3 = i + 1 < g.nx && r + 1 < g.ny;
    const int ndh = (g.nd + 1) >> 1;
    const double refx = tile_ref(it, g.nx), refy = tile_ref(rt, g.ny);
    const float di = (float)(tx - refx), dr = (float)(ty - refy);
    float2 t[4][4];   // [quad pixel][(T_0, T_1), (T_2, T_3), (U_0, U_1), (U_2, U_3)]
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int k = 0; k < 4; ++k) t[q][k] = make_float2(0.f, 0.f);
    for (int v0 = vbeg; v0 < vend; v0 += BP_CHUNK) {
        const int nvc = min(BP_CHUNK, vend - v0);
        __syncthreads();
        for (int k = tid; k < nvc; k += BP_QUAD_THREADS) {
            if (tvtab) {   // precomputed with the geometry
                const long long tt = (long long)tile * g.nv + v0 + k;
                const float4 u0 = __ldg(tvtab + 2 * tt), u1 = __ldg(tvtab + 2 * tt + 1);
                TileViewS<float> T;
                T.Dt = u0.x; T.yt = u0.y; T.a1 = u0.z; T.b1 = u0.w; T.rho = u1.x; T.phi = u1.y; T.hc = u1.z; T.hs = u1.w;
                tv[k] = T;
                tj[k] = __ldg(tjtab + tt);
            } else {
                tile_view_f32(g, view_cs[2 * (v0 + k)], view_cs[2 * (v0 + k) + 1], it + refx, rt + refy, tv[k],
                              tj[k]);
            }
        }
        __syncthreads();
        if (!in0) continue;
        for (int vv = 0; vv < nvc; ++vv) {
            const int v = v0 + vv;
            const TileViewS<float> T = tv[vv];
            const int J = tj[vv];
            const float *arow = ac + 8 * (long long)v * ndh;
            const float *yrow = y8 + 8 * (long long)v * ndh;
            const long long uoff = 8LL * nk * ndh;   // U8 after T8
            const QuadView Q = quad_view_setup<ARC>(T, di, dr, in1, in2, in3, a);
            const BpPixel4 P0 = bp_pixel4<ARC>(Q.P0, J, a), P1 = bp_pixel4<ARC>(Q.P1, J, a);
            const BpPixel4 P2 = bp_pixel4<ARC>(Q.P2, J, a), P3 = bp_pixel4<ARC>(Q.P3, J, a);
            if (Q.col) {   // P1 is quad pixel 2, P2 quad pixel 1
                bp_view2_rot8<ARC, EXACT>(P0, P1, Q.hwc, J, a, g.nd, yrow, arow, uoff, t[0], t[2]);
                bp_view2_rot8<ARC, EXACT>(P2, P3, Q.hwc, J, a, g.nd, yrow, arow, uoff, t[1], t[3]);
            } else {
                bp_view2_rot8<ARC, EXACT>(P0, P1, Q.hwc, J, a, g.nd, yrow, arow, uoff, t[0], t[1]);
                bp_view2_rot8<ARC, EXACT>(P2, P3, Q.hwc, J, a, g.nd, yrow, arow, uoff, t[2], t[3]);
            }
        }
    }
    if (in0) {
        const long long nn = (long long)g.nx * g.ny;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int iq = i + (q & 1), rq = r + (q >> 1);
            if (iq >= g.nx || rq >= g.ny) continue;
#pragma unroll
            for (int k = 0; k < 8; ++k)
                partial[(8LL * blockIdx.y + k) * nn + (long long)rq * g.nx + iq] =
                    ((k & 1) ? t[q][k >> 1].y : t[q][k >> 1].x) * a.h2q;
        }
    }
}

// img[n] = sum_m T_m(R^-m n) + sum_m U_m(M R^-m n), T_m and U_m the sums of partial[8 s + m]
// and partial[8 s + 4 + m] over the view parts s (in part order), through eight 32 x 32
// shared-memory tiles: M (i, r) = (i, N-1-r), M R^-1 (i, r) = (r, i), M R^-2 (i, r) =
// (N-1-i, r), M R^-3 (i, r) = (N-1-r, N-1-i).
template <int NS, bool BATCH>
__global__ void __launch_bounds__(1024) orbit_sum8_kernel(const float *__restrict__ partial, float *__restrict__ img,
                                                          int n)
{
    __shared__ float s[8][32][33];
    const int i0 = blockIdx.x * 32, r0 = blockIdx.y * 32, tx = threadIdx.x, a = threadIdx.y;
    const long long nn = (long long)n * n;
    if (BATCH) {   // image z of a batch
        partial += 8LL * NS * nn * blockIdx.z;
        img += nn * blockIdx.z;
    }
    // source rows and columns of the eight tiles at (a, tx)
    const int rows[8] = {r0 + a, n - i0 - 32 + a, n - r0 - 32 + a, i0 + a,
                         n - r0 - 32 + a, i0 + a, r0 + a, n - i0 - 32 + a};
    const int cols[8] = {i0 + tx, r0 + tx, n - i0 - 32 + tx, n - r0 - 32 + tx,
                         i0 + tx, r0 + tx, n - i0 - 32 + tx, n - r0 - 32 + tx};
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        float v = 0.f;
        if (rows[c] >= 0 && rows[c] < n && cols[c] >= 0 && cols[c] < n) {
            const float *src = partial + (long long)c * nn + (long long)rows[c] * n + cols[c];
            float w[NS];
#pragma unroll
            for (int sp = 0; sp < NS; ++sp) w[sp] = __ldg(src + 8LL * sp * nn);   // all loads in flight
            v = w[0];
#pragma unroll
            for (int sp = 1; sp < NS; ++sp) v += w[sp];
        }
        s[c][a][tx] = v;
    }
    __syncthreads();
    if (i0 + tx < n && r0 + a < n) {
        const float tsum = ((s[0][a][tx] + s[1][31 - tx][a]) + s[2][31 - a][31 - tx]) + s[3][tx][31 - a];
        const float usum = ((s[4][31 - a][tx] + s[5][tx][a]) + s[6][a][31 - tx]) + s[7][31 - tx][31 - a];
        img[(long long)(r0 + a) * n + i0 + tx] = tsum + usum;
    }
}

// img[n] = sum_k T_k(R^-k n), T_k the sum of partial[4 s + k] over the view parts s (in part
// order), through four 32 x 32 shared-memory tiles: R^-1 (i, r) = (r, N-1-i),
// R^-2 (i, r) = (N-1-i, N-1-r), R^-3 (i, r) = (N-1-r, i).
template <int NS, bool BATCH>
__global__ void __launch_bounds__(1024) orbit_sum_kernel(const float *__restrict__ partial, float *__restrict__ img,
                                                         int n)
{
    __shared__ float s[4][32][33];
    const int i0 = blockIdx.x * 32, r0 = blockIdx.y * 32, tx = threadIdx.x, a = threadIdx.y;
    const long long nn = (long long)n * n;
    if (BATCH) {   // image z of a batch
        partial += 4LL * NS * nn * blockIdx.z;
        img += nn * blockIdx.z;
    }
    const int rows[4] = {r0 + a, n - i0 - 32 + a, n - r0 - 32 + a, i0 + a};
    const int cols[4] = {i0 + tx, r0 + tx, n - i0 - 32 + tx, n - r0 - 32 + tx};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        float v = 0.f;
        if (rows[c] >= 0 && rows[c] < n && cols[c] >= 0 && cols[c] < n) {
            const float *src = partial + (long long)c * nn + (long long)rows[c] * n + cols[c];
            float w[NS];
#pragma unroll
            for (int sp = 0; sp < NS; ++sp) w[sp] = __ldg(src + 4LL * sp * nn);   // all loads in flight
            v = w[0];
#pragma unroll
            for (int sp = 1; sp < NS; ++sp) v += w[sp];
        }
        s[c][a][tx] = v;
    }
    __syncthreads();
    if (i0 + tx < n && r0 + a < n)
        img[(long long)(r0 + a) * n + i0 + tx] = ((s[0][a][tx] + s[1][31 - tx][a]) + s[2][31 - a][31 - tx]) + s[3][tx][31 - a];
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
    const double refx = tile_ref(it, g.nx), refy = tile_ref(rt, g.ny);
    const double di = tx - refx, dr = ty - refy;
    double acc = 0.0;
    for (int v0 = 0; v0 < g.nv; v0 += chunk) {
        const int nvc = min(chunk, g.nv - v0);
        __syncthreads();
        if (tid < nvc) {
            double c = view_cs[2 * (v0 + tid)], s = view_cs[2 * (v0 + tid) + 1];
            TileViewS<double> T;
            int J;
            tile_view_double(g, c, s, it + refx, rt + refy, &T.Dt, &T.yt, &T.a1, &T.b1, &T.rho, &T.phi, &J, &T.hc,
                             &T.hs);
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
            const double sig = g.arc ? T.phi + atan((T.a1 * di + T.b1 * dr) / (Dn * T.Dt + yp * T.yt)) * (g.dps / g.ds)
                                     : T.phi + (T.rho + T.a1 * di + T.b1 * dr) / Dn;
            const double R = sqrt(Dn * Dn + yp * yp);
            const double zs = fabs(yp * T.hc - Dn * T.hs) + fabs(yp * T.hs + Dn * T.hc);
            const double hwc = kz * zs / (Dn * Dn) * (1.02 + 2.0 * g.h / Dn) + ke;
            const int jlo = max((int)ceil(sig - hwc), -J);
            const int jhi = min((int)floor(sig + hwc), g.nd - 1 - J);
            double part = 0.0;
            for (int jl = jlo; jl <= jhi; ++jl) {
                const int j = J + jl;
                const double sg = celld[4 * j], cg = celld[4 * j + 1], dt = celld[4 * j + 2];
                // normal of the cell's ray: sin(g_j) u + cos(g_j) w (parallel rays: w)
                const double nxv = sg * c - cg * s, nyv = sg * s + cg * c;
                const double B = g.h * fmax(fabs(nxv), fabs(nyv)), C = g.h * fmin(fabs(nxv), fabs(nyv));
                const BoxConsts<double> bc = make_box_consts<double>(B, C, g.h);
                // |s'|: parallel ds |sigma - j|; flat D_n (ds / L_j) |sigma - j|; arc R |sin(angle)|
                const double x = g.par ? fabs(g.ds * (sig - jl))
                                 : g.arc ? fabs(R * sin((g.ds / g.dps) * (sig - jl)))
                                         : fabs(Dn * (g.ds * cg / g.dps) * (sig - jl));
                // tau'/2 = depth along the cell's ray * dtan_j / 2
                const double e = g.par ? 0.5 * g.tau : (cg * Dn + sg * yp) * 0.5 * dt;
                const double w = window_diff(x, e, bc.q, bc.p * bc.iC, bc.iC, 0.5 * C);
                part += yrow[j] * bc.nrm * (w / e);
            }
            acc += part;
        }
    }
    if (inside) img[(b * g.ny + r) * g.nx + i] = acc;
}

// The orbit sums for the view-part counts the launchers use (powers of two up to 32).
static void launch_orbit_sum8(const float *partial, float *img, int n, int nsplit, int nb, cudaStream_t st)
{
    const unsigned nt = (unsigned)((n + 31) / 32);
    const dim3 grd(nt, nt, nb), blk(32, 32);
    switch (nsplit) {
        case 1: (nb > 1 ? orbit_sum8_kernel<1, true> : orbit_sum8_kernel<1, false>)<<<grd, blk, 0, st>>>(partial, img, n); break;
        case 2: (nb > 1 ? orbit_sum8_kernel<2, true> : orbit_sum8_kernel<2, false>)<<<grd, blk, 0, st>>>(partial, img, n); break;
        case 4: (nb > 1 ? orbit_sum8_kernel<4, true> : orbit_sum8_kernel<4, false>)<<<grd, blk, 0, st>>>(partial, img, n); break;
        case 8: (nb > 1 ? orbit_sum8_kernel<8, true> : orbit_sum8_kernel<8, false>)<<<grd, blk, 0, st>>>(partial, img, n); break;
        case 16: (nb > 1 ? orbit_sum8_kernel<16, true> : orbit_sum8_kernel<16, false>)<<<grd, blk, 0, st>>>(partial, img, n); break;
        default: (nb > 1 ? orbit_sum8_kernel<32, true> : orbit_sum8_kernel<32, false>)<<<grd, blk, 0, st>>>(partial, img, n); break;
    }
}

static void launch_orbit_sum4(const float *partial, float *img, int n, int nsplit, int nb, cudaStream_t st)
{
    const unsigned nt = (unsigned)((n + 31) / 32);
    const dim3 grd(nt, nt, nb), blk(32, 32);
    switch (nsplit) {
        case 1: (nb > 1 ? orbit_sum_kernel<1, true> : orbit_sum_kernel<1, false>)<<<grd, blk, 0, st>>>(partial, img, n); break;
        case 2: (nb > 1 ? orbit_sum_kernel<2, true> : orbit_sum_kernel<2, false>)<<<grd, blk, 0, st>>>(partial, img, n); break;
        case 4: (nb > 1 ? orbit_sum_kernel<4, true> : orbit_sum_kernel<4, false>)<<<grd, blk, 0, st>>>(partial, img, n); break;
        case 8: (nb > 1 ? orbit_sum_kernel<8, true> : orbit_sum_kernel<8, false>)<<<grd, blk, 0, st>>>(partial, img, n); break;
        case 16: (nb > 1 ? orbit_sum_kernel<16, true> : orbit_sum_kernel<16, false>)<<<grd, blk, 0, st>>>(partial, img, n); break;
        default: (nb > 1 ? orbit_sum_kernel<32, true> : orbit_sum_kernel<32, false>)<<<grd, blk, 0, st>>>(partial, img, n); break;
    }
}

// The sinogram as weighted cell pairs of parity o: y2[b][v][m] = (w y[b][v][2m + o],
// w' y[b][v][2m + o + 1]) with w = 2/B of that (view, cell) (the normalisation h^2/(2B) of
// Eq. 18 without h^2/4), 0 for cells past n_det.
__global__ void sino_pairs_kernel(const float *__restrict__ y, const BoxF *__restrict__ box, float2 *__restrict__ y2,
                                  long long nrows, int nv, int nd, int o)
{
    const int ndh = (nd + 1) >> 1;
    const long long n = nrows * ndh;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const long long row = t / ndh;
        const int j = 2 * (int)(t - row * ndh) + o;
        const float *yr = y + row * nd;
        const BoxF *br = box + (row % nv) * nd;
        float2 v = make_float2(0.f, 0.f);
        if (j < nd) v.x = yr[j] / (br[j].q - br[j].hC);
        if (j + 1 < nd) v.y = yr[j + 1] / (br[j + 1].q - br[j + 1].hC);
        y2[t] = v;
    }
}

// View parts per tile of the FP32 single-image gather: enough blocks for several waves, so
// each tile's views are split (up to 32 parts of at least 16 views) when the tiles alone
// give fewer than ~32 blocks per SM (partial images, then a fixed-order sum).
static int bp_view_parts(const cnsf_geometry *geo, int batch)
{
    const GeomConsts &g = geo->gc;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, geo->device);
    const long long blocks = (long long)((g.nx + BP_T - 1) / BP_T) * ((g.ny + BP_T - 1) / BP_T) * batch;
    int nsplit = 1;
    while (nsplit < 32 && blocks * nsplit < 32LL * std::max(sms, 1) && g.nv / (2 * nsplit) >= 16) nsplit *= 2;
    return nsplit;
}

// View parts of the eight-value gather (over the views 0 .. V/8).
static int bp_view_parts_rot8(const cnsf_geometry *geo)
{
    const GeomConsts &g = geo->gc;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, geo->device);
    const long long blocks = (long long)((g.nx + BP_T - 1) / BP_T) * ((g.ny + BP_T - 1) / BP_T);
    int nsplit = 1;
    while (nsplit < 32 && blocks * nsplit < 32LL * std::max(sms, 1) && (g.nv / 8 + 1) / (2 * nsplit) >= 8) nsplit *= 2;
    return nsplit;
}

// Bytes of one image's scratch on the eight-value path (cell-pair records, partial images).
static size_t back_rot8_image_bytes(const cnsf_geometry *geo)
{
    const GeomConsts &g = geo->gc;
    const size_t y8 = (size_t)(g.nv / 8 + 1) * ((g.nd + 1) / 2) * 16 * sizeof(float);
    return y8 + (size_t)bp_view_parts_rot8(geo) * 8 * g.nx * g.ny * sizeof(float);
}

// FP32 back projection of a batch by the eight-value gather (geo->sym8), in groups of
// sym_batch_group() images (one grid layer per image); every image takes the kernel, view
// parts and part order of a single-image call.
static int launch_back_rot8(const cnsf_geometry *geo, const float *sino, float *img, int batch, cudaStream_t st)
{
    const GeomConsts &g = geo->gc;
    const int nk = g.nv / 8 + 1, ndh = (g.nd + 1) / 2, n = g.nx;
    const int nsplit = bp_view_parts_rot8(geo);
    const size_t ny8 = (size_t)nk * ndh * 16;   // T8 and U8 of one image, floats
    const size_t per = back_rot8_image_bytes(geo);
    const int grp = sym_batch_group(per, batch);
    char *buf = nullptr;
    cudaError_t e = scratch_alloc((void **)&buf, (size_t)grp * per, st);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? (record_cuda_error(e), CNSF_ERR_NOMEM) : record_cuda_error(e);
    const double dg = g.arc ? g.ds / g.dps : 0.0;
    BpArgs a{(float)geo->bw.kz, (float)geo->bw.ke, (float)(2.0 * g.h), (float)(2.0 * g.h * g.h), (float)(0.25 * g.h * g.h),
             (float)(g.arc ? g.dps / g.ds : 0.0), (float)dg, (float)(-dg * dg / 6.0), 8LL * g.nv * ndh, 8 * ndh,
             (float)g.s0, (float)g.ds, (float)(g.par ? 0.0 : 1.0 / g.dps),
             (float)(g.arc ? tan(0.5 * g.tau / g.dps) / (g.ds / g.dps) : 0.0), (float)(g.arc ? -0.5 * (g.ds / g.dps) * (g.ds / g.dps) : 0.0)};
    const int ntx = (g.nx + BP_T - 1) / BP_T, nty = (g.ny + BP_T - 1) / BP_T;
    float *y8 = reinterpret_cast<float *>(buf), *partial = y8 + grp * ny8;
    const long long npair = (long long)nk * ndh;
    auto kern1 = g.arc ? (geo->exact ? bp_rot8_f32_kernel<true, true, false> : bp_rot8_f32_kernel<true, false, false>)
                       : (geo->exact ? bp_rot8_f32_kernel<false, true, false> : bp_rot8_f32_kernel<false, false, false>);
    auto kernb = g.arc ? (geo->exact ? bp_rot8_f32_kernel<true, true, true> : bp_rot8_f32_kernel<true, false, true>)
                       : (geo->exact ? bp_rot8_f32_kernel<false, true, true> : bp_rot8_f32_kernel<false, false, true>);
    for (int b0 = 0; b0 < batch; b0 += grp) {
        const int gb = std::min(grp, batch - b0);
        auto kern = gb > 1 ? kernb : kern1;
        sino_pairs_rot8_kernel<<<dim3((unsigned)std::min<long long>((npair + 255) / 256, 8192), gb), 256, 0, st>>>(
            sino + (size_t)b0 * g.nv * g.nd, geo->d_box, reinterpret_cast<float4 *>(y8), g.nv, g.nd);
        kern<<<dim3(ntx * nty, nsplit, gb), dim3(BP_QUAD_THREADS), 0, st>>>(g, geo->d_ac, y8, a, geo->d_bp_order, ntx,
                                                                         nsplit, partial, geo->d_view_cs, geo->d_tv,
                                                                         geo->d_tj);
        launch_orbit_sum8(partial, img + (size_t)b0 * n * n, n, nsplit, gb, st);
    }
    cudaFreeAsync(buf, st);
    e = cudaGetLastError();
    return e == cudaSuccess ? CNSF_OK : record_cuda_error(e);
}

// View parts of the four-rotation gather (over the first quarter of the views).
static int bp_view_parts_rot4(const cnsf_geometry *geo)
{
    const GeomConsts &g = geo->gc;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, geo->device);
    const long long blocks = (long long)((g.nx + BP_T - 1) / BP_T) * ((g.ny + BP_T - 1) / BP_T);
    int nsplit = 1;
    while (nsplit < 32 && blocks * nsplit < 32LL * std::max(sms, 1) && (g.nv / 4) / (2 * nsplit) >= 8) nsplit *= 2;
    return nsplit;
}

static size_t back_rot4_image_bytes(const cnsf_geometry *geo)
{
    const GeomConsts &g = geo->gc;
    const size_t y4 = 2 * (size_t)(g.nv / 4) * ((g.nd + 1) / 2) * 8 * sizeof(float);
    return y4 + (size_t)bp_view_parts_rot4(geo) * 4 * g.nx * g.ny * sizeof(float);
}

// FP32 back projection of a batch by the four-rotation gather (geo->sym), grouped as
// launch_back_rot8.
static int launch_back_rot4(const cnsf_geometry *geo, const float *sino, float *img, int batch, cudaStream_t st)
{
    const GeomConsts &g = geo->gc;
    const int nv4 = g.nv / 4, ndh = (g.nd + 1) / 2, n = g.nx;
    const int nsplit = bp_view_parts_rot4(geo);
    const size_t ny4 = 2 * (size_t)nv4 * ndh * 8;
    const size_t per = back_rot4_image_bytes(geo);
    const int grp = sym_batch_group(per, batch);
    char *buf = nullptr;
    cudaError_t e = scratch_alloc((void **)&buf, (size_t)grp * per, st);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? (record_cuda_error(e), CNSF_ERR_NOMEM) : record_cuda_error(e);
    const double dg = g.arc ? g.ds / g.dps : 0.0;
    BpArgs a{(float)geo->bw.kz, (float)geo->bw.ke, (float)(2.0 * g.h), (float)(2.0 * g.h * g.h), (float)(0.25 * g.h * g.h),
             (float)(g.arc ? g.dps / g.ds : 0.0), (float)dg, (float)(-dg * dg / 6.0), 8LL * g.nv * ndh, 8 * ndh,
             (float)g.s0, (float)g.ds, (float)(g.par ? 0.0 : 1.0 / g.dps),
             (float)(g.arc ? tan(0.5 * g.tau / g.dps) / (g.ds / g.dps) : 0.0), (float)(g.arc ? -0.5 * (g.ds / g.dps) * (g.ds / g.dps) : 0.0)};
    const int ntx = (g.nx + BP_T - 1) / BP_T, nty = (g.ny + BP_T - 1) / BP_T;
    float *y4 = reinterpret_cast<float *>(buf), *partial = y4 + grp * ny4;
    const long long npair = 2LL * nv4 * ndh;
    auto kern1 = g.arc ? (geo->exact ? bp_rot4_f32_kernel<true, true, false> : bp_rot4_f32_kernel<true, false, false>)
                       : (geo->exact ? bp_rot4_f32_kernel<false, true, false> : bp_rot4_f32_kernel<false, false, false>);
    auto kernb = g.arc ? (geo->exact ? bp_rot4_f32_kernel<true, true, true> : bp_rot4_f32_kernel<true, false, true>)
                       : (geo->exact ? bp_rot4_f32_kernel<false, true, true> : bp_rot4_f32_kernel<false, false, true>);
    for (int b0 = 0; b0 < batch; b0 += grp) {
        const int gb = std::min(grp, batch - b0);
        auto kern = gb > 1 ? kernb : kern1;
        sino_pairs_rot4_kernel<<<dim3((unsigned)std::min<long long>((npair + 255) / 256, 8192), gb), 256, 0, st>>>(
            sino + (size_t)b0 * g.nv * g.nd, geo->d_box, reinterpret_cast<float4 *>(y4), g.nv, g.nd);
        kern<<<dim3(ntx * nty, nsplit, gb), dim3(BP_QUAD_THREADS), 0, st>>>(g, geo->d_ac, y4, a, geo->d_bp_order, ntx,
                                                                         nsplit, partial, geo->d_view_cs, geo->d_tv,
                                                                         geo->d_tj);
        launch_orbit_sum4(partial, img + (size_t)b0 * n * n, n, nsplit, gb, st);
    }
    cudaFreeAsync(buf, st);
    e = cudaGetLastError();
    return e == cudaSuccess ? CNSF_OK : record_cuda_error(e);
}

int launch_back_sym(const cnsf_geometry *geo, const float *sino, float *img, int batch, cudaStream_t st)
{
    if (batch == 0) return CNSF_OK;
    if (geo->sym8) return launch_back_rot8(geo, sino, img, batch, st);
    if (geo->sym) return launch_back_rot4(geo, sino, img, batch, st);
    return CNSF_ERR_UNSUPPORTED;
}

size_t back_alloc_bytes(const cnsf_geometry *geo, int batch, int dtype)
{
    if (batch <= 0 || dtype != CNSF_F32) return 0;
    if (geo->sym8) return (size_t)sym_batch_group(back_rot8_image_bytes(geo), batch) * back_rot8_image_bytes(geo);
    if (geo->sym) return (size_t)sym_batch_group(back_rot4_image_bytes(geo), batch) * back_rot4_image_bytes(geo);
    if (batch >= 2) return back_batch_alloc_bytes(geo);
    const GeomConsts &g = geo->gc;
    const int nsplit = bp_view_parts(geo, batch);
    const size_t npair = (size_t)batch * g.nv * ((g.nd + 1) / 2);
    // the weighted sinogram pairs in both alignments
    return (nsplit > 1 ? (size_t)nsplit * batch * g.nx * g.ny * sizeof(float) : 0) + 2 * npair * sizeof(float2);
}

int launch_back(const cnsf_geometry *geo, const void *sino, void *img, int batch, int dtype, cudaStream_t st)
{
    if (batch == 0) return CNSF_OK;
    if (dtype == CNSF_F32 && (geo->sym8 || geo->sym))
        return launch_back_sym(geo, (const float *)sino, (float *)img, batch, st);
    if (dtype == CNSF_F32 && batch >= 2) return launch_back_batch(geo, (const float *)sino, (float *)img, batch, st);
    const GeomConsts &g = geo->gc;
    dim3 blk(BP_T, BP_T), grd((g.nx + BP_T - 1) / BP_T, (g.ny + BP_T - 1) / BP_T, batch);
    if (dtype == CNSF_F32) {
        const double dg = g.arc ? g.ds / g.dps : 0.0;
        BpArgs a{(float)geo->bw.kz, (float)geo->bw.ke, (float)(2.0 * g.h), (float)(2.0 * g.h * g.h),
                 (float)(0.25 * g.h * g.h),
                 (float)(g.arc ? g.dps / g.ds : 0.0), (float)dg, (float)(-dg * dg / 6.0),
                 8LL * g.nv * ((g.nd + 1) / 2), 8 * ((g.nd + 1) / 2),
             (float)g.s0, (float)g.ds, (float)(g.par ? 0.0 : 1.0 / g.dps),
             (float)(g.arc ? tan(0.5 * g.tau / g.dps) / (g.ds / g.dps) : 0.0), (float)(g.arc ? -0.5 * (g.ds / g.dps) * (g.ds / g.dps) : 0.0)};
        const int nsplit = bp_view_parts(geo, batch);
        float *partial = nullptr;
        const long long nimg = (long long)batch * g.nx * g.ny;
        if (nsplit > 1) {
            cudaError_t e = scratch_alloc((void **)&partial, (size_t)nsplit * nimg * sizeof(float), st);
            if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? (record_cuda_error(e), CNSF_ERR_NOMEM) : record_cuda_error(e);
        }
        // the sinogram as weighted cell pairs in both alignments (copies: each value carries
        // the 2/B of its view and cell)
        const long long nrows = (long long)batch * g.nv, npair = nrows * ((g.nd + 1) / 2);
        float2 *copy = nullptr;
        cudaError_t e = scratch_alloc((void **)&copy, (size_t)2 * npair * sizeof(float2), st);
        if (e != cudaSuccess) {
            if (partial) cudaFreeAsync(partial, st);
            return e == cudaErrorMemoryAllocation ? (record_cuda_error(e), CNSF_ERR_NOMEM) : record_cuda_error(e);
        }
        const unsigned pblocks = (unsigned)std::min<long long>((npair + 255) / 256, 8192);
        sino_pairs_kernel<<<pblocks, 256, 0, st>>>((const float *)sino, geo->d_box, copy, nrows, g.nv, g.nd, 1);
        sino_pairs_kernel<<<pblocks, 256, 0, st>>>((const float *)sino, geo->d_box, copy + npair, nrows, g.nv, g.nd, 0);
        const float2 *y2 = copy + npair;
        auto kern = g.arc ? (geo->exact ? bp_f32_kernel<true, true> : bp_f32_kernel<true, false>)
                          : (geo->exact ? bp_f32_kernel<false, true> : bp_f32_kernel<false, false>);
        kern<<<dim3(grd.x * grd.y, nsplit, grd.z), dim3(BP_QUAD_THREADS), 0, st>>>(
            g, geo->d_view_cs, geo->d_box2, geo->d_cell2, y2, copy, (float *)img, a, geo->d_bp_order,
            (int)grd.x, nsplit, partial, geo->d_tv, geo->d_tj);
        if (copy) cudaFreeAsync(copy, st);
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
