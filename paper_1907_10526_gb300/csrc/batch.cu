// batch.cu -- forward and back projection of a batch of images (FP32), each entry of A
// evaluated once per chunk of up to 16 images.
//
// The per-image kernels evaluate the footprint (Eq. 18) once per (view, cell, pixel) and
// image.  For a batch, the entry is the same for every image, so these kernels evaluate it
// once and apply it to a chunk of NB = 4, 8 or 16 images.  Both directions read their
// input from a batch-interleaved copy (the NB values of one pixel, or of one cell, are
// contiguous), so the chunk costs NB/4 16-byte loads and NB FMAs per entry.
#include <cuda_runtime.h>

#include <algorithm>

#include "cnsf_internal.cuh"
#include "cnsf_runtime.h"
#include "footprint.cuh"

namespace cnsf {

// ------------------------------------------------------------------ interleaved copies
// out[row][c][q] (q < NB fastest) = img[b0 + q][row][c - pad], zero outside the image or
// beyond the batch.  transposed: rows are image columns.
__global__ void pad_interleave_kernel(const float *__restrict__ img, float *__restrict__ out, int nx, int ny,
                                      int pad, int pitch, int b0, int nb_used, int NB, int transposed)
{
    const long long total = (long long)(transposed ? nx : ny) * pitch * NB;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(t % NB);
        const long long rc = t / NB;
        const int c = (int)(rc % pitch), row = (int)(rc / pitch);
        const int a = c - pad;   // index across the line
        float v = 0.f;
        if (q < nb_used) {
            const int i = transposed ? row : a, r = transposed ? a : row;
            if (a >= 0 && a < (transposed ? ny : nx))
                v = img[((long long)(b0 + q) * ny + r) * nx + i];
        }
        out[t] = v;
    }
}

// out[v][j][q] = y[b0 + q][v][j] (0 beyond the batch)
__global__ void sino_interleave_kernel(const float *__restrict__ y, float *__restrict__ out, long long nvd, int b0,
                                       int nb_used, int NB)
{
    const long long total = nvd * NB;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(t % NB);
        const long long vj = t / NB;
        out[t] = q < nb_used ? y[(long long)(b0 + q) * nvd + vj] : 0.f;
    }
}

template <int NB4>
struct Acc {
    float4 v[NB4];
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int k = 0; k < NB4; ++k) v[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    // packed FP32x2 (FFMA2/FADD2): two images per instruction, the same rounding per image
    __device__ __forceinline__ void fma_from(float w, const float4 *__restrict__ p)
    {
        const float2 w2 = make_float2(w, w);
#pragma unroll
        for (int k = 0; k < NB4; ++k) {
            const float4 c = __ldg(p + k);
            const float2 lo = __ffma2_rn(w2, make_float2(c.x, c.y), make_float2(v[k].x, v[k].y));
            const float2 hi = __ffma2_rn(w2, make_float2(c.z, c.w), make_float2(v[k].z, v[k].w));
            v[k] = make_float4(lo.x, lo.y, hi.x, hi.y);
        }
    }
    // the same with the chunk's values already in registers
    __device__ __forceinline__ void fma_with(float w, const float4 (&c)[NB4])
    {
        const float2 w2 = make_float2(w, w);
#pragma unroll
        for (int k = 0; k < NB4; ++k) {
            const float2 lo = __ffma2_rn(w2, make_float2(c[k].x, c[k].y), make_float2(v[k].x, v[k].y));
            const float2 hi = __ffma2_rn(w2, make_float2(c[k].z, c[k].w), make_float2(v[k].z, v[k].w));
            v[k] = make_float4(lo.x, lo.y, hi.x, hi.y);
        }
    }
    __device__ __forceinline__ void add(const Acc &o)
    {
#pragma unroll
        for (int k = 0; k < NB4; ++k) {
            const float2 lo = __fadd2_rn(make_float2(v[k].x, v[k].y), make_float2(o.v[k].x, o.v[k].y));
            const float2 hi = __fadd2_rn(make_float2(v[k].z, v[k].w), make_float2(o.v[k].z, o.v[k].w));
            v[k] = make_float4(lo.x, lo.y, hi.x, hi.y);
        }
    }
};

// ------------------------------------------------------------------ forward
// KC candidates per line; KC = 0: R.kc of them (windows wider than 8 pixels, cells much
// wider than pixels).
template <int KC, int NB4, bool EXACT>
__device__ __forceinline__ void fp_batch_walk(const RayF &R, const float4 *__restrict__ base, int pitch4, float B,
                                              float q, float piC, float iC, float hC, Acc<NB4> &acc)
{
    long long A = R.A0 + 0xFFFFFFFFLL;   // ceil-ready: high word = ceil(f - hw)
    float er = R.e0;
    const int kc = KC > 0 ? KC : R.kc;
    Acc<NB4> part;
    part.zero();
    for (int rr = 0; rr < R.nrows; ++rr) {
        const int ilo = (int)(A >> 32);
        const float u0 = fmaf(__uint2float_rn((unsigned)A), -1.0f / 4294967296.0f, 1.0f) - R.hw;
        const float4 *rp = base + (long long)ilo * NB4;
#pragma unroll
        for (int m = 0; m < kc; ++m) {
            const float um = u0 + (float)m;
            const float e = fmaf(R.kap, um, er);
            const float d = wdiff<EXACT>(fabsf(B * um), e, q, piC, iC, hC);
            part.fma_from(d * rcp_approx(e), rp + m * NB4);
        }
        A += R.G;
        er += R.de;
        base += pitch4;
        if ((rr & 15) == 15) {
            acc.add(part);
            part.zero();
        }
    }
    acc.add(part);
}

// One ray's walk over its lines [l0, l1), a part of [R.r0, R.r0 + R.nrows), added to acc.
template <int NB4, bool EXACT>
__device__ __forceinline__ void fp_batch_walk_lines(RayF R, int l0, int l1, const float4 *__restrict__ P,
                                                    const float4 *__restrict__ Tt, int pitchP, int pitchT, int pad,
                                                    float B, float q, float piC, float iC, float hC, Acc<NB4> &acc)
{
    if (l1 <= l0) return;
    const int k = l0 - R.r0;
    R.A0 += (long long)k * R.G;
    R.e0 += (float)k * R.de;
    R.r0 = l0;
    R.nrows = l1 - l0;
    const bool tr = (R.flags & 1) != 0;
    const int pitch = tr ? pitchT : pitchP;
    const float4 *base = (tr ? Tt : P) + ((long long)R.r0 * pitch + pad) * NB4;
    const int p4 = pitch * NB4;
    switch (R.kc) {
        case 1: fp_batch_walk<1, NB4, EXACT>(R, base, p4, B, q, piC, iC, hC, acc); break;
        case 2: fp_batch_walk<2, NB4, EXACT>(R, base, p4, B, q, piC, iC, hC, acc); break;
        case 3: fp_batch_walk<3, NB4, EXACT>(R, base, p4, B, q, piC, iC, hC, acc); break;
        case 4: fp_batch_walk<4, NB4, EXACT>(R, base, p4, B, q, piC, iC, hC, acc); break;
        case 5: fp_batch_walk<5, NB4, EXACT>(R, base, p4, B, q, piC, iC, hC, acc); break;
        case 6: fp_batch_walk<6, NB4, EXACT>(R, base, p4, B, q, piC, iC, hC, acc); break;
        case 7: fp_batch_walk<7, NB4, EXACT>(R, base, p4, B, q, piC, iC, hC, acc); break;
        case 8: fp_batch_walk<8, NB4, EXACT>(R, base, p4, B, q, piC, iC, hC, acc); break;
        default: fp_batch_walk<0, NB4, EXACT>(R, base, p4, B, q, piC, iC, hC, acc); break;
    }
}

// Trapezoid constants of one ray (Eq. 16 widths): q, p/C, 1/C, C/2 and B = 2(q - C/2).
struct RayBox {
    float q, piC, iC, hC, B;
};

// Two adjacent rays of one view (cells j, j + 1) walking the same line family, over the
// lines both walk: on each line the candidates of the two windows' union are loaded once
// (the chunk's 16 NB4 bytes per candidate are what bounds this kernel) and evaluated for
// both rays.  A candidate outside one ray's own window lies outside its support, so its
// entry for that ray is exactly 0 (image pixels lie in front of the source, so tau'/2 > 0
// there; padding pixels are 0).  The union lies between the two windows, inside the padded
// line.
template <int NB4, bool EXACT>
__device__ __forceinline__ void fp_batch_walk_joint(const RayF &Ra, const RayF &Rb, const RayBox &Xa,
                                                    const RayBox &Xb, int j0, int j1, const float4 *__restrict__ base,
                                                    int p4, Acc<NB4> &acca, Acc<NB4> &accb)
{
    long long Aa = Ra.A0 + (long long)(j0 - Ra.r0) * Ra.G + 0xFFFFFFFFLL;   // ceil-ready states
    long long Ab = Rb.A0 + (long long)(j0 - Rb.r0) * Rb.G + 0xFFFFFFFFLL;
    float era = Ra.e0 + (float)(j0 - Ra.r0) * Ra.de, erb = Rb.e0 + (float)(j0 - Rb.r0) * Rb.de;
    Acc<NB4> parta, partb;
    parta.zero();
    partb.zero();
    for (int L = j0; L < j1; ++L) {
        const int ia = (int)(Aa >> 32), ib = (int)(Ab >> 32);
        const float ua0 = fmaf(__uint2float_rn((unsigned)Aa), -1.0f / 4294967296.0f, 1.0f) - Ra.hw;
        const float ub0 = fmaf(__uint2float_rn((unsigned)Ab), -1.0f / 4294967296.0f, 1.0f) - Rb.hw;
        const int lo = min(ia, ib), hi = max(ia + Ra.kc, ib + Rb.kc);
        for (int c = lo; c < hi; ++c) {
            float4 v[NB4];
#pragma unroll
            for (int k = 0; k < NB4; ++k) v[k] = __ldg(base + (long long)c * NB4 + k);
            const float ua = ua0 + (float)(c - ia), ub = ub0 + (float)(c - ib);
            const float ea = fmaf(Ra.kap, ua, era), eb = fmaf(Rb.kap, ub, erb);
            const float da = wdiff<EXACT>(fabsf(Xa.B * ua), ea, Xa.q, Xa.piC, Xa.iC, Xa.hC);
            const float db = wdiff<EXACT>(fabsf(Xb.B * ub), eb, Xb.q, Xb.piC, Xb.iC, Xb.hC);
            parta.fma_with(da * rcp_approx(ea), v);
            partb.fma_with(db * rcp_approx(eb), v);
        }
        Aa += Ra.G;
        Ab += Rb.G;
        era += Ra.de;
        erb += Rb.de;
        base += p4;
        if (((L - j0) & 15) == 15) {   // blocked summation: partial sums of 16 lines
            acca.add(parta);
            accb.add(partb);
            parta.zero();
            partb.zero();
        }
    }
    acca.add(parta);
    accb.add(partb);
}

// Two rays per thread: rays 2t and 2t + 1 of a block's 128 (64 threads), walked jointly
// over their common lines when they are adjacent cells of one view with the same walk axis,
// each alone over the rest of its lines; otherwise each alone.  The pairing does not depend
// on the batch, so neither does any image's result.
template <int NB4, bool EXACT>
__global__ void __launch_bounds__(64) fp_batch_kernel(const int *__restrict__ order, const RayF *__restrict__ rays,
                                                      const BoxF *__restrict__ box,
                                                      float h2q, const float4 *__restrict__ P,
                                                      const float4 *__restrict__ Tt, int pitchP, int pitchT,
                                                      int pad, int nr, int nd, float *__restrict__ sino, int b0,
                                                      int nb_used)
{
    const int q = order[blockIdx.x] * 128 + 2 * threadIdx.x;   // longest walks first
    if (q >= nr) return;
    const bool has1 = q + 1 < nr;
    RayF R[2];
    RayBox X[2];
    Acc<NB4> acc[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        R[s] = rays[s == 0 || !has1 ? q : q + 1];
        const float4 bx = __ldg(reinterpret_cast<const float4 *>(box + (s == 0 || !has1 ? q : q + 1)));
        X[s].q = bx.x; X[s].piC = bx.y; X[s].iC = bx.z; X[s].hC = bx.w;
        X[s].B = 2.f * (bx.x - bx.w);
        if (R[s].nrows > 0) tighten_window(R[s], X[s].q, X[s].B);
        acc[s].zero();
    }
    const int la0 = R[0].r0, la1 = R[0].r0 + max(R[0].nrows, 0);
    const int lb0 = R[1].r0, lb1 = R[1].r0 + max(R[1].nrows, 0);
    const int j0 = max(la0, lb0), j1 = min(la1, lb1);
    const bool joint = has1 && (q + 1) % nd != 0 && R[0].nrows > 0 && R[1].nrows > 0 &&
                       (R[0].flags & 1) == (R[1].flags & 1) && j0 < j1;
    if (joint) {
        // each ray alone before and after the common lines, then both together
        fp_batch_walk_lines<NB4, EXACT>(R[0], la0, j0, P, Tt, pitchP, pitchT, pad, X[0].B, X[0].q, X[0].piC, X[0].iC,
                                 X[0].hC, acc[0]);
        fp_batch_walk_lines<NB4, EXACT>(R[0], j1, la1, P, Tt, pitchP, pitchT, pad, X[0].B, X[0].q, X[0].piC, X[0].iC,
                                 X[0].hC, acc[0]);
        fp_batch_walk_lines<NB4, EXACT>(R[1], lb0, j0, P, Tt, pitchP, pitchT, pad, X[1].B, X[1].q, X[1].piC, X[1].iC,
                                 X[1].hC, acc[1]);
        fp_batch_walk_lines<NB4, EXACT>(R[1], j1, lb1, P, Tt, pitchP, pitchT, pad, X[1].B, X[1].q, X[1].piC, X[1].iC,
                                 X[1].hC, acc[1]);
        const bool tr = (R[0].flags & 1) != 0;
        const int pitch = tr ? pitchT : pitchP;
        const float4 *base = (tr ? Tt : P) + ((long long)j0 * pitch + pad) * NB4;
        fp_batch_walk_joint<NB4, EXACT>(R[0], R[1], X[0], X[1], j0, j1, base, pitch * NB4, acc[0], acc[1]);
    } else {
#pragma unroll
        for (int s = 0; s < 2; ++s)
            if ((s == 0 || has1) && R[s].nrows > 0)
                fp_batch_walk_lines<NB4, EXACT>(R[s], R[s].r0, R[s].r0 + R[s].nrows, P, Tt, pitchP, pitchT, pad, X[s].B,
                                         X[s].q, X[s].piC, X[s].iC, X[s].hC, acc[s]);
    }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        if (s == 1 && !has1) break;
        const float nrm = R[s].nrows > 0 ? h2q / (X[s].q - X[s].hC) : 0.f;
        const float *a = reinterpret_cast<const float *>(acc[s].v);
#pragma unroll
        for (int k = 0; k < 4 * NB4; ++k)
            if (k < nb_used) sino[(long long)(b0 + k) * nr + q + s] = a[k] * nrm;
    }
}

// ------------------------------------------------------------------ back
constexpr int BPB_T = 16;
constexpr int BPB_CHUNK = 256;
constexpr int BPB_THREADS = BPB_T * BPB_T / 2;   // one thread per pair of pixels

struct alignas(16) TileViewB {
    float Dt, yt, a1, b1, rho, phi, hc, hs;
};

// Two pixels per thread, rows r and r + 1 of one column (128 threads per 16 x 16 tile, a
// warp covering 8 x 8 pixels), gathered per view over the union of their cell windows:
// each cell's constants and the chunk's sinogram values are loaded once for both pixels (the
// loads, 16 + 16 + 16 NB4 bytes per lane and cell, are what bounds this kernel).  A cell of
// the union outside one pixel's own window lies outside its support: its entry is exactly 0.
// The pixel below takes the per-pixel values by one addition (D_n, y' and the numerator of
// sigma are affine in the offset).  Per-view sums are added to the accumulators in shared
// memory every 16 views (blocked summation), in the same order for every chunk size, so an
// image's result does not depend on the batch it is projected in.
template <int NB4, bool EXACT>
__global__ void __launch_bounds__(BPB_THREADS) bp_batch_kernel(GeomConsts g, const double *__restrict__ view_cs,
                                                               const float4 *__restrict__ box,
                                                               const float4 *__restrict__ cell,
                                                               const float4 *__restrict__ Y, float *__restrict__ img,
                                                               float kz, float ke, float h2, float h2q, int b0,
                                                               int nb_used, const int *__restrict__ order, int ntx,
                                                               float kscale, float dg, float nk6)
{
    __shared__ TileViewB tv[BPB_CHUNK];
    __shared__ int tj[BPB_CHUNK];
    __shared__ float4 accs[2 * NB4][BPB_THREADS];   // blocked-summation accumulators
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tx = (warp & 1) * 8 + (lane & 7), ty = (warp >> 1) * 8 + 2 * (lane >> 3);
    const int tile = order[blockIdx.x];   // heaviest tiles first
    const int it = (tile % ntx) * BPB_T, rt = (tile / ntx) * BPB_T;
    const int i = it + tx, r = rt + ty;
    const bool in0 = i < g.nx && r < g.ny, in1 = i < g.nx && r + 1 < g.ny;
    // reference point: the centre of the tile's part inside the image (in front of the source)
    const double refx = 0.5 * (min(BPB_T, g.nx - it) - 1), refy = 0.5 * (min(BPB_T, g.ny - rt) - 1);
    const float di = (float)(tx - refx), dr = (float)(ty - refy);
#pragma unroll
    for (int k = 0; k < 2 * NB4; ++k) accs[k][tid] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int v0 = 0; v0 < g.nv; v0 += BPB_CHUNK) {
        const int nvc = min(BPB_CHUNK, g.nv - v0);
        __syncthreads();
        for (int k = tid; k < nvc; k += BPB_THREADS) {
            double c = view_cs[2 * (v0 + k)], s = view_cs[2 * (v0 + k) + 1];
            double Dt, yt, a1, b1, rho, phi, hc, hs;
            int J;
            tile_view_double(g, c, s, it + refx, rt + refy, &Dt, &yt, &a1, &b1, &rho, &phi, &J, &hc, &hs);
            TileViewB T;
            T.Dt = (float)Dt; T.yt = (float)yt; T.a1 = (float)a1; T.b1 = (float)b1;
            T.rho = (float)rho; T.phi = (float)phi; T.hc = (float)hc; T.hs = (float)hs;
            tv[k] = T;
            tj[k] = J;
        }
        __syncthreads();
        if (!in0) continue;
        Acc<NB4> part0, part1;
        part0.zero();
        part1.zero();
        for (int vv = 0; vv < nvc; ++vv) {
            const TileViewB T = tv[vv];
            const int J = tj[vv];
            const long long vrow = (long long)(v0 + vv) * g.nd;
            const float Dn0 = fmaf(-T.hc, di, fmaf(-T.hs, dr, T.Dt));
            const float yp0 = fmaf(-T.hs, di, fmaf(T.hc, dr, T.yt));
            const float nu0 = g.arc ? fmaf(T.a1, di, T.b1 * dr) : fmaf(T.a1, di, fmaf(T.b1, dr, T.rho));
            const float Dn1 = Dn0 - T.hs, yp1 = yp0 + T.hc, nu1 = nu0 + T.b1;   // one row down
            const float rD0 = rcp_approx(Dn0), rD1 = rcp_approx(Dn1);
            // cell coordinate - J: perspective ratio (flat, parallel) or angle (arc detector)
            const float sig0 = g.arc ? fmaf(atan_small(nu0 * rcp_approx(fmaf(Dn0, T.Dt, yp0 * T.yt))), kscale, T.phi)
                                     : fmaf(nu0, rD0, T.phi);
            float sig1 = g.arc ? fmaf(atan_small(nu1 * rcp_approx(fmaf(Dn1, T.Dt, yp1 * T.yt))), kscale, T.phi)
                               : fmaf(nu1, rD1, T.phi);
            // arc: |s'| = R sin(dg d) ~ R dg d (1 - (dg d)^2/6)
            const float G0 = g.arc ? sqrtf(fmaf(Dn0, Dn0, yp0 * yp0)) * dg : 0.f;
            const float G1 = g.arc ? sqrtf(fmaf(Dn1, Dn1, yp1 * yp1)) * dg : 0.f;
            const float za0 = fmaf(yp0, T.hc, -Dn0 * T.hs), zb0 = fmaf(yp0, T.hs, Dn0 * T.hc);
            const float za1 = fmaf(yp1, T.hc, -Dn1 * T.hs), zb1 = fmaf(yp1, T.hs, Dn1 * T.hc);
            const float hwc0 = fmaf(kz * (fabsf(za0) + fabsf(zb0)) * rD0 * rD0, fmaf(h2, rD0, 1.02f), ke);
            float hwc1 = fmaf(kz * (fabsf(za1) + fabsf(zb1)) * rD1 * rD1, fmaf(h2, rD1, 1.02f), ke);
            if (!in1) { sig1 = sig0; hwc1 = hwc0; }   // a pixel below the image takes the window above
            const int jlo = max((int)ceilf(fminf(sig0 - hwc0, sig1 - hwc1)), -J);
            const int jhi = min((int)floorf(fmaxf(sig0 + hwc0, sig1 + hwc1)), g.nd - 1 - J);
            float d0 = sig0 - (float)jlo, d1 = sig1 - (float)jlo;
            for (int jl = jlo; jl <= jhi; ++jl) {
                const long long q = vrow + J + jl;
                const float4 A = __ldg(box + q);
                const float4 C = __ldg(cell + J + jl);
                float4 yv[NB4];
#pragma unroll
                for (int k = 0; k < NB4; ++k) yv[k] = __ldg(Y + q * NB4 + k);
                const float x0 = g.arc ? fabsf(G0 * d0 * fmaf(d0 * d0, nk6, 1.f)) : fabsf(Dn0 * C.x * d0);
                const float x1 = g.arc ? fabsf(G1 * d1 * fmaf(d1 * d1, nk6, 1.f)) : fabsf(Dn1 * C.x * d1);
                const float e0 = fmaf(Dn0, C.y, yp0 * C.z), e1 = fmaf(Dn1, C.y, yp1 * C.z);
                const float w0 = wdiff<EXACT>(x0, e0, A.x, A.y, A.z, A.w);
                const float w1 = wdiff<EXACT>(x1, e1, A.x, A.y, A.z, A.w);
                part0.fma_with(w0 * rcp_approx((A.x - A.w) * e0), yv);   // (B/2) tau'/2
                part1.fma_with(w1 * rcp_approx((A.x - A.w) * e1), yv);
                d0 -= 1.f;
                d1 -= 1.f;
            }
            if ((vv & 15) == 15 || vv == nvc - 1) {   // blocked summation over groups of 16 views
#pragma unroll
                for (int k = 0; k < NB4; ++k) {
                    float4 u = accs[k][tid], w = accs[NB4 + k][tid];
                    const float2 u0 = __fadd2_rn(make_float2(u.x, u.y), make_float2(part0.v[k].x, part0.v[k].y));
                    const float2 u1 = __fadd2_rn(make_float2(u.z, u.w), make_float2(part0.v[k].z, part0.v[k].w));
                    const float2 w0 = __fadd2_rn(make_float2(w.x, w.y), make_float2(part1.v[k].x, part1.v[k].y));
                    const float2 w1 = __fadd2_rn(make_float2(w.z, w.w), make_float2(part1.v[k].z, part1.v[k].w));
                    accs[k][tid] = make_float4(u0.x, u0.y, u1.x, u1.y);
                    accs[NB4 + k][tid] = make_float4(w0.x, w0.y, w1.x, w1.y);
                }
                part0.zero();
                part1.zero();
            }
        }
    }
    if (in0) {
#pragma unroll
        for (int k = 0; k < 4 * NB4; ++k) {
            if (k >= nb_used) continue;
            const float4 u = accs[k >> 2][tid], w = accs[NB4 + (k >> 2)][tid];
            const float a0 = (k & 3) == 0 ? u.x : (k & 3) == 1 ? u.y : (k & 3) == 2 ? u.z : u.w;
            const float a1 = (k & 3) == 0 ? w.x : (k & 3) == 1 ? w.y : (k & 3) == 2 ? w.z : w.w;
            img[((long long)(b0 + k) * g.ny + r) * g.nx + i] = a0 * h2q;
            if (in1) img[((long long)(b0 + k) * g.ny + r + 1) * g.nx + i] = a1 * h2q;
        }
    }
}

// ------------------------------------------------------------------ launchers
static int chunk_nb4(int left) { return left > 8 ? 4 : (left > 4 ? 2 : 1); }

// Interleaved copies of a chunk of up to 16 images (both padded layouts).
size_t forward_batch_alloc_bytes(const cnsf_geometry *geo)
{
    const GeomConsts &g = geo->gc;
    const size_t per = (size_t)g.ny * (g.nx + 2 * geo->pad) + (size_t)g.nx * (g.ny + 2 * geo->pad);
    return per * 16 * sizeof(float);
}

// Interleaved copy of a chunk of up to 16 sinograms.
size_t back_batch_alloc_bytes(const cnsf_geometry *geo)
{
    return (size_t)geo->gc.nv * geo->gc.nd * 16 * sizeof(float);
}

int launch_forward_batch(const cnsf_geometry *geo, const float *img, float *sino, int batch, cudaStream_t st)
{
    const GeomConsts &g = geo->gc;
    const int nr = g.nv * g.nd, pad = geo->pad;
    const int pitchP = g.nx + 2 * pad, pitchT = g.ny + 2 * pad;
    float *buf = nullptr;
    cudaError_t e = scratch_alloc((void **)&buf, forward_batch_alloc_bytes(geo), st);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? (record_cuda_error(e), CNSF_ERR_NOMEM) : record_cuda_error(e);
    for (int b0 = 0; b0 < batch;) {
        const int nb4 = chunk_nb4(batch - b0), NB = 4 * nb4, used = std::min(NB, batch - b0);
        float *P = buf, *Tt = buf + (size_t)g.ny * pitchP * NB;
        const long long nP = (long long)g.ny * pitchP * NB, nT = (long long)g.nx * pitchT * NB;
        pad_interleave_kernel<<<(unsigned)std::min<long long>((nP + 255) / 256, 8192), 256, 0, st>>>(
            img, P, g.nx, g.ny, pad, pitchP, b0, used, NB, 0);
        pad_interleave_kernel<<<(unsigned)std::min<long long>((nT + 255) / 256, 8192), 256, 0, st>>>(
            img, Tt, g.nx, g.ny, pad, pitchT, b0, used, NB, 1);
        dim3 blk(64), grd((nr + 127) / 128);   // two rays per thread, 128 per block
        const float h2q = (float)(0.25 * g.h * g.h);
        const float4 *P4 = reinterpret_cast<const float4 *>(P), *T4 = reinterpret_cast<const float4 *>(Tt);
        if (nb4 == 4)
            (geo->exact ? fp_batch_kernel<4, true> : fp_batch_kernel<4, false>)<<<grd, blk, 0, st>>>(geo->d_fp_order, geo->d_ray, geo->d_box, h2q, P4, T4, pitchP, pitchT, pad, nr, g.nd, sino, b0, used);
        else if (nb4 == 2)
            (geo->exact ? fp_batch_kernel<2, true> : fp_batch_kernel<2, false>)<<<grd, blk, 0, st>>>(geo->d_fp_order, geo->d_ray, geo->d_box, h2q, P4, T4, pitchP, pitchT, pad, nr, g.nd, sino, b0, used);
        else
            (geo->exact ? fp_batch_kernel<1, true> : fp_batch_kernel<1, false>)<<<grd, blk, 0, st>>>(geo->d_fp_order, geo->d_ray, geo->d_box, h2q, P4, T4, pitchP, pitchT, pad, nr, g.nd, sino, b0, used);
        b0 += used;
    }
    cudaFreeAsync(buf, st);
    e = cudaGetLastError();
    return e == cudaSuccess ? CNSF_OK : record_cuda_error(e);
}

int launch_back_batch(const cnsf_geometry *geo, const float *sino, float *img, int batch, cudaStream_t st)
{
    const GeomConsts &g = geo->gc;
    const long long nvd = (long long)g.nv * g.nd;
    float *buf = nullptr;
    cudaError_t e = scratch_alloc((void **)&buf, back_batch_alloc_bytes(geo), st);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? (record_cuda_error(e), CNSF_ERR_NOMEM) : record_cuda_error(e);
    const int ntx = (g.nx + BPB_T - 1) / BPB_T, nty = (g.ny + BPB_T - 1) / BPB_T;
    dim3 blk(BPB_THREADS), grd(ntx * nty);
    const float kz = (float)geo->bw.kz, ke = (float)geo->bw.ke, h2 = (float)(2.0 * g.h), h2q = (float)(0.25 * g.h * g.h);
    const double dgd = g.arc ? g.ds / g.dps : 0.0;
    const float kscale = (float)(g.arc ? g.dps / g.ds : 0.0), dg = (float)dgd, nk6 = (float)(-dgd * dgd / 6.0);
    const float4 *box = reinterpret_cast<const float4 *>(geo->d_box), *cell = reinterpret_cast<const float4 *>(geo->d_cellf);
    for (int b0 = 0; b0 < batch;) {
        const int nb4 = chunk_nb4(batch - b0), NB = 4 * nb4, used = std::min(NB, batch - b0);
        sino_interleave_kernel<<<(unsigned)std::min<long long>((nvd * NB + 255) / 256, 8192), 256, 0, st>>>(
            sino, buf, nvd, b0, used, NB);
        const float4 *Y = reinterpret_cast<const float4 *>(buf);
        if (nb4 == 4)
            (geo->exact ? bp_batch_kernel<4, true> : bp_batch_kernel<4, false>)<<<grd, blk, 0, st>>>(g, geo->d_view_cs, box, cell, Y, img, kz, ke, h2, h2q, b0, used, geo->d_bp_order, ntx, kscale, dg, nk6);
        else if (nb4 == 2)
            (geo->exact ? bp_batch_kernel<2, true> : bp_batch_kernel<2, false>)<<<grd, blk, 0, st>>>(g, geo->d_view_cs, box, cell, Y, img, kz, ke, h2, h2q, b0, used, geo->d_bp_order, ntx, kscale, dg, nk6);
        else
            (geo->exact ? bp_batch_kernel<1, true> : bp_batch_kernel<1, false>)<<<grd, blk, 0, st>>>(g, geo->d_view_cs, box, cell, Y, img, kz, ke, h2, h2q, b0, used, geo->d_bp_order, ntx, kscale, dg, nk6);
        b0 += used;
    }
    cudaFreeAsync(buf, st);
    e = cudaGetLastError();
    return e == cudaSuccess ? CNSF_OK : record_cuda_error(e);
}

}  // namespace cnsf
