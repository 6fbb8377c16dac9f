// forward.cu -- forward projection y = A c (Eq. 6 with the entries of Eq. 18).
//
// Detector-driven gather, no atomics: one thread per (view, cell, image) walks the lines
// of the image that its central ray crosses most steeply and, on each line, the kc pixels
// whose footprint can reach the ray.  The crossing of line rb is carried in 32.32 fixed
// point (FP32 path), so the distance between ray and pixel centre keeps ~1e-7 pixel
// accuracy although the coordinates themselves are hundreds of millimetres.  The image is
// first copied into two zero-padded layouts -- rows for steep rays, the transpose for flat
// ones -- so that the candidates of one line are contiguous, adjacent cells of a warp read
// adjacent pixels, and no bounds test is needed inside the walk.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "cnsf_internal.cuh"
#include "cnsf_runtime.h"
#include "footprint.cuh"

namespace cnsf {

// ------------------------------------------------------------------ padded copies
template <typename T>
__global__ void pad_rows_kernel(const T *__restrict__ img, T *__restrict__ out, int nx, int ny, int pad,
                                int pitch, int ones)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    int r = blockIdx.y;
    long long b = blockIdx.z;
    if (c >= pitch) return;
    int i = c - pad;
    T v = T(0);
    if (i >= 0 && i < nx) v = ones ? T(1) : img[(b * ny + r) * nx + i];
    out[(b * ny + r) * pitch + c] = v;
}

template <typename T>
__global__ void pad_transpose_kernel(const T *__restrict__ img, T *__restrict__ out, int nx, int ny, int pad,
                                     int pitch, int ones)
{
    __shared__ T tile[32][33];
    long long b = blockIdx.z;
    int i0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
        int r = c0 - pad + yy, i = i0 + threadIdx.x;
        T v = T(0);
        if (r >= 0 && r < ny && i < nx) v = ones ? T(1) : img[(b * ny + r) * nx + i];
        tile[yy][threadIdx.x] = v;
    }
    __syncthreads();
    for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
        int i = i0 + yy, c = c0 + threadIdx.x;
        if (i < nx && c < pitch) out[(b * nx + i) * pitch + c] = tile[threadIdx.x][yy];
    }
}

// ------------------------------------------------------------------ FP32 walk
// One line of the walk with KC candidates, fully unrolled.  u is the signed a-offset
// (ia - f) of the first candidate.
template <int KC, bool COUNT, bool EXACT>
__device__ __forceinline__ float line_sum(const float *__restrict__ rp, float u, float er, float kap,
                                          float B, float q, float piC, float iC, float hC)
{
    float s = 0.f;
#pragma unroll
    for (int m = 0; m < KC; ++m) {
        float um = u + (float)m;
        float x = fabsf(B * um);
        float e = fmaf(kap, um, er);
        float c = __ldg(rp + m);
        if (COUNT) {
            // strictly inside the support |s'| < (B + C + tau')/2 of M_[B,C,tau']
            s += (x < q + e) ? c : 0.f;
        } else {
            float d = wdiff<EXACT>(x, e, q, piC, iC, hC);
            s = fmaf(c, d * rcp_approx(e), s);
        }
    }
    return s;
}

// Two consecutive lines of the walk at once with packed FP32 arithmetic: lane .x of every
// float2 belongs to line rb, lane .y to line rb + 1, and the KC candidates of both lines
// are evaluated pair by pair (no padding candidates).
template <int KC, bool EXACT>
__device__ __forceinline__ float2 line_pair_sum(const float *__restrict__ rp0, const float *__restrict__ rp1,
                                                float2 u, float2 er2, float2 kap2, float2 B2, float2 ne1,
                                                float q, float piC, float iC, float2 nhC2)
{
    float2 s = make_float2(0.f, 0.f);
    // B u and tau'/2 grow by B and kap per candidate
    float2 xs = __fmul2_rn(B2, u), e = __ffma2_rn(kap2, u, er2);
#pragma unroll
    for (int m = 0; m < KC; ++m) {
        const float2 x = make_float2(fabsf(xs.x), fabsf(xs.y));
        const float2 d = wdiff2<EXACT>(x, e, ne1, q, piC, iC, nhC2);
        const float2 w = __fmul2_rn(d, make_float2(rcp_approx(e.x), rcp_approx(e.y)));
        const float2 c = make_float2(__ldg(rp0 + m), __ldg(rp1 + m));
        s = __ffma2_rn(c, w, s);
        xs = __fadd2_rn(xs, B2);
        e = __fadd2_rn(e, kap2);
    }
    return s;
}

// The walk state is Bc = A + 2^32 - 1, A the 32.32 fixed point of f - hw: its high word is
// the first candidate ilo = ceil(f - hw) and its low word l gives rho = ilo - (f - hw) =
// 1 - (l + 1)/2^32 (to 2^-32; 0 when f - hw is an integer), so a line's window costs no
// ALU-pipe instruction: the high word is a register of the pair, the low word goes through
// an integer-to-float conversion (XU pipe) and one FMA.
__device__ __forceinline__ void fx_window(long long Bc, int &ilo, float &rho)
{
    ilo = (int)(Bc >> 32);
    rho = fmaf(__uint2float_rn((unsigned)Bc), -1.0f / 4294967296.0f, 1.0f);
}

template <int KC, bool EXACT>
__device__ __forceinline__ float walk2(const RayF &R, const float *__restrict__ base, int pitch, float B,
                                       float q, float piC, float iC, float hC)
{
    long long A = R.A0 + 0xFFFFFFFFLL;   // ceil-ready walk state (fx_window)
    const long long G = R.G;
    float2 er2 = make_float2(R.e0, R.e0 + R.de);
    const float2 de2 = make_float2(2.f * R.de, 2.f * R.de), kap2 = make_float2(R.kap, R.kap);
    const float2 B2 = make_float2(B, B), ne1 = make_float2(-1.0f, -1.0f);
    const float2 nhC2 = make_float2(-hC, -hC);
    const float hw = R.hw;
    float2 acc = make_float2(0.f, 0.f), part = make_float2(0.f, 0.f);
    int rr = 0;
    for (; rr + 1 < R.nrows; rr += 2) {
        int ilo0, ilo1;
        float rho0, rho1;
        fx_window(A, ilo0, rho0);
        fx_window(A + G, ilo1, rho1);
        const float2 u = make_float2(rho0 - hw, rho1 - hw);
        part = __fadd2_rn(part, line_pair_sum<KC, EXACT>(base + ilo0, base + pitch + ilo1, u, er2, kap2, B2, ne1, q,
                                                  piC, iC, nhC2));
        A += 2 * G;
        er2 = __fadd2_rn(er2, de2);
        base += 2 * pitch;
        if ((rr & 15) == 14) {   // blocked summation: partial sums of 16 lines
            acc = __fadd2_rn(acc, part);
            part = make_float2(0.f, 0.f);
        }
    }
    acc = __fadd2_rn(acc, part);
    float tot = acc.x + acc.y;
    if (rr < R.nrows) {   // odd line count: the last line alone
        int ilo;
        float rho;
        fx_window(A, ilo, rho);
        tot += line_sum<KC, false, EXACT>(base + ilo, rho - hw, er2.x, R.kap, B, q, piC, iC, hC);
    }
    return tot;
}

template <int KC, bool COUNT, bool EXACT>
__device__ __forceinline__ float walk(const RayF &R, const float *__restrict__ base, int pitch, float B,
                                      float q, float piC, float iC, float hC)
{
    long long A = R.A0;
    float er = R.e0;
    float acc = 0.f, part = 0.f;
    const float hw = R.hw, kap = R.kap, de = R.de;
    const long long G = R.G;
    for (int rr = 0; rr < R.nrows; ++rr) {
        // first candidate ilo = ceil(f - hw); rho = ilo - (f - hw) in [0, 1) from the low word
        int ilo = (int)(A >> 32) + (((unsigned)A) != 0u ? 1 : 0);
        unsigned nl = 0u - (unsigned)A;
        float rho = __uint_as_float(0x3f800000u | (nl >> 9)) - 1.0f;
        part += line_sum<KC, COUNT, EXACT>(base + ilo, rho - hw, er, kap, B, q, piC, iC, hC);
        A += G;
        er += de;
        base += pitch;
        if ((rr & 15) == 15) {  // blocked summation: partial sums of 16 lines
            acc += part;
            part = 0.f;
        }
    }
    return acc + part;
}

template <bool COUNT, bool EXACT>
__global__ void __launch_bounds__(128) fp_f32_kernel(const int *__restrict__ order, const RayF *__restrict__ rays,
                                                     const BoxF *__restrict__ box, float h2q,
                                                     const float *__restrict__ imgP, const float *__restrict__ imgT,
                                                     int pitchP, int pitchT, long long strideP, long long strideT,
                                                     int pad, int nr, float *__restrict__ sino, int nsplit,
                                                     float *__restrict__ partial)
{
    // blocks of 128 rays in the geometry's launch order (longest walks first)
    int q = order[blockIdx.x] * 128 + threadIdx.x;
    if (q >= nr) return;
    long long b = blockIdx.y;
    RayF R = rays[q];
    // blockIdx.z: which part of the ray's lines this block walks (parts summed afterwards in
    // a fixed order)
    if (nsplit > 1) {
        const int l0 = (int)((long long)R.nrows * blockIdx.z / nsplit), l1 = (int)((long long)R.nrows * (blockIdx.z + 1) / nsplit);
        R.A0 += (long long)l0 * R.G;
        R.e0 += (float)l0 * R.de;
        R.r0 += l0;
        R.nrows = l1 - l0;
    }
    float acc = 0.f;
    if (R.nrows > 0) {
        const float4 bx = __ldg(reinterpret_cast<const float4 *>(box + q));
        const float qw = bx.x, piC = bx.y, iC = bx.z, hC = bx.w;
        const float B = 2.f * (qw - hC);
        tighten_window(R, qw, B);
        const bool tr = (R.flags & 1) != 0;
        const int pitch = tr ? pitchT : pitchP;
        const float *base = (tr ? imgT + b * strideT : imgP + b * strideP) + pad + (long long)R.r0 * pitch;
        const int kcase = COUNT ? R.kc : 100 + R.kc;
        switch (kcase) {
            case 1: acc = walk<1, COUNT, EXACT>(R, base, pitch, B, qw, piC, iC, hC); break;
            case 2: acc = walk<2, COUNT, EXACT>(R, base, pitch, B, qw, piC, iC, hC); break;
            case 3: acc = walk<3, COUNT, EXACT>(R, base, pitch, B, qw, piC, iC, hC); break;
            case 4: acc = walk<4, COUNT, EXACT>(R, base, pitch, B, qw, piC, iC, hC); break;
            case 5: acc = walk<5, COUNT, EXACT>(R, base, pitch, B, qw, piC, iC, hC); break;
            case 6: acc = walk<6, COUNT, EXACT>(R, base, pitch, B, qw, piC, iC, hC); break;
            case 7: acc = walk<7, COUNT, EXACT>(R, base, pitch, B, qw, piC, iC, hC); break;
            case 8: acc = walk<8, COUNT, EXACT>(R, base, pitch, B, qw, piC, iC, hC); break;
            case 101: acc = walk2<1, EXACT>(R, base, pitch, B, qw, piC, iC, hC); break;
            case 102: acc = walk2<2, EXACT>(R, base, pitch, B, qw, piC, iC, hC); break;
            case 103: acc = walk2<3, EXACT>(R, base, pitch, B, qw, piC, iC, hC); break;
            case 104: acc = walk2<4, EXACT>(R, base, pitch, B, qw, piC, iC, hC); break;
            case 105: acc = walk2<5, EXACT>(R, base, pitch, B, qw, piC, iC, hC); break;
            case 106: acc = walk2<6, EXACT>(R, base, pitch, B, qw, piC, iC, hC); break;
            case 107: acc = walk2<7, EXACT>(R, base, pitch, B, qw, piC, iC, hC); break;
            case 108: acc = walk2<8, EXACT>(R, base, pitch, B, qw, piC, iC, hC); break;
            default: {
                // wide windows (cells much wider than pixels): generic loop
                long long A = R.A0;
                float er = R.e0;
                for (int rr = 0; rr < R.nrows; ++rr) {
                    int ilo = (int)(A >> 32) + (((unsigned)A) != 0u ? 1 : 0);
                    unsigned nl = 0u - (unsigned)A;
                    float u = (__uint_as_float(0x3f800000u | (nl >> 9)) - 1.0f) - R.hw;
                    for (int m = 0; m < R.kc; ++m, u += 1.0f) {
                        float e = fmaf(R.kap, u, er);
                        float x = fabsf(B * u);
                        float c = __ldg(base + ilo + m);
                        if (COUNT)
                            acc += (x < qw + e) ? c : 0.f;
                        else
                            acc += c * wdiff<EXACT>(x, e, qw, piC, iC, hC) * rcp_approx(e);
                    }
                    A += R.G;
                    er += R.de;
                    base += pitch;
                }
            }
        }
        if (!COUNT) acc *= h2q / (qw - hC);   // h^2/(2B), B = 2(q - C/2)
    }
    if (nsplit > 1)
        partial[((long long)blockIdx.z * gridDim.y + b) * nr + q] = acc;
    else
        sino[b * nr + q] = acc;
}

// sino = sum over the line parts, in part order (NS parts, every load issued at once)
template <int NS>
__global__ void fp_sum_parts_kernel(const float *__restrict__ partial, float *__restrict__ sino, long long n)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        float w[NS];
#pragma unroll
        for (int k = 0; k < NS; ++k) w[k] = __ldg(partial + k * n + t);
        float s = w[0];
#pragma unroll
        for (int k = 1; k < NS; ++k) s += w[k];
        sino[t] = s;
    }
}

// The part sum for the part counts of the launchers (powers of two up to 8).
static void launch_fp_sum_parts(const float *partial, float *sino, long long n, int nsplit, cudaStream_t st)
{
    const unsigned blocks = (unsigned)std::min<long long>((n + 255) / 256, 4096);
    switch (nsplit) {
        case 2: fp_sum_parts_kernel<2><<<blocks, 256, 0, st>>>(partial, sino, n); break;
        case 4: fp_sum_parts_kernel<4><<<blocks, 256, 0, st>>>(partial, sino, n); break;
        default: fp_sum_parts_kernel<8><<<blocks, 256, 0, st>>>(partial, sino, n); break;
    }
}

// ------------------------------------------------------------------ FP32 walk, four rotations
// A square image centred on the rotation axis, with views closed under a quarter turn
// (theta_{v + V/4} = theta_v + pi/2): the acquisition of view v + kV/4 is that of view v
// turned by k quarter turns (source, detector and cells alike, Sec. II.A), and a quarter
// turn maps the pixel lattice onto itself, pixel (i, r) to R(i, r) = (N-1-r, i), with the
// square pixel basis unchanged (the widths of Eq. 16 swap roles).  So every entry of Eq. (18)
// satisfies a(v + kV/4, j, n) = a(v, j, R^-k n), and
//     y[v + kV/4][j] = sum_m a(v, j, m) c[R^k m].
// One thread per ray of the first quarter of the views evaluates each entry once and applies
// it to the four values c4[m] = (c[m], c[Rm], c[R^2 m], c[R^3 m]) of an interleaved copy of
// the image, producing the four sinogram values at once.

// c4 in both zero-padded layouts (rows: P4[r][pad + i]; transposed: T4[i][pad + r]), through
// four 32 x 32 shared-memory tiles of the image (the rotated reads stay coalesced).
template <bool BATCH>
__global__ void pad_rot4_kernel(const float *__restrict__ img, float4 *__restrict__ P4, float4 *__restrict__ T4, int n,
                                int pad, int pitch)
{
    __shared__ float s[4][32][33];
    const int i0 = blockIdx.x * 32, r0 = blockIdx.y * 32, tx = threadIdx.x;
    if (BATCH) {   // image z of a batch: its own copies
        img += (long long)blockIdx.z * n * n;
        P4 += (long long)blockIdx.z * n * pitch;
        T4 += (long long)blockIdx.z * n * pitch;
    }
    auto at = [&](int row, int col) { return (row >= 0 && row < n && col >= 0 && col < n) ? img[(long long)row * n + col] : 0.f; };
    for (int a = threadIdx.y; a < 32; a += blockDim.y) {
        s[0][a][tx] = at(r0 + a, i0 + tx);                      // c[m]       = img[r][i]
        s[1][a][tx] = at(i0 + a, n - r0 - 32 + tx);             // c[R m]     = img[i][n-1-r]
        s[2][a][tx] = at(n - r0 - 32 + a, n - i0 - 32 + tx);    // c[R^2 m]   = img[n-1-r][n-1-i]
        s[3][a][tx] = at(n - i0 - 32 + a, r0 + tx);             // c[R^3 m]   = img[n-1-i][r]
    }
    __syncthreads();
    for (int a = threadIdx.y; a < 32; a += blockDim.y) {
        // rows layout: pixel (i0 + tx, r0 + a)
        if (i0 + tx < n && r0 + a < n)
            P4[(long long)(r0 + a) * pitch + pad + i0 + tx] =
                make_float4(s[0][a][tx], s[1][tx][31 - a], s[2][31 - a][31 - tx], s[3][31 - tx][a]);
        // transposed layout: pixel (i0 + a, r0 + tx)
        if (i0 + a < n && r0 + tx < n)
            T4[(long long)(i0 + a) * pitch + pad + r0 + tx] =
                make_float4(s[0][tx][a], s[1][a][31 - tx], s[2][31 - tx][31 - a], s[3][31 - a][tx]);
    }
    // the zero margins of the rows (and transposed rows) of this tile
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    const int tid = threadIdx.y * 32 + tx, nt = 32 * blockDim.y;
    if (blockIdx.x == 0 || blockIdx.x == gridDim.x - 1)
        for (int t = tid; t < 32 * pad; t += nt) {
            const int a = t / pad, c = t - a * pad;
            if (r0 + a >= n) continue;
            if (blockIdx.x == 0) P4[(long long)(r0 + a) * pitch + c] = z;
            if (blockIdx.x == gridDim.x - 1) P4[(long long)(r0 + a) * pitch + pad + n + c] = z;
        }
    if (blockIdx.y == 0 || blockIdx.y == gridDim.y - 1)
        for (int t = tid; t < 32 * pad; t += nt) {
            const int a = t / pad, c = t - a * pad;
            if (i0 + a >= n) continue;
            if (blockIdx.y == 0) T4[(long long)(i0 + a) * pitch + c] = z;
            if (blockIdx.y == gridDim.y - 1) T4[(long long)(i0 + a) * pitch + pad + n + c] = z;
        }
}

// The candidates of two consecutive lines, evaluated packed as in line_pair_sum, each entry
// applied to the four rotated values of its pixel as two packed pairs of neighbouring values
// (adjacent registers of the 16-byte load); s[i] accumulates rotations 2i and 2i + 1 over
// both lines.  KC = 0: kc candidates (wide cells).
template <int KC, bool EXACT>
__device__ __forceinline__ void line_pair_sum_rot4(const float4 *__restrict__ rp0, const float4 *__restrict__ rp1,
                                                   int kc, float2 u, float2 er2, float2 kap2, float2 B2, float2 ne1,
                                                   float q, float piC, float iC, float2 nhC2, float2 (&s)[2])
{
    float2 xs = __fmul2_rn(B2, u), e = __ffma2_rn(kap2, u, er2);
#pragma unroll
    for (int m = 0; m < (KC > 0 ? KC : kc); ++m) {
        const float2 x = make_float2(fabsf(xs.x), fabsf(xs.y));
        const float2 d = wdiff2<EXACT>(x, e, ne1, q, piC, iC, nhC2);
        const float2 w = __fmul2_rn(d, make_float2(rcp_approx(e.x), rcp_approx(e.y)));
        const float4 c0 = __ldg(rp0 + m), c1 = __ldg(rp1 + m);
        const float2 w0 = make_float2(w.x, w.x), w1 = make_float2(w.y, w.y);
        s[0] = __ffma2_rn(make_float2(c1.x, c1.y), w1, __ffma2_rn(make_float2(c0.x, c0.y), w0, s[0]));
        s[1] = __ffma2_rn(make_float2(c1.z, c1.w), w1, __ffma2_rn(make_float2(c0.z, c0.w), w0, s[1]));
        xs = __fadd2_rn(xs, B2);
        e = __fadd2_rn(e, kap2);
    }
}

// walk2 for the four rotations: two lines per packed step, blocked sums of 16 lines.
template <int KC, bool EXACT>
__device__ __forceinline__ void walk2_rot4(const RayF &R, const float4 *__restrict__ base, int pitch, float B,
                                           float q, float piC, float iC, float hC, float (&out)[4])
{
    long long A = R.A0 + 0xFFFFFFFFLL;   // ceil-ready walk state (fx_window)
    const long long G = R.G;
    const int kc = KC > 0 ? KC : R.kc;
    float2 er2 = make_float2(R.e0, R.e0 + R.de);
    const float2 de2 = make_float2(2.f * R.de, 2.f * R.de), kap2 = make_float2(R.kap, R.kap);
    const float2 B2 = make_float2(B, B), ne1 = make_float2(-1.0f, -1.0f), nhC2 = make_float2(-hC, -hC);
    const float hw = R.hw;
    float2 acc[2], part[2];   // rotations (0, 1) and (2, 3)
#pragma unroll
    for (int k = 0; k < 2; ++k) acc[k] = part[k] = make_float2(0.f, 0.f);
    int rr = 0;
    for (; rr + 1 < R.nrows; rr += 2) {
        int ilo0, ilo1;
        float rho0, rho1;
        fx_window(A, ilo0, rho0);
        fx_window(A + G, ilo1, rho1);
        line_pair_sum_rot4<KC, EXACT>(base + ilo0, base + pitch + ilo1, kc, make_float2(rho0 - hw, rho1 - hw), er2, kap2,
                               B2, ne1, q, piC, iC, nhC2, part);
        A += 2 * G;
        er2 = __fadd2_rn(er2, de2);
        base += 2 * pitch;
        if ((rr & 15) == 14) {   // blocked summation: partial sums of 16 lines
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                acc[k] = __fadd2_rn(acc[k], part[k]);
                part[k] = make_float2(0.f, 0.f);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        acc[k] = __fadd2_rn(acc[k], part[k]);
        out[2 * k] = acc[k].x;
        out[2 * k + 1] = acc[k].y;
    }
    if (rr < R.nrows) {   // odd line count: the last line alone
        int ilo;
        float rho;
        fx_window(A, ilo, rho);
        float um = rho - hw;
        for (int m = 0; m < kc; ++m, um += 1.0f) {
            const float e = fmaf(R.kap, um, er2.x);
            const float w = wdiff<EXACT>(fabsf(B * um), e, q, piC, iC, hC) * rcp_approx(e);
            const float4 c = __ldg(base + ilo + m);
            out[0] = fmaf(c.x, w, out[0]);
            out[1] = fmaf(c.y, w, out[1]);
            out[2] = fmaf(c.z, w, out[2]);
            out[3] = fmaf(c.w, w, out[3]);
        }
    }
}

// One thread per ray (v, j) of views v < V/4 (and line part): the four sinogram values
// y[v + kV/4][j], k = 0..3, written to rows v + kV/4 (nr4 = V/4 n_det rays apart).
template <bool EXACT, bool BATCH>
__global__ void __launch_bounds__(128) fp_rot4_f32_kernel(const int *__restrict__ order, const RayF *__restrict__ rays,
                                                          const BoxF *__restrict__ box, float h2q,
                                                          const float4 *__restrict__ imgP, const float4 *__restrict__ imgT,
                                                          int pitch, int pad, int nr, int nr4,
                                                          float *__restrict__ sino, int nsplit,
                                                          float *__restrict__ partial)
{
    const int q = order[blockIdx.x] * 128 + threadIdx.x;   // longest walks first
    if (q >= nr4) return;
    // image of a batch (one kernel and part order for every image); the single-image
    // instantiation carries no offsets (they cost the kernel its constant-bank addressing)
    const long long b = BATCH ? blockIdx.y : 0;
    if (BATCH) {
        imgP += b * (pitch - 2 * pad) * pitch;
        imgT += b * (pitch - 2 * pad) * pitch;
    }
    RayF R = rays[q];
    if (nsplit > 1) {
        const int l0 = (int)((long long)R.nrows * blockIdx.z / nsplit), l1 = (int)((long long)R.nrows * (blockIdx.z + 1) / nsplit);
        R.A0 += (long long)l0 * R.G;
        R.e0 += (float)l0 * R.de;
        R.r0 += l0;
        R.nrows = l1 - l0;
    }
    float out[4] = {0.f, 0.f, 0.f, 0.f};
    if (R.nrows > 0) {
        const float4 bx = __ldg(reinterpret_cast<const float4 *>(box + q));
        const float qw = bx.x, piC = bx.y, iC = bx.z, hC = bx.w;
        const float B = 2.f * (qw - hC);
        tighten_window(R, qw, B);
        const float4 *base = ((R.flags & 1) ? imgT : imgP) + pad + (long long)R.r0 * pitch;
        switch (R.kc) {
            case 1: walk2_rot4<1, EXACT>(R, base, pitch, B, qw, piC, iC, hC, out); break;
            case 2: walk2_rot4<2, EXACT>(R, base, pitch, B, qw, piC, iC, hC, out); break;
            case 3: walk2_rot4<3, EXACT>(R, base, pitch, B, qw, piC, iC, hC, out); break;
            case 4: walk2_rot4<4, EXACT>(R, base, pitch, B, qw, piC, iC, hC, out); break;
            case 5: walk2_rot4<5, EXACT>(R, base, pitch, B, qw, piC, iC, hC, out); break;
            case 6: walk2_rot4<6, EXACT>(R, base, pitch, B, qw, piC, iC, hC, out); break;
            case 7: walk2_rot4<7, EXACT>(R, base, pitch, B, qw, piC, iC, hC, out); break;
            case 8: walk2_rot4<8, EXACT>(R, base, pitch, B, qw, piC, iC, hC, out); break;
            default: walk2_rot4<0, EXACT>(R, base, pitch, B, qw, piC, iC, hC, out); break;
        }
        const float nrm = h2q / (qw - hC);   // h^2/(2B)
#pragma unroll
        for (int k = 0; k < 4; ++k) out[k] *= nrm;
    }
    float *dst = nsplit > 1 ? partial + ((long long)blockIdx.z * (BATCH ? gridDim.y : 1) + b) * nr : sino + b * nr;
#pragma unroll
    for (int k = 0; k < 4; ++k) dst[q + (long long)k * nr4] = out[k];
}

// ------------------------------------------------------------------ FP32 walk, rotations and reflections
// With a centred detector and views closed under theta -> -theta as well, the mirror image M
// of the acquisition of view k in the x axis is view -k with cell j at n_det - 1 - j, and M
// maps pixel (i, r) to (i, N-1-r): a(-k, n_det - 1 - j, M n) = a(k, j, n).  So for a ray
// (k, j) of the views k = 0 .. V/8,
//     y[k + mV/4][j]                = sum_q a(k, j, q) c[R^m q],
//     y[-k + mV/4][n_det - 1 - j]   = sum_q a(k, j, q) c[R^m M q],
// eight sinogram values from one walk over c8[q] = (c[R^m q], c[R^m M q]), m = 0..3 (32
// bytes per pixel).  Views k = 0 and k = V/8 (when V/8 is whole) are their own mirror images
// up to a quarter turn: their four rotation values are all they produce.

// c8 in both zero-padded layouts, 32 bytes per pixel (two float4), through eight 32 x 32
// shared-memory tiles of the image.
template <bool BATCH>
__global__ void pad_rot8_kernel(const float *__restrict__ img, float4 *__restrict__ P8, float4 *__restrict__ T8, int n,
                                int pad, int pitch)
{
    __shared__ float s[8][32][33];
    const int i0 = blockIdx.x * 32, r0 = blockIdx.y * 32, tx = threadIdx.x;
    if (BATCH) {   // image z of a batch: its own copies
        img += (long long)blockIdx.z * n * n;
        P8 += 2LL * blockIdx.z * n * pitch;
        T8 += 2LL * blockIdx.z * n * pitch;
    }
    auto at = [&](int row, int col) { return (row >= 0 && row < n && col >= 0 && col < n) ? img[(long long)row * n + col] : 0.f; };
    for (int a = threadIdx.y; a < 32; a += blockDim.y) {
        s[0][a][tx] = at(r0 + a, i0 + tx);                      // c[q]        = img[r][i]
        s[1][a][tx] = at(i0 + a, n - r0 - 32 + tx);             // c[R q]      = img[i][n-1-r]
        s[2][a][tx] = at(n - r0 - 32 + a, n - i0 - 32 + tx);    // c[R^2 q]    = img[n-1-r][n-1-i]
        s[3][a][tx] = at(n - i0 - 32 + a, r0 + tx);             // c[R^3 q]    = img[n-1-i][r]
        s[4][a][tx] = at(n - r0 - 32 + a, i0 + tx);             // c[M q]      = img[n-1-r][i]
        s[5][a][tx] = at(i0 + a, r0 + tx);                      // c[R M q]    = img[i][r]
        s[6][a][tx] = at(r0 + a, n - i0 - 32 + tx);             // c[R^2 M q]  = img[r][n-1-i]
        s[7][a][tx] = at(n - i0 - 32 + a, n - r0 - 32 + tx);    // c[R^3 M q]  = img[n-1-i][n-1-r]
    }
    __syncthreads();
    for (int a = threadIdx.y; a < 32; a += blockDim.y) {
        // rows layout: pixel (i0 + tx, r0 + a): ix = tx, ry = a
        if (i0 + tx < n && r0 + a < n) {
            float4 *o = P8 + 2 * ((long long)(r0 + a) * pitch + pad + i0 + tx);
            o[0] = make_float4(s[0][a][tx], s[1][tx][31 - a], s[2][31 - a][31 - tx], s[3][31 - tx][a]);
            o[1] = make_float4(s[4][31 - a][tx], s[5][tx][a], s[6][a][31 - tx], s[7][31 - tx][31 - a]);
        }
        // transposed layout: pixel (i0 + a, r0 + tx): ix = a, ry = tx
        if (i0 + a < n && r0 + tx < n) {
            float4 *o = T8 + 2 * ((long long)(i0 + a) * pitch + pad + r0 + tx);
            o[0] = make_float4(s[0][tx][a], s[1][a][31 - tx], s[2][31 - tx][31 - a], s[3][31 - a][tx]);
            o[1] = make_float4(s[4][31 - tx][a], s[5][a][tx], s[6][tx][31 - a], s[7][31 - a][31 - tx]);
        }
    }
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    const int tid = threadIdx.y * 32 + tx, nt = 32 * blockDim.y;
    if (blockIdx.x == 0 || blockIdx.x == gridDim.x - 1)
        for (int t = tid; t < 32 * pad; t += nt) {
            const int a = t / pad, c = t - a * pad;
            if (r0 + a >= n) continue;
            if (blockIdx.x == 0) { float4 *o = P8 + 2 * ((long long)(r0 + a) * pitch + c); o[0] = z; o[1] = z; }
            if (blockIdx.x == gridDim.x - 1) { float4 *o = P8 + 2 * ((long long)(r0 + a) * pitch + pad + n + c); o[0] = z; o[1] = z; }
        }
    if (blockIdx.y == 0 || blockIdx.y == gridDim.y - 1)
        for (int t = tid; t < 32 * pad; t += nt) {
            const int a = t / pad, c = t - a * pad;
            if (i0 + a >= n) continue;
            if (blockIdx.y == 0) { float4 *o = T8 + 2 * ((long long)(i0 + a) * pitch + c); o[0] = z; o[1] = z; }
            if (blockIdx.y == gridDim.y - 1) { float4 *o = T8 + 2 * ((long long)(i0 + a) * pitch + pad + n + c); o[0] = z; o[1] = z; }
        }
}

// line_pair_sum_rot4 with the eight values per pixel (one 256-bit load per candidate and
// line): the two lines' entries are evaluated packed, then each is applied to its pixel's
// eight values as four packed pairs of neighbouring values (the pairs a 256-bit load leaves
// in adjacent registers); s[i] accumulates values 2i and 2i + 1 over both lines.
template <int KC, bool EXACT>
__device__ __forceinline__ void line_pair_sum_rot8(const float *__restrict__ rp0, const float *__restrict__ rp1, int kc,
                                                   float2 u, float2 er2, float2 kap2, float2 B2, float2 ne1, float q,
                                                   float piC, float iC, float2 nhC2, float2 (&s)[4])
{
    float2 xs = __fmul2_rn(B2, u), e = __ffma2_rn(kap2, u, er2);
#pragma unroll
    for (int m = 0; m < (KC > 0 ? KC : kc); ++m) {
        const float2 x = make_float2(fabsf(xs.x), fabsf(xs.y));
        const float2 d = wdiff2<EXACT>(x, e, ne1, q, piC, iC, nhC2);
        const float2 w = __fmul2_rn(d, make_float2(rcp_approx(e.x), rcp_approx(e.y)));
        float c0[8], c1[8];
        ldg256(rp0 + 8 * m, c0);
        ldg256(rp1 + 8 * m, c1);
        const float2 w0 = make_float2(w.x, w.x), w1 = make_float2(w.y, w.y);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            s[i] = __ffma2_rn(make_float2(c0[2 * i], c0[2 * i + 1]), w0, s[i]);
            s[i] = __ffma2_rn(make_float2(c1[2 * i], c1[2 * i + 1]), w1, s[i]);
        }
        xs = __fadd2_rn(xs, B2);
        e = __fadd2_rn(e, kap2);
    }
}

template <int KC, bool EXACT>
__device__ __forceinline__ void walk2_rot8(const RayF &R, const float *__restrict__ base, int pitch8, float B, float q,
                                           float piC, float iC, float hC, float (&out)[8])
{
    long long A = R.A0 + 0xFFFFFFFFLL;   // ceil-ready walk state (fx_window)
    const long long G = R.G;
    const int kc = KC > 0 ? KC : R.kc;
    float2 er2 = make_float2(R.e0, R.e0 + R.de);
    const float2 de2 = make_float2(2.f * R.de, 2.f * R.de), kap2 = make_float2(R.kap, R.kap);
    const float2 B2 = make_float2(B, B), ne1 = make_float2(-1.0f, -1.0f), nhC2 = make_float2(-hC, -hC);
    const float hw = R.hw;
    // one sum per value, without the 16-line blocks of the other walks: the block registers
    // would cost resident warps, and a line part (an eighth of the ray's lines,
    // fp_line_parts_rot8) is short enough for plain FP32 sums
    float2 acc[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[i] = make_float2(0.f, 0.f);
    int rr = 0;
    for (; rr + 1 < R.nrows; rr += 2) {
        int ilo0, ilo1;
        float rho0, rho1;
        fx_window(A, ilo0, rho0);
        fx_window(A + G, ilo1, rho1);
        line_pair_sum_rot8<KC, EXACT>(base + 8LL * ilo0, base + pitch8 + 8LL * ilo1, kc,
                                      make_float2(rho0 - hw, rho1 - hw), er2, kap2, B2, ne1, q, piC, iC, nhC2, acc);
        A += 2 * G;
        er2 = __fadd2_rn(er2, de2);
        base += 2 * pitch8;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        out[2 * i] = acc[i].x;
        out[2 * i + 1] = acc[i].y;
    }
    if (rr < R.nrows) {   // odd line count: the last line alone
        int ilo;
        float rho;
        fx_window(A, ilo, rho);
        float um = rho - hw;
        for (int m = 0; m < kc; ++m, um += 1.0f) {
            const float e = fmaf(R.kap, um, er2.x);
            const float w = wdiff<EXACT>(fabsf(B * um), e, q, piC, iC, hC) * rcp_approx(e);
            float c[8];
            ldg256(base + 8LL * (ilo + m), c);
#pragma unroll
            for (int k = 0; k < 8; ++k) out[k] = fmaf(c[k], w, out[k]);
        }
    }
}

// One thread per ray (k, j) of the views k = 0 .. V/8 (and line part), blocks of FP8_VT views x
// FP8_CT cells: rotation values at rows k + mV/4, mirror values at rows -k + mV/4 (mod V),
// cell n_det - 1 - j.
template <bool EXACT, bool BATCH>
__global__ void __launch_bounds__(128) fp_rot8_f32_kernel(const int *__restrict__ order, const RayF *__restrict__ rays,
                                                          const BoxF *__restrict__ box, float h2q,
                                                          const float *__restrict__ imgP, const float *__restrict__ imgT,
                                                          int pitch, int pad, int nv, int nd,
                                                          float *__restrict__ sino, int nsplit,
                                                          float *__restrict__ partial)
{
    const int tile = order[blockIdx.x], ntc = fp8_cell_tiles(nd);   // blocks with the longest walks first
    const int k = (tile / ntc) * FP8_VT + threadIdx.x / FP8_CT, j = (tile % ntc) * FP8_CT + threadIdx.x % FP8_CT;
    if (k > nv / 8 || j >= nd) return;
    const int q = k * nd + j;
    const long long b = BATCH ? blockIdx.y : 0;   // image of a batch, as fp_rot4_f32_kernel
    if (BATCH) {
        imgP += 8 * b * (pitch - 2 * pad) * pitch;
        imgT += 8 * b * (pitch - 2 * pad) * pitch;
    }
    RayF R = rays[q];
    if (nsplit > 1) {
        const int l0 = (int)((long long)R.nrows * blockIdx.z / nsplit), l1 = (int)((long long)R.nrows * (blockIdx.z + 1) / nsplit);
        R.A0 += (long long)l0 * R.G;
        R.e0 += (float)l0 * R.de;
        R.r0 += l0;
        R.nrows = l1 - l0;
    }
    float out[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (R.nrows > 0) {
        const float4 bx = __ldg(reinterpret_cast<const float4 *>(box + q));
        const float qw = bx.x, piC = bx.y, iC = bx.z, hC = bx.w;
        const float B = 2.f * (qw - hC);
        tighten_window(R, qw, B);
        const float *base = ((R.flags & 1) ? imgT : imgP) + 8LL * (pad + (long long)R.r0 * pitch);
        const int pitch8 = 8 * pitch;
        switch (R.kc) {
            case 1: walk2_rot8<1, EXACT>(R, base, pitch8, B, qw, piC, iC, hC, out); break;
            case 2: walk2_rot8<2, EXACT>(R, base, pitch8, B, qw, piC, iC, hC, out); break;
            case 3: walk2_rot8<3, EXACT>(R, base, pitch8, B, qw, piC, iC, hC, out); break;
            case 4: walk2_rot8<4, EXACT>(R, base, pitch8, B, qw, piC, iC, hC, out); break;
            case 5: walk2_rot8<5, EXACT>(R, base, pitch8, B, qw, piC, iC, hC, out); break;
            case 6: walk2_rot8<6, EXACT>(R, base, pitch8, B, qw, piC, iC, hC, out); break;
            default: walk2_rot8<0, EXACT>(R, base, pitch8, B, qw, piC, iC, hC, out); break;
        }
        const float nrm = h2q / (qw - hC);   // h^2/(2B)
#pragma unroll
        for (int k = 0; k < 8; ++k) out[k] *= nrm;
    }
    float *dst = nsplit > 1 ? partial + ((long long)blockIdx.z * (BATCH ? gridDim.y : 1) + b) * nv * nd
                            : sino + b * nv * nd;
    const int v4 = nv >> 2;
    const bool self = k == 0 || 8 * k == nv;   // its own mirror image up to a quarter turn
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        dst[(long long)(k + m * v4) * nd + j] = out[m];
        if (!self) dst[(long long)((nv - k + m * v4) % nv) * nd + (nd - 1 - j)] = out[4 + m];
    }
}

// ------------------------------------------------------------------ FP64 walk
// Same enumeration (fixed-point windows of the ray table); the arithmetic, including the
// crossing f = f0 + rb g, is recomputed in FP64 from the view and cell angles.
__global__ void __launch_bounds__(128) fp_f64_kernel(GeomConsts g, const double *__restrict__ view_cs,
                                                     const RayF *__restrict__ rays,
                                                     const double *__restrict__ imgP,
                                                     const double *__restrict__ imgT, int pitchP, int pitchT,
                                                     long long strideP, long long strideT, int pad, int nr,
                                                     double *__restrict__ sino)
{
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nr) return;
    long long b = blockIdx.y;
    const RayF F = rays[q];
    double acc = 0.0;
    if (F.nrows > 0) {
        int k = q / g.nd, j = q - k * g.nd;
        RayParams<double> R = make_ray_params<double>(g, view_cs[2 * k], view_cs[2 * k + 1], j);
        BoxConsts<double> bc = make_box_consts<double>(R.B, R.C, g.h);
        const double hC = 0.5 * R.C, piC = bc.p * bc.iC;
        const bool tr = (F.flags & 1) != 0;
        const int pitch = tr ? pitchT : pitchP;
        const double *base = (tr ? imgT + b * strideT : imgP + b * strideP) + pad + (long long)F.r0 * pitch;
        long long A = F.A0;
        double part = 0.0;
        for (int rr = 0; rr < F.nrows; ++rr) {
            int rb = F.r0 + rr;
            int ilo = (int)(A >> 32) + (((unsigned)A) != 0u ? 1 : 0);
            double f = R.f0 + rb * R.g;
            double er = R.e0 + rb * R.de;
            for (int m = 0; m < F.kc; ++m) {
                double u = (double)(ilo + m) - f;
                double e = fma(R.kap, u, er);
                double d = window_diff(fabs(R.B * u), e, bc.q, piC, bc.iC, hC);
                part += base[ilo + m] * (d / e);
            }
            A += F.G;
            base += pitch;
            if ((rr & 15) == 15) {
                acc += part;
                part = 0.0;
            }
        }
        acc = (acc + part) * bc.nrm;
    }
    sino[b * nr + q] = acc;
}

// ------------------------------------------------------------------ launchers
template <typename T>
static int make_padded(const cnsf_geometry *geo, const T *img, int batch, int ones, cudaStream_t st, T **buf,
                       int *pitchP, int *pitchT, long long *strideP, long long *strideT)
{
    const GeomConsts &g = geo->gc;
    int pad = geo->pad;
    *pitchP = g.nx + 2 * pad;
    *pitchT = g.ny + 2 * pad;
    *strideP = (long long)g.ny * *pitchP;
    *strideT = (long long)g.nx * *pitchT;
    size_t elems = (size_t)batch * (size_t)(*strideP + *strideT);
    cudaError_t e = scratch_alloc((void **)buf, elems * sizeof(T), st);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? (record_cuda_error(e), CNSF_ERR_NOMEM) : record_cuda_error(e);
    T *P = *buf, *Tt = *buf + (size_t)batch * *strideP;
    dim3 blk(128), grd((*pitchP + 127) / 128, g.ny, batch);
    pad_rows_kernel<T><<<grd, blk, 0, st>>>(img, P, g.nx, g.ny, pad, *pitchP, ones);
    dim3 blk2(32, 8), grd2((*pitchT + 31) / 32, (g.nx + 31) / 32, batch);
    pad_transpose_kernel<T><<<grd2, blk2, 0, st>>>(img, Tt, g.nx, g.ny, pad, *pitchT, ones);
    return CNSF_OK;
}

// Line parts per ray of the FP32 single-image walk: several when the rays alone give fewer
// than 128 blocks (of 128 rays) per SM.
static int fp_line_parts(const cnsf_geometry *geo)
{
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, geo->device);
    const long long blocks = ((long long)geo->gc.nv * geo->gc.nd + 127) / 128;
    int nsplit = 1;
    while (nsplit < 4 && blocks * nsplit < 128LL * std::max(sms, 1)) nsplit *= 2;
    return nsplit;
}

// The same over the rays of the first quarter of the views (the four-rotation kernel).
static int fp_line_parts_rot4(const cnsf_geometry *geo)
{
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, geo->device);
    const long long blocks = ((long long)(geo->gc.nv / 4) * geo->gc.nd + 127) / 128;
    int nsplit = 1;
    while (nsplit < 8 && blocks * nsplit < 128LL * std::max(sms, 1)) nsplit *= 2;
    return nsplit;
}

// Line parts of the eight-value walk (views 0 .. V/8): always 8.  They fill the GPU (the
// base views alone give few rays) and keep each of the walk's unblocked sums to an eighth
// of a ray's lines.
static int fp_line_parts_rot8(const cnsf_geometry *)
{
    return 8;
}

// Bytes of one image's scratch on the eight-value path (its copies and part sums).
static size_t forward_rot8_image_bytes(const cnsf_geometry *geo)
{
    const GeomConsts &g = geo->gc;
    const int nsplit = fp_line_parts_rot8(geo);
    const size_t img8 = 2 * (size_t)g.nx * (g.nx + 2 * geo->pad) * 2 * sizeof(float4);
    return img8 + (nsplit > 1 ? (size_t)nsplit * g.nv * g.nd * sizeof(float) : 0);
}

static size_t forward_rot4_image_bytes(const cnsf_geometry *geo)
{
    const GeomConsts &g = geo->gc;
    const int nsplit = fp_line_parts_rot4(geo);
    const size_t img4 = 2 * (size_t)g.nx * (g.nx + 2 * geo->pad) * sizeof(float4);
    return img4 + (nsplit > 1 ? (size_t)nsplit * g.nv * g.nd * sizeof(float) : 0);
}

// FP32 forward projection of a batch by the eight-value kernel (geo->sym8): groups of
// sym_batch_group() images, each launch covering a group (one grid row per image).  Every
// image takes the kernel, line parts and part order of a single-image call, so its result
// does not depend on the batch or the group.
static int launch_forward_rot8(const cnsf_geometry *geo, const float *img, float *sino, int batch, cudaStream_t st)
{
    const GeomConsts &g = geo->gc;
    const int n = g.nx, pad = geo->pad, pitch = n + 2 * pad;
    const int nr = g.nv * g.nd;
    const int nsplit = fp_line_parts_rot8(geo);
    const size_t per = forward_rot8_image_bytes(geo);
    const int grp = sym_batch_group(per, batch);
    char *buf = nullptr;
    cudaError_t e = scratch_alloc((void **)&buf, (size_t)grp * per, st);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? (record_cuda_error(e), CNSF_ERR_NOMEM) : record_cuda_error(e);
    float4 *P8 = reinterpret_cast<float4 *>(buf), *T8 = P8 + 2 * (size_t)grp * n * pitch;
    float *partial = nsplit > 1 ? reinterpret_cast<float *>(T8 + 2 * (size_t)grp * n * pitch) : nullptr;
    const unsigned nt = (unsigned)((n + 31) / 32);
    for (int b0 = 0; b0 < batch; b0 += grp) {
        const int gb = std::min(grp, batch - b0);
        const float *im = img + (size_t)b0 * n * n;
        float *sn = sino + (size_t)b0 * nr;
        (gb > 1 ? pad_rot8_kernel<true> : pad_rot8_kernel<false>)<<<dim3(nt, nt, gb), dim3(32, 32), 0, st>>>(
            im, P8, T8, n, pad, pitch);
        auto kern = gb > 1 ? (geo->exact ? fp_rot8_f32_kernel<true, true> : fp_rot8_f32_kernel<false, true>)
                           : (geo->exact ? fp_rot8_f32_kernel<true, false> : fp_rot8_f32_kernel<false, false>);
        kern<<<dim3(fp8_blocks(g.nv, g.nd), gb, nsplit), 128, 0, st>>>(
            geo->d_fp_order8, geo->d_ray, geo->d_box, (float)(0.25 * g.h * g.h), reinterpret_cast<const float *>(P8),
            reinterpret_cast<const float *>(T8), pitch, pad, g.nv, g.nd, sn, nsplit, partial);
        if (nsplit > 1)
            launch_fp_sum_parts(partial, sn, (long long)gb * nr, nsplit, st);
    }
    cudaFreeAsync(buf, st);
    e = cudaGetLastError();
    return e == cudaSuccess ? CNSF_OK : record_cuda_error(e);
}

// FP32 forward projection of a batch by the four-rotation kernel (geo->sym), grouped as
// launch_forward_rot8.
static int launch_forward_rot4(const cnsf_geometry *geo, const float *img, float *sino, int batch, cudaStream_t st)
{
    const GeomConsts &g = geo->gc;
    const int n = g.nx, pad = geo->pad, pitch = n + 2 * pad;
    const int nr = g.nv * g.nd, nr4 = (g.nv / 4) * g.nd;
    const int nsplit = fp_line_parts_rot4(geo);
    const size_t per = forward_rot4_image_bytes(geo);
    const int grp = sym_batch_group(per, batch);
    char *buf = nullptr;
    cudaError_t e = scratch_alloc((void **)&buf, (size_t)grp * per, st);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? (record_cuda_error(e), CNSF_ERR_NOMEM) : record_cuda_error(e);
    float4 *P4 = reinterpret_cast<float4 *>(buf), *T4 = P4 + (size_t)grp * n * pitch;
    float *partial = nsplit > 1 ? reinterpret_cast<float *>(T4 + (size_t)grp * n * pitch) : nullptr;
    const unsigned nt = (unsigned)((n + 31) / 32);
    for (int b0 = 0; b0 < batch; b0 += grp) {
        const int gb = std::min(grp, batch - b0);
        const float *im = img + (size_t)b0 * n * n;
        float *sn = sino + (size_t)b0 * nr;
        (gb > 1 ? pad_rot4_kernel<true> : pad_rot4_kernel<false>)<<<dim3(nt, nt, gb), dim3(32, 32), 0, st>>>(
            im, P4, T4, n, pad, pitch);
        auto kern = gb > 1 ? (geo->exact ? fp_rot4_f32_kernel<true, true> : fp_rot4_f32_kernel<false, true>)
                           : (geo->exact ? fp_rot4_f32_kernel<true, false> : fp_rot4_f32_kernel<false, false>);
        kern<<<dim3((nr4 + 127) / 128, gb, nsplit), 128, 0, st>>>(
            geo->d_fp_order4, geo->d_ray, geo->d_box, (float)(0.25 * g.h * g.h), P4, T4, pitch, pad, nr, nr4, sn,
            nsplit, partial);
        if (nsplit > 1)
            launch_fp_sum_parts(partial, sn, (long long)gb * nr, nsplit, st);
    }
    cudaFreeAsync(buf, st);
    e = cudaGetLastError();
    return e == cudaSuccess ? CNSF_OK : record_cuda_error(e);
}

int launch_forward_sym(const cnsf_geometry *geo, const float *img, float *sino, int batch, cudaStream_t st)
{
    if (batch == 0) return CNSF_OK;
    if (geo->sym8) return launch_forward_rot8(geo, img, sino, batch, st);
    if (geo->sym) return launch_forward_rot4(geo, img, sino, batch, st);
    return CNSF_ERR_UNSUPPORTED;
}

size_t forward_alloc_bytes(const cnsf_geometry *geo, int batch, int dtype)
{
    if (batch <= 0) return 0;
    if (dtype == CNSF_F32 && geo->sym8)
        return (size_t)sym_batch_group(forward_rot8_image_bytes(geo), batch) * forward_rot8_image_bytes(geo);
    if (dtype == CNSF_F32 && geo->sym)
        return (size_t)sym_batch_group(forward_rot4_image_bytes(geo), batch) * forward_rot4_image_bytes(geo);
    if (dtype == CNSF_F32 && batch >= 2) return forward_batch_alloc_bytes(geo);
    size_t bytes = forward_scratch_bytes(geo, batch, dtype);   // padded copies
    if (dtype == CNSF_F32) {
        const int nsplit = fp_line_parts(geo);
        if (nsplit > 1) bytes += (size_t)nsplit * batch * geo->gc.nv * geo->gc.nd * sizeof(float);
    }
    return bytes;
}

int launch_forward(const cnsf_geometry *geo, const void *img, void *sino, int batch, int dtype, cudaStream_t st)
{
    if (batch == 0) return CNSF_OK;
    if (dtype == CNSF_F32 && (geo->sym8 || geo->sym))
        return launch_forward_sym(geo, (const float *)img, (float *)sino, batch, st);
    if (dtype == CNSF_F32 && batch >= 2) return launch_forward_batch(geo, (const float *)img, (float *)sino, batch, st);
    const GeomConsts &g = geo->gc;
    const int nr = g.nv * g.nd;
    int pitchP, pitchT;
    long long strideP, strideT;
    dim3 blk(128), grd((nr + 127) / 128, batch);
    if (dtype == CNSF_F32) {
        float *buf = nullptr;
        int s = make_padded<float>(geo, (const float *)img, batch, 0, st, &buf, &pitchP, &pitchT, &strideP, &strideT);
        if (s != CNSF_OK) return s;
        const int nsplit = fp_line_parts(geo);
        float *partial = nullptr;
        const long long nout = (long long)nr * batch;
        if (nsplit > 1) {
            cudaError_t e = scratch_alloc((void **)&partial, (size_t)nsplit * nout * sizeof(float), st);
            if (e != cudaSuccess) { cudaFreeAsync(buf, st); return record_cuda_error(e); }
        }
        (geo->exact ? fp_f32_kernel<false, true> : fp_f32_kernel<false, false>)<<<dim3(grd.x, grd.y, nsplit), blk, 0, st>>>(
            geo->d_fp_order, geo->d_ray, geo->d_box, (float)(0.25 * g.h * g.h), buf, buf + (size_t)batch * strideP,
            pitchP, pitchT, strideP, strideT, geo->pad, nr, (float *)sino, nsplit, partial);
        if (nsplit > 1) {
            launch_fp_sum_parts(partial, (float *)sino, nout, nsplit, st);
            cudaFreeAsync(partial, st);
        }
        cudaFreeAsync(buf, st);
    } else {
        double *buf = nullptr;
        int s = make_padded<double>(geo, (const double *)img, batch, 0, st, &buf, &pitchP, &pitchT, &strideP,
                                    &strideT);
        if (s != CNSF_OK) return s;
        fp_f64_kernel<<<grd, blk, 0, st>>>(g, geo->d_view_cs, geo->d_ray, buf, buf + (size_t)batch * strideP,
                                           pitchP, pitchT, strideP, strideT, geo->pad, nr, (double *)sino);
        cudaFreeAsync(buf, st);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? CNSF_OK : record_cuda_error(e);
}

// Forward projection whose padded copies go into a buffer the caller provides (no
// allocation).  Returns CNSF_ERR_UNSUPPORTED when the buffer is smaller than
// forward_scratch_bytes().
size_t forward_scratch_bytes(const cnsf_geometry *geo, int batch, int dtype)
{
    const GeomConsts &g = geo->gc;
    size_t per = (size_t)g.ny * (g.nx + 2 * geo->pad) + (size_t)g.nx * (g.ny + 2 * geo->pad);
    return (size_t)batch * per * (dtype == CNSF_F64 ? sizeof(double) : sizeof(float));
}

int launch_forward_with_scratch(const cnsf_geometry *geo, const void *img, void *sino, int batch, int dtype,
                                void *scratch, size_t scratch_bytes, cudaStream_t st)
{
    if (batch == 0) return CNSF_OK;
    if (forward_scratch_bytes(geo, batch, dtype) > scratch_bytes) return CNSF_ERR_UNSUPPORTED;
    const GeomConsts &g = geo->gc;
    const int nr = g.nv * g.nd, pad = geo->pad;
    const int pitchP = g.nx + 2 * pad, pitchT = g.ny + 2 * pad;
    const long long strideP = (long long)g.ny * pitchP, strideT = (long long)g.nx * pitchT;
    dim3 blk(128), grdr((pitchP + 127) / 128, g.ny, batch);
    dim3 blkt(32, 8), grdt((pitchT + 31) / 32, (g.nx + 31) / 32, batch);
    dim3 grd((nr + 127) / 128, batch);
    // FP32 on a geometry with the quarter-turn symmetry: the four-rotation walk with unsplit
    // lines, image by image in one image's four-rotation copies when they fit (each image
    // then takes exactly the arithmetic of a single-image call through this entry point)
    const size_t img4 = 2 * (size_t)g.nx * pitchP * sizeof(float4);
    if (dtype == CNSF_F32 && geo->sym && img4 <= scratch_bytes) {
        float4 *P4 = (float4 *)scratch, *T4 = P4 + (size_t)g.nx * pitchP;
        const int nr4 = (g.nv / 4) * g.nd;
        const unsigned nt = (unsigned)((g.nx + 31) / 32);
        auto kern = geo->exact ? fp_rot4_f32_kernel<true, false> : fp_rot4_f32_kernel<false, false>;
        for (int b = 0; b < batch; ++b) {
            pad_rot4_kernel<false><<<dim3(nt, nt), dim3(32, 32), 0, st>>>((const float *)img + (size_t)b * g.nx * g.ny,
                                                                       P4, T4, g.nx, pad, pitchP);
            kern<<<(nr4 + 127) / 128, 128, 0, st>>>(geo->d_fp_order4, geo->d_ray, geo->d_box, (float)(0.25 * g.h * g.h),
                                                    P4, T4, pitchP, pad, nr, nr4, (float *)sino + (size_t)b * nr, 1,
                                                    nullptr);
        }
        cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? CNSF_OK : record_cuda_error(e);
    }
    if (dtype == CNSF_F32) {
        float *P = (float *)scratch, *Tt = P + (size_t)batch * strideP;
        pad_rows_kernel<float><<<grdr, blk, 0, st>>>((const float *)img, P, g.nx, g.ny, pad, pitchP, 0);
        pad_transpose_kernel<float><<<grdt, blkt, 0, st>>>((const float *)img, Tt, g.nx, g.ny, pad, pitchT, 0);
        (geo->exact ? fp_f32_kernel<false, true> : fp_f32_kernel<false, false>)<<<grd, blk, 0, st>>>(geo->d_fp_order, geo->d_ray, geo->d_box, (float)(0.25 * g.h * g.h), P, Tt, pitchP, pitchT,
                                                  strideP, strideT, pad, nr, (float *)sino, 1, nullptr);
    } else {
        double *P = (double *)scratch, *Tt = P + (size_t)batch * strideP;
        pad_rows_kernel<double><<<grdr, blk, 0, st>>>((const double *)img, P, g.nx, g.ny, pad, pitchP, 0);
        pad_transpose_kernel<double><<<grdt, blkt, 0, st>>>((const double *)img, Tt, g.nx, g.ny, pad, pitchT, 0);
        fp_f64_kernel<<<grd, blk, 0, st>>>(g, geo->d_view_cs, geo->d_ray, P, Tt, pitchP, pitchT, strideP, strideT,
                                           pad, nr, (double *)sino);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? CNSF_OK : record_cuda_error(e);
}

// Non-zero entries: pairs strictly inside the support of M_[B, C, tau'], found by the
// forward walk over an image of ones (the zero padding contributes nothing).
int count_nonzeros(const cnsf_geometry *geo, uint64_t *count, cudaStream_t st)
{
    const GeomConsts &g = geo->gc;
    const int nr = g.nv * g.nd;
    int pitchP, pitchT;
    long long strideP, strideT;
    float *buf = nullptr, *out = nullptr;
    int s = make_padded<float>(geo, nullptr, 1, 1, st, &buf, &pitchP, &pitchT, &strideP, &strideT);
    if (s != CNSF_OK) return s;
    cudaError_t e = scratch_alloc((void **)&out, (size_t)nr * sizeof(float), st);
    if (e != cudaSuccess) { cudaFreeAsync(buf, st); return record_cuda_error(e); }
    dim3 blk(128), grd((nr + 127) / 128, 1);
    fp_f32_kernel<true, false><<<grd, blk, 0, st>>>(geo->d_fp_order, geo->d_ray, geo->d_box, (float)(0.25 * g.h * g.h), buf, buf + strideP, pitchP,
                                             pitchT, strideP, strideT, geo->pad, nr, out, 1, nullptr);
    std::vector<float> host(nr);
    e = cudaMemcpyAsync(host.data(), out, (size_t)nr * sizeof(float), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(buf, st);
    cudaFreeAsync(out, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return record_cuda_error(e);
    uint64_t tot = 0;
    for (int q = 0; q < nr; ++q) tot += (uint64_t)host[q];
    *count = tot;
    return CNSF_OK;
}

}  // namespace cnsf
