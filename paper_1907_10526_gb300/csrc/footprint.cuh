// footprint.cuh -- device evaluation of the CNSF entry (Eq. 18).
//
// With B >= C the two footprint widths of Eq. (16) (h|n_a|, h|n_b|) and tau' = 2e the
// effective blur of Eq. (17), the blurred footprint is the three-direction box spline
// M_[B, C, 2e](s') = box_B * box_C * box_2e (Sec. III.A).  It is evaluated as the window
// average of the trapezoid T = box_B * box_C:
//
//   M(x) = (G(x + e) - G(x - e)) / (2e),   G(y) = sgn(y) H(|y|),  H' = T,  H(0) = 0,
//   B H(z) = min(z, q) - (C/2) r(z)^2,   r(z) = sat((z - p)/C),
//
// with p = (B - C)/2, q = (B + C)/2 (the plateau and outer half-widths).  B H is the
// identity on the plateau, bends over the ramp and is B/2 beyond q.  The ramp term carries
// its own factor C, so no step divides a difference by a small width: the
// 1/(zeta1 zeta2 tau') of the literal divided-difference form of Eq. (18) never appears,
// and C = 0 (axis-aligned rays, M_0 = delta) needs no branch (r is then 0 or 1).  The one
// remaining difference G(x + e) - G(x - e) ~ 2e T(x) loses about log2(B / 2e) bits (a few
// at the blur widths of fan-beam CT; window_diff_exact below has no such loss).
// window_diff returns B * 2e * M(x) for x = |s'| from the constants q, p/C, 1/C and C/2.
#pragma once

#include <cuda_runtime.h>

namespace cnsf {

__device__ __forceinline__ float sat01(float x) { return __saturatef(x); }
__device__ __forceinline__ double sat01(double x) { return fmin(fmax(x, 0.0), 1.0); }

template <typename T>
__device__ __forceinline__ T window_diff(T x, T e, T q, T piC, T iC, T hC)
{
    T z1 = x + e;                 // >= 0
    T z0 = x - e;                 // either sign
    T a0 = fabs(z0);
    T r1 = sat01(fma(z1, iC, -piC));
    T r0 = sat01(fma(a0, iC, -piC));
    T h1 = fma(-hC * r1, r1, fmin(z1, q));   // B H(z1)
    T h0 = fma(-hC * r0, r0, fmin(a0, q));   // B H(|z0|)
    return h1 - copysign(h0, z0);
}

// 1/x by the hardware approximation (max error ~1 ulp); x is a blur half-width or a
// depth here, never denormal or huge, so the range handling of IEEE division is not needed.
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// arctan of a small ratio (the angle between a pixel's ray and its tile's reference ray):
// the Taylor (Gregory) series x - x^3/3 + x^5/5 - x^7/7 + x^9/9 for |x| < 1/8, where the
// first omitted term is below 1e-10 relative; atanf beyond.
__device__ __forceinline__ float atan_small(float x)
{
    const float t = x * x;
    if (!(t < 0.015625f)) return atanf(x);
    return x * fmaf(fmaf(fmaf(fmaf(t, 1.f / 9.f, -1.f / 7.f), t, 0.2f), t, -1.f / 3.f), t, 1.f);
}

// 32 bytes from global memory through the read-only path in one 256-bit load (sm_100+);
// p must be 32-byte aligned.
__device__ __forceinline__ void ldg256(const float *p, float (&r)[8])
{
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7])
        : "l"(p));
}

// Two entries at once with the packed FP32 instructions of sm_100+ (FADD2/FMUL2/FFMA2):
// the same arithmetic as window_diff, lane by lane, for candidates that share the
// trapezoid constants (q, p/C, 1/C given as scalars, -C/2 as a pair).  min, saturate and
// sign handling have no packed form and stay scalar.
__device__ __forceinline__ float2 window_diff2(float2 x, float2 e, float2 ne1, float q, float piC, float iC,
                                               float2 nhC2)
{
    const float2 z1 = __fadd2_rn(x, e);
    const float2 z0 = __ffma2_rn(e, ne1, x);          // x - e
    const float a0x = fabsf(z0.x), a0y = fabsf(z0.y);
    const float2 r1 = make_float2(sat01(fmaf(z1.x, iC, -piC)), sat01(fmaf(z1.y, iC, -piC)));
    const float2 r0 = make_float2(sat01(fmaf(a0x, iC, -piC)), sat01(fmaf(a0y, iC, -piC)));
    const float2 h1 = __ffma2_rn(__fmul2_rn(nhC2, r1), r1, make_float2(fminf(z1.x, q), fminf(z1.y, q)));
    const float2 h0 = __ffma2_rn(__fmul2_rn(nhC2, r0), r0, make_float2(fminf(a0x, q), fminf(a0y, q)));
    const float2 cs = make_float2(copysignf(h0.x, z0.x), copysignf(h0.y, z0.y));
    return __ffma2_rn(cs, ne1, h1);                   // B H(z1) - sgn(z0) B H(|z0|)
}

// Two entries with different trapezoid constants (cells j and j + 1), packed: q, p/C, 1/C
// and nhC = -C/2 are pairs.  Same arithmetic as window_diff, lane by lane.
__device__ __forceinline__ float2 window_diff2p(float2 x, float2 e, float2 ne1, float2 q, float2 piC, float2 iC,
                                                float2 nhC)
{
    const float2 z1 = __fadd2_rn(x, e);
    const float2 z0 = __ffma2_rn(e, ne1, x);          // x - e
    const float a0x = fabsf(z0.x), a0y = fabsf(z0.y);
    const float2 r1 = make_float2(sat01(fmaf(z1.x, iC.x, -piC.x)), sat01(fmaf(z1.y, iC.y, -piC.y)));
    const float2 r0 = make_float2(sat01(fmaf(a0x, iC.x, -piC.x)), sat01(fmaf(a0y, iC.y, -piC.y)));
    const float2 h1 = __ffma2_rn(__fmul2_rn(nhC, r1), r1, make_float2(fminf(z1.x, q.x), fminf(z1.y, q.y)));
    const float2 h0 = __ffma2_rn(__fmul2_rn(nhC, r0), r0, make_float2(fminf(a0x, q.x), fminf(a0y, q.y)));
    const float2 cs = make_float2(copysignf(h0.x, z0.x), copysignf(h0.y, z0.y));
    return __ffma2_rn(cs, ne1, h1);
}

// ---------------------------------------------------------------- exact window difference
// The same B * 2e * M(x) (x >= 0) without the cancellation: with G the odd extension of
// B H, G(z) = clamp(z, -q, q) - (C/2) (r+(z)^2 - r-(z)^2), r+(z) = sat((z - p)/C),
// r-(z) = sat((-z - p)/C), the difference over the window [z0, z1] = [x - e, x + e] is
//   G(z1) - G(z0) = L - (C/2) (dr (r+(z1) + r+(z0)) + r-(z0)^2)
// (r-(z1) = 0 for x >= 0), where L = |[z0, z1] n [-q, q]| = max(0, min(2e, 2q, (q - x) + e))
// and dr = r+(z1) - r+(z0) = max(0, min(2e/C, 1, 1 - (q - x)/C + e/C, (q - x)/C + e/C)), the
// clipped lengths written with the cut points relative to x.  Every term is formed from
// q - x, e and constants, none as the difference of two values of size B, so the result
// keeps ~1e-7 of 2e however thin the blur (the plain form loses log2(B / 2e) bits); the one
// subtraction left cancels only where the window leaves the footprint's ramp, and there the
// value itself is small.  About twice the instructions of window_diff.
template <typename T>
__device__ __forceinline__ T window_diff_exact(T x, T e, T q, T piC, T iC, T hC)
{
    const T one = T(1), zero = T(0);
    const T u = q - x;                                       // distance to the outer edge
    const T L = fmax(zero, fmin(fmin(e + e, q + q), u + e));
    const T ep = e * iC, v = u * iC;                         // e/C, (q - x)/C
    const T ope = one + ep;
    const T t1 = ope - v;                                    // (x + e - p)/C
    const T b = v + ep;                                      // (q - x + e)/C = 1 - (x - e - p)/C
    const T dr = fmax(zero, fmin(fmin(ep + ep, one), fmin(t1, b)));
    const T sr = sat01(t1) + sat01((one - ep) - v);          // r+(z1) + r+(z0)
    const T rm = sat01(ope - fma(x, iC, piC + one));         // r-(z0) = sat((e - x - p)/C)
    return fma(-hC, fma(dr, sr, rm * rm), L);
}

// Packed forms of window_diff_exact (shared constants; pair constants), lane by lane the
// same arithmetic.
__device__ __forceinline__ float2 window_diff2p_exact(float2 x, float2 e, float2 ne1, float2 q, float2 piC, float2 iC,
                                                      float2 nhC)
{
    const float2 one = make_float2(1.f, 1.f);
    const float2 u = __ffma2_rn(x, ne1, q);
    const float2 eu = __fadd2_rn(u, e), e2 = __fadd2_rn(e, e), q2 = __fadd2_rn(q, q);
    const float2 L = make_float2(fmaxf(0.f, fminf(fminf(e2.x, q2.x), eu.x)), fmaxf(0.f, fminf(fminf(e2.y, q2.y), eu.y)));
    const float2 ep = __fmul2_rn(e, iC), v = __fmul2_rn(u, iC);
    const float2 ope = __fadd2_rn(one, ep);
    const float2 t1 = __ffma2_rn(v, ne1, ope);
    const float2 b = __fadd2_rn(v, ep), ep2 = __fadd2_rn(ep, ep);
    const float2 dr = make_float2(fmaxf(0.f, fminf(fminf(ep2.x, 1.f), fminf(t1.x, b.x))),
                                  fmaxf(0.f, fminf(fminf(ep2.y, 1.f), fminf(t1.y, b.y))));
    const float2 t0 = __ffma2_rn(v, ne1, __ffma2_rn(ep, ne1, one));
    const float2 sr = __fadd2_rn(make_float2(sat01(t1.x), sat01(t1.y)), make_float2(sat01(t0.x), sat01(t0.y)));
    const float2 w = __ffma2_rn(x, iC, __fadd2_rn(piC, one));
    const float2 m = __ffma2_rn(w, ne1, ope);
    const float2 rm = make_float2(sat01(m.x), sat01(m.y));
    return __ffma2_rn(nhC, __ffma2_rn(rm, rm, __fmul2_rn(dr, sr)), L);
}

__device__ __forceinline__ float2 window_diff2_exact(float2 x, float2 e, float2 ne1, float q, float piC, float iC,
                                                     float2 nhC2)
{
    return window_diff2p_exact(x, e, ne1, make_float2(q, q), make_float2(piC, piC), make_float2(iC, iC), nhC2);
}

// The form a kernel instantiation uses: EXACT selects the cancellation-free differences.
template <bool EXACT, typename T>
__device__ __forceinline__ T wdiff(T x, T e, T q, T piC, T iC, T hC)
{
    return EXACT ? window_diff_exact(x, e, q, piC, iC, hC) : window_diff(x, e, q, piC, iC, hC);
}
template <bool EXACT>
__device__ __forceinline__ float2 wdiff2(float2 x, float2 e, float2 ne1, float q, float piC, float iC, float2 nhC2)
{
    return EXACT ? window_diff2_exact(x, e, ne1, q, piC, iC, nhC2) : window_diff2(x, e, ne1, q, piC, iC, nhC2);
}
template <bool EXACT>
__device__ __forceinline__ float2 wdiff2p(float2 x, float2 e, float2 ne1, float2 q, float2 piC, float2 iC, float2 nhC)
{
    return EXACT ? window_diff2p_exact(x, e, ne1, q, piC, iC, nhC) : window_diff2p(x, e, ne1, q, piC, iC, nhC);
}

}  // namespace cnsf
