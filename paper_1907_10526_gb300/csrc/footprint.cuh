// footprint.cuh -- device evaluation of the CNSF entry (Eq. 18).
//
// With B >= C the two footprint widths of Eq. (16) (h|n_a|, h|n_b|) and tau' = 2e the
// effective blur of Eq. (17), the blurred footprint is the three-direction box spline
// M_[B, C, 2e](s') = box_B * box_C * box_2e (Sec. III.A).  It is evaluated as the window
// average of the trapezoid T = box_B * box_C:
//
//   M(x) = (G(x + e) - G(x - e)) / (2e),   G(y) = 1/2 + sgn(y) H(|y|),  H' = T,
//   B H(z) = min(z, p) + C/2 - (C/2) v(z)^2,   v(z) = sat((q - z)/C),
//
// with p = (B - C)/2, q = (B + C)/2.  The C/(2C) ramps carry their own factor C, so
// no step divides a difference by a small width: the 1/(zeta1 zeta2 tau') of the
// literal divided-difference form of Eq. (18) never appears, and C = 0 (axis-aligned
// rays, M_0 = delta) needs no branch (v is then 0 or 1).  window_diff returns
// B * 2e * M(x) for x = |s'|.
#pragma once

#include <cuda_runtime.h>

namespace cnsf {

__device__ __forceinline__ float sat01(float x) { return __saturatef(x); }
__device__ __forceinline__ double sat01(double x) { return fmin(fmax(x, 0.0), 1.0); }

template <typename T>
__device__ __forceinline__ T window_diff(T x, T e, T p, T qiC, T iC, T hC)
{
    T z1 = x + e;                 // >= 0
    T z0 = x - e;                 // either sign
    T a0 = fabs(z0);
    T m1 = fmin(z1, p);
    T m0 = fmin(a0, p);
    T v1 = sat01(fma(-z1, iC, qiC));
    T v0 = sat01(fma(-a0, iC, qiC));
    T h1 = fma(-hC * v1, v1, m1);          // B H(z1) - C/2
    T h0 = fma(-hC * v0, v0, m0) + hC;     // B H(|z0|)
    return (h1 + hC) - copysign(h0, z0);
}

}  // namespace cnsf
