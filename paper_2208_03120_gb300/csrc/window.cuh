// Polynomial window taps of the fast summation (included by nfft.cu only, which defines c_win).
#pragma once
#include "common.cuh"

// Window taps.  The Kaiser-Bessel window normalised to 1 at 0,
//   psi(delta) = (a/r) sinh(b r) / sinh(a b),  r = sqrt(a^2 - delta^2),  |delta| <= a = m + 1,
// is evaluated at the 10 taps of a point with fractional grid position f = u - floor(u) by
// one degree-8 polynomial per tap, w_j = p_j(f) for delta = f + 4 - j (Horner); the
// coefficients interpolate psi at Chebyshev nodes (max error 2.8e-9, below FP32 rounding).
#define MOT_WDEG 8
__constant__ float c_win[MOT_W][MOT_WDEG + 1];

__device__ __forceinline__ void window_taps(float f, float* w) {
#pragma unroll
    for (int j = 0; j < MOT_W; ++j) {
        float p = c_win[j][MOT_WDEG];
#pragma unroll
        for (int k = MOT_WDEG - 1; k >= 0; --k) p = fmaf(p, f, c_win[j][k]);
        w[j] = p;
    }
}

