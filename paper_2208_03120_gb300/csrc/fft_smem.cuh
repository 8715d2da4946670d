// Radix-2 complex FFT of power-of-two rows held in shared memory, done by a whole CTA.
// Used for the small oversampled grids of the fast summation (n = 16..4096 per dimension);
// the grids are L2-resident and the transforms are latency-, not bandwidth-bound.
#pragma once
#include "common.cuh"

__device__ __forceinline__ int bitrev(int x, int logn) {
    return (int)(__brev((unsigned int)x) >> (32 - logn));
}

// tw[k] = exp(-2 pi i k / L), k < L/2.
__device__ __forceinline__ void make_twiddles(float2* tw, int L) {
    for (int k = threadIdx.x; k < (L >> 1); k += blockDim.x) {
        float s, c;
        sincospif(2.f * (float)k / (float)L, &s, &c);
        tw[k] = make_float2(c, -s);
    }
}

// In-place decimation-in-time FFT of `nrows` rows of length L = 2^logL (row stride rs).
// Input rows must be in bit-reversed order; output is in natural order.
// inverse = 0: sum_l a_l e^{-2 pi i k l / L};  inverse = 1: sum_k a_k e^{+2 pi i k l / L} (unscaled).
__device__ __forceinline__ void fft_rows(float2* buf, int nrows, int rs, int logL, const float2* tw, int inverse) {
    const int L = 1 << logL;
    const int hb = L >> 1;
    const int nb = nrows * hb;
    for (int half = 1; half < L; half <<= 1) {
        const int tstep = L / (2 * half);
        for (int t = threadIdx.x; t < nb; t += blockDim.x) {
            int row = t >> (logL - 1);
            int j = t & (hb - 1);
            int pos = j & (half - 1);
            int i0 = ((j - pos) << 1) + pos;
            float2 w = tw[pos * tstep];
            if (inverse) w.y = -w.y;
            float2* r = buf + row * rs;
            float2 a = r[i0], b = r[i0 + half];
            float2 bw = make_float2(b.x * w.x - b.y * w.y, b.x * w.y + b.y * w.x);
            r[i0] = make_float2(a.x + bw.x, a.y + bw.y);
            r[i0 + half] = make_float2(a.x - bw.x, a.y - bw.y);
        }
        __syncthreads();
    }
}
