// Dense direct summation (Eq. fastsum-sum) on the SIMT pipes, FP32, and the epilogue kernel
// that turns raw sums into messages / scaling updates.
//
// The kernel entry exp(-||x_i - y_j||^2 / eta) is formed on the fly: coordinates are in grid
// units, so the exponent is c * r^2 with c = -log2(e) / eta_u and the exponential is the
// hardware ex2 (MUFU).  Each CTA owns 512 targets (2 per thread) and one slice of the sources,
// staged through shared memory; partial sums are added atomically.
#include "kernels.h"

namespace {

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

constexpr int DENSE_TPB = 256;
constexpr int DENSE_TGT = 2 * DENSE_TPB;   // targets per CTA
constexpr int DENSE_CHUNK = 1024;          // sources staged per round

template <int D>
__global__ void __launch_bounds__(DENSE_TPB) k_dense(const Task* __restrict__ tasks, Globals G, int ntb,
                                                     int nsplit) {
    __shared__ Task T;
    __shared__ FacCache fc;
    __shared__ float s_u[D][DENSE_CHUNK];
    __shared__ float s_v[DENSE_CHUNK];
    load_task(T, tasks + blockIdx.y);
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) task_resets(T, G, 0);
    if (T.alpha == nullptr) load_factors(fc, G.fac, T.sf0, T.snf);
    const int tb = blockIdx.x % ntb, sp = blockIdx.x / ntb;
    const int Nt = T.tgt.n, Ns = T.src.n;
    const int i0 = tb * DENSE_TGT + threadIdx.x, i1 = i0 + DENSE_TPB;
    float xa[D], xb[D];
#pragma unroll
    for (int t = 0; t < D; ++t) {
        xa[t] = i0 < Nt ? T.tgt.u[t * Nt + i0] : 0.f;
        xb[t] = i1 < Nt ? T.tgt.u[t * Nt + i1] : 0.f;
    }
    const float c = -1.4426950408889634f / T.eta_u;
    const int chunk = (Ns + nsplit - 1) / nsplit;
    const int s0 = sp * chunk, s1 = min(Ns, s0 + chunk);
    // Two-level summation: FP32 partial sums over 16 sources, added to a compensated
    // (Kahan) FP32 accumulator, so the rounding error does not grow with the source count.
    float acc0 = 0.f, acc1 = 0.f, cmp0 = 0.f, cmp1 = 0.f;
    for (int base = s0; base < s1; base += DENSE_CHUNK) {
        const int cnt = min(DENSE_CHUNK, s1 - base);
        for (int q = threadIdx.x; q < cnt; q += DENSE_TPB) {
            const int j = base + q;
#pragma unroll
            for (int t = 0; t < D; ++t) s_u[t][q] = T.src.u[t * Ns + j];
            s_v[q] = T.alpha ? T.alpha[j] : eval_prod(fc, j);
        }
        __syncthreads();
        for (int q0 = 0; q0 < cnt; q0 += 16) {
            const int qe = min(cnt, q0 + 16);
            float p0 = 0.f, p1 = 0.f;
#pragma unroll 4
            for (int q = q0; q < qe; ++q) {
                float da = 0.f, db = 0.f;
#pragma unroll
                for (int t = 0; t < D; ++t) {
                    const float y = s_u[t][q];
                    const float ea = xa[t] - y, eb = xb[t] - y;
                    da = fmaf(ea, ea, da);
                    db = fmaf(eb, eb, db);
                }
                const float v = s_v[q];
                p0 = fmaf(v, ex2_approx(c * da), p0);
                p1 = fmaf(v, ex2_approx(c * db), p1);
            }
            float y0 = p0 - cmp0, t0 = acc0 + y0;
            cmp0 = (t0 - acc0) - y0;
            acc0 = t0;
            float y1 = p1 - cmp1, t1 = acc1 + y1;
            cmp1 = (t1 - acc1) - y1;
            acc1 = t1;
        }
        __syncthreads();
    }
    if (s0 < s1) {
        if (i0 < Nt) atomicAdd(&T.raw[i0], acc0);
        if (i1 < Nt) atomicAdd(&T.raw[i1], acc1);
    }
}

// Epilogue over raw sums (dense path) or with raw = 1 (node steps).  Zeroes raw after use.
__global__ void __launch_bounds__(256) k_epi(const Task* __restrict__ tasks, Globals G) {
    __shared__ Task T;
    __shared__ FacCache fc, tf;
    __shared__ double sLsrc;
    __shared__ EpiConst sC;
    __shared__ EpiPre sP;
    load_task(T, tasks + blockIdx.y);
    __syncthreads();
    load_task_consts(T, G, fc, tf, sP, sC, sLsrc);
    __syncthreads();
    const double Lsrc = sLsrc;
    const EpiConst C = sC;
    EpiPartial ep;
    epi_zero(ep);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < T.tgt.n; i += gridDim.x * blockDim.x) {
        float raw = 1.f;
        if (T.raw) {
            raw = T.raw[i];
            T.raw[i] = 0.f;
        }
        epilogue_point(T, tf, C, G.floor_, i, raw, ep);
    }
    epi_block_finish(T, G, tf, Lsrc, ep, sP.iter, C);
}

}  // namespace

cudaError_t launch_dense(int d, const Task* tasks, int ntask, int ntb, int nsplit, const Globals& G,
                         cudaStream_t st) {
    if (ntask <= 0) return cudaSuccess;
    dim3 grid(ntb * nsplit, ntask);
    switch (d) {
    case 1: k_dense<1><<<grid, DENSE_TPB, 0, st>>>(tasks, G, ntb, nsplit); break;
    case 2: k_dense<2><<<grid, DENSE_TPB, 0, st>>>(tasks, G, ntb, nsplit); break;
    default: k_dense<3><<<grid, DENSE_TPB, 0, st>>>(tasks, G, ntb, nsplit); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_epi(int d, const Task* tasks, int ntask, int grid_x, const Globals& G, cudaStream_t st) {
    (void)d;
    if (ntask <= 0) return cudaSuccess;
    k_epi<<<dim3(grid_x, ntask), 256, 0, st>>>(tasks, G);
    return cudaGetLastError();
}
