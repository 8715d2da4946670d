// NFFT-based fast summation kernels (Section 5, Algorithm 4) for sm_103a.
//
//   spread  : g[l]  = sum_j v_j psi(u_j - l)             (adjoint NFFT gridding, Eq. ndft*)
//   fftconv : h     = IFFT( D . FFT(g) ),  D = w kappa_hat / Psi^2 on |k_t| <= M   (Eq. fastsum_mat)
//   gather  : beta_i = sum_l h[l] psi(u_i - l)           (NFFT interpolation, Eq. ndft)
//
// Points are binned into tiles of the periodic grid; one CTA handles one subproblem (<= P
// points of one tile) and accumulates into a padded tile in shared memory, which is then added
// to the L2-resident grid.  The window has 2m+2 = 10 taps per dimension.
#include "kernels.h"
#include "fft_smem.cuh"

namespace {

constexpr unsigned FULL = 0xffffffffu;

template <int D>
__device__ __forceinline__ void tile_origin(int tile, int ntd, int TS, int* o) {
#pragma unroll
    for (int t = 0; t < D; ++t) {
        o[t] = (tile % ntd) * TS - MOT_WHALF;
        tile /= ntd;
    }
}

template <int D>
__device__ __forceinline__ int tile_to_global(int idx, int P, const int* o, int n) {
    int g = 0, stride = 1;
#pragma unroll
    for (int t = 0; t < D; ++t) {
        int lt = idx % P;
        idx /= P;
        g += wrap_idx(o[t] + lt, n) * stride;
        stride *= n;
    }
    return g;
}

// ------------------------------------------------------------------------------------------
// spread
// ------------------------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(256) k_spread(const Task* __restrict__ tasks, Globals G, int bump_iter) {
    __shared__ Task T;
    __shared__ FacCache fc;
    extern __shared__ float tile[];
    if (threadIdx.x == 0) T = tasks[blockIdx.y];
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) task_resets(T, G, bump_iter && blockIdx.y == 0);
    if (T.alpha == nullptr) load_factors(fc, G.fac, T.sf0, T.snf);

    const int n = G.n_grid;
    const int TS = mot_tile_size(D, n), P = TS + MOT_W - 1, ntd = n / TS;
    int npad = P;
    if (D >= 2) npad *= P;
    if (D >= 3) npad *= P;
    const int N = T.src.n;
    const int nsub = *T.src.nsub;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;

    for (int s = blockIdx.x; s < nsub; s += gridDim.x) {
        const Sub sb = T.src.subs[s];
        int o[3];
        tile_origin<D>(sb.tile, ntd, TS, o);
        for (int i = threadIdx.x; i < npad; i += blockDim.x) tile[i] = 0.f;
        __syncthreads();
        const int j1 = sb.start + sb.len;
        if (D == 1) {
            for (int j = sb.start + threadIdx.x; j < j1; j += blockDim.x) {
                const float v = T.alpha ? T.alpha[j] : eval_prod(fc, j);
                const float u = T.src.u[j];
                const float fl = floorf(u);
                const int b0 = (int)fl - MOT_WHALF - o[0];
#pragma unroll
                for (int a = 0; a < MOT_W; ++a)
                    atomicAdd(&tile[b0 + a], v * kb_window(u - (fl - MOT_WHALF + a)));
            }
        } else {
            for (int j = sb.start + warp; j < j1; j += nwarps) {
                const float v = T.alpha ? T.alpha[j] : eval_prod(fc, j);
                float wt[D];
                int b[D];
#pragma unroll
                for (int t = 0; t < D; ++t) {
                    const float u = T.src.u[t * N + j];
                    const float fl = floorf(u);
                    b[t] = (int)fl - MOT_WHALF - o[t];
                    wt[t] = lane < MOT_W ? kb_window(u - (fl - MOT_WHALF + lane)) : 0.f;
                }
#pragma unroll
                for (int it = 0; it < (MOT_W * MOT_W + 31) / 32; ++it) {
                    const int tap = it * 32 + lane;
                    const int a = tap % MOT_W;
                    const int bb = min(tap / MOT_W, MOT_W - 1);
                    const float wab = v * __shfl_sync(FULL, wt[0], a) * __shfl_sync(FULL, wt[1], bb);
                    const bool ok = tap < MOT_W * MOT_W;
                    if (D == 2) {
                        if (ok) atomicAdd(&tile[(b[1] + bb) * P + b[0] + a], wab);
                    } else {
#pragma unroll
                        for (int c = 0; c < MOT_W; ++c) {
                            const float wc = __shfl_sync(FULL, wt[D - 1], c);
                            if (ok) atomicAdd(&tile[((b[D - 1] + c) * P + b[1] + bb) * P + b[0] + a], wab * wc);
                        }
                    }
                }
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < npad; i += blockDim.x) {
            const float val = tile[i];
            if (val != 0.f) atomicAdd(&T.grid[tile_to_global<D>(i, P, o, n)], val);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------------
// gather + epilogue
// ------------------------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(256) k_gather(const Task* __restrict__ tasks, Globals G) {
    __shared__ Task T;
    __shared__ FacCache tf;
    __shared__ double sLsrc;
    extern __shared__ float tile[];
    if (threadIdx.x == 0) T = tasks[blockIdx.y];
    __syncthreads();
    load_factors(tf, G.fac, T.tf0, T.tnf);
    if (threadIdx.x == 0) {
        double L = 0.0;
        if (T.alpha == nullptr)
            for (int f = 0; f < T.snf; ++f) L += factor_L(G.fac[T.sf0 + f]);
        sLsrc = L;
    }
    __syncthreads();
    const double Lsrc = sLsrc;
    EpiPartial ep;
    epi_zero(ep);

    if (T.hgrid == nullptr) {
        // node step without a kernel product (root update / root marginal)
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < T.tgt.n; i += gridDim.x * blockDim.x)
            epilogue_point(T, tf, Lsrc, G.floor_, i, 1.f, ep);
    } else {
        const int n = G.n_grid;
        const int TS = mot_tile_size(D, n), P = TS + MOT_W - 1, ntd = n / TS;
        int npad = P;
        if (D >= 2) npad *= P;
        if (D >= 3) npad *= P;
        const int N = T.tgt.n;
        const int nsub = *T.tgt.nsub;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
        for (int s = blockIdx.x; s < nsub; s += gridDim.x) {
            const Sub sb = T.tgt.subs[s];
            int o[3];
            tile_origin<D>(sb.tile, ntd, TS, o);
            for (int i = threadIdx.x; i < npad; i += blockDim.x) tile[i] = __ldg(&T.hgrid[tile_to_global<D>(i, P, o, n)]);
            __syncthreads();
            const int j1 = sb.start + sb.len;
            if (D == 1) {
                for (int j = sb.start + threadIdx.x; j < j1; j += blockDim.x) {
                    const float u = T.tgt.u[j];
                    const float fl = floorf(u);
                    const int b0 = (int)fl - MOT_WHALF - o[0];
                    float acc = 0.f;
#pragma unroll
                    for (int a = 0; a < MOT_W; ++a) acc += tile[b0 + a] * kb_window(u - (fl - MOT_WHALF + a));
                    epilogue_point(T, tf, Lsrc, G.floor_, j, acc, ep);
                }
            } else {
                for (int j = sb.start + warp; j < j1; j += nwarps) {
                    float wt[D];
                    int b[D];
#pragma unroll
                    for (int t = 0; t < D; ++t) {
                        const float u = T.tgt.u[t * N + j];
                        const float fl = floorf(u);
                        b[t] = (int)fl - MOT_WHALF - o[t];
                        wt[t] = lane < MOT_W ? kb_window(u - (fl - MOT_WHALF + lane)) : 0.f;
                    }
                    float acc = 0.f;
#pragma unroll
                    for (int it = 0; it < (MOT_W * MOT_W + 31) / 32; ++it) {
                        const int tap = it * 32 + lane;
                        const int a = tap % MOT_W;
                        const int bb = min(tap / MOT_W, MOT_W - 1);
                        const float wab = __shfl_sync(FULL, wt[0], a) * __shfl_sync(FULL, wt[1], bb);
                        const bool ok = tap < MOT_W * MOT_W;
                        if (D == 2) {
                            if (ok) acc += tile[(b[1] + bb) * P + b[0] + a] * wab;
                        } else {
#pragma unroll
                            for (int c = 0; c < MOT_W; ++c) {
                                const float wc = __shfl_sync(FULL, wt[D - 1], c);
                                if (ok) acc += tile[((b[D - 1] + c) * P + b[1] + bb) * P + b[0] + a] * (wab * wc);
                            }
                        }
                    }
                    acc = warp_sum(acc);
                    if (lane == 0) epilogue_point(T, tf, Lsrc, G.floor_, j, acc, ep);
                }
            }
            __syncthreads();
        }
    }
    epi_block_finish(T, G, tf, Lsrc, ep);
}

// ------------------------------------------------------------------------------------------
// FFT convolution with the spectral multiplier D
// ------------------------------------------------------------------------------------------
// D layouts (half spectrum in the first coordinate, k0 in [0, M]; other k_t in [-M, M]):
//   d=1: D[k0];  d=2: D[(k1+M)(M+1) + k0];  d=3: D[((k2+M)(2M+1) + k1+M)(M+1) + k0].
// D already carries the factor 2 for k0 >= 1 (the mirrored negative half) and the weight 1/2
// on each coordinate with |k_t| = M, so the real output is Re sum_{k0 >= 0} ... e^{+i...}.

__global__ void __launch_bounds__(256) k_fftconv1(const Task* __restrict__ tasks, int n, int logn, int M) {
    extern __shared__ float2 sm[];
    float2* A = sm;
    float2* A2 = sm + n;
    float2* tw = sm + 2 * n;
    const Task& T = tasks[blockIdx.x];
    float* g = T.grid;
    float* h = T.hgrid;
    const float* Dh = T.D;
    make_twiddles(tw, n);
    for (int x = threadIdx.x; x < n; x += blockDim.x) {
        float v = g[x];
        g[x] = 0.f;
        A[bitrev(x, logn)] = make_float2(v, 0.f);
    }
    __syncthreads();
    fft_rows(A, 1, n, logn, tw, 0);
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        float2 val = make_float2(0.f, 0.f);
        if (q <= M) {
            float dd = Dh[q];
            val = make_float2(A[q].x * dd, A[q].y * dd);
        }
        A2[bitrev(q, logn)] = val;
    }
    __syncthreads();
    fft_rows(A2, 1, n, logn, tw, 1);
    for (int x = threadIdx.x; x < n; x += blockDim.x) h[x] = A2[x].x;
}

// One CTA per task: the whole n x n grid (n <= 64) in shared memory.
__global__ void __launch_bounds__(256) k_fftconv2(const Task* __restrict__ tasks, int n, int logn, int M) {
    extern __shared__ float2 sm[];
    float2* A = sm;                       // n*n
    float2* B = sm + n * n;               // (M+1)*n
    float2* tw = B + (M + 1) * n;         // n/2
    const Task& T = tasks[blockIdx.x];
    float* g = T.grid;
    float* h = T.hgrid;
    const float* Dh = T.D;
    const int nn = n * n, mn = (M + 1) * n;
    make_twiddles(tw, n);
    for (int i = threadIdx.x; i < nn; i += blockDim.x) {
        float v = g[i];
        g[i] = 0.f;
        int y = i >> logn, x = i & (n - 1);
        A[(y << logn) + bitrev(x, logn)] = make_float2(v, 0.f);
    }
    __syncthreads();
    fft_rows(A, n, n, logn, tw, 0);                               // along x
    for (int i = threadIdx.x; i < mn; i += blockDim.x) {
        int kx = i >> logn, y = i & (n - 1);
        B[(kx << logn) + bitrev(y, logn)] = A[(y << logn) + kx];
    }
    __syncthreads();
    fft_rows(B, M + 1, n, logn, tw, 0);                           // along y
    for (int i = threadIdx.x; i < mn; i += blockDim.x) {
        int kx = i >> logn, kyi = i & (n - 1);
        int ky = kyi < (n >> 1) ? kyi : kyi - n;
        float2 val = make_float2(0.f, 0.f);
        if (ky >= -M && ky <= M) {
            float dd = Dh[(ky + M) * (M + 1) + kx];
            float2 b = B[i];
            val = make_float2(b.x * dd, b.y * dd);
        }
        A[(kx << logn) + bitrev(kyi, logn)] = val;
    }
    __syncthreads();
    fft_rows(A, M + 1, n, logn, tw, 1);                           // inverse along y
    for (int i = threadIdx.x; i < mn; i += blockDim.x) B[i] = A[i];
    __syncthreads();
    for (int i = threadIdx.x; i < nn; i += blockDim.x) {
        int y = i >> logn, q = i & (n - 1);
        int kx = bitrev(q, logn);
        A[i] = kx <= M ? B[(kx << logn) + y] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    fft_rows(A, n, n, logn, tw, 1);                               // inverse along x
    for (int i = threadIdx.x; i < nn; i += blockDim.x) h[i] = A[i].x;
}

// 3-D: planes z (x, y transforms) -> columns (z transform, multiply, inverse) -> planes.
// Intermediate spectrum layout: spec[(z*(2M+1) + ky+M)*(M+1) + kx].
__global__ void __launch_bounds__(256) k_fft3_xy_fwd(const Task* __restrict__ tasks, int n, int logn, int M) {
    extern __shared__ float2 sm[];
    float2* A = sm;
    float2* B = sm + n * n;
    float2* tw = B + (M + 1) * n;
    const Task& T = tasks[blockIdx.y];
    const int z = blockIdx.x;
    const int nn = n * n, mn = (M + 1) * n;
    float* g = T.grid + (size_t)z * nn;
    float2* spec = T.spec + (size_t)z * (2 * M + 1) * (M + 1);
    make_twiddles(tw, n);
    for (int i = threadIdx.x; i < nn; i += blockDim.x) {
        float v = g[i];
        g[i] = 0.f;
        int y = i >> logn, x = i & (n - 1);
        A[(y << logn) + bitrev(x, logn)] = make_float2(v, 0.f);
    }
    __syncthreads();
    fft_rows(A, n, n, logn, tw, 0);
    for (int i = threadIdx.x; i < mn; i += blockDim.x) {
        int kx = i >> logn, y = i & (n - 1);
        B[(kx << logn) + bitrev(y, logn)] = A[(y << logn) + kx];
    }
    __syncthreads();
    fft_rows(B, M + 1, n, logn, tw, 0);
    const int nky = 2 * M + 1;
    for (int i = threadIdx.x; i < nky * (M + 1); i += blockDim.x) {
        int kyo = i / (M + 1), kx = i - kyo * (M + 1);
        int ky = kyo - M;
        int kyi = ky < 0 ? ky + n : ky;
        spec[i] = B[(kx << logn) + kyi];
    }
}

#define FFT3_COLS 8
__global__ void __launch_bounds__(256) k_fft3_z(const Task* __restrict__ tasks, int n, int logn, int M) {
    extern __shared__ float2 sm[];
    float2* A = sm;                         // FFT3_COLS * n
    float2* A2 = sm + FFT3_COLS * n;        // FFT3_COLS * n
    float2* tw = A2 + FFT3_COLS * n;
    const Task& T = tasks[blockIdx.y];
    const int ncol = (2 * M + 1) * (M + 1);
    const int c0 = blockIdx.x * FFT3_COLS;
    float2* spec = T.spec;
    const float* Dh = T.D;
    make_twiddles(tw, n);
    for (int i = threadIdx.x; i < FFT3_COLS * n; i += blockDim.x) {
        int c = i >> logn, z = i & (n - 1);
        int col = c0 + c;
        A[(c << logn) + bitrev(z, logn)] = col < ncol ? spec[(size_t)z * ncol + col] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    fft_rows(A, FFT3_COLS, n, logn, tw, 0);
    for (int i = threadIdx.x; i < FFT3_COLS * n; i += blockDim.x) {
        int c = i >> logn, q = i & (n - 1);
        int col = c0 + c;
        int kz = q < (n >> 1) ? q : q - n;
        float2 val = make_float2(0.f, 0.f);
        if (col < ncol && kz >= -M && kz <= M) {
            float dd = Dh[(size_t)(kz + M) * ncol + col];
            val = make_float2(A[i].x * dd, A[i].y * dd);
        }
        A2[(c << logn) + bitrev(q, logn)] = val;
    }
    __syncthreads();
    fft_rows(A2, FFT3_COLS, n, logn, tw, 1);
    for (int i = threadIdx.x; i < FFT3_COLS * n; i += blockDim.x) {
        int c = i >> logn, z = i & (n - 1);
        int col = c0 + c;
        if (col < ncol) spec[(size_t)z * ncol + col] = A2[i];
    }
}

__global__ void __launch_bounds__(256) k_fft3_xy_inv(const Task* __restrict__ tasks, int n, int logn, int M) {
    extern __shared__ float2 sm[];
    float2* A = sm;
    float2* B = sm + n * n;
    float2* tw = B + (M + 1) * n;
    const Task& T = tasks[blockIdx.y];
    const int z = blockIdx.x;
    const int nn = n * n, mn = (M + 1) * n;
    float* h = T.hgrid + (size_t)z * nn;
    const float2* spec = T.spec + (size_t)z * (2 * M + 1) * (M + 1);
    make_twiddles(tw, n);
    for (int i = threadIdx.x; i < mn; i += blockDim.x) {
        int kx = i >> logn, kyi = i & (n - 1);
        int ky = kyi < (n >> 1) ? kyi : kyi - n;
        float2 val = make_float2(0.f, 0.f);
        if (ky >= -M && ky <= M) val = spec[(ky + M) * (M + 1) + kx];
        A[(kx << logn) + bitrev(kyi, logn)] = val;
    }
    __syncthreads();
    fft_rows(A, M + 1, n, logn, tw, 1);
    for (int i = threadIdx.x; i < mn; i += blockDim.x) B[i] = A[i];
    __syncthreads();
    for (int i = threadIdx.x; i < nn; i += blockDim.x) {
        int y = i >> logn, q = i & (n - 1);
        int kx = bitrev(q, logn);
        A[i] = kx <= M ? B[(kx << logn) + y] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    fft_rows(A, n, n, logn, tw, 1);
    for (int i = threadIdx.x; i < nn; i += blockDim.x) h[i] = A[i].x;
}

int ilog2(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

}  // namespace

int spread_smem_bytes(int d, int n) {
    int TS = mot_tile_size(d, n), P = TS + MOT_W - 1;
    int np = P;
    for (int i = 1; i < d; ++i) np *= P;
    return np * (int)sizeof(float);
}

cudaError_t launch_spread(int d, const Task* tasks, int ntask, int grid_x, const Globals& G, int bump_iter,
                          cudaStream_t st) {
    if (ntask <= 0) return cudaSuccess;
    dim3 grid(grid_x, ntask);
    int sm = spread_smem_bytes(d, G.n_grid);
    switch (d) {
    case 1: k_spread<1><<<grid, 256, sm, st>>>(tasks, G, bump_iter); break;
    case 2: k_spread<2><<<grid, 256, sm, st>>>(tasks, G, bump_iter); break;
    default: k_spread<3><<<grid, 256, sm, st>>>(tasks, G, bump_iter); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_gather(int d, const Task* tasks, int ntask, int grid_x, const Globals& G, cudaStream_t st) {
    if (ntask <= 0) return cudaSuccess;
    dim3 grid(grid_x, ntask);
    int sm = spread_smem_bytes(d, G.n_grid);
    switch (d) {
    case 1: k_gather<1><<<grid, 256, sm, st>>>(tasks, G); break;
    case 2: k_gather<2><<<grid, 256, sm, st>>>(tasks, G); break;
    default: k_gather<3><<<grid, 256, sm, st>>>(tasks, G); break;
    }
    return cudaGetLastError();
}

// Raise the dynamic shared-memory limit of a kernel once (never while a stream is captured).
template <class F>
cudaError_t ensure_smem(F* fn, size_t bytes, int* configured) {
    if (bytes <= 48 * 1024 || (int)bytes <= *configured) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) *configured = (int)bytes;
    return e;
}

size_t fftconv_smem(int d, int n) {
    const int M = n / 4;
    if (d == 1) return (size_t)(2 * n + n / 2) * sizeof(float2);
    return (size_t)(n * n + (M + 1) * n + n / 2) * sizeof(float2);
}

cudaError_t prepare_fftconv(int d, int n) {
    static int c1 = 0, c2 = 0, c3a = 0, c3b = 0;
    size_t sm = fftconv_smem(d, n);
    cudaError_t e = cudaSuccess;
    if (d == 1) e = ensure_smem(k_fftconv1, sm, &c1);
    else if (d == 2) e = ensure_smem(k_fftconv2, sm, &c2);
    else {
        e = ensure_smem(k_fft3_xy_fwd, sm, &c3a);
        if (e == cudaSuccess) e = ensure_smem(k_fft3_xy_inv, sm, &c3b);
    }
    return e;
}

cudaError_t launch_fftconv(int d, const Task* tasks, int ntask, const Globals& G, cudaStream_t st, int* nlaunch) {
    if (ntask <= 0) return cudaSuccess;
    const int n = G.n_grid, M = G.M, logn = ilog2(n);
    const size_t sm = fftconv_smem(d, n);
    if (d == 1) {
        k_fftconv1<<<ntask, 256, sm, st>>>(tasks, n, logn, M);
        if (nlaunch) *nlaunch += 1;
    } else if (d == 2) {
        k_fftconv2<<<ntask, 256, sm, st>>>(tasks, n, logn, M);
        if (nlaunch) *nlaunch += 1;
    } else {
        k_fft3_xy_fwd<<<dim3(n, ntask), 256, sm, st>>>(tasks, n, logn, M);
        const int ncol = (2 * M + 1) * (M + 1);
        size_t smz = (size_t)(2 * FFT3_COLS * n + n / 2) * sizeof(float2);
        k_fft3_z<<<dim3((ncol + FFT3_COLS - 1) / FFT3_COLS, ntask), 256, smz, st>>>(tasks, n, logn, M);
        k_fft3_xy_inv<<<dim3(n, ntask), 256, sm, st>>>(tasks, n, logn, M);
        if (nlaunch) *nlaunch += 3;
    }
    return cudaGetLastError();
}
