// Circle-structure kernels (Section 4.2, Algorithm 3).
//
// The matrices beta_k (n_k x n_1) and gamma_k^T (n_k x n_1) are stored column-major: column c
// (a point of the first marginal) is one contiguous vector of the node's points, so a matrix
// product with a kernel matrix is a batch of independent kernel matrix-vector products (one
// per column), done by the fast-summation or dense kernels.  The scaling updates need
//   rowdot: raw_i = sum_c beta_k[c][i] phi^1_c gamma_k^T[c][i]      (phi^k, k >= 2)
//   colsum: raw_c = sum_j K^{(2,1)}[c][j] phi^2_j beta_2[c][j]        (phi^1)
// with every factor taken as its normalised mantissa (divided by its maximum).  For d = 1 the
// batched fast summation of the message matrices (k_c1_spread / k_c1_gather) is here as well.
#include "kernels.h"

namespace {

// Partial row sums over a slice of the columns, added atomically (two-level compensated sum).
__global__ void __launch_bounds__(256) k_rowdot(const float* __restrict__ B, const VecScale* sB,
                                                const float* __restrict__ Gm, const VecScale* sG,
                                                const float* __restrict__ phi, const VecScale* sP, int ni, int nc,
                                                int nsplit, float* raw) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int chunk = (nc + nsplit - 1) / nsplit;
    const int c0 = blockIdx.y * chunk, c1 = min(nc, c0 + chunk);
    if (i >= ni || c0 >= c1) return;
    const float scale = (1.f / mx_of(sB, 0)) * (1.f / mx_of(sG, 0)) * (1.f / mx_of(sP, 0));
    float acc = 0.f, cmp = 0.f;
    for (int cb = c0; cb < c1; cb += 16) {
        const int ce = min(c1, cb + 16);
        float p = 0.f;
        if (ce - cb == 16) {        // 32 independent loads in flight
            float bv[16], gv[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                bv[u] = __ldg(B + (size_t)(cb + u) * ni + i);
                gv[u] = __ldg(Gm + (size_t)(cb + u) * ni + i);
            }
#pragma unroll
            for (int u = 0; u < 16; ++u) p = fmaf(bv[u] * gv[u], __ldg(phi + cb + u), p);
        } else {
            for (int c = cb; c < ce; ++c)
                p = fmaf(B[(size_t)c * ni + i] * Gm[(size_t)c * ni + i], __ldg(phi + c), p);
        }
        const float y = p - cmp, t = acc + y;
        cmp = (t - acc) - y;
        acc = t;
    }
    atomicAdd(raw + i, acc * scale);
}

// One block per column c: raw_c = sum_j A[c][j] B[c][j] phi_j.
__global__ void __launch_bounds__(256) k_colsum(const float* __restrict__ A, const VecScale* sA,
                                                const float* __restrict__ B, const VecScale* sB,
                                                const float* __restrict__ phi, const VecScale* sP, int nj,
                                                float* raw) {
    const int c = blockIdx.x;
    const float* a = A + (size_t)c * nj;
    const float* b = B + (size_t)c * nj;
    double acc = 0.0;
    float part = 0.f;
    int cnt = 0;
    for (int j = threadIdx.x; j < nj; j += blockDim.x) {
        part = fmaf(a[j] * b[j], __ldg(phi + j), part);
        if (++cnt == 16) {
            acc += part;
            part = 0.f;
            cnt = 0;
        }
    }
    acc += part;
    acc = warp_sum_d(acc);
    __shared__ double s[32];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) t += s[w];
        const float scale = (1.f / mx_of(sA, 0)) * (1.f / mx_of(sB, 0)) * (1.f / mx_of(sP, 0));
        raw[c] = (float)t * scale;
    }
}

// Dense kernel matrix, column-major: K[c][i] = exp(-||y_i - x_c||^2 / eta_u) (grid units).
__global__ void k_kernel_matrix(const float* __restrict__ ui, int ni, const float* __restrict__ uc, int nc, int d,
                                float eta_u, float* K, VecScale* sc) {
    const float k2 = -1.4426950408889634f / eta_u;
    const long long total = (long long)ni * nc;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(idx / ni), i = (int)(idx - (long long)c * ni);
        float r2 = 0.f;
        for (int t = 0; t < d; ++t) {
            const float e = ui[(size_t)t * ni + i] - uc[(size_t)t * nc + c];
            r2 = fmaf(e, e, r2);
        }
        K[idx] = exp2f(k2 * r2);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        sc->ls = 0.0;
        sc->mx_bits = __float_as_uint(1.f);
        sc->clamped = 0u;
        sc->ls_prev = 0.0;
        sc->mx_prev_bits = __float_as_uint(1.f);
    }
}

// Closing-edge points of the generalised Euler flow (Section 6.3): x_close (caller order,
// [n][d]) in node 1's sorted order and in grid units, u[t][j] = (x_close[perm[j]][t] - c_t) n / s
// + n/2.  Not wrapped onto the torus: the closing kernel matrix is formed directly.
__global__ void k_close_points(const float* __restrict__ x, const int* __restrict__ perm, int n, int d, double c0,
                               double c1, double c2, double inv_s, int n_grid, float* u, int* err) {
    const double c[3] = {c0, c1, c2};
    const double half = 0.5 * n_grid;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const size_t src = (size_t)perm[j] * d;
        for (int t = 0; t < d; ++t) {
            const float xf = x[src + t];
            if (!isfinite(xf)) atomicOr(err, 1);
            u[(size_t)t * n + j] = (float)(((double)xf - c[t]) * inv_s * n_grid + half);
        }
    }
}

// Pair marginal of a circle (Section 6.3): Pi[c][i] = phi^1_c Gam_k[c][i] beta_k[c][i] phi^k_i with
// every factor at its true scale (mantissa x exp(ls)), FP64, written row-major [n1][nk] in the
// caller's point order.  Gam_k and beta_k are column-major [c][i] in the sorted orders.
__global__ void k_pair(const float* __restrict__ phi1, const VecScale* s1, const int* __restrict__ perm1, int n1,
                       const float* __restrict__ phik, const VecScale* sk, const int* __restrict__ permk, int nk,
                       const float* __restrict__ G, const VecScale* sG, const float* __restrict__ B,
                       const VecScale* sB, double* out) {
    const double L = ls_of(s1, 0) + ls_of(sk, 0) + ls_of(sG, 0) + ls_of(sB, 0);
    const long long total = (long long)n1 * nk;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(idx / nk), i = (int)(idx - (long long)c * nk);
        const double p = (double)phi1[c] * (double)phik[i] * (double)G[idx] * (double)B[idx];
        out[(size_t)perm1[c] * nk + permk[i]] = p > 0.0 ? exp(log(p) + L) : 0.0;
    }
}


// ------------------------------------------------------------------------------------------
// Batched 1-D fast summation of the circle (Algorithm 3, N right-hand sides, d = 1).
//
// In one dimension the oversampled grid (n <= 128) is far smaller than the point sets, so a
// batch Y[c] = K (phi (.) X[c]), c < n0, runs as two passes over the message matrices:
//   k_c1_spread : G[c] = sum_j X[c][j] phi_j psi(u_j - .)   (32 columns per CTA, lane = column;
//                 the point's taps are the same for every column and are broadcast)
//   k_c1_gather : H[c] = C G[c] with the circulant C of Eq. (fastsum_mat) (c(m) = sum_{q<=M}
//                 D_q cos(2 pi q m / n), the real part of IFFT(D FFT(.))), then
//                 Y[c][i] = sum_a H[c][l0_i + a] psi_a(u_i) and the message epilogue
// The window taps and base cells of every point are computed once per solve (k_c1_taps).
// ------------------------------------------------------------------------------------------
constexpr int C1_COLS = 32;      // columns per CTA
constexpr int C1_CHUNK = 128;    // source points staged per step
constexpr int C1_TGT = 512;      // targets per gather CTA (2 per thread)

__global__ void k_c1_circulant(const float* __restrict__ D, int M, int n, float* __restrict__ c) {
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int q = 0; q <= M; ++q) s += (double)D[q] * cospi(2.0 * (double)((q * m) % n) / (double)n);
        c[m] = (float)s;
    }
}

// grid (ceil(n0 / 32), splits): CTA (b, p) spreads points [p ns / splits, (p+1) ns / splits) of
// columns [32 b, 32 b + 32) and adds its partial grids to G (zeroed by the caller).
__global__ void __launch_bounds__(256, 3) k_c1_spread(const float* __restrict__ X, const VecScale* sX,
                                                   const float* __restrict__ phi, const VecScale* sP,
                                                   const int* __restrict__ l0, const float* __restrict__ w, int ns,
                                                   int n0, int ng, int splits, float* __restrict__ G) {
    __shared__ float sV[C1_CHUNK][C1_COLS + 1];
    __shared__ __align__(16) float sW[C1_CHUNK][12];
    __shared__ int sL[C1_CHUNK];
    __shared__ float sG[C1_COLS][128 + 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int mask = ng - 1;
    const float sx = 1.f / mx_of(sX, 0), sp = 1.f / mx_of(sP, 0);
    const int nitems = ((n0 + C1_COLS - 1) / C1_COLS) * splits;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {   // (column group, point split)
    const int c0 = (item / splits) * C1_COLS, sidx = item % splits;
    const int pb = (int)((long long)sidx * ns / splits), pe = (int)((long long)(sidx + 1) * ns / splits);
    __syncthreads();                                        // the previous item's grid is written out
    for (int i = tid; i < C1_COLS * ng; i += blockDim.x) sG[i / ng][i % ng] = 0.f;
    float acc[MOT_W];
#pragma unroll
    for (int a = 0; a < MOT_W; ++a) acc[a] = 0.f;
    int cur = 0;
    bool have = false;
    auto flush = [&]() {
#pragma unroll
        for (int a = 0; a < MOT_W; ++a) {
            atomicAdd(&sG[lane][(cur + a) & mask], acc[a]);
            acc[a] = 0.f;
        }
    };
    const int per_warp = C1_CHUNK / nwarps;
    // the next chunk's loads (messages, then the points' taps) are issued before the current
    // chunk is accumulated, so their latency overlaps the arithmetic
    constexpr int PER = C1_COLS * C1_CHUNK / 256;
    static_assert(C1_CHUNK <= 256, "one point per thread for the taps");
    float v[PER], tw[MOT_W], tp = 0.f;
    int tl = 0;
    auto load_chunk = [&](int jb0) {
        const int cnt0 = min(C1_CHUNK, pe - jb0);
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int idx = tid + 256 * r, q = idx / C1_CHUNK, jj = idx - q * C1_CHUNK;
            v[r] = (jj < cnt0 && c0 + q < n0) ? __ldg(X + (size_t)(c0 + q) * ns + jb0 + jj) : 0.f;
        }
        if (tid < cnt0) {
            tp = phi[jb0 + tid];
            tl = l0[jb0 + tid];
#pragma unroll
            for (int a = 0; a < MOT_W; ++a) tw[a] = w[(size_t)(jb0 + tid) * MOT_W + a];
        }
    };
    if (pb < pe) load_chunk(pb);
    for (int jb = pb; jb < pe; jb += C1_CHUNK) {
        const int cnt = min(C1_CHUNK, pe - jb);
        __syncthreads();                                    // the previous chunk is consumed
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int idx = tid + 256 * r, q = idx / C1_CHUNK, jj = idx - q * C1_CHUNK;
            sV[jj][q] = v[r] * sx;
        }
        if (tid < cnt) {
            const float pj = tp * sp;
            sL[tid] = tl;
#pragma unroll
            for (int a = 0; a < MOT_W; ++a) sW[tid][a] = tw[a] * pj;
        }
        __syncthreads();
        if (jb + C1_CHUNK < pe) load_chunk(jb + C1_CHUNK);
        const int p0 = warp * per_warp, p1 = min(cnt, p0 + per_warp);
        for (int p = p0; p < p1; ++p) {
            const int l = sL[p];
            if (!have || l != cur) {                        // uniform over the warp
                if (have) flush();
                cur = l;
                have = true;
            }
            const float v = sV[p][lane];
            const float4 w0 = *reinterpret_cast<const float4*>(&sW[p][0]);
            const float4 w1 = *reinterpret_cast<const float4*>(&sW[p][4]);
            const float2 w2 = *reinterpret_cast<const float2*>(&sW[p][8]);
            acc[0] = fmaf(v, w0.x, acc[0]);
            acc[1] = fmaf(v, w0.y, acc[1]);
            acc[2] = fmaf(v, w0.z, acc[2]);
            acc[3] = fmaf(v, w0.w, acc[3]);
            acc[4] = fmaf(v, w1.x, acc[4]);
            acc[5] = fmaf(v, w1.y, acc[5]);
            acc[6] = fmaf(v, w1.z, acc[6]);
            acc[7] = fmaf(v, w1.w, acc[7]);
            acc[8] = fmaf(v, w2.x, acc[8]);
            acc[9] = fmaf(v, w2.y, acc[9]);
        }
    }
    if (have) flush();
    __syncthreads();
    for (int i = tid; i < C1_COLS * ng; i += blockDim.x) {
        const int q = i / ng, x = i - q * ng;
        const float val = sG[q][x];
        if (c0 + q < n0 && val != 0.f) atomicAdd(&G[(size_t)(c0 + q) * ng + x], val);
    }
    }   // item
}

// grid (ceil(nt / C1_TGT), ceil(n0 / 32)): convolution of 32 columns' grids, then two targets per
// thread for each column, message epilogue (floor, maximum, clamp count) and block reduction.
// With R.raw (a batch producing Gam_k, k >= 2): the row dots of phi^k's update are formed as the
// columns are produced, raw_i += sum_c beta_k[c][i] phi^1_c Gam_k[c][i] over the block's columns
// (beta_k and phi^1 normalised by their maxima, Gam_k as its mantissas: its maximum is not known
// yet, so R.raw_sc carries Gam_k's log-scale with a unit maximum), added atomically.
struct C1Rowdot {
    const float* beta;        // beta_k [c][i] (nt per column)
    const VecScale* s_beta;
    const float* phi1;        // phi^1 [n0]
    const VecScale* s_phi1;
    float* raw;               // [nt]; nullptr: no row dots
    VecScale* raw_sc;         // log-scale of Gam_k with maximum 1
};

__global__ void __launch_bounds__(256) k_c1_gather(const float* __restrict__ G, const float* __restrict__ cvec,
                                                   const int* __restrict__ l0, const float* __restrict__ w, int nt,
                                                   int n0, int ng, float* __restrict__ Y, float floor_,
                                                   VecScale* out_sc, const VecScale* sA, const VecScale* sB,
                                                   C1Rowdot R) {
    __shared__ float sGc[C1_COLS][128 + 1];
    __shared__ float sH[C1_COLS][128 + 1];
    __shared__ float sC[128];
    __shared__ float sPh[C1_COLS];       // row dots: phi^1 of the block's columns, normalised
    __shared__ float s_mx[8];
    __shared__ unsigned int s_cl[8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int c0 = blockIdx.y * C1_COLS, mask = ng - 1;
    const int ncol = min(C1_COLS, n0 - c0);
    for (int i = tid; i < ng; i += blockDim.x) sC[i] = cvec[i];
    for (int i = tid; i < ncol * ng; i += blockDim.x) sGc[i / ng][i % ng] = G[(size_t)c0 * ng + i];
    const bool rd = R.raw != nullptr;
    if (rd && tid < C1_COLS) sPh[tid] = tid < ncol ? R.phi1[c0 + tid] * (1.f / mx_of(R.s_phi1, 0)) : 0.f;
    __syncthreads();
    // only the cells this block's targets read (targets are sorted by cell): [l0 of the first,
    // l0 of the last + MOT_W - 1], about a quarter of the grid per block
    int xlo = 0, nx = ng;
    {
        const int i_first = blockIdx.x * C1_TGT, i_last = min(nt, i_first + C1_TGT) - 1;
        const int lo = l0[i_first], hi = l0[i_last] + MOT_W - 1;
        if (hi - lo + 1 < ng) {
            xlo = lo;
            nx = hi - lo + 1;
        }
    }
    for (int i = tid; i < ncol * nx; i += blockDim.x) {
        const int q = i / nx, x = (xlo + (i - q * nx)) & mask;
        float s = 0.f;
        for (int xp = 0; xp < ng; ++xp) s = fmaf(sC[(x - xp) & mask], sGc[q][xp], s);
        sH[q][x] = s;
    }
    __syncthreads();
    float mx = 0.f;
    unsigned int clamps = 0u;
    const float sbeta = rd ? 1.f / mx_of(R.s_beta, 0) : 0.f;
    float part = 0.f;                                       // this thread's row dot of target i
    auto emit = [&](float s, int q, int i, float b) {      // b: beta_k[c0 + q][i] (row dots)
        if (!(s >= floor_)) {
            s = floor_;
            clamps++;
        }
        mx = fmaxf(mx, s);
        Y[(size_t)(c0 + q) * nt + i] = s;
        if (rd) part = fmaf(sPh[q] * b, s, part);
    };
    for (int k = 0; k < C1_TGT / 256; ++k) {
        const int i = blockIdx.x * C1_TGT + k * blockDim.x + tid;
        if (i >= nt) break;
        part = 0.f;
        float t[MOT_W];
        const float* hp[MOT_W];                             // column 0 of each tap's grid cell
        const int b = l0[i];
#pragma unroll
        for (int a = 0; a < MOT_W; ++a) {
            t[a] = w[(size_t)i * MOT_W + a];
            hp[a] = &sH[0][(b + a) & mask];
        }
        if (ncol == C1_COLS) {
            // the row dots' beta_k values of this target: all loads issued before the columns' sums
            float bv[C1_COLS];
#pragma unroll
            for (int q = 0; q < C1_COLS; ++q) bv[q] = rd ? __ldg(R.beta + (size_t)(c0 + q) * nt + i) : 0.f;
#pragma unroll
            for (int q = 0; q < C1_COLS; ++q) {             // constant offsets q * (128 + 1)
                float s = 0.f;
#pragma unroll
                for (int a = 0; a < MOT_W; ++a) s = fmaf(hp[a][q * (128 + 1)], t[a], s);
                emit(s, q, i, bv[q]);
            }
        } else {
            for (int q = 0; q < ncol; ++q) {
                float s = 0.f;
#pragma unroll
                for (int a = 0; a < MOT_W; ++a) s = fmaf(hp[a][q * (128 + 1)], t[a], s);
                emit(s, q, i, rd ? __ldg(R.beta + (size_t)(c0 + q) * nt + i) : 0.f);
            }
        }
        if (rd) atomicAdd(R.raw + i, part * sbeta);
    }
    mx = warp_max(mx);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) clamps += __shfl_xor_sync(0xffffffffu, clamps, o);
    if (lane == 0) {
        s_mx[warp] = mx;
        s_cl[warp] = clamps;
    }
    __syncthreads();
    if (tid == 0) {
        float m = 0.f;
        unsigned int c = 0u;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            m = fmaxf(m, s_mx[k]);
            c += s_cl[k];
        }
        out_sc->ls = sA->ls + (double)logf(mx_of(sA, 0)) + sB->ls + (double)logf(mx_of(sB, 0));
        if (rd) R.raw_sc->ls = out_sc->ls;       // its maximum stays 1 (never set)
        atomic_max_pos(&out_sc->mx_bits, m);
        if (c) atomicAdd(&out_sc->clamped, c);
    }
}

}  // namespace

cudaError_t launch_close_points(const float* x, const int* perm, int n, int d, const double* c, double s, int n_grid,
                                float* u, int* err, cudaStream_t st) {
    const int blocks = std::max(1, std::min((n + 255) / 256, 1024));
    k_close_points<<<blocks, 256, 0, st>>>(x, perm, n, d, c[0], d > 1 ? c[1] : 0.0, d > 2 ? c[2] : 0.0, 1.0 / s,
                                           n_grid, u, err);
    return cudaGetLastError();
}

cudaError_t launch_pair(const float* phi1, const VecScale* s1, const int* perm1, int n1, const float* phik,
                        const VecScale* sk, const int* permk, int nk, const float* G, const VecScale* sG,
                        const float* B, const VecScale* sB, double* out, cudaStream_t st) {
    const long long total = (long long)n1 * nk;
    const int blocks = (int)std::max<long long>(1, std::min<long long>((total + 255) / 256, 4 * 152 * 8));
    k_pair<<<blocks, 256, 0, st>>>(phi1, s1, perm1, n1, phik, sk, permk, nk, G, sG, B, sB, out);
    return cudaGetLastError();
}

cudaError_t launch_rowdot(const float* B, const VecScale* sB, const float* G, const VecScale* sG, const float* phi,
                          const VecScale* sP, int ni, int nc, float* raw, cudaStream_t st) {
    const int bx = (ni + 255) / 256;
    int nsplit = std::max(1, std::min(64, (4 * 152 + bx - 1) / bx));
    nsplit = std::min(nsplit, std::max(1, nc / 16));
    k_rowdot<<<dim3(bx, nsplit), 256, 0, st>>>(B, sB, G, sG, phi, sP, ni, nc, nsplit, raw);
    return cudaGetLastError();
}

cudaError_t launch_colsum(const float* A, const VecScale* sA, const float* B, const VecScale* sB, const float* phi,
                          const VecScale* sP, int nj, int nc, float* raw, cudaStream_t st) {
    k_colsum<<<nc, 256, 0, st>>>(A, sA, B, sB, phi, sP, nj, raw);
    return cudaGetLastError();
}

cudaError_t launch_kernel_matrix(const float* ui, int ni, const float* uc, int nc, int d, float eta_u, float* K,
                                 VecScale* sc, cudaStream_t st) {
    long long total = (long long)ni * nc;
    int blocks = (int)std::min<long long>((total + 255) / 256, 8192);
    k_kernel_matrix<<<blocks, 256, 0, st>>>(ui, ni, uc, nc, d, eta_u, K, sc);
    return cudaGetLastError();
}

bool c1_supported(int d, int n) { return d == 1 && n >= 16 && n <= 128; }

cudaError_t launch_c1_circulant(const float* D, int M, int n, float* c, cudaStream_t st) {
    k_c1_circulant<<<1, 128, 0, st>>>(D, M, n, c);
    return cudaGetLastError();
}

cudaError_t launch_c1_batch(const float* X, const VecScale* sX, const float* phi, const VecScale* sP, const int* l0s,
                            const float* ws, int ns, const int* l0t, const float* wt, int nt, int n0, int ng,
                            const float* cvec, float* G, float* Y, float floor_, VecScale* out_sc, cudaStream_t st,
                            int stage, const float* rd_beta, const VecScale* rd_sbeta, const float* rd_phi1,
                            const VecScale* rd_sphi1, float* rd_raw, VecScale* rd_raw_sc) {
    const int nb = (n0 + C1_COLS - 1) / C1_COLS;
    if (stage == 0) {
        cudaError_t e = cudaMemsetAsync(G, 0, sizeof(float) * (size_t)n0 * ng, st);
        if (e != cudaSuccess) return e;
        // work items (column group, point split); a grid of at most one wave of resident CTAs (three
        // per SM at 80 registers and 40 KB of shared memory) loops over them
        const int splits = std::max(1, std::min(std::min(8, std::max(1, (3 * 152) / nb)), std::max(1, ns / C1_CHUNK)));
        const int items = nb * splits;
        k_c1_spread<<<std::min(items, 3 * 152), 256, 0, st>>>(X, sX, phi, sP, l0s, ws, ns, n0, ng, splits, G);
    } else {
        const C1Rowdot R{rd_beta, rd_sbeta, rd_phi1, rd_sphi1, rd_raw, rd_raw_sc};
        k_c1_gather<<<dim3((nt + C1_TGT - 1) / C1_TGT, nb), 256, 0, st>>>(G, cvec, l0t, wt, nt, n0, ng, Y, floor_,
                                                                         out_sc, sP, sX, R);
    }
    return cudaGetLastError();
}
