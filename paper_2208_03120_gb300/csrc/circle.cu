// Circle-structure kernels (Section 4.2, Algorithm 3).
//
// The matrices beta_k (n_k x n_1) and gamma_k^T (n_k x n_1) are stored column-major: column c
// (a point of the first marginal) is one contiguous vector of the node's points, so a matrix
// product with a kernel matrix is a batch of independent kernel matrix-vector products (one
// per column), done by the fast-summation or dense kernels.  The scaling updates need
//   rowdot: raw_i = sum_c beta_k[c][i] phi^1_c gamma_k^T[c][i]      (phi^k, k >= 2)
//   colsum: raw_c = sum_j K^{(2,1)}[c][j] phi^2_j beta_2[c][j]        (phi^1)
// with every factor taken as its normalised mantissa (divided by its maximum).
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
