// Set-up kernels: normalisation onto the torus, binning, the spectral multiplier D
// (Eqs. Ker-reg, kappa_tilde, fft; Algorithm 4, precomputation), scalings in / out.
#include <algorithm>

#include "kernels.h"

namespace {

__device__ __forceinline__ unsigned int ord_enc(float f) {
    unsigned int b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// Block-level reductions first (one global atomic per block and value: thousands of warps
// hitting the same words serialise in L2).
__global__ void k_box(const PrepSet* __restrict__ sets, int d, unsigned int* box) {
    __shared__ unsigned int smn[3], smx[3];
    const PrepSet S = sets[blockIdx.y];
    if (threadIdx.x < 3) {
        smn[threadIdx.x] = 0xffffffffu;
        smx[threadIdx.x] = 0u;
    }
    __syncthreads();
    unsigned int mn[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, mx[3] = {0u, 0u, 0u};
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < S.n; j += gridDim.x * blockDim.x) {
        for (int t = 0; t < d; ++t) {
            unsigned int e = ord_enc(S.x[(size_t)j * d + t]);
            mn[t] = min(mn[t], e);
            mx[t] = max(mx[t], e);
        }
    }
    for (int t = 0; t < d; ++t) {
        unsigned int a = __reduce_min_sync(0xffffffffu, mn[t]);
        unsigned int b = __reduce_max_sync(0xffffffffu, mx[t]);
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&smn[t], a);
            atomicMax(&smx[t], b);
        }
    }
    __syncthreads();
    if (threadIdx.x < d) {
        atomicMin(&box[2 * threadIdx.x], smn[threadIdx.x]);
        atomicMax(&box[2 * threadIdx.x + 1], smx[threadIdx.x]);
    }
}

__device__ __forceinline__ float ord_dec(unsigned int e) {
    unsigned int b = (e & 0x80000000u) ? (e & 0x7fffffffu) : ~e;
    return __uint_as_float(b);
}

__global__ void k_radius(const PrepSet* __restrict__ sets, int d, unsigned int* box) {
    const PrepSet S = sets[blockIdx.y];
    float c[3] = {0.f, 0.f, 0.f};
    for (int t = 0; t < d; ++t) c[t] = 0.5f * (ord_dec(box[2 * t]) + ord_dec(box[2 * t + 1]));
    float r2 = 0.f;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < S.n; j += gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int t = 0; t < d; ++t) {
            float e = S.x[(size_t)j * d + t] - c[t];
            s = fmaf(e, e, s);
        }
        r2 = fmaxf(r2, s);
    }
    __shared__ unsigned int sr;
    if (threadIdx.x == 0) sr = 0u;
    __syncthreads();
    r2 = warp_max(r2);
    if ((threadIdx.x & 31) == 0) atomicMax(&sr, __float_as_uint(r2));
    __syncthreads();
    if (threadIdx.x == 0) atomicMax(&box[2 * d], sr);
}

__global__ void k_decode(const unsigned int* box, int d, float* out) {
    int t = threadIdx.x;
    if (t < 2 * d) out[t] = ord_dec(box[t]);
    if (t == 2 * d) out[t] = __uint_as_float(box[t]);
}

struct PrepArgs {
    int d, n_grid, TS, ntd, psub;
    double c[3];
    double inv_s;
};

__global__ void k_prep_points(const PrepSet* __restrict__ sets, PrepArgs A, int* err) {
    const PrepSet S = sets[blockIdx.y];
    const double half = 0.5 * A.n_grid;
    int tcells = 1;
    for (int t = 0; t < A.d; ++t) tcells *= A.TS;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < S.n; j += gridDim.x * blockDim.x) {
        int tile = 0, mult = 1, local = 0, lmult = 1;
        for (int t = 0; t < A.d; ++t) {
            float xf = S.x[(size_t)j * A.d + t];
            if (!isfinite(xf)) atomicOr(err, 1);
            double u = ((double)xf - A.c[t]) * A.inv_s * A.n_grid + half;
            float uf = (float)u;
            if (!(uf >= 0.f && uf < (float)A.n_grid)) {   // outside the fundamental domain: wrap
                double w = fmod(u, (double)A.n_grid);
                if (w < 0) w += A.n_grid;
                uf = (float)w;
                if (!(uf < (float)A.n_grid)) uf = 0.f;
            }
            S.u_tmp[(size_t)t * S.n + j] = uf;
            int cell = min((int)floorf(uf), A.n_grid - 1);
            tile += (cell / A.TS) * mult;
            mult *= A.ntd;
            local += (cell % A.TS) * lmult;
            lmult *= A.TS;
        }
        // sort key: tile-major, then the cell inside the tile
        const int key = tile * tcells + local;
        S.tile_of[j] = key;
        atomicAdd(&S.counts[key], 1);
        if (S.mu) {
            double m = S.mu[j];
            if (!(m >= 0.0) || isinf(m)) atomicOr(err, 2);
        }
    }
}

// Exclusive scan of the per-cell counts (one block per set), then the subproblem list: every
// tile's points are contiguous and split into runs of at most psub points.
__global__ void __launch_bounds__(1024) k_prep_scan(const PrepSet* __restrict__ sets, int ncells, int tcells,
                                                    int psub) {
    const PrepSet S = sets[blockIdx.x];
    __shared__ int part[1024];
    const int t = threadIdx.x, nt = blockDim.x;
    const int chunk = (ncells + nt - 1) / nt;
    const int c0 = min(ncells, t * chunk), c1 = min(ncells, c0 + chunk);
    int local = 0;
    for (int c = c0; c < c1; ++c) local += S.counts[c];
    part[t] = local;
    __syncthreads();
    for (int off = 1; off < nt; off <<= 1) {          // inclusive Hillis-Steele scan
        int v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int run = part[t] - local;                        // exclusive prefix of this chunk
    for (int c = c0; c < c1; ++c) {
        const int cnt = S.counts[c];
        S.cursor[c] = run;
        run += cnt;
    }
    __syncthreads();
    if (t != 0) return;
    const int ntiles = ncells / tcells;
    int ns = 0;
    for (int tile = 0; tile < ntiles; ++tile) {
        const int start = S.cursor[tile * tcells];
        const int end = tile + 1 < ntiles ? S.cursor[(tile + 1) * tcells] : S.n;
        for (int s = start; s < end; s += psub) {
            if (ns < S.maxsub) {
                Sub sb;
                sb.tile = tile;
                sb.start = s;
                sb.len = min(psub, end - s);
                sb.pad = 0;
                S.subs[ns] = sb;
            }
            ++ns;
        }
    }
    *S.nsub = min(ns, S.maxsub);
}

__global__ void k_prep_scatter(const PrepSet* __restrict__ sets, int d) {
    const PrepSet S = sets[blockIdx.y];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < S.n; j += gridDim.x * blockDim.x) {
        int pos = atomicAdd(&S.cursor[S.tile_of[j]], 1);
        for (int t = 0; t < d; ++t) S.u[(size_t)t * S.n + pos] = S.u_tmp[(size_t)t * S.n + j];
        S.perm[pos] = j;
        if (S.mu) {
            double m = S.mu[j];
            if (S.mu_f) S.mu_f[pos] = (float)m;
            if (S.mu_d) S.mu_d[pos] = m;
        }
    }
}

// ---- kappa_hat and D ----------------------------------------------------------------------

#define MOT_MAXPOLY 17

struct KernelArgs {
    int d, M;
    double eta, a, tau, epsB;
    int deg;
    double poly[MOT_MAXPOLY];   // kappa_B in t = r - a
};

__device__ double kappa_R(double r, const KernelArgs& K) {
    // Eq. (Ker-reg) on |x| = r
    if (r <= K.a) return exp(-r * r / K.eta);
    double t = (r <= K.tau ? r : K.tau) - K.a;
    double v = 0.0;
    for (int i = K.deg; i >= 0; --i) v = v * t + K.poly[i];
    return v;
}

// Samples kappa_tilde(j / (2M)) on {-M..M-1}^d (Eq. kappa_tilde with tau = 1/2), layout
// index = sum_t (j_t + M) (2M)^t.
__global__ void k_khat_samples(double* S, KernelArgs K) {
    const int L = 2 * K.M;
    long long total = 1;
    for (int t = 0; t < K.d; ++t) total *= L;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        long long r = idx;
        double s2 = 0.0;
        for (int t = 0; t < K.d; ++t) {
            int j = (int)(r % L) - K.M;
            r /= L;
            double x = (double)j / (double)L;
            s2 += x * x;
        }
        S[idx] = kappa_R(sqrt(s2), K);
    }
}

// One separable pass of the (2M)-point DFT of Eq. (fft): the kernel is even in every
// coordinate, so the transform is a cosine sum; only m in [0, M] is kept.
//   out[(p (M+1) + m) post + q] = (2M)^-1 sum_{j} in[(p 2M + j) post + q] cos(pi m (j - M) / M)
__global__ void k_cos_pass(const double* __restrict__ in, double* __restrict__ out, long long pre, long long post,
                           int M) {
    const int L = 2 * M;
    extern __shared__ double ctab[];                       // cos(pi a / M), a = 0..2M-1
    for (int a = threadIdx.x; a < L; a += blockDim.x) ctab[a] = cospi((double)a / (double)M);
    __syncthreads();
    const long long total = pre * (M + 1) * post;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        long long q = idx % post;
        long long rest = idx / post;
        int m = (int)(rest % (M + 1));
        long long p = rest / (M + 1);
        const double* src = in + (p * L) * post + q;
        double acc = 0.0;
        int a = (int)(((long long)m * (L - M)) % L);        // m (j - M) mod 2M at j = 0
        for (int j = 0; j < L; ++j) {
            acc += src[(long long)j * post] * ctab[a];
            a += m;
            if (a >= L) a -= L;
        }
        out[idx] = acc / (double)L;
    }
}

// Modified Bessel function I_0 by its power series sum_j ((z/2)^j / j!)^2 (all terms positive).
__device__ double bessel_i0_series(double z) {
    double q = 0.25 * z * z, term = 1.0, sum = 1.0;
    for (int j = 1; j < 200; ++j) {
        term *= q / ((double)j * (double)j);
        sum += term;
        if (term < 1e-18 * sum) break;
    }
    return sum;
}

// Fourier transform of the normalised window at grid frequency k:
//   Psi(k) = I_0(a sqrt(b^2 - w^2)) * pi a / sinh(a b),  w = 2 pi k / n  (|w| <= b).
__device__ double window_ft(int k, int n) {
    const double a = (double)(MOT_WHALF + 1);
    const double b = 3.14159265358979323846 * 1.5;
    double w = 2.0 * 3.14159265358979323846 * (double)k / (double)n;
    double z2 = b * b - w * w;
    double i0 = bessel_i0_series(a * sqrt(z2 > 0 ? z2 : 0.0));
    return i0 * 3.14159265358979323846 * a / sinh(a * b);
}

// deconv = 0: the weighted coefficients alone (for the exact trigonometric sums, which need no
// window deconvolution).
__global__ void k_make_D(const double* __restrict__ khat, float* D, int d, int M, int n, int deconv) {
    extern __shared__ double inv_psi2[];                   // 1 / Psi(k)^2, k = 0..M
    for (int k = threadIdx.x; k <= M; k += blockDim.x) {
        const double p = deconv ? window_ft(k, n) : 1.0;
        inv_psi2[k] = 1.0 / (p * p);
    }
    __syncthreads();
    const int nk = 2 * M + 1, nh = M + 1;
    long long total = nh;
    for (int t = 1; t < d; ++t) total *= nk;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        long long r = idx;
        int k[3] = {0, 0, 0};
        k[0] = (int)(r % nh);
        r /= nh;
        for (int t = 1; t < d; ++t) {
            k[t] = (int)(r % nk) - M;
            r /= nk;
        }
        double w = (k[0] == 0) ? 1.0 : 2.0;   // mirrored negative half in the first coordinate
        long long kidx = 0, mult = 1;
        for (int t = 0; t < d; ++t) {
            int a = abs(k[t]);
            if (a == M) w *= 0.5;              // symmetric weight on the faces |k_t| = M
            kidx += a * mult;
            mult *= nh;
            w *= inv_psi2[a];
        }
        D[idx] = (float)(w * khat[kidx]);
    }
}

// ---- scalings in / out ----------------------------------------------------------------------

__global__ void k_output(const float* __restrict__ phi, const VecScale* sc, const int* __restrict__ perm, int n,
                         double eta, double* u_out) {
    const double ls = sc->ls;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        u_out[perm[i]] = eta * (log((double)phi[i]) + ls);
}

// Every set of a solve in one launch (blockIdx.y = set).
__global__ void k_output_batch(OutBatch B) {
    const OutSet S = B.s[blockIdx.y];
    if (S.u == nullptr) return;
    const double ls = S.sc->ls;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S.n; i += gridDim.x * blockDim.x)
        S.u[S.perm[i]] = B.eta * (log((double)S.phi[i]) + ls);
}

__global__ void k_init_cold_batch(OutBatch B) {
    const OutSet S = B.s[blockIdx.y];
    float* phi = const_cast<float*>(S.phi);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S.n; i += gridDim.x * blockDim.x) phi[i] = 1.f;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        VecScale* sc = const_cast<VecScale*>(S.sc);
        sc->ls = 0.0;
        sc->mx_bits = __float_as_uint(1.f);
        sc->clamped = 0u;
        sc->ls_prev = 0.0;
        sc->mx_prev_bits = __float_as_uint(1.f);
    }
}

__global__ void k_init_cold(float* phi, VecScale* sc, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) phi[i] = 1.f;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        sc->ls = 0.0;
        sc->mx_bits = __float_as_uint(1.f);
        sc->clamped = 0u;
        sc->ls_prev = 0.0;
        sc->mx_prev_bits = __float_as_uint(1.f);
    }
}

__global__ void k_warm_max(const int* __restrict__ perm, int n, const double* u, double inv_eta, unsigned int* mx) {
    unsigned int m = 0u;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        m = max(m, ord_enc((float)(u[perm[i]] * inv_eta)));
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0) atomicMax(mx, m);
}

__global__ void k_warm_set(float* phi, VecScale* sc, const int* __restrict__ perm, const double* __restrict__ mu_d,
                           int n, const double* u, double inv_eta, const unsigned int* mx, double* logphi) {
    const double shift = (double)ord_dec(*mx);
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double l = u[perm[i]] * inv_eta;
        phi[i] = (float)exp(l - shift);
        if (mu_d) acc += mu_d[i] * l;
    }
    acc = warp_sum_d(acc);
    if ((threadIdx.x & 31) == 0 && acc != 0.0) atomicAdd(logphi, acc);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        sc->ls = shift;
        sc->mx_bits = __float_as_uint(1.f);
        sc->clamped = 0u;
        sc->ls_prev = shift;
        sc->mx_prev_bits = __float_as_uint(1.f);
    }
}

__global__ void k_permute_in(const float* __restrict__ src, const int* __restrict__ perm, int n, float* dst) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = src[perm[i]];
}
__global__ void k_permute_out(const float* __restrict__ src, const int* __restrict__ perm, int n, float* dst) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[perm[i]] = src[i];
}

int blocks_for(long long n, int tpb = 256, int cap = 4096) {
    long long b = (n + tpb - 1) / tpb;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

}  // namespace

cudaError_t launch_bounds(const PrepSet* sets, int nsets, int d, float* box_raw, float* out, cudaStream_t st) {
    // box_raw: 2d+1 uints of scratch
    unsigned int init[7] = {0xffffffffu, 0u, 0xffffffffu, 0u, 0xffffffffu, 0u, 0u};
    init[2 * d] = 0u;
    cudaError_t e = cudaMemcpyAsync(box_raw, init, sizeof(unsigned int) * (2 * d + 1), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    k_box<<<dim3(16, nsets), 256, 0, st>>>(sets, d, (unsigned int*)box_raw);
    k_radius<<<dim3(16, nsets), 256, 0, st>>>(sets, d, (unsigned int*)box_raw);
    k_decode<<<1, 32, 0, st>>>((const unsigned int*)box_raw, d, out);
    return cudaGetLastError();
}

cudaError_t launch_prep(const PrepSet* sets_dev, const PrepSet* sets_host, int nsets, int d, int n_grid,
                        const double* c, double s, int* err_flag, cudaStream_t st) {
    PrepArgs A;
    A.d = d;
    A.n_grid = n_grid;
    A.TS = mot_tile_size(d, n_grid);
    A.ntd = n_grid / A.TS;
    A.psub = mot_sub_points(d);
    for (int t = 0; t < 3; ++t) A.c[t] = t < d ? c[t] : 0.0;
    A.inv_s = 1.0 / s;
    const int ncells = mot_ncells(d, n_grid);
    int tcells = 1;
    for (int t = 0; t < d; ++t) tcells *= A.TS;
    int maxn = 1;
    for (int k = 0; k < nsets; ++k) {
        cudaError_t e = cudaMemsetAsync(sets_host[k].counts, 0, sizeof(int) * ncells, st);
        if (e != cudaSuccess) return e;
        if (sets_host[k].n > maxn) maxn = sets_host[k].n;
    }
    const int bx = blocks_for(maxn, 256, 1024);
    k_prep_points<<<dim3(bx, nsets), 256, 0, st>>>(sets_dev, A, err_flag);
    k_prep_scan<<<nsets, 1024, 0, st>>>(sets_dev, ncells, tcells, A.psub);
    k_prep_scatter<<<dim3(bx, nsets), 256, 0, st>>>(sets_dev, d);
    return cudaGetLastError();
}

size_t make_D_scratch_doubles(int d, int M) {
    size_t L = 2 * (size_t)M, s = 1;
    for (int t = 0; t < d; ++t) s *= L;
    return s;
}

size_t D_floats(int d, int M) {
    size_t s = M + 1;
    for (int t = 1; t < d; ++t) s *= (2 * (size_t)M + 1);
    return s;
}

cudaError_t launch_make_D(int d, int M, int n, double eta_n, double tau, double epsB, int p, const double* poly,
                          double* scratch_a, double* scratch_b, float* D, cudaStream_t st, bool deconv) {
    KernelArgs K;
    K.d = d;
    K.M = M;
    K.eta = eta_n;
    K.tau = tau;
    K.epsB = epsB;
    K.a = tau - epsB;
    K.deg = 2 * p;
    if (K.deg + 1 > MOT_MAXPOLY) return cudaErrorInvalidValue;
    for (int i = 0; i < MOT_MAXPOLY; ++i) K.poly[i] = i <= K.deg ? poly[i] : 0.0;
    const long long L = 2LL * M;
    long long total = 1;
    for (int t = 0; t < d; ++t) total *= L;
    k_khat_samples<<<blocks_for(total), 256, 0, st>>>(scratch_a, K);
    // passes over dims 0..d-1 (dim 0 fastest): in [pre][L][post] -> out [pre][M+1][post]
    double* in = scratch_a;
    double* out = scratch_b;
    long long post = 1;
    for (int t = 0; t < d; ++t) {
        long long pre = 1;
        for (int s = t + 1; s < d; ++s) pre *= L;
        long long outn = pre * (M + 1) * post;
        k_cos_pass<<<blocks_for(outn), 256, sizeof(double) * L, st>>>(in, out, pre, post, M);
        post *= (M + 1);
        double* tmp = in;
        in = out;
        out = tmp;
    }
    k_make_D<<<blocks_for((long long)D_floats(d, M)), 256, sizeof(double) * (M + 1), st>>>(in, D, d, M, n, deconv ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_output_batch(const OutBatch& B, cudaStream_t st) {
    int nmax = 0;
    for (int k = 0; k < B.nsets; ++k) nmax = std::max(nmax, B.s[k].n);
    if (B.nsets <= 0 || nmax <= 0) return cudaSuccess;
    k_output_batch<<<dim3(std::min((nmax + 255) / 256, 64), B.nsets), 256, 0, st>>>(B);
    return cudaGetLastError();
}

cudaError_t launch_init_cold_batch(const OutBatch& B, cudaStream_t st) {
    int nmax = 0;
    for (int k = 0; k < B.nsets; ++k) nmax = std::max(nmax, B.s[k].n);
    if (B.nsets <= 0 || nmax <= 0) return cudaSuccess;
    k_init_cold_batch<<<dim3(std::min((nmax + 255) / 256, 64), B.nsets), 256, 0, st>>>(B);
    return cudaGetLastError();
}

cudaError_t launch_output(const float* phi, const VecScale* sc, const int* perm, int n, double eta, double* u_out,
                          cudaStream_t st) {
    k_output<<<blocks_for(n), 256, 0, st>>>(phi, sc, perm, n, eta, u_out);
    return cudaGetLastError();
}

cudaError_t launch_init_phi(float* phi, VecScale* sc, const int* perm, const double* mu_d, int n, const double* u_warm,
                            double eta, double* logphi, float* scratch_max, cudaStream_t st) {
    if (u_warm == nullptr) {
        k_init_cold<<<blocks_for(n), 256, 0, st>>>(phi, sc, n);
        return cudaGetLastError();
    }
    cudaError_t e = cudaMemsetAsync(scratch_max, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    k_warm_max<<<blocks_for(n), 256, 0, st>>>(perm, n, u_warm, 1.0 / eta, (unsigned int*)scratch_max);
    k_warm_set<<<blocks_for(n), 256, 0, st>>>(phi, sc, perm, mu_d, n, u_warm, 1.0 / eta,
                                             (const unsigned int*)scratch_max, logphi);
    return cudaGetLastError();
}

cudaError_t launch_permute_in(const float* src, const int* perm, int n, float* dst, cudaStream_t st) {
    k_permute_in<<<blocks_for(n), 256, 0, st>>>(src, perm, n, dst);
    return cudaGetLastError();
}
cudaError_t launch_permute_out(const float* src, const int* perm, int n, float* dst, cudaStream_t st) {
    k_permute_out<<<blocks_for(n), 256, 0, st>>>(src, perm, n, dst);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Timing aid: one thread sleeps until `ns` nanoseconds have passed (a bounded wait on the clock,
// on nothing else), so that the host can enqueue the launches of a timed chunk ahead of the GPU
// and the per-launch events measure device time only.
// ------------------------------------------------------------------------------------------
namespace {
__global__ void k_delay(unsigned long long ns) {
    if (threadIdx.x != 0) return;
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    do {
        __nanosleep(20000);
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    } while (t - t0 < ns);
}
}  // namespace

cudaError_t launch_delay(unsigned long long ns, cudaStream_t st) {
    k_delay<<<1, 32, 0, st>>>(ns < 100000000ull ? ns : 100000000ull);
    return cudaGetLastError();
}
