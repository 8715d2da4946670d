// Small-eta local path (Section 6.1, closing remark): for very small eta the Gaussian kernel is so
// concentrated that the sum of Eq. (fastsum-sum) may be truncated to the pairs within a cutoff
// radius r_cut.  At such eta the scalings exp(u / eta) leave every floating-point range, so this
// path runs Algorithm 2 with the logarithms of the scalings and messages (FP64 vectors), and every
// truncated kernel sum as a log-sum-exp:
//
//     log beta_i = log sum_{j : |x_i - y_j| <= r_cut} exp(l_j - |x_i - y_j|^2 / eta)
//
// Points are binned into a common grid of cells no smaller than r_cut, so the pairs within r_cut
// of a target lie in the 3^d cells around the target's cell.
//   k_lsrc : per source cell, L_c = max_j l_j (FP64) and delta_j = l_j - L_c (FP32; the values
//            within a cell differ by a bounded amount, so FP32 keeps them to ~1e-6 absolute);
//   k_lse  : one CTA per (target cell, product): the neighbour cells whose bound
//            L_c - dmin(T, c)^2 / eta lies more than 60 below the best lower bound of the cell
//            pair maxima are dropped (their terms are below e^-60 of the largest); per target an
//            FP64 reference ref_i >= every term (max over the kept cells of L_c - dist(x_i,
//            box_c)^2 / eta), then an online log-sum-exp in FP32 of
//            e = (L_c - ref_i) + delta_j - |x_i - y_j|^2 / eta  (e <= 0), staged cell by cell
//            through shared memory; log beta_i = ref_i + m + log s in FP64;
//   epilogues: the message itself (b_k), or the scaling update of Algorithm 2 in log form
//            (f^k = log mu^k - g_k - sum_c b_c), or the exact marginal of the check pass.
#include <algorithm>
#include <cmath>

#include "kernels.h"

namespace {

__device__ __forceinline__ void cell_coords(int c, const LGrid& g, int* cc) {
    cc[0] = c % g.dims[0];
    cc[1] = g.d > 1 ? (c / g.dims[0]) % g.dims[1] : 0;
    cc[2] = g.d > 2 ? c / (g.dims[0] * g.dims[1]) : 0;
}

__device__ __forceinline__ int cell_of(const float* x, const LGrid& g) {
    int c = 0, mult = 1;
    for (int t = 0; t < g.d; ++t) {
        int q = (int)floorf((x[t] - g.lo[t]) * g.inv_h);
        q = min(max(q, 0), g.dims[t] - 1);
        c += q * mult;
        mult *= g.dims[t];
    }
    return c;
}

// ---- binning: counts, exclusive scan, scatter (all sets of a problem in one launch each) ------
__global__ void k_lbin_count(const LBinSet* __restrict__ sets, LGrid g, int* err) {
    const LBinSet S = sets[blockIdx.y];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < S.n; j += gridDim.x * blockDim.x) {
        float x[3] = {0.f, 0.f, 0.f};
        for (int t = 0; t < g.d; ++t) {
            x[t] = S.x[(size_t)j * g.d + t];
            if (!isfinite(x[t])) atomicOr(err, 1);
        }
        const int c = cell_of(x, g);
        S.cell[j] = c;
        atomicAdd(&S.cstart[c], 1);
        const double m = S.mu[j];
        if (!(m >= 0.0) || isinf(m)) atomicOr(err, 2);
    }
}

__global__ void __launch_bounds__(1024) k_lbin_scan(const LBinSet* __restrict__ sets, int ncells, int* maxcount) {
    const LBinSet S = sets[blockIdx.x];
    __shared__ int part[1024];
    const int t = threadIdx.x, nt = blockDim.x;
    const int chunk = (ncells + nt - 1) / nt;
    const int c0 = min(ncells, t * chunk), c1 = min(ncells, c0 + chunk);
    int local = 0, mx = 0;
    for (int c = c0; c < c1; ++c) {
        local += S.cstart[c];
        mx = max(mx, S.cstart[c]);
    }
    atomicMax(maxcount + blockIdx.x, mx);
    part[t] = local;
    __syncthreads();
    for (int off = 1; off < nt; off <<= 1) {
        const int v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int run = part[t] - local;
    for (int c = c0; c < c1; ++c) {
        const int cnt = S.cstart[c];
        S.cstart[c] = run;
        S.cursor[c] = run;
        run += cnt;
    }
    if (t == nt - 1) S.cstart[ncells] = part[t];
}

__global__ void k_lbin_scatter(const LBinSet* __restrict__ sets, int d) {
    const LBinSet S = sets[blockIdx.y];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < S.n; j += gridDim.x * blockDim.x) {
        const int pos = atomicAdd(&S.cursor[S.cell[j]], 1);
        for (int t = 0; t < d; ++t) S.u[(size_t)t * S.n + pos] = S.x[(size_t)j * d + t];
        S.perm[pos] = j;
        const double m = S.mu[j];
        S.mu_s[pos] = m;
        S.logmu[pos] = m > 0.0 ? log(m) : -INFINITY;
    }
}

// ---- source side: per-cell maxima and offsets ----------------------------------------------
__device__ __forceinline__ double lsrc_value(const LFac* F, int f0, int nf, int j) {
    double l = 0.0;
    for (int f = 0; f < nf; ++f) {
        const double v = F[f0 + f].v[j];
        l = F[f0 + f].sign > 0 ? l + v : l - v;
    }
    return l;
}

// One warp per (cell, product): L_c = max l_j, delta_j = l_j - L_c.
__global__ void __launch_bounds__(256) k_lsrc(const LTask* __restrict__ tasks, const LFac* __restrict__ F,
                                              int ncells, int* err) {
    const LTask& T = tasks[blockIdx.y];
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= ncells) return;
    const int c = warp;
    const int j0 = T.src.cstart[c], j1 = T.src.cstart[c + 1];
    double mx = -INFINITY;
    bool bad = false;
    for (int j = j0 + lane; j < j1; j += 32) {
        const double l = lsrc_value(F, T.sf0, T.snf, j);
        if (isnan(l) || l == INFINITY) bad = true;
        mx = fmax(mx, l);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(err, 1);
    if (lane == 0) T.Lc[c] = mx;
    for (int j = j0 + lane; j < j1; j += 32) {
        const double l = lsrc_value(F, T.sf0, T.snf, j);
        T.delta[j] = mx == -INFINITY ? -INFINITY : (float)(l - mx);
    }
}

// ---- the truncated log-sum-exp and its epilogue ---------------------------------------------
constexpr int LSE_THREADS = LSE_TARGETS;
constexpr int LSE_CAP = 1024;           // staged source points per round (coordinates + delta)
constexpr int LSE_MAXNB = 27;           // neighbour cells (3^d)

__device__ __forceinline__ double box_d2(const float* x, const int* cc, const LGrid& g) {
    // squared distance from x to the box of cell cc
    double s = 0.0;
    for (int t = 0; t < g.d; ++t) {
        const double lo = (double)g.lo[t] + (double)cc[t] * (double)g.h, hi = lo + (double)g.h;
        const double v = (double)x[t];
        const double e = v < lo ? lo - v : (v > hi ? v - hi : 0.0);
        s += e * e;
    }
    return s;
}

__device__ __forceinline__ double warp_sum_dd(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block reduction of three FP64 partials; thread 0 receives the totals.
__device__ __forceinline__ void block_sum3(double& a, double& b, double& c) {
    __shared__ double s3[3][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    a = warp_sum_dd(a);
    b = warp_sum_dd(b);
    c = warp_sum_dd(c);
    if (lane == 0) {
        s3[0][w] = a;
        s3[1][w] = b;
        s3[2][w] = c;
    }
    __syncthreads();
    if (w == 0) {
        a = lane < nw ? s3[0][lane] : 0.0;
        b = lane < nw ? s3[1][lane] : 0.0;
        c = lane < nw ? s3[2][lane] : 0.0;
        a = warp_sum_dd(a);
        b = warp_sum_dd(b);
        c = warp_sum_dd(c);
    }
    __syncthreads();
}

// The fast pass sums 2^e2 (exponents in log2 units, e2 <= 0 against the reference, so no term
// overflows).  Its result is kept when the sum is at least 2^-LSE_MIN2: every term that underflowed
// is then below 2^-(126 - LSE_MIN2) of the sum.  No constant is added inside exp2 (that would
// round the argument at the constant's magnitude).
constexpr float LSE_MIN2 = 100.f;
constexpr float LOG2E = 1.4426950408889634f;

template <int D>
__global__ void __launch_bounds__(LSE_THREADS) k_lse(const LTask* __restrict__ tasks, const LFac* __restrict__ F,
                                                     LGrid g, LGlobals G) {
    const LTask& T = tasks[blockIdx.y];
    const int cT = blockIdx.x;
    // this CTA's chunk of the target cell's points (blockIdx.z)
    const int i0 = T.tgt.cstart[cT] + (int)blockIdx.z * LSE_THREADS;
    const int i1 = min(T.tgt.cstart[cT + 1], i0 + LSE_THREADS);
    if (i0 >= i1) return;                       // uniform over the block
    __shared__ float sx[3][LSE_CAP];
    __shared__ float sdel[LSE_CAP];
    __shared__ int s_nb[LSE_MAXNB];
    __shared__ double s_L[LSE_MAXNB];
    __shared__ int s_nnb;
    const int tid = threadIdx.x;
    const float r2 = T.r2, ie = T.inv_eta;
    const double ied = T.inv_eta_d;
    int cc[3];
    cell_coords(cT, g, cc);
    // neighbour cells kept after the bound test (thread 0)
    if (tid == 0) {
        int nb[LSE_MAXNB];
        double dmin2[LSE_MAXNB], dmax2[LSE_MAXNB];
        int m = 0;
        const int span[3] = {1, g.d > 1 ? 1 : 0, g.d > 2 ? 1 : 0};
        for (int dz = -span[2]; dz <= span[2]; ++dz)
            for (int dy = -span[1]; dy <= span[1]; ++dy)
                for (int dx = -span[0]; dx <= span[0]; ++dx) {
                    const int q[3] = {cc[0] + dx, cc[1] + dy, cc[2] + dz};
                    bool ok = true;
                    for (int t = 0; t < g.d; ++t) ok = ok && q[t] >= 0 && q[t] < g.dims[t];
                    if (!ok) continue;
                    const int c = q[0] + g.dims[0] * (q[1] + g.dims[1] * q[2]);
                    if (T.src.cstart[c] == T.src.cstart[c + 1] || T.Lc[c] == -INFINITY) continue;
                    const int dd[3] = {abs(dx), abs(dy), abs(dz)};
                    double a = 0.0, b = 0.0;
                    for (int t = 0; t < g.d; ++t) {
                        const double lo = (double)max(dd[t] - 1, 0) * (double)g.h, hi = (double)(dd[t] + 1) * (double)g.h;
                        a += lo * lo;
                        b += hi * hi;
                    }
                    if (a > (double)r2) continue;
                    nb[m] = c;
                    dmin2[m] = a;
                    dmax2[m] = b;
                    ++m;
                }
        // lower bound of every target's largest term: a cell whose every pair is within r_cut
        double LB = -INFINITY;
        for (int q = 0; q < m; ++q)
            if (dmax2[q] <= (double)r2) LB = fmax(LB, T.Lc[nb[q]] - dmax2[q] * ied);
        int k = 0;
        for (int q = 0; q < m; ++q) {
            const double UB = T.Lc[nb[q]] - dmin2[q] * ied;
            if (UB < LB - 60.0) continue;
            s_nb[k] = nb[q];
            s_L[k] = T.Lc[nb[q]];
            ++k;
        }
        s_nnb = k;
    }
    __syncthreads();
    const int nnb = s_nnb;
    double acc1 = 0.0, acc2 = 0.0, acc3 = 0.0;
    for (int base = i0; base < i1; base += LSE_THREADS) {
        const int i = base + tid;
        const bool act = i < i1;
        float xi[3] = {0.f, 0.f, 0.f};
        double ref = -INFINITY;
        if (act) {
            for (int t = 0; t < g.d; ++t) xi[t] = T.tgt.u[(size_t)t * T.tgt.n + i];
            for (int q = 0; q < nnb; ++q) {
                int qc[3];
                cell_coords(s_nb[q], g, qc);
                ref = fmax(ref, s_L[q] - box_d2(xi, qc, g) * ied);
            }
        }
        // one pass with a fixed offset (branch-free: one exp2 per pair within r_cut); a target whose
        // sum left the FP32 range is redone below with a running maximum
        const float ie2 = ie * LOG2E;
        float s2 = 0.f;
        for (int q = 0; q < nnb; ++q) {
            const int c = s_nb[q];
            const int j0 = T.src.cstart[c], j1 = T.src.cstart[c + 1];
            const float off2 = act && ref > -INFINITY ? (float)((s_L[q] - ref) * (double)LOG2E) : -INFINITY;
            for (int jb = j0; jb < j1; jb += LSE_CAP) {
                const int cnt = min(LSE_CAP, j1 - jb);
                __syncthreads();
                for (int p = tid; p < cnt; p += LSE_THREADS) {
#pragma unroll
                    for (int t = 0; t < D; ++t) sx[t][p] = T.src.u[(size_t)t * T.src.n + jb + p];
                    sdel[p] = T.delta[jb + p] * LOG2E;
                }
                __syncthreads();
                if (act && off2 > -INFINITY) {
#pragma unroll 4
                    for (int p = 0; p < cnt; ++p) {
                        float d2 = 0.f;
#pragma unroll
                        for (int t = 0; t < D; ++t) {
                            const float e = xi[t] - sx[t][p];
                            d2 = fmaf(e, e, d2);
                        }
                        const float v = exp2f(fmaf(-d2, ie2, off2 + sdel[p]));
                        s2 += d2 <= r2 ? v : 0.f;
                    }
                }
            }
        }
        float m = 0.f, s = 0.f;                          // log beta = ref + m + log s
        if (act && s2 >= exp2f(-LSE_MIN2)) s = s2;
        const bool redo = act && !(s > 0.f);
        if (__syncthreads_or(redo)) {
            m = redo ? -INFINITY : m;
            float sr = redo ? 0.f : s;
            for (int q = 0; q < nnb; ++q) {
                const int c = s_nb[q];
                const int j0 = T.src.cstart[c], j1 = T.src.cstart[c + 1];
                const float off = redo && ref > -INFINITY ? (float)(s_L[q] - ref) : -INFINITY;
                for (int jb = j0; jb < j1; jb += LSE_CAP) {
                    const int cnt = min(LSE_CAP, j1 - jb);
                    __syncthreads();
                    for (int p = tid; p < cnt; p += LSE_THREADS) {
                        for (int t = 0; t < D; ++t) sx[t][p] = T.src.u[(size_t)t * T.src.n + jb + p];
                        sdel[p] = T.delta[jb + p];
                    }
                    __syncthreads();
                    if (redo && off > -INFINITY) {
                        for (int p = 0; p < cnt; ++p) {
                            float d2 = 0.f;
                            for (int t = 0; t < D; ++t) {
                                const float e = xi[t] - sx[t][p];
                                d2 = fmaf(e, e, d2);
                            }
                            if (d2 > r2) continue;
                            const float e = off + sdel[p] - d2 * ie;
                            if (e > m) {
                                sr = sr * __expf(m - e) + 1.f;      // rescale to the new maximum
                                m = e;
                            } else {
                                sr += __expf(e - m);
                            }
                        }
                    }
                }
            }
            s = sr;
        }
        if (act) {
            double lb = -INFINITY;
            if (s > 0.f) lb = ref + (double)m + (double)logf(s);
            else atomicOr(G.err, 8);                   // no source within r_cut of this target
            T.out[i] = lb;
            if (T.mode == LEPI_FWD) {
                double tsum = 0.0;
                for (int f = 0; f < T.tnf; ++f) tsum += F[T.tf0 + f].v[i];
                const double fk = T.tgt.logmu[i] - lb - tsum;
                T.f[i] = fk;
                const double mu = T.tgt.mu[i];
                if (mu > 0.0) acc1 += mu * fk;
            } else if (T.mode == LEPI_CHK) {
                double tsum = 0.0;
                for (int f = 0; f < T.tnf; ++f) tsum += F[T.tf0 + f].v[i];
                const double fk = T.f[i];
                const double lp = fk + lb + tsum;
                const double P = exp(lp);
                acc1 += fabs(P - T.tgt.mu[i]);
                acc2 += P > 0.0 ? P * fk : 0.0;
                acc3 += P;
            }
        }
    }
    if (T.mode == LEPI_FWD) {
        block_sum3(acc1, acc2, acc3);
        if (tid == 0 && acc1 != 0.0) {
            const int iter = *G.iter - T.iter_off;
            atomicAdd(&G.acc[(iter + 1) % G.R].logphi, acc1);
        }
    } else if (T.mode == LEPI_CHK) {
        block_sum3(acc1, acc2, acc3);
        if (tid == 0) {
            atomicAdd(T.acc_node + 0, acc1);
            atomicAdd(T.acc_node + 1, acc2);
            atomicAdd(T.acc_node + 2, acc3);
        }
    }
}

// Root steps (no kernel sum): LEPI_ROOT = mass and root violation of the last iterate, then
// f^1 = log mu^1 - sum_c b_c;  LEPI_CHKROOT = the root's exact marginal at the current scalings.
__global__ void __launch_bounds__(256) k_lroot(const LTask* __restrict__ tasks, const LFac* __restrict__ F,
                                               LGlobals G) {
    const LTask& T = tasks[blockIdx.y];
    double acc1 = 0.0, acc2 = 0.0, acc3 = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < T.tgt.n; i += gridDim.x * blockDim.x) {
        double tsum = 0.0;
        for (int f = 0; f < T.tnf; ++f) tsum += F[T.tf0 + f].v[i];
        const double fo = T.f[i];
        const double P = exp(fo + tsum);
        const double mu = T.tgt.mu[i];
        if (T.mode == LEPI_ROOT) {
            acc3 += P;
            acc1 += fabs(P - mu);
            const double fn = T.tgt.logmu[i] - tsum;
            T.f[i] = fn;
            if (mu > 0.0) acc2 += mu * fn;
        } else {
            acc1 += fabs(P - mu);
            acc2 += P > 0.0 ? P * fo : 0.0;
            acc3 += P;
        }
    }
    block_sum3(acc1, acc2, acc3);
    if (threadIdx.x == 0) {
        if (T.mode == LEPI_ROOT) {
            const int iter = *G.iter - T.iter_off;
            IterAcc* cur = G.acc + (iter % G.R);
            atomicAdd(&cur->mass, acc3);
            atomicAdd(&cur->rootviol, acc1);
            if (acc2 != 0.0) atomicAdd(&G.acc[(iter + 1) % G.R].logphi, acc2);
        } else {
            atomicAdd(T.acc_node + 0, acc1);
            atomicAdd(T.acc_node + 1, acc2);
            atomicAdd(T.acc_node + 2, acc3);
        }
    }
}

// f = u / eta in sorted order (warm start) or 0, and sum mu f into *logphi.
__global__ void k_linit(double* f, const int* perm, const double* mu, int n, const double* u, double inv_eta,
                        double* logphi) {
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double v = u ? u[perm[i]] * inv_eta : 0.0;
        f[i] = v;
        if (mu[i] > 0.0) acc += mu[i] * v;
    }
    acc = warp_sum_dd(acc);
    if ((threadIdx.x & 31) == 0 && acc != 0.0) atomicAdd(logphi, acc);
}

__global__ void k_lout(const double* f, const int* perm, int n, double eta, double* u) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) u[perm[i]] = eta * f[i];
}

int blocks_of(long long n, int per) { return (int)std::min<long long>((n + per - 1) / per, 4096); }

}  // namespace

cudaError_t launch_lbin(const LBinSet* sets_dev, int nsets, int nmax, const LGrid& g, int* err, int* maxcount,
                        cudaStream_t st) {
    const int bx = blocks_of(nmax, 256);
    k_lbin_count<<<dim3(bx, nsets), 256, 0, st>>>(sets_dev, g, err);
    k_lbin_scan<<<nsets, 1024, 0, st>>>(sets_dev, g.ncells, maxcount);
    k_lbin_scatter<<<dim3(bx, nsets), 256, 0, st>>>(sets_dev, g.d);
    return cudaGetLastError();
}

cudaError_t launch_lsrc(const LTask* tasks, int ntask, const LFac* F, int ncells, int* err, cudaStream_t st) {
    if (ntask <= 0) return cudaSuccess;
    k_lsrc<<<dim3((ncells * 32 + 255) / 256, ntask), 256, 0, st>>>(tasks, F, ncells, err);
    return cudaGetLastError();
}

cudaError_t launch_lse(const LTask* tasks, int ntask, int tchunks, const LFac* F, const LGrid& g, const LGlobals& G,
                       cudaStream_t st) {
    if (ntask <= 0) return cudaSuccess;
    const dim3 grid(g.ncells, ntask, std::max(1, tchunks));
    if (g.d == 1) k_lse<1><<<grid, LSE_THREADS, 0, st>>>(tasks, F, g, G);
    else if (g.d == 2) k_lse<2><<<grid, LSE_THREADS, 0, st>>>(tasks, F, g, G);
    else k_lse<3><<<grid, LSE_THREADS, 0, st>>>(tasks, F, g, G);
    return cudaGetLastError();
}

cudaError_t launch_lroot(const LTask* tasks, int ntask, const LFac* F, int nmax, const LGlobals& G, cudaStream_t st) {
    if (ntask <= 0) return cudaSuccess;
    k_lroot<<<dim3(blocks_of(nmax, 256), ntask), 256, 0, st>>>(tasks, F, G);
    return cudaGetLastError();
}

cudaError_t launch_linit(double* f, const int* perm, const double* mu, int n, const double* u, double eta,
                         double* logphi, cudaStream_t st) {
    k_linit<<<blocks_of(n, 256), 256, 0, st>>>(f, perm, mu, n, u, 1.0 / eta, logphi);
    return cudaGetLastError();
}

cudaError_t launch_lout(const double* f, const int* perm, int n, double eta, double* u, cudaStream_t st) {
    k_lout<<<blocks_of(n, 256), 256, 0, st>>>(f, perm, n, eta, u);
    return cudaGetLastError();
}
