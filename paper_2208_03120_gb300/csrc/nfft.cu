// NFFT-based fast summation kernels (Section 5, Algorithm 4) for sm_103a.
//
//   spread  : g[l]  = sum_j v_j psi(u_j - l)             (adjoint NFFT gridding, Eq. ndft*)
//   fftconv : h     = IFFT( D . FFT(g) ),  D = w kappa_hat / Psi^2 on |k_t| <= M   (Eq. fastsum_mat)
//   gather  : beta_i = sum_l h[l] psi(u_i - l)           (NFFT interpolation, Eq. ndft)
//
// Points are binned into tiles of the periodic grid; one CTA handles one subproblem (<= P
// points of one tile) and accumulates into a padded tile in shared memory, which is then added
// to the L2-resident grid.  The window has 2m+2 = 10 taps per dimension.
#include <cooperative_groups.h>
#include <mutex>
#include <vector>
#include <cmath>

#include "kernels.h"
#include "fft_smem.cuh"
#include "window.cuh"
#include "wave.cuh"

constexpr int kMaxDevices = 64;   // per-device one-time set-up tables

namespace {

template <int D>
__device__ __forceinline__ void tile_origin(int tile, int ntd, int TS, int* o) {
#pragma unroll
    for (int t = 0; t < D; ++t) {
        o[t] = (tile % ntd) * TS - MOT_WHALF;
        tile /= ntd;
    }
}

// Visit every element of a padded tile (P^D, origin o on the periodic grid of length n): a warp
// per row of P elements, lanes along x; f(tile index, grid index).  Indices advance row by row,
// with one wrap per coordinate instead of a division per element.
template <int D, class F>
__device__ __forceinline__ void for_tile(int P, const int* o, int n, F f) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    auto wrap = [n](int v) { return v < 0 ? v + n : (v >= n ? v - n : v); };
    if (D == 1) {
        for (int x = threadIdx.x; x < P; x += blockDim.x) f(x, wrap(o[0] + x));
        return;
    }
    const int rows = D == 2 ? P : P * P;
    for (int row = warp; row < rows; row += nwarps) {
        int ty = row, gz = 0;
        if (D == 3) {
            const int tz = row / P;
            ty = row - tz * P;
            gz = wrap(o[2] + tz);
        }
        const int gy = wrap(o[1] + ty);
        const int gbase = (gz * n + gy) * n, tbase = row * P;
        for (int x = lane; x < P; x += 32) f(tbase + x, gbase + wrap(o[0] + x));
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
// spread.  Points are sorted by grid cell inside each tile.  A warp walks a contiguous run of
// points; its lanes own the taps of the window (2-D: 100 taps, 4 per lane; 3-D: 100 (x, y)
// pairs x 10 z taps, 40 per lane), accumulate consecutive points of the same cell in
// registers, and add them to shared memory only when the cell changes (distinct addresses
// per instruction, one atomic per tap per occupied cell instead of per point).
// ------------------------------------------------------------------------------------------
template <int D>
struct RunSpread {
    static constexpr int NI = D == 1 ? 1 : 4;       // tap groups per lane
    static constexpr int NC = D == 3 ? MOT_W : 1;   // z taps per group
    float acc[NI][NC];
    int a[NI], b[NI];
    bool ok[NI];
    int lane;

    __device__ __forceinline__ void init(int lane_) {
        lane = lane_;
#pragma unroll
        for (int i = 0; i < NI; ++i) {
            const int q = lane + 32 * i;
            if (D == 1) {
                ok[i] = lane < MOT_W;
                a[i] = lane < MOT_W ? lane : 0;
                b[i] = 0;
            } else {
                ok[i] = q < MOT_W * MOT_W;
                a[i] = q % MOT_W;
                b[i] = min(q / MOT_W, MOT_W - 1);
            }
        }
        zero();
    }
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int i = 0; i < NI; ++i)
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[i][c] = 0.f;
    }
    // Lane-distributed window weights: lane L < 10 D holds tap (L % 10) of dimension L / 10.
    __device__ __forceinline__ float lane_weight(const float (*cw)[MOT_WDEG + 1], const float* f) const {
        const int dim = lane / MOT_W, tap = lane % MOT_W;
        if (dim >= D) return 0.f;
        const float fl = dim == 0 ? f[0] : (dim == 1 ? f[D > 1 ? 1 : 0] : f[D - 1]);
        float w = cw[tap][MOT_WDEG];
#pragma unroll
        for (int k = MOT_WDEG - 1; k >= 0; --k) w = fmaf(w, fl, cw[tap][k]);
        return w;
    }
    __device__ __forceinline__ void add(float v, float w) {
        if (D == 1) {
            acc[0][0] = fmaf(v, w, acc[0][0]);
        } else {
            float wab[NI];
#pragma unroll
            for (int i = 0; i < NI; ++i)
                wab[i] = v * __shfl_sync(0xffffffffu, w, a[i]) * __shfl_sync(0xffffffffu, w, MOT_W + b[i]);
            if (D == 2) {
#pragma unroll
                for (int i = 0; i < NI; ++i) acc[i][0] += wab[i];
            } else {
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const float wc = __shfl_sync(0xffffffffu, w, 2 * MOT_W + c);
#pragma unroll
                    for (int i = 0; i < NI; ++i) acc[i][c] = fmaf(wab[i], wc, acc[i][c]);
                }
            }
        }
    }
};

// ------------------------------------------------------------------------------------------
// 2-D spread, batched: a warp takes SP2_B cell-sorted points at a time.  Lane (p, t) =
// (lane & 15, lane >> 4) evaluates the 10 window taps of point p along dimension t (Horner
// with the coefficients in constant memory) and stages them in shared memory, the x taps
// scaled by the point's value v_p.  Lanes (a, blk) = (lane % 10, lane / 10) then form the
// grid contributions g[a][4 blk + i] = sum_p (v wx)_p[a] wy_p[4 blk + i] of consecutive points
// of one cell in registers and add them to the shared grid only when the cell changes.
// ------------------------------------------------------------------------------------------
constexpr int SP2_B = 16;         // points per warp batch
constexpr int SP2_ROW = 24;       // staged floats per point: v wx [0,10), wy [12,24) in the order
                                  // 0 3 6 9 | 1 4 7 - | 2 5 8 - (one float4 per lane row group)
constexpr int SP2_WARP = SP2_B * SP2_ROW;

// Lane (a, blk) = (lane % 10, lane / 10), lanes < 30, owns tap column a and tap rows blk, blk + 3,
// blk + 6 (, blk + 9 for blk = 0): the rows of one flush instruction are then consecutive, and in a
// grid whose row stride is 10 mod 32 the 30 lanes of every atomic hit 30 different banks.
struct Spread2Acc {
    float acc[4];
    int a, b0, nb;
    bool on;
    __device__ __forceinline__ void init(int lane) {
        on = lane < 30;
        a = on ? lane % MOT_W : 0;
        b0 = on ? lane / MOT_W : 2;               // lanes 30, 31 read a valid slot and never add
        nb = b0 == 0 ? 4 : 3;
        zero();
    }
    __device__ __forceinline__ int row(int i) const { return b0 + 3 * i; }
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i] = 0.f;
    }
    __device__ __forceinline__ void step(const float* row) {
        const float xa = row[a];
        const float4 y = *reinterpret_cast<const float4*>(row + 12 + 4 * b0);   // wy[b0], wy[b0+3], ...
        acc[0] = fmaf(xa, y.x, acc[0]);
        acc[1] = fmaf(xa, y.y, acc[1]);
        acc[2] = fmaf(xa, y.z, acc[2]);
        acc[3] = fmaf(xa, y.w, acc[3]);
    }
};

// Stage one batch: lane (p, t) handles point jb + p along dimension t.  `value(j)` gives v_j,
// `cell(lx, ly)` the key of the cell whose window starts at (lx, ly) (= floor(u) - MOT_WHALF).
// Returns the cell key of point `lane` on lanes < cnt.
template <class Value, class Cell>
__device__ __forceinline__ int spread2_stage(float* stg, int lane, int jb, int cnt, const float* __restrict__ ux,
                                             const float* __restrict__ uy, Value value, Cell cell) {
    const int p = lane & 15, t = lane >> 4;
    const bool ok = p < cnt;
    const int j = jb + p;
    int l = 0;
    float w[MOT_W];
    if (ok) {
        const float u = t == 0 ? ux[j] : uy[j];
        const float fl = floorf(u);
        window_taps(u - fl, w);
        l = (int)fl - MOT_WHALF;
    }
    const int lx = __shfl_sync(0xffffffffu, l, p), ly = __shfl_sync(0xffffffffu, l, p + 16);
    const int key = cell(lx, ly);
    if (ok) {
        float* row = stg + p * SP2_ROW;
        if (t == 0) {
            const float v = value(j);
#pragma unroll
            for (int q = 0; q < MOT_W; ++q) w[q] *= v;
            *reinterpret_cast<float4*>(row) = make_float4(w[0], w[1], w[2], w[3]);
            *reinterpret_cast<float4*>(row + 4) = make_float4(w[4], w[5], w[6], w[7]);
            *reinterpret_cast<float2*>(row + 8) = make_float2(w[8], w[9]);
        } else {
            *reinterpret_cast<float4*>(row + 12) = make_float4(w[0], w[3], w[6], w[9]);
            *reinterpret_cast<float4*>(row + 16) = make_float4(w[1], w[4], w[7], 0.f);
            *reinterpret_cast<float4*>(row + 20) = make_float4(w[2], w[5], w[8], 0.f);
        }
    }
    __syncwarp();
    return key;
}

// Accumulate a staged batch; `flush(key, acc)` adds a finished cell to the shared grid.  The
// starts of new cells are found up front (one ballot over the keys held by lanes < cnt), so
// the loop over the batch is unrolled and its shared-memory reads are issued back to back.
template <class Flush>
__device__ __forceinline__ void spread2_accumulate(const float* stg, int cnt, int key, int lane, Spread2Acc& A,
                                                   int& cur, Flush flush) {
    const int prev = __shfl_up_sync(0xffffffffu, key, 1);
    const unsigned starts = __ballot_sync(0xffffffffu, lane < cnt && key != (lane == 0 ? cur : prev));
    if (starts == 0u) {
        if (cnt == SP2_B) {
#pragma unroll
            for (int q = 0; q < SP2_B; ++q) A.step(stg + q * SP2_ROW);
        } else {
            for (int q = 0; q < cnt; ++q) A.step(stg + q * SP2_ROW);
        }
    } else {
#pragma unroll 4
        for (int q = 0; q < cnt; ++q) {
            if ((starts >> q) & 1u) {
                if (cur >= 0) flush(cur, A);
                A.zero();
                cur = __shfl_sync(0xffffffffu, key, q);
            }
            A.step(stg + q * SP2_ROW);
        }
    }
    __syncwarp();
}

template <int D>
__global__ void __launch_bounds__(256) k_spread(const Task* __restrict__ tasks, Globals G) {
    __shared__ Task T;
    __shared__ FacCache fc;
    __shared__ float cw[MOT_W][MOT_WDEG + 1];
    extern __shared__ float tile[];
    load_task(T, tasks + blockIdx.y);
    for (int i = threadIdx.x; i < MOT_W * (MOT_WDEG + 1); i += blockDim.x) (&cw[0][0])[i] = (&c_win[0][0])[i];
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) task_resets(T, G, 0);
    if (T.alpha == nullptr) load_factors(fc, G.fac, T.sf0, T.snf);

    const int n = G.n_grid;
    const int TS = mot_tile_size(D, n), P = TS + MOT_W - 1, ntd = n / TS;
    int npad = P;
    if (D >= 2) npad *= P;
    if (D >= 3) npad *= P;
    const int N = T.src.n;
    const int nsub = *T.src.nsub;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    float* stg = tile + ((npad + 3) & ~3) + warp * SP2_WARP;     // 2-D staging (per warp)

    // A contiguous range of subproblems per CTA: consecutive subproblems mostly share a tile,
    // which then stays in shared memory and is added to the grid once.
    const int per = (nsub + gridDim.x - 1) / gridDim.x;
    const int sbeg = min(nsub, (int)blockIdx.x * per), send = min(nsub, sbeg + per);
    int cur_tile = -1;
    int o[3] = {0, 0, 0};
    auto flush_tile = [&]() {
        __syncthreads();
        for_tile<D>(P, o, n, [&](int ti, int gi) {
            const float val = tile[ti];
            if (val != 0.f) atomicAdd(&T.grid[gi], val);
        });
    };
    for (int s = sbeg; s < send; ++s) {
        const Sub sb = T.src.subs[s];
        if (sb.tile != cur_tile) {
            if (cur_tile >= 0) flush_tile();
            __syncthreads();
            for (int i = threadIdx.x; i < npad; i += blockDim.x) tile[i] = 0.f;
            tile_origin<D>(sb.tile, ntd, TS, o);
            cur_tile = sb.tile;
            __syncthreads();
        }
        const int chunk = (sb.len + nwarps - 1) / nwarps;
        const int j0 = sb.start + min(sb.len, warp * chunk), j1 = sb.start + min(sb.len, (warp + 1) * chunk);
        if (D == 2) {
            Spread2Acc A;
            A.init(lane);
            int cur = -1;
            auto value = [&](int j) { return T.alpha ? T.alpha[j] : eval_prod(fc, j); };
            auto cell = [&](int lx, int ly) { return (ly - o[1]) * P + (lx - o[0]); };
            auto flush = [&](int key, const Spread2Acc& S) {
                if (S.on)
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        if (i < S.nb) atomicAdd(&tile[key + S.row(i) * P + S.a], S.acc[i]);
            };
            for (int jb = j0; jb < j1; jb += SP2_B) {
                const int cnt = min(SP2_B, j1 - jb);
                const int key = spread2_stage(stg, lane, jb, cnt, T.src.u, T.src.u + N, value, cell);
                spread2_accumulate(stg, cnt, key, lane, A, cur, flush);
            }
            if (cur >= 0) flush(cur, A);
            continue;
        }
        RunSpread<D> rs;
        rs.init(lane);
        int cur = -1;
        for (int jb = j0; jb < j1; jb += 32) {
          // coalesced prefetch of 32 points, then broadcast one at a time
          const int jl = jb + lane;
          float pv = 0.f, pu[D];
#pragma unroll
          for (int t = 0; t < D; ++t) pu[t] = 0.f;
          if (jl < j1) {
              pv = T.alpha ? T.alpha[jl] : eval_prod(fc, jl);
#pragma unroll
              for (int t = 0; t < D; ++t) pu[t] = T.src.u[t * N + jl];
          }
          const int cnt = min(32, j1 - jb);
          for (int k = 0; k < cnt; ++k) {
            const float v = __shfl_sync(0xffffffffu, pv, k);
            float f[D];
            int base = 0, stride = 1;
#pragma unroll
            for (int t = 0; t < D; ++t) {
                const float u = __shfl_sync(0xffffffffu, pu[t], k);
                const float fl = floorf(u);
                f[t] = u - fl;
                base += ((int)fl - MOT_WHALF - o[t]) * stride;
                stride *= P;
            }
            if (base != cur) {
                if (cur >= 0) {
#pragma unroll
                    for (int i = 0; i < RunSpread<D>::NI; ++i)
#pragma unroll
                        for (int c = 0; c < RunSpread<D>::NC; ++c)
                            if (rs.ok[i]) atomicAdd(&tile[cur + (c * P + rs.b[i]) * (D >= 2 ? P : 0) + rs.a[i]], rs.acc[i][c]);
                    rs.zero();
                }
                cur = base;
            }
            rs.add(v, rs.lane_weight(cw, f));
          }
        }
        if (cur >= 0) {
#pragma unroll
            for (int i = 0; i < RunSpread<D>::NI; ++i)
#pragma unroll
                for (int c = 0; c < RunSpread<D>::NC; ++c)
                    if (rs.ok[i]) atomicAdd(&tile[cur + (c * P + rs.b[i]) * (D >= 2 ? P : 0) + rs.a[i]], rs.acc[i][c]);
        }
    }
    if (cur_tile >= 0) flush_tile();
}

// ------------------------------------------------------------------------------------------
// gather + epilogue: one thread per target point
// ------------------------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(256) k_gather(const Task* __restrict__ tasks, Globals G) {
    __shared__ Task T;
    __shared__ FacCache fc, tf;
    __shared__ double sLsrc;
    __shared__ EpiConst sC;
    __shared__ EpiPre sP;
    extern __shared__ float tile[];
    load_task(T, tasks + blockIdx.y);
    __syncthreads();
    load_task_consts(T, G, fc, tf, sP, sC, sLsrc);
    __syncthreads();
    const double Lsrc = sLsrc;
    const EpiConst C = sC;
    EpiPartial ep;
    epi_zero(ep);

    if (T.hgrid == nullptr) {
        // node step without a kernel product (root update / root marginal)
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < T.tgt.n; i += gridDim.x * blockDim.x)
            epilogue_point(T, tf, C, G.floor_, i, 1.f, ep);
    } else {
        const int n = G.n_grid;
        const int TS = mot_tile_size(D, n), P = TS + MOT_W - 1, ntd = n / TS;
        int npad = P;
        if (D >= 2) npad *= P;
        if (D >= 3) npad *= P;
        const int N = T.tgt.n;
        const int nsub = *T.tgt.nsub;
        const int per = (nsub + gridDim.x - 1) / gridDim.x;
        const int sbeg = min(nsub, (int)blockIdx.x * per), send = min(nsub, sbeg + per);
        int cur_tile = -1;
        int o[3] = {0, 0, 0};
        for (int s = sbeg; s < send; ++s) {
            const Sub sb = T.tgt.subs[s];
            if (sb.tile != cur_tile) {      // consecutive subproblems mostly share the tile
                __syncthreads();
                tile_origin<D>(sb.tile, ntd, TS, o);
                for_tile<D>(P, o, n, [&](int ti, int gi) { tile[ti] = __ldg(&T.hgrid[gi]); });
                cur_tile = sb.tile;
                __syncthreads();
            }
            const int j1 = sb.start + sb.len;
            for (int j = sb.start + threadIdx.x; j < j1; j += blockDim.x) {
                const EpiIn in = epi_load(T, tf, j);
                float w[D][MOT_W];
                int base = 0, stride = 1;
#pragma unroll
                for (int t = 0; t < D; ++t) {
                    const float u = T.tgt.u[t * N + j];
                    const float fl = floorf(u);
                    window_taps(u - fl, w[t]);
                    base += ((int)fl - MOT_WHALF - o[t]) * stride;
                    stride *= P;
                }
                float acc = 0.f;
                if (D == 1) {
#pragma unroll
                    for (int a = 0; a < MOT_W; ++a) acc = fmaf(tile[base + a], w[0][a], acc);
                } else if (D == 2) {
#pragma unroll
                    for (int b = 0; b < MOT_W; ++b) {
                        const float* row = tile + base + b * P;
                        float r = 0.f;
#pragma unroll
                        for (int a = 0; a < MOT_W; ++a) r = fmaf(row[a], w[0][a], r);
                        acc = fmaf(r, w[1][b], acc);
                    }
                } else {
                    for (int c = 0; c < MOT_W; ++c) {
                        float pc = 0.f;
#pragma unroll
                        for (int b = 0; b < MOT_W; ++b) {
                            const float* row = tile + base + (c * P + b) * P;
                            float r = 0.f;
#pragma unroll
                            for (int a = 0; a < MOT_W; ++a) r = fmaf(row[a], w[0][a], r);
                            pc = fmaf(r, w[1][b], pc);
                        }
                        acc = fmaf(pc, w[D - 1][0], acc);
#pragma unroll
                        for (int q = 0; q < MOT_W - 1; ++q) w[D - 1][q] = w[D - 1][q + 1];
                    }
                }
                epilogue_point_in(T, C, G.floor_, j, acc, in, ep);
            }
        }
    }
    epi_block_finish(T, G, tf, Lsrc, ep, sP.iter, C);
}

// ------------------------------------------------------------------------------------------
// Window taps and base cell of every point, once per solve (the batched 1-D circle products
// of circle.cu read them for every column).
// ------------------------------------------------------------------------------------------
__global__ void k_c1_taps(const float* __restrict__ u, int n, int* __restrict__ l0, float* __restrict__ w) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const float x = u[j], fl = floorf(x);
        float t[MOT_W];
        window_taps(x - fl, t);
        l0[j] = (int)fl - MOT_WHALF;
#pragma unroll
        for (int a = 0; a < MOT_W; ++a) w[(size_t)j * MOT_W + a] = t[a];
    }
}

// ------------------------------------------------------------------------------------------
// Fused 2-D fast summation for grids n <= 64: one thread-block cluster per task.
//
//   1. each CTA spreads 1/CS of the sources into a private n x n grid in shared memory;
//   2. CTA r sums rows [rR, rR+R) over the cluster (distributed shared memory) and
//      transforms them along x, keeping k_x in [0, M];
//   3. CTA r takes the columns k_x = r, r+CS, ...: DFT along y for k_y in [-M, M], multiply by
//      D, inverse DFT back to all y;
//   4. CTA r forms rows [rR, rR+R) of h by the inverse x transform (real part);
//   5. every CTA copies the whole h into its own shared memory and interpolates 1/CS of the
//      targets, followed by the epilogue.
// The DFTs are direct sums over the pruned frequency set (|k_t| <= M = n/4): on these grids
// they are cheaper than radix-2 FFT stages separated by barriers.
// ------------------------------------------------------------------------------------------
#define F2_N 64
#define F2_M 16
#define F2_MAXR 8          // rows per CTA (n / CS) for CS >= 8
#define F2_MAXC 3          // columns per CTA (ceil((M+1) / CS)) for CS >= 8
#define F2_THREADS 640
#define F2_MAXPTS 32768    // largest point set of the fused kernel (per-rank source slots below)
#define F2_SLOTS (F2_MAXPTS / 8)
// dynamic shared memory: spread staging (SP2_WARP floats per warp), then the rank's source
// coordinates and values (3 x F2_SLOTS floats; a rank holds at most 1/8 of the sources)
#define F2_LD 74           // row stride of the shared grid: 10 mod 32 (conflict-free spread flushes)
#define F2_DYN_SMEM ((F2_THREADS / 32 * SP2_WARP + 3 * F2_SLOTS) * 4)

// Sum of `v` over groups of G consecutive lanes (G a power of two <= 32).
template <int G>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Static shared memory of one fused product (one CTA of the cluster).
struct __align__(16) F2Sh {
    Task T;
    FacCache fc, tf;
    EpiConst sC;
    EpiPre sP;
    double sLsrc;
    int s_ylo, s_yhi;                   // window rows of this CTA's targets
    int s_next;                         // next spread batch of this CTA
    float Gs[F2_N * F2_LD];
    float Grow[F2_MAXR * F2_N];
    float2 Gx[F2_MAXR * (F2_M + 1)];
    float2 Ycol[F2_MAXC][F2_N];
    float2 Hk[F2_MAXC][2 * F2_M + 1];
    float2 Acol[F2_MAXC][F2_N];
    float2 Arow[F2_MAXR * (F2_M + 1)];
    float Hrow[F2_MAXR * F2_N];
    float2 tw[F2_N];
};

// Twiddles e^{-2 pi i k / n} (once per kernel: they depend on n only).
__device__ __forceinline__ void f2_twiddles(F2Sh& S, int n) {
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        float sn, cs;
        sincospif(2.f * (float)k / (float)n, &sn, &cs);
        S.tw[k] = make_float2(cs, -sn);
    }
}

// Part of a product that reads only its own (static) task: the descriptor into shared memory,
// the spread grid zeroed.  Visible to the block after the caller's next barrier.
__device__ __forceinline__ void f2_prep(F2Sh& S, const Task* task, int n) {
    load_task(S.T, task);
    if (threadIdx.x == 0) {
        S.s_ylo = 1 << 30;
        S.s_yhi = -(1 << 30);
        S.s_next = 0;
    }
    for (int i = threadIdx.x; i < n * F2_LD; i += blockDim.x) S.Gs[i] = 0.f;
}

// The product itself, after f2_prep and a block barrier, once the results of the products it
// reads are complete.  Every CTA of the cluster calls it; it passes through the cluster barriers
// below whatever the data.
// MSG: the task is a message product (EPI_MSG with a kernel sum): the instance carries only that
// epilogue, which keeps its code (fetched cold at every launch of the one-shot kernel) small.  The
// persistent kernel runs the general instance for every product (its code stays resident, and a
// second inlined instance would push it past the register budget of 640 threads).
template <bool MSG>
__device__ __forceinline__ void f2_run(F2Sh& S, float* f2_stage, const Globals& G,
                                       cooperative_groups::cluster_group& cluster) {
    const Task& T = S.T;
    FacCache& fc = S.fc;
    FacCache& tf = S.tf;
    float* Gs = S.Gs;
    float* Grow = S.Grow;
    float2* Gx = S.Gx;
    auto& Ycol = S.Ycol;
    auto& Hk = S.Hk;
    auto& Acol = S.Acol;
    float2* Arow = S.Arow;
    float* Hrow = S.Hrow;
    const float2* tw = S.tw;
    float* sUx = f2_stage + (F2_THREADS / 32) * SP2_WARP;   // this rank's sources: x, y, value
    float* sUy = sUx + F2_SLOTS;
    float* sVv = sUy + F2_SLOTS;

    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int CS = (int)cluster.num_blocks();
    const int r = (int)cluster.block_rank();
    const int n = G.n_grid, M = G.M, mask = n - 1;
    if (r == 0 && tid == 0) task_resets(T, G, 0);
    if constexpr (MSG) {
        if (warp == 0) fill_factors_warp(fc, G.fac, T.sf0, T.snf, lane);
        __syncthreads();
    } else {
        load_task_consts(T, G, fc, tf, S.sP, S.sC, S.sLsrc);   // constants visible after the next barrier
    }
    const bool fast = MSG || T.hgrid != nullptr;
    EpiPartial ep;
    epi_zero(ep);
    // the first target of this thread: coordinates and epilogue inputs fetched now, used after
    // the spread and the transforms (their latency hides behind those phases)
    const int Nt = T.tgt.n;
    const int ti0 = (int)((long long)r * Nt / CS), ti1 = (int)((long long)(r + 1) * Nt / CS);
    float pux = 0.f, puy = 0.f;
    EpiIn pin;
    if (fast && ti0 + tid < ti1) {
        pux = T.tgt.u[ti0 + tid];
        puy = T.tgt.u[Nt + ti0 + tid];
        if constexpr (!MSG) pin = epi_load(T, tf, ti0 + tid);
    }

    if (fast) {
        // ---- 1. spread: warps walk contiguous runs of cell-sorted points ----------------------
        // 16-point batches: rank r takes every CS-th batch of the sorted sources (so sparse
        // regions, one flush per point, and dense ones, long runs, are shared evenly between the
        // CTAs), and its warps claim them one at a time from a shared counter
        const int Ns = T.src.n;
        {
            const int nbatch = (Ns + SP2_B - 1) / SP2_B;
            // prepass: this rank's batches r, r + CS, ... (coordinates and values) into shared
            // memory in one round of loads; the batch loop then reads no global memory
            const int nbr = r < nbatch ? (nbatch - r + CS - 1) / CS : 0;
            for (int q = tid; q < nbr * SP2_B; q += nt) {
                const int j = (r + CS * (q / SP2_B)) * SP2_B + (q % SP2_B);
                if (j < Ns) {
                    sUx[q] = T.src.u[j];
                    sUy[q] = T.src.u[Ns + j];
                    sVv[q] = T.alpha ? T.alpha[j] : eval_prod(fc, j);
                }
            }
            __syncthreads();
            float* stg = f2_stage + warp * SP2_WARP;
            Spread2Acc A;
            A.init(lane);
            int cur = -1;
            auto value = [&](int q) { return sVv[q]; };
            auto cell = [&](int lx, int ly) { return ((ly & mask) << 8) | (lx & mask); };
            auto flush = [&](int key, const Spread2Acc& S) {
                const int clx = key & 255, cly = key >> 8;
                if (S.on)
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        if (i < S.nb) atomicAdd(&Gs[((cly + S.row(i)) & mask) * F2_LD + ((clx + S.a) & mask)], S.acc[i]);
            };
            for (;;) {
                int k = 0;
                if (lane == 0) k = atomicAdd(&S.s_next, 1);
                k = __shfl_sync(0xffffffffu, k, 0);
                if (k >= nbr) break;
                const int cnt = min(SP2_B, Ns - (r + CS * k) * SP2_B);
                cur = -1;
                const int key = spread2_stage(stg, lane, k * SP2_B, cnt, sUx, sUy, value, cell);
                spread2_accumulate(stg, cnt, key, lane, A, cur, flush);
                flush(cur, A);
            }
        }
        {   // rows of h this CTA's targets will read: [min ly, max ly + 9] (targets are cell-sorted)
            const int i0 = ti0, i1 = ti1;
            int lo = 1 << 30, hi = -(1 << 30);
            for (int i = i0 + tid; i < i1; i += nt) {
                const int ly = (int)floorf(i == i0 + tid ? puy : T.tgt.u[Nt + i]) - MOT_WHALF;
                lo = min(lo, ly);
                hi = max(hi, ly);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
                hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
            }
            if (lane == 0 && lo <= hi) {
                atomicMin(&S.s_ylo, lo);
                atomicMax(&S.s_yhi, hi);
            }
        }
        cluster.sync();
        // ---- 2. reduce owned rows, DFT along x (4 lanes per output) ---------------------
        const int R = n / CS;
        const int y0 = r * R;
        {
            const float* peer[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) peer[q] = cluster.map_shared_rank(Gs, q < CS ? q : 0);
            for (int i = tid; i < R * n; i += nt) {
                float part[16];
                const int gi = (y0 + i / n) * F2_LD + (i % n);
#pragma unroll
                for (int q = 0; q < 16; ++q) part[q] = q < CS ? peer[q][gi] : 0.f;
                float s = 0.f;
#pragma unroll
                for (int q = 0; q < 16; ++q) s += part[q];
                Grow[i] = s;
            }
        }
        __syncthreads();
        {
            const int nout = R * (M + 1);
            for (int base = 0; base < nout * 4; base += nt) {
                const int gi = base + tid, o = gi >> 2, sub = gi & 3;
                float2 acc = make_float2(0.f, 0.f);
                if (o < nout) {
                    const int yy = o / (M + 1), kx = o - yy * (M + 1);
                    const float* g = Grow + yy * n;
                    for (int x = sub; x < n; x += 4) {
                        const float2 e = tw[(kx * x) & mask];
                        acc.x = fmaf(g[x], e.x, acc.x);
                        acc.y = fmaf(g[x], e.y, acc.y);
                    }
                }
                acc.x = group_sum<4>(acc.x);
                acc.y = group_sum<4>(acc.y);
                if (o < nout && sub == 0) Gx[o] = acc;
            }
        }
        cluster.sync();
        // ---- 3. owned columns: DFT along y, multiply by D, inverse DFT -------------------
        int ncols = 0;
        int kxs[F2_MAXC];
        for (int kx = r; kx <= M; kx += CS) kxs[ncols++] = kx;
        for (int i = tid; i < ncols * n; i += nt) {
            const int c = i / n, y = i - c * n;
            const int owner = y / R;
            Ycol[c][y] = cluster.map_shared_rank(Gx, owner)[(y - owner * R) * (M + 1) + kxs[c]];
        }
        __syncthreads();
        {
            const int nout = ncols * (2 * M + 1);
            for (int base = 0; base < nout * 4; base += nt) {
                const int gi = base + tid, o = gi >> 2, sub = gi & 3;
                float2 acc = make_float2(0.f, 0.f);
                int c = 0, kyo = 0;
                if (o < nout) {
                    c = o / (2 * M + 1);
                    kyo = o - c * (2 * M + 1);
                    const int ky = kyo - M;
                    for (int y = sub; y < n; y += 4) {
                        const float2 e = tw[(ky * y) & mask];
                        const float2 a = Ycol[c][y];
                        acc.x = fmaf(a.x, e.x, fmaf(-a.y, e.y, acc.x));
                        acc.y = fmaf(a.x, e.y, fmaf(a.y, e.x, acc.y));
                    }
                }
                acc.x = group_sum<4>(acc.x);
                acc.y = group_sum<4>(acc.y);
                if (o < nout && sub == 0) {
                    const float dd = T.D[kyo * (M + 1) + kxs[c]];
                    Hk[c][kyo] = make_float2(acc.x * dd, acc.y * dd);
                }
            }
        }
        __syncthreads();
        {
            const int nout = ncols * n;
            for (int base = 0; base < nout * 4; base += nt) {
                const int gi = base + tid, o = gi >> 2, sub = gi & 3;
                float2 acc = make_float2(0.f, 0.f);
                if (o < nout) {
                    const int c = o / n, y = o - c * n;
                    for (int kyo = sub; kyo <= 2 * M; kyo += 4) {
                        const float2 e = tw[((kyo - M) * y) & mask];   // conj: e^{+2 pi i ky y / n}
                        const float2 h = Hk[c][kyo];
                        acc.x = fmaf(h.x, e.x, fmaf(h.y, e.y, acc.x));
                        acc.y = fmaf(h.y, e.x, fmaf(-h.x, e.y, acc.y));
                    }
                }
                acc.x = group_sum<4>(acc.x);
                acc.y = group_sum<4>(acc.y);
                if (o < nout && sub == 0) Acol[o / n][o % n] = acc;
            }
        }
        cluster.sync();
        // ---- 4. owned rows of h: inverse DFT along x (real part), 2 lanes per output -----
        for (int i = tid; i < R * (M + 1); i += nt) {
            const int yy = i / (M + 1), kx = i - yy * (M + 1);
            const int owner = kx % CS, slot = kx / CS;
            Arow[i] = cluster.map_shared_rank(&Acol[0][0], owner)[slot * F2_N + y0 + yy];
        }
        __syncthreads();
        {
            const int nout = R * n;
            for (int base = 0; base < nout * 2; base += nt) {
                const int gi = base + tid, o = gi >> 1, sub = gi & 1;
                float acc = 0.f;
                if (o < nout) {
                    const int yy = o / n, x = o - yy * n;
                    for (int kx = sub; kx <= M; kx += 2) {
                        const float2 e = tw[(kx * x) & mask];
                        const float2 a = Arow[yy * (M + 1) + kx];
                        acc = fmaf(a.x, e.x, fmaf(a.y, e.y, acc));
                    }
                }
                acc = group_sum<2>(acc);
                if (o < nout && sub == 0) Hrow[o] = acc;
            }
        }
        cluster.sync();
        // ---- 5. copy the rows of h this CTA reads, interpolate (one thread per target) -------
        {
            int ylo = S.s_ylo, nrows = S.s_yhi >= S.s_ylo ? S.s_yhi - S.s_ylo + MOT_W : 0;
            if (nrows >= n) {
                ylo = 0;
                nrows = n;
            }
            const int cnt = nrows * n;
            for (int i0 = tid; i0 < cnt; i0 += 4 * nt) {
                float vals[4];
                int dst[4];
#pragma unroll
                for (int u4 = 0; u4 < 4; ++u4) {
                    const int i = i0 + u4 * nt;
                    vals[u4] = 0.f;
                    dst[u4] = -1;
                    if (i < cnt) {
                        const int q = i / n;
                        const int y = (ylo + q) & mask, x = i - q * n;
                        const int owner = y / R;
                        vals[u4] = cluster.map_shared_rank(Hrow, owner)[(y - owner * R) * n + x];
                        dst[u4] = y * F2_LD + x;
                    }
                }
#pragma unroll
                for (int u4 = 0; u4 < 4; ++u4)
                    if (dst[u4] >= 0) Gs[dst[u4]] = vals[u4];
            }
        }
        cluster.sync();      // peers may now leave; Hrow of this CTA is no longer read
        EpiConst C;
        if constexpr (!MSG) C = S.sC;
        const int i0 = ti0, i1 = ti1;
        for (int i = i0 + tid; i < i1; i += nt) {
            const bool first = i == i0 + tid;       // prefetched at the kernel's start
            EpiIn in;
            if constexpr (!MSG) in = first ? pin : epi_load(T, tf, i);
            const float ux = first ? pux : T.tgt.u[i], uy = first ? puy : T.tgt.u[Nt + i];
            const float fx = floorf(ux), fy = floorf(uy);
            float wx[MOT_W], wy[MOT_W];
            window_taps(ux - fx, wx);
            window_taps(uy - fy, wy);
            const int lx = (int)fx - MOT_WHALF, ly = (int)fy - MOT_WHALF;
            float acc = 0.f;
#pragma unroll
            for (int b = 0; b < MOT_W; ++b) {
                const float* row = Gs + ((ly + b) & mask) * F2_LD;
                float s2 = 0.f;
#pragma unroll
                for (int a = 0; a < MOT_W; ++a) s2 = fmaf(row[(lx + a) & mask], wx[a], s2);
                acc = fmaf(s2, wy[b], acc);
            }
            if constexpr (MSG) {
                float g = acc;
                if (!(g >= G.floor_)) {
                    g = G.floor_;
                    ep.clamps++;
                }
                T.out[i] = g;
                ep.mx_out = fmaxf(ep.mx_out, g);
            } else {
                epilogue_point_in(T, C, G.floor_, i, acc, in, ep);
            }
        }
    } else if constexpr (!MSG) {
        // node step without a kernel product; the cluster barrier orders the reset above
        cluster.sync();
        const EpiConst C = S.sC;
        for (int i = ti0 + tid; i < ti1; i += nt) epilogue_point(T, tf, C, G.floor_, i, 1.f, ep);
    }
    if constexpr (MSG)
        epi_block_finish_msg(T, fc.L, ep);
    else
        epi_block_finish(T, G, tf, S.sLsrc, ep, S.sP.iter, S.sC);
}

// One product per cluster (blockIdx.y): the launch-per-level form of the fused product.
template <bool MSG>
__global__ void __launch_bounds__(F2_THREADS, 1) k_fastsum2d(const Task* __restrict__ tasks, Globals G) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    __shared__ F2Sh S;
    extern __shared__ float4 f2_dyn[];             // spread staging, SP2_WARP floats per warp
    f2_prep(S, tasks + blockIdx.y, G.n_grid);
    f2_twiddles(S, G.n_grid);
    // Launched with programmatic stream serialisation: everything above uses only this launch's
    // own (static) task; from here on the kernel reads what the previous launch wrote (scale
    // records, messages, scalings), so it waits for that grid to complete and flush.  The next
    // launch may then be scheduled: its blocks do their own set-up and wait in the same way, so
    // at most one launch runs ahead.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    __syncthreads();
    f2_run<MSG>(S, reinterpret_cast<float*>(f2_dyn), G, cluster);
}

// ------------------------------------------------------------------------------------------
// Persistent wavefront kernel: every product of a chunk of tree sweeps in one launch.
//
// Clusters claim products from a counter in the order of the host's list schedule (a
// topological order of the chunk's dependency graph), and a product waits until every product
// it depends on has completed (per-product flags holding the launch's epoch).  A cluster waits
// only for products claimed before its own, and those are held by clusters that are already
// running, so the chunk completes whether or not all clusters are resident at once.  Claims run
// one product ahead (the next index is taken while the current product runs, published by its
// first cluster barrier and read by every CTA before the product's last one, so that rank 0 may
// leave as soon as the others have passed it).  Completion: every thread fences its writes, the cluster barrier, then
// rank 0 stores the flag with release semantics; a waiting CTA reads the flags with acquire
// semantics before its block barrier.  Every wait is bounded (wait_ns of %globaltimer): on expiry
// the CTA sets bit 2 (value 4) of the error word and the abort word, which stops all claims; the
// cluster still runs its product (on whatever data) so that every CTA meets every cluster barrier.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(F2_THREADS, 1) k_wave2d(WaveArgs A, Globals G) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    __shared__ F2Sh S;
    __shared__ int s_claim;                         // rank 0's latest claim
    extern __shared__ float4 f2_dyn[];
    float* dyn = reinterpret_cast<float*>(f2_dyn);
    const int tid = threadIdx.x;
    const int r = (int)cluster.block_rank();
    const int n = G.n_grid;
    const int epoch = *reinterpret_cast<volatile int*>(&A.ctl->epoch);   // advanced by the prologue
    f2_twiddles(S, n);
    if (r == 0 && tid == 0) s_claim = wave_claim(A);
    cluster.sync();
    int i = *cluster.map_shared_rank(&s_claim, 0);
    // A CTA may leave only once no peer reads its shared memory any more: every read of rank 0's
    // claim is followed by a cluster barrier before the loop test can end the kernel.
    cluster.sync();
    while (i < A.ntask) {
        f2_prep(S, A.tasks + i, n);
        // the next claim, written before f2_run and published by its first cluster barrier
        if (r == 0 && tid == 0) s_claim = wave_claim(A);
        if (tid < 32) wave_wait_warp(A, i, epoch, tid);
        __syncthreads();
        f2_run<false>(S, dyn, G, cluster);   // one instance for every mode (code stays resident)
        const int next = *cluster.map_shared_rank(&s_claim, 0);
        __threadfence();
        cluster.sync();                      // product complete; every read of s_claim done
        if (r == 0 && tid == 0) st_release_gpu(A.flags + i, epoch);
        i = next;
    }
}

// ------------------------------------------------------------------------------------------
// One-block iteration prologue: bump the iteration counter, zero the accumulators of the
// next iterate, keep the previous scale of the scalings and reset the records that this
// iteration produces.  Runs alone, so every later kernel of the iteration sees it.
// ------------------------------------------------------------------------------------------
__global__ void k_prologue(VecScale* const* __restrict__ list, int nlist, int save_prev, int bump,
                           double* zero_d, int zero_n, Globals G, WaveCtl* ctl, int* zero_i, int zero_in) {
    // launched with programmatic stream serialisation: wait for the previous grid, then let the
    // next launch get scheduled (it waits for this one in the same way)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int t = threadIdx.x;
    for (int i = t; i < nlist; i += blockDim.x) {
        VecScale* s = list[i];
        if (save_prev) {
            s->ls_prev = s->ls;
            s->mx_prev_bits = s->mx_bits;
        }
        s->mx_bits = 0u;
        s->clamped = 0u;
    }
    for (int i = t; i < zero_n; i += blockDim.x) zero_d[i] = 0.0;
    for (int i = t; i < zero_in; i += blockDim.x) zero_i[i] = 0;
    if (ctl != nullptr && t == 0) {
        ctl->next = 0;
        ctl->abort = 0;
        ctl->epoch = ctl->epoch + 1;
    }
    // advance the sweep counter by `bump` sweeps and clear their accumulator slots: sweep s adds
    // its scalings' logarithms to slot s + 1 and its root mass to slot s
    if (bump > 0 && t == 0) {
        const int old = *G.iter;
        *G.iter = old + bump;
        for (int s = 1; s <= bump; ++s) {
            IterAcc* a = G.acc + ((old + s + 1) % G.R);
            a->logphi = 0.0;
            a->mass = 0.0;
            a->rootviol = 0.0;
            a->pad = 0.0;
        }
    }
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

int gather_smem_bytes(int d, int n) {
    int TS = mot_tile_size(d, n), P = TS + MOT_W - 1;
    int np = P;
    for (int i = 1; i < d; ++i) np *= P;
    return np * (int)sizeof(float);
}

// padded tile, plus the per-warp staging of the batched 2-D spread (8 warps)
int spread_smem_bytes(int d, int n) {
    const int tile = ((gather_smem_bytes(d, n) / 4 + 3) & ~3) * 4;
    return tile + (d == 2 ? 8 * SP2_WARP * (int)sizeof(float) : 0);
}

cudaError_t launch_spread(int d, const Task* tasks, int ntask, int grid_x, const Globals& G, cudaStream_t st) {
    if (ntask <= 0) return cudaSuccess;
    dim3 grid(grid_x, ntask);
    int sm = spread_smem_bytes(d, G.n_grid);
    switch (d) {
    case 1: k_spread<1><<<grid, 256, sm, st>>>(tasks, G); break;
    case 2: k_spread<2><<<grid, 256, sm, st>>>(tasks, G); break;
    default: k_spread<3><<<grid, 256, sm, st>>>(tasks, G); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_gather(int d, const Task* tasks, int ntask, int grid_x, const Globals& G, cudaStream_t st) {
    if (ntask <= 0) return cudaSuccess;
    dim3 grid(grid_x, ntask);
    int sm = gather_smem_bytes(d, G.n_grid);
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
    // limits raised so far, per device (kernel attributes belong to the current device)
    static std::mutex mu;
    static int lim[kMaxDevices][10] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    int &c1 = lim[dev][0], &c2 = lim[dev][1], &c3a = lim[dev][2], &c3b = lim[dev][3], &s1 = lim[dev][4],
        &s2 = lim[dev][5], &s3 = lim[dev][6], &g1 = lim[dev][7], &g2 = lim[dev][8], &g3 = lim[dev][9];
    size_t sm = fftconv_smem(d, n);
    // padded tiles of the spread / gather kernels (3-D: 25^3 floats)
    const size_t ss = (size_t)spread_smem_bytes(d, n), gs = (size_t)gather_smem_bytes(d, n);
    if (d == 1) e = ensure_smem(k_spread<1>, ss, &s1);
    else if (d == 2) e = ensure_smem(k_spread<2>, ss, &s2);
    else e = ensure_smem(k_spread<3>, ss, &s3);
    if (e != cudaSuccess) return e;
    if (d == 1) e = ensure_smem(k_gather<1>, gs, &g1);
    else if (d == 2) e = ensure_smem(k_gather<2>, gs, &g2);
    else e = ensure_smem(k_gather<3>, gs, &g3);
    if (e != cudaSuccess) return e;
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

// ---- fused 2-D path -------------------------------------------------------------------------
namespace {
// cluster size of the fused kernel per device: 0 not yet probed, -1 no cluster fits
int g_cluster_size[kMaxDevices] = {};
// clusters of the fused kernel that fit on the GPU at once (cudaOccupancyMaxActiveClusters)
int g_cluster_active[kMaxDevices] = {};
// the same for the persistent wavefront kernel
int g_wave_active[kMaxDevices] = {};

int current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 0;
    return dev;
}
}

int fused2d_cluster_size() { return g_cluster_size[current_device()]; }
int fused2d_max_active_clusters() { return g_cluster_active[current_device()]; }
int wave2d_max_active_clusters() { return g_wave_active[current_device()]; }

bool fused2d_supported(int d, int n) {
    return d == 2 && n >= 16 && n <= F2_N && g_cluster_size[current_device()] > 0;
}
int fused2d_max_points() { return F2_MAXPTS; }

cudaError_t prepare_fused2d() {
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    int& csz = g_cluster_size[current_device()];
    if (csz != 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    for (auto fn : {k_fastsum2d<false>, k_fastsum2d<true>}) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) cudaGetLastError();
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, F2_DYN_SMEM);
        if (e != cudaSuccess) return e;
    }
    e = cudaFuncSetAttribute(k_wave2d, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) cudaGetLastError();
    e = cudaFuncSetAttribute(k_wave2d, cudaFuncAttributeMaxDynamicSharedMemorySize, F2_DYN_SMEM);
    if (e != cudaSuccess) return e;
    auto active = [](const void* fn, int cs) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cs, 1, 1);
        cfg.blockDim = dim3(F2_THREADS, 1, 1);
        cfg.dynamicSmemBytes = F2_DYN_SMEM;
        cudaLaunchAttribute attr;
        attr.id = cudaLaunchAttributeClusterDimension;
        attr.val.clusterDim.x = cs;
        attr.val.clusterDim.y = 1;
        attr.val.clusterDim.z = 1;
        cfg.attrs = &attr;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return nclusters;
    };
    for (int cs : {16, 8}) {
        const int nc = active((const void*)k_fastsum2d<false>, cs);
        if (nc > 0) {
            g_cluster_active[current_device()] = nc;
            g_wave_active[current_device()] = active((const void*)k_wave2d, cs);
            csz = cs;
            return cudaSuccess;
        }
    }
    csz = -1;
    return cudaSuccess;
}

cudaError_t launch_fused2d(const Task* tasks, int ntask, const Globals& G, cudaStream_t st, bool msg_only) {
    if (ntask <= 0) return cudaSuccess;
    const int cs = g_cluster_size[current_device()];
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs, ntask, 1);
    cfg.blockDim = dim3(F2_THREADS, 1, 1);
    cfg.dynamicSmemBytes = F2_DYN_SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;   // see griddepcontrol in the kernel
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return msg_only ? cudaLaunchKernelEx(&cfg, k_fastsum2d<true>, tasks, G)
                    : cudaLaunchKernelEx(&cfg, k_fastsum2d<false>, tasks, G);
}

cudaError_t launch_wave2d(const WaveArgs& A, int nclusters, const Globals& G, cudaStream_t st) {
    if (A.ntask <= 0) return cudaSuccess;
    const int cs = g_cluster_size[current_device()];
    if (cs <= 0 || nclusters <= 0) return cudaErrorInvalidConfiguration;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs * nclusters, 1, 1);
    cfg.blockDim = dim3(F2_THREADS, 1, 1);
    cfg.dynamicSmemBytes = F2_DYN_SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;   // no programmatic serialisation: the kernel
    attr.val.clusterDim.x = cs;                      // reads the prologue's epoch at its start
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_wave2d, A, G);
}

cudaError_t launch_prologue(VecScale* const* list, int nlist, int save_prev, int bump, double* zero_d, int zero_n,
                            const Globals& G, cudaStream_t st, WaveCtl* ctl, int* zero_i, int zero_in) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(1, 1, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.stream = st;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_prologue, list, nlist, save_prev, bump, zero_d, zero_n, G, ctl, zero_i, zero_in);
}

// ---- window coefficients ----------------------------------------------------------------------
// Degree-8 interpolation of the normalised Kaiser-Bessel window on each tap's unit interval at
// Chebyshev nodes, solved as a Vandermonde system in FP64 (host), uploaded once per device.
static double kb_exact(double delta) {
    const double a = MOT_WHALF + 1, b = 1.5 * 3.14159265358979323846;
    const double t = a * a - delta * delta;
    if (t <= 0.0) return 0.0;
    const double r = std::sqrt(t);
    if (r < 1e-12) return a * b / std::sinh(a * b);
    return (a / r) * std::sinh(b * r) / std::sinh(a * b);
}

cudaError_t prepare_window() {
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
    const int K = MOT_WDEG + 1;
    float coef[MOT_W][MOT_WDEG + 1];
    for (int j = 0; j < MOT_W; ++j) {
        std::vector<double> A(K * K), f(K), c(K);
        for (int i = 0; i < K; ++i) {
            const double x = 0.5 + 0.5 * std::cos((2.0 * i + 1.0) * 3.14159265358979323846 / (2.0 * K));
            double pw = 1.0;
            for (int k = 0; k < K; ++k) {
                A[i * K + k] = pw;
                pw *= x;
            }
            f[i] = kb_exact(x + MOT_WHALF - j);
        }
        for (int col = 0; col < K; ++col) {              // Gaussian elimination, partial pivoting
            int piv = col;
            for (int rr = col + 1; rr < K; ++rr)
                if (std::fabs(A[rr * K + col]) > std::fabs(A[piv * K + col])) piv = rr;
            if (piv != col) {
                for (int k = 0; k < K; ++k) std::swap(A[col * K + k], A[piv * K + k]);
                std::swap(f[col], f[piv]);
            }
            for (int rr = col + 1; rr < K; ++rr) {
                const double m = A[rr * K + col] / A[col * K + col];
                for (int k = col; k < K; ++k) A[rr * K + k] -= m * A[col * K + k];
                f[rr] -= m * f[col];
            }
        }
        for (int rr = K - 1; rr >= 0; --rr) {
            double s = f[rr];
            for (int k = rr + 1; k < K; ++k) s -= A[rr * K + k] * c[k];
            c[rr] = s / A[rr * K + rr];
        }
        for (int k = 0; k < K; ++k) coef[j][k] = (float)c[k];
    }
    e = cudaMemcpyToSymbol(c_win, coef, sizeof(coef));
    if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
    return e;
}

cudaError_t launch_c1_taps(const float* u, int n, int* l0, float* w, cudaStream_t st) {
    k_c1_taps<<<std::min((n + 255) / 256, 1024), 256, 0, st>>>(u, n, l0, w);
    return cudaGetLastError();
}

