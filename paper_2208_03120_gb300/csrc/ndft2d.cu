// Fused 2-D fast summation with the trigonometric sums evaluated exactly (Section 5, Eqs. ndft
// and ndft*) for sm_103a: one thread-block cluster per kernel product.
//
// The fast summation (Eq. fastsum) replaces the kernel by its regularised Fourier series on the
// frequencies |k_t| <= M and evaluates, in grid units u in [0, n)^2,
//     ghat_k = sum_j v_j e^{-2 pi i k.u_j / n}                     (Eq. ndft*)
//     beta_i = Re sum_{k_x >= 0} D_k ghat_k e^{+2 pi i k.u_i / n}  (Eq. ndft; D_k = w_k kappa_hat_k)
// The NFFT (nfft.cu) computes both through the oversampled grid, with the window error of
// Section 5.  On the grids of the fused kernel (n <= 64, M <= 16) the two sums are small dense
// contractions.  With C_k = cos(2 pi k u / n) (k = 0..16) and S_k = sin(2 pi k u / n) (k = 1..16)
// per dimension, 33 trigonometric values e = [C_0..C_16, S_1..S_16] per coordinate:
//     A = sum_j e(u_j^y) (v_j e(u_j^x))^T                  (33 x 33, FP32)
//     beta_i = e(u_i^y)^T B e(u_i^x)                        (per target)
// where B folds A's four blocks (cos / sin in y and x) into the half spectrum times D
// (nd_combine).  Every source costs the same (no atomics, no dependence on how the points
// cluster), and the only exchange between the CTAs of the cluster is A.  The sums are exact up
// to FP32 rounding.
//
// Rank r of the cluster takes sources and targets [r N / CS, (r + 1) N / CS), in chunks of ND_CH:
//   1. every thread writes one source's e(u^y) and v e(u^x) to shared memory ([point][36]); warp w
//      takes a slice of the chunk's sources, its lanes a 8 x 4 tile of A's leading 32 x 32 block
//      (row 32 and column 32 on the side), all lanes reading the same sources (broadcast reads of
//      128 contiguous bytes), with packed FP32 FMAs (fma.rn.f32x2);
//   2. the 20 slices are summed through shared memory; every target's e(u^y), e(u^x) is written
//      ([value][target]); every rank pushes the four entries (cc, ss, cs, sc) of each frequency
//      pair to the pair's owner (rank p mod CS) as one 16-byte store into distributed shared
//      memory; after the first cluster barrier each owner sums the CS partials, forms its pairs'
//      entries of B^T and pushes them to every rank; after the second every CTA holds B^T;
//   3. warp w takes 32 targets, its lanes a 4-target x 8-row tile of T = E_x B^T, then
//      beta_i = sum_r T_ir e_r(u_i^y) (the 4 row groups summed by shuffles), and one thread per
//      target runs the epilogue of the sweep step (epilogue.cuh).
#include <cooperative_groups.h>
#include <mutex>

#include "kernels.h"
#include "wave.cuh"

constexpr int kNdMaxDevices = 64;

namespace {

#define ND_THREADS 640      // 20 warps (96 registers each)
#define ND_WARPS (ND_THREADS / 32)
#define ND_KF 17            // frequencies 0..16 per dimension
#define ND_E 33             // trigonometric values per coordinate: C_0..C_16, S_1..S_16
#define ND_S 16             // value index of S_k is ND_S + k (k >= 1)
#define ND_R 36             // padded row length of A, B^T and the source records
#define ND_NA (ND_R * ND_R)
#define ND_CH 640           // sources / targets per chunk (32 targets per warp)
#define ND_MAXPTS 32768     // largest point set per product (as the grid-based fused kernel)
#define ND_WSZ (35 * 32)    // one warp's partial A: 32 tile slots + 2 side + 1 corner, x 32 lanes
#define ND_PAIRS_RANK 37    // frequency pairs per rank for clusters of 8 or more: ceil(17 * 17 / 8)
                            // (pair p belongs to rank p % CS)
// dynamic shared memory: source records P [ND_CH][ND_R], Q [ND_CH][ND_R] (then the per-warp partial
// A, [ND_WARPS][ND_WSZ], within the bound below); target values E_y [ND_E][ND_CH], E_x [ND_E][ND_CH]
#define ND_DYN_FLOATS (2 * ND_CH * ND_R > ND_WARPS * ND_NA ? 2 * ND_CH * ND_R : ND_WARPS * ND_NA)
#define ND_DYN_SMEM (ND_DYN_FLOATS * 4)

struct __align__(16) NDSh {
    Task T;
    FacCache fc, tf;
    EpiConst sC;
    EpiPre sP;
    double sLsrc;
    __align__(16) float A[ND_NA];    // this rank's partial A
    float4 R4[16][ND_PAIRS_RANK];    // partial A of the pairs this rank owns, from every rank (cc, ss, cs, sc)
    float4 B4[ND_KF * ND_KF];        // B^T entries of every pair (cc, ss, cs, sc), from their owners
    __align__(16) float BT[ND_NA];   // B^T: BT[c * ND_R + r] multiplies e_r(u^y) e_c(u^x)
    __align__(16) float f[ND_CH];    // kernel sums of the chunk's targets
};
static_assert(2 * ND_E * ND_CH <= ND_DYN_FLOATS, "target values fit the dynamic shared memory");

__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;"
        : "=l"(d)
        : "l"(*reinterpret_cast<unsigned long long*>(&a)), "l"(*reinterpret_cast<unsigned long long*>(&b)),
          "l"(*reinterpret_cast<unsigned long long*>(&c)));
    return *reinterpret_cast<float2*>(&d);
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// Distributed shared memory: the address of this CTA's shared variable p in rank q's copy, and a
// 16-byte store there.
__device__ __forceinline__ unsigned nd_mapa(const void* p, int q) {
    unsigned a = (unsigned)__cvta_generic_to_shared(p), r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(q));
    return r;
}
__device__ __forceinline__ void nd_st_cluster4(unsigned a, float4 v) {
    asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}

// z_k = e^{+2 pi i k u / n} for k = 0..16 (emit(k, z)): exact anchors z_1, z_4 (sincospif of an
// exactly scaled argument; n is a power of two), the rest by at most four complex products.
template <class Emit>
__device__ __forceinline__ void nd_powers(float u, float inv_n, Emit emit) {
    float s1, c1, s4, c4;
    sincospif(2.f * u * inv_n, &s1, &c1);
    sincospif(8.f * u * inv_n, &s4, &c4);
    const float2 z1 = make_float2(c1, s1), z4 = make_float2(c4, s4);
    const float2 z2 = cmul(z1, z1), z3 = cmul(z2, z1);
    const float2 z8 = cmul(z4, z4), z12 = cmul(z8, z4), z16 = cmul(z8, z8);
    emit(0, make_float2(1.f, 0.f));
    emit(1, z1);
    emit(2, z2);
    emit(3, z3);
    emit(4, z4);
    emit(5, cmul(z4, z1));
    emit(6, cmul(z4, z2));
    emit(7, cmul(z4, z3));
    emit(8, z8);
    emit(9, cmul(z8, z1));
    emit(10, cmul(z8, z2));
    emit(11, cmul(z8, z3));
    emit(12, z12);
    emit(13, cmul(z12, z1));
    emit(14, cmul(z12, z2));
    emit(15, cmul(z12, z3));
    emit(16, z16);
}

// e(u) = [C_0..C_16, S_1..S_16] scaled by s: put(index, value).
template <class Put>
__device__ __forceinline__ void nd_values(float u, float inv_n, float s, Put put) {
    nd_powers(u, inv_n, [&](int k, float2 z) {
        put(k, s * z.x);
        if (k > 0) put(ND_S + k, s * z.y);
    });
}

// Part of a product that reads only its own (static) task.  Visible after the caller's next barrier.
__device__ __forceinline__ void nd_prep(NDSh& S, const Task* task) { load_task(S.T, task); }

// Frequency pair (ky', kx) = (p / 17, p % 17) of the cluster's A, a = its entries (cc, ss, cs, sc)
// (A's rows index e(u^y), its columns e(u^x); S_0 = 0 has no entry): the half spectrum ghat for
// ky = +ky' and -ky' (Eq. ndft*), times D, folded into the four entries of B^T that multiply
// (C_ky' C_kx, S_ky' S_kx, C_ky' S_kx, S_ky' C_kx) of a target's (y, x).  With s = sign(ky):
//   ghat = (Acc - s Ass) - i (Acs + s Asc),  Re(H e^{+i(kx tx + ky ty)}) = a (CxCy - s SxSy) - b (SxCy + s CxSy).
__device__ __forceinline__ float4 nd_combine(float4 a, int p, int M, float Dp, float Dm) {
    const int ky = p / ND_KF, kx = p - ky * ND_KF;
    float4 b = make_float4(0.f, 0.f, 0.f, 0.f);
    if (ky <= M && kx <= M) {
        const float acc = a.x;
        const float ass = ky > 0 && kx > 0 ? a.y : 0.f;
        const float acs = kx > 0 ? a.z : 0.f;
        const float asc = ky > 0 ? a.w : 0.f;
        const float ap = Dp * (acc - ass), bp = -Dp * (acs + asc);
        if (ky == 0) {
            b.x = ap;
            b.z = -bp;
        } else {
            const float am = Dm * (acc + ass), bm = -Dm * (acs - asc);
            b.x = ap + am;
            b.y = am - ap;
            b.z = -(bp + bm);
            b.w = bm - bp;
        }
    }
    return b;
}

// Positions of pair p's four entries in A (row-major, rows e(u^y)) or B^T (row-major, rows e(u^x)).
__device__ __forceinline__ void nd_pair_rc(int p, int (&row)[4], int (&col)[4]) {
    const int ky = p / ND_KF, kx = p - ky * ND_KF;
    row[0] = ky;        col[0] = kx;          // C_ky' C_kx
    row[1] = ND_S + ky; col[1] = ND_S + kx;   // S_ky' S_kx
    row[2] = ky;        col[2] = ND_S + kx;   // C_ky' S_kx
    row[3] = ND_S + ky; col[3] = kx;          // S_ky' C_kx
}

// e(u^y) and e(u^x) of the chunk's targets [i0, i0 + cnt) into Ey = dyn [ND_E][ND_CH] and
// Ex = Ey + ND_E * ND_CH (thread q writes target i0 + q: consecutive addresses).
__device__ __forceinline__ void nd_target_values(const Task& T, float* dyn, int i0, int cnt, float inv_n) {
    const int Nt = T.tgt.n;
    float* Ey = dyn;
    float* Ex = dyn + ND_E * ND_CH;
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
        const float ux = T.tgt.u[i0 + q], uy = T.tgt.u[Nt + i0 + q];
        nd_values(uy, inv_n, 1.f, [&](int e, float v) { Ey[e * ND_CH + q] = v; });
        nd_values(ux, inv_n, 1.f, [&](int e, float v) { Ex[e * ND_CH + q] = v; });
    }
}

// Kernel sums of the chunk's targets into f[0, cnt): warp w takes targets 32 w .. 32 w + 31,
// lane (tg, rg) = (lane & 7, lane >> 3) the 4 targets 32 w + 4 tg .. + 3 and the rows
// 8 rg .. 8 rg + 7 of T = E_x B^T (row 32 on the side), then sum_r T_ir e_r(u_i^y).
__device__ __forceinline__ void nd_target_sums(const float* dyn, const float* BT, float* f, int cnt) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tg = lane & 7, rg = lane >> 3;
    const int i0 = 32 * warp + 4 * tg;
    if (32 * warp >= cnt) return;                      // whole warp idle (cnt is warp-uniform)
    const float* Ey = dyn;
    const float* Ex = dyn + ND_E * ND_CH;
    float2 acc[4][4];                                  // acc[t][rp] = (T[t][8rg + 2rp], T[t][8rg + 2rp + 1])
    float2 side[2];                                    // (T[0][32], T[1][32]), (T[2][32], T[3][32])
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int rp = 0; rp < 4; ++rp) acc[t][rp] = make_float2(0.f, 0.f);
    side[0] = side[1] = make_float2(0.f, 0.f);
#pragma unroll 3
    for (int c = 0; c < ND_E; ++c) {
        const float4 x = *reinterpret_cast<const float4*>(Ex + c * ND_CH + i0);
        const float4 b0 = *reinterpret_cast<const float4*>(BT + c * ND_R + 8 * rg);
        const float4 b1 = *reinterpret_cast<const float4*>(BT + c * ND_R + 8 * rg + 4);
        const float b32 = BT[c * ND_R + 32];
        const float xs[4] = {x.x, x.y, x.z, x.w};
        const float2 bp[4] = {make_float2(b0.x, b0.y), make_float2(b0.z, b0.w), make_float2(b1.x, b1.y),
                              make_float2(b1.z, b1.w)};
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int rp = 0; rp < 4; ++rp) acc[t][rp] = ffma2(make_float2(xs[t], xs[t]), bp[rp], acc[t][rp]);
        side[0] = ffma2(make_float2(x.x, x.y), make_float2(b32, b32), side[0]);
        side[1] = ffma2(make_float2(x.z, x.w), make_float2(b32, b32), side[1]);
    }
    float s[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int rp = 0; rp < 4; ++rp) {
        const float4 y0 = *reinterpret_cast<const float4*>(Ey + (8 * rg + 2 * rp) * ND_CH + i0);
        const float4 y1 = *reinterpret_cast<const float4*>(Ey + (8 * rg + 2 * rp + 1) * ND_CH + i0);
        s[0] = fmaf(acc[0][rp].x, y0.x, fmaf(acc[0][rp].y, y1.x, s[0]));
        s[1] = fmaf(acc[1][rp].x, y0.y, fmaf(acc[1][rp].y, y1.y, s[1]));
        s[2] = fmaf(acc[2][rp].x, y0.z, fmaf(acc[2][rp].y, y1.z, s[2]));
        s[3] = fmaf(acc[3][rp].x, y0.w, fmaf(acc[3][rp].y, y1.w, s[3]));
    }
    if (rg == 0) {
        const float4 y = *reinterpret_cast<const float4*>(Ey + 32 * ND_CH + i0);
        s[0] = fmaf(side[0].x, y.x, s[0]);
        s[1] = fmaf(side[0].y, y.y, s[1]);
        s[2] = fmaf(side[1].x, y.z, s[2]);
        s[3] = fmaf(side[1].y, y.w, s[3]);
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        s[t] += __shfl_xor_sync(0xffffffffu, s[t], 8);
        s[t] += __shfl_xor_sync(0xffffffffu, s[t], 16);
    }
    if (rg == 0) *reinterpret_cast<float4*>(f + i0) = make_float4(s[0], s[1], s[2], s[3]);
}

// Records of the chunk's sources [c0, c0 + cnt): P[q] = e(u_j^y), Q[q] = v_j e(u_j^x) (ND_R floats
// each, stored as float4: rows of consecutive threads fall in distinct bank groups).
__device__ __forceinline__ void nd_source_records(const Task& T, const FacCache& fc, float* dyn, int c0, int cnt,
                                                  float inv_n) {
    const int Ns = T.src.n;
    float* P = dyn;
    float* Q = dyn + ND_CH * ND_R;
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
        const int j = c0 + q;
        const float ux = T.src.u[j], uy = T.src.u[Ns + j];
        const float v = T.alpha ? T.alpha[j] : eval_prod(fc, j);
        float e[ND_R];
        e[33] = e[34] = e[35] = 0.f;
        nd_values(uy, inv_n, 1.f, [&](int i, float val) { e[i] = val; });
        float4* p = reinterpret_cast<float4*>(P + q * ND_R);
#pragma unroll
        for (int m = 0; m < ND_R / 4; ++m) p[m] = make_float4(e[4 * m], e[4 * m + 1], e[4 * m + 2], e[4 * m + 3]);
        nd_values(ux, inv_n, v, [&](int i, float val) { e[i] = val; });
        float4* qq = reinterpret_cast<float4*>(Q + q * ND_R);
#pragma unroll
        for (int m = 0; m < ND_R / 4; ++m) qq[m] = make_float4(e[4 * m], e[4 * m + 1], e[4 * m + 2], e[4 * m + 3]);
    }
}

// Partial A of this warp's slice [k0, k1) of the chunk's records, accumulated into acc / side /
// corner: lane (g, h) = (lane >> 3, lane & 7) holds rows 8g..8g+7 x columns 4h..4h+3 of the leading
// 32 x 32 block as acc[ip][j] = (A[8g + 2ip][4h + j], A[8g + 2ip + 1][4h + j]), side = (A[32][lane],
// A[lane][32]) and corner = A[32][32].
__device__ __forceinline__ void nd_source_sums(const float* dyn, int k0, int k1, float2 (&acc)[4][4], float2& side,
                                               float& corner) {
    const int lane = threadIdx.x & 31, g = lane >> 3, h = lane & 7;
    const float* P = dyn;
    const float* Q = dyn + ND_CH * ND_R;
#pragma unroll 2
    for (int k = k0; k < k1; ++k) {
        const float* pr = P + k * ND_R;
        const float* qr = Q + k * ND_R;
        const float4 pa = *reinterpret_cast<const float4*>(pr + 8 * g);
        const float4 pb = *reinterpret_cast<const float4*>(pr + 8 * g + 4);
        const float4 q = *reinterpret_cast<const float4*>(qr + 4 * h);
        const float p32 = pr[32], q32 = qr[32], pl = pr[lane], ql = qr[lane];
        const float2 pp[4] = {make_float2(pa.x, pa.y), make_float2(pa.z, pa.w), make_float2(pb.x, pb.y),
                              make_float2(pb.z, pb.w)};
        const float qs[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int ip = 0; ip < 4; ++ip)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[ip][j] = ffma2(pp[ip], make_float2(qs[j], qs[j]), acc[ip][j]);
        side = ffma2(make_float2(p32, pl), make_float2(ql, q32), side);
        corner = fmaf(p32, q32, corner);
    }
}

// The product itself, after nd_prep and a block barrier, once the results of the products it reads
// are complete.  Every CTA of the cluster calls it and passes its two cluster barriers whatever
// the data (one on a task without a kernel product).  Every access to a peer's shared memory (the
// partial A to the owners of its frequency pairs, the owners' entries of B^T to every rank) lies
// between the product's two cluster barriers, so on return no peer touches this CTA's shared
// memory for this product: the CTA may start its next product or exit.  The peers must be running
// before the first access (a cluster barrier at the kernel's start).
template <bool MSG>
__device__ __forceinline__ void nd_run(NDSh& S, float* dyn, const Globals& G,
                                       cooperative_groups::cluster_group& cluster) {
    const Task& T = S.T;
    FacCache& fc = S.fc;
    FacCache& tf = S.tf;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int CS = (int)cluster.num_blocks();
    const int r = (int)cluster.block_rank();
    const int M = G.M;
    const float inv_n = 1.f / (float)G.n_grid;
    if (r == 0 && tid == 0) task_resets(T, G, 0);
    // factor caches now; the FP64 epilogue constants later, by a thread idle in phase 2
    if constexpr (MSG) {
        if (warp == 0) fill_factors_warp(fc, G.fac, T.sf0, T.snf, lane);
        __syncthreads();
    } else {
        load_task_caches(T, G, fc, tf, S.sP);
    }
    const bool fast = MSG || T.hgrid != nullptr;
    EpiPartial ep;
    epi_zero(ep);
    const int Nt = T.tgt.n;
    const int ti0 = (int)((long long)r * Nt / CS), ti1 = (int)((long long)(r + 1) * Nt / CS);
    // the epilogue inputs of this thread's first target and the two D entries of its frequency
    // pair: fetched now, used after the source phase
    EpiIn pin;
    if constexpr (!MSG)
        if (fast && ti0 + tid < ti1) pin = epi_load(T, tf, ti0 + tid);

    if (fast) {
        // D of the frequency pair p = r + CS (tid >> 4) that this thread combines in phase 2
        float Dp = 0.f, Dm = 0.f;
        {
            const int p = r + CS * (tid >> 4);
            const int ky = p / ND_KF, kx = p - ky * ND_KF;
            if (p < ND_KF * ND_KF && ky <= M && kx <= M) {
                Dp = __ldg(T.D + (ky + M) * (M + 1) + kx);
                Dm = __ldg(T.D + (M - ky) * (M + 1) + kx);
            }
        }
        // ---- 1. partial A over this rank's sources ------------------------------------------
        const int Ns = T.src.n;
        const int s0 = (int)((long long)r * Ns / CS), s1 = (int)((long long)(r + 1) * Ns / CS);
        float2 acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
        float2 side = make_float2(0.f, 0.f);
        float corner = 0.f;
        for (int c0 = s0; c0 < s1; c0 += ND_CH) {
            const int cnt = min(ND_CH, s1 - c0);
            nd_source_records(T, fc, dyn, c0, cnt, inv_n);
            __syncthreads();
            const int per = (cnt + ND_WARPS - 1) / ND_WARPS;
            const int k0 = min(cnt, warp * per), k1 = min(cnt, k0 + per);
            nd_source_sums(dyn, k0, k1, acc, side, corner);
            __syncthreads();                              // the records are written again / reused
        }
        // the slices of the 20 warps through shared memory: W[warp][slot][lane], slots 0..31 the
        // tile (slot 8 ip + 2 j + half), 32 / 33 side, 34 corner; summed by one thread per (slot,
        // lane) (consecutive addresses)
        {
            float* W = dyn + warp * ND_WSZ;
#pragma unroll
            for (int ip = 0; ip < 4; ++ip)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    W[(8 * ip + 2 * j) * 32 + lane] = acc[ip][j].x;
                    W[(8 * ip + 2 * j + 1) * 32 + lane] = acc[ip][j].y;
                }
            W[32 * 32 + lane] = side.x;
            W[33 * 32 + lane] = side.y;
            W[34 * 32 + lane] = corner;
        }
        __syncthreads();
        for (int t = tid; t < ND_WSZ; t += nt) {
            float s = 0.f;
#pragma unroll 4
            for (int w = 0; w < ND_WARPS; ++w) s += dyn[w * ND_WSZ + t];
            const int slot = t >> 5, ln = t & 31;
            int row, col;
            if (slot < 32) {
                row = 8 * (ln >> 3) + 2 * (slot >> 3) + (slot & 1);
                col = 4 * (ln & 7) + ((slot & 7) >> 1);
            } else if (slot == 32) {
                row = 32;
                col = ln;
            } else if (slot == 33) {
                row = ln;
                col = 32;
            } else {
                row = ln == 0 ? 32 : -1;
                col = 32;
            }
            if (row >= 0) S.A[row * ND_R + col] = s;
        }
        __syncthreads();                                  // W is read: the target values may follow
        if (tid < ND_KF * ND_KF) {
            const int p = tid;
            int row[4], col[4];
            nd_pair_rc(p, row, col);
            const float4 a = make_float4(S.A[row[0] * ND_R + col[0]], S.A[row[1] * ND_R + col[1]],
                                         S.A[row[2] * ND_R + col[2]], S.A[row[3] * ND_R + col[3]]);
            nd_st_cluster4(nd_mapa(&S.R4[r][p / CS], p % CS), a);
        }
        int tc0 = ti0;
        int tcnt = min(ND_CH, ti1 - tc0);
        if (tcnt > 0) nd_target_values(T, dyn, tc0, tcnt, inv_n);
        cluster.sync();      // every rank's partial A is with the owners of its pairs
        // ---- 2. the cluster's A, then B^T ----------------------------------------------------
        // rank r owns the frequency pairs p = r + CS m: each rank's partial (cc, ss, cs, sc) of
        // pair p went to R4[rank][m] of its owner before the barrier; thread (m, q) = (t >> 4,
        // t & 15) sums them, forms pair p's entries of B^T and writes them to B4[p] of rank q
        const int npair = (ND_KF * ND_KF - r + CS - 1) / CS;
        if (tid < 16 * npair) {
            const int m = tid >> 4, q = tid & 15;
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int k = 0; k < CS; ++k) {
                const float4 v = S.R4[k][m];
                a.x += v.x;
                a.y += v.y;
                a.z += v.z;
                a.w += v.w;
            }
            const int p = r + CS * m;
            const float4 b = nd_combine(a, p, M, Dp, Dm);
            if (q < CS) nd_st_cluster4(nd_mapa(&S.B4[p], q), b);
        }
        if constexpr (!MSG)
            if (tid == nt - 1) task_consts(T, fc, tf, S.sP, S.sC, S.sLsrc);   // read after the barrier
        cluster.sync();      // every pair's entries of B^T are in every rank's shared memory
        if (tid < ND_KF * ND_KF) {
            const int p = tid;
            const float4 b = S.B4[p];
            const float bv[4] = {b.x, b.y, b.z, b.w};
            int row[4], col[4];
            nd_pair_rc(p, row, col);
            const int ky = p / ND_KF, kx = p - ky * ND_KF;
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if ((e == 0) || (e == 1 && ky > 0 && kx > 0) || (e == 2 && kx > 0) || (e == 3 && ky > 0))
                    S.BT[col[e] * ND_R + row[e]] = bv[e];
        }
        __syncthreads();
        // ---- 3. targets, in chunks of ND_CH ------------------------------------------------
        EpiConst C;
        if constexpr (!MSG) C = S.sC;
        for (;;) {
            if (tcnt > 0) nd_target_sums(dyn, S.BT, S.f, tcnt);
            __syncthreads();
            if (tid < tcnt) {
                const int i = tc0 + tid;
                const float acc_i = S.f[tid];
                if constexpr (MSG) {
                    float gv = acc_i;
                    if (!(gv >= G.floor_)) {
                        gv = G.floor_;
                        ep.clamps++;
                    }
                    T.out[i] = gv;
                    ep.mx_out = fmaxf(ep.mx_out, gv);
                } else {
                    const EpiIn in = tc0 == ti0 ? pin : epi_load(T, tf, i);
                    epilogue_point_in(T, C, G.floor_, i, acc_i, in, ep);
                }
            }
            tc0 += ND_CH;
            if (tc0 >= ti1) break;
            tcnt = min(ND_CH, ti1 - tc0);
            __syncthreads();                              // f and the target values are reused
            nd_target_values(T, dyn, tc0, tcnt, inv_n);
            __syncthreads();
        }
    } else {
        // node step without a kernel product; the cluster barrier orders the reset above
        if constexpr (!MSG)
            if (tid == 0) task_consts(T, fc, tf, S.sP, S.sC, S.sLsrc);
        cluster.sync();
        if constexpr (!MSG) {
            const EpiConst C = S.sC;
            for (int i = ti0 + tid; i < ti1; i += nt) epilogue_point(T, tf, C, G.floor_, i, 1.f, ep);
        }
    }
    if constexpr (MSG)
        epi_block_finish_msg(T, fc.L, ep);
    else
        epi_block_finish(T, G, tf, S.sLsrc, ep, S.sP.iter, S.sC);
}

// One product per cluster (blockIdx.y): the launch-per-level form.
template <bool MSG>
__global__ void __launch_bounds__(ND_THREADS, 1) k_ndft2d(const Task* __restrict__ tasks, Globals G) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    __shared__ NDSh S;
    extern __shared__ float4 nd_dyn[];
    nd_prep(S, tasks + blockIdx.y);
    cluster.sync();      // every CTA of the cluster runs: its shared memory may be written
    // Launched with programmatic stream serialisation: everything above uses only this launch's
    // own (static) task; from here on the kernel reads what the previous launch wrote, so it waits
    // for that grid to complete and flush, then lets the next launch be scheduled.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    __syncthreads();
    nd_run<MSG>(S, reinterpret_cast<float*>(nd_dyn), G, cluster);
}

// Persistent wavefront kernel (the schedule of k_wave2d in nfft.cu: claims in the host's
// topological order, one claim ahead, completion flags with the launch's epoch, bounded waits)
// running this file's product.
__global__ void __launch_bounds__(ND_THREADS, 1) k_wave_nd(WaveArgs A, Globals G) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    __shared__ NDSh S;
    __shared__ int s_claim;                         // rank 0's latest claim
    extern __shared__ float4 nd_dyn[];
    float* dyn = reinterpret_cast<float*>(nd_dyn);
    const int tid = threadIdx.x;
    const int r = (int)cluster.block_rank();
    const int epoch = *reinterpret_cast<volatile int*>(&A.ctl->epoch);   // advanced by the prologue
    if (r == 0 && tid == 0) s_claim = wave_claim(A);
    cluster.sync();
    int i = *cluster.map_shared_rank(&s_claim, 0);
    // a CTA may leave only once no peer reads its shared memory any more: every read of rank 0's
    // claim is followed by a cluster barrier before the loop test can end it
    cluster.sync();
    while (i < A.ntask) {
        nd_prep(S, A.tasks + i);
        // the next claim, written before nd_run and published by its cluster barrier
        if (r == 0 && tid == 0) s_claim = wave_claim(A);
        if (tid < 32) wave_wait_warp(A, i, epoch, tid);
        __syncthreads();
        nd_run<false>(S, dyn, G, cluster);   // one instance for every mode (code stays resident)
        const int next = *cluster.map_shared_rank(&s_claim, 0);
        __threadfence();
        cluster.sync();                      // product complete; every read of s_claim done
        if (r == 0 && tid == 0) st_release_gpu(A.flags + i, epoch);
        i = next;
    }
}

int current_device_nd() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNdMaxDevices) return 0;
    return dev;
}

int g_nd_cluster_size[kNdMaxDevices] = {};   // 0: not set up; -1: no cluster size fits
int g_nd_active[kNdMaxDevices] = {};
int g_nd_wave_active[kNdMaxDevices] = {};

cudaLaunchConfig_t nd_config(int cs, int nclusters_x, int ny, cudaStream_t st, cudaLaunchAttribute* attr, bool pdl) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs * nclusters_x, ny, 1);
    cfg.blockDim = dim3(ND_THREADS, 1, 1);
    cfg.dynamicSmemBytes = ND_DYN_SMEM;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.numAttrs = 1;
    if (pdl) {
        attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[1].val.programmaticStreamSerializationAllowed = 1;
        cfg.numAttrs = 2;
    }
    cfg.attrs = attr;
    return cfg;
}
}  // namespace

bool ndft2d_supported(int d, int M) { return d == 2 && M <= 16 && g_nd_cluster_size[current_device_nd()] > 0; }
int ndft2d_max_active_clusters() { return g_nd_active[current_device_nd()]; }
int ndft2d_wave_max_active_clusters() { return g_nd_wave_active[current_device_nd()]; }

cudaError_t prepare_ndft2d() {
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    int& csz = g_nd_cluster_size[current_device_nd()];
    if (csz != 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    const void* fns[3] = {(const void*)k_ndft2d<false>, (const void*)k_ndft2d<true>, (const void*)k_wave_nd};
    for (const void* fn : fns) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) cudaGetLastError();
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, ND_DYN_SMEM);
        if (e != cudaSuccess) return e;
    }
    auto active = [](const void* fn, int cs) {
        cudaLaunchAttribute attr[2];
        cudaLaunchConfig_t cfg = nd_config(cs, 1, 1, 0, attr, false);
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return nclusters;
    };
    for (int cs : {16, 8}) {
        const int nc = active((const void*)k_ndft2d<false>, cs);
        if (nc > 0) {
            g_nd_active[current_device_nd()] = nc;
            g_nd_wave_active[current_device_nd()] = active((const void*)k_wave_nd, cs);
            csz = cs;
            return cudaSuccess;
        }
    }
    csz = -1;
    return cudaSuccess;
}

cudaError_t launch_ndft2d(const Task* tasks, int ntask, const Globals& G, cudaStream_t st, bool msg_only) {
    if (ntask <= 0) return cudaSuccess;
    const int cs = g_nd_cluster_size[current_device_nd()];
    if (cs <= 0) return cudaErrorInvalidConfiguration;
    cudaLaunchAttribute attr[2];
    cudaLaunchConfig_t cfg = nd_config(cs, 1, ntask, st, attr, true);
    return msg_only ? cudaLaunchKernelEx(&cfg, k_ndft2d<true>, tasks, G)
                    : cudaLaunchKernelEx(&cfg, k_ndft2d<false>, tasks, G);
}

cudaError_t launch_wave_nd(const WaveArgs& A, int nclusters, const Globals& G, cudaStream_t st) {
    if (A.ntask <= 0) return cudaSuccess;
    const int cs = g_nd_cluster_size[current_device_nd()];
    if (cs <= 0 || nclusters <= 0) return cudaErrorInvalidConfiguration;
    cudaLaunchAttribute attr[2];   // no programmatic serialisation: the kernel reads the prologue's
    cudaLaunchConfig_t cfg = nd_config(cs, nclusters, 1, st, attr, false);   // epoch at its start
    return cudaLaunchKernelEx(&cfg, k_wave_nd, A, G);
}
