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
#define ND_MAXDEP 64        // dependency lists up to this length are prefetched into shared memory
#define ND_WSZ (35 * 32)    // one warp's partial A: 32 tile slots + 2 side + 1 corner, x 32 lanes
#define ND_PAIRS_RANK 37    // frequency pairs per rank for clusters of 8 or more: ceil(17 * 17 / 8)
                            // (pair p belongs to rank p % CS)
// dynamic shared memory: source records P [ND_CH][ND_R], Q [ND_CH][ND_R] (then the per-warp partial
// A, [ND_WARPS][ND_WSZ], within the bound below); target values E_y [ND_E][ND_CH], E_x [ND_E][ND_CH]
#define ND_DYN_FLOATS (2 * ND_CH * ND_R > ND_WARPS * ND_NA ? 2 * ND_CH * ND_R : ND_WARPS * ND_NA)
#define ND_DYN_SMEM (ND_DYN_FLOATS * 4)

struct __align__(16) NDSh {
    Task Tb[2];                      // the product's task and, in the persistent kernel, the next one
    Factor Fs[MOT_MAXFAC], Ft[MOT_MAXFAC];   // persistent kernel: the next task's factor structs
    int dl[ND_MAXDEP];               // persistent kernel: the next task's dependency list
    int claim[2];                    // persistent kernel: rank 0's claims, alternating buffers
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
__device__ __forceinline__ void nd_prep(NDSh& S, const Task* task) { load_task(S.Tb[0], task); }

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

// Source record of one point in row q of the chunk: P[q] = e(u^y), Q[q] = s e(u^x) (ND_R floats
// each, stored as float4: rows of consecutive threads fall in distinct bank groups).
__device__ __forceinline__ void nd_record_row(float* row, float u, float inv_n, float s) {
    float e[ND_R];
    e[33] = e[34] = e[35] = 0.f;
    nd_values(u, inv_n, s, [&](int i, float val) { e[i] = val; });
    float4* p = reinterpret_cast<float4*>(row);
#pragma unroll
    for (int m = 0; m < ND_R / 4; ++m) p[m] = make_float4(e[4 * m], e[4 * m + 1], e[4 * m + 2], e[4 * m + 3]);
}

// Product of nf factors F at point j, each mantissa times 1 / the maximum of its scale record
// (the arithmetic of eval_prod on a factor cache), read by the calling thread itself.
__device__ __forceinline__ float nd_factor_prod(const Factor* F, int nf, int j) {
    float v = 1.f;
    for (int f = 0; f < nf; ++f) {
        const Factor g = F[f];
        const float x = __ldg(g.mant + j) * (1.f / mx_of(g.sc, g.use_prev));
        v = g.inv ? v / x : v * x;
    }
    return v;
}

// v_j of source j: the plain right-hand side or the product of the task's source factors Fs.
__device__ __forceinline__ float nd_source_v(const Task& T, const Factor* Fs, int j) {
    return T.alpha ? T.alpha[j] : nd_factor_prod(Fs, T.snf, j);
}

// The epilogue inputs of target i (epi_load) with the target factors' product formed from their
// structs Ft, so that no factor cache is needed yet.
__device__ __forceinline__ EpiIn nd_epi_load(const Task& T, const Factor* Ft, int i) {
    EpiIn in;
    in.t = 1.f;
    in.muf = 0.f;
    in.phi = 0.f;
    in.mud = 0.0;
    switch (T.mode) {
    case EPI_PHI:
        in.t = nd_factor_prod(Ft, T.tnf, i);
        in.muf = T.mu_f[i];
        break;
    case EPI_ROOT:
        in.t = nd_factor_prod(Ft, T.tnf, i);
        in.phi = T.phi[i];
        if (!T.free_node) {
            in.muf = T.mu_f[i];
            in.mud = T.mu_d[i];
        }
        break;
    case EPI_CROOT:
        in.phi = T.phi[i];
        in.muf = T.mu_f[i];
        in.mud = T.mu_d[i];
        break;
    case EPI_MARG:
        in.t = nd_factor_prod(Ft, T.tnf, i);
        in.phi = T.phi[i];
        if (T.mu_d) in.mud = T.mu_d[i];
        break;
    default:
        break;
    }
    return in;
}

// Asynchronous copies into shared memory (cp.async; each thread waits for its own copies).
__device__ __forceinline__ void nd_cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void nd_cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void nd_cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void nd_cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Warp 0 fills the factor caches of a task from its factor structs Fs / Ft (shared or global
// memory): lanes 0-15 the source factors, lanes 16-31 the target factors, each half summing its
// log-scales; lane 0 then reads the scale records of the epilogue.  No barrier.
template <bool MSG>
__device__ __forceinline__ void nd_fill_caches(const Task& T, const Globals& G, const Factor* Fs, const Factor* Ft,
                                               FacCache& fc, FacCache& tf, EpiPre& pre, int lane) {
    const bool src = lane < 16;
    const int hl = lane & 15;
    FacCache& c = src ? fc : tf;
    const Factor* F = src ? Fs : Ft;
    const int nf = src ? (T.alpha ? 0 : T.snf) : (MSG ? 0 : T.tnf);
    double L = 0.0;
    for (int t = hl; t < nf; t += 16) {
        const Factor f = F[t];
        const float mx = mx_of(f.sc, f.use_prev);
        c.mant[t] = f.mant;
        c.scale[t] = 1.f / mx;
        c.inv[t] = f.inv;
        const double Lt = ls_of(f.sc, f.use_prev) + (double)logf(mx);
        L += f.inv ? -Lt : Lt;
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) L += __shfl_xor_sync(0xffffffffu, L, o);
    if (hl == 0 && (src || !MSG)) {
        c.nf = nf;
        c.L = L;
    }
    if constexpr (!MSG) {
        if (lane == 0) {
            pre.ls_phi_k = ls_of(T.phi_sc, 0);
            pre.Lold = ls_of(T.phi_sc, 1) + (double)logf(mx_of(T.phi_sc, 1));
            pre.inv_mx_old = 1.f / mx_of(T.phi_sc, 1);
            pre.iter = (G.iter ? *G.iter : 0) - T.iter_off;
        }
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

// The product itself.  Every CTA of the cluster calls it and passes its two cluster barriers
// whatever the data (one on a task without a kernel product).  Every access to a peer's shared
// memory (the partial A to the owners of its frequency pairs, the owners' entries of B^T to every
// rank, the persistent kernel's claims) lies before the product's last cluster barrier, so on
// return no peer touches this CTA's shared memory for this product: the CTA may start its next
// product or exit.  The peers must be running before the first access (a cluster barrier at the
// kernel's start).  T is in shared memory and visible to every thread; Fs / Ft are its source and
// target factor structs.  The hooks wait for the products this one reads (Hooks::wait, followed by
// a block barrier with Hooks::kBarrierAfterWait) and carry the persistent kernel's claims and
// prefetches; with Hooks::kEarlyCoords the first chunk's source coordinates (constant inputs) are
// fetched before the wait.  The source values v_j and the first targets' epilogue inputs are
// formed by each thread from Fs / Ft; the factor caches (for the epilogue constants and later
// chunks) are filled by the last warp beside its slice of the adjoint contraction.
template <bool MSG, class Hooks>
__device__ __forceinline__ void nd_run(NDSh& S, const Task& T, float* dyn, const Globals& G,
                                       cooperative_groups::cluster_group& cluster, const Factor* Fs,
                                       const Factor* Ft, Hooks& hk) {
    FacCache& fc = S.fc;
    FacCache& tf = S.tf;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int CS = (int)cluster.num_blocks();
    const int r = (int)cluster.block_rank();
    const int M = G.M;
    const float inv_n = 1.f / (float)G.n_grid;
    const bool fast = MSG || T.hgrid != nullptr;
    const int Ns = T.src.n;
    const int s0 = (int)((long long)r * Ns / CS), s1 = (int)((long long)(r + 1) * Ns / CS);
    const int cnt0 = fast ? min(ND_CH, s1 - s0) : 0;
    float* P = dyn;
    float* Q = dyn + ND_CH * ND_R;
    // thread q < cnt0 owns row q of the first chunk's records; with Hooks::kEarlyCoords its
    // source's coordinates (constant inputs) are fetched before the wait
    float ux = 0.f, uy = 0.f;
    if constexpr (Hooks::kEarlyCoords)
        if (tid < cnt0) {
            ux = T.src.u[s0 + tid];
            uy = T.src.u[Ns + s0 + tid];
        }
    hk.wait(T, warp, lane);
    if constexpr (Hooks::kBarrierAfterWait) __syncthreads();
    // from here every thread may read what the products this one depends on wrote
    if constexpr (!Hooks::kEarlyCoords)
        if (tid < cnt0) {
            ux = T.src.u[s0 + tid];
            uy = T.src.u[Ns + s0 + tid];
        }
    if (r == 0 && tid == 0) task_resets(T, G, 0);
    EpiPartial ep;
    epi_zero(ep);
    const int Nt = T.tgt.n;
    const int ti0 = (int)((long long)r * Nt / CS), ti1 = (int)((long long)(r + 1) * Nt / CS);
    // the epilogue inputs of this thread's first target: fetched now, used after the source phase
    EpiIn pin;
    if constexpr (!MSG)
        if (fast && ti0 + tid < ti1) pin = nd_epi_load(T, Ft, ti0 + tid);

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
        float2 acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
        float2 side = make_float2(0.f, 0.f);
        float corner = 0.f;
        for (int c0 = s0; c0 < s1; c0 += ND_CH) {
            const int cnt = min(ND_CH, s1 - c0);
            if (tid < cnt) {
                const int j = c0 + tid;
                if (c0 != s0) {
                    ux = T.src.u[j];
                    uy = T.src.u[Ns + j];
                }
                const float v = nd_source_v(T, Fs, j);
                nd_record_row(P + tid * ND_R, uy, inv_n, 1.f);
                nd_record_row(Q + tid * ND_R, ux, inv_n, v);
            }
            if (c0 == s0) hk.before_first_barrier(tid, r, CS);
            __syncthreads();
            // the factor caches (the epilogue's) by the last warp, whose slice is the shortest
            if (c0 == s0 && warp == ND_WARPS - 1) nd_fill_caches<MSG>(T, G, Fs, Ft, fc, tf, S.sP, lane);
            const int per = (cnt + ND_WARPS - 1) / ND_WARPS;
            const int k0 = min(cnt, warp * per), k1 = min(cnt, k0 + per);
            nd_source_sums(dyn, k0, k1, acc, side, corner);
            __syncthreads();                              // the records are written again / reused
        }
        if (s0 >= s1) {
            hk.before_first_barrier(tid, r, CS);
            if (warp == ND_WARPS - 1) nd_fill_caches<MSG>(T, G, Fs, Ft, fc, tf, S.sP, lane);
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
        // the first cluster barrier in two halves: arrive once this thread's pushes are issued,
        // wait after the target values (local work), so that they hide the other ranks' lag
        asm volatile("barrier.cluster.arrive.release;" ::: "memory");
        int tc0 = ti0;
        int tcnt = min(ND_CH, ti1 - tc0);
        if (tcnt > 0) nd_target_values(T, dyn, tc0, tcnt, inv_n);
        asm volatile("barrier.cluster.wait.acquire;" ::: "memory");   // every rank's partial A is with its owners
        hk.after_first_barrier(warp, lane);
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
            if (tc0 == ti0) hk.after_targets(warp, lane);
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
        if (warp == 0) {
            nd_fill_caches<MSG>(T, G, Fs, Ft, fc, tf, S.sP, lane);
            __syncwarp();      // lane 16's target-cache sum is read by lane 0
            if constexpr (!MSG)
                if (tid == 0) task_consts(T, fc, tf, S.sP, S.sC, S.sLsrc);
        }
        hk.before_first_barrier(tid, r, CS);
        cluster.sync();
        hk.after_first_barrier(warp, lane);
        if constexpr (!MSG) {
            const EpiConst C = S.sC;
            for (int i = ti0 + tid; i < ti1; i += nt) epilogue_point(T, tf, C, G.floor_, i, 1.f, ep);
        }
        hk.after_targets(warp, lane);
    }
    if (MSG || T.mode == EPI_MSG)
        epi_block_finish_msg(T, fc.L, ep);       // message products: the maximum and clamp count only
    else
        epi_block_finish(T, G, tf, S.sLsrc, ep, S.sP.iter, S.sC);
}

// Hooks of the launch-per-level kernel: no claims or prefetches; the wait is for the previous
// grid (programmatic dependent launch), by every thread, before anything that grid may write is read.
struct NdLevelHooks {
    static constexpr bool kEarlyCoords = false;
    static constexpr bool kBarrierAfterWait = false;   // every thread waits itself
    __device__ __forceinline__ void wait(const Task&, int, int) const {
        asm volatile("griddepcontrol.wait;" ::: "memory");
        asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    }
    __device__ __forceinline__ void before_first_barrier(int, int, int) const {}
    __device__ __forceinline__ void after_first_barrier(int, int) const {}
    __device__ __forceinline__ void after_targets(int, int) const {}
};

// One product per cluster (blockIdx.y): the launch-per-level form.
template <bool MSG>
__global__ void __launch_bounds__(ND_THREADS, 1) k_ndft2d(const Task* __restrict__ tasks, Globals G) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    __shared__ NDSh S;
    extern __shared__ float4 nd_dyn[];
    nd_prep(S, tasks + blockIdx.y);
    // every CTA of the cluster runs (its shared memory may be written) and the task is visible.
    // Launched with programmatic stream serialisation: up to here the kernel reads only its own
    // (static) task; nd_run waits for the previous grid before it reads anything else.
    cluster.sync();
    NdLevelHooks hk;
    nd_run<MSG>(S, S.Tb[0], reinterpret_cast<float*>(nd_dyn), G, cluster, G.fac + S.Tb[0].sf0,
                G.fac + S.Tb[0].tf0, hk);
}

// The persistent kernel's task pipeline.  Product t runs task S.Tb[b]; rank 0 claims task t + 1
// at the start of product t and pushes the claim into every rank's S.claim[b ^ 1] (a 4-byte store
// into distributed shared memory, published by the product's first cluster barrier); after that
// barrier the last warp of every CTA copies the claimed task into S.Tb[b ^ 1] with cp.async, and
// after the target contraction its dependency list and factor structs (which read the task's
// fields) into S.dl / S.Fs / S.Ft; the copies complete before the next product's first barrier.
// Buffer reuse: S.claim[x] and S.Tb[x] are written again two products later, after the writer has
// passed the intervening product's cluster barriers, which every reader reaches only after its
// reads; S.dl / S.Fs / S.Ft are read at the start of a product, before its prefetch writes them.
__device__ __forceinline__ void nd_fetch_task(Task& dst, const Task* src, int lane) {
    static_assert(sizeof(Task) % 8 == 0, "Task is copied in 8-byte words");
    const char* s = reinterpret_cast<const char*>(src);
    char* d = reinterpret_cast<char*>(&dst);
    for (int w = lane; w < (int)(sizeof(Task) / 8); w += 32) nd_cp_async8(d + 8 * w, s + 8 * w);
    nd_cp_async_commit();
}
// Called by one whole warp once its task copy was issued: waits for it, then copies the lists.
__device__ __forceinline__ void nd_fetch_lists(NDSh& S, const Task& T, const int* deps, const Factor* fac, int lane) {
    static_assert(sizeof(Factor) % 8 == 0, "Factor is copied in 8-byte words");
    nd_cp_async_wait_all();
    __syncwarp();
    if (T.ndep <= ND_MAXDEP)
        for (int w = lane; w < T.ndep; w += 32) nd_cp_async4(&S.dl[w], deps + T.dep0 + w);
    constexpr int fw = (int)(sizeof(Factor) / 8);
    if (T.alpha == nullptr) {
        const char* s = reinterpret_cast<const char*>(fac + T.sf0);
        for (int w = lane; w < min(T.snf, MOT_MAXFAC) * fw; w += 32)
            nd_cp_async8(reinterpret_cast<char*>(S.Fs) + 8 * w, s + 8 * w);
    }
    {
        const char* s = reinterpret_cast<const char*>(fac + T.tf0);
        for (int w = lane; w < min(T.tnf, MOT_MAXFAC) * fw; w += 32)
            nd_cp_async8(reinterpret_cast<char*>(S.Ft) + 8 * w, s + 8 * w);
    }
    nd_cp_async_commit();
}

// A warp waits for the products task T reads: flags[product] counts the CTAs that completed it
// (each adds 1 after a fence; the chunk prologue zeroes the counts), and lane q polls the counts of
// dependencies q, q + 32, ... with acquire loads until all CS CTAs are in, each wait bounded by
// A.wait_ns (on expiry: error bit 2 and the abort word).
__device__ __forceinline__ void nd_wait_flags(const WaveArgs& A, const Task& T, const int* dl_smem, int CS, int lane) {
    const int* dl = T.ndep <= ND_MAXDEP ? dl_smem : A.deps + T.dep0;
    unsigned long long t0 = 0;
    for (int q = lane; q < T.ndep; q += 32) {
        const int* f = A.flags + dl[q];
        while (ld_acquire_gpu(f) < CS) {
            if (*reinterpret_cast<volatile int*>(&A.ctl->abort)) return;
            const unsigned long long now = f2_globaltimer();
            if (t0 == 0) {
                t0 = now;
            } else if (now - t0 > A.wait_ns) {
                atomicOr(A.err, 4);
                atomicExch(&A.ctl->abort, 1);
                return;
            }
            __nanosleep(32);
        }
    }
}

struct NdWaveHooks {
    static constexpr bool kEarlyCoords = true;
    static constexpr bool kBarrierAfterWait = true;    // warp 0 waits for the CTA
    NDSh* S;
    const WaveArgs* A;
    const Factor* fac;
    int nb;       // buffer of the next task
    int CS;       // CTAs per cluster
    int claim;    // rank 0, thread 0: the next claim (its atomic issued before the product)
    __device__ __forceinline__ void wait(const Task& T, int warp, int lane) const {
        if (warp == 0) nd_wait_flags(*A, T, S->dl, CS, lane);
    }
    __device__ __forceinline__ void before_first_barrier(int tid, int r, int CS) const {
        if (r == 0 && tid == 0)
            for (int q = 0; q < CS; ++q) {
                const unsigned a = nd_mapa(&S->claim[nb], q);
                asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(a), "r"(claim) : "memory");
            }
    }
    __device__ __forceinline__ void after_first_barrier(int warp, int lane) const {
        if (warp == ND_WARPS - 1) {
            const int next = S->claim[nb];
            if (next < A->ntask) nd_fetch_task(S->Tb[nb], A->tasks + next, lane);
        }
    }
    __device__ __forceinline__ void after_targets(int warp, int lane) const {
        if (warp == ND_WARPS - 1 && S->claim[nb] < A->ntask) nd_fetch_lists(*S, S->Tb[nb], A->deps, fac, lane);
    }
};

// Rank 0's claim of the next task: the abort word and the counter are read together, so that
// the thread stalls only where the result is used.
__device__ __forceinline__ int nd_claim_issue(const WaveArgs& A) {
    const int ab = *reinterpret_cast<volatile int*>(&A.ctl->abort);
    const int c = atomicAdd(&A.ctl->next, 1);
    return ab ? A.ntask : c;
}

// Persistent wavefront kernel (the schedule of k_wave2d in nfft.cu: claims in the host's
// topological order, one claim ahead, bounded waits) running this file's product, with the task
// pipeline above; a product's completion is counted per CTA (no cluster barrier at its end).
__global__ void __launch_bounds__(ND_THREADS, 1) k_wave_nd(WaveArgs A, Globals G) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    __shared__ NDSh S;
    extern __shared__ float4 nd_dyn[];
    float* dyn = reinterpret_cast<float*>(nd_dyn);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int r = (int)cluster.block_rank();
    if (r == 0 && tid == 0) S.claim[0] = wave_claim(A);
    cluster.sync();
    int i = *cluster.map_shared_rank(&S.claim[0], 0);
    if (i < A.ntask && warp == ND_WARPS - 1) {
        nd_fetch_task(S.Tb[0], A.tasks + i, lane);
        nd_fetch_lists(S, S.Tb[0], A.deps, G.fac, lane);
    }
    // every read of rank 0's first claim is done before rank 0 writes S.claim again
    cluster.sync();
    int b = 0;
    while (i < A.ntask) {
        if (warp == ND_WARPS - 1) nd_cp_async_wait_all();
        __syncthreads();                     // task i, its dependency list and factor structs are in S
        NdWaveHooks hk;
        hk.S = &S;
        hk.A = &A;
        hk.fac = G.fac;
        hk.nb = b ^ 1;
        hk.CS = (int)cluster.num_blocks();
        hk.claim = (r == 0 && tid == 0) ? nd_claim_issue(A) : 0;
        nd_run<false>(S, S.Tb[b], dyn, G, cluster, S.Fs, S.Ft, hk);   // ends with a block barrier
        // this CTA's part of product i is complete (the block barrier above orders every thread's
        // writes before the fence)
        if (tid == 0) {
            __threadfence();
            atomicAdd(A.flags + i, 1);
        }
        i = S.claim[b ^ 1];
        b ^= 1;
    }
    // no peer reads or writes this CTA's shared memory any more
    cluster.sync();
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
    // no programmatic serialisation: the kernel claims and counts from the prologue's zeroes
    cudaLaunchAttribute attr[2];
    cudaLaunchConfig_t cfg = nd_config(cs, nclusters, 1, st, attr, false);
    return cudaLaunchKernelEx(&cfg, k_wave_nd, A, G);
}
