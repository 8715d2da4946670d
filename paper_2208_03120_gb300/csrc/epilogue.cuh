// Source-side products and target-side epilogues of one kernel product (Algorithm 2 / 4).
#pragma once
#include "common.cuh"

struct Globals {
    int* iter;          // device iteration counter (-1 before the first iteration)
    IterAcc* acc;       // ring of per-iteration accumulators
    int R;              // ring length
    float floor_;       // positive floor of fast-summation outputs
    int n_grid;         // grid length per dimension
    int M;              // Fourier half-degree
    const Factor* fac;  // factor array referenced by the tasks
};

// Element-wise product of a factor list, loaded once per block into shared memory.
struct FacCache {
    const float* mant[MOT_MAXFAC];
    float scale[MOT_MAXFAC];
    int inv[MOT_MAXFAC];
    int nf;
    double L;           // log-scale of the normalised product
};

// Log-scale of a factor list, summed by warp 0 (lanes in parallel); valid on lane 0.
__device__ __forceinline__ double factors_L_warp(const Factor* F, int f0, int nf) {
    double L = 0.0;
    for (int t = threadIdx.x; t < nf; t += 32) L += factor_L(F[f0 + t]);
    return warp_sum_d(L);
}

__device__ __forceinline__ void load_factors(FacCache& fc, const Factor* F, int f0, int nf) {
    for (int t = threadIdx.x; t < nf; t += blockDim.x) {
        Factor f = F[f0 + t];
        fc.mant[t] = f.mant;
        fc.scale[t] = 1.f / mx_of(f.sc, f.use_prev);
        fc.inv[t] = f.inv;
    }
    if (threadIdx.x < 32) {
        const double L = factors_L_warp(F, f0, nf);
        if (threadIdx.x == 0) {
            fc.nf = nf;
            fc.L = L;
        }
    }
    __syncthreads();
}

// Per-block constants of an epilogue (computed once by thread 0, read by all threads).
struct EpiConst {
    double lsphi;      // log-scale of the scalings written (EPI_PHI / EPI_ROOT)
    double E;          // exp(total log-scale) of P_i = raw_i T_i e^{L} (EPI_MARG / EPI_ROOT)
    double invEs;      // 1 / max(E, 1): |P_i - mu_i| is summed in FP32 scaled by it
    double Es;         // max(E, 1)
    double ls_phi_k;   // log-scale of the node's current scaling (EPI_MARG)
    float inv_mx_old;  // 1 / mx of the previous root scaling (EPI_ROOT)
};

__device__ __forceinline__ float eval_prod(const FacCache& fc, int i) {
    float v = 1.f;
    for (int f = 0; f < fc.nf; ++f) {
        float x = __ldg(fc.mant[f] + i) * fc.scale[f];
        v = fc.inv[f] ? v / x : v * x;
    }
    return v;
}

// Per-thread partial results of an epilogue, reduced once per block.  The sums are FP32 with
// every large scale factored out (FP64 arithmetic is slow on this part: a block's reduction in
// FP64 took longer than its kernel sum); the block combines them with the scales in FP64:
//   sum_i mu_i log phi_i     = lphi + lsphi * musum        (lsphi: the scalings' log-scale)
//   mass = sum_i P_i          = E * a                        (P_i = E a_i, a_i = raw_i T_i <= N)
//   viol = sum_i |P_i - mu_i| = max(E, 1) * dv
//   sum_i P_i log phi^k_i     = E * alog + ls_phi_k * mass
// Each block sums at most a few points per thread and some hundreds of threads, so the FP32
// sums carry a relative error of about 1e-7, the size of the FP32 logarithms they add.
struct EpiPartial {
    float mx_out, mx_phi;
    float lphi, musum, a, dv, alog;
    unsigned int clamps;
};

__device__ __forceinline__ void epi_zero(EpiPartial& e) {
    e.mx_out = 0.f; e.mx_phi = 0.f; e.lphi = 0.f; e.musum = 0.f; e.a = 0.f; e.dv = 0.f; e.alog = 0.f; e.clamps = 0u;
}

// Block-start duties carried by a task: reset scale records (and keep the previous values of
// the root scaling) and zero the accumulators of the next iteration.  Run by one thread.
__device__ __forceinline__ void task_resets(const Task& T, const Globals& G, int bump_iter) {
    for (int r = 0; r < T.zero_n; ++r) T.zero_d[r] = 0.0;
    for (int r = 0; r < T.reset_n; ++r) {
        VecScale* s = T.reset_list[r];
        if (T.save_prev) { s->ls_prev = s->ls; s->mx_prev_bits = s->mx_bits; }
        s->mx_bits = 0u;
        s->clamped = 0u;
    }
    if (bump_iter) {
        int it = *G.iter + 1;
        *G.iter = it;
        IterAcc* a = G.acc + ((it + 1) % G.R);
        a->logphi = 0.0; a->mass = 0.0; a->rootviol = 0.0; a->pad = 0.0;
    }
}

// Epilogue of target point i given the raw kernel sum (raw = 1 for EPI_ROOT).
// Lsrc: log-scale of the source product; tf: target-side factors.
// lsphi: log-scale of the scaling written by EPI_PHI (-(Lsrc + tf.L)) or EPI_ROOT (-tf.L).
__device__ __forceinline__ double phi_logscale(const Task& T, const FacCache& tf, double Lsrc) {
    if (T.mode == EPI_PHI_FREE || (T.mode == EPI_ROOT && T.free_node)) return 0.0;
    if (T.mode == EPI_CROOT) return -Lsrc;
    return T.mode == EPI_ROOT ? -tf.L : -(Lsrc + tf.L);
}

// Thread 0: fill the per-block constants (the only FP64 transcendentals of an epilogue).
__device__ __forceinline__ void epi_prepare(const Task& T, const FacCache& tf, double Lsrc, EpiConst& C) {
    C.lsphi = phi_logscale(T, tf, Lsrc);
    C.E = 1.0;
    C.ls_phi_k = 0.0;
    C.inv_mx_old = 1.f;
    if (T.mode == EPI_MARG) {
        C.E = exp(Lsrc + tf.L);
        C.ls_phi_k = ls_of(T.phi_sc, 0);
    } else if (T.mode == EPI_ROOT || T.mode == EPI_CROOT) {
        const double Lold = ls_of(T.phi_sc, 1) + (double)logf(mx_of(T.phi_sc, 1));
        C.E = exp(Lold + (T.mode == EPI_ROOT ? tf.L : Lsrc));
        C.inv_mx_old = 1.f / mx_of(T.phi_sc, 1);
    }
    C.Es = fmax(C.E, 1.0);
    C.invEs = 1.0 / C.Es;
}

// One warp fills a factor cache: lanes stride over the factors, reading each factor and its
// scale record once, and the log-scale is summed over the warp.  No barrier.
__device__ __forceinline__ void fill_factors_warp(FacCache& fc, const Factor* F, int f0, int nf, int lane) {
    double L = 0.0;
    for (int t = lane; t < nf; t += 32) {
        const Factor f = F[f0 + t];
        const float mx = mx_of(f.sc, f.use_prev);
        fc.mant[t] = f.mant;
        fc.scale[t] = 1.f / mx;
        fc.inv[t] = f.inv;
        const double Lt = ls_of(f.sc, f.use_prev) + (double)logf(mx);
        L += f.inv ? -Lt : Lt;
    }
    L = warp_sum_d(L);
    if (lane == 0) {
        fc.nf = nf;
        fc.L = L;
    }
}

// Scale-record values of the epilogue that depend on the task alone, and the iteration counter
// (constant while a sweep's kernels run: the prologue kernel advances it).
struct EpiPre {
    double ls_phi_k, Lold;
    float inv_mx_old;
    int iter;
};

// Factor caches of a task with one barrier: warps 0 / 1 fill the source / target caches, warp 2
// reads the scale records.  Needs at least 3 warps.
__device__ __forceinline__ void load_task_caches(const Task& T, const Globals& G, FacCache& fc, FacCache& tf,
                                                 EpiPre& pre) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        if (T.alpha == nullptr) {
            fill_factors_warp(fc, G.fac, T.sf0, T.snf, lane);
        } else if (lane == 0) {
            fc.nf = 0;
            fc.L = 0.0;
        }
    } else if (warp == 1) {
        fill_factors_warp(tf, G.fac, T.tf0, T.tnf, lane);
    } else if (warp == 2 && lane == 0) {
        pre.ls_phi_k = ls_of(T.phi_sc, 0);
        pre.Lold = ls_of(T.phi_sc, 1) + (double)logf(mx_of(T.phi_sc, 1));
        pre.inv_mx_old = 1.f / mx_of(T.phi_sc, 1);
        pre.iter = (G.iter ? *G.iter : 0) - T.iter_off;
    }
    __syncthreads();
}

// The epilogue constants from the caches (one thread; the FP64 part of a task's set-up).
__device__ __forceinline__ void task_consts(const Task& T, const FacCache& fc, const FacCache& tf, const EpiPre& pre,
                                            EpiConst& C, double& sLsrc) {
    {
        const double Lsrc = T.alpha == nullptr ? fc.L : 0.0;
        sLsrc = Lsrc;
        C.lsphi = phi_logscale(T, tf, Lsrc);
        C.E = 1.0;
        C.ls_phi_k = 0.0;
        C.inv_mx_old = 1.f;
        if (T.mode == EPI_MARG) {
            C.E = exp(Lsrc + tf.L);
            C.ls_phi_k = pre.ls_phi_k;
        } else if (T.mode == EPI_ROOT || T.mode == EPI_CROOT) {
            C.E = exp(pre.Lold + (T.mode == EPI_ROOT ? tf.L : Lsrc));
            C.inv_mx_old = pre.inv_mx_old;
        }
        C.Es = fmax(C.E, 1.0);
        C.invEs = 1.0 / C.Es;
    }
}

// Factor caches and epilogue constants of a task with one barrier; thread 0 derives the
// constants, which the other threads may read after the caller's next barrier.
__device__ __forceinline__ void load_task_consts(const Task& T, const Globals& G, FacCache& fc, FacCache& tf,
                                                 EpiPre& pre, EpiConst& C, double& sLsrc) {
    load_task_caches(T, G, fc, tf, pre);
    if (threadIdx.x == 0) task_consts(T, fc, tf, pre, C, sLsrc);
}

// Target-side inputs of the epilogue of point i, loaded ahead of the kernel sum so that their
// latency overlaps it.
struct EpiIn {
    float t;      // product of the target-side factors
    float muf;    // mu_i (FP32)
    float phi;    // current scaling mantissa
    double mud;   // mu_i (FP64)
};

__device__ __forceinline__ EpiIn epi_load(const Task& T, const FacCache& tf, int i) {
    EpiIn in;
    in.t = 1.f;
    in.muf = 0.f;
    in.phi = 0.f;
    in.mud = 0.0;
    switch (T.mode) {
    case EPI_PHI:
        in.t = eval_prod(tf, i);
        in.muf = T.mu_f[i];
        break;
    case EPI_ROOT:
        in.t = eval_prod(tf, i);
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
        in.t = eval_prod(tf, i);                 // phi^k and the children's messages
        in.phi = T.phi[i];
        if (T.mu_d) in.mud = T.mu_d[i];
        break;
    default:
        break;
    }
    return in;
}

__device__ __forceinline__ void epilogue_point_in(const Task& T, const EpiConst& C, float floor_, int i, float raw,
                                                  const EpiIn& in, EpiPartial& ep) {
    switch (T.mode) {
    case EPI_RAW:
        T.out[i] = raw;
        break;
    case EPI_MSG: {
        float g = raw;
        if (!(g >= floor_)) { g = floor_; ep.clamps++; }
        T.out[i] = g;
        ep.mx_out = fmaxf(ep.mx_out, g);
        break;
    }
    case EPI_PHI: {
        float g = raw;
        if (!(g >= floor_)) { g = floor_; ep.clamps++; }
        if (T.out) T.out[i] = g;
        const float ph = in.muf / (g * in.t);
        T.phi[i] = ph;
        ep.mx_phi = fmaxf(ep.mx_phi, ph);
        if (in.muf > 0.f) {
            ep.lphi = fmaf(in.muf, logf(ph), ep.lphi);
            ep.musum += in.muf;
        }
        break;
    }
    case EPI_PHI_FREE:
        if (T.out) {                            // a free node's gamma feeds its children
            float g = raw;
            if (!(g >= floor_)) { g = floor_; ep.clamps++; }
            T.out[i] = g;
            ep.mx_out = fmaxf(ep.mx_out, g);
        }
        T.phi[i] = 1.f;
        ep.mx_phi = 1.f;
        break;
    case EPI_ROOT: {
        // mass and violation of the last iterate (scale record prev), then the update
        const float old = in.phi * C.inv_mx_old;
        const float a = old * in.t;
        ep.a += a;
        if (T.free_node) {
            ep.mx_phi = 1.f;
        } else {
            ep.dv += (float)(fabs((double)a * C.E - in.mud) * C.invEs);
            const float ph = in.muf / in.t;
            T.phi[i] = ph;
            ep.mx_phi = fmaxf(ep.mx_phi, ph);
            if (in.muf > 0.f) {
                ep.lphi = fmaf(in.muf, logf(ph), ep.lphi);
                ep.musum += in.muf;
            }
        }
        break;
    }
    case EPI_CROOT: {
        // raw = sum over the root's column of the circle product (normalised factors)
        const float old = in.phi * C.inv_mx_old;
        const float a = old * raw;
        ep.a += a;
        ep.dv += (float)(fabs((double)a * C.E - in.mud) * C.invEs);
        float g = raw;
        if (!(g >= floor_)) { g = floor_; ep.clamps++; }
        const float ph = in.muf / g;
        T.phi[i] = ph;
        ep.mx_phi = fmaxf(ep.mx_phi, ph);
        if (in.muf > 0.f) {
            ep.lphi = fmaf(in.muf, logf(ph), ep.lphi);
            ep.musum += in.muf;
        }
        break;
    }
    case EPI_MARG: {
        float g = raw;
        if (!(g >= floor_)) { g = floor_; ep.clamps++; }
        if (T.out) T.out[i] = g;
        ep.mx_out = fmaxf(ep.mx_out, g);
        const float a = g * in.t;
        ep.a += a;
        if (T.mu_d) ep.dv += (float)(fabs((double)a * C.E - in.mud) * C.invEs);
        if (a > 0.f) ep.alog = fmaf(a, logf(in.phi), ep.alog);
        break;
    }
    default:
        break;
    }
}

__device__ __forceinline__ void epilogue_point(const Task& T, const FacCache& tf, const EpiConst& C,
                                               float floor_, int i, float raw, EpiPartial& ep) {
    epilogue_point_in(T, C, floor_, i, raw, epi_load(T, tf, i), ep);
}

// Reduce the partials of the block and publish them.  All threads call it.  Only the
// quantities the task's mode produces are reduced (the FP64 ones cost most); warp 0 combines
// the warps' partials lane-parallel.  `iter` is the sweep counter read at the kernel's start.
__device__ __forceinline__ void epi_block_finish(const Task& T, const Globals& G, const FacCache& tf,
                                                 double Lsrc, EpiPartial ep, int iter, const EpiConst& C) {
    __shared__ float s_f[7][32];
    __shared__ unsigned int s_c[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    const int mode = T.mode;
    const bool has_out = (mode == EPI_MSG || mode == EPI_MARG ||
                          ((mode == EPI_PHI || mode == EPI_PHI_FREE) && T.out != nullptr)) && T.out_sc != nullptr;
    const bool has_phi = mode == EPI_PHI || mode == EPI_ROOT || mode == EPI_PHI_FREE || mode == EPI_CROOT;
    const bool d_log = mode == EPI_PHI || mode == EPI_ROOT || mode == EPI_CROOT;
    const bool d_vm = mode == EPI_MARG || mode == EPI_ROOT || mode == EPI_CROOT;
    const bool d_pl = mode == EPI_MARG;
    float v[7] = {has_out ? ep.mx_out : 0.f, has_phi ? ep.mx_phi : 0.f, d_log ? ep.lphi : 0.f,
                  d_log ? ep.musum : 0.f, d_vm ? ep.a : 0.f, d_vm ? ep.dv : 0.f, d_pl ? ep.alog : 0.f};
    v[0] = warp_max(v[0]);
    v[1] = warp_max(v[1]);
#pragma unroll
    for (int q = 2; q < 7; ++q) v[q] = warp_sum(v[q]);
    unsigned int c = ep.clamps;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < 7; ++q) s_f[q][w] = v[q];
        s_c[w] = c;
    }
    __syncthreads();
    if (w == 0) {
        const bool in = lane < nw;
#pragma unroll
        for (int q = 0; q < 7; ++q) v[q] = in ? s_f[q][lane] : 0.f;
        v[0] = warp_max(v[0]);
        v[1] = warp_max(v[1]);
#pragma unroll
        for (int q = 2; q < 7; ++q) v[q] = warp_sum(v[q]);
        c = in ? s_c[lane] : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) {
            // FP64 only here, and only what the mode produces: the block's sums with their scales
            // (products only: this part's FP64 division is slow)
            if (has_out) {
                T.out_sc->ls = Lsrc;
                atomic_max_pos(&T.out_sc->mx_bits, v[0]);
                if (c) atomicAdd(&T.out_sc->clamped, c);
            }
            if (mode == EPI_MARG && T.acc_node) {
                const double m = C.E * (double)v[4];
                atomicAdd(T.acc_node + 0, (double)v[5] * C.Es);
                atomicAdd(T.acc_node + 1, C.E * (double)v[6] + C.ls_phi_k * m);
                atomicAdd(T.acc_node + 2, m);
            }
            if (has_phi) {
                T.phi_sc->ls = C.lsphi;
                atomic_max_pos(&T.phi_sc->mx_bits, v[1]);
                IterAcc* nxt = G.acc + ((iter + 1) % G.R);
                if (d_log) {
                    const double l = (double)v[2] + C.lsphi * (double)v[3];
                    if (l != 0.0) atomicAdd(&nxt->logphi, l);
                }
                if (mode == EPI_ROOT || mode == EPI_CROOT) {
                    IterAcc* cur = G.acc + (iter % G.R);
                    atomicAdd(&cur->mass, C.E * (double)v[4]);
                    atomicAdd(&cur->rootviol, (double)v[5] * C.Es);
                }
            }
        }
    }
    __syncthreads();
}

// Message-only variant of the block reduction (every task of the launch is EPI_MSG): the maximum
// and clamp count of the messages written, no FP64 quantities.
__device__ __forceinline__ void epi_block_finish_msg(const Task& T, double Lsrc, const EpiPartial& ep) {
    __shared__ float s_mx[32];
    __shared__ unsigned int s_c[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    float a = warp_max(ep.mx_out);
    unsigned int c = ep.clamps;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) {
        s_mx[w] = a;
        s_c[w] = c;
    }
    __syncthreads();
    if (w == 0) {
        a = warp_max(lane < nw ? s_mx[lane] : 0.f);
        c = lane < nw ? s_c[lane] : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0 && T.out_sc) {
            T.out_sc->ls = Lsrc;
            atomic_max_pos(&T.out_sc->mx_bits, a);
            if (c) atomicAdd(&T.out_sc->clamped, c);
        }
    }
    __syncthreads();
}
