// Dense kernel products on the 5th-generation tensor cores (the dense comparison path of the
// circle, Algorithm 3, and of the kernel matrix-vector product Eq. (fastsum-sum)).
//
//   Y[c][i] = sum_j A[c][j] * B[i][j]
//
// A (M x K): the source vectors of a batch, one row per column c of a circle message matrix
// (or per right-hand side), A[c][j] = phi_j * X[c][j] normalised by the maxima of its factors.
// B (N x K): the kernel matrix B[i][j] = exp(-w ||y_i - x_j||^2 / eta), fixed for a solve.
// Both operands are split once into BF16 pairs v = hi + lo (hi = bf16(v), lo = bf16(v - hi)),
// and the product is accumulated in FP32 as  Ahi Bhi + Ahi Blo + Alo Bhi  (the Alo Blo term is
// below 2^-16 relative and dropped), which keeps ~16 significant bits per term.
//
// Kernel structure (one 128 x BN output tile per CTA, 128 threads; BN in {128, 160, 192, 224,
// 256} chosen so the tiles fill the SMs in as few waves as possible; a 1-D grid rasterised in
// groups of 8 tile rows so that the B panels of a wave are reused from L2):
//   warp 0 / lane 0   TMA producer: per stage of 32 k-values four tiles (Ahi, Alo, Bhi, Blo),
//                     64-byte swizzled, 4-6 stages, completion counted on the stage's full
//                     mbarrier;
//   warp 1            allocates the TMEM columns; lane 0 issues tcgen05.mma (M=128, N=BN, K=16,
//                     BF16 in, FP32 accumulate in TMEM) and frees stages with tcgen05.commit;
//   warps 0..3        epilogue: tcgen05.ld of their 32 TMEM lanes (= 32 output rows), floor /
//                     maximum / clamp count of a message (Algorithm 3 normalisation), staged
//                     through shared memory so each warp stores whole 128-byte row segments.
// Every mbarrier wait is bounded (globaltimer, 1 s unless a test shortens it through
// mot_test_tc_wait); on expiry the CTA sets bit 2 (value 4) of the error word, drains its own
// outstanding copies (bounded), frees TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <atomic>
#include <mutex>

#include "kernels.h"

namespace {

constexpr int TC_BM = 128;
constexpr int TC_BK = 32;                       // 32 BF16 = one 64-byte swizzle row per stage
constexpr unsigned long long kWaitNs = 1000000000ull;   // 1 s per wait (default)
// test hook (mot_test_tc_wait): the wait limit, and a switch that makes the producer issue no
// loads, so that the MMA thread's first wait runs out
std::atomic<long long> g_wait_ns{(long long)kWaitNs};
std::atomic<int> g_stall_loads{0};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0u;
}

// Wait for the phase of the given parity to complete; false after `limit` ns.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned long long limit) {
    const uint32_t a = smem_u32(bar);
    if (mbar_try_wait(a, parity)) return true;
    const unsigned long long t0 = globaltimer();
    while (!mbar_try_wait(a, parity))
        if (globaltimer() - t0 > limit) return false;
    return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major tile, 64-byte swizzle (rows of 32 BF16), 8-row groups
// 512 bytes apart.
__device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);           // start address
    d |= (uint64_t)1u << 16;                           // leading byte offset (unused when swizzled)
    d |= (uint64_t)(512u >> 4) << 32;                  // stride byte offset: next 8-row group
    d |= (uint64_t)1u << 46;                           // descriptor version
    d |= (uint64_t)4u << 61;                           // 64-byte swizzle
    return d;
}

// Instruction descriptor of kind::f16: BF16 A and B (K-major), FP32 D, M = 128, N = bn.
__host__ __device__ constexpr uint32_t idesc_bf16(int bn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(bn >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 consecutive FP32 columns of this warp's 32 TMEM lanes (one row per thread).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

constexpr uint32_t kMaxSmem = 232448;               // opt-in shared memory per CTA

template <int BN>
struct TcCfg {
    static constexpr uint32_t A_BYTES = TC_BM * TC_BK * 2;
    static constexpr uint32_t B_BYTES = BN * TC_BK * 2;
    static constexpr uint32_t STAGE = 2 * A_BYTES + 2 * B_BYTES;
    static constexpr int STAGES_FIT = (int)((kMaxSmem - 1024 - 256) / STAGE);
    static constexpr int STAGES = STAGES_FIT < 6 ? STAGES_FIT : 6;
    static constexpr uint32_t SMEM = STAGES * STAGE + 1024 /* alignment */ + 256 /* barriers */;
    static constexpr uint32_t TMEM_COLS = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
    static_assert(BN % 16 == 0 && BN <= 256, "MMA N");
    static_assert(STAGES >= 2, "pipeline depth");
    static_assert(STAGE % 1024 == 0 || (A_BYTES % 512 == 0 && B_BYTES % 512 == 0), "tile alignment");
};

template <int BN>
__global__ void __launch_bounds__(128, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
              const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl, TcEpi E) {
    using Cfg = TcCfg<BN>;
    constexpr int STAGES = Cfg::STAGES;
    extern __shared__ uint8_t smem_raw[];
    // 1024-byte alignment of the shared-window address (swizzle atoms must start on their own size)
    const uint32_t raw_base = smem_u32(smem_raw);
    uint8_t* smem = smem_raw + (((raw_base + 1023u) & ~1023u) - raw_base);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * Cfg::STAGE);
    uint64_t* empty = full + STAGES;
    uint64_t* accb = empty + STAGES;
    uint32_t* s_taddr = reinterpret_cast<uint32_t*>(accb + 1);
    int* s_fail = reinterpret_cast<int*>(s_taddr + 1);
    int* s_issued = s_fail + 1;     // k-blocks whose loads were issued
    int* s_consumed = s_fail + 2;   // k-blocks whose loads were waited for by the MMA thread
    float* s_mx = reinterpret_cast<float*>(s_fail + 4);        // [4]
    unsigned int* s_cl = reinterpret_cast<unsigned int*>(s_mx + 4);   // [4]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // grouped raster over a 1-D grid: 8 tile rows share the B panels in flight (L2 reuse)
    const int num_m = (E.M + TC_BM - 1) / TC_BM, num_n = (E.N + BN - 1) / BN;
    const int group = (int)blockIdx.x / (8 * num_n), first_m = group * 8;
    const int gm = min(num_m - first_m, 8), in_group = (int)blockIdx.x - group * 8 * num_n;
    const int m0 = (first_m + in_group % gm) * TC_BM, n0 = (in_group / gm) * BN;
    const int nkb = (E.K + TC_BK - 1) / TC_BK;
    const unsigned long long lim = E.wait_ns;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        mbar_init(accb, 1);
        *s_fail = 0;
        *s_issued = 0;
        *s_consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_taddr)),
                     "r"(Cfg::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_taddr;

    if (warp == 0 && lane == 0) {
        // ---- producer ----
        int kb = 0;
        const int nkb_load = E.stall_loads ? 0 : nkb;   // test hook: no loads, nothing in flight
        for (; kb < nkb_load; ++kb) {
            const int s = kb % STAGES;
            const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
            if (!mbar_wait(empty + s, ph ^ 1u, lim)) {
                atomicOr(s_fail, 1);
                break;
            }
            if (*reinterpret_cast<volatile int*>(s_fail)) break;
            uint8_t* st = smem + s * Cfg::STAGE;
            mbar_expect_tx(full + s, Cfg::STAGE);
            tma_load_2d(st, &mAh, full + s, kb * TC_BK, m0);
            tma_load_2d(st + Cfg::A_BYTES, &mAl, full + s, kb * TC_BK, m0);
            tma_load_2d(st + 2 * Cfg::A_BYTES, &mBh, full + s, kb * TC_BK, n0);
            tma_load_2d(st + 2 * Cfg::A_BYTES + Cfg::B_BYTES, &mBl, full + s, kb * TC_BK, n0);
        }
        *s_issued = kb;
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer ----
        constexpr uint32_t idesc = idesc_bf16(BN);
        int kb = 0;
        for (; kb < nkb; ++kb) {
            const int s = kb % STAGES;
            const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
            if (!mbar_wait(full + s, ph, lim)) {
                atomicOr(s_fail, 2);
                break;
            }
            tc_fence_after();
            const uint32_t base = smem_u32(smem + s * Cfg::STAGE);
            const uint64_t ah = sw64_desc(base), al = sw64_desc(base + Cfg::A_BYTES);
            const uint64_t bh = sw64_desc(base + 2 * Cfg::A_BYTES);
            const uint64_t bl = sw64_desc(base + 2 * Cfg::A_BYTES + Cfg::B_BYTES);
#pragma unroll
            for (int kk = 0; kk < TC_BK / 16; ++kk) {
                const uint64_t adv = (uint64_t)(kk * 32 >> 4);   // 16 BF16 = 32 bytes along K
                mma_bf16(tmem, ah + adv, bh + adv, idesc, (kb | kk) != 0);
                mma_bf16(tmem, ah + adv, bl + adv, idesc, 1u);
                mma_bf16(tmem, al + adv, bh + adv, idesc, 1u);
            }
            mma_commit(empty + s);
        }
        *s_consumed = kb;
        mma_commit(accb);   // arrives once every MMA issued above has completed
    }
    __syncwarp();

    // ---- epilogue: all four warps ----
    const bool acc_ok = mbar_wait(accb, 0u, lim);
    if (!acc_ok && lane == 0) atomicOr(s_fail, 4);
    tc_fence_after();
    float mx = 0.f;
    unsigned int clamps = 0u;
    __syncthreads();
    const bool ok = *reinterpret_cast<volatile int*>(s_fail) == 0;
    if (ok) {
        float* stage = reinterpret_cast<float*>(smem) + warp * (32 * 33);   // stages are idle now
        const int row_base = m0 + warp * 32;
        for (int j = 0; j < (BN + 31) / 32; ++j) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(j * 32), v);
            const bool row_ok = row_base + lane < E.M;
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                float g = v[q];
                if (E.mode == 1) {
                    const bool col_ok = n0 + j * 32 + q < E.N;
                    if (!(g >= E.floor_)) {
                        g = E.floor_;
                        if (row_ok && col_ok) clamps++;
                    }
                    if (row_ok && col_ok) mx = fmaxf(mx, g);
                }
                stage[lane * 33 + q] = g;
            }
            __syncwarp();
            const int col = n0 + j * 32 + lane;
            if (col < E.N) {
                for (int r = 0; r < 32; ++r) {
                    const int row = row_base + r;
                    if (row >= E.M) break;
                    E.out[(size_t)row * E.ldo + col] = stage[r * 33 + lane];
                }
            }
            __syncwarp();
        }
    }
    if (E.mode == 1) {
        mx = warp_max(mx);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) clamps += __shfl_xor_sync(0xffffffffu, clamps, o);
        if (lane == 0) {
            s_mx[warp] = mx;
            s_cl[warp] = clamps;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
        if (*s_fail) {
            // drain the copies still in flight into this CTA's shared memory (bounded)
            for (int kb = *s_consumed; kb < *s_issued; ++kb)
                mbar_wait(full + (kb % STAGES), (uint32_t)(kb / STAGES) & 1u, lim);
            if (E.err) atomicOr(E.err, 4);
        } else if (E.mode == 1) {
            float m = fmaxf(fmaxf(s_mx[0], s_mx[1]), fmaxf(s_mx[2], s_mx[3]));
            unsigned int c = s_cl[0] + s_cl[1] + s_cl[2] + s_cl[3];
            double L = 0.0;
            if (E.s_a) L += E.s_a->ls + (double)logf(mx_of(E.s_a, 0));
            if (E.s_b) L += E.s_b->ls + (double)logf(mx_of(E.s_b, 0));
            E.out_sc->ls = L;
            atomic_max_pos(&E.out_sc->mx_bits, m);
            if (c) atomicAdd(&E.out_sc->clamped, c);
        }
    }
    __syncthreads();
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Cfg::TMEM_COLS)
                     : "memory");
}

// A[c][j] = (phi_j / max phi) (X[c][j] / max X), split into BF16 hi / lo; row stride ld.
// Four consecutive j per thread: one 8-byte store each for hi and lo (ld is a multiple of 8).
__device__ __forceinline__ void split4(const float (&a)[4], __nv_bfloat16* hi, __nv_bfloat16* lo) {
    __nv_bfloat162 h01 = __floats2bfloat162_rn(a[0], a[1]), h23 = __floats2bfloat162_rn(a[2], a[3]);
    const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
    __nv_bfloat162 l01 = __floats2bfloat162_rn(a[0] - f01.x, a[1] - f01.y);
    __nv_bfloat162 l23 = __floats2bfloat162_rn(a[2] - f23.x, a[3] - f23.y);
    uint2 hv, lv;
    hv.x = *reinterpret_cast<uint32_t*>(&h01);
    hv.y = *reinterpret_cast<uint32_t*>(&h23);
    lv.x = *reinterpret_cast<uint32_t*>(&l01);
    lv.y = *reinterpret_cast<uint32_t*>(&l23);
    *reinterpret_cast<uint2*>(hi) = hv;
    *reinterpret_cast<uint2*>(lo) = lv;
}

__global__ void __launch_bounds__(256) k_split_src(const float* __restrict__ X, const VecScale* sX,
                                                   const float* __restrict__ phi, const VecScale* sP, int ns, int nrow,
                                                   int ld, __nv_bfloat16* __restrict__ hi,
                                                   __nv_bfloat16* __restrict__ lo) {
    const float sx = 1.f / mx_of(sX, 0), sp = phi ? 1.f / mx_of(sP, 0) : 1.f;
    const int nq = (ns + 3) >> 2;
    for (int c = blockIdx.y; c < nrow; c += gridDim.y) {
        const float* x = X + (size_t)c * ns;
        for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
            const int j0 = q << 2;
            float a[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int j = j0 + t;
                a[t] = 0.f;
                if (j < ns) {
                    a[t] = x[j] * sx;
                    if (phi) a[t] *= __ldg(phi + j) * sp;
                }
            }
            // the padding columns [ns, ld) receive zeros (never read: the tensor map stops at ns)
            split4(a, hi + (size_t)c * ld + j0, lo + (size_t)c * ld + j0);
        }
    }
}

// Kernel matrix B[i][j] = exp(-||u_i - v_j||^2 / eta_u) (grid units), split into BF16 hi / lo.
__global__ void __launch_bounds__(256) k_kernel_split(const float* __restrict__ ut, int nt,
                                                      const float* __restrict__ us, int ns, int d, float eta_u,
                                                      int ld, __nv_bfloat16* __restrict__ hi,
                                                      __nv_bfloat16* __restrict__ lo) {
    const float k2 = -1.4426950408889634f / eta_u;
    for (int i = blockIdx.y; i < nt; i += gridDim.y) {
        float yi[3] = {0.f, 0.f, 0.f};
        for (int t = 0; t < d; ++t) yi[t] = ut[(size_t)t * nt + i];
        for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < ns; j += gridDim.x * blockDim.x) {
            float r2 = 0.f;
            for (int t = 0; t < d; ++t) {
                const float e = yi[t] - us[(size_t)t * ns + j];
                r2 = fmaf(e, e, r2);
            }
            const float kv = exp2f(k2 * r2);
            const __nv_bfloat16 h = __float2bfloat16_rn(kv);
            hi[(size_t)i * ld + j] = h;
            lo[(size_t)i * ld + j] = __float2bfloat16_rn(kv - __bfloat162float(h));
        }
    }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link against libcuda).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// rows x cols BF16 matrix with row stride ld elements; box = 32 columns x box_rows rows.
bool encode_bf16(unsigned char* out, const void* base, int rows, int cols, int ld, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    if ((reinterpret_cast<uintptr_t>(base) & 15) || (ld % 8) != 0 || rows < 1 || cols < 1) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(reinterpret_cast<CUtensorMap*>(out), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base),
                    dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int BN>
cudaError_t launch_cfg(const TcGemm& g, const TcEpi& e, cudaStream_t st) {
    const CUtensorMap* m = reinterpret_cast<const CUtensorMap*>(g.maps);
    const unsigned grid = (unsigned)(((g.N + BN - 1) / BN) * ((g.M + TC_BM - 1) / TC_BM));
    k_tc_gemm<BN><<<grid, 128, TcCfg<BN>::SMEM, st>>>(m[0], m[1], m[2], m[3], e);
    return cudaGetLastError();
}

template <int BN>
cudaError_t set_smem() {
    return cudaFuncSetAttribute(k_tc_gemm<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcCfg<BN>::SMEM);
}

constexpr int kTileN[5] = {256, 224, 192, 160, 128};

}  // namespace

static_assert(sizeof(CUtensorMap) == 128, "tensor map size");

int tc_ld(int k) { return (k + 7) & ~7; }

cudaError_t prepare_tc_gemm() {
    static std::mutex mu;
    static bool done[64] = {};                  // per device: kernel attributes are per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev]) return cudaSuccess;
    e = set_smem<256>();
    if (e == cudaSuccess) e = set_smem<224>();
    if (e == cudaSuccess) e = set_smem<192>();
    if (e == cudaSuccess) e = set_smem<160>();
    if (e == cudaSuccess) e = set_smem<128>();
    if (e == cudaSuccess) done[dev] = true;
    return e;
}

bool tc_prepare(TcGemm* g, const void* a_hi, const void* a_lo, int M, int lda, const void* b_hi, const void* b_lo,
                int N, int ldb, int K) {
    g->M = M;
    g->N = N;
    g->K = K;
    // tile width: fewest waves over the 152 SMs times the per-tile work (ties: wider tiles)
    long long best = -1;
    for (int bn : kTileN) {
        const long long tiles = (long long)((N + bn - 1) / bn) * ((M + TC_BM - 1) / TC_BM);
        const long long cost = ((tiles + 151) / 152) * bn;
        if (best < 0 || cost < best) {
            best = cost;
            g->bn = bn;
        }
    }
    return encode_bf16(g->maps[0], a_hi, M, K, lda, TC_BM) && encode_bf16(g->maps[1], a_lo, M, K, lda, TC_BM) &&
           encode_bf16(g->maps[2], b_hi, N, K, ldb, g->bn) && encode_bf16(g->maps[3], b_lo, N, K, ldb, g->bn);
}

cudaError_t launch_tc_gemm(const TcGemm& g, TcEpi e, cudaStream_t st) {
    if (g.M <= 0 || g.N <= 0) return cudaSuccess;
    e.M = g.M;
    e.N = g.N;
    e.K = g.K;
    e.wait_ns = (unsigned long long)g_wait_ns.load();
    e.stall_loads = g_stall_loads.load();
    switch (g.bn) {
    case 256: return launch_cfg<256>(g, e, st);
    case 224: return launch_cfg<224>(g, e, st);
    case 192: return launch_cfg<192>(g, e, st);
    case 160: return launch_cfg<160>(g, e, st);
    default: return launch_cfg<128>(g, e, st);
    }
}

cudaError_t launch_split_src(const float* X, const VecScale* sX, const float* phi, const VecScale* sP, int ns,
                             int nrow, int ld, void* hi, void* lo, cudaStream_t st) {
    if (nrow <= 0 || ns <= 0) return cudaSuccess;
    const int bx = std::min((ns + 1023) / 1024, 8);
    k_split_src<<<dim3(bx, std::min(nrow, 65535)), 256, 0, st>>>(X, sX, phi, sP, ns, nrow, ld, static_cast<__nv_bfloat16*>(hi),
                                                static_cast<__nv_bfloat16*>(lo));
    return cudaGetLastError();
}

cudaError_t launch_kernel_split(const float* ut, int nt, const float* us, int ns, int d, float eta_u, int ld,
                                void* hi, void* lo, cudaStream_t st) {
    if (nt <= 0 || ns <= 0) return cudaSuccess;
    const int bx = std::min((ns + 255) / 256, 8);
    k_kernel_split<<<dim3(bx, std::min(nt, 65535)), 256, 0, st>>>(ut, nt, us, ns, d, eta_u, ld, static_cast<__nv_bfloat16*>(hi),
                                                 static_cast<__nv_bfloat16*>(lo));
    return cudaGetLastError();
}

// Test hook of the bounded waits (declared in motfft.h).
extern "C" int mot_test_tc_wait(long long wait_ns, int stall_loads) {
    if (wait_ns < 1000 || wait_ns > 10000000000ll) return MOT_EINVAL;
    g_wait_ns.store(wait_ns);
    g_stall_loads.store(stall_loads ? 1 : 0);
    return MOT_OK;
}
