// Shared device-side types and helpers of libmotfft (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "motfft.h"

#define MOT_WARP 32

// Window: 2m+2 = 10 taps per dimension (m = 4), Kaiser-Bessel shape of half-width a = m+1 grid
// cells, shape parameter b = pi (2 - 1/sigma) with oversampling sigma = n / (2M) = 2.
#define MOT_W 10
#define MOT_WHALF 4   // taps start at floor(u) - MOT_WHALF

// Largest factor list of one vector product (1 + max number of children in a tree).
#define MOT_MAXFAC 72

// Scale record of a vector stored as FP32 mantissas: true value_i = mant_i * exp(ls).
// mx_bits is the maximum mantissa (FP32 bits; mantissas are >= 0), produced with atomicMax.
// Consumers read the normalised view mant_i / mx with log-scale ls + log(mx).
struct VecScale {
    double ls;
    unsigned int mx_bits;
    unsigned int clamped;
    double ls_prev;              // ls / mx of the previous iterate (root scaling only)
    unsigned int mx_prev_bits;
    unsigned int pad;
};

// One factor of an element-wise product: (mant[i] / mx)^(+1 or -1); sc == nullptr means the
// factor is stored at its true scale (ls = 0, mx = 1), e.g. a marginal mu^k.
struct Factor {
    const float* mant;
    const VecScale* sc;
    int inv;                     // 1: the factor divides
    int use_prev;                // 1: read ls_prev / mx_prev (root scaling of the last iterate)
};

// Subproblem of a binned point set: points [start, start+len) all lie in tile `tile`.
struct Sub {
    int tile, start, len, pad;
};

// A binned point set on the torus grid.
struct PointSet {
    int n;                       // number of points
    const float* u;              // SoA [d][n] coordinates in grid units, in [0, n_grid)
    const Sub* subs;             // subproblem list
    const int* nsub;             // device count of subproblems
    int maxsub;                  // capacity of subs
};

// Epilogue of a kernel product on the target side.
enum EpiMode : int {
    EPI_RAW = 0,       // out[i] = raw                                   (plain matvec)
    EPI_MSG = 1,       // out[i] = max(raw, floor), scale record of out  (message beta / gamma)
    EPI_PHI = 2,       // phi_i = mu_i / (raw_i T_i)                      (scaling update)
    EPI_MARG = 3,      // store raw as message; P_i = raw_i T_i e^{L}; accumulate violation
    EPI_ROOT = 4,      // raw = 1: mass / root violation from the last iterate, then phi update
    EPI_PHI_FREE = 5,  // phi_i = 1 (node without marginal constraint)
    EPI_CROOT = 6,     // circle root: mass / violation of the last iterate from raw, phi = mu / raw
};

// Accumulators of one iteration (FP64).
struct IterAcc {
    double logphi;     // sum_k mu^k . log phi^k
    double mass;       // sum of K (.) Phi (root)
    double rootviol;   // ||P_1 - mu^1||_1
    double pad;
};

// One kernel-product task: v on the source side, K v on the target side, then an epilogue.
struct Task {
    // source side
    PointSet src;
    int sf0, snf;                // factors of v_j = prod_f (...)  (indices into the factor array)
    const float* alpha;          // if not null: v_j = alpha[j] (plain matvec, true scale)
    // grids (fast summation)
    float* grid;                 // spread target g, n^d floats; zeroed again by its reader
    float* hgrid;                // interpolation source h = IFFT(D FFT(g)), n^d floats
    float2* spec;                // 3-D intermediate spectrum
    const float* D;              // spectral multiplier (half spectrum)
    float eta_u;                 // eta in squared grid units (dense path)
    float* raw;                  // dense path: raw sums (zeroed again by the epilogue)
    // target side
    PointSet tgt;
    int mode;                    // EpiMode
    int tf0, tnf;                // target-side factors T_i = prod_f (...)
    int free_node;               // EPI_ROOT: keep phi = 1
    const float* mu_f;           // mu^k (FP32, sorted order) on the targets
    const double* mu_d;          // mu^k (FP64, sorted order); NULL: no marginal constraint
    float* out;                  // message mantissas / plain output
    VecScale* out_sc;
    float* phi;                  // scaling mantissas
    VecScale* phi_sc;
    double* acc_node;            // per-node accumulators [3]: violation, P.log(phi), mass
    // duties of block 0 of the first kernel that carries the task
    int reset_n;                 // number of scale records to reset
    VecScale* const* reset_list; // records whose mx / clamp count are reset
    int save_prev;               // keep ls / mx in ls_prev / mx_prev before the reset
    double* zero_d;              // doubles to zero
    int zero_n;
    int iter_off;                // this task's sweep is the counter minus iter_off (sweeps of a
                                 // pipelined chunk share one counter value)
    int dep0, ndep;              // persistent wavefront kernel: indices (into its dependency
                                 // array) of the products that must complete before this one
};

__device__ __forceinline__ float mx_of(const VecScale* s, int use_prev) {
    if (s == nullptr) return 1.f;
    unsigned int b = use_prev ? s->mx_prev_bits : s->mx_bits;
    float m = __uint_as_float(b);
    return (m > 0.f && m < 3.0e38f) ? m : 1.f;
}

__device__ __forceinline__ double ls_of(const VecScale* s, int use_prev) {
    if (s == nullptr) return 0.0;
    return use_prev ? s->ls_prev : s->ls;
}

// Normalised log-scale of one factor: ls + log(mx), signed by inv (log of the FP32 maximum in
// FP32: its rounding is that of the FP32 mantissas themselves).
__device__ __forceinline__ double factor_L(const Factor& f) {
    double L = ls_of(f.sc, f.use_prev) + (double)logf(mx_of(f.sc, f.use_prev));
    return f.inv ? -L : L;
}

__device__ __forceinline__ void atomic_max_pos(unsigned int* addr, float v) {
    // valid for v >= 0 (FP32 order equals unsigned order of the bits)
    atomicMax(addr, __float_as_uint(v));
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ int wrap_idx(int l, int n) {
    l %= n;
    return l < 0 ? l + n : l;
}

// Copy a task descriptor into shared memory with all threads of the block (word by word).
__device__ __forceinline__ void load_task(Task& dst, const Task* src) {
    static_assert(sizeof(Task) % 4 == 0, "Task is copied in 32-bit words");
    const unsigned int* s = reinterpret_cast<const unsigned int*>(src);
    unsigned int* d = reinterpret_cast<unsigned int*>(&dst);
    for (int i = threadIdx.x; i < (int)(sizeof(Task) / 4); i += blockDim.x) d[i] = __ldg(s + i);
}
