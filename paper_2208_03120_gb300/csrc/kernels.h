// Host-side launchers of the libmotfft kernels (implemented in nfft.cu, dense.cu, prep.cu).
#pragma once
#include <cuda_runtime.h>
#include "common.cuh"
#include "epilogue.cuh"

// Binning geometry of the oversampled grid, shared by the binning and the spread / gather kernels.
inline __host__ __device__ int mot_tile_size(int d, int n) {
    int t = d == 1 ? 256 : 16;
    return t < n ? t : n;
}
// Subproblem size: 3-D tiles (16^3 cells, ~10^3 points at the workloads' densities) are loaded and
// flushed once per subproblem, so a subproblem takes about a tile's points.
inline __host__ __device__ int mot_sub_points(int d) { return d == 2 ? 256 : 1024; }
inline __host__ __device__ int mot_ncells(int d, int n) {
    int t = 1;
    for (int i = 0; i < d; ++i) t *= n;
    return t;
}
inline __host__ __device__ int mot_ntiles(int d, int n) {
    int per = n / mot_tile_size(d, n);
    int t = 1;
    for (int i = 0; i < d; ++i) t *= per;
    return t;
}

// ---- fast summation (nfft.cu) -------------------------------------------------------
// All take a device array of `ntask` tasks and launch on `st`.
cudaError_t launch_spread(int d, const Task* tasks, int ntask, int grid_x, const Globals& G, cudaStream_t st);
cudaError_t launch_fftconv(int d, const Task* tasks, int ntask, const Globals& G, cudaStream_t st, int* nlaunch);
// Configure the shared-memory limits of the FFT kernels for grid length n (call before launching / capturing).
cudaError_t prepare_fftconv(int d, int n);
cudaError_t launch_gather(int d, const Task* tasks, int ntask, int grid_x, const Globals& G, cudaStream_t st);
int spread_smem_bytes(int d, int n);
// Window coefficients to constant memory (once per device; call before launching / capturing).
cudaError_t prepare_window();
// Fused 2-D fast summation (one thread-block cluster per task) for grids n <= 64.
cudaError_t prepare_fused2d();
bool fused2d_supported(int d, int n);
int fused2d_max_points();     // largest point set per product the fused kernel takes
int fused2d_cluster_size();
int fused2d_max_active_clusters();   // co-resident clusters of the fused kernel (0 before set-up)
// msg_only: every task is a message product with a kernel sum (lean instance).
cudaError_t launch_fused2d(const Task* tasks, int ntask, const Globals& G, cudaStream_t st, bool msg_only);
// Persistent wavefront kernel: all products of a chunk in one launch of `nclusters` clusters, which
// claim products in array order (a topological order) and wait for their dependencies' flags.
struct WaveCtl {                 // zeroed once; the chunk prologue resets next / abort, advances epoch
    int next;                    // claim counter
    int epoch;                   // flags[i] == epoch: product i of the current launch completed
    int abort;                   // set when a bounded wait ran out: no further claims
    int pad;
};
struct WaveArgs {
    const Task* tasks;
    int ntask;
    const int* deps;             // dependency lists (Task.dep0 / Task.ndep)
    int* flags;                  // [ntask] completion flags: k_wave2d stores the launch's epoch; k_wave_nd
                                 // counts the CTAs that completed the product (zeroed by the prologue)
    WaveCtl* ctl;
    int* err;                    // bit 2 (value 4): a wait ran out
    unsigned long long wait_ns;  // limit of every wait
};
int wave2d_max_active_clusters();    // co-resident clusters of the persistent kernel (0 before set-up)
cudaError_t launch_wave2d(const WaveArgs& A, int nclusters, const Globals& G, cudaStream_t st);
// The same two kernels with the exact trigonometric sums (ndft2d.cu) in place of the oversampled
// grid: d = 2, M <= 16, D without window deconvolution (launch_make_D deconv = false).
cudaError_t prepare_ndft2d();
bool ndft2d_supported(int d, int M);
int ndft2d_max_active_clusters();
int ndft2d_wave_max_active_clusters();
cudaError_t launch_ndft2d(const Task* tasks, int ntask, const Globals& G, cudaStream_t st, bool msg_only);
cudaError_t launch_wave_nd(const WaveArgs& A, int nclusters, const Globals& G, cudaStream_t st);
// Batched 1-D fast summation of the circle (grids n <= 128): per-point window taps and base cells
// (once per solve), the circulant of D (once per edge), and one batch Y[c] = K (phi (.) X[c]):
// stage 0 zeroes G and spreads, stage 1 convolves, interpolates and writes the messages.
bool c1_supported(int d, int n);
cudaError_t launch_c1_taps(const float* u, int n, int* l0, float* w, cudaStream_t st);
cudaError_t launch_c1_circulant(const float* D, int M, int n, float* c, cudaStream_t st);
cudaError_t launch_c1_batch(const float* X, const VecScale* sX, const float* phi, const VecScale* sP, const int* l0s,
                            const float* ws, int ns, const int* l0t, const float* wt, int nt, int n0, int ng,
                            const float* cvec, float* G, float* Y, float floor_, VecScale* out_sc, cudaStream_t st,
                            int stage, const float* rd_beta = nullptr, const VecScale* rd_sbeta = nullptr,
                            const float* rd_phi1 = nullptr, const VecScale* rd_sphi1 = nullptr,
                            float* rd_raw = nullptr, VecScale* rd_raw_sc = nullptr);
// One-block iteration prologue (resets, iteration counter, accumulators; with ctl: the persistent
// kernel's claim counter and abort word reset and its epoch advanced).
cudaError_t launch_prologue(VecScale* const* list, int nlist, int save_prev, int bump, double* zero_d, int zero_n,
                            const Globals& G, cudaStream_t st, WaveCtl* ctl = nullptr, int* zero_i = nullptr,
                            int zero_in = 0);

// ---- dense direct summation (dense.cu) ----------------------------------------------
cudaError_t launch_dense(int d, const Task* tasks, int ntask, int ntb, int nsplit, const Globals& G,
                         cudaStream_t st);
cudaError_t launch_epi(int d, const Task* tasks, int ntask, int grid_x, const Globals& G, cudaStream_t st);

// ---- set-up (prep.cu) ---------------------------------------------------------------
struct PrepSet {                 // one point set to normalise and bin
    const float* x;              // caller points [n][d]
    const double* mu;            // caller weights or NULL
    int n;
    float* u_tmp;                // [d][n] scratch
    int* tile_of;                // [n] scratch
    int* counts;                 // [n_grid^d] scratch (points per grid cell)
    int* cursor;                 // [n_grid^d] scratch
    float* u;                    // [d][n] sorted coordinates (grid units)
    int* perm;                   // [n] sorted position -> caller index
    float* mu_f;                 // [n] or NULL
    double* mu_d;                // [n] or NULL
    Sub* subs;                   // [maxsub]
    int* nsub;                   // [1]
    int maxsub;
};
// Bounding box + radius of the union of sets: out[0..2d) = (min, max) per dim, out[2d] = R^2
// about the box centre.  `sets` is a device array.
cudaError_t launch_bounds(const PrepSet* sets, int nsets, int d, float* box_raw, float* out, cudaStream_t st);
// Normalise (x - c) / s onto the torus in grid units, bin into tiles, sort, build subproblems.
cudaError_t launch_prep(const PrepSet* sets_dev, const PrepSet* sets_host, int nsets, int d, int n_grid,
                        const double* c, double s, int* err_flag, cudaStream_t st);
// kappa_hat by the (2M)^d FFT of Eq. (fft) in FP64, then the half-spectrum multiplier
// D = w kappa_hat / Psi^2 for the grid of length n per dimension (deconv = false: D = w kappa_hat,
// the multiplier of the exact trigonometric sums).
cudaError_t launch_make_D(int d, int M, int n, double eta_n, double tau, double epsB, int p,
                          const double* poly /* host [2p+1] coefficients in t = r - (tau-epsB) */,
                          double* scratch_a, double* scratch_b, float* D, cudaStream_t st, bool deconv = true);
size_t make_D_scratch_doubles(int d, int M);
size_t D_floats(int d, int M);
// Per-set arguments of the batched output / cold-start launches (one launch for all sets).
struct OutSet {
    const float* phi;
    const VecScale* sc;
    const int* perm;
    int n;
    double* u;                   // output (nullptr: skip the set)
};
struct OutBatch {
    int nsets;
    double eta;
    OutSet s[64];
};
// u[k][perm[i]] = eta * (log(phi[k][i]) + ls_k) for every set k
cudaError_t launch_output_batch(const OutBatch& B, cudaStream_t st);
// phi[k] = 1 and a fresh scale record for every set k (u: unused)
cudaError_t launch_init_cold_batch(const OutBatch& B, cudaStream_t st);
// u_out[perm[i]] = eta * (log(phi[i]) + ls)
cudaError_t launch_output(const float* phi, const VecScale* sc, const int* perm, int n, double eta,
                          double* u_out, cudaStream_t st);
// phi = 1 (cold) or exp(u_warm[perm[i]]/eta - shift) (warm); sets the scale record and adds
// sum mu log phi to *logphi.
cudaError_t launch_init_phi(float* phi, VecScale* sc, const int* perm, const double* mu_d, int n,
                            const double* u_warm, double eta, double* logphi, float* scratch_max,
                            cudaStream_t st);
// Timing aid: a single-thread sleep of at most 0.1 s on the device clock.
cudaError_t launch_delay(unsigned long long ns, cudaStream_t st);
// Scatter a plain vector into sorted order and back.
cudaError_t launch_permute_in(const float* src, const int* perm, int n, float* dst, cudaStream_t st);
cudaError_t launch_permute_out(const float* src, const int* perm, int n, float* dst, cudaStream_t st);

// ---- circle structure (circle.cu) --------------------------------------------------------
#include <algorithm>
// raw[i] += sum_c B[c][i] G[c][i] phi[c] over normalised factors (raw zeroed by the caller).
cudaError_t launch_rowdot(const float* B, const VecScale* sB, const float* G, const VecScale* sG, const float* phi,
                          const VecScale* sP, int ni, int nc, float* raw, cudaStream_t st);
// raw[c] = sum_j A[c][j] B[c][j] phi[j] over normalised factors.
cudaError_t launch_colsum(const float* A, const VecScale* sA, const float* B, const VecScale* sB, const float* phi,
                          const VecScale* sP, int nj, int nc, float* raw, cudaStream_t st);
// K[c][i] = exp(-||u_i - u_c||^2 / eta_u) (column-major, grid units); scale record ls = 0, mx = 1.
cudaError_t launch_kernel_matrix(const float* ui, int ni, const float* uc, int nc, int d, float eta_u, float* K,
                                 VecScale* sc, cudaStream_t st);
// Generalised Euler flow (Section 6.3): the closing edge's node-1 points sigma(x^1), sorted like
// node 1 and in grid units (not wrapped); non-finite input sets bit 0 of *err.
cudaError_t launch_close_points(const float* x, const int* perm, int n, int d, const double* c, double s, int n_grid,
                                float* u, int* err, cudaStream_t st);
// Pair marginal Pi_{1,k}[perm1[c]][permk[i]] = phi^1_c Gam_k[c][i] beta_k[c][i] phi^k_i (FP64).
cudaError_t launch_pair(const float* phi1, const VecScale* s1, const int* perm1, int n1, const float* phik,
                        const VecScale* sk, const int* permk, int nk, const float* G, const VecScale* sG,
                        const float* B, const VecScale* sB, double* out, cudaStream_t st);

// ---- small-eta local path: truncated kernel sums in the log domain (local.cu) -------------------
struct LGrid {                   // common grid of cells (side h >= r_cut) over all point sets
    int d;
    int dims[3];
    float lo[3];                 // box corner
    float h, inv_h;
    int ncells;
};
struct LBinSet {                 // one point set to bin
    int n;
    const float* x;              // caller points [n][d]
    const double* mu;            // caller weights [n]
    int* cell;                   // [n] scratch
    int* cstart;                 // [ncells + 1] out: first sorted point of each cell (zeroed by the caller)
    int* cursor;                 // [ncells] scratch
    float* u;                    // [d][n] out: sorted coordinates
    int* perm;                   // [n] out: sorted position -> caller index
    double* mu_s;                // [n] out: sorted mu
    double* logmu;               // [n] out: sorted log mu (-inf where mu = 0)
};
struct LSet {                    // a binned point set
    int n;
    const float* u;
    const int* cstart;
    const double* logmu;
    const double* mu;
};
struct LFac {                    // one term of a sum of log-vectors: +-v
    const double* v;
    int sign;
};
enum LEpi : int {
    LEPI_MSG = 0,                // out = log of the kernel sum (a message b_k)
    LEPI_FWD = 1,                // out = g_k; f^k = log mu^k - g_k - sum_c b_c; sum mu f into the next slot
    LEPI_CHK = 2,                // out = g-ex_k; exact marginal of node k into acc_node
    LEPI_ROOT = 3,               // root: mass / violation of the last iterate, then f^1 = log mu^1 - sum_c b_c
    LEPI_CHKROOT = 4,            // root: exact marginal into acc_node
};
struct LTask {
    LSet src, tgt;
    int sf0, snf;                // source log-values l_j = sum of the factors
    int tf0, tnf;                // target-side log-messages (children's b)
    float* delta;                // [src.n] scratch: l_j - L_c
    double* Lc;                  // [ncells] scratch: max l over each source cell
    float inv_eta, r2;           // 1 / eta_e and r_cut^2
    double inv_eta_d;
    int mode;                    // LEpi
    double* out;                 // [tgt.n] log kernel sum
    double* f;                   // [tgt.n] log phi of the target node
    double* acc_node;            // check: [3] violation, sum P f, mass
    int iter_off;
    int tchunks;                 // chunks of LSE_TARGETS targets in the fullest target cell
};
struct LGlobals {
    int* iter;
    IterAcc* acc;
    int R;
    int* err;                    // bit 0: non-finite input; bit 1: negative weight; bit 3: a target
};                               // has no source within r_cut
cudaError_t launch_lbin(const LBinSet* sets_dev, int nsets, int nmax, const LGrid& g, int* err, int* maxcount,
                        cudaStream_t st);
constexpr int LSE_TARGETS = 256;   // targets per CTA of the log-sum-exp kernel
cudaError_t launch_lsrc(const LTask* tasks, int ntask, const LFac* F, int ncells, int* err, cudaStream_t st);
// grid (cells, tasks, tchunks): tchunks = the largest LTask.tchunks of the launch
cudaError_t launch_lse(const LTask* tasks, int ntask, int tchunks, const LFac* F, const LGrid& g, const LGlobals& G,
                       cudaStream_t st);
cudaError_t launch_lroot(const LTask* tasks, int ntask, const LFac* F, int nmax, const LGlobals& G, cudaStream_t st);
cudaError_t launch_linit(double* f, const int* perm, const double* mu, int n, const double* u, double eta,
                         double* logphi, cudaStream_t st);
cudaError_t launch_lout(const double* f, const int* perm, int n, double eta, double* u, cudaStream_t st);

// ---- dense products on the tensor cores, BF16 hi + lo split (tc_gemm.cu) ------------------
// Y[c][i] = sum_j A[c][j] B[i][j] with A = Ahi + Alo (M x K), B = Bhi + Blo (N x K), BF16,
// row strides lda / ldb (multiples of 8 elements); FP32 accumulation of Ahi Bhi + Ahi Blo + Alo Bhi.
struct TcGemm {
    alignas(64) unsigned char maps[4][128];   // TMA tensor maps of Ahi, Alo, Bhi, Blo
    int M, N, K, bn;
};
struct TcEpi {
    int M, N, K;              // filled from the TcGemm by the launcher
    float* out;               // out[c * ldo + i]
    long long ldo;
    int mode;                 // 0: plain product; 1: message (floor, maximum, clamp count, log-scale)
    float floor_;
    VecScale* out_sc;         // mode 1: scale record of the output (mx reset by the caller)
    const VecScale* s_a;      // mode 1: scale records whose log-scales sum to that of the output
    const VecScale* s_b;
    int* err;                 // bit 2 (value 4) set when a bounded wait expired
    unsigned long long wait_ns;  // limit of every bounded wait (filled by the launcher)
    int stall_loads;          // test hook: the producer issues no loads (filled by the launcher)
};
int tc_ld(int k);             // padded row stride (elements) of a split operand with k columns
cudaError_t prepare_tc_gemm();
bool tc_prepare(TcGemm* g, const void* a_hi, const void* a_lo, int M, int lda, const void* b_hi, const void* b_lo,
                int N, int ldb, int K);
cudaError_t launch_tc_gemm(const TcGemm& g, TcEpi e, cudaStream_t st);
// hi/lo[c][j] of (phi_j / max phi)(X[c][j] / max X), X column c contiguous over j (phi may be null).
cudaError_t launch_split_src(const float* X, const VecScale* sX, const float* phi, const VecScale* sP, int ns,
                             int nrow, int ld, void* hi, void* lo, cudaStream_t st);
// hi/lo[i][j] of exp(-||ut_i - us_j||^2 / eta_u) (grid units).
cudaError_t launch_kernel_split(const float* ut, int nt, const float* us, int ns, int d, float eta_u, int ld,
                                void* hi, void* lo, cudaStream_t st);
