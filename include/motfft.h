/*
 * motfft.h -- C ABI of the NFFT-accelerated multi-marginal Sinkhorn library (libmotfft.so).
 *
 * The library computes entropy-regularised multi-marginal optimal transport with a
 * tree- or circle-structured squared-Euclidean cost (Ba & Quellmalz, "Accelerating the
 * Sinkhorn algorithm for sparse multi-marginal optimal transport by fast Fourier
 * transforms", 2022).  The kernel matrix-vector products on the edges are done by
 * NFFT-based fast summation (Section 5, Algorithm 4) or, for comparison, by dense
 * direct summation (Eq. fastsum-sum).
 *
 * Conventions shared by every entry point
 *   - Pointers documented as "device" point to CUDA device memory owned by the caller
 *     (e.g. the storage of torch tensors).  The library never allocates device memory
 *     inside these calls: scratch comes from the caller's workspace, whose size the
 *     *_workspace_bytes queries return.  The workspace must be 256-byte aligned.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *     Work is enqueued on it; the calls return after a final readback of a few scalars
 *     on that stream (they synchronise that stream, not the device).
 *   - Node labels are 0-based: the paper's node k is label k-1.
 *   - Return value: MOT_OK or one of the MOT_E* codes below.  No exception crosses the
 *     ABI.  On an error the output buffers are unspecified.
 */
#ifndef MOTFFT_H
#define MOTFFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MOT_ABI_VERSION 5

/* ---- status codes ---------------------------------------------------------------- */
#define MOT_OK           0
#define MOT_EINVAL       1  /* bad argument: NULL pointer, size out of range, bad option       */
#define MOT_ENOTTREE     2  /* MOT_TREE edges do not form a tree on K nodes                    */
#define MOT_ENOMEM       3  /* caller workspace smaller than the *_workspace_bytes query       */
#define MOT_ENUMERIC     4  /* NaN / Inf, or a marginal weight that is negative                */
#define MOT_ENOCONV      5  /* stop test not met within max_iter (results are still valid)     */
#define MOT_ETIMEOUT     6  /* a bounded device-side wait gave up                              */
#define MOT_ECUDA        7  /* a CUDA runtime call failed (see mot_last_cuda_error)             */
#define MOT_EUNSUPPORTED 8  /* valid request outside what this build implements                */

/* ---- enums ----------------------------------------------------------------------- */
#define MOT_TREE   0        /* Section 4.1: cost decouples along the edges of a tree           */
#define MOT_CIRCLE 1        /* Section 4.2: edges {k, k+1 mod K}                               */

#define MOT_ROOT_CENTRE      (-1)  /* mot_problem.root: choose a centre of the tree               */

#define MOT_PATH_NFFT         0  /* fast summation, Algorithm 4 (window spread, FFT, D, iFFT, gather), FP32 */
#define MOT_PATH_DENSE        1  /* direct summation, Eq. (fastsum-sum), FP32 SIMT                          */
#define MOT_PATH_DENSE_BF16X3 2  /* direct summation on tensor cores, split hi+lo BF16, FP32 accumulate     */
#define MOT_PATH_LOCAL        3  /* trees, small eta (Section 6.1, closing remark): Algorithm 2 with the
                                    logarithms of scalings and messages (FP64), every kernel sum truncated
                                    to the pairs within options.r_cut and evaluated as a log-sum-exp over a
                                    cell list (FP32 terms against FP64 references)                        */

/* Kernel classes for the optional per-kernel timing of mot_result. */
#define MOT_K_SPREAD   0    /* window spreading onto the oversampled grid (adjoint NFFT)       */
#define MOT_K_FFTCONV  1    /* FFT, multiply by D, inverse FFT                                 */
#define MOT_K_GATHER   2    /* window interpolation from the grid (NFFT) + sweep epilogue      */
#define MOT_K_DENSE    3    /* dense direct matrix-vector product                              */
#define MOT_K_NODE     4    /* element-wise sweep updates and FP64 reductions                  */
#define MOT_K_SETUP    5    /* normalisation, binning, kernel Fourier coefficients             */
#define MOT_K_CIRCLE   6    /* circle row-dot / column-sum scaling updates                     */
#define MOT_K_FUSED    7    /* fused 2-D fast summation (spread, DFTs, gather in one cluster)  */
#define MOT_K_TCGEMM   8    /* split-BF16 kernel product on the tensor cores (tcgen05)         */
#define MOT_K_SPLIT    9    /* scaled source matrix split into BF16 hi / lo                    */
#define MOT_K_WAVE     10   /* persistent wavefront kernel: a chunk of tree sweeps + check pass */
#define MOT_K_LOCAL    11   /* truncated log-sum-exp kernel sums of the small-eta local path     */
#define MOT_NKCLASS    12

/* ---- problem --------------------------------------------------------------------- */
/* Section 2 / Section 4: K marginals mu^k on points x^k in R^d, a tree or a circle, eta. */
typedef struct {
    int K;                          /* number of marginals, 2 <= K <= 64                      */
    int d;                          /* space dimension, 1..3                                  */
    const int64_t* n;               /* host [K]: n_k, 1 <= n_k <= 2^26                         */
    const float* const* x;          /* host [K] of device pointers: x^k, row-major [n_k][d]   */
    const double* const* mu;        /* host [K] of device pointers: mu^k [n_k], >= 0, sum 1    */
    int topology;                   /* MOT_TREE or MOT_CIRCLE                                 */
    const int* edges;               /* MOT_TREE: host [2*(K-1)] node pairs; ignored otherwise */
    const double* edge_w;           /* host weights w_e > 0 of the squared distance
                                       (Section 6.2): [K-1] in edge order (tree) or [K] for
                                       edges {k, k+1 mod K} (circle); NULL = all 1            */
    const unsigned char* free_nodes;/* host [K] or NULL: 1 = node without marginal constraint,
                                       its scaling is held at 1 (Section 6.2, tree only).
                                       The root must be constrained (MOT_EUNSUPPORTED
                                       otherwise); MOT_ROOT_CENTRE picks a constrained node */
    double eta;                     /* entropic regularisation eta > 0 (Eq. MOTe)             */
    int root;                       /* tree root label (the paper's node 1), or
                                       MOT_ROOT_CENTRE: a centre of the tree (least
                                       eccentricity, smallest label on ties), which gives
                                       the backward pass the fewest sequential levels         */
    const float* x_close;           /* MOT_CIRCLE only, device [n_1][d] or NULL: the points that
                                       the closing edge {K, 1} compares x^K with, in place of
                                       x^1 -- sigma(x^1) for the connection map sigma of the
                                       generalised Euler flow (Section 6.3).  The edge's kernel
                                       is exp(-w ||x^K_i - x_close_j||^2 / eta); every other
                                       use of node 1 keeps x^1.  Non-NULL for a tree:
                                       MOT_EINVAL                                             */
} mot_problem;

/* ---- options (zero-initialised fields take the defaults in brackets) ------------- */
typedef struct {
    int path;           /* MOT_PATH_* [MOT_PATH_NFFT]                                          */
    int max_iter;       /* iteration cap [1000]                                                */
    double tol_viol;    /* stop once max_k ||P_k - mu^k||_1 <= tol_viol [1e-6]; < 0 disables    */
    double delta_S;     /* stop once |S^(r) - S^(r-1)| < delta_S (Algorithm 2 test) [off]        */
    int check_every;    /* iterations between stop tests (each test = one host readback) [10]  */
    int min_iter;       /* iterations always run [0]                                           */
    int n_grid;         /* oversampled grid length per dimension, power of two 16..4096
                           (d=1), ..128 (d=2), ..64 (d=3) [64]; M = n_grid/4                     */
    int m;              /* window cutoff: 2m+2 grid taps per dimension; only m = 4 [4]         */
    int p;              /* smoothness p of the regularised kernel (Eq. Ker-reg) [3]            */
    double eps_B;       /* boundary width eps_B of Eq. (Ker-reg), in units of the normalised
                           period 2*tau = 1 [1/16]                                             */
    int use_graphs;     /* 1 = replay iterations as a CUDA graph, -1 = plain launches [1]      */
    int timing;         /* 1 = time every kernel class with CUDA events (slower) [0]          */
    int wavefront;      /* trees on the fused 2-D path: pipeline the sweeps of each stop-test chunk
                           (up to 32 sweeps) as a wavefront -- the same products on the same inputs
                           as the sweep-by-sweep order of Algorithm 2, products of several sweeps
                           in flight at once.  1 = one persistent launch per chunk whose clusters
                           take the products in a topological order and start each one as soon as
                           the products it reads have completed; 2 = one launch per step of the
                           host's list schedule; -1 = sweep by sweep [1]                         */
    double r_cut;       /* MOT_PATH_LOCAL: pairs farther apart than r_cut leave every kernel sum
                           [0 = sqrt(40 eta / w_e) per edge, where the kernel is below e^-40].  Every
                           target needs a source point within r_cut (MOT_ENUMERIC otherwise)     */
    int ndft;           /* d = 2, MOT_PATH_NFFT, n_grid <= 64 (M <= 16), point sets of up to 32768:
                           1 = evaluate the trigonometric sums of the fast summation, Eq. (ndft*)
                           for ghat and Eq. (ndft) for the result, exactly as dense FP32
                           contractions in one thread-block cluster per product; -1 = through the
                           oversampled grid (NFFT, with the window error of Section 5) [1]       */
} mot_options;

/* Fill *o with the defaults. */
void mot_options_default(mot_options* o);

/* ---- result ---------------------------------------------------------------------- */
typedef struct {
    double* const* u;       /* in: host [K] of device pointers or NULL.  out: u^k = eta log phi^k
                               [n_k] FP64 in the caller's point order (scalings, Theorem 3.1)  */
    double violation;       /* max_k ||P_k(K (.) Phi) - mu^k||_1 at the returned scalings, the
                               marginals computed with the path's own kernel operator           */
    double cost_dual;       /* Sinkhorn function S at the returned scalings (Eq. dual_problem) */
    double cost_primal;     /* Eq. (MOTe) objective at Pi = K (.) Phi                           */
    double mass;            /* sum of K (.) Phi                                                */
    double S_last, S_prev;  /* the last two S^(r) of the iteration (Algorithm 2 / 3)           */
    int iters;              /* Sinkhorn iterations run                                        */
    int status;             /* same as the return value                                       */
    long long clamped;      /* fast-summation outputs raised to the positive floor            */
    long long launches;     /* kernels launched by the call (graph replays counted per node)  */
    double scale;           /* normalisation x' = (x - c) / scale onto the unit torus          */
    double eta_norm;        /* eta / scale^2                                                   */
    int n_grid, M;          /* grid length per dimension and Fourier half-degree used          */
    double kernel_ms[MOT_NKCLASS];        /* with options.timing: device ms per kernel class   */
    long long kernel_launches[MOT_NKCLASS];
    double* const* pair;    /* in: MOT_CIRCLE only, host [K] of device pointers or NULL (entry 0
                               is ignored and entries may be NULL).  out: pair[k] (k = 1..K-1)
                               = the pair marginal Pi_{1,k+1} of K (.) Phi at the returned
                               scalings (Section 6.3), FP64 row-major [n_1][n_{k+1}] in the
                               caller's point order; row sums are P_1, column sums P_{k+1}.
                               Non-NULL for a tree: MOT_EINVAL                                */
} mot_result;

/* ---- entry points ---------------------------------------------------------------- */

/* Human-readable text for a status code (static storage). */
const char* mot_strerror(int status);

/* Text of the last CUDA error seen by this thread ("" if none). */
const char* mot_last_cuda_error(void);

/* MOT_ABI_VERSION of the loaded library. */
int mot_abi_version(void);

/* sizeof of the ABI structs as compiled into the library (bindings check their mirrors):
   out[0] mot_problem, out[1] mot_options, out[2] mot_result, out[3] mot_server_result. */
void mot_struct_sizes(size_t out[4]);

/*
 * Host-only helper (no GPU): the launch schedule that options.wavefront uses for a chunk of S
 * sweeps of Algorithm 2 on a tree, exposed so that it can be inspected and tested.
 *   parent:  host [K], the tree in breadth-first labels (parent[0] = -1, parent[k] < k).
 *   cap:     most products per launch (the solver uses the fused kernel's co-resident clusters).
 *   tF, tB:  host [S*K] out, entry s*K + k (k >= 1): launch of sweep s's forward product of node k
 *            (gamma_k and the update of phi^k) and of its backward product (beta_k).
 *   tR:      host [S] out, launch of sweep s's root update.
 *   carrier: host [S] out, the child c of the root whose backward product of sweep s-1 saves the
 *            root scaling's scale record for the root update of sweep s (-1 for s = 0).
 *   nlaunch: out, launches of the chunk.
 * Every product is in a later launch than the products whose results it reads and than the
 * previous sweep's readers of the beta copy it overwrites (two copies, alternating by sweep).
 * Returns MOT_OK, MOT_EINVAL (bad tree or sizes, NULL pointers) or MOT_EUNSUPPORTED.
 */
int mot_wave_schedule(int K, const int* parent, int S, int cap, int* tF, int* tB, int* tR, int* carrier,
                      int* nlaunch);

/*
 * Host-only helper (no GPU): the boundary polynomial kappa_B of the regularised kernel, Eq.
 * (Ker-reg) (Section 5, worked example in Fig. 3), as the solver builds it: degree 2p with
 * kappa_B^(r) = kappa^(r) at a = tau - eps_B for r = 0..p and kappa_B^(r)(tau) = 0 for r = 1..p,
 * kappa(x) = exp(-x^2 / eta).  coef: host [2p+1] out, coefficients of kappa_B(a + t) in powers of
 * t.  Returns MOT_OK, MOT_EINVAL (eta <= 0, p outside 1..8, eps_B outside (0, tau)) or
 * MOT_ENUMERIC (singular system).
 */
int mot_boundary_poly(double eta, double tau, double eps_B, int p, double* coef);

/*
 * Host-only helper (no GPU): the normalisation and grid the solver picks (Section 5): points
 * within `radius` of their centre are scaled by 1/scale onto the unit torus (tau = 1/2) so that
 * every pairwise distance stays below tau - eps_B, and the grid length n (M = n/4 Fourier
 * half-degree) is the smallest power of two (16 .. the dimension's maximum, or exactly n_grid if
 * > 0) for which both neglected terms -- the kernel of width eta_max at tau - eps_B and the Fourier
 * tail of width eta_min beyond M -- are below exp(-18); err_exp receives the smaller of the two
 * exponents reached.  Returns MOT_OK or MOT_EINVAL.
 */
int mot_plan_grid(int d, double radius, double eta_min, double eta_max, int n_grid, double eps_B, int* n_out,
                  double* scale_out, double* err_exp_out);

/*
 * Workspace bytes needed by mot_solve for this problem and these options (depends on the
 * sizes only, not on the data).  Returns MOT_EINVAL / MOT_ENOTTREE for a malformed problem.
 */
int mot_workspace_bytes(const mot_problem* prob, const mot_options* opt, size_t* bytes);

/*
 * Sinkhorn for a tree (Algorithm 2) or a circle (Algorithm 3) with the kernel products on
 * the path selected by opt->path.  Runs until the marginal violation is <= tol_viol (tested
 * every check_every iterations), |S^(r) - S^(r-1)| < delta_S, or max_iter.  Initial
 * scalings phi^(0) = 1, or exp(u_warm^k / eta) when u_warm (host [K] of device pointers,
 * caller order) is not NULL.  Writes u^k and the scalar fields of *res.
 *   ws/ws_bytes : device workspace of at least mot_workspace_bytes() bytes.
 *   Errors      : MOT_EINVAL, MOT_ENOTTREE, MOT_ENOMEM, MOT_ENUMERIC, MOT_ECUDA;
 *                 MOT_ENOCONV when a stop test was requested and not met (results valid).
 */
int mot_solve(const mot_problem* prob, const mot_options* opt, void* ws, size_t ws_bytes,
              const double* const* u_warm, mot_result* res, void* stream);

/*
 * The kernel matrix-vector product of Eq. (fastsum-sum) on its own:
 *   beta_r[i] = sum_j alpha_r[j] exp(-||x_tgt[i] - x_src[j]||^2 / eta),  r = 0..nrhs-1,
 * by the fast summation of Algorithm 4 (opt->path = MOT_PATH_NFFT), directly on the SIMT
 * pipes (MOT_PATH_DENSE), or directly on the tensor cores (MOT_PATH_DENSE_BF16X3: alpha and
 * the kernel matrix split into BF16 hi + lo, three products accumulated in FP32; relative
 * error ~2^-16 per term).  x_src: device [n_src][d] FP32; x_tgt: device [n_tgt][d];
 * alpha: device [nrhs][n_src] FP32; beta: device [nrhs][n_tgt] FP32 (written).
 * Both point sets are mapped onto the torus together.  *scale_out (may be NULL)
 * receives the normalisation scale.  Errors: MOT_EINVAL, MOT_ENOMEM, MOT_ECUDA,
 * MOT_ETIMEOUT (a bounded wait of the tensor-core kernel expired).
 */
int mot_fastsum_workspace_bytes(int d, int64_t n_src, int64_t n_tgt, int nrhs,
                                const mot_options* opt, size_t* bytes);
int mot_fastsum(int d, double eta, const float* x_src, int64_t n_src, const float* x_tgt,
                int64_t n_tgt, const float* alpha, int nrhs, float* beta,
                const mot_options* opt, void* ws, size_t ws_bytes, double* scale_out,
                void* stream);

/* ---- serving: continuous batching of solves ---------------------------------------- */
/*
 * A server runs many mot_solve-equivalent requests at once.  Each admitted request gets its
 * own CUDA stream, its own captured iteration graph and a region of the caller's device pool
 * sized by mot_workspace_bytes (admission in arrival order while a slot and pool memory are
 * free); requests that arrive while others run are admitted as slots and memory free up, and
 * their kernels overlap on the GPU.  Results equal mot_solve's for the same request (up to
 * floating-point summation order).  The API is driven by the caller and not thread-safe.
 */
typedef struct mot_server_s* mot_server;
typedef struct {
    long long tag;          /* the submit tag                                                 */
    int status;             /* MOT_OK, MOT_ENOCONV, or the error of the request               */
    int iters;
    double violation, cost_dual, cost_primal;
    double submit_ms, admit_ms, done_ms;  /* host clock since mot_server_create              */
} mot_server_result;
/* pool: device memory owned by the caller (256-byte aligned) shared by the requests'
   workspaces; max_active: concurrent requests (1..256).  Creates max_active streams and
   pinned host stat buffers (32 KiB each). */
int mot_server_create(void* pool, size_t pool_bytes, int max_active, mot_server* out);
/* Queue a request.  The problem's arrays are copied; the device buffers it points to (x, mu)
   and u (host [K] of device pointers, may be NULL) must stay valid until its result is polled.
   A request larger than the whole pool completes with MOT_ENOMEM. */
int mot_server_submit(mot_server s, const mot_problem* prob, const mot_options* opt, double* const* u,
                      long long tag);
/* Non-blocking step: advance running requests whose last chunk finished (stop test, next chunk
   or outputs), complete finished ones and admit pending ones (admission performs the request's
   set-up, which reads back the point-cloud radius). */
int mot_server_progress(mot_server s, int* n_active, int* n_pending);
/* Move up to max completed results into out. */
int mot_server_poll(mot_server s, mot_server_result* out, int max, int* n_out);
int mot_server_destroy(mot_server s);

/*
 * Allocation-free variant of mot_fastsum (the paper has no counterpart).  It serves callers that
 * cannot allocate GPU memory or lend a workspace: plug-ins whose host application owns all
 * device memory through its own pool, and real-time loops where an allocation could block.
 * Same arguments and result as mot_fastsum, without ws / ws_bytes: the scratch is a static
 * device array of MOT_STATIC_SCRATCH_BYTES per GPU, held from library load until exit.
 *   - A request whose mot_fastsum_workspace_bytes exceeds MOT_STATIC_SCRATCH_BYTES returns
 *     MOT_ENOMEM before any GPU work (pass opt->n_grid = 64 for large d = 3 problems).
 *   - The first call on a device (with that device current) looks up the array's address;
 *     make it before any stream capture.
 *   - All calls on a device share the array: calls that overlap on the GPU race and must be
 *     serialised by the caller.  What must start at zero is cleared by every call.
 *   - Calls no cudaMalloc / cudaFree or any allocating routine.  Like mot_fastsum, the call ends
 *     by reading a few scalars back on its stream and synchronising that stream.
 */
#define MOT_STATIC_SCRATCH_BYTES (32u << 20)
int mot_fastsum_static(int d, double eta, const float* x_src, int64_t n_src, const float* x_tgt,
                       int64_t n_tgt, const float* alpha, int nrhs, float* beta,
                       const mot_options* opt, double* scale_out, void* stream);

/* ---- test hook ------------------------------------------------------------------------ */
/*
 * Error-path testing of the tensor-core kernel (MOT_PATH_DENSE_BF16X3) without a GPU fault (the
 * paper has no counterpart).  Every wait of that kernel on its own mbarriers is bounded by
 * wait_ns (default 10^9, i.e. 1 s); on expiry the kernel records the failure, waits (bounded) for
 * its own copies in flight, frees its tensor memory and returns, and the call returns
 * MOT_ETIMEOUT.  stall_loads = 1 makes the kernel's load thread issue no copies at all, so that
 * the first wait for operands runs out after wait_ns while nothing is in flight; the context stays
 * usable.  Process-wide; applies to launches made after the call (a captured graph keeps the
 * values it was captured with).  Restore with mot_test_tc_wait(1000000000, 0).
 * Returns MOT_OK or MOT_EINVAL (wait_ns outside [10^3, 10^10]).
 */
int mot_test_tc_wait(long long wait_ns, int stall_loads);

/*
 * Test hook of the persistent wavefront kernel (options.wavefront = 1; the paper has no
 * counterpart): launch it with `nclusters` thread-block clusters instead of as many as fit on the
 * GPU at once (0 restores that default).  Its products are claimed in a topological order and each
 * waits only for products claimed before it, so the result does not depend on how many clusters
 * run, nor on how many are resident together (1 runs the chunk's products one after another; more
 * than fit run in later waves).  Process-wide; applies to solves set up after the call.
 * Returns MOT_OK or MOT_EINVAL (nclusters outside [0, 1024]).
 */
int mot_test_wave_clusters(int nclusters);

#ifdef __cplusplus
}
#endif
#endif /* MOTFFT_H */
