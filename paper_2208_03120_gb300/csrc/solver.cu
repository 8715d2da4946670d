// Host orchestration of libmotfft: C-ABI entry points, plans and the Sinkhorn sweeps.
//
// Tree (Algorithm 2).  With the identity phi^p (.) gamma_p (.) beta^{C_p \ k} = mu^p / beta_k,
// valid right after phi^p is updated from gamma_p and the beta of the previous sweep, the
// forward messages gamma_k of all children of constrained nodes are independent, so the
// forward pass is one batched launch (plus dependent levels below free nodes).  The backward
// pass recomputes beta_k level by level from the leaves.  Every message and scaling is stored
// as FP32 mantissas with an FP64 log-scale (VecScale); the dual value, marginal violation and
// cost are FP64 reductions.
#include <atomic>
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <string>
#include <vector>

#include "plan.h"

namespace {
thread_local std::string g_cuda_err;
const double kPi = 3.14159265358979323846;
const double kTau = 0.5;            // half period of the unit torus
const double kErrExp = 18.0;        // target exponent: boundary / Fourier-tail terms below e^-18 ~ 1.5e-8
const int kRing = 64;               // iteration accumulator ring
}  // namespace

void set_cuda_error(cudaError_t e, const char* what) {
    g_cuda_err = std::string(what) + ": " + cudaGetErrorString(e);
}

#define CK(x)                                    \
    do {                                         \
        cudaError_t _e = (x);                    \
        if (_e != cudaSuccess) {                 \
            set_cuda_error(_e, #x);              \
            return MOT_ECUDA;                    \
        }                                        \
    } while (0)

#define RET(x)                                   \
    do {                                         \
        int _r = (x);                            \
        if (_r != MOT_OK) return _r;             \
    } while (0)

// test hook (mot_test_wave_clusters): clusters of the persistent wavefront kernel, 0 = as many as
// are co-resident on an idle GPU
std::atomic<int> g_wave_clusters_override{0};

int max_grid(int d) { return d == 1 ? 4096 : (d == 2 ? 128 : 64); }

GridChoice choose_grid(int d, double R, double eta_min, double eta_max, int n_grid_opt, double epsB) {
    GridChoice g;
    const double width = kTau - epsB;
    const double s_min = 2.0 * R / width;
    std::vector<int> cands;
    if (n_grid_opt > 0) {
        cands.push_back(n_grid_opt);
    } else {
        for (int n = 16; n <= max_grid(d); n *= 2) cands.push_back(n);
    }
    for (size_t i = 0; i < cands.size(); ++i) {
        const int n = cands[i];
        const int M = n / 4;
        const double A = width * width / eta_max;
        const double B = kPi * kPi * eta_min * (double)M * (double)M;
        double s2 = std::sqrt(B / A);
        if (s2 < s_min * s_min) s2 = s_min * s_min;
        const double E = std::min(A * s2, B / s2);
        g.n = n;
        g.M = M;
        g.s = std::sqrt(s2);
        g.err_exp = E;
        if (E >= kErrExp) break;
    }
    if (!(g.s > 0.0)) g.s = 1.0;
    return g;
}

bool boundary_poly(double eta, double tau, double epsB, int p, double* c) {
    // kappa^(r)(a) = (-1/sqrt(eta))^r H_r(a / sqrt(eta)) exp(-a^2/eta), H_r the physicists'
    // Hermite polynomials (H_{r+1} = 2y H_r - 2r H_{r-1}).
    const int n = 2 * p + 1;
    const double a = tau - epsB;
    const double se = std::sqrt(eta), y = a / se, e0 = std::exp(-a * a / eta);
    std::vector<double> H(p + 1);
    H[0] = 1.0;
    if (p >= 1) H[1] = 2.0 * y;
    for (int r = 1; r < p; ++r) H[r + 1] = 2.0 * y * H[r] - 2.0 * r * H[r - 1];
    std::vector<double> Amat(n * n, 0.0), rhs(n, 0.0);
    int row = 0;
    double fact = 1.0;
    for (int r = 0; r <= p; ++r, ++row) {      // value / derivatives at t = 0
        if (r > 0) fact *= r;
        Amat[row * n + r] = fact;
        rhs[row] = std::pow(-1.0 / se, r) * H[r] * e0;
    }
    for (int r = 1; r <= p; ++r, ++row) {      // derivatives vanish at t = eps_B
        for (int j = r; j < n; ++j) {
            double f = 1.0;
            for (int q = j - r + 1; q <= j; ++q) f *= q;
            Amat[row * n + j] = f * std::pow(epsB, j - r);
        }
        rhs[row] = 0.0;
    }
    // Gaussian elimination with partial pivoting
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (std::fabs(Amat[r * n + col]) > std::fabs(Amat[piv * n + col])) piv = r;
        if (std::fabs(Amat[piv * n + col]) < 1e-300) return false;
        if (piv != col) {
            for (int j = 0; j < n; ++j) std::swap(Amat[col * n + j], Amat[piv * n + j]);
            std::swap(rhs[col], rhs[piv]);
        }
        for (int r = col + 1; r < n; ++r) {
            double f = Amat[r * n + col] / Amat[col * n + col];
            if (f == 0.0) continue;
            for (int j = col; j < n; ++j) Amat[r * n + j] -= f * Amat[col * n + j];
            rhs[r] -= f * rhs[col];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = rhs[r];
        for (int j = r + 1; j < n; ++j) s -= Amat[r * n + j] * c[j];
        c[r] = s / Amat[r * n + r];
    }
    return true;
}

void fill_defaults(mot_options& o, const mot_options* in) {
    std::memset(&o, 0, sizeof(o));
    if (in) o = *in;
    if (o.max_iter <= 0) o.max_iter = 1000;
    if (o.tol_viol == 0.0) o.tol_viol = 1e-6;
    if (o.check_every <= 0) o.check_every = 10;
    if (o.check_every > kRing - 4) o.check_every = kRing - 4;
    if (o.m <= 0) o.m = 4;
    if (o.p <= 0) o.p = 3;
    if (o.eps_B <= 0.0) o.eps_B = 1.0 / 16.0;
    if (o.use_graphs == 0) o.use_graphs = 1;
    if (o.wavefront == 0) o.wavefront = 1;
    if (o.ndft == 0) o.ndft = 1;
}

// =============================================================================================
// shared set-up: normalisation, binning and the spectral multipliers
// =============================================================================================
namespace {

struct SetBufs {
    int n = 0;
    float* u = nullptr;
    int* perm = nullptr;
    Sub* subs = nullptr;
    int* nsub = nullptr;
    int maxsub = 0;
    float* mu_f = nullptr;
    double* mu_d = nullptr;
    // scratch
    float* u_tmp = nullptr;
    int* tile_of = nullptr;
    int* counts = nullptr;
    int* cursor = nullptr;
};

void layout_set(Arena& A, SetBufs& S, int n, int d, int n_grid, bool with_mu) {
    S.n = n;
    const int ntiles = mot_ntiles(d, n_grid);
    S.maxsub = (n + mot_sub_points(d) - 1) / mot_sub_points(d) + ntiles;
    S.u = A.take<float>((size_t)d * n);
    S.perm = A.take<int>(n);
    S.subs = A.take<Sub>(S.maxsub);
    S.nsub = A.take<int>(1);
    if (with_mu) {
        S.mu_f = A.take<float>(n);
        S.mu_d = A.take<double>(n);
    }
    S.u_tmp = A.take<float>((size_t)d * n);
    S.tile_of = A.take<int>(n);
    S.counts = A.take<int>(mot_ncells(d, n_grid));
    S.cursor = A.take<int>(mot_ncells(d, n_grid));
}

PointSet pointset_of(const SetBufs& S) {
    PointSet p;
    p.n = S.n;
    p.u = S.u;
    p.subs = S.subs;
    p.nsub = S.nsub;
    p.maxsub = S.maxsub;
    return p;
}

PrepSet prepset_of(const SetBufs& S, const float* x, const double* mu) {
    PrepSet P;
    P.x = x;
    P.mu = mu;
    P.n = S.n;
    P.u_tmp = S.u_tmp;
    P.tile_of = S.tile_of;
    P.counts = S.counts;
    P.cursor = S.cursor;
    P.u = S.u;
    P.perm = S.perm;
    P.mu_f = S.mu_f;
    P.mu_d = S.mu_d;
    P.subs = S.subs;
    P.nsub = S.nsub;
    P.maxsub = S.maxsub;
    return P;
}

// Bounding radius of the union of point sets (one host readback), then the grid choice.
int measure_and_choose(const std::vector<PrepSet>& sets, PrepSet* d_sets, float* box_scratch, float* box_out, int d,
                       double eta_min, double eta_max, const mot_options& o, GridChoice& g, cudaStream_t st) {
    CK(cudaMemcpyAsync(d_sets, sets.data(), sizeof(PrepSet) * sets.size(), cudaMemcpyHostToDevice, st));
    CK(launch_bounds(d_sets, (int)sets.size(), d, box_scratch, box_out, st));
    float h[7] = {0, 0, 0, 0, 0, 0, 0};
    CK(cudaMemcpyAsync(h, box_out, sizeof(float) * (2 * d + 1), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    double c[3] = {0, 0, 0};
    for (int t = 0; t < d; ++t) {
        if (!std::isfinite(h[2 * t]) || !std::isfinite(h[2 * t + 1])) return MOT_ENUMERIC;
        c[t] = 0.5 * ((double)h[2 * t] + (double)h[2 * t + 1]);
    }
    // radius about the FP32 box centre used on the device; add the centre rounding
    double R = std::sqrt((double)h[2 * d]);
    double dc = 0.0;
    for (int t = 0; t < d; ++t) {
        double cf = (double)(0.5f * (h[2 * t] + h[2 * t + 1]));
        dc += (cf - c[t]) * (cf - c[t]);
    }
    R = R * (1.0 + 1e-6) + std::sqrt(dc) + 1e-30;
    if (!std::isfinite(R)) return MOT_ENUMERIC;
    g = choose_grid(d, R, eta_min, eta_max, o.n_grid, o.eps_B);
    for (int t = 0; t < 3; ++t) g.c[t] = c[t];
    return MOT_OK;
}

int make_D_for(double eta_e_norm, const GridChoice& g, int d, const mot_options& o, double* sa, double* sb,
               float* D, cudaStream_t st, bool deconv = true) {
    double poly[2 * 8 + 1];
    if (o.p > 8) return MOT_EINVAL;
    if (!boundary_poly(eta_e_norm, kTau, o.eps_B, o.p, poly)) return MOT_ENUMERIC;
    CK(launch_make_D(d, g.M, g.n, eta_e_norm, kTau, o.eps_B, o.p, poly, sa, sb, D, st, deconv));
    return MOT_OK;
}

// =============================================================================================
// tree plan
// =============================================================================================
struct Level {
    std::vector<Task> src, tgt;   // host copies
    std::vector<int> node;        // wavefront chunk: graph node of every tgt task
    Task* d_src = nullptr;
    Task* d_tgt = nullptr;
    int grid_src = 1, grid_tgt = 1, ntb = 1, nsplit = 1;
    bool msg_only = false;        // every task: EPI_MSG with a kernel sum (fused kernel's lean instance)
};

struct TreePlan {
    // problem
    int K = 0, d = 0, path = MOT_PATH_NFFT;
    double eta = 0.0;
    std::vector<int> order, new_of, parent, depth;
    int root_label = 0;
    std::vector<std::vector<int>> children;
    std::vector<int> n;            // BFS labels
    std::vector<double> w;         // weight of edge {p(k), k}
    std::vector<unsigned char> free_;
    GridChoice g;
    mot_options o;
    // device buffers
    std::vector<SetBufs> sets;
    std::vector<float*> phi, beta, gam, gex, grid, hgrid, rawf, rawb, rawc;
    std::vector<float2*> spec;
    std::vector<float*> D;          // per edge
    VecScale* sc = nullptr;         // [4K]: phi, beta, gamma, gex
    IterAcc* acc = nullptr;
    int* iter = nullptr;
    double* acc_node = nullptr;     // [3K]
    int* err = nullptr;
    Factor* d_fac = nullptr;
    VecScale** d_resets = nullptr;
    size_t n_resets = 0;
    PrepSet* d_sets = nullptr;
    float* box_scratch = nullptr;
    float* box_out = nullptr;
    double* dscr_a = nullptr;
    double* dscr_b = nullptr;
    char* stats_begin = nullptr;    // contiguous readback region: acc ring, acc_node, sc, err
    size_t stats_bytes = 0;
    Task* d_tasks = nullptr;
    size_t n_tasks_total = 0;
    // host-side task construction
    std::vector<Factor> fac;
    std::vector<VecScale*> resets;
    std::vector<Level> fwd, bwd, chk;
    size_t it_reset0 = 0, it_reset_n = 0;     // iteration prologue: phi (prev kept) and gamma records
    size_t ck_reset0 = 0, ck_reset_n = 0;     // check prologue: gamma-ex records (+ acc_node zeroed)
    bool fused = false;                        // 2-D grids <= 64: one cluster kernel per level
    bool ndft = false;                         // ... evaluating the trigonometric sums exactly (ndft2d.cu)
    // wavefront schedule (fused path): beta_k alternates between two copies from sweep to sweep
    std::vector<float*> beta2;                 // the second copy of every beta_k
    std::vector<Level> chk1;                   // check pass reading the second copy
    bool wave = false;
    int par = 0;                               // copy holding the latest beta, in enqueue order
    std::vector<Level> wlev;                   // the launches of one chunk
    int wave_S = -1, wave_q0 = -1;             // chunk length and starting copy of wlev
    size_t fac_base = 0, res_base = 0;         // where the chunk's factors / resets start
    size_t fac_cap = 0, res_cap = 0;
    Task* d_wtasks = nullptr;
    size_t wtask_cap = 0;
    int graph_par = -1;                        // starting copy of the captured chunk
    size_t wave_root_reset = 0;                // reset-list entry of the root's scale record
    long long launches_per_chunk = 0;
    // persistent wavefront kernel (options.wavefront = 1): the whole chunk in one launch
    bool persist = false;
    int wave_clusters = 0;                     // clusters launched (co-resident on an idle GPU)
    int wave_ntask = 0;
    int* d_deps = nullptr;                     // dependency lists of the chunk's products
    size_t deps_cap = 0;
    int* d_flags = nullptr;                    // completion flags (epoch of the launch)
    WaveCtl* d_ctl = nullptr;
    bool wave_chk = false;                     // the chunk schedule ends with the check pass
    bool check_done = false;                   // the last chunk run included the check pass
    Globals G;
    // graph
    cudaGraphExec_t gexec = nullptr;
    int graph_iters = 0;
    long long launches_per_iter = 0, launches_per_check = 0;

    VecScale* phi_sc(int k) const { return sc + k; }
    VecScale* beta_sc(int k) const { return sc + K + k; }
    VecScale* gam_sc(int k) const { return sc + 2 * K + k; }
    VecScale* gex_sc(int k) const { return sc + 3 * K + k; }
    VecScale* beta_sc_q(int k, int q) const { return q ? sc + 4 * K + k : sc + K + k; }
    float* beta_q(int k, int q) const { return q ? beta2[k] : beta[k]; }
};

constexpr int kWaveMax = 32;                   // longest chunk pipelined as one wavefront

int validate_problem(const mot_problem* P) {
    if (!P) return MOT_EINVAL;
    if (P->K < 2 || P->K > 64 || P->d < 1 || P->d > 3) return MOT_EINVAL;
    if (!P->n || !P->x || !P->mu) return MOT_EINVAL;
    if (!(P->eta > 0.0) || !std::isfinite(P->eta)) return MOT_EINVAL;
    for (int k = 0; k < P->K; ++k) {
        if (P->n[k] < 1 || P->n[k] > (1 << 26)) return MOT_EINVAL;
        if (!P->x[k] || !P->mu[k]) return MOT_EINVAL;
    }
    if (P->topology != MOT_TREE && P->topology != MOT_CIRCLE) return MOT_EINVAL;
    if (P->topology == MOT_TREE) {
        if (!P->edges || P->x_close) return MOT_EINVAL;
        if (P->root < MOT_ROOT_CENTRE || P->root >= P->K) return MOT_EINVAL;
    }
    int ne = P->topology == MOT_TREE ? P->K - 1 : P->K;
    if (P->edge_w)
        for (int e = 0; e < ne; ++e)
            if (!(P->edge_w[e] > 0.0) || !std::isfinite(P->edge_w[e])) return MOT_EINVAL;
    return MOT_OK;
}

// BFS relabelling so that p(k) < k (Section 4.1).
int tree_structure(const mot_problem* P, TreePlan& T) {
    const int K = P->K;
    std::vector<std::vector<std::pair<int, double>>> adj(K);
    for (int e = 0; e < K - 1; ++e) {
        int a = P->edges[2 * e], b = P->edges[2 * e + 1];
        if (a < 0 || a >= K || b < 0 || b >= K || a == b) return MOT_ENOTTREE;
        double w = P->edge_w ? P->edge_w[e] : 1.0;
        adj[a].push_back({b, w});
        adj[b].push_back({a, w});
    }
    for (auto& v : adj) std::sort(v.begin(), v.end());
    int root = P->root;
    if (root == MOT_ROOT_CENTRE) {
        // a centre: the node of least eccentricity (smallest label on ties), so that the
        // backward pass of Algorithm 2 has the fewest sequential depth levels
        int best = K + 1;
        for (int r = 0; r < K; ++r) {
            std::vector<int> dist(K, -1);
            std::deque<int> bq{r};
            dist[r] = 0;
            int ecc = 0, seen = 1;
            while (!bq.empty()) {
                int u = bq.front();
                bq.pop_front();
                for (auto& vw : adj[u])
                    if (dist[vw.first] < 0) {
                        dist[vw.first] = dist[u] + 1;
                        ecc = std::max(ecc, dist[vw.first]);
                        ++seen;
                        bq.push_back(vw.first);
                    }
            }
            if (seen != K) return MOT_ENOTTREE;
            if (P->free_nodes && P->free_nodes[r]) continue;   // the root must be constrained
            if (ecc < best) {
                best = ecc;
                root = r;
            }
        }
    }
    T.K = K;
    T.root_label = root;
    T.order.assign(1, root);
    T.new_of.assign(K, -1);
    T.new_of[root] = 0;
    T.parent.assign(1, -1);
    T.depth.assign(1, 0);
    T.w.assign(1, 1.0);
    std::deque<int> q{root};
    while (!q.empty()) {
        int u = q.front();
        q.pop_front();
        for (auto& vw : adj[u]) {
            int v = vw.first;
            if (T.new_of[v] >= 0) continue;
            T.new_of[v] = (int)T.order.size();
            T.order.push_back(v);
            T.parent.push_back(T.new_of[u]);
            T.depth.push_back(T.depth[T.new_of[u]] + 1);
            T.w.push_back(vw.second);
            q.push_back(v);
        }
    }
    if ((int)T.order.size() != K) return MOT_ENOTTREE;
    // With a free root the sibling updates of Algorithm 2 act as a Jacobi step on the scaling
    // gauge (period-2 oscillation for two children, divergence for more): not supported.
    if (P->free_nodes && P->free_nodes[root]) return MOT_EUNSUPPORTED;
    T.children.assign(K, {});
    for (int k = 1; k < K; ++k) T.children[T.parent[k]].push_back(k);
    for (int k = 0; k < K; ++k)
        if ((int)T.children[k].size() + 1 > MOT_MAXFAC - 2) return MOT_EUNSUPPORTED;
    T.n.resize(K);
    T.free_.assign(K, 0);
    for (int k = 0; k < K; ++k) {
        T.n[k] = (int)P->n[T.order[k]];
        if (P->free_nodes) T.free_[k] = P->free_nodes[T.order[k]] ? 1 : 0;
    }
    return MOT_OK;
}

// Workspace layout of a tree plan (sizes only depend on the problem's shape and the grid).
void layout_tree(Arena& A, TreePlan& T) {
    const int K = T.K, d = T.d;
    const bool nfft = T.path == MOT_PATH_NFFT;
    const int ng = T.g.n, M = T.g.M;
    size_t gsz = 1;
    for (int t = 0; t < d; ++t) gsz *= ng;
    T.sets.assign(K, SetBufs());
    for (int k = 0; k < K; ++k) layout_set(A, T.sets[k], T.n[k], d, ng, true);
    T.phi.assign(K, nullptr);
    T.beta.assign(K, nullptr);
    T.beta2.assign(K, nullptr);
    T.gam.assign(K, nullptr);
    T.gex.assign(K, nullptr);
    T.grid.assign(K, nullptr);
    T.hgrid.assign(K, nullptr);
    T.spec.assign(K, nullptr);
    T.D.assign(K, nullptr);
    T.rawf.assign(K, nullptr);
    T.rawb.assign(K, nullptr);
    T.rawc.assign(K, nullptr);
    for (int k = 0; k < K; ++k) T.phi[k] = A.take<float>(T.n[k]);
    for (int k = 1; k < K; ++k) {
        const int p = T.parent[k];
        T.beta[k] = A.take<float>(T.n[p]);
        T.beta2[k] = A.take<float>(T.n[p]);
        T.gam[k] = A.take<float>(T.n[k]);
        T.gex[k] = A.take<float>(T.n[k]);
        if (nfft) {
            T.grid[k] = A.take<float>(gsz);
            T.hgrid[k] = A.take<float>(gsz);
            if (d == 3) T.spec[k] = A.take<float2>((size_t)ng * (2 * M + 1) * (M + 1));
            T.D[k] = A.take<float>(D_floats(d, M));
        } else {
            T.rawf[k] = A.take<float>(T.n[k]);
            T.rawb[k] = A.take<float>(T.n[p]);
            T.rawc[k] = A.take<float>(T.n[k]);
        }
    }
    // readback region (scale records: phi, beta, gamma, gamma-ex, second beta copy)
    size_t stats = sizeof(IterAcc) * kRing + sizeof(double) * 3 * K + sizeof(VecScale) * 5 * K + 16;
    T.stats_begin = A.take<char>(stats);
    T.stats_bytes = stats;
    if (!A.measure) {
        T.acc = reinterpret_cast<IterAcc*>(T.stats_begin);
        T.acc_node = reinterpret_cast<double*>(T.stats_begin + sizeof(IterAcc) * kRing);
        T.sc = reinterpret_cast<VecScale*>(T.stats_begin + sizeof(IterAcc) * kRing + sizeof(double) * 3 * K);
        T.err = reinterpret_cast<int*>(T.stats_begin + stats - 16);
        T.iter = T.err + 1;
    }
    T.d_sets = A.take<PrepSet>(K);
    T.box_scratch = A.take<float>(8);
    T.box_out = A.take<float>(8);
    if (nfft) {
        size_t s = make_D_scratch_doubles(d, M);
        T.dscr_a = A.take<double>(s);
        T.dscr_b = A.take<double>(s);
    }
    // factor, reset and task arrays: generous upper bounds for the sweep-by-sweep levels and the
    // check passes, plus one wavefront chunk (per sweep at most 2 (K - 1) + 1 tasks, 6 K factors
    // and 3 K + 1 resets)
    T.fac_cap = (size_t)16 * K + 8 * (size_t)K * 4 + 64 * (size_t)K + (size_t)kWaveMax * 6 * K;
    T.res_cap = 8 * (size_t)K + 8 + (size_t)kWaveMax * (3 * (size_t)K + 1);
    T.d_fac = A.take<Factor>(T.fac_cap);
    T.d_resets = A.take<VecScale*>(T.res_cap);
    T.d_tasks = A.take<Task>(24 * (size_t)K + 16);
    T.wtask_cap = (size_t)kWaveMax * (2 * (size_t)K + 1);
    T.d_wtasks = A.take<Task>(T.wtask_cap);
    // dependency lists: per sweep at most about 6 K edges, and the check pass at most K (K + 2)
    T.deps_cap = (size_t)kWaveMax * (7 * (size_t)K + 8) + (size_t)K * (K + 4);
    T.d_deps = A.take<int>(T.deps_cap);
    T.d_flags = A.take<int>(T.wtask_cap);
    T.d_ctl = A.take<WaveCtl>(1);
}

// ---- task construction ------------------------------------------------------------------
int add_factor(TreePlan& T, const float* mant, const VecScale* sc, int inv) {
    Factor f;
    f.mant = mant;
    f.sc = sc;
    f.inv = inv;
    f.use_prev = 0;
    T.fac.push_back(f);
    return (int)T.fac.size() - 1;
}

Task blank_task() {
    Task t;
    std::memset(&t, 0, sizeof(t));
    return t;
}

PointSet ps_of(const TreePlan& T, int k) { return pointset_of(T.sets[k]); }

// Source side of the message from node `src` towards neighbour `dst`, built from the current
// scalings: phi^src (.) [gamma-ex_src] (.) prod of the children's beta except dst.
// `q` selects the copy of the children's beta (the wavefront alternates two copies).
void src_general(TreePlan& T, Task& t, int src, int exclude_child, bool with_phi, int gamma_kind, int q = 0) {
    t.src = ps_of(T, src);
    t.sf0 = (int)T.fac.size();
    if (with_phi && !T.free_[src]) add_factor(T, T.phi[src], T.phi_sc(src), 0);
    if (gamma_kind == 1 && src != 0) add_factor(T, T.gam[src], T.gam_sc(src), 0);
    if (gamma_kind == 2 && src != 0) add_factor(T, T.gex[src], T.gex_sc(src), 0);
    for (int c : T.children[src])
        if (c != exclude_child) add_factor(T, T.beta_q(c, q), T.beta_sc_q(c, q), 0);
    t.snf = (int)T.fac.size() - t.sf0;
}

void tgt_children(TreePlan& T, Task& t, int k, bool with_phi, int q = 0) {
    t.tf0 = (int)T.fac.size();
    if (with_phi && !T.free_[k]) add_factor(T, T.phi[k], T.phi_sc(k), 0);
    for (int c : T.children[k]) add_factor(T, T.beta_q(c, q), T.beta_sc_q(c, q), 0);
    t.tnf = (int)T.fac.size() - t.tf0;
}

void edge_grids(TreePlan& T, Task& t, int k, float* raw) {
    t.grid = T.grid[k];
    t.hgrid = T.hgrid[k];
    t.spec = T.spec[k];
    t.D = T.D[k];
    t.raw = raw;
    const double eta_e = T.eta / T.w[k];
    const double eta_n = eta_e / (T.g.s * T.g.s);
    t.eta_u = (float)(eta_n * (double)T.g.n * (double)T.g.n);
}

// Check pass task of node k (Theorem 4.1 at the current scalings, beta copy q): EPI_MARG with the
// exact forward message gamma-ex_k = K^T (phi^p (.) gamma-ex_p (.) beta^{C_p \ k}), or for the root
// (no kernel sum) its marginal from its children's messages.
Task check_task(TreePlan& T, int k, int q) {
    Task t = blank_task();
    if (k > 0) {
        src_general(T, t, T.parent[k], k, true, 2, q);
        edge_grids(T, t, k, T.rawc[k]);
        t.out = T.gex[k];
        t.out_sc = T.gex_sc(k);
    }
    t.tgt = ps_of(T, k);
    t.mode = EPI_MARG;
    tgt_children(T, t, k, true, q);
    t.mu_d = T.free_[k] ? nullptr : T.sets[k].mu_d;
    t.phi = T.phi[k];
    t.phi_sc = T.phi_sc(k);
    t.acc_node = T.acc_node + 3 * k;
    return t;
}

void build_tasks(TreePlan& T) {
    const int K = T.K;
    T.fac.clear();
    T.resets.clear();
    T.fwd.clear();
    T.bwd.clear();
    T.chk.clear();
    int maxdepth = 0;
    for (int k = 0; k < K; ++k) maxdepth = std::max(maxdepth, T.depth[k]);

    // ---- forward pass: gamma_k and phi^k ------------------------------------------------
    std::vector<int> flev(K, 0);
    int nfl = 1;
    for (int k = 1; k < K; ++k) {
        const int p = T.parent[k];
        flev[k] = (p == 0 || !T.free_[p]) ? 0 : flev[p] + 1;
        nfl = std::max(nfl, flev[k] + 1);
    }
    T.fwd.assign(nfl, Level());
    for (int k = 1; k < K; ++k) {
        const int p = T.parent[k];
        Task t = blank_task();
        if (!T.free_[p]) {
            // phi^p (.) gamma_p (.) beta^{C_p \ k} = mu^p / beta_k
            t.src = ps_of(T, p);
            t.sf0 = (int)T.fac.size();
            add_factor(T, T.sets[p].mu_f, nullptr, 0);
            add_factor(T, T.beta[k], T.beta_sc(k), 1);
            t.snf = 2;
        } else {
            src_general(T, t, p, k, false, 1);
        }
        edge_grids(T, t, k, T.rawf[k]);
        t.tgt = ps_of(T, k);
        t.mode = T.free_[k] ? EPI_PHI_FREE : EPI_PHI;
        tgt_children(T, t, k, false);
        t.mu_f = T.sets[k].mu_f;
        t.mu_d = T.sets[k].mu_d;
        t.out = T.gam[k];
        t.out_sc = T.gam_sc(k);
        t.phi = T.phi[k];
        t.phi_sc = T.phi_sc(k);
        T.fwd[flev[k]].src.push_back(t);
        T.fwd[flev[k]].tgt.push_back(t);
    }
    {   // root step: mass and root violation of the last iterate, then phi^1
        Task t = blank_task();
        t.tgt = ps_of(T, 0);
        t.mode = EPI_ROOT;
        t.free_node = T.free_[0];
        tgt_children(T, t, 0, false);
        t.mu_f = T.sets[0].mu_f;
        t.mu_d = T.sets[0].mu_d;
        t.phi = T.phi[0];
        t.phi_sc = T.phi_sc(0);
        T.fwd[0].tgt.push_back(t);
    }
    // iteration prologue: keep the scale of the last scalings (root mass), reset the scaling
    // and gamma records that the forward pass produces
    T.it_reset0 = T.resets.size();
    for (int k = 0; k < K; ++k) T.resets.push_back(T.phi_sc(k));
    for (int k = 1; k < K; ++k) T.resets.push_back(T.gam_sc(k));
    T.it_reset_n = T.resets.size() - T.it_reset0;

    // ---- backward pass: beta_k from the deepest level up ---------------------------------
    T.bwd.assign(std::max(maxdepth, 1), Level());
    for (int k = K - 1; k >= 1; --k) {
        Task t = blank_task();
        src_general(T, t, k, -1, true, 0);
        edge_grids(T, t, k, T.rawb[k]);
        t.tgt = ps_of(T, T.parent[k]);
        t.mode = EPI_MSG;
        t.out = T.beta[k];
        t.out_sc = T.beta_sc(k);
        size_t r0 = T.resets.size();
        T.resets.push_back(T.beta_sc(k));
        t.reset_n = 1;
        t.reset_list = (VecScale* const*)(uintptr_t)r0;
        const int lev = maxdepth - T.depth[k];       // deepest first
        T.bwd[lev].src.push_back(t);
        T.bwd[lev].tgt.push_back(t);
    }

    // ---- check pass: exact marginals at the current scalings (Theorem 4.1), for either copy
    // of beta ----------------------------------------------------------------------------------
    for (int q = 0; q < 2; ++q) {
        std::vector<Level>& chk = q ? T.chk1 : T.chk;
        chk.assign(std::max(maxdepth, 1), Level());
        for (int k = 1; k < K; ++k) {
            Task t = check_task(T, k, q);
            chk[T.depth[k] - 1].src.push_back(t);
            chk[T.depth[k] - 1].tgt.push_back(t);
        }
        chk[0].tgt.push_back(check_task(T, 0, q));
    }
    T.ck_reset0 = T.resets.size();
    for (int k = 1; k < K; ++k) T.resets.push_back(T.gex_sc(k));
    T.ck_reset_n = T.resets.size() - T.ck_reset0;
}

// Copy task arrays to the device, resolving reset-list offsets to device pointers.
int upload_tasks(TreePlan& T, cudaStream_t st) {
    if (T.fac.size() > T.fac_cap - (size_t)kWaveMax * 6 * T.K) return MOT_EUNSUPPORTED;
    if (T.resets.size() > T.res_cap - (size_t)kWaveMax * (3 * (size_t)T.K + 1)) return MOT_EUNSUPPORTED;
    T.fac_base = T.fac.size();
    T.res_base = T.resets.size();
    T.wave_S = T.wave_q0 = -1;
    CK(cudaMemcpyAsync(T.d_fac, T.fac.data(), sizeof(Factor) * T.fac.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(T.d_resets, T.resets.data(), sizeof(VecScale*) * T.resets.size(), cudaMemcpyHostToDevice, st));
    std::vector<Task> all;
    auto place = [&](std::vector<Level>& levels) {
        for (auto& L : levels) {
            L.msg_only = !L.tgt.empty();
            for (auto& t : L.tgt) L.msg_only = L.msg_only && t.mode == EPI_MSG && t.hgrid != nullptr;
            for (auto* v : {&L.src, &L.tgt}) {
                for (auto& t : *v)
                    if (t.reset_n > 0) t.reset_list = T.d_resets + (uintptr_t)t.reset_list;
            }
        }
    };
    place(T.fwd);
    place(T.bwd);
    place(T.chk);
    place(T.chk1);
    for (auto* lv : {&T.fwd, &T.bwd, &T.chk, &T.chk1})
        for (auto& L : *lv) {
            for (auto& t : L.src) all.push_back(t);
            for (auto& t : L.tgt) all.push_back(t);
        }
    if (all.size() > 24 * (size_t)T.K + 16) return MOT_EUNSUPPORTED;
    CK(cudaMemcpyAsync(T.d_tasks, all.data(), sizeof(Task) * all.size(), cudaMemcpyHostToDevice, st));
    size_t off = 0;
    for (auto* lv : {&T.fwd, &T.bwd, &T.chk, &T.chk1})
        for (auto& L : *lv) {
            L.d_src = T.d_tasks + off;
            off += L.src.size();
            L.d_tgt = T.d_tasks + off;
            off += L.tgt.size();
            int ms = 1, mt = 1, maxn = 1;
            for (auto& t : L.src) ms = std::max(ms, t.src.maxsub);
            for (auto& t : L.tgt) {
                mt = std::max(mt, t.hgrid ? t.tgt.maxsub : (t.tgt.n + 255) / 256);
                maxn = std::max(maxn, t.tgt.n);
            }
            L.grid_src = std::min(ms, 1024);
            L.grid_tgt = std::min(mt, 1024);
            if (T.path != MOT_PATH_NFFT) {
                L.grid_tgt = std::min((maxn + 255) / 256, 1024);
                L.ntb = (maxn + 511) / 512;
                int ns = (int)L.src.size();
                int target = 4 * 152;
                int split = target / std::max(1, L.ntb * std::max(ns, 1));
                L.nsplit = std::max(1, std::min(split, 64));
            }
        }
    T.G.iter = T.iter;
    T.G.acc = T.acc;
    T.G.R = kRing;
    T.G.floor_ = 1e-30f;
    T.G.n_grid = T.g.n;
    T.G.M = T.g.M;
    T.G.fac = T.d_fac;
    return MOT_OK;
}

// ---- wavefront chunk --------------------------------------------------------------------------
// Sweep s of a chunk (s = 0..S-1) reads the copy q_s = (q0 + s) mod 2 of every beta and writes the
// other copy.  With the forward identity above, the products of Algorithm 2 depend on
//   F_k(s) (gamma_k, then phi^k)  <- B_k(s-1) and B_c(s-1) for the children c of k
//   R(s)   (root update)          <- B_c(s-1) for the children of the root
//   B_k(s) (beta_k)               <- F_k(s) and B_c(s)
// and, as a copy is rewritten every second sweep, B_k(s) also waits for the readers of the copy it
// overwrites in sweep s-1: F_k(s-1) and F_{p(k)}(s-1), or R(s-1) when p(k) is the root.  Every
// product goes into the first launch after its inputs that has room.  The scale record of the root
// scaling is saved and reset (R(s) reads the previous one) by a product that runs between R(s-1)
// and R(s), and by the chunk prologue for s = 0.
// The launch of every product of an S-sweep chunk on a tree given by parent[] (BFS labels:
// parent[0] = -1, parent[k] < k), at most `cap` products per launch.  Fills tF / tB [S][K]
// (entries k >= 1), tR [S], the carrier child of each R(s) (s >= 1, -1 for s = 0) and the number
// of launches.  MOT_EUNSUPPORTED if no child of the root can carry the root's record.
int wave_times(int K, const int* parent, int S, int cap, int* tF, int* tB, int* tR, int* carrier, int* nlaunch,
               std::vector<std::vector<int>>* pred_out = nullptr) {
    if (K < 2 || S < 1 || cap < 1 || !parent || parent[0] != -1) return MOT_EINVAL;
    std::vector<std::vector<int>> children(K);
    for (int k = 1; k < K; ++k) {
        if (parent[k] < 0 || parent[k] >= k) return MOT_EINVAL;
        children[parent[k]].push_back(k);
    }
    // tasks of sweep s: R(s) = s W, F(s, k) = s W + k, B(s, k) = s W + K - 1 + k (W = 2K - 1); the
    // order R(s), F(s, 1..K-1), B(s, K-1..1), s = 0..S-1, is topological
    const int W = 2 * K - 1, N = S * W;
    auto R_ = [&](int s) { return s * W; };
    auto F_ = [&](int s, int k) { return s * W + k; };
    auto B_ = [&](int s, int k) { return s * W + K - 1 + k; };
    std::vector<std::vector<int>> pred(N), succ(N);
    auto edge = [&](int u, int v) {
        pred[v].push_back(u);
        succ[u].push_back(v);
    };
    for (int s = 0; s < S; ++s) {
        if (s > 0)
            for (int c : children[0]) edge(B_(s - 1, c), R_(s));            // R(s) <- B_c(s-1)
        for (int k = 1; k < K; ++k) {
            if (s > 0) {
                edge(B_(s - 1, k), F_(s, k));                                // F_k(s) <- B_k(s-1)
                for (int c : children[k]) edge(B_(s - 1, c), F_(s, k));      //         <- B_c(s-1)
            }
            edge(F_(s, k), B_(s, k));                                        // B_k(s) <- F_k(s)
            for (int c : children[k]) edge(B_(s, c), B_(s, k));              //         <- B_c(s)
            if (s > 0) {                                                     // readers of the copy
                edge(F_(s - 1, k), B_(s, k));                                // B_k(s) overwrites
                edge(parent[k] == 0 ? R_(s - 1) : F_(s - 1, parent[k]), B_(s, k));
            }
            if (parent[k] == 0) edge(R_(s), B_(s, k));   // so that it can carry R(s+1)'s record
        }
    }
    // topological order and the longest remaining chain of every task (its priority)
    std::vector<int> order;
    order.reserve(N);
    for (int s = 0; s < S; ++s) {
        order.push_back(R_(s));
        for (int k = 1; k < K; ++k) order.push_back(F_(s, k));
        for (int k = K - 1; k >= 1; --k) order.push_back(B_(s, k));
    }
    std::vector<int> chain(N, 1);
    for (int i = N - 1; i >= 0; --i) {
        const int u = order[i];
        for (int v : succ[u]) chain[u] = std::max(chain[u], chain[v] + 1);
    }
    // list scheduling: each launch takes up to `cap` of the tasks whose predecessors all ran in
    // earlier launches, longest remaining chain first (then earlier sweep, then task order)
    std::vector<int> when(N, -1), waiting(N), ready_at(N, 0), rank(N);
    for (int i = 0; i < N; ++i) rank[order[i]] = i;
    std::vector<int> pool;
    for (int u = 0; u < N; ++u) {
        waiting[u] = (int)pred[u].size();
        if (waiting[u] == 0) pool.push_back(u);
    }
    int placed = 0, t = 0;
    while (placed < N) {
        std::vector<int> cand;
        for (int u : pool)
            if (ready_at[u] <= t) cand.push_back(u);
        if (cand.empty()) return MOT_EUNSUPPORTED;   // (never: the graph is acyclic)
        std::sort(cand.begin(), cand.end(), [&](int x, int y) {
            if (chain[x] != chain[y]) return chain[x] > chain[y];
            return rank[x] < rank[y];
        });
        const int take = std::min<int>(cap, (int)cand.size());
        for (int i = 0; i < take; ++i) {
            const int u = cand[i];
            when[u] = t;
            ++placed;
            pool.erase(std::find(pool.begin(), pool.end(), u));
            for (int v : succ[u]) {
                ready_at[v] = std::max(ready_at[v], t + 1);
                if (--waiting[v] == 0) pool.push_back(v);
            }
        }
        ++t;
    }
    *nlaunch = t;
    for (int s = 0; s < S; ++s) {
        tR[s] = when[R_(s)];
        tF[(size_t)s * K] = tB[(size_t)s * K] = -1;
        for (int k = 1; k < K; ++k) {
            tF[(size_t)s * K + k] = when[F_(s, k)];
            tB[(size_t)s * K + k] = when[B_(s, k)];
        }
    }
    if (pred_out) *pred_out = pred;
    // the root scaling's record is saved and reset by the last product B_c(s-1) of a child c of the
    // root: it runs after R(s-1) (an edge above) and before R(s) (which waits for it)
    carrier[0] = -1;
    for (int s = 1; s < S; ++s) {
        int best = -1;
        for (int c : children[0])
            if (best < 0 || when[B_(s - 1, c)] > when[B_(s - 1, best)]) best = c;
        if (best < 0 || !(when[B_(s - 1, best)] > tR[s - 1] && when[B_(s - 1, best)] < tR[s])) return MOT_EUNSUPPORTED;
        carrier[s] = best;
    }
    return MOT_OK;
}

// with_check (persistent kernel only): the chunk ends with the check pass at its final scalings,
// each check product waiting for exactly the products whose results it reads.
int build_wave(TreePlan& T, int S, int q0, bool with_check, cudaStream_t st) {
    const int K = T.K;
    T.fac.resize(T.fac_base);
    T.resets.resize(T.res_base);
    // a launch takes at most as many products as clusters fit on the GPU at once (one more would
    // run as a second wave); a product that finds its first possible launch full takes the next
    // (the persistent kernel: as many products as it runs clusters)
    const int ncl = T.persist ? T.wave_clusters
                              : (T.ndft ? ndft2d_max_active_clusters() : fused2d_max_active_clusters());
    const int cap = std::max(1, ncl > 0 ? ncl : 8);
    std::vector<int> tFf((size_t)S * K), tBf((size_t)S * K), tR(S), carrier(S);
    int nlaunch = 0;
    std::vector<std::vector<int>> pred;
    RET(wave_times(K, T.parent.data(), S, cap, tFf.data(), tBf.data(), tR.data(), carrier.data(), &nlaunch, &pred));
    const int W = 2 * K - 1;                   // graph nodes of sweep s: R = sW, F_k = sW + k, B_k = sW + K - 1 + k
    auto tF = [&](int s, int k) { return tFf[(size_t)s * K + k]; };
    auto tB = [&](int s, int k) { return tBf[(size_t)s * K + k]; };
    T.wlev.assign(nlaunch, Level());
    T.wave_root_reset = T.resets.size();
    T.resets.push_back(T.phi_sc(0));
    for (int s = 0; s < S; ++s) {
        const int q = (q0 + s) & 1, qn = q ^ 1;
        const int off = S - 1 - s;
        for (int k = 1; k < K; ++k) {         // F_k(s): gamma_k = K^T (mu^p / beta_k), then phi^k
            const int p = T.parent[k];
            Task t = blank_task();
            t.src = ps_of(T, p);
            t.sf0 = (int)T.fac.size();
            add_factor(T, T.sets[p].mu_f, nullptr, 0);
            add_factor(T, T.beta_q(k, q), T.beta_sc_q(k, q), 1);
            t.snf = 2;
            edge_grids(T, t, k, T.rawf[k]);
            t.tgt = ps_of(T, k);
            t.mode = EPI_PHI;
            tgt_children(T, t, k, false, q);
            t.mu_f = T.sets[k].mu_f;
            t.mu_d = T.sets[k].mu_d;
            t.out = T.gam[k];
            t.out_sc = T.gam_sc(k);
            t.phi = T.phi[k];
            t.phi_sc = T.phi_sc(k);
            const size_t r0 = T.resets.size();
            T.resets.push_back(T.phi_sc(k));
            T.resets.push_back(T.gam_sc(k));
            t.reset_n = 2;
            t.reset_list = (VecScale* const*)(uintptr_t)r0;
            t.iter_off = off;
            T.wlev[tF(s, k)].tgt.push_back(t);
            T.wlev[tF(s, k)].node.push_back(s * W + k);
        }
        {                                      // R(s): mass of the last iterate, then phi^1
            Task t = blank_task();
            t.tgt = ps_of(T, 0);
            t.mode = EPI_ROOT;
            tgt_children(T, t, 0, false, q);
            t.mu_f = T.sets[0].mu_f;
            t.mu_d = T.sets[0].mu_d;
            t.phi = T.phi[0];
            t.phi_sc = T.phi_sc(0);
            t.iter_off = off;
            T.wlev[tR[s]].tgt.push_back(t);
            T.wlev[tR[s]].node.push_back(s * W);
        }
        for (int k = K - 1; k >= 1; --k) {    // B_k(s) into the other copy
            Task t = blank_task();
            src_general(T, t, k, -1, true, 0, qn);
            edge_grids(T, t, k, T.rawb[k]);
            t.tgt = ps_of(T, T.parent[k]);
            t.mode = EPI_MSG;
            t.out = T.beta_q(k, qn);
            t.out_sc = T.beta_sc_q(k, qn);
            const size_t r0 = T.resets.size();
            T.resets.push_back(T.beta_sc_q(k, qn));
            t.reset_n = 1;
            if (s + 1 < S && carrier[s + 1] == k) {
                T.resets.push_back(T.phi_sc(0));
                t.reset_n = 2;
                t.save_prev = 1;
            }
            t.reset_list = (VecScale* const*)(uintptr_t)r0;
            T.wlev[tB(s, k)].tgt.push_back(t);
            T.wlev[tB(s, k)].node.push_back(s * W + K - 1 + k);
        }
    }
    // the check pass (Theorem 4.1 at the chunk's final scalings, beta copy qf): node S W + k;
    // BFS order puts every parent before its children.  Each check product resets the record of
    // the message it writes and zeroes its node's accumulators (it is their only writer).
    const int qf = (q0 + S) & 1;
    if (with_check) {
        T.wlev.emplace_back();
        Level& L = T.wlev.back();
        for (int k = 0; k < K; ++k) {
            Task t = check_task(T, k, qf);
            t.zero_d = T.acc_node + 3 * k;
            t.zero_n = 3;
            if (k > 0) {
                const size_t r0 = T.resets.size();
                T.resets.push_back(T.gex_sc(k));
                t.reset_n = 1;
                t.reset_list = (VecScale* const*)(uintptr_t)r0;
            }
            L.tgt.push_back(t);
            L.node.push_back(S * W + k);
        }
        pred.resize((size_t)S * W + K);
        const int s = S - 1;
        auto Fn = [&](int k) { return k == 0 ? s * W : s * W + k; };   // producer of phi^k
        auto Bn = [&](int k) { return s * W + K - 1 + k; };
        for (int k = 0; k < K; ++k) {
            std::vector<int>& pr = pred[(size_t)S * W + k];
            pr.push_back(Fn(k));                                       // phi^k
            for (int c : T.children[k]) pr.push_back(Bn(c));           // its children's beta
            if (k > 0) {
                const int p = T.parent[k];
                pr.push_back(Fn(p));                                   // phi^p
                if (p > 0) pr.push_back(S * W + p);                    // gamma-ex_p
                for (int c : T.children[p])
                    if (c != k) pr.push_back(Bn(c));                   // the siblings' beta
            }
        }
    }
    // upload the chunk's factors, resets and tasks
    if (T.fac.size() > T.fac_cap || T.resets.size() > T.res_cap) return MOT_EUNSUPPORTED;
    std::vector<Task> all;
    std::vector<int> flat_of((size_t)S * W + K, -1), node_of;
    for (auto& L : T.wlev) {
        L.src.clear();
        L.msg_only = !L.tgt.empty();
        for (auto& t : L.tgt) {
            if (t.reset_n > 0) t.reset_list = T.d_resets + (uintptr_t)t.reset_list;
            L.msg_only = L.msg_only && t.mode == EPI_MSG && t.hgrid != nullptr;
        }
        for (size_t j = 0; j < L.tgt.size(); ++j) {
            flat_of[L.node[j]] = (int)all.size();
            node_of.push_back(L.node[j]);
            all.push_back(L.tgt[j]);
        }
    }
    if (all.size() > T.wtask_cap) return MOT_EUNSUPPORTED;
    if (T.persist) {
        // claim order of the persistent kernel: the start order of a greedy schedule simulated on
        // its clusters, each free cluster taking the ready product with the longest remaining
        // chain of dependent work.  Products are weighted by their measured cost (a message
        // product 1; a scaling update 1.1; a check product 1.25; the root updates, which have no
        // kernel sum, 0.4).  Start times follow finish times of predecessors, so the order is
        // topological.
        const int n = (int)all.size();
        std::vector<double> wgt(n);
        for (int i = 0; i < n; ++i) {
            const int u = node_of[i];
            if (u >= S * W) wgt[i] = u == S * W ? 0.4 : 1.25;       // check products
            else if (u % W == 0) wgt[i] = 0.4;                       // R(s)
            else if (u % W < K) wgt[i] = 1.1;                        // F_k(s)
            else wgt[i] = 1.0;                                       // B_k(s)
        }
        std::vector<std::vector<int>> ps(n), sc(n);
        for (int i = 0; i < n; ++i)
            for (int u : pred[node_of[i]]) {
                const int j = flat_of[u];
                if (j < 0 || j >= i) return MOT_EUNSUPPORTED;        // (never: launch order is topological)
                ps[i].push_back(j);
                sc[j].push_back(i);
            }
        std::vector<double> tail(n, 0.0), fin(n, 0.0), start(n, 0.0), ready_t(n, 0.0);
        for (int i = n - 1; i >= 0; --i) {
            double m = 0.0;
            for (int v : sc[i]) m = std::max(m, tail[v]);
            tail[i] = wgt[i] + m;
        }
        std::vector<int> pending(n), ready;
        for (int i = 0; i < n; ++i) {
            pending[i] = (int)ps[i].size();
            if (pending[i] == 0) ready.push_back(i);
        }
        std::vector<double> cf(std::max(1, T.wave_clusters), 0.0);
        for (int placed = 0; placed < n; ++placed) {
            const int c = (int)(std::min_element(cf.begin(), cf.end()) - cf.begin());
            double t = cf[c], tmin = 1e300;
            for (int v : ready) tmin = std::min(tmin, ready_t[v]);
            if (ready.empty()) return MOT_EUNSUPPORTED;                // (never: acyclic)
            t = std::max(t, tmin);
            int best = -1;
            for (int v : ready)
                if (ready_t[v] <= t && (best < 0 || tail[v] > tail[best] || (tail[v] == tail[best] && v < best))) best = v;
            start[best] = t;
            fin[best] = t + wgt[best];
            cf[c] = fin[best];
            ready.erase(std::find(ready.begin(), ready.end(), best));
            for (int v : sc[best])
                if (--pending[v] == 0) {
                    double rt = 0.0;
                    for (int u : ps[v]) rt = std::max(rt, fin[u]);
                    ready_t[v] = rt;
                    ready.push_back(v);
                }
        }
        std::vector<int> perm(n);
        for (int i = 0; i < n; ++i) perm[i] = i;
        std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return start[a] < start[b]; });
        std::vector<Task> all2(n);
        std::vector<int> node2(n);
        for (int i = 0; i < n; ++i) {
            all2[i] = all[perm[i]];
            node2[i] = node_of[perm[i]];
            flat_of[node2[i]] = i;
        }
        all.swap(all2);
        node_of.swap(node2);
    }
    // dependency lists of the persistent kernel: the products each one waits for (all earlier in
    // the array, which is in a topological order)
    std::vector<int> deps;
    for (size_t i = 0; i < all.size(); ++i) {
        all[i].dep0 = (int)deps.size();
        for (int u : pred[node_of[i]]) {
            const int j = flat_of[u];
            if (j < 0 || j >= (int)i) return MOT_EUNSUPPORTED;   // (never: the order is topological)
            deps.push_back(j);
        }
        all[i].ndep = (int)deps.size() - all[i].dep0;
    }
    if (deps.size() > T.deps_cap) return MOT_EUNSUPPORTED;
    if (!deps.empty()) CK(cudaMemcpyAsync(T.d_deps, deps.data(), sizeof(int) * deps.size(), cudaMemcpyHostToDevice, st));
    T.wave_ntask = (int)all.size();
    CK(cudaMemcpyAsync(T.d_fac + T.fac_base, T.fac.data() + T.fac_base, sizeof(Factor) * (T.fac.size() - T.fac_base),
                       cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(T.d_resets + T.res_base, T.resets.data() + T.res_base,
                       sizeof(VecScale*) * (T.resets.size() - T.res_base), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(T.d_wtasks, all.data(), sizeof(Task) * all.size(), cudaMemcpyHostToDevice, st));
    size_t o = 0;
    for (auto& L : T.wlev) {
        L.d_src = nullptr;
        L.d_tgt = T.d_wtasks + o;
        o += L.tgt.size();
    }
    T.wave_S = S;
    T.wave_q0 = q0;
    T.wave_chk = with_check;
    return MOT_OK;
}

// ---- launching --------------------------------------------------------------------------
// Per-launch device timing (options.timing): an event pair around every launch.  Sweep chunks are
// captured into a graph together with their events (event-record nodes), so the timestamps come
// from the GPU's own back-to-back execution and not from the host's launch rate.
struct Timer {
    bool on = false;
    cudaStream_t st = nullptr;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev;
    std::vector<cudaEvent_t> pool;
    size_t next = 0;
    std::vector<cudaGraphExec_t> execs;   // timed graphs, kept until the events are read
    int reserve(size_t n) {               // create events ahead of a capture
        while (pool.size() < next + n) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e));
            pool.push_back(e);
        }
        return 0;
    }
    int take(cudaEvent_t* e) {
        RET(reserve(1));
        *e = pool[next++];
        return 0;
    }
    int begin(int cls, cudaEvent_t* a) {
        if (!on) return 0;
        cudaEvent_t e0, e1;
        RET(take(&e0));
        RET(take(&e1));
        RET(record(e0));
        ev.push_back({cls, {e0, e1}});
        *a = e1;
        return 0;
    }
    int end(cudaEvent_t e1) {
        if (!on) return 0;
        return record(e1);
    }
    // inside a capture an external record becomes an event-record node of the graph (timable);
    // outside one the plain record is used (the external flag is valid during capture only)
    int record(cudaEvent_t e) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        CK(cudaStreamIsCapturing(st, &cs));
        if (cs == cudaStreamCaptureStatusActive)
            CK(cudaEventRecordWithFlags(e, st, cudaEventRecordExternal));
        else
            CK(cudaEventRecord(e, st));
        return 0;
    }
    int collect(mot_result* r) {
        if (!on) return 0;
        CK(cudaStreamSynchronize(st));
        for (auto& x : ev) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, x.second.first, x.second.second));
            if (r) {
                r->kernel_ms[x.first] += ms;
                r->kernel_launches[x.first] += 1;
            }
        }
        ev.clear();
        for (auto g : execs) cudaGraphExecDestroy(g);
        execs.clear();
        for (auto e : pool) cudaEventDestroy(e);
        pool.clear();
        next = 0;
        return 0;
    }
    // Capture `count` sweeps of `body` with their events into a graph and launch it.
    template <class Body>
    int timed_graph(int count, size_t events_per_sweep, Body body) {
        RET(reserve(events_per_sweep * (size_t)count));
        cudaGraph_t graph;
        CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        long long dummy = 0;
        int rc = MOT_OK;
        for (int i = 0; i < count && rc == MOT_OK; ++i) rc = body(dummy);
        cudaError_t ce = cudaStreamEndCapture(st, &graph);
        if (rc != MOT_OK) return rc;
        CK(ce);
        cudaGraphExec_t ex = nullptr;
        cudaError_t ie = cudaGraphInstantiate(&ex, graph, 0);
        cudaGraphDestroy(graph);
        CK(ie);
        execs.push_back(ex);
        CK(cudaGraphLaunch(ex, st));
        return MOT_OK;
    }
};

int run_level(TreePlan& T, Level& L, cudaStream_t st, Timer& tm, long long& nl) {
    cudaEvent_t e = nullptr;
    if (T.path == MOT_PATH_NFFT && T.fused) {
        RET(tm.begin(MOT_K_FUSED, &e));
        if (T.ndft)
            CK(launch_ndft2d(L.d_tgt, (int)L.tgt.size(), T.G, st, L.msg_only));
        else
            CK(launch_fused2d(L.d_tgt, (int)L.tgt.size(), T.G, st, L.msg_only));
        RET(tm.end(e));
        nl += 1;
    } else if (T.path == MOT_PATH_NFFT) {
        if (!L.src.empty()) {
            RET(tm.begin(MOT_K_SPREAD, &e));
            CK(launch_spread(T.d, L.d_src, (int)L.src.size(), L.grid_src, T.G, st));
            RET(tm.end(e));
            int nf = 0;
            RET(tm.begin(MOT_K_FFTCONV, &e));
            CK(launch_fftconv(T.d, L.d_src, (int)L.src.size(), T.G, st, &nf));
            RET(tm.end(e));
            nl += 1 + nf;
        }
        RET(tm.begin(MOT_K_GATHER, &e));
        CK(launch_gather(T.d, L.d_tgt, (int)L.tgt.size(), L.grid_tgt, T.G, st));
        RET(tm.end(e));
        nl += 1;
    } else {
        if (!L.src.empty()) {
            RET(tm.begin(MOT_K_DENSE, &e));
            CK(launch_dense(T.d, L.d_src, (int)L.src.size(), L.ntb, L.nsplit, T.G, st));
            RET(tm.end(e));
            nl += 1;
        }
        RET(tm.begin(MOT_K_NODE, &e));
        CK(launch_epi(T.d, L.d_tgt, (int)L.tgt.size(), L.grid_tgt, T.G, st));
        RET(tm.end(e));
        nl += 1;
    }
    return MOT_OK;
}

int run_iteration(TreePlan& T, cudaStream_t st, Timer& tm, long long& nl) {
    cudaEvent_t e = nullptr;
    RET(tm.begin(MOT_K_NODE, &e));
    CK(launch_prologue(T.d_resets + T.it_reset0, (int)T.it_reset_n, 1, 1, nullptr, 0, T.G, st));
    RET(tm.end(e));
    nl += 1;
    for (auto& L : T.fwd) RET(run_level(T, L, st, tm, nl));
    for (auto& L : T.bwd) RET(run_level(T, L, st, tm, nl));
    return MOT_OK;
}

int run_check(TreePlan& T, cudaStream_t st, Timer& tm, long long& nl) {
    cudaEvent_t e = nullptr;
    RET(tm.begin(MOT_K_NODE, &e));
    CK(launch_prologue(T.d_resets + T.ck_reset0, (int)T.ck_reset_n, 0, 0, T.acc_node, 3 * T.K, T.G, st));
    RET(tm.end(e));
    nl += 1;
    for (auto& L : (T.par ? T.chk1 : T.chk)) RET(run_level(T, L, st, tm, nl));
    return MOT_OK;
}

// One wavefront chunk of S sweeps: prologue (the root's scale of the last iterate kept, the sweep
// counter advanced by S, their accumulator slots cleared), then the chunk's launches.
int run_wave(TreePlan& T, int S, cudaStream_t st, Timer& tm, long long& nl) {
    cudaEvent_t e = nullptr;
    RET(tm.begin(MOT_K_NODE, &e));
    // the exact-sum persistent kernel counts completed CTAs per product: its flags start at zero
    const bool counts = T.persist && T.ndft;
    CK(launch_prologue(T.d_resets + T.wave_root_reset, 1, 1, S, nullptr, 0, T.G, st, T.persist ? T.d_ctl : nullptr,
                       counts ? T.d_flags : nullptr, counts ? T.wave_ntask : 0));
    RET(tm.end(e));
    nl += 1;
    if (T.persist) {
        WaveArgs A;
        A.tasks = T.d_wtasks;
        A.ntask = T.wave_ntask;
        A.deps = T.d_deps;
        A.flags = T.d_flags;
        A.ctl = T.d_ctl;
        A.err = T.err;
        A.wait_ns = 1000000000ull;            // 1 s per wait (a chunk takes about a millisecond)
        RET(tm.begin(MOT_K_WAVE, &e));
        if (T.ndft)
            CK(launch_wave_nd(A, T.wave_clusters, T.G, st));
        else
            CK(launch_wave2d(A, T.wave_clusters, T.G, st));
        RET(tm.end(e));
        nl += 1;
        return MOT_OK;
    }
    for (auto& L : T.wlev) RET(run_level(T, L, st, tm, nl));
    return MOT_OK;
}

// One chunk with the schedule in T.wlev (built for this length and starting copy).
int run_wave_chunk(TreePlan& T, int count, cudaStream_t st, Timer& tm, long long& nl, bool graphs) {
    if (graphs && tm.on && st != nullptr) {
        long long per = 0;
        RET(tm.timed_graph(1, 2 * (T.wlev.size() + 2), [&](long long& d) {
            const long long before = d;
            const int rc = run_wave(T, count, st, tm, d);
            per = d - before;
            return rc;
        }));
        nl += per;
    } else if (graphs && st != nullptr) {
        if (T.gexec == nullptr || T.graph_iters != count || T.graph_par != T.par) {
            if (T.gexec) {
                cudaGraphExecDestroy(T.gexec);
                T.gexec = nullptr;
            }
            cudaGraph_t graph;
            CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            long long d = 0;
            const int rc = run_wave(T, count, st, tm, d);
            cudaError_t ce = cudaStreamEndCapture(st, &graph);
            if (rc != MOT_OK) return rc;
            CK(ce);
            CK(cudaGraphInstantiate(&T.gexec, graph, 0));
            cudaGraphDestroy(graph);
            T.graph_iters = count;
            T.graph_par = T.par;
            T.launches_per_chunk = d;
        }
        CK(cudaGraphLaunch(T.gexec, st));
        nl += T.launches_per_chunk;
    } else {
        RET(run_wave(T, count, st, tm, nl));
    }
    T.par = (T.par + count) & 1;
    return MOT_OK;
}

int run_iterations(TreePlan& T, int count, cudaStream_t st, Timer& tm, long long& nl, bool graphs) {
    if (count <= 0) return MOT_OK;
    if (T.wave) {
        // chunks longer than kWaveMax run as equal parts (the parts reuse one schedule)
        const int parts = (count + kWaveMax - 1) / kWaveMax;
        for (int i = 0; i < parts; ++i) {
            const int c = count / parts + (i < count % parts ? 1 : 0);
            const bool chk = T.persist && i == parts - 1;   // the persistent launch ends with the check
            if (T.wave_S != c || T.wave_q0 != T.par || T.wave_chk != chk) {
                const int rc = build_wave(T, c, T.par, chk, st);
                if (rc != MOT_OK) {
                    // no valid wavefront (never expected): sweep by sweep, which reads the first
                    // beta copy, so only from a point where that copy is the latest
                    if (rc != MOT_EUNSUPPORTED || T.par != 0) return rc;
                    T.wave = false;
                    return run_iterations(T, count - (count / parts) * i - std::min(i, count % parts), st, tm, nl,
                                          graphs);
                }
                if (T.gexec) {
                    cudaGraphExecDestroy(T.gexec);
                    T.gexec = nullptr;
                }
            }
            RET(run_wave_chunk(T, c, st, tm, nl, graphs));
            if (chk) T.check_done = true;
        }
        return MOT_OK;
    }
    if (graphs && tm.on && st != nullptr) {
        long long per = 0;
        RET(tm.timed_graph(count, 2 * (size_t)(4 * T.K + 8), [&](long long& d) {
            const long long before = d;
            const int rc = run_iteration(T, st, tm, d);
            per = d - before;
            return rc;
        }));
        nl += per * count;
        return MOT_OK;
    }
    if (graphs && !tm.on && st != nullptr) {
        if (T.gexec == nullptr || T.graph_iters != count || T.graph_par != -1) {
            if (T.gexec) {
                cudaGraphExecDestroy(T.gexec);
                T.gexec = nullptr;
            }
            T.graph_par = -1;
            cudaGraph_t graph;
            CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            long long dummy = 0;
            int rc = MOT_OK;
            for (int i = 0; i < count && rc == MOT_OK; ++i) rc = run_iteration(T, st, tm, dummy);
            cudaError_t ce = cudaStreamEndCapture(st, &graph);
            if (rc != MOT_OK) return rc;
            CK(ce);
            CK(cudaGraphInstantiate(&T.gexec, graph, 0));
            cudaGraphDestroy(graph);
            T.graph_iters = count;
            T.launches_per_iter = dummy / count;
        }
        CK(cudaGraphLaunch(T.gexec, st));
        nl += T.launches_per_iter * count;
        return MOT_OK;
    }
    for (int i = 0; i < count; ++i) RET(run_iteration(T, st, tm, nl));
    return MOT_OK;
}

struct Stats {
    std::vector<char> buf;
    const IterAcc* acc() const { return reinterpret_cast<const IterAcc*>(buf.data()); }
    const double* node(int K) const { (void)K; return reinterpret_cast<const double*>(buf.data() + sizeof(IterAcc) * kRing); }
    const VecScale* sc(int K) const {
        return reinterpret_cast<const VecScale*>(buf.data() + sizeof(IterAcc) * kRing + sizeof(double) * 3 * K);
    }
    int err() const { return *reinterpret_cast<const int*>(buf.data() + buf.size() - 16); }
};

int read_stats(TreePlan& T, Stats& S, cudaStream_t st) {
    S.buf.resize(T.stats_bytes);
    CK(cudaMemcpyAsync(S.buf.data(), T.stats_begin, T.stats_bytes, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return MOT_OK;
}

int tree_plan_setup(const mot_problem* P, const mot_options& o, TreePlan& T, void* ws, size_t ws_bytes,
                    bool measure_only, size_t* need, cudaStream_t st) {
    RET(tree_structure(P, T));
    T.d = P->d;
    T.eta = P->eta;
    T.path = o.path;
    T.o = o;
    if (T.path != MOT_PATH_NFFT && T.path != MOT_PATH_DENSE) return MOT_EUNSUPPORTED;
    // eta_e = eta / w_e
    double emin = 1e300, emax = 0.0;
    for (int k = 1; k < T.K; ++k) {
        double e = T.eta / T.w[k];
        emin = std::min(emin, e);
        emax = std::max(emax, e);
    }
    if (measure_only) {
        // the grid size depends on the data radius only through the choice of n; lay out for
        // the largest grid the options allow
        T.g = GridChoice();
        if (o.n_grid > 0) {
            T.g.n = o.n_grid;
        } else {
            T.g.n = max_grid(T.d);
        }
        T.g.M = T.g.n / 4;
        Arena A;
        A.measure = true;
        layout_tree(A, T);
        *need = A.off + 256;
        return MOT_OK;
    }
    // lay out with the largest grid first (matches the workspace query), then choose
    GridChoice gmax;
    gmax.n = o.n_grid > 0 ? o.n_grid : max_grid(T.d);
    gmax.M = gmax.n / 4;
    T.g = gmax;
    Arena A;
    A.measure = false;
    A.base = reinterpret_cast<char*>(ws);
    A.cap = ws_bytes;
    layout_tree(A, T);
    if (A.off > ws_bytes) return MOT_ENOMEM;
    // measure the data and choose the grid (<= the laid-out maximum)
    std::vector<PrepSet> sets;
    for (int k = 0; k < T.K; ++k) sets.push_back(prepset_of(T.sets[k], P->x[T.order[k]], P->mu[T.order[k]]));
    GridChoice g;
    RET(measure_and_choose(sets, T.d_sets, T.box_scratch, T.box_out, T.d, emin, emax, o, g, st));
    if (g.n > gmax.n) g.n = gmax.n;
    g.M = g.n / 4;
    T.g = g;
    // prep: normalise, bin, sort
    CK(cudaMemsetAsync(T.stats_begin, 0, T.stats_bytes, st));
    {
        // rebuild the set descriptors for the chosen grid (tile counts depend on n)
        std::vector<PrepSet> s2;
        for (int k = 0; k < T.K; ++k) {
            T.sets[k].maxsub = (T.n[k] + mot_sub_points(T.d) - 1) / mot_sub_points(T.d) + mot_ntiles(T.d, g.n);
            s2.push_back(prepset_of(T.sets[k], P->x[T.order[k]], P->mu[T.order[k]]));
        }
        CK(cudaMemcpyAsync(T.d_sets, s2.data(), sizeof(PrepSet) * s2.size(), cudaMemcpyHostToDevice, st));
        CK(launch_prep(T.d_sets, s2.data(), T.K, T.d, g.n, g.c, g.s, T.err, st));
    }
    // spectral multipliers per edge, grids zeroed
    if (T.path == MOT_PATH_NFFT) {
        CK(prepare_window());
        CK(prepare_fftconv(T.d, g.n));
        CK(prepare_fused2d());
        // one 16-CTA cluster per product: worth it while a product is small enough that the
        // kernel's fixed phases dominate; larger sets use the whole GPU through the 3-kernel path
        int nmax = 0;
        for (int k = 0; k < T.K; ++k) nmax = std::max(nmax, T.n[k]);
        T.fused = fused2d_supported(T.d, g.n) && nmax <= fused2d_max_points();
        T.ndft = false;
        if (T.fused && o.ndft > 0) {
            CK(prepare_ndft2d());
            T.ndft = ndft2d_supported(T.d, g.M);
        }
        bool any_free = false;
        for (int k = 0; k < T.K; ++k) any_free = any_free || T.free_[k];
        T.wave = T.fused && !any_free && o.wavefront > 0;
        T.wave_clusters = g_wave_clusters_override.load() > 0
                              ? g_wave_clusters_override.load()
                              : (T.ndft ? ndft2d_wave_max_active_clusters() : wave2d_max_active_clusters());
        T.persist = T.wave && o.wavefront == 1 && T.wave_clusters > 0;
        if (T.wave) {
            CK(cudaMemsetAsync(T.d_flags, 0, sizeof(int) * T.wtask_cap, st));
            CK(cudaMemsetAsync(T.d_ctl, 0, sizeof(WaveCtl), st));
        }
        size_t gsz = 1;
        for (int t = 0; t < T.d; ++t) gsz *= g.n;
        for (int k = 1; k < T.K; ++k) {
            // edges with the same weight share one multiplier
            int same = -1;
            for (int q = 1; q < k && same < 0; ++q)
                if (T.w[q] == T.w[k]) same = q;
            if (same > 0) {
                T.D[k] = T.D[same];
            } else {
                double eta_n = (T.eta / T.w[k]) / (g.s * g.s);
                RET(make_D_for(eta_n, g, T.d, o, T.dscr_a, T.dscr_b, T.D[k], st, !T.ndft));
            }
            CK(cudaMemsetAsync(T.grid[k], 0, gsz * sizeof(float), st));
        }
    } else {
        for (int k = 1; k < T.K; ++k) {
            CK(cudaMemsetAsync(T.rawf[k], 0, sizeof(float) * T.n[k], st));
            CK(cudaMemsetAsync(T.rawb[k], 0, sizeof(float) * T.n[T.parent[k]], st));
            CK(cudaMemsetAsync(T.rawc[k], 0, sizeof(float) * T.n[k], st));
        }
    }
    build_tasks(T);
    RET(upload_tasks(T, st));
    return MOT_OK;
}



// =============================================================================================
// circle plan (Algorithm 3)
// =============================================================================================
//
// Nodes 0..K-1 with edges {k, k+1 mod K} (edge k).  beta_k (k = 1..K-1) and Gam_k = gamma_k^T
// (k = 1..K-1) are n_k x n_0 matrices stored column by column (column c = point c of node 0).
// beta_{K-1} = K^{(K-1,0)} and Gam_1 = K^{(1,0)} are fixed dense kernel matrices; the others are
// batches of kernel matrix-vector products, one per column:
//   Gam_k[c]  = K^{(k,k-1)} (phi^{k-1} (.) Gam_{k-1}[c]),  k = 2..K-1   (forward)
//   beta_k[c] = K^{(k,k+1)} (phi^{k+1} (.) beta_{k+1}[c]), k = K-2..1   (backward)
// phi^0_c = mu^0_c / sum_j Gam_1[c][j] phi^1_j beta_1[c][j]  (column sums)
// phi^k_i = mu^k_i / sum_c beta_k[c][i] phi^0_c Gam_k[c][i]   (row dots), k = 1..K-1.
struct CBatch {
    int s = 0, t = 0, edge = 0;
    std::vector<Task> tasks;
    Task* d_tasks = nullptr;
    VecScale* out_sc = nullptr;
    int grid_src = 1, grid_tgt = 1, ntb = 1, nsplit = 1;
    // tensor-core path: Y = X' K^T with X' = split(phi^s (.) X), K = kernel matrix (n_t x n_s)
    float* X = nullptr;
    VecScale* sX = nullptr;
    float* Y = nullptr;
    uint16_t* kt_hi = nullptr;
    uint16_t* kt_lo = nullptr;
    TcGemm tc;
};

struct CirclePlan {
    int K = 0, d = 0, path = MOT_PATH_NFFT, n0 = 0, CB = 1;
    double eta = 0.0;
    std::vector<double> w;          // edge weights, edge k = {k, k+1 mod K}
    std::vector<int> n;
    GridChoice g;
    mot_options o;
    std::vector<SetBufs> sets;
    std::vector<float*> phi, beta, gam, raw, D;
    std::vector<float*> grid, hgrid, rawm;   // per column slot of a chunk
    std::vector<float2*> spec;
    VecScale* sc = nullptr;         // [4K]: phi, beta, gam, raw
    IterAcc* acc = nullptr;
    int* iter = nullptr;
    double* acc_node = nullptr;
    int* err = nullptr;
    Factor* d_fac = nullptr;
    size_t fac_cap = 0;
    VecScale** d_resets = nullptr;
    Task* d_tasks = nullptr;
    size_t task_cap = 0;
    PrepSet* d_sets = nullptr;
    float* box_scratch = nullptr;
    float* box_out = nullptr;
    double* dscr_a = nullptr;
    double* dscr_b = nullptr;
    char* stats_begin = nullptr;
    size_t stats_bytes = 0;
    std::vector<Factor> fac;
    std::vector<VecScale*> resets;
    size_t it_r0 = 0, it_rn = 0, bw_r0 = 0, bw_rn = 0, ck_r0 = 0, ck_rn = 0;
    std::vector<CBatch> fwd, bwd;   // fwd[k] produces Gam_k (k >= 2); bwd[k] produces beta_k (k <= K-2)
    bool c1 = false;                // 1-D batched fast summation (k_c1_*) for the batches
    std::vector<int*> c1_l0;        // per node: base cell of each point's window
    std::vector<float*> c1_w;       // per node: window taps [n_k][10]
    std::vector<float*> c1_c;       // per edge: circulant of D (n floats)
    float* c1_G = nullptr;          // n0 x n spread grids of one batch
    bool has_close = false;         // closing edge against sigma(x^0) (Section 6.3)
    float* u_close = nullptr;       // [d][n0] sigma(x^0) in node 0's sorted order, grid units
    uint16_t* a_hi = nullptr;       // tensor-core path: split source matrix, n0 x ld (BF16 pairs)
    uint16_t* a_lo = nullptr;
    std::vector<uint16_t*> ktf_hi, ktf_lo, ktb_hi, ktb_lo;   // split kernel matrices per batch
    std::vector<Task> node_tasks;   // [0] root update, [1..K-1] phi^k updates, [K..2K-1] check marginals
    Task* d_node = nullptr;
    Globals G;
    cudaGraphExec_t gexec = nullptr;
    int graph_iters = 0;
    long long launches_per_iter = 0;

    VecScale* phi_sc(int k) const { return sc + k; }
    VecScale* beta_sc(int k) const { return sc + K + k; }
    VecScale* gam_sc(int k) const { return sc + 2 * K + k; }
    VecScale* raw_sc(int k) const { return sc + 3 * K + k; }
};

void layout_circle(Arena& A, CirclePlan& C) {
    const int K = C.K, d = C.d, ng = C.g.n, M = C.g.M;
    const bool nfft = C.path == MOT_PATH_NFFT;
    const bool tc = C.path == MOT_PATH_DENSE_BF16X3;
    size_t gsz = 1;
    for (int t = 0; t < d; ++t) gsz *= ng;
    int nmax = 0, ldmax = 0;
    for (int k = 0; k < K; ++k) {
        nmax = std::max(nmax, C.n[k]);
        ldmax = std::max(ldmax, tc_ld(C.n[k]));
    }
    C.sets.assign(K, SetBufs());
    for (int k = 0; k < K; ++k) layout_set(A, C.sets[k], C.n[k], d, ng, true);
    C.phi.assign(K, nullptr);
    C.raw.assign(K, nullptr);
    C.beta.assign(K, nullptr);
    C.gam.assign(K, nullptr);
    C.D.assign(K, nullptr);
    for (int k = 0; k < K; ++k) {
        C.phi[k] = A.take<float>(C.n[k]);
        C.raw[k] = A.take<float>(C.n[k]);
    }
    for (int k = 1; k < K; ++k) {
        C.beta[k] = A.take<float>((size_t)C.n[k] * C.n0);
        C.gam[k] = A.take<float>((size_t)C.n[k] * C.n0);
    }
    C.grid.assign(C.CB, nullptr);
    C.hgrid.assign(C.CB, nullptr);
    C.spec.assign(C.CB, nullptr);
    C.rawm.assign(C.CB, nullptr);
    for (int c = 0; c < C.CB; ++c) {
        if (nfft) {
            C.grid[c] = A.take<float>(gsz);
            C.hgrid[c] = A.take<float>(gsz);
            if (d == 3) C.spec[c] = A.take<float2>((size_t)ng * (2 * M + 1) * (M + 1));
        } else if (!tc) {
            C.rawm[c] = A.take<float>(nmax);
        }
    }
    C.c1_l0.assign(K, nullptr);
    C.c1_w.assign(K, nullptr);
    C.c1_c.assign(K, nullptr);
    if (nfft && d == 1) {
        for (int k = 0; k < K; ++k) {
            C.c1_l0[k] = A.take<int>(C.n[k]);
            C.c1_w[k] = A.take<float>((size_t)C.n[k] * MOT_W);
            C.c1_c[k] = A.take<float>(128);
        }
        C.c1_G = A.take<float>((size_t)C.n0 * 128);
    }
    C.ktf_hi.assign(K, nullptr);
    C.ktf_lo.assign(K, nullptr);
    C.ktb_hi.assign(K, nullptr);
    C.ktb_lo.assign(K, nullptr);
    if (tc) {
        C.a_hi = A.take<uint16_t>((size_t)C.n0 * ldmax);
        C.a_lo = A.take<uint16_t>((size_t)C.n0 * ldmax);
        for (int k = 2; k < K; ++k) {       // Gam_k from Gam_{k-1}: n_k x n_{k-1}
            C.ktf_hi[k] = A.take<uint16_t>((size_t)C.n[k] * tc_ld(C.n[k - 1]));
            C.ktf_lo[k] = A.take<uint16_t>((size_t)C.n[k] * tc_ld(C.n[k - 1]));
        }
        for (int k = 1; k <= K - 2; ++k) {  // beta_k from beta_{k+1}: n_k x n_{k+1}
            C.ktb_hi[k] = A.take<uint16_t>((size_t)C.n[k] * tc_ld(C.n[k + 1]));
            C.ktb_lo[k] = A.take<uint16_t>((size_t)C.n[k] * tc_ld(C.n[k + 1]));
        }
    }
    if (nfft)
        for (int k = 0; k < K; ++k) C.D[k] = A.take<float>(D_floats(d, M));
    size_t stats = sizeof(IterAcc) * kRing + sizeof(double) * 3 * K + sizeof(VecScale) * 4 * K + 16;
    C.stats_begin = A.take<char>(stats);
    C.stats_bytes = stats;
    if (!A.measure) {
        C.acc = reinterpret_cast<IterAcc*>(C.stats_begin);
        C.acc_node = reinterpret_cast<double*>(C.stats_begin + sizeof(IterAcc) * kRing);
        C.sc = reinterpret_cast<VecScale*>(C.stats_begin + sizeof(IterAcc) * kRing + sizeof(double) * 3 * K);
        C.err = reinterpret_cast<int*>(C.stats_begin + stats - 16);
        C.iter = C.err + 1;
    }
    if (C.has_close) C.u_close = A.take<float>((size_t)d * C.n0);
    C.d_sets = A.take<PrepSet>(K);
    C.box_scratch = A.take<float>(8);
    C.box_out = A.take<float>(8);
    if (nfft) {
        size_t sd = make_D_scratch_doubles(d, M);
        C.dscr_a = A.take<double>(sd);
        C.dscr_b = A.take<double>(sd);
    }
    C.fac_cap = (size_t)4 * K * C.n0 + 16 * (size_t)K + 64;
    C.d_fac = A.take<Factor>(C.fac_cap);
    C.d_resets = A.take<VecScale*>(8 * (size_t)K + 8);
    C.task_cap = (size_t)2 * K * C.n0 + 4 * (size_t)K + 8;
    C.d_tasks = A.take<Task>(C.task_cap);
}

int c_add_factor(CirclePlan& C, const float* mant, const VecScale* sc) {
    Factor f;
    f.mant = mant;
    f.sc = sc;
    f.inv = 0;
    f.use_prev = 0;
    C.fac.push_back(f);
    return (int)C.fac.size() - 1;
}

// Batch of column products: Y = K^{(t,s)} (phi^s (.) X), X = mats[s] (n_s x n0), Y = mats[t].
void c_build_batch(CirclePlan& C, CBatch& B, int s, int t, int edge, float* X, VecScale* sX, float* Y, VecScale* sY) {
    B.s = s;
    B.t = t;
    B.edge = edge;
    B.out_sc = sY;
    B.X = X;
    B.sX = sX;
    B.Y = Y;
    B.tasks.clear();
    const double eta_n = (C.eta / C.w[edge]) / (C.g.s * C.g.s);
    for (int c = 0; c < C.n0; ++c) {
        Task tk = blank_task();
        tk.src = pointset_of(C.sets[s]);
        tk.sf0 = (int)C.fac.size();
        c_add_factor(C, C.phi[s], C.phi_sc(s));
        c_add_factor(C, X + (size_t)c * C.n[s], sX);
        tk.snf = 2;
        const int slot = c % C.CB;
        tk.grid = C.grid[slot];
        tk.hgrid = C.hgrid[slot];
        tk.spec = C.spec[slot];
        tk.D = C.D[edge];
        tk.raw = C.rawm[slot];
        tk.eta_u = (float)(eta_n * (double)C.g.n * (double)C.g.n);
        tk.tgt = pointset_of(C.sets[t]);
        tk.mode = EPI_MSG;
        tk.out = Y + (size_t)c * C.n[t];
        tk.out_sc = sY;
        B.tasks.push_back(tk);
    }
    int ms = 1, mt = 1;
    ms = std::max(ms, C.sets[s].maxsub);
    mt = std::max(mt, C.sets[t].maxsub);
    B.grid_src = std::min(ms, 1024);
    B.grid_tgt = C.path == MOT_PATH_NFFT ? std::min(mt, 1024) : std::min((C.n[t] + 255) / 256, 1024);
    B.ntb = (C.n[t] + 511) / 512;
    B.nsplit = std::max(1, std::min(64, 4 * 152 / std::max(1, B.ntb * std::min(C.CB, C.n0))));
}

void c_build(CirclePlan& C) {
    const int K = C.K;
    C.fac.clear();
    C.resets.clear();
    C.fwd.assign(K, CBatch());
    C.bwd.assign(K, CBatch());
    for (int k = 2; k < K; ++k)
        c_build_batch(C, C.fwd[k], k - 1, k, k - 1, C.gam[k - 1], C.gam_sc(k - 1), C.gam[k], C.gam_sc(k));
    for (int k = K - 2; k >= 1; --k)
        c_build_batch(C, C.bwd[k], k + 1, k, k, C.beta[k + 1], C.beta_sc(k + 1), C.beta[k], C.beta_sc(k));
    // node tasks (k_epi): raw = row dots / column sums
    C.node_tasks.assign(2 * K, blank_task());
    for (int k = 0; k < K; ++k) {
        for (int pass = 0; pass < 2; ++pass) {
            Task t = blank_task();
            t.tgt = pointset_of(C.sets[k]);
            t.raw = C.raw[k];
            t.sf0 = (int)C.fac.size();
            if (k == 0) {
                c_add_factor(C, C.gam[1], C.gam_sc(1));
                c_add_factor(C, C.phi[1], C.phi_sc(1));
                c_add_factor(C, C.beta[1], C.beta_sc(1));
            } else {
                c_add_factor(C, C.beta[k], C.beta_sc(k));
                c_add_factor(C, C.phi[0], C.phi_sc(0));
                // row dots formed in the batch (k >= 2 on the 1-D path) take Gam_k unnormalised:
                // its log-scale with a unit maximum
                c_add_factor(C, C.gam[k], (C.c1 && k >= 2) ? C.raw_sc(k) : C.gam_sc(k));
            }
            t.snf = 3;
            t.phi = C.phi[k];
            t.phi_sc = C.phi_sc(k);
            t.mu_f = C.sets[k].mu_f;
            t.mu_d = C.sets[k].mu_d;
            if (pass == 0) {
                t.mode = k == 0 ? EPI_CROOT : EPI_PHI;
                t.tf0 = (int)C.fac.size();
                t.tnf = 0;
            } else {
                t.mode = EPI_MARG;
                t.tf0 = (int)C.fac.size();
                c_add_factor(C, C.phi[k], C.phi_sc(k));
                t.tnf = 1;
                t.acc_node = C.acc_node + 3 * k;
            }
            C.node_tasks[pass * K + k] = t;
        }
    }
    C.it_r0 = C.resets.size();
    for (int k = 0; k < K; ++k) C.resets.push_back(C.phi_sc(k));
    for (int k = 2; k < K; ++k) C.resets.push_back(C.gam_sc(k));
    C.it_rn = C.resets.size() - C.it_r0;
    C.bw_r0 = C.resets.size();
    for (int k = 1; k <= K - 2; ++k) C.resets.push_back(C.beta_sc(k));
    C.bw_rn = C.resets.size() - C.bw_r0;
    C.ck_r0 = C.resets.size();
    for (int k = 2; k < K; ++k) C.resets.push_back(C.gam_sc(k));
    C.ck_rn = C.resets.size() - C.ck_r0;
}

int c_upload(CirclePlan& C, cudaStream_t st) {
    if (C.fac.size() > C.fac_cap) return MOT_EUNSUPPORTED;
    CK(cudaMemcpyAsync(C.d_fac, C.fac.data(), sizeof(Factor) * C.fac.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(C.d_resets, C.resets.data(), sizeof(VecScale*) * C.resets.size(), cudaMemcpyHostToDevice, st));
    size_t off = 0;
    std::vector<Task> all;
    for (auto* v : {&C.fwd, &C.bwd})
        for (auto& B : *v) {
            B.d_tasks = C.d_tasks + off;
            off += B.tasks.size();
            all.insert(all.end(), B.tasks.begin(), B.tasks.end());
        }
    C.d_node = C.d_tasks + off;
    all.insert(all.end(), C.node_tasks.begin(), C.node_tasks.end());
    if (all.size() > C.task_cap) return MOT_EUNSUPPORTED;
    CK(cudaMemcpyAsync(C.d_tasks, all.data(), sizeof(Task) * all.size(), cudaMemcpyHostToDevice, st));
    C.G.iter = C.iter;
    C.G.acc = C.acc;
    C.G.R = kRing;
    C.G.floor_ = 1e-30f;
    C.G.n_grid = C.g.n;
    C.G.M = C.g.M;
    C.G.fac = C.d_fac;
    return MOT_OK;
}

int c_run_batch_tc(CirclePlan& C, CBatch& B, cudaStream_t st, Timer& tm, long long& nl);

int c_run_batch(CirclePlan& C, CBatch& B, cudaStream_t st, Timer& tm, long long& nl) {
    if (C.path == MOT_PATH_DENSE_BF16X3) return c_run_batch_tc(C, B, st, tm, nl);
    cudaEvent_t e = nullptr;
    if (C.c1) {
        const int s = B.s, t = B.t;
        // a batch producing Gam_t (t >= 2) also forms the row dots of phi^t's update (c_node)
        const bool rows = t >= 2 && B.Y == C.gam[t];
        for (int stage = 0; stage < 2; ++stage) {
            RET(tm.begin(stage == 0 ? MOT_K_SPREAD : MOT_K_GATHER, &e));
            if (rows)
                CK(launch_c1_batch(B.X, B.sX, C.phi[s], C.phi_sc(s), C.c1_l0[s], C.c1_w[s], C.n[s], C.c1_l0[t],
                                   C.c1_w[t], C.n[t], C.n0, C.g.n, C.c1_c[B.edge], C.c1_G, B.Y, C.G.floor_,
                                   B.out_sc, st, stage, C.beta[t], C.beta_sc(t), C.phi[0], C.phi_sc(0), C.raw[t],
                                   C.raw_sc(t)));
            else
                CK(launch_c1_batch(B.X, B.sX, C.phi[s], C.phi_sc(s), C.c1_l0[s], C.c1_w[s], C.n[s], C.c1_l0[t],
                                   C.c1_w[t], C.n[t], C.n0, C.g.n, C.c1_c[B.edge], C.c1_G, B.Y, C.G.floor_,
                                   B.out_sc, st, stage));
            RET(tm.end(e));
        }
        nl += 3;                // memset, spread, gather
        return MOT_OK;
    }
    for (int c0 = 0; c0 < C.n0; c0 += C.CB) {
        const int cnt = std::min(C.CB, C.n0 - c0);
        const Task* tk = B.d_tasks + c0;
        if (C.path == MOT_PATH_NFFT) {
            RET(tm.begin(MOT_K_SPREAD, &e));
            CK(launch_spread(C.d, tk, cnt, B.grid_src, C.G, st));
            RET(tm.end(e));
            int nf = 0;
            RET(tm.begin(MOT_K_FFTCONV, &e));
            CK(launch_fftconv(C.d, tk, cnt, C.G, st, &nf));
            RET(tm.end(e));
            RET(tm.begin(MOT_K_GATHER, &e));
            CK(launch_gather(C.d, tk, cnt, B.grid_tgt, C.G, st));
            RET(tm.end(e));
            nl += 2 + nf;
        } else {
            RET(tm.begin(MOT_K_DENSE, &e));
            CK(launch_dense(C.d, tk, cnt, B.ntb, B.nsplit, C.G, st));
            RET(tm.end(e));
            RET(tm.begin(MOT_K_NODE, &e));
            CK(launch_epi(C.d, tk, cnt, B.grid_tgt, C.G, st));
            RET(tm.end(e));
            nl += 2;
        }
    }
    return MOT_OK;
}

// Tensor-core batch: the whole n_t x n0 message matrix as one split-BF16 product.
int c_run_batch_tc(CirclePlan& C, CBatch& B, cudaStream_t st, Timer& tm, long long& nl) {
    cudaEvent_t e = nullptr;
    RET(tm.begin(MOT_K_SPLIT, &e));
    CK(launch_split_src(B.X, B.sX, C.phi[B.s], C.phi_sc(B.s), C.n[B.s], C.n0, tc_ld(C.n[B.s]), C.a_hi, C.a_lo, st));
    RET(tm.end(e));
    TcEpi ep;
    std::memset(&ep, 0, sizeof(ep));
    ep.out = B.Y;
    ep.ldo = C.n[B.t];
    ep.mode = 1;
    ep.floor_ = C.G.floor_;
    ep.out_sc = B.out_sc;
    ep.s_a = C.phi_sc(B.s);
    ep.s_b = B.sX;
    ep.err = C.err;
    RET(tm.begin(MOT_K_TCGEMM, &e));
    CK(launch_tc_gemm(B.tc, ep, st));
    RET(tm.end(e));
    nl += 2;
    return MOT_OK;
}

int c_node(CirclePlan& C, int k, int pass, cudaStream_t st, Timer& tm, long long& nl) {
    cudaEvent_t e = nullptr;
    // on the 1-D path the row dots of k >= 2 were formed by the batch that produced Gam_k
    if (!(C.c1 && k >= 2)) {
        RET(tm.begin(MOT_K_CIRCLE, &e));
        if (k == 0)
            CK(launch_colsum(C.gam[1], C.gam_sc(1), C.beta[1], C.beta_sc(1), C.phi[1], C.phi_sc(1), C.n[1], C.n0,
                             C.raw[0], st));
        else
            CK(launch_rowdot(C.beta[k], C.beta_sc(k), C.gam[k], C.gam_sc(k), C.phi[0], C.phi_sc(0), C.n[k], C.n0,
                             C.raw[k], st));
        RET(tm.end(e));
        nl += 1;
    }
    RET(tm.begin(MOT_K_NODE, &e));
    CK(launch_epi(C.d, C.d_node + pass * C.K + k, 1, std::min((C.n[k] + 255) / 256, 1024), C.G, st));
    RET(tm.end(e));
    nl += 1;
    return MOT_OK;
}

int c_backward(CirclePlan& C, cudaStream_t st, Timer& tm, long long& nl) {
    for (int k = C.K - 2; k >= 1; --k) RET(c_run_batch(C, C.bwd[k], st, tm, nl));
    return MOT_OK;
}

int c_iteration(CirclePlan& C, cudaStream_t st, Timer& tm, long long& nl) {
    cudaEvent_t e = nullptr;
    RET(tm.begin(MOT_K_NODE, &e));
    CK(launch_prologue(C.d_resets + C.it_r0, (int)C.it_rn, 1, 1, nullptr, 0, C.G, st));
    RET(tm.end(e));
    nl += 1;
    RET(c_node(C, 0, 0, st, tm, nl));
    for (int k = 1; k < C.K; ++k) {
        if (k >= 2) RET(c_run_batch(C, C.fwd[k], st, tm, nl));
        RET(c_node(C, k, 0, st, tm, nl));
    }
    RET(tm.begin(MOT_K_NODE, &e));
    CK(launch_prologue(C.d_resets + C.bw_r0, (int)C.bw_rn, 0, 0, nullptr, 0, C.G, st));
    RET(tm.end(e));
    nl += 1;
    return c_backward(C, st, tm, nl);
}

int c_check(CirclePlan& C, cudaStream_t st, Timer& tm, long long& nl) {
    cudaEvent_t e = nullptr;
    RET(tm.begin(MOT_K_NODE, &e));
    CK(launch_prologue(C.d_resets + C.ck_r0, (int)C.ck_rn, 0, 0, C.acc_node, 3 * C.K, C.G, st));
    RET(tm.end(e));
    nl += 1;
    RET(c_node(C, 0, 1, st, tm, nl));
    for (int k = 1; k < C.K; ++k) {
        if (k >= 2) RET(c_run_batch(C, C.fwd[k], st, tm, nl));
        RET(c_node(C, k, 1, st, tm, nl));
    }
    return MOT_OK;
}

int c_run_iterations(CirclePlan& C, int count, cudaStream_t st, Timer& tm, long long& nl, bool graphs) {
    if (count <= 0) return MOT_OK;
    if (graphs && tm.on && st != nullptr) {
        long long per = 0;
        const size_t chunks = (size_t)((C.n0 + C.CB - 1) / C.CB);
        RET(tm.timed_graph(count, 2 * (size_t)(4 * C.K * (3 * chunks + 2) + 8), [&](long long& d) {
            const long long before = d;
            const int rc = c_iteration(C, st, tm, d);
            per = d - before;
            return rc;
        }));
        nl += per * count;
        return MOT_OK;
    }
    if (graphs && !tm.on && st != nullptr) {
        if (C.gexec == nullptr || C.graph_iters != count) {
            if (C.gexec) {
                cudaGraphExecDestroy(C.gexec);
                C.gexec = nullptr;
            }
            cudaGraph_t graph;
            CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            long long dummy = 0;
            int rc = MOT_OK;
            for (int i = 0; i < count && rc == MOT_OK; ++i) rc = c_iteration(C, st, tm, dummy);
            cudaError_t ce = cudaStreamEndCapture(st, &graph);
            if (rc != MOT_OK) return rc;
            CK(ce);
            CK(cudaGraphInstantiate(&C.gexec, graph, 0));
            cudaGraphDestroy(graph);
            C.graph_iters = count;
            C.launches_per_iter = dummy / count;
        }
        CK(cudaGraphLaunch(C.gexec, st));
        nl += C.launches_per_iter * count;
        return MOT_OK;
    }
    for (int i = 0; i < count; ++i) RET(c_iteration(C, st, tm, nl));
    return MOT_OK;
}

int circle_setup(const mot_problem* P, const mot_options& o, CirclePlan& C, void* ws, size_t ws_bytes, bool measure,
                 size_t* need, cudaStream_t st) {
    const int K = P->K;
    if (K < 3) return MOT_EUNSUPPORTED;
    if (P->free_nodes)
        for (int k = 0; k < K; ++k)
            if (P->free_nodes[k]) return MOT_EUNSUPPORTED;
    C.K = K;
    C.d = P->d;
    C.eta = P->eta;
    C.path = o.path;
    C.o = o;
    if (C.path != MOT_PATH_NFFT && C.path != MOT_PATH_DENSE && C.path != MOT_PATH_DENSE_BF16X3)
        return MOT_EUNSUPPORTED;
    C.n.resize(K);
    for (int k = 0; k < K; ++k) C.n[k] = (int)P->n[k];
    C.n0 = C.n[0];
    C.has_close = P->x_close != nullptr;
    C.w.assign(K, 1.0);
    if (P->edge_w)
        for (int k = 0; k < K; ++k) C.w[k] = P->edge_w[k];
    C.CB = C.d == 1 ? C.n0 : (C.d == 2 ? std::min(C.n0, 256) : std::min(C.n0, 16));
    GridChoice gmax;
    gmax.n = o.n_grid > 0 ? o.n_grid : max_grid(C.d);
    gmax.M = gmax.n / 4;
    C.g = gmax;
    Arena A;
    A.measure = measure;
    A.base = reinterpret_cast<char*>(ws);
    A.cap = ws_bytes;
    layout_circle(A, C);
    if (measure) {
        *need = A.off + 256;
        return MOT_OK;
    }
    if (A.off > ws_bytes) return MOT_ENOMEM;
    double emin = 1e300, emax = 0.0;
    for (int k = 0; k < K; ++k) {
        emin = std::min(emin, C.eta / C.w[k]);
        emax = std::max(emax, C.eta / C.w[k]);
    }
    std::vector<PrepSet> sets;
    for (int k = 0; k < K; ++k) sets.push_back(prepset_of(C.sets[k], P->x[k], P->mu[k]));
    GridChoice g;
    RET(measure_and_choose(sets, C.d_sets, C.box_scratch, C.box_out, C.d, emin, emax, o, g, st));
    if (g.n > gmax.n) g.n = gmax.n;
    g.M = g.n / 4;
    C.g = g;
    CK(cudaMemsetAsync(C.stats_begin, 0, C.stats_bytes, st));
    std::vector<PrepSet> s2;
    for (int k = 0; k < K; ++k) {
        C.sets[k].maxsub = (C.n[k] + mot_sub_points(C.d) - 1) / mot_sub_points(C.d) + mot_ntiles(C.d, g.n);
        s2.push_back(prepset_of(C.sets[k], P->x[k], P->mu[k]));
    }
    CK(cudaMemcpyAsync(C.d_sets, s2.data(), sizeof(PrepSet) * s2.size(), cudaMemcpyHostToDevice, st));
    CK(launch_prep(C.d_sets, s2.data(), K, C.d, g.n, g.c, g.s, C.err, st));
    if (C.has_close) CK(launch_close_points(P->x_close, C.sets[0].perm, C.n0, C.d, g.c, g.s, g.n, C.u_close, C.err, st));
    for (int k = 0; k < K; ++k) CK(cudaMemsetAsync(C.raw[k], 0, sizeof(float) * C.n[k], st));
    if (C.path == MOT_PATH_NFFT) {
        CK(prepare_window());
        CK(prepare_fftconv(C.d, g.n));
        size_t gsz = 1;
        for (int t = 0; t < C.d; ++t) gsz *= g.n;
        for (int k = 0; k < K; ++k) {
            int same = -1;
            for (int q = 0; q < k && same < 0; ++q)
                if (C.w[q] == C.w[k]) same = q;
            if (same >= 0)
                C.D[k] = C.D[same];
            else
                RET(make_D_for((C.eta / C.w[k]) / (g.s * g.s), g, C.d, o, C.dscr_a, C.dscr_b, C.D[k], st));
        }
        for (int c = 0; c < C.CB; ++c) CK(cudaMemsetAsync(C.grid[c], 0, gsz * sizeof(float), st));
        C.c1 = c1_supported(C.d, g.n) && C.c1_G != nullptr;
        if (C.c1) {
            for (int k = 0; k < K; ++k) CK(launch_c1_taps(C.sets[k].u, C.n[k], C.c1_l0[k], C.c1_w[k], st));
            for (int k = 0; k < K; ++k) CK(launch_c1_circulant(C.D[k], g.M, g.n, C.c1_c[k], st));
        }
    } else if (C.path == MOT_PATH_DENSE) {
        int nmax = 0;
        for (int k = 0; k < K; ++k) nmax = std::max(nmax, C.n[k]);
        for (int c = 0; c < C.CB; ++c) CK(cudaMemsetAsync(C.rawm[c], 0, sizeof(float) * nmax, st));
    }
    // fixed dense kernel matrices: beta_{K-1} = K^{(K-1,0)} (against sigma(x^0) for an Euler flow,
    // Section 6.3), Gam_1 = K^{(1,0)}
    auto eta_u = [&](int edge) { return (float)((C.eta / C.w[edge]) / (g.s * g.s) * (double)g.n * (double)g.n); };
    if (C.path == MOT_PATH_DENSE_BF16X3) {
        // split kernel matrices of the batched products (fixed for the solve)
        CK(prepare_tc_gemm());
        for (int k = 2; k < K; ++k)
            CK(launch_kernel_split(C.sets[k].u, C.n[k], C.sets[k - 1].u, C.n[k - 1], C.d, eta_u(k - 1),
                                   tc_ld(C.n[k - 1]), C.ktf_hi[k], C.ktf_lo[k], st));
        for (int k = 1; k <= K - 2; ++k)
            CK(launch_kernel_split(C.sets[k].u, C.n[k], C.sets[k + 1].u, C.n[k + 1], C.d, eta_u(k),
                                   tc_ld(C.n[k + 1]), C.ktb_hi[k], C.ktb_lo[k], st));
    }
    CK(launch_kernel_matrix(C.sets[K - 1].u, C.n[K - 1], C.has_close ? C.u_close : C.sets[0].u, C.n0, C.d,
                            eta_u(K - 1), C.beta[K - 1], C.beta_sc(K - 1), st));
    CK(launch_kernel_matrix(C.sets[1].u, C.n[1], C.sets[0].u, C.n0, C.d, eta_u(0), C.gam[1], C.gam_sc(1), st));
    c_build(C);
    if (C.path == MOT_PATH_DENSE_BF16X3) {
        for (int k = 2; k < K; ++k) {
            const int ld = tc_ld(C.n[k - 1]);
            if (!tc_prepare(&C.fwd[k].tc, C.a_hi, C.a_lo, C.n0, ld, C.ktf_hi[k], C.ktf_lo[k], C.n[k], ld, C.n[k - 1]))
                return MOT_ECUDA;
        }
        for (int k = 1; k <= K - 2; ++k) {
            const int ld = tc_ld(C.n[k + 1]);
            if (!tc_prepare(&C.bwd[k].tc, C.a_hi, C.a_lo, C.n0, ld, C.ktb_hi[k], C.ktb_lo[k], C.n[k], ld, C.n[k + 1]))
                return MOT_ECUDA;
        }
    }
    RET(c_upload(C, st));
    return MOT_OK;
}


// =============================================================================================
// resumable solve: a plan plus the stop-test loop, shared by mot_solve and the server
// =============================================================================================
struct PlanOps {
    virtual ~PlanOps() {}
    virtual int init(const double* const* u_warm, cudaStream_t st, Timer& tm, long long& nl) = 0;
    virtual int iterations(int count, cudaStream_t st, Timer& tm, long long& nl, bool graphs) = 0;
    virtual int check(cudaStream_t st, Timer& tm, long long& nl) = 0;
    virtual char* stats_dev() = 0;
    virtual size_t stats_bytes() const = 0;
    virtual int K() const = 0;
    virtual int n_scales() const = 0;          // scale records in the stats region
    virtual bool constrained(int k) const = 0;
    virtual double eta() const = 0;
    virtual int output(double* const* u, double* const* pair, cudaStream_t st, long long& nl) = 0;
    virtual void geometry(mot_result* r) const = 0;
};

struct TreeOps : PlanOps {
    TreePlan T;
    int init(const double* const* u_warm, cudaStream_t st, Timer& tm, long long& nl) override {
        int minus1 = -1;
        CK(cudaMemcpyAsync(T.iter, &minus1, sizeof(int), cudaMemcpyHostToDevice, st));
        OutBatch cold;                                             // every cold start in one launch
        cold.nsets = 0;
        cold.eta = T.eta;
        for (int k = 0; k < T.K; ++k) {
            const double* uw = (u_warm && !T.free_[k]) ? u_warm[T.order[k]] : nullptr;
            if (uw == nullptr && T.K <= 64) {
                cold.s[cold.nsets++] = OutSet{T.phi[k], T.phi_sc(k), T.sets[k].perm, T.n[k], nullptr};
                continue;
            }
            CK(launch_init_phi(T.phi[k], T.phi_sc(k), T.sets[k].perm, T.sets[k].mu_d, T.n[k], uw, T.eta,
                               &T.acc[0].logphi, T.box_scratch, st));
            nl += uw ? 2 : 1;
        }
        if (cold.nsets > 0) {
            CK(launch_init_cold_batch(cold, st));
            nl += 1;
        }
        T.par = 0;                                                 // the first beta copy
        for (auto& L : T.bwd) RET(run_level(T, L, st, tm, nl));   // Algorithm 2, steps 3-5
        return MOT_OK;
    }
    int iterations(int count, cudaStream_t st, Timer& tm, long long& nl, bool graphs) override {
        return run_iterations(T, count, st, tm, nl, graphs);
    }
    int check(cudaStream_t st, Timer& tm, long long& nl) override {
        if (T.check_done) {          // the persistent wavefront launch already ran the check pass
            T.check_done = false;
            return MOT_OK;
        }
        return run_check(T, st, tm, nl);
    }
    char* stats_dev() override { return T.stats_begin; }
    size_t stats_bytes() const override { return T.stats_bytes; }
    int K() const override { return T.K; }
    int n_scales() const override { return 5 * T.K; }
    bool constrained(int k) const override { return !T.free_[k]; }
    double eta() const override { return T.eta; }
    int output(double* const* u, double* const*, cudaStream_t st, long long& nl) override {
        if (!u) return MOT_OK;
        OutBatch B;                                                // every set's potentials in one launch
        B.nsets = T.K;
        B.eta = T.eta;
        for (int k = 0; k < T.K; ++k) B.s[k] = OutSet{T.phi[k], T.phi_sc(k), T.sets[k].perm, T.n[k], u[T.order[k]]};
        CK(launch_output_batch(B, st));
        nl += 1;
        return MOT_OK;
    }
    void geometry(mot_result* r) const override {
        r->scale = T.g.s;
        r->eta_norm = T.eta / (T.g.s * T.g.s);
        r->n_grid = T.path == MOT_PATH_NFFT ? T.g.n : 0;
        r->M = T.path == MOT_PATH_NFFT ? T.g.M : 0;
    }
    ~TreeOps() override {
        if (T.gexec) cudaGraphExecDestroy(T.gexec);
    }
};

struct CircleOps : PlanOps {
    CirclePlan C;
    int init(const double* const* u_warm, cudaStream_t st, Timer& tm, long long& nl) override {
        int minus1 = -1;
        CK(cudaMemcpyAsync(C.iter, &minus1, sizeof(int), cudaMemcpyHostToDevice, st));
        OutBatch cold;                                             // every cold start in one launch
        cold.nsets = 0;
        cold.eta = C.eta;
        for (int k = 0; k < C.K; ++k) {
            const double* uw = u_warm ? u_warm[k] : nullptr;
            if (uw == nullptr) {
                cold.s[cold.nsets++] = OutSet{C.phi[k], C.phi_sc(k), C.sets[k].perm, C.n[k], nullptr};
                continue;
            }
            CK(launch_init_phi(C.phi[k], C.phi_sc(k), C.sets[k].perm, C.sets[k].mu_d, C.n[k], uw, C.eta,
                               &C.acc[0].logphi, C.box_scratch, st));
            nl += 2;
        }
        if (cold.nsets > 0) {
            CK(launch_init_cold_batch(cold, st));
            nl += 1;
        }
        cudaEvent_t e = nullptr;                                   // Algorithm 3, steps 3-5
        RET(tm.begin(MOT_K_NODE, &e));
        CK(launch_prologue(C.d_resets + C.bw_r0, (int)C.bw_rn, 0, 0, nullptr, 0, C.G, st));
        RET(tm.end(e));
        return c_backward(C, st, tm, nl);
    }
    int iterations(int count, cudaStream_t st, Timer& tm, long long& nl, bool graphs) override {
        return c_run_iterations(C, count, st, tm, nl, graphs);
    }
    int check(cudaStream_t st, Timer& tm, long long& nl) override { return c_check(C, st, tm, nl); }
    char* stats_dev() override { return C.stats_begin; }
    size_t stats_bytes() const override { return C.stats_bytes; }
    int K() const override { return C.K; }
    int n_scales() const override { return 4 * C.K; }
    bool constrained(int) const override { return true; }
    double eta() const override { return C.eta; }
    int output(double* const* u, double* const* pair, cudaStream_t st, long long& nl) override {
        if (u) {
            OutBatch B;                                            // every set's potentials in one launch
            B.nsets = C.K;
            B.eta = C.eta;
            for (int k = 0; k < C.K; ++k) B.s[k] = OutSet{C.phi[k], C.phi_sc(k), C.sets[k].perm, C.n[k], u[k]};
            CK(launch_output_batch(B, st));
            nl += 1;
        }
        // pair marginals Pi_{0,k} (Section 6.3): after a full sweep and the check pass, Gam_k and
        // beta_k are the chains 0 -> k and k -> 0 at the returned scalings
        for (int k = 1; k < C.K && pair; ++k) {
            if (!pair[k]) continue;
            CK(launch_pair(C.phi[0], C.phi_sc(0), C.sets[0].perm, C.n0, C.phi[k], C.phi_sc(k), C.sets[k].perm,
                           C.n[k], C.gam[k], C.gam_sc(k), C.beta[k], C.beta_sc(k), pair[k], st));
            nl += 1;
        }
        return MOT_OK;
    }
    void geometry(mot_result* r) const override {
        r->scale = C.g.s;
        r->eta_norm = C.eta / (C.g.s * C.g.s);
        r->n_grid = C.path == MOT_PATH_NFFT ? C.g.n : 0;
        r->M = C.path == MOT_PATH_NFFT ? C.g.M : 0;
    }
    ~CircleOps() override {
        if (C.gexec) cudaGraphExecDestroy(C.gexec);
    }
};

// Build the plan of a problem inside `ws` (sizes: mot_workspace_bytes) and enqueue its set-up.
// =============================================================================================
// small-eta local path (Section 6.1, closing remark): Algorithm 2 in the log domain with every
// kernel sum truncated to the pairs within r_cut (local.cu)
// =============================================================================================
constexpr int kLocalMaxCells = 1 << 16;      // cells of the common grid (h grows until they fit)

struct LocalPlan {
    TreePlan S;                              // tree structure only (BFS labels, parents, depths)
    int K = 0, d = 0;
    double eta = 0.0, h = 0.0;
    std::vector<double> r_e;                 // cutoff of edge {p(k), k}
    LGrid grid{};
    int nmax = 0;
    // per node (BFS labels)
    std::vector<LBinSet> bins;
    std::vector<double*> f;
    // per edge k >= 1
    std::vector<double*> b, g, gx, Lc_f, Lc_b, Lc_c;
    std::vector<float*> dl_f, dl_b, dl_c;
    // tasks: forward (one launch), root, backward levels, check levels, check root
    std::vector<LTask> fwd, root, chkroot;
    std::vector<std::vector<LTask>> bwd, chk;
    LTask* d_fwd = nullptr;
    LTask* d_root = nullptr;
    LTask* d_chkroot = nullptr;
    std::vector<LTask*> d_bwd, d_chk;
    LTask* d_tasks = nullptr;
    size_t task_cap = 0;
    std::vector<LFac> fac;
    LFac* d_fac = nullptr;
    size_t fac_cap = 0;
    LBinSet* d_bins = nullptr;
    int* d_maxcount = nullptr;               // [K] most points in one cell, per set
    std::vector<int> maxcount;
    float* box_scratch = nullptr;
    float* box_out = nullptr;
    PrepSet* d_sets = nullptr;
    // stats region: the accumulator ring, per-node check accumulators, error word and counter
    char* stats_begin = nullptr;
    size_t stats_bytes = 0;
    IterAcc* acc = nullptr;
    double* acc_node = nullptr;
    int* err = nullptr;
    int* iter = nullptr;
    LGlobals LG{};
    Globals G{};
    cudaGraphExec_t gexec = nullptr;
    int graph_iters = 0;
    long long launches_per_iter = 0;
};

void layout_local(Arena& A, LocalPlan& L) {
    const int K = L.K, d = L.d;
    const int nc = kLocalMaxCells;
    L.bins.assign(K, LBinSet());
    L.f.assign(K, nullptr);
    for (int k = 0; k < K; ++k) {
        const int n = L.S.n[k];
        LBinSet& B = L.bins[k];
        B.n = n;
        B.cell = A.take<int>(n);
        B.cstart = A.take<int>(nc + 1);
        B.cursor = A.take<int>(nc);
        B.u = A.take<float>((size_t)d * n);
        B.perm = A.take<int>(n);
        B.mu_s = A.take<double>(n);
        B.logmu = A.take<double>(n);
        L.f[k] = A.take<double>(n);
    }
    for (auto* v : {&L.b, &L.g, &L.gx, &L.Lc_f, &L.Lc_b, &L.Lc_c}) v->assign(K, nullptr);
    for (auto* v : {&L.dl_f, &L.dl_b, &L.dl_c}) v->assign(K, nullptr);
    for (int k = 1; k < K; ++k) {
        const int p = L.S.parent[k], nk = L.S.n[k], np = L.S.n[p];
        L.b[k] = A.take<double>(np);
        L.g[k] = A.take<double>(nk);
        L.gx[k] = A.take<double>(nk);
        L.dl_f[k] = A.take<float>(np);
        L.dl_b[k] = A.take<float>(nk);
        L.dl_c[k] = A.take<float>(np);
        L.Lc_f[k] = A.take<double>(nc);
        L.Lc_b[k] = A.take<double>(nc);
        L.Lc_c[k] = A.take<double>(nc);
    }
    L.stats_bytes = sizeof(IterAcc) * kRing + sizeof(double) * 3 * K + 16;
    L.stats_begin = A.take<char>(L.stats_bytes);
    if (!A.measure) {
        L.acc = reinterpret_cast<IterAcc*>(L.stats_begin);
        L.acc_node = reinterpret_cast<double*>(L.stats_begin + sizeof(IterAcc) * kRing);
        L.err = reinterpret_cast<int*>(L.stats_begin + L.stats_bytes - 16);
        L.iter = L.err + 1;
    }
    L.task_cap = 3 * (size_t)K + 4;
    L.d_tasks = A.take<LTask>(L.task_cap);
    L.fac_cap = 6 * (size_t)K + 8;
    for (int k = 0; k < K; ++k) L.fac_cap += 2 * L.S.children[k].size();
    L.d_fac = A.take<LFac>(L.fac_cap);
    L.d_bins = A.take<LBinSet>(K);
    L.d_maxcount = A.take<int>(K);
    L.d_sets = A.take<PrepSet>(K);
    L.box_scratch = A.take<float>(8);
    L.box_out = A.take<float>(8);
}

LSet lset_of(const LocalPlan& L, int k) {
    LSet s;
    s.n = L.S.n[k];
    s.u = L.bins[k].u;
    s.cstart = L.bins[k].cstart;
    s.logmu = L.bins[k].logmu;
    s.mu = L.bins[k].mu_s;
    return s;
}

LTask ltask_blank() {
    LTask t;
    std::memset(&t, 0, sizeof(t));
    return t;
}

int lchunks(const LocalPlan& L, int node) { return (L.maxcount[node] + LSE_TARGETS - 1) / LSE_TARGETS; }

void ltask_kernel(LocalPlan& L, LTask& t, int k) {
    const double eta_e = L.eta / L.S.w[k];
    t.inv_eta = (float)(1.0 / eta_e);
    t.inv_eta_d = 1.0 / eta_e;
    t.r2 = (float)(L.r_e[k] * L.r_e[k]);
}

void lfac(LocalPlan& L, const double* v, int sign) {
    LFac f;
    f.v = v;
    f.sign = sign;
    L.fac.push_back(f);
}

void local_build(LocalPlan& L) {
    const int K = L.K;
    const TreePlan& S = L.S;
    L.fac.clear();
    L.fwd.clear();
    for (int k = 1; k < K; ++k) {          // gamma_k = K^T (mu^p / beta_k), then f^k (Algorithm 2, forward)
        const int p = S.parent[k];
        LTask t = ltask_blank();
        t.src = lset_of(L, p);
        t.sf0 = (int)L.fac.size();
        lfac(L, L.bins[p].logmu, +1);
        lfac(L, L.b[k], -1);
        t.snf = 2;
        t.tgt = lset_of(L, k);
        t.tf0 = (int)L.fac.size();
        for (int c : S.children[k]) lfac(L, L.b[c], +1);
        t.tnf = (int)L.fac.size() - t.tf0;
        t.delta = L.dl_f[k];
        t.Lc = L.Lc_f[k];
        ltask_kernel(L, t, k);
        t.mode = LEPI_FWD;
        t.out = L.g[k];
        t.f = L.f[k];
        t.tchunks = lchunks(L, k);
        L.fwd.push_back(t);
    }
    auto root_task = [&](int mode) {
        LTask t = ltask_blank();
        t.tgt = lset_of(L, 0);
        t.tf0 = (int)L.fac.size();
        for (int c : S.children[0]) lfac(L, L.b[c], +1);
        t.tnf = (int)L.fac.size() - t.tf0;
        t.mode = mode;
        t.f = L.f[0];
        t.acc_node = L.acc_node;
        return t;
    };
    L.root.assign(1, root_task(LEPI_ROOT));
    int maxdepth = 0;
    for (int k = 0; k < K; ++k) maxdepth = std::max(maxdepth, S.depth[k]);
    L.bwd.assign(std::max(maxdepth, 1), {});
    for (int k = K - 1; k >= 1; --k) {     // beta_k = K (phi^k (.) beta^{C_k}), deepest level first
        LTask t = ltask_blank();
        t.src = lset_of(L, k);
        t.sf0 = (int)L.fac.size();
        lfac(L, L.f[k], +1);
        for (int c : S.children[k]) lfac(L, L.b[c], +1);
        t.snf = (int)L.fac.size() - t.sf0;
        t.tgt = lset_of(L, S.parent[k]);
        t.delta = L.dl_b[k];
        t.Lc = L.Lc_b[k];
        ltask_kernel(L, t, k);
        t.mode = LEPI_MSG;
        t.out = L.b[k];
        t.tchunks = lchunks(L, S.parent[k]);
        L.bwd[maxdepth - S.depth[k]].push_back(t);
    }
    L.chk.assign(std::max(maxdepth, 1), {});
    for (int k = 1; k < K; ++k) {          // check pass: gamma-ex_k from the root down (Theorem 4.1)
        const int p = S.parent[k];
        LTask t = ltask_blank();
        t.src = lset_of(L, p);
        t.sf0 = (int)L.fac.size();
        lfac(L, L.f[p], +1);
        if (p != 0) lfac(L, L.gx[p], +1);
        for (int c : S.children[p])
            if (c != k) lfac(L, L.b[c], +1);
        t.snf = (int)L.fac.size() - t.sf0;
        t.tgt = lset_of(L, k);
        t.tf0 = (int)L.fac.size();
        for (int c : S.children[k]) lfac(L, L.b[c], +1);
        t.tnf = (int)L.fac.size() - t.tf0;
        t.delta = L.dl_c[k];
        t.Lc = L.Lc_c[k];
        ltask_kernel(L, t, k);
        t.mode = LEPI_CHK;
        t.out = L.gx[k];
        t.f = L.f[k];
        t.acc_node = L.acc_node + 3 * k;
        t.tchunks = lchunks(L, k);
        L.chk[S.depth[k] - 1].push_back(t);
    }
    L.chkroot.assign(1, root_task(LEPI_CHKROOT));
}

int local_upload(LocalPlan& L, cudaStream_t st) {
    if (L.fac.size() > L.fac_cap) return MOT_EUNSUPPORTED;
    std::vector<LTask> all;
    auto place = [&](std::vector<LTask>& v) {
        LTask* p = L.d_tasks + all.size();
        for (auto& t : v) all.push_back(t);
        return p;
    };
    L.d_fwd = place(L.fwd);
    L.d_root = place(L.root);
    L.d_chkroot = place(L.chkroot);
    L.d_bwd.clear();
    for (auto& v : L.bwd) L.d_bwd.push_back(place(v));
    L.d_chk.clear();
    for (auto& v : L.chk) L.d_chk.push_back(place(v));
    if (all.size() > L.task_cap) return MOT_EUNSUPPORTED;
    CK(cudaMemcpyAsync(L.d_fac, L.fac.data(), sizeof(LFac) * L.fac.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(L.d_tasks, all.data(), sizeof(LTask) * all.size(), cudaMemcpyHostToDevice, st));
    return MOT_OK;
}

int local_setup(const mot_problem* P, const mot_options& o, LocalPlan& L, void* ws, size_t ws_bytes, bool measure,
                size_t* need, cudaStream_t st) {
    RET(tree_structure(P, L.S));
    if (P->free_nodes)
        for (int k = 0; k < P->K; ++k)
            if (P->free_nodes[k]) return MOT_EUNSUPPORTED;
    if (o.r_cut < 0.0 || !std::isfinite(o.r_cut)) return MOT_EINVAL;
    L.K = P->K;
    L.d = P->d;
    L.eta = P->eta;
    L.r_e.assign(L.K, 0.0);
    L.h = 0.0;
    for (int k = 1; k < L.K; ++k) {
        // the kernel of edge k is below e^-40 beyond sqrt(40 eta_e) unless the caller sets r_cut
        L.r_e[k] = o.r_cut > 0.0 ? o.r_cut : std::sqrt(40.0 * P->eta / L.S.w[k]);
        L.h = std::max(L.h, L.r_e[k]);
    }
    Arena A;
    A.measure = measure;
    A.base = reinterpret_cast<char*>(ws);
    A.cap = ws_bytes;
    layout_local(A, L);
    if (measure) {
        *need = A.off + 256;
        return MOT_OK;
    }
    if (A.off > ws_bytes) return MOT_ENOMEM;
    // bounding box of all points (one readback), then the cell grid
    std::vector<PrepSet> sets;
    for (int k = 0; k < L.K; ++k) {
        PrepSet ps;
        std::memset(&ps, 0, sizeof(ps));
        ps.x = P->x[L.S.order[k]];
        ps.n = L.S.n[k];
        sets.push_back(ps);
    }
    CK(cudaMemcpyAsync(L.d_sets, sets.data(), sizeof(PrepSet) * sets.size(), cudaMemcpyHostToDevice, st));
    CK(launch_bounds(L.d_sets, L.K, L.d, L.box_scratch, L.box_out, st));
    float hb[7] = {0, 0, 0, 0, 0, 0, 0};
    CK(cudaMemcpyAsync(hb, L.box_out, sizeof(float) * (2 * L.d + 1), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    double h = L.h;
    for (int t = 0; t < L.d; ++t)
        if (!std::isfinite(hb[2 * t]) || !std::isfinite(hb[2 * t + 1])) return MOT_ENUMERIC;
    for (;;) {
        long long cells = 1;
        for (int t = 0; t < L.d; ++t) cells *= std::max(1LL, (long long)std::ceil(((double)hb[2 * t + 1] - hb[2 * t]) / h + 1e-9));
        if (cells <= kLocalMaxCells) break;
        h *= 1.25;                            // larger cells: still every pair within r_cut is in the 3^d block
    }
    L.grid.d = L.d;
    L.grid.ncells = 1;
    for (int t = 0; t < 3; ++t) {
        L.grid.dims[t] = 1;
        L.grid.lo[t] = 0.f;
    }
    for (int t = 0; t < L.d; ++t) {
        L.grid.lo[t] = hb[2 * t];
        L.grid.dims[t] = std::max(1, (int)std::ceil(((double)hb[2 * t + 1] - hb[2 * t]) / h + 1e-9));
        L.grid.ncells *= L.grid.dims[t];
    }
    L.grid.h = (float)h;
    L.grid.inv_h = (float)(1.0 / h);
    // binning
    CK(cudaMemsetAsync(L.stats_begin, 0, L.stats_bytes, st));
    L.nmax = 0;
    for (int k = 0; k < L.K; ++k) {
        L.bins[k].x = P->x[L.S.order[k]];
        L.bins[k].mu = P->mu[L.S.order[k]];
        L.nmax = std::max(L.nmax, L.S.n[k]);
        CK(cudaMemsetAsync(L.bins[k].cstart, 0, sizeof(int) * (L.grid.ncells + 1), st));
    }
    CK(cudaMemcpyAsync(L.d_bins, L.bins.data(), sizeof(LBinSet) * L.K, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(L.d_maxcount, 0, sizeof(int) * L.K, st));
    CK(launch_lbin(L.d_bins, L.K, L.nmax, L.grid, L.err, L.d_maxcount, st));
    // the fullest cell of each set sizes the log-sum-exp grid (one readback)
    L.maxcount.assign(L.K, 0);
    CK(cudaMemcpyAsync(L.maxcount.data(), L.d_maxcount, sizeof(int) * L.K, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    L.LG.iter = L.iter;
    L.LG.acc = L.acc;
    L.LG.R = kRing;
    L.LG.err = L.err;
    std::memset(&L.G, 0, sizeof(L.G));
    L.G.iter = L.iter;
    L.G.acc = L.acc;
    L.G.R = kRing;
    local_build(L);
    RET(local_upload(L, st));
    return MOT_OK;
}

// One level of truncated kernel sums: per-cell source maxima, then the log-sum-exp (timed as
// MOT_K_NODE and MOT_K_LOCAL).
int local_level(LocalPlan& L, const LTask* d, const std::vector<LTask>& h, cudaStream_t st, Timer& tm, long long& nl) {
    cudaEvent_t e = nullptr;
    const int n = (int)h.size();
    int tch = 1;
    for (const LTask& t : h) tch = std::max(tch, t.tchunks);
    if (tch > 65535) return MOT_EUNSUPPORTED;             // a cell of more than 2^24 points
    RET(tm.begin(MOT_K_NODE, &e));
    CK(launch_lsrc(d, n, L.d_fac, L.grid.ncells, L.err, st));
    RET(tm.end(e));
    RET(tm.begin(MOT_K_LOCAL, &e));
    CK(launch_lse(d, n, tch, L.d_fac, L.grid, L.LG, st));
    RET(tm.end(e));
    nl += 2;
    return MOT_OK;
}

int local_backward(LocalPlan& L, cudaStream_t st, Timer& tm, long long& nl) {
    for (size_t l = 0; l < L.bwd.size(); ++l) RET(local_level(L, L.d_bwd[l], L.bwd[l], st, tm, nl));
    return MOT_OK;
}

int local_iteration(LocalPlan& L, cudaStream_t st, Timer& tm, long long& nl) {
    cudaEvent_t e = nullptr;
    RET(tm.begin(MOT_K_NODE, &e));
    CK(launch_prologue(nullptr, 0, 0, 1, nullptr, 0, L.G, st));
    RET(tm.end(e));
    nl += 1;
    RET(local_level(L, L.d_fwd, L.fwd, st, tm, nl));
    RET(tm.begin(MOT_K_NODE, &e));
    CK(launch_lroot(L.d_root, 1, L.d_fac, L.nmax, L.LG, st));
    RET(tm.end(e));
    nl += 1;
    return local_backward(L, st, tm, nl);
}

int local_check(LocalPlan& L, cudaStream_t st, Timer& tm, long long& nl) {
    cudaEvent_t e = nullptr;
    RET(tm.begin(MOT_K_NODE, &e));
    CK(launch_prologue(nullptr, 0, 0, 0, L.acc_node, 3 * L.K, L.G, st));
    CK(launch_lroot(L.d_chkroot, 1, L.d_fac, L.nmax, L.LG, st));
    RET(tm.end(e));
    nl += 2;
    for (size_t l = 0; l < L.chk.size(); ++l) RET(local_level(L, L.d_chk[l], L.chk[l], st, tm, nl));
    return MOT_OK;
}

int local_iterations(LocalPlan& L, int count, cudaStream_t st, Timer& tm, long long& nl, bool graphs) {
    if (count <= 0) return MOT_OK;
    if (graphs && tm.on && st != nullptr) {
        long long per = 0;
        RET(tm.timed_graph(count, 2 * (size_t)(4 * L.K + 8), [&](long long& dn) {
            const long long before = dn;
            const int rc = local_iteration(L, st, tm, dn);
            per = dn - before;
            return rc;
        }));
        nl += per * count;
        return MOT_OK;
    }
    if (graphs && !tm.on && st != nullptr) {
        if (L.gexec == nullptr || L.graph_iters != count) {
            if (L.gexec) {
                cudaGraphExecDestroy(L.gexec);
                L.gexec = nullptr;
            }
            cudaGraph_t graph;
            CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            long long dn = 0;
            int rc = MOT_OK;
            for (int i = 0; i < count && rc == MOT_OK; ++i) rc = local_iteration(L, st, tm, dn);
            cudaError_t ce = cudaStreamEndCapture(st, &graph);
            if (rc != MOT_OK) return rc;
            CK(ce);
            CK(cudaGraphInstantiate(&L.gexec, graph, 0));
            cudaGraphDestroy(graph);
            L.graph_iters = count;
            L.launches_per_iter = dn / count;
        }
        CK(cudaGraphLaunch(L.gexec, st));
        nl += L.launches_per_iter * count;
        return MOT_OK;
    }
    for (int i = 0; i < count; ++i) RET(local_iteration(L, st, tm, nl));
    return MOT_OK;
}

struct LocalOps : PlanOps {
    LocalPlan L;
    int init(const double* const* u_warm, cudaStream_t st, Timer& tm, long long& nl) override {
        (void)tm;
        int minus1 = -1;
        CK(cudaMemcpyAsync(L.iter, &minus1, sizeof(int), cudaMemcpyHostToDevice, st));
        for (int k = 0; k < L.K; ++k) {
            const double* uw = u_warm ? u_warm[L.S.order[k]] : nullptr;
            CK(launch_linit(L.f[k], L.bins[k].perm, L.bins[k].mu_s, L.S.n[k], uw, L.eta, &L.acc[0].logphi, st));
            nl += 1;
        }
        return local_backward(L, st, tm, nl);    // Algorithm 2, steps 3-5
    }
    int iterations(int count, cudaStream_t st, Timer& tm, long long& nl, bool graphs) override {
        return local_iterations(L, count, st, tm, nl, graphs);
    }
    int check(cudaStream_t st, Timer& tm, long long& nl) override { return local_check(L, st, tm, nl); }
    char* stats_dev() override { return L.stats_begin; }
    size_t stats_bytes() const override { return L.stats_bytes; }
    int K() const override { return L.K; }
    int n_scales() const override { return 0; }
    bool constrained(int) const override { return true; }
    double eta() const override { return L.eta; }
    int output(double* const* u, double* const*, cudaStream_t st, long long& nl) override {
        for (int k = 0; k < L.K && u; ++k) {
            if (!u[L.S.order[k]]) continue;
            CK(launch_lout(L.f[k], L.bins[k].perm, L.S.n[k], L.eta, u[L.S.order[k]], st));
            nl += 1;
        }
        return MOT_OK;
    }
    void geometry(mot_result* r) const override {
        r->scale = 1.0;
        r->eta_norm = L.eta;
        r->n_grid = 0;
        r->M = 0;
    }
    ~LocalOps() override {
        if (L.gexec) cudaGraphExecDestroy(L.gexec);
    }
};

int make_ops(const mot_problem* P, const mot_options& o, void* ws, size_t ws_bytes, cudaStream_t st, PlanOps** out) {
    if (o.path == MOT_PATH_LOCAL) {
        if (P->topology != MOT_TREE) return MOT_EUNSUPPORTED;
        LocalOps* l = new LocalOps();
        int rc = local_setup(P, o, l->L, ws, ws_bytes, false, nullptr, st);
        if (rc != MOT_OK) {
            delete l;
            return rc;
        }
        *out = l;
        return MOT_OK;
    }
    if (P->topology == MOT_TREE) {
        TreeOps* t = new TreeOps();
        int rc = tree_plan_setup(P, o, t->T, ws, ws_bytes, false, nullptr, st);
        if (rc != MOT_OK) {
            delete t;
            return rc;
        }
        *out = t;
    } else {
        CircleOps* c = new CircleOps();
        int rc = circle_setup(P, o, c->C, ws, ws_bytes, false, nullptr, st);
        if (rc != MOT_OK) {
            delete c;
            return rc;
        }
        *out = c;
    }
    return MOT_OK;
}

struct Solve {
    PlanOps* ops = nullptr;
    mot_options o;
    cudaStream_t st = nullptr;
    Timer tm;
    long long nl = 0;
    int iters = 0, status = MOT_OK;
    double viol = INFINITY, S_last = NAN, S_prev = NAN;
    bool met = false, done = false;
    char* hstats = nullptr;           // host copy of the stats region (pinned for the server)
    cudaEvent_t ev = nullptr;

    int start(const double* const* u_warm) {
        tm.on = o.timing != 0;
        tm.st = st;
        if (tm.on) CK(launch_delay(3000000ull, st));    // let the host run ahead of the timed launches
        return ops->init(u_warm, st, tm, nl);
    }
    // enqueue the next chunk of iterations, the check pass and the stats copy; record ev
    int launch() {
        const int chunk = std::min(o.check_every, o.max_iter - iters);
        RET(ops->iterations(chunk, st, tm, nl, o.use_graphs > 0));
        iters += chunk;
        RET(ops->check(st, tm, nl));
        CK(cudaMemcpyAsync(hstats, ops->stats_dev(), ops->stats_bytes(), cudaMemcpyDeviceToHost, st));
        CK(cudaEventRecord(ev, st));
        return MOT_OK;
    }
    // after ev completed: stop test (sets done)
    int evaluate(mot_result* res) {
        RET(tm.collect(res));
        const size_t sb = ops->stats_bytes();
        const int K = ops->K();
        const IterAcc* acc = reinterpret_cast<const IterAcc*>(hstats);
        const double* node = reinterpret_cast<const double*>(hstats + sizeof(IterAcc) * kRing);
        if (const int e = *reinterpret_cast<const int*>(hstats + sb - 16)) return (e & 4) ? MOT_ETIMEOUT : MOT_ENUMERIC;
        viol = 0.0;
        for (int k = 0; k < K; ++k)
            if (ops->constrained(k)) viol = std::max(viol, node[3 * k]);
        auto Sval = [&](int r) { const IterAcc& a = acc[r % kRing]; return ops->eta() * (a.logphi - a.mass); };
        if (iters >= 1) S_last = Sval(iters - 1);
        if (iters >= 2) S_prev = Sval(iters - 2);
        if (!std::isfinite(viol)) return MOT_ENUMERIC;
        const bool want_viol = o.tol_viol >= 0.0;
        if (iters >= o.min_iter) {
            if (want_viol && viol <= o.tol_viol) met = true;
            if (o.delta_S > 0.0 && iters >= 2 && std::fabs(S_last - S_prev) < o.delta_S) met = true;
        }
        if (met || iters >= o.max_iter) {
            done = true;
            if (!met && (want_viol || o.delta_S > 0.0)) status = MOT_ENOCONV;
        }
        return MOT_OK;
    }
    // fill the scalar results and enqueue u^k
    int finish(mot_result* res, double* const* u, double* const* pair) {
        const int K = ops->K();
        const IterAcc* acc = reinterpret_cast<const IterAcc*>(hstats);
        const double* node = reinterpret_cast<const double*>(hstats + sizeof(IterAcc) * kRing);
        const VecScale* scs = reinterpret_cast<const VecScale*>(hstats + sizeof(IterAcc) * kRing + sizeof(double) * 3 * K);
        if (u || pair) RET(ops->output(u, pair, st, nl));
        if (res) {
            double mass = node[2], plogphi = 0.0;
            for (int k = 0; k < K; ++k) plogphi += node[3 * k + 1];
            const IterAcc& cur = acc[iters % kRing];
            res->violation = viol;
            res->mass = mass;
            res->cost_dual = ops->eta() * (cur.logphi - mass);
            res->cost_primal = ops->eta() * (plogphi - mass);
            res->S_last = S_last;
            res->S_prev = S_prev;
            res->iters = iters;
            long long cl = 0;
            for (int i = 0; i < ops->n_scales(); ++i) cl += scs[i].clamped;
            res->clamped = cl;
            ops->geometry(res);
            res->launches = nl;
            res->status = status;
        }
        return MOT_OK;
    }
};

// Blocking solve on `st` (the mot_solve entry point).
int solve_blocking(const mot_problem* P, const mot_options& o, void* ws, size_t ws_bytes, const double* const* u_warm,
                   mot_result* res, cudaStream_t st) {
    Solve S;
    S.o = o;
    S.st = st;
    RET(make_ops(P, o, ws, ws_bytes, st, &S.ops));
    std::vector<char> h(S.ops->stats_bytes());
    S.hstats = h.data();
    int rc = cudaEventCreateWithFlags(&S.ev, cudaEventDisableTiming) == cudaSuccess ? MOT_OK : MOT_ECUDA;
    if (rc == MOT_OK) rc = S.start(u_warm);
    while (rc == MOT_OK && !S.done) {
        rc = S.launch();
        if (rc != MOT_OK) break;
        cudaError_t e = cudaEventSynchronize(S.ev);
        if (e != cudaSuccess) {
            set_cuda_error(e, "cudaEventSynchronize");
            rc = MOT_ECUDA;
            break;
        }
        rc = S.evaluate(res);
    }
    if (rc == MOT_OK) rc = S.finish(res, res ? res->u : nullptr, res ? res->pair : nullptr);
    if (rc == MOT_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = MOT_ECUDA;
    if (S.ev) cudaEventDestroy(S.ev);
    delete S.ops;
    return rc == MOT_OK ? S.status : rc;
}

// =============================================================================================
// server: continuous batching of solves (admission by workspace bytes, one stream per slot)
// =============================================================================================
struct Pool {   // first-fit allocator over [0, size) in 256-byte units of the caller's pool
    std::vector<std::pair<size_t, size_t>> free_;     // (offset, bytes), sorted, coalesced
    size_t size = 0;
    void init(size_t n) {
        size = n & ~(size_t)255;
        free_.assign(1, {0, size});
    }
    bool alloc(size_t n, size_t* off) {
        n = (n + 255) & ~(size_t)255;
        for (size_t i = 0; i < free_.size(); ++i) {
            if (free_[i].second >= n) {
                *off = free_[i].first;
                free_[i].first += n;
                free_[i].second -= n;
                if (free_[i].second == 0) free_.erase(free_.begin() + i);
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t n) {
        n = (n + 255) & ~(size_t)255;
        auto it = free_.begin();
        while (it != free_.end() && it->first < off) ++it;
        it = free_.insert(it, {off, n});
        const size_t i = it - free_.begin();
        if (i + 1 < free_.size() && free_[i].first + free_[i].second == free_[i + 1].first) {
            free_[i].second += free_[i + 1].second;
            free_.erase(free_.begin() + i + 1);
        }
        if (i > 0 && free_[i - 1].first + free_[i - 1].second == free_[i].first) {
            free_[i - 1].second += free_[i].second;
            free_.erase(free_.begin() + i);
        }
    }
};

struct Request {
    long long tag = 0;
    mot_problem prob;
    mot_options o;
    std::vector<int64_t> n;
    std::vector<const float*> x;
    std::vector<const double*> mu;
    std::vector<int> edges;
    std::vector<double> w;
    std::vector<unsigned char> freen;
    std::vector<double*> u;
    size_t ws_bytes = 0;
    double t_submit = 0.0;
};

struct Active {
    Request req;
    size_t off = 0;
    int slot = 0;
    Solve solve;
    mot_result res;
    bool finishing = false;
    double t_admit = 0.0;
};

const size_t kSlotStats = 32768;   // pinned host bytes per slot (stats of K <= 64)

}  // namespace

struct mot_server_s {
    char* base = nullptr;
    Pool pool;
    int max_active = 0;
    std::deque<Request> pending;
    std::vector<Active*> active;
    std::vector<mot_server_result> done;
    std::vector<cudaStream_t> streams;
    std::vector<char*> pinned;
    std::vector<bool> slot_busy;
    std::chrono::steady_clock::time_point t0;
    double now() const {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

void server_complete(mot_server_s* S, Active* a, int status) {
    mot_server_result r;
    std::memset(&r, 0, sizeof(r));
    r.tag = a->req.tag;
    r.status = status;
    r.iters = a->res.iters;
    r.violation = a->res.violation;
    r.cost_dual = a->res.cost_dual;
    r.cost_primal = a->res.cost_primal;
    r.submit_ms = a->req.t_submit;
    r.admit_ms = a->t_admit;
    r.done_ms = S->now();
    S->done.push_back(r);
    if (a->solve.ev) cudaEventDestroy(a->solve.ev);
    delete a->solve.ops;
    S->pool.release(a->off, a->req.ws_bytes);
    S->slot_busy[a->slot] = false;
    delete a;
}

void server_reject(mot_server_s* S, const Request& q, int status) {
    mot_server_result r;
    std::memset(&r, 0, sizeof(r));
    r.tag = q.tag;
    r.status = status;
    r.submit_ms = q.t_submit;
    r.admit_ms = r.done_ms = S->now();
    S->done.push_back(r);
}

}  // namespace

// =============================================================================================
// fast summation on its own
// =============================================================================================
namespace {

struct FsPlan {
    SetBufs src, tgt;
    std::vector<float*> grid, hgrid, raw;
    std::vector<float2*> spec;
    float* D = nullptr;
    float* a_sorted = nullptr;   // [nrhs][n_src]
    uint16_t* a_hi = nullptr;    // tensor-core path: split alpha [nrhs][ld] and kernel [n_tgt][ld]
    uint16_t* a_lo = nullptr;
    uint16_t* kt_hi = nullptr;
    uint16_t* kt_lo = nullptr;
    float* b_sorted = nullptr;   // [nrhs][n_tgt]
    PrepSet* d_sets = nullptr;
    float* box_scratch = nullptr;
    float* box_out = nullptr;
    double* dscr_a = nullptr;
    double* dscr_b = nullptr;
    Task* d_tasks = nullptr;
    int* err = nullptr;
    int* iter = nullptr;
    IterAcc* acc = nullptr;
};

void layout_fs(Arena& A, FsPlan& F, int d, int64_t ns, int64_t nt, int nrhs, int path, int ng) {
    const int M = ng / 4;
    layout_set(A, F.src, (int)ns, d, ng, false);
    layout_set(A, F.tgt, (int)nt, d, ng, false);
    size_t gsz = 1;
    for (int t = 0; t < d; ++t) gsz *= ng;
    F.grid.assign(nrhs, nullptr);
    F.hgrid.assign(nrhs, nullptr);
    F.spec.assign(nrhs, nullptr);
    F.raw.assign(nrhs, nullptr);
    for (int r = 0; r < nrhs; ++r) {
        if (path == MOT_PATH_NFFT) {
            F.grid[r] = A.take<float>(gsz);
            F.hgrid[r] = A.take<float>(gsz);
            if (d == 3) F.spec[r] = A.take<float2>((size_t)ng * (2 * M + 1) * (M + 1));
        } else if (path == MOT_PATH_DENSE) {
            F.raw[r] = A.take<float>(nt);
        }
    }
    if (path == MOT_PATH_DENSE_BF16X3) {
        const size_t ld = (size_t)tc_ld((int)ns);
        F.a_hi = A.take<uint16_t>((size_t)nrhs * ld);
        F.a_lo = A.take<uint16_t>((size_t)nrhs * ld);
        F.kt_hi = A.take<uint16_t>((size_t)nt * ld);
        F.kt_lo = A.take<uint16_t>((size_t)nt * ld);
    }
    if (path == MOT_PATH_NFFT) {
        F.D = A.take<float>(D_floats(d, M));
        size_t s = make_D_scratch_doubles(d, M);
        F.dscr_a = A.take<double>(s);
        F.dscr_b = A.take<double>(s);
    }
    F.a_sorted = A.take<float>((size_t)nrhs * ns);
    F.b_sorted = A.take<float>((size_t)nrhs * nt);
    F.d_sets = A.take<PrepSet>(2);
    F.box_scratch = A.take<float>(8);
    F.box_out = A.take<float>(8);
    F.d_tasks = A.take<Task>(nrhs);
    F.err = A.take<int>(4);
    F.iter = F.err + 1;
    F.acc = A.take<IterAcc>(2);
}

int fastsum_impl(int d, double eta, const float* x_src, int64_t n_src, const float* x_tgt, int64_t n_tgt,
                 const float* alpha, int nrhs, float* beta, const mot_options& o, void* ws, size_t ws_bytes,
                 double* scale_out, cudaStream_t st, bool measure, size_t* need) {
    if (d < 1 || d > 3 || n_src < 1 || n_tgt < 1 || nrhs < 1 || nrhs > 65535) return MOT_EINVAL;
    if (n_src > (1 << 26) || n_tgt > (1 << 26)) return MOT_EINVAL;
    if (!(eta > 0.0) || !std::isfinite(eta)) return MOT_EINVAL;
    if (o.path != MOT_PATH_NFFT && o.path != MOT_PATH_DENSE && o.path != MOT_PATH_DENSE_BF16X3)
        return MOT_EUNSUPPORTED;
    const int ngmax = o.n_grid > 0 ? o.n_grid : max_grid(d);
    if (ngmax < 16 || ngmax > max_grid(d) || (ngmax & (ngmax - 1))) return MOT_EINVAL;
    FsPlan F;
    Arena A;
    A.measure = measure;
    A.base = reinterpret_cast<char*>(ws);
    A.cap = ws_bytes;
    layout_fs(A, F, d, n_src, n_tgt, nrhs, o.path, ngmax);
    if (measure) {
        *need = A.off + 256;
        return MOT_OK;
    }
    if (!x_src || !x_tgt || !alpha || !beta || !ws) return MOT_EINVAL;
    if (A.off > ws_bytes) return MOT_ENOMEM;
    CK(cudaMemsetAsync(F.err, 0, sizeof(int) * 4, st));
    std::vector<PrepSet> sets = {prepset_of(F.src, x_src, nullptr), prepset_of(F.tgt, x_tgt, nullptr)};
    GridChoice g;
    RET(measure_and_choose(sets, F.d_sets, F.box_scratch, F.box_out, d, eta, eta, o, g, st));
    if (g.n > ngmax) {
        g.n = ngmax;
        g.M = g.n / 4;
    }
    if (scale_out) *scale_out = g.s;
    F.src.maxsub = (F.src.n + mot_sub_points(d) - 1) / mot_sub_points(d) + mot_ntiles(d, g.n);
    F.tgt.maxsub = (F.tgt.n + mot_sub_points(d) - 1) / mot_sub_points(d) + mot_ntiles(d, g.n);
    sets = {prepset_of(F.src, x_src, nullptr), prepset_of(F.tgt, x_tgt, nullptr)};
    CK(cudaMemcpyAsync(F.d_sets, sets.data(), sizeof(PrepSet) * 2, cudaMemcpyHostToDevice, st));
    CK(launch_prep(F.d_sets, sets.data(), 2, d, g.n, g.c, g.s, F.err, st));
    const double eta_n = eta / (g.s * g.s);
    size_t gsz = 1;
    for (int t = 0; t < d; ++t) gsz *= g.n;
    // d = 2 on grids of up to 64 with sets of up to 32768 points: the exact trigonometric sums in
    // one cluster per right-hand side (ndft2d.cu) instead of spread / FFT / gather
    bool nd = false;
    if (o.path == MOT_PATH_NFFT && d == 2 && o.ndft > 0 && g.M <= 16 && n_src <= fused2d_max_points() &&
        n_tgt <= fused2d_max_points()) {
        CK(prepare_ndft2d());
        nd = ndft2d_supported(d, g.M);
    }
    if (o.path == MOT_PATH_NFFT) {
        CK(prepare_window());
        CK(prepare_fftconv(d, g.n));
        RET(make_D_for(eta_n, g, d, o, F.dscr_a, F.dscr_b, F.D, st, !nd));
        for (int r = 0; r < nrhs; ++r) CK(cudaMemsetAsync(F.grid[r], 0, gsz * sizeof(float), st));
    } else if (o.path == MOT_PATH_DENSE) {
        for (int r = 0; r < nrhs; ++r) CK(cudaMemsetAsync(F.raw[r], 0, sizeof(float) * n_tgt, st));
    }
    for (int r = 0; r < nrhs; ++r)
        CK(launch_permute_in(alpha + (size_t)r * n_src, F.src.perm, (int)n_src, F.a_sorted + (size_t)r * n_src, st));
    std::vector<Task> tasks(nrhs);
    for (int r = 0; r < nrhs; ++r) {
        Task t = blank_task();
        t.src = pointset_of(F.src);
        t.alpha = F.a_sorted + (size_t)r * n_src;
        t.grid = F.grid[r];
        t.hgrid = F.hgrid[r];
        t.spec = F.spec[r];
        t.D = F.D;
        t.raw = F.raw[r];
        t.eta_u = (float)(eta_n * (double)g.n * (double)g.n);
        t.tgt = pointset_of(F.tgt);
        t.mode = EPI_RAW;
        t.out = F.b_sorted + (size_t)r * n_tgt;
        tasks[r] = t;
    }
    CK(cudaMemcpyAsync(F.d_tasks, tasks.data(), sizeof(Task) * nrhs, cudaMemcpyHostToDevice, st));
    Globals G;
    G.iter = F.iter;
    G.acc = F.acc;
    G.R = 2;
    G.floor_ = 0.f;
    G.n_grid = g.n;
    G.M = g.M;
    G.fac = nullptr;
    if (nd) {
        CK(launch_ndft2d(F.d_tasks, nrhs, G, st, false));
    } else if (o.path == MOT_PATH_NFFT) {
        int gx = std::min(F.src.maxsub, 1024), gt = std::min(F.tgt.maxsub, 1024);
        CK(launch_spread(d, F.d_tasks, nrhs, gx, G, st));
        CK(launch_fftconv(d, F.d_tasks, nrhs, G, st, nullptr));
        CK(launch_gather(d, F.d_tasks, nrhs, gt, G, st));
    } else if (o.path == MOT_PATH_DENSE_BF16X3) {
        const int ld = tc_ld((int)n_src);
        CK(prepare_tc_gemm());
        CK(launch_kernel_split(F.tgt.u, (int)n_tgt, F.src.u, (int)n_src, d, (float)(eta_n * (double)g.n * (double)g.n),
                               ld, F.kt_hi, F.kt_lo, st));
        CK(launch_split_src(F.a_sorted, nullptr, nullptr, nullptr, (int)n_src, nrhs, ld, F.a_hi, F.a_lo, st));
        TcGemm tg;
        if (!tc_prepare(&tg, F.a_hi, F.a_lo, nrhs, ld, F.kt_hi, F.kt_lo, (int)n_tgt, ld, (int)n_src)) return MOT_ECUDA;
        TcEpi ep;
        std::memset(&ep, 0, sizeof(ep));
        ep.out = F.b_sorted;
        ep.ldo = n_tgt;
        ep.mode = 0;
        ep.err = F.err;
        CK(launch_tc_gemm(tg, ep, st));
    } else {
        int ntb = (int)((n_tgt + 511) / 512);
        int split = std::max(1, std::min(64, 4 * 152 / std::max(1, ntb * nrhs)));
        CK(launch_dense(d, F.d_tasks, nrhs, ntb, split, G, st));
        CK(launch_epi(d, F.d_tasks, nrhs, std::min((int)((n_tgt + 255) / 256), 1024), G, st));
    }
    for (int r = 0; r < nrhs; ++r)
        CK(launch_permute_out(F.b_sorted + (size_t)r * n_tgt, F.tgt.perm, (int)n_tgt, beta + (size_t)r * n_tgt, st));
    int err = 0;
    CK(cudaMemcpyAsync(&err, F.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (err) return (err & 4) ? MOT_ETIMEOUT : MOT_ENUMERIC;
    return MOT_OK;
}

}  // namespace

// =============================================================================================
// C ABI
// =============================================================================================
extern "C" {

void mot_options_default(mot_options* o) {
    if (!o) return;
    fill_defaults(*o, nullptr);
    o->n_grid = 0;
}

const char* mot_strerror(int s) {
    switch (s) {
    case MOT_OK: return "ok";
    case MOT_EINVAL: return "invalid argument";
    case MOT_ENOTTREE: return "edges do not form a tree";
    case MOT_ENOMEM: return "workspace too small";
    case MOT_ENUMERIC: return "non-finite input or negative weight";
    case MOT_ENOCONV: return "stop test not met within max_iter";
    case MOT_ETIMEOUT: return "bounded device wait timed out";
    case MOT_ECUDA: return "CUDA runtime error";
    case MOT_EUNSUPPORTED: return "unsupported request";
    default: return "unknown status";
    }
}

const char* mot_last_cuda_error(void) { return g_cuda_err.c_str(); }

int mot_abi_version(void) { return MOT_ABI_VERSION; }

int mot_test_wave_clusters(int nclusters) {
    if (nclusters < 0 || nclusters > 1024) return MOT_EINVAL;
    g_wave_clusters_override.store(nclusters);
    return MOT_OK;
}

void mot_struct_sizes(size_t out[4]) {
    if (!out) return;
    out[0] = sizeof(mot_problem);
    out[1] = sizeof(mot_options);
    out[2] = sizeof(mot_result);
    out[3] = sizeof(mot_server_result);
}

int mot_wave_schedule(int K, const int* parent, int S, int cap, int* tF, int* tB, int* tR, int* carrier,
                      int* nlaunch) {
    if (!tF || !tB || !tR || !carrier || !nlaunch) return MOT_EINVAL;
    return wave_times(K, parent, S, cap, tF, tB, tR, carrier, nlaunch);
}

int mot_boundary_poly(double eta, double tau, double eps_B, int p, double* coef) {
    if (!coef || !(eta > 0.0) || p < 1 || p > 8 || !(eps_B > 0.0) || !(eps_B < tau)) return MOT_EINVAL;
    return boundary_poly(eta, tau, eps_B, p, coef) ? MOT_OK : MOT_ENUMERIC;
}

int mot_plan_grid(int d, double radius, double eta_min, double eta_max, int n_grid, double eps_B, int* n_out,
                  double* scale_out, double* err_exp_out) {
    if (d < 1 || d > 3 || !(radius >= 0.0) || !(eta_min > 0.0) || !(eta_max >= eta_min) || !(eps_B > 0.0) ||
        !(eps_B < kTau) || !n_out || !scale_out || !err_exp_out)
        return MOT_EINVAL;
    if (n_grid && (n_grid < 16 || n_grid > max_grid(d) || (n_grid & (n_grid - 1)))) return MOT_EINVAL;
    const GridChoice g = choose_grid(d, radius, eta_min, eta_max, n_grid, eps_B);
    *n_out = g.n;
    *scale_out = g.s;
    *err_exp_out = g.err_exp;
    return MOT_OK;
}

int mot_workspace_bytes(const mot_problem* prob, const mot_options* opt, size_t* bytes) {
    if (!bytes) return MOT_EINVAL;
    RET(validate_problem(prob));
    mot_options o;
    fill_defaults(o, opt);
    if (o.n_grid && (o.n_grid < 16 || o.n_grid > max_grid(prob->d) || (o.n_grid & (o.n_grid - 1)))) return MOT_EINVAL;
    if (o.m != 4) return MOT_EUNSUPPORTED;
    if (o.path == MOT_PATH_LOCAL) {
        if (prob->topology != MOT_TREE) return MOT_EUNSUPPORTED;
        LocalPlan L;
        return local_setup(prob, o, L, nullptr, 0, true, bytes, nullptr);
    }
    if (prob->topology == MOT_CIRCLE) {
        CirclePlan C;
        return circle_setup(prob, o, C, nullptr, 0, true, bytes, nullptr);
    }
    TreePlan T;
    return tree_plan_setup(prob, o, T, nullptr, 0, true, bytes, nullptr);
}

int mot_solve(const mot_problem* prob, const mot_options* opt, void* ws, size_t ws_bytes,
              const double* const* u_warm, mot_result* res, void* stream) {
    g_cuda_err.clear();
    RET(validate_problem(prob));
    mot_options o;
    fill_defaults(o, opt);
    if (o.n_grid && (o.n_grid < 16 || o.n_grid > max_grid(prob->d) || (o.n_grid & (o.n_grid - 1)))) return MOT_EINVAL;
    if (o.m != 4) return MOT_EUNSUPPORTED;
    if (!ws) return MOT_EINVAL;
    if (reinterpret_cast<uintptr_t>(ws) & 255) return MOT_EINVAL;
    if (res && res->pair && prob->topology != MOT_CIRCLE) return MOT_EINVAL;
    if (res) {
        double* const* u = res->u;
        double* const* pair = res->pair;
        std::memset(res, 0, sizeof(*res));
        *const_cast<double* const**>(&res->u) = u;
        *const_cast<double* const**>(&res->pair) = pair;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // The legacy default stream cannot be captured into a graph: run on a private stream
    // ordered after / before the caller's work by events.
    cudaStream_t own = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    if (st == nullptr && o.use_graphs > 0) {
        CK(cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&ev_out, cudaEventDisableTiming));
        CK(cudaEventRecord(ev_in, nullptr));
        CK(cudaStreamWaitEvent(own, ev_in, 0));
    }
    int rc = solve_blocking(prob, o, ws, ws_bytes, u_warm, res, own ? own : st);
    if (own) {
        cudaEventRecord(ev_out, own);
        cudaStreamWaitEvent(nullptr, ev_out, 0);
        cudaStreamSynchronize(own);
        cudaEventDestroy(ev_in);
        cudaEventDestroy(ev_out);
        cudaStreamDestroy(own);
    }
    if (res) res->status = rc;
    return rc;
}

int mot_fastsum_workspace_bytes(int d, int64_t n_src, int64_t n_tgt, int nrhs, const mot_options* opt,
                                size_t* bytes) {
    if (!bytes) return MOT_EINVAL;
    mot_options o;
    fill_defaults(o, opt);
    return fastsum_impl(d, 1.0, nullptr, n_src, nullptr, n_tgt, nullptr, nrhs, nullptr, o, nullptr, 0, nullptr,
                        nullptr, true, bytes);
}

int mot_fastsum(int d, double eta, const float* x_src, int64_t n_src, const float* x_tgt, int64_t n_tgt,
                const float* alpha, int nrhs, float* beta, const mot_options* opt, void* ws, size_t ws_bytes,
                double* scale_out, void* stream) {
    g_cuda_err.clear();
    mot_options o;
    fill_defaults(o, opt);
    if (reinterpret_cast<uintptr_t>(ws) & 255) return MOT_EINVAL;
    return fastsum_impl(d, eta, x_src, n_src, x_tgt, n_tgt, alpha, nrhs, beta, o, ws, ws_bytes, scale_out,
                        reinterpret_cast<cudaStream_t>(stream), false, nullptr);
}


int mot_server_create(void* pool, size_t pool_bytes, int max_active, mot_server* out) {
    if (!out || !pool || pool_bytes < 4096 || max_active < 1 || max_active > 256) return MOT_EINVAL;
    if (reinterpret_cast<uintptr_t>(pool) & 255) return MOT_EINVAL;
    mot_server_s* S = new mot_server_s();
    S->base = reinterpret_cast<char*>(pool);
    S->pool.init(pool_bytes);
    S->max_active = max_active;
    S->t0 = std::chrono::steady_clock::now();
    for (int i = 0; i < max_active; ++i) {
        cudaStream_t st = nullptr;
        char* h = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaHostAlloc(reinterpret_cast<void**>(&h), kSlotStats, cudaHostAllocDefault) != cudaSuccess) {
            set_cuda_error(cudaGetLastError(), "mot_server_create");
            mot_server_destroy(S);
            return MOT_ECUDA;
        }
        S->streams.push_back(st);
        S->pinned.push_back(h);
        S->slot_busy.push_back(false);
    }
    *out = S;
    return MOT_OK;
}

int mot_server_submit(mot_server S, const mot_problem* prob, const mot_options* opt, double* const* u, long long tag) {
    if (!S) return MOT_EINVAL;
    RET(validate_problem(prob));
    Request q;
    q.tag = tag;
    fill_defaults(q.o, opt);
    if (q.o.m != 4 || q.o.timing) return MOT_EUNSUPPORTED;
    const int K = prob->K;
    q.n.assign(prob->n, prob->n + K);
    q.x.assign(prob->x, prob->x + K);
    q.mu.assign(prob->mu, prob->mu + K);
    if (prob->topology == MOT_TREE) q.edges.assign(prob->edges, prob->edges + 2 * (K - 1));
    const int ne = prob->topology == MOT_TREE ? K - 1 : K;
    if (prob->edge_w) q.w.assign(prob->edge_w, prob->edge_w + ne);
    if (prob->free_nodes) q.freen.assign(prob->free_nodes, prob->free_nodes + K);
    if (u) q.u.assign(u, u + K);
    q.prob = *prob;
    q.prob.n = q.n.data();
    q.prob.x = q.x.data();
    q.prob.mu = q.mu.data();
    q.prob.edges = q.edges.empty() ? nullptr : q.edges.data();
    q.prob.edge_w = q.w.empty() ? nullptr : q.w.data();
    q.prob.free_nodes = q.freen.empty() ? nullptr : q.freen.data();
    RET(mot_workspace_bytes(&q.prob, &q.o, &q.ws_bytes));
    q.t_submit = S->now();
    S->pending.push_back(std::move(q));
    // the vectors moved with the request: re-point the problem at the stored copies
    Request& b = S->pending.back();
    b.prob.n = b.n.data();
    b.prob.x = b.x.data();
    b.prob.mu = b.mu.data();
    b.prob.edges = b.edges.empty() ? nullptr : b.edges.data();
    b.prob.edge_w = b.w.empty() ? nullptr : b.w.data();
    b.prob.free_nodes = b.freen.empty() ? nullptr : b.freen.data();
    return MOT_OK;
}

int mot_server_progress(mot_server S, int* n_active, int* n_pending) {
    if (!S) return MOT_EINVAL;
    // 1. advance active solves whose last chunk completed
    for (size_t i = 0; i < S->active.size();) {
        Active* a = S->active[i];
        cudaError_t q = cudaEventQuery(a->solve.ev);
        if (q == cudaErrorNotReady) {
            ++i;
            continue;
        }
        int rc = q == cudaSuccess ? MOT_OK : MOT_ECUDA;
        if (rc != MOT_OK) set_cuda_error(q, "mot_server_progress");
        bool complete = false;
        if (rc == MOT_OK && a->finishing) {
            complete = true;
        } else if (rc == MOT_OK) {
            rc = a->solve.evaluate(&a->res);
            if (rc == MOT_OK && !a->solve.done) {
                rc = a->solve.launch();
            } else if (rc == MOT_OK) {
                rc = a->solve.finish(&a->res, a->req.u.empty() ? nullptr : a->req.u.data(), nullptr);
                if (rc == MOT_OK && cudaEventRecord(a->solve.ev, a->solve.st) != cudaSuccess) rc = MOT_ECUDA;
                a->finishing = true;
            }
        }
        if (rc != MOT_OK || complete) {
            cudaStreamSynchronize(a->solve.st);
            server_complete(S, a, rc != MOT_OK ? rc : a->solve.status);
            S->active.erase(S->active.begin() + i);
            continue;
        }
        ++i;
    }
    // 2. admit pending requests in arrival order while a slot and pool memory are free
    while (!S->pending.empty() && (int)S->active.size() < S->max_active) {
        Request& q = S->pending.front();
        if (q.ws_bytes > S->pool.size) {
            server_reject(S, q, MOT_ENOMEM);
            S->pending.pop_front();
            continue;
        }
        size_t off = 0;
        if (!S->pool.alloc(q.ws_bytes, &off)) break;          // wait for memory to free up
        int slot = 0;
        while (S->slot_busy[slot]) ++slot;
        Active* a = new Active();
        a->req = std::move(q);
        S->pending.pop_front();
        Request& r = a->req;
        r.prob.n = r.n.data();
        r.prob.x = r.x.data();
        r.prob.mu = r.mu.data();
        r.prob.edges = r.edges.empty() ? nullptr : r.edges.data();
        r.prob.edge_w = r.w.empty() ? nullptr : r.w.data();
        r.prob.free_nodes = r.freen.empty() ? nullptr : r.freen.data();
        a->off = off;
        a->slot = slot;
        S->slot_busy[slot] = true;
        a->t_admit = S->now();
        std::memset(&a->res, 0, sizeof(a->res));
        Solve& sv = a->solve;
        sv.o = r.o;
        sv.st = S->streams[slot];
        sv.hstats = S->pinned[slot];
        int rc = cudaEventCreateWithFlags(&sv.ev, cudaEventDisableTiming) == cudaSuccess ? MOT_OK : MOT_ECUDA;
        if (rc == MOT_OK) rc = make_ops(&r.prob, r.o, S->base + off, r.ws_bytes, sv.st, &sv.ops);
        if (rc == MOT_OK && sv.ops->stats_bytes() > kSlotStats) rc = MOT_EUNSUPPORTED;
        if (rc == MOT_OK) rc = sv.start(nullptr);
        if (rc == MOT_OK) rc = sv.launch();
        if (rc != MOT_OK) {
            cudaStreamSynchronize(sv.st);
            server_complete(S, a, rc);
            continue;
        }
        S->active.push_back(a);
    }
    if (n_active) *n_active = (int)S->active.size();
    if (n_pending) *n_pending = (int)S->pending.size();
    return MOT_OK;
}

int mot_server_poll(mot_server S, mot_server_result* out, int max, int* n_out) {
    if (!S || !n_out || (max > 0 && !out)) return MOT_EINVAL;
    const int n = std::min<int>(max, (int)S->done.size());
    for (int i = 0; i < n; ++i) out[i] = S->done[i];
    S->done.erase(S->done.begin(), S->done.begin() + n);
    *n_out = n;
    return MOT_OK;
}

int mot_server_destroy(mot_server S) {
    if (!S) return MOT_EINVAL;
    for (Active* a : S->active) {
        cudaStreamSynchronize(a->solve.st);
        if (a->solve.ev) cudaEventDestroy(a->solve.ev);
        delete a->solve.ops;
        delete a;
    }
    for (auto st : S->streams) cudaStreamDestroy(st);
    for (auto h : S->pinned) cudaFreeHost(h);
    delete S;
    return MOT_OK;
}

}  // extern "C"
