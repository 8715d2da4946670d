"""Dense FP64 Sinkhorn for tree- and circle-structured multi-marginal OT.

Test infrastructure only (see ``oracle/__init__.py``).

Paper passages followed:
  * Section 3, Eq. (Pk): marginal projection P_k; Theorem 3.1, Eq. (dual_problem):
    Sinkhorn function S; Proposition 3.2: optimal plan K (.) Phi;
    Algorithm 1: Sinkhorn for a general cost (used here only by brute force).
  * Section 4, Eqs. (cost_sparse), (K-sparse), (K-matrix): graph-structured kernel.
  * Section 4.1: tree notation (root 1, parent p(k) < k, children C_k, leaves);
    Theorem 4.1 (tree marginals), the beta / gamma recursions (Eq. gamma_tree,
    Eq. comp_wise_multi_beta_tree) and Algorithm 2.
  * Section 4.2: circle; Theorems 4.2 / 4.3, the alpha / lambda matrix
    recursions and Algorithm 3.
  * Section 6.3 (generalised Euler flows): the circle whose closing edge
    {K, 1} compares x^K with sigma(x^1), and the pair marginals Pi_{1,k}.
  * Section 6.1, closing remark (small eta): Algorithm 2 in the log domain,
    optionally with every kernel sum truncated to nearby pairs.

Conventions: node labels are 0-based (the paper's node 1 is label 0).  A
problem's edge list may use any labels; :func:`tree_structure` relabels by
breadth-first search from the root so that p(k) < k, as the paper assumes
without loss of generality.

Readings of passages that are silent or ambiguous:
  * Initial scalings phi^(0) = 1 (the paper leaves the value open).
  * Algorithm 1 increments r inside the loop over k; the reading is one
    increment per sweep over all K marginals.
  * Algorithm 2 computes gamma_k from the siblings' beta of the previous sweep
    (implemented literally: for a star, the siblings' messages are stale).
  * S^(r) in Algorithms 2 and 3 uses phi^(r) and phi^{1,(r+1)}; the term
    (mu^1 / phi^{1,(r+1)})^T phi^{1,(r)} equals the total mass of K (.) Phi^(r),
    so S^(r) = S(phi^(r)) of Eq. (dual_problem).
  * Edge weights w_e (Section 6.2) scale the squared distance of edge e.
"""
from __future__ import annotations

import math
from collections import deque
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from .kernel import kernel_matrix, direct_sum, log_kernel_sum


# ---------------------------------------------------------------------------
# edge kernels
# ---------------------------------------------------------------------------

class EdgeKernel:
    """K^{(a,b)}_{ij} = exp(-w ||x^a_i - x^b_j||^2 / eta) (Eq. K-matrix).

    Dense when small; otherwise applied block by block by direct summation.
    """

    DENSE_LIMIT = 16_000_000

    def __init__(self, xa: np.ndarray, xb: np.ndarray, eta: float, w: float = 1.0):
        self.xa = np.asarray(xa, dtype=np.float64)
        self.xb = np.asarray(xb, dtype=np.float64)
        self.eta_eff = eta / w if w != 0 else np.inf
        self.w = w
        self.shape = (self.xa.shape[0], self.xb.shape[0])
        self.mat = None
        if self.shape[0] * self.shape[1] <= self.DENSE_LIMIT:
            self.mat = self.dense()

    def dense(self) -> np.ndarray:
        if self.mat is not None:
            return self.mat
        if self.w == 0:
            return np.ones(self.shape)
        return kernel_matrix(self.xa, self.xb, self.eta_eff)

    def matvec(self, v: np.ndarray) -> np.ndarray:
        """K v (v over the columns' points)."""
        if self.mat is not None:
            return self.mat @ v
        if self.w == 0:
            return np.broadcast_to(v.sum(axis=0), (self.shape[0],) + v.shape[1:]).copy()
        return direct_sum(self.xa, self.xb, v, self.eta_eff)

    def rmatvec(self, v: np.ndarray) -> np.ndarray:
        """K^T v (v over the rows' points)."""
        if self.mat is not None:
            return self.mat.T @ v
        if self.w == 0:
            return np.broadcast_to(v.sum(axis=0), (self.shape[1],) + v.shape[1:]).copy()
        return direct_sum(self.xb, self.xa, v, self.eta_eff)


# ---------------------------------------------------------------------------
# tree structure (Section 4.1)
# ---------------------------------------------------------------------------

@dataclass
class Tree:
    K: int
    order: List[int]            # new label -> original node id
    new_of: List[int]           # original node id -> new label
    parent: List[int]           # parent[k] (new labels), parent[0] = -1
    children: List[List[int]]   # C_k (new labels, increasing)
    weight: List[float]         # weight of edge {p(k), k}; weight[0] unused

    @property
    def leaves(self) -> List[int]:
        # L = nodes with exactly one neighbour
        out = []
        for k in range(self.K):
            deg = len(self.children[k]) + (1 if self.parent[k] >= 0 else 0)
            if deg == 1:
                out.append(k)
        return out


def tree_structure(K: int, edges, root: int = 0, edge_w: Optional[Sequence[float]] = None) -> Tree:
    """Relabel a tree by BFS from ``root`` so that p(k) < k (Section 4.1).

    Raises ValueError if the edges do not form a tree on K nodes.
    """
    edges = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    if edges.shape[0] != K - 1:
        raise ValueError("a tree on K nodes has K-1 edges")
    adj: Dict[int, List[Tuple[int, float]]] = {k: [] for k in range(K)}
    for e, (a, b) in enumerate(edges):
        w = 1.0 if edge_w is None else float(edge_w[e])
        if not (0 <= a < K and 0 <= b < K) or a == b:
            raise ValueError("bad edge")
        adj[int(a)].append((int(b), w))
        adj[int(b)].append((int(a), w))
    order = [root]
    new_of = [-1] * K
    new_of[root] = 0
    parent = [-1]
    weight = [0.0]
    q = deque([root])
    while q:
        u = q.popleft()
        for v, w in sorted(adj[u]):
            if new_of[v] < 0:
                new_of[v] = len(order)
                order.append(v)
                parent.append(new_of[u])
                weight.append(w)
                q.append(v)
    if len(order) != K:
        raise ValueError("edges do not connect all K nodes")
    children: List[List[int]] = [[] for _ in range(K)]
    for k in range(1, K):
        children[parent[k]].append(k)
    return Tree(K, order, new_of, parent, children, weight)


def _prod(vecs, n):
    out = np.ones(n)
    for v in vecs:
        out = out * v
    return out


# ---------------------------------------------------------------------------
# Algorithm 2: tree
# ---------------------------------------------------------------------------

@dataclass
class SolveResult:
    phi: List[np.ndarray]               # scalings in the caller's labels
    S: List[float] = field(default_factory=list)   # S^(r), r = 0..iters-1
    iters: int = 0


class TreeSinkhorn:
    """Algorithm 2 with dense FP64 kernel matrix-vector products.

    The state (phi, beta) lives in BFS labels; inputs and outputs use the
    caller's labels.
    """

    def __init__(self, x: Sequence[np.ndarray], mu: Sequence[np.ndarray], edges, eta: float,
                 root: int = 0, edge_w=None):
        self.K = len(x)
        self.tree = tree_structure(self.K, edges, root, edge_w)
        t = self.tree
        self.eta = float(eta)
        self.x = [np.asarray(x[t.order[k]], dtype=np.float64) for k in range(self.K)]
        self.mu = [np.asarray(mu[t.order[k]], dtype=np.float64) for k in range(self.K)]
        self.n = [xi.shape[0] for xi in self.x]
        # K^{(p(k),k)} in ℝ^{n_{p(k)} x n_k}
        self.Kpk = [None] + [EdgeKernel(self.x[t.parent[k]], self.x[k], eta, t.weight[k])
                             for k in range(1, self.K)]

    # -- message pieces ----------------------------------------------------
    def beta_prod(self, beta, k, exclude=None):
        """beta^{(.) U} of Eq. (comp_wise_multi_beta_tree) with U = C_k minus ``exclude``."""
        return _prod([beta[t] for t in self.tree.children[k] if t != exclude], self.n[k])

    def compute_beta(self, phi, beta, k):
        """beta_k = K^{(p(k),k)} (phi^k (.) beta^{(.) C_k}) (Algorithm 2, step 4)."""
        return self.Kpk[k].matvec(phi[k] * self.beta_prod(beta, k))

    def compute_gamma(self, phi, beta, gamma, k):
        """gamma_k = (K^{(p(k),k)})^T (phi^{p(k)} (.) gamma_{p(k)} (.) beta^{(.) C_{p(k)} minus k}) (Eq. gamma_tree)."""
        p = self.tree.parent[k]
        return self.Kpk[k].rmatvec(phi[p] * gamma[p] * self.beta_prod(beta, p, exclude=k))

    def init_beta(self, phi):
        beta = [None] * self.K
        for k in range(self.K - 1, 0, -1):
            beta[k] = self.compute_beta(phi, beta, k)
        return beta

    def to_user(self, vecs):
        out = [None] * self.K
        for k in range(self.K):
            out[self.tree.order[k]] = vecs[k]
        return out

    def from_user(self, vecs):
        return [np.asarray(vecs[self.tree.order[k]], dtype=np.float64) for k in range(self.K)]

    # -- Algorithm 2 ---------------------------------------------------------
    def run(self, iters: int, phi0=None, free_nodes: Sequence[int] = (), delta: float = 0.0,
            callback=None) -> SolveResult:
        """Run ``iters`` sweeps of Algorithm 2 (or stop when |S^(r) - S^(r-1)| < delta).

        ``free_nodes`` (caller labels) get phi = 1 in every sweep: the
        barycenter modification of Section 6.2 (nodes without a marginal
        constraint).
        """
        K = self.K
        phi = [np.ones(n) for n in self.n] if phi0 is None else self.from_user(phi0)
        free = {self.tree.new_of[k] for k in free_nodes}
        beta = self.init_beta(phi)                               # steps 3-5
        S_trace = []
        r = 0
        while r < iters:
            gamma = [None] * K
            phi_new = [None] * K
            for k in range(K):                                   # steps 7-13
                if k == 0:
                    gamma[0] = np.ones(self.n[0])
                else:
                    gamma[k] = self.compute_gamma(phi_new, beta, gamma, k)
                if k in free:
                    phi_new[k] = np.ones(self.n[k])
                else:
                    phi_new[k] = self.mu[k] / (gamma[k] * self.beta_prod(beta, k))
            if 0 in free:
                # phi^1 is pinned to 1, so mu^1 / phi^{1,(r+1)} is not the root's message
                # product; read the mass of K (.) Phi^(r) off the root directly.
                mass = float(np.dot(phi[0], self.beta_prod(beta, 0)))
            else:
                mass = float(np.dot(self.mu[0] / phi_new[0], phi[0]))   # step 16 (second term)
            S = self.eta * (sum(float(np.dot(self.mu[k], np.log(phi[k]))) for k in range(K) if k not in free)
                            - mass)
            for k in range(K - 1, 0, -1):                        # steps 14-15
                beta[k] = self.compute_beta(phi_new, beta, k)
            phi = phi_new
            S_trace.append(S)
            r += 1
            if callback is not None:
                callback(r, self.to_user(phi))
            if delta > 0 and len(S_trace) >= 2 and abs(S_trace[-1] - S_trace[-2]) < delta:
                break
        return SolveResult(self.to_user(phi), S_trace, r)


def tree_marginals(x, phi, edges, eta, root: int = 0, edge_w=None) -> List[np.ndarray]:
    """Theorem 4.1: P_k(K (.) Phi) = phi^k (.) gamma_k (.) beta^{(.) C_k} for arbitrary phi.

    beta by the upward recursion and gamma by the downward one (Section 4.1),
    with exact FP64 kernels.  Caller labels in and out.
    """
    ts = TreeSinkhorn(x, [np.ones(len(a)) for a in x], edges, eta, root, edge_w)
    ph = ts.from_user(phi)
    beta = ts.init_beta(ph)
    gamma = [np.ones(ts.n[0])] + [None] * (ts.K - 1)
    for k in range(1, ts.K):
        gamma[k] = ts.compute_gamma(ph, beta, gamma, k)
    P = [ph[k] * gamma[k] * ts.beta_prod(beta, k) for k in range(ts.K)]
    return ts.to_user(P)


# ---------------------------------------------------------------------------
# Algorithm 2 in the log domain (small eta, truncated kernel sums)
# ---------------------------------------------------------------------------

@dataclass
class LogSolveResult:
    logphi: List[np.ndarray]            # log phi^k in the caller's labels
    S: List[float] = field(default_factory=list)
    iters: int = 0


def _logsumexp(v: np.ndarray) -> float:
    m = float(np.max(v))
    if not np.isfinite(m):
        return m
    return m + math.log(float(np.exp(v - m).sum()))


class TreeSinkhornLog:
    """Algorithm 2 with every scaling and message held as its logarithm, FP64.

    f^k = log phi^k, b_k = log beta_k, g_k = log gamma_k.  Each kernel product
    of Algorithm 2 becomes a log-sum-exp (``log_kernel_sum``), each
    element-wise product a sum and each quotient a difference, in the same
    order, so the iterates are those of ``TreeSinkhorn`` wherever both are
    representable.  For small eta the scalings grow like exp(+-cost / eta) and
    leave the floating-point range; their logarithms do not.  ``r_cut``
    truncates every kernel sum to the pairs within that distance, the
    truncation the paper suggests for very small eta.
    """

    def __init__(self, x: Sequence[np.ndarray], mu: Sequence[np.ndarray], edges, eta: float,
                 root: int = 0, edge_w=None, r_cut: Optional[float] = None):
        self.K = len(x)
        self.tree = tree_structure(self.K, edges, root, edge_w)
        t = self.tree
        self.eta = float(eta)
        self.x = [np.asarray(x[t.order[k]], dtype=np.float64).reshape(len(x[t.order[k]]), -1)
                  for k in range(self.K)]
        self.mu = [np.asarray(mu[t.order[k]], dtype=np.float64) for k in range(self.K)]
        with np.errstate(divide="ignore"):
            self.logmu = [np.log(m) for m in self.mu]
        self.n = [xi.shape[0] for xi in self.x]
        self.r_cut = r_cut
        # kernel exp(-w ||.||^2 / eta) of edge {p(k), k} as exp(-||.||^2 / eta_e)
        self.eta_e = [None] + [self.eta / t.weight[k] if t.weight[k] != 0 else np.inf for k in range(1, self.K)]

    def _sum_b(self, b, k, exclude=None):
        """log beta^{(.) U}, U = C_k minus ``exclude``."""
        out = np.zeros(self.n[k])
        for t in self.tree.children[k]:
            if t != exclude:
                out = out + b[t]
        return out

    def compute_b(self, f, b, k):
        """log beta_k = log K^{(p(k),k)} exp(f^k + log beta^{(.) C_k}) (Algorithm 2, step 4)."""
        p = self.tree.parent[k]
        return log_kernel_sum(self.x[p], self.x[k], f[k] + self._sum_b(b, k), self.eta_e[k], self.r_cut)

    def compute_g(self, f, b, g, k):
        """log gamma_k = log (K^{(p(k),k)})^T exp(f^{p(k)} + log gamma_{p(k)} + log beta^{(.) C_{p(k)} minus k})."""
        p = self.tree.parent[k]
        return log_kernel_sum(self.x[k], self.x[p], f[p] + g[p] + self._sum_b(b, p, exclude=k), self.eta_e[k],
                              self.r_cut)

    def to_user(self, vecs):
        out = [None] * self.K
        for k in range(self.K):
            out[self.tree.order[k]] = vecs[k]
        return out

    def from_user(self, vecs):
        return [np.asarray(vecs[self.tree.order[k]], dtype=np.float64) for k in range(self.K)]

    def init_b(self, f):
        b = [None] * self.K
        for k in range(self.K - 1, 0, -1):
            b[k] = self.compute_b(f, b, k)
        return b

    def run(self, iters: int, logphi0=None, callback=None) -> LogSolveResult:
        K = self.K
        f = [np.zeros(n) for n in self.n] if logphi0 is None else self.from_user(logphi0)
        b = self.init_b(f)                                            # steps 3-5
        S_trace = []
        for r in range(iters):
            g = [None] * K
            fn = [None] * K
            for k in range(K):                                       # steps 7-13
                g[k] = np.zeros(self.n[0]) if k == 0 else self.compute_g(fn, b, g, k)
                fn[k] = self.logmu[k] - g[k] - self._sum_b(b, k)
            mass = math.exp(_logsumexp(f[0] + self._sum_b(b, 0)))   # mass of K (.) Phi^(r)
            S = self.eta * (sum(float(np.sum(np.where(m > 0, m * fk, 0.0))) for m, fk in zip(self.mu, f)) - mass)
            for k in range(K - 1, 0, -1):                            # steps 14-15
                b[k] = self.compute_b(fn, b, k)
            f = fn
            S_trace.append(S)
            if callback is not None:
                callback(r + 1, self.to_user(f))
        return LogSolveResult(self.to_user(f), S_trace, iters)


def tree_marginals_log(x, logphi, edges, eta, root: int = 0, edge_w=None, r_cut: Optional[float] = None):
    """Theorem 4.1 in the log domain: log P_k = f^k + log gamma_k + log beta^{(.) C_k}, for any
    f = log phi (caller labels in and out); with ``r_cut`` the marginals of the truncated kernel."""
    ts = TreeSinkhornLog(x, [np.ones(len(a)) for a in x], edges, eta, root, edge_w, r_cut)
    f = ts.from_user(logphi)
    b = ts.init_b(f)
    g = [np.zeros(ts.n[0])] + [None] * (ts.K - 1)
    for k in range(1, ts.K):
        g[k] = ts.compute_g(f, b, g, k)
    return ts.to_user([f[k] + g[k] + ts._sum_b(b, k) for k in range(ts.K)])


# ---------------------------------------------------------------------------
# Algorithm 3: circle
# ---------------------------------------------------------------------------

def _row_dot(G: np.ndarray, H: np.ndarray) -> np.ndarray:
    """<G, H> = (sum_j G_ij H_ij)_i, the inner product over the second dimension (Section 4.2)."""
    return (G * H).sum(axis=1)


class CircleSinkhorn:
    """Algorithm 3 with dense FP64 matrices.

    Edges {k, k+1} for k = 1..K with K+1 = 1 (0-based: {k, (k+1) mod K}).
    ``edge_w[k]`` weights edge {k, k+1}; a zero weight makes that kernel the
    all-ones matrix.  ``x_close`` (Section 6.3) replaces the points of node 1
    on the closing edge {K, 1} only: its kernel becomes
    exp(-w ||x^K_i - x_close_j||^2 / eta), x_close = sigma(x^1) for a
    connection map sigma.
    """

    def __init__(self, x: Sequence[np.ndarray], mu: Sequence[np.ndarray], eta: float, edge_w=None,
                 x_close=None):
        self.K = len(x)
        self.eta = float(eta)
        self.x = [np.asarray(a, dtype=np.float64) for a in x]
        self.mu = [np.asarray(m, dtype=np.float64) for m in mu]
        self.n = [a.shape[0] for a in self.x]
        w = [1.0] * self.K if edge_w is None else [float(v) for v in edge_w]
        closing = self.x[0] if x_close is None else np.asarray(x_close, dtype=np.float64).reshape(self.x[0].shape)
        # Kn[k] = K^{(k, k+1)} in ℝ^{n_k x n_{k+1}}
        self.Kn = [EdgeKernel(self.x[k], closing if k == self.K - 1 else self.x[k + 1], eta, w[k]).dense()
                   for k in range(self.K)]

    def compute_betas(self, phi):
        """beta_K = K^{(K,1)}; beta_k = K^{(k,k+1)} (phi^{k+1} (.) beta_{k+1}), k = K-1..2 (steps 3-5)."""
        K = self.K
        beta = [None] * K
        beta[K - 1] = self.Kn[K - 1]
        for k in range(K - 2, 0, -1):
            beta[k] = self.Kn[k] @ (phi[k + 1][:, None] * beta[k + 1])
        return beta

    def run(self, iters: int, phi0=None, delta: float = 0.0, callback=None) -> SolveResult:
        K = self.K
        phi = [np.ones(n) for n in self.n] if phi0 is None else [np.asarray(p, dtype=np.float64) for p in phi0]
        beta = self.compute_betas(phi)
        S_trace = []
        r = 0
        while r < iters:
            phi_new = [None] * K
            # step 7: phi^1 = mu^1 / <K^{(1,2)}, (phi^2 (.) beta_2)^T>
            phi_new[0] = self.mu[0] / _row_dot(self.Kn[0], (phi[1][:, None] * beta[1]).T)
            gamma = None
            for k in range(1, K):                                # steps 8-12
                if k == 1:
                    gamma = self.Kn[0]                           # gamma_2 = K^{(1,2)}
                else:
                    gamma = gamma @ (phi_new[k - 1][:, None] * self.Kn[k - 1])
                phi_new[k] = self.mu[k] / _row_dot(beta[k], (phi_new[0][:, None] * gamma).T)
            mass = float(np.dot(self.mu[0] / phi_new[0], phi[0]))
            S = self.eta * (sum(float(np.dot(self.mu[k], np.log(phi[k]))) for k in range(K)) - mass)
            beta = self.compute_betas(phi_new)                   # steps 13-15
            phi = phi_new
            S_trace.append(S)
            r += 1
            if callback is not None:
                callback(r, phi)
            if delta > 0 and len(S_trace) >= 2 and abs(S_trace[-1] - S_trace[-2]) < delta:
                break
        return SolveResult(phi, S_trace, r)


def circle_marginals(x, phi, eta, edge_w=None, x_close=None) -> List[np.ndarray]:
    """Theorem 4.3: P_1 = phi^1 (.) <K^{(1,2)}, (phi^2 (.) alpha^{(2,1)})^T>,
    P_k = phi^k (.) <alpha^{(k,1)}, (phi^1 (.) lambda^{(1,k)})^T> for k >= 2."""
    cs = CircleSinkhorn(x, [np.ones(len(a)) for a in x], eta, edge_w, x_close)
    K = cs.K
    ph = [np.asarray(p, dtype=np.float64) for p in phi]
    alpha = cs.compute_betas(ph)                 # alpha^{(k,1)} for k = 2..K
    P = [None] * K
    P[0] = ph[0] * _row_dot(cs.Kn[0], (ph[1][:, None] * alpha[1]).T)
    lam = None
    for k in range(1, K):
        lam = cs.Kn[0] if k == 1 else lam @ (ph[k - 1][:, None] * cs.Kn[k - 1])
        P[k] = ph[k] * _row_dot(alpha[k], (ph[0][:, None] * lam).T)
    return P


def circle_pair_marginals(x, phi, eta, edge_w=None, x_close=None) -> List[Optional[np.ndarray]]:
    """Pair marginals Pi_{1,k} of K (.) Phi for a circle (Section 6.3), k = 2..K.

    Summing the plan over every index but i_1 and i_k splits the circle at
    nodes 1 and k into the chain 1 -> 2 -> ... -> k, whose summed kernel is
    lambda^{(1,k)} (Theorem 4.3's matrix, phi^2..phi^{k-1} inside), and the
    chain k -> k+1 -> ... -> K -> 1, whose summed kernel is alpha^{(k,1)}
    (phi^{k+1}..phi^K inside).  So
    Pi_{1,k}[i_1, i_k] = phi^1_{i_1} lambda^{(1,k)}[i_1, i_k] alpha^{(k,1)}[i_k, i_1] phi^k_{i_k}.
    Returns a list of K entries: [0] is None, [k] has shape (n_1, n_k).
    """
    cs = CircleSinkhorn(x, [np.ones(len(a)) for a in x], eta, edge_w, x_close)
    K = cs.K
    ph = [np.asarray(p, dtype=np.float64) for p in phi]
    alpha = cs.compute_betas(ph)
    out: List[Optional[np.ndarray]] = [None] * K
    lam = None
    for k in range(1, K):
        lam = cs.Kn[0] if k == 1 else lam @ (ph[k - 1][:, None] * cs.Kn[k - 1])
        out[k] = ph[0][:, None] * lam * alpha[k].T * ph[k][None, :]
    return out


# ---------------------------------------------------------------------------
# values of a scaling
# ---------------------------------------------------------------------------

def total_mass(P: Sequence[np.ndarray]) -> float:
    """sum_i (K (.) Phi)_i, read off any marginal."""
    return float(np.sum(P[0]))


def dual_value(mu, phi, mass, eta) -> float:
    """Eq. (dual_problem): S = eta sum_k mu^k . log phi^k - eta sum_i K_i Phi_i."""
    return float(eta * (sum(float(np.dot(m, np.log(p))) for m, p in zip(mu, phi)) - mass))


def primal_value(P, phi, mass, eta) -> float:
    """Eq. (MOTe) objective at Pi = K (.) Phi.

    With log Pi_i = -C_i/eta + sum_k log phi^k_{i_k}, <Pi, C> + eta <Pi, log Pi - 1>
    collapses to eta sum_k P_k . log phi^k - eta mass.
    """
    return float(eta * (sum(float(np.dot(Pk, np.log(p))) for Pk, p in zip(P, phi)) - mass))


def violation(P, mu) -> float:
    """max_k ||P_k - mu^k||_1."""
    return float(max(np.abs(np.asarray(Pk) - np.asarray(m)).sum() for Pk, m in zip(P, mu)))


def gauge_fix(u: Sequence[np.ndarray], mu: Sequence[np.ndarray]) -> List[np.ndarray]:
    """Remove the gauge of the dual potentials u^k = eta log phi^k.

    Adding c_k to u^k with sum_k c_k = 0 leaves K (.) Phi unchanged.  Shift
    every u^k, k >= 1 (0-based), to zero mu^k-weighted mean and give the total
    shift to u^0.
    """
    out = [np.asarray(a, dtype=np.float64).copy() for a in u]
    total = 0.0
    for k in range(1, len(out)):
        c = float(np.dot(mu[k], out[k]) / np.sum(mu[k]))
        out[k] -= c
        total += c
    out[0] += total
    return out


# ---------------------------------------------------------------------------
# brute force over the full N^K tensor (tiny cases)
# ---------------------------------------------------------------------------

def full_kernel_tensor(x, graph_edges, eta, edge_w=None, x_close=None) -> np.ndarray:
    """Eq. (cost_sparse) / Eq. (K-sparse): K_i = exp(-sum_{edges} w_e ||x^{k1}_{i_k1} - x^{k2}_{i_k2}||^2 / eta).

    Built directly from the cost tensor C (not from the factorisation), as
    the independent reference for the message-passing recursions.  With
    ``x_close`` the edge (K, 1) compares x^K with x_close in place of x^1:
    the generalised Euler-flow cost of Section 6.3 with x_close = sigma(x^1).
    """
    K = len(x)
    xs = [np.asarray(a, dtype=np.float64).reshape(len(a), -1) for a in x]
    shape = tuple(a.shape[0] for a in xs)
    C = np.zeros(shape)
    for e, (a, b) in enumerate(graph_edges):
        w = 1.0 if edge_w is None else float(edge_w[e])
        xa, xb = xs[a], xs[b]
        if x_close is not None and (a, b) == (K - 1, 0):
            xb = np.asarray(x_close, dtype=np.float64).reshape(xb.shape)
        diff = xa[:, None, :] - xb[None, :, :]
        D2 = (diff * diff).sum(axis=-1)
        sh = [1] * K
        sh[a] = shape[a]
        sh[b] = shape[b]
        if a < b:
            C = C + w * D2.reshape(sh)
        else:
            C = C + w * D2.T.reshape(sh)
    return np.exp(-C / eta)


def plan_tensor(Kt: np.ndarray, phi) -> np.ndarray:
    """Pi = K (.) Phi with Phi = phi^1 (x) ... (x) phi^K (Theorem 3.1, Proposition 3.2)."""
    P = Kt.copy()
    K = Kt.ndim
    for k in range(K):
        sh = [1] * K
        sh[k] = Kt.shape[k]
        P = P * np.asarray(phi[k], dtype=np.float64).reshape(sh)
    return P


def tensor_marginals(Pi: np.ndarray) -> List[np.ndarray]:
    """Eq. (Pk): P_k(Pi) = sum over all indices but i_k."""
    K = Pi.ndim
    return [Pi.sum(axis=tuple(a for a in range(K) if a != k)) for k in range(K)]


def tensor_pair_marginal(Pi: np.ndarray, a: int, b: int) -> np.ndarray:
    """Pi_{a,b}: the sum of Pi over all indices but i_a and i_b (a < b), shape (n_a, n_b)."""
    return Pi.sum(axis=tuple(t for t in range(Pi.ndim) if t not in (a, b)))


def sinkhorn_bruteforce(Kt: np.ndarray, mu, iters: int, phi0=None):
    """Algorithm 1 on the full tensor; returns the phi after every sweep."""
    K = Kt.ndim
    phi = [np.ones(Kt.shape[k]) for k in range(K)] if phi0 is None else [np.asarray(p, float).copy() for p in phi0]
    history = []
    for _ in range(iters):
        for k in range(K):
            Pk = tensor_marginals(plan_tensor(Kt, phi))[k]
            phi[k] = np.asarray(mu[k]) * phi[k] / Pk
        history.append([p.copy() for p in phi])
    return history


def primal_bruteforce(Kt: np.ndarray, x, graph_edges, phi, eta, edge_w=None) -> float:
    """<Pi, C> + eta <Pi, log Pi - 1> summed entry by entry over the full tensor (Eq. MOTe)."""
    Pi = plan_tensor(Kt, phi)
    C = -eta * np.log(Kt)
    return float((Pi * C).sum() + eta * (Pi * (np.log(Pi) - 1.0)).sum())
