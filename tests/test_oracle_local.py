"""Pins of the oracle's small-eta pieces (no GPU): the truncated kernel sum and Algorithm 2
in the log domain, which the paper's closing remark of Section 6.1 motivates (for very small
eta the kernel is concentrated, so its sum may be truncated to nearby pairs, and the scalings
exp(+-cost / eta) leave the floating-point range).

The truncated sum is checked against the plain sum (exact beyond the diameter, within the tail
bound otherwise) and against a loop over pairs; the log-domain sum against the plain sum and
its shift invariance; the log-domain Algorithm 2 against the scaling-form Algorithm 2 where both
are representable and, at a small eta where the scaling form breaks down, against Algorithm 1
on the full tensor written in log form from the cost (Eq. cost_sparse).
"""
import itertools
import math

import numpy as np
import pytest

from oracle import kernel as OK
from oracle import sinkhorn as OS
from paper_2208_03120_gb300 import workloads as W


def test_truncated_sum_equals_direct_beyond_the_diameter():
    rng = np.random.default_rng(1)
    x, y = rng.uniform(-0.2, 0.2, (60, 2)), rng.uniform(-0.2, 0.2, (45, 2))
    a = rng.uniform(0.1, 1.0, 45)
    np.testing.assert_allclose(OK.truncated_sum(x, y, a, 0.02, 1.0), OK.direct_sum(x, y, a, 0.02), rtol=1e-14)


@pytest.mark.parametrize("r_cut", [0.05, 0.1, 0.2])
def test_truncated_sum_within_the_tail_bound(r_cut):
    """Every left-out term is at most exp(-r_cut^2 / eta) |alpha_j|, so the truncated sum is
    below the plain one (positive weights) by at most that times sum |alpha|."""
    rng = np.random.default_rng(2)
    x, y = rng.uniform(0, 1, (80, 2)), rng.uniform(0, 1, (70, 2))
    a = rng.uniform(0.1, 1.0, 70)
    eta = 0.004
    t, d = OK.truncated_sum(x, y, a, eta, r_cut), OK.direct_sum(x, y, a, eta)
    assert np.all(t <= d * (1 + 1e-14))
    assert np.max(d - t) <= math.exp(-r_cut * r_cut / eta) * a.sum() * (1 + 1e-12)
    assert np.max(d - t) > 0.0          # something was left out


def test_truncated_sum_matches_a_loop_over_pairs():
    rng = np.random.default_rng(3)
    x, y = rng.uniform(0, 1, (7, 3)), rng.uniform(0, 1, (9, 3))
    a = rng.normal(size=9)
    eta, r = 0.05, 0.6
    ref = np.zeros(7)
    for i in range(7):
        for j in range(9):
            dist = math.sqrt(sum((x[i, t] - y[j, t]) ** 2 for t in range(3)))
            if dist <= r:
                ref[i] += a[j] * math.exp(-dist * dist / eta)
    np.testing.assert_allclose(OK.truncated_sum(x, y, a, eta, r), ref, rtol=1e-13, atol=1e-300)


def test_log_kernel_sum_matches_direct_and_is_shift_invariant():
    rng = np.random.default_rng(4)
    x, y = rng.uniform(0, 1, (50, 2)), rng.uniform(0, 1, (40, 2))
    lv = rng.normal(size=40)
    np.testing.assert_allclose(np.exp(OK.log_kernel_sum(x, y, lv, 0.03)), OK.direct_sum(x, y, np.exp(lv), 0.03),
                               rtol=1e-13)
    # offsets far beyond the exponent range of FP64 shift the result and nothing else
    for c in (900.0, -900.0):
        got = OK.log_kernel_sum(x, y, lv + c, 0.03)
        assert np.all(np.isfinite(got))
        np.testing.assert_allclose(got - c, OK.log_kernel_sum(x, y, lv, 0.03), rtol=0, atol=1e-12)
    # an eta so small that every kernel entry underflows in exp(): the log form stays finite
    got = OK.log_kernel_sum(x, y, lv, 1e-6)
    assert np.all(np.isfinite(got))
    d2 = ((x[:, None, :] - y[None, :, :]) ** 2).sum(-1)
    np.testing.assert_allclose(got, np.max(lv[None, :] - d2 / 1e-6, axis=1), rtol=1e-12)
    # truncated: -inf where no pair is left, the truncated sum elsewhere
    t = OK.log_kernel_sum(x, y, lv, 0.03, r_cut=0.1)
    ref = OK.truncated_sum(x, y, np.exp(lv), 0.03, 0.1)
    with np.errstate(divide="ignore"):
        np.testing.assert_allclose(t, np.log(ref), rtol=1e-13)


@pytest.mark.parametrize("shape", ["path", "star", "tree-random"])
def test_log_sinkhorn_equals_scaling_sinkhorn(shape):
    """Where both are representable, the log-domain Algorithm 2 produces log of the scaling-form
    iterates, sweep by sweep, and the same S^(r)."""
    rng = np.random.default_rng(7)
    prob = W.random_problem(rng, W.TREE, 5, 2, [30, 25, 40, 35, 20], eta=0.2, shape=shape)
    w = rng.uniform(0.5, 2.0, 4)
    h1, h2 = [], []
    r1 = OS.TreeSinkhorn(prob.x64(), prob.mu, prob.edges, prob.eta, root=2, edge_w=w).run(
        6, callback=lambda r, p: h1.append([q.copy() for q in p]))
    r2 = OS.TreeSinkhornLog(prob.x64(), prob.mu, prob.edges, prob.eta, root=2, edge_w=w).run(
        6, callback=lambda r, p: h2.append([q.copy() for q in p]))
    for a, b in zip(h1, h2):
        for pa, pb in zip(a, b):
            np.testing.assert_allclose(np.exp(pb), pa, rtol=1e-11)
    np.testing.assert_allclose(r2.S, r1.S, rtol=1e-11)


def _log_kernel_tensor_path(xs, eta):
    """log K_i = -sum_k ||x^{k+1}_{i_{k+1}} - x^k_{i_k}||^2 / eta for a path 1-2-...-K, entry by entry."""
    shape = tuple(len(a) for a in xs)
    L = np.empty(shape)
    for idx in itertools.product(*[range(m) for m in shape]):
        c = 0.0
        for k in range(len(xs) - 1):
            c += float(((xs[k + 1][idx[k + 1]] - xs[k][idx[k]]) ** 2).sum())
        L[idx] = -c / eta
    return L


def _log_marginals(L, f):
    K = L.ndim
    T = L.copy()
    for k in range(K):
        sh = [1] * K
        sh[k] = L.shape[k]
        T = T + f[k].reshape(sh)
    out = []
    for k in range(K):
        axes = tuple(a for a in range(K) if a != k)
        m = np.max(T, axis=axes, keepdims=True)
        out.append((m + np.log(np.exp(T - m).sum(axis=axes, keepdims=True))).reshape(-1))
    return out


def test_log_sinkhorn_at_small_eta_equals_log_bruteforce():
    """Two marginals far apart and eta = 1e-4: every kernel entry between them underflows in
    FP64, so the scaling form divides zero by zero; the log-domain Algorithm 2 on the path is
    the Gauss-Seidel sweep of Algorithm 1, here written in log form on the full tensor from the
    cost, and converges to the marginals."""
    rng = np.random.default_rng(11)
    x = [rng.uniform(0.0, 0.1, (4, 1)), rng.uniform(0.9, 1.0, (3, 1)), rng.uniform(0.4, 0.6, (5, 1))]
    mu = [np.full(4, 0.25), np.full(3, 1 / 3), np.full(5, 0.2)]
    edges = W.path_edges(3)
    eta = 1e-4
    with np.errstate(all="ignore"):
        rs = OS.TreeSinkhorn(x, mu, edges, eta).run(2)
    assert not all(np.all(np.isfinite(p)) and np.all(p > 0) for p in rs.phi)
    hist = []
    OS.TreeSinkhornLog(x, mu, edges, eta).run(8, callback=lambda r, f: hist.append([q.copy() for q in f]))
    L = _log_kernel_tensor_path(x, eta)
    f = [np.zeros(4), np.zeros(3), np.zeros(5)]
    for sweep in range(8):
        for k in range(3):
            f[k] = np.log(mu[k]) + f[k] - _log_marginals(L, f)[k]
        scale = max(float(np.max(np.abs(v))) for v in f)
        for a, b in zip(hist[sweep], f):
            np.testing.assert_allclose(a, b, rtol=0, atol=1e-10 * scale)
    # run on to the fixed point: the full tensor's marginals are the measures
    res = OS.TreeSinkhornLog(x, mu, edges, eta).run(1000)
    P = [np.exp(v) for v in _log_marginals(L, res.logphi)]
    for Pk, m in zip(P, mu):
        np.testing.assert_allclose(Pk, m, rtol=1e-9)


def test_truncated_log_sinkhorn_within_the_tail_bound():
    """Truncating every kernel sum of the log-domain Algorithm 2 at r drops terms
    exp(l_j - d^2 / eta) with d > r; while the log-potentials l vary by at most D over a point
    set, each dropped term is below exp(D - r^2 / eta) times the largest kept one, so every log
    message moves by at most N exp(D - r^2 / eta).  Point clouds that are small perturbations of
    one another (eta = 1e-3, r with r^2 / eta = 40): 20 sweeps agree to that bound."""
    rng = np.random.default_rng(12)
    K, n, eta = 4, 200, 1e-3
    x0 = rng.uniform(0.1, 0.9, (n, 2))
    x = [x0 + rng.normal(0, 0.003, (n, 2)) for _ in range(K)]
    mu = [np.full(n, 1.0 / n) for _ in range(K)]
    edges = W.path_edges(K)
    r_cut = math.sqrt(40 * eta)
    hf, ht = [], []
    OS.TreeSinkhornLog(x, mu, edges, eta).run(20, callback=lambda r, f: hf.append([q.copy() for q in f]))
    OS.TreeSinkhornLog(x, mu, edges, eta, r_cut=r_cut).run(20, callback=lambda r, f: ht.append([q.copy() for q in f]))
    for a, b in zip(hf, ht):
        D = max(float(np.ptp(v)) for v in a)
        bound = 4 * K * n * math.exp(D - r_cut * r_cut / eta)
        assert bound < 1e-6
        for va, vb in zip(a, b):
            assert np.max(np.abs(va - vb)) <= max(bound * 20, 1e-12)
    # the cut drops most pairs: the truncated sums are local
    d2 = ((x[0][:, None, :] - x[1][None, :, :]) ** 2).sum(-1)
    assert np.mean(d2 <= r_cut * r_cut) < 0.5
