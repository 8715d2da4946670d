"""GPU parity of the small-eta local path (MOT_PATH_LOCAL) through the C ABI.

Section 6.1 closes with the remark that for very small eta the kernel is so concentrated that its
sum may be truncated to nearby pairs.  At such eta the scalings exp(u / eta) under- and overflow
every floating-point format, so the CUDA path runs Algorithm 2 on the logarithms of the scalings
and messages, with every kernel sum truncated to |x - y| <= r_cut and evaluated as a log-sum-exp.
The reference is the oracle's ``TreeSinkhornLog`` with the same ``r_cut`` (pinned in
``tests/test_oracle_local.py`` to the plain sums, a loop over pairs and Algorithm 1 in log form on
the full tensor).

Bars: log-potentials f^k = log phi^k (gauge-fixed) within 1e-3 absolute after the same number of
sweeps (the FP32 terms carry ~1e-6 relative error per kernel sum, which compounds over the
sweeps), the violation of the oracle's truncated marginals within 1e-4, and S within 1e-4 of
max(|S|, eta) (S / eta = sum mu.log phi - mass is the quantity computed; at small eta S itself can
be far smaller than its terms).
"""
import math

import numpy as np
import pytest

from oracle import sinkhorn as OS
from paper_2208_03120_gb300 import workloads as W
from tests.gpu_helpers import problem_tensors

pytestmark = pytest.mark.gpu

REL = 1e-4


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2208_03120_gb300 import build, motfft
    build.build()
    return motfft


def local_solve(M, prob, r_cut, **opt):
    import torch
    x, mu = problem_tensors(prob)
    out = M.mot_solve(x, mu, prob.eta, M.MOT_TREE, edges=prob.edges, edge_w=prob.edge_w, root=prob.root,
                      opt=M.options(path=M.MOT_PATH_LOCAL, r_cut=r_cut, **opt))
    torch.cuda.synchronize()
    return out, [t.cpu().numpy() / prob.eta for t in out.u]     # log phi^k


def oracle_log(prob, r_cut, iters):
    ts = OS.TreeSinkhornLog(prob.x64(), prob.mu, prob.edges, prob.eta, root=prob.root, edge_w=prob.edge_w,
                            r_cut=r_cut)
    return ts.run(iters)


def log_report(prob, f, r_cut):
    """Oracle evaluation of log-scalings: truncated exact marginals (Theorem 4.1 in log form),
    violation and the dual value S."""
    lp = OS.tree_marginals_log(prob.x64(), f, prob.edges, prob.eta, root=prob.root, edge_w=prob.edge_w,
                               r_cut=r_cut)
    P = [np.exp(a) for a in lp]
    mass = float(P[0].sum())
    S = prob.eta * (sum(float(np.sum(np.where(m > 0, m * fk, 0.0))) for m, fk in zip(prob.mu, f)) - mass)
    return dict(viol=OS.violation(P, prob.mu), S=S)


def gauge(f, mu):
    return OS.gauge_fix(f, mu)


def small_eta_problem(shape, K, d, n, eta, seed):
    rng = np.random.default_rng(seed)
    prob = W.random_problem(rng, W.TREE, K, d, n, eta, shape=shape)
    # a regime the FP32 mantissas of the scaling form cannot span: the kernel between the farthest
    # points is below the FP32 range (e^-87), and for the smallest eta below FP64's (e^-745)
    diam2 = max(float(np.max(np.sum((a[:, None, :] - b[None, :, :]) ** 2, axis=-1)))
                for a in prob.x64() for b in prob.x64()[:1])
    assert diam2 / eta > 87.0
    return prob


@pytest.mark.parametrize("shape,K,d,n,eta", [("path", 4, 2, 400, 2e-4), ("star", 5, 3, 300, 1e-3),
                                              ("tree-random", 6, 1, 500, 1e-4)])
def test_local_fixed_sweeps_match_oracle(M, shape, K, d, n, eta):
    """30 sweeps of Algorithm 2 in the log domain with truncated sums equal the oracle's 30."""
    prob = small_eta_problem(shape, K, d, n, eta, seed=11 + K + d)
    r_cut = math.sqrt(40.0 * eta)
    out, f = local_solve(M, prob, r_cut, max_iter=30, tol_viol=-1.0, check_every=10)
    assert out.iters == 30
    res = oracle_log(prob, r_cut, 30)
    a, b = gauge(f, prob.mu), gauge(res.logphi, prob.mu)
    for va, vb, m in zip(a, b, prob.mu):
        assert np.max(np.abs(va - vb)) <= 1e-3, np.max(np.abs(va - vb))
    assert abs(out.S_last - res.S[-1]) <= REL * max(abs(res.S[-1]), prob.eta)
    rg, ro = log_report(prob, f, r_cut), log_report(prob, res.logphi, r_cut)
    assert abs(rg["viol"] - ro["viol"]) <= REL
    assert abs(out.cost_dual - ro["S"]) <= REL * max(abs(ro["S"]), prob.eta)


def test_local_to_tolerance_matches_oracle_solution(M):
    """A path of 5 in d = 2 at eta = 2e-3 solved to violation 1e-6 against the oracle's converged
    truncated solution (``tests/golden/oracle_local_path5_d2.json``, written by the oracle-only
    script ``tests/golden/make_oracle_goldens.py``): the oracle's truncated marginals of the CUDA
    scalings meet 1e-4, S within 1e-4, log-potentials within 1e-3 on the points with mass."""
    import json
    import os
    import zlib
    prob = W.random_problem(np.random.default_rng(5), W.TREE, 5, 2, 400, 2e-3, shape="path")
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_local_path5_d2.json")) as fh:
        g = json.load(fh)
    c = 0
    for a in prob.x:
        c = zlib.crc32(np.ascontiguousarray(a, dtype=np.float32).tobytes(), c)
    for m in prob.mu:
        c = zlib.crc32(np.ascontiguousarray(m, dtype=np.float64).tobytes(), c)
    assert c == g["inputs_crc"] and g["violation"] <= 1e-7
    r_cut = g["r_cut"]
    out, f = local_solve(M, prob, r_cut, tol_viol=1e-6, max_iter=5000)
    assert out.status == 0, (out.iters, out.violation)
    rg = log_report(prob, f, r_cut)
    assert rg["viol"] <= REL
    assert abs(out.cost_dual - g["dual"]) <= REL * max(abs(g["dual"]), prob.eta)
    a = gauge(f, prob.mu)
    for va, vb, m in zip(a, g["logphi"], prob.mu):
        w = m > 1e-3 / len(m)
        assert np.max(np.abs(va - np.asarray(vb))[w]) <= 1e-3


def test_local_edge_weights_and_user_cutoff(M):
    """Edge weights w_e (kernel exp(-w_e |x - y|^2 / eta)) and an explicit r_cut."""
    prob = small_eta_problem("tree-random", 5, 2, 350, 3e-4, seed=8)
    prob.edge_w = np.array([0.5, 1.0, 2.0, 1.5])
    r_cut = 0.12
    out, f = local_solve(M, prob, r_cut, max_iter=20, tol_viol=-1.0, check_every=10)
    res = oracle_log(prob, r_cut, 20)
    a, b = gauge(f, prob.mu), gauge(res.logphi, prob.mu)
    for va, vb in zip(a, b):
        assert np.max(np.abs(va - vb)) <= 1e-3
    assert abs(out.S_last - res.S[-1]) <= REL * max(abs(res.S[-1]), prob.eta)


def test_local_rejects_a_cutoff_that_leaves_a_target_alone(M):
    """A cutoff so small that some target has no source within it: MOT_ENUMERIC, no fault."""
    prob = small_eta_problem("path", 3, 2, 200, 2e-4, seed=9)
    with pytest.raises(M.MotError) as ei:
        local_solve(M, prob, 1e-6, max_iter=5, tol_viol=-1.0, check_every=5)
    assert ei.value.status == M.MOT_ENUMERIC
