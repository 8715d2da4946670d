"""GPU parity of circle-structured Sinkhorn (Algorithm 3) through the C ABI.

The NFFT path (batched fast summation over the N columns) and the dense direct path are
compared with the FP64 oracle (Algorithm 3 with dense matrices; pinned to brute force and
to the path tree by tests/test_oracle_sinkhorn.py).  Bars as for trees: violation and
cost within 1e-4 of the oracle; the marginals of the CUDA scalings are evaluated by the
oracle's exact kernels (Theorem 4.3).
"""
import zlib

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


def gpu_solve(M, prob, **opt):
    import torch
    x, mu = problem_tensors(prob)
    out = M.mot_solve(x, mu, prob.eta, M.MOT_CIRCLE, edge_w=prob.edge_w, opt=M.options(**opt))
    torch.cuda.synchronize()
    return out, [t.cpu().numpy() for t in out.u]


def exact_report(prob, u):
    phi = [np.exp(a / prob.eta) for a in u]
    P = OS.circle_marginals(prob.x64(), phi, prob.eta, edge_w=prob.edge_w)
    mass = OS.total_mass(P)
    return dict(viol=OS.violation(P, prob.mu), dual=OS.dual_value(prob.mu, phi, mass, prob.eta),
                primal=OS.primal_value(P, phi, mass, prob.eta))


def oracle_solve(prob, iters):
    res = OS.CircleSinkhorn(prob.x64(), prob.mu, prob.eta, edge_w=prob.edge_w).run(iters)
    return [prob.eta * np.log(p) for p in res.phi], res


def assert_parity(prob, u_gpu, u_or, out):
    rg, ro = exact_report(prob, u_gpu), exact_report(prob, u_or)
    assert abs(rg["viol"] - ro["viol"]) <= REL, (rg, ro)
    assert abs(rg["dual"] - ro["dual"]) <= REL * abs(ro["dual"]), (rg, ro)
    assert abs(rg["primal"] - ro["primal"]) <= REL * abs(ro["primal"]), (rg, ro)
    assert abs(out.cost_dual - ro["dual"]) <= REL * abs(ro["dual"])
    a, b = OS.gauge_fix(u_gpu, prob.mu), OS.gauge_fix(u_or, prob.mu)
    scale = max(float(np.max(np.abs(v))) for v in b) + prob.eta
    for va, vb in zip(a, b):
        assert np.max(np.abs(va - vb)) <= 1e-3 * scale


@pytest.mark.parametrize("path", [0, 1, 2])
@pytest.mark.parametrize("K,d,n,eta", [(3, 1, 300, 0.05), (4, 2, 250, 0.03), (5, 1, 500, 0.05), (3, 3, 200, 0.1)])
def test_small_circles_to_tolerance(M, path, K, d, n, eta):
    rng = np.random.default_rng(zlib.crc32(f"circle-{K}-{d}-{n}".encode()))
    prob = W.random_problem(rng, W.CIRCLE, K, d, [n + 17 * k for k in range(K)], eta)
    out, u = gpu_solve(M, prob, path=path, tol_viol=1e-6, max_iter=4000)
    assert out.status == 0, (out.iters, out.violation)
    u_or, _ = oracle_solve(prob, 3000)
    assert_parity(prob, u, u_or, out)


def test_circle_fixed_iterations_match_oracle(M):
    """Algorithm 3 step by step: after 30 sweeps from phi = 1 the CUDA scalings equal the
    oracle's 30 sweeps (same Gauss-Seidel order)."""
    rng = np.random.default_rng(31)
    prob = W.random_problem(rng, W.CIRCLE, 4, 1, 400, 0.05)
    out, u = gpu_solve(M, prob, max_iter=30, tol_viol=-1.0, check_every=10)
    assert out.iters == 30
    u_or, res = oracle_solve(prob, 30)
    assert_parity(prob, u, u_or, out)
    assert abs(out.S_last - res.S[-1]) <= REL * abs(res.S[-1])


def test_circle5_workload_full_size(M):
    """The 5-marginal d=1 circle workload at full size (N = 2000, eta = 0.05): NFFT, dense SIMT
    and dense tensor-core paths to violation 1e-6; the oracle evaluates every result with
    exact kernels."""
    prob = W.circle5_d1()
    outs = [gpu_solve(M, prob, path=p, tol_viol=1e-6, max_iter=3000) for p in (0, 1, 2)]
    for o, _ in outs:
        assert o.status == 0, (o.iters, o.violation)
    reps = [exact_report(prob, u) for _, u in outs]
    for (o, _), r in zip(outs, reps):
        assert r["viol"] <= REL
        assert abs(r["dual"] - reps[1]["dual"]) <= REL * abs(reps[1]["dual"])
        assert abs(o.cost_dual - r["dual"]) <= REL * abs(r["dual"])


# ---------------------------------------------------------------------------
# generalised Euler flows (Section 6.3)
# ---------------------------------------------------------------------------

def euler_solve(M, prob, **opt):
    import torch
    from tests.gpu_helpers import to_dev_points
    x, mu = problem_tensors(prob)
    out = M.mot_solve(x, mu, prob.eta, M.MOT_CIRCLE, x_close=to_dev_points(prob.x_close), pair=True,
                      opt=M.options(**opt))
    torch.cuda.synchronize()
    return out, [t.cpu().numpy() for t in out.u], [None] + [t.cpu().numpy() for t in out.pair[1:]]


@pytest.mark.parametrize("path", [0, 1, 2])
@pytest.mark.parametrize("sigma", ["reflect", "fold"])
def test_euler_flow_to_tolerance(M, path, sigma):
    """The Section 6.3 workload (K = 5, N = 400 on [0, 1], eta = 0.05) with the closing edge
    against sigma(x^1): violation, dual and primal values and the gauge-fixed potentials within
    1e-4 of the oracle's converged solve; the returned pair marginals Pi_{1,k} agree with the
    oracle's Pi_{1,k} at the same scalings (exact kernels) to 1e-4 in l1 (the marginal
    violation bar) and their row / column sums are mu^1 / mu^k to the solve's violation plus 1e-4 (each pair
    marginal reaches P_1 through its own chain of approximate products)."""
    prob = W.euler5_d1(sigma=sigma)
    xc = prob.x_close64()
    out, u, pairs = euler_solve(M, prob, path=path, tol_viol=1e-6, max_iter=2000)
    assert out.status == 0, (out.iters, out.violation)
    res = OS.CircleSinkhorn(prob.x64(), prob.mu, prob.eta, x_close=xc).run(200)
    u_or = [prob.eta * np.log(p) for p in res.phi]
    phi_g = [np.exp(a / prob.eta) for a in u]

    def report(phi):
        P = OS.circle_marginals(prob.x64(), phi, prob.eta, x_close=xc)
        mass = OS.total_mass(P)
        return dict(viol=OS.violation(P, prob.mu), dual=OS.dual_value(prob.mu, phi, mass, prob.eta),
                    primal=OS.primal_value(P, phi, mass, prob.eta))
    rg, ro = report(phi_g), report(res.phi)
    assert abs(rg["viol"] - ro["viol"]) <= REL, (rg, ro)
    assert abs(rg["dual"] - ro["dual"]) <= REL * abs(ro["dual"]), (rg, ro)
    assert abs(rg["primal"] - ro["primal"]) <= REL * abs(ro["primal"]), (rg, ro)
    assert abs(out.cost_dual - ro["dual"]) <= REL * abs(ro["dual"])
    a, b = OS.gauge_fix(u, prob.mu), OS.gauge_fix(u_or, prob.mu)
    scale = max(float(np.max(np.abs(v))) for v in b) + prob.eta
    for va, vb in zip(a, b):
        assert np.max(np.abs(va - vb)) <= 1e-3 * scale
    ref = OS.circle_pair_marginals(prob.x64(), phi_g, prob.eta, x_close=xc)
    for k in range(1, prob.K):
        assert pairs[k].shape == (prob.n[0], prob.n[k])
        assert np.all(pairs[k] >= 0.0)
        assert np.abs(pairs[k] - ref[k]).sum() <= REL, k
        assert np.abs(pairs[k].sum(axis=1) - prob.mu[0]).sum() <= out.violation + REL
        assert np.abs(pairs[k].sum(axis=0) - prob.mu[k]).sum() <= out.violation + REL


def test_euler_flow_fixed_iterations_match_oracle(M):
    """Algorithm 3 with the sigma-closing edge, step by step: after 30 sweeps from phi = 1 the
    CUDA scalings and pair marginals equal the oracle's 30 sweeps (dense SIMT path, so that
    the only differences are FP32 rounding)."""
    prob = W.euler5_d1(n=300, sigma="fold", seed=77)
    xc = prob.x_close64()
    out, u, pairs = euler_solve(M, prob, path=1, max_iter=30, tol_viol=-1.0, check_every=10)
    assert out.iters == 30
    res = OS.CircleSinkhorn(prob.x64(), prob.mu, prob.eta, x_close=xc).run(30)
    a = OS.gauge_fix(u, prob.mu)
    b = OS.gauge_fix([prob.eta * np.log(p) for p in res.phi], prob.mu)
    scale = max(float(np.max(np.abs(v))) for v in b) + prob.eta
    for va, vb in zip(a, b):
        assert np.max(np.abs(va - vb)) <= 1e-4 * scale
    assert abs(out.S_last - res.S[-1]) <= REL * abs(res.S[-1])
    ref = OS.circle_pair_marginals(prob.x64(), res.phi, prob.eta, x_close=xc)
    for k in range(1, prob.K):
        assert np.abs(pairs[k] - ref[k]).sum() <= REL * ref[k].sum(), k


def test_euler_identity_map_equals_plain_circle(M):
    """x_close = x^1 (sigma = identity) reproduces the plain circle solve on the same path (to
    the rounding of its atomic sums)."""
    import torch
    from tests.gpu_helpers import to_dev_points
    prob = W.circle5_d1(n=500)
    x, mu = problem_tensors(prob)
    a = M.mot_solve(x, mu, prob.eta, M.MOT_CIRCLE, opt=M.options(tol_viol=1e-6, max_iter=500, path=1))
    b = M.mot_solve(x, mu, prob.eta, M.MOT_CIRCLE, x_close=to_dev_points(prob.x[0]),
                    opt=M.options(tol_viol=1e-6, max_iter=500, path=1))
    torch.cuda.synchronize()
    assert a.iters == b.iters
    assert abs(a.cost_dual - b.cost_dual) <= 1e-6 * abs(a.cost_dual)
