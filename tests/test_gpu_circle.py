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
