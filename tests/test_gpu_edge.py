"""GPU parity on degenerate and ragged inputs (Algorithms 2 and 3 through the C ABI).

Two-marginal trees (one edge), marginals with a single point, ragged point counts across the
nodes, and a circle whose first marginal has one point (a single column in the batched
products), on the NFFT and dense paths; each result is evaluated by the FP64 oracle with exact
kernels (violation and cost within 1e-4 of the oracle's converged solve).
"""
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


def _tree_problem(rng, d, n, edges, eta):
    x = [W.uniform_ball(rng, m, d, 0.24).astype(np.float32) for m in n]
    mu = [np.full(m, 1.0 / m) if m > 1 else np.ones(1) for m in n]
    mu = [m * rng.uniform(0.5, 1.5, m.shape) for m in mu]
    mu = [m / m.sum() for m in mu]
    return W.Problem("edge-tree", W.TREE, len(n), d, x, mu, eta, np.asarray(edges, dtype=np.int32))


def _report_tree(prob, u):
    phi = [np.exp(a / prob.eta) for a in u]
    P = OS.tree_marginals(prob.x64(), phi, prob.edges, prob.eta, root=prob.root)
    mass = OS.total_mass(P)
    return OS.violation(P, prob.mu), OS.dual_value(prob.mu, phi, mass, prob.eta)


@pytest.mark.parametrize("path", [0, 1])
@pytest.mark.parametrize("d,n,edges", [
    (2, [1, 300], [[0, 1]]),                               # one edge, a one-point marginal
    (1, [5, 7], [[1, 0]]),                                 # one edge, tiny sets
    (2, [3, 1000, 17, 250], [[0, 1], [1, 2], [1, 3]]),     # ragged star-like tree
    (3, [64, 1, 300, 129], [[0, 1], [1, 2], [2, 3]]),      # one-point marginal inside a path
])
def test_degenerate_and_ragged_trees(M, path, d, n, edges):
    import torch
    rng = np.random.default_rng(sum(n) + 31 * d)
    prob = _tree_problem(rng, d, n, edges, 0.05)
    x, mu = problem_tensors(prob)
    out = M.mot_solve(x, mu, prob.eta, M.MOT_TREE, edges=prob.edges, opt=M.options(path=path, tol_viol=1e-6,
                                                                                    max_iter=3000))
    torch.cuda.synchronize()
    assert out.status == 0, (out.iters, out.violation)
    u = [t.cpu().numpy() for t in out.u]
    res = OS.TreeSinkhorn(prob.x64(), prob.mu, prob.edges, prob.eta).run(2000)
    vg, dg = _report_tree(prob, u)
    vo, do = _report_tree(prob, [prob.eta * np.log(p) for p in res.phi])
    assert vg <= vo + REL
    assert abs(dg - do) <= REL * abs(do)
    assert abs(out.cost_dual - do) <= REL * abs(do)


@pytest.mark.parametrize("path", [0, 1])
def test_circle_with_a_one_point_first_marginal(M, path):
    """n_1 = 1: the batched column products of Algorithm 3 have a single column."""
    import torch
    rng = np.random.default_rng(5)
    n = [1, 40, 33, 57]
    x = [rng.uniform(-0.24, 0.24, (m, 1)).astype(np.float32) for m in n]
    mu = [np.ones(1)] + [W._normalised(rng.uniform(0.2, 1.0, m)) for m in n[1:]]
    prob = W.Problem("edge-circle", W.CIRCLE, 4, 1, x, mu, 0.05, None)
    xt, mt = problem_tensors(prob)
    out = M.mot_solve(xt, mt, prob.eta, M.MOT_CIRCLE, opt=M.options(path=path, tol_viol=1e-6, max_iter=3000))
    torch.cuda.synchronize()
    assert out.status == 0, (out.iters, out.violation)
    u = [t.cpu().numpy() for t in out.u]
    res = OS.CircleSinkhorn(prob.x64(), prob.mu, prob.eta).run(2000)

    def report(phi):
        P = OS.circle_marginals(prob.x64(), phi, prob.eta)
        mass = OS.total_mass(P)
        return OS.violation(P, prob.mu), OS.dual_value(prob.mu, phi, mass, prob.eta)
    vg, dg = report([np.exp(a / prob.eta) for a in u])
    vo, do = report(res.phi)
    assert vg <= vo + REL
    assert abs(dg - do) <= REL * abs(do)
