"""Serving (continuous batching) through the C ABI: requests of different K, N, d and
tree / circle shape run concurrently on their own streams, are admitted as slots and pool
memory free up, and every result equals the same request solved alone (mot_solve) within
the parity tolerance."""
import numpy as np
import pytest

from oracle import sinkhorn as OS
from paper_2208_03120_gb300 import workloads as W
from tests.gpu_helpers import problem_tensors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2208_03120_gb300 import build, motfft
    build.build()
    return motfft


def _requests(n=10):
    reqs = W.serving_stream(n_requests=n, rate_hz=1e6, seed=7, n_range=(300, 2500), k_range=(3, 6),
                            circle_n_max=800)
    return [r.problem for r in reqs]


def _solve_alone(M, prob, opt):
    import torch
    x, mu = problem_tensors(prob)
    out = M.mot_solve(x, mu, prob.eta, prob.topology, edges=prob.edges, opt=opt)
    torch.cuda.synchronize()
    return out, [t.cpu().numpy() for t in out.u]


def _compare(prob, u_mix, cost_mix, u_alone, cost_alone):
    assert abs(cost_mix - cost_alone) <= 1e-4 * abs(cost_alone)
    a, b = OS.gauge_fix(u_mix, prob.mu), OS.gauge_fix(u_alone, prob.mu)
    scale = max(float(np.max(np.abs(v))) for v in b) + prob.eta
    for va, vb in zip(a, b):
        assert np.max(np.abs(va - vb)) <= 1e-3 * scale


def test_server_results_equal_solo(M):
    import torch
    probs = _requests(10)
    opt = M.options(tol_viol=1e-6, max_iter=3000)
    srv = M.Server(pool_bytes=2 << 30, max_active=6)
    tens = [problem_tensors(p) for p in probs]
    # first half submitted together, the rest while those are running
    for i in range(5):
        srv.submit(*tens[i], probs[i].eta, probs[i].topology, edges=probs[i].edges, opt=opt, tag=i)
    results, max_active, admitted_while_busy = {}, 0, False
    submitted = 5
    while len(results) < len(probs):
        a, p = srv.progress()
        max_active = max(max_active, a)
        if submitted < len(probs) and a > 0:
            srv.submit(*tens[submitted], probs[submitted].eta, probs[submitted].topology,
                       edges=probs[submitted].edges, opt=opt, tag=submitted)
            submitted += 1
            admitted_while_busy = True
        for r in srv.poll():
            results[r["tag"]] = r
    torch.cuda.synchronize()
    srv.close()
    assert max_active >= 2 and admitted_while_busy
    for i, prob in enumerate(probs):
        r = results[i]
        assert r["status"] == 0, (i, r)
        out, u_alone = _solve_alone(M, prob, opt)
        u_mix = [t.cpu().numpy() for t in r["u"]]
        _compare(prob, u_mix, r["cost_dual"], u_alone, out.cost_dual)


def test_server_admission_by_memory(M):
    """A pool that holds about one request at a time serialises admission; a request larger
    than the whole pool completes with MOT_ENOMEM."""
    import torch
    probs = _requests(4)
    opt = M.options(tol_viol=1e-6, max_iter=3000)
    tens = [problem_tensors(p) for p in probs]
    need = [M.mot_workspace_bytes(*t, p.eta, p.topology, edges=p.edges, opt=opt) for t, p in zip(tens, probs)]
    pool = int(max(need) * 1.2) + 4096
    srv = M.Server(pool_bytes=pool, max_active=4)
    for i, p in enumerate(probs):
        srv.submit(*tens[i], p.eta, p.topology, edges=p.edges, opt=opt, tag=i)
    big = W.random_problem(np.random.default_rng(1), W.TREE, 3, 2, 1_000_000, 0.05, shape="path")
    tb = problem_tensors(big)
    assert M.mot_workspace_bytes(*tb, big.eta, big.topology, edges=big.edges, opt=opt) > pool
    srv.submit(*tb, big.eta, big.topology, edges=big.edges, opt=opt, tag=99)
    results, max_active = {}, 0
    while len(results) < len(probs) + 1:
        a, _ = srv.progress()
        max_active = max(max_active, a)
        for r in srv.poll():
            results[r["tag"]] = r
    srv.close()
    torch.cuda.synchronize()
    assert results[99]["status"] == M.MOT_ENOMEM
    assert all(results[i]["status"] == 0 for i in range(len(probs)))
    if sum(need) > pool:
        assert max_active < len(probs)
