"""Error paths of the C ABI on the GPU, in forms that fault nothing.

* Non-finite points and negative or non-finite weights are rejected with MOT_ENUMERIC: the
  bounding-box readback of the set-up sees a non-finite box before any point is binned, and the
  binning kernel flags a weight outside [0, inf) (it never indexes with a weight).
* The tensor-core kernel's bounded waits: with the test hook ``mot_test_tc_wait`` the kernel's
  load thread issues no copies and the wait limit is 2 ms, so the first wait for operands runs out
  (an mbarrier that nothing completes); the call returns MOT_ETIMEOUT, and the next call with the
  defaults restored computes the right product on the same context.
* The stop test of Algorithms 2 / 3 on the dual value, |S^(r) - S^(r-1)| < delta: the sweep at
  which the CUDA solve stops equals the one the oracle's S trace gives.
"""
import numpy as np
import pytest

from oracle import kernel as OK
from oracle import sinkhorn as OS
from paper_2208_03120_gb300 import workloads as W
from tests.gpu_helpers import inf_rel_err, problem_tensors, to_dev_points

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2208_03120_gb300 import build, motfft
    build.build()
    return motfft


def _solve_status(M, prob, topology, **opt):
    import torch
    x, mu = problem_tensors(prob)
    try:
        if topology == W.TREE:
            M.mot_solve(x, mu, prob.eta, M.MOT_TREE, edges=prob.edges, opt=M.options(**opt))
        else:
            M.mot_solve(x, mu, prob.eta, M.MOT_CIRCLE, opt=M.options(**opt))
    except M.MotError as e:
        torch.cuda.synchronize()
        return e.status
    torch.cuda.synchronize()
    return M.MOT_OK


@pytest.mark.parametrize("topology", [W.TREE, W.CIRCLE])
@pytest.mark.parametrize("what", ["x_nan", "x_inf", "mu_neg", "mu_nan"])
def test_non_finite_or_negative_inputs_are_rejected(M, topology, what):
    rng = np.random.default_rng(5)
    prob = W.random_problem(rng, topology, 4, 2, 300, 0.05, shape="path")
    if what == "x_nan":
        prob.x[2][17, 1] = np.nan
    elif what == "x_inf":
        prob.x[1][3, 0] = np.inf
    elif what == "mu_neg":
        prob.mu[3][5] = -prob.mu[3][5]
    else:
        prob.mu[0][9] = np.nan
    assert _solve_status(M, prob, topology, max_iter=20, check_every=10) == M.MOT_ENUMERIC
    # the context is still usable: the clean problem solves
    clean = W.random_problem(np.random.default_rng(5), topology, 4, 2, 300, 0.05, shape="path")
    assert _solve_status(M, clean, topology, max_iter=20, check_every=10, tol_viol=-1.0) == M.MOT_OK


def test_tensor_core_wait_runs_out_and_context_survives(M):
    import torch
    rng = np.random.default_rng(8)
    ps = W.uniform_ball(rng, 700, 2, 0.24).astype(np.float32)
    pt = W.uniform_ball(rng, 500, 2, 0.24).astype(np.float32)
    an = rng.uniform(0.1, 1.0, size=(3, 700)).astype(np.float32)
    xs, xt = to_dev_points(ps), to_dev_points(pt)
    a = torch.from_numpy(an).cuda()
    opt = M.options(path=M.MOT_PATH_DENSE_BF16X3)
    M.hook_tc_wait(2_000_000, stall_loads=True)
    try:
        with pytest.raises(M.MotError) as ei:
            M.mot_fastsum(xs, xt, a, 0.02, opt=opt)
        torch.cuda.synchronize()
        assert ei.value.status == M.MOT_ETIMEOUT
    finally:
        M.hook_tc_wait()
    b, _ = M.mot_fastsum(xs, xt, a, 0.02, opt=opt)
    torch.cuda.synchronize()
    exact = OK.direct_sum(pt.astype(np.float64), ps.astype(np.float64), an.T.astype(np.float64), 0.02)
    assert inf_rel_err(b.cpu().numpy().T, exact) <= 5e-5


def test_tc_wait_hook_validates_its_limit(M):
    assert M.lib().mot_test_tc_wait(10, 0) == M.MOT_EINVAL
    assert M.lib().mot_test_tc_wait(1_000_000_000, 0) == M.MOT_OK


@pytest.mark.parametrize("topology", [W.TREE, W.CIRCLE])
def test_delta_S_stop_matches_oracle_trace(M, topology):
    """Algorithm 2 / 3 stop when |S^(r) - S^(r-1)| < delta (tested after every sweep here).
    delta is put halfway (geometrically) between two consecutive differences of the oracle's trace
    that differ by at least a factor 4 and are at least 1e-6, so that delta is at least 1e-6 away
    from both: FP32 rounding of the CUDA path's S differences (~1e-7 here) cannot move the stop."""
    import torch
    if topology == W.TREE:
        prob = W.path3_d1()
        res = OS.TreeSinkhorn(prob.x64(), prob.mu, prob.edges, prob.eta).run(200)
    else:
        prob = W.random_problem(np.random.default_rng(31), W.CIRCLE, 4, 1, 400, 0.05)
        res = OS.CircleSinkhorn(prob.x64(), prob.mu, prob.eta).run(200)
    dS = np.abs(np.diff(res.S))                     # dS[r-2] = |S^(r) - S^(r-1)| after r sweeps
    stop = None
    for i in range(1, len(dS) - 1):
        if dS[i] >= 1e-6 and np.all(dS[:i] >= 4.0 * dS[i]):
            stop = i
            break
    assert stop is not None
    delta = float(np.sqrt(dS[stop] * dS[stop - 1]))
    expected = stop + 2                              # sweeps run when the oracle stops
    x, mu = problem_tensors(prob)
    opt = M.options(delta_S=delta, tol_viol=-1.0, check_every=1, max_iter=500)
    if topology == W.TREE:
        out = M.mot_solve(x, mu, prob.eta, M.MOT_TREE, edges=prob.edges, opt=opt)
        ores = OS.TreeSinkhorn(prob.x64(), prob.mu, prob.edges, prob.eta).run(500, delta=delta)
    else:
        out = M.mot_solve(x, mu, prob.eta, M.MOT_CIRCLE, opt=opt)
        ores = OS.CircleSinkhorn(prob.x64(), prob.mu, prob.eta).run(500, delta=delta)
    torch.cuda.synchronize()
    assert ores.iters == expected
    assert out.status == 0 and out.iters == expected, (out.status, out.iters, expected)
    assert abs(out.S_last - out.S_prev) < delta
