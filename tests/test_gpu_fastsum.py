"""GPU parity of the kernel matrix-vector product (Eq. fastsum-sum) through the C ABI.

The NFFT fast summation (Algorithm 4) and the dense direct path are compared with
the FP64 oracle's direct summation, element by element; the bar is the matvec
tolerance: max relative error (infinity norm) <= 1e-5 in FP32.
"""
import math

import numpy as np
import pytest

from oracle import kernel as OK
from paper_2208_03120_gb300 import workloads as W
from tests.gpu_helpers import inf_rel_err, to_dev_points

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2208_03120_gb300 import build, motfft
    build.build()
    return motfft


def _run(M, xs, xt, alpha, eta, **opt):
    import torch
    a = torch.from_numpy(np.ascontiguousarray(alpha, dtype=np.float32)).cuda()
    beta, scale = M.mot_fastsum(to_dev_points(xs), to_dev_points(xt), a, eta, M.options(**opt))
    torch.cuda.synchronize()
    return beta.cpu().numpy().astype(np.float64), scale


@pytest.mark.parametrize("path", [0, 1])
@pytest.mark.parametrize("d,n_src,n_tgt,eta", [
    (1, 1000, 777, 0.05), (1, 3001, 2999, 0.01),
    (2, 2000, 1537, 0.01), (2, 5003, 4099, 0.05),
    (3, 3001, 2049, 0.02), (3, 1500, 1777, 0.1),
])
def test_fastsum_matches_direct_sum(M, path, d, n_src, n_tgt, eta):
    """Several tiles and subproblems with ragged tails (sizes not multiples of 256)."""
    rng = np.random.default_rng(100 + d * 7 + n_src)
    xs = W.uniform_ball(rng, n_src, d, 0.24).astype(np.float32)
    xt = W.uniform_ball(rng, n_tgt, d, 0.24).astype(np.float32)
    alpha = rng.uniform(0.0, 1.0, size=n_src)
    beta, _ = _run(M, xs, xt, alpha, eta, path=path)
    ref = OK.direct_sum(xt.astype(np.float64), xs.astype(np.float64), alpha.astype(np.float32).astype(np.float64), eta)
    assert inf_rel_err(beta, ref) <= TOL


def test_fastsum_clustered_workload_full_size(M):
    """The 10-node d=2 workload's point cloud (3-Gaussian mixture, N = 10^4) at full size,
    with a Dirichlet-like weight vector, in the launch configuration of the solve."""
    prob = W.path10_d2()
    xs, xt = prob.x[3], prob.x[4]
    alpha = prob.mu[3] * 1e4
    beta, _ = _run(M, xs, xt, alpha, prob.eta)
    ref = OK.direct_sum(xt.astype(np.float64), xs.astype(np.float64), alpha.astype(np.float32).astype(np.float64), prob.eta)
    assert inf_rel_err(beta, ref) <= TOL


def test_fastsum_ball3d_full_size_sampled(M):
    """d = 3, N = 5*10^4 per set (the star workload's marginals), checked on 1500 sampled targets."""
    prob = W.star9_d3()
    xs, xt = prob.x[1], prob.x[2]
    alpha = np.random.default_rng(5).uniform(0, 1, size=xs.shape[0])
    beta, _ = _run(M, xs, xt, alpha, prob.eta)
    idx = np.random.default_rng(6).choice(xt.shape[0], 1500, replace=False)
    ref = OK.direct_sum(xt[idx].astype(np.float64), xs.astype(np.float64), alpha.astype(np.float32).astype(np.float64), prob.eta)
    # normalise by the full-vector maximum estimated on the sample
    err = np.max(np.abs(beta[idx] - ref)) / np.max(np.abs(ref))
    assert err <= TOL


def test_fastsum_multiple_rhs_and_edge_cases(M):
    rng = np.random.default_rng(9)
    xs = W.uniform_ball(rng, 700, 2, 0.2).astype(np.float32)
    xt = W.uniform_ball(rng, 300, 2, 0.2).astype(np.float32)
    A = rng.uniform(size=(3, 700))
    beta, _ = _run(M, xs, xt, A, 0.03)
    for r in range(3):
        ref = OK.direct_sum(xt.astype(np.float64), xs.astype(np.float64), A[r].astype(np.float32).astype(np.float64), 0.03)
        assert inf_rel_err(beta[r], ref) <= TOL
    # one source, one target
    b1, _ = _run(M, xs[:1], xt[:1], np.array([2.0]), 0.03)
    ref1 = 2.0 * math.exp(-float(((xs[0].astype(np.float64) - xt[0]) ** 2).sum()) / 0.03)
    assert abs(b1[0] - ref1) <= TOL * ref1
    # all points identical: beta = sum(alpha)
    same = np.repeat(xs[:1], 257, axis=0)
    b2, _ = _run(M, same, same[:5], np.ones(257), 0.03)
    np.testing.assert_allclose(b2, 257.0, rtol=TOL)


def test_fastsum_grid_override_and_invariance(M):
    """An explicit grid length gives the same product; translating and scaling the points
    together with eta (x -> a x + b, eta -> a^2 eta) leaves it unchanged."""
    rng = np.random.default_rng(11)
    xs = W.uniform_ball(rng, 900, 2, 0.24).astype(np.float32)
    xt = W.uniform_ball(rng, 800, 2, 0.24).astype(np.float32)
    alpha = rng.uniform(size=900)
    b_auto, _ = _run(M, xs, xt, alpha, 0.05)
    b_128, _ = _run(M, xs, xt, alpha, 0.05, n_grid=128)
    ref = OK.direct_sum(xt.astype(np.float64), xs.astype(np.float64), alpha.astype(np.float32).astype(np.float64), 0.05)
    assert inf_rel_err(b_auto, ref) <= TOL and inf_rel_err(b_128, ref) <= TOL
    b_s, _ = _run(M, (3.0 * xs + 5.0).astype(np.float32), (3.0 * xt + 5.0).astype(np.float32), alpha, 9 * 0.05)
    ref_s = OK.direct_sum((3.0 * xt + 5.0).astype(np.float32).astype(np.float64),
                          (3.0 * xs + 5.0).astype(np.float32).astype(np.float64),
                          alpha.astype(np.float32).astype(np.float64), 9 * 0.05)
    assert inf_rel_err(b_s, ref_s) <= TOL


@pytest.mark.parametrize("n_src,n_tgt,eta", [(2000, 1537, 0.01), (10363, 9001, 0.02), (37, 5, 0.05), (1, 700, 0.03)])
def test_exact_sums_match_oracle_ndft(M, n_src, n_tgt, eta):
    """d = 2 on the 64^2 grid (M = 16) evaluates the trigonometric sums of the fast summation
    exactly (Eq. ndft* for ghat, Eq. ndft for the result): the product equals the oracle's
    Algorithm 4 with direct NDFTs (``fastsum_ndft``, pinned to the direct sum in
    ``tests/test_oracle_kernel.py``) on the same normalised points up to FP32 rounding -- no
    window error.  Sizes: several 640-point chunks per CTA with a ragged tail (10363 sources over
    16 CTAs), a handful of points per CTA, and a single source (15 CTAs without sources)."""
    rng = np.random.default_rng(300 + n_src)
    xs = W.uniform_ball(rng, n_src, 2, 0.24).astype(np.float32)
    xt = W.uniform_ball(rng, n_tgt, 2, 0.24).astype(np.float32)
    alpha = rng.uniform(0.0, 1.0, size=n_src)
    beta, s = _run(M, xs, xt, alpha, eta, n_grid=64)
    # the library maps x to x / s on the unit torus (period 2 tau = 1) with eta / s^2; the kernel
    # of Eq. (Ker-reg) depends only on differences, so the centre of that map drops out
    ref = OK.fastsum_ndft(xt.astype(np.float64) / s, xs.astype(np.float64) / s,
                          alpha.astype(np.float32).astype(np.float64), eta / (s * s), 0.5, 1.0 / 16.0, 3, 16)
    assert np.max(np.abs(beta - ref)) <= 2e-6 * np.max(np.abs(ref))
    # the grid path on the same input carries the window error on top
    b_grid, _ = _run(M, xs, xt, alpha, eta, n_grid=64, ndft=-1)
    ref_d = OK.direct_sum(xt.astype(np.float64), xs.astype(np.float64), alpha.astype(np.float32).astype(np.float64), eta)
    assert inf_rel_err(b_grid, ref_d) <= TOL and inf_rel_err(beta, ref_d) <= TOL


def test_exact_sums_multiple_rhs(M):
    """Several right-hand sides: one cluster per right-hand side, each equal to its own product."""
    rng = np.random.default_rng(12)
    xs = W.uniform_ball(rng, 3000, 2, 0.2).astype(np.float32)
    xt = W.uniform_ball(rng, 2500, 2, 0.2).astype(np.float32)
    A = rng.uniform(size=(4, 3000))
    beta, _ = _run(M, xs, xt, A, 0.02)
    for r in range(4):
        b1, _ = _run(M, xs, xt, A[r], 0.02)
        np.testing.assert_allclose(beta[r], b1[0] if b1.ndim > 1 else b1, rtol=0, atol=1e-6 * np.max(np.abs(b1)))
        ref = OK.direct_sum(xt.astype(np.float64), xs.astype(np.float64), A[r].astype(np.float32).astype(np.float64), 0.02)
        assert inf_rel_err(beta[r], ref) <= TOL


@pytest.mark.parametrize("n_grid,M_", [(32, 8)])
def test_exact_sums_smaller_grids(M, n_grid, M_):
    """A grid of 32 (M = 8): the frequencies beyond M carry no weight, and the product still equals
    the oracle's direct-NDFT fast summation with that M.  (The library weights the frequencies at
    |k_t| = M by 1/2 on both sides where the oracle keeps -M once; for d = 2 the two differ by the
    corner terms of size kappa_hat(M, M), which at M = 4 exceed the 2e-6 bar.)"""
    rng = np.random.default_rng(500 + n_grid)
    xs = W.uniform_ball(rng, 3001, 2, 0.24).astype(np.float32)
    xt = W.uniform_ball(rng, 2222, 2, 0.24).astype(np.float32)
    alpha = rng.uniform(0.0, 1.0, size=3001)
    eta = 0.08
    beta, s = _run(M, xs, xt, alpha, eta, n_grid=n_grid)
    ref = OK.fastsum_ndft(xt.astype(np.float64) / s, xs.astype(np.float64) / s,
                          alpha.astype(np.float32).astype(np.float64), eta / (s * s), 0.5, 1.0 / 16.0, 3, M_)
    assert np.max(np.abs(beta - ref)) <= 2e-6 * np.max(np.abs(ref))


def test_exact_sums_largest_sets_sampled(M):
    """The largest sets of the exact-sum kernel (32768 points: 2048 per CTA, four chunks of up to
    640), checked against the oracle's direct-NDFT fast summation on 2000 sampled targets."""
    rng = np.random.default_rng(77)
    n = 32768
    xs = W.uniform_ball(rng, n, 2, 0.24).astype(np.float32)
    xt = W.uniform_ball(rng, n, 2, 0.24).astype(np.float32)
    alpha = rng.uniform(0.0, 1.0, size=n)
    beta, s = _run(M, xs, xt, alpha, 0.02, n_grid=64)
    idx = np.random.default_rng(78).choice(n, 2000, replace=False)
    ref = OK.fastsum_ndft(xt[idx].astype(np.float64) / s, xs.astype(np.float64) / s,
                          alpha.astype(np.float32).astype(np.float64), 0.02 / (s * s), 0.5, 1.0 / 16.0, 3, 16)
    assert np.max(np.abs(beta[idx] - ref)) <= 2e-6 * np.max(np.abs(ref))
