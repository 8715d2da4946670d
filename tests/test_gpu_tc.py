"""GPU parity of the tensor-core dense path (split BF16, tcgen05) through the C ABI.

The product is sum_j alpha_j K_ij with alpha and K each split into BF16 pairs v = hi + lo and
accumulated in FP32 as hi*hi + hi*lo + lo*hi.  With unit roundoff u = 2^-8 of BF16 the split
leaves |v - hi - lo| <= u^2 |v|, and the dropped lo*lo term is <= u^2 |ab|, so each term carries
a relative error of at most ~3 u^2 = 4.6e-5; for non-negative terms the same bound holds for
the sum.  The bar below is 5e-5 (relative to the largest output, or to sum_j |alpha_j| K_ij
for signed weights), against the FP64 oracle's direct summation.
"""
import numpy as np
import pytest

from oracle import kernel as OK
from paper_2208_03120_gb300 import workloads as W
from tests.gpu_helpers import to_dev_points

pytestmark = pytest.mark.gpu

TC_TOL = 5e-5


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2208_03120_gb300 import build, motfft
    build.build()
    return motfft


def _run(M, xs, xt, alpha, eta):
    import torch
    a = torch.from_numpy(np.ascontiguousarray(alpha, dtype=np.float32)).cuda()
    beta, _ = M.mot_fastsum(to_dev_points(xs), to_dev_points(xt), a, eta, M.options(path=M.MOT_PATH_DENSE_BF16X3))
    torch.cuda.synchronize()
    return beta.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("d,n_src,n_tgt,nrhs,eta", [
    (1, 1000, 777, 1, 0.05),      # one row tile, ragged column tile, ragged k tail
    (2, 2000, 1537, 3, 0.01),
    (3, 1237, 2049, 2, 0.02),     # n_src not a multiple of 8: padded row stride
    (2, 61, 9, 1, 0.1),           # smaller than one tile in every dimension
    (1, 5003, 300, 130, 0.05),    # two row tiles (130 right-hand sides)
    (2, 4099, 4099, 1, 0.05),     # 17 column tiles of 256
])
def test_tc_fastsum_matches_direct_sum(M, d, n_src, n_tgt, nrhs, eta):
    rng = np.random.default_rng(700 + 13 * d + n_src + nrhs)
    xs = W.uniform_ball(rng, n_src, d, 0.24).astype(np.float32)
    xt = W.uniform_ball(rng, n_tgt, d, 0.24).astype(np.float32)
    alpha = rng.uniform(0.0, 1.0, size=(nrhs, n_src)).astype(np.float32)
    beta = _run(M, xs, xt, alpha, eta).reshape(nrhs, n_tgt)
    for r in range(nrhs):
        ref = OK.direct_sum(xt.astype(np.float64), xs.astype(np.float64), alpha[r].astype(np.float64), eta)
        err = np.max(np.abs(beta[r] - ref)) / np.max(np.abs(ref))
        assert err <= TC_TOL, (r, err)


def test_tc_fastsum_signed_weights(M):
    """Signed weights: the error of each output is bounded relative to sum_j |alpha_j| K_ij."""
    rng = np.random.default_rng(811)
    xs = W.uniform_ball(rng, 3001, 2, 0.24).astype(np.float32)
    xt = W.uniform_ball(rng, 2500, 2, 0.24).astype(np.float32)
    alpha = rng.uniform(-1.0, 1.0, size=3001).astype(np.float32)
    beta = _run(M, xs, xt, alpha, 0.02)
    x64s, x64t = xs.astype(np.float64), xt.astype(np.float64)
    ref = OK.direct_sum(x64t, x64s, alpha.astype(np.float64), 0.02)
    ref_abs = OK.direct_sum(x64t, x64s, np.abs(alpha).astype(np.float64), 0.02)
    assert np.max(np.abs(beta - ref) / ref_abs) <= TC_TOL


def test_tc_fastsum_tiny_and_large_dynamic_range(M):
    """Kernel entries down to exp(-40) and one source: the split keeps the relative accuracy
    (BF16 has the FP32 exponent range)."""
    rng = np.random.default_rng(9)
    xs = rng.uniform(-0.24, 0.24, size=(1, 1)).astype(np.float32)
    xt = np.linspace(-0.24, 0.24, 333, dtype=np.float32)[:, None]
    beta = _run(M, xs, xt, np.array([0.75], dtype=np.float32), 0.005)
    ref = OK.direct_sum(xt.astype(np.float64), xs.astype(np.float64), np.array([0.75]), 0.005)
    assert np.all(np.abs(beta - ref) <= TC_TOL * ref)


@pytest.mark.parametrize("nrhs,n_src,n_tgt", [
    (2560, 300, 1000),   # 128-row tiles x 160-wide tiles (140 tiles)
    (3200, 301, 1000),   # 192-wide tiles (150 tiles), ragged source count
    (2000, 700, 2000),   # 224-wide tiles (144 tiles): the circle workload's shape
])
def test_tc_fastsum_tile_widths(M, nrhs, n_src, n_tgt):
    """Every tile width the launcher picks (fewest waves over the SMs) against the FP64 product
    of the kernel matrix with the weights."""
    rng = np.random.default_rng(nrhs + n_src)
    xs = W.uniform_ball(rng, n_src, 1, 0.24).astype(np.float32)
    xt = W.uniform_ball(rng, n_tgt, 1, 0.24).astype(np.float32)
    alpha = rng.uniform(0.0, 1.0, size=(nrhs, n_src)).astype(np.float32)
    beta = _run(M, xs, xt, alpha, 0.05).reshape(nrhs, n_tgt)
    Kmat = OK.kernel_matrix(xt.astype(np.float64), xs.astype(np.float64), 0.05)
    ref = alpha.astype(np.float64) @ Kmat.T
    err = np.max(np.abs(beta - ref), axis=1) / np.max(np.abs(ref), axis=1)
    assert np.max(err) <= TC_TOL
