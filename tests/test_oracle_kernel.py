"""Pins of the FP64 oracle's kernel and fast-summation pieces (no GPU).

Each test ties the oracle to something other than itself: a value printed in
the paper, a closed form, or an identity whose failure would expose a dropped
term, a wrong sign or a transposed operand.
"""
import math
import os

import numpy as np
import pytest

from oracle import kernel as OK

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return rows


def test_fig3_boundary_polynomial():
    """Fig. 3 prints kappa_B = 1.26471 - 2.47375 x + 1.23688 x^2 for eta=1/4, tau=1,
    eps_B=0.2, p=1.  Pins the reading of the Hermite conditions (degree 2p,
    r = 0..p at tau - eps_B, r = 1..p at tau) and the derivative recursion."""
    (eta, tau, epsB, p, c0, c1, c2), = _golden_rows("fig3_kappa_B.txt")
    P = OK.boundary_polynomial(eta, tau, epsB, int(p))
    assert P.degree() == 2
    np.testing.assert_allclose(P.coef, [c0, c1, c2], atol=6e-6)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("eta,tau,epsB", [(0.25, 1.0, 0.2), (0.1, 0.5, 1 / 16), (0.05, 0.5, 3 / 32)])
def test_regularised_kernel_is_Cp(p, eta, tau, epsB):
    """Eq. (Ker-reg) makes kappa_R p times continuously differentiable: compare
    one-sided finite-difference derivatives at both junctions (|x| = tau - eps_B
    and |x| = tau) up to order p (orders above 2 get a looser bound)."""
    a = tau - epsB
    for x0 in (a, tau):
        h = 1e-3 * epsB
        for r in range(1, min(p, 2) + 1):
            left = np.array([x0 - (j * h) for j in range(r + 3)])[::-1]
            right = np.array([x0 + (j * h) for j in range(r + 3)])
            fl = OK.kappa_R(left, eta, tau, epsB, p)
            fr = OK.kappa_R(right, eta, tau, epsB, p)
            # backward / forward differences of order r
            dl = np.diff(fl, n=r)[-1] / h ** r
            dr = np.diff(fr, n=r)[0] / h ** r
            scale = max(1.0, abs(dl), abs(dr)) / eta ** r
            assert abs(dl - dr) <= 0.05 * scale, (x0, r, dl, dr)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_kappa_hat_poisson_closed_form(d):
    """When the kernel is negligible at the boundary, kappa_hat of Eq. (fft) is
    the Fourier coefficient of the Gaussian on the torus of period 2 tau:
    (pi eta)^{d/2} (2 tau)^{-d} exp(-pi^2 eta ||m||^2 / (4 tau^2)) (Poisson
    summation).  eta = 0.005 puts the kernel below 1e-16 at |x| = tau - eps_B
    and the aliased tail exp(-pi^2 eta M^2) near 1e-12 for M = 24."""
    eta, tau, epsB, p = 0.005, 0.5, 1 / 16, 3
    M = 24
    kh = OK.kappa_hat(eta, tau, epsB, p, M, d)
    m = np.arange(-M, M)
    grids = np.meshgrid(*([m] * d), indexing="ij")
    m2 = sum(g.astype(float) ** 2 for g in grids)
    exact = (math.pi * eta) ** (d / 2) / (2 * tau) ** d * np.exp(-math.pi ** 2 * eta * m2 / (4 * tau ** 2))
    np.testing.assert_allclose(kh, exact, atol=1e-10 * exact.max(), rtol=0)


def test_kappa_hat_real_even_and_interpolates():
    """The coefficients of the real, radial kernel are real and even in every
    coordinate, and the trigonometric sum reproduces kappa_tilde at the FFT
    nodes (inverse DFT) -- in particular sum_m kappa_hat(m) = kappa_tilde(0) = 1."""
    eta, tau, epsB, p, M, d = 0.2, 0.5, 3 / 32, 3, 8, 2
    kh = OK.kappa_hat(eta, tau, epsB, p, M, d)
    inner = kh[1:, 1:]                         # m in {-M+1..M-1}^2
    np.testing.assert_allclose(inner, inner[::-1, :], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(inner, inner[:, ::-1], rtol=1e-12, atol=1e-15)
    assert abs(kh.sum() - 1.0) < 1e-13
    # evaluate the series at a grid node x = tau j / M
    j = np.array([3, -5])
    x = tau * j / M
    m = np.arange(-M, M)
    phase = np.exp(1j * math.pi / tau * np.add.outer(m * x[0], m * x[1]))
    val = (kh * phase).sum()
    assert abs(val.imag) < 1e-13
    assert abs(val.real - OK.kappa_tilde(x[None, :], eta, tau, epsB, p)[0]) < 1e-13


@pytest.mark.parametrize("d", [1, 2, 3])
def test_direct_sum_gaussian_integral(d):
    """Eq. (fastsum-sum) with sources on a uniform grid of spacing h and weights
    h^d is a Riemann sum of the Gaussian integral: beta(x) = (pi eta)^{d/2}
    for targets well inside the grid (trapezoid error ~ exp(-pi^2 eta / h^2),
    truncation ~ exp(-dist^2/eta), both below 1e-12 here)."""
    eta = 0.01
    h = 0.02 if d == 3 else 0.01
    L = 0.62
    g = np.arange(-L, L + h / 2, h)
    grids = np.meshgrid(*([g] * d), indexing="ij")
    src = np.stack([a.ravel() for a in grids], axis=1)
    alpha = np.full(src.shape[0], h ** d)
    rng = np.random.default_rng(0)
    tgt = rng.uniform(-0.05, 0.05, size=(5, d))
    beta = OK.direct_sum(tgt, src, alpha, eta)
    np.testing.assert_allclose(beta, (math.pi * eta) ** (d / 2), rtol=1e-11)


def test_direct_sum_multi_rhs_and_symmetry():
    """K^{(k,l)} = (K^{(l,k)})^T (Eq. K-matrix is symmetric in its two point
    sets): <u, K v> computed both ways agrees; several right-hand sides give the
    same result as one at a time."""
    rng = np.random.default_rng(1)
    x = rng.uniform(-0.3, 0.3, size=(40, 2))
    y = rng.uniform(-0.3, 0.3, size=(30, 2))
    u = rng.uniform(size=40)
    V = rng.uniform(size=(30, 3))
    KV = OK.direct_sum(x, y, V, 0.05)
    KTu = OK.direct_sum(y, x, u, 0.05)
    np.testing.assert_allclose(u @ KV, KTu @ V, rtol=1e-13)
    for c in range(3):
        np.testing.assert_allclose(KV[:, c], OK.direct_sum(x, y, V[:, c], 0.05), rtol=1e-14)


@pytest.mark.parametrize("d,eta,M", [(1, 0.01, 16), (2, 0.01, 16), (3, 0.01, 16), (1, 0.005, 24)])
def test_fastsum_ndft_matches_direct_sum(d, eta, M):
    """Algorithm 4 with exact NDFTs approximates K alpha (Eq. fastsum_mat).  With
    points well inside the ball of radius (tau - eps_B)/2 and a kernel
    negligible at the regularisation boundary, the only error is the Fourier
    truncation, below 1e-9 relative here.  A wrong sign in either NDFT, a wrong
    period or a dropped normalisation fails this."""
    rng = np.random.default_rng(2 + d)
    tau, epsB, p = 0.5, 1 / 16, 3
    r = 0.18
    xs = rng.uniform(-r / math.sqrt(d), r / math.sqrt(d), size=(60, d)) + 0.01
    xt = rng.uniform(-r / math.sqrt(d), r / math.sqrt(d), size=(50, d)) - 0.02
    alpha = rng.uniform(0.1, 1.0, size=60)
    ref = OK.direct_sum(xt, xs, alpha, eta)
    approx = OK.fastsum_ndft(xt, xs, alpha, eta, tau, epsB, p, M)
    err = np.max(np.abs(approx - ref)) / np.max(np.abs(ref))
    assert err < 1e-9, err


def test_fastsum_ndft_error_decreases_with_M():
    """Section 6.1: with the kernel not negligible at the boundary (eta = 0.1 on
    [-0.2, 0.2], the regularised part is active) the error of the fast
    summation decreases as M grows (kappa_tilde is only C^p)."""
    rng = np.random.default_rng(7)
    tau, epsB, p, eta = 0.5, 1 / 16, 3, 0.1
    xs = rng.uniform(-0.2, 0.2, size=(80, 1))
    xt = rng.uniform(-0.2, 0.2, size=(70, 1))
    alpha = rng.uniform(size=80)
    ref = OK.direct_sum(xt, xs, alpha, eta)
    errs = []
    for M in (8, 16, 32, 64, 128):
        approx = OK.fastsum_ndft(xt, xs, alpha, eta, tau, epsB, p, M)
        errs.append(np.max(np.abs(approx - ref)) / np.max(ref))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-6, errs
