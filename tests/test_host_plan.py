"""Host logic of the solver's set-up (no GPU): the boundary polynomial of the regularised kernel
(Eq. Ker-reg) and the normalisation / grid choice of Section 5, through the library's host-only
entry points.

kappa_B is pinned to the worked example the paper prints in Fig. 3, to the oracle's boundary
polynomial (itself pinned to Fig. 3), and to its defining Hermite conditions; the grid choice to
the conditions it must meet (every pairwise distance below tau - eps_B after scaling, both
neglected terms below e^-18 when a grid within the limits reaches it, the smallest such grid).
"""
import math
import os

import numpy as np
import pytest
from numpy.polynomial import Polynomial

from oracle import kernel as OK

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fig3_kappa_B.txt")


@pytest.fixture(scope="module")
def M():
    from paper_2208_03120_gb300 import build, motfft
    build.build()
    return motfft


def _in_x(coef_t, a):
    """Coefficients in powers of t = x - a -> polynomial in x."""
    return Polynomial(coef_t)(Polynomial([-a, 1.0]))


def test_boundary_poly_reproduces_fig3(M):
    rows = [ln.split() for ln in open(GOLDEN) if ln.strip() and not ln.startswith("#")]
    for r in rows:
        eta, tau, eps_B, p = float(r[0]), float(r[1]), float(r[2]), int(r[3])
        printed = [float(v) for v in r[4:]]
        P = _in_x(M.boundary_poly(eta, tau, eps_B, p), tau - eps_B)
        np.testing.assert_allclose(P.coef, printed, atol=6e-6)     # printed to five decimals


@pytest.mark.parametrize("p", [1, 2, 3, 4, 6, 8])
@pytest.mark.parametrize("eta,eps_B", [(0.01, 1 / 16), (0.0125, 3 / 32), (0.05, 0.1)])
def test_boundary_poly_matches_oracle_and_hermite_conditions(M, p, eta, eps_B):
    """The Hermite conditions hold in t = x - a (where the coefficients are well scaled); the
    oracle's polynomial agrees for p <= 4 (in powers of x, higher degrees cancel badly)."""
    tau = 0.5
    a = tau - eps_B
    Pt = Polynomial(M.boundary_poly(eta, tau, eps_B, p))
    der = OK.kappa_derivatives_at(a, eta, p)
    ref = max(abs(v) for v in der)
    for r in range(p + 1):                       # kappa_B^(r)(a) = kappa^(r)(a)
        assert abs(Pt.deriv(r)(0.0) - der[r]) <= 1e-12 * max(1.0, abs(der[r]))
    c = Pt.coef
    for r in range(1, p + 1):                    # kappa_B^(r)(tau) = 0, relative to the size of its terms
        terms = [abs(c[j]) * math.factorial(j) / math.factorial(j - r) * eps_B ** (j - r) for j in range(r, len(c))]
        assert abs(Pt.deriv(r)(eps_B)) <= 1e-12 * max(sum(terms), ref)
    if p <= 4:                                   # the oracle's polynomial, back in t = x - a
        Qt = OK.boundary_polynomial(eta, tau, eps_B, p)(Polynomial([a, 1.0])).coef
        np.testing.assert_allclose(Pt.coef, Qt, rtol=0, atol=1e-9 * float(np.max(np.abs(Qt))))


def test_boundary_poly_rejects_bad_arguments(M):
    for args in [(0.0, 0.5, 0.1, 2), (0.01, 0.5, 0.6, 2), (0.01, 0.5, 0.1, 0), (0.01, 0.5, 0.1, 9)]:
        with pytest.raises(M.MotError):
            M.boundary_poly(*args)


@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("eta", [0.1, 0.05, 0.02, 0.01, 0.005])
def test_plan_grid_meets_its_conditions(M, d, eta):
    R, eps_B, tau = 0.24, 1 / 16, 0.5
    n, s, e = M.plan_grid(d, R, eta, eta, 0, eps_B)
    assert n >= 16 and n & (n - 1) == 0 and n <= {1: 4096, 2: 128, 3: 64}[d]
    assert 2 * R / s <= (tau - eps_B) * (1 + 1e-12)          # diameter after scaling within tau - eps_B
    # the two neglected exponents at this scale: kernel at tau - eps_B, Fourier tail beyond M = n/4
    A = (tau - eps_B) ** 2 * s * s / eta
    B = math.pi ** 2 * (eta / (s * s)) * (n / 4) ** 2
    assert abs(e - min(A, B)) <= 1e-9 * max(1.0, e)
    if e >= 18.0 and n > 16:
        # the next smaller grid would not have reached the target
        n2, s2, e2 = M.plan_grid(d, R, eta, eta, n // 2, eps_B)
        assert e2 < 18.0
    if e < 18.0:
        assert n == {1: 4096, 2: 128, 3: 64}[d]              # best effort at the largest grid


def test_plan_grid_is_monotone_in_eta_and_honours_an_explicit_grid(M):
    ns = [M.plan_grid(2, 0.24, eta, eta)[0] for eta in (0.2, 0.1, 0.05, 0.02, 0.01, 0.005)]
    assert ns == sorted(ns)
    n, s, e = M.plan_grid(2, 0.24, 0.01, 0.01, 64)
    assert n == 64
    with pytest.raises(M.MotError):
        M.plan_grid(2, 0.24, 0.01, 0.01, 48)                # not a power of two
    with pytest.raises(M.MotError):
        M.plan_grid(3, 0.24, 0.01, 0.01, 128)               # above the 3-D limit
