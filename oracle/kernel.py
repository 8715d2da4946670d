"""Gaussian kernel, its regularisation and the fast-summation approximation, FP64.

Test infrastructure only (see ``oracle/__init__.py``).

Paper passages followed (Section 5):
  * Eq. (kappa)        kappa(x) = exp(-x^2 / eta)
  * Eq. (Ker-reg)      regularised kernel kappa_R with boundary polynomial kappa_B
  * Fig. 3             worked example of kappa_B (eta=1/4, tau=1, eps_B=0.2, p=1)
  * Eq. (kappa_tilde)  2 tau-periodic kernel kappa_R(||x||) on [-tau, tau)^d
  * Eq. (fft)          Fourier coefficients kappa_hat(m), m in {-M..M-1}^d
  * Eq. (fastsum-sum)  direct summation beta = K alpha
  * Eqs. (ndft), (ndft*), (fastsum_mat), Algorithm 4: beta ~ F_k(kappa_hat * F*_l alpha)
  * Section 6.1, closing remark: for very small eta the sum of Eq. (fastsum-sum)
    may simply be truncated to nearby pairs (``truncated_sum``); the same sum
    in log-sum-exp form (``log_kernel_sum``) serves Sinkhorn in the log domain

Readings of passages that are garbled or silent:
  * Hermite conditions of kappa_B: the printed rule gives p or 2p-1 conditions
    for a degree-p polynomial, which cannot hold together.  The reading that
    reproduces the printed Fig. 3 polynomial is: kappa_B has degree 2p,
    kappa_B^(r)(tau - eps_B) = kappa^(r)(tau - eps_B) for r = 0..p and
    kappa_B^(r)(tau) = 0 for r = 1..p  (2p + 1 conditions).
  * The condition on tau squares the distance; the branches of kappa_R compare
    |x| (unsquared) with tau - eps_B, so the reading is
    tau - eps_B >= max ||x^k_i - x^l_j||_2.
  * Eq. (ndft) carries exp(-i ...) while Eq. (fastsum1) needs exp(+i ...); the
    evaluation below uses the pair of Eq. (fastsum1) (adjoint with the minus
    sign, evaluation with the plus sign) and returns the real part, the
    approximation of a real matrix-vector product.
"""
from __future__ import annotations

import math

import numpy as np
from numpy.polynomial import Polynomial


def kappa(x, eta):
    """Eq. (kappa): kappa(x) = exp(-x^2/eta)."""
    x = np.asarray(x, dtype=np.float64)
    return np.exp(-x * x / eta)


def kappa_derivatives_at(x0: float, eta: float, order: int) -> np.ndarray:
    """kappa^(r)(x0) for r = 0..order.

    kappa^(r) = P_r * kappa with P_0 = 1 and P_{r+1} = P_r' - (2x/eta) P_r
    (product rule applied to P_r(x) exp(-x^2/eta)).
    """
    P = Polynomial([1.0])
    two_x_over_eta = Polynomial([0.0, 2.0 / eta])
    out = []
    k0 = math.exp(-x0 * x0 / eta)
    for _ in range(order + 1):
        out.append(P(x0) * k0)
        P = P.deriv() - two_x_over_eta * P
    return np.array(out)


def boundary_polynomial(eta: float, tau: float, eps_B: float, p: int) -> Polynomial:
    """kappa_B of Eq. (Ker-reg) as a polynomial in x (degree 2p).

    Conditions (reading pinned by Fig. 3): with a = tau - eps_B,
      kappa_B^(r)(a)   = kappa^(r)(a),  r = 0..p
      kappa_B^(r)(tau) = 0,             r = 1..p.
    Written in t = x - a, the first group fixes the Taylor coefficients
    c_r = kappa^(r)(a) / r! (r <= p); the second is a p x p linear system for
    c_{p+1..2p}.
    """
    a = tau - eps_B
    deg = 2 * p
    der = kappa_derivatives_at(a, eta, p)
    c = np.zeros(deg + 1)
    for r in range(p + 1):
        c[r] = der[r] / math.factorial(r)
    if p > 0:
        # d^r/dt^r sum_j c_j t^j at t = eps_B equals sum_{j>=r} c_j j!/(j-r)! eps_B^(j-r)
        A = np.zeros((p, p))
        rhs = np.zeros(p)
        for row, r in enumerate(range(1, p + 1)):
            for j in range(r, deg + 1):
                coef = math.factorial(j) / math.factorial(j - r) * eps_B ** (j - r)
                if j > p:
                    A[row, j - p - 1] += coef
                else:
                    rhs[row] -= coef * c[j]
        c[p + 1:] = np.linalg.solve(A, rhs)
    Pt = Polynomial(c)
    return Pt(Polynomial([-a, 1.0]))  # substitute t = x - a


def kappa_R(r, eta: float, tau: float, eps_B: float, p: int):
    """Eq. (Ker-reg): regularised kernel as a function of |x| (r >= 0)."""
    r = np.abs(np.asarray(r, dtype=np.float64))
    kB = boundary_polynomial(eta, tau, eps_B, p)
    out = np.empty_like(r)
    inner = r <= tau - eps_B
    mid = (r > tau - eps_B) & (r <= tau)
    outer = r > tau
    out[inner] = kappa(r[inner], eta)
    out[mid] = kB(r[mid])
    out[outer] = kB(tau)
    return out


def kappa_tilde(x, eta: float, tau: float, eps_B: float, p: int):
    """Eq. (kappa_tilde): 2 tau-periodic kernel kappa_R(||x||) for x in [-tau, tau)^d.

    ``x`` has shape (..., d); points outside [-tau, tau)^d are first reduced
    into it by the period 2 tau.
    """
    x = np.asarray(x, dtype=np.float64)
    xr = (x + tau) % (2.0 * tau) - tau
    return kappa_R(np.sqrt((xr * xr).sum(axis=-1)), eta, tau, eps_B, p)


def kappa_hat(eta: float, tau: float, eps_B: float, p: int, M: int, d: int) -> np.ndarray:
    """Eq. (fft): kappa_hat(m) = (2M)^-d sum_{x in (tau/M){-M..M-1}^d} kappa_tilde(x) e^{-i pi m.x/tau}.

    Returned as a real array of shape (2M,)*d indexed by m + M (the
    coefficients of the real, even kernel are real; the imaginary part left by
    rounding is dropped after a check).
    """
    j = np.arange(-M, M)
    xs = tau * j / M
    grids = np.meshgrid(*([xs] * d), indexing="ij")
    pts = np.stack(grids, axis=-1)
    samples = kappa_tilde(pts, eta, tau, eps_B, p)
    # numpy's FFT sums over index q = j mod 2M with e^{-2 pi i m q/(2M)} = e^{-i pi m x/tau}
    F = np.fft.fftn(np.fft.ifftshift(samples)) / float(2 * M) ** d
    F = np.fft.fftshift(F)
    assert np.max(np.abs(F.imag)) <= 1e-12 * max(1.0, np.max(np.abs(F.real)))
    return F.real.copy()


def _as2d(x):
    x = np.asarray(x, dtype=np.float64)
    return x[:, None] if x.ndim == 1 else x


def direct_sum(x_tgt, x_src, alpha, eta: float, block: int = 2048) -> np.ndarray:
    """Eq. (fastsum-sum): beta_i = sum_j alpha_j exp(-||x_i - y_j||^2 / eta), FP64.

    ``alpha`` may have shape (n_src,) or (n_src, r) for r right-hand sides.
    Evaluated block by block over the targets to bound memory.
    """
    xt = _as2d(x_tgt)
    xs = _as2d(x_src)
    a = np.asarray(alpha, dtype=np.float64)
    out = np.empty((xt.shape[0],) + a.shape[1:])
    for s in range(0, xt.shape[0], block):
        diff = xt[s:s + block, None, :] - xs[None, :, :]
        Kb = np.exp(-(diff * diff).sum(axis=-1) / eta)
        out[s:s + block] = Kb @ a
    return out


def truncated_sum(x_tgt, x_src, alpha, eta: float, r_cut: float, block: int = 2048) -> np.ndarray:
    """Eq. (fastsum-sum) with every term of ||x_i - y_j|| > r_cut left out, FP64.

    The truncation the paper suggests for very small eta, where the kernel is
    concentrated near zero.  Each left-out term is at most exp(-r_cut^2/eta)
    |alpha_j|, so |truncated - direct| <= exp(-r_cut^2/eta) sum_j |alpha_j|.
    """
    xt = _as2d(x_tgt)
    xs = _as2d(x_src)
    a = np.asarray(alpha, dtype=np.float64)
    out = np.empty((xt.shape[0],) + a.shape[1:])
    r2 = float(r_cut) * float(r_cut)
    for s in range(0, xt.shape[0], block):
        diff = xt[s:s + block, None, :] - xs[None, :, :]
        d2 = (diff * diff).sum(axis=-1)
        Kb = np.where(d2 <= r2, np.exp(-d2 / eta), 0.0)
        out[s:s + block] = Kb @ a
    return out


def log_kernel_sum(x_tgt, x_src, log_v, eta: float, r_cut: float | None = None, block: int = 2048) -> np.ndarray:
    """log beta_i = log sum_j exp(log_v_j - ||x_i - y_j||^2 / eta), FP64.

    Eq. (fastsum-sum) with positive weights v_j = exp(log_v_j) held as their
    logarithms: each target's exponents are shifted by their maximum before
    summing (log-sum-exp), so no term overflows or underflows to an all-zero
    sum.  With ``r_cut`` only the pairs with ||x_i - y_j|| <= r_cut enter
    (``truncated_sum`` in log form).  -inf where no term is left.
    """
    xt = _as2d(x_tgt)
    xs = _as2d(x_src)
    lv = np.asarray(log_v, dtype=np.float64)
    out = np.empty(xt.shape[0])
    for s in range(0, xt.shape[0], block):
        diff = xt[s:s + block, None, :] - xs[None, :, :]
        d2 = (diff * diff).sum(axis=-1)
        E = lv[None, :] - d2 / eta
        if r_cut is not None:
            E = np.where(d2 <= float(r_cut) * float(r_cut), E, -np.inf)
        m = np.max(E, axis=1)
        finite = np.isfinite(m)
        shift = np.where(finite, m, 0.0)
        with np.errstate(divide="ignore"):
            out[s:s + block] = np.where(finite, shift + np.log(np.exp(E - shift[:, None]).sum(axis=1)), -np.inf)
    return out


def kernel_matrix(x_rows, x_cols, eta: float) -> np.ndarray:
    """Eq. (K-matrix): K_ij = exp(-||x_i - y_j||^2 / eta) as a dense FP64 matrix."""
    xr = _as2d(x_rows)
    xc = _as2d(x_cols)
    diff = xr[:, None, :] - xc[None, :, :]
    return np.exp(-(diff * diff).sum(axis=-1) / eta)


def _fourier_factors(x, M: int, tau: float, sign: float) -> np.ndarray:
    """exp(sign * i pi m x_t / tau) for m in {-M..M-1}, per point and dimension: (n, d, 2M)."""
    m = np.arange(-M, M, dtype=np.float64)
    x = _as2d(x)
    return np.exp(sign * 1j * math.pi / tau * x[:, :, None] * m[None, None, :])


_LETTERS = "abc"


def adjoint_ndft(x_src, alpha, M: int, tau: float) -> np.ndarray:
    """Eq. (ndft*): [F*_l alpha]_m = sum_j alpha_j exp(-i pi m.x_j / tau), m in {-M..M-1}^d.

    The exponential factorises over the coordinates, so the sum is one
    einsum over j of alpha_j times d per-coordinate factors.  Returns a
    complex array of shape (2M,)*d indexed by m + M.
    """
    E = _fourier_factors(x_src, M, tau, -1.0)
    d = E.shape[1]
    spec = "j," + ",".join("j" + _LETTERS[t] for t in range(d)) + "->" + _LETTERS[:d]
    return np.einsum(spec, np.asarray(alpha, dtype=np.float64), *[E[:, t, :] for t in range(d)])


def ndft(x_tgt, coeffs: np.ndarray, M: int, tau: float) -> np.ndarray:
    """sum_m coeffs(m) exp(+i pi m.x_i / tau) at each target (the sign of Eq. fastsum1)."""
    E = _fourier_factors(x_tgt, M, tau, +1.0)
    d = E.shape[1]
    spec = _LETTERS[:d] + "," + ",".join("i" + _LETTERS[t] for t in range(d)) + "->i"
    return np.einsum(spec, np.asarray(coeffs), *[E[:, t, :] for t in range(d)])


def fastsum_ndft(x_tgt, x_src, alpha, eta: float, tau: float, eps_B: float, p: int, M: int) -> np.ndarray:
    """Algorithm 4 with the NDFTs done directly: beta ~ Re F_k(kappa_hat * F*_l alpha).

    Steps in the paper's order: kappa_R (Eq. Ker-reg) -> kappa_tilde
    (Eq. kappa_tilde) -> kappa_hat by FFT (Eq. fft) -> adjoint NDFT
    (Eq. ndft*) -> pointwise product -> NDFT (Eq. fastsum1) -> real part.
    Cost O(M^d (n_src + n_tgt)); used for small cases to separate the Fourier
    truncation error of the method from the window error of an NFFT.
    """
    xs = _as2d(x_src)
    d = xs.shape[1]
    kh = kappa_hat(eta, tau, eps_B, p, M, d)
    a_hat = adjoint_ndft(xs, alpha, M, tau)
    b = ndft(_as2d(x_tgt), kh * a_hat, M, tau)
    return b.real
