"""FP64 CPU oracle for NFFT-accelerated multi-marginal Sinkhorn (Ba & Quellmalz, 2022).

TEST INFRASTRUCTURE ONLY.  Nothing here is part of the product path: only the
test suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference leg
of ``bench.py`` may import or run it.  It shares no code with the CUDA library
(no kernels, headers, helpers, tables or constant generators) and imports
nothing from the package except through the callers, who pass it plain
NumPy arrays.

Contents
--------
``oracle.kernel``   -- the Gaussian kernel, its boundary regularisation
                       (Eq. Ker-reg, Fig. 3), periodisation (Eq. kappa_tilde),
                       Fourier coefficients by FFT (Eq. fft), direct summation
                       (Eq. fastsum-sum) and the fast-summation approximation
                       written with direct NDFTs (Eqs. ndft, ndft*, fastsum_mat,
                       Algorithm 4).
``oracle.sinkhorn`` -- tree structure (Section 4.1), dense Sinkhorn for trees
                       (Algorithm 2) and circles (Algorithm 3), message-passing
                       marginals (Theorems 4.1 and 4.3), dual / primal values and
                       marginal violation, and brute force over the full N^K
                       tensor (Eq. K-sparse, Algorithm 1) for tiny cases.

Every function works in float64 and follows the paper's steps in its order and
notation; library primitives (numpy FFT, matmul, linear solve) serve as steps.
All functions are pinned by ``tests/test_oracle_*.py`` against values or
properties fixed by the paper or by mathematics (see each test's docstring).
"""
from . import kernel, sinkhorn  # noqa: F401
