"""Host logic of the wavefront schedule (no GPU): the launch plan that `mot_wave_schedule`
returns -- the one the solver builds for trees on the fused 2-D path -- respects every data
dependency of Algorithm 2's sweeps and every write-after-read hazard of the two beta copies, never
exceeds the per-launch cap, and, executed launch by launch with dense kernels, reproduces the
sweep-by-sweep iterates exactly.

Sweep s of Algorithm 2 with the forward identity phi^p gamma_p beta^{C_p minus k} = mu^p / beta_k
(valid right after phi^p's update) is: F_k(s) gamma_k = K^T (mu^p / beta_k) and phi^k = mu^k /
(gamma_k prod_{c in C_k} beta_c); R(s) phi^1 = mu^1 / prod_{c in C_1} beta_c; B_k(s) beta_k =
K (phi^k prod_{c in C_k} beta_c), children before parents.
"""
import numpy as np
import pytest

from paper_2208_03120_gb300 import workloads as W


@pytest.fixture(scope="module")
def M():
    from paper_2208_03120_gb300 import build, motfft
    build.build()
    return motfft


def _children(parent):
    ch = [[] for _ in parent]
    for k in range(1, len(parent)):
        ch[parent[k]].append(k)
    return ch


def _trees():
    rng = np.random.default_rng(3)
    out = {"path10_centre": [-1, 0, 0, 1, 2, 3, 4, 5, 6, 7],     # the 10-node path rooted at a centre
           "path10_end": [-1] + list(range(9)),
           "star9": [-1] + [0] * 8,
           "two_nodes": [-1, 0]}
    for i in range(4):
        K = int(rng.integers(3, 21))
        out[f"random{i}"] = [-1] + [int(rng.integers(0, k)) for k in range(1, K)]
    return out


def _check_constraints(parent, S, cap, F, B, R, carrier, n):
    K = len(parent)
    ch = _children(parent)
    load = np.zeros(n, dtype=int)
    for s in range(S):
        load[R[s]] += 1
        for k in range(1, K):
            load[F[s][k]] += 1
            load[B[s][k]] += 1
    assert load.max() <= cap and load.min() >= 1 and load.sum() == S * (2 * (K - 1) + 1)
    for s in range(S):
        for k in range(1, K):
            if s > 0:
                assert F[s][k] > B[s - 1][k]
                assert all(F[s][k] > B[s - 1][c] for c in ch[k])
            assert B[s][k] > F[s][k]
            assert all(B[s][k] > B[s][c] for c in ch[k])
            if s > 0:                           # the copy it overwrites was read in sweep s-1
                p = parent[k]
                assert B[s][k] > F[s - 1][k]
                assert B[s][k] > (R[s - 1] if p == 0 else F[s - 1][p])
        if s > 0:
            assert all(R[s] > B[s - 1][c] for c in ch[0])
            c = carrier[s]
            assert c in ch[0] and R[s - 1] < B[s - 1][c] < R[s]
    assert carrier[0] == -1


@pytest.mark.parametrize("cap", [1, 2, 7, 20])
@pytest.mark.parametrize("S", [1, 2, 3, 10, 32])
def test_schedule_respects_dependencies_and_cap(M, S, cap):
    for name, parent in _trees().items():
        F, B, R, carrier, n = M.wave_schedule(parent, S, cap)
        _check_constraints(parent, S, cap, F, B, R, carrier, n)


def _run_sequential(parent, Km, mu, beta0, sweeps):
    K = len(parent)
    ch = _children(parent)
    prod = lambda vs, m: np.prod(vs, axis=0) if vs else np.ones(m)
    beta = list(beta0)
    for _ in range(sweeps):
        phi = [None] * K
        for k in range(1, K):
            g = Km[k].T @ (mu[parent[k]] / beta[k])
            phi[k] = mu[k] / (g * prod([beta[c] for c in ch[k]], len(mu[k])))
        phi[0] = mu[0] / prod([beta[c] for c in ch[0]], len(mu[0]))
        for k in range(K - 1, 0, -1):
            beta[k] = Km[k] @ (phi[k] * prod([beta[c] for c in ch[k]], len(mu[k])))
    return phi, beta


def _run_wave(M, parent, Km, mu, beta0, S, chunks, cap):
    """Execute the schedule launch by launch: each launch reads the state as it was before the
    launch and writes afterwards; beta in two copies alternating by sweep."""
    K = len(parent)
    ch = _children(parent)
    prod = lambda vs, m: np.prod(vs, axis=0) if vs else np.ones(m)
    copies = [list(beta0), [None] * K]
    phi = [np.ones(len(m)) for m in mu]
    q0 = 0
    for _ in range(chunks):
        F, B, R, carrier, n = M.wave_schedule(parent, S, cap)
        for t in range(n):
            writes = []
            for s in range(S):
                q = (q0 + s) & 1
                for k in range(1, K):
                    if F[s][k] == t:
                        g = Km[k].T @ (mu[parent[k]] / copies[q][k])
                        writes.append(("phi", k, mu[k] / (g * prod([copies[q][c] for c in ch[k]], len(mu[k])))))
                    if B[s][k] == t:
                        v = Km[k] @ (phi[k] * prod([copies[q ^ 1][c] for c in ch[k]], len(mu[k])))
                        writes.append(("beta", (q ^ 1, k), v))
                if R[s] == t:
                    writes.append(("phi", 0, mu[0] / prod([copies[q][c] for c in ch[0]], len(mu[0]))))
            for kind, key, v in writes:
                if kind == "phi":
                    phi[key] = v
                else:
                    copies[key[0]][key[1]] = v
        q0 = (q0 + S) & 1
    return phi, copies[q0]


@pytest.mark.parametrize("S,chunks,cap", [(10, 2, 7), (3, 3, 2), (7, 2, 20), (1, 4, 1), (32, 1, 7)])
def test_schedule_reproduces_sweep_by_sweep_iterates(M, S, chunks, cap):
    rng = np.random.default_rng(S * 100 + cap)
    for name, parent in _trees().items():
        K = len(parent)
        n = [int(rng.integers(3, 7)) for _ in range(K)]
        Km = [None] + [rng.uniform(0.1, 1.0, (n[parent[k]], n[k])) for k in range(1, K)]
        mu = [rng.uniform(0.1, 1.0, m) for m in n]
        mu = [m / m.sum() for m in mu]
        ch = _children(parent)
        beta0 = [None] * K
        for k in range(K - 1, 0, -1):
            beta0[k] = Km[k] @ np.prod([beta0[c] for c in ch[k]], axis=0) if ch[k] else Km[k] @ np.ones(n[k])
        ps, bs = _run_sequential(parent, Km, mu, beta0, S * chunks)
        pw, bw = _run_wave(M, parent, Km, mu, beta0, S, chunks, cap)
        for a, b in zip(ps, pw):
            np.testing.assert_array_equal(a, b)
        for a, b in zip(bs[1:], bw[1:]):
            np.testing.assert_array_equal(a, b)


def test_schedule_shortens_the_headline_chunk(M):
    """The 10-node path rooted at a centre, 10 sweeps, seven products per launch (the clusters
    that fit on a GB300): 30 launches where the sweep-by-sweep order takes 60."""
    parent = _trees()["path10_centre"]
    F, B, R, carrier, n = M.wave_schedule(parent, 10, 7)
    assert n <= 30


def test_schedule_rejects_bad_trees(M):
    with pytest.raises(M.MotError):
        M.wave_schedule([-1, 1, 0], 3, 4)          # parent[k] >= k
    with pytest.raises(M.MotError):
        M.wave_schedule([0, 0], 3, 4)              # no root
    with pytest.raises(M.MotError):
        M.wave_schedule([-1, 0], 0, 4)             # no sweeps
