"""Seeded synthetic inputs shaped like the paper's experiments (Section 6).

This module draws random point clouds, marginal weights and graph structures.
It holds none of the method's arithmetic: no kernel, no transform, no Sinkhorn
step.  Both the CUDA path and the FP64 oracle receive exactly the arrays
returned here, so that every comparison is made on identical inputs.

Points are generated in float64, rounded to float32 (the precision the CUDA
path stores), and the rounded values are handed to both sides (the oracle
promotes them back to float64).  Weights are float64, non-negative, sum 1.

Workloads (seed = 2208031200 + workload index):

* ``path3_d1``   -- path tree 1-2-3, d=1, N=100 per marginal, x ~ U[-0.2, 0.2],
  mu ~ U(0,1) normalised, eta=0.05 (Section 6.1 shape, small enough for brute
  force over the full N^K tensor).
* ``path10_d2``  -- path tree of 10 nodes, d=2, N=10,000 per marginal drawn
  from one 3-component Gaussian mixture (sigma=0.05; centres uniform in the
  ball of radius 0.12) and radially projected onto the ball of radius 0.24;
  Dirichlet(1) weights; eta=0.01 (the d=2, K=10, N=10^4 shape of Fig. 6).
* ``star9_d3``   -- star tree, centre = root plus 8 leaves, d=3, N=50,000 per
  marginal uniform in the ball of radius 0.24, uniform weights, eta=0.02
  (barycenter-like tree of Section 6.2).
* ``circle5_d1`` -- circle of K=5 marginals, d=1, N=2,000 uniform in
  [-0.24, 0.24], weights U(0,1) normalised, eta=0.05 (Section 6.1 circle).
* ``euler5_d1``  -- generalised Euler flow (Section 6.3): circle of K=5
  marginals, d=1, N=400 points uniform on [0, 1] per time step, uniform
  weights, eta=0.05, closing edge against sigma(x^1) with the connection map
  sigma(x) = 1 - x or sigma(x) = min(2x, 2 - 2x).
* ``serving``    -- a Poisson-arrival stream of solve requests mixing the
  three topologies (see :func:`serving_stream`).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

SEED_BASE = 2208031200

TREE = 0
CIRCLE = 1


@dataclasses.dataclass
class Problem:
    """One multi-marginal problem instance (Section 2 notation)."""

    name: str
    topology: int                      # TREE or CIRCLE
    K: int                             # number of marginals
    d: int                             # space dimension
    x: List[np.ndarray]                # K arrays, float32, shape (n_k, d)
    mu: List[np.ndarray]               # K arrays, float64, shape (n_k,), sum 1
    eta: float                         # entropic regularisation
    edges: Optional[np.ndarray]        # tree: int32 (K-1, 2) node pairs; circle: None
    edge_w: Optional[np.ndarray] = None  # per-edge cost weights (None = 1)
    root: int = 0
    iters: int = 0                     # suggested iteration count (0 = to tolerance)
    x_close: Optional[np.ndarray] = None  # circle: sigma(x^1), float32 (n_1, d), used by the
                                          # closing edge {K, 1} in place of x^1 (Section 6.3)

    @property
    def n(self) -> List[int]:
        return [int(a.shape[0]) for a in self.x]

    def x64(self) -> List[np.ndarray]:
        return [a.astype(np.float64) for a in self.x]

    def x_close64(self) -> Optional[np.ndarray]:
        return None if self.x_close is None else self.x_close.astype(np.float64)


def _rng(index: int, seed: Optional[int] = None) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + index if seed is None else seed))


def _normalised(w: np.ndarray) -> np.ndarray:
    w = np.asarray(w, dtype=np.float64)
    return w / w.sum()


def path_edges(K: int) -> np.ndarray:
    return np.array([[k, k + 1] for k in range(K - 1)], dtype=np.int32)


def star_edges(K: int) -> np.ndarray:
    return np.array([[0, k] for k in range(1, K)], dtype=np.int32)


def uniform_ball(rng: np.random.Generator, n: int, d: int, radius: float) -> np.ndarray:
    """Uniform points in the d-ball: Gaussian direction, radius * U^(1/d)."""
    g = rng.standard_normal((n, d))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    r = radius * rng.random(n) ** (1.0 / d)
    return g * r[:, None]


def gaussian_mixture_clipped(rng: np.random.Generator, n: int, d: int, centres: np.ndarray,
                             sigma: float, radius: float) -> np.ndarray:
    """Equal-weight Gaussian mixture; points outside the ball are projected radially onto it."""
    comp = rng.integers(0, centres.shape[0], size=n)
    x = centres[comp] + sigma * rng.standard_normal((n, d))
    r = np.linalg.norm(x, axis=1)
    far = r > radius
    x[far] *= (radius / r[far])[:, None]
    return x


def path3_d1(n: int = 100, seed: Optional[int] = None) -> Problem:
    rng = _rng(0, seed)
    K, d = 3, 1
    x = [rng.uniform(-0.2, 0.2, size=(n, d)).astype(np.float32) for _ in range(K)]
    mu = [_normalised(rng.uniform(0.0, 1.0, size=n)) for _ in range(K)]
    return Problem("path3_d1", TREE, K, d, x, mu, 0.05, path_edges(K), iters=200)


def path10_d2(n: int = 10_000, K: int = 10, seed: Optional[int] = None) -> Problem:
    rng = _rng(1, seed)
    d = 2
    centres = uniform_ball(rng, 3, d, 0.12)
    x = [gaussian_mixture_clipped(rng, n, d, centres, 0.05, 0.24).astype(np.float32) for _ in range(K)]
    mu = [_normalised(rng.exponential(1.0, size=n)) for _ in range(K)]  # Dirichlet(1)
    return Problem("path10_d2", TREE, K, d, x, mu, 0.01, path_edges(K))


def star9_d3(n: int = 50_000, leaves: int = 8, seed: Optional[int] = None) -> Problem:
    rng = _rng(2, seed)
    d, K = 3, leaves + 1
    x = [uniform_ball(rng, n, d, 0.24).astype(np.float32) for _ in range(K)]
    mu = [np.full(n, 1.0 / n) for _ in range(K)]
    return Problem("star9_d3", TREE, K, d, x, mu, 0.02, star_edges(K))


def circle5_d1(n: int = 2_000, K: int = 5, seed: Optional[int] = None) -> Problem:
    rng = _rng(3, seed)
    d = 1
    x = [rng.uniform(-0.24, 0.24, size=(n, d)).astype(np.float32) for _ in range(K)]
    mu = [_normalised(rng.uniform(0.0, 1.0, size=n)) for _ in range(K)]
    return Problem("circle5_d1", CIRCLE, K, d, x, mu, 0.05, None)


# Connection maps of Section 6.3 (the problem's input, applied to the initial positions).
# "fold" reads the printed min(2x, 1 - 2x), which leaves [0, 1], as the tent map min(2x, 2 - 2x).
CONNECTION_MAPS = {
    "reflect": lambda x: 1.0 - x,
    "fold": lambda x: np.minimum(2.0 * x, 2.0 - 2.0 * x),
}


def euler5_d1(n: int = 400, K: int = 5, sigma: str = "reflect", seed: Optional[int] = None) -> Problem:
    rng = _rng(4, seed)
    d = 1
    x = [rng.uniform(0.0, 1.0, size=(n, d)).astype(np.float32) for _ in range(K)]
    mu = [np.full(n, 1.0 / n) for _ in range(K)]
    x_close = CONNECTION_MAPS[sigma](x[0].astype(np.float64)).astype(np.float32)
    return Problem(f"euler5_d1_{sigma}", CIRCLE, K, d, x, mu, 0.05, None, x_close=x_close)


def random_tree_edges(rng: np.random.Generator, K: int) -> np.ndarray:
    """Uniformly random recursive tree on K nodes with shuffled labels."""
    labels = rng.permutation(K)
    edges = [[int(labels[int(rng.integers(0, k))]), int(labels[k])] for k in range(1, K)]
    return np.array(edges, dtype=np.int32)


def random_problem(rng: np.random.Generator, topology: int, K: int, d: int, n: Sequence[int] | int,
                   eta: float, shape: str = "tree-random", radius: float = 0.24) -> Problem:
    """Small random instance for tests: uniform points in a ball, U(0,1) weights."""
    if isinstance(n, int):
        n = [n] * K
    x = [uniform_ball(rng, n[k], d, radius).astype(np.float32) for k in range(K)]
    mu = [_normalised(rng.uniform(0.05, 1.0, size=n[k])) for k in range(K)]
    if topology == CIRCLE:
        edges = None
    elif shape == "path":
        edges = path_edges(K)
    elif shape == "star":
        edges = star_edges(K)
    else:
        edges = random_tree_edges(rng, K)
    return Problem(f"random-{shape}", topology, K, d, x, mu, eta, edges)


@dataclasses.dataclass
class Request:
    arrival_s: float
    problem: Problem


def serving_stream(n_requests: int = 2000, rate_hz: float = 100.0, seed: Optional[int] = None,
                   n_range: Tuple[int, int] = (500, 20_000), k_range: Tuple[int, int] = (3, 20),
                   circle_n_max=None) -> List[Request]:
    """Poisson arrivals; topology uniform over {path, star, circle}; K ~ U{3..20};
    d ~ U{1,2,3}; N log-uniform on [500, 20000]; eta in {0.01, 0.05, 0.1}.
    ``circle_n_max`` caps N of circle requests (their cost grows as K N^2): an int for every
    dimension, or a dict {d: cap} (dimensions not listed are not capped)."""
    rng = _rng(4, seed)
    t = 0.0
    out = []
    for i in range(n_requests):
        t += rng.exponential(1.0 / rate_hz)
        kind = int(rng.integers(0, 3))
        K = int(rng.integers(k_range[0], k_range[1] + 1))
        d = int(rng.integers(1, 4))
        N = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        eta = float(rng.choice([0.01, 0.05, 0.1]))
        sub = np.random.Generator(np.random.PCG64(int(rng.integers(0, 2**63 - 1))))
        if kind == 2:
            cap = circle_n_max.get(d) if isinstance(circle_n_max, dict) else circle_n_max
            if cap is not None:
                N = min(N, cap)
            prob = random_problem(sub, CIRCLE, K, d, N, eta)
        else:
            prob = random_problem(sub, TREE, K, d, N, eta, shape="path" if kind == 0 else "star")
        prob.name = f"req{i}"
        out.append(Request(t, prob))
    return out


WORKLOADS = {
    "path3_d1": path3_d1,
    "path10_d2": path10_d2,
    "star9_d3": star9_d3,
    "circle5_d1": circle5_d1,
}
