"""Write the oracle's converged solutions of the full-size workloads to tests/golden/.

Calls only ``oracle/`` (and the seeded input generator, which holds none of the
method's arithmetic).  Nothing here touches the CUDA library.  Each golden file is
JSON with:

  * ``inputs_crc``: CRC-32 of the generated points and weights, so that a test can
    check that it regenerated the same inputs;
  * the oracle's sweep count, marginal violation (exact FP64 kernels), dual value S
    (Eq. dual_problem), primal value (Eq. MOTe) and total mass at its final scalings;
  * the gauge-fixed potentials u^k = eta log phi^k (``oracle.sinkhorn.gauge_fix`` on the
    full vectors) at a seeded sample of point indices per marginal.

Workloads (the bench's shapes):
  * path10_d2       -- Algorithm 2, path of 10, d=2, N=10^4, eta=0.01;
  * star9_d3_n5000  -- Algorithm 2, star (centre + 8 leaves), d=3, N=5000, eta=0.02;
  * circle5_d1      -- Algorithm 3, circle of 5, d=1, N=2000, eta=0.05.
Each is run in chunks of sweeps from phi = 1 until the exact violation is at most
``TOL`` (or the sweep cap), far below the 1e-6 the CUDA path stops at, so that the
golden stands for the fixed point.

  * local_path5_d2 -- Algorithm 2 in the log domain with every kernel sum truncated to
                      |x - y| <= sqrt(40 eta) (Section 6.1, closing remark): path of 5, d=2,
                      N=400, eta=2e-3 (a regime the FP32 scaling form cannot span); the
                      potentials are stored as log phi^k.

Usage: python tests/golden/make_oracle_goldens.py [path10_d2|star9_d3_n5000|circle5_d1|local_path5_d2 ...]
"""
from __future__ import annotations

import json
import os
import sys
import time
import zlib

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import sinkhorn as OS  # noqa: E402
from paper_2208_03120_gb300 import workloads as W  # noqa: E402

TOL = 1e-9
SAMPLES = 400


def inputs_crc(prob) -> int:
    c = 0
    for a in prob.x:
        c = zlib.crc32(np.ascontiguousarray(a, dtype=np.float32).tobytes(), c)
    for m in prob.mu:
        c = zlib.crc32(np.ascontiguousarray(m, dtype=np.float64).tobytes(), c)
    return c


def sample_indices(n: int, k: int) -> np.ndarray:
    rng = np.random.default_rng(1000 + k)
    return np.sort(rng.choice(n, size=min(SAMPLES, n), replace=False))


def tree_report(prob, phi):
    P = OS.tree_marginals(prob.x64(), phi, prob.edges, prob.eta, root=prob.root, edge_w=prob.edge_w)
    mass = OS.total_mass(P)
    return dict(violation=OS.violation(P, prob.mu), dual=OS.dual_value(prob.mu, phi, mass, prob.eta),
                primal=OS.primal_value(P, phi, mass, prob.eta), mass=mass)


def circle_report(prob, phi):
    P = OS.circle_marginals(prob.x64(), phi, prob.eta, edge_w=prob.edge_w)
    mass = OS.total_mass(P)
    return dict(violation=OS.violation(P, prob.mu), dual=OS.dual_value(prob.mu, phi, mass, prob.eta),
                primal=OS.primal_value(P, phi, mass, prob.eta), mass=mass)


def solve(prob, chunk: int, cap: int):
    if prob.topology == W.TREE:
        solver = OS.TreeSinkhorn(prob.x64(), prob.mu, prob.edges, prob.eta, root=prob.root, edge_w=prob.edge_w)
        report = tree_report
    else:
        solver = OS.CircleSinkhorn(prob.x64(), prob.mu, prob.eta, edge_w=prob.edge_w)
        report = circle_report
    phi, sweeps, S = None, 0, []
    t0 = time.time()
    while True:
        res = solver.run(chunk, phi0=phi)
        phi, sweeps = res.phi, sweeps + res.iters
        S += res.S
        rep = report(prob, phi)
        print(f"  {prob.name}: {sweeps} sweeps, violation {rep['violation']:.3e}, S {rep['dual']:.12f} "
              f"({time.time() - t0:.0f} s)", flush=True)
        if rep["violation"] <= TOL or sweeps >= cap:
            return phi, sweeps, S, rep


def write(name: str, prob, chunk: int, cap: int, extra: dict) -> None:
    print(f"{name}: K={prob.K} d={prob.d} n={prob.n[0]} eta={prob.eta}", flush=True)
    # keep every edge's kernel matrix in memory (10^8 FP64 entries per edge at N = 10^4): the same
    # products, formed once instead of block by block at every sweep
    OS.EdgeKernel.DENSE_LIMIT = max(OS.EdgeKernel.DENSE_LIMIT, max(prob.n) ** 2)
    phi, sweeps, S, rep = solve(prob, chunk, cap)
    u = OS.gauge_fix([prob.eta * np.log(p) for p in phi], prob.mu)
    idx = [sample_indices(len(v), k) for k, v in enumerate(u)]
    doc = dict(workload=name, K=prob.K, d=prob.d, n=prob.n, eta=prob.eta, inputs_crc=inputs_crc(prob),
               oracle_sweeps=sweeps, S_trace_tail=S[-5:], **rep, **extra,
               index=[i.tolist() for i in idx], u=[v[i].tolist() for v, i in zip(u, idx)],
               u_span=[float(np.max(v) - np.min(v)) for v in u])
    with open(os.path.join(HERE, f"oracle_{name}.json"), "w") as f:
        json.dump(doc, f, indent=0)
        f.write("\n")


def local_problem():
    return W.random_problem(np.random.default_rng(5), W.TREE, 5, 2, 400, 2e-3, shape="path")


def write_local(name: str) -> None:
    import math
    prob = local_problem()
    r_cut = math.sqrt(40.0 * prob.eta)
    print(f"{name}: K={prob.K} d={prob.d} n={prob.n[0]} eta={prob.eta} r_cut={r_cut}", flush=True)
    ts = OS.TreeSinkhornLog(prob.x64(), prob.mu, prob.edges, prob.eta, r_cut=r_cut)
    f, sweeps, S = None, 0, []
    t0 = time.time()
    while True:
        res = ts.run(50, logphi0=f)
        f, sweeps = res.logphi, sweeps + res.iters
        S += res.S
        lp = OS.tree_marginals_log(prob.x64(), f, prob.edges, prob.eta, r_cut=r_cut)
        P = [np.exp(a) for a in lp]
        viol = OS.violation(P, prob.mu)
        mass = float(P[0].sum())
        dual = prob.eta * (sum(float(np.sum(np.where(m > 0, m * fk, 0.0))) for m, fk in zip(prob.mu, f)) - mass)
        print(f"  {name}: {sweeps} sweeps, violation {viol:.3e}, S {dual:.12e} ({time.time() - t0:.0f} s)", flush=True)
        if viol <= 1e-8 or sweeps >= 2000:
            break
    g = OS.gauge_fix(f, prob.mu)
    doc = dict(workload=name, K=prob.K, d=prob.d, n=prob.n, eta=prob.eta, r_cut=r_cut, inputs_crc=inputs_crc(prob),
               oracle_sweeps=sweeps, violation=viol, dual=dual, mass=mass, S_trace_tail=S[-5:],
               note="TreeSinkhornLog with r_cut rooted at node 0; logphi gauge-fixed (all points stored)",
               logphi=[v.tolist() for v in g])
    with open(os.path.join(HERE, f"oracle_{name}.json"), "w") as fh:
        json.dump(doc, fh, indent=0)
        fh.write("\n")


JOBS = {
    "local_path5_d2": lambda: write_local("local_path5_d2"),
    "path10_d2": lambda: write("path10_d2", W.path10_d2(), 20, 400,
                               dict(note="Algorithm 2 rooted at node 0; the fixed point does not depend on the root")),
    "star9_d3_n5000": lambda: write("star9_d3_n5000", W.star9_d3(n=5000), 20, 600,
                                    dict(note="Algorithm 2 rooted at the centre (node 0)")),
    "circle5_d1": lambda: write("circle5_d1", W.circle5_d1(), 20, 600, dict(note="Algorithm 3")),
}


if __name__ == "__main__":
    names = sys.argv[1:] or list(JOBS)
    for nm in names:
        JOBS[nm]()
