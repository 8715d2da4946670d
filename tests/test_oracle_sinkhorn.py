"""Pins of the FP64 oracle's Sinkhorn pieces (no GPU).

The message-passing marginals and the tree / circle algorithms are checked
against brute force over the full N^K tensor built directly from the cost
(Eq. cost_sparse), against Algorithm 1 iterate by iterate where the paper's
algorithms coincide with it, against the classical two-marginal Sinkhorn, and
against the invariants the theory fixes (duality, monotonicity, symmetry,
scale invariance).
"""
import math

import numpy as np
import pytest

from oracle import sinkhorn as OS
from paper_2208_03120_gb300 import workloads as W


def _rand_phi(rng, n):
    return [rng.uniform(0.3, 3.0, size=k) for k in n]


def _tree_graph_edges(edges):
    return [(int(a), int(b)) for a, b in edges]


def _circle_graph_edges(K):
    return [(k, (k + 1) % K) for k in range(K)]


@pytest.mark.parametrize("shape", ["path", "star", "tree-random"])
@pytest.mark.parametrize("d", [1, 2, 3])
def test_tree_marginals_match_bruteforce(shape, d):
    """Theorem 4.1: P_k(K (.) Phi) by the beta / gamma recursions equals the
    marginal of the full tensor K (.) Phi for arbitrary positive phi."""
    rng = np.random.default_rng(10 + d)
    K = 5
    prob = W.random_problem(rng, W.TREE, K, d, [3, 4, 2, 3, 4], eta=0.3, shape=shape)
    phi = _rand_phi(rng, prob.n)
    P_mp = OS.tree_marginals(prob.x64(), phi, prob.edges, prob.eta, root=int(rng.integers(0, K)))
    Kt = OS.full_kernel_tensor(prob.x64(), _tree_graph_edges(prob.edges), prob.eta)
    P_bf = OS.tensor_marginals(OS.plan_tensor(Kt, phi))
    for a, b in zip(P_mp, P_bf):
        np.testing.assert_allclose(a, b, rtol=1e-12)


@pytest.mark.parametrize("K", [3, 4, 5])
def test_circle_marginals_match_bruteforce(K):
    """Theorems 4.2 / 4.3: the circle's alpha / lambda matrix recursions give the
    marginals of the full tensor for arbitrary positive phi."""
    rng = np.random.default_rng(20 + K)
    n = [3, 4, 2, 3, 4][:K]
    prob = W.random_problem(rng, W.CIRCLE, K, 2, n, eta=0.3)
    phi = _rand_phi(rng, prob.n)
    P_mp = OS.circle_marginals(prob.x64(), phi, prob.eta)
    Kt = OS.full_kernel_tensor(prob.x64(), _circle_graph_edges(K), prob.eta)
    P_bf = OS.tensor_marginals(OS.plan_tensor(Kt, phi))
    for a, b in zip(P_mp, P_bf):
        np.testing.assert_allclose(a, b, rtol=1e-12)


def test_tree_structure_relabels_and_rejects():
    """Section 4.1: after relabelling every non-root node has p(k) < k and the
    edge set is preserved; a cycle or a disconnected graph is rejected."""
    rng = np.random.default_rng(3)
    edges = W.random_tree_edges(rng, 9)
    t = OS.tree_structure(9, edges, root=4)
    assert t.order[0] == 4
    for k in range(1, 9):
        assert t.parent[k] < k
    got = {frozenset((t.order[t.parent[k]], t.order[k])) for k in range(1, 9)}
    assert got == {frozenset(map(int, e)) for e in edges}
    with pytest.raises(ValueError):
        OS.tree_structure(4, [[0, 1], [1, 2], [2, 0]])
    with pytest.raises(ValueError):
        OS.tree_structure(4, [[0, 1], [2, 3], [0, 1]])


def test_path_tree_algorithm2_equals_algorithm1():
    """On a path rooted at an end, every gamma and beta that Algorithm 2 uses is
    current, so its sweep equals the Gauss-Seidel sweep of Algorithm 1 on the
    full tensor: the iterates agree sweep by sweep."""
    rng = np.random.default_rng(5)
    prob = W.random_problem(rng, W.TREE, 4, 2, [4, 3, 5, 4], eta=0.2, shape="path")
    ts = OS.TreeSinkhorn(prob.x64(), prob.mu, prob.edges, prob.eta)
    hist = []
    ts.run(6, callback=lambda r, phi: hist.append([p.copy() for p in phi]))
    Kt = OS.full_kernel_tensor(prob.x64(), _tree_graph_edges(prob.edges), prob.eta)
    bf = OS.sinkhorn_bruteforce(Kt, prob.mu, 6)
    for a, b in zip(hist, bf):
        for pa, pb in zip(a, b):
            np.testing.assert_allclose(pa, pb, rtol=1e-11)


def test_circle_algorithm3_equals_algorithm1():
    """Algorithm 3 updates phi^1..phi^K in order with current matrices, i.e. the
    Gauss-Seidel sweep of Algorithm 1 for the circle-structured cost."""
    rng = np.random.default_rng(6)
    prob = W.random_problem(rng, W.CIRCLE, 4, 1, [4, 3, 5, 4], eta=0.2)
    cs = OS.CircleSinkhorn(prob.x64(), prob.mu, prob.eta)
    hist = []
    cs.run(6, callback=lambda r, phi: hist.append([p.copy() for p in phi]))
    Kt = OS.full_kernel_tensor(prob.x64(), _circle_graph_edges(4), prob.eta)
    bf = OS.sinkhorn_bruteforce(Kt, prob.mu, 6)
    for a, b in zip(hist, bf):
        for pa, pb in zip(a, b):
            np.testing.assert_allclose(pa, pb, rtol=1e-11)


def test_star_tree_reaches_algorithm1_fixed_point():
    """For a star, Algorithm 2 uses the siblings' beta of the previous sweep, so
    only the fixed point is shared with Algorithm 1: the converged plans agree
    and reproduce every marginal (Proposition 3.2)."""
    rng = np.random.default_rng(8)
    prob = W.random_problem(rng, W.TREE, 5, 1, 3, eta=0.5, shape="star")
    ts = OS.TreeSinkhorn(prob.x64(), prob.mu, prob.edges, prob.eta)
    res = ts.run(400)
    Kt = OS.full_kernel_tensor(prob.x64(), _tree_graph_edges(prob.edges), prob.eta)
    bf = OS.sinkhorn_bruteforce(Kt, prob.mu, 400)[-1]
    Pi_a = OS.plan_tensor(Kt, res.phi)
    Pi_b = OS.plan_tensor(Kt, bf)
    np.testing.assert_allclose(Pi_a, Pi_b, rtol=1e-9, atol=1e-14)
    for Pk, m in zip(OS.tensor_marginals(Pi_a), prob.mu):
        np.testing.assert_allclose(Pk, m, rtol=1e-9)


def test_circle_with_unit_closing_edge_is_path_tree():
    """A circle whose closing edge {K, 1} has weight 0 (kernel identically 1) has
    the cost of the path 1-2-...-K: Algorithm 3 and Algorithm 2 produce the same
    iterates (both are the Gauss-Seidel sweep of Algorithm 1)."""
    rng = np.random.default_rng(9)
    prob = W.random_problem(rng, W.CIRCLE, 4, 2, [5, 4, 6, 3], eta=0.15)
    w = [1.0, 1.0, 1.0, 0.0]
    rc = OS.CircleSinkhorn(prob.x64(), prob.mu, prob.eta, edge_w=w).run(8)
    rt = OS.TreeSinkhorn(prob.x64(), prob.mu, W.path_edges(4), prob.eta).run(8)
    for a, b in zip(rc.phi, rt.phi):
        np.testing.assert_allclose(a, b, rtol=1e-11)
    np.testing.assert_allclose(rc.S, rt.S, rtol=1e-12)


def test_two_marginals_is_classical_sinkhorn():
    """K = 2 (one edge) reduces to two-marginal Sinkhorn: a = mu^1 / (K b),
    b = mu^2 / (K^T a), from a = b = 1 updated in that order."""
    rng = np.random.default_rng(11)
    prob = W.random_problem(rng, W.TREE, 2, 2, [7, 5], eta=0.1, shape="path")
    x0, x1 = prob.x64()
    Kmat = np.exp(-((x0[:, None, :] - x1[None, :, :]) ** 2).sum(-1) / prob.eta)
    a, b = np.ones(7), np.ones(5)
    for _ in range(25):
        a = prob.mu[0] / (Kmat @ b)
        b = prob.mu[1] / (Kmat.T @ a)
    res = OS.TreeSinkhorn(prob.x64(), prob.mu, prob.edges, prob.eta).run(25)
    np.testing.assert_allclose(res.phi[0], a, rtol=1e-12)
    np.testing.assert_allclose(res.phi[1], b, rtol=1e-12)


def test_dual_monotone_and_gap_closes():
    """Sinkhorn is block-coordinate ascent on S (Theorem 3.1): S^(r) is
    non-decreasing; at convergence the primal value of Eq. (MOTe) at
    K (.) Phi (computed entry by entry on the full tensor) equals S."""
    rng = np.random.default_rng(12)
    prob = W.random_problem(rng, W.TREE, 4, 2, 4, eta=0.2, shape="tree-random")
    res = OS.TreeSinkhorn(prob.x64(), prob.mu, prob.edges, prob.eta).run(300)
    S = np.array(res.S)
    assert np.all(np.diff(S) >= -1e-13 * np.abs(S[1:]))
    Kt = OS.full_kernel_tensor(prob.x64(), _tree_graph_edges(prob.edges), prob.eta)
    P = OS.tensor_marginals(OS.plan_tensor(Kt, res.phi))
    mass = OS.total_mass(P)
    dual = OS.dual_value(prob.mu, res.phi, mass, prob.eta)
    primal = OS.primal_bruteforce(Kt, prob.x64(), None, res.phi, prob.eta)
    assert abs(primal - dual) < 1e-10 * abs(dual)
    assert OS.violation(P, prob.mu) < 1e-10


def test_primal_value_formula_matches_tensor():
    """The collapsed primal value eta sum_k P_k . log phi^k - eta mass equals
    <Pi, C> + eta <Pi, log Pi - 1> summed over the full tensor, for any phi."""
    rng = np.random.default_rng(13)
    prob = W.random_problem(rng, W.CIRCLE, 3, 1, [4, 5, 3], eta=0.25)
    phi = _rand_phi(rng, prob.n)
    Kt = OS.full_kernel_tensor(prob.x64(), _circle_graph_edges(3), prob.eta)
    P = OS.tensor_marginals(OS.plan_tensor(Kt, phi))
    v1 = OS.primal_value(P, phi, OS.total_mass(P), prob.eta)
    v2 = OS.primal_bruteforce(Kt, prob.x64(), None, phi, prob.eta)
    assert abs(v1 - v2) < 1e-12 * max(1.0, abs(v2))


def test_scale_and_translation_invariance():
    """exp(-||x - y||^2 / eta) is unchanged under x -> (x - c)/s, eta -> eta/s^2,
    so the iterates are identical."""
    rng = np.random.default_rng(14)
    prob = W.random_problem(rng, W.TREE, 3, 2, 6, eta=0.05, shape="path")
    c, s = np.array([0.3, -0.1]), 1.7
    xs = [(a - c) / s for a in prob.x64()]
    r1 = OS.TreeSinkhorn(prob.x64(), prob.mu, prob.edges, prob.eta).run(20)
    r2 = OS.TreeSinkhorn(xs, prob.mu, prob.edges, prob.eta / s ** 2).run(20)
    for a, b in zip(r1.phi, r2.phi):
        np.testing.assert_allclose(a, b, rtol=1e-10)


def test_root_choice_leaves_fixed_point():
    """Relabelling the root changes the sweep order but not the solution of the
    strictly convex problem: gauge-fixed potentials agree at convergence."""
    rng = np.random.default_rng(15)
    prob = W.random_problem(rng, W.TREE, 5, 1, 4, eta=0.3, shape="tree-random")
    r0 = OS.TreeSinkhorn(prob.x64(), prob.mu, prob.edges, prob.eta, root=0).run(500)
    r3 = OS.TreeSinkhorn(prob.x64(), prob.mu, prob.edges, prob.eta, root=3).run(500)
    u0 = OS.gauge_fix([prob.eta * np.log(p) for p in r0.phi], prob.mu)
    u3 = OS.gauge_fix([prob.eta * np.log(p) for p in r3.phi], prob.mu)
    for a, b in zip(u0, u3):
        np.testing.assert_allclose(a, b, atol=1e-9)


def test_path3_workload_against_bruteforce():
    """The 3-marginal, N=100 path workload: 200 sweeps of Algorithm 2 equal 200
    sweeps of Algorithm 1 on the full 100^3 tensor (every 50 sweeps compared),
    and the final marginals of the tensor plan are close to mu."""
    prob = W.path3_d1()
    ts = OS.TreeSinkhorn(prob.x64(), prob.mu, prob.edges, prob.eta)
    hist = {}
    ts.run(prob.iters, callback=lambda r, phi: hist.__setitem__(r, [p.copy() for p in phi]) if r % 50 == 0 else None)
    Kt = OS.full_kernel_tensor(prob.x64(), _tree_graph_edges(prob.edges), prob.eta)
    phi = [np.ones(100) for _ in range(3)]
    for r in range(1, prob.iters + 1):
        phi = OS.sinkhorn_bruteforce(Kt, prob.mu, 1, phi0=phi)[-1]
        if r % 50 == 0:
            for a, b in zip(hist[r], phi):
                np.testing.assert_allclose(a, b, rtol=1e-9)
    P = OS.tensor_marginals(OS.plan_tensor(Kt, phi))
    assert OS.violation(P, prob.mu) < 1e-6


@pytest.mark.parametrize("root", [1, 2])
def test_free_centre_star_is_two_marginal_sinkhorn_on_composite_kernel(root):
    """Barycenter modification (Section 6.2): a star whose centre carries no marginal
    constraint (phi = 1) couples its two leaves through the composite kernel
    G = K^{(a,c)} K^{(c,b)}, so at convergence the leaves' coupling diag(phi_a) G diag(phi_b)
    equals the one of a textbook two-marginal Sinkhorn on G (written out here), with edge
    weights w_e on the squared distances."""
    rng = np.random.default_rng(2024)
    n = [30, 25, 35]                      # centre 0, leaves 1 and 2
    x = [rng.uniform(-0.3, 0.3, size=(m, 1)) for m in n]
    mu = [np.full(n[0], 1.0 / n[0])] + [rng.uniform(0.2, 1.0, m) for m in n[1:]]
    mu = [m / m.sum() for m in mu]
    eta, w = 0.05, [0.7, 1.6]
    edges = np.array([[0, 1], [0, 2]])
    ts = OS.TreeSinkhorn(x, mu, edges, eta, root=root, edge_w=w)
    res = ts.run(3000, free_nodes=[0])
    assert np.allclose(res.phi[0], 1.0)

    def kern(a, b, we):
        return np.exp(-we * (a[:, 0][:, None] - b[:, 0][None, :]) ** 2 / eta)

    G = kern(x[1], x[0], w[0]) @ kern(x[0], x[2], w[1])
    pa, pb = np.ones(n[1]), np.ones(n[2])
    for _ in range(3000):
        pa = mu[1] / (G @ pb)
        pb = mu[2] / (G.T @ pa)
    P_ref = pa[:, None] * G * pb[None, :]
    P_tree = res.phi[1][:, None] * G * res.phi[2][None, :]
    assert np.max(np.abs(P_tree - P_ref)) <= 1e-10 * np.max(P_ref)
    # the free centre's marginal is the pushforward of that coupling through the kernels
    P = OS.tree_marginals(x, res.phi, edges, eta, root=root, edge_w=w)
    Kac, Kcb = kern(x[1], x[0], w[0]), kern(x[0], x[2], w[1])
    centre = np.einsum("a,ac,cb,b->c", pa, Kac, Kcb, pb)
    assert np.allclose(P[0], centre, rtol=1e-8, atol=1e-14)


def test_free_root_sibling_updates_do_not_converge():
    """With a free root (phi = 1 at the root, Section 6.2 modification) the leaves of a star
    are updated from each other's previous messages (Algorithm 2's sibling order), a Jacobi
    step in the scaling gauge: scaling every leaf by c maps to c^{-(L-1)}.  For two leaves the
    total mass alternates between two values instead of converging; this is why the CUDA path
    requires a constrained root whenever free nodes are present."""
    rng = np.random.default_rng(5)
    n = [20, 15, 18]
    x = [rng.uniform(-0.3, 0.3, size=(m, 1)) for m in n]
    mu = [np.full(m, 1.0 / m) for m in n]
    ts = OS.TreeSinkhorn(x, mu, np.array([[0, 1], [0, 2]]), 0.05, root=0)
    masses = []
    ts.run(400, free_nodes=[0], callback=lambda r, phi: masses.append(
        float(OS.total_mass(OS.tree_marginals(x, phi, np.array([[0, 1], [0, 2]]), 0.05)))))
    tail = np.array(masses[-6:])
    assert np.max(np.abs(np.log(tail))) > 1e-3          # mass stays away from 1
    assert np.allclose(tail[::2], tail[0], rtol=1e-9) and np.allclose(tail[1::2], tail[1], rtol=1e-9)
    assert abs(np.log(tail[0]) + np.log(tail[1])) < 1e-6  # period 2: c and 1/c


# ---------------------------------------------------------------------------
# generalised Euler flows (Section 6.3): closing edge against sigma(x^1), pair marginals
# ---------------------------------------------------------------------------

def _euler_problem(rng, K, n, sigma="fold"):
    x = [rng.uniform(0.0, 1.0, size=(m, 1)).astype(np.float32) for m in n]
    mu = [np.full(m, 1.0 / m) for m in n]
    x_close = W.CONNECTION_MAPS[sigma](x[0].astype(np.float64)).astype(np.float32)
    return W.Problem("euler-test", W.CIRCLE, K, 1, x, mu, 0.3, None, x_close=x_close)


def _euler_tensor_by_loops(prob):
    """The Section 6.3 cost C_i = |x^K_{i_K} - sigma(x^1_{i_1})|^2 + sum_k |x^{k+1}_{i_{k+1}} - x^k_{i_k}|^2,
    entry by entry, and K = exp(-C / eta)."""
    import itertools
    xs = [a[:, 0].astype(np.float64) for a in prob.x]
    xc = prob.x_close[:, 0].astype(np.float64)
    Kt = np.empty(tuple(prob.n))
    for idx in itertools.product(*[range(m) for m in prob.n]):
        c = (xs[-1][idx[-1]] - xc[idx[0]]) ** 2
        for k in range(prob.K - 1):
            c += (xs[k + 1][idx[k + 1]] - xs[k][idx[k]]) ** 2
        Kt[idx] = math.exp(-c / prob.eta)
    return Kt


@pytest.mark.parametrize("sigma", ["fold", "reflect"])
def test_euler_circle_marginals_and_pairs_match_bruteforce(sigma):
    """Section 6.3: with the closing edge measured against sigma(x^1), the circle's matrix
    recursions (Theorem 4.3) still give the marginals of the full tensor, and
    phi^1 lambda^{(1,k)} alpha^{(k,1)} phi^k gives its pair marginals Pi_{1,k}, for
    arbitrary positive phi; the tensor is built entry by entry from the printed cost."""
    rng = np.random.default_rng(41)
    prob = _euler_problem(rng, 4, [3, 4, 2, 3], sigma)
    phi = _rand_phi(rng, prob.n)
    Kt = _euler_tensor_by_loops(prob)
    np.testing.assert_allclose(OS.full_kernel_tensor(prob.x64(), _circle_graph_edges(4), prob.eta,
                                                     x_close=prob.x_close64()), Kt, rtol=1e-13)
    Pi = OS.plan_tensor(Kt, phi)
    P_mp = OS.circle_marginals(prob.x64(), phi, prob.eta, x_close=prob.x_close64())
    for a, b in zip(P_mp, OS.tensor_marginals(Pi)):
        np.testing.assert_allclose(a, b, rtol=1e-12)
    pairs = OS.circle_pair_marginals(prob.x64(), phi, prob.eta, x_close=prob.x_close64())
    assert pairs[0] is None
    for k in range(1, 4):
        np.testing.assert_allclose(pairs[k], OS.tensor_pair_marginal(Pi, 0, k), rtol=1e-12)
        np.testing.assert_allclose(pairs[k].sum(axis=1), P_mp[0], rtol=1e-12)
        np.testing.assert_allclose(pairs[k].sum(axis=0), P_mp[k], rtol=1e-12)


def test_euler_circle_algorithm3_equals_algorithm1():
    """Algorithm 3 with the sigma-closing edge is the Gauss-Seidel sweep of Algorithm 1 on
    the Section 6.3 cost tensor: the iterates agree sweep by sweep."""
    rng = np.random.default_rng(42)
    prob = _euler_problem(rng, 4, [4, 3, 5, 4])
    cs = OS.CircleSinkhorn(prob.x64(), prob.mu, prob.eta, x_close=prob.x_close64())
    hist = []
    cs.run(6, callback=lambda r, phi: hist.append([p.copy() for p in phi]))
    bf = OS.sinkhorn_bruteforce(_euler_tensor_by_loops(prob), prob.mu, 6)
    for a, b in zip(hist, bf):
        for pa, pb in zip(a, b):
            np.testing.assert_allclose(pa, pb, rtol=1e-11)


def test_euler_identity_map_is_plain_circle():
    """sigma = identity gives back the plain circle of Algorithm 3."""
    rng = np.random.default_rng(43)
    prob = W.random_problem(rng, W.CIRCLE, 4, 2, [5, 4, 6, 3], eta=0.15)
    ra = OS.CircleSinkhorn(prob.x64(), prob.mu, prob.eta).run(5)
    rb = OS.CircleSinkhorn(prob.x64(), prob.mu, prob.eta, x_close=prob.x64()[0]).run(5)
    for a, b in zip(ra.phi, rb.phi):
        np.testing.assert_array_equal(a, b)


def test_euler_pair_marginals_at_convergence_carry_the_measures():
    """At the Sinkhorn fixed point of the Section 6.3 problem every pair marginal Pi_{1,k} is
    a coupling of mu^1 and mu^k (row sums mu^1, column sums mu^k)."""
    prob = W.euler5_d1(n=40)
    res = OS.CircleSinkhorn(prob.x64(), prob.mu, prob.eta, x_close=prob.x_close64()).run(400)
    pairs = OS.circle_pair_marginals(prob.x64(), res.phi, prob.eta, x_close=prob.x_close64())
    for k in range(1, prob.K):
        np.testing.assert_allclose(pairs[k].sum(axis=1), prob.mu[0], atol=1e-8)
        np.testing.assert_allclose(pairs[k].sum(axis=0), prob.mu[k], atol=1e-8)


def test_bruteforce_update_reproduces_the_measure():
    """Algorithm 1 on the full tensor: right after the update of phi^k the marginal P_k of the
    plan equals mu^k (P_k is linear in phi^k), and the total mass equals sum mu^k = 1 then."""
    rng = np.random.default_rng(51)
    prob = W.random_problem(rng, W.TREE, 4, 2, [3, 4, 2, 5], eta=0.3, shape="tree-random")
    Kt = OS.full_kernel_tensor(prob.x64(), _tree_graph_edges(prob.edges), prob.eta)
    phi = _rand_phi(rng, prob.n)
    for k in range(4):
        Pk = OS.tensor_marginals(OS.plan_tensor(Kt, phi))[k]
        phi[k] = prob.mu[k] * phi[k] / Pk
        P = OS.tensor_marginals(OS.plan_tensor(Kt, phi))
        np.testing.assert_allclose(P[k], prob.mu[k], rtol=1e-12)
        np.testing.assert_allclose([p.sum() for p in P], 1.0, rtol=1e-12)


def test_euler_closing_edge_in_two_dimensions():
    """The sigma-closing circle of Section 6.3 in d = 2 (sigma a rotation by 90 degrees about the
    centre of the unit square): message-passing marginals and pair marginals equal brute force
    over the tensor of the printed cost."""
    rng = np.random.default_rng(52)
    n = [3, 4, 3, 2]
    x = [rng.uniform(0, 1, (m, 2)).astype(np.float32) for m in n]
    mu = [np.full(m, 1.0 / m) for m in n]
    x1 = x[0].astype(np.float64)
    x_close = np.stack([1.0 - x1[:, 1], x1[:, 0]], axis=1)
    phi = _rand_phi(rng, n)
    xs = [a.astype(np.float64) for a in x]
    import itertools
    Kt = np.empty(tuple(n))
    for idx in itertools.product(*[range(m) for m in n]):
        c = float(((xs[-1][idx[-1]] - x_close[idx[0]]) ** 2).sum())
        for k in range(3):
            c += float(((xs[k + 1][idx[k + 1]] - xs[k][idx[k]]) ** 2).sum())
        Kt[idx] = math.exp(-c / 0.3)
    Pi = OS.plan_tensor(Kt, phi)
    P = OS.circle_marginals(xs, phi, 0.3, x_close=x_close)
    for a, b in zip(P, OS.tensor_marginals(Pi)):
        np.testing.assert_allclose(a, b, rtol=1e-12)
    pairs = OS.circle_pair_marginals(xs, phi, 0.3, x_close=x_close)
    for k in range(1, 4):
        np.testing.assert_allclose(pairs[k], OS.tensor_pair_marginal(Pi, 0, k), rtol=1e-12)


@pytest.mark.parametrize("topology", ["tree", "circle"])
def test_gauge_fix_keeps_the_plan_and_removes_only_the_gauge(topology):
    """``gauge_fix`` (the map every potential comparison goes through) against the plan built
    entry by entry over the full tensor: (a) the fixed potentials give the same K (.) Phi, hence
    the same marginals, mass and dual / primal values (Theorem 3.1: only sum_k u^k_{i_k} enters);
    (b) for k >= 1 the fixed u^k have zero mu^k-weighted mean; (c) it is idempotent; (d) two
    gauges of one solution (u^k + c_k with sum_k c_k = 0) map to the same output, while a shift
    that changes the plan (sum_k c_k != 0) does not."""
    rng = np.random.default_rng(61 if topology == "tree" else 62)
    K, n, eta = 4, [3, 4, 2, 5], 0.3
    if topology == "tree":
        prob = W.random_problem(rng, W.TREE, K, 2, n, eta=eta, shape="tree-random")
        graph = _tree_graph_edges(prob.edges)
    else:
        prob = W.random_problem(rng, W.CIRCLE, K, 2, n, eta=eta)
        graph = _circle_graph_edges(K)
    Kt = OS.full_kernel_tensor(prob.x64(), graph, eta)
    u = [eta * np.log(p) for p in _rand_phi(rng, n)]

    def plan(v):
        return OS.plan_tensor(Kt, [np.exp(a / eta) for a in v])

    g = OS.gauge_fix(u, prob.mu)
    # (a) same plan entry by entry, so the same marginals and values
    np.testing.assert_allclose(plan(g), plan(u), rtol=1e-12)
    Pu, Pg = OS.tensor_marginals(plan(u)), OS.tensor_marginals(plan(g))
    for a, b in zip(Pu, Pg):
        np.testing.assert_allclose(a, b, rtol=1e-12)
    phi_u, phi_g = [np.exp(a / eta) for a in u], [np.exp(a / eta) for a in g]
    mass = OS.total_mass(Pu)
    assert abs(OS.dual_value(prob.mu, phi_g, mass, eta) - OS.dual_value(prob.mu, phi_u, mass, eta)) <= 1e-12
    assert abs(OS.primal_value(Pg, phi_g, mass, eta) - OS.primal_value(Pu, phi_u, mass, eta)) <= 1e-12
    # (b) the normalisation it states
    for k in range(1, K):
        assert abs(float(np.dot(prob.mu[k], g[k]))) <= 1e-14
    assert not np.allclose(g[0], u[0])            # the total shift went to u^0
    # (c) idempotent
    for a, b in zip(OS.gauge_fix(g, prob.mu), g):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-14)
    # (d) every gauge of the same plan maps to one output; a plan-changing shift does not
    c = rng.normal(size=K)
    c -= c.mean()
    g2 = OS.gauge_fix([a + ck for a, ck in zip(u, c)], prob.mu)
    for a, b in zip(g2, g):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-13)
    g3 = OS.gauge_fix([a + 0.1 for a in u], prob.mu)
    assert max(float(np.max(np.abs(a - b))) for a, b in zip(g3, g)) > 0.1
