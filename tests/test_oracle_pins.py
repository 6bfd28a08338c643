"""Pins of the FP64 oracle against facts fixed by the paper and the mathematics.

Each test names what it pins; together they are chosen so that a dropped
term, a wrong sign or index, or a transposed operand anywhere in the oracle
fails at least one of them.
"""
import os

import numpy as np
import pytest

import oracle as O
import synth
from tests import pins

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def small_problem(n=12, p=3, k=3, seed=5, missing=0.0):
    X, _ = synth.gaussian_mixture(n, p, 3, seed=seed)
    X = X.astype(np.float64)
    mask = None
    if missing > 0:
        rng = np.random.default_rng(seed + 100)
        mask = synth.random_mask(rng, n, p, missing)
        mask[:, 0] = 1  # keep every row with data
    ei, ej, w, _, _ = O.knn_gaussian_weights(X, mask, k, 0.1, False)
    return X, mask, O.EdgeGraph(n, ei, ej, w)


# --------------------------------------------------------------- two points
@pytest.mark.parametrize("mu,eps_rel", [(0.05, 1e-2), (0.4, 1e-2), (0.05, 1e-3), (2.0, 1e-2), (0.3, 0.3)])
def test_two_point_closed_form(mu, eps_rel):
    """Pins projection (1/3 factor), d_m, the U update and the V prox at once."""
    rng = np.random.default_rng(1)
    X = rng.normal(size=(2, 4))
    w = 0.7
    G = O.EdgeGraph(2, [0], [1], [w])
    Y0 = O.fill_missing(X, None)
    rho, eps = O.pd_constants(Y0, G.w, mu, 2.0, eps_rel)
    U, V, d, fused, it, res, ok = O.solve_gamma(X, None, G, mu, rho, eps, X, np.zeros((1, 4)),
                                               tol=1e-14, max_iter=400000)
    assert ok
    Delta = X[0] - X[1]
    Dn = np.linalg.norm(Delta)
    delta, v, fz = pins.two_point_fixed_point(Dn, mu, w, rho, eps)
    e = Delta / Dn
    xbar = X.mean(axis=0)
    U_ref = np.vstack([xbar + 0.5 * delta * e, xbar - 0.5 * delta * e])
    assert bool(fused[0]) == fz
    assert np.allclose(U, U_ref, rtol=0, atol=1e-9 * Dn)
    assert np.allclose(V[0], v * e, rtol=0, atol=1e-9 * Dn)


def test_two_point_tends_to_eq1_solution():
    """As eps -> 0 the PD fixed point tends to the two-point solution of Eq. 1."""
    D, w, rho = 3.0, 1.0, 20.0
    for mu in (0.3, 1.0, 2.0):
        exact = D * max(0.0, 1.0 - 2.0 * mu * w / D)
        errs = [abs(pins.two_point_fixed_point(D, mu, w, rho, eps)[0] - exact) for eps in (1e-2, 1e-4, 1e-8)]
        assert errs[2] < 1e-3 and (errs[2] < errs[0] or errs[0] < 1e-12)


# --------------------------------------------------------------- projection
def test_projection_matches_paper_block_descent():
    """The exact projection equals the paper's Gauss-Seidel block updates run to rest."""
    X, _, G = small_problem(n=9, p=2, k=2, seed=3)
    rng = np.random.default_rng(2)
    U = rng.normal(size=X.shape)
    V = rng.normal(size=(G.m, X.shape[1]))
    A, B = O.project(U, V, G)
    A2, B2 = pins.gauss_seidel_projection(U, V, G.ei, G.ej)
    assert np.allclose(A, A2, atol=1e-10)
    assert np.allclose(B, B2, atol=1e-10)


def test_projection_stationarity_and_idempotence():
    X, _, G = small_problem(n=10, p=3, k=3, seed=4)
    rng = np.random.default_rng(3)
    U = rng.normal(size=X.shape)
    V = rng.normal(size=(G.m, 3))
    A, B = O.project(U, V, G)
    # the paper's stationarity equations, node by node
    for i in range(G.n):
        r = A[i] - U[i]
        for e in range(G.m):
            a, b = G.ei[e], G.ej[e]
            if a == i:
                r += A[i] - A[b] - V[e]
            elif b == i:
                r -= A[a] - A[i] - V[e]
        assert np.max(np.abs(r)) < 1e-10
    A2, B2 = O.project(A, B, G)
    assert np.allclose(A2, A, atol=1e-12) and np.allclose(B2, B, atol=1e-12)
    # and the dense orthogonal projector agrees
    P = pins.projection_matrix(G.n, G.ei, G.ej)
    Z = P @ np.vstack([U, V])
    assert np.allclose(Z[:G.n], A, atol=1e-10) and np.allclose(Z[G.n:], B, atol=1e-10)


def test_projection_complete_graph_closed_form():
    """Complete graph: (I + L) = (1+n) I - 11^T, so A = (R + 1 1^T R) / (1 + n)."""
    n, p = 7, 3
    ei, ej = np.triu_indices(n, 1)
    G = O.EdgeGraph(n, ei, ej, np.ones(ei.size))
    rng = np.random.default_rng(4)
    U = rng.normal(size=(n, p))
    V = rng.normal(size=(G.m, p))
    R = U + pins.incidence(n, ei, ej).T @ V
    A_ref = (R + R.sum(axis=0, keepdims=True)) / (1 + n)
    A, _ = O.project(U, V, G)
    assert np.allclose(A, A_ref, atol=1e-12)


# --------------------------------------------------------------- MM step
@pytest.mark.parametrize("missing", [0.0, 0.2])
def test_literal_mm_monotone(missing):
    """Each literal MM step does not increase the approximate objective (MM principle)."""
    X, mask, G = small_problem(n=12, p=3, k=3, seed=6, missing=missing)
    Y0 = O.fill_missing(X, mask)
    mu = 0.5
    rho, eps = O.pd_constants(Y0, G.w, mu)
    U, V = Y0.copy(), np.zeros((G.m, 3))
    f = O.objective(U, V, X, mask, G, mu, rho, eps)
    for _ in range(300):
        U, V, _, _ = O.mm_step(U, V, X, mask, G, mu, rho, eps)
        f2 = O.objective(U, V, X, mask, G, mu, rho, eps)
        assert f2 <= f + 1e-12 * abs(f)
        f = f2


def test_prox_is_optimal():
    """The V update minimises mu w ||v|| + rho/(2 d) ||v - b||^2; b = 0 gives v = 0."""
    from scipy.optimize import minimize
    X, _, G = small_problem(n=8, p=3, k=2, seed=7)
    rng = np.random.default_rng(5)
    U = X + 0.3 * rng.normal(size=X.shape)
    V = rng.normal(size=(G.m, 3))
    mu, rho, eps = 0.8, 5.0, 1e-2
    _, Vn, d, fused = O.mm_step(U, V, X, None, G, mu, rho, eps)
    _, B = O.project(U, V, G)
    for e in range(G.m):
        def obj(v):
            return mu * G.w[e] * np.linalg.norm(v) + rho / (2 * d) * np.sum((v - B[e]) ** 2)
        best = minimize(obj, B[e], method="Nelder-Mead", options={"xatol": 1e-12, "fatol": 1e-15, "maxiter": 20000}).x
        assert obj(Vn[e]) <= obj(best) + 1e-10
    # zero difference gives zero
    G2 = O.EdgeGraph(2, [0], [1], [1.0])
    Xs = np.ones((2, 2))
    _, V2, _, f2 = O.mm_step(Xs, np.zeros((1, 2)), Xs, None, G2, 1.0, 3.0, 1e-4)
    assert f2[0] and np.all(V2 == 0)


def test_fixed_point_satisfies_kkt_of_smoothed_objective():
    """The oracle's result minimises F (plain definition of the PD fixed point)."""
    for missing in (0.0, 0.15):
        X, mask, G = small_problem(n=10, p=2, k=3, seed=8, missing=missing)
        Y0 = O.fill_missing(X, mask)
        for mu in (0.2, 3.0):
            rho, eps = O.pd_constants(Y0, G.w, mu, 2.0, 1e-2)
            U, V, d, fused, it, res, ok = O.solve_gamma(X, mask, G, mu, rho, eps, Y0, np.zeros((G.m, 2)),
                                                       tol=1e-13, max_iter=400000)
            assert ok
            r = pins.kkt_residual(U, V, X, mask, G.ei, G.ej, G.w, mu, rho, eps, fused)
            assert r < 1e-7, (missing, mu, r)


def test_literal_and_accelerated_reach_same_fixed_point():
    X, _, G = small_problem(n=8, p=2, k=2, seed=9)
    mu = 0.5
    rho, eps = O.pd_constants(X, G.w, mu, 2.0, 0.2)
    a = O.solve_gamma(X, None, G, mu, rho, eps, X, np.zeros((G.m, 2)), tol=1e-12, accelerate=True)
    b = O.solve_gamma(X, None, G, mu, rho, eps, X, np.zeros((G.m, 2)), tol=1e-12, accelerate=False,
                      max_iter=2_000_000)
    assert a[6] and b[6]
    assert np.allclose(a[0], b[0], atol=1e-8)


# --------------------------------------------------------------- special cases / invariances
def test_mu_zero_gives_data():
    X, _, G = small_problem(n=10, p=3, k=3, seed=10)
    path = O.solve_path(X, None, G, [0.0], tol=1e-12)
    assert np.allclose(path[0].U, X, atol=1e-9)
    assert not path[0].fused.any()


def test_large_mu_fuses_connected_graph_to_mean():
    X, _, G = small_problem(n=10, p=3, k=4, seed=11)
    labels_graph = O.fused_labels(G.n, G.ei, G.ej, np.ones(G.m, bool))
    assert labels_graph.max() == 0  # connected
    path = O.solve_path(X, None, G, [1e4], tol=1e-12)
    r = path[0]
    assert r.fused.all() and (r.labels == 0).all()
    Xc = X - X.mean(axis=0)
    # full fusion up to the eps smoothing bias (order eps_rel)
    assert np.linalg.norm(r.U - X.mean(axis=0)) <= 1e-2 * np.linalg.norm(Xc)


def test_mean_preserved_every_iterate_and_at_fixed_point():
    """Sum of u_i equals sum of x_i (no missing data): the exact projection keeps
    1^T A = 1^T U, and the U update is a convex combination with X."""
    X, _, G = small_problem(n=11, p=3, k=3, seed=12)
    mu = 1.0
    rho, eps = O.pd_constants(X, G.w, mu)
    U, V = X.copy(), np.zeros((G.m, 3))
    for _ in range(50):
        U, V, _, _ = O.mm_step(U, V, X, None, G, mu, rho, eps)
        assert np.allclose(U.mean(axis=0), X.mean(axis=0), atol=1e-12)


def test_weight_rescaling_equals_mu_rescaling():
    """U(mu, c w) = U(c mu, w) (normalising weights is equivalent to rescaling mu)."""
    X, _, G = small_problem(n=10, p=2, k=3, seed=13)
    c = 3.7
    G2 = O.EdgeGraph(G.n, G.ei, G.ej, c * G.w)
    a = O.solve_path(X, None, G2, [0.4], tol=1e-13)[0]
    b = O.solve_path(X, None, G, [0.4 * c], tol=1e-13)[0]
    assert np.allclose(a.U, b.U, atol=1e-9)
    assert (a.fused == b.fused).all()


def test_equivariance_translation_rotation_permutation():
    X, _, G = small_problem(n=9, p=3, k=3, seed=14)
    mu = 0.8
    base = O.solve_path(X, None, G, [mu], tol=1e-13)[0]
    t = np.array([5.0, -2.0, 1.5])
    tr = O.solve_path(X + t, None, G, [mu], tol=1e-13)[0]
    assert np.allclose(tr.U, base.U + t, atol=1e-8)
    Q, _ = np.linalg.qr(np.random.default_rng(0).normal(size=(3, 3)))
    ro = O.solve_path(X @ Q, None, G, [mu], tol=1e-13)[0]
    assert np.allclose(ro.U, base.U @ Q, atol=1e-8)
    perm = np.random.default_rng(1).permutation(G.n)
    inv = np.argsort(perm)            # new index of old case i is inv[i]
    a, b = inv[G.ei], inv[G.ej]
    G3 = O.EdgeGraph(G.n, np.minimum(a, b), np.maximum(a, b), G.w)
    pe = O.solve_path(X[perm], None, G3, [mu], tol=1e-13)[0]
    assert np.allclose(pe.U, base.U[perm], atol=1e-8)


def test_all_observed_mask_is_unmasked_solver():
    X, _, G = small_problem(n=9, p=3, k=3, seed=15)
    a = O.solve_path(X, None, G, [0.3, 1.2], tol=1e-12)
    b = O.solve_path(X, np.ones(X.shape, np.uint8), G, [0.3, 1.2], tol=1e-12)
    for r1, r2 in zip(a, b):
        assert np.array_equal(r1.U, r2.U) and np.array_equal(r1.fused, r2.fused)


def test_disconnected_components_never_merge():
    X1, _ = synth.gaussian_mixture(6, 2, 1, seed=1)
    X = np.vstack([X1, X1 + 100.0]).astype(np.float64)
    ei = [0, 1, 2, 3, 4, 6, 7, 8, 9, 10]
    ej = [1, 2, 3, 4, 5, 7, 8, 9, 10, 11]
    G = O.EdgeGraph(12, ei, ej, np.ones(10))
    r = O.solve_path(X, None, G, [1e3], tol=1e-12)[0]
    assert set(r.labels[:6]) == {0} and set(r.labels[6:]) == {1}


# --------------------------------------------------------------- true minimiser of Eq. 1
def test_pd_fixed_point_approaches_convex_clustering_minimizer():
    """As eps -> 0 the PD fixed point tends to the unique minimiser of Eq. 1."""
    X, _, G = small_problem(n=8, p=2, k=3, seed=16)
    mu = 0.6
    Ustar, gap = pins.convex_clustering_minimizer(X, G.ei, G.ej, G.w, mu)
    assert gap < 1e-9
    errs = []
    for eps_rel in (1e-1, 1e-2, 1e-3):
        r = O.solve_path(X, None, G, [mu], eps_rel=eps_rel, tol=1e-13)[0]
        errs.append(np.linalg.norm(r.U - Ustar) / np.linalg.norm(Ustar))
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < 2e-3


# --------------------------------------------------------------- weights and labels
def _golden_knn():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "knn_line.txt")) if ln.strip() and not ln.startswith("#")]
    out = {}
    for c, i, j, d2, w in rows:
        out.setdefault(c, []).append((int(i), int(j), float(d2), float(w)))
    return out


def test_knn_weights_hand_example():
    g = _golden_knn()
    X = np.array([[0.0], [1.0], [3.0], [7.0]])
    ei, ej, w, d2, _ = O.knn_gaussian_weights(X, None, 1, 0.5, False)
    assert [(a, b) for a, b, _, _ in g["A"]] == list(zip(ei.tolist(), ej.tolist()))
    assert np.allclose(d2, [r[2] for r in g["A"]], rtol=0, atol=0)
    assert np.allclose(w, [r[3] for r in g["A"]], rtol=1e-15)
    X = np.array([[0.0], [1.0], [2.0]])
    ei, ej, w, d2, _ = O.knn_gaussian_weights(X, None, 1, 0.0, True)
    assert [(a, b) for a, b, _, _ in g["B"]] == list(zip(ei.tolist(), ej.tolist()))
    assert np.allclose(w, [r[3] for r in g["B"]], rtol=1e-15)


def test_knn_automatic_phi_hand_example():
    """phi = "auto" is one over the median squared distance of the union edges (odd and even edge
    counts), worked by hand in knn_line.txt cases C and D."""
    g = _golden_knn()
    X = np.array([[0.0], [1.0], [3.0], [7.0]])
    ei, ej, w, d2, phi = O.knn_gaussian_weights(X, None, 1, "auto", False)
    assert phi == 0.25
    assert [(a, b) for a, b, _, _ in g["C"]] == list(zip(ei.tolist(), ej.tolist()))
    assert np.allclose(w, [r[3] for r in g["C"]], rtol=1e-15, atol=0)
    X = np.array([[0.0], [1.0], [3.0], [7.0], [15.0]])
    ei, ej, w, d2, phi = O.knn_gaussian_weights(X, None, 1, "auto", True)
    assert phi == pytest.approx(0.1, rel=1e-15)
    assert [(a, b) for a, b, _, _ in g["D"]] == list(zip(ei.tolist(), ej.tolist()))
    assert d2.tolist() == [r[2] for r in g["D"]]
    assert np.allclose(w, [r[3] for r in g["D"]], rtol=1e-14, atol=0)
    # the composite rule with alpha = 1 reads phi the same way
    cw = O.knn_composite_weights(X, None, np.zeros((5, 2)), 1.0, 1, "auto", True)
    assert cw[4] == pytest.approx(0.1, rel=1e-15) and np.allclose(cw[2], w, rtol=1e-14, atol=0)


def test_pd_constants_hand_example():
    """rho = rho_scale (||Y_c||_F + mu ||w||_2) and eps = (eps_rel ||Y_c||_F)^2 on a 3 x 2 example
    worked by hand.  Y_0 = [[1, 2], [3, 0], [5, 4]] has column means (3, 2), so
    Y_c = [[-2, 0], [0, -2], [2, 2]] and ||Y_c||_F = 4 (the uncentred norm is sqrt(55));
    w = (3, 4) has ||w||_2 = 5 (||w||_1 = 7).  With mu = 0.5 and the defaults rho_scale = 2,
    eps_rel = 1e-3: rho = 2 (4 + 2.5) = 13, eps = (4e-3)^2 = 1.6e-5."""
    Y0 = np.array([[1.0, 2.0], [3.0, 0.0], [5.0, 4.0]])
    w = np.array([3.0, 4.0])
    rho, eps = O.pd_constants(Y0, w, 0.5)
    assert rho == pytest.approx(13.0, rel=1e-15)
    assert eps == pytest.approx(1.6e-5, rel=1e-12)
    # the slips this rules out: no centring, or the 1-norm of w
    assert abs(rho - 2.0 * (np.sqrt(55.0) + 2.5)) > 1.0 and abs(rho - 2.0 * (4.0 + 3.5)) > 1.0
    assert abs(eps - (1e-3 * np.sqrt(55.0)) ** 2) > 1e-6
    rho3, eps3 = O.pd_constants(Y0, w, 0.5, rho_scale=3.0, eps_rel=1e-2)
    assert rho3 == pytest.approx(19.5, rel=1e-15) and eps3 == pytest.approx(1.6e-3, rel=1e-12)
    # translating the data (a column shift) leaves both unchanged: only Y_c enters
    r2, e2 = O.pd_constants(Y0 + np.array([10.0, -7.0]), w, 0.5)
    assert r2 == pytest.approx(rho, rel=1e-14) and e2 == pytest.approx(eps, rel=1e-12)
    # degenerate data (all rows equal): rho = rho_scale, eps = eps_rel^2
    r0, e0 = O.pd_constants(np.ones((4, 3)), w, 0.0)
    assert r0 == 2.0 and e0 == pytest.approx(1e-6, rel=1e-15)


def test_pd_constants_bound_a_lipschitz_constant_of_the_loss():
    """rho / rho_scale bounds the gradient norm of 1/2 ||Y - U||^2 + mu sum w ||v|| wherever U lies
    between Y_0 and its centroid (U = Y_0 - t Y_c, 0 <= t <= 1) and V has no zero row; so
    rho > that Lipschitz constant, as the paper's exact-penalty argument asks."""
    rng = np.random.default_rng(3)
    Y0 = rng.normal(size=(7, 4)) + 5.0
    w = rng.uniform(0.1, 2.0, 9)
    mu = 0.8
    rho, _ = O.pd_constants(Y0, w, mu)
    Yc = Y0 - Y0.mean(axis=0)
    for t in np.linspace(0.0, 1.0, 11):
        U = Y0 - t * Yc
        V = rng.normal(size=(w.size, 4))
        gU = U - Y0
        gV = mu * w[:, None] * V / np.linalg.norm(V, axis=1, keepdims=True)
        gnorm = np.sqrt(np.sum(gU * gU) + np.sum(gV * gV))
        assert gnorm <= rho / 2.0 * (1 + 1e-12)
        # the V part is at its maximum mu ||w||_2 for every V; the U part reaches ||Y_c||_F at t = 1
        assert np.sqrt(np.sum(gV * gV)) == pytest.approx(mu * np.linalg.norm(w), rel=1e-13)
    assert np.linalg.norm(Yc) + mu * np.linalg.norm(w) == pytest.approx(rho / 2.0, rel=1e-15)


def test_knn_union_properties():
    X, _ = synth.gaussian_mixture(40, 5, 3, seed=2)
    ei, ej, w, d2, _ = O.knn_gaussian_weights(X, None, 4, 0.3, True)
    n = 40
    deg = np.bincount(ei, minlength=n) + np.bincount(ej, minlength=n)
    assert deg.min() >= 4 and np.all(ei < ej)
    assert abs(w.sum() - 1.0) < 1e-12
    # exact distances
    Xd = X.astype(np.float64)
    assert np.allclose(d2, np.sum((Xd[ei] - Xd[ej]) ** 2, axis=1), rtol=1e-14)
    # every listed neighbour of i is at least as close as every non-neighbour
    D2 = np.sum((Xd[:, None] - Xd[None]) ** 2, axis=-1)
    for i in range(n):
        nb = set(ej[ei == i].tolist()) | set(ei[ej == i].tolist())
        kth = np.sort(np.delete(D2[i], i))[3]
        near = [j for j in range(n) if j != i and D2[i, j] < kth]
        assert set(near) <= nb


def test_fused_labels_canonical():
    lab = O.fused_labels(6, [0, 1, 2, 3], [1, 2, 4, 5], [False, True, False, True])
    # components: {0}, {1,2}, {3,5}, {4}
    assert lab.tolist() == [0, 1, 1, 2, 3, 2]


def test_min_connected_k_two_clusters_closed_form():
    """Two tight clusters far apart: a case of the smaller cluster (size a) reaches the other
    cluster only among its a nearest, so the union graph connects exactly at k = min(a, b)."""
    rng = np.random.default_rng(4)
    for a, b in [(4, 7), (6, 6), (9, 3)]:
        X = np.vstack([rng.normal(0.0, 0.1, (a, 3)), rng.normal(50.0, 0.1, (b, 3))])
        assert O.min_connected_k(X, None, 20) == min(a, b)
        assert O.min_connected_k(X, None, min(a, b) - 1) == 0


def test_min_connected_k_chain_and_brute_force():
    # equally spaced points: each case's nearest neighbour (ties to the smaller index) links a chain
    X = np.arange(10, dtype=np.float64)[:, None]
    assert O.min_connected_k(X, None, 5) == 1
    # random data: the first connected k from an independent construction (scipy distances,
    # stable argsort, scipy connected components)
    sp = pytest.importorskip("scipy.sparse.csgraph")
    from scipy.spatial.distance import cdist
    from scipy.sparse import coo_matrix
    for seed in range(3):
        X, _ = synth.gaussian_mixture(45, 4, 4, seed=seed)
        D = cdist(X.astype(np.float64), X.astype(np.float64), "sqeuclidean")
        np.fill_diagonal(D, np.inf)
        order = np.argsort(D, axis=1, kind="stable")
        want = 0
        for k in range(1, 44):
            rows = np.repeat(np.arange(45), k)
            cols = order[:, :k].ravel()
            ncomp = sp.connected_components(coo_matrix((np.ones(rows.size), (rows, cols)), shape=(45, 45)),
                                            directed=False)[0]
            if ncomp == 1:
                want = k
                break
        assert O.min_connected_k(X, None, 44) == want


def test_geo_distance_geometry():
    """Geographic distances pinned by geometry, not by the formulas."""
    g = O.geo_distance
    # modulo arithmetic: longitudes 179 and -179 are 2 degrees apart; differences never exceed 180
    assert g((0, 179), (0, -179), False) == pytest.approx(2.0, abs=1e-12)
    assert g((3, 0), (-1, 540), False) == pytest.approx(np.hypot(4, 180), abs=1e-12)
    assert g((10, -20), (13, -16), False) == pytest.approx(5.0, abs=1e-12)
    # great circles: along a meridian or the equator the arc is the coordinate difference
    assert g((10, 40), (55, 40), True) == pytest.approx(45.0, abs=1e-10)
    assert g((0, 170), (0, -170), True) == pytest.approx(20.0, abs=1e-10)
    # the pole is 90 degrees from every equator point; antipodes are 180 apart
    for lon in (-120.0, 0.0, 33.0):
        assert g((90, 0), (0, lon), True) == pytest.approx(90.0, abs=1e-10)
    assert g((10, 20), (-10, -160), True) == pytest.approx(180.0, abs=1e-9)
    # an octant: the three axis points are pairwise 90 degrees apart
    pts = [(0, 0), (0, 90), (90, 0)]
    for a in range(3):
        for b in range(a + 1, 3):
            assert g(pts[a], pts[b], True) == pytest.approx(90.0, abs=1e-10)
    # short arcs at latitude 60 shrink the longitude difference by cos(60) = 1/2
    assert g((60, 0), (60, 0.001), True) == pytest.approx(0.0005, rel=1e-6)


def test_composite_weights_special_cases():
    X, _ = synth.gaussian_mixture(30, 6, 3, seed=8)
    rng = np.random.default_rng(9)
    coords = np.c_[rng.uniform(-60, 60, 30), rng.uniform(-180, 180, 30)]
    # alpha = 1: the Euclidean rule of Eq. 8 exactly
    a = O.knn_composite_weights(X, None, coords, 1.0, 4, 0.2, True)
    b = O.knn_gaussian_weights(X, None, 4, 0.2, True)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.allclose(a[2], b[2], rtol=1e-12) and np.allclose(a[3], b[3], rtol=1e-12)
    # alpha = 0 with identical genotypes: neighbours by geography alone.  Four cases on the
    # equator at longitudes -179, 179, 10, 20: the pairs across the date line and 10-20 are nearest
    Xs = np.zeros((4, 3))
    cs = np.array([[0.0, -179.0], [0.0, 179.0], [0.0, 10.0], [0.0, 20.0]])
    for geodesic in (False, True):
        ei, ej, w, d2, _ = O.knn_composite_weights(Xs, None, cs, 0.0, 1, 0.0, False, geodesic)
        assert list(zip(ei.tolist(), ej.tolist())) == [(0, 1), (2, 3)]
        assert np.allclose(d2, [4.0, 100.0], rtol=1e-12)


def test_principal_axes_closed_forms():
    rng = np.random.default_rng(12)
    # rank one around a mean: the only axis is the direction b, its variance var(t) |b|^2
    b = np.array([3.0, -4.0, 0.0, 12.0])
    t = rng.normal(size=200)
    X = 5.0 + np.outer(t, b)
    A, var = O.principal_axes(X, None, 1)
    assert np.allclose(A[0], b / np.linalg.norm(b) * np.sign(b[np.argmax(np.abs(b))]), atol=1e-12)
    assert var[0] == pytest.approx(np.var(t) * b @ b, rel=1e-10)
    # independent coordinates with variances 9, 4, 1 along known orthonormal directions
    Q, _ = np.linalg.qr(rng.normal(size=(5, 5)))
    N = 500
    R = rng.normal(size=(N, 3))
    R -= R.mean(axis=0)
    Qz, _ = np.linalg.qr(R)                       # centred orthonormal columns (they stay centred)
    Z = np.sqrt(N) * Qz * [3.0, 2.0, 1.0]         # covariance exactly diag(9, 4, 1)
    X = Z @ Q[:3] + 1.0
    A, var = O.principal_axes(X, None, 3)
    assert np.allclose(var, [9.0, 4.0, 1.0], rtol=1e-8)
    for c in range(3):
        assert abs(abs(A[c] @ Q[c]) - 1.0) < 1e-8
        assert A[c, np.argmax(np.abs(A[c]))] > 0
    # scores: the centred data itself projects to its coordinates along the axes
    S = O.project_path(X, X, None, A)
    assert np.allclose(np.abs(S), np.abs(Z @ np.eye(3)), atol=1e-7)


def test_fusion_scale_is_the_two_point_threshold():
    """For one edge the scale is the mu at which Eq. 1 fuses the pair: below it the exact
    minimiser (dual solver, independent of the oracle) keeps the points apart, above it merges them."""
    X = np.array([[0.0, 1.0, -2.0], [3.0, -1.0, 0.5]])
    w = 0.7
    g0 = O.fusion_scale(X, None, [0], [1], [w])
    assert g0 == pytest.approx(np.linalg.norm(X[0] - X[1]) / (2 * w), rel=1e-15)
    U_lo, gap_lo = pins.convex_clustering_minimizer(X, [0], [1], [w], 0.98 * g0)
    U_hi, gap_hi = pins.convex_clustering_minimizer(X, [0], [1], [w], 1.02 * g0)
    assert np.linalg.norm(U_lo[0] - U_lo[1]) > 0.01 * np.linalg.norm(X[0] - X[1])
    assert np.linalg.norm(U_hi[0] - U_hi[1]) < 1e-8
    # several edges: the median of the per-edge thresholds (odd count: the middle one)
    Xs = np.array([[0.0], [1.0], [3.0], [7.0]])
    g = O.fusion_scale(Xs, None, [0, 1, 2], [1, 2, 3], [1.0, 0.5, 2.0])
    assert g == pytest.approx(sorted([1 / 2, 2 / 1, 4 / 4])[1])


def test_standardize_hand_example():
    """Observed-entry standardisation worked by hand.  Column 0 has observed 1, 3, 8: mean 4, squared
    deviations 9, 1, 16, variance 26/3 (divisor 3), so the entries are -3, -1, 4 over sqrt(26/3).
    Column 1 has observed 2 and 6 (the 100 at row 1 is masked): mean 4, variance 4, giving -1 and +1,
    the missing entry 0.  Column 2 is constant on its observed entries:
    centred only, all 0.  Column 3 has no observed entry: 0."""
    X = np.array([[1.0, 2.0, 7.0, 1.0], [3.0, 100.0, 7.0, 2.0], [8.0, 6.0, 7.0, 3.0]])
    mask = np.array([[1, 1, 1, 0], [1, 0, 1, 0], [1, 1, 0, 0]], np.uint8)
    Z = O.standardize(X, mask)
    s = np.sqrt(26.0 / 3.0)
    assert np.allclose(Z[:, 0], [-3.0 / s, -1.0 / s, 4.0 / s], rtol=1e-15, atol=0)
    assert Z[:, 1].tolist() == [-1.0, 0.0, 1.0]
    assert Z[:, 2].tolist() == [0.0, 0.0, 0.0] and Z[:, 3].tolist() == [0.0, 0.0, 0.0]
    # without a mask: every column has mean 0 and (population) variance 1 unless constant
    rng = np.random.default_rng(4)
    Y = rng.normal(3.0, 2.0, (9, 5))
    Y[:, 2] = -1.5
    Zy = O.standardize(Y, None)
    assert np.allclose(Zy.mean(axis=0), 0.0, atol=1e-15)
    assert np.allclose((Zy ** 2).mean(axis=0), [1, 1, 0, 1, 1], rtol=1e-14, atol=1e-30)
    # invariant to a positive affine change of each column
    assert np.allclose(O.standardize(4.0 * Y - 7.0, None), Zy, atol=1e-13)


def test_fill_missing_hand_example():
    X = np.array([[1.0, 9.0], [3.0, 2.0], [8.0, 4.0]])
    mask = np.array([[1, 0], [1, 1], [0, 1]], np.uint8)
    Y = O.fill_missing(X, mask)
    assert Y.tolist() == [[1.0, 3.0], [3.0, 2.0], [2.0, 4.0]]
