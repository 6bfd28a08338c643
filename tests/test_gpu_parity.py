"""Parity of the CUDA solver with the FP64 oracle, through the C ABI.

Bar (stated per assertion):
  * U: relative Frobenius error <= 1e-4 at every gamma (FP32 path), <= 1e-6
    for the FP64 path (its output is rounded to float32 once);
  * fused flags equal edge by edge, except edges whose oracle margin
    |mu w d / (rho ||b||) - 1| is below 1e-5 (both sides decide the same
    comparison, in different rounding);
  * labels identical whenever the fused sets are identical, and otherwise the
    connected components of the GPU's own fused set;
  * no double recompute of ||b|| at the returned iterate when every oracle
    margin exceeds 1e-4;
  * kNN edge sets bit-exact, weights to 1e-12 relative.
"""
import os

import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
MARGIN = 1e-5


@pytest.fixture(scope="module")
def ccx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1409_2065_gb300 as m
    return m


def oracle_margins(r, X, mask, G):
    A, B = O.project(r.U, r.V, G)
    nb = np.linalg.norm(B, axis=1)
    ratio = r.mu * G.w * r.d / (r.rho * np.maximum(nb, 1e-300))
    return np.abs(ratio - 1.0)


def check_fused(fused, labels, ref_fused, ref_labels, margin, n, ei, ej, tag):
    """Fused flags edge by edge outside the rounding band, then the labels."""
    got = np.asarray(fused).astype(bool)
    ref_fused = np.asarray(ref_fused).astype(bool)
    far = margin >= MARGIN
    bad = np.nonzero((got != ref_fused) & far)[0]
    assert bad.size == 0, f"{tag}: fused flags differ on edges {bad[:10]} (margins {margin[bad[:10]]})"
    if np.array_equal(got, ref_fused):
        assert np.array_equal(labels, ref_labels), f"{tag}: labels differ with equal fused sets"
    else:
        assert np.array_equal(labels, O.fused_labels(n, ei, ej, got)), f"{tag}: labels are not the components"


def solve_fused(pr, gammas, opts=None):
    m = pr.get_edges()[0].size
    fused = np.zeros((len(gammas), m), np.uint8)
    U, labels, stats, st = pr.solve_path(gammas, opts, fused_out=fused)
    return U, labels, fused, stats, st


def compare_path(U, labels, fused, stats, ref, X, mask, G, utol, tag=""):
    for g, r in enumerate(ref):
        err = np.linalg.norm(U[g].astype(np.float64) - r.U) / max(np.linalg.norm(r.U), 1e-300)
        assert err <= utol, f"{tag} gamma={r.mu}: U rel err {err:.3e} > {utol}"
        assert stats[g]["converged"] in (1, 2), f"{tag} gamma={r.mu} not converged"
        margin = oracle_margins(r, X, mask, G)
        check_fused(fused[g], labels[g], r.fused, r.labels, margin, G.n, G.ei, G.ej, f"{tag} gamma={r.mu}")
        if margin.min() > 1e-4:
            assert stats[g]["n_recomputed"] == 0, f"{tag} gamma={r.mu}: {stats[g]}"


def knn_graph(X, mask, k, phi, normalize=False):
    ei, ej, w, _, _ = O.knn_gaussian_weights(X.astype(np.float64), mask, k, phi, normalize)
    return O.EdgeGraph(X.shape[0], ei, ej, w)


@pytest.mark.parametrize("precision,utol", [(1, 1e-6), (0, 1e-4)])
def test_tiny_path(ccx, precision, utol):
    X, _ = synth.gaussian_mixture(12, 3, 3, seed=5)
    G = knn_graph(X, None, 3, 0.1)
    gammas = [0.0, 0.05, 0.5, 5.0, 50.0]
    pr = ccx.Problem(X, None, precision)
    pr.set_edges(G.ei, G.ej, G.w)
    U, labels, fused, stats, st = solve_fused(pr, gammas)
    ref = O.solve_path(X.astype(np.float64), None, G, gammas, tol=1e-12)
    compare_path(U, labels, fused, stats, ref, X, None, G, utol, "tiny")
    assert np.linalg.norm(U[0] - X) <= 1e-5 * np.linalg.norm(X)   # gamma = 0 returns the data


def test_ragged_missing_fp32(ccx):
    """n = 70, p = 37 (ten 4-column slices, ragged last slice), 10 % missing."""
    X, _ = synth.gaussian_mixture(70, 37, 4, seed=11)
    rng = np.random.default_rng(12)
    mask = synth.random_mask(rng, 70, 37, 0.1)
    G = knn_graph(X, mask, 5, 0.02)
    Y0 = O.fill_missing(X, mask)
    g0 = O.fusion_scale(X, mask, G.ei, G.ej, G.w)
    gammas = synth.log_grid(1e-2 * g0, 3.0 * g0, 5)
    pr = ccx.Problem(X, mask, ccx.CCX_FP32)
    pr.set_edges(G.ei, G.ej, G.w)
    assert abs(pr.fusion_scale() - g0) <= 1e-6 * g0
    U, labels, fused, stats, st = solve_fused(pr, gammas)
    ref = O.solve_path(X.astype(np.float64), mask, G, gammas, tol=1e-12)
    compare_path(U, labels, fused, stats, ref, X, mask, G, 1e-4, "ragged")
    assert Y0.shape == X.shape


@pytest.mark.parametrize("precision,utol", [(1, 1e-6), (0, 1e-4)])
def test_plain_workload_against_stored_oracle(ccx, precision, utol):
    """n = 200, p = 10, kNN k = 10, 20 gamma (values written by tests/golden/make_golden.py)."""
    z = np.load(os.path.join(GOLDEN, "plain_n200_p10.npz"))
    X = z["X"]
    pr = ccx.Problem(X, None, precision)
    pr.build_knn(10, phi=0.5)
    ei, ej, w = pr.get_edges()
    assert np.array_equal(ei, z["ei"]) and np.array_equal(ej, z["ej"])
    assert np.allclose(w, z["w"], rtol=1e-12, atol=0)
    U, labels, fused, stats, st = solve_fused(pr, z["gammas"])
    for g in range(len(z["gammas"])):
        err = np.linalg.norm(U[g] - z["U"][g]) / np.linalg.norm(z["U"][g])
        assert err <= utol, (g, err)
        assert stats[g]["converged"] in (1, 2)
        check_fused(fused[g], labels[g], z["fused"][g], z["labels"][g], np.abs(z["margin"][g]), 200, z["ei"],
                    z["ej"], f"plain gamma {g}")


def test_knn_matches_oracle_missing_normalized(ccx):
    X, _ = synth.gaussian_mixture(90, 23, 3, seed=21)
    rng = np.random.default_rng(22)
    mask = synth.random_mask(rng, 90, 23, 0.05)
    pr = ccx.Problem(X, mask, ccx.CCX_FP32)
    pr.build_knn(7, phi_auto=True, normalize=True)
    ei, ej, w = pr.get_edges()
    oei, oej, ow, _, _ = O.knn_gaussian_weights(X.astype(np.float64), mask, 7, "auto", True)
    assert np.array_equal(ei, oei) and np.array_equal(ej, oej)
    assert np.allclose(w, ow, rtol=1e-12, atol=0)
    assert abs(w.sum() - 1.0) < 1e-12


@pytest.mark.parametrize("gram", [0, 1, 2])
@pytest.mark.parametrize("n,p,k,frac", [(400, 2000, 10, 0.05), (130, 37, 5, 0.0), (257, 300, 9, 0.1)])
def test_knn_tensor_core_gram_shapes(ccx, n, p, k, frac, gram):
    """Candidate selection from the Gram (tensor cores on TF32 or BF16 operands, or FP32 CUDA cores):
    tiles with ragged rows (n not a multiple of 128), short and long K (p = 300 leaves half a BF16
    stage), missing data; the edge set must equal brute force exactly for every Gram."""
    X, mask, _ = synth.genotype_like(n, p, 5, seed=31, fst=0.05, frac_missing=frac)
    if frac == 0.0:
        mask = None
    pr = ccx.Problem(X, mask, ccx.CCX_FP32)
    pr.build_knn(k, phi_auto=True, normalize=True, gram=gram)
    ei, ej, w = pr.get_edges()
    oei, oej, ow, _, _ = O.knn_gaussian_weights(X.astype(np.float64), mask, k, "auto", True)
    assert np.array_equal(ei, oei) and np.array_equal(ej, oej)
    assert np.allclose(w, ow, rtol=1e-12, atol=0)


def test_streamed_edge_arrays_identical(ccx):
    """The iteration kernel's variant for large edge sets (indices and per-edge accumulators in
    global memory) gives bit-identical results to the staged variant."""
    X, mask, _ = synth.genotype_like(300, 64, 5, seed=41, fst=0.05, frac_missing=0.05)
    gammas = None
    out = []
    for stream in (0, 1):
        pr = ccx.Problem(X, mask, ccx.CCX_FP32)
        pr.build_knn(10, phi_auto=True, normalize=True)
        if gammas is None:
            g0 = pr.fusion_scale()
            gammas = synth.log_grid(0.05 * g0, 2.0 * g0, 4)
        o = ccx.opts_default()
        o.stream_edges = stream
        U, labels, stats, st = pr.solve_path(gammas, o)
        out.append((U, labels, [s["iters"] for s in stats]))
        pr.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1]) and out[0][2] == out[1][2]


def test_large_problem_needs_streamed_arrays(ccx):
    """n = 1400 with a kNN graph: the edge arrays no longer fit beside the rows in shared memory, so
    the streamed variant runs; parity by the fixed point's invariants (the oracle is too slow at this
    size): with no missing data the mean of U equals the mean of X, and gamma = 0 returns X."""
    X, _ = synth.gaussian_mixture(1400, 16, 6, seed=43)
    pr = ccx.Problem(X, None, ccx.CCX_FP32)
    pr.build_knn(10, phi=0.05)
    ei, ej, w = pr.get_edges()
    assert ei.size > 7000          # staged layout would need > 227 KB of shared memory
    g0 = pr.fusion_scale()
    U, labels, stats, st = pr.solve_path([0.0, 0.1 * g0, 1.0 * g0])
    assert np.linalg.norm(U[0] - X) <= 1e-5 * np.linalg.norm(X)
    for g in range(3):
        assert stats[g]["converged"] in (1, 2)
        assert np.allclose(U[g].mean(axis=0), X.mean(axis=0), atol=1e-4 * np.abs(X).max())


@pytest.mark.parametrize("n,p,frac", [(60, 5, 0.0), (300, 40, 0.05), (700, 300, 0.0)])
def test_min_connected_k_matches_oracle(ccx, n, p, frac):
    """Bisection over GPU connected components gives the oracle's linear-scan answer exactly."""
    X, _ = synth.gaussian_mixture(n, p, 5, seed=n + p)
    mask = synth.random_mask(np.random.default_rng(n), n, p, frac) if frac > 0 else None
    pr = ccx.Problem(X, mask, ccx.CCX_FP32)
    for k_max in (3, 40):
        assert pr.min_connected_k(k_max) == O.min_connected_k(X.astype(np.float64), mask, k_max)
    # two far clusters: connects exactly at the smaller cluster's size
    rng = np.random.default_rng(1)
    Xc = np.vstack([rng.normal(0, 0.1, (13, 4)), rng.normal(40, 0.1, (30, 4))]).astype(np.float32)
    assert ccx.Problem(Xc).min_connected_k(50) == 13


@pytest.mark.parametrize("alpha,geodesic,frac", [(0.7, False, 0.0), (0.3, True, 0.05), (0.05, True, 0.0)])
def test_knn_composite_matches_oracle(ccx, alpha, geodesic, frac):
    """Composite genetic + geographic kNN weights: exact edge set and weights against brute force."""
    n, p = 150, 40
    X, mask, _ = synth.genotype_like(n, p, 4, seed=51, fst=0.05, frac_missing=frac)
    if frac == 0.0:
        mask = None
    rng = np.random.default_rng(52)
    coords = np.c_[rng.uniform(-70, 70, n), rng.uniform(-180, 180, n)]
    pr = ccx.Problem(X, mask, ccx.CCX_FP32)
    pr.build_knn_composite(6, coords, alpha, phi_auto=True, normalize=True, geodesic=geodesic)
    ei, ej, w = pr.get_edges()
    oei, oej, ow, _, _ = O.knn_composite_weights(X.astype(np.float64), mask, coords, alpha, 6, "auto", True,
                                                 geodesic)
    assert np.array_equal(ei, oei) and np.array_equal(ej, oej)
    assert np.allclose(w, ow, rtol=1e-10, atol=0)


def _spectrum_data(n, p, seed):
    """Data with a well separated spectrum: independent scores along orthonormal directions with
    standard deviations 10, 6, 3.5, 2, then an isotropic unit background."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.normal(size=(p, 4)))
    Z = rng.normal(size=(n, 4)) * [10.0, 6.0, 3.5, 2.0]
    return (Z @ Q.T + rng.normal(size=(n, p)) + 2.0).astype(np.float32)


@pytest.mark.parametrize("n,p,q,frac", [(400, 300, 3, 0.0), (250, 1000, 2, 0.05)])
def test_principal_axes_match_oracle(ccx, n, p, q, frac):
    X = _spectrum_data(n, p, n + p)
    mask = synth.random_mask(np.random.default_rng(7), n, p, frac) if frac > 0 else None
    pr = ccx.Problem(X, mask, ccx.CCX_FP32)
    axes, var = pr.principal_axes(q)
    oaxes, ovar = O.principal_axes(X.astype(np.float64), mask, q)
    assert np.allclose(var, ovar, rtol=1e-5)
    assert np.abs(axes - oaxes).max() <= 1e-5
    assert np.allclose(axes @ axes.T, np.eye(q), atol=1e-10)


def test_projected_path_matches_projection_of_U(ccx):
    """Scores written on the GPU equal the oracle's projection of the same path's centroids."""
    X = _spectrum_data(200, 60, 3)
    pr = ccx.Problem(X, None, ccx.CCX_FP32)
    pr.build_knn(8, phi_auto=True, normalize=True)
    g0 = pr.fusion_scale()
    gam = synth.log_grid(0.05 * g0, 2.0 * g0, 4)
    U, L, _, _ = pr.solve_path(gam)
    pr.reset_path()
    S, L2, stats, st = pr.solve_path_projected(gam, 2)
    Sd, L3, _, _ = (pr.reset_path(), pr.solve_path_projected(gam, 2, device=True))[1]
    axes, _ = O.principal_axes(X.astype(np.float64), None, 2)
    for g in range(len(gam)):
        ref = O.project_path(U[g], X.astype(np.float64), None, axes)
        assert np.abs(S[g] - ref).max() <= 1e-4 * np.abs(ref).max()
    assert np.array_equal(L2, L) and np.array_equal(S, Sd.cpu().numpy())


def test_knn_all_pairs(ccx):
    X, _ = synth.expression_like(20, 300, 3, 40, seed=2)
    pr = ccx.Problem(X, None, ccx.CCX_FP32)
    pr.build_knn(19, phi_auto=True, normalize=True)
    ei, ej, w = pr.get_edges()
    assert ei.size == 190
    oei, oej, ow, _, _ = O.knn_gaussian_weights(X.astype(np.float64), None, 19, "auto", True)
    assert np.array_equal(ei, oei) and np.allclose(w, ow, rtol=1e-12, atol=0)


@pytest.mark.parametrize("rule", ["auto_norm", "auto", "fixed_norm", "fixed", "underflow_norm"])
@pytest.mark.parametrize("n,k", [(61, 4), (100, 6)])
def test_knn_weight_rules_on_device(ccx, rule, n, k):
    """The union, phi (automatic: 1 / median d2, odd and even edge counts), the Gaussian weights and
    their normalisation, all formed on the device: edges equal the oracle's exactly, weights within
    1e-12, and a rebuild is bit-identical.  With phi = 2000 / median (normalised) most weights
    underflow to zero and those edges are dropped, as in the oracle."""
    X, mask, _ = synth.genotype_like(n, 40, 3, seed=n + k, fst=0.05, frac_missing=0.05)
    X64 = X.astype(np.float64)
    _, _, _, d2, phi_med = O.knn_gaussian_weights(X64, mask, k, "auto", False)
    auto = rule.startswith("auto")
    norm = rule.endswith("norm")
    phi = "auto" if auto else (2000.0 * phi_med if rule.startswith("underflow") else 0.7 * phi_med)
    oei, oej, ow, _, _ = O.knn_gaussian_weights(X64, mask, k, phi, norm)
    if rule.startswith("underflow"):
        assert 0 < oei.size < d2.size            # some weights are exactly zero
    got = []
    for _ in range(2):
        pr = ccx.Problem(X, mask, ccx.CCX_FP32)
        pr.build_knn(k, phi=0.0 if auto else phi, phi_auto=auto, normalize=norm)
        got.append(pr.get_edges())
        pr.close()
    ei, ej, w = got[0]
    assert np.array_equal(ei, oei) and np.array_equal(ej, oej)
    assert np.allclose(w, ow, rtol=1e-12, atol=0)
    assert np.array_equal(w, got[1][2])
    if norm:
        assert abs(w.sum() - 1.0) < 1e-12


def test_knn_edge_counts_of_both_parities():
    """The automatic phi above takes the median of an odd and of an even number of edges."""
    counts = set()
    for n, k in [(61, 4), (100, 6)]:
        X, mask, _ = synth.genotype_like(n, 40, 3, seed=n + k, fst=0.05, frac_missing=0.05)
        counts.add(O.knn_gaussian_weights(X.astype(np.float64), mask, k, "auto", False)[0].size % 2)
    assert counts == {0, 1}


def test_edge_cases(ccx):
    # a single case: no edges, U = X
    X1 = np.array([[1.0, -2.0, 3.0]], np.float32)
    pr = ccx.Problem(X1)
    U, labels, stats, _ = pr.solve_path([0.0, 1.0])
    assert np.allclose(U[:, 0], X1, atol=1e-6) and labels.tolist() == [[0], [0]]
    # no edges at all: every case its own cluster, U = X
    X, _ = synth.gaussian_mixture(9, 2, 3, seed=3)
    pr = ccx.Problem(X)
    U, labels, stats, _ = pr.solve_path([3.0])
    assert np.allclose(U[0], X, atol=1e-5) and labels[0].tolist() == list(range(9))
    # p = 1, a chain graph and a disconnected pair of components
    Xc = np.array([[0.0], [0.1], [0.3], [10.0], [10.2]], np.float32)
    pr = ccx.Problem(Xc, None, ccx.CCX_FP64)
    pr.set_edges([0, 1, 3], [1, 2, 4], [1.0, 1.0, 1.0])
    U, labels, stats, _ = pr.solve_path([100.0])
    assert labels[0].tolist() == [0, 0, 0, 1, 1]
    G = O.EdgeGraph(5, [0, 1, 3], [1, 2, 4], [1.0, 1.0, 1.0])
    ref = O.solve_path(Xc.astype(np.float64), None, G, [100.0], tol=1e-12)
    assert np.linalg.norm(U[0] - ref[0].U) <= 1e-6 * np.linalg.norm(ref[0].U)


def test_complete_graph(ccx):
    X, _ = synth.expression_like(16, 40, 3, 8, seed=4)
    n = 16
    ei, ej = np.triu_indices(n, 1)
    w = np.full(ei.size, 1.0 / ei.size)
    G = O.EdgeGraph(n, ei, ej, w)
    g0 = O.fusion_scale(X, None, ei, ej, w)
    gammas = [0.05 * g0, 0.3 * g0, 2.0 * g0]
    pr = ccx.Problem(X)
    pr.set_edges(ei, ej, w)
    U, labels, fused, stats, _ = solve_fused(pr, gammas)
    ref = O.solve_path(X.astype(np.float64), None, G, gammas, tol=1e-12)
    compare_path(U, labels, fused, stats, ref, X, None, G, 1e-4, "complete")


def test_deterministic_and_device_outputs(ccx):
    import torch
    X, _ = synth.gaussian_mixture(50, 17, 3, seed=8)
    G = knn_graph(X, None, 4, 0.05)
    gammas = [0.1, 1.0]
    outs = []
    for _ in range(2):
        pr = ccx.Problem(X)
        pr.set_edges(G.ei, G.ej, G.w)
        outs.append(pr.solve_path(gammas))
        pr.close()
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    pr = ccx.Problem(torch.from_numpy(X).cuda())
    pr.set_edges(G.ei, G.ej, G.w)
    Ud, Ld, _, _ = pr.solve_path(gammas, device=True)
    assert np.array_equal(Ud.cpu().numpy(), outs[0][0]) and np.array_equal(Ld.cpu().numpy(), outs[0][1])


def test_path_continues_across_calls(ccx):
    X, _ = synth.gaussian_mixture(30, 5, 3, seed=9)
    G = knn_graph(X, None, 4, 0.1)
    gammas = [0.02, 0.2, 2.0]
    pr = ccx.Problem(X)
    pr.set_edges(G.ei, G.ej, G.w)
    Ua, _, _, _ = pr.solve_path(gammas)
    pr.reset_path()
    Ub0, _, _, _ = pr.solve_path(gammas[:2])
    Ub1, _, _, _ = pr.solve_path(gammas[2:])
    ref = O.solve_path(X.astype(np.float64), None, G, gammas, tol=1e-12)
    for g in range(3):
        Ug = Ub0[g] if g < 2 else Ub1[g - 2]
        for Uc in (Ua[g], Ug):
            assert np.linalg.norm(Uc - ref[g].U) <= 1e-4 * np.linalg.norm(ref[g].U)


def test_invalid_inputs(ccx):
    X, _ = synth.gaussian_mixture(6, 2, 2, seed=1)
    bad = X.copy()
    bad[2, 1] = np.nan
    with pytest.raises(ccx.CcxError) as e:
        ccx.Problem(bad)
    assert e.value.status == 1
    m = np.ones((6, 2), np.uint8)
    m[3, :] = 0
    with pytest.raises(ccx.CcxError) as e:
        ccx.Problem(X, m)
    assert e.value.status == 1
    bad_m = bad.copy()
    mm = np.ones((6, 2), np.uint8)
    mm[2, 1] = 0      # the NaN is masked out: accepted
    ccx.Problem(bad_m, mm).close()
    pr = ccx.Problem(X)
    for ei, ej, w in (([0], [0], [1.0]), ([1], [0], [1.0]), ([0], [9], [1.0]), ([0], [1], [-1.0]),
                      ([0, 0], [1, 1], [1.0, 1.0]), ([0], [1], [np.inf])):
        with pytest.raises(ccx.CcxError) as e:
            pr.set_edges(ei, ej, w)
        assert e.value.status == 1
    pr.set_edges([0, 1], [1, 2], [1.0, 0.0])     # zero weight dropped
    assert pr.get_edges()[0].size == 1
    with pytest.raises(ccx.CcxError) as e:
        pr.solve_path([-1.0])
    assert e.value.status == 1
    with pytest.raises(ccx.CcxError) as e:
        pr.solve_path([np.nan])
    assert e.value.status == 1


@pytest.mark.parametrize("precision", [0, 1])
def test_standardize_matches_oracle(ccx, precision):
    """Observed-entry standardisation on the GPU (a constant column, a column with nothing observed,
    5 % missing) equals the oracle's, rounded once to float32; the kNN weights and the path on the
    standardised data then match the oracle's on its own standardised data."""
    G, mask, _ = synth.genotype_codes(90, 57, 3, seed=71, fst=0.05, frac_missing=0.05)
    G[:, 5] = 1.0                          # constant on its observed entries: centred only
    mask[:, 9] = 0                         # nothing observed: stays 0
    pr = ccx.Problem(G, mask, precision, standardize=True)
    Z = O.standardize(G, mask)
    Y = pr.get_start()
    ref = O.fill_missing(Z.astype(np.float32).astype(np.float64), mask)
    assert np.max(np.abs(Y - ref) / np.maximum(1.0, np.abs(ref))) <= 1e-6
    assert np.all(Y[:, 5] == 0.0) and np.all(Y[:, 9] == 0.0)
    Z32 = Z.astype(np.float32)
    pr.build_knn(6, phi_auto=True, normalize=True)
    ei, ej, w = pr.get_edges()
    oei, oej, ow, _, _ = O.knn_gaussian_weights(Z32.astype(np.float64), mask, 6, "auto", True)
    assert np.array_equal(ei, oei) and np.array_equal(ej, oej)
    assert np.allclose(w, ow, rtol=1e-6, atol=0)
    Gr = O.EdgeGraph(90, oei, oej, ow)
    g0 = O.fusion_scale(Z32, mask, oei, oej, ow)
    gammas = [0.05 * g0, 0.3 * g0, 2.0 * g0]
    U, labels, fused, stats, st = solve_fused(pr, gammas)
    assert st == 0
    ref_path = O.solve_path(Z32.astype(np.float64), mask, Gr, gammas, tol=1e-12)
    compare_path(U, labels, fused, stats, ref_path, Z32, mask, Gr, 1e-4, "standardised")
    # calling it again on standardised data changes nothing beyond rounding, and clears the edges
    pr.get_edges()
    import paper_1409_2065_gb300 as m
    m.binding.standardize(pr.h)
    assert pr.get_edges()[0].size == 0
    assert np.max(np.abs(pr.get_start() - Y)) <= 1e-6
    pr.close()


def test_size_limits_and_empty_grid(ccx):
    """The documented limits answer with CCX_EUNSUPPORTED (7) and a message, without running a kernel
    on sizes the kernels do not handle: n > 65535 for the iteration kernel (16-bit node indices), n > 4096
    for the kNN build.  An empty gamma grid returns at once with nothing written."""
    n = 70000
    X = np.linspace(0.0, 1.0, n, dtype=np.float32).reshape(n, 1)
    pr = ccx.Problem(X)
    ei = np.arange(n - 1)
    pr.set_edges(ei, ei + 1, np.ones(n - 1))
    with pytest.raises(ccx.CcxError) as e:
        pr.solve_path([0.1])
    assert e.value.status == 7 and "65535" in e.value.message
    with pytest.raises(ccx.CcxError) as e:
        pr.build_knn(3, phi=1.0)
    assert e.value.status == 7 and "4096" in e.value.message
    pr.close()
    Xs, _ = synth.gaussian_mixture(20, 3, 2, seed=3)
    pr = ccx.Problem(Xs)
    pr.build_knn(3, phi=0.1)
    U, labels, stats, st = pr.solve_path([])
    assert st == 0 and U.shape == (0, 20, 3) and labels.shape == (0, 20)
    pr.close()
