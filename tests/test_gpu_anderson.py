"""Anderson mixing of the MM map (ccx_opts.anderson) against the FP64 oracle, through the C ABI.

The mixing changes the route to the fixed point, not the fixed point: every case here must meet
the same bar as without it (U relative Frobenius error <= 1e-4 on the FP32 path, <= 1e-6 on the
FP64 path; fused flags edge by edge outside the 1e-5 rounding band; labels), and gammas before any
fusion must actually have been mixed.
"""
import os

import numpy as np
import pytest

import oracle as O
import synth
from tests.test_gpu_multislice import check_fused

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def ccx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_1409_2065_gb300 as m
    return m


def _opts(ccx, m, **kw):
    o = ccx.opts_default()
    o.anderson = m
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _solve(ccx, pr, gammas, o):
    fused = np.zeros((len(gammas), pr.get_edges()[0].size), np.uint8)
    U, L, stats, st = pr.solve_path(gammas, o, fused_out=fused)
    assert st == 0, st
    return U, L, fused, stats


@pytest.mark.parametrize("m", [3, 5, 8, 16])
def test_genotype_multislice_with_mixing(ccx, m):
    """The stored genotype-like case (n = 48, p = 2502, 5 % missing): the first gamma (no fusion) is
    mixed, the second starts mixed and hands over when its edges fuse, later ones are not mixed."""
    z = dict(np.load(os.path.join(GOLDEN, "genotype_n48_p2502.npz")))
    n = z["X"].shape[0]
    pr = ccx.Problem(z["X"], z["mask"], ccx.CCX_FP32)
    pr.set_edges(z["ei"], z["ej"], z["w"])
    U, L, F, stats = _solve(ccx, pr, z["gammas"], _opts(ccx, m))
    for g in range(len(z["gammas"])):
        ref = z["U"][g].astype(np.float64)
        err = np.linalg.norm(U[g] - ref) / np.linalg.norm(ref)
        assert err <= 1e-4, (g, err, stats[g])
        assert stats[g]["converged"] in (1, 2), (g, stats[g])
        check_fused(F[g], L[g], z, g, n, f"genotype aa{m}")
    assert stats[0]["mixing_iters"] > 0
    assert all(s["mixing_iters"] == 0 for s in stats[2:])
    pr.close()


def test_allpairs_multislice_with_mixing(ccx):
    """The stored all-pairs case (n = 32, p = 5000, 496 edges, eight or nine slices per CTA) with
    mixing: stored rows element by element, every row's norm, fused flags and labels."""
    z = dict(np.load(os.path.join(GOLDEN, "allpairs_n32_p5000.npz")))
    X, _ = synth.expression_like(32, 5000, 3, 150, seed=62)
    n = X.shape[0]
    pr = ccx.Problem(X, None, ccx.CCX_FP32)
    pr.set_edges(z["ei"], z["ej"], z["w"])
    U, L, F, stats = _solve(ccx, pr, z["gammas"], _opts(ccx, 5))
    rows = z["rows"]
    for g in range(len(z["gammas"])):
        ref = z["U_rows"][g].astype(np.float64)
        err = np.linalg.norm(U[g][rows] - ref) / np.linalg.norm(ref)
        assert err <= 1e-4, (g, err, stats[g])
        rn = np.linalg.norm(U[g].astype(np.float64), axis=1)
        assert np.max(np.abs(rn - z["row_norm"][g])) <= 1e-4 * z["fro"][g] / np.sqrt(n), g
        assert stats[g]["converged"] in (1, 2), (g, stats[g])
        check_fused(F[g], L[g], z, g, n, "allpairs aa5")
    assert stats[0]["mixing_iters"] > 0
    pr.close()


@pytest.mark.parametrize("precision,utol", [(1, 1e-6), (0, 1e-4)])
def test_plain_workload_with_mixing(ccx, precision, utol):
    """n = 200, p = 10, 20 gammas against the stored oracle values; the 17 gammas before the first
    fusion are mixed."""
    z = np.load(os.path.join(GOLDEN, "plain_n200_p10.npz"))
    pr = ccx.Problem(z["X"], None, precision)
    pr.set_edges(z["ei"], z["ej"], z["w"])
    U, L, F, stats = _solve(ccx, pr, z["gammas"], _opts(ccx, 5))
    zz = dict(z)
    for g in range(len(z["gammas"])):
        err = np.linalg.norm(U[g] - z["U"][g]) / np.linalg.norm(z["U"][g])
        assert err <= utol, (g, err, stats[g])
        assert stats[g]["converged"] in (1, 2)
        check_fused(F[g], L[g], zz, g, 200, f"plain aa p{precision}")
    assert stats[0]["mixing_iters"] > 0
    pr.close()


def test_ragged_missing_with_mixing_and_determinism(ccx):
    X, _ = synth.gaussian_mixture(70, 37, 4, seed=11)
    mask = synth.random_mask(np.random.default_rng(12), 70, 37, 0.1)
    ei, ej, w, _, _ = O.knn_gaussian_weights(X.astype(np.float64), mask, 5, 0.02, False)
    G = O.EdgeGraph(70, ei, ej, w)
    g0 = O.fusion_scale(X, mask, ei, ej, w)
    gammas = synth.log_grid(1e-2 * g0, 3.0 * g0, 5)
    ref = O.solve_path(X.astype(np.float64), mask, G, gammas, tol=1e-12)
    outs = []
    for _ in range(2):
        pr = ccx.Problem(X, mask, ccx.CCX_FP32)
        pr.set_edges(ei, ej, w)
        outs.append(_solve(ccx, pr, gammas, _opts(ccx, 5)))
        pr.close()
    U, L, F, stats = outs[0]
    for g, r in enumerate(ref):
        assert np.linalg.norm(U[g] - r.U) <= 1e-4 * np.linalg.norm(r.U), (g, stats[g])
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][2], outs[1][2])


def test_batch_with_mixing_equals_alone(ccx):
    specs = []
    rng = np.random.default_rng(31)
    for i in range(4):
        n, p = int(rng.integers(40, 200)), int(rng.integers(5, 90))
        X, _ = synth.gaussian_mixture(n, p, 3, seed=3100 + i)
        specs.append(X)
    o = _opts(ccx, 4)
    alone, probs, grids = [], [], []
    for X in specs:
        pr = ccx.Problem(X)
        pr.build_knn(6, phi_auto=True, normalize=True)
        g0 = pr.fusion_scale()
        gam = synth.log_grid(0.03 * g0, 3.0 * g0, 6)
        U, L, _, st = pr.solve_path(gam, o)
        assert st == 0
        alone.append((U, L))
        pr.reset_path()
        probs.append(pr)
        grids.append(gam)
    Us, Ls, stats, status, st = ccx.solve_batch(probs, grids, opts=o, max_active=4)
    assert st == 0 and all(s == 0 for s in status)
    for i in range(len(specs)):
        assert np.array_equal(Us[i], alone[i][0]) and np.array_equal(Ls[i], alone[i][1]), i
    for pr in probs:
        pr.close()


def test_time_iterations_mixing(ccx):
    """The instrumentation call times the mixing kernels (positive mean times at a gamma before any
    fusion) and refuses a history of 0."""
    X, mask, _ = synth.genotype_like(120, 64, 3, seed=5, fst=0.05, frac_missing=0.05)
    pr = ccx.Problem(X, mask, ccx.CCX_FP32)
    pr.build_knn(6, phi_auto=True, normalize=True)
    g0 = pr.fusion_scale()
    a, b, c = pr.time_iterations_mixing(0.01 * g0, 20, _opts(ccx, 4))
    assert a > 0 and b > 0 and c > 0
    with pytest.raises(ccx.CcxError):
        pr.time_iterations_mixing(0.01 * g0, 20, _opts(ccx, 0))
    a, b, c16 = pr.time_iterations_mixing(0.01 * g0, 20, _opts(ccx, 16))   # the long-history kernels
    assert c16 > 0
    with pytest.raises(ccx.CcxError):                 # above the longest history
        pr.solve_path([0.01 * g0], _opts(ccx, 17))
    pr.close()
