"""Parity with the FP64 oracle on the iteration kernel's multi-slice path, and the
near-threshold fuse decision, through the C ABI.

The benchmark workload gives every CTA of the iteration kernel many 4-column
slices: the slice loop, the staging of the next slice while the current one is
processed, and the float accumulation of each edge's ||b||^2 over a CTA's
slices all run there.  The stored cases (written by tests/golden/make_golden.py,
which calls only the oracle) have p large enough for four to nine slices per
CTA on a 152-SM GB300.

Bar, per gamma:
  * U: relative Frobenius error <= 1e-4 (FP32 path), on the whole matrix or on
    the stored rows, and every row's norm within 1e-4 of the whole matrix's norm
    over sqrt(n);
  * fused flags equal edge by edge, except edges whose oracle margin
    |mu w d / (rho ||b||) - 1| is below 1e-5; labels equal to the oracle's when
    every flag agrees, else equal to the components of the GPU's own flags;
  * the two staging variants bit-identical to each other.
"""
import os

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
MARGIN = 1e-5


@pytest.fixture(scope="module")
def ccx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_1409_2065_gb300 as m
    return m


def _sms():
    import torch
    return torch.cuda.get_device_properties(0).multi_processor_count


def check_fused(fused, labels, z, g, n, tag):
    """Edge-by-edge fused flags against the oracle's, outside the rounding band; then labels."""
    ref = z["fused"][g].astype(bool)
    got = fused.astype(bool)
    far = np.abs(z["margin"][g]) >= MARGIN
    bad = np.nonzero((got != ref) & far)[0]
    assert bad.size == 0, f"{tag} gamma {g}: fused flags differ on edges {bad[:10]} (margins {z['margin'][g][bad[:10]]})"
    if np.array_equal(got, ref):
        assert np.array_equal(labels, z["labels"][g]), f"{tag} gamma {g}: labels differ with equal fused sets"
    else:
        own = O.fused_labels(n, z["ei"], z["ej"], got)
        assert np.array_equal(labels, own), f"{tag} gamma {g}: labels are not the components of the fused set"


def run(ccx, pr, gammas, m, **opt):
    o = ccx.opts_default()
    for k, v in opt.items():
        setattr(o, k, v)
    fused = np.zeros((len(gammas), m), np.uint8)
    U, L, stats, st = pr.solve_path(gammas, o, fused_out=fused)
    assert st == 0, st
    return U, L, fused, stats


@pytest.fixture(scope="module")
def genotype():
    return dict(np.load(os.path.join(GOLDEN, "genotype_n48_p2502.npz")))


@pytest.mark.parametrize("variant", [1, 2])
def test_genotype_multislice_against_stored_oracle(ccx, genotype, variant):
    """n = 48, p = 2502 (626 slices, a 2-column tail), 5 % missing, kNN k = 10: four or five slices
    per CTA, with the double-buffered (1) and the single-buffer (2) staging of slices."""
    z = genotype
    n, p = z["X"].shape
    assert (p + 3) // 4 >= 4 * _sms()          # several slices per CTA
    pr = ccx.Problem(z["X"], z["mask"], ccx.CCX_FP32)
    pr.build_knn(10, phi_auto=True, normalize=True)
    ei, ej, w = pr.get_edges()
    assert np.array_equal(ei, z["ei"]) and np.array_equal(ej, z["ej"])
    assert np.allclose(w, z["w"], rtol=1e-12, atol=0)
    U, L, F, stats = run(ccx, pr, z["gammas"], ei.size, slice_variant=variant)
    for g in range(len(z["gammas"])):
        ref = z["U"][g].astype(np.float64)
        err = np.linalg.norm(U[g] - ref) / np.linalg.norm(ref)
        assert err <= 1e-4, (g, err)
        assert stats[g]["converged"] in (1, 2), (g, stats[g])
        check_fused(F[g], L[g], z, g, n, f"genotype v{variant}")
        if np.min(np.abs(z["margin"][g])) > 1e-4:
            assert stats[g]["n_recomputed"] == 0, (g, stats[g])
    assert 0 < int(z["fused"].sum(axis=1).max()) and int(z["fused"][0].sum()) == 0   # the grid spans fusion
    pr.close()


def test_genotype_multislice_fp64_path(ccx, genotype):
    """The FP64 instantiation of the iteration kernel on the same multi-slice case (double rows, float
    per-edge partials, so near-threshold decisions go through the double recompute): U within 1e-6 of
    the oracle (the stored values are float32, 6e-8 relative), fused flags and labels as above."""
    z = genotype
    n, p = z["X"].shape
    pr = ccx.Problem(z["X"], z["mask"], ccx.CCX_FP64)
    pr.set_edges(z["ei"], z["ej"], z["w"])
    U, L, F, stats = run(ccx, pr, z["gammas"], z["ei"].size)
    for g in range(len(z["gammas"])):
        ref = z["U"][g].astype(np.float64)
        err = np.linalg.norm(U[g] - ref) / np.linalg.norm(ref)
        assert err <= 1e-6, (g, err)
        assert stats[g]["converged"] in (1, 2), (g, stats[g])
        check_fused(F[g], L[g], z, g, n, "genotype fp64")
    pr.close()


def test_genotype_staging_variants_identical_and_grid_cap(ccx, genotype):
    """The two staging variants compute the same arithmetic in the same order: bit-identical results.
    A grid of 16 CTAs (39 or 40 slices each) still matches the oracle."""
    z = genotype
    n, p = z["X"].shape
    out = []
    for variant in (1, 2):
        pr = ccx.Problem(z["X"], z["mask"], ccx.CCX_FP32)
        pr.set_edges(z["ei"], z["ej"], z["w"])
        out.append(run(ccx, pr, z["gammas"][:3], z["ei"].size, slice_variant=variant))
        pr.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][2], out[1][2])
    assert [s["iters"] for s in out[0][3]] == [s["iters"] for s in out[1][3]]
    pr = ccx.Problem(z["X"], z["mask"], ccx.CCX_FP32)
    pr.set_edges(z["ei"], z["ej"], z["w"])
    U, L, F, stats = run(ccx, pr, z["gammas"], z["ei"].size, max_ctas=16)
    for g in range(len(z["gammas"])):
        ref = z["U"][g].astype(np.float64)
        assert np.linalg.norm(U[g] - ref) / np.linalg.norm(ref) <= 1e-4, g
        check_fused(F[g], L[g], z, g, n, "genotype 16 CTAs")
    pr.close()


def test_allpairs_multislice_against_stored_oracle(ccx):
    """n = 32, p = 5000 (1250 slices, eight or nine per CTA), all 496 pairs: stored rows element by
    element, every row's norm, fused flags and labels."""
    z = dict(np.load(os.path.join(GOLDEN, "allpairs_n32_p5000.npz")))
    import synth
    X, _ = synth.expression_like(32, 5000, 3, 150, seed=62)
    n, p = X.shape
    assert (p + 3) // 4 >= 8 * _sms()
    pr = ccx.Problem(X, None, ccx.CCX_FP32)
    pr.build_knn(31, phi_auto=True, normalize=True)
    ei, ej, w = pr.get_edges()
    assert ei.size == 496 and np.array_equal(ei, z["ei"]) and np.array_equal(ej, z["ej"])
    assert np.allclose(w, z["w"], rtol=1e-12, atol=0)
    U, L, F, stats = run(ccx, pr, z["gammas"], ei.size)
    rows = z["rows"]
    for g in range(len(z["gammas"])):
        ref = z["U_rows"][g].astype(np.float64)
        err = np.linalg.norm(U[g][rows] - ref) / np.linalg.norm(ref)
        assert err <= 1e-4, (g, err)
        rn = np.linalg.norm(U[g].astype(np.float64), axis=1)
        assert np.max(np.abs(rn - z["row_norm"][g])) <= 1e-4 * z["fro"][g] / np.sqrt(n), g
        assert stats[g]["converged"] in (1, 2)
        check_fused(F[g], L[g], z, g, n, "allpairs")
    pr.close()


def test_threshold_edge_recomputed_in_double(ccx):
    """An edge whose oracle margin is 1.8e-7 at the stored penalty (the gamma at which it fuses): the
    fuse decision is taken from ||b|| recomputed in double, n_recomputed counts it, and the labels equal
    the oracle's.  With the recompute off nothing is counted."""
    z = dict(np.load(os.path.join(GOLDEN, "threshold_edge.npz")))
    e = int(z["edge"])
    assert abs(z["margin"][e]) < 3e-7 and np.sort(np.abs(z["margin"]))[1] > 1e-2
    m = z["ei"].size
    pr = ccx.Problem(z["X"], None, ccx.CCX_FP64)
    pr.set_edges(z["ei"], z["ej"], z["w"])
    U, L, F, stats = run(ccx, pr, [float(z["gamma"])], m, tol=1e-13)
    assert stats[0]["n_recomputed"] >= 1 and stats[0]["recomputes"] >= 1, stats[0]
    assert np.array_equal(F[0].astype(bool), z["fused"]), (F[0], z["fused"])
    assert np.array_equal(L[0], z["labels"])
    assert np.linalg.norm(U[0] - z["U"]) <= 1e-6 * np.linalg.norm(z["U"])
    pr.close()
    pr = ccx.Problem(z["X"], None, ccx.CCX_FP64)
    pr.set_edges(z["ei"], z["ej"], z["w"])
    U2, L2, F2, stats2 = run(ccx, pr, [float(z["gamma"])], m, tol=1e-13, fuse_delta=0.0)
    assert stats2[0]["n_recomputed"] == 0 and stats2[0]["recomputes"] == 0
    pr.close()
