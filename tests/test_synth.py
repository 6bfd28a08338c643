"""The seeded synthetic inputs have the structure the workloads state: shapes,
value sets, standardisation, missing fractions, group structure, seeds."""
import numpy as np

import synth


def test_genotype_like_structure():
    X, mask, lab = synth.genotype_like(500, 2000, 5, seed=1, fst=0.05, frac_missing=0.05)
    assert X.shape == (500, 2000) and X.dtype == np.float32 and mask.dtype == np.uint8
    assert np.bincount(lab).tolist() == [100] * 5 and np.all(np.diff(lab) >= 0)
    obs = mask.astype(bool)
    assert abs(1.0 - obs.mean() - 0.05) < 0.005
    assert np.all(X[~obs] == 0.0)
    # standardised on the observed entries of every column (skip monomorphic columns)
    cnt = obs.sum(axis=0)
    mean = (X * obs).sum(axis=0) / cnt
    var = ((X - mean) ** 2 * obs).sum(axis=0) / cnt
    poly = var > 0
    assert np.abs(mean).max() < 1e-5 and np.abs(var[poly] - 1.0).max() < 1e-4
    # genotype codes: each standardised column takes at most three distinct observed values
    for c in range(0, 2000, 97):
        assert len(np.unique(np.round(X[obs[:, c], c], 5))) <= 3
    # population structure: between-population variance share of a column ~ Fst on average
    between = np.mean([np.var([X[lab == k, c][obs[lab == k, c]].mean() for k in range(5)])
                       for c in range(0, 2000, 10)])
    assert 0.02 < between < 0.12
    # the same seed gives the same data
    X2, mask2, _ = synth.genotype_like(500, 2000, 5, seed=1, fst=0.05, frac_missing=0.05)
    assert np.array_equal(X, X2) and np.array_equal(mask, mask2)


def test_expression_like_structure():
    X, lab = synth.expression_like(60, 3000, 3, 200, seed=2)
    assert X.shape == (60, 3000) and np.bincount(lab).tolist() == [20, 20, 20]
    assert np.abs(X.mean(axis=0)).max() < 1e-5
    assert np.abs(X.var(axis=0) - 1.0).max() < 1e-4
    # each group's own gene block is shifted up: its block mean is clearly above the others'
    rng = np.random.default_rng(2)
    rng.normal(0.0, 1.0, size=(60, 3000))           # the draws the generator makes before the permutation
    genes = rng.permutation(3000)
    for g in range(3):
        block = genes[g * 200:(g + 1) * 200]
        inside = X[lab == g][:, block].mean()
        outside = X[lab != g][:, block].mean()
        assert inside - outside > 0.5


def test_gaussian_mixture_and_grids():
    X, lab = synth.gaussian_mixture(203, 7, 4, seed=0)
    assert X.shape == (203, 7) and np.bincount(lab).tolist() == [51, 51, 51, 50]
    g = synth.log_grid(1e-3, 10.0, 20)
    assert g.size == 20 and g[0] == 1e-3 and abs(g[-1] - 10.0) < 1e-12
    assert np.allclose(np.diff(np.log(g)), np.log(1e4) / 19)
    t = synth.poisson_arrivals(50.0, 4000, seed=4)
    assert np.all(np.diff(t) > 0) and abs(np.mean(np.diff(t)) - 0.02) < 0.002
    probs = synth.batched_problems(6, seed=3)
    assert [pp["seed"] for pp in probs] == [3000 + i for i in range(6)]
    assert all(50 <= pp["n"] <= 2000 and 10 <= pp["p"] <= 5000 and 2 <= pp["k"] <= 8 for pp in probs)
