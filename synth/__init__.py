"""Seeded synthetic inputs for the convex-clustering solver and its oracle.

This module only draws data.  It holds none of the clustering method's
arithmetic (no distances, weights, projections or shrinkage); the solver
library and the FP64 oracle both take what it returns as plain inputs.

Recipes (all rows are cases, columns are predictors; float32 at the
boundary):

* ``gaussian_mixture`` -- ``n`` points in ``p`` dimensions split into
  ``k`` equal clusters; cluster means ~ N(0, 9 I), points = mean + N(0, I).
  This is the "plain" workload (n=200, p=10, 4 clusters, seed 0).
* ``genotype_codes`` / ``genotype_like`` -- Balding-Nichols allele frequencies: ancestral
  frequency p0 ~ U(0.05, 0.5) per SNP, population frequency
  ~ Beta(p0 (1-F)/F, (1-p0)(1-F)/F), genotype ~ Binomial(2, freq); codes
  are standardised with the observed entries and a fraction of entries is
  masked missing (iid).  Stands in for the paper's microsatellite/SNP data
  (HGDP, POPRES), which are not available here.
* ``expression_like`` -- log-normal expression, z ~ N(0, 1) with a mean
  shift of +1 on each group's own disjoint block of genes, x = exp(z),
  columns standardised.  Stands in for the breast-cancer microarray.
* ``batched_problems`` -- many independent Gaussian-mixture problems with
  uneven sizes n ~ U[n_lo, n_hi], p ~ U[p_lo, p_hi], 2-8 clusters.
* ``poisson_arrivals`` -- arrival times of a Poisson process.

Standardisation (centre each column on its observed mean, divide by its
observed standard deviation, centre only when that deviation is zero) is
data preparation, done here in float64 and rounded once to float32, so
every consumer sees the same float32 matrix.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "gaussian_mixture",
    "genotype_codes",
    "genotype_like",
    "expression_like",
    "batched_problems",
    "poisson_arrivals",
    "standardize_observed",
    "log_grid",
    "random_mask",
]


def standardize_observed(X: np.ndarray, mask: np.ndarray | None) -> np.ndarray:
    """Centre and scale columns using observed entries only (float64 in, float64 out).

    Missing entries are left at 0 after centring (their value is never used
    as data: the solver treats them through the mask).
    """
    X = np.asarray(X, dtype=np.float64)
    obs = np.ones(X.shape, dtype=bool) if mask is None else mask.astype(bool)
    cnt = obs.sum(axis=0)
    safe = np.maximum(cnt, 1)
    mean = np.where(obs, X, 0.0).sum(axis=0) / safe
    dev = np.where(obs, X - mean, 0.0)
    var = (dev * dev).sum(axis=0) / safe
    sd = np.sqrt(var)
    scale = np.where(sd > 0, sd, 1.0)
    return np.where(obs, dev / scale, 0.0)


def random_mask(rng: np.random.Generator, n: int, p: int, frac_missing: float) -> np.ndarray:
    """uint8 mask, 1 = observed, 0 = missing, iid with the given missing fraction."""
    return (rng.random((n, p)) >= frac_missing).astype(np.uint8)


def gaussian_mixture(n: int = 200, p: int = 10, k: int = 4, seed: int = 0,
                     mean_sd: float = 3.0, noise_sd: float = 1.0):
    """Gaussian clusters of (near) equal size.  Returns (X float32 n x p, cluster ids)."""
    rng = np.random.default_rng(seed)
    means = rng.normal(0.0, mean_sd, size=(k, p))
    sizes = [n // k + (1 if c < n % k else 0) for c in range(k)]
    lab = np.repeat(np.arange(k), sizes)
    X = means[lab] + rng.normal(0.0, noise_sd, size=(n, p))
    return X.astype(np.float32), lab


def genotype_codes(n: int = 1000, p: int = 10000, pops: int = 5, seed: int = 1,
                   fst: float = 0.05, frac_missing: float = 0.05):
    """Balding-Nichols genotype codes {0, 1, 2}, unstandardised.

    Returns (codes float32 n x p, mask uint8 n x p (1 = observed), population ids).
    """
    rng = np.random.default_rng(seed)
    p0 = rng.uniform(0.05, 0.5, size=p)
    a = p0 * (1.0 - fst) / fst
    b = (1.0 - p0) * (1.0 - fst) / fst
    freq = rng.beta(a, b, size=(pops, p))
    sizes = [n // pops + (1 if c < n % pops else 0) for c in range(pops)]
    lab = np.repeat(np.arange(pops), sizes)
    G = rng.binomial(2, freq[lab]).astype(np.float32)
    mask = random_mask(rng, n, p, frac_missing)
    return G, mask, lab


def genotype_like(n: int = 1000, p: int = 10000, pops: int = 5, seed: int = 1,
                  fst: float = 0.05, frac_missing: float = 0.05):
    """Balding-Nichols genotypes (genotype_codes), standardised on observed entries.

    Returns (X float32 n x p, mask uint8 n x p (1 = observed), population ids).
    """
    G, mask, lab = genotype_codes(n, p, pops, seed, fst, frac_missing)
    X = standardize_observed(G, mask)
    return X.astype(np.float32), mask, lab


def expression_like(n: int = 100, p: int = 20000, groups: int = 3, shift_genes: int = 500,
                    seed: int = 2, shift: float = 1.0):
    """Log-normal expression with group-specific up-shifted gene blocks, standardised.

    Returns (X float32 n x p, group ids).
    """
    rng = np.random.default_rng(seed)
    sizes = [n // groups + (1 if c < n % groups else 0) for c in range(groups)]
    lab = np.repeat(np.arange(groups), sizes)
    z = rng.normal(0.0, 1.0, size=(n, p))
    genes = rng.permutation(p)
    for g in range(groups):
        block = genes[g * shift_genes:(g + 1) * shift_genes]
        rows = np.nonzero(lab == g)[0]
        z[np.ix_(rows, block)] += shift
    X = standardize_observed(np.exp(z), None)
    return X.astype(np.float32), lab


def batched_problems(count: int = 256, seed: int = 3, n_lo: int = 50, n_hi: int = 2000,
                     p_lo: int = 10, p_hi: int = 5000, k_lo: int = 2, k_hi: int = 8):
    """Independent Gaussian-mixture problems of uneven size; problem i uses seed 1000*seed + i.

    Returns a list of dicts with keys X (float32), n, p, k, seed.
    """
    out = []
    for i in range(count):
        s = 1000 * seed + i
        rng = np.random.default_rng(s)
        n = int(rng.integers(n_lo, n_hi + 1))
        p = int(rng.integers(p_lo, p_hi + 1))
        k = int(rng.integers(k_lo, k_hi + 1))
        X, lab = gaussian_mixture(n, p, k, seed=s)
        out.append({"X": X, "n": n, "p": p, "k": k, "seed": s, "labels": lab})
    return out


def poisson_arrivals(rate: float, count: int, seed: int = 4) -> np.ndarray:
    """Arrival times (seconds from 0) of ``count`` jobs of a Poisson process."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=count))


def log_grid(lo: float, hi: float, count: int) -> np.ndarray:
    """``count`` log-spaced values from lo to hi inclusive (float64)."""
    if count == 1:
        return np.array([lo], dtype=np.float64)
    return np.logspace(np.log10(lo), np.log10(hi), count)
