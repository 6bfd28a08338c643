"""Write the stored expected values of the GPU parity tests.

Calls only the FP64 oracle (oracle/) and the seeded generators (synth/).
Run from the repository root:  python tests/golden/make_golden.py [name ...]

plain_n200_p10.npz -- the "plain" workload: n = 200, p = 10, 4 Gaussian
clusters (means ~ N(0, 9 I), noise N(0, I)), seed 0; kNN k = 10 with
w_ij = exp(-0.5 ||x_i - x_j||^2) unnormalised; 20 gamma log-spaced 1e-3..1e1;
no missing data.  Stores X, the edge set, the gamma grid and, per gamma, the
oracle's U, fused flags, labels, d and each edge's signed margin
mu w d / (rho ||b||) - 1 at the oracle's fixed point.

genotype_n48_p2502.npz -- genotype-like data (5 Balding-Nichols populations,
Fst = 0.05, seed 61, 5 % missing) with n = 48 cases and p = 2502 SNPs: 626
four-column slices, the last one two columns wide, so one CTA per SM of a
GB300 processes four or five slices -- the multi-slice loop, the staging of
the next slice and the float accumulation of ||b||^2 over a CTA's slices that
the benchmark workload runs.  kNN k = 10, phi automatic, normalised weights;
five gammas from before the first fusion to complete fusion.  Stores the
whole of U per gamma (float32), the fused flags, labels, d and each edge's
margin |mu w d / (rho ||b||) - 1| at the oracle's fixed point.

allpairs_n32_p5000.npz -- expression-like data (log-normal, 3 groups with
150 up-shifted genes each, seed 62) with n = 32 samples and p = 5000 genes,
all 496 pairs weighted (phi automatic, normalised): 1250 slices, eight or
nine per CTA.  Five gammas around the abrupt fusion of the complete graph.
Stores 12 fixed rows of U per gamma (float32) and the norm of every row, the
fused flags, labels, d and margins.

threshold_edge.npz -- a 12-case problem (3 Gaussian clusters, p = 3, kNN
k = 3, phi = 0.1) at the penalty where its first edge fuses, found by
bisection on gamma so that the oracle's margin of that edge is below 3e-7:
the fuse decision there sits within the rounding of float partial sums.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
import synth  # noqa: E402


def _margins(r, G):
    """Signed margin mu w d / (rho ||b||) - 1 of every edge at an oracle fixed point (>= 0: fused)."""
    _, B = O.project(r.U, r.V, G)
    nb = np.linalg.norm(B, axis=1)
    return r.mu * G.w * r.d / (r.rho * np.maximum(nb, 1e-300)) - 1.0


def plain_n200():
    X, lab = synth.gaussian_mixture(200, 10, 4, seed=0)
    Xd = X.astype(np.float64)
    ei, ej, w, d2, phi = O.knn_gaussian_weights(Xd, None, 10, 0.5, False)
    G = O.EdgeGraph(200, ei, ej, w)
    gammas = synth.log_grid(1e-3, 1e1, 20)
    res = O.solve_path(Xd, None, G, gammas, tol=1e-12)
    np.savez_compressed(
        os.path.join(HERE, "plain_n200_p10.npz"), X=X, ei=ei, ej=ej, w=w, gammas=gammas,
        U=np.stack([r.U for r in res]), fused=np.stack([r.fused for r in res]),
        labels=np.stack([r.labels for r in res]), d=np.array([r.d for r in res]),
        iters=np.array([r.iters for r in res]), converged=np.array([r.converged for r in res]),
        margin=np.stack([_margins(r, G) for r in res]))
    print("plain_n200_p10: iters", [r.iters for r in res], "fused", [int(r.fused.sum()) for r in res])


def _path_arrays(res, G, rows=None):
    U = np.stack([r.U for r in res])
    out = dict(fused=np.stack([r.fused for r in res]), labels=np.stack([r.labels for r in res]),
               d=np.array([r.d for r in res]), iters=np.array([r.iters for r in res]),
               converged=np.array([r.converged for r in res]), margin=np.stack([_margins(r, G) for r in res]),
               row_norm=np.linalg.norm(U, axis=2), fro=np.linalg.norm(U, axis=(1, 2)))
    if rows is None:
        out["U"] = U.astype(np.float32)
    else:
        out["rows"] = np.asarray(rows)
        out["U_rows"] = U[:, rows, :].astype(np.float32)
    return out


def genotype_n48():
    X, mask, _ = synth.genotype_like(48, 2502, 5, seed=61, fst=0.05, frac_missing=0.05)
    Xd = X.astype(np.float64)
    ei, ej, w, _, phi = O.knn_gaussian_weights(Xd, mask, 10, "auto", True)
    G = O.EdgeGraph(48, ei, ej, w)
    g0 = O.fusion_scale(Xd, mask, ei, ej, w)
    gammas = g0 * np.array([0.05, 0.22, 0.24, 0.27, 0.4])
    res = O.solve_path(Xd, mask, G, gammas, tol=1e-12)
    np.savez_compressed(os.path.join(HERE, "genotype_n48_p2502.npz"), X=X, mask=mask, ei=ei, ej=ej, w=w,
                        gammas=gammas, g0=g0, **_path_arrays(res, G))
    print("genotype_n48_p2502: iters", [r.iters for r in res], "fused", [int(r.fused.sum()) for r in res],
          "of", G.m, "converged", [r.converged for r in res])


def allpairs_n32():
    X, _ = synth.expression_like(32, 5000, 3, 150, seed=62)
    Xd = X.astype(np.float64)
    ei, ej, w, _, phi = O.knn_gaussian_weights(Xd, None, 31, "auto", True)
    G = O.EdgeGraph(32, ei, ej, w)
    g0 = O.fusion_scale(Xd, None, ei, ej, w)
    gammas = g0 * np.array([0.03, 0.062, 0.065, 0.068, 0.12])
    res = O.solve_path(Xd, None, G, gammas, tol=1e-12)
    rows = np.sort(np.random.default_rng(63).choice(32, 12, replace=False))
    np.savez_compressed(os.path.join(HERE, "allpairs_n32_p5000.npz"), ei=ei, ej=ej, w=w, gammas=gammas, g0=g0,
                        **_path_arrays(res, G, rows))
    print("allpairs_n32_p5000: iters", [r.iters for r in res], "fused", [int(r.fused.sum()) for r in res],
          "of", G.m, "converged", [r.converged for r in res])


def threshold_edge():
    X, _ = synth.gaussian_mixture(12, 3, 3, seed=5)
    Xd = X.astype(np.float64)
    ei, ej, w, _, _ = O.knn_gaussian_weights(Xd, None, 3, 0.1, False)
    G = O.EdgeGraph(12, ei, ej, w)
    Y0 = O.fill_missing(Xd, None)

    def solve(mu, U0=None, V0=None):
        rho, eps = O.pd_constants(Y0, G.w, mu)
        U0 = Y0 if U0 is None else U0
        V0 = np.zeros((G.m, 3)) if V0 is None else V0
        U, V, d, fz, it, res, ok = O.solve_gamma(Xd, None, G, mu, rho, eps, U0, V0, tol=1e-14, max_iter=2_000_000)
        assert ok
        r = O.GammaResult(mu, rho, eps, U, V, d, fz, O.fused_labels(12, G.ei, G.ej, fz), it, res, ok)
        return r

    # the first gamma of a log grid at which some edge fuses, then bisection in
    # log gamma on the signed margin of the edge that fuses first
    grid = np.logspace(-3, 2, 60)
    prev = solve(grid[0])
    assert not prev.fused.any()
    for mu in grid[1:]:
        cur = solve(mu, prev.U, prev.V)
        if cur.fused.any():
            break
        prev = cur
    e = int(np.argmax(_margins(cur, G)))
    lo, hi, r_lo = prev.mu, cur.mu, prev
    for _ in range(200):
        mid = float(np.sqrt(lo * hi))
        r = solve(mid, r_lo.U, r_lo.V)
        m = _margins(r, G)[e]
        if abs(m) < 3e-7 and m > 0:
            break
        if m >= 0:
            hi = mid
        else:
            lo, r_lo = mid, r
    m_all = _margins(r, G)
    order = np.sort(np.abs(m_all))
    np.savez_compressed(os.path.join(HERE, "threshold_edge.npz"), X=X, ei=ei, ej=ej, w=w, gamma=r.mu, edge=e,
                        U=r.U, fused=r.fused, labels=r.labels, d=r.d, margin=m_all)
    print("threshold_edge: gamma", r.mu, "edge", e, "margin", m_all[e], "next smallest |margin|", order[1],
          "fused", int(r.fused.sum()))


CASES = {"plain": plain_n200, "genotype": genotype_n48, "allpairs": allpairs_n32, "threshold": threshold_edge}

if __name__ == "__main__":
    for name in (sys.argv[1:] or list(CASES)):
        CASES[name]()
