"""Write the stored expected values of the GPU parity tests.

Calls only the FP64 oracle (oracle/) and the seeded generators (synth/).
Run from the repository root:  python tests/golden/make_golden.py

plain_n200_p10.npz -- the "plain" workload: n = 200, p = 10, 4 Gaussian
clusters (means ~ N(0, 9 I), noise N(0, I)), seed 0; kNN k = 10 with
w_ij = exp(-0.5 ||x_i - x_j||^2) unnormalised; 20 gamma log-spaced 1e-3..1e1;
no missing data.  Stores X, the edge set, the gamma grid and, per gamma, the
oracle's U, fused flags, labels and d.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
import synth  # noqa: E402


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
        iters=np.array([r.iters for r in res]), converged=np.array([r.converged for r in res]))
    print("plain_n200_p10: iters", [r.iters for r in res], "fused", [int(r.fused.sum()) for r in res])


if __name__ == "__main__":
    plain_n200()
