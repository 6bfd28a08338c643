"""Feature-sharded iteration (ccx_shard_*) on one GPU, through the C ABI.

One problem is split by columns into shard problems that share its edge set;
per MM iteration every shard runs its column work, the shards' partial sums
are stacked in shard order (the exchange that ranks would do with an
all-gather), and every shard reduces them in that order.  The shards here run
one after another on one GPU; no kernel waits on another shard's kernel.

Bar: one shard reproduces ccx_solve_path bit for bit; two or three shards agree
with the unsharded path within the rounding of the partial sums (FP64: 1e-8
relative; FP32: 2e-5) and with the stored FP64 oracle within 1e-4, with the
same labels.
"""
import os

import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def ccx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_1409_2065_gb300 as m
    return m


def _shards(ccx, X, mask, cuts, edges, precision):
    out = []
    for a, b in zip(cuts[:-1], cuts[1:]):
        pr = ccx.Problem(np.ascontiguousarray(X[:, a:b]),
                         None if mask is None else np.ascontiguousarray(mask[:, a:b]), precision)
        pr.set_edges(*edges)
        out.append(pr)
    return out


def _ragged():
    X, _ = synth.gaussian_mixture(70, 37, 4, seed=11)
    mask = synth.random_mask(np.random.default_rng(12), 70, 37, 0.1)
    G = O.knn_gaussian_weights(X.astype(np.float64), mask, 5, 0.02, False)
    g0 = O.fusion_scale(X, mask, G[0], G[1], G[2])
    return X, mask, (G[0], G[1], G[2]), synth.log_grid(1e-2 * g0, 3.0 * g0, 5)


@pytest.mark.parametrize("precision", [0, 1])
def test_one_shard_is_the_unsharded_path(ccx, precision):
    X, mask, edges, gammas = _ragged()
    pr = ccx.Problem(X, mask, precision)
    pr.set_edges(*edges)
    U, L, stats, st = pr.solve_path(gammas)
    assert st == 0
    sh = _shards(ccx, X, mask, [0, X.shape[1]], edges, precision)
    Us, Ls, sst = ccx.solve_path_sharded(sh, gammas)
    for g in range(len(gammas)):
        assert np.array_equal(Us[0][g], U[g]), g
        assert np.array_equal(Ls[g], L[g]), g
        assert sst[g]["iters"] == stats[g]["iters"], g
    for s in sh + [pr]:
        s.close()


@pytest.mark.parametrize("precision,rtol", [(1, 1e-8), (0, 2e-5)])
def test_column_shards_agree_with_unsharded(ccx, precision, rtol):
    X, mask, edges, gammas = _ragged()
    pr = ccx.Problem(X, mask, precision)
    pr.set_edges(*edges)
    U, L, stats, st = pr.solve_path(gammas)
    for cuts in ([0, 18, 37], [0, 4, 21, 37]):          # slice-aligned and ragged splits
        sh = _shards(ccx, X, mask, cuts, edges, precision)
        Us, Ls, sst = ccx.solve_path_sharded(sh, gammas)
        for g in range(len(gammas)):
            Ug = np.concatenate([Us[k][g] for k in range(len(sh))], axis=1)
            err = np.linalg.norm(Ug.astype(np.float64) - U[g]) / np.linalg.norm(U[g])
            assert err <= rtol, (cuts, g, err)
            assert np.array_equal(Ls[g], L[g]), (cuts, g)
            assert sst[g]["converged"] in (1, 2)
        for s in sh:
            s.close()
    pr.close()


def test_shards_of_the_multislice_case_match_the_oracle(ccx):
    """The stored genotype-like case (n = 48, p = 2502, 5 % missing) in two column shards of 1252 and
    1250 columns: each shard still gives its CTAs two or more slices."""
    z = dict(np.load(os.path.join(GOLDEN, "genotype_n48_p2502.npz")))
    X, mask = z["X"], z["mask"]
    sh = _shards(ccx, X, mask, [0, 1252, X.shape[1]], (z["ei"], z["ej"], z["w"]), ccx.CCX_FP32)
    Us, Ls, sst = ccx.solve_path_sharded(sh, z["gammas"])
    for g in range(len(z["gammas"])):
        Ug = np.concatenate([Us[0][g], Us[1][g]], axis=1).astype(np.float64)
        ref = z["U"][g].astype(np.float64)
        assert np.linalg.norm(Ug - ref) / np.linalg.norm(ref) <= 1e-4, g
        if np.all(np.abs(z["margin"][g]) >= 1e-5):
            assert np.array_equal(Ls[g], z["labels"][g]), g
    for s in sh:
        s.close()


def test_shard_calls_validate(ccx):
    X, mask, edges, gammas = _ragged()
    pr = ccx.Problem(X, mask)
    pr.set_edges(*edges)
    import torch
    part = torch.empty(ccx.binding.shard_partials_len(pr.h), dtype=torch.float64, device="cuda")
    with pytest.raises(ccx.CcxError):                  # no gamma begun yet
        ccx.binding.shard_partials(pr.h, part)
    with pytest.raises(ccx.CcxError):
        ccx.binding.shard_begin_gamma(pr.h, -1.0, None, 1.0, 1.0)
    ccx.binding.shard_begin_gamma(pr.h, float(gammas[0]), None, *ccx.binding.shard_norms(pr.h))
    with pytest.raises(ccx.CcxError):                  # host memory is refused
        ccx.binding.shard_partials(pr.h, part.cpu())
    pr.close()
