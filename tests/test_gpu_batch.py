"""Batched solves (ccx_solve_batch) through the C ABI on the GPU.

Several independent problems of different shapes run together, each on its own
stream; every result must be bit-identical to solving that problem alone.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ccx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_1409_2065_gb300 as ccx
    return ccx


def _problem_set(n_probs, seed):
    """Mixed sizes, with and without missing data; kNN weights built on the GPU."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_probs):
        n = int(rng.integers(30, 260))
        p = int(rng.integers(3, 120))
        X, _ = synth.gaussian_mixture(n, p, int(rng.integers(2, 6)), seed=seed * 100 + i)
        mask = synth.random_mask(rng, n, p, 0.05) if i % 3 == 1 else None
        k = int(rng.integers(4, 9))
        out.append((X, mask, k, int(rng.integers(3, 7))))
    return out


def _build(ccx, spec, precision):
    X, mask, k, _ = spec
    pr = ccx.Problem(X, mask, precision)
    pr.build_knn(k, phi_auto=True, normalize=True)
    return pr


def _grid(pr, count):
    g0 = pr.fusion_scale()
    return synth.log_grid(0.05 * g0, 2.0 * g0, count)


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_alone(ccx, precision):
    specs = _problem_set(7, 5 + precision)
    alone = []
    for sp in specs:
        pr = _build(ccx, sp, precision)
        gam = _grid(pr, sp[3])
        U, L, stats, st = pr.solve_path(gam)
        alone.append((gam, U, L, [s["iters"] for s in stats]))
        pr.close()
    probs = [_build(ccx, sp, precision) for sp in specs]
    Us, Ls, stats, status, st = ccx.solve_batch(probs, [a[0] for a in alone], max_active=4)
    assert st == 0 and all(s == 0 for s in status), (st, status)
    for i, a in enumerate(alone):
        assert np.array_equal(Us[i], a[1]), i
        assert np.array_equal(Ls[i], a[2]), i
        assert [s["iters"] for s in stats[i]] == a[3], i
    for pr in probs:
        pr.close()


def test_batch_device_outputs_and_reuse(ccx):
    """Device outputs equal host outputs; a second batch continues each path from its last gamma."""
    specs = _problem_set(4, 11)
    probs = [_build(ccx, sp, 0) for sp in specs]
    grids = [_grid(pr, 3) for pr in probs]
    Uh, Lh, _, _, _ = ccx.solve_batch(probs, grids)
    for pr in probs:
        pr.reset_path()
    Ud, Ld, _, _, _ = ccx.solve_batch(probs, grids, device=True, max_active=2)
    for i in range(len(probs)):
        assert np.array_equal(Ud[i].cpu().numpy(), Uh[i])
        assert np.array_equal(Ld[i].cpu().numpy(), Lh[i])
    # continuing: the next call starts from the last iterate of the previous one
    Uc, _, stc, _, _ = ccx.solve_batch(probs, [g[-1:] for g in grids])
    for i in range(len(probs)):
        assert np.linalg.norm(Uc[i][0] - Uh[i][-1]) <= 1e-4 * np.linalg.norm(Uh[i][-1])
    for pr in probs:
        pr.close()


def test_batch_reports_errors_per_problem(ccx):
    """A problem the iteration kernel cannot take (n > 65535) fails alone; the others finish and
    their results equal solving them alone."""
    specs = _problem_set(3, 21)
    probs = [_build(ccx, sp, 0) for sp in specs]
    grids = [_grid(pr, 2) for pr in probs]
    ref = []
    for sp, g in zip(specs, grids):
        q = _build(ccx, sp, 0)
        ref.append(q.solve_path(g)[0])
        q.close()
    bad = ccx.Problem(np.zeros((70000, 1), np.float32))
    with pytest.raises(ccx.CcxError) as e:
        ccx.solve_batch(probs + [bad], grids + [[1.0]])
    assert e.value.status == 7 and "problem 3" in e.value.message
    for pr in probs:
        pr.reset_path()
    Us, _, _, status, _ = ccx.solve_batch(probs, grids)
    for i in range(len(probs)):
        assert np.array_equal(Us[i], ref[i])
    for pr in probs + [bad]:
        pr.close()


def test_tuned_grids_batch_equals_alone(ccx):
    """ccx_tune_grid picks a grid per problem (from timing); a batch of tuned problems gives, for each,
    exactly the result of solving it alone with the same grid, and agrees with the default grid within
    the FP32 parity bar (1e-4 relative, the grid changes only the rounding of partial sums)."""
    specs = _problem_set(6, 17)
    probs, grids, tuned = [], [], []
    for sp in specs:
        pr = _build(ccx, sp, 0)
        g, ms = pr.tune_grid(1)
        assert g >= 1 and ms > 0.0
        tuned.append(g)
        probs.append(pr)
        grids.append(_grid(pr, sp[3]))
    Us, Ls, stats, status, st = ccx.solve_batch(probs, grids, max_active=6)
    assert st == 0 and all(s == 0 for s in status), status
    for i, sp in enumerate(specs):
        alone = _build(ccx, sp, 0)
        o = ccx.opts_default()
        o.max_ctas = tuned[i]
        U, L, _, s1 = alone.solve_path(grids[i], o)
        assert s1 == 0
        assert np.array_equal(Us[i], U) and np.array_equal(Ls[i], L), i
        alone.reset_path()
        U0, L0, _, s0 = alone.solve_path(grids[i])
        assert s0 == 0
        for g in range(len(grids[i])):
            assert np.linalg.norm(U0[g] - U[g]) <= 1e-4 * np.linalg.norm(U0[g]), (i, g)
        alone.close()
    for pr in probs:
        pr.close()
    with pytest.raises(ccx.CcxError):          # tuning needs a fresh path
        pr2 = _build(ccx, specs[0], 0)
        pr2.solve_path([0.1])
        pr2.tune_grid(1)


def test_grid_changes_between_solves_rebuild_the_iteration_graph(ccx):
    """A solve on a smaller grid reallocates the per-CTA partial buffers; the next solve on the first
    grid must not reuse the iteration graph captured before (it holds the old buffers).  Same problem,
    default grid -> 8 CTAs -> default grid (and tuning in between): the last result equals the first."""
    sp = _problem_set(1, 23)[0]
    pr = _build(ccx, sp, 0)
    gam = _grid(pr, 3)
    U1, L1, _, s1 = pr.solve_path(gam)
    o = ccx.opts_default()
    o.max_ctas = 8
    pr.reset_path()
    U2, _, _, s2 = pr.solve_path(gam, o)
    pr.reset_path()
    U3, L3, _, s3 = pr.solve_path(gam)
    assert s1 == s2 == s3 == 0
    assert np.array_equal(U1, U3) and np.array_equal(L1, L3)
    pr.reset_path()
    g, _ = pr.tune_grid(1)
    U4, L4, _, s4 = pr.solve_path(gam)
    fresh = _build(ccx, sp, 0)
    o.max_ctas = g
    U5, L5, _, s5 = fresh.solve_path(gam, o)
    assert s4 == s5 == 0 and np.array_equal(U4, U5) and np.array_equal(L4, L5)
    pr.close()
    fresh.close()
