"""The iteration kernel's work layout, checked on the CPU (the layout is host
code in the library; these checks need no GPU).

Every index the kernel follows comes from this plan, so its invariants are
checked directly: each CSR entry (both directions of every edge) sits at
exactly one node-sweep position; run t holds the consecutive entries
[t la, (t + 1) la) with each row contiguous and rows in order; the edge sweep
covers every edge once with runs of consecutive edge ids; and the order
inside rows lowers the shared-memory bank conflicts of the neighbour gathers.
"""
import numpy as np
import pytest

import synth

ccx = pytest.importorskip("paper_1409_2065_gb300")


def _graph(n, p, k, seed):
    import oracle as O
    X, _ = synth.gaussian_mixture(n, p, 4, seed=seed)
    ei, ej, w, _, _ = O.knn_gaussian_weights(X.astype(np.float64), None, k, 0.0, False)
    return ei.astype(np.int32), ej.astype(np.int32)


def _wavefronts(nbr, T, L, groups):
    """Shared-memory wavefronts of 16-byte gathers: per step and eight-lane phase, the largest
    number of lanes whose rows fall in the same bank group (node mod groups)."""
    tot = 0
    A = nbr.reshape(L, T)
    for k in range(L):
        for g in range(0, T, 8):
            v = A[k, g:g + 8]
            v = v[v >= 0]
            if v.size:
                tot += np.bincount(v % groups, minlength=groups).max()
    return tot


@pytest.mark.parametrize("n,p,k,seed", [(300, 6, 8, 1), (1000, 20, 10, 2), (57, 3, 5, 3)])
def test_sweep_plan_invariants(n, p, k, seed):
    ei, ej = _graph(n, p, k, seed)
    m = ei.size
    T, la, le, ns, row, nbr, eid = ccx.sweep_plan(n, ei, ej)
    assert la * T >= 2 * m and le * T >= m and la == max(1, -(-2 * m // T)) and le == max(1, -(-m // T))
    # node sweep: every directed edge exactly once
    pos = np.nonzero(row >= 0)[0]
    got = sorted(zip(row[pos].tolist(), nbr[pos].tolist()))
    want = sorted(list(zip(ei.tolist(), ej.tolist())) + list(zip(ej.tolist(), ei.tolist())))
    assert got == want
    # run t: entries [t la, (t+1) la) of the row-major CSR, rows contiguous and increasing
    R = row.reshape(la, T)
    starts = np.r_[0, np.cumsum(np.bincount(np.r_[ei, ej], minlength=n))]
    slots = 0
    for t in range(T):
        r = R[:, t]
        r = r[r >= 0]
        q0 = t * la
        assert r.size == max(0, min(la, 2 * m - q0))
        if r.size:
            assert np.all(np.diff(r) >= 0)
            # the rows a run covers are exactly those of CSR entries q0 .. q0 + size - 1
            rows_of_q = np.searchsorted(starts, np.arange(q0, q0 + r.size), side="right") - 1
            assert np.array_equal(r, rows_of_q)
            slots += 1 + int(np.count_nonzero(np.diff(r)))
    assert slots == ns
    # edge sweep: every edge once; run t holds edges [t le, (t+1) le) in some order, grouped by ei
    E = eid.reshape(le, T)
    assert sorted(eid[eid >= 0].tolist()) == list(range(m))
    for t in range(T):
        e = E[:, t]
        e = e[e >= 0]
        assert sorted(e.tolist()) == list(range(t * le, min((t + 1) * le, m)))
        assert np.all(np.diff(ei[e]) >= 0)


def test_sweep_plan_lowers_bank_conflicts():
    ei, ej = _graph(1000, 20, 10, 2)
    T, la, le, ns, row, nbr, eid = ccx.sweep_plan(1000, ei, ej)
    # natural order: the same runs without the reordering inside rows
    m = ei.size
    order = np.lexsort((np.r_[ej, ei], np.r_[ei, ej]))
    csr_nbr = np.r_[ej, ei][order]
    natural = np.full(la * T, -1, np.int64)
    q = np.arange(2 * m)
    natural[(q % la) * T + q // la] = csr_nbr
    before, after = _wavefronts(natural, T, la, 8), _wavefronts(nbr, T, la, 8)
    assert after < 0.75 * before


def test_sweep_plan_rejects_bad_edges():
    with pytest.raises(ccx.CcxError):
        ccx.sweep_plan(10, [3, 1], [4, 2])           # not sorted
    with pytest.raises(ccx.CcxError):
        ccx.sweep_plan(10, [2], [2])                 # self loop
    with pytest.raises(ccx.CcxError):
        ccx.sweep_plan(10, [0], [10])                # out of range
