"""Serving (ccx_server_*) through the C ABI on the GPU.

Jobs arrive while others run; every result must equal solving the same problem
alone, waits never block past their limit, and shutdown cancels jobs that have
not started.
"""
import threading
import time

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


def _jobs(ccx, count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n, p = int(rng.integers(30, 200)), int(rng.integers(3, 80))
        X, _ = synth.gaussian_mixture(n, p, int(rng.integers(2, 6)), seed=seed * 100 + i)
        mask = synth.random_mask(rng, n, p, 0.05) if i % 4 == 3 else None
        out.append((X, mask, int(rng.integers(4, 8)), int(rng.integers(2, 5))))
    return out


def _problem(ccx, job):
    X, mask, k, _ = job
    pr = ccx.Problem(X, mask)
    pr.build_knn(k, phi_auto=True, normalize=True)
    return pr


def _alone(ccx, jobs):
    ref = []
    for job in jobs:
        pr = _problem(ccx, job)
        g0 = pr.fusion_scale()
        gam = synth.log_grid(0.05 * g0, 2.0 * g0, job[3])
        U, L, _, _ = pr.solve_path(gam)
        ref.append((gam, U, L))
        pr.close()
    return ref


def test_poisson_mix_equals_alone(ccx):
    jobs = _jobs(ccx, 10, 7)
    ref = _alone(ccx, jobs)
    probs = [_problem(ccx, j) for j in jobs]
    srv = ccx.Server(max_active=4)
    rng = np.random.default_rng(8)
    tickets = [None] * len(jobs)

    def arrivals():
        for i in range(len(jobs)):
            time.sleep(float(rng.exponential(0.01)))
            tickets[i] = srv.submit(probs[i], ref[i][0])

    th = threading.Thread(target=arrivals)
    th.start()
    th.join()
    for i, t in enumerate(tickets):
        st, U, L, stats = srv.wait(t, 120000)
        assert st == 0, (i, st)
        assert np.array_equal(U, ref[i][1]), i
        assert np.array_equal(L, ref[i][2]), i
    srv.close()
    for pr in probs:
        pr.close()


def test_wait_times_out_without_blocking(ccx):
    X, _ = synth.gaussian_mixture(400, 64, 4, seed=5)
    pr = ccx.Problem(X)
    pr.build_knn(10, phi_auto=True, normalize=True)
    g0 = pr.fusion_scale()
    srv = ccx.Server()
    t = srv.submit(pr, synth.log_grid(0.05 * g0, 2.0 * g0, 6))
    t0 = time.perf_counter()
    st = srv.wait(t, 0)[0]
    assert time.perf_counter() - t0 < 0.5
    if st == 5:                                  # still running: a later wait returns the result
        st = srv.wait(t, -1)[0]
    assert st == 0
    with pytest.raises(ccx.CcxError):            # the ticket was released by the wait that returned it
        srv.wait(t, 0)
    srv.close()
    pr.close()


def test_small_memory_budget_runs_one_at_a_time(ccx):
    jobs = _jobs(ccx, 4, 9)
    ref = _alone(ccx, jobs)
    probs = [_problem(ccx, j) for j in jobs]
    srv = ccx.Server(hbm_budget=1)               # only the first job may hold memory: one after another
    ts = [srv.submit(pr, r[0]) for pr, r in zip(probs, ref)]
    for i, t in enumerate(ts):
        st, U, L, _ = srv.wait(t, -1)
        assert st == 0, (i, st)
        assert np.array_equal(U, ref[i][1]) and np.array_equal(L, ref[i][2])
    srv.close()
    for pr in probs:
        pr.close()


def test_shutdown_cancels_queued_jobs(ccx):
    jobs = _jobs(ccx, 6, 13)
    probs = [_problem(ccx, j) for j in jobs]
    srv = ccx.Server(hbm_budget=1, max_active=1)
    ts = [srv.submit(pr, [0.1, 1.0, 10.0]) for pr in probs]
    first = srv.wait(ts[0], -1)[0]
    assert first == 0
    # the rest run one at a time; a queued job can be waited for with a limit, and
    # destroying the server ends the jobs that have not started with CCX_ECANCELLED
    statuses = [srv.wait(t, 0)[0] for t in ts[1:]]
    assert all(s in (0, 5) for s in statuses)
    srv.close()
    for pr in probs:
        pr.close()
