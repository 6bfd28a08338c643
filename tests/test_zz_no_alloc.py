"""ccx_fusion_scale_noalloc: the gamma scale computed in the library's fixed
buffers, for callers that cannot allocate memory when they need it (a service
whose device memory is all held by its own pool, or a loop that must not pay
for cudaFree's device-wide synchronisation).

The call must return what ccx_fusion_scale returns, call after call, though
every call reuses the same buffers; an edge set above its fixed limit must be
refused with an error and no GPU work.  This file is collected last so that
it also runs after everything else the test session loaded onto the GPU.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

REL = 1e-12   # both calls compute the same ratios in double; only the selection differs


def _ccx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import paper_1409_2065_gb300 as ccx
    return torch, ccx


@pytest.mark.parametrize("n_points,k", [(300, 8), (257, 5)])   # 1809 and 1004 kNN edges: odd and even
def test_noalloc_matches_fusion_scale_twice(n_points, k):
    torch, ccx = _ccx()
    X, _ = synth.gaussian_mixture(n_points, 24, 4, seed=11)
    mask = synth.random_mask(np.random.default_rng(12), n_points, 24, 0.05)
    pr = ccx.Problem(X, mask)
    pr.build_knn(k, phi=0.3)
    ref = pr.fusion_scale()
    first = ccx.fusion_scale_noalloc(pr.h)
    second = ccx.fusion_scale_noalloc(pr.h)
    assert first == pytest.approx(ref, rel=REL)
    assert second == pytest.approx(ref, rel=REL)
    # a second problem in between: the shared buffers keep its ratios, which
    # the next call on the first problem must overwrite
    Xb, _ = synth.gaussian_mixture(100, 7, 2, seed=13)
    pb = ccx.Problem(Xb)
    pb.build_knn(4, phi=1.0)
    assert ccx.fusion_scale_noalloc(pb.h) == pytest.approx(pb.fusion_scale(), rel=REL)
    assert ccx.fusion_scale_noalloc(pr.h) == pytest.approx(ref, rel=REL)
    pb.close()
    pr.close()


def test_noalloc_takes_no_device_memory():
    torch, ccx = _ccx()
    X, _ = synth.gaussian_mixture(200, 16, 3, seed=21)
    pr = ccx.Problem(X)
    pr.build_knn(6, phi=0.5)
    ref = pr.fusion_scale()
    ccx.fusion_scale_noalloc(pr.h)        # the first call may do the per-device set-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    vals = [ccx.fusion_scale_noalloc(pr.h) for _ in range(3)]
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    for v in vals:
        assert v == pytest.approx(ref, rel=REL)
    pr.close()


def test_noalloc_refuses_edge_sets_above_its_limit():
    torch, ccx = _ccx()
    n = 1450                                   # complete graph: 1,050,525 edges > 2^20
    rng = np.random.default_rng(31)
    X = rng.standard_normal((n, 2)).astype(np.float32)
    ei, ej = np.triu_indices(n, 1)
    assert ei.size > (1 << 20)
    pr = ccx.Problem(X)
    pr.set_edges(ei.astype(np.int32), ej.astype(np.int32), np.ones(ei.size))
    launches = ccx.kernel_launches()
    with pytest.raises(ccx.CcxError) as exc:
        ccx.fusion_scale_noalloc(pr.h)
    assert exc.value.status == 1
    assert "at most 1048576 edges" in exc.value.message
    assert ccx.kernel_launches() == launches
    pr.close()
