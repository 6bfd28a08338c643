"""The C-ABI library loads and exports every function include/ccx.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ccx.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ccx_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ccx_problem_create", "ccx_set_edges", "ccx_build_knn", "ccx_get_edges", "ccx_solve_path",
                     "ccx_problem_destroy", "ccx_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import paper_1409_2065_gb300 as ccx
    lib = ctypes.CDLL(ccx.binding.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in ccx.binding.EXPORTED, name


def test_defaults_and_version():
    import paper_1409_2065_gb300 as ccx
    o = ccx.opts_default()
    assert (o.rho_scale, o.eps_rel, o.tol, o.max_iter, o.accelerate, o.chunk, o.extrapolate, o.stream_edges,
            o.slice_variant, o.max_ctas, o.fuse_delta, o.anderson) == (2.0, 1e-3, 1e-6, 200000, 1, 64, 1, 0, 0, 0,
                                                                       1e-5, 0)
    assert "sm_103a" in ccx.version()


def test_no_silent_cpu_path():
    """Without a GPU the library reports a CUDA error instead of computing anything."""
    import numpy as np
    import torch
    import paper_1409_2065_gb300 as ccx
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(ccx.CcxError) as ei:
        ccx.problem_create(np.zeros((4, 3), np.float32))
    assert ei.value.status == 3
