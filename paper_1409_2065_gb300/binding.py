"""Thin Python binding of the ccx C ABI (include/ccx.h).

Argument marshalling only: every step of the solver runs in libccx.so.  The
functions keep the C names without the ``ccx_`` prefix.  Arrays may be numpy
arrays (host) or torch tensors (host or CUDA); outputs are allocated as numpy
arrays, or as CUDA torch tensors when ``device=True``.

Importing this module loads the compiled library and raises ImportError if
it has not been built (``__graft_entry__.build()`` or
``python paper_1409_2065_gb300/build.py``); there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libccx.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"ccx CUDA library not built ({LIB_PATH} missing); run __graft_entry__.build()")
_lib = C.CDLL(LIB_PATH)

CCX_FP32, CCX_FP64 = 0, 1
STATUS = {0: "CCX_OK", 1: "CCX_EINVAL", 2: "CCX_ENOMEM", 3: "CCX_ECUDA", 4: "CCX_ENOTCONV",
          5: "CCX_ETIMEOUT", 6: "CCX_ECANCELLED", 7: "CCX_EUNSUPPORTED"}


class KnnRule(C.Structure):
    _fields_ = [("k", C.c_int), ("phi", C.c_double), ("phi_auto", C.c_int), ("normalize", C.c_int),
                ("gram", C.c_int)]


class Opts(C.Structure):
    _fields_ = [("rho_scale", C.c_double), ("eps_rel", C.c_double), ("tol", C.c_double),
                ("max_iter", C.c_int), ("accelerate", C.c_int), ("chunk", C.c_int), ("extrapolate", C.c_int),
                ("stream_edges", C.c_int), ("slice_variant", C.c_int), ("max_ctas", C.c_int),
                ("fuse_delta", C.c_double), ("anderson", C.c_int)]


class GammaStats(C.Structure):
    _fields_ = [("iters", C.c_int), ("converged", C.c_int), ("n_fused", C.c_int), ("n_clusters", C.c_int),
                ("gamma", C.c_double), ("rho", C.c_double), ("eps", C.c_double), ("d_final", C.c_double),
                ("err_est", C.c_double), ("seconds", C.c_double), ("n_recomputed", C.c_int),
                ("recomputes", C.c_longlong), ("mixing_iters", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = C.c_void_p
_sigs = {
    "ccx_opts_default": (None, [C.POINTER(Opts)]),
    "ccx_problem_create": (C.c_int, [_P, _P, C.c_int64, C.c_int64, C.c_int64, C.c_int, _P, C.POINTER(_P)]),
    "ccx_set_edges": (C.c_int, [_P, C.c_int64, _P, _P, _P]),
    "ccx_standardize": (C.c_int, [_P]),
    "ccx_get_start": (C.c_int, [_P, _P]),
    "ccx_build_knn": (C.c_int, [_P, C.POINTER(KnnRule)]),
    "ccx_get_edges": (C.c_int, [_P, C.POINTER(C.c_int64), _P, _P, _P]),
    "ccx_min_connected_k": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int)]),
    "ccx_build_knn_composite": (C.c_int, [_P, C.POINTER(KnnRule), _P, C.c_double, C.c_int]),
    "ccx_principal_axes": (C.c_int, [_P, C.c_int, _P, _P]),
    "ccx_solve_path_projected": (C.c_int, [_P, _P, C.c_int, C.POINTER(Opts), C.c_int, _P, _P, _P]),
    "ccx_fusion_scale": (C.c_int, [_P, C.POINTER(C.c_double)]),
    "ccx_fusion_scale_noalloc": (C.c_int, [_P, C.POINTER(C.c_double)]),
    "ccx_solve_path": (C.c_int, [_P, _P, C.c_int, C.POINTER(Opts), _P, _P, _P]),
    "ccx_solve_path_fused": (C.c_int, [_P, _P, C.c_int, C.POINTER(Opts), _P, _P, _P, _P]),
    "ccx_solve_batch": (C.c_int, [_P, C.c_int, _P, _P, C.POINTER(Opts), _P, _P, _P, C.c_int, _P]),
    "ccx_server_create": (C.c_int, [C.POINTER(Opts), C.c_size_t, C.c_int, C.POINTER(_P)]),
    "ccx_submit": (C.c_int, [_P, _P, _P, C.c_int, _P, _P, _P, C.POINTER(C.c_uint64)]),
    "ccx_wait": (C.c_int, [_P, C.c_uint64, C.c_int64]),
    "ccx_server_destroy": (C.c_int, [_P]),
    "ccx_shard_norms": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "ccx_shard_begin_gamma": (C.c_int, [_P, C.c_double, C.POINTER(Opts), C.c_double, C.c_double]),
    "ccx_shard_partials": (C.c_int, [_P, _P, C.POINTER(C.c_int64)]),
    "ccx_shard_reduce": (C.c_int, [_P, _P, C.c_int, C.POINTER(C.c_int)]),
    "ccx_shard_end_gamma": (C.c_int, [_P, _P, _P, C.POINTER(GammaStats)]),
    "ccx_tune_grid": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "ccx_reset_path": (C.c_int, [_P]),
    "ccx_problem_destroy": (C.c_int, [_P]),
    "ccx_time_iterations": (C.c_int, [_P, C.c_double, C.c_int, C.POINTER(Opts), C.POINTER(C.c_double),
                                      C.POINTER(C.c_double)]),
    "ccx_time_iterations_mixing": (C.c_int, [_P, C.c_double, C.c_int, C.POINTER(Opts), C.POINTER(C.c_double),
                                             C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "ccx_kernel_launches": (C.c_uint64, []),
    "ccx_sweep_plan": (C.c_int, [C.c_int64, C.c_int64, _P, _P, C.c_int, _P, _P, _P, _P]),
    "ccx_last_error": (C.c_char_p, []),
    "ccx_version": (C.c_char_p, []),
}
for _name, (_res, _args) in _sigs.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

# every symbol the header declares, for the export check in the tests
EXPORTED = tuple(_sigs)


class CcxError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
        self.message = message


def last_error() -> str:
    return _lib.ccx_last_error().decode()


def version() -> str:
    return _lib.ccx_version().decode()


def _check(st: int, allow=(0,)) -> int:
    if st not in allow:
        raise CcxError(st, last_error())
    return st


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype):
    """(pointer, keepalive) for a numpy array or torch tensor of the given numpy dtype."""
    if x is None:
        return None, None
    if _is_torch(x):
        import torch
        tdt = {np.float32: torch.float32, np.uint8: torch.uint8, np.int32: torch.int32,
               np.float64: torch.float64}[dtype]
        if x.dtype != tdt or not x.is_contiguous():
            x = x.to(tdt).contiguous()
        return x.data_ptr(), x
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data, a


def opts_default() -> Opts:
    o = Opts()
    _lib.ccx_opts_default(C.byref(o))
    return o


def problem_create(X, mask=None, precision=CCX_FP32, stream=None):
    """Create a problem from X (n x p).  Returns an opaque handle (int)."""
    n, p = int(X.shape[0]), int(X.shape[1])
    xp, xk = _ptr(X, np.float32)
    mp, mk = _ptr(mask, np.uint8)
    h = _P()
    st = stream if stream is None or isinstance(stream, int) else stream.cuda_stream
    _check(_lib.ccx_problem_create(xp, mp, n, p, p, int(precision), st, C.byref(h)))
    del xk, mk
    return h.value


def standardize(h) -> None:
    """Standardise the problem's columns on their observed entries (ccx_standardize)."""
    _check(_lib.ccx_standardize(h))


def get_start(h, n: int, p: int):
    """Y_0 as the solver sees it (n x p float32)."""
    Y = np.empty((n, p), np.float32)
    _check(_lib.ccx_get_start(h, Y.ctypes.data))
    return Y


def problem_destroy(h) -> None:
    _check(_lib.ccx_problem_destroy(h))


def set_edges(h, ei, ej, w) -> None:
    ei = np.ascontiguousarray(ei, dtype=np.int32)
    ej = np.ascontiguousarray(ej, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.float64)
    _check(_lib.ccx_set_edges(h, ei.size, ei.ctypes.data, ej.ctypes.data, w.ctypes.data))


def build_knn(h, k: int, phi: float = 0.0, phi_auto: bool = False, normalize: bool = False, gram: int = 0) -> None:
    """kNN Gaussian-kernel weights; gram: 0 TF32 tensor cores, 1 BF16 tensor cores, 2 FP32 CUDA cores."""
    r = KnnRule(int(k), float(phi), int(bool(phi_auto)), int(bool(normalize)), int(gram))
    _check(_lib.ccx_build_knn(h, C.byref(r)))


def build_knn_composite(h, k: int, coords, alpha: float, phi: float = 0.0, phi_auto: bool = False,
                        normalize: bool = False, geodesic: bool = False) -> None:
    """kNN weights on alpha * genetic + (1 - alpha) * geographic distance; coords: n x 2 (lat, lon) degrees."""
    r = KnnRule(int(k), float(phi), int(bool(phi_auto)), int(bool(normalize)), 0)
    c = np.ascontiguousarray(coords, dtype=np.float64)
    _check(_lib.ccx_build_knn_composite(h, C.byref(r), c.ctypes.data, float(alpha), int(bool(geodesic))))


def principal_axes(h, q: int, p: int):
    """(axes q x p, variances q) of the column-centred Y_0."""
    axes = np.zeros((q, p), np.float64)
    var = np.zeros(q, np.float64)
    _check(_lib.ccx_principal_axes(h, int(q), axes.ctypes.data, var.ctypes.data))
    return axes, var


def solve_path_projected(h, gammas, n: int, q: int, opts: Opts | None = None, device: bool = False):
    """Path with each gamma's centroids projected on the q principal axes on the GPU.
    Returns (scores (G x n x q float32), labels (G x n int32), stats list, status)."""
    g = np.ascontiguousarray(gammas, dtype=np.float64)
    G = g.size
    if device:
        import torch
        S = torch.empty((G, n, q), dtype=torch.float32, device="cuda")
        L = torch.empty((G, n), dtype=torch.int32, device="cuda")
        sp, lp = S.data_ptr(), L.data_ptr()
    else:
        S = np.empty((G, n, q), np.float32)
        L = np.empty((G, n), np.int32)
        sp, lp = S.ctypes.data, L.ctypes.data
    stats = (GammaStats * max(G, 1))()
    o = C.byref(opts) if opts is not None else None
    st = _check(_lib.ccx_solve_path_projected(h, g.ctypes.data, G, o, int(q), sp, lp, stats), allow=(0, 4))
    return S, L, [stats[k].as_dict() for k in range(G)], st


def min_connected_k(h, k_max: int) -> int:
    """Smallest k <= k_max whose kNN union graph is connected (0 if none)."""
    k = C.c_int(0)
    _check(_lib.ccx_min_connected_k(h, int(k_max), C.byref(k)))
    return k.value


def get_edges(h):
    m = C.c_int64(0)
    _check(_lib.ccx_get_edges(h, C.byref(m), None, None, None))
    ei = np.zeros(m.value, np.int32)
    ej = np.zeros(m.value, np.int32)
    w = np.zeros(m.value, np.float64)
    _check(_lib.ccx_get_edges(h, C.byref(m), ei.ctypes.data, ej.ctypes.data, w.ctypes.data))
    return ei, ej, w


def fusion_scale(h) -> float:
    g = C.c_double(0.0)
    _check(_lib.ccx_fusion_scale(h, C.byref(g)))
    return g.value


def fusion_scale_noalloc(h) -> float:
    """ccx_fusion_scale through the library's fixed buffers: no memory is allocated."""
    g = C.c_double(0.0)
    _check(_lib.ccx_fusion_scale_noalloc(h, C.byref(g)))
    return g.value


def solve_path(h, gammas, n: int, p: int, opts: Opts | None = None, want_U: bool = True,
               want_labels: bool = True, device: bool = False, U_out=None, labels_out=None, fused_out=None):
    """Solve the warm-started path.  Returns (U (G x n x p float32), labels (G x n int32), stats list, status).

    With device=True the outputs are CUDA torch tensors written directly by the
    library; otherwise numpy arrays.  Preallocated outputs may be passed;
    fused_out (G x n_edges uint8, numpy or torch) also receives each gamma's
    fused flags (ccx_solve_path_fused).
    """
    g = np.ascontiguousarray(gammas, dtype=np.float64)
    G = g.size
    if device:
        import torch
        if want_U and U_out is None:
            U_out = torch.empty((G, n, p), dtype=torch.float32, device="cuda")
        if want_labels and labels_out is None:
            labels_out = torch.empty((G, n), dtype=torch.int32, device="cuda")
    else:
        if want_U and U_out is None:
            U_out = np.empty((G, n, p), np.float32)
        if want_labels and labels_out is None:
            labels_out = np.empty((G, n), np.int32)
    up, _ = _ptr(U_out, np.float32) if U_out is not None else (None, None)
    lp, _ = _ptr(labels_out, np.int32) if labels_out is not None else (None, None)
    stats = (GammaStats * max(G, 1))()
    o = C.byref(opts) if opts is not None else None
    if fused_out is not None:
        fp, _fk = _ptr(fused_out, np.uint8)
        if not _is_torch(fused_out) and fp != fused_out.ctypes.data:
            raise ValueError("fused_out must be a contiguous uint8 array")
        st = _check(_lib.ccx_solve_path_fused(h, g.ctypes.data, G, o, up, lp, fp, stats), allow=(0, 4))
    else:
        st = _check(_lib.ccx_solve_path(h, g.ctypes.data, G, o, up, lp, stats), allow=(0, 4))
    return U_out, labels_out, [stats[k].as_dict() for k in range(G)], st


def solve_batch(problems, gammas_list, opts: Opts | None = None, want_U: bool = True, want_labels: bool = True,
                device: bool = False, max_active: int = 0):
    """Solve several problems' paths together (ccx_solve_batch).

    problems: list of Problem; gammas_list: one gamma sequence per problem.  Returns
    (U list, labels list, stats lists, per-problem status list, overall status).
    """
    k = len(problems)
    gs = [np.ascontiguousarray(g, dtype=np.float64) for g in gammas_list]
    if len(gs) != k:
        raise ValueError("one gamma sequence per problem")
    Us, Ls = [], []
    stats = [(GammaStats * max(g.size, 1))() for g in gs]
    for pb, g in zip(problems, gs):
        U = L = None
        if device:
            import torch
            if want_U:
                U = torch.empty((g.size, pb.n, pb.p), dtype=torch.float32, device="cuda")
            if want_labels:
                L = torch.empty((g.size, pb.n), dtype=torch.int32, device="cuda")
        else:
            if want_U:
                U = np.empty((g.size, pb.n, pb.p), np.float32)
            if want_labels:
                L = np.empty((g.size, pb.n), np.int32)
        Us.append(U)
        Ls.append(L)
    ptr = lambda x: 0 if x is None else (x.data_ptr() if _is_torch(x) else x.ctypes.data)
    handles = (_P * k)(*[pb.h for pb in problems])
    gptr = (_P * k)(*[g.ctypes.data for g in gs])
    ng = (C.c_int * k)(*[g.size for g in gs])
    uptr = (_P * k)(*[ptr(u) for u in Us]) if want_U else None
    lptr = (_P * k)(*[ptr(l) for l in Ls]) if want_labels else None
    sptr = (_P * k)(*[C.addressof(st) for st in stats])
    status = (C.c_int * k)()
    o = C.byref(opts) if opts is not None else None
    st = _check(_lib.ccx_solve_batch(handles, k, gptr, ng, o, uptr, lptr, sptr, int(max_active), status),
                allow=(0, 4))
    return Us, Ls, [[s_[j].as_dict() for j in range(g.size)] for s_, g in zip(stats, gs)], list(status), st


class Server:
    """Background scheduler of path solves (ccx_server_*).  submit() returns a ticket;
    wait(ticket) returns (status, U, labels, stats) once the job is done."""

    def __init__(self, opts: Opts | None = None, hbm_budget: int = 0, max_active: int = 0):
        h = _P()
        o = C.byref(opts) if opts is not None else None
        _check(_lib.ccx_server_create(o, int(hbm_budget), int(max_active), C.byref(h)))
        self.h = h.value
        self._jobs = {}

    def submit(self, problem, gammas, device: bool = False):
        g = np.ascontiguousarray(gammas, dtype=np.float64)
        G = g.size
        if device:
            import torch
            U = torch.empty((G, problem.n, problem.p), dtype=torch.float32, device="cuda")
            L = torch.empty((G, problem.n), dtype=torch.int32, device="cuda")
            up, lp = U.data_ptr(), L.data_ptr()
        else:
            U = np.empty((G, problem.n, problem.p), np.float32)
            L = np.empty((G, problem.n), np.int32)
            up, lp = U.ctypes.data, L.ctypes.data
        stats = (GammaStats * max(G, 1))()
        t = C.c_uint64(0)
        _check(_lib.ccx_submit(self.h, problem.h, g.ctypes.data, G, up, lp, stats, C.byref(t)))
        self._jobs[t.value] = (g, U, L, stats, problem)
        return t.value

    def wait(self, ticket, timeout_ms: int = -1):
        st = _lib.ccx_wait(self.h, int(ticket), int(timeout_ms))
        if st == 5:
            return st, None, None, None
        if st not in (0, 4):
            self._jobs.pop(ticket, None)
            raise CcxError(st, last_error())
        g, U, L, stats, _ = self._jobs.pop(ticket)
        return st, U, L, [stats[k].as_dict() for k in range(g.size)]

    def close(self):
        if self.h:
            _check(_lib.ccx_server_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------- feature shards
def shard_norms(h):
    """(||Y_c||_F^2, ||Y_0||_F^2) of this column shard."""
    a, b = C.c_double(0.0), C.c_double(0.0)
    _check(_lib.ccx_shard_norms(h, C.byref(a), C.byref(b)))
    return a.value, b.value


def shard_begin_gamma(h, gamma: float, opts: Opts | None, yc_sq_total: float, y0_sq_total: float) -> None:
    o = C.byref(opts) if opts is not None else None
    _check(_lib.ccx_shard_begin_gamma(h, float(gamma), o, float(yc_sq_total), float(y0_sq_total)))


def shard_partials_len(h) -> int:
    n = C.c_int64(0)
    _check(_lib.ccx_shard_partials(h, None, C.byref(n)))
    return int(n.value)


def shard_partials(h, part) -> None:
    """One iteration's column work; its partial sums into `part` (CUDA float64 tensor)."""
    n = C.c_int64(part.numel())
    _check(_lib.ccx_shard_partials(h, part.data_ptr(), C.byref(n)))


def shard_reduce(h, parts, want_done: bool = True):
    """The iteration's reduction over `parts` (CUDA float64 tensor, n_shards x len, shard order)."""
    d = C.c_int(0)
    _check(_lib.ccx_shard_reduce(h, parts.data_ptr(), int(parts.shape[0]), C.byref(d) if want_done else None))
    return bool(d.value) if want_done else None


def shard_end_gamma(h, n: int, p: int):
    U = np.empty((n, p), np.float32)
    L = np.empty(n, np.int32)
    st = GammaStats()
    _check(_lib.ccx_shard_end_gamma(h, U.ctypes.data, L.ctypes.data, C.byref(st)))
    return U, L, st.as_dict()


def allgather_parts(part, group=None):
    """Exchange of the feature-sharded iteration across ranks (one shard per rank):
    every rank's partial vector, stacked in rank order (an all-gather; the sum in
    that fixed order happens inside ccx_shard_reduce)."""
    import torch
    import torch.distributed as dist
    ws = dist.get_world_size(group)
    bufs = [torch.empty_like(part) for _ in range(ws)]
    dist.all_gather(bufs, part, group=group)
    return torch.stack(bufs)


def ordered_sum(values, group=None):
    """Sum of one float per rank in rank order, identical on every rank."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in np.atleast_1d(values)], dtype=torch.float64)
    ws = dist.get_world_size(group)
    bufs = [torch.empty_like(t) for _ in range(ws)]
    dist.all_gather(bufs, t, group=group)
    out = torch.zeros_like(t)
    for b in bufs:
        out += b
    return out.numpy()


def solve_path_sharded(shards, gammas, opts: Opts | None = None, exchange=None, check_every: int = 16,
                       norms=None):
    """Warm-started path of one problem split by columns into `shards` (Problems on
    column blocks with the same edge set), driven iteration by iteration through
    the ccx_shard_* calls.  exchange(list of local partial tensors) returns the
    n_shards x len tensor in shard order (default: all shards in this process,
    stacked); norms: the whole problem's (||Y_c||^2, ||Y_0||^2) (default: the sum
    over `shards`).  Returns ([U of each shard per gamma], labels per gamma, stats
    of the first shard per gamma)."""
    import torch
    if norms is None:
        nn = [shard_norms(s.h) for s in shards]
        norms = (sum(a for a, _ in nn), sum(b for _, b in nn))
    L = shard_partials_len(shards[0].h)
    parts = [torch.empty(L, dtype=torch.float64, device="cuda") for _ in shards]
    if exchange is None:
        exchange = torch.stack
    Us, labels, stats = [[] for _ in shards], [], []
    for g in np.asarray(gammas, dtype=np.float64):
        for s in shards:
            shard_begin_gamma(s.h, g, opts, norms[0], norms[1])
        it = 0
        while True:
            for s, part in zip(shards, parts):
                shard_partials(s.h, part)
            allp = exchange(parts)
            it += 1
            check = it % check_every == 0
            done = [shard_reduce(s.h, allp, want_done=check) for s in shards]
            if check and all(done):
                break
        for k, s in enumerate(shards):
            U, lab, st = shard_end_gamma(s.h, s.n, s.p)
            Us[k].append(U)
            if k == 0:
                labels.append(lab)
                stats.append(st)
    return Us, labels, stats


def reset_path(h) -> None:
    _check(_lib.ccx_reset_path(h))


def tune_grid(h, g_min: int = 1):
    """(grid, ms per iteration) chosen by ccx_tune_grid for this problem."""
    g, ms = C.c_int(0), C.c_double(0.0)
    _check(_lib.ccx_tune_grid(h, int(g_min), C.byref(g), C.byref(ms)))
    return g.value, ms.value


def time_iterations(h, gamma: float, n_iter: int, opts: Opts | None = None):
    """(mean ms of the fused iteration kernel, mean ms of the reduction kernel) over n_iter iterations."""
    a, b = C.c_double(0.0), C.c_double(0.0)
    o = C.byref(opts) if opts is not None else None
    _check(_lib.ccx_time_iterations(h, float(gamma), int(n_iter), o, C.byref(a), C.byref(b)))
    return a.value, b.value


def time_iterations_mixing(h, gamma: float, n_iter: int, opts: Opts):
    """(mean ms of the iteration kernel, of the reduction kernel, of the two Anderson mixing kernels)
    over n_iter iterations with mixing history opts.anderson."""
    a, b, c = C.c_double(0.0), C.c_double(0.0), C.c_double(0.0)
    _check(_lib.ccx_time_iterations_mixing(h, float(gamma), int(n_iter), C.byref(opts), C.byref(a), C.byref(b),
                                           C.byref(c)))
    return a.value, b.value, c.value


def sweep_plan(n: int, ei, ej, precision=CCX_FP32):
    """Work layout of the iteration kernel (host only): (T, la, le, nslots, node_row, node_nbr, edge_id),
    the arrays indexed by position k * T + t (-1 past the end of a run)."""
    ei = np.ascontiguousarray(ei, dtype=np.int32)
    ej = np.ascontiguousarray(ej, dtype=np.int32)
    sz = np.zeros(4, np.int32)
    _check(_lib.ccx_sweep_plan(int(n), ei.size, ei.ctypes.data, ej.ctypes.data, int(precision), sz.ctypes.data,
                               None, None, None))
    T, la, le, ns = (int(v) for v in sz)
    row = np.empty(la * T, np.int32)
    nbr = np.empty(la * T, np.int32)
    eid = np.empty(le * T, np.int32)
    _check(_lib.ccx_sweep_plan(int(n), ei.size, ei.ctypes.data, ej.ctypes.data, int(precision), sz.ctypes.data,
                               row.ctypes.data, nbr.ctypes.data, eid.ctypes.data))
    return T, la, le, ns, row, nbr, eid


def kernel_launches() -> int:
    return int(_lib.ccx_kernel_launches())


class Problem:
    """Owning wrapper around a problem handle."""

    def __init__(self, X, mask=None, precision=CCX_FP32, stream=None, standardize=False):
        self.n, self.p = int(X.shape[0]), int(X.shape[1])
        self.h = problem_create(X, mask, precision, stream)
        if standardize:
            globals()["standardize"](self.h)

    def get_start(self):
        return get_start(self.h, self.n, self.p)

    def set_edges(self, ei, ej, w):
        set_edges(self.h, ei, ej, w)

    def build_knn(self, k, phi=0.0, phi_auto=False, normalize=False, gram=0):
        build_knn(self.h, k, phi, phi_auto, normalize, gram)

    def get_edges(self):
        return get_edges(self.h)

    def min_connected_k(self, k_max):
        return min_connected_k(self.h, k_max)

    def principal_axes(self, q):
        return principal_axes(self.h, q, self.p)

    def solve_path_projected(self, gammas, q, opts=None, device=False):
        return solve_path_projected(self.h, gammas, self.n, q, opts, device)

    def build_knn_composite(self, k, coords, alpha, phi=0.0, phi_auto=False, normalize=False, geodesic=False):
        build_knn_composite(self.h, k, coords, alpha, phi, phi_auto, normalize, geodesic)

    def fusion_scale(self):
        return fusion_scale(self.h)

    def solve_path(self, gammas, opts=None, **kw):
        return solve_path(self.h, gammas, self.n, self.p, opts, **kw)

    def reset_path(self):
        reset_path(self.h)

    def tune_grid(self, g_min=1):
        return tune_grid(self.h, g_min)

    def time_iterations(self, gamma, n_iter, opts=None):
        return time_iterations(self.h, gamma, n_iter, opts)

    def time_iterations_mixing(self, gamma, n_iter, opts):
        return time_iterations_mixing(self.h, gamma, n_iter, opts)

    def close(self):
        if self.h:
            problem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
