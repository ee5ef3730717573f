"""Thin ctypes binding of libmcf (``include/mcf.h``): argument marshalling only.

The functions carry the C entry points' names.  Arrays may be numpy arrays
(host memory) or torch tensors (host or CUDA memory); every computation runs
in the library's CUDA kernels.  Importing this module does not load the
library; the first call does, and raises if ``libmcf.so`` has not been built
(``__graft_entry__.build()`` or ``python paper_2308_01037_gb300/build.py``).
There is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

MCF_OK = 0
MCF_F64 = 0
MCF_F32W_F64ACC = 1
MCF_GRAPH_DEVICE_PTRS = 1
MCF_GRAPH_NONSYMMETRIC = 2
MCF_MAX_COEFFS = 256

STATUS_NAMES = {
    0: "MCF_OK", 1: "MCF_ERR_INVALID_ARG", 2: "MCF_ERR_INVALID_GRAPH", 3: "MCF_ERR_OOM", 4: "MCF_ERR_CUDA",
    5: "MCF_ERR_ADMISSION", 6: "MCF_ERR_TIMEOUT", 7: "MCF_ERR_CANCELLED", 8: "MCF_ERR_ACCURACY_BUDGET",
    9: "MCF_WARN_OVERFLOW", 10: "MCF_ERR_UNSUPPORTED",
}


class McfError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class mcf_params(ctypes.Structure):
    _fields_ = [("coeffs", ctypes.c_void_p), ("n_coeffs", ctypes.c_int32), ("scale", ctypes.c_double),
                ("n_walks", ctypes.c_int64), ("walks_per_node", ctypes.c_int64), ("w_cutoff", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("request_id", ctypes.c_uint32), ("precision", ctypes.c_int32),
                ("deterministic", ctypes.c_int32), ("error_estimate", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("target_rel_err", ctypes.c_double), ("max_walks", ctypes.c_int64)]


class mcf_query(ctypes.Structure):
    _fields_ = [("graph", ctypes.c_void_p), ("kind", ctypes.c_int32), ("katz_terms", ctypes.c_int32),
                ("katz_gamma", ctypes.c_double), ("params", mcf_params), ("v", ctypes.c_void_p),
                ("nodes", ctypes.c_void_p), ("n_nodes", ctypes.c_int64), ("out", ctypes.c_void_p)]


MCF_QUERY_TOTAL_COMMUNICABILITY = 0
MCF_QUERY_KATZ = 1
MCF_QUERY_SUBGRAPH_CENTRALITY = 2
MCF_QUERY_ACTION = 3
MCF_BATCH_CUDA_GRAPH = 1
MCF_BATCH_AUTOTUNE = 2


class mcf_server_config(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_inflight", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("batch_window_ms", ctypes.c_double)]


class mcf_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("rejected", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("cancelled", ctypes.c_int64), ("walk_steps", ctypes.c_int64),
                ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("busy_s", ctypes.c_double), ("device_overlap_ms", ctypes.c_double),
                ("max_concurrent_batches", ctypes.c_int64), ("plan_s", ctypes.c_double), ("run_s", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class mcf_stats(ctypes.Structure):
    _fields_ = [("walks", ctypes.c_int64), ("walk_steps", ctypes.c_int64), ("kernel_ms", ctypes.c_double),
                ("flags", ctypes.c_uint32), ("max_rel_se", ctypes.c_double), ("est_rel_err", ctypes.c_double),
                ("replicas", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# Every entry point declared in include/mcf.h, with its ctypes signature.
_P, _I64, _I32, _U32, _D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32, ctypes.c_double
SIGNATURES = {
    "mcf_create_graph": ([_I64, _P, _P, _P, _U32, _P], ctypes.c_int),
    "mcf_destroy_graph": ([_P], ctypes.c_int),
    "mcf_graph_info": ([_P, _P, _P, _P, _P], ctypes.c_int),
    "mcf_spectral_radius": ([_P, _D, _I32, _P], ctypes.c_int),
    "mcf_gershgorin": ([_P, _P], ctypes.c_int),
    "mcf_action": ([_P, _P, _P, _P, _P], ctypes.c_int),
    "mcf_action_nodes": ([_P, _P, _P, _P, _I64, _P, _P], ctypes.c_int),
    "mcf_total_communicability": ([_P, _P, _P, _P], ctypes.c_int),
    "mcf_subgraph_centrality": ([_P, _P, _P, _I64, _P, _P], ctypes.c_int),
    "mcf_katz": ([_P, _D, _I32, _P, _P, _P], ctypes.c_int),
    "mcf_funm_full": ([_P, _P, _P, _P], ctypes.c_int),
    "mcf_mc_classic": ([_P, _P, _P, _P, _I64, _P, _P], ctypes.c_int),
    "mcf_batch_create": ([_P, _I32, _U32, _P, _P], ctypes.c_int),
    "mcf_batch_run": ([_P, _P, _P], ctypes.c_int),
    "mcf_batch_destroy": ([_P], ctypes.c_int),
    "mcf_server_create": ([_P, _P], ctypes.c_int),
    "mcf_server_submit": ([_P, _P, _P], ctypes.c_int),
    "mcf_server_poll": ([_P, ctypes.c_uint64, _P, _P], ctypes.c_int),
    "mcf_server_wait": ([_P, ctypes.c_uint64, _D, _P, _P], ctypes.c_int),
    "mcf_server_get_stats": ([_P, _P], ctypes.c_int),
    "mcf_server_destroy": ([_P], ctypes.c_int),
    "mcf_server_release": ([_P, ctypes.c_uint64], ctypes.c_int),
    "mcf_server_cancel": ([_P, ctypes.c_uint64], ctypes.c_int),
    "mcf_query_footprint": ([_P, _P], ctypes.c_int),
    "mcf_batch_device_bytes": ([_P, _P], ctypes.c_int),
    "mcf_total_communicability_noalloc": ([_I64, _I64, _P, _P, _P, _P], ctypes.c_int),
    "mcf_gather_probe": ([_I64, _I64, _P, _P], ctypes.c_int),
    "mcf_second_moment_radius": ([_P, _D, _D, _I32, _P], ctypes.c_int),
    "mcf_kernel_launches": ([_P], ctypes.c_int),
    "mcf_inject_allocation_failure": ([_I64], ctypes.c_int),
    "mcf_last_error": ([], ctypes.c_char_p),
    "mcf_version": ([], ctypes.c_char_p),
}

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load():
    """Loads libmcf.so (must already be built) and declares its prototypes."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(f"libmcf.so is not built ({path}); run __graft_entry__.build()")
            lib = ctypes.CDLL(path)
            for name, (args, res) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def _check(status: int):
    if status != MCF_OK:
        raise McfError(status, (load().mcf_last_error() or b"").decode())


MCF_ERR_ACCURACY_BUDGET = 8


def _solved(status: int, y, st, stats: bool):
    """Result of a solve entry point.  An accuracy-targeted solve that stops at
    its walk cap still returns its mean: with ``stats=True`` the result comes
    back with ``budget_met = False`` in the stats; without, the binding raises."""
    met = status != MCF_ERR_ACCURACY_BUDGET
    if status != MCF_OK and not (stats and not met):
        _check(status)
    if stats:
        d = st.as_dict()
        d["budget_met"] = met
        return y, d
    return y


# ---------------------------------------------------------------- marshalling helpers
def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype):
    """(pointer, keep-alive object) of a numpy array or torch tensor in the given dtype."""
    if x is None:
        return None, None
    if _is_torch(x):
        import torch

        tdt = {np.int64: torch.int64, np.int32: torch.int32, np.float32: torch.float32,
               np.float64: torch.float64}[dtype]
        if x.dtype != tdt or not x.is_contiguous():
            x = x.to(tdt).contiguous()
        return x.data_ptr(), x
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data, a


def _out_ptr(x):
    """Pointer of an output buffer the library writes in place: it must already be
    float64 and contiguous (a converted copy would take the results instead)."""
    if _is_torch(x):
        import torch

        if x.dtype != torch.float64 or not x.is_contiguous():
            raise TypeError(f"output must be a contiguous float64 tensor, got {x.dtype}"
                            f"{'' if x.is_contiguous() else ' (not contiguous)'}")
        return x.data_ptr(), x
    if not (isinstance(x, np.ndarray) and x.dtype == np.float64 and x.flags.c_contiguous and x.flags.writeable):
        raise TypeError("output must be a writeable C-contiguous float64 numpy array or torch tensor")
    return x.ctypes.data, x


def _stream_of(*arrays):
    for a in arrays:
        if a is not None and _is_torch(a) and a.is_cuda:
            import torch

            return torch.cuda.current_stream(a.device).cuda_stream
    return None


def _params(coeffs, scale=0.0, n_walks=0, walks_per_node=0, w_cutoff=0.0, seed=0, request_id=0,
            precision=MCF_F32W_F64ACC, stream=None, error_estimate=False, target_rel_err=0.0, max_walks=0,
            deterministic=False):
    c = np.ascontiguousarray(coeffs, dtype=np.float64)
    p = mcf_params(c.ctypes.data, len(c), float(scale), int(n_walks), int(walks_per_node), float(w_cutoff),
                   int(seed) & 0xFFFFFFFFFFFFFFFF, int(request_id) & 0xFFFFFFFF, int(precision),
                   1 if deterministic else 0, 1 if error_estimate else 0, stream if stream else None,
                   float(target_rel_err), int(max_walks))
    return p, c


class GraphHandle:
    """Owns an mcf_graph_t; released by mcf_destroy_graph when collected or closed."""

    def __init__(self, handle: int, n: int, nnz: int):
        self.handle = handle
        self.n = n
        self.nnz = nnz

    def close(self):
        if self.handle:
            load().mcf_destroy_graph(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- entry points
def mcf_create_graph(n, row_ptr, col_idx, values=None, symmetric=True) -> GraphHandle:
    """Uploads a CSR matrix (numpy or torch; device tensors copied device to device);
    ``symmetric=False`` accepts a general A (MCF_GRAPH_NONSYMMETRIC)."""
    lib = load()
    rp, krp = _ptr(row_ptr, np.int64)
    ci, kci = _ptr(col_idx if len(col_idx) else np.zeros(1, np.int32), np.int32)
    va, kva = _ptr(values, np.float32)
    dev = 1 if (_is_torch(row_ptr) and row_ptr.is_cuda) else 0
    flags = (MCF_GRAPH_DEVICE_PTRS if dev else 0) | (0 if symmetric else MCF_GRAPH_NONSYMMETRIC)
    h = ctypes.c_void_p()
    _check(lib.mcf_create_graph(int(n), rp, ci, va, flags, ctypes.byref(h)))
    nnz = int(krp[-1])
    return GraphHandle(h.value, int(n), nnz)


def mcf_destroy_graph(g: GraphHandle):
    g.close()


def mcf_graph_info(g: GraphHandle) -> dict:
    vals = [ctypes.c_int64() for _ in range(4)]
    _check(load().mcf_graph_info(g.handle, *[ctypes.byref(v) for v in vals]))
    return dict(zip(("n", "nnz", "max_degree", "n_loops"), (v.value for v in vals)))


def mcf_spectral_radius(g: GraphHandle, tol=1e-10, max_iter=10000) -> float:
    out = ctypes.c_double()
    _check(load().mcf_spectral_radius(g.handle, float(tol), int(max_iter), ctypes.byref(out)))
    return out.value


def mcf_second_moment_radius(g: GraphHandle, scale, tol=1e-8, max_iter=10000) -> float:
    """Spectral radius of diag(sum_j |a'_ij|) |A'| with A' = scale * A (the walk weights' second-moment growth)."""
    out = ctypes.c_double()
    _check(load().mcf_second_moment_radius(g.handle, float(scale), float(tol), int(max_iter), ctypes.byref(out)))
    return out.value


def mcf_gershgorin(g: GraphHandle) -> float:
    out = ctypes.c_double()
    _check(load().mcf_gershgorin(g.handle, ctypes.byref(out)))
    return out.value


def _output(out, m, like):
    """The caller's output, else a new one: on the device of a CUDA ``like``,
    otherwise host memory (page-locked when CUDA is present, see _host_output)."""
    if out is not None:
        return out
    if like is not None and _is_torch(like) and like.is_cuda:
        import torch

        return torch.empty(max(m, 0), dtype=torch.float64, device=like.device)
    return _host_output(m)


def _host_output(m):
    """A float64 host array for a result the library writes in full.  With CUDA
    present it lives in page-locked memory from torch's caching host allocator
    (a numpy view, which keeps the block alive): the library's device-to-host
    copy into it is a plain DMA, while a copy into pageable memory is staged by
    the driver, serialises with other threads' pageable copies and, into a
    fresh np.zeros array, first faults in every page (measured on the request
    server with six workers: 370 against 200 solves/s)."""
    try:
        import torch

        if torch.cuda.is_available():
            return torch.empty(max(m, 0), dtype=torch.float64, pin_memory=True).numpy()
    except (ImportError, RuntimeError):
        pass
    return np.zeros(max(m, 0), dtype=np.float64)


def mcf_action(g: GraphHandle, v, coeffs, out=None, device_out=None, stats=False, **kw):
    """f(A')v by RandFunmAction; keyword arguments fill mcf_params."""
    y = _output(out, g.n, device_out if device_out is not None else v)
    vp, kv = _ptr(v, np.float64)
    yp, ky = _out_ptr(y)
    st = mcf_stats()
    p, kc = _params(coeffs, stream=kw.pop("stream", None) or _stream_of(v, y), **kw)
    rc = load().mcf_action(g.handle, ctypes.byref(p), vp, yp, ctypes.byref(st) if stats else None)
    return _solved(rc, y, st, stats)


def mcf_action_nodes(g: GraphHandle, nodes, coeffs, v=None, out=None, device_out=None, stats=False, **kw):
    """Entries ``nodes`` of f(A')v (v = None: total communicability), walking only their neighbours."""
    y = _output(out, len(nodes), device_out if device_out is not None else nodes)
    vp, kv = _ptr(v, np.float64)
    npt, kn = _ptr(nodes, np.int64)
    yp, ky = _out_ptr(y)
    st = mcf_stats()
    p, kc = _params(coeffs, stream=kw.pop("stream", None) or _stream_of(nodes, y), **kw)
    rc = load().mcf_action_nodes(g.handle, ctypes.byref(p), vp, npt, int(len(nodes)), yp,
                                 ctypes.byref(st) if stats else None)
    return _solved(rc, y, st, stats)


def mcf_total_communicability(g: GraphHandle, coeffs, out=None, device_out=None, stats=False, **kw):
    """f(A')1 (total communicability)."""
    y = _output(out, g.n, device_out)
    yp, ky = _out_ptr(y)
    st = mcf_stats()
    p, kc = _params(coeffs, stream=kw.pop("stream", None) or _stream_of(y), **kw)
    rc = load().mcf_total_communicability(g.handle, ctypes.byref(p), yp, ctypes.byref(st) if stats else None)
    return _solved(rc, y, st, stats)


def mcf_subgraph_centrality(g: GraphHandle, coeffs, nodes=None, out=None, device_out=None, stats=False, **kw):
    """diag f(A') by RandFunmDiag, all nodes or ``nodes``."""
    m = g.n if nodes is None else len(nodes)
    d = _output(out, m, device_out if device_out is not None else nodes)
    npt, kn = _ptr(nodes, np.int64)
    dp, kd = _out_ptr(d)
    st = mcf_stats()
    p, kc = _params(coeffs, stream=kw.pop("stream", None) or _stream_of(nodes, d), **kw)
    rc = load().mcf_subgraph_centrality(g.handle, ctypes.byref(p), npt, int(m), dp,
                                        ctypes.byref(st) if stats else None)
    return _solved(rc, d, st, stats)


def mcf_katz(g: GraphHandle, gamma, K=0, out=None, device_out=None, stats=False, **kw):
    """(I - gamma A)^{-1} 1 as the truncated Neumann series (K = 0: from the tail bound)."""
    y = _output(out, g.n, device_out)
    yp, ky = _out_ptr(y)
    st = mcf_stats()
    p, kc = _params([1.0], stream=kw.pop("stream", None) or _stream_of(y), **kw)
    rc = load().mcf_katz(g.handle, float(gamma), int(K), ctypes.byref(p), yp, ctypes.byref(st) if stats else None)
    return _solved(rc, y, st, stats)


MCF_FULL_MAX_NODES = 16384


def mcf_funm_full(g: GraphHandle, coeffs, out=None, device_out=None, stats=False, **kw):
    """Dense estimate F (n x n, row-major) of f(A') by RandFunm (Algorithm 2)."""
    F = _output(out, g.n * g.n, device_out)
    Fp, kf = _out_ptr(F)
    st = mcf_stats()
    p, kc = _params(coeffs, stream=kw.pop("stream", None) or _stream_of(F), **kw)
    _check(load().mcf_funm_full(g.handle, ctypes.byref(p), Fp, ctypes.byref(st) if stats else None))
    F = F.reshape(g.n, g.n)
    return (F, st.as_dict()) if stats else F


def mcf_mc_classic(g: GraphHandle, coeffs, walks_per_row, v=None, nodes=None, out=None, device_out=None,
                   stats=False, **kw):
    """Entries of f(A')v by the classical Monte Carlo method (Algorithm 1), float64."""
    m = g.n if nodes is None else len(nodes)
    y = _output(out, m, device_out if device_out is not None else (nodes if nodes is not None else v))
    vp, kv = _ptr(v, np.float64)
    npt, kn = _ptr(nodes, np.int64)
    yp, ky = _out_ptr(y)
    st = mcf_stats()
    kw.setdefault("precision", MCF_F64)
    p, kc = _params(coeffs, walks_per_node=int(walks_per_row), stream=kw.pop("stream", None) or _stream_of(v, nodes, y),
                    **kw)
    _check(load().mcf_mc_classic(g.handle, ctypes.byref(p), vp, npt, int(m), yp,
                                 ctypes.byref(st) if stats else None))
    return (y, st.as_dict()) if stats else y


def _query_struct(q):
    """mcf_query for a dict (see mcf_batch_create) plus the objects it points into."""
    g = q["graph"]
    kind = q["kind"]
    nodes = q.get("nodes")
    m = len(nodes) if (kind == MCF_QUERY_SUBGRAPH_CENTRALITY and nodes is not None) else g.n
    out = q.get("out")
    if out is None:
        out = _output(None, m, q.get("device_out"))
    op, ko = _out_ptr(out)
    vp, kv = _ptr(q.get("v"), np.float64)
    npt, kn = _ptr(nodes, np.int64)
    pkw = {k: q[k] for k in ("scale", "n_walks", "walks_per_node", "w_cutoff", "seed", "request_id", "precision",
                             "target_rel_err", "max_walks", "deterministic") if k in q}
    p, kc = _params(q.get("coeffs", [1.0]), **pkw)
    st = mcf_query(g.handle, kind, int(q.get("katz_terms", 0)), float(q.get("katz_gamma", 0.0)), p, vp, npt,
                   int(0 if nodes is None else len(nodes)), op)
    return st, out, [ko, kv, kn, kc, g]


class BatchHandle:
    """Owns an mcf_batch_t and keeps the arrays its queries point to alive."""

    def __init__(self, handle, keep, outputs):
        self.handle = handle
        self._keep = keep
        self.outputs = outputs

    def close(self):
        if self.handle:
            load().mcf_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mcf_batch_create(queries, flags=0, stream=None):
    """Plans a batch.  ``queries``: list of dicts with keys graph (GraphHandle),
    kind (MCF_QUERY_*), coeffs, out (array; allocated when absent), and the
    mcf_params keywords (scale, n_walks, walks_per_node, w_cutoff, seed,
    request_id, precision), plus katz_gamma/katz_terms, v, nodes."""
    arr = (mcf_query * len(queries))()
    keep, outputs = [], []
    for i, q in enumerate(queries):
        arr[i], out, k = _query_struct(q)
        outputs.append(out)
        keep += k
    h = ctypes.c_void_p()
    _check(load().mcf_batch_create(arr, len(queries), int(flags), stream, ctypes.byref(h)))
    return BatchHandle(h.value, keep + [arr], outputs)


def mcf_batch_run(b: BatchHandle, stream=None, stats=False):
    st = mcf_stats()
    _check(load().mcf_batch_run(b.handle, stream, ctypes.byref(st) if stats else None))
    return (b.outputs, st.as_dict()) if stats else b.outputs


def mcf_batch_destroy(b: BatchHandle):
    b.close()


class ServerHandle:
    """Owns an mcf_server_t and the arrays of its pending requests."""

    def __init__(self, handle):
        self.handle = handle
        self.pending = {}

    def close(self):
        if self.handle:
            load().mcf_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mcf_server_create(hbm_budget_bytes, max_inflight=2, max_batch=16, batch_window_ms=0.0) -> ServerHandle:
    cfg = mcf_server_config(int(hbm_budget_bytes), int(max_inflight), int(max_batch), float(batch_window_ms))
    h = ctypes.c_void_p()
    _check(load().mcf_server_create(ctypes.byref(cfg), ctypes.byref(h)))
    return ServerHandle(h.value)


def mcf_server_submit(s: ServerHandle, query: dict) -> int:
    """Queues a request (dict as for mcf_batch_create); returns its ticket."""
    st, out, keep = _query_struct(query)
    t = ctypes.c_uint64()
    _check(load().mcf_server_submit(s.handle, ctypes.byref(st), ctypes.byref(t)))
    s.pending[t.value] = (out, keep + [st])
    return t.value


def mcf_server_poll(s: ServerHandle, ticket: int):
    done, res = ctypes.c_int32(), ctypes.c_int()
    _check(load().mcf_server_poll(s.handle, ctypes.c_uint64(ticket), ctypes.byref(done), ctypes.byref(res)))
    return bool(done.value), res.value


def mcf_server_wait(s: ServerHandle, ticket: int, timeout_s: float = -1.0, accept_budget_miss: bool = False):
    """Waits for a ticket; returns (output array, latency in ms); raises on a failed request
    (an accuracy-targeted request that stopped at its walk cap counts as served when
    ``accept_budget_miss`` is set: its mean is in the output)."""
    res, lat = ctypes.c_int(), ctypes.c_double()
    _check(load().mcf_server_wait(s.handle, ctypes.c_uint64(ticket), float(timeout_s), ctypes.byref(res),
                                  ctypes.byref(lat)))
    if not (accept_budget_miss and res.value == MCF_ERR_ACCURACY_BUDGET):
        _check(res.value)
    out, _ = s.pending.pop(ticket)
    return out, lat.value


def mcf_server_cancel(s: ServerHandle, ticket: int):
    """Cancels a queued request (it completes with MCF_ERR_CANCELLED)."""
    _check(load().mcf_server_cancel(s.handle, ctypes.c_uint64(ticket)))


def mcf_server_release(s: ServerHandle, ticket: int):
    """Forgets a completed request."""
    _check(load().mcf_server_release(s.handle, ctypes.c_uint64(ticket)))
    s.pending.pop(ticket, None)


def mcf_query_footprint(query: dict) -> int:
    """Device bytes the server charges a request (see mcf_batch_create for the dict)."""
    st, out, keep = _query_struct(query)
    b = ctypes.c_size_t()
    _check(load().mcf_query_footprint(ctypes.byref(st), ctypes.byref(b)))
    return int(b.value)


def mcf_batch_device_bytes(b: BatchHandle) -> int:
    out = ctypes.c_size_t()
    _check(load().mcf_batch_device_bytes(b.handle, ctypes.byref(out)))
    return int(out.value)


def mcf_server_get_stats(s: ServerHandle) -> dict:
    st = mcf_server_stats()
    _check(load().mcf_server_get_stats(s.handle, ctypes.byref(st)))
    return st.as_dict()


def mcf_server_destroy(s: ServerHandle):
    s.close()


def mcf_total_communicability_noalloc(n, row_ptr, col_idx, coeffs, out, **kw):
    """f(A')1 with no device allocation by the library; CSR and ``out`` must be CUDA tensors."""
    rp, krp = _ptr(row_ptr, np.int64)
    ci, kci = _ptr(col_idx, np.int32)
    yp, ky = _out_ptr(out)
    nnz = int(col_idx.numel()) if _is_torch(col_idx) else len(col_idx)
    p, kc = _params(coeffs, stream=kw.pop("stream", None) or _stream_of(out), **kw)
    _check(load().mcf_total_communicability_noalloc(int(n), nnz, rp, ci, ctypes.byref(p), yp))
    return out


def mcf_gather_probe(array_bytes, reads, stream=None) -> float:
    """Random 8-byte reads per second over a device array of ``array_bytes``."""
    out = ctypes.c_double()
    _check(load().mcf_gather_probe(int(array_bytes), int(reads), stream, ctypes.byref(out)))
    return out.value


def mcf_kernel_launches() -> int:
    """Kernel executions of the library on the current device since it was loaded."""
    out = ctypes.c_uint64()
    _check(load().mcf_kernel_launches(ctypes.byref(out)))
    return int(out.value)


def mcf_inject_allocation_failure(after: int):
    """The next scratch allocation after ``after`` successful ones fails with MCF_ERR_OOM (< 0: off)."""
    _check(load().mcf_inject_allocation_failure(int(after)))


def mcf_last_error() -> str:
    return (load().mcf_last_error() or b"").decode()


def mcf_version() -> str:
    return (load().mcf_version() or b"").decode()
