"""ctypes binding of ``mcf_oracle.c`` (ORACLE -- test infrastructure only).

Every function takes the CSR arrays of a symmetric graph (``row_ptr`` int64,
``col_idx`` int32, optional float32 ``values``) and follows the paper's
notation: ``gamma`` scales A (f(gamma A), Section 2.2), ``coeffs`` are
zeta_0..zeta_K (Eq. power_series), ``n_walks`` is N_s, ``w_cutoff`` is W_c
(Eq. weight_cutoff).  Precision 0 computes in float64 throughout; precision 1
keeps the walk weight, coefficients and r in float32 and accumulates in
float64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRC = os.path.join(_HERE, "mcf_oracle.c")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles the C oracle (no fused multiply-add) into ``_build/liboracle.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _lib_():
    global _lib
    with _lock:
        if _lib is None:
            # MCF_ORACLE_LIB names another build of mcf_oracle.c: the tests
            # that plant mistakes in a copy of the oracle load it this way
            lib = ctypes.CDLL(os.environ.get("MCF_ORACLE_LIB") or build())
            P, i64, u64, u32, dbl, i32 = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32,
                                          ctypes.c_double, ctypes.c_int)
            lib.orc_philox4x32_10.argtypes = [P, P, P]
            lib.orc_philox4x32_10.restype = None
            lib.orc_action.argtypes = [i64, P, P, P, dbl, P, P, i32, i64, i64, dbl, u64, u32, i32, P, i64, P, P, P]
            lib.orc_diag.argtypes = [i64, P, P, P, dbl, P, i32, i64, i64, dbl, u64, u32, i32, P, i64, P, P]
            lib.orc_funm_full.argtypes = [i64, P, P, P, dbl, P, i32, i64, i64, dbl, u64, u32, i32, P]
            lib.orc_action_se.argtypes = [i64, P, P, P, dbl, P, P, i32, i64, i64, dbl, u64, u32, i32, P, i64, P]
            lib.orc_sample_counts.argtypes = [i64, P, P, P, i64, i64, u64, u32, P]
            lib.orc_mc_classic_action.argtypes = [i64, P, P, P, dbl, P, P, i32, i64, dbl, u64, u32, P, i64, P]
            lib.orc_allocation.argtypes = [i64, P, P, P, dbl, i64, i64, P, P, P, P]
            lib.orc_alias_row.argtypes = [i64, P, P, P]
            for f in ("orc_action", "orc_diag", "orc_funm_full", "orc_mc_classic_action", "orc_allocation",
                      "orc_alias_row", "orc_action_se", "orc_sample_counts"):
                getattr(lib, f).restype = i32
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _csr(g, values):
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(g.col_idx, dtype=np.int32)
    if ci.size == 0:
        ci = np.zeros(1, dtype=np.int32)
    val = None if values is None else np.ascontiguousarray(values, dtype=np.float32)
    return rp, ci, val


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with status {rc}")


def philox4x32_10(ctr, key) -> np.ndarray:
    """One Philox4x32-10 block for counter (4 x u32) and key (2 x u32)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _lib_().orc_philox4x32_10(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


def allocation(g, gamma=1.0, n_walks=0, walks_per_node=0, values=None):
    """Returns (rowabs, colnorm, N_i, walk offsets) of Definition 1."""
    rp, ci, val = _csr(g, values)
    n = g.n
    ra, cn = np.zeros(n), np.zeros(n)
    nw, off = np.zeros(n, np.int64), np.zeros(n + 1, np.int64)
    _check(_lib_().orc_allocation(n, _p(rp), _p(ci), _p(val), gamma, n_walks, walks_per_node,
                                  _p(ra), _p(cn), _p(nw), _p(off)), "allocation")
    return ra, cn, nw, off


def alias_row(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    prob = np.zeros(len(a), np.float32)
    alias = np.zeros(len(a), np.int32)
    _check(_lib_().orc_alias_row(len(a), _p(a), _p(prob), _p(alias)), "alias_row")
    return prob, alias


def action(g, coeffs, v=None, gamma=1.0, n_walks=0, walks_per_node=0, w_cutoff=0.0, seed=0,
           request_id=0, precision=0, nodes=None, values=None, return_q=False):
    """RandFunmAction (Algorithm 3): estimate of f(gamma A) v (v = 1 by default).

    With ``nodes`` only those entries are returned, computed from the walks of
    their neighbours (same walk ids as the full run)."""
    rp, ci, val = _csr(g, values)
    n = g.n
    vv = np.ones(n) if v is None else np.ascontiguousarray(v, dtype=np.float64)
    z = np.ascontiguousarray(coeffs, dtype=np.float64)
    nd = None if nodes is None else np.ascontiguousarray(nodes, dtype=np.int64)
    m = n if nd is None else len(nd)
    y = np.zeros(max(m, 1))
    q = np.zeros(max(n, 1)) if return_q else None
    stats = np.zeros(2, np.int64)
    _check(_lib_().orc_action(n, _p(rp), _p(ci), _p(val), gamma, _p(vv), _p(z), len(z), n_walks, walks_per_node,
                              w_cutoff, seed, request_id, precision, _p(nd), 0 if nd is None else len(nd),
                              _p(y), _p(q), _p(stats)), "action")
    out = {"y": y[:m], "walks": int(stats[0]), "steps": int(stats[1])}
    if return_q:
        out["q"] = q[:n]
    return out


def diag(g, coeffs, gamma=1.0, n_walks=0, walks_per_node=0, w_cutoff=0.0, seed=0, request_id=0, precision=0,
         nodes=None, values=None):
    """RandFunmDiag (Section 3.3): estimate of diag f(gamma A), all nodes or ``nodes``."""
    rp, ci, val = _csr(g, values)
    n = g.n
    z = np.ascontiguousarray(coeffs, dtype=np.float64)
    nd = None if nodes is None else np.ascontiguousarray(nodes, dtype=np.int64)
    m = n if nd is None else len(nd)
    d = np.zeros(max(m, 1))
    stats = np.zeros(2, np.int64)
    _check(_lib_().orc_diag(n, _p(rp), _p(ci), _p(val), gamma, _p(z), len(z), n_walks, walks_per_node, w_cutoff,
                            seed, request_id, precision, _p(nd), 0 if nd is None else len(nd), _p(d), _p(stats)),
           "diag")
    return {"d": d[:m], "walks": int(stats[0]), "steps": int(stats[1])}


def action_se(g, coeffs, v=None, gamma=1.0, n_walks=0, walks_per_node=0, w_cutoff=0.0, seed=0, request_id=0,
              precision=0, nodes=None, values=None):
    """Per-entry standard error of RandFunmAction from the sample variance of the walks (Section 3.5)."""
    rp, ci, val = _csr(g, values)
    n = g.n
    vv = np.ones(n) if v is None else np.ascontiguousarray(v, dtype=np.float64)
    z = np.ascontiguousarray(coeffs, dtype=np.float64)
    nd = None if nodes is None else np.ascontiguousarray(nodes, dtype=np.int64)
    se = np.zeros(n if nd is None else len(nd))
    _check(_lib_().orc_action_se(n, _p(rp), _p(ci), _p(val), gamma, _p(vv), _p(z), len(z), n_walks, walks_per_node,
                                 w_cutoff, seed, request_id, precision, _p(nd), 0 if nd is None else len(nd),
                                 _p(se)), "action_se")
    return se


def sample_counts(g, row, n_draws, seed=0, request_id=0, values=None):
    """How often SelectNextState picks each position of ``row`` in n_draws walk steps."""
    rp, ci, val = _csr(g, values)
    d = int(g.row_ptr[row + 1] - g.row_ptr[row])
    counts = np.zeros(d, dtype=np.int64)
    _check(_lib_().orc_sample_counts(g.n, _p(rp), _p(ci), _p(val), int(row), int(n_draws), seed, request_id,
                                     _p(counts)), "sample_counts")
    return counts


def funm_full(g, coeffs, gamma=1.0, n_walks=0, walks_per_node=0, w_cutoff=0.0, seed=0, request_id=0,
              precision=0, values=None):
    """RandFunm (Algorithm 2): dense estimate F of f(gamma A) (n <= 4096)."""
    rp, ci, val = _csr(g, values)
    n = g.n
    z = np.ascontiguousarray(coeffs, dtype=np.float64)
    F = np.zeros((n, n))
    _check(_lib_().orc_funm_full(n, _p(rp), _p(ci), _p(val), gamma, _p(z), len(z), n_walks, walks_per_node,
                                 w_cutoff, seed, request_id, precision, _p(F)), "funm_full")
    return F


def mc_classic_action(g, coeffs, nodes, walks_per_row, v=None, gamma=1.0, w_cutoff=0.0, seed=0, request_id=0,
                      values=None):
    """Classical Monte Carlo (Algorithm 1) for the entries ``nodes`` of f(gamma A) v."""
    rp, ci, val = _csr(g, values)
    n = g.n
    vv = np.ones(n) if v is None else np.ascontiguousarray(v, dtype=np.float64)
    z = np.ascontiguousarray(coeffs, dtype=np.float64)
    nd = np.ascontiguousarray(nodes, dtype=np.int64)
    y = np.zeros(len(nd))
    _check(_lib_().orc_mc_classic_action(n, _p(rp), _p(ci), _p(val), gamma, _p(vv), _p(z), len(z), walks_per_row,
                                         w_cutoff, seed, request_id, _p(nd), len(nd), _p(y)), "mc_classic")
    return y
