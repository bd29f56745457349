"""Thin ctypes binding of libgbfmm.so (include/gbfmm.h), same names as the C ABI.

Argument marshalling only: tensors are passed as raw device pointers with torch's current
CUDA stream; every step of the evaluation runs in the library's CUDA kernels.  There is no
CPU fallback: if the library is missing or fails to load, the import-time helpers raise.
"""
from __future__ import annotations

import ctypes
import os
import re

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB_PATH = os.path.join(HERE, "_build", "libgbfmm.so")
HEADER = os.path.join(ROOT, "include", "gbfmm.h")

GBFMM_OK, GBFMM_EINVAL, GBFMM_ENOMEM, GBFMM_ECUDA, GBFMM_ETIMEOUT, GBFMM_EUNSUPPORTED = range(6)
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "EUNSUPPORTED"}
METHOD_FMM, METHOD_TREECODE = 0, 1
TREE_UNIFORM, TREE_ADAPTIVE = 0, 1
LIST_P2P, LIST_M2L, LIST_U, LIST_V, LIST_W, LIST_X = range(6)
FLAG_STAGE_TIMING = 1
FLAG_M2L_CUDA_CORES = 2
FLAG_SERIAL = 4
FLAG_M2L_GATHERED = 8
FLAG_M2L_ROTATION = 16
STAGES = ["box+keys", "sort", "cells+lists", "P2M", "M2M", "M2L/M2P", "L2L", "L2P", "P2P", "operators"]


class gbfmm_params(ctypes.Structure):
    _fields_ = [
        ("p", ctypes.c_int32),
        ("leaf_size", ctypes.c_int32),
        ("tree", ctypes.c_int32),
        ("method", ctypes.c_int32),
        ("eps2", ctypes.c_double),
        ("has_box", ctypes.c_int32),
        ("flags", ctypes.c_int32),
        ("box_origin", ctypes.c_double * 3),
        ("box_side", ctypes.c_double),
    ]


class GbfmmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def declared_symbols() -> list[str]:
    """Function names declared in include/gbfmm.h."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char \*)\s*\**(gbfmm_\w+)\s*\(", text, flags=re.M)))


def lib():
    """Load libgbfmm.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libgbfmm.so not built ({LIB_PATH}); run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    i = ctypes.c_int
    i64 = ctypes.c_int64
    sig = {
        "gbfmm_version": (i, []),
        "gbfmm_default_params": (i, [ctypes.POINTER(gbfmm_params)]),
        "gbfmm_create": (i, [ctypes.POINTER(P), i]),
        "gbfmm_destroy": (i, [P]),
        "gbfmm_last_error": (ctypes.c_char_p, [P]),
        "gbfmm_plan": (i, [ctypes.POINTER(gbfmm_params), i64, ctypes.POINTER(ctypes.c_int32),
                           ctypes.POINTER(ctypes.c_size_t)]),
        "gbfmm_evaluate": (i, [P, ctypes.POINTER(gbfmm_params), i64, P, P, P, ctypes.c_size_t, P]),
        "gbfmm_evaluate_host": (i, [P, ctypes.POINTER(gbfmm_params), i64, P, P, P]),
        "gbfmm_sync_status": (i, [P, P]),
        "gbfmm_direct": (i, [P, i64, P, i64, P, ctypes.c_double, P, P]),
        "gbfmm_export_tree": (i, [P, P, P, P, P, P]),
        "gbfmm_export_lists": (i, [P, i, P, P, i64, ctypes.POINTER(i64)]),
        "gbfmm_export_expansions": (i, [P, i, P]),
        "gbfmm_export_adaptive_tree": (i, [P, P, ctypes.POINTER(i64), P, P, P, P, P, P]),
        "gbfmm_stage_times": (i, [P, P, i, ctypes.POINTER(i)]),
        "gbfmm_last_launch_count": (i, [P, ctypes.POINTER(i64)]),
        "gbfmm_sort_static": (i, [ctypes.POINTER(gbfmm_params), i64, P, P, P, P, P, P]),
        "gbfmm_selftest_wait": (i, [P, ctypes.c_double, P]),
        "gbfmm_engine_create": (i, [ctypes.POINTER(P), i, ctypes.c_int32, ctypes.c_size_t]),
        "gbfmm_engine_destroy": (i, [P]),
        "gbfmm_engine_prepare": (i, [P, P, ctypes.c_int32]),
        "gbfmm_engine_submit": (i, [P, ctypes.POINTER(gbfmm_params), i64, P, P, ctypes.POINTER(i64)]),
        "gbfmm_engine_wait": (i, [P, i64, ctypes.c_double, ctypes.POINTER(ctypes.c_int32),
                                  ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
        "gbfmm_engine_run_batch": (i, [P, ctypes.c_int32, P, P, P, P, P]),
        "gbfmm_graph_create": (i, [ctypes.POINTER(P), P, ctypes.POINTER(gbfmm_params), i64, P, P, P,
                                   ctypes.c_size_t]),
        "gbfmm_graph_launch": (i, [P, P]),
        "gbfmm_graph_destroy": (i, [P]),
        "gbfmm_tune_leaf": (i, [P, ctypes.POINTER(gbfmm_params), i64, P, P, ctypes.c_int32,
                                ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_float)]),
        "gbfmm_tune": (i, [P, ctypes.POINTER(gbfmm_params), i64, P, P, ctypes.c_int32, P, ctypes.c_int32,
                           ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                           ctypes.POINTER(ctypes.c_float)]),
        "gbfmm_set_p2p_leaves_per_cta": (i, [P, ctypes.c_int32]),
        "gbfmm_batch_create": (i, [ctypes.POINTER(P), P, ctypes.c_int32, P, P, P, P, ctypes.c_int32]),
        "gbfmm_batch_launch": (i, [P, P]),
        "gbfmm_batch_info": (i, [P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(i64)]),
        "gbfmm_batch_destroy": (i, [P]),
        "gbfmm_evaluate_batch": (i, [P, ctypes.c_int32, P, P, P, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(ctx, rc):
    if rc != GBFMM_OK:
        msg = lib().gbfmm_last_error(ctx).decode() if ctx else ""
        raise GbfmmError(rc, msg)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _np_ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


# ---- same names as the C ABI ----------------------------------------------------------------

def gbfmm_version() -> int:
    return lib().gbfmm_version()


def gbfmm_default_params(**kw) -> gbfmm_params:
    prm = gbfmm_params()
    _check(None, lib().gbfmm_default_params(ctypes.byref(prm)))
    for k, v in kw.items():
        if k == "box_origin":
            prm.box_origin[:] = list(v)
        else:
            setattr(prm, k, v)
    return prm


def gbfmm_create(device: int = 0):
    ctx = ctypes.c_void_p()
    _check(None, lib().gbfmm_create(ctypes.byref(ctx), int(device)))
    return ctx


def gbfmm_destroy(ctx) -> None:
    lib().gbfmm_destroy(ctx)


def gbfmm_last_error(ctx) -> str:
    return lib().gbfmm_last_error(ctx).decode()


def gbfmm_plan(prm: gbfmm_params, n: int) -> tuple[int, int]:
    lv = ctypes.c_int32()
    ws = ctypes.c_size_t()
    _check(None, lib().gbfmm_plan(ctypes.byref(prm), int(n), ctypes.byref(lv), ctypes.byref(ws)))
    return lv.value, ws.value


def gbfmm_evaluate(ctx, prm: gbfmm_params, xyzq: torch.Tensor, out: torch.Tensor, workspace: torch.Tensor,
                   stream=None) -> None:
    n = xyzq.shape[0]
    assert xyzq.is_cuda and xyzq.dtype == torch.float32 and xyzq.is_contiguous() and xyzq.shape[1] == 4
    assert out.is_cuda and out.dtype == torch.float32 and out.is_contiguous() and out.shape == xyzq.shape
    _check(ctx, lib().gbfmm_evaluate(ctx, ctypes.byref(prm), n, _ptr(xyzq), _ptr(out), _ptr(workspace),
                                     workspace.numel() * workspace.element_size(), _stream(stream)))


def gbfmm_evaluate_host(ctx, prm: gbfmm_params, xyzq: torch.Tensor, out: torch.Tensor, stream=None) -> None:
    """xyzq, out: CPU float32 (n, 4) tensors (pinned for asynchronous copies)."""
    assert not xyzq.is_cuda and not out.is_cuda and xyzq.is_contiguous() and out.is_contiguous()
    _check(ctx, lib().gbfmm_evaluate_host(ctx, ctypes.byref(prm), xyzq.shape[0], _ptr(xyzq), _ptr(out),
                                          _stream(stream)))


def gbfmm_sync_status(ctx, stream=None) -> None:
    _check(ctx, lib().gbfmm_sync_status(ctx, _stream(stream)))


def gbfmm_direct(ctx, src: torch.Tensor, tgt: torch.Tensor, out: torch.Tensor, eps2: float = 0.0,
                 stream=None) -> None:
    _check(ctx, lib().gbfmm_direct(ctx, src.shape[0], _ptr(src), tgt.shape[0], _ptr(tgt), float(eps2), _ptr(out),
                                   _stream(stream)))


def gbfmm_export_tree(ctx, n: int, ncells: int) -> dict:
    import numpy as np

    os_ = np.zeros(4)
    keys = np.zeros(n, dtype=np.uint32)
    perm = np.zeros(n, dtype=np.uint32)
    begin = np.zeros(ncells, dtype=np.int32)
    count = np.zeros(ncells, dtype=np.int32)
    _check(ctx, lib().gbfmm_export_tree(ctx, _np_ptr(os_), _np_ptr(keys), _np_ptr(perm), _np_ptr(begin),
                                        _np_ptr(count)))
    return dict(origin=os_[:3].copy(), side=float(os_[3]), sorted_leaf_keys=keys, perm=perm, begin=begin,
                count=count)


def gbfmm_export_adaptive_tree(ctx, n: int) -> dict:
    import numpy as np

    nc = ctypes.c_int64()
    _check(ctx, lib().gbfmm_export_adaptive_tree(ctx, None, ctypes.byref(nc), None, None, None, None, None, None))
    c = nc.value
    os_ = np.zeros(4)
    level = np.zeros(c, dtype=np.int32)
    key = np.zeros(c, dtype=np.uint64)
    begin = np.zeros(c, dtype=np.int32)
    count = np.zeros(c, dtype=np.int32)
    parent = np.zeros(c, dtype=np.int32)
    perm = np.zeros(n, dtype=np.uint32)
    _check(ctx, lib().gbfmm_export_adaptive_tree(ctx, _np_ptr(os_), ctypes.byref(nc), _np_ptr(level), _np_ptr(key),
                                                 _np_ptr(begin), _np_ptr(count), _np_ptr(parent), _np_ptr(perm)))
    return dict(origin=os_[:3].copy(), side=float(os_[3]), ncells=c, level=level, key=key, begin=begin,
                count=count, parent=parent, perm=perm)


def gbfmm_export_lists(ctx, kind: int, rows: int) -> tuple:
    import numpy as np

    ne = ctypes.c_int64()
    offs = np.zeros(rows + 1, dtype=np.int32)
    _check(ctx, lib().gbfmm_export_lists(ctx, kind, _np_ptr(offs), None, 0, ctypes.byref(ne)))
    ids = np.zeros(max(1, ne.value), dtype=np.int32)
    _check(ctx, lib().gbfmm_export_lists(ctx, kind, _np_ptr(offs), _np_ptr(ids), len(ids), ctypes.byref(ne)))
    return offs, ids[: ne.value]


def gbfmm_export_expansions(ctx, which: int, ncells: int, p: int):
    import numpy as np

    nt = p * (p + 1) // 2
    buf = np.zeros(ncells * 2 * nt)
    _check(ctx, lib().gbfmm_export_expansions(ctx, which, _np_ptr(buf)))
    return (buf[0::2] + 1j * buf[1::2]).reshape(ncells, nt)


def gbfmm_stage_times(ctx) -> dict:
    import numpy as np

    ms = np.zeros(len(STAGES), dtype=np.float32)
    cnt = ctypes.c_int()
    _check(ctx, lib().gbfmm_stage_times(ctx, _np_ptr(ms), len(STAGES), ctypes.byref(cnt)))
    return {STAGES[i]: float(ms[i]) for i in range(cnt.value)}


def gbfmm_last_launch_count(ctx) -> int:
    c = ctypes.c_int64()
    _check(ctx, lib().gbfmm_last_launch_count(ctx, ctypes.byref(c)))
    return c.value


def gbfmm_selftest_wait(ctx, limit_ms: float, stream=None) -> None:
    _check(ctx, lib().gbfmm_selftest_wait(ctx, float(limit_ms), _stream(stream)))


def gbfmm_sort_static(prm: gbfmm_params, xyzq: torch.Tensor, sorted_xyzq: torch.Tensor, perm: torch.Tensor,
                      sorted_leaf_keys: torch.Tensor, status: torch.Tensor = None, stream=None) -> None:
    """Allocation-free Morton sort (library-owned static scratch; see include/gbfmm.h).

    `status`, if given, is a one-element int32 device tensor the call clears and its kernels
    raise (1: non-finite coordinate, 2: a bounded wait gave up)."""
    assert perm.dtype == torch.int32 and sorted_leaf_keys.dtype == torch.int32  # uint32 bit patterns
    assert status is None or (status.dtype == torch.int32 and status.numel() >= 1)
    _check(None, lib().gbfmm_sort_static(ctypes.byref(prm), xyzq.shape[0], _ptr(xyzq), _ptr(sorted_xyzq),
                                         _ptr(perm), _ptr(sorted_leaf_keys),
                                         _ptr(status), _stream(stream)))


def gbfmm_engine_create(device: int = 0, workers: int = 4, memory_budget_bytes: int = 40 << 30):
    e = ctypes.c_void_p()
    _check(None, lib().gbfmm_engine_create(ctypes.byref(e), int(device), int(workers), int(memory_budget_bytes)))
    return e


def gbfmm_engine_destroy(e) -> None:
    lib().gbfmm_engine_destroy(e)


def gbfmm_engine_prepare(e, orders) -> None:
    import numpy as np

    o = np.ascontiguousarray(orders, dtype=np.int32)
    _check(None, lib().gbfmm_engine_prepare(e, _np_ptr(o), len(o)))


def gbfmm_engine_submit(e, prm: gbfmm_params, h_xyzq, h_out) -> int:
    """h_xyzq, h_out: host float32 (n, 4) arrays (numpy or CPU tensors) kept alive by the caller
    until gbfmm_engine_wait returns for the ticket."""
    t = ctypes.c_int64()
    ptr_in = h_xyzq.ctypes.data_as(ctypes.c_void_p) if hasattr(h_xyzq, "ctypes") else _ptr(h_xyzq)
    ptr_out = h_out.ctypes.data_as(ctypes.c_void_p) if hasattr(h_out, "ctypes") else _ptr(h_out)
    _check(None, lib().gbfmm_engine_submit(e, ctypes.byref(prm), int(h_xyzq.shape[0]), ptr_in, ptr_out,
                                           ctypes.byref(t)))
    return t.value


def gbfmm_engine_wait(e, ticket: int, timeout_ms: float = 60000.0):
    """Returns (status, queue_ms, latency_ms); raises GbfmmError(ETIMEOUT) if not done in time."""
    st, q, lat = ctypes.c_int32(), ctypes.c_double(), ctypes.c_double()
    _check(None, lib().gbfmm_engine_wait(e, int(ticket), float(timeout_ms), ctypes.byref(st), ctypes.byref(q),
                                         ctypes.byref(lat)))
    return st.value, q.value, lat.value


def gbfmm_engine_run_batch(e, offsets, params, xyzq: torch.Tensor, out: torch.Tensor):
    """offsets: nb + 1 ascending particle offsets; params: list of gbfmm_params; xyzq, out:
    device float32 (total, 4) tensors.  Returns the per-instance status list."""
    import numpy as np

    nb = len(params)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    assert len(off) == nb + 1
    arr = (gbfmm_params * max(nb, 1))(*params)
    st = np.zeros(max(nb, 1), dtype=np.int32)
    rc = lib().gbfmm_engine_run_batch(e, nb, _np_ptr(off), ctypes.cast(arr, ctypes.c_void_p), _ptr(xyzq), _ptr(out),
                                      _np_ptr(st))
    if rc != GBFMM_OK:
        raise GbfmmError(rc, "batch")
    return st[:nb].tolist()


def gbfmm_graph_create(ctx, prm: gbfmm_params, xyzq: torch.Tensor, out: torch.Tensor, workspace: torch.Tensor):
    """Captures one uniform-tree evaluation of these buffers into a CUDA graph; returns its handle."""
    assert xyzq.is_cuda and out.is_cuda and xyzq.shape == out.shape
    g = ctypes.c_void_p()
    _check(ctx, lib().gbfmm_graph_create(ctypes.byref(g), ctx, ctypes.byref(prm), xyzq.shape[0], _ptr(xyzq), _ptr(out),
                                         _ptr(workspace), workspace.numel() * workspace.element_size()))
    return g


def gbfmm_graph_launch(g, stream=None) -> None:
    rc = lib().gbfmm_graph_launch(g, _stream(stream))
    if rc != GBFMM_OK:
        raise GbfmmError(rc, "graph launch")


def gbfmm_graph_destroy(g) -> None:
    lib().gbfmm_graph_destroy(g)


def _batch_args(offsets, params):
    import numpy as np

    nb = len(params)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    assert len(off) == nb + 1
    arr = (gbfmm_params * max(nb, 1))(*params)
    return nb, off, arr


def gbfmm_batch_create(ctx, offsets, params, xyzq: torch.Tensor, out: torch.Tensor, lanes: int = 16):
    """Captures the batch (instance i: rows offsets[i]:offsets[i+1] of the device (total, 4)
    tensors, parameters params[i]) into one CUDA graph; returns its handle."""
    assert xyzq.is_cuda and out.is_cuda and xyzq.shape == out.shape
    nb, off, arr = _batch_args(offsets, params)
    b = ctypes.c_void_p()
    _check(ctx, lib().gbfmm_batch_create(ctypes.byref(b), ctx, nb, _np_ptr(off), ctypes.cast(arr, ctypes.c_void_p),
                                         _ptr(xyzq), _ptr(out), lanes))
    return b


def gbfmm_batch_launch(ctx, b, stream=None) -> None:
    _check(ctx, lib().gbfmm_batch_launch(b, _stream(stream)))


def gbfmm_batch_info(b) -> tuple:
    """(lanes, kernel nodes of the graph)."""
    lanes = ctypes.c_int32()
    nodes = ctypes.c_int64()
    rc = lib().gbfmm_batch_info(b, ctypes.byref(lanes), ctypes.byref(nodes))
    if rc != GBFMM_OK:
        raise GbfmmError(rc, "batch info")
    return int(lanes.value), int(nodes.value)


def gbfmm_batch_destroy(b) -> None:
    lib().gbfmm_batch_destroy(b)


def gbfmm_evaluate_batch(ctx, offsets, params, xyzq: torch.Tensor, out: torch.Tensor, stream=None) -> None:
    """The batch through the graph the context keeps (captured at the first call with these
    arguments, replayed after)."""
    assert xyzq.is_cuda and out.is_cuda and xyzq.shape == out.shape
    nb, off, arr = _batch_args(offsets, params)
    _check(ctx, lib().gbfmm_evaluate_batch(ctx, nb, _np_ptr(off), ctypes.cast(arr, ctypes.c_void_p), _ptr(xyzq),
                                           _ptr(out), _stream(stream)))


def gbfmm_tune_leaf(ctx, prm: gbfmm_params, xyzq: torch.Tensor, candidates) -> tuple:
    """Leaf-size autotuner: (fastest candidate, its evaluation time in ms)."""
    import numpy as np

    assert xyzq.is_cuda and xyzq.dtype == torch.float32 and xyzq.is_contiguous()
    c = np.ascontiguousarray(candidates, dtype=np.int32)
    best = ctypes.c_int32()
    ms = ctypes.c_float()
    _check(ctx, lib().gbfmm_tune_leaf(ctx, ctypes.byref(prm), xyzq.shape[0], _ptr(xyzq), _np_ptr(c), len(c),
                                      ctypes.byref(best), ctypes.byref(ms)))
    return int(best.value), float(ms.value)


def gbfmm_tune(ctx, prm: gbfmm_params, xyzq: torch.Tensor, leaf_candidates, lpc_candidates) -> tuple:
    """Autotuner over leaf size x P2P launch shape (target leaves per P2P CTA): (leaf, leaves per
    CTA, ms) of the fastest pair; the context keeps that launch shape."""
    import numpy as np

    assert xyzq.is_cuda and xyzq.dtype == torch.float32 and xyzq.is_contiguous()
    c = np.ascontiguousarray(leaf_candidates, dtype=np.int32)
    d = np.ascontiguousarray(lpc_candidates, dtype=np.int32)
    leaf, lpc, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
    _check(ctx, lib().gbfmm_tune(ctx, ctypes.byref(prm), xyzq.shape[0], _ptr(xyzq), _np_ptr(c), len(c),
                                 _np_ptr(d) if len(d) else None, len(d), ctypes.byref(leaf), ctypes.byref(lpc),
                                 ctypes.byref(ms)))
    return int(leaf.value), int(lpc.value), float(ms.value)


def gbfmm_set_p2p_leaves_per_cta(ctx, leaves: int) -> None:
    """The context's P2P launch shape: about `leaves` target leaves per CTA (0: the library's)."""
    _check(ctx, lib().gbfmm_set_p2p_leaves_per_cta(ctx, int(leaves)))


# ---- convenience wrapper (torch-allocated workspace) -----------------------------------------

def level_offset(l: int) -> int:
    return (8 ** l - 1) // 7


class FMM:
    """Owns a context and a torch-allocated workspace; evaluate() runs on the current stream."""

    def __init__(self, device: int = 0, **params):
        self.device = device
        self.ctx = gbfmm_create(device)
        self.params = gbfmm_default_params(**params)
        self.workspace = None

    def close(self):
        if self.ctx:
            gbfmm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def plan(self, n: int):
        return gbfmm_plan(self.params, n)

    def ensure_workspace(self, n: int) -> torch.Tensor:
        _, ws = gbfmm_plan(self.params, n)  # 0 for the adaptive tree (library-owned buffers)
        if self.workspace is None or self.workspace.numel() < ws:
            self.workspace = torch.empty(max(ws, 256), dtype=torch.uint8, device=f"cuda:{self.device}")
        return self.workspace

    def evaluate(self, xyzq: torch.Tensor, out: torch.Tensor | None = None, check: bool = True) -> torch.Tensor:
        if out is None:
            out = torch.empty_like(xyzq)
        ws = self.ensure_workspace(xyzq.shape[0])
        gbfmm_evaluate(self.ctx, self.params, xyzq, out, ws)
        if check:
            gbfmm_sync_status(self.ctx)
        return out
