"""FP64 CPU oracle for the Laplace treecode / FMM (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference legs
may import this package.  It shares no code with the CUDA path and the CUDA path
never calls it.

The arithmetic lives in fmm_oracle.c (plain C, FP64, built with
-ffp-contract=off so that the key quantisation is the exact IEEE sequence); this
module compiles it with gcc on first use, marshals numpy arrays, and orchestrates
the stages in the order of the paper's Fig. 1 flow: root box -> Morton keys ->
sort -> cells -> interaction lists -> P2M, M2M, M2L (or M2P), L2L, L2P, P2P.
The sort is numpy's stable lexsort (a library primitive used as one step).

Parity unpinned: nothing here; every function is pinned by tests/test_oracle_*.py
against closed forms, library routines, invariants or brute force.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fmm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libfmm_oracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile fmm_oracle.c into _build/libfmm_oracle.so (atomic replace)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_BUILD)
    os.close(fd)
    cmd = ["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.c_void_p
            i64 = ctypes.c_int64
            d = ctypes.c_double
            ci = ctypes.c_int
            sig = {
                "orc_version": (ci, []),
                "orc_threads": (ci, []),
                "orc_legendre": (None, [ci, d, P]),
                "orc_ynm_ri": (None, [ci, d, d, P]),
                "orc_direct": (None, [i64, P, i64, P, d, P]),
                "orc_p2m_ri": (None, [ci, P, i64, P, P]),
                "orc_m2p_ri": (None, [ci, P, P, P, P]),
                "orc_l2p_ri": (None, [ci, P, P, P, P]),
                "orc_m2l_ri": (None, [ci, P, P, P, P]),
                "orc_m2m_ri": (None, [ci, P, P, P, P]),
                "orc_l2l_ri": (None, [ci, P, P, P, P]),
                "orc_root_box": (ci, [i64, P, P, P]),
                "orc_keys": (None, [i64, P, P, d, P]),
                "orc_key_decode": (None, [ctypes.c_uint64, ci, P]),
                "orc_cell_centre": (None, [P, d, ci, ctypes.c_uint64, P]),
                "orc_cells": (None, [ci, i64, P, P, P]),
                "orc_list_p2p": (i64, [ci, P, P, P]),
                "orc_list_m2l": (i64, [ci, P, P, P]),
                "orc_fmm_passes": (ci, [ci, ci, ci, d, P, d, i64, P, P, P, P, P, P, P, P, P, P, P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def threads() -> int:
    """OpenMP threads the oracle's parallel loops use."""
    return int(lib().orc_threads())


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ----------------------------------------------------------------------------
# Special functions and single operators (complex coefficients, m >= 0 stored)
# ----------------------------------------------------------------------------

def ntri(p: int) -> int:
    return p * (p + 1) // 2


def tri(n: int, m: int) -> int:
    return n * (n + 1) // 2 + m


def legendre(nmax: int, x: float) -> np.ndarray:
    """P_n^m(x) (Eq. 7-9, Condon-Shortley phase), triangular array."""
    out = np.zeros(ntri(nmax))
    lib().orc_legendre(nmax, float(x), _p(out))
    return out


def ynm(nmax: int, alpha: float, beta: float) -> np.ndarray:
    """Y_n^m(alpha, beta), m >= 0 (Eq. 6), complex triangular array."""
    ri = np.zeros(2 * ntri(nmax))
    lib().orc_ynm_ri(nmax, float(alpha), float(beta), _p(ri))
    return ri[0::2] + 1j * ri[1::2]


def _cri(c: np.ndarray) -> np.ndarray:
    out = np.empty(2 * len(c))
    out[0::2] = np.real(c)
    out[1::2] = np.imag(c)
    return out


def _ric(ri: np.ndarray) -> np.ndarray:
    return ri[0::2] + 1j * ri[1::2]


def p2m(p: int, centre, xyzq) -> np.ndarray:
    xyzq = _c(xyzq, np.float64).reshape(-1, 4)
    ri = np.zeros(2 * ntri(p))
    lib().orc_p2m_ri(p, _p(_c(centre, np.float64)), len(xyzq), _p(xyzq), _p(ri))
    return _ric(ri)


def m2p(p: int, centre, M, x) -> np.ndarray:
    out = np.zeros(4)
    lib().orc_m2p_ri(p, _p(_c(centre, np.float64)), _p(_cri(np.asarray(M))), _p(_c(x, np.float64)), _p(out))
    return out


def l2p(p: int, centre, Lc, x) -> np.ndarray:
    out = np.zeros(4)
    lib().orc_l2p_ri(p, _p(_c(centre, np.float64)), _p(_cri(np.asarray(Lc))), _p(_c(x, np.float64)), _p(out))
    return out


def m2l(p: int, src_centre, tgt_centre, M) -> np.ndarray:
    ri = np.zeros(2 * ntri(p))
    lib().orc_m2l_ri(p, _p(_c(src_centre, np.float64)), _p(_c(tgt_centre, np.float64)), _p(_cri(np.asarray(M))), _p(ri))
    return _ric(ri)


def m2m(p: int, child_centre, parent_centre, M) -> np.ndarray:
    ri = np.zeros(2 * ntri(p))
    lib().orc_m2m_ri(p, _p(_c(child_centre, np.float64)), _p(_c(parent_centre, np.float64)), _p(_cri(np.asarray(M))), _p(ri))
    return _ric(ri)


def l2l(p: int, parent_centre, child_centre, Lp) -> np.ndarray:
    ri = np.zeros(2 * ntri(p))
    lib().orc_l2l_ri(p, _p(_c(parent_centre, np.float64)), _p(_c(child_centre, np.float64)), _p(_cri(np.asarray(Lp))), _p(ri))
    return _ric(ri)


# ----------------------------------------------------------------------------
# Direct sum
# ----------------------------------------------------------------------------

def direct(xyzq, targets=None, eps2: float = 0.0) -> np.ndarray:
    """Eq. 1 by the O(N^2) sum in FP64: (phi, dphi/dx, dphi/dy, dphi/dz) per target.

    targets: optional index array into xyzq (defaults to all particles)."""
    src = _c(xyzq, np.float64).reshape(-1, 4)
    idx = np.arange(len(src)) if targets is None else np.asarray(targets)
    tgt = _c(src[idx, :3], np.float64)
    out = np.zeros((len(idx), 4))
    lib().orc_direct(len(idx), _p(tgt), len(src), _p(src), float(eps2), _p(out))
    return out


# ----------------------------------------------------------------------------
# Tree, keys, lists
# ----------------------------------------------------------------------------

MAX_LEVEL = 8


def uniform_depth(n: int, leaf_size: int) -> int:
    """Smallest L >= 0 with n <= leaf_size * 8^L (mean leaf occupancy <= leaf_size)."""
    L = 0
    while n > leaf_size * (8 ** L):
        L += 1
    return L


def level_offset(l: int) -> int:
    return (8 ** l - 1) // 7


def root_box(xyzq):
    xyzq = _c(xyzq, np.float32).reshape(-1, 4)
    origin = np.zeros(3)
    side = np.zeros(1)
    bad = lib().orc_root_box(len(xyzq), _p(xyzq), _p(origin), _p(side))
    return origin, float(side[0]), int(bad)


def morton_keys(xyzq, origin, side) -> np.ndarray:
    xyzq = _c(xyzq, np.float32).reshape(-1, 4)
    keys = np.zeros(len(xyzq), dtype=np.uint64)
    lib().orc_keys(len(xyzq), _p(xyzq), _p(_c(origin, np.float64)), float(side), _p(keys))
    return keys


def key_decode(key: int, bits: int):
    out = np.zeros(3, dtype=np.int64)
    lib().orc_key_decode(int(key), bits, _p(out))
    return out


def cell_centre(origin, side, level: int, key: int) -> np.ndarray:
    out = np.zeros(3)
    lib().orc_cell_centre(_p(_c(origin, np.float64)), float(side), level, int(key), _p(out))
    return out


def build_tree(xyzq, leaf_size: int, level: int | None = None) -> dict:
    """Uniform octree: root box, 63-bit keys, leaf level L, permutation sorting the
    particles by (leaf key, original index), and dense per-level cell ranges."""
    xyzq = _c(xyzq, np.float32).reshape(-1, 4)
    n = len(xyzq)
    origin, side, bad = root_box(xyzq)
    L = uniform_depth(n, leaf_size) if level is None else level
    if L > MAX_LEVEL:
        raise ValueError(f"oracle tree depth {L} exceeds {MAX_LEVEL}")
    keys = morton_keys(xyzq, origin, side)
    leaf = keys >> np.uint64(3 * (21 - L))
    perm = np.lexsort((np.arange(n), leaf)).astype(np.int64)  # ascending (leaf key, index)
    sleaf = np.ascontiguousarray(leaf[perm])
    C = level_offset(L + 1)
    begin = np.zeros(C, dtype=np.int32)
    count = np.zeros(C, dtype=np.int32)
    lib().orc_cells(L, n, _p(sleaf), _p(begin), _p(count))
    return dict(n=n, L=L, origin=origin, side=side, bad=bad, keys=keys, leaf_keys=leaf,
                perm=perm, sorted_leaf_keys=sleaf, begin=begin, count=count)


def build_lists(tree: dict) -> dict:
    L = tree["L"]
    count = tree["count"]
    nl = 8 ** L
    C = level_offset(L + 1)
    p2p_offs = np.zeros(nl + 1, dtype=np.int32)
    p2p_ids = np.zeros(27 * nl, dtype=np.int32)
    e1 = lib().orc_list_p2p(L, _p(count), _p(p2p_offs), _p(p2p_ids))
    m2l_offs = np.zeros(C + 1, dtype=np.int32)
    m2l_ids = np.zeros(max(1, 189 * C), dtype=np.int32)
    e2 = lib().orc_list_m2l(L, _p(count), _p(m2l_offs), _p(m2l_ids))
    return dict(p2p_offs=p2p_offs, p2p_ids=p2p_ids[:e1].copy(), m2l_offs=m2l_offs, m2l_ids=m2l_ids[:e2].copy())


# ----------------------------------------------------------------------------
# Whole evaluation
# ----------------------------------------------------------------------------

FMM, TREECODE = 0, 1


def fmm(xyzq, p: int, leaf_size: int, method: int = FMM, eps2: float = 0.0, targets=None,
        level: int | None = None, keep: bool = False) -> dict:
    """FP64 FMM (method=0) or treecode (method=1) on the uniform tree.

    Returns dict with 'out' = (n, 4) (phi, grad) in original particle order.
    targets: optional particle indices; when given, only the leaves holding them
    are evaluated (the rows of 'out' for other particles are zero).
    keep: also return the tree, lists and the complex M / L of every cell."""
    xyzq32 = _c(xyzq, np.float32).reshape(-1, 4)
    n = len(xyzq32)
    tree = build_tree(xyzq32, leaf_size, level)
    lists = build_lists(tree)
    L = tree["L"]
    nt = ntri(p)
    C = level_offset(L + 1)
    sx = _c(xyzq32[tree["perm"]].astype(np.float64), np.float64)
    M = np.zeros(2 * C * nt)
    Lc = np.zeros(2 * C * nt)
    out_s = np.zeros((n, 4))
    need = None
    if targets is not None:
        need = np.zeros(8 ** L, dtype=np.uint8)
        need[tree["leaf_keys"][np.asarray(targets)].astype(np.int64)] = 1
    rc = lib().orc_fmm_passes(
        p, L, method, float(eps2), _p(tree["origin"]), float(tree["side"]), n, _p(sx),
        _p(tree["begin"]), _p(tree["count"]), _p(lists["p2p_offs"]), _p(lists["p2p_ids"]),
        _p(lists["m2l_offs"]), _p(lists["m2l_ids"]), _p(need) if need is not None else None,
        _p(M), _p(Lc), _p(out_s))
    if rc != 0:
        raise MemoryError("oracle passes failed")
    out = np.zeros((n, 4))
    out[tree["perm"]] = out_s
    res = dict(out=out, L=L)
    if keep:
        res.update(tree=tree, lists=lists, M=(M[0::2] + 1j * M[1::2]).reshape(C, nt),
                   Lc=(Lc[0::2] + 1j * Lc[1::2]).reshape(C, nt))
    return res


def rel_l2(a: np.ndarray, ref: np.ndarray) -> float:
    """Normalised L2 error sqrt(sum |a - ref|^2 / sum |ref|^2) (the paper's force error norm)."""
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = float(np.sum(ref * ref))
    return float(np.sqrt(np.sum((a - ref) ** 2) / den)) if den > 0 else float(np.sqrt(np.sum((a - ref) ** 2)))


# ----------------------------------------------------------------------------
# Adaptive tree (cells split while they hold more than leaf_size particles)
# ----------------------------------------------------------------------------

ADAPTIVE_MAX_LEVEL = 21
LIST_U, LIST_V, LIST_W, LIST_X = 0, 1, 2, 3


def _adaptive_sigs():
    L = lib()
    P = ctypes.c_void_p
    i64 = ctypes.c_int64
    ci = ctypes.c_int
    d = ctypes.c_double
    if getattr(L, "_adaptive_ready", False):
        return L
    for name, res, args in (
        ("orc_adaptive_tree", i64, [i64, P, ci, ci, i64, P, P, P, P, P, P, P, P]),
        ("orc_adaptive_colleagues", None, [i64, P, P, P, P, P, P]),
        ("orc_adaptive_list", i64, [ci, i64, P, P, P, P, P, P, P, P, i64]),
        ("orc_adaptive_passes", ci, [ci, ci, d, P, d, i64, P, P, P, P, P, P, P, P, ci, P, P, P, P, P, P, P, P, P, P,
                                     P, P, P]),
        ("orc_p2l_ri", None, [ci, P, i64, P, P]),
    ):
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    L._adaptive_ready = True
    return L


def p2l(p: int, centre, xyzq) -> np.ndarray:
    """Eq. 3's L_n^m of a set of charges about `centre` (P2L)."""
    L = _adaptive_sigs()
    xyzq = _c(xyzq, np.float64).reshape(-1, 4)
    ri = np.zeros(2 * ntri(p))
    L.orc_p2l_ri(p, _p(_c(centre, np.float64)), len(xyzq), _p(xyzq), _p(ri))
    return _ric(ri)


def build_adaptive_tree(xyzq, leaf_size: int, max_level: int = ADAPTIVE_MAX_LEVEL) -> dict:
    """Adaptive octree over the root cube: particles sorted by (63-bit key, index); a cell
    splits while it holds more than leaf_size particles and is above max_level."""
    L = _adaptive_sigs()
    xyzq = _c(xyzq, np.float32).reshape(-1, 4)
    n = len(xyzq)
    origin, side, bad = root_box(xyzq)
    keys = morton_keys(xyzq, origin, side)
    perm = np.lexsort((np.arange(n), keys)).astype(np.int64)
    sk = np.ascontiguousarray(keys[perm])
    cap = 4 * n + 64
    while True:
        a = {k: np.zeros(cap, dtype=np.int32) for k in ("level", "begin", "count", "parent", "child_begin", "nchild")}
        key = np.zeros(cap, dtype=np.uint64)
        ls = np.zeros(max_level + 2, dtype=np.int32)
        nc = L.orc_adaptive_tree(n, _p(sk), leaf_size, max_level, cap, _p(a["level"]), _p(key), _p(a["begin"]),
                                 _p(a["count"]), _p(a["parent"]), _p(a["child_begin"]), _p(a["nchild"]), _p(ls))
        if nc >= 0:
            break
        cap *= 2
    t = {k: v[:nc].copy() for k, v in a.items()}
    t.update(n=n, ncells=int(nc), key=key[:nc].copy(), level_start=ls, origin=origin, side=side, bad=bad,
             keys=keys, perm=perm, sorted_keys=sk, max_level=max_level)
    coll = np.zeros(27 * max(nc, 1), dtype=np.int32)
    L.orc_adaptive_colleagues(nc, _p(t["level"]), _p(t["key"]), _p(t["parent"]), _p(t["child_begin"]),
                              _p(t["nchild"]), _p(coll))
    t["colleagues"] = coll.reshape(-1, 27)[:nc]
    return t


def build_adaptive_lists(tree: dict) -> dict:
    L = _adaptive_sigs()
    nc = tree["ncells"]
    coll = np.ascontiguousarray(tree["colleagues"].reshape(-1))
    out = {}
    for kind, name in ((LIST_U, "u"), (LIST_V, "v"), (LIST_W, "w"), (LIST_X, "x")):
        cap = 64 * nc + 64
        while True:
            offs = np.zeros(nc + 1, dtype=np.int32)
            ids = np.zeros(cap, dtype=np.int32)
            e = L.orc_adaptive_list(kind, nc, _p(tree["level"]), _p(tree["key"]), _p(tree["parent"]),
                                    _p(tree["child_begin"]), _p(tree["nchild"]), _p(coll), _p(offs), _p(ids), cap)
            if e >= 0:
                break
            cap *= 4
        out[name + "_offs"] = offs
        out[name + "_ids"] = ids[:e].copy()
    return out


def fmm_adaptive(xyzq, p: int, leaf_size: int, eps2: float = 0.0, targets=None, keep: bool = False,
                 max_level: int = ADAPTIVE_MAX_LEVEL, method: int = FMM) -> dict:
    """FP64 adaptive FMM (method=FMM): U (P2P), V (M2L), W (M2P), X (P2L) lists; or the
    adaptive treecode (method=TREECODE): M2P over W and over V of the leaf and its ancestors,
    P2P over U and over X of the leaf and its ancestors.  Returns 'out' (n, 4) in original
    order; with `targets`, only the leaves holding them are evaluated."""
    L = _adaptive_sigs()
    xyzq32 = _c(xyzq, np.float32).reshape(-1, 4)
    n = len(xyzq32)
    t = build_adaptive_tree(xyzq32, leaf_size, max_level)
    ls = build_adaptive_lists(t)
    nc = t["ncells"]
    nt = ntri(p)
    sx = _c(xyzq32[t["perm"]].astype(np.float64), np.float64)
    M = np.zeros(2 * nc * nt)
    Lc = np.zeros(2 * nc * nt)
    out_s = np.zeros((n, 4))
    need = None
    if targets is not None:
        need = np.zeros(nc, dtype=np.uint8)
        leaf_of = leaf_of_sorted(t)
        inv = np.empty(n, dtype=np.int64)
        inv[t["perm"]] = np.arange(n)
        need[leaf_of[inv[np.asarray(targets)]]] = 1
    rc = L.orc_adaptive_passes(
        p, int(method), float(eps2), _p(t["origin"]), float(t["side"]), nc, _p(t["level"]), _p(t["key"]), _p(t["begin"]),
        _p(t["count"]), _p(t["parent"]), _p(t["child_begin"]), _p(t["nchild"]), _p(t["level_start"]),
        max_level, _p(sx), _p(ls["u_offs"]), _p(ls["u_ids"]), _p(ls["v_offs"]), _p(ls["v_ids"]),
        _p(ls["w_offs"]), _p(ls["w_ids"]), _p(ls["x_offs"]), _p(ls["x_ids"]),
        _p(need) if need is not None else None, _p(M), _p(Lc), _p(out_s))
    if rc != 0:
        raise MemoryError("oracle adaptive passes failed")
    out = np.zeros((n, 4))
    out[t["perm"]] = out_s
    res = dict(out=out, tree=t)
    if keep:
        res.update(lists=ls, M=(M[0::2] + 1j * M[1::2]).reshape(nc, nt), Lc=(Lc[0::2] + 1j * Lc[1::2]).reshape(nc, nt))
    return res


def leaf_of_sorted(tree: dict) -> np.ndarray:
    """Leaf cell index of every sorted particle position."""
    leaf_of = np.zeros(tree["n"], dtype=np.int64)
    leaves = np.nonzero(tree["nchild"] == 0)[0]
    for c in leaves:
        leaf_of[tree["begin"][c]: tree["begin"][c] + tree["count"][c]] = c
    return leaf_of
