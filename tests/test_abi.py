"""C-ABI checks that need no GPU: the library loads, exports every symbol the header
declares, and rejects bad parameters in planning."""
import ctypes

import pytest

import oracle as O
from paper_1010_1482_gb300 import build as cuda_build
from paper_1010_1482_gb300 import gbfmm as G


@pytest.fixture(scope="module")
def lib():
    cuda_build.build()
    return G.lib()


def test_exports_every_declared_symbol(lib):
    names = G.declared_symbols()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name
    assert G.gbfmm_version() == 1


def test_default_params_and_plan(lib):
    prm = G.gbfmm_default_params()
    assert (prm.p, prm.leaf_size, prm.method, prm.eps2) == (10, 64, 0, 0.0)
    L, ws = G.gbfmm_plan(prm, 1 << 20)
    assert L == O.uniform_depth(1 << 20, 64) == 5
    assert ws > (1 << 20) * 64
    for n, leaf in [(4096, 64), (1, 64), (0, 64), (512, 64), (513, 64), (100000, 7)]:
        prm = G.gbfmm_default_params(p=4, leaf_size=leaf)
        assert G.gbfmm_plan(prm, n)[0] == O.uniform_depth(n, leaf)


@pytest.mark.parametrize("kw,code", [
    (dict(p=5), G.GBFMM_EUNSUPPORTED),
    (dict(p=12), G.GBFMM_EUNSUPPORTED),
    (dict(leaf_size=0), G.GBFMM_EINVAL),
    (dict(method=7), G.GBFMM_EINVAL),
    (dict(eps2=-1.0), G.GBFMM_EINVAL),
    (dict(has_box=1, box_side=0.0), G.GBFMM_EINVAL),
    (dict(leaf_size=1), G.GBFMM_EUNSUPPORTED),  # depth > 10 for n = 2^31 - 1
])
def test_plan_rejects_bad_parameters(lib, kw, code):
    prm = G.gbfmm_default_params(**kw)
    with pytest.raises(G.GbfmmError) as ei:
        G.gbfmm_plan(prm, (1 << 31) - 1 if kw.get("leaf_size") == 1 else 1000)
    assert ei.value.code == code


def test_negative_n_and_null_context(lib):
    prm = G.gbfmm_default_params()
    with pytest.raises(G.GbfmmError):
        G.gbfmm_plan(prm, -1)
    assert lib.gbfmm_evaluate(None, ctypes.byref(prm), 10, None, None, None, 0, None) == G.GBFMM_EINVAL
    assert lib.gbfmm_destroy(None) == G.GBFMM_OK
    assert lib.gbfmm_set_p2p_leaves_per_cta(None, 4) == G.GBFMM_EINVAL
    assert lib.gbfmm_tune(None, ctypes.byref(prm), 10, None, None, 0, None, 0, None, None, None) == G.GBFMM_EINVAL


def test_workspace_grows_linearly(lib):
    prm = G.gbfmm_default_params(p=10, leaf_size=64)
    _, a = G.gbfmm_plan(prm, 1 << 20)
    _, b = G.gbfmm_plan(prm, 1 << 23)
    assert 6 < b / a < 10


def test_header_constants_match_binding():
    """Every enumerator and GBFMM_FLAG_* macro of the header has the value the Python binding
    uses (GBFMM_X in the header is X in the binding, error codes keep their prefix)."""
    import os
    import re

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    text = open(os.path.join(root, "include", "gbfmm.h")).read()
    consts = {m.group(1): int(m.group(2)) for m in re.finditer(r"^#define (GBFMM_FLAG_\w+)\s+(\d+)", text, re.M)}
    consts.update({m.group(1): int(m.group(2)) for m in re.finditer(r"\b(GBFMM_[A-Z0-9_]+)\s*=\s*(\d+)", text)})
    assert {"GBFMM_FLAG_STAGE_TIMING", "GBFMM_FLAG_M2L_CUDA_CORES", "GBFMM_FLAG_SERIAL", "GBFMM_OK",
            "GBFMM_LIST_X", "GBFMM_TREE_ADAPTIVE", "GBFMM_METHOD_TREECODE"} <= set(consts)
    for name, value in consts.items():
        py = name if (name == "GBFMM_OK" or name.startswith("GBFMM_E")) else name[len("GBFMM_"):]
        assert getattr(G, py) == value, name


def test_sort_static_rejects_before_any_launch(lib):
    """The allocation-free sort refuses, on the host and before any CUDA call, what its static
    scratch cannot hold (the adaptive tree's 63-bit keys, n > 2^20) and outputs that share
    bytes with its input or with each other.  The pointers are never dereferenced."""
    P = ctypes.c_void_p
    f = lib.gbfmm_sort_static
    n = 4096
    a, b, c, d, s = 1 << 20, 2 << 20, 3 << 20, 4 << 20, 5 << 20  # disjoint, aligned, never touched
    adaptive = G.gbfmm_default_params(p=4, leaf_size=64, tree=G.TREE_ADAPTIVE)
    assert f(ctypes.byref(adaptive), n, P(a), P(b), P(c), P(d), P(s), None) == G.GBFMM_EUNSUPPORTED
    uniform = G.gbfmm_default_params(p=4, leaf_size=64)
    assert f(ctypes.byref(uniform), (1 << 20) + 1, P(a), P(b), P(c), P(d), None, None) == G.GBFMM_EUNSUPPORTED
    for bad in [(a, a, c, d, s), (a, a + 16 * n - 16, c, d, s), (a, b, c, c, s), (a, b, c, d, d + 8),
                (a, b, a + 64, d, s), (a, b, c, b + 4 * n, s)]:
        assert f(ctypes.byref(uniform), n, *map(P, bad), None) == G.GBFMM_EINVAL, bad
    assert f(ctypes.byref(uniform), n, P(a), P(b), P(c + 2), P(d), None, None) == G.GBFMM_EINVAL  # misaligned
    assert f(None, n, P(a), P(b), P(c), P(d), None, None) == G.GBFMM_EINVAL
    assert f(ctypes.byref(uniform), -1, P(a), P(b), P(c), P(d), None, None) == G.GBFMM_EINVAL
