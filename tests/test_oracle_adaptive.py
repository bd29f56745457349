"""Pins of the oracle's adaptive octree, U/V/W/X lists, P2L and adaptive passes."""
import numpy as np
import pytest

import oracle as O
from paper_1010_1482_gb300 import inputs


def _subtree_particles(t, c):
    return t["begin"][c], t["begin"][c] + t["count"][c]


def test_tree_splits_exactly_when_over_leaf_size():
    x = inputs.plummer(4000, 21)
    t = O.build_adaptive_tree(x, 20)
    leaf = t["nchild"] == 0
    assert np.all(t["count"][leaf] <= 20) or np.all(t["level"][leaf & (t["count"] > 20)] == O.ADAPTIVE_MAX_LEVEL)
    assert np.all(t["count"][~leaf] > 20)
    assert t["count"][leaf].sum() == 4000
    for c in np.nonzero(~leaf)[0]:
        ch = slice(t["child_begin"][c], t["child_begin"][c] + t["nchild"][c])
        assert t["count"][ch].sum() == t["count"][c]
        assert np.all(t["level"][ch] == t["level"][c] + 1)
        assert np.all(t["parent"][ch] == c)
        assert np.all((t["key"][ch] >> np.uint64(3)) == t["key"][c])


def test_lists_cover_every_pair_exactly_once():
    """Every (target leaf, source particle) pair is covered once by U(B), W(B), and V / X of B
    and its ancestors (the adaptive FMM's completeness property), by brute force."""
    x = inputs.plummer(2000, 8)
    t = O.build_adaptive_tree(x, 8)
    ls = O.build_adaptive_lists(t)
    n = 2000
    for b in np.nonzero(t["nchild"] == 0)[0]:
        cover = np.zeros(n, dtype=np.int32)

        def add(cells):
            for c in cells:
                lo, hi = _subtree_particles(t, c)
                cover[lo:hi] += 1

        add(ls["u_ids"][ls["u_offs"][b]: ls["u_offs"][b + 1]])
        add(ls["w_ids"][ls["w_offs"][b]: ls["w_offs"][b + 1]])
        a = b
        while a >= 0:
            add(ls["v_ids"][ls["v_offs"][a]: ls["v_offs"][a + 1]])
            add(ls["x_ids"][ls["x_offs"][a]: ls["x_offs"][a + 1]])
            a = t["parent"][a]
        assert np.all(cover == 1), (b, np.unique(cover, return_counts=True))


def test_w_and_x_are_dual():
    x = inputs.plummer(3000, 5)
    t = O.build_adaptive_tree(x, 8)
    ls = O.build_adaptive_lists(t)
    w = {(b, c) for b in range(t["ncells"]) for c in ls["w_ids"][ls["w_offs"][b]: ls["w_offs"][b + 1]]}
    xx = {(c, b) for b in range(t["ncells"]) for c in ls["x_ids"][ls["x_offs"][b]: ls["x_offs"][b + 1]]}
    assert w == xx and len(w) > 0


def _lattice(level, per_cell, seed):
    """per_cell points in every cell of the given level of the unit cube, plus the 8 corners
    so that the root cube is exactly [0, 1]^3."""
    side = 2 ** level
    g = np.stack(np.meshgrid(*[np.arange(side)] * 3, indexing="ij"), -1).reshape(-1, 3)
    u = inputs.uniform01(seed, len(g) * per_cell * 3).reshape(len(g) * per_cell, 3)
    pts = (np.repeat(g, per_cell, axis=0) + 0.1 + 0.8 * u) / side
    corners = np.array([[i, j, k] for i in (0, 1) for j in (0, 1) for k in (0, 1)], dtype=float)
    pts = np.vstack([corners * (1 - 1e-7) + 0.5e-7, pts])  # inside the lattice cells next to the faces
    x = np.empty((len(pts), 4), dtype=np.float32)
    x[:, :3] = pts
    x[:, 3] = 0.5 + inputs.uniform01(seed + 1, len(pts))
    return x


def test_adaptive_reduces_to_uniform_on_a_lattice():
    x = _lattice(3, 6, 4)
    leaf = 7  # 6 per cell plus at most one corner point
    ta = O.build_adaptive_tree(x, leaf)
    assert np.all(ta["level"][ta["nchild"] == 0] == 3)
    la = O.build_adaptive_lists(ta)
    assert len(la["w_ids"]) == 0 and len(la["x_ids"]) == 0
    tu = O.build_tree(x, leaf, level=3)
    lu = O.build_lists(tu)
    # map adaptive cells (level, key) to uniform global indices
    glob = np.array([O.level_offset(l) + int(k) for l, k in zip(ta["level"], ta["key"])])
    leaves = np.nonzero(ta["nchild"] == 0)[0]
    for b in leaves:
        u = sorted(glob[la["u_ids"][la["u_offs"][b]: la["u_offs"][b + 1]]])
        k = glob[b] - O.level_offset(3)
        assert u == sorted(lu["p2p_ids"][lu["p2p_offs"][k]: lu["p2p_offs"][k + 1]].tolist())
    for b in range(ta["ncells"]):
        v = sorted(glob[la["v_ids"][la["v_offs"][b]: la["v_offs"][b + 1]]])
        g = glob[b]
        assert v == sorted(lu["m2l_ids"][lu["m2l_offs"][g]: lu["m2l_offs"][g + 1]].tolist())
    fa = O.fmm_adaptive(x, 6, leaf)["out"]
    fu = O.fmm(x, 6, leaf, level=3)["out"]
    assert np.allclose(fa, fu, rtol=1e-12, atol=1e-12 * np.abs(fu).max())


def test_p2l_is_the_local_expansion_of_a_charge():
    # L2P(P2L(q at x0), x) -> q/|x - x0| (and its gradient) for |x - c| < |x0 - c|, with p
    c = np.array([0.1, 0.2, 0.3])
    src = np.array([[1.4, -0.6, 0.9, 0.8], [-1.1, 1.2, 0.5, -0.3]])
    x = c + np.array([0.15, -0.1, 0.2])
    ref = O.direct(np.vstack([src, [[*x, 0.0]]]), targets=[2])[0]
    errs = [O.rel_l2(O.l2p(p, c, O.p2l(p, c, src), x), ref) for p in (2, 4, 8, 12, 16)]
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-9


@pytest.mark.parametrize("dist", ["plummer", "uniform"])
def test_adaptive_error_falls_with_p(dist):
    x = inputs.make_particles(2500, dist, 31)
    ref = O.direct(x)
    errs = [O.rel_l2(O.fmm_adaptive(x, p, 12)["out"][:, 1:], ref[:, 1:]) for p in (2, 4, 6, 8, 10)]
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-4


def test_adaptive_target_subset_matches_full():
    x = inputs.plummer(3000, 13)
    tg = inputs.sample_indices(3000, 60, 2)
    full = O.fmm_adaptive(x, 6, 16)["out"]
    part = O.fmm_adaptive(x, 6, 16, targets=tg)["out"]
    assert np.array_equal(full[tg], part[tg])


def test_duplicates_beyond_leaf_size_stop_at_max_level():
    x = np.repeat(inputs.uniform_cube(3, 2), 30, axis=0)
    t = O.build_adaptive_tree(x, 8, max_level=6)
    assert t["level"].max() == 6
    leaves = t["nchild"] == 0
    assert np.all(t["count"][leaves & (t["level"] < 6)] <= 8) and t["count"][leaves].max() == 30
    ref = O.direct(x)
    e4 = O.rel_l2(O.fmm_adaptive(x, 4, 8, max_level=6)["out"], ref)
    e10 = O.rel_l2(O.fmm_adaptive(x, 10, 8, max_level=6)["out"], ref)
    assert e10 < e4 < 1e-2 and e10 < 1e-5


def test_adaptive_treecode_reduces_to_uniform_treecode_on_a_lattice():
    # with every leaf at level 3, W and X are empty and V along the ancestor chain is the
    # uniform treecode's M2L list of the leaf and its ancestors
    x = _lattice(3, 6, 9)
    ta = O.fmm_adaptive(x, 6, 7, method=O.TREECODE)
    assert np.all(ta["tree"]["level"][ta["tree"]["nchild"] == 0] == 3)
    fu = O.fmm(x, 6, 7, level=3, method=O.TREECODE)["out"]
    assert np.allclose(ta["out"], fu, rtol=1e-12, atol=1e-12 * np.abs(fu).max())
    # and differs from the FMM on the same tree (local expansions are not formed)
    ff = O.fmm_adaptive(x, 6, 7)["out"]
    assert not np.allclose(ta["out"], ff, rtol=1e-12, atol=1e-12 * np.abs(fu).max())


@pytest.mark.parametrize("dist", ["plummer", "uniform"])
def test_adaptive_treecode_error_falls_with_p(dist):
    x = inputs.make_particles(2500, dist, 37)
    ref = O.direct(x)
    errs = [O.rel_l2(O.fmm_adaptive(x, p, 12, method=O.TREECODE)["out"][:, 1:], ref[:, 1:])
            for p in (2, 4, 6, 8, 10)]
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-5


def test_adaptive_treecode_single_leaf_is_the_direct_sum():
    x = inputs.plummer(300, 4)
    ref = O.direct(x, eps2=1e-4)
    tc = O.fmm_adaptive(x, 4, 300, eps2=1e-4, method=O.TREECODE)["out"]
    assert np.allclose(tc, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


def test_adaptive_treecode_x_sources_are_direct():
    # a heavy cluster next to a sparse region: leaves with X lists exist, and the treecode's
    # error stays at the multipole truncation of the V and W cells alone
    x = np.vstack([inputs.plummer(1500, 3) * np.array([0.05, 0.05, 0.05, 1.0], dtype=np.float32),
                   inputs.uniform_cube(400, 5)]).astype(np.float32)
    t = O.build_adaptive_tree(x, 10)
    ls = O.build_adaptive_lists(t)
    assert len(ls["x_ids"]) > 0
    ref = O.direct(x)
    e = O.rel_l2(O.fmm_adaptive(x, 10, 10, method=O.TREECODE)["out"][:, 1:], ref[:, 1:])
    assert e < 1e-5


def test_adaptive_treecode_target_subset_matches_full():
    x = inputs.plummer(3000, 17)
    tg = inputs.sample_indices(3000, 60, 3)
    full = O.fmm_adaptive(x, 6, 16, method=O.TREECODE)["out"]
    part = O.fmm_adaptive(x, 6, 16, targets=tg, method=O.TREECODE)["out"]
    assert np.array_equal(full[tg], part[tg])
