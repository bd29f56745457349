"""Pins of the oracle's root box, Morton keys, sort, cells and interaction lists.

Checks use hand-computable keys, exact geometric containment (rational
arithmetic), brute-force pair coverage, and the list sizes the paper prints.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_1010_1482_gb300 import inputs

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


def _every_key_bit(axis):
    return sum(1 << (3 * b + axis) for b in range(21))


def test_corner_keys_by_hand():
    pts = np.array([[x, y, z, 1.0] for z in (0, 1) for y in (0, 1) for x in (0, 1)], dtype=np.float32)
    origin, side, bad = O.root_box(pts)
    assert bad == 0 and side == 1.0 and list(origin) == [0.0, 0.0, 0.0]
    keys = O.morton_keys(pts, origin, side)
    for i, (x, y, z, _) in enumerate(pts):
        expect = int(x) * _every_key_bit(0) + int(y) * _every_key_bit(1) + int(z) * _every_key_bit(2)
        assert int(keys[i]) == expect
    assert int(keys[-1]) == (1 << 63) - 1


def test_root_box_degenerate_and_nonfinite():
    one = np.array([[0.25, 0.5, 0.75, 1.0]], dtype=np.float32)
    origin, side, bad = O.root_box(one)
    assert side == 1.0 and bad == 0
    assert list(origin) == [0.25 - 0.5, 0.0, 0.75 - 0.5]
    nan = np.array([[0.1, np.nan, 0.2, 1.0], [0.3, 0.2, 0.1, 1.0]], dtype=np.float32)
    assert O.root_box(nan)[2] == 1


@pytest.mark.parametrize("dist", ["uniform", "plummer"])
def test_keys_contain_particles_exactly(dist):
    x = inputs.make_particles(3000, dist, 99)
    origin, side, _ = O.root_box(x)
    keys = O.morton_keys(x, origin, side)
    S = Fraction(side)
    for i in range(0, 3000, 37):
        k = O.key_decode(int(keys[i]), 21)
        for d in range(3):
            t = (Fraction(float(x[i, d])) - Fraction(float(origin[d]))) / S * (1 << 21)
            # the cell index is floor of the exact scaled coordinate, clamped (FP64 rounding can
            # move it by one only when the exact value is within an ulp of an integer)
            exact = min(max(int(np.floor(float(t))), 0), (1 << 21) - 1)
            assert abs(int(k[d]) - exact) <= 1
            if abs(float(t) - round(float(t))) > 1e-6:
                assert int(k[d]) == exact


def test_sort_is_stable_permutation_and_cells_are_consistent():
    x = inputs.uniform_cube(5000, 5)
    t = O.build_tree(x, 16)
    perm = t["perm"]
    assert sorted(perm.tolist()) == list(range(5000))
    sk = t["sorted_leaf_keys"]
    assert np.all(np.diff(sk.astype(np.int64)) >= 0)
    same = np.diff(sk.astype(np.int64)) == 0
    assert np.all(np.diff(perm)[same] > 0)  # ties keep the original index order
    L = t["L"]
    for l in range(L + 1):
        off = O.level_offset(l)
        cnt = t["count"][off: off + 8 ** l]
        assert cnt.sum() == 5000
        if l < L:
            ch = t["count"][O.level_offset(l + 1): O.level_offset(l + 1) + 8 ** (l + 1)]
            assert np.array_equal(ch.reshape(-1, 8).sum(axis=1), cnt)
        beg = t["begin"][off: off + 8 ** l]
        nz = cnt > 0
        keys_l = sk >> np.uint64(3 * (L - l))
        for c in np.nonzero(nz)[0][:50]:
            assert np.all(keys_l[beg[c]: beg[c] + cnt[c]] == c)


def test_uniform_depth_rule():
    assert O.uniform_depth(4096, 64) == 2
    assert O.uniform_depth(1 << 20, 64) == 5
    assert O.uniform_depth(512, 64) == 1
    assert O.uniform_depth(1, 64) == 0
    assert O.uniform_depth(0, 64) == 0


def _full_tree(L):
    x = inputs.uniform_cube(8 ** L * 20, 3)
    t = O.build_tree(x, 8, level=L)
    assert np.all(t["count"] > 0)
    return t


def test_interior_list_sizes_match_paper():
    t = _full_tree(3)
    ls = O.build_lists(t)
    L = 3
    sizes = np.diff(ls["p2p_offs"])
    m2l_sizes = np.diff(ls["m2l_offs"])
    side = 1 << L
    for key in range(8 ** L):
        ix = O.key_decode(key, L)
        interior = all(1 <= c <= side - 2 for c in ix)
        if interior:
            assert sizes[key] == GOLD["p2p_neighbour_cells_interior"]["value"]
        # closed form per dimension: parent-neighbour children range minus own neighbour range
        tot_far, tot_near = 1, 1
        for c in ix:
            pc = c >> 1
            lo, hi = max(0, 2 * (pc - 1)), min(side - 1, 2 * (pc + 1) + 1)
            tot_far *= hi - lo + 1
            tot_near *= min(side - 1, c + 1) - max(0, c - 1) + 1
        assert m2l_sizes[O.level_offset(L) + key] == tot_far - tot_near
        assert sizes[key] == tot_near
    assert m2l_sizes.max() == GOLD["m2l_list_max"]["value"]


def test_lists_cover_every_leaf_pair_exactly_once():
    L = 3
    t = _full_tree(L)
    ls = O.build_lists(t)
    nl = 8 ** L
    offL = O.level_offset(L)
    cover = np.zeros((nl, nl), dtype=np.int32)
    for tk in range(nl):
        for s in ls["p2p_ids"][ls["p2p_offs"][tk]: ls["p2p_offs"][tk + 1]]:
            cover[tk, s - offL] += 1
        for l in range(2, L + 1):
            a = O.level_offset(l) + (tk >> (3 * (L - l)))
            for s in ls["m2l_ids"][ls["m2l_offs"][a]: ls["m2l_offs"][a + 1]]:
                sk = s - O.level_offset(l)
                span = 8 ** (L - l)
                cover[tk, sk * span: (sk + 1) * span] += 1
    assert np.all(cover == 1)


def test_well_separation_is_the_papers_theta():
    # every (target particle, M2L source cell): cell size / distance to the source centre <= 2/3
    num, den = GOLD["treecode_mac_theta"]["value"]
    x = inputs.uniform_cube(2000, 8)
    t = O.build_tree(x, 8)
    ls = O.build_lists(t)
    L = t["L"]
    xs = x[t["perm"]].astype(np.float64)
    worst = 0.0
    offL = O.level_offset(L)
    for tk in range(0, 8 ** L, 7):
        g = offL + tk
        pts = xs[t["begin"][g]: t["begin"][g] + t["count"][g], :3]
        if len(pts) == 0:
            continue
        for l in range(2, L + 1):
            a = O.level_offset(l) + (tk >> (3 * (L - l)))
            h = t["side"] / 2**l
            for s in ls["m2l_ids"][ls["m2l_offs"][a]: ls["m2l_offs"][a + 1]]:
                c = O.cell_centre(t["origin"], t["side"], l, s - O.level_offset(l))
                d = np.min(np.linalg.norm(pts - c, axis=1))
                worst = max(worst, h / d)
    assert worst <= num / den + 1e-12
    assert worst > 0.6  # attained up to the particles' positions
