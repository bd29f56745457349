"""GPU parity of the adaptive-tree FMM (U, V, W, X lists of Cheng, Greengard & Rokhlin 1999,
the FMM the paper cites for its translation operators) against the FP64 adaptive oracle.

Tolerances as for the uniform tree:
  * cells (level, key, particle range, parent), sort permutation and the four lists: bit-exact;
  * potentials and gradients vs the oracle adaptive FMM or treecode (same tree, same p):
    relative L2 <= 1e-5;
  * expansions: per-degree relative L2 of the scaled coefficients <= 1e-4.
"""
import numpy as np
import pytest

import oracle as O
from paper_1010_1482_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FMM = 1e-5


@pytest.fixture(scope="module")
def G():
    from paper_1010_1482_gb300 import gbfmm

    gbfmm.lib()
    return gbfmm


@pytest.fixture(scope="module")
def ctx(G):
    c = G.gbfmm_create(0)
    yield c
    G.gbfmm_destroy(c)


def run(G, ctx, x, **kw):
    prm = G.gbfmm_default_params(tree=G.TREE_ADAPTIVE, **kw)
    lv, ws = G.gbfmm_plan(prm, len(x))
    assert lv == O.ADAPTIVE_MAX_LEVEL and ws == 0
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()
    out = torch.empty_like(xd)
    G.gbfmm_evaluate(ctx, prm, xd, out, torch.empty(0, dtype=torch.uint8, device="cuda"))
    G.gbfmm_sync_status(ctx)
    return out.cpu().numpy().astype(np.float64)


def sorted_rows(offs, ids):
    row = np.repeat(np.arange(len(offs) - 1), np.diff(offs))
    return ids[np.lexsort((ids, row))]


# ("plummer", 1000000, 8) has more than 2^17 cells (list rows a thread per cell); ("plummer",
# 60000, 20000) has a leaf size beyond the one-pass construction's window (level-by-level
# rounds); the 5,000,000-particle case sorts in the reduce-then-scan form (2^22 and more)
TREE_CASES = [("plummer", 30000, 32), ("plummer", 100000, 64), ("uniform", 20000, 16), ("plummer", 1000000, 8),
              ("plummer", 60000, 20000), ("plummer", 5000000, 64)]


@pytest.mark.parametrize("dist,n,leaf", TREE_CASES)
def test_adaptive_tree_and_lists_bit_exact(G, ctx, dist, n, leaf):
    x = inputs.make_particles(n, dist, 3000 + n)
    run(G, ctx, x, p=4, leaf_size=leaf)
    t = O.build_adaptive_tree(x, leaf)
    g = G.gbfmm_export_adaptive_tree(ctx, n)
    assert np.array_equal(g["origin"], t["origin"]) and g["side"] == t["side"]
    assert g["ncells"] == t["ncells"]
    for k in ("level", "begin", "count", "parent"):
        assert np.array_equal(g[k], t[k]), k
    assert np.array_equal(g["key"], t["key"])
    assert np.array_equal(g["perm"].astype(np.int64), t["perm"])
    ls = O.build_adaptive_lists(t)
    nc = t["ncells"]
    for kind, name in ((G.LIST_U, "u"), (G.LIST_V, "v"), (G.LIST_W, "w"), (G.LIST_X, "x")):
        offs, ids = G.gbfmm_export_lists(ctx, kind, nc)
        assert np.array_equal(offs, ls[name + "_offs"]), name
        assert np.array_equal(ids, sorted_rows(ls[name + "_offs"], ls[name + "_ids"])), name
    if dist == "plummer" and leaf < 1000:
        # a clustered set has leaves at several levels: W and X are not empty
        assert len(ls["w_ids"]) > 0 and len(ls["x_ids"]) > 0


def test_adaptive_keys_on_depth21_faces(G, ctx):
    # coordinates on faces of the depth-21 grid of the unit box (the 8 corners pin the root box
    # to [0, 1]^3, so the key scale is 2^21) and one float step to either side, each with a
    # partner one grid unit away; leaf size 1 resolves every pair down to the level where it
    # parts, so a key coordinate off by one changes the tree.  The keys' float-float estimate
    # cannot decide these coordinates and takes the FP64 steps.
    m = 1500
    u = inputs.uniform01(77, 7 * m).reshape(m, 7)
    j = np.floor(u[:, :3] * (2 ** 21 - 2)).astype(np.int64) + 1
    c = (j / 2.0 ** 21).astype(np.float32)
    step = np.floor(u[:, 3:6] * 3).astype(np.int64) - 1  # -1, 0, +1 float steps
    c = np.where(step < 0, np.nextafter(c, np.float32(0)), np.where(step > 0, np.nextafter(c, np.float32(1)), c))
    partner = (c + np.float32(2.0 ** -21) * np.where(u[:, 6:7] < 0.5, -1, 1)).astype(np.float32)
    pts = np.vstack([c, np.clip(partner, 0, 1)])
    corners = np.array([[a, b, d] for a in (0, 1) for b in (0, 1) for d in (0, 1)], dtype=np.float32)
    pts = np.vstack([corners, pts])
    x = np.concatenate([pts, np.ones((len(pts), 1), np.float32)], axis=1).astype(np.float32)
    run(G, ctx, x, p=4, leaf_size=1)
    t = O.build_adaptive_tree(x, 1)
    assert t["side"] == 1.0 and np.all(t["origin"] == 0.0)
    g = G.gbfmm_export_adaptive_tree(ctx, len(x))
    assert g["ncells"] == t["ncells"]
    for k in ("level", "begin", "count", "parent"):
        assert np.array_equal(g[k], t[k]), k
    assert np.array_equal(g["key"], t["key"])
    assert np.array_equal(g["perm"].astype(np.int64), t["perm"])
    assert t["level"].max() == O.ADAPTIVE_MAX_LEVEL


@pytest.mark.parametrize("p", [4, 6, 8, 10])
def test_adaptive_fmm_matches_oracle(G, ctx, p):
    n, leaf = 20000, 32
    x = inputs.plummer(n, 4242)
    out = run(G, ctx, x, p=p, leaf_size=leaf)
    ref = O.fmm_adaptive(x, p, leaf)["out"]
    assert O.rel_l2(out[:, 0], ref[:, 0]) <= TOL_FMM
    assert O.rel_l2(out[:, 1:], ref[:, 1:]) <= TOL_FMM
    d = O.direct(x)
    e_or = O.rel_l2(ref[:, 1:], d[:, 1:])
    assert O.rel_l2(out[:, 1:], d[:, 1:]) <= e_or + TOL_FMM


@pytest.mark.parametrize("p,n,leaf", [(8, 30000, 32), (4, 200000, 64), (10, 20000, 16), (6, 3000, 8)])
def test_adaptive_m2l_forms_agree(G, ctx, p, n, leaf):
    # the block form (default: one GEMM per parent offset over the cells with children), the
    # list form over the V lists (gathered) and the FP32 CUDA-core form
    x = inputs.plummer(n, 77 + p)
    blk = run(G, ctx, x, p=p, leaf_size=leaf)
    gat = run(G, ctx, x, p=p, leaf_size=leaf, flags=G.FLAG_M2L_GATHERED)
    cc = run(G, ctx, x, p=p, leaf_size=leaf, flags=G.FLAG_M2L_CUDA_CORES)
    ref = O.fmm_adaptive(x, p, leaf)["out"]
    for out in (blk, gat, cc):
        assert O.rel_l2(out, ref) <= TOL_FMM
    assert O.rel_l2(blk, cc) <= 5e-6 and O.rel_l2(gat, cc) <= 5e-6


@pytest.mark.parametrize("p", [4, 10])
def test_adaptive_expansions_match_oracle(G, ctx, p):
    n, leaf = 20000, 32
    x = inputs.plummer(n, 515)
    run(G, ctx, x, p=p, leaf_size=leaf)
    r = O.fmm_adaptive(x, p, leaf, keep=True)
    t = r["tree"]
    nc = t["ncells"]
    Mg = G.gbfmm_export_expansions(ctx, 0, nc, p)
    Lg = G.gbfmm_export_expansions(ctx, 1, nc, p)
    h = t["side"] / 2.0 ** t["level"]
    deep = t["level"] >= 2
    assert np.all(Mg[~deep] == 0) and np.all(Lg[~deep] == 0)
    for n_ in range(p):
        cols = slice(n_ * (n_ + 1) // 2, (n_ + 1) * (n_ + 2) // 2)
        for A, B, sc in ((Mg, r["M"], h ** (-n_)), (Lg, r["Lc"], h ** (n_ + 1))):
            a = A[deep, cols] * sc[deep, None]
            b = B[deep, cols] * sc[deep, None]
            assert np.linalg.norm(a - b) <= 1e-4 * np.linalg.norm(b), n_


@pytest.mark.parametrize("kind", ["one", "two", "below_leaf", "duplicates", "shell"])
def test_adaptive_degenerate_inputs(G, ctx, kind):
    if kind == "one":
        x, leaf = np.array([[0.3, 0.2, 0.1, 1.0]], dtype=np.float32), 64
    elif kind == "two":
        x, leaf = np.array([[0.3, 0.2, 0.1, 1.0], [0.7, 0.1, 0.9, 2.0]], dtype=np.float32), 64
    elif kind == "below_leaf":
        x, leaf = inputs.uniform_cube(50, 4), 64
    elif kind == "duplicates":
        # 200 copies of one point: its cell splits down to level 21 and stays over-full there
        base = inputs.uniform_cube(3000, 8)
        dup = np.repeat(base[:1], 200, axis=0)
        x, leaf = np.concatenate([base, dup]).astype(np.float32), 16
    else:  # particles on a thin spherical shell: leaves at many levels
        u = inputs.uniform_cube(8000, 9).astype(np.float64)
        v = u[:, :3] - 0.5
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        x = np.concatenate([v * 0.5 + 0.5, u[:, 3:]], axis=1).astype(np.float32)
        leaf = 16
    out = run(G, ctx, x, p=6, leaf_size=leaf)
    ref = O.fmm_adaptive(x, 6, leaf)["out"]
    scale = max(1.0, float(np.max(np.abs(ref))))
    assert np.max(np.abs(out - ref)) <= 2e-5 * scale
    if kind == "one":
        assert np.all(out == 0.0)


def test_adaptive_uniform_lattice_reduces_to_uniform_tree(G, ctx):
    # 16^3 lattice points, leaf 8: every leaf sits at level 3 and the adaptive result equals
    # the uniform-tree result (same lists, W = X = empty)
    g = (np.arange(16) + 0.5) / 16
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    q = inputs.uniform_cube(4096, 11)[:, 3]
    x = np.stack([X.ravel(), Y.ravel(), Z.ravel(), q], axis=1).astype(np.float32)
    ad = run(G, ctx, x, p=8, leaf_size=8)
    prm = G.gbfmm_default_params(p=8, leaf_size=8)
    L, ws = G.gbfmm_plan(prm, len(x))
    assert L == 3
    xd = torch.from_numpy(x).cuda()
    out = torch.empty_like(xd)
    G.gbfmm_evaluate(ctx, prm, xd, out, torch.empty(ws, dtype=torch.uint8, device="cuda"))
    G.gbfmm_sync_status(ctx)
    un = out.cpu().numpy().astype(np.float64)
    assert O.rel_l2(ad, un) <= 1e-6


@pytest.mark.parametrize("n,leaf", [(50000, 32), (3000, 64)])
def test_adaptive_concurrent_near_field_equals_serial(G, ctx, n, leaf):
    """P2P over the U lists on a second stream beside the expansions gives the serial output
    (all stages on the caller's stream; the timed evaluation) bit for bit.  Trees without a
    far field (fewer particles than a leaf holds) take the same path in
    test_adaptive_degenerate_inputs."""
    x = inputs.plummer(n, 515)
    a = run(G, ctx, x, p=8, leaf_size=leaf)
    b = run(G, ctx, x, p=8, leaf_size=leaf, flags=G.FLAG_SERIAL)
    c = run(G, ctx, x, p=8, leaf_size=leaf, flags=G.FLAG_STAGE_TIMING)
    assert np.array_equal(a, b) and np.array_equal(a, c)
    for _ in range(2):
        assert np.array_equal(a, run(G, ctx, x, p=8, leaf_size=leaf))
    ref = O.fmm_adaptive(x, 8, leaf)["out"]
    assert O.rel_l2(a, ref) <= TOL_FMM


def test_adaptive_host_path_and_timing(G, ctx):
    x = inputs.plummer(10000, 31)
    prm = G.gbfmm_default_params(tree=G.TREE_ADAPTIVE, p=4, leaf_size=32, flags=G.FLAG_STAGE_TIMING)
    xh = torch.from_numpy(x).pin_memory()
    oh = torch.empty_like(xh).pin_memory()
    G.gbfmm_evaluate_host(ctx, prm, xh, oh)
    ref = O.fmm_adaptive(x, 4, 32)["out"]
    assert O.rel_l2(oh.numpy().astype(np.float64), ref) <= TOL_FMM
    st = G.gbfmm_stage_times(ctx)
    assert st["P2P"] > 0 and st["M2L/M2P"] > 0
    assert G.gbfmm_last_launch_count(ctx) > 0
    with pytest.raises(G.GbfmmError):  # the uniform-tree export refuses an adaptive evaluation
        G.gbfmm_export_tree(ctx, len(x), 1)


def test_large_plummer_p8_sampled(G, ctx):
    """16,777,216 Plummer particles (scale radius 1, truncated at r = 20), equal masses 1/N,
    adaptive tree, p = 8, leaf 64, in the bench's launch shape: 2048 seeded targets against
    the FP64 direct sum over all sources, 256 of them against the FP64 adaptive FMM."""
    w = inputs.workload("plummer_16m_p8")
    x = inputs.make_particles(w["n"], w["dist"], w["seed"])
    out = run(G, ctx, x, p=w["p"], leaf_size=w["leaf_size"])
    assert np.all(np.isfinite(out))
    tg = inputs.sample_indices(w["n"], 2048, w["seed"])
    d = O.direct(x, targets=tg)
    e_phi = O.rel_l2(out[tg, 0], d[:, 0])
    e_grad = O.rel_l2(out[tg, 1:], d[:, 1:])
    assert e_phi <= 1e-4 and e_grad <= 1e-4, (e_phi, e_grad)
    sub = tg[:256]
    f = O.fmm_adaptive(x, w["p"], w["leaf_size"], targets=sub)["out"]
    assert O.rel_l2(out[sub], f[sub]) <= TOL_FMM


# the treecode on the adaptive tree: the level-by-level tree (leaf 20000), one leaf (no
# expansions), a shell (leaves at many levels), softening
TC_CASES = [("plummer", 30000, 32, 8, 0.0), ("uniform", 20000, 16, 6, 0.0), ("plummer", 60000, 20000, 4, 0.0),
            ("plummer", 40, 64, 6, 0.0), ("shell", 8000, 16, 10, 0.0), ("plummer", 20000, 24, 4, 1e-4)]


def _shell(n, seed):
    u = inputs.uniform_cube(n, seed).astype(np.float64)
    v = u[:, :3] - 0.5
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return np.concatenate([v * 0.5 + 0.5, u[:, 3:]], axis=1).astype(np.float32)


@pytest.mark.parametrize("dist,n,leaf,p,eps2", TC_CASES)
def test_adaptive_treecode_matches_oracle(G, ctx, dist, n, leaf, p, eps2):
    x = _shell(n, 41) if dist == "shell" else inputs.make_particles(n, dist, 4100 + n)
    out = run(G, ctx, x, p=p, leaf_size=leaf, method=G.METHOD_TREECODE, eps2=eps2)
    ref = O.fmm_adaptive(x, p, leaf, eps2=eps2, method=O.TREECODE)["out"]
    assert O.rel_l2(out[:, 0], ref[:, 0]) <= TOL_FMM
    assert O.rel_l2(out[:, 1:], ref[:, 1:]) <= TOL_FMM
    if n >= 20000 and leaf < 1000:
        # the treecode's error against the direct sum is the oracle treecode's, not the FMM's
        d = O.direct(x, targets=np.arange(0, n, 97), eps2=eps2)
        e_or = O.rel_l2(ref[::97, 1:], d[:, 1:])
        assert O.rel_l2(out[::97, 1:], d[:, 1:]) <= e_or + TOL_FMM


def test_adaptive_treecode_expansions_and_stages(G, ctx):
    n, leaf, p = 20000, 32, 6
    x = inputs.plummer(n, 616)
    prm = dict(p=p, leaf_size=leaf, method=G.METHOD_TREECODE)
    a = run(G, ctx, x, **prm)
    r = O.fmm_adaptive(x, p, leaf, keep=True, method=O.TREECODE)
    t = r["tree"]
    nc = t["ncells"]
    Mg = G.gbfmm_export_expansions(ctx, 0, nc, p)
    Lg = G.gbfmm_export_expansions(ctx, 1, nc, p)
    assert np.all(Lg == 0)  # no local expansions are formed
    h = t["side"] / 2.0 ** t["level"]
    deep = t["level"] >= 2
    for n_ in range(p):
        cols = slice(n_ * (n_ + 1) // 2, (n_ + 1) * (n_ + 2) // 2)
        sc = h ** (-n_)
        a_ = Mg[deep, cols] * sc[deep, None]
        b_ = r["M"][deep, cols] * sc[deep, None]
        assert np.linalg.norm(a_ - b_) <= 1e-4 * np.linalg.norm(b_), n_
    b = run(G, ctx, x, flags=G.FLAG_STAGE_TIMING, **prm)
    assert np.array_equal(a, b)
    st = G.gbfmm_stage_times(ctx)
    assert st["P2P"] > 0 and st["M2L/M2P"] > 0
