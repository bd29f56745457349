"""Repeated evaluations through a captured CUDA graph, and the leaf-size autotuner.

* A graph replays the captured uniform-tree evaluation of the same buffers: after new particle
  positions are written into the input buffer, a replay gives bit for bit the result of an eager
  gbfmm_evaluate of the new positions.
* The adaptive tree cannot be captured (EUNSUPPORTED).
* gbfmm_tune_leaf returns one of the candidates with a positive time, skips invalid ones, and an
  evaluation with the chosen leaf size matches the oracle FMM of that leaf size.
* The P2P launch shape (target leaves per CTA) changes no bit of the result on either tree;
  gbfmm_tune picks a (leaf size, launch shape) pair from the candidates, the context keeps the
  shape, and out-of-range shapes are rejected.
"""
import numpy as np
import pytest

import oracle as O
from paper_1010_1482_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def test_graph_replay_equals_eager_evaluation(G, ctx):
    n = 200000
    prm = G.gbfmm_default_params(p=8, leaf_size=64)
    _, ws_bytes = G.gbfmm_plan(prm, n)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    xd = torch.from_numpy(inputs.uniform_cube(n, 41)).cuda()
    out = torch.empty_like(xd)
    g = G.gbfmm_graph_create(ctx, prm, xd, out, ws)
    try:
        for seed in (42, 43):
            xd.copy_(torch.from_numpy(inputs.uniform_cube(n, seed)))
            G.gbfmm_graph_launch(g)
            G.gbfmm_sync_status(ctx)
            replay = out.clone()
            ref = torch.empty_like(xd)
            G.gbfmm_evaluate(ctx, prm, xd, ref, ws)
            G.gbfmm_sync_status(ctx)
            assert torch.equal(replay, ref)
    finally:
        G.gbfmm_graph_destroy(g)


def test_graph_rejects_adaptive_tree(G, ctx):
    prm = G.gbfmm_default_params(p=4, leaf_size=32, tree=G.TREE_ADAPTIVE)
    xd = torch.from_numpy(inputs.plummer(5000, 3)).cuda()
    out = torch.empty_like(xd)
    with pytest.raises(G.GbfmmError) as ei:
        G.gbfmm_graph_create(ctx, prm, xd, out, torch.empty(256, dtype=torch.uint8, device="cuda"))
    assert ei.value.code == G.GBFMM_EUNSUPPORTED


@pytest.mark.parametrize("dist,tree", [("uniform", 0), ("plummer", 1)])
def test_tune_leaf(G, ctx, dist, tree):
    n = 20000
    x = inputs.make_particles(n, dist, 77)
    xd = torch.from_numpy(x).cuda()
    prm = G.gbfmm_default_params(p=6, leaf_size=64, tree=tree)
    cands = [0 if tree == 1 else -5, 16, 32, 64, 128]  # the first is rejected by gbfmm_plan
    leaf, ms = G.gbfmm_tune_leaf(ctx, prm, xd, cands)
    assert leaf in (16, 32, 64, 128) and ms > 0.0
    prm2 = G.gbfmm_default_params(p=6, leaf_size=leaf, tree=tree)
    _, wsb = G.gbfmm_plan(prm2, n)
    out = torch.empty_like(xd)
    G.gbfmm_evaluate(ctx, prm2, xd, out, torch.empty(max(wsb, 256), dtype=torch.uint8, device="cuda"))
    G.gbfmm_sync_status(ctx)
    got = out.cpu().numpy().astype(np.float64)
    ref = (O.fmm_adaptive(x, 6, leaf) if tree == 1 else O.fmm(x, 6, leaf))["out"]
    assert O.rel_l2(got, ref) <= 1e-5


@pytest.mark.parametrize("dist,tree", [("uniform", 0), ("plummer", 1)])
def test_p2p_launch_shape_and_tune(G, ctx, dist, tree):
    n = 60000
    x = inputs.make_particles(n, dist, 78)
    xd = torch.from_numpy(x).cuda()
    prm = G.gbfmm_default_params(p=6, leaf_size=32, tree=tree)
    _, wsb = G.gbfmm_plan(prm, n)
    ws = torch.empty(max(wsb, 256), dtype=torch.uint8, device="cuda")
    outs = []
    try:
        for lpc in (0, 1, 3, 64):
            G.gbfmm_set_p2p_leaves_per_cta(ctx, lpc)
            out = torch.empty_like(xd)
            G.gbfmm_evaluate(ctx, prm, xd, out, ws)
            G.gbfmm_sync_status(ctx)
            outs.append(out.cpu())
        for o in outs[1:]:
            assert torch.equal(o, outs[0])
        leaf, lpc, ms = G.gbfmm_tune(ctx, prm, xd, [16, 32], [1, 4])
        assert leaf in (16, 32) and lpc in (1, 4) and ms > 0.0
        with pytest.raises(G.GbfmmError) as ei:
            G.gbfmm_set_p2p_leaves_per_cta(ctx, 65)
        assert ei.value.code == G.GBFMM_EINVAL
    finally:
        G.gbfmm_set_p2p_leaves_per_cta(ctx, 0)

