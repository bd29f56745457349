"""One captured CUDA graph for a batch of uneven instances (gbfmm_batch_*, gbfmm_evaluate_batch).

Every instance of a replay is bit-identical to the same instance evaluated alone with
gbfmm_evaluate (the same kernels in the same order on its own data; only the concurrency between
instances differs), including after the arrays were refilled with other particles of the same
counts.  An adaptive instance whose tree outgrows the capacities of the capture is reported
(ENOMEM from the status word) while the other instances stay exact and the context stays usable.
One instance per tree is also checked against the FP64 oracle."""
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


def _mixed(G, seed):
    """Instances of both trees and methods, orders 4..10, softening, one particle, none."""
    spec = [("uniform", 3000, 4, 0, 0, 64), ("plummer", 20000, 8, 1, 0, 64), ("uniform", 12000, 8, 1, 0, 32),
            ("plummer", 5000, 4, 1, 1, 32), ("uniform", 1, 6, 0, 0, 64), ("plummer", 0, 4, 1, 0, 64),
            ("plummer", 9000, 10, 1, 0, 48), ("uniform", 25000, 6, 0, 1, 64), ("plummer", 700, 6, 1, 0, 64),
            ("uniform", 8000, 10, 1, 0, 16), ("plummer", 15000, 6, 0, 0, 64), ("plummer", 30000, 4, 1, 0, 128)]
    xs, prms = [], []
    for i, (dist, n, p, tree, method, leaf) in enumerate(spec):
        xs.append(inputs.make_particles(n, dist, seed * 100 + i) if n else np.zeros((0, 4), np.float32))
        prms.append(G.gbfmm_default_params(p=p, tree=tree, method=method, leaf_size=leaf,
                                           eps2=1e-6 if i == 7 else 0.0))
    off = np.concatenate([[0], np.cumsum([len(x) for x in xs])]).astype(np.int64)
    return np.concatenate(xs).astype(np.float32), off, prms


def _alone(G, ctx, x, off, prms):
    """Every instance through gbfmm_evaluate on its own (serial stages, as in the batch)."""
    out = np.zeros_like(x)
    for i, prm in enumerate(prms):
        a, b = int(off[i]), int(off[i + 1])
        if b == a:
            continue
        p = G.gbfmm_default_params(p=prm.p, tree=prm.tree, method=prm.method, leaf_size=prm.leaf_size, eps2=prm.eps2,
                                   flags=G.FLAG_SERIAL)
        _, ws = G.gbfmm_plan(p, b - a)
        xd = torch.from_numpy(np.ascontiguousarray(x[a:b])).cuda()
        od = torch.empty_like(xd)
        G.gbfmm_evaluate(ctx, p, xd, od, torch.empty(max(ws, 1), dtype=torch.uint8, device="cuda"))
        G.gbfmm_sync_status(ctx)
        out[a:b] = od.cpu().numpy()
    return out


def test_batch_graph_replays_bit_identical(G, ctx):
    x, off, prms = _mixed(G, 1)
    xd = torch.from_numpy(x).cuda()
    out = torch.zeros_like(xd)
    b = G.gbfmm_batch_create(ctx, off, prms, xd, out, lanes=4)
    try:
        lanes, nodes = G.gbfmm_batch_info(b)
        assert lanes == 4 and nodes > 100
        ref = _alone(G, ctx, x, off, prms)
        assert np.array_equal(out.cpu().numpy(), ref)  # the creating evaluation
        for _ in range(2):
            out.zero_()
            G.gbfmm_batch_launch(ctx, b)
            G.gbfmm_sync_status(ctx)
            assert np.array_equal(out.cpu().numpy(), ref)
        # other particles of the same counts, written into the same arrays
        x2, off2, _ = _mixed(G, 2)
        assert np.array_equal(off2, off)
        xd.copy_(torch.from_numpy(x2))
        out.zero_()
        G.gbfmm_batch_launch(ctx, b)
        G.gbfmm_sync_status(ctx)
        got = out.cpu().numpy()
        assert np.array_equal(got, _alone(G, ctx, x2, off, prms))
    finally:
        G.gbfmm_batch_destroy(b)
    # one instance of each tree against the FP64 oracle
    for i in (1, 2):
        a, e = int(off[i]), int(off[i + 1])
        xs = x2[a:e]
        f = (O.fmm_adaptive(xs, prms[i].p, prms[i].leaf_size, method=prms[i].method) if prms[i].tree
             else O.fmm(xs, prms[i].p, prms[i].leaf_size, method=prms[i].method))["out"]
        assert O.rel_l2(got[a:e].astype(np.float64), f) <= TOL_FMM, i


def test_batch_capacity_overflow_is_reported(G, ctx):
    # instance 0 is captured on a uniform cube; refilled with a tight cluster of the same count its
    # adaptive tree is far deeper than the capture's capacities
    n0, n1 = 6000, 4000
    x0 = inputs.uniform_cube(n0, 5)
    x1 = inputs.plummer(n1, 6)
    prms = [G.gbfmm_default_params(p=6, tree=G.TREE_ADAPTIVE, leaf_size=32),
            G.gbfmm_default_params(p=6, tree=G.TREE_ADAPTIVE, leaf_size=32)]
    off = np.array([0, n0, n0 + n1], dtype=np.int64)
    xd = torch.from_numpy(np.concatenate([x0, x1])).cuda()
    out = torch.zeros_like(xd)
    b = G.gbfmm_batch_create(ctx, off, prms, xd, out, lanes=2)
    try:
        clustered = inputs.plummer(n0, 7) * np.array([1e-3, 1e-3, 1e-3, 1.0], dtype=np.float32)
        clustered[:8, :3] = inputs.uniform_cube(8, 8)[:, :3]  # the same root box, a deep tree inside
        xd[:n0] = torch.from_numpy(clustered).cuda()
        out.fill_(7.0)
        G.gbfmm_batch_launch(ctx, b)
        with pytest.raises(G.GbfmmError) as ei:
            G.gbfmm_sync_status(ctx)
        assert ei.value.code == G.GBFMM_ENOMEM
        got = out.cpu().numpy()
        assert np.all(got[:n0] == 7.0)  # the overflowing instance wrote nothing
        ref = _alone(G, ctx, xd.cpu().numpy(), off, prms)
        assert np.array_equal(got[n0:], ref[n0:])
        # the context stays usable and the status word was cleared
        xd[:n0] = torch.from_numpy(x0).cuda()
        G.gbfmm_batch_launch(ctx, b)
        G.gbfmm_sync_status(ctx)
        assert np.array_equal(out.cpu().numpy(), _alone(G, ctx, xd.cpu().numpy(), off, prms))
    finally:
        G.gbfmm_batch_destroy(b)


def test_evaluate_batch_keeps_its_graph(G, ctx):
    inst = inputs.batch_instances(count=16, n_lo=1000, n_hi=20000)
    xs = [inputs.make_particles(r["n"], r["dist"], r["seed"]) for r in inst]
    off = np.concatenate([[0], np.cumsum([len(x) for x in xs])]).astype(np.int64)
    prms = [G.gbfmm_default_params(p=r["p"], tree=G.TREE_ADAPTIVE if r["dist"] == "plummer" else G.TREE_UNIFORM)
            for r in inst]
    xd = torch.from_numpy(np.concatenate(xs)).cuda()
    out = torch.zeros_like(xd)
    G.gbfmm_evaluate_batch(ctx, off, prms, xd, out)
    G.gbfmm_sync_status(ctx)
    first = out.clone()
    out.zero_()
    G.gbfmm_evaluate_batch(ctx, off, prms, xd, out)  # the kept graph
    G.gbfmm_sync_status(ctx)
    assert torch.equal(out, first)
    assert np.array_equal(first.cpu().numpy(), _alone(G, ctx, xd.cpu().numpy(), off, prms))
