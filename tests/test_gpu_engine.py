"""The multi-instance engine (gbfmm_engine_*): batched uneven instances and a served request
stream give every instance the result it gets alone, bit for bit (each request runs the
unchanged single-instance evaluation; only the overlap differs), and respect the memory
budget's admission rule."""
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
def S():
    from paper_1010_1482_gb300 import serving

    return serving


def alone(G, S, x, dist, p):
    fmm = G.FMM(0)
    fmm.params = S.params_for(dist, p)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    out = fmm.evaluate(xd).cpu().numpy()
    fmm.close()
    return out


def test_batch_matches_single_instances(G, S):
    inst = inputs.batch_instances(count=24, n_lo=500, n_hi=30000)
    x, offsets, params = S.make_batch(inst, "cuda")
    out = torch.empty_like(x)
    e = G.gbfmm_engine_create(0, 4, 8 << 30)
    try:
        G.gbfmm_engine_prepare(e, [4, 8])
        st = G.gbfmm_engine_run_batch(e, offsets, params, x, out)
    finally:
        G.gbfmm_engine_destroy(e)
    assert st == [0] * len(inst)
    got = out.cpu().numpy()
    xh = x.cpu().numpy()
    for i, r in enumerate(inst):
        a, b = offsets[i], offsets[i + 1]
        ref = alone(G, S, xh[a:b], r["dist"], r["p"])
        assert np.array_equal(got[a:b], ref), i
    # and against the oracle for two of them (one per tree)
    for i in (0, 1):
        a, b = offsets[i], offsets[i + 1]
        r = inst[i]
        f = O.fmm(xh[a:b], r["p"], 64)["out"] if r["dist"] == "uniform" else O.fmm_adaptive(xh[a:b], r["p"], 64)["out"]
        assert O.rel_l2(got[a:b].astype(np.float64), f) <= 1e-5


def test_served_results_identical_alone_and_in_mix(G, S):
    reqs = inputs.served_requests(rate=2000.0, duration=0.03, n_lo=1e3, n_hi=6e4, seed=77)
    assert len(reqs) >= 20
    e = G.gbfmm_engine_create(0, 4, 8 << 30)
    try:
        G.gbfmm_engine_prepare(e, [4, 6, 10])
        bufs, tickets = [], []
        for r in reqs:  # a burst: everything is queued at once and overlaps on the device
            hin = inputs.make_particles(r["n"], r["dist"], r["seed"])
            hout = np.empty_like(hin)
            bufs.append((hin, hout, r))
            tickets.append(G.gbfmm_engine_submit(e, S.params_for(r["dist"], r["p"]), hin, hout))
        lat = []
        for t in tickets:
            st, q, l = G.gbfmm_engine_wait(e, t)
            assert st == 0
            assert 0 <= q <= l
            lat.append(l)
    finally:
        G.gbfmm_engine_destroy(e)
    for hin, hout, r in bufs:
        assert np.array_equal(hout, alone(G, S, hin, r["dist"], r["p"]))


def test_tiny_budget_runs_one_at_a_time(G, S):
    e = G.gbfmm_engine_create(0, 3, 1)  # 1 byte: every request is larger than the budget
    x = inputs.uniform_cube(20000, 5)
    outs = [np.empty_like(x) for _ in range(4)]
    try:
        ts = [G.gbfmm_engine_submit(e, S.params_for("uniform", 4), x, o) for o in outs]
        res = [G.gbfmm_engine_wait(e, t) for t in ts]
    finally:
        G.gbfmm_engine_destroy(e)
    assert all(r[0] == 0 for r in res)
    ref = alone(G, S, x, "uniform", 4)
    for o in outs:
        assert np.array_equal(o, ref)
    # admission: with nothing fitting the budget, request k starts only after request k - 1 is
    # done (FIFO), so its queueing time covers the previous request's latency
    for k in range(1, len(res)):
        assert res[k][1] >= res[k - 1][2] - 0.5, (k, res)


def test_engine_rejects_bad_requests(G, S):
    e = G.gbfmm_engine_create(0, 1, 1 << 30)
    try:
        x = inputs.uniform_cube(100, 1)
        with pytest.raises(G.GbfmmError) as ei:
            G.gbfmm_engine_submit(e, G.gbfmm_default_params(p=5), x, np.empty_like(x))
        assert ei.value.code == G.GBFMM_EUNSUPPORTED
        with pytest.raises(G.GbfmmError) as ei:
            G.gbfmm_engine_wait(e, 12345, 10.0)
        assert ei.value.code == G.GBFMM_EINVAL
    finally:
        G.gbfmm_engine_destroy(e)
