"""Load drivers for the multi-instance engine (include/gbfmm.h, gbfmm_engine_*): a served
request stream with latency percentiles and a batch of uneven instances against the plain
one-at-a-time evaluation.  Argument marshalling and timing only; every evaluation runs in the
library's kernels.
"""
from __future__ import annotations

import threading
import time

import numpy as np
import torch

from . import gbfmm as G
from . import inputs

LEAF = 64


def params_for(dist: str, p: int, leaf: int = LEAF) -> G.gbfmm_params:
    """Uniform-cube sets use the uniform octree, clustered (Plummer) sets the adaptive one."""
    tree = G.TREE_UNIFORM if dist == "uniform" else G.TREE_ADAPTIVE
    return G.gbfmm_default_params(p=p, leaf_size=leaf, tree=tree)


def run_stream(engine, requests: list[dict], pools: dict, timeout_s: float = 120.0) -> dict:
    """Submit each request at its arrival time (seconds from the start) and collect latencies
    (submit -> result in host memory).  Returns percentiles and throughput."""
    n_req = len(requests)
    outs = [None] * n_req
    tickets = [None] * n_req
    lat = np.zeros(n_req)
    queue = np.zeros(n_req)
    status = np.zeros(n_req, dtype=np.int64)
    submitted = threading.Semaphore(0)
    done_at = np.zeros(n_req)

    def collect():
        for i in range(n_req):
            submitted.acquire()
            st, q, l = G.gbfmm_engine_wait(engine, tickets[i], timeout_ms=timeout_s * 1e3)
            status[i], queue[i], lat[i] = st, q, l
            done_at[i] = time.perf_counter()
            outs[i] = None  # release the output buffer

    th = threading.Thread(target=collect)
    th.start()
    t0 = time.perf_counter()
    for i, r in enumerate(requests):
        pool = pools[r["dist"]]
        off = int(r["slot"] * (len(pool) - r["n"]))
        h_in = pool[off: off + r["n"]]
        outs[i] = (h_in, np.empty((r["n"], 4), dtype=np.float32))
        wait = r["t"] - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        tickets[i] = G.gbfmm_engine_submit(engine, params_for(r["dist"], r["p"]), outs[i][0], outs[i][1])
        submitted.release()
    th.join()
    wall = float(done_at.max() - t0) if n_req else 0.0
    parts = float(sum(r["n"] for r in requests))
    return {
        "requests": n_req, "failed": int(np.count_nonzero(status)),
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "mean_ms": float(lat.mean()), "max_ms": float(lat.max()),
        "queue_p50_ms": float(np.percentile(queue, 50)), "queue_p99_ms": float(np.percentile(queue, 99)),
        "particles": parts, "wall_s": wall, "particles_per_s": parts / wall if wall > 0 else 0.0,
        "offered_particles_per_s": parts / requests[-1]["t"] if n_req else 0.0,
    }


def tune_leaves(ctx, x, offsets, instances: list[dict], candidates=(32, 64, 128, 256)) -> dict:
    """Leaf size per (distribution, p, floor(log2 N)) bucket, chosen by gbfmm_tune_leaf on the
    bucket's first instance."""
    import math

    chosen = {}
    for i, r in enumerate(instances):
        key = (r["dist"], r["p"], int(math.log2(max(r["n"], 1))))
        if key in chosen:
            continue
        a, b = int(offsets[i]), int(offsets[i + 1])
        chosen[key], _ = G.gbfmm_tune_leaf(ctx, params_for(r["dist"], r["p"]), x[a:b], list(candidates))
    return chosen


def tuned_params(instances: list[dict], leaves: dict) -> list:
    import math

    return [params_for(r["dist"], r["p"], leaves[(r["dist"], r["p"], int(math.log2(max(r["n"], 1))))])
            for r in instances]


def make_batch(instances: list[dict], device) -> tuple:
    """Concatenated device particles of the instances, their offsets and parameters."""
    xs = [inputs.make_particles(r["n"], r["dist"], r["seed"]) for r in instances]
    offsets = np.concatenate([[0], np.cumsum([len(x) for x in xs])]).astype(np.int64)
    x = torch.from_numpy(np.concatenate(xs)).to(device)
    params = [params_for(r["dist"], r["p"]) for r in instances]
    return x, offsets, params


def run_plain(ctx, x, offsets, params, stream=None) -> float:
    """The one-at-a-time form: every instance through gbfmm_evaluate on one context and one
    stream, in order.  Returns (seconds, outputs)."""
    out = torch.empty_like(x)
    ws = torch.empty(256, dtype=torch.uint8, device=x.device)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i, prm in enumerate(params):
        a, b = int(offsets[i]), int(offsets[i + 1])
        _, need = G.gbfmm_plan(prm, b - a)
        if need > ws.numel():
            ws = torch.empty(need, dtype=torch.uint8, device=x.device)
        G.gbfmm_evaluate(ctx, prm, x[a:b], out[a:b], ws, stream)
    G.gbfmm_sync_status(ctx, stream)
    torch.cuda.synchronize()
    return time.perf_counter() - t0, out
