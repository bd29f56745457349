"""Benchmark: FMM particles/s on the 1,048,576-particle uniform workload (p = 10, leaf 64).

One step = one full evaluation (root box, keys, sort, cells, lists, P2M, M2M, M2L, L2L, L2P,
P2P and the scatter to the original order) of the workload with inputs resident in HBM.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gbfmm|reference]
                  [--workload NAME] [--no-cpu-baseline]

N > 1 runs under torchrun: every rank evaluates its own replica (independent problems, no
data-path collective; weak scaling).  --impl reference times the FP64 CPU oracle on a bounded
sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1010_1482_gb300 import inputs  # noqa: E402

METRIC = "FMM particles/s at rel L2 err<=1e-4 on 1 GB300; served p50/p99 latency"
UNIT = "particles/s"
L2_FLUSH_BYTES = 256 << 20
CPU_SAMPLE_N = 131072      # oracle sample (reference arm and cpu_baseline): same distribution, p and mean leaf occupancy, depth 4
CPU_ONE_CORE_N = 16384     # single-thread oracle sample (the paper's one-core CPU convention), depth 3
ERROR_TARGETS = 4096


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_seed(seed: int, rank: int) -> int:
    """Each rank evaluates its own independent replica of the workload (weak scaling)."""
    return seed + rank


def max_over_ranks(value: float, device) -> float:
    """The job's time is the slowest rank's: all-reduce MAX (a no-op on one rank)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(n_per_rank: int, world: int, total_ms: float, steps: int) -> float:
    """Whole-job particles/s: every rank's particles over the slowest rank's time per step."""
    return n_per_rank * world / (total_ms / steps / 1e3)


def fp32_peak_tflops(sm_count: int) -> tuple[float, float]:
    """FP32 CUDA-core peak: SMs x 128 lanes x 2 flop (FFMA) x max SM clock."""
    mhz = 2070.0
    try:
        mp = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        mhz = float(mp.get("sm_max_mhz", mhz))
    except Exception:
        pass
    return sm_count * 128 * 2 * mhz * 1e6 / 1e12, mhz


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while active."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                self.out = ""

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), hw=parts[5], hwt=parts[6], swt=parts[7],
                                 pcap=parts[8]))
            except ValueError:
                continue
        if not rows:
            return None
        reasons = []
        for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"), ("swt", "sw_thermal_slowdown"),
                          ("pcap", "sw_power_cap")):
            if any(r[key].lower() == "active" for r in rows):
                reasons.append(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["smax"] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def kernel_source_text(src_text: str, kname: str) -> str:
    """The source of one __global__ kernel: from the template (or __global__) line that opens its
    definition to the next section comment ("// ----") or the end of the file."""
    m = re.search(r"__global__[^;{]*?\b" + re.escape(kname) + r"\s*\(", src_text)
    if not m:
        return ""
    start = src_text.rfind("\ntemplate", 0, m.start())
    gl = src_text.rfind("\n__global__", 0, m.start() + 1)
    if start < 0 or (gl > start and src_text[start:gl].count("\n") > 2):
        start = gl
    end = src_text.find("\n// ----", m.end())
    return src_text[start:end if end >= 0 else len(src_text)]


def kernel_sha16(kernel_file: str, kname: str) -> str:
    src = os.path.join(ROOT, "paper_1010_1482_gb300", "csrc", kernel_file)
    text = kernel_source_text(open(src, encoding="utf-8").read(), kname)
    return hashlib.sha256(text.encode()).hexdigest()[:16] if text else ""


def traffic_from_profile(kernel_file: str, summary: str, kname: str):
    """DRAM bytes per launch recorded by an ncu capture, if the kernel's own source is unchanged
    (the recorded hash is kernel_sha16 of the kernel's text)."""
    path = os.path.join(ROOT, "profiles", summary)
    src = os.path.join(ROOT, "paper_1010_1482_gb300", "csrc", kernel_file)
    if not (os.path.exists(path) and os.path.exists(src)):
        return None
    text = open(path).read()
    sha = kernel_sha16(kernel_file, kname)
    m_sha = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    m_tr = re.search(r"dram_bytes_per_launch_full_size:\s*([0-9.eE+]+)", text)
    if not (m_sha and m_tr) or m_sha.group(1) != sha:
        return None
    return float(m_tr.group(1))


# ------------------------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ------------------------------------------------------------------------------------------

def oracle_fmm(oracle, x, w):
    """The oracle FMM on the workload's tree kind."""
    if w["tree"] == "adaptive":
        return oracle.fmm_adaptive(x, w["p"], w["leaf_size"])
    return oracle.fmm(x, w["p"], w["leaf_size"])


def oracle_sample_text(oracle, n_sample, w):
    if w["tree"] == "adaptive":
        return (f"oracle FP64 adaptive FMM, full evaluation of {n_sample} particles of the same distribution, "
                f"p={w['p']}, leaf {w['leaf_size']}")
    return (f"oracle FP64 FMM, full evaluation of {n_sample} particles of the same distribution, p={w['p']}, "
            f"leaf {w['leaf_size']} (depth {oracle.uniform_depth(n_sample, w['leaf_size'])}, mean leaf occupancy "
            f"32 as in the full workload)")


def oracle_one_thread(w) -> dict:
    """The oracle FMM on one host thread (the paper's single-core CPU convention), in a fresh
    interpreter with OMP_NUM_THREADS=1 (OpenMP reads it at start-up)."""
    code = (
        "import sys, time, json; sys.path.insert(0, %r)\n"
        "import oracle\n"
        "from paper_1010_1482_gb300 import inputs\n"
        "w = inputs.workload(%r)\n"
        "x = inputs.make_particles(%d, w['dist'], w['seed'])\n"
        "t0 = time.perf_counter()\n"
        "(oracle.fmm_adaptive(x, w['p'], w['leaf_size']) if w['tree'] == 'adaptive' else oracle.fmm(x, w['p'], w['leaf_size']))\n"
        "print(json.dumps({'dt': time.perf_counter() - t0, 'threads': oracle.threads()}))\n"
    ) % (ROOT, w["name"], CPU_ONE_CORE_N)
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
        d = json.loads(r.stdout.strip().splitlines()[-1])
    except Exception as e:  # reported, not fatal: the GPU line stands without it
        return {"error": str(e)[:200]}
    return {"value": CPU_ONE_CORE_N / d["dt"], "unit": UNIT, "cores": d["threads"],
            "sample": f"oracle FP64 FMM of {CPU_ONE_CORE_N} particles of the same distribution, p={w['p']}, "
                      f"leaf {w['leaf_size']}, one thread, {d['dt']:.1f} s"}


def run_reference(args, w):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle

    x = inputs.make_particles(CPU_SAMPLE_N, w["dist"], w["seed"])
    for _ in range(args.warmup):
        oracle_fmm(oracle, x, w)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_fmm(oracle, x, w)
    dt = time.perf_counter() - t0
    value = CPU_SAMPLE_N * args.steps / dt
    sample = oracle_sample_text(oracle, CPU_SAMPLE_N, w) + " per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["name"], "n": w["n"], "p": w["p"], "leaf_size": w["leaf_size"],
                   "distribution": w["dist"], "sample_n": CPU_SAMPLE_N},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------

def run_gpu(args, w):
    import torch

    from paper_1010_1482_gb300 import gbfmm as G

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    else:
        torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    G.lib()

    n = w["n"]
    adaptive = w["tree"] == "adaptive"
    tree_kind = G.TREE_ADAPTIVE if adaptive else G.TREE_UNIFORM
    x = inputs.make_particles(n, w["dist"], replica_seed(w["seed"], rank))
    fmm = G.FMM(local, p=w["p"], leaf_size=w["leaf_size"], tree=tree_kind, flags=G.FLAG_STAGE_TIMING)
    L, ws_bytes = fmm.plan(n)
    xd = torch.from_numpy(x).to(dev)
    out = torch.empty_like(xd)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    for _ in range(max(args.warmup, 3)):
        fmm.evaluate(xd, out)
    torch.cuda.synchronize()

    # algorithmic work of the dominant kernels (from this evaluation's own lists)
    if adaptive:
        tree = G.gbfmm_export_adaptive_tree(fmm.ctx, n)
        C = tree["ncells"]
        L = int(tree["level"].max())
        m2l_offs, _ = G.gbfmm_export_lists(fmm.ctx, G.LIST_V, C)
        p2p_offs, p2p_ids = G.gbfmm_export_lists(fmm.ctx, G.LIST_U, C)
        cnt_leaf = tree["count"].astype(np.int64)  # U rows of non-leaves are empty
        # block-form M2L units: the cells of levels >= 1 with children (the parents of the cells of
        # levels >= 2), 128 per tile
        deep = tree["level"] >= 2
        units = int(np.unique(tree["parent"][deep]).size)
    else:
        C = G.level_offset(L + 1)
        m2l_offs, _ = G.gbfmm_export_lists(fmm.ctx, G.LIST_M2L, C)
        tree = G.gbfmm_export_tree(fmm.ctx, n, C)
        p2p_offs, p2p_ids = G.gbfmm_export_lists(fmm.ctx, G.LIST_P2P, 8 ** L)
        cnt_leaf = tree["count"][G.level_offset(L): G.level_offset(L) + 8 ** L].astype(np.int64)
    m2l_pairs = int(m2l_offs[-1])
    cs = np.concatenate([[0], np.cumsum(tree["count"][p2p_ids[:p2p_offs[-1]]].astype(np.int64))])
    src_per_leaf = cs[p2p_offs[1:]] - cs[p2p_offs[:-1]]
    p2p_pairs = int(np.sum(cnt_leaf * src_per_leaf))
    P = w["p"]
    m2l_flops = m2l_pairs * 2 * P ** 4
    p2p_flops = p2p_pairs * 20

    step_ms, stage_acc, launches = [], {}, 0
    clock_ctx = ClockSampler(local) if rank == 0 else None
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()
    torch.cuda.synchronize()
    if clock_ctx:
        clock_ctx.__enter__()
    for _ in range(args.steps):
        flush.zero_()  # write 256 MiB (> 129 MB L2) so no step starts from a warm L2
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        G.gbfmm_evaluate(fmm.ctx, fmm.params, xd, out, fmm.workspace)
        e.record(stream)
        e.synchronize()
        step_ms.append(s.elapsed_time(e))
        for k, v in G.gbfmm_stage_times(fmm.ctx).items():
            stage_acc.setdefault(k, []).append(v)
        launches += G.gbfmm_last_launch_count(fmm.ctx)
    torch.cuda.synchronize()
    if clock_ctx:
        clock_ctx.__exit__()
    G.gbfmm_sync_status(fmm.ctx)
    total_ms = max_over_ranks(float(sum(step_ms)), dev)
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()
    ms_per_step = total_ms / args.steps
    value = job_rate(n, ws, total_ms, args.steps)
    stages = {k: float(np.mean(v)) for k, v in stage_acc.items()}

    # the FP32 CUDA-core M2L (Eq. 4 on the same lists) measured beside the tensor-core default
    cc_params = G.gbfmm_default_params(p=w["p"], leaf_size=w["leaf_size"], tree=tree_kind,
                                       flags=G.FLAG_STAGE_TIMING | G.FLAG_M2L_CUDA_CORES)
    cc_ms = []
    for i in range(4):
        flush.zero_()
        G.gbfmm_evaluate(fmm.ctx, cc_params, xd, out, fmm.workspace)
        torch.cuda.synchronize()
        if i > 0:
            cc_ms.append(G.gbfmm_stage_times(fmm.ctx)["M2L/M2P"])
    # the same evaluation with every stage on the caller's stream, one after another (P2P not
    # beside the expansions): per-kernel times without the other stream's interference
    ser_params = G.gbfmm_default_params(p=w["p"], leaf_size=w["leaf_size"], tree=tree_kind,
                                        flags=G.FLAG_STAGE_TIMING | G.FLAG_SERIAL)
    ser_ms, ser_acc = [], {}
    for i in range(4):
        flush.zero_()
        s0, e0 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        G.gbfmm_evaluate(fmm.ctx, ser_params, xd, out, fmm.workspace)
        e0.record(stream)
        e0.synchronize()
        if i > 0:
            ser_ms.append(s0.elapsed_time(e0))
            for k, v in G.gbfmm_stage_times(fmm.ctx).items():
                ser_acc.setdefault(k, []).append(v)
    ser_stages = {k: float(np.median(v)) for k, v in ser_acc.items()}
    G.gbfmm_evaluate(fmm.ctx, fmm.params, xd, out, fmm.workspace)  # leave the default result in `out`
    torch.cuda.synchronize()

    # end to end through the host-buffer ABI call (pinned host memory, copies in the timed region)
    hin = torch.from_numpy(x).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    for _ in range(2):
        G.gbfmm_evaluate_host(fmm.ctx, fmm.params, hin, hout)
    torch.cuda.synchronize()
    e2e_ms = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        G.gbfmm_evaluate_host(fmm.ctx, fmm.params, hin, hout)  # waits for the result on the host
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_total = max_over_ranks(float(sum(e2e_ms)), dev)
    e2e_value = job_rate(n, ws, e2e_total, args.steps)

    peak, peak_mhz = fp32_peak_tflops(torch.cuda.get_device_properties(dev).multi_processor_count)
    try:
        hbm_peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except Exception:
        hbm_peak = 6800.0
    # keys: 32-bit leaf keys (uniform tree) or 63-bit keys at depth 21 (adaptive tree)
    kb = 8 if adaptive else 4
    sort_passes = 8 if adaptive else -(-(3 * L) // 8)
    sort_bytes = sort_passes * 2 * (kb + 4) + kb + 32
    box_bytes = 16 + kb + 4
    m2l_ms = stages.get("M2L/M2P", float("nan"))
    m2l_tf = m2l_flops / (m2l_ms / 1e3) / 1e12
    p2p_tf = p2p_flops / (stages["P2P"] / 1e3) / 1e12
    try:
        bf16 = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
        tpeak, tbasis = bf16, f"measured BF16 dense burst {bf16:.1f} TFLOP/s (FP16 dense has the same nominal rate; of measured)"
    except Exception:
        tpeak, tbasis = 1900.0, "fallback 1900 TFLOP/s dense FP16/BF16 (of fallback)"
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    nt = {4: 128, 6: 144, 8: 256, 10: 208}[P]
    nstride = 200 if P == 10 else nt
    kd = 8 * P * P
    ntiles_n = -(-kd // nstride)
    if adaptive:
        # block kernel over units: per tile 128 units (MMA M) x NT outputs over the 26 parent
        # offsets, K = 8 p^2 per offset (colleagues' children gathered); 3 MMAs per product;
        # offset ranges per tile from the particle count (m2l_ablk_ksplit)
        ablk_tiles = -(-units // 128) * ntiles_n
        est = -(-(n // (4 * w["leaf_size"]) + 1) // 128) * ntiles_n
        ksplit = 1 if est >= 152 else min(26, -(-304 // est))
        kname, ksrc, kprof = "k_m2l_ablk", "m2l_blk.cu", f"m2l_ablk_{w['name']}.md"
        tensor_flops = ablk_tiles * 26 * kd * 3 * 2 * 128 * nt
        m2l_launches = -(-(ablk_tiles * ksplit) // sms)
        kshape = (f"{ablk_tiles} tiles of 128 units (cells with children) x {nt} outputs (of 8p^2 = {kd}), K = {kd} "
                  f"per parent offset, 26 offsets, offsets split over {ksplit} CTA(s) per tile; the M2L stage "
                  "also holds P2L over the X lists")
    else:
        # block kernel: per tile 128 target parents (MMA M) x NT outputs (MMA N) over the 26 parent
        # offsets, K = 8 p^2 per offset; 3 MMAs per product
        blk_tiles = sum(max(1, 8 ** (l - 1) // 128) * ntiles_n for l in range(2, L + 1))
        ksplit = 1 if blk_tiles >= 152 else min(26, -(-304 // blk_tiles))
        kname, ksrc, kprof = "k_m2l_blk", "m2l_blk.cu", f"m2l_blk_{w['name']}.md"
        tensor_flops = blk_tiles * 26 * kd * 3 * 2 * 128 * nt
        m2l_launches = -(-(blk_tiles * ksplit) // sms)
        kshape = (f"{blk_tiles} tiles of 128 target parents x {nt} outputs (of 8p^2 = {kd}), K = {kd} per parent "
                  f"offset, 26 offsets, offsets split over {ksplit} CTA(s) per tile")
    traffic = traffic_from_profile(ksrc, kprof, kname)
    m2l_roof = {"kernel": kname, "bound": "tensor", "achieved": m2l_tf, "peak": tpeak, "unit": "TFLOP/s",
                "frac": m2l_tf / tpeak,
                "traffic": traffic,
                "launches_per_evaluation": m2l_launches,
                "work": f"{m2l_pairs} M2L pairs x 2p^4 = {m2l_flops:.4g} flop per evaluation, "
                        f"{m2l_flops / m2l_launches:.4g} per launch ({m2l_launches} launch(es) of <= {sms} CTAs); "
                        "achieved = flop / the launches' summed duration",
                "shape": kshape,
                "peak_basis": tbasis,
                "tensor_flop_issued": tensor_flops,
                "tensor_pipe_frac": tensor_flops / (m2l_ms / 1e3) / 1e12 / tpeak,
                "achieved_alone": m2l_flops / (ser_stages["M2L/M2P"] / 1e3) / 1e12,
                "frac_alone": m2l_flops / (ser_stages["M2L/M2P"] / 1e3) / 1e12 / tpeak,
                "tensor_pipe_frac_alone": tensor_flops / (ser_stages["M2L/M2P"] / 1e3) / 1e12 / tpeak,
                "measured": "achieved: CUDA events around the M2L launches on their stream in the timed "
                            "steps (P2P runs beside it on a second stream); alone: the serial evaluation",
                "traffic_basis": "DRAM bytes per launch from the ncu capture in profiles/ (ncu starts each "
                                 "launch from a cold L2); null if the kernel source changed since",
                "note": "FP32-accurate products as 3 FP16 MMAs (hi*hi + lo*hi + hi*lo): frac <= 1/3 by "
                        "construction; tensor_pipe_frac counts every issued MMA flop"}
    p2p_alone = p2p_flops / (ser_stages["P2P"] / 1e3) / 1e12
    p2p_roof = {"kernel": "k_p2p_ws", "bound": "alu", "achieved": p2p_tf, "peak": peak, "unit": "TFLOP/s",
                "frac": p2p_tf / peak,
                "traffic": traffic_from_profile("p2p.cu", f"p2p_{w['name']}.md", "k_p2p_ws"),
                "launches_per_evaluation": 1,
                "work": f"{p2p_pairs} pairs x 20 flop (the paper's 19 + 1 for phi) = {p2p_flops:.4g} flop per "
                        "evaluation, one launch",
                "pairs": p2p_pairs, "flop_per_pair": 20,
                "achieved_alone": p2p_alone, "frac_alone": p2p_alone / peak,
                "measured": "achieved: CUDA events around the P2P launch on its stream (the low-priority "
                            "stream, beside P2M .. L2L) in the timed steps; alone: the serial evaluation",
                "peak_basis": f"derived FP32 CUDA-core peak: SMs x 128 FP32 lanes x 2 flop x {peak_mhz:.0f} MHz",
                "traffic_basis": "DRAM bytes per launch from the ncu capture in profiles/ (ncu starts each "
                                 "launch from a cold L2); null if the kernel source changed since",
                "note": "13 FP32-pipe operations + 1 reciprocal square root per pair: at 100% of the FP32 "
                        "pipe the 20-flop rate is 20/26 = 0.77 of the peak"}
    # the roofline follows the step's dominant kernel: the larger serial stage time
    p2p_dominant = ser_stages["P2P"] >= ser_stages["M2L/M2P"]
    roofline = dict(p2p_roof if p2p_dominant else m2l_roof)
    roofline["dominant_basis"] = (f"largest serial stage time: P2P {ser_stages['P2P']:.3f} ms, M2L/M2P "
                                  f"{ser_stages['M2L/M2P']:.3f} ms of the {float(np.median(ser_ms)):.3f} ms serial step")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": w["name"], "n": n, "p": P, "leaf_size": w["leaf_size"], "levels": L,
                   "tree": w["tree"], "cells": int(C), "distribution": w["dist"], "parallelism": f"replicas x{ws}",
                   "l2": "flushed between steps (256 MiB write outside the per-step events)"},
        "roofline": roofline,
        "kernels": {
            ("m2l" if p2p_dominant else "p2p"): (m2l_roof if p2p_dominant else p2p_roof),
            "m2l_fp32_cores": {"kernel": "k_m2l", "ms": float(np.median(cc_ms)),
                               "achieved_tflops": m2l_flops / (float(np.median(cc_ms)) / 1e3) / 1e12,
                               "frac": m2l_flops / (float(np.median(cc_ms)) / 1e3) / 1e12 / peak, "peak": peak,
                               "bound": "alu", "note": "same lists and Eq. 4 on the FP32 CUDA cores "
                                                       "(GBFMM_FLAG_M2L_CUDA_CORES), timed on the same data"},
            "box_keys": {"bytes_per_particle": box_bytes,
                         "achieved_gbs": box_bytes * n / (stages["box+keys"] / 1e3) / 1e9,
                         "peak_gbs": hbm_peak, "bound": "hbm",
                         "note": f"read x,y,z,q (16 B) for the box and again for the keys, write key + index "
                                 f"({kb + 4} B); the box read is counted once"},
            "sort": {"bytes_per_particle": sort_bytes, "achieved_gbs": sort_bytes * n / (stages["sort"] / 1e3) / 1e9,
                     "peak_gbs": hbm_peak, "bound": "hbm",
                     "note": f"one histogram read of the keys (4 B), {sort_passes} radix passes x (read key + index 8 B, "
                             "write 8 B), gather (16 B in, 16 B out)"},
        },
        "stages_ms": stages,
        "serial": {"ms_per_step": float(np.median(ser_ms)), "stages_ms": ser_stages,
                   "m2l_achieved": m2l_flops / (ser_stages["M2L/M2P"] / 1e3) / 1e12,
                   "note": "GBFMM_FLAG_SERIAL: every stage on one stream (the timed steps run P2P on a "
                           "second, low-priority stream beside P2M .. L2L; their stage times overlap)"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 16 * n, "d2h_bytes_per_step": 16 * n},
        "gpu_launches": launches,
        "clocks": clock_ctx.summary() if clock_ctx else None,
    }

    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle

        xs = inputs.make_particles(CPU_SAMPLE_N, w["dist"], w["seed"])
        t0 = time.perf_counter()
        oracle_fmm(oracle, xs, w)
        dt = time.perf_counter() - t0
        # accuracy of the timed result on seeded targets against the FP64 direct sum (the O(N^2)
        # oracle, timed: its full-N cost is extrapolated x N / targets)
        tg = inputs.sample_indices(n, ERROR_TARGETS, w["seed"])
        t1 = time.perf_counter()
        ref = oracle.direct(x, targets=tg)
        dt_direct = time.perf_counter() - t1
        got = out.cpu().numpy().astype(np.float64)[tg]
        line["error_vs_fp64_direct"] = {"targets": len(tg), "phi_rel_l2": oracle.rel_l2(got[:, 0], ref[:, 0]),
                                        "grad_rel_l2": oracle.rel_l2(got[:, 1:], ref[:, 1:])}
        line["cpu_baseline"] = {
            "value": CPU_SAMPLE_N / dt, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": oracle_sample_text(oracle, CPU_SAMPLE_N, w) + f", {dt:.1f} s (the reference arm's sample)",
            "one_core": oracle_one_thread(w),
            "direct": {"value": n / (dt_direct * n / len(tg)), "unit": UNIT, "cores": oracle.threads(),
                       "extrapolated": True,
                       "sample": f"oracle FP64 O(N^2) direct sum: {len(tg)} seeded targets over all {n} sources in "
                                 f"{dt_direct:.2f} s, full-N time extrapolated x N/{len(tg)}"},
        }
    if rank == 0 and ws == 1 and not args.no_serving:
        line.update(run_next_rows(args, G, dev, local))
    if rank == 0:
        print(json.dumps(line), flush=True)
    fmm.close()
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def run_next_rows(args, G, dev, local) -> dict:
    """Batched uneven instances (512 sets, N log-uniform in [1e3, 2e5], half uniform cube on the
    uniform octree and half Plummer on the adaptive one, p in {4, 8}) as one captured CUDA graph
    (gbfmm_batch_*) against the plain one-at-a-time evaluation and the engine's host workers, and
    a served Poisson request stream (200 req/s, N log-uniform in [1e3, 1e6], p in {4, 6, 10})
    with latency percentiles."""
    import torch

    from paper_1010_1482_gb300 import serving

    res = {}
    inst = inputs.batch_instances()
    x, offsets, params = serving.make_batch(inst, dev)
    total = int(offsets[-1])
    ctx = G.gbfmm_create(local)
    serving.run_plain(ctx, x, offsets, params)  # warm-up (operator tables, workspace)
    t_plain, out_plain = serving.run_plain(ctx, x, offsets, params)

    def graph_batch(prms, ref, lanes=64, reps=10):
        """Create the batch's graph (timed on the host), replay it `reps` times (CUDA events per
        replay, median), compare with the plain outputs, then refill the arrays with another
        sample of the same counts and compare one replay with that sample's plain outputs."""
        out = torch.empty_like(x)
        t0 = time.perf_counter()
        b = G.gbfmm_batch_create(ctx, offsets, prms, x, out, lanes=lanes)
        create_s = time.perf_counter() - t0
        nl, nodes = G.gbfmm_batch_info(b)
        for _ in range(3):
            G.gbfmm_batch_launch(ctx, b)
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            G.gbfmm_batch_launch(ctx, b)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        G.gbfmm_sync_status(ctx)
        same = bool(torch.equal(out, ref))
        x_keep = x.clone()
        x2, off2, _ = serving.make_batch([dict(r, seed=r["seed"] + 10 ** 6) for r in inst], dev)
        assert np.array_equal(off2, offsets)
        x.copy_(x2)
        G.gbfmm_batch_launch(ctx, b)
        G.gbfmm_sync_status(ctx)
        _, ref2 = serving.run_plain(ctx, x, offsets, prms)
        same2 = bool(torch.equal(out, ref2))
        x.copy_(x_keep)
        G.gbfmm_batch_destroy(b)
        ms = float(np.median(ts))
        return {"lanes": nl, "kernel_nodes": nodes, "create_s": create_s, "replay_ms": ms,
                "batched_particles_per_s": total / (ms / 1e3), "identical_to_plain": same,
                "new_sample_identical_to_plain": same2}, out

    g64, out_g = graph_batch(params, out_plain)
    # the engine: independent gbfmm_evaluate calls on host worker threads (contexts, streams)
    e = G.gbfmm_engine_create(local, args.workers, 40 << 30)
    G.gbfmm_engine_prepare(e, [4, 6, 8, 10])
    out = torch.empty_like(x)
    G.gbfmm_engine_run_batch(e, offsets, params, x, out)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = G.gbfmm_engine_run_batch(e, offsets, params, x, out)
    torch.cuda.synchronize()
    t_engine = time.perf_counter() - t0
    res["batched"] = dict(g64, **{
        "instances": len(inst), "particles": total,
        "plain_particles_per_s": total / t_plain,
        "speedup_vs_plain": t_plain / (g64["replay_ms"] / 1e3),
        "engine_particles_per_s": total / t_engine, "engine_workers": args.workers,
        "engine_failed": int(sum(1 for v in st if v != 0)),
        "engine_identical_to_plain": bool(torch.equal(out, out_plain)),
        "note": "batched = one replay of the captured graph of all 512 instances (gbfmm_batch_launch), device time; "
                "plain = gbfmm_evaluate one instance at a time on one stream, wall clock; engine = "
                "gbfmm_engine_run_batch over host worker threads, wall clock; new_sample = the arrays refilled "
                "with another seeded sample of the same counts and replayed",
    })
    # the same batch with leaf sizes from the autotuner (gbfmm_tune_leaf per (distribution, p,
    # log2 N) bucket, candidates 32 / 64 / 128 / 256)
    leaves = serving.tune_leaves(ctx, x, offsets, inst)
    tparams = serving.tuned_params(inst, leaves)
    serving.run_plain(ctx, x, offsets, tparams)
    t_plain_t, out_plain_t = serving.run_plain(ctx, x, offsets, tparams)
    gt, _ = graph_batch(tparams, out_plain_t)
    # accuracy of both leaf choices on 8 instances, 256 seeded targets each, vs FP64 direct
    import oracle

    errs = {"leaf_64": [], "tuned": []}
    for i in range(0, len(inst), len(inst) // 8)[:8]:
        a, b = int(offsets[i]), int(offsets[i + 1])
        xs = x[a:b].cpu().numpy()
        tg = inputs.sample_indices(b - a, min(256, b - a), inputs.SEED_BASE + 9)
        ref = oracle.direct(xs, targets=tg)
        for name, o in (("leaf_64", out_plain), ("tuned", out_plain_t)):
            got = o[a:b].cpu().numpy().astype(np.float64)[tg]
            errs[name].append(oracle.rel_l2(got[:, 1:], ref[:, 1:]))
    res["batched_tuned"] = dict(gt, **{
        "leaf_sizes": {f"{d}/p{p}/2^{k}": v for (d, p, k), v in sorted(leaves.items())},
        "plain_particles_per_s": total / t_plain_t,
        "grad_err_max": {k: float(max(v)) for k, v in errs.items()},
    })
    G.gbfmm_destroy(ctx)
    del x, out, out_plain, out_plain_t, out_g
    res["graph"] = run_graph(G, dev, local)
    reqs = inputs.served_requests(duration=args.serve_seconds)
    warm = inputs.served_requests(duration=0.5, seed=inputs.SEED_BASE + 6)
    serving.run_stream(e, warm)
    keep = serving.keep_per_class(reqs, 4)
    stats, kept = serving.run_stream(e, reqs, keep=keep)
    G.gbfmm_engine_destroy(e)
    stats.update({"rate_per_s": 200.0, "duration_s": args.serve_seconds, "workers": args.workers,
                  "budget_bytes": 40 << 30,
                  "latency": "submit of host arrays -> result in host memory (copies included)",
                  "inputs": "each request an independent seeded particle set, generated by host threads ahead "
                            "of its arrival; late_* = submission behind the arrival schedule",
                  "error_per_class": serving.class_errors(reqs, kept, oracle.direct, oracle.rel_l2),
                  "error_basis": "grad phi / phi rel L2 vs the FP64 direct sum on 256 seeded targets, the first "
                                 "4 requests of each (distribution, p) class"})
    res["served"] = stats
    res["crossover"] = run_crossover(G, dev, local)
    res["sort_16m"] = run_sort_16m(G, dev, local)
    return res


def run_sort_16m(G, dev, local) -> dict:
    """Keys and sort of 16,777,216 particles: the uniform tree (leaf 64: depth 8, 24-bit keys, 3
    radix passes) and the adaptive tree of the Plummer set (63-bit keys, 8 passes), from the
    stage timing of serial evaluations (median of 3 after one warm-up)."""
    import torch

    out_rows = {}
    ctx = G.gbfmm_create(local)
    hbm = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    for name, dist, tree, kbytes, passes in (("uniform_16m", "uniform", G.TREE_UNIFORM, 4, 3),
                                             ("plummer_16m_adaptive", "plummer", G.TREE_ADAPTIVE, 8, 8)):
        n = 1 << 24
        xd = torch.from_numpy(inputs.make_particles(n, dist, inputs.SEED_BASE + 10)).to(dev)
        out = torch.empty_like(xd)
        prm = G.gbfmm_default_params(p=4, leaf_size=64, tree=tree, flags=G.FLAG_STAGE_TIMING)
        _, wsb = G.gbfmm_plan(prm, n)
        ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device=dev)
        sts = []
        for _ in range(4):
            G.gbfmm_evaluate(ctx, prm, xd, out, ws)
            torch.cuda.synchronize()
            sts.append(G.gbfmm_stage_times(ctx))
        G.gbfmm_sync_status(ctx)
        med = {k: float(np.median([st[k] for st in sts[1:]])) for k in ("box+keys", "sort", "cells+lists")}
        sort_bytes = kbytes + passes * 2 * (kbytes + 4) + 32
        out_rows[name] = {"n": n, "radix_passes": passes, "sort_ms": med["sort"], "sort_bytes_per_particle": sort_bytes,
                          "sort_achieved_gbs": sort_bytes * n / (med["sort"] / 1e3) / 1e9,
                          "sort_frac": sort_bytes * n / (med["sort"] / 1e3) / 1e9 / hbm,
                          "box_keys_ms": med["box+keys"], "cells_lists_ms": med["cells+lists"]}
        del xd, out, ws
    G.gbfmm_destroy(ctx)
    out_rows["note"] = ("algorithmic bytes: one histogram read of the keys, every pass reads and writes key + index, "
                        "the gather reads and writes 16 B; frac of the measured HBM copy rate")
    return out_rows


def run_graph(G, dev, local) -> dict:
    """The bench workload evaluated repeatedly in the same buffers: eager gbfmm_evaluate calls
    against replays of one captured CUDA graph (device time per evaluation, L2 not flushed)."""
    import torch

    w = inputs.workload("uniform_1m_p10")
    x = inputs.make_particles(w["n"], w["dist"], w["seed"])
    prm = G.gbfmm_default_params(p=w["p"], leaf_size=w["leaf_size"])
    _, wsb = G.gbfmm_plan(prm, w["n"])
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    xd = torch.from_numpy(x).to(dev)
    out = torch.empty_like(xd)
    ctx = G.gbfmm_create(local)
    g = G.gbfmm_graph_create(ctx, prm, xd, out, ws)
    reps = 20

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        for _ in range(reps):
            fn()
        ev[1].record()
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]) / reps

    eager = timed(lambda: G.gbfmm_evaluate(ctx, prm, xd, out, ws))
    ref = out.clone()
    graph = timed(lambda: G.gbfmm_graph_launch(g))
    G.gbfmm_sync_status(ctx)
    same = bool(torch.equal(out, ref))
    G.gbfmm_graph_destroy(g)
    G.gbfmm_destroy(ctx)
    return {"workload": w["name"], "eager_ms": eager, "graph_ms": graph, "identical": same,
            "note": "back-to-back evaluations of the same buffers on one stream (inputs resident)"}


def run_crossover(G, dev, local) -> dict:
    """Direct sum vs treecode vs FMM on the uniform cube (the paper's Fig. 4 comparison): device
    time of one evaluation and the gradient error vs FP64 direct on 256 seeded targets, for each
    method at p = 4, 6, 8, 10, leaf 64."""
    import torch

    import oracle

    rows = []
    ctx = G.gbfmm_create(local)
    for n in (4096, 32768, 262144, 1048576):
        x = inputs.uniform_cube(n, inputs.SEED_BASE + 7)
        xd = torch.from_numpy(x).to(dev)
        out = torch.empty_like(xd)
        tg = inputs.sample_indices(n, 256, inputs.SEED_BASE + 7)
        ref = oracle.direct(x, targets=tg)

        def timed(fn, reps=3):
            fn()
            torch.cuda.synchronize()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record()
            for _ in range(reps):
                fn()
            ev[1].record()
            torch.cuda.synchronize()
            return ev[0].elapsed_time(ev[1]) / reps

        ms = timed(lambda: G.gbfmm_direct(ctx, xd, xd, out), reps=1 if n > 300000 else 3)
        err = oracle.rel_l2(out.cpu().numpy().astype(np.float64)[tg, 1:], ref[:, 1:])
        rows.append({"n": n, "method": "direct", "p": None, "ms": ms, "grad_err": err})
        for method, name in ((G.METHOD_TREECODE, "treecode"), (G.METHOD_FMM, "fmm")):
            for p in (4, 6, 8, 10):
                prm = G.gbfmm_default_params(p=p, leaf_size=64, method=method)
                _, wsb = G.gbfmm_plan(prm, n)
                wsp = torch.empty(max(wsb, 256), dtype=torch.uint8, device=dev)
                ms = timed(lambda: G.gbfmm_evaluate(ctx, prm, xd, out, wsp))
                G.gbfmm_sync_status(ctx)
                err = oracle.rel_l2(out.cpu().numpy().astype(np.float64)[tg, 1:], ref[:, 1:])
                rows.append({"n": n, "method": name, "p": p, "ms": ms, "grad_err": err})
    G.gbfmm_destroy(ctx)
    best = {}
    for r in rows:
        if r["grad_err"] <= 1e-4:
            k = (r["n"], r["method"])
            if k not in best or r["ms"] < best[k]["ms"]:
                best[k] = r
    fastest = {str(n): min((v for (m, _), v in best.items() if m == n), key=lambda v: v["ms"])["method"]
               for n in sorted({r["n"] for r in rows})}
    return {"rows": rows, "fastest_at_1e-4": fastest,
            "note": "uniform cube, leaf 64, device time of one evaluation (CUDA events); the error bar is the "
                    "gradient rel L2 <= 1e-4 vs FP64 direct on 256 seeded targets"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gbfmm", choices=["gbfmm", "reference"])
    ap.add_argument("--workload", default="uniform_1m_p10")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="skip the batched and served measurements")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--workers", type=int, default=8)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    w = inputs.workload(args.workload)
    if args.impl == "reference":
        return run_reference(args, w)
    return run_gpu(args, w)


if __name__ == "__main__":
    sys.exit(main())
