"""Benchmark: short-range forces/s of the truncated FMM on the clustered
N = 128^3 set (70% of the particles in 2000 NFW haloes, 30% uniform; PM 128^3,
r_s = 1.25 cells, R_c = 4.5 r_s; solved with leaves <= 48, theta 0.35, p 6, the
setting that meets the 1e-4 RMS accuracy bar), one GB300.

One step = one pass of the whole short-range path over the resident particle
set: wrap + Morton keys, sort, octree, P2M/M2M, traversal, list grouping, M2L,
L2L, L2P + P2P, accelerations in input order.  L2 is flushed (a 512 MB write)
before every timed step.  `value` counts particles with forces per second of
device time (CUDA events on the launching stream); `e2e` repeats the step
through the host-buffer C entry point with the copies inside the timing.
`arms` times the metric's other arm on the same set in the same run (learned
acceptance with the committed network and 3xTF32 tensor-core M2L) and checks
both against the same FP64 accuracy sinks (their direct sums come from the
CPU-baseline leg, the one place this arm runs the oracle: it times the direct
sum on those sinks and on random ones; without it, accuracy is null); `kd_tree` times the ORB / k-d tree
variant (tree 1) with the same parameters and sinks.  The roofline's FP32 peak is
measured in the same process by the library's FMA probe.  `--split poly` runs
the polynomial truncation of Sec. 5 instead (accuracy against its own direct
sum).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "short-range forces/s, N=2M clustered, rms err≤1e-4: learned+TF32 vs plain"
UNIT = "forces/s"
FP32_LANES_PER_SM = 128
N_SM = 152
# FP32 work of one P2P pair inside the cut-off (FMA = 2 flop): separation (3),
# r^2 (1 mul + 2 fma = 5), rsqrt (1), u = r^2 r^-1 - R_c / 2 (1 fma = 2), the
# truncation factor S = exp2(r^2 k) Q(u) with Q of degree 9 (exponent 1 +
# exp2 1 + 9 fma 18 + product 1 = 21), -S m / r^3 (4), accumulation (3 fma = 6).
P2P_FLOPS_PER_PAIR = 42
# The same count for the polynomial split (Sec. 5): separation 3, r^2 5,
# rsqrt 1, r^-3 2, -(r^-3 + c0 + c1 r^2) m (1 fma + 1 add + 1 mul = 4),
# accumulation 6.
P2P_FLOPS_PER_PAIR_POLY = 21


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="nfw-2m")
    ap.add_argument("--n", type=int, default=0, help="same kind of set at another N (profiling only)")
    ap.add_argument("--theta", type=float, default=0.0, help="acceptance parameter (0: the workload's own)")
    ap.add_argument("--order", type=int, default=0, help="expansion order (0: the workload's own)")
    ap.add_argument("--leaf-max", type=int, default=0, help="octree leaf capacity (0: the workload's own)")
    ap.add_argument("--m2l-precision", type=int, default=0,
                    help="0 FP32 CUDA cores, 1 3xTF32 tensor cores, 2 BF16x3 tensor cores")
    ap.add_argument("--graph", type=int, default=0, help="1: the whole short-range call as one CUDA graph")
    ap.add_argument("--tuned", default="", help="autotuner cache (JSON) to take the launch shapes from")
    ap.add_argument("--m2l-tables", type=int, default=0, help="1: same-level M2L operators from the (level, offset) table")
    ap.add_argument("--mac", default="geometric", choices=["geometric", "learned"])
    ap.add_argument("--mlp-weights", default=os.path.join(ROOT, "paper_2006_14952_gb300", "weights", "mac_weights.bin"))
    ap.add_argument("--split", default="gauss", choices=["gauss", "poly"],
                    help="truncation of the force split: Gaussian (Sec. 2.2) or polynomial (Sec. 5)")
    ap.add_argument("--mutual", type=int, default=0, help="1: mutual (third-law) P2P")
    ap.add_argument("--kdk", type=int, default=1, help="1: also time the whole KDK step, direct and as one graph")
    ap.add_argument("--compare", type=int, default=1,
                    help="1: also time the metric's other arm (learned acceptance + 3xTF32 M2L) on the same set")
    ap.add_argument("--compare-theta", type=float, default=0.5, help="safety bound of the learned arm")
    ap.add_argument("--kd-compare", type=int, default=1,
                    help="1: also time the ORB / k-d tree variant (tree 1) with the same parameters and sinks")
    ap.add_argument("--tree", default="octree", choices=["octree", "kd"],
                    help="tree of the timed arm: Morton octree or the ORB / k-d tree (Sec. 2.1, Sec. 4)")
    ap.add_argument("--accuracy-sinks", type=int, default=20000)
    ap.add_argument("--cpu-seconds", type=float, default=25.0, help="target CPU time of the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_config(cfg, rank, ws):
    """Each rank solves its own seeded copy of the workload (replicas, weak scaling)."""
    import dataclasses

    return dataclasses.replace(cfg, seed=cfg.seed + rank) if ws > 1 else cfg


def max_over_ranks(x, device=None):
    """The largest of every rank's x (a float); x itself on one rank."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(ws, n, steps, seconds):
    """Units processed by all ranks per second of the slowest rank."""
    return ws * n * steps / seconds


def workload_desc(cfg):
    if cfg.kind == "nfw":
        return (f"{cfg.name}: N={cfg.n} in L=1, {int(cfg.halo_frac * 100)}% in {cfg.halo_count} NFW haloes "
                f"(dN/dM~M^-1.9 over 3 decades, c~U[5,15], truncated at r_200), rest uniform; PM {cfg.pm_grid}^3, "
                f"r_s={cfg.rs_cells} cells, R_c={cfg.rcut_rs} r_s")
    return f"{cfg.name}: N={cfg.n}, kind={cfg.kind}, PM {cfg.pm_grid}^3"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "25"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.25)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9 and parts[1].isdigit():
                    rows.append(parts)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"], "samples": 0}
        sm = [int(r[1]) for r in rows]
        smax = max(int(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        pw = [float(r[3]) for r in rows if r[3].replace(".", "", 1).isdigit()]
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": reasons, "samples": len(rows),
                "power_w_max": max(pw) if pw else None}


# ------------------------------------------------------------------ oracle (CPU)
def cpu_oracle_sample(pos, mass, cfg, target_s, seed=7, split="gauss", fixed_sinks=None):
    """Direct FP64 truncated sum (the oracle) on a bounded sink sample: the fixed
    sinks (the accuracy sinks, whose forces are returned as the reference of the
    accuracy checks) and random ones up to about target_s seconds in all.
    Returns (the baseline's record, the reference forces [3][len(fixed_sinks)] or None)."""
    import oracle

    oracle.build()
    n = pos.shape[1]
    probe = np.sort(np.random.default_rng(seed).choice(n, size=min(500, n), replace=False))
    t0 = time.perf_counter()
    oracle.direct_sr(pos, mass, cfg.box, cfg.rs, cfg.rc, sinks=probe, split=split)
    rate = min(n, 500) / max(time.perf_counter() - t0, 1e-3)  # sinks per second
    ref, k0, t_fixed = None, 0, 0.0
    if fixed_sinks is not None and len(fixed_sinks):
        k0 = len(fixed_sinks)
        t0 = time.perf_counter()
        ref = oracle.direct_sr(pos, mass, cfg.box, cfg.rs, cfg.rc, sinks=fixed_sinks, split=split)
        t_fixed = time.perf_counter() - t0
    k = int(min(n, max(500, rate * max(target_s - t_fixed, 0.0))))
    sinks = np.sort(np.random.default_rng(seed + 1).choice(n, size=k, replace=False))
    t0 = time.perf_counter()
    oracle.direct_sr(pos, mass, cfg.box, cfg.rs, cfg.rc, sinks=sinks, split=split)
    dt = time.perf_counter() - t0
    return ({"value": (k0 + k) / (t_fixed + dt), "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
             "sample": f"FP64 direct truncated sum (oracle) for {k0} fixed (accuracy) and {k} random sinks "
                       f"against all {n} sources, {t_fixed + dt:.1f} s"}, ref)


def run_reference(args, cfg):
    """The oracle as the reference arm: each step is a bounded sink sample."""
    from paper_2006_14952_gb300 import workloads as W
    import oracle

    ws, rank, _ = dist_env()
    if rank != 0:
        return
    oracle.build()
    pos, mass = W.make(cfg)
    n = pos.shape[1]
    k = 2000
    rng = np.random.default_rng(99)
    for _ in range(args.warmup):
        oracle.direct_sr(pos, mass, cfg.box, cfg.rs, cfg.rc, sinks=np.sort(rng.choice(n, 200, replace=False)))
    tot = 0.0
    for _ in range(args.steps):
        sinks = np.sort(rng.choice(n, k, replace=False))
        t0 = time.perf_counter()
        oracle.direct_sr(pos, mass, cfg.box, cfg.rs, cfg.rc, sinks=sinks)
        tot += time.perf_counter() - t0
    v = k * args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_desc(cfg), "reference": "FP64 CPU oracle, direct truncated sum"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"{k} random sinks per step against all {n} sources"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def src_sha(name):
    p = os.path.join(ROOT, "paper_2006_14952_gb300", "csrc", name)
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:16]


def measured_traffic(kernel, src):
    """DRAM bytes per launch from the committed ncu summary, if the kernel is unchanged since."""
    try:
        d = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
        e = d.get(kernel)
        if e and e.get("src_sha") == src_sha(src):
            return e["bytes_per_launch_full"]
    except Exception:
        pass
    return None


def accuracy_of(acc, sinks, ref, split="gauss"):
    """Per-particle relative force error against the FP64 direct sum on the sinks."""
    a = acc.cpu().numpy()[:, sinks].astype(np.float64)
    e = np.linalg.norm(a - ref, axis=0) / np.linalg.norm(ref, axis=0)
    what = "FP64 direct truncated sum" + (" (polynomial split)" if split == "poly" else "")
    return {"rms_rel": float(math.sqrt((e ** 2).mean())), "p99_rel": float(np.percentile(e, 99)),
            "max_rel": float(e.max()), "sinks": int(len(sinks)), "against": what}


def measured_fp32_peak():
    """FP32 fused multiply-add rate of this GPU (TFLOP/s), the larger of the
    scalar and packed FP32x2 probes (hfmm_alu_peak), with the clock it ran at."""
    from paper_2006_14952_gb300 import hfmm

    out = {}
    for kind in ("ffma", "ffma2", "ex2", "rsqrt"):
        best = 0.0
        for _ in range(3):
            r, _ms = hfmm.alu_peak(kind, 8192 if kind.startswith("ffma") else 2048)
            best = max(best, r)
        out[kind] = best / 1e12
    return out


def time_arm(hfmm, torch, common, wts, dpos, dmass, acc, flush, steps, warmup, stream):
    """Warm up, then time `steps` steps (tree build + short-range forces) with CUDA
    events; returns (step times in ms, per-step phase stats, launches in the timed steps)."""
    s = hfmm.Solver(profile=1, **common)
    if wts is not None:
        s.load_mlp(wts)

    def step():
        s.build_tree(dpos, dmass)
        s.short_range_forces(acc)

    for _ in range(warmup):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()
    l0 = s.get_stats()["launches"]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    phases = []
    for k in range(steps):
        flush.fill_(1.0)
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
        phases.append(s.get_stats())
    torch.cuda.synchronize()
    l1 = s.get_stats()["launches"]
    s.close()
    return [a.elapsed_time(b) for a, b in ev], phases, l1 - l0


def time_kdk(hfmm, torch, common, pos, mass, flush, steps, warmup, stream, graph):
    """The whole kick-drift-kick step (first kick, drift, tree build, short range,
    PM long range, second kick) from the same seeded start, by direct launches
    (graph 0) or as one CUDA graph (graph 1): step times in ms (CUDA events, L2
    flushed before each step), launches per timed step and the graph counters."""
    rng = np.random.default_rng(2718)
    dev = torch.device("cuda", torch.cuda.current_device())
    s = hfmm.Solver(**dict(common, use_graph=graph))
    p = torch.from_numpy(pos).to(dev)
    m = torch.from_numpy(mass).to(dev)
    v = torch.from_numpy((0.05 * rng.standard_normal(pos.shape)).astype(np.float32)).to(dev)
    s.build_tree(p, m)
    a = s.short_range_forces()
    s.pm_long_range(a)
    dt = 1e-4
    for _ in range(warmup):
        flush.fill_(1.0)
        s.step(p, v, a, dt)
    torch.cuda.synchronize()
    st0 = s.get_stats()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.fill_(1.0)
        ev[k][0].record(stream)
        s.step(p, v, a, dt)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    st1 = s.get_stats()
    s.close()
    return ([x.elapsed_time(y) for x, y in ev], (st1["launches"] - st0["launches"]) / steps,
            st1["step_graphs"] - st0["step_graphs"], st1["graph_captures"] - st0["graph_captures"])


def main():
    args = parse()
    from paper_2006_14952_gb300 import workloads as W

    cfg = W.CONFIGS[args.workload]
    if args.n:
        cfg = W.scaled(cfg, args.n)
    if args.leaf_max:
        cfg = W.dataclasses.replace(cfg, leaf_max=args.leaf_max)
    args.theta = args.theta or cfg.theta
    args.order = args.order or cfg.order
    if args.impl == "reference":
        run_reference(args, cfg)
        return

    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_2006_14952_gb300 import hfmm

    # replicas: every rank solves its own seeded copy of the workload (weak scaling)
    cfg_r = replica_config(cfg, rank, ws)
    pos, mass = W.make(cfg_r)
    n = pos.shape[1]
    # timed solver: phase events only (profile bit 0); the pair counts come from
    # one untimed run of a second context with counting on (bit 1)
    learned = args.mac == "learned"
    mac_kw = dict(mac_mode=1) if learned else {}
    tiles = {}
    if args.tuned:
        from paper_2006_14952_gb300 import autotune

        key = autotune.cache_key(torch.cuda.get_device_name(dev), cfg.name,
                                 dict(theta=args.theta, order=args.order, leaf_max=cfg.leaf_max,
                                      mac_mode=1 if learned else 0, m2l_precision=args.m2l_precision,
                                      m2l_tables=args.m2l_tables, pm_grid=cfg.pm_grid))
        tiles = autotune.lookup(args.tuned, key) or {}
    common = dict(pm_grid=cfg.pm_grid, rs_cells=cfg.rs_cells, rcut_rs=cfg.rcut_rs, theta=args.theta,
                  order=args.order, leaf_max=cfg.leaf_max, m2l_precision=args.m2l_precision,
                  m2l_tables=args.m2l_tables, use_graph=args.graph, split=1 if args.split == "poly" else 0,
                  p2p_mutual=args.mutual, tree=1 if args.tree == "kd" else 0,
                  **tiles, **mac_kw)
    wts = np.fromfile(args.mlp_weights, dtype=np.uint16) if learned else None
    s = hfmm.Solver(profile=1, **common)
    if learned:
        s.load_mlp(wts)
    dpos = torch.from_numpy(pos).to(dev)
    dmass = torch.from_numpy(mass).to(dev)
    acc = torch.empty((3, n), dtype=torch.float32, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        s.build_tree(dpos, dmass)
        s.short_range_forces(acc)

    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()
    sc = hfmm.Solver(profile=3, **common)
    if learned:
        sc.load_mlp(wts)
    sc.build_tree(dpos, dmass)
    sc.short_range_forces(torch.empty_like(acc))
    counts = sc.get_stats()
    sc.close()
    del sc

    # the accuracy sinks: their FP64 direct sums come from the CPU-baseline leg (rank 0,
    # after the GPU work); each arm keeps its accelerations until then
    sinks = W.subsample(n, args.accuracy_sinks, 2024) if args.accuracy_sinks > 0 else None

    # timed region
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    l0 = s.get_stats()["launches"]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    phases = []
    with ClockSampler(torch.cuda.current_device()) as clk:
        for k in range(args.steps):
            flush.fill_(1.0)
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
            phases.append(s.get_stats())  # synchronises; outside the events
        torch.cuda.synchronize()
    clocks = clk.summary()
    l1 = s.get_stats()["launches"]
    step_ms = [a.elapsed_time(b) for a, b in ev]
    tot_ms = sum(step_ms)
    tot_ms = max_over_ranks(tot_ms, dev)
    if ws > 1:
        torch.distributed.barrier()
    value = whole_job_rate(ws, n, args.steps, tot_ms / 1e3)

    # end to end through the host-buffer entry point, copies included
    pin_pos = torch.from_numpy(pos).pin_memory()
    pin_mass = torch.from_numpy(mass).pin_memory()
    pin_acc = torch.empty((3, n), dtype=torch.float32).pin_memory()
    s2 = hfmm.Solver(**common)
    if learned:
        s2.load_mlp(wts)
    for _ in range(2):
        s2.short_range_forces_host(pin_pos, pin_mass, pin_acc)
    e2e_s = 0.0
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2.short_range_forces_host(pin_pos, pin_mass, pin_acc)
        e2e_s += time.perf_counter() - t0
    e2e_v = whole_job_rate(ws, n, args.steps, max_over_ranks(e2e_s, dev))

    # phase breakdown (mean over timed steps) and the dominant kernel's roofline
    keys = ["t_keys_sort", "t_tree", "t_upward", "t_traverse", "t_lists", "t_m2l", "t_l2l", "t_p2p"]
    mean = {k: statistics.mean(p[k] for p in phases) for k in keys}
    st = counts
    derived_fp32 = N_SM * FP32_LANES_PER_SM * 2 * 2070e6 / 1e12
    alu = measured_fp32_peak()
    peak_fp32 = max(alu["ffma"], alu["ffma2"])
    peak_src = (f"measured: FP32 FMA probe (hfmm_alu_peak), max of scalar {alu['ffma']:.1f} and packed FP32x2 "
                f"{alu['ffma2']:.1f} TFLOP/s (derived at 2070 MHz: {derived_fp32:.1f})")
    if mean["t_p2p"] < 0:  # graph mode: the post-traversal phases are timed as one graph
        roof = {"kernel": "short-range graph (upward, walk, lists, M2L, L2L/L2P, P2P)", "bound": "alu", "achieved": None,
                "peak": peak_fp32, "unit": "TFLOP/s", "frac": None, "traffic": None,
                "note": "graph mode times the graph as a whole; run without --graph for the P2P roofline"}
    elif mean["t_p2p"] >= mean["t_m2l"]:
        fpp = P2P_FLOPS_PER_PAIR_POLY if args.split == "poly" else P2P_FLOPS_PER_PAIR
        flops = st["p2p_useful_pairs"] * fpp
        achieved = flops / (mean["t_p2p"] / 1e3) / 1e12
        kd_main = args.tree == "kd"
        roof = {"kernel": "k_kd_p2p (cut-off P2P on the k-d tree)" if kd_main else "k_p2p (cut-off P2P)",
                "bound": "alu", "achieved": achieved, "peak": peak_fp32,
                "unit": "TFLOP/s", "frac": achieved / peak_fp32,
                "traffic": measured_traffic("k_p2p", "p2p.cu") if args.split == "gauss" and not kd_main else None,
                "peak_source": peak_src,
                "algorithmic": f"{st['p2p_useful_pairs']} pairs inside R_c x {fpp} flop" + (
                    " (ordered pairs: the mutual kernel evaluates each unordered pair once and counts both "
                    "forces)" if args.mutual else ""),
                "mufu_peaks_tops": {"ex2": round(alu["ex2"], 3), "rsqrt": round(alu["rsqrt"], 3)}}
    else:
        p = args.order
        fl_pair = 2 * math.comb(p + 6, 6)  # for the learned path: counted at the largest order (an upper bound)
        achieved = st["nm2l"] * fl_pair / (mean["t_m2l"] / 1e3) / 1e12
        roof = {"kernel": f"k_m2l<{p}> (CUDA cores)", "bound": "alu", "achieved": achieved, "peak": peak_fp32,
                "unit": "TFLOP/s", "frac": achieved / peak_fp32,
                "traffic": measured_traffic("k_m2l", "m2l.cu"),
                "peak_source": peak_src,
                "algorithmic": f"{st['nm2l']} M2L pairs x {fl_pair} flop (2 C(p+6,6))"}

    # the metric's other arm on the same resident set and the same accuracy sinks:
    # learned acceptance with the committed network + 3xTF32 tensor-core M2L
    arms = None
    if args.compare and not learned and args.split == "gauss" and args.m2l_precision == 0:
        lcommon = dict(common, mac_mode=1, m2l_precision=1, theta=args.compare_theta, use_graph=0, p2p_mutual=0)
        lw = np.fromfile(args.mlp_weights, dtype=np.uint16)
        lacc = torch.empty_like(acc)
        l_ms, l_ph, _ = time_arm(hfmm, torch, lcommon, lw, dpos, dmass, lacc, flush, args.steps, args.warmup, stream)
        l_ms_tot = max_over_ranks(sum(l_ms), dev)
        lval = whole_job_rate(ws, n, args.steps, l_ms_tot / 1e3)
        lmean = {k[2:]: round(statistics.mean(p[k] for p in l_ph), 4) for k in keys}
        arms = {"plain": {"path": "geometric acceptance, FP32 CUDA-core M2L", "value": value,
                          "accuracy": None},
                "learned_tf32": {"path": f"learned acceptance (committed network, safety bound theta "
                                         f"{args.compare_theta}), 3xTF32 tensor-core M2L",
                                 "value": lval, "accuracy": None, "breakdown_ms": lmean,
                                 "ms_per_step": l_ms_tot / args.steps},
                "ratio_learned_tf32_over_plain": lval / value, "both_within_1e-4": None}

    # the ORB / k-d tree variant with the same parameters, on the same set and sinks
    kd_arm = None
    if args.kd_compare and args.tree == "octree" and not learned and args.split == "gauss" \
            and args.m2l_precision == 0 and not args.mutual and not args.m2l_tables and args.order <= 6:
        kcommon = dict(common, tree=1, use_graph=0)
        kacc = torch.empty_like(acc)
        k_ms, k_ph, k_launch = time_arm(hfmm, torch, kcommon, None, dpos, dmass, kacc, flush, args.steps,
                                        args.warmup, stream)
        k_tot = max_over_ranks(sum(k_ms), dev)
        kmean = {k[2:]: round(statistics.mean(p[k] for p in k_ph), 4) for k in keys}
        kst = k_ph[-1]
        # pair counts from one untimed statistics run (profile bit 1), for the k-d P2P roofline
        skc = hfmm.Solver(profile=3, **kcommon)
        skc.build_tree(dpos, dmass)
        skc.short_range_forces(torch.empty_like(acc))
        kcnt = skc.get_stats()
        skc.close()
        del skc
        k_ach = kcnt["p2p_useful_pairs"] * P2P_FLOPS_PER_PAIR / (kmean["p2p"] / 1e3) / 1e12
        kd_arm = {"path": "ORB / k-d tree (tree 1): median splits along the longest axis of the particles' "
                          "bounding box, box geometry in the acceptance rules, geometric acceptance, FP32 M2L",
                  "value": whole_job_rate(ws, n, args.steps, k_tot / 1e3), "unit": UNIT,
                  "ms_per_step": k_tot / args.steps,
                  "accuracy": None,
                  "ratio_over_octree": (whole_job_rate(ws, n, args.steps, k_tot / 1e3) / value),
                  "breakdown_ms": kmean, "launches_per_step": k_launch / args.steps,
                  "roofline": {"kernel": "k_kd_p2p (cut-off P2P on the k-d tree)", "bound": "alu",
                               "achieved": k_ach, "peak": peak_fp32, "unit": "TFLOP/s",
                               "frac": k_ach / peak_fp32, "traffic": None,
                               "algorithmic": f"{kcnt['p2p_useful_pairs']} pairs inside R_c x "
                                              f"{P2P_FLOPS_PER_PAIR} flop"},
                  "counts": {"nodes": kst["nnodes"], "leaves": kst["nleaves"], "levels": kst["nlevels"],
                             "walk_levels": kst["traverse_iters"], "p2p_leaf_pairs": kst["np2p"],
                             "m2l_pairs": kst["nm2l"], "frontier_pairs": kst["frontier_pairs"],
                             "p2p_pairs_on_lists": kcnt["p2p_particle_pairs"],
                             "p2p_pairs_useful": kcnt["p2p_useful_pairs"]}}

    # the whole KDK step (with the PM long range), direct and as one graph
    kdk = None
    if args.kdk and args.split == "gauss" and not learned and args.m2l_precision == 0 and not args.mutual:
        kdk = {"what": "kick, drift, tree build, short range, PM long range, kick (dt 1e-4 from a seeded "
                       "start with 0.05 rms velocities); L2 flushed before every step"}
        for mode in (0, 1):
            k_ms, k_launch, k_graphs, k_caps = time_kdk(hfmm, torch, dict(common, m2l_tables=0), pos, mass, flush,
                                                        args.steps, args.warmup, stream, mode)
            k_tot = max_over_ranks(sum(k_ms), dev)
            kdk["graph" if mode else "direct"] = {
                "ms_per_step": k_tot / args.steps, "value": whole_job_rate(ws, n, args.steps, k_tot / 1e3),
                "unit": UNIT, "launches_per_step": k_launch, "step_ms": [round(x, 4) for x in k_ms],
                **({"steps_as_one_graph": k_graphs, "captures": k_caps} if mode else {})}

    # the CPU-baseline leg: the oracle's direct sum on a bounded sample that holds the
    # accuracy sinks, whose forces then check every arm (rank 0 at N = 1, after the GPU work)
    cpu = accuracy = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu, ref = cpu_oracle_sample(pos, mass, cfg, args.cpu_seconds, split=args.split, fixed_sinks=sinks)
        if ref is not None:
            accuracy = accuracy_of(acc, sinks, ref, args.split)
            if arms is not None:
                l_acc = accuracy_of(lacc, sinks, ref)
                arms["plain"]["accuracy"] = accuracy
                arms["learned_tf32"]["accuracy"] = l_acc
                arms["both_within_1e-4"] = bool(accuracy["rms_rel"] <= 1e-4 and l_acc["rms_rel"] <= 1e-4)
            if kd_arm is not None:
                kd_arm["accuracy"] = accuracy_of(kacc, sinks, ref)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_desc(cfg),
                       "split": "polynomial (Sec. 5)" if args.split == "poly" else "Gaussian (Sec. 2.2)",
                       "p2p": "mutual (third law)" if args.mutual else "one-sided",
                       "tree": "ORB / k-d tree" if args.tree == "kd" else "Morton octree",
                       "path": ("learned acceptance (network, safety bound theta), " if learned else
                                "geometric acceptance, ") + (
                           {1: "3xTF32 tensor-core M2L", 2: "BF16x3 tensor-core M2L"}.get(args.m2l_precision)
                           or "FP32 CUDA-core M2L" + (" with (level, offset) operator tables"
                                                      if args.m2l_tables else "")),
                       "theta": args.theta, "order": args.order, "leaf_max": cfg.leaf_max,
                       "transition_rule": 1, "size_rule": 1, "l2": "flushed (512 MB write) before every step",
                       "graph": bool(args.graph), "tiles": tiles or "defaults",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU"},
            "accuracy": accuracy,
            "arms": arms,
            "kdk_step": kdk,
            "kd_tree": kd_arm,
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": n * (24 + 4), "d2h_bytes_per_step": n * 12},
            "gpu_launches": int(l1 - l0 - 0),
            "clocks": clocks,
            "breakdown_ms": {k[2:]: round(v, 4) for k, v in mean.items()},
            # the same steps without the tree build (keys, sort, octree): forces per second of the
            # short-range call on an existing tree
            "excluding_tree": {"value": whole_job_rate(ws, n, 1, max(tot_ms / args.steps - mean["t_keys_sort"]
                                                                     - mean["t_tree"], 1e-9) / 1e3),
                               "unit": UNIT, "ms_per_step": tot_ms / args.steps - mean["t_keys_sort"] - mean["t_tree"]},
            "counts": {"nodes": st["nnodes"], "leaves": st["nleaves"], "levels": st["nlevels"],
                       "traverse_iters": st["traverse_iters"], "p2p_leaf_pairs": st["np2p"],
                       "m2l_pairs": st["nm2l"], "m2l_pairs_table": st["nm2l_table"], "frontier_pairs": st["frontier_pairs"],
                       "p2p_pairs_evaluated": st["p2p_particle_pairs"],
                       "p2p_pairs_useful": st["p2p_useful_pairs"]},
            "step_ms": [round(x, 4) for x in step_ms],
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
