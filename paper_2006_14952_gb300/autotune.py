"""Autotuner for the launch shapes of the short-range solver.

The `tile_*` parameters of `hfmm_params` choose launch shapes that do not change
what is computed (only the FP32 summation order within a sink can move):

  tile_p2p_stage    source particles staged per P2P warp (128 or 256)
  tile_p2p_blocks   resident P2P blocks per SM (the persistent grid)
  tile_m2l_blocks   cap on M2L blocks per SM
  tile_trav_blocks  traversal blocks per SM (cooperative launch)

`tune()` times each knob's candidates on the caller's particle set through the
library's own per-phase CUDA events (profile bit 0), one knob at a time with the
others at their best so far (coordinate search), and returns the best setting
with the times it was chosen on.  `save()` / `lookup()` keep a JSON cache keyed
by GPU name, workload label and the solver parameters that change the work
(theta, order, leaf size, acceptance mode).

    python -m paper_2006_14952_gb300.autotune --workload nfw-2m \\
        --out paper_2006_14952_gb300/tuning/cache.json
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import time

# knob -> (candidates, the phase timing it is scored on); the first candidate is the default
KNOBS = {
    "tile_p2p_stage": ([256, 128], "t_p2p"),
    "tile_p2p_blocks": ([8, 4, 2], "t_p2p"),
    "tile_m2l_blocks": ([64, 16, 8, 4], "t_m2l"),
    "tile_trav_blocks": ([4, 3, 2], "t_traverse"),
}
# parameters that change the work (part of the cache key)
KEY_PARAMS = ("theta", "order", "leaf_max", "mac_mode", "m2l_precision", "m2l_tables", "pm_grid")


def cache_key(gpu: str, workload: str, params: dict) -> str:
    parts = [gpu, workload] + [f"{k}={params.get(k)}" for k in KEY_PARAMS]
    return "|".join(str(p) for p in parts)


def coordinate_search(measure, knobs=KNOBS):
    """measure(tiles: dict) -> {phase: ms}.  Returns (best tiles, {knob: {value: ms}})."""
    best = {k: v[0][0] for k, v in knobs.items()}
    trials = {}
    for knob, (values, phase) in knobs.items():
        res = {}
        for v in values:
            t = dict(best)
            t[knob] = v
            res[v] = measure(t)[phase]
        trials[knob] = res
        best[knob] = min(values, key=lambda v: (res[v], values.index(v)))
    return best, trials


def tune(pos, mass, params: dict, reps: int = 3, mlp_weights=None):
    """Tile setting for this particle set (device tensors pos [3][n] f64, mass [n] f32)."""
    import torch

    from . import hfmm

    def measure(tiles):
        s = hfmm.Solver(profile=1, **params, **tiles)
        if mlp_weights is not None:
            s.load_mlp(mlp_weights)
        s.build_tree(pos, mass)
        acc = torch.empty((3, pos.shape[1]), dtype=torch.float32, device=pos.device)
        s.short_range_forces(acc)  # warm-up (buffers, capacities)
        ts = {}
        for _ in range(reps):
            s.short_range_forces(acc)
            st = s.get_stats()
            for ph in ("t_p2p", "t_m2l", "t_traverse"):
                ts.setdefault(ph, []).append(st[ph])
        s.close()
        return {ph: statistics.median(v) for ph, v in ts.items()}

    return coordinate_search(measure)


def save(path: str, key: str, tiles: dict, trials: dict, extra: dict | None = None):
    data = {}
    if os.path.exists(path):
        with open(path) as f:
            data = json.load(f)
    data[key] = {"tiles": tiles, "trials_ms": {k: {str(v): t for v, t in r.items()} for k, r in trials.items()},
                 **(extra or {})}
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def lookup(path: str, key: str):
    """The cached tiles for `key`, or None."""
    if not os.path.exists(path):
        return None
    with open(path) as f:
        e = json.load(f).get(key)
    return None if e is None else {k: int(v) for k, v in e["tiles"].items()}


def main():
    import numpy as np
    import torch

    from . import workloads as W

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="nfw-2m", choices=sorted(W.CONFIGS))
    ap.add_argument("--theta", type=float, default=0.0, help="0: the workload's own")
    ap.add_argument("--order", type=int, default=0, help="0: the workload's own")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning",
                                                  "cache.json"))
    args = ap.parse_args()
    cfg = W.CONFIGS[args.workload]
    args.theta = args.theta or cfg.theta
    args.order = args.order or cfg.order
    pos, mass = W.make(cfg)
    params = dict(pm_grid=cfg.pm_grid, rs_cells=cfg.rs_cells, rcut_rs=cfg.rcut_rs, theta=args.theta,
                  order=args.order, leaf_max=cfg.leaf_max)
    t0 = time.time()
    best, trials = tune(torch.from_numpy(pos).cuda(), torch.from_numpy(np.asarray(mass)).cuda(), params, args.reps)
    gpu = torch.cuda.get_device_name(0)
    key = cache_key(gpu, args.workload, dict(params, mac_mode=0, m2l_precision=0, m2l_tables=0))
    save(args.out, key, best, trials, {"seconds": round(time.time() - t0, 1)})
    print(json.dumps({"key": key, "tiles": best, "trials_ms": trials}), flush=True)


if __name__ == "__main__":
    main()
