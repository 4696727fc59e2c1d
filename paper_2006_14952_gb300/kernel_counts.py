"""Interaction counts of the truncated FMM against a conventional FMM (Sec. 3,
Figs. 5-6): M2L cell pairs and P2P pairs over the opening angle, for leaves of
one particle and of at most 32, on a uniform and on a clustered set.

The counts depend only on the tree and the acceptance criterion, so only the
GPU walk runs (``Solver.interaction_counts``), on the Morton octree or (``--tree
kd``) on the ORB / k-d tree the paper uses: the hybrid acceptance of Sec. 2.3
(cut-off skip, transition region, 27 nearest periodic images) and a
conventional FMM's (the opening-angle test alone, primary box from the root
pair).  The paper's sets (a uniform early-time box and a z = 0 snapshot) are
not available; seeded stand-ins of the same kinds are used.

    python -m paper_2006_14952_gb300.kernel_counts [--n 262144] [--pm-grid 64] [--tree kd]
"""
from __future__ import annotations

import argparse
import json
import sys


def sets(n: int, seed: int):
    from . import workloads as W

    return {
        "uniform": W.uniform(n, seed),
        "clustered": W.nfw_clustered(n, max(1, n // 1024), 0.85, seed + 1),
    }


def counts(pos, mass, leaf_max: int, theta: float, pm_grid: int, tree: int = 0) -> dict:
    import numpy as np
    import torch

    from . import hfmm

    s = hfmm.Solver(pm_grid=pm_grid, leaf_max=leaf_max, theta=theta, order=2, tree=tree)
    s.build_tree(torch.from_numpy(np.ascontiguousarray(pos)).cuda(), torch.from_numpy(mass).cuda())
    out = {"hybrid": s.interaction_counts(), "conventional": s.interaction_counts(conventional=True)}
    st = s.get_stats()
    out["nodes"], out["leaves"] = st["nnodes"], st["nleaves"]
    s.close()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=262144)
    ap.add_argument("--pm-grid", type=int, default=64)
    ap.add_argument("--seed", type=int, default=3001)
    ap.add_argument("--leaves", default="1,32")
    ap.add_argument("--thetas", default="0.3,0.4,0.5,0.6,0.7")
    ap.add_argument("--tree", default="octree", choices=["octree", "kd"],
                    help="Morton octree, or the ORB / k-d tree the paper's counts were taken on")
    args = ap.parse_args(argv)
    leaves = [int(x) for x in args.leaves.split(",")]
    thetas = [float(x) for x in args.thetas.split(",")]
    rows = []
    for name, (pos, mass) in sets(args.n, args.seed).items():
        for leaf in leaves:
            for th in thetas:
                c = counts(pos, mass, leaf, th, args.pm_grid, 1 if args.tree == "kd" else 0)
                row = {"set": name, "tree": args.tree, "n": args.n, "pm_grid": args.pm_grid, "leaf_max": leaf,
                       "theta": th, **c}
                rows.append(row)
                print(json.dumps(row), flush=True)
    print("\n| set | leaf | theta | M2L hybrid | M2L conventional | P2P leaf pairs hybrid | "
          "P2P leaf pairs conventional | P2P particle pairs hybrid | P2P particle pairs conventional |",
          file=sys.stderr)
    print("|---|---:|---:|---:|---:|---:|---:|---:|---:|", file=sys.stderr)
    for r in rows:
        h, c = r["hybrid"], r["conventional"]
        print(f"| {r['set']} | {r['leaf_max']} | {r['theta']} | {h['m2l']:.3e} | {c['m2l']:.3e} | {h['p2p']:.3e} | "
              f"{c['p2p']:.3e} | {h['p2p_particle_pairs']:.3e} | {c['p2p_particle_pairs']:.3e} |", file=sys.stderr)


if __name__ == "__main__":
    main()
