"""Train the learned-acceptance network with the library's own kernels.

Pipeline (all on the GPU through the C ABI):
  1. training sets: seeded synthetic particle sets (a uniform set and a
     clustered set, smaller versions of the benchmark workloads);
  2. hfmm_collect_training_pairs on an order-8 context: features of sampled
     candidate pairs and the measured error of M2L at orders 2..8 against the
     pair's own direct sum;
  3. labels: the lowest order whose error is within the per-pair budget
     `eps` (class q - 1), or "open" (class 0) when none is;
  4. hfmm_mlp_grad + hfmm_mlp_adam for `steps` full-batch Adam steps.
The BF16 weights go to mac_weights.bin (5512 little-endian uint16) with a
JSON summary beside them.

    python -m paper_2006_14952_gb300.train_mac [--eps 3e-4] [--theta-safety 0.35] [--max-order 6]
                                               [--steps 500] [--out DIR]
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_OUT = os.path.join(HERE, "weights")


def make_sets(scale: float = 1.0):
    from . import workloads as W

    sets = [W.scaled(W.CONFIGS["uniform-32k"], 32768, seed=2001),
            W.scaled(W.CONFIGS["nfw-2m"], int(262144 * scale), halo_count=250, seed=2002),
            W.scaled(W.CONFIGS["nfw-2m"], int(262144 * scale), halo_count=250, halo_frac=0.85, seed=2003)]
    return sets


def collect(cfg, theta_safety: float, max_pairs: int, sample_mod: int):
    import torch

    from . import hfmm, workloads as W

    pos, mass = W.make(cfg)
    s = hfmm.Solver(pm_grid=cfg.pm_grid, rs_cells=cfg.rs_cells, rcut_rs=cfg.rcut_rs, order=8, theta=theta_safety,
                    leaf_max=cfg.leaf_max)
    s.build_tree(torch.from_numpy(pos).cuda(), torch.from_numpy(mass).cuda())
    feat, err = s.collect_training_pairs(max_pairs, sample_mod)
    torch.cuda.synchronize()
    return feat.clone(), err.clone()


def make_labels(err, eps: float, max_order: int = 8):
    import torch

    ok = err[:, : max_order - 1] <= eps  # [n][max_order - 1], orders 2..max_order
    first = torch.where(ok.any(dim=1), ok.float().argmax(dim=1) + 1, torch.zeros_like(ok[:, 0], dtype=torch.long))
    return first.to(torch.int32)  # 0 = open, k = order k + 1


def init_weights(seed: int):
    rng = np.random.default_rng(seed)
    w = np.zeros(5512, dtype=np.float32)
    o = 0
    for fan_in, fan_out in ((12, 64), (64, 64), (64, 8)):
        w[o:o + fan_in * fan_out] = rng.standard_normal(fan_in * fan_out) * np.sqrt(2.0 / fan_in)
        o += fan_in * fan_out
        o += fan_out  # biases start at zero
    return w


def train(x, y, steps: int, lr: float, seed: int = 7, log=None):
    import torch

    from . import hfmm

    ctx = hfmm.Solver()
    w = torch.from_numpy(init_weights(seed)).cuda()
    m1 = torch.zeros_like(w)
    m2 = torch.zeros_like(w)
    wb = torch.empty(5512, dtype=torch.bfloat16, device="cuda")
    counts = torch.bincount(y.long(), minlength=8).float()
    cw = torch.where(counts > 0, (counts.sum() / (8 * counts.clamp(min=1))) ** 0.5, torch.zeros_like(counts)).cuda()
    losses = []
    for step in range(1, steps + 1):
        grad, loss = ctx.mlp_grad(w, x, y, cw)
        hfmm.mlp_adam(grad, lr, step, w, m1, m2, wb)
        if step % 50 == 0 or step == steps:
            losses.append((step, float(loss.item())))
            if log:
                log(f"step {step} loss {losses[-1][1]:.4f}")
    return w, wb, losses, cw


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--eps", type=float, default=3e-4, help="per-pair relative error budget of an accepted M2L")
    ap.add_argument("--theta-safety", type=float, default=0.35)
    ap.add_argument("--max-order", type=int, default=6, help="largest order a label may choose")
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--max-pairs", type=int, default=200000)
    ap.add_argument("--sample-mod", type=int, default=7)
    ap.add_argument("--out", default=DEFAULT_OUT)
    args = ap.parse_args()
    import torch

    from . import hfmm

    t0 = time.time()
    xs, es = [], []
    for cfg in make_sets():
        f, e = collect(cfg, args.theta_safety, args.max_pairs, args.sample_mod)
        xs.append(f)
        es.append(e)
        print(f"{cfg.name}: {f.shape[0]} pairs", flush=True)
    x = torch.cat(xs).contiguous()
    err = torch.cat(es).contiguous()
    y = make_labels(err, args.eps, args.max_order).contiguous()
    hist = torch.bincount(y.long(), minlength=8).tolist()
    print("label histogram (open, q=2..8):", hist, flush=True)
    w, wb, losses, cw = train(x, y, args.steps, args.lr, log=lambda s: print(s, flush=True))
    logits, cls = hfmm.mlp_infer(wb, x)
    acc = float((cls == y).float().mean().item())
    # a decision is safe when it opens, or accepts an order whose measured error is within budget
    q = cls.long()
    q = q.clamp(max=args.max_order - 1)
    safe = (q == 0) | (err.gather(1, (q - 1).clamp(min=0).unsqueeze(1)).squeeze(1) <= args.eps)
    os.makedirs(args.out, exist_ok=True)
    wb.cpu().view(torch.int16).numpy().astype(np.int16).view(np.uint16).tofile(os.path.join(args.out, "mac_weights.bin"))
    meta = {"eps": args.eps, "theta_safety": args.theta_safety, "max_order": args.max_order,
            "pairs": int(x.shape[0]), "labels": hist,
            "train_accuracy": acc, "safe_fraction": float(safe.float().mean().item()), "losses": losses,
            "class_weights": cw.cpu().tolist(), "steps": args.steps, "lr": args.lr, "seconds": time.time() - t0,
            "sets": [c.name for c in make_sets()]}
    json.dump(meta, open(os.path.join(args.out, "mac_weights.json"), "w"), indent=1)
    print(json.dumps({k: v for k, v in meta.items() if k != "losses"}), flush=True)


if __name__ == "__main__":
    main()
