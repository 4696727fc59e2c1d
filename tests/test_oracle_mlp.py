"""Pins for the oracle's learned-acceptance pieces: BF16 rounding against
torch's conversion, a network whose weights make the logits equal the (BF16)
inputs, the backward pass against finite differences, the FMM on given lists
against the oracle's own FMM, and the per-pair M2L error falling with order."""
import numpy as np
import pytest

import oracle
from paper_2006_14952_gb300 import workloads as W


def test_bf16_rounding_matches_torch():
    import torch

    x = np.random.default_rng(0).standard_normal(2000) * 10.0 ** np.random.default_rng(1).uniform(-6, 6, 2000)
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([oracle.bf16(v) for v in x])
    np.testing.assert_array_equal(got, ref)


def passthrough_weights():
    w = np.zeros(oracle.MLP_WEIGHTS)
    W1 = w[0:768].reshape(64, 12)
    for k in range(12):
        W1[k, k] = 1.0
        W1[12 + k, k] = -1.0
    W2 = w[832:832 + 4096].reshape(64, 64)
    for k in range(24):
        W2[k, k] = 1.0
    W3 = w[832 + 4096 + 64:832 + 4096 + 64 + 512].reshape(8, 64)
    for o in range(8):
        W3[o, o] = 1.0
        W3[o, 12 + o] = -1.0
    return w


def test_forward_of_a_passthrough_network():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((50, 12))
    lo = oracle.mlp_forward(passthrough_weights(), x, rnd=0)
    np.testing.assert_allclose(lo, x[:, :8], rtol=0, atol=1e-15)
    lo1 = oracle.mlp_forward(passthrough_weights(), x, rnd=1)
    np.testing.assert_array_equal(lo1, np.vectorize(oracle.bf16)(x[:, :8]))


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(3)
    w = rng.standard_normal(oracle.MLP_WEIGHTS) * 0.3
    x = rng.standard_normal((40, 12))
    y = rng.integers(0, 8, 40)
    cw = rng.uniform(0.5, 2.0, 8)
    loss, g = oracle.mlp_loss_grad(w, x, y, cw, rnd=0)
    h = 1e-6
    for i in rng.choice(oracle.MLP_WEIGHTS, 60, replace=False).tolist() + [5511, 5504, 832, 0]:
        e = np.zeros_like(w)
        e[i] = h
        fd = (oracle.mlp_loss_grad(w + e, x, y, cw, rnd=0)[0] - oracle.mlp_loss_grad(w - e, x, y, cw, rnd=0)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-8), i


def test_fmm_on_given_lists_equals_own_fmm_and_orders_matter():
    cfg = W.scaled(W.CONFIGS["nfw-2m"], 8000, pm_grid=24, halo_count=10)
    pos, mass = W.make(cfg)
    f = oracle.FMM(box=1.0, rs=cfg.rs, rc=cfg.rc, theta=0.5, order=6, leaf_max=16)
    f.build_tree(pos, mass)
    ref = f.forces()
    p2p, m2l = f.lists()
    got = f.forces_given_lists(p2p, m2l, np.full(len(m2l), 6))
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    direct = oracle.direct_sr(pos, mass, 1.0, cfg.rs, cfg.rc)
    e6 = np.linalg.norm(got - direct) / np.linalg.norm(direct)
    e2 = np.linalg.norm(f.forces_given_lists(p2p, m2l, np.full(len(m2l), 2)) - direct) / np.linalg.norm(direct)
    assert e2 > 3 * e6


def test_pair_error_falls_with_order():
    cfg = W.scaled(W.CONFIGS["nfw-2m"], 8000, pm_grid=24, halo_count=10)
    pos, mass = W.make(cfg)
    f = oracle.FMM(box=1.0, rs=cfg.rs, rc=cfg.rc, theta=0.5, order=8, leaf_max=16)
    f.build_tree(pos, mass)
    f.traverse()
    _, m2l = f.lists()
    rng = np.random.default_rng(4)
    falls = 0
    for a, b, s in m2l[rng.choice(len(m2l), 30, replace=False)]:
        e = [f.pair_error(a, b, s, q) for q in range(2, 9)]
        assert all(e1 <= 1.05 * e0 for e0, e1 in zip(e, e[1:])), e  # non-increasing in q
        falls += e[-1] < 0.2 * e[0]
    assert falls >= 25
