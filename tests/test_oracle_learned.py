"""Pins for the oracle half of the learned acceptance (an addition to the
opening-angle rule of Sec. 2.3) and for the per-pair M2L error that labels its
training data:

- the 12 pair features on hand-computed configurations (point masses in
  known cells, their dipoles and quadrupoles, a periodic image, cells of
  different levels);
- the network's forward bound contains every FP32 evaluation an independent
  numpy emulation produces (random summation orders, perturbed features);
- the learned walk with networks whose decision is known in advance: always
  open equals the geometric walk at theta 0, always the top class equals the
  geometric walk at the safety angle, a network graded by S_c / R_c gives the
  orders its logits fix; every close particle pair is covered exactly once;
- the per-pair M2L error against an independent evaluation: the truncated
  Taylor series of the printed force law along each sink-source ray, taken at
  high precision with mpmath.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2006_14952_gb300 import workloads as W


# ---------------------------------------------------------------- features
def _hand_tree():
    # box 1, leaves of at most one particle: level-1 octants (0,0,0) and (1,0,0)
    # hold one particle each, octant (1,1,0) holds two and splits to level 2
    pos = np.array([[0.1, 0.1, 0.1], [0.6, 0.1, 0.1], [0.6, 0.6, 0.1], [0.9, 0.9, 0.4]]).T.copy()
    mass = np.array([0.25, 0.5, 0.125, 0.125])
    f = oracle.FMM(box=1.0, rs=0.1, rc=0.45, theta=0.5, order=4, leaf_max=1)
    f.build_tree(pos, mass)
    f.upward()
    return f


def test_features_of_two_adjacent_point_masses():
    f = _hand_tree()
    a, b = f.find_node(1, 0, 0, 0), f.find_node(1, 1, 0, 0)
    got = f.pair_features([[a, b, 13]])[0]
    # centres (.25,.25,.25) and (.75,.25,.25), sides 0.5: S_c = 0.5, the cubes touch,
    # S_max = |(1, .5, .5)|; source particle at offset (-.15,-.15,-.15) = -0.3 sides
    # per axis: scaled dipole 0.3 per axis, scaled quadrupole 0.09/2 (xx) and 0.09 (xy)
    expect = [0.5 / 0.1, 0.0, math.sqrt(1.5) / 0.45, 1.0, 1.0, 1.0, 0.0, 1 / 16, 1 / 16,
              0.3 * math.sqrt(3), math.sqrt(3 * 0.045 ** 2 + 3 * 0.09 ** 2), 0.5 / 0.45]
    np.testing.assert_allclose(got, expect, rtol=1e-13, atol=1e-15)


def test_features_of_a_periodic_image():
    f = _hand_tree()
    a, b = f.find_node(1, 0, 0, 0), f.find_node(1, 1, 0, 0)
    # sink b, source a displaced by +L in y (shift index (0+1)*9 + (1+1)*3 + (0+1) = 16):
    # centre (.25, 1.25, .25) against (.75, .25, .25): offsets (-.5, 1, 0)
    got = f.pair_features([[b, a, 16]])[0]
    sc = math.sqrt(1.25)
    expect = [sc / 0.1, 0.5 / 0.1, math.sqrt(1.0 + 2.25 + 0.25) / 0.45, 0.5 / sc, 0.5 / sc, 0.5 / sc, 0.0,
              1 / 16, 1 / 16, 0.3 * math.sqrt(3), math.sqrt(3 * 0.045 ** 2 + 3 * 0.09 ** 2), sc / 0.45]
    np.testing.assert_allclose(got, expect, rtol=1e-13, atol=1e-15)


def test_features_across_levels_and_of_a_two_particle_cell():
    f = _hand_tree()
    a = f.find_node(1, 0, 0, 0)
    c = f.find_node(2, 2, 2, 0)  # side .25, centre (.625, .625, .125), holds (.6, .6, .1)
    got = f.pair_features([[a, c, 13]])[0]
    d = (0.375, 0.375, 0.125)
    sc = math.sqrt(sum(x * x for x in d))
    expect = [sc / 0.1, 0.0, math.sqrt(0.75 ** 2 * 2 + 0.5 ** 2) / 0.45, 0.5 / sc, 0.25 / sc, 0.5 / sc,
              (1 - 2) / 8, 1 / 16, 1 / 16, 0.1 * math.sqrt(3), math.sqrt(3 * 0.005 ** 2 + 3 * 0.01 ** 2), sc / 0.45]
    np.testing.assert_allclose(got, expect, rtol=1e-13, atol=1e-15)
    # the level-1 cell (1,1,0): centre (.75,.75,.25), side .5, masses 1/8 at offsets
    # (-.15,-.15,-.15) and (.15,.15,.15): the dipoles cancel, the quadrupoles add
    e = f.find_node(1, 1, 1, 0)
    got = f.pair_features([[a, e, 13]])[0]
    q = 2 * 0.125 * 0.09 / 0.25  # per (mass * (d/h)^m / m!) with d/h = +-0.3
    assert got[8] == pytest.approx(math.log2(3) / 16, rel=1e-15)
    assert got[9] == pytest.approx(0.0, abs=1e-15)
    assert got[10] == pytest.approx(math.sqrt(3 * (q / 2) ** 2 + 3 * q ** 2), rel=1e-13)


# ---------------------------------------------------------------- network bound
def _bf16(a):
    import torch

    return torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float32).numpy()


def _fp32_evaluation(w, x, rng):
    """The network in FP32 with the inputs and activations rounded to BF16, each
    unit's sum accumulated in a random order of its terms (bias included)."""
    def layer(Wm, bias, inp, hidden):
        out = np.zeros(Wm.shape[0], dtype=np.float32)
        for u in range(Wm.shape[0]):
            terms = np.concatenate([[bias[u]], Wm[u] * inp]).astype(np.float32)
            acc = np.float32(0.0)
            for t in terms[rng.permutation(len(terms))]:
                acc = np.float32(acc + t)
            out[u] = acc
        return _bf16(np.maximum(out, 0)) if hidden else out

    w32 = w.astype(np.float32)
    W1, b1 = w32[0:768].reshape(64, 12), w32[768:832]
    W2, b2 = w32[832:4928].reshape(64, 64), w32[4928:4992]
    W3, b3 = w32[4992:5504].reshape(8, 64), w32[5504:5512]
    h = layer(W1, b1, _bf16(x.astype(np.float32)), True)
    h = layer(W2, b2, h, True)
    return layer(W3, b3, h, False)


@pytest.mark.parametrize("rel,ab,sharp", [(2.0 ** -20, 2.0 ** -24, True), (1e-4, 1e-5, False)])
def test_forward_bound_contains_fp32_evaluations(rel, ab, sharp):
    rng = np.random.default_rng(11)
    w = np.vectorize(oracle.bf16)(rng.standard_normal(oracle.MLP_WEIGHTS) * 0.4)
    x = rng.uniform(0, 2, (300, 12))
    xtol = rel * np.abs(x) + ab
    lo, bound, cls, mask = oracle.mlp_forward_bound(w, x, xtol)
    if sharp:  # at the feature tolerance of an FP32 evaluation the bound stays small
        assert np.median(bound) < 1e-3 * np.abs(lo).max()
    ambiguous = 0
    for i in range(len(x)):
        for _ in range(3):
            xe = x[i] + rng.uniform(-1, 1, 12) * xtol[i]
            le = _fp32_evaluation(w, xe, rng).astype(np.float64)
            assert np.all(np.abs(le - lo[i]) <= bound[i]), (i, np.abs(le - lo[i]) / bound[i])
            k = int(np.argmax(le))
            assert (mask[i] >> k) & 1, i
        ambiguous += bin(int(mask[i])).count("1") > 1
        assert (mask[i] >> cls[i]) & 1
    assert ambiguous < (0.05 if sharp else 0.5) * len(x)


def test_forward_bound_without_tolerance_is_the_plain_forward():
    rng = np.random.default_rng(12)
    w = np.vectorize(oracle.bf16)(rng.standard_normal(oracle.MLP_WEIGHTS) * 0.4)
    x = rng.uniform(0, 2, (200, 12))
    lo, bound, cls, _ = oracle.mlp_forward_bound(w, x)
    np.testing.assert_allclose(lo, oracle.mlp_forward(w, x, rnd=1), rtol=0, atol=1e-12 * np.abs(lo).max())
    np.testing.assert_array_equal(cls, lo.argmax(axis=1))


# ---------------------------------------------------------------- learned walk
def _net_constant_class(k):
    w = np.zeros(oracle.MLP_WEIGHTS)
    w[5504 + k] = 1.0  # b3[k]: every logit 0 but class k's
    return w


def graded_weights():
    """logit_k = 16 k f - k^2 with f = S_c / R_c (feature 11), exact in BF16."""
    w = np.zeros(oracle.MLP_WEIGHTS)
    w[0 * 12 + 11] = 1.0
    w[832 + 0 * 64 + 0] = 1.0
    for k in range(8):
        w[832 + 4096 + 64 + k * 64] = 16.0 * k
        w[832 + 4096 + 64 + 512 + k] = -float(k * k)
    return w


TOL_REL = np.full(12, 2.0 ** -20)
TOL_ABS = np.full(12, 2.0 ** -24)


def _rows(a):
    return set(map(tuple, np.asarray(a).reshape(-1, np.asarray(a).shape[-1]).tolist()))


def _set_up(n=6000, order=6, theta=0.6, leaf=8, seed=5):
    pos, mass = W.nfw_clustered(n, 12, 0.7, seed)
    rs = 1.25 / 24
    f = oracle.FMM(box=1.0, rs=rs, rc=4.5 * rs, theta=theta, order=order, leaf_max=leaf)
    f.build_tree(pos, mass)
    return f, pos, mass, rs


def test_learned_walk_always_open_equals_the_geometric_walk_at_theta_zero():
    f, pos, mass, rs = _set_up()
    st = f.traverse_learned(_net_constant_class(0), TOL_REL, TOL_ABS)
    assert st["candidates"] > 1000 and st["ambiguous"] == 0
    p2p, m2l = f.lists()
    g = oracle.FMM(box=1.0, rs=rs, rc=4.5 * rs, theta=0.0, order=6, leaf_max=8)
    g.build_tree(pos, mass)
    g.traverse()
    gp, gm = g.lists()
    assert len(m2l) == 0 and len(gm) == 0
    assert _rows(p2p) == _rows(gp)


def test_learned_walk_top_class_equals_the_geometric_walk_at_the_safety_angle():
    f, *_ = _set_up()
    st = f.traverse_learned(_net_constant_class(7), TOL_REL, TOL_ABS)
    p2p, m2l = f.lists()
    orders = f.m2l_orders()
    f.traverse()
    gp, gm = f.lists()
    assert st["candidates"] == len(gm) > 1000
    assert _rows(p2p) == _rows(gp) and _rows(m2l) == _rows(gm)
    assert set(orders.tolist()) == {6}


def test_learned_walk_orders_follow_the_graded_logits():
    f, *_ = _set_up(order=8)
    st = f.traverse_learned(graded_weights(), TOL_REL, TOL_ABS)
    _, m2l = f.lists()
    orders = f.m2l_orders()
    nodes = f.nodes()
    assert len(m2l) > 500 and st["ambiguous"] < 0.01 * st["candidates"]
    # S_c / R_c from the integer cells, then the class the exact logits pick
    lev, ic = nodes[:, 0], nodes[:, 1:4]
    w = 2.0 ** (21 - lev)
    ca = 2 * ic[m2l[:, 0]] * w[m2l[:, 0], None] + w[m2l[:, 0], None]
    sv = np.stack([m2l[:, 2] // 9 - 1, (m2l[:, 2] // 3) % 3 - 1, m2l[:, 2] % 3 - 1], axis=1)
    cb = 2 * ic[m2l[:, 1]] * w[m2l[:, 1], None] + w[m2l[:, 1], None] + sv * 2.0 ** 22
    sc = np.sqrt(((cb - ca) ** 2).sum(1)) / 2.0 ** 22
    fb = _bf16(sc / f.rc).astype(np.float64)
    k = np.arange(8)
    logits = 16 * k[None, :] * fb[:, None] - k[None, :] ** 2
    kstar = logits.argmax(axis=1)
    clear = np.sort(logits, axis=1)[:, -1] > np.sort(logits, axis=1)[:, -2]
    assert clear.mean() > 0.95 and (kstar >= 1).all()
    np.testing.assert_array_equal(orders[clear], np.minimum(kstar[clear] + 1, 8))
    assert len(set(orders.tolist())) >= 3


def test_learned_walk_covers_every_close_pair_once():
    n = 400
    pos, mass = W.nfw_clustered(n, 4, 0.6, 43)
    rc = 0.2
    f = oracle.FMM(box=1.0, rs=rc / 4.5, rc=rc, theta=0.7, order=8, leaf_max=4)
    f.build_tree(pos, mass)
    f.traverse_learned(graded_weights(), TOL_REL, TOL_ABS)
    p2p, m2l = f.lists()
    assert len(m2l) > 0 and len(set(f.m2l_orders().tolist())) > 1
    nodes = f.nodes()
    _, _, xs = f.particles()
    cov = {}
    for lst in (p2p, m2l):
        for a, b, sh in lst:
            for i in range(nodes[a, 4], nodes[a, 4] + nodes[a, 5]):
                for j in range(nodes[b, 4], nodes[b, 4] + nodes[b, 5]):
                    cov[(i, j, sh)] = cov.get((i, j, sh), 0) + 1
    assert max(cov.values()) == 1
    for i in range(n):
        d_raw = xs[i][None, :] - xs
        d_img = d_raw - np.round(d_raw)
        r = np.sqrt((d_img ** 2).sum(1))
        for j in np.nonzero((r < rc) & (np.arange(n) != i))[0]:
            sv = np.round(d_raw[j] - d_img[j]).astype(int)
            sh = (sv[0] + 1) * 9 + (sv[1] + 1) * 3 + (sv[2] + 1)
            assert cov.get((i, j, sh), 0) == 1


# ---------------------------------------------------------------- per-pair M2L error
def _taylor_pair_error(xs, mass, za, zb, sv, idx_a, idx_b, rs, q):
    """sqrt(sum |a_q - a|^2 / sum |a|^2) over the sampled sinks, where a is the
    pair's direct sum with the printed force law (no cut-off: the pair's M2L is
    compared with the smooth kernel it approximates) and a_q the gradient of the
    order-q Taylor series of the potential about the centre offset R: component
    i is the order-(q-1) Taylor polynomial, along the ray R + t w, of the force
    law's i-th component, taken at t = 1 (w the particle offsets)."""
    import mpmath as mp

    mp.mp.dps = 40
    rs_m = mp.mpf(rs)

    def f1(r):  # f_(1)(r), the printed force prefactor
        x = r / (2 * rs_m)
        return -(mp.erfc(x) + r / (rs_m * mp.sqrt(mp.pi)) * mp.exp(-x * x)) / r ** 3

    R = [mp.mpf(za[d]) - (mp.mpf(zb[d]) + mp.mpf(sv[d])) for d in range(3)]
    num = den = 0.0
    for i in idx_a:
        u = [mp.mpf(xs[i, d]) - mp.mpf(za[d]) for d in range(3)]
        ex = np.zeros(3)
        ap = np.zeros(3)
        for j in idx_b:
            v = [mp.mpf(xs[j, d]) - mp.mpf(zb[d]) for d in range(3)]
            wv = [u[d] - v[d] for d in range(3)]
            y = [R[d] + wv[d] for d in range(3)]
            r = mp.sqrt(sum(t * t for t in y))
            fr = f1(r)
            for d in range(3):
                ex[d] += float(mass[j] * fr * y[d])

                def h(t, d=d):
                    yy = [R[e] + t * wv[e] for e in range(3)]
                    return f1(mp.sqrt(sum(s * s for s in yy))) * yy[d]

                c = mp.taylor(h, 0, q - 1)
                ap[d] += float(mass[j] * mp.fsum(c))
        num += float(((ap - ex) ** 2).sum())
        den += float((ex ** 2).sum())
    return math.sqrt(num / den)


def test_pair_error_matches_an_independent_taylor_evaluation():
    pytest.importorskip("mpmath")
    pos, mass = W.nfw_clustered(3000, 6, 0.6, 17)
    rs = 1.25 / 24
    f = oracle.FMM(box=1.0, rs=rs, rc=4.5 * rs, theta=0.7, order=8, leaf_max=6)
    f.build_tree(pos, mass)
    f.traverse()
    _, m2l = f.lists()
    nodes = f.nodes()
    _, perm, xs = f.particles()
    ms = mass[perm]
    rng = np.random.default_rng(9)
    picks = [t for t in rng.permutation(len(m2l)) if nodes[m2l[t, 0], 5] >= 3 and nodes[m2l[t, 1], 5] >= 2][:4]
    assert len(picks) == 4
    for t in picks:
        a, b, s = m2l[t]
        lev_a, lev_b = nodes[a, 0], nodes[b, 0]
        za = (nodes[a, 1:4] + 0.5) / 2.0 ** lev_a
        zb = (nodes[b, 1:4] + 0.5) / 2.0 ** lev_b
        sv = np.array([s // 9 - 1, (s // 3) % 3 - 1, s % 3 - 1], dtype=float)
        na = nodes[a, 5]
        ns = min(na, 32)
        idx_a = [nodes[a, 4] + (k * na) // ns for k in range(ns)]
        idx_b = list(range(nodes[b, 4], nodes[b, 4] + nodes[b, 5]))
        for q in (2, 4):
            ref = _taylor_pair_error(xs, ms, za, zb, sv, idx_a, idx_b, rs, q)
            got = f.pair_error(a, b, s, q)
            assert got == pytest.approx(ref, rel=1e-7), (t, q)
