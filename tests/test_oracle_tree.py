"""Pins for the oracle's Morton keys, octree and dual-tree traversal (Secs. 2.1, 2.3).

The keys are recomputed with the magic-number bit spreading (a different
algorithm from the oracle's bit loop), the tree by a recursive Python builder,
and the interaction lists are checked by brute force: every ordered particle
pair closer than R_c is covered exactly once, by one P2P leaf pair or one M2L
cell pair, and every list entry satisfies the three acceptance rules.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2006_14952_gb300 import workloads as W


def spread3(v):
    v = v.astype(np.uint64) & np.uint64(0x1FFFFF)
    v = (v | (v << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
    v = (v | (v << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
    v = (v | (v << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
    v = (v | (v << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
    v = (v | (v << np.uint64(2))) & np.uint64(0x1249249249249249)
    return v


def ref_keys(pos, box=1.0):
    w = pos - box * np.floor(pos / box)
    k = np.clip(np.floor(w / box * 2.0 ** 21), 0, 2 ** 21 - 1).astype(np.uint64)
    return (spread3(k[0]) << np.uint64(2)) | (spread3(k[1]) << np.uint64(1)) | spread3(k[2])


def ref_tree(keys_sorted, leaf_max):
    """Breadth-first octree over sorted keys, by recursion on prefixes."""
    levels = [[(0, 0, 0, 0, len(keys_sorted))]]  # (ix, iy, iz, first, count)
    out = []
    while levels[-1]:
        lev = len(levels) - 1
        nxt = []
        for (ix, iy, iz, f, c) in levels[-1]:
            kids = []
            if c > leaf_max and lev < 21:
                sh = np.uint64(3 * (21 - lev - 1))
                dig = ((keys_sorted[f:f + c] >> sh) & np.uint64(7)).astype(np.int64)
                for o in range(8):
                    sel = np.nonzero(dig == o)[0]
                    if len(sel):
                        kids.append((2 * ix + (o >> 2 & 1), 2 * iy + (o >> 1 & 1), 2 * iz + (o & 1), f + sel[0], len(sel)))
            out.append((lev, ix, iy, iz, f, c, len(kids)))
            nxt.extend(kids)
        levels.append(nxt)
    return out


@pytest.mark.parametrize("kind", ["uniform", "nfw"])
def test_keys_sort_and_tree_match_independent_builders(kind):
    n = 3000
    if kind == "uniform":
        pos, mass = W.uniform(n, 5)
    else:
        pos, mass = W.nfw_clustered(n, 20, 0.7, 6)
    pos[:, :3] = [[-0.25, 1.0, 2.5], [0.0, 0.999999999, -1e-18], [1.0 - 1e-17, 0.5, 3.0]]
    f = oracle.FMM(box=1.0, rs=0.01, rc=0.045, theta=0.5, order=3, leaf_max=16)
    f.build_tree(pos, mass)
    key, perm, xs = f.particles()
    k = ref_keys(pos)
    order = np.lexsort((np.arange(n), k))
    np.testing.assert_array_equal(perm, order)
    np.testing.assert_array_equal(key, k[order])
    nodes = f.nodes()
    ref = ref_tree(k[order], 16)
    assert len(ref) == len(nodes)
    for r, nd in zip(ref, nodes):
        assert tuple(int(v) for v in r) == (nd[0], nd[1], nd[2], nd[3], nd[4], nd[5], nd[7])
    # children are contiguous and partition the parent's particle range
    for nd in nodes:
        if nd[7]:
            ch = nodes[nd[6]:nd[6] + nd[7]]
            assert (ch[:, 0] == nd[0] + 1).all()
            assert ch[0, 4] == nd[4] and ch[:, 5].sum() == nd[5]
            assert (ch[1:, 4] == ch[:-1, 4] + ch[:-1, 5]).all()
        else:
            assert nd[5] <= 16 or nd[0] == 21
    # every particle lies inside its leaf
    for nd in nodes[nodes[:, 7] == 0]:
        h = 1.0 / 2 ** nd[0]
        x = xs[nd[4]:nd[4] + nd[5]]
        lo = nd[1:4] * h
        assert ((x >= lo - 1e-15) & (x <= lo + h + 1e-15)).all()


def test_depth_cap_with_coincident_particles():
    pos = np.full((3, 40), 0.3)
    mass = np.full(40, 1 / 40, dtype=np.float32)
    f = oracle.FMM(box=1.0, rs=0.01, rc=0.045, theta=0.5, order=2, leaf_max=16)
    f.build_tree(pos, mass)
    nodes = f.nodes()
    leaves = nodes[nodes[:, 7] == 0]
    assert len(leaves) == 1 and leaves[0, 0] == 21 and leaves[0, 5] == 40
    assert len(nodes) == 22


def _min_image(d, box=1.0):
    return d - box * np.round(d / box)


def _covered(f, xs_sorted):
    """Map (i, j, shift) -> number of covering list entries, over sorted particle indices."""
    nodes = f.nodes()
    p2p, m2l = f.lists()
    cov = {}
    for lst in (p2p, m2l):
        for a, b, s in lst:
            ia = range(nodes[a, 4], nodes[a, 4] + nodes[a, 5])
            ib = range(nodes[b, 4], nodes[b, 4] + nodes[b, 5])
            for i in ia:
                for j in ib:
                    cov[(i, j, s)] = cov.get((i, j, s), 0) + 1
    return cov


def _shift_index(d_raw, d_img, box=1.0):
    # x_i - (x_j + s L) = d_img  =>  s = (d_raw - d_img) / L
    s = np.round((d_raw - d_img) / box).astype(int)
    return (s[0] + 1) * 9 + (s[1] + 1) * 3 + (s[2] + 1)


@pytest.mark.parametrize("rule", [0, 1])
@pytest.mark.parametrize("theta,leaf", [(0.5, 4), (0.7, 1), (0.3, 8)])
def test_lists_cover_every_close_pair_exactly_once(rule, theta, leaf):
    n = 300
    pos, mass = W.nfw_clustered(n, 4, 0.6, 40 + leaf)
    rc = 0.2
    f = oracle.FMM(box=1.0, rs=rc / 4.5, rc=rc, theta=theta, order=2, leaf_max=leaf, transition_rule=rule)
    f.build_tree(pos, mass)
    f.traverse()
    _, _, xs = f.particles()
    cov = _covered(f, xs)
    assert max(cov.values()) == 1  # no (i, j, shift) counted twice
    close = 0
    for i in range(n):
        d_raw = xs[i][None, :] - xs
        d_img = _min_image(d_raw)
        r = np.sqrt((d_img ** 2).sum(1))
        for j in np.nonzero((r < rc) & (np.arange(n) != i))[0]:
            s = _shift_index(d_raw[j], d_img[j])
            assert cov.get((i, j, s), 0) == 1, (i, j, s)
            close += 1
    assert close > 1000


def _cell_geom(nd, box=1.0):
    h = box / 2 ** nd[0]
    return (nd[1:4] + 0.5) * h, h


@pytest.mark.parametrize("rule", [0, 1])
def test_every_list_entry_obeys_the_acceptance_rules(rule):
    cfg = W.scaled(W.CONFIGS["nfw-2m"], 6000, pm_grid=32)
    pos, mass = W.make(cfg)
    f = oracle.FMM(box=1.0, rs=cfg.rs, rc=cfg.rc, theta=0.5, order=2, leaf_max=16, transition_rule=rule)
    f.build_tree(pos, mass)
    f.traverse()
    nodes = f.nodes()
    p2p, m2l = f.lists()
    assert len(m2l) > 0 and len(p2p) > 0
    shifts = np.array(list(itertools.product([-1, 0, 1], repeat=3)), dtype=float)
    rc = cfg.rc
    for lst, is_m2l in ((m2l, True), (p2p, False)):
        for a, b, s in lst[:: max(1, len(lst) // 3000)]:
            za, ha = _cell_geom(nodes[a])
            zb, hb = _cell_geom(nodes[b])
            dv = np.abs(zb + shifts[s] - za)
            sc = np.sqrt((dv ** 2).sum())
            sm = np.sqrt((np.maximum(dv - (ha + hb) / 2, 0) ** 2).sum())
            smax = np.sqrt(((dv + (ha + hb) / 2) ** 2).sum())
            assert sm <= rc * (1 + 1e-12)
            trans = (sc > rc) if rule == 0 else (smax > rc)
            hl = max(ha, hb)  # theta = L / S_c with L the larger side of the pair
            accept = (not trans) and hl <= 0.5 * sc * (1 + 1e-12)
            if is_m2l:
                assert accept
            else:
                assert nodes[a, 7] == 0 and nodes[b, 7] == 0 and not (
                    (not trans) and hl < 0.5 * sc * (1 - 1e-12))


def test_theta_zero_gives_no_m2l():
    pos, mass = W.uniform(2000, 3)
    f = oracle.FMM(box=1.0, rs=0.02, rc=0.09, theta=0.0, order=2, leaf_max=8)
    f.build_tree(pos, mass)
    f.traverse()
    assert f.size("m2l") == 0 and f.size("p2p") > 0
