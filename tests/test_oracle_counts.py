"""Pins for the oracle's conventional-FMM walk, the baseline of the interaction
counts compared in Sec. 3 (Figs. 5-6).

A conventional FMM accepts a cell pair on the opening-angle test alone (Sec. 2.3,
second item), with no cut-off skip and no transition region, and walks the
primary box from (root, root).  Checked here against what fixes it independently
of the tree code: every ordered particle pair (a particle with itself included)
is covered exactly once; every entry obeys the test in floating point; theta = 0
leaves only leaf pairs; and on a complete lattice octree at theta = 1/2 the
counts equal the textbook interaction lists (a cell's M2L partners are the
children of its parent's neighbours that are not its own neighbours, 189 for an
interior cell; its P2P partners are its 27 neighbours including itself).
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2006_14952_gb300 import workloads as W


def _fmm(theta, leaf, rc=0.2, size_rule=1):
    return oracle.FMM(box=1.0, rs=rc / 4.5, rc=rc, theta=theta, order=2, leaf_max=leaf, size_rule=size_rule)


@pytest.mark.parametrize("theta,leaf", [(0.5, 4), (0.7, 1), (0.3, 8)])
def test_conventional_lists_cover_every_particle_pair_exactly_once(theta, leaf):
    n = 300
    pos, mass = W.nfw_clustered(n, 4, 0.6, 70 + leaf)
    f = _fmm(theta, leaf)
    f.build_tree(pos, mass)
    f.traverse(conventional=True)
    nodes = f.nodes()
    p2p, m2l = f.lists()
    assert len(m2l) > 0 and len(p2p) > 0
    assert (p2p[:, 2] == 13).all() and (m2l[:, 2] == 13).all()  # primary box only
    cov = np.zeros((n, n), dtype=np.int64)
    for lst in (p2p, m2l):
        for a, b, _ in lst:
            cov[nodes[a, 4]:nodes[a, 4] + nodes[a, 5], nodes[b, 4]:nodes[b, 4] + nodes[b, 5]] += 1
    assert (cov == 1).all()
    c = f.counts()
    assert c["m2l"] == len(m2l) and c["p2p"] == len(p2p)
    cnt = nodes[:, 5]
    assert c["p2p_particle_pairs"] + int((cnt[m2l[:, 0]] * cnt[m2l[:, 1]]).sum()) == n * n


@pytest.mark.parametrize("size_rule", [0, 1])
def test_conventional_entries_obey_the_opening_angle_test(size_rule):
    theta = 0.5
    pos, mass = W.nfw_clustered(4000, 12, 0.7, 77)
    f = _fmm(theta, 8, size_rule=size_rule)
    f.build_tree(pos, mass)
    f.traverse(conventional=True)
    nodes = f.nodes()
    p2p, m2l = f.lists()

    def geom(nd):
        h = 1.0 / 2 ** nd[0]
        return (nd[1:4] + 0.5) * h, h

    for lst, is_m2l in ((m2l, True), (p2p, False)):
        for a, b, _ in lst[:: max(1, len(lst) // 3000)]:
            za, ha = geom(nodes[a])
            zb, hb = geom(nodes[b])
            sc = np.sqrt(((zb - za) ** 2).sum())
            side = hb if size_rule == 0 else max(ha, hb)
            if is_m2l:
                assert side <= theta * sc * (1 + 1e-12)
            else:
                assert nodes[a, 7] == 0 and nodes[b, 7] == 0
                assert not side < theta * sc * (1 - 1e-12)


def test_conventional_theta_zero_leaves_only_leaf_pairs():
    pos, mass = W.uniform(1500, 8)
    f = _fmm(0.0, 8)
    f.build_tree(pos, mass)
    f.traverse(conventional=True)
    nodes = f.nodes()
    nleaves = int((nodes[:, 7] == 0).sum())
    assert f.counts() == {"m2l": 0, "p2p": nleaves * nleaves, "p2p_particle_pairs": 1500 * 1500}


def lattice_counts(k):
    """Textbook interaction-list counts of a complete octree of depth k (open
    boundary): per level, pairs whose parents are neighbours (or equal) while
    the cells are not; at the leaves, pairs of neighbours (or equal)."""
    m2l = 0
    for lev in range(1, k + 1):
        g = np.array(list(itertools.product(range(2 ** lev), repeat=3)))
        d = np.abs(g[:, None, :] - g[None, :, :]).max(axis=2)
        dp = np.abs(g[:, None, :] // 2 - g[None, :, :] // 2).max(axis=2)
        m2l += int(((dp <= 1) & (d >= 2)).sum())
    g = np.array(list(itertools.product(range(2 ** k), repeat=3)))
    p2p = int((np.abs(g[:, None, :] - g[None, :, :]).max(axis=2) <= 1).sum())
    return m2l, p2p


def lattice(k):
    n = 2 ** k
    g = (np.array(list(itertools.product(range(n), repeat=3))).T + 0.5) / n
    return g, np.full(n ** 3, 1.0 / n ** 3)


def test_conventional_counts_on_a_lattice_equal_the_textbook_interaction_lists():
    k = 3
    pos, mass = lattice(k)
    f = _fmm(0.5, 1)
    f.build_tree(pos, mass)
    assert f.size("levels") == k + 1
    f.traverse(conventional=True)
    m2l_ref, p2p_ref = lattice_counts(k)
    c = f.counts()
    assert (c["m2l"], c["p2p"], c["p2p_particle_pairs"]) == (m2l_ref, p2p_ref, p2p_ref)
    # an interior leaf: 189 M2L partners at its own level, 27 P2P partners
    nodes = f.nodes()
    p2p, m2l = f.lists()
    a = f.find_node(3, 3, 4, 3)
    lev_b = nodes[m2l[m2l[:, 0] == a, 1], 0]
    assert ((lev_b == 3).sum(), (p2p[:, 0] == a).sum()) == (189, 27)


def test_the_hybrid_walk_is_unchanged_by_the_conventional_one():
    pos, mass = W.nfw_clustered(3000, 10, 0.7, 79)
    f = _fmm(0.5, 4, rc=0.1)
    f.build_tree(pos, mass)
    f.traverse()
    h1 = f.counts()
    p1, m1 = f.lists()
    f.traverse(conventional=True)
    assert f.counts() != h1
    f.traverse()
    p2, m2 = f.lists()
    assert f.counts() == h1 and (p1 == p2).all() and (m1 == m2).all()
