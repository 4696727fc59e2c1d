"""Pins for the oracle's ORB / k-d tree variant (Sec. 2.1, Fig. 1: an ORB tree
with a leaf limiter whose cells split their particles almost equally between
two children; Sec. 4: a k-d tree inside each domain).

Checked against what fixes it independently of orc_kd.c:
  - the tree equals one built here from the definition with numpy (bounding
    boxes by min / max, split axis by argmax, halves by lexsort), node by node,
    box by box and particle by particle, also with coincident particles, tied
    coordinates, a single leaf and an empty set;
  - the walk's lists cover every ordered particle pair with its periodic shift
    at most once and every pair closer than R_c exactly once (brute force over
    all pairs and the 27 shifts); theta = 0 leaves only leaf pairs;
  - the FMM forces on the tree: theta = 0 gives the direct truncated sum up to
    rounding, the error falls with the order and is below 2e-6 at p = 8; the
    forces on the walk's own lists given back equal the forces of the walk.
"""
import numpy as np
import pytest

import oracle
from paper_2006_14952_gb300 import workloads as W

RS = 1.25 / 32
RC = 4.5 * RS


def _wrap(pos, box=1.0):
    q = np.floor(pos / box)
    return pos - box * q


def kd_reference(pos, leaf_max, box=1.0):
    """The tree from its definition: (nodes [k][5], boxes [k][6], perm [n])."""
    x = _wrap(np.asarray(pos, dtype=np.float64), box).T  # [n][3]
    n = len(x)
    order = np.arange(n)
    nodes, boxes = [], []
    if n == 0:
        return np.zeros((0, 5), np.int64), np.zeros((0, 6)), order
    level = [(0, n)]
    nodes.append([0, 0, n, -1, -1])
    start, lev = 0, 0
    while level:
        nxt = []
        for j, (f, c) in enumerate(level):
            k = start + j
            ids = order[f:f + c]
            lo, hi = x[ids].min(axis=0), x[ids].max(axis=0)
            boxes.append(np.concatenate([lo, hi]))
            if c <= leaf_max:
                continue
            ax = int(np.argmax(hi - lo))
            ids = ids[np.lexsort((ids, x[ids, ax]))]
            order[f:f + c] = ids
            nodes[k][3] = len(nodes)
            nodes[k][4] = ax
            for (cf, cc) in ((f, c // 2), (f + c // 2, c - c // 2)):
                nodes.append([lev + 1, cf, cc, -1, -1])
                nxt.append((cf, cc))
        start += len(level)
        level = nxt
        lev += 1
    nodes = np.array(nodes, dtype=np.int64)
    for k in np.nonzero(nodes[:, 3] < 0)[0]:
        f, c = nodes[k, 1], nodes[k, 2]
        ids = order[f:f + c]
        order[f:f + c] = ids[np.lexsort((ids, x[ids, 0]))]
    return nodes, np.array(boxes), order


def _kd(leaf, theta=0.5, order=4, rule=1, size_rule=1):
    return oracle.KdFMM(box=1.0, rs=RS, rc=RC, theta=theta, order=order, leaf_max=leaf,
                        transition_rule=rule, size_rule=size_rule)


def _sets():
    pos_u, m_u = W.uniform(700, 90)
    pos_c, m_c = W.nfw_clustered(900, 6, 0.7, 91)
    tied = np.round(W.uniform(600, 92)[0] * 8) / 8  # many equal coordinates and coincident points
    same = np.full((3, 40), 0.3)  # every particle at one point
    edge = np.array([[0.0, 1.0, -1e-300, 0.5, 1 - 2 ** -53, 3.25, -0.75],
                     [0.0, 0.999, 0.5, 2.0, 0.25, -3.5, 0.1],
                     [1e-300, 0.0, 0.5, 0.5, 0.75, 0.2, 0.9]])
    return {"uniform": (pos_u, m_u), "clustered": (pos_c, m_c), "tied": (tied, np.ones(600) / 600),
            "coincident": (same, np.ones(40) / 40), "edge": (edge, np.ones(7) / 7)}


@pytest.mark.parametrize("name", ["uniform", "clustered", "tied", "coincident", "edge"])
@pytest.mark.parametrize("leaf", [1, 4, 16, 64])
def test_tree_equals_the_definition(name, leaf):
    pos, mass = _sets()[name]
    f = _kd(leaf)
    f.build_tree(pos, mass)
    nodes, boxes, perm = f.tree()
    rn, rb, rp = kd_reference(pos, leaf)
    np.testing.assert_array_equal(nodes, rn)
    np.testing.assert_array_equal(boxes, rb)
    np.testing.assert_array_equal(perm, rp)
    assert f.size("levels") == (int(rn[:, 0].max()) + 1 if len(rn) else 0)


def test_tree_invariants_on_a_clustered_set():
    pos, mass = W.nfw_clustered(5000, 20, 0.7, 93)
    f = _kd(12)
    f.build_tree(pos, mass)
    nodes, boxes, perm = f.tree()
    x = _wrap(pos).T
    assert sorted(perm.tolist()) == list(range(5000))
    leaves = nodes[nodes[:, 3] < 0]
    assert (leaves[:, 2] <= 12).all() and (leaves[:, 2] >= 6).all()
    assert leaves[:, 2].sum() == 5000
    for k, (lev, first, cnt, ch, ax) in enumerate(nodes):
        ids = perm[first:first + cnt]
        np.testing.assert_array_equal(boxes[k, :3], x[ids].min(axis=0))
        np.testing.assert_array_equal(boxes[k, 3:], x[ids].max(axis=0))
        if ch < 0:
            continue
        a, b = nodes[ch], nodes[ch + 1]
        assert a[0] == b[0] == lev + 1 and a[1] == first and a[2] == cnt // 2 and b[1] == first + cnt // 2
        ext = boxes[k, 3:] - boxes[k, :3]
        assert ext[ax] == ext.max() and (ext[:ax] < ext[ax]).all()
        assert x[perm[a[1]:a[1] + a[2]], ax].max() <= x[perm[b[1]:b[1] + b[2]], ax].min()


def test_empty_set_and_single_leaf():
    f = _kd(16)
    f.build_tree(np.zeros((3, 0)), np.zeros(0))
    assert f.size("nodes") == 0
    np.testing.assert_array_equal(f.forces(), np.zeros((3, 0)))
    pos, mass = W.uniform(10, 94)
    f.build_tree(pos, mass)
    nodes, _, _ = f.tree()
    assert len(nodes) == 1 and nodes[0, 3] == -1
    np.testing.assert_allclose(f.forces(), oracle.direct_sr(pos, mass, 1.0, RS, RC), rtol=1e-12, atol=1e-14)


def _coverage(f, pos):
    """Times each ordered (sink, source, shift) particle triple is covered by a list entry."""
    nodes, _, perm = f.tree()
    p2p, m2l = f.lists()
    n = pos.shape[1]
    cov = np.zeros((27, n, n), dtype=np.int64)
    for lst in (p2p, m2l):
        for a, b, s in lst:
            ia = perm[nodes[a, 1]:nodes[a, 1] + nodes[a, 2]]
            ib = perm[nodes[b, 1]:nodes[b, 1] + nodes[b, 2]]
            cov[s][np.ix_(ia, ib)] += 1
    return cov, p2p, m2l


def _close(pos):
    """[27][n][n] True where 0 < |x_j + sL - x_i| < R_c."""
    x = _wrap(pos).T
    out = np.zeros((27, len(x), len(x)), dtype=bool)
    for s in range(27):
        sh = np.array([s // 9 - 1, (s // 3) % 3 - 1, s % 3 - 1], dtype=np.float64)
        d = x[None, :, :] + sh - x[:, None, :]
        r2 = (d * d).sum(axis=2)
        out[s] = (r2 > 0) & (r2 < RC * RC)
    return out


@pytest.mark.parametrize("theta,leaf,rule,size_rule", [(0.5, 4, 1, 1), (0.7, 2, 0, 0), (0.3, 8, 1, 0),
                                                        (0.6, 6, 0, 1)])
def test_lists_cover_every_close_pair_exactly_once(theta, leaf, rule, size_rule):
    n = 400
    pos, mass = W.nfw_clustered(n, 5, 0.6, 95 + leaf)
    f = _kd(leaf, theta=theta, rule=rule, size_rule=size_rule)
    f.build_tree(pos, mass)
    f.traverse()
    cov, p2p, m2l = _coverage(f, pos)
    assert len(p2p) > 0 and len(m2l) > 0
    assert cov.max() == 1
    assert (cov[_close(pos)] == 1).all()
    nodes, _, _ = f.tree()
    assert (nodes[p2p[:, 0], 3] < 0).all() and (nodes[p2p[:, 1], 3] < 0).all()


@pytest.mark.parametrize("leaf", [1, 4])
def test_theta_zero_leaves_only_leaf_pairs(leaf):
    pos, mass = W.nfw_clustered(400, 5, 0.6, 99)
    f = _kd(leaf, theta=0.0)
    f.build_tree(pos, mass)
    f.traverse()
    p2p, m2l = f.lists()
    assert len(m2l) == 0 and len(p2p) > 0


def test_single_particle_leaves_and_coincident_particles():
    """Leaves of one particle have boxes of side 0: every close pair of distinct
    points may go to M2L (exact for a point mass), but a leaf never against
    itself and never two leaves at one point (S_c = 0); coincident particles
    exert no force on each other, as in the direct sum."""
    pos, mass = W.nfw_clustered(300, 4, 0.6, 101)
    pos = np.concatenate([pos, pos[:, :40]], axis=1)  # 40 particles doubled
    mass = np.concatenate([mass, mass[:40]])
    f = _kd(1, theta=0.3, order=8)
    f.build_tree(pos, mass)
    a = f.forces()
    p2p, m2l = f.lists()
    nodes, boxes, _ = f.tree()
    c = 0.5 * (boxes[:, :3] + boxes[:, 3:])
    sh = np.stack([m2l[:, 2] // 9 - 1, (m2l[:, 2] // 3) % 3 - 1, m2l[:, 2] % 3 - 1], axis=1)
    assert (np.abs(c[m2l[:, 1]] + sh - c[m2l[:, 0]]).sum(axis=1) > 0).all()
    ref = oracle.direct_sr(pos, mass, 1.0, RS, RC)
    assert _err(a, ref) < 1e-5


@pytest.fixture(scope="module")
def clustered():
    pos, mass = W.nfw_clustered(6000, 12, 0.7, 100)
    return pos, mass, oracle.direct_sr(pos, mass, 1.0, RS, RC)


def _err(a, ref):
    return float(np.sqrt(((a - ref) ** 2).sum() / (ref ** 2).sum()))


def test_theta_zero_forces_are_the_direct_sum(clustered):
    pos, mass, ref = clustered
    f = _kd(16, theta=0.0)
    f.build_tree(pos, mass)
    assert _err(f.forces(), ref) < 1e-13


def test_forces_converge_with_order(clustered):
    pos, mass, ref = clustered
    errs = []
    for p in (2, 4, 6, 8):
        f = _kd(16, theta=0.35, order=p)
        f.build_tree(pos, mass)
        errs.append(_err(f.forces(), ref))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 2e-6 and errs[1] < 1e-3


def test_forces_on_given_lists_equal_the_walk(clustered):
    pos, mass, _ = clustered
    f = _kd(16, theta=0.5, order=4)
    f.build_tree(pos, mass)
    a = f.forces()
    p2p, m2l = f.lists()
    rng = np.random.default_rng(0)
    np.testing.assert_allclose(f.forces_given_lists(p2p[rng.permutation(len(p2p))], m2l[rng.permutation(len(m2l))]),
                               a, rtol=0, atol=0)
    with pytest.raises(RuntimeError):
        f.forces_given_lists(np.array([[0, 10 ** 9, 13]]), m2l)


@pytest.mark.parametrize("theta,leaf", [(0.5, 4), (0.7, 1), (0.3, 8)])
def test_conventional_lists_cover_every_particle_pair_exactly_once(theta, leaf):
    """The conventional FMM's walk on the k-d tree (Sec. 3): the opening-angle test
    alone from (root, root) of the primary box covers every ordered particle pair,
    a particle with itself included, exactly once, and every accepted pair passes
    the test."""
    n = 300
    pos, mass = W.nfw_clustered(n, 4, 0.6, 70 + leaf)
    f = _kd(leaf, theta=theta)
    f.build_tree(pos, mass)
    f.traverse(conventional=True)
    nodes, boxes, perm = f.tree()
    p2p, m2l = f.lists()
    assert len(m2l) > 0 and len(p2p) > 0
    assert (p2p[:, 2] == 13).all() and (m2l[:, 2] == 13).all()
    cov = np.zeros((n, n), dtype=np.int64)
    for lst in (p2p, m2l):
        for a, b, _ in lst:
            cov[np.ix_(perm[nodes[a, 1]:nodes[a, 1] + nodes[a, 2]], perm[nodes[b, 1]:nodes[b, 1] + nodes[b, 2]])] += 1
    assert (cov == 1).all()
    side = (boxes[:, 3:] - boxes[:, :3]).max(axis=1)
    c = 0.5 * (boxes[:, :3] + boxes[:, 3:])
    sc2 = ((c[m2l[:, 1]] - c[m2l[:, 0]]) ** 2).sum(axis=1)
    wl = np.maximum(side[m2l[:, 0]], side[m2l[:, 1]])
    assert (wl * wl <= theta * theta * sc2 * (1 + 1e-12)).all() and (sc2 > 0).all()
    cnt = f.counts()
    assert cnt["p2p_particle_pairs"] + int((nodes[m2l[:, 0], 2] * nodes[m2l[:, 1], 2]).sum()) == n * n


def test_conventional_theta_zero_leaves_only_leaf_pairs_and_hybrid_is_unchanged():
    pos, mass = W.nfw_clustered(400, 5, 0.6, 99)
    f = _kd(4, theta=0.0)
    f.build_tree(pos, mass)
    f.traverse(conventional=True)
    p2p, m2l = f.lists()
    nleaves = int((f.tree()[0][:, 3] < 0).sum())
    assert len(m2l) == 0 and len(p2p) == nleaves * nleaves
    g = _kd(4, theta=0.5)
    g.build_tree(pos, mass)
    g.traverse()
    before = [x.copy() for x in g.lists()]
    g.traverse(conventional=True)
    g.traverse()
    for x, y in zip(g.lists(), before):
        np.testing.assert_array_equal(x, y)


def test_polynomial_split_theta_zero_is_its_direct_sum_and_converges():
    """The k-d FMM with the polynomial truncation of Sec. 5: theta = 0 gives that
    split's direct truncated sum, and its error falls with the order."""
    pos, mass = W.nfw_clustered(6000, 12, 0.7, 100)
    ref = oracle.direct_sr(pos, mass, 1.0, RS, RC, split="poly")
    f = oracle.KdFMM(box=1.0, rs=RS, rc=RC, theta=0.0, order=4, leaf_max=16, split="poly")
    f.build_tree(pos, mass)
    assert _err(f.forces(), ref) < 1e-13
    errs = []
    for p in (2, 4, 6):
        g = oracle.KdFMM(box=1.0, rs=RS, rc=RC, theta=0.35, order=p, leaf_max=16, split="poly")
        g.build_tree(pos, mass)
        errs.append(_err(g.forces(), ref))
    assert errs[2] < errs[1] < errs[0] and errs[2] < 1e-5 and errs[0] > 1e-8, errs


@pytest.mark.parametrize("box", [0.5, 3.0])
def test_tree_equals_the_definition_for_other_box_sides(box):
    """A power-of-two box side and one that is not, with positions outside the
    box on both sides (the wrap x - L floor(x / L) brings them in)."""
    pos, mass = W.nfw_clustered(900, 6, 0.7, 104)
    pos = pos * box
    pos[:, :50] -= 1.37 * box
    pos[:, 50:100] += 2.11 * box
    f = oracle.KdFMM(box=box, rs=RS * box, rc=RC * box, theta=0.5, order=4, leaf_max=8)
    f.build_tree(pos, mass)
    nodes, boxes, perm = f.tree()
    rn, rb, rp = kd_reference(pos, 8, box=box)
    np.testing.assert_array_equal(nodes, rn)
    np.testing.assert_array_equal(boxes, rb)
    np.testing.assert_array_equal(perm, rp)
    assert (boxes[:, :3] >= 0).all() and (boxes[:, 3:] <= box).all()
