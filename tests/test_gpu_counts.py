"""Interaction counts of Sec. 3 (Figs. 5-6) through the C ABI: the GPU walk with
the hybrid acceptance and with the conventional FMM's, against the FP64 oracle.

Bit-exact: the lists of both walks (sorted sets) and the three counts (M2L cell
pairs, P2P leaf pairs, particle pairs on the P2P lists); on a complete lattice
octree at theta = 1/2 the conventional counts equal the textbook interaction
lists.  A count walk replaces the lists but leaves the forces of the next
short_range_forces call unchanged, bit for bit.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2006_14952_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _solver_on(pos, mass, **kw):
    import torch

    from paper_2006_14952_gb300 import hfmm

    s = hfmm.Solver(**kw)
    s.build_tree(torch.from_numpy(np.ascontiguousarray(pos)).cuda(),
                 torch.from_numpy(np.ascontiguousarray(mass, dtype=np.float32)).cuda())
    return s


def _oracle_on(pos, mass, s):
    p = s.params
    f = oracle.FMM(box=p.box, rs=s.rs, rc=s.rc, G=p.G, theta=p.theta, order=2, leaf_max=p.leaf_max,
                   transition_rule=p.transition_rule, size_rule=p.size_rule)
    f.build_tree(pos, mass)
    return f


def _rows(a):
    a = np.asarray(a, dtype=np.int64).reshape(-1, 3)
    return a[np.lexsort((a[:, 2], a[:, 1], a[:, 0]))]


CASES = {
    "nfw-20000-leaf1": (lambda: W.nfw_clustered(20000, 30, 0.7, 81), 1, 0.5),
    "nfw-40000-leaf32": (lambda: W.nfw_clustered(40000, 40, 0.7, 82), 32, 0.35),
    "uniform-32768-leaf1": (lambda: W.uniform(32768, 83), 1, 0.6),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("conventional", [False, True])
def test_walk_lists_and_counts_bit_exact(case, conventional):
    make, leaf, theta = CASES[case]
    pos, mass = make()
    s = _solver_on(pos, mass, pm_grid=64, order=2, leaf_max=leaf, theta=theta)
    c = s.interaction_counts(conventional=conventional)
    f = _oracle_on(pos, mass, s)
    f.traverse(conventional=conventional)
    p2p, m2l = f.lists()
    assert np.array_equal(_rows(s.export("p2p")), _rows(p2p))
    assert np.array_equal(_rows(s.export("m2l")), _rows(m2l))
    ref = f.counts()
    assert (c["m2l"], c["p2p"], c["p2p_particle_pairs"]) == (ref["m2l"], ref["p2p"], ref["p2p_particle_pairs"])
    assert c["frontier_pairs"] >= c["m2l"] + c["p2p"]
    if conventional:
        cnt = f.nodes()[:, 5]
        assert c["p2p_particle_pairs"] + int((cnt[m2l[:, 0]] * cnt[m2l[:, 1]]).sum()) == len(mass) ** 2


def test_conventional_counts_on_a_lattice_equal_the_textbook_interaction_lists():
    k = 4
    n = 2 ** k
    pos = (np.array(list(itertools.product(range(n), repeat=3))).T + 0.5) / n
    mass = np.full(n ** 3, 1.0 / n ** 3)
    s = _solver_on(pos, mass, pm_grid=32, order=2, leaf_max=1, theta=0.5)
    c = s.interaction_counts(conventional=True)
    m2l = 0
    for lev in range(1, k + 1):
        g = np.array(list(itertools.product(range(2 ** lev), repeat=3)))
        d = np.abs(g[:, None, :] - g[None, :, :]).max(axis=2)
        dp = np.abs(g[:, None, :] // 2 - g[None, :, :] // 2).max(axis=2)
        m2l += int(((dp <= 1) & (d >= 2)).sum())
    g = np.array(list(itertools.product(range(n), repeat=3)))
    p2p = int((np.abs(g[:, None, :] - g[None, :, :]).max(axis=2) <= 1).sum())
    assert (c["m2l"], c["p2p"], c["p2p_particle_pairs"]) == (m2l, p2p, p2p)


def test_a_count_walk_leaves_the_next_forces_unchanged():
    import torch

    pos, mass = W.nfw_clustered(30000, 40, 0.7, 84)
    s = _solver_on(pos, mass, pm_grid=32, order=4, leaf_max=16, theta=0.5)
    a0 = s.short_range_forces().cpu().numpy()
    st0 = s.get_stats()
    h = s.interaction_counts()
    assert (h["m2l"], h["p2p"]) == (st0["nm2l"], st0["np2p"])  # the hybrid count walk is the force walk
    c = s.interaction_counts(conventional=True)
    assert s.get_stats()["nm2l"] == c["m2l"]
    a1 = s.short_range_forces().cpu().numpy()
    torch.cuda.synchronize()
    assert np.array_equal(a0, a1)


def test_count_call_edge_cases():
    import ctypes

    import torch

    from paper_2006_14952_gb300 import hfmm

    s = hfmm.Solver(pm_grid=32)
    with pytest.raises(hfmm.HfmmError, match="before build_tree"):
        s.interaction_counts()
    s.build_tree(torch.zeros((3, 0), dtype=torch.float64, device="cuda"),
                 torch.zeros(0, dtype=torch.float32, device="cuda"))
    assert s.interaction_counts(conventional=True) == {"m2l": 0, "p2p": 0, "p2p_particle_pairs": 0,
                                                       "frontier_pairs": 0}
    out = (ctypes.c_int64 * 4)()
    assert s._lib.hfmm_interaction_counts(s._h, 2, out, None) == -1  # HFMM_ERR_ARG
    assert s._lib.hfmm_interaction_counts(s._h, 0, None, None) == -1  # HFMM_ERR_ARG
    one = _solver_on(np.full((3, 1), 0.25), np.ones(1), pm_grid=32, leaf_max=1)
    for conv in (False, True):
        c = one.interaction_counts(conventional=conv)
        assert (c["m2l"], c["p2p_particle_pairs"]) == (0, 1 if conv else 27)
