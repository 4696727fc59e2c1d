"""GPU parity of the ORB / k-d tree variant (tree = 1; the ORB tree with a leaf
limiter of Sec. 2.1, Fig. 1, and the k-d tree of Sec. 4) against the FP64
oracle (oracle/orc_kd.c), through the C ABI.

Bit-exact: tree nodes (level, particle range, children, split axis), bounding
boxes, particle order, and the P2P / M2L lists as sorted sets (the walk's rules
are FP64 with every operation rounded on its own on both sides).  Forces: FP32
GPU against the FP64 oracle FMM on identical lists, within 1e-5 relative RMS
and the per-particle bound of force_check; theta = 0 against the direct sum;
the 2M clustered set of the benchmark against the direct sum on sampled sinks.
The PM long range does not depend on the tree (deterministic fixed-point
deposit), so it equals the octree context's bit for bit, and a step equals a
fresh build at the drifted positions.  Edge cases: N = 0, 1, one-particle
leaves, coincident particles, positions outside the box, a box side that is
not a power of two, walk buffers grown from tiny capacities, unsupported
combinations refused.
"""
import math

import numpy as np
import pytest

import oracle
from force_check import assert_forces_close
from paper_2006_14952_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def solver(**kw):
    from paper_2006_14952_gb300 import hfmm

    return hfmm.Solver(tree=1, **kw)


def dev(a, dt):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).cuda()


def run_gpu(pos, mass, **kw):
    import torch

    s = solver(**kw)
    s.build_tree(dev(pos, np.float64), dev(mass, np.float32))
    acc = s.short_range_forces()
    torch.cuda.synchronize()
    return s, acc.cpu().numpy().astype(np.float64)


def run_oracle(pos, mass, s):
    p = s.params
    f = oracle.KdFMM(box=p.box, rs=s.rs, rc=s.rc, G=p.G, theta=p.theta, order=p.order, leaf_max=p.leaf_max,
                     transition_rule=p.transition_rule, size_rule=p.size_rule,
                     split="poly" if p.split == 1 else "gauss")
    f.build_tree(pos, np.asarray(mass, dtype=np.float32).astype(np.float64))
    return f


def sorted_rows(a):
    a = np.asarray(a, dtype=np.int64).reshape(-1, 3)
    return a[np.lexsort((a[:, 2], a[:, 1], a[:, 0]))]


def assert_tree_equal(s, f):
    nodes, boxes, perm = f.tree()
    np.testing.assert_array_equal(s.export("kd_nodes"), nodes)
    np.testing.assert_array_equal(s.export("kd_boxes"), boxes)
    np.testing.assert_array_equal(s.export("perm").astype(np.int64), perm)
    st = s.get_stats()
    assert st["nnodes"] == len(nodes) and st["nlevels"] == f.size("levels")
    assert st["nleaves"] == int((nodes[:, 3] < 0).sum())


CASES = {
    "uniform-50000": lambda: W.uniform(50000, 11),
    "nfw-50000": lambda: W.nfw_clustered(50000, 60, 0.7, 12),
    "zeldovich-32768": lambda: W.zeldovich(32, 13, halo_count=20, halo_frac=0.4),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("leaf", [16, 48])
def test_tree_bit_exact(case, leaf):
    pos, mass = CASES[case]()
    pos = pos.copy()
    pos[:, :4] = [[-0.3, 1.0, 1.7, 0.5], [2.2, -1e-17, 0.25, 0.5], [0.999999999999, 0.5, -2.0, 0.5]]
    top = 1.0 - 2.0 ** -53
    pos[:, 4:8] = [[0.0, 5e-324, 1e-300, top], [1e-300, 0.0, 5e-324, 0.25], [top, 1e-300, 0.0, 5e-324]]
    s, _ = run_gpu(pos, mass, pm_grid=32, leaf_max=leaf)
    assert_tree_equal(s, run_oracle(pos, mass, s))


@pytest.mark.parametrize("box", [0.5, 3.0])
def test_tree_bit_exact_for_other_box_sides(box):
    pos, mass = W.nfw_clustered(20000, 30, 0.7, 61)
    pos = pos * box
    pos[:, :500] -= 1.37 * box
    pos[:, 500:1000] += 2.11 * box
    s, _ = run_gpu(pos, mass, pm_grid=32, box=box)
    f = run_oracle(pos, mass, s)
    assert_tree_equal(s, f)
    f.traverse()
    p2p, m2l = f.lists()
    np.testing.assert_array_equal(sorted_rows(s.export("p2p")), sorted_rows(p2p))
    np.testing.assert_array_equal(sorted_rows(s.export("m2l")), sorted_rows(m2l))


@pytest.mark.parametrize("rule,size_rule,theta,leaf", [(1, 1, 0.5, 16), (0, 1, 0.5, 16), (1, 0, 0.5, 16),
                                                        (0, 0, 0.7, 8), (1, 1, 0.3, 4), (1, 1, 0.7, 1),
                                                        (1, 1, 0.0, 16), (1, 1, 0.35, 48), (1, 1, 0.35, 64)])
def test_interaction_lists_bit_exact(rule, size_rule, theta, leaf):
    pos, mass = W.nfw_clustered(20000 if leaf > 1 else 4000, 30, 0.7, 21)
    s, _ = run_gpu(pos, mass, pm_grid=32, theta=theta, leaf_max=leaf, transition_rule=rule, size_rule=size_rule,
                   order=2)
    f = run_oracle(pos, mass, s)
    f.traverse()
    p2p, m2l = f.lists()
    np.testing.assert_array_equal(sorted_rows(s.export("p2p")), sorted_rows(p2p))
    np.testing.assert_array_equal(sorted_rows(s.export("m2l")), sorted_rows(m2l))
    st = s.get_stats()
    assert st["np2p"] == len(p2p) and st["nm2l"] == len(m2l)
    if theta == 0.0:
        assert len(m2l) == 0


def test_walk_grows_its_buffers_from_tiny_capacities():
    """Frontier and lists start at 64 entries (list_init): levels of the walk
    overflow, their buffers grow and the level is walked again.  The lists equal
    the oracle's and the forces are bit-identical to a run that never overflowed."""
    import torch

    pos, mass = W.nfw_clustered(20000, 30, 0.7, 21)
    kw = dict(pm_grid=32, theta=0.5, leaf_max=16, order=4)
    s0, _ = run_gpu(pos, mass, **kw)
    acc0 = s0.short_range_forces().cpu().numpy().astype(np.float64)  # the capacities the first call grew
    torch.cuda.synchronize()
    s, acc = run_gpu(pos, mass, list_init=64, **kw)
    assert s0.get_stats()["traverse_walks"] == 1 and s.get_stats()["traverse_walks"] > 1
    f = run_oracle(pos, mass, s)
    f.traverse()
    p2p, m2l = f.lists()
    np.testing.assert_array_equal(sorted_rows(s.export("p2p")), sorted_rows(p2p))
    np.testing.assert_array_equal(sorted_rows(s.export("m2l")), sorted_rows(m2l))
    np.testing.assert_array_equal(acc, acc0)


@pytest.mark.parametrize("case,order,leaf,theta", [("uniform-50000", 4, 16, 0.5), ("nfw-50000", 2, 16, 0.5),
                                                   ("nfw-50000", 4, 16, 0.5), ("nfw-50000", 6, 48, 0.35),
                                                   ("nfw-50000", 5, 64, 0.3), ("zeldovich-32768", 3, 32, 0.4)])
def test_forces_match_fp64_fmm_on_identical_lists(case, order, leaf, theta):
    pos, mass = CASES[case]()
    s, acc = run_gpu(pos, mass, pm_grid=32, order=order, leaf_max=leaf, theta=theta)
    f = run_oracle(pos, mass, s)
    ref = f.forces()  # the oracle's own walk: its lists equal the GPU's (test above)
    assert f.size("m2l") > 0 and f.size("p2p") > 0
    assert s.get_stats()["nm2l"] == f.size("m2l")
    print("relative RMS %.3e, per particle %.3e" % assert_forces_close(acc, ref))


def test_forces_are_reproducible():
    pos, mass = CASES["nfw-50000"]()
    _, a = run_gpu(pos, mass, pm_grid=32, order=4)
    _, b = run_gpu(pos, mass, pm_grid=32, order=4)
    np.testing.assert_array_equal(a, b)


def test_theta_zero_equals_direct_sum():
    pos, mass = W.make(W.CONFIGS["uniform-32k"])
    s, acc = run_gpu(pos, mass, pm_grid=32, theta=0.0)
    assert s.get_stats()["nm2l"] == 0
    assert_forces_close(acc, oracle.direct_sr(pos, mass, 1.0, s.rs, s.rc))


def test_edge_cases_empty_single_coincident():
    import torch

    s = solver()
    s.build_tree(torch.zeros((3, 0), dtype=torch.float64, device="cuda"), torch.zeros(0, device="cuda"))
    assert s.short_range_forces().shape == (3, 0)
    assert s.get_stats()["nnodes"] == 0
    s.build_tree(torch.tensor([[0.3], [0.4], [0.5]], dtype=torch.float64, device="cuda"), torch.ones(1, device="cuda"))
    assert torch.all(s.short_range_forces() == 0)
    # 40 coincident particles plus two neighbours, in leaves of 16 and of 1
    pos = np.full((3, 42), 0.3)
    pos[0, 40] = 0.31
    pos[0, 41] = 0.29
    mass = np.full(42, 1 / 42, dtype=np.float32)
    ref = oracle.direct_sr(pos, mass, 1.0, 1.25 / 32, 4.5 * 1.25 / 32)
    one = oracle.direct_sr(pos[:, [0, 40]], mass[[0, 40]], 1.0, 1.25 / 32, 4.5 * 1.25 / 32)
    for leaf in (16, 1):
        s2, acc = run_gpu(pos, mass, pm_grid=32, leaf_max=leaf, order=6, theta=0.3)
        assert_tree_equal(s2, run_oracle(pos, mass, s2))
        assert_forces_close(acc, ref, scale=float(np.linalg.norm(one[:, 0])))


def test_full_size_clustered_set_in_the_bench_configuration():
    """The 2M clustered set with the benchmark's parameters (leaf 48, theta 0.35,
    p 6) on the k-d tree: nodes, boxes and particle order bit-exact against the
    oracle; forces on 4000 sampled sinks against the FP64 direct truncated sum
    within the accuracy bar (RMS 1e-4, 99th percentile 1e-3)."""
    cfg = W.CONFIGS["nfw-2m"]
    pos, mass = W.make(cfg)
    s, acc = run_gpu(pos, mass, pm_grid=cfg.pm_grid, rs_cells=cfg.rs_cells, rcut_rs=cfg.rcut_rs, theta=cfg.theta,
                     order=cfg.order, leaf_max=cfg.leaf_max)
    assert_tree_equal(s, run_oracle(pos, mass, s))
    sinks = W.subsample(cfg.n, 4000, 31)
    ref = oracle.direct_sr(pos, mass, cfg.box, cfg.rs, cfg.rc, sinks=sinks)
    e = np.linalg.norm(acc[:, sinks] - ref, axis=0) / np.linalg.norm(ref, axis=0)
    print("RMS %.3e p99 %.3e" % (math.sqrt((e ** 2).mean()), np.percentile(e, 99)), s.get_stats())
    assert math.sqrt((e ** 2).mean()) < 1e-4
    assert np.percentile(e, 99) < 1e-3


def test_host_entry_point_pm_and_step():
    import torch

    pos, mass = CASES["nfw-50000"]()
    kw = dict(pm_grid=32, order=4)
    s, acc = run_gpu(pos, mass, **kw)
    np.testing.assert_array_equal(solver(**kw).short_range_forces_host(np.ascontiguousarray(pos), mass),
                                  acc.astype(np.float32))
    # PM: the same long range as the octree context, bit for bit
    from paper_2006_14952_gb300 import hfmm

    o = hfmm.Solver(**kw)
    o.build_tree(dev(pos, np.float64), dev(mass, np.float32))
    a_kd = torch.zeros((3, pos.shape[1]), device="cuda")
    a_oc = torch.zeros_like(a_kd)
    s.pm_long_range(a_kd)
    o.pm_long_range(a_oc)
    assert torch.equal(a_kd, a_oc) and float(a_kd.abs().max()) > 0
    # a step: the accelerations it leaves are those of a fresh build at the drifted positions
    rng = np.random.default_rng(5)
    p, m = dev(pos, np.float64), dev(mass, np.float32)
    v = dev(0.05 * rng.normal(size=pos.shape), np.float32)
    s.build_tree(p, m)
    a = s.short_range_forces()
    s.pm_long_range(a)
    s.step(p, v, a, 2e-3)
    torch.cuda.synchronize()
    f = solver(**kw)
    f.build_tree(p.clone(), m)
    a2 = f.short_range_forces()
    f.pm_long_range(a2)
    assert torch.equal(a, a2)


def test_unsupported_combinations_are_refused():
    import torch

    from paper_2006_14952_gb300 import hfmm

    for kw in (dict(mac_mode=1), dict(m2l_precision=1), dict(m2l_tables=1), dict(p2p_mutual=1, size_rule=1),
               dict(order=7)):
        with pytest.raises(hfmm.HfmmError, match="ARG"):
            solver(**kw)
    with pytest.raises(hfmm.HfmmError, match="ARG"):
        hfmm.Solver(tree=2)
    s, _ = run_gpu(*W.uniform(5000, 3), pm_grid=32)
    for what in ("keys", "nodes"):
        with pytest.raises(hfmm.HfmmError, match="ARG"):
            s.export(what)
    o = hfmm.Solver(pm_grid=32)
    o.build_tree(torch.zeros((3, 4), dtype=torch.float64, device="cuda") + 0.5, torch.ones(4, device="cuda"))
    with pytest.raises(hfmm.HfmmError, match="ARG"):
        o.export("kd_nodes")


def test_statistics_counts_of_the_p2p_pairs():
    """profile bit 1: the particle pairs on the P2P list (sum of n_sink n_source,
    exact) and the pairs inside (0, R_c) the kernel evaluated, against an FP64
    count over the oracle's list (equal up to pairs within FP32 rounding of R_c)."""
    pos, mass = W.nfw_clustered(20000, 30, 0.7, 23)
    s, _ = run_gpu(pos, mass, pm_grid=32, theta=0.4, leaf_max=32, order=4, profile=3)
    st = s.get_stats()
    f = run_oracle(pos, mass, s)
    f.traverse()
    nodes, _, perm = f.tree()
    p2p, _ = f.lists()
    cnt = nodes[:, 2]
    assert st["p2p_particle_pairs"] == int((cnt[p2p[:, 0]] * cnt[p2p[:, 1]]).sum())
    x = (pos - np.floor(pos)).T
    useful = 0
    for a, b, sh in p2p:
        ia = perm[nodes[a, 1]:nodes[a, 1] + nodes[a, 2]]
        ib = perm[nodes[b, 1]:nodes[b, 1] + nodes[b, 2]]
        shv = np.array([sh // 9 - 1, (sh // 3) % 3 - 1, sh % 3 - 1], dtype=np.float64)
        d = x[ib][None, :, :] + shv - x[ia][:, None, :]
        r2 = (d * d).sum(axis=2)
        useful += int(((r2 > 0) & (r2 < s.rc * s.rc)).sum())
    assert abs(st["p2p_useful_pairs"] - useful) <= max(2, useful // 100000), (st["p2p_useful_pairs"], useful)


@pytest.mark.parametrize("theta,leaf", [(0.3, 1), (0.5, 8), (0.7, 32)])
def test_interaction_counts_bit_exact(theta, leaf):
    """hfmm_interaction_counts on the k-d tree (Sec. 3): the hybrid and the
    conventional walk give the oracle's lists (as sorted sets) and counts."""
    pos, mass = W.nfw_clustered(20000 if leaf > 1 else 5000, 30, 0.7, 29)
    s, _ = run_gpu(pos, mass, pm_grid=32, theta=theta, leaf_max=leaf, order=2)
    f = run_oracle(pos, mass, s)
    for conv in (False, True):
        c = s.interaction_counts(conventional=conv)
        f.traverse(conventional=conv)
        p2p, m2l = f.lists()
        np.testing.assert_array_equal(sorted_rows(s.export("p2p")), sorted_rows(p2p))
        np.testing.assert_array_equal(sorted_rows(s.export("m2l")), sorted_rows(m2l))
        ref = f.counts()
        assert (c["m2l"], c["p2p"], c["p2p_particle_pairs"]) == (ref["m2l"], ref["p2p"], ref["p2p_particle_pairs"])
        if conv:
            nodes = f.tree()[0]
            assert c["p2p_particle_pairs"] + int((nodes[m2l[:, 0], 2] * nodes[m2l[:, 1], 2]).sum()) == len(mass) ** 2
    # the forces afterwards walk again with the hybrid rules
    acc = s.short_range_forces().cpu().numpy().astype(np.float64)
    f2 = run_oracle(pos, mass, s)
    assert_forces_close(acc, f2.forces())
    assert s.get_stats()["nm2l"] == f2.size("m2l")


@pytest.mark.parametrize("order,leaf,theta", [(4, 16, 0.5), (6, 48, 0.35)])
def test_polynomial_split_forces_on_identical_lists(order, leaf, theta):
    """The polynomial truncation of Sec. 5 (split 1) on the k-d tree: forces
    against the oracle's k-d FMM in that split (its lists equal the GPU's: the
    walk does not depend on the split), and theta = 0 against its direct sum."""
    pos, mass = CASES["nfw-50000"]()
    s, acc = run_gpu(pos, mass, pm_grid=32, order=order, leaf_max=leaf, theta=theta, split=1)
    f = run_oracle(pos, mass, s)
    assert f.split == "poly" and f.size("nodes") == s.get_stats()["nnodes"]
    print("relative RMS %.3e, per particle %.3e" % assert_forces_close(acc, f.forces()))
    assert s.get_stats()["nm2l"] == f.size("m2l") > 0
    s0, acc0 = run_gpu(pos, mass, pm_grid=32, theta=0.0, split=1)
    assert_forces_close(acc0, oracle.direct_sr(pos, mass, 1.0, s0.rs, s0.rc, split="poly"))
