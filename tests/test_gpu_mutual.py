"""Mutual P2P (p2p_mutual = 1, Newton's third law) against the FP64 oracle.

- The walk keeps exactly one ordered pair of each mirror couple: the GPU's P2P
  list equals the oracle's list restricted to the owned pairs (the deeper sink
  leaf; at equal depth A < B for odd A + B and A > B for even; A = B with
  s <= 13), bit-exact as sorted sets; the M2L list is unchanged.
- Forces on identical interaction pairs: the mutual evaluation against the
  oracle's one-sided FMM (the same particle pairs), within the FP32 tolerances
  of the one-sided path, for both splits, several leaf sizes and orders.
- The reaction partials are summed in a fixed order: two runs give the same
  bits; and the result equals the one-sided GPU kernel's to FP32 rounding.
- theta = 0 at the full uniform size against the direct sum.
"""
import numpy as np
import pytest

import oracle
from force_check import assert_forces_close, rel_rms
from paper_2006_14952_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def run_gpu(pos, mass, **kw):
    import torch

    from paper_2006_14952_gb300 import hfmm

    s = hfmm.Solver(**kw)
    s.build_tree(torch.from_numpy(np.ascontiguousarray(pos)).cuda(), torch.from_numpy(mass).cuda())
    acc = s.short_range_forces()
    torch.cuda.synchronize()
    return s, acc.cpu().numpy().astype(np.float64)


def oracle_fmm(pos, mass, s, split="gauss"):
    p = s.params
    f = oracle.FMM(box=p.box, rs=s.rs, rc=s.rc, G=p.G, theta=p.theta, order=p.order, leaf_max=p.leaf_max,
                   transition_rule=p.transition_rule, size_rule=p.size_rule, split=split)
    f.build_tree(pos, mass)
    return f


def sorted_rows(a):
    a = np.asarray(a, dtype=np.int64).reshape(-1, 3)
    return a[np.lexsort((a[:, 2], a[:, 1], a[:, 0]))]


@pytest.mark.parametrize("leaf,theta", [(16, 0.5), (48, 0.35), (1, 0.7)])
def test_mutual_walk_keeps_one_of_each_mirror_pair(leaf, theta):
    pos, mass = W.nfw_clustered(20000 if leaf > 1 else 4000, 30, 0.7, 21)
    s, _ = run_gpu(pos, mass, pm_grid=32, theta=theta, leaf_max=leaf, order=2, p2p_mutual=1)
    f = oracle_fmm(pos, mass, s)
    f.traverse()
    p2p, m2l = f.lists()
    lev = f.nodes()[:, 0]
    a, b, sh = p2p[:, 0], p2p[:, 1], p2p[:, 2]
    same = lev[a] == lev[b]
    odd = ((a ^ b) & 1) == 1
    owned = np.where(a == b, sh <= 13,
                     np.where(same, np.where(odd, a < b, a > b), lev[a] > lev[b]))
    assert 0.45 * len(p2p) < owned.sum() < 0.6 * len(p2p)
    np.testing.assert_array_equal(sorted_rows(s.export("p2p")), sorted_rows(p2p[owned]))
    np.testing.assert_array_equal(sorted_rows(s.export("m2l")), sorted_rows(m2l))


@pytest.mark.parametrize("case,order,leaf,theta,split", [
    ("nfw", 4, 16, 0.5, "gauss"), ("nfw", 6, 48, 0.35, "gauss"), ("uniform", 4, 16, 0.5, "gauss"),
    ("nfw", 6, 64, 0.35, "gauss"), ("nfw", 4, 8, 0.4, "gauss"), ("nfw", 6, 48, 0.35, "poly")])
def test_mutual_forces_match_fp64_fmm_on_the_same_pairs(case, order, leaf, theta, split):
    pos, mass = W.nfw_clustered(50000, 60, 0.7, 12) if case == "nfw" else W.uniform(50000, 11)
    s, acc = run_gpu(pos, mass, pm_grid=32, order=order, leaf_max=leaf, theta=theta, p2p_mutual=1,
                     split=1 if split == "poly" else 0)
    f = oracle_fmm(pos, mass, s, split)
    ref = f.forces()
    assert f.size("p2p") > 0 and f.size("m2l") > 0
    print("relative RMS %.3e, per particle %.3e" % assert_forces_close(acc, ref))


def test_mutual_forces_are_reproducible_and_equal_the_one_sided_kernel():
    pos, mass = W.nfw_clustered(200000, 120, 0.7, 77)
    kw = dict(pm_grid=64, order=6, leaf_max=48, theta=0.35)
    _, a1 = run_gpu(pos, mass, p2p_mutual=1, **kw)
    _, a2 = run_gpu(pos, mass, p2p_mutual=1, **kw)
    np.testing.assert_array_equal(a1, a2)
    _, a0 = run_gpu(pos, mass, **kw)
    e = rel_rms(a1, a0)
    print("mutual vs one-sided relative RMS %.3e" % e)
    assert e < 2e-6


def test_mutual_theta_zero_equals_direct_sum_at_full_uniform_size():
    pos, mass = W.make(W.CONFIGS["uniform-32k"])
    s, acc = run_gpu(pos, mass, pm_grid=32, theta=0.0, p2p_mutual=1)
    assert s.get_stats()["nm2l"] == 0
    ref = oracle.direct_sr(pos, mass, 1.0, s.rs, s.rc)
    assert_forces_close(acc, ref)


def test_mutual_edge_cases_and_rejections():
    import torch

    from paper_2006_14952_gb300 import hfmm

    s = hfmm.Solver(p2p_mutual=1)
    s.build_tree(torch.zeros((3, 0), dtype=torch.float64, device="cuda"), torch.zeros(0, device="cuda"))
    assert s.short_range_forces().shape == (3, 0)
    one = torch.tensor([[0.3], [0.4], [0.5]], dtype=torch.float64, device="cuda")
    s.build_tree(one, torch.ones(1, device="cuda"))
    assert torch.all(s.short_range_forces() == 0)
    # two particles in different leaves, one mirror pair: equal and opposite forces
    pos = np.array([[0.30, 0.33], [0.5, 0.5], [0.5, 0.5]])
    mass = np.array([0.25, 0.75], dtype=np.float32)
    s2, acc = run_gpu(pos, mass, pm_grid=32, leaf_max=1, p2p_mutual=1)
    ref = oracle.direct_sr(pos, mass, 1.0, s2.rs, s2.rc)
    np.testing.assert_allclose(acc, ref, rtol=1e-5)
    assert abs(acc[0, 0] * 0.25 + acc[0, 1] * 0.75) < 1e-6 * abs(acc[0, 0] * 0.25)
    for kw in (dict(mac_mode=1), dict(size_rule=0), dict(p2p_mutual=2)):
        args = dict(p2p_mutual=1)
        args.update(kw)
        with pytest.raises(hfmm.HfmmError, match="HFMM_ERR_ARG"):
            hfmm.Solver(**args)
