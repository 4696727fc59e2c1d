"""Short-range forces in sink batches (sink_batches): the walk over the top
levels, then each batch of sinks walked to the leaves and evaluated before the
next.  The batches partition the walk: the M2L and P2P entry totals equal those
of one walk exactly, the forces match the FP64 oracle FMM (the same lists as
one walk) within the FP32 tolerance and the one-batch forces to rounding (a
leaf above the batch level sums its entries in two groups), and list overflows
inside a batch are grown and repeated per batch."""
import math

import numpy as np
import pytest

import oracle
from force_check import assert_forces_close
from paper_2006_14952_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def run(pos, mass, **kw):
    import torch

    from paper_2006_14952_gb300 import hfmm

    s = hfmm.Solver(**kw)
    s.build_tree(torch.from_numpy(np.ascontiguousarray(pos)).cuda(), torch.from_numpy(mass).cuda())
    a = s.short_range_forces()
    torch.cuda.synchronize()
    return s, a.cpu().numpy().astype(np.float64)


def rel(a, b):
    return math.sqrt(((a - b) ** 2).sum() / (b ** 2).sum())


@pytest.mark.parametrize("nbatch", [2, 3, 7, 40])
def test_sink_batches_partition_the_walk_and_match_the_oracle(nbatch):
    pos, mass = W.nfw_clustered(60000, 60, 0.7, 81)
    kw = dict(pm_grid=32, theta=0.4, order=5, leaf_max=16)
    s1, a1 = run(pos, mass, sink_batches=1, **kw)
    sb, ab = run(pos, mass, sink_batches=nbatch, **kw)
    st1, stb = s1.get_stats(), sb.get_stats()
    assert stb["sink_batches"] == nbatch and st1["sink_batches"] == 1
    assert stb["nm2l"] == st1["nm2l"] and stb["np2p"] == st1["np2p"]
    assert stb["traverse_walks"] >= 2
    assert rel(ab, a1) < 1e-6
    f = oracle.FMM(box=1.0, rs=s1.rs, rc=s1.rc, theta=0.4, order=5, leaf_max=16)
    f.build_tree(pos, mass)
    assert_forces_close(ab, f.forces())


def test_sink_batches_grow_overflowing_lists_per_batch():
    pos, mass = W.nfw_clustered(40000, 40, 0.7, 82)
    kw = dict(pm_grid=32, theta=0.5, order=4, leaf_max=16)
    s1, a1 = run(pos, mass, **kw)
    sb, ab = run(pos, mass, sink_batches=5, list_init=64, **kw)
    stb = sb.get_stats()
    assert stb["traverse_walks"] > 6  # the top walk and five batches, some repeated
    assert stb["nm2l"] == s1.get_stats()["nm2l"] and stb["np2p"] == s1.get_stats()["np2p"]
    assert rel(ab, a1) < 1e-6


def test_sink_batches_lists_are_not_exported():
    from paper_2006_14952_gb300 import hfmm

    pos, mass = W.uniform(20000, 83)
    sb, _ = run(pos, mass, pm_grid=32, sink_batches=3)
    with pytest.raises(hfmm.HfmmError, match="STATE"):
        sb.export("p2p")
    assert sb.export("perm").shape[0] == 20000


@pytest.mark.parametrize("kw", [dict(m2l_precision=1), dict(p2p_mutual=1), dict(split=1)])
def test_sink_batches_with_the_other_paths(kw):
    pos, mass = W.nfw_clustered(30000, 30, 0.7, 84)
    base = dict(pm_grid=32, theta=0.4, order=4, leaf_max=16)
    _, a1 = run(pos, mass, sink_batches=1, **base, **kw)
    _, ab = run(pos, mass, sink_batches=4, **base, **kw)
    assert rel(ab, a1) < (5e-6 if kw.get("p2p_mutual") else 1e-6)


def test_automatic_batches_above_the_list_guess():
    """At 8M particles the first guess of the P2P list passes 2^28 entries:
    the call takes several batches by itself, with the same totals as one."""
    pos, mass = W.uniform(8_000_000, 85)
    kw = dict(pm_grid=128, theta=0.5, order=4, leaf_max=48)
    sa, aa = run(pos, mass, **kw)
    s1, a1 = run(pos, mass, sink_batches=1, **kw)
    assert sa.get_stats()["sink_batches"] > 1
    assert sa.get_stats()["np2p"] == s1.get_stats()["np2p"]
    assert rel(aa, a1) < 1e-6
