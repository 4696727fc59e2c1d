"""M2L through the per-(level, offset) operator table, against the FP64 oracle.

Same-level pairs whose integer cell offset o has |o_d| <= K = 2 floor(1/theta) + 1
read their operator T_c = D_c(-o h) h^(|c|+1) (Eq. m2l, truncated D of Sec. 2.2)
from the table; the others evaluate it per pair.  Checked here: which pairs take
the table path (exact count from the exported lists), forces of the table path
and of the per-pair path against the FP64 FMM on identical lists (1e-5 relative
RMS), and the two FP32 paths against each other.
"""
import math

import numpy as np
import pytest

import oracle
from force_check import assert_forces_close
from paper_2006_14952_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-5


def run(pos, mass, **kw):
    import torch

    from paper_2006_14952_gb300 import hfmm

    s = hfmm.Solver(**kw)
    s.build_tree(torch.from_numpy(np.ascontiguousarray(pos)).cuda(), torch.from_numpy(mass).cuda())
    acc = s.short_range_forces()
    torch.cuda.synchronize()
    return s, acc.cpu().numpy().astype(np.float64)


def rel_rms(a, ref):
    return math.sqrt(((a - ref) ** 2).sum() / max((ref ** 2).sum(), 1e-300))


def table_pairs(nodes, m2l, theta):
    """Number of M2L rows with equal levels and |o_d| <= 2 floor(1/theta) + 1."""
    k = 2 * int(math.floor(1.0 / theta)) + 1
    a, b, s = m2l[:, 0], m2l[:, 1], m2l[:, 2]
    lev = nodes[:, 0]
    ic = nodes[:, 1:4]
    sh = np.stack([s // 9 - 1, (s // 3) % 3 - 1, s % 3 - 1], axis=1)
    same = lev[a] == lev[b]
    o = ic[b] - ic[a] + sh * (1 << lev[a])[:, None]
    return int((same & (np.abs(o).max(axis=1) <= k)).sum())


@pytest.mark.parametrize("theta,order", [(0.5, 4), (0.3, 5), (0.4, 7)])
def test_table_pair_count_and_forces(theta, order):
    pos, mass = W.nfw_clustered(60000, 60, 0.7, 21)
    s, acc = run(pos, mass, pm_grid=32, theta=theta, order=order, m2l_tables=1, profile=2)
    st = s.get_stats()
    nodes = s.export("nodes")
    m2l = s.export("m2l")
    want = table_pairs(nodes, m2l, theta)
    assert st["nm2l_table"] == want
    assert want > 0.5 * len(m2l)  # the table serves most pairs
    p = s.params
    f = oracle.FMM(box=p.box, rs=s.rs, rc=s.rc, G=p.G, theta=theta, order=order, leaf_max=p.leaf_max,
                   transition_rule=p.transition_rule, size_rule=p.size_rule)
    f.build_tree(pos, mass)
    ref = f.forces()
    assert_forces_close(acc, ref)


def test_table_and_per_pair_operators_agree():
    pos, mass = W.nfw_clustered(60000, 60, 0.7, 22)
    s1, a1 = run(pos, mass, pm_grid=32, theta=0.3, order=5, m2l_tables=1, profile=2)
    s0, a0 = run(pos, mass, pm_grid=32, theta=0.3, order=5, m2l_tables=0, profile=2)
    assert s0.get_stats()["nm2l_table"] == 0
    assert s1.get_stats()["nm2l_table"] > 0
    p = s1.params
    f = oracle.FMM(box=p.box, rs=s1.rs, rc=s1.rc, G=p.G, theta=0.3, order=5, leaf_max=p.leaf_max,
                   transition_rule=p.transition_rule, size_rule=p.size_rule)
    f.build_tree(pos, mass)
    ref = f.forces()
    assert_forces_close(a1, ref)
    assert_forces_close(a0, ref)
    # both are FP32 evaluations of the same sums: they differ by rounding only
    assert rel_rms(a1, a0) < FORCE_TOL


def test_table_local_expansions_match_oracle():
    """Local expansions after M2L + L2L, degree by degree, with the table path on."""
    pos, mass = W.nfw_clustered(40000, 40, 0.7, 23)
    order = 5
    s, _ = run(pos, mass, pm_grid=32, theta=0.3, order=order, m2l_tables=1)
    p = s.params
    f = oracle.FMM(box=p.box, rs=s.rs, rc=s.rc, G=p.G, theta=0.3, order=order, leaf_max=p.leaf_max,
                   transition_rule=p.transition_rule, size_rule=p.size_rule)
    f.build_tree(pos, mass)
    f.forces()
    nodes = f.nodes()
    h = 1.0 / 2.0 ** nodes[:, 0]
    deg = oracle.multi_indices(order).sum(axis=1)
    Lg = s.export("locals").astype(np.float64) / h[:, None] ** (deg[None, :] + 1)
    Lo = f.expansions("L")
    for k in range(order + 1):
        sel = deg == k
        err = np.sqrt(((Lg[:, sel] - Lo[:, sel]) ** 2).sum() / max((Lo[:, sel] ** 2).sum(), 1e-300))
        assert err < 1e-5, (k, err)
