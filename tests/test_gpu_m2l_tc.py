"""Split-precision M2L on tcgen05 tensor cores against the FP64 oracle FMM on
identical lists and against the FP32 CUDA-core M2L.

3xTF32 (m2l_precision = 1): 1e-5 relative RMS, the stated tolerance of the FP32
path.  BF16x3 (m2l_precision = 2): each operand is hi + lo with hi = bf16(x) and
lo = bf16(x - hi), so x is represented to 2^-16 relative and the dropped lo*lo
term is below 2^-16 of the product: at most 3 * 2^-16 = 4.6e-5 relative per
product.  The tolerance is that bound, 5e-5 relative RMS, for the forces and for
the local expansions (the RMS of sums of such products with independent
roundings stays under the per-product bound)."""
import math

import numpy as np
import pytest

import oracle
from force_check import assert_forces_close
from paper_2006_14952_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _run(pos, mass, **kw):
    import torch

    from paper_2006_14952_gb300 import hfmm

    s = hfmm.Solver(**kw)
    s.build_tree(torch.from_numpy(np.ascontiguousarray(pos)).cuda(), torch.from_numpy(mass).cuda())
    acc = s.short_range_forces()
    torch.cuda.synchronize()
    return s, acc.cpu().numpy().astype(np.float64)


def _rel(a, b):
    return math.sqrt(((a - b) ** 2).sum() / (b ** 2).sum())


@pytest.mark.parametrize("order", [2, 4, 5, 6])
def test_tensor_core_m2l_matches_oracle(order):
    pos, mass = W.nfw_clustered(30000, 40, 0.7, 31)
    s, acc = _run(pos, mass, pm_grid=32, order=order, m2l_precision=1)
    p = s.params
    f = oracle.FMM(box=1.0, rs=s.rs, rc=s.rc, theta=p.theta, order=order, leaf_max=p.leaf_max)
    f.build_tree(pos, mass)
    ref = f.forces()
    assert f.size("m2l") > 0
    assert_forces_close(acc, ref)
    _, acc0 = _run(pos, mass, pm_grid=32, order=order, m2l_precision=0)
    assert _rel(acc, acc0) < 1e-5


def test_tensor_core_m2l_locals_match_cuda_core_locals():
    pos, mass = W.nfw_clustered(30000, 40, 0.7, 32)
    s1, _ = _run(pos, mass, pm_grid=32, order=5, m2l_precision=1)
    s0, _ = _run(pos, mass, pm_grid=32, order=5, m2l_precision=0)
    L1, L0 = s1.export("locals").astype(np.float64), s0.export("locals").astype(np.float64)
    assert _rel(L1, L0) < 1e-5


BF16X3_TOL = 5e-5


@pytest.mark.parametrize("order", [2, 4, 6])
def test_bf16x3_m2l_matches_oracle(order):
    pos, mass = W.nfw_clustered(30000, 40, 0.7, 33)
    s, acc = _run(pos, mass, pm_grid=32, order=order, m2l_precision=2)
    p = s.params
    f = oracle.FMM(box=1.0, rs=s.rs, rc=s.rc, theta=p.theta, order=order, leaf_max=p.leaf_max)
    f.build_tree(pos, mass)
    ref = f.forces()
    assert f.size("m2l") > 0
    assert_forces_close(acc, ref, rms_tol=BF16X3_TOL)
    _, acc0 = _run(pos, mass, pm_grid=32, order=order, m2l_precision=0)
    assert _rel(acc, acc0) < BF16X3_TOL


def test_bf16x3_locals_are_a_distinct_split_within_bound():
    """BF16x3 locals within the bound of the FP32 ones, and not the 3xTF32 result
    (which is ~2^-21 away from FP32): the BF16 path is the one that ran."""
    pos, mass = W.nfw_clustered(30000, 40, 0.7, 34)
    s2, _ = _run(pos, mass, pm_grid=32, order=5, m2l_precision=2)
    s1, _ = _run(pos, mass, pm_grid=32, order=5, m2l_precision=1)
    s0, _ = _run(pos, mass, pm_grid=32, order=5, m2l_precision=0)
    L2, L1, L0 = (x.export("locals").astype(np.float64) for x in (s2, s1, s0))
    e2, e1 = _rel(L2, L0), _rel(L1, L0)
    assert e2 < BF16X3_TOL
    assert e1 < 1e-5
    assert e2 > 2 * e1


def test_tensor_core_m2l_rejects_unsupported_order():
    from paper_2006_14952_gb300 import hfmm

    for prec in (1, 2, 3, 4):
        with pytest.raises(hfmm.HfmmError, match="orders 1..6"):
            hfmm.Solver(order=7, m2l_precision=prec)
    with pytest.raises(hfmm.HfmmError, match="m2l_precision"):
        hfmm.Solver(m2l_precision=5)


@pytest.mark.parametrize("precision", [1, 2])
def test_tensor_core_wait_give_up_returns_timeout_and_leaves_the_device_usable(precision):
    """With tc_wait_polls = -1 every chunk's bounded wait gives up without polling:
    the call returns HFMM_ERR_TIMEOUT (each CTA first waits, with the full limit,
    for the MMAs it issued, then frees its tensor memory).  The same context
    fails the same way again, and afterwards a fresh context on the same device
    computes forces that match the oracle."""
    import torch

    from paper_2006_14952_gb300 import hfmm

    pos, mass = W.nfw_clustered(30000, 40, 0.7, 34)
    s = hfmm.Solver(pm_grid=32, order=4, m2l_precision=precision, tc_wait_polls=-1)
    s.build_tree(torch.from_numpy(np.ascontiguousarray(pos)).cuda(), torch.from_numpy(mass).cuda())
    for _ in range(2):
        with pytest.raises(hfmm.HfmmError, match="HFMM_ERR_TIMEOUT"):
            s.short_range_forces()
        torch.cuda.synchronize()
    s2, acc = _run(pos, mass, pm_grid=32, order=4, m2l_precision=precision)
    p = s2.params
    f = oracle.FMM(box=1.0, rs=s2.rs, rc=s2.rc, theta=p.theta, order=4, leaf_max=p.leaf_max)
    f.build_tree(pos, mass)
    assert_forces_close(acc, f.forces(), rms_tol=1e-5 if precision == 1 else BF16X3_TOL)


# ---------------------------------------------------------------- (level, offset) tiles
@pytest.mark.parametrize("precision,order,theta", [(3, 2, 0.5), (3, 4, 0.5), (3, 6, 0.35), (3, 5, 0.6),
                                                   (4, 4, 0.5), (4, 6, 0.35)])
def test_level_offset_tensor_core_m2l_matches_oracle(precision, order, theta):
    """M2L as per-(level, offset) contractions on the tensor cores with the
    accumulators in tensor memory (m2l_precision 3 = 3xTF32, 4 = BF16x3; the
    pairs outside the operator table on the FP32 per-pair kernel): forces
    against the FP64 FMM on identical lists, and the FP32 path on the same set."""
    pos, mass = W.nfw_clustered(40000, 50, 0.7, 35)
    kw = dict(pm_grid=32, order=order, theta=theta, leaf_max=16)
    s, acc = _run(pos, mass, m2l_precision=precision, **kw)
    p = s.params
    f = oracle.FMM(box=1.0, rs=s.rs, rc=s.rc, theta=theta, order=order, leaf_max=16)
    f.build_tree(pos, mass)
    ref = f.forces()
    assert f.size("m2l") > 0
    tol = 1e-5 if precision == 3 else BF16X3_TOL
    print("relative RMS %.3e, per particle %.3e" % assert_forces_close(acc, ref, rms_tol=tol))
    _, acc0 = _run(pos, mass, m2l_precision=0, **kw)
    assert _rel(acc, acc0) < tol


@pytest.mark.parametrize("precision", [3, 4])
def test_level_offset_locals_match_cuda_core_and_are_reproducible(precision):
    pos, mass = W.nfw_clustered(40000, 50, 0.7, 36)
    kw = dict(pm_grid=32, order=6, theta=0.35, leaf_max=16)
    s1, a1 = _run(pos, mass, m2l_precision=precision, **kw)
    s2, a2 = _run(pos, mass, m2l_precision=precision, **kw)
    np.testing.assert_array_equal(a1, a2)
    s0, _ = _run(pos, mass, m2l_precision=0, **kw)
    L1, L0 = s1.export("locals").astype(np.float64), s0.export("locals").astype(np.float64)
    e = _rel(L1, L0)
    print("locals relative RMS %.3e" % e)
    assert e < (1e-5 if precision == 3 else BF16X3_TOL)
    if precision == 4:  # the BF16 split is a different arithmetic from FP32, not the same numbers
        assert e > 1e-8


def test_level_offset_m2l_with_learned_orders_matches_oracle_on_the_same_lists():
    import os

    from paper_2006_14952_gb300 import hfmm

    pos, mass = W.nfw_clustered(30000, 40, 0.7, 44)
    wbits = np.fromfile(os.path.join(os.path.dirname(hfmm.__file__), "weights", "mac_weights.bin"), dtype=np.uint16)
    import torch

    s = hfmm.Solver(pm_grid=32, order=6, theta=0.5, mac_mode=1, m2l_precision=3)
    s.load_mlp(wbits)
    s.build_tree(torch.from_numpy(np.ascontiguousarray(pos)).cuda(), torch.from_numpy(mass).cuda())
    acc = s.short_range_forces().cpu().numpy().astype(np.float64)
    p2p, m2l, orders = s.export("p2p"), s.export("m2l"), s.export("m2l_order")
    assert len(set(orders.tolist())) >= 2
    f = oracle.FMM(box=1.0, rs=s.rs, rc=s.rc, theta=0.5, order=6, leaf_max=16)
    f.build_tree(pos, mass)
    ref = f.forces_given_lists(p2p, m2l, orders)
    assert_forces_close(acc, ref)


@pytest.mark.parametrize("precision", [3, 4])
def test_level_offset_wait_give_up_returns_timeout(precision):
    import torch

    from paper_2006_14952_gb300 import hfmm

    pos, mass = W.nfw_clustered(30000, 40, 0.7, 37)
    s = hfmm.Solver(pm_grid=32, order=4, m2l_precision=precision, tc_wait_polls=-1)
    s.build_tree(torch.from_numpy(np.ascontiguousarray(pos)).cuda(), torch.from_numpy(mass).cuda())
    with pytest.raises(hfmm.HfmmError, match="HFMM_ERR_TIMEOUT"):
        s.short_range_forces()
    torch.cuda.synchronize()
    s2, acc = _run(pos, mass, pm_grid=32, order=4, m2l_precision=precision)
    f = oracle.FMM(box=1.0, rs=s2.rs, rc=s2.rc, theta=s2.params.theta, order=4, leaf_max=16)
    f.build_tree(pos, mass)
    assert_forces_close(acc, f.forces(), rms_tol=1e-5 if precision == 3 else BF16X3_TOL)
