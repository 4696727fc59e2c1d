"""Split-precision M2L (3xTF32 on tcgen05 tensor cores, m2l_precision = 1)
against the FP64 oracle FMM on identical lists (1e-5 relative RMS, the stated
tolerance for the FP32 path) and against the FP32 CUDA-core M2L."""
import math

import numpy as np
import pytest

import oracle
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
    assert _rel(acc, ref) < 1e-5
    _, acc0 = _run(pos, mass, pm_grid=32, order=order, m2l_precision=0)
    assert _rel(acc, acc0) < 1e-5


def test_tensor_core_m2l_locals_match_cuda_core_locals():
    pos, mass = W.nfw_clustered(30000, 40, 0.7, 32)
    s1, _ = _run(pos, mass, pm_grid=32, order=5, m2l_precision=1)
    s0, _ = _run(pos, mass, pm_grid=32, order=5, m2l_precision=0)
    L1, L0 = s1.export("locals").astype(np.float64), s0.export("locals").astype(np.float64)
    assert _rel(L1, L0) < 1e-5


def test_tensor_core_m2l_rejects_unsupported_order():
    from paper_2006_14952_gb300 import hfmm

    with pytest.raises(hfmm.HfmmError, match="orders 1..6"):
        hfmm.Solver(order=7, m2l_precision=1)
