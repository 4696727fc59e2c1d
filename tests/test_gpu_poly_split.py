"""The polynomial truncation of the force split (Sec. 5; split = 1, kernel
1/r - P(r) inside R_c) on the GPU against the FP64 oracle in the same split:

- forces on identical lists (the oracle's FMM in its polynomial mode) within
  the tolerances of the Gaussian path, at several orders and leaf sizes;
- theta = 0 (all P2P) against the oracle's direct sum with the polynomial pair
  law at full size;
- the pair law over (0.03, 1) R_c, pair by pair;
- the PM long range with the polynomial split's Green function against the PM
  oracle given the same (separately pinned) Green function;
- parameter combinations the split does not support are rejected.
"""
import math

import numpy as np
import pytest

import oracle
from force_check import assert_forces_close
from oracle import pm as opm
from oracle import poly_split as PS
from paper_2006_14952_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def run_gpu(pos, mass, **kw):
    import torch

    from paper_2006_14952_gb300 import hfmm

    s = hfmm.Solver(split=1, **kw)
    s.build_tree(torch.from_numpy(np.ascontiguousarray(pos)).cuda(), torch.from_numpy(mass).cuda())
    acc = s.short_range_forces()
    torch.cuda.synchronize()
    return s, acc.cpu().numpy().astype(np.float64)


def oracle_fmm(pos, mass, s):
    p = s.params
    f = oracle.FMM(box=p.box, rs=s.rs, rc=s.rc, G=p.G, theta=p.theta, order=p.order, leaf_max=p.leaf_max,
                   transition_rule=p.transition_rule, size_rule=p.size_rule, split="poly")
    f.build_tree(pos, mass)
    return f


@pytest.mark.parametrize("order,leaf,theta", [(2, 16, 0.5), (4, 16, 0.5), (6, 48, 0.35), (8, 16, 0.4)])
def test_forces_match_fp64_fmm_on_identical_lists(order, leaf, theta):
    pos, mass = W.nfw_clustered(50000, 60, 0.7, 12)
    s, acc = run_gpu(pos, mass, pm_grid=32, order=order, leaf_max=leaf, theta=theta)
    f = oracle_fmm(pos, mass, s)
    ref = f.forces()
    assert f.size("m2l") > 0 and f.size("p2p") > 0
    print("relative RMS %.3e, per particle %.3e" % assert_forces_close(acc, ref))


def test_theta_zero_equals_the_polynomial_direct_sum_at_full_uniform_size():
    pos, mass = W.make(W.CONFIGS["uniform-32k"])
    s, acc = run_gpu(pos, mass, pm_grid=32, theta=0.0)
    assert s.get_stats()["nm2l"] == 0
    ref = oracle.direct_sr(pos, mass, 1.0, s.rs, s.rc, split="poly")
    assert_forces_close(acc, ref)


def test_pair_force_law_across_the_cutoff_range():
    """1000 isolated pairs, separations log-spaced over (0.03, 1) R_c, against the
    FP64 law m f_(1)(r) r, f_(1) = -1/r^3 + 5/(2 R_c^3) - 3 r^2/(2 R_c^5).  The
    law cancels to zero at R_c, so errors are measured in units of the Newtonian
    pull m / r^2 of the pair: 3e-6 for the FP32 evaluation at given FP32
    separations (rsqrt a few 2^-22, sums a few ulp), plus the rounding of the
    separation carried through the three terms (each at most cubic in r):
    3 * 2 * 2^-24 * (1 + sqrt(3) h_leaf / r)."""
    rng = np.random.default_rng(5)
    g = (np.arange(10) + 0.5) / 10.0
    cx, cy, cz = np.meshgrid(g, g, g, indexing="ij")
    centres = np.stack([cx.ravel(), cy.ravel(), cz.ravel()])
    from paper_2006_14952_gb300 import hfmm

    rc = hfmm.Solver(pm_grid=128, split=1).rc
    r = rc * np.logspace(-1.5, np.log10(0.9999), 1000)
    d = rng.standard_normal((3, 1000))
    d /= np.linalg.norm(d, axis=0)
    pos = np.concatenate([centres, centres + r * d], axis=1)
    mass = np.full(2000, 1 / 2000, dtype=np.float32)
    s, acc = run_gpu(pos, mass, pm_grid=128)
    ref = oracle.direct_sr(pos, mass, 1.0, s.rs, s.rc, split="poly")
    rr = np.concatenate([r, r])
    newton = (1 / 2000) / rr ** 2
    e = np.linalg.norm(acc - ref, axis=0) / newton
    nodes = s.export("nodes")
    h_leaf = (1.0 / 2.0 ** nodes[nodes[:, 7] == 0, 0]).max()
    bound = 3e-6 + 6 * 2.0 ** -24 * (1 + np.sqrt(3) * h_leaf / rr)
    w = int(np.argmax(e / bound))
    assert np.all(e < bound), f"worst r/R_c {rr[w] / rc:.4f}: err {e[w]:.3e} > bound {bound[w]:.3e}"
    # and the law itself: the FP64 reference is the pinned closed form
    m = float(mass[0])  # the FP32 mass the particles carry
    np.testing.assert_allclose(ref[:, :1000], (m * PS.pair_factor(r, s.rc))[None, :] * (-r * d),
                               rtol=1e-12, atol=1e-14 * np.abs(ref).max())


@pytest.mark.parametrize("ng,n", [(32, 40000), (48, 30001)])
def test_pm_with_the_polynomial_green_function_matches_oracle(ng, n):
    import torch

    from paper_2006_14952_gb300 import hfmm

    pos, mass = W.nfw_clustered(n, 40, 0.6, 91 + ng)
    s = hfmm.Solver(pm_grid=ng, split=1)
    s.build_tree(torch.from_numpy(pos).cuda(), torch.from_numpy(mass).cuda())
    a = s.pm_long_range().cpu().numpy().astype(np.float64)
    rc = s.rc
    ref = opm.pm_long_range(pos, mass.astype(np.float32).astype(np.float64), 1.0, ng, s.rs, 1.0,
                            green_k2=lambda k2: PS.green_long(np.sqrt(k2), rc))
    err = math.sqrt(((a - ref) ** 2).sum() / (ref ** 2).sum())
    assert err < 1e-5, err
    # a different split gives a different long range (the table is the one in use)
    g = hfmm.Solver(pm_grid=ng)
    g.build_tree(torch.from_numpy(pos).cuda(), torch.from_numpy(mass).cuda())
    ag = g.pm_long_range().cpu().numpy().astype(np.float64)
    assert math.sqrt(((ag - ref) ** 2).sum() / (ref ** 2).sum()) > 1e-3


def test_unsupported_combinations_are_rejected():
    from paper_2006_14952_gb300 import hfmm

    for kw in (dict(mac_mode=1), dict(m2l_precision=1), dict(m2l_tables=1), dict(split=2)):
        args = dict(split=1)
        args.update(kw)
        with pytest.raises(hfmm.HfmmError, match="HFMM_ERR_ARG"):
            hfmm.Solver(**args)
