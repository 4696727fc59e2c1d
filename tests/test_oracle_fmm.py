"""Pins for the oracle's direct truncated sum and whole FMM (Secs. 2.1-2.3).

Direct sum: the two-particle closed form of the force law g(r) (Sec. 2.2), zero
force on a perfect lattice, pairwise antisymmetry (total momentum change 0),
the hard cutoff, and an O(N^2) all-images brute force.  FMM: with theta = 0 no
M2L is accepted and the result is the direct sum up to rounding; with theta > 0
the error falls with the expansion order and with the opening angle (the trend
of Fig. 4).
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2006_14952_gb300 import workloads as W


def g_printed(d, rs):
    r = math.sqrt(d @ d)
    return -(d / r ** 3) * (math.erfc(r / (2 * rs)) + r / (rs * math.sqrt(math.pi)) * math.exp(-r * r / (4 * rs * rs)))


def test_two_particle_closed_form_and_periodic_image():
    rs, rc = 0.04, 0.18
    pos = np.array([[0.1, 0.97], [0.5, 0.52], [0.5, 0.49]])  # separation through the x boundary
    mass = np.array([0.25, 0.75])
    acc = oracle.direct_sr(pos, mass, 1.0, rs, rc, G=2.0)
    d = np.array([0.1 - (0.97 - 1.0), 0.5 - 0.52, 0.5 - 0.49])
    np.testing.assert_allclose(acc[:, 0], 2.0 * 0.75 * g_printed(d, rs), rtol=1e-13)
    np.testing.assert_allclose(acc[:, 1], 2.0 * 0.25 * g_printed(-d, rs), rtol=1e-13)
    # beyond the cutoff nothing acts
    pos2 = np.array([[0.1, 0.1 + rc * 1.0000001], [0.5, 0.5], [0.5, 0.5]])
    assert np.all(oracle.direct_sr(pos2, mass, 1.0, rs, rc) == 0.0)
    pos3 = np.array([[0.1, 0.1 + rc * 0.9999999], [0.5, 0.5], [0.5, 0.5]])
    assert np.all(oracle.direct_sr(pos3, mass, 1.0, rs, rc)[0] != 0.0)


def test_lattice_has_zero_force():
    pos, mass = W.lattice(12)
    acc = oracle.direct_sr(pos, mass, 1.0, 1.25 / 12, 4.5 * 1.25 / 12)
    ref = abs(0.75 / 144 * g_printed(np.array([1 / 12, 0, 0]), 1.25 / 12)[0])
    assert np.abs(acc).max() < 1e-12 * ref


def test_antisymmetry_total_momentum():
    pos, mass = W.nfw_clustered(4000, 10, 0.7, 3)
    mass = mass * np.random.default_rng(0).uniform(0.5, 1.5, len(mass))
    acc = oracle.direct_sr(pos, mass, 1.0, 0.02, 0.09)
    tot = (acc * mass).sum(axis=1)
    scale = (np.abs(acc) * mass).sum()
    assert np.abs(tot).max() < 1e-12 * scale


def test_direct_sum_equals_all_images_brute_force():
    pos, mass = W.nfw_clustered(150, 3, 0.5, 9)
    rs, rc = 0.07, 0.3
    acc = oracle.direct_sr(pos, mass, 1.0, rs, rc)
    ref = np.zeros_like(acc)
    for i in range(150):
        for j in range(150):
            for s in itertools.product([-1, 0, 1], repeat=3):
                d = pos[:, i] - (pos[:, j] + np.array(s))
                r2 = d @ d
                if 0 < r2 < rc * rc:
                    ref[:, i] += mass[j] * g_printed(d, rs)
    np.testing.assert_allclose(acc, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    sinks = np.array([5, 77, 149])
    np.testing.assert_array_equal(oracle.direct_sr(pos, mass, 1.0, rs, rc, sinks=sinks), acc[:, sinks])


@pytest.mark.parametrize("kind", ["uniform", "nfw"])
def test_fmm_with_theta_zero_is_the_direct_sum(kind):
    n = 5000
    pos, mass = (W.uniform(n, 1) if kind == "uniform" else W.nfw_clustered(n, 12, 0.7, 2))
    rs = 1.25 / 24
    rc = 4.5 * rs
    f = oracle.FMM(box=1.0, rs=rs, rc=rc, theta=0.0, order=4, leaf_max=16)
    f.build_tree(pos, mass)
    a = f.forces()
    assert f.size("m2l") == 0
    ref = oracle.direct_sr(pos, mass, 1.0, rs, rc)
    np.testing.assert_allclose(a, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


def rel_err(a, ref):
    e = np.linalg.norm(a - ref, axis=0) / np.linalg.norm(ref, axis=0)
    return math.sqrt((e ** 2).mean()), float(np.percentile(e, 99))


@pytest.fixture(scope="module")
def clustered_small():
    cfg = W.scaled(W.CONFIGS["nfw-2m"], 20000, pm_grid=32, halo_count=40)
    pos, mass = W.make(cfg)
    ref = oracle.direct_sr(pos, mass, 1.0, cfg.rs, cfg.rc)
    return cfg, pos, mass, ref


def test_fmm_error_falls_with_order(clustered_small):
    cfg, pos, mass, ref = clustered_small
    errs = []
    for p in (2, 4, 6):
        f = oracle.FMM(box=1.0, rs=cfg.rs, rc=cfg.rc, theta=0.5, order=p, leaf_max=16)
        f.build_tree(pos, mass)
        errs.append(rel_err(f.forces(), ref)[0])
    assert errs[1] < 0.5 * errs[0] and errs[2] < 0.5 * errs[1]


def test_fmm_error_falls_with_opening_angle(clustered_small):
    cfg, pos, mass, ref = clustered_small
    errs = []
    for th in (0.7, 0.5, 0.3):
        f = oracle.FMM(box=1.0, rs=cfg.rs, rc=cfg.rc, theta=th, order=4, leaf_max=16)
        f.build_tree(pos, mass)
        errs.append(rel_err(f.forces(), ref)[0])
    assert errs[0] > errs[1] > errs[2]


def test_fmm_reaches_the_direct_sum_at_small_theta_high_order(clustered_small):
    cfg, pos, mass, ref = clustered_small
    f = oracle.FMM(box=1.0, rs=cfg.rs, rc=cfg.rc, theta=0.3, order=6, leaf_max=16)
    f.build_tree(pos, mass)
    rms, p99 = rel_err(f.forces(), ref)
    assert rms < 5e-5 and p99 < 2e-4
