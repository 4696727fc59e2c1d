"""Pins of the PM (long-range) oracle and the KDK step against closed forms.

- A plane-wave mass field on the mesh points gives, in closed form,
  a_x = -4 pi G rho A sin(k x) exp(-k^2 r_s^2) / (k W(k)^2) (normalisation, sign,
  Green function, window and inverse-FFT scaling all enter).
- Two particles: the PM acceleration approaches the periodic long-range pair
  force summed directly over Fourier modes (no mesh) within the mesh error.
- That spectral long-range force plus the FP64 short-range pair force equals
  the periodic Newtonian force -G m r / r^3 + (4 pi / 3) G m r / L^3 (the
  neutralising background of a cubic lattice) up to the next lattice term,
  relative size O((r/L)^5): erfc + erf = 1 (Sec. 2.2 force split).
- Momentum: with the same CIC kernel for assignment and interpolation and an
  odd gradient operator, sum_i m_i a_i = 0 to rounding.
- KDK: a harmonic force field against the leapfrog recurrence.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import pm


def test_plane_wave_closed_form():
    ng, box, rs, G = 32, 1.0, 1.25 / 32, 1.0
    n1, A, mbar = 3, 0.2, 1.0 / ng ** 3
    g = np.arange(ng)
    gx, gy, gz = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([gx.ravel(), gy.ravel(), gz.ravel()]).astype(np.float64) * (box / ng)
    k = 2 * np.pi * n1 / box
    mass = mbar * (1 + A * np.cos(k * pos[0]))
    a = pm.pm_long_range(pos, mass, box, ng, rs, G)
    h = box / ng
    w = (math.sin(k * h / 2) / (k * h / 2)) ** 2
    rho = mbar * ng ** 3 / box ** 3
    want = -4 * np.pi * G * rho * A * np.sin(k * pos[0]) * math.exp(-k * k * rs * rs) / (k * w * w)
    scale = np.abs(want).max()
    assert np.abs(a[0] - want).max() < 1e-10 * scale
    assert np.abs(a[1]).max() < 1e-10 * scale and np.abs(a[2]).max() < 1e-10 * scale


# CIC mesh error of the deconvolved Gaussian-filtered force at r_s = 1.25 cells,
# largest at the shortest separations, where the short-range part dominates
@pytest.mark.parametrize("sep_cells,tol", [(2.0, 0.06), (3.0, 0.04), (5.0, 0.03), (8.0, 0.012)])
def test_two_particles_match_spectral_long_range_force(sep_cells, tol):
    ng, box, G = 64, 1.0, 1.0
    h = box / ng
    rs = 1.25 * h
    rng = np.random.default_rng(int(sep_cells * 10))
    worst = 0.0
    for _ in range(6):
        src = rng.random(3)
        d = rng.normal(size=3)
        d *= sep_cells * h / np.linalg.norm(d)
        pos = np.stack([src, src + d], axis=1)
        a = pm.pm_long_range(pos, np.array([1.0, 0.0]), box, ng, rs, G)[:, 1]
        ref = pm.lr_pair_spectral(d, 1.0, box, rs, G)
        worst = max(worst, np.linalg.norm(a - ref) / np.linalg.norm(ref))
    assert worst < tol, worst


@pytest.mark.parametrize("r_rc", [0.3, 0.7, 1.0, 1.5])
def test_short_plus_long_range_is_newtonian(r_rc):
    box, G = 1.0, 1.0
    rs = 1.25 / 128
    rc = 4.5 * rs
    r = r_rc * rc
    d = np.array([0.6, -0.48, 0.64])
    d *= r / np.linalg.norm(d)
    src = np.array([0.3, 0.4, 0.5])
    pos = np.stack([src, src + d], axis=1)
    # the short-range sum is truncated at R_c: beyond it the long-range part alone must do
    sr = oracle.direct_sr(pos, np.array([1.0, 0.0]), box, rs, rc, G)[:, 1]
    if r >= rc:
        x = r / rs
        s = math.erfc(x / 2) + x / math.sqrt(math.pi) * math.exp(-x * x / 4)
        sr = -G * s * d / r ** 3  # what the untruncated short-range kernel would add
    lr = pm.lr_pair_spectral(d, 1.0, box, rs, G, kmax_rs=8.0)
    newton = -G * d / r ** 3 + 4 * np.pi / 3 * G * d / box ** 3
    err = np.linalg.norm(sr + lr - newton) / np.linalg.norm(newton)
    # the reference omits the next (quartic, cubic-harmonic) term of the periodic
    # lattice potential; its relative size is O((r/L)^5), about 8 (r/L)^5 along d
    assert err < 10 * (r / box) ** 5 + 1e-9, err


def test_momentum_is_conserved():
    rng = np.random.default_rng(5)
    n, ng = 4000, 32
    pos = rng.random((3, n))
    pos[:, : n // 2] = 0.5 + 0.05 * rng.normal(size=(3, n // 2))
    mass = rng.random(n) / n
    a = pm.pm_long_range(pos, mass, 1.0, ng, 1.25 / ng)
    p = (a * mass).sum(axis=1)
    scale = (np.abs(a) * mass).sum()
    assert np.abs(p).max() < 1e-12 * scale


def test_uniform_lattice_has_no_long_range_force():
    ng = 16
    g = (np.arange(2 * ng) + 0.5) / (2 * ng)
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([x.ravel(), y.ravel(), z.ravel()])
    a = pm.pm_long_range(pos, np.full(pos.shape[1], 1.0 / pos.shape[1]), 1.0, ng, 1.25 / ng)
    assert np.abs(a).max() < 1e-12


def test_kdk_matches_leapfrog_recurrence_for_harmonic_force():
    w2, dt = 4.0, 0.01
    x0 = np.array([[0.5 + 0.01], [0.5], [0.5]])
    v0 = np.zeros((3, 1))

    def forces(p):
        return -w2 * (p - 0.5)

    x, v, a = x0.copy(), v0.copy(), forces(x0)
    for _ in range(10):
        x, v, a = pm.kdk_step(x, v, a, dt, 1.0, forces)
    # leapfrog of the oscillator: exact recurrence in the displacement q
    q, p = 0.01, 0.0
    for _ in range(10):
        p += 0.5 * dt * (-w2 * q)
        q += dt * p
        p += 0.5 * dt * (-w2 * q)
    assert abs((x[0, 0] - 0.5) - q) < 1e-15 and abs(v[0, 0] - p) < 1e-15
