"""Pins for the oracle's expansion operators (Sec. 2.1, Eqs. p2m, m2m, m2l, l2l, l2p).

Exact identities: M2M after P2M equals P2M about the new centre, the monopole is
the total mass, L2L is exact for the degree-p polynomial a local expansion
represents, and M2L + L2P converges geometrically in p to the direct sum of the
truncated potential (computed here from the printed force law, not the oracle).
"""
import math

import numpy as np
import pytest

import oracle


def test_monopole_and_dipole():
    rng = np.random.default_rng(1)
    x = rng.random((20, 3))
    mu = rng.random(20)
    z = np.array([0.5, 0.5, 0.5])
    M = oracle.p2m(x, mu, z, 4)
    im = {tuple(int(v) for v in m): c for c, m in enumerate(oracle.multi_indices(4))}
    assert M[im[(0, 0, 0)]] == pytest.approx(mu.sum(), rel=1e-14)
    # (-1)^1 / 1! sum mu (x - z)
    for d, e in enumerate([(1, 0, 0), (0, 1, 0), (0, 0, 1)]):
        assert M[im[e]] == pytest.approx(-(mu * (x[:, d] - z[d])).sum(), rel=1e-13)
    # second moment xx: + 1/2 sum mu dx^2
    assert M[im[(2, 0, 0)]] == pytest.approx(0.5 * (mu * (x[:, 0] - z[0]) ** 2).sum(), rel=1e-13)


@pytest.mark.parametrize("p", [2, 4, 7])
def test_m2m_of_p2m_is_p2m_at_new_centre(p):
    rng = np.random.default_rng(p)
    x = rng.random((30, 3)) * 0.25
    mu = rng.random(30)
    z = np.array([0.125, 0.125, 0.125])
    shift = np.array([0.125, -0.125, 0.125])
    M = oracle.p2m(x, mu, z, p)
    M2 = oracle.m2m(M, shift, p)
    ref = oracle.p2m(x, mu, z + shift, p)
    np.testing.assert_allclose(M2, ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())


@pytest.mark.parametrize("p", [1, 4, 8])
def test_l2l_exact_for_polynomials(p):
    rng = np.random.default_rng(10 + p)
    L = rng.standard_normal(oracle.ncoef(p))
    x = rng.standard_normal(3) * 0.3
    for _ in range(5):
        u = rng.standard_normal(3) * 0.2
        ph1, a1 = oracle.l2p(oracle.l2l(L, x, p), u, p)
        ph0, a0 = oracle.l2p(L, x + u, p)
        assert ph1 == pytest.approx(ph0, rel=1e-11, abs=1e-12)
        np.testing.assert_allclose(a1, a0, rtol=1e-11, atol=1e-12)


def test_l2p_gradient_matches_finite_difference_of_potential():
    p = 5
    rng = np.random.default_rng(3)
    L = rng.standard_normal(oracle.ncoef(p))
    u = np.array([0.1, -0.05, 0.2])
    _, a = oracle.l2p(L, u, p)
    h = 1e-6
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        fd = (oracle.l2p(L, u + e, p)[0] - oracle.l2p(L, u - e, p)[0]) / (2 * h)
        assert a[d] == pytest.approx(fd, rel=1e-6)


def _direct_potential_and_acc(xs, mu, xb, rs):
    """Sum of the Sec. 2.2 potential erfc(r/2rs)/r and force f_(1) r (printed forms), no cutoff."""
    phi, acc = 0.0, np.zeros(3)
    for xa, m in zip(xs, mu):
        d = xb - xa
        r = math.sqrt(d @ d)
        phi += m * math.erfc(r / (2 * rs)) / r
        f1 = -(1 / r ** 3) * (math.erfc(r / (2 * rs)) + r / (rs * math.sqrt(math.pi)) * math.exp(-r * r / (4 * rs * rs)))
        acc += m * f1 * d
    return phi, acc


def test_m2l_l2p_converges_geometrically_to_direct_sum():
    rng = np.random.default_rng(7)
    h = 0.1
    zA = np.array([0.05, 0.05, 0.05])
    zB = zA + np.array([3 * h, h, 0.0])
    xs = zA + (rng.random((25, 3)) - 0.5) * h
    mu = rng.random(25)
    xb = zB + (rng.random(3) - 0.5) * h
    rs = 0.2
    phi_ref, a_ref = _direct_potential_and_acc(xs, mu, xb, rs)
    errs = []
    for p in (2, 4, 6, 8, 10):
        M = oracle.p2m(xs, mu, zA, p)
        L = oracle.m2l(M, zB - zA, rs, p)
        phi, a = oracle.l2p(L, xb - zB, p)
        errs.append(np.linalg.norm(a - a_ref) / np.linalg.norm(a_ref))
        assert phi == pytest.approx(phi_ref, rel=10 * errs[-1] + 1e-12)
    # separation ~3.2 cell sides: the error falls by well over 2x per two orders
    for e0, e1 in zip(errs, errs[1:]):
        assert e1 < 0.4 * e0
    assert errs[-1] < 2e-5


def test_m2l_newtonian_limit():
    """With r_s -> infinity the truncated M2L becomes the Newtonian one (1/r kernel)."""
    rng = np.random.default_rng(8)
    xs = (rng.random((10, 3)) - 0.5) * 0.1
    mu = rng.random(10)
    zB = np.array([0.4, 0.1, -0.1])
    xb = zB + np.array([0.01, -0.02, 0.015])
    ref = np.zeros(3)
    for x, m in zip(xs, mu):
        d = xb - x
        ref += -m * d / np.linalg.norm(d) ** 3
    errs = []
    for p in (4, 8, 10):
        L = oracle.m2l(oracle.p2m(xs, mu, np.zeros(3), p), zB, 0.0, p)
        _, a = oracle.l2p(L, xb - zB, p)
        errs.append(np.linalg.norm(a - ref) / np.linalg.norm(ref))
    # (source radius + sink offset) / separation ~ 0.27: error ~ 0.27^(p+1)
    assert errs[0] < 1e-3 and errs[1] < 1e-5 and errs[2] < 0.3 * errs[1]
