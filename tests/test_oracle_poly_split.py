"""Pins for the polynomial truncation of the force split (oracle/poly_split.py).

Sec. 5 allows a polynomial truncation function in place of the Gaussian one,
with the prefactors generated as in Sec. 2.2.  The oracle's reading is checked
here against what fixes it independently of its own formulas: the even quartic
P is solved for from the three conditions at R_c (value and two derivatives of
1/r - P vanish), the prefactors are differentiated symbolically, the Fourier
transform of the short-range kernel is integrated symbolically, and the pair
sum is checked for antisymmetry, the cut-off and the Newtonian limit.
"""
import math

import numpy as np
import pytest

from oracle import poly_split as PS

sp = pytest.importorskip("sympy")

RC = 0.17


def _symbolic_kernel():
    r, R = sp.symbols("r R", positive=True)
    a0, a2, a4 = sp.symbols("a0 a2 a4")
    P = a0 + a2 * r ** 2 + a4 * r ** 4  # an even quartic
    psi = 1 / r - P
    sol = sp.solve([psi.subs(r, R), sp.diff(psi, r).subs(r, R), sp.diff(psi, r, 2).subs(r, R)], [a0, a2, a4],
                   dict=True)[0]
    return r, R, sp.simplify(psi.subs(sol))


def test_the_quartic_is_fixed_by_the_three_conditions_at_the_cutoff():
    r, R, psi = _symbolic_kernel()
    f = sp.lambdify((r, R), psi, "math")
    for x in (0.01, 0.2, 0.5, 0.9, 0.999):
        assert PS.psi_sr(x * RC, RC) == pytest.approx(f(x * RC, RC), rel=1e-13)
    assert PS.psi_sr(RC, RC) == 0.0 and PS.psi_sr(1.2 * RC, RC) == 0.0 and PS.psi_sr(0.0, RC) == 0.0


@pytest.mark.parametrize("x", [0.05, 0.3, 0.62, 0.97])
def test_prefactors_are_the_symbolic_radial_derivatives(x):
    r, R, psi = _symbolic_kernel()
    expr = psi
    p = 6
    got = PS.prefactors(x * RC, RC, p)
    for k in range(p + 1):
        want = float(expr.subs({r: x * RC, R: RC}))
        assert got[k] == pytest.approx(want, rel=1e-11), k
        expr = sp.diff(expr, r) / r
    # beyond k = 2 the polynomial part is gone: the Newtonian prefactors remain
    newton = [(-1) ** k * math.prod(range(1, 2 * k, 2)) / (x * RC) ** (2 * k + 1) for k in range(3, p + 1)]
    assert np.allclose(got[3:], newton, rtol=1e-13)


def test_pair_factor_is_the_first_prefactor_inside_and_zero_outside():
    rs = np.array([1e-3, 0.1, 0.5, 0.9, 0.99]) * RC
    assert np.allclose(PS.pair_factor(rs, RC), [PS.prefactors(v, RC, 1)[1] for v in rs], rtol=1e-14)
    assert (PS.pair_factor(np.array([0.0, RC, 1.5 * RC]), RC) == 0).all()
    # the force goes to zero continuously at the cut-off (second-order contact)
    eps = 1e-4
    assert abs(PS.pair_factor((1 - eps) * RC, RC)) * RC ** 3 < 10 * eps ** 2


def test_newtonian_limit_for_a_far_cutoff():
    r = np.array([0.01, 0.1, 0.3])
    assert np.allclose(PS.pair_factor(r, 1e6), -1.0 / r ** 3, rtol=1e-12)


def test_transform_matches_the_symbolic_integral():
    r, R, psi = _symbolic_kernel()
    k = sp.symbols("k", positive=True)
    hat = 4 * sp.pi / k * sp.integrate(sp.expand(r * psi) * sp.sin(k * r), (r, 0, R))
    # the closed form cancels heavily at small k R_c: evaluate it with 60 digits
    mpmath = pytest.importorskip("mpmath")
    f = sp.lambdify((k, R), hat, "mpmath")
    with mpmath.workdps(60):
        for u in (0.05, 0.7, 3.0, 11.0, 40.0):
            kv = u / RC
            want = float(f(mpmath.mpf(u) / mpmath.mpf(RC), mpmath.mpf(RC)))
            assert PS.psi_sr_hat(kv, RC)[0] == pytest.approx(want, rel=1e-10), u
    # small-k limit: 4 pi int r^2 psi_SR = 4 pi R_c^2 / 14
    assert PS.psi_sr_hat(1e-4 / RC, RC)[0] == pytest.approx(4 * math.pi * RC ** 2 / 14, rel=1e-7)


def test_long_range_green_function_is_finite_at_small_k_and_decays():
    k = np.array([1e-3, 1e-2]) / RC
    # 4 pi / k^2 - G_L(k) -> 4 pi R_c^2 / 14
    assert np.allclose(4 * math.pi / k ** 2 - PS.green_long(k, RC), 4 * math.pi * RC ** 2 / 14, rtol=1e-5)
    big = np.array([60.0, 90.0]) / RC
    assert (np.abs(PS.green_long(big, RC)) * big ** 2 < 0.05 * 4 * math.pi).all()


def test_direct_sum_is_antisymmetric_and_truncated():
    rng = np.random.default_rng(5)
    pos = rng.random((3, 300))
    mass = rng.random(300)
    a = PS.direct_sr(pos, mass, 1.0, RC)
    assert np.abs((a * mass).sum(1)).max() < 1e-9 * np.abs(a * mass).sum()
    two = np.array([[0.1, 0.1 + 0.9 * RC], [0.5, 0.5], [0.5, 0.5]])
    a2 = PS.direct_sr(two, np.array([1.0, 2.0]), 1.0, RC)
    d = -0.9 * RC
    assert a2[0, 0] == pytest.approx(2.0 * PS.pair_factor(0.9 * RC, RC) * d, rel=1e-14)
    far = np.array([[0.1, 0.1 + 1.01 * RC], [0.5, 0.5], [0.5, 0.5]])
    assert (PS.direct_sr(far, np.ones(2), 1.0, RC) == 0).all()


# ---------------------------------------------------------------- the C oracle's split mode
import oracle  # noqa: E402
from oracle import pm as PM  # noqa: E402


@pytest.mark.parametrize("x", [0.05, 0.3, 0.62, 0.97])
def test_c_prefactors_are_the_symbolic_radial_derivatives(x):
    r, R, psi = _symbolic_kernel()
    expr = psi
    got = oracle.prefactors_poly(x * RC, RC, 8)
    for k in range(9):
        want = float(expr.subs({r: x * RC, R: RC}))
        assert got[k] == pytest.approx(want, rel=1e-11), k
        expr = sp.diff(expr, r) / r


def test_c_derivative_tensor_is_the_symbolic_cartesian_derivative():
    X, Y, Z = sp.symbols("X Y Z", real=True)
    s2 = X ** 2 + Y ** 2 + Z ** 2
    psi = 1 / sp.sqrt(s2) - (15 - 10 * s2 / RC ** 2 + 3 * s2 ** 2 / RC ** 4) / (8 * RC)
    Rv = np.array([0.031, -0.047, 0.069])  # |R| < R_c
    p = 5
    D = oracle.deriv_tensor(Rv, 0.0, p, split="poly", rc=RC)
    mi = oracle.multi_indices(p)
    sub = {X: Rv[0], Y: Rv[1], Z: Rv[2]}
    for c, (a, b, g) in enumerate(mi):
        e = psi
        if a:
            e = sp.diff(e, X, int(a))
        if b:
            e = sp.diff(e, Y, int(b))
        if g:
            e = sp.diff(e, Z, int(g))
        want = float(e.subs(sub))
        assert D[c] == pytest.approx(want, rel=1e-9, abs=1e-9 * abs(D).max()), (a, b, g)


def test_c_direct_sum_matches_the_numpy_pair_sum():
    rng = np.random.default_rng(6)
    pos = rng.random((3, 400))
    mass = rng.random(400) / 400
    ref = PS.direct_sr(pos, mass, 1.0, RC)
    got = oracle.direct_sr(pos, mass, 1.0, 0.0, RC, split="poly")
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_fmm_with_the_polynomial_split_converges_to_its_direct_sum():
    from paper_2006_14952_gb300 import workloads as W

    pos, mass = W.nfw_clustered(6000, 10, 0.7, 8)
    rc = 0.12
    direct = PS.direct_sr(pos, mass, 1.0, rc)
    f0 = oracle.FMM(box=1.0, rs=rc / 4.5, rc=rc, theta=0.0, order=2, leaf_max=16, split="poly")
    f0.build_tree(pos, mass)
    np.testing.assert_allclose(f0.forces(), direct, rtol=1e-12, atol=1e-12 * np.abs(direct).max())
    errs = []
    for p in (2, 4, 6):
        f = oracle.FMM(box=1.0, rs=rc / 4.5, rc=rc, theta=0.5, order=p, leaf_max=16, split="poly")
        f.build_tree(pos, mass)
        a = f.forces()
        assert f.size("m2l") > 0
        errs.append(np.linalg.norm(a - direct) / np.linalg.norm(direct))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 0.1 * errs[0], errs


def test_mesh_with_a_given_green_function_reproduces_the_gaussian_mesh():
    rng = np.random.default_rng(7)
    pos = rng.random((3, 500))
    mass = rng.random(500)
    rs = 1.25 / 16
    a0 = PM.pm_long_range(pos, mass, 1.0, 16, rs)
    a1 = PM.pm_long_range(pos, mass, 1.0, 16, rs, green_k2=lambda k2: 4 * np.pi * np.exp(-k2 * rs ** 2) / k2)
    np.testing.assert_allclose(a1, a0, rtol=1e-12, atol=1e-12 * np.abs(a0).max())
