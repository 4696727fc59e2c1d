"""Pins for the oracle's split-kernel prefactors f_(k) and derivative tensors D_n.

Each check ties the oracle to something other than its own formula: the
prefactors printed in Sec. 2.2 for k = 1..4, symbolic differentiation of the
potential of Sec. 2.2 (sympy), the Newtonian prefactors of Eq. pref as the
r_s -> infinity limit, the Laplacian of the truncated potential, and finite
differences.
"""
import math

import numpy as np
import pytest
import sympy as sp

import oracle

SQPI = math.sqrt(math.pi)


def printed_f(k, r, rs):
    """f_(1..4) exactly as printed in Sec. 2.2 (force law and the f_(2)..f_(4) display)."""
    e = math.exp(-r * r / (4 * rs * rs)) / SQPI
    ec = math.erfc(r / (2 * rs))
    if k == 0:
        return ec / r
    if k == 1:
        return -(1 / r ** 3) * (ec + r / (rs * SQPI) * math.exp(-r * r / (4 * rs * rs)))
    if k == 2:
        return 3 / r ** 5 * ec + e * (3 / (rs * r ** 4) + 1 / (2 * rs ** 3 * r ** 2))
    if k == 3:
        return -15 / r ** 7 * ec - e * (15 / (rs * r ** 6) + 5 / (2 * rs ** 3 * r ** 4) + 1 / (4 * rs ** 5 * r ** 2))
    if k == 4:
        return 105 / r ** 9 * ec + e * (105 / (rs * r ** 8) + 35 / (2 * rs ** 3 * r ** 6) + 7 / (4 * rs ** 5 * r ** 4)
                                        + 1 / (8 * rs ** 7 * r ** 2))
    raise ValueError


@pytest.mark.parametrize("r,rs", [(0.05, 0.04), (0.3, 0.1), (1.7, 1.0), (4.4, 1.0), (0.01, 0.0390625)])
def test_closed_form_matches_printed_f1_to_f4(r, rs):
    f = oracle.prefactors(r, rs, 4)
    for k in range(5):
        ref = printed_f(k, r, rs)
        assert f[k] == pytest.approx(ref, rel=1e-12), k


def _sympy_radial(kmax):
    r, rs = sp.symbols("r r_s", positive=True)
    g = sp.erfc(r / (2 * rs)) / r
    out = [g]
    for _ in range(kmax):
        g = sp.diff(g, r) / r
        out.append(g)
    return r, rs, out


def test_prefactors_equal_symbolic_radial_derivatives_up_to_order_8():
    r, rs, fs = _sympy_radial(8)
    for rv, rsv in [(0.07, 0.05), (0.9, 0.4), (2.5, 0.6)]:
        f = oracle.prefactors(rv, rsv, 8)
        for k in range(9):
            ref = float(fs[k].subs({r: rv, rs: rsv}).evalf(30))
            assert f[k] == pytest.approx(ref, rel=1e-11), k


def test_corrected_recurrence_and_printed_recurrence_is_garbled():
    """f_(p+1) = (1/r) d f_(p)/dr gives
    r^2 f_(p+1) = -(2p+1) f_(p) + (-1)^(p+1) e^(-x^2/4) / (2^p sqrt(pi) rs^(2p+1)).
    The recurrence as printed in Sec. 2.2 does not hold (checked at x = 1.7)."""
    rs = 1.0
    for r in (0.3, 1.7, 3.9):
        f = oracle.prefactors(r, rs, 7)
        x = r / rs
        for p in range(6):
            rhs = -(2 * p + 1) * f[p] + (-1) ** (p + 1) * math.exp(-x * x / 4) / (2 ** p * SQPI * rs ** (2 * p + 1))
            assert r * r * f[p + 1] == pytest.approx(rhs, rel=1e-11)
    f = oracle.prefactors(1.7, 1.0, 3)
    x = 1.7
    p = 2
    printed = ((2 * p - 1) * f[p] + math.exp(-x * x / 4) / (2 ** (p - 1) * SQPI)) / (-(x * x))
    assert abs(printed - f[p + 1]) > 1e-3 * abs(f[p + 1])


def test_newtonian_limit_of_prefactors():
    """r_s -> infinity recovers Eq. pref, f~_(n) = (-1)^n (2n-1)!!/r^(2n+1)."""
    r = 0.37
    f = oracle.prefactors(r, 1e7, 6)
    for n in range(7):
        dfact = 1
        for i in range(2 * n - 1, 1, -2):
            dfact *= i
        ref = (-1) ** n * dfact / r ** (2 * n + 1)
        assert f[n] == pytest.approx(ref, rel=1e-6)


def test_split_kernels_sum_to_newton():
    """Short-range erfc part + long-range erf part = Newtonian force law (Sec. 2.2)."""
    rsym, rss = sp.symbols("r r_s", positive=True)
    lr = sp.erf(rsym / (2 * rss)) / rsym
    f1_lr = sp.lambdify((rsym, rss), sp.diff(lr, rsym) / rsym, "math")
    for r, rs in [(0.01, 0.04), (0.2, 0.04), (1.3, 0.5)]:
        f1 = oracle.prefactors(r, rs, 1)[1]
        assert f1 + f1_lr(r, rs) == pytest.approx(-1.0 / r ** 3, rel=1e-12)


@pytest.fixture(scope="module")
def sympy_D():
    x, y, z = sp.symbols("x y z", real=True)
    rs = sp.Rational(3, 10)
    rr = sp.sqrt(x * x + y * y + z * z)
    psi = sp.erfc(rr / (2 * rs)) / rr
    return (x, y, z), rs, psi


def test_deriv_tensor_equals_symbolic_derivatives(sympy_D):
    (x, y, z), rs, psi = sympy_D
    p = 5
    idx = oracle.multi_indices(p)
    for R in ([0.21, -0.13, 0.08], [-0.05, 0.4, -0.33]):
        D = oracle.deriv_tensor(R, float(rs), p)
        sub = {x: R[0], y: R[1], z: R[2]}
        for c, (nx, ny, nz) in enumerate(idx):
            e = psi
            if nx:
                e = sp.diff(e, x, int(nx))
            if ny:
                e = sp.diff(e, y, int(ny))
            if nz:
                e = sp.diff(e, z, int(nz))
            ref = float(e.subs(sub).evalf(25))
            assert D[c] == pytest.approx(ref, rel=1e-10, abs=1e-10 * abs(D[0])), (nx, ny, nz)


def _index_map(p):
    return {tuple(int(v) for v in m): c for c, m in enumerate(oracle.multi_indices(p))}


def test_trace_identity_truncated_and_traceless_newtonian():
    """sum_i D_{n+2e_i} = d^n Lap(psi): Lap psi_SR = e^(-r^2/4rs^2)/(2 sqrt(pi) rs^3) for r > 0,
    and 0 for the Newtonian potential (the traceless case of Sec. 2.1)."""
    p = 6
    im = _index_map(p)
    R = np.array([0.11, 0.07, -0.09])
    rs = 0.06
    D = oracle.deriv_tensor(R, rs, p)
    r2 = R @ R
    lap = math.exp(-r2 / (4 * rs * rs)) / (2 * SQPI * rs ** 3)
    tr0 = D[im[(2, 0, 0)]] + D[im[(0, 2, 0)]] + D[im[(0, 0, 2)]]
    assert tr0 == pytest.approx(lap, rel=1e-11)
    # first derivatives of the Laplacian: d/dx_i of a Gaussian = -x_i/(2 rs^2) * gaussian
    for i, e in enumerate([(1, 0, 0), (0, 1, 0), (0, 0, 1)]):
        tr = sum(D[im[tuple(e[k] + 2 * (k == j) for k in range(3))]] for j in range(3))
        assert tr == pytest.approx(-R[i] / (2 * rs * rs) * lap, rel=1e-10)
    Dn = oracle.deriv_tensor(R, 0.0, p)
    for m, c in im.items():
        if sum(m) + 2 > p:
            continue
        tr = sum(Dn[im[tuple(m[k] + 2 * (k == j) for k in range(3))]] for j in range(3))
        assert abs(tr) < 1e-9 * np.abs(Dn[: len(im)]).max()


def test_deriv_tensor_finite_differences():
    p = 5
    im = _index_map(p)
    R = np.array([0.13, -0.2, 0.05])
    rs = 0.1
    h = 1e-5
    for m, c in im.items():
        if sum(m) >= p:
            continue
        for d in range(3):
            e = np.zeros(3)
            e[d] = h
            fd = (oracle.deriv_tensor(R + e, rs, p)[c] - oracle.deriv_tensor(R - e, rs, p)[c]) / (2 * h)
            up = tuple(m[k] + (k == d) for k in range(3))
            ex = oracle.deriv_tensor(R, rs, p)[im[up]]
            assert fd == pytest.approx(ex, rel=2e-6, abs=1e-8 * abs(ex) + 1e-6), (m, d)
