"""Pins of the oracle's Cauchy-Kovalevskaya (Lax-Wendroff) procedure, Eq. (2.6) and Section 3.1.

The oracle gets the spatial derivatives of an exact smooth solution at a point and must return
that solution's mixed space-time derivatives.  The exact solutions come from the method of
characteristics (an implicit equation solved as a truncated power series by fixed-point
iteration), or from the closed form of the translating isentropic vortex of Example 5.8 --
neither uses the PDE recursion the oracle uses:
  * Burgers: u = u0(x - u t);
  * 1D Euler isentropic simple wave: u - 2c/(g-1) = J constant, u + c = lam(x, t) with
    lam = lam0(x - lam t); rho = (c^2/(g K))^{1/(g-1)} = const * c^5 for g = 7/5;
  * the same simple wave along an oblique direction in 2D with a constant tangential velocity;
  * the isentropic vortex moving with velocity (1, 1).
"""
import math

import numpy as np
import pytest
import sympy as sp

from oracle import oracle as O

X, Y, T = sp.symbols("X Y T")
ORDER = 4


def trunc(e, vars_=(X, T)):
    e = sp.expand(e)
    if e == 0:
        return sp.Integer(0)
    P = sp.Poly(e, *vars_)
    return sum(c * sp.prod([v ** k for v, k in zip(vars_, mon)])
               for mon, c in zip(P.monoms(), P.coeffs()) if sum(mon) <= ORDER)


def characteristic_series(f0, x0):
    """Truncated series in (X, T) of the solution lam of lam = f0(x0 + X - lam T)."""
    s = sp.Symbol("s")
    derivs = [float(sp.diff(f0(s), s, j).subs(s, x0)) for j in range(ORDER + 1)]
    lam = sp.Float(derivs[0])
    for _ in range(ORDER + 2):
        d = X - lam * T
        lam = trunc(sum(derivs[j] * d ** j / math.factorial(j) for j in range(ORDER + 1)))
    return lam


def coeff(e, m, k, n=0, vars_=(X, T)):
    P = sp.Poly(sp.expand(e), *vars_) if e != 0 else None
    if P is None:
        return 0.0
    mon = (m, k) if len(vars_) == 2 else (m, n, k)
    return float(P.as_dict().get(mon, 0.0))


def check_ck(P, nc, series, vars_):
    """series[q]: truncated series of W_q in vars_ ((X,T) in 1D, (X,Y,T) in 2D)."""
    d = np.zeros((nc, 5, 5))
    two_d = len(vars_) == 3
    for q in range(nc):
        for m in range(5):
            for n in range(5 - m if two_d else 1):
                d[q, m, n] = coeff(series[q], m, 0, n, vars_) * math.factorial(m) * math.factorial(n)
    out = O.ck(P, d)
    checked = 0
    for q in range(nc):
        for m in range(5):
            for n in range(5 - m if two_d else 1):
                for k in range(5 - m - n):
                    exact = coeff(series[q], m, k, n, vars_) * math.factorial(m) * math.factorial(n) * math.factorial(k)
                    scale = max(1.0, abs(exact))
                    assert abs(out[q, m, n, k] - exact) <= 1e-10 * scale, (q, m, n, k, out[q, m, n, k], exact)
                    checked += 1
    return checked


@pytest.mark.parametrize("x0", [0.3, 1.1])
def test_ck_burgers_characteristics(x0):
    u = characteristic_series(lambda s: 0.5 + sp.sin(sp.pi * s), x0)
    P = O.make_problem(1, O.EQ_BURGERS, 8)
    assert check_ck(P, 1, [u], (X, T)) == 15


def simple_wave_1d(x0, g=sp.Rational(7, 5), J=-3.0, K=0.8):
    """Series of (rho, m, E, u, p) of the isentropic simple wave around (x0, 0)."""
    lam = characteristic_series(lambda s: 1.6 + 0.3 * sp.sin(2 * s) + 0.1 * sp.cos(5 * s), x0)
    c = (lam - J) * (g - 1) / (g + 1)
    u = lam - c
    # c^2 = g K rho^(g-1)  ->  rho = (c^2/(g K))^(5/2) = c^5 / (g K)^(5/2) for g = 7/5
    rho = trunc(c ** 5) / float((g * K) ** sp.Rational(5, 2))
    p = trunc(rho * c ** 2 / g)  # p = K rho^g = rho c^2 / g
    m = trunc(rho * u)
    E = trunc(p / (g - 1) + rho * u * u / 2)
    return rho, m, E, u, p


@pytest.mark.parametrize("x0", [0.2, 2.0])
def test_ck_euler1d_simple_wave(x0):
    rho, m, E, _, _ = simple_wave_1d(x0)
    P = O.make_problem(1, O.EQ_EULER, 8)
    assert check_ck(P, 3, [rho, m, E], (X, T)) == 45


@pytest.mark.parametrize("theta", [0.4, 2.2])
def test_ck_euler2d_oblique_simple_wave(theta):
    """The 1D simple wave along the direction (cos th, sin th) with a constant tangential
    velocity: every conserved component is a function of X cos th + Y sin th and T."""
    rho, _, _, un, p = simple_wave_1d(0.7)
    g = sp.Rational(7, 5)
    ut = 0.35
    ct, st = math.cos(theta), math.sin(theta)
    u = un * ct - ut * st
    v = un * st + ut * ct
    mx = trunc(rho * u)
    my = trunc(rho * v)
    E = trunc(p / (g - 1) + trunc(rho * (u * u + v * v)) / 2)
    to2d = lambda e: trunc(sp.expand(e.subs(X, X * ct + Y * st)), (X, Y, T))
    series = [to2d(w) for w in (rho, mx, my, E)]
    P = O.make_problem(2, O.EQ_EULER, 8, 8)
    assert check_ck(P, 4, series, (X, Y, T)) == 4 * 35


def series_pow(e, a, vars_):
    """(e)^a as a truncated series: binomial expansion around the constant term."""
    e = sp.expand(e)
    c0 = float(sp.Poly(e, *vars_).as_dict().get((0,) * len(vars_), 0.0))
    d = trunc(e - c0, vars_)
    out, term = sp.Integer(0), sp.Integer(1)
    for j in range(ORDER + 1):
        out += float(sp.binomial(a, j)) * c0 ** (a - j) * term
        term = trunc(term * d, vars_)
    return trunc(out, vars_)


def series_exp(e, vars_):
    e = sp.expand(e)
    c0 = float(sp.Poly(e, *vars_).as_dict().get((0,) * len(vars_), 0.0))
    d = trunc(e - c0, vars_)
    out, term = sp.Integer(0), sp.Integer(1)
    for j in range(ORDER + 1):
        out += math.exp(c0) / math.factorial(j) * term
        term = trunc(term * d, vars_)
    return trunc(out, vars_)


def test_ck_isentropic_vortex():
    """Exact vortex of Example 5.8 (strength 5, velocity (1,1)) around (5.6, 4.3, 0): the
    closed form expanded by exp and binomial series; all 35 mixed derivatives per component."""
    V = (X, Y, T)
    g = 1.4
    xr, yr = 0.6 + X - T, -0.7 + Y - T
    e = series_exp((1 - xr ** 2 - yr ** 2) / 2, V)
    base = 1 - (g - 1) * 25 / (8 * g * math.pi ** 2) * trunc(e * e, V)
    rho = series_pow(base, 1 / (g - 1), V)
    p = series_pow(base, g / (g - 1), V)  # p = rho^g
    u = trunc(1 - 5 / (2 * math.pi) * e * yr, V)
    v = trunc(1 + 5 / (2 * math.pi) * e * xr, V)
    W = [rho, trunc(rho * u, V), trunc(rho * v, V),
         trunc(p / (g - 1) + trunc(rho * trunc(u * u + v * v, V), V) / 2, V)]
    P = O.make_problem(2, O.EQ_EULER, 8, 8)
    assert check_ck(P, 4, W, V) == 4 * 35


def test_ck_translation_of_density_wave():
    """u, v, p constant: rho is advected, so d^k rho/dt^k = (-u d/dx - v d/dy)^k rho."""
    P = O.make_problem(2, O.EQ_EULER, 8, 8)
    rng = np.random.default_rng(9)
    dr = rng.normal(size=(5, 5)) * 0.1
    u, v, p, g = 0.7, -0.4, 1.3, 1.4
    d = np.zeros((4, 5, 5))
    for m in range(5):
        for n in range(5 - m):
            d[0, m, n] = dr[m, n] + (1.2 if m == n == 0 else 0.0)
            d[1, m, n] = u * d[0, m, n]
            d[2, m, n] = v * d[0, m, n]
            d[3, m, n] = 0.5 * (u * u + v * v) * d[0, m, n] + (p / (g - 1) if m == n == 0 else 0.0)
    out = O.ck(P, d)
    for k in range(1, 5):
        exact = sum(math.comb(k, a) * (-u) ** a * (-v) ** (k - a) * d[0, a, k - a] for a in range(k + 1))
        assert out[0, 0, 0, k] == pytest.approx(exact, rel=1e-11, abs=1e-12)
