"""Pins of reading R1' (quintic p1 that matches the three cell averages and all three derivative
averages of the big stencil; an alternative to R1's quartic for the reconstruction the paper
omits in Section 2.4).

Fixed by mathematics: six conditions determine a quintic uniquely, so quintics are reproduced
exactly (and R1's quartic is not); for data of a quartic both readings agree; the smoothness
indicator of xi^5 has a closed form; the scheme keeps its order on smooth problems."""
import math

import numpy as np
import pytest
import sympy as sp

from oracle import oracle as O
from paper_2304_09724_gb300 import workloads as WL

H = sp.Rational(1, 2)


def poly_data(coef):
    xi = sp.Symbol("xi")
    P = sum(sp.Rational(c) * xi ** k for k, c in enumerate(coef))
    Wb = [sp.integrate(P, (xi, l - H, l + H)) for l in (-1, 0, 1)]
    v = [P.subs(xi, l + H) - P.subs(xi, l - H) for l in (-1, 0, 1)]
    return P, xi, [float(a) for a in Wb], [float(a) for a in v]


@pytest.mark.parametrize("seed", range(5))
def test_quintic_reproduced_exactly(seed):
    rng = np.random.default_rng(100 + seed)
    coef = [sp.Rational(int(c), 9) for c in rng.integers(-20, 21, size=6)]
    P, xi, Wb, v = poly_data(coef)
    c = O.big_poly_deg(Wb, v, quintic=True)
    np.testing.assert_allclose(c, [float(a) for a in coef], rtol=0, atol=1e-12)
    for x0 in (0.5, -0.5):
        d = O.recon_deg(Wb, v, x0, quintic=True, linear=True)
        exact = [float(sp.diff(P, xi, k).subs(xi, x0)) for k in range(5)]
        np.testing.assert_allclose(d, exact, rtol=0, atol=1e-11)
    # the quartic reading cannot reproduce a genuine quintic
    d4 = O.recon_deg(Wb, v, 0.5, quintic=False, linear=True)
    exact = [float(sp.diff(P, xi, k).subs(xi, H)) for k in range(5)]
    assert np.max(np.abs(d4 - exact)) > 1e-3


def test_readings_agree_on_quartic_data():
    coef = [sp.Rational(3, 7), -1, sp.Rational(2, 5), sp.Rational(-4, 3), sp.Rational(5, 2), 0]
    P, xi, Wb, v = poly_data(coef)
    for x0 in (0.5, -0.5):
        a = O.recon_deg(Wb, v, x0, quintic=True, linear=True)
        b = O.recon_deg(Wb, v, x0, quintic=False, linear=True)
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-11)
    np.testing.assert_allclose(O.big_poly_deg(Wb, v, True)[:5], O.big_poly_deg(Wb, v, False)[:5], atol=1e-12)


def test_smoothness_of_xi5():
    xi = sp.Symbol("xi")
    p = xi ** 5
    beta = sum(sp.integrate(sp.diff(p, xi, a) ** 2, (xi, -H, H)) for a in range(1, 6))
    assert O.smoothness_deg([0, 0, 0, 0, 0, 1.0]) == pytest.approx(float(beta), rel=1e-14)


def test_order_quintic_reading():
    errs = {}
    for n in (20, 40, 80):
        wl = WL.euler1d_sine(n)
        P = O.make_problem(1, WL.EULER, n, 1, *wl.domain, bc=wl.bc, quintic=True)
        st, _, _ = O.run(P, wl.state, 2.0, wl.cfl)
        errs[n] = float(np.mean(np.abs(st["W"][0] - wl.exact(2.0)[0])))
    assert math.log2(errs[40] / errs[80]) > 4.5
    # 2D with the linear weights (with the nonlinear weights the quintic's smoothness indicator
    # keeps the weights away from gamma on the vortex at these sizes: the reason R1 is the default)
    errs = {}
    for n in (20, 40):
        wl = WL.vortex(n)
        P = O.make_problem(2, WL.EULER, n, n, *wl.domain, bc=wl.bc, quintic=True, linear=True)
        st, _, _ = O.run(P, wl.state, 0.25, wl.cfl)
        errs[n] = float(np.mean(np.abs(st["W"][0] - wl.exact(0.25)[0])))
    assert math.log2(errs[20] / errs[40]) > 4.5
