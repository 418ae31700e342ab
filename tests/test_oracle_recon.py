"""Pins of the oracle's SHWENO reconstruction (Section 2.4 reading; Section 3.2).

Each check is fixed by mathematics, not by the oracle itself: exact reproduction of quartics
(the five conditions determine p1 uniquely), closed-form smoothness indicators, the weights'
limits, and mirror symmetry.
"""
import numpy as np
import pytest
import sympy as sp

from oracle import oracle as O

GAM = (0.994, 0.003, 0.003)


def quartic_data(coef):
    """Exact cell averages over cells -1, 0, +1 and derivative averages over cells -1, +1 of the
    polynomial sum coef[k] xi^k (cells of unit width centred on -1, 0, 1)."""
    xi = sp.Symbol("xi")
    P = sum(sp.Rational(c) * xi ** k for k, c in enumerate(coef))
    Wb = [sp.integrate(P, (xi, l - sp.Rational(1, 2), l + sp.Rational(1, 2))) for l in (-1, 0, 1)]
    v = [P.subs(xi, l + sp.Rational(1, 2)) - P.subs(xi, l - sp.Rational(1, 2)) for l in (-1, 1)]
    return P, xi, [float(a) for a in Wb], [float(a) for a in v]


@pytest.mark.parametrize("seed", range(6))
def test_big_poly_reproduces_quartics(seed):
    rng = np.random.default_rng(seed)
    coef = [sp.Rational(int(c), 7) for c in rng.integers(-20, 21, size=5)]
    P, xi, Wb, v = quartic_data(coef)
    c = O.big_poly(Wb, v)
    np.testing.assert_allclose(c, [float(a) for a in coef], rtol=0, atol=1e-12)
    # linear weights: the SHWENO polynomial is p1, so every derivative at both ends is exact
    for x0 in (0.5, -0.5, 0.3):
        d = O.recon(Wb, v, x0, linear=True)
        exact = [float(sp.diff(P, xi, k).subs(xi, sp.nsimplify(x0))) for k in range(5)]
        np.testing.assert_allclose(d, exact, rtol=0, atol=1e-11)


def test_big_poly_rational_table_matches_sympy_solution():
    """Solve the five conditions symbolically and compare the derivative rows at xi = +1/2."""
    xi = sp.Symbol("xi")
    c = sp.symbols("c0:5")
    Wm, W0, Wp, vm, vp = sp.symbols("Wm W0 Wp vm vp")
    P = sum(c[k] * xi ** k for k in range(5))
    half = sp.Rational(1, 2)
    eqs = [sp.integrate(P, (xi, l - half, l + half)) - w for l, w in ((-1, Wm), (0, W0), (1, Wp))]
    eqs += [P.subs(xi, l + half) - P.subs(xi, l - half) - w for l, w in ((-1, vm), (1, vp))]
    sol = sp.solve(eqs, c)
    Ps = P.subs(sol)
    rng = np.random.default_rng(7)
    for _ in range(4):
        vals = rng.normal(size=5)
        sub = dict(zip((Wm, W0, Wp, vm, vp), vals))
        d = O.recon(vals[:3], vals[3:], 0.5, linear=True)
        exact = [float(sp.diff(Ps, xi, k).subs(xi, half).subs(sub)) for k in range(5)]
        np.testing.assert_allclose(d, exact, rtol=1e-12, atol=1e-12)


def test_smoothness_closed_forms():
    # beta of a + b xi is b^2; of xi^2 it is int (2 xi)^2 + int 2^2 = 1/3 + 4
    assert O.smoothness([3.0, -2.0, 0, 0, 0]) == pytest.approx(4.0, abs=1e-14)
    assert O.smoothness([0, 0, 1.0, 0, 0]) == pytest.approx(1.0 / 3.0 + 4.0, abs=1e-13)
    # random quartic against sympy's integral
    xi = sp.Symbol("xi")
    rng = np.random.default_rng(3)
    c = rng.normal(size=5)
    P = sum(float(c[k]) * xi ** k for k in range(5))
    beta = sum(sp.integrate(sp.diff(P, xi, a) ** 2, (xi, -0.5, 0.5)) for a in range(1, 5))
    assert O.smoothness(c) == pytest.approx(float(beta), rel=1e-12)


def test_weights_linear_data_give_linear_weights():
    # for data of a linear function all three polynomials coincide, so beta1 = beta2 = beta3,
    # tau = 0 and the nonlinear weights equal the linear ones
    Wb = [0.3 - 0.7, 0.3, 0.3 + 0.7]
    v = [0.7, 0.7]
    np.testing.assert_allclose(O.weights(Wb, v), GAM, rtol=0, atol=1e-15)


def test_weights_tend_to_linear_for_smooth_data():
    devs = []
    for h in (0.2, 0.1, 0.05, 0.025):
        xs = np.array([-1, 0, 1]) * h
        f = lambda x: np.exp(x)  # antiderivative of exp; averages and derivative averages exact
        Wb = [(f(x + h / 2) - f(x - h / 2)) / h for x in xs]
        v = [f(xs[0] + h / 2) - f(xs[0] - h / 2), f(xs[2] + h / 2) - f(xs[2] - h / 2)]
        devs.append(np.max(np.abs(O.weights(Wb, v) - GAM) / GAM))
    assert devs[-1] < 1e-3
    assert all(b < a for a, b in zip(devs, devs[1:]))


def test_weights_step_data_suppress_big_stencil():
    w = O.weights([0.0, 0.0, 1.0], [0.0, 0.0])
    assert w[0] < 1e-3 * GAM[0]
    # the smooth small stencil {I_{j-1}, I_j} takes over
    assert w[1] > 0.9


@pytest.mark.parametrize("seed", range(4))
def test_nonlinear_recon_exact_for_linear_data(seed):
    rng = np.random.default_rng(100 + seed)
    a, b = rng.normal(size=2)
    Wb = [a - b, a, a + b]
    v = [b, b]
    for x0 in (0.5, -0.5):
        d = O.recon(Wb, v, x0)
        np.testing.assert_allclose(d, [a + b * x0, b, 0, 0, 0], atol=1e-13)


@pytest.mark.parametrize("linear", [True, False])
def test_mirror_symmetry(linear):
    """Reflecting the data (cells swap, derivative averages change sign) reflects the result."""
    rng = np.random.default_rng(11)
    for _ in range(5):
        Wb = rng.normal(size=3)
        v = rng.normal(size=2)
        d = O.recon(Wb, v, 0.5, linear=linear)
        dm = O.recon(Wb[::-1], -v[::-1], -0.5, linear=linear)
        np.testing.assert_allclose(dm, d * np.array([1, -1, 1, -1, 1]), rtol=1e-12, atol=1e-12)


def test_weights_sum_to_one_and_positive():
    rng = np.random.default_rng(5)
    for _ in range(50):
        w = O.weights(rng.normal(size=3) * 10, rng.normal(size=2) * 10)
        assert abs(w.sum() - 1.0) < 1e-14
        assert (w > 0).all()


def test_quadrature_rules_exact():
    lam, lw, gs, gw = O.quadrature()
    for k in range(6):  # 4-node Lobatto on [0,1] and 3-node Gauss on [-1/2,1/2] are exact to degree 5
        assert np.dot(lw, lam ** k) == pytest.approx(1.0 / (k + 1), abs=1e-15)
        exact = 0.0 if k % 2 else 2 * 0.5 ** (k + 1) / (k + 1)
        assert np.dot(gw, gs ** k) == pytest.approx(exact, abs=1e-15)
    assert lam[0] == 0.0 and lam[-1] == 1.0  # the rule holds both ends (Remark 2)
    # degree 6 is not integrated exactly by the 3-node Gauss rule (so the rule is not larger)
    assert abs(np.dot(gw, gs ** 6) - 2 * 0.5 ** 7 / 7) > 1e-6
