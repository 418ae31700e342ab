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


# ---------------------------------------------------------------- weights evaluated by hand
# Two data sets whose big-stencil quartic, smoothness indicators and weights are worked out in
# exact rationals below, independently of the oracle (which solves the 5x5 system numerically and
# integrates the squared derivatives monomial by monomial).  Reading R1 of Section 2.4 (the
# simple-WENO form): tau = ((|b1 - b2| + |b1 - b3|)/2)^2, w~_l = gamma_l (1 + tau/(b_l + eps)),
# w_l = w~_l / sum w~, eps = 1e-6, gamma = (0.994, 0.003, 0.003).
HALF = sp.Rational(1, 2)
GAM_Q = (sp.Rational(994, 1000), sp.Rational(3, 1000), sp.Rational(3, 1000))
EPS_Q = sp.Rational(1, 10 ** 6)
XI = sp.Symbol("xi")
HAND_CASES = [
    # step data: W = (0, 0, 1), v = (0, 0).
    #   p1 = -xi^4/2 - xi^3/4 + 5 xi^2/4 + 13 xi/16 - 47/480, beta1 = 219889/1344,
    #   p2 = 0 (beta2 = 0), p3 = xi (beta3 = 1), tau = (beta1 - 1/2)^2 since beta1 > 1
    dict(W=(0, 0, 1), v=(0, 0),
         p1=-XI ** 4 / 2 - XI ** 3 / 4 + sp.Rational(5, 4) * XI ** 2 + sp.Rational(13, 16) * XI
         - sp.Rational(47, 480),
         beta=(sp.Rational(219889, 1344), 0, 1)),
    # averages and derivative averages of the quadratic p = xi^2/20 + 3 xi/20 + 23/240:
    #   W = (0, 1/10, 3/10), v = (1/20, 1/4); p1 = p, beta1 = (3/20)^2 + (1/10)^2/12 + (1/10)^2
    #   = 1/30, beta2 = (1/10)^2, beta3 = (1/5)^2, tau = ((7/300 + 2/300)/2)^2 = (3/200)^2
    dict(W=(0, sp.Rational(1, 10), sp.Rational(3, 10)), v=(sp.Rational(1, 20), sp.Rational(1, 4)),
         p1=XI ** 2 / 20 + sp.Rational(3, 20) * XI + sp.Rational(23, 240),
         beta=(sp.Rational(1, 30), sp.Rational(1, 100), sp.Rational(1, 25))),
]


def _exact_weights(beta, tau_of=lambda b: ((abs(b[0] - b[1]) + abs(b[0] - b[2])) / 2) ** 2,
                   shape=lambda g, t, b: g * (1 + t / (b + EPS_Q))):
    tau = tau_of(beta)
    wt = [shape(g, tau, b) for g, b in zip(GAM_Q, beta)]
    s = sum(wt)
    return [w / s for w in wt]


@pytest.mark.parametrize("case", range(len(HAND_CASES)))
def test_weights_hand_evaluated(case):
    c = HAND_CASES[case]
    xi = XI
    p1 = c["p1"]
    # the quartic satisfies the five conditions of reading R1 (cell averages over cells -1, 0, +1
    # and derivative averages over cells -1, +1), which fix it uniquely
    for l, w in zip((-1, 0, 1), c["W"]):
        assert sp.integrate(p1, (xi, l - HALF, l + HALF)) == w
    for l, w in zip((-1, 1), c["v"]):
        assert p1.subs(xi, l + HALF) - p1.subs(xi, l - HALF) == w
    # smoothness indicators: the stated closed forms equal the integrals of the squared derivatives
    b1 = sum(sp.integrate(sp.diff(p1, xi, a) ** 2, (xi, -HALF, HALF)) for a in range(1, 5))
    assert b1 == c["beta"][0]
    W = c["W"]
    assert (W[1] - W[0]) ** 2 == c["beta"][1] and (W[2] - W[1]) ** 2 == c["beta"][2]
    Wf, vf = [float(a) for a in W], [float(a) for a in c["v"]]
    assert O.smoothness(O.big_poly(Wf, vf)) == pytest.approx(float(b1), rel=1e-13)
    expect = [float(w) for w in _exact_weights(c["beta"])]
    got = O.weights(Wf, vf)
    np.testing.assert_allclose(got, expect, rtol=1e-12, atol=1e-15)
    # the case tells the formula apart from its plausible slips: tau left unsquared, the 1/2
    # dropped, or the bracket squared all move some weight by far more than the tolerance
    slips = [
        _exact_weights(c["beta"], tau_of=lambda b: (abs(b[0] - b[1]) + abs(b[0] - b[2])) / 2),
        _exact_weights(c["beta"], tau_of=lambda b: (abs(b[0] - b[1]) + abs(b[0] - b[2])) ** 2),
        _exact_weights(c["beta"], shape=lambda g, t, b: g * (1 + t / (b + EPS_Q)) ** 2),
    ]
    for s in slips:
        rel = max(abs(float(a) - e) / e for a, e in zip(s, expect))
        assert rel > 1e-6
