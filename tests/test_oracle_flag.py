"""Pins of the oracle side of the learned troubled-cell flag (not in the paper): the FP64 MLP
against finite differences and the Adam formula, the feature and label definitions against
hand-computed cases."""
import math

import numpy as np
import pytest

from oracle import mlp_oracle as M
from oracle import oracle as O
from paper_2304_09724_gb300 import workloads as WL


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    theta = M.init(3)
    X = rng.normal(size=(40, M.NIN))
    y = (rng.random(40) < 0.3).astype(float)
    g = M.grad(theta, X, y, 2.5)
    idx = rng.choice(M.NPARAMS, size=60, replace=False)
    h = 1e-6
    for k in idx:
        e = np.zeros(M.NPARAMS)
        e[k] = h
        fd = (M.loss(theta + e, X, y, 2.5) - M.loss(theta - e, X, y, 2.5)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1e-3, abs(g[k])) + 1e-9, (k, fd, g[k])


def test_mlp_shapes_and_loss_limits():
    assert M.NPARAMS == 1825
    theta = np.zeros(M.NPARAMS)
    X = np.zeros((5, M.NIN))
    # zero network: sigmoid(0) = 1/2, loss = mean(pw y + (1-y)) log 2
    y = np.array([1, 0, 0, 1, 0.0])
    assert M.loss(theta, X, y, 3.0) == pytest.approx(np.mean(3.0 * y + (1 - y)) * math.log(2), rel=1e-14)


def test_adam_first_step_is_sign_step():
    theta = np.zeros(4)
    g = np.array([1.0, -2.0, 3e-3, 0.0])
    t1, m, v = M.adam(theta, g, np.zeros(4), np.zeros(4), 1, 0.01)
    # bias-corrected first step: m/(1-b1) = g, v/(1-b2) = g^2 -> update lr * g / (|g| + eps)
    np.testing.assert_allclose(t1, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_features_hand_case():
    """A cell left of a vertical density jump: known normalised differences."""
    n = 8
    W = np.zeros((4, n, n))
    W[0] = 1.0
    W[0][:, 5:] = 3.0  # jump between columns 4 and 5
    W[3] = 2.5
    st = {"W": W, "V": np.zeros_like(W), "Y": np.zeros_like(W), "Z": np.zeros_like(W)}
    P = O.make_problem(2, 1, n, n, 0.0, 1.0, 0.0, 1.0, bc=(1, 1, 1, 1))
    f = O.features2d(P, st).reshape(n, n, 22)
    c = f[3, 4]  # cell (i=4, j=3): right neighbours are 3.0, others 1.0
    s = 2.0 + 1e-12 * 1.0 + 1e-300
    expect = np.array([0, 0, 2, 0, 2, 0, 0, 2]) / s
    np.testing.assert_allclose(c[:8], expect, rtol=1e-14)
    assert c[8] == 0 and c[9] == 0
    assert c[10] == pytest.approx(math.log10(2.0 / 1.0 + 1e-16) / 8, rel=1e-14)
    # E is constant: zero differences, range 0 -> log10(1e-16)/8 = -2
    np.testing.assert_allclose(c[11:19], 0.0)
    assert c[21] == pytest.approx(-2.0)


def test_weight_deviation_cases():
    P = O.make_problem(2, 1, 10, 10, bc=(0, 0, 0, 0))
    const = WL.constant_state(2, 1, 10, 10)
    assert O.weight_deviation2d(P, const).max() == 0.0
    # four-quadrant data: large deviations at the jumps, none in the constant corners
    wl = WL.riemann2d(10, WL.LAX_LIU_SHOCKS)
    Pj = O.make_problem(2, 1, 10, 10, *wl.domain, bc=wl.bc)
    d = O.weight_deviation2d(Pj, wl.state)
    assert d.max() > 1.0  # cells at the quadrant jumps
    assert d[0, 0] == 0.0 and d[9, 9] == 0.0  # corners far from the jumps are constant


def test_face_deviation_hand_case_and_limits():
    """Label source of the face-value form, evaluated by hand.  Step data W = (0, 0, 1), v = (0, 0):
    p1's end values are 67/120 (xi = +1/2) and -23/120 (xi = -1/2) (rows of the quartic's end
    values), p2 = 0 and p3 = xi, and with the weights w (evaluated in exact rationals in
    test_oracle_recon) p = A p1 + B p2 + C p3, A = w1/g1, B = w2 - A g2, C = w3 - A g3, so
    p - p1 = (A - 1) p1 + C xi at the ends; the range of the averages is 1."""
    import sympy as sp

    from tests.test_oracle_recon import HAND_CASES, GAM_Q, _exact_weights

    w = _exact_weights(HAND_CASES[0]["beta"])
    A = w[0] / GAM_Q[0]
    C = w[2] - A * GAM_Q[2]
    half = sp.Rational(1, 2)
    right = (A - 1) * sp.Rational(67, 120) + C * half
    left = (A - 1) * sp.Rational(-23, 120) - C * half
    expect = float(max(abs(right), abs(left)))
    assert O.face_deviation([0.0, 0.0, 1.0], [0.0, 0.0]) == pytest.approx(expect, rel=1e-12)
    # data of a linear function: all three polynomials coincide, whatever the weights
    assert O.face_deviation([0.3 - 0.7, 0.3, 0.3 + 0.7], [0.7, 0.7]) < 1e-15
    # a smooth quadratic barely moves the end values (the weights are close to linear and
    # p2, p3 differ from p1 by O(h^2)), a step moves them by a large fraction of the range
    assert O.face_deviation([0.0, 0.1, 0.3], [0.05, 0.25]) < 1e-3 * O.face_deviation([0.0, 0.0, 1.0], [0.0, 0.0])
    # the floor of the scale: |p - p1| is the same, the scale grows by (floor - 1e-9) |W0|
    Wb, v = [1.0, 1.0, 2.0], [0.0, 0.0]
    d9, d3 = O.face_deviation(Wb, v), O.face_deviation(Wb, v, floor_rel=1e-3)
    assert d3 == pytest.approx(d9 * (1.0 + 1e-9) / (1.0 + 1e-3), rel=1e-12)


def test_face_deviation2d_cases():
    """Constant data move no end value (up to rounding, which the 1e-9 |W0| floor of the scale
    keeps near 1e-7); four-quadrant data move them at the jumps only."""
    P = O.make_problem(2, 1, 10, 10, bc=(0, 0, 0, 0))
    assert O.face_deviation2d(P, WL.constant_state(2, 1, 10, 10)).max() < 1e-6
    wl = WL.riemann2d(10, WL.LAX_LIU_SHOCKS)
    Pj = O.make_problem(2, 1, 10, 10, *wl.domain, bc=wl.bc)
    d = O.face_deviation2d(Pj, wl.state)
    assert d.max() > 0.1 and d[0, 0] < 1e-6 and d[9, 9] < 1e-6
    # the face-value label is the weight label's companion: at rounding level where the weights
    # do not move
    dw = O.weight_deviation2d(Pj, wl.state)
    assert np.all(d[dw == 0.0] < 1e-6)
