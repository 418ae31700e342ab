"""Pins of the oracle's Riemann solvers (Eq. 2.5, 3.6), eigensystems and the linearised
derivative Riemann problem (Eq. 2.8, 3.7).

Fixed by: textbook Burgers cases, HLLC consistency / contact / supersonic cases, the integral
consistency of the HLLC fan (sampled through Galilean frame shifts), the flux Jacobian derived
symbolically by sympy, and the limits of the upwinding.
"""
import numpy as np
import pytest
import sympy as sp

from oracle import oracle as O

G = 1.4


def cons(rho, u, p, v=None):
    if v is None:
        return np.array([rho, rho * u, p / (G - 1) + 0.5 * rho * u * u])
    return np.array([rho, rho * u, rho * v, p / (G - 1) + 0.5 * rho * (u * u + v * v)])


def prob(dim, eq=O.EQ_EULER):
    return O.make_problem(dim, eq, 8, 8)


@pytest.mark.parametrize("uL,uR,expect", [
    (2.0, 1.0, 2.0),    # right-moving shock
    (-1.0, -2.0, -2.0),  # left-moving shock
    (1.0, -1.0, 1.0),   # stationary shock takes the left state
    (1.0, 2.0, 1.0),    # right-moving rarefaction
    (-2.0, -1.0, -1.0),  # left-moving rarefaction
    (-1.0, 2.0, 0.0),   # sonic rarefaction: u = 0 at x/t = 0
    (0.7, 0.7, 0.7),
])
def test_burgers_godunov(uL, uR, expect):
    assert O.burgers_godunov(uL, uR) == expect


@pytest.mark.parametrize("dim", [1, 2])
def test_hllc_consistency_and_supersonic(dim):
    P = prob(dim)
    U = cons(1.3, 0.4, 2.0) if dim == 1 else cons(1.3, 0.4, 2.0, -0.7)
    np.testing.assert_allclose(O.hllc(P, 0, U, U), U, rtol=1e-14)
    if dim == 2:
        np.testing.assert_allclose(O.hllc(P, 1, U, U), U, rtol=1e-14)
    # supersonic to the right: the left state is sampled; to the left: the right state
    UL = cons(1.0, 3.0, 0.5) if dim == 1 else cons(1.0, 3.0, 0.5, 0.2)
    UR = cons(0.5, 2.5, 0.4) if dim == 1 else cons(0.5, 2.5, 0.4, -0.1)
    np.testing.assert_allclose(O.hllc(P, 0, UL, UR), UL)
    UL2 = cons(1.0, -3.0, 0.5) if dim == 1 else cons(1.0, -3.0, 0.5, 0.2)
    UR2 = cons(0.5, -2.8, 0.4) if dim == 1 else cons(0.5, -2.8, 0.4, -0.1)
    np.testing.assert_allclose(O.hllc(P, 0, UL2, UR2), UR2)


def test_hllc_resolves_stationary_contact_and_shear():
    P = prob(2)
    UL = cons(1.0, 0.0, 1.0, 0.3)
    UR = cons(0.25, 0.0, 1.0, -0.8)
    # contact at rest: the sampled state is the left one (tie rule), flux-consistent
    np.testing.assert_allclose(O.hllc(P, 0, UL, UR), UL, rtol=1e-14)
    # a contact moving right: the left state up to x/t = u
    UL = cons(1.0, 0.2, 1.0, 0.3)
    UR = cons(0.25, 0.2, 1.0, -0.8)
    np.testing.assert_allclose(O.hllc(P, 0, UL, UR), UL, rtol=1e-13)
    UL = cons(1.0, -0.2, 1.0, 0.3)
    UR = cons(0.25, -0.2, 1.0, -0.8)
    np.testing.assert_allclose(O.hllc(P, 0, UL, UR), UR, rtol=1e-13)


@pytest.mark.parametrize("dE", [-1, 1])
def test_hllc_contact_at_rest_within_rounding_is_standing(dE):
    """A gas at rest whose two sides differ in pressure by one rounding step still counts as a
    standing contact: the left star state, the same whichever way the rounding went (reading of
    the leading term at a contact of speed zero)."""
    P = prob(1)
    UL = cons(1.0, 0.0, 1.0)
    UR = cons(0.25, 0.0, 1.0)
    exact = O.hllc(P, 0, UL, UR)
    np.testing.assert_allclose(exact, UL, rtol=1e-14)
    URp = UR.copy()
    URp[2] = np.nextafter(UR[2], UR[2] + dE)
    got = O.hllc(P, 0, UL, URp)
    np.testing.assert_allclose(got, UL, rtol=1e-14, atol=1e-15)
    # a contact moving at a small but resolved speed still goes by its sign
    URm = cons(0.25, 0.0, 1.0 + 1e-6 * dE)
    ULm = cons(1.0, 0.0, 1.0)
    s = O.hllc(P, 0, ULm, URm)
    assert abs(s[0] - 1.0) < 1e-5 if dE < 0 else abs(s[0] - 0.25) < 1e-5


def test_hllc_y_direction_is_x_direction_rotated():
    P = prob(2)
    rng = np.random.default_rng(2)
    for _ in range(10):
        a = cons(rng.uniform(0.3, 2), rng.uniform(-1, 1), rng.uniform(0.3, 2), rng.uniform(-1, 1))
        b = cons(rng.uniform(0.3, 2), rng.uniform(-1, 1), rng.uniform(0.3, 2), rng.uniform(-1, 1))
        swap = lambda U: U[[0, 2, 1, 3]]
        np.testing.assert_allclose(O.hllc(P, 1, a, b), swap(O.hllc(P, 0, swap(a), swap(b))), rtol=1e-13)


def euler_flux(U):
    rho, m, E = U
    u = m / rho
    p = (G - 1) * (E - 0.5 * rho * u * u)
    return np.array([m, m * u + p, u * (E + p)])


def shift(U, w):
    """Galilean boost by velocity w (1D conserved state)."""
    rho, m, E = U
    return np.array([rho, m + rho * w, E + m * w + 0.5 * rho * w * w])


@pytest.mark.parametrize("case", [((1.0, 0.0, 1.0), (0.125, 0.0, 0.1)),
                                  ((0.445, 0.698, 3.528), (0.5, 0.0, 0.571)),
                                  ((1.0, -1.0, 0.4), (1.0, 1.0, 0.4))])
def test_hllc_fan_integral_consistency(case):
    """The HLLC fan is a weak solution of the Riemann problem's integral form over the wave
    fan: int_a^b U(xi) dxi = b U_R - a U_L - (F(U_R) - F(U_L)) for a < S_L, S_R < b.  U(xi) is
    sampled by solving the problem in a frame moving with velocity -xi (the solver and the Davis
    speeds are Galilean invariant)."""
    P = prob(1)
    UL, UR = cons(*case[0]), cons(*case[1])
    a, b, n = -8.0, 8.0, 64000
    xs = a + (np.arange(n) + 0.5) * (b - a) / n
    integ = np.zeros(3)
    for x in xs:
        s = O.hllc(P, 0, shift(UL, -x), shift(UR, -x))
        integ += shift(s, x)
    integ *= (b - a) / n
    expect = b * UR - a * UL - (euler_flux(UR) - euler_flux(UL))
    np.testing.assert_allclose(integ, expect, rtol=2e-3, atol=2e-3)


def sympy_jacobian(dim, dir_):
    if dim == 1:
        r, m, E = sp.symbols("r m E", positive=True)
        W = sp.Matrix([r, m, E])
        p = (G - 1) * (E - m ** 2 / (2 * r))
        F = sp.Matrix([m, m ** 2 / r + p, m / r * (E + p)])
    else:
        r, m, n, E = sp.symbols("r m n E", positive=True)
        W = sp.Matrix([r, m, n, E])
        p = (G - 1) * (E - (m ** 2 + n ** 2) / (2 * r))
        if dir_ == 0:
            F = sp.Matrix([m, m ** 2 / r + p, m * n / r, m / r * (E + p)])
        else:
            F = sp.Matrix([n, m * n / r, n ** 2 / r + p, n / r * (E + p)])
    return W, F.jacobian(W)


@pytest.mark.parametrize("dim,dir_", [(1, 0), (2, 0), (2, 1)])
def test_eigensystem_against_symbolic_jacobian(dim, dir_):
    P = prob(dim)
    Wsym, J = sympy_jacobian(dim, dir_)
    rng = np.random.default_rng(dim * 10 + dir_)
    for _ in range(5):
        U = cons(rng.uniform(0.3, 2), rng.uniform(-2, 2), rng.uniform(0.3, 3)) if dim == 1 else \
            cons(rng.uniform(0.3, 2), rng.uniform(-2, 2), rng.uniform(0.3, 3), rng.uniform(-2, 2))
        A = np.array(J.subs(dict(zip(Wsym, U))).evalf(), dtype=float)
        lam, R, L = O.eigen(P, dir_, U)
        np.testing.assert_allclose(A @ R, R @ np.diag(lam), rtol=1e-12, atol=1e-11)
        np.testing.assert_allclose(R @ L, np.eye(len(U)), atol=1e-12)


def test_upwind_limits():
    P = prob(2)
    rng = np.random.default_rng(4)
    dL, dR = rng.normal(size=4), rng.normal(size=4)
    # supersonic right-moving: every lambda > 0 -> left data
    Ws = cons(1.0, 3.0, 0.5, 0.1)
    np.testing.assert_allclose(O.upwind(P, 0, Ws, dL, dR), dL, rtol=1e-12, atol=1e-12)
    Ws = cons(1.0, -3.0, 0.5, 0.1)
    np.testing.assert_allclose(O.upwind(P, 0, Ws, dL, dR), dR, rtol=1e-12, atol=1e-12)
    # continuous data is left unchanged whatever the state
    Ws = cons(1.0, 0.2, 1.0, 0.1)
    np.testing.assert_allclose(O.upwind(P, 0, Ws, dL, dL), dL, rtol=1e-12, atol=1e-12)
    # at rest: acoustic waves split, the two waves with lambda = 0 take the mean of both sides
    Ws = cons(1.0, 0.0, 1.0, 0.0)
    lam, R, L = O.eigen(P, 0, Ws)
    H = np.where(lam > 0, 1.0, np.where(lam < 0, 0.0, 0.5))
    np.testing.assert_allclose(O.upwind(P, 0, Ws, dL, dR), R @ (H * (L @ dL) + (1 - H) * (L @ dR)),
                               rtol=1e-12, atol=1e-12)
    # scalar Burgers: sign of u*
    Pb = prob(1, O.EQ_BURGERS)
    assert O.upwind(Pb, 0, [0.5], [1.0], [2.0])[0] == 1.0
    assert O.upwind(Pb, 0, [-0.5], [1.0], [2.0])[0] == 2.0
    assert O.upwind(Pb, 0, [0.0], [1.0], [2.0])[0] == 1.5
