"""Pins of the oracle's 2D scalar Burgers scheme, u_t + (u^2/2)_x + (u^2/2)_y = 0 (Section 3
applied to the scalar law of Eq. 5.1 in two dimensions).

Fixed by the mathematics, not by the oracle itself:
  * data that depend on x only (or y only) reduce one 2D step to the 1D scheme of Section 2 along
    that direction, exactly up to rounding (the other direction's fluxes cancel);
  * swapping x and y swaps V and Y (F = G);
  * periodic sums of W are conserved and the sums of V, Y, Z vanish (telescoping of Eq. 3.2/3.10);
  * a constant state stays constant;
  * design order: the diagonal wave u = u0(x + y - 2ut) (Newton at every quadrature point),
    fifth order approached under refinement.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2304_09724_gb300 import workloads as WL


def prob2(nx, ny, x1=1.0, y1=1.0, bc=(0, 0, 0, 0)):
    return O.make_problem(2, WL.BURGERS, nx, ny, 0.0, x1, 0.0, y1, bc=bc)


@pytest.mark.parametrize("axis", [0, 1])
def test_one_direction_data_equal_1d(axis):
    n, m = 20, 5
    W1, V1 = WL.random_smooth_1d(7, n, eq=WL.BURGERS)
    P1 = O.make_problem(1, WL.BURGERS, n, x0=0.0, x1=1.0)
    if axis == 0:
        W2 = np.repeat(W1[:, None, :], m, axis=1)
        D2 = np.repeat(V1[:, None, :], m, axis=1)
        st2 = {"W": W2, "V": D2, "Y": np.zeros_like(W2), "Z": np.zeros_like(W2)}
        P2 = prob2(n, m, 1.0, 0.7)
    else:
        W2 = np.repeat(W1[:, :, None], m, axis=2)
        D2 = np.repeat(V1[:, :, None], m, axis=2)
        st2 = {"W": W2, "V": np.zeros_like(W2), "Y": D2, "Z": np.zeros_like(W2)}
        P2 = prob2(m, n, 0.7, 1.0)
    s1, s2 = {"W": W1, "V": V1}, st2
    for _ in range(3):
        s1 = O.step(P1, s1, 0.01)
        s2 = O.step(P2, s2, 0.01)
    along, across = ("V", "Y") if axis == 0 else ("Y", "V")
    for r in range(m):
        w = s2["W"][0, r] if axis == 0 else s2["W"][0, :, r]
        d = s2[along][0, r] if axis == 0 else s2[along][0, :, r]
        np.testing.assert_allclose(w, s1["W"][0], rtol=1e-13, atol=1e-14)
        np.testing.assert_allclose(d, s1["V"][0], rtol=1e-10, atol=1e-11)
    np.testing.assert_allclose(s2[across], 0.0, atol=1e-11)
    np.testing.assert_allclose(s2["Z"], 0.0, atol=1e-9)


def test_transposition_symmetry():
    nx, ny = 9, 7
    W, V, Y, Z = WL.random_smooth_2d(5, nx, ny, eq=WL.BURGERS)
    tr = lambda a: np.ascontiguousarray(np.transpose(a, (0, 2, 1)))
    a = O.step(prob2(nx, ny), {"W": W, "V": V, "Y": Y, "Z": Z}, 0.01)
    b = O.step(prob2(ny, nx), {"W": tr(W), "V": tr(Y), "Y": tr(V), "Z": tr(Z)}, 0.01)
    np.testing.assert_allclose(tr(a["W"]), b["W"], rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(tr(a["V"]), b["Y"], rtol=1e-10, atol=1e-11)
    np.testing.assert_allclose(tr(a["Y"]), b["V"], rtol=1e-10, atol=1e-11)


def test_conservation_and_derivative_sums():
    W, V, Y, Z = WL.random_smooth_2d(6, 10, 8, eq=WL.BURGERS)
    P = prob2(10, 8)
    st = {"W": W, "V": V, "Y": Y, "Z": Z}
    for _ in range(3):
        st = O.step(P, st, 0.01)
    assert abs(st["W"].sum() - W.sum()) < 1e-12 * np.abs(W).sum()
    for k in "VYZ":
        assert abs(st[k].sum()) < 1e-9


def test_free_stream():
    st = WL.constant_state(2, WL.BURGERS, 8, 6, value=[0.7])
    out = O.step(prob2(8, 6, bc=(1, 1, 2, 2)), st, 0.01)
    for k in st:
        np.testing.assert_allclose(out[k], st[k], rtol=0, atol=1e-14)


def test_design_order_diagonal_wave():
    errs = {}
    for n in (20, 40, 80):
        wl = WL.burgers2d_sine(n)
        P = O.make_problem(2, WL.BURGERS, n, n, *wl.domain, bc=wl.bc)
        st, steps, t = O.run(P, wl.state, wl.t_final, wl.cfl)
        assert steps > 0 and t == pytest.approx(wl.t_final, rel=1e-14)
        errs[n] = float(np.mean(np.abs(st["W"][0] - wl.exact(t)[0])))
    assert errs[80] < 3e-7
    assert math.log2(errs[20] / errs[40]) > 4.0
    assert math.log2(errs[40] / errs[80]) > 4.0
