"""Pins of the oracle's characteristic-wise reconstruction option (reconstruction across a face
in the characteristic fields of the face-normal Jacobian at the mean of the two adjacent
states; an option beside the paper's componentwise reconstruction).

Fixed by the mathematics:
  * with the linear weights the reconstruction is linear in the data, so projecting onto any
    basis and back changes nothing: charwise = componentwise (1D and 2D);
  * a scalar law has a one-field basis: charwise = componentwise exactly;
  * 2D data that depend on x only (or y only) reduce to the 1D charwise scheme along that axis,
    which fixes the normal direction of the eigenvectors used at x- and y-faces;
  * the design order on smooth data and Sod's problem against the exact Riemann solution.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2304_09724_gb300 import workloads as WL
from tests import exact_riemann


def run_wl(wl, T, **kw):
    P = O.make_problem(wl.dim, wl.eq, wl.nx, wl.ny, *wl.domain, bc=wl.bc, inflow=wl.inflow, **kw)
    return O.run(P, wl.state, T, wl.cfl)


@pytest.mark.parametrize("maker,T", [(lambda: WL.sod(60), 0.1), (lambda: WL.euler1d_sine(20), 0.3),
                                     (lambda: WL.riemann2d(12, WL.LAX_LIU_SHOCKS), 0.02)])
def test_linear_weights_charwise_equals_componentwise(maker, T):
    wl = maker()
    a, na, _ = run_wl(wl, T, linear=True)
    b, nb, _ = run_wl(wl, T, linear=True, charwise=True)
    assert na == nb
    for k in a:
        scale = np.max(np.abs(a[k])) + 1e-300
        assert np.max(np.abs(a[k] - b[k])) <= 1e-11 * scale, k


def test_scalar_charwise_is_componentwise():
    wl = WL.burgers2d_riemann(12)
    a, _, _ = run_wl(wl, 0.05)
    b, _, _ = run_wl(wl, 0.05, charwise=True)
    for k in a:
        assert np.array_equal(a[k], b[k])


def test_charwise_differs_with_nonlinear_weights():
    wl = WL.sod(60)
    a, _, _ = run_wl(wl, 0.1)
    b, _, _ = run_wl(wl, 0.1, charwise=True)
    assert np.max(np.abs(a["W"] - b["W"])) > 1e-6


@pytest.mark.parametrize("axis", [0, 1])
def test_2d_one_direction_data_equal_1d_charwise(axis):
    n, m = 40, 5
    wl1 = WL.sod(n)
    W1, V1 = wl1.state["W"], wl1.state["V"]
    rho, mom, E = W1
    zero = np.zeros_like(rho)
    if axis == 0:
        comps = [rho, mom, zero, E]
        W2 = np.stack([np.repeat(c[None, :], m, axis=0) for c in comps])
        D2 = np.stack([np.repeat(c[None, :], m, axis=0) for c in (V1[0], V1[1], zero, V1[2])])
        st2 = {"W": W2, "V": D2, "Y": np.zeros_like(W2), "Z": np.zeros_like(W2)}
        P2 = O.make_problem(2, WL.EULER, n, m, 0.0, 1.0, 0.0, 0.3, bc=(1, 1, 0, 0), charwise=True)
    else:
        comps = [rho, zero, mom, E]
        W2 = np.stack([np.repeat(c[:, None], m, axis=1) for c in comps])
        D2 = np.stack([np.repeat(c[:, None], m, axis=1) for c in (V1[0], zero, V1[1], V1[2])])
        st2 = {"W": W2, "V": np.zeros_like(W2), "Y": D2, "Z": np.zeros_like(W2)}
        P2 = O.make_problem(2, WL.EULER, m, n, 0.0, 0.3, 0.0, 1.0, bc=(0, 0, 1, 1), charwise=True)
    P1 = O.make_problem(1, WL.EULER, n, x0=0.0, x1=1.0, bc=(1, 1), charwise=True)
    s1, s2 = wl1.state, st2
    for _ in range(4):
        s1 = O.step(P1, s1, 0.004)
        s2 = O.step(P2, s2, 0.004)
    along = "V" if axis == 0 else "Y"
    q2 = (0, 1, 3) if axis == 0 else (0, 2, 3)
    for qa, qb in zip(q2, (0, 1, 2)):
        for r in range(m):
            w = s2["W"][qa, r] if axis == 0 else s2["W"][qa, :, r]
            d = s2[along][qa, r] if axis == 0 else s2[along][qa, :, r]
            np.testing.assert_allclose(w, s1["W"][qb], rtol=1e-11, atol=1e-12)
            np.testing.assert_allclose(d, s1["V"][qb], rtol=1e-9, atol=1e-9)


def test_order_euler1d_charwise():
    errs = {}
    for n in (20, 40, 80):
        wl = WL.euler1d_sine(n)
        st, _, _ = run_wl(wl, 2.0, charwise=True)
        errs[n] = float(np.mean(np.abs(st["W"][0] - wl.exact(2.0)[0])))
    assert math.log2(errs[40] / errs[80]) > 4.5


def test_order_vortex_charwise():
    errs = {}
    for n in (20, 40):
        wl = WL.vortex(n)
        st, _, _ = run_wl(wl, 0.25, charwise=True)
        errs[n] = float(np.mean(np.abs(st["W"][0] - wl.exact(0.25)[0])))
    assert math.log2(errs[20] / errs[40]) > 4.0


def test_sod_charwise_against_exact():
    L, R = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    errs = {}
    for n in (100, 200):
        wl = WL.sod(n)
        st, _, _ = run_wl(wl, wl.t_final, charwise=True)
        ex = exact_riemann.density_averages(L, R, 0.0, 1.0, n, 0.5, wl.t_final)
        rho = st["W"][0]
        errs[n] = float(np.mean(np.abs(rho - ex)))
        assert rho.min() > 0.125 * 0.97 and rho.max() < 1.0 * 1.03
    assert errs[200] < 0.75 * errs[100]
    assert errs[200] < 4e-3


def test_2d_reflective_wall_along_y_equals_1d_charwise():
    """A shock running into a reflective wall along y in 2D (data depending on y only) gives the
    1D characteristic-wise scheme with the same wall, on every column."""
    n, m = 60, 4
    wl1 = WL.riemann1d(n, (3.0, -1.5, 5.0), (1.0, -1.5, 1.0), xs=0.5, bc=(WL.REFLECTIVE, WL.OUTFLOW))
    W1, V1 = wl1.state["W"], wl1.state["V"]
    rho, mom, E = W1
    zero = np.zeros_like(rho)
    W2 = np.stack([np.repeat(c[:, None], m, axis=1) for c in (rho, zero, mom, E)])
    D2 = np.stack([np.repeat(c[:, None], m, axis=1) for c in (V1[0], zero, V1[1], V1[2])])
    s2 = {"W": W2, "V": np.zeros_like(W2), "Y": D2, "Z": np.zeros_like(W2)}
    P1 = O.make_problem(1, WL.EULER, n, x0=0.0, x1=1.0, bc=(WL.REFLECTIVE, WL.OUTFLOW), charwise=True)
    P2 = O.make_problem(2, WL.EULER, m, n, 0.0, 0.2, 0.0, 1.0, bc=(0, 0, WL.REFLECTIVE, WL.OUTFLOW),
                        charwise=True)
    s1 = wl1.state
    for _ in range(40):
        s1 = O.step(P1, s1, 0.002)
        s2 = O.step(P2, s2, 0.002)
    for q2, q1 in ((0, 0), (2, 1), (3, 2)):
        for c in range(m):
            np.testing.assert_allclose(s2["W"][q2][:, c], s1["W"][q1], rtol=1e-12, atol=1e-12)
