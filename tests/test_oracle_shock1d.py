"""Oracle pins on the 1D shock examples of Section 5 (Examples 5.3-5.6).

Fixed by the mathematics and the textbook:
  * Lax's problem (Example 5.3) against the exact Riemann solution: L1 error of the density
    decreasing under refinement, no large overshoot;
  * the Shu-Osher problem (Example 5.4): the Mach 3 shock front moves at about 3 sound speeds of
    the gas ahead, so its position at T = 1.8 is fixed within a few cells;
  * Woodward-Colella blast waves (Example 5.6): reflective walls on both sides carry no mass and
    no energy (the mirrored Riemann problem has a star velocity of exactly zero), so total mass
    and energy stay constant to round-off, and the state stays physical at N = 200 and 400;
  * the initial data of all four are exact cell and derivative averages of the piecewise data.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2304_09724_gb300 import workloads as WL
from tests import exact_riemann


def run_wl(wl, T, **kw):
    P = O.make_problem(1, WL.EULER, wl.nx, 1, *wl.domain, bc=wl.bc, inflow=wl.inflow, **kw)
    return O.run(P, wl.state, T, wl.cfl)


def test_lax_against_exact_riemann_solution():
    L, R = (0.445, 0.698, 3.528), (0.5, 0.0, 0.571)
    errs = {}
    for n in (100, 200):
        wl = WL.lax(n)
        st, _, t = run_wl(wl, wl.t_final)
        ex = exact_riemann.density_averages(L, R, -5.0, 5.0, n, 0.0, t)
        rho = st["W"][0]
        errs[n] = float(np.mean(np.abs(rho - ex)))
        assert rho.max() < ex.max() * 1.03 and rho.min() > ex.min() * 0.95  # a few % at the contact
    assert errs[200] < 0.8 * errs[100]
    assert errs[200] < 2.5e-2


def test_shu_osher_shock_position():
    wl = WL.shu_osher(400)
    st, _, t = run_wl(wl, wl.t_final)
    rho = st["W"][0]
    x = np.linspace(-5, 5, 401)[:-1] + 0.0125
    front = x[np.argmax(np.abs(np.diff(rho))) ]  # steepest jump: the shock
    speed = 3.0 * math.sqrt(1.4)  # Mach 3 into gas at rest with p = rho = 1 (on average)
    assert abs(front - (-4.0 + speed * t)) < 0.15
    assert rho.min() > 0.75 and rho.max() < 4.8


@pytest.mark.parametrize("n", [200, 400])
def test_blast_waves_conserve_mass_and_energy(n):
    wl = WL.blast_waves(n)
    st, steps, t = run_wl(wl, wl.t_final)
    assert t == pytest.approx(0.038, rel=1e-14)
    for q in (0, 2):
        assert abs(st["W"][q].sum() - wl.state["W"][q].sum()) < 1e-12 * abs(wl.state["W"][q]).sum()
    assert np.isfinite(st["W"]).all() and st["W"][0].min() > 0


def test_piecewise_initial_averages_exact():
    # a cell cut by a jump holds the length-weighted mix; derivative averages are edge differences
    wl = WL.blast_waves(10)
    E = lambda p: p / 0.4
    np.testing.assert_allclose(wl.state["W"][2], [E(1000.0)] + [E(0.01)] * 8 + [E(100.0)], rtol=1e-15)
    np.testing.assert_allclose(wl.state["V"], 0.0, atol=0)
    wl = WL.blast_waves(15)  # jumps at 0.1 = 1.5 cells and 0.9 = 13.5 cells: cut cells
    assert wl.state["W"][2][1] == pytest.approx(0.5 * (E(1000.0) + E(0.01)), rel=1e-14)
    assert wl.state["V"][2][1] == pytest.approx((E(0.01) - E(1000.0)) * 15, rel=1e-14)
    wl = WL.shu_osher(40)
    xr = -5.0 + 10.0 * np.arange(1, 41) / 40
    xl = xr - 0.25
    rho_avg = np.where(xl >= -4.0, 1.0 + 0.2 * (np.cos(5 * xl) - np.cos(5 * xr)) / (5 * 0.25), 3.857143)
    np.testing.assert_allclose(wl.state["W"][0], rho_avg, rtol=1e-12)
