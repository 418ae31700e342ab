"""GPU parity of 2D scalar Burgers (u_t + (u^2/2)_x + (u^2/2)_y = 0, Section 3 with the scalar
flux of Example 5.1): the CUDA step through the C ABI against the oracle, on smooth data with
sign changes (sonic points), at sizes spanning several 128-face CTAs with ragged tails, every
boundary kind, and a four-quadrant Riemann problem with shocks and rarefactions."""
import numpy as np
import pytest

from paper_2304_09724_gb300 import shweno as S
from paper_2304_09724_gb300 import workloads as WL
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


def smooth(nx, ny, seed=3, bc=(WL.PERIODIC,) * 4):
    W, V, Y, Z = WL.random_smooth_2d(seed, nx, ny, eq=WL.BURGERS)
    wl = WL.burgers2d_sine(8)
    wl.nx, wl.ny, wl.domain, wl.bc = nx, ny, (0.0, 1.0, 0.0, 1.0), bc
    wl.state = {"W": W, "V": V, "Y": Y, "Z": Z}
    return wl


@pytest.mark.parametrize("nx,ny", [(4, 4), (7, 5), (130, 9), (9, 131), (150, 37)])
def test_smooth_sizes(nx, ny):
    wl = smooth(nx, ny)
    dt = 0.1 / max(nx, ny)
    g, o = U.steps_both(wl, [dt, dt])
    U.check(g, o, U.fields(wl), shocked=False, what=f"burgers2d {nx}x{ny}", wl=wl)


@pytest.mark.parametrize("bc", [(WL.OUTFLOW, WL.REFLECTIVE, WL.REFLECTIVE, WL.OUTFLOW),
                                (WL.INFLOW, WL.OUTFLOW, WL.PERIODIC, WL.PERIODIC)])
def test_smooth_boundaries(bc):
    wl = smooth(20, 14, seed=5, bc=bc)
    wl.inflow = [[0.3, 0.0, 0.0, 0.0]] * 4
    g, o = U.steps_both(wl, [0.004] * 3)
    U.check(g, o, U.fields(wl), shocked=False, what=f"burgers2d bc {bc}", wl=wl)


def test_diagonal_wave_run_device_time_loop():
    wl = WL.burgers2d_sine(48)
    g, o, (t, n), (t_o, n_o) = U.run_both(wl, wl.t_final)
    assert n == n_o and t == t_o
    U.check(g, o, U.fields(wl), shocked=False, what="burgers2d diagonal wave", wl=wl)


def test_four_quadrant_riemann_problem():
    wl = WL.burgers2d_riemann(40)
    g, o, (t, n), (t_o, n_o) = U.run_both(wl, 0.1)
    assert n == n_o
    U.check(g, o, U.fields(wl), shocked=True, what="burgers2d riemann", wl=wl)


def test_linear_weights_and_per_cell_flags():
    wl = smooth(24, 18, seed=6)
    g, o = U.steps_both(wl, [0.004] * 2, flag_mode=1, linear=True)
    U.check(g, o, U.fields(wl), shocked=False, what="burgers2d linear weights", wl=wl)
    rng = np.random.default_rng(4)
    flag = (rng.random((18, 24)) < 0.5).astype(np.uint8)
    g, o = U.steps_both(wl, [0.004] * 2, flag=flag, flag_mode=2)
    U.check(g, o, U.fields(wl), shocked=False, what="burgers2d per-cell flags", wl=wl)


def test_conservation_periodic():
    wl = smooth(40, 24, seed=8)
    sol = U.solver_of(wl)
    sol.set_state(wl.state)
    for _ in range(5):
        sol.step(0.003)
    g = sol.get_state()
    sol.close()
    assert abs(g["W"].sum() - wl.state["W"].sum()) < 1e-12 * np.abs(wl.state["W"]).sum()


def test_dmr_boundaries_rejected_for_burgers():
    with pytest.raises(S.ShwenoError) as e:
        S.Solver(2, S.BURGERS, 16, 8, (0.0, 4.0, 0.0, 1.0), (WL.INFLOW, WL.OUTFLOW, 4, 5))
    assert e.value.status == S.E_INVALID
