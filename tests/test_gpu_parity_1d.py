"""GPU parity, one space dimension: the CUDA step through the C ABI against the oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2304_09724_gb300 import workloads as WL
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


def test_burgers_example_5_1_full_run_n200():
    """The small configuration: Burgers, N = 200, CFL 0.6, T = 0.5/pi, device-side time loop."""
    wl = WL.burgers_sine(200)
    g, o, (t, n), (t_o, n_o) = U.run_both(wl, wl.t_final)
    assert n == n_o and t == t_o == wl.t_final
    U.check(g, o, U.fields(wl), shocked=False, what="burgers N=200", wl=wl)


@pytest.mark.parametrize("n", [4, 5, 17, 64, 129, 300])
def test_burgers_sizes_fixed_steps(n):
    """Sizes below, at and across the 128-face CTA width, with ragged tails."""
    W, V = WL.random_smooth_1d(n, n, eq=WL.BURGERS)
    wl = WL.burgers_sine(n)
    wl.domain = (0.0, 1.0, 0.0, 1.0)
    wl.state = {"W": W, "V": V}
    g, o = U.steps_both(wl, [0.2 / n] * 3)
    U.check(g, o, U.fields(wl), shocked=False, what=f"burgers n={n}", wl=wl)


@pytest.mark.parametrize("n", [16, 130])
@pytest.mark.parametrize("bc", [(WL.PERIODIC, WL.PERIODIC), (WL.OUTFLOW, WL.REFLECTIVE), (WL.REFLECTIVE, WL.INFLOW)])
def test_euler1d_smooth_all_bcs(n, bc):
    W, V = WL.random_smooth_1d(7, n)
    wl = WL.euler1d_sine(n)
    wl.domain = (0.0, 1.0, 0.0, 1.0)
    wl.bc = bc + (0, 0)
    wl.inflow = [list(W[:, -1]) + [0.0]] * 4
    wl.state = {"W": W, "V": V}
    g, o = U.steps_both(wl, [0.1 / n] * 4)
    U.check(g, o, U.fields(wl), shocked=False, what=f"euler1d n={n} bc={bc}", wl=wl)


def test_euler1d_example_5_2_run():
    wl = WL.euler1d_sine(40)
    g, o, (t, n), (t_o, n_o) = U.run_both(wl, 1.0)
    assert n == n_o and t == t_o == 1.0
    U.check(g, o, U.fields(wl), shocked=False, what="euler1d sine", wl=wl)


@pytest.mark.parametrize("maker", [lambda: WL.sod(100), lambda: WL.lax(200), lambda: WL.random_riemann1d(3, nx=257)])
def test_euler1d_shocked_runs(maker):
    wl = maker()
    T = min(wl.t_final, 0.05 if wl.name.startswith("riemann") else wl.t_final)
    g, o, (t, n), (t_o, n_o) = U.run_both(wl, T)
    assert n == n_o
    U.check(g, o, U.fields(wl), shocked=True, what=wl.name, wl=wl)


def test_linear_weights_mode():
    W, V = WL.random_smooth_1d(11, 50)
    wl = WL.euler1d_sine(50)
    wl.domain = (0.0, 1.0, 0.0, 1.0)
    wl.state = {"W": W, "V": V}
    g, o = U.steps_both(wl, [0.002] * 3, flag_mode=1, linear=True)
    U.check(g, o, U.fields(wl), shocked=False, what="linear weights", wl=wl)


def test_per_cell_flags():
    """Random flags in smooth regions, nonlinear weights kept within four cells of the jump."""
    wl = WL.sod(64)
    rng = np.random.default_rng(1)
    flag = (rng.random(64) < 0.5).astype(np.uint8)
    flag[28:36] = 1
    g, o = U.steps_both(wl, [0.004] * 3, flag=flag, flag_mode=2)
    U.check(g, o, U.fields(wl), shocked=True, what="per-cell flags", wl=wl)
    W, V = WL.random_smooth_1d(12, 64)
    wl.state = {"W": W, "V": V}
    flag = (rng.random(64) < 0.5).astype(np.uint8)
    g, o = U.steps_both(wl, [0.002] * 3, flag=flag, flag_mode=2)
    U.check(g, o, U.fields(wl), shocked=False, what="per-cell flags, smooth", wl=wl)


@pytest.mark.parametrize("eps", [1e-2, 1e-10])
def test_epsilon_option(eps):
    """The epsilon of the nonlinear weights is an option (shweno_opts.eps): parity with the
    oracle's same epsilon on a shocked and a smooth 1D run, and on a 2D Riemann problem."""
    for wl, T, shocked in ((WL.lax(200), 0.5, True), (WL.euler1d_sine(40), 0.5, False)):
        sol = U.solver_of(wl, eps=eps)
        sol.set_state(wl.state)
        t, n = sol.run(T, wl.cfl)
        g = sol.get_state()
        sol.close()
        o, n_o, t_o = O.run(U.problem_of(wl, eps=eps), wl.state, T, wl.cfl)
        assert n == n_o
        U.check(g, o, U.fields(wl), shocked=shocked, what=f"{wl.name} eps={eps}", wl=wl)
    wl = WL.riemann2d(24, WL.LAX_LIU_SHOCKS)
    sol = U.solver_of(wl, eps=eps)
    sol.set_state(wl.state)
    sol.run(0.03, wl.cfl)
    g = sol.get_state()
    sol.close()
    o, _, _ = O.run(U.problem_of(wl, eps=eps), wl.state, 0.03, wl.cfl)
    U.check(g, o, U.fields(wl), shocked=True, what=f"2D eps={eps}", wl=wl)
