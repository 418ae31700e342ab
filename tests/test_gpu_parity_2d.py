"""GPU parity, two space dimensions: the CUDA step through the C ABI against the oracle.

Sizes span several 128-face CTAs along both directions with ragged tails; the full-size
2048 x 2048 vortex (the benchmark's workload, same launch configuration) is checked on sampled
cells that the oracle evaluates one by one."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2304_09724_gb300 import shweno as S
from paper_2304_09724_gb300 import workloads as WL
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


def smooth2d(nx, ny, seed=3, bc=(WL.PERIODIC,) * 4):
    W, V, Y, Z = WL.random_smooth_2d(seed, nx, ny)
    wl = WL.vortex(8)
    wl.nx, wl.ny, wl.domain, wl.bc = nx, ny, (0.0, 1.0, 0.0, 1.0), bc
    wl.state = {"W": W, "V": V, "Y": Y, "Z": Z}
    return wl


@pytest.mark.parametrize("nx,ny", [(4, 4), (7, 5), (16, 16), (130, 9), (9, 131), (150, 37)])
def test_smooth_sizes(nx, ny):
    wl = smooth2d(nx, ny)
    dt = 0.15 / max(nx, ny)
    g, o = U.steps_both(wl, [dt, dt])
    U.check(g, o, U.fields(wl), shocked=False, what=f"smooth {nx}x{ny}", wl=wl)


@pytest.mark.parametrize("bc", [(WL.OUTFLOW, WL.REFLECTIVE, WL.REFLECTIVE, WL.OUTFLOW),
                                (WL.REFLECTIVE, WL.PERIODIC, WL.INFLOW, WL.OUTFLOW)])
def test_smooth_boundaries(bc):
    if (bc[0] == WL.PERIODIC) != (bc[1] == WL.PERIODIC):
        bc = (WL.REFLECTIVE, WL.REFLECTIVE) + bc[2:]
    wl = smooth2d(20, 14, seed=5, bc=bc)
    wl.inflow = [[1.0, 0.4, -0.3, 2.6]] * 4
    g, o = U.steps_both(wl, [0.005] * 3)
    U.check(g, o, U.fields(wl), shocked=False, what=f"bc {bc}", wl=wl)


def test_vortex_run_device_time_loop():
    wl = WL.vortex(24)
    g, o, (t, n), (t_o, n_o) = U.run_both(wl, 0.5)
    assert n == n_o and t == t_o == 0.5
    U.check(g, o, U.fields(wl), shocked=False, what="vortex 24^2", wl=wl)


def test_four_shock_riemann_problem():
    wl = WL.riemann2d(40, WL.LAX_LIU_SHOCKS)
    g, o, (t, n), (t_o, n_o) = U.run_both(wl, 0.05)
    assert n == n_o
    U.check(g, o, U.fields(wl), shocked=True, what="Example 5.9 shocks", wl=wl)


def test_random_quadrants_ragged():
    wl = WL.riemann2d(33, WL.random_quadrants(4))
    g, o, _, _ = U.run_both(wl, 0.03)
    U.check(g, o, U.fields(wl), shocked=True, what="random quadrants", wl=wl)


def test_double_mach_reflection_small():
    wl = WL.dmr(64, 16)
    g, o, (t, n), (t_o, n_o) = U.run_both(wl, 0.004)
    assert n == n_o
    U.check(g, o, U.fields(wl), shocked=True, what="DMR 64x16", wl=wl)


def test_linear_weights_smooth():
    wl = smooth2d(24, 18, seed=6)
    g, o = U.steps_both(wl, [0.005] * 2, flag_mode=1, linear=True)
    U.check(g, o, U.fields(wl), shocked=False, what="linear weights", wl=wl)


def test_per_cell_flags():
    """Random flags away from the discontinuities; nonlinear weights within three cells of the
    quadrant boundaries (what a troubled-cell flag must guarantee)."""
    n = 24
    wl = WL.riemann2d(n, WL.LAX_LIU_CONTACTS)
    rng = np.random.default_rng(2)
    flag = (rng.random((n, n)) < 0.4).astype(np.uint8)
    near = np.zeros((n, n), bool)
    near[:, n // 2 - 3:n // 2 + 3] = True
    near[n // 2 - 3:n // 2 + 3, :] = True
    flag[near] = 1
    g, o = U.steps_both(wl, [0.002] * 2, flag=flag, flag_mode=2)
    U.check(g, o, U.fields(wl), shocked=True, what="per-cell flags", wl=wl)


def test_conservation_periodic():
    wl = smooth2d(40, 24, seed=8)
    sol = U.solver_of(wl)
    sol.set_state(wl.state)
    for _ in range(5):
        sol.step(0.004)
    g = sol.get_state()
    np.testing.assert_allclose(g["W"].sum(axis=(1, 2)), wl.state["W"].sum(axis=(1, 2)), rtol=1e-13)
    sol.close()


def test_full_size_vortex_2048_sampled_cells():
    """Configuration of the benchmark: 2048 x 2048 vortex, one CFL step through the C ABI with
    device-resident inputs (torch memory), compared on sampled cells (corners, edges, the
    vortex core, random interior) evaluated by the oracle cell by cell."""
    import torch

    wl = WL.vortex(2048)
    sol = U.solver_of(wl)
    dev = {k: torch.from_numpy(v).cuda() for k, v in wl.state.items()}
    sol.set_state(dev)
    dt, _ = S.shweno_cfl_dt(sol.h, wl.cfl)
    sol.step(dt)
    g = sol.get_state()
    sol.close()
    rng = np.random.default_rng(0)
    cells = [(0, 0), (2047, 2047), (0, 2047), (2047, 0), (1024, 1024), (1023, 1000), (5, 2046)]
    cells += [tuple(int(x) for x in rng.integers(0, 2048, size=2)) for _ in range(25)]
    P = U.problem_of(wl)
    o = O.step2d_cells(P, wl.state, dt, cells)
    gs = {k: np.array([g[k][:, j, i] for (i, j) in cells]) for k in "WVYZ"}
    U.check(gs, o, "WVYZ", shocked=False, what="2048^2 sampled cells", wl=wl)


def test_checkpoint_resume_bitwise():
    wl = WL.riemann2d(36, WL.LAX_LIU_SHOCKS)
    a = U.solver_of(wl)
    a.set_state(wl.state)
    for _ in range(6):
        a.step(0.002)
    ga = a.get_state()
    b = U.solver_of(wl)
    b.set_state(wl.state)
    for _ in range(3):
        b.step(0.002)
    t, n = b.time()
    mid = b.get_state()
    b.close()
    c = U.solver_of(wl)
    c.set_state(mid, t)
    for _ in range(3):
        c.step(0.002)
    gc = c.get_state()
    for k in "WVYZ":
        assert np.array_equal(ga[k], gc[k])
    a.close()
    c.close()
