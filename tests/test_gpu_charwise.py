"""GPU parity of the characteristic-wise reconstruction option (reconstruction across each face
in the characteristic fields of the face-normal flux Jacobian at the mean of the two adjacent
states) against the oracle's same option: 1D Riemann problems and the shock / density-wave
examples, smooth data at sizes with ragged tails, 2D Riemann problems, the vortex, the double
Mach reflection and per-cell flags; the batch refuses 2D characteristic-wise handles."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2304_09724_gb300 import shweno as S
from paper_2304_09724_gb300 import workloads as WL
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("maker,T", [(lambda: WL.sod(100), 0.2), (lambda: WL.lax(200), 1.3),
                                     (lambda: WL.shu_osher(400), 0.6),
                                     (lambda: WL.blast_waves(400), 0.01),
                                     (lambda: WL.random_riemann1d(5, nx=300), 0.1)])
def test_1d_shocks(maker, T):
    wl = maker()
    g, o, (t, n), (t_o, n_o) = U.run_both(wl, T, charwise=True)
    assert n == n_o and t == t_o
    U.check(g, o, U.fields(wl), shocked=True, what=f"{wl.name} charwise", wl=wl)


@pytest.mark.parametrize("n", [4, 129, 300])
def test_1d_smooth_sizes(n):
    W, V = WL.random_smooth_1d(n, n)
    wl = WL.euler1d_sine(n)
    wl.domain, wl.state = (0.0, 1.0, 0.0, 1.0), {"W": W, "V": V}
    g, o = U.steps_both(wl, [0.2 / n] * 3, charwise=True)
    U.check(g, o, U.fields(wl), shocked=False, what=f"smooth 1D n={n} charwise", wl=wl)


@pytest.mark.parametrize("nx,ny", [(7, 5), (130, 9), (9, 131)])
def test_2d_smooth_sizes(nx, ny):
    W, V, Y, Z = WL.random_smooth_2d(3, nx, ny)
    wl = WL.vortex(8)
    wl.nx, wl.ny, wl.domain = nx, ny, (0.0, 1.0, 0.0, 1.0)
    wl.state = {"W": W, "V": V, "Y": Y, "Z": Z}
    dt = 0.15 / max(nx, ny)
    g, o = U.steps_both(wl, [dt, dt], charwise=True)
    U.check(g, o, U.fields(wl), shocked=False, what=f"smooth {nx}x{ny} charwise", wl=wl)


def test_vortex_run():
    wl = WL.vortex(24)
    g, o, (t, n), (t_o, n_o) = U.run_both(wl, 0.5, charwise=True)
    assert n == n_o and t == t_o
    U.check(g, o, U.fields(wl), shocked=False, what="vortex charwise", wl=wl)


@pytest.mark.parametrize("maker,T", [(lambda: WL.riemann2d(40, WL.LAX_LIU_SHOCKS), 0.05),
                                     (lambda: WL.riemann2d(33, WL.random_quadrants(103)), 0.05)])
def test_2d_shocks(maker, T):
    wl = maker()
    g, o, (t, n), (t_o, n_o) = U.run_both(wl, T, charwise=True)
    assert n == n_o
    U.check(g, o, U.fields(wl), shocked=True, what=f"{wl.name} charwise", wl=wl)


def test_dmr_charwise_nonphysical_like_the_oracle():
    """The characteristic-wise option leaves the physical range at the shock foot on the wall of
    the double Mach reflection within two steps; the library stops at the same step as the
    oracle and keeps the same last good state."""
    wl = WL.dmr(64, 16)
    with pytest.raises(O.NonPhysical) as eo:
        O.run(U.problem_of(wl, charwise=True), wl.state, 0.004, wl.cfl)
    sol = U.solver_of(wl, charwise=True)
    sol.set_state(wl.state)
    with pytest.raises(S.ShwenoError) as eg:
        sol.run(0.004, wl.cfl)
    assert eg.value.status == S.E_NONPHYSICAL
    t, n = sol.time()
    assert n == eo.value.steps and t == pytest.approx(eo.value.t, rel=1e-12)
    g = sol.get_state()
    sol.close()
    U.check(g, eo.value.state, U.fields(wl), shocked=True, what="DMR charwise last good state", wl=wl)


def test_per_cell_flags_charwise():
    n = 24
    wl = WL.riemann2d(n, WL.LAX_LIU_CONTACTS)
    rng = np.random.default_rng(2)
    flag = (rng.random((n, n)) < 0.4).astype(np.uint8)
    near = np.zeros((n, n), bool)
    near[:, n // 2 - 3:n // 2 + 3] = True
    near[n // 2 - 3:n // 2 + 3, :] = True
    flag[near] = 1
    g, o = U.steps_both(wl, [0.002] * 2, flag=flag, flag_mode=2, charwise=True)
    U.check(g, o, U.fields(wl), shocked=True, what="per-cell flags charwise", wl=wl)


def test_batch_refuses_2d_charwise_and_runs_1d_charwise():
    wl2 = WL.riemann2d(16, WL.LAX_LIU_SHOCKS)
    s2 = U.solver_of(wl2, charwise=True)
    s2.set_state(wl2.state)
    with pytest.raises(S.ShwenoError) as e:
        S.Batch([s2])
    assert e.value.status == S.E_INVALID
    s2.close()
    wl1 = WL.random_riemann1d(7, nx=333)
    a = U.solver_of(wl1, charwise=True)
    a.set_state(wl1.state)
    b = S.Batch([a])
    b.run([0.05], wl1.cfl)
    b.close()
    ga, (ta, na) = a.get_state(), a.time()
    a.close()
    g, o, (t, n), _ = U.run_both(wl1, 0.05, charwise=True)
    assert na == n
    U.check(ga, g, U.fields(wl1), shocked=True, what="batched 1D charwise", wl=wl1)
