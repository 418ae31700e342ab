"""GPU parity of the R1' option (quintic p1 that also matches the cell's own derivative average,
the alternative reading of the reconstruction the paper omits in Section 2.4) against the
oracle's same option: 1D and 2D, Burgers and Euler, smooth and shocked, sizes with ragged tails,
together with the characteristic-wise option, the linear weights and per-cell flags; the batch
refuses R1' handles."""
import numpy as np
import pytest

from paper_2304_09724_gb300 import shweno as S
from paper_2304_09724_gb300 import workloads as WL
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("maker,T,shocked", [(lambda: WL.burgers_sine(200), None, False),
                                             (lambda: WL.euler1d_sine(40), 0.5, False),
                                             (lambda: WL.sod(100), 0.2, True),
                                             (lambda: WL.lax(200), 1.3, True)])
def test_1d_runs(maker, T, shocked):
    wl = maker()
    g, o, (t, n), (t_o, n_o) = U.run_both(wl, wl.t_final if T is None else T, quintic=True)
    assert n == n_o and t == t_o
    U.check(g, o, U.fields(wl), shocked=shocked, what=f"{wl.name} R1'", wl=wl)


@pytest.mark.parametrize("nx,ny", [(7, 5), (130, 9), (9, 131)])
def test_2d_smooth_sizes(nx, ny):
    W, V, Y, Z = WL.random_smooth_2d(3, nx, ny)
    wl = WL.vortex(8)
    wl.nx, wl.ny, wl.domain = nx, ny, (0.0, 1.0, 0.0, 1.0)
    wl.state = {"W": W, "V": V, "Y": Y, "Z": Z}
    dt = 0.15 / max(nx, ny)
    g, o = U.steps_both(wl, [dt, dt], quintic=True)
    U.check(g, o, U.fields(wl), shocked=False, what=f"smooth {nx}x{ny} R1'", wl=wl)


def test_vortex_and_burgers2d_runs():
    for wl, T in ((WL.vortex(24), 0.5), (WL.burgers2d_sine(32), None)):
        g, o, (t, n), (t_o, n_o) = U.run_both(wl, wl.t_final if T is None else T, quintic=True)
        assert n == n_o and t == t_o
        U.check(g, o, U.fields(wl), shocked=False, what=f"{wl.name} R1'", wl=wl)


@pytest.mark.parametrize("charwise", [False, True])
def test_2d_shocks(charwise):
    wl = WL.riemann2d(40, WL.LAX_LIU_SHOCKS)
    g, o, (t, n), (t_o, n_o) = U.run_both(wl, 0.05, quintic=True, charwise=charwise)
    assert n == n_o
    U.check(g, o, U.fields(wl), shocked=True, what=f"Example 5.9 R1' charwise={charwise}", wl=wl)


def test_linear_weights_and_flags():
    W, V, Y, Z = WL.random_smooth_2d(6, 24, 18)
    wl = WL.vortex(8)
    wl.nx, wl.ny, wl.domain = 24, 18, (0.0, 1.0, 0.0, 1.0)
    wl.state = {"W": W, "V": V, "Y": Y, "Z": Z}
    g, o = U.steps_both(wl, [0.005] * 2, flag_mode=1, linear=True, quintic=True)
    U.check(g, o, U.fields(wl), shocked=False, what="R1' linear weights", wl=wl)
    rng = np.random.default_rng(9)
    flag = (rng.random((18, 24)) < 0.5).astype(np.uint8)
    g, o = U.steps_both(wl, [0.005] * 2, flag=flag, flag_mode=2, quintic=True)
    U.check(g, o, U.fields(wl), shocked=False, what="R1' per-cell flags", wl=wl)


def test_batch_refuses_quintic():
    wl = WL.sod(64)
    s = U.solver_of(wl, quintic=True)
    s.set_state(wl.state)
    with pytest.raises(S.ShwenoError) as e:
        S.Batch([s])
    assert e.value.status == S.E_INVALID
    s.close()
