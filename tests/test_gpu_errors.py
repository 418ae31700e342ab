"""Failure handling on the GPU without faulting it: non-physical states are detected on the
device, reported as SHWENO_E_NONPHYSICAL, and the step that produced them is not committed."""
import numpy as np
import pytest

from paper_2304_09724_gb300 import shweno as S
from paper_2304_09724_gb300 import workloads as WL
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


def test_nonphysical_initial_state_rejected():
    wl = WL.sod(32)
    st = {k: v.copy() for k, v in wl.state.items()}
    st["W"][2, 5] = -1.0  # negative energy -> negative pressure
    sol = U.solver_of(wl)
    sol.set_state(st)
    with pytest.raises(S.ShwenoError) as e:
        sol.run(0.1, 0.6)
    assert e.value.status == S.E_NONPHYSICAL
    assert sol.time() == (0.0, 0)
    sol.close()


@pytest.mark.parametrize("dim", [1, 2])
def test_failed_step_is_not_committed(dim):
    wl = WL.sod(64) if dim == 1 else WL.riemann2d(32, WL.LAX_LIU_SHOCKS)
    sol = U.solver_of(wl)
    sol.set_state(wl.state)
    sol.step(1e-3)
    before = sol.get_state()
    t0, n0 = sol.time()
    with pytest.raises(S.ShwenoError) as e:
        sol.step(5.0)  # CFL ~ 100: the update leaves the physical range
    assert e.value.status == S.E_NONPHYSICAL
    after = sol.get_state()
    for k in before:
        assert np.array_equal(before[k], after[k])
    assert sol.time() == (t0, n0)
    # the handle stays usable
    sol.step(1e-3)
    assert sol.time()[1] == n0 + 1
    sol.close()


def test_run_stops_at_last_good_state():
    wl = WL.sod(64)
    sol = U.solver_of(wl)
    sol.set_state(wl.state)
    with pytest.raises(S.ShwenoError) as e:
        sol.run(0.2, 60.0)
    assert e.value.status == S.E_NONPHYSICAL
    t, n = sol.time()
    g = sol.get_state()
    assert np.isfinite(g["W"]).all() and (g["W"][0] > 0).all()
    sol.close()


def test_invalid_calls():
    wl = WL.sod(16)
    sol = U.solver_of(wl)
    with pytest.raises(S.ShwenoError) as e:
        sol.step(-1.0)
    assert e.value.status == S.E_INVALID
    sol2 = U.solver_of(wl, flag_mode=2)
    sol2.set_state(wl.state)
    with pytest.raises(S.ShwenoError) as e:
        sol2.step(1e-3)
    assert e.value.status == S.E_STATE
    sol.close()
    sol2.close()
