"""The batched persistent launch against the oracle, problem by problem.

A ragged batch of 1D Riemann problems (40 ... 1000 cells), random four-quadrant 2D Riemann
problems, the 2D Burgers Riemann problem, a small isentropic vortex and the 1D Burgers wave of
Example 5.1 runs to its end times in one persistent launch; every problem must take the oracle's
number of CFL steps, end at the oracle's time and hold the oracle's state (Section 2 and Section 3
scheme, each problem with its own step size and end time; a problem that leaves the physical range
must stop where the oracle stops).  A batch with the learned flag is advanced one step per launch,
and the oracle is given the flags the batch used for that step and its own CFL step size (in
both modes: the persistent kernel and lockstep rounds).  Four
problems of the seeded 512-problem 1D set (their smallest meshes) run to the set's end time
T = 0.15 in one launch and end where the oracle's full runs end."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2304_09724_gb300 import flagnet as F
from paper_2304_09724_gb300 import shweno as S
from paper_2304_09724_gb300 import workloads as WL
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


def oracle_run(wl, T):
    """(state, steps, t, status) of the oracle's CFL run to T."""
    try:
        o, n, t = O.run(U.problem_of(wl), wl.state, T, wl.cfl)
        return o, n, t, S.OK
    except O.NonPhysical as e:
        return e.state, e.steps, e.t, S.E_NONPHYSICAL


def test_mixed_ragged_batch_equals_oracle():
    wls = [WL.random_riemann1d(s, nx=n) for s, n in zip(range(6), (40, 129, 300, 513, 77, 1000))]
    T = [0.01] * 6
    wls += [WL.riemann2d(n, WL.random_quadrants(s)) for s, n in zip((10, 11, 12), (24, 32, 40))]
    T += [0.01] * 3
    wls += [WL.burgers2d_riemann(36), WL.vortex(32), WL.burgers_sine(150)]
    T += [0.1, 0.3, 0.1]
    sols = []
    for wl in wls:
        s = U.solver_of(wl)
        s.set_state(wl.state)
        sols.append(s)
    b = S.Batch(sols)
    st, per = b.run(T, wls[0].cfl)
    assert st == S.OK
    got = [(s.get_state(), s.time()) for s in sols]
    b.close()
    for s in sols:
        s.close()
    for wl, tf, (g, (t, n)), status in zip(wls, T, got, per):
        o, n_o, t_o, st_o = oracle_run(wl, tf)
        what = f"{wl.name} {wl.nx}x{wl.ny}"
        assert status == st_o, what
        assert n == n_o, (what, n, n_o)
        assert t == pytest.approx(t_o, rel=1e-12, abs=1e-300), what
        U.check(g, o, U.fields(wl), shocked=True, what=what, wl=wl)


@pytest.mark.parametrize("mode", [S.BATCH_PERSISTENT, S.BATCH_LOCKSTEP])
def test_learned_batch_step_by_step_equals_oracle_given_its_flags(mode):
    import torch

    torch.cuda.set_device(0)
    params, thr = F.load()
    net = (torch.from_numpy(params).cuda(), thr)
    wls = [WL.riemann2d(n, WL.random_quadrants(s)) for s, n in zip((20, 21), (48, 36))]
    wls.append(WL.random_riemann1d(7, nx=150))
    sols = []
    for wl in wls:
        s = U.solver_of(wl, flag_mode=2 if wl.dim == 2 else 0)
        s.set_state(wl.state)
        if wl.dim == 2:
            S.shweno_set_flag_net(s.h, *net)
        sols.append(s)
    b = S.Batch(sols)
    b.set_mode(mode)
    orc = [{"P": U.problem_of(wl), "state": wl.state, "t": 0.0} for wl in wls]
    flagged = []
    for k in range(4):
        st, per = b.run([1.0] * len(wls), wls[0].cfl, max_steps=1)
        assert st == S.OK and all(p == S.OK for p in per)
        for wl, s, o in zip(wls, sols, orc):
            t, n = s.time()
            assert n == k + 1
            dt = wl.cfl / O.max_rate(o["P"], o["state"]["W"])
            assert t - o["t"] == pytest.approx(dt, rel=1e-11)
            flag = None
            if wl.dim == 2:
                flag = np.empty((wl.ny, wl.nx), dtype=np.uint8)
                S.shweno_get_flags(s.h, flag)
                flagged.append(flag.mean())
            o["state"] = O.step(o["P"], o["state"], dt, t=o["t"], flag=flag)
            o["t"] += dt
            U.check(s.get_state(), o["state"], U.fields(wl), shocked=True,
                    what=f"{wl.name} {wl.nx}x{wl.ny} step {k + 1}", wl=wl)
    b.close()
    for s in sols:
        s.close()
    # the flags are neither all on nor all off, so both kinds of cells were exercised
    assert 0.0 < min(flagged) and max(flagged) < 1.0


def test_1d_riemann_set_to_its_end_time_equals_oracle():
    small = sorted(range(512), key=lambda s: WL.random_riemann1d(s).nx)[:4]
    wls = [WL.random_riemann1d(s) for s in small]
    sols = []
    for wl in wls:
        s = U.solver_of(wl)
        s.set_state(wl.state)
        sols.append(s)
    b = S.Batch(sols)
    st, per = b.run(0.15, wls[0].cfl)
    got = [(s.get_state(), s.time()) for s in sols]
    b.close()
    for s in sols:
        s.close()
    for wl, (g, (t, n)), status in zip(wls, got, per):
        o, n_o, t_o, st_o = oracle_run(wl, 0.15)
        what = f"{wl.name} {wl.nx} cells to T = 0.15"
        assert status == st_o and n == n_o, (what, n, n_o)
        assert t == pytest.approx(t_o, rel=1e-12), what
        U.check(g, o, U.fields(wl), shocked=True, what=what, wl=wl)
