"""Batched launches: many uneven problems in one persistent kernel, or in lockstep rounds of one
launch per phase, give what each handle gives on its own (same status, same step count, states
equal to round-off: the same device functions are inlined into different kernels, whose FMA
contraction may differ by an ulp), 1D, 2D, mixed and with the learned flag; the two modes agree
with each other; the autotuner leaves the states untouched; a device-side wait that runs out is
reported as TIMEOUT and leaves every handle usable."""
import numpy as np
import pytest

from paper_2304_09724_gb300 import shweno as S
from paper_2304_09724_gb300 import workloads as WL
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


def solo(wl, T, flag_net=None, max_steps=0):
    """(state, (t, steps), status) of the handle run on its own."""
    s = U.solver_of(wl, flag_mode=2 if flag_net else 0)
    s.set_state(wl.state)
    if flag_net:
        S.shweno_set_flag_net(s.h, *flag_net)
    status = S.OK
    try:
        if max_steps:
            S.shweno_advance(s.h, max_steps, wl.cfl)
            S.shweno_sync(s.h)
        else:
            s.run(T, wl.cfl)
    except S.ShwenoError as e:
        status = e.status
    out = s.get_state(), s.time(), status
    s.close()
    return out


def batch_of(wls, T, flag_net=None, max_steps=0, tile1d=0, mode=None):
    sols = []
    for wl in wls:
        s = U.solver_of(wl, flag_mode=2 if flag_net and wl.dim == 2 else 0)
        s.set_state(wl.state)
        if flag_net and wl.dim == 2:
            S.shweno_set_flag_net(s.h, *flag_net)
        sols.append(s)
    b = S.Batch(sols)
    if tile1d:
        b.set(tile1d=tile1d)
    if mode is not None:
        b.set_mode(mode)
    st, per = b.run([T] * len(wls) if np.isscalar(T) else T, wls[0].cfl, max_steps=max_steps)
    outs = [(s.get_state(), s.time()) for s in sols]
    b.close()
    for s in sols:
        s.close()
    return outs, per


def same(a, b, wl, status=None):
    """a: (state, (t, steps)) from the batch; b: solo (state, (t, steps), status)."""
    if status is not None:
        assert status == b[2]
    assert a[1][1] == b[1][1]
    assert a[1][0] == pytest.approx(b[1][0], rel=1e-12, abs=1e-300)
    U.check(a[0], b[0], U.fields(wl), shocked=True, what=wl.name, wl=wl)


@pytest.mark.parametrize("tile1d", [128, 512])
def test_batch_1d_ragged_equals_solo(tile1d):
    wls = [WL.random_riemann1d(s, nx=n) for s, n in zip(range(6), (40, 129, 300, 513, 77, 1000))]
    outs, per = batch_of(wls, 0.03, tile1d=tile1d)
    for wl, o, st in zip(wls, outs, per):
        same(o, solo(wl, 0.03), wl, st)


@pytest.mark.parametrize("mode", [S.BATCH_PERSISTENT, S.BATCH_LOCKSTEP])
def test_batch_2d_and_mixed_equals_solo(mode):
    wls = [WL.riemann2d(n, WL.random_quadrants(s)) for s, n in zip((10, 11, 12), (24, 40, 70))]
    wls.append(WL.vortex(32))
    wls.append(WL.random_riemann1d(3, nx=200))
    wls.append(WL.burgers2d_riemann(36))
    wls.append(WL.burgers_sine(150))
    T = [0.02, 0.02, 0.02, 0.3, 0.02, 0.1, 0.1]
    outs, per = batch_of(wls, T, mode=mode)
    for wl, t, o, st in zip(wls, T, outs, per):
        same(o, solo(wl, t), wl, st)


@pytest.mark.parametrize("mode", [S.BATCH_PERSISTENT, S.BATCH_LOCKSTEP])
def test_batch_learned_flag_equals_solo(mode):
    import torch

    from paper_2304_09724_gb300 import flagnet as F

    params, thr = F.load()
    net = (torch.from_numpy(params).cuda(), thr)
    wls = [WL.riemann2d(n, WL.random_quadrants(s)) for s, n in zip((20, 21), (48, 36))]
    outs, per = batch_of(wls, 0.02, flag_net=net, mode=mode)
    for wl, o, st in zip(wls, outs, per):
        same(o, solo(wl, 0.02, flag_net=net), wl, st)


@pytest.mark.parametrize("mode", [S.BATCH_PERSISTENT, S.BATCH_LOCKSTEP])
def test_batch_max_steps_and_nonphysical_problem_stops_alone(mode):
    good = WL.random_riemann1d(4, nx=120)
    bad = WL.random_riemann1d(5, nx=64)
    bad.state["W"][2, 10] = -1.0  # negative energy: non-physical from the start
    outs, per = batch_of([good, bad], 0.05, max_steps=7, mode=mode)
    assert per[0] == S.OK and per[1] == S.E_NONPHYSICAL
    assert outs[0][1][1] == 7
    same(outs[0], solo(good, 0.05, max_steps=7), good, per[0])
    assert outs[1][1] == (0.0, 0)


def test_autotune_keeps_states():
    wls = [WL.random_riemann1d(s, nx=n) for s, n in zip(range(30, 34), (100, 300, 700, 1500))]
    sols = []
    for wl in wls:
        s = U.solver_of(wl)
        s.set_state(wl.state)
        sols.append(s)
    b = S.Batch(sols)
    tile, occ = b.autotune(0.05, wls[0].cfl, trial_steps=3)
    assert tile in (128, 256, 512, 1024) and occ in (1, 2)
    for wl, s in zip(wls, sols):
        g = s.get_state()
        assert np.array_equal(g["W"], wl.state["W"]) and s.time() == (0.0, 0)
    st, per = b.run(0.02, wls[0].cfl)
    for wl, s, pst in zip(wls, sols, per):
        same((s.get_state(), s.time()), solo(wl, 0.02), wl, pst)
    b.close()
    for s in sols:
        s.close()


def test_wait_that_runs_out_reports_timeout_and_handles_stay_usable():
    wls = [WL.random_riemann1d(s, nx=300) for s in range(40, 44)]
    sols = []
    for wl in wls:
        s = U.solver_of(wl)
        s.set_state(wl.state)
        sols.append(s)
    b = S.Batch(sols)
    b.set(spin_limit=1)  # every CTA that finds the queue empty gives up at once
    st, per = b.run(0.05, wls[0].cfl, check=False)
    assert st == S.E_TIMEOUT
    b.close()
    # the committed state of every handle is consistent: continuing alone reaches the same result
    for wl, s in zip(wls, sols):
        try:
            s.run(0.05, wl.cfl)
            status = S.OK
        except S.ShwenoError as e:
            status = e.status
        same((s.get_state(), s.time()), solo(wl, 0.05), wl, status)
        s.close()


def test_1d_only_batch_runs_up_to_four_ctas_per_sm():
    """A batch of 1D problems runs the lighter 1D-only kernel: 3 and 4 CTAs per SM give what the
    handles give on their own; a batch with a 2D problem refuses more than 2."""
    wls = [WL.random_riemann1d(s, nx=n) for s, n in zip(range(40, 44), (300, 1000, 77, 2048))]
    for occ in (3, 4):
        sols = []
        for wl in wls:
            s = U.solver_of(wl)
            s.set_state(wl.state)
            sols.append(s)
        b = S.Batch(sols)
        b.set(ctas_per_sm=occ)
        st, per = b.run([0.03] * len(wls), wls[0].cfl)
        outs = [(s.get_state(), s.time()) for s in sols]
        b.close()
        for s in sols:
            s.close()
        for wl, o, p in zip(wls, outs, per):
            same(o, solo(wl, 0.03), wl, p)
    wl2 = WL.riemann2d(16, WL.LAX_LIU_SHOCKS)
    s2 = U.solver_of(wl2)
    s2.set_state(wl2.state)
    b = S.Batch([s2])
    with pytest.raises(S.ShwenoError) as e:
        b.set(ctas_per_sm=3)
    assert e.value.status == S.E_INVALID
    b.close()
    s2.close()


def test_lockstep_and_persistent_modes_agree():
    """The same mixed batch (1D and 2D Euler, 2D Burgers, learned-flag 2D problems, one problem
    that turns non-physical, uneven end times) in both modes: the same statuses, step counts and
    times, states equal to round-off; the default mode is lockstep for a batch of 2D problems only
    and persistent otherwise; the autotuner has nothing to tune for a lockstep batch of 2D
    problems; an unknown mode is refused."""
    import torch

    from paper_2304_09724_gb300 import flagnet as F

    params, thr = F.load()
    net = (torch.from_numpy(params).cuda(), thr)
    wls = [WL.riemann2d(n, WL.random_quadrants(s)) for s, n in zip((30, 31), (40, 56))]
    wls += [WL.random_riemann1d(6, nx=333), WL.burgers2d_riemann(28), WL.vortex(24)]
    bad = WL.random_riemann1d(8, nx=90)
    bad.state["W"][0, 40] = -0.5  # negative density: non-physical from the start
    wls.append(bad)
    T = [0.03, 0.02, 0.04, 0.1, 0.2, 0.05]
    runs = {}
    for mode in (S.BATCH_PERSISTENT, S.BATCH_LOCKSTEP):
        sols = []
        for k, wl in enumerate(wls):
            learned = wl.dim == 2 and k < 2
            s = U.solver_of(wl, flag_mode=2 if learned else 0)
            s.set_state(wl.state)
            if learned:
                S.shweno_set_flag_net(s.h, *net)
            sols.append(s)
        b = S.Batch(sols)
        assert b.mode == S.BATCH_PERSISTENT  # a 1D problem is in the batch
        b.set_mode(mode)
        assert b.mode == mode
        st, per = b.run(T, wls[0].cfl)
        runs[mode] = ([(s.get_state(), s.time()) for s in sols], per)
        b.close()
        for s in sols:
            s.close()
    (a, pa), (c, pc) = runs[S.BATCH_PERSISTENT], runs[S.BATCH_LOCKSTEP]
    assert pa == pc and pa[-1] == S.E_NONPHYSICAL and all(p == S.OK for p in pa[:-1])
    for wl, x, y in zip(wls, a, c):
        assert x[1][1] == y[1][1] and x[1][0] == pytest.approx(y[1][0], rel=1e-13, abs=1e-300)
        U.check(y[0], x[0], U.fields(wl), shocked=True, what=wl.name, wl=wl)
    # mode resolution and validation
    only2d = [U.solver_of(wl) for wl in wls if wl.dim == 2]
    for s, wl in zip(only2d, [w for w in wls if w.dim == 2]):
        s.set_state(wl.state)
    b = S.Batch(only2d)
    assert b.mode == S.BATCH_LOCKSTEP
    # nothing to tune in lockstep rounds of 2D problems: the current shape comes back, nothing runs
    assert b.autotune(0.01, wls[0].cfl) == (512, 2)
    assert all(s.time() == (0.0, 0) for s in only2d)
    b.set_mode(S.BATCH_PERSISTENT)
    assert b.mode == S.BATCH_PERSISTENT
    with pytest.raises(S.ShwenoError) as e:
        b.set_mode(7)
    assert e.value.status == S.E_INVALID
    b.close()
    for s in only2d:
        s.close()
