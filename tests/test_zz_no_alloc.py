"""The allocation-free 1D step (shweno_step1d_noalloc) against the handle-based step and the oracle.

Callers that cannot allocate device memory when they step -- a real-time loop that cannot take an
allocation's latency or the synchronisation that freeing memory implies, or a framework that owns
all device memory through its own pool -- use the allocation-free entry point, whose scratch is a
fixed array inside the library.  This file is named so that pytest collects it last: it checks,
through the C ABI, that two calls in a row give what the ordinary entry point (a handle and
shweno_step) gives and what the oracle gives, at ordinary sizes and at the array's maximum size,
with the nonlinear and with the linear weights; that a call leaves the device's memory use as it
was; and that sizes beyond the array's capacity and other bad arguments are refused."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2304_09724_gb300 import shweno as S
from paper_2304_09724_gb300 import workloads as WL
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


def _case(name):
    """(workload, equation, the two step sizes)."""
    if name.startswith("euler"):
        n = S.NOALLOC_MAX_NX if name.endswith("max") else 300
        W, V = WL.random_smooth_1d(21, n)
        wl = WL.euler1d_sine(n)
        bc = (WL.OUTFLOW, WL.REFLECTIVE, 0, 0) if "outflow" in name else (WL.PERIODIC,) * 4
        wl.domain, wl.bc = (0.0, 1.0, 0.0, 1.0), bc
        wl.state = {"W": W, "V": V}
        return wl, S.EULER, [0.4 / n, 0.3 / n]
    n = S.NOALLOC_MAX_NX if name.endswith("max") else 200
    wl = WL.burgers_sine(n)
    return wl, S.BURGERS, [0.6 / n, 0.8 / n]


def _handle_steps(wl, dts, flag_mode):
    sol = U.solver_of(wl, flag_mode=flag_mode)
    sol.set_state(wl.state)
    out = []
    for dt in dts:
        sol.step(dt)
        out.append(sol.get_state())
    sol.close()
    return out


def _oracle_steps(wl, dts, flag_mode):
    P = U.problem_of(wl, linear=flag_mode == 1)
    o, t, out = wl.state, 0.0, []
    for dt in dts:
        o = O.step(P, o, dt, t=t)
        out.append(o)
        t += dt
    return out


@pytest.mark.parametrize("flag_mode", [0, 1])
@pytest.mark.parametrize("case", ["euler_outflow_reflective", "burgers_periodic", "euler_periodic_max",
                                  "burgers_periodic_max"])
def test_noalloc_matches_handle_step_and_oracle_twice(case, flag_mode):
    import torch

    wl, eq, dts = _case(case)
    ref = _handle_steps(wl, dts, flag_mode)
    orc = _oracle_steps(wl, dts, flag_mode)

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    W, V = wl.state["W"], wl.state["V"]
    nc = W.shape[0]
    a = torch.from_numpy(np.concatenate([W, V]).reshape(2, nc, wl.nx).copy()).cuda()
    b = torch.empty_like(a)
    torch.cuda.synchronize()  # the copies above ran on the default stream
    x0, x1 = wl.domain[0], wl.domain[1]
    t = 0.0
    for k, dt in enumerate(dts):
        if k == 1:  # the second call allocates nothing: device memory use is unchanged across it
            torch.cuda.synchronize()
            alloc0, free0 = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]
        s = S.shweno_step1d_noalloc(eq, wl.nx, x0, x1, 1.4, wl.bc[:2], None, flag_mode, a, b, t, dt,
                                    stream.cuda_stream)
        assert s == S.OK, S.STATUS_NAMES.get(s, s)
        torch.cuda.synchronize()
        if k == 1:
            assert torch.cuda.memory_allocated() == alloc0
            assert torch.cuda.mem_get_info()[0] == free0
        got = b.cpu().numpy()
        g = {"W": got[0], "V": got[1]}
        U.check(g, ref[k], ("W", "V"), shocked=False, what=f"no-alloc call {k + 1} vs shweno_step", wl=wl)
        U.check(g, orc[k], ("W", "V"), shocked=False, what=f"no-alloc call {k + 1} vs oracle", wl=wl)
        a, b = b, a
        t += dt


def test_noalloc_inflow_side():
    """An INFLOW side with its imposed state gives what the handle and the oracle give."""
    import torch

    n = 256
    W, V = WL.random_smooth_1d(22, n)
    inflow = [[1.0, 0.5, 2.5, 0.0], [0.0] * 4, [0.0] * 4, [0.0] * 4]
    wl = WL.euler1d_sine(n)
    wl.domain, wl.bc, wl.inflow, wl.state = (0.0, 1.0, 0.0, 1.0), (WL.INFLOW, WL.OUTFLOW, 0, 0), inflow, {"W": W, "V": V}
    dt = 0.3 / n
    ref = _handle_steps(wl, [dt], 0)[0]
    orc = _oracle_steps(wl, [dt], 0)[0]
    a = torch.from_numpy(np.concatenate([W, V]).reshape(2, 3, n).copy()).cuda()
    b = torch.empty_like(a)
    torch.cuda.synchronize()
    s = S.shweno_step1d_noalloc(S.EULER, n, 0.0, 1.0, 1.4, wl.bc[:2], inflow[:2], 0, a, b, 0.0, dt)
    assert s == S.OK
    got = b.cpu().numpy()
    g = {"W": got[0], "V": got[1]}
    U.check(g, ref, ("W", "V"), shocked=False, what="inflow vs shweno_step", wl=wl)
    U.check(g, orc, ("W", "V"), shocked=False, what="inflow vs oracle", wl=wl)


def test_noalloc_rejects_oversize_and_bad_arguments():
    import torch

    n = S.NOALLOC_MAX_NX + 1
    a = torch.zeros((2, 1, n), dtype=torch.float64, device="cuda")
    b = torch.zeros_like(a)
    assert S.shweno_step1d_noalloc(S.BURGERS, n, 0.0, 1.0, 1.4, (0, 0), None, 0, a, b, 0.0, 1e-3) == S.E_INVALID
    small_a, small_b = a[:, :, :64].contiguous(), b[:, :, :64].contiguous()
    # same buffer in and out, bad dt, unpaired periodic sides, an INFLOW side without its state,
    # a flag mode other than 0 or 1
    assert S.shweno_step1d_noalloc(S.BURGERS, 64, 0.0, 1.0, 1.4, (0, 0), None, 0, small_a, small_a, 0.0, 1e-3) == S.E_INVALID
    assert S.shweno_step1d_noalloc(S.BURGERS, 64, 0.0, 1.0, 1.4, (0, 0), None, 0, small_a, small_b, 0.0, -1.0) == S.E_INVALID
    assert S.shweno_step1d_noalloc(S.BURGERS, 64, 0.0, 1.0, 1.4, (0, 1), None, 0, small_a, small_b, 0.0, 1e-3) == S.E_INVALID
    assert S.shweno_step1d_noalloc(S.BURGERS, 64, 0.0, 1.0, 1.4, (3, 1), None, 0, small_a, small_b, 0.0, 1e-3) == S.E_INVALID
    assert S.shweno_step1d_noalloc(S.BURGERS, 64, 0.0, 1.0, 1.4, (1, 3), None, 0, small_a, small_b, 0.0, 1e-3) == S.E_INVALID
    assert S.shweno_step1d_noalloc(S.BURGERS, 64, 0.0, 1.0, 1.4, (0, 0), None, 2, small_a, small_b, 0.0, 1e-3) == S.E_INVALID
