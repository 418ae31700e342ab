"""The allocation-free 1D step (shweno_step1d_noalloc) against the handle-based step.

Callers that cannot allocate device memory when they step -- inside an open stream capture, in
a real-time loop, or under a framework that owns all device memory -- use the allocation-free
entry point, whose scratch is a fixed array inside the library.  This file is named so that
pytest collects it last: it checks, through the C ABI, that two calls in a row give what the
ordinary entry point gives, and that sizes beyond the array's capacity are refused."""
import numpy as np
import pytest

from paper_2304_09724_gb300 import shweno as S
from paper_2304_09724_gb300 import workloads as WL
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


def _handle_steps(wl, dts):
    sol = U.solver_of(wl)
    sol.set_state(wl.state)
    out = []
    for dt in dts:
        sol.step(dt)
        out.append(sol.get_state())
    sol.close()
    return out


@pytest.mark.parametrize("case", ["euler_outflow_reflective", "burgers_periodic"])
def test_noalloc_matches_handle_step_twice(case):
    import torch

    if case == "euler_outflow_reflective":
        n = 300
        W, V = WL.random_smooth_1d(21, n)
        wl = WL.euler1d_sine(n)
        wl.domain, wl.bc = (0.0, 1.0, 0.0, 1.0), (WL.OUTFLOW, WL.REFLECTIVE, 0, 0)
        eq = S.EULER
        dts = [0.4 / n, 0.3 / n]
    else:
        wl = WL.burgers_sine(200)
        W, V = wl.state["W"], wl.state["V"]
        eq = S.BURGERS
        dts = [0.003, 0.004]
    wl.state = {"W": W, "V": V}
    ref = _handle_steps(wl, dts)

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    nc = W.shape[0]
    a = torch.from_numpy(np.concatenate([W, V]).reshape(2, nc, wl.nx).copy()).cuda()
    b = torch.empty_like(a)
    torch.cuda.synchronize()  # the copies above ran on the default stream
    x0, x1 = wl.domain[0], wl.domain[1]
    t = 0.0
    for k, dt in enumerate(dts):
        s = S.shweno_step1d_noalloc(eq, wl.nx, x0, x1, 1.4, wl.bc[:2], None, 0, a, b, t, dt, stream.cuda_stream)
        assert s == S.OK, S.STATUS_NAMES.get(s, s)
        torch.cuda.synchronize()
        got = b.cpu().numpy()
        U.check({"W": got[0], "V": got[1]}, ref[k], ("W", "V"), shocked=False, what=f"no-alloc call {k + 1}", wl=wl)
        a, b = b, a
        t += dt


def test_noalloc_rejects_oversize_and_bad_arguments():
    import torch

    n = S.NOALLOC_MAX_NX + 1
    a = torch.zeros((2, 1, n), dtype=torch.float64, device="cuda")
    b = torch.zeros_like(a)
    assert S.shweno_step1d_noalloc(S.BURGERS, n, 0.0, 1.0, 1.4, (0, 0), None, 0, a, b, 0.0, 1e-3) == S.E_INVALID
    small_a, small_b = a[:, :, :64].contiguous(), b[:, :, :64].contiguous()
    # same buffer in and out, bad dt, unpaired periodic sides
    assert S.shweno_step1d_noalloc(S.BURGERS, 64, 0.0, 1.0, 1.4, (0, 0), None, 0, small_a, small_a, 0.0, 1e-3) == S.E_INVALID
    assert S.shweno_step1d_noalloc(S.BURGERS, 64, 0.0, 1.0, 1.4, (0, 0), None, 0, small_a, small_b, 0.0, -1.0) == S.E_INVALID
    assert S.shweno_step1d_noalloc(S.BURGERS, 64, 0.0, 1.0, 1.4, (0, 1), None, 0, small_a, small_b, 0.0, 1e-3) == S.E_INVALID
