"""Parity at the largest sizes: the 1D mesh of 2^26 cells (the largest the C ABI accepts) and a
2D mesh of 8192 x 8192 cells (67 M cells; about 105 GB of state, copies and step scratch).

The oracle cannot step such meshes, so the check goes through a property that holds at any
size: the scheme is translation invariant, so a periodic state made of R copies of a small
periodic state is advanced to R copies of the small state's result.  The mesh widths are powers
of two, equal on the small and the large mesh, so both see the same dx and dt bit for bit.  Every
cell of the large result is compared, on the device, with the oracle's step of the small mesh."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2304_09724_gb300 import shweno as S
from paper_2304_09724_gb300 import workloads as WL
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


def _compare_tiled(g, o, reps_shape):
    """g: device tensor [nc][*big] made of copies of o's shape; o: numpy [nc][*small].  Returns
    (max |g - o| over every copy, max difference between a copy and the first one)."""
    import torch

    nc = o.shape[0]
    ot = torch.from_numpy(np.ascontiguousarray(o)).cuda()
    if o.ndim == 2:  # 1D: [nc][reps][n]
        d = (g.view(nc, reps_shape[0], o.shape[1]) - ot[:, None, :]).abs()
        spread = (g.view(nc, reps_shape[0], o.shape[1]) - g.view(nc, reps_shape[0], o.shape[1])[:, :1, :]).abs()
    else:  # 2D: [nc][ry][ny][rx][nx]
        ry, rx = reps_shape
        gv = g.view(nc, ry, o.shape[1], rx, o.shape[2])
        d = (gv - ot[:, None, :, None, :]).abs()
        spread = (gv - gv[:, :1, :, :1, :]).abs()
    return float(d.max()), float(spread.max())


def _check(errs, o_state, dx, dy, what):
    wmax = float(np.max(np.abs(o_state["W"])))
    for k, (err, spread) in errs.items():
        scale = U.SMOOTH_TOL * float(np.max(np.abs(o_state[k]))) + U.deriv_floor(k, wmax, dx, dy)
        assert err <= scale, f"{what} {k}: max |gpu - oracle| {err:.3e} > {scale:.3e}"
        # every copy is advanced alike (the step has no position-dependent arithmetic)
        assert spread <= 1e-3 * scale, f"{what} {k}: copies differ by {spread:.3e}"


def test_1d_euler_at_the_largest_mesh():
    import torch

    torch.cuda.set_device(0)
    n, reps = 256, 1 << 18  # 2^26 cells on (0, 2^18): dx = 2^-8 as on (0, 1) with 256 cells
    W, V = WL.random_smooth_1d(7, n)
    small = {"W": W, "V": V}
    P = O.make_problem(1, O.EQ_EULER, n, x0=0.0, x1=1.0)
    dt = 0.6 / O.max_rate(P, W)
    o = small
    for _ in range(2):
        o = O.step(P, o, dt)
    nx = n * reps
    sol = S.Solver(1, S.EULER, nx, domain=(0.0, float(reps), 0.0, 1.0), bc=(0, 0))
    dev = {k: torch.from_numpy(v).cuda().repeat(1, reps) for k, v in small.items()}
    sol.set_state(dev)
    del dev
    for _ in range(2):
        sol.step(dt)
    g = {k: torch.empty((3, nx), dtype=torch.float64, device="cuda") for k in "WV"}
    S.shweno_get_state(sol.h, g["W"], g["V"], None, None)
    sol.close()
    errs = {k: _compare_tiled(g[k], o[k], (reps,)) for k in "WV"}
    _check(errs, o, 1.0 / n, 1.0, f"1D Euler nx = {nx}")


def test_2d_euler_8192_squared():
    import torch

    torch.cuda.set_device(0)
    n, reps = 128, 64  # 8192^2 cells on (0, 640)^2: dx = 10/128 as for the vortex at 128^2
    wl = WL.vortex(n)
    P = U.problem_of(wl)
    dt = 0.6 / O.max_rate(P, wl.state["W"])
    o = wl.state
    for _ in range(2):
        o = O.step(P, o, dt)
    N = n * reps
    L = 10.0 * reps
    sol = S.Solver(2, S.EULER, N, N, (0.0, L, 0.0, L), (0, 0, 0, 0))
    dev = {k: torch.from_numpy(v).cuda().repeat(1, reps, reps) for k, v in wl.state.items()}
    sol.set_state(dev)
    del dev
    for _ in range(2):
        sol.step(dt)
    g = {k: torch.empty((4, N, N), dtype=torch.float64, device="cuda") for k in "WVYZ"}
    S.shweno_get_state(sol.h, g["W"], g["V"], g["Y"], g["Z"])
    sol.close()
    dx = 10.0 / n
    errs = {}
    for k in "WVYZ":
        errs[k] = _compare_tiled(g[k], o[k], (reps, reps))
        del g[k]
    _check(errs, o, dx, dx, f"2D Euler {N}^2")
