"""Parity at the largest configurations of the workloads, in the launch configuration the library
uses for them: the double Mach reflection at 4096 x 1024 with the learned flag (the oracle is
given the flags the library used), the largest four-quadrant problem (2048 x 2048), compared on
sampled cells that the oracle evaluates one by one, and the largest 1D Riemann problem of the
batch (16384 cells) over its first 40 steps."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2304_09724_gb300 import flagnet as F
from paper_2304_09724_gb300 import shweno as S
from paper_2304_09724_gb300 import workloads as WL
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


def sampled(g, cells):
    return {k: np.array([g[k][:, j, i] for (i, j) in cells]) for k in "WVYZ"}


def test_dmr_4096x1024_learned_sampled_cells():
    import torch

    torch.cuda.set_device(0)
    wl = WL.dmr(4096, 1024)
    params, thr = F.load()
    sol = U.solver_of(wl, flag_mode=2)
    sol.set_state({k: torch.from_numpy(np.array(v)).cuda() for k, v in wl.state.items()})
    S.shweno_set_flag_net(sol.h, torch.from_numpy(params).cuda(), thr)
    for _ in range(3):
        dt, _ = S.shweno_cfl_dt(sol.h, wl.cfl)
        sol.step(dt)
    before = sol.get_state()
    t3, _ = sol.time()
    dt, _ = S.shweno_cfl_dt(sol.h, wl.cfl)
    sol.step(dt)
    after = sol.get_state()
    flags = np.empty((1024, 4096), dtype=np.uint8)
    S.shweno_get_flags(sol.h, flags)
    sol.close()
    assert 0.0 < flags.mean() < 0.5
    rng = np.random.default_rng(3)
    foot = int(4096 / 4 / 6)  # the shock meets the wall at x = 1/6
    cells = [(0, 0), (4095, 0), (0, 1023), (4095, 1023), (foot, 0), (foot + 1, 0), (foot - 1, 1),
             (foot + 3, 5), (2000, 1023), (2100, 1022), (4095, 500)]
    cells += [tuple(int(x) for x in (rng.integers(0, 4096), rng.integers(0, 1024))) for _ in range(21)]
    o = O.step2d_cells(U.problem_of(wl), before, dt, cells, t=t3, flag=flags)
    U.check(sampled(after, cells), o, "WVYZ", shocked=True, what="DMR 4096x1024 learned", wl=wl)


def test_largest_quadrant_problem_sampled_cells():
    wl = WL.riemann2d(2048, WL.random_quadrants(5))
    sol = U.solver_of(wl)
    sol.set_state(wl.state)
    dt, _ = S.shweno_cfl_dt(sol.h, wl.cfl)
    sol.step(dt)
    g = sol.get_state()
    sol.close()
    rng = np.random.default_rng(4)
    cells = [(1023, 1023), (1024, 1024), (1023, 1024), (1024, 1023), (1022, 1025), (0, 0), (2047, 2047),
             (1024, 0), (0, 1024), (2047, 1023)]
    cells += [tuple(int(x) for x in rng.integers(0, 2048, size=2)) for _ in range(22)]
    o = O.step2d_cells(U.problem_of(wl), wl.state, dt, cells)
    U.check(sampled(g, cells), o, "WVYZ", shocked=True, what="quadrants 2048^2", wl=wl)


def test_largest_1d_riemann_problem_run():
    wl = WL.random_riemann1d(11, nx=16384)
    g, o, (t, n), (t_o, n_o) = U.run_both(wl, 0.0003)  # about 40 steps
    assert n == n_o and t == t_o
    U.check(g, o, U.fields(wl), shocked=True, what="1D Riemann 16384 cells", wl=wl)
