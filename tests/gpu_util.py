"""Helpers of the GPU parity tests: run the same seeded inputs through the CUDA library (C ABI)
and through the oracle, and compare with the tolerances of the specification:
relative L-infinity <= 1e-10 on smooth runs, relative L1 <= 1e-9 on shocked runs."""
import numpy as np

from oracle import oracle as O
from paper_2304_09724_gb300 import shweno as S

SMOOTH_TOL = 1e-10   # rel Linf = max|g - o| / max|o|
SHOCK_TOL = 1e-9     # rel L1 = sum|g - o| / sum|o|


def rel_linf(g, o):
    return float(np.max(np.abs(g - o)) / max(np.max(np.abs(o)), 1e-300))


def rel_l1(g, o):
    return float(np.sum(np.abs(g - o)) / max(np.sum(np.abs(o)), 1e-300))


def solver_of(wl, flag_mode=0, **kw):
    return S.Solver(wl.dim, wl.eq, wl.nx, wl.ny, wl.domain, wl.bc, inflow=wl.inflow, flag_mode=flag_mode, **kw)


def problem_of(wl, **kw):
    return O.make_problem(wl.dim, wl.eq, wl.nx, wl.ny, *wl.domain, bc=wl.bc, inflow=wl.inflow, **kw)


def fields(wl):
    return ("W", "V") if wl.dim == 1 else ("W", "V", "Y", "Z")


def check(g, o, keys, shocked, what=""):
    for k in keys:
        err = rel_l1(g[k], o[k]) if shocked else rel_linf(g[k], o[k])
        tol = SHOCK_TOL if shocked else SMOOTH_TOL
        assert err <= tol, f"{what} {k}: {'rel L1' if shocked else 'rel Linf'} {err:.3e} > {tol:.0e}"


def steps_both(wl, dts, flag=None, flag_mode=0, linear=False, t0=0.0):
    """Fixed-dt steps on both sides; returns (gpu_state, oracle_state)."""
    sol = solver_of(wl, flag_mode=flag_mode)
    sol.set_state(wl.state, t0)
    if flag is not None:
        sol.set_flags(flag)
    for dt in dts:
        sol.step(dt)
    g = sol.get_state()
    sol.close()
    P = problem_of(wl, linear=linear)
    o = wl.state
    t = t0
    for dt in dts:
        o = O.step(P, o, dt, t=t, flag=flag)
        t += dt
    return g, o


def run_both(wl, t_final, flag=None, flag_mode=0, linear=False):
    sol = solver_of(wl, flag_mode=flag_mode)
    sol.set_state(wl.state)
    if flag is not None:
        sol.set_flags(flag)
    t, n = sol.run(t_final, wl.cfl)
    g = sol.get_state()
    sol.close()
    P = problem_of(wl, linear=linear)
    o, n_o, t_o = O.run(P, wl.state, t_final, wl.cfl, flag=flag)
    return g, o, (t, n), (t_o, n_o)
