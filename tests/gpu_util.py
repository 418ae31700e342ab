"""Helpers of the GPU parity tests: run the same seeded inputs through the CUDA library (C ABI)
and through the oracle, and compare with the tolerances of the specification:
relative L-infinity <= 1e-10 on smooth runs, relative L1 <= 1e-9 on shocked runs.

The derivative averages are differences of interface values divided by the mesh size
(Eq. 2.11, 3.10): V and Y by dx or dy, Z by dx dy.  Two correct FP64 implementations that
round differently disagree in those interface values by a few ulp of |W|, which the division
amplifies; so V, Y and Z get an absolute floor of DERIV_ULP * max|W| / dx (/ dy, / (dx dy)) on
top of the relative tolerance.  W itself is held to the plain tolerance."""
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


DERIV_ULP = 1e-14


def deriv_floor(k, wmax, dx, dy):
    return {"W": 0.0, "V": DERIV_ULP * wmax / dx, "Y": DERIV_ULP * wmax / dy,
            "Z": DERIV_ULP * wmax / (dx * dy)}[k]


def check(g, o, keys, shocked, what="", wl=None):
    wmax = float(np.max(np.abs(o["W"])))
    if wl is not None:
        dx = (wl.domain[1] - wl.domain[0]) / wl.nx
        dy = (wl.domain[3] - wl.domain[2]) / wl.ny if wl.dim == 2 else 1.0
    for k in keys:
        floor = deriv_floor(k, wmax, dx, dy) if wl is not None else 0.0
        d = np.abs(g[k] - o[k])
        if shocked:
            err = float(np.sum(d) / (SHOCK_TOL * np.sum(np.abs(o[k])) + floor * d.size))
        else:
            err = float(np.max(d) / (SMOOTH_TOL * np.max(np.abs(o[k])) + floor))
        assert err <= 1.0, (f"{what} {k}: {'rel L1' if shocked else 'rel Linf'} "
                            f"{(rel_l1 if shocked else rel_linf)(g[k], o[k]):.3e} (ratio to tolerance {err:.2f})")


def steps_both(wl, dts, flag=None, flag_mode=0, linear=False, t0=0.0, charwise=False, quintic=False):
    """Fixed-dt steps on both sides; returns (gpu_state, oracle_state)."""
    sol = solver_of(wl, flag_mode=flag_mode, charwise=charwise, quintic=quintic)
    sol.set_state(wl.state, t0)
    if flag is not None:
        sol.set_flags(flag)
    for dt in dts:
        sol.step(dt)
    g = sol.get_state()
    sol.close()
    P = problem_of(wl, linear=linear, charwise=charwise, quintic=quintic)
    o = wl.state
    t = t0
    for dt in dts:
        o = O.step(P, o, dt, t=t, flag=flag)
        t += dt
    return g, o


def run_both(wl, t_final, flag=None, flag_mode=0, linear=False, charwise=False, quintic=False):
    sol = solver_of(wl, flag_mode=flag_mode, charwise=charwise, quintic=quintic)
    sol.set_state(wl.state)
    if flag is not None:
        sol.set_flags(flag)
    t, n = sol.run(t_final, wl.cfl)
    g = sol.get_state()
    sol.close()
    P = problem_of(wl, linear=linear, charwise=charwise, quintic=quintic)
    o, n_o, t_o = O.run(P, wl.state, t_final, wl.cfl, flag=flag)
    return g, o, (t, n), (t_o, n_o)
