"""Seeded synthetic inputs: initial cell averages and derivative averages of the paper's test
problems, plus exact solutions where the paper states them.

This module holds none of the scheme's arithmetic.  It only projects analytic initial data onto
the mesh (Section 2 and Eq. 3.9 define the averages W, V = avg W_x, Y = avg W_y, Z = avg W_xy)
and is the one module that both the CUDA library's tests/benchmark and the oracle's tests read
inputs from.  Arrays are float64, component-major: [comp][nx] in 1D, [comp][ny][nx] in 2D.

Averages of derivatives are computed from their exact definition: the x-derivative average of a
cell is the difference of the values on its right and left edges (taken as limits from inside
the cell) divided by dx, averaged along the edge; the xy-average is the corner combination.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = 1.4
BURGERS, EULER = 0, 1
PERIODIC, OUTFLOW, REFLECTIVE, INFLOW, DMR_BOTTOM, DMR_TOP = range(6)


@dataclass
class Workload:
    name: str
    dim: int
    eq: int
    nx: int
    ny: int
    domain: tuple  # (x0, x1, y0, y1)
    bc: tuple      # (xlo, xhi, ylo, yhi)
    t_final: float
    cfl: float
    state: dict    # W, V (, Y, Z)
    inflow: list = field(default_factory=lambda: [[0.0] * 4 for _ in range(4)])
    exact: object = None  # callable(t) -> exact cell averages of W, or None
    shocked: bool = False

    @property
    def ncomp(self):
        return 1 if self.eq == BURGERS else (3 if self.dim == 1 else 4)

    @property
    def cells(self):
        return self.nx * (self.ny if self.dim == 2 else 1)


def _gauss(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * x, 0.5 * w  # on [-1/2, 1/2], weights summing to 1


def euler_conserved(rho, u, p, v=None, gamma=GAMMA):
    if v is None:
        return np.stack([rho, rho * u, p / (gamma - 1.0) + 0.5 * rho * u * u])
    return np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])


# --------------------------------------------------------------------------- projections
def project_1d(fun, x0, x1, nx, nq=6, eps_edge=0.0):
    """Cell averages (nq-point Gauss) and derivative averages of fun(x) -> [nc, ...]."""
    dx = (x1 - x0) / nx
    xc = x0 + (np.arange(nx) + 0.5) * dx
    s, w = _gauss(nq)
    W = sum(wk * fun(xc + sk * dx) for sk, wk in zip(s, w))
    e = eps_edge * dx
    V = (fun(xc + 0.5 * dx - e) - fun(xc - 0.5 * dx + e)) / dx
    return np.ascontiguousarray(W), np.ascontiguousarray(V)


def project_pieces_1d(pieces, x0, x1, nx, nq=6):
    """Cell and derivative averages of piecewise-smooth data: pieces = [(a, b, fun)] covering
    [x0, x1] in order.  Each cell's average integrates every piece over its part of the cell
    (nq-point Gauss on that part), so a jump inside a cell is exact; an edge value is the limit
    from inside the cell."""
    dx = (x1 - x0) / nx
    xl = x0 + np.arange(nx) * dx
    xr = xl + dx
    s, w = _gauss(nq)
    W = 0.0
    for a, b, f in pieces:
        lo, hi = np.maximum(xl, a), np.minimum(xr, b)
        ln = np.maximum(hi - lo, 0.0)
        mid = 0.5 * (lo + hi)
        W = W + sum(wk * f(mid + sk * ln) for sk, wk in zip(s, w)) * (ln / dx)
    right_edge = 0.0
    left_edge = 0.0
    for a, b, f in pieces:
        right_edge = right_edge + np.where((a < xr) & (xr <= b), f(xr), 0.0)
        left_edge = left_edge + np.where((a <= xl) & (xl < b), f(xl), 0.0)
    V = (right_edge - left_edge) / dx
    return np.ascontiguousarray(W), np.ascontiguousarray(V)


def _prim_piece(rho, u, p):
    """fun(x) -> conserved (rho, rho u, E) of primitive data given as numbers or callables."""
    def f(x):
        ev = lambda v: v(x) if callable(v) else np.full_like(x, v, dtype=np.float64)
        return euler_conserved(ev(rho), ev(u), ev(p))
    return f


def shu_osher(nx=400, t_final=1.8, cfl=0.6):
    """Example 5.4: a Mach 3 shock meeting the density wave 1 + 0.2 sin(5x) on (-5, 5),
    inflow/outflow sides (the states at the ends do not change before T)."""
    pieces = [(-5.0, -4.0, _prim_piece(3.857143, 2.629369, 10.333333)),
              (-4.0, 5.0, _prim_piece(lambda x: 1.0 + 0.2 * np.sin(5.0 * x), 0.0, 1.0))]
    W, V = project_pieces_1d(pieces, -5.0, 5.0, nx)
    return Workload("shu_osher", 1, EULER, nx, 1, (-5.0, 5.0, 0.0, 1.0), (OUTFLOW, OUTFLOW, 0, 0),
                    t_final, cfl, {"W": W, "V": V}, shocked=True)


def turbulence_interaction(nx=1500, t_final=5.0, cfl=0.6):
    """Example 5.5: a shock meeting the density wave 1 + 0.1 sin(20 pi x) on (-5, 5)."""
    pieces = [(-5.0, -4.5, _prim_piece(1.515695, 0.523346, 1.80500)),
              (-4.5, 5.0, _prim_piece(lambda x: 1.0 + 0.1 * np.sin(20.0 * np.pi * x), 0.0, 1.0))]
    W, V = project_pieces_1d(pieces, -5.0, 5.0, nx)
    return Workload("turbulence_interaction", 1, EULER, nx, 1, (-5.0, 5.0, 0.0, 1.0),
                    (OUTFLOW, OUTFLOW, 0, 0), t_final, cfl, {"W": W, "V": V}, shocked=True)


def blast_waves(nx=800, t_final=0.038, cfl=0.6):
    """Example 5.6 (Woodward-Colella): pressures 1000 / 0.01 / 100 split at 0.1 and 0.9 on
    (0, 1), rho = 1, u = 0, reflective walls at both ends."""
    pieces = [(0.0, 0.1, _prim_piece(1.0, 0.0, 1000.0)), (0.1, 0.9, _prim_piece(1.0, 0.0, 0.01)),
              (0.9, 1.0, _prim_piece(1.0, 0.0, 100.0))]
    W, V = project_pieces_1d(pieces, 0.0, 1.0, nx)
    return Workload("blast_waves", 1, EULER, nx, 1, (0.0, 1.0, 0.0, 1.0), (REFLECTIVE, REFLECTIVE, 0, 0),
                    t_final, cfl, {"W": W, "V": V}, shocked=True)


def project_2d(fun, x0, x1, y0, y1, nx, ny, nq=6, eps_edge=0.0):
    """W, V, Y, Z of fun(x, y) -> [nc, ...] by nq-point Gauss rules (tensor rule for W, edge rule
    for V and Y, corners for Z).  eps_edge > 0 takes edge values just inside the cell, which is
    the limit from inside for piecewise-constant data."""
    dx, dy = (x1 - x0) / nx, (y1 - y0) / ny
    # broadcastable coordinates ([1, nx] and [ny, 1]): separable functions stay cheap
    X = (x0 + (np.arange(nx) + 0.5) * dx)[None, :]
    Yg = (y0 + (np.arange(ny) + 0.5) * dy)[:, None]
    s, w = _gauss(nq)
    W = 0.0
    for sa, wa in zip(s, w):
        for sb, wb in zip(s, w):
            W = W + wa * wb * fun(X + sa * dx, Yg + sb * dy)
    ex, ey = eps_edge * dx, eps_edge * dy
    V = 0.0
    Y = 0.0
    for sk, wk in zip(s, w):
        V = V + wk * (fun(X + 0.5 * dx - ex, Yg + sk * dy) - fun(X - 0.5 * dx + ex, Yg + sk * dy))
        Y = Y + wk * (fun(X + sk * dx, Yg + 0.5 * dy - ey) - fun(X + sk * dx, Yg - 0.5 * dy + ey))
    V = V / dx
    Y = Y / dy
    Z = (fun(X + 0.5 * dx - ex, Yg + 0.5 * dy - ey) - fun(X - 0.5 * dx + ex, Yg + 0.5 * dy - ey)
         - fun(X + 0.5 * dx - ex, Yg - 0.5 * dy + ey) + fun(X - 0.5 * dx + ex, Yg - 0.5 * dy + ey)) / (dx * dy)
    full = (np.shape(W)[0], ny, nx)
    c = lambda a: np.ascontiguousarray(np.broadcast_to(a, full))
    return c(W), c(V), c(Y), c(Z)


# --------------------------------------------------------------------------- Example 5.1
def burgers_sine(nx, t_final=0.5 / math.pi, cfl=0.6):
    """u_t + (u^2/2)_x = 0 on (0,2), u0 = 0.5 + sin(pi x), periodic (Example 5.1)."""
    f = lambda x: (0.5 + np.sin(np.pi * x))[None]
    W, V = project_1d(f, 0.0, 2.0, nx)

    def exact(t, nq=6):
        # u = u0(x - u t) solved by Newton's iteration at every quadrature point.
        def u_at(x):
            u = 0.5 + np.sin(np.pi * x)
            for _ in range(100):
                g = u - 0.5 - np.sin(np.pi * (x - u * t))
                dg = 1.0 + np.pi * t * np.cos(np.pi * (x - u * t))
                du = g / dg
                u = u - du
                if np.max(np.abs(du)) < 1e-15:
                    break
            return u[None]
        return project_1d(u_at, 0.0, 2.0, nx, nq)[0]

    return Workload("burgers_sine", 1, BURGERS, nx, 1, (0.0, 2.0, 0.0, 1.0),
                    (PERIODIC, PERIODIC, PERIODIC, PERIODIC), t_final, cfl, {"W": W, "V": V},
                    exact=exact)


def burgers2d_sine(n, t_final=0.25 / math.pi, cfl=0.6):
    """u_t + (u^2/2)_x + (u^2/2)_y = 0 on (0,2)^2, u0 = 0.5 + sin(pi (x + y)), periodic: the 2D
    scalar law of Section 3 with the data of Example 5.1 laid along the diagonal.  The solution
    is u = u0(x + y - 2 u t) (smooth until t = 1/(2 pi)); T defaults to half of that."""
    f = lambda x, y: (0.5 + np.sin(np.pi * (x + y)))[None]
    W, V, Y, Z = project_2d(f, 0.0, 2.0, 0.0, 2.0, n, n)

    def exact(t, nq=6):
        def u_at(x, y):
            s = x + y
            u = 0.5 + np.sin(np.pi * s)
            for _ in range(100):
                g = u - 0.5 - np.sin(np.pi * (s - 2.0 * u * t))
                dg = 1.0 + 2.0 * np.pi * t * np.cos(np.pi * (s - 2.0 * u * t))
                du = g / dg
                u = u - du
                if np.max(np.abs(du)) < 1e-15:
                    break
            return u[None]
        return project_2d(u_at, 0.0, 2.0, 0.0, 2.0, n, n, nq)[0]

    return Workload("burgers2d_sine", 2, BURGERS, n, n, (0.0, 2.0, 0.0, 2.0), (PERIODIC,) * 4,
                    t_final, cfl, {"W": W, "V": V, "Y": Y, "Z": Z}, exact=exact)


def burgers2d_riemann(n, values=(-1.0, -0.2, 0.5, 0.8), t_final=0.5, cfl=0.6):
    """Four-quadrant Riemann problem of 2D Burgers on (0,1)^2, split at (1/2, 1/2), outflow
    sides; values for the quadrants NE, NW, SW, SE (shocks, rarefactions and a sonic point)."""
    if n % 2:
        raise ValueError("n must be even: the split lines are then cell edges")
    W = np.empty((1, n, n))
    h = n // 2
    W[0, h:, h:], W[0, h:, :h], W[0, :h, :h], W[0, :h, h:] = values
    Z0 = np.zeros_like(W)
    return Workload("burgers2d_riemann", 2, BURGERS, n, n, (0.0, 1.0, 0.0, 1.0), (OUTFLOW,) * 4,
                    t_final, cfl, {"W": W, "V": Z0, "Y": Z0.copy(), "Z": Z0.copy()}, shocked=True)


# --------------------------------------------------------------------------- Example 5.2
def euler1d_sine(nx, t_final=10.0, cfl=0.6):
    """rho = 1 + 0.2 sin(pi x), u = p = 1 on (0,2), periodic (Example 5.2); exact: translation."""
    def at(t):
        return lambda x: euler_conserved(1.0 + 0.2 * np.sin(np.pi * (x - t)), np.ones_like(x), np.ones_like(x))
    W, V = project_1d(at(0.0), 0.0, 2.0, nx)
    return Workload("euler1d_sine", 1, EULER, nx, 1, (0.0, 2.0, 0.0, 1.0),
                    (PERIODIC,) * 4, t_final, cfl, {"W": W, "V": V},
                    exact=lambda t: project_1d(at(t), 0.0, 2.0, nx)[0])


# --------------------------------------------------------------------------- Example 5.7
def euler2d_sine(n, t_final=1.0, cfl=0.6):
    """rho = 1 + 0.2 sin(pi (x+y)), u = v = p = 1 on (0,2)^2, periodic (Example 5.7)."""
    def at(t):
        return lambda x, y: euler_conserved(1.0 + 0.2 * np.sin(np.pi * (x + y - 2 * t)),
                                            np.ones_like(x), np.ones_like(x), np.ones_like(x))
    W, V, Y, Z = project_2d(at(0.0), 0.0, 2.0, 0.0, 2.0, n, n)
    return Workload("euler2d_sine", 2, EULER, n, n, (0.0, 2.0, 0.0, 2.0), (PERIODIC,) * 4,
                    t_final, cfl, {"W": W, "V": V, "Y": Y, "Z": Z},
                    exact=lambda t: project_2d(at(t), 0.0, 2.0, 0.0, 2.0, n, n)[0])


# --------------------------------------------------------------------------- Example 5.8
def vortex_fun(t=0.0, L=10.0, strength=5.0, gamma=GAMMA):
    """Isentropic vortex of Example 5.8 moving with (1,1) on the periodic box (0,L)^2."""
    def f(x, y):
        # periodic image nearest to the vortex centre, which sits at (5+t, 5+t) mod L
        cx = (5.0 + t) % L
        cy = (5.0 + t) % L
        xr = (x - cx + 0.5 * L) % L - 0.5 * L
        yr = (y - cy + 0.5 * L) % L - 0.5 * L
        # exp((1 - r^2)/2) = e^(1/2) exp(-xr^2/2) exp(-yr^2/2): one exp per coordinate
        e = math.exp(0.5) * np.exp(-0.5 * xr * xr) * np.exp(-0.5 * yr * yr)
        base = 1.0 - (gamma - 1.0) * strength ** 2 / (8.0 * gamma * math.pi ** 2) * e * e
        if gamma == 1.4:  # rho = base^2.5, p = rho^1.4 = base^3.5, without pow
            rho = base * base * np.sqrt(base)
            p = rho * base
        else:
            rho = base ** (1.0 / (gamma - 1.0))
            p = rho ** gamma
        u = 1.0 - strength / (2.0 * math.pi) * e * yr
        v = 1.0 + strength / (2.0 * math.pi) * e * xr
        return euler_conserved(rho, u, p, v, gamma)
    return f


def vortex_core_mask(n, t, radius=2.5, L=10.0):
    """Cells of the n x n vortex mesh whose centres lie within `radius` (periodic distance) of the
    vortex centre at time t.  The nearest-image vortex of Example 5.8 is not smooth across the
    seams of the periodic box: its tangential velocity jumps by about 5e-5 there (the vortex's
    tail at distance 5).  The seams travel with the flow and shed acoustic waves (density about
    1.5e-8 at 512^2, falling about linearly with the mesh width) that cross the box at the sound
    speed and reach this core only after about t = 1.5 for the default radius."""
    c = (5.0 + t) % L
    x = (np.arange(n) + 0.5) * (L / n)
    d = (x - c + 0.5 * L) % L - 0.5 * L
    return (d[None, :] ** 2 + d[:, None] ** 2) <= radius * radius


def vortex(n, t_final=10.0, cfl=0.6):
    W, V, Y, Z = project_2d(vortex_fun(0.0), 0.0, 10.0, 0.0, 10.0, n, n)
    return Workload("isentropic_vortex", 2, EULER, n, n, (0.0, 10.0, 0.0, 10.0), (PERIODIC,) * 4,
                    t_final, cfl, {"W": W, "V": V, "Y": Y, "Z": Z},
                    exact=lambda t: project_2d(vortex_fun(t), 0.0, 10.0, 0.0, 10.0, n, n)[0])


# --------------------------------------------------------------------------- Riemann data
def riemann1d(nx, left, right, x0=0.0, x1=1.0, xs=0.5, t_final=0.15, cfl=0.6, name="riemann1d",
              bc=(OUTFLOW, OUTFLOW)):
    """Piecewise-constant primitive states (rho, u, p) split at xs.  Exact averages: a cell cut
    by the jump holds the length-weighted mix, and its derivative average is the jump over dx."""
    dx = (x1 - x0) / nx
    xl = x0 + np.arange(nx) * dx
    xr = xl + dx
    UL = euler_conserved(*[np.float64(v) for v in left])
    UR = euler_conserved(*[np.float64(v) for v in right])
    frac_left = np.clip((xs - xl) / dx, 0.0, 1.0)
    W = UL[:, None] * frac_left[None] + UR[:, None] * (1.0 - frac_left[None])
    inside = (xl < xs) & (xs < xr)
    V = np.where(inside[None], (UR - UL)[:, None] / dx, 0.0)
    return Workload(name, 1, EULER, nx, 1, (x0, x1, 0.0, 1.0), (bc[0], bc[1], 0, 0), t_final, cfl,
                    {"W": np.ascontiguousarray(W), "V": np.ascontiguousarray(V)}, shocked=True)


def sod(nx=100, t_final=0.2, cfl=0.6):
    return riemann1d(nx, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), t_final=t_final, cfl=cfl, name="sod")


def lax(nx=200, t_final=1.3, cfl=0.6):
    """Lax problem of Example 5.3 on (-5, 5)."""
    return riemann1d(nx, (0.445, 0.698, 3.528), (0.5, 0.0, 0.571), x0=-5.0, x1=5.0, xs=0.0,
                     t_final=t_final, cfl=cfl, name="lax")


def random_riemann1d(seed, nx=None, t_final=0.15, cfl=0.6):
    """One problem of the seeded batch: rho ~ U[0.1,2], u ~ U[-1,1], p ~ U[0.1,10] on each side,
    jump at x = 0.5 on [0,1], outflow, N ~ U{400..16384} unless given."""
    rng = np.random.default_rng(10_000 + seed)
    L = (rng.uniform(0.1, 2.0), rng.uniform(-1.0, 1.0), rng.uniform(0.1, 10.0))
    R = (rng.uniform(0.1, 2.0), rng.uniform(-1.0, 1.0), rng.uniform(0.1, 10.0))
    n = int(rng.integers(400, 16385)) if nx is None else nx
    return riemann1d(n, L, R, t_final=t_final, cfl=cfl, name=f"riemann1d_seed{seed}")


def quadrant_fun(states, xs=0.5, ys=0.5):
    """states: primitive (rho, u, v, p) for quadrants NE, NW, SW, SE (the paper's order)."""
    S = [euler_conserved(np.float64(r), np.float64(u), np.float64(p), np.float64(v))
         for (r, u, v, p) in states]

    def f(x, y):
        east, north = x >= xs, y >= ys
        out = np.empty((4,) + np.broadcast_shapes(np.shape(x), np.shape(y)))
        for q in range(4):
            out[q] = np.where(north, np.where(east, S[0][q], S[1][q]), np.where(east, S[3][q], S[2][q]))
        return out
    return f


def riemann2d(n, states, t_final=0.25, cfl=0.6, name="riemann2d"):
    """Four-quadrant problem on (0,1)^2 with outflow (non-reflecting) sides (Example 5.9)."""
    if n % 2 == 0:
        # the split lines x = 1/2, y = 1/2 are cell edges: every cell average is a quadrant state
        # and no cell contains a jump, so V, Y and Z vanish exactly
        S = [euler_conserved(np.float64(r), np.float64(u), np.float64(p), np.float64(v))
             for (r, u, v, p) in states]
        W = np.empty((4, n, n))
        h = n // 2
        for q in range(4):
            W[q, h:, h:], W[q, h:, :h], W[q, :h, :h], W[q, :h, h:] = S[0][q], S[1][q], S[2][q], S[3][q]
        Z0 = np.zeros_like(W)
        W, V, Y, Z = W, Z0, Z0.copy(), Z0.copy()
    else:
        f = quadrant_fun(states)
        W, V, Y, Z = project_2d(f, 0.0, 1.0, 0.0, 1.0, n, n, eps_edge=1e-9)
    return Workload(name, 2, EULER, n, n, (0.0, 1.0, 0.0, 1.0), (OUTFLOW,) * 4, t_final, cfl,
                    {"W": W, "V": V, "Y": Y, "Z": Z}, shocked=True)


# Example 5.9, first configuration (four shocks), quadrants NE, NW, SW, SE as (rho, u, v, p).
LAX_LIU_SHOCKS = [(1.1, 0.0, 0.0, 1.1), (0.5065, 0.8939, 0.0, 0.35),
                  (1.1, 0.8939, 0.8939, 1.1), (0.5065, 0.0, 0.8939, 0.35)]
# Example 5.9, second configuration (four contacts).
LAX_LIU_CONTACTS = [(1.0, 0.75, -0.5, 1.0), (2.0, 0.5, 0.5, 1.0),
                    (1.0, -0.75, 0.5, 1.0), (3.0, -0.75, -0.5, 1.0)]


def random_quadrants(seed):
    rng = np.random.default_rng(20_000 + seed)
    return [(rng.uniform(0.1, 2.0), rng.uniform(-1.0, 1.0), rng.uniform(-1.0, 1.0), rng.uniform(0.1, 2.0))
            for _ in range(4)]


def random_riemann2d(seed, n=None, t_final=0.25, cfl=0.6):
    """One problem of the seeded 2D batch: quadrant states rho ~ U[0.1,2], u,v ~ U[-1,1],
    p ~ U[0.1,2], split at (0.5,0.5), side ~ U{512..2048} in multiples of 32 unless given."""
    rng = np.random.default_rng(30_000 + seed)
    side = int(rng.integers(16, 65)) * 32 if n is None else n
    return riemann2d(side, random_quadrants(seed), t_final=t_final, cfl=cfl, name=f"riemann2d_seed{seed}")


# --------------------------------------------------------------------------- Example 5.10
DMR_POST = (8.0, 57.1597, -33.0012, 563.544)
DMR_PRE = (1.4, 0.0, 0.0, 2.5)


def _above_area(xa, xb, ya, yb, slope, xoff):
    """Area of [xa,xb] x [ya,yb] where y >= slope (x - xoff) (slope > 0), exactly."""
    h = yb - ya

    def Hf(u):  # integral_0^u clamp(w, 0, h) dw
        return np.where(u <= 0, 0.0, np.where(u <= h, 0.5 * u * u, 0.5 * h * h + h * (u - h)))
    ua = yb - slope * (xa - xoff)
    ub = yb - slope * (xb - xoff)
    return (Hf(ua) - Hf(ub)) / slope


def dmr(nx=4096, ny=1024, t_final=0.2, cfl=0.6):
    """Double Mach reflection (Example 5.10) on (0,4) x (0,1): post-shock state where
    y >= sqrt(3) (x - 1/6), pre-shock elsewhere.  Exact area fractions for W, exact edge fractions
    for V and Y, corner values for Z."""
    s3 = math.sqrt(3.0)
    x0, x1, y0, y1 = 0.0, 4.0, 0.0, 1.0
    dx, dy = (x1 - x0) / nx, (y1 - y0) / ny
    xl = x0 + np.arange(nx) * dx
    yl = y0 + np.arange(ny) * dy
    XA, YA = np.meshgrid(xl, yl)
    XB, YB = XA + dx, YA + dy
    post = np.array(DMR_POST)[:, None, None]
    pre = np.array(DMR_PRE)[:, None, None]
    fpost = _above_area(XA, XB, YA, YB, s3, 1.0 / 6.0) / (dx * dy)
    W = pre + (post - pre) * fpost[None]

    def edge_frac_vertical(xe):  # fraction of the vertical edge at xe (rows) above the line
        yline = s3 * (xe - 1.0 / 6.0)
        return np.clip((YB - np.maximum(YA, yline)) / dy, 0.0, 1.0)

    def edge_frac_horizontal(ye):  # fraction of the horizontal edge at ye left of the line
        xline = 1.0 / 6.0 + ye / s3
        return np.clip((np.minimum(XB, xline) - XA) / dx, 0.0, 1.0)

    V = (post - pre) * ((edge_frac_vertical(XB) - edge_frac_vertical(XA)) / dx)[None]
    Y = (post - pre) * ((edge_frac_horizontal(YB) - edge_frac_horizontal(YA)) / dy)[None]

    def corner(xc, yc):
        return np.where((yc >= s3 * (xc - 1.0 / 6.0))[None], post, pre)
    Z = (corner(XB, YB) - corner(XA, YB) - corner(XB, YA) + corner(XA, YA)) / (dx * dy)
    c = np.ascontiguousarray
    return Workload("double_mach_reflection", 2, EULER, nx, ny, (x0, x1, y0, y1),
                    (INFLOW, OUTFLOW, DMR_BOTTOM, DMR_TOP), t_final, cfl,
                    {"W": c(W), "V": c(V), "Y": c(Y), "Z": c(Z)},
                    inflow=[list(DMR_POST), [0.0] * 4, [0.0] * 4, [0.0] * 4], shocked=True)


def constant_state(dim, eq, nx, ny=1, value=None):
    """A uniform state with zero derivative averages (free-stream test)."""
    nc = 1 if eq == BURGERS else (3 if dim == 1 else 4)
    if value is None:
        value = [0.7] if eq == BURGERS else (list(euler_conserved(1.2, 0.3, 0.9)) if dim == 1
                                            else list(euler_conserved(1.2, 0.3, 0.9, -0.4)))
    shape = (nc, nx) if dim == 1 else (nc, ny, nx)
    W = np.empty(shape)
    for q in range(nc):
        W[q] = value[q]
    st = {"W": W, "V": np.zeros(shape)}
    if dim == 2:
        st["Y"], st["Z"] = np.zeros(shape), np.zeros(shape)
    return st


def smooth_flow_2d(seed, n, t_final=0.1, cfl=0.6, kmax=4):
    """Seeded smooth periodic 2D Euler flow on (0,1)^2 (training data of the learned flag): for
    each of rho, u, v, p a base value plus three random Fourier modes sin(2 pi k . x + phase),
    k a nonzero integer vector with entries in -kmax..kmax.  The amplitude is 10^U[-10, -0.5]
    times the base (rho, p) or 1 (u, v), so the data span nearly constant flows (a vortex's far
    field) to strong smooth waves."""
    rng = np.random.default_rng(60_000 + seed)
    base = np.array([rng.uniform(0.5, 2.0), rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5), rng.uniform(0.5, 2.0)])
    rel = 10.0 ** rng.uniform(-10.0, -0.5)
    amp = np.array([base[0], 1.0, 1.0, base[3]]) * rel * rng.uniform(0.5, 1.0, size=4)
    ks = []
    while len(ks) < 3:
        k = rng.integers(-kmax, kmax + 1, size=2)
        if k.any():
            ks.append(k)
    a = rng.uniform(-1.0, 1.0, size=(4, 3)) / 3.0
    ph = rng.uniform(0, 2 * math.pi, size=(4, 3))

    def f(x, y):
        fld = [base[c] + amp[c] * sum(a[c, m] * np.sin(2 * math.pi * (ks[m][0] * x + ks[m][1] * y) + ph[c, m])
                                      for m in range(3)) for c in range(4)]
        return euler_conserved(fld[0], fld[1], fld[3], fld[2])
    W, V, Y, Z = project_2d(f, 0.0, 1.0, 0.0, 1.0, n, n)
    return Workload(f"smooth2d_seed{seed}", 2, EULER, n, n, (0.0, 1.0, 0.0, 1.0), (PERIODIC,) * 4,
                    t_final, cfl, {"W": W, "V": V, "Y": Y, "Z": Z})


def smooth_bumps_2d(seed, n, t_final=0.1, cfl=0.6):
    """Seeded smooth periodic 2D Euler flow on (0,1)^2 made of localised structures (training data
    of the learned flag): a uniform state plus three Gaussian bumps exp(-r^2 / (2 w^2)) (periodic
    distance r, width w ~ U[0.02, 0.15], random centre), each adding up to +-45 % of the base to
    rho and p and up to +-1 to u and v."""
    rng = np.random.default_rng(70_000 + seed)
    base = np.array([rng.uniform(0.5, 2.0), rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5), rng.uniform(0.5, 2.0)])
    cen = rng.uniform(0.0, 1.0, size=(3, 2))
    wid = rng.uniform(0.02, 0.15, size=3)
    amp = rng.uniform(-1.0, 1.0, size=(3, 4)) * np.array([0.15 * base[0], 0.33, 0.33, 0.15 * base[3]])

    def f(x, y):
        fld = [base[c] + 0.0 * (x + y) for c in range(4)]
        for b in range(3):
            dx = (x - cen[b, 0] + 0.5) % 1.0 - 0.5
            dy = (y - cen[b, 1] + 0.5) % 1.0 - 0.5
            g = np.exp(-(dx * dx + dy * dy) / (2.0 * wid[b] ** 2))
            for c in range(4):
                fld[c] = fld[c] + amp[b, c] * g
        return euler_conserved(fld[0], fld[1], fld[3], fld[2])
    W, V, Y, Z = project_2d(f, 0.0, 1.0, 0.0, 1.0, n, n)
    return Workload(f"bumps2d_seed{seed}", 2, EULER, n, n, (0.0, 1.0, 0.0, 1.0), (PERIODIC,) * 4,
                    t_final, cfl, {"W": W, "V": V, "Y": Y, "Z": Z})


def random_smooth_1d(seed, nx, eq=EULER, amp=0.1):
    """Seeded smooth periodic data on (0,1): a few random Fourier modes on a positive state."""
    rng = np.random.default_rng(40_000 + seed)
    ks = rng.integers(1, 4, size=3)
    ph = rng.uniform(0, 2 * math.pi, size=(3, 3))
    a = rng.uniform(-amp, amp, size=(3, 3))

    def f(x):
        pert = [sum(a[c, m] * np.sin(2 * math.pi * ks[m] * x + ph[c, m]) for m in range(3)) for c in range(3)]
        if eq == BURGERS:
            return (0.3 + 5 * pert[0])[None]
        return euler_conserved(1.0 + pert[0], 0.5 + pert[1], 1.0 + pert[2])
    return project_1d(f, 0.0, 1.0, nx)


def random_smooth_2d(seed, nx, ny, amp=0.1, eq=EULER):
    """Seeded smooth periodic data on (0,1)^2 (Burgers: a field that changes sign)."""
    rng = np.random.default_rng(50_000 + seed)
    kx = rng.integers(1, 3, size=4)
    ky = rng.integers(0, 3, size=4)
    ph = rng.uniform(0, 2 * math.pi, size=4)
    a = rng.uniform(-amp, amp, size=4)

    def f(x, y):
        m = [a[c] * np.sin(2 * math.pi * (kx[c] * x + ky[c] * y) + ph[c]) for c in range(4)]
        if eq == BURGERS:
            return (0.1 + 5 * m[0] + 3 * m[1] + 0 * y)[None]
        return euler_conserved(1.0 + m[0], 0.4 + m[1], 1.0 + m[2], -0.3 + m[3])
    return project_2d(f, 0.0, 1.0, 0.0, 1.0, nx, ny)
