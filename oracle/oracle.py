"""ctypes front end of the ADER-SHWENO oracle -- TEST INFRASTRUCTURE ONLY.

The oracle is the plain single-threaded FP64 C++ restatement of the paper's scheme in
``shweno_oracle.cpp`` (see its header for the steps and the paper passages each one follows).
Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` import this
module; the CUDA library never does.  ``build()`` compiles the shared object with g++ beside the
source; nothing here imports the library package.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "shweno_oracle.cpp")
LIB = os.path.join(HERE, "liboracle.so")

EQ_BURGERS, EQ_EULER = 0, 1
BC_PERIODIC, BC_OUTFLOW, BC_REFLECTIVE, BC_INFLOW, BC_DMR_BOTTOM, BC_DMR_TOP = range(6)
GAMMA_LINEAR = (0.994, 0.003, 0.003)  # Section 2.4


class Problem(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int32), ("eq", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("x0", ctypes.c_double), ("y0", ctypes.c_double), ("dx", ctypes.c_double), ("dy", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("bc", ctypes.c_int32 * 4),
        ("inflow", (ctypes.c_double * 4) * 4),
        ("linear", ctypes.c_int32),
        ("eps", ctypes.c_double),
        ("gam", ctypes.c_double * 3),
        ("charwise", ctypes.c_int32),
        ("quintic", ctypes.c_int32),
    ]


def build(force: bool = False) -> str:
    """Compiles liboracle.so with g++ (portable flags only: it is built on x86 and Arm)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, SRC])
        os.replace(tmp, LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(Problem)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        L.orc_big_poly.argtypes = [dp, dp, dp]
        L.orc_smoothness.argtypes = [dp]
        L.orc_smoothness.restype = ctypes.c_double
        L.orc_weights.argtypes = [dp, dp, ctypes.c_int, ctypes.c_double, dp, dp]
        L.orc_recon.argtypes = [dp, dp, ctypes.c_int, ctypes.c_double, dp, ctypes.c_double, dp]
        L.orc_recon_deg.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, dp,
                                    ctypes.c_double, dp]
        L.orc_big_poly_deg.argtypes = [dp, dp, ctypes.c_int, dp]
        L.orc_smoothness_deg.argtypes = [dp]
        L.orc_smoothness_deg.restype = ctypes.c_double
        L.orc_quadrature.argtypes = [dp, dp, dp, dp]
        L.orc_burgers_godunov.argtypes = [ctypes.c_double, ctypes.c_double]
        L.orc_burgers_godunov.restype = ctypes.c_double
        L.orc_hllc.argtypes = [pp, ctypes.c_int, dp, dp, dp]
        L.orc_eigen.argtypes = [pp, ctypes.c_int, dp, dp, dp, dp]
        L.orc_upwind.argtypes = [pp, ctypes.c_int, dp, dp, dp, dp]
        L.orc_ck.argtypes = [pp, dp, dp]
        L.orc_grp_point.argtypes = [pp, ctypes.c_int, dp, dp, dp]
        L.orc_max_rate.argtypes = [pp, dp]
        L.orc_max_rate.restype = ctypes.c_double
        L.orc_step.argtypes = [pp, dp, dp, dp, dp, u8p, ctypes.c_double, ctypes.c_double, dp, dp, dp, dp]
        L.orc_run.argtypes = [pp, dp, dp, dp, dp, u8p, ctypes.c_double, ctypes.c_double,
                              ctypes.c_int64, dp, ctypes.POINTER(ctypes.c_int32)]
        L.orc_step2d_cells.argtypes = [pp, dp, dp, dp, dp, u8p, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int, ctypes.POINTER(ctypes.c_int32), dp]
        L.orc_run.restype = ctypes.c_int64
        L.orc_weight_deviation2d.argtypes = [pp, dp, dp, dp, dp, ctypes.c_double, dp]
        L.orc_features2d.argtypes = [pp, dp, dp, dp, dp, ctypes.c_double, dp]
        L.orc_face_deviation2d.argtypes = [pp, dp, dp, dp, dp, ctypes.c_double, ctypes.c_double, dp]
        L.orc_face_deviation.argtypes = [dp, dp, ctypes.c_double, dp, ctypes.c_double]
        L.orc_face_deviation.restype = ctypes.c_double
        L.orc_step2d_window.argtypes = [pp, dp, dp, dp, dp, u8p, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def make_problem(dim, eq, nx, ny=1, x0=0.0, x1=1.0, y0=0.0, y1=1.0, gamma=1.4, bc=(0, 0, 0, 0),
                 inflow=None, linear=False, eps=1e-6, gam=GAMMA_LINEAR, charwise=False,
                 quintic=False) -> Problem:
    P = Problem()
    P.dim, P.eq, P.nx, P.ny = dim, eq, nx, (ny if dim == 2 else 1)
    P.x0, P.y0 = x0, y0
    P.dx = (x1 - x0) / nx
    P.dy = (y1 - y0) / ny if dim == 2 else 1.0
    P.gamma = gamma
    for k in range(4):
        P.bc[k] = bc[k] if k < len(bc) else 0
    if inflow is not None:
        for s in range(4):
            for q in range(4):
                P.inflow[s][q] = inflow[s][q]
    P.linear = 1 if linear else 0
    P.eps = eps
    for k in range(3):
        P.gam[k] = gam[k]
    P.charwise = 1 if charwise else 0
    P.quintic = 1 if quintic else 0
    return P


def ncomp(P: Problem) -> int:
    return 1 if P.eq == EQ_BURGERS else (3 if P.dim == 1 else 4)


# ---------------------------------------------------------------- pieces of the method
def big_poly(Wb, v):
    c = np.zeros(5)
    lib().orc_big_poly(_dp(_f64(Wb)), _dp(_f64(v)), _dp(c))
    return c


def smoothness(c):
    return lib().orc_smoothness(_dp(_f64(c)))


def weights(Wb, v, linear=False, eps=1e-6, gam=GAMMA_LINEAR):
    w = np.zeros(3)
    lib().orc_weights(_dp(_f64(Wb)), _dp(_f64(v)), int(linear), eps, _dp(_f64(gam)), _dp(w))
    return w


def recon(Wb, v, xi, linear=False, eps=1e-6, gam=GAMMA_LINEAR):
    """d^k p/dxi^k (k = 0..4) of the SHWENO polynomial of the middle cell at xi."""
    d = np.zeros(5)
    lib().orc_recon(_dp(_f64(Wb)), _dp(_f64(v)), int(linear), eps, _dp(_f64(gam)), xi, _dp(d))
    return d


def big_poly_deg(Wb, v3, quintic):
    """p1 coefficients c[0..5] from v3 = (h V_-1, h V_0, h V_+1) (reading R1 ignores h V_0)."""
    c = np.zeros(6)
    lib().orc_big_poly_deg(_dp(_f64(Wb)), _dp(_f64(v3)), int(quintic), _dp(c))
    return c


def smoothness_deg(c6):
    return lib().orc_smoothness_deg(_dp(_f64(c6)))


def recon_deg(Wb, v3, xi, quintic, linear=False, eps=1e-6, gam=GAMMA_LINEAR):
    """recon() with v3 = (h V_-1, h V_0, h V_+1) and the choice of reading R1 / R1'."""
    d = np.zeros(5)
    lib().orc_recon_deg(_dp(_f64(Wb)), _dp(_f64(v3)), int(quintic), int(linear), eps, _dp(_f64(gam)),
                        xi, _dp(d))
    return d


def quadrature():
    a, b, c, d = np.zeros(4), np.zeros(4), np.zeros(3), np.zeros(3)
    lib().orc_quadrature(_dp(a), _dp(b), _dp(c), _dp(d))
    return a, b, c, d


def burgers_godunov(uL, uR):
    return lib().orc_burgers_godunov(uL, uR)


def hllc(P, dir_, WL, WR):
    out = np.zeros(ncomp(P))
    lib().orc_hllc(ctypes.byref(P), dir_, _dp(_f64(WL)), _dp(_f64(WR)), _dp(out))
    return out


def eigen(P, dir_, W):
    n = ncomp(P)
    lam, R, L = np.zeros(n), np.zeros(n * n), np.zeros(n * n)
    lib().orc_eigen(ctypes.byref(P), dir_, _dp(_f64(W)), _dp(lam), _dp(R), _dp(L))
    return lam, R.reshape(n, n), L.reshape(n, n)


def upwind(P, dir_, Ws, dL, dR):
    out = np.zeros(ncomp(P))
    lib().orc_upwind(ctypes.byref(P), dir_, _dp(_f64(Ws)), _dp(_f64(dL)), _dp(_f64(dR)), _dp(out))
    return out


def ck(P, d):
    """d: [nc][5][5] spatial derivatives (m+n <= 4).  Returns [nc][5][5][5] d^{m+n+k}/dx^m dy^n dt^k."""
    n = ncomp(P)
    d = _f64(d).reshape(n, 5, 5)
    out = np.zeros((n, 5, 5, 5))
    lib().orc_ck(ctypes.byref(P), _dp(d), _dp(out))
    return out


def grp_point(P, dir_, dL, dR):
    n = ncomp(P)
    tc = np.zeros((n, 5))
    lib().orc_grp_point(ctypes.byref(P), dir_, _dp(_f64(dL).reshape(n, 5, 5)),
                        _dp(_f64(dR).reshape(n, 5, 5)), _dp(tc))
    return tc


def max_rate(P, W):
    return lib().orc_max_rate(ctypes.byref(P), _dp(_f64(W)))


# ---------------------------------------------------------------- whole steps
def _flag_ptr(flag):
    if flag is None:
        return None, None
    f = np.ascontiguousarray(flag, dtype=np.uint8)
    return f, f.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def step(P, state, dt, t=0.0, flag=None):
    """One step.  state: dict with 'W','V' (and 'Y','Z' in 2D) arrays [nc][ny][nx] / [nc][nx]."""
    W, V = _f64(state["W"]), _f64(state["V"])
    Y = _f64(state["Y"]) if P.dim == 2 else None
    Z = _f64(state["Z"]) if P.dim == 2 else None
    Wn, Vn = np.empty_like(W), np.empty_like(V)
    Yn = np.empty_like(Y) if Y is not None else None
    Zn = np.empty_like(Z) if Z is not None else None
    fl, fp = _flag_ptr(flag)
    lib().orc_step(ctypes.byref(P), _dp(W), _dp(V), _dp(Y), _dp(Z), fp, t, dt, _dp(Wn), _dp(Vn),
                   _dp(Yn), _dp(Zn))
    out = {"W": Wn, "V": Vn}
    if P.dim == 2:
        out["Y"], out["Z"] = Yn, Zn
    return out


def step2d_cells(P, state, dt, cells, t=0.0, flag=None):
    """One 2D step evaluated only at the listed (i, j) cells.  Returns {'W','V','Y','Z'}: [n][nc]."""
    W, V, Y, Z = (_f64(state[k]) for k in "WVYZ")
    ij = np.ascontiguousarray(np.asarray(cells, dtype=np.int32).reshape(-1, 2))
    n, nc = len(ij), ncomp(P)
    out = np.zeros((n, 4, nc))
    fl, fp = _flag_ptr(flag)
    lib().orc_step2d_cells(ctypes.byref(P), _dp(W), _dp(V), _dp(Y), _dp(Z), fp, t, dt, n,
                           ij.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(out))
    return {k: out[:, f, :] for f, k in enumerate("WVYZ")}


def step2d_window(P, state, dt, i0, j0, w, h, t=0.0, flag=None):
    """One 2D step evaluated on the window [i0, i0+w) x [j0, j0+h).  Returns {'W',...}: [nc][h][w]."""
    W, V, Y, Z = (_f64(state[k]) for k in "WVYZ")
    nc = ncomp(P)
    out = np.zeros((4, nc, h, w))
    fl, fp = _flag_ptr(flag)
    lib().orc_step2d_window(ctypes.byref(P), _dp(W), _dp(V), _dp(Y), _dp(Z), fp, t, dt, i0, j0, w, h,
                            _dp(out))
    return {k: out[f] for f, k in enumerate("WVYZ")}


def weight_deviation2d(P, state, t=0.0):
    """Per cell: max relative deviation of the 16 first-pass nonlinear weights from gamma [ny][nx]."""
    W, V, Y, Z = (_f64(state[k]) for k in "WVYZ")
    out = np.zeros((P.ny, P.nx))
    lib().orc_weight_deviation2d(ctypes.byref(P), _dp(W), _dp(V), _dp(Y), _dp(Z), t, _dp(out))
    return out


def face_deviation(Wb, v, eps=1e-6, gam=GAMMA_LINEAR, floor_rel=1e-9):
    """max over xi = -1/2, +1/2 of |p(xi) - p1(xi)| / (range of Wb + floor_rel |W0| + 1e-300) for
    the reconstruction of the middle cell (v = (h V_-1, h V_+1))."""
    return lib().orc_face_deviation(_dp(_f64(Wb)), _dp(_f64(v)), eps, _dp(_f64(gam)), floor_rel)


def face_deviation2d(P, state, t=0.0, floor_rel=1e-9):
    """Per cell: the largest relative change the nonlinear weights make to the end values of its
    16 first-pass reconstructions [ny][nx]."""
    W, V, Y, Z = (_f64(state[k]) for k in "WVYZ")
    out = np.zeros((P.ny, P.nx))
    lib().orc_face_deviation2d(ctypes.byref(P), _dp(W), _dp(V), _dp(Y), _dp(Z), t, floor_rel, _dp(out))
    return out


def features2d(P, state, t=0.0):
    """Per-cell flag-network inputs [ny*nx][22] (see shweno_oracle.cpp)."""
    W, V, Y, Z = (_f64(state[k]) for k in "WVYZ")
    out = np.zeros((P.ny * P.nx, 22))
    lib().orc_features2d(ctypes.byref(P), _dp(W), _dp(V), _dp(Y), _dp(Z), t, _dp(out))
    return out


class NonPhysical(RuntimeError):
    """A step of run() left the physical range; state/steps/t are those before that step."""

    def __init__(self, state, steps, t):
        super().__init__(f"non-physical state after {steps} steps at t = {t}")
        self.state, self.steps, self.t = state, steps, t


def run(P, state, t_final, cfl, flag=None, max_steps=10 ** 9):
    """Runs to t_final (CFL step size, last step shortened).  Returns (state, steps, t); raises
    NonPhysical when a step leaves the physical range (that step is not kept)."""
    W, V = _f64(state["W"]).copy(), _f64(state["V"]).copy()
    Y = _f64(state["Y"]).copy() if P.dim == 2 else None
    Z = _f64(state["Z"]).copy() if P.dim == 2 else None
    fl, fp = _flag_ptr(flag)
    t = ctypes.c_double(0.0)
    bad = ctypes.c_int32(0)
    n = lib().orc_run(ctypes.byref(P), _dp(W), _dp(V), _dp(Y), _dp(Z), fp, t_final, cfl,
                      max_steps, ctypes.byref(t), ctypes.byref(bad))
    out = {"W": W, "V": V}
    if P.dim == 2:
        out["Y"], out["Z"] = Y, Z
    if bad.value:
        raise NonPhysical(out, n, t.value)
    return out, n, t.value
