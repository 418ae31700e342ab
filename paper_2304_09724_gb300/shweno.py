"""Thin ctypes binding of libshweno.so (include/shweno.h): the same entry points under the same
names, with argument marshalling only.  Every step of the method runs in the library's CUDA
kernels; nothing here computes.  Importing succeeds without the library, but every call raises
if libshweno.so is missing or cannot be loaded: there is no fallback.

Device memory and streams come from PyTorch when the caller uses torch tensors: a CUDA tensor
is passed by its data_ptr() with on_device=1, and a torch stream by its cuda_stream handle.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libshweno.so")

OK, E_INVALID, E_CUDA, E_NOMEM, E_NONPHYSICAL, E_TIMEOUT, E_STATE = range(7)
BURGERS, EULER = 0, 1
BC_PERIODIC, BC_OUTFLOW, BC_REFLECTIVE, BC_INFLOW, BC_DMR_BOTTOM, BC_DMR_TOP = range(6)
STATUS_NAMES = {0: "OK", 1: "INVALID", 2: "CUDA", 3: "NOMEM", 4: "NONPHYSICAL", 5: "TIMEOUT", 6: "STATE"}


class shweno_grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("eq", ctypes.c_int32), ("nx", ctypes.c_int64),
                ("ny", ctypes.c_int64), ("x0", ctypes.c_double), ("x1", ctypes.c_double),
                ("y0", ctypes.c_double), ("y1", ctypes.c_double)]


class shweno_bc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32 * 4), ("inflow", (ctypes.c_double * 4) * 4)]


class shweno_opts(ctypes.Structure):
    _fields_ = [("flag_mode", ctypes.c_int32), ("eps", ctypes.c_double), ("gam", ctypes.c_double * 3),
                ("charwise", ctypes.c_int32), ("quintic", ctypes.c_int32)]


class ShwenoError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"shweno {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


EXPORTS = ["shweno_create", "shweno_set_state", "shweno_get_state", "shweno_step", "shweno_run",
           "shweno_advance", "shweno_sync", "shweno_set_timing", "shweno_get_timing",
           "shweno_kernel_name", "shweno_cfl_dt", "shweno_get_time", "shweno_set_flags",
           "shweno_destroy", "shweno_last_error", "shweno_set_allocator", "shweno_step1d_noalloc",
           "shweno_fp64_probe",
           "shweno_flag_features", "shweno_weight_deviation", "shweno_face_deviation", "shweno_mlp_forward",
           "shweno_mlp_grad",
           "shweno_mlp_adam", "shweno_set_flag_net", "shweno_get_flags", "shweno_batch_create",
           "shweno_batch_run", "shweno_batch_autotune", "shweno_batch_set", "shweno_batch_destroy",
           "shweno_batch_last_error", "shweno_batch_set_mode", "shweno_batch_get_mode"]
FLAG_FEATURES, FLAG_PARAMS = 22, 1825
BATCH_AUTO, BATCH_PERSISTENT, BATCH_LOCKSTEP = 0, 1, 2
NOALLOC_MAX_NX = 65536

_lib = None


def lib():
    """Loads libshweno.so (raises if it is missing: the library has no CPU path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libshweno.so not built ({LIB_PATH}); run paper_2304_09724_gb300.build")
    L = ctypes.CDLL(LIB_PATH)
    vp, dp, i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)
    st = ctypes.c_int
    L.shweno_create.argtypes = [ctypes.POINTER(shweno_grid), ctypes.c_double, ctypes.POINTER(shweno_bc),
                                ctypes.POINTER(shweno_opts), vp, ctypes.POINTER(vp)]
    L.shweno_set_state.argtypes = [vp, vp, vp, vp, vp, ctypes.c_double, ctypes.c_int]
    L.shweno_get_state.argtypes = [vp, vp, vp, vp, vp, ctypes.c_int]
    L.shweno_step.argtypes = [vp, ctypes.c_double]
    L.shweno_run.argtypes = [vp, ctypes.c_double, ctypes.c_double, dp, i64p]
    L.shweno_cfl_dt.argtypes = [vp, ctypes.c_double, dp, dp]
    L.shweno_get_time.argtypes = [vp, dp, i64p]
    L.shweno_set_flags.argtypes = [vp, vp, ctypes.c_int]
    L.shweno_destroy.argtypes = [vp]
    L.shweno_advance.argtypes = [vp, ctypes.c_int64, ctypes.c_double]
    L.shweno_sync.argtypes = [vp]
    L.shweno_set_timing.argtypes = [vp, ctypes.c_int]
    L.shweno_get_timing.argtypes = [vp, dp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), i64p]
    L.shweno_kernel_name.argtypes = [vp, ctypes.c_int]
    L.shweno_kernel_name.restype = ctypes.c_char_p
    L.shweno_set_allocator.argtypes = [vp, vp, vp]
    L.shweno_step1d_noalloc.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, ctypes.POINTER(ctypes.c_int32),
                                        ctypes.POINTER(ctypes.c_double * 4), ctypes.c_int32, vp, vp,
                                        ctypes.c_double, ctypes.c_double, vp]
    L.shweno_fp64_probe.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, vp, dp, dp]
    L.shweno_flag_features.argtypes = [vp, vp]
    L.shweno_weight_deviation.argtypes = [vp, vp]
    L.shweno_face_deviation.argtypes = [vp, ctypes.c_double, vp]
    L.shweno_mlp_forward.argtypes = [vp, vp, ctypes.c_int64, vp, vp]
    L.shweno_mlp_grad.argtypes = [vp, vp, vp, ctypes.c_int64, ctypes.c_float, vp, vp, vp]
    L.shweno_mlp_adam.argtypes = [vp, vp, vp, vp, ctypes.c_int64, ctypes.c_float, ctypes.c_float,
                                  ctypes.c_float, ctypes.c_float, vp]
    L.shweno_set_flag_net.argtypes = [vp, vp, ctypes.c_double, ctypes.c_int]
    L.shweno_get_flags.argtypes = [vp, vp, ctypes.c_int]
    L.shweno_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, vp, ctypes.POINTER(vp)]
    L.shweno_batch_run.argtypes = [vp, dp, ctypes.c_double, ctypes.c_int64, ctypes.POINTER(ctypes.c_int)]
    L.shweno_batch_autotune.argtypes = [vp, dp, ctypes.c_double, ctypes.c_int64, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int)]
    L.shweno_batch_set.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int64]
    L.shweno_batch_destroy.argtypes = [vp]
    L.shweno_batch_last_error.argtypes = [vp]
    L.shweno_batch_last_error.restype = ctypes.c_char_p
    L.shweno_batch_set_mode.argtypes = [vp, ctypes.c_int]
    L.shweno_batch_get_mode.argtypes = [vp]
    L.shweno_batch_get_mode.restype = ctypes.c_int
    L.shweno_last_error.argtypes = [vp]
    L.shweno_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("shweno_last_error", "shweno_kernel_name", "shweno_batch_last_error",
                        "shweno_batch_get_mode"):
            getattr(L, name).restype = st
    _lib = L
    return L


def _check(status, h=None):
    if status != OK:
        msg = lib().shweno_last_error(h).decode()
        raise ShwenoError(status, msg)


def _ptr(a):
    """(pointer, on_device) of a numpy array or a torch tensor (float64 or uint8, contiguous)."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data, 0
    # torch tensor
    if not a.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return a.data_ptr(), 1 if a.is_cuda else 0


# --------------------------------------------------------------------------- C names
def shweno_create(grid: shweno_grid, gamma: float, bc: shweno_bc, opts: shweno_opts | None = None,
                  stream: int = 0):
    h = ctypes.c_void_p()
    s = lib().shweno_create(ctypes.byref(grid), gamma, ctypes.byref(bc),
                            ctypes.byref(opts) if opts is not None else None, stream or None, ctypes.byref(h))
    _check(s, None)
    return h


def shweno_set_state(h, W, V, Y=None, Z=None, t=0.0):
    ptrs = [_ptr(a) for a in (W, V, Y, Z)]
    dev = ptrs[0][1]
    _check(lib().shweno_set_state(h, ptrs[0][0], ptrs[1][0], ptrs[2][0], ptrs[3][0], t, dev), h)


def shweno_get_state(h, W, V, Y=None, Z=None):
    ptrs = [_ptr(a) for a in (W, V, Y, Z)]
    _check(lib().shweno_get_state(h, ptrs[0][0], ptrs[1][0], ptrs[2][0], ptrs[3][0], ptrs[0][1]), h)


def shweno_step(h, dt):
    _check(lib().shweno_step(h, dt), h)


def shweno_run(h, t_final, cfl):
    t = ctypes.c_double()
    n = ctypes.c_int64()
    _check(lib().shweno_run(h, t_final, cfl, ctypes.byref(t), ctypes.byref(n)), h)
    return t.value, n.value


def shweno_cfl_dt(h, cfl):
    dt, rate = ctypes.c_double(), ctypes.c_double()
    _check(lib().shweno_cfl_dt(h, cfl, ctypes.byref(dt), ctypes.byref(rate)), h)
    return dt.value, rate.value


def shweno_get_time(h):
    t, n = ctypes.c_double(), ctypes.c_int64()
    _check(lib().shweno_get_time(h, ctypes.byref(t), ctypes.byref(n)), h)
    return t.value, n.value


def shweno_set_flags(h, flags):
    p, dev = _ptr(flags)
    _check(lib().shweno_set_flags(h, p, dev), h)


def shweno_advance(h, nsteps, cfl):
    _check(lib().shweno_advance(h, nsteps, cfl), h)


def shweno_sync(h):
    _check(lib().shweno_sync(h), h)


def shweno_set_timing(h, enable):
    _check(lib().shweno_set_timing(h, 1 if enable else 0), h)


def shweno_get_timing(h, max_kernels=8):
    """Returns ({kernel name: total ms}, timed steps) and clears the totals."""
    ms = (ctypes.c_double * max_kernels)()
    nk, ns = ctypes.c_int(), ctypes.c_int64()
    _check(lib().shweno_get_timing(h, ms, max_kernels, ctypes.byref(nk), ctypes.byref(ns)), h)
    names = [lib().shweno_kernel_name(h, k).decode() for k in range(nk.value)]
    return {n: ms[k] for k, n in enumerate(names)}, ns.value


def shweno_step1d_noalloc(eq, nx, x0, x1, gamma, bc, inflow, flag_mode, state_in, state_out, t, dt,
                          stream=0):
    """One 1D step without any device allocation (see include/shweno.h); returns the status."""
    kinds = (ctypes.c_int32 * 2)(*bc)
    infl = ((ctypes.c_double * 4) * 2)(*[(ctypes.c_double * 4)(*inflow[s]) for s in range(2)]) if inflow else None
    return lib().shweno_step1d_noalloc(eq, nx, x0, x1, gamma, kinds, infl, flag_mode, _ptr(state_in)[0],
                                       _ptr(state_out)[0], t, dt, stream or None)


FP64_FMA, FP64_MUL, FP64_ADD, FP64_MIX = 0, 1, 2, 3


def shweno_fp64_probe(op=FP64_FMA, warps_per_sm=8, iters=1 << 16, stream=0):
    """Measured FP64 rate of the current device (see include/shweno.h): returns
    (TFLOP/s with a fused multiply-add counted 2, operations per SM clock per SM)."""
    tf, per_clk = ctypes.c_double(), ctypes.c_double()
    _check(lib().shweno_fp64_probe(op, warps_per_sm, iters, stream or None, ctypes.byref(tf),
                                   ctypes.byref(per_clk)))
    return tf.value, per_clk.value


def shweno_flag_features(h, out):
    """out: CUDA float32 tensor [cells][22]."""
    _check(lib().shweno_flag_features(h, _ptr(out)[0]), h)


def shweno_weight_deviation(h, out):
    """out: CUDA float64 tensor [cells]."""
    _check(lib().shweno_weight_deviation(h, _ptr(out)[0]), h)


def shweno_face_deviation(h, out, floor_rel=1e-9):
    """out: CUDA float64 tensor [cells]."""
    _check(lib().shweno_face_deviation(h, floor_rel, _ptr(out)[0]), h)


def shweno_mlp_forward(params, x, prob, stream=0):
    _check(lib().shweno_mlp_forward(_ptr(params)[0], _ptr(x)[0], x.shape[0], _ptr(prob)[0], stream or None))


def shweno_mlp_grad(params, x, y, pos_weight, grad, loss, stream=0):
    _check(lib().shweno_mlp_grad(_ptr(params)[0], _ptr(x)[0], _ptr(y)[0], x.shape[0], pos_weight,
                                 _ptr(grad)[0], _ptr(loss)[0], stream or None))


def shweno_mlp_adam(params, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=0):
    _check(lib().shweno_mlp_adam(_ptr(params)[0], _ptr(grad)[0], _ptr(m)[0], _ptr(v)[0], step, lr, beta1,
                                 beta2, eps, stream or None))


def shweno_set_flag_net(h, params, threshold):
    p, dev = _ptr(params)
    _check(lib().shweno_set_flag_net(h, p, threshold, dev), h)


def shweno_get_flags(h, out):
    p, dev = _ptr(out)
    _check(lib().shweno_get_flags(h, p, dev), h)


def shweno_destroy(h):
    if h:
        lib().shweno_destroy(h)


def shweno_last_error(h=None):
    return lib().shweno_last_error(h).decode()


class Batch:
    """Many handles advanced together (shweno_batch_*): one persistent launch, or lockstep rounds
    of one launch per phase (the default for batches of 2D problems)."""

    def __init__(self, solvers, stream=0):
        self.solvers = list(solvers)  # keeps the handles alive
        arr = (ctypes.c_void_p * len(self.solvers))(*[s.h.value for s in self.solvers])
        b = ctypes.c_void_p()
        st = lib().shweno_batch_create(arr, len(self.solvers), stream or None, ctypes.byref(b))
        if st != OK:
            raise ShwenoError(st, "shweno_batch_create failed")
        self.b = b

    def _err(self, st):
        if st != OK:
            raise ShwenoError(st, lib().shweno_batch_last_error(self.b).decode())

    def run(self, t_final, cfl, max_steps=0, check=True):
        n = len(self.solvers)
        tf = (ctypes.c_double * n)(*([t_final] * n if np.isscalar(t_final) else list(t_final)))
        per = (ctypes.c_int * n)()
        st = lib().shweno_batch_run(self.b, tf, cfl, max_steps, per)
        if check:
            self._err(st)
        return st, list(per)

    def autotune(self, t_final, cfl, trial_steps=3):
        n = len(self.solvers)
        tf = (ctypes.c_double * n)(*([t_final] * n if np.isscalar(t_final) else list(t_final)))
        a, b = ctypes.c_int(), ctypes.c_int()
        self._err(lib().shweno_batch_autotune(self.b, tf, cfl, trial_steps, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def set(self, tile1d=0, ctas_per_sm=0, spin_limit=0):
        self._err(lib().shweno_batch_set(self.b, tile1d, ctas_per_sm, spin_limit))

    def set_mode(self, mode):
        """BATCH_AUTO, BATCH_PERSISTENT or BATCH_LOCKSTEP (shweno_batch_set_mode)."""
        self._err(lib().shweno_batch_set_mode(self.b, mode))

    @property
    def mode(self):
        """The mode the next run takes: BATCH_PERSISTENT or BATCH_LOCKSTEP."""
        return lib().shweno_batch_get_mode(self.b)

    def close(self):
        if self.b:
            lib().shweno_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------- convenience
def make_grid(dim, eq, nx, ny=1, x0=0.0, x1=1.0, y0=0.0, y1=1.0):
    g = shweno_grid()
    g.dim, g.eq, g.nx, g.ny, g.x0, g.x1, g.y0, g.y1 = dim, eq, nx, ny, x0, x1, y0, y1
    return g


def make_bc(kinds, inflow=None):
    b = shweno_bc()
    for k in range(4):
        b.kind[k] = kinds[k] if k < len(kinds) else 0
    if inflow is not None:
        for s in range(4):
            for q in range(4):
                b.inflow[s][q] = inflow[s][q]
    return b


def make_opts(flag_mode=0, eps=1e-6, gam=(0.994, 0.003, 0.003), charwise=False, quintic=False):
    o = shweno_opts()
    o.flag_mode, o.eps, o.charwise, o.quintic = flag_mode, eps, 1 if charwise else 0, 1 if quintic else 0
    for k in range(3):
        o.gam[k] = gam[k]
    return o


class Solver:
    """Owns one handle.  Arrays are float64 [ncomp][nx] (1D) or [ncomp][ny][nx] (2D), numpy (host)
    or torch CUDA tensors (device)."""

    def __init__(self, dim, eq, nx, ny=1, domain=(0.0, 1.0, 0.0, 1.0), bc=(0, 0, 0, 0), gamma=1.4,
                 inflow=None, flag_mode=0, eps=1e-6, stream=0, charwise=False, quintic=False):
        self.dim, self.eq, self.nx, self.ny = dim, eq, nx, (ny if dim == 2 else 1)
        self.ncomp = 1 if eq == BURGERS else (3 if dim == 1 else 4)
        self.h = shweno_create(make_grid(dim, eq, nx, ny, *domain), gamma, make_bc(bc, inflow),
                               make_opts(flag_mode, eps, charwise=charwise, quintic=quintic), stream)

    @property
    def shape(self):
        return (self.ncomp, self.nx) if self.dim == 1 else (self.ncomp, self.ny, self.nx)

    def set_state(self, st, t=0.0):
        f = lambda k: np.ascontiguousarray(st[k], dtype=np.float64) if isinstance(st[k], np.ndarray) else st[k]
        if self.dim == 1:
            shweno_set_state(self.h, f("W"), f("V"), None, None, t)
        else:
            shweno_set_state(self.h, f("W"), f("V"), f("Y"), f("Z"), t)

    def get_state(self):
        out = {k: np.empty(self.shape) for k in (("W", "V") if self.dim == 1 else ("W", "V", "Y", "Z"))}
        shweno_get_state(self.h, out["W"], out["V"], out.get("Y"), out.get("Z"))
        return out

    def step(self, dt):
        shweno_step(self.h, dt)

    def run(self, t_final, cfl):
        return shweno_run(self.h, t_final, cfl)

    def set_flags(self, flags):
        if isinstance(flags, np.ndarray):
            flags = np.ascontiguousarray(flags, dtype=np.uint8)
        shweno_set_flags(self.h, flags)

    def time(self):
        return shweno_get_time(self.h)

    def close(self):
        if self.h:
            shweno_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
