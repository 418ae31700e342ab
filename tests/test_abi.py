"""Host-side checks of the C ABI (no GPU needed, no compute calls): the library builds, loads,
exports every function include/shweno.h declares, and rejects invalid arguments before it
touches the device."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2304_09724_gb300 import build as libbuild
from paper_2304_09724_gb300 import shweno as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:shweno_status|const char\*|int)\s+(shweno_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built():
    return libbuild.build()


def test_library_exports_every_declared_function(built):
    decl = declared_functions()
    assert len(decl) >= 10
    out = subprocess.check_output(["nm", "-D", "--defined-only", built]).decode()
    exported = set(re.findall(r" T (shweno_\w+)$", out, flags=re.M))
    missing = [n for n in decl if n not in exported]
    assert not missing, missing
    L = S.lib()
    for n in decl:
        assert hasattr(L, n)
    assert set(S.EXPORTS) <= set(decl)


def test_invalid_arguments_rejected_before_device_use(built):
    L = S.lib()
    h = ctypes.c_void_p()
    bad = [
        S.make_grid(3, 1, 16, 16),            # dim
        S.make_grid(2, 1, 2, 16),             # too few cells
        S.make_grid(1, 7, 16),                # equation
        S.make_grid(1, 1, 16, x0=1.0, x1=1.0),  # empty domain
    ]
    for g in bad:
        s = L.shweno_create(ctypes.byref(g), 1.4, ctypes.byref(S.make_bc((0, 0, 0, 0))), None, None, ctypes.byref(h))
        assert s == S.E_INVALID
        assert h.value is None
        assert S.shweno_last_error(None) != ""
    # unpaired periodic sides, DMR kinds on the wrong side, bad gamma, bad weights
    g = S.make_grid(2, 1, 16, 16)
    for bc, gamma, opts in [((0, 1, 0, 0), 1.4, None), ((4, 1, 1, 1), 1.4, None),
                            ((1, 1, 1, 1), 0.9, None), ((1, 1, 1, 1), 1.4, S.make_opts(0, 1e-6, (0.5, 0.5, 0.5))),
                            ((1, 1, 1, 1), 1.4, S.make_opts(5))]:
        s = L.shweno_create(ctypes.byref(g), gamma, ctypes.byref(S.make_bc(bc)),
                            ctypes.byref(opts) if opts is not None else None, None, ctypes.byref(h))
        assert s == S.E_INVALID, (bc, gamma)
    # FP64 probe: operation, warps per SM, iteration count and output pointer checked before any launch
    tf = ctypes.c_double()
    assert L.shweno_fp64_probe(4, 4, 100, None, ctypes.byref(tf), None) == S.E_INVALID
    assert L.shweno_fp64_probe(-1, 4, 100, None, ctypes.byref(tf), None) == S.E_INVALID
    assert L.shweno_fp64_probe(0, 0, 100, None, ctypes.byref(tf), None) == S.E_INVALID
    assert L.shweno_fp64_probe(0, 33, 100, None, ctypes.byref(tf), None) == S.E_INVALID
    assert L.shweno_fp64_probe(0, 4, 0, None, ctypes.byref(tf), None) == S.E_INVALID
    assert L.shweno_fp64_probe(0, 4, 100, None, None, None) == S.E_INVALID
    # null handle
    assert L.shweno_step(None, 0.1) == S.E_INVALID
    assert L.shweno_destroy(None) == S.OK
    # batch entry points: a null batch or an empty handle list is refused before any device use
    b = ctypes.c_void_p()
    assert L.shweno_batch_create(None, 1, None, ctypes.byref(b)) == S.E_INVALID
    assert L.shweno_batch_create((ctypes.c_void_p * 1)(None), 0, None, ctypes.byref(b)) == S.E_INVALID
    assert L.shweno_batch_set_mode(None, S.BATCH_LOCKSTEP) == S.E_INVALID
    assert L.shweno_batch_get_mode(None) == -1
    assert L.shweno_batch_set(None, 256, 1, 0) == S.E_INVALID
    assert L.shweno_batch_destroy(None) == S.OK


def test_binding_raises_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(S, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(S, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        S.lib()
