"""Example 5.9 (two 2D Riemann problems of Lax and Liu, outflow sides): the four-shock problem to
T = 0.25 and the four-contact (shear) problem to T = 0.8.  Full runs against the oracle at 32 x 32;
at the paper's 400 x 400 the library's runs complete in the physical range, and the learned-flag
form stays within the accuracy it is held to against the always-nonlinear form."""
import numpy as np
import pytest

from paper_2304_09724_gb300 import flagnet as F
from paper_2304_09724_gb300 import shweno as S
from paper_2304_09724_gb300 import workloads as WL
from tests import gpu_util as U

pytestmark = pytest.mark.gpu

CASES = {"shocks": (WL.LAX_LIU_SHOCKS, 0.25), "contacts": (WL.LAX_LIU_CONTACTS, 0.8)}


@pytest.mark.parametrize("name", ["shocks", "contacts"])
def test_full_run_parity_32(name):
    states, T = CASES[name]
    wl = WL.riemann2d(32, states)
    g, o, (t, n), (t_o, n_o) = U.run_both(wl, T)
    assert n == n_o and t == t_o
    U.check(g, o, U.fields(wl), shocked=True, what=f"Example 5.9 {name} 32^2", wl=wl)


@pytest.mark.parametrize("name", ["shocks", "contacts"])
def test_paper_resolution_400_plain_and_learned(name):
    import torch

    states, T = CASES[name]
    wl = WL.riemann2d(400, states)
    out = {}
    for mode in ("plain", "learned"):
        sol = U.solver_of(wl, flag_mode=2 if mode == "learned" else 0)
        sol.set_state(wl.state)
        if mode == "learned":
            params, thr = F.load()
            S.shweno_set_flag_net(sol.h, torch.from_numpy(params).cuda(), thr)
        t, n = sol.run(T, wl.cfl)
        assert t == T and n > 0
        out[mode] = sol.get_state()
        sol.close()
        rho = out[mode]["W"][0]
        assert np.isfinite(out[mode]["W"]).all() and rho.min() > 0
    dev = np.sum(np.abs(out["learned"]["W"] - out["plain"]["W"])) / np.sum(np.abs(out["plain"]["W"]))
    assert dev <= 1e-3, dev
