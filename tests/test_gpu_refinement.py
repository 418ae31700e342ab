"""Design order of the library under mesh refinement (Example 5.8): the isentropic vortex on the
periodic box (0, 10)^2 at 128^2, 256^2 and 512^2, run with the plain scheme to T = 2, where the
exact solution is the vortex translated by (2, 2).  The density L1 and L-infinity errors against
the exact cell averages must fall at the scheme's fifth order: observed order at least 4.7 over
128^2 -> 512^2 (Table 5.4 prints 4.82-5.00 for the finest pairs it shows)."""
import math

import numpy as np
import pytest

from paper_2304_09724_gb300 import shweno as S
from paper_2304_09724_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

T = 2.0


def errors(n):
    wl = WL.vortex(n)
    sol = S.Solver(2, S.EULER, n, n, wl.domain, wl.bc)
    sol.set_state(wl.state)
    t, _ = sol.run(T, wl.cfl)
    e = sol.get_state()["W"][0] - wl.exact(T)[0]
    sol.close()
    assert t == T
    return float(np.mean(np.abs(e))), float(np.max(np.abs(e)))


def test_vortex_design_order_128_to_512():
    e = {n: errors(n) for n in (128, 256, 512)}
    for k, name in enumerate(("L1", "Linf")):
        order = math.log(e[128][k] / e[512][k]) / math.log(4.0)
        assert order >= 4.7, (name, order, e)
        for a, b in ((128, 256), (256, 512)):
            assert math.log(e[a][k] / e[b][k]) / math.log(2.0) >= 4.4, (name, a, b, e)
