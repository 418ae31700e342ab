"""The seeded training-data generators of the learned flag (smooth flows of every amplitude and
smooth Gaussian bumps): the same seed gives the same bytes, every state is physical (positive
density and pressure), the smooth flows span many decades of amplitude, and the derivative
averages are the edge-value differences of the cell averages' underlying field (so a periodic
field's x-derivative averages sum to zero along every row)."""
import numpy as np

from paper_2304_09724_gb300 import workloads as WL


def _rho_p(W):
    rho = W[0]
    p = 0.4 * (W[3] - 0.5 * (W[1] ** 2 + W[2] ** 2) / rho)
    return rho, p


def test_generators_are_seeded_and_physical():
    amps = []
    for s in range(12):
        for make in (lambda: WL.smooth_flow_2d(s, 32, kmax=8), lambda: WL.smooth_bumps_2d(s, 32)):
            a, b = make(), make()
            for k in "WVYZ":
                assert np.array_equal(a.state[k], b.state[k])
            rho, p = _rho_p(a.state["W"])
            assert rho.min() > 0.0 and p.min() > 0.0
        rho, _ = _rho_p(WL.smooth_flow_2d(s, 32).state["W"])
        amps.append((rho.max() - rho.min()) / rho.mean())
    # amplitudes from nearly constant to strong waves
    assert min(amps) < 1e-6 and max(amps) > 1e-2


def test_periodic_derivative_averages_telescope():
    for make in (lambda: WL.smooth_flow_2d(3, 24), lambda: WL.smooth_bumps_2d(3, 24)):
        st = make().state
        # V = (W(x_{i+1/2}) - W(x_{i-1/2})) / dx integrated along y: sums to zero over a periodic row
        assert np.max(np.abs(st["V"].sum(axis=2))) <= 1e-9 * np.max(np.abs(st["V"])) * st["V"].shape[2]
        assert np.max(np.abs(st["Y"].sum(axis=1))) <= 1e-9 * np.max(np.abs(st["Y"])) * st["Y"].shape[1]
