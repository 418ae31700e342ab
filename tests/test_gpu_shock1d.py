"""GPU regression suite on the 1D shock examples of Section 5: the CUDA path through the C ABI
against the oracle on Example 5.4 (Shu-Osher, N = 400), Example 5.6 (blast waves between
reflective walls, N = 400, T = 0.038) and Example 5.5 (turbulence interaction, N = 1500, first
unit of time); at the paper's N = 800 the blast waves leave the physical range (no positivity
limiter in the scheme) and the library stops at the same step as the oracle.

Behind the Shu-Osher shock the componentwise scheme amplifies rounding differences between two
correct FP64 implementations by about 100x per 0.2 time units (measured: rel L1 of W 2e-16 at
t = 0.05, 4e-13 at 0.4, 7e-11 at 0.6, 4e-6 at 1.8; the characteristic-wise option stays at 1e-15
to t = 0.6).  The parity bar therefore holds to t = 0.4.  The full run to T = 1.8 is held to the
oracle's own drift: the oracle run from initial data perturbed by a relative 1e-15 (three seeded
sign patterns) ends 4e-7 ... 5e-6 (rel L1) from the unperturbed oracle run, and the library must
end within 10x the largest of those from it."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2304_09724_gb300 import shweno as S
from paper_2304_09724_gb300 import workloads as WL
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("maker,T", [(lambda: WL.shu_osher(400), 0.4),
                                     (lambda: WL.blast_waves(400), 0.038),
                                     (lambda: WL.turbulence_interaction(1500), 1.0)])
def test_shock_examples_parity(maker, T):
    wl = maker()
    g, o, (t, n), (t_o, n_o) = U.run_both(wl, T)
    assert n == n_o and t == t_o
    U.check(g, o, U.fields(wl), shocked=True, what=wl.name, wl=wl)


def test_shu_osher_full_run_within_the_oracles_own_drift():
    wl = WL.shu_osher(400)
    g, o, (t, n), (t_o, n_o) = U.run_both(wl, wl.t_final)
    assert n == n_o and t == t_o == wl.t_final
    P = U.problem_of(wl)
    drift = []
    for seed in (1, 2, 3):
        rng = np.random.default_rng(seed)
        st = {k: v * (1.0 + 1e-15 * rng.choice([-1.0, 1.0], size=v.shape)) for k, v in wl.state.items()}
        op, n_p, _ = O.run(P, st, wl.t_final, wl.cfl)
        assert n_p == n_o
        drift.append(U.rel_l1(op["W"], o["W"]))
    rel = U.rel_l1(g["W"], o["W"])
    assert rel <= 10.0 * max(drift), (rel, drift)


def test_blast_waves_conservation_on_gpu():
    wl = WL.blast_waves(400)
    sol = U.solver_of(wl)
    sol.set_state(wl.state)
    sol.run(wl.t_final, wl.cfl)
    g = sol.get_state()
    sol.close()
    for q in (0, 2):
        assert abs(g["W"][q].sum() - wl.state["W"][q].sum()) < 1e-12 * np.abs(wl.state["W"][q]).sum()


def test_blast_waves_800_nonphysical_like_the_oracle():
    wl = WL.blast_waves(800)
    with pytest.raises(O.NonPhysical) as eo:
        O.run(U.problem_of(wl), wl.state, wl.t_final, wl.cfl)
    sol = U.solver_of(wl)
    sol.set_state(wl.state)
    with pytest.raises(S.ShwenoError) as eg:
        sol.run(wl.t_final, wl.cfl)
    assert eg.value.status == S.E_NONPHYSICAL
    t, n = sol.time()
    assert n == eo.value.steps and t == pytest.approx(eo.value.t, rel=1e-12)
    g = sol.get_state()
    sol.close()
    U.check(g, eo.value.state, U.fields(wl), shocked=True, what="blast waves 800 last good state", wl=wl)
