"""GPU checks of the learned troubled-cell flag: features, labels and the network kernels
(forward, gradient, Adam) against the FP64 oracle; the learned-mode step against the oracle given
the same flags; the trained network's recall and solution deviation."""
import os

import numpy as np
import pytest

from oracle import mlp_oracle as M
from oracle import oracle as O
from paper_2304_09724_gb300 import flagnet as F
from paper_2304_09724_gb300 import shweno as S
from paper_2304_09724_gb300 import workloads as WL
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


def _torch():
    import torch

    torch.cuda.set_device(0)
    return torch


def test_features_and_deviation_match_oracle():
    torch = _torch()
    wl = WL.riemann2d(40, WL.random_quadrants(7))
    sol = U.solver_of(wl)
    sol.set_state(wl.state)
    sol.run(0.03, wl.cfl)
    st = sol.get_state()
    x = torch.empty((40 * 40, 22), dtype=torch.float32, device="cuda")
    d = torch.empty(40 * 40, dtype=torch.float64, device="cuda")
    fd = torch.empty(40 * 40, dtype=torch.float64, device="cuda")
    S.shweno_flag_features(sol.h, x)
    S.shweno_weight_deviation(sol.h, d)
    S.shweno_face_deviation(sol.h, fd, 1e-9)
    t, _ = sol.time()
    sol.close()
    P = U.problem_of(wl)
    fo = O.features2d(P, st, t)
    do = O.weight_deviation2d(P, st, t).ravel()
    np.testing.assert_allclose(x.cpu().numpy(), fo, rtol=2e-6, atol=2e-6)
    dg = d.cpu().numpy()
    np.testing.assert_allclose(dg, do, rtol=1e-9, atol=1e-12)
    delta = 0.05
    tie = np.abs(do - delta) < 1e-9
    assert np.array_equal((dg > delta)[~tie], (do > delta)[~tie])
    # face-value label: the two sides round p - p1 differently, which matters only where the
    # deviation is at rounding level (about 1e-7 of the scale); the labels agree off ties
    fg, fo_ = fd.cpu().numpy(), O.face_deviation2d(P, st, t).ravel()
    np.testing.assert_allclose(fg, fo_, rtol=1e-8, atol=1e-6)
    assert fo_.max() > 0.1
    tie = np.abs(fo_ - F.DELTA_FACE) < 1e-6
    assert np.array_equal((fg > F.DELTA_FACE)[~tie], (fo_ > F.DELTA_FACE)[~tie])
    # a larger floor of the scale (changes measured against 1e-3 of the cell's own average too)
    sol = U.solver_of(wl)
    sol.set_state(st, t)
    S.shweno_face_deviation(sol.h, fd, 1e-3)
    sol.close()
    np.testing.assert_allclose(fd.cpu().numpy(), O.face_deviation2d(P, st, t, floor_rel=1e-3).ravel(),
                               rtol=1e-8, atol=1e-9)


def test_network_kernels_match_oracle():
    torch = _torch()
    rng = np.random.default_rng(1)
    n = 1000  # several 128-sample CTAs and a ragged tail
    theta = M.init(5) * 1.3
    X = rng.normal(size=(n, 22))
    y = (rng.random(n) < 0.25).astype(float)
    pw = 3.0
    tp = torch.from_numpy(theta.astype(np.float32)).cuda()
    Xd = torch.from_numpy(X.astype(np.float32)).cuda()
    yd = torch.from_numpy(y.astype(np.float32)).cuda()
    # the oracle sees exactly the FP32-rounded inputs
    th32, X32 = theta.astype(np.float32).astype(np.float64), X.astype(np.float32).astype(np.float64)
    prob = torch.empty(n, dtype=torch.float32, device="cuda")
    S.shweno_mlp_forward(tp, Xd, prob)
    np.testing.assert_allclose(prob.cpu().numpy(), M.prob(th32, X32), rtol=2e-5, atol=1e-6)
    grad = torch.empty_like(tp)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    S.shweno_mlp_grad(tp, Xd, yd, pw, grad, loss)
    go = M.grad(th32, X32, y, pw)
    gg = grad.cpu().numpy()
    assert np.max(np.abs(gg - go)) <= 1e-4 * np.max(np.abs(go))
    assert float(loss.item()) == pytest.approx(M.loss(th32, X32, y, pw), rel=1e-5)
    m = torch.zeros_like(tp)
    v = torch.zeros_like(tp)
    S.shweno_mlp_adam(tp, grad, m, v, 1, 1e-3)
    t1, _, _ = M.adam(th32, gg.astype(np.float64), np.zeros_like(th32), np.zeros_like(th32), 1, 1e-3)
    np.testing.assert_allclose(tp.cpu().numpy(), t1, rtol=1e-6, atol=1e-7)


def test_training_from_scratch_on_the_gpu():
    """A fresh network trained end to end by the library's forward, gradient and Adam kernels on
    labels the plain scheme generates (seeded four-quadrant problems at 96 x 96): the weighted
    cross-entropy falls at least 5x, and at the threshold that keeps recall 0.999 on the training
    data the held-out recall is at least 0.95."""
    torch = _torch()
    X, y = F.dataset([300, 301, 302, 303], n=96, times=(0.0, 0.05, 0.1))
    Xv, yv = F.dataset([950, 951], n=96, times=(0.0, 0.05, 0.1))
    assert 0.0 < float(y.mean().item()) < 1.0
    hist = []
    params, pw = F.train(X, y, epochs=30, batch=4096, seed=3, history=hist)
    start = F.mean_loss(torch.from_numpy(F.init_params(3)).cuda(), X, y, pw)
    end = F.mean_loss(params, X, y, pw)
    assert start / end >= 5.0, (start, end, hist)
    thr = F.threshold_for_recall(params, X, y, 0.999)
    ev = F.evaluate(params, thr, Xv, yv)
    assert ev["recall"] >= 0.95, ev


def test_learned_mode_step_matches_oracle_with_the_same_flags():
    torch = _torch()
    n = 48
    wl = WL.riemann2d(n, WL.LAX_LIU_SHOCKS)
    sol = U.solver_of(wl, flag_mode=2)
    sol.set_state(wl.state)
    params = torch.from_numpy(M.init(11).astype(np.float32)).cuda()
    # threshold at the 97th percentile of this untrained net's outputs: a few raw flags, which
    # the one-cell dilation spreads
    x = torch.empty((n * n, 22), dtype=torch.float32, device="cuda")
    S.shweno_flag_features(sol.h, x)
    p = torch.empty(n * n, dtype=torch.float32, device="cuda")
    S.shweno_mlp_forward(params, x, p)
    thr = float(torch.quantile(p, 0.97).item())
    S.shweno_set_flag_net(sol.h, params, min(max(thr, 1e-6), 1 - 1e-6))
    sol.step(0.002)
    flags = np.empty((n, n), dtype=np.uint8)
    S.shweno_get_flags(sol.h, flags)
    g = sol.get_state()
    sol.close()
    assert 0 < flags.mean() < 1
    o = O.step(U.problem_of(wl), wl.state, 0.002, flag=flags)
    U.check(g, o, "WVYZ", shocked=True, what="learned-mode step", wl=wl)


@pytest.mark.skipif(not os.path.exists(F.DEFAULT_WEIGHTS), reason="no trained flag network committed")
def test_trained_network_recall_and_solution_deviation():
    torch = _torch()
    params, thr = F.load()
    pd = torch.from_numpy(params).cuda()
    # held-out seeds: recall of the raw network on the plain scheme's labels
    X, y = F.dataset([900, 901], n=128, times=(0.0, 0.05, 0.1))
    ev = F.evaluate(pd, thr, X, y)
    # the threshold keeps recall 0.995 on the validation data; the 3x3 dilation of the flags is
    # the margin beyond it
    assert ev["recall"] >= 0.98, ev
    # learned flag vs always-nonlinear on a held-out problem: relative L1 deviation at the end
    wl = WL.riemann2d(128, WL.random_quadrants(902))
    plain = U.solver_of(wl)
    plain.set_state(wl.state)
    plain.run(0.1, wl.cfl)
    a = plain.get_state()
    plain.close()
    learned = U.solver_of(wl, flag_mode=2)
    learned.set_state(wl.state)
    S.shweno_set_flag_net(learned.h, pd, thr)
    learned.run(0.1, wl.cfl)
    b = learned.get_state()
    flags = np.empty((128, 128), dtype=np.uint8)
    S.shweno_get_flags(learned.h, flags)
    learned.close()
    dev = U.rel_l1(b["W"], a["W"])
    assert dev <= 1e-3, dev
    assert flags.mean() < 0.9


@pytest.mark.skipif(not os.path.exists(F.DEFAULT_WEIGHTS), reason="no trained flag network committed")
def test_trained_network_on_double_mach_reflection():
    """Example 5.10 at the paper's coarser mesh (480 x 120) to T = 0.2: the learned flag keeps the
    solution within 1e-3 relative L1 of the always-nonlinear scheme and flags a minority of cells."""
    torch = _torch()
    params, thr = F.load()
    pd = torch.from_numpy(params).cuda()
    wl = WL.dmr(480, 120)
    out = {}
    for mode in ("plain", "learned"):
        sol = U.solver_of(wl, flag_mode=0 if mode == "plain" else 2)
        sol.set_state(wl.state)
        if mode == "learned":
            S.shweno_set_flag_net(sol.h, pd, thr)
        sol.run(0.2, wl.cfl)
        out[mode] = sol.get_state()
        if mode == "learned":
            flags = np.empty((120, 480), dtype=np.uint8)
            S.shweno_get_flags(sol.h, flags)
        sol.close()
    dev = U.rel_l1(out["learned"]["W"], out["plain"]["W"])
    assert dev <= 1e-3, dev
    assert flags.mean() < 0.6, flags.mean()
