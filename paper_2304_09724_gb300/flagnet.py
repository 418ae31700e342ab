"""Training and evaluation driver of the learned troubled-cell flag.

The network and its training step run in the library's own CUDA kernels (shweno_mlp_forward,
shweno_mlp_grad, shweno_mlp_adam through the C ABI); PyTorch only holds the device buffers.
Labels come from the plain scheme itself: seeded random four-quadrant Riemann problems (rho ~
U[0.1,2], u, v ~ U[-1,1], p ~ U[0.1,2]) at 256 x 256, seeded smooth periodic flows of every
amplitude from 1e-10 to 0.3 at 128^2 ... 1024^2 (workloads.smooth_flow_2d) and seeded smooth
Gaussian bumps at 256^2 ... 1024^2 (workloads.smooth_bumps_2d) are advanced with the
always-nonlinear scheme; at several snapshots every cell gets the features of
shweno_flag_features and the label 1 if shweno_face_deviation (floor FACE_FLOOR) exceeds
DELTA_FACE: the nonlinear weights of some reconstruction anchored on the cell move its end values
by more than that fraction of the range of its cell averages plus FACE_FLOOR of its own average.
(label="weights" keeps the earlier label: shweno_weight_deviation above 0.05, the weights
themselves deviating from the linear ones by more than 5 %.)

    python -m paper_2304_09724_gb300.flagnet --out flagnet_weights.npz
"""
from __future__ import annotations

import argparse
import math
import os
import time

import numpy as np

from . import shweno as S
from . import workloads as WL

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "flagnet_weights.npz")
NIN, NH = S.FLAG_FEATURES, 32


def init_params(seed):
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0, math.sqrt(2 / NIN), (NH, NIN)), np.zeros(NH),
             rng.normal(0, math.sqrt(2 / NH), (NH, NH)), np.zeros(NH),
             rng.normal(0, math.sqrt(1 / NH), NH), np.zeros(1)]
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


DELTA_FACE = 1e-3    # label threshold of the face-value form
FACE_FLOOR = 1e-3    # floor of its scale, relative to the cell's own average
DELTA_WEIGHTS = 0.05  # label threshold of the weight form


def snapshot_data(seed, n=256, times=(0.0, 0.05, 0.1, 0.175, 0.25), label="face", delta=None,
                  kind="quadrants", keep=1.0, kmax=4):
    """(features [k*cells][22], labels [k*cells], deviations) of one seeded problem (CUDA tensors):
    kind "quadrants" a four-quadrant Riemann problem, "smooth" a smooth periodic flow
    (workloads.smooth_flow_2d), "bumps" smooth Gaussian bumps (workloads.smooth_bumps_2d); keep < 1
    keeps that fraction of each snapshot's cells (seeded).
    A problem whose plain run leaves the physical range keeps the snapshots taken before."""
    if delta is None:
        delta = DELTA_FACE if label == "face" else DELTA_WEIGHTS
    import torch

    if kind == "quadrants":
        wl = WL.riemann2d(n, WL.random_quadrants(seed))
    elif kind == "smooth":
        wl = WL.smooth_flow_2d(seed, n, kmax=kmax)
    else:
        wl = WL.smooth_bumps_2d(seed, n)
    sol = S.Solver(2, S.EULER, n, n, wl.domain, wl.bc, flag_mode=0)
    sol.set_state(wl.state)
    X, D = [], []
    for t in times:
        if t > 0:
            try:
                sol.run(t, wl.cfl)
            except S.ShwenoError as e:
                if e.status != S.E_NONPHYSICAL:
                    raise
                break
        x = torch.empty((n * n, NIN), dtype=torch.float32, device="cuda")
        d = torch.empty(n * n, dtype=torch.float64, device="cuda")
        S.shweno_flag_features(sol.h, x)
        if label == "face":
            S.shweno_face_deviation(sol.h, d, FACE_FLOOR)
        else:
            S.shweno_weight_deviation(sol.h, d)
        if keep < 1.0:
            g = torch.Generator(device="cuda")
            g.manual_seed(seed * 7919 + len(X))
            idx = torch.randperm(n * n, device="cuda", generator=g)[: int(keep * n * n)]
            x, d = x[idx], d[idx]
        X.append(x)
        D.append(d)
    sol.close()
    X, D = torch.cat(X), torch.cat(D)
    return X, (D > delta).float(), D


def dataset(seeds, **kw):
    import torch

    parts = [snapshot_data(s, **kw) for s in seeds]
    return torch.cat([p[0] for p in parts]), torch.cat([p[1] for p in parts])


SMOOTH_SIZES = (128, 256, 512, 1024)
BUMP_SIZES = (256, 512, 1024)


def smooth_dataset(seeds, times=(0.0, 0.05), **kw):
    """Smooth periodic flows at the mesh sizes SMOOTH_SIZES in turn (every other one with
    wavenumbers up to 8 instead of 4), each snapshot thinned to about 65536 cells: the fine-mesh
    smooth data, of every amplitude, that the quadrant problems at 256^2 lack."""
    import torch

    parts = []
    for k, s in enumerate(seeds):
        n = SMOOTH_SIZES[k % len(SMOOTH_SIZES)]
        parts.append(snapshot_data(s, n=n, times=times, kind="smooth", keep=min(1.0, 65536 / (n * n)),
                                   kmax=8 if k % 2 else 4, **kw))
    return torch.cat([p[0] for p in parts]), torch.cat([p[1] for p in parts])


def bump_dataset(seeds, times=(0.0, 0.05), **kw):
    """Smooth localised structures (workloads.smooth_bumps_2d: Gaussian bumps of random width and
    amplitude) at the mesh sizes BUMP_SIZES in turn, each snapshot thinned to about 65536 cells:
    steep but resolved smooth features, which the quadrant problems only show next to jumps."""
    import torch

    parts = []
    for k, s in enumerate(seeds):
        n = BUMP_SIZES[k % len(BUMP_SIZES)]
        parts.append(snapshot_data(s, n=n, times=times, kind="bumps", keep=min(1.0, 65536 / (n * n)), **kw))
    return torch.cat([p[0] for p in parts]), torch.cat([p[1] for p in parts])


def train(X, y, epochs=6, batch=16384, lr=2e-3, seed=0, log=None, history=None):
    """Adam on the weighted BCE with the library's kernels; returns (parameters (CUDA), positive-class
    weight).  history (a list), if given, receives the mean training loss of every epoch."""
    import torch

    n = X.shape[0]
    npos = float(y.sum().item())
    pw = (n - npos) / max(npos, 1.0)
    params = torch.from_numpy(init_params(seed)).cuda()
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    grad = torch.zeros_like(params)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    step = 0
    for ep in range(epochs):
        perm = torch.randperm(n, device="cuda", generator=gen)
        tot = 0.0
        for b0 in range(0, n, batch):
            idx = perm[b0:b0 + batch]
            xb, yb = X[idx].contiguous(), y[idx].contiguous()
            S.shweno_mlp_grad(params, xb, yb, pw, grad, loss)
            step += 1
            S.shweno_mlp_adam(params, grad, m, v, step, lr)
            tot += float(loss.item()) * xb.shape[0]
        if log:
            log(f"epoch {ep}: mean loss {tot / n:.4f}")
        if history is not None:
            history.append(tot / n)
    return params, pw


def mean_loss(params, X, y, pw):
    """Weighted BCE of the network on (X, y), from the library's gradient kernel."""
    import torch

    grad = torch.empty_like(params)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    S.shweno_mlp_grad(params, X, y, pw, grad, loss)
    return float(loss.item())


def probabilities(params, X):
    import torch

    p = torch.empty(X.shape[0], dtype=torch.float32, device="cuda")
    S.shweno_mlp_forward(params, X, p)
    return p


def threshold_for_recall(params, X, y, recall=0.999):
    """Largest threshold whose recall on (X, y) is at least `recall`."""
    import torch

    p = probabilities(params, X)
    pos = torch.sort(p[y > 0.5]).values
    if pos.numel() == 0:
        return 0.5
    k = int(math.floor((1.0 - recall) * pos.numel()))
    thr = float(pos[k].item()) * (1.0 - 1e-6)
    return min(max(thr, 1e-6), 1.0 - 1e-6)


def evaluate(params, thr, X, y):
    p = probabilities(params, X)
    pred = p > thr
    pos = y > 0.5
    tp = float((pred & pos).sum().item())
    return {"recall": tp / max(float(pos.sum().item()), 1.0), "flagged": float(pred.float().mean().item()),
            "positives": float(pos.float().mean().item())}


def save(path, params, thr, meta):
    np.savez(path, params=params.cpu().numpy(), threshold=np.float64(thr), **{k: np.asarray(v) for k, v in meta.items()})


def load(path=DEFAULT_WEIGHTS):
    z = np.load(path)
    return z["params"].astype(np.float32), float(z["threshold"])


def main():
    """The committed network's recipe: four-quadrant problems (seeds 100-111, 256^2, five
    snapshots), smooth flows (seeds 0-29) and smooth bumps (seeds 0-23) for training, seeds
    500-503, 1000-1009 and 1000-1007 for validation, face-value labels, 15 epochs of Adam, the
    threshold that keeps recall 0.995 on the validation data (the 3x3 dilation of the flags is the
    margin beyond it)."""
    import torch

    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    ap.add_argument("--train-seeds", type=int, default=12)
    ap.add_argument("--smooth-seeds", type=int, default=30)
    ap.add_argument("--bump-seeds", type=int, default=24)
    ap.add_argument("--val-seeds", type=int, default=4)
    ap.add_argument("--val-smooth-seeds", type=int, default=10)
    ap.add_argument("--val-bump-seeds", type=int, default=8)
    ap.add_argument("--epochs", type=int, default=15)
    ap.add_argument("--recall", type=float, default=0.995)
    args = ap.parse_args()
    torch.cuda.set_device(0)
    t0 = time.time()
    parts = [dataset(range(100, 100 + args.train_seeds)), smooth_dataset(range(0, args.smooth_seeds)),
             bump_dataset(range(0, args.bump_seeds))]
    Xt, yt = torch.cat([p[0] for p in parts]), torch.cat([p[1] for p in parts])
    parts = [dataset(range(500, 500 + args.val_seeds)), smooth_dataset(range(1000, 1000 + args.val_smooth_seeds)),
             bump_dataset(range(1000, 1000 + args.val_bump_seeds))]
    Xv, yv = torch.cat([p[0] for p in parts]), torch.cat([p[1] for p in parts])
    t1 = time.time()
    params, pw = train(Xt, yt, epochs=args.epochs, log=print)
    torch.cuda.synchronize()
    t2 = time.time()
    thr = threshold_for_recall(params, Xv, yv, args.recall)
    ev_t, ev_v = evaluate(params, thr, Xt, yt), evaluate(params, thr, Xv, yv)
    print(f"data {t1 - t0:.1f}s ({Xt.shape[0]} train / {Xv.shape[0]} val samples), train {t2 - t1:.1f}s, "
          f"pos_weight {pw:.2f}, threshold {thr:.4g}")
    print("train", ev_t)
    print("val", ev_v)
    save(args.out, params, thr, {"val_recall": ev_v["recall"], "val_flagged": ev_v["flagged"],
                                 "val_positives": ev_v["positives"], "pos_weight": pw})
    print("saved", args.out)


if __name__ == "__main__":
    main()
