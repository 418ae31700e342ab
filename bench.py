#!/usr/bin/env python
"""Throughput benchmark of the ADER-SHWENO step on a GB300: 2D Euler isentropic vortex
(Example 5.8: strength 5, centre (5,5), periodic (0,10)^2, mean state rho = u = v = p = 1),
2048 x 2048 cells, FP64, CFL 0.6.  One benchmark step = one time step of the whole path
(SHWENO reconstruction, HLLC + derivative Riemann problems, Cauchy-Kovalevskaya, Lobatto flux,
update of W, V, Y, Z, fused CFL reduction for the next step).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--n 2048]

Prints one JSON line (rank 0).  Metric: cell-updates/s (whole job).  For N > 1 (torchrun, one
process per GPU) every rank advances its own replica of the mesh ("replicas only": one mesh
needs no exchange on one GPU), and value = all ranks' cell-updates / max-over-ranks time.
--impl reference times the oracle (plain single-threaded C++) on the host cores instead, on a
bounded window of the same mesh per step.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CFL = 0.6
# FP64 peak derived from unit counts and clocks: 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
FP64_SLOTS_PER_S = 152 * 2 * 2.070e9  # FP64 thread instructions per second (DFMA, DMUL, DADD alike)
# FP64 operations (DFMA counted as 2) and FP64 thread instructions (DFMA + DMUL + DADD, each one
# pipe slot) per x-face point of xface2d, from ncu's instruction counters of the current kernel on
# the 2048^2 launch, and its DRAM bytes per point from a capture at 512^2 (traffic grows in
# proportion to the points).
FLOPS_PER_XFACE_POINT = 5028.1
FP64_INST_PER_XFACE_POINT = 2984.5
DRAM_BYTES_PER_XFACE_POINT = 308.0
BYTES_PER_CELL_UPDATE = 256  # 16 doubles read + 16 written per cell (ideal reuse)


def method_flops_per_xface_launch(n):
    """Floating-point operations of the method itself in one x-face launch of an n x n Euler mesh
    (3 (n+1) n Gauss points, (n+1)^2 corner points), counted from the formulas each step needs in
    its minimal form (a fused multiply-add counts 2, a division or square root 1): the denominator
    that would expose redundant work, beside the kernel's own executed FP64 count.  Per point:
      first pass   the 2 NC first-pass quartics of the point's column shifted to the point
                   (10 multiply-adds each; none at the middle Gauss node; a corner averages the
                   traces of two rows: two shifts and the mean);
      weights      per component of the cell: p1's coefficients (4 sums, 12 products), beta1
                   (8 products, 4 sums), beta2, beta3, tau, the three weights and one division;
      end values   per component, tangential order k and cross order p <= 4 - k of the cell: the
                   even and odd parts U_p, V_p (their nonzero terms), both ends with the weights
                   (two fused operations each; one product when V_p = 0), the small stencils'
                   terms for p <= 1;
      leading      HLLC: two primitive states, the wave speeds, S*, the star state;
      upwinding    eigenvectors at the leading term, 14 derivative vectors (difference, one
                   projection onto the acoustic wave that carries weight, its correction);
      ck           the generated Cauchy-Kovalevskaya recursion (its own term count);
      flux         four Lobatto nodes: Horner in time at the three nodes after the first (whose
                   state is the leading term), the physical flux (one division for the three later
                   nodes), the weighted sum (a corner point only evaluates the state at the last
                   node)."""
    import importlib.util

    NC = 4
    spec = importlib.util.spec_from_file_location(
        "gen_ck", os.path.join(ROOT, "paper_2304_09724_gb300", "csrc", "gen_ck.py"))
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    g = gen.Gen(2, "euler")
    g.emit("ck")
    ck = g.flops
    shift = 2 * 10  # one quartic moved to a new centre: 10 multiply-adds
    first_gauss = 2 * NC * shift * 2 / 3  # two of the three Gauss nodes need the shift
    first_corner = 2 * NC * (2 * shift + 2 * 5)
    p1_coeffs = 4 + (5 + 3 + 5 + 3 + 5)  # s, a, dv, sv; c0..c4 (three or two terms each)
    beta1, beta23, tau = 15, 4, 5
    mix = 3 + 4 * 3 + 2 + 1 + 2 + 3 + 3  # e_l, the three unnormalised weights, sum, 1/sum, A, B, C
    weights = NC * (p1_coeffs + beta1 + beta23 + tau + mix)
    end = 0
    for k in range(5):
        end += 4 + 11  # the symmetric sums, g and h with their halves
        for p in range(5 - k):
            u = 5 if p != 2 else 3
            v = 3 if p != 4 else 0
            both = 8 if p <= 1 else (4 + 1 if p < 4 else 1)
            end += u + v + both
    end *= NC
    prim = 1 + 2 + 6 + 2 + 3
    leading = 2 * prim + 4 + 4 + 8 + 14
    upwind = prim + 40 + 14 * (NC + (2 * NC - 1) + 2 * NC)
    flux = 3 * NC * 2 * 4 + 4 * 14 + (1 + 6) + 4 * NC * 2
    at_corner = NC * 2 * 4
    common = weights + end + leading + upwind + ck
    per_gauss = first_gauss + common + flux
    per_corner = first_corner + common + at_corner
    total = 3 * (n + 1) * n * per_gauss + (n + 1) ** 2 * per_corner
    parts = {"first_pass_gauss": first_gauss, "first_pass_corner": first_corner, "weights": weights,
             "end_values": end, "leading_term": leading, "upwinding": upwind, "ck": ck, "flux": flux}
    return total, {k: round(v, 1) for k, v in parts.items()}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
        except Exception:
            pass
        finally:
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if "Active" in r[5 + k] and "Not" not in r[5 + k]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(x, world, device="cuda"):
    """Maximum of x over the ranks (identity for one rank)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, cells, steps, seconds):
    """Whole-job cell-updates/s: every rank advanced `cells` cells `steps` times; the job took the
    slowest rank's time."""
    return world * cells * steps / seconds


def oracle_sample(wl, window, steps):
    """Times the oracle (single-threaded C++) on a window x window block of the mesh, `steps`
    times; returns (cell-updates/s, seconds)."""
    from oracle import oracle as O

    P = O.make_problem(2, wl.eq, wl.nx, wl.ny, *wl.domain, bc=wl.bc)
    dt = CFL / O.max_rate(P, wl.state["W"])
    i0 = wl.nx // 2 - window // 2
    t0 = time.perf_counter()
    for _ in range(steps):
        O.step2d_window(P, wl.state, dt, i0, i0, window, window)
    el = time.perf_counter() - t0
    return window * window * steps / el, el


L2_BYTES = 129e6  # GB300 L2


def workload_config(n, world):
    """The config block of the main workload, shared by both arms."""
    state_mb = 16 * n * n * 8 / 1e6
    scratch_gb = 132 * n * n * 8 / 1e9  # first-pass tables, face fluxes/states, corner states
    sizes = f"state 2x{state_mb:.0f} MB, step scratch {scratch_gb:.1f} GB"
    # every step reads the state and writes the next one, and each kernel streams the scratch the
    # previous one wrote: the bound that matters is the scratch against L2
    l2 = (f"inputs larger than L2 ({sizes})" if scratch_gb * 1e9 > L2_BYTES
          else f"working set fits in L2 ({sizes}): a small case, not the timing configuration")
    return {"workload": f"2D Euler isentropic vortex {n}x{n} (Example 5.8), FP64, CFL {CFL}, plain (nonlinear weights)",
            "parallelism": f"replicas{world}", "l2": l2}


def bench_reference(args):
    """Reference arm: the oracle on the host cores (rank 0 only)."""
    world, rank, _ = dist_init()
    if rank != 0:
        return
    from paper_2304_09724_gb300 import workloads as WL

    wl = WL.vortex(args.n)
    win = args.ref_window
    oracle_sample(wl, win, args.warmup)
    rate, el = oracle_sample(wl, win, args.steps)
    line = {
        "impl": "reference", "metric": "2D Euler cell-updates/s", "value": rate, "unit": "cell-updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * el / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.n, args.gpus),
        "cpu_baseline": {"value": rate, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} steps, each one step of a {win}x{win}-cell window of the "
                                   f"{args.n}^2 mesh (faces inside the window computed once)"},
        "e2e": {"value": rate, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def measure_form(S, torch, wl, steps, warmup, flag_net=None):
    """cell-updates/s of `steps` CFL steps (after `warmup`) of workload wl, plain or learned;
    returns (rate, state after the steps, flagged fraction or None)."""
    import numpy as np

    stream = torch.cuda.Stream()
    sol = S.Solver(2, S.EULER, wl.nx, wl.ny, wl.domain, wl.bc, inflow=wl.inflow,
                   flag_mode=2 if flag_net else 0, stream=stream.cuda_stream)
    dev = {k: torch.from_numpy(np.array(v)).cuda() for k, v in wl.state.items()}
    torch.cuda.synchronize()
    sol.set_state(dev)
    if flag_net:
        S.shweno_set_flag_net(sol.h, torch.from_numpy(flag_net[0]).cuda(), flag_net[1])
    S.shweno_advance(sol.h, warmup, CFL)
    S.shweno_sync(sol.h)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    S.shweno_advance(sol.h, steps, CFL)
    e1.record(stream)
    S.shweno_sync(sol.h)
    torch.cuda.synchronize()
    rate = wl.nx * wl.ny * steps / (e0.elapsed_time(e1) / 1000.0)
    st = sol.get_state()
    frac = None
    if flag_net:
        flags = np.empty((wl.ny, wl.nx), dtype=np.uint8)
        S.shweno_get_flags(sol.h, flags)
        frac = float(flags.mean())
    sol.close()
    return rate, st, frac


def learned_vs_plain(S, torch, WL, steps, warmup, vortex_wl):
    """The learned-flag form against the always-nonlinear form on the vortex (the main workload)
    and on the double Mach reflection at 4096 x 1024 (the learned flag's workload): rates, the
    flagged fraction and the relative L1 deviation of W after the same steps."""
    import numpy as np

    from paper_2304_09724_gb300 import flagnet as F

    net = F.load()
    out = {}
    for name, wl in (("isentropic_vortex_%dx%d" % (vortex_wl.nx, vortex_wl.ny), vortex_wl),
                     ("double_mach_reflection_4096x1024", WL.dmr(4096, 1024))):
        rp, sp, _ = measure_form(S, torch, wl, steps, warmup)
        rl, sl, frac = measure_form(S, torch, wl, steps, warmup, flag_net=net)
        dev = float(np.sum(np.abs(sl["W"] - sp["W"])) / np.sum(np.abs(sp["W"])))
        out[name] = {"plain": rp, "learned": rl, "speedup": rl / rp, "flagged_fraction": frac,
                     "rel_l1_vs_plain_after_steps": dev, "steps": steps}
    return out


def _batch_tools(S, torch):
    """Helpers of the batched measurements: handles from workloads, cell-updates since a
    snapshot, one timed batch run, the handles advanced one after another."""

    def make(wls, learned=False, net=None):
        sols = []
        for wl in wls:
            s = S.Solver(wl.dim, wl.eq, wl.nx, wl.ny, wl.domain, wl.bc, inflow=wl.inflow,
                         flag_mode=2 if learned else 0)
            s.set_state(wl.state)
            if learned:
                S.shweno_set_flag_net(s.h, torch.from_numpy(net[0]).cuda(), net[1])
            sols.append(s)
        torch.cuda.synchronize()
        return sols

    def updates(sols, before):
        return sum(s.nx * s.ny * (s.time()[1] - b) for s, b in zip(sols, before))

    def timed_batch(sols, T, steps, tune, mode=None):
        b = S.Batch(sols)
        if mode is not None:
            b.set_mode(mode)
        tuned = b.autotune(T, CFL, trial_steps=2) if tune else None
        before = [s.time()[1] for s in sols]
        torch.cuda.synchronize()
        with ClockSampler(torch.cuda.current_device()) as clk:
            t0 = time.perf_counter()
            st, per = b.run(T, CFL, max_steps=steps, check=False)
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
        n = updates(sols, before)
        ran = "lockstep" if b.mode == S.BATCH_LOCKSTEP else "persistent"
        b.close()
        return n / el, el, tuned, per, clk.summary(), ran

    def timed_solo(sols, steps):
        before = [s.time()[1] for s in sols]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for s in sols:
            S.shweno_advance(s.h, steps, CFL)
        for s in sols:
            try:
                S.shweno_sync(s.h)
            except S.ShwenoError:
                pass
        el = time.perf_counter() - t0
        return updates(sols, before) / el, el

    return make, updates, timed_batch, timed_solo


def batched_1d(S, torch, WL, steps):
    """512 seeded 1D Riemann problems (rho ~ U[0.1,2], u ~ U[-1,1], p ~ U[0.1,10], jump at 1/2,
    outflow, N ~ U{400..16384}, end time 0.15) in one persistent launch with autotuned tiles,
    `steps` steps per problem, against the same handles advanced one after another."""
    make, _, timed_batch, timed_solo = _batch_tools(S, torch)
    wls = [WL.random_riemann1d(s) for s in range(512)]
    sols = make(wls)
    rate_b, el_b, tuned, per, clk, _ = timed_batch(sols, 0.15, steps, True)
    for s in sols:
        s.close()
    sols = make(wls)
    rate_s, el_s = timed_solo(sols, steps)
    for s in sols:
        s.close()
    return {"workload": "512 1D Euler Riemann problems, N ~ U{400..16384}, FP64, CFL 0.6",
            "cells": int(sum(w.nx for w in wls)), "steps_per_problem": steps,
            "batch_cell_updates_per_s": rate_b, "batch_s": el_b,
            "per_instance_cell_updates_per_s": rate_s, "per_instance_s": el_s, "speedup": rate_b / rate_s,
            "autotuned": {"tile1d": tuned[0], "ctas_per_sm": tuned[1]},
            "nonphysical_problems": int(sum(1 for x in per if x == S.E_NONPHYSICAL)), "clocks": clk}


def batched_2d(S, torch, WL, steps, problems):
    """`problems` seeded four-quadrant 2D Riemann problems (rho ~ U[0.1,2], u, v ~ U[-1,1],
    p ~ U[0.1,2], sides 512..2048, end time 0.25): `steps` steps per problem, plain and learned
    flag in the default mode (lockstep rounds for a batch of 2D problems) and plain in one
    persistent launch, against the plain handles advanced one after another (each on its own
    stream)."""
    import numpy as np

    from paper_2304_09724_gb300 import flagnet as F

    make, _, timed_batch, timed_solo = _batch_tools(S, torch)
    net = F.load()
    wls = [WL.random_riemann2d(s) for s in range(problems)]
    res = {"workload": f"{problems} 2D Euler four-quadrant Riemann problems, sides 512..2048, FP64, CFL 0.6",
           "problems": len(wls), "cells": int(sum(w.nx * w.ny for w in wls)), "steps_per_problem": steps}
    for mode in ("plain", "learned", "plain_persistent"):
        sols = make(wls, learned=(mode == "learned"), net=net)
        r, el, _, per, clk, ran = timed_batch(sols, 0.25, steps, False,
                                              S.BATCH_PERSISTENT if mode == "plain_persistent" else None)
        res[f"batch_{mode}_mode"] = ran
        res[f"batch_{mode}_cell_updates_per_s"] = r
        res[f"batch_{mode}_s"] = el
        res[f"batch_{mode}_clocks"] = clk
        res[f"nonphysical_problems_{mode}"] = int(sum(1 for x in per if x == S.E_NONPHYSICAL))
        if mode == "learned":
            fr = []
            for s in sols:
                fl = np.empty((s.ny, s.nx), dtype=np.uint8)
                S.shweno_get_flags(s.h, fl)
                fr.append(fl.mean())
            res["learned_flagged_fraction"] = float(np.mean(fr))
        for s in sols:
            s.close()
    sols = make(wls)
    r, el = timed_solo(sols, steps)
    for s in sols:
        s.close()
    res["per_instance_plain_cell_updates_per_s"] = r
    res["per_instance_plain_s"] = el
    res["batch_plain_vs_per_instance"] = res["batch_plain_cell_updates_per_s"] / r
    res["batch_learned_vs_per_instance"] = res["batch_learned_cell_updates_per_s"] / r
    res["batch_plain_persistent_vs_per_instance"] = res["batch_plain_persistent_cell_updates_per_s"] / r
    return res


def bench_batched_full(args):
    """Opt-in suite (--suite batched-full): the 512 seeded 1D Riemann problems of the batch run to
    their end time T = 0.15 in one persistent launch (autotuned), every problem with its own CFL
    step: wall time, cell-updates/s, steps per problem, the problems that leave the physical range.
    (tests/test_gpu_batch_oracle.py holds problems of this set to the oracle at T = 0.15.)"""
    import numpy as np
    import torch

    from paper_2304_09724_gb300 import shweno as S
    from paper_2304_09724_gb300 import workloads as WL

    torch.cuda.set_device(0)
    make, updates, _, _ = _batch_tools(S, torch)
    wls = [WL.random_riemann1d(s) for s in range(512)]
    sols = make(wls)
    b = S.Batch(sols)
    tuned = b.autotune(0.15, CFL, trial_steps=2)
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        t0 = time.perf_counter()
        st, per = b.run(0.15, CFL, check=False)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
    b.close()
    steps = np.array([s.time()[1] for s in sols])
    tend = np.array([s.time()[0] for s in sols])
    n_upd = updates(sols, [0] * len(sols))
    for s_ in sols:
        s_.close()
    ok = [x == S.OK for x in per]
    print(json.dumps({"suite": "batched-full", "workload": "512 1D Euler Riemann problems to T = 0.15, N ~ U{400..16384}",
                      "status": int(st), "seconds": el, "cell_updates": int(n_upd), "cell_updates_per_s": n_upd / el,
                      "steps_per_problem": {"min": int(steps.min()), "mean": float(steps.mean()), "max": int(steps.max())},
                      "reached_T": int(sum(1 for k in range(len(ok)) if ok[k] and tend[k] == 0.15)),
                      "nonphysical_problems": int(sum(1 for x in per if x == S.E_NONPHYSICAL)),
                      "autotuned": {"tile1d": tuned[0], "ctas_per_sm": tuned[1]}, "clocks": clk.summary(),
                      "dtype": "f64", "data": "synthetic"}), flush=True)


def bench_batched(args):
    """Opt-in suite (--suite batched): the two batched workloads with --steps steps per problem."""
    import torch

    from paper_2304_09724_gb300 import shweno as S
    from paper_2304_09724_gb300 import workloads as WL

    torch.cuda.set_device(0)
    out = {"suite": "batched", "steps_per_problem": args.steps, "dtype": "f64", "data": "synthetic",
           "batched_1d_riemann_512": batched_1d(S, torch, WL, args.steps),
           "batched_2d_quadrants": batched_2d(S, torch, WL, args.steps, args.c5_problems)}
    print(json.dumps(out), flush=True)


def bench_gpu(args):
    import numpy as np
    import torch

    from paper_2304_09724_gb300 import shweno as S
    from paper_2304_09724_gb300 import workloads as WL

    world, rank, local = dist_init()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    barrier = (lambda: __import__("torch.distributed").distributed.barrier()) if world > 1 else (lambda: None)

    n = args.n
    wl = WL.vortex(n)
    cells = wl.nx * wl.ny
    stream = torch.cuda.Stream()
    sol = S.Solver(2, S.EULER, n, n, wl.domain, wl.bc, stream=stream.cuda_stream)
    dev = {k: torch.from_numpy(np.array(v)).cuda() for k, v in wl.state.items()}
    torch.cuda.synchronize()  # the copies ran on the default stream; the solver uses `stream`
    sol.set_state(dev)
    torch.cuda.synchronize()

    # warm-up (W >= 3 steps), then K timed steps with per-kernel events
    S.shweno_advance(sol.h, args.warmup, CFL)
    S.shweno_sync(sol.h)
    S.shweno_set_timing(sol.h, True)
    S.shweno_get_timing(sol.h)  # clear
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        S.shweno_advance(sol.h, args.steps, CFL)
        e1.record(stream)
        S.shweno_sync(sol.h)
        torch.cuda.synchronize()
    barrier()
    ms = reduce_max(e0.elapsed_time(e1), world)
    kernel_ms, timed_steps = S.shweno_get_timing(sol.h)
    S.shweno_set_timing(sol.h, False)
    clocks = clk.summary()
    sec = ms / 1000.0
    value = job_value(world, cells, args.steps, sec)

    # end to end through the C ABI with host buffers: per step, copy the state in from pinned
    # host memory, take one CFL step, copy the state out
    host_in = {k: torch.from_numpy(v).pin_memory() for k, v in wl.state.items()}
    host_out = {k: torch.empty_like(v).pin_memory() for k, v in host_in.items()}
    e2e_steps = max(1, min(args.steps, 5))
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        S.shweno_set_state(sol.h, host_in["W"], host_in["V"], host_in["Y"], host_in["Z"], 0.0)
        S.shweno_advance(sol.h, 1, CFL)
        S.shweno_get_state(sol.h, host_out["W"], host_out["V"], host_out["Y"], host_out["Z"])
    e2e_sec = reduce_max(time.perf_counter() - t0, world)
    state_bytes = sum(v.numel() * 8 for v in host_in.values())
    assert np.isfinite(host_out["W"].numpy()).all()
    sol.close()
    # the FP64 rate this GPU reaches on independent fused multiply-add chains (outside the timing)
    fp64_tf, fp64_per_clk = S.shweno_fp64_probe(S.FP64_FMA, 8, 1 << 16)

    if rank != 0:
        return
    pk = peaks()
    total_k = sum(kernel_ms.values())
    dom = max(kernel_ms, key=kernel_ms.get)
    dom_ms = kernel_ms[dom] / max(timed_steps, 1)
    # x-face kernel: (n+1) faces x n rows x 3 Gauss points + (n+1)^2 corner points per launch
    xpoints = 3 * (n + 1) * n + (n + 1) * (n + 1)
    sm_hz = (clocks.get("sm_mhz") or 2070.0) * 1e6
    inst_per_clk = FP64_INST_PER_XFACE_POINT * xpoints / (dom_ms / 1000.0) / (152 * sm_hz)
    roof = None
    if dom == "xface2d" and FLOPS_PER_XFACE_POINT:
        flops = FLOPS_PER_XFACE_POINT * xpoints
        ach = flops / (dom_ms / 1000.0) / 1e12
        mflops, mparts = method_flops_per_xface_launch(n)
        mach = mflops / (dom_ms / 1000.0) / 1e12
        roof = {"bound": "alu", "kernel": dom, "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / FP64_PEAK_TFLOPS, "traffic": DRAM_BYTES_PER_XFACE_POINT * xpoints,
                # the same launch counted by the method's own operations (minimal forms), not the
                # kernel's executed instructions: work the kernel repeats would lower this fraction
                "method": {"flops_per_launch": mflops, "flops_per_point": mflops / xpoints,
                           "per_point_parts": mparts, "achieved": mach, "frac": mach / FP64_PEAK_TFLOPS},
                "flops_per_launch": flops, "launch_ms": dom_ms,
                "fp64_pipe_slot_frac": FP64_INST_PER_XFACE_POINT * xpoints / (dom_ms / 1000.0) / FP64_SLOTS_PER_S,
                "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz (FP64 pipe)",
                # the FP64 pipe as measured: fused multiply-add chains on every SM, outside the timing
                "fp64_probe": {"tflops": fp64_tf, "dfma_per_clk_per_sm": fp64_per_clk, "warps_per_sm": 8,
                               "frac_of_probe": ach / fp64_tf,
                               "fp64_inst_per_clk_per_sm": inst_per_clk,
                               "issue_frac_of_probe": inst_per_clk / fp64_per_clk}}
    hbm_gbs = cells * BYTES_PER_CELL_UPDATE / (sec / (world * args.steps)) / 1e9 / world
    line = {
        "metric": "2D Euler cell-updates/s", "value": value, "unit": "cell-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": workload_config(n, world),
        "roofline": roof,
        "kernels_ms_per_step": {k: v / max(timed_steps, 1) for k, v in kernel_ms.items()},
        "dominant_kernel_share": kernel_ms[dom] / total_k if total_k else None,
        "hbm": {"achieved_gbs": hbm_gbs, "peak_gbs": pk.get("hbm_gbs", 6750.0),
                "frac": hbm_gbs / pk.get("hbm_gbs", 6750.0), "bytes_per_cell_update": BYTES_PER_CELL_UPDATE},
        "clocks": clocks,
        "e2e": {"value": job_value(world, cells, e2e_steps, e2e_sec), "unit": "cell-updates/s",
                "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": state_bytes},
        "gpu_launches": 3 + 6 * args.steps,
    }
    if not args.no_learned:
        with ClockSampler(local) as clk_l:
            line["learned_flag"] = learned_vs_plain(S, torch, WL, args.steps, args.warmup, wl)
        line["learned_flag"]["clocks"] = clk_l.summary()
    if not args.no_batched:
        line["batched_1d"] = batched_1d(S, torch, WL, args.c4_steps)
        line["batched_2d"] = batched_2d(S, torch, WL, args.c5_steps, args.c5_problems)
    if not args.no_cpu_baseline:
        rate, el = oracle_sample(wl, args.cpu_window, 1)
        line["cpu_baseline"] = {"value": rate, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
                                "sample": f"one step of a {args.cpu_window}x{args.cpu_window}-cell window of the {n}^2 mesh ({el:.1f} s)"}
    print(json.dumps(line), flush=True)


def bench_learned_run(args):
    """Opt-in suite (--suite learned-run): the double Mach reflection (Example 5.10) at --dmr-nx x
    --dmr-nx/4 cells run with the always-nonlinear weights, with the learned flag, and with the
    always-nonlinear weights from initial averages perturbed by a relative 1e-12 (seeded signs),
    each to the times --learned-t (default 0.2) in turn.  At every time: the relative L1 deviation
    of the learned and of the perturbed solution from the plain one over all cell averages, the
    learned form's flagged fraction, and each form's rate over the segment since the previous time
    (CUDA events; device-side time loop).  The perturbed run measures how far two runs that differ
    at rounding level drift apart: the floor below which no approximation of the weights can be
    told apart."""
    import numpy as np
    import torch

    from paper_2304_09724_gb300 import flagnet as F
    from paper_2304_09724_gb300 import shweno as S
    from paper_2304_09724_gb300 import workloads as WL

    torch.cuda.set_device(0)
    nx = args.dmr_nx
    times = [float(x) for x in args.learned_t.split(",")]
    wl = WL.dmr(nx, nx // 4)
    net = F.load()
    out = {"suite": "learned-run", "workload": f"double Mach reflection {nx}x{nx // 4}, CFL {CFL}",
           "times": times, "dtype": "f64", "data": "synthetic"}
    shape = (4, wl.ny, wl.nx)
    snaps = {}
    for mode in ("plain", "learned", "perturbed"):
        stream = torch.cuda.Stream()
        sol = S.Solver(2, S.EULER, wl.nx, wl.ny, wl.domain, wl.bc, inflow=wl.inflow,
                       flag_mode=2 if mode == "learned" else 0, stream=stream.cuda_stream)
        init = {k: np.array(v) for k, v in wl.state.items()}
        if mode == "perturbed":
            rng = np.random.default_rng(1)
            for k in init:
                init[k] = init[k] * (1.0 + 1e-12 * rng.choice([-1.0, 1.0], size=init[k].shape))
        sol.set_state({k: torch.from_numpy(v).cuda() for k, v in init.items()})
        if mode == "learned":
            S.shweno_set_flag_net(sol.h, torch.from_numpy(net[0]).cuda(), net[1])
        torch.cuda.synchronize()
        rows, status, n_total = [], "ok", 0
        snaps[mode] = []
        for T in times:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            try:
                t, n = sol.run(T, CFL)
            except S.ShwenoError as e:
                status = "nonphysical" if e.status == S.E_NONPHYSICAL else str(e)
                t, n = sol.time()
            e1.record(stream)
            torch.cuda.synchronize()
            sec = e0.elapsed_time(e1) / 1000.0
            # run() returns the steps this call took: the segment since the previous time
            n_total += n
            row = {"T": T, "t": t, "steps": n, "steps_total": n_total, "seconds": sec,
                   "cell_updates_per_s": wl.nx * wl.ny * n / sec if sec > 0 else None}
            if mode == "learned":
                fl = np.empty((wl.ny, wl.nx), dtype=np.uint8)
                S.shweno_get_flags(sol.h, fl)
                row["flagged_fraction"] = float(fl.mean())
            Wd = torch.empty(shape, dtype=torch.float64, device="cuda")
            dummy = [torch.empty(shape, dtype=torch.float64, device="cuda") for _ in range(3)]
            S.shweno_get_state(sol.h, Wd, *dummy)
            snaps[mode].append(Wd)
            del dummy
            rows.append(row)
            if status != "ok":
                break
        sol.close()
        out[mode] = {"status": status, "rows": rows}
    for mode in ("learned", "perturbed"):
        for k, row in enumerate(out[mode]["rows"]):
            a, b = snaps["plain"][k], snaps[mode][k]
            row["rel_l1_vs_plain_W"] = float((b - a).abs().sum() / a.abs().sum())
    for k, row in enumerate(out["learned"]["rows"]):
        row["speedup_segment"] = row["cell_updates_per_s"] / out["plain"]["rows"][k]["cell_updates_per_s"]
    print(json.dumps(out), flush=True)


def bench_euler1d(args):
    """Opt-in suite (--suite euler1d): one large 1D Euler problem (--n1d cells, seeded smooth
    periodic data, fixed dt = 0.2 / n), `warmup` then `steps` steps through shweno_step: cell-updates/s
    from CUDA events and the per-kernel split."""
    import torch

    from paper_2304_09724_gb300 import shweno as S
    from paper_2304_09724_gb300 import workloads as WL

    torch.cuda.set_device(0)
    n = args.n1d
    W, V = WL.random_smooth_1d(3, n)
    sol = S.Solver(1, S.EULER, n, domain=(0.0, 1.0, 0.0, 1.0), bc=(0, 0))
    sol.set_state({"W": W, "V": V})
    dt = 0.2 / n
    for _ in range(args.warmup):
        sol.step(dt)
    torch.cuda.synchronize()
    S.shweno_set_timing(sol.h, True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        sol.step(dt)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    kms, k = S.shweno_get_timing(sol.h)
    sol.close()
    print(json.dumps({"suite": "euler1d", "cells": n, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": ms / args.steps, "cell_updates_per_s": n * args.steps / (ms / 1000.0),
                      "kernels_ms_per_step": {a: b / max(k, 1) for a, b in kms.items()},
                      "dtype": "f64", "data": "synthetic"}), flush=True)


def bench_refinement(args):
    """Opt-in suite (--suite refinement): the design order on the GPU (Example 5.8, Table 5.4).  The
    isentropic vortex at each --refine-sizes N x N runs to --refine-t with the plain scheme; the
    density L1 (mean |e|) and L-infinity errors against the exact cell averages of the translated
    vortex over the whole box and over its core (cells within 2.5 of the vortex centre, which the
    acoustic waves shed by the seams of the periodic data reach only after about t = 1.5), and the
    observed order of each refinement."""
    import numpy as np
    import torch

    from paper_2304_09724_gb300 import shweno as S
    from paper_2304_09724_gb300 import workloads as WL

    torch.cuda.set_device(0)
    T = args.refine_t
    rows = []
    for n in (int(x) for x in args.refine_sizes.split(",")):
        wl = WL.vortex(n)
        sol = S.Solver(2, S.EULER, n, n, wl.domain, wl.bc)
        sol.set_state(wl.state)
        t0 = time.perf_counter()
        t, steps = sol.run(T, CFL)
        el = time.perf_counter() - t0
        e = sol.get_state()["W"][0] - wl.exact(T)[0]
        sol.close()
        core = WL.vortex_core_mask(n, T)
        rows.append({"n": n, "t": t, "steps": steps, "seconds": el, "l1": float(np.mean(np.abs(e))),
                     "linf": float(np.max(np.abs(e))), "core_l1": float(np.mean(np.abs(e[core]))),
                     "core_linf": float(np.max(np.abs(e[core])))})
    for a, b in zip(rows, rows[1:]):
        r = b["n"] / a["n"]
        for k in ("l1", "linf", "core_l1", "core_linf"):
            b["order_" + k] = math.log(a[k] / b[k]) / math.log(r)
    print(json.dumps({"suite": "refinement", "workload": f"2D Euler isentropic vortex to T = {T}, CFL {CFL}, plain",
                      "rows": rows, "dtype": "f64", "data": "synthetic"}), flush=True)


def bench_fp64_probe(args):
    """Opt-in suite (--suite fp64-probe): the FP64 pipe's rate for fused multiply-add, multiply and
    add chains, and for the three interleaved, at 4..32 warps per SM (one CTA per SM), in
    operations per SM clock and TFLOP/s."""
    import torch

    from paper_2304_09724_gb300 import shweno as S

    torch.cuda.set_device(0)
    rows = []
    for op, name in ((S.FP64_FMA, "dfma"), (S.FP64_MUL, "dmul"), (S.FP64_ADD, "dadd"),
                     (S.FP64_MIX, "dfma,dfma,dmul,dadd")):
        for w in (4, 8, 16, 32):
            tf, per_clk = S.shweno_fp64_probe(op, w, 1 << 14)
            rows.append({"op": name, "warps_per_sm": w, "ops_per_clk_per_sm": per_clk, "tflops": tf})
    print(json.dumps({"suite": "fp64-probe", "chains_per_thread": 4, "rows": rows}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--cpu-window", type=int, default=160)
    ap.add_argument("--ref-window", type=int, default=48)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="main line without the batched workloads")
    ap.add_argument("--c4-steps", type=int, default=10, help="steps per problem of the 1D batch on the main line")
    ap.add_argument("--c5-steps", type=int, default=2, help="steps per problem of the 2D batch on the main line")
    ap.add_argument("--suite", default="main", choices=["main", "batched", "batched-full", "learned-run", "euler1d",
                                                      "fp64-probe", "refinement"])
    ap.add_argument("--n1d", type=int, default=4194304, help="euler1d: cells of the 1D problem")
    ap.add_argument("--dmr-nx", type=int, default=1024, help="learned-run: DMR mesh is N x N/4")
    ap.add_argument("--learned-t", default="0.2", help="learned-run: comma-separated end times")
    ap.add_argument("--c5-problems", type=int, default=64)
    ap.add_argument("--refine-sizes", default="128,256,512,1024", help="refinement: mesh sides")
    ap.add_argument("--refine-t", type=float, default=1.0, help="refinement: final time")
    args = ap.parse_args()
    if args.impl == "reference":
        bench_reference(args)
    elif args.suite == "euler1d":
        bench_euler1d(args)
    elif args.suite == "fp64-probe":
        bench_fp64_probe(args)
    elif args.suite == "refinement":
        bench_refinement(args)
    elif args.suite == "learned-run":
        bench_learned_run(args)
    elif args.suite == "batched":
        bench_batched(args)
    elif args.suite == "batched-full":
        bench_batched_full(args)
    else:
        bench_gpu(args)


if __name__ == "__main__":
    main()
