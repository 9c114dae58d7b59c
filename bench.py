#!/usr/bin/env python3
"""QV-Tree Search benchmark: plans/s and belief-state updates/s on GB300.

Default workload: the 512x512 plain configuration (rooms of 32 cells with
1-cell walls and 3-wide doors plus random walls to 25 %, 64 beacons with
range 8 and accuracy 0.8, slip 0.1, discount 0.97, Gaussian b0 with sigma 4,
depth 3, K = 4, FP32 beliefs and Q).  A step is R planning requests
(different start cells on the same map), each a complete plan from b0 to the
chosen action, run either as one plan per launch on concurrent streams or as
one batched launch of all R plans (the faster of the two in a short trial,
unless --execution says which).  The offline value iteration is run once
per map and reported separately.  The 128x128 configuration, the batched
forms and the other parts of the method are timed as sub-measurements.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Multi-GPU runs (torchrun) give every rank
its own disjoint episodes (weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "QV-Tree plans/sec and belief-state updates/sec (1 GB300) and % HBM peak"
L2_FLUSH_BYTES = 256 << 20
# algorithmic bytes of one offline sweep per cell (FP32, no cost map): the
# value iteration reads and writes V and reads the cell word; the FIB
# iteration reads and writes five alpha planes and reads the cell word
VI_BYTES_PER_CELL = 4 + 4 + 2
FIB_BYTES_PER_CELL = 5 * 4 + 5 * 4 + 2
# nominal dense TF32 / BF16 tensor rates (1.1 and 2.25 PFLOP/s): the PBVI
# contraction runs as TF32 MMAs, so its peak is the measured BF16 one
# scaled by this ratio
TF32_PER_BF16 = 1.1 / 2.25
SMI_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["mid", "large", "tiny"], default="large")
    ap.add_argument("--plans-per-step", type=int, default=32)
    ap.add_argument("--execution", choices=["auto", "plain", "batched"], default="auto",
                    help="how a step's requests run: one plan per launch on streams (plain), all in one launch "
                         "(batched), or the faster of the two in a short trial (auto)")
    ap.add_argument("--leaf-mode", choices=["fused", "materialise"], default="fused")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--profile-steps", type=int, default=10)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--reference-seconds", type=float, default=120.0,
                    help="bound on the reference arm's timed plans (it stops early and reports the plans it timed)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-tune", action="store_true", help="keep the default launch shape (no autotuner)")
    ap.add_argument("--streams", type=int, default=0,
                    help="streams the step's single-plan launches run on concurrently (each plan then takes "
                         "1/streams of the co-resident CTAs); 0 = the fastest of 1, 2, 4 and 8 in a short trial")
    ap.add_argument("--gradient-only", action="store_true",
                    help="only time the gradient of the root value on the differentiation workload")
    ap.add_argument("--offline-only", action="store_true",
                    help="only time the offline solves (value iteration, FIB) on the workload's map")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the batched (256 uneven maps) and 512x512 sub-measurements")
    ap.add_argument("--extra-steps", type=int, default=20)
    ap.add_argument("--sm-max-mhz", type=float, default=NOMINAL_SM_MHZ,
                    help="SM clock of the FP32 peak (replaced by the sampled maximum when clocks are sampled)")
    return ap.parse_args()


def time_device(run, steps, flush, stream):
    """Sum of per-step CUDA-event times of run(), L2 flushed before each step
    outside the events."""
    import torch
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for k in range(steps):
        flush.fill_(k & 255)
        ev0[k].record(stream)
        run()
        ev1[k].record(stream)
    torch.cuda.synchronize()
    return sum(ev0[k].elapsed_time(ev1[k]) for k in range(steps))


def time_offline(solve):
    """(result, first-call ms, median ms of three later calls) of a solver
    that synchronises (the value iteration, the FIB iteration)."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = solve()
    torch.cuda.synchronize()
    first = 1e3 * (time.perf_counter() - t0)
    runs = []
    for _ in range(3):
        t0 = time.perf_counter()
        r = solve()
        torch.cuda.synchronize()
        runs.append(1e3 * (time.perf_counter() - t0))
    return r, first, statistics.median(runs)


_L2_GBPS = None


def l2_bandwidth():
    """Copy bandwidth of a buffer that stays in L2 (2 x 24 MiB, read + write
    bytes, best of 20 back-to-back copies timed with CUDA events), measured
    once per process: the roof of the offline solves, whose state fits L2."""
    global _L2_GBPS
    if _L2_GBPS is None:
        import torch
        a = torch.ones(24 << 20, dtype=torch.uint8, device="cuda")
        b = torch.empty_like(a)
        for _ in range(5):
            b.copy_(a)
        best = None
        for _ in range(20):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            b.copy_(a)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        _L2_GBPS = 2 * a.numel() / (best * 1e-3) / 1e9
    return _L2_GBPS


def offline_line(r, first_ms, ms, model, bytes_per_cell, peak):
    """Sweeps, time and per-sweep bandwidth of an offline solve; the
    algorithmic bytes of one sweep are `bytes_per_cell` for every cell of the
    padded grid (values in and out, the cell word).  The state of a solve
    fits L2, so the fraction of the L2 copy bandwidth measured in this
    process is reported beside the HBM one."""
    cells = model.H * model.P
    sweep_s = ms / 1e3 / max(r["sweeps"], 1)
    gbps = cells * bytes_per_cell / sweep_s / 1e9
    l2 = l2_bandwidth()
    return {"sweeps": r["sweeps"], "ms": ms, "first_call_ms": first_ms, "cells": model.H * model.W,
            "us_per_sweep": 1e6 * sweep_s, "cell_sweeps_per_s": model.H * model.W * r["sweeps"] / (ms / 1e3),
            "bytes_per_cell_sweep": bytes_per_cell, "GBps": gbps, "frac_of_measured_hbm": gbps / peak,
            "l2_copy_GBps_measured": l2, "frac_of_measured_l2": gbps / l2}


def pbvi_measurement(args, dev, K, flush, stream, with_cpu=True):
    """The PBVI lower bound (Eq. 8) on the mid map: belief sets of 256 and
    1024 points grown by the expansion rounds from b0, then one Eq. 8 backup
    of every point timed with CUDA events (L2 flushed before each), with the
    contraction's flops against the TF32 tensor peak."""
    import torch
    import oracle as O
    from paper_1810_00204_gb300 import api, workloads as WL
    w = WL.mid(args.seed)
    m = api.Model(w, device=dev)
    out = {}
    for rounds in (8, 10):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g = api.pbvi_solve(m, rounds=rounds, iters=4, seed=args.seed)
        torch.cuda.synchronize()
        solve_ms = 1e3 * (time.perf_counter() - t0)
        pb, G = g["pbvi"], g["G"]
        nB, nG = g["B"].shape[0], G.shape[0]
        Gout = torch.empty_like(G)
        for _ in range(3):
            pb.backup(G, out=Gout)
        ms = time_device(lambda: pb.backup(G, out=Gout), K, flush, stream) / K
        Kp, _ = pb.layout()
        flops = 2.0 * 5 * nB * nG * Kp
        tfl = flops / (ms * 1e-3) / 1e12
        bf16, src = measured_peak("bf16_tflops")
        tf32 = bf16 * TF32_PER_BF16
        line = {"points": nB, "vectors": nG, "backup_ms": ms, "point_backups_per_s": nB / (ms * 1e-3),
                "solve_ms": solve_ms, "solve_schedule": f"{rounds} expansion rounds, 4 backups after each",
                "contraction": {"flops_per_backup": flops, "label_ordered_cells": Kp,
                                "achieved_tflops_whole_backup": tfl, "bound": "tensor", "unit": "TFLOP/s",
                                "peak": tf32, "peak_source": f"{src} bf16_tflops x {TF32_PER_BF16:.3f} (TF32)",
                                "frac": tfl / tf32,
                                # each product is three TF32 MMAs (hi.hi + hi.lo + lo.hi)
                                "issued_tf32_tflops": 3.0 * tfl, "issued_frac": 3.0 * tfl / tf32},
                "v_pbvi_b0": float(g["value"][0])}
        if with_cpu and rounds == 8:
            # the oracle's Eq. 8 backup of a few points against the same vectors
            Bh = m.from_grid(g["B"]).reshape(nB, -1).astype("float64")
            Gh = m.from_grid(G).reshape(nG, -1).astype("float64")
            npts = max(1, min(O.num_threads(), 8))
            t0 = time.perf_counter()
            O.pbvi_backup(w, Bh[:npts], Gh)
            el = time.perf_counter() - t0
            line["cpu_baseline"] = {"value": npts / el, "unit": "point backups/s", "cores": O.num_threads(),
                                    "kind": "oracle",
                                    "sample": f"{npts} of the {nB} points backed up against all {nG} vectors, "
                                              f"{el:.1f} s, FP64 C oracle with OpenMP over points"}
        out[f"points_{nB}"] = line
        del g, pb, G, Gout
        torch.cuda.empty_cache()
    return out


def aems_measurement(args, dev, K, stream):
    """The paper's node fields on the mid map (Alg. 5-7, Eq. 9): U from FIB
    leaf alpha-vectors, L from PBVI at the materialised leaf beliefs (256
    points), then L, H and E up to the root.  Times each stage with CUDA
    events (inputs resident, after warm-up)."""
    import torch
    from paper_1810_00204_gb300 import _native as N
    from paper_1810_00204_gb300 import api, workloads as WL
    w = WL.mid(args.seed)
    m = api.Model(w, device=dev)
    Q = api.fib_value_iterate(m, dtype="f32", want_alpha=False)["Q"]
    g = api.pbvi_solve(m, rounds=8, iters=4, seed=args.seed)
    plan = api.Plan([m], [Q], [m.b0()], depth=w.depth, K=w.K, seed=w.seed, episode=w.episode,
                    leaf_mode=N.QV_LEAF_MATERIALISE)
    plan.run()
    leaves = plan.level(0, w.depth)
    nleaf = leaves["count"]
    lb = leaves["belief"]
    L = torch.empty(nleaf, dtype=torch.float32, device=dev)

    def timed(fn):
        for _ in range(3):
            fn()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        ev[0].record(stream)
        for _ in range(K):
            fn()
        ev[1].record(stream)
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]) / K

    ms_plan = timed(plan.run)
    ms_leafL = timed(lambda: L.copy_(g["pbvi"].value(g["G"], lb)[0]))
    b = plan.bounds(L)
    ms_bounds = timed(lambda: plan.bounds(L))
    b = plan.bounds(L)
    res = plan.read()[0]
    Kp, _ = g["pbvi"].layout()
    nG = g["G"].shape[0]
    return {"leaves": nleaf, "pbvi_vectors": nG, "plan_ms": ms_plan, "leaf_pbvi_value_ms": ms_leafL,
            "leaf_pbvi_tflops": 2.0 * nleaf * nG * Kp / (ms_leafL * 1e-3) / 1e12,
            "bounds_ms_incl_host": ms_bounds,
            "root": {"U": res["value"], "L": float(b[0]["LV"][0]), "H": float(b[0]["HV"][0]),
                     "E_leaf": int(b[0]["EV"][0])},
            "note": "plan in the materialised mode with FIB leaves; bounds_ms includes the host-side level "
                    "views and the per-level launches"}


def bestfirst_measurement(args, dev, stream, iters=400):
    """Alg. 1's best-first planning loop on the mid map: U from FIB, L from a
    256-point PBVI, K = 8; `iters` expansions timed with CUDA events (the
    tree resident on the device, one reset before the timed run), with the
    oracle's loop on a bounded sample as the CPU baseline."""
    import torch
    import oracle as O
    from paper_1810_00204_gb300 import api, workloads as WL
    w = WL.mid(args.seed)
    m = api.Model(w, device=dev)
    Q = api.fib_value_iterate(m, dtype="f32", want_alpha=False)["Q"]
    g = api.pbvi_solve(m, rounds=8, iters=4, seed=args.seed)
    nz = w.B + 1
    bf = api.BestFirst(m, Q, g["pbvi"], g["G"], K=w.K, seed=w.seed, episode=w.episode, max_depth=6,
                       max_nodes=1 + iters * 5 * min(w.K, nz))
    # a first search finds how many iterations run before planning stops;
    # the timed search runs exactly that many (no no-op iterations timed)
    bf.reset()
    bf.run(iters)
    n_run = max(1, bf.read()["iterations"])
    bf.reset()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    bf.run(n_run)
    ev[1].record(stream)
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1])
    r = bf.read()
    out = {"iterations": r["iterations"], "requested": iters, "stopped": r["stopped"], "nodes": r["nodes"],
           "ms": ms, "expansions_per_s": r["iterations"] / (ms * 1e-3), "us_per_expansion": 1e3 * ms / max(1, r["iterations"]),
           "root": {"U": r["U"], "L": r["L"], "H": r["H"], "action": r["root_action"]},
           "launches_per_expansion": 10,
           "note": "the first expansion of a run is issued eagerly, the rest replay a CUDA graph of one expansion",
           "pbvi_vectors": int(g["G"].shape[0])}
    if not args.no_cpu:
        Qh = m.from_grid(Q).reshape(5, -1).astype("float64")
        Gh = m.from_grid(g["G"]).reshape(g["G"].shape[0], -1).astype("float64")
        n = 20
        t0 = time.perf_counter()
        ro = O.bestfirst(w, Qh, Gh, n, K=w.K, max_depth=6)
        el = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": ro["iterations"] / el, "unit": "expansions/s", "cores": 1, "kind": "oracle",
                               "sample": f"the oracle's first {n} expansions of the same loop, {el:.1f} s, one thread"}
    return out


def episodes_measurement(args, dev, stream, E=64, max_steps=200):
    """Closed-loop episodes (Alg. 1's outer loop) on the mid map with its
    planning configuration (d = 3, K = 8, QMDP leaves): E robots from
    different start cells; each step one batched plan, the true system's
    step and the belief update.  Timed with CUDA events (host check of the
    end every 8 steps included)."""
    import torch
    import oracle as O
    from paper_1810_00204_gb300 import api, workloads as WL
    w = WL.mid(args.seed)
    m = api.Model(w, device=dev)
    Q = api.mdp_value_iterate(m, dtype="f32")["Q"]
    eps = WL.episodes(w, E, seed=args.seed + 11)
    b0s = [m.to_grid(e.b0) for e in eps]
    starts = [e.start for e in eps]
    api.run_episodes(m, Q, b0s[:4], starts[:4], depth=w.depth, K=w.K, seed=w.seed, max_steps=3)  # warm-up
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ev[0].record(stream)
    g = api.run_episodes(m, Q, b0s, starts, depth=w.depth, K=w.K, seed=w.seed, max_steps=max_steps)
    ev[1].record(stream)
    torch.cuda.synchronize()
    wall_ms = 1e3 * (time.perf_counter() - t0)
    ms = ev[0].elapsed_time(ev[1])
    # where the loop's time goes: the device time of one batched plan of the
    # robots' start beliefs and of their beliefs after the loop (the plan is
    # most of a step's GPU work; its support windows follow the beliefs)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    plan_ms = {}
    for tag, bel in (("start_beliefs", b0s), ("end_beliefs", list(g["beliefs"].unbind(0)))):
        p_ = api.Plan([m] * E, [Q] * E, [b.contiguous() for b in bel], depth=w.depth, K=w.K, seed=w.seed)
        for _ in range(2):
            p_.run()
        plan_ms[tag] = time_device(p_.run, 10, flush, stream) / 10
        del p_
    del flush
    robot_steps = int(g["steps"].sum())
    ok = g["success"].astype(bool)
    out = {"episodes": E, "max_steps": max_steps, "steps_run": g["steps_run"], "ms": ms,
           "robot_steps": robot_steps, "robot_steps_per_s": robot_steps / (ms * 1e-3),
           "plans_per_s": E * g["steps_run"] / (ms * 1e-3),
           "success_rate": float(ok.mean()), "mean_steps_success": float(g["steps"][ok].mean()) if ok.any() else None,
           "mean_return": float(g["ret"].mean()), "wall_ms": wall_ms,
           "plan_device_ms": plan_ms,
           "note": "plans for finished episodes still run inside the batch (counted in plans_per_s); "
                   "plan_device_ms: one batched plan of the 64 beliefs alone, L2 flushed"}
    if not args.no_cpu:
        Qh = m.from_grid(Q).reshape(5, -1).astype("float64")
        t0 = time.perf_counter()
        ro = O.closed_loop(w, Qh, [eps[0].b0], [eps[0].start], max_steps=10)
        el = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": int(ro["steps"][0]) / el, "unit": "robot steps/s", "cores": O.num_threads(),
                               "kind": "oracle",
                               "sample": f"the oracle's first {int(ro['steps'][0])} steps of one episode, {el:.1f} s"}
    return out


def extra_measurements(args, dev, flush, stream, plans_per_s, arm, model, Qd, eps, w, plain_arm=None,
                       batched_arm=None, exec_trial=None):
    """Sub-measurements beside the headline: the step's requests as one
    batched launch against one launch per plan (same requests); the
    256-episode batch of uneven maps as one launch against one launch per
    episode (same episodes); the 128x128 configuration; the 512x512 plan
    with materialised leaves; the other parts of the method."""
    import torch
    from paper_1810_00204_gb300 import _native as N
    from paper_1810_00204_gb300 import api, workloads as WL
    out = {}
    K = max(3, args.extra_steps)
    peak, peak_kind = measured_peak()
    alu_peak = alu_peak_tflops(torch.cuda.get_device_properties(dev).multi_processor_count, args.sm_max_mhz)
    leaf_mode = N.QV_LEAF_FUSED if args.leaf_mode == "fused" else N.QV_LEAF_MATERIALISE
    b0s = [model.to_grid(e.b0) for e in eps]
    # (1) the same R requests in one launch (E = R episodes on one map)
    # against one launch per request, both timed over K steps
    if plain_arm is not None and batched_arm is not None:
        ms_p = plain_arm.time(K)
        ms_b = batched_arm.time(K)
        same = [r["nodes_per_level"] for r in batched_arm.plan.read()]
        plain_nodes = [p.read()[0]["nodes_per_level"] for p in plain_arm.plans]
        R = len(eps)
        out["same_requests_one_launch"] = {
            "plans_per_s": R * K / (ms_b / 1e3), "E": R, "plain_plans_per_s": R * K / (ms_p / 1e3),
            "vs_plain": ms_p / ms_b, "tuning": batched_arm.plan.tuning, "plain_streams": plain_arm.S,
            "same_trees_as_plain": same == plain_nodes,
            "workspace_GB": batched_arm.plan.workspace_bytes / 1e9,
            "note": "the headline's requests (same map, b0s, seeds and episode words): one batched launch against "
                    "one launch per plan on streams"}
    # (1a) the same batched launch with the deepest level in its per-child
    # stencil form instead of the contraction form (same requests and trees)
    if batched_arm is not None and leaf_mode == N.QV_LEAF_FUSED and w.depth >= 2:
        R = len(eps)
        pf = api.Plan([model] * R, [Qd] * R, b0s, depth=w.depth, K=w.K, seed=w.seed, episode=eps[0].episode,
                      leaf_mode=leaf_mode, band_cells=batched_arm.plan.tuning["band_cells"],
                      items_per_cta=batched_arm.plan.tuning["items_per_cta"], deepest_form=N.QV_DEEPEST_STENCIL)
        pf.capture_graph()
        for _ in range(3):
            pf.run()
        ms_f = time_device(pf.run, K, flush, stream)
        ms_c = batched_arm.time(K)
        out["deepest_level_forms"] = {
            "contraction_plans_per_s": R * K / (ms_c / 1e3), "stencil_plans_per_s": R * K / (ms_f / 1e3),
            "contraction_vs_stencil": ms_f / ms_c,
            "same_trees": [r["nodes_per_level"] for r in pf.read()] == [r["nodes_per_level"]
                                                                         for r in batched_arm.plan.read()],
            "note": "the headline's batched launch with the deepest level's sums as the contraction of every "
                    "child's belief with the planes (default) or as each child's five-action stencil"}
        del pf
        torch.cuda.empty_cache()
    # (1b) the headline's workload with more requests per batched launch: the
    # deepest level's work grows with the batch, the upper levels' latency
    # chain is shared by more plans
    scaling = {}
    for R2 in (64, 128):
        eps2 = WL.episodes(w, R2, seed=args.seed)
        b02 = [model.to_grid(e.b0) for e in eps2]
        api.autotune([model] * R2, [Qd] * R2, b02, depth=w.depth, K=w.K, seed=w.seed, episode=eps2[0].episode,
                     leaf_mode=leaf_mode, reps=3)
        p2 = api.Plan([model] * R2, [Qd] * R2, b02, depth=w.depth, K=w.K, seed=w.seed, episode=eps2[0].episode,
                      leaf_mode=leaf_mode)
        p2.capture_graph()
        for _ in range(3):
            p2.run()
        ms2 = time_device(p2.run, K, flush, stream)
        scaling[str(R2)] = {"plans_per_s": R2 * K / (ms2 / 1e3), "ms_per_launch": ms2 / K, "tuning": p2.tuning,
                            "workspace_GB": p2.workspace_bytes / 1e9}
        del p2, b02
        torch.cuda.empty_cache()
    out["batch_size_scaling"] = dict(scaling, note="plans per batched launch on the headline's map (episodes of "
                                                   "the same generator, L2 flushed before every launch); the "
                                                   "headline keeps the step's requests per launch")
    # (2) 256 independent episodes on maps of uneven size: one launch per
    # step against one launch per episode, the same episodes
    ws = WL.batched(args.seed, E=256)
    ms_ = [api.Model(x, device=dev) for x in ws]
    Qs = [api.mdp_value_iterate(m, dtype="f32")["Q"] for m in ms_]
    b3 = [m.b0() for m in ms_]
    api.autotune(ms_, Qs, b3, depth=3, K=8, seed=args.seed, episode=0, reps=3)
    p3 = api.Plan(ms_, Qs, b3, depth=3, K=8, seed=args.seed, episode=0)
    p3.capture_graph()
    for _ in range(2):
        p3.run()
    res = p3.read()
    ms3 = time_device(p3.run, K, flush, stream)
    nodes = [sum(r["nodes_per_level"][1:]) for r in res]
    tuning3 = p3.tuning
    ws_gb = p3.workspace_bytes / 1e9
    del p3
    torch.cuda.empty_cache()
    arm3 = PlainArm(api, ms_, Qs, b3, list(range(256)), 3, 8, args.seed, N.QV_LEAF_FUSED, {}, True, flush, stream,
                    [1, 4, 8, 16])
    ms3p = arm3.time(K)
    same3 = [p.read()[0]["nodes_per_level"] for p in arm3.plans] == [r["nodes_per_level"] for r in res]
    out["batched_256_uneven"] = {"plans_per_s": 256 * K / (ms3 / 1e3), "ms_per_launch": ms3 / K,
                                 "tuning": tuning3, "updates_per_s": sum(nodes) * K / (ms3 / 1e3),
                                 "plain_plans_per_s": 256 * K / (ms3p / 1e3), "vs_plain": ms3p / ms3,
                                 "plain_streams": arm3.S, "plain_trial_plans_per_s": arm3.trial,
                                 "same_trees_as_plain": same3,
                                 "cells_mean": float(sum(x.H * x.W for x in ws) / 256), "workspace_GB": ws_gb,
                                 "note": "plain = one k_plan launch per episode from a CUDA graph, on streams"}
    del arm3, Qs, ms_
    torch.cuda.empty_cache()
    # (3) the 128x128 configuration, one plan per launch
    wm, descm = make_workload("mid", args.seed)
    mm = api.Model(wm, device=dev)
    r, f, t = time_offline(lambda: api.mdp_value_iterate(mm, dtype="f32"))
    Qm = r["Q"]
    mid = {"workload": descm, "vi": offline_line(r, f, t, mm, VI_BYTES_PER_CELL, peak)}
    r, f, t = time_offline(lambda: api.fib_value_iterate(mm, dtype="f32", want_alpha=False))
    mid["fib"] = offline_line(r, f, t, mm, FIB_BYTES_PER_CELL, peak)
    epm = WL.episodes(wm, args.plans_per_step, seed=args.seed)
    bm = [mm.to_grid(e.b0) for e in epm]
    api.autotune([mm], [Qm], [bm[0]], depth=wm.depth, K=wm.K, seed=wm.seed, episode=epm[0].episode, reps=3)
    armm = PlainArm(api, [mm] * len(epm), [Qm] * len(epm), bm, [e.episode for e in epm], wm.depth, wm.K, wm.seed,
                    N.QV_LEAF_FUSED, {}, True, flush, stream, [1, 4, 8, 16])
    msm = armm.time(K)
    pps = len(epm) * K / (msm / 1e3)
    ndm = [p.read()[0]["nodes_per_level"] for p in armm.plans]
    nda = [sum(n[l] for n in ndm) / len(ndm) for l in range(wm.depth + 1)]
    rl, _ = plan_roofline(api, mm, Qm, bm[0], epm[0], "fused", N.QV_LEAF_FUSED, {},
                          armm.plans[0] if armm.S > 1 else None, flush, 5, peak, peak_kind, alu_peak,
                          support_cells(epm[0].b0, wm.occ, wm.depth), job_plans_per_s=pps, nodes_avg=nda)
    mid.update({"plans_per_s": pps, "streams": armm.S, "trial_plans_per_s": armm.trial,
                "updates_per_s": sum(sum(n[1:]) for n in ndm) * K / (msm / 1e3), "roofline": rl})
    out["mid_128"] = mid
    del armm
    torch.cuda.empty_cache()
    # (4) the headline map with materialised leaves, one plan per launch
    if args.workload == "large":
        Ncell = model.H * model.P
        api.autotune([model], [Qd], [b0s[0]], depth=w.depth, K=w.K, seed=w.seed, episode=eps[0].episode,
                     leaf_mode=N.QV_LEAF_MATERIALISE, reps=3)
        torch.cuda.empty_cache()
        p4 = api.Plan([model], [Qd], [b0s[0]], depth=w.depth, K=w.K, seed=w.seed, episode=eps[0].episode,
                      leaf_mode=N.QV_LEAF_MATERIALISE)
        p4.capture_graph()
        for _ in range(2):
            p4.run()
        r4 = p4.read()[0]
        ms4 = time_device(p4.run, K, flush, stream)
        nodes = r4["nodes_per_level"]
        phases = {}
        prof_runs = [p4.profile() for _ in range(3)]
        for it in prof_runs[0][1:]:
            nm, lv = it["name"].split(":", 1)[1], it["level"]
            t = statistics.mean(pr[i]["ms"] for pr in prof_runs for i in range(len(pr))
                                if pr[i]["name"] == it["name"] and pr[i]["level"] == lv)
            if nm in ("update", "leaf"):  # the dense leaf passes: every leaf written and read in full
                b = phase_bytes(nm, lv, nodes, Ncell, w.depth, "materialise")
                gbps = b / (t * 1e-3) / 1e9 if t > 0 else None
                phases[f"{nm}[{lv}]"] = {"ms": t, "bytes": b, "GBps": gbps,
                                         "frac_of_measured_hbm": (gbps / peak) if gbps else None}
            else:
                phases[f"{nm}[{lv}]"] = {"ms": t}
        sb = survey_bytes(nodes, Ncell, w.depth, "materialise")
        out["large_512_materialise"] = {"plans_per_s": K / (ms4 / 1e3), "ms_per_plan": ms4 / K,
                                        "nodes_per_level": nodes,
                                        "updates_per_s": sum(nodes[1:]) * K / (ms4 / 1e3), "phases": phases,
                                        "algorithmic_bytes_per_plan": sb,
                                        "frac_of_measured_hbm": sb / (ms4 * 1e-3) / 1e9 / peak,
                                        "tuning": p4.tuning, "workspace_GB": p4.workspace_bytes / 1e9}
        del p4
        torch.cuda.empty_cache()
    # (5) the gradient of the root value on the 128x128 differentiation workload
    out["gradient_diff_128"] = gradient_measurement(args, dev, K, peak)
    # (6) the single-belief primitives of the C ABI on inputs larger than L2
    out["primitives"] = primitive_measurement(args, dev, K, peak)
    # (7) the PBVI lower bound (Eq. 8) on the mid map
    out["pbvi_mid"] = pbvi_measurement(args, dev, K, flush, stream, with_cpu=not args.no_cpu)
    # (8) the paper's node fields U, L, H, E on the mid map
    out["aems_fields_mid"] = aems_measurement(args, dev, K, stream)
    # (9) the best-first planning loop of Alg. 1 on the mid map
    out["bestfirst_mid"] = bestfirst_measurement(args, dev, stream)
    # (10) closed-loop episodes (Alg. 1's outer loop) on the mid map
    out["episodes_mid"] = episodes_measurement(args, dev, stream)
    # (11) the paper's experimental model (Sec. V) on the mid map
    out["model9_mid"] = model9_measurement(args, dev, stream, with_cpu=not args.no_cpu)
    return out


def model9_measurement(args, dev, stream, plans=20, with_cpu=True):
    """The paper's experimental model (Sec. V: nine actions, four occupancy
    sensors) on the mid map at its planning configuration (d = 3, K = 8):
    FP32 value iteration to 1e-4, then `plans` plans from b0 (episode words
    0, 1, ...) timed with CUDA events around the calls (each call
    synchronises once per level).  Algorithmic bytes per plan: every
    expanded node reads its belief once for all nine actions (4 B per cell),
    a node of the deepest expanded level also Q (36 B per cell), every
    materialised child reads its parent and writes itself (8 B per cell)."""
    import torch
    import oracle as O
    from paper_1810_00204_gb300 import api, workloads as WL
    w = WL.mid(args.seed)
    m = api.Model9(w, device=dev, stream=stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    vi = m.value_iterate("f32", tol=1e-4, stream=stream)
    ev[1].record(stream)
    torch.cuda.synchronize()
    vi_ms = ev[0].elapsed_time(ev[1])
    Q = vi["Q"]
    for k in range(3):
        g = m.plan(Q, episode=1000 + k, stream=stream)
    torch.cuda.synchronize()
    ev[0].record(stream)
    for k in range(plans):
        g = m.plan(Q, episode=k, stream=stream)
    ev[1].record(stream)
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1]) / plans
    nl = g["nodes_per_level"]
    n = w.H * w.W
    byts = sum(nl[l] * n * (4 + (36 if l == len(nl) - 2 else 0)) for l in range(len(nl) - 1))
    byts += sum(nl[l] * n * 8 for l in range(1, len(nl) - 1))
    peak, src = measured_peak()
    out = {"workload": "mid 128x128 map, nine actions (45-degree slips, eps 0.1), four sensors p 0.95, "
                       "gamma 0.97, d = 3, K = 8",
           "vi": {"sweeps": vi["sweeps"], "ms": vi_ms, "tol": 1e-4},
           "plan": {"ms_per_plan": ms, "plans_per_s": 1e3 / ms, "nodes_per_level": nl, "plans": plans,
                    "note": "each call synchronises once per level to size the next"},
           "roofline": {"bound": "hbm", "algorithmic_bytes_per_plan": byts, "achieved": byts / (ms * 1e-3) / 1e9,
                        "peak": peak, "unit": "GB/s", "frac": byts / (ms * 1e-3) / 1e9 / peak,
                        "peak_source": src}}
    if with_cpu:
        Qh = Q.cpu().numpy().reshape(9, -1).astype("float64")
        t0 = time.perf_counter()
        O.tree_plan9(w, Qh, depth=2, K=w.K)
        el = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": 1.0 / el, "unit": "depth-2 plans/s", "cores": 1, "kind": "oracle",
                               "sample": f"one depth-2 plan of the same map and K ({el:.1f} s, one thread); the "
                                         "depth-3 plan adds about 27,000 leaves (80 s on the build host)"}
    return out


def primitive_measurement(args, dev, K, peak):
    """belief_predict and belief_correct on one 16384x2048 belief (128 MiB,
    larger than L2), leaf_value on 256 beliefs of 512x512 (256 MiB): device
    time per call with CUDA events, algorithmic bytes / time against the
    measured HBM bandwidth."""
    import torch
    from paper_1810_00204_gb300 import api, workloads as WL
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(reps):
            fn()
        ev1.record()
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / reps

    res = {}
    w = WL.tiny(args.seed, H=16384, W=2048)
    m = api.Model(w, device=dev)
    N = m.H * m.P
    b = torch.rand((m.H, m.P), device=dev) * (m.occ == 0)
    b /= b.sum()
    out = torch.empty_like(b)
    ms = timed(lambda: api.belief_predict(m, b, 1, out), K)
    nbytes = N * (4 + 4 + 2)  # belief in, predicted belief out, cell words
    res["belief_predict"] = {"cells": N, "ms": ms, "GBps": nbytes / (ms * 1e-3) / 1e9,
                             "frac_of_measured_hbm": nbytes / (ms * 1e-3) / 1e9 / peak}
    ms = timed(lambda: api.belief_correct(m, out, 2, b), K)
    nbytes = N * (4 + 2) * 2 + N * 4  # P(z) pass and scale pass read bbar and the cell words; b' written
    res["belief_correct"] = {"cells": N, "ms": ms, "GBps": nbytes / (ms * 1e-3) / 1e9,
                             "frac_of_measured_hbm": nbytes / (ms * 1e-3) / 1e9 / peak}
    del b, out
    torch.cuda.empty_cache()
    # the no-allocation variant beside the workspace version, on the largest
    # grid its fixed scratch takes (2048 x 2048 cells; 16 MiB beliefs, so
    # both stay L2-resident between the back-to-back calls)
    ws_ = WL.tiny(args.seed, H=2048, W=2048)
    ms_ = api.Model(ws_, device=dev)
    Ns = ms_.H * ms_.P
    bs = torch.rand((ms_.H, ms_.P), device=dev) * (ms_.occ == 0)
    bs /= bs.sum()
    outs = torch.empty_like(bs)
    pz = torch.empty(1, dtype=torch.float32, device=dev)
    t_ws = timed(lambda: api.belief_correct(ms_, bs, 2, outs), K)
    t_na = timed(lambda: api.belief_correct_noalloc(ms_, bs, 2, outs, pz), K)
    res["belief_correct_noalloc"] = {"cells": Ns, "ms": t_na, "workspace_version_ms": t_ws,
                                     "note": "same 2048x2048 grid for both; L2-resident"}
    del bs, outs
    torch.cuda.empty_cache()
    wl = WL.large(args.seed)
    ml = api.Model(wl, device=dev)
    Ql = api.mdp_value_iterate(ml, dtype="f32")["Q"]
    n = 256
    bl = torch.rand((n, ml.H, ml.P), device=dev) * (ml.occ == 0)
    bl /= bl.sum(dim=(1, 2), keepdim=True)
    Nl = ml.H * ml.P
    ms = timed(lambda: api.leaf_value(ml, Ql, bl), K)
    nbytes = n * Nl * 4 + 20 * Nl
    res["leaf_value"] = {"beliefs": n, "cells": Nl, "ms": ms, "GBps": nbytes / (ms * 1e-3) / 1e9,
                         "frac_of_measured_hbm": nbytes / (ms * 1e-3) / 1e9 / peak}
    # Alg. 4's ancestral sampler: 256 (belief, action) pairs of 512x512, 64
    # samples each; per pair it reads the belief and the cell words and
    # writes the prefix sums (the samples' own reads are L2 hits)
    Ks = 64
    ms = timed(lambda: api.forward_sample(ml, bl, [k % 5 for k in range(n)], list(range(n)), Ks, level=1), K)
    nbytes = n * Nl * (4 + 2 + 4)
    res["forward_sample_ancestral"] = {"pairs": n, "samples_per_pair": Ks, "cells": Nl, "ms": ms,
                                       "samples_per_s": n * Ks / (ms * 1e-3), "GBps": nbytes / (ms * 1e-3) / 1e9,
                                       "frac_of_measured_hbm": nbytes / (ms * 1e-3) / 1e9 / peak}
    return res


def gradient_measurement(args, dev, K, peak):
    """Forward (checkpointed FP64 value iteration + one plan) and backward
    (tree adjoint + value-iteration adjoint) of the root value on the
    128x128, depth-3, K=8, 200-sweep workload, each part timed with CUDA
    events; one full gradient = the four parts in sequence."""
    import torch
    from paper_1810_00204_gb300 import api, workloads as WL
    w = WL.diff(args.seed)
    m = api.Model(w, device=dev)
    S, every = 200, 16
    times = {"vi_forward": [], "plan_forward": [], "tree_backward": [], "vi_backward": []}
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    for it in range(K + 2):
        torch.cuda.synchronize()
        ev[0].record()
        vi = api.mdp_value_iterate_checkpointed(m, S, every)
        ev[1].record()
        plan = api.Plan([m], [vi["Q"]], [m.b0()], depth=3, K=8, seed=w.seed, episode=w.episode)
        plan.run()
        ev[2].record()
        tb = api.qv_tree_backward(plan, 0, dL=1.0)
        ev[3].record()
        api.mdp_value_backward(m, vi, tb["Qbar"], tb["dslip"], tb["dcost"])
        ev[4].record()
        torch.cuda.synchronize()
        if it >= 2:
            for i, k in enumerate(times):
                times[k].append(ev[i].elapsed_time(ev[i + 1]))
    res = plan.read()[0]
    ms = {k: statistics.median(v) for k, v in times.items()}
    total = sum(ms.values())
    N = m.H * m.P
    # value-iteration adjoint, bytes per sweep if every array went to DRAM once:
    # recompute (V_k read, V_k+1 write, argmax write, cell words) and reverse
    # step (lambda read/write, V_k, argmax, dcost read-modify-write, cell words)
    vib = S * N * ((8 + 8 + 1 + 2) + (8 + 8 + 8 + 1 + 16 + 2))
    return {"gradients_per_s": 1e3 / total, "ms_per_gradient": total, "ms": ms,
            "nodes_per_level": res["nodes_per_level"], "sweeps": S, "checkpoint_every": every,
            "dslip": float(tb["dslip"][0]), "dacc": float(tb["dacc"][0]),
            "vi_backward_us_per_sweep": 1e3 * ms["vi_backward"] / S,
            "vi_backward_GBps_if_dram": vib / (ms["vi_backward"] * 1e-3) / 1e9,
            "vi_backward_frac_of_measured_hbm": vib / (ms["vi_backward"] * 1e-3) / 1e9 / peak,
            "note": "128x128 state fits L2 (the value-iteration adjoint's working set is about 2.5 MB): "
                    "bound by the neighbour hand-off of its 2 steps per sweep, not by HBM"}


def make_workload(name, seed):
    from paper_1810_00204_gb300 import workloads as WL
    if name == "mid":
        w = WL.mid(seed)
        desc = ("mid 128x128, 20% rect obstacles, B=16 range 5 acc 0.85, slip 0.1, gamma 0.97, "
                "gaussian b0 sigma 4, depth 3, K=8")
    elif name == "large":
        w = WL.large(seed)
        desc = ("large 512x512 rooms+walls 25%, B=64 range 8 acc 0.8, slip 0.1, gamma 0.97, "
                "gaussian b0 sigma 4, depth 3, K=4")
    else:
        w = WL.tiny(seed)
        desc = "tiny 20x20, 15% iid obstacles, B=4 range 3 acc 0.9, depth 2, K=4"
    return w, desc


def headline_config(args, w, desc, use_graph, world_size):
    """The `config` object of the JSON line, the same for both arms."""
    return {"workload": desc, "plans_per_step": args.plans_per_step, "depth": w.depth, "K": w.K,
            "leaf_mode": args.leaf_mode, "cuda_graph": use_graph,
            "l2": "flushed before every step (256 MiB device write outside the timed events)",
            "parallelism": "replicas" if world_size > 1 else "single GPU"}


# ---------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(prefix="qv_clocks_", suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={SMI_FIELDS}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.gpu_index)], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for ln in f:
                p = [x.strip() for x in ln.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def gpu_index(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if local_rank < len(ids):
            return ids[local_rank]
    return str(local_rank)


# ---------------------------------------------------------------- roofline helpers
def measured_peak(key="hbm_gbs"):
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            j = json.load(f)
        return float(j[key]), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}[key], "fallback"


def tree_sources_sha():
    h = hashlib.sha256()
    for p in ("paper_1810_00204_gb300/csrc/qv_tree.cu", "paper_1810_00204_gb300/csrc/qv_tree_device.cuh",
              "paper_1810_00204_gb300/csrc/qv_common.cuh"):
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel, level, workload):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel sources (else None)."""
    sha = tree_sources_sha()
    pat = re.compile(r"^traffic\s+kernel=(\S+)\s+level=(\d+)\s+workload=(\S+)\s+bytes_per_launch=(\d+)"
                     r"\s+source_sha=(\S+)")
    d = os.path.join(ROOT, "profiles")
    if not os.path.isdir(d):
        return None
    for fn in sorted(os.listdir(d)):
        if not fn.endswith((".txt", ".md")):
            continue
        with open(os.path.join(d, fn)) as f:
            for ln in f:
                m = pat.match(ln.strip())
                if m and m.group(1) == kernel and int(m.group(2)) == level and m.group(3) == workload \
                        and m.group(5) == sha:
                    return int(m.group(4))
    return None


def phase_bytes(name, level, nodes, N, depth, leaf_mode):
    """Bytes a phase must move at minimum: every belief it reads or writes
    once (4 B per cell), the cell words (2 B) once, Q (20 B) once when read.
    expand(l) reads the level l-1 beliefs (b0 at the root) and writes level l
    when a later phase reads it back."""
    b = 4 * N
    if name in ("expand", "expand_fused"):
        rd = b if level == 0 else nodes[level - 1] * b
        stored = level > 0 and (level < depth - 1 or leaf_mode == "materialise")
        wr = nodes[level] * b if stored else 0
        return rd + wr + 2 * N + (20 * N if name == "expand_fused" else 0)
    if name == "update":
        return nodes[level] * b + nodes[level + 1] * b + 2 * N
    if name == "leaf":
        return nodes[level] * b + 20 * N
    return 0


def plan_phases(depth, leaf_mode):
    ph = [("expand_fused" if (l == depth - 1 and leaf_mode == "fused") else "expand", l) for l in range(depth)]
    if depth > 0 and leaf_mode == "materialise":
        ph.append(("update", depth - 1))
    if depth == 0 or leaf_mode == "materialise":
        ph.append(("leaf", depth))
    return ph


# ---------------------------------------------------------------- oracle arm
def oracle_plans(episodes, Q64, seconds, max_plans=None):
    import oracle as O
    t0 = time.perf_counter()
    n = 0
    while True:
        w = episodes[n % len(episodes)]
        O.tree_plan(w, Q64)
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds or (max_plans and n >= max_plans):
            return n, el


def run_reference(args, rank):
    """The reference arm: the FP64 oracle on the host cores, one plan of the
    same workload per step (a bounded sample of the R-plan step), with the
    same config object as our arm.  It stops early, after
    --reference-seconds of timed plans, and then reports the plans it timed."""
    if rank != 0:
        return
    import numpy as np
    import oracle as O
    from paper_1810_00204_gb300 import workloads as WL
    O.build()
    w, desc = make_workload(args.workload, args.seed)
    eps = WL.episodes(w, max(args.plans_per_step, 1), seed=args.seed)
    Q64 = O.value_iteration(w)["Q"].astype(np.float32).astype(np.float64)
    for i in range(args.warmup):
        O.tree_plan(eps[i % len(eps)], Q64)
    t, n = 0.0, 0
    for k in range(args.steps):
        t0 = time.perf_counter()
        O.tree_plan(eps[(args.warmup + k) % len(eps)], Q64)
        t += time.perf_counter() - t0
        n += 1
        if t >= args.reference_seconds:
            break
    value = n / t
    cores = O.num_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "plans/s", "n_gpus": args.gpus,
        "steps": n, "warmup": args.warmup, "ms_per_step": 1e3 * t / n,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": headline_config(args, w, desc, not args.no_graph, 1),
        "cpu_baseline": {"value": value, "unit": "plans/s", "cores": cores, "kind": "oracle",
                         "sample": f"{n} plans of the workload (of the {args.steps} steps asked for), one per step, "
                                   f"the step's start cells cycled, FP64 C oracle (OpenMP over tree nodes, "
                                   f"{cores} threads)"},
        "e2e": {"value": value, "unit": "plans/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm
def survey_bytes(nodes, N, depth, leaf_mode):
    """Algorithmic bytes of one plan in the paper's unfused form, with FP32
    beliefs of 4 N bytes: every V-node whose children are materialised reads
    its belief twice (once for P(z | b, a) and R(b, a), once for the Bayes
    correction of its children) and each child is written once, 8 N + 4 N C
    bytes for C children; a V-node of the deepest internal level reads its
    belief once, 4 N bytes, and gets every leaf value from the factorised
    leaf sums; materialised leaves are also written and read back once."""
    b = 4 * N
    if depth == 0:
        return b
    tot = 0
    for lv in range(depth):
        if lv < depth - 1 or leaf_mode == "materialise":
            tot += 2 * nodes[lv] * b + nodes[lv + 1] * b
        else:
            tot += nodes[lv] * b
    if leaf_mode == "materialise":
        tot += nodes[depth] * b
    return tot


def support_cells(b0, occ, depth):
    """Cells of the support window of every level d = 0 .. depth + 1: the
    bounding box of b0's nonzero cells dilated by d cells and clipped to the
    grid -- the window k_plan restricts level d's sums to (the motion stencil
    moves mass by one cell per level)."""
    import numpy as np
    occ = np.asarray(occ)
    b = np.asarray(b0).reshape(occ.shape)
    r, c = np.nonzero(b != 0)
    if r.size == 0:
        return [0] * (depth + 2)
    H, W = occ.shape
    out = []
    for d in range(depth + 2):
        rows = min(H, int(r.max()) + d + 1) - max(0, int(r.min()) - d)
        cols = min(W, int(c.max()) + d + 1) - max(0, int(c.min()) - d)
        out.append(rows * cols)
    return out


def window_bytes(nodes, cells, depth, leaf_mode):
    """survey_bytes with each belief's N the cells of its level's support
    window (cells[l] for a level-l belief): the same reads and writes, over
    the cells where the belief can be nonzero."""
    if depth == 0:
        return 4 * cells[0]
    tot = 0
    for lv in range(depth):
        if lv < depth - 1 or leaf_mode == "materialise":
            tot += 2 * nodes[lv] * 4 * cells[lv] + nodes[lv + 1] * 4 * cells[lv + 1]
        else:
            tot += nodes[lv] * 4 * cells[lv]
    if leaf_mode == "materialise":
        tot += nodes[depth] * 4 * cells[depth]
    return tot


# FP32 operations (an FMA counts two) of the expand pass per cell of a
# level-l node's task window (the window of level l + 1): forming the node's
# belief from its parent (one action's stencil and the observation weight,
# l > 0), the five actions' predicted masses (two shared slip sums and four
# multiply-adds per move action), the reward and null-label sums (the reward
# of the cell, five multiply-adds, five masks and five adds) and, at the
# fused level, the 25 Q-weighted null sums.
FLOPS_CHILD, FLOPS_STENCIL, FLOPS_SUMS, FLOPS_QSUMS = 7, 20, 21, 50
# The deepest fused level of a plan of depth >= 2 runs in the contraction
# form: per (child, cell of its level's own window) the child's belief (one
# multiply) and 35 multiply-adds against the planes; per (parent, cell) the
# five actions' predicted masses (FLOPS_STENCIL); per cell the planes once
# (five actions, up to four moves each: the reward multiply-add, the null
# mask, its add and five Q multiply-adds).
FLOPS_CTR_CHILD, FLOPS_CTR_PLANES = 71, 280
FP32_LANES_PER_SM = 128
NOMINAL_SM_MHZ = 2070.0


def expand_flops(nodes, cells, depth, leaf_mode):
    """FP32 operations of one plan's expand phases: level l's nodes over the
    window of level l + 1 (cells[l + 1]); the deepest fused level (depth >=
    2) in its contraction form over its own window (cells[l]).  The finalize
    phase's label histograms (the beacons' sensing diamonds inside the
    window) are not counted."""
    tot = 0
    for lv in range(depth):
        if lv == depth - 1 and leaf_mode == "fused" and depth >= 2:
            tot += cells[lv] * (nodes[lv] * FLOPS_CTR_CHILD + nodes[lv - 1] * FLOPS_STENCIL + FLOPS_CTR_PLANES)
            continue
        f = FLOPS_STENCIL + FLOPS_SUMS + (FLOPS_CHILD if lv > 0 else 0)
        if lv == depth - 1 and leaf_mode == "fused":
            f += FLOPS_QSUMS
        tot += nodes[lv] * cells[lv + 1] * f
    return tot


def alu_peak_tflops(sms, sm_mhz=NOMINAL_SM_MHZ):
    """FP32 peak from the unit counts: SMs x 128 FP32 lanes x 2 (FMA) x clock."""
    return sms * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


class PlainArm:
    """R single-plan launches per step (the plain one-tree-per-launch form):
    each request is its own plan and its own k_plan launch from a CUDA
    graph; with S streams every launch takes 1/S of the co-resident CTAs so
    that up to S plans overlap.  A short trial picks S among `choices`."""

    def __init__(self, api, models, Qs, b0s, episodes, depth, K, seed, leaf_mode, knobs, use_graph, flush, stream,
                 choices):
        self.api, self.models, self.Qs, self.b0s = api, models, Qs, b0s
        self.episodes, self.depth, self.K, self.seed = episodes, depth, K, seed
        self.leaf_mode, self.knobs, self.use_graph = leaf_mode, knobs, use_graph
        self.flush, self.stream = flush, stream
        self.full_grid = api.Plan([models[0]], [Qs[0]], [b0s[0]], depth=depth, K=K, seed=seed, episode=episodes[0],
                                  leaf_mode=leaf_mode, **knobs).grid
        self.trial = {}
        best_S, best_rate = choices[0], -1.0
        for S in choices:
            self._make(S)
            for _ in range(3):
                self.step()
            if len(choices) > 1:
                import torch
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                ms_t = 0.0
                for k in range(6):
                    flush.fill_(k & 255)
                    e0.record(stream)
                    self.step()
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ms_t += e0.elapsed_time(e1)
                rate = len(models) * 6 / (ms_t * 1e-3)
                self.trial[S] = rate
            else:
                rate = 0.0
            if rate > best_rate:
                best_S, best_rate = S, rate
            self.plans = self.streams = None
        self.S = best_S
        self._make(best_S)

    def _make(self, S):
        import torch
        g = 0 if S == 1 else max(1, self.full_grid // S)
        self.plans = [self.api.Plan([m], [q], [b], depth=self.depth, K=self.K, seed=self.seed, episode=e,
                                    leaf_mode=self.leaf_mode, grid_ctas=g, **self.knobs)
                      for m, q, b, e in zip(self.models, self.Qs, self.b0s, self.episodes)]
        if self.use_graph:
            for p in self.plans:
                p.capture_graph()
        self.streams = [torch.cuda.Stream() for _ in range(S)] if S > 1 else [self.stream]

    @property
    def grid_ctas(self):
        return self.plans[0].grid

    def step(self):
        ps, ss = self.plans, self.streams
        if len(ss) == 1:
            for p in ps:
                p.run()
            return
        for s_ in ss:
            s_.wait_stream(self.stream)
        for i, p in enumerate(ps):
            p.run(ss[i % len(ss)])
        for s_ in ss:
            self.stream.wait_stream(s_)

    def time(self, steps):
        """Device ms of `steps` steps (L2 flushed before each, outside the events)."""
        return time_device(self.step, steps, self.flush, self.stream)


class BatchedArm:
    """The R requests of a step as one batched launch (pattern 2): one plan
    of E = R episodes (consecutive episode words, so the same trees as one
    plan per request) with its autotuned launch shape, from a CUDA graph."""

    def __init__(self, api, models, Qs, b0s, episodes, depth, K, seed, leaf_mode, use_graph, flush, stream,
                 tune=True):
        self.flush, self.stream = flush, stream
        if tune:
            api.autotune(models, Qs, b0s, depth=depth, K=K, seed=seed, episode=episodes[0], leaf_mode=leaf_mode,
                         reps=3)
        self.plan = api.Plan(models, Qs, b0s, depth=depth, K=K, seed=seed, episode=episodes[0], leaf_mode=leaf_mode)
        if use_graph:
            self.plan.capture_graph()
        self.plans, self.streams, self.S, self.trial = [self.plan], [stream], 1, {}
        self.full_grid = self.grid_ctas = self.plan.grid

    def step(self):
        self.plan.run()

    def time(self, steps):
        return time_device(self.step, steps, self.flush, self.stream)


def e2e_pipelined(api, arm, b0_all, models, Qs, episodes, w, leaf_mode, use_graph, flush, stream, n):
    """End to end through the public API with host buffers, as a serving loop
    runs it: every step copies its R start beliefs in from pinned host memory
    (one transfer of the [R][H][P] batch, on a copy stream), flushes L2, runs
    the batched plan and copies its results back into pinned memory; the host
    decodes them.  Two plans on two device batches alternate, so step k's
    copy in overlaps step k - 1's plan and the host decodes step k - 1 while
    step k runs.  Every copy, flush, launch and decode is inside the timed
    region; value = R n / wall time."""
    import torch
    pinned = b0_all.cpu().pin_memory()
    b0_b = torch.empty_like(b0_all)
    other = api.Plan(models, Qs, list(b0_b.unbind(0)), depth=w.depth, K=w.K, seed=w.seed, episode=episodes[0],
                     leaf_mode=leaf_mode)
    if use_graph:
        other.capture_graph()
    plans, bufs = [arm.plan, other], [b0_all, b0_b]
    rbufs = [p.readback_buffer() for p in plans]
    cs = torch.cuda.Stream()
    copied = [torch.cuda.Event() for _ in range(2)]
    done = [torch.cuda.Event() for _ in range(2)]
    R = b0_all.shape[0]

    def loop(steps):
        got, pending = [], None
        for k in range(steps):
            j = k & 1
            if k >= 2:
                cs.wait_event(done[j])  # plan j's previous run has read its batch
            with torch.cuda.stream(cs):
                bufs[j].copy_(pinned, non_blocking=True)
                copied[j].record(cs)
            stream.wait_event(copied[j])
            with torch.cuda.stream(stream):
                flush.fill_(k & 255)
            plans[j].run(stream)
            plans[j].read_async(rbufs[j], stream)
            done[j].record(stream)
            if pending is not None:
                done[pending].synchronize()
                got = plans[pending].decode(rbufs[pending])
            pending = j
        done[pending].synchronize()
        return plans[pending].decode(rbufs[pending])

    loop(4)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    got = loop(n)
    t = time.perf_counter() - t0
    assert len(got) == R and all(g["nodes_per_level"][0] == 1 for g in got)
    return {"value": R * n / t, "unit": "plans/s", "h2d_bytes_per_step": int(b0_all.numel() * 4),
            "d2h_bytes_per_step": int(rbufs[0].numel()), "steps": n,
            "note": "pinned [R][H][P] batch in (one copy), L2 flush, batched plan, results out and decoded, "
                    "every step; two plans alternate so a step's copy in overlaps the previous step's plan"}


def plan_roofline(api, model, Q, b0, w, leaf_mode_name, leaf_mode, knobs, slice_plan, flush, reps, peak, peak_kind,
                  alu_peak, cells, job_plans_per_s=None, nodes_avg=None):
    """The dominant kernel (k_plan, the whole plan in one launch) against its
    roofline, one plan alone on the whole grid, L2 flushed before each
    launch: FP32 operations of the expand passes over the levels' support
    windows (expand_flops) against the FP32 peak -- the windowed passes do
    about 100 operations per 4 bytes of belief, so the kernel is bound by
    arithmetic issue, not HBM; beside it the window bytes (window_bytes)
    against measured HBM, and the paper's dense byte count over the same
    time (a dense-equivalent rate, not a bandwidth).  Also the same launch on
    the benchmark's slice of the grid and the per-phase device times."""
    full = api.Plan([model], [Q], [b0], depth=w.depth, K=w.K, seed=w.seed, episode=w.episode,
                    leaf_mode=leaf_mode, **knobs)
    for _ in range(3):
        full.run()
    nodes = full.read()[0]["nodes_per_level"]
    Ncell = model.H * model.P
    ms_full, ms_slice, ph_ms = [], [], {}
    for k in range(max(1, reps)):
        flush.fill_(k & 255)
        lst = full.profile()
        ms_full.append(lst[0]["ms"])
        for it in lst[1:]:
            ph_ms.setdefault((it["name"].split(":", 1)[1], it["level"]), []).append(it["ms"])
        if slice_plan is not None:
            flush.fill_(k & 255)
            ms_slice.append(slice_plan.profile()[0]["ms"])
    avg = statistics.mean(ms_full)
    sec = avg * 1e-3
    flops = expand_flops(nodes, cells, w.depth, leaf_mode_name)
    wbytes = window_bytes(nodes, cells, w.depth, leaf_mode_name)
    nd = nodes if nodes_avg is None else nodes_avg
    dbytes = survey_bytes(nodes, Ncell, w.depth, leaf_mode_name)
    achieved = flops / sec / 1e12
    out = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s", "frac": achieved / alu_peak,
           "traffic": None, "kernel": "k_plan (whole plan, one launch)", "kernel_share": 1.0,
           "flops_per_launch": flops,
           "flops_rule": "FP32 operations of the expand passes, level l's nodes over the window of level l+1: "
                         f"{FLOPS_STENCIL + FLOPS_SUMS} per cell, +{FLOPS_CHILD} below the root; the deepest fused "
                         f"level (contraction form) over its own window: {FLOPS_CTR_CHILD} per (child, cell), "
                         f"{FLOPS_STENCIL} per (parent, cell), {FLOPS_CTR_PLANES} per cell for the planes "
                         "(label histograms not counted)",
           "peak_source": "SMs x 128 FP32 lanes x 2 x the sampled maximum SM clock",
           "nodes_per_level": nodes, "window_cells_per_level": cells,
           "avg_launch_ms": avg, "launch": f"one plan alone on the whole grid ({full.grid} CTAs), L2 flushed",
           "hbm_window": {"bytes_per_launch": wbytes, "achieved": wbytes / sec / 1e9, "peak": peak,
                          "unit": "GB/s", "frac": wbytes / sec / 1e9 / peak,
                          "rule": "8N + 4N C per V-node with materialised children, 4N per leaf-parent V-node, "
                                  "N = the cells of the belief's support window",
                          "peak_source": "measured hbm_gbs, MEASURED_PEAKS.json" if peak_kind == "measured"
                          else "fallback 6800 GB/s"},
           "dense_equivalent": {"bytes_per_launch": dbytes, "GBps": dbytes / sec / 1e9,
                                "of_measured_hbm": dbytes / sec / 1e9 / peak,
                                "note": "the dense per-plan count (N = every cell of the grid) over the launch "
                                        "time; the kernel skips the cells outside the support windows, which "
                                        "are exactly zero, so this is a rate, not a bandwidth"}}
    per_phase = {}
    for (nm, lv), v in ph_ms.items():
        per_phase[f"{nm}[{lv}]"] = {"ms": statistics.mean(v)}
    out["phases"] = per_phase
    if ms_slice:
        s_avg = statistics.mean(ms_slice)
        out["slice"] = {"avg_launch_ms": s_avg, "grid_ctas": slice_plan.grid,
                        "achieved": flops / (s_avg * 1e-3) / 1e12, "frac": flops / (s_avg * 1e-3) / 1e12 / alu_peak}
    if job_plans_per_s is not None:
        out["job_dense_equivalent_GBps"] = survey_bytes(nd, Ncell, w.depth, leaf_mode_name) * job_plans_per_s / 1e9
    return out, full


def main():
    args = parse()
    from paper_1810_00204_gb300 import replicas
    rank, local_rank, world_size = replicas.world()
    if args.impl == "reference":
        run_reference(args, rank)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    import __graft_entry__ as G
    from paper_1810_00204_gb300 import _native as N
    from paper_1810_00204_gb300 import api, workloads as WL

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world_size > 1 and not dist.is_initialized():
        dist.init_process_group("nccl", device_id=dev)
    if rank == 0:
        G.build()
    replicas.barrier(dev)
    N.lib()
    stream = torch.cuda.current_stream()
    if args.gradient_only:
        # the differentiation workload alone (forward + adjoint), for profiling
        if rank == 0:
            peak, _ = measured_peak()
            print(json.dumps({"gradient_diff_128": gradient_measurement(args, dev, max(3, args.extra_steps), peak)}),
                  flush=True)
        return

    w, desc = make_workload(args.workload, args.seed)
    if args.offline_only:
        # the offline alpha-vector solves alone, for profiling
        if rank == 0:
            peak, _ = measured_peak()
            model = api.Model(w, device=dev)
            vi, f, t = time_offline(lambda: api.mdp_value_iterate(model, dtype="f32"))
            out = {"workload": desc, "vi": offline_line(vi, f, t, model, VI_BYTES_PER_CELL, peak)}
            fib, f, t = time_offline(lambda: api.fib_value_iterate(model, dtype="f32", want_alpha=False))
            out["fib"] = offline_line(fib, f, t, model, FIB_BYTES_PER_CELL, peak)
            if args.workload == "mid":
                flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
                out["pbvi"] = pbvi_measurement(args, dev, max(3, args.extra_steps), flush, stream,
                                               with_cpu=not args.no_cpu)
                out["aems_fields"] = aems_measurement(args, dev, max(3, args.extra_steps), stream)
                out["bestfirst"] = bestfirst_measurement(args, dev, stream)
                out["episodes"] = episodes_measurement(args, dev, stream)
                out["model9"] = model9_measurement(args, dev, stream, with_cpu=not args.no_cpu)
            print(json.dumps(out), flush=True)
        return
    R = args.plans_per_step
    ep_ids = replicas.episode_range(rank, world_size, R)
    eps = WL.episodes(w, R, seed=args.seed, first_episode=ep_ids.start)
    model = api.Model(w, device=dev)
    # offline value iteration (once per map), timed on its own
    # (the first call in a process also loads the library's kernels: timed
    # apart from the steady-state solve)
    vi, vi_first_ms, vi_ms = time_offline(lambda: api.mdp_value_iterate(model, dtype="f32"))
    fib, fib_first_ms, fib_ms = time_offline(lambda: api.fib_value_iterate(model, dtype="f32", want_alpha=False))
    Qd = vi["Q"]
    leaf_mode = N.QV_LEAF_FUSED if args.leaf_mode == "fused" else N.QV_LEAF_MATERIALISE
    # the step's start beliefs as one device batch [R][H][P] (views per request),
    # so that the end-to-end leg copies a step's inputs in with one transfer
    b0_all = torch.stack([model.to_grid(e.b0) for e in eps])
    b0s = list(b0_all.unbind(0))
    # launch-shape autotuner (offline, like the value iteration): the choice is
    # cached in the library and taken by the plans created below
    tune = None
    if not args.no_tune:
        best, table = api.autotune([model], [Qd], [b0s[0]], depth=w.depth, K=w.K, seed=w.seed,
                                   episode=eps[0].episode, leaf_mode=leaf_mode, reps=5)
        dflt = [t["ms"] for t in table if t["band_cells"] == 2048 and t["items_per_cta"] == 2]
        tune = {"band_cells": best["band_cells"], "items_per_cta": best["items_per_cta"],
                "tuned_ms": best["ms"], "default_ms": dflt[0] if dflt else None, "candidates": len(table)}
    use_graph = not args.no_graph
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    knobs = {}
    if tune is not None:
        knobs = dict(band_cells=tune["band_cells"], items_per_cta=tune["items_per_cta"])
    choices = [args.streams] if args.streams > 0 else [1, 2, 4, 8]
    plain = batched = None
    if args.execution in ("auto", "plain"):
        plain = PlainArm(api, [model] * R, [Qd] * R, b0s, [e.episode for e in eps], w.depth, w.K, w.seed,
                         leaf_mode, knobs, use_graph, flush, stream, choices)
    if args.execution in ("auto", "batched"):
        batched = BatchedArm(api, [model] * R, [Qd] * R, b0s, [e.episode for e in eps], w.depth, w.K, w.seed,
                             leaf_mode, use_graph, flush, stream, tune=not args.no_tune)
    exec_trial = {}
    if plain is not None and batched is not None:
        for name, a_ in (("plain", plain), ("batched", batched)):
            for _ in range(3):
                a_.step()
            exec_trial[name] = R * 6 / (a_.time(6) * 1e-3)
        arm = batched if exec_trial["batched"] > exec_trial["plain"] else plain
    else:
        arm = plain if plain is not None else batched
    execution = "batched" if arm is batched else "plain"

    # warm-up
    for k in range(max(args.warmup, 0)):
        flush.fill_(k & 255)
        arm.step()
    torch.cuda.synchronize()
    results = [g for p in arm.plans for g in p.read()]  # every episode of every plan
    nodes_per_plan = [r["nodes_per_level"] for r in results]
    updates_per_step = sum(sum(n[1:]) for n in nodes_per_plan)

    # timed region: K steps, each bracketed by events on the launching stream;
    # L2 flushed (256 MiB write) before every step, outside the events
    K = args.steps
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    sampler = ClockSampler(gpu_index(local_rank))
    sampler.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    replicas.barrier(dev)
    wall0 = time.perf_counter()
    for k in range(K):
        flush.fill_((k + 7) & 255)
        ev0[k].record(stream)
        arm.step()
        ev1[k].record(stream)
    torch.cuda.synchronize()
    replicas.barrier(dev)
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    dev_ms = sum(ev0[k].elapsed_time(ev1[k]) for k in range(K))
    dev_ms_max = replicas.reduce_max(dev_ms, dev)
    total_plans = R * K * world_size
    plans_per_s = total_plans / (dev_ms_max / 1e3)
    updates_per_s = replicas.reduce_sum(updates_per_step * K, dev) / (dev_ms_max / 1e3)

    # the dominant kernel against its roofline: one plan alone on the whole
    # grid and on the step's slice, with the mean level sizes of the step
    peak, peak_kind = measured_peak()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    if clocks and clocks.get("sm_max_mhz"):
        args.sm_max_mhz = float(clocks["sm_max_mhz"])
    alu_peak = alu_peak_tflops(sms, args.sm_max_mhz)
    nodes_avg = [sum(n[l] for n in nodes_per_plan) / len(nodes_per_plan) for l in range(w.depth + 1)]
    cells_per_plan = [support_cells(e.b0, w.occ, w.depth) for e in eps]
    roofline, _ = plan_roofline(api, model, Qd, b0s[0], eps[0], args.leaf_mode, leaf_mode, knobs,
                                arm.plans[0] if (arm is plain and arm.S > 1) else None, flush, args.profile_steps,
                                peak, peak_kind, alu_peak, cells_per_plan[0],
                                job_plans_per_s=plans_per_s / world_size, nodes_avg=nodes_avg)
    # the step's work, summed over its R plans (each with its own tree and windows)
    step_flops = sum(expand_flops(n, c, w.depth, args.leaf_mode) for n, c in zip(nodes_per_plan, cells_per_plan))
    step_wbytes = sum(window_bytes(n, c, w.depth, args.leaf_mode) for n, c in zip(nodes_per_plan, cells_per_plan))
    step_dbytes = sum(survey_bytes(n, model.H * model.P, w.depth, args.leaf_mode) for n in nodes_per_plan)
    if arm is batched:
        # the dominant kernel as the timed region runs it: the batched
        # launch of the step's R plans, L2 flushed before each launch
        ms_b, ph_b = [], {}
        for k in range(max(1, args.profile_steps)):
            flush.fill_(k & 255)
            lst = batched.plan.profile()
            ms_b.append(lst[0]["ms"])
            for it in lst[1:]:
                ph_b.setdefault(f'{it["name"].split(":", 1)[1]}[{it["level"]}]', []).append(it["ms"])
        solo = {k: roofline[k] for k in ("achieved", "frac", "avg_launch_ms", "launch", "flops_per_launch",
                                          "hbm_window", "dense_equivalent", "phases")}
        b_ms = statistics.mean(ms_b)
        sec = b_ms * 1e-3
        roofline.update({
            "achieved": step_flops / sec / 1e12, "frac": step_flops / sec / 1e12 / alu_peak,
            "avg_launch_ms": b_ms, "flops_per_launch": step_flops,
            "kernel": f"k_plan ({R} plans, one batched launch)",
            "launch": f"the step's batched launch ({batched.plan.grid} CTAs), L2 flushed",
            "hbm_window": dict(roofline["hbm_window"], bytes_per_launch=step_wbytes, achieved=step_wbytes / sec / 1e9,
                               frac=step_wbytes / sec / 1e9 / peak),
            "dense_equivalent": dict(roofline["dense_equivalent"], bytes_per_launch=step_dbytes,
                                     GBps=step_dbytes / sec / 1e9, of_measured_hbm=step_dbytes / sec / 1e9 / peak),
            "phases": {k: {"ms": statistics.mean(v)} for k, v in ph_b.items()},
            "solo": solo})
    # DRAM bytes of the timed launch from a committed ncu summary taken on the
    # current sources: the batched launch of R plans, or one plan alone
    roofline["traffic"] = recorded_traffic("k_plan", 0, f"{args.workload}_b{R}" if arm is batched
                                           else f"{args.workload}_p1")

    # end to end through the public API with host buffers: pinned b0 -> device,
    # run, results -> host, every step
    e2e = None
    if not args.no_e2e and arm is batched:
        e2e = e2e_pipelined(api, arm, b0_all, [model] * R, [Qd] * R, [e.episode for e in eps], w, leaf_mode,
                            use_graph, flush, stream, max(3, min(K, 200)))
        e2e["value"] = replicas.reduce_sum(e2e["value"], dev) if world_size > 1 else e2e["value"]
    elif not args.no_e2e:
        pinned = [torch.from_numpy(np.ascontiguousarray(
            np.pad(e.b0.astype(np.float32), ((0, 0), (0, model.P - model.W))))).pin_memory() for e in eps]
        h2d = sum(p.numel() * 4 for p in pinned)
        # every plan's result bytes copied back asynchronously into pinned
        # memory, one synchronisation per step, then decoded
        rbufs = [p.readback_buffer() for p in arm.plans]
        d2h = sum(b.numel() for b in rbufs)
        t_e2e = 0.0
        n_e2e = max(3, min(K, 200))
        for k in range(n_e2e):
            flush.fill_(k & 255)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for s_ in arm.streams:
                s_.wait_stream(stream)
            # every request's b0 in from pinned memory on its plan's stream
            for i in range(R):
                with torch.cuda.stream(arm.streams[(i if arm is plain else 0) % len(arm.streams)]):
                    b0s[i].copy_(pinned[i], non_blocking=True)
            for i, p in enumerate(arm.plans):
                s_ = arm.streams[i % len(arm.streams)]
                p.run(s_)
                p.read_async(rbufs[i], s_)
            for s_ in arm.streams:
                s_.synchronize()
            got = [g for i, p in enumerate(arm.plans) for g in p.decode(rbufs[i])]
            t_e2e += time.perf_counter() - t0
        assert len(got) == R and all(g["nodes_per_level"][0] == 1 for g in got)
        e2e_val = R * n_e2e / t_e2e
        e2e_val = replicas.reduce_sum(e2e_val, dev) if world_size > 1 else e2e_val
        e2e = {"value": e2e_val, "unit": "plans/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "steps": n_e2e}

    launch = {"execution": execution, "execution_trial_plans_per_s": exec_trial, "autotune": tune,
              "streams": arm.S, "grid_ctas": arm.grid_ctas, "full_grid": arm.full_grid,
              "concurrency_trial_plans_per_s": arm.trial,
              "batched_tuning": batched.plan.tuning if batched is not None else None}
    extra = None
    if not args.no_extra and rank == 0:
        extra = extra_measurements(args, dev, flush, stream, plans_per_s / world_size, arm, model, Qd, eps, w,
                                   plain_arm=plain, batched_arm=batched, exec_trial=exec_trial)

    # oracle CPU baseline (rank 0, N = 1 only), bounded sample
    cpu = None
    if rank == 0 and world_size == 1 and not args.no_cpu:
        import oracle as O
        O.build()
        oq = O.value_iteration(w)["Q"].astype(np.float32).astype(np.float64)
        n, el = oracle_plans(eps, oq, args.cpu_seconds)
        cores = O.num_threads()
        cpu = {"value": n / el, "unit": "plans/s", "cores": cores, "kind": "oracle",
               "sample": f"{n} plans of this workload (same map, start cells cycled), {el:.1f} s, FP64 C oracle "
                         f"with OpenMP over tree nodes"}
        if extra is not None and "gradient_diff_128" in extra:
            # the oracle's reverse mode on the same differentiation workload, one gradient
            from paper_1810_00204_gb300 import workloads as WLd
            wd = WLd.diff(args.seed)
            t0 = time.perf_counter()
            O.root_value_grad(wd, 200, depth=3, K=8)
            el = time.perf_counter() - t0
            extra["gradient_diff_128"]["cpu_baseline"] = {
                "value": 1.0 / el, "unit": "gradients/s", "cores": O.num_threads(), "kind": "oracle",
                "sample": "one FP64 reverse-mode gradient (200 VI sweeps, depth-3 K=8 tree, tree adjoint "
                          "single-threaded)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": plans_per_s, "unit": "plans/s", "n_gpus": world_size,
            "steps": K, "warmup": args.warmup, "ms_per_step": dev_ms_max / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": headline_config(args, w, desc, use_graph, world_size),
            "launch": launch,
            "nodes_per_level": nodes_per_plan[0],
            "updates_per_s": updates_per_s,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": (R if arm is plain else 1) * K,
            "clocks": clocks,
            "vi": dict(offline_line(vi, vi_first_ms, vi_ms, model, VI_BYTES_PER_CELL, peak),
                       note="offline, once per map; not part of plans/s; ms = median of 3 calls after the first"),
            "fib": dict(offline_line(fib, fib_first_ms, fib_ms, model, FIB_BYTES_PER_CELL, peak),
                        note="Fast Informed Bound alpha-vectors (Eq. 7), FP32; offline like vi"),
            "wall_s": wall,
            "extra": extra,
        }
        print(json.dumps(line), flush=True)
    if world_size > 1:
        replicas.barrier(dev)
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
