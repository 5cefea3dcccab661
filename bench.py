#!/usr/bin/env python3
"""Benchmark of the hot path: G(x) on the production bubble grid.

Workload (one step): the equal-mass scalar bubble, D = 4, mu2 = 1, on the
1024 x 1024 cell-centred grid over Re x in [-10, 5], Im x in [-5, 5], with
2048 radial x 256 angular Gauss-Legendre nodes, for the three masses
m in {0.5, 1, 2}: 3 * 2^20 points and 1.65e12 node evaluations.

Prints one JSON line (rank 0). `value` is points/s of the FP64 form over all
ranks (weak scaling: rank r takes rows [r*1024, (r+1)*1024) of an
(N*1024) x 1024 grid over the same rectangle). The same line carries the
mixed-precision study (points/s and per-point error against the FP64
results), the end-to-end number through the host-buffer C-ABI call, the
roofline of the dominant kernel, the clocks seen during the timed region and
the oracle's CPU throughput.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gfc|reference]
    python bench.py --serve            # the serving mix (p50/p99 latency)
"""
from __future__ import annotations

import argparse
import datetime
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "complex p² points/s (2048×256 nodes), FP64 vs mixed @1e-6; serve p50/p99 ms"
RECT = (-10.0, 5.0, -5.0, 5.0)
SIDE = 1024
MASSES2 = (0.25, 1.0, 4.0)          # m in {0.5, 1, 2}
NR, NA = 2048, 256
# the workload both arms (this library and the oracle) name in their JSON line
WORKLOAD = ("bubble m in {0.5,1,2}, D=4, mu2=1, 1024x1024 per GPU over [-10,5]x[-5,5], "
            "2048x256 nodes, FP64")
FLOP_PER_NODE_EVAL = 11              # 22 flops per +-psi pair (9 FMA + 4 MUL)
# DRAM bytes per point of the FP64 evaluation kernel (ncu, one 256x256 launch of the
# current kernel: 243,456 B read, 0 B written back before the launch ended)
TRAFFIC_PER_POINT = 243456 / 65536
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
FP64_FMA_PER_SM_CLK = 2              # nominal GB300 FP64 rate (1.25 TFLOP/s)
FP32_FMA_PER_SM_CLK = 128
L2_FLUSH_BYTES = 256 << 20


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def shard_rows(rank: int, world: int, side: int = None):
    """Rows of the (world*side) x side global grid owned by `rank`, and the
    rectangle of that block."""
    side = SIDE if side is None else side
    re0, re1, im0, im1 = RECT
    total = world * side
    dre = (re1 - re0) / total
    r0 = rank * side
    return (re0 + r0 * dre, re0 + (r0 + side) * dre, im0, im1), (r0, r0 + side)


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running.
    Started before the warm-up (its start-up can stall the GPU briefly, which
    must not fall into a timed region); stop(t0, t1) keeps the samples whose
    nvidia-smi timestamp lies in the timed window [t0, t1] (local time)."""

    QUERY = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self, t0=None, t1=None):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [t.strip() for t in ln.split(",")]
            if len(f) < 10:
                continue
            if t0 is not None:
                try:
                    ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f")
                except ValueError:
                    continue
                if not (t0 <= ts <= t1):
                    continue
            try:
                sm.append(float(f[2]))
                smax.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[6:10]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_points_per_s(npoints: int, seed: int = 5):
    """The oracle (as it stands) on a seeded sample of the production grid
    points, all three masses, on every host core."""
    import oracle
    import synthetic_inputs as si
    idx = si.sample_indices(seed, SIDE * SIDE, npoints)
    x = oracle.grid_points(*RECT, SIDE, SIDE)[idx]
    par = dict(dim=4, mu2=1.0, n_radial=NR, n_angular=NA)
    t0 = time.perf_counter()
    for m2 in MASSES2:
        oracle.eval_points({"kind": "scalar", "m2": m2}, par, x, nthreads=cpu_cores())
    dt = time.perf_counter() - t0
    return 3 * npoints / dt, dt


def run_reference(args):
    ws, rank, _ = dist_setup()
    if rank != 0:
        return 0
    cores = cpu_cores()
    n = args.ref_points
    for _ in range(args.warmup):
        oracle_points_per_s(max(16, n // 8))
    times = []
    for k in range(args.steps):
        v, dt = oracle_points_per_s(n, seed=100 + k)
        times.append(dt)
    tot = sum(times)
    value = args.steps * 3 * n / tot
    sample = f"{n} seeded points of the 1024x1024 grid x 3 masses per step"
    line = {"metric": METRIC, "value": value, "unit": "points/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD,
                       "reference_sample": sample},
            "cpu_baseline": {"value": value, "unit": "points/s", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args):
    import torch
    import paper_1205_0752_gb300 as gfc
    import synthetic_inputs as si
    reqs = si.serving_mix(5, args.serve_requests, rate_hz=args.serve_rate)
    srv = gfc.Server(0, hbm_budget_bytes=40 << 30, max_slots=64)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tickets = []
    for r in reqs:
        now = time.perf_counter() - t0
        if r["t_arrival"] > now:
            time.sleep(r["t_arrival"] - now)
        par = dict(dim=r["dim"], mu2=r["mu2"], n_radial=r["n_radial"],
                   n_angular=r["n_angular"], precision=r["precision"])
        t, _ = srv.submit(r["prop"], par, (*r["rect"], r["side"], r["side"]))
        tickets.append(t)
    for t in tickets:
        srv.wait(t)
    wall = time.perf_counter() - t0
    st = srv.stats()
    if args.serve_log:
        # one JSON line per request: its parameters and the server's record
        with open(args.serve_log, "w") as f:
            for t, r in zip(tickets, reqs):
                rec = {"ticket": int(t), "kind": r["prop"]["kind"], "side": r["side"],
                       "dim": r["dim"], "n_radial": r["n_radial"], "n_angular": r["n_angular"],
                       "precision": r["precision"], "t_arrival_s": r["t_arrival"]}
                rec.update(srv.request_info(t))
                f.write(json.dumps(rec) + "\n")
    srv.close()
    pts = sum(r["side"] ** 2 for r in reqs)
    line = {"metric": "serve p50/p99 ms", "value": st.p99_ms, "unit": "ms",
            "higher_is_better": False, "p50_ms": st.p50_ms, "p99_ms": st.p99_ms,
            "points_per_s": pts / wall, "requests": len(reqs), "completed": st.completed,
            "launches": st.launches, "wall_s": wall, "rate_hz": args.serve_rate,
            "data": "synthetic", "n_gpus": 1,
            "config": {"workload": "serving mix: Poisson arrivals, square grids side in "
                                   "{32..512}, bubble or dressed, D in {3,4}, nodes (256x64)"
                                   "..(2048x256), FP64 or mixed, 40 GB budget"}}
    print(json.dumps(line), flush=True)
    return 0


def run_gfc(args):
    import torch
    ws, rank, local = dist_setup()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    import paper_1205_0752_gb300 as gfc

    side = args.side
    rect, _ = shard_rows(rank, ws, side)
    grid = gfc.make_grid(*rect, side, side)
    # --quick --precision P times the headline workload in precision P (for
    # profiling the other kernels on a small case); the full line is FP64
    par64 = gfc.make_params(dim=4, mu2=1.0, n_radial=NR, n_angular=NA,
                            precision=args.precision if args.quick else "fp64")
    parmx = gfc.make_params(dim=4, mu2=1.0, n_radial=NR, n_angular=NA, precision="mixed")
    props = [gfc.make_prop({"kind": "scalar", "m2": m2}) for m2 in MASSES2]
    outs = [torch.empty((side, side), dtype=torch.complex128, device=dev) for _ in MASSES2]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    npts_step = 3 * side * side

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    def max_over_ranks(v):
        if ws == 1:
            return v
        import torch.distributed as dist
        t = torch.tensor([v], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def step(params, per_launch=None):
        for p, G in zip(props, outs):
            if per_launch is not None:
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                gfc.eval_grid(p, params, grid, out=G, stream=stream)
                b.record(stream)
                per_launch.append((a, b))
            else:
                gfc.eval_grid(p, params, grid, out=G, stream=stream)

    def timed(params, steps, warmup, per_launch=None, clocks=None):
        if clocks:
            clocks.start()
        for _ in range(warmup):
            flush.zero_()                     # also loads the fill kernel before timing
            step(params)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        tw0 = datetime.datetime.now()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            flush.zero_()                     # write 256 MB (> L2) between steps
            step(params, per_launch)
        e1.record(stream)
        torch.cuda.synchronize()
        tw1 = datetime.datetime.now()
        barrier()
        torch.cuda.synchronize()
        ck = clocks.stop(tw0, tw1) if clocks else None
        return max_over_ranks(e0.elapsed_time(e1) / 1e3), ck

    # ---- FP64: the headline ------------------------------------------------
    per_launch = []
    sampler = ClockSampler(dev.index or 0)
    t64, clocks = timed(par64, args.steps, args.warmup, per_launch, sampler)
    launch_ms = [a.elapsed_time(b) for a, b in per_launch]
    st64 = gfc.last_stats()
    node_evals_launch = st64.node_evals
    value = ws * npts_step * args.steps / t64
    G64 = [G.clone() for G in outs]
    if args.quick:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": ws * npts_step * args.steps / t64,
                              "unit": "points/s", "quick": True, "side": side,
                              "precision": args.precision,
                              "launch_ms": [round(v, 3) for v in launch_ms]}), flush=True)
        return 0

    # ---- mixed precision study --------------------------------------------
    per_launch_mx = []
    tmx, _ = timed(parmx, args.steps, 1, per_launch_mx)
    stmx = gfc.last_stats()
    mixed_value = ws * npts_step * args.steps / tmx
    errs = []
    for Gm, Gd in zip(outs, G64):
        a = Gm.cpu().numpy().ravel()
        b = Gd.cpu().numpy().ravel()
        tau = 1e-3 * np.max(np.abs(b))
        errs.append(np.abs(a - b) / np.maximum(np.abs(b), tau))
    err = np.concatenate(errs)
    abs_err = np.concatenate([np.abs(Gm.cpu().numpy().ravel() - Gd.cpu().numpy().ravel())
                              for Gm, Gd in zip(outs, G64)])
    fp64_frac = stmx.points_fp64 / max(1, stmx.points)

    # ---- double-float: FP64-class accuracy on the binary32 pipes ----------
    pardf = gfc.make_params(dim=4, mu2=1.0, n_radial=NR, n_angular=NA, precision="f32x2")
    tdf, _ = timed(pardf, args.steps, 1)
    df_value = ws * npts_step * args.steps / tdf
    errs_df = []
    for Gm, Gd in zip(outs, G64):
        a = Gm.cpu().numpy().ravel()
        b = Gd.cpu().numpy().ravel()
        tau = 1e-3 * np.max(np.abs(b))
        errs_df.append(np.abs(a - b) / np.maximum(np.abs(b), tau))
    err_df = np.concatenate(errs_df)
    # mixed precision whose routed points use the FP64 kernel
    parmd = gfc.make_params(dim=4, mu2=1.0, n_radial=NR, n_angular=NA, precision="mixed",
                            mixed_fallback="fp64")
    tmd, _ = timed(parmd, args.steps, 1)
    md_value = ws * npts_step * args.steps / tmd
    errs_md = []
    for Gm, Gd in zip(outs, G64):
        a = Gm.cpu().numpy().ravel()
        b = Gd.cpu().numpy().ravel()
        tau = 1e-3 * np.max(np.abs(b))
        errs_md.append(np.abs(a - b) / np.maximum(np.abs(b), tau))
    err_md = np.concatenate(errs_md)

    # ---- the paper's angular rule: 49-node tanh-sinh in z (Sect. 4) --------
    paper_rule = {}
    for prec in ("fp64", "f32x2", "mixed"):
        parts = gfc.make_params(dim=4, mu2=1.0, n_radial=NR, n_angular=49,
                                angular_rule="tanh-sinh", precision=prec)
        tts, _ = timed(parts, 1, 1)
        paper_rule[prec] = ws * npts_step / tts

    # ---- the psi integral in closed form (no angular quadrature error) -----
    exact_rule = {}
    for nr in (NR, 4 * NR):
        for prec in ("fp64", "f32x2", "mixed"):
            parex = gfc.make_params(dim=4, mu2=1.0, n_radial=nr, n_angular=2,
                                    angular_rule="exact", precision=prec)
            tex, _ = timed(parex, 1, 1)
            exact_rule[f"{prec}_nr{nr}"] = ws * npts_step / tex

    # ---- near-axis accuracy: closed-form angle + clustered radial rule -----
    clustered = {}
    for prec in ("fp64", "f32x2", "mixed"):
        parcl = gfc.make_params(dim=4, mu2=1.0, n_radial=NR, n_angular=2, angular_rule="exact",
                                radial_rule="clustered", precision=prec)
        tcl, _ = timed(parcl, 1, 1)
        clustered[prec] = ws * npts_step / tcl

    # ---- Step 3 diagnostics: region-1 map and the y-plane map of B --------
    diag = {}
    xg = gfc.grid_points((*rect, side, side), stream=stream).reshape(-1)
    for name, fn in (("region_map_points_per_s", lambda: gfc.region_map(props[1], xg, stream=stream)),
                     ("angular_map_gl256_y_per_s",
                      lambda: gfc.angular_map(props[1], par64, -2.0 + 1.0j, xg, stream=stream)),
                     ("angular_map_exact_y_per_s",
                      lambda: gfc.angular_map(props[1], gfc.make_params(angular_rule="exact"),
                                              -2.0 + 1.0j, xg, stream=stream))):
        fn()
        a_ev, b_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a_ev.record(stream)
        fn()
        b_ev.record(stream)
        torch.cuda.synchronize()
        diag[name] = xg.numel() / (a_ev.elapsed_time(b_ev) / 1e3)

    # ---- end to end through the host-buffer C-ABI call --------------------
    # the block's grid points, made by the library's own Kernel 1 and held in
    # pinned host memory before the timed region
    xh = gfc.grid_points((*rect, side, side), stream=stream).reshape(-1).cpu().pin_memory()
    Gh = torch.empty_like(xh).pin_memory()
    for _ in range(1):
        for p in props:
            gfc.eval_points_host(p, par64, xh, Gh, stream=stream)
    barrier()
    t0 = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 2))
    for _ in range(e2e_steps):
        for p in props:
            gfc.eval_points_host(p, par64, xh, Gh, stream=stream)
    e2e_t = max_over_ranks(time.perf_counter() - t0)
    e2e_value = ws * npts_step * e2e_steps / e2e_t

    def decade_hist(e):
        """counts of relative errors per decade from 1e-15 to 1e-6, plus the
        open ends below 1e-15 and from 1e-6 up"""
        edges = [0.0] + [10.0 ** k for k in range(-15, -5)] + [np.inf]
        counts, _ = np.histogram(e, bins=edges)
        names = ["<1e-15"] + [f"1e{k}..1e{k + 1}" for k in range(-15, -6)] + [">=1e-6"]
        return dict(zip(names, (int(v) for v in counts)))

    # ---- roofline of the dominant kernel ----------------------------------
    avg_launch_s = float(np.mean(launch_ms)) / 1e3
    achieved = FLOP_PER_NODE_EVAL * node_evals_launch / avg_launch_s / 1e12
    peak64 = SM_COUNT * FP64_FMA_PER_SM_CLK * 2 * SM_MAX_MHZ * 1e6 / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t64 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD,
                   "points_per_step": ws * npts_step, "node_evals_per_step": 3 * node_evals_launch * ws,
                   "l2": "256 MB buffer written before every step (> 129 MB L2)",
                   "parallelism": f"rows sharded over {ws} GPU(s), no collective"},
        "node_evals_per_s": 3 * node_evals_launch * ws * args.steps / t64,
        "clocks": clocks,
        "gpu_launches": 2 * 3 * args.steps,
        "roofline": {"bound": "alu", "kernel": "eval_kernel<double,128,1>",
                     "achieved": achieved, "peak": peak64, "unit": "TFLOP/s",
                     "frac": achieved / peak64, "traffic": TRAFFIC_PER_POINT * side * side,
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one "
                                       "256x256 launch (243,456 B), scaled by points per launch",
                     "peak_source": "derived: 152 SM x 2 FP64 FMA/clk x 2 flop x 2070 MHz "
                                    "(ncu: dfma peak_sustained 304/clk = 152 x 2)",
                     "algorithmic": "11 flop per node-eval (22 per +-psi pair)",
                     "executed_pairs_per_launch": st64.pairs_evaluated,
                     "algorithmic_pairs_per_launch": node_evals_launch // 2,
                     "executed_fraction": st64.pairs_evaluated / max(1, node_evals_launch // 2),
                     "executed_tflops": 2 * FLOP_PER_NODE_EVAL * st64.pairs_evaluated / avg_launch_s / 1e12,
                     "executed_frac": 2 * FLOP_PER_NODE_EVAL * st64.pairs_evaluated / avg_launch_s / 1e12 / peak64,
                     "note": "compressed angular rules evaluate executed_fraction of the "
                             "algorithmic pairs for the same sums (to rounding), so the "
                             "algorithmic rate exceeds the FP64 pipe peak; executed_frac counts "
                             "the same 22 flop per pair actually evaluated; ncu shows the FP64 "
                             "pipe 89.6% busy (profiles/eval_kernel_fp64_production_bubble.md)"},
        "mixed": {"value": mixed_value, "unit": "points/s", "ms_per_step": 1e3 * tmx / args.steps,
                  "max_rel_err": float(err.max()), "p99_rel_err": float(np.percentile(err, 99)),
                  "median_rel_err": float(np.median(err)), "max_abs_err": float(abs_err.max()),
                  "frac_rel_err_gt_1e-6": float(np.mean(err > 1e-6)),
                  "rel_err_hist": decade_hist(err),
                  "fp64_point_fraction": fp64_frac,
                  "error_vs": "FP64 GPU results (parity <= 1e-10 with the oracle)",
                  "fp32_peak_tflops": SM_COUNT * FP32_FMA_PER_SM_CLK * 2 * SM_MAX_MHZ * 1e6 / 1e12,
                  "achieved_tflops": FLOP_PER_NODE_EVAL * 3 * node_evals_launch * args.steps / tmx / 1e12},
        "f32x2": {"value": df_value, "unit": "points/s", "ms_per_step": 1e3 * tdf / args.steps,
                  "max_rel_err": float(err_df.max()), "median_rel_err": float(np.median(err_df)),
                  "rel_err_hist": decade_hist(err_df),
                  "error_vs": "FP64 GPU results",
                  "arith": "double-float (pairs of binary32) on the binary32 pipes"},
        "mixed_fp64_fallback": {"value": md_value, "unit": "points/s",
                                 "ms_per_step": 1e3 * tmd / args.steps,
                                 "max_rel_err": float(err_md.max()),
                                 "frac_rel_err_gt_1e-6": float(np.mean(err_md > 1e-6))},
        "paper_angular_rule": {"rule": "tanh-sinh, 49 nodes in z = cos psi (Sect. 4)",
                               "n_radial": NR, "unit": "points/s",
                               "fp64": paper_rule["fp64"], "f32x2": paper_rule["f32x2"],
                               "mixed": paper_rule["mixed"]},
        "exact_angular": dict({"rule": "psi integral in closed form (limit of every angular "
                                         "rule); radial Gauss-Legendre n_radial as named",
                               "unit": "points/s"}, **exact_rule),
        "clustered_radial": dict({"rule": "closed-form angle, radial rule sinh-clustered at the "
                                          "pole nearest the ray (n_radial 2048)",
                                  "unit": "points/s"}, **clustered),
        "diagnostics": dict({"grid": f"{side}x{side} x (region map) or y (map of B at x = -2 + i)",
                             "propagator": "bubble m = 1"}, **diag),
        "e2e": {"value": e2e_value, "unit": "points/s", "h2d_bytes_per_step": 3 * 16 * side * side,
                "d2h_bytes_per_step": 3 * 16 * side * side},
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        v, dt = oracle_points_per_s(args.ref_points)
        line["cpu_baseline"] = {"value": v, "unit": "points/s", "cores": cpu_cores(),
                                "kind": "oracle",
                                "sample": f"{args.ref_points} seeded grid points x 3 masses "
                                          f"({dt:.1f} s)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gfc", choices=["gfc", "reference"])
    # ~13 s of the oracle on 16 host cores (3 x 6144 points at ~1.4e3 points/s)
    ap.add_argument("--ref-points", type=int, default=6144)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--side", type=int, default=SIDE,
                    help="grid side per GPU (the benchmark workload is 1024)")
    ap.add_argument("--quick", action="store_true",
                    help="FP64 timing only (profiling runs)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "f32x2", "mixed"],
                    help="with --quick: the precision of the timed workload")
    ap.add_argument("--serve", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-log", default=None,
                    help="with --serve: write one JSON line per request to this file")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.serve:
        return run_serve(args)
    return run_gfc(args)


if __name__ == "__main__":
    sys.exit(main())
