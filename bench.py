#!/usr/bin/env python3
"""Benchmark of the hot path: G(x) on the production bubble grid.

Workload (one step): the equal-mass scalar bubble, D = 4, mu2 = 1, on the
1024 x 1024 cell-centred grid over Re x in [-10, 5], Im x in [-5, 5], with
2048 radial x 256 angular Gauss-Legendre nodes, for the three masses
m in {0.5, 1, 2}: 3 * 2^20 points and 1.65e12 node evaluations.

Prints one JSON line (rank 0). `value` is points/s of the FP64 form over all
ranks (weak scaling: rank r takes the rows i = r (mod N) of an (N*1024) x 1024
grid over the same rectangle, so every rank carries the same mix of cheap and
expensive points). The same line carries the mixed-precision and
double-float studies (points/s and per-point error against the FP64
results), the other workload configurations (the paper's worked example, the
64 x 64 bubble, the dressed 512 x 512 grids), the serving mix (p50/p99
latency), the end-to-end number through the host-buffer C-ABI call, the
roofline of the dominant kernel against the pipe rates measured on the
device, the clocks seen during the timed region and the oracle's CPU
throughput.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gfc|reference]
    python bench.py --serve            # the serving mix alone (p50/p99 latency)

With --gpus N > 1 and no torch.distributed environment, the script starts
itself again under torch.distributed.run with N ranks on this node.
"""
from __future__ import annotations

import argparse
import datetime
import json
import os
import socket
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
L2_FLUSH_BYTES = 256 << 20

# Executed work of the evaluation kernels, per unit of their own counters:
# thread instructions per angular pair on a compressed rule, per pair over
# the full table and per contour node, for each model key (see
# model_values): fp64 the FP64 pipe's thread slots (32 per warp instruction),
# dfma/dmul/dadd the binary64 instructions, fma_ops the binary32 FMA-pipe
# operations (paired forms twice), inst the warp instructions issued. Fitted
# by `bench.py --fit-exec-model` to ncu's counters of the --calib launches
# (256 x 256 grids of the production bubble): tuples (per compressed pair,
# per full-table pair, per node, per point); every fit reproduces its
# launches' counts to <= 1.4 % (inst of the binary64 list: its empty
# launches aside). fp64 is the FP64 kernel, list64 the mixed form's binary64
# list, f32x2 the double-float kernel, bulk32p the mixed form's binary32 bulk,
# nodes_df its double-float node groups.
EXEC_MODEL = {
    "fp64": {"dfma": (7.0, 7.0, 33.313, 0.0), "dmul": (0.0, 2.0, 27.079, 0.0),
             "dadd": (0.004, 0.016, 2.609, 0.0), "fp64": (7.008, 9.016, 63.296, 0.0),
             "fma_ops": (0.002, 0.0, 10.927, 0.0), "inst": (1.261, 1.528, 13.301, 0.0)},
    "list64": {"dfma": (7.0, 7.0, 33.313, 0.0), "dmul": (0.0, 2.0, 27.079, 0.0),
               "dadd": (0.0, 0.016, 2.656, 0.0), "fp64": (7.0, 9.016, 63.391, 0.0),
               "fma_ops": (-0.002, 0.0, 10.965, 0.0), "inst": (0.945, 1.507, 16.584, 0.0)},
    "f32x2": {"dfma": (0.0, 0.0, 0.673, 0.0), "dmul": (0.0, 0.0, 0.313, 0.0),
              "dadd": (0.004, 0.0, 0.578, 0.0), "fp64": (0.008, 0.001, 2.124, 0.0),
              "fma_ops": (63.002, 77.0, 740.286, 0.0), "inst": (2.314, 2.716, 26.613, 0.0)},
    "bulk32p": {"dfma": (0.0, 0.0, 0.64, 0.0), "dmul": (0.0, 0.0, 0.281, 0.0),
                "dadd": (0.0, 0.0, 0.171, 0.0), "fp64": (0.019, 0.001, 1.509, 0.0),
                "fma_ops": (6.766, 6.057, 182.052, 0.0), "inst": (0.388, 0.293, 10.945, 0.0)},
    "nodes_df": {"dfma": (0.0, 0.0, 0.0, 1218.0), "dmul": (0.0, 0.0, 0.0, 544.0),
                 "dadd": (0.0, 0.0, 0.0, 1151.885), "fp64": (0.0, 0.0, -0.001, 4063.77),
                 "fma_ops": (63.001, 77.0, 729.867, 21385.077), "inst": (2.311, 2.716, 25.927, 2681.82)},
}
# DRAM bytes per point of the FP64 evaluation kernel: ncu's
# dram__bytes_read.sum + dram__bytes_write.sum of the calibration launches of
# the production grid (256 x 256 points, compressed rules, m^2 = 0.25, 1, 4:
# 5.11, 4.73, 4.15 B per point), scaled to a launch by its points. Below the
# 16 B of output per point: the output drains from L2 after the kernel ends.
TRAFFIC_PER_POINT = 4.66


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def shard_rect(rank: int, world: int, side: int = None):
    """The rows i = rank (mod world) of the (world*side) x side cell-centred
    grid over RECT, as a side x side cell-centred grid of their own: row j of
    the shard is global row world*j + rank."""
    side = SIDE if side is None else side
    re0, re1, im0, im1 = RECT
    dre = (re1 - re0) / (world * side)
    a = re0 + (rank + 0.5 - 0.5 * world) * dre
    return (a, a + (re1 - re0), im0, im1)


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def relaunch(nprocs: int, argv, script: str = None, **run_kw):
    """Runs `script` (this file by default) under torch.distributed.run with
    nprocs ranks on this node (rendezvous on 127.0.0.1); returns the
    CompletedProcess."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
           f"--nproc-per-node={nprocs}", "--master-addr", "127.0.0.1",
           "--master-port", str(_free_port()), script or os.path.abspath(__file__)] + list(argv)
    return subprocess.run(cmd, **run_kw)


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


# --------------------------------------------------------------------------
# serving
# --------------------------------------------------------------------------

def serve_warmup(gfc, srv):
    """One 32 x 32 request of every request class of the mix (propagator
    kind, D, node orders, precision), waited for: the node tables of every
    class are built and every kernel variant loaded before the timed
    requests, as for a server that has run a while."""
    import synthetic_inputs as si
    rect = si.grid_rect("small")
    tickets = []
    for prop in ({"kind": "scalar", "m2": 1.0}, {"kind": "dressed", "a": 1.25, "b": 0.5, "c": 2.5}):
        for dim in (3, 4):
            for nr, na in si.SERVING_NODES:
                for prec in ("fp64", "mixed"):
                    par = dict(dim=dim, mu2=1.0, n_radial=nr, n_angular=na, precision=prec)
                    tickets.append(srv.submit(prop, par, (*rect, 32, 32))[0])
    for t in tickets:
        srv.wait(t)


def serve_mix(gfc, reqs, log_path=None):
    """Submits the requests at their arrival times to a 40 GB server (after
    its warm-up), waits for all of them, and returns the latency and
    throughput record of these requests."""
    import torch
    srv = gfc.Server(0, hbm_budget_bytes=40 << 30, max_slots=64)
    serve_warmup(gfc, srv)
    st0 = srv.stats()
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
    bad = sum(1 for t in tickets if srv.wait(t) != 0)
    wall = time.perf_counter() - t0
    st = srv.stats()
    infos = [srv.request_info(t) for t in tickets]
    if log_path:
        with open(log_path, "w") as f:
            for t, r, info in zip(tickets, reqs, infos):
                rec = {"ticket": int(t), "kind": r["prop"]["kind"], "side": r["side"],
                       "dim": r["dim"], "n_radial": r["n_radial"], "n_angular": r["n_angular"],
                       "precision": r["precision"], "t_arrival_s": r["t_arrival"]}
                rec.update(info)
                f.write(json.dumps(rec) + "\n")
    srv.close()
    pts = sum(r["side"] ** 2 for r in reqs)
    lat = np.array([i["total_ms"] for i in infos])
    return {"requests": len(reqs), "completed": int(st.completed - st0.completed), "failed": bad,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "max_ms": float(lat.max()), "points_per_s": pts / wall, "wall_s": wall,
            "launches": int(st.launches - st0.launches),
            "offered_points_per_s": pts / max(reqs[-1]["t_arrival"], 1e-9),
            "warmup": "one 32x32 request of each of the 32 request classes before the timed requests"}


def serve_study(gfc, n_spec=2000, rate=200.0, n_load=600, load=0.7):
    """The specified mix (Poisson arrivals at `rate`), then a run at `load`
    times the capacity the first run measured (the same request
    distribution, another seed)."""
    import synthetic_inputs as si
    spec = serve_mix(gfc, si.serving_mix(5, n_spec, rate_hz=rate))
    probe = si.serving_mix(6, n_load, rate_hz=1.0)
    mean_pts = np.mean([r["side"] ** 2 for r in probe])
    rate70 = load * spec["points_per_s"] / mean_pts
    sus = serve_mix(gfc, si.serving_mix(6, n_load, rate_hz=rate70))
    sus["rate_hz"] = rate70
    spec["rate_hz"] = rate
    return {"unit": "ms", "spec": spec, "load70": sus,
            "workload": "serving mix: Poisson arrivals, square grids side in {32..512}, bubble "
                        "(m in {0.5,1,2}) or dressed, D in {3,4}, nodes (256x64)..(2048x256), FP64 "
                        "or mixed, 40 GB budget, 64 slots; load70 at 70% of the capacity the "
                        "specified run measured"}


def run_serve(args):
    import paper_1205_0752_gb300 as gfc
    import synthetic_inputs as si
    rec = serve_mix(gfc, si.serving_mix(5, args.serve_requests, rate_hz=args.serve_rate),
                    args.serve_log)
    line = {"metric": "serve p50/p99 ms", "value": rec["p99_ms"], "unit": "ms",
            "higher_is_better": False, "rate_hz": args.serve_rate, "data": "synthetic",
            "n_gpus": 1, **rec,
            "config": {"workload": "serving mix: Poisson arrivals, square grids side in "
                                   "{32..512}, bubble or dressed, D in {3,4}, nodes (256x64)"
                                   "..(2048x256), FP64 or mixed, 40 GB budget"}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# executed work and rooflines
# --------------------------------------------------------------------------

def executed(arith, pairs, pairs_full, nodes, points=0):
    """Thread instructions per pipe (and issued warp instructions) of a launch
    of the `arith` kernel (a key of EXEC_MODEL) from its counters."""
    if not EXEC_MODEL or arith not in EXEC_MODEL:
        return None
    m = EXEC_MODEL[arith]
    pc = pairs - pairs_full
    return {k: m[k][0] * pc + m[k][1] * pairs_full + m[k][2] * nodes + m[k][3] * points
            for k in m}


def fp64_pipe_seconds(ex, peaks):
    """Time the FP64 pipe needs for the executed FP64-pipe instructions (32
    thread slots per warp instruction: DFMA, DMUL, DADD, conversions and
    compares) at the rate measured for a stream of binary64 FMA, multiply and
    add in the FP64 kernel's proportions (the pipe issues a mixed stream
    faster than any one of them alone)."""
    return ex["fp64"] / peaks["fp64_mix_per_s"]


def fma_pipe_seconds(ex, peaks):
    """Time the FP32 FMA pipes need for the executed FFMA, FMUL and FADD
    (paired forms count twice) at the measured FFMA rate."""
    return ex["fma_ops"] / peaks["ffma_per_s"]


# --------------------------------------------------------------------------
# calibration of the executed-work model (EXEC_MODEL) from ncu counters
# --------------------------------------------------------------------------
# ncu metrics of one calibration capture, and what each model key is made of
CALIB_METRICS = [
    "gpu__time_duration.sum", "smsp__inst_executed.sum", "sm__inst_executed_pipe_fp64.sum",
    "sm__sass_thread_inst_executed_op_dfma_pred_on.sum",
    "sm__sass_thread_inst_executed_op_dmul_pred_on.sum",
    "sm__sass_thread_inst_executed_op_dadd_pred_on.sum",
    "sm__sass_thread_inst_executed_op_ffma_pred_on.sum",
    "sm__sass_thread_inst_executed_op_fmul_pred_on.sum",
    "sm__sass_thread_inst_executed_op_fadd_pred_on.sum",
    "sm__sass_thread_inst_executed_op_ffma2_pred_on.sum",
    "sm__sass_thread_inst_executed_op_fmul2_pred_on.sum",
    "sm__sass_thread_inst_executed_op_fadd2_pred_on.sum",
    "sm__pipe_fp64_cycles_active.avg.pct_of_peak_sustained_elapsed",
    "sm__pipe_fma_cycles_active.avg.pct_of_peak_sustained_elapsed",
    "smsp__issue_active.avg.pct_of_peak_sustained_elapsed",
    "dram__bytes_read.sum", "dram__bytes_write.sum",
]
# calibration cases: 256 x 256 grids of the production bubble (2048 x 256 nodes)
CALIB_CASES = [("m2=1", 1.0, RECT, False), ("m2=1 full table", 1.0, RECT, False),
               ("m2=0.25", 0.25, RECT, False), ("m2=4", 4.0, RECT, False),
               ("right half-plane m2=1", 1.0, (0.5, 5.0, -5.0, 5.0), False)]


def run_calib(args):
    """One call per calibration case in the given precision (after one
    untimed call of the first case), each followed by a JSON line of its
    counters: the launches an ncu capture of eval_kernel / eval_bulk sees,
    in order."""
    import torch
    import paper_1205_0752_gb300 as gfc
    from paper_1205_0752_gb300 import binding
    par = gfc.make_params(dim=4, mu2=1.0, n_radial=NR, n_angular=NA, precision=args.precision)
    side = 256
    for k, (name, m2, rect, _) in enumerate([CALIB_CASES[0]] + CALIB_CASES):
        binding.test_full_angular_rule("full table" in name and k > 0)
        try:
            gfc.eval_grid(gfc.make_prop({"kind": "scalar", "m2": m2}), par, (*rect, side, side))
            torch.cuda.synchronize()
            st = gfc.last_stats()
        finally:
            binding.test_full_angular_rule(False)
        rec = {"case": name if k > 0 else "warm-up", "precision": args.precision}
        rec.update({f: int(getattr(st, f)) for f in st.__dataclass_fields__})
        print(json.dumps(rec), flush=True)
    return 0


def calib_units(rec, kernel):
    """(pairs on compressed rules, pairs over the full table, contour nodes,
    points) of one kernel of a calibration call: 'fp64' and 'f32x2' the whole
    call, 'bulk32p' / 'nodes_df' / 'list64' the three kernels of a mixed call
    (the fallback's points are its node-list entries, the binary64 list's
    the points evaluated whole in binary64)."""
    na = NA
    if kernel in ("fp64", "f32x2"):
        p, pf, n = rec["pairs_evaluated"], rec["pairs_full_table"], rec["node_evals"] // na
        pts = rec["points"]
    elif kernel == "nodes_df":
        p, pf, n = rec["pairs_fallback"], rec["pairs_full_table_fallback"], rec["node_evals_fallback"] // na
        pts = rec["points_partial"]
    elif kernel == "list64":
        p, pf, n = rec["pairs_list64"], rec["pairs_full_table_list64"], rec["node_evals_list64"] // na
        pts = rec["points_fp64"]
    else:
        p = rec["pairs_evaluated"] - rec["pairs_fallback"] - rec["pairs_list64"]
        pf = rec["pairs_full_table"] - rec["pairs_full_table_fallback"] - rec["pairs_full_table_list64"]
        n = (rec["node_evals"] - rec["node_evals_fallback"] - rec["node_evals_list64"]) // na
        pts = rec["points"]
    return p - pf, pf, n, pts


def kernel_class(name: str, precision: str) -> str:
    """Model key of an ncu launch of a calibration call."""
    if "eval_bulk_partial_kernel" in name:
        return "bulk32p"
    if "gfc::df" in name or "eval_kernel<df" in name:
        return "nodes_df" if precision == "mixed" else "f32x2"
    return "list64" if precision == "mixed" else "fp64"


def model_values(row):
    """The model's per-launch quantities from one ncu launch's metrics:
    fp64 (FP64-pipe thread slots: 32 per warp instruction), dfma, dmul, dadd
    (thread instructions), fma_ops (binary32 FMA-pipe operations, paired
    forms twice) and inst (warp instructions issued)."""
    g = lambda k: float(row.get(k, 0.0) or 0.0)
    t = "sm__sass_thread_inst_executed_op_%s_pred_on.sum"
    return {"fp64": 32.0 * g("sm__inst_executed_pipe_fp64.sum"),
            "dfma": g(t % "dfma"), "dmul": g(t % "dmul"), "dadd": g(t % "dadd"),
            "fma_ops": g(t % "ffma") + g(t % "fmul") + g(t % "fadd") +
                       2.0 * (g(t % "ffma2") + g(t % "fmul2") + g(t % "fadd2")),
            "inst": g("smsp__inst_executed.sum")}


def read_ncu_csv(path):
    """Launches of an `ncu --csv --metrics ...` log: a list of (kernel name,
    {metric: value}) in launch order."""
    import csv
    rows = {}
    with open(path) as f:
        lines = [ln for ln in f if ln.startswith('"')]
    for r in csv.DictReader(lines):
        key = int(r["ID"])
        name = r.get("Kernel Name", "")
        val = r.get("Metric Value", "").replace(",", "")
        try:
            v = float(val)
        except ValueError:
            continue
        unit = r.get("Metric Unit", "")
        if unit in ("msecond", "ms"):
            v *= 1e-3
        elif unit in ("usecond", "us"):
            v *= 1e-6
        elif unit in ("nsecond", "ns"):
            v *= 1e-9
        rows.setdefault(key, (name, {}))[1][r["Metric Name"]] = v
    return [rows[k] for k in sorted(rows)]


def fit_exec_model(pairs_of_files):
    """Least-squares fit of every model key of every kernel class: value per
    launch = a (compressed pairs) + b (full-table pairs) + c (nodes) + d
    (points), over the calibration launches (the warm-up call left out); the
    points column only for the mixed form's fallback and binary64 list, and
    left out (d = 0) where it is proportional to the nodes (every point with
    the same contour), its work then counted per node.
    Returns the model, the worst relative residual per kernel and key, and
    ncu's own pipe figures beside the model's counts."""
    samples = {}
    for csv_path, counters_path in pairs_of_files:
        recs = [json.loads(ln) for ln in open(counters_path) if ln.startswith("{")]
        launches = read_ncu_csv(csv_path)
        prec = recs[0]["precision"]
        # group the launches by call: a call starts with its first eval kernel
        # (mixed: the binary32 bulk; else one kernel per call)
        calls, cur = [], None
        for name, row in launches:
            kc = kernel_class(name, prec)
            if prec != "mixed" or kc == "bulk32p" or cur is None:
                cur = []
                calls.append(cur)
            cur.append((kc, row))
        assert len(calls) == len(recs), (csv_path, len(calls), len(recs))
        for rec, call in zip(recs[1:], calls[1:]):
            for kc, row in call:
                samples.setdefault(kc, []).append((calib_units(rec, kc), model_values(row), row,
                                                   rec["case"]))
    model, report = {}, {}
    for kc, rows in sorted(samples.items()):
        X = np.array([u for u, _, _, _ in rows], dtype=float)
        # columns with no work in any launch (e.g. no full-table pairs) fit to
        # 0; a per-point term only for the kernels whose points carry very
        # different numbers of nodes (the fallback's node groups, the binary64
        # list), and only where it is not proportional to the nodes
        used = np.any(X != 0, axis=0)
        used[3] = used[3] and kc in ("nodes_df", "list64")
        if used[3] and np.linalg.matrix_rank(X[:, used]) < int(used.sum()):
            used[3] = False
        model[kc] = {}
        for key in ("dfma", "dmul", "dadd", "fp64", "fma_ops", "inst"):
            y = np.array([v[key] for _, v, _, _ in rows])
            coef = np.zeros(4)
            if used.any():
                coef[used] = np.linalg.lstsq(X[:, used], y, rcond=None)[0]
            pred = X @ coef
            # relative to the launch's count, launches without work (a few
            # hundred instructions of set-up) held to an absolute floor
            res = np.max(np.abs(pred - y) / np.maximum(np.abs(y), 1e6))
            model[kc][key] = tuple(round(float(c), 3) for c in coef)
            report.setdefault(kc, {})[key] = float(res)
        report[kc]["launches"] = [
            {"case": c, "ms": 1e3 * r.get("gpu__time_duration.sum", 0.0),
             "dram_bytes": r.get("dram__bytes_read.sum", 0.0) + r.get("dram__bytes_write.sum", 0.0),
             "fp64_pipe_pct": r.get("sm__pipe_fp64_cycles_active.avg.pct_of_peak_sustained_elapsed"),
             "fma_pipe_pct": r.get("sm__pipe_fma_cycles_active.avg.pct_of_peak_sustained_elapsed"),
             "issue_pct": r.get("smsp__issue_active.avg.pct_of_peak_sustained_elapsed")}
            for _, _, r, c in rows]
    return model, report


# --------------------------------------------------------------------------
# the library's arm
# --------------------------------------------------------------------------

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
    import synthetic_inputs as si
    from paper_1205_0752_gb300 import binding

    side = args.side
    rect = shard_rect(rank, ws, side)
    grid = gfc.make_grid(*rect, side, side)
    # --quick --precision P times the headline workload in precision P (for
    # profiling the other kernels on a small case); the full line is FP64
    prec0 = args.precision if args.quick else "fp64"
    par64 = gfc.make_params(dim=4, mu2=1.0, n_radial=NR, n_angular=NA, precision=prec0)
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

    def step(params, per_launch=None, stats=None, props_=None, outs_=None, grid_=None):
        for k, (p, G) in enumerate(zip(props_ or props, outs_ or outs)):
            if per_launch is not None:
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                gfc.eval_grid(p, params, grid_ or grid, out=G, stream=stream)
                b.record(stream)
                per_launch.setdefault(k, []).append((a, b))
            else:
                gfc.eval_grid(p, params, grid_ or grid, out=G, stream=stream)
            if stats is not None:
                stats.append(gfc.last_stats())    # (synchronises: warm-up only)

    def timed(params, steps, warmup, per_launch=None, clocks=None, stats=None, **kw):
        """K timed steps after W warm-up steps (the first warm-up step records
        each launch's counters), L2 flushed before every step."""
        if clocks:
            clocks.start()
        for w in range(warmup):
            flush.zero_()                     # also loads the fill kernel before timing
            step(params, stats=stats if w == 0 else None, **kw)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        tw0 = datetime.datetime.now()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            flush.zero_()                     # write 256 MB (> L2) between steps
            step(params, per_launch, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        tw1 = datetime.datetime.now()
        barrier()
        torch.cuda.synchronize()
        ck = clocks.stop(tw0, tw1) if clocks else None
        return max_over_ranks(e0.elapsed_time(e1) / 1e3), ck

    def launch_seconds(per_launch):
        """mean CUDA-event seconds of each launch index over the timed steps"""
        return [float(np.mean([a.elapsed_time(b) for a, b in per_launch[k]])) / 1e3
                for k in sorted(per_launch)]

    def rel_errors(got, ref):
        errs = []
        for a, b in zip(got, ref):
            a = a.cpu().numpy().ravel() if hasattr(a, "cpu") else np.ravel(a)
            b = b.cpu().numpy().ravel() if hasattr(b, "cpu") else np.ravel(b)
            tau = 1e-3 * np.max(np.abs(b))
            errs.append(np.abs(a - b) / np.maximum(np.abs(b), tau))
        return np.concatenate(errs)

    # ---- measured pipe rates (the roofline denominators) --------------------
    peaks = gfc.measure_pipe_peaks(0.2, stream=stream)

    # ---- FP64: the headline ------------------------------------------------
    per_launch, st64 = {}, []
    sampler = ClockSampler(dev.index or 0)
    t64, clocks = timed(par64, args.steps, max(args.warmup, 1), per_launch, sampler, st64)
    launch_s = launch_seconds(per_launch)
    value = ws * npts_step * args.steps / t64
    if args.quick:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "points/s", "quick": True,
                              "side": side, "precision": args.precision,
                              "launch_ms": [round(1e3 * v, 3) for v in launch_s]}), flush=True)
        return 0
    G64 = [G.clone() for G in outs]
    node_evals_step = sum(s.node_evals for s in st64)

    def roofline_fp64(stats, secs):
        """FP64-pipe fraction of the FP64 kernel over the given launches."""
        out = {"algorithmic_node_evals": int(sum(s.node_evals for s in stats)),
               "pairs_evaluated": int(sum(s.pairs_evaluated for s in stats)),
               "pairs_full_table": int(sum(s.pairs_full_table for s in stats)),
               "seconds": float(sum(secs))}
        out["effective_tflops"] = FLOP_PER_NODE_EVAL * out["algorithmic_node_evals"] / out["seconds"] / 1e12
        ex = [executed("fp64", s.pairs_evaluated, s.pairs_full_table, s.node_evals // (2 * NA // 2),
                       s.points)
              for s in stats]
        if ex[0] is not None:
            busy = sum(fp64_pipe_seconds(e, peaks) for e in ex)
            fl = sum(2 * e["dfma"] + e["dmul"] + e["dadd"] for e in ex)
            out.update(pipe_frac=busy / out["seconds"], executed_tflops=fl / out["seconds"] / 1e12,
                       fp64_pipe_inst=float(sum(e["fp64"]
                                                for e in ex)))
        return out

    rf = roofline_fp64(st64, launch_s)
    peak_fma_tflops = 2 * peaks["fp64_mix_per_s"] / 1e12
    frac = rf.get("pipe_frac")
    roofline = {
        "bound": "alu", "kernel": "eval_kernel<double,128,1,0>",
        "unit": "TFLOP/s",
        # FMA-equivalent rate: every FP64-pipe instruction counted as one FMA
        # slot (2 flop) at the measured DFMA/DMUL/DADD rates, so that
        # achieved/peak is the FP64 pipe's busy fraction
        "achieved": frac * peak_fma_tflops if frac is not None else None,
        "peak": peak_fma_tflops,
        "frac": frac,
        "traffic": TRAFFIC_PER_POINT * side * side if TRAFFIC_PER_POINT else None,
        "peak_source": "measured on this device by gfc_measure_pipe_peaks: binary64 FMA, "
                       "multiply and add chains in the kernel's proportions 5:2:1 (best of 4 "
                       "launch shapes), each instruction one FMA slot; of measured",
        "executed_tflops": rf.get("executed_tflops"),
        "effective_tflops": rf["effective_tflops"],
        "effective_note": "11 flop per algorithmic node-eval of the 2048x256 quadrature over "
                          "the kernel time; the compressed angular rules evaluate "
                          "pairs_evaluated of the node_evals/2 pairs for the same sums, so this "
                          "rate is not bounded by the pipe",
        "pairs_evaluated_per_step": rf["pairs_evaluated"],
        "pairs_full_table_per_step": rf["pairs_full_table"],
        "algorithmic_pairs_per_step": rf["algorithmic_node_evals"] // 2,
        "per_mass": [dict(m2=m2, launch_ms=1e3 * s,
                          pipe_frac=roofline_fp64([st], [s]).get("pipe_frac"))
                     for m2, st, s in zip(MASSES2, st64, launch_s)],
        "measured_peaks": peaks,
    }

    # ---- mixed precision ---------------------------------------------------
    def mixed_roofline(stats, secs, fallback):
        """Issue and pipe fractions of a mixed step: the binary32 bulk and the
        fallback kernel (double-float or FP64) together."""
        if not EXEC_MODEL or fallback != "f32x2":
            return {}
        fma_s = fp64_s = 0.0
        for s in stats:
            # the three kernels of a mixed call: the binary32 bulk (whole
            # points outside the cut band), the node groups re-evaluated in
            # double-float, and the cut band in binary64
            n_fb, n_64 = s.node_evals_fallback // NA, s.node_evals_list64 // NA
            n_b = s.node_evals // NA - n_fb - n_64
            pf_b = s.pairs_full_table - s.pairs_full_table_fallback - s.pairs_full_table_list64
            eb = executed("bulk32p", s.pairs_evaluated - s.pairs_fallback - s.pairs_list64, pf_b, n_b,
                          s.points)
            ef = executed("nodes_df", s.pairs_fallback, s.pairs_full_table_fallback, n_fb,
                          s.points_partial)
            e6 = executed("list64", s.pairs_list64, s.pairs_full_table_list64, n_64, s.points_fp64)
            if None in (eb, ef, e6):
                # (a kernel of the call has no calibrated instruction model)
                return {}
            fma_s += sum(fma_pipe_seconds(e, peaks) for e in (eb, ef, e6))
            fp64_s += sum(fp64_pipe_seconds(e, peaks) for e in (eb, ef, e6))
        T = float(sum(secs))
        return {"fma_pipe_frac": fma_s / T, "fp64_pipe_frac": fp64_s / T,
                "peak_ffma_tflops": 2 * peaks["ffma_per_s"] / 1e12}

    per_launch_mx, stmx = {}, []
    tmx, _ = timed(parmx, args.steps, 1, per_launch_mx, stats=stmx)
    mixed_value = ws * npts_step * args.steps / tmx
    err = rel_errors(outs, G64)
    abs_err = np.concatenate([np.abs(Gm.cpu().numpy().ravel() - Gd.cpu().numpy().ravel())
                              for Gm, Gd in zip(outs, G64)])

    def decade_hist(e):
        """counts of relative errors per decade from 1e-15 to 1e-6, plus the
        open ends below 1e-15 and from 1e-6 up"""
        edges = [0.0] + [10.0 ** k for k in range(-15, -5)] + [np.inf]
        counts, _ = np.histogram(e, bins=edges)
        names = ["<1e-15"] + [f"1e{k}..1e{k + 1}" for k in range(-15, -6)] + [">=1e-6"]
        return dict(zip(names, (int(v) for v in counts)))

    mixed = {"value": mixed_value, "unit": "points/s", "ms_per_step": 1e3 * tmx / args.steps,
             "max_rel_err": float(err.max()), "p99_rel_err": float(np.percentile(err, 99)),
             "median_rel_err": float(np.median(err)), "max_abs_err": float(abs_err.max()),
             "frac_rel_err_gt_1e-6": float(np.mean(err > 1e-6)),
             "rel_err_hist": decade_hist(err),
             "error_vs": "FP64 GPU results (parity <= 1e-10 with the oracle)",
             "fallback": "double-float (f32x2)",
             # per mass: the share of points evaluated whole in binary64 (the
             # cut band and points next to a pinch), of points with node groups
             # re-evaluated in double-float, and of node evaluations done in
             # double-float
             "routed_fraction_per_mass": [dict(m2=m2, points_binary64_whole=s.points_fp64 / s.points,
                                               points_with_fallback_groups=s.points_partial / s.points,
                                               fallback_node_evals=s.node_evals_fallback / max(1, s.node_evals))
                                          for m2, s in zip(MASSES2, stmx)],
             "per_mass_ms": [1e3 * s for s in launch_seconds(per_launch_mx)],
             **mixed_roofline(stmx, launch_seconds(per_launch_mx), "f32x2")}

    # ---- double-float: FP64-class accuracy on the binary32 pipes ----------
    pardf = gfc.make_params(dim=4, mu2=1.0, n_radial=NR, n_angular=NA, precision="f32x2")
    per_launch_df, stdf = {}, []
    tdf, _ = timed(pardf, args.steps, 1, per_launch_df, stats=stdf)
    err_df = rel_errors(outs, G64)
    f32x2 = {"value": ws * npts_step * args.steps / tdf, "unit": "points/s",
             "ms_per_step": 1e3 * tdf / args.steps,
             "max_rel_err": float(err_df.max()), "median_rel_err": float(np.median(err_df)),
             "rel_err_hist": decade_hist(err_df), "error_vs": "FP64 GPU results",
             "arith": "double-float (pairs of binary32) on the binary32 pipes"}
    if EXEC_MODEL:
        T = sum(launch_seconds(per_launch_df))
        ex = [executed("f32x2", s.pairs_evaluated, s.pairs_full_table, s.node_evals // NA, s.points)
              for s in stdf]
        f32x2["fma_pipe_frac"] = sum(fma_pipe_seconds(e, peaks) for e in ex) / T

    # mixed precision whose routed work uses the FP64 kernel
    parmd = gfc.make_params(dim=4, mu2=1.0, n_radial=NR, n_angular=NA, precision="mixed",
                            mixed_fallback="fp64")
    nmd = max(3, min(args.steps, 5))
    tmd, _ = timed(parmd, nmd, 1)
    err_md = rel_errors(outs, G64)
    mixed_fp64 = {"value": ws * npts_step * nmd / tmd, "unit": "points/s", "steps": nmd,
                  "ms_per_step": 1e3 * tmd / nmd, "max_rel_err": float(err_md.max()),
                  "frac_rel_err_gt_1e-6": float(np.mean(err_md > 1e-6))}

    # ---- end to end through the host-buffer C-ABI call --------------------
    # the block's grid points, made by the library's own Kernel 1 and held in
    # pinned host memory before the timed region; the same K steps as `value`
    xh = gfc.grid_points((*rect, side, side), stream=stream).reshape(-1).cpu().pin_memory()
    Gh = torch.empty_like(xh).pin_memory()
    for p in props:
        gfc.eval_points_host(p, par64, xh, Gh, stream=stream)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for p in props:
            gfc.eval_points_host(p, par64, xh, Gh, stream=stream)
    e2e_t = max_over_ranks(time.perf_counter() - t0)
    e2e_value = ws * npts_step * args.steps / e2e_t

    line = {
        "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": ws,
        "steps": args.steps, "warmup": max(args.warmup, 1), "ms_per_step": 1e3 * t64 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD,
                   "points_per_step": ws * npts_step, "node_evals_per_step": node_evals_step * ws,
                   "l2": "256 MB buffer written before every step (> 129 MB L2)",
                   "parallelism": f"rows interleaved over {ws} GPU(s) (rank r: rows r mod {ws}), "
                                  "no collective"},
        "node_evals_per_s": node_evals_step * ws * args.steps / t64,
        "clocks": clocks,
        "gpu_launches": 2 * 3 * args.steps,
        "roofline": roofline,
        "mixed": mixed,
        "f32x2": f32x2,
        "mixed_fp64_fallback": mixed_fp64,
        "e2e": {"value": e2e_value, "unit": "points/s", "steps": args.steps,
                "h2d_bytes_per_step": 3 * 16 * side * side,
                "d2h_bytes_per_step": 3 * 16 * side * side},
    }

    if ws == 1 and not args.no_studies:
        line.update(single_gpu_studies(gfc, si, torch, stream, flush, timed, rel_errors, peaks,
                                       par64, props, rect, side, args))
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        v, dt = oracle_points_per_s(args.cpu_baseline_points)
        line["cpu_baseline"] = {"value": v, "unit": "points/s", "cores": cpu_cores(),
                                "kind": "oracle",
                                "sample": f"{args.cpu_baseline_points} seeded grid points x 3 masses "
                                          f"({dt:.1f} s)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def single_gpu_studies(gfc, si, torch, stream, flush, timed, rel_errors, peaks, par64, props,
                       rect, side, args):
    """The other workload configurations, the paper's angular rules, the
    closed-form angle, the clustered radial rule, the Step 3 diagnostics and
    the serving mix (one GPU)."""
    import oracle
    dev = torch.device("cuda", torch.cuda.current_device())
    out = {}
    nst = max(5, min(args.steps, 10))

    # ---- every workload configuration: points/s and error vs the oracle ----
    a, b, c = si.dressed_draws(3, 1)[0]
    dressed = {"kind": "dressed", "a": a, "b": b, "c": c}
    cases = [
        ("paper_example_128x128", {"kind": "cpair", "mk2": 0.5j, "mq2": -0.5j},
         dict(dim=4, mu2=0.0, n_radial=256, n_angular=64), si.grid_rect("paper"), 128, 1024),
        ("bubble_64x64", {"kind": "scalar", "m2": 1.0},
         dict(dim=4, mu2=1.0, n_radial=256, n_angular=64), si.grid_rect("small"), 64, 4096),
        ("dressed_512x512_D3", dressed, dict(dim=3, mu2=1.0, n_radial=1024, n_angular=128),
         si.grid_rect("small"), 512, 256),
        ("dressed_512x512_D4", dressed, dict(dim=4, mu2=1.0, n_radial=1024, n_angular=128),
         si.grid_rect("small"), 512, 256),
    ]
    configs = {}
    for name, prop, par, crect, n, nsample in cases:
        g = gfc.make_grid(*crect, n, n)
        x = oracle.grid_points(*crect, n, n)
        idx = si.sample_indices(11, n * n, min(nsample, n * n))
        ref = oracle.eval_points(prop, par, x[idx])
        rec = {"points": n * n, "nodes": f"{par['n_radial']}x{par['n_angular']}", "D": par["dim"],
               "steps": nst, "oracle_sample": int(idx.size)}
        for prec in ("fp64", "mixed"):
            pp = gfc.make_params(dict(par, precision=prec))
            G = torch.empty((n, n), dtype=torch.complex128, device=dev)
            per, st = {}, []
            t, _ = timed(pp, nst, 2, per, stats=st, props_=[gfc.make_prop(prop)], outs_=[G],
                         grid_=g)
            e = rel_errors([G.cpu().numpy().ravel()[idx]], [ref])
            r = {"points_per_s": n * n * nst / t, "max_rel_err_vs_oracle": float(e.max())}
            if prec == "fp64" and EXEC_MODEL and prop["kind"] == "scalar":
                # (the model is calibrated on ray nodes of the scalar bubble)
                s = st[0]
                ex = executed("fp64", s.pairs_evaluated, s.pairs_full_table,
                              s.node_evals // (2 * ((par["n_angular"] + 1) // 2)), s.points)
                r["fp64_pipe_frac"] = fp64_pipe_seconds(ex, peaks) / (t / nst)
            rec[prec] = r
        configs[name] = rec
    out["configs"] = configs

    # ---- the paper's angular rule: 49-node tanh-sinh in z (Sect. 4) --------
    paper_rule = {}
    for prec in ("fp64", "f32x2", "mixed"):
        parts = gfc.make_params(dim=4, mu2=1.0, n_radial=NR, n_angular=49,
                                angular_rule="tanh-sinh", precision=prec)
        tts, _ = timed(parts, 3, 1)
        paper_rule[prec] = 3 * len(MASSES2) * side * side / tts
    out["paper_angular_rule"] = dict({"rule": "tanh-sinh, 49 nodes in z = cos psi (Sect. 4)",
                                      "n_radial": NR, "unit": "points/s", "steps": 3}, **paper_rule)

    # ---- the psi integral in closed form (no angular quadrature error) -----
    exact_rule = {}
    for nr in (NR, 4 * NR):
        for prec in ("fp64", "f32x2", "mixed"):
            parex = gfc.make_params(dim=4, mu2=1.0, n_radial=nr, n_angular=2,
                                    angular_rule="exact", precision=prec)
            tex, _ = timed(parex, 3, 1)
            exact_rule[f"{prec}_nr{nr}"] = 3 * len(MASSES2) * side * side / tex
    out["exact_angular"] = dict({"rule": "psi integral in closed form (limit of every angular "
                                         "rule); radial Gauss-Legendre n_radial as named",
                                 "unit": "points/s", "steps": 3}, **exact_rule)

    # ---- near-axis accuracy: closed-form angle + clustered radial rule -----
    clustered = {}
    for prec in ("fp64", "f32x2", "mixed"):
        parcl = gfc.make_params(dim=4, mu2=1.0, n_radial=NR, n_angular=2, angular_rule="exact",
                                radial_rule="clustered", precision=prec)
        tcl, _ = timed(parcl, 3, 1)
        clustered[prec] = 3 * len(MASSES2) * side * side / tcl
    out["clustered_radial"] = dict({"rule": "closed-form angle, radial rule sinh-clustered at the "
                                            "pole nearest the ray (n_radial 2048)",
                                    "unit": "points/s", "steps": 3}, **clustered)

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
        for _ in range(3):
            fn()
        b_ev.record(stream)
        torch.cuda.synchronize()
        diag[name] = 3 * xg.numel() / (a_ev.elapsed_time(b_ev) / 1e3)
    out["diagnostics"] = dict({"grid": f"{side}x{side} x (region map) or y (map of B at x = -2 + i)",
                               "propagator": "bubble m = 1", "steps": 3}, **diag)

    # ---- serving: continuous batching --------------------------------------
    if not args.no_serve:
        out["serve"] = serve_study(gfc, n_spec=args.serve_requests, rate=args.serve_rate)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gfc", choices=["gfc", "reference"])
    # ~13 s of the oracle on 16 host cores (3 x 6144 points at ~1.4e3 points/s)
    ap.add_argument("--ref-points", type=int, default=6144)
    # the cpu_baseline leg of the library's arm: one bounded sample (~27 s on
    # 16 host cores at ~1.8e3 points/s)
    ap.add_argument("--cpu-baseline-points", type=int, default=16384)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-studies", action="store_true",
                    help="leave out the other configurations, rule studies and serving")
    ap.add_argument("--no-serve", action="store_true", help="leave out the serving runs")
    ap.add_argument("--side", type=int, default=SIDE,
                    help="grid side per GPU (the benchmark workload is 1024)")
    ap.add_argument("--quick", action="store_true",
                    help="FP64 timing only (profiling runs)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "f32x2", "mixed"],
                    help="with --quick: the precision of the timed workload")
    ap.add_argument("--calib", action="store_true",
                    help="the calibration calls of the executed-work model in --precision "
                         "(run under ncu --metrics with the CALIB_METRICS list)")
    ap.add_argument("--fit-exec-model", nargs="+", metavar="CSV=COUNTERS",
                    help="fit the executed-work model: pairs of an ncu --csv log and the "
                         "--calib output of the same run")
    ap.add_argument("--serve", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-log", default=None,
                    help="with --serve: write one JSON line per request to this file")
    args = ap.parse_args()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        return relaunch(args.gpus, sys.argv[1:]).returncode
    if args.fit_exec_model:
        model, report = fit_exec_model([a.split("=", 1) for a in args.fit_exec_model])
        print(json.dumps({"model": model, "report": report}, indent=1))
        return 0
    if args.impl == "reference":
        return run_reference(args)
    if args.calib:
        return run_calib(args)
    if args.serve:
        return run_serve(args)
    return run_gfc(args)


if __name__ == "__main__":
    sys.exit(main())
