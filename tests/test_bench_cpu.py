"""The benchmark's reference arm (the oracle timed on the host cores) keeps
the one-JSON-line contract without a GPU, and names the same metric and
workload as the library's arm."""
import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--ref-points", "4"], cwd=ROOT, capture_output=True,
                         text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["unit"] == "points/s" and d["higher_is_better"] is True
    assert d["config"]["workload"] == bench.WORKLOAD
    assert d["steps"] == 1 and d["warmup"] == 0 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "points/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def _ncu_rows(launch_id, kernel, metrics):
    head = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream",'
            '"Block Size","Grid Size","Device","CC","Section Name","Metric Name","Metric Unit",'
            '"Metric Value"\n')
    rows = [f'"{launch_id}","1","python","h","{kernel}","1","7","(256, 1, 1)","(1216, 1, 1)",'
            f'"0","10.3","Command line profiler metrics","{k}","{u}","{v}"\n'
            for k, (u, v) in metrics.items()]
    return head, rows


def test_exec_model_fit_recovers_known_coefficients(tmp_path):
    """The executed-work fit recovers per-pair and per-node costs from ncu
    rows that a known model generated, for the one-kernel calls of FP64 and
    the three-kernel calls of mixed precision (launches grouped by call)."""
    import numpy as np
    rng = np.random.default_rng(3)
    truth = {"fp64": (7.0, 9.0, 60.0, 0.0), "bulk32p": (3.0, 4.0, 200.0, 0.0),
             "nodes_df": (60.0, 70.0, 900.0, 5000.0), "list64": (7.0, 9.0, 80.0, 3000.0)}
    names = {"fp64": "void gfc::eval_kernel<double, 128, 1, 0, 0>(gfc::KParams, ...)",
             "list64": "void gfc::eval_kernel<double, 128, 1, 0, 0>(gfc::KParams, ...)",
             "bulk32p": "void gfc::eval_bulk_partial_kernel<float, 128, 1, 0>(gfc::KParams, ...)",
             "nodes_df": "void gfc::eval_kernel<gfc::df, 0, 1, 0, 1>(gfc::KParams, ...)"}

    def counts(kc, units):
        return float(np.dot(truth[kc], units))

    for prec, kernels in (("fp64", ["fp64"]), ("mixed", ["bulk32p", "nodes_df", "list64"])):
        recs, lines, lid, head = [], [], 0, None
        for call in range(6):
            u = {kc: rng.integers(1, 10**6, 4) for kc in kernels}
            rec = {"case": f"c{call}", "precision": prec}
            if prec == "fp64":
                p, pf, n, _ = u["fp64"]
                rec.update(pairs_evaluated=int(p + pf), pairs_full_table=int(pf),
                           node_evals=int(n) * bench.NA, points=int(u["fp64"][3]))
            else:
                rec.update(pairs_fallback=int(u["nodes_df"][0] + u["nodes_df"][1]),
                           pairs_full_table_fallback=int(u["nodes_df"][1]),
                           node_evals_fallback=int(u["nodes_df"][2]) * bench.NA,
                           pairs_list64=int(u["list64"][0] + u["list64"][1]),
                           pairs_full_table_list64=int(u["list64"][1]),
                           node_evals_list64=int(u["list64"][2]) * bench.NA,
                           points=int(u["bulk32p"][3]), points_partial=int(u["nodes_df"][3]),
                           points_fp64=int(u["list64"][3]))
                rec.update(pairs_evaluated=int(sum(v[0] + v[1] for v in u.values())),
                           pairs_full_table=int(sum(v[1] for v in u.values())),
                           node_evals=int(sum(v[2] for v in u.values())) * bench.NA)
            recs.append(rec)
            for kc in kernels:
                c = counts(kc, u[kc])
                head, rows = _ncu_rows(lid, names[kc], {
                    "sm__inst_executed_pipe_fp64.sum": ("inst", c / 32.0),
                    "sm__sass_thread_inst_executed_op_dfma_pred_on.sum": ("inst", c),
                    "smsp__inst_executed.sum": ("inst", 2 * c),
                    "gpu__time_duration.sum": ("msecond", 1.5)})
                lines += rows
                lid += 1
        (tmp_path / f"{prec}.csv").write_text("==PROF== noise\n" + head + "".join(lines))
        (tmp_path / f"{prec}.json").write_text("\n".join(json.dumps(r) for r in recs) + "\n")
    model, report = bench.fit_exec_model(
        [(str(tmp_path / f"{p}.csv"), str(tmp_path / f"{p}.json")) for p in ("fp64", "mixed")])
    for kc, coef in truth.items():
        assert np.allclose(model[kc]["fp64"], coef, rtol=1e-6), (kc, model[kc])
        assert np.allclose(model[kc]["dfma"], coef, rtol=1e-6)
        assert np.allclose(model[kc]["inst"], [2 * c for c in coef], rtol=1e-6)
        assert report[kc]["fp64"] < 1e-9
        assert all(abs(l["ms"] - 1.5) < 1e-12 for l in report[kc]["launches"])
