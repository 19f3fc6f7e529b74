#!/usr/bin/env python
"""Benchmark of the batched Dufort-Frankel wall update on one GB300 (or N).

Workload: 4096 ragged 1D walls (1-3 layers, 50-400 nodes, 0.05-0.4 m), seeded
synthetic materials and forcing, dt = 600 s, one year (52560 steps) per run.
One benchmark step = one hygro_run of the whole year on all walls with the
persistent FP32 kernel (state carried over from step to step), inputs already
resident in HBM; the L2 cache is flushed (512 MB write) between timed runs.
Prints one JSON line (rank 0). ``--impl reference`` times the FP64 CPU oracle
instead, on a bounded sample of the same workload. The line also carries the
FP64 GPU comparators, the whole-building workload (64 rooms x 6 walls) and the
2D thermal-bridge sections (64 x 512 x 512, 10000 steps) and the gradient workload (adjoint of 1024
walls over 30 days) under other_workloads.

Metric: DF cell-updates/s (one node advanced one step for both T and Pv).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "DF cell-updates/s, batched FP32 vs plain FP64 on GB300 at ≤1e-4 rel L∞; % roofline"
UNIT = "cell-updates/s"
# Algorithmic FP32 operations per cell-update of the DF increment form, each add, multiply or fused
# multiply-add counted once (they all issue to the FMA pipe); reciprocals run on the MUFU pipe apart.
# The neighbour sums are counted in their shortest form, sum_f F u_nb - S u^{n-1} (3 operations for two
# faces, S being needed for the denominator anyway):
# The latent cross flux X = sum_f F (Pv_nb - Pv_bar) is the node's vapour balance A dPv - g (1 operation).
#   general wall:     coefficients 5 (kM, kTT, A, B, chi A), faces 2, Pv 8 (S, num 3, denominator,
#                     dPv, X, update), T 9 (ST, num 3, latent, cTM, denominator, dT, update)
#                     = 24 (+ 2 reciprocals)
#   simple-heat wall: (kTT, cTT independent of Pv, cTM = 0: constant thermal faces and T denominators)
#                     coefficients 2, face 1, Pv 8, T 6 (num 3, latent, dT, update) = 17 (+ 1 reciprocal)
OPS_GENERAL = 24
OPS_SIMPLE_HEAT = 17
# adjoint, per differentiated cell-update: forward step 24, its recompute 24, reverse step 76 (the
# recomputed forward quantities 25 with the neighbour differences the reverse needs, the transposed
# step 36, the face chain 15)
OPS_ADJOINT = 124
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0
KERNEL_SOURCES = ["paper_1703_10119_gb300/csrc/df1d_persistent.cuh", "paper_1703_10119_gb300/csrc/df1d_common.cuh",
                  "paper_1703_10119_gb300/csrc/hygro_internal.cuh"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "df1d_persistent_f32_traffic.json")
# 2D sections: compulsory DRAM bytes of one cell-update when every step is a pass over memory (read the
# (T, Pv) pairs of levels n and n-1, write the pair of level n+1, 4-byte reals)
BYTES_PER_CELL_UPDATE_2D = 24
STEPS_PER_LAUNCH_2D = 4
# 2D sections, algorithmic FP32 operations per cell-update of the five-point increment form for the
# workload's materials (kTT, cTT independent of Pv, no cTM: constant thermal faces and T denominators),
# each face counted once (shared by its two nodes): coefficients 2 (kM half-value, A), faces 2, Pv 12
# (S 3, num 5, denominator, dPv, X, update), T 8 (num 5, latent, dT, update) = 24 (+ 1 reciprocal)
OPS_2D = 24
KERNEL_SOURCES_2D = ["paper_1703_10119_gb300/csrc/df2d.cuh", "paper_1703_10119_gb300/csrc/df1d_common.cuh"]
TRAFFIC_FILE_2D = os.path.join(ROOT, "profiles", "df2d_f32_traffic.json")
FALLBACK_HBM_GBS = 6800.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--walls", type=int, default=4096)
    p.add_argument("--year-steps", type=int, default=52560)
    p.add_argument("--cpu-walls", type=int, default=256, help="walls of the CPU-baseline sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--no-2d", action="store_true")
    p.add_argument("--no-adjoint", action="store_true")
    p.add_argument("--only-2d", action="store_true", help="run only the 2D sections (profiling cases)")
    p.add_argument("--sections", type=int, default=64, help="2D sections of 512 x 512")
    p.add_argument("--section-steps", type=int, default=10000)
    p.add_argument("--only-adjoint", action="store_true", help="run only the gradient workload (profiling cases)")
    p.add_argument("--adjoint-steps", type=int, default=43200, help="steps of the gradient workload")
    return p.parse_args()


def kernel_source_hash(sources=None) -> str:
    h = hashlib.sha256()
    for f in sources or KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(path=None, sources=None):
    """DRAM bytes per launch from the committed ncu summary, if it matches the current kernel source and
    was taken on a launch like the timed ones (starting at step 0)."""
    try:
        with open(path or TRAFFIC_FILE) as fh:
            t = json.load(fh)
        if t.get("kernel_source_sha") == kernel_source_hash(sources) and t.get("launch_start_step", 0) == 0:
            return t.get("dram_bytes_per_launch")
    except (OSError, ValueError):
        pass
    return None


def measure_peaks(H, device: int, stream) -> dict:
    """Arithmetic peaks of this GPU by microbenchmark (hygro_peak_probe), in T lane-operations/s, with
    the SM clock sampled while they run."""
    out = {}
    with ClockSampler(device) as cs:
        for name, kind, ms in (("ffma", H.HYGRO_PEAK_FFMA, 200.0), ("ffma2", H.HYGRO_PEAK_FFMA2, 200.0),
                               ("rcp", H.HYGRO_PEAK_RCP, 100.0), ("dfma", H.HYGRO_PEAK_DFMA, 100.0)):
            ops, t = H.hygro_peak_probe(kind, device, stream, ms)
            out[name + "_tops"] = ops / 1e12
            out[name + "_ms"] = t
    out["clocks"] = cs.summary()
    # the FP32 roof: the faster of the scalar and the packed fused multiply-add, one operation per lane
    # and FMA (the unit of the algorithmic counts)
    out["fp32_tops"] = max(out["ffma_tops"], out["ffma2_tops"])
    out["source"] = ("measured in this run: 8 independent FMA (scalar and f32x2), rcp.approx or FP64 FMA "
                     "chains per thread, SMs x 4 blocks x 256 threads, CUDA events")
    return out


def fp32_peak(peaks, sms: int):
    """The FP32 roof in T operations/s: measured in this run when the probes ran, else nominal."""
    if peaks and peaks.get("fp32_tops"):
        return peaks["fp32_tops"], "measured (hygro_peak_probe, this run)"
    return sms * FP32_LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e12, f"nominal: {sms} SMs x {FP32_LANES_PER_SM} lanes x {SM_MAX_MHZ:.0f} MHz"


def relinf(x, ref) -> float:
    ref = np.asarray(ref, np.float64)
    return float(np.max(np.abs(np.asarray(x, np.float64) - ref)) / np.max(np.abs(ref)))


def rel_dev_linf(x, ref, init) -> float:
    """Error relative to the reference's largest departure from the initial state (the stricter view of
    the relative L-infinity error)."""
    ref = np.asarray(ref, np.float64)
    return float(np.max(np.abs(np.asarray(x, np.float64) - ref)) / np.max(np.abs(ref - init)))


def measured_hbm_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return FALLBACK_HBM_GBS


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = [r.split(",") for r in (self.out or "").strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist

        import torch

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend, init_method="env://")
        pg = dist
    return world, rank, local, pg


def reduce_max(pg, x: float) -> float:
    if pg is None:
        return x
    import torch

    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(pg, x: float) -> float:
    if pg is None:
        return x
    import torch

    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


def algorithmic_ops_per_step(wl, reciprocals: bool = False) -> float:
    """FP32 FMA-pipe operations of one DF step over all walls (see OPS_GENERAL / OPS_SIMPLE_HEAT); with
    reciprocals, the MUFU reciprocals instead (the Pv denominator, and the T one unless the wall's heat
    coefficients are constant, when it is set up once)."""
    off = wl.layer_offset()
    ops = 0.0
    for w in range(wl.n_walls):
        lp = wl.layer_par[off[w]:off[w + 1]]
        simple = bool(np.all(lp[:, 5] == 0) and np.all(lp[:, 7] == 0) and np.all(lp[:, 8] == 0))
        if reciprocals:
            ops += wl.n_nodes[w] * (1 if simple else 2)
        else:
            ops += wl.n_nodes[w] * (OPS_SIMPLE_HEAT if simple else OPS_GENERAL)
    return ops


def cpu_sample(wl, n_walls: int):
    step = max(1, wl.n_walls // n_walls)
    pick = np.arange(0, wl.n_walls, step)[:n_walls]
    return pick, wl.subset(pick)


def run_oracle_sample(sub, n_steps: int):
    import oracle

    o = oracle.Oracle(sub)
    t = time.perf_counter()
    o.run(n_steps)
    el = time.perf_counter() - t
    return o, el


def batch_config(wl, n_steps: int) -> dict:
    """The benchmark workload as both arms name it."""
    return {"workload": (f"{wl.n_walls} ragged 1D walls per GPU (1-3 layers, 50-400 nodes), "
                         f"dt=600 s x {n_steps} steps (one year)"),
            "nodes_per_gpu": int(wl.total_nodes), "cell_updates_per_gpu_per_step": int(wl.total_nodes) * int(n_steps)}


def bench_reference(args):
    from paper_1703_10119_gb300 import workloads as wk
    import oracle

    wl = wk.wall_batch(n_walls=args.walls, n_steps=args.year_steps)
    # the same sample as the cpu_baseline leg of the other arm (every 16th wall of 4096 by default): large
    # enough that the host threads stay balanced
    pick, sub = cpu_sample(wl, args.cpu_walls)
    units = sub.total_nodes * args.year_steps
    for _ in range(args.warmup):
        run_oracle_sample(sub, args.year_steps // 8)
    times = []
    for _ in range(args.steps):
        _, el = run_oracle_sample(sub, args.year_steps)
        times.append(el)
    ms = 1e3 * float(np.mean(times))
    value = units / (ms / 1e3)
    cores = oracle.default_threads()
    sample = (f"{len(pick)} of {wl.n_walls} walls (every {wl.n_walls // len(pick)}th), all {args.year_steps} "
              f"steps, FP64 oracle, OpenMP over walls")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {**batch_config(wl, args.year_steps), "path": "FP64 oracle on the host cores",
                       "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def bench_sections(args, H, wk, stream, local, rank, peaks=None):
    """The 2D thermal-bridge workload: throughput, its HBM roofline and parity on sampled sections."""
    import torch

    sec = wk.sections_2d(seed=4 + rank, n_grids=args.sections, n_steps=args.section_steps)
    h = H.Hygro2D(sec, precision="fp32", device=local, stream=stream.cuda_stream)
    with torch.cuda.stream(stream):
        h.run(100)
    torch.cuda.synchronize()
    # the library's autotuner picks the temporal blocking depth on a short prefix of this workload
    k, tune_ms = h.autotune(16)
    graph_launches = h.option(H.HYGRO2D_OPT_GRAPH_LAUNCHES)

    def timed_run():
        with torch.cuda.stream(stream):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h.run(sec.n_steps)
            e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    ms = timed_run()   # whole intervals of launches replayed from CUDA graphs
    h.set_option(H.HYGRO2D_OPT_GRAPH_LAUNCHES, 0)
    ms_plain = timed_run()   # the same run from one launch at a time
    h.sync()
    h.close()
    units = sec.total_nodes * sec.n_steps
    value = units / (ms / 1e3)
    workload = f"{sec.n_grids} sections {sec.nx}x{sec.ny}, {sec.n_steps} steps, FP32, {k} fused steps per launch"
    launches = -(-sec.n_steps // k)
    ms_launch = ms / launches
    # two roofs: HBM at the compulsory traffic of k fused steps per pass (24 / k B per cell-update) and
    # the FP32 ALU at OPS_2D operations per cell-update; the lower one binds
    bytes_cu = BYTES_PER_CELL_UPDATE_2D / k
    hbm_peak = measured_hbm_gbs()
    hbm_achieved = bytes_cu * value / 1e9
    hbm_roof = hbm_peak * 1e9 / bytes_cu
    alu_peak = peaks["fp32_tops"] if peaks else None
    alu_achieved = OPS_2D * value / 1e12
    alu_roof = alu_peak * 1e12 / OPS_2D if alu_peak else None
    traffic = measured_traffic(TRAFFIC_FILE_2D, KERNEL_SOURCES_2D)
    binding = "hbm" if alu_roof is None or hbm_roof <= alu_roof else "alu"
    if binding == "hbm":
        roof = {"bound": "hbm", "achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": hbm_achieved / hbm_peak}
    else:
        roof = {"bound": "alu", "achieved": alu_achieved, "peak": alu_peak, "unit": "Top/s",
                "frac": alu_achieved / alu_peak}
    roof.update({
        "traffic": traffic,
        "hbm_frac": hbm_achieved / hbm_peak, "hbm_bytes_per_cell_update": bytes_cu,
        "alu_frac": alu_achieved / alu_peak if alu_peak else None, "alu_ops_per_cell_update": OPS_2D,
        "note": (f"{k} fused steps per launch: {BYTES_PER_CELL_UPDATE_2D}/{k} B of compulsory HBM traffic per "
                 "cell-update (read T, Pv at n and n-1, write T, Pv at n+1 once per launch, FP32) against the "
                 f"measured copy bandwidth; {OPS_2D} algorithmic FP32 operations per cell-update against the "
                 "measured FP32 FMA peak; the roof with the lower cell-update rate binds; kernel df2d_kernel<float>")})
    out = {"value": value, "unit": UNIT, "workload": workload, "ms_per_run": ms, "launches": launches,
           "steps_per_launch": k, "roofline": roof,
           "autotune": {"chosen_steps_per_launch": k, "ms_per_step_by_depth": [float(x) for x in tune_ms],
                        "probe": "16 steps from the state after 100 steps, each depth from the same state"},
           "graph": {"launches_per_graph": graph_launches, "ms_per_run_graph": ms, "ms_per_run_plain_launches": ms_plain,
                     "value_plain_launches": units / (ms_plain / 1e3)}}
    if rank == 0 and not args.no_cpu_baseline:
        import oracle

        n = 200
        pick = [0, sec.n_grids - 1]
        sub = sec.subset(pick)
        g2 = H.Hygro2D(sub, precision="fp32", device=local, stream=stream.cuda_stream)
        g2.run(n)
        T, P = g2.fields(0)
        g2.close()
        o = oracle.Oracle2D(sub)
        o.run(n)
        Ti = np.asarray(sub.T_init, np.float64)[:, None, None]
        Pi = np.asarray(sub.P_init, np.float64)[:, None, None]
        out["parity_vs_oracle"] = {"sections_checked": len(pick), "steps": n,
                                   "rel_linf_T": relinf(T, o.T_cur), "rel_linf_P": relinf(P, o.P_cur),
                                   "rel_dev_linf_T": rel_dev_linf(T, o.T_cur, Ti),
                                   "rel_dev_linf_P": rel_dev_linf(P, o.P_cur, Pi)}
    return out


def bench_table1(args, H, wk, stream, local, rank):
    """256 walls of the Table-1 material (Sec. 4: 10 cm, N = 101, dt = 3.6 s), 2 h of it (2000 steps) on
    the plain kernel in FP32 and FP64; parity of two walls' surface samples and final fields against the
    oracle over the same 2 h."""
    import torch

    wl = wk.table1_walls(seed=6 + rank, n_walls=256, hours=2.0)
    n = wl.n_steps
    out = {"workload": f"{wl.n_walls} walls of the Table-1 material, N=101, dt=3.6 s x {n} steps, plain kernel",
           "unit": UNIT}
    res = {}
    for prec in ("fp32", "fp64"):
        h = H.Hygro(wl, precision=prec, kernel="plain", device=local, stream=stream.cuda_stream)
        s0 = h.get_state()
        with torch.cuda.stream(stream):
            h.run(200)
        torch.cuda.synchronize()
        h.set_state(s0)
        with torch.cuda.stream(stream):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h.run(n)
            e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        T, P = h.fields(0)
        h.close()
        res[prec] = (T, P)
        out[f"value_{prec}"] = wl.total_nodes * n / (ms / 1e3)
        out[f"ms_per_run_{prec}"] = ms
    out["value"] = out["value_fp32"]
    out["note"] = ("one launch per step (launch-bound at 25 856 nodes per launch); each node evaluates the "
                   "Table-1 laws (isotherm, its derivative, permeabilities, saturation pressure) for itself and "
                   "its two neighbours")
    if rank == 0 and not args.no_cpu_baseline:
        import oracle

        pick = [0, wl.n_walls - 1]
        sub = wl.subset(pick)
        o = oracle.Oracle(sub)
        o.run(n)
        off = np.concatenate([[0], np.cumsum(wl.n_nodes)])
        par = {}
        for prec, (T, P) in res.items():
            Tg = np.concatenate([T[off[w]:off[w + 1]] for w in pick])
            Pg = np.concatenate([P[off[w]:off[w + 1]] for w in pick])
            par[prec] = {"rel_linf_T": relinf(Tg, o.T_cur), "rel_linf_P": relinf(Pg, o.P_cur)}
        out["parity_vs_oracle"] = par
    return out


def bench_cpu_schemes(wk):
    """The paper's CPU time comparison (Table tab:CPU_time) on this host's cores: DF (the oracle), Euler
    implicit with the fixed-point sub-iterations of Alg. 1 (tolerance 0.01 dt*, dt* = dt / 1 h, Euclidean
    norm) and Euler explicit within its stability bound, on the one-zone case (Sec. 5.2, 8 h of the 80 h) and
    one Table-1 wall (Sec. 4, 2 h). The paper (Matlab, Intel i7): one zone DF 8.5 s vs implicit 95 s (9 %);
    Table-1 wall DF 150 s, explicit 164 s, implicit 530 s (28 %, 31 %)."""
    import oracle

    out = {}
    for name, wl, n in (("one_zone_8h", wk.one_zone(), 8000), ("table1_wall_2h", wk.table1_walls(n_walls=1, hours=2.0), 2000)):
        eta = 0.01 * wl.dt / 3600.0
        rec = {}
        for scheme in ("df", "implicit", "explicit"):
            o = oracle.Oracle(wl)
            t = time.perf_counter()
            if scheme == "df":
                o.run(n)
            elif scheme == "implicit":
                rec["implicit_subiterations_per_step"] = o.run_implicit(n, eta=eta, norm="l2") / n
            else:
                rec["explicit_substeps_per_step"] = o.run_explicit(n, 1.0) / n
            rec[f"{scheme}_seconds"] = time.perf_counter() - t
        rec["df_over_implicit"] = rec["df_seconds"] / rec["implicit_seconds"]
        rec["explicit_over_implicit"] = rec["explicit_seconds"] / rec["implicit_seconds"]
        rec["steps"] = n
        out[name] = rec
    out["cores"] = oracle.default_threads()
    out["paper"] = {"one_zone_df_over_implicit": 8.5 / 95.0, "table1_df_over_implicit": 150.0 / 530.0,
                    "table1_explicit_over_implicit": 164.0 / 530.0, "hardware": "Matlab on an Intel i7 (paper)"}
    return out


def bench_adjoint(args, H, wk, stream, local, rank, peaks=None):
    """Gradient workload: misfit loss and its gradient over 30 days of 1024 two-layer walls (FP32 adjoint,
    sqrt(T) checkpoints), observations resident on the device; parity on sampled walls vs the oracle."""
    import torch

    wl, s = wk.gradient_walls(seed=5 + rank, n_steps=args.adjoint_steps)
    dev = torch.device("cuda", local)
    obs = torch.from_numpy(s.obs).to(dev)
    grad = torch.zeros((len(wl.layer_par), 9), dtype=torch.float64, device=dev)
    h = H.Hygro(wl, precision="fp32", device=local, stream=stream.cuda_stream)
    H.hygro_loss_grad(h.ctx, min(600, wl.n_steps), s.sample_every, obs, s.wT, s.wP, 0, grad)   # warm-up (short run)
    torch.cuda.synchronize()
    t = time.perf_counter()
    with torch.cuda.stream(stream):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        L = H.hygro_loss_grad(h.ctx, wl.n_steps, s.sample_every, obs, s.wT, s.wP, 0, grad)
        e1.record(stream)
    torch.cuda.synchronize()
    el = time.perf_counter() - t
    ms = e0.elapsed_time(e1)
    g = grad.cpu().numpy()
    # the same gradient with every level kept in HBM (one checkpoint stretch: no recompute), when the
    # device has room for it (slots per lane x 32 lanes x 2 fields x (steps + 2) levels per wall)
    all_levels = None
    need = wl.n_walls * 7 * 32 * 2 * (wl.n_steps + 2) * 4   # 7 slots per lane at N = 200
    free, _ = torch.cuda.mem_get_info(dev)
    if need < 0.8 * free:
        grad2 = torch.zeros_like(grad)
        with torch.cuda.stream(stream):
            e2 = torch.cuda.Event(enable_timing=True)
            e3 = torch.cuda.Event(enable_timing=True)
            e2.record(stream)
            L2 = H.hygro_loss_grad(h.ctx, wl.n_steps, s.sample_every, obs, s.wT, s.wP, wl.n_steps, grad2)
            e3.record(stream)
        torch.cuda.synchronize()
        ms2 = e2.elapsed_time(e3)
        g2 = grad2.cpu().numpy()
        big = np.max(np.abs(g * wl.layer_par))
        all_levels = {"ms_per_gradient": ms2, "value": wl.total_nodes * wl.n_steps / (ms2 / 1e3),
                      "loss_equal": L2 == L, "grad_scaled_max_diff": float(np.max(np.abs((g2 - g) * wl.layer_par)) / big),
                      "note": "checkpoint_every = n_steps: the first run stores every level (about "
                              f"{need / 1e9:.0f} GB) and the reverse sweep reads them; no recompute"}
        del grad2
    h.close()
    C = int(np.ceil(np.sqrt(wl.n_steps)))
    value = wl.total_nodes * wl.n_steps / (ms / 1e3)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak, peak_source = fp32_peak(peaks, sms)
    achieved = OPS_ADJOINT * value / 1e12
    out = {"value": value, "unit": UNIT + " (forward steps differentiated)",
           "workload": f"{wl.n_walls} two-layer walls N=200, dt=60 s x {wl.n_steps} steps, sensors every "
                       f"{s.sample_every} steps, FP32 adjoint, checkpoints every {C} steps",
           "ms_per_gradient": ms, "seconds_call": el, "loss": L, "all_levels_in_hbm": all_levels,
           "note": "forward + recompute + reverse sweep in one launch; cell-updates of the forward run per second; "
                   "the time is the whole hygro_loss_grad call (buffer allocation and copies included)",
           "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Top/s", "frac": achieved / peak,
                        "traffic": None, "peak_source": peak_source,
                        "note": f"FP32 FMA-pipe roof; {OPS_ADJOINT} algorithmic FP32 ops per differentiated "
                                "cell-update (forward 24, recompute 24, reverse step 76) plus 6 reciprocals; "
                                "kernel adjoint_reg_kernel<float>"}}
    if rank == 0 and not args.no_cpu_baseline:
        import oracle

        pick = [0, wl.n_walls - 1]
        sub = wl.subset(pick)
        t = time.perf_counter()
        L0, g0 = oracle.loss_and_gradient(sub, wl.n_steps, s.obs[:, pick].astype(np.float64), s.sample_every,
                                          s.wT, s.wP)
        el0 = time.perf_counter() - t
        h2 = H.Hygro(sub, precision="fp32", device=local, stream=stream.cuda_stream)
        L2, _ = h2.loss_grad(wl.n_steps, s.sample_every, s.obs[:, pick], s.wT, s.wP)
        h2.close()
        rows = np.concatenate([np.arange(2 * w, 2 * w + 2) for w in pick])
        big = np.max(np.abs(g0 * sub.layer_par))
        # per component: the relative error of each parameter's gradient, over the active parameters
        # (kM0, a, cM0, b, kTT0, cTT0: the workload's aT = bT = chi = 0 leave the other three at zero)
        active = [0, 1, 2, 3, 4, 6]
        comp = np.abs(g[rows][:, active] - g0[:, active]) / np.maximum(np.abs(g0[:, active]), 1e-300)
        out["parity_vs_oracle"] = {"walls_checked": len(pick), "loss_rel": abs(L2 - L0) / abs(L0),
                                   "grad_scaled_max_rel": float(np.max(np.abs((g[rows] - g0) * sub.layer_par)) / big),
                                   "grad_component_rel_max": float(np.max(comp)),
                                   "grad_component_rel_median": float(np.median(comp)),
                                   "oracle_seconds": el0}
    return out


def bench_ours(args):
    import torch

    world, rank, local, pg = dist_setup(args)
    assert torch.cuda.is_available(), "bench.py needs a CUDA device (no CPU fallback)"
    torch.cuda.set_device(local)
    from paper_1703_10119_gb300 import hygro as H
    from paper_1703_10119_gb300 import workloads as wk

    H.lib(build_if_missing=True)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    peaks = measure_peaks(H, local, stream.cuda_stream)
    if args.only_2d:
        out = bench_sections(args, H, wk, stream, local, rank, peaks)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "unit": UNIT, "only": "2d sections", **out}))
        return
    if args.only_adjoint:
        out = bench_adjoint(args, H, wk, stream, local, rank, peaks)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "unit": UNIT, "only": "gradient workload", **out}))
        return
    wl = wk.wall_batch(seed=2 + rank, n_walls=args.walls, n_steps=args.year_steps)
    units_per_run = wl.total_nodes * args.year_steps
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    g = H.Hygro(wl, precision="fp32", kernel="persistent", device=local, stream=stream.cuda_stream)
    # every run (parity, warm-up, timed) is the same year from the initial state: a run continuing the
    # previous one would start past the end of the hourly noise tables, which are then held constant
    s0 = g.get_state()
    # the library's autotuner refits the wall schedule's step-time model on a probe of this workload and
    # keeps the faster schedule (the state is restored afterwards)
    ta, tb, tms = g.autotune(2000)
    autotune = {"probe_steps": 2000, "model_a_ns": [float(x) for x in ta], "model_b_ns": [float(x) for x in tb],
                "probe_ms_previous_schedule": float(tms[0]), "probe_ms_refitted_schedule": float(tms[1]),
                "kept": "refitted" if tms[1] <= tms[0] else "previous"}

    # parity of one full run from the initial state against the oracle on a sample of walls
    parity = None
    cpu_baseline = None
    pick, sub = cpu_sample(wl, args.cpu_walls)
    # the parity run also takes daily surface samples, so that every output of the run is compared
    se = 144 if args.year_steps >= 144 else 1
    smp = np.zeros((args.year_steps // se, wl.n_walls, 2, 2), np.float32)
    with torch.cuda.stream(stream):
        g.run(args.year_steps, se, smp)
    g.sync()
    T, P = g.fields(0)
    flux, cum = g.fluxes()
    if rank == 0 and not args.no_cpu_baseline:
        import oracle

        o = oracle.Oracle(sub)
        t0 = time.perf_counter()
        ro = o.run(args.year_steps, se)
        times = [time.perf_counter() - t0]
        # the baseline is the best of three runs of the same sample (the first one's output is the parity
        # reference)
        for _ in range(2):
            o2 = oracle.Oracle(sub)
            t0 = time.perf_counter()
            o2.run(args.year_steps, se)
            times.append(time.perf_counter() - t0)
            del o2
        el = min(times)
        off = np.concatenate([[0], np.cumsum(wl.n_nodes)])
        Tg = np.concatenate([T[off[w]:off[w + 1]] for w in pick])
        Pg = np.concatenate([P[off[w]:off[w + 1]] for w in pick])
        Ti = np.repeat(np.asarray(sub.T_init, np.float64), sub.n_nodes)
        Pi = np.repeat(np.asarray(sub.P_init, np.float64), sub.n_nodes)
        sg, so = smp[:, pick], ro["samples"]
        sTi = np.asarray(sub.T_init, np.float64)[None, :, None]
        sPi = np.asarray(sub.P_init, np.float64)[None, :, None]
        # every output of the FP32 run against the FP64 oracle: the final fields, the daily surface samples,
        # the last step's surface fluxes and their running sums (relative to the largest of the batch);
        # rel_dev: relative to the largest departure from the initial state instead
        parity = {"walls_checked": int(len(pick)), "samples": f"surface T, Pv every {se} steps",
                  "rel_linf_T": relinf(Tg, o.T_cur), "rel_linf_P": relinf(Pg, o.P_cur),
                  "rel_dev_linf_T": rel_dev_linf(Tg, o.T_cur, Ti), "rel_dev_linf_P": rel_dev_linf(Pg, o.P_cur, Pi),
                  "samples_rel_linf_T": relinf(sg[..., 0], so[..., 0]),
                  "samples_rel_linf_P": relinf(sg[..., 1], so[..., 1]),
                  "samples_rel_dev_linf_T": rel_dev_linf(sg[..., 0], so[..., 0], sTi),
                  "samples_rel_dev_linf_P": rel_dev_linf(sg[..., 1], so[..., 1], sPi),
                  "flux_heat_rel_linf": relinf(flux[pick][..., 0], ro["flux"][..., 0]),
                  "flux_moisture_rel_linf": relinf(flux[pick][..., 1], ro["flux"][..., 1]),
                  "cumulative_heat_rel_linf": relinf(cum[pick][..., 0], o.cumul[..., 0]),
                  "cumulative_moisture_rel_linf": relinf(cum[pick][..., 1], o.cumul[..., 1])}
        cpu_baseline = {"value": sub.total_nodes * args.year_steps / el, "unit": UNIT,
                        "cores": oracle.default_threads(), "kind": "oracle",
                        "sample": f"{len(pick)} of {wl.n_walls} walls (every {wl.n_walls // len(pick)}th), "
                                  f"all {args.year_steps} steps, best of 3 runs: {el:.1f} s "
                                  f"({', '.join(f'{x:.1f}' for x in times)} s)"}

    for _ in range(max(0, args.warmup - 1)):
        g.set_state(s0)
        with torch.cuda.stream(stream):
            g.run(args.year_steps)
    torch.cuda.synchronize()
    if pg is not None:
        pg.barrier()

    times = []
    with ClockSampler(local) as cs:
        torch.cuda.synchronize()
        if pg is not None:
            pg.barrier()
        t_wall = time.perf_counter()
        for _ in range(args.steps):
            g.set_state(s0)   # host call, outside the events; it waits for the context's stream first
            with torch.cuda.stream(stream):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                g.run(args.year_steps)
                e1.record(stream)
            times.append((e0, e1))
        torch.cuda.synchronize()
        if pg is not None:
            pg.barrier()
        t_wall = time.perf_counter() - t_wall
    g.sync()
    ms_list = [a.elapsed_time(b) for a, b in times]
    ms = float(np.mean(ms_list))
    ms_max = reduce_max(pg, ms)
    units_total = reduce_sum(pg, float(units_per_run))
    value = units_total / (ms_max / 1e3)

    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak, peak_source = fp32_peak(peaks, sms)
    ops_per_step = algorithmic_ops_per_step(wl)
    achieved = ops_per_step * args.year_steps / (ms / 1e3) / 1e12
    traffic = measured_traffic()
    nominal = sms * FP32_LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e12
    # the second ALU roof: MUFU reciprocals against the measured rcp rate; the roof with the lower
    # cell-update rate binds
    rcp_per_step = algorithmic_ops_per_step(wl, reciprocals=True)
    mufu = None
    if peaks and peaks.get("rcp_tops"):
        mufu_achieved = rcp_per_step * args.year_steps / (ms / 1e3) / 1e12
        mufu = {"achieved": mufu_achieved, "peak": peaks["rcp_tops"], "unit": "T rcp/s",
                "frac": mufu_achieved / peaks["rcp_tops"],
                "rcp_per_cell_update": rcp_per_step / wl.total_nodes}
    binding = "fma" if mufu is None or achieved / peak >= mufu["frac"] else "mufu"
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Top/s", "frac": achieved / peak,
                "traffic": traffic, "peak_source": peak_source, "frac_of_nominal": achieved / nominal,
                "mufu": mufu, "binding_alu_roof": binding,
                "target_frac": 0.6,
                "note": (f"FP32 FMA roof (measured FMA microbenchmark; nominal {sms} SMs x {FP32_LANES_PER_SM} "
                         f"lanes x {SM_MAX_MHZ:.0f} MHz = {nominal:.2f} T); "
                         f"{ops_per_step / wl.total_nodes:.1f} algorithmic FP32 ops per cell-update "
                         f"({OPS_SIMPLE_HEAT} on simple-heat walls, {OPS_GENERAL} otherwise) plus reciprocals on "
                         "the MUFU pipe; kernel df1d_persistent_kernel<float>, one launch per run")}

    # plain FP64 comparator (one thread per node, one launch per step)
    comparators = {}
    if not args.no_fp64:
        for kernel in ("plain", "persistent"):
            h = H.Hygro(wl, precision="fp64", kernel=kernel, device=local, stream=stream.cuda_stream)
            n = args.year_steps if kernel == "persistent" else args.year_steps // 4
            s64 = h.get_state()   # the timed run starts from the initial state, like the FP32 runs
            with torch.cuda.stream(stream):
                h.run(min(n, 2000))
            torch.cuda.synchronize()
            h.set_state(s64)
            with torch.cuda.stream(stream):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                h.run(n)
                e1.record(stream)
            torch.cuda.synchronize()
            el = e0.elapsed_time(e1) / 1e3
            comparators[f"fp64_{kernel}"] = {"value": wl.total_nodes * n / el, "unit": UNIT,
                                             "steps_timed": n, "seconds": el}
            h.close()
        comparators["fp32_persistent_over_fp64_plain"] = value / world / comparators["fp64_plain"]["value"]

    # whole-building workload (64 rooms x 6 walls, FP64 room nodes, 30 days): walls + rooms per run
    other = {}
    if not args.no_fp64:
        wl3 = wk.building(seed=3 + rank)
        h = H.Hygro(wl3, precision="fp32", kernel="persistent", device=local, stream=stream.cuda_stream)
        s3 = h.get_state()   # each run is the same 30 days from the initial state (walls and room air)
        with torch.cuda.stream(stream):
            h.run(wl3.n_steps)
        torch.cuda.synchronize()
        tl = []
        for _ in range(3):
            h.set_state(s3)
            with torch.cuda.stream(stream):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                h.run(wl3.n_steps)
                e1.record(stream)
            torch.cuda.synchronize()
            tl.append(e0.elapsed_time(e1))
        h.close()
        ms3 = float(np.mean(tl))
        other["rooms_64x6_30days"] = {"value": wl3.total_nodes * wl3.n_steps / (ms3 / 1e3), "unit": UNIT,
                                      "ms_per_run": ms3, "walls": wl3.n_walls, "rooms": 64,
                                      "note": "wall cell-updates/s; one block per room, FP64 room nodes"}

    # the paper's one-zone case (Sec. 5.2: 4 walls + 1 zone, 80 h at dt = 3.6 s), FP32 and FP64; parity of
    # the hourly surface samples against the oracle
    if not args.no_fp64:
        wl5 = wk.one_zone()
        res = {}
        for prec in ("fp32", "fp64"):
            h = H.Hygro(wl5, precision=prec, device=local, stream=stream.cuda_stream)
            smp = np.zeros((wl5.n_steps // 1000, wl5.n_walls, 2, 2), np.float32 if prec == "fp32" else np.float64)
            with torch.cuda.stream(stream):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                h.run(wl5.n_steps, 1000, smp)
                e1.record(stream)
            torch.cuda.synchronize()
            ms5 = e0.elapsed_time(e1)
            h.close()
            res[prec] = {"value": wl5.total_nodes * wl5.n_steps / (ms5 / 1e3), "ms_per_run": ms5, "samples": smp}
        out5 = {"value": res["fp32"]["value"], "unit": UNIT, "ms_per_run_fp32": res["fp32"]["ms_per_run"],
                "ms_per_run_fp64": res["fp64"]["ms_per_run"],
                "workload": "4 walls N=101 around one zone, 80 h at dt = 3.6 s (80 000 steps), FP32",
                "note": "one block (the zone's); latency-bound, reported, not roofline-graded; the time includes the "
                        "hourly samples copied to the host"}
        if rank == 0 and not args.no_cpu_baseline:
            import oracle

            t = time.perf_counter()
            r5 = oracle.Oracle(wl5).run(wl5.n_steps, 1000)
            el5 = time.perf_counter() - t
            ref = r5["samples"]
            out5["parity_vs_oracle"] = {
                prec: {f: float(np.max(np.abs(res[prec]["samples"][..., i] - ref[..., i])) / np.max(np.abs(ref[..., i])))
                       for i, f in enumerate(("rel_linf_T", "rel_linf_P"))} for prec in ("fp32", "fp64")}
            out5["oracle_seconds"] = el5
        other["one_zone_80h"] = out5

    # the Table-1 material of Sec. 4 (nonlinear coefficients of T and Pv) on the plain kernel: throughput and
    # parity of a sampled wall against the oracle
    if not args.no_fp64:
        other["table1_material_256walls"] = bench_table1(args, H, wk, stream, local, rank)

    # the paper's comparison schemes on the host cores (CPU time ratios of Sec. 4 and Sec. 5.2)
    if rank == 0 and not args.no_cpu_baseline:
        other["cpu_schemes"] = bench_cpu_schemes(wk)

    # gradient workload (1024 walls x 30 days, reverse-time adjoint)
    if not args.no_adjoint:
        other["adjoint_1024x200_30days"] = bench_adjoint(args, H, wk, stream, local, rank, peaks)

    # 2D sections (64 x 512 x 512, 10000 steps, FP32, 4 fused steps per TMA-tiled launch)
    if not args.no_2d:
        other["sections_64x512x512_10000steps"] = bench_sections(args, H, wk, stream, local, rank, peaks)

    # end to end through the C ABI with host buffers: inputs H2D, run, samples and fluxes D2H
    e2e = None
    if not args.no_e2e:
        import ctypes as C

        lay = (H.hygro_layer * len(wl.layer_par))(*[H.hygro_layer(*map(float, r)) for r in wl.layer_par])
        bcs = []

        def pinned(shape, dtype, fill=None):
            # page-locked host memory (the caller's side of the copies), viewed as numpy
            t = torch.empty(shape, dtype=dtype, pin_memory=True)
            a = t.numpy()
            a[...] = 0 if fill is None else fill
            return t, a

        # the inputs live in pinned host memory, as a caller that streams them would keep them
        pin_keep = []
        noise = []
        for z in wl.noise:
            if z is None:
                noise.append(None)
                continue
            t, a = pinned(z.shape, torch.float32, z)
            pin_keep.append(t)
            noise.append(a)
        for f in range(2):
            arr = (H.hygro_bc * wl.n_walls)()
            for w in range(wl.n_walls):
                b = arr[w]
                b.kind = int(wl.bc_kind[w, f])
                (b.hT, b.hM, b.q_inf, b.g_inf, b.T_mean, b.T_amp, b.P_mean, b.P_amp, b.period, b.phase_T,
                 b.phase_P, b.noise_dt, b.period_P) = map(float, wl.bc_par[w, f])
                if noise[f] is not None:
                    b.noise = noise[f][w].ctypes.data
                    b.noise_len = noise[f].shape[1]
            bcs.append(arr)
        nl = np.ascontiguousarray(wl.n_layers, np.int32)
        lf = np.ascontiguousarray(wl.layer_first, np.int32)
        Ti = np.ascontiguousarray(wl.T_init, np.float64)
        Pi = np.ascontiguousarray(wl.P_init, np.float64)
        se = 1440
        ts, samples = pinned((args.year_steps // se, wl.n_walls, 2, 2), torch.float32)
        tf, flux = pinned((wl.n_walls, 2, 2), torch.float64)
        tc, cum = pinned((wl.n_walls, 2, 2), torch.float64)
        pin_keep += [ts, tf, tc]
        h2d = (nl.nbytes + lf.nbytes + C.sizeof(lay) + Ti.nbytes + Pi.nbytes + sum(C.sizeof(a) for a in bcs)
               + sum(z.nbytes for z in noise if z is not None))
        d2h = samples.nbytes + flux.nbytes + cum.nbytes
        k = max(1, args.steps)   # the same steps as the timed kernel runs (the upload time varies from call to call)

        def e2e_step():
            H.hygro_set_materials(g.ctx, nl, lf, lay, Ti, Pi)
            H.hygro_set_bc(g.ctx, 0, bcs[0])
            H.hygro_set_bc(g.ctx, 1, bcs[1])
            H.hygro_run(g.ctx, args.year_steps, se, samples)
            H.hygro_fluxes(g.ctx, flux, cum)

        e2e_step()   # warm-up: the context's first upload allocates its staging buffers
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(k):
            e2e_step()
        el = (time.perf_counter() - t) / k
        el = reduce_max(pg, el)
        e2e = {"value": units_total / el, "unit": UNIT, "host_memory": "pinned", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "seconds_per_step": el}
    g.close()

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {**batch_config(wl, args.year_steps), "path": "FP32 persistent kernel",
                           "l2": "flushed between timed runs (512 MB write)", "parallelism": f"replicas x{world}"},
                "roofline": roofline, "cpu_baseline": cpu_baseline, "e2e": e2e,
                "gpu_launches": args.steps, "clocks": cs.summary(), "parity_vs_oracle": parity,
                "comparators": comparators, "other_workloads": other, "wall_seconds_timed": t_wall,
                "peaks": peaks, "autotune": autotune}
        print(json.dumps(line))
    if pg is not None:
        pg.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        if int(os.environ.get("RANK", "0")) != 0:
            return
        bench_reference(args)
    else:
        bench_ours(args)


if __name__ == "__main__":
    main()
