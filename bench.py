#!/usr/bin/env python
"""Throughput of the GB300 Friedkin-Johnsen solver: certified solves per second.

One step = one complete fj_solve (ImprovedBLISOR to eps = 1e-6 with the FP64
certificate and restarts, Section 5) of the workload's opinion vector, inputs
resident in HBM.  The default workload is the directed R-MAT scale-22 graph
(4,194,304 nodes, 67,108,864 generated arcs, a = 0.57, b = c = 0.19, weights
U(0.5, 1.5) FP32, s ~ U[0, 1] FP32), FP32 push with an FP64 certificate.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
(FIFO ImprovedBLISOR) on the host cores instead.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOADS = {
    # name: generator, precision, omega, schedule
    "rmat22_dir": dict(gen="rmat_dir", scale=22, precision="fp32", omega=1.6, palette=8),
    "ba20k": dict(gen="ba", n=20000, precision="fp64", omega=1.5),
    "rmat24_und": dict(gen="rmat_und", scale=24, precision="fp32", omega=1.8, palette=12, cpu_scale=20),
    "rmat23_und": dict(gen="rmat_und", scale=23, precision="fp32", omega=1.8, cpu_scale=20),
    "rmat22_und": dict(gen="rmat_und", scale=22, precision="fp32", omega=1.8, cpu_scale=20),
    "rmat16_dir": dict(gen="rmat_dir", scale=16, precision="fp32", omega=1.6),
    "rmat20_dir": dict(gen="rmat_dir", scale=20, precision="fp32", omega=1.6),
    # the paper's other two opinion laws on the same graph: exponential (x_min = 1) and
    # power law (alpha = 2.5, x_min = 1), each normalised by its maximum (kinds 4 and 5)
    "rmat22_dir_exp": dict(gen="rmat_dir", scale=22, precision="fp32", omega=1.6, palette=8, opinions=4),
    "rmat22_dir_pareto": dict(gen="rmat_dir", scale=22, precision="fp32", omega=1.6, palette=8, opinions=5),
    # 64 opinion vectors (U[0,1], Beta(1/2,1/2), +-1 labels) as one multi-right-hand-side push
    "rmat22_und_k64": dict(gen="rmat_und_multi", scale=22, nvec=64, precision="fp32", omega=1.7, cpu_scale=19),
    "rmat16_und_k64": dict(gen="rmat_und_multi", scale=16, nvec=64, precision="fp32", omega=1.7),
    "rmat20_und_k64": dict(gen="rmat_und_multi", scale=20, nvec=64, precision="fp32", omega=1.7),
    # 256 BA graphs (m = 5), n log-uniform in [1e3, 2e5], one U[0,1] vector each, as one ragged handle
    "ragged256_ba": dict(gen="ragged", count=256, lo=1000, hi=200000, precision="fp32", omega=1.5, cpu_scale=None),
    # learned warm start: train on SBM/BA triples, then held-out directed R-MAT with 16 vectors
    "rmat23_warm16": dict(gen="warm", scale=23, nvec=16, precision="fp32", omega=1.6, palette=8,
                          train_steps=1200, lr=2e-3, cpu_scale=18),
    "rmat18_warm16": dict(gen="warm", scale=18, nvec=16, precision="fp32", omega=1.6, palette=8,
                          train_steps=200, lr=2e-3),
}
EPS = 1e-6
REF_BUDGET_S = 240.0  # timed oracle work of one --impl reference run
METRIC = "FJ solves/s to 1e-6 rel. err (GTEPS, % HBM roofline): plain vs batched/warm-start"


def make_workload(name, scale_override=None):
    from fjsynth import workloads as W
    spec = dict(WORKLOADS[name])
    if scale_override is not None:
        spec["scale"] = scale_override
    if spec["gen"] == "warm":
        g = W.rmat_directed(spec["scale"], nvec=spec["nvec"])
        src, dst, w = g["src"], g["dst"], g["w"]
    elif spec["gen"] == "rmat_dir":
        g = W.rmat_directed(spec["scale"], kind=spec.get("opinions", W.OP_UNIFORM))
        src, dst, w = g["src"], g["dst"], g["w"]
    elif spec["gen"] == "rmat_und":
        g = W.rmat_undirected(spec["scale"])
        src, dst, w = W.symmetrize_arcs(g["src"], g["dst"], None)
    elif spec["gen"] == "rmat_und_multi":
        g = W.rmat_multirhs(spec["scale"], spec["nvec"])
        src, dst, w = W.symmetrize_arcs(g["src"], g["dst"], None)
    else:
        g = W.ba_graph(spec["n"], 5)
        src, dst, w = W.symmetrize_arcs(g["src"], g["dst"], None)
    return spec, g, src, dst, w


def clocks_start():
    try:
        f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        p = subprocess.Popen(
            ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
             "--format=csv,noheader,nounits", "-lms", "200"], stdout=f, stderr=subprocess.DEVNULL)
        return p, f.name
    except Exception:
        return None, None


def clocks_stop(p, path, device_index=0):
    if p is None:
        return None
    p.terminate()
    try:
        p.wait(timeout=5)
    except Exception:
        p.kill()
    rows = []
    with open(path) as fh:
        for rec in csv.reader(io.StringIO(fh.read())):
            if len(rec) < 9:
                continue
            try:
                if int(rec[0]) != device_index:
                    continue
                rows.append([x.strip() for x in rec])
            except ValueError:
                continue
    os.unlink(path)
    if not rows:
        return None
    sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
    mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "reasons": reasons, "samples": len(rows)}




# Name of the single-vector sweep kernel the roofline object reports.
SWEEP_KERNEL = "k_sweep_gather + k_sweep_apply (one colour class)"

# DRAM bytes (read + write) per launch of the single-vector sweep, as a
# multiple of the dense bytes it streams, from one ncu capture per graph kind
# (key: generator, single vector).  Filled in from captures listed under
# profiles/; a kind without a capture reports traffic null.
SWEEP_TRAFFIC_RATIO = {
    ("rmat_und", True): (109.6 / 148.3, "ncu dram__bytes_read.sum + dram__bytes_write.sum of k_sweep_gather + "
                         "k_sweep_apply over the 16 class launches of one sweep of undirected R-MAT s23 (109.6 MB "
                         "per class against 148.3 MB dense), scaled to this launch's dense bytes"),
}


def roofline_of(p, kernel, traffic_key=None):
    """Roofline object of the push kernel from one profiled solve's info record.

    achieved = the method's own bytes of the profiled launches (per residual
    update the column, weight and increment, per push 32 bytes: the unit of
    work of Alg. 1-3) over their summed CUDA-event time.  The dense bytes the
    pull-form sweep actually streams (every nonzero of every class, every
    sweep) are reported beside it."""
    peak, peak_kind = measured_peak_hbm()
    secs = p["push_ms"] / 1e3
    launches = max(1, p["push_launches"])
    achieved = p["method_bytes"] / secs / 1e9 if secs > 0 else None
    dense = p["push_bytes"] / secs / 1e9 if secs > 0 else None
    ratio = SWEEP_TRAFFIC_RATIO.get(traffic_key)
    r = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
         "frac": achieved / peak if achieved else None,
         "traffic": ratio[0] * p["push_bytes"] / launches if ratio else None,
         "kernel": kernel, "peak_source": peak_kind,
         "bytes_per_launch": p["method_bytes"] / launches,
         "bytes_basis": "method: 4 col + 4 w (weighted) + sizeof(T) increment per residual update, 32 per push",
         "dense_bytes_per_launch": p["push_bytes"] / launches,
         "dense_achieved": dense, "dense_frac": dense / peak if dense else None,
         "avg_launch_us": 1e3 * p["push_ms"] / launches}
    if ratio:
        r["traffic_source"] = ratio[1]
    return r


ARM_PARTS = {"0xd4f": "Arm Neoverse-V2 (NVIDIA Grace)", "0xd40": "Arm Neoverse-V1", "0xd0c": "Arm Neoverse-N1"}


def host_cpu():
    """Host CPU model (lscpu, else /proc/cpuinfo) and logical core count."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    low = line.lower()
                    if low.startswith("model name"):
                        model = line.split(":", 1)[1].strip()
                        break
                    if low.startswith("cpu part") and model is None:
                        part = line.split(":", 1)[1].strip()
                        model = ARM_PARTS.get(part, "Arm CPU part " + part)
        except OSError:
            pass
    return {"model": model, "host_cores": os.cpu_count()}


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x: float, device) -> float:
    """The largest value of x over all ranks (replicas exchange only this scalar)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_step: float, steps: int, world: int, ms: float) -> float:
    """Units all ranks processed per second, over the slowest rank's time."""
    return world * steps * units_per_step / (ms / 1e3)


# ------------------------------------------------------------------ oracle arm

def oracle_solve_time(name, scale, omega, allcore=True):
    """One FIFO ImprovedBLISOR solve (FP64, one host thread) of the workload at `scale`,
    and the synchronous push rounds of Alg. 1 (omega 1, FP64) on every host core.

    Returns (fifo seconds, nnz, fifo finished, rounds seconds, threads, rounds, rounds finished)."""
    import oracle
    spec, g, src, dst, w = make_workload(name, scale)
    rp, col, wc = oracle.csr_from_arcs(g["n"], src, dst, w)
    s = g["S"][0]
    t0 = time.perf_counter()
    z, r, pushes, upd, ok = oracle.blisor_fifo(g["n"], rp, col, wc, s, EPS, omega)
    dt = time.perf_counter() - t0
    if not allcore:
        return dt, int(rp[-1]), ok, None, 0, 0, False
    t0 = time.perf_counter()
    _, _, _, _, rounds, ok_r, threads = oracle.push_rounds_threads(g["n"], rp, col, wc, s, EPS, 1.0)
    dt_r = time.perf_counter() - t0
    return dt, int(rp[-1]), ok, dt_r, threads, rounds, ok_r


def run_reference(args):
    """The oracle's FIFO ImprovedBLISOR (FP64, one host thread) on the full workload.

    Every timed step is one complete solve of the same graph and opinion vector
    the GPU arm solves.  A full-size solve of the large workloads takes minutes,
    so the run times as many of the requested steps as fit in REF_BUDGET_S
    (at least one) and skips the warm-up steps (a CPU loop has nothing to warm);
    the line reports the steps actually timed."""
    world, rank, _ = dist_init()
    if rank != 0:
        return 0
    import oracle
    spec = WORKLOADS[args.workload]
    omega = args.omega if args.omega is not None else spec["omega"]
    if spec["gen"] in ("ragged", "warm"):
        print(json.dumps({"impl": "reference", "unavailable": "the reference arm covers the single-graph "
                          "workloads; %s is timed by its own GPU-arm modes" % args.workload}), flush=True)
        return 0
    t0 = time.perf_counter()
    _, g, src, dst, w = make_workload(args.workload)
    n = g["n"]
    rp, col, wc = oracle.csr_from_arcs(n, src, dst, w)
    del src, dst
    S = g["S"]
    prep_s = time.perf_counter() - t0
    times, info = [], None
    while len(times) < max(1, args.steps):
        j = len(times) % len(S)
        t1 = time.perf_counter()
        z, r, pushes, upd, ok = oracle.blisor_fifo(n, rp, col, wc, S[j], EPS, omega)
        times.append(time.perf_counter() - t1)
        assert ok, "the oracle's FIFO solve did not finish"
        info = {"pushes": pushes, "updates": upd}
        if sum(times) * (len(times) + 1) / len(times) > REF_BUDGET_S:
            break
    tot = sum(times)
    value = len(times) / tot
    cpu = host_cpu()
    sample = (f"{len(times)} complete FIFO ImprovedBLISOR solve(s) (omega={omega}, eps={EPS}, FP64, one host "
              f"thread) of the full workload (n={n}, nnz={int(rp[-1])}); warm-up skipped; the run stops "
              f"after the step that reaches {REF_BUDGET_S:.0f} s; graph build {prep_s:.1f} s untimed")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": len(times), "warmup": 0, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "n": n, "nnz": int(rp[-1]),
                                            "omega": omega, "eps": EPS},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": sample,
                             "host_cpu": cpu["model"], "host_cores": cpu["host_cores"]},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "detail": {"pushes": info["pushes"], "updates": info["updates"], "steps_requested": args.steps,
                       "warmup_requested": args.warmup}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm

def run_gpu(args):
    import torch

    world, rank, local = dist_init()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2507_14864_gb300 import capi

    spec, g, src, dst, w = make_workload(args.workload)
    n = g["n"]
    omega = args.omega if args.omega is not None else spec["omega"]
    prec = capi.FJ_PREC_FP32 if spec["precision"] == "fp32" else capi.FJ_PREC_FP64
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    src_d = torch.from_numpy(src).to(dev)
    dst_d = torch.from_numpy(dst).to(dev)
    w_d = torch.from_numpy(w).to(dev) if w is not None else None
    G = capi.Graph.from_arcs(n, src_d, dst_d, w_d, directed=g["directed"])
    del src_d, dst_d, w_d
    ginfo = G.info()
    k = int(spec.get("nvec", 1))
    s_host = g["S"][0] if k == 1 else np.ascontiguousarray(np.stack(g["S"], axis=1))
    del g["S"]
    s_d = torch.from_numpy(s_host).to(dev)
    z_d = torch.empty_like(s_d)
    omega_est = None
    if args.omega_opt:
        # Eq. 17 from a power-iteration estimate of rho((I + D)^{-1} A), outside the timed region
        t0 = time.perf_counter()
        mu, omega = G.omega_opt(args.omega_opt)
        omega_est = {"mu": mu, "omega": omega, "iters": args.omega_opt, "s": time.perf_counter() - t0}
    opts = dict(eps=EPS, omega=omega, precision=prec, schedule=args.schedule)
    palette = args.palette if args.palette is not None else spec.get("palette")
    if palette is not None:
        opts["palette"] = palette

    cols = None
    if k > 1 and args.plain_loop:
        # the same k vectors, solved one fj_solve call each (the plain method)
        cols = [s_d[:, j].contiguous() for j in range(k)]
        zcol = torch.empty_like(cols[0])

    def solve(s, out, **kw):
        if k == 1:
            res = G.solve(s, out=out, **kw)
            if "profile" not in kw:
                G.metrics(s, res[0])  # a8: the Table 1 measures of the solve
            return res
        if cols is not None:
            infos_ = []
            if s is s_d:
                for c in cols:
                    infos_.extend(G.solve(c, out=zcol, **kw)[1])
                    if "profile" not in kw:
                        G.metrics(c, zcol)
            else:  # host buffers: one column at a time through the C ABI
                for j in range(k):
                    zj = np.empty(s.shape[0])
                    sj = np.ascontiguousarray(s[:, j])
                    infos_.extend(G.solve(sj, out=zj, **kw)[1])
                    G.metrics(sj, zj)
                    out[:, j] = zj
            return out, infos_, 0
        res = G.solve_batch(s, out=out, **kw)
        if "profile" not in kw:
            G.metrics_batch(s, res[0])  # a8 for every vector of the batch
        return res
    if args.check_every:
        opts["check_every"] = args.check_every
    if args.max_sweeps:
        opts["max_sweeps"] = args.max_sweeps

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    tuned = None
    if args.tune and cols is None:
        # autotuner (outside the timed region): schedule, palette, omega (and the batch gather depth)
        t0 = time.perf_counter()
        if k == 1:
            best, best_ms = G.tune(s_d, reps=1, **opts)
        else:
            best, best_ms = G.tune_batch(s_d, reps=1, **opts)
        opts.update(best)
        palette = best["palette"]
        omega = best["omega"]
        tuned = dict(best, tune_s=time.perf_counter() - t0, best_ms=best_ms)
    for _ in range(args.warmup):
        solve(s_d, z_d, **opts)
    barrier()
    clk, clk_path = clocks_start() if rank == 0 else (None, None)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    ev0.record(stream)
    for _ in range(args.steps):
        _, info, _ = solve(s_d, z_d, **opts)
        infos.extend(info)
    ev1.record(stream)
    barrier()
    clocks = clocks_stop(clk, clk_path, local) if rank == 0 else None
    ms = max_over_ranks(ev0.elapsed_time(ev1), dev)
    ms_per_step = ms / args.steps
    value = whole_job_value(k, args.steps, world, ms)
    assert all(i["converged"] == 1 for i in infos), "a timed solve did not certify"

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    s_pin = torch.from_numpy(s_host).pin_memory().numpy()
    z_pin = torch.empty(s_host.shape, dtype=torch.float64).pin_memory().numpy()
    solve(s_pin, z_pin, **opts)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        solve(s_pin, z_pin, **opts)
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dev)
    e2e_value = whole_job_value(k, args.steps, world, e2e_s * 1e3)

    # roofline of the push kernel: algorithmic bytes over CUDA-event time of its launches
    if cols is not None:
        _, pinfo, _ = G.solve(cols[0], out=zcol, profile=1, **opts)
    else:
        _, pinfo, _ = solve(s_d, z_d, profile=1, **opts)
    p = pinfo[0]
    kernel = (SWEEP_KERNEL if (k == 1 or cols is not None) else
              "%s (one colour class, %d vectors)"
              % ("k_sweep_batch_bulk" if (spec["precision"] == "fp32" and k % 4 == 0 and k <= 64)
                 else "k_sweep_batch", k))
    roofline = roofline_of(p, kernel, traffic_key=(spec["gen"], k == 1 or cols is not None))
    info0 = infos[-1]
    detail = {"sweeps": info0["sweeps"], "pushes": info0["pushes"], "edges": info0["edges"],
              "refine_passes": info0["refine_passes"], "resid_rel_max": info0["resid_rel_max"],
              "eps_prime": info0["eps_prime"], "gteps": info0["edges"] / (ms_per_step / 1e3) / 1e9,
              "ncolours": G.info()["ncolours"], "vectors_per_step": k}
    if args.trace and k == 1:
        # relative residual against time for one more solve, outside the timed region (Fig. 1's axes)
        _, _, _, tr = G.solve_trace(s_d, out=z_d, **opts)
        detail["trace"] = [[round(float(a), 4), int(b), float(c), int(d)] for a, b, c, d in tr]

    cpu = cpu_all = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu_scale = args.cpu_scale if args.cpu_scale is not None else spec.get("cpu_scale")
        dt, nnz_c, ok, dt_r, threads, rounds, ok_r = oracle_solve_time(args.workload, cpu_scale, omega)
        scale_f = nnz_c / ginfo["nnz"]
        hc = host_cpu()
        where = ("the full workload" if cpu_scale is None else
                 f"the same generator at scale {cpu_scale} (a bounded sample: a full-size solve "
                 f"takes minutes; bench.py --impl reference times full-size solves), rate scaled "
                 f"by nnz {nnz_c}/{ginfo['nnz']}")
        cpu = {"value": scale_f / dt, "unit": "solves/s", "cores": 1, "kind": "oracle",
               "sample": (f"one FIFO ImprovedBLISOR solve (omega={omega}, eps={EPS}, FP64, one host thread) of "
                          + where + f", {dt:.1f} s"),
               "host_cpu": hc["model"], "host_cores": hc["host_cores"]}
        cpu_all = {"value": scale_f / dt_r, "unit": "solves/s", "cores": threads, "kind": "oracle",
                   "sample": (f"the synchronous push rounds of Alg. 1 (omega 1, eps={EPS}, FP64; {rounds} rounds"
                              f"{'' if ok_r else ', unfinished'}) on {threads} host threads of " + where
                              + f", {dt_r:.1f} s"),
                   "host_cpu": hc["model"], "host_cores": hc["host_cores"]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec == capi.FJ_PREC_FP32 else "f64", "data": "synthetic",
            "config": {"workload": args.workload, "n": n, "nnz": ginfo["nnz"], "directed": g["directed"],
                       "vectors": k, "palette": palette,
                       "mode": ("batched (fj_solve_batch)" if k > 1 and cols is None else
                                "plain (one fj_solve per vector)"), "tuned": tuned,
                       "omega": opts["omega"], "omega_eq17": omega_est, "eps": EPS,
                       "schedule": {0: "auto (multicolour)", 1: "jacobi", 2: "multicolour"}[opts["schedule"]],
                       "precision": "FP32 push, FP64 estimate and certificate" if prec == capi.FJ_PREC_FP32
                       else "FP64", "l2": "inputs larger than L2 (CSR %.2f GB)" % (
                           ginfo["nnz"] * (8 if w is not None else 4) / 1e9),
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "e2e": {"value": e2e_value, "unit": "solves/s",
                    "h2d_bytes_per_step": (24 if k == 1 else 8) * n * k, "d2h_bytes_per_step": 8 * n * k},
            # solve launches plus the five of each metrics call
            "gpu_launches": int(sum(i["launches"] for i in (infos if cols is not None else infos[::k])))
            + 5 * args.steps * (k if cols is not None else 1),
            "roofline": roofline, "cpu_baseline": cpu, "cpu_baseline_allcore": cpu_all, "clocks": clocks,
            "detail": detail,
        }
        print(json.dumps(line), flush=True)
    G.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_omega_sweep(args):
    """One graph, several relaxation factors (Section 5.2's omega search; the
    update counts of Fig. 2): per omega, certified solves/s, sweeps, pushes and
    residual updates of the GPU schedule, next to the pushes and updates of the
    oracle's FIFO ImprovedBLISOR at the same omega (host, untimed).  omega = 1
    runs both synchronous rounds (JACOBI, the round view of Alg. 1) and the
    multicolour Gauss-Seidel order.  The line's value is the fastest entry."""
    import torch

    world, rank, local = dist_init()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    from paper_2507_14864_gb300 import capi

    spec, g, src, dst, w = make_workload(args.workload)
    n = g["n"]
    prec = capi.FJ_PREC_FP32 if spec["precision"] == "fp32" else capi.FJ_PREC_FP64
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    G = capi.Graph.from_arcs(n, torch.from_numpy(src).to(dev), torch.from_numpy(dst).to(dev),
                             None if w is None else torch.from_numpy(w).to(dev), directed=g["directed"])
    ginfo = G.info()
    s_host = g["S"][0]
    s_d = torch.from_numpy(s_host).to(dev)
    z_d = torch.empty_like(s_d)
    small = n <= 2_000_000
    rp = col = wc = None
    if small and rank == 0:
        rp, col, wc = oracle.csr_from_arcs(n, src, dst, w)
    omegas = [float(x) for x in args.omega_sweep.split(",")]
    cases = []
    for om in omegas:
        if om == 1.0:
            cases.append((om, capi.FJ_SCHED_JACOBI))
        cases.append((om, capi.FJ_SCHED_MULTICOLOUR))

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    rows = []
    clk, clk_path = clocks_start() if rank == 0 else (None, None)
    for om, sched in cases:
        opts = dict(eps=EPS, omega=om, precision=prec, schedule=sched)
        if spec.get("palette") is not None:
            opts["palette"] = spec["palette"]
        for _ in range(args.warmup):
            G.solve(s_d, out=z_d, **opts)
            G.metrics(s_d, z_d)
        barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        infos = []
        ev0.record(stream)
        for _ in range(args.steps):
            _, inf, _ = G.solve(s_d, out=z_d, **opts)
            G.metrics(s_d, z_d)
            infos.extend(inf)
        ev1.record(stream)
        barrier()
        ms = max_over_ranks(ev0.elapsed_time(ev1), dev)
        assert all(i["converged"] == 1 for i in infos), "a timed solve did not certify"
        i0 = infos[-1]
        row = {"omega": om, "schedule": "jacobi" if sched == capi.FJ_SCHED_JACOBI else "multicolour",
               "solves_per_s": whole_job_value(1, args.steps, world, ms), "ms_per_solve": ms / args.steps,
               "sweeps": i0["sweeps"], "pushes": i0["pushes"], "updates": i0["edges"],
               "launches": i0["launches"], "opts": opts}
        if rp is not None:
            _, _, fp, fu, ok = oracle.blisor_fifo(n, rp, col, wc, s_host, EPS, om)
            row.update(oracle_fifo_pushes=fp, oracle_fifo_updates=fu)
        rows.append(row)
    clocks = clocks_stop(clk, clk_path, local) if rank == 0 else None
    best = max(rows, key=lambda r: r["solves_per_s"])
    opts = best.pop("opts")
    for r in rows:
        r.pop("opts", None)

    s_pin = torch.from_numpy(s_host).pin_memory().numpy()
    z_pin = torch.empty(n, dtype=torch.float64).pin_memory().numpy()
    G.solve(s_pin, out=z_pin, **opts)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        G.solve(s_pin, out=z_pin, **opts)
        G.metrics(s_pin, z_pin)
    barrier()
    e2e_value = whole_job_value(1, args.steps, world, max_over_ranks(time.perf_counter() - t0, dev) * 1e3)
    _, pinfo, _ = G.solve(s_d, out=z_d, profile=1, **opts)
    roofline = roofline_of(pinfo[0], SWEEP_KERNEL)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and rp is not None:
        t0 = time.perf_counter()
        reps = 0
        while reps < 1 or time.perf_counter() - t0 < 10.0:
            oracle.blisor_fifo(n, rp, col, wc, s_host, EPS, best["omega"])
            reps += 1
        dt = (time.perf_counter() - t0) / reps
        hc = host_cpu()
        cpu = {"value": 1.0 / dt, "unit": "solves/s", "cores": 1, "kind": "oracle",
               "sample": f"{reps} complete FIFO ImprovedBLISOR solves of the full workload (omega="
                         f"{best['omega']}, eps={EPS}, FP64, one host thread)",
               "host_cpu": hc["model"], "host_cores": hc["host_cores"]}
    if rank == 0:
        line = {
            "metric": METRIC, "value": best["solves_per_s"], "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": best["ms_per_solve"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if prec == capi.FJ_PREC_FP32 else "f64", "data": "synthetic",
            "config": {"workload": args.workload, "n": n, "nnz": ginfo["nnz"], "directed": g["directed"],
                       "omega": best["omega"], "schedule": best["schedule"], "eps": EPS,
                       "mode": "omega sweep " + args.omega_sweep, "l2": "inputs smaller than L2: the "
                       "whole graph and state stay L2-resident (a latency-bound small solve)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n},
            "gpu_launches": int(sum(r["launches"] for r in rows)) * args.steps + 5 * args.steps * len(rows),
            "roofline": roofline, "cpu_baseline": cpu, "clocks": clocks,
            "detail": {"omega_sweep": rows},
        }
        print(json.dumps(line), flush=True)
    G.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_warm(args):
    """Learned warm start: solves/s of (predict z0 + push from z0) against the
    zero start on the same vectors, both to the same certificate."""
    import torch

    world, rank, local = dist_init()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2507_14864_gb300 import capi
    from fjsynth import workloads as W

    spec = WORKLOADS[args.workload]
    dev = torch.device("cuda", local)
    omega = args.omega if args.omega is not None else spec["omega"]
    prec = capi.FJ_PREC_FP32
    palette = args.palette if args.palette is not None else spec.get("palette")
    opts = dict(eps=EPS, omega=omega, precision=prec, schedule=args.schedule)
    if palette is not None:
        opts["palette"] = palette

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # ---- training (outside the timed region): triples from the plain solver
    t0 = time.perf_counter()
    triples, graphs = [], []
    for gd in W.warm_training_set():
        if gd["directed"]:
            a, b, ww = gd["src"], gd["dst"], gd["w"]
        else:
            a, b, ww = W.symmetrize_arcs(gd["src"], gd["dst"], None)
        G = capi.Graph.from_arcs(gd["n"], torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev),
                                 None if ww is None else torch.from_numpy(ww).to(dev), directed=gd["directed"])
        graphs.append(G)
        # targets: the plain solver (SOR only where it is safe, omega 1 on directed graphs)
        topts = dict(opts, omega=1.0 if gd["directed"] else omega)
        for sv in gd["S"]:
            s_d = torch.from_numpy(sv).to(dev)
            z_d, info, _ = G.solve(s_d, **topts)
            triples.append((G, s_d, z_d))
    net = capi.MPNN(capi.MPNN.initial_params(1))
    losses = []
    nsteps = spec["train_steps"]
    for it in range(nsteps):
        G, s_d, z_d = triples[it % len(triples)]
        # cosine decay of the learning rate to a tenth over the run
        lr = spec["lr"] * (0.55 + 0.45 * np.cos(np.pi * it / nsteps))
        losses.append(net.train_step(G, s_d, z_d, lr))
    barrier()
    train_s = time.perf_counter() - t0

    # ---- held-out evaluation graph
    _, g, src, dst, w = make_workload(args.workload)
    n = g["n"]
    G = capi.Graph.from_arcs(n, torch.from_numpy(src).to(dev), torch.from_numpy(dst).to(dev),
                             torch.from_numpy(w).to(dev), directed=True)
    ginfo = G.info()
    k = spec["nvec"]
    S = [torch.from_numpy(sv).to(dev) for sv in g["S"]]
    z_d = torch.empty_like(S[0])
    z0_d = torch.empty_like(S[0])

    def warm_step(infos=None):
        for s_d in S:
            net.predict(G, s_d, out=z0_d)
            _, inf, _ = G.solve(s_d, out=z_d, z0=z0_d, **opts)
            if infos is not None:
                infos.extend(inf)

    def zero_step(infos=None):
        for s_d in S:
            _, inf, _ = G.solve(s_d, out=z_d, **opts)
            if infos is not None:
                infos.extend(inf)

    # the batched forms: the k vectors as one multi-right-hand-side push, from
    # zero or from the network's starts (each judged against its zero start)
    S_b = torch.stack(S, dim=1).contiguous()
    Z_b = torch.empty_like(S_b)
    Z0_b = torch.empty_like(S_b)

    def warm_batch_step(infos=None):
        for j, s_d in enumerate(S):
            net.predict(G, s_d, out=z0_d)
            Z0_b[:, j].copy_(z0_d)
        _, inf, _ = G.solve_batch(S_b, out=Z_b, Z0=Z0_b, **opts)
        if infos is not None:
            infos.extend(inf)

    def zero_batch_step(infos=None):
        _, inf, _ = G.solve_batch(S_b, out=Z_b, **opts)
        if infos is not None:
            infos.extend(inf)

    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        barrier()
        infos = []
        ev0.record(stream)
        for _ in range(args.steps):
            fn(infos)
        ev1.record(stream)
        barrier()
        return max_over_ranks(ev0.elapsed_time(ev1), dev), infos

    ms_zero, inf_zero = timed(zero_step)
    clk, clk_path = clocks_start() if rank == 0 else (None, None)
    ms_warm, inf_warm = timed(warm_step)
    clocks = clocks_stop(clk, clk_path, local) if rank == 0 else None
    ms_zero_b, inf_zero_b = timed(zero_batch_step)
    ms_warm_b, inf_warm_b = timed(warm_batch_step)
    assert all(i["converged"] == 1 for i in inf_warm + inf_zero + inf_zero_b + inf_warm_b), \
        "a timed solve did not certify"
    value = whole_job_value(k, args.steps, world, ms_warm)
    zero_value = whole_job_value(k, args.steps, world, ms_zero)
    batch = {"zero_batch_solves_per_s": whole_job_value(k, args.steps, world, ms_zero_b),
             "warm_batch_solves_per_s": whole_job_value(k, args.steps, world, ms_warm_b),
             "sweeps_zero_batch": inf_zero_b[-1]["sweeps"], "sweeps_warm_batch": inf_warm_b[-1]["sweeps"],
             "warm_batch_starts_kept": int(sum(1 for i in inf_warm_b[-k:] if i["warm_start"] == 1))}
    batch["warm_batch_vs_zero_batch"] = batch["warm_batch_solves_per_s"] / batch["zero_batch_solves_per_s"]
    # predict time alone
    barrier()
    ev0.record(stream)
    for s_d in S:
        net.predict(G, s_d, out=z0_d)
    ev1.record(stream)
    barrier()
    predict_ms = ev0.elapsed_time(ev1) / k

    # end to end with host buffers through the C ABI: predict and warm solve per vector
    s_pin = [torch.from_numpy(sv).pin_memory().numpy() for sv in g["S"]]
    z0_pin = torch.empty(n, dtype=torch.float64).pin_memory().numpy()
    z_pin = torch.empty(n, dtype=torch.float64).pin_memory().numpy()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for sp in s_pin:
            net.predict(G, sp, out=z0_pin)
            G.solve(sp, out=z_pin, z0=z0_pin, **opts)
    barrier()
    e2e_value = whole_job_value(k, args.steps, world, max_over_ranks(time.perf_counter() - t0, dev) * 1e3)

    _, pinfo, _ = G.solve(S[0], out=z_d, z0=z0_d, profile=1, **opts)
    p = pinfo[0]
    roofline = roofline_of(p, SWEEP_KERNEL)
    # quality of the start: z0 against the certified zero-start solution, and the
    # share of nodes whose initial residual is above threshold (zero start: all)
    zq = {}
    for j in range(min(k, 4)):
        net.predict(G, S[j], out=z0_d)
        _, inf0, _ = G.solve(S[j], out=z_d, **opts)
        z0 = z0_d.cpu().numpy()
        zz = z_d.cpu().numpy()
        zq.setdefault("z0_err_inf_rel", []).append(float(np.max(np.abs(z0 - zz)) / np.max(np.abs(zz))))
        zq.setdefault("z0_err_rms", []).append(float(np.sqrt(np.mean((z0 - zz) ** 2))))
        sv = g["S"][j]
        zq.setdefault("s_err_rms", []).append(float(np.sqrt(np.mean((sv - zz) ** 2))))
    zq = {key: float(np.mean(v)) for key, v in zq.items()}
    mean = lambda xs: float(np.mean(xs)) if xs else None
    detail = {"zero_start_solves_per_s": zero_value, "warm_vs_zero": value / zero_value, **batch,
              "starts_kept": int(sum(1 for i in inf_warm[-k:] if i["warm_start"] == 1)),
              "sweeps_warm": mean([i["sweeps"] for i in inf_warm]),
              "sweeps_zero": mean([i["sweeps"] for i in inf_zero]),
              "predict_ms": predict_ms, "train_s": train_s, "train_steps": spec["train_steps"],
              "train_loss_first": losses[0], "train_loss_last": float(np.mean(losses[-20:])),
              "ncolours": G.info()["ncolours"], "vectors_per_step": k, **zq}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu_scale = args.cpu_scale if args.cpu_scale is not None else spec.get("cpu_scale")
        dt, nnz_c, ok = oracle_solve_time(args.workload, cpu_scale, omega, allcore=False)[:3]
        cpu = {"value": (nnz_c / ginfo["nnz"]) / dt, "unit": "solves/s", "cores": 1, "kind": "oracle",
               "sample": (f"one FIFO ImprovedBLISOR solve (omega={omega}, eps={EPS}, FP64, zero start, one host "
                          f"thread) of the same generator at scale {cpu_scale}, rate scaled by nnz "
                          f"{nnz_c}/{ginfo['nnz']}, {dt:.1f} s")}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_warm / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "n": n, "nnz": ginfo["nnz"], "directed": True, "vectors": k,
                       "palette": palette, "mode": "learned warm start (predict + fj_solve_warm)",
                       "omega": omega, "eps": EPS, "precision": "FP32 push, FP64 estimate and certificate; "
                       "network BF16 GEMMs with FP32 accumulation",
                       "l2": "inputs larger than L2 (CSR %.2f GB)" % (ginfo["nnz"] * 8 / 1e9),
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": 24 * n * k,
                    "d2h_bytes_per_step": 16 * n * k},
            "gpu_launches": int(sum(i["launches"] for i in inf_warm)) + 6 * k * args.steps,
            "roofline": roofline, "cpu_baseline": cpu, "clocks": clocks, "detail": detail,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_ragged(args):
    """Ragged batch: every graph of the batch solved (and its metrics taken) by one
    solve over the block-diagonal handle; --plain-loop solves them one handle each."""
    import torch

    world, rank, local = dist_init()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2507_14864_gb300 import capi
    from fjsynth import workloads as W

    spec = WORKLOADS[args.workload]
    dev = torch.device("cuda", local)
    omega = args.omega if args.omega is not None else spec["omega"]
    opts = dict(eps=EPS, omega=omega, precision=capi.FJ_PREC_FP32, schedule=args.schedule)
    palette = args.palette if args.palette is not None else spec.get("palette")
    if palette is not None:
        opts["palette"] = palette
    r = W.ragged_ba(spec["count"], spec["lo"], spec["hi"])
    parts = []
    for gr in r["graphs"]:
        a, b, _ = W.symmetrize_arcs(gr["src"], gr["dst"])
        parts.append((gr["n"], a, b, None))
    s_host = np.concatenate([gr["s"] for gr in r["graphs"]])
    ng = len(parts)
    n = int(s_host.shape[0])

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    if args.plain_loop:
        handles = [capi.Graph.from_arcs(pn, torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev), None,
                                        directed=False) for pn, a, b, _ in parts]
        svecs = [torch.from_numpy(gr["s"]).to(dev) for gr in r["graphs"]]
        nnz = sum(h.info()["nnz"] for h in handles)

        def step(infos=None):
            for h, sv in zip(handles, svecs):
                z, inf, _ = h.solve(sv, **opts)
                h.metrics(sv, z)
                if infos is not None:
                    infos.extend(inf)
        mode = "plain (one handle and one fj_solve per graph)"
    else:
        G = capi.Graph.ragged_from_arcs(parts, directed=False)
        nnz = G.info()["nnz"]
        s_d = torch.from_numpy(s_host).to(dev)
        z_d = torch.empty_like(s_d)

        def step(infos=None):
            _, inf, _ = G.solve(s_d, out=z_d, **opts)
            G.metrics(s_d, z_d)
            if infos is not None:
                infos.extend(inf)
        mode = "ragged (one handle, one fj_solve for all graphs)"
    for _ in range(args.warmup):
        step()
    barrier()
    clk, clk_path = clocks_start() if rank == 0 else (None, None)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    infos = []
    ev0.record(stream)
    for _ in range(args.steps):
        step(infos)
    ev1.record(stream)
    barrier()
    clocks = clocks_stop(clk, clk_path, local) if rank == 0 else None
    ms = max_over_ranks(ev0.elapsed_time(ev1), dev)
    assert all(i["converged"] == 1 for i in infos), "a timed solve did not certify"
    value = whole_job_value(ng, args.steps, world, ms)
    e2e_value = None
    if not args.plain_loop:
        s_pin = torch.from_numpy(s_host).pin_memory().numpy()
        z_pin = torch.empty(n, dtype=torch.float64).pin_memory().numpy()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            G.solve(s_pin, out=z_pin, **opts)
            G.metrics(s_pin, z_pin)
        barrier()
        e2e_value = whole_job_value(ng, args.steps, world, max_over_ranks(time.perf_counter() - t0, dev) * 1e3)
        _, pinfo, _ = G.solve(s_d, out=z_d, profile=1, **opts)
        p = pinfo[0]
    else:
        _, pinfo, _ = handles[-1].solve(svecs[-1], profile=1, **opts)
        p = pinfo[0]
    roofline = roofline_of(p, SWEEP_KERNEL)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "graphs": ng, "n": n, "nnz": nnz, "directed": False,
                       "mode": mode, "omega": omega, "eps": EPS, "palette": palette,
                       "precision": "FP32 push, FP64 estimate, certificate and metrics",
                       "l2": "inputs larger than L2", "parallelism": "replicas" if world > 1 else "single GPU"},
            "e2e": None if e2e_value is None else {"value": e2e_value, "unit": "solves/s",
                                                   "h2d_bytes_per_step": 24 * n, "d2h_bytes_per_step": 8 * n},
            "gpu_launches": int(sum(i["launches"] for i in infos[::ng])) if not args.plain_loop else
            int(sum(i["launches"] for i in infos)),
            "roofline": roofline, "cpu_baseline": None, "clocks": clocks,
            "detail": {"sweeps": max(i["sweeps"] for i in infos), "graphs_per_step": ng},
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rmat24_und", choices=sorted(WORKLOADS))
    ap.add_argument("--omega", type=float, default=None)
    ap.add_argument("--omega-opt", type=int, default=0, metavar="ITERS",
                    help="take omega from Eq. 17 with mu from ITERS power-iteration steps (fj_graph_omega_opt)")
    ap.add_argument("--trace", action="store_true",
                    help="add one traced solve's [ms, sweeps, max|r|/s', kind] rows to detail (fj_solve_trace)")
    ap.add_argument("--schedule", type=int, default=2, help="1 Jacobi rounds, 2 multicolour")
    ap.add_argument("--check-every", type=int, default=0)
    ap.add_argument("--max-sweeps", type=int, default=0, help="sweeps per pass before a refinement restart")
    ap.add_argument("--cpu-scale", type=int, default=None,
                    help="R-MAT scale of the CPU-baseline sample (default: the full workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--palette", type=int, default=None)
    ap.add_argument("--tune", action="store_true",
                    help="run the autotuner (fj_graph_tune / fj_graph_tune_batch) before timing")
    ap.add_argument("--omega-sweep", default=None, metavar="W1,W2,...",
                    help="time the workload at each relaxation factor (omega = 1 also as Jacobi rounds)")
    ap.add_argument("--plain-loop", action="store_true",
                    help="multi-vector workloads: solve the vectors one fj_solve call each")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.omega_sweep:
        return run_omega_sweep(args)
    if WORKLOADS[args.workload]["gen"] == "warm":
        return run_warm(args)
    if WORKLOADS[args.workload]["gen"] == "ragged":
        return run_ragged(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
