#!/usr/bin/env python3
"""Benchmark of the volumetric path-graph hot path on GB300.

One step = one pass of the whole hot path over the heterogeneous-cloud
workload (128^3 fBm medium, albedo 0.99, HG g = 0.8, sun + sky, 256x256
pixels, 16 spp, depth 64, about 8.7M scattering vertices; k = 16, 30 sweeps,
FP32 weights): graph build, aggregation, propagation with history, output,
and the adjoint sweep for an image loss.

Prints one JSON line (rank 0). `value` is propagation edge-updates per
second of the whole step (forward + reverse sweeps over the step's wall time
on the device); per-stage times, the propagation-only rate, the 16-bit
weight variants, the roofline of the sweep kernel and the FP64 oracle's rate
on the host cores are reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "propagation edge-updates/s & % HBM peak; 16-bit vs FP32 weights at <=2e-3 rel err"
UNIT = "edge-updates/s"
L2_BYTES = 129 * 2 ** 20


WORKLOADS = ("cloud128", "dense256")
EXTRA_M = 4  # extra emitter samples per path for the output-option timings
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # nominal FP32 FMA rate at the maximum SM clock


def _scene(name):
    import pgrec

    return {"cloud128": pgrec.CLOUD128, "dense256": pgrec.CLOUD256_DENSE}[name]


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- GPU arm
def run_gpu(args):
    import torch

    import paper_2404_11894_gb300 as pg
    import pgrec

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    from paper_2404_11894_gb300.dist import combine_throughput, rank_seed

    sc = _scene(args.workload)
    wdtype = args.weights or (sc.weight_dtypes[0] if sc.weight_dtypes else "f32")
    if args.scale != 1.0:  # smaller image of the same scene (profiling captures)
        sc = sc.with_(width=int(sc.width * args.scale), height=int(sc.height * args.scale))
    if world > 1:  # independent renders (replicas), one per rank
        sc = sc.with_(seed=rank_seed(sc.seed, rank))
    # the extra first-vertex samples come from a random stream of their own:
    # the path records are the same with or without them
    t_tr = time.perf_counter()
    rec = pgrec.trace(sc if args.quick else sc.with_(extra_direct=EXTRA_M))
    host_trace_s = time.perf_counter() - t_tr
    n, P = rec["n"], rec["n_paths"]
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    # host copies in pinned memory (for the end-to-end leg)
    def pinned(a):
        t = torch.from_numpy(np.ascontiguousarray(a))
        return t.pin_memory()

    host = {k: pinned(rec[k]) for k in pg.VERTEX_F32 + ("e_delta", "succ", "L0", "first", "bg", "voxel")}
    rng = np.random.default_rng(0)
    target = rec["pt_image"].astype(np.float32) * rng.uniform(0.9, 1.1, rec["pt_image"].shape).astype(np.float32)
    host_target = pinned(target)
    dev_in = {k: v.to(dev) for k, v in host.items()}
    dev_target = host_target.to(dev)
    V = pg.Vertices({k: dev_in[k] for k in pg.VERTEX_F32 + ("e_delta", "succ")})
    solver = pg.Solver(k=sc.k, iters=sc.iters, wdtype=wdtype, adjoint=not args.no_adjoint,
                       cluster_size=args.clusters, cluster_seed=sc.seed,
                       recompute_weights=args.adjoint_mode, want_g=False, n_vox=sc.grid_res ** 3)

    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def step(V, L0, first, bg, tgt, marks=None):
        return solver.step(V, L0, first, bg, sc.spp, sc.width, sc.height, tgt, marks=marks,
                           voxel=dev_in["voxel"], sigma_t=dev_in["sigma_t"])

    for _ in range(args.warmup):
        step(V, dev_in["L0"], dev_in["first"], dev_in["bg"], dev_target)
    torch.cuda.synchronize()
    info = solver.graph.info()
    nnz = info["nnz_swept"]
    sweeps_per_step = sc.iters * (2 if not args.no_adjoint else 1)
    edge_updates_step = nnz * sweeps_per_step

    # ---- device-timed region (inputs resident in HBM)
    stage_names = ["build", "aggregate", "propagate", "gather", "adjoint"]
    marks_all = []
    launches0 = pg.launch_count()
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = ev(), ev()
    e0.record(stream)
    for _ in range(args.steps):
        marks = {nm: (ev(), ev()) for nm in stage_names}
        step(V, dev_in["L0"], dev_in["first"], dev_in["bg"], dev_target, marks=marks)
        marks_all.append(marks)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = pg.launch_count() - launches0
    t_dev, total_updates = combine_throughput(e0.elapsed_time(e1) / 1e3, float(edge_updates_step) * args.steps,
                                              device=dev)
    stage_ms = {nm: float(np.mean([m[nm][0].elapsed_time(m[nm][1]) for m in marks_all if m[nm][0].query()]))
                for nm in stage_names if not (args.no_adjoint and nm == "adjoint")}

    # ---- end to end through the C ABI's host-buffer entry point (pg_step_host):
    # host records -> image and gradient on the host (measured right after the
    # device-timed steps, in the same state)
    e2e_t = []
    h2d = sum(int(v.numel() * v.element_size()) for v in host.values()) + host_target.numel() * 4
    # the image, and with the adjoint the per-voxel albedo gradient
    d2h = sc.width * sc.height * 4 + (0 if args.no_adjoint else 4 * sc.grid_res ** 3)
    for i in range(args.steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        img = solver.solve_host(host, host_target, sc.spp, sc.width, sc.height)
        t1 = time.perf_counter()
        if i > 0:
            e2e_t.append(t1 - t0)
    e2e_value = edge_updates_step / float(np.mean(e2e_t))

    pt = rec["pt_image"].astype(np.float64)
    solver_img_ratio = float(solver.last_image.double().mean()) / float(pt.mean()) if pt.mean() > 0 else None

    # ---- sweep kernel roofline: the propagate stage of the timed steps minus its
    # prologue/epilogue (pg_propagate with zero sweeps, started on an idle
    # device as in the step, where the aggregation synchronised), per sweep
    prop_base = solver.time_propagate(0, reps=5, keep_history=not args.no_adjoint, from_idle=True)
    sweep_ms = (stage_ms["propagate"] - prop_base) / sc.iters
    # the same kernel outside the step, back to back (a diagnostic beside the in-step figure)
    iso = {}
    for hist in (False, True):
        iso["history" if hist else "ping_pong"] = (solver.time_propagate(sc.iters, reps=3, keep_history=hist)
                                                   - solver.time_propagate(0, reps=5, keep_history=hist)) / sc.iters
    w16 = wdtype != "f32"
    bytes_sweep = nnz * (4 + (2 if w16 else 4)) + info["n_active"] * (16 if w16 else 12)
    achieved = bytes_sweep / (sweep_ms / 1e3) / 1e9
    peak, peak_kind = _peaks()
    traffic = _profile_traffic("sweep_f32", n) if not w16 else (
        _profile_traffic("sweep_u16", n) if wdtype == "u16" else None)
    others = {}
    if not args.no_adjoint and args.adjoint_mode == 0:
        # transposed (reverse) sweep: adjoint time after T and after 1 forward sweeps
        first_d = dev_in["first"]
        a_T = solver.time_adjoint(sc.iters, sc.spp, sc.width, sc.height, first_d)
        a_1 = solver.time_adjoint(1, sc.spp, sc.width, sc.height, first_d)
        ts_ms = (a_T - a_1) / (sc.iters - 1)
        ts_bytes = nnz * 8 + info["n_active"] * (32 if w16 else 28)
        others["tsweep_pf_kernel<%s,4>" % ("float" if not w16 else wdtype)] = {
            "launch_ms": ts_ms, "algorithmic_bytes_per_launch": ts_bytes,
            "achieved": ts_bytes / (ts_ms / 1e3) / 1e9, "frac": ts_bytes / (ts_ms / 1e3) / 1e9 / peak,
            "launches_per_step": sc.iters + 1}

    # ---- the adjoint with the HG g gradient as well (not part of the step)
    adj_g_ms = None
    if not args.no_adjoint and not args.quick:
        e2, e3 = ev(), ev()
        solver.want_g = True
        step(V, dev_in["L0"], dev_in["first"], dev_in["bg"], dev_target)
        torch.cuda.synchronize()
        step(V, dev_in["L0"], dev_in["first"], dev_in["bg"], dev_target, marks={"adjoint": (e2, e3)})
        torch.cuda.synchronize()
        adj_g_ms = e2.elapsed_time(e3)
        solver.want_g = False

    # ---- 16-bit weights: propagation rate and error against FP32 (same inputs)
    prec = {}
    if not args.quick and not w16:
        img32 = solver.last_image.clone()
        gold = _golden("cloud128") if sc.name == pgrec.CLOUD128.name and args.scale == 1.0 else None
        for wd in ("bf16", "f16", "u16"):
            s16 = pg.Solver(k=sc.k, iters=sc.iters, wdtype=wd, adjoint=False)
            s16.step(V, dev_in["L0"], dev_in["first"], dev_in["bg"], sc.spp, sc.width, sc.height, None)
            torch.cuda.synchronize()
            pb = s16.time_propagate(0, reps=5)
            pf = s16.time_propagate(sc.iters, reps=3)
            sw = (pf - pb) / sc.iters
            a = img32.double()
            b = s16.last_image.double()
            den = torch.clamp(a.abs(), min=1e-3 * float(a.abs().mean()))
            prec[wd] = {"sweep_ms": round(sw, 4), "edge_updates_per_s": nnz / (sw / 1e3),
                        "algorithmic_GBps": (nnz * (4 + 2) + info["n_active"] * 16) / (sw / 1e3) / 1e9,
                        "speedup_vs_f32": round(sweep_ms / sw, 3),
                        "max_rel_err_vs_f32": float(((a - b).abs() / den).max()),
                        "mean_rel_err_vs_f32": float(((a - b).abs() / den).mean())}
            if gold is not None:
                y0, x0, crop = gold["crop"]
                e = _pixel_err(b.cpu().numpy()[y0:y0 + crop.shape[0], x0:x0 + crop.shape[1]], crop,
                               1e-3 * np.abs(gold["stride"][1]).mean())
                prec[wd]["crop_64x64_vs_fp64_oracle"] = {"max_rel_err": float(e.max()), "mean_rel_err": float(e.mean())}
            s16.close()

    # ---- output options on the step's graph and L (not part of the step):
    # extra first-vertex emitter samples and the final gather
    outopt = {}
    if not args.quick:
        xs = pg.extra_from_records(rec)

        def t_out(reps=5, **kw):
            def f():
                return pg.pg_gather_ex(solver.graph, solver.L, solver.D, dev_in["first"], dev_in["bg"], sc.spp,
                                       sc.width, sc.height, **kw)
            img = f()
            torch.cuda.synchronize()
            a, b = ev(), ev()
            a.record(stream)
            for _ in range(reps):
                f()
            b.record(stream)
            torch.cuda.synchronize()
            return {"ms": a.elapsed_time(b) / reps,
                    "image_mean_over_path_tracer": float(img.double().mean()) / float(pt.mean())}

        outopt["gather"] = t_out()
        outopt["extra_direct_m%d" % EXTRA_M] = t_out(extra=xs)
        for kf in (8, 16, 32):
            outopt["final_gather_k%d" % kf] = t_out(final_gather_k=kf)
        outopt["final_gather_k16_extra_m%d" % EXTRA_M] = t_out(final_gather_k=16, extra=xs)

    # ---- how the output changes with the number of sweeps (the paper's study
    # of path-graph iterations): image after T sweeps against the image after
    # the step's sweep count, on the step's graph
    iter_study = None
    if not args.quick:
        Ts = [t for t in (0, 1, 2, 3, 5, 10, 15, 20, 30, 50) if t <= sc.iters]
        imgs = {}
        for T in Ts:
            L_T = pg.pg_propagate(solver.graph, dev_in["L0"], T)
            imgs[T] = pg.pg_gather(solver.graph, L_T, solver.D, dev_in["first"], dev_in["bg"], sc.spp, sc.width,
                                   sc.height).double()
        ref_img = imgs[Ts[-1]]
        den = float(ref_img.norm())
        _, res_hist, _ = pg.pg_propagate(solver.graph, dev_in["L0"], sc.iters, want_residual=True)
        iter_study = {"sweeps": Ts,
                      "image_rel_l2_change_vs_last": [float((imgs[T] - ref_img).norm()) / den for T in Ts],
                      "image_mean_over_path_tracer": [float(imgs[T].mean()) / float(pt.mean()) for T in Ts],
                      "residual_per_sweep": [float(x) for x in res_hist]}
        del imgs

    # ---- the path recorder on the GPU (not part of the step: the step starts
    # from recorded paths), against the host recorder's wall time above
    recorder = None
    if not args.quick:
        dens, alb = (torch.from_numpy(a).to(dev) for a in pgrec.medium(sc))
        scx = sc.with_(extra_direct=EXTRA_M)
        g_rec = pg.pg_record(scx, dens, alb)
        torch.cuda.synchronize()
        same = g_rec["n"] == n and bool(torch.equal(g_rec["px"].cpu(), torch.from_numpy(rec["px"])))
        del g_rec
        a, b = ev(), ev()
        a.record(stream)
        for _ in range(3):
            pg.pg_record(scx, dens, alb)
        b.record(stream)
        torch.cuda.synchronize()
        recorder = {"gpu_ms": a.elapsed_time(b) / 3, "host_s": host_trace_s, "host_threads": os.cpu_count(),
                    "vertices": n, "extra_samples_per_path": EXTRA_M, "same_records_as_host": same}

    value = total_updates / t_dev
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_dev / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": sc.name, "vertices": n, "paths": P, "k": sc.k, "iters": sc.iters,
                   "weights": wdtype, "nnz_per_sweep": nnz, "n_active": info["n_active"],
                   "sweeps_per_step": sweeps_per_step, "edge_updates_per_step": edge_updates_step,
                   "step": "build+aggregate+propagate(history)+gather" + (
                       "" if args.no_adjoint else "+adjoint(sigma_s, per-voxel albedo)"),
                   "adjoint_mode": ["transposed", "recompute", "scatter"][args.adjoint_mode],
                   "neighbourhoods": "clusters K=%d" % args.clusters if args.clusters else "kNN",
                   "l2": "inputs larger than L2 (vertex records %.0f MB > 129 MB)" % (
                       sum(int(v.numel() * v.element_size()) for v in dev_in.values()) / 1e6),
                   "parallelism": "replicas" if world > 1 else "single"},
        "stages_ms": stage_ms,
        "image_mean_over_path_tracer": solver_img_ratio,
        "adjoint_with_g_gradient_ms": adj_g_ms,
        "propagate_edge_updates_per_s": nnz / (sweep_ms / 1e3),
        "build_vertices_per_s": n / (stage_ms["build"] / 1e3),
        # two phase-function evaluations per neighbour entry in each of the two
        # aggregation passes, and two per row for the non-aggregated direct term
        "aggregate_hg_evals_per_s": (4 * info["k"] * n + 2 * n) / (stage_ms["aggregate"] / 1e3),
        # the same against the FP32 rate: about 30 floating-point operations
        # per phase-function evaluation (1 + o.d from |o + d|^2 and the
        # vectors' norm errors, the Henyey-Greenstein power with a refined
        # rsqrt); peak = 152 SMs x 128 FP32 lanes x 2 (FMA) x 2.07 GHz
        "aggregate_alu": {"bound": "alu", "flop_per_hg_eval": 30, "peak_tflops": FP32_PEAK_TFLOPS,
                          "achieved_tflops": 30 * (4 * info["k"] * n + 2 * n) / (stage_ms["aggregate"] / 1e3) / 1e12,
                          "frac": 30 * (4 * info["k"] * n + 2 * n) / (stage_ms["aggregate"] / 1e3) / 1e12
                          / FP32_PEAK_TFLOPS},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "sweep_kernel<16,%s,1024,2,2>" % wdtype if w16 else "sweep_pf_kernel<16,float,1024,1>",
                     "sweep_ms": sweep_ms, "sweep_ms_outside_step": iso,
                     "algorithmic_bytes_per_launch": bytes_sweep, "peak_kind": peak_kind,
                     "other_kernels": others},
        "precision": prec,
        "output_options_ms": outopt,
        "path_recorder": recorder,
        "iteration_study": iter_study,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk,
    }
    solver.close()
    if world == 1 and not args.quick and args.scale == 1.0 and not args.clusters and args.workload == "cloud128":
        out["configs"] = bench_configs(pg, args, peak)
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        out["cpu_baseline"] = cpu_baseline(rec, sc, args)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def _time_config(pg, sc, wdtype, dev, target, steps, warmup, adjoint, n_vox=0, peak=6800.0):
    """Times ``steps`` whole steps (graph, aggregation, sweeps, output, and
    the adjoint when ``adjoint``) of one workload on device-resident records
    ``dev``; returns the solver (holding the last step) and the record."""
    import torch

    solver = pg.Solver(k=sc.k, iters=sc.iters, wdtype=wdtype, adjoint=adjoint, want_g=False, n_vox=n_vox)
    V = pg.Vertices({k: dev[k] for k in pg.VERTEX_F32 + ("e_delta", "succ")})
    kw = dict(voxel=dev["voxel"], sigma_t=dev["sigma_t"]) if n_vox else {}

    def step(marks=None):
        return solver.step(V, dev["L0"], dev["first"], dev["bg"], sc.spp, sc.width, sc.height, target,
                           marks=marks, **kw)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    names = ["build", "aggregate", "propagate", "gather"] + (["adjoint"] if adjoint else [])
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    s = torch.cuda.current_stream()
    e0, e1 = ev(), ev()
    allm = []
    e0.record(s)
    for _ in range(steps):
        m = {nm: (ev(), ev()) for nm in names}
        step(marks=m)
        allm.append(m)
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    stage = {nm: float(np.mean([m[nm][0].elapsed_time(m[nm][1]) for m in allm])) for nm in names}
    info = solver.graph.info()
    nnz, na, n = info["nnz_swept"], info["n_active"], info["n"]
    base = solver.time_propagate(0, reps=3, keep_history=adjoint, from_idle=True)
    sweep_ms = (stage["propagate"] - base) / sc.iters
    w16 = wdtype != "f32"
    nbytes = nnz * (4 + (2 if w16 else 4)) + na * (16 if w16 else 12)
    sweeps = sc.iters * (2 if adjoint else 1)
    rec = {"workload": sc.name, "weights": wdtype, "vertices": n, "n_active": na, "k": sc.k, "iters": sc.iters,
           "nnz_per_sweep": nnz, "sweeps_per_step": sweeps, "steps": steps, "warmup": warmup,
           "step": "build+aggregate+propagate+gather" + ("+adjoint" + ("(per-voxel albedo)" if n_vox else "")
                                                         if adjoint else ""),
           "ms_per_step": ms, "edge_updates_per_s": nnz * sweeps / (ms / 1e3), "stages_ms": stage,
           "propagate_edge_updates_per_s": nnz / (sweep_ms / 1e3),
           "sweep_roofline": {"bound": "hbm", "launch_ms": sweep_ms, "algorithmic_bytes_per_launch": nbytes,
                              "achieved": nbytes / (sweep_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                              "frac": nbytes / (sweep_ms / 1e3) / 1e9 / peak},
           "build_vertices_per_s": n / (stage["build"] / 1e3)}
    return solver, rec


def bench_configs(pg, args, peak):
    """Every other workload of the method at 1 GPU, each on its own stored
    FP64 oracle values: the plain-method cube (FP32), the differentiation
    cloud (FP32, forward + adjoint with the per-voxel albedo gradient), and
    the large dense medium (U16 weights, forward + adjoint, records from the
    GPU recorder)."""
    import torch

    import pgrec

    out = {}
    dev = torch.device("cuda")
    tens = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    fields = pg.VERTEX_F32 + ("e_delta", "succ", "L0", "first", "bg", "voxel")

    # plain method: 32^3 constant cube, k = 8, 10 sweeps, FP32
    sc = pgrec.CUBE_CONST
    rec = pgrec.trace(sc)
    d = {k: tens(rec[k]) for k in fields}
    solver, r = _time_config(pg, sc, "f32", d, None, 20, 3, False, peak=peak)
    g = _golden("cube32")
    if g is not None:
        e = _pixel_err(solver.last_image.cpu().numpy(), g["image"], 1e-3 * np.abs(g["image"]).mean())
        r["image_vs_fp64_oracle"] = {"max_rel_err": float(e.max()), "mean_rel_err": float(e.mean()), "bar": 1e-5,
                                     "pixels": int(e.size)}
    solver.close()
    out["cube32"] = r
    del d

    # differentiation: 64^3 cloud, forward + adjoint, L2 loss against a seeded target render
    sc = pgrec.CLOUD64_GRAD
    rec = pgrec.trace(sc)
    d = {k: tens(rec[k]) for k in fields}
    g = _golden("cloud64")
    st = rec["sigma_t"].astype(np.float64)
    offs = g["module"].target_albedo_offsets(sc.grid_res) if g is not None else np.zeros(sc.grid_res ** 3)
    sig_t = tens(((sc.albedo + offs[rec["voxel"]]) * st).astype(np.float32))
    tsolver = pg.Solver(k=sc.k, iters=sc.iters, adjoint=False)
    Vt = pg.Vertices({**{k: d[k] for k in pg.VERTEX_F32 + ("e_delta", "succ")}, "sigma_s": sig_t})
    target = tsolver.step(Vt, d["L0"], d["first"], d["bg"], sc.spp, sc.width, sc.height).clone()
    tsolver.close()
    solver, r = _time_config(pg, sc, "f32", d, target, 10, 3, True, n_vox=sc.grid_res ** 3, peak=peak)
    if g is not None:
        img = solver.last_image.cpu().numpy()
        s_ = g["stride"]
        e = _pixel_err(img[::s_, ::s_], g["image"], 1e-3 * np.abs(g["image"]).mean())
        r["image_vs_fp64_oracle"] = {"max_rel_err": float(e.max()), "mean_rel_err": float(e.mean()), "bar": 1e-5,
                                     "pixels": int(e.size)}
        ga = solver.grads["grad_albedo"].cpu().numpy().astype(np.float64)[g["voxels"]]
        ef = _pixel_err(ga, g["fd"], 1e-3 * np.abs(g["fd"]).max())
        ea = _pixel_err(ga, g["adjoint"], 1e-3 * np.abs(g["adjoint"]).max())
        r["albedo_gradient"] = {"voxels": int(len(ga)), "bar": 1e-3,
                                "max_rel_err_vs_fp64_central_differences_h1e-3": float(ef.max()),
                                "max_rel_err_vs_fp64_oracle_adjoint": float(ea.max())}
    solver.close()
    out["cloud64_grad"] = r
    del d, target, sig_t

    # large dense medium: records from the GPU recorder, U16 weights, forward + adjoint
    sc = pgrec.CLOUD256_DENSE
    dens, alb = (torch.from_numpy(a).to(dev) for a in pgrec.medium(sc))
    d = pg.pg_record(sc, dens, alb)
    torch.cuda.synchronize()
    pt = d["pt_value"].view(sc.height, sc.width, sc.spp).mean(dim=2).float()
    target = (0.9 * pt).contiguous()
    del dens, alb
    solver, r = _time_config(pg, sc, "u16", d, target, 3, 3, True, peak=peak)
    r["records"] = "GPU path recorder (pg_record_count, pg_record_fill)"
    g = _golden("dense256")
    if g is not None:
        img = solver.last_image.cpu().numpy().astype(np.float64)
        y0, x0, crop = g["crop"]
        st_, strided = g["stride"]
        fl = 1e-3 * np.abs(strided).mean()
        e = np.concatenate([_pixel_err(img[y0:y0 + crop.shape[0], x0:x0 + crop.shape[1]], crop, fl).ravel(),
                            _pixel_err(img[::st_, ::st_], strided, fl).ravel()])
        r["image_vs_fp64_oracle"] = {"max_rel_err": float(e.max()), "mean_rel_err": float(e.mean()), "bar": 2e-3,
                                     "pixels": int(e.size), "pixels_sampled": "central 64x64 crop and every "
                                     f"{st_}th pixel"}
    solver.close()
    out["dense256"] = r
    del d, target
    torch.cuda.empty_cache()
    return out


def _golden(name):
    """Parsed stored FP64 oracle values for workload ``name`` (written by
    tests/golden/make_<name>_reference.py), or None when absent."""
    import importlib.util

    d = os.path.join(ROOT, "tests", "golden")
    path = os.path.join(d, f"make_{name}_reference.py")
    spec = importlib.util.spec_from_file_location(f"golden_{name}", path)
    mod = importlib.util.module_from_spec(spec)
    sys.path.insert(0, d)
    try:
        spec.loader.exec_module(mod)
        if not os.path.exists(mod.OUT):
            return None
        g = mod.load()
    finally:
        sys.path.remove(d)
    g["module"] = mod
    return g


def _pixel_err(got, ref, floor):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    return np.abs(got - ref) / np.maximum(np.abs(ref), floor)


def _profile_traffic(kind, n):
    """DRAM bytes per sweep launch from the committed ncu summary, if any."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(kind)
    if not e:
        return None
    # counters describe the kernel as it was compiled then: null once its source changed
    import hashlib

    src = b"".join(open(os.path.join(ROOT, "paper_2404_11894_gb300", "csrc", f), "rb").read()
                   for f in ("pg_propagate.cu", "pg_internal.cuh"))
    if hashlib.sha256(src).hexdigest() != e.get("source_sha256"):
        return None
    return e["dram_bytes_per_launch"] * (n / e["vertices"]) if e.get("scale_with_n") else e["dram_bytes_per_launch"]


# ----------------------------------------------------------------------------- oracle arm
def oracle_sample(rec, sc, stride, offset=(0, 0)):
    """Every `stride`-th pixel in x and y from pixel ``offset``, all of its paths."""
    import pgrec

    sub = pgrec.sample_pixels(rec, sc.width, sc.height, sc.spp, stride, offset)
    return sub, sub["n_paths"]


def oracle_step(sub, sc, npix, adjoint=True):
    import oracle

    t0 = time.perf_counter()
    q = oracle.quantize(sub["px"], sub["py"], sub["pz"], (0, 0, 0), (1, 1, 1))
    nbr = oracle.knn(q, sc.k)
    agg = oracle.aggregate(sub, nbr)
    L, hist, res = oracle.propagate(sub, nbr, agg["A"], agg["c"], sub["L0"], sc.iters, keep_history=adjoint)
    vals = oracle.path_values(sub, nbr, agg["A"], L, agg["D"], sub["first"], sub["bg"])
    img = vals.reshape(-1, sc.spp).mean(axis=1)
    if adjoint:
        dI = img - 0.5 * img  # any image-loss gradient of the right shape
        w = npix
        oracle.adjoint(sub, nbr, sc.iters, sub["L0"], dI.reshape(1, w), sub["first"], sub["bg"], sc.spp, w, 1)
    t = time.perf_counter() - t0
    succ = np.asarray(sub["succ"])
    has_pred = np.zeros(sub["n"], bool)
    has_pred[succ[succ >= 0]] = True
    real = (nbr >= 0) & (succ[np.where(nbr >= 0, nbr, 0)] >= 0)
    nnz = int(real[has_pred].sum())
    return t, nnz * sc.iters * (2 if adjoint else 1)


def _oracle_worker(args):
    """One host core: `reps` oracle steps of its own pixel sample."""
    os.environ["OMP_NUM_THREADS"] = "1"
    sub, sc_name, adjoint, reps = args
    import pgrec

    sc = pgrec.SCENES[sc_name]
    out = []
    for _ in range(reps):
        out.append(oracle_step(sub, sc, sub["n_paths"] // sc.spp, adjoint=adjoint))
    return out


class OraclePool:
    """The FP64 oracle on every host core: one spawned process per core, each
    running whole oracle steps on its own disjoint sample of the workload
    (every `stride`-th pixel in x and y from its own pixel offset)."""

    def __init__(self, rec, sc, stride, adjoint, cores=None):
        import multiprocessing as mp

        self.sc, self.adjoint = sc, adjoint
        self.cores = cores or os.cpu_count() or 1
        offs = [(i // stride % stride, i % stride) for i in range(self.cores)]
        self.subs = [oracle_sample(rec, sc, stride, o)[0] for o in offs]
        self.stride = stride
        self.pool = mp.get_context("spawn").Pool(self.cores)

    def step(self, reps=1):
        """Wall time of `reps` steps on every core, and the edge updates done."""
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_worker, [(s, self.sc.name, self.adjoint, reps) for s in self.subs])
        t = time.perf_counter() - t0
        return t, sum(u for r in res for _, u in r)

    def describe(self, total_paths):
        paths = sum(s["n_paths"] for s in self.subs)
        verts = sum(s["n"] for s in self.subs)
        return (f"{self.cores} disjoint samples, one per host core, each every {self.stride}th pixel in x and y "
                f"from its own offset: {paths} of {total_paths} paths ({verts} vertices) of {self.sc.name}; "
                f"whole oracle step (kNN, aggregation, {self.sc.iters} sweeps, output"
                f"{', adjoint' if self.adjoint else ''}) per sample")

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline(rec, sc, args):
    pool = OraclePool(rec, sc, args.oracle_stride, not args.no_adjoint)
    try:
        pool.step()  # warm-up: process start and imports
        t, updates = pool.step()
    finally:
        pool.close()
    return {"value": updates / t, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
            "sample": pool.describe(rec["n_paths"]) + f"; one step on all cores took {t:.1f} s"}


def run_reference(args):
    import pgrec

    rank, world, local = _dist()
    if rank != 0:
        return
    sc = pgrec.CLOUD128
    rec = pgrec.trace(sc)
    pool = OraclePool(rec, sc, args.oracle_stride, not args.no_adjoint)
    try:
        for _ in range(args.warmup):
            pool.step()
        ts, ups = [], 0
        for _ in range(args.steps):
            t, u = pool.step()
            ts.append(t)
            ups += u
    finally:
        pool.close()
    value = ups / sum(ts)
    sample = pool.describe(rec["n_paths"])
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(ts)) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": sc.name, "k": sc.k, "iters": sc.iters, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true", help="skip the 16-bit weight runs")
    ap.add_argument("--oracle-stride", type=int, default=10)
    ap.add_argument("--scale", type=float, default=1.0, help="image resolution factor (profiling only)")
    ap.add_argument("--clusters", type=int, default=0, metavar="K",
                    help="neighbourhoods from the paper's disjoint clusters of expected size K (0: kNN)")
    ap.add_argument("--workload", default="cloud128", choices=WORKLOADS,
                    help="cloud128: the headline workload; dense256: the 158.7M-vertex BF16 workload "
                         "(stage times at scale, not the headline line)")
    ap.add_argument("--weights", default=None, choices=["f32", "bf16", "f16", "u16"],
                    help="edge-weight storage of the timed step (default: the workload's own)")
    ap.add_argument("--adjoint-mode", type=int, default=0, choices=[0, 1, 2],
                    help="reverse sweep: 0 transposed copy, 1 recomputed weights, 2 atomic scatter")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
