"""Throughput of the P-Tucker row-wise ALS sweep on GB300.

Workload (the 4-order Zipf tensor): 100000 x 50000 x 30 x 24, 10^7 observed
entries, Zipf(1.1) indices on modes 1-2 and uniform on modes 3-4, values from a
planted J=(10,10,10,10) Tucker model plus N(0, 0.1^2) noise, model initialised
with U(0,1) entries, lambda = 0.01, seed 0 (synthetic; the paper's datasets are
not available).  A step is one iteration of Alg. 2: the row-wise update of all
four factor matrices (delta, Gram, FP64 row solves) plus the error pass.
Metric: observed entries x modes per second = 4 * 10^7 / (seconds per sweep).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision P] [--impl reference]

One JSON line is printed by rank 0.  With N > 1 (torchrun) every rank runs an
independent replica of the workload (weak scaling; the sweep has no exchange
step on one tensor per GPU) and the time is the maximum over ranks.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DIMS = (100_000, 50_000, 30, 24)
NNZ = 10_000_000
J = (10, 10, 10, 10)
LAM = 0.01
METRIC = "observed entries*modes/s per ALS sweep"
UNIT = "entry*modes/s"
FP32_ALU_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # FP32 lanes x FMA x max SM clock


def max_over_ranks(x: float, dist=None) -> float:
    """The job's time is the slowest rank's: all-reduce MAX (NCCL on the GPU,
    or gloo on the CPU)."""
    if dist is None:
        return x
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, units_per_rank: float, seconds: float) -> float:
    """Whole-job throughput of `world` replicas, each processing
    `units_per_rank` units, timed as the slowest rank's `seconds`."""
    return world * units_per_rank / seconds


def recorded_traffic(kernel: str, units: int):
    """DRAM bytes per launch of `kernel` from the committed ncu record, scaled
    to `units` entries; None when the kernel source changed since the capture."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[kernel]
        src = open(os.path.join(ROOT, rec["source"]), "rb").read()
    except Exception:
        return None
    if hashlib.sha256(src).hexdigest() != rec["sha256"]:
        return None
    return rec["dram_bytes_per_entry"] * units


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "fallback": True}


def workload(scale: float, seed: int = 0):
    import synth
    dims = (max(16, int(DIMS[0] * scale)), max(16, int(DIMS[1] * scale)), DIMS[2], DIMS[3])
    nnz = max(1000, int(NNZ * scale))
    t = synth.make_tensor(dims, nnz, J, dist=[("zipf", 1.1), ("zipf", 1.1), "uniform", "uniform"], seed=seed,
                          n_test=0)
    m0 = synth.init_model(dims, J, seed=seed)
    return t, m0


def serving(P, torch, precision: str, n_req: int = 3000, seed: int = 0, loads=(0.25, 0.5, 0.8, 0.95),
            max_arrival_s: float = 2.0, engine: str = "device"):
    """Fold-in serving on a 1000 x 1000 x 1000 model with J=(10,10,10): new
    mode-1 slices with log-uniform 5-5000 observed entries and 100 query
    coordinates each, values from a planted row plus N(0, 0.1^2) noise.

    engine "device": the request loop runs on the GPU (ptk_dserver_*), each
    request's latency runs from its SCHEDULED arrival time to the host seeing
    its result; "host": the host-driven batching server (ptk_server_*),
    latency from submit to result.  Saturation: all requests submitted at
    once, rate = requests / wall time.  Then Poisson arrivals at fractions of
    that rate, p50/p99 over the requests of each load."""
    import synth
    t = synth.make_tensor((1000, 1000, 1000), 1000, (10, 10, 10), seed=seed + 5, n_test=0)
    core, facs = t.planted_core, t.planted_factors
    model = P.Model.from_numpy(core, facs, dtype=torch.float32)
    reqs = synth.foldin_requests(t.dims, n_req, seed=seed, planted=(core, facs))
    if engine == "device":
        srv = P.DeviceServer(model, 0, lam=LAM, ring=4096, arena_bytes=256 << 20, max_queries=128, idle_ms=200.0)
        clock = P.DeviceServer.clock
    else:
        srv = P.Server(model, 0, lam=LAM, precision=precision, max_batch_requests=256, max_batch_entries=1 << 19,
                       max_batch_queries=256 * 100, memory_cap_bytes=1 << 30, slots=3)
        clock = time.perf_counter
    try:
        def run(schedule):
            tickets = []
            t0 = clock()
            for i, r in enumerate(reqs[:len(schedule)]):
                due = t0 + schedule[i]
                while clock() < due:
                    pass
                if engine == "device":
                    tickets.append(srv.submit(r["obs_idx"], r["obs_vals"], r["query_idx"], arrival_s=due))
                else:
                    tickets.append(srv.submit(r["obs_idx"], r["obs_vals"], r["query_idx"]))
            res = [srv.wait(tk, nq) for tk, nq in tickets]
            wall = clock() - t0
            return res, wall

        run(np.zeros(min(300, n_req)))                          # warm-up
        res, wall = run(np.zeros(n_req))
        sat = n_req / wall
        obs = sum(len(r["obs_vals"]) for r in reqs)
        sq = sum(float(np.sum((p.astype(np.float64) - r["query_vals"]) ** 2)) for (_, p, _), r in zip(res, reqs))
        ref = sum(float(np.sum(r["query_vals"].astype(np.float64) ** 2)) for r in reqs)
        out = {"workload": "fold-in of new mode-1 slices on a 1000x1000x1000 J=(10,10,10) model; "
                           "log-uniform 5-5000 observed entries + 100 queries per request",
               "engine": ("device-resident request loop (persistent CTAs polling a ring in mapped host memory)"
                          if engine == "device" else "host worker thread batching onto streams"),
               "latency_from": "scheduled arrival" if engine == "device" else "submit",
               "precision": precision if engine == "host" else "fp32 (CUDA cores)",
               "requests": n_req, "saturation_req_per_s": sat, "saturation_entries_per_s": obs / wall,
               "query_rel_rmse_vs_planted": (sq / max(ref, 1e-300)) ** 0.5, "loads": []}
        rng = np.random.default_rng(seed + 99)
        for frac in loads:
            rate = frac * sat
            n = int(min(n_req, max(200, rate * max_arrival_s)))
            sched = np.cumsum(rng.exponential(1.0 / rate, size=n))
            res, wall = run(sched)
            lat = np.array([r[2] for r in res])
            out["loads"].append({"load": frac, "offered_req_per_s": n / sched[-1], "requests": n,
                                 "served_req_per_s": n / wall, "p50_ms": float(np.percentile(lat, 50)),
                                 "p99_ms": float(np.percentile(lat, 99))})
        out["stats"] = srv.stats()
        return out
    finally:
        srv.close()


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.p = None
        # raw samples next to the run's other outputs (PTK_BENCH_OUT), else in the temp directory
        out_dir = os.environ.get("PTK_BENCH_OUT", tempfile.gettempdir())
        self.path = os.path.join(out_dir, f"clocks_bench_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.f.close()

    def summary(self):
        if self.p is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# The other paper-shaped configurations, one JSON line each (``--workload``).

FP64_PEAK_TFLOPS = 1.25   # GB300 FP64 (nominal; far below its BF16 tensor rate)


def _line(metric, value, unit, steps, warmup, ms, dtype, config, roofline, launches, clocks, **kw):
    out = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": steps, "warmup": warmup,
           "ms_per_step": ms / max(steps, 1), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": dtype, "data": "synthetic", "config": config, "roofline": roofline, "gpu_launches": launches,
           "clocks": clocks}
    out.update(kw)
    print(json.dumps(out))


def _timed_sweeps(P, torch, ctx, x, sl, model, steps, warmup, reset, **opts):
    reset()
    for _ in range(warmup):
        P.als_sweep(ctx, x, sl, model, sync_stats=False, **opts)
    torch.cuda.synchronize()
    ctx.read_timers()
    ctx.set_timing(True)
    l0 = P.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        ev0.record()
        for _ in range(steps):
            P.als_sweep(ctx, x, sl, model, sync_stats=False, **opts)
        ev1.record()
        torch.cuda.synchronize()
    ctx.set_timing(False)
    try:
        st = P.sweep_stats_read(ctx)
    except P.PtkError as e:
        st = {"rmse": float("nan"), "status": str(e)}
    return ev0.elapsed_time(ev1), P.launch_count() - l0, ctx.read_timers(), clk.summary(), st


def _slice_rate(P, torch, ctx, x, reps=3):
    """Slice layout of every mode (step a1): entries x modes per second."""
    sl = P.build_all_slices(ctx, x)
    for s in sl:
        s.close()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        sl = P.build_all_slices(ctx, x)
        torch.cuda.synchronize()
        for s in sl:
            s.close()
    el = (time.perf_counter() - t0) / reps
    return {"value": len(x.dims) * int(x.vals.shape[0]) / el, "unit": UNIT, "ms": el * 1e3,
            "note": "host-timed, includes the per-call allocation of the slice arrays"}


def workload_plain3_fp64(P, torch, args):
    """Plain P-Tucker in FP64: 3-order 1000^3, 10^5 uniform entries, planted
    J=(5,5,5) core N(0,1), factors U(0,1), sigma 0.1, lambda 0.01, 5 sweeps."""
    import synth
    t = synth.workload_plain_fp64(seed=0)
    m0 = synth.init_model(t.dims, (5, 5, 5), seed=0)
    ctx = P.Context(0)
    x = P.SparseObs.from_numpy(t.idx, t.vals, t.dims, dtype=torch.float64)
    sl = P.build_all_slices(ctx, x, dtype=torch.float64)
    model = P.Model.from_numpy(m0.core, m0.factors, dtype=torch.float64)
    init = [f.clone() for f in model.factors]

    def reset():
        for f, f0 in zip(model.factors, init):
            f.copy_(f0)

    E, N = len(t.vals), 3
    ms, launches, timers, clocks, st = _timed_sweeps(P, torch, ctx, x, sl, model, args.steps, args.warmup, reset,
                                                     precision="fp64", lam=LAM)
    # the same five sweeps through Alg. 2's driver: one eager sweep, then one
    # CUDA graph whose device-side loop runs the rest
    reset()
    P.fit(ctx, x, sl, model, precision="fp64", lam=LAM, max_sweeps=5)
    reset()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    errs = P.fit(ctx, x, sl, model, precision="fp64", lam=LAM, max_sweeps=5)
    fit_s = time.perf_counter() - t0
    d_ms, _, d_groups = timers["delta"]
    per = d_ms / max(d_groups, 1)
    flops = 2.0 * 125 * E
    ach = flops / (per / 1e3) / 1e12
    roof = {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": ach / FP64_PEAK_TFLOPS, "traffic": None, "kernel": "delta (FP64 CUDA cores)",
            "peak_source": "GB300 FP64 nominal 1.25 TFLOP/s", "delta_ms_per_launch": per}
    _line(METRIC, N * E * args.steps / (ms / 1e3), UNIT, args.steps, args.warmup, ms, "f64",
          {"workload": "plain3-fp64: 1000x1000x1000, 100000 uniform entries, J=(5,5,5), lambda=0.01, FP64",
           "l2": "inputs fit in L2 (launch-bound workload; no flush)"}, roof, launches, clocks,
          kernel_ms_per_step={k: round(v[0] / args.steps, 4) for k, v in timers.items() if v[0] > 0},
          fit_5_sweeps={"ms": fit_s * 1e3, "value": N * E * 5 / fit_s, "unit": UNIT, "errors": errs,
                        "note": "host wall time of ptk_fit (eager first sweep + one graph for sweeps 2-5)"},
          train_rmse=st["rmse"], slices=_slice_rate(P, torch, ctx, x))
    for s in sl:
        s.close()
    ctx.close()


def workload_cache1m(P, torch, args):
    """P-Tucker-Cache on the first 10^6 entries of the 4-order Zipf workload
    (Pres table 10^6 x 10^4 FP32 = 40 GB) beside plain FP32 on the same entries."""
    import synth
    t = synth.workload_zipf4(seed=0, nnz=1_000_000)
    m0 = synth.init_model(t.dims, J, seed=0)
    ctx = P.Context(0)
    x = P.SparseObs.from_numpy(t.idx, t.vals, t.dims, dtype=torch.float32)
    sl = P.build_all_slices(ctx, x)
    model = P.Model.from_numpy(m0.core, m0.factors, dtype=torch.float32)
    init = [f.clone() for f in model.factors]

    def reset():
        for f, f0 in zip(model.factors, init):
            f.copy_(f0)

    E, N, G = len(t.vals), 4, int(np.prod(J))
    ms, launches, timers, clocks, st = _timed_sweeps(P, torch, ctx, x, sl, model, args.steps, args.warmup, reset,
                                                     variant="cache", precision="fp32", lam=LAM)
    pms, _, ptimers, _, pst = _timed_sweeps(P, torch, ctx, x, sl, model, args.steps, args.warmup, reset,
                                            variant="plain", precision="fp32", lam=LAM)
    c_ms = timers["cache"][0] / args.steps
    # algorithmic bytes of the table per sweep: build writes it once; each mode
    # reads it for delta and reads + writes it in the rescale
    table = 4.0 * E * G
    bytes_sweep = table * (1 + 3 * N)
    ach = bytes_sweep / (c_ms / 1e3) / 1e9
    pk = peaks()["hbm_gbs"]
    roof = {"bound": "hbm", "achieved": ach, "peak": pk, "unit": "GB/s", "frac": ach / pk, "traffic": None,
            "kernel": "Pres table passes (build, delta, rescale)", "peak_source": "of measured",
            "algorithmic_bytes_per_sweep": bytes_sweep, "cache_ms_per_sweep": c_ms}
    _line(METRIC, N * E * args.steps / (ms / 1e3), UNIT, args.steps, args.warmup, ms, "f32",
          {"workload": "cache1m: zipf4 shape 100000x50000x30x24, first 10^6 entries, J=(10,10,10,10), "
                       "P-Tucker-Cache, FP32", "l2": "the 40 GB table exceeds L2"}, roof, launches, clocks,
          kernel_ms_per_step={k: round(v[0] / args.steps, 4) for k, v in timers.items() if v[0] > 0},
          train_rmse=st["rmse"], plain_fp32={"value": N * E * args.steps / (pms / 1e3), "unit": UNIT,
                                             "train_rmse": pst["rmse"]})
    for s in sl:
        s.close()
    ctx.close()


def workload_scal3_approx(P, torch, args):
    """Scalability: 3-order 10^7 x 10^7 x 10^7, 10^8 uniform entries, planted
    J=(10,10,10), sigma 0.1; P-Tucker-Approx removing 20 % of the core's
    non-zeros per sweep; FP32 accumulation; 10 sweeps."""
    import synth.device as sd
    dims, E, JJ = (10_000_000,) * 3, 100_000_000, (10, 10, 10)
    t = sd.make_tensor(dims, E, JJ, seed=0)
    core0, f0 = sd.init_model(dims, JJ, seed=0)
    ctx = P.Context(0)
    x = P.SparseObs(t.idx, t.vals, dims)
    sl_info = _slice_rate(P, torch, ctx, x, reps=1)
    sl = P.build_all_slices(ctx, x)
    model = P.Model.from_numpy(core0, f0, dtype=torch.float32)
    core_init = model.core.clone()
    init = [f.clone() for f in model.factors]

    def reset():
        model.core.copy_(core_init)
        for f, fi in zip(model.factors, init):
            f.copy_(fi)

    out = {}
    for rule in ("magnitude", "r_beta"):
        ms, launches, timers, clocks, st = _timed_sweeps(
            P, torch, ctx, x, sl, model, args.steps, args.warmup, reset, variant="approx", precision=args.scal_precision,
            lam=LAM, trunc_rate=0.2, trunc_rule=rule)
        out[rule] = (ms, launches, timers, clocks, st, int(torch.count_nonzero(model.core)))
    ms, launches, timers, clocks, st, nnzg = out["magnitude"]
    N = 3
    d_ms, _, d_groups = timers["delta"]
    per = d_ms / max(d_groups, 1)
    # delta reads the entry (3 int32 + value) and gathers two factor rows of
    # 40 B (64 B rows at sector granularity), writes J+1 values padded to 12
    bytes_launch = E * (16 + 2 * 64 + 48)
    ach = bytes_launch / (per / 1e3) / 1e9
    pk = peaks()["hbm_gbs"]
    roof = {"bound": "hbm", "achieved": ach, "peak": pk, "unit": "GB/s", "frac": ach / pk, "traffic": None,
            "kernel": "delta", "peak_source": "of measured", "algorithmic_bytes_per_launch": bytes_launch,
            "delta_ms_per_launch": per}
    rb = out["r_beta"]
    _line(METRIC, N * E * args.steps / (ms / 1e3), UNIT, args.steps, args.warmup, ms,
          {"fp32": "f32", "bf16": "bf16", "tf32": "tf32", "bf16x3": "bf16x3"}[args.scal_precision],
          {"workload": "scal3-approx: 10^7 x 10^7 x 10^7, 10^8 uniform entries, J=(10,10,10), P-Tucker-Approx "
                       "p=0.2 per sweep (smallest |G| rule)", "l2": "inputs larger than L2 (5.6 GB of factors "
                                                                 "and entries)"},
          roof, launches, clocks,
          kernel_ms_per_step={k: round(v[0] / args.steps, 4) for k, v in timers.items() if v[0] > 0},
          train_rmse=st["rmse"], core_nnz_after=nnzg, slices=sl_info,
          r_beta_rule={"value": N * E * args.steps / (rb[0] / 1e3), "unit": UNIT, "train_rmse": rb[4]["rmse"],
                       "core_nnz_after": rb[5],
                       "kernel_ms_per_step": {k: round(v[0] / args.steps, 4) for k, v in rb[2].items() if v[0] > 0}})
    for s in sl:
        s.close()
    ctx.close()


def workload_batched512(P, torch, args):
    """512 independent tensors: order U{3,4,5}, mode sizes log-uniform in
    10^2..10^5, nnz log-uniform in 10^4..5*10^6, J uniform in 3..16, planted
    models plus noise sigma 0.1; factorised together by ptk_fit."""
    import synth
    import synth.device as sd
    shapes = synth.batched_shapes(args.batch_count, seed=0)
    ctx = P.Context(0)
    probs, inits = [], []
    for sh in shapes:
        t = sd.make_tensor(sh["dims"], sh["nnz"], sh["J"], seed=sh["seed"])
        c0, f0 = sd.init_model(sh["dims"], sh["J"], seed=sh["seed"])
        x = P.SparseObs(t.idx, t.vals, sh["dims"])
        sl = P.build_all_slices(ctx, x)
        model = P.Model.from_numpy(c0, f0, dtype=torch.float32)
        probs.append((x, sl, model))
        inits.append([f.clone() for f in model.factors])
        del t
    torch.cuda.synchronize()

    def reset():
        for (_, _, m), init in zip(probs, inits):
            for f, fi in zip(m.factors, init):
                f.copy_(fi)

    work = sum(len(x.dims) * int(x.vals.shape[0]) for x, _, _ in probs)
    S = args.steps
    reset()
    tt = time.perf_counter()
    P.fit_many(ctx, probs, precision=args.batch_precision, lam=LAM, max_sweeps=1, lanes=args.lanes,
               autotune=not args.no_autotune)   # warm-up (and the launch-shape tuning of every class)
    warm_s = time.perf_counter() - tt
    reset()
    torch.cuda.synchronize()
    l0 = P.launch_count()
    with ClockSampler(torch.cuda.current_device()) as clk:
        t0 = time.perf_counter()
        errs = P.fit_many(ctx, probs, precision=args.batch_precision, lam=LAM, max_sweeps=S, lanes=args.lanes)
        el = time.perf_counter() - t0
    launches = P.launch_count() - l0
    # one problem at a time, eagerly, for comparison (the first 64 problems)
    sub = probs[:64]
    reset()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    P.fit_many(ctx, sub, precision=args.batch_precision, lam=LAM, max_sweeps=S, lanes=1, graphs=False)
    el_seq = time.perf_counter() - t0
    reset()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    P.fit_many(ctx, sub, precision=args.batch_precision, lam=LAM, max_sweeps=S, lanes=args.lanes)
    el_sub = time.perf_counter() - t0
    sub_work = sum(len(x.dims) * int(x.vals.shape[0]) for x, _, _ in sub)
    total_flops = sum(len(x.dims) * int(x.vals.shape[0]) * 2.0 * int(np.prod(m.J)) for x, _, m in probs) * S
    ach = total_flops / el / 1e12
    roof = {"bound": "alu", "achieved": ach,
            "peak": FP32_ALU_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": ach / FP32_ALU_PEAK_TFLOPS, "traffic": None,
            "kernel": "whole fit (delta flops 2|G| per entry and mode over the wall time); the largest cores "
                      "run on CUDA cores at any precision",
            "peak_source": "FP32 CUDA-core peak: 152 SMs x 128 lanes x 2 flop x 2.07 GHz"}
    _line(METRIC, work * S / el, UNIT, S, 1, el * 1e3, args.batch_precision,
          {"workload": f"batched{len(probs)}: order 3-5, I_n log-uniform 1e2-1e5, nnz log-uniform 1e4-5e6 "
                       f"(total {sum(int(x.vals.shape[0]) for x, _, _ in probs)}), J uniform 3-16",
           "l2": "inputs larger than L2", "lanes": args.lanes},
          roof, launches, clk.summary(), final_errors_first8=[e[-1] for e in errs[:8]],
          warmup_fit_s=warm_s, autotuned=not args.no_autotune,
          first64={"batched_lanes_graphs": sub_work * S / el_sub, "one_at_a_time_eager": sub_work * S / el_seq,
                   "unit": UNIT})
    for _, sl, _ in probs:
        for s in sl:
            s.close()
    ctx.close()


def _sweep_ms(P, torch, ctx, x, sl, model, init, reps, **opts):
    """Mean device time of one sweep (after one warm-up), with the model reset first."""
    for f, f0 in zip(model.factors, init):
        f.copy_(f0)
    P.als_sweep(ctx, x, sl, model, sync_stats=False, **opts)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(reps):
        P.als_sweep(ctx, x, sl, model, sync_stats=False, **opts)
    ev1.record()
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / reps


def workload_tradeoff(P, torch, args):
    """The paper's variant trade-off on the GPU: P-Tucker vs P-Tucker-Cache
    across tensor orders (I_n = 100, 1000 entries, J = 3 per mode, orders 3-8)
    and across ranks (4-order 100000 x 50000 x 30 x 24 Zipf shape, 10^6
    entries, J = 3..11)."""
    import synth
    ctx = P.Context(0)
    order_rows, rank_rows = [], []
    for N in range(3, 9):
        dims, J = (100,) * N, (3,) * N
        t = synth.make_tensor(dims, 1000, J, seed=N, n_test=0)
        m0 = synth.init_model(dims, J, seed=N)
        x = P.SparseObs.from_numpy(t.idx, t.vals, dims, dtype=torch.float32)
        sl = P.build_all_slices(ctx, x)
        model = P.Model.from_numpy(m0.core, m0.factors, dtype=torch.float32)
        init = [f.clone() for f in model.factors]
        row = {"order": N}
        for variant in ("plain", "cache"):
            ms = _sweep_ms(P, torch, ctx, x, sl, model, init, 20, variant=variant, precision="fp32", lam=LAM)
            row[variant + "_ms"] = ms
            row[variant + "_entry_modes_per_s"] = N * 1000 / (ms / 1e3)
        order_rows.append(row)
        for q in sl:
            q.close()
    for Jr in (3, 5, 7, 9, 11):
        J4 = (Jr,) * 4
        t = synth.workload_zipf4(seed=0, nnz=1_000_000)
        m0 = synth.init_model(t.dims, J4, seed=0)
        x = P.SparseObs.from_numpy(t.idx, t.vals, t.dims, dtype=torch.float32)
        sl = P.build_all_slices(ctx, x)
        model = P.Model.from_numpy(m0.core, m0.factors, dtype=torch.float32)
        init = [f.clone() for f in model.factors]
        row = {"J": Jr}
        for variant, prec in (("plain", "fp32"), ("plain", "bf16"), ("cache", "fp32")):
            if prec == "bf16" and not P.tc_available(model, "bf16"):
                continue
            ms = _sweep_ms(P, torch, ctx, x, sl, model, init, 3, variant=variant, precision=prec, lam=LAM)
            row[f"{variant}_{prec}_ms"] = ms
        rank_rows.append(row)
        for q in sl:
            q.close()
    ctx.close()
    print(json.dumps({"metric": "ms per ALS sweep (variant trade-off)", "workload": "tradeoff", "data": "synthetic",
                      "orders": order_rows, "ranks": rank_rows}))


def approx_curve_data(P, torch, sweeps):
    """Per-sweep device time (CUDA events), error and core size of
    P-Tucker-Approx (both selection rules, p = 0.2) and of plain P-Tucker,
    FP32, on 10^6 entries of the 4-order Zipf shape."""
    import synth
    t = synth.workload_zipf4(seed=0, nnz=1_000_000)
    m0 = synth.init_model(t.dims, J, seed=0)
    ctx = P.Context(0)
    x = P.SparseObs.from_numpy(t.idx, t.vals, t.dims, dtype=torch.float32)
    sl = P.build_all_slices(ctx, x)
    out = {}
    for name, opts in (("plain", dict(variant="plain")), ("approx_r_beta", dict(variant="approx", trunc_rule="r_beta")),
                       ("approx_magnitude", dict(variant="approx", trunc_rule="magnitude"))):
        model = P.Model.from_numpy(m0.core, m0.factors, dtype=torch.float32)
        curve = []
        for s in range(sweeps):
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record()
            st = P.als_sweep(ctx, x, sl, model, precision="fp32", lam=LAM, trunc_rate=0.2, **opts)
            ev1.record()
            torch.cuda.synchronize()
            curve.append({"sweep": s + 1, "ms": ev0.elapsed_time(ev1), "error": st["error"],
                          "core_nnz": st["core_nnz"]})
        out[name] = curve
    for q in sl:
        q.close()
    ctx.close()
    return out


def workload_approx_curve(P, torch, args):
    """Per-sweep time, error and core size of P-Tucker-Approx against plain
    P-Tucker over --steps sweeps (the paper stops at 20): the paper's
    time-per-iteration comparison."""
    print(json.dumps({"metric": "per-sweep time and error (Approx vs plain)", "workload": "approx-curve",
                      "data": "synthetic", "curves": approx_curve_data(P, torch, args.steps)}))


def other_configs(P, torch):
    """Compact measurements of two further configurations, for the headline
    line: plain P-Tucker in FP64 (3-order, 10^5 entries; 20 timed sweeps)
    and the Approx time-per-sweep curve (20 sweeps, both rules)."""
    import synth
    t = synth.workload_plain_fp64(seed=0)
    m0 = synth.init_model(t.dims, (5, 5, 5), seed=0)
    ctx = P.Context(0)
    x = P.SparseObs.from_numpy(t.idx, t.vals, t.dims, dtype=torch.float64)
    sl = P.build_all_slices(ctx, x, dtype=torch.float64)
    model = P.Model.from_numpy(m0.core, m0.factors, dtype=torch.float64)
    init = [f.clone() for f in model.factors]

    def reset():
        for f, f0 in zip(model.factors, init):
            f.copy_(f0)

    steps, E = 20, len(t.vals)
    ms, _, timers, _, st = _timed_sweeps(P, torch, ctx, x, sl, model, steps, 3, reset, precision="fp64", lam=LAM)
    plain3 = {"workload": "plain3-fp64: 1000x1000x1000, 100000 uniform entries, J=(5,5,5), lambda=0.01, FP64",
              "value": 3 * E * steps / (ms / 1e3), "unit": UNIT, "ms_per_sweep": ms / steps,
              "kernel_ms_per_sweep": {k: round(v[0] / steps, 4) for k, v in timers.items() if v[0] > 0},
              "train_rmse": st["rmse"]}
    for q in sl:
        q.close()
    ctx.close()
    curves = approx_curve_data(P, torch, 20)
    approx = {"workload": "approx-curve: zipf4 shape, 1000000 entries, J=(10,10,10,10), FP32, p=0.2, 20 sweeps",
              "sweep_ms": {k: [round(c["ms"], 3) for c in v] for k, v in curves.items()},
              "core_nnz_after": {k: [c["core_nnz"] for c in v] for k, v in curves.items()},
              "error_after": {k: [round(c["error"], 2) for c in v] for k, v in curves.items()},
              "note": "device time of each sweep (CUDA events); the first sweep includes one-time set-up"}
    return {"plain3_fp64": plain3, "approx_curve": approx}


def workload_schedule(P, torch, args):
    """Sec. 3.4's scheduling question on the GPU: the row sums B_i, c_i with
    the work split by entries (the default) against one warp per row, the rows
    dealt statically (row r to warp r mod W) or dynamically (a shared counter),
    and the default choice between them per mode ("auto").
    Two inputs: the 4-order Zipf workload (10^7 entries; the largest mode-1 row
    holds about 13 % of them, modes 3 and 4 have 30 and 24 rows) and a uniform
    3-order tensor (10^6 rows per mode, 10^7 entries, about 10 per row).  BF16
    delta; device time per sweep and of the Gram step."""
    import synth
    ctx = P.Context(0)
    steps = max(1, min(args.steps, 5))
    cases = []
    t, m0 = workload(args.scale)
    cases.append(("zipf4", t, m0))
    du = (1_000_000,) * 3
    tu = synth.make_tensor(du, int(10_000_000 * args.scale), (10, 10, 10), seed=1, n_test=0)
    cases.append(("uniform3", tu, synth.init_model(du, (10, 10, 10), seed=1)))
    out = []
    for name, t, m0 in cases:
        x = P.SparseObs.from_numpy(t.idx, t.vals, t.dims, dtype=torch.float32)
        sl = P.build_all_slices(ctx, x)
        model = P.Model.from_numpy(m0.core, m0.factors, dtype=torch.float32)
        init = [f.clone() for f in model.factors]
        prec = "bf16" if P.tc_available(model, "bf16") else "fp32"

        def reset():
            for f, f0 in zip(model.factors, init):
                f.copy_(f0)

        row = {"workload": name, "dims": list(t.dims), "entries": int(len(t.vals)), "precision": prec,
               "largest_row_share": [float(np.bincount(t.idx[:, k]).max() / len(t.vals)) for k in range(len(t.dims))]}
        for sched in ("auto", "entries", "rows_static", "rows_dynamic"):
            ms, launches, tim, clk, st = _timed_sweeps(P, torch, ctx, x, sl, model, steps, 1, reset, precision=prec,
                                                       lam=LAM, schedule=sched)
            row[sched] = {"sweep_ms": ms / steps, "gram_ms": tim["gram"][0] / steps,
                          "entry_modes_per_s": len(t.dims) * len(t.vals) / (ms / steps / 1e3),
                          "train_rmse": st.get("rmse"), "clocks": clk}
        for sched in ("rows_static", "rows_dynamic"):
            row[sched]["gram_slowdown_vs_entries"] = row[sched]["gram_ms"] / row["entries"]["gram_ms"]
        out.append(row)
        for q in sl:
            q.close()
    ctx.close()
    print(json.dumps({"metric": "ms per ALS sweep and per Gram step by work split", "workload": "schedule",
                      "data": "synthetic", "steps": steps, "cases": out}))


WORKLOADS = {"plain3-fp64": workload_plain3_fp64, "cache1m": workload_cache1m, "scal3-approx": workload_scal3_approx,
             "batched512": workload_batched512, "tradeoff": workload_tradeoff, "approx-curve": workload_approx_curve,
             "schedule": workload_schedule}


# ---------------------------------------------------------------------------
TEST_RMSE_DIMS, TEST_RMSE_NNZ, TEST_RMSE_SWEEPS, TEST_RMSE_TOL = (600, 400, 30, 24), 40_000, 2, 0.005


def heldout_rmse_vs_oracle(P, torch, precision: str, seed: int = 0):
    """Held-out RMSE of `precision` against the FP64 oracle's after the same
    sweeps from the same initialisation, on the zipf4 recipe (Zipf 1.1 on
    modes 1-2, J = 10, sigma 0.1) scaled down so that the oracle's sweeps take
    seconds: 600x400x30x24, 40k training and 4k held-out entries."""
    import oracle
    import synth
    dims, E = TEST_RMSE_DIMS, TEST_RMSE_NNZ
    t = synth.make_tensor(dims, E, J, dist=[("zipf", 1.1), ("zipf", 1.1), "uniform", "uniform"], seed=seed,
                          n_test=E // 10)
    m0 = synth.init_model(dims, J, seed=seed)
    f32 = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)  # noqa: E731
    core, F0, vals = f32(m0.core), [f32(a) for a in m0.factors], f32(t.vals)
    ctx = P.Context(torch.cuda.current_device())
    x = P.SparseObs.from_numpy(t.idx, vals, dims, dtype=torch.float32)
    sl = P.build_all_slices(ctx, x)
    model = P.Model.from_numpy(core, F0, dtype=torch.float32)
    Fr = F0
    s0 = time.perf_counter()
    for _ in range(TEST_RMSE_SWEEPS):
        P.als_sweep(ctx, x, sl, model, precision=precision, lam=LAM)
        Fr, _ = oracle.sweep(dims, core, Fr, t.idx, vals, LAM, nthreads=oracle.max_threads())
    xt = P.SparseObs.from_numpy(t.test_idx, t.test_vals, dims, dtype=torch.float32)
    got = P.error(ctx, xt, model, LAM)["rmse"]
    ref = oracle.error_stats(core, Fr, t.test_idx, t.test_vals)["rmse"]
    for q in sl:
        q.close()
    ctx.close()
    rel = (got - ref) / ref
    return {"precision": precision, "test_rmse": got, "oracle_test_rmse": ref, "rel_err": rel,
            "tolerance": TEST_RMSE_TOL, "within_tolerance": abs(rel) <= TEST_RMSE_TOL,
            "sample": f"zipf4 recipe at {dims[0]}x{dims[1]}x{dims[2]}x{dims[3]}, {E} training and {E // 10} held-out "
                      f"entries, {TEST_RMSE_SWEEPS} sweeps from the same U(0,1) initialisation (FP32-rounded), "
                      f"oracle in FP64 on {oracle.max_threads()} host threads",
            "seconds": round(time.perf_counter() - s0, 1)}


def cpu_oracle_rate(t, m0, target_s: float, max_entries: int | None = None):
    """Times the FP64 oracle's sweep on a bounded prefix of the entries with all
    host cores; returns (entry*modes/s, cores, sample description)."""
    import oracle
    cores = oracle.max_threads()
    N = len(t.dims)
    # calibrate on a small prefix
    e0 = min(len(t.vals), 2000)
    s = time.perf_counter()
    oracle.sweep(t.dims, m0.core, m0.factors, t.idx[:e0], t.vals[:e0], LAM, nthreads=cores)
    dt = max(time.perf_counter() - s, 1e-3)
    E = int(min(len(t.vals), max(e0, e0 * target_s / dt)))
    if max_entries:
        E = min(E, max_entries)
    s = time.perf_counter()
    oracle.sweep(t.dims, m0.core, m0.factors, t.idx[:E], t.vals[:E], LAM, nthreads=cores)
    el = time.perf_counter() - s
    return N * E / el, cores, f"one FP64 oracle sweep (all {N} modes) over the first {E} of the {len(t.vals)} " \
                              f"entries, {cores} OpenMP threads, {el:.1f} s"


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    t, m0 = workload(args.scale)
    N = len(t.dims)
    import oracle
    cores = oracle.max_threads()
    # each step: one oracle sweep over a bounded prefix, sized so that the
    # whole run (warm-up and timed steps) takes about two minutes at most
    step_s = min(args.ref_step_s, 120.0 / max(1, args.steps + args.warmup))
    e0 = min(len(t.vals), 2000)
    s = time.perf_counter()
    oracle.sweep(t.dims, m0.core, m0.factors, t.idx[:e0], t.vals[:e0], LAM, nthreads=cores)
    dt = max(time.perf_counter() - s, 1e-3)
    E = int(min(len(t.vals), max(e0, e0 * step_s / dt)))
    for _ in range(args.warmup):
        oracle.sweep(t.dims, m0.core, m0.factors, t.idx[:E], t.vals[:E], LAM, nthreads=cores)
    s = time.perf_counter()
    for _ in range(args.steps):
        oracle.sweep(t.dims, m0.core, m0.factors, t.idx[:E], t.vals[:E], LAM, nthreads=cores)
    el = time.perf_counter() - s
    value = N * E * args.steps / el
    sample = f"each step: one FP64 oracle sweep over the first {E} of {len(t.vals)} entries, {cores} threads"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"zipf4: {t.dims[0]}x{t.dims[1]}x{t.dims[2]}x{t.dims[3]}, {len(t.vals)} entries "
                               f"(Zipf 1.1 on modes 1-2), J=(10,10,10,10), lambda={LAM}, plain P-Tucker, FP64 oracle "
                               f"on a prefix of the entries per step",
                   "parallelism": "host cores"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=260)  # about 1 s of timed sweeps
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="auto", choices=["auto", "fp32", "tf32", "bf16", "bf16x3"])
    ap.add_argument("--scale", type=float, default=1.0, help="shrink the workload (tests only)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-target-s", type=float, default=12.0)
    ap.add_argument("--ref-step-s", type=float, default=6.0)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-side", action="store_true", help="skip the other configurations' summaries")
    ap.add_argument("--accuracy-sweeps", type=int, default=5)
    ap.add_argument("--serve-precision", default="fp32", choices=["fp32", "tf32", "bf16", "bf16x3"])
    ap.add_argument("--serve-requests", type=int, default=3000)
    ap.add_argument("--workload", default="zipf4", choices=["zipf4"] + list(WORKLOADS))
    ap.add_argument("--scal-precision", default="fp32", choices=["fp32", "tf32", "bf16", "bf16x3"])
    ap.add_argument("--batch-precision", default="fp32", choices=["fp32", "tf32", "bf16", "bf16x3"])
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--lanes", type=int, default=8)
    ap.add_argument("--no-autotune", action="store_true")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        return reference_arm(args)

    import torch
    if args.workload != "zipf4":
        import paper_1710_02261_gb300 as P
        torch.cuda.set_device(0)
        return WORKLOADS[args.workload](P, torch, args)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_1710_02261_gb300 as P

    t, m0 = workload(args.scale, seed=rank)
    N = len(t.dims)
    E = len(t.vals)
    ctx = P.Context(local)
    x = P.SparseObs.from_numpy(t.idx, t.vals, t.dims, dtype=torch.float32)
    sl = P.build_all_slices(ctx, x)
    model = P.Model.from_numpy(m0.core, m0.factors, dtype=torch.float32)
    init_state = [f.clone() for f in model.factors]
    precision = args.precision
    if precision == "auto":
        # BF16x3 on the tensor cores (FP32 operands as BF16 high + low parts):
        # the delta that keeps the held-out RMSE within 0.5 % of the FP64
        # oracle's on Zipf-tailed data with a wide margin (0.01 %); a BF16
        # delta moves the one- and two-entry tail rows by a few %, a TF32 one
        # by up to 0.6 % depending on the seed
        precision = "bf16x3" if P.tc_available(model, "bf16x3") else "fp32"

    def reset():
        for f, f0 in zip(model.factors, init_state):
            f.copy_(f0)

    def step(prec):
        P.als_sweep(ctx, x, sl, model, precision=prec, lam=LAM, error_pass=True, sync_stats=False)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    def timed(prec, steps, warmup, soak_s=0.0):
        """W warm-up steps, then exactly `steps` timed steps (CUDA events on
        this stream, barrier + synchronize on both sides).  With soak_s > 0 the
        clock sampler also covers soak_s seconds of the same steps before and
        after the timed ones (untimed), so that it sees the clocks under this
        load for longer than one short timed window."""
        reset()
        for _ in range(warmup):
            step(prec)
        barrier()
        pre = post = 0
        if soak_s > 0:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(3):
                step(prec)
            e1.record()
            torch.cuda.synchronize()
            est = max(e0.elapsed_time(e1) / 3.0, 1e-3)
            pre = post = int(math.ceil(soak_s * 1e3 / est))
        ctx.read_timers()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            for _ in range(pre):
                step(prec)
            barrier()
            ctx.set_timing(True)
            l0 = P.launch_count()
            ev0.record()
            for _ in range(steps):
                step(prec)
            ev1.record()
            barrier()
            launches = P.launch_count() - l0
            ctx.set_timing(False)
            for _ in range(post):
                step(prec)
            torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        ms = max_over_ranks(ms, dist)
        timers = ctx.read_timers()
        summ = clk.summary()
        summ["window"] = f"sampled over {pre} + {steps} + {post} steps (untimed soak, timed, untimed soak)"
        return ms, launches, timers, summ

    ms, launches, timers, clocks = timed(precision, args.steps, args.warmup, soak_s=0.6)
    try:
        stats = P.sweep_stats_read(ctx)
    except P.PtkError as e:  # report, do not hide, rows whose system was not positive definite
        stats = {"rmse": float("nan"), "status": str(e)}
    value = job_throughput(world, N * E * args.steps, ms / 1e3)
    gsize = int(np.prod(J))
    # dominant kernel: the delta contraction (Eq. delta), 2|G| algorithmic flops per entry and mode
    d_ms, d_launch, d_groups = timers["delta"]
    per_launch_ms = d_ms / max(d_groups, 1)
    flops_per_launch = 2.0 * gsize * E
    achieved_tflops = flops_per_launch / (per_launch_ms / 1e3) / 1e12
    pk = peaks()
    if precision in ("bf16", "tf32", "bf16x3"):
        peak = pk["bf16_tflops"] * (0.5 if precision == "tf32" else 1.0)
        bound, peak_note = "tensor", ("of measured" + (" (bf16 x 0.5 nominal tf32 ratio)" if precision == "tf32"
                                                        else "") +
                                      (" (three BF16 MMAs per product; algorithmic flops counted once)"
                                       if precision == "bf16x3" else ""))
    else:
        peak, bound = FP32_ALU_PEAK_TFLOPS, "alu"
        peak_note = "FP32 CUDA-core peak: 152 SMs x 128 lanes x 2 flop x 2.07 GHz"
    traffic = recorded_traffic({"bf16": "delta_tc_kernel<10,2,bf16>", "tf32": "delta_tc_kernel_tm<10,2,tf32>",
                                "bf16x3": "delta_tc_kernel_tm<10,2,bf16x3>"}.get(precision, ""), E)
    roof_delta = {"bound": bound, "achieved": achieved_tflops, "peak": peak, "unit": "TFLOP/s",
                  "frac": achieved_tflops / peak, "traffic": traffic, "kernel": "delta", "peak_source": peak_note,
                  "delta_ms_per_launch": per_launch_ms, "algorithmic_flops_per_launch": flops_per_launch,
                  "traffic_note": "DRAM bytes per launch from the ncu capture in profiles/ (3e6 entries) scaled by "
                                  "entries; a lower bound (the tail of Delta stays in L2)" if traffic else None}
    if precision in ("bf16", "tf32", "bf16x3"):
        kq = 8 if precision == "tf32" else 16
        rup = lambda v, q: (v + q - 1) // q * q  # noqa: E731
        n_mma, k_mma = rup(J[0] * J[0], 16), rup(J[0] ** (len(J) - 2), kq)
        products = 3 if precision == "bf16x3" else 1
        mma_flops = 2.0 * n_mma * k_mma * products * E  # M = 128 entries per tile: per entry N x K x 2
        roof_delta["mma_issued_tflops"] = mma_flops / (per_launch_ms / 1e3) / 1e12
        roof_delta["mma_issued_frac"] = roof_delta["mma_issued_tflops"] / peak
        roof_delta["mma_note"] = ("tensor-pipe work the MMAs issue (N = J_n J_L and the K-group width padded to "
                                  "the instruction shape, " + ("three BF16 products per algorithmic one"
                                  if products == 3 else "one product") + ") per launch time")
    # the row sums B_i, c_i (Eqs. rowB, rowC), bound by HBM: per launch (one
    # mode) the Delta rows [delta, x] are read once (4 (J + 1) bytes per entry)
    # and every row's J(J+1)/2 + J sums are written once as FP64
    g_ms, _, g_groups = timers["gram"]
    g_per_launch = g_ms / max(g_groups, 1)
    nout = J[0] * (J[0] + 1) // 2 + J[0]
    g_bytes = 4.0 * (J[0] + 1) * E + 8.0 * nout * float(np.mean(t.dims))
    g_gbs = g_bytes / (g_per_launch / 1e3) / 1e9
    roof_gram = {"bound": "hbm", "achieved": g_gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                 "frac": g_gbs / pk["hbm_gbs"], "traffic": recorded_traffic("gram_tc_kernel<10,3>", E),
                 "kernel": "row sums (tensor-core chunks of the long rows + row-per-warp short rows, one mode)",
                 "peak_source": "of measured (MEASURED_PEAKS.json hbm_gbs)",
                 "gram_ms_per_launch": g_per_launch, "algorithmic_bytes_per_launch": g_bytes,
                 "traffic_note": "DRAM bytes per entry of the committed ncu capture (mode 1 of the workload at 0.3 "
                                 "scale) times the entries; below the algorithmic bytes because part of Delta is "
                                 "still in L2 from the delta kernel"}
    # `roofline` is the kernel group with the larger device time in the timed sweeps
    if g_ms > d_ms:
        roofline, roofline_other = roof_gram, roof_delta
    else:
        roofline, roofline_other = roof_delta, roof_gram
    kernel_ms = {k: round(v[0] / max(args.steps, 1), 4) for k, v in timers.items() if v[0] > 0}

    # plain FP32 form beside the tensor-core form ("vs plain FP32")
    plain = None
    if precision != "fp32":
        pms, _, _, _ = timed("fp32", max(2, args.steps // 2), 3)
        plain = {"value": world * N * E * max(2, args.steps // 2) / (pms / 1e3), "unit": UNIT}

    # accuracy at equal work: training RMSE after the same sweeps from the same
    # initialisation, each precision against the FP32 CUDA-core form
    accuracy = None
    if not args.no_accuracy:
        accuracy = {"sweeps": args.accuracy_sweeps}
        for prec in ["fp32"] + [q for q in ("bf16", "bf16x3", "tf32") if q != "fp32"]:
            if prec != "fp32" and not P.tc_available(model, prec):
                continue
            reset()
            for _ in range(args.accuracy_sweeps):
                step(prec)
            try:
                accuracy[prec] = P.sweep_stats_read(ctx)["rmse"]
            except P.PtkError as e:
                accuracy[prec] = str(e)
        ref = accuracy["fp32"]
        accuracy["rel_diff_vs_fp32"] = {q: (accuracy[q] - ref) / ref for q in ("bf16", "bf16x3", "tf32")
                                        if isinstance(accuracy.get(q), float)}

    # the timed precision against the FP64 oracle on held-out coordinates
    test_rmse = None
    if not args.no_accuracy and rank == 0:
        test_rmse = heldout_rmse_vs_oracle(P, torch, precision)

    # end to end through the C ABI from pinned host buffers
    e2e = None
    if not args.no_e2e:
        import paper_1710_02261_gb300 as P2
        idx_h = torch.from_numpy(t.idx).pin_memory()
        val_h = torch.from_numpy(t.vals.astype(np.float32)).pin_memory()
        idx_d = torch.empty_like(idx_h, device="cuda")
        val_d = torch.empty_like(val_h, device="cuda")
        e2e_steps = max(2, args.steps // 2)

        def e2e_step():
            idx_d.copy_(idx_h, non_blocking=True)
            val_d.copy_(val_h, non_blocking=True)
            xx = P2.SparseObs(idx_d, val_d, t.dims)
            ss = P2.build_all_slices(ctx, xx)
            P2.als_sweep(ctx, xx, ss, model, precision=precision, lam=LAM, error_pass=True, sync_stats=False)
            try:
                st = P2.sweep_stats_read(ctx)
            except P2.PtkError as e:
                st = {"status": str(e)}
            for q in ss:
                q.close()
            return st

        reset()
        for _ in range(2):
            e2e_step()
        barrier()
        s0 = time.perf_counter()
        for _ in range(e2e_steps):
            e2e_step()
        barrier()
        el = time.perf_counter() - s0
        el = max_over_ranks(el, dist)
        e2e = {"value": world * N * E * e2e_steps / el, "unit": UNIT,
               "h2d_bytes_per_step": int(idx_h.numel() * 4 + val_h.numel() * 4),
               "d2h_bytes_per_step": 48, "includes": "H2D of the entries, slice layout of all modes, sweep, "
                                                     "error statistics read back"}

    serve = serve_host = None
    if not args.no_serving:
        serve = serving(P, torch, args.serve_precision, n_req=args.serve_requests, seed=rank, engine="device")
        serve_host = serving(P, torch, args.serve_precision, n_req=args.serve_requests, seed=rank, engine="host")
    side = other_configs(P, torch) if rank == 0 and world == 1 and not args.no_side else None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, sample = cpu_oracle_rate(t, m0, args.cpu_target_s)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp32": "f32", "bf16": "bf16", "tf32": "tf32", "bf16x3": "bf16x3"}[precision],
            "data": "synthetic",
            "config": {"workload": f"zipf4: {t.dims[0]}x{t.dims[1]}x{t.dims[2]}x{t.dims[3]}, {E} entries "
                                   f"(Zipf 1.1 on modes 1-2), J=(10,10,10,10), lambda={LAM}, plain P-Tucker, "
                                   f"delta precision {precision}, FP64 row solves",
                       "l2": "inputs larger than L2 (slice-ordered entries and Delta of a mode exceed 129 MB)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": roofline, "roofline_other": roofline_other, "kernel_ms_per_step": kernel_ms,
            "gpu_launches": launches, "train_rmse_after_timed_steps": stats["rmse"], "sweep_status": stats.get("status", "ok"),
            "plain_fp32": plain, "accuracy_vs_fp32": accuracy, "test_rmse_vs_oracle": test_rmse, "e2e": e2e,
            "cpu_baseline": cpu, "clocks": clocks,
            "serving": serve, "serving_host_loop": serve_host, "other_configs": side,
        }
        if serve and serve["loads"]:
            pick = min(serve["loads"], key=lambda d: abs(d["load"] - 0.8))
            out["foldin_p50_ms"], out["foldin_p99_ms"] = pick["p50_ms"], pick["p99_ms"]
            out["foldin_load"] = pick["load"]
        print(json.dumps(out))
    for s in sl:
        s.close()
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
