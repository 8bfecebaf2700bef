"""Benchmark of the SWF hot path on GB300.

One step = one solve of the batched (2+1)D Schwinger workload through the C ABI: 128 instances
(8 x 8 electron momenta in [-1, 1]^2, both spins, E drawn per instance) on a 256^2 grid, box 40,
1000 fixed Dormand-Prince steps from t = 20 back to t = -20 in complex64, then the FP64
C-spectrum |C(m, (r, q))|^2 over every grid positron (2 * 256^2 probabilities per instance).

Metric: spinor site-updates per second (one grid point of one instance advanced one full step);
the pair probabilities per second are reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Multi-GPU (torchrun): every rank solves its own copy of the batch (weak scaling, no collective
on the data path); value = all ranks' site-updates / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "spinor site-updates/s & pair probabilities/s per GB300 at rel.err <=1e-4 vs FP64"
UNIT = "site-updates/s"
WORKLOAD = "schwinger_batched: (2+1)D Schwinger, 256x256 grid, box 40, 128 instances, 1000 DP5 steps, c64 march + FP64 C-spectrum"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ CPU oracle (baseline arm)
def _single_thread():
    """Pool initialiser: one BLAS/FFT thread per worker process (one worker per core)."""
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"


def _oracle_warm(_):
    import numpy  # noqa: F401
    from oracle import swf_oracle  # noqa: F401
    return os.getpid()


def _oracle_march(job):
    """Marches instance i of the workload for n_rk_steps Dormand-Prince steps with the FP64
    oracle; returns (site-updates, seconds)."""
    i, n_rk_steps = job
    import numpy as np
    from oracle import swf_oracle as O
    from paper_2512_16889_gb300 import workloads as W
    from tests import oracle_adapter as OA
    d = W.schwinger_batched()[i]
    g, f, bg = OA.grid(d), OA.field(d), OA.background(d, 0)
    h = (d["t_in"] - d["t_out"]) / d["n_steps"]
    t0 = time.perf_counter()
    O.march_scattered(f, g, bg, d["t_out"] + n_rk_steps * h, d["t_out"], n_rk_steps)
    return int(np.prod(d["n"])) * n_rk_steps, time.perf_counter() - t0


def _oracle_project(i):
    """The oracle's C-spectrum of instance i (one projection at t_in); returns seconds."""
    import numpy as np
    from oracle import swf_oracle as O
    from paper_2512_16889_gb300 import workloads as W
    from tests import oracle_adapter as OA
    d = W.schwinger_batched()[i]
    g = OA.grid(d)
    psi = np.zeros((4,) + g.n, dtype=complex)
    psi[0] = 1e-3
    t0 = time.perf_counter()
    O.c_spectrum(psi, g, d["t_in"])
    return time.perf_counter() - t0


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


class OraclePool:
    """One spawned worker process per host core (spawn: the parent may already hold a CUDA
    context, which a forked child must not inherit)."""

    def __init__(self):
        import multiprocessing as mp
        try:
            self.cores = len(os.sched_getaffinity(0))
        except AttributeError:
            self.cores = os.cpu_count() or 1
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_single_thread)
        self.pool.map(_oracle_warm, range(self.cores), chunksize=1)

    def close(self):
        self.pool.close()
        self.pool.join()

    def sample(self, n_rk_steps=40):
        """The FP64 oracle on `cores` instances of the workload at once (instance j on core j),
        each for a bounded number of steps, and one C-spectrum per core; scaled to the metric's
        unit: site-updates/s = all cores' site-updates / the wall time of the march."""
        jobs = [(j % 128, n_rk_steps) for j in range(self.cores)]
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_march, jobs, chunksize=1)
        wall = time.perf_counter() - t0
        t0 = time.perf_counter()
        proj = self.pool.map(_oracle_project, [j % 128 for j in range(self.cores)], chunksize=1)
        wall_proj = time.perf_counter() - t0
        su = sum(r[0] for r in res)
        n_sites, n_steps = 256 * 256, 1000
        # one full solve per core: the march extrapolated from the sample, plus its projection
        t_full = statistics.mean(r[1] for r in res) * n_steps / n_rk_steps + statistics.mean(proj)
        return {"value": su / wall, "unit": UNIT, "cores": self.cores, "kind": "oracle",
                "cpu_model": cpu_model(),
                "sample": f"{self.cores} of 128 instances at once (one per core), {n_rk_steps} of {n_steps} steps "
                          f"each ({wall:.1f} s wall) + one C-spectrum per core ({wall_proj:.1f} s), numpy FP64; "
                          f"full-solve time extrapolated linearly in the steps",
                "probabilities_per_s": self.cores * 2 * n_sites / t_full}


def oracle_sample(n_rk_steps=40):
    pool = OraclePool()
    try:
        return pool.sample(n_rk_steps)
    finally:
        pool.close()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    times = []
    base = None
    pool = OraclePool()
    try:
        for i in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            base = pool.sample(n_rk_steps=10)
            if i >= args.warmup:
                times.append(time.perf_counter() - t0)
    finally:
        pool.close()
    line = {"impl": "reference", "metric": METRIC, "value": base["value"], "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": base["sample"]},
            "cpu_baseline": {"value": base["value"], "unit": UNIT, "cores": base["cores"], "kind": "oracle",
                             "cpu_model": base["cpu_model"], "sample": base["sample"]},
            "e2e": {"value": base["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def measured_traffic(kernel):
    """DRAM bytes (read + write) of one full-size launch of the march kernel from the committed
    ncu counters, or None when the kernel source changed since they were taken."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", kernel + "_counters.json")) as fh:
            d = json.load(fh)
        with open(os.path.join(ROOT, d["source"]), "rb") as fh:
            if hashlib.sha256(fh.read()).hexdigest() != d["source_sha256"]:
                return None
        full = d.get("full_launch")
        return float(full["dram_bytes_read"] + full["dram_bytes_write"]) if full else None
    except Exception:
        return None


# ------------------------------------------------------------------ clocks during the timed region
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.device)], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for ln in open(self.path):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" == r[5 + i] or r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ multi-rank aggregation
def aggregate(local_ms, units_per_rank, steps, world, device=None):
    """Max-over-ranks time and whole-job throughput: every rank processed units_per_rank units
    per step (weak scaling); the job's time is the slowest rank's."""
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, world * units_per_rank * steps / (ms_max / 1e3)


# ------------------------------------------------------------------ accuracy and the FP64 comparator
# The FP64 march's probabilities are claimed at 1e-10 relative for entries at or above
# FP64_1E10_FLOOR of their spectrum's maximum, and at 1e-4 at or above FP64_1E4_FLOOR:
# tests/test_gpu_parity.py checks the FP64 march against the oracle's whole spectra of two
# full-size instances and asserts both on every entry in those ranges.
FP64_1E10_FLOOR = 1e-7
FP64_1E4_FLOOR = 1e-19


def accuracy_vs_fp64(ctx, swf, ds, spec32_dev, stream, n_sample=16):
    """Solves every (128 / n_sample)-th instance of the workload with the plain FP64 GPU march
    (complex128) and compares the complex64 solve's probabilities |C|^2 with it entry by entry.
    Returns the fraction of all entries within 1e-4 relative, a table per decade of |C|^2 below
    each instance's maximum (entries, fraction within 1e-4, median relative error), and the FP64
    march's own rates (site-updates/s, probabilities/s, and those at 1e-10)."""
    import numpy as np
    import torch
    n_inst = len(ds)
    idx = list(range(0, n_inst, max(1, n_inst // n_sample)))[:n_sample]
    sub = [swf.from_workload(ds[i]) for i in idx]
    n2 = 2 * int(np.prod(ds[0]["n"]))
    res = torch.empty(len(sub) * swf.C.sizeof(swf.Result), dtype=torch.uint8, device="cuda")
    spec64 = torch.empty(len(sub) * n2, dtype=torch.float64, device="cuda")
    # warm-up at two steps: complex128 workspace and the pass kernels' launch shapes for this grid
    warm = [swf.from_workload(dict(ds[i], n_steps=2)) for i in idx]
    ctx.solve_dev(warm, res, spec64, swf.SCHWINGER, swf.C128, stream=stream)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    ctx.solve_dev(sub, res, spec64, swf.SCHWINGER, swf.C128, stream=stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms64 = ev0.elapsed_time(ev1)
    s64 = spec64.view(len(sub), n2).cpu().numpy()
    s32 = spec32_dev.view(n_inst, n2)[idx].cpu().numpy()
    mx = s64.max(axis=1, keepdims=True)
    with np.errstate(divide="ignore", invalid="ignore"):
        rel = np.where(s64 > 0, np.abs(s32 - s64) / s64, np.where(s32 == 0, 0.0, np.inf))
        dec = np.floor(np.log10(np.where(s64 > 0, s64 / mx, 1e-300)))
    within = rel <= 1e-4
    table = {"reference": f"complex128 march of instances {idx[0]}, {idx[1]}, ... (every {idx[1] - idx[0]}th, "
                          f"{len(idx)} of {n_inst})", "entries": int(rel.size),
             "frac_within_1e-4": float(within.mean()), "decades": []}
    for d in range(0, -31, -1):
        m = dec == d
        if m.any():
            table["decades"].append({"decade": d, "entries": int(m.sum()), "frac_within_1e-4": float(within[m].mean()),
                                     "median_rel_err": float(np.median(rel[m]))})
    below = dec < -30
    table["below_1e-30_of_max"] = {"entries": int(below.sum()), "frac_within_1e-4": float(within[below].mean())
                                   if below.any() else None}
    su = len(sub) * int(np.prod(ds[0]["n"])) * ds[0]["n_steps"]
    f10 = float((s64 >= FP64_1E10_FLOOR * mx).mean())
    f4 = float((s64 >= FP64_1E4_FLOOR * mx).mean())
    p64 = len(sub) * n2 / (ms64 / 1e3)
    fp64 = {"what": "plain FP64 GPU march: complex128, pass kernels, FP64 C-spectrum", "instances": len(sub),
            "ms": ms64, "site_updates_per_s": su / (ms64 / 1e3), "probabilities_per_s": p64,
            "probabilities_per_s_at_1e-10": p64 * f10, "frac_at_1e-10": f10,
            "probabilities_per_s_at_1e-4": p64 * f4, "frac_at_1e-4": f4,
            "at_accuracy": f"entries >= {FP64_1E10_FLOOR:g} (1e-10) and >= {FP64_1E4_FLOOR:g} (1e-4) of their "
                           f"spectrum's maximum: the ranges the parity tests assert against the oracle's whole spectra"}
    return {"frac_within_1e-4": float(within.mean()), "table": table, "fp64": fp64}


# ------------------------------------------------------------------ the other configurations (bounded samples)
def other_configs(swf, W):
    """One timed solve (CUDA events, after a two-step warm-up that sizes the workspace and tunes
    the launch shapes) of each other workload of the family, each in a fresh context: the single
    FP64 Schwinger workload in full (128^2, 1000 steps, both marches of the full pair number), the
    uneven-grid Breit-Wheeler workload on its first 32 instances for 300 of its 2605 steps, and the
    (3+1)D workload on its 16 instances for 10 of its 2000 steps.  Site-updates/s of each."""
    import numpy as np
    import torch
    out = {}
    cases = (
        ("c0_fp64_single_full", [dict(d, flags=("spectrum", "full_n")) for d in W.schwinger_fp64_single()],
         swf.SCHWINGER, swf.C128, 2, None),
        ("c2_bw_uneven_32x300", W.bw_uneven()[:32], swf.BREIT_WHEELER, swf.C64, 2, 300),
        ("c3_3d_16x10", W.schwinger_3d(), swf.SCHWINGER, swf.C64, 1, 10),
    )
    for name, ds, process, prec, fields, cap in cases:
        ds = [dict(d) for d in ds]
        if cap:
            for d in ds:
                frac = cap / d["n_steps"]
                d["t_in"] = d["t_out"] - frac * (d["t_out"] - d["t_in"])
                d["n_steps"] = cap
        insts = [swf.from_workload(d) for d in ds]
        ctx = swf.Context(0)
        ctx.solve([swf.from_workload(dict(d, n_steps=2)) for d in ds], process, prec)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.solve(insts, process, prec)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        ctx.close()
        su = sum(int(np.prod(d["n"])) * d["n_steps"] * fields for d in ds)
        out[name] = {"instances": len(ds), "n_steps": ds[0]["n_steps"], "grids": sorted({d["n"] for d in ds}),
                     "precision": "complex128" if prec == swf.C128 else "complex64", "s": t,
                     "site_updates_per_s": su / t}
    return out


# ------------------------------------------------------------------ GPU arm
def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2512_16889_gb300 import build, swf
    from paper_2512_16889_gb300 import workloads as W

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()

    def barrier():
        if world > 1:
            dist.barrier()

    ds = W.schwinger_batched()
    insts = [swf.from_workload(d) for d in ds]
    arr = swf.instance_array(insts)
    prec = swf.C64
    n_inst = len(ds)
    site_updates = sum(int(np.prod(d["n"])) * d["n_steps"] for d in ds)
    probs = sum(2 * int(np.prod(d["n"])) for d in ds)
    ctx = swf.Context(local)
    # every instance is marched (the workload's stated work): the library's exact reuse of the
    # other spin's march, which would skip the instances whose two spins share a field, is off
    ctx.set_dedupe(False)
    stream = torch.cuda.current_stream()
    res_dev = torch.empty(n_inst * swf.C.sizeof(swf.Result), dtype=torch.uint8, device="cuda")
    spec_dev = torch.empty(probs, dtype=torch.float64, device="cuda")

    def step():
        ctx.solve_dev(None, res_dev, spec_dev, swf.SCHWINGER, prec, stream=stream, arr=arr)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    ms_max, value = aggregate(ms, site_updates, args.steps, world, device="cuda")
    ms_step = ms_max / args.steps
    # per-kernel device times and launch counts: one more step with CUDA-event timing of every
    # launch (kernel by kernel, so it runs a little slower than the timed steps above)
    ctx.profile_read()  # clear counters
    fused0 = ctx.fields_fused()
    ctx.profile_enable(True)
    step()
    torch.cuda.synchronize()
    ctx.profile_enable(False)
    prof1, launches1 = ctx.profile_read()
    fused_fields = ctx.fields_fused() - fused0
    prof = {k: (v[0] * args.steps, v[1] * args.steps) for k, v in prof1.items()}
    launches = launches1 * args.steps

    # the plain FP64 GPU march (complex128, pass kernels) on a sample of the instances, and the
    # accuracy of the complex64 probabilities against it (untimed for the headline value)
    acc = accuracy_vs_fp64(ctx, swf, ds, spec_dev, stream)

    others = other_configs(swf, W) if rank == 0 and not args.no_other_configs else None

    # end to end through the host-pointer API (copies of inputs and outputs included)
    e2e_steps = max(1, min(args.steps, 2))
    ctx.solve(insts, swf.SCHWINGER, prec)  # warm the host path once
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ctx.solve(insts, swf.SCHWINGER, prec)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    _, e2e_value = aggregate(e2e_s * 1e3, site_updates, 1, world, device="cuda")

    # roofline of the dominant kernel, the fused cluster march (algorithmic 14 S bytes per
    # site-update, S = 32 B in c64): the site-updates of the fields it marched (the library gives
    # the rest to the pass kernels, run concurrently on the SMs its clusters leave free) over its
    # own event-timed duration
    hbm, peak_kind = peaks()
    dominant = max(prof.items(), key=lambda kv: kv[1][0])[0] if prof else None
    S = 32.0
    su_field = 256 * 256 * 1000
    fk = "k_fused3" if "k_fused3" in prof else "k_fused"  # the fused variant the library ran
    fused_ms = prof.get(fk, (0.0, 0))[0] / args.steps
    fused_su = su_field * fused_fields
    alg_bytes = 14.0 * S * fused_su
    achieved = alg_bytes / (fused_ms / 1e3) / 1e9 if fused_ms > 0 else None
    march = {k: v for k, v in prof.items() if k in ("k_first", "k_mid", "k_last", fk)}
    roof = {"bound": "hbm", "kernel": fk + " (one launch per solve)",
            "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm if achieved else None, "traffic": measured_traffic(fk),
            "peak_kind": peak_kind + " (burst copy)", "launches_per_step": prof.get(fk, (0, 0))[1] / args.steps,
            "algorithmic_bytes_per_launch": alg_bytes, "fields_per_launch": fused_fields,
            "fields_on_pass_kernels": n_inst - fused_fields,
            "whole_march_frac": 14.0 * S * site_updates / (ms_step / 1e3) / 1e9 / hbm}
    # What binds the fused kernel instead of HBM: its two transposes per evaluation through the
    # cluster network (distributed shared memory).  Per evaluation of a z-spin sector every CTA of
    # the 16-CTA cluster sends 15 remote 16 x 16 blocks of both components (8 B each) per
    # transpose: 2 x 15 x 16 x 16 x 2 x 8 B = 120 KiB per CTA, 16 CTAs per sector; 2 sectors per
    # field, 1 + 6 n_steps evaluations.  Peak: the 13 B per cycle per SM that probes of pulls and of
    # bulk-copy pushes measured in 16-CTA clusters, on the SMs the clusters occupy, at the sampled
    # SM clock.
    dsm_bytes = 2 * fused_fields * (1 + 6 * 1000) * 16 * (2 * 15 * 16 * 16 * 2 * 8)
    clk_hz = (clk.get("sm_mhz") or 2070.0) * 1e6
    dsm_peak = 13.0 * 16 * 7 * clk_hz
    roof["limiter"] = {
        "what": "cluster network (distributed shared memory) during the two transposes per evaluation, "
                "pushed by the bulk-copy engine and partly hidden behind the local term and the next stage "
                "combine; FFT passes and block and cluster barriers elsewhere",
        "dsmem_bytes_per_launch": dsm_bytes,
        "dsmem_achieved_GBps": dsm_bytes / (fused_ms / 1e3) / 1e9 if fused_ms > 0 else None,
        "dsmem_peak_GBps": dsm_peak / 1e9,
        "dsmem_frac": dsm_bytes / (fused_ms / 1e3) / dsm_peak if fused_ms > 0 else None,
        "peak_kind": "measured probe: 13 B/clk/SM within a 16-CTA cluster (pulls and bulk-copy pushes alike), "
                     "x 112 SMs x sampled SM clock"}
    kernels = {k: {"ms_per_step": v[0] / args.steps, "launches_per_step": v[1] / args.steps} for k, v in prof.items()}
    # FFT flops alongside: 5 N log2 N per complex transform, 8 transforms (4 components forward
    # and back) per evaluation, 6 evaluations per FSAL step; FP32 lane peak = SMs x 128 lanes x
    # 2 (FMA) x the maximum SM clock
    n_sites = 256 * 256
    fft_flops = 6 * 8 * 5 * np.log2(n_sites) * site_updates
    props = torch.cuda.get_device_properties(local)
    sm_max = (clk.get("sm_max_mhz") or 2070.0) * 1e6
    fp32_peak = props.multi_processor_count * 128 * 2 * sm_max
    fft_rate = fft_flops / (ms_step / 1e3) if ms_step > 0 else None
    alu = {"fft_flops_per_site_update": fft_flops / site_updates, "achieved_tflops": fft_rate / 1e12 if fft_rate else None,
           "fp32_peak_tflops": fp32_peak / 1e12, "frac": fft_rate / fp32_peak if fft_rate else None}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "grid": "256x256", "instances": n_inst, "n_steps": 1000,
                           "precision": "complex64 march, FP64 projections",
                           "l2": "inputs larger than L2 (2.3 GB working set per GPU)"},
                "probabilities_per_s": world * probs * args.steps / (ms_max / 1e3),
                "probabilities_per_s_at_1e-4": world * probs * args.steps / (ms_max / 1e3) * acc["frac_within_1e-4"],
                "accuracy": acc["table"], "fp64_comparator": acc["fp64"], "other_configs": others,
                "roofline": roof, "fft_flops": alu, "kernels": kernels, "dominant_kernel": dominant,
                "gpu_launches": int(launches),
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": n_inst * swf.C.sizeof(swf.Instance),
                        "d2h_bytes_per_step": n_inst * swf.C.sizeof(swf.Result) + probs * 8},
                "clocks": clk}
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = oracle_sample()
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_surrogate(args):
    """Times the surrogate network on one GPU: inference over 10^6 scan points (the screening
    pass) and Adam training steps at batch 256, against the measured BF16 tensor peak."""
    import numpy as np
    import torch
    from paper_2512_16889_gb300 import build, surrogate as S, swf
    build.build()
    rng = np.random.default_rng(8)
    n_inf = args.limit or 1_000_000
    X = np.stack([rng.choice([0.2, 0.3, 0.4], n_inf), rng.uniform(0.3, 0.7, n_inf), rng.uniform(3, 8, n_inf),
                  rng.uniform(-1, 1, n_inf), rng.uniform(-1, 1, n_inf), rng.choice([1.0, -1.0], n_inf)],
                 axis=1).astype(np.float32)
    y = (-10.0 + np.tanh(X[:, 0] * 4) + 0.3 * X[:, 3] * X[:, 4]).astype(np.float32)
    sur = swf.Surrogate(S.init_params(0), S.normalisation(X, y), max_batch=65536)
    Xd = torch.from_numpy(X).cuda()
    yd = torch.from_numpy(y).cuda()
    out = torch.empty(n_inf, 2, dtype=torch.float32, device="cuda")
    flops_fwd = 2.0 * sum(i * o for i, o in zip((6, 256, 256, 256, 256), (256, 256, 256, 256, 2)))
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(3):
        sur.forward(Xd, out)
    torch.cuda.synchronize()
    reps = max(1, args.steps)
    ev0.record(stream)
    for _ in range(reps):
        sur.forward(Xd, out)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_inf = ev0.elapsed_time(ev1) / 1e3 / reps
    # training: Adam steps at batch 256 (forward, backward, update)
    bt = 256
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    xb, yb = Xd[:bt].contiguous(), yd[:bt].contiguous()
    for _ in range(5):
        sur.train_step(xb, yb, 1e-4, loss)
    torch.cuda.synchronize()
    n_tr = 200
    ev0.record(stream)
    for _ in range(n_tr):
        sur.train_step(xb, yb, 1e-4, loss)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_tr = ev0.elapsed_time(ev1) / 1e3 / n_tr
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            bf16 = float(json.load(fh)["bf16_tflops"])
        kind = "measured"
    except Exception:
        bf16, kind = 1900.0, "fallback"
    inf_tflops = flops_fwd * n_inf / t_inf / 1e12
    line = {"metric": "surrogate scan points/s", "value": n_inf / t_inf, "unit": "points/s", "n_gpus": 1,
            "steps": reps, "warmup": 3, "ms_per_step": 1e3 * t_inf, "higher_is_better": True, "dtype": "bf16",
            "data": "synthetic", "config": {"workload": "surrogate: MLP 6-4x256(GELU)-2, BF16 operands, FP32 accumulate",
                                             "inference_points": n_inf, "train_batch": bt},
            "roofline": {"bound": "tensor", "achieved": inf_tflops, "peak": bf16, "unit": "TFLOP/s",
                         "frac": inf_tflops / bf16, "peak_kind": kind + " (burst bf16)",
                         "flops_per_point": flops_fwd},
            "train": {"ms_per_step": 1e3 * t_tr, "samples_per_s": bt / t_tr,
                      "tflops": 3 * flops_fwd * bt / t_tr / 1e12}}
    print(json.dumps(line), flush=True)
    sur.close()
    return 0


def run_surrogate_scan(args):
    """The learned screen end to end on one GPU, at a reduced solver resolution (64^2 grid, box
    40, 200 steps): a momentum scan (p in [-1, 1]^2, both spins) of the E = 0.3 field; train on
    8192 solver samples (3000 epochs, Adam 5e-4), calibrate the sigma threshold on 1024 held-out
    samples for tolerances 5e-2 and 1e-2 in ln P, then screen a 16384-point scan and solve the
    rejected points.  Reports acceptance, accuracy of the accepted points against the solver, and
    the time of the screened scan against solving every point."""
    import numpy as np
    import torch
    from paper_2512_16889_gb300 import build, surrogate as S, swf
    build.build()
    grid = dict(n=64, L=40.0, n_steps=200, t_window=20.0)
    ctx = swf.Context(0)

    def scan(n, seed):
        rng = np.random.default_rng(seed)
        return {"E": np.full(n, 0.3), "omega": np.full(n, 0.5), "lam": np.full(n, 5.0),
                "px": rng.uniform(-1, 1, n), "py": rng.uniform(-1, 1, n), "s": rng.choice([1, -1], n)}

    n_tr, n_sc = (args.limit or 8192), 16384
    tr, ho, sc = scan(n_tr, 4), scan(1024, 5), scan(n_sc, 6)
    t0 = time.perf_counter()
    y_tr = S.solve_targets(ctx, tr, **grid)
    t_train_data = time.perf_counter() - t0
    y_ho = S.solve_targets(ctx, ho, **grid)
    t0 = time.perf_counter()
    y_sc = S.solve_targets(ctx, sc, **grid)  # the method without the network
    t_all = time.perf_counter() - t0
    X_tr = S.features(tr)
    sur = swf.Surrogate(S.init_params(0), S.normalisation(X_tr, y_tr), max_batch=512)
    t0 = time.perf_counter()
    hist = S.train(sur, X_tr, y_tr, epochs=3000, batch=256, lr=5e-4)
    t_fit = time.perf_counter() - t0
    out = {"metric": "surrogate-screened scan", "unit": "s", "higher_is_better": False, "n_gpus": 1,
           "data": "synthetic", "config": {"workload": "surrogate_scan: momentum scan of E = 0.3, 64^2 grid, 200 steps",
                                            "train_samples": n_tr, "scan_points": n_sc, "epochs": 3000},
           "solver_s_per_point": t_all / n_sc, "train_data_s": t_train_data, "fit_s": t_fit,
           "final_loss": hist[-1], "all_solver_s": t_all, "screens": []}
    for tol, cov in ((5e-2, 0.95), (1e-2, 0.99)):
        thr = S.calibrate(sur, S.features(ho), y_ho, tol, coverage=cov)
        vals, acc, t_net, t_sol = S.screened_scan(sur, ctx, sc, thr, **grid)
        err = np.abs(vals - y_sc)
        out["screens"].append({"tol_lnP": tol, "coverage": cov, "accepted": float(acc.mean()),
                               "accepted_within_tol": float((err[acc] <= tol).mean()) if acc.any() else None,
                               "screened_s": t_net + t_sol, "speedup_vs_all_solver": t_all / (t_net + t_sol)})
    out["value"] = out["screens"][0]["screened_s"]
    print(json.dumps(out), flush=True)
    sur.close()
    ctx.close()
    return 0


def run_surrogate_spec(args):
    """The learned screen at the scale the workload states, on one GPU: 20 000 solver samples of
    the batched workload's grid and window (256^2, box 40, 1000 steps over [-20, 20], complex64
    march, FP64 overlaps) with E ~ U[0.15, 0.45], omega ~ U[0.2, 0.8], lambda ~ U[3, 8], p ~
    U[-1, 1]^2, drawn as 10 000 (field, p) points with both spins (the other spin's march is
    the first's with two components negated, so 10 000 marches serve 20 000 samples); training
    by the library's BF16 kernels (Adam, batch 256); the sigma threshold calibrated on 2 048
    held-out solver samples for 1e-2 in ln P at 99 % coverage (and 5e-2 at 95 %); inference over
    a 10^6-point scan.  The scan's fallback (a solve for every rejected point) is measured on a
    random sample of the rejected points and extrapolated, and a random sample of the accepted
    points is solved to audit them: both samples are reported with their sizes."""
    import numpy as np
    import torch
    from paper_2512_16889_gb300 import build, surrogate as S, swf
    from paper_2512_16889_gb300 import workloads as W
    build.build()
    ctx = swf.Context(0)
    grid = dict(n=256, L=40.0, n_steps=1000, t_window=20.0)

    def paired(n, seed):
        # both spins of each (field, p) next to each other, so that one call marches them once
        t = W.surrogate_samples(n // 2, seed=seed)
        out = {k: np.repeat(np.asarray(v), 2) for k, v in t.items()}
        out["s"] = np.tile([1.0, -1.0], n // 2)
        return out

    n_train = args.limit or 20000
    tr, ho = paired(n_train, 4), paired(2048, 5)
    t0 = time.perf_counter()
    y_tr = S.solve_targets(ctx, tr, batch=256, **grid)
    t_data = time.perf_counter() - t0
    y_ho = S.solve_targets(ctx, ho, batch=256, **grid)
    X_tr = S.features(tr)
    sur = swf.Surrogate(S.init_params(0), S.normalisation(X_tr, y_tr), max_batch=1 << 20)
    epochs = args.epochs or 1500
    t0 = time.perf_counter()
    hist = S.train(sur, X_tr, y_tr, epochs=epochs, batch=256, lr=5e-4)
    t_fit = time.perf_counter() - t0
    sc = W.surrogate_samples(1_000_000, seed=6)
    Xs = torch.from_numpy(S.features(sc)).cuda()
    out = torch.empty(len(Xs), 2, dtype=torch.float32, device="cuda")
    sur.forward(Xs, out)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    sur.forward(Xs, out)
    ev1.record()
    torch.cuda.synchronize()
    t_inf = ev0.elapsed_time(ev1) / 1e3
    o = out.cpu().numpy().astype(float)
    mu, sig = o[:, 0], np.exp(0.5 * o[:, 1])
    rng = np.random.default_rng(9)
    line = {"metric": "surrogate-screened scan at the stated scale", "unit": "s", "higher_is_better": False,
            "n_gpus": 1, "data": "synthetic",
            "config": {"workload": "surrogate_spec: 256^2, box 40, 1000 steps, E in [0.15, 0.45], omega in [0.2, 0.8], "
                                   "lambda in [3, 8], p in [-1, 1]^2, both spins",
                       "train_samples": len(y_tr), "heldout_samples": len(y_ho), "scan_points": len(mu),
                       "epochs": epochs, "batch": 256},
            "train_data_s": t_data, "fit_s": t_fit, "final_loss": hist[-1], "inference_s": t_inf,
            "y_range": [float(y_tr.min()), float(y_tr.max())], "screens": []}
    n_audit = 1024
    t_per_solve = None
    for tol, cov in ((1e-2, 0.99), (5e-2, 0.95)):
        thr = S.calibrate(sur, S.features(ho), y_ho, tol, coverage=cov)
        acc = sig <= thr
        scr = {"tol_lnP": tol, "coverage": cov, "threshold": thr, "accepted": float(acc.mean())}
        for name, mask in (("audit_accepted", acc), ("fallback_rejected", ~acc)):
            idx = np.nonzero(mask)[0]
            if len(idx) == 0:
                continue
            pick = rng.choice(idx, min(n_audit, len(idx)), replace=False)
            sub = {k: np.asarray(v)[pick] for k, v in sc.items()}
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            y_sub = S.solve_targets(ctx, sub, batch=256, **grid)
            dt = time.perf_counter() - t1
            if name == "fallback_rejected":
                t_per_solve = dt / len(pick)
                scr["fallback_sample"] = len(pick)
                scr["fallback_s_per_point"] = t_per_solve
            else:
                err = np.abs(mu[pick] - y_sub)
                scr["audit_sample"] = len(pick)
                scr["audit_within_tol"] = float((err <= tol).mean())
                scr["audit_median_err"] = float(np.median(err))
        if t_per_solve:
            n_rej = int((~acc).sum())
            scr["screened_scan_s_extrapolated"] = t_inf + n_rej * t_per_solve
            scr["all_solver_s_extrapolated"] = len(mu) * t_per_solve
            scr["speedup"] = scr["all_solver_s_extrapolated"] / scr["screened_scan_s_extrapolated"]
        line["screens"].append(scr)
    line["value"] = line["screens"][0].get("screened_scan_s_extrapolated")
    print(json.dumps(line), flush=True)
    sur.close()
    ctx.close()
    return 0


def run_cross_section(args):
    """The paper's (2+1)D momentum cross sections (Sec. V, Eqs. 11-12): N(p_1, q_1) on a 100 x 100
    grid through swf_pair_matrix (complex64 march, FP64 overlaps), for the single field
    (--workload cross_section_single) or the double field (cross_section_double).  Reports
    pairs/s and where the spectrum peaks."""
    import numpy as np
    import torch
    from paper_2512_16889_gb300 import build, swf
    from paper_2512_16889_gb300 import workloads as W
    build.build()
    kind = "single_e" if args.workload.endswith("single") else "double_e"
    els, pos = W.paper_cross_section(kind)
    E = [swf.from_workload(d) for d in els]
    P = [swf.from_workload(d) for d in pos]
    ctx = swf.Context(0)
    ctx.pair_matrix(E[:2], P[:2], swf.C64)  # warm-up
    times = []
    for _ in range(max(1, args.steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mat = ctx.pair_matrix(E, P, swf.C64)
        times.append(time.perf_counter() - t0)
    t = min(times)
    N = np.array([[mat[m][n].prob[0] for n in range(len(P))] for m in range(len(E))])
    m, n = np.unravel_index(np.argmax(N), N.shape)
    d = els[0]
    line = {"metric": "full pair numbers N(m, n)/s", "value": N.size / t, "unit": "pairs/s", "n_gpus": 1,
            "steps": len(times), "warmup": 1, "ms_per_step": 1e3 * t, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic", "config": {"workload": f"cross_section: {kind}, E0 = 1/4, omega = E0, "
                                                         f"kappa_x = kappa_y = E0/2, 100 x 100 (p1, q1)",
                                             "grid": list(d["n"]), "box": list(d["L"]), "window": [d["t_in"], d["t_out"]],
                                             "n_steps": d["n_steps"], "precision": "complex64 march, FP64 overlaps"},
            "peak": {"p1": els[m]["p"][0], "q1": pos[n]["q"][0], "N": float(N[m, n])},
            "two_lines_max_rel_diff": float(np.max(np.abs(
                np.array([[mat[i][j].prob[1] for j in range(len(P))] for i in range(len(E))]) - N)) / N.max())}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_pair_scan(args):
    """Times the all-pairs full pair number on one GPU: 128 electrons x 128 positrons of one
    field on the 256^2 grid (1000 steps, complex64 march, FP64 overlaps) through swf_pair_matrix:
    256 marches plus the overlap products, against 2 x 128 x 128 marches pair by pair."""
    import torch
    from paper_2512_16889_gb300 import build, swf
    from paper_2512_16889_gb300 import workloads as W
    build.build()
    els, pos = W.pair_scan()
    if args.limit:
        els, pos = els[:args.limit], pos[:args.limit]
    E = [swf.from_workload(d) for d in els]
    P = [swf.from_workload(d) for d in pos]
    ctx = swf.Context(0)
    # warm-up: the same scan at two steps (workspace, launch-shape tuning, first launches)
    ctx.pair_matrix([swf.from_workload(dict(d, n_steps=2)) for d in els],
                    [swf.from_workload(dict(d, n_steps=2)) for d in pos], swf.C64)
    times = []
    m0 = ctx.fields_marched()
    for _ in range(max(1, args.steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.pair_matrix(E, P, swf.C64)
        times.append(time.perf_counter() - t0)
    marched = (ctx.fields_marched() - m0) // len(times)
    t = min(times)
    ctx.profile_read()
    ctx.profile_enable(True)
    mat = ctx.pair_matrix(E, P, swf.C64)
    ctx.profile_enable(False)
    prof, _ = ctx.profile_read()
    n_pairs = len(E) * len(P)
    import numpy as np
    l2 = np.array([[r.prob[0] for r in row] for row in mat])
    l1 = np.array([[r.prob[1] for r in row] for row in mat])
    su = marched * 256 * 256 * els[0]["n_steps"]  # site-updates actually marched
    line = {"metric": "full pair numbers N(m, n)/s", "value": n_pairs / t, "unit": "pairs/s", "n_gpus": 1,
            "steps": len(times), "warmup": 1, "ms_per_step": 1e3 * t, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic", "config": {"workload": "pair_scan: 256^2, box 40, 1000 steps, E = 0.3",
                                             "electrons": len(E), "positrons": len(P),
                                             "precision": "complex64 march, FP64 overlaps"},
            "site_updates_per_s": su / t, "fields": len(E) + len(P), "fields_marched": marched,
            "max_N": float(l2.max()), "two_lines_max_rel_diff": float(np.max(np.abs(l1 - l2)) / l2.max()),
            "kernels": {k: {"ms": v[0], "launches": v[1]} for k, v in prof.items()}}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_photon_scan(args):
    """Times the Breit-Wheeler photon scan on one GPU: 64 photons for one pair of the uneven-grid
    workload (192^2, 2605 steps, complex64) from one march of U and V (swf_bw_photons), against
    the same 64 amplitudes as 64 instances of one batched solve (a march each)."""
    import numpy as np
    import torch
    from paper_2512_16889_gb300 import build, swf
    from paper_2512_16889_gb300 import workloads as W
    build.build()
    d, ks, es = W.bw_photon_scan()
    if args.limit:
        ks, es = ks[:args.limit], es[:args.limit]
    inst = swf.from_workload(d)
    n = len(ks)
    w = np.exp(-0.5 * (np.array([k[0] for k in ks]) / 0.5) ** 2).astype(complex)  # a Gaussian packet in k_x
    ctx = swf.Context(0)
    ctx.bw_photons(inst, ks[:2], es[:2], swf.C64)  # warm-up
    times = []
    for _ in range(max(1, args.steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        amps, packet = ctx.bw_photons(inst, ks, es, swf.C64, weights=w)
        times.append(time.perf_counter() - t0)
    t = min(times)
    ctx.profile_read()
    ctx.profile_enable(True)
    ctx.bw_photons(inst, ks, es, swf.C64, weights=w)
    ctx.profile_enable(False)
    prof, _ = ctx.profile_read()
    insts = [swf.from_workload(dict(d, k=tuple(k), eps=tuple(e))) for k, e in zip(ks, es)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res, _ = ctx.solve(insts, swf.BREIT_WHEELER, swf.C64)
    t_sep = time.perf_counter() - t0
    sep = np.array([complex(r.amp[6], r.amp[7]) for r in res])
    line = {"metric": "Breit-Wheeler photon amplitudes/s", "value": n / t, "unit": "amplitudes/s", "n_gpus": 1,
            "steps": len(times), "warmup": 1, "ms_per_step": 1e3 * t, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic", "config": {"workload": "bw_photon_scan: one 192^2 pair of bw_uneven, 2605 steps",
                                             "photons": n, "precision": "complex64 march, FP64 phases"},
            "separate_solves_s": t_sep, "speedup_vs_separate": t_sep / t,
            "max_abs_diff_vs_separate": float(np.max(np.abs(amps[:, 3] - sep))),
            "packet_M": [float(packet[3].real), float(packet[3].imag)],
            "kernels": {k: {"ms": v[0], "launches": v[1]} for k, v in prof.items()}}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_workload(args):
    """Times another workload of the benchmark family on one GPU (not the headline line):
    schwinger_fp64_single (128^2, complex128, full pair number), schwinger_batched_fp64 (the
    headline workload marched in complex128 on the pass kernels: the plain FP64 GPU march),
    bw_uneven (Breit-Wheeler, uneven grids) and schwinger_3d ((3+1)D 256^3).  --limit bounds the
    number of instances and --max-steps the Dormand-Prince steps; both are reported."""
    import numpy as np
    import torch
    from paper_2512_16889_gb300 import build, swf
    from paper_2512_16889_gb300 import workloads as W
    build.build()
    name = args.workload
    process, prec = swf.SCHWINGER, swf.C64
    if name == "schwinger_fp64_single":
        ds = [dict(d, flags=("spectrum", "full_n")) for d in W.schwinger_fp64_single()]
        prec = swf.C128
    elif name == "schwinger_batched_fp64":
        ds, prec = W.schwinger_batched(), swf.C128
    elif name == "bw_uneven":
        ds, process = W.bw_uneven(), swf.BREIT_WHEELER
    elif name == "schwinger_3d":
        ds = W.schwinger_3d()
    else:
        raise SystemExit(f"unknown workload {name}")
    if args.limit:
        ds = ds[:args.limit]
    if args.adaptive and args.bw_partial:
        raise SystemExit("--adaptive and --bw-partial do not combine (the partial-integration form uses fixed steps)")
    if args.adaptive:
        ds = [dict(d, flags=tuple(d.get("flags", ())) + ("adaptive",)) for d in ds]
    if args.bw_partial:
        if process != swf.BREIT_WHEELER:
            raise SystemExit("--bw-partial applies to Breit-Wheeler workloads")
        ds = [dict(d, flags=tuple(d.get("flags", ())) + ("bw_partial",)) for d in ds]
    if args.max_steps:
        for d in ds:
            if d["n_steps"] > args.max_steps:
                frac = args.max_steps / d["n_steps"]
                d["t_in"] = d["t_out"] - frac * (d["t_out"] - d["t_in"])
                d["n_steps"] = args.max_steps
    insts = [swf.from_workload(d) for d in ds]
    fields = 2 if process == swf.BREIT_WHEELER else (2 if name == "schwinger_fp64_single" else 1)
    su = sum(int(np.prod(d["n"])) * d["n_steps"] * fields for d in ds)
    ctx = swf.Context(0)
    ctx.set_multi_grid(0 if args.no_multi_grid else (2 if args.multi_grid else 1))
    # warm-up: the same instances at two fixed steps (plans, launch-shape tuning per grid group and
    # first launches happen here, not in the timed solves)
    ctx.solve([swf.from_workload(dict(d, n_steps=2, flags=tuple(f for f in d.get("flags", ()) if f != "adaptive")))
               for d in ds], process, prec)
    times = []
    for _ in range(max(1, args.steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res, _ = ctx.solve(insts, process, prec)
        times.append(time.perf_counter() - t0)
    t = min(times)
    prof = {}
    if not args.no_profile:
        ctx.profile_read()  # per-kernel device times of one more solve
        ctx.profile_enable(True)
        ctx.solve(insts, process, prec)
        ctx.profile_enable(False)
        prof, _ = ctx.profile_read()
    if args.adaptive:  # site-updates of the accepted steps (the last march's count for every field)
        su = sum(int(np.prod(d["n"])) * ctx.march_stats()[0] * fields for d in ds)
    forms = None
    if args.bw_partial:  # the same instances with past + finite terms (untimed): the gap between the forms
        ref = [swf.from_workload(dict(d, flags=())) for d in ds]
        r1, _ = ctx.solve(ref, process, prec)
        m1 = np.array([complex(x.amp[6], x.amp[7]) for x in r1])
        m2 = np.array([complex(x.amp[6], x.amp[7]) for x in res])
        forms = {"integrand": "partial integration (Eqs. 30-33)",
                 "max_rel_gap_to_past_finite": float(np.max(np.abs(m2 - m1) / np.abs(m1)))}
    line = {"metric": METRIC, "value": su / t, "unit": UNIT, "n_gpus": 1, "steps": len(times), "warmup": 1,
            "ms_per_step": 1e3 * t, "higher_is_better": True, "dtype": "f64" if prec == swf.C128 else "f32",
            "data": "synthetic", "config": {"workload": name, "instances": len(ds),
                                             "n_steps": ds[0]["n_steps"], "grids": sorted({d["n"] for d in ds}),
                                             "precision": "complex128" if prec == swf.C128 else "complex64"},
            "results_per_s": len(ds) / t, "site_updates_per_step": su, "multi_grid": 0 if args.no_multi_grid else (2 if args.multi_grid else 1),
            "step_control": ({"rtol": 1e-5, "atol": 1e-10, "accepted_rejected": ctx.march_stats()}
                             if args.adaptive else None),
            "bw_form": forms,
            "kernels": {k: {"ms": v[0], "launches": v[1]} for k, v in prof.items()}}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_small_march(args):
    """One march for profiler captures, complex64, through swf_march_dev: 14 instances (28
    sectors) of the batched workload for 20 steps (--small-march), all 128 instances for the
    full 1000 steps in one fused launch with no fields on the pass kernels (--fused-march), or 16
    instances for 4 steps on the pass kernels alone with their default launch shapes
    (--small-pass)."""
    import torch
    from paper_2512_16889_gb300 import build, swf
    from paper_2512_16889_gb300 import workloads as W
    build.build()
    ctx = swf.Context(0)
    if args.fused_march:
        ctx.set_dedupe(False)
        ctx.set_march_path(2)
        ds = W.schwinger_batched()
    elif args.small_pass:
        ctx.set_dedupe(False)
        ctx.set_march_path(1)
        ctx.set_autotune(False)
        ds = W.schwinger_batched(n_steps=4)[:16]
    else:
        ds = W.schwinger_batched(n_steps=20, t_window=0.4)[:14]
    out = torch.zeros(len(ds) * 8 * 256 * 256, dtype=torch.float32, device="cuda")
    ctx.march_dev([swf.from_workload(d) for d in ds], out, bg=0, prec=swf.C64)
    torch.cuda.synchronize()
    print("small march ok", float(out.abs().sum()))
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-other-configs", action="store_true", help="skip the other workloads' samples")
    ap.add_argument("--small-march", action="store_true", help="one small march for profiler captures")
    ap.add_argument("--fused-march", action="store_true",
                    help="the benchmark's march as one fused launch, for profiler captures at full size")
    ap.add_argument("--small-pass", action="store_true",
                    help="a small march on the pass kernels alone, for profiler captures")
    ap.add_argument("--workload", default=None, help="time another workload (see run_workload)")
    ap.add_argument("--limit", type=int, default=0, help="at most this many instances (--workload)")
    ap.add_argument("--max-steps", type=int, default=0, help="at most this many steps (--workload)")
    ap.add_argument("--adaptive", action="store_true", help="step-size-controlled marches (--workload)")
    ap.add_argument("--epochs", type=int, default=0, help="training epochs (--workload surrogate_spec)")
    ap.add_argument("--no-profile", action="store_true",
                    help="skip the extra solve with per-kernel timing (--workload; for long workloads)")
    ap.add_argument("--no-multi-grid", action="store_true",
                    help="march the grid groups one after another (--workload)")
    ap.add_argument("--multi-grid", action="store_true",
                    help="march grid groups that share a time grid together whatever their size (--workload)")
    ap.add_argument("--bw-partial", action="store_true",
                    help="partial-integration form of the Breit-Wheeler terms (--workload bw_uneven)")
    args = ap.parse_args()
    if args.small_march or args.fused_march or args.small_pass:
        return run_small_march(args)
    if args.workload == "surrogate":
        return run_surrogate(args)
    if args.workload == "bw_photon_scan":
        return run_photon_scan(args)
    if args.workload == "pair_scan":
        return run_pair_scan(args)
    if args.workload in ("cross_section_single", "cross_section_double"):
        return run_cross_section(args)
    if args.workload == "surrogate_scan":
        return run_surrogate_scan(args)
    if args.workload == "surrogate_spec":
        return run_surrogate_spec(args)
    if args.workload:
        return run_workload(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
