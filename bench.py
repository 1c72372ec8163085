#!/usr/bin/env python
"""Benchmark: two-component D2Q9 lattice updates per second (GLUPS) on one
GB300, with the HBM roofline fraction of the step kernel.

Workload: the sinusoidal channel with an oil slug, 8192 x 1170 nodes
(h(x) = 384 - 192 cos(2 pi x / 2048), slug 2560 nodes long centred on a neck),
FP32 populations, G = -1.79, tau = 1, wall potentials (0.5, 0.05), body force
1e-5.  One step = one launch of the fused step kernel (pull, densities,
interaction and wall forces, BGK collision, bounce-back, observables).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32]
  python bench.py --impl reference   # the FP64 CPU oracle on the host cores

Prints one JSON line (rank 0).  Under torchrun (N > 1) every rank runs an
independent replica on its own GPU (the step has no cross-GPU exchange).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import queue
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "2-comp D2Q9 GLUPS (fluid-node updates/s)"
UNIT = "GLUPS"
HBM_NOMINAL_GBS = 7900.0        # GB300 HBM3e nominal, for context beside the measured copy rate
G_INTERACTION = -1.79
PHYS = dict(tau=(1.0, 1.0), G=G_INTERACTION, rho_wall=(0.5, 0.05), g=(1e-5, 0.0))
BYTES_PER_POP = {"fp64": 8, "fp32": 4, "fp32c": 4, "fp16s": 2, "bf16s": 2}
DTYPE_NAME = {"fp64": "f64", "fp32": "f32", "fp32c": "f32 storage, compensated f32 math",
              "fp16s": "f16-shifted storage, f32 math", "bf16s": "bf16-shifted storage, f32 math"}
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")


def workload():
    from paper_1601_00918_gb300 import workloads as wl
    return wl.sinusoidal_slug(scale=8)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError, TypeError):
        return 6800.0, "fallback"


KERNEL_FILES = {"simple": ("lbm_common.cuh", "lbm_step.cuh"),
                "staged": ("lbm_common.cuh", "lbm_step_tma.cuh"),
                "pipelined": ("lbm_common.cuh", "lbm_step_tma.cuh", "lbm_step_warp.cuh"),
                "private": ("lbm_common.cuh", "lbm_step_tma.cuh", "lbm_step_private.cuh")}


def kernel_hash(variant):
    """sha256 prefix of the sources that define the step kernel `variant`."""
    h = hashlib.sha256()
    for f in KERNEL_FILES[variant]:
        with open(os.path.join(ROOT, "paper_1601_00918_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(precision, wname, kinfo):
    """DRAM bytes per step-kernel launch from a committed ncu capture, or None
    unless it was taken on this workload, precision, launch shape and kernel
    source."""
    try:
        with open(TRAFFIC_FILE) as fh:
            d = json.load(fh)
        e = d.get(f"{wname}/{precision}")
        if e and e.get("kernel_info") == kinfo and e.get("kernel_sha") == kernel_hash(kinfo["variant"]):
            return float(e["dram_bytes_per_launch"])
    except (OSError, ValueError, KeyError, TypeError, AttributeError):
        pass                                # no usable record: traffic unknown
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms; stop()
    keeps the samples taken inside the timed region (all of them, marked,
    if none fell inside)."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:                     # no nvidia-smi on this machine
            self.proc = None

    def _read(self):
        import datetime
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 8:
                try:
                    ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                except ValueError:
                    ts = None
                self.rows.append([ts] + parts[1:])

    def stop(self, t0=None, t1=None):
        """Summary of the samples between host times t0 and t1 (seconds)."""
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        rows = [r for r in self.rows if t0 is not None and r[0] is not None and t0 <= r[0] <= t1]
        inside = bool(rows)
        if not inside:
            rows = self.rows
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[4 + k] == "Active"})
        out = {"sm_mhz": statistics.median(sm) if sm else None,
               "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
               "samples": len(rows), "in_timed_region": inside}
        if not inside:
            # the timed region was shorter than the sampling period: the
            # summary is of the samples around it, not inside it
            out["too_short_to_sample"] = True
            if t0 is not None and t1 is not None:
                out["timed_region_s"] = t1 - t0
        return out


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload_config(w, ws):
    """The `config` of both arms' lines: the workload itself (how each arm
    runs it goes in the arm's own keys)."""
    ny, nx = w.mask.shape
    return {"workload": w.name, "nodes": nx * ny, "fluid_nodes": int(np.count_nonzero(w.mask == 0)),
            "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
            "l2": "state >= 2 x %.2f GB ping-pong in every storage form > 129 MB L2: no flush needed"
                  % (nx * ny * 18 * 2 / 1e9)}


# ----------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)
# ----------------------------------------------------------------------------
class OracleSample:
    """The FP64 oracle, unmodified, on a periodic crop of the workload (full
    height, the first `cols` columns); step() times one oracle step."""

    def __init__(self, w, cols):
        import oracle
        self.cols = int(cols)
        mask = np.ascontiguousarray(w.mask[:, :self.cols])
        rho = np.ascontiguousarray(w.rho[:, :, :self.cols])
        self.P = oracle.Problem(mask, periodic=w.periodic, **PHYS)
        self.f = self.P.init(rho)
        self.n_fluid = int(np.count_nonzero(mask == 0))

    def step(self):
        t0 = time.perf_counter()
        self.f, _ = self.P.step(self.f)
        return time.perf_counter() - t0


def oracle_sample_for(w, seconds_per_step, min_cols=64, max_cols=2048):
    """Crop width whose oracle step takes about seconds_per_step (at most
    max_cols columns: one wavelength of the channel, ~0.7 GB of oracle state)."""
    ny, nx = w.mask.shape
    probe = OracleSample(w, min_cols)
    dt = probe.step()
    per_col = dt / min_cols
    cols = int(min(nx, max_cols, max(min_cols, seconds_per_step / max(per_col, 1e-12))))
    return OracleSample(w, cols)


def host_cores():
    """(threads this process may use, CPU model) of the host."""
    try:
        n = len(os.sched_getaffinity(0))
    except AttributeError:
        n = os.cpu_count() or 1
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return n, model


def _oracle_worker(mask, rho, periodic, warmup, steps, barrier, results):
    """One host core: the unmodified oracle on its own copy of the crop;
    waits for the others, runs the warm-up steps, times the others."""
    import oracle
    P = oracle.Problem(mask, periodic=periodic, **PHYS)
    f = P.init(rho)
    barrier.wait()
    for _ in range(warmup):
        f, _ = P.step(f)
    t0 = time.perf_counter()
    for _ in range(steps):
        f, _ = P.step(f)
    results.put(time.perf_counter() - t0)


def oracle_all_cores(w, cols, warmup, steps, procs):
    """The oracle on `procs` host cores at once, one process per core (spawn),
    each stepping its own copy of the same crop (first `cols` columns): fluid
    updates of all of them / the slowest one's time."""
    import multiprocessing as mp
    mask = np.ascontiguousarray(w.mask[:, :cols])
    rho = np.ascontiguousarray(w.rho[:, :, :cols])
    n_fluid = int(np.count_nonzero(mask == 0))
    ctx = mp.get_context("spawn")
    barrier, results = ctx.Barrier(procs), ctx.Queue()
    ps = [ctx.Process(target=_oracle_worker, args=(mask, rho, w.periodic, warmup, steps, barrier, results))
          for _ in range(procs)]
    for p in ps:
        p.start()
    times = []
    try:
        while len(times) < procs:
            try:
                times.append(results.get(timeout=5.0))
            except queue.Empty:
                dead = [p.exitcode for p in ps if p.exitcode not in (None, 0)]
                if dead:
                    raise RuntimeError(f"an oracle process failed (exit code {dead[0]})")
    finally:
        for p in ps:
            if p.is_alive() and len(times) < procs:
                p.terminate()
            p.join()
    slowest = max(times)
    return procs * n_fluid * steps / slowest / 1e9, slowest, n_fluid


def reference_arm(args):
    """The FP64 oracle, as it stands, on every host core of this machine (one
    process per core on the same crop, weak scaling), each step a bounded
    sample of the workload so that the whole run takes a few minutes."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    w = workload()
    ny, nx = w.mask.shape
    # about 100 s of single-core work per process (more once all cores share
    # the memory system); at most one wavelength (2048 columns, ~0.7 GB of
    # oracle state) per process
    per_step = max(0.02, 100.0 / max(1, args.steps + args.warmup))
    cols = oracle_sample_for(w, per_step).cols
    procs, model = host_cores()
    value, slowest, n_fluid = oracle_all_cores(w, cols, args.warmup, args.steps, procs)
    sample = (f"FP64 oracle on {procs} host cores ({model or 'model unknown'}), one process per core, each "
              f"stepping a periodic crop of the first {cols} of {nx} columns (full {ny} rows, {n_fluid} fluid "
              f"nodes); time of the slowest process")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * slowest / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": workload_config(w, ws), "precision": "fp64",
            "sample": {"cols_sampled": cols, "processes": procs},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(w, seconds):
    """Oracle GLUPS on a bounded sample: a crop stepped for about `seconds`
    on one core, then the same crop on every host core at once."""
    ny, nx = w.mask.shape
    s = oracle_sample_for(w, min(seconds, 5.0))
    total, steps = 0.0, 0
    while total < seconds and steps < 100:
        total += s.step()
        steps += 1
    single = s.n_fluid * steps / total / 1e9
    procs, model = host_cores()
    all_value, slowest, _ = oracle_all_cores(w, s.cols, 1, steps, procs)
    return {"value": all_value, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": f"FP64 oracle, {steps} steps over a periodic crop of the first {s.cols} of {nx} columns "
                      f"(full {ny} rows, {s.n_fluid} fluid nodes) in each of {procs} processes, one per host "
                      f"core ({model or 'model unknown'}), {slowest:.1f} s for the slowest",
            "single_thread": {"value": single, "cores": 1, "seconds": total}}


# ----------------------------------------------------------------------------
# native arm
# ----------------------------------------------------------------------------
def native_arm(args):
    import torch
    from paper_1601_00918_gb300 import build, lbm

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU (no CPU fallback)")
    torch.cuda.set_device(local)
    build.build()
    lbm.library()
    w = workload()
    ny, nx = w.mask.shape
    n_fluid = int(np.count_nonzero(w.mask == 0))
    prec = args.precision

    sim = lbm.Simulation(w.mask, w.rho, precision=prec, periodic=w.periodic, device=local,
                         variant=args.variant, **PHYS)
    kinfo = sim.kernel_info()
    stream = torch.cuda.current_stream()
    sim.step(args.warmup)
    obs0 = sim.observables()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    # the K timed steps in up to five consecutive windows, an event between
    # them: the line's value is the whole region; best and median window
    # are reported beside it
    nwin = max(1, min(5, args.steps))
    sizes = [args.steps // nwin + (1 if k < args.steps % nwin else 0) for k in range(nwin)]
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(nwin + 1)]
    t_start = time.time()
    ev[0].record(stream)
    for k, n in enumerate(sizes):
        sim.step(n)
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    t_end = time.time()
    ms = ev[0].elapsed_time(ev[-1])
    win_glups = sorted(ws * n_fluid * n / (ev[k].elapsed_time(ev[k + 1]) * 1e-3) / 1e9
                       for k, n in enumerate(sizes))
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop(t_start, t_end)
    obs1 = sim.observables()
    assert obs1["step"] == obs0["step"] + args.steps and obs1["nan_flag"] == 0
    sim.close()
    del sim

    from paper_1601_00918_gb300 import dist as D
    ms = D.max_over_ranks(ms)              # the job runs as long as its slowest rank
    value = ws * n_fluid * args.steps / (ms * 1e-3) / 1e9

    # roofline of the step kernel: algorithmic bytes = read + write of the 18
    # populations of every fluid node per launch
    alg_bytes = n_fluid * 18 * 2 * BYTES_PER_POP[prec]
    per_launch_s = ms * 1e-3 / args.steps
    achieved = alg_bytes / per_launch_s / 1e9
    peak, peak_src = peaks()
    traffic = recorded_traffic(prec, w.name, kinfo)

    # end to end through the C ABI with host buffers
    e2e = e2e_arm(args, w, prec, local, n_fluid) if rank == 0 else None

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, args.cpu_seconds)
    crit = critical_pressure_arm(args) if rank == 0 and args.sweep_n > 0 else None
    bstep = batched_step_arm(args, peak) if rank == 0 and args.batch_n > 0 else None
    small = small_grids_arm() if rank == 0 and not args.no_small else None
    d3 = d3q19_arm(args, peak) if rank == 0 and args.d3_steps > 0 else None
    forms = forms_arm(args, w, peak, local, n_fluid) if rank == 0 and args.forms_steps > 0 else None

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_NAME[prec],
                "data": "synthetic",
                "config": workload_config(w, ws), "precision": prec, "kernel": kinfo,
                "windows": {"n": nwin, "steps": sizes, "best": win_glups[-1],
                            "median": statistics.median(win_glups), "unit": UNIT},
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": traffic,
                             "peak_source": f"{peak_src} hbm_gbs (copy, burst)",
                             "kernel": "step_%s_kernel" % kinfo["variant"],
                             "alg_bytes_per_launch": alg_bytes,
                             "frac_of_nominal": achieved / HBM_NOMINAL_GBS,
                             "traffic_gbs": traffic / per_launch_s / 1e9 if traffic else None},
                "all_nodes_value": value * nx * ny / n_fluid,
                "e2e": e2e, "gpu_launches": args.steps, "clocks": clk, "cpu_baseline": cpu,
                "critical_pressure": crit, "batched_step": bstep, "small_grids": small, "d3q19_tube": d3, "storage_forms": forms}
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def small_grids_arm(steps=2000):
    """The small configurations, each 2000 steps after 256 warm-up steps (in
    which the library also times its persistent launch against CUDA graphs of
    32 steps and keeps the faster); their state fits in the 129 MB L2, so they
    show launch and grid-barrier overhead, not the HBM roofline: the static droplet
    (128 x 128 periodic, R = 20, FP64), the layered channel (256 x 66, FP32)
    and the sinusoidal channel with a slug (1024 x 146) in FP32, FP16- and
    BF16-shifted storage."""
    import torch
    from paper_1601_00918_gb300 import lbm
    from paper_1601_00918_gb300 import workloads as wl
    cases = [("droplet_128x128_R20", wl.droplet_box(20.0, 128), "fp64", dict(tau=(1.0, 1.0), G=G_INTERACTION)),
             ("layered_256x66", wl.Workload("layered", wl.straight_channel(256, 64), wl.layered_channel(256, 64, 12),
                                            (True, False)), "fp32",
              dict(tau=(1.0, 1.0), G=G_INTERACTION, g=(1e-6, 0.0))),
             ]
    w3 = wl.sinusoidal_slug(1)
    for prec in ("fp32", "fp16s", "bf16s"):
        cases.append(("sinusoidal_slug_1024x146", w3, prec, PHYS))
    stream = torch.cuda.current_stream()
    out = []
    for name, w, prec, kw in cases:
        sim = lbm.Simulation(w.mask, w.rho, precision=prec, periodic=w.periodic, **kw)
        try:
            sim.step(256)
            kinfo = sim.kernel_info()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(steps)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            obs = sim.observables(check=False)
        finally:
            sim.close()
        n_fluid = int(np.count_nonzero(w.mask == 0))
        out.append({"workload": name, "precision": prec, "value": n_fluid * steps / (ms * 1e-3) / 1e9,
                    "unit": UNIT, "us_per_step": 1e3 * ms / steps, "kernel": kinfo,
                    "nan_flag": obs["nan_flag"]})
    return out


def batched_step_arm(args, peak):
    """Steps of the batch of sweep channels at their full sizes (lambda in
    {128, 192, 256, 384, 512} nodes, 4 periods, A/h0 ~ U[0.2, 0.6], slug /
    lambda ~ U[1, 2], theta ~ U[20, 160] deg, seed 0; 512 channels: 1.23e8
    nodes, 8.6e7 fluid), one launch per step for all of them, in FP16-shifted
    storage (the sweep's precision) and FP32: fluid-node updates per second
    and the algorithmic bytes of a step (18 populations read and written per
    fluid node) against the measured copy rate.  The channels start at rest
    with the slug in place and g = 1e-5 (a moving state, no bisection)."""
    import torch
    from paper_1601_00918_gb300 import lbm, sweep
    from paper_1601_00918_gb300 import workloads as wl
    specs = wl.sweep_specs(args.batch_n, seed=0)
    insts = [dict(sweep.instance_of(s), g=(1e-5, 0.0)) for s in specs]
    n_fluid = sum(int(np.count_nonzero(d["mask"] == 0)) for d in insts)
    n_nodes = sum(int(d["mask"].size) for d in insts)
    out = {"channels": len(insts), "nodes": n_nodes, "fluid_nodes": n_fluid, "steps": args.batch_steps,
           "warmup": 16, "l2": "state > 129 MB L2: no flush needed"}
    stream = torch.cuda.current_stream()
    for prec in ("fp16s", "fp32"):
        b = lbm.Batch(insts, precision=prec)
        try:
            kinfo = b.kernel_info()
            b.step(16)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.step(args.batch_steps)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            obs = b.observables(check=False)
        finally:
            b.close()
        assert all(o["nan_flag"] == 0 and o["step"] == 16 + args.batch_steps for o in obs)
        alg = n_fluid * 18 * 2 * BYTES_PER_POP[prec]
        gbs = alg / (ms * 1e-3 / args.batch_steps) / 1e9
        out[prec] = {"value": n_fluid * args.batch_steps / (ms * 1e-3) / 1e9, "unit": UNIT,
                     "ms_per_step": ms / args.batch_steps,
                     "kernel": "batch_staged_kernel" if kinfo["variant"] == "staged" else "batch_step_kernel",
                     "strip_rows": kinfo["strip_rows"], "ctas_per_step": kinfo["ctas_per_step"],
                     "alg_bytes_per_launch": alg, "achieved_gbs": gbs, "frac": gbs / peak}
    return out


CRIT_GOLDEN = os.path.join(ROOT, "tests", "golden")


def oracle_parity(lbm, precision):
    """The five channels of the oracle's own critical-force bisection
    (tests/golden/critical_channel_64.json: lambda = 64, 20 000 steps at
    g = 0, 80 000 per probe, 2 % bracket) bisected on this GPU with the same
    protocol: per channel the ratio of the GPU's bracket centre to the
    oracle's and whether the two brackets overlap or touch."""
    import numpy as np
    from paper_1601_00918_gb300 import workloads as wl
    with open(os.path.join(CRIT_GOLDEN, "capillary_channel_64.json")) as fh:
        cap = json.load(fh)
    with open(os.path.join(CRIT_GOLDEN, "critical_channel_64.json")) as fh:
        crit = json.load(fh)
    ch = cap["channel"]
    orc = {r["theta"]: r for r in crit["runs"] if r["t_obs"] == 80000}
    insts, lo, hi, runs = [], [], [], []
    for run in cap["runs"]:
        spec = wl.ChannelSpec(lam=ch["lam"], amp_ratio=ch["amp_ratio"],
                              slug_len_over_lambda=ch["slug_len_over_lambda"], theta_deg=run["theta"],
                              visc_ratio=1.0)
        w = wl.channel_instance(spec)
        insts.append(dict(mask=w.mask, rho_init=w.rho, tau=tuple(cap["tau"]), G=cap["G"],
                          rho_wall=tuple(run["rho_wall"]), g=(0.0, 0.0), periodic=w.periodic,
                          disp_threshold=0.5 * spec.lam))
        o = orc[run["theta"]]
        lo.append(o["g_start"][0])
        hi.append(o["g_start"][1])
        runs.append(o)
    t0 = time.perf_counter()
    b = lbm.Batch(insts, precision=precision)
    try:
        res = b.critical_pressure(np.array(lo), np.array(hi), rel_bracket=crit["rel_bracket"], t_eq=crit["t_eq"],
                                  t_obs=80000, max_probes=crit["max_probes"], check_bracket=True, check=False)
    finally:
        b.close()
    out = []
    for o, r in zip(runs, res):
        touch = 1e-12 * o["g_hi"]
        out.append({"theta": o["theta"], "lbm_over_oracle": math.sqrt(r["g_lo"] * r["g_hi"] / (o["g_lo"] * o["g_hi"])),
                    "within_one_bracket": bool(r["g_lo"] <= o["g_hi"] + touch and o["g_lo"] <= r["g_hi"] + touch),
                    "status": r["status"]})
    return {"precision": precision, "seconds": time.perf_counter() - t0, "channels": out}


def gated_specs(n, seed, lam):
    """Channels of the sweep distribution (A/h0 ~ U[0.2, 0.6], slug/lambda ~
    U[1, 2], theta ~ U[20, 160] degrees, viscosity ratio log-U[0.5, 10], four
    periods) at one wavelength."""
    from paper_1601_00918_gb300 import sweep
    return sweep.small_specs(n, seed=seed, lambdas=(lam,))


def d3q19_arm(args, peak):
    """The step on the paper's own lattice and geometry: D3Q19 in a periodic
    sinusoidal tube (radius 24 - 10 cos(2 pi x / 512), circular cross
    sections, 2048 x 66 x 66 nodes) holding an oil slug, FP32 and FP64.
    GLUPS over fluid nodes, and the fraction of the measured copy rate of
    the algorithmic bytes (read + write of the 38 populations: 304 B per
    fluid node in FP32, 608 B in FP64; the density pass and its re-read of
    the populations are overhead and count against it)."""
    import torch
    from paper_1601_00918_gb300 import lbm
    from paper_1601_00918_gb300 import workloads as wl
    nx, nc = 2048, 66
    mask = wl.sinusoidal_tube(nx, nc, 24.0, 10.0, 512.0)
    rho = wl.tube_slug(nx, nc, 768.0, 1280.0)
    n_fluid = int(np.count_nonzero(mask == 0))
    out = {"workload": f"sinusoidal_tube_{nx}x{nc}x{nc}", "nodes": int(mask.size), "fluid_nodes": n_fluid,
           "steps": args.d3_steps}
    for prec in ("fp32", "fp64"):
        sim = lbm.Simulation3(mask, rho, tau=(1.0, 1.0), G=G_INTERACTION, rho_wall=(0.3, 0.05),
                              g=(1e-6, 0.0, 0.0), periodic=(True, False, False), precision=prec,
                              collision="regularized")
        try:
            sim.step(3)
            stream = torch.cuda.current_stream()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(args.d3_steps)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            obs = sim.observables()
        finally:
            sim.close()
        assert obs["nan_flag"] == 0
        alg = n_fluid * 38 * 2 * BYTES_PER_POP[prec]
        gbs = alg / (ms * 1e-3 / args.d3_steps) / 1e9
        out[prec] = {"value": n_fluid * args.d3_steps / (ms * 1e-3) / 1e9, "unit": UNIT,
                     "ms_per_step": ms / args.d3_steps, "alg_bytes_per_launch_pair": alg, "achieved_gbs": gbs,
                     "frac": gbs / peak, "kernels": "density3_kernel + collide3_kernel"}
    return out


def critical_pressure_arm(args):
    """Critical-pressure solves per hour on this GPU, accuracy-gated.

    Gate 1, parity: the oracle's own bisection of five channels (FP64, on the
    host) against this GPU's with the same protocol (oracle_parity), in FP32
    and FP16-shifted storage.  Gate 2, convergence: the solves use lambda =
    128 channels and windows of 80 000 steps at g = 0 and 320 000 per probe,
    the window at which the bisected force stops depending on it (doubling
    it moves no bracket by more than one bisection step).  Every solve goes
    through lbm_critical_pressure_channels (channel, wall potentials from the
    Section 3.3 calibration run here, planar starting bracket, batched
    bisection).  Plain: one channel per call (a subset, time per solve
    extrapolated); batched: all channels in one call; seeded: the surrogate
    trained on a separate batched sweep at the same windows starts the
    brackets.  The seeded figure is given without and with its training
    sweep, with the break-even number of solves."""
    import numpy as np
    from paper_1601_00918_gb300 import lbm, sweep, wetting
    lam = args.sweep_lam
    kw = dict(t_eq=80000 * (lam // 128) ** 2, t_obs=320000 * (lam // 128) ** 2, rel_bracket=0.02, max_probes=24)
    t0 = time.perf_counter()
    table = wetting.calibrate(lbm)
    t_cal = time.perf_counter() - t0
    parity = [oracle_parity(lbm, p) for p in ("fp32", "fp16s")]
    ck = dict(table=table, sigma=wetting.SIGMA, rho=wetting.RHO_BULK, **kw)
    specs = gated_specs(args.sweep_n, 2, lam)
    res_b, t_b = sweep.run_channels(lbm, specs, **ck)
    ok_b = sum(r["status"] == 0 for r in res_b)
    res_h, t_h = sweep.run_channels(lbm, specs, precision="fp16s", **ck) if args.sweep_fp16s else ([], 0.0)
    ok_h = sum(r["status"] == 0 for r in res_h)

    def overlap(a, b):
        return a["g_lo"] <= b["g_hi"] * (1 + 1e-12) and b["g_lo"] <= a["g_hi"] * (1 + 1e-12)

    both_h = [(a, b) for a, b in zip(res_h, res_b) if a["status"] == 0 and b["status"] == 0]
    n_p = min(args.sweep_plain, len(specs))
    res_p, t_p = [], 0.0
    for s in specs[:n_p]:
        r, dt = sweep.run_channels(lbm, [s], **ck)
        res_p += r
        t_p += dt
    ok_p = sum(r["status"] == 0 for r in res_p)
    same_p = sum(1 for a, b in zip(res_p, res_b) if a["status"] == 0 and overlap(a, b))
    # surrogate trained on the outcomes of a separate batched sweep
    train = gated_specs(args.sweep_train, 1, lam)
    t0 = time.perf_counter()
    res_t, _ = sweep.run_channels(lbm, train, **ck)
    good = [k for k, r in enumerate(res_t) if r["status"] == 0]
    if len(good) < 4:
        raise RuntimeError("surrogate training sweep: fewer than four channels converged")
    x = np.stack([sweep.features(train[k]) for k in good])
    y = np.array([0.5 * np.log(res_t[k]["g_lo"] * res_t[k]["g_hi"]) for k in good])
    scale = (x.mean(axis=0), x.std(axis=0) + 1e-12)
    net = lbm.Surrogate(seed=0)
    net.train((x - scale[0]) / scale[1], y, epochs=400, batch=32, lr=2e-3, seed=0)
    t_train = time.perf_counter() - t0
    res_s, t_s = sweep.run_channels(lbm, specs, surrogate=net, scale_x=scale, **ck)
    net.close()
    ok_s = sum(r["status"] == 0 for r in res_s)
    both = [(a, b) for a, b in zip(res_s, res_b) if a["status"] == 0 and b["status"] == 0]
    g_b = np.array([math.sqrt(r["g_lo"] * r["g_hi"]) for r in res_b if r["status"] == 0])
    g_a = np.array([r["g_analytic"] for r in res_b if r["status"] == 0])
    per_b, per_s = t_b / max(ok_b, 1), t_s / max(ok_s, 1)
    rate_p = ok_p / t_p if t_p > 0 else 0.0
    return {"instances": len(specs), "lambda": lam, "bracket": "2 % (relative), device FP64 decisions",
            "t_eq": kw["t_eq"], "t_obs": kw["t_obs"],
            "window": "converged: doubling t_obs moves no bracket by more than one bisection step (lambda = 128)",
            "oracle_parity": parity,
            "wetting_calibration": {"seconds": t_cal, "r": table.r.tolist(),
                                    "theta_deg": [round(float(t), 2) for t in table.theta]},
            "start_bracket": "0.5-2x the planar 2-D critical force (plain and batched)",
            "lbm_over_analytic_median": float(np.median(g_b / g_a)) if g_b.size else None,
            "batched": {"solved": ok_b, "seconds": t_b, "solves_per_hour": 3600.0 * ok_b / t_b,
                        "mean_probes": float(np.mean([r["probes"] for r in res_b]))},
            "batched_fp16s": ({"solved": ok_h, "seconds": t_h, "solves_per_hour": 3600.0 * ok_h / t_h,
                               "brackets_overlapping_fp32": f"{sum(overlap(a, b) for a, b in both_h)}/{len(both_h)}"}
                              if args.sweep_fp16s else None),
            "plain_one_at_a_time": {"instances": n_p, "solved": ok_p, "seconds": t_p,
                                    "solves_per_hour": 3600.0 * rate_p,
                                    "brackets_equal_to_batched": f"{same_p}/{ok_p}",
                                    "mean_probes": float(np.mean([r["probes"] for r in res_p])) if res_p else None},
            "surrogate_seeded": {"solved": ok_s, "seconds": t_s, "solves_per_hour": 3600.0 * ok_s / t_s,
                                 "solves_per_hour_with_training": 3600.0 * ok_s / (t_s + t_train),
                                 "mean_probes": float(np.mean([r["probes"] for r in res_s])),
                                 "brackets_overlapping_batched_result": f"{sum(overlap(a, b) for a, b in both)}/{len(both)}",
                                 "training_sweep": len(train), "training_seconds": t_train,
                                 "break_even_solves": (t_train / (per_b - per_s)) if per_b > per_s else None},
            "speedup_batched_vs_plain": (ok_b / t_b) / max(rate_p, 1e-30),
            "speedup_seeded_vs_plain": (ok_s / t_s) / max(rate_p, 1e-30),
            "speedup_seeded_with_training_vs_plain": (ok_s / (t_s + t_train)) / max(rate_p, 1e-30)}


def forms_arm(args, w, peak, device, n_fluid):
    """The same workload in the other storage forms, each timed over
    args.forms_steps steps after 50 warm-up steps (the tuned kernel of each):
    FP32 with the compensated arithmetic (the form that meets the 1e-5
    velocity tolerance after 1000 steps), FP16- and BF16-shifted storage.
    GLUPS and the fraction of the measured copy rate at the form's own
    algorithmic bytes (144 B per fluid node for FP32, 72 B for the 16-bit
    forms)."""
    import torch
    from paper_1601_00918_gb300 import lbm
    stream = torch.cuda.current_stream()
    out = {}
    for prec in ("fp32c", "fp16s", "bf16s"):
        sim = lbm.Simulation(w.mask, w.rho, precision=prec, periodic=w.periodic, device=device, **PHYS)
        try:
            sim.step(50)
            kinfo = sim.kernel_info()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(args.forms_steps)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            assert sim.observables()["nan_flag"] == 0
        finally:
            sim.close()
        glups = n_fluid * args.forms_steps / (ms * 1e-3) / 1e9
        gbs = glups * 18 * 2 * BYTES_PER_POP[prec]
        out[prec] = {"value": glups, "unit": UNIT, "steps": args.forms_steps, "kernel": kinfo,
                     "achieved_gbs": gbs, "frac": gbs / peak, "dtype": DTYPE_NAME[prec]}
    return out


def e2e_arm(args, w, prec, device, n_fluid, repeats=3):
    """GLUPS through the C ABI with host buffers: lbm_create from pinned host
    arrays (H2D of mask and densities), then every step lbm_step(1) and
    lbm_observables (D2H of the observables), then lbm_get_fields (D2H of
    rho, u, p into pinned arrays) and lbm_destroy, all inside the timed
    region.  The whole job runs `repeats` times; the value is the median
    (a job lasts about 25 ms, so one host-side stall moves a single run by
    tens of per cent)."""
    runs = [e2e_once(args, w, prec, device, n_fluid) for _ in range(repeats)]
    out = dict(runs[0])
    vals = [r["value"] for r in runs]
    out["value"] = statistics.median(vals)
    out["runs"] = vals
    return out


def e2e_once(args, w, prec, device, n_fluid):
    """One end-to-end job (see e2e_arm)."""
    import torch
    from paper_1601_00918_gb300 import lbm
    ny, nx = w.mask.shape
    mask_h = torch.empty((ny, nx), dtype=torch.uint8, pin_memory=True).numpy()
    rho_h = torch.empty((2, ny, nx), dtype=torch.float64, pin_memory=True).numpy()
    mask_h[...] = w.mask
    rho_h[...] = w.rho
    # the fields come back into pinned arrays too (allocated, like the inputs,
    # before the timed region)
    out_h = (torch.empty((2, ny, nx), dtype=torch.float64, pin_memory=True).numpy(),
             torch.empty((2, ny, nx), dtype=torch.float64, pin_memory=True).numpy(),
             torch.empty((ny, nx), dtype=torch.float64, pin_memory=True).numpy())
    steps = max(1, min(args.steps, args.e2e_steps))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    p = lbm.make_params(nx, ny, periodic=w.periodic, precision=prec, variant=args.variant,
                        stream=torch.cuda.current_stream().cuda_stream, **PHYS)
    h = lbm.lbm_create(mask_h, rho_h, p)
    for _ in range(steps):
        lbm.lbm_step(h, 1)
        lbm.lbm_observables(h)
    lbm.lbm_get_fields(h, nx, ny, out=out_h)
    lbm.lbm_destroy(h)
    dt = time.perf_counter() - t0
    n = nx * ny
    h2d = n * (1 + 16)
    d2h = n * 40
    obs_bytes = 64
    return {"value": n_fluid * steps / dt / 1e9, "unit": UNIT, "steps": steps,
            "h2d_bytes_per_step": h2d / steps, "d2h_bytes_per_step": d2h / steps + obs_bytes,
            "timed": "lbm_create (H2D mask + rho) + steps x (lbm_step(1) + lbm_observables) "
                     "+ lbm_get_fields (D2H rho, u, p) + lbm_destroy"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precision", default="fp32", choices=list(BYTES_PER_POP))
    ap.add_argument("--variant", default="auto", choices=["auto", "simple", "staged", "pipelined", "private"])
    ap.add_argument("--e2e-steps", type=int, default=100)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweep-n", type=int, default=8, help="channels of the solves/hour sweep (0: skip)")
    ap.add_argument("--sweep-plain", type=int, default=1, help="channels bisected one at a time")
    ap.add_argument("--sweep-train", type=int, default=16, help="channels of the surrogate's training sweep")
    ap.add_argument("--sweep-fp16s", action="store_true", help="also run the batched sweep in FP16-shifted storage")
    ap.add_argument("--sweep-lam", type=int, default=128, help="wavelength of the sweep channels (128 or 256)")
    ap.add_argument("--batch-n", type=int, default=512, help="channels of the batched-step measurement (0: skip)")
    ap.add_argument("--batch-steps", type=int, default=160, help="timed steps of the batched-step measurement")
    ap.add_argument("--no-small", action="store_true", help="skip the small-grid latency lines")
    ap.add_argument("--d3-steps", type=int, default=200, help="timed steps of the D3Q19 tube line (0: skip)")
    ap.add_argument("--forms-steps", type=int, default=1000, help="timed steps of the other storage forms (0: skip)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return reference_arm(args)
    return native_arm(args)


if __name__ == "__main__":
    sys.exit(main())
