"""Throughput benchmark of the EHD lattice Boltzmann solver on GB300.

One step = one time step of all five lattice Boltzmann equations (with its 20
potential sweeps) on the 2048 x 2048 FP32 droplet case.  The state (~1.35 GB)
is larger than L2, so no flush is needed between steps.  Prints one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: the method has no cross-lattice exchange here, so N > 1 runs N
independent replicas (one lattice per rank, weak scaling, no collective on
the data path); value is the sum over ranks of node updates / the slowest
rank's time.  ``--impl reference`` times the FP64 CPU oracle on a 256 x 256
copy of the case (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS over 5 LB fields, % HBM roofline; served cases/h vs plain, p99 latency"
N = 2048
SWEEPS = 20
SAMPLE_N = 256          # oracle sample: a 256^2 copy of the case (R = 32)
TIMING_EVERY = 4        # kernel-class events on every 4th timed step
# Algorithmic bytes per node and potential sweep, 10 s + 8 with s bytes per
# stored population (5 populations read and written, phi and q read): 48 in
# FP32, 28 with FP16 storage.  This is the per-sweep unit of the byte model;
# one launch of the fused kernel processes sweeps_per_launch such units per
# node while its DRAM traffic is that of a single sweep.
def sweep_bytes_per_node(storage_bytes: int) -> int:
    return 10 * storage_bytes + 8


def prep_bytes_per_node(storage_bytes: int) -> int:
    """k_prep: h (9), p (5), n (5) populations read; phi, dphi (with ghost
    rows) and q written as float."""
    return 19 * storage_bytes + 12


def main_model_bytes(storage_bytes: int) -> int:
    """Byte model of the f, h, p, n update and the carried scalars (no
    sweeps): 56 s + 24 per node-step."""
    return 56 * storage_bytes + 24


def step_model_bytes(storage_bytes: int, sweeps: int) -> int:
    """Whole-step byte model of the unfused method: 56 s + 24 + (10 s + 8) S."""
    return 56 * storage_bytes + 24 + (10 * storage_bytes + 8) * sweeps


# bytes of the control block ehdlb_step reads back after every call (sums,
# residual, counters)
CONTROL_BYTES = 120
# steps of the end-to-end runs (fixed, whatever --steps is): one state upload
# then E2E_STEPS steps that each return the step's counters and D; and
# E2E_FIELD_STEPS steps that each read the phi field back
E2E_STEPS = 200
E2E_FIELD_STEPS = 100
# fused sweep kernel of each tile shape (ehdlb_set_tuning)
SWEEP_KERNELS = {
    0: ("k_sweep_tb", "potential sweeps fused in shared memory, 64 x 32 regions"),
    1: ("k_sweep_tb", "potential sweeps fused in shared memory, 64 x 32 regions"),
    2: ("k_sweep_cl", "potential sweeps fused across clusters of 2 x 4 blocks"),
    3: ("k_sweep_tb", "potential sweeps fused in shared memory, 64 x 64 regions"),
    4: ("k_sweep_tbr", "potential sweeps fused in registers, persistent, 64 x 32 regions"),
    5: ("k_sweep_tbr", "potential sweeps fused in registers, persistent, 64 x 40 regions"),
    6: ("k_sweep_tbr_fp", "potential sweeps fused in registers, 64 x 40 regions, the prep pass in the first launch"),
    7: ("k_sweep_tbw", "potential sweeps fused in registers, 64 x 40 regions walked down column strips"),
}

PRECISIONS = {"fp32": ("FP32", 4, "f32"), "fp16s": ("FP16 storage, FP32 arithmetic", 2, "f32"),
              "fp64": ("FP64", 8, "f64")}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n", type=int, default=N, help="lattice side (default: the 2048^2 case)")
    ap.add_argument("--sweeps-per-launch", type=int, default=-1,
                    help="potential sweeps fused per kernel launch (default: the library's)")
    ap.add_argument("--tile-shape", type=int, default=-1,
                    help="region shape of the fused sweep kernel (default: the library's)")
    ap.add_argument("--main-staging", type=int, default=-1,
                    help="step kernel staging, 0 per node, 1 16-byte segments (default: the library's)")
    ap.add_argument("--precision", default="fp32", choices=sorted(PRECISIONS),
                    help="fp32 (the headline form), fp16s (FP16 storage) or fp64")
    ap.add_argument("--mode", default="step", choices=["step", "batch", "serve", "cpu-probe"],
                    help="step: the 2048^2 case (the headline); batch: the 96 uneven cases, batched "
                         "against one by one; serve: a stream of arriving cases, continuous batching "
                         "against one by one")
    ap.add_argument("--probe", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--batch-steps", type=int, default=10000, help="steps per case in --mode batch")
    ap.add_argument("--serve-cases", type=int, default=300)
    ap.add_argument("--serve-max-steps", type=int, default=8000)
    ap.add_argument("--serve-load", type=float, default=3.5,
                    help="offered load as a multiple of the measured batch throughput, with each case's "
                         "work counted at the step cap")
    ap.add_argument("--serve-precision", default="fp16s", choices=["fp32", "fp16s"])
    return ap.parse_args()


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock and throttle sampling around the timed region: the
    sampler runs every 50 ms from before the region (its first sample read
    before the region starts) to after it; the summary takes the samples
    received inside the region, or, for a region shorter than the sampling
    period, the last one before it and the first one after it."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 50

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.lines: list[tuple[float, str]] = []
        self.proc = None
        self.first = threading.Event()
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", str(self.PERIOD_MS)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            self.first.wait(timeout=10.0)
        except OSError:
            self.proc = None
        return self

    def start(self):
        """Mark the start of the timed region."""
        self.t0 = time.monotonic()

    def stop(self):
        """Mark its end; let one more sample arrive."""
        self.t1 = time.monotonic()
        if self.proc:
            deadline = self.t1 + 3 * self.PERIOD_MS / 1e3
            while time.monotonic() < deadline and not any(t > self.t1 for t, _ in self.lines[-2:]):
                time.sleep(0.005)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))
            self.first.set()

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def _chosen(self):
        if self.t0 is None or self.t1 is None:
            return [ln for _, ln in self.lines], "all"
        inside = [ln for t, ln in self.lines if self.t0 <= t <= self.t1]
        if inside:
            return inside, "inside"
        before = [ln for t, ln in self.lines if t < self.t0][-1:]
        after = [ln for t, ln in self.lines if t > self.t1][:1]
        return before + after, "bracketing"

    def summary(self):
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines, how = self._chosen()
        for ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                mhz.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        region_ms = (self.t1 - self.t0) * 1e3 if self.t0 is not None and self.t1 is not None else None
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(mhz), "samples_taken": how,
                "period_ms": self.PERIOD_MS,
                "region_ms": round(region_ms, 1) if region_ms is not None else None}


def reduce_max(value: float, device) -> float:
    """Largest value over the ranks of the default process group (identity
    without one): the slowest replica sets the whole-job time."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(nodes: int, steps: int, world: int, seconds: float) -> float:
    """Whole-job MLUPS of `world` independent replicas of `nodes` lattice
    nodes each, `steps` steps in `seconds` (the slowest rank's time)."""
    return nodes * steps * world / seconds / 1e6


def kernel_source_digest() -> str | None:
    import hashlib
    try:
        with open(os.path.join(ROOT, "paper_2501_04920_gb300", "csrc", "ehdlb_kernels.cuh"), "rb") as f:
            return hashlib.sha256(f.read()).hexdigest()[:16]
    except OSError:
        return None


def profile_record(kernel: str, key: str):
    """A per-node figure of kernel (key: dram_bytes_per_node or
    warp_inst_per_node) from profiles/traffic.json, or None when the kernel
    source changed since the ncu capture it came from."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)[kernel]
    except (OSError, KeyError, ValueError):
        return None
    if rec.get("source_sha256_16") != kernel_source_digest():
        return None
    return rec.get(key)


def measured_traffic(kernel: str, n: int):
    """DRAM bytes per launch of kernel at n x n (ncu), or None."""
    v = profile_record(kernel, "dram_bytes_per_node")
    return v * n * n if v is not None else None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0}, "fallback"


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_probe(case: str, n: int, steps: int, budget_s: float) -> dict:
    """Time the FP64 oracle in this process: `steps` time steps of the case
    (at most budget_s seconds), after its set-up."""
    import oracle
    from paper_2501_04920_gb300 import workloads
    prm = workloads.droplet64() if case == "droplet64" else workloads.droplet(n)
    t0 = time.perf_counter()
    o = oracle.Oracle(n, n, prm)
    setup = time.perf_counter() - t0
    done, t0 = 0, time.perf_counter()
    while done < steps and (done == 0 or time.perf_counter() - t0 < budget_s):
        o.step(1)
        done += 1
    dt = time.perf_counter() - t0
    return {"case": case, "n": n, "steps": done, "seconds": dt, "setup_s": setup,
            "mlups": n * n * done / dt / 1e6}


def oracle_timing(case: str, n: int, steps: int, budget_s: float, threads: int) -> dict:
    """oracle_probe in a fresh process with `threads` OpenMP threads."""
    env = dict(os.environ, OMP_NUM_THREADS=str(threads))
    spec = json.dumps({"case": case, "n": n, "steps": steps, "budget": budget_s})
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--mode", "cpu-probe", "--probe", spec],
                       capture_output=True, text=True, env=env, timeout=budget_s * 4 + 600)
    if r.returncode != 0:
        raise RuntimeError(f"oracle timing failed: {r.stderr[-2000:]}")
    rec = json.loads(r.stdout.strip().splitlines()[-1])
    rec["threads"] = threads
    return rec


def cpu_baseline_block() -> dict:
    """The oracle on the host cores, bounded samples (about half a minute in
    all): the 256^2 copy of the 2048^2 case on all cores (the reported value)
    and on one core, the 64^2 FP64 case (2000 steps, residual-driven sweeps),
    and one step of the 2048^2 case itself, each extrapolated to its full
    step count where it was cut short."""
    cores = os.cpu_count() or 1
    allc = oracle_timing("droplet", SAMPLE_N, 1000, 10.0, cores)
    one = oracle_timing("droplet", SAMPLE_N, 1000, 6.0, 1)
    c1 = oracle_timing("droplet64", 64, 2000, 6.0, 1)
    big = oracle_timing("droplet", N, 1, 1.0, cores)
    full = {"droplet256": 20000, "droplet64": 2000, "droplet2048": 20000}
    return {
        "value": round(allc["mlups"], 4), "unit": "MLUPS", "cores": cores, "kind": "oracle",
        "sample": f"FP64 CPU oracle (OpenMP, {cores} threads), {SAMPLE_N}x{SAMPLE_N} copy of the 2048^2 case "
                  f"(R = {SAMPLE_N // 8}, {SWEEPS} sweeps/step), {allc['steps']} steps in {allc['seconds']:.1f} s",
        "cpu_model": cpu_model(),
        "single_thread": {"value": round(one["mlups"], 4), "unit": "MLUPS", "threads": 1,
                          "sample": f"{SAMPLE_N}x{SAMPLE_N} copy, {one['steps']} steps in {one['seconds']:.1f} s"},
        "droplet64": {"mlups": round(c1["mlups"], 4), "steps": c1["steps"], "seconds": round(c1["seconds"], 2),
                      "threads": 1, "full_steps": full["droplet64"],
                      "full_seconds": round(c1["seconds"] / c1["steps"] * full["droplet64"], 1),
                      "label": ("measured over all 2000 steps" if c1["steps"] >= full["droplet64"] else
                                f"extrapolated from {c1['steps']} steps"),
                      "workload": "64x64 FP64 case, sweeps to residual 1e-8 (cap 200)"},
        "droplet2048": {"mlups": round(big["mlups"], 4), "steps": big["steps"], "seconds": round(big["seconds"], 2),
                        "setup_s": round(big["setup_s"], 2), "threads": cores,
                        "full_hours": round(big["seconds"] / big["steps"] * full["droplet2048"] / 3600, 2),
                        "label": f"extrapolated from {big['steps']} step(s) to 20000 steps",
                        "workload": "the 2048x2048 case itself, 20 sweeps/step"},
        "droplet256_full_seconds": round(allc["seconds"] / allc["steps"] * full["droplet256"], 1),
    }


def workload_config(n: int, precision: str, world: int) -> dict:
    """The config of the timed workload (both arms report it)."""
    label, sbytes, _ = PRECISIONS[precision]
    return {"workload": f"droplet {n}x{n} {label}, 20 potential sweeps per step "
                        f"(R = {n // 8}, eps_r = 4, mu_r = 2, dpsi = 2)",
            "nx": n, "ny": n, "sweeps_per_step": SWEEPS, "storage_bytes": sbytes,
            "l2": "inputs larger than L2 (state ~1.35 GB), no flush",
            "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"}


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    # warm-up steps, then the timed steps, each one oracle time step on the sample
    import oracle
    from paper_2501_04920_gb300 import workloads
    n = SAMPLE_N
    o = oracle.Oracle(n, n, workloads.droplet(n))
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    value = n * n * args.steps / dt / 1e6
    sample = (f"FP64 CPU oracle on a {n}x{n} copy of the {args.n}^2 droplet case (R = {n // 8}, "
              f"{SWEEPS} sweeps/step), {args.steps} timed steps after {args.warmup} warm-up")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_config(args.n, args.precision, world),
                       sample=f"each timed step is one FP64 oracle step of the {n}x{n} copy (R = {n // 8}) "
                              f"on the host cores; MLUPS counts its nodes"),
        "cpu_baseline": {"value": round(value, 4), "unit": "MLUPS", "cores": threads,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    from paper_2501_04920_gb300 import ehdlb, workloads

    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    n = args.n
    prm = workloads.droplet(n)
    label, sbytes, dtype = PRECISIONS[args.precision]
    prec = {"fp32": ehdlb.FP32, "fp16s": ehdlb.FP16S, "fp64": ehdlb.FP64}[args.precision]
    lat = ehdlb.Lattice(n, n, prm, precision=prec, cuda_stream=stream.cuda_stream)
    ehdlb.ehdlb_set_tuning(lat.ctx, args.sweeps_per_launch, args.tile_shape, args.main_staging)
    nn = n * n

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    # warm-up
    lat.step(args.warmup)
    # per-class device times from CUDA events around the kernel classes of
    # every TIMING_EVERY-th timed step (the other steps run without events
    # between their kernels, which start as programmatic dependents)
    ehdlb.ehdlb_set_timing(lat.ctx, TIMING_EVERY)
    torch.cuda.synchronize(dev)
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize(dev)
        clk.start()
        ev0.record(stream)
        status, st = lat.step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        clk.stop()
    barrier()
    ms = reduce_max(ev0.elapsed_time(ev1), dev)
    value = replica_value(nn, args.steps, world, ms / 1e3)
    peaks, peak_kind = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    sm_mhz_peak = float(peaks.get("sm_max_mhz", 2070.0))
    sweep_kernel = SWEEP_KERNELS.get(int(st.tile_shape), SWEEP_KERNELS[1])
    launches = int(st.launches)
    ehdlb.ehdlb_set_timing(lat.ctx, False)
    clocks = clk.summary()
    sm_mhz = clocks["sm_mhz"] or sm_mhz_peak
    suffix = "" if args.precision == "fp32" else f"_{args.precision}"
    sweep_launches_per_step = max(1, st.sweep_launches) / args.steps
    sweeps_per_launch = SWEEPS / sweep_launches_per_step

    # Every kernel class of a step.  hbm: bytes per node of the byte model
    # (56 s + 24 for the f, h, p, n update and the carried scalars, s the
    # storage bytes of a population; 10 s + 8 per potential sweep) and the DRAM bytes ncu measured
    # for the current kernel source, each over the class's device time per
    # step, against the measured copy bandwidth.  The fused sweeps keep five
    # sweeps on chip per DRAM round trip, so their model bytes are no floor
    # for them: they are reported against the issue rate as well (warp
    # instructions ncu counted per node and launch, over 4 issue slots per SM
    # and clock at the sampled SM clock).
    def kernel_line(model_bytes_per_node, ms_per_step, key, launches_per_step=1.0):
        line = {"ms_per_step": round(ms_per_step, 4), "launches_per_step": round(launches_per_step, 3),
                "model_bytes_per_node": model_bytes_per_node}
        sec = ms_per_step / 1e3
        model_gbs = model_bytes_per_node * nn / sec / 1e9
        line["model_achieved"] = round(model_gbs, 1)
        line["model_frac"] = round(model_gbs / hbm, 4)
        dram = profile_record(key + suffix, "dram_bytes_per_node")
        if dram is not None:
            dram_gbs = dram * launches_per_step * nn / sec / 1e9
            line.update(dram_bytes_per_node=round(dram * launches_per_step, 1), dram_achieved=round(dram_gbs, 1),
                        dram_frac=round(dram_gbs / hbm, 4))
        inst = profile_record(key + suffix, "warp_inst_per_node")
        if inst is not None:
            rate = inst * launches_per_step * nn / sec          # warp instructions per second
            peak_issue = 4.0 * 152 * sm_mhz * 1e6
            line.update(warp_inst_per_node=round(inst * launches_per_step, 3),
                        issue_achieved_ginst_s=round(rate / 1e9, 1), issue_frac=round(rate / peak_issue, 4))
        return line

    kernel_ms = {"prep": st.ms_prep / args.steps, "sweeps": st.ms_sweeps / args.steps,
                 "main": st.ms_main / args.steps}
    roofline_kernels = {"unit": "GB/s", "peak": hbm, "peak_source": peak_kind,
                        "timed": f"CUDA events around the kernel classes of every {TIMING_EVERY}th timed step, "
                                 "scaled to all steps"}
    if kernel_ms["prep"] > 0:
        roofline_kernels["k_prep"] = kernel_line(prep_bytes_per_node(sbytes), kernel_ms["prep"], "k_prep")
    roofline_kernels[sweep_kernel[0]] = kernel_line(sweep_bytes_per_node(sbytes) * SWEEPS, kernel_ms["sweeps"],
                                                    sweep_kernel[0], sweep_launches_per_step)
    roofline_kernels[sweep_kernel[0]]["sweeps_per_launch"] = sweeps_per_launch
    roofline_kernels["k_main"] = kernel_line(main_model_bytes(sbytes), kernel_ms["main"], "k_main")
    step_model = step_model_bytes(sbytes, SWEEPS)
    roofline_kernels["step"] = {"model_bytes_per_node_step": step_model,
                                "model_achieved": round(step_model * value * 1e6 / world / 1e9, 1),
                                "model_frac": round(step_model * value * 1e6 / world / 1e9 / hbm, 4)}
    dram_step = [roofline_kernels[k].get("dram_bytes_per_node") for k in ("k_prep", sweep_kernel[0], "k_main")
                 if k in roofline_kernels]
    if all(v is not None for v in dram_step):
        tot = sum(dram_step)
        roofline_kernels["step"].update(dram_bytes_per_node_step=round(tot, 1),
                                        dram_frac=round(tot * value * 1e6 / world / 1e9 / hbm, 4))

    # The headline roofline: the step kernel, the longest launch of a step,
    # bound by HBM; algorithmic bytes per launch from the byte model.
    main_ms = kernel_ms["main"]
    main_alg = main_model_bytes(sbytes) * nn
    achieved = main_alg / (main_ms / 1e3) / 1e9
    traffic = measured_traffic("k_main" + suffix, n)
    roofline = {"bound": "hbm", "kernel": "k_main (reaction, forces, u, p, f/h/p/n collide and push)",
                "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s", "frac": round(achieved / hbm, 4),
                "peak_source": peak_kind, "traffic": traffic, "algorithmic_bytes_per_launch": main_alg,
                "algorithmic_bytes_per_node": main_model_bytes(sbytes), "launch_ms": round(main_ms, 4),
                "dram_achieved": round(traffic / (main_ms / 1e3) / 1e9, 1) if traffic else None,
                "dram_frac": round(traffic / (main_ms / 1e3) / 1e9 / hbm, 4) if traffic else None}

    # end to end through the public API with host buffers: the job's input,
    # a full state (35 doubles per node with D2Q5 ions) in pinned host memory,
    # goes to the device (ehdlb_set_state), then every step is one ehdlb_step
    # call that returns its control block (the step's sums and residual) and
    # the step's deformation factor D (Eq. 63, reduced on the device): the
    # per-step result a driver of the solver watches.  The reporting option
    # captures phi alone and computes D within the call.
    e2e_steps = E2E_STEPS
    state_len = ehdlb.ehdlb_state_len(lat.ctx)
    host_state = torch.empty(state_len, dtype=torch.float64).pin_memory()
    state_np = host_state.numpy()
    ehdlb.ehdlb_get_state(lat.ctx, state_np)
    torch.cuda.synchronize(dev)
    barrier()
    ehdlb.ehdlb_set_reporting(lat.ctx, 1 << ehdlb.FIELDS.index("phi"), 1)
    t0 = time.perf_counter()
    ehdlb.ehdlb_set_state(lat.ctx, state_np)
    for _ in range(e2e_steps):
        _, st_e = lat.step(1)
        d_last = st_e.deformation
    e2e_s = reduce_max(time.perf_counter() - t0, dev)
    ehdlb.ehdlb_set_reporting(lat.ctx, (1 << len(ehdlb.FIELDS)) - 1, 0)
    e2e_value = replica_value(nn, e2e_steps, world, e2e_s)
    state_bytes = 8 * state_len
    # the same with the whole phi field of every step read into pinned host memory
    host_phi = torch.empty(nn, dtype=torch.float64).pin_memory()
    phi_np = host_phi.numpy()
    fld_steps = E2E_FIELD_STEPS
    torch.cuda.synchronize(dev)
    barrier()
    t0 = time.perf_counter()
    for _ in range(fld_steps):
        lat.step(1)
        ehdlb.ehdlb_get_fields(lat.ctx, 1 << 0, phi_np)
    fld_s = reduce_max(time.perf_counter() - t0, dev)
    fld_value = replica_value(nn, fld_steps, world, fld_s)

    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline_block()
    out = {
        "metric": METRIC, "value": round(value, 2), "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
        "data": "synthetic",
        "config": workload_config(n, args.precision, world),
        "roofline": roofline,
        "roofline_kernels": roofline_kernels,
        "gpu_launches": launches,
        "kernel_ms": kernel_ms,
        "clocks": clocks,
        "status": ehdlb.STATUS_NAMES.get(status, status),
        "e2e": {"value": round(e2e_value, 2), "unit": "MLUPS", "steps": e2e_steps,
                "h2d_bytes_per_step": round(state_bytes / e2e_steps), "d2h_bytes_per_step": CONTROL_BYTES + 8,
                "input": f"the initial state, {state_bytes} bytes from pinned host memory (ehdlb_set_state), "
                         f"once per {e2e_steps} steps",
                "result": "per step: ehdlb_step(1) returning its control block (sum phi, sum q, residual) "
                          "and D of Eq. 63 (ehdlb_set_reporting: phi captured, D computed in the call)",
                "last_D": d_last},
        "e2e_fields": {"value": round(fld_value, 2), "unit": "MLUPS", "steps": fld_steps,
                       "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 8 * nn + CONTROL_BYTES,
                       "result": "per step: ehdlb_step(1) and the phi field (FP64) into pinned memory"},
    }
    if cpu:
        out["cpu_baseline"] = cpu
    print(json.dumps(out), flush=True)
    lat.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def run_batch(args):
    """Cases per hour of the 96 uneven cases, each run for its 10000 steps:
    one batch against the same cases run one at a time, both measured over
    the whole job (set-up, autotuning and every step) on the wall clock."""
    import torch
    from paper_2501_04920_gb300 import ehdlb, workloads
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    prec = {"fp32": ehdlb.FP32, "fp16s": ehdlb.FP16S}[args.precision]
    cases = workloads.uneven_cases()
    total_steps = args.batch_steps
    params = [ehdlb.ehdlb_params_from_physical(c["nx"], c["ny"], c["d_mm"], c["dpsi_kV"], c["eps_r"], c["mu_r"])
              for c in cases]
    budget = int(1.05 * sum(ehdlb.ehdlb_batch_footprint(prec, c["nx"], c["ny"]) for c in cases)) + (64 << 20)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        # batched: autotune on a scratch copy of the batch, then the job
        t0 = time.perf_counter()
        b = ehdlb.Batch(budget, 20, precision=prec)
        for c, p in zip(cases, params):
            b.add(c["nx"], c["ny"], p)
        spl, shape, tune_ms = b.autotune(3)
        b.close()
        b = ehdlb.Batch(budget, 20, precision=prec)
        for c, p in zip(cases, params):
            b.add(c["nx"], c["ny"], p)
        b.set_tuning(spl, shape)
        _, st = b.step(total_steps)
        assert st.unstable_cases == 0
        D_batch = b.deformation(list(range(len(cases))))
        b.close()
        total_b = time.perf_counter() - t0
        batch_mlups = st.mlups
        # one case at a time, the plain way
        t0 = time.perf_counter()
        D_plain = []
        for c, p in zip(cases, params):
            lat = ehdlb.Lattice(c["nx"], c["ny"], p, precision=prec)
            lat.step(total_steps)
            D_plain.append(lat.deformation())
            lat.close()
        total_p = time.perf_counter() - t0
    nodes = sum(c["nx"] * c["ny"] for c in cases)
    out = {
        "metric": "served cases/h vs plain (uneven batch)", "mode": "batch",
        "value": round(len(cases) * 3600 / total_b, 1), "unit": "cases/h", "n_gpus": 1,
        "steps_per_case": total_steps, "higher_is_better": True,
        "plain_value": round(len(cases) * 3600 / total_p, 1),
        "speedup_vs_plain": round(total_p / total_b, 3),
        "seconds": {"batched": round(total_b, 2), "plain": round(total_p, 2)},
        "batch_mlups": round(batch_mlups, 1),
        "D_equal_in_both_arms": bool(all(a == b_ for a, b_ in zip(D_batch, D_plain))),
        "autotune": {"sweeps_per_launch": spl, "tile_shape": shape, "ms_per_step": tune_ms},
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{len(cases)} uneven droplet cases (nx 128-768, ny in [nx, 2nx], physical "
                               f"mapping), {total_steps} steps each, 20 sweeps/step, "
                               f"{'FP16 storage' if args.precision == 'fp16s' else 'FP32'}",
                   "nodes": nodes, "timing": "wall clock of the whole job, measured (no projection)"},
        "clocks": clk.summary(),
    }
    print(json.dumps(out), flush=True)


def run_serve(args):
    """Continuous batching of a Poisson stream of cases against serving them
    one by one: latency percentiles and completed cases per hour.  The
    arrival rate is set from the batch's throughput measured first on a
    sample of the stream, so that the offered load exceeds what one GPU can
    serve and both arms are bound by their own throughput."""
    import torch
    from paper_2501_04920_gb300 import ehdlb, workloads
    from paper_2501_04920_gb300.serve import Case, Server, percentile, serve_one_by_one
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    n, max_steps, check = args.serve_cases, args.serve_max_steps, 1000
    prec_name = args.serve_precision
    prec = {"fp32": ehdlb.FP32, "fp16s": ehdlb.FP16S}[prec_name]
    raw = workloads.arrivals(n, rate_per_s=1.0)
    unit = [Case(t=0.0, nx=a["nx"], ny=a["ny"], d_mm=a["d_mm"], dpsi_kV=a["dpsi_kV"], eps_r=a["eps_r"],
                 mu_r=a["mu_r"], key=i) for i, a in enumerate(raw)]
    budget = 150 << 30
    # capacity: node updates per second of the batch on the first cases of
    # the stream (as many as the budget holds, at most 48), after autotuning
    b = ehdlb.Batch(budget, 20, precision=prec)
    for c in unit[:48]:
        if b.add(c.nx, c.ny, c.params(20)) is None:
            break
    spl, shape, _ = b.autotune(3)
    b.step(20)
    cap_steps = 200
    _, st = b.step(cap_steps)
    capacity = st.mlups * 1e6
    b.close()
    # offered load: load_factor x capacity, counting each case's work as
    # nodes x max_steps (an upper bound: steady cases stop earlier)
    mean_work = sum(c.nx * c.ny for c in unit) / n * max_steps
    rate = args.serve_load * capacity / mean_work
    cases = [Case(t=a["t"] / rate, nx=c.nx, ny=c.ny, d_mm=c.d_mm, dpsi_kV=c.dpsi_kV, eps_r=c.eps_r,
                  mu_r=c.mu_r, key=c.key) for a, c in zip(raw, unit)]
    b = ehdlb.Batch(budget, 20, precision=prec)
    b.set_tuning(spl, shape)
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        res = Server(b, check_every=check, max_steps=max_steps, tol=1e-6).run(cases)
        span_b = time.perf_counter() - t0
    b.close()
    t0 = time.perf_counter()
    res_p = serve_one_by_one(cases, check_every=check, max_steps=max_steps, tol=1e-6, precision=prec)
    span_p = time.perf_counter() - t0
    lb, lp = [r.latency for r in res], [r.latency for r in res_p]
    done_work = sum(unit[r.key].nx * unit[r.key].ny * r.steps for r in res)
    arrival_span = cases[-1].t if cases else 0.0
    same = all(a.steps == b_.steps for a, b_ in zip(sorted(res, key=lambda r: r.key),
                                                    sorted(res_p, key=lambda r: r.key)))
    out = {
        "metric": "served cases/h vs plain, p99 latency (continuous batching)", "mode": "serve",
        "value": round(n * 3600 / span_b, 1), "unit": "cases/h", "n_gpus": 1, "higher_is_better": True,
        "plain_value": round(n * 3600 / span_p, 1), "speedup_vs_plain": round(span_p / span_b, 3),
        "latency_s": {"p50": percentile(lb, 50), "p99": percentile(lb, 99)},
        "plain_latency_s": {"p50": percentile(lp, 50), "p99": percentile(lp, 99)},
        "steady_fraction": sum(r.steady for r in res) / n,
        "steps_equal_in_both_arms": same,
        "capacity_mlups": round(capacity / 1e6, 1),
        "offered_load": {"factor_of_capacity_at_max_steps": args.serve_load,
                         "actual_factor": round(done_work / max(arrival_span, 1e-9) / capacity, 3),
                         "rate_per_s": rate},
        "dtype": "f32", "data": "synthetic", "storage": prec_name,
        "autotune": {"sweeps_per_launch": spl, "tile_shape": shape},
        "config": {"workload": f"{n} Poisson arrivals, square sides 128*8^U rounded to 64, physical "
                               f"parameters as the uneven batch; steady when |D(t) - D(t - {check})| / {check} "
                               f"< 1e-6, at most {max_steps} steps; budget 150 GB; "
                               f"{'FP16 storage' if prec_name == 'fp16s' else 'FP32'}",
                   "arrivals": n, "max_steps": max_steps},
        "clocks": clk.summary(),
    }
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.mode == "cpu-probe":
        p = json.loads(args.probe)
        print(json.dumps(oracle_probe(p["case"], p["n"], p["steps"], p["budget"])), flush=True)
    elif args.impl == "reference":
        run_reference(args)
    elif args.mode == "batch":
        run_batch(args)
    elif args.mode == "serve":
        run_serve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
