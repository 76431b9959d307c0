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


def main_bytes_per_node(storage_bytes: int) -> int:
    """k_main: f (8), h (9), p (5), n (5) read and written, (phi u)(t-1)
    read and written, g (4 float) read, dphi, phi_ref, grad phi_ref (2) and
    mu_ref read as float."""
    return 2 * 27 * storage_bytes + 2 * 2 * storage_bytes + 16 + 20


def step_model_bytes(storage_bytes: int, sweeps: int) -> int:
    """Whole-step byte model of the unfused method: 56 s + 24 + (10 s + 8) S."""
    return 56 * storage_bytes + 24 + (10 * storage_bytes + 8) * sweeps


# bytes of the control block ehdlb_step reads back after every call (sums,
# residual, counters)
CONTROL_BYTES = 120
# fused sweep kernel of each tile shape (ehdlb_set_tuning)
SWEEP_KERNELS = {
    0: ("k_sweep_tb", "potential sweeps fused in shared memory, 64 x 32 regions"),
    1: ("k_sweep_tb", "potential sweeps fused in shared memory, 64 x 32 regions"),
    2: ("k_sweep_cl", "potential sweeps fused across clusters of 2 x 4 blocks"),
    3: ("k_sweep_tb", "potential sweeps fused in shared memory, 64 x 64 regions"),
    4: ("k_sweep_tbr", "potential sweeps fused in registers, persistent, 64 x 32 regions"),
    5: ("k_sweep_tbr", "potential sweeps fused in registers, persistent, 64 x 40 regions"),
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
    ap.add_argument("--mode", default="step", choices=["step", "batch", "serve"],
                    help="step: the 2048^2 case (the headline); batch: the 96 uneven cases, batched "
                         "against one by one; serve: a stream of arriving cases, continuous batching "
                         "against one by one")
    ap.add_argument("--serve-cases", type=int, default=64)
    ap.add_argument("--serve-max-steps", type=int, default=4000)
    return ap.parse_args()


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock and throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.lines: list[str] = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
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
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(mhz)}


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


def measured_traffic(kernel: str, n: int):
    """DRAM bytes per launch of kernel at n x n from profiles/traffic.json,
    or None when the kernel source changed since the capture."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)[kernel]
        src = os.path.join(ROOT, "paper_2501_04920_gb300", "csrc", "ehdlb_kernels.cuh")
        with open(src, "rb") as f:
            digest = hashlib.sha256(f.read()).hexdigest()[:16]
    except (OSError, KeyError, ValueError):
        return None
    if rec.get("source_sha256_16") != digest:
        return None
    return rec["dram_bytes_per_node"] * n * n


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0}, "fallback"


def oracle_rate(n: int, steps: int, budget_s: float):
    """FP64 oracle on an n x n copy of the case: (MLUPS, steps run, seconds, threads)."""
    import oracle
    from paper_2501_04920_gb300 import workloads
    o = oracle.Oracle(n, n, workloads.droplet(n))
    done, t0 = 0, time.perf_counter()
    while done < steps:
        o.step(1)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return n * n * done / dt / 1e6, done, dt, threads


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
        "config": workload_config(args.n, args.precision, world),
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
    ehdlb.ehdlb_set_timing(lat.ctx, True)
    torch.cuda.synchronize(dev)
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize(dev)
        ev0.record(stream)
        status, st = lat.step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
    barrier()
    ms = reduce_max(ev0.elapsed_time(ev1), dev)
    value = replica_value(nn, args.steps, world, ms / 1e3)
    sweep_launch_ms = st.ms_sweeps / max(1, st.sweep_launches)
    sweeps_per_launch = args.steps * SWEEPS / max(1, st.sweep_launches)
    peaks, peak_kind = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    unit_bytes = sweep_bytes_per_node(sbytes)
    achieved = unit_bytes * sweeps_per_launch * nn / (sweep_launch_ms / 1e3) / 1e9
    sweep_kernel = SWEEP_KERNELS.get(int(st.tile_shape), SWEEP_KERNELS[1])
    tkey = sweep_kernel[0] if args.precision == "fp32" else f"{sweep_kernel[0]}_{args.precision}"
    traffic = measured_traffic(tkey, n)
    launches = int(st.launches)
    ehdlb.ehdlb_set_timing(lat.ctx, False)

    # every kernel class of a step against the measured copy bandwidth:
    # algorithmic bytes per step / device time per step, and the DRAM bytes
    # ncu measured for it (profiles/traffic.json) while its source is unchanged
    launches_per_step = max(1, st.sweep_launches) / args.steps
    suffix = "" if args.precision == "fp32" else f"_{args.precision}"

    def kernel_line(alg_bytes_per_node, ms_per_step, dram_key, dram_launches=1.0):
        achieved_k = alg_bytes_per_node * nn / (ms_per_step / 1e3) / 1e9
        t = measured_traffic(dram_key + suffix, n)
        return {"algorithmic_bytes_per_node": alg_bytes_per_node, "ms_per_step": round(ms_per_step, 4),
                "achieved": round(achieved_k, 1), "frac": round(achieved_k / hbm, 4),
                "dram_bytes_per_node": (round(t * dram_launches / nn, 1) if t else None)}

    roofline_kernels = {
        "unit": "GB/s", "peak": hbm,
        "k_prep": kernel_line(prep_bytes_per_node(sbytes), st.ms_prep / args.steps, "k_prep"),
        sweep_kernel[0]: kernel_line(unit_bytes * SWEEPS, st.ms_sweeps / args.steps, sweep_kernel[0],
                                     launches_per_step),
        "k_main": kernel_line(main_bytes_per_node(sbytes), st.ms_main / args.steps, "k_main"),
        "step": {"model_bytes_per_node_step": step_model_bytes(sbytes, SWEEPS),
                 "achieved": round(step_model_bytes(sbytes, SWEEPS) * value * 1e6 / world / 1e9, 1),
                 "frac": round(step_model_bytes(sbytes, SWEEPS) * value * 1e6 / world / 1e9 / hbm, 4)},
    }

    # end to end through the public API with host buffers: the job's input,
    # a full state (35 doubles per node with D2Q5 ions) in pinned host memory,
    # goes to the device (ehdlb_set_state), then every step is one ehdlb_step
    # call that returns its control block (the step's sums and residual) and
    # the step's deformation factor D (Eq. 63, reduced on the device): the
    # per-step result a driver of the solver watches.  The reporting option
    # captures phi alone and computes D within the call.
    e2e_steps = max(10, args.steps // 3)
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
    fld_steps = max(10, args.steps // 6)
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
        rate, done, dt, threads = oracle_rate(SAMPLE_N, 1000, 12.0)
        cpu = {"value": round(rate, 4), "unit": "MLUPS", "cores": threads, "kind": "oracle",
               "sample": f"FP64 CPU oracle, {SAMPLE_N}x{SAMPLE_N} copy of the case "
                         f"(R = {SAMPLE_N // 8}, {SWEEPS} sweeps/step), {done} steps in {dt:.1f} s"}
    out = {
        "metric": METRIC, "value": round(value, 2), "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
        "data": "synthetic",
        "config": workload_config(n, args.precision, world),
        "roofline": {"bound": "hbm", "kernel": f"{sweep_kernel[0]} ({sweep_kernel[1]})",
                     "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                     "frac": round(achieved / hbm, 4), "peak_source": peak_kind,
                     "traffic": traffic,
                     "bytes_per_launch": unit_bytes * sweeps_per_launch * nn,
                     "sweeps_per_launch": sweeps_per_launch, "launch_ms": sweep_launch_ms,
                     "dram_achieved": (round(traffic / (sweep_launch_ms / 1e3) / 1e9, 1)
                                       if traffic else None)},
        "roofline_kernels": roofline_kernels,
        "gpu_launches": launches,
        "kernel_ms": {"prep": st.ms_prep / args.steps, "sweeps": st.ms_sweeps / args.steps,
                      "main": st.ms_main / args.steps},
        "clocks": clk.summary(),
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
    """Cases per hour of the 96 uneven cases (10000 steps each): one batch
    against the same cases run one at a time."""
    import torch
    from paper_2501_04920_gb300 import ehdlb, workloads
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    prec = {"fp32": ehdlb.FP32, "fp16s": ehdlb.FP16S}[args.precision]
    cases = workloads.uneven_cases()
    total_steps = workloads.STEPS["uneven"]
    params = [ehdlb.ehdlb_params_from_physical(c["nx"], c["ny"], c["d_mm"], c["dpsi_kV"], c["eps_r"], c["mu_r"])
              for c in cases]
    budget = int(1.05 * sum(ehdlb.ehdlb_batch_footprint(prec, c["nx"], c["ny"]) for c in cases)) + (64 << 20)
    # autotune on a scratch copy of the batch
    b = ehdlb.Batch(budget, 20, precision=prec)
    for c, p in zip(cases, params):
        b.add(c["nx"], c["ny"], p)
    spl, shape, tune_ms = b.autotune(3)
    b.close()
    # the timed batch
    t0 = time.perf_counter()
    b = ehdlb.Batch(budget, 20, precision=prec)
    for c, p in zip(cases, params):
        b.add(c["nx"], c["ny"], p)
    b.set_tuning(spl, shape)
    setup_b = time.perf_counter() - t0
    b.step(max(3, args.warmup))
    with ClockSampler(local) as clk:
        _, st = b.step(args.steps)
    per_step_b = st.device_ms / 1e3 / args.steps
    batch_mlups = st.mlups
    b.close()
    total_b = setup_b + per_step_b * total_steps
    # one case at a time
    total_p, k = 0.0, 20
    for c, p in zip(cases, params):
        t0 = time.perf_counter()
        lat = ehdlb.Lattice(c["nx"], c["ny"], p, precision=prec)
        setup = time.perf_counter() - t0
        lat.step(2)
        _, s1 = lat.step(k)
        total_p += setup + s1.seconds / k * total_steps
        lat.close()
    nodes = sum(c["nx"] * c["ny"] for c in cases)
    out = {
        "metric": "served cases/h vs plain (uneven batch)", "mode": "batch",
        "value": round(len(cases) * 3600 / total_b, 1), "unit": "cases/h", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
        "plain_value": round(len(cases) * 3600 / total_p, 1),
        "speedup_vs_plain": round(total_p / total_b, 3),
        "ms_per_batch_step": per_step_b * 1e3, "batch_mlups": round(batch_mlups, 1),
        "autotune": {"sweeps_per_launch": spl, "tile_shape": shape, "ms_per_step": tune_ms},
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{len(cases)} uneven droplet cases (nx 128-768, ny in [nx, 2nx], physical "
                               f"mapping), {total_steps} steps each, 20 sweeps/step, "
                               f"{'FP16 storage' if args.precision == 'fp16s' else 'FP32'}",
                   "nodes": nodes, "projection": f"setup + {total_steps} x measured time per step"},
        "clocks": clk.summary(),
    }
    print(json.dumps(out), flush=True)


def run_serve(args):
    """Continuous batching of a Poisson stream of cases against serving them
    one by one: latency percentiles and completed cases per hour."""
    import torch
    from paper_2501_04920_gb300 import ehdlb, workloads
    from paper_2501_04920_gb300.serve import Case, Server, percentile, serve_one_by_one
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    n, max_steps, check = args.serve_cases, args.serve_max_steps, 500
    raw = workloads.arrivals(n, rate_per_s=1.0)
    # offered load ~1.2x the batch's capacity at the throughput of the
    # 2048^2 case: rate = 1.2 * node updates per s / mean node updates per case
    mean_work = sum(a["nx"] * a["ny"] for a in raw) / n * max_steps
    rate = 1.2 * 6.5e9 / mean_work
    cases = [Case(t=a["t"] / rate, nx=a["nx"], ny=a["ny"], d_mm=a["d_mm"], dpsi_kV=a["dpsi_kV"],
                  eps_r=a["eps_r"], mu_r=a["mu_r"], key=i) for i, a in enumerate(raw)]
    budget = 150 << 30
    b = ehdlb.Batch(budget, 20)
    t0 = time.perf_counter()
    res = Server(b, check_every=check, max_steps=max_steps, tol=1e-6).run(cases)
    span_b = time.perf_counter() - t0
    b.close()
    t0 = time.perf_counter()
    res_p = serve_one_by_one(cases, check_every=check, max_steps=max_steps, tol=1e-6)
    span_p = time.perf_counter() - t0
    lb, lp = [r.latency for r in res], [r.latency for r in res_p]
    out = {
        "metric": "served cases/h vs plain, p99 latency (continuous batching)", "mode": "serve",
        "value": round(n * 3600 / span_b, 1), "unit": "cases/h", "n_gpus": 1, "higher_is_better": True,
        "plain_value": round(n * 3600 / span_p, 1), "speedup_vs_plain": round(span_p / span_b, 3),
        "latency_s": {"p50": percentile(lb, 50), "p99": percentile(lb, 99)},
        "plain_latency_s": {"p50": percentile(lp, 50), "p99": percentile(lp, 99)},
        "steady_fraction": sum(r.steady for r in res) / n,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{n} Poisson arrivals at {rate:.3f}/s (offered ~1.2x capacity), square "
                               f"sides 128*8^U rounded to 64, physical parameters as the uneven batch; "
                               f"steady when |dD|/{check} steps < 1e-6, at most {max_steps} steps; "
                               f"budget 150 GB", "rate_per_s": rate},
    }
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "batch":
        run_batch(args)
    elif args.mode == "serve":
        run_serve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
