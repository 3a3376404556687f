"""Benchmark of the multipath Metropolis hot path on one node.

A step is one full multipath run of the benchmark workload: simple cubic
L=16 (4096 spins), J=1, h=0, 21 temperatures uniformly spaced in [0.5, 2.5],
4096 independent paths per temperature, 2000 thermalisation + 2000
measurement checkerboard sweeps, FP32 spins in shared memory with FP64
accumulators, then the FP64 cross-path reduction.  Inputs are synthetic
(random unit-spin lattices drawn from Philox inside the kernel).

value: spin-update attempts/s over all ranks (N x paths x sweeps x systems /
device time of the timed steps, max over ranks).  Each rank runs its own full
workload (weak scaling; paths of different ranks use different seeds; no
collective on the data path).

--impl reference times the FP64 CPU oracle (the reference arm of this
project) on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("spin-update attempts/s and independent path samples/s at stated σ "
          "vs FP64 GPU form")
L, N_T, PATHS, N_THERM, N_MEAS = 16, 21, 4096, 2000, 2000
TEMPS = [0.5 + 2.0 * k / (N_T - 1) for k in range(N_T)]
N_SITES = L ** 3
SWEEPS = N_THERM + N_MEAS
WORKLOAD = (f"simple cubic L={L} periodic, J=1, h=0, {N_T} temperatures in [0.5,2.5], "
            f"{PATHS} paths per temperature, {N_THERM}+{N_MEAS} checkerboard sweeps, "
            "FP32 spins in shared memory, FP64 accumulators and reduction")
# Algorithmic lane operations of one Metropolis attempt on this path:
# Philox4x32-10 40 (10 rounds x 2 wide multiplies + 2 three-input xors),
# 3 uniforms 6, trial direction 9 (z, sqrt via rsqrt, phi, sin, cos, x, y),
# own spin 3 loads, local field 33 (18 neighbour loads + 15 adds),
# dE 8, accept 5 (scale, exp, two compares, select), store 3,
# measurement 2 (about 4.5 on the half of the sweeps that measure).
OPS_PER_ATTEMPT = 109
CPU_SAMPLE_PATHS = 2        # oracle paths per temperature in the CPU baseline
REF_STEP_PATHS = 1          # oracle paths per temperature per reference-arm step


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def oracle_sample(paths_per_T: int, threads: int | None = None):
    """Run the FP64 oracle on `paths_per_T` paths of every temperature; returns (attempts, seconds)."""
    import oracle

    oracle.build()
    systems = [oracle.System(L, T, n_paths=PATHS, path_begin=0, path_count=paths_per_T) for T in TEMPS]
    t0 = time.perf_counter()
    oracle.run(systems, N_THERM, N_MEAS, seed=1, threads=threads)
    dt = time.perf_counter() - t0
    return N_SITES * paths_per_T * N_T * SWEEPS, dt


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", gpu_id, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[5:9]):
                if flag.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "power_w_max": max(power), "reasons": sorted(reasons)}


def emit(obj):
    print(json.dumps(obj), flush=True)


def run_reference(args, rank):
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle_sample(REF_STEP_PATHS, cores)
    total_att, total_s = 0, 0.0
    for _ in range(args.steps):
        att, dt = oracle_sample(REF_STEP_PATHS, cores)
        total_att += att
        total_s += dt
    value = total_att / total_s
    sample = (f"{REF_STEP_PATHS} path per temperature x {N_T} temperatures x {SWEEPS} sweeps "
              f"of L={L} per step (FP64 oracle, {cores} threads)")
    emit({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "attempts/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": value, "unit": "attempts/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "attempts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    })


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    # shorter runs of the same launch (for profiling captures only)
    ap.add_argument("--n-therm", type=int, default=N_THERM)
    ap.add_argument("--n-meas", type=int, default=N_MEAS)
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch

    import __graft_entry__

    __graft_entry__.build()
    import paper_1305_6758_gb300 as mp

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    seed = 1 + rank
    n_therm, n_meas = args.n_therm, args.n_meas
    sweeps = n_therm + n_meas
    systems = [mp.System(L, T, n_paths=PATHS) for T in TEMPS]
    sim = mp.Simulation(systems, n_therm, n_meas, seed=seed, precision=mp.FP32, device=dev)
    stream = sim.stream
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2

    for _ in range(args.warmup):
        sim.run()
    barrier()

    props = torch.cuda.get_device_properties(dev)
    gpu_id = str(getattr(props, "uuid", local_rank))
    if gpu_id and not gpu_id.startswith("GPU-") and len(gpu_id) == 36:
        gpu_id = "GPU-" + gpu_id
    clocks = ClockSampler(gpu_id)
    step_ms, sweep_ms, reduce_ms = [], [], []
    barrier()
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.run()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        a, b = sim.timing()
        sweep_ms.append(a)
        reduce_ms.append(b)
    barrier()
    clk = clocks.stop()

    total_ms = sum(step_ms)
    if dist is not None:
        t = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = t.item()
    attempts_rank = N_SITES * PATHS * N_T * sweeps
    value = attempts_rank * world * args.steps / (total_ms / 1e3)
    paths_per_s = PATHS * N_T * world * args.steps / (total_ms / 1e3)
    ests = [sim.estimates(k) for k in range(N_T)]

    # end to end through the public API: create (system and work tables H2D),
    # run, read every system's estimates (D2H), destroy -- all inside the clock
    e2e_s = []
    import ctypes

    h2d = ctypes.sizeof(mp.MPSystem) * N_T  # the caller's system table
    for k in range(max(1, min(2, args.steps))):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        with mp.Simulation(systems, n_therm, n_meas, seed=seed + 1000 * (k + 1), device=dev) as s2:
            s2.run()
            for j in range(N_T):
                s2.estimates(j)
            plan = s2.plan()
        e2e_s.append(time.perf_counter() - t0)
    # the library uploads its DevSystem (80 B) and WorkItem (16 B) tables too
    h2d_total = h2d + 80 * N_T + 16 * plan["n_items"] + 8 * N_T
    d2h_total = ctypes.sizeof(mp.MPEstimates) * N_T
    e2e_value = attempts_rank * world / (sum(e2e_s) / len(e2e_s))

    peaks, peak_kind = load_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = props.multi_processor_count
    peak_ops = n_sm * 128 * sm_max * 1e6 / 1e12  # lane-ops/s in units of 1e12
    sweep_avg = sum(sweep_ms) / len(sweep_ms)
    achieved = OPS_PER_ATTEMPT * attempts_rank / (sweep_avg / 1e3) / 1e12

    fp64 = None
    if not args.no_fp64:
        sub = 64
        with mp.Simulation([mp.System(L, T, n_paths=sub) for T in TEMPS], n_therm, n_meas, seed=seed,
                           precision=mp.FP64, device=dev) as s64:
            s64.run()
            torch.cuda.synchronize(dev)
            a64, _ = s64.timing()
            e64 = [s64.estimates(k) for k in range(N_T)]
        att64 = N_SITES * sub * N_T * sweeps
        v64 = att64 / (a64 / 1e3)
        worst = max(abs(ests[k]["e"] - e64[k]["e"]) / (ests[k]["e_se"] ** 2 + e64[k]["e_se"] ** 2) ** 0.5
                    for k in range(N_T))
        fp64 = {"value": v64, "unit": "attempts/s", "sample": f"{sub} paths per temperature, same sweeps",
                "fp32_over_fp64": (attempts_rank / (sweep_avg / 1e3)) / v64,
                "max_e_diff_in_combined_se": worst}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        att, dt = oracle_sample(CPU_SAMPLE_PATHS, cores)
        cpu = {"value": att / dt, "unit": "attempts/s", "cores": cores, "kind": "oracle",
               "sample": f"{CPU_SAMPLE_PATHS} paths per temperature x {N_T} temperatures x {SWEEPS} sweeps "
                         f"of L={L} ({att:.3g} attempts, {dt:.1f} s)"}

    if rank == 0:
        emit({
            "metric": METRIC, "value": value, "unit": "attempts/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "L": L, "temperatures": N_T, "paths_per_temperature": PATHS,
                       "n_therm": n_therm, "n_meas": n_meas, "parallelism": f"replicas x{world}",
                       "l2": "flushed between timed steps (256 MB write)", "plan": sim.plan()},
            "paths_per_s": paths_per_s,
            "sigma": {"e_se_max": max(e["e_se"] for e in ests), "m_se_max": max(e["m_se"] for e in ests),
                      "e_at_T": {f"{TEMPS[k]:.1f}": [ests[k]["e"], ests[k]["e_se"]] for k in (0, 10, 20)}},
            "fp64_form": fp64,
            "e2e": {"value": e2e_value, "unit": "attempts/s", "h2d_bytes_per_step": h2d_total,
                    "d2h_bytes_per_step": d2h_total},
            "gpu_launches": 2 * args.steps,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_ops, "unit": "Tops/s",
                         "frac": achieved / peak_ops, "traffic": None,
                         "kernel": "sweep_kernel<float>", "ops_per_attempt": OPS_PER_ATTEMPT,
                         "peak_basis": f"{n_sm} SMs x 128 lanes x {sm_max:.0f} MHz ({peak_kind} max clock)",
                         "sweep_ms": sweep_avg, "reduce_ms": sum(reduce_ms) / len(reduce_ms)},
            "cpu_baseline": cpu,
            "clocks": clk,
        })
    sim.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
