"""Benchmark of the multipath Metropolis hot path on one node.

A step is one full multipath run of a workload: every path of every system
from its random initial state through its thermalisation and measurement
sweeps, then the FP64 cross-path reduction.  Inputs are synthetic (random
unit-spin lattices drawn from Philox inside the kernels).  Workloads:

  sc16     (default) simple cubic L=16 (4096 spins), J=1, h=0, 21 temperatures
           uniformly spaced in [0.5, 2.5], 4096 paths per temperature,
           2000 thermalisation + 2000 measurement sweeps, FP32 spins in shared
           memory, FP64 accumulators.
  large    simple cubic L=64 (262144 spins), T in {1.40, 1.44, 1.48}, 1024 paths
           each, 500 + 1000 sweeps, FP32 spins streamed from HBM.
  batched  uneven sizes in one persistent launch: L in {8,12,16,20,24,32} with
           8192/4096/2048/1024/512/256 paths, T=1.44, 1000 + 1000 sweeps, FP32.
  plain    simple cubic L=4, T=1.5, 256 paths, 1000 + 1000 sweeps, FP64.
  ising    Appendix A: square-lattice Ising L=60, T in {1.0, 2.0, 2.269, 3.0},
           10^4 paths each, 10^4 + 2x10^4 sweeps (3x10^4 as in the appendix).
  random   the paper's literal order (N attempts at random sites per sweep):
           simple cubic L=10, T=1.0, 10^4 paths, 500 + 500 sweeps, FP32.

value: spin-update attempts/s over all ranks (sites x paths x sweeps /
device time of the timed steps, max over ranks).  Each rank runs a full
workload's worth of paths, path ids rank x P .. (rank + 1) x P - 1 of every
system with the same seed, so N ranks form one ensemble of N x P paths per
system (weak scaling; no collective on the data path; rank_path_range and
gather_records below, with mp_reduce, turn the ranks' records into that
ensemble's estimates).

--impl reference times the FP64 CPU oracle (this project's reference arm) on
a bounded sample of the same workload on the host cores.
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
TEMPS21 = [0.5 + 2.0 * k / 20 for k in range(21)]

WORKLOADS = {
    "sc16": dict(
        systems=[(16, T, 4096) for T in TEMPS21], n_therm=2000, n_meas=2000, precision="fp32",
        bound="alu", cpu_paths=6, ref_paths=1, fp64_paths=64,
        text=("simple cubic L=16 periodic, J=1, h=0, 21 temperatures in [0.5,2.5], 4096 paths per "
              "temperature, 2000+2000 checkerboard sweeps, FP32 spins in shared memory, FP64 "
              "accumulators and reduction")),
    "large": dict(
        systems=[(64, T, 1024) for T in (1.40, 1.44, 1.48)], n_therm=500, n_meas=1000,
        precision="fp32", bound="hbm", cpu_paths=1, ref_paths=1, fp64_paths=0,
        text=("simple cubic L=64 periodic, J=1, h=0, T in {1.40,1.44,1.48}, 1024 paths each, "
              "500+1000 checkerboard sweeps, FP32 spins streamed from HBM through TMA-staged "
              "half-plane buffers")),
    "batched": dict(
        systems=[(Lb, 1.44, P) for Lb, P in ((8, 8192), (12, 4096), (16, 2048), (20, 1024), (24, 512),
                                             (32, 256))],
        n_therm=1000, n_meas=1000, precision="fp32", bound="alu", cpu_paths=1, ref_paths=1,
        fp64_paths=0,
        text=("uneven sizes in one persistent launch: simple cubic L in {8,12,16,20,24,32} with "
              "8192/4096/2048/1024/512/256 paths, T=1.44, J=1, h=0, 1000+1000 sweeps, FP32 spins, "
              "FP64 reductions")),
    "plain": dict(
        systems=[(4, 1.5, 256)], n_therm=1000, n_meas=1000, precision="fp64", bound="alu",
        cpu_paths=256, ref_paths=16, fp64_paths=0,
        text=("plain method, FP64: simple cubic L=4, J=1, h=0, T=1.5, 256 paths, 1000+1000 "
              "checkerboard sweeps")),
    "ising": dict(
        systems=[(60, T, 10000, "ising") for T in (1.0, 2.0, 2.269, 3.0)], n_therm=10000,
        n_meas=20000, precision="fp32", bound="alu_ising", cpu_paths=1, ref_paths=1, fp64_paths=0,
        text=("square-lattice Ising L=60 periodic (Appendix A), J=1, h=0, T in {1.0,2.0,2.269,3.0}, "
              "10^4 paths each, 10^4+2x10^4 checkerboard sweeps, byte spins in shared memory, "
              "integer acceptance thresholds, FP64 accumulators")),
    "random": dict(
        systems=[(10, 1.0, 10000)], n_therm=500, n_meas=500, precision="fp32", bound="alu",
        cpu_paths=2, ref_paths=2, fp64_paths=0, flags="random_site", order="random",
        text=("the paper's literal order, N attempts at random sites per sweep: simple cubic L=10, "
              "J=1, h=0, T=1.0, 10^4 paths, 500+500 sweeps, FP32, one thread per path, lattices "
              "in HBM")),
}

LATTICES = {"sc": 0, "chain": 1, "ising": 2}


def sites(entry) -> int:
    """Sites of a workload system (L, T, paths[, lattice])."""
    L, kind = entry[0], (entry[3] if len(entry) > 3 else "sc")
    return L ** 2 if kind == "ising" else (L if kind == "chain" else L ** 3)


def lattice_of(entry) -> int:
    return LATTICES[entry[3] if len(entry) > 3 else "sc"]

# Algorithmic lane operations of one Metropolis attempt (instruction-bound
# kernels): Philox4x32-10 40 (10 rounds x 2 wide multiplies + 2 three-input
# xors), 3 uniforms 6, trial direction 9 (z, sqrt via rsqrt, phi, sin, cos,
# x, y), own spin 3 loads, local field 33 (18 neighbour loads + 15 adds), dE 8,
# accept 5 (scale, exp, two compares, select), store 3, measurement 2 (about
# 4.5 on the half of the sweeps that measure).
OPS_PER_ATTEMPT = 109
# Ising (Appendix A kernel): a quarter Philox call 10, own spin and four
# neighbour byte loads 5, three adds 3, threshold index and load 3, compare 1,
# flip store and count 2 (on accept; counted once), measurement 1.
OPS_PER_ATTEMPT_ISING = 25
# Algorithmic HBM bytes of one attempt when the lattice streams from HBM:
# each spin is read once and written once per sweep, 3 components x 4 bytes.
BYTES_PER_ATTEMPT_FP32 = 24


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the dominant kernel, from ncu captures of the kernels built from the sources
# with this hash (sha256 over csrc/, first 16 hex digits); any change of the
# sources voids it and the roofline reports traffic null.  Each is the timed
# launch of the workload's bench command, captured at full size (one ncu pass):
# sc16 reads 0.86 MB (tables; the lattices stay in shared memory), batched
# 0.73 MB (every size, L = 32 included, stays in shared memory), large moves
# 28.95 TB against 28.99 TB of algorithmic bytes, ising 0.36 MB.
TRAFFIC = {
    "sc16": {"sources": "95a18dbaf2d46fb2", "bytes": 0.860672e6},
    "large": {"sources": "95a18dbaf2d46fb2", "bytes": 14.458694e12 + 14.496286e12},
    "batched": {"sources": "95a18dbaf2d46fb2", "bytes": 0.734208e6},
    "ising": {"sources": "95a18dbaf2d46fb2", "bytes": 0.356608e6},
}


def sources_hash() -> str:
    import hashlib

    d = os.path.join(ROOT, "paper_1305_6758_gb300", "csrc")
    h = hashlib.sha256()
    for f in sorted(os.listdir(d)):
        h.update(f.encode())
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def launch_traffic(name: str):
    t = TRAFFIC.get(name)
    if t and t["sources"] == sources_hash():
        return t["bytes"]
    return None


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def attempts_of(systems, sweeps, paths_override=None):
    return sum(sites(e) * (paths_override or e[2]) * sweeps for e in systems)


def oracle_sample(w, paths_per_system: int, threads: int | None = None, total_paths: int | None = None):
    """Run the FP64 oracle on the first paths of every system; returns (attempts, seconds).

    With total_paths, that many paths are dealt round-robin over the systems
    (path j of the sample is path j // n_systems of system j % n_systems), so
    that a sample of exactly `threads` equal paths keeps every host core busy.
    """
    import oracle

    oracle.build()
    ns = len(w["systems"])
    counts = ([min(paths_per_system, e[2]) for e in w["systems"]] if total_paths is None else
              [min(e[2], total_paths // ns + (1 if k < total_paths % ns else 0))
               for k, e in enumerate(w["systems"])])
    systems = [oracle.System(e[0], e[1], n_paths=e[2], path_begin=0, path_count=c, lattice=lattice_of(e))
               for e, c in zip(w["systems"], counts) if c > 0]
    order = oracle.ORDER_RANDOM if w.get("order") == "random" else oracle.ORDER_CHECKER
    t0 = time.perf_counter()
    oracle.run(systems, w["n_therm"], w["n_meas"], seed=1, threads=threads, order_mode=order)
    dt = time.perf_counter() - t0
    att = sum(s.N * s.path_count * (w["n_therm"] + w["n_meas"]) for s in systems)
    return att, dt


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


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """The largest of every rank's x (the timed duration of the job)."""
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def rank_path_range(n_paths: int, rank: int, world: int, weak: bool = True) -> tuple[int, int]:
    """(path_begin, count) of one rank's share of a system's ensemble.

    weak: every rank runs n_paths paths of its own, ids rank * n_paths onward,
    so N ranks form one ensemble of N * n_paths paths; otherwise the n_paths
    ids are split into contiguous blocks (the first n_paths % world ranks one
    path more)."""
    if weak:
        return rank * n_paths, n_paths
    q, r = divmod(n_paths, world)
    begin = rank * q + min(rank, r)
    return begin, q + (1 if rank < r else 0)


def gather_records(rec, dist=None):
    """Every rank's per-path records (arrays of rows), concatenated in rank
    order on every rank; with path ranges from rank_path_range they are the
    records of one process running all the paths."""
    import numpy as np

    rec = np.asarray(rec)
    if dist is None:
        return rec
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, rec)
    return np.concatenate(parts, axis=0)


def job_throughput(units_per_rank: float, world: int, steps: int, total_ms: float) -> float:
    """Weak scaling: every rank runs its own full workload; units/s of the whole job."""
    return units_per_rank * world * steps / (total_ms / 1e3)


def run_reference(args, w, rank):
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    # one path per host core per step, dealt round-robin over the systems
    n_ref = min(cores * w["ref_paths"], sum(e[2] for e in w["systems"]))
    for _ in range(args.warmup):
        oracle_sample(w, 0, cores, total_paths=n_ref)
    total_att, total_s = 0, 0.0
    for _ in range(args.steps):
        att, dt = oracle_sample(w, 0, cores, total_paths=n_ref)
        total_att += att
        total_s += dt
    value = total_att / total_s
    sample = (f"{n_ref} paths per step (up to {w['ref_paths']} per host core), dealt round-robin over the "
              f"{len(w['systems'])} systems, all {w['n_therm'] + w['n_meas']} sweeps (FP64 oracle, "
              f"{cores} threads)")
    emit({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "attempts/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["text"], "sample": sample},
        "cpu_baseline": {"value": value, "unit": "attempts/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "attempts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    })


def make_systems(mp, w, paths_override=None, rank=0):
    """The workload's systems; rank r runs path ids r x P onward of each."""
    out = []
    for e in w["systems"]:
        P = paths_override or e[2]
        out.append(mp.System(e[0], e[1], n_paths=P, lattice=lattice_of(e), path_begin=rank * P))
    return out


def timed_runs(mp, torch, w, dev, seed, steps, warmup, flush, barrier, gpu_id, nvtx=None, rank=0):
    """W untimed runs, then K runs each bracketed by CUDA events on the
    simulation's own stream (L2 flushed before each); the clocks are sampled
    during the timed runs.  Returns the simulation (open) and the timings."""
    precision = mp.FP64 if w["precision"] == "fp64" else mp.FP32
    tune = mp.FLAG_AUTOTUNE | (mp.FLAG_RANDOM_SITE if w.get("flags") == "random_site" else 0)
    sim = mp.Simulation(make_systems(mp, w, rank=rank), w["n_therm"], w["n_meas"], seed=seed,
                        precision=precision, device=dev, flags=tune)
    for _ in range(warmup):
        sim.run()
    barrier()
    clocks = ClockSampler(gpu_id)
    step_ms, sweep_ms, reduce_ms = [], [], []
    barrier()
    if nvtx:
        # an NVTX range around the timed steps lets a profiler select their launches
        torch.cuda.nvtx.range_push(nvtx)
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(sim.stream)
        sim.run()
        e1.record(sim.stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        a, b = sim.timing()
        sweep_ms.append(a)
        reduce_ms.append(b)
    if nvtx:
        torch.cuda.nvtx.range_pop()
    barrier()
    return sim, dict(step_ms=step_ms, sweep_ms=sweep_ms, reduce_ms=reduce_ms, clocks=clocks.stop(),
                     precision=precision, tune=tune)


def roofline_of(name, w, sweep_avg_ms, n_sm, full_size):
    """The dominant kernel against its roofline: ALU issue for lattices held in
    shared memory, HBM bandwidth for streamed ones (algorithmic units per launch
    / the kernel's average event-timed duration)."""
    peaks, peak_kind = load_peaks()
    kernel_rate = attempts_of(w["systems"], w["n_therm"] + w["n_meas"]) / (sweep_avg_ms / 1e3)
    if w["bound"] == "hbm":
        peak = float(peaks["hbm_gbs"])
        achieved = BYTES_PER_ATTEMPT_FP32 * kernel_rate / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": launch_traffic(name) if full_size else None,
                "bytes_per_attempt": BYTES_PER_ATTEMPT_FP32,
                "peak_basis": f"{peak_kind} HBM copy bandwidth"}
    else:
        sm_max = float(peaks.get("sm_max_mhz", 2070.0))
        peak = n_sm * 128 * sm_max * 1e6 / 1e12  # lane-ops/s in units of 1e12
        ops = OPS_PER_ATTEMPT_ISING if w["bound"] == "alu_ising" else OPS_PER_ATTEMPT
        achieved = ops * kernel_rate / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
                "traffic": launch_traffic(name) if full_size else None, "ops_per_attempt": ops,
                "peak_basis": f"{n_sm} SMs x 128 lanes x {sm_max:.0f} MHz ({peak_kind} max clock)"}
    kernel = {"ising": "ising_kernel", "random_site": "random_site_kernel"}.get(
        "ising" if w["bound"] == "alu_ising" else w.get("flags"), "sweep_kernel")
    roof.update(kernel=kernel, sweep_ms=sweep_avg_ms)
    return roof, kernel_rate


# Estimates of Sec. 2.2 from pooled per-path means (record columns), for the
# paired FP32 - FP64 comparison below: chi and C_V of Eq. (cv), U_L of Eq. (kum).
REC_COL = {"e": 0, "e2": 1, "m": 2, "m2": 3, "m4": 4}


def _estimate(key, mu, N, beta):
    e, e2, m, m2, m4 = (mu[..., REC_COL[k]] for k in ("e", "e2", "m", "m2", "m4"))
    if key == "chi":
        return N * beta * (m2 - m * m)
    if key == "cv":
        return N * beta * beta * (e2 - e * e)
    if key == "binder":
        return 1.0 - m4 / (3.0 * m2 * m2)
    return mu[..., REC_COL[key]]


def paired_difference(rec_a, rec_b, key, N, beta):
    """Estimate of run a minus that of run b over the same paths, and its
    delete-one jackknife standard error (one path left out of both runs)."""
    import numpy as np

    P = rec_a.shape[0]
    d = float(_estimate(key, rec_a.mean(axis=0), N, beta) - _estimate(key, rec_b.mean(axis=0), N, beta))
    la = (rec_a.sum(axis=0) - rec_a) / (P - 1)
    lb = (rec_b.sum(axis=0) - rec_b) / (P - 1)
    th = _estimate(key, la, N, beta) - _estimate(key, lb, N, beta)
    return d, float(np.sqrt((P - 1) / P * np.sum((th - th.mean()) ** 2)))


def precision_record(mp, torch, w, dev, seed):
    """FP32 against the FP64 GPU form on the same paths and seed (paired), at
    three temperatures of the scan; also the FP64 form's throughput."""
    temps, P = (0.5, 1.5, 2.5), 1024
    L = w["systems"][0][0]
    N = L ** 3
    systems = [mp.System(L, T, n_paths=P) for T in temps]
    out = {}
    for prec in (mp.FP32, mp.FP64):
        with mp.Simulation(systems, w["n_therm"], w["n_meas"], seed=seed, precision=prec, device=dev) as sim:
            sim.run()
            torch.cuda.synchronize(dev)
            sweep_ms, _ = sim.timing()
            out[prec] = ([sim.paths(k) for k in range(len(temps))], [sim.estimates(k) for k in range(len(temps))],
                         sweep_ms)
    rows = []
    for k, T in enumerate(temps):
        r32, e32 = out[mp.FP32][0][k], out[mp.FP32][1][k]
        r64, e64 = out[mp.FP64][0][k], out[mp.FP64][1][k]
        row = {"T": T}
        for key, se_key in (("e", "e_se"), ("m", "m_se"), ("chi", "chi_se"), ("cv", "cv_se"),
                            ("binder", "binder_se")):
            d, pse = paired_difference(r32, r64, key, N, 1.0 / T)
            row[key] = {"fp32": e32[key], "fp64": e64[key], "diff": d, "paired_se": pse,
                        "combined_se": (e32[se_key] ** 2 + e64[se_key] ** 2) ** 0.5}
        rows.append(row)
    att64 = N * P * len(temps) * (w["n_therm"] + w["n_meas"])
    v64 = att64 / (out[mp.FP64][2] / 1e3)
    return rows, {"value": v64, "unit": "attempts/s",
                  "sample": f"L={L}, T in {list(temps)}, {P} paths each, {w['n_therm']}+{w['n_meas']} sweeps"}


# Sub-workloads timed beside the headline (default) workload: (steps, warmup).
SUBRECORDS = {"batched": (5, 2), "large": (2, 1)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sc16", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-sub", action="store_true", help="skip the batched and large sub-records")
    # shorter runs of the same launch (for profiling captures only)
    ap.add_argument("--n-therm", type=int, default=None)
    ap.add_argument("--n-meas", type=int, default=None)
    args = ap.parse_args()
    w = dict(WORKLOADS[args.workload])
    full_size = args.n_therm is None and args.n_meas is None
    if args.n_therm is not None:
        w["n_therm"] = args.n_therm
    if args.n_meas is not None:
        w["n_meas"] = args.n_meas

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, w, rank)
        return

    import ctypes

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

    seed = 1  # one ensemble: the ranks differ in their path ids
    n_therm, n_meas = w["n_therm"], w["n_meas"]
    sweeps = n_therm + n_meas
    n_sys = len(w["systems"])
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2
    props = torch.cuda.get_device_properties(dev)
    gpu_id = str(getattr(props, "uuid", local_rank))
    if gpu_id and not gpu_id.startswith("GPU-") and len(gpu_id) == 36:
        gpu_id = "GPU-" + gpu_id
    n_sm = props.multi_processor_count

    sim, t = timed_runs(mp, torch, w, dev, seed, args.steps, args.warmup, flush, barrier, gpu_id, nvtx="timed",
                        rank=rank)
    precision, tune = t["precision"], t["tune"]
    systems = make_systems(mp, w, rank=rank)
    total_ms = max_over_ranks(sum(t["step_ms"]), dist, dev)
    attempts_rank = attempts_of(w["systems"], sweeps)
    paths_rank = sum(e[2] for e in w["systems"])
    value = job_throughput(attempts_rank, world, args.steps, total_ms)
    paths_per_s = job_throughput(paths_rank, world, args.steps, total_ms)
    ests = [sim.estimates(k) for k in range(n_sys)]
    plan_main = sim.plan()
    autotuned = [sim.system_plan(k) for k in (range(n_sys) if n_sys <= 8 else sorted({0, n_sys // 2, n_sys - 1}))]
    sim.close()

    # end to end through the public API: create (the plan's tables H2D),
    # run, read every system's estimates (D2H), destroy -- all inside the clock;
    # the library remembers the autotuner's choice for a batch of this shape,
    # so these creates do not time layouts again
    e2e_s = []
    for k in range(max(1, min(2, args.steps))):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        with mp.Simulation(systems, n_therm, n_meas, seed=seed + 1000 * (k + 1), precision=precision,
                           device=dev, flags=tune) as s2:
            s2.run()
            for j in range(n_sys):
                s2.estimates(j)
            upload = s2.upload_bytes()
        e2e_s.append(time.perf_counter() - t0)
    # the caller's system table, then the library's plan tables (systems, work
    # items, offsets, Ising thresholds, column-walk units) as the library counts them
    h2d_total = ctypes.sizeof(mp.MPSystem) * n_sys + upload
    d2h_total = ctypes.sizeof(mp.MPEstimates) * n_sys
    e2e_value = attempts_rank * world / (sum(e2e_s) / len(e2e_s))

    sweep_avg = sum(t["sweep_ms"]) / len(t["sweep_ms"])
    roof, kernel_rate = roofline_of(args.workload, w, sweep_avg, n_sm, full_size)
    roof["reduce_ms"] = sum(t["reduce_ms"]) / len(t["reduce_ms"])

    # FP32 against the FP64 GPU form, estimate by estimate (paired over the
    # same paths), and the FP64 form's throughput on the same lattice
    fp64, prec_rows = None, None
    if w["fp64_paths"] and not args.no_fp64 and precision == mp.FP32 and full_size:
        prec_rows, fp64 = precision_record(mp, torch, w, dev, seed)
        fp64["fp32_over_fp64"] = kernel_rate / fp64["value"]

    # the batch of uneven sizes (the target form) and the large streamed
    # lattice, each timed on its own beside the headline workload
    subs = {}
    if args.workload == "sc16" and full_size and not args.no_sub:
        for name, (k_steps, k_warm) in SUBRECORDS.items():
            ws = WORKLOADS[name]
            s_sim, st = timed_runs(mp, torch, ws, dev, seed, k_steps, k_warm, flush, barrier, gpu_id, rank=rank)
            s_plan = s_sim.plan()
            s_sim.close()
            s_ms = max_over_ranks(sum(st["step_ms"]), dist, dev)
            s_att = attempts_of(ws["systems"], ws["n_therm"] + ws["n_meas"])
            s_roof, _ = roofline_of(name, ws, sum(st["sweep_ms"]) / len(st["sweep_ms"]), n_sm, True)
            subs[name] = {"value": job_throughput(s_att, world, k_steps, s_ms), "unit": "attempts/s",
                          "steps": k_steps, "warmup": k_warm, "ms_per_step": s_ms / k_steps,
                          "config": {"workload": ws["text"], "plan": s_plan}, "roofline": s_roof,
                          "clocks": st["clocks"], "gpu_launches": 2 * k_steps}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        att, dt = oracle_sample(w, w["cpu_paths"], cores)
        cpu = {"value": att / dt, "unit": "attempts/s", "cores": cores, "kind": "oracle",
               "sample": f"{w['cpu_paths']} path(s) of each of the {n_sys} systems, all {sweeps} sweeps "
                         f"({att:.3g} attempts, {dt:.1f} s)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "attempts/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if precision == mp.FP64 else "f32", "data": "synthetic",
            "config": {"workload": w["text"], "name": args.workload, "n_therm": n_therm, "n_meas": n_meas,
                       "systems": n_sys, "paths": paths_rank,
                       "parallelism": f"path-id shards x{world} (one ensemble of {world} x {paths_rank} paths)",
                       "l2": "flushed between timed steps (256 MB write)", "plan": plan_main,
                       "autotuned": autotuned},
            "paths_per_s": paths_per_s,
            "sigma": {"e_se_max": max(e["e_se"] for e in ests), "m_se_max": max(e["m_se"] for e in ests),
                      "e": [[e["T"], e["e"], e["e_se"]] for e in ests[:: max(1, n_sys // 3)]]},
            "fp64_form": fp64,
            "precision": prec_rows,
            "e2e": {"value": e2e_value, "unit": "attempts/s", "h2d_bytes_per_step": h2d_total,
                    "d2h_bytes_per_step": d2h_total,
                    "layout": ("autotuned once per process: each step's new handle takes the layout "
                               "measured at the first create")},
            "gpu_launches": 2 * args.steps,
            "roofline": roof,
            "cpu_baseline": cpu,
            "clocks": t["clocks"],
        }
        if subs:
            line["workloads"] = subs
        emit(line)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
