#!/usr/bin/env python
"""Benchmark of the estimator's hot path: rho*_s solves/s on GB300.

Workload (one "step" = one solve = one rdm_estimate call over the whole hot path):
long-range transverse-field Ising model H = sum_{i<j} |i-j|^-1.5 Z_i Z_j + g sum X_i,
N = 22 spins (D = 2^22), N_s = 2 (d_s = 4), lambda = 1, g swept over 16 values in
[0.2, 2.0] (step i uses g-index i mod 16), beta = 1, n_v = 32 normalised Gaussian
bath vectors (block of 128 float32 columns), k = 60 Lanczos steps, two passes.
Synthetic, seeded inputs; every Krylov block (2.1 GB) is larger than the 129 MB L2,
so no L2 flush is needed between steps.

Prints ONE JSON line (rank 0). ``--impl reference`` times the CPU oracle instead.
Multi-GPU (torchrun): each rank runs its own solves (independent g values, no
data-path collective), value = all ranks' solves / max-over-ranks time.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "rho* solves/s and SpMM GB/s vs roofline; p50/p99 latency, vs plain FP64 form"
WORKLOAD = "lr_tfim_N22_Ns2_nv32_k60_beta1_fp32"
N_G = 16


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=16)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--oracle-cores", type=int, default=0,
                   help="worker processes timing the oracle (0 = every host core the memory allows)")
    p.add_argument("--ref-steps", type=int, default=2,
                   help="reference arm: Lanczos steps per bath vector in one timed step")
    p.add_argument("--no-plain", action="store_true", help="skip the plain FP64 one-vector form")
    p.add_argument("--n-sites", type=int, default=22,
                   help="spins of the workload (22 = the benchmark; smaller only for profiling)")
    p.add_argument("--k", type=int, default=60, help="Lanczos steps (60 = the benchmark)")
    p.add_argument("--n-v", type=int, default=32,
                   help="bath vectors per solve (32 = the benchmark; fewer only for profiling)")
    p.add_argument("--no-serving", action="store_true", help="skip the serving sub-benchmark")
    p.add_argument("--serving-requests", type=int, default=32)
    p.add_argument("--no-small", action="store_true", help="skip the small-chain latency sub-benchmark")
    p.add_argument("--serving-stream", action="store_true",
                   help="only the serving stream: --serving-requests requests with N in --serving-n "
                        "(default 12..22), at saturation and 0.5x/0.8x/1.0x Poisson load; one JSON line")
    p.add_argument("--serving-n", default="12,22")
    p.add_argument("--serving-budget-gib", type=int, default=160)
    p.add_argument("--config", default="c2", choices=["c2", "c3", "c5"],
                   help="c2 = the benchmark line; c3 / c5 = one full-size solve of the long-range "
                        "XXZ configurations (25 spins, 64 vectors, 32 betas; 30 spins, 4 vectors) "
                        "timed once, one JSON line")
    p.add_argument("--model", default="tfim", choices=["tfim", "xxz"],
                   help="profiling cases only: xxz = long-range XXZ (J/|i-j|, Delta=1, h=0.1, N_s=1, "
                        "Rademacher), the all-to-all XX+YY shape of the 25- and 30-spin configurations")
    return p.parse_args()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------- oracle timing (CPU)
#
# The oracle (float64 NumPy, one recurrence per process) is timed on the host's cores:
# a pool of worker processes (started with `spawn`, one thread each) runs Lanczos steps
# of different bath vectors of the workload side by side. A solve of the workload is
# n_v vectors x (k steps of the first pass + k steps of the Gram-form rerun), so a
# sample of `steps` steps on C vectors at once, taking `wall` seconds, extrapolates to
#     seconds per solve = t_setup + n_v * 2k * wall / (C * steps),
# t_setup being the oracle's operator build for one Hamiltonian (one core).

_ORACLE = {}


def _oracle_init():
    import workloads as W_
    from oracle import lanczos, spin_ops
    c = W_.config_c2(0)
    t0 = time.perf_counter()
    ham = spin_ops.TensorHamiltonian(c["spec"])
    ham.diagonal()
    _ORACLE.update(t_setup=time.perf_counter() - t0, c=c,
                   est=lanczos.Estimator(c["spec"], apply_h=ham, hnorm=ham.norm_bound()))


def _oracle_task(args):
    l, steps = args
    from oracle import lanczos
    c, est = _ORACLE["c"], _ORACLE["est"]
    v = est.starting_block(l, c["seed"], c["dist"])
    t0 = time.perf_counter()
    for _ in lanczos.block_lanczos(est.apply_h, v, steps, est.hnorm):
        pass
    return time.perf_counter() - t0, _ORACLE["t_setup"]


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _mem_available_gb() -> float:
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) / 1e6
    except OSError:
        pass
    return 64.0


class OraclePool:
    """Worker processes running the oracle on bath vectors of the workload, one
    vector per worker. Each worker holds about 1 GB (the N = 22 blocks in float64), so
    the count is bounded by the free host memory as well as by the cores."""

    GB_PER_WORKER = 2.5

    def __init__(self, cores: int | None = None):
        import multiprocessing as mp
        avail = host_cores()
        n = cores if cores else avail
        n = max(1, min(n, avail, int(_mem_available_gb() / self.GB_PER_WORKER) or 1))
        for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[var] = "1"
        self.cores = n
        self.pool = mp.get_context("spawn").Pool(n, initializer=_oracle_init)
        self.t_setup = None

    def sample(self, steps: int) -> dict:
        """`steps` Lanczos steps on each of `cores` bath vectors at once."""
        n_v = W.config_c2(0)["n_v"]
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_task, [(i % n_v, steps) for i in range(self.cores)], chunksize=1)
        wall = time.perf_counter() - t0
        self.t_setup = max(r[1] for r in res)
        return {"wall": wall, "steps": steps, "vectors": self.cores, "t_setup": self.t_setup}

    def solves_per_s(self, s: dict) -> float:
        c = W.config_c2(0)
        per_solve = s["t_setup"] + c["n_v"] * 2 * c["k"] * s["wall"] / (s["vectors"] * s["steps"])
        return 1.0 / per_solve

    def close(self):
        self.pool.close()
        self.pool.join()


def _bench_case(a) -> bool:
    return (a.n_sites, a.k, a.n_v, a.model) == (22, 60, 32, "tfim")


def _config(a, world: int) -> dict:
    """The workload description both arms print (the benchmark, or a profiling case)."""
    bench_case = _bench_case(a)
    xxz = a.model == "xxz"
    return {"workload": WORKLOAD if bench_case else f"profiling_{a.model}_N{a.n_sites}_k{a.k}_nv{a.n_v}",
            "n_sites": a.n_sites, "n_sys": 1 if xxz else 2, "n_v": a.n_v, "k": a.k,
            "beta": [1.0], "g_values": 1 if xxz else N_G, "block_columns": (2 if xxz else 4) * a.n_v,
            "l2": "inputs larger than L2",
            "parallelism": f"replicas{world}"}


def run_reference(a):
    """The oracle timed on the host cores (the reference arm: the paper has no code).
    Each step is a bounded sample of the workload: `--ref-steps` Lanczos steps of the
    first pass on one bath vector per core, all cores at once. `ms_per_step` is the wall
    time of those samples as run; `value` is the solves/s they extrapolate to (labelled
    in `value_kind`). Under torchrun only rank 0 works."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    t_start = time.perf_counter()
    pool = OraclePool(a.oracle_cores)
    try:
        pool.sample(1)  # starts the workers (operator build), not timed
        for _ in range(a.warmup):
            pool.sample(a.ref_steps)
        samples = [pool.sample(a.ref_steps) for _ in range(a.steps)]
    finally:
        pool.close()
    walls = [s["wall"] for s in samples]
    rates = [pool.solves_per_s(s) for s in samples]
    value = statistics.median(rates)
    c = W.config_c2(0)
    sample = (f"per step: {a.ref_steps} Lanczos steps (first pass) on each of {pool.cores} bath vectors at "
              f"once, one per worker process, at full size (D=2^22, 4 columns, float64 NumPy); "
              f"extrapolated to {c['n_v']} vectors x 2 x {c['k']} steps per solve plus the operator build "
              f"({pool.t_setup:.1f} s)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "value_kind": "extrapolated from the timed samples (see cpu_baseline.sample)",
        "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": 1000.0 * statistics.mean(walls),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": _config(a, int(os.environ.get("WORLD_SIZE", "1"))),
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": pool.cores, "kind": "oracle",
                         "sample": sample, "host_cores": host_cores()},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": time.perf_counter() - t_start,
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- GPU clocks

class Clocks:
    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                if self.uuid and self.uuid not in parts[0]:
                    continue
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": num(rows[0][2]), "reasons": reasons, "samples": len(rows),
                "power_w_max": max((num(r[3]) or 0.0) for r in rows)}


# ---------------------------------------------------------------- our arm

def run_ours(a):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")

    # The oracle's CPU baseline: worker processes started with spawn, before this
    # process makes its first CUDA call; a bounded sample (one warm step, then 5 timed
    # Lanczos steps on one bath vector per core).
    cpu_sample = cpu_pool = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline and _bench_case(a):
        cpu_pool = OraclePool(a.oracle_cores)
        try:
            cpu_pool.sample(1)
            cpu_sample = cpu_pool.sample(5)
        finally:
            cpu_pool.close()
    torch.cuda.set_device(local)

    from paper_2204_08147_gb300 import rdm
    ctx = rdm.Context(local)
    cfgs = [W.config_c2(g) for g in range(N_G)]
    if not _bench_case(a):  # profiling case, not a benchmark number
        for c in cfgs:
            c["spec"] = (W.long_range_tfim(a.n_sites, 2, 1.5, float(c["spec"].gx[0])) if a.model == "tfim"
                         else W.long_range_xxz(a.n_sites, 1, 1.0, 1.0, 0.1))
            if a.model == "xxz":
                c["dist"] = "rademacher"
            c["k"] = a.k
            c["n_v"] = a.n_v
    hams = [rdm.Hamiltonian(ctx, c["spec"]) for c in cfgs]

    def solve(i):
        c = cfgs[i % N_G]
        return hams[i % N_G].estimate(c["betas"], c["n_v"], c["k"], c["seed"], precision="fp32",
                                      dist=c["dist"])

    base = rank * (a.warmup + a.steps)
    for i in range(a.warmup):
        solve(base + i)
    ctx.synchronize()

    props = torch.cuda.get_device_properties(local)
    uuid = str(getattr(props, "uuid", "")) or None
    clocks = Clocks(uuid)
    # The timed region runs the library's default path (graph replay of the first pass,
    # no per-launch events). The context runs on torch's current stream, so these
    # events bracket its work.
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    lat = []
    for i in range(a.steps):
        t0 = time.perf_counter()
        solve(base + a.warmup + i)
        lat.append(time.perf_counter() - t0)
    ev1.record()
    torch.cuda.synchronize()
    ctx.synchronize()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    if dist:
        t = torch.tensor([ms], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())

    # Per-kernel split: the same solves again with per-launch CUDA events on the
    # launching stream (rdm_profile; graphs are not replayed while it records).
    n_prof = max(1, min(a.steps, 8))
    ctx.profile(True)
    for i in range(n_prof):
        solve(base + a.warmup + i)
    ctx.synchronize()
    stats = ctx.profile_stats()
    ctx.profile(False)
    total_solves = a.steps * world
    value = total_solves / (ms / 1000.0)

    # End to end through the public API from host buffers: build the Hamiltonian
    # from the host model (descriptor upload), estimate, read the result back.
    e2e_steps = max(2, min(a.steps, 4))
    if dist:
        dist.barrier()
    ctx.synchronize()
    t0 = time.perf_counter()
    h2d = d2h = 0
    for i in range(e2e_steps):
        c = cfgs[(base + i) % N_G]
        h = rdm.Hamiltonian(ctx, c["spec"])
        info = h.info()
        out = h.estimate(c["betas"], c["n_v"], c["k"], c["seed"], precision="fp32", dist=c["dist"])
        h.close()
        h2d += out["h2d_bytes"] + 24 * info["n_flip"] + 16 * info["n_diag"]
        d2h += out["d2h_bytes"]
    ctx.synchronize()
    e2e_s = time.perf_counter() - t0
    if dist:
        t = torch.tensor([e2e_s], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_value = e2e_steps * world / e2e_s

    # Plain FP64 form: the same method one bath vector at a time (block width d_s).
    plain = None
    if rank == 0 and not a.no_plain:
        t0 = time.perf_counter()
        c = cfgs[0]
        for l_ in range(c["n_v"]):
            hams[0].estimate(c["betas"], 1, c["k"], c["seed"] + 7919 * l_, precision="fp64", dist=c["dist"])
        plain = {"value": 1.0 / (time.perf_counter() - t0), "unit": "solves/s",
                 "form": "float64, one bath vector per call (32 calls = one solve), no batching"}

    # Precision: float32 path against the float64 path on the same seeds (one g value).
    precision = None
    if rank == 0 and _bench_case(a):
        c = cfgs[0]
        r32 = hams[0].estimate(c["betas"], c["n_v"], c["k"], c["seed"], precision="fp32", dist=c["dist"])
        r64 = hams[0].estimate(c["betas"], c["n_v"], c["k"], c["seed"], precision="fp64", dist=c["dist"])
        b = float(c["betas"][0])
        precision = {
            "rho_max_abs": float(np.abs(r32["rho"] - r64["rho"]).max()),
            "hstar_max_abs": float(np.abs(rdm.mean_force(r32["rho"][0], b) - rdm.mean_force(r64["rho"][0], b)).max()),
            "entropy_abs": abs(rdm.entropy(r32["rho"][0]) - rdm.entropy(r64["rho"][0])),
            "lnZ_abs": float(abs(r32["lnZ"][0] - r64["lnZ"][0])),
            "against": "float64 path of this library, same bath vectors (g index 0)",
        }

    l2_rate = dram_rate = None
    if rank == 0:
        l2_rate = ctx.probe_copy_rate(32 << 20)
        dram_rate = ctx.probe_copy_rate(4 << 30)

    serving = batch = None
    if rank == 0 and not a.no_serving:
        serving = serving_bench(rdm, ctx, a.serving_requests)
        batch = batch_bench(rdm, ctx)
    small = sweep = ladder = None
    if rank == 0 and not a.no_small:
        small = small_chain_bench(rdm, ctx)
        sweep = sweep_bench(rdm, ctx)
        ladder = ladder_bench(rdm, ctx)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    peak, peak_kind = _peaks()
    host_dense = stats.pop("host_small_dense", None)  # host wall time, not a kernel
    sp = [stats["spmm_pass1"], stats["spmm_pass2"]]
    sp_ms = sum(s["ms"] for s in sp)
    sp_launch = sum(s["launches"] for s in sp)
    sp_bytes = sum(s["bytes"] for s in sp)
    dev_ms_total = sum(s["ms"] for s in stats.values())
    achieved = (sp_bytes / sp_launch) / (sp_ms / sp_launch / 1000.0) / 1e9 if sp_ms > 0 else None
    n_flip = hams[0].info()["n_flip"]
    d_s = 2 if a.model == "xxz" else 4
    cols = d_s * a.n_v
    blk = (1 << a.n_sites) * cols * 4
    # flips applied per row: every transverse-field term; half of the XX+YY pair terms
    # (only antiparallel pairs hop), N(N-1)/4 for all-to-all couplings
    f_off = a.n_sites * (a.n_sites - 1) / 4 if a.model == "xxz" else n_flip
    roof = {"kernel": "k_spmm (pass 1 + pass 2)", "bound": "hbm", "achieved": achieved, "peak": peak,
            "unit": "GB/s", "frac": (achieved / peak) if achieved else None,
            "traffic": _traffic_from_profiles() if _bench_case(a) else None,
            "peak_kind": peak_kind,
            "algorithmic_bytes_per_launch": sp_bytes / max(1, sp_launch),
            "avg_launch_ms": sp_ms / max(1, sp_launch),
            "operand_gbs": ((f_off + 2) * blk) / (sp_ms / sp_launch / 1000.0) / 1e9 if sp_ms > 0 else None,
            "share_of_timed_kernels": sp_ms / dev_ms_total if dev_ms_total else None}
    # Whole Lanczos step against the compulsory traffic of Algorithm 1 (read Q_{j-1},
    # Q_j, write Q_{j+1}: 3 blocks), and the SpMM's flops 2 D B (flips + 1) against the
    # FP32 FMA peak (SMs x 128 lanes x 2 flops x max SM clock).
    orth = stats.get("orth_pass1", {"ms": 0.0, "launches": 0})
    step_ms = (stats["spmm_pass1"]["ms"] + orth["ms"]) / max(1, stats["spmm_pass1"]["launches"])
    step_c = 3.0 * blk
    roof["step"] = {"compulsory_bytes": step_c, "ms_spmm_plus_orth": step_ms,
                    "gbs": step_c / (step_ms / 1000.0) / 1e9 if step_ms > 0 else None,
                    "frac": (step_c / (step_ms / 1000.0) / 1e9) / peak if step_ms > 0 else None,
                    # against the 6 blocks any streaming form moves when A_j = W_j^T Z must
                    # be complete before W_{j+1} can be written
                    "frac_two_pass": (2.0 * step_c / (step_ms / 1000.0) / 1e9) / peak if step_ms > 0 else None}
    sm_max = clk.get("sm_max_mhz") or 2070.0
    fp32_peak = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12
    spmm_tflops = 2.0 * (1 << a.n_sites) * cols * (f_off + 1) / (sp_ms / sp_launch / 1000.0) / 1e12 \
        if sp_ms > 0 else None
    roof["spmm_fp32"] = {"tflops": spmm_tflops, "peak_tflops": fp32_peak,
                         "frac": spmm_tflops / fp32_peak if spmm_tflops else None}
    # On-chip level: the tiled SpMM copies, per 1024-state tile, its own tile, one
    # partner tile per distinct high part of the flip masks and the W_{j-1} tile
    # (none at j = 1) from L2 into shared memory; the denominator is the library's
    # own bulk-copy probe on an L2-resident buffer, measured in this run.
    if l2_rate:
        units = 1 + _partner_tiles(cfgs[0]["spec"]) + (a.k - 1) / a.k
        l2_gbs = units * blk / (sp_ms / sp_launch / 1000.0) / 1e9
        roof["l2_to_smem"] = {"achieved": l2_gbs, "peak": l2_rate, "unit": "GB/s", "frac": l2_gbs / l2_rate,
                              "tiles_per_tile": units, "dram_to_smem_probe": dram_rate,
                              "peak_kind": "probe: rdm_probe_copy_rate, 32 MB L2-resident buffer, 32 KB "
                                           "bulk copies, 6 in flight per SM"}
    # launches of the library's kernels in the timed region: the profiled pass runs the
    # same solves' launch sequence (graph replay launches the same kernel nodes)
    launches = int(round(sum(s["launches"] for s in stats.values()) * a.steps / n_prof))
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": _config(a, world),
        "latency_ms": {"p50": 1000 * float(np.percentile(lat, 50)), "p99": 1000 * float(np.percentile(lat, 99))},
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": h2d / e2e_steps,
                "d2h_bytes_per_step": d2h / e2e_steps},
        "gpu_launches": launches,
        "kernel_ms_per_solve": {k: round(v["ms"] / n_prof, 3) for k, v in stats.items() if v["launches"]},
        "kernel_split": f"per-launch CUDA events on the launching stream over {n_prof} profiled solves "
                        f"run after the timed region (same workload)",
        "host_small_dense_ms_per_solve": (host_dense["ms"] / host_dense["launches"])
        if host_dense and host_dense["launches"] else None,
        "roofline": roof,
        "plain_fp64": plain,
        "precision_fp32_vs_fp64": precision,
        "serving": serving,
        "batch": batch,
        "small_chain": small,
        "sweep": sweep,
        "ladder": ladder,
    }
    if cpu_sample is not None:
        c = W.config_c2(0)
        line["cpu_baseline"] = {
            "value": cpu_pool.solves_per_s(cpu_sample), "unit": "solves/s", "cores": cpu_pool.cores,
            "kind": "oracle", "host_cores": host_cores(), "wall_s": cpu_sample["wall"],
            "sample": f"5 Lanczos steps (first pass) on each of {cpu_pool.cores} bath vectors at once, one "
                      f"per worker process, at full size (D=2^22, float64 NumPy), extrapolated to "
                      f"{c['n_v']} vectors x 2 x {c['k']} steps per solve plus the operator build"}
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


def serving_bench(rdm, ctx, n_req: int, n_min: int = 12, n_max: int = 18, budget_gib: int = 64) -> dict:
    """Mixed request stream (XXZ or LR-TFIM, N in n_min..n_max, mixed beta grids, n_v, k)
    through the library's request loop: first all requests at once (saturated
    throughput, after one untimed pass of the same stream), then Poisson arrivals at
    0.5x, 0.8x and 1.0x that rate (latency percentiles from submission to completion)."""
    reqs = W.serving_requests(n_req, seed=20220419, n_min=n_min, n_max=n_max)
    budget = budget_gib << 30

    def run(gaps):
        ctx.serve_start(budget, max_inflight=4)
        try:
            t0 = time.perf_counter()
            tickets, t_next = [], t0
            for r, g in zip(reqs, gaps):
                t_next += g
                while time.perf_counter() < t_next:
                    time.sleep(min(0.001, max(0.0, t_next - time.perf_counter())))
                tickets.append(ctx.submit(r["spec"], r["betas"], r["n_v"], r["k"], r["seed"], precision="fp32"))
            for t in tickets:
                ctx.wait(t)
            wall = time.perf_counter() - t0
            lat = [ctx.request_times(t)[0] for t in tickets]
        finally:
            ctx.serve_stop()
        return wall, lat

    run([0.0] * n_req)  # warm: workspaces, autotuner size classes, graphs
    wall, _ = run([0.0] * n_req)
    rate = n_req / wall
    rng = np.random.default_rng(7)
    loads = {}
    for frac in (0.5, 0.8, 1.0):
        wall2, lat = run(list(rng.exponential(1.0 / (frac * rate), size=n_req)))
        loads[f"{frac}x"] = {"rate_per_s": frac * rate, "solves_per_s": n_req / wall2,
                             "latency_ms": {"p50": 1000 * float(np.percentile(lat, 50)),
                                            "p99": 1000 * float(np.percentile(lat, 99))}}
    return {"requests": n_req, "saturated_solves_per_s": rate, "poisson": loads,
            "stream": f"XXZ/LR-TFIM mix, N {n_min}..{n_max}, N_s 1-2, 8-64 betas, n_v 8-64, k 30-100, float32; "
                      "small requests share packed launches",
            "max_inflight": 4, "budget_gib": budget >> 30}


def batch_bench(rdm, ctx, n_req: int = 48) -> dict:
    """Uneven small instances (the serving stream's XXZ / LR-TFIM mix with N 8..14, N_s 1-2,
    8-64 betas, n_v 8-64, k 30-100, float32) estimated one at a time through rdm_estimate
    and all at once through rdm_estimate_batch (their first passes in one persistent
    cooperative launch), after one warm-up of each (the batch's warm-up runs the
    autotuner). Host-timed around the blocking calls; the device time of the packed
    launch and of the per-item launches comes from a profiled repeat."""
    reqs = W.serving_requests(n_req, seed=20220422, n_min=8, n_max=14)
    hams = [rdm.Hamiltonian(ctx, r["spec"]) for r in reqs]
    jobs = [dict(ham=h, betas=r["betas"], n_v=r["n_v"], k=r["k"], seed=r["seed"], precision="fp32")
            for h, r in zip(hams, reqs)]

    def singles():
        for jb in jobs:
            jb["ham"].estimate(jb["betas"], jb["n_v"], jb["k"], jb["seed"], precision="fp32")
    singles()
    ctx.estimate_batch(jobs)
    ctx.synchronize()
    t0 = time.perf_counter()
    singles()
    t_single = time.perf_counter() - t0
    t0 = time.perf_counter()
    ctx.estimate_batch(jobs)
    t_batch = time.perf_counter() - t0
    ctx.profile(True)
    singles()
    st_single = ctx.profile_stats()
    ctx.profile(True)
    ctx.estimate_batch(jobs)
    st_batch = ctx.profile_stats()
    ctx.profile(False)
    for h in hams:
        h.close()
    keys, runs = ctx.packed_tuning()

    def dev(st):
        return {"launches": sum(v["launches"] for k, v in st.items() if k != "host_small_dense"),
                "host_small_dense_ms": st.get("host_small_dense", {}).get("ms")}
    return {"requests": n_req, "stream": "XXZ/LR-TFIM mix, N 8..14, N_s 1-2, 8-64 betas, n_v 8-64, k 30-100, "
                                         "float32",
            "one_by_one_solves_per_s": n_req / t_single, "batched_solves_per_s": n_req / t_batch,
            "speedup": t_single / t_batch, "one_by_one": dev(st_single), "batched": dev(st_batch),
            "packed_pass1_ms": st_batch.get("packed_pass1", {}).get("ms"),
            "autotuner": {"size_classes": keys, "candidate_launches": runs}}


def ladder_bench(rdm, ctx) -> dict:
    """The ladder of Sec. 5.2 (10 rungs, J_leg = 1, J_rung = -0.45, h = 1, system = rung 2,
    k = 30, n_v = 50, 16 betas in [0.1, 10], float32), its sites numbered leg by leg:
    solves with the library's bath-bit order (chosen from the coupling graph) and with
    the caller's order, SpMM time per launch from per-launch events."""
    spec = W.spin_ladder(10, 2, numbering="leg")
    order, before, after = rdm.bath_order(spec)
    betas = W.beta_grid(16, 0.1, 10.0)
    out = {"workload": "xy_ladder_L10_sys_rung2_leg_numbered_nv50_k30_16beta_fp32",
           "partner_tiles_caller_order": before, "partner_tiles_chosen_order": after}
    for name, on in (("chosen_order", True), ("caller_order", False)):
        ctx.set_bath_order(on)
        ham = rdm.Hamiltonian(ctx, spec)
        ham.estimate(betas, 50, 30, 20220423, precision="fp32", dist="gauss")
        ctx.synchronize()
        t0 = time.perf_counter()
        for _ in range(3):
            ham.estimate(betas, 50, 30, 20220423, precision="fp32", dist="gauss")
        dt = (time.perf_counter() - t0) / 3
        ctx.profile(True)
        ham.estimate(betas, 50, 30, 20220423, precision="fp32", dist="gauss")
        st = ctx.profile_stats()
        ctx.profile(False)
        ham.close()
        sp = st["spmm_pass1"]
        out[name] = {"ms_per_solve": 1000 * dt, "spmm_ms_per_launch": sp["ms"] / max(1, sp["launches"])}
    ctx.set_bath_order(True)
    return out


def small_chain_bench(rdm, ctx, n_solves: int = 50) -> dict:
    """Latency of one small solve (periodic XXZ chain N=10, N_s=1, n_v=16 Rademacher,
    k=40, 3 betas, float64: the whole problem is L2-resident, so launch and host
    latency set the time). Each solve is timed on the host around the blocking call."""
    c = W.config_c1()
    ham = rdm.Hamiltonian(ctx, c["spec"])

    def one():
        return ham.estimate(c["betas"], c["n_v"], c["k"], c["seed"], precision="fp64", dist=c["dist"])
    for _ in range(3):
        one()
    ctx.synchronize()
    lat = []
    for _ in range(n_solves):
        t0 = time.perf_counter()
        one()
        lat.append(time.perf_counter() - t0)
    # launch count and host share from separately profiled solves (the per-kernel
    # events would add to the latency above)
    n_prof = 10
    ctx.profile(True)
    for _ in range(n_prof):
        one()
    stats = ctx.profile_stats()
    ctx.profile(False)
    host = stats.pop("host_small_dense", None)
    # the same solve as a batch of one: its first pass in one persistent launch
    job = [dict(ham=ham, betas=c["betas"], n_v=c["n_v"], k=c["k"], seed=c["seed"], precision="fp64",
                dist=c["dist"])]
    for _ in range(3):
        ctx.estimate_batch(job)
    lat_b = []
    for _ in range(n_solves):
        t0 = time.perf_counter()
        ctx.estimate_batch(job)
        lat_b.append(time.perf_counter() - t0)
    ham.close()
    return {"workload": "xxz_chain_N10_Ns1_nv16_k40_3beta_fp64", "solves": n_solves,
            "us_per_solve_p50": 1e6 * float(np.percentile(lat, 50)),
            "us_per_solve_p99": 1e6 * float(np.percentile(lat, 99)),
            "launches_per_solve": sum(s["launches"] for s in stats.values()) / n_prof,
            "kernel_us_per_solve": {k: round(1e3 * v["ms"] / n_prof, 1) for k, v in stats.items() if v["launches"]},
            "host_small_dense_us_per_solve": 1e3 * host["ms"] / n_prof if host else None,
            "packed_us_per_solve_p50": 1e6 * float(np.percentile(lat_b, 50)),
            "packed_us_per_solve_p99": 1e6 * float(np.percentile(lat_b, 99))}


def _partner_tiles(spec, tile_bits: int = 10) -> float:
    """Partner tiles one 1024-state tile of the tiled SpMM copies, on average over tiles.
    Flip masks are grouped by their high part (mask >> tile_bits; site q is bit N-1-q;
    X on one site and XX/YY on a pair flip those bits). A group is copied by every tile
    unless all its masks lie above the tile bits and its one coefficient depends on the
    parity of the flipped spins (c_odd or c_even zero, e.g. XX+YY with J^x = J^y, which
    only hops antiparallel pairs): then only the tiles where that parity gives a nonzero
    coefficient copy it, half of them."""
    n = spec.n_sites
    groups = {}
    for q in range(n):
        if spec.gx[q] != 0:
            m = 1 << (n - 1 - q)
            groups.setdefault(m >> tile_bits, []).append((m, 1.0, 1.0))
    for i in range(n):
        for j in range(i + 1, n):
            jx, jy = spec.jx[i, j], spec.jy[i, j]
            if jx != 0 or jy != 0:
                m = (1 << (n - 1 - i)) | (1 << (n - 1 - j))
                groups.setdefault(m >> tile_bits, []).append((m, jx + jy, jx - jy))
    total = 0.0
    for h, terms in groups.items():
        if h == 0:
            continue
        low_free = all((m & ((1 << tile_bits) - 1)) == 0 for m, _, _ in terms)
        parity_only = len(terms) == 1 and (terms[0][1] == 0 or terms[0][2] == 0)
        total += 0.5 if (low_free and parity_only) else 1.0
    return total


def sweep_bench(rdm, ctx) -> dict:
    """A parameter sweep shaped like the paper's entropy phase plot (Sec. 5.3.1):
    long-range XY chain N=16, J/|i-j|, N_s=2, field h over 8 values in [0, 2.2],
    n_v=400 Gaussian bath vectors, k=60, 8 betas in [0.5, 4], float32; one solve per
    h value, back to back (each solve's Krylov block is 2^16 x 1600 columns)."""
    hs = np.linspace(0.0, 2.2, 8)
    betas = W.beta_grid(8, 0.5, 4.0)
    hams = [rdm.Hamiltonian(ctx, W.long_range_xxz(16, 2, alpha=1.0, delta=0.0, h=float(h), lam=1.0)) for h in hs]

    def one(i):
        return hams[i].estimate(betas, 400, 60, 20220421, precision="fp32", dist="gauss")
    one(0)
    ctx.synchronize()
    lat = []
    t0 = time.perf_counter()
    for i in range(len(hs)):
        t1 = time.perf_counter()
        one(i)
        lat.append(time.perf_counter() - t1)
    wall = time.perf_counter() - t0
    for h in hams:
        h.close()
    return {"workload": "lr_xy_N16_Ns2_alpha1_h0-2.2x8_nv400_k60_8beta_fp32", "solves": len(hs),
            "solves_per_s": len(hs) / wall, "ms_per_solve_p50": 1000 * float(np.percentile(lat, 50)),
            "block_mb": (1 << 16) * 1600 * 4 / 1e6}


def spmm_source_hash() -> str:
    """sha256 (16 hex) of the tiled SpMM's source: its region of kernels.cu plus the
    layout and tile definitions it compiles against (rdm_internal.h). A committed
    DRAM-traffic figure is only reported while this matches the hash it was measured
    with."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2204_08147_gb300", "csrc")
    src = open(os.path.join(csrc, "kernels.cu")).read()
    hdr = open(os.path.join(csrc, "rdm_internal.h")).read()
    a = src.index("// ---------------------------------------------------------------- tiled SpMM")
    b = src.index("// ---------------------------------------------------------------- orthogonalisation")
    h = hashlib.sha256(src[a:b].encode())
    for s0, s1 in (("// Geometry of a Krylov block", "// Bath-bit order of a Hamiltonian"),
                   ("constexpr int kTiledLanesLog", "// A table of the tiled diagonal (TileDiag), out[tile]")):
        h.update(hdr[hdr.index(s0):hdr.index(s1)].encode())
    return h.hexdigest()[:16]


def _traffic_from_profiles():
    """DRAM bytes per k_spmm launch from the committed ncu summary, if it was taken
    on the current kernel source (else null)."""
    path = os.path.join(ROOT, "profiles", "k_spmm_tiled_lr_tfim_N22_dram.md")
    try:
        h = spmm_source_hash()
        for line in open(path):
            if line.startswith("traffic_bytes_per_launch:"):
                fields = line.split()
                return float(fields[1]) if fields[-1] == h else None
    except Exception:
        return None
    return None


def run_config(a):
    """One full-size solve of c3 or c5 (float32, the basis recomputed in pass 2 since it
    does not fit), timed on the host around the blocking call, with the per-kernel
    split from rdm_profile."""
    from paper_2204_08147_gb300 import rdm
    cfg = W.config_c3() if a.config == "c3" else W.config_c5()
    ctx = rdm.Context(0)
    ham = rdm.Hamiltonian(ctx, cfg["spec"])
    ctx.profile(True)
    ctx.synchronize()
    t0 = time.perf_counter()
    out = ham.estimate(cfg["betas"], cfg["n_v"], cfg["k"], cfg["seed"], precision="fp32", dist=cfg["dist"])
    secs = time.perf_counter() - t0
    st = ctx.profile_stats()
    ctx.profile(False)
    sp = [st[k] for k in ("spmm_pass1", "spmm_pass2") if k in st]
    rho = out["rho"]
    names = {"c3": "lr_xxz_N25_alpha1_delta1_h0.1_Ns1_nv64_k80_32beta_fp32",
             "c5": "lr_xxz_N30_alpha1.5_delta0.5_Ns1_nv4_k50_beta2_fp32"}
    line = {"config": a.config, "workload": names[a.config], "n_sites": cfg["spec"].n_sites,
            "n_v": cfg["n_v"], "k": cfg["k"], "n_beta": len(cfg["betas"]), "dtype": "f32",
            "seconds_per_solve": secs,
            "spmm_launches": sum(x["launches"] for x in sp),
            "spmm_ms_per_launch": sum(x["ms"] for x in sp) / max(1, sum(x["launches"] for x in sp)),
            "kernel_ms": {k: round(v["ms"], 1) for k, v in st.items() if v["launches"]},
            "trace_minus_1": float(np.abs(np.trace(rho, axis1=1, axis2=2) - 1).max()),
            "min_eig_rho": float(min(np.linalg.eigvalsh(r).min() for r in rho))}
    print(json.dumps(line))
    ham.close()
    ctx.close()
    return 0


def _launch_ranks(a) -> int | None:
    """`--gpus N` outside torchrun: re-run this command under torch.distributed.run with
    N ranks on this node (127.0.0.1 rendezvous) and return its exit code. Under torchrun
    the world size must equal N."""
    world = os.environ.get("WORLD_SIZE")
    if world is not None:
        if int(world) != a.gpus:
            sys.stderr.write(f"bench.py: --gpus {a.gpus} but WORLD_SIZE={world}\n")
            return 2
        return None
    if a.gpus <= 1:
        return None
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={a.gpus}",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__)] + sys.argv[1:]
    return subprocess.call(cmd)


def main():
    a = _args()
    rc = _launch_ranks(a)
    if rc is not None:
        return rc
    if a.impl == "reference":
        return run_reference(a)
    if a.config != "c2":
        return run_config(a)
    if a.serving_stream:
        from paper_2204_08147_gb300 import rdm
        lo, hi = (int(x) for x in a.serving_n.split(","))
        ctx = rdm.Context(0)
        line = serving_bench(rdm, ctx, a.serving_requests, lo, hi, a.serving_budget_gib)
        print(json.dumps({"serving_stream": line}))
        ctx.close()
        return 0
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
