"""Benchmark: trajectory*site*steps/s of the tensor jump method on GB300.

Workload (one GPU): XXX chain L = 1000, J = 1, g = 0.5, sigma^- and Z noise at
gamma = 0.1 on every site, dt = 0.1, chi_max = 64, 256 trajectories, <Z_i>
sampled at every step, started from a seeded random MPS with every bulk bond
at chi = 64 (the bond-saturated regime the chi = 64 throughput refers to).
A step is one full TJM time step of every trajectory: U[dt] (dynamic TDVP),
the sampling layer J'(D[dt/2]) with the observables, and J(D[dt]).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank simulates its own 256 trajectories (global ids
rank*256 ...), weak scaling, no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "trajectory*site*steps/s at L=1000 chi=64"
UNIT = "trajectory*site*steps/s"
# --precision value -> (library precision code, dtype of the JSON line)
PRECISIONS = {"f32+df64": (3, "f32+df64"), "f32+f64": (1, "f32+f64"), "f32": (2, "f32"), "f64": (0, "f64")}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="f32+df64", choices=list(PRECISIONS),
                   help="f32+df64: FP32 contractions, QR/SVD in emulated FP64 (double-float); f32+f64: the same "
                        "with native FP64 QR/SVD; f32: QR/SVD in FP32 too; f64: everything FP64")
    p.add_argument("--L", type=int, default=1000)
    p.add_argument("--chi", type=int, default=64)
    p.add_argument("--ntraj", type=int, default=256)
    p.add_argument("--no-fp64", action="store_true", help="skip the plain-FP64 GPU arm")
    p.add_argument("--fp64-traj", type=int, default=0,
                   help="trajectories of the plain-FP64 GPU arm (0: one per SM, at most the main arm's count)")
    p.add_argument("--e2e-steps", type=int, default=2, help="steps of the end-to-end tjm_run measurement")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    p.add_argument("--serve-requests", type=int, default=8,
                   help="serving replay: the first R arrivals of the Poisson request stream (0: skip)")
    p.add_argument("--serve-traj-scale", type=float, default=1.0 / 64)
    p.add_argument("--serve-max-steps", type=int, default=5)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--ref-sites", type=int, default=200,
                   help="reference arm: sites of the chi-saturated chain each oracle trajectory steps through")
    return p.parse_args()


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return

        def reader():
            for line in self.proc.stdout:
                self.rows.append([x.strip() for x in line.split(",")])
        self.thread = threading.Thread(target=reader, daemon=True)
        self.thread.start()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() in ("active", "1"):
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- the oracle (CPU)
def _oracle_step_job(args):
    """One oracle TJM step of one trajectory on an L-site chi-saturated chain; returns seconds."""
    L, chi, traj, seed = args
    import numpy as np
    from oracle import mps_tjm as O1
    from oracle.philox import uniforms
    from paper_2501_17913_gb300 import inputs as I
    W = I.xxx_mpo(L, 1.0, 0.5)
    prob = O1.Problem(W, I.noise(L, 0.1, 0.1), 0.1, chi, 1e-10)
    _, sites = I.random_mps(L, chi, seed)
    mps = [np.array(s) for s in sites]
    for l in range(L - 1, 0, -1):
        O1.rq_move_left(mps, l)
    mps[0] = mps[0] / np.linalg.norm(mps[0])
    D_half = [O1.dissipator_site(prob, l, 0.05) for l in range(L)]
    D_full = [O1.dissipator_site(prob, l, 0.1) for l in range(L)]
    t0 = time.perf_counter()
    sw = O1.Sweeper(prob)
    sw.build_right_envs(mps)
    sw.sweep(mps, 0.05)
    X = [m.copy() for m in mps]
    O1.dissipate_and_jump(X, prob, D_half, *uniforms(seed, traj, 1, 1))
    O1.measure(X, I.z_observables(L))
    O1.dissipate_and_jump(mps, prob, D_full, *uniforms(seed, traj, 1, 0))
    return time.perf_counter() - t0


def oracle_rate(pool, cores, L, chi, first, seed):
    """One timed oracle step: `cores` trajectories (one per core, in parallel) on an L-site slice.
    Returns (wall seconds of the step, busy CPU seconds)."""
    t0 = time.perf_counter()
    per = pool.map(_oracle_step_job, [(L, chi, first + t, seed) for t in range(cores)])
    return time.perf_counter() - t0, sum(per)


def oracle_sample(cores, L, chi):
    """The CPU baseline: the oracle as it stands on one step of `cores` trajectories of an L-site slice of
    the benchmark's chi-saturated family, one trajectory per host core; rate from the wall time."""
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_step_job, [(8, chi, t, 11) for t in range(cores)])      # start-up of the workers
        wall, busy = oracle_rate(pool, cores, L, chi, 0, 2025)
    return {"value": cores * L / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d trajectories (one per core) x 1 TJM step of an L=%d slice of the chi=%d random "
                      "chi-saturated family (seed 2025, same H, noise, dt), numpy FP64 oracle; per-site rate from "
                      "the wall time of the step" % (cores, L, chi),
            "wall_s": wall, "cpu_s": busy}


def workload_config(a, world, state_bytes_per_elem):
    L, chi, N = a.L, a.chi, a.ntraj
    return {"workload": "xxx_L%d_chi%d_N%d_random_chi_saturated" % (L, chi, N), "L": L, "chi_max": chi,
            "trajectories_per_gpu": N, "dt": 0.1, "gamma": 0.1, "g": 0.5,
            "l2": "inputs larger than L2 (trajectory state %.1f GB)" %
            (N * (L * 2 * chi * chi + 2 * (L + 1) * 5 * chi * chi) * state_bytes_per_elem / 1e9),
            "parallelism": "trajectories" + ("x%d" % world if world > 1 else "")}


def run_reference(a):
    """The oracle arm: the CPU FP64 oracle on a bounded sample of the bench workload.

    Each timed step is one oracle TJM step of `cores` trajectories (one per host core, in parallel)
    on a --ref-sites chain of the same random chi-saturated family (the bench's seed, same H, noise
    and dt), reported per site from the measured wall time of the step: a full L=1000 oracle step
    takes ~100 s per core, so the slice keeps the run to a few minutes; its ~5 % of edge sites with
    chi < 64 make the per-site rate slightly optimistic for the CPU.  The warm-up steps run the same
    code on an 8-site chain.
    """
    cores = max(1, min(os.cpu_count() or 1, 16))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    import multiprocessing as mp
    Ls = min(a.L, a.ref_sites)
    t0 = time.perf_counter()
    walls = []
    with mp.get_context("spawn").Pool(cores) as pool:
        for _ in range(a.warmup):
            pool.map(_oracle_step_job, [(8, a.chi, t, 11) for t in range(cores)])
        for k in range(a.steps):
            walls.append(oracle_rate(pool, cores, Ls, a.chi, k * cores, 2025)[0])
    wall = sum(walls)
    value = a.steps * cores * Ls / wall
    sample = ("%d trajectories (one per core) x 1 oracle TJM step per timed step, on an L=%d slice of the "
              "chi=%d random chi-saturated family (seed 2025), numpy FP64; per-site rate from the wall time"
              % (cores, Ls, a.chi))
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
           "ms_per_step": 1000.0 * wall / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic", "impl": "reference", "config": workload_config(a, 1, 8),
           "step": "one oracle TJM step of %d trajectories on the L=%d slice (measured)" % (cores, Ls),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "wall_s": time.perf_counter() - t0}
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------------------- roofline inputs
def csrc_digest():
    """Digest of the CUDA sources: identifies the kernel version a profile was taken of."""
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2501_17913_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh", ".h")):
            h.update(f.encode())
            with open(os.path.join(d, f), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel_file, units_per_launch):
    """DRAM bytes per launch of the dominant kernel from its committed ncu summary, scaled to this launch's
    units; None unless the summary was taken of the current sources (its `csrc digest:` line matches)."""
    p = os.path.join(ROOT, "profiles", kernel_file)
    try:
        txt = open(p).read()
    except OSError:
        return None, "no profile"
    import re
    dg = re.search(r"csrc digest:\s*([0-9a-f]{16})", txt)
    per = re.search(r"dram bytes per unit:\s*([0-9.eE+]+)", txt)
    if not dg or not per:
        return None, "profile lacks digest or per-unit bytes"
    if dg.group(1) != csrc_digest():
        return None, "kernel changed since the profile (%s)" % dg.group(1)
    return float(per.group(1)) * units_per_launch, "profiles/%s scaled by units" % kernel_file


# ----------------------------------------------------------------------------- serving replay
def run_serving(a, prec, device):
    """Replay the first --serve-requests arrivals of the Poisson stream (20 req/s, seed 11) through the
    continuous-batching loop, each request's trajectory count scaled by --serve-traj-scale and its step
    count capped at --serve-max-steps; p50 / p99 completion latency, offered and sustained load."""
    import math as _m
    from paper_2501_17913_gb300 import inputs as I
    from paper_2501_17913_gb300.serve import Server
    stream = I.request_stream()[:a.serve_requests]
    srv = Server(precision=prec, steps_per_tick=1, device=device)
    t0 = time.perf_counter()
    for (t_arr, wl) in stream:
        wl.n_traj = max(1, int(_m.ceil(wl.n_traj * a.serve_traj_scale)))
        wl.n_steps = min(wl.n_steps, a.serve_max_steps)
        wl.sample_steps = [wl.n_steps]
        srv.submit(wl, t0 + t_arr)
    srv.drain()
    t1 = time.perf_counter()
    rep = srv.report(t0, t1)
    rep["stream"] = ("first %d arrivals of the Poisson stream (20/s, seed 11), trajectory counts x %.4g, at most %d "
                     "steps each" % (a.serve_requests, a.serve_traj_scale, a.serve_max_steps))
    srv.close()
    return rep


# ----------------------------------------------------------------------------- ours (GPU)
def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
        return
    import numpy as np
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2501_17913_gb300 import build as B
    from paper_2501_17913_gb300 import inputs as I
    from paper_2501_17913_gb300 import tjm
    if rank == 0 or world == 1:
        B.build()
    if dist:
        dist.barrier()
    prec, dtype = PRECISIONS[a.precision]
    L, chi, N, dt = a.L, a.chi, a.ntraj, 0.1
    n_total = a.warmup + a.steps
    W = I.xxx_mpo(L, 1.0, 0.5)
    jumps = I.noise(L, 0.1, 0.1)
    obs = I.z_observables(L)
    psi = I.random_mps(L, chi, 2025)
    times = [dt * j for j in range(n_total + 1)]
    t_main = time.perf_counter()
    ctx = tjm.Context(W, jumps, dt, chi, 1e-10, precision=prec, device=local)
    rid = ctx.prepare(psi, N, 0, obs, times, first_traj=rank * N)
    stream = torch.cuda.ExternalStream(ctx.stream())
    ctx.advance(rid, 0)                      # initialisation, F_0
    # warm-up steps double as the GEMM tile autotuner's trial launches
    from paper_2501_17913_gb300.autotune import TileAutotuner
    tuner = TileAutotuner()
    for _ in range(a.warmup):
        tuner.advance(ctx, rid, 1)
    rule = tuner.next_rule(tuner.key(ctx))
    ctx.set_tile_rule(rid, rule)
    ctx.sync()
    s0 = ctx.stats(rid)
    launches0 = ctx.launches()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        ctx.advance(rid, 1)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1)
    s1 = ctx.stats(rid)
    t_main = time.perf_counter() - t_main
    gpu_launches = ctx.launches() - launches0   # trajectory-kernel launches (each preceded by a counter memset)
    from paper_2501_17913_gb300.shard import job_rate
    value, t_max = job_rate(N * L * a.steps, ms)       # all ranks' units over the slowest rank's time
    fc = s1["flops_contract"] - s0["flops_contract"]
    fd = s1["flops_decomp"] - s0["flops_decomp"]
    cyc = {k: s1["cycles"][k] - s0["cycles"][k] for k in s1["cycles"]}
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    achieved = fc / (ms / 1000.0) / 1e12
    # The contractions' roofline is the tensor pipe.  TF32 (the FP32-input tensor format) runs at half the
    # BF16 rate; the denominator is the measured sustained cuBLAS BF16 rate (a kernel timed inside a long
    # step) halved, else the recipe's fallback.
    if "bf16_tflops_sustained" in peaks:
        bf16, src = float(peaks["bf16_tflops_sustained"]), "measured"
    else:
        bf16, src = 1700.0, "fallback"
    fp32_core = n_sm * 128 * 2 * sm_max * 1e6 / 1e12
    fp64_core = n_sm * 2 * 2 * sm_max * 1e6 / 1e12       # FP64 FMA: 2 per SM per clock on GB300
    if prec == tjm.PREC_FP64:
        roof = {"bound": "alu", "achieved": achieved, "peak": fp64_core, "unit": "TFLOP/s",
                "frac": achieved / fp64_core,
                "peak_source": "derived: %d SMs x 2 FP64 FMA/clk x 2 flop x %.0f MHz" % (n_sm, sm_max)}
    else:
        tf32 = bf16 / 2.0
        roof = {"bound": "tensor", "achieved": achieved, "peak": tf32, "unit": "TFLOP/s", "frac": achieved / tf32,
                "peak_source": "TF32 = %s sustained BF16 %.1f TFLOP/s / 2 (of %s)" % (src, bf16, src),
                "cuda_core_fp32": {"peak": fp32_core, "frac": achieved / fp32_core,
                                   "peak_source": "derived: %d SMs x 128 FP32 lanes x 2 flop x %.0f MHz"
                                                  % (n_sm, sm_max)}}
    roof["kernel"] = "tjm::advance_kernel"
    roof["achieved_counts"] = "contraction flops counted on device (8 per complex MAC) / CUDA-event time of the launches"
    traffic, tsrc = profiled_traffic("advance_kernel_traffic_bench.md", N * L)
    roof["traffic"] = traffic
    roof["traffic_source"] = tsrc
    roof["decomp_tflops"] = fd / (ms / 1000.0) / 1e12
    tot_cyc = max(1, sum(v for k, v in cyc.items() if k in ("tdvp", "dissipate_jump", "env_build", "measure")))
    roof["phase_share"] = {k: cyc[k] / tot_cyc for k in ("gemm", "mpo_contract", "lanczos", "qr", "svd", "matvec",
                                                         "krylov_expm", "tdvp", "dissipate_jump", "env_build",
                                                         "measure")}
    ctx.close()                              # frees the trajectory state before the other arms allocate theirs
    ctx = None
    extra = {}
    phase_wall = {}
    # end to end through the C ABI with host buffers: tjm_run (init + F_0 + K steps) and tjm_result
    if not a.no_e2e:
        ke = max(1, min(a.steps, a.e2e_steps))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx2 = tjm.Context(W, jumps, dt, chi, 1e-10, precision=prec, device=local, tile_rule=rule)
        times2 = [dt * j for j in range(ke + 1)]
        r2 = ctx2.run(psi, N, 0, obs, times2, first_traj=rank * N)
        mean, sem, pt = ctx2.result(r2)
        t_e2e = time.perf_counter() - t0
        h2d = sum(x.size for x in psi[1]) * 16 + len(psi[0]) * 4
        d2h = pt.nbytes + mean.nbytes + sem.nbytes
        e2e = {"value": world * N * L * ke / t_e2e, "unit": UNIT, "h2d_bytes_per_step": h2d // ke,
               "d2h_bytes_per_step": d2h // ke, "wall_s": t_e2e, "steps": ke,
               "note": "tjm_run from host inputs (upload, init, F_0, %d steps) + tjm_result to host" % ke}
        ctx2.close()
        phase_wall["e2e"] = t_e2e
    else:
        e2e = None
    # plain FP64 GPU path on the same workload (L, chi, H, noise, dt, random chi-saturated start): one timed step
    if not a.no_fp64 and rank == 0:
        t3 = time.perf_counter()
        ctx3 = tjm.Context(W, jumps, dt, chi, 1e-10, precision=tjm.PREC_FP64, device=local)
        # FP64 is bound by the SM's FP64 pipe: one CTA per SM already takes nearly all of it (measured at
        # L = 100: 152 trajectories 669, 304 trajectories 692 trajectory*site*steps/s), while a count between
        # one and two per SM leaves the two-CTA SMs setting the step time.  One trajectory per SM is the
        # FP64 path's best use of the GPU per unit of time.
        N64 = a.fp64_traj or min(N, n_sm)
        r3 = ctx3.prepare(psi, N64, 0, obs, [dt, 2 * dt])
        ctx3.advance(r3, 0)
        ctx3.sync()
        st3 = torch.cuda.ExternalStream(ctx3.stream())
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(st3)
        ctx3.advance(r3, 1)
        f1.record(st3)
        f1.synchronize()
        ms64 = f0.elapsed_time(f1)
        extra["fp64_gpu"] = {"value": N64 * L / (ms64 / 1000.0), "unit": UNIT, "same_config": True,
                             "slice": "%d trajectories x 1 timed step, L=%d, chi=%d (random chi-saturated MPS, the "
                                      "bench's seed), FP64 contractions and factorizations" % (N64, L, chi),
                             "ms": ms64}
        ctx3.close()
        phase_wall["fp64_arm"] = time.perf_counter() - t3
    serving = None
    if a.serve_requests > 0 and rank == 0:
        t4 = time.perf_counter()
        serving = run_serving(a, prec, local)
        phase_wall["serving"] = time.perf_counter() - t4
    cpu = None
    if not a.no_cpu and rank == 0:
        t5 = time.perf_counter()
        cpu = oracle_sample(max(1, min(os.cpu_count() or 1, 16)), min(L, a.ref_sites), chi)
        phase_wall["cpu_baseline"] = time.perf_counter() - t5
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
               "warmup": a.warmup, "ms_per_step": t_max / a.steps, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": dtype, "data": "synthetic",
               "arithmetic": {"f32+df64": "FP32 contractions (FP32 accumulation); QR/SVD in double-float emulated "
                                          "FP64; norms, jump weights, Lanczos coefficients in FP64",
                              "f32+f64": "FP32 contractions; QR/SVD in native FP64; FP64 reductions",
                              "f32": "FP32 contractions and QR/SVD; FP64 reductions",
                              "f64": "FP64 throughout"}[a.precision],
               "config": workload_config(a, world, 8 if prec else 16),
               "roofline": roof, "clocks": clocks, "gpu_launches": gpu_launches,
               "tile_autotune": {"rule": rule, "trials": tuner.report()},
               "e2e": e2e, "cpu_baseline": cpu, "serving": serving,
               "stats": {"jumps": s1["jumps"] - s0["jumps"],
                         "matvecs_one_site": s1["matvec_one_site"] - s0["matvec_one_site"],
                         "matvecs_bond": s1["matvec_bond"] - s0["matvec_bond"],
                         "matvecs_two_site": s1["matvec_two_site"] - s0["matvec_two_site"],
                         "contract_gflop": fc / 1e9, "decomp_gflop": fd / 1e9}}
        out["wall_s"] = dict(phase_wall, main_arm=t_main)
        if "fp64_gpu" in extra:
            out["fp64_gpu"] = extra["fp64_gpu"]
            out["vs_fp64_gpu"] = value / world / extra["fp64_gpu"]["value"]
        print(json.dumps(out), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
