#!/usr/bin/env python
"""Benchmark of the fused lattice Boltzmann stream-collide step on one GB300.

Workload (one "step" = one lattice update of the whole grid through the C ABI):
D3Q19, BGK, FP32 populations in the two-buffer pull layout, 256^3 periodic 3D
Taylor-Green vortex at Re 1600 and Ma 0.1 (u0 = 0.1 c_s), tau from Re. Prints one
JSON line with GLUPS, the HBM roofline of the stream-collide kernel, an end-to-end
number through host buffers, the oracle's CPU baseline, and side measurements
(AA layout, half-precision storage, the adjoint/forward step-time ratio).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica on its own GPU
(the method needs no data exchange between replicas); the time is the maximum
over ranks and the value is the total of lattice updates over all ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import lbinputs  # noqa: E402

METRIC = "GLUPS & % HBM roofline, fused stream-collide; adjoint/forward step time ratio"
UNIT = "GLUPS"
N_GRID = 256
U0 = 0.1 / math.sqrt(3.0)
RE = 1600.0
Q19 = 19
BYTES_PER_LU = {  # algorithmic bytes per lattice update: read Q + write Q populations (+ force read)
    (st, sto): 2 * q * b for st, q in (("D2Q9", 9), ("D3Q19", 19), ("D3Q27", 27))
    for sto, b in (("f64", 8), ("f32", 4), ("f16", 2), ("bf16", 2))
}
# DRAM traffic per launch of the D3Q19 FP32 AB stream-collide kernel at 256^3 from one ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum), valid only for the kernel sources
# with the listed hash; the hash is recomputed at run time and the figure dropped if it differs.
NCU_TRAFFIC = {"kernel_hash": "797b088c562b681a", "bytes_per_launch": 2493599488}  # ncu of --only ab_f32, 256^3
KERNEL_SOURCES = ["lb_device.cuh", "lb_collide.cuh", "lb_kernels.cuh"]


def kernel_hash() -> str:
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2106_12929_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def stream_peak(stream, nbytes=1 << 30, reps=10):
    """Read + write bandwidth (GB/s) of lb_stream_copy between two 1 GiB device buffers, best of
    reps (CUDA events on the stream): a bandwidth reference from this library's own kernel."""
    import torch
    from paper_2106_12929_gb300 import _lib
    a = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    b = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    a.fill_(1)
    lib = _lib.load()
    best = float("inf")
    for k in range(reps + 2):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _lib.check(lib.lb_stream_copy(a.data_ptr(), b.data_ptr(), nbytes, stream.cuda_stream), "lb_stream_copy")
        e1.record(stream)
        torch.cuda.synchronize()
        if k >= 2:
            best = min(best, e0.elapsed_time(e1) / 1e3)
    del a, b
    return 2.0 * nbytes / best / 1e9


def measured_peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons. A reader thread stamps
    each line with the host time it arrived, so that stop() can keep the samples taken inside
    the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        import threading
        self.proc = None
        self.lines = []  # (host time, line)
        self.thread = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line))

    def wait_first_sample(self, timeout: float = 3.0):
        """Block until nvidia-smi has printed its first sample (or the timeout passed)."""
        t0 = time.time()
        while self.proc is not None and not self.lines and time.time() - t0 < timeout:
            time.sleep(0.01)

    def stop(self, window=None):
        """Summary of the samples: those stamped inside window = (t0, t1) when there are any,
        else all of them."""
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)
        stamped = list(self.lines)
        inside = [ln for t, ln in stamped if window and window[0] <= t <= window[1]]
        return self.summarise(inside if inside else [ln for _, ln in stamped], in_window=bool(inside))

    @staticmethod
    def summarise(lines, in_window=True):
        sm, smax, reasons = [], [], set()
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"],
                                 parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "in_timed_region": in_window}


def dist_info():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value: float, world: int, device: str = "cuda"):
    """Maximum of a per-rank value over all ranks (the slowest replica sets the time)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(nodes_per_rank: int, steps: int, seconds_this_rank: float, world: int, device: str = "cuda"):
    """Whole-job lattice updates per second: every rank advances its own replica of
    nodes_per_rank nodes for `steps` steps; the job takes as long as the slowest rank."""
    t = max_over_ranks(seconds_this_rank, world, device)
    return world * nodes_per_rank * steps / t, t


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


BAD_CLOCK_REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown")


def clocks_rejected(clocks) -> bool:
    """A timed region whose clock record shows a hardware or thermal slowdown, or SM clocks well
    below their maximum with no reason given (a clock lock left by another user), is not valid;
    a power cap alone is kept."""
    if not clocks:
        return False
    if any(r in BAD_CLOCK_REASONS for r in clocks["reasons"]):
        return True
    return not clocks["reasons"] and clocks["sm_mhz"] < 0.9 * clocks["sm_max_mhz"]


MIN_TIMED_SECONDS = 0.8  # clock samples come every 200 ms: repeat the K-step region this long


def timed_region(lat, k: int, stream, gpu_index: int, world: int, device: str = "cuda"):
    """K steps timed on the device with the clocks sampled meanwhile. The K-step region is
    timed `reps` times back to back (at least three, and for at least MIN_TIMED_SECONDS so that
    nvidia-smi's 200 ms samples fall inside it; every rank runs the same count) and the median
    is returned. The whole measurement is taken once more when the clock record rejects the
    first attempt (the decision is the same on every rank). Returns (seconds, clocks,
    launches per region); clocks["remeasured"] says whether the second attempt was used and
    clocks["repeats"] how many regions were timed."""
    for attempt in range(2):
        sampler = ClockSampler(gpu_index)
        sampler.wait_first_sample()
        launches0 = lat.launch_count()
        t0 = time.time()
        barrier(world)
        first = time_steps(lat, k, stream)
        barrier(world)
        per = max_over_ranks(first, world, device)
        reps = int(min(max(3, math.ceil(MIN_TIMED_SECONDS / max(per, 1e-6))), 1000))
        times = [first]
        for _ in range(reps - 1):
            barrier(world)
            times.append(time_steps(lat, k, stream))
            barrier(world)
        t1 = time.time()
        clocks = sampler.stop(window=(t0, t1))
        launches = (lat.launch_count() - launches0) // reps
        retry = max_over_ranks(1.0 if clocks_rejected(clocks) else 0.0, world, device) > 0.0
        if attempt == 0 and retry:
            continue
        if clocks is not None:
            clocks["remeasured"] = attempt == 1
            clocks["repeats"] = reps
        return statistics.median(times), clocks, launches


def time_steps(lat, k: int, stream):
    """Device time of k steps of lat (CUDA events on the context's stream), seconds."""
    import torch
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(stream)
    lat.step(k)
    end.record(stream)
    torch.cuda.synchronize()
    return start.elapsed_time(end) / 1e3


def workload_config(world, n=N_GRID):
    """The `config` object of the benchmark line (both arms): the n^3 TGV workload (256^3
    unless the reference arm had to time a smaller grid)."""
    tau = lbinputs.tau_from_reynolds(RE, U0, n)
    return {"workload": f"D3Q19 BGK FP32 two-buffer pull stream-collide, {n}^3 periodic 3D Taylor-Green "
                        f"vortex, Re {RE:g}, Ma 0.1 (u0 = {U0:.6f}), tau = {tau:.6f}",
            "grid": [n, n, n], "nodes": n ** 3, "parallelism": f"replicas x{world}",
            "l2": f"inputs larger than L2 (two {19 * 4 * n ** 3 / 1e9:.2f} GB population buffers per replica)"}


def tgv_workload(n=N_GRID):
    tau = lbinputs.tau_from_reynolds(RE, U0, n)
    dims, rho, u = lbinputs.taylor_green_3d(n, u0=U0)
    return dims, tau, rho, u


ONLY = {  # single-workload runs (for profiling): (stencil, storage, layout, collision)
    "ab_f32": ("D3Q19", "f32", "ab", "bgk"), "aa_f32": ("D3Q19", "f32", "aa", "bgk"),
    "ab_f16": ("D3Q19", "f16", "ab", "bgk"), "ab_bf16": ("D3Q19", "bf16", "ab", "bgk"),
    "aa_f16": ("D3Q19", "f16", "aa", "bgk"), "ab_f64": ("D3Q19", "f64", "ab", "bgk"),
    "d3q27_reg_f32": ("D3Q27", "f32", "ab", "regularized"), "d3q27_reg_f16": ("D3Q27", "f16", "ab", "regularized"),
    "d2q9_f32": ("D2Q9", "f32", "ab", "bgk"), "d2q9_f16": ("D2Q9", "f16", "ab", "bgk"),
    "tgv2d_64_f64": ("D2Q9", "f64", "ab", "bgk"),
    "d3q19_trt_f32": ("D3Q19", "f32", "ab", "trt"), "d3q19_trt_f16": ("D3Q19", "f16", "ab", "trt"),
    "d3q27_kbc_f32": ("D3Q27", "f32", "ab", "kbc"), "d3q27_kbc_f16": ("D3Q27", "f16", "ab", "kbc"),
    "d2q9_kbc_f32": ("D2Q9", "f32", "ab", "kbc"), "d2q9_mrt_f32": ("D2Q9", "f32", "ab", "mrt"),
    "d2q9_trt_f32": ("D2Q9", "f32", "ab", "trt"),
    "d3q19_duct_f32": ("D3Q19", "f32", "ab", "bgk"), "d3q19_duct_f16": ("D3Q19", "f16", "ab", "bgk"),
    "d3q19_force_f32": ("D3Q19", "f32", "ab", "bgk"), "d3q19_force_f16": ("D3Q19", "f16", "ab", "bgk"),
}
DUCT = ("d3q19_duct_f32", "d3q19_duct_f16")  # walls: duct with a sphere (radius n/8), driven by F_x
FORCED = DUCT + ("d3q19_force_f32", "d3q19_force_f16")  # constant body force F_x (Guo source)
LEARNED_ONLY = ("learned", "learned_tc", "learned3", "learned3_tc")  # network, tensor-core option


def workload(stencil: str, n: int | None):
    """(dims, tau, rho, u) of the benchmark flow of a velocity set: 3D Taylor-Green vortex
    (Re 1600, Ma 0.1) for the 3D sets at n^3 (default 256), 2D Taylor-Green vortex
    (u0 = 0.05, tau = 0.8) for D2Q9 at n^2 (default 4096)."""
    if stencil == "D2Q9":
        n = n or 4096
        dims, rho, u = lbinputs.taylor_green_2d(n, u0=0.05)
        return dims, 0.8, rho, u
    return tgv_workload(n or N_GRID)


def run_only(args):
    """One workload only, K timed steps after W warm-up steps: a small, repeatable command
    for profilers. Prints a JSON line with its GLUPS and roofline fraction."""
    import torch
    from paper_2106_12929_gb300 import Lattice, build
    build.build()
    if args.only == "adjoint":
        print(json.dumps({"only": "adjoint", **adjoint_ratio(torch.cuda.current_stream(), n=args.grid or 1024,
                                                             steps=args.steps)}))
        return
    if args.only == "spectral":
        print(json.dumps({"only": "spectral", **spectral_control(torch.cuda.current_stream(), n=args.grid or 128,
                                                               steps=args.steps)}))
        return
    if args.only in LEARNED_ONLY:
        print(json.dumps({"only": args.only, **learned_throughput(torch.cuda.current_stream(), n=args.grid or 2048,
                                                                  steps=args.steps, tc=args.only.endswith("_tc"),
                                                                  net=args.only.split("_")[0])}))
        return
    stencil, storage, layout, coll = ONLY[args.only]
    dims, tau, rho, u = workload(stencil, args.grid)
    N = int(np.prod(dims))
    lat = Lattice(stencil, dims, tau, coll, storage=storage, layout=layout, graphs=not args.no_graphs,
                  nodes_per_thread=args.nodes_per_thread)
    lat.init_from_moments(torch.tensor(rho, device="cuda"), torch.tensor(u, device="cuda"))
    if args.only in FORCED:
        F = np.zeros((3, N))
        F[0] = 1e-6
        lat.set_force(torch.tensor(F, dtype=torch.float64 if storage == "f64" else torch.float32, device="cuda"))
    if args.only in DUCT:
        lat.set_solid(lbinputs.duct_with_obstacle(dims, radius=dims[0] / 8.0))
    lat.step(args.warmup)
    t = time_steps(lat, args.steps, torch.cuda.current_stream())
    lat.check()
    g = N * args.steps / t / 1e9
    bpl = BYTES_PER_LU[(stencil, storage)]
    if args.only in FORCED:  # + force read (arithmetic type)
        bpl += 3 * (8 if storage == "f64" else 4)
    if args.only in DUCT:  # + the 4-byte link word of every node
        bpl += 4
    print(json.dumps({"only": args.only, "grid": list(dims), "steps": args.steps, "graphs": not args.no_graphs,
                      "nodes_per_thread": args.nodes_per_thread,
                      "glups": round(g, 3),
                      "hbm_frac": round(g * bpl / measured_peak_hbm()[0], 4)}))


def run_ours(args):
    import torch
    from paper_2106_12929_gb300 import Lattice, build

    world, rank, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.cuda.current_device()
    build.build()
    stream = torch.cuda.current_stream()
    dims, tau, rho, u = tgv_workload()
    N = int(np.prod(dims))
    rho_d = torch.tensor(rho, device="cuda")
    u_d = torch.tensor(u, device="cuda")

    lat = Lattice("D3Q19", dims, tau, "bgk", storage="f32", layout="ab")
    lat.init_from_moments(rho_d, u_d)
    lat.step(args.warmup)
    barrier(world)
    torch.cuda.synchronize()
    t, clocks, launches = timed_region(lat, args.steps, stream, dev, world)
    lat.check()
    lups, t_max = job_throughput(N, args.steps, t, world)
    glups = lups / 1e9

    # roofline of the dominant kernel (one stream-collide launch per step)
    per_launch = t / args.steps
    alg_bytes = BYTES_PER_LU[("D3Q19", "f32")] * N
    peak, peak_kind = measured_peak_hbm()
    achieved = alg_bytes / per_launch / 1e9
    traffic = NCU_TRAFFIC["bytes_per_launch"] if NCU_TRAFFIC["kernel_hash"] == kernel_hash() else None
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "kernel": "k_update_pair<D3Q19, float, BGK, AB>", "peak_kind": peak_kind,
                "algorithmic_bytes_per_launch": alg_bytes}
    # the library's own streaming copy (16-byte vectors) beside the measured copy peak
    sp = stream_peak(stream)
    roofline["stream_copy_gbs"] = round(sp, 1)
    roofline["frac_of_stream_copy"] = round(achieved / sp, 4)

    extra = {}
    if rank == 0 and not args.quick:
        extra = side_measurements(lat, stream, dims, tau, rho_d, u_d, args, glups / world)
    lat.close()

    # end to end through the public API with host buffers: H2D of (rho, u), K steps, D2H of (rho, u)
    # (page-locked host buffers, allocated once like the inputs; the kernels read and write them
    # in place)
    rho_h = torch.tensor(rho).pin_memory()
    u_h = torch.tensor(u).pin_memory()
    r_out = torch.empty_like(rho_h).pin_memory()
    u_out = torch.empty_like(u_h).pin_memory()
    lat = Lattice("D3Q19", dims, tau, "bgk", storage="f32", layout="ab")
    lat.init_from_moments(rho_h, u_h)
    lat.step(args.warmup)
    lat.moments(out=(r_out, u_out))
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    lat.init_from_moments(rho_h, u_h)
    lat.step(args.steps)
    lat.moments(out=(r_out, u_out))
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    barrier(world)
    t_e2e = max_over_ranks(t_e2e, world)
    lat.close()
    e2e = {"value": round(world * N * args.steps / t_e2e / 1e9, 3), "unit": UNIT,
           "h2d_bytes_per_step": int((rho_h.numel() + u_h.numel()) * 8 / args.steps),
           "d2h_bytes_per_step": int((r_out.numel() + u_out.numel()) * 8 / args.steps),
           "what": "lb_init_from_moments(page-locked host rho, u) + lb_step(K) + lb_moments(page-locked host), "
                   "wall clock; the kernels read and write the host arrays over the host link"}

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    cpu = None if args.no_cpu_baseline or world > 1 else cpu_baseline()
    line = {
        "metric": METRIC, "value": round(glups, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(t_max / args.steps * 1e3, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(world),
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
        "clocks": clocks, "extra": extra,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def side_measurements(lat_ab, stream, dims, tau, rho_d, u_d, args, glups_ab):
    """AA layout, half-precision storage and the adjoint/forward ratio (rank 0, not in `value`)."""
    import torch
    from paper_2106_12929_gb300 import Lattice
    N = int(np.prod(dims))
    k = max(50, args.steps // 2)
    out = {"d3q19_f32_ab_glups": round(glups_ab, 3)}
    for layout, storage in [("aa", "f32"), ("ab", "f16"), ("ab", "bf16"), ("aa", "f16")]:
        lat = Lattice("D3Q19", dims, tau, "bgk", storage=storage, layout=layout)
        lat.init_from_moments(rho_d, u_d)
        lat.step(4)
        t = time_steps(lat, k, stream)
        g = N * k / t / 1e9
        out[f"d3q19_{storage}_{layout}_glups"] = round(g, 3)
        out[f"d3q19_{storage}_{layout}_hbm_frac"] = round(
            g * BYTES_PER_LU[("D3Q19", storage)] / measured_peak_hbm()[0], 4)
        lat.close()
    out["f16_over_f32_glups"] = round(out["d3q19_f16_ab_glups"] / glups_ab, 3)
    for key in ("d3q27_reg_f32", "d3q27_reg_f16", "d2q9_f32", "d2q9_f16", "d3q19_trt_f32", "d3q27_kbc_f32",
                "d3q27_kbc_f16", "d2q9_kbc_f32", "d2q9_mrt_f32"):
        st, sto, lay, coll = ONLY[key]
        dims2, tau2, r2, u2 = workload(st, None)
        lat = Lattice(st, dims2, tau2, coll, storage=sto, layout=lay)
        lat.init_from_moments(torch.tensor(r2, device="cuda"), torch.tensor(u2, device="cuda"))
        lat.step(4)
        t = time_steps(lat, k, stream)
        g = int(np.prod(dims2)) * k / t / 1e9
        out[f"{key}_glups"] = round(g, 3)
        out[f"{key}_hbm_frac"] = round(g * BYTES_PER_LU[(st, sto)] / measured_peak_hbm()[0], 4)
        lat.close()
    out.update(adjoint_ratio(stream))
    for key, tc, net in (("learned_f32", False, "learned"), ("learned_tc", True, "learned"),
                         ("learned3_f32", False, "learned3"), ("learned3_tc", True, "learned3")):
        r = learned_throughput(stream, n=2048, steps=100, tc=tc, net=net)
        out[f"{key}_forward_glups"] = r["forward_glups"]
        out[f"{key}_backward_ms_per_step"] = r["backward_ms_per_step"]
        if not tc:  # the training path: its forward step is the one the ratio divides by
            out[f"{key}_backward_over_forward"] = r["backward_over_forward"]
            out[f"{key}_backward_over_forward_checkpoint_every_2"] = r["backward_over_forward_checkpoint_every_2"]
            out[f"{key}_backward_over_forward_every_state_stored"] = r["backward_over_forward_every_state_stored"]
    # the learned forward step streams the same 72 B per lattice update as FP32 BGK (9 populations
    # read and written); its network runs on the tensor cores (FP16 splits), so HBM is its roof
    for key in ("learned_f32", "learned_tc", "learned3_f32", "learned3_tc"):
        out[f"{key}_forward_hbm_frac"] = round(
            out[f"{key}_forward_glups"] * BYTES_PER_LU[("D2Q9", "f32")] / measured_peak_hbm()[0], 4)
    for n in (128, 1024):
        r = spectral_control(stream, n=n, steps=200)
        out[f"spectral_{n}_controlled_us_per_step"] = r["controlled_us_per_step"]
        out[f"spectral_{n}_plain_us_per_step"] = r["plain_us_per_step"]
    return out


def adjoint_ratio(stream, n=1024, steps=500, k=50):
    """D2Q9 BGK + Guo force, FP32, 1024^2 shear layer, 500 steps, checkpoints every 50:
    (recompute + adjoint) time over forward-with-recording time."""
    import torch
    from paper_2106_12929_gb300 import Lattice
    dims, rho, u = lbinputs.shear_layer(n, u0=0.05)
    N = n * n
    F = torch.tensor(lbinputs.smooth_force(dims, 1e-5, seed=12929), dtype=torch.float32, device="cuda")
    et = torch.full((N,), 1e-3, dtype=torch.float32, device="cuda")
    lat = Lattice("D2Q9", dims, 0.51, "bgk", storage="f32", record_every=k)
    lat.set_force(F)
    rho_d = torch.tensor(rho, dtype=torch.float32, device="cuda")
    u_d = torch.tensor(u, dtype=torch.float32, device="cuda")
    res = {}
    for rep in range(2):  # the first pass allocates checkpoints and recompute buffers
        lat.init_from_moments(rho_d, u_d)
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        lat.step(steps)
        e1.record(stream)
        gF = torch.zeros((2, N), dtype=torch.float32, device="cuda")
        _, lamT = lat.loss_energy(et, grad_F=gF)
        torch.cuda.synchronize()
        e1b = torch.cuda.Event(enable_timing=True)
        e1b.record(stream)
        lat.step_adjoint(lamT, steps, grad_F=gF, want_lambda0=False)
        e2.record(stream)
        torch.cuda.synchronize()
        fwd = e0.elapsed_time(e1) / 1e3
        bwd = e1b.elapsed_time(e2) / 1e3
        res = {"adjoint_forward_ratio": round(bwd / fwd, 3), "adjoint_fwd_ms_per_step": round(fwd / steps * 1e3, 4),
               "adjoint_bwd_ms_per_step": round(bwd / steps * 1e3, 4),
               "adjoint_workload": "D2Q9 BGK+Guo FP32 1024^2 shear layer, 500 steps, checkpoint every 50"}
    lat.close()
    return res


# network MACs x 2 + moments / invariants / collision, per lattice update
LEARNED_FLOP_PER_LU = {"learned": 2 * (6 * 24 + 24 * 24 + 24) + 200, "learned3": 2 * (6 * 53 + 53 * 3) + 200}
N_THETA = {"learned": 793, "learned3": 533}


def learned_throughput(stream, n=2048, steps=200, tc=False, net="learned"):
    """Learned collision (Eq. 5, D2Q9, FP32) on n^2 decaying turbulence: GLUPS of the forward
    step and of the adjoint step with the parameter gradient. net: "learned" (6-24-24-1,
    one shared higher-moment rate) or "learned3" (6-53-3, one rate per higher moment)."""
    import torch
    from paper_2106_12929_gb300 import Lattice
    dims = (n, n, 1)
    rho, u = lbinputs.random_spectrum_velocity(dims, 12.0, 0.05, 30000)
    tau = 0.5 + 3.0 * 0.05 * (n / (2.0 * math.pi)) / 30000.0
    gen = lbinputs.random_mlp3_params if net == "learned3" else lbinputs.random_mlp_params
    th = gen(7, out_bias=math.log(tau - 0.5), out_scale=0.5)
    values = np.concatenate([th, np.zeros(6), np.array([400.0, 100.0, 1e3, 1e6, 1e6, 1e6])])
    lat = Lattice("D2Q9", dims, tau, net, storage="f32", record_every=10, learned_tc=tc)
    lat.set_mlp(values)
    lat.init_from_moments(torch.tensor(rho, device="cuda"), torch.tensor(u, device="cuda"))
    lat.step(5)
    t = time_steps(lat, steps, stream)
    fwd = n * n * steps / t / 1e9
    lat.close()
    # adjoint: recorded run of k steps, then the backward pass; checkpoints every 10 steps (the
    # backward pass recomputes 9 of every 10 states), every 2 steps (recomputes every other
    # state) and every step (no recomputation: 50 stored states, 7.5 GB at 2048^2, which HBM
    # holds easily)
    k = 50
    bwd = {}
    for every in (10, 2, 1):
        lat = Lattice("D2Q9", dims, tau, net, storage="f32", record_every=every, learned_tc=tc)
        lat.set_mlp(values)
        lat.init_from_moments(torch.tensor(rho, device="cuda"), torch.tensor(u, device="cuda"))
        lat.step(k)
        lam = torch.zeros((9, n * n), dtype=torch.float32, device="cuda")
        lam[0] = 1.0
        gth = torch.zeros(N_THETA[net], dtype=torch.float32, device="cuda")
        lat.step_adjoint(lam, k, grad_theta=gth, want_lambda0=False)  # allocates the buffers
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lat.step_adjoint(lam, k, grad_theta=gth, want_lambda0=False)
        e1.record(stream)
        torch.cuda.synchronize()
        bwd[every] = e0.elapsed_time(e1) / 1e3 / k
        lat.close()
    fwd_ms = n * n / fwd / 1e9 * 1e3
    return {"grid": [n, n], "forward_glups": round(fwd, 3),
            "forward_tflops": round(fwd * LEARNED_FLOP_PER_LU[net] / 1e3, 2),
            "backward_ms_per_step": round(bwd[10] * 1e3, 4),
            "backward_over_forward": round(bwd[10] * 1e3 / fwd_ms, 3),
            "backward_over_forward_checkpoint_every_2": round(bwd[2] * 1e3 / fwd_ms, 3),
            "backward_ms_per_step_every_state_stored": round(bwd[1] * 1e3, 4),
            "backward_over_forward_every_state_stored": round(bwd[1] * 1e3 / fwd_ms, 3),
            "forward_ms_per_step": round(fwd_ms, 4)}


def spectral_control(stream, n=128, steps=200, storage="f32", kappa=5e-4):
    """Spectral flow control (Sec. 3.2) on n^2 2D turbulence at Re 2000, Ma 0.1: time per
    controlled step (velocity shift from the state by FFTs, then the shifted BGK step) and
    per plain BGK step of the same lattice, both through lb_step."""
    import torch
    from paper_2106_12929_gb300 import Lattice
    dims = (n, n, 1)
    u0 = 0.1 / math.sqrt(3.0)
    rho, u = lbinputs.random_spectrum_velocity(dims, 8.0 * n / 128.0, u0, 2000)
    tau = 0.5 + 3.0 * u0 * (n / (2.0 * math.pi)) / 2000.0
    lat = Lattice("D2Q9", dims, tau, "bgk", storage=storage)
    rd, ud = torch.tensor(rho, device="cuda"), torch.tensor(u, device="cuda")
    lat.init_from_moments(rd, ud)
    sigma0 = lat.spectrum()
    lat.step(5)
    t_plain = time_steps(lat, steps, stream)
    lat.init_from_moments(rd, ud)
    lat.set_spectral_control(sigma0, kappa=kappa)
    lat.step(5)
    l0 = lat.launch_count()
    t_ctrl = time_steps(lat, steps, stream)
    launches = (lat.launch_count() - l0) / steps
    _, R = lat.spectrum(with_cost=True)
    lat.check()
    lat.close()
    return {"grid": [n, n], "storage": storage, "kappa": kappa,
            "plain_us_per_step": round(t_plain / steps * 1e6, 2),
            "controlled_us_per_step": round(t_ctrl / steps * 1e6, 2),
            "controlled_glups": round(n * n * steps / t_ctrl / 1e9, 3),
            "launches_per_controlled_step": launches, "cost_after": R}


def cpu_baseline(sample_steps: int = 20):  # 10-20 s of oracle work on 16 Arm cores
    """The FP64 CPU oracle on this host, on a bounded sample of the same workload: the full
    256^3 D3Q19 grid for `sample_steps` step(s)."""
    import oracle
    dims, tau, rho, u = tgv_workload()
    N = int(np.prod(dims))
    f = oracle.init_eq("D3Q19", dims, rho, u)
    t0 = time.perf_counter()
    oracle.step("D3Q19", dims, tau, "bgk", f, nsteps=sample_steps)
    dt = time.perf_counter() - t0
    return {"value": round(N * sample_steps / dt / 1e9, 5), "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"D3Q19 BGK FP64, 256^3 TGV, {sample_steps} step(s) ({dt:.1f} s wall)"}


def cpu_baseline_table():
    """The FP64 CPU oracle on this host's cores (as many as OMP_NUM_THREADS allows) on bounded
    samples of each workload: the 2D TGV at 64^2 (all 1000 steps), the 3D TGV at 64^3 and
    256^3, D3Q27 regularized turbulence at 384^3, and the forced D2Q9 shear layer at 1024^2
    forward plus adjoint. One JSON object per sample, in MLUPS."""
    import oracle
    rows = []

    def timed(label, nodes, steps, fn):
        t0 = time.perf_counter()
        fn()
        dt = time.perf_counter() - t0
        rows.append({"sample": label, "mlups": round(nodes * steps / dt / 1e6, 3), "seconds": round(dt, 2)})

    dims, rho, u = lbinputs.taylor_green_2d(64, u0=0.05)
    f = oracle.init_eq("D2Q9", dims, rho, u)
    timed("D2Q9 BGK FP64 TGV 64^2 x 1000 steps", 64 * 64, 1000, lambda: oracle.step("D2Q9", dims, 0.8, "bgk", f, 1000))
    for n, steps in ((64, 100), (256, 10)):
        dims, tau, rho, u = tgv_workload(n)
        f = oracle.init_eq("D3Q19", dims, rho, u)
        timed(f"D3Q19 BGK FP64 TGV {n}^3 x {steps} steps", n ** 3, steps,
              lambda: oracle.step("D3Q19", dims, tau, "bgk", f, steps))
    # 384^3 holds three 12 GB FP64 population arrays on the host; smaller hosts take 256^3
    avail = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    n = 384 if avail > 200e9 else 256
    dims = (n, n, n)
    rho, u = lbinputs.random_spectrum_velocity(dims, 8.0, 0.04, 2106)
    f = oracle.init_eq("D3Q27", dims, rho, u)
    tau = 0.5 + 3.0 * 0.04 * (n / (2.0 * math.pi)) / 3000.0
    timed(f"D3Q27 regularized FP64 turbulence {n}^3 x 3 steps", n ** 3, 3,
          lambda: oracle.step("D3Q27", dims, tau, "regularized", f, 3))
    del f, rho, u
    dims, rho, u = lbinputs.shear_layer(1024, u0=0.05)
    N = 1024 * 1024
    F = lbinputs.smooth_force(dims, 1e-5, seed=12929)
    f0 = oracle.init_eq("D2Q9", dims, rho, u)
    lam = lbinputs.random_field((9, N), seed=1)
    timed("D2Q9 BGK+Guo FP64 shear layer 1024^2 x 20 steps, forward", N, 20,
          lambda: oracle.step("D2Q9", dims, 0.51, "bgk", f0, 20, F=F))
    timed("D2Q9 BGK+Guo FP64 shear layer 1024^2 x 20 steps, adjoint (with its forward sweep)", N, 20,
          lambda: oracle.adjoint("D2Q9", dims, 0.51, "bgk", f0, 20, lam, F=F))
    return {"cores": oracle.num_threads(), "samples": rows}


REFERENCE_LU_BUDGET = 6e9  # lattice updates the reference arm may spend (~200 s at 30 MLUPS)


def reference_grid(steps: int, warmup: int) -> int:
    """Edge of the grid the reference arm times: the 256^3 workload itself when its K + W
    steps fit the budget (short runs such as 20 timed after 5 warm-up steps), else the largest of
    128^3, 64^3 that does."""
    for n in (N_GRID, 128, 64):
        if (steps + warmup) * n ** 3 <= REFERENCE_LU_BUDGET:
            return n
    return 32


def run_reference(args):
    """The oracle timed on the host cores as the reference arm: each step is one lattice
    update of the periodic TGV at the same Re and Ma on the grid reference_grid() picks
    (256^3, the benchmark's own grid, unless K + W steps of it would take minutes); the
    line's `config` names the grid that was timed."""
    world, rank, _ = dist_info()
    if rank != 0:
        return
    import oracle
    n = reference_grid(args.steps, args.warmup)
    dims, tau, rho, u = tgv_workload(n)
    N = n ** 3
    f = oracle.init_eq("D3Q19", dims, rho, u)
    f = oracle.step("D3Q19", dims, tau, "bgk", f, nsteps=args.warmup)
    t0 = time.perf_counter()
    f = oracle.step("D3Q19", dims, tau, "bgk", f, nsteps=args.steps)
    dt = time.perf_counter() - t0
    value = N * args.steps / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(world, n),
        "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"FP64 oracle (plain C, OpenMP over nodes), each step one update of the {n}^3 "
                                   f"grid of the same flow (Re {RE:g}, Ma 0.1, tau = {tau:.6f}), "
                                   f"{args.steps} steps after {args.warmup}"},
        "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)  # the 2000 steps of the 256^3 TGV workload
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--quick", action="store_true", help="skip the side measurements")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-table", action="store_true",
                    help="time the CPU oracle on bounded samples of every workload (no GPU work)")
    ap.add_argument("--only", choices=sorted(list(ONLY) + ["adjoint", "spectral", *LEARNED_ONLY]),
                    default=None,
                    help="run a single workload (profiling aid); no contract line")
    ap.add_argument("--grid", type=int, default=None, help="grid size for --only (default 256, adjoint 1024)")
    ap.add_argument("--no-graphs", action="store_true", help="--only: one launch per kernel instead of graph replay")
    ap.add_argument("--nodes-per-thread", type=int, default=0, choices=[0, 1, 2, 4],
                    help="--only: stream-collide launch shape (0 = chosen from the grid)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.cpu_table:
        print(json.dumps(cpu_baseline_table()))
    elif args.impl == "reference":
        run_reference(args)
    elif args.only:
        run_only(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
