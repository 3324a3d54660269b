#!/usr/bin/env python
"""Throughput of the string method on one GB300 (or N replicas under torchrun).

Workload: the Bloch-point collapse string -- 64x64x8 lattice (32768 spins), 32 images, J=1, D=0.25,
K=0.1, w=0.02, dipole by FFT convolution, 2000 iterations of dt=0.1.  One bench step is the whole hot
path once: set the initial path, run 2000 iterations (field, step, per-image energies, equal-arc-length
reparametrisation), evaluate the barrier.  Metric: spin-updates/s = spins x images x iterations / time.

  value     device-timed (CUDA events on the calling stream), initial path already resident in HBM
  e2e       the same through the public API with the path copied from pinned host memory each step and
            the energies read back
  roofline  the dominant kernel's algorithmic bytes per launch / its mean event-timed duration
  cpu_baseline / --impl reference   the FP64 CPU oracle on a bounded sample (one iteration of an
            8-image sub-string of the same workload), timed on this host's cores

N > 1 (torchrun): every rank runs its own replica of the workload (independent strings; weak scaling,
no collective on the data path); time = max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1804_07135_gb300 import workloads  # noqa: E402

L2_FLUSH_BYTES = 256 << 20
# Compulsory bytes per site-image of each kernel (FP32): each input read once, each output written once.
#   xfwd: read sp 12, write s 12, write the pair spectrum 3 * 8 * (Px/nx) / 2 per image = 24
#   yz:   read + write the pair spectrum 24 + 24 (plus the tensor octant once per launch)
#   xinv: read the spectrum 24, read s 12, write sp 12
#   arc:  read sp 12 (its last CTAs then reduce per-image partials and write the interpolation table)
KERNEL_NAMES = ("xfwd", "yz", "xinv", "arc")
BYTES_PER_SITE_IMAGE = {"xfwd": 48, "yz": 48, "xinv": 48, "arc": 12, "spline": 24}
# the climbing-image kernels touch one image per string: F, s at kc and kc +- 1 read twice, the step written
CLIMB_BYTES_PER_SITE = 9 * 12
REF_IMAGES = 8


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=("ours", "reference"), default="ours")
    p.add_argument("--iters", type=int, default=None, help="iterations per step (default: the workload's)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-accuracy", action="store_true", help="skip the FP64-GPU barrier comparison")
    p.add_argument("--no-other-workloads", action="store_true", help="skip the short runs of the batch workloads")
    p.add_argument("--variant", choices=tuple(VARIANTS), default="plain",
                   help="run the timed steps under a method variant (the headline is 'plain')")
    return p.parse_args()


# method variants: (interpolation, climbing image, integrator, dynamics)
VARIANTS = {
    "plain": ("linear", False, "euler", "string"),
    "spline": ("spline", False, "euler", "string"),
    "climbing_image": ("linear", True, "euler", "string"),
    "spline_and_climbing_image": ("spline", True, "euler", "string"),
    "dopri5_per_string": ("linear", False, "dopri5", "string"),
    "dopri5_per_image": ("linear", False, "dopri5_image", "string"),
    "llg_euler": ("linear", False, "euler", "llg"),
}
LLG_ALPHA = 0.1


def apply_variant(binding, sm, name, rtol=1e-6, atol=1e-8):
    interp, climb, integ, dyn = VARIANTS[name]
    if dyn == "llg":
        sm.set_dynamics(binding.SS_DYN_LLG, LLG_ALPHA)
    sm.set_reparam(binding.SS_INTERP_SPLINE if interp == "spline" else binding.SS_INTERP_LINEAR, climb)
    if integ != "euler":
        sm.set_integrator(binding.SS_INT_DOPRI5 if integ == "dopri5" else binding.SS_INT_DOPRI5_IMAGE, rtol, atol)


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = max(mx, float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_sample(spec, dt, n_images=REF_IMAGES):
    """One oracle iteration (field, step, reparam) of the first n_images images of the workload's path."""
    import oracle
    cores = len(os.sched_getaffinity(0))
    oracle.set_threads(cores)
    m = oracle.model(spec.nx, spec.ny, spec.nz, spec.J, spec.D, spec.K, spec.w)
    path = spec.initial_path()[:n_images]
    t0 = time.perf_counter()
    oracle.string_run(m, path, 1, dt, with_energies=False)
    t = time.perf_counter() - t0
    units = spec.n_sites * n_images
    return units / t, min(cores, n_images), t  # the oracle's threads run over images


def kernel_source_hash():
    h = hashlib.sha256()
    for f in sorted(os.listdir(os.path.join(ROOT, "paper_1804_07135_gb300", "csrc"))):
        with open(os.path.join(ROOT, "paper_1804_07135_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, units: int):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it was taken on these sources."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        with open(path) as f:
            for line in f:
                if line.startswith("#") or not line.strip():
                    continue
                kv = dict(x.split("=", 1) for x in line.split())
                if kv.get("kernel") == kernel and kv.get("sources") == kernel_source_hash():
                    per_unit = float(kv["dram_bytes"]) / float(kv["units"])
                    return per_unit * units
    except (OSError, ValueError, KeyError):
        pass
    return None


def max_over_ranks(pg, values, device):
    """Each timing's maximum over the ranks (the slowest replica sets the job's time); pg is
    torch.distributed or None for one rank."""
    if pg is None:
        return list(values)
    import torch
    t = torch.tensor(values, device=device, dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return t.tolist()


def whole_job_value(units_per_rank, world, seconds):
    """Weak scaling: every rank runs its own replica of the workload, so the job processes
    world x units in the slowest rank's time."""
    return units_per_rank * world / seconds


def run_reference(args, rank, world):
    if rank != 0:
        return
    wl = workloads.bloch_collapse()
    spec = wl.strings[0]
    times = []
    cores = len(os.sched_getaffinity(0))
    for i in range(args.warmup + args.steps):
        v, cores, t = cpu_oracle_sample(spec, wl.dt)
        if i >= args.warmup:
            times.append(t)
    units = spec.n_sites * REF_IMAGES
    value = units * len(times) / sum(times)
    sample = f"one oracle iteration (direct O(N^2) dipole) of the first {REF_IMAGES} images of the 64x64x8 path"
    line = {
        "impl": "reference", "metric": "spin-updates/s", "value": value, "unit": "spin-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "lattice": [spec.nx, spec.ny, spec.nz], "images": REF_IMAGES,
                   "iterations_per_step": 1},
        "cpu_baseline": {"value": value, "unit": "spin-updates/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "spin-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, local_rank, world = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    from paper_1804_07135_gb300 import binding

    torch.cuda.set_device(local_rank)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
        pg = dist

    wl = workloads.bloch_collapse()
    spec = wl.strings[0]
    n_iter = args.iters or wl.n_iter
    desc = (spec.nx, spec.ny, spec.nz, spec.J, spec.D, spec.K, spec.w, spec.n_images)
    path = spec.initial_path().astype(np.float32)
    path_dev = torch.from_numpy(path).cuda()
    path_host = torch.from_numpy(path).pin_memory()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    sm = binding.StringMethod([desc], dt=wl.dt, stream=stream.cuda_stream)
    apply_variant(binding, sm, args.variant)
    kpi = sm.kernels_per_iteration()

    def one_step(src):
        sm.set_path(0, src)
        sm.step(n_iter)
        return sm.barrier(0)

    def timed(src, n):
        out = []
        for _ in range(n):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            one_step(src)
            e1.record(stream)
            torch.cuda.synchronize()
            out.append(e0.elapsed_time(e1) / 1e3)
        return out

    def barrier_all():
        if pg:
            pg.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        one_step(path_dev)
    barrier_all()
    rk = VARIANTS[args.variant][2] != "euler"
    with ClockSampler(local_rank) as clk:
        t_dev = timed(path_dev, args.steps)
        if rk:  # attempts of the last timed step (set_path restarts the counts each step)
            rk_attempts = [sum(sm.integrator_state(0, k)[1:]) for k in range(spec.n_images)]
        barrier_all()
        t_e2e = timed(path_host, args.steps)
        barrier_all()
    step_s, e2e_s = max_over_ranks(pg, [float(np.mean(t_dev)), float(np.mean(t_e2e))], "cuda")
    units = spec.n_sites * spec.n_images * n_iter
    value = whole_job_value(units, world, step_s)
    e2e_value = whole_job_value(units, world, e2e_s)
    dE, kmax = sm.barrier(0)

    if rank != 0:
        sm.close()
        if pg:
            pg.destroy_process_group()
        return

    # per-kernel roofline (kernels launched one by one on the library stream, CUDA-event timed)
    sm.set_path(0, path_dev)
    if rk:  # the field kernels are timed in the Euler iteration
        sm.set_integrator(binding.SS_INT_EULER)
    ms = sm.time_kernels(reps=20)
    interp, climb, integ, dyn = VARIANTS[args.variant]
    names = ["xfwd", "yz", "xinv"] + (["climb"] if climb else []) + ["arc"] + (["spline"] if interp == "spline" else [])
    share = ms / ms.sum()
    dom = int(np.argmax(ms))
    dname = names[dom]
    launch_units = spec.n_sites * spec.n_images
    peaks, peak_kind = measured_peaks()
    alg_bytes = (CLIMB_BYTES_PER_SITE * spec.n_sites if dname == "climb" else
                 BYTES_PER_SITE_IMAGE[dname] * launch_units)
    if dname == "yz":
        alg_bytes += 4 * 6 * spec.nz * (padded(spec.nx) // 2 + 1) * (padded(spec.ny) // 2 + 1)
    achieved = alg_bytes / (ms[dom] * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": dname, "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "peak_source": peak_kind,
                "traffic": ncu_traffic(dname, launch_units),
                "kernel_ms": {n: float(v) for n, v in zip(names, ms)},
                "kernel_share": {n: float(v) for n, v in zip(names, share)},
                "launch_config": sm.launch_config(0),
                "x_config_env": "SS_X_CONFIG={threads_xfwd}:{rows_xfwd}:{threads_xinv}:{rows_xinv}".format(**sm.launch_config(0)),
                "alg_bytes_per_launch": alg_bytes}
    if "yz" in names:
        # the y/z kernel is not HBM-bound (its working set is L2-resident): its FP32 arithmetic against
        # the FP32 (non-tensor) peak, 152 SMs x 128 FMA lanes x 2 FLOP x the maximum SM clock
        flops = yz_flops(spec)
        peak_tf = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        ach_tf = flops / (ms[names.index("yz")] * 1e-3) / 1e12
        roofline["secondary"] = {"kernel": "yz", "bound": "alu", "achieved": ach_tf, "peak": peak_tf,
                                 "unit": "TFLOP/s", "frac": ach_tf / peak_tf, "flops_per_launch": flops,
                                 "peak_source": "152 SMs x 128 FP32 lanes x 2 x sm_max_mhz"}

    line = {
        "metric": "spin-updates/s", "value": value, "unit": "spin-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl.name, "variant": args.variant, "lattice": [spec.nx, spec.ny, spec.nz],
                   "images": spec.n_images,
                   "iterations_per_step": n_iter, "dt": wl.dt, "J": spec.J, "D": spec.D, "K": spec.K, "w": spec.w,
                   "padded_xy": [padded(spec.nx), padded(spec.ny)],
                   "precision": "fp32 spins, fields and FFTs; fp64 energy and arc-length reductions",
                   "l2": "flushed before every step (256 MB write); the step's working set stays on chip across its iterations",
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": e2e_value, "unit": "spin-updates/s", "h2d_bytes_per_step": int(path.nbytes),
                "d2h_bytes_per_step": int(spec.n_images * 8)},
        "gpu_launches": int(args.steps * (2 + n_iter * kpi + 4)) if not rk else
        # per attempt round 7 x (assemble, x-forward, y/z, x-inverse) + finish, control, commit; per
        # iteration the gather, the controller's start and the arc kernel; rounds = the string's attempts
        # (per-image control: the most attempts of one image, a lower bound)
        int(args.steps * (2 + 4 + 3 * n_iter + (7 * kpi + 3) *  # kpi: the 3 or 4 field kernels and arc -> assemble
                          (max(rk_attempts) if args.variant == "dopri5_per_image" else rk_attempts[0]))),
        "roofline": roofline,
        "clocks": clk.summary(),
        "barrier": {"dE": dE, "k_max": kmax},
    }
    if not args.no_accuracy:
        iters64 = min(n_iter, 200)
        with binding.StringMethod([desc], dt=wl.dt, precision=binding.SS_PREC_FP64, stream=stream.cuda_stream) as s64:
            s64.set_path(0, path_dev)
            s64.step(1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s64.step(iters64)
            torch.cuda.synchronize()
            t64 = time.perf_counter() - t0
            s64.set_path(0, path_dev)
            s64.step(n_iter)
            dE64, k64 = s64.barrier(0)
        line["fp64_gpu"] = {"value": spec.n_sites * spec.n_images * iters64 / t64, "unit": "spin-updates/s",
                            "iterations_timed": iters64, "barrier_dE": dE64, "k_max": k64}
        line["speedup_vs_fp64_gpu"] = value / line["fp64_gpu"]["value"]
        line["barrier_abs_err_vs_fp64_gpu"] = abs(dE - dE64)
    if not args.no_other_workloads:
        line["other_workloads"] = {w.name: other_workload(binding, w, stream) for w in
                                   (workloads.boundary_sweep(), workloads.uneven_study(),
                                    workloads.paper_monolayer_workload(), workloads.paper_phase_diagram())}
        line["variants"] = variant_runs(binding, wl, stream, plain_ms=step_s * 1e3 / n_iter)
        line["adaptive_rk"] = {name: adaptive_rk(binding, wl, stream, kind, per_iter_euler_ms=step_s * 1e3 / n_iter)
                               for name, kind in (("dopri5_per_string", binding.SS_INT_DOPRI5),
                                                  ("dopri5_per_image", binding.SS_INT_DOPRI5_IMAGE))}
    if not args.no_cpu_baseline and world == 1:
        v, cores, t = cpu_oracle_sample(spec, wl.dt)
        line["cpu_baseline"] = {"value": v, "unit": "spin-updates/s", "cores": cores, "kind": "oracle",
                                "sample": f"one oracle iteration (direct O(N^2) dipole) of the first {REF_IMAGES} "
                                          f"images of the 64x64x8 path, {t:.1f} s"}
    sm.close()
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


def variant_runs(binding, wl, stream, plain_ms, iters=128, warm=64):
    """Device-timed Euler iterations of the bench workload under the variants that replay a CUDA graph
    (natural cubic spline, climbing image, both, precessional LLG), inputs resident."""
    import torch
    spec = wl.strings[0]
    desc = (spec.nx, spec.ny, spec.nz, spec.J, spec.D, spec.K, spec.w, spec.n_images)
    out = {}
    for name in ("spline", "climbing_image", "spline_and_climbing_image", "llg_euler"):
        with binding.StringMethod([desc], dt=wl.dt, stream=stream.cuda_stream) as sm:
            apply_variant(binding, sm, name)
            sm.set_path(0, torch.from_numpy(spec.initial_path().astype(np.float32)).cuda())
            sm.step(warm)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            sm.step(iters)
            e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 1e3
            kc = sm.climbing_image(0)
            kpi = sm.kernels_per_iteration()
        units = spec.n_sites * spec.n_images
        out[name] = {"value": units * iters / t, "unit": "spin-updates/s", "iterations_timed": iters,
                     "ms_per_iter": 1e3 * t / iters, "vs_plain_ms_per_iter": (1e3 * t / iters) / plain_ms,
                     "kernels_per_iter": kpi, "climbing_image": kc}
        if name == "llg_euler":
            out[name]["alpha"] = LLG_ALPHA
    return out


def adaptive_rk(binding, wl, stream, kind, per_iter_euler_ms, iters=10, warm=2, rtol=1e-6, atol=1e-8):
    """Device-timed Dormand-Prince evolution of the bench workload (each iteration integrates every image
    over the workload's dt, then reparametrises): spin-updates/s counted like the Euler path (N K per
    iteration) and force evaluations/s (7 per attempt and site-image), inputs resident."""
    import torch
    spec = wl.strings[0]
    desc = (spec.nx, spec.ny, spec.nz, spec.J, spec.D, spec.K, spec.w, spec.n_images)
    with binding.StringMethod([desc], dt=wl.dt, stream=stream.cuda_stream) as sm:
        sm.set_integrator(kind, rtol, atol)
        sm.set_path(0, torch.from_numpy(spec.initial_path().astype(np.float32)).cuda())
        sm.step(warm)
        _, a0, r0 = sm.integrator_state(0)
        att0 = [sum(sm.integrator_state(0, k)[1:]) for k in range(spec.n_images)]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        sm.step(iters)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        step, a1, r1 = sm.integrator_state(0)
        att1 = [sum(sm.integrator_state(0, k)[1:]) for k in range(spec.n_images)]
    units = spec.n_sites * spec.n_images
    attempts = a1 + r1 - a0 - r0  # summed over the string's systems
    # every system of the group takes part in each round, so the rounds per interval are set by the
    # system with the most attempts; with one system per string they equal its attempts
    rounds = max(b - a for a, b in zip(att0, att1)) if kind == binding.SS_INT_DOPRI5_IMAGE else attempts
    return {"value": units * iters / t, "unit": "spin-updates/s", "iterations_timed": iters, "rtol": rtol,
            "atol": atol, "interval": wl.dt, "ms_per_iter": 1e3 * t / iters,
            "attempts_per_iter": attempts / iters, "accepted": a1 - a0, "rejected": r1 - r0,
            "rounds_per_iter_min": rounds / iters, "carried_step_min": step,
            "force_evals_per_s": 7 * units * rounds / t,
            "ms_per_round_vs_7_euler_iters": (1e3 * t / max(rounds, 1)) / (7 * per_iter_euler_ms)}


def other_workload(binding, wl, stream, iters=20, warm=3):
    """Device-timed spin-updates/s of a short run of another workload (a batch of strings in one
    context): `iters` graph-replayed iterations after `warm`, inputs resident."""
    import torch
    descs = [(s.nx, s.ny, s.nz, s.J, s.D, s.K, s.w, s.n_images) for s in wl.strings]
    with binding.StringMethod(descs, dt=wl.dt, stream=stream.cuda_stream) as sm:
        for i, s in enumerate(wl.strings):
            sm.set_path(i, torch.from_numpy(s.initial_path().astype(np.float32)).cuda())
        sm.step(warm)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        sm.step(iters)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        ms = sm.time_kernels(reps=3)
    return {"value": wl.spin_updates_per_iter * iters / t, "unit": "spin-updates/s", "iterations_timed": iters,
            "strings": len(wl.strings), "spin_updates_per_iter": wl.spin_updates_per_iter,
            "ms_per_iter": 1e3 * t / iters, "kernel_ms_total": float(ms.sum())}


def yz_flops(spec):
    """Algorithmic FP32 operations of one y/z launch: per image pair and kx, the forward and inverse y
    transforms of 3 nz lines of length Py at the nominal 5 P log2 P each, and per frequency the
    z-convolution's 9 nz^2 real-by-complex products (4 FLOP each)."""
    px, py, nz = padded(spec.nx), padded(spec.ny), spec.nz
    pairs = (spec.n_images + 1) // 2
    fft = 2 * px * 3 * nz * 5 * py * math.log2(py)
    conv = px * py * 36 * nz * nz
    return pairs * (fft + conv)


def padded(n):
    """The library's padded transform length: smallest 2^a 3^b >= 2n - 1, or the power of two >= 2n - 1
    when that is at most 1/8 longer."""
    m = max(1, 2 * n - 1)
    while True:
        q = m
        while q % 2 == 0:
            q //= 2
        while q % 3 == 0:
            q //= 3
        if q == 1:
            break
        m += 1
    p2 = 1
    while p2 < 2 * n - 1:
        p2 *= 2
    return p2 if 8 * p2 <= 9 * m else m


if __name__ == "__main__":
    main()
