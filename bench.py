#!/usr/bin/env python
"""Throughput of the string method on one GB300 (or N replicas under torchrun).

Headline workload: the uneven-size parameter study -- 20 strings of 32 images on lattices drawn from
{64^2 x 4, 96^2 x 4, 128^2 x 8, 192^2 x 8} (seed 7), K ~ U[0, 0.2], D ~ U[0.15, 0.4], w = 0.01, dipole by
FFT convolution, dt = 0.1: four size groups, 72.1M spin-updates per iteration.  One bench step is the
whole hot path once over that batch: set the 20 initial paths, run ITERS_PER_STEP iterations (field,
step, per-image energies, equal-arc-length reparametrisation), evaluate the 20 barriers in FP64.
Metric: spin-updates/s = sum over strings of spins x images x iterations / time.  The study runs 5000
iterations in all; a step runs ITERS_PER_STEP of them so that the timed region stays near a minute.

  value     device-timed (CUDA events on the calling stream), initial paths already resident in HBM
  e2e       the same through the public API with the paths copied from pinned host memory each step and
            the energies read back
  roofline  the dominant kernel's algorithmic bytes per launch / its mean event-timed duration
  cpu_baseline / --impl reference   the FP64 CPU oracle on a bounded sample (one iteration of an
            8-image sub-string of the study's first 64 x 64 x 4 string), timed on this host's cores

The line also carries the previous headline (the 64x64x8, 32-image Bloch-point string, 2000 iterations
per step, with its FP64-GPU barrier comparison), the other workloads, the method variants and the plain
FP64 GPU method's rate on the headline workload.

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
    p.add_argument("--iters", type=int, default=None, help=f"iterations per step (default {ITERS_PER_STEP})")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-accuracy", action="store_true", help="skip the FP64-GPU barrier comparison")
    p.add_argument("--no-other-workloads", action="store_true", help="skip the short runs of the batch workloads")
    p.add_argument("--variant", choices=tuple(VARIANTS), default="plain",
                   help="run the timed steps under a method variant (the headline is 'plain')")
    p.add_argument("--workload", choices=tuple(WORKLOADS), default=HEADLINE,
                   help=f"the timed workload (default: the headline, {HEADLINE})")
    p.add_argument("--lattice", default=None, help="time only the workload's strings of this lattice, NXxNYxNZ")
    p.add_argument("--strings", type=int, default=None, help="time only the first K strings (after --lattice)")
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


def rk_kind(binding, integ):
    """The library's integrator constant for a variant's Runge-Kutta integrator name."""
    return binding.SS_INT_DOPRI5 if integ == "dopri5" else binding.SS_INT_DOPRI5_IMAGE


def apply_variant(binding, sm, name, rtol=1e-6, atol=1e-8):
    interp, climb, integ, dyn = VARIANTS[name]
    if dyn == "llg":
        sm.set_dynamics(binding.SS_DYN_LLG, LLG_ALPHA)
    sm.set_reparam(binding.SS_INTERP_SPLINE if interp == "spline" else binding.SS_INTERP_LINEAR, climb)
    if integ != "euler":
        sm.set_integrator(rk_kind(binding, integ), rtol, atol)


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


ITERS_PER_STEP = 200       # iterations of the headline workload per bench step (of its 5000)
C2_ITERS_PER_STEP = 2000   # the 64x64x8 string: its full iteration count per step


def headline_workload():
    return workloads.uneven_study()


# the workloads bench.py can time (the first is the headline); the others are also measured briefly in
# the headline run's side entries
WORKLOADS = {w.name: w for w in (workloads.uneven_study(), workloads.bloch_collapse(), workloads.boundary_sweep(),
                                 workloads.paper_monolayer_workload(), workloads.paper_phase_diagram())}
HEADLINE = headline_workload().name


def selected_workload(name, lattice=None, n_strings=None):
    """The named workload, restricted to the strings of one lattice ("NXxNYxNZ") and to its first
    n_strings strings when given (small cases of the same kernels, e.g. for ncu captures)."""
    wl = WORKLOADS[name]
    strings, tag = list(wl.strings), []
    n_total = len(strings)
    if lattice:
        strings = [s for s in strings if f"{s.nx}x{s.ny}x{s.nz}" == lattice]
        if not strings:
            raise SystemExit(f"{name} has no {lattice} strings")
        tag.append(lattice)
    if n_strings:
        strings = strings[:n_strings]
        tag.append(f"{len(strings)} of {n_total} strings")
    if not tag:
        return wl
    return workloads.Workload(f"{wl.name}[{', '.join(tag)}]", tuple(strings), wl.n_iter, wl.dt)


def oracle_sample_spec(wl=None):
    """The string the CPU baseline samples: the workload's first string of the smallest lattice (the
    oracle's direct dipole sum costs N^2 per image); for the headline study its first 64 x 64 x 4 string."""
    wl = wl or headline_workload()
    return min(wl.strings, key=lambda s: s.n_sites)


def oracle_sample_images(spec):
    """Images of the sample: REF_IMAGES for lattices up to 64 x 64 x 4 sites, fewer (at least 2) for
    larger ones, so that the sample's N^2 cost stays near that of 8 images of 16384 sites."""
    return max(2, min(REF_IMAGES, int(REF_IMAGES * (16384 / spec.n_sites) ** 2)))


def cpu_oracle_sample(spec, dt, n_images=REF_IMAGES, threads=None):
    """One oracle iteration (field, step, reparam) of the first n_images images of spec's path; returns
    (spin-updates/s, threads used, seconds)."""
    import oracle
    cores = len(os.sched_getaffinity(0)) if threads is None else threads
    oracle.set_threads(cores)
    m = oracle.model(spec.nx, spec.ny, spec.nz, spec.J, spec.D, spec.K, spec.w)
    path = spec.initial_path()[:n_images]
    t0 = time.perf_counter()
    oracle.string_run(m, path, 1, dt, with_energies=False)
    t = time.perf_counter() - t0
    units = spec.n_sites * n_images
    return units / t, min(cores, n_images), t  # the oracle's threads run over images


def oracle_sample_text(spec, n_images=REF_IMAGES, wl_name=None):
    return (f"one oracle iteration (direct O(N^2) dipole) of the first {n_images} images of "
            f"{wl_name or headline_workload().name}'s first {spec.nx}x{spec.ny}x{spec.nz} string")


# the files that define the iteration's kernels (the host-side API and the no-allocation entry point
# launch them but do not change their code)
KERNEL_SOURCES = ("ss_fft.cuh", "ss_internal.h", "ss_kernels.cuh", "ss_kernels_f32.cu", "ss_kernels_f64.cu")


def kernel_source_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
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
    wl = selected_workload(args.workload, args.lattice, args.strings)
    spec = oracle_sample_spec(wl)
    n_img = oracle_sample_images(spec)
    times = []
    cores = len(os.sched_getaffinity(0))
    for i in range(args.warmup + args.steps):
        v, cores, t = cpu_oracle_sample(spec, wl.dt, n_img)
        if i >= args.warmup:
            times.append(t)
    units = spec.n_sites * n_img
    value = units * len(times) / sum(times)
    line = {
        "impl": "reference", "metric": "spin-updates/s", "value": value, "unit": "spin-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "sampled_string": [spec.nx, spec.ny, spec.nz], "images": n_img,
                   "iterations_per_step": 1},
        "cpu_baseline": {"value": value, "unit": "spin-updates/s", "cores": cores, "kind": "oracle",
                         "sample": oracle_sample_text(spec, n_img, wl.name)},
        "e2e": {"value": value, "unit": "spin-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def working_set_gb(wl):
    """Device bytes an iteration touches (GB): per string the FP32 state before and after the step
    (2 x 12 bytes per site-image) and the complex spectrum of its image pairs (Px x ny x nz x 3 x 8
    bytes per pair)."""
    b = 0
    for s in wl.strings:
        b += 24 * s.n_sites * s.n_images + (s.n_images + 1) // 2 * padded(s.nx) * s.ny * s.nz * 24
    return b / 1e9


def l2_note(wl):
    ws = working_set_gb(wl)
    where = "exceeds the 129 MB L2" if ws > 0.129 else "stays in L2 across a step's iterations"
    return f"flushed before every step (256 MB write); the working set (about {ws:.2g} GB) {where}"


def group_keys(wl):
    """Size groups of a workload in the library's order (first appearance) with their image counts."""
    keys, imgs = [], {}
    for s in wl.strings:
        k = (s.nx, s.ny, s.nz)
        if k not in imgs:
            keys.append(k)
            imgs[k] = 0
        imgs[k] += s.n_images
    return keys, imgs


def kernel_roofline(sm, wl, names_per_group, peaks, peak_kind, ms):
    """The dominant kernel's HBM roofline: algorithmic bytes per launch / event-timed mean duration."""
    keys, imgs = group_keys(wl)
    entries = []
    i = 0
    for k in keys:
        for n in names_per_group:
            entries.append((k, n))
            i += 1
    dom = int(np.argmax(ms))
    (nx, ny, nz), dname = entries[dom]
    units = nx * ny * nz * imgs[(nx, ny, nz)]
    alg = BYTES_PER_SITE_IMAGE[dname] * units
    if dname == "yz":
        alg += 4 * 6 * nz * (padded(nx) // 2 + 1) * (padded(ny) // 2 + 1)
    achieved = alg / (ms[dom] * 1e-3) / 1e9
    tag = f"{dname}[{nx}x{ny}x{nz}]"
    total_alg = sum(BYTES_PER_SITE_IMAGE[n] * k[0] * k[1] * k[2] * imgs[k] for k, n in entries)
    secondary = None
    if dname == "yz":
        # the y/z kernel's FP32 arithmetic against the FP32 (non-tensor) peak of this device: its SM count
        # x 128 FP32 lanes x 2 FLOP x the maximum SM clock
        import torch
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        peak_tf = sms * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        flops = yz_flops_group(nx, ny, nz, imgs[(nx, ny, nz)])
        ach_tf = flops / (ms[dom] * 1e-3) / 1e12
        secondary = {"kernel": tag, "bound": "alu", "achieved": ach_tf, "peak": peak_tf, "unit": "TFLOP/s",
                     "frac": ach_tf / peak_tf, "flops_per_launch": flops,
                     "peak_source": f"{sms} SMs (device query) x 128 FP32 lanes x 2 x sm_max_mhz"}
    return {"bound": "hbm", "kernel": tag, "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "peak_source": peak_kind, "secondary": secondary,
            "traffic": ncu_traffic(tag, units), "alg_bytes_per_launch": alg, "units_per_launch": units,
            "kernel_ms": {f"{n}[{k[0]}x{k[1]}x{k[2]}]": float(v) for (k, n), v in zip(entries, ms)},
            "kernel_share": {f"{n}[{k[0]}x{k[1]}x{k[2]}]": float(v / ms.sum()) for (k, n), v in zip(entries, ms)},
            "iteration": {"alg_bytes": total_alg, "kernel_ms_sum": float(ms.sum()),
                          "achieved_gbs": total_alg / (ms.sum() * 1e-3) / 1e9,
                          "frac": total_alg / (ms.sum() * 1e-3) / 1e9 / peaks["hbm_gbs"]}}


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

    wl = selected_workload(args.workload, args.lattice, args.strings)
    n_iter = args.iters or ITERS_PER_STEP
    n_str = len(wl.strings)
    descs = [(s.nx, s.ny, s.nz, s.J, s.D, s.K, s.w, s.n_images) for s in wl.strings]
    paths = [s.initial_path().astype(np.float32) for s in wl.strings]
    paths_dev = [torch.from_numpy(p).cuda() for p in paths]
    paths_host = [torch.from_numpy(p).pin_memory() for p in paths]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    sm = binding.StringMethod(descs, dt=wl.dt, stream=stream.cuda_stream)
    apply_variant(binding, sm, args.variant)
    kpi = sm.kernels_per_iteration()

    def one_step(srcs):
        for i, src in enumerate(srcs):
            sm.set_path(i, src)
        sm.step(n_iter)
        return [sm.barrier(i) for i in range(n_str)]

    def timed(srcs, n):
        out = []
        for _ in range(n):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            one_step(srcs)
            e1.record(stream)
            torch.cuda.synchronize()
            out.append(e0.elapsed_time(e1) / 1e3)
        return out

    def barrier_all():
        if pg:
            pg.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        one_step(paths_dev)
    barrier_all()
    rk = VARIANTS[args.variant][2] != "euler"
    with ClockSampler(local_rank) as clk:
        t_dev = timed(paths_dev, args.steps)
        if rk:  # attempts of the last timed step of string 0 (set_path restarts the counts each step)
            rk_attempts = [sum(sm.integrator_state(0, k)[1:]) for k in range(wl.strings[0].n_images)]
        barrier_all()
        one_step(paths_host)  # one untimed step of the end-to-end path (its first host upload is the slowest)
        barrier_all()
        t_e2e = timed(paths_host, args.steps)
        barrier_all()
    step_s, e2e_s = max_over_ranks(pg, [float(np.mean(t_dev)), float(np.mean(t_e2e))], "cuda")
    units = wl.spin_updates_per_iter * n_iter
    value = whole_job_value(units, world, step_s)
    e2e_value = whole_job_value(units, world, e2e_s)
    barriers = [sm.barrier(i) for i in range(n_str)]

    if rank != 0:
        sm.close()
        if pg:
            pg.destroy_process_group()
        return

    # per-kernel roofline (kernels launched one by one on the library stream, CUDA-event timed)
    for i, p in enumerate(paths_dev):
        sm.set_path(i, p)
    rk_kernels = None
    if rk:  # the round's kernels one by one (single-string workloads), then the field kernels in the Euler iteration
        if n_str == 1:
            rk_kernels = rk_kernel_times(binding, sm, wl.strings[0], rk_kind(binding, VARIANTS[args.variant][2]))
        sm.set_integrator(binding.SS_INT_EULER)
    ms = sm.time_kernels(reps=10)
    interp, climb, integ, dyn = VARIANTS[args.variant]
    names = ["xfwd", "yz", "xinv"] + (["climb"] if climb else []) + ["arc"] + (["spline"] if interp == "spline" else [])
    peaks, peak_kind = measured_peaks()
    roofline = kernel_roofline(sm, wl, names, peaks, peak_kind, ms) if not climb else None
    keys, _ = group_keys(wl)
    line = {
        "metric": "spin-updates/s", "value": value, "unit": "spin-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl.name, "variant": args.variant, "strings": n_str,
                   "images": int(sum(s.n_images for s in wl.strings)),
                   "lattices": sorted({f"{s.nx}x{s.ny}x{s.nz}" for s in wl.strings}),
                   "padded_xy": {f"{k[0]}x{k[1]}x{k[2]}": [padded(k[0]), padded(k[1])] for k in keys},
                   "spin_updates_per_iteration": wl.spin_updates_per_iter,
                   "iterations_per_step": n_iter, "workload_iterations": wl.n_iter, "dt": wl.dt, "w": 0.01,
                   "precision": "fp32 spins, fields and FFTs; fp64 energy and arc-length reductions; "
                                "barriers from an fp64 evaluation of the fp32 state",
                   "l2": l2_note(wl),
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": e2e_value, "unit": "spin-updates/s",
                "h2d_bytes_per_step": int(sum(p.nbytes for p in paths)),
                "d2h_bytes_per_step": int(sum(8 * s.n_images for s in wl.strings))},
        # per step: the 20 path uploads (conversion kernels), n_iter graph-replayed iterations, and per
        # size group the FP64 evaluation of the barriers (gather, widen, x-forward, y/z, x-inverse, reduce)
        "gpu_launches": int(args.steps * (2 * n_str + n_iter * kpi + 6 * len(keys))) if not rk else None,
        "roofline": roofline,
        "clocks": clk.summary(),
        "barriers": [{"dE": b[0], "k_max": b[1]} for b in barriers],
    }
    if rk_kernels:
        line["rk_kernels"] = rk_kernels
    if rk:
        # per iteration and group: the interval's opening (x-forward, control), per attempt round seven
        # stages of kpi launches, finish, control, commit and the round condition, and the arc kernel
        line["gpu_launches"] = int(args.steps * (2 * n_str + 6 * len(keys) + 3 * n_iter + (7 * kpi + 4) *
                                                 (max(rk_attempts) if args.variant == "dopri5_per_image" else rk_attempts[0])))
    if not args.no_accuracy:
        line["fp64_gpu"] = fp64_gpu_rate(binding, wl, stream, paths_dev)
        line["speedup_vs_fp64_gpu"] = line["fp64_gpu"]["ms_per_iter"] / (1e3 * step_s / n_iter)
    if not args.no_other_workloads:
        line["size_groups_alone"] = group_standalone(binding, wl, stream)
        line["bloch_64x64x8"] = bloch_64x64x8(binding, stream, peaks, peak_kind, no_accuracy=args.no_accuracy)
        line["other_workloads"] = {w.name: other_workload(binding, w, stream) for w in
                                   (workloads.boundary_sweep(), workloads.paper_monolayer_workload(),
                                    workloads.paper_phase_diagram())}
        c2 = workloads.bloch_collapse()
        line["variants"] = variant_runs(binding, c2, stream, plain_ms=line["bloch_64x64x8"]["ms_per_iter"])
        line["adaptive_rk"] = {name: adaptive_rk(binding, c2, stream, kind,
                                                 per_iter_euler_ms=line["bloch_64x64x8"]["ms_per_iter"])
                               for name, kind in (("dopri5_per_string", binding.SS_INT_DOPRI5),
                                                  ("dopri5_per_image", binding.SS_INT_DOPRI5_IMAGE))}
    if not args.no_cpu_baseline and world == 1:
        spec = oracle_sample_spec(wl)
        n_img = oracle_sample_images(spec)
        v, cores, t = cpu_oracle_sample(spec, wl.dt, n_img)
        v1, _, t1 = cpu_oracle_sample(spec, wl.dt, n_img, threads=1)
        line["cpu_baseline"] = {"value": v, "unit": "spin-updates/s", "cores": cores, "kind": "oracle",
                                "sample": f"{oracle_sample_text(spec, n_img, wl.name)}, {t:.1f} s",
                                "single_thread": {"value": v1, "cores": 1, "seconds": t1}}
    sm.close()
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


def fp64_gpu_rate(binding, wl, stream, paths_dev, iters=10):
    """The plain FP64 GPU method on the headline workload: device-timed iterations (CUDA events), the
    one-iteration graph captured in the warm-up so that no capture falls in the timed region."""
    import torch
    descs = [(s.nx, s.ny, s.nz, s.J, s.D, s.K, s.w, s.n_images) for s in wl.strings]
    with binding.StringMethod(descs, dt=wl.dt, precision=binding.SS_PREC_FP64, stream=stream.cuda_stream) as s64:
        for i, p in enumerate(paths_dev):
            s64.set_path(i, p)
        s64.step(1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s64.step(iters)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
    return {"value": wl.spin_updates_per_iter * iters / t, "unit": "spin-updates/s", "iterations_timed": iters,
            "ms_per_iter": 1e3 * t / iters}


def bloch_64x64x8(binding, stream, peaks, peak_kind, no_accuracy=False, steps=3):
    """The 64x64x8, 32-image Bloch-point string (2000 iterations per step, L2-resident working set):
    device-timed steps as the headline's, its kernel roofline, and the barrier against the plain FP64 GPU
    method after the same 2000 iterations (split into the evaluation and the drift of the FP32
    trajectory) with the FP64 method's rate (its 64-iteration graph captured before the timed region)."""
    import torch
    wl = workloads.bloch_collapse()
    spec = wl.strings[0]
    desc = (spec.nx, spec.ny, spec.nz, spec.J, spec.D, spec.K, spec.w, spec.n_images)
    path_dev = torch.from_numpy(spec.initial_path().astype(np.float32)).cuda()
    n_iter = C2_ITERS_PER_STEP
    out = {}
    with binding.StringMethod([desc], dt=wl.dt, stream=stream.cuda_stream) as sm:
        for _ in range(2):
            sm.set_path(0, path_dev)
            sm.step(n_iter)
            sm.barrier(0)
        ts = []
        for _ in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sm.set_path(0, path_dev)
            sm.step(n_iter)
            dE, k = sm.barrier(0)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        g32 = sm.get_path(0)
        sm.set_path(0, path_dev)
        ms = sm.time_kernels(reps=20)
        roof = kernel_roofline(sm, wl, ["xfwd", "yz", "xinv", "arc"], peaks, peak_kind, ms)
    t = float(np.mean(ts))
    units = spec.n_sites * spec.n_images * n_iter
    out.update({"value": units / t, "unit": "spin-updates/s", "iterations_per_step": n_iter,
                "ms_per_step": 1e3 * t, "ms_per_iter": 1e3 * t / n_iter, "barrier": {"dE": dE, "k_max": k},
                "l2": "the step's working set (about 55 MB) stays in L2 across its iterations",
                "roofline": roof})
    if not no_accuracy:
        with binding.StringMethod([desc], dt=wl.dt, precision=binding.SS_PREC_FP64, stream=stream.cuda_stream) as s64:
            s64.set_path(0, path_dev)
            s64.step(64)  # captures the 64-iteration graph outside the timed region
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s64.step(192)
            e1.record(stream)
            torch.cuda.synchronize()
            t64 = e0.elapsed_time(e1) / 1e3 / 192
            s64.set_path(0, path_dev)
            s64.step(n_iter)
            dE64, k64 = s64.barrier(0)
            s64.set_path(0, g32)  # the FP32 final state, evaluated by the FP64 method
            dE64_of_32, _ = s64.barrier(0)
        out["fp64_gpu"] = {"value": spec.n_sites * spec.n_images / t64, "unit": "spin-updates/s",
                           "iterations_timed": 192, "ms_per_iter": 1e3 * t64, "barrier_dE": dE64, "k_max": k64}
        out["speedup_vs_fp64_gpu"] = t64 / (t / n_iter)
        out["barrier_abs_err_vs_fp64_gpu"] = abs(dE - dE64)
        out["barrier_err_split"] = {"evaluation": dE - dE64_of_32, "drift": dE64_of_32 - dE64}
    return out


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


def rk_stages(binding, kind):
    return 7 if kind in (binding.SS_INT_DOPRI5, binding.SS_INT_DOPRI5_IMAGE) else 6


def rk_kernel_times(binding, sm, spec, kind, reps=5):
    """The kernels of one attempt round of a one-string, one-lattice context, each launched on its own
    (ss_time_kernels), summed by kind, with the element-wise Runge-Kutta kernels' rates."""
    stages = rk_stages(binding, kind)
    ms = sm.time_kernels(reps=reps)
    names = ["open"] + ["assemble", "xfwd", "yz", "xinv"] * stages + ["finish", "control", "commit", "arc"]
    per = {}
    for n, t in zip(names, ms):
        per[n] = per.get(n, 0.0) + float(t)
    units = spec.n_sites * spec.n_images
    # algorithmic bytes per site-image (FP32 components, 12 bytes per spin vector): stage s assembles
    # from y0 and s earlier stages into the stage state, (s + 2) x 12; finish reads y0 and every stage
    # and writes y5, (stages + 2) x 12
    b_asm = sum((st + 2) * 12 for st in range(stages)) * units
    b_fin = (stages + 2) * 12 * units
    peaks, _ = measured_peaks()
    return {"ms_per_round": {k: round(v, 5) for k, v in per.items()},
            "assemble_gbs": b_asm / (per["assemble"] * 1e-3) / 1e9,
            "finish_gbs": b_fin / (per["finish"] * 1e-3) / 1e9,
            "hbm_peak_gbs": peaks["hbm_gbs"],
            "note": f"launched one by one; the round's arrays (about {(stages + 4) * 12 * units / 1e9:.2g} GB) "
                    "may partly stay in L2, so these rates can exceed what HBM alone allows"}


def adaptive_rk(binding, wl, stream, kind, per_iter_euler_ms, iters=16, warm=9, rtol=1e-6, atol=1e-8):
    """Device-timed Dormand-Prince evolution of the bench workload (each iteration integrates every image
    over the workload's dt, then reparametrises): spin-updates/s counted like the Euler path (N K per
    iteration) and force evaluations/s (7 per attempt and site-image), inputs resident.  The warm-up
    (8 + 1 iterations) captures both of the integrator's graphs (8 iterations and one) before the timed
    region, which replays the 8-iteration graph twice."""
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
        rk_kernels = rk_kernel_times(binding, sm, spec, kind)
    units = spec.n_sites * spec.n_images
    stages = rk_stages(binding, kind)
    attempts = a1 + r1 - a0 - r0  # summed over the string's systems
    # every system of the group takes part in each round, so the rounds per interval are set by the
    # system with the most attempts; with one system per string they equal its attempts
    rounds = max(b - a for a, b in zip(att0, att1)) if kind == binding.SS_INT_DOPRI5_IMAGE else attempts
    return {"value": units * iters / t, "unit": "spin-updates/s", "iterations_timed": iters, "rtol": rtol,
            "atol": atol, "interval": wl.dt, "ms_per_iter": 1e3 * t / iters,
            "attempts_per_iter": attempts / iters, "accepted": a1 - a0, "rejected": r1 - r0,
            "rounds_per_iter_min": rounds / iters, "carried_step_min": step,
            "force_evals_per_s": stages * units * rounds / t,
            "ms_per_round_vs_7_euler_iters": (1e3 * t / max(rounds, 1)) / (7 * per_iter_euler_ms),
            "kernels": rk_kernels}


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


def group_standalone(binding, wl, stream, iters=20, warm=3):
    """Each size group of a batch workload run alone (its strings in a context of their own), device-timed
    as other_workload, against all groups in one context; the sum of the lone groups' times per iteration
    against the combined one shows what running the groups as concurrent graph branches saves."""
    import torch
    keys, _ = group_keys(wl)
    out = {}
    for k in keys + [None]:
        strings = [s for s in wl.strings if k is None or (s.nx, s.ny, s.nz) == k]
        descs = [(s.nx, s.ny, s.nz, s.J, s.D, s.K, s.w, s.n_images) for s in strings]
        with binding.StringMethod(descs, dt=wl.dt, stream=stream.cuda_stream) as sm:
            for i, s in enumerate(strings):
                sm.set_path(i, torch.from_numpy(s.initial_path().astype(np.float32)).cuda())
            sm.step(warm)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            sm.step(iters)
            e1.record(stream)
            torch.cuda.synchronize()
            out["combined" if k is None else f"{k[0]}x{k[1]}x{k[2]}"] = e0.elapsed_time(e1) / iters
    combined = out.pop("combined")
    total = sum(out.values())
    return {"ms_per_iter": out, "sum_ms_per_iter": total, "combined_ms_per_iter": combined,
            "combined_vs_sum": combined / total}


def yz_flops_group(nx, ny, nz, n_img):
    """yz_flops for a size group of n_img images (image pairs formed over the group)."""
    px, py = padded(nx), padded(ny)
    pairs = (n_img + 1) // 2
    fft = 2 * px * 3 * nz * 5 * py * math.log2(py)
    conv = px * py * 36 * nz * nz
    return pairs * (fft + conv)


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
