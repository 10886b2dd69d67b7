#!/usr/bin/env python
"""Benchmark: H|psi> throughput of the plane-wave Kohn-Sham operator on GB300.

Workload (one step): H|psi> on a block of 128 bands of the C1 cell -- cubic
a = 20 bohr, 64 seeded random atoms (min. separation 2.5 bohr), Gaussian
V_loc, 8 Gaussian projectors per atom (512), ecutwfc = 40 Ry (34 265 plane
waves), FFT grid 96^3, complex128 (FP64 path).  Inputs (beta 281 MB, psi 70 MB)
are larger than L2, so no explicit L2 flush is done between steps.

Also reported (not part of `value`): the mixed-precision H|psi> rate on the
same cell, per-kernel device times, the roofline of the dominant kernel, an
end-to-end rate through the C ABI with host buffers, the FP64 oracle on the
host cores, and the SM clocks sampled during the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Multi-GPU (torchrun): every rank runs its own replica of the workload
(independent band blocks, no collective on the data path); value = bands
processed by all ranks / max-over-ranks time (weak scaling).
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
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import qeinputs  # noqa: E402

METRIC = "Hψ bands/s & Davidson solves/s, mixed vs FP64 @1e-6 Ry; serve p50/p99"
WORKLOAD = "C1: H|psi> 128 bands, cubic a=20 bohr, 64 atoms, 512 projectors, 40 Ry (34265 PW), grid 96^3"
FP64_NOMINAL_TFLOPS = 1.25       # GB300 FP64 (vector and DMMA), nominal
FP32_NOMINAL_TFLOPS = 2.07e9 * 152 * 128 * 2 / 1e12   # 128 FP32 lanes/SM at 2.07 GHz


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def fft_flops(n):
    return 5.0 * n * math.log2(n) if n > 1 else 0.0


def kernel_flops(name, c, npw, nst, nax, nb, nproj):
    """Algorithmic FLOPs of one launch covering `nb` bands (5 N log2 N per
    length-N complex transform; 8 flops per complex multiply-add)."""
    n1, n2, n3 = c["grid"]
    if name in ("k_zinv", "k_zfwd"):
        return nb * nst * fft_flops(n3)
    if name == "k_plane":
        per_plane = 2 * (nax * fft_flops(n2) + n2 * fft_flops(n1)) + 2.0 * n1 * n2
        return nb * n3 * per_plane
    if name in ("k_gemm_inner", "k_gemm_outer"):
        return 8.0 * nproj * nb * npw
    if name == "k_dmul":
        return 4.0 * nproj * nproj * nb
    return 0.0


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms in the background."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def src_hash(*names):
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_2104_10502_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


KERNEL_SOURCES = {"k_plane": ("fft.cu", "fft_device.cuh"), "k_zinv": ("fft.cu", "fft_device.cuh"),
                  "k_zfwd": ("fft.cu", "fft_device.cuh"), "k_gemm_inner": ("gemm.cu",),
                  "k_gemm_outer": ("gemm.cu",), "k_dmul": ("gemm.cu",)}


def traffic_for(kernel, tag):
    """DRAM bytes per launch from the committed ncu summary, if the kernel's
    sources are unchanged since the capture (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
        e = d[f"{kernel}:{tag}"]
        if e.get("src") != src_hash(*KERNEL_SOURCES[kernel]):
            return None
        return e["bytes_per_launch"]
    except Exception:
        return None


def c1_cpu_inputs(c):
    import oracle
    lat, k, ecut, grid = c["lat"], c["k"], c["ecut"], c["grid"]
    v = oracle.vloc_gaussian(lat, grid, c["tau"])
    beta = oracle.beta_gaussian(lat, k, ecut, c["tau"], c["widths"])
    d = qeinputs.d_matrix(len(c["tau"]), len(c["widths"]))
    _, kin, _ = oracle.gsphere(lat, k, ecut)
    return v, beta, d, kin


def cpu_oracle_rate(c, inputs, nb_sample, reps):
    """Oracle H|psi> on `nb_sample` bands, `reps` times; returns bands/s."""
    import oracle
    v, beta, d, kin = inputs
    psi = qeinputs.start_bands(kin, nb_sample, c["psi_seed"])
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.hpsi(c["lat"], c["k"], c["ecut"], c["grid"], v, beta, d, psi)
    dt = time.perf_counter() - t0
    return nb_sample * reps / dt


def run_reference(args, rank):
    if rank != 0:
        return
    c = qeinputs.config("C1")
    cores = len(os.sched_getaffinity(0))
    inputs = c1_cpu_inputs(c)
    nb_sample = 2
    for _ in range(args.warmup):
        cpu_oracle_rate(c, inputs, nb_sample, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        cpu_oracle_rate(c, inputs, nb_sample, 1)
    dt = time.perf_counter() - t0
    value = nb_sample * args.steps / dt
    sample = f"{nb_sample} of the 128 C1 bands per step, FP64 NumPy/SciPy oracle"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "bands/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": value, "unit": "bands/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "bands/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gpu(args, rank, world, local_rank):
    import torch
    import paper_2104_10502_gb300 as q

    dist = world > 1
    if dist:
        import torch.distributed as td
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    c = qeinputs.config("C1")
    lat, k, ecut, grid = c["lat"], c["k"], c["ecut"], c["grid"]
    nb = c["nbnd"]
    ctx = q.Context(local_rank)
    _, kin = q.gsphere(lat, k, ecut, grid)
    npw = len(kin)
    natom = len(c["tau"])
    nproj = 4 * len(c["widths"]) * natom
    v = torch.empty((grid[2], grid[1], grid[0]), dtype=torch.float64, device=dev)
    ctx.vloc_gaussian(lat, grid, c["tau"], v)
    beta = torch.empty((nproj, npw, 2), dtype=torch.float64, device=dev)
    ctx.beta_gaussian(lat, k, ecut, c["tau"], c["widths"], beta)
    dmat_h = qeinputs.d_matrix(natom, len(c["widths"]))
    dmat = torch.from_numpy(dmat_h).to(dev)
    psi_h = qeinputs.start_bands(kin, nb, c["psi_seed"] + rank)
    psi = torch.from_numpy(psi_h.view(np.float64).reshape(nb, npw, 2).copy()).to(dev)
    hpsi = torch.empty_like(psi)
    prob = ctx.problem(lat, k, ecut, grid, v, beta, dmat, nb)
    stream = torch.cuda.current_stream(dev)

    def timed(precision, steps, warmup, prof=False):
        for _ in range(warmup):
            ctx.hpsi(prob, psi, hpsi, precision)
        torch.cuda.synchronize(dev)
        if dist:
            td.barrier()
        torch.cuda.synchronize(dev)
        if prof:
            ctx.profile(True)
        sampler = ClockSampler(local_rank) if prof else None
        if sampler:
            sampler.start()
            time.sleep(0.3)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            ctx.hpsi(prob, psi, hpsi, precision)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if dist:
            td.barrier()
        torch.cuda.synchronize(dev)
        clocks = sampler.stop() if sampler else None
        ms = e0.elapsed_time(e1)
        kern = None
        launches = None
        if prof:
            kern, launches = ctx.profile_read()
            ctx.profile(False)
        if dist:
            t = torch.tensor([ms], dtype=torch.float64, device=dev)
            td.all_reduce(t, op=td.ReduceOp.MAX)
            ms = float(t.item())
        return ms, kern, launches, clocks

    # FP64 (the headline) with per-kernel timing, then the mixed path
    ms64, kern, launches, clocks = timed(q.QE_FP64, args.steps, args.warmup, prof=True)
    ms_mixed, kern_mixed, _, _ = timed(q.QE_MIXED, args.steps, args.warmup, prof=True)
    value = world * nb * args.steps / (ms64 / 1e3)
    mixed_value = world * nb * args.steps / (ms_mixed / 1e3)

    # dominant kernel of the FP64 step and its roofline (FP64 ALU-bound):
    # algorithmic FLOPs of all its launches in the timed region / their device time
    pk, pk_kind = peaks()
    plan_nst, plan_nax = stick_counts(c)
    dom = max(kern, key=lambda n: kern[n][1])
    calls, tot = kern[dom]
    avg_ms = tot / calls
    fl_step = kernel_flops(dom, c, npw, plan_nst, plan_nax, nb, nproj)
    fl = fl_step * args.steps / calls
    achieved = fl_step * args.steps / (tot / 1e3) / 1e12
    roof = {"kernel": dom, "bound": "alu", "achieved": achieved, "peak": FP64_NOMINAL_TFLOPS,
            "unit": "TFLOP/s", "frac": achieved / FP64_NOMINAL_TFLOPS,
            "traffic": traffic_for(dom, "fp64"),
            "peak_source": "nominal FP64 of GB300 (recipe table); measured DFMA loop 1.17-1.19",
            "flops_per_launch": fl, "avg_launch_ms": avg_ms}
    kernels = {n: {"launches": kern[n][0], "ms": kern[n][1], "share": kern[n][1] / sum(x[1] for x in kern.values())}
               for n in kern}
    kernels_mixed = {n: {"launches": kern_mixed[n][0], "ms": kern_mixed[n][1]} for n in kern_mixed}

    # end to end through the C ABI with host (pinned) buffers, copies in the timed region
    e2e = None
    if True:
        pin = lambda shape: torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
        vh = pin(tuple(v.shape))
        vh[...] = v.cpu().numpy()
        bh = pin(tuple(beta.shape))
        bh[...] = beta.cpu().numpy()
        dh = pin(dmat_h.shape)
        dh[...] = dmat_h
        ph = pin((nb, npw, 2))
        ph[...] = psi.cpu().numpy()
        oh = pin((nb, npw, 2))
        prob_h = ctx.problem(lat, k, ecut, grid, vh, bh, dh, nb)
        esteps = max(3, args.steps // 4)
        for _ in range(2):
            ctx.hpsi(prob_h, ph, oh, q.QE_FP64)
        if dist:
            td.barrier()
        t0 = time.perf_counter()
        for _ in range(esteps):
            ctx.hpsi(prob_h, ph, oh, q.QE_FP64)
        dt = time.perf_counter() - t0
        if dist:
            t = torch.tensor([dt], dtype=torch.float64, device=dev)
            td.all_reduce(t, op=td.ReduceOp.MAX)
            dt = float(t.item())
        h2d = vh.nbytes + bh.nbytes + dh.nbytes + ph.nbytes
        e2e = {"value": world * nb * esteps / dt, "unit": "bands/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(oh.nbytes), "steps": esteps}

    line = None
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            cinp = c1_cpu_inputs(c)
            cpu_oracle_rate(c, cinp, 1, 1)
            rate = cpu_oracle_rate(c, cinp, 2, 3)
            cpu = {"value": rate, "unit": "bands/s", "cores": len(os.sched_getaffinity(0)),
                   "kind": "oracle", "sample": "6 band applications (3 x 2 bands) of the C1 workload"}
        line = {"metric": METRIC, "value": value, "unit": "bands/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms64 / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "bands": nb, "npw": npw, "nproj": nproj,
                           "grid": list(grid), "l2": "inputs larger than L2 (beta 281 MB, psi 70 MB); no flush",
                           "parallelism": f"replicas x{world}"},
                "e2e": e2e, "gpu_launches": launches, "clocks": clocks, "roofline": roof,
                "cpu_baseline": cpu,
                "mixed": {"value": mixed_value, "unit": "bands/s", "ms_per_step": ms_mixed / args.steps,
                          "dtype": "fp32 FFT + fp32 SIMT products", "kernels": kernels_mixed},
                "kernels": kernels, "peaks": pk_kind}
        print(json.dumps(line), flush=True)
    ctx.close()
    return line


def stick_counts(c):
    import paper_2104_10502_gb300 as q
    m, _ = q.gsphere(c["lat"], c["k"], c["ecut"], c["grid"])
    n1, n2 = c["grid"][0], c["grid"][1]
    xy = set(((int(a) % n1), (int(b) % n2)) for a, b in m[:, :2])
    ax = set(x for x, _ in xy)
    return len(xy), len(ax)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as td
        torch.cuda.set_device(local_rank)
        td.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        run_gpu(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as td
            td.destroy_process_group()


if __name__ == "__main__":
    main()
