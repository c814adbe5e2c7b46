#!/usr/bin/env python3
"""Throughput of the MOFF imaging hot path on one GB300 (or N replicas).

Headline workload (the largest single-GPU configuration): a wide-field array
of 32768 antennas on a 256 x 128 wavelength lattice (1 lambda pitch, 5 %
jitter; 512 x 256 cells, so x wraps the 512 grid), full pol with per-antenna
9x9 kernels whose taps are 2x2 Jones matrices (seeded smooth beam, leakage and
a non-coplanar w-phase), 4096 channels, 512 x 512 grid, integrations of 4000
samples accumulated in FP64 across blocks.  It runs on the FP16 tensor-core
path (the factored-DFT route: FP32 gridding, both transform axes as tcgen05
contractions).  One step = one block of 128 samples of every channel =
524,288 channel-snapshots; its 34 GB of voltages are far larger than L2, so
no flush is needed between steps.

Named legs: the same array on the FP32 path; the 16384-antenna filled-aperture
precision workload (512 grid, 7x7 kernels, FP16 tensor-core and FP32); the
1024-antenna dual-pol workload with the 8-bit ADC F-stage (128 grid, FP32 and
the FP16 row-spectrum route, feedback calibration, beams, channel sets,
oversampling); serving and batching.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on a bounded sample of the headline workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MOFF channel-snapshots/s"
UNIT = "channel-snapshots/s"

# Dense workloads: (synth config, sizes, block of samples per step, integration length).
DENSE = {
    "widefield": dict(cfg="config_widefield", n_ant=32768, n_pol=2, n_chan=4096, grid_n=512, ksize=9, jones=True,
                      block=128, t_int=4000, seed=8123669 + 4,
                      name="wide-field 32768-antenna 256x128-lambda lattice (1 lambda pitch, 5% jitter), 9x9 Jones "
                           "kernels with w-phase, full pol, 4096 channels, 512x512 grid, XX/YY/XY, 4000-sample "
                           "integrations accumulated in FP64 across blocks of 128 samples (one step = one block)"),
    "precision": dict(cfg="config_precision", n_ant=16384, n_pol=2, n_chan=1024, grid_n=512, ksize=7, jones=False,
                      block=128, t_int=2000, seed=8123669 + 2,
                      name="filled aperture 16384 antennas on a 128x128-lambda lattice (5% jitter), dual pol, 7x7 "
                           "kernels, 1024 channels, 512x512 grid (zero-padded x2), 2000-sample integrations in "
                           "blocks of 128 samples"),
}
# The dual-pol F-stage workload (a named leg of the bench line).
WL = dict(n_ant=1024, n_pol=2, n_chan=1024, grid_n=128, ksize=7, ntaps=8, frames=1000)
SEED = 8123669 + 1
DUALPOL_NAME = ("dual-pol 1024-antenna hex core (1.5 lambda, 5% jitter), 8-bit ADC -> 8-tap x 2048 PFB -> 1024 "
                "channels 4+4-bit, 128x128 grid, 7x7 complex kernels, XX/YY/XY, 1000 samples per step")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="widefield", choices=sorted(DENSE),
                    help="headline dense workload (widefield is the bench line; precision gives a profiling case)")
    ap.add_argument("--block", type=int, default=0, help="samples per step (0: the workload's block)")
    ap.add_argument("--chan", type=int, default=0, help="channels (0: the workload's; fewer give a profiling case)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp32", action="store_true", help="skip the FP32 comparison on the headline workload")
    ap.add_argument("--no-precision", action="store_true", help="skip the filled-aperture precision leg")
    ap.add_argument("--no-dualpol", action="store_true", help="skip the dual-pol F-stage legs")
    ap.add_argument("--no-fp16tc", action="store_true", help="skip the dual-pol FP16 row-spectrum leg")
    ap.add_argument("--no-serving", action="store_true", help="skip the request-stream (serving) leg")
    ap.add_argument("--no-feedback", action="store_true",
                    help="skip the legs of the method's extensions (feedback calibration, beams and autocorrelation "
                         "subtraction, channel-dependent positions and kernels, edge-padded oversampling)")
    ap.add_argument("--no-plain", action="store_true", help="skip the batching leg (graph + autotune vs one channel at a time)")
    ap.add_argument("--serve-requests", type=int, default=24,
                    help="requests per load point of the serving leg (the full sweep uses 200)")
    ap.add_argument("--only", default="", choices=["", "dualpol"],
                    help="profiling case: run this leg alone and print its JSON (not a bench line)")
    ap.add_argument("--cpu-sample", default="", help=argparse.SUPPRESS)
    ap.add_argument("--frames", type=int, default=WL["frames"],
                    help="dual-pol leg: samples per step (smaller values give a profiling case, not a bench line)")
    ap.add_argument("--channels", type=int, default=WL["n_chan"],
                    help="dual-pol leg: channels (smaller values give a profiling case, not a bench line)")
    return ap.parse_args()


# ----------------------------------------------------------------------------- multi-rank helpers

def rank_info():
    """(world, rank, local_rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x, dist=None, device="cpu"):
    """The largest value of ``x`` over all ranks (the job ends when the slowest rank ends)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, seconds_max):
    """Whole-job throughput: every rank processes ``units_per_rank`` independent
    units (replicas, weak scaling), and the job takes the slowest rank's time."""
    return units_per_rank * world / seconds_max


# ----------------------------------------------------------------------------- algorithmic work

def reached_rows(pos, N, K):
    """Grid rows some kernel footprint reaches (rows no kernel reaches carry no field)."""
    import numpy as np
    h = K // 2
    ay = np.floor(np.asarray(pos)[:, 1] + 0.5).astype(int) % N
    r = np.zeros(N, bool)
    for d in range(-h, h + 1):
        r[(ay + d) % N] = True
    return int(r.sum())


def active_tiles(pos, N, K):
    """8 x 8-cell tiles some kernel footprint reaches (the tensor-core gridding writes those)."""
    import numpy as np
    h = K // 2
    anc = np.floor(np.asarray(pos) + 0.5).astype(int) % N
    t = np.zeros((N // 8, N // 8), bool)
    for dy in range(-h, h + 1):
        for dx in range(-h, h + 1):
            t[((anc[:, 1] + dy) % N) // 8, ((anc[:, 0] + dx) % N) // 8] = True
    return int(t.sum())


def dense_work(route, pos, taps, N, P, Tb):
    """Method's work per channel-snapshot of each kernel kind of a route:
    {kind: {"alu": FP32 flops, "tensor": tensor flops, "bytes": DRAM bytes}}.

    Gridding: 8 flops per nonzero kernel tap (complex multiply-add, Jones taps
    counted per (p_out, p_in)) + 6 per voltage weighting (on the tensor-core
    gridding route the taps' flops are its tensor work, the padded tile products
    it executes are not counted).  Transforms: FP32 path
    5 N log2 N per N-point transform (radix-2 count); tensor-core path the
    factored DFT's real products, 8 N (16 + N/16) per N-point transform.  Only
    reached grid rows carry a row transform.  Bytes: the 4-bit voltages, the FP16
    (8 B FP32) field between the two axes written once and read once, and the FP64
    accumulators read and written once per chunk of Tb samples."""
    import numpy as np
    A = len(pos)
    nnz = int(np.count_nonzero(np.asarray(taps)))
    R = reached_rows(pos, N, int(np.asarray(taps).shape[-1]))
    nprod = 1 if P == 1 else 4
    acc_b = 2 * nprod * N * N * 8 / max(Tb, 1)
    sq = (16 if P == 2 else 4) * N * N
    if route == "fp16_tcgrid":
        fac = 8 * N * (16 + N // 16)
        T = active_tiles(pos, N, int(np.asarray(taps).shape[-1]))
        return {"volt_prep": {"alu": 0, "tensor": 0, "bytes": A * P + A * P * 4},
                "grid_rows": {"alu": 0, "tensor": 8 * nnz, "bytes": A * P * 4 + T * 64 * P * 4},
                "row_transform": {"alu": 0, "tensor": R * P * fac, "bytes": T * 64 * P * 4 + R * P * N * 4},
                "cols_integrate": {"alu": sq, "tensor": N * P * fac, "bytes": R * P * N * 4 + acc_b}}
    if route == "fp16_dft":
        fac = 8 * N * (16 + N // 16)
        return {"grid_rows": {"alu": 8 * nnz + 6 * A * P, "tensor": R * P * fac, "bytes": A * P + R * P * N * 4},
                "cols_integrate": {"alu": sq, "tensor": N * P * fac, "bytes": R * P * N * 4 + acc_b}}
    rad = 5 * N * math.log2(N)
    return {"grid_rows": {"alu": 8 * nnz + 6 * A * P + R * P * rad, "tensor": 0, "bytes": A * P + R * P * N * 8},
            "cols_integrate": {"alu": N * P * rad + sq, "tensor": 0, "bytes": R * P * N * 8 + acc_b}}


def device_peaks(torch):
    """Measured peaks (MEASURED_PEAKS.json) and the derived FP32 FMA peak of this device."""
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    return {"hbm_gbs": float(peaks.get("hbm_gbs", 6800.0)), "hbm_basis": "of measured" if "hbm_gbs" in peaks else "of fallback",
            "bf16_tflops": float(peaks.get("bf16_tflops", 1900.0)),
            "bf16_tflops_sustained": float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1700.0))),
            "tensor_basis": "of measured" if "bf16_tflops" in peaks else "of fallback",
            "alu_tflops": sms * 128 * 2 * sm_max * 1e6 / 1e12, "sms": sms, "sm_max_mhz": sm_max}


def kernel_rooflines(kern, work, snaps, peaks):
    """Per kernel kind: achieved FP32 / tensor / HBM rates from the method's work
    and the live CUDA-event time, each against its peak (tensor: the measured
    sustained bf16 dense figure, FP16 nominally equal -- these kernels run inside
    seconds-long steps; HBM: the measured copy; FP32: derived from the unit
    counts and the maximum SM clock)."""
    out = {}
    for name, v in kern.items():
        w = work.get(name)
        if not w or not v.get("ms_total"):
            continue
        sec = v["ms_total"] / 1e3
        r = {"ms_per_launch": v["ms_total"] / max(v["launches"], 1), "launches": v["launches"]}
        cand = []
        if w["alu"]:
            a = snaps * w["alu"] / sec / 1e12
            r["alu"] = {"achieved": a, "peak": peaks["alu_tflops"], "unit": "TFLOP/s", "frac": a / peaks["alu_tflops"],
                        "basis": f"FP32 FMA {peaks['sms']} SMs x 128 x 2 flop x {peaks['sm_max_mhz']:.0f} MHz (of derived)"}
            cand.append(("alu", r["alu"]))
        if w["tensor"]:
            a = snaps * w["tensor"] / sec / 1e12
            pk = peaks["bf16_tflops_sustained"]
            r["tensor"] = {"achieved": a, "peak": pk, "unit": "TFLOP/s", "frac": a / pk,
                           "basis": f"factored-DFT real products; bf16 dense sustained ({peaks['tensor_basis']})"}
            cand.append(("tensor", r["tensor"]))
        a = snaps * w["bytes"] / sec / 1e9
        r["hbm"] = {"achieved": a, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": a / peaks["hbm_gbs"],
                    "bytes_per_snapshot": w["bytes"], "basis": f"HBM copy ({peaks['hbm_basis']})"}
        cand.append(("hbm", r["hbm"]))
        r["bound"] = max(cand, key=lambda c: c[1]["frac"])[0]
        out[name] = r
    return out


# ----------------------------------------------------------------------------- dual-pol work model

def flops_per_snapshot(kind, A=WL["n_ant"], P=WL["n_pol"], N=WL["grid_n"], K=WL["ksize"]):
    """Algorithmic FP32 flops per channel-snapshot of each kernel (5 N log2 N per
    N-point transform, 8 per complex multiply-add, 6 per complex multiply)."""
    fft_axis = P * N * 5 * N * math.log2(N)
    if kind == 1:      # calibrate + grid + row transforms
        return 6 * A * P + 8 * A * P * K * K + fft_axis
    if kind == 2:      # column transforms + square-and-integrate
        return fft_axis + (16 if P == 2 else 4) * N * N
    raise ValueError(kind)


def tc_row_flops_per_snapshot(pos, N=WL["grid_n"], P=WL["n_pol"], K=WL["ksize"]):
    """Tensor-core flops per channel-snapshot of the row contraction as executed:
    per (pol, grid row, kx tile of KX = min(N, 128)) 2 x (2 KX output columns:
    real and imaginary parts) x the contraction length (64 per chunk of 32 voltages,
    padding included)."""
    import numpy as np
    KX = min(N, 128)
    h = K // 2
    ay = np.floor(np.asarray(pos)[:, 1] + 0.5).astype(int) % N
    cnt = np.bincount(ay, minlength=N)          # antennas per anchor row
    kp = np.zeros(N)
    for ry in range(N):
        # the antennas anchored in the cyclic window [ry - h, ry + h]: one run, two where it wraps;
        # each run is cut into chunks of 32 voltages, 64 contraction rows (real, imaginary) each
        if ry - h < 0:
            runs = [cnt[: ry + h + 1].sum(), cnt[N + ry - h:].sum()]
        elif ry + h >= N:
            runs = [cnt[ry - h:].sum(), cnt[: ry + h - N + 1].sum()]
        else:
            runs = [cnt[ry - h: ry + h + 1].sum()]
        kp[ry] = sum(64 * ((n + 31) // 32) for n in runs)
    return P * (N // KX) * float(np.sum(2 * (2 * KX) * kp))


def tc_row_bytes_per_snapshot(pos, N=WL["grid_n"], P=WL["n_pol"], K=WL["ksize"]):
    """DRAM bytes per channel-snapshot the row contraction must move: the FP16
    row-transformed field (half2 per kx) of every grid row some kernel row reaches
    (rows no kernel row reaches are not written), and the weighted voltages read
    once as FP16 real and imaginary planes."""
    import numpy as np
    h = K // 2
    ay = np.floor(np.asarray(pos)[:, 1] + 0.5).astype(int) % N
    reached = np.zeros(N, bool)
    for d in range(-h, h + 1):
        reached[(ay + d) % N] = True
    return P * int(reached.sum()) * N * 4 + len(pos) * P * 2 * 2


def pfb_flops_per_stream_frame(C=WL["n_chan"], ntaps=WL["ntaps"]):
    M = 2 * C
    return 2 * ntaps * M + 5 * C * math.log2(C) + 10 * C


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); smax.append(float(f[2])); power.append(float(f[3]))
            except ValueError:
                continue
            for name, v in zip(self.NAMES, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- oracle (CPU) samples

def cpu_model():
    """The host CPU's model name (lscpu, else the platform string)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.TimeoutExpired):
        pass
    return platform.processor() or platform.machine()


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_setup(wl_name, n_chan, n_time, seed):
    """Inputs of a bounded oracle sample of a dense workload: the gridding matrix
    (the plan's set-up, untimed), gains of ``n_chan`` channels and 4-bit noise
    voltages (sigma 2 per component) of ``n_chan`` channels x ``n_time`` samples."""
    import numpy as np

    import oracle
    import synth
    wl = DENSE[wl_name]
    cfg = getattr(synth, wl["cfg"])(n_chan=n_chan)
    rng = np.random.default_rng(seed)
    shape = (n_time, n_chan, wl["n_ant"], wl["n_pol"])
    re = np.clip(np.rint(2 * rng.standard_normal(size=shape, dtype=np.float32)), -7, 7).astype(np.int8)
    im = np.clip(np.rint(2 * rng.standard_normal(size=shape, dtype=np.float32)), -7, 7).astype(np.int8)
    W = oracle.grid_matrix(cfg["pos"], cfg["taps"], wl["grid_n"], wl["n_pol"], jones=wl["jones"])
    return W, synth.pack_4bit(re, im), cfg["gains"]


def oracle_channels(W, codes, gains, N, P):
    """Eq. m6 for every channel of a sample, in the oracle's steps (decode, weight,
    grid, transform, square and sum); returns the channel-snapshots imaged."""
    import oracle
    for c in range(codes.shape[1]):
        y = oracle.calibrate(oracle.unpack_4bit(codes[:, c]), gains[c])
        oracle.integrate(oracle.sky_transform(oracle.grid(y, W, N, P)))
    return codes.shape[0] * codes.shape[1]


_POOL_W = None


def _pool_init(W):
    global _POOL_W
    _POOL_W = W


def _pool_task(item):
    codes, gains, N, P = item
    return oracle_channels(_POOL_W, codes, gains, N, P)


def run_cpu_sample(wl_name):
    """One-core and all-core oracle rates on a bounded sample of the workload (run in
    a process without a GPU; the all-core leg is a spawn pool, one channel per core)."""
    import multiprocessing as mp
    wl = DENSE[wl_name]
    N, P = wl["grid_n"], wl["n_pol"]
    cores = host_cores()
    T1, C1, Tm = 64, 8, 256                  # about 10 s of one core, and of every core
    W, codes, gains = oracle_setup(wl_name, max(C1, cores), max(T1, Tm), 8123669 + 77)
    oracle_channels(W, codes[:2, :1], gains[:1], N, P)                # warm
    t0 = time.perf_counter()
    n1 = oracle_channels(W, codes[:T1, :C1], gains[:C1], N, P)
    dt1 = time.perf_counter() - t0
    ctx = mp.get_context("spawn")
    items = [(codes[:Tm, c:c + 1].copy(), gains[c:c + 1], N, P) for c in range(cores)]
    with ctx.Pool(cores, initializer=_pool_init, initargs=(W,)) as pool:
        pool.map(_pool_task, [(it[0][:2], it[1], N, P) for it in items])   # start-up and warm-up
        t0 = time.perf_counter()
        nm = sum(pool.map(_pool_task, items))
        dtm = time.perf_counter() - t0
    print(json.dumps({
        "value": n1 / dt1, "unit": UNIT, "cores": 1, "kind": "oracle", "seconds": dt1,
        "sample": f"{C1} channels x {T1} samples of the {wl_name} workload ({n1} channel-snapshots), "
                  "FP64 numpy/scipy, gridding matrix built beforehand (plan set-up), 1 thread",
        "all_core": {"value": nm / dtm, "unit": UNIT, "cores": cores, "seconds": dtm,
                     "sample": f"{cores} channels x {Tm} samples ({nm} channel-snapshots), one channel per "
                               "single-threaded process"},
        "nproc": cores, "cpu_model": cpu_model(), "machine": platform.machine()}), flush=True)


def cpu_baseline_subprocess(wl_name):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample", wl_name], env=env,
                       capture_output=True, text=True, timeout=1200)
    for line in r.stdout.splitlines()[::-1]:
        if line.startswith("{"):
            return json.loads(line)
    return {"error": (r.stderr or r.stdout)[-300:]}


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands on the host cores, on the
    headline workload, each step a bounded sample (one channel x 8 samples)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    wl = DENSE[args.workload]
    N, P = wl["grid_n"], wl["n_pol"]
    T = 8
    W, codes, gains = oracle_setup(args.workload, 1, T, 8123669 + 78)
    for _ in range(args.warmup):
        oracle_channels(W, codes[:2], gains, N, P)
    units, secs = 0, 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        units += oracle_channels(W, codes, gains, N, P)
        secs += time.perf_counter() - t0
    v = units / secs
    sample = f"each step: 1 channel x {T} samples of the {args.workload} workload, gridding matrix built beforehand"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["name"], "sample_snapshots_per_step": T, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                         "cpu_model": cpu_model(), "nproc": host_cores()},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ----------------------------------------------------------------------------- GPU arm

def source_sha1(src):
    """SHA-1 of a kernel's source: each entry is a file, (file, end) for the part
    of the file before the first occurrence of `end` (the kernel and what precedes
    it, not the kernels after it), or (file, start, end) for the part from the
    first occurrence of `start` up to the next `end` (the kernel and its own
    helpers only)."""
    h = hashlib.sha1()
    for f in src:
        path, start, end = (f, None, None) if isinstance(f, str) else ((f[0], None, f[1]) if len(f) == 2 else f)
        text = open(os.path.join(ROOT, path), "rb").read()
        if start is not None:
            i = text.find(start.encode())
            text = text[i:] if i >= 0 else text
        if end is not None:
            cut = text.find(end.encode())
            text = text[:cut] if cut >= 0 else text
        h.update(text)
    return h.hexdigest()


# The source each traffic figure depends on (see profiles/traffic.json).
KERNEL_SOURCES = {
    "grid_rows": [("paper_0812_3669_gb300/csrc/moff_image_kernels.cuh", "struct ColShape"),
                  "paper_0812_3669_gb300/csrc/moff_fft.cuh"],
    "cols_integrate": [("paper_0812_3669_gb300/csrc/moff_image_kernels.cuh", "template <int N>\nstruct ColShape",
                        "size_t col_smem_bytes_t"),
                       "paper_0812_3669_gb300/csrc/moff_fft.cuh"],
    "pfb_fstage": ["paper_0812_3669_gb300/csrc/moff_fstage.cu", "paper_0812_3669_gb300/csrc/moff_fft.cuh"],
    # the factored-DFT tensor-core route of the dense workloads
    "grid_rows_dft": [("paper_0812_3669_gb300/csrc/moff_image_kernels.cuh", "struct ColShape"),
                      "paper_0812_3669_gb300/csrc/moff_dft.cuh"],
    "cols_dft": [("paper_0812_3669_gb300/csrc/moff_dft_kernels.cu", "struct ColDftShape",
                  "template <int N, int P>\nstruct RowDftShape"), "paper_0812_3669_gb300/csrc/moff_dft.cuh"],
    "rows_dft": [("paper_0812_3669_gb300/csrc/moff_dft_kernels.cu", "template <int N, int P>\nstruct RowDftShape",
                  "template <int N, int P>\ncudaError_t launch_rows_dft_t"), "paper_0812_3669_gb300/csrc/moff_dft.cuh"],
    "rows_dft8": [("paper_0812_3669_gb300/csrc/moff_dft_kernels.cu", "template <int P>\nstruct RowDft8Shape",
                   "}  // namespace"), "paper_0812_3669_gb300/csrc/moff_dft.cuh"],
    "grid_tc": ["paper_0812_3669_gb300/csrc/moff_gridtc.cu", "paper_0812_3669_gb300/csrc/moff_tc.cuh"],
    "volt_prep": ["paper_0812_3669_gb300/csrc/moff_tc_kernels.cu"],
}
# kernel kind (moff_timing) -> its name in KERNEL_SOURCES, per route
ROUTE_KERNELS = {"fp16_dft": {"grid_rows": "grid_rows_dft", "cols_integrate": "cols_dft"},
                 "fp16_tcgrid": {"grid_rows": "grid_tc", "row_transform": "rows_dft", "cols_integrate": "cols_dft",
                                 "volt_prep": "volt_prep"}}


def route_kernel(route, kind, N):
    """Name (in KERNEL_SOURCES) of the kernel behind a timing kind on a route: the tensor-core
    gridding route's row transform is the 8 x 64 kernel on the 512 grid (unless MOFF_ROWS8=0)."""
    k = ROUTE_KERNELS.get(route, {}).get(kind, kind)
    if k == "rows_dft" and N == 512 and os.environ.get("MOFF_ROWS8", "1") != "0":
        return "rows_dft8"
    return k


def traffic_for(kernel_key, src, units_per_launch=None):
    """Per-launch DRAM bytes from the committed ncu summary, if the kernel's
    source is unchanged since the capture (else None).  A record captured on a
    smaller launch holds bytes per unit (channel-snapshot) and is scaled to
    this launch's units; that holds where every byte the kernel moves grows
    with the units it processes."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path)).get(kernel_key)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("source_sha1") != source_sha1(src):
        return None
    if "bytes_per_unit" in rec:
        return rec["bytes_per_unit"] * units_per_launch if units_per_launch else None
    return rec.get("bytes_per_launch")


SERVE_LOADS = (0.3, 0.5, 0.7, 0.85)


def serving_leg(args, moff, synth, torch, fp16tc=False, images=None):
    """Request stream over sub-arrays of uneven size (MOFF_SERVED plans, one
    moff_server): first a closed burst to find the saturation rate, then Poisson
    arrivals at fractions of it.  Reports p50/p99 block latency and throughput
    per load point.  With fp16tc, each sub-array takes the FP16 tensor-core path
    where its density allows (the row-spectrum contraction for sparse rows, the
    tensor-core gridding and factored DFT for dense arrays on 256 and 512 grids)
    and FP32 otherwise.  Both streams draw the same request order, so every plan
    ends with the same blocks summed; with ``images`` (a list) each plan's image
    divided by its sample count is appended, on the device."""
    import numpy as np
    mix = synth.config_serving()
    plans, blocks, prec = [], [], []
    for i, a in enumerate(mix):
        pl = None
        if fp16tc:
            try:
                pl = moff.Plan(a["pos"], a["taps"], a["N"], a["C"], 2, served=True, fp16tc=True)
                prec.append(pl.route())
            except moff.MoffError:
                pl = None
        if pl is None:
            pl = moff.Plan(a["pos"], a["taps"], a["N"], a["C"], 2, served=True)
            prec.append("fp32")
        pl.set_gains(synth.device_gains(SEED + 600 + i, a["C"], a["A"], 2))
        plans.append(pl)
        blocks.append(synth.device_codes(SEED + 500 + i, a["T"], a["C"], a["A"], 2))
    torch.cuda.synchronize()
    units = [a["C"] * a["T"] for a in mix]
    rng = np.random.default_rng(SEED + 77)
    nreq = args.serve_requests
    pool, slots = 32 << 30, 4
    srv = moff.Server(pool, slots)
    try:
        for i in range(len(plans)):                       # warm every plan once
            srv.submit(plans[i], blocks[i])
        srv.wait(0, 1800000)
        srv.stats(reset=True)
        # saturation: everything at once
        order = rng.integers(0, len(plans), size=nreq)
        t0 = time.perf_counter()
        for i in order:
            srv.submit(plans[i], blocks[i])
        srv.wait(0, 1800000)
        wall = time.perf_counter() - t0
        sat = srv.stats(reset=True)
        sat_req_s = len(order) / wall
        points = []
        for load in SERVE_LOADS:
            rate = load * sat_req_s
            order = rng.integers(0, len(plans), size=nreq)
            gaps = rng.exponential(1.0 / rate, size=len(order))
            t0 = time.perf_counter()
            due = t0
            for i, g in zip(order, gaps):
                due += g
                while True:
                    now = time.perf_counter()
                    if now >= due:
                        break
                    time.sleep(min(due - now, 0.002))
                srv.submit(plans[i], blocks[i])
            srv.wait(0, 1800000)
            wall = time.perf_counter() - t0
            st = srv.stats(reset=True)
            points.append({"load": load, "offered_req_per_s": rate, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
                           "throughput": st["throughput"], "requests": st["completed"], "wall_s": wall})
        if images is not None:
            for pl in plans:
                img = torch.empty((pl.C, pl.n_prod, pl.N, pl.N), dtype=torch.float32, device="cuda")
                _, n = pl.read_image(out=img)
                images.append(img.div_(float(n)))
    finally:
        srv.close()
        for pl in plans:
            pl.close()
        del blocks
        torch.cuda.empty_cache()
    return {
        "unit": UNIT, "precision": "FP16 tensor-core route where the array allows, else fp32" if fp16tc else "fp32",
        "slots": slots, "pool_bytes": pool, "requests_per_point": nreq,
        "mix": [{"antennas": a["A"], "grid_n": a["N"], "channels": a["C"], "samples": a["T"], "route": p}
                for a, p in zip(mix, prec)],
        "saturation": {"req_per_s": sat_req_s, "throughput": sat["throughput"], "p50_ms": sat["p50_ms"],
                       "p99_ms": sat["p99_ms"], "requests": sat["completed"]},
        "points": points, "mean_units_per_request": float(np.mean(units)),
    }


def batching_leg(args, moff, synth, torch):
    """All channels and pols of a block in one graph launch (MOFF_GRAPH) with
    the autotuned gridding shape (MOFF_AUTOTUNE), against the plain FP32 form:
    the same kernels run one channel per launch pair (field scratch sized for a
    single channel).  Bench array, 64 channels x 1000 samples of device codes
    (no F-stage), FP32 throughout."""
    A, P, N = WL["n_ant"], WL["n_pol"], WL["grid_n"]
    Cs, F = 64, args.frames
    cfg = synth.config_dualpol(n_chan=Cs)
    codes = synth.device_codes(SEED + 900, F, Cs, A, P)

    def timed(pl, reps=3):
        pl.set_gains(cfg["gains"])
        pl.submit(codes)
        pl.sync()
        pl.reset()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(reps):
            pl.submit(codes)
        ev1.record()
        torch.cuda.synchronize()
        return reps * Cs * F / (ev0.elapsed_time(ev1) / 1e3)

    per = P * N * N * 8
    old = os.environ.get("MOFF_SCRATCH_MB")
    os.environ["MOFF_SCRATCH_MB"] = str(32 * per / 1048576.0)
    try:
        plain = moff.Plan(cfg["pos"], cfg["taps"], N, Cs, P)
    finally:
        if old is None:
            os.environ.pop("MOFF_SCRATCH_MB", None)
        else:
            os.environ["MOFF_SCRATCH_MB"] = old
    pinfo = plain.info()
    v_plain = timed(plain, reps=1)
    plain.close()
    direct = moff.Plan(cfg["pos"], cfg["taps"], N, Cs, P)
    v_direct = timed(direct)
    rule = direct.tuning()
    direct.close()
    t0 = time.perf_counter()
    batched = moff.Plan(cfg["pos"], cfg["taps"], N, Cs, P, autotune=True, graph=True)
    tune_s = time.perf_counter() - t0
    v_batched = timed(batched)
    binfo, tuned = batched.info(), batched.tuning()
    img_b = torch.empty((Cs, 4, N, N), dtype=torch.float32, device="cuda")
    batched.read_image(out=img_b, reset=True)
    batched.close()
    # every chunk of the block in one persistent launch (work queue, bounded dependency waits),
    # autotuned among the shapes it is built for, replayed as a graph
    t0 = time.perf_counter()
    pers = moff.Plan(cfg["pos"], cfg["taps"], N, Cs, P, autotune=True, graph=True, persist=True)
    ptune_s = time.perf_counter() - t0
    v_pers = timed(pers)
    pinfo2, ptuned = pers.info(), pers.tuning()
    img_p = torch.empty((Cs, 4, N, N), dtype=torch.float32, device="cuda")
    pers.read_image(out=img_p, reset=True)
    pers.close()
    pdiff = image_diff(torch, img_p, img_b)
    del img_b, img_p
    return {"unit": UNIT, "channels": Cs, "samples": F, "dtype": "f32",
            "persistent_graph": {"value": v_pers, "time_batch": ptuned["time_batch"],
                                 "cells_per_lane": ptuned["cells_per_lane"], "wide_rows": ptuned["wide_rows"],
                                 "tune_source": ptuned["source"], "plan_create_s": ptune_s,
                                 "chan_chunk": pinfo2["chan_chunk"], "time_chunk": pinfo2["time_chunk"],
                                 "launches_per_block": 1, "max_norm_diff_vs_batched_direct": pdiff},
            "plain_one_channel": {"value": v_plain, "chan_chunk": pinfo["chan_chunk"],
                                  "time_chunk": pinfo["time_chunk"]},
            "batched_rule_direct": {"value": v_direct, "time_batch": rule["time_batch"], "staged": rule["staged"],
                                    "cells_per_lane": rule["cells_per_lane"]},
            "batched_autotuned_graph": {"value": v_batched, "time_batch": tuned["time_batch"], "staged": tuned["staged"],
                                        "cells_per_lane": tuned["cells_per_lane"], "wide_rows": tuned["wide_rows"],
                                        "tune_source": tuned["source"], "plan_create_s": tune_s,
                                        "chan_chunk": binfo["chan_chunk"], "time_chunk": binfo["time_chunk"],
                                        "graph_launches_per_block": 1},
            "speedup_vs_plain": v_batched / v_plain}


def dualpol_leg(args, ctx):
    """The 1024-antenna dual-pol workload with the F-stage: 8-bit ADC streams in,
    FP32 imaging (autotuned gridding), and on the same input the FP16 row-spectrum
    route, feedback calibration, beams + autocorrelation subtraction, channel-
    dependent positions and kernels, edge-padded oversampling, and end to end
    through pinned host ADC buffers.  One step = one 1000-sample integration."""
    moff, synth, torch, np = ctx.moff, ctx.synth, ctx.torch, ctx.np
    world, rank, local, dist = ctx.world, ctx.rank, ctx.local, ctx.dist

    def barrier():
        ctx.barrier()

    A, P, C, N, K, ntaps, F = (WL["n_ant"], WL["n_pol"], args.channels, WL["grid_n"], WL["ksize"], WL["ntaps"],
                               args.frames)
    M = 2 * C
    S = (F + ntaps - 1) * M
    cfg = synth.config_dualpol(n_chan=C)
    pos, taps, gains = cfg["pos"], cfg["taps"], cfg["gains"]
    adc = synth.device_adc(SEED + 1000 * rank, pos, P, S, M, N,
                           sources=tuple((kx, ky, ch * C // WL["n_chan"], amp)
                                         for (kx, ky, ch, amp) in ((40, 70, 100, 12.0), (90, 30, 600, 8.0),
                                                                   (64, 64, 900, 6.0))))

    def make_plan(fp16tc):
        pl = moff.Plan(pos, taps, N, C, P, fstage=True, fp16tc=fp16tc, autotune=not fp16tc)
        pl.set_gains(gains)
        # requantisation gain from a short calibration block: noise sigma ~ 2 codes per component
        calib = adc[:, :, : (ntaps + 3) * M].contiguous()
        pl.set_fstage(ntaps, None, 1.0)
        spec = pl.channelise(calib, kind=1)
        pl.set_fstage(ntaps, None, float(2.0 / np.std(np.concatenate([spec.real.ravel(), spec.imag.ravel()]))))
        return pl

    gpu_idx = local
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis and vis.split(",")[local].strip().isdigit():
        gpu_idx = int(vis.split(",")[local])

    def measure(pl, steps, warmup, sample_clocks=False):
        """Time `steps` integrations (CUDA events on the plan stream), max over ranks."""
        stream = torch.cuda.current_stream()
        for _ in range(warmup):
            pl.submit_adc(adc)
        pl.sync()
        pl.reset()
        pl.set_timing(True)
        clocks = ClockSampler(gpu_idx) if sample_clocks else None
        barrier()
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            pl.submit_adc(adc)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
        clk = clocks.stop() if clocks else None
        ms = max_over_ranks(ev0.elapsed_time(ev1), dist, "cuda")
        kern = {}
        for kind, name in moff.KERNEL_KINDS.items():
            tot, n = pl.timing(kind)
            if n:
                kern[name] = {"ms_total": tot, "launches": n}
        pl.set_timing(False)
        img, nsamp = pl.read_image(reset=True)
        assert nsamp == steps * F and np.isfinite(img).all()
        return ms, kern, clk, img

    plan = make_plan(False)
    ms_max, kern, clk, img32 = measure(plan, args.steps, args.warmup, sample_clocks=True)
    value = job_rate(args.steps * F * C, world, ms_max / 1000.0)
    snaps = args.steps * F * C
    total_kernel_ms = sum(v["ms_total"] for v in kern.values())
    flops = {
        "grid_rows": snaps * flops_per_snapshot(1),
        "cols_integrate": snaps * flops_per_snapshot(2),
        "pfb_fstage": args.steps * F * A * P * pfb_flops_per_stream_frame(),
    }
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    sm_max = ctx.peaks["sm_max_mhz"]
    alu_peak = ctx.peaks["alu_tflops"]                       # FP32 FMA TFLOP/s at max SM clock
    for name, v in kern.items():
        v["share"] = v["ms_total"] / total_kernel_ms if total_kernel_ms else None
        v["tflops"] = flops[name] / (v["ms_total"] / 1e3) / 1e12 if v["ms_total"] and name in flops else None
    dom = max(kern, key=lambda k: kern[k]["ms_total"])
    src = KERNEL_SOURCES.get(dom, [])
    launches = kern[dom]["launches"]
    achieved = kern[dom]["tflops"]
    roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": achieved / alu_peak if achieved else None,
                "peak_basis": f"FP32 FMA: {ctx.peaks['sms']} SMs x 128 lanes x 2 flop x {sm_max:.0f} MHz (of derived peak)",
                "flops_per_launch": flops[dom] / max(launches, 1),
                "ms_per_launch": kern[dom]["ms_total"] / max(launches, 1),
                "traffic": traffic_for(dom + "@dualpol1024", src, snaps / max(launches, 1))}
    gpu_launches = sum(v["launches"] for v in kern.values())
    # DRAM traffic against the method's own bytes: the gridding kernel's algorithmic input is
    # the 4-bit voltages (the row-transformed field it writes is an intermediate); the column
    # kernel's is its share of the FP64 accumulators (read and written once per chunk)
    # (every launch reads and writes the FP64 accumulators of its chunk's channels once)
    snaps_launch = snaps / max(launches, 1)
    alg = {"grid_rows": A * P * snaps_launch,
           "cols_integrate": 2 * 4 * N * N * 8 * plan.info()["chan_chunk"]}
    for name in ("grid_rows", "cols_integrate"):
        if name in kern:
            t = traffic_for(name + "@dualpol1024", KERNEL_SOURCES.get(name, []),
                            snaps / max(kern[name]["launches"], 1))
            kern[name]["algorithmic_bytes_per_launch"] = alg[name]
            kern[name]["traffic_bytes_per_launch"] = t
            kern[name]["traffic_over_algorithmic"] = t / alg[name] if t else None

    # ---------------------------------------------------------------- FP16 tensor-core variant, same input
    fp16 = None
    if not args.no_fp16tc:
        plan16 = make_plan(True)
        ms16, kern16, _, img16 = measure(plan16, args.steps, max(1, args.warmup))
        plan16.close()
        tc_flops = snaps * tc_row_flops_per_snapshot(pos)
        den = np.maximum(np.abs(img32).reshape(C, 4, -1).max(-1), 1e-30)
        den[:, 2:] = np.maximum(den[:, :1], den[:, 1:2])
        diff = np.abs(img16 - img32).reshape(C, 4, -1).max(-1) / den
        rk = kern16.get("grid_rows", {})
        fp16 = {"value": job_rate(args.steps * F * C, world, ms16 / 1000.0), "unit": UNIT,
                "ms_per_step": ms16 / args.steps, "kernels": kern16,
                "max_norm_diff_vs_fp32": float(diff.max()),
                "row_contraction_tensor": {"bound": "tensor", "achieved": tc_flops / (rk["ms_total"] / 1e3) / 1e12
                                           if rk.get("ms_total") else None,
                                           "peak": float(peaks.get("bf16_tflops", 1933.3)), "unit": "TFLOP/s",
                                           "peak_basis": "measured bf16 dense burst (fp16 nominal equal) (of measured)"}}
        r = fp16["row_contraction_tensor"]
        r["frac"] = r["achieved"] / r["peak"] if r["achieved"] else None
        tc_bytes = snaps * tc_row_bytes_per_snapshot(pos)
        fp16["row_contraction_hbm"] = {"bound": "hbm", "achieved": tc_bytes / (rk["ms_total"] / 1e3) / 1e9
                                       if rk.get("ms_total") else None,
                                       "peak": float(peaks.get("hbm_gbs", 6779.0)), "unit": "GB/s",
                                       "bytes_per_snapshot": tc_row_bytes_per_snapshot(pos),
                                       "peak_basis": "measured HBM copy (of measured)"}
        r = fp16["row_contraction_hbm"]
        r["frac"] = r["achieved"] / r["peak"] if r["achieved"] else None
        # the same contraction against the method's own work: gridding (8 flops per tap) and the
        # row transform (5 N log2 N per row), not the padded product the tensor cores execute
        meth = snaps * (flops_per_snapshot(1) - 6 * A * P)
        fp16["row_contraction_method"] = {"bound": "tensor", "achieved": meth / (rk["ms_total"] / 1e3) / 1e12
                                          if rk.get("ms_total") else None,
                                          "peak": float(peaks.get("bf16_tflops", 1933.3)), "unit": "TFLOP/s",
                                          "flops_per_snapshot": flops_per_snapshot(1) - 6 * A * P,
                                          "peak_basis": "method's flops (gridding + row FFT) over the measured bf16 "
                                                        "dense burst (of measured)"}
        r = fp16["row_contraction_method"]
        r["frac"] = r["achieved"] / r["peak"] if r["achieved"] else None

    # ---------------------------------------------------------------- feedback calibration leg (Sec. 6)
    feedback = None
    if not args.no_feedback:
        planfb = make_plan(False)
        planfb.set_calibrator(40, 70)            # the first injected source's pixel
        msfb, kernfb, _, _ = measure(planfb, max(1, args.steps // 2), 1)
        R, S, nfb = planfb.read_feedback()
        planfb.close()
        fk = kernfb.get("feedback_corr", {})
        fb_bytes = (args.steps // 2 or 1) * F * C * A * P          # codes re-read per step (pixel taps are tiny)
        feedback = {"value": job_rate(max(1, args.steps // 2) * F * C, world, msfb / 1000.0), "unit": UNIT,
                    "ms_per_step": msfb / max(1, args.steps // 2), "kernels": kernfb, "calibrator_pixel": [40, 70],
                    "samples_summed": nfb,
                    "corr_kernel_roofline": {"bound": "hbm", "achieved": fb_bytes / (fk["ms_total"] / 1e3) / 1e9
                                             if fk.get("ms_total") else None,
                                             "peak": float(peaks.get("hbm_gbs", 6779.0)), "unit": "GB/s",
                                             "peak_basis": "measured HBM copy (of measured)"}}
        r = feedback["corr_kernel_roofline"]
        r["frac"] = r["achieved"] / r["peak"] if r["achieved"] else None

    # ---------------------------------------------------------------- beams + autocorrelation subtraction leg
    taps_leg = None
    if not args.no_feedback:
        planb = make_plan(False)
        bk = [(40, 70), (90, 30), (64, 64), (10, 10)] * 4                  # 16 tied-array beam pixels
        planb.set_beams([b[0] for b in bk], [b[1] for b in bk])
        planb.set_autocorr(True)
        nst = max(1, args.steps // 2)
        msb, kernb, _, _ = measure(planb, nst, 1)
        planb.set_autocorr(True)                                            # measure() reset the image; restart the sums
        planb.submit_adc(adc)
        t0 = time.perf_counter()
        _, nb_ = planb.read_image_cross()
        cross_ms = 1000 * (time.perf_counter() - t0)
        beams = planb.read_beams()
        planb.close()
        ak = kernb.get("autocorr", {})
        a_bytes = nst * F * C * A * P
        taps_leg = {"value": job_rate(nst * F * C, world, msb / 1000.0), "unit": UNIT, "ms_per_step": msb / nst,
                    "beams": len(bk), "beam_block_shape": list(beams.shape), "kernels": kernb,
                    "read_image_cross_ms": cross_ms,
                    "autocorr_kernel_roofline": {"bound": "hbm", "achieved": a_bytes / (ak["ms_total"] / 1e3) / 1e9
                                                 if ak.get("ms_total") else None,
                                                 "peak": float(peaks.get("hbm_gbs", 6779.0)), "unit": "GB/s",
                                                 "peak_basis": "measured HBM copy (of measured)"}}
        r = taps_leg["autocorr_kernel_roofline"]
        r["frac"] = r["achieved"] / r["peak"] if r["achieved"] else None

    # ---------------------------------------------------------------- channel-dependent positions/kernels leg
    # Positions in wavelengths scale with frequency: 32 sets across the band (0.9 to 1.1 of the
    # reference positions about the grid centre), kernels re-evaluated at each set's subpixel
    # offsets; channel c takes set 32 c / C.  Then the same array edge-padded onto a 2N grid.
    sets_leg = None
    if not args.no_feedback:
        G = 32
        scales = 0.9 + 0.2 * np.arange(G) / (G - 1)
        cen = N / 2.0
        pos_sets = np.stack([cen + (pos - cen) * sc for sc in scales])
        taps_sets = np.stack([synth.taps_gaussian(np.random.default_rng(synth.SEED_BASE + 50), ps, WL["ksize"], 1.2,
                                                  n_pol=P, subpixel=True, phase_slope=0.3) for ps in pos_sets])
        grp = (np.arange(C) * G) // C
        plans = make_plan(False)
        t0 = time.perf_counter()
        plans.set_channel_groups(pos_sets, taps_sets, grp)
        bin_s = time.perf_counter() - t0
        nst = max(1, args.steps // 2)
        mss, kerns, _, _ = measure(plans, nst, 1)
        tun = plans.tuning()
        plans.close()
        gk = kerns.get("grid_rows", {})
        g_flops = nst * F * C * flops_per_snapshot(1)
        sets_leg = {"value": job_rate(nst * F * C, world, mss / 1000.0), "unit": UNIT, "ms_per_step": mss / nst,
                    "sets": G, "scale_range": [0.9, 1.1], "binning_s": bin_s, "kernels": kerns,
                    "grid_shape": {"time_batch": tun["time_batch"], "cells_per_lane": tun["cells_per_lane"],
                                   "wide_rows": tun["wide_rows"]},
                    "grid_kernel_roofline": {"bound": "alu",
                                             "achieved": g_flops / (gk["ms_total"] / 1e3) / 1e12
                                             if gk.get("ms_total") else None,
                                             "peak": alu_peak, "unit": "TFLOP/s",
                                             "peak_basis": f"FP32 FMA: {ctx.peaks['sms']} SMs x 128 lanes x 2 flop x {sm_max:.0f} MHz "
                                                           "(of derived peak)"}}
        r = sets_leg["grid_kernel_roofline"]
        r["frac"] = r["achieved"] / r["peak"] if r["achieved"] else None
        # image oversampling by edge padding: the array centred on a 2N grid
        plo = moff.Plan(pos + N / 2.0, taps, 2 * N, C, P, fstage=True, autotune=True)
        plo.set_gains(gains)
        calib = adc[:, :, : (ntaps + 3) * M].contiguous()
        plo.set_fstage(ntaps, None, 1.0)
        spec = plo.channelise(calib, kind=1)
        plo.set_fstage(ntaps, None, float(2.0 / np.std(np.concatenate([spec.real.ravel(), spec.imag.ravel()]))))
        mso, kerno, _, _ = measure(plo, 1, 1)
        plo.close()
        sets_leg["oversampled_2x"] = {"grid_n": 2 * N, "value": job_rate(F * C, world, mso / 1000.0), "unit": UNIT,
                                      "ms_per_step": mso, "kernels": kerno}

    # ---------------------------------------------------------------- end to end through host buffers
    e2e = None
    if not args.no_e2e and args.e2e_steps > 0:
        adc_h = torch.empty(adc.shape, dtype=torch.int8, pin_memory=True)
        adc_h.copy_(adc)
        del adc
        torch.cuda.empty_cache()
        out_h = torch.empty((C, 4, N, N), dtype=torch.float32, pin_memory=True)
        for _ in range(2):                     # warm both staging buffers
            plan.submit_adc(adc_h)
            plan.read_image(out=out_h, reset=True)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            plan.submit_adc(adc_h)
            plan.read_image(out=out_h, reset=True)
        dt = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
        e2e = {"value": job_rate(args.e2e_steps * F * C, world, dt), "unit": UNIT,
               "h2d_bytes_per_step": int(adc_h.numel()), "d2h_bytes_per_step": int(out_h.numel() * 4),
               "steps": args.e2e_steps, "api": "moff_submit_adc(host pinned ADC) + moff_read_image(host)"}
    plan.close()

    fx_eq = value * A * (A - 1) / 2 * 4
    return {"workload": DUALPOL_NAME, "value": value, "unit": UNIT, "ms_per_step": ms_max / args.steps,
            "steps": args.steps, "dtype": "f32", "fx_equiv_tcmac_per_s": fx_eq / 1e12,
            "config": {"antennas": A, "pols": P, "channels": C, "grid_n": N, "kernel": K, "pfb_taps": ntaps,
                       "samples_per_step": F, "channel_snapshots_per_step": F * C},
            "roofline": roofline, "kernels": kern, "gpu_launches": gpu_launches, "clocks": clk, "e2e": e2e,
            "fp16tc_rowspec": fp16, "feedback": feedback, "beams_autocorr": taps_leg, "channel_sets": sets_leg}


# ----------------------------------------------------------------------------- dense workloads

class Ctx:
    """What every leg needs: the modules, the rank layout and the device's peaks."""

    def __init__(self, moff, synth, torch, np, world, rank, local, dist, peaks, gpu_idx):
        self.moff, self.synth, self.torch, self.np = moff, synth, torch, np
        self.world, self.rank, self.local, self.dist = world, rank, local, dist
        self.peaks, self.gpu_idx = peaks, gpu_idx

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()


def measure_blocks(ctx, pl, codes, steps, warmup, sample_clocks=False):
    """Submit ``steps`` blocks of device voltages (after ``warmup`` untimed ones),
    timed with CUDA events on the plan's stream, max over ranks.  Returns
    (ms, per-kernel device times, clock record)."""
    torch, moff = ctx.torch, ctx.moff
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        pl.submit(codes)
    pl.sync()
    pl.reset()
    pl.set_timing(True)
    clocks = ClockSampler(ctx.gpu_idx) if sample_clocks else None
    ctx.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        pl.submit(codes)
    ev1.record(stream)
    torch.cuda.synchronize()
    ctx.barrier()
    clk = clocks.stop() if clocks else None
    ms = max_over_ranks(ev0.elapsed_time(ev1), ctx.dist, "cuda")
    kern = {}
    for kind, name in moff.KERNEL_KINDS.items():
        tot, n = pl.timing(kind)
        if n:
            kern[name] = {"ms_total": tot, "launches": n}
    pl.set_timing(False)
    total = sum(v["ms_total"] for v in kern.values())
    for v in kern.values():
        v["share"] = v["ms_total"] / total if total else None
    return ms, kern, clk


def image_diff(torch, a, b):
    """Max-normalised difference per (channel, product) of two device images
    [C][4][N][N] (cross products normalised by max(max XX, max YY)); its maximum."""
    C, Q = a.shape[0], a.shape[1]
    err = (a - b).abs().reshape(C, Q, -1).amax(-1)
    den = b.abs().reshape(C, Q, -1).amax(-1)
    if Q == 4:
        d = torch.maximum(den[:, 0], den[:, 1])
        den = torch.stack([den[:, 0], den[:, 1], d, d], 1)
    return float((err / den.clamp_min(1e-30)).max())


def dense_leg(args, ctx, wl_name, steps, warmup, fp16=True, headline=False, keep_image=False):
    """One dense workload on the FP16 tensor-core path (fp16) or the FP32 path:
    blocks of device voltages into the plan's FP64 accumulators."""
    moff, synth, torch, np = ctx.moff, ctx.synth, ctx.torch, ctx.np
    wl = DENSE[wl_name]
    C = args.chan or wl["n_chan"]
    B = args.block or wl["block"]
    A, P, N = wl["n_ant"], wl["n_pol"], wl["grid_n"]
    cfg = getattr(synth, wl["cfg"])(n_chan=C, with_gains=False)
    pos, taps = cfg["pos"], cfg["taps"]
    gains = synth.device_gains(wl["seed"] + 11, C, A, P)
    codes = synth.device_codes(wl["seed"] + 1000 * ctx.rank, B, C, A, P)
    torch.cuda.empty_cache()                  # the draws' temporaries: the plan allocates outside torch's cache
    t0 = time.perf_counter()
    pl = moff.Plan(pos, taps, N, C, P, jones=wl["jones"], fp16tc=fp16)
    setup_s = time.perf_counter() - t0
    pl.set_gains(gains)
    ms, kern, clk = measure_blocks(ctx, pl, codes, steps, warmup, sample_clocks=headline)
    snaps = steps * B * C
    info, route, tun = pl.info(), pl.route(), pl.tuning()
    work = dense_work(route, pos, taps, N, P, info["time_chunk"])
    roofs = kernel_rooflines(kern, work, snaps, ctx.peaks)
    for kind, r in roofs.items():             # DRAM bytes from the committed capture against the method's bytes
        kname = route_kernel(route, kind, N)
        units = snaps / max(r["launches"], 1)
        t = traffic_for(kname + "@" + wl_name, KERNEL_SOURCES.get(kname, []), units)
        r["traffic_bytes_per_launch"] = t
        r["traffic_over_algorithmic"] = t / (work[kind]["bytes"] * units) if t else None
    out = {"value": job_rate(snaps, ctx.world, ms / 1000.0), "unit": UNIT, "ms_per_step": ms / steps,
           "steps": steps, "warmup": warmup, "route": route, "dtype": "f16 tensor-core, f32 accumulate" if fp16 else "f32",
           "samples_per_step": B, "channels": C, "plan_create_s": setup_s, "chunk": [info["time_chunk"], info["chan_chunk"]],
           "grid_shape": {"time_batch": tun["time_batch"], "cells_per_lane": tun["cells_per_lane"]},
           "kernels": kern, "kernel_rooflines": roofs, "gpu_launches": sum(v["launches"] for v in kern.values()),
           "clocks": clk}
    img = None
    if keep_image:
        img = torch.empty((C, 4 if P == 2 else 1, N, N), dtype=torch.float32, device="cuda")
        _, n = pl.read_image(out=img)
        img /= float(n)
    if headline and not args.no_e2e and args.e2e_steps > 0:
        host = torch.empty(codes.shape, dtype=torch.uint8, pin_memory=True)
        host.copy_(codes)
        del codes                             # the end-to-end steps stage the block from host memory
        torch.cuda.empty_cache()
        out["e2e"] = dense_e2e(args, ctx, pl, host, C, P, N, B)
        del host
        codes = None
    pl.close()
    del codes, gains
    torch.cuda.empty_cache()
    return out, img, (pos, taps)


def dense_e2e(args, ctx, pl, host, C, P, N, B):
    """End to end through the C ABI with host buffers: every step copies its block
    of 4-bit voltages from pinned host memory (moff_submit with a host pointer
    stages it on the plan's copy stream); the integration's image is read back to
    pinned host memory once at the end (its bytes shared over the steps)."""
    torch = ctx.torch
    nq = 4 if P == 2 else 1
    out_h = torch.empty((C, nq, N, N), dtype=torch.float32, pin_memory=True)
    for _ in range(2):                          # warm both staging buffers and the read-back
        pl.submit(host)
    pl.read_image(out=out_h, reset=True)
    ctx.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        pl.submit(host)
    pl.read_image(out=out_h, reset=True)
    dt = max_over_ranks(time.perf_counter() - t0, ctx.dist, "cuda")
    n = args.e2e_steps
    return {"value": job_rate(n * B * C, ctx.world, dt), "unit": UNIT, "h2d_bytes_per_step": int(host.numel()),
            "d2h_bytes_per_step": int(out_h.numel() * 4 // n), "steps": n,
            "api": "moff_submit(host pinned voltages) per step + moff_read_image(host) of the integration at the end"}


def run_ours(args):
    import numpy as np
    import torch

    import paper_0812_3669_gb300 as moff
    import synth

    world, rank, local = rank_info()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or world > 1:
        moff.build()
    if dist is not None:
        dist.barrier()
    gpu_idx = local
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis and vis.split(",")[local].strip().isdigit():
        gpu_idx = int(vis.split(",")[local])
    ctx = Ctx(moff, synth, torch, np, world, rank, local, dist, device_peaks(torch), gpu_idx)

    if args.only == "dualpol":
        if rank == 0:
            print(json.dumps({"only": "dualpol", "dualpol_fstage": dualpol_leg(args, ctx)}), flush=True)
        return

    # ---------------------------------------------------------------- headline: the largest workload, FP16 tensor core
    wl = DENSE[args.workload]
    head, img16, (pos, taps) = dense_leg(args, ctx, args.workload, args.steps, args.warmup, fp16=True, headline=True,
                                         keep_image=not args.no_fp32)
    roofs = head["kernel_rooflines"]
    dom = max(roofs, key=lambda k: roofs[k]["ms_per_launch"] * roofs[k]["launches"])
    b = roofs[dom]["bound"]
    rd = roofs[dom][b]
    kname = route_kernel(head["route"], dom, wl["grid_n"])
    work = dense_work(head["route"], pos, taps, wl["grid_n"], wl["n_pol"], head["chunk"][0])[dom]
    per_launch = head["steps"] * head["samples_per_step"] * head["channels"] / max(roofs[dom]["launches"], 1)
    traffic = traffic_for(kname + "@" + args.workload, KERNEL_SOURCES.get(kname, []), per_launch)
    roofline = {"bound": b, "kernel": kname, "achieved": rd["achieved"], "peak": rd["peak"], "unit": rd["unit"],
                "frac": rd["frac"], "peak_basis": rd["basis"], "traffic": traffic,
                "work_per_launch": (work["tensor"] if b == "tensor" else work["alu"] if b == "alu" else work["bytes"])
                * per_launch,
                "ms_per_launch": roofs[dom]["ms_per_launch"],
                "traffic_over_algorithmic": traffic / (work["bytes"] * per_launch) if traffic else None}

    # ---------------------------------------------------------------- the same workload on the FP32 path
    fp32 = None
    if not args.no_fp32:
        fp32, img32, _ = dense_leg(args, ctx, args.workload, 2, 1, fp16=False, keep_image=True)
        fp32["max_norm_diff_fp16_vs_fp32"] = image_diff(torch, img16, img32)
        fp32["fp16_speedup"] = head["value"] / fp32["value"]
        del img32
    del img16
    torch.cuda.empty_cache()

    # ---------------------------------------------------------------- filled-aperture precision workload
    precision = None
    if not args.no_precision and args.workload != "precision":
        save = (args.chan, args.block)
        args.chan, args.block = 0, 0
        p16, i16, _ = dense_leg(args, ctx, "precision", 3, 1, fp16=True, keep_image=True)
        p32, i32, _ = dense_leg(args, ctx, "precision", 2, 1, fp16=False, keep_image=True)
        args.chan, args.block = save
        precision = {"workload": DENSE["precision"]["name"], "fp16tc": p16, "fp32": p32,
                     "fp16_speedup": p16["value"] / p32["value"],
                     "max_norm_diff_fp16_vs_fp32": image_diff(torch, i16, i32)}
        del i16, i32
        torch.cuda.empty_cache()

    # ---------------------------------------------------------------- dual-pol F-stage workload and its legs
    dualpol = None
    if not args.no_dualpol:
        dualpol = dualpol_leg(args, ctx)
    serving = None
    if not args.no_serving:
        im32, im16 = [], []
        serving = serving_leg(args, moff, synth, torch, images=im32)
        serving["fp16tc_stream"] = serving_leg(args, moff, synth, torch, fp16tc=True, images=im16)
        # the two streams summed the same blocks per plan: FP16 routes against the FP32 path, max-normalised
        serving["fp16tc_stream"]["max_norm_diff_vs_fp32"] = [image_diff(torch, a, b) for a, b in zip(im16, im32)]
        serving["fp16tc_stream"]["saturation_speedup"] = (serving["fp16tc_stream"]["saturation"]["throughput"]
                                                          / serving["saturation"]["throughput"])
        del im32, im16
        torch.cuda.empty_cache()
    batching = None
    if not args.no_plain:
        batching = batching_leg(args, moff, synth, torch)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline_subprocess(args.workload)

    if rank == 0:
        A, P = wl["n_ant"], wl["n_pol"]
        value = head["value"]
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f16 tensor-core (f32 accumulate, f64 across blocks)",
            "data": "synthetic",
            "config": {"workload": wl["name"], "antennas": A, "pols": P, "jones": wl["jones"],
                       "channels": head["channels"], "grid_n": wl["grid_n"], "kernel": wl["ksize"],
                       "samples_per_step": head["samples_per_step"], "integration_samples": wl["t_int"],
                       "channel_snapshots_per_step": head["samples_per_step"] * head["channels"],
                       "route": head["route"], "l2": "inputs larger than L2 (voltages per step >> 129 MB), no flush",
                       "parallelism": f"{world} independent replica(s), one block stream each"},
            "fx_equiv_tcmac_per_s": value * A * (A - 1) / 2 * 4 / 1e12,
            "roofline": roofline, "kernels": head["kernels"], "kernel_rooflines": roofs,
            "gpu_launches": head["gpu_launches"], "clocks": head["clocks"], "e2e": head.get("e2e"),
            "cpu_baseline": cpu, "plan_create_s": head["plan_create_s"],
            "legs": {"fp32_same_workload": fp32, "precision_filled_aperture": precision, "dualpol_fstage": dualpol,
                     "serving": serving, "batching": batching},
        }), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse_args()
    if args.cpu_sample:
        run_cpu_sample(args.cpu_sample)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    run_ours(args)


if __name__ == "__main__":
    main()
