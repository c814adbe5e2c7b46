#!/usr/bin/env python3
"""Throughput of the MOFF imaging hot path on one GB300 (or N replicas).

Workload (one step = one integration): 1024 dual-pol antennas hex-packed at
1.5 lambda with 5 % jitter; real 8-bit ADC streams (noise sigma 20 plus three
narrow-band sky sources) channelised by an 8-tap, 2048-sample polyphase
filter bank into 1024 channels and requantised to 4+4 bits; each channel
gridded on a 128x128 grid through 7x7 complex per-antenna kernels,
transformed, squared and summed over 1000 samples into XX, YY, Re XY, Im XY.
All arithmetic FP32 (FP64 cross-chunk sums).  A step processes
1000 x 1024 = 1,024,000 channel-snapshots; its 4.2 GB of ADC input is far
larger than L2, so no flush is needed between steps.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on a bounded sample of the same workload instead.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WL = dict(n_ant=1024, n_pol=2, n_chan=1024, grid_n=128, ksize=7, ntaps=8, frames=1000)
SEED = 8123669 + 1
METRIC = "MOFF channel-snapshots/s"
UNIT = "channel-snapshots/s"
WORKLOAD_NAME = ("dual-pol 1024-antenna hex core (1.5 lambda, 5% jitter), 8-bit ADC -> 8-tap x 2048 PFB "
                 "-> 1024 channels 4+4-bit, 128x128 grid, 7x7 complex kernels, XX/YY/XY, 1000 samples per step")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp16tc", action="store_true", help="skip the FP16 tensor-core leg")
    ap.add_argument("--no-serving", action="store_true", help="skip the request-stream (serving) leg")
    ap.add_argument("--no-feedback", action="store_true",
                    help="skip the legs of the method's extensions (feedback calibration, beams and autocorrelation "
                         "subtraction, channel-dependent positions and kernels, edge-padded oversampling)")
    ap.add_argument("--no-plain", action="store_true", help="skip the batching leg (graph + autotune vs one channel at a time)")
    ap.add_argument("--serve-requests", type=int, default=32, help="requests per load point of the serving leg")
    ap.add_argument("--cpu-sample", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--frames", type=int, default=WL["frames"],
                    help="samples per step (smaller values give a profiling case, not a bench line)")
    ap.add_argument("--channels", type=int, default=WL["n_chan"],
                    help="channels (smaller values give a profiling case, not a bench line)")
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


# ----------------------------------------------------------------------------- oracle (CPU) sample

def oracle_step(n_frames=2, seed=SEED):
    """The FP64 oracle on a bounded sample of the workload: the whole array's
    F-stage for ``n_frames`` frames, then every channel imaged for those frames.
    Returns (channel-snapshots, seconds)."""
    import numpy as np

    import oracle
    import synth
    cfg = synth.config_dualpol()
    A, P, C, N, ntaps = WL["n_ant"], WL["n_pol"], WL["n_chan"], WL["grid_n"], WL["ntaps"]
    M = 2 * C
    rng = np.random.default_rng(seed)
    adc = synth.adc_stream(rng, A, P, (n_frames + ntaps - 1) * M, sigma=20.0,
                           tones=[(100.0 / M, 12.0), (600.0 / M, 8.0)])
    gains = cfg["gains"]
    W = oracle.grid_matrix(cfg["pos"], cfg["taps"], N, P)      # plan set-up, not timed
    t0 = time.perf_counter()
    h = oracle.pfb_window(ntaps, M)
    X = oracle.pfb_spectra(adc, h, ntaps, M)
    scale = 2.0 / np.std(np.concatenate([X.real.ravel(), X.imag.ravel()]))
    codes, _ = oracle.channelise(adc, h, ntaps, M, scale)
    img = np.zeros((4, N, N))
    for c in range(C):
        y = oracle.calibrate(oracle.unpack_4bit(codes[:, c]), gains[c])
        img += oracle.integrate(oracle.sky_transform(oracle.grid(y, W, N, P)))
    dt = time.perf_counter() - t0
    return n_frames * C, dt


def cpu_baseline_subprocess():
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample"], env=env, capture_output=True,
                       text=True, timeout=900)
    for line in r.stdout.splitlines()[::-1]:
        if line.startswith("{"):
            return json.loads(line)
    return {"error": (r.stderr or r.stdout)[-300:]}


def run_cpu_sample():
    units, dt = oracle_step(n_frames=6)
    print(json.dumps({"value": units / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "seconds": dt,
                      "sample": f"whole-array F-stage for 6 frames + all {WL['n_chan']} channels imaged "
                                f"({units} channel-snapshots), FP64 numpy/scipy, 1 thread"}))


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    for _ in range(args.warmup):
        oracle_step(n_frames=1)
    units = 0
    secs = 0.0
    for _ in range(args.steps):
        u, dt = oracle_step()
        units += u
        secs += dt
    v = units / secs
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME, "sample_frames_per_step": 2, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "each step: whole-array F-stage for 2 frames + all 1024 channels imaged"},
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
}


def traffic_for(kernel_key, src):
    """Per-launch DRAM bytes from the committed ncu summary, if the kernel's
    source is unchanged since the capture (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path)).get(kernel_key)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("source_sha1") != source_sha1(src):
        return None
    return rec.get("bytes_per_launch")


def serving_leg(args, moff, synth, torch, fp16tc=False):
    """Request stream over sub-arrays of uneven size (MOFF_SERVED plans, one
    moff_server): first a closed burst to find the saturation rate, then Poisson
    arrivals at fractions of it.  Reports p50/p99 block latency and throughput.
    With fp16tc, each sub-array takes the FP16 tensor-core path where its density
    allows (at most 128 antennas' kernel rows on a grid row) and FP32 otherwise."""
    import numpy as np
    mix = synth.config_serving()
    plans, blocks, prec = [], [], []
    for i, a in enumerate(mix):
        pl = None
        if fp16tc:
            try:
                pl = moff.Plan(a["pos"], a["taps"], a["N"], a["C"], 2, served=True, fp16tc=True)
                prec.append("fp16tc")
            except moff.MoffError:
                pl = None
        if pl is None:
            pl = moff.Plan(a["pos"], a["taps"], a["N"], a["C"], 2, served=True)
            prec.append("fp32")
        pl.set_gains(a["gains"])
        plans.append(pl)
        blocks.append(synth.device_codes(SEED + 500 + i, a["T"], a["C"], a["A"], 2))
    torch.cuda.synchronize()
    units = [a["C"] * a["T"] for a in mix]
    rng = np.random.default_rng(SEED + 77)
    srv = moff.Server(24 << 30, 4)
    try:
        for i in range(len(plans)):                       # warm every plan once
            srv.submit(plans[i], blocks[i])
        srv.wait(0, 600000)
        srv.stats(reset=True)
        # saturation: everything at once
        order = rng.integers(0, len(plans), size=args.serve_requests)
        t0 = time.perf_counter()
        for i in order:
            srv.submit(plans[i], blocks[i])
        srv.wait(0, 600000)
        wall = time.perf_counter() - t0
        sat = srv.stats(reset=True)
        sat_req_s = len(order) / wall
        points = []
        for load in (0.5, 0.9):
            rate = load * sat_req_s
            order = rng.integers(0, len(plans), size=args.serve_requests)
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
            srv.wait(0, 600000)
            st = srv.stats(reset=True)
            points.append({"load": load, "offered_req_per_s": rate, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
                           "throughput": st["throughput"], "requests": st["completed"]})
    finally:
        srv.close()
        for pl in plans:
            pl.close()
    return {
        "unit": UNIT, "precision": "fp16tc where the array allows, else fp32" if fp16tc else "fp32",
        "slots": 4, "pool_bytes": 24 << 30,
        "mix": [{"antennas": a["A"], "grid_n": a["N"], "channels": a["C"], "samples": a["T"], "path": p}
                for a, p in zip(mix, prec)],
        "mix_note": "request sizes scaled to channels in {64,128,256} and 100-300 samples so a sweep takes seconds",
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
    batched.close()
    return {"unit": UNIT, "channels": Cs, "samples": F, "dtype": "f32",
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

    def barrier():
        if dist is not None:
            dist.barrier()

    if rank == 0 or world > 1:
        moff.build()
    barrier()

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
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12          # FP32 FMA TFLOP/s at max SM clock
    for name, v in kern.items():
        v["share"] = v["ms_total"] / total_kernel_ms if total_kernel_ms else None
        v["tflops"] = flops[name] / (v["ms_total"] / 1e3) / 1e12 if v["ms_total"] and name in flops else None
    dom = max(kern, key=lambda k: kern[k]["ms_total"])
    src = KERNEL_SOURCES.get(dom, [])
    launches = kern[dom]["launches"]
    achieved = kern[dom]["tflops"]
    roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": achieved / alu_peak if achieved else None,
                "peak_basis": f"FP32 FMA: 152 SMs x 128 lanes x 2 flop x {sm_max:.0f} MHz (of derived peak)",
                "flops_per_launch": flops[dom] / max(launches, 1),
                "ms_per_launch": kern[dom]["ms_total"] / max(launches, 1),
                "traffic": traffic_for(dom + "@dualpol1024", src)}
    gpu_launches = sum(v["launches"] for v in kern.values())

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
                                             "peak_basis": f"FP32 FMA: 152 SMs x 128 lanes x 2 flop x {sm_max:.0f} MHz "
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

    serving = None
    if not args.no_serving:
        serving = serving_leg(args, moff, synth, torch)
        serving["fp16tc_stream"] = serving_leg(args, moff, synth, torch, fp16tc=True)
    batching = None
    if not args.no_plain:
        batching = batching_leg(args, moff, synth, torch)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline_subprocess()

    if rank == 0:
        fx_eq = value * A * (A - 1) / 2 * 4
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME, "antennas": A, "pols": P, "channels": C, "grid_n": N,
                       "kernel": K, "pfb_taps": ntaps, "samples_per_step": F, "channel_snapshots_per_step": F * C,
                       "l2": "inputs larger than L2 (4.2 GB of ADC per step), no flush",
                       "parallelism": f"{world} independent replica(s), one integration each"},
            "fx_equiv_tcmac_per_s": fx_eq / 1e12,
            "roofline": roofline, "kernels": kern, "gpu_launches": gpu_launches, "clocks": clk,
            "e2e": e2e, "cpu_baseline": cpu, "fp16tc": fp16, "serving": serving, "batching": batching, "feedback": feedback,
            "beams_autocorr": taps_leg, "channel_sets": sets_leg,
        }), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse_args()
    if args.cpu_sample:
        run_cpu_sample()
        return
    if args.impl == "reference":
        run_reference(args)
        return
    run_ours(args)


if __name__ == "__main__":
    main()
