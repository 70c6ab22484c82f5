#!/usr/bin/env python
"""Benchmark: pulses/s of online sparse-SAR reconstruction (per pulse: phase
synthesis, dictionary apply, Gram + data-vector update, lambda and power
iteration for L, then a FISTA burst of up to m = 20 steps to tol = 1e-4) on
the 128 x 128 workload (N = 16384 pixels, M = 32768 Gaussian atoms,
K = 512 frequencies, 256 pulses over 45 deg) in the split-BF16 precision
form, against the plain FP64 GPU path and the FP64 CPU oracle.

One JSON line on rank 0.  `--impl reference` times the FP64 CPU oracle on
the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("pulses/s online (Gram update + FISTA burst to tol) at 128×128 "
          "vs FP64 path")
WORKLOAD = "c2_128x128_split_bf16"
INNER_STEPS = 20
TOL = 1e-4
POWER_ITERS = 4      # power steps per pulse after the first (library default)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=251,
                    help="timed pulses (default: the rest of the 256-pulse "
                         "aperture after the warm-up, less the time-to-tol pulse)")
    ap.add_argument("--warmup", type=int, default=4)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the 256x256 leg (with and without online "
                         "lambda tuning)")
    ap.add_argument("--fp64-pulses", type=int, default=2)
    ap.add_argument("--fp32-pulses", type=int, default=4)
    ap.add_argument("--forms", action="store_true",
                    help="also time the other configurations (32x32 FP64, the "
                         "64x64 adjoint, the 96-scene batch, the 256x256 form)")
    ap.add_argument("--no-overlap", action="store_true",
                    help="run each pulse's dictionary product on the main "
                         "stream instead of beside the previous burst")
    ap.add_argument("--no-fuse", action="store_true",
                    help="separate Gram passes for the last power step and "
                         "the first FISTA step of a pulse")
    ap.add_argument("--fuse-power-gram", type=int, choices=[0, 1], default=1,
                    help="1: the Gram update's epilogue also forms the "
                         "pulse's first power step (one Gram pass fewer)")
    ap.add_argument("--tc-pairs", type=int, default=3,
                    help="tensor-core products on SM pairs: bit 0 dictionary "
                         "product, bit 1 Gram update (0: one SM per tile)")
    ap.add_argument("--gram-ahead", type=int, choices=[0, 1, 2], default=1,
                    help="the Gram update beside the previous burst into a second "
                         "Gram buffer: 0 never, 1 when the library's model expects "
                         "it to pay (default), 2 always")
    ap.add_argument("--prof-every", type=int, default=1,
                    help="bracket one matvec launch in this many with CUDA events "
                         "in the timed region (a stride that shares a factor with "
                         "the passes per pulse samples some step positions only)")
    ap.add_argument("--synth-ctas", type=int, default=0,
                    help="SMs for the overlapped dictionary product (0: auto)")
    ap.add_argument("--defer-gram", type=int, choices=[0, 1], default=0,
                    help="1: each pulse's Gram update runs on the side stream "
                         "beside its power steps and burst, which add the "
                         "pulse's block term to G_{n-1} x")
    ap.add_argument("--pixel-gram", action="store_true",
                    help="dictionary workloads: run the pixel-space Gram form "
                         "(P_n, N x N) instead of the stored M x M Gram (for "
                         "profiler captures of its dictionary products)")
    ap.add_argument("--gram-superblock", type=int, default=0,
                    help="Gram update tile order: super-blocks of this many "
                         "blocks (0: the library's 32)")
    ap.add_argument("--workload", choices=["c2", "probe8k", "probe_dict", "probe16k"],
                    default="c2",
                    help="c2: the 128x128 headline workload; probe8k: a "
                         "64x128 pixel-basis scene (M = 8192, 272 MB packed "
                         "Gram) for profiler captures; probe_dict: a 64x64 "
                         "scene with 8192 Gaussian atoms (dictionary product "
                         "of 0.4 TFLOP) for profiler captures")
    return ap.parse_args()


# ----------------------------------------------------------------- helpers --

def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def max_over_ranks(x: float, device="cpu") -> float:
    """Largest value of x over all ranks (the job's time is its slowest
    rank's); identity without an initialised process group."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Units all ranks processed per second of the slowest rank (weak scaling:
    every rank runs its own replica of the workload)."""
    return world * units_per_rank / seconds


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0,
                "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,"
              "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def kernel_source_hash() -> str:
    path = os.path.join(ROOT, "paper_2603_08582_gb300", "csrc", "matvec.cuh")
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]


def profiled_traffic(kind: str):
    """DRAM bytes per launch from the committed ncu summary, when it was taken
    on the kernel source now in the tree (else None)."""
    path = os.path.join(ROOT, "profiles", f"{kind}_ncu.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    vals = {}
    for ln in text.splitlines():
        if ":" in ln and ln.strip().startswith("- "):
            k, v = ln.strip()[2:].rsplit(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("matvec.cuh sha256[:16]") != kernel_source_hash():
        return None
    try:
        return float(vals["dram bytes per full-size launch"])
    except (KeyError, ValueError):
        return None


# -------------------------------------------------------------- workload ---

def workload(name="c2"):
    from paper_2603_08582_gb300 import synth
    if name == "probe8k":
        return synth.Workload(
            name="probe8k_64x128", nx=128, ny=64, n_freq=512, f_lo_hz=9.75e9,
            f_hi_hz=10.25e9, n_pulses=64, span_deg=45.0, sparsity=0.03,
            snr_db=25.0, seed=8)
    if name == "probe16k":
        return synth.Workload(
            name="probe16k_128x64_M16384", nx=128, ny=64, n_freq=512,
            f_lo_hz=9.75e9, f_hi_hz=10.25e9, n_pulses=64, span_deg=45.0,
            dictionary="gaussian", n_atoms=16384, dict_seed=2, sparsity=0.03,
            snr_db=25.0, seed=10)
    if name == "probe_dict":
        return synth.Workload(
            name="probe_dict_64x64_M8192", nx=64, ny=64, n_freq=512,
            f_lo_hz=9.75e9, f_hi_hz=10.25e9, n_pulses=64, span_deg=45.0,
            dictionary="gaussian", n_atoms=8192, dict_seed=2, sparsity=0.03,
            snr_db=25.0, seed=9)
    return synth.workloads()[WORKLOAD]


def make_ctx(w, precision, stream, overlap=True, synth_ctas=0, tc_pairs=3,
             fuse=True, defer=False, power_gram=True, gram_superblock=0,
             pixel_gram=False, gram_ahead=0):
    from paper_2603_08582_gb300 import osar
    gauss = w.dictionary == "gaussian"
    cfg = osar.make_config(w.nx, w.ny, w.n_freq, w.f_lo_hz, w.f_hi_hz,
                           pixel_m=w.pixel_m, precision=precision,
                           dictionary="gaussian" if gauss else None,
                           n_atoms=w.m_atoms if gauss else None,
                           dict_seed=w.dict_seed, lam=w.lambda_rel,
                           stream=stream, overlap_synthesis=overlap,
                           synth_ctas=synth_ctas, tc_pairs=tc_pairs,
                           fuse_first_step=fuse,
                           defer_gram=(defer and overlap and gauss
                                       and precision == "split_bf16"),
                           fuse_power_gram=power_gram,
                           gram_superblock=gram_superblock,
                           pixel_gram=pixel_gram and gauss,
                           gram_ahead=(gram_ahead if overlap and not defer
                                       and not pixel_gram and precision == "split_bf16"
                                       else 0))
    return osar.Osar(cfg)


def pulse_data(ctx, w, n_pulses):
    """Noisy pulses d_s = G_s c_true + noise (SNR per pulse), simulated by the
    library on the device; the noise draws come from the input generator.
    Past the aperture's last pulse the sequence starts over (same work per
    pulse)."""
    from paper_2603_08582_gb300 import synth
    track = synth.workload_track(w)
    c_true = synth.workload_scene(w)
    p = min(n_pulses, w.n_pulses)
    noise = synth.unit_noise(w.n_pulses, w.n_freq, w.seed)
    clean = np.stack([ctx.simulate_pulse(track[s], c_true) for s in range(p)])
    data = clean + synth.scale_noise(clean, noise[:p], w.snr_db)
    idx = np.arange(n_pulses) % p
    return track[idx], np.ascontiguousarray(data[idx])


# ------------------------------------------------------------------ ours ---

def run_ours(args):
    import torch
    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2603_08582_gb300 import osar

    w = workload(args.workload)
    W, K = args.warmup, args.steps
    stream = torch.cuda.Stream()
    ov = dict(overlap=not args.no_overlap, synth_ctas=args.synth_ctas,
              tc_pairs=args.tc_pairs, fuse=not args.no_fuse,
              defer=bool(args.defer_gram) and not args.no_overlap,
              power_gram=bool(args.fuse_power_gram),
              gram_superblock=args.gram_superblock,
              pixel_gram=args.pixel_gram, gram_ahead=args.gram_ahead)
    ctx = make_ctx(w, "split_bf16", stream.cuda_stream, **ov)
    # the order of the stored Gram: M, or N in the pixel-space form
    gdim = w.n_pixels if args.pixel_gram and w.dictionary == "gaussian" else w.m_atoms
    # power steps per pulse that are Gram passes of their own
    power_passes = POWER_ITERS - (1 if ov["power_gram"] and not ov["defer"] else 0)
    # pulses: warm-up, timed, the per-kernel breakdown window, time to tol
    NBRK = 5
    total = W + K + NBRK + 1
    track, data = pulse_data(ctx, w, total)
    d_dev = torch.from_numpy(data).to(f"cuda:{local_rank}")
    torch.cuda.synchronize()
    d_ptr = d_dev.data_ptr()
    row = w.n_freq * 16

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    with torch.cuda.stream(stream):
        for s in range(W):
            ctx.push_pulse_dev(track[s], d_ptr + s * row)
            ctx.iterate(INNER_STEPS, TOL, want_count=False)
        ctx.synchronize()
        ctx.profile_reset()
        # the timed region brackets only the kernels its rooflines need (each
        # bracket adds two event records to the stream); the other classes
        # are timed in a short window after it
        ctx.profile_select("matvec", "gram_gemm", "dict_gemm")
        ctx.profile_sample("matvec", args.prof_every)
        ctx.profile_enable(True)
        launches0 = ctx.launch_count()
        sampler = ClockSampler(local_rank)
        sampler.start()
        barrier()
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for s in range(W, W + K):
            ctx.push_pulse_dev(track[s], d_ptr + s * row)
            ctx.iterate(INNER_STEPS, TOL, want_count=False)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
        clocks = sampler.stop()
        ms = ev0.elapsed_time(ev1)
        launches = ctx.launch_count() - launches0
        prof = {k: ctx.profile_read(k) for k in osar.KERNEL_CLASSES}
        passes = ctx.profile_passes()
        pushes_ahead, ahead_sms = ctx.profile_ahead(with_grid=True)
        # the same pass with the GPU to itself (Gram applies after the timed
        # region, nothing running beside them)
        ctx.profile_reset()
        ctx.profile_sample("matvec", 1)
        xs = np.random.default_rng(0).standard_normal(gdim).astype(np.complex128)
        for _ in range(8):
            ctx.gram_apply(xs)
        mv_alone = ctx.profile_read("matvec")
        # per-kernel breakdown: the next pulses with every class bracketed.
        # The first one is pushed with the GPU idle, so that its Gram update
        # runs in order on the whole GPU with nothing beside it (`alone`)
        ctx.profile_select()
        ctx.synchronize()
        ctx.profile_reset()
        gram_alone = (0, 0.0)
        for s in range(W + K, W + K + NBRK):
            ctx.push_pulse_dev(track[s], d_ptr + s * row)
            if s == W + K:
                gram_alone = ctx.profile_read("gram_gemm")
            ctx.iterate(INNER_STEPS, TOL, want_count=False)
        brk = {k: ctx.profile_read(k) for k in osar.KERNEL_CLASSES}
        ctx.profile_enable(False)

        # time to tolerance: the next pulse with its burst run until the
        # stop rule |c - z| <= tol |c| holds (at most 2000 steps)
        ev2 = torch.cuda.Event(enable_timing=True)
        ev3 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev2.record(stream)
        ctx.push_pulse_dev(track[W + K + NBRK], d_ptr + (W + K + NBRK) * row)
        steps_tt = ctx.iterate(2000, TOL)
        ev3.record(stream)
        torch.cuda.synchronize()
        ttt = {"tol": TOL, "pulse": W + K + NBRK + 1, "steps": int(steps_tt),
               "ms": round(ev2.elapsed_time(ev3), 3),
               "converged": bool(steps_tt < 2000)}
        ctx.close()

        # end to end on a second context, the same pulses: host data in,
        # coefficients back, every step
        ctx_e = make_ctx(w, "split_bf16", stream.cuda_stream, **ov)
        for s in range(W):
            ctx_e.push_pulse_dev(track[s], d_ptr + s * row)
            ctx_e.iterate(INNER_STEPS, TOL, want_count=False)
        pinned = torch.from_numpy(data[W:W + K].copy()).pin_memory().numpy()
        out_t = [torch.empty(w.m_atoms, dtype=torch.complex128).pin_memory()
                 for _ in range(2)]
        outs = [t.numpy() for t in out_t]
        ctx_e.synchronize()
        ctx_e.profile_reset()
        torch.cuda.synchronize()
        # one pulse in flight: the image of pulse s is read back while pulse
        # s + 1 is already queued (its dictionary product overlaps burst s)
        ev4 = torch.cuda.Event(enable_timing=True)
        ev5 = torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        ev4.record(stream)
        for q, s in enumerate(range(W, W + K)):
            ctx_e.push_pulse(track[s], pinned[q])
            ctx_e.iterate(INNER_STEPS, TOL, want_count=False)
            ctx_e.coeffs_async(outs[q % 2], slot=q % 2)
            if q:
                ctx_e.wait_coeffs((q - 1) % 2)
        ctx_e.wait_coeffs((K - 1) % 2)
        ev5.record(stream)
        e2e_s = time.perf_counter() - t0
        torch.cuda.synchronize()
        # the device time of the same window: the end-to-end wall time can
        # only exceed it (both run on this second context, after the timed
        # region of the first; their spread against `value` is run-to-run)
        e2e_dev_ms = ev4.elapsed_time(ev5)
        fista_steps = (ctx_e.profile_passes() - K * power_passes
                       + (0 if args.no_fuse else K))
        ctx_e.close()

    ms = max_over_ranks(ms, f"cuda:{local_rank}")
    e2e_s = max_over_ranks(e2e_s, f"cuda:{local_rank}")
    value = whole_job_rate(K, world, ms / 1e3)
    e2e_value = whole_job_rate(K, world, e2e_s)

    peaks, peak_src = measured_peaks()
    nblk = ctx_blocks(gdim)
    gram_bytes = nblk * 128 * 128 * 8
    mv_n, mv_ms = prof["matvec"]
    if args.prof_every == 1:
        # launches skipped after the stop rule held return at once: average
        # over the passes that streamed the Gram (their time dominates mv_ms)
        mv_avg = mv_ms / max(passes, 1)
    else:
        # a sample of the launches was bracketed: its average (every launch
        # of the window streams the Gram when mean_iters_per_pulse is the
        # step limit)
        mv_avg = mv_ms / max(mv_n, 1)
    achieved = gram_bytes / (mv_avg / 1e3) / 1e9
    traffic = profiled_traffic("matvec_c2")
    roofline = {"bound": "hbm", "kernel": "k_matvec<float> (packed upper Gram)",
                "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": round(achieved / peaks["hbm_gbs"], 4),
                "traffic": traffic, "peak_source": f"{peak_src} hbm_gbs",
                "algorithmic_bytes_per_launch": gram_bytes,
                "avg_launch_ms": round(mv_avg, 4), "launches": mv_n,
                "bracketed": ("every launch" if args.prof_every == 1 else
                              f"one launch in {args.prof_every} (CUDA events)"),
                "frac_of_spec_7900_gbs": round(achieved / 7900.0, 4),
                "passes": passes,
                "note": ("timed-region average: part of the passes share the "
                         "GPU with the next pulse's dictionary product"
                         + (" and, when the update runs ahead, its Gram update "
                            "(fewer SMs for the passes, HBM shared with its "
                            "read-modify-write); `alone` is the same pass with "
                            "the GPU to itself" if pushes_ahead else "")),
                "alone": {"avg_launch_ms": round(mv_alone[1] / max(mv_alone[0], 1), 4),
                          "achieved": round(gram_bytes / (mv_alone[1] / max(mv_alone[0], 1) / 1e3) / 1e9, 1),
                          "frac": round(gram_bytes / (mv_alone[1] / max(mv_alone[0], 1) / 1e3) / 1e9
                                        / peaks["hbm_gbs"], 4),
                          "launches": mv_alone[0]}}
    kp = ((w.n_freq + 127) // 128) * 128
    npx = ((w.n_pixels + 127) // 128) * 128
    gram_flops = nblk * 3 * 2 * 128 * 256 * 2 * kp
    dict_flops = (w.m_atoms // 128) * (kp // 128) * 3 * 2 * 128 * 256 * 2 * npx
    g_n, g_ms = prof["gram_gemm"]
    d_n, d_ms = prof["dict_gemm"]
    tens = {
        "gram": {"bound": "tensor", "executed_flops_per_launch": gram_flops,
                 "avg_launch_ms": round(g_ms / max(g_n, 1), 4),
                 "achieved": round(gram_flops / (g_ms / max(g_n, 1) / 1e3) / 1e12, 1),
                 "peak": peaks.get("bf16_tflops_sustained", 1724.5),
                 "unit": "TFLOP/s", "peak_source": f"{peak_src} bf16_tflops_sustained"},
        "dict": {"bound": "tensor", "executed_flops_per_launch": dict_flops,
                 "avg_ms_per_pulse": round(d_ms / max(g_n, 1), 4),
                 "achieved": round(dict_flops / max(d_ms / max(g_n, 1) / 1e3, 1e-12) / 1e12, 1),
                 "peak": peaks.get("bf16_tflops_sustained", 1724.5),
                 "unit": "TFLOP/s", "peak_source": f"{peak_src} bf16_tflops_sustained",
                 "overlapped": (None if args.no_overlap else
                                "side stream, a subset of the SMs, beside the "
                                "previous burst: its time is not on the "
                                "critical path and its frac is of the whole GPU")},
    }
    if d_ms <= 0:
        tens.pop("dict")
    if gram_alone[0] > 0:
        ga_ms = gram_alone[1] / gram_alone[0]
        ga = gram_flops / (ga_ms / 1e3) / 1e12
        tens["gram"]["alone"] = {
            "avg_launch_ms": round(ga_ms, 4), "achieved": round(ga, 1),
            "frac": round(ga / tens["gram"]["peak"], 4), "launches": gram_alone[0],
            "note": "the first pulse after the timed region, pushed with the GPU idle"}
    if pushes_ahead and ahead_sms:
        sm_all = torch.cuda.get_device_properties(local_rank).multi_processor_count
        tens["gram"]["overlapped"] = (
            f"side stream, {ahead_sms} of {sm_all} SMs, beside the previous burst "
            f"({pushes_ahead} of {K} pushes): frac is of the whole GPU")
        tens["gram"]["frac_of_its_sms"] = round(
            tens["gram"]["achieved"] / (tens["gram"]["peak"] * ahead_sms / sm_all), 4)
    for v in tens.values():
        v["frac"] = round(v["achieved"] / v["peak"], 4)
    # the whole pulse against HBM: the bytes its algorithm must move (the Gram
    # passes, the compensated Gram's read-modify-write, one read of the
    # dictionary planes) over the timed time per pulse; the Gram update's and
    # the product's tensor work overlap the passes when they run beside them
    step_bytes = (passes / K * gram_bytes + 2 * nblk * 128 * 128 * 12
                  + (w.m_atoms * npx * 8 if w.dictionary == "gaussian" else 0))
    step_roofline = {
        "bound": "hbm", "unit": "GB/s", "peak": peaks["hbm_gbs"],
        "bytes_per_pulse": int(step_bytes),
        "achieved": round(step_bytes / (ms / K / 1e3) / 1e9, 1),
        "frac": round(step_bytes / (ms / K / 1e3) / 1e9 / peaks["hbm_gbs"], 4),
        "counts": ("per pulse: Gram passes x packed Gram bytes, the compensated "
                   "Gram's read and write (12 B per stored entry each way), one read "
                   "of the split dictionary planes (8 B per entry)")}
    if args.pixel_gram:
        step_roofline = None  # the pixel-space form moves other bytes
    per_kernel = {k: {"launches": n, "total_ms": round(t, 3)} for k, (n, t) in brk.items()}
    per_kernel["window"] = (f"pulses {W + K + 1}..{W + K + NBRK}, after the timed "
                            "region, every kernel class bracketed by events")

    fp64 = fp32 = None
    if not args.no_fp64 and rank == 0 and args.workload == "c2":
        fp64 = run_precision_path(w, "fp64", track, data, stream, args.fp64_pulses)
        fp32 = run_precision_path(w, "fp32", track, data, stream, args.fp32_pulses)
    cpu = accuracy = large_ref = None
    if not args.no_cpu_baseline and rank == 0 and world == 1 and args.workload == "c2":
        # the CPU-baseline leg: the oracle timed on the 128 x 128 workload,
        # and its results on the first pulses of the 128 x 128 and (when that
        # leg runs) 256 x 256 workloads, which the accuracy entries compare
        # with the GPU path
        kept = {}
        cpu = cpu_baseline(w, pulses=1, keep=kept)
        if not args.no_large:
            large_ref = oracle_reference_large()
        accuracy = precision_report(w, kept, stream, ov)
        kept.clear()

    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "pulses/s",
        "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": round(ms / K, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3 (split-BF16) / fp32",
        "data": "synthetic (seeded scene, Philox Gaussian dictionary, device-simulated pulses + 25 dB noise)",
        "config": {"workload": w.name, "nx": w.nx, "ny": w.ny,
                   "n_pixels": w.n_pixels, "n_atoms": w.m_atoms,
                   "n_freq": w.n_freq, "pulses_total": w.n_pulses,
                   "pulses_timed": f"{W + 1}..{W + K} (after {W} warm-up)"
                                   + ("; the aperture repeats past 256" if W + K + 1 > w.n_pulses else ""),
                   "inner_steps_max": INNER_STEPS, "tol": TOL,
                   "precision": "split_bf16 (compensated)",
                   "overlap_synthesis": not args.no_overlap,
                   "synth_ctas": args.synth_ctas or "auto",
                   "tc_pairs": {0: "off", 1: "dictionary product", 2: "Gram update",
                                3: "dictionary product and Gram update"}[args.tc_pairs & 3],
                   "fused_first_step": not args.no_fuse,
                   "power_step_in_gram_update": bool(args.fuse_power_gram) and not ov["defer"],
                   "deferred_gram_update": bool(ov["defer"]),
                   "gram_ahead": {0: "off", 1: "model", 2: "always"}[args.gram_ahead],
                   "pushes_with_gram_ahead": f"{pushes_ahead} of {K}",
                   "gram_ahead_side_sms": ahead_sms,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "inputs larger than L2 (packed Gram 4.3 GB streamed per step)"},
        "clocks": clocks,
        "e2e": {"value": round(e2e_value, 3), "unit": "pulses/s",
                "h2d_bytes_per_step": w.n_freq * 16 + 24,
                "d2h_bytes_per_step": w.m_atoms * 16 + 4,
                "mean_iters_per_pulse": round(fista_steps / K, 2),
                "pipelined": "image of pulse s read while pulse s+1 is queued",
                "device_ms_per_step_same_window": round(e2e_dev_ms / K, 4),
                "wall_ms_per_step": round(1e3 * e2e_s / K, 4)},
        # Gram passes per pulse: the power steps (less the first one when
        # the Gram update forms it), plus the FISTA steps less the first one
        # when it shares the last power step's pass
        "mean_iters_per_pulse": round((passes - K * power_passes) / K
                                      + (0 if args.no_fuse else 1), 2),
        "time_to_tol": ttt,
        "gpu_launches": int(launches),
        "roofline": roofline,
        "tensor_rooflines": tens,
        "step_roofline": step_roofline,
        "per_kernel": per_kernel,
    }
    if fp64 is not None:
        line["fp64_path"] = fp64
        line["speedup_vs_fp64_path"] = round(value / fp64["value"], 2)
    if fp32 is not None:
        line["fp32_path"] = fp32
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if accuracy is not None:
        line["accuracy_vs_fp64_oracle"] = accuracy
    if rank == 0 and args.workload == "c2" and not args.no_large:
        line["pixel_space_gram_128x128"] = run_pixel_space_dense(stream, w)
        line["large_online_256x256"] = run_large_online(stream, ref=large_ref,
                                                        gram_ahead=args.gram_ahead)
    if args.forms and rank == 0:
        line["forms"] = run_forms(stream)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_pixel_space_dense(stream, w, warmup=4, pulses=16):
    """The 128 x 128 / M = 32768 Gaussian workload in the pixel-space Gram
    form (P_n, N x N; G_n applied as D^H P_n D): early pulses, every burst
    its 20 steps, against the stored-Gram form on the same pulses."""
    import torch
    from paper_2603_08582_gb300 import osar
    peaks, src = measured_peaks()
    out = {"workload": w.name + " (pixel-space Gram form)", "pulses_timed": pulses,
           "pulses_warmup": warmup, "inner_steps": INNER_STEPS}
    track = data = None
    for pixel in (False, True):
        cfg = osar.make_config(w.nx, w.ny, w.n_freq, w.f_lo_hz, w.f_hi_hz,
                               pixel_m=w.pixel_m, precision="split_bf16",
                               dictionary="gaussian", n_atoms=w.m_atoms,
                               dict_seed=w.dict_seed, lam=w.lambda_rel,
                               stream=stream.cuda_stream, pixel_gram=pixel)
        ctx = osar.Osar(cfg)
        if track is None:
            track, data = pulse_data(ctx, w, warmup + pulses)
        for s in range(warmup):
            ctx.push_pulse(track[s], data[s])
            ctx.iterate(INNER_STEPS, 0.0, want_count=False)
        ctx.synchronize()
        ctx.profile_reset()
        ctx.profile_enable(True)
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for s in range(warmup, warmup + pulses):
            ctx.push_pulse(track[s], data[s])
            ctx.iterate(INNER_STEPS, 0.0, want_count=False)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / pulses
        prof = {k: ctx.profile_read(k) for k in ("matvec", "dict_apply", "gram_gemm")}
        ctx.profile_enable(False)
        res = {"ms_per_pulse": round(ms, 2), "pulses_per_s": round(1e3 / ms, 2),
               "device_gb": round(ctx.device_bytes() / 1e9, 2)}
        if pixel:
            nbp = (w.n_pixels + 127) // 128
            p_bytes = nbp * (nbp + 1) // 2 * 128 * 128 * 8
            d_bytes = 4 * 2 * ((w.m_atoms + 127) // 128 * 128) * ((w.n_pixels + 127) // 128 * 128)
            mv_n, mv_ms = prof["matvec"]
            da_n, da_ms = prof["dict_apply"]
            mv_a, da_a = mv_ms / max(mv_n, 1), da_ms / max(da_n, 1)
            res["per_step_kernels"] = {
                "dictionary product (u = D x, or D^H w with its step)": {
                    "avg_ms": round(da_a, 4), "bytes": d_bytes, "launches": da_n,
                    "gbs": round(d_bytes / da_a / 1e6, 1),
                    "frac_of_hbm": round(d_bytes / da_a / 1e6 / peaks["hbm_gbs"], 3)},
                "w = P_n u (packed P_n pass)": {"avg_ms": round(mv_a, 4), "bytes": p_bytes,
                                               "gbs": round(p_bytes / mv_a / 1e6, 1),
                                               "frac_of_hbm": round(p_bytes / mv_a / 1e6
                                                                    / peaks["hbm_gbs"], 3)}}
            res["gram_update_ms"] = round(prof["gram_gemm"][1] / max(prof["gram_gemm"][0], 1), 3)
            out["pixel_space_form"] = res
        else:
            out["stored_gram_form"] = res
        ctx.close()
    out["peak_source"] = src
    return out


def run_large_online(stream, warmup=4, pulses=24, tune_every=8, ref=None,
                     gram_ahead=0):
    """The 256 x 256 pixel-basis workload (N = M = 65536, K = 1024, 10 FISTA
    steps per pulse, split-BF16), without and with online lambda tuning (the
    burst's adjoint every `tune_every` pulses against the synthetic scene,
    osar_set_lambda from the next pulse on)."""
    import torch
    from paper_2603_08582_gb300 import synth
    from paper_2603_08582_gb300.tuning import OnlineLambdaTuner
    w = synth.workloads()["c5_256x256_split_bf16"]
    steps = w.inner_steps
    c_true = synth.workload_scene(w)
    peaks, src = measured_peaks()
    out = {"workload": w.name, "n_atoms": w.m_atoms, "n_freq": w.n_freq,
           "inner_steps": steps, "pulses_timed": pulses,
           "pulses_warmup": warmup}
    track = data = None
    for tuned in (False, True):
        ctx = make_ctx(w, "split_bf16", stream.cuda_stream, gram_ahead=gram_ahead)
        if track is None:
            track, data = pulse_data(ctx, w, warmup + pulses)
        tuner = (OnlineLambdaTuner(ctx, c_true, rho=w.lambda_rel, steps=steps,
                                   every=tune_every) if tuned else None)
        for s in range(warmup):
            ctx.push_pulse(track[s], data[s])
            if tuner:
                tuner.after_push(s)
            ctx.iterate(steps, 0.0, want_count=False)
        ctx.synchronize()
        ctx.profile_reset()
        ctx.profile_enable(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for s in range(warmup, warmup + pulses):
            ctx.push_pulse(track[s], data[s])
            if tuner:
                tuner.after_push(s)
            ctx.iterate(steps, 0.0, want_count=False)
        ctx.synchronize()
        wall = time.perf_counter() - t0
        g_n, g_ms = ctx.profile_read("gram_gemm")
        mv_n, mv_ms = ctx.profile_read("matvec")
        passes = ctx.profile_passes()
        ahead, ahead_sms = ctx.profile_ahead(with_grid=True)
        ctx.profile_enable(False)
        err = float(np.linalg.norm(ctx.coeffs() - c_true) / np.linalg.norm(c_true))
        nblk = ctx_blocks(w.m_atoms)
        kp = ((w.n_freq + 127) // 128) * 128
        gram_flops = nblk * 3 * 2 * 128 * 256 * 2 * kp
        gram_bytes = nblk * 128 * 128 * 8
        mv_avg = mv_ms / max(passes, 1)
        res = {"pulses_per_s": round(pulses / wall, 3),
               "ms_per_pulse": round(1e3 * wall / pulses, 2),
               "device_gb": round(ctx.device_bytes() / 1e9, 1),
               "rel_err_vs_scene": round(err, 4),
               "gram_ahead": f"{ahead} of {pulses} pushes, {ahead_sms} side SMs",
               "gram_update": {"avg_ms": round(g_ms / max(g_n, 1), 3),
                               "tflops": round(gram_flops / (g_ms / max(g_n, 1) / 1e3) / 1e12, 1),
                               "frac_of_sustained": round(gram_flops / (g_ms / max(g_n, 1) / 1e3) / 1e12
                                                          / peaks["bf16_tflops_sustained"], 3)},
               "matvec": {"avg_ms_per_pass": round(mv_avg, 4),
                          "gbs": round(gram_bytes / mv_avg / 1e6, 1),
                          "frac_of_hbm": round(gram_bytes / mv_avg / 1e6 / peaks["hbm_gbs"], 3)}}
        if tuner:
            hist = tuner.history
            res["lambda_tuning"] = {
                "rule": "log rho -= 0.25 clip(lambda dL/dlambda / L, -1, 1) every "
                        f"{tune_every} pulses; L = |c_T - c_scene|^2 through the "
                        f"{steps}-step burst (osar_unroll_grad)",
                "updates": len(hist),
                "rho_first_last": [round(hist[0]["rho"], 5), round(tuner.rho, 5)] if hist else None,
                "loss_first_last": [hist[0]["loss"], hist[-1]["loss"]] if hist else None}
            out["tuned"] = res
        else:
            out["untuned"] = res
        ctx.close()
    if ref is not None:
        # accuracy against the FP64 oracle's run that the CPU-baseline leg made
        ctx = make_ctx(w, "split_bf16", stream.cuda_stream)
        acc = compare_with_oracle(ctx, ref, steps, 0.0)
        ctx.close()
        out["accuracy_vs_fp64_oracle"] = acc
    out["peak_source"] = src
    return out


def ctx_blocks(m):
    nb = (m + 127) // 128
    return nb * (nb + 1) // 2


def run_precision_path(w, precision, track, data, stream, pulses):
    """Another precision form on the same workload, a few pulses after one
    untimed pulse: the plain FP64 path (Gram and dictionary products on the
    FP64 pipes) or FP32 (SIMT FP32 products, FP32 Gram and matvec)."""
    import torch
    ctx = make_ctx(w, precision, stream.cuda_stream)
    with torch.cuda.stream(stream):
        ctx.push_pulse(track[0], data[0])
        ctx.iterate(INNER_STEPS, TOL)
        ctx.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for s in range(1, 1 + pulses):
            ctx.push_pulse(track[s], data[s])
            ctx.iterate(INNER_STEPS, TOL, want_count=False)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    ctx.close()
    return {"value": round(pulses / (ms / 1e3), 4), "unit": "pulses/s",
            "pulses_timed": pulses, "ms_per_pulse": round(ms / pulses, 2),
            "dtype": {"fp64": "f64", "fp32": "f32"}[precision]}


# -------------------------------------------------------- other forms ---

def _time(fn, stream):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def _pixel_ctx(w, prec, stream):
    from paper_2603_08582_gb300 import osar
    return osar.Osar(osar.make_config(
        w.nx, w.ny, w.n_freq, w.f_lo_hz, w.f_hi_hz, pixel_m=w.pixel_m,
        precision=prec, lam=w.lambda_rel, stream=stream.cuda_stream))


def _sim_pulses(ctx, w, n):
    from paper_2603_08582_gb300 import synth
    track = synth.workload_track(w)
    c_true = synth.workload_scene(w)
    noise = synth.unit_noise(w.n_pulses, w.n_freq, w.seed)
    clean = np.stack([ctx.simulate_pulse(track[s], c_true) for s in range(n)])
    return track, clean + synth.scale_noise(clean, noise[:n], w.snr_db), c_true


def run_forms(stream):
    """Pulses/s (or gradient time) of the other configurations, device-timed
    with CUDA events on the library's stream."""
    import torch
    from paper_2603_08582_gb300 import osar, synth
    out = {}
    wl = synth.workloads()
    with torch.cuda.stream(stream):
        # 32 x 32 pixel basis, FP64 (plain method) and split-BF16
        w = wl["c1_32x32_fp64"]
        for prec in ("fp64", "split_bf16"):
            ctx = _pixel_ctx(w, prec, stream)
            track, data, _ = _sim_pulses(ctx, w, w.n_pulses)

            def run(c=ctx, tr=track, dd=data):
                for s in range(w.n_pulses):
                    c.push_pulse(tr[s], dd[s])
                    c.iterate(w.inner_steps, 0.0, want_count=False)
            ms = _time(run, stream)
            out[f"c1_32x32_{prec}"] = {"pulses": w.n_pulses, "ms": round(ms, 2),
                                       "pulses_per_s": round(w.n_pulses / (ms / 1e3), 1)}
            ctx.close()
        # 64 x 64 differentiation form: gradient through T = 64 steps
        w = wl["c3_64x64_adjoint"]
        T, C = w.extra["unroll_T"], w.extra["checkpoint_every"]
        for prec in ("fp64", "fp32"):
            ctx = _pixel_ctx(w, prec, stream)
            track, data, c_true = _sim_pulses(ctx, w, w.n_pulses)
            for s in range(w.n_pulses):
                ctx.push_pulse(track[s], data[s])
            st = ctx.state()
            c0 = np.zeros(w.m_atoms, complex)
            ctx.unroll_grad(T, C, st["lambda"], 1.0 / st["lipschitz"], c0, c_true)
            ms = _time(lambda: ctx.unroll_grad(T, C, st["lambda"], 1.0 / st["lipschitz"],
                                               c0, c_true), stream)
            out[f"c3_adjoint_{prec}"] = {"T": T, "checkpoint_every": C,
                                         "ms_per_gradient": round(ms, 3)}
            ctx.close()
        # 96 uneven scenes in one batch: scene-pulses per second
        ws = synth.batch_workloads(96)
        tracks = [synth.workload_track(x) for x in ws]
        rng = np.random.default_rng(0)
        datas = [[rng.standard_normal(x.n_freq) + 1j * rng.standard_normal(x.n_freq)
                  for x in ws] for _ in range(7)]
        first = {}  # every scene's coefficients after the first pulse
        for prec, pulses in (("split_bf16", 6), ("fp32", 6), ("fp64", 1)):
            cfgs = [osar.make_config(x.nx, x.ny, x.n_freq, x.f_lo_hz, x.f_hi_hz,
                                     precision=prec) for x in ws]
            b = osar.OsarBatch(cfgs, stream=stream.cuda_stream)
            seg = b.autotune()
            tuning = b.tuning()
            b.push([1] * len(ws), np.stack([t[0] for t in tracks]), datas[0])
            b.iterate(20, 0.0, want_counts=False)
            first[prec] = [b.coeffs(q) for q in range(len(ws))]

            def runb(bb=b, dd=datas):
                for s in range(1, pulses + 1):
                    bb.push([1] * len(ws), np.stack([t[s] for t in tracks]), dd[s])
                    bb.iterate(20, 0.0, want_counts=False)
            ms = _time(runb, stream)
            out[f"c4_batch96_{prec}"] = {
                "batch_pulses": pulses, "scene_pulses_per_s": round(96 * pulses / (ms / 1e3), 1),
                "ms_per_batch_pulse": round(ms / pulses, 2), "segment_blocks": seg,
                "tuning": tuning,
                "device_gb": round(b.info()["device_bytes"] / 1e9, 2)}
            b.close()
        if "c4_batch96_fp64" in out:
            base = out["c4_batch96_fp64"]["scene_pulses_per_s"]
            for prec in ("split_bf16", "fp32"):
                out[f"c4_batch96_{prec}"]["speedup_vs_fp64"] = round(
                    out[f"c4_batch96_{prec}"]["scene_pulses_per_s"] / base, 1)
                # the accuracy that speed-up comes at: each scene's
                # coefficients after the first pulse (20 steps) against the
                # FP64 batch's (which meets the oracle to 1e-7)
                errs = [float(np.linalg.norm(a - r) / max(np.linalg.norm(r), 1e-300))
                        for a, r in zip(first[prec], first["fp64"])]
                out[f"c4_batch96_{prec}"]["rel_err_vs_fp64_first_pulse"] = {
                    "max_over_scenes": max(errs), "median": float(np.median(errs))}
        # 256 x 256 large online form, split-BF16, 10 steps per pulse
        w = wl["c5_256x256_split_bf16"]
        ctx = _pixel_ctx(w, "split_bf16", stream)
        track, data, _ = _sim_pulses(ctx, w, 5)
        ctx.push_pulse(track[0], data[0])
        ctx.iterate(w.inner_steps, 0.0, want_count=False)

        def run5():
            for s in range(1, 5):
                ctx.push_pulse(track[s], data[s])
                ctx.iterate(w.inner_steps, 0.0, want_count=False)
        ms = _time(run5, stream)
        out["c5_256x256_split_bf16"] = {"pulses": 4, "ms_per_pulse": round(ms / 4, 2),
                                        "pulses_per_s": round(4 / (ms / 1e3), 2),
                                        "device_gb": round(ctx.device_bytes() / 1e9, 1)}
        ctx.close()
        # lambda path on the 128 x 128 workload: 4 lambdas on one Gram (each
        # pass serves two solutions) against one lambda, 20 steps per pulse
        w = wl["c2_128x128_split_bf16"]
        lams = [0.02, 0.05, 0.08, 0.12]
        res = {}
        for n in (1, len(lams)):
            cfg = osar.make_config(
                w.nx, w.ny, w.n_freq, w.f_lo_hz, w.f_hi_hz, pixel_m=w.pixel_m,
                precision="split_bf16", dictionary="gaussian", n_atoms=w.m_atoms,
                dict_seed=w.dict_seed, lam=lams[0], stream=stream.cuda_stream,
                lambdas=lams[:n], gram_ahead=1)
            ctx = osar.Osar(cfg)
            track, data, _ = _sim_pulses(ctx, w, 7)
            for s in range(3):
                ctx.push_pulse(track[s], data[s])
                ctx.iterate(INNER_STEPS, 0.0, want_count=False)

            def runp(c=ctx, tr=track, dd=data):
                for s in range(3, 7):
                    c.push_pulse(tr[s], dd[s])
                    c.iterate(INNER_STEPS, 0.0, want_count=False)
            res[n] = _time(runp, stream) / 4
            ctx.close()
        out["c2_lambda_path"] = {
            "lambdas": len(lams), "pulses": 4, "steps": INNER_STEPS,
            "gram_ahead": "model (both runs)",
            "ms_per_pulse": round(res[len(lams)], 2),
            "ms_per_pulse_one_lambda": round(res[1], 2),
            "solution_pulses_per_s": round(len(lams) / (res[len(lams)] / 1e3), 1),
            "speedup_vs_separate": round(len(lams) * res[1] / res[len(lams)], 2)}
        out.update(run_edgelet_forms(stream))
    return out


def run_edgelet_forms(stream):
    """The edgelet dictionary (§III-A): the 128 x 128 geometry with the
    square scenes' dictionary (M = 2N = 32768 atoms, as the Gaussian
    workload), and scenes like the experiments' four, each run until the
    number of large coefficients (|c| > 0.02) reaches its true atom count
    (4, 8, 5, 5)."""
    from paper_2603_08582_gb300 import osar, synth
    out = {}
    w0 = synth.workloads()["c2_128x128_split_bf16"]
    w = synth.Workload(**{**w0.as_dict(), "name": "c2_128x128_edgelet",
                          "dictionary": "edgelet", "n_atoms": None,
                          "edgelet_lengths": (4,), "edgelet_angles": (0.0, 90.0)})
    # the stored-Gram form (G_n, M x M), then the pixel-space Gram form
    # (P_n, N x N, G_n applied as H^H P_n H) on the same pulses
    c_stored = None
    for pixel in (False, True):
        cfg = osar.make_config(w.nx, w.ny, w.n_freq, w.f_lo_hz, w.f_hi_hz,
                               pixel_m=w.pixel_m, precision="split_bf16",
                               dictionary="edgelet", edgelet_lengths=[4],
                               edgelet_angles=[0.0, 90.0], lam=w.lambda_rel,
                               stream=stream.cuda_stream, pixel_gram=pixel)
        ctx = osar.Osar(cfg)
        W, P = 4, 32
        track, data, _ = _sim_pulses(ctx, w, W + P)
        for s in range(W):
            ctx.push_pulse(track[s], data[s])
            ctx.iterate(INNER_STEPS, TOL, want_count=False)
        ctx.synchronize()
        ctx.profile_reset()
        ctx.profile_enable(True)
        steps = []

        def rune():
            for s in range(W, W + P):
                ctx.push_pulse(track[s], data[s])
                steps.append(ctx.iterate(INNER_STEPS, TOL))
        ms = _time(rune, stream) / P
        ph = ctx.profile_read("phase")[1] / P
        dg = ctx.profile_read("dict_gemm")[1] / P
        gr = ctx.profile_read("gram_gemm")[1] / P
        mv_n, mv_ms = ctx.profile_read("matvec")
        ctx.profile_enable(False)
        # the packed Gram one matvec pass reads (G_n, or P_n in the pixel form)
        nbg = ((w.n_pixels if pixel else w.m_atoms) + 127) // 128
        pass_bytes = nbg * (nbg + 1) // 2 * 128 * 128 * 8
        mv_avg = mv_ms / max(mv_n, 1)
        hbm = measured_peaks()[0]["hbm_gbs"]
        res = {
            "pulses": P, "ms_per_pulse": round(ms, 2),
            "pulses_per_s": round(1e3 / ms, 1), "mean_iters": round(float(np.mean(steps)), 2),
            "synthesis_ms_per_pulse": {"phases": round(ph, 3), "edgelet_block": round(dg, 3)},
            "gram_ms_per_pulse": round(gr, 3), "device_gb": round(ctx.device_bytes() / 1e9, 1),
            "matvec": {"bytes_per_pass": pass_bytes, "avg_launch_ms": round(mv_avg, 4),
                       "achieved_gbs": round(pass_bytes / mv_avg / 1e6, 1),
                       "frac_of_measured_hbm": round(pass_bytes / mv_avg / 1e6 / hbm, 3)}}
        c_hat = ctx.coeffs()
        if not pixel:
            c_stored = c_hat
            out["c2_128x128_edgelet_split_bf16"] = res
        else:
            res["gram_order"] = {"stored_form": w.m_atoms, "pixel_form": w.n_pixels}
            res["coeffs_rel_diff_vs_stored_gram_form"] = float(
                np.linalg.norm(c_hat - c_stored) / max(np.linalg.norm(c_stored), 1e-300))
            out["c2_128x128_edgelet_pixel_gram_split_bf16"] = res
        ctx.close()
    # the experiments' four scenes (a square: 4 atoms; two squares: 8; lines
    # of varying intensity, spaced or adjoined: 5 each): 4 km radius, 1 km
    # up, 1000 positions over 2 degrees, pulses kept with p = 0.3, m = 20
    scenes = [("paper_scene1_32x32_split_bf16", "square"),
              ("paper_scene2_32x32_split_bf16", "two_squares"),
              ("paper_scene3_32x32_split_bf16", "lines_spaced"),
              ("paper_scene4_32x32_split_bf16", "lines_adjoined")]
    for key, kind in scenes:
        out[key] = paper_scene_form(kind, stream)
    return out


def paper_scene_form(kind, stream):
    """Run one of the experiments' scenes until its large-coefficient count
    (|c| > 0.02) equals the number of true atoms, or to the last pulse."""
    from paper_2603_08582_gb300 import osar, synth
    lengths, angles, c_true = synth.paper_scene(kind, 32, 32)
    ideal = int(np.count_nonzero(c_true))
    sw = synth.Workload(name=f"paper_{kind}_32x32", nx=32, ny=32, n_freq=128,
                        f_lo_hz=9.9e9, f_hi_hz=10.1e9, n_pulses=1000, span_deg=2.0,
                        radius_m=4000.0, height_m=1000.0, dictionary="edgelet",
                        edgelet_lengths=lengths, edgelet_angles=angles,
                        snr_db=20.0, seed=7)
    track = synth.sampled_track(1000, 4000.0, 1000.0, 2.0, 0.3, sw.seed)
    cfg = osar.make_config(sw.nx, sw.ny, sw.n_freq, sw.f_lo_hz, sw.f_hi_hz,
                           precision="split_bf16", dictionary="edgelet",
                           edgelet_lengths=list(lengths), edgelet_angles=list(angles),
                           lam=0.05, stream=stream.cuda_stream)
    ctx = osar.Osar(cfg)
    clean = np.stack([ctx.simulate_pulse(g, c_true) for g in track])
    noise = synth.unit_noise(len(track), sw.n_freq, sw.seed)
    data = clean + synth.scale_noise(clean, noise, sw.snr_db)
    # the experiments' figures (large-coefficient count, Eq. 18's SNR read
    # in the coefficient domain: the scene's atoms against the rest) from
    # the library's device reduction, every pulse
    support = np.flatnonzero(c_true)
    counts, reached, m = [], None, None
    e0 = time.perf_counter()
    for s in range(len(track)):
        ctx.push_pulse(track[s], data[s])
        ctx.iterate(20, 0.0, want_count=False)
        m = ctx.metrics(2e-2, support)
        counts.append(m["n_large"])
        if m["n_large"] == ideal:
            reached = s + 1
            break
    wall = time.perf_counter() - e0
    ctx.close()
    return {
        "scene": kind, "true_atoms": ideal, "positions": 1000,
        "pulses_available": int(len(track)),
        "pulses_to_ideal_count": reached, "final_count": counts[-1],
        "large_are_the_true_atoms": bool(m["n_large"] == ideal
                                         and m["large_outside_support"] == 0),
        "coefficient_snr_db": round(m["snr_db"], 1),
        "count_after_pulses": {str(k): counts[k - 1] for k in (1, 5, 10, 20, 50, 100)
                               if k <= len(counts)},
        "ms_per_pulse_with_readback": round(1e3 * wall / len(counts), 3)}


# ------------------------------------------------------------ CPU oracle ---

def _dict_chunk(args):
    n, j0, j1, seed = args
    from paper_2603_08582_gb300 import synth
    return j0, synth.gaussian_dictionary_columns(n, np.arange(j0, j1), seed)


def host_dictionary(w, procs):
    """The same Philox dictionary on the host, generated by a spawn pool."""
    import multiprocessing as mp
    d = np.empty((w.n_pixels, w.m_atoms), dtype=np.complex128, order="F")
    chunk = 512
    jobs = [(w.n_pixels, j, min(w.m_atoms, j + chunk), w.dict_seed)
            for j in range(0, w.m_atoms, chunk)]
    with mp.get_context("spawn").Pool(procs) as pool:
        for j0, cols in pool.imap_unordered(_dict_chunk, jobs):
            d[:, j0:j0 + cols.shape[1]] = cols
    return d


def cpu_baseline(w, pulses=1, warmup=1, keep=None):
    """FP64 oracle on the host cores: `warmup` untimed pulses, then `pulses`
    timed pulses of the full 128 x 128 / M = 32768 workload.  Its inputs are
    made on the host: the dictionary by the input generator, the pulse data
    by the oracle's own forward model (d_s = F_s (H c_true) + noise)."""
    from oracle import osar_oracle as orc
    from paper_2603_08582_gb300 import synth
    cores = os.cpu_count() or 1
    t_setup = time.perf_counter()
    d = host_dictionary(w, cores)
    track = synth.workload_track(w)
    c_true = synth.workload_scene(w)
    noise = synth.unit_noise(w.n_pulses, w.n_freq, w.seed)
    rho = d @ c_true
    x = orc.pixel_positions(w.nx, w.ny, w.pixel_m)
    f = orc.frequencies(w.n_freq, w.f_lo_hz, w.f_hi_hz)
    total = warmup + pulses
    clean = np.stack([orc.phase_matrix(track[s], x, f) @ rho
                      for s in range(total)])
    data = clean + synth.scale_noise(clean, noise[:total], w.snr_db)
    of = orc.OnlineFista(orc.OracleConfig(
        nx=w.nx, ny=w.ny, pixel_m=w.pixel_m, n_freq=w.n_freq,
        f_lo_hz=w.f_lo_hz, f_hi_hz=w.f_hi_hz, dictionary=d, lam=w.lambda_rel))
    for s in range(warmup):
        of.push_pulse(track[s], data[s])
        of.iterate(INNER_STEPS, TOL)
    setup = time.perf_counter() - t_setup
    t0 = time.perf_counter()
    for s in range(warmup, total):
        of.push_pulse(track[s], data[s])
        of.iterate(INNER_STEPS, TOL)
    dt = time.perf_counter() - t0
    if keep is not None:
        # what the precision report compares the GPU path with (arrays only)
        keep.update(oracle_state(of, track[:total], data, INNER_STEPS, TOL))
    return {"value": round(pulses / dt, 5), "unit": "pulses/s", "cores": cores,
            "kind": "oracle",
            "sample": (f"{pulses} full pulse(s) (pulse index {warmup}..{total - 1}) of "
                       f"the 128x128 / M=32768 workload after {warmup} untimed "
                       f"pulse(s); setup {setup:.1f} s untimed; numpy FP64, BLAS on "
                       "all host cores")}


def _errors(got, ref):
    """Relative 2-norm error and worst element relative to max |ref|."""
    got, ref = np.asarray(got), np.asarray(ref)
    den = float(np.linalg.norm(ref))
    scale = float(np.max(np.abs(ref))) if ref.size else 0.0
    return {"rel_2norm": float(np.linalg.norm(got - ref) / den) if den > 0 else None,
            "worst_rel_max": float(np.max(np.abs(got - ref)) / scale) if scale > 0 else None}


def oracle_state(of, track, data, steps, tol, gram_sample=64):
    """Part of the CPU-baseline leg: the oracle's state after the pulses it
    ran, as plain arrays (sampled Gram entries, b, c_hat, the last pre-shrink
    vector u, lambda_n, L_n), so that the GPU comparison runs no oracle
    code."""
    rng = np.random.default_rng(0)
    cols = np.sort(rng.choice(of.m, gram_sample, replace=False))
    rr, cc = np.meshgrid(cols, cols, indexing="ij")
    rows, cols2 = rr.ravel(), cc.ravel()
    entries = (of.s.gram.entries(rows, cols2) if of.matrix_free
               else of.s.gram[rows, cols2])
    return {"track": track, "data": data, "steps": steps, "tol": tol,
            "rows": rows, "cols": cols2, "gram_entries": np.array(entries),
            "b": of.s.b.copy(), "c_hat": of.s.c_hat.copy(), "u": of.s.u.copy(),
            "lam": of.s.lam, "lip": of.s.lip}


def oracle_reference_large(pulses=2):
    """Part of the CPU-baseline leg: the FP64 oracle in its matrix-free mode
    (Eq. 10; the 69 GB FP64 Gram does not fit in host memory) on the first
    pulses of the 256 x 256 workload, 10 steps each, host data from the
    oracle's own forward model."""
    from oracle import osar_oracle as orc
    from paper_2603_08582_gb300 import synth
    w = synth.workloads()["c5_256x256_split_bf16"]
    tr = synth.workload_track(w)[:pulses]
    c_true = synth.workload_scene(w)
    x = orc.pixel_positions(w.nx, w.ny, w.pixel_m)
    f = orc.frequencies(w.n_freq, w.f_lo_hz, w.f_hi_hz)
    clean = np.stack([orc.phase_matrix(g, x, f) @ c_true for g in tr])
    noise = synth.unit_noise(w.n_pulses, w.n_freq, w.seed)[:pulses]
    dd = clean + synth.scale_noise(clean, noise, w.snr_db)
    of = orc.OnlineFista(orc.OracleConfig(
        nx=w.nx, ny=w.ny, pixel_m=w.pixel_m, n_freq=w.n_freq, f_lo_hz=w.f_lo_hz,
        f_hi_hz=w.f_hi_hz, lam=w.lambda_rel), matrix_free=True)
    for s in range(pulses):
        of.push_pulse(tr[s], dd[s])
        of.iterate(w.inner_steps)
    ref = oracle_state(of, tr, dd, w.inner_steps, 0.0, gram_sample=48)
    ref["oracle"] = ("FP64 CPU oracle in its matrix-free mode (Eq. 10), the "
                     "oracle's forward model for the data")
    return ref


def precision_report(w, kept, stream, ov):
    """The split-BF16 path with the bench's launch configuration against the
    FP64 oracle on the pulses the CPU baseline ran (the aperture's first
    ones, the same host data): sampled Gram entries, b, the coefficients
    (with the support difference), lambda_n and L_n, each as a relative
    error; and the pixel-space Gram form on the same pulses."""
    ctx = make_ctx(w, "split_bf16", stream.cuda_stream, **ov)
    out = compare_with_oracle(ctx, kept, INNER_STEPS, TOL)
    ctx.close()
    from paper_2603_08582_gb300 import osar
    cfg = osar.make_config(w.nx, w.ny, w.n_freq, w.f_lo_hz, w.f_hi_hz,
                           pixel_m=w.pixel_m, precision="split_bf16",
                           dictionary="gaussian", n_atoms=w.m_atoms,
                           dict_seed=w.dict_seed, lam=w.lambda_rel,
                           stream=stream.cuda_stream, pixel_gram=True)
    pix = osar.Osar(cfg)
    out["pixel_space_form"] = compare_with_oracle(pix, kept, INNER_STEPS, TOL,
                                                  with_gram=False)
    pix.close()
    out["oracle"] = "FP64 CPU oracle, same host data (d_s = F_s (H c_true) + noise)"
    return out


def compare_with_oracle(ctx, ref, steps, tol, with_gram=True):
    """Push the oracle's pulses through ctx and compare its state with the
    oracle's arrays (oracle_state): sampled Gram entries, b, the
    coefficients with their support difference, lambda_n and L_n."""
    track, data = ref["track"], ref["data"]
    used = []
    for s in range(track.shape[0]):
        ctx.push_pulse(track[s], data[s])
        used.append(ctx.iterate(steps, tol))
    res = {"pulses": int(track.shape[0]), "steps_per_pulse_gpu": used}
    if with_gram:
        g_gpu = ctx.gram_entries(ref["rows"], ref["cols"])
        res["gram_sampled_entries"] = {**_errors(g_gpu, ref["gram_entries"]),
                                       "entries": int(ref["gram_entries"].size)}
    c_gpu, c_orc = ctx.coeffs(), ref["c_hat"]
    st = ctx.state()
    sup_gpu, sup_orc = np.abs(c_gpu) > 0, np.abs(c_orc) > 0
    alpha = ref["lam"] / ref["lip"]
    near = np.abs(np.abs(ref["u"]) - alpha) <= 1e-3 * np.max(np.abs(ref["u"]))
    diff = sup_gpu != sup_orc
    res.update({
        "b": _errors(ctx.b(), ref["b"]),
        "coefficients": {**_errors(c_gpu, c_orc),
                         "support_size_oracle": int(np.count_nonzero(sup_orc)),
                         "support_differences": int(np.count_nonzero(diff)),
                         "support_differences_outside_threshold_band":
                             int(np.count_nonzero(diff & ~near)),
                         "threshold_band": "||u_i| - lambda tau| <= 1e-3 max|u|"},
        "lambda_rel_err": abs(st["lambda"] - ref["lam"]) / ref["lam"],
        "lipschitz_rel_err": abs(st["lipschitz"] - ref["lip"]) / ref["lip"]})
    if "oracle" in ref:
        res["oracle"] = ref["oracle"]
    return res


def run_reference(args):
    rank, local_rank, world = dist_env()
    if rank != 0:
        return
    w = workload()
    steps = max(1, min(args.steps, 2))
    warm = max(1, min(args.warmup, 3))
    res = cpu_baseline(w, pulses=steps, warmup=warm)
    line = {"impl": "reference", "metric": METRIC, "value": res["value"],
            "unit": "pulses/s", "n_gpus": world, "steps": steps,
            "warmup": warm, "ms_per_step": round(1e3 / res["value"], 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD},
            "cpu_baseline": res,
            "e2e": {"value": res["value"], "unit": "pulses/s",
                    "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "note": ("each step is one full oracle pulse (tens of seconds); steps "
                     "are capped at 2 and warm-up pulses at 3 so the run ends "
                     "within a few minutes")}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
