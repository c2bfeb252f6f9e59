#!/usr/bin/env python3
"""Benchmark of the Fourier-domain dedispersion path on GB300.

One step is the whole path over one batch of synthetic input resident in HBM:
unpack/transpose and chunking, channel R2C transforms (Eq. 3), the
phase-rotate-and-sum over channels for every trial DM (Eqs. 4, 7), the
inverse transforms with 1/L scaling (Eq. 6) and the valid-sample placement.

Default workload: survey-shaped plain FDD, one beam -- 1024 channels over
1210-1520 MHz, 64 us sampling, 2^20 uint8 samples (Gaussian mean 128, sigma 16,
clipped, five dispersed pulses), 2048 trials 0..1023.5 step 0.5, overlap-save
chunks of 2^18 samples, FP32 phasors and accumulation.

The metric counts DM x channel x bin phasor-MACs (8 flops each).  Prints one
JSON line.  ``--impl reference`` times the FP64 CPU oracle on a bounded sample
of the same workload instead (the reference arm of this benchmark).

Multi-GPU (torchrun): every rank processes its own beam of the same shape
(independent problems, no data-path collective): weak scaling.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "DM·channel·bin phasor-MACs/s and % of FP32/tensor peak, batched TC vs plain FP32"
UNIT = "phasor-MAC/s"
DEFAULT_WORKLOAD = "fdd_1024ch_2p20t_2048dm"
FLOPS_PER_MAC = 8
MAC_SOURCE = os.path.join(ROOT, "paper_2110_03482_gb300", "csrc", "fdd_mac_fp32.cu")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "mac_g12_survey_1024ch_2048dm.md")


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["fdd", "reference"], default="fdd")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(synth.WORKLOADS))
    ap.add_argument("--seed", type=int, default=20211007)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tc", action="store_true",
                    help="skip the tensor-core form's timing on the 32-beam workload")
    ap.add_argument("--no-tdd", action="store_true",
                    help="skip the brute-force time-domain dedispersion on the same workload")
    ap.add_argument("--sweep-window", type=int, default=0,
                    help="with --mac-sweep: time a window of this many bins in the middle of "
                         "the whole transform (fdd_dedisperse_spectra_bins) instead of all bins")
    ap.add_argument("--downsample-sweep", action="store_true",
                    help="time the workload's whole call at down-sampling factors 1, 2, 4, 8 "
                         "and print one JSON line per factor")
    ap.add_argument("--spin-sweep", action="store_true",
                    help="whole call in the FP32 form and with spin-frequency DM grids (FP16 "
                         "tensor cores, groups of 16 and 32 bins), with the grids' error")
    ap.add_argument("--spin-tol", type=float, default=0.01,
                    help="with --spin-sweep: the largest DM contraction within a group")
    ap.add_argument("--crossover", action="store_true",
                    help="time Fourier- and time-domain dedispersion of the workload at "
                         "128..n_dm trials (one JSON line per trial count)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="target wall time of the CPU-baseline sample")
    ap.add_argument("--n-t", type=int, default=0,
                    help="override samples per beam (smaller cases for profiler captures)")
    ap.add_argument("--n-dm", type=int, default=0,
                    help="override the workload's trial count (kernel sweeps)")
    ap.add_argument("--chunk-len", type=int, default=-1,
                    help="override the overlap-save chunk length")
    ap.add_argument("--mac-variant", type=int, default=0,
                    help="0 = automatic, else 1 + FDD_MAC_* kernel variant")
    ap.add_argument("--batch", default="",
                    help="time the batching form on a BATCH_WORKLOADS entry instead "
                         "(one JSON line)")
    ap.add_argument("--batch-precision", default="fp32",
                    choices=["fp32", "fp16", "bf16", "bf16_hilo", "fp8"],
                    help="with --batch: the FP32 form (persistent launch per wave) or a "
                         "tensor-core form (groups of beams sharing their phasors)")
    ap.add_argument("--batch-n-t-div", type=int, default=16,
                    help="divide the batch workload's beam lengths (device memory bound)")
    ap.add_argument("--precision", default="fp16", choices=["fp16", "bf16", "bf16_hilo", "fp8"],
                    help="tensor-core form of the multi-beam workloads")
    ap.add_argument("--workspace-gib", type=float, default=200.0,
                    help="device workspace limit of the multi-beam plans (GiB)")
    ap.add_argument("--mac-sweep", default="",
                    help="comma-separated FDD_MAC_* variants, by number or name, or tc / tc1 / tc16 / "
                         "tc8 for the tensor-core form in BF16 hi+lo / BF16 / FP16 / FP8 (or 'all'): "
                         "time the "
                         "phase-rotate-and-sum kernel alone for each on one chunk of the "
                         "workload and print one JSON line per variant")
    return ap.parse_args()


def workload_from_args(args) -> synth.Workload:
    w = synth.WORKLOADS[args.workload]
    kw = {}
    if args.n_t:
        kw["n_t"] = args.n_t
    if args.chunk_len >= 0:
        kw["chunk_len"] = args.chunk_len
    if args.n_dm:
        kw["n_dm"] = args.n_dm
    if kw:
        w = w.scaled(name=w.name + "_scaled", **kw)
    return w


# ------------------------------------------------------------------ helpers
def load_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def plan_params(w: synth.Workload, fdd) -> dict:
    return dict(n_chan=w.n_chan, nu_lo_mhz=w.nu_lo_mhz, dnu_mhz=w.dnu_mhz, t_samp_s=w.t_samp_s,
                n_t=w.n_t, dm_list=w.dms(), chunk_len=w.chunk_len, n_beams=1,
                in_dtype=fdd.FDD_IN_U8 if w.dtype == "u8" else fdd.FDD_IN_F32,
                output={"time": fdd.FDD_OUT_TIME, "spectra": fdd.FDD_OUT_SPECTRA,
                        "power": fdd.FDD_OUT_POWER}[w.output])


def workload_config(w: synth.Workload, info: dict | None) -> dict:
    cfg = {"workload": w.name, "n_chan": w.n_chan, "band_mhz": [w.band_lo_mhz, w.band_hi_mhz],
           "t_samp_s": w.t_samp_s, "n_t": w.n_t, "in_dtype": w.dtype, "n_dm": w.n_dm,
           "dm_range": [w.dm0, w.dm0 + w.ddm * (w.n_dm - 1)], "chunk_len": w.chunk_len,
           "beams_per_gpu": 1, "output": w.output,
           "l2": "no flush: inputs, spectra and outputs (GBs) exceed the 129 MB L2"}
    if info:
        cfg.update({"fft_len": info["fft_len"], "n_bins": info["n_bins"],
                    "n_chunks": info["n_chunks"], "d_max": info["d_max"]})
    return cfg


def macs_per_beam(w: synth.Workload, info: dict) -> int:
    return int(info["n_chunks"]) * w.n_dm * w.n_chan * int(info["n_bins"])


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_id: str):
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={gpu_id}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.flush()
        with open(self.tmp.name) as f:
            rows = [r.strip().split(",") for r in f if r.strip()]
        os.unlink(self.tmp.name)
        sm, mx, pw, reasons = [], [], [], set()
        for r in rows:
            if len(r) < 8:
                continue
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
                pw.append(float(r[2]))
            except ValueError:
                continue
            for name, v in zip(self.NAMES, r[4:8]):
                if v.strip() == "Active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def gpu_uuid(props, index: int) -> str:
    """nvidia-smi --id for a torch device (its UUID when torch exposes one)."""
    u = str(getattr(props, "uuid", "") or "")
    if not u:
        return str(index)
    return u if u.startswith("GPU-") else "GPU-" + u


def read_traffic_summary() -> float | None:
    """Per-launch DRAM bytes of the MAC kernel from the committed ncu summary,
    only if that summary was taken on the current kernel source."""
    try:
        with open(TRAFFIC_FILE) as f:
            text = f.read()
        with open(MAC_SOURCE, "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
    except OSError:
        return None
    m_sha = re.search(r"kernel_source_sha256:\s*([0-9a-f]{64})", text)
    m_b = re.search(r"dram_bytes_per_launch_full:\s*([0-9.eE+]+)", text)
    if not m_sha or not m_b or m_sha.group(1) != sha:
        return None
    return float(m_b.group(1))


# ------------------------------------------------------------------ CPU legs
def oracle_sample_setup(w: synth.Workload, seed: int):
    """Spectra of chunk 0 (all channels) by the oracle FFT, outside any timing."""
    import oracle
    d = oracle.delays(w.channel_centres(), w.dms(), w.t_samp_s)
    geo = oracle.geometry(w.n_t, w.chunk_len, d)
    fb, _ = synth.filterbank(w, seed=seed, rows=geo.L)
    X = oracle.spectra(fb.T.astype(np.float64), geo, 0)
    return d, geo, X


def oracle_rate(d, geo, X, n_bins: int, rng: np.random.Generator):
    """Time the oracle's phase-rotate-and-sum on n_bins sampled bins x all DMs x all
    channels; returns (MACs, seconds)."""
    import oracle
    fixed = [0, 1, geo.K - 1]
    extra = rng.choice(np.arange(2, geo.K - 1), size=max(0, n_bins - 3), replace=False)
    bins = np.unique(np.concatenate([fixed, extra]).astype(np.int64))
    t0 = time.perf_counter()
    Y = oracle.fdd_bins(X[:, bins], bins, geo.L, d)
    dt = time.perf_counter() - t0
    oracle_rate.last = (bins, Y)
    return d.shape[0] * d.shape[1] * bins.size, dt


def _gpu_sampled(plan, X, bins, n_dm, pitch):
    """The CUDA path's spectra of the given bins, from complex spectra X [series][chan][K]."""
    import torch
    ns, nc, K = X.shape
    host = np.zeros((ns, nc, pitch, 2), dtype=np.float32)
    host[..., :K, 0] = X.real
    host[..., :K, 1] = X.imag
    dX = torch.from_numpy(host).cuda()
    dY = torch.empty((ns, n_dm, K, 2), device="cuda")
    plan.dedisperse_spectra(dX, pitch, ns, 0, n_dm, dY, K)
    out = dY.index_select(2, torch.from_numpy(bins).cuda()).cpu().numpy().astype(np.float64)
    del dX, dY
    return out[..., 0] + 1j * out[..., 1]


def _rel(a, b) -> float:
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def oracle_small_full() -> dict:
    """The oracle's whole path (delays, FFT, Eq. 7 over every bin, inverse) on
    the complete 64-channel workload, timed once."""
    import oracle
    w = synth.WORKLOADS["fdd_64ch_4096t_128dm"]
    fb, _ = synth.filterbank(w, seed=20211008)
    t0 = time.perf_counter()
    d = oracle.delays(w.channel_centres(), w.dms(), w.t_samp_s)
    oracle.fdd_time(fb.T.astype(np.float64), d, w.chunk_len)
    dt = time.perf_counter() - t0
    K = w.n_t // 2 + 1
    return {"workload": w.name, "seconds": dt,
            "macs_per_s": w.n_dm * w.n_chan * K / dt,
            "note": "whole oracle path on the complete workload (not a sample)"}


def cpu_baseline(w: synth.Workload, seed: int, target_s: float, plan=None,
                 macs_step: int | None = None) -> dict:
    """Time the oracle on sampled bins; when a plan is given, also report the CUDA
    path's relative L2 error on those bins (same FP64-derived spectra in)."""
    import oracle
    d, geo, X = oracle_sample_setup(w, seed)
    rng = np.random.default_rng(seed)
    macs, dt = oracle_rate(d, geo, X, 16, rng)
    nb = int(min(geo.K, max(16, 16 * target_s / max(dt, 1e-3))))
    macs, dt = oracle_rate(d, geo, X, nb, rng)
    out = {"value": macs / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
           "sample": f"FP64 oracle phase-rotate-and-sum of {nb} sampled bins (incl. DC, 1, "
                     f"Nyquist) x {w.n_dm} DMs x {w.n_chan} channels of chunk 0 "
                     f"({macs:.3g} MACs in {dt:.1f} s; oracle FFT of the chunk untimed)",
           "seconds": dt}
    if macs_step:
        # labelled as an extrapolation: the sampled rate applied to a whole step
        out["extrapolated_seconds_per_step"] = macs_step / (macs / dt)
    out["small_full"] = oracle_small_full()
    if plan is not None:
        bins, Y = oracle_rate.last
        G = _gpu_sampled(plan, X[None].astype(np.complex64), bins, w.n_dm,
                         plan.info["bin_pitch"])[0]
        out["gpu_rel_l2_vs_oracle"] = _rel(G, Y)
        out["gpu_rel_l2_vs_oracle_no_dc"] = _rel(G[:, bins > 0], Y[:, bins > 0])
    return out


TC_WORKLOAD = "fdd_32beam_1024ch_2p19t_4096dm"
TC_N_T = 4096  # 2049 bins: a bounded slice of the 32-beam workload


def tc_accuracy(seed: int) -> dict:
    """Relative L2 error of both tensor-core precisions vs the FP64 oracle on 8
    sampled bins of 2 beams (all 4096 trials, 1024 channels)."""
    import oracle
    import paper_2110_03482_gb300 as fdd
    w = synth.WORKLOADS[TC_WORKLOAD].scaled(n_t=TC_N_T)
    d = oracle.delays(w.channel_centres(), w.dms(), w.t_samp_s)
    geo = oracle.geometry(w.n_t, w.chunk_len, d)
    rng = np.random.default_rng(seed)
    X = (rng.standard_normal((2, w.n_chan, geo.K)) +
         1j * rng.standard_normal((2, w.n_chan, geo.K))).astype(np.complex64)
    bins = np.unique(np.concatenate([[0, 1, geo.K - 1], rng.integers(2, geo.K - 1, 5)]))
    refs = np.stack([oracle.fdd_bins(X[b][:, bins].astype(np.complex128), bins, geo.L, d)
                     for b in range(2)])
    res = {}
    for name, prec in (("bf16_hilo", fdd.FDD_PREC_BF16_HILO), ("bf16", fdd.FDD_PREC_BF16),
                       ("fp16", fdd.FDD_PREC_FP16)):
        with fdd.Plan(**dict(plan_params(w, fdd), output=fdd.FDD_OUT_SPECTRA, n_beams=2,
                             precision=prec)) as plan:
            G = _gpu_sampled(plan, X, bins, w.n_dm, plan.info["bin_pitch"])
        res[name] = _rel(G, refs)
    return {"rel_l2_vs_oracle": res,
            "sample": f"8 bins x {w.n_dm} DMs x {w.n_chan} channels x 2 beams"}


def run_reference(args, rank: int, world: int) -> None:
    if rank != 0:
        return
    import oracle
    w = workload_from_args(args)
    d, geo, X = oracle_sample_setup(w, args.seed)
    rng = np.random.default_rng(args.seed)
    nb = 64
    for _ in range(args.warmup):
        oracle_rate(d, geo, X, nb, rng)
    tot_macs, tot_s = 0, 0.0
    for _ in range(args.steps):
        m, s = oracle_rate(d, geo, X, nb, rng)
        tot_macs += m
        tot_s += s
    value = tot_macs / tot_s
    sample = (f"each step: FP64 oracle phase-rotate-and-sum of {nb} sampled bins x {w.n_dm} DMs x "
              f"{w.n_chan} channels of chunk 0 ({tot_macs // args.steps:.3g} MACs)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded survey-shaped filterbank)",
            "config": workload_config(w, None),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU leg
def measure_tc(args, fdd, torch, value_per_mac_kernel: float) -> dict:
    """Kernel-only timing of the tensor-core form (both precisions) on a bounded
    slice of the 32-beam workload: 32 beams x 1024 channels x 2049 bins x 4096
    trials per launch (random spectra; every output written)."""
    w = synth.WORKLOADS[TC_WORKLOAD].scaled(n_t=TC_N_T)
    peaks = load_peaks()
    bf16_peak = float(peaks.get("bf16_tflops") or 1895.5)
    res = {"workload": f"{TC_WORKLOAD} slice: {w.n_beams} beams x {w.n_chan} channels x "
                       f"{TC_N_T // 2 + 1} bins x {w.n_dm} trials",
           "unit": UNIT}
    X = Y = None
    for name, prec, passes in (("bf16_hilo", fdd.FDD_PREC_BF16_HILO, 2),
                               ("bf16", fdd.FDD_PREC_BF16, 1),
                               ("fp16", fdd.FDD_PREC_FP16, 1)):
        with fdd.Plan(**dict(plan_params(w, fdd), output=fdd.FDD_OUT_SPECTRA,
                             n_beams=w.n_beams, precision=prec)) as plan:
            g = plan.info
            if X is None:
                gen = torch.Generator(device="cuda").manual_seed(args.seed)
                X = torch.randn((w.n_beams, w.n_chan, g["bin_pitch"], 2), device="cuda",
                                generator=gen)
                Y = torch.empty((w.n_beams, w.n_dm, g["n_bins"], 2), device="cuda")
            call = lambda: plan.dedisperse_spectra(X, g["bin_pitch"], w.n_beams, 0, w.n_dm, Y,
                                                   g["n_bins"])
            call()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(3):
                call()
            e1.record()
            torch.cuda.synchronize()
            plan.query()
            ms = e0.elapsed_time(e1) / 3
        macs = w.n_beams * w.n_dm * w.n_chan * g["n_bins"]
        tf = FLOPS_PER_MAC * macs / (ms / 1e3) / 1e12
        res[name] = {"value": macs / (ms / 1e3), "ms_per_launch": ms, "tflops_algorithmic": tf,
                     "tflops_tensor_physical": passes * tf,
                     "frac_bf16_peak_physical": passes * tf / bf16_peak,
                     "speedup_vs_fp32_kernel": tf / value_per_mac_kernel}
    del X, Y
    return res


def max_over_ranks(dist, ms: float, device: str) -> float:
    """The job's time: the largest of every rank's (the slowest rank ends it)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank_step: float, steps: int, world: int, ms_max: float) -> float:
    """Whole-job throughput: the units every rank processed over the job's time
    (weak scaling: each rank dedisperses its own beam of the same shape)."""
    return units_per_rank_step * steps * world / (ms_max / 1e3)


TDD_SMEM_ADDS_PER_CLK = 32  # one 4-byte shared load per add, 128 B per clock per SM


def measure_tdd(plan, w, info, d_in, stream, torch, sm_count, fdd_ms_per_step, reps=3) -> dict:
    """Brute-force time-domain dedispersion (Eq. 2) of the same beam with the
    same plan: whole call (unpack + shift-and-sum), CUDA events."""
    out_len = w.n_t - info["d_max"]
    y = torch.empty((w.n_dm, out_len), dtype=torch.float32, device="cuda")
    plan.tdd_execute(d_in, y, stream)
    torch.cuda.synchronize()
    plan.profile_enable(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        plan.tdd_execute(d_in, y, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    prof = plan.profile_read()
    plan.profile_enable(False)
    ms = e0.elapsed_time(e1) / reps
    kernel_ms = prof["ms"]["tdd"] / max(prof["launches"]["tdd"], 1)
    adds = w.n_dm * w.n_chan * out_len
    peak = TDD_SMEM_ADDS_PER_CLK * sm_count * float(load_peaks().get("sm_max_mhz") or 2070) * 1e6
    del y
    return {"method": "brute-force time-domain shift-and-sum (Eq. 2), same workload",
            "ms_per_step": ms, "kernel_ms": kernel_ms,
            "adds_per_s_kernel": adds / (kernel_ms / 1e3),
            "frac_smem_bound": adds / (kernel_ms / 1e3) / peak,
            "bound": f"shared memory: {TDD_SMEM_ADDS_PER_CLK} adds (4-byte loads) per clock per SM",
            "output_samples_per_trial": out_len,
            "fdd_over_tdd_time": fdd_ms_per_step / ms}


def run_crossover(args) -> None:
    """Fourier-domain (this library's default path) against brute-force
    time-domain dedispersion on the workload's shape at 128, 256, .. n_dm
    trials of the same grid (the comparison of Sect. 4)."""
    import torch

    import paper_2110_03482_gb300 as fdd

    fdd.build()
    w0 = workload_from_args(args)
    fb, _ = synth.filterbank(w0, seed=args.seed)
    d_in = torch.from_numpy(fb.reshape(-1)).cuda()
    stream = torch.cuda.current_stream()
    n = 128
    while n <= w0.n_dm:
        w = w0.scaled(n_dm=n)
        with fdd.Plan(**plan_params(w, fdd)) as plan:
            info = plan.info
            out = torch.empty(info["out_elems"], dtype=torch.float32, device="cuda")
            y = torch.empty((n, w.n_t - info["d_max"]), dtype=torch.float32, device="cuda")
            res = {}
            for name, call in (("fdd", lambda: plan.execute(d_in, out, stream)),
                               ("tdd", lambda: plan.tdd_execute(d_in, y, stream))):
                for _ in range(max(args.warmup, 1)):
                    call()
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(args.steps):
                    call()
                e1.record(stream)
                torch.cuda.synchronize()
                res[name] = e0.elapsed_time(e1) / args.steps
            print(json.dumps({"crossover": w0.name, "n_dm": n, "fdd_ms": res["fdd"],
                              "tdd_ms": res["tdd"], "tdd_over_fdd_time": res["tdd"] / res["fdd"],
                              "fdd_tile": fdd.MAC_VARIANT_NAMES[info["mac_variant"]],
                              "fft_len": info["fft_len"], "n_chunks": info["n_chunks"]}),
                  flush=True)
            del out, y
        n *= 2


def run_downsample_sweep(args) -> None:
    """The workload's whole call (unpack, R2C, MAC, C2R, scatter) at
    down-sampling factors 1, 2, 4, 8 (Sect. 2.2, last paragraph: the MAC on
    the bins k <= L / 2f only and an inverse transform of length L / f), one
    JSON line per factor with the MACs the call actually does."""
    import torch

    import paper_2110_03482_gb300 as fdd

    fdd.build()
    w = workload_from_args(args)
    fb, _ = synth.filterbank(w, seed=args.seed)
    d_in = torch.from_numpy(fb.reshape(-1)).cuda()
    stream = torch.cuda.current_stream()
    ms1 = None
    for f in (1, 2, 4, 8):
        with fdd.Plan(**dict(plan_params(w, fdd), downsample=f)) as plan:
            info = plan.info
            out = torch.empty(info["out_elems"], dtype=torch.float32, device="cuda")
            for _ in range(max(args.warmup, 1)):
                plan.execute(d_in, out, stream)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                plan.execute(d_in, out, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            ms1 = ms if ms1 is None else ms1
            bins = info["fft_len"] // f // 2 + 1
            macs = int(info["n_chunks"]) * w.n_dm * w.n_chan * bins
            print(json.dumps({"downsample": f, "workload": w.name, "ms_per_call": ms,
                              "out_len": info["out_len"], "mac_bins_per_chunk": bins,
                              "macs_per_s": macs / (ms / 1e3), "time_over_f1": ms / ms1,
                              "tile": fdd.MAC_VARIANT_NAMES[info["mac_variant"]]}), flush=True)
            del out


def run_spin_sweep(args) -> None:
    """The workload's whole call (time output) in the FP32 form and with the
    spin-frequency-dependent DM grids on FP16 tensor cores (Sect. 2.3; groups
    of 16 and 32 bins at the given contraction tolerance), one JSON line
    each, with the spin form's rel-L2 on sampled bins of chunk 0 against
    Eq. 7 (the oracle's exact sum) and against the oracle's restatement of
    the same approximation."""
    import torch

    import oracle
    import paper_2110_03482_gb300 as fdd

    fdd.build()
    w = workload_from_args(args)
    fb, _ = synth.filterbank(w, seed=args.seed)
    d_in = torch.from_numpy(fb.reshape(-1)).cuda()
    stream = torch.cuda.current_stream()
    d, geo, X = oracle_sample_setup(w, args.seed)
    rng = np.random.default_rng(args.seed)
    bins = np.unique(np.concatenate([[1, geo.K // 2, geo.K - 1], rng.integers(2, geo.K - 1, 29)]))
    ref = oracle.fdd_bins(X[:, bins], bins, geo.L, d)
    ms_fp32 = None
    for G in (0, 16, 32):
        kw = dict(plan_params(w, fdd))
        if G:
            kw.update(precision=fdd.FDD_PREC_FP16, spin_group=G, spin_tol=args.spin_tol)
        with fdd.Plan(**kw) as plan:
            info = plan.info
            out = torch.empty(info["out_elems"], dtype=torch.float32, device="cuda")
            for _ in range(max(args.warmup, 1)):
                plan.execute(d_in, out, stream)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                plan.execute(d_in, out, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            del out
        ms_fp32 = ms if G == 0 else ms_fp32
        line = {"spin_group": G, "workload": w.name, "ms_per_call": ms,
                "macs_per_s": macs_per_beam(w, info) / (ms / 1e3),
                "speedup_vs_fp32": ms_fp32 / ms}
        if G:
            # the dedispersed spectra of chunk 0 at the sampled bins
            with fdd.Plan(**dict(kw, output=fdd.FDD_OUT_SPECTRA)) as plan:
                sp = torch.empty(plan.info["out_elems"] * 2, dtype=torch.float32, device="cuda")
                plan.execute(d_in, sp, stream)
                torch.cuda.synchronize()
                Y = sp.view(-1, 2)[: w.n_dm * geo.K].view(w.n_dm, geo.K, 2)
                Yb = Y[:, torch.from_numpy(bins).cuda()].cpu().numpy().astype(np.float64)
                got = Yb[..., 0] + 1j * Yb[..., 1]
                del sp, Y
            appr = oracle.fdd_bins_spin(X[:, bins], bins, geo.L, w.channel_centres(), w.dm0,
                                        w.ddm, w.n_dm, w.t_samp_s, G, args.spin_tol)
            line.update(spin_k_min=info["spin_k_min"], spin_tol=args.spin_tol,
                        rel_l2_vs_eq7=_rel(got, ref), rel_l2_vs_restatement=_rel(got, appr),
                        restatement_vs_eq7=_rel(appr, ref),
                        sample=f"{bins.size} bins of chunk 0 (1, K/2, Nyquist, random), "
                               f"all {w.n_dm} trials")
        print(json.dumps(line), flush=True)


def run_fdd(args, rank: int, world: int, dist) -> None:
    import torch

    import paper_2110_03482_gb300 as fdd

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    fdd.build()
    w = workload_from_args(args)
    props = torch.cuda.get_device_properties(local)
    sm_count = props.multi_processor_count
    gpu_id = gpu_uuid(props, local)

    fb, _ = synth.filterbank(w, seed=args.seed, beam=rank)
    plan = fdd.Plan(**plan_params(w, fdd), mac_variant=args.mac_variant)
    info = plan.info
    stream = torch.cuda.current_stream()
    d_in = torch.from_numpy(fb.reshape(-1)).cuda()
    out_dtype = torch.float32
    n_out = info["out_elems"] * (2 if w.output == "spectra" else 1)
    d_out = torch.empty(n_out, dtype=out_dtype, device="cuda")
    macs_step = macs_per_beam(w, info)

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(max(args.warmup, 0)):
        plan.execute(d_in, d_out, stream)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()

    plan.profile_enable(True)
    clocks = Clocks(gpu_id)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        plan.execute(d_in, d_out, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier()
    ms = e0.elapsed_time(e1)
    prof = plan.profile_read()
    plan.profile_enable(False)

    ms_max = max_over_ranks(dist, ms, "cuda")
    value = job_rate(macs_step, args.steps, world, ms_max)

    # dominant kernel: the phasor-MAC
    mac_n = prof["launches"]["mac"]
    mac_ms = prof["ms"]["mac"] / max(mac_n, 1)
    flops_launch = FLOPS_PER_MAC * min(info["dm_batch"], w.n_dm) * w.n_chan * info["n_bins"]
    achieved = flops_launch / (mac_ms / 1e3) / 1e12
    peaks = load_peaks()
    max_mhz = float(peaks.get("sm_max_mhz") or clk.get("sm_max_mhz") or 2070.0)
    peak = sm_count * 128 * 2 * max_mhz * 1e6 / 1e12
    traffic = read_traffic_summary()
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": "phase-rotate-and-sum (Eqs. 4 and 7), variant "
                          + fdd.MAC_VARIANT_NAMES[info["mac_variant"]],
                "peak_source": f"derived: {sm_count} SMs x 128 FP32 lanes x 2 flop x "
                               f"{max_mhz:.0f} MHz max SM clock (FP32 FFMA; "
                               "MEASURED_PEAKS.json has no FP32 figure)",
                "algorithmic_flops_per_launch": flops_launch,
                "mac_ms_per_launch": mac_ms, "mac_launches_timed": mac_n}
    if clk.get("sm_mhz"):
        roofline["frac_at_sampled_clock"] = achieved / (peak * clk["sm_mhz"] / max_mhz)
    stage_share = {k: v / max(sum(prof["ms"].values()), 1e-9) for k, v in prof["ms"].items()}
    own_launches = prof["kernels"]

    # end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        h_in = torch.from_numpy(fb.reshape(-1)).pin_memory()
        h_out = torch.empty(n_out, dtype=out_dtype, pin_memory=True)
        plan.execute_host(h_in, h_out, stream)
        torch.cuda.synchronize()
        barrier()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.e2e_steps):
            plan.execute_host(h_in, h_out, stream)
        f1.record(stream)
        torch.cuda.synchronize()
        e_ms = max_over_ranks(dist, f0.elapsed_time(f1), "cuda")
        e2e = {"value": job_rate(macs_step, args.e2e_steps, world, e_ms), "unit": UNIT,
               "h2d_bytes_per_step": int(h_in.numel() * h_in.element_size()),
               "d2h_bytes_per_step": int(h_out.numel() * h_out.element_size()),
               "ms_per_step": e_ms / args.e2e_steps}
        del h_in, h_out

    tdd = None
    if not args.no_tdd and world == 1:
        tdd = measure_tdd(plan, w, info, d_in, stream, torch, sm_count,
                          fdd_ms_per_step=ms_max / args.steps)
    tc = None if args.no_tc else measure_tc(args, fdd, torch, value_per_mac_kernel=achieved)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, args.seed, args.cpu_seconds, plan, macs_step=macs_step)
        if tc is not None:
            tc.update(tc_accuracy(args.seed))
    plan.close()

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic (seeded survey-shaped filterbank)",
                "config": dict(workload_config(w, info), parallelism=f"beam-replicas x{world}"),
                "gpu_launches": own_launches,
                "clocks": clk, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "tc": tc,
                "tdd": tdd,
                "stage_ms_share": stage_share,
                "fp32_frac_whole_step": value * FLOPS_PER_MAC / 1e12 / (peak * world),
                "macs_per_step": macs_step * world}
        print(json.dumps(line), flush=True)


def run_mac_sweep(args) -> None:
    """Kernel-only timing of phase-rotate-and-sum variants on one chunk's spectra."""
    import torch

    import paper_2110_03482_gb300 as fdd

    fdd.build()
    w = workload_from_args(args)
    tc_prec = {"tc": fdd.FDD_PREC_BF16_HILO, "tc1": fdd.FDD_PREC_BF16,
               "tc16": fdd.FDD_PREC_FP16, "tc8": fdd.FDD_PREC_FP8}

    def variant(v: str):
        if v in tc_prec:
            return v
        return fdd.MAC_VARIANT_NAMES.index(v) if v in fdd.MAC_VARIANT_NAMES else int(v)

    vs = list(range(fdd.FDD_MAC_VARIANTS)) if args.mac_sweep == "all" else \
        [variant(v) for v in args.mac_sweep.split(",")]
    props = torch.cuda.get_device_properties(0)
    peaks = load_peaks()
    max_mhz = float(peaks.get("sm_max_mhz") or 2070.0)
    peak = props.multi_processor_count * 128 * 2 * max_mhz * 1e6 / 1e12
    g = None
    X = Y = None
    bf16_peak = float(peaks.get("bf16_tflops") or 1895.5)
    for v in vs:
        tc = v in tc_prec
        ns = w.n_beams if tc else 1
        kw = dict(plan_params(w, fdd), output=fdd.FDD_OUT_SPECTRA)
        if tc:
            kw.update(precision=tc_prec[v], n_beams=ns,
                      workspace_limit=int(args.workspace_gib * (1 << 30)))
        else:
            kw.update(mac_variant=v + 1)
        with fdd.Plan(**kw) as plan:
            g = plan.info
            # the whole transform's bins, or (--sweep-window N) a window of N bins
            # in its middle through fdd_dedisperse_spectra_bins
            nb = min(args.sweep_window, g["n_bins"]) if args.sweep_window > 0 else g["n_bins"]
            b0 = (g["n_bins"] - nb) // 2 if args.sweep_window > 0 else 0
            pitch = nb if args.sweep_window > 0 else g["bin_pitch"]
            if X is None or X.shape[0] != ns:
                X = Y = None
                gen = torch.Generator(device="cuda").manual_seed(args.seed)
                X = torch.randn((ns, w.n_chan, pitch, 2), device="cuda", generator=gen)
                Y = torch.empty((ns, w.n_dm, nb, 2), device="cuda")

            def call():
                if args.sweep_window > 0:
                    plan.dedisperse_spectra_bins(X, pitch, ns, b0, nb, 0, w.n_dm, Y, nb)
                else:
                    plan.dedisperse_spectra(X, pitch, ns, 0, w.n_dm, Y, nb)

            for _ in range(max(args.warmup, 1)):
                call()
            torch.cuda.synchronize()
            clocks = Clocks(gpu_uuid(props, 0))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.steps):
                call()
            e1.record()
            torch.cuda.synchronize()
            clk = clocks.stop()
            ms = e0.elapsed_time(e1) / args.steps
            plan.query()  # raises if a kernel reported a device-side timeout
        flops = FLOPS_PER_MAC * ns * w.n_dm * w.n_chan * nb
        tf = flops / (ms / 1e3) / 1e12
        extra = {"frac_bf16_peak_algorithmic": tf / bf16_peak,
                 "tensor_tflops_physical": (2 if v == "tc" else 1) * tf} if tc else {}
        print(json.dumps({"sweep": {"tc": "TC_hilo", "tc1": "TC_bf16",
                                    "tc16": "TC_fp16", "tc8": "TC_fp8"}.get(v, None) or
                          fdd.MAC_VARIANT_NAMES[v], "variant": v,
                          "ms_per_launch": ms, "beams": ns, "macs_per_s": tf * 1e12 / 8,
                          "tflops": tf, "frac_fp32_peak": tf / peak, "workload": w.name,
                          **extra,
                          "sm_mhz": clk.get("sm_mhz"), "reasons": clk.get("reasons"),
                          "n_bins": nb, "bin_window_start": b0, "n_dm": w.n_dm,
                          "n_chan": w.n_chan}),
              flush=True)


TC_PREC = {"fp16": 3, "bf16": 2, "bf16_hilo": 1, "fp8": 4}  # FDD_PREC_* of the tensor-core forms
RESIDENT_INPUT_BYTES = 100 << 30  # larger inputs stream from the generator


def tc_workload_accuracy(fdd, w: synth.Workload, prec: int, seed: int, beams) -> dict:
    """rel-L2 of the tensor-core form against the FP64 oracle on sampled bins of
    the workload's own first chunk (beam 0: the counter-based input, made on
    the device and copied back; oracle FFT of every channel), all trials."""
    import torch

    import oracle
    d = oracle.delays(w.channel_centres(), w.dms(), w.t_samp_s)
    geo = oracle.geometry(w.n_t, w.chunk_len, d)
    rows = min(geo.L, w.n_t)
    buf = torch.empty(rows * w.n_chan, dtype=torch.float32, device="cuda")
    beams.fill(0, buf.data_ptr(), 0, rows, torch.cuda.current_stream().cuda_stream)
    fb = buf.cpu().numpy().reshape(rows, w.n_chan)
    del buf
    X = oracle.spectra(fb.T.astype(np.float64), geo, 0)
    rng = np.random.default_rng(seed)
    bins = np.unique(np.concatenate([[0, 1, geo.K - 1], rng.integers(2, geo.K - 1, 5)]))
    ref = oracle.fdd_bins(X[:, bins], bins, geo.L, d)
    res = {"by_form": {}}
    nb = bins.size
    host = np.zeros((1, w.n_chan, nb, 2), dtype=np.float32)
    Xs = X[:, bins].astype(np.complex64)
    host[0, :, :, 0] = Xs.real
    host[0, :, :, 1] = Xs.imag
    dX = torch.from_numpy(host).cuda()
    for name, pr in sorted(TC_PREC.items(), key=lambda kv: kv[1] != prec):
        with fdd.Plan(**dict(plan_params(w, fdd), output=fdd.FDD_OUT_SPECTRA, n_beams=1,
                             precision=pr, workspace_limit=8 << 30)) as plan:
            got = np.zeros((w.n_dm, nb), dtype=np.complex128)
            for q, k in enumerate(bins):  # bin windows of one bin (absolute phases)
                dY = torch.empty((1, w.n_dm, 1, 2), device="cuda")
                plan.dedisperse_spectra_bins(dX[:, :, q:q + 1].contiguous(), 1, 1, int(k), 1, 0,
                                             w.n_dm, dY, 1)
                y = dY.cpu().numpy().astype(np.float64)[0, :, 0]
                got[:, q] = y[:, 0] + 1j * y[:, 1]
        res["by_form"][name] = {"rel_l2_vs_oracle": _rel(got, ref),
                                "rel_l2_vs_oracle_no_dc": _rel(got[:, bins > 0], ref[:, bins > 0])}
        if pr == prec:
            res.update(res["by_form"][name])
    res["sample"] = (f"beam 0, chunk 0: {bins.size} bins (DC, 1, Nyquist, 5 random) x "
                     f"{w.n_dm} trials x {w.n_chan} channels, oracle FFT spectra in; every "
                     "tensor-core form")
    return res


def run_tc_workload(args) -> None:
    """A multi-beam workload on the tensor-core form (beams share every bin's
    phasors), streamed: whole input resident on the device when it fits,
    else each (beam, chunk) window generated on the device by the
    counter-based generator; output blocks handed to a sink that reads them
    (``value``: device line, sink discards), or copied to a pinned host ring
    (``e2e``: host input windows in, every output block back to the host)."""
    import ctypes

    import torch

    import paper_2110_03482_gb300 as fdd
    import synth.gpu

    fdd.build()
    synth.gpu.build()
    w = workload_from_args(args)
    prec = TC_PREC[args.precision]
    props = torch.cuda.get_device_properties(0)
    gpu_id = gpu_uuid(props, 0)
    stream = torch.cuda.current_stream()
    s_handle = stream.cuda_stream
    params = dict(plan_params(w, fdd), n_beams=w.n_beams, precision=prec,
                  workspace_limit=int(args.workspace_gib * (1 << 30)))
    esz = 1 if w.dtype == "u8" else 4
    in_bytes = w.n_beams * w.n_t * w.n_chan * esz
    beams = synth.gpu.BeamWindows([synth.philox_beam_args(w, args.seed, b)[0]
                                   for b in range(w.n_beams)])
    t_plan = time.perf_counter()
    plan = fdd.Plan(**params)
    plan_s = time.perf_counter() - t_plan
    info = plan.info
    resident = in_bytes <= RESIDENT_INPUT_BYTES
    d_in = None
    if resident:
        d_in = torch.empty(in_bytes, dtype=torch.uint8, device="cuda")
        for b in range(w.n_beams):
            beams.fill(b, d_in.data_ptr() + b * w.n_t * w.n_chan * esz, 0, w.n_t, s_handle)
        stream.synchronize()
    out_esz = 4 if w.output in ("time", "power") else 8
    out_bytes = int(info["out_bytes"])
    blocks = [0, 0]

    def source(beam, t0, n, d_window, ready, s):  # stream-ordered on s
        beams.fill(beam, d_window, t0, n, s)

    def sink(blk, s):  # the device line consumes nothing: count what arrived
        blocks[0] += 1
        blocks[1] += blk["n_beams"] * blk["n_dm"] * blk["row_len"] * out_esz
        return None

    def step():
        if resident:
            plan.execute_stream(None, sink, stream, d_in=d_in)
        else:
            plan.execute_stream(source, sink, stream)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    plan.profile_enable(True)
    clocks = Clocks(gpu_id)
    blocks[:] = [0, 0]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    prof = plan.profile_read()
    plan.profile_enable(False)
    plan.query()  # raises if a kernel reported a device-side timeout
    macs_step = w.n_beams * int(info["n_chunks"]) * w.n_dm * w.n_chan * int(info["n_bins"])
    value = macs_step * args.steps / (ms / 1e3)
    mac_n = prof["launches"]["mac"]
    mac_ms = prof["ms"]["mac"] / max(mac_n, 1)
    macs_launch = macs_step / max(mac_n / args.steps, 1)
    achieved = FLOPS_PER_MAC * macs_launch / (mac_ms / 1e3) / 1e12
    peaks = load_peaks()
    peak = float(peaks.get("bf16_tflops_sustained") or 1723.8)
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "kernel": f"tensor-core phase-rotate-and-sum ({args.precision}), per-bin "
                          "maxima pass and bin-major output included",
                "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (measured; FP16 "
                               "and BF16 dense rates are equal, nominal ratio 1)",
                "algorithmic_flops_per_launch": FLOPS_PER_MAC * macs_launch,
                "mac_ms_per_launch": mac_ms, "mac_launches_timed": mac_n}
    if args.precision == "bf16_hilo":
        roofline["tensor_frac_physical"] = 2 * achieved / peak
    stage_share = {k: v / max(sum(prof["ms"].values()), 1e-9) for k, v in prof["ms"].items()}

    # end to end: pinned host input (or a pool of generated windows when the
    # input exceeds host memory), every output block back to a pinned host ring
    e2e = None
    if not args.no_e2e:
        rt = fdd.cudart()
        vp = ctypes.c_void_p
        rt.cudaEventCreateWithFlags.argtypes = [ctypes.POINTER(vp), ctypes.c_uint]
        rt.cudaEventRecord.argtypes = [vp, vp]
        rt.cudaStreamWaitEvent.argtypes = [vp, vp, ctypes.c_uint]
        rt.cudaEventDestroy.argtypes = [vp]

        def new_event():
            e = vp()
            rt.cudaEventCreateWithFlags(ctypes.byref(e), 2)
            return e.value
        rt.cudaHostAlloc.argtypes = [ctypes.POINTER(vp), ctypes.c_size_t, ctypes.c_uint]
        rt.cudaFreeHost.argtypes = [vp]

        def host_pinned(nbytes):  # page-locked, released explicitly below
            p = vp()
            if rt.cudaHostAlloc(ctypes.byref(p), nbytes, 0) != 0:
                raise RuntimeError(f"cudaHostAlloc of {nbytes} bytes failed")
            return p.value
        h2d, d2h = torch.cuda.Stream(), torch.cuda.Stream()
        win_bytes = w.n_chan * int(info["fft_len"]) * esz
        if resident:
            h_in_ptr = host_pinned(in_bytes)
            fdd.memcpy_async(h_in_ptr, d_in.data_ptr(), in_bytes, s_handle)
            stream.synchronize()
            pool = None
        else:
            pool = 2  # distinct generated windows, reused cyclically
            h_in_ptr = host_pinned(pool * win_bytes)
            tmp = torch.empty(win_bytes, dtype=torch.uint8, device="cuda")
            for i in range(pool):
                beams.fill(i % w.n_beams, tmp.data_ptr(), 0,
                           min(int(info["fft_len"]), w.n_t), s_handle)
                fdd.memcpy_async(h_in_ptr + i * win_bytes, tmp.data_ptr(), win_bytes, s_handle)
                stream.synchronize()
            del tmp
        blk_max = max(1, int(info["stream_bytes"]) // 2 - win_bytes)
        # one host slot: the copies back run in order on one stream, and the
        # host keeps nothing of a block once the next one arrives
        ring_ptr = host_pinned(blk_max)
        ev_pool = [new_event() for _ in range(8)]
        state = {"win": 0, "blk": 0, "h2d": 0, "d2h": 0}

        def host_source(beam, t0, n, d_window, ready, s):
            e_full = ev_pool[state["win"] % 2]
            if ready:
                rt.cudaStreamWaitEvent(h2d.cuda_stream, ready, 0)
            nbytes = n * w.n_chan * esz
            if pool is None:
                src = h_in_ptr + (beam * w.n_t + t0) * w.n_chan * esz
            else:
                src = h_in_ptr + (state["win"] % pool) * win_bytes
            fdd.memcpy_async(d_window, src, nbytes, h2d.cuda_stream)
            rt.cudaEventRecord(e_full, h2d.cuda_stream)
            rt.cudaStreamWaitEvent(s, e_full, 0)
            state["win"] += 1
            state["h2d"] += nbytes

        def host_sink(blk, s):
            k = state["blk"] % 2
            e_done, e_rel = ev_pool[2 + k], ev_pool[4 + k]
            rt.cudaEventRecord(e_done, s)
            rt.cudaStreamWaitEvent(d2h.cuda_stream, e_done, 0)
            rows = blk["n_beams"] * blk["n_dm"]
            width = blk["row_len"] * out_esz
            fdd.memcpy2d_async(ring_ptr, width, blk["d_data"],
                               blk["row_pitch"] * out_esz, width, rows, d2h.cuda_stream)
            rt.cudaEventRecord(e_rel, d2h.cuda_stream)
            state["blk"] += 1
            state["d2h"] += rows * width
            return e_rel

        def e2e_step():
            plan.execute_stream(host_source, host_sink, stream)
            end = ev_pool[6]
            rt.cudaEventRecord(end, d2h.cuda_stream)
            rt.cudaStreamWaitEvent(s_handle, end, 0)

        e2e_step()
        torch.cuda.synchronize()
        state.update(h2d=0, d2h=0)
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.e2e_steps):
            e2e_step()
        f1.record(stream)
        torch.cuda.synchronize()
        e_ms = f0.elapsed_time(f1)
        e2e = {"value": macs_step * args.e2e_steps / (e_ms / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": state["h2d"] // args.e2e_steps,
               "d2h_bytes_per_step": state["d2h"] // args.e2e_steps,
               "ms_per_step": e_ms / args.e2e_steps,
               "input": ("whole input from pinned host memory" if pool is None else
                         f"every window from a pinned host pool of {pool} generated windows "
                         f"(the {in_bytes / 1e9:.0f} GB input exceeds host memory)"),
               "output": "every output block to a pinned host buffer (one block)"}
        for e in ev_pool:
            rt.cudaEventDestroy(e)
        rt.cudaFreeHost(h_in_ptr)
        rt.cudaFreeHost(ring_ptr)
    # the timed plan's workspace and the resident input go back before the
    # accuracy plans are made
    plan.close()
    d_in = None
    torch.cuda.empty_cache()
    acc = tc_workload_accuracy(fdd, w, prec, args.seed, beams) if not args.no_cpu_baseline \
        else None
    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_baseline(w.scaled(n_beams=1), args.seed, args.cpu_seconds,
                           macs_step=macs_step)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.precision,
            "data": "synthetic (seeded counter-based filterbank, generated on the device)",
            "form": "tensor cores, beams share each bin's phasors; streamed output blocks",
            "config": dict(workload_config(w, info), beams_per_gpu=w.n_beams,
                           precision=args.precision, dm_batch=info["dm_batch"],
                           block_dm=info["block_dm"],
                           tc_form=("CTA pairs" if info["mac_variant"] == fdd.FDD_MAC_TC_PAIR
                                    else "one CTA per SM"),
                           input=("resident in HBM" if resident else
                                  "generated per (beam, chunk) window on the device "
                                  f"({in_bytes / 1e9:.0f} GB exceeds HBM)"),
                           output_bytes_per_step=out_bytes,
                           output_bytes_delivered=blocks[1] // max(args.steps, 1),
                           workspace_gib=info["workspace_bytes"] / 2 ** 30,
                           plan_seconds=plan_s),
            "gpu_launches": prof["kernels"],
            "clocks": clk, "roofline": roofline, "e2e": e2e, "accuracy": acc,
            "cpu_baseline": cpu, "stage_ms_share": stage_share,
            "macs_per_step": macs_step}
    print(json.dumps(line), flush=True)


def run_batch(args) -> None:
    """Whole-batch throughput of the batching form (unpack, transforms and one
    persistent phase-rotate-and-sum launch per wave).  Resident when input and
    output fit (replayed as a CUDA graph), else streamed: every beam's window
    generated on the device by the source, every beam's output block handed
    to a sink that counts it."""
    import torch

    import paper_2110_03482_gb300 as fdd

    import synth.gpu

    fdd.build()
    synth.gpu.build()
    bw = synth.BATCH_WORKLOADS[args.batch]
    beams = bw.beams(args.seed, n_t_div=args.batch_n_t_div)
    common = dict(n_chan=bw.n_chan, nu_lo_mhz=bw.nu_lo_mhz, dnu_mhz=bw.dnu_mhz,
                  t_samp_s=bw.t_samp_s, in_dtype=fdd.FDD_IN_F32, chunk_len=0,
                  output={"spectra": fdd.FDD_OUT_SPECTRA, "power": fdd.FDD_OUT_POWER}[bw.output])
    tc = args.batch_precision != "fp32"
    if tc:  # plans of up to 16 beams, each within the limit (streamed output)
        common.update(precision=TC_PREC[args.batch_precision],
                      workspace_limit=int(args.workspace_gib * (1 << 30)))
    else:  # waves of spectra, leaving room for two output slots per wave
        common.update(workspace_limit=int(min(args.workspace_gib, 100.0) * (1 << 30)))
    gen_kw = [synth.batch_beam_args(bw, desc, args.seed, b)[0] for b, desc in enumerate(beams)]
    t0 = time.perf_counter()
    # (--mac-variant pins the FP32 tile and skips the autotuner)
    with fdd.Batch(beams, autotune=not args.mac_variant, mac_variant=args.mac_variant,
                   **common) as batch:
        plan_s = time.perf_counter() - t0
        info = batch.info
        in_bytes = 4 * info["in_elems"]
        out_bytes = int(info["out_bytes"])
        resident = in_bytes + out_bytes <= RESIDENT_INPUT_BYTES
        stream = torch.cuda.current_stream()
        s_handle = stream.cuda_stream
        gen = synth.gpu.BeamWindows(gen_kw)
        delivered = [0]
        if resident:
            # float32 N(0,1) noise with one dispersed pulse per beam, made on the
            # device by the counter-based generator (beam by beam, in place)
            d_in = torch.empty(info["in_elems"], dtype=torch.float32, device="cuda")
            for b, desc in enumerate(beams):
                gen.fill(b, d_in.data_ptr() + 4 * batch.in_offsets[b], 0, desc[0], s_handle)
            out = torch.empty(info["out_elems"] * (2 if bw.output == "spectra" else 1),
                              device="cuda")

            def step():
                batch.execute(d_in, out, stream)
        else:
            def source(beam, t_begin, n, d_window, ready, s):
                gen.fill(beam, d_window, t_begin, n, s)

            def sink(blk, s):
                delivered[0] += blk["n_dm"] * blk["row_len"] * (8 if bw.output == "spectra" else 4)
                return None

            def step():
                batch.execute_stream(source, sink, stream)
        for _ in range(max(args.warmup, 1)):
            step()
        torch.cuda.synchronize()
        delivered[0] = 0
        clocks = Clocks(gpu_uuid(torch.cuda.get_device_properties(0), 0))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        ms = e0.elapsed_time(e1) / args.steps
    macs = sum(n_dm * bw.n_chan * (oracle_free_pow2(n_t) // 2 + 1) for n_t, _, _, n_dm in beams)
    props = torch.cuda.get_device_properties(0)
    peak = props.multi_processor_count * 128 * 2 * float(load_peaks().get("sm_max_mhz") or 2070) * 1e6
    n_ts = [b[0] for b in beams]
    tc_peak = float(load_peaks().get("bf16_tflops_sustained") or 1700.0) * 1e12
    line = {"metric": METRIC, "value": macs / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.batch_precision if tc else "f32",
            "data": "synthetic (seeded Philox4x32-10 noise + one dispersed pulse per beam, "
                    "generated on the device)",
            "form": ("batching on tensor cores (beams grouped by shared phasors, one plan "
                     "per group of up to 16 beams)" if tc else
                     "batching (persistent launch per wave, autotuned tile)") +
                    (", CUDA graph" if resident and not tc else
                     ", streamed windows and output blocks"),
            "config": {"workload": bw.name, "beams": bw.n_beams, "n_chan": bw.n_chan,
                       "n_t_range": [min(n_ts), max(n_ts)], "n_t_divisor": args.batch_n_t_div,
                       "trials_range": [min(b[3] for b in beams), max(b[3] for b in beams)],
                       "output": bw.output, "waves": info["n_waves"],
                       "work_items": info["work_items"], "ctas": info["ctas"],
                       "tile": ("TC" if tc else fdd.MAC_VARIANT_NAMES[info["mac_variant"]]),
                       "plans_resident": bool(tc and info["workspace_bytes"] > 0),
                       "tail_tile": (fdd.MAC_VARIANT_NAMES[info["tail_variant"]]
                                     if info["tail_variant"] >= 0 else None),
                       "autotune_ms": info["autotune_ms"], "plan_seconds": plan_s,
                       "input_bytes": in_bytes, "output_bytes": out_bytes,
                       "io": "resident" if resident else
                             "streamed (input windows generated per beam on the device; output "
                             f"blocks counted: {delivered[0] // max(args.steps, 1)} B per step)"},
            "fp32_frac_whole_step": FLOPS_PER_MAC * macs / (ms / 1e3) / peak,
            "tensor_frac_whole_step": (FLOPS_PER_MAC * macs / (ms / 1e3) / tc_peak
                                       if tc else None),
            "macs_per_step": macs, "clocks": clk}
    print(json.dumps(line), flush=True)


def oracle_free_pow2(n: int) -> int:
    p = 2
    while p < n:
        p <<= 1
    return p


def main():
    args = parse_args()
    if args.batch:
        run_batch(args)
        return
    if args.mac_sweep:
        run_mac_sweep(args)
        return
    if args.crossover:
        run_crossover(args)
        return
    if args.downsample_sweep:
        run_downsample_sweep(args)
        return
    if args.spin_sweep:
        run_spin_sweep(args)
        return
    if args.impl == "fdd" and synth.WORKLOADS[args.workload].n_beams > 1:
        run_tc_workload(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        tdist.init_process_group("nccl")
        dist = tdist
    try:
        run_fdd(args, rank, world, dist)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
