#!/usr/bin/env python3
"""Throughput benchmark of the SPIIR filter bank on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload batched|plain|multirate|adjoint|precision]
                    [--precision plain|compensated|chunked_fp64|chunked_tc] [--graph]

Workload (default): the batched bank -- 4096 templates with 100..300 complex
single-pole filters each, 3 detectors, 65536 samples (64 s at 1024 Hz) of
white N(0,1) strain, synthetic and seeded.  One step = one spiir_filter call
over the 64 s block (strain staging, recurrence, filter sum, z store of
6.4 GB, running peak) plus spiir_peak.  The stream continues across steps.

Metric: complex IIR filter-updates/s (one update = one filter advanced by one
sample), whole job over all ranks.  N > 1: one process per GPU (torchrun);
templates are independent, so each rank filters its own 4096-template shard
(weak scaling) with no collective on the data path.

Prints ONE JSON line (rank 0).  --impl reference times the FP64 CPU oracle
(the reference arm: there is no other implementation) on the host cores,
each step a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from spiir_inputs import WORKLOADS, updates, workload_bank, workload_strain  # noqa: E402

# DRAM bytes (read + write) per launch of the dominant kernel from an ncu
# capture of the current kernel, by (workload, precision); None where no
# capture of the current kernel applies.  See profiles/.
TRAFFIC = {
    ("batched", "plain"): (
        6.592e9, "k1_plain: 412.0 MB per launch captured on the same bank at 4096 samples "
                 "(profiles/k1_plain_batched_medium.md), scaled by samples to 65536 "
                 "(z writes dominate and grow in proportion); algorithmic bytes 6.44e9"),
}
LANE_OPS_PER_UPDATE = 8      # 4 FMA + 2 MUL + 2 ADD (FP32 lane operations)
# coincidence windows (samples at 1024 Hz) of the detectors after the
# reference: about the light travel time between two sites ~3000 km apart
# (10 ms) and between sites ~8000 km apart (27 ms), plus a sample
NETWORK_WINDOWS = [0, 10, 28]
LANE_OPS_ADJOINT = 20        # reverse pass per filter-update: recompute 6, adjoint 6, grads 8
LANE_OPS_TANGENT = 20        # tangent form: u 4, v 4, g_a sum 4, shifted adjoint 4, g_x 2, g_b 2
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batched",
                    choices=["batched", "plain", "multirate", "adjoint", "precision", "design",
                             "veto", "adjoint-forms", "ceiling"])
    ap.add_argument("--precision", default="plain",
                    choices=["plain", "compensated", "chunked_fp64", "chunked_tc"])
    ap.add_argument("--no-graph", action="store_true",
                    help="time direct calls only (default: also replays of a captured CUDA "
                         "graph of the step, which give the headline value)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default layout (default: the plan times candidate "
                         "layouts and launch modes on its first call)")
    ap.add_argument("--headline-only", action="store_true",
                    help="skip the other workloads' sub-lines of the default run")
    ap.add_argument("--samples", type=int, default=0,
                    help="override the stream length per step (profiling runs)")
    ap.add_argument("--templates", type=int, default=0,
                    help="keep only the bank's first N templates (profiling runs)")
    ap.add_argument("--front-end", action="store_true",
                    help="multirate: windowed-sinc anti-aliasing FIRs (8 R - 1 taps) on the "
                         "decimated bands instead of plain subsampling")
    ap.add_argument("--adjoint-form", default="auto", choices=["auto", "tangent", "reverse"],
                    help="--workload adjoint: evaluation of g_a, g_b (the plan option)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def describe(name, bank, n):
    w = WORKLOADS[name]
    counts = bank.counts()
    return {
        "workload": f"{name} bank: {bank.n_templates} templates x "
                    f"{int(counts.min())}..{int(counts.max())} filters x {bank.n_det} "
                    f"detectors x {n} samples @ {w['rate']} Hz",
        "templates": bank.n_templates, "filters": bank.n_filters, "detectors": bank.n_det,
        "samples": n, "rate_hz": w["rate"], "pole_r": list(w["r_range"]),
        "max_delay": w["d_max"],
    }


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ------------------------------------------------------------ clocks ---
class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------ CPU baseline ---
def oracle_run(bank, x):
    """The oracle on a (sub-)bank, peaks only."""
    import oracle
    if bank.band_of is not None:
        return oracle.filter_multirate(bank.off, bank.a, bank.b, bank.d, bank.band_of,
                                       bank.decim, x, want_z=False)
    return oracle.filter_bank(bank.off, bank.a, bank.b, bank.d, x, want_z=False)


def cpu_baseline(name, bank, x, seconds=15.0):
    """The FP64 oracle, as it stands, on the host cores: a bounded sample of
    the workload's templates (all detectors, full length)."""
    import oracle
    n = x.shape[1]
    # calibrate on enough templates to occupy every core
    cal = bank.subset(range(min(bank.n_templates, 2 * oracle.max_threads())))
    t = time.perf_counter()
    oracle_run(cal, x)
    rate = updates(cal, n) / (time.perf_counter() - t)
    per_t = updates(bank, n) / bank.n_templates
    k = int(max(1, min(bank.n_templates, seconds * rate / per_t)))
    sub = bank.subset(range(k))
    t = time.perf_counter()
    oracle_run(sub, x)
    dt = time.perf_counter() - t
    return {"value": updates(sub, n) / dt, "unit": "filter-updates/s",
            "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"first {k} of {bank.n_templates} templates, all {bank.n_det} "
                      f"detectors, {n} samples ({dt:.1f} s of CPU time, FP64, "
                      f"OpenMP over template x detector)"}


# --------------------------------------------------------- reference ---
def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle
    bank = workload_bank(args.workload)
    x = workload_strain(args.workload)
    n = x.shape[1]
    # size each step to ~3 s of host time
    cal = bank.subset(range(min(bank.n_templates, 2 * oracle.max_threads())))
    t = time.perf_counter()
    oracle_run(cal, x)
    rate = updates(cal, n) / (time.perf_counter() - t)
    per_t = updates(bank, n) / bank.n_templates
    k = int(max(1, min(bank.n_templates, 3.0 * rate / per_t)))
    times = []
    for step in range(args.warmup + args.steps):
        lo = (step * k) % max(1, bank.n_templates - k)
        sub = bank.subset(range(lo, lo + k))
        t = time.perf_counter()
        oracle_run(sub, x)
        dt = time.perf_counter() - t
        if step >= args.warmup:
            times.append((updates(sub, n), dt))
    total_u = sum(u for u, _ in times)
    total_t = sum(t for _, t in times)
    value = total_u / total_t
    sample = (f"{k} templates of {bank.n_templates} per step, all {bank.n_det} detectors, "
              f"{n} samples; FP64, OpenMP over template x detector")
    line = {
        "impl": "reference", "metric": "filter-updates/s", "value": value,
        "unit": "filter-updates/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_t / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded)", "config": describe(args.workload, bank, n),
        "cpu_baseline": {"value": value, "unit": "filter-updates/s",
                         "cores": oracle.max_threads(), "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "filter-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# -------------------------------------------------------------- ours ---
def max_over_ranks(value, dist, device):
    """The largest of every rank's value (the job's time is its slowest rank's)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard_bank(name, rank):
    """Rank 0 filters the workload's bank; rank r > 0 its own shard of a
    world-times-larger bank (independent templates, same distributions)."""
    from spiir_inputs import make_bank, make_multirate_bank
    if rank == 0:
        return workload_bank(name)
    w = WORKLOADS[name]
    if w["kind"] == "multirate":
        return make_multirate_bank(w["n_templates"], w["band_filters"], w["decim"],
                                   w["r_range"], w["d_max"], w["seed"] + 1000 * rank, w["n_det"])
    return make_bank(w["n_templates"], w["filters"], w["r_range"], w["d_max"],
                     w["seed"] + 1000 * rank, w["n_det"])


def device_fp32_peak(dev, sm_max_mhz):
    """FP32 lane-ops/s of the device (T/s): SMs x 128 FP32 lanes x max clock."""
    import torch
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    return n_sm * FP32_LANES_PER_SM * sm_max_mhz * 1e6 / 1e12, n_sm


def alu_roofline(kernel, lane_ops, kernel_ms, peak_lane, n_sm, sm_max, timing, ops_note,
                 traffic=None, traffic_note=None):
    achieved = lane_ops / (kernel_ms / 1e3) / 1e12
    return {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": peak_lane,
            "unit": "T FP32 lane-ops/s", "frac": achieved / peak_lane, "traffic": traffic,
            "traffic_note": traffic_note,
            "note": f"{ops_note} / {timing}; peak = {n_sm} SMs x 128 FP32 lanes x "
                    f"{sm_max:.0f} MHz (derived from unit counts and the measured max clock)"}


def tc_roofline(updates_per_step, tc_ms, peaks, segments=0):
    """Tensor-core projection: 3 split-BF16 products of the (2 rows per
    filter) x (2 x 256 window) weights against one window per 256-sample
    chunk, i.e. 24 algorithmic flops per filter-update it covers.  The
    start states of P time segments need the chunks before the last
    segment's start only, (P - 1) / P of the call (segments = P); the
    chunked tensor-core form covers every chunk (segments = 0)."""
    tc_peak = peaks.get("bf16_tflops") or 1800.0
    cover = (segments - 1) / segments if segments > 1 else 1.0
    ach = 24.0 * updates_per_step * cover / (tc_ms / 1e3) / 1e12
    return {"bound": "tensor", "kernel": "tc_project_kernel", "achieved": ach, "peak": tc_peak,
            "unit": "TFLOP/s", "frac": ach / tc_peak, "traffic": None, "ms_per_step": tc_ms,
            "note": "24 algorithmic BF16 flops per filter-update covered "
                    + (f"((P - 1) / P = {cover:.3f} of the call's updates: the chunks before the "
                       f"last of {segments} segments)" if segments > 1 else "(every chunk)")
                    + " / its own CUDA-event time; "
                    + ("peak = measured cuBLAS bf16 burst" if peaks.get("bf16_tflops")
                       else "peak = fallback 1.8 PFLOP/s bf16")}


def max_rel_error(z_gpu, z_ref):
    """Per (detector, template): max_k |z_gpu - z_ref| / rms_k |z_ref|; the
    largest over the sample, and the absolute error that goes with it."""
    z_gpu = np.asarray(z_gpu).astype(np.complex128)
    diff = np.abs(z_gpu - z_ref).max(axis=-1)
    rms = np.sqrt(np.mean(np.abs(z_ref) ** 2, axis=-1))
    rel = diff / np.maximum(rms, 1e-300)
    return float(rel.max()), float(diff.max()), rel, diff


def argmax_agrees(z_gpu, z_ref, diff):
    """(exact, in_eps_tie, total): the GPU's first argmax of |z|^2 (float32,
    as the kernel decides it) against the oracle's: equal, or among the
    oracle's samples within 4x the measured error of its top."""
    zr = np.ascontiguousarray(np.asarray(z_gpu).real, np.float32)
    zi = np.ascontiguousarray(np.asarray(z_gpu).imag, np.float32)
    idx = np.argmax(zr * zr + zi * zi, axis=-1)
    mag = np.abs(z_ref)
    exact = tie = total = 0
    for i in np.ndindex(mag.shape[:-1]):
        total += 1
        top = int(np.argmax(mag[i]))
        if int(idx[i]) == top:
            exact += 1
        elif mag[i][int(idx[i])] >= mag[i].max() - 4 * diff[i]:
            tie += 1
    return exact, tie, total


def oracle_sample(bank, x, templates, want_z=True):
    """The CPU-baseline leg of a sub-configuration: the FP64 oracle, as it
    stands, on a template sample of the workload (all detectors, full
    length), timed on the host cores.  Its z is what the sub-configuration's
    accuracy figures compare the GPU's z with."""
    import oracle
    sub = bank.subset(templates)
    n = x.shape[1]
    t = time.perf_counter()
    if sub.band_of is not None:
        z, _, _ = oracle.filter_multirate(sub.off, sub.a, sub.b, sub.d, sub.band_of, sub.decim,
                                          x, want_z=want_z)
    else:
        z, _, _ = oracle.filter_bank(sub.off, sub.a, sub.b, sub.d, x, want_z=want_z)
    dt = time.perf_counter() - t
    base = {"value": updates(sub, n) / dt, "unit": "filter-updates/s",
            "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"{len(templates)} of {bank.n_templates} templates (seeded), all "
                      f"{bank.n_det} detectors, {n} samples ({dt:.1f} s, FP64, OpenMP over "
                      f"template x detector)"}
    return base, z


def timed(stream, fn, steps):
    """Mean CUDA-event milliseconds of fn() over `steps` calls on `stream`."""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / steps


# ------------------------------------------------------ sub-configs ---
def sub_plain(sp, dev, stream, peak_lane, n_sm, sm_max):
    """Plain workload (16 templates x 64 filters, 1 detector, 16384 samples
    at 4096 Hz): latency-bound.  Graph-replay latency of the whole call and
    of a 1 s block, with the automatic time segments and without; the
    oracle on the whole workload is both the CPU baseline and the accuracy
    reference."""
    import torch
    bank = workload_bank("plain")
    x_host = workload_strain("plain")
    x = torch.from_numpy(x_host).to(dev)
    D, n = x.shape
    T = bank.n_templates
    upd = updates(bank, n)
    base, zref = oracle_sample(bank, x_host, list(range(T)))
    out = {"workload": describe("plain", bank, n)["workload"], "cpu_baseline": base}
    with ClockSampler(dev.index) as clk:
        for name, seg in (("segmented", 0), ("unsegmented", 1)):
            plan = sp.Plan(bank, device=dev.index, time_segments=seg, kernel_timing=True)
            z = torch.empty((D, T, n), dtype=torch.complex64, device=dev)
            pa = torch.empty((D, T), dtype=torch.float32, device=dev)
            pi = torch.empty((D, T), dtype=torch.int64, device=dev)
            with torch.cuda.stream(stream):
                # accuracy of the call from zero state
                plan.reset(stream=stream)
                plan.filter(x, z, stream=stream)
                plan.peak(pa, pi, stream=stream)
                stream.synchronize()
                zg = z.cpu().numpy()
                rel, err, _, diff = max_rel_error(zg, zref)
                ex, tie, tot = argmax_agrees(zg, zref, diff)
                # K1's own time (events around its launches) over 20 direct calls
                plan.kernel_times()
                for _ in range(20):
                    plan.filter(x, z, stream=stream)
                stream.synchronize()
                kt = plan.kernel_times()
                segs = plan.info()["last_call_segments"]
                res = {"time_segments": segs, "max_rel_err": rel, "max_abs_err": err,
                       "argmax": {"exact": ex, "eps_tie": tie, "of": tot}}
                for what, nb in (("whole call (4 s)", n), ("1 s block", 4096)):
                    xb = x[:, :nb].contiguous()
                    zb = torch.empty((D, T, nb), dtype=torch.complex64, device=dev)
                    g, _, _, _ = plan.capture(xb, zb, pa, pi, warmup=True)
                    lat = []
                    for _ in range(100):
                        a0 = torch.cuda.Event(enable_timing=True)
                        a1 = torch.cuda.Event(enable_timing=True)
                        a0.record(stream)
                        g.replay()
                        a1.record(stream)
                        a1.synchronize()
                        lat.append(a0.elapsed_time(a1))
                    res[f"latency_ms {what}"] = {"median": float(np.median(lat)),
                                                 "min": float(np.min(lat))}
                    del g
            k_ms, k_n = kt["filter"]
            tc_ms, tc_n = kt["projection"]
            med = res["latency_ms whole call (4 s)"]["median"]
            res["value"] = upd / (med / 1e3)
            res["unit"] = "filter-updates/s (whole call, graph replay median)"
            res["roofline"] = alu_roofline(
                "k1_plain", 8 * upd, k_ms / 20, peak_lane, n_sm, sm_max,
                f"{k_ms / 20:.4f} ms of K1 per call (CUDA events around its launches, 20 calls)",
                "8 algorithmic lane-ops per filter-update")
            if tc_n:
                res["roofline_projection"] = tc_roofline(upd, tc_ms / 20, measured_peaks(),
                                                         segments=segs)
            out[name] = res
            plan.close()
    out["clocks"] = clk.summary()
    out["note"] = ("latency-bound: 1.7e7 updates fill a few microseconds of the GPU; the "
                   "segmented plan runs the call as parallel time segments whose start "
                   "states come from the tensor-core projection")
    return out


def sub_multirate(sp, dev, stream, peak_lane, n_sm, sm_max, steps=5, warmup=2):
    """Injection + multirate workload (2048 templates x (60 @ 4096 Hz, 120 @
    1024 Hz, 120 @ 256 Hz), 2^20 samples at 4096 Hz): one signal, template
    1234's own top-rate response, time-reversed (s[m] = A Re h[k0 - m]) at
    sample 700016 with normalised SNR 12 (reading 7), in seeded N(0,1) noise.
    h and every template's noise rms come from the library's own impulse
    responses; the recovery check is that the template with the largest
    normalised peak is the injected one, at the injected time."""
    import torch
    bank = workload_bank("multirate")
    x_noise = workload_strain("multirate")
    D, n = x_noise.shape
    T = bank.n_templates
    tau, k0, lh = 1234, 700_016, 1 << 18
    # every template's response to an impulse at the stream start (4.3 GB)
    plan_h = sp.Plan(bank, device=dev.index)
    delta = torch.zeros((1, lh), dtype=torch.float32, device=dev)
    delta[0, 0] = 1.0
    h = plan_h.filter(delta)
    sigma = torch.sqrt(0.5 * (h[0].abs() ** 2).sum(dim=-1).double()).cpu().numpy()   # [T]
    ht = h[0, tau].cpu().numpy().astype(np.complex128)
    del h
    plan_h.close()
    torch.cuda.empty_cache()
    s = np.zeros((1, n))
    m = np.arange(max(0, k0 - lh + 1), k0 + 1)
    s[0, m] = ht[k0 - m].real
    # the noiseless z_tau[k0] of the signal alone (the bands' subsampling
    # makes the bank time-varying at the top rate, so it is filtered, not
    # taken from h)
    plan_1 = sp.Plan(bank.subset([tau]), device=dev.index)
    zs = plan_1.filter(torch.from_numpy(s.astype(np.float32)).to(dev))
    zs_k0 = complex(zs[0, 0, k0].item())
    plan_1.close()
    del zs
    amp = 12.0 * sigma[tau] / abs(zs_k0)
    x_host = np.ascontiguousarray((x_noise.astype(np.float64) + amp * s).astype(np.float32))
    x = torch.from_numpy(x_host).to(dev)
    upd = updates(bank, n)
    plan = sp.Plan(bank, device=dev.index, kernel_timing=True)
    pa = torch.empty((D, T), dtype=torch.float32, device=dev)
    pi = torch.empty((D, T), dtype=torch.int64, device=dev)

    def call():
        plan.filter(x, emit_z=False, stream=stream)
        plan.peak(pa, pi, stream=stream)

    with torch.cuda.stream(stream):
        plan.reset(stream=stream)
        call()
        stream.synchronize()
        rho = pa[0].cpu().numpy() / sigma
        t_hat = int(pi[0, tau].item())
        won = int(np.argmax(rho))
        for _ in range(warmup - 1):
            call()
        stream.synchronize()
        plan.kernel_times()
        with ClockSampler(dev.index) as clk:
            ms = timed(stream, call, steps)
        kt = plan.kernel_times()
    plan.check(stream)
    k_ms, k_n = kt["filter"]
    tc_ms, tc_n = kt["projection"]
    info = plan.info()
    picks = sorted(set([tau] + [int(t) for t in np.random.default_rng(331).choice(T, 3, replace=False)]))
    base, _ = oracle_sample(bank, x_host, picks, want_z=False)
    out = {"workload": describe("multirate", bank, n)["workload"] + " + injection",
           "value": upd / (ms / 1e3), "unit": "filter-updates/s (band-rate updates)",
           "ms_per_step": ms, "steps": steps, "warmup": warmup,
           "time_segments": info["last_call_segments"],
           "injection": {"template": tau, "sample": k0, "snr": 12.0,
                         "recovered": bool(won == tau and abs(t_hat - k0) <= 16),
                         "argmax_template": won, "peak_sample": t_hat,
                         "rho_injected": float(rho[tau]),
                         "rho_runner_up": float(np.sort(rho)[-2]),
                         "rule": "argmax over all 2048 templates of peak |z| / sigma_tau "
                                 "(sigma_tau^2 = 1/2 sum |h_tau|^2), time within one "
                                 "coarsest-band sample (16)"},
           "roofline": alu_roofline(
               "k1_plain (3 bands)", 8 * upd, ms, peak_lane, n_sm, sm_max,
               f"the step's wall time, {ms:.3f} ms (CUDA events around each step: the bands' "
               f"{k_n / steps:.0f} K1 launches and their projections overlap on two streams, "
               f"so the K1 launches' own event times, {k_ms / steps:.3f} ms summed, exceed it)",
               "8 algorithmic lane-ops per band-rate filter-update"),
           "clocks": clk.summary(), "cpu_baseline": base,
           "l2": "strain (4 MB) L2-resident as in streaming use; no z stored"}
    if tc_n:
        out["roofline_projection"] = tc_roofline(upd, tc_ms / steps, measured_peaks(),
                                                 segments=info["last_call_segments"])
    plan.close()
    return out


def sub_precision(sp, dev, stream, peak_lane, n_sm, sm_max, steps=2):
    """Precision-stress workload (16384 templates x 200 filters, poles
    0.9999 <= |a| <= 0.999995, 2^20 samples at 1024 Hz): every precision
    form's speed (two timed full-length calls after a warm-up) and its
    accuracy on 16 seeded templates of the same full launch (the plan
    streams the 2^20 samples again in 16 calls of 65536 with z stored, and
    the sampled rows are compared with the oracle's)."""
    import torch
    bank = workload_bank("precision")
    x_host = workload_strain("precision")
    x = torch.from_numpy(x_host).to(dev)
    D, n = x.shape
    T = bank.n_templates
    upd = updates(bank, n)
    picks = sorted(int(t) for t in np.random.default_rng(404).choice(T, 16, replace=False))
    base, zref = oracle_sample(bank, x_host, picks)
    piece = 1 << 16
    zbuf = torch.empty((D, T, piece), dtype=torch.complex64, device=dev)
    pick_t = torch.tensor(picks, device=dev)
    out = {"workload": describe("precision", bank, n)["workload"], "cpu_baseline": base,
           "accuracy_sample": f"templates {picks} of the full launch, all {n} samples",
           "forms": {}}
    kernel = {"plain": "k1_plain", "compensated": "k1_compensated",
              "chunked_fp64": "k1_chunked", "chunked_tc": "k1_anchored"}
    with ClockSampler(dev.index) as clk:
        for form in ("plain", "compensated", "chunked_fp64", "chunked_tc"):
            plan = sp.Plan(bank, device=dev.index, precision=form, kernel_timing=True)
            xs = x[:, :piece].contiguous()

            def call():
                plan.filter(x, emit_z=False, stream=stream)

            with torch.cuda.stream(stream):
                plan.filter(xs, emit_z=False, stream=stream)       # warm-up (weights, tiles)
                plan.reset(stream=stream)
                stream.synchronize()
                plan.kernel_times()
                ms = timed(stream, call, steps)
                kt = plan.kernel_times()
                # accuracy: the same plan from zero state, z of the sampled rows
                plan.reset(stream=stream)
                parts = []
                for at in range(0, n, piece):
                    plan.filter(x[:, at:at + piece].contiguous(), zbuf, stream=stream)
                    parts.append(zbuf.index_select(1, pick_t).cpu().numpy())
                stream.synchronize()
            plan.check(stream)
            zg = np.concatenate(parts, axis=-1)
            rel, err, _, diff = max_rel_error(zg, zref)
            ex, tie, tot = argmax_agrees(zg, zref, diff)
            k_ms, k_n = kt["filter"]
            tc_ms, tc_n = kt["projection"]
            res = {"value": upd / (ms / 1e3), "unit": "filter-updates/s", "ms_per_step": ms,
                   "steps": steps, "max_rel_err": rel, "max_abs_err": err,
                   "argmax": {"exact": ex, "eps_tie": tie, "of": tot},
                   "roofline": alu_roofline(
                       kernel[form], 8 * upd, k_ms / steps, peak_lane, n_sm, sm_max,
                       f"{k_n / steps:.0f} launch(es), {k_ms / steps:.2f} ms per step (CUDA "
                       f"events around each launch)",
                       "8 algorithmic lane-ops per filter-update (the form's extra work is "
                       "not counted)")}
            if tc_n:
                res["roofline_projection"] = tc_roofline(upd, tc_ms / steps, measured_peaks())
            out["forms"][form] = res
            plan.close()
    plain = out["forms"]["plain"]["value"]
    for form, res in out["forms"].items():
        res["speed_vs_plain"] = res["value"] / plain
    out["clocks"] = clk.summary()
    del zbuf
    torch.cuda.empty_cache()
    return out


def sub_adjoint(sp, dev, stream, peak_lane, n_sm, sm_max, steps=10, warmup=3):
    """Adjoint workload (256 templates x 200 filters, 65536 samples at 1024
    Hz): spiir_filter_backward (dL/da, dL/db, dL/dx for a seeded g_z) against
    the forward call on the same plan, in both evaluations of g_a, g_b (the
    tangent form, the plan's default here, and the reverse form); the
    oracle's adjoint on 8 sampled templates is the CPU baseline and the
    reference of g_a, g_b there."""
    import torch

    import oracle
    bank = workload_bank("adjoint")
    x_host = workload_strain("adjoint")
    x = torch.from_numpy(x_host).to(dev)
    D, n = x.shape
    T = bank.n_templates
    upd = updates(bank, n)
    g = torch.Generator(device=dev).manual_seed(7)
    gz = torch.randn((D, T, n), dtype=torch.complex64, device=dev, generator=g)
    picks = sorted(int(t) for t in np.random.default_rng(505).choice(T, 8, replace=False))
    sub = bank.subset(picks)
    gz_sub = gz[:, picks].cpu().numpy()
    t0 = time.perf_counter()
    ra, rb, _ = oracle.adjoint(sub.off, sub.a, sub.b, sub.d, x_host, gz_sub, want_gx=False)
    dt = time.perf_counter() - t0
    fil = np.concatenate([np.arange(bank.off[t], bank.off[t + 1]) for t in picks])

    def run_form(form):
        plan = sp.Plan(bank, device=dev.index, kernel_timing=True, adjoint_form=form)
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                ga, gb, gx = plan.backward(x, gz, stream=stream)
            stream.synchronize()
            plan.kernel_times()
            with ClockSampler(dev.index) as clk:
                bw_ms = timed(stream, lambda: plan.backward(x, gz, stream=stream), steps)
                kt = plan.kernel_times()
                plan.reset(stream=stream)
                fw_ms = timed(stream, lambda: plan.filter(x, emit_z=False, stream=stream), steps)
            ga, gb, gx = plan.backward(x, gz, stream=stream)
            stream.synchronize()
        plan.check(stream)
        launches = plan.info()["last_call_launches"]
        ga_s = ga.cpu().numpy()[fil]
        gb_s = gb.cpu().numpy()[fil]
        err_a = float(np.max(np.abs(ga_s - ra)) / np.max(np.abs(ra)))
        err_b = float(np.max(np.abs(gb_s - rb)) / np.max(np.abs(rb)))
        a_ms, _ = kt["adjoint"]
        plan.close()
        if form == "reverse":
            kernel, ops = "k6_adjoint + k7_adjoint_x", LANE_OPS_ADJOINT
            what = ("k6 (reverse pass) and k7 (input-gradient pass)",
                    f"{LANE_OPS_ADJOINT} algorithmic lane-ops per filter-update of the reverse "
                    "pass (recompute 6, adjoint recurrence 6, grad a 4, grad b 2, grad x 2)")
        else:
            kernel, ops = "kt_tangent + adj_project + k7_adjoint_x", LANE_OPS_TANGENT
            what = ("kt_tangent (g_a), the reverse projection and k7 (g_x, g_b)",
                    f"{LANE_OPS_TANGENT} algorithmic lane-ops per filter-update (u 4, v 4, the "
                    "g_a sum 4, shifted adjoint recurrence 4, g_x term 2, g_b sum 2)")
        return {
            "value": upd / (bw_ms / 1e3), "unit": "filter-updates/s of the backward",
            "backward_ms": bw_ms, "forward_ms": fw_ms, "backward_over_forward": bw_ms / fw_ms,
            "launches_per_backward": launches,
            "grad_rel_err": {"g_a": err_a, "g_b": err_b,
                             "of": f"templates {picks}: max |g_gpu - g_oracle| / max |g_oracle|"},
            "roofline": alu_roofline(
                kernel, ops * upd, a_ms / steps, peak_lane, n_sm, sm_max,
                f"{a_ms / steps:.3f} ms per backward of {what[0]} (CUDA events around their "
                f"launches)", what[1]),
            "clocks": clk.summary(),
        }

    forms = {f: run_form(f) for f in ("tangent", "reverse")}
    head = forms["tangent"]
    return {
        "workload": describe("adjoint", bank, n)["workload"],
        "form": "tangent (the plan's default for this bank)",
        "value": head["value"], "unit": head["unit"],
        "backward_ms": head["backward_ms"], "forward_ms": head["forward_ms"],
        "backward_over_forward": head["backward_over_forward"],
        "steps": steps, "warmup": warmup,
        "grad_rel_err": head["grad_rel_err"],
        "roofline": head["roofline"],
        "clocks": head["clocks"],
        "forms": forms,
        "tangent_speedup_over_reverse": forms["reverse"]["backward_ms"] / head["backward_ms"],
        "cpu_baseline": {"value": updates(sub, n) / dt, "unit": "filter-updates/s (adjoint)",
                         "cores": oracle.max_threads(), "kind": "oracle",
                         "sample": f"the FP64 adjoint of {len(picks)} of {T} templates, "
                                   f"{n} samples, g_a and g_b only ({dt:.1f} s)"},
    }


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_1602_05573_b300 as sp

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)

    bank = shard_bank(args.workload, rank)
    if args.templates:
        bank = bank.subset(list(range(min(args.templates, bank.n_templates))))
    x_host = workload_strain(args.workload, args.samples or None)
    n = x_host.shape[1]
    T, D = bank.n_templates, bank.n_det
    upd = updates(bank, n)
    # z is stored for the workloads whose series fit comfortably in HBM
    emit_z = args.workload in ("batched", "plain")
    adjoint = args.workload == "adjoint"
    use_graph = not args.no_graph and not adjoint

    # kernel_timing: the plan records CUDA events around each of its filter,
    # projection and adjoint launches, on the launching stream (not in graphs)
    plan = sp.Plan(bank, device=local_rank, precision=args.precision,
                   autotune=not args.no_autotune and args.precision == "plain",
                   kernel_timing=True, adjoint_form=args.adjoint_form)
    if args.front_end and bank.decim is not None:
        for j, R in enumerate(bank.decim):
            if R > 1:   # low-pass at the band's Nyquist rate, Hann-windowed sinc
                k = np.arange(8 * R - 1) - (8 * R - 2) / 2
                h = np.sinc(k / R) / R * np.hanning(8 * R + 1)[1:-1]
                plan.set_band_fir(j, (h / h.sum()).astype(np.float32))
    stream = torch.cuda.Stream(device=dev)
    x = torch.from_numpy(x_host).to(dev)
    z = torch.empty((D, T, n), dtype=torch.complex64, device=dev) if emit_z else None
    pa = torch.empty((D, T), dtype=torch.float32, device=dev)
    pi = torch.empty((D, T), dtype=torch.int64, device=dev)
    gz = None
    if adjoint:
        g = torch.Generator(device=dev).manual_seed(7)
        gz = torch.randn((D, T, n), dtype=torch.complex64, device=dev, generator=g)
    lib = sp.library()
    sh = stream.cuda_stream
    zp = z.data_ptr() if z is not None else None

    def call():
        if adjoint:
            plan.backward(x, gz, stream=stream)
            return
        st = lib.spiir_filter(plan.handle, x.data_ptr(), n, zp, sh)
        st |= lib.spiir_peak(plan.handle, pa.data_ptr(), pi.data_ptr(), sh)
        if st != 0:
            raise RuntimeError("spiir call failed: " + lib.spiir_last_error_detail().decode())

    def barrier():
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()

    def timed_steps(step):
        """K steps bracketed by a barrier and a device sync on both sides;
        per-step CUDA events on the launching stream."""
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        barrier()
        with ClockSampler(local_rank) as clk:
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            for i in range(args.steps):
                ev[i][0].record(stream)
                step()
                ev[i][1].record(stream)
            t1.record(stream)
            barrier()
        return t0.elapsed_time(t1), [a.elapsed_time(b) for a, b in ev], clk.summary()

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):   # the first call runs the autotuner
            call()
        barrier()
        plan.kernel_times()   # drop the warm-up launches' events
        direct_ms, direct_steps, direct_clk = timed_steps(call)
        plan.check(stream)
        ktimes = plan.kernel_times()   # the direct steps' kernels, per class
        graph = None
        if use_graph:
            graph, _, _, _ = plan.capture(x, z, pa, pi, emit_z=emit_z, warmup=False)
            for _ in range(2):
                graph.replay()
            graph_ms, graph_steps, graph_clk = timed_steps(graph.replay)
            plan.check(stream)
    direct_ms = max_over_ranks(direct_ms, dist, dev)
    if graph is not None:
        graph_ms = max_over_ranks(graph_ms, dist, dev)
        total_ms, clocks = graph_ms, graph_clk
    else:
        total_ms, clocks = direct_ms, direct_clk
    ms_step = total_ms / args.steps
    value = upd * world * args.steps / (total_ms / 1e3)

    extra = {}
    if graph is not None:
        extra["direct"] = {"value": upd * world * args.steps / (direct_ms / 1e3),
                           "ms_per_step": direct_ms / args.steps, "clocks": direct_clk,
                           "what": "the same step as direct C-ABI calls (no graph)"}
    if adjoint:  # forward time on the same plan, for the backward/forward ratio
        with torch.cuda.stream(stream):
            plan.filter(x, emit_z=False, stream=stream)
            barrier()
            fwd_ms = timed(stream, lambda: plan.filter(x, emit_z=False, stream=stream),
                           args.steps)
        extra["adjoint"] = {"backward_ms": ms_step, "forward_ms": fwd_ms,
                            "backward_over_forward": ms_step / fwd_ms}

    if not adjoint and WORKLOADS[args.workload]["kind"] == "single":
        # peak-SNR latency: graph replay of a call on strain already on the
        # device until the running peaks are ready (the plan's sample counter
        # moves on; the throughput numbers above are already taken)
        rate = WORKLOADS[args.workload]["rate"]
        nb = min(rate, n)
        xb = x[:, :nb].contiguous()
        zb = torch.empty((D, T, nb), dtype=torch.complex64, device=dev) if emit_z else None
        with torch.cuda.stream(stream):
            g2, _, _, _ = plan.capture(xb, zb, pa, pi, emit_z=emit_z, warmup=True)
            lat = []
            for _ in range(100):
                a0 = torch.cuda.Event(enable_timing=True)
                a1 = torch.cuda.Event(enable_timing=True)
                a0.record(stream)
                g2.replay()
                a1.record(stream)
                a1.synchronize()
                lat.append(a0.elapsed_time(a1))
            del g2
        extra["latency_ms"] = {f"{nb / rate:g} s block": {"median": float(np.median(lat)),
                                                          "min": float(np.min(lat))},
                               "what": "graph replay of filter+peak (strain resident), "
                                       "median and min of 100"}

    if emit_z and D > 1 and not adjoint:
        # coincidence across detectors on the stored z (spiir_network_peak),
        # timed on its own after the filter steps: HBM-bound, z > L2 so every
        # pass streams it from DRAM
        window = [0] + NETWORK_WINDOWS[1:D] + [NETWORK_WINDOWS[-1]] * max(0, D - len(NETWORK_WINDOWS))
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                sp.network_peak(z, window, stream=stream)
            stream.synchronize()
            net_ms = timed(stream, lambda: sp.network_peak(z, window, stream=stream), args.steps)
        # algorithmic bytes: z once; the kernel also re-reads a 2w halo per
        # 2048 outputs of every detector d >= 1
        net_bytes = float(z.numel() * 8)
        hbm = measured_peaks().get("hbm_gbs") or 6400.0
        net_gbs = net_bytes / (net_ms / 1e3) / 1e9
        extra["network_peak"] = {
            "kernel": "network_peak_kernel + network_finish_kernel", "windows": window,
            "ms": net_ms,
            "bound": "hbm", "achieved": net_gbs, "peak": hbm, "unit": "GB/s",
            "frac": net_gbs / hbm,
            "note": (f"per template the first t maximising |z_0(t)|^2 + sum_d max_(|u|<=w_d) "
                     f"|z_d(t+u)|^2; algorithmic bytes = z read once ({net_bytes / 1e9:.2f} GB) / "
                     f"CUDA-event time of {args.steps} calls on the launching stream; peak = "
                     f"measured copy bandwidth")}

    # end to end through the public API: pinned host strain in, peaks out
    e2e = None
    if not args.no_e2e and not adjoint:
        xh = torch.from_numpy(x_host).pin_memory()
        pah = torch.empty((D, T), dtype=torch.float32).pin_memory()
        pih = torch.empty((D, T), dtype=torch.int64).pin_memory()
        with torch.cuda.stream(stream):
            def e2e_step():
                x.copy_(xh, non_blocking=True)
                plan.filter(x, z, emit_z=emit_z, stream=stream)
                plan.peak(pa, pi, stream=stream)
                pah.copy_(pa, non_blocking=True)
                pih.copy_(pi, non_blocking=True)
            for _ in range(2):
                e2e_step()
            barrier()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            for _ in range(args.steps):
                e2e_step()
            a1.record(stream)
            barrier()
        e_ms = max_over_ranks(a0.elapsed_time(a1), dist, dev)
        e2e = {"value": upd * world * args.steps / (e_ms / 1e3), "unit": "filter-updates/s",
               "h2d_bytes_per_step": int(xh.numel() * 4),
               "d2h_bytes_per_step": int(pah.numel() * 4 + pih.numel() * 8),
               "ms_per_step": e_ms / args.steps}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    info = plan.info()
    # our kernels per step, as the plan counted them for the last call (K1
    # passes, decimation, segment carry/merge, counter advance; the adjoint:
    # checkpointed K1, projection, K6, K7, finalize), plus the spiir_peak copy
    launches_per_step = info["last_call_launches"] + (0 if adjoint else 1)
    peaks = measured_peaks()
    sm_max = peaks.get("sm_max_mhz") or clocks.get("sm_max_mhz") or 2032.0
    peak_lane, n_sm = device_fp32_peak(dev, sm_max)
    kernel = {"plain": "k1_plain", "compensated": "k1_compensated",
              "chunked_fp64": "k1_chunked", "chunked_tc": "k1_anchored"}[args.precision]
    # the dominant kernel's own device time over the direct timed steps
    # (events the plan records around each launch; graph replays record none)
    k_ms, k_n = ktimes["adjoint" if adjoint else "filter"]
    # the auto form is the tangent one on a bank this size (>= 8 warps per SM)
    reverse = adjoint and args.adjoint_form == "reverse"
    lane_ops = ((LANE_OPS_ADJOINT if reverse else LANE_OPS_TANGENT) if adjoint
                else LANE_OPS_PER_UPDATE) * upd
    kernel_ms = k_ms / args.steps
    timing = (f"{k_n / args.steps:.0f} launch(es) per step, {kernel_ms:.3f} ms per step "
              f"(CUDA events around each launch on the launching stream, direct steps)")
    if WORKLOADS[args.workload]["kind"] != "single":
        # multirate: the bands' launches overlap on two streams; their summed
        # event times exceed the step, so the step's wall time is the divisor
        kernel_ms = direct_ms / args.steps
        timing = (f"the direct steps' wall time, {kernel_ms:.3f} ms per step (the bands' "
                  f"{k_n / args.steps:.0f} K1 launches overlap on two streams; their own event "
                  f"times sum to {k_ms / args.steps:.3f} ms)")
    if adjoint:
        kernel = ("k6_adjoint + k7_adjoint_x" if reverse else
                  "kt_tangent + adj_project + k7_adjoint_x")
    traffic, traffic_note = None, None
    key = ("adjoint" if adjoint else args.workload, args.precision)
    if key in TRAFFIC and not args.samples and not args.templates:
        traffic, traffic_note = TRAFFIC[key]
    ops_note = ("20 algorithmic lane-ops per filter-update of the reverse pass (recompute 6, "
                "adjoint recurrence 6, grad a 4, grad b 2, grad x 2) over the device time of "
                "the reverse pass (k6) and the input-gradient pass (k7)" if reverse else
                "20 algorithmic lane-ops per filter-update (u 4, v 4, the g_a sum 4, shifted "
                "adjoint recurrence 4, g_x term 2, g_b sum 2) over the device time of the "
                "tangent pass, the reverse projection and k7" if adjoint else
                "8 algorithmic lane-ops per filter-update")
    line = {
        "metric": "filter-updates/s", "value": value, "unit": "filter-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded N(0,1) strain, random poles/gains/delays)",
        "config": dict(describe(args.workload, bank, n),
                       precision=args.precision, graph=bool(graph is not None),
                       autotune=not args.no_autotune and args.precision == "plain",
                       z_stored=emit_z, front_end=bool(args.front_end),
                       parallelism=f"template shards x{world}" if world > 1 else "1 GPU",
                       l2=("each step writes the z series (> 126 MB L2), which evicts the "
                           "previous step; the strain stays L2-resident as in streaming use")
                       if emit_z else "strain (<= 4 MB) L2-resident as in streaming use; "
                                      "no z stored",
                       plan={k: info[k] for k in ("warps_per_cta", "block_len", "ring_copies",
                                                  "history_len", "smem_bytes",
                                                  "max_filters_per_lane",
                                                  "bank_conflict_ratio", "n_slots", "n_units",
                                                  "persistent", "tail_templates",
                                                  "last_call_segments")},
                       autotune_report=plan.tune_report()),
        "roofline": alu_roofline(kernel, lane_ops, kernel_ms, peak_lane, n_sm, sm_max, timing,
                                 f"{ops_note} x {upd:.4g} updates per step", traffic,
                                 traffic_note),
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "filter_ms": float(np.mean(graph_steps if graph is not None else direct_steps)),
        # templates (all detectors, mean filter count) whose 1 s of data is
        # filtered in 1 s at this throughput
        "templates_realtime": upd * world / (ms_step / 1e3) / (bank.n_filters / T * D)
                              / WORKLOADS[args.workload]["rate"],
    }
    tc_ms, tc_n = ktimes["projection"]
    if tc_n > 0:
        line["roofline_projection"] = tc_roofline(
            upd, tc_ms / args.steps, peaks,
            segments=0 if args.precision == "chunked_tc" else info["last_call_segments"])
        line["roofline_projection"]["launches_per_step"] = tc_n / args.steps
    line.update(extra)
    if e2e:
        line["e2e"] = e2e
    if not args.no_cpu_baseline and not adjoint:
        line["cpu_baseline"] = cpu_baseline(args.workload, bank, x_host)
    plan.close()
    del z
    torch.cuda.empty_cache()
    # the other workloads, each with its own clocks and roofline (one GPU)
    if world == 1 and args.workload == "batched" and not args.headline_only:
        subs = {}
        for name, fn in (("plain", sub_plain), ("multirate", sub_multirate),
                         ("precision", sub_precision), ("adjoint", sub_adjoint)):
            t = time.perf_counter()
            subs[name] = fn(sp, dev, stream, peak_lane, n_sm, sm_max)
            subs[name]["wall_s"] = time.perf_counter() - t
            torch.cuda.empty_cache()
        line["configs"] = subs
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_design(args):
    """IIR bank design: gains of 64 synthetic chirp templates (360 filters
    each) fitted by conjugate gradients whose products run in the library's
    forward and adjoint kernels; one GPU, rank 0."""
    import torch

    import paper_1602_05573_b300 as sp
    from paper_1602_05573_b300 import design
    from spiir_inputs import chirp_template
    T, L, rate = 64, 360, 2048
    targets = [design.matched_target(chirp_template(rate, 60, 500, f0=f0))
               for f0 in np.linspace(110.0, 160.0, T)]
    N = max(len(t) for t in targets)
    targets = np.stack([np.pad(t, (0, N - len(t))) for t in targets])
    placed = [design.place_filters(t, L) for t in targets]
    a = np.stack([p[0] for p in placed])
    d = np.stack([p[1] for p in placed])
    b0 = np.stack([p[2] for p in placed])
    for _ in range(args.warmup):
        design.fit_gains(sp, a, d, targets, b0=b0, iters=5)
    times, iters, ov = [], 0, None
    with ClockSampler(0) as clk:
        for _ in range(args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            _, z, iters = design.fit_gains(sp, a, d, targets, b0=b0)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            ov = design.overlap(z, targets)
    ms = float(np.mean(times))
    # poles and gains (variable projection through the adjoint's g_a) on a
    # smaller bank of 220 filters per template, once
    L2 = 220
    placed2 = [design.place_filters(t, L2) for t in targets]
    a2 = np.stack([p[0] for p in placed2])
    d2 = np.stack([p[1] for p in placed2])
    b2 = np.stack([p[2] for p in placed2])
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    _, _, _, hist = design.fit_bank(sp, a2, d2, targets, b0=b2, outer=40)
    e1.record()
    torch.cuda.synchronize()
    refine = {"filters": L2, "outer_steps": 40, "ms": e0.elapsed_time(e1),
              "overlap_gains_only_min": float(hist[0].min()),
              "overlap_min": float(hist[-1].min()), "overlap_mean": float(hist[-1].mean()),
              "per_step": "line search on the poles along -g_a (spiir_filter_backward, "
                          "g_z = 2 (z - t)), then the gains refitted by conjugate gradients"}
    line = {
        "metric": "fit iterations/s", "value": iters / (ms / 1e3), "unit": "CG iterations/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic chirps (leading-order inspiral, 60-500 Hz at 2048 Hz)",
        "config": {"workload": f"IIR bank design: {T} chirp templates x {L} filters x "
                               f"{N} samples", "templates": T, "filters": L, "samples": N,
                   "rate_hz": rate},
        "design": {"cg_iterations": iters, "fit_ms": ms, "overlap_min": float(ov.min()),
                   "overlap_mean": float(ov.mean()),
                   "per_iteration": "one spiir_filter on an impulse (A p) and one "
                                    "spiir_filter_backward (A^H v) for all templates"},
        "pole_refinement": refine,
        "clocks": clk.summary(),
    }
    print(json.dumps(line))
    return 0


def run_adjoint_forms(args):
    """The two evaluations of the adjoint's g_a, g_b (reverse and tangent
    form) on banks from a few templates to thousands, with and without g_x:
    the crossovers behind the plan's automatic choice.  ms per backward, CUDA
    events around `steps` calls after `warmup`; one GPU, rank 0."""
    import torch

    import paper_1602_05573_b300 as sp
    from spiir_inputs import make_bank, make_strain
    dev = torch.device("cuda", 0)
    shapes = [(7, 100, 3000, 1), (16, 64, 16384, 1), (64, 360, 27904, 1), (128, 200, 65536, 1),
              (256, 200, 65536, 1), (1024, 200, 16384, 1), (64, 200, 65536, 3)]
    rows = []
    with ClockSampler(0) as clk:
        for T, L, n, D in shapes:
            bank = make_bank(T, L, (0.99, 0.9995), 1024, seed=5, n_det=D)
            x = torch.from_numpy(make_strain(D, n, seed=6)).to(dev)
            g = torch.Generator(device=dev).manual_seed(7)
            gz = torch.randn((D, T, n), dtype=torch.complex64, device=dev, generator=g)
            row = {"templates": T, "filters": L, "samples": n, "detectors": D}
            for want_gx in (False, True):
                for form in ("reverse", "tangent"):
                    plan = sp.Plan(bank, device=0, adjoint_form=form)
                    for _ in range(max(1, args.warmup)):
                        plan.backward(x, gz, want_gx=want_gx)
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    torch.cuda.synchronize(dev)
                    e0.record()
                    for _ in range(args.steps):
                        plan.backward(x, gz, want_gx=want_gx)
                    e1.record()
                    torch.cuda.synchronize(dev)
                    row[f"{form}_{'gx' if want_gx else 'no_gx'}_ms"] = e0.elapsed_time(e1) / args.steps
                    plan.close()
            rows.append(row)
    print(json.dumps({"metric": "ms per backward", "unit": "ms", "higher_is_better": False,
                      "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "dtype": "f32", "data": "synthetic (seeded N(0,1) strain, random banks)",
                      "config": {"workload": "adjoint forms: reverse vs tangent over bank sizes"},
                      "rows": rows, "clocks": clk.summary()}))
    return 0


def run_veto(args):
    """Chi^2 veto on the batched bank: the bank regrouped into 4 frequency
    bins per template (chi2_split), one filter call writing every bin's
    series, then spiir_chi2_peak; one GPU, rank 0."""
    import torch

    import paper_1602_05573_b300 as sp
    p = 4
    bank = workload_bank("batched", n_templates=args.templates or None)
    x = torch.from_numpy(workload_strain("batched")).cuda()
    D, n = x.shape
    T = bank.n_templates
    split = sp.chi2_split(bank, p)
    # bins hold about a quarter of a template's filters (energy-balanced, so
    # some exceed 96): half warps measured faster for this bank as a whole
    small = int(np.diff(split.off).max()) <= 160
    plan = sp.Plan(split, lanes_per_template=16 if small else 0)
    zg = torch.empty((D, T * p, n), dtype=torch.complex64, device="cuda")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            plan.filter(x, zg, stream=stream)
            sp.chi2_peak(zg, p, stream=stream)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3 * args.steps)]
        stream.synchronize()
        with ClockSampler(0) as clk:
            for k in range(args.steps):
                ev[3 * k].record(stream)
                plan.filter(x, zg, stream=stream)
                ev[3 * k + 1].record(stream)
                sp.chi2_peak(zg, p, stream=stream)
                ev[3 * k + 2].record(stream)
            stream.synchronize()
    plan.check()
    f_ms = float(np.mean([ev[3 * k].elapsed_time(ev[3 * k + 1]) for k in range(args.steps)]))
    c_ms = float(np.mean([ev[3 * k + 1].elapsed_time(ev[3 * k + 2]) for k in range(args.steps)]))
    upd = updates(bank, n)
    nbytes = float(zg.numel() * 8)
    hbm = measured_peaks().get("hbm_gbs") or 6400.0
    gbs = nbytes / (c_ms / 1e3) / 1e9
    line = {
        "metric": "filter-updates/s", "value": upd / ((f_ms + c_ms) / 1e3),
        "unit": "filter-updates/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": f_ms + c_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded N(0,1) strain, random poles/gains/delays)",
        "config": dict(describe("batched", bank, n), bins=p,
                       l2="every step writes the bins' series (25.8 GB > 126 MB L2)"),
        "veto": {"filter_ms": f_ms, "chi2_ms": c_ms, "bins": p,
                 "lanes_per_template": plan.info()["lanes_per_template"]},
        "roofline": {"bound": "hbm", "kernel": "chi2_peak_kernel", "achieved": gbs, "peak": hbm,
                     "unit": "GB/s", "frac": gbs / hbm, "traffic": None,
                     "note": f"algorithmic bytes = the bins' series read once "
                             f"({nbytes / 1e9:.1f} GB) / its CUDA-event time"},
        "clocks": clk.summary(),
    }
    print(json.dumps(line))
    plan.close()
    return 0


def run_ceiling(args):
    """The filter step's FP32 rate in isolation (paper_1602_05573_b300/probe:
    the recurrence and the cross-lane sum on register-resident coefficients
    and a conflict-free shared window; no ring, barriers, combine or z
    stores), for the (filters per lane, lanes per template) cases of the
    batched bank's layout and for 64 slots per template over 32, 16 and 8
    lanes; beside the stand-in without the cross-lane sum.  Read against
    the filter kernel's own rate (per slot-update: the headline's useful
    fraction times slots / filters)."""
    import ctypes
    import torch
    here = os.path.dirname(os.path.abspath(__file__))
    path = os.path.join(here, "paper_1602_05573_b300", "_lib", "libspiir_probe.so")
    if not os.path.exists(path):
        raise RuntimeError("the probe library is missing: run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    lib.spiir_probe_step.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    lib.spiir_probe_step.restype = ctypes.c_int
    torch.cuda.init()
    dev = torch.device("cuda", 0)

    def probe(F, G, ctas=4):
        ms, fr = ctypes.c_double(), ctypes.c_double()
        rc = lib.spiir_probe_step(F, G, ctas, max(1000, 40000 // F), ctypes.byref(ms), ctypes.byref(fr))
        if rc != 0:
            raise RuntimeError(f"spiir_probe_step({F}, {G}, {ctas}) returned {rc}")
        return fr.value
    # the batched bank's layout as the library builds it: its lanes per
    # template G (whole warps for this bank), ceil(n / G) filters per lane
    import paper_1602_05573_b300 as sp
    bank = workload_bank("batched")
    plan = sp.Plan(bank, device=dev.index)
    G = int(plan.info()["lanes_per_template"])
    plan.close()
    counts = np.diff(np.asarray(bank.off))
    slots = {}
    for c in counts:
        F = -(-int(c) // G)
        slots[(F, G)] = slots.get((F, G), 0) + F * G
    with ClockSampler(dev.index) as clk:
        cases = {}
        for (F, G) in sorted(slots):
            cases[f"F{F}/G{G}"] = {"with_sum": probe(F, G), "without_sum": probe(F, 0),
                                   "slot_share": slots[(F, G)] / sum(slots.values())}
        mean = sum(v["with_sum"] * v["slot_share"] for v in cases.values())
        slots64 = {f"F{F}/G{G}": probe(F, G) for F, G in ((2, 32), (4, 16), (8, 8))}
    line = {"metric": "FP32 fraction of the filter step in isolation",
            "value": mean, "unit": "of 128 FP32 lanes x SMs x clock",
            "workload": "probe: 16 warps per SM, 8 lane-ops per filter-update, "
                        "cross-lane sum over G lanes every 8 samples",
            "batched_layout": cases,
            "batched_slot_weighted": mean,
            "slots64_top_band_shapes": slots64,
            "clocks": clk.summary()}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.workload == "ceiling" and args.impl != "reference":
        return run_ceiling(args) if int(os.environ.get("RANK", 0)) == 0 else 0
    if args.workload == "design" and args.impl != "reference":
        return run_design(args) if int(os.environ.get("RANK", 0)) == 0 else 0
    if args.workload == "veto" and args.impl != "reference":
        return run_veto(args) if int(os.environ.get("RANK", 0)) == 0 else 0
    if args.workload == "adjoint-forms" and args.impl != "reference":
        return run_adjoint_forms(args) if int(os.environ.get("RANK", 0)) == 0 else 0
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
