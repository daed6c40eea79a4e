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
        6.547e9, "k1_plain: 409.2 MB per launch captured on the same bank at 4096 samples "
                 "(profiles/k1_plain_batched_medium.md), scaled by samples to 65536 "
                 "(z writes dominate and grow in proportion); algorithmic bytes 6.44e9"),
}
LANE_OPS_PER_UPDATE = 8      # 4 FMA + 2 MUL + 2 ADD (FP32 lane operations)
# coincidence windows (samples at 1024 Hz) of the detectors after the
# reference: about the light travel time between two sites ~3000 km apart
# (10 ms) and between sites ~8000 km apart (27 ms), plus a sample
NETWORK_WINDOWS = [0, 10, 28]
LANE_OPS_ADJOINT = 20        # reverse pass per filter-update: recompute 6, adjoint 6, grads 8
B300_SMS = 148
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batched",
                    choices=["batched", "plain", "multirate", "adjoint", "precision", "design",
                             "veto"])
    ap.add_argument("--precision", default="plain",
                    choices=["plain", "compensated", "chunked_fp64", "chunked_tc"])
    ap.add_argument("--graph", action="store_true",
                    help="time replays of a captured CUDA graph of the step")
    ap.add_argument("--autotune", action="store_true",
                    help="let the plan time candidate layouts on its first call")
    ap.add_argument("--samples", type=int, default=0,
                    help="override the stream length per step (profiling runs)")
    ap.add_argument("--templates", type=int, default=0,
                    help="keep only the bank's first N templates (profiling runs)")
    ap.add_argument("--front-end", action="store_true",
                    help="multirate: windowed-sinc anti-aliasing FIRs (8 R - 1 taps) on the "
                         "decimated bands instead of plain subsampling")
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

    # kernel_timing: the plan records CUDA events around each of its filter,
    # projection and adjoint launches, on the launching stream (not in graphs)
    plan = sp.Plan(bank, device=local_rank, precision=args.precision,
                   autotune=args.autotune, kernel_timing=True)
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

    graph = None
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            call()
        barrier()
        if args.graph and not adjoint:
            graph, _, _, _ = plan.capture(x, z, pa, pi, emit_z=emit_z, warmup=False)
            barrier()
        step = graph.replay if graph is not None else call
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        plan.kernel_times()   # drop the warm-up launches' events
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
        plan.check(stream)
    ktimes = plan.kernel_times()   # the timed steps' kernels, per class
    total_ms = t0.elapsed_time(t1)
    step_times = [a.elapsed_time(b) for a, b in ev]
    filt_ms = float(np.mean(step_times))
    total_ms = max_over_ranks(total_ms, dist, dev)
    ms_step = total_ms / args.steps
    value = upd * world * args.steps / (total_ms / 1e3)

    extra = {}
    if adjoint:  # forward time on the same plan, for the backward/forward ratio
        with torch.cuda.stream(stream):
            plan.filter(x, emit_z=False, stream=stream)
            barrier()
            f0 = torch.cuda.Event(enable_timing=True)
            f1 = torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            for _ in range(args.steps):
                plan.filter(x, emit_z=False, stream=stream)
            f1.record(stream)
            barrier()
        fwd_ms = f0.elapsed_time(f1) / args.steps
        extra["adjoint"] = {"backward_ms": ms_step, "forward_ms": fwd_ms,
                            "backward_over_forward": ms_step / fwd_ms}
    def graph_latency(xb, zb, emit):
        """Median/min of 100 graph replays of one filter+peak call on xb."""
        with torch.cuda.stream(stream):
            g2, _, _, _ = plan.capture(xb, zb, pa, pi, emit_z=emit, warmup=True)
            lat = []
            for _ in range(100):
                a0 = torch.cuda.Event(enable_timing=True)
                a1 = torch.cuda.Event(enable_timing=True)
                a0.record(stream)
                g2.replay()
                a1.record(stream)
                a1.synchronize()
                lat.append(a0.elapsed_time(a1))
        return float(np.median(lat)), float(np.min(lat))

    if not adjoint and WORKLOADS[args.workload]["kind"] == "single":
        # peak-SNR latency: graph replay of a call on strain already on the
        # device until the running peaks are ready (the plan's sample counter
        # moves on; the throughput numbers above are already taken)
        rate = WORKLOADS[args.workload]["rate"]
        lat = {}
        blocks = [("1 s", rate)]
        if args.workload == "plain":
            blocks.append((f"{n / rate:g} s (the whole call)", n))
        for what, nb in blocks:
            if nb > n:
                continue
            xb = x[:, :nb].contiguous()
            zb = torch.empty((D, T, nb), dtype=torch.complex64, device=dev) if emit_z else None
            med, mn = graph_latency(xb, zb, emit_z)
            lat[what] = {"median": med, "min": mn}
        extra["latency_ms"] = dict(lat, what="graph replay of filter+peak (strain resident), "
                                             "median and min of 100")

    if emit_z and D > 1 and not adjoint:
        # coincidence across detectors on the stored z (spiir_network_peak),
        # timed on its own after the filter steps: HBM-bound, z > L2 so every
        # pass streams it from DRAM
        window = [0] + NETWORK_WINDOWS[1:D] + [NETWORK_WINDOWS[-1]] * max(0, D - len(NETWORK_WINDOWS))
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                sp.network_peak(z, window, stream=stream)
            stream.synchronize()
            n0 = torch.cuda.Event(enable_timing=True)
            n1 = torch.cuda.Event(enable_timing=True)
            n0.record(stream)
            for _ in range(args.steps):
                sp.network_peak(z, window, stream=stream)
            n1.record(stream)
            n1.synchronize()
        net_ms = n0.elapsed_time(n1) / args.steps
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
    clocks = clk.summary()
    peaks = measured_peaks()
    sm_max = peaks.get("sm_max_mhz") or clocks.get("sm_max_mhz") or 2032.0
    peak_lane = B300_SMS * FP32_LANES_PER_SM * sm_max * 1e6 / 1e12   # T lane-ops/s
    kernel = {"plain": "k1_plain", "compensated": "k1_compensated",
              "chunked_fp64": "k1_chunked", "chunked_tc": "k1_anchored"}[args.precision]
    # the dominant kernel's own device time over the timed steps (events the
    # plan records around each launch); graph replays record none, then the
    # step time stands in
    k_ms, k_n = ktimes["adjoint" if adjoint else "filter"]
    lane_ops = (LANE_OPS_ADJOINT if adjoint else LANE_OPS_PER_UPDATE) * upd
    if k_n > 0:
        kernel_ms = k_ms / args.steps
        timing = (f"{k_n / args.steps:.0f} launch(es) per step, {kernel_ms:.3f} ms per step "
                  f"(CUDA events around each launch on the launching stream)")
    else:
        kernel_ms = filt_ms
        timing = f"mean step time {filt_ms:.3f} ms (graph replay: no per-launch events)"
    achieved = lane_ops / (kernel_ms / 1e3) / 1e12
    if adjoint:
        kernel = "k6_adjoint + k7_adjoint_x"
    traffic, traffic_note = None, None
    key = ("adjoint" if adjoint else args.workload, args.precision)
    if key in TRAFFIC and not args.samples and not args.templates:
        traffic, traffic_note = TRAFFIC[key]
    ops_note = ("20 algorithmic lane-ops per filter-update of the reverse pass (recompute 6, "
                "adjoint recurrence 6, grad a 4, grad b 2, grad x 2) over the device time of "
                "the reverse pass (k6) and the input-gradient pass (k7)" if adjoint else
                "8 algorithmic lane-ops per filter-update")
    line = {
        "metric": "filter-updates/s", "value": value, "unit": "filter-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded N(0,1) strain, random poles/gains/delays)",
        "config": dict(describe(args.workload, bank, n),
                       precision=args.precision, graph=bool(graph is not None),
                       z_stored=emit_z, front_end=bool(args.front_end),
                       parallelism=f"template shards x{world}" if world > 1 else "1 GPU",
                       l2=("each step writes the z series (> 126 MB L2), which evicts the "
                           "previous step; the strain stays L2-resident as in streaming use")
                       if emit_z else "strain (<= 4 MB) L2-resident as in streaming use; "
                                      "no z stored",
                       plan={k: info[k] for k in ("warps_per_cta", "block_len", "ring_copies",
                                                  "history_len", "smem_bytes",
                                                  "max_filters_per_lane",
                                                  "bank_conflict_ratio", "n_slots",
                                                  "last_call_segments")}),
        "roofline": {"bound": "alu", "kernel": kernel, "achieved": achieved,
                     "peak": peak_lane, "unit": "T FP32 lane-ops/s",
                     "frac": achieved / peak_lane, "traffic": traffic,
                     "traffic_note": traffic_note,
                     "note": f"{ops_note} x {upd:.4g} updates per step / {timing}; "
                             f"peak = 148 SMs x 128 FP32 lanes x {sm_max:.0f} MHz (derived "
                             f"from unit counts and the measured max clock)"},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "filter_ms": filt_ms,
        # templates (all detectors, mean filter count) whose 1 s of data is
        # filtered in 1 s at this throughput
        "templates_realtime": upd * world / (ms_step / 1e3) / (bank.n_filters / T * D)
                              / WORKLOADS[args.workload]["rate"],
    }
    tc_ms, tc_n = ktimes["projection"]
    if tc_n > 0:
        # tensor-core projection: 3 split-BF16 products of the (2 rows per
        # filter) x (2 x 256 window) weights against one window per 256-sample
        # chunk, i.e. 24 algorithmic flops per filter-update
        tc_flops = 24.0 * upd
        tc_peak = peaks.get("bf16_tflops") or 1800.0
        tc_ach = tc_flops / (tc_ms / args.steps / 1e3) / 1e12
        line["roofline_projection"] = {
            "bound": "tensor", "kernel": "tc_project_kernel", "achieved": tc_ach,
            "peak": tc_peak, "unit": "TFLOP/s", "frac": tc_ach / tc_peak, "traffic": None,
            "ms_per_step": tc_ms / args.steps, "launches_per_step": tc_n / args.steps,
            "note": "24 algorithmic BF16 flops per filter-update / its own CUDA-event time; "
                    "peak = measured cuBLAS bf16 burst (MEASURED_PEAKS.json)"
                    if peaks.get("bf16_tflops") else "peak = fallback 1.8 PFLOP/s bf16"}
    line.update(extra)
    if e2e:
        line["e2e"] = e2e
    if not args.no_cpu_baseline and not adjoint:
        line["cpu_baseline"] = cpu_baseline(args.workload, bank, x_host)
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


def main():
    args = parse()
    if args.workload == "design" and args.impl != "reference":
        return run_design(args) if int(os.environ.get("RANK", 0)) == 0 else 0
    if args.workload == "veto" and args.impl != "reference":
        return run_veto(args) if int(os.environ.get("RANK", 0)) == 0 else 0
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
