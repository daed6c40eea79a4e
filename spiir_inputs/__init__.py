"""Seeded synthetic workloads for the SPIIR filter bank.

This module only draws random numbers: filter poles, gains and delays, and
white-noise detector streams.  It holds none of the filtering arithmetic, so
both the FP64 oracle (tests) and the CUDA path (tests, bench) can take their
inputs from it without sharing any of the method's code.

Recipe (shapes of the paper's SPIIR workloads: one complex single-pole filter
bank per template, whitened detector strain as input):
  pole    a = r * exp(i w), r ~ U(r_lo, r_hi), w ~ U(0, pi), drawn in float64
          and rounded once to complex64 (the canonical value both sides use)
  gain    b ~ CN(0, 1) / 64, i.e. Re, Im ~ N(0, 1/2) / 64, rounded to complex64
  delay   d ~ U{0 .. d_max} (integer samples at the filter's band rate)
  strain  x ~ N(0, 1) float32, independent per detector
RNG: numpy default_rng (PCG64) with a fixed seed per workload.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np


@dataclass
class Bank:
    """A template bank in CSR form (filters of template t: off[t]..off[t+1])."""
    off: np.ndarray                 # int64 [T+1]
    a: np.ndarray                   # complex64 [Ltot] poles
    b: np.ndarray                   # complex64 [Ltot] gains
    d: np.ndarray                   # int32 [Ltot] delays (band samples)
    n_det: int = 1
    band_of: Optional[np.ndarray] = None   # int32 [Ltot] (multirate only)
    decim: Optional[np.ndarray] = None     # int32 [n_bands], 1 = top rate
    # float64 draws behind a and b, kept for seeded perturbations
    r64: Optional[np.ndarray] = field(default=None, repr=False)
    w64: Optional[np.ndarray] = field(default=None, repr=False)
    b64: Optional[np.ndarray] = field(default=None, repr=False)

    @property
    def n_templates(self) -> int:
        return int(self.off.shape[0] - 1)

    @property
    def n_filters(self) -> int:
        return int(self.off[-1])

    def counts(self) -> np.ndarray:
        return np.diff(self.off)

    def subset(self, templates) -> "Bank":
        """The bank restricted to the given template indices (in that order)."""
        templates = np.asarray(templates, np.int64)
        idx = np.concatenate([np.arange(self.off[t], self.off[t + 1]) for t in templates]) \
            if len(templates) else np.zeros(0, np.int64)
        counts = self.counts()[templates]
        off = np.zeros(len(templates) + 1, np.int64)
        off[1:] = np.cumsum(counts)
        pick = (lambda v: None if v is None else v[idx])
        return Bank(off, self.a[idx], self.b[idx], self.d[idx], self.n_det,
                    pick(self.band_of), self.decim, pick(self.r64), pick(self.w64),
                    pick(self.b64))


def _draw_filters(rng, n, r_range, d_max):
    r = rng.uniform(r_range[0], r_range[1], n)
    w = rng.uniform(0.0, np.pi, n)
    b = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) * np.sqrt(0.5) / 64.0
    d = rng.integers(0, d_max + 1, n).astype(np.int32)
    return r, w, b, d


def _finish(r, w, b, d, counts, n_det, band_of=None, decim=None) -> Bank:
    off = np.zeros(len(counts) + 1, np.int64)
    off[1:] = np.cumsum(counts)
    a = (r * np.exp(1j * w)).astype(np.complex64)
    return Bank(off, a, b.astype(np.complex64), d, n_det, band_of, decim, r, w, b)


def make_bank(n_templates: int, filters, r_range, d_max: int, seed: int,
              n_det: int = 1) -> Bank:
    """Single-rate bank.  `filters` is an int (same count everywhere) or an
    inclusive (lo, hi) range drawn uniformly per template."""
    rng = np.random.default_rng(seed)
    if isinstance(filters, (tuple, list)):
        counts = rng.integers(filters[0], filters[1] + 1, n_templates)
    else:
        counts = np.full(n_templates, int(filters))
    r, w, b, d = _draw_filters(rng, int(counts.sum()), r_range, d_max)
    return _finish(r, w, b, d, counts, n_det)


def make_multirate_bank(n_templates: int, band_filters, decim, r_range, d_max: int,
                        seed: int, n_det: int = 1) -> Bank:
    """Multirate bank: every template has band_filters[j] filters in band j,
    which runs at the top rate divided by decim[j]."""
    rng = np.random.default_rng(seed)
    per_t = int(sum(band_filters))
    counts = np.full(n_templates, per_t)
    r, w, b, d = _draw_filters(rng, per_t * n_templates, r_range, d_max)
    one = np.concatenate([np.full(c, j, np.int32) for j, c in enumerate(band_filters)])
    band_of = np.tile(one, n_templates)
    return _finish(r, w, b, d, counts, n_det, band_of, np.asarray(decim, np.int32))


def perturb(bank: Bank, seed: int, rel: float = 0.01) -> Bank:
    """Seeded +-rel perturbation of every pole and gain, keeping |a| < 1:
    r' = 1 - (1 - r)(1 + rel u1), w' = w (1 + rel u2), b' = b (1 + rel (u3 + i u4)),
    u ~ U(-1, 1)."""
    rng = np.random.default_rng(seed)
    n = bank.n_filters
    u = rng.uniform(-1.0, 1.0, (4, n))
    r = 1.0 - (1.0 - bank.r64) * (1.0 + rel * u[0])
    w = bank.w64 * (1.0 + rel * u[1])
    b = bank.b64 * (1.0 + rel * (u[2] + 1j * u[3]))
    return _finish(r, w, b, bank.d.copy(), bank.counts(), bank.n_det,
                   bank.band_of, bank.decim)


def chirp_template(rate: float, f_lo: float, f_hi: float, f0: float = 135.0) -> np.ndarray:
    """Synthetic inspiral chirp from f_lo to f_hi Hz at `rate` samples/s,
    complex128, time running forward: frequency f(tau) = f0 tau^(-3/8) at
    tau seconds before coalescence (the leading-order chirp; f0 ~ 135 Hz for
    a 1.2 solar-mass chirp mass), phase 2 pi times its integral, amplitude
    growing as f^(2/3).  A stand-in waveform: no waveform library exists here."""
    tau_lo = (f0 / f_lo) ** (8.0 / 3.0)
    tau_hi = (f0 / f_hi) ** (8.0 / 3.0)
    n = int(np.ceil((tau_lo - tau_hi) * rate))
    tau = tau_lo - np.arange(n) / rate
    phase = -2.0 * np.pi * f0 * (8.0 / 5.0) * tau ** (5.0 / 8.0)
    amp = (tau / tau_lo) ** (-0.25)
    return amp * np.exp(1j * phase)


def make_strain(n_det: int, n: int, seed: int) -> np.ndarray:
    """White N(0, 1) float32 noise, [n_det][n] (whitened detector strain)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n_det, n), dtype=np.float64).astype(np.float32)


# ---------------------------------------------------------------------------
# The five workloads.  Each entry: bank builder kwargs, strain length, rate.
# ---------------------------------------------------------------------------
WORKLOADS = {
    # 16 templates x 64 filters, 1 detector, 16384 samples at 4096 Hz
    "plain": dict(kind="single", n_templates=16, filters=64, r_range=(0.99, 0.9995),
                  d_max=1024, n_det=1, n=16384, rate=4096, seed=101),
    # 4096 templates, 100..300 filters, 3 detectors, 65536 samples at 1024 Hz
    "batched": dict(kind="single", n_templates=4096, filters=(100, 300),
                    r_range=(0.99, 0.9999), d_max=4096, n_det=3, n=65536, rate=1024,
                    seed=202),
    # 2048 templates x (60 @ 4096 Hz, 120 @ 1024 Hz, 120 @ 256 Hz), 256 s
    "multirate": dict(kind="multirate", n_templates=2048, band_filters=(60, 120, 120),
                      decim=(1, 4, 16), r_range=(0.99, 0.9995), d_max=1024, n_det=1,
                      n=1 << 20, rate=4096, seed=303),
    # 16384 templates x 200 filters, poles very close to the unit circle, 2^20 samples
    "precision": dict(kind="single", n_templates=16384, filters=200,
                      r_range=(0.9999, 0.999995), d_max=1024, n_det=1, n=1 << 20,
                      rate=1024, seed=404),
    # 256 templates x 200 filters, 65536 samples at 1024 Hz (adjoint)
    "adjoint": dict(kind="single", n_templates=256, filters=200, r_range=(0.99, 0.9995),
                    d_max=1024, n_det=1, n=65536, rate=1024, seed=505),
}


def workload_bank(name: str, n_templates: Optional[int] = None) -> Bank:
    """The named workload's bank; n_templates truncates it (same draws for the
    templates kept only when the filter count is fixed)."""
    w = WORKLOADS[name]
    nt = w["n_templates"] if n_templates is None else int(n_templates)
    if w["kind"] == "multirate":
        return make_multirate_bank(nt, w["band_filters"], w["decim"], w["r_range"],
                                   w["d_max"], w["seed"], w["n_det"])
    return make_bank(nt, w["filters"], w["r_range"], w["d_max"], w["seed"], w["n_det"])


def workload_strain(name: str, n: Optional[int] = None) -> np.ndarray:
    w = WORKLOADS[name]
    return make_strain(w["n_det"], w["n"] if n is None else int(n), w["seed"] + 1)


def updates(bank: Bank, n: int) -> int:
    """Filter updates (one complex recurrence step) for an n-sample call."""
    if bank.band_of is None:
        return int(bank.n_filters) * int(bank.n_det) * int(n)
    total = 0
    for j, R in enumerate(bank.decim):
        nb = (int(n) + int(R) - 1) // int(R)
        total += int(np.count_nonzero(bank.band_of == j)) * nb
    return total * int(bank.n_det)
