"""SPIIR filter bank on NVIDIA B300 (sm_103a): thin Python binding.

The compute path is the C-ABI library ``_lib/libspiir.so`` (declared in
``include/spiir.h``), built from ``csrc/`` by ``build.py``.  This module only
marshals arguments: numpy arrays for the bank (host), torch CUDA tensors for
strain, SNR series and gradients (device memory and streams).  Every step of
the filtering runs in the library's CUDA kernels; there is no CPU fallback,
and importing this package fails if the library is missing.

The method (paper, section "GPU accelerated SPIIR method", subsection "SPIIR
method"): each template is a bank of single-pole complex IIR filters
``y_l[k] = a_l y_l[k-1] + b_l x[k-d_l]`` summed into ``z[k] = sum_l y_l[k]``,
whose peak ``max_k |z[k]|`` flags a candidate signal.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libspiir.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"SPIIR CUDA library not built ({LIB_PATH} missing); run "
        "`python paper_1602_05573_b300/build.py` (nvcc, sm_103a)")

_lib = ctypes.CDLL(LIB_PATH)

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED = range(6)
PRECISIONS = {"plain": 0, "compensated": 1, "chunked_fp64": 2, "chunked_tc": 3}
PROJECTIONS = {"auto": 0, "recurrence": 1, "tensor": 2}
KERNEL_CLASSES = 3

# exported symbols (include/spiir.h)
SYMBOLS = [
    "spiir_options_default", "spiir_plan_create", "spiir_plan_destroy",
    "spiir_plan_get_info", "spiir_plan_get_slots", "spiir_reset", "spiir_filter",
    "spiir_peak", "spiir_filter_backward", "spiir_state_get", "spiir_state_set",
    "spiir_check", "spiir_selftest_bounded_wait", "spiir_status_str",
    "spiir_last_error_detail", "spiir_filter_noalloc", "spiir_set_coefficients",
    "spiir_network_peak", "spiir_set_band_fir", "spiir_chi2_peak", "spiir_chi2_split",
    "spiir_plan_tune_report",
]


class BankDesc(ctypes.Structure):
    _fields_ = [("n_templates", ctypes.c_int64), ("n_detectors", ctypes.c_int32),
                ("n_bands", ctypes.c_int32), ("filter_off", ctypes.c_void_p),
                ("a_reim", ctypes.c_void_p), ("b_reim", ctypes.c_void_p),
                ("delay", ctypes.c_void_p), ("band_of_filter", ctypes.c_void_p),
                ("band_decim", ctypes.c_void_p)]


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("chunk_len", ctypes.c_int32),
                ("block_len", ctypes.c_int32), ("warps_per_cta", ctypes.c_int32),
                ("ring_copies", ctypes.c_int32), ("device", ctypes.c_int32),
                ("autotune", ctypes.c_int32), ("max_filters_per_lane", ctypes.c_int32),
                ("lanes_per_template", ctypes.c_int32), ("time_segments", ctypes.c_int32),
                ("projection", ctypes.c_int32), ("kernel_timing", ctypes.c_int32),
                ("tile_chunks", ctypes.c_int32), ("persistent", ctypes.c_int32),
                ("tail_split", ctypes.c_int32), ("adjoint_form", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 1)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("n_templates", ctypes.c_int64), ("n_filters", ctypes.c_int64),
                ("n_slots", ctypes.c_int64), ("n_units", ctypes.c_int64),
                ("n_detectors", ctypes.c_int32), ("warps_per_cta", ctypes.c_int32),
                ("block_len", ctypes.c_int32), ("ring_copies", ctypes.c_int32),
                ("history_len", ctypes.c_int32), ("smem_bytes", ctypes.c_int32),
                ("max_filters_per_lane", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("bank_conflict_ratio", ctypes.c_double),
                ("lanes_per_template", ctypes.c_int32), ("last_call_launches", ctypes.c_int32),
                ("last_call_segments", ctypes.c_int32), ("persistent", ctypes.c_int32),
                ("tail_templates", ctypes.c_int64), ("resident_ctas", ctypes.c_int64)]


_P = ctypes.c_void_p
_st = ctypes.c_int


def _configure(lib):
    """Declare the C signatures of include/spiir.h on a loaded library."""
    lib.spiir_options_default.argtypes = [ctypes.POINTER(Options)]
    lib.spiir_options_default.restype = None
    lib.spiir_plan_create.argtypes = [ctypes.POINTER(BankDesc), ctypes.POINTER(Options),
                                       ctypes.POINTER(_P)]
    lib.spiir_plan_create.restype = _st
    lib.spiir_plan_destroy.argtypes = [_P]
    lib.spiir_plan_destroy.restype = _st
    lib.spiir_plan_get_info.argtypes = [_P, ctypes.POINTER(PlanInfo)]
    lib.spiir_plan_get_info.restype = _st
    lib.spiir_plan_tune_report.argtypes = [_P]
    lib.spiir_plan_tune_report.restype = ctypes.c_char_p
    lib.spiir_plan_get_slots.argtypes = [_P, _P, _P]
    lib.spiir_plan_get_slots.restype = _st
    lib.spiir_reset.argtypes = [_P, _P]
    lib.spiir_reset.restype = _st
    lib.spiir_filter.argtypes = [_P, _P, ctypes.c_int64, _P, _P]
    lib.spiir_filter.restype = _st
    lib.spiir_peak.argtypes = [_P, _P, _P, _P]
    lib.spiir_peak.restype = _st
    lib.spiir_filter_backward.argtypes = [_P, _P, ctypes.c_int64, _P, _P, _P, _P, _P]
    lib.spiir_filter_backward.restype = _st
    lib.spiir_network_peak.argtypes = [_P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, _P,
                                       _P, _P, _P, _P]
    lib.spiir_network_peak.restype = _st
    lib.spiir_set_band_fir.argtypes = [_P, ctypes.c_int32, _P, ctypes.c_int32]
    lib.spiir_set_band_fir.restype = _st
    lib.spiir_chi2_peak.argtypes = [_P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32,
                                    ctypes.c_int64, _P, _P, _P, _P]
    lib.spiir_chi2_peak.restype = _st
    lib.spiir_chi2_split.argtypes = [ctypes.POINTER(BankDesc), ctypes.c_int32, _P, _P, _P, _P,
                                     _P]
    lib.spiir_chi2_split.restype = _st
    lib.spiir_state_get.argtypes = [_P, _P, _P, ctypes.POINTER(ctypes.c_int64)]
    lib.spiir_state_get.restype = _st
    lib.spiir_state_set.argtypes = [_P, _P, _P, ctypes.c_int64]
    lib.spiir_state_set.restype = _st
    lib.spiir_check.argtypes = [_P, _P]
    lib.spiir_check.restype = _st
    lib.spiir_selftest_bounded_wait.argtypes = [_P, ctypes.c_uint64, _P]
    lib.spiir_selftest_bounded_wait.restype = _st
    lib.spiir_set_coefficients.argtypes = [_P, _P, _P, _P]
    lib.spiir_set_coefficients.restype = _st
    lib.spiir_filter_noalloc.argtypes = [ctypes.POINTER(BankDesc), _P, ctypes.c_int64, _P, _P,
                                          _P, _P]
    lib.spiir_filter_noalloc.restype = _st
    lib.spiir_status_str.argtypes = [_st]
    lib.spiir_status_str.restype = ctypes.c_char_p
    lib.spiir_last_error_detail.argtypes = []
    lib.spiir_last_error_detail.restype = ctypes.c_char_p
    if hasattr(lib, "spiir_kernel_times"):
        lib.spiir_kernel_times.argtypes = [_P, _P, _P]
        lib.spiir_kernel_times.restype = _st
    return lib


def load_library(path: str):
    """Load and configure a build of the SPIIR library (e.g. another build
    of the same sources); the package itself uses LIB_PATH."""
    return _configure(ctypes.CDLL(path))


_configure(_lib)


class SpiirError(RuntimeError):
    def __init__(self, status: int, where: str, lib=None):
        lib = lib if lib is not None else _lib
        self.status = status
        detail = lib.spiir_last_error_detail().decode()
        super().__init__(f"{where}: {lib.spiir_status_str(status).decode()}"
                         + (f" ({detail})" if detail else ""))


def _check(status: int, where: str, lib=None):
    if status != OK:
        raise SpiirError(status, where, lib)


def library():
    """The loaded ctypes library (for tests that call the C-ABI directly)."""
    return _lib


def _ptr(arr) -> Optional[int]:
    if arr is None:
        return None
    if hasattr(arr, "data_ptr"):
        return arr.data_ptr()
    return arr.ctypes.data


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def bank_desc(bank):
    """(BankDesc, keep-alive arrays) for a bank object (see Plan)."""
    off = np.ascontiguousarray(bank.off, np.int64)
    a = np.ascontiguousarray(bank.a, np.complex64).view(np.float32)
    b = np.ascontiguousarray(bank.b, np.complex64).view(np.float32)
    d = np.ascontiguousarray(bank.d, np.int32)
    keep = [off, a, b, d]
    desc = BankDesc()
    desc.n_templates = off.shape[0] - 1
    desc.n_detectors = int(bank.n_det)
    desc.filter_off, desc.a_reim, desc.b_reim, desc.delay = (
        _ptr(off), _ptr(a), _ptr(b), _ptr(d))
    band_of = getattr(bank, "band_of", None)
    decim = getattr(bank, "decim", None)
    if band_of is not None and decim is not None and len(decim) > 1:
        band_of = np.ascontiguousarray(band_of, np.int32)
        decim = np.ascontiguousarray(decim, np.int32)
        keep += [band_of, decim]
        desc.n_bands = int(decim.shape[0])
        desc.band_of_filter, desc.band_decim = _ptr(band_of), _ptr(decim)
    return desc, keep


def filter_noalloc(bank, x, z=None, peak_abs=None, peak_idx=None, *, emit_z=True,
                   stream=None):
    """One-shot filter call through spiir_filter_noalloc (no device
    allocation inside the library; the outputs are allocated here by torch
    unless passed in).  Returns (z or None, peak_abs, peak_idx)."""
    import torch
    desc, keep = bank_desc(bank)
    D, n = x.shape
    T = int(desc.n_templates)
    if emit_z and z is None:
        z = torch.empty((D, T, n), dtype=torch.complex64, device=x.device)
    if peak_abs is None:
        peak_abs = torch.empty((D, T), dtype=torch.float32, device=x.device)
    if peak_idx is None:
        peak_idx = torch.empty((D, T), dtype=torch.int64, device=x.device)
    _check(_lib.spiir_filter_noalloc(ctypes.byref(desc), _ptr(x), n,
                                     _ptr(z) if z is not None else None, _ptr(peak_abs),
                                     _ptr(peak_idx), _stream_handle(stream)),
           "spiir_filter_noalloc")
    del keep
    return z, peak_abs, peak_idx


class Plan:
    """A SPIIR bank prepared for the GPU (or host-only, device=-1).

    bank: object with numpy fields off (int64 [T+1]), a, b (complex64 [Ltot]),
    d (int32 [Ltot]), n_det, and optionally band_of (int32 [Ltot]) and
    decim (int32 [n_bands]).
    """

    def __init__(self, bank, *, precision: str = "plain", device: int = 0,
                 block_len: int = 0, warps_per_cta: int = 0, ring_copies: int = 0,
                 chunk_len: int = 256, autotune: bool = False,
                 max_filters_per_lane: int = 0, lanes_per_template: int = 0,
                 time_segments: int = 0, projection: str = "auto",
                 kernel_timing: bool = False, tile_chunks: int = 0, persistent: str = "auto",
                 tail_split: int = 0, adjoint_form: str = "auto", lib=None):
        self._h = None
        self._lib = lib if lib is not None else _lib
        off = np.ascontiguousarray(bank.off, np.int64)
        a = np.ascontiguousarray(bank.a, np.complex64).view(np.float32)
        b = np.ascontiguousarray(bank.b, np.complex64).view(np.float32)
        d = np.ascontiguousarray(bank.d, np.int32)
        band_of = getattr(bank, "band_of", None)
        decim = getattr(bank, "decim", None)
        self._keep = [off, a, b, d]
        desc = BankDesc()
        desc.n_templates = off.shape[0] - 1
        desc.n_detectors = int(bank.n_det)
        desc.filter_off, desc.a_reim, desc.b_reim, desc.delay = (
            _ptr(off), _ptr(a), _ptr(b), _ptr(d))
        if band_of is not None and decim is not None and len(decim) > 1:
            band_of = np.ascontiguousarray(band_of, np.int32)
            decim = np.ascontiguousarray(decim, np.int32)
            self._keep += [band_of, decim]
            desc.n_bands = int(decim.shape[0])
            desc.band_of_filter, desc.band_decim = _ptr(band_of), _ptr(decim)
        opt = Options()
        self._lib.spiir_options_default(ctypes.byref(opt))
        opt.precision = PRECISIONS[precision]
        opt.device = int(device)
        opt.block_len = int(block_len)
        opt.warps_per_cta = int(warps_per_cta)
        opt.ring_copies = int(ring_copies)
        opt.chunk_len = int(chunk_len)
        opt.autotune = int(bool(autotune))
        opt.max_filters_per_lane = int(max_filters_per_lane)
        opt.lanes_per_template = int(lanes_per_template)
        opt.time_segments = int(time_segments)
        opt.projection = PROJECTIONS[projection]
        opt.kernel_timing = 1 if kernel_timing else 0
        opt.tile_chunks = int(tile_chunks)
        opt.persistent = {"auto": 0, "off": 1, "on": 2}[persistent]
        opt.tail_split = int(tail_split)
        opt.adjoint_form = {"auto": 0, "reverse": 1, "tangent": 2}[adjoint_form]
        h = _P()
        _check(self._lib.spiir_plan_create(ctypes.byref(desc), ctypes.byref(opt), ctypes.byref(h)),
               "spiir_plan_create", self._lib)
        self._h = h
        self.device = int(device)
        self.n_templates = int(desc.n_templates)
        self.n_det = int(bank.n_det)
        self.n_filters = int(off[-1])

    # -- lifecycle ------------------------------------------------------------
    def close(self):
        if self._h is not None and self._h.value:
            self._lib.spiir_plan_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        inf = PlanInfo()
        _check(self._lib.spiir_plan_get_info(self._h, ctypes.byref(inf)), "spiir_plan_get_info", self._lib)
        return {name: getattr(inf, name) for name, _ in PlanInfo._fields_
                if name != "reserved"}

    def tune_report(self) -> str:
        """The autotuner's timing per candidate layout ("" if it has not run)."""
        return self._lib.spiir_plan_tune_report(self._h).decode()

    def slots(self):
        n = self.info()["n_slots"]
        sf = np.empty(n, np.int64)
        st = np.empty(n, np.int64)
        _check(self._lib.spiir_plan_get_slots(self._h, _ptr(sf), _ptr(st)), "spiir_plan_get_slots", self._lib)
        return sf, st

    # -- streaming ------------------------------------------------------------
    def reset(self, stream=None):
        _check(self._lib.spiir_reset(self._h, _stream_handle(stream)), "spiir_reset", self._lib)

    def filter(self, x, z=None, *, emit_z: bool = True, stream=None):
        """Filter the next samples.  x: CUDA float32 [D][n] (contiguous).
        Returns z (complex64 [D][T][n]) or None when emit_z is False."""
        import torch
        assert x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()
        D, n = x.shape
        assert D == self.n_det
        if emit_z and z is None:
            z = torch.empty((D, self.n_templates, n), dtype=torch.complex64, device=x.device)
        if z is not None:
            assert z.is_cuda and z.dtype == torch.complex64 and z.is_contiguous()
            assert tuple(z.shape) == (D, self.n_templates, n)
        _check(self._lib.spiir_filter(self._h, _ptr(x), n, _ptr(z) if z is not None else None,
                                 _stream_handle(stream)), "spiir_filter", self._lib)
        return z

    def peak(self, out_abs=None, out_idx=None, *, stream=None):
        """Running peak since reset: (abs float32 [D][T], idx int64 [D][T]) on the GPU."""
        import torch
        dev = torch.device("cuda", self.device)
        if out_abs is None:
            out_abs = torch.empty((self.n_det, self.n_templates), dtype=torch.float32, device=dev)
        if out_idx is None:
            out_idx = torch.empty((self.n_det, self.n_templates), dtype=torch.int64, device=dev)
        _check(self._lib.spiir_peak(self._h, _ptr(out_abs), _ptr(out_idx), _stream_handle(stream)),
               "spiir_peak", self._lib)
        return out_abs, out_idx

    def capture(self, x, z=None, peak_abs=None, peak_idx=None, *, emit_z: bool = True,
                warmup: bool = True):
        """Record one spiir_filter + spiir_peak call on fixed buffers into a
        CUDA graph; each replay() filters the next len(x) samples of the
        stream (the sample counter lives on the device).  The warm-up call
        (which allocates workspace outside the capture) advances the stream;
        reset() afterwards to start from zero.  Returns (graph, z, abs, idx)."""
        import torch
        D, n = x.shape
        if emit_z and z is None:
            z = torch.empty((D, self.n_templates, n), dtype=torch.complex64, device=x.device)
        if peak_abs is None:
            peak_abs = torch.empty((D, self.n_templates), dtype=torch.float32, device=x.device)
        if peak_idx is None:
            peak_idx = torch.empty((D, self.n_templates), dtype=torch.int64, device=x.device)
        side = torch.cuda.Stream(device=x.device)
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            if warmup:
                self.filter(x, z, emit_z=emit_z, stream=side)
                self.peak(peak_abs, peak_idx, stream=side)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize(x.device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            cur = torch.cuda.current_stream()
            self.filter(x, z, emit_z=emit_z, stream=cur)
            self.peak(peak_abs, peak_idx, stream=cur)
        return g, z, peak_abs, peak_idx

    def backward(self, x, grad_z, *, want_gx: bool = True, stream=None):
        """VJP of one zero-state filter call: (g_a, g_b complex64 [Ltot], g_x float32 [D][n])."""
        import torch
        D, n = x.shape
        ga = torch.empty(self.n_filters, dtype=torch.complex64, device=x.device)
        gb = torch.empty(self.n_filters, dtype=torch.complex64, device=x.device)
        gx = torch.empty((D, n), dtype=torch.float32, device=x.device) if want_gx else None
        gz = grad_z.contiguous()
        _check(self._lib.spiir_filter_backward(self._h, _ptr(x), n, _ptr(gz), _ptr(ga), _ptr(gb),
                                          _ptr(gx), _stream_handle(stream)),
               "spiir_filter_backward", self._lib)
        return ga, gb, gx

    def set_band_fir(self, band: int, taps):
        """Front end of band `band`: x_band[k] = sum_i taps[i] x[R k - i]
        (whitening / anti-aliasing before subsampling); None or [] restores
        plain subsampling."""
        t = np.ascontiguousarray(np.zeros(0) if taps is None else taps, np.float32).ravel()
        _check(self._lib.spiir_set_band_fir(self._h, int(band), t.ctypes.data if t.size else None,
                                            int(t.size)), "spiir_set_band_fir", self._lib)

    def set_coefficients(self, a, b, *, stream=None):
        """Replace every filter's pole and gain: a, b CUDA complex64 [Ltot]."""
        import torch
        a = a.detach().to(torch.complex64).contiguous()
        b = b.detach().to(torch.complex64).contiguous()
        assert a.is_cuda and b.is_cuda and a.numel() == b.numel() == self.n_filters
        _check(self._lib.spiir_set_coefficients(self._h, _ptr(a), _ptr(b),
                                                _stream_handle(stream)),
               "spiir_set_coefficients", self._lib)

    def state_get(self):
        inf = self.info()
        st = np.zeros((self.n_det, self.n_filters), np.complex64)
        hist = np.zeros((self.n_det, inf["history_len"]), np.float32)
        t = ctypes.c_int64()
        _check(self._lib.spiir_state_get(self._h, _ptr(st), _ptr(hist), ctypes.byref(t)),
               "spiir_state_get", self._lib)
        return st, hist, int(t.value)

    def state_set(self, state, history, samples):
        state = np.ascontiguousarray(state, np.complex64)
        history = np.ascontiguousarray(history, np.float32)
        _check(self._lib.spiir_state_set(self._h, _ptr(state), _ptr(history), int(samples)),
               "spiir_state_set", self._lib)

    def kernel_times(self) -> dict:
        """Device milliseconds and launch counts per kernel class since the last
        read (plans made with kernel_timing=True): filter, tensor-core
        projection, adjoint reverse pass."""
        ms = (ctypes.c_double * KERNEL_CLASSES)()
        n = (ctypes.c_int64 * KERNEL_CLASSES)()
        _check(self._lib.spiir_kernel_times(self._h, ms, n), "spiir_kernel_times", self._lib)
        return {name: (ms[i], n[i]) for i, name in enumerate(("filter", "projection", "adjoint"))}

    def check(self, stream=None):
        """Wait for the plan's work; raise SpiirError(ETIMEOUT) if a bounded wait gave up."""
        _check(self._lib.spiir_check(self._h, _stream_handle(stream)), "spiir_check", self._lib)


def _autograd_function():
    import torch

    class SpiirFilterFunction(torch.autograd.Function):
        """z = SPIIR bank (poles a, gains b, the plan's delays) applied to x
        from zero state; backward runs spiir_filter_backward (the adjoint
        kernel).  Gradients follow PyTorch's complex convention."""

        @staticmethod
        def forward(ctx, x, a, b, plan):
            plan.set_coefficients(a, b)
            plan.reset()
            z = plan.filter(x.contiguous())
            ctx.save_for_backward(x)
            ctx.plan = plan
            return z

        @staticmethod
        def backward(ctx, gz):
            (x,) = ctx.saved_tensors
            ga, gb, gx = ctx.plan.backward(x.contiguous(), gz.contiguous(),
                                          want_gx=ctx.needs_input_grad[0])
            return gx, ga, gb, None

    return SpiirFilterFunction


def network_peak(z, window, *, want_shift: bool = True, stream=None, lib=None):
    """Network peak across detectors through spiir_network_peak: z CUDA
    complex64 [D][T][n] (spiir_filter's layout), window ints [D] (offsets
    allowed per detector, window[0] ignored).  Returns (rho float32 [T],
    t int64 [T], shift int32 [T][D] or None)."""
    import torch
    lib = lib or library()
    assert z.is_cuda and z.dtype == torch.complex64 and z.dim() == 3
    z = z.contiguous()
    D, T, n = z.shape
    w = np.ascontiguousarray(np.asarray(window, np.int32).reshape(D))
    rho = torch.empty(T, dtype=torch.float32, device=z.device)
    t = torch.empty(T, dtype=torch.int64, device=z.device)
    shift = torch.empty((T, D), dtype=torch.int32, device=z.device) if want_shift else None
    with torch.cuda.device(z.device):
        _check(lib.spiir_network_peak(_ptr(z), D, T, n, w.ctypes.data, _ptr(rho), _ptr(t),
                                      _ptr(shift), _stream_handle(stream)),
               "spiir_network_peak", lib)
    return rho, t, shift


def chi2_split(bank, n_bins: int, *, lib=None):
    """The bank regrouped for the chi^2 veto by spiir_chi2_split: every
    template's filters, ordered by frequency arg(a), cut into n_bins
    contiguous bins of (as nearly as whole filters allow) equal
    impulse-response energy; bin i of template t becomes template
    t * n_bins + i (empty bins stay empty).  Returns a bank object (off, a,
    b, d, n_det, and filter_of: the bank filter at each position) for Plan;
    spiir_filter on it writes the bin series [D][T][n_bins][n] that
    chi2_peak reads.  Bins of a large bank run faster in half warps
    (Plan(..., lanes_per_template=16)) when every bin fits 160 filters."""
    import types
    lib = lib or library()
    desc, keep = bank_desc(bank)
    T = int(desc.n_templates)
    ltot = int(keep[0][-1])
    off = np.empty(T * int(n_bins) + 1, np.int64)
    filter_of = np.empty(max(ltot, 1), np.int64)
    a = np.empty(max(ltot, 1), np.complex64)
    b = np.empty(max(ltot, 1), np.complex64)
    d = np.empty(max(ltot, 1), np.int32)
    _check(lib.spiir_chi2_split(ctypes.byref(desc), int(n_bins), _ptr(off), _ptr(filter_of),
                                _ptr(a), _ptr(b), _ptr(d)), "spiir_chi2_split", lib)
    del keep
    return types.SimpleNamespace(off=off, a=a[:ltot], b=b[:ltot], d=d[:ltot],
                                 filter_of=filter_of[:ltot], n_det=int(bank.n_det))


def chi2_peak(zg, n_bins: int, *, stream=None, lib=None):
    """spiir_chi2_peak: zg CUDA complex64 [D][T * n_bins][n] (or [D][T][n_bins][n]).
    Returns (peak float32 [D][T], t int64 [D][T], chi2 float32 [D][T])."""
    import torch
    lib = lib or library()
    assert zg.is_cuda and zg.dtype == torch.complex64
    zg = zg.contiguous()
    D, n = zg.shape[0], zg.shape[-1]
    T = zg.numel() // (D * n * n_bins)
    peak = torch.empty((D, T), dtype=torch.float32, device=zg.device)
    t = torch.empty((D, T), dtype=torch.int64, device=zg.device)
    chi2 = torch.empty((D, T), dtype=torch.float32, device=zg.device)
    with torch.cuda.device(zg.device):
        _check(lib.spiir_chi2_peak(_ptr(zg), D, T, int(n_bins), n, _ptr(peak), _ptr(t),
                                   _ptr(chi2), _stream_handle(stream)), "spiir_chi2_peak", lib)
    return peak, t, chi2


def spiir_filter(x, a, b, plan):
    """Differentiable filter: z[D][T][n] from strain x[D][n] (float32) and
    complex64 coefficient tensors a, b [Ltot] (bank order).  The plan fixes
    the bank's structure and delays; its streaming state is reset."""
    return _autograd_function().apply(x, a, b, plan)
