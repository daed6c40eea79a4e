"""FP64 CPU oracle for the SPIIR hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path
(``paper_1602_05573_b300``) and neither imports the other.

What it computes (paper, section "GPU accelerated SPIIR method", subsection
"SPIIR method"): each template is a parallel bank of single-pole complex IIR
filters ``y_l[k] = a_l y_l[k-1] + b_l x[k-d_l]`` whose outputs are summed into
the template's SNR series ``z[k] = sum_l y_l[k]``; the peak is the largest
``|z|`` (first index on ties).  The arithmetic lives in ``spiir_ref.c`` as
plain double-precision loops; this module only compiles it with gcc and
marshals numpy arrays.

Every function here is pinned by ``tests/test_oracle_pins.py`` against
closed forms, brute force and exact rational arithmetic.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spiir_ref.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libspiir_ref.so")
_lock = threading.Lock()
_lib = None

# planted mistakes understood by spiir_ref_filter (mutation tests only)
MUTATIONS = {
    "conj_pole": 1,
    "delay_off_by_one": 2,
    "drop_gain_imag": 3,
    "skip_last_filter": 4,
    "peak_last_on_tie": 5,
    "swap_re_im_out": 6,
}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FMA contraction, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-std=c99", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64 = ctypes.c_int64
            lib.spiir_ref_filter.argtypes = [i64, i64, P, P, P, P, P, i64, P, P, P,
                                             ctypes.c_int, ctypes.c_int]
            lib.spiir_ref_filter.restype = ctypes.c_int
            lib.spiir_ref_filter_multirate.argtypes = [
                i64, i64, P, P, P, P, P, ctypes.c_int32, P, P, i64, P, P, P, ctypes.c_int]
            lib.spiir_ref_filter_multirate.restype = ctypes.c_int
            lib.spiir_ref_adjoint.argtypes = [i64, i64, P, P, P, P, P, i64, P, P, P, P,
                                              ctypes.c_int]
            lib.spiir_ref_adjoint.restype = ctypes.c_int
            lib.spiir_ref_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().spiir_ref_max_threads())


def _ptr(arr):
    return None if arr is None else arr.ctypes.data_as(ctypes.c_void_p)


def _as_reim(v) -> np.ndarray:
    """complex array -> contiguous float64 [N][2], promoted exactly."""
    v = np.asarray(v)
    out = np.empty((v.shape[0], 2), np.float64)
    out[:, 0] = v.real
    out[:, 1] = v.imag
    return out


def _bank_arrays(off, a, b, d):
    off = np.ascontiguousarray(off, np.int64)
    return (off, _as_reim(a), _as_reim(b), np.ascontiguousarray(d, np.int32))


def filter_bank(off, a, b, d, x, *, want_z=True, n_threads=None, mutation=0):
    """Summed single-rate IIR bank on every detector stream.

    off: int64 [T+1] CSR offsets; a, b: complex [Ltot]; d: int [Ltot];
    x: real [D][n].  Returns (z, peak_abs2, peak_idx): z complex128
    [D][T][n] (None unless want_z), peak_abs2 float64 [D][T] (largest |z|^2),
    peak_idx int64 [D][T] (first index attaining it).
    """
    lib = _load()
    off, a2, b2, d = _bank_arrays(off, a, b, d)
    x = np.ascontiguousarray(np.atleast_2d(x), np.float64)
    D, n = x.shape
    T = off.shape[0] - 1
    z = np.zeros((D, T, n, 2), np.float64) if want_z else None
    pa = np.zeros((D, T), np.float64)
    pi = np.zeros((D, T), np.int64)
    nt = n_threads or max_threads()
    rc = lib.spiir_ref_filter(T, D, _ptr(off), _ptr(a2), _ptr(b2), _ptr(d), _ptr(x), n,
                              _ptr(z), _ptr(pa), _ptr(pi), nt, int(mutation))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    zc = None if z is None else (z[..., 0] + 1j * z[..., 1])
    return zc, pa, pi


def filter_multirate(off, a, b, d, band_of, decim, x, *, want_z=True, n_threads=None):
    """Multirate bank: each band filtered at its own rate (plain subsampling
    by decim[band]), linearly interpolated back to the top rate, summed."""
    lib = _load()
    off, a2, b2, d = _bank_arrays(off, a, b, d)
    band_of = np.ascontiguousarray(band_of, np.int32)
    decim = np.ascontiguousarray(decim, np.int32)
    x = np.ascontiguousarray(np.atleast_2d(x), np.float64)
    D, n = x.shape
    T = off.shape[0] - 1
    z = np.zeros((D, T, n, 2), np.float64) if want_z else None
    pa = np.zeros((D, T), np.float64)
    pi = np.zeros((D, T), np.int64)
    nt = n_threads or max_threads()
    rc = lib.spiir_ref_filter_multirate(T, D, _ptr(off), _ptr(a2), _ptr(b2), _ptr(d),
                                        _ptr(band_of), int(decim.shape[0]), _ptr(decim),
                                        _ptr(x), n, _ptr(z), _ptr(pa), _ptr(pi), nt)
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    zc = None if z is None else (z[..., 0] + 1j * z[..., 1])
    return zc, pa, pi


def band_input(x, taps):
    """Front end of one band at the top rate, before its subsampling: the
    causal FIR sum_i taps[i] x[k - i] (x[< 0] = 0; whitening and/or
    anti-aliasing), float64.  x: [D][n]."""
    x = np.atleast_2d(np.asarray(x, np.float64))
    taps = np.asarray(taps, np.float64)
    n = x.shape[1]
    return np.stack([np.convolve(row, taps)[:n] for row in x])


def filter_multirate_fir(off, a, b, d, band_of, decim, x, band_fir, *, n_threads=None):
    """Multirate bank whose band j sees its front end's output subsampled,
    sum_i band_fir[j][i] x[R_j k - i] (None: plain subsampling x[R_j k]).
    Bands are independent until their interpolated sums add, so each band
    runs through filter_multirate alone on its own top-rate input and the
    band results are summed (float64).  Returns z complex128 [D][T][n]."""
    off = np.asarray(off, np.int64)
    band_of = np.asarray(band_of, np.int32)
    x = np.atleast_2d(np.asarray(x, np.float64))
    T = off.shape[0] - 1
    z = 0.0
    for j in range(len(decim)):
        keep = band_of == j
        counts = np.array([int(keep[off[t]:off[t + 1]].sum()) for t in range(T)], np.int64)
        off_j = np.concatenate([[0], np.cumsum(counts)])
        xj = x if band_fir[j] is None else band_input(x, band_fir[j])
        zj, _, _ = filter_multirate(off_j, np.asarray(a)[keep], np.asarray(b)[keep],
                                    np.asarray(d)[keep], band_of[keep], decim, xj,
                                    n_threads=n_threads)
        z = z + zj
    return z


def adjoint(off, a, b, d, x, gz, *, want_gx=True, n_threads=None):
    """Vector-Jacobian product of filter_bank: given g_z (PyTorch convention,
    dL/dRe z + i dL/dIm z, complex [D][T][n]) return (g_a, g_b, g_x):
    complex128 [Ltot], complex128 [Ltot], float64 [D][n] (or None)."""
    lib = _load()
    off, a2, b2, d = _bank_arrays(off, a, b, d)
    x = np.ascontiguousarray(np.atleast_2d(x), np.float64)
    D, n = x.shape
    T = off.shape[0] - 1
    gz = np.asarray(gz)
    g2 = np.empty(gz.shape + (2,), np.float64)
    g2[..., 0] = gz.real
    g2[..., 1] = gz.imag
    ltot = int(off[-1])
    ga = np.zeros((ltot, 2), np.float64)
    gb = np.zeros((ltot, 2), np.float64)
    gx = np.zeros((D, n), np.float64) if want_gx else None
    nt = n_threads or max_threads()
    rc = lib.spiir_ref_adjoint(T, D, _ptr(off), _ptr(a2), _ptr(b2), _ptr(d), _ptr(x), n,
                               _ptr(g2), _ptr(ga), _ptr(gb), _ptr(gx), nt)
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return ga[:, 0] + 1j * ga[:, 1], gb[:, 0] + 1j * gb[:, 1], gx


# planted mistakes understood by network_peak (mutation tests only)
NETWORK_MUTATIONS = ("window_short", "last_on_tie", "skip_detector", "shift_last")


def network_peak(z, window, *, mutation=None):
    """Coincidence of one template's SNR series across detectors (the network
    SNR, maximised over arrival-time offsets that the detector separations
    allow; the review's multi-messenger section localises a source from such
    arrival-time differences).  Detector 0 is the reference; for detector
    d >= 1 an offset u with |u| <= window[d] is allowed, positions outside the
    series [0, n) excluded:

        s(t) = |z_0(t)|^2 + sum_{d>=1} max_{|u| <= w_d, 0 <= t+u < n} |z_d(t+u)|^2

    Per template: t* = the first t maximising s, rho = sqrt(s(t*)), and for
    every d >= 1 the first u (from -w_d upward) whose |z_d(t*+u)|^2 reaches
    the max at t* (0 for d = 0).

    The values decide integers (t*, u), so they are taken in float32, as the
    kernel takes them: |z|^2 = re*re + im*im with separately rounded products,
    the detector terms added in detector order, a correctly rounded sqrt.
    z: complex64 [D][T][n]; window: ints [D] (window[0] is ignored).
    Returns (rho float32 [T], t int64 [T], shift int32 [T][D])."""
    z = np.asarray(z, np.complex64)
    D, T, n = z.shape
    window = [int(w) - (1 if mutation == "window_short" and int(w) > 0 else 0) for w in window]
    D_used = D - 1 if mutation == "skip_detector" and D > 1 else D
    re = z.real.astype(np.float32)
    im = z.imag.astype(np.float32)
    p = re * re + im * im                       # float32, two roundings then one
    s = p[0].copy()
    wmax = []
    for d in range(1, D_used):
        w = int(window[d])
        m = np.full((T, n), -np.inf, np.float32)
        for u in range(-w, w + 1):
            lo, hi = max(0, -u), min(n, n - u)
            if lo < hi:
                m[:, lo:hi] = np.maximum(m[:, lo:hi], p[d][:, lo + u:hi + u])
        wmax.append(m)
        s = s + m                               # float32, detector order
    t = np.argmax(s, axis=1).astype(np.int64)   # first index of the max
    if mutation == "last_on_tie":
        t = (n - 1 - np.argmax(s[:, ::-1], axis=1)).astype(np.int64)
    rows = np.arange(T)
    rho = np.sqrt(s[rows, t]).astype(np.float32)
    shift = np.zeros((T, D), np.int32)
    for d in range(1, D_used):
        w = int(window[d])
        order = range(w, -w - 1, -1) if mutation == "shift_last" else range(-w, w + 1)
        for k in range(T):
            tk = int(t[k])
            for u in order:
                if 0 <= tk + u < n and p[d][k, tk + u] == wmax[d - 1][k, tk]:
                    shift[k, d] = u
                    break
    return rho, t, shift


def ls_gains(a, d, target):
    """Least-squares gains of one template's filters (poles a, delays d) for
    the impulse-response target t[0..N): argmin_b sum_k |sum_l b_l phi_l[k]
    - t[k]|^2 with phi_l[k] = a_l^(k - d_l) for k >= d_l (the response of
    filter l with unit gain to an impulse at k = 0), float64 lstsq on the
    explicit N x L matrix.  Returns (b complex128 [L], response complex128 [N])."""
    a = np.asarray(a, np.complex128)
    d = np.asarray(d, np.int64)
    t = np.asarray(target, np.complex128)
    N = t.shape[0]
    k = np.arange(N)
    A = np.zeros((N, a.shape[0]), np.complex128)
    for l in range(a.shape[0]):
        m = k >= d[l]
        A[m, l] = a[l] ** (k[m] - d[l])
    b, *_ = np.linalg.lstsq(A, t, rcond=None)
    return b, A @ b


# planted mistakes understood by chi2_energy / chi2_groups (mutation tests only)
CHI2_MUTATIONS = ("energy_no_gain", "energy_one_minus_abs", "bin_of_end")


def chi2_energy(a, b, *, mutation=None):
    """Energy of each filter's impulse response, the power a chi^2 bin
    counts: sum_{k>=0} |b a^k|^2 = |b|^2 / (1 - |a|^2) (float64)."""
    a = np.asarray(a, np.complex128)
    b = np.asarray(b, np.complex128)
    if mutation == "energy_no_gain":
        return 1.0 / (1.0 - np.abs(a) ** 2)
    if mutation == "energy_one_minus_abs":
        return np.abs(b) ** 2 / (1.0 - np.abs(a))
    return np.abs(b) ** 2 / (1.0 - np.abs(a) ** 2)


def chi2_groups(off, a, b, p, *, mutation=None):
    """Allen's chi^2 bins for every template, read for a bank of single-pole
    filters: a template's filters sorted by frequency arg(a_l) and cut into p
    contiguous groups of (as nearly as whole filters allow) equal energy,
    filter l's energy being that of its impulse response (chi2_energy).
    Filter l goes to the group holding the midpoint of its share of the
    cumulative energy, floor(p * (E_cum(l) - E_l / 2) / E_total), at most
    p - 1; a template of zero energy puts every filter in group 0.  Returns
    int32 [Ltot] group indices in 0..p-1."""
    off = np.asarray(off, np.int64)
    a = np.asarray(a, np.complex128)
    b = np.asarray(b, np.complex128)
    g = np.zeros(a.shape[0], np.int32)
    for t in range(off.shape[0] - 1):
        idx = np.arange(off[t], off[t + 1])
        if idx.size == 0:
            continue
        order = idx[np.argsort(np.angle(a[idx]), kind="stable")]
        e = chi2_energy(a[order], b[order], mutation=mutation)
        total = np.sum(e)
        if total == 0.0:
            continue
        point = np.cumsum(e) if mutation == "bin_of_end" else np.cumsum(e) - 0.5 * e
        g[order] = np.minimum((point / total * p).astype(np.int32), p - 1)
    return g


def chi2_at_peak(z_groups, p):
    """z_groups: complex [D][T][p][n] partial SNR series of each template's p
    groups.  z = sum_i z_i; per (detector, template) the first t maximising
    |z(t)|^2 and chi^2 = p sum_i |z_i(t) - z(t) / p|^2 there (raw z units;
    for unit white noise its mean is (p - 1) times a group's noise power).
    Returns (peak |z| float64 [D][T], t int64 [D][T], chi2 float64 [D][T])."""
    zg = np.asarray(z_groups, np.complex128)
    z = zg.sum(axis=2)
    m2 = np.abs(z) ** 2
    t = np.argmax(m2, axis=-1)
    D, T = t.shape
    dd, tt = np.meshgrid(np.arange(D), np.arange(T), indexing="ij")
    zt = z[dd, tt, t]
    zi = zg[dd, tt, :, t]                       # [D][T][p]
    chi2 = p * np.sum(np.abs(zi - zt[..., None] / p) ** 2, axis=-1)
    return np.abs(zt), t.astype(np.int64), chi2
