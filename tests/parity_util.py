"""Comparison helpers for the GPU parity tests.

Floating-point bar (relative error of the SNR series, per detector and
template): rel = max_k |z_gpu[k] - z_ref[k]| / rms_k |z_ref[k]| <= 1e-4,
with z_ref from the FP64 oracle.  The peak is an integer decided by floating
point, so it is checked two ways: (1) bit-exactly against the GPU's own z,
re-evaluated on the host in float32 with the kernel's formula
(re*re + im*im, no fused multiply-add, first index on ties); (2) against the
oracle: the GPU index must be the oracle's argmax, or -- when other samples
come within 4x the measured error of the oracle's top value (an "epsilon
tie") -- one of those samples.
"""
import numpy as np

REL_TOL = 1e-4


def rel_errors(z_gpu, z_ref):
    """Per-(detector, template) max abs error / rms of the reference."""
    z_gpu = np.asarray(z_gpu).astype(np.complex128)
    diff = np.abs(z_gpu - z_ref).max(axis=-1)
    rms = np.sqrt(np.mean(np.abs(z_ref) ** 2, axis=-1))
    return diff / np.maximum(rms, 1e-300), diff


def host_peak_f32(z_gpu):
    """The kernel's peak rule evaluated on the host in float32."""
    zr = np.ascontiguousarray(z_gpu.real, dtype=np.float32)
    zi = np.ascontiguousarray(z_gpu.imag, dtype=np.float32)
    p = (zr * zr).astype(np.float32) + (zi * zi).astype(np.float32)
    idx = np.argmax(p, axis=-1)
    best = np.take_along_axis(p, idx[..., None], axis=-1)[..., 0]
    return np.sqrt(best).astype(np.float32), idx


def check_peaks(z_gpu, z_ref, peak_abs, peak_idx, t0=0):
    """Returns (n_exact, n_eps_tie); raises AssertionError on a mismatch."""
    habs, hidx = host_peak_f32(z_gpu)
    assert np.array_equal(peak_idx - t0, hidx), "peak index differs from the GPU's own z"
    assert np.array_equal(peak_abs, habs), "peak value differs from the GPU's own z"
    _, err = rel_errors(z_gpu, z_ref)
    mag = np.abs(z_ref)
    exact = ties = 0
    for i in np.ndindex(mag.shape[:-1]):
        m = mag[i]
        top = m.max()
        cand = np.flatnonzero(m >= top - 4 * err[i])
        k = int(peak_idx[i] - t0)
        assert k in cand, f"{i}: GPU peak at {k}, oracle candidates {cand[:8]}"
        if len(cand) == 1:
            exact += 1
        else:
            ties += 1
    return exact, ties
