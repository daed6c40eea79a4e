"""IIR bank design: filters for a chirp template, gains fitted on the GPU.

The SPIIR method approximates each template's matched filter by a parallel
bank of single-pole complex IIR filters (section "GPU accelerated SPIIR
method", subsection "SPIIR method": the summed responses reach more than 99%
overlap with the matched filter).  The matched filter of a complex template
h[0..N) has the impulse response t[k] = conj(h[N-1-k]): it starts at the
coalescence and runs back through the inspiral, so damped complex
sinusoids started at the right delays can follow it.

place_filters: delays that split t into segments of equal phase advance,
poles exp(-decay / length + i omega) with omega the per-sample phase advance
of t at the segment's middle.  fit_gains: the gains minimising
sum_k |z[k] - t[k]|^2 for the bank's impulse response z = A b (linear in b),
by conjugate gradients on the normal equations A^H A b = A^H t; every A p
is a spiir_filter call on an impulse and every A^H v a spiir_filter_backward
call (its g_b for g_z = v), so the fit runs in the library's kernels; the
per-template dot products in between are on vectors of a few hundred gains.
"""
from __future__ import annotations

import numpy as np


def matched_target(h: np.ndarray) -> np.ndarray:
    """Impulse response of h's matched filter, unit norm: conj(h[N-1-k])."""
    t = np.conj(np.asarray(h, np.complex128)[::-1])
    return t / np.linalg.norm(t)


def place_filters(target: np.ndarray, n_filters: int, decay: float = 0.2):
    """(poles complex64 [L], delays int32 [L], initial gains complex64 [L])
    for one target; L <= n_filters (segments that would be empty merge)."""
    t = np.asarray(target, np.complex128)
    N = t.shape[0]
    w = np.angle(t[1:] * np.conj(t[:-1]))
    Phi = np.concatenate([[0.0], np.cumsum(np.abs(w))])
    kb = np.unique(np.searchsorted(Phi, np.linspace(0.0, Phi[-1], n_filters + 1)[:-1]))
    ke = np.concatenate([kb[1:], [N]])
    mid = np.minimum((kb + ke) // 2, N - 2)
    a = np.exp(-decay / (ke - kb) + 1j * w[mid])
    b = t[kb]
    return a.astype(np.complex64), kb.astype(np.int32), b.astype(np.complex64)


def overlap(z, target) -> np.ndarray:
    """|<z, t>| / (|z| |t|) per template (last axis: samples)."""
    z = np.asarray(z, np.complex128)
    t = np.asarray(target, np.complex128)
    num = np.abs(np.sum(np.conj(z) * t, axis=-1))
    return num / (np.linalg.norm(z, axis=-1) * np.linalg.norm(t, axis=-1))


def fit_gains(sp, a, d, targets, *, b0=None, iters: int = 400, tol: float = 1e-7,
              device: int = 0):
    """Least-squares gains for T templates of L filters each (a, d: [T][L]
    poles and delays; targets: [T][N] complex).  Returns (b complex64 [T][L],
    the bank's impulse response [T][N] complex64, CG iterations run).  sp is
    the paper_1602_05573_b300 module."""
    import types

    import torch

    a = np.asarray(a, np.complex64)
    d = np.asarray(d, np.int32)
    T, L = a.shape
    N = int(np.asarray(targets).shape[-1])
    dev = torch.device("cuda", device)
    off = np.arange(T + 1, dtype=np.int64) * L
    b_init = np.ones((T, L), np.complex64) if b0 is None else np.asarray(b0, np.complex64)
    bank = types.SimpleNamespace(off=off, a=a.ravel(), b=b_init.ravel(), d=d.ravel(), n_det=1)
    plan = sp.Plan(bank, device=device)
    x = torch.zeros((1, N), dtype=torch.float32, device=dev)
    x[0, 0] = 1.0
    at = torch.from_numpy(a.ravel()).to(dev)
    tg = torch.from_numpy(np.asarray(targets, np.complex64)).to(dev).reshape(1, T, N)

    def A(p):                        # bank impulse response with gains p
        plan.set_coefficients(at, p.reshape(-1))
        plan.reset()
        return plan.filter(x)        # [1][T][N]

    def AH(v):                       # A^H v through the adjoint
        _, gb, _ = plan.backward(x, v, want_gx=False)
        return gb.reshape(T, L)

    def dot(u, v):                   # per template Re <u, v>
        return torch.sum((torch.conj(u) * v).real, dim=-1, keepdim=True)

    b = torch.from_numpy(b_init).to(dev)
    r = AH(tg - A(b))
    p = r.clone()
    rs = dot(r, r)
    rs0 = rs.clone()
    it = 0
    for it in range(1, iters + 1):
        Mp = AH(A(p))
        alpha = rs / torch.clamp(dot(p, Mp), min=1e-30)
        b = b + alpha * p
        r = r - alpha * Mp
        rs_new = dot(r, r)
        if bool(torch.all(rs_new <= (tol * tol) * rs0)):
            rs = rs_new
            break
        p = r + (rs_new / torch.clamp(rs, min=1e-30)) * p
        rs = rs_new
    z = A(b)
    plan.check()
    plan.close()
    return b.cpu().numpy(), z[0].cpu().numpy(), it
