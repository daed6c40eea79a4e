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


class BankFit:
    """T templates of L filters (delays d [T][L] fixed) against impulse-
    response targets [T][N], on one plan whose poles and gains change with
    spiir_set_coefficients.  A(a, b): the bank's impulse response (one
    spiir_filter on an impulse); adjoint(v): (g_a, g_b) of Re <v, z> by
    spiir_filter_backward (g_b = A^H v)."""

    def __init__(self, sp, a, d, targets, device: int = 0):
        import types

        import torch
        self.torch = torch
        a = np.asarray(a, np.complex64)
        self.T, self.L = a.shape
        self.N = int(np.asarray(targets).shape[-1])
        self.dev = torch.device("cuda", device)
        off = np.arange(self.T + 1, dtype=np.int64) * self.L
        bank = types.SimpleNamespace(off=off, a=a.ravel(), b=np.ones(a.size, np.complex64),
                                     d=np.asarray(d, np.int32).ravel(), n_det=1)
        self.plan = sp.Plan(bank, device=device)
        self.x = torch.zeros((1, self.N), dtype=torch.float32, device=self.dev)
        self.x[0, 0] = 1.0
        self.t = torch.from_numpy(np.asarray(targets, np.complex64)).to(self.dev).reshape(
            1, self.T, self.N)
        self.a = torch.from_numpy(a).to(self.dev)

    def close(self):
        self.plan.check()
        self.plan.close()

    def A(self, b, a=None):
        a = self.a if a is None else a
        self.plan.set_coefficients(a.reshape(-1), b.reshape(-1))
        self.plan.reset()
        return self.plan.filter(self.x)          # [1][T][N]

    def adjoint(self, v):
        ga, gb, _ = self.plan.backward(self.x, v, want_gx=False)
        return ga.reshape(self.T, self.L), gb.reshape(self.T, self.L)

    def loss(self, z):                           # per template sum |z - t|^2, [T]
        return self.torch.sum(self.torch.abs(z - self.t) ** 2, dim=-1)[0]

    def fit_gains(self, b, iters: int = 400, tol: float = 1e-7, check_every: int = 8):
        """Conjugate gradients on A^H A b = A^H t from b (per template).  A
        template whose residual has dropped by tol stops moving (its step is
        zeroed on the device); the host reads the convergence flags only every
        check_every iterations, so the iterations queue without a sync."""
        torch = self.torch

        def dot(u, v):
            return torch.sum((torch.conj(u) * v).real, dim=-1, keepdim=True)
        AH = lambda v: self.adjoint(v)[1]          # noqa: E731
        r = AH(self.t - self.A(b))
        p = r.clone()
        rs = dot(r, r)
        rs0 = torch.clamp(rs.clone(), min=1e-30)
        active = rs > (tol * tol) * rs0
        it = 0
        for it in range(1, iters + 1):
            Mp = AH(self.A(p))
            alpha = torch.where(active, rs / torch.clamp(dot(p, Mp), min=1e-30),
                                torch.zeros_like(rs))
            b = b + alpha * p
            r = r - alpha * Mp
            rs_new = dot(r, r)
            active = active & (rs_new > (tol * tol) * rs0)
            if it % check_every == 0 and not bool(torch.any(active)):
                break
            p = torch.where(active, r + (rs_new / torch.clamp(rs, min=1e-30)) * p, p)
            rs = torch.where(active, rs_new, rs)
        return b, it


def fit_gains(sp, a, d, targets, *, b0=None, iters: int = 400, tol: float = 1e-7,
              device: int = 0):
    """Least-squares gains for T templates of L filters each (a, d: [T][L]
    poles and delays; targets: [T][N] complex).  Returns (b complex64 [T][L],
    the bank's impulse response [T][N] complex64, CG iterations run).  sp is
    the paper_1602_05573_b300 module."""
    import torch
    f = BankFit(sp, a, d, targets, device)
    T, L = f.T, f.L
    b = torch.from_numpy(np.ones((T, L), np.complex64) if b0 is None
                         else np.asarray(b0, np.complex64)).to(f.dev)
    b, it = f.fit_gains(b, iters, tol)
    z = f.A(b)
    out = b.cpu().numpy(), z[0].cpu().numpy(), it
    f.close()
    return out


def fit_bank(sp, a, d, targets, *, b0=None, outer: int = 25, cg_iters: int = 200,
             step: float = 1e-3, device: int = 0):
    """Poles and gains by variable projection: for fixed poles the gains are
    the least-squares ones (fit_gains), and the loss as a function of the
    poles alone has the gradient g_a that the adjoint returns for
    g_z = 2 (z - t) at those gains.  Each outer step moves every template's
    poles along -g_a (largest move `step`, |a| kept <= 1 - 1e-5), halving the
    step for templates whose loss did not drop (gains held), then refits the
    gains.  Returns (a complex64 [T][L], b complex64 [T][L], response
    [T][N] complex64, overlap per outer step [outer + 1][T])."""
    import torch
    f = BankFit(sp, a, d, targets, device)
    T, L = f.T, f.L
    b = torch.from_numpy(np.ones((T, L), np.complex64) if b0 is None
                         else np.asarray(b0, np.complex64)).to(f.dev)
    b, _ = f.fit_gains(b, cg_iters)
    z = f.A(b)
    history = [overlap(z[0].cpu().numpy(), f.t[0].cpu().numpy())]
    eta = torch.full((T, 1), step, device=f.dev)
    for _ in range(outer):
        loss = f.loss(z)
        ga, _ = f.adjoint(2.0 * (z - f.t))
        gmax = torch.clamp(torch.abs(ga).amax(dim=-1, keepdim=True), min=1e-30)
        a0 = f.a
        done = torch.zeros((T, 1), dtype=torch.bool, device=f.dev)
        for _try in range(8):
            an = a0 - (eta / gmax) * ga
            mag = torch.abs(an)
            an = torch.where(mag > 1.0 - 1e-5, an / mag * (1.0 - 1e-5), an)
            better = (f.loss(f.A(b, an)) < loss).reshape(T, 1) & ~done
            f.a = torch.where(better, an, f.a)
            done = done | better
            if bool(torch.all(done)):
                break
            eta = torch.where(done, eta, eta * 0.5)
        eta = torch.where(done, eta * 1.5, eta)   # accepted: try a longer step next
        b, _ = f.fit_gains(b, cg_iters)
        z = f.A(b)
        history.append(overlap(z[0].cpu().numpy(), f.t[0].cpu().numpy()))
    out = (f.a.cpu().numpy(), b.cpu().numpy(), z[0].cpu().numpy(), np.stack(history))
    f.close()
    return out
