"""Multirate banks on the GPU against oracle.filter_multirate.

Each band runs at its own rate on plain-subsampled strain x[R k]; the band
sums are linearly interpolated to the top rate and added (the multirate
reading of the SPIIR bank).  The injection tests follow the matched-filter
reading: a signal equal to the time-reversed real part of the template's
own top-rate impulse response, scaled to SNR 12, must be found at its
template and time (to within one sample of the coarsest band).
"""
import numpy as np
import pytest

import oracle
from parity_util import REL_TOL, check_peaks, rel_errors
from spiir_inputs import make_multirate_bank, make_strain, workload_bank

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sp(cuda_device):
    import paper_1602_05573_b300
    return paper_1602_05573_b300


def c3_bank(n_templates, seed=303):
    """The injection+multirate workload's distributions on fewer templates."""
    return make_multirate_bank(n_templates, (60, 120, 120), (1, 4, 16), (0.99, 0.9995), 1024,
                               seed)


def oracle_mr(bank, x):
    return oracle.filter_multirate(bank.off, bank.a, bank.b, bank.d, bank.band_of, bank.decim, x)


def gpu_mr(sp, bank, x, chunks=None, emit_z=True, **opts):
    plan = sp.Plan(bank, **opts)
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    n = x.shape[1]
    parts, at = [], 0
    for c in (chunks or []) + [n - sum(chunks or [])]:
        zc = plan.filter(xt[:, at:at + c].contiguous(), emit_z=emit_z)
        if emit_z:
            parts.append(zc.cpu().numpy())
        at += c
    pa, pi = plan.peak()
    plan.check()
    z = np.concatenate(parts, axis=-1) if emit_z else None
    return z, pa.cpu().numpy(), pi.cpu().numpy()


@pytest.mark.parametrize("n", [32768, 5003])
def test_multirate_parity(sp, n):
    bank = c3_bank(24)
    x = make_strain(1, n, seed=310)
    z, pa, pi = gpu_mr(sp, bank, x)
    zref, _, _ = oracle_mr(bank, x)
    rel, _ = rel_errors(z, zref)
    assert rel.max() <= REL_TOL, rel.max()
    check_peaks(z, zref, pa, pi)


@pytest.mark.parametrize("filters,decim", [((40, 60), (1, 2)), ((30, 50, 70, 40), (1, 2, 4, 8))])
def test_multirate_band_counts(sp, filters, decim):
    """Two bands (one lower band: no second stream) and four (three lower
    bands, alternating over the plan's two streams), two detectors, a call
    ending inside the coarsest band's sample."""
    bank = make_multirate_bank(9, filters, decim, (0.99, 0.9995), 300, seed=320, n_det=2)
    n = 6 * 1024 + 8 * 37 + 3
    x = make_strain(2, n, seed=321)
    z, pa, pi = gpu_mr(sp, bank, x)
    zref, _, _ = oracle_mr(bank, x)
    rel, _ = rel_errors(z, zref)
    assert rel.max() <= REL_TOL, rel.max()
    check_peaks(z, zref, pa, pi)


def test_multirate_streaming_matches_one_call_outside_hold(sp):
    """Calls of whole multiples of the largest decimation continue the
    stream; only the last 16 samples of each non-final call (interpolated
    with the hold rule) differ from one call."""
    bank = c3_bank(8)
    x = make_strain(1, 12000, seed=311)
    z1, _, _ = gpu_mr(sp, bank, x, time_segments=1)
    chunks = [4096, 16, 3200]
    z2, _, _ = gpu_mr(sp, bank, x, chunks=chunks, time_segments=1)
    mask = np.ones(x.shape[1], bool)
    for end in np.cumsum(chunks):
        mask[end - 16:end] = False
    assert np.array_equal(z1[..., mask], z2[..., mask])


def test_multirate_rejects_misaligned_stream(sp):
    bank = c3_bank(2)
    plan = sp.Plan(bank)
    x = torch.from_numpy(make_strain(1, 100, seed=312)).cuda()
    plan.filter(x)  # 100 is not a multiple of 16: no further call may follow
    with pytest.raises(sp.SpiirError) as e:
        plan.filter(x)
    assert e.value.status == sp.EINVAL


def injected_strain(bank, tau, k0, n, snr=12.0, seed=320, lh=1 << 16):
    """Noise plus A * Re h[k0 - m] (h = template tau's top-rate impulse
    response from the oracle), A chosen so the noiseless |z[k0]| is snr
    times the noise rms per quadrature of that template (also from the
    oracle)."""
    sub = bank.subset([tau])
    delta = np.zeros((1, lh))
    delta[0, 0] = 1.0
    h, _, _ = oracle_mr(sub, delta)
    h = h[0, 0]
    s = np.zeros((1, n))
    m = np.arange(max(0, k0 - lh + 1), k0 + 1)
    s[0, m] = h[k0 - m].real
    zs, _, _ = oracle_mr(sub, s)
    noise = make_strain(1, n, seed=seed).astype(np.float64)
    zn, _, _ = oracle_mr(sub, noise)
    sigma = np.sqrt(np.mean(np.abs(zn[0, 0, lh:]) ** 2) / 2)
    amp = snr * sigma / abs(zs[0, 0, k0])
    return (noise + amp * s).astype(np.float32), sigma


def test_injection_recovered(sp):
    """128 templates, 64 s at 4096 Hz, one injection at SNR 12."""
    bank = c3_bank(128, seed=330)
    n, tau, k0 = 1 << 18, 77, 200_000
    x, sigma = injected_strain(bank, tau, k0, n)
    z, pa, pi = gpu_mr(sp, bank, x)
    # SNR per template: peak |z| over that template's noise rms per quadrature
    rms = np.sqrt(np.mean(np.abs(z[0].astype(np.complex128)) ** 2, axis=-1) / 2)
    rho = pa[0] / rms
    assert int(np.argmax(rho)) == tau
    assert abs(int(pi[0, tau]) - k0) <= 16
    assert 10.0 < pa[0, tau] / sigma < 14.0
    sub = bank.subset([tau])
    zref, _, _ = oracle_mr(sub, x)
    rel, _ = rel_errors(z[:, tau:tau + 1], zref)
    assert rel.max() <= REL_TOL


def noise_rms_all(sp, bank, lh=1 << 18):
    """Noise rms per quadrature of every template, sqrt(1/2 sum |h|^2), from
    its top-rate response to an impulse at the stream start (the library's;
    lh samples hold its energy to ~1e-7 for the slowest band's poles)."""
    plan = sp.Plan(bank)
    delta = torch.zeros((1, lh), dtype=torch.float32, device="cuda")
    delta[0, 0] = 1.0
    h = plan.filter(delta)
    sig = torch.sqrt(0.5 * (h[0].abs() ** 2).double().sum(dim=-1)).cpu().numpy()
    plan.close()
    del h
    torch.cuda.empty_cache()
    return sig


def test_multirate_workload_full_size(sp):
    """The full injection+multirate workload (2048 templates x 3 bands,
    2^20 samples at 4096 Hz) without storing z: the injected template has
    the largest normalised peak (peak |z| / its noise rms) of all 2048 and
    peaks at the injection time, and 6 sampled templates match the oracle."""
    bank = workload_bank("multirate")
    n, tau, k0 = 1 << 20, 1234, 700_016
    x, sigma = injected_strain(bank, tau, k0, n)
    _, pa, pi = gpu_mr(sp, bank, x, emit_z=False)
    assert abs(int(pi[0, tau]) - k0) <= 16
    assert 10.0 < pa[0, tau] / sigma < 14.0
    sig_all = noise_rms_all(sp, bank)
    rho = pa[0] / sig_all
    assert int(np.argmax(rho)) == tau, (int(np.argmax(rho)), rho[tau], np.sort(rho)[-2])
    rng = np.random.default_rng(331)
    picks = sorted(set([tau] + [int(t) for t in rng.choice(2048, 5, replace=False)]))
    # the library's noise rms of the sampled templates against the oracle's
    delta = np.zeros((1, 1 << 18))
    delta[0, 0] = 1.0
    href, _, _ = oracle_mr(bank.subset(picks), delta)
    sig_ref = np.sqrt(0.5 * np.sum(np.abs(href[0]) ** 2, axis=-1))
    np.testing.assert_allclose(sig_all[picks], sig_ref, rtol=1e-4)
    sub = bank.subset(picks)
    zsub, pas, pis = gpu_mr(sp, sub, x)
    zref, _, _ = oracle_mr(sub, x)
    rel, _ = rel_errors(zsub, zref)
    assert rel.max() <= REL_TOL, rel.max()
    check_peaks(zsub, zref, pas, pis)
    # the full-bank launch agrees with the sub-bank launch on these templates
    np.testing.assert_allclose(pa[0, picks], pas[0], rtol=1e-4)
    for j, t in enumerate(picks):
        mag = np.abs(zref[0, j])
        _, err = rel_errors(zsub[:, j:j + 1], zref[:, j:j + 1])
        cand = np.flatnonzero(mag >= mag.max() - 4 * err[0, 0])
        assert int(pi[0, t]) in cand
