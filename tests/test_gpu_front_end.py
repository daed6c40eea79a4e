"""Band front ends (spiir_set_band_fir): band j of a multirate bank sees
sum_i h_j[i] x[R_j k - i] (whitening / anti-aliasing before subsampling)
instead of x[R_j k].  Against oracle.filter_multirate_fir, which
tests/test_oracle_pins.py pins to plain subsampling (identity taps), to a
delayed and scaled strain (one tap) and to a direct convolution loop."""
import numpy as np
import pytest

import oracle
from parity_util import REL_TOL, rel_errors
from spiir_inputs import make_multirate_bank, make_strain

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sp(cuda_device):
    import paper_1602_05573_b300
    return paper_1602_05573_b300


def lowpass(R, taps):
    """Windowed-sinc anti-alias filter with cut-off at the band's Nyquist."""
    k = np.arange(taps) - (taps - 1) / 2
    h = np.sinc(k / R) / R * np.hanning(taps + 2)[1:-1]
    return (h / h.sum()).astype(np.float32)


def run(sp, bank, x, firs, chunks=None, **opts):
    plan = sp.Plan(bank, **opts)
    for j, h in enumerate(firs):
        if h is not None:
            plan.set_band_fir(j, h)
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    n = x.shape[1]
    parts, at = [], 0
    for c in (chunks or []) + [n - sum(chunks or [])]:
        parts.append(plan.filter(xt[:, at:at + c].contiguous()).cpu().numpy())
        at += c
    plan.check()
    plan.close()
    return np.concatenate(parts, axis=-1)


BANK = dict(n_templates=10, band_filters=(30, 40, 40), decim=(1, 4, 16), r_range=(0.99, 0.9995),
            d_max=300)


FIRS = [np.array([1.0, -0.6, 0.15], np.float32),   # a short whitening FIR at the top rate
        lowpass(4, 63), lowpass(16, 255)]


@pytest.mark.parametrize("n", [20000, 3001])
def test_front_end_matches_oracle(sp, n):
    bank = make_multirate_bank(seed=170, n_det=2, **BANK)
    x = make_strain(2, n, seed=171)
    z = run(sp, bank, x, FIRS)
    zref = oracle.filter_multirate_fir(bank.off, bank.a, bank.b, bank.d, bank.band_of,
                                       bank.decim, x, [f.astype(np.float64) for f in FIRS])
    rel, _ = rel_errors(z, zref)
    assert rel.max() <= REL_TOL, rel.max()


def test_front_end_streaming_matches_one_call_outside_hold(sp):
    """The front ends keep the last 511 top-rate samples across calls: calls
    of whole multiples of the largest decimation give one call's z, bit for
    bit, except the last 16 samples of each non-final call (the multirate
    hold rule at a call's end)."""
    bank = make_multirate_bank(seed=176, n_det=2, **BANK)
    x = make_strain(2, 20000, seed=177)
    z1 = run(sp, bank, x, FIRS, time_segments=1)
    chunks = [4096, 16, 8192]
    z2 = run(sp, bank, x, FIRS, chunks, time_segments=1)
    mask = np.ones(x.shape[1], bool)
    for end in np.cumsum(chunks):
        mask[end - 16:end] = False
    assert np.array_equal(z1[..., mask], z2[..., mask])


def test_identity_taps_are_plain_subsampling_bit_for_bit(sp):
    bank = make_multirate_bank(seed=172, **BANK)
    x = make_strain(1, 9000, seed=173)
    one = np.array([1.0], np.float32)
    assert np.array_equal(run(sp, bank, x, [one, one, one]), run(sp, bank, x, [None] * 3))


def test_front_end_can_be_removed_and_rejects_bad_arguments(sp):
    bank = make_multirate_bank(seed=174, **BANK)
    x = make_strain(1, 4096, seed=175)
    plan = sp.Plan(bank)
    plan.set_band_fir(1, lowpass(4, 31))
    plan.set_band_fir(1, None)                           # back to plain subsampling
    z = plan.filter(torch.from_numpy(x).cuda()).cpu().numpy()
    plan.check()
    assert np.array_equal(z, run(sp, bank, x, [None] * 3))
    with pytest.raises(sp.SpiirError):
        plan.set_band_fir(3, [1.0])                      # no such band
    with pytest.raises(sp.SpiirError):
        plan.set_band_fir(0, np.ones(513, np.float32))   # above 512 taps
    plan.set_band_fir(2, [0.5, 0.5])
    st, hist, t = plan.state_get()
    with pytest.raises(sp.SpiirError):
        plan.state_set(st, hist, t)                      # front-end history is not in the state
    plan.close()


def test_whitening_fir_on_a_single_rate_bank(sp):
    """A single-rate bank's only band takes a front end too: z equals the
    oracle's filter bank on the FIR-filtered strain (oracle.band_input)."""
    from spiir_inputs import make_bank
    bank = make_bank(6, (20, 100), (0.99, 0.9995), 300, seed=178, n_det=2)
    x = make_strain(2, 6000, seed=179)
    taps = np.array([0.9, -0.5, 0.2, -0.05], np.float32)
    plan = sp.Plan(bank)
    plan.set_band_fir(0, taps)
    xt = torch.from_numpy(x).cuda()
    z = np.concatenate([plan.filter(xt[:, :2048].contiguous()).cpu().numpy(),
                        plan.filter(xt[:, 2048:].contiguous()).cpu().numpy()], axis=-1)
    plan.check()
    plan.close()
    zref, _, _ = oracle.filter_bank(bank.off, bank.a, bank.b, bank.d,
                                    oracle.band_input(x, taps.astype(np.float64)))
    rel, _ = rel_errors(z, zref)
    assert rel.max() <= REL_TOL, rel.max()
