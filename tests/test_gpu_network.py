"""Network peak across detectors (spiir_network_peak) against the oracle's
network_peak, which tests/test_oracle_pins.py pins to closed forms, brute
force and shift invariance.  The peak time and the per-detector offsets are
integers decided by float32 values that both sides form the same way, so
they must match exactly; rho too (same operations, correctly rounded sqrt).
"""
import numpy as np
import pytest

import oracle
from spiir_inputs import make_bank, make_strain, workload_bank, workload_strain

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sp(cuda_device):
    import paper_1602_05573_b300
    return paper_1602_05573_b300


def gpu_net(sp, z, window):
    zt = torch.from_numpy(np.ascontiguousarray(z.astype(np.complex64))).cuda()
    rho, t, sh = sp.network_peak(zt, window)
    torch.cuda.synchronize()
    return rho.cpu().numpy(), t.cpu().numpy(), sh.cpu().numpy()


def assert_same(got, want):
    for g, w, name in zip(got, want, ("rho", "t", "shift")):
        assert np.array_equal(g, w), (name, np.flatnonzero(g != w)[:10])


@pytest.mark.parametrize("D,T,n,window", [
    (3, 37, 5000, [0, 10, 27]),      # several 2048-output tiles and a ragged tail
    (2, 5, 2049, [0, 1]),            # one output past a tile
    (1, 9, 777, [0]),                # single detector: the plain peak
    (4, 6, 300, [0, 0, 600, 1024]),  # windows wider than the series
    (8, 3, 1500, [0, 1, 2, 3, 5, 8, 13, 21]),
    (3, 4, 1, [0, 3, 9]),            # one sample
    (3, 4, 7, [0, 2, 700]),          # shorter than a thread's run of 8 outputs
    (2, 3, 4100, [0, 300]),          # window past the scan limit: doubling levels
    (3, 37, 5000, [0, 40, 60]),      # wide scanned windows: runs of 16 outputs per thread
    (2, 11, 6000, [0, 64]),          # the widest scanned window, runs of 8
    (4, 5, 2500, [0, 6, 64, 64]),    # runs of 16 with a 13-sample window (two runs of 8)
])
def test_network_peak_matches_oracle(sp, D, T, n, window):
    rng = np.random.default_rng(D * 1000 + n)
    z = (rng.standard_normal((D, T, n)) + 1j * rng.standard_normal((D, T, n))).astype(np.complex64)
    assert_same(gpu_net(sp, z, window), oracle.network_peak(z, window))


def test_network_peak_ties(sp):
    """Small-integer series: exact ties of |z|^2 inside windows and of the
    network statistic across t (earliest t, then earliest offset)."""
    rng = np.random.default_rng(77)
    z = (rng.integers(-2, 3, (3, 16, 3000)) + 1j * rng.integers(-2, 3, (3, 16, 3000)))
    z = z.astype(np.complex64)
    assert_same(gpu_net(sp, z, [0, 7, 30]), oracle.network_peak(z, [0, 7, 30]))
    assert_same(gpu_net(sp, z, [0, 50, 60]), oracle.network_peak(z, [0, 50, 60]))
    zero = np.zeros((2, 3, 100), np.complex64)
    assert_same(gpu_net(sp, zero, [0, 5]), oracle.network_peak(zero, [0, 5]))
    # series of several tiles, split across CTAs in time chunks: the equal
    # maxima of different chunks resolve to the earliest t
    zero = np.zeros((2, 3, 9000), np.complex64)
    assert_same(gpu_net(sp, zero, [0, 5]), oracle.network_peak(zero, [0, 5]))
    spikes = np.zeros((2, 3, 9000), np.complex64)
    spikes[0, :, [8500, 4100, 2050]] = 3 + 4j
    assert_same(gpu_net(sp, spikes, [0, 5]), oracle.network_peak(spikes, [0, 5]))


def test_network_peak_of_filtered_event(sp):
    """SNR series of a filtered three-detector event: a template's impulse
    response injected at arrival times 0, +6 and -11 samples apart is found
    with those offsets."""
    bank = make_bank(6, 40, (0.9, 0.99), 30, seed=150, n_det=3)
    n = 4000
    x = 0.001 * make_strain(3, n, seed=151)
    for d, off in enumerate((0, 6, -11)):
        x[d, 2000 + off] += 1.0
    z, _, _ = oracle.filter_bank(bank.off, bank.a, bank.b, bank.d, x)
    z = z.astype(np.complex64)
    want = oracle.network_peak(z, [0, 10, 20])
    assert_same(gpu_net(sp, z, [0, 10, 20]), want)
    # the response peaks at the same delay after each detector's arrival
    assert (want[2][:, 1] == 6).all() and (want[2][:, 2] == -11).all()


def test_network_peak_on_kernel_output_full_size_sampled(sp):
    """On the batched bank's own z (3 detectors, 65536 samples, every
    template): a sample of templates against the oracle, and the GPU call
    in the stream that spiir_filter wrote z on."""
    bank = workload_bank("batched")
    x = torch.from_numpy(workload_strain("batched")).cuda()
    D, n = x.shape
    plan = sp.Plan(bank)
    z = torch.empty((D, bank.n_templates, n), dtype=torch.complex64, device="cuda")
    plan.filter(x, z)
    window = [0, 10, 28]
    rho, t, sh = sp.network_peak(z, window)
    torch.cuda.synchronize()
    pick = np.random.default_rng(5).choice(bank.n_templates, 24, replace=False)
    zs = z[:, torch.from_numpy(pick).cuda(), :].cpu().numpy()
    want = oracle.network_peak(zs, window)
    got = (rho.cpu().numpy()[pick], t.cpu().numpy()[pick], sh.cpu().numpy()[pick])
    assert_same(got, want)
    plan.close()


def test_network_peak_rejects_bad_arguments(sp):
    z = torch.zeros((9, 2, 10), dtype=torch.complex64, device="cuda")
    with pytest.raises(sp.SpiirError):
        sp.network_peak(z, [0] * 9)                  # more than 8 detectors
    z = torch.zeros((2, 2, 10), dtype=torch.complex64, device="cuda")
    with pytest.raises(sp.SpiirError):
        sp.network_peak(z, [0, 1025])                # window above 1024
    with pytest.raises(sp.SpiirError):
        sp.network_peak(z[:, :, :0], [0, 1])         # empty series
