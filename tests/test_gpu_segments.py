"""Time-segmented calls against the FP64 oracle.

A call of n samples split into P segments runs every segment at once: a
zero-state pass gives each segment's contribution to its end state, an FP64
carry y_start(q+1) = a^n_seg y_start(q) + y_end^0(q) gives every segment its
true start state (the same linear recurrence of the SPIIR filter, applied a
segment at a time), and the filtering pass runs each segment from there.
The start states come either from a zero-state FP32 pass with an FP64 carry
("recurrence") or from chunk sums computed as a split-BF16 tensor-core GEMM
followed by an FP32 chunk scan ("tensor").  Either way the result must meet
the same element-wise bar as the unsegmented path, and the peak must be the
earliest largest |z| over the whole call.
"""
import numpy as np
import pytest

import oracle
from parity_util import REL_TOL, check_peaks, rel_errors
from spiir_inputs import make_bank, make_multirate_bank, make_strain, workload_bank, \
    workload_strain

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sp(cuda_device):
    import paper_1602_05573_b300
    return paper_1602_05573_b300


def run(sp, bank, x, chunks=None, **opts):
    plan = sp.Plan(bank, **opts)
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    n = x.shape[1]
    parts, at = [], 0
    for c in (chunks or []) + [n - sum(chunks or [])]:
        parts.append(plan.filter(xt[:, at:at + c].contiguous()).cpu().numpy())
        at += c
    pa, pi = plan.peak()
    plan.check()
    return np.concatenate(parts, axis=-1), pa.cpu().numpy(), pi.cpu().numpy(), plan


PROJ = ["tensor", "recurrence"]


@pytest.mark.parametrize("projection", PROJ)
@pytest.mark.parametrize("P", [2, 3, 7])
@pytest.mark.parametrize("n", [6000, 4096 + 513])
def test_forced_segments_match_oracle(sp, P, n, projection):
    bank = make_bank(11, (20, 150), (0.99, 0.9995), 900, seed=401, n_det=2)
    x = make_strain(2, n, seed=402)
    z, pa, pi, _ = run(sp, bank, x, time_segments=P, block_len=256, projection=projection)
    zref, _, _ = oracle.filter_bank(bank.off, bank.a, bank.b, bank.d, x)
    rel, _ = rel_errors(z, zref)
    assert rel.max() <= REL_TOL, rel.max()
    check_peaks(z, zref, pa, pi)


@pytest.mark.parametrize("projection", PROJ)
def test_segments_continue_a_stream(sp, projection):
    """Segmented calls of assorted lengths (the first one starting from a
    non-zero state) continue the stream to within the parity bar, and peak
    indices count from the stream start."""
    bank = make_bank(6, (30, 120), (0.995, 0.9999), 700, seed=403)
    x = make_strain(1, 20000, seed=404)
    z, pa, pi, _ = run(sp, bank, x, chunks=[3000, 257, 9000], time_segments=5, block_len=256,
                       projection=projection)
    zref, _, _ = oracle.filter_bank(bank.off, bank.a, bank.b, bank.d, x)
    rel, _ = rel_errors(z, zref)
    assert rel.max() <= REL_TOL, rel.max()
    check_peaks(z, zref, pa, pi)


@pytest.mark.parametrize("projection", PROJ)
def test_segments_in_half_warp_mode(sp, projection):
    bank = make_bank(20, (8, 60), (0.99, 0.999), 400, seed=405, n_det=2)
    x = make_strain(2, 7000, seed=406)
    z, pa, pi, plan = run(sp, bank, x, time_segments=4, lanes_per_template=16, block_len=256,
                          projection=projection)
    assert plan.info()["lanes_per_template"] == 16
    zref, _, _ = oracle.filter_bank(bank.off, bank.a, bank.b, bank.d, x)
    rel, _ = rel_errors(z, zref)
    assert rel.max() <= REL_TOL, rel.max()
    check_peaks(z, zref, pa, pi)


def test_segment_count_is_clamped_by_call_length(sp):
    """More segments than 1-block pieces of the call: fewer segments run,
    and a call shorter than that runs unsegmented."""
    bank = make_bank(3, 40, (0.99, 0.999), 100, seed=407)
    for n in [300, 1100]:
        x = make_strain(1, n, seed=408)
        z, pa, pi, _ = run(sp, bank, x, time_segments=64, block_len=256)
        zref, _, _ = oracle.filter_bank(bank.off, bank.a, bank.b, bank.d, x)
        rel, _ = rel_errors(z, zref)
        assert rel.max() <= REL_TOL
        check_peaks(z, zref, pa, pi)


@pytest.mark.parametrize("projection", PROJ)
def test_segments_on_multirate_bank(sp, projection):
    bank = make_multirate_bank(12, (60, 120, 120), (1, 4, 16), (0.99, 0.9995), 1024, 409)
    x = make_strain(1, 40000, seed=410)
    plan = sp.Plan(bank, time_segments=6, projection=projection)
    z = plan.filter(torch.from_numpy(x).cuda()).cpu().numpy()
    pa, pi = plan.peak()
    plan.check()
    zref, _, _ = oracle.filter_multirate(bank.off, bank.a, bank.b, bank.d, bank.band_of,
                                        bank.decim, x)
    rel, _ = rel_errors(z, zref)
    assert rel.max() <= REL_TOL, rel.max()
    check_peaks(z, zref, pa.cpu().numpy(), pi.cpu().numpy())


def test_auto_segments_on_the_plain_workload(sp):
    """16 templates x 64 filters, 16384 samples: far fewer warps than the GPU
    holds, so the default splits the call; the result still meets the bar."""
    bank = workload_bank("plain")
    x = workload_strain("plain")
    z, pa, pi, _ = run(sp, bank, x)
    zref, _, _ = oracle.filter_bank(bank.off, bank.a, bank.b, bank.d, x)
    rel, _ = rel_errors(z, zref)
    assert rel.max() <= REL_TOL, rel.max()
    check_peaks(z, zref, pa, pi)


def test_segmented_graph_replay(sp):
    """A captured segmented call replays equal to ordinary segmented calls."""
    bank = make_bank(5, (20, 90), (0.99, 0.9995), 500, seed=411, n_det=2)
    blk, nb = 4096, 3
    x = make_strain(2, blk * nb, seed=412)
    ref = sp.Plan(bank, time_segments=4)
    zs = [ref.filter(torch.from_numpy(x[:, i * blk:(i + 1) * blk].copy()).cuda()).cpu().numpy()
          for i in range(nb)]
    pa_ref, pi_ref = ref.peak()
    plan = sp.Plan(bank, time_segments=4)
    xbuf = torch.zeros((2, blk), dtype=torch.float32, device="cuda")
    g, z, pa, pi = plan.capture(xbuf)
    plan.reset()
    torch.cuda.synchronize()
    for i in range(nb):
        xbuf.copy_(torch.from_numpy(x[:, i * blk:(i + 1) * blk].copy()))
        g.replay()
        assert np.array_equal(z.cpu().numpy(), zs[i])
    assert torch.equal(pa, pa_ref) and torch.equal(pi, pi_ref)


def test_tensor_projection_long_delays_and_slow_poles(sp):
    """Delays up to 4096 (16 chunks of history) and poles up to r = 0.99999:
    the chunk scan carries states across many chunks."""
    bank = make_bank(8, (100, 300), (0.999, 0.99999), 4096, seed=413, n_det=3)
    x = make_strain(3, 30000, seed=414)
    z, pa, pi, _ = run(sp, bank, x, chunks=[12000], time_segments=6, projection="tensor")
    zref, _, _ = oracle.filter_bank(bank.off, bank.a, bank.b, bank.d, x)
    rel, _ = rel_errors(z, zref)
    assert rel.max() <= REL_TOL, rel.max()
    check_peaks(z, zref, pa, pi)


def test_tensor_projection_follows_new_coefficients(sp):
    """spiir_set_coefficients invalidates the projection weights: the next
    segmented call uses the new poles and gains."""
    bank = make_bank(6, 64, (0.99, 0.9995), 500, seed=415)
    new = make_bank(6, 64, (0.99, 0.9995), 500, seed=416)
    x = make_strain(1, 8000, seed=417)
    plan = sp.Plan(bank, time_segments=4, projection="tensor")
    xt = torch.from_numpy(x).cuda()
    plan.filter(xt)
    plan.reset()
    # same template sizes and delays, new poles and gains
    a2 = torch.from_numpy(new.a.astype(np.complex64)).cuda()
    b2 = torch.from_numpy(new.b.astype(np.complex64)).cuda()
    plan.set_coefficients(a2, b2)
    z = plan.filter(xt).cpu().numpy()
    plan.check()
    zref, _, _ = oracle.filter_bank(bank.off, new.a, new.b, bank.d, x)
    rel, _ = rel_errors(z, zref)
    assert rel.max() <= REL_TOL, rel.max()
