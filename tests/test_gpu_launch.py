"""Batched-launch features: CUDA-graph replay of a streaming call, the
persistent launch (resident CTAs taking units from a counter), the tail
split of the layout and the autotuner.  Each must agree with the FP64
oracle (and the graph replay with ordinary calls bit for bit)."""
import numpy as np
import pytest

import oracle
from parity_util import REL_TOL, check_peaks, rel_errors
from spiir_inputs import make_bank, make_strain, workload_bank, workload_strain

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sp(cuda_device):
    import paper_1602_05573_b300
    return paper_1602_05573_b300


def test_graph_replay_continues_the_stream(sp):
    """A captured filter+peak call, replayed on successive blocks, equals the
    same blocks filtered by ordinary calls (bit for bit), and its peak
    indices count from the stream start."""
    bank = make_bank(10, (20, 150), (0.99, 0.9995), 900, seed=150, n_det=2)
    blk, nb = 2048, 4
    x = make_strain(2, blk * nb, seed=151)
    ref = sp.Plan(bank)
    zs = [ref.filter(torch.from_numpy(x[:, i * blk:(i + 1) * blk].copy()).cuda()).cpu().numpy()
          for i in range(nb)]
    pa_ref, pi_ref = ref.peak()
    plan = sp.Plan(bank)
    xbuf = torch.zeros((2, blk), dtype=torch.float32, device="cuda")
    g, z, pa, pi = plan.capture(xbuf)
    plan.reset()
    torch.cuda.synchronize()
    zref, _, _ = oracle.filter_bank(bank.off, bank.a, bank.b, bank.d, x)
    for i in range(nb):
        xbuf.copy_(torch.from_numpy(x[:, i * blk:(i + 1) * blk].copy()))
        g.replay()
        zi = z.cpu().numpy()
        assert np.array_equal(zi, zs[i])
        # against the oracle's stream, not only against the ordinary calls
        rel, _ = rel_errors(zi, zref[..., i * blk:(i + 1) * blk])
        assert rel.max() <= REL_TOL, (i, rel.max())
    assert torch.equal(pa, pa_ref) and torch.equal(pi, pi_ref)
    check_peaks(np.concatenate(zs, axis=-1), zref, pa.cpu().numpy(), pi.cpu().numpy())
    _, _, t = plan.state_get()
    assert t == blk * nb


@pytest.mark.parametrize("persistent,tail", [("on", 0), ("on", 100), ("off", 100), ("on", -1)])
def test_persistent_launch_and_tail_split_match_oracle(sp, persistent, tail):
    """A bank of more units than resident CTAs, so persistent CTAs take
    several units each (their block barriers' phases carry over between
    units); the tail split gives the smallest templates two warps."""
    bank = make_bank(2400, (20, 300), (0.99, 0.9995), 600, seed=154, n_det=2)
    x = make_strain(2, 1500, seed=155)
    plan = sp.Plan(bank, persistent=persistent, tail_split=tail)
    info = plan.info()
    assert info["n_units"] > 592
    assert info["persistent"] == (1 if persistent == "on" else 0)
    if tail > 0:
        assert info["tail_templates"] > 0
    z = plan.filter(torch.from_numpy(x).cuda()).cpu().numpy()
    pa, pi = plan.peak()
    plan.check()
    zref, _, _ = oracle.filter_bank(bank.off, bank.a, bank.b, bank.d, x)
    rel, _ = rel_errors(z, zref)
    assert rel.max() <= REL_TOL, rel.max()
    check_peaks(z, zref, pa.cpu().numpy(), pi.cpu().numpy())


def test_batched_workload_persistent_graph_sampled(sp):
    """The full batched workload (4096 templates, 3 detectors, 65536 samples)
    as one persistent launch captured in a CUDA graph, autotuned layout:
    twelve sampled (detector, template) series of a replay from zero state
    against the oracle on the matching sub-bank."""
    bank = workload_bank("batched")
    x = workload_strain("batched")
    plan = sp.Plan(bank, persistent="on", autotune=True)
    xt = torch.from_numpy(x).cuda()
    g, z, pa, pi = plan.capture(xt)            # the warm-up call runs the autotuner
    assert plan.info()["persistent"] == 1
    plan.reset()
    torch.cuda.synchronize()
    g.replay()
    plan.check()
    rng = np.random.default_rng(156)
    for det, t in [(int(rng.integers(0, 3)), int(t)) for t in rng.choice(4096, 12, replace=False)]:
        sub = bank.subset([t])
        zref, _, _ = oracle.filter_bank(sub.off, sub.a, sub.b, sub.d, x[det:det + 1])
        zg = z[det, t].cpu().numpy()[None, None]
        rel, _ = rel_errors(zg, zref)
        assert rel.max() <= REL_TOL, (det, t, rel.max())
        check_peaks(zg, zref, pa[det, t].cpu().numpy()[None, None],
                    pi[det, t].cpu().numpy()[None, None])
    del g, z
    torch.cuda.empty_cache()


def test_autotune_picks_a_layout_and_stays_exact(sp):
    bank = make_bank(40, (50, 300), (0.99, 0.9995), 1500, seed=152, n_det=2)
    x = make_strain(2, 9000, seed=153)
    # unsegmented calls: the autotuner times its candidates the way they run
    plan = sp.Plan(bank, autotune=True, time_segments=1)
    z = plan.filter(torch.from_numpy(x).cuda()).cpu().numpy()
    pa, pi = plan.peak()
    plan.check()
    zref, _, _ = oracle.filter_bank(bank.off, bank.a, bank.b, bank.d, x)
    rel, _ = rel_errors(z, zref)
    assert rel.max() <= REL_TOL
    check_peaks(z, zref, pa.cpu().numpy(), pi.cpu().numpy())
    info = plan.info()
    assert info["warps_per_cta"] in (2, 4, 8) and info["block_len"] in (256, 512)
    # later calls continue the stream on the chosen layout
    z2 = plan.filter(torch.from_numpy(x[:, :1000].copy()).cuda()).cpu().numpy()
    assert np.isfinite(z2).all()


def test_autotune_skips_time_segmented_banks(sp):
    """A bank whose calls run in time segments keeps the default layout (the
    autotuner's unsegmented prefix trials would not time it as it runs) and
    filters exactly."""
    bank = make_bank(12, (50, 120), (0.99, 0.9995), 500, seed=158)
    x = make_strain(1, 40000, seed=159)
    plan = sp.Plan(bank, autotune=True)
    z = plan.filter(torch.from_numpy(x).cuda()).cpu().numpy()
    plan.check()
    assert plan.info()["last_call_segments"] > 1
    assert plan.tune_report().startswith("skipped")
    zref, _, _ = oracle.filter_bank(bank.off, bank.a, bank.b, bank.d, x)
    rel, _ = rel_errors(z, zref)
    assert rel.max() <= REL_TOL
