"""Batched-launch features: CUDA-graph replay of a streaming call and the
autotuner.  Both must leave the results identical to ordinary calls / the
oracle."""
import numpy as np
import pytest

import oracle
from parity_util import REL_TOL, check_peaks, rel_errors
from spiir_inputs import make_bank, make_strain

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
    for i in range(nb):
        xbuf.copy_(torch.from_numpy(x[:, i * blk:(i + 1) * blk].copy()))
        g.replay()
        assert np.array_equal(z.cpu().numpy(), zs[i])
    assert torch.equal(pa, pa_ref) and torch.equal(pi, pi_ref)
    _, _, t = plan.state_get()
    assert t == blk * nb


def test_autotune_picks_a_layout_and_stays_exact(sp):
    bank = make_bank(40, (50, 300), (0.99, 0.9995), 1500, seed=152, n_det=2)
    x = make_strain(2, 9000, seed=153)
    plan = sp.Plan(bank, autotune=True)
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
