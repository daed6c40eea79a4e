"""Chi^2 veto (spiir_chi2_peak on the series of chi2_split's regrouped bank)
against the oracle: oracle.chi2_groups / chi2_at_peak (pinned in
tests/test_oracle_pins.py) and the FP64 filter bank on the oracle's own
grouping.  The peak index is decided in float32 by the kernel: it must be
the oracle's or one within the oracle's epsilon-tie set (reading 4); chi^2
and the peak are compared at the kernel's index."""
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


def gpu_chi2(sp, bank, x, p):
    sb = sp.chi2_split(bank, p)
    plan = sp.Plan(sb)
    zg = plan.filter(torch.from_numpy(np.ascontiguousarray(x)).cuda())
    plan.check()
    plan.close()
    pk, t, c = sp.chi2_peak(zg, p)
    torch.cuda.synchronize()
    D, n = x.shape
    return pk.cpu().numpy(), t.cpu().numpy(), c.cpu().numpy(), zg.cpu().numpy().reshape(
        D, bank.n_templates, p, n)


def oracle_groups(bank, x, p):
    """z_i of every template and group from the FP64 oracle on its own grouping."""
    g = oracle.chi2_groups(bank.off, bank.a, bank.b, p)
    D, n = x.shape
    out = np.zeros((D, bank.n_templates, p, n), np.complex128)
    for t in range(bank.n_templates):
        for i in range(p):
            sel = np.arange(bank.off[t], bank.off[t + 1])
            sel = sel[g[sel] == i]
            if sel.size:
                zi, _, _ = oracle.filter_bank(np.array([0, sel.size]), bank.a[sel], bank.b[sel],
                                              bank.d[sel], x)
                out[:, t, i] = zi[:, 0]
    return out


def check(pk, t, c, zg_ref, p):
    z = zg_ref.sum(axis=2)
    m = np.abs(z)
    err = 3e-5 * np.sqrt(np.mean(m ** 2, axis=-1))        # per (det, template) error scale
    D, T = t.shape
    for dd in range(D):
        for k in range(T):
            tt = int(t[dd, k])
            assert m[dd, k, tt] >= m[dd, k].max() - 4 * err[dd, k], (dd, k, tt)
            assert abs(pk[dd, k] - m[dd, k, tt]) <= 4 * err[dd, k]
            zi = zg_ref[dd, k, :, tt]
            want = p * np.sum(np.abs(zi - z[dd, k, tt] / p) ** 2)
            scale = m[dd, k].max() ** 2
            assert abs(c[dd, k] - want) <= 1e-4 * scale, (dd, k, c[dd, k], want)


@pytest.mark.parametrize("p,n", [(4, 3000), (8, 1234), (1, 700)])
def test_chi2_matches_oracle(sp, p, n):
    bank = make_bank(9, (12, 150), (0.98, 0.9995), 200, seed=195 + p, n_det=2)
    x = make_strain(2, n, seed=196)
    pk, t, c, zg = gpu_chi2(sp, bank, x, p)
    check(pk, t, c, oracle_groups(bank, x, p), p)
    if p == 1:
        assert np.all(c <= 1e-6 * pk ** 2)                # one bin: chi^2 = 0


def test_chi2_kernel_on_its_own_series(sp):
    """The kernel against oracle.chi2_at_peak on the very series it read."""
    bank = make_bank(6, (40, 90), (0.98, 0.999), 100, seed=197)
    x = make_strain(1, 5000, seed=198)
    pk, t, c, zg = gpu_chi2(sp, bank, x, 4)
    check(pk, t, c, zg.astype(np.complex128), 4)


def test_chi2_on_the_batched_bank_sampled(sp):
    bank = workload_bank("batched", n_templates=512)
    x = workload_strain("batched", n=8192)
    pk, t, c, zg = gpu_chi2(sp, bank, x, 4)
    pick = np.random.default_rng(7).choice(512, 6, replace=False)
    sub = bank.subset(pick)
    check(pk[:, pick], t[:, pick], c[:, pick], oracle_groups(sub, x, 4), 4)
