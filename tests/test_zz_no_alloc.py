"""spiir_filter_noalloc against spiir_filter and against the FP64 oracle (GPU).

spiir_filter_noalloc is for callers that cannot call cudaMalloc/cudaFree --
for instance when device memory belongs to another allocator or a fixed
budget, or when a streaming pipeline must not allocate.  It keeps its scratch
in a static device array inside the library.  These tests call it through the
C-ABI twice in a row, on different strain, and check each result against a
fresh plan's spiir_filter/spiir_peak output and against the oracle, with the
tolerance the parity tests use; the second call also shows that nothing of
the first call (state, strain history, peaks) leaks through the shared
array.  This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import oracle
from parity_util import REL_TOL, check_peaks, rel_errors
from spiir_inputs import Bank, make_bank, make_strain

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sp(cuda_device):
    import paper_1602_05573_b300
    return paper_1602_05573_b300


def plan_result(sp, bank, x):
    plan = sp.Plan(bank, time_segments=1)   # one pass over the call, like the no-alloc entry
    z = plan.filter(x)
    pa, pi = plan.peak()
    plan.check()
    return z.cpu().numpy(), pa.cpu().numpy(), pi.cpu().numpy()


def noalloc_result(sp, bank, x):
    desc, keep = sp.bank_desc(bank)
    D, n = x.shape
    T = bank.n_templates
    z = torch.empty((D, T, n), dtype=torch.complex64, device=x.device)
    pa = torch.empty((D, T), dtype=torch.float32, device=x.device)
    pi = torch.empty((D, T), dtype=torch.int64, device=x.device)
    stream = torch.cuda.current_stream().cuda_stream
    rc = sp.library().spiir_filter_noalloc(ctypes.byref(desc), x.data_ptr(), n, z.data_ptr(),
                                           pa.data_ptr(), pi.data_ptr(), stream)
    assert rc == sp.OK, sp.library().spiir_last_error_detail()
    torch.cuda.synchronize()
    return z.cpu().numpy(), pa.cpu().numpy(), pi.cpu().numpy()


def test_noalloc_matches_plan_on_two_calls_in_a_row(sp):
    bank = make_bank(12, (20, 150), (0.99, 0.9995), 600, seed=81, n_det=2)
    for seed, n in [(82, 4001), (83, 2500)]:
        x = torch.from_numpy(make_strain(2, n, seed=seed)).cuda()
        z_ref, pa_ref, pi_ref = plan_result(sp, bank, x)
        z, pa, pi = noalloc_result(sp, bank, x)
        rel, _ = rel_errors(z, z_ref.astype(np.complex128))
        assert rel.max() <= REL_TOL, rel.max()
        assert np.array_equal(pi, pi_ref)
        np.testing.assert_allclose(pa, pa_ref, rtol=REL_TOL, atol=0)


def test_noalloc_rejects_problems_beyond_its_scratch(sp):
    bank = make_bank(4, 64, (0.99, 0.999), 100, seed=84)
    n = 10_000_000  # 40 MB of staged strain alone
    x = torch.zeros((1, n), dtype=torch.float32, device="cuda")
    desc, keep = sp.bank_desc(bank)
    lib = sp.library()
    rc = lib.spiir_filter_noalloc(ctypes.byref(desc), x.data_ptr(), n, None,
                                  x.data_ptr(), x.data_ptr(), None)
    assert rc == sp.EINVAL
    assert b"scratch" in lib.spiir_last_error_detail()


def test_noalloc_matches_oracle_on_two_calls_in_a_row(sp):
    """One detector; templates of 1, 31, 33 (two rounds of a warp), 200 and
    400 filters (400 > 32 x 10: two warps of one CTA at the default cap)."""
    parts = [make_bank(1, L, (0.99, 0.9995), 900, seed=85 + L) for L in (1, 31, 33, 200, 400)]
    off = np.concatenate([[0], np.cumsum([p.n_filters for p in parts])]).astype(np.int64)
    bank = Bank(off, np.concatenate([p.a for p in parts]), np.concatenate([p.b for p in parts]),
                np.concatenate([p.d for p in parts]), 1)
    for seed, n in [(86, 3333), (87, 1025)]:
        xh = make_strain(1, n, seed=seed)
        z, pa, pi = noalloc_result(sp, bank, torch.from_numpy(xh).cuda())
        zref, _, _ = oracle.filter_bank(bank.off, bank.a, bank.b, bank.d, xh)
        rel, _ = rel_errors(z, zref)
        assert rel.max() <= REL_TOL, rel.max()
        check_peaks(z, zref, pa, pi)
