"""IIR bank design (paper_1602_05573_b300.design): filters placed on a
synthetic chirp's matched filter, gains fitted by conjugate gradients whose
products are spiir_filter (A p) and spiir_filter_backward (A^H v) calls.
Against the oracle's float64 least squares (oracle.ls_gains, pinned in
tests/test_oracle_pins.py): the fitted response's overlap with the target
must match the least-squares optimum, and it must exceed the SPIIR method's
99% overlap where the oracle's does."""
import numpy as np
import pytest

import oracle
from spiir_inputs import chirp_template

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sp(cuda_device):
    import paper_1602_05573_b300
    return paper_1602_05573_b300


def test_fitted_gains_reach_the_least_squares_overlap(sp):
    from paper_1602_05573_b300 import design
    L = 360
    targets, a_all, d_all, b_all, ref_ov = [], [], [], [], []
    for f0 in (120.0, 135.0, 150.0):
        t = design.matched_target(chirp_template(2048, 60, 500, f0=f0))
        targets.append(t)
    N = max(len(t) for t in targets)
    targets = [np.pad(t, (0, N - len(t))) for t in targets]
    for t in targets:
        a, d, b = design.place_filters(t, L)
        assert len(a) == L
        a_all.append(a), d_all.append(d), b_all.append(b)
        _, resp = oracle.ls_gains(a, d, t)
        ref_ov.append(design.overlap(resp, t))
    b, z, iters = design.fit_gains(sp, np.stack(a_all), np.stack(d_all), np.stack(targets),
                                   b0=np.stack(b_all))
    ov = design.overlap(z, np.stack(targets))
    ref_ov = np.array(ref_ov)
    assert np.all(ov >= ref_ov - 2e-4), (ov, ref_ov, iters)
    assert np.all(ref_ov > 0.99) and np.all(ov > 0.99), (ov, ref_ov)
