"""The adjoint kernel (spiir_filter_backward) against the FP64 oracle's
adjoint, which tests/test_oracle_pins.py pins to central differences and to
the transpose identity.  Both evaluations of g_a, g_b run every case: the
reverse form (checkpointed forward, reverse-time recurrence) and the tangent
form (forward-time derivative recurrences); g_x comes from the shifted-frame
pass seeded by the reverse pass or by its own projection.

Gradient tolerance: the kernel accumulates each g_a, g_b over n samples in
FP32 from FP32 states, and g_x in shared memory, then into global memory
with float atomics (so its last bits depend on summation order); the bar is
1e-3 of the largest entry of g_a, g_b and |g_x|.
"""
import numpy as np
import pytest

import oracle
from spiir_inputs import make_bank, make_strain, perturb, workload_bank, workload_strain

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
GRAD_TOL = 1e-3
FORMS = ["reverse", "tangent"]


@pytest.fixture(scope="module")
def sp(cuda_device):
    import paper_1602_05573_b300
    return paper_1602_05573_b300


def rel_inf(got, want):
    return float(np.max(np.abs(got - want)) / max(np.max(np.abs(want)), 1e-300))


def gpu_backward(sp, bank, x, gz, **opts):
    plan = sp.Plan(bank, **opts)
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    gzt = torch.from_numpy(np.ascontiguousarray(gz.astype(np.complex64))).cuda()
    ga, gb, gx = plan.backward(xt, gzt)
    plan.check()
    return ga.cpu().numpy(), gb.cpu().numpy(), gx.cpu().numpy()


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("n,D,opts", [(3000, 2, {}), (1024, 1, {}), (777, 1, {"warps_per_cta": 1}),
                                      (2500, 3, {"max_filters_per_lane": 2}), (5, 1, {})])
def test_adjoint_matches_oracle(sp, n, D, opts, form):
    bank = make_bank(7, (20, 150), (0.99, 0.9995), 700, seed=90 + n, n_det=D)
    x = make_strain(D, n, seed=91)
    rng = np.random.default_rng(92)
    gz = (rng.standard_normal((D, 7, n)) + 1j * rng.standard_normal((D, 7, n))).astype(np.complex64)
    ga, gb, gx = gpu_backward(sp, bank, x, gz, adjoint_form=form, **opts)
    ra, rb, rx = oracle.adjoint(bank.off, bank.a, bank.b, bank.d, x, gz)
    assert rel_inf(ga, ra) <= GRAD_TOL
    assert rel_inf(gb, rb) <= GRAD_TOL
    assert rel_inf(gx, rx) <= GRAD_TOL


@pytest.mark.parametrize("form", FORMS)
def test_adjoint_half_warp_templates(sp, form):
    """Templates of <= 64 filters share warps (16 lanes each) in the forward
    layout; the adjoint reads each half's own g_z."""
    bank = make_bank(5, (10, 64), (0.99, 0.9995), 500, seed=98, n_det=2)
    x = make_strain(2, 2100, seed=99)
    rng = np.random.default_rng(100)
    gz = (rng.standard_normal((2, 5, 2100)) + 1j * rng.standard_normal((2, 5, 2100))).astype(
        np.complex64)
    ga, gb, gx = gpu_backward(sp, bank, x, gz, lanes_per_template=16, adjoint_form=form)
    ra, rb, rx = oracle.adjoint(bank.off, bank.a, bank.b, bank.d, x, gz)
    assert rel_inf(ga, ra) <= GRAD_TOL
    assert rel_inf(gb, rb) <= GRAD_TOL
    assert rel_inf(gx, rx) <= GRAD_TOL


def test_adjoint_leaves_streaming_state_alone(sp):
    bank = make_bank(3, 40, (0.99, 0.999), 100, seed=93)
    x = torch.from_numpy(make_strain(1, 2000, seed=94)).cuda()
    plan = sp.Plan(bank)
    z1 = plan.filter(x[:, :1000].contiguous())
    plan.backward(x, torch.ones((1, 3, 2000), dtype=torch.complex64, device="cuda"))
    z2 = plan.filter(x[:, 1000:].contiguous())
    ref = sp.Plan(bank)
    r1 = ref.filter(x[:, :1000].contiguous())
    r2 = ref.filter(x[:, 1000:].contiguous())
    assert torch.equal(z1, r1) and torch.equal(z2, r2)


def test_adjoint_workload_full_size(sp):
    """256 templates x 200 filters, 65536 samples; loss = sum |z_fit -
    z_target|^2 with z_target from +-1% perturbed coefficients.  g_z and the
    reference gradients come from the oracle."""
    bank = workload_bank("adjoint")
    target = perturb(bank, seed=506)
    x = workload_strain("adjoint")
    z_fit, _, _ = oracle.filter_bank(bank.off, bank.a, bank.b, bank.d, x)
    z_tgt, _, _ = oracle.filter_bank(target.off, target.a, target.b, target.d, x)
    gz = (2 * (z_fit - z_tgt)).astype(np.complex64)
    del z_fit, z_tgt
    ga, gb, gx = gpu_backward(sp, bank, x, gz)
    ra, rb, rx = oracle.adjoint(bank.off, bank.a, bank.b, bank.d, x, gz)
    assert rel_inf(ga, ra) <= GRAD_TOL
    assert rel_inf(gb, rb) <= GRAD_TOL
    assert rel_inf(gx, rx) <= GRAD_TOL


def test_autograd_function_and_a_fitting_step(sp):
    """loss.backward() through the autograd Function equals the direct
    adjoint call, and a small gradient step lowers the mismatch."""
    bank = make_bank(4, 30, (0.99, 0.999), 200, seed=95)
    target = perturb(bank, seed=96)
    x = torch.from_numpy(make_strain(1, 4096, seed=97)).cuda()
    plan = sp.Plan(bank)
    tplan = sp.Plan(target)
    z_t = tplan.filter(x).detach()
    a = torch.from_numpy(bank.a).cuda().requires_grad_(True)
    b = torch.from_numpy(bank.b).cuda().requires_grad_(True)
    xg = x.clone().requires_grad_(True)
    z = sp.spiir_filter(xg, a, b, plan)
    loss = torch.sum(torch.abs(z - z_t) ** 2)
    loss.backward()
    gz = (2 * (z - z_t)).detach()
    ga, gb, gx = plan.backward(x, gz)
    # autograd forms g_z through abs() and pow(), so it differs from 2 (z - z_t)
    # in the last bits; g_x also depends on the atomics' summation order
    for got, want in [(a.grad, ga), (b.grad, gb), (xg.grad, gx)]:
        assert rel_inf(got.cpu().numpy(), want.cpu().numpy()) <= 1e-5
    with torch.no_grad():
        b2 = b - 1e-3 * b.grad / b.grad.abs().max() * b.abs().max()
        loss2 = torch.sum(torch.abs(sp.spiir_filter(x, a.detach(), b2, plan) - z_t) ** 2)
    assert float(loss2) < float(loss.detach())


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("P", [1, 3, 5])
def test_adjoint_time_segments(sp, P, form):
    """The reverse pass split into P time segments of whole checkpoint
    intervals (each from the adjoint state projected to its end) gives the
    oracle's gradients."""
    bank = make_bank(6, (40, 160), (0.995, 0.9999), 900, seed=120, n_det=2)
    n = 9000
    x = make_strain(2, n, seed=121)
    rng = np.random.default_rng(122)
    gz = (rng.standard_normal((2, 6, n)) + 1j * rng.standard_normal((2, 6, n))).astype(np.complex64)
    ga, gb, gx = gpu_backward(sp, bank, x, gz, time_segments=P, adjoint_form=form)
    ra, rb, rx = oracle.adjoint(bank.off, bank.a, bank.b, bank.d, x, gz)
    assert rel_inf(ga, ra) <= GRAD_TOL
    assert rel_inf(gb, rb) <= GRAD_TOL
    assert rel_inf(gx, rx) <= GRAD_TOL


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("delays", ["equal", "distinct"])
def test_adjoint_delay_extremes(sp, delays, form):
    """g_x gathers every filter's contribution at k - d in shared memory:
    equal delays everywhere make every filter of a round add to the same
    address at once, delays equal to the filter's index in its template make
    every address of a round different."""
    import dataclasses
    bank = make_bank(5, (70, 200), (0.99, 0.9995), 300, seed=140, n_det=2)
    counts = np.diff(bank.off)
    if delays == "equal":
        d = np.full(bank.d.shape, 37, np.int32)
    else:
        d = np.concatenate([np.arange(c, dtype=np.int32) for c in counts])
    bank = dataclasses.replace(bank, d=d)
    n = 2600
    x = make_strain(2, n, seed=141)
    rng = np.random.default_rng(142)
    gz = (rng.standard_normal((2, 5, n)) + 1j * rng.standard_normal((2, 5, n))).astype(np.complex64)
    ga, gb, gx = gpu_backward(sp, bank, x, gz, adjoint_form=form)
    ra, rb, rx = oracle.adjoint(bank.off, bank.a, bank.b, bank.d, x, gz)
    assert rel_inf(ga, ra) <= GRAD_TOL
    assert rel_inf(gb, rb) <= GRAD_TOL
    assert rel_inf(gx, rx) <= GRAD_TOL


@pytest.mark.parametrize("D", [1, 3])
def test_adjoint_tangent_filter_pairs(sp, D):
    """A bank of 220 templates x 151..251 filters: on one detector the
    tangent pass holds one filter per thread; on three it is large enough to
    hold two filters of one template per thread (>= 12 warps per SM at
    pairs), where odd filter counts leave half-empty pairs and warps hold the
    end of one template and the start of the next."""
    bank = make_bank(220, (151, 251), (0.99, 0.9995), 600, seed=150, n_det=D)
    n = 2100
    x = make_strain(D, n, seed=151)
    rng = np.random.default_rng(152)
    gz = (rng.standard_normal((D, 220, n)) + 1j * rng.standard_normal((D, 220, n))).astype(
        np.complex64)
    for want_gx in (True, False):
        plan = sp.Plan(bank, adjoint_form="tangent")
        xt = torch.from_numpy(x).cuda()
        ga, gb, gx = plan.backward(xt, torch.from_numpy(gz).cuda(), want_gx=want_gx)
        plan.check()
        ra, rb, rx = oracle.adjoint(bank.off, bank.a, bank.b, bank.d, x, gz, want_gx=want_gx)
        assert rel_inf(ga.cpu().numpy(), ra) <= GRAD_TOL
        assert rel_inf(gb.cpu().numpy(), rb) <= GRAD_TOL
        if want_gx:
            assert rel_inf(gx.cpu().numpy(), rx) <= GRAD_TOL
