"""Pins of the FP64 oracle to facts that do not come from the oracle itself.

The paper prints no worked example and no coefficients, so every pin comes
from the mathematics of the recurrence in the SPIIR method (section "GPU
accelerated SPIIR method", subsection "SPIIR method"):
  y_l[k] = a_l y_l[k-1] + b_l x[k-d_l],   z[k] = sum_l y_l[k]
Pins: a hand-worked example (tests/golden), the impulse and step responses in
closed form, linearity and time invariance, brute-force direct convolution
with the summed impulse response, exact rational arithmetic, the stationary
noise variance, brute-force argmax, the multirate definition against
numpy.interp, and the adjoint against central differences and the
transpose identity.  The mutation tests at the end plant mistakes in the
oracle and check that some pin fails for each.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from spiir_inputs import make_bank, make_multirate_bank, make_strain

HERE = os.path.dirname(os.path.abspath(__file__))


def one_filter(a, b, d):
    return (np.array([0, 1]), np.array([a], np.complex128), np.array([b], np.complex128),
            np.array([d], np.int32))


def rel_err(got, want):
    scale = max(np.max(np.abs(want)), 1e-300)
    return float(np.max(np.abs(np.asarray(got) - np.asarray(want))) / scale)


# ----------------------------------------------------------------- pins ---

def pin_hand_example(mutation=0):
    g = json.load(open(os.path.join(HERE, "golden", "hand_example.json")))
    a = np.array([complex(*v) for v in g["a"]])
    b = np.array([complex(*v) for v in g["b"]])
    z, pa, pi = oracle.filter_bank(g["off"], a, b, g["d"], [g["x"]], n_threads=1,
                                   mutation=mutation)
    want = np.array([complex(*v) for v in g["z"]])
    return (np.array_equal(z[0, 0], want) and pa[0, 0] == g["peak_abs2"]
            and pi[0, 0] == g["peak_idx"])


def pin_impulse(mutation=0):
    """Impulse at k0: z[k] = b a^(k-k0-d) for k >= k0+d, else 0."""
    ok = True
    for a, b, d in [(0.97 * np.exp(0.7j), 0.3 - 0.8j, 5), (-0.5 + 0.6j, 1.25j, 0),
                    (0.999 * np.exp(2.9j), -0.01 + 0.02j, 17)]:
        n, k0 = 300, 11
        x = np.zeros((1, n))
        x[0, k0] = 1.0
        z, _, _ = oracle.filter_bank(*one_filter(a, b, d), x, n_threads=1, mutation=mutation)
        k = np.arange(n)
        want = np.where(k >= k0 + d, b * np.power(a, np.maximum(k - k0 - d, 0)), 0)
        ok &= rel_err(z[0, 0], want) < 1e-12
    return ok


def pin_step(mutation=0):
    """x = 1 from k = 0: y[k] = b (1 - a^(k-d+1)) / (1 - a) for k >= d."""
    a, b, d, n = 0.995 * np.exp(0.05j), 0.4 + 0.1j, 9, 2000
    x = np.ones((1, n))
    z, _, _ = oracle.filter_bank(*one_filter(a, b, d), x, n_threads=1, mutation=mutation)
    k = np.arange(n)
    want = np.where(k >= d, b * (1 - np.power(a, np.maximum(k - d + 1, 0))) / (1 - a), 0)
    return rel_err(z[0, 0], want) < 1e-11


def pin_direct_convolution(mutation=0):
    """Tiny banks: z = x * h with h[m] = sum_l b_l a_l^(m-d_l) [m >= d_l],
    truncated at n (exact for the first n outputs)."""
    ok = True
    rng = np.random.default_rng(7)
    for L, n in [(1, 64), (3, 200), (4, 256)]:
        a = rng.uniform(0.5, 0.99, L) * np.exp(1j * rng.uniform(0, np.pi, L))
        b = rng.standard_normal(L) + 1j * rng.standard_normal(L)
        d = rng.integers(0, 20, L).astype(np.int32)
        x = rng.standard_normal(n)
        m = np.arange(n)
        h = np.zeros(n, np.complex128)
        for l in range(L):
            h += np.where(m >= d[l], b[l] * np.power(a[l], np.maximum(m - d[l], 0)), 0)
        want = np.convolve(x, h)[:n]
        z, _, _ = oracle.filter_bank([0, L], a, b, d, x[None], n_threads=1,
                                     mutation=mutation)
        ok &= rel_err(z[0, 0], want) < 1e-12
    return ok


def pin_exact_rational(mutation=0):
    """Exact recurrence in Fractions on binary-exact inputs (<= 64 samples)."""
    bank = make_bank(1, 3, (0.9, 0.99), 6, seed=11)
    x = make_strain(1, 64, seed=12)
    A = [(Fraction(float(v.real)), Fraction(float(v.imag))) for v in bank.a]
    B = [(Fraction(float(v.real)), Fraction(float(v.imag))) for v in bank.b]
    X = [Fraction(float(v)) for v in x[0]]
    n = len(X)
    zr = [Fraction(0)] * n
    zi = [Fraction(0)] * n
    for l in range(3):
        yr, yi = Fraction(0), Fraction(0)
        (ar, ai), (br, bi), dl = A[l], B[l], int(bank.d[l])
        for k in range(n):
            xk = X[k - dl] if k >= dl else Fraction(0)
            yr, yi = ar * yr - ai * yi + br * xk, ar * yi + ai * yr + bi * xk
            zr[k] += yr
            zi[k] += yi
    want = np.array([float(r) + 1j * float(i) for r, i in zip(zr, zi)])
    z, _, _ = oracle.filter_bank(bank.off, bank.a, bank.b, bank.d, x, n_threads=1,
                                 mutation=mutation)
    return rel_err(z[0, 0], want) < 1e-14


def pin_time_shift(mutation=0):
    """Prepending s zeros shifts z by s samples, bit for bit."""
    bank = make_bank(2, 5, (0.9, 0.999), 30, seed=13)
    x = make_strain(1, 500, seed=14)
    s = 37
    xs = np.concatenate([np.zeros((1, s), np.float32), x], axis=1)
    z, _, _ = oracle.filter_bank(bank.off, bank.a, bank.b, bank.d, x, mutation=mutation)
    zs, _, _ = oracle.filter_bank(bank.off, bank.a, bank.b, bank.d, xs, mutation=mutation)
    return np.array_equal(zs[:, :, s:], z) and not np.any(zs[:, :, :s])


def pin_linearity(mutation=0):
    """z(2 x1 - 3 x2) = 2 z(x1) - 3 z(x2) (integer inputs, so the combined
    input is exact); z with gains 2b is exactly 2 z."""
    bank = make_bank(3, 6, (0.9, 0.999), 40, seed=15)
    rng = np.random.default_rng(16)
    x1 = rng.integers(-8, 9, (1, 400)).astype(np.float64)
    x2 = rng.integers(-8, 9, (1, 400)).astype(np.float64)
    f = lambda x, b=bank.b: oracle.filter_bank(bank.off, bank.a, b, bank.d, x,
                                                mutation=mutation)[0]
    ok = rel_err(f(2 * x1 - 3 * x2), 2 * f(x1) - 3 * f(x2)) < 1e-12
    ok &= np.array_equal(f(x1, 2 * bank.b.astype(np.complex128)), 2 * f(x1))
    return ok


def pin_superposition(mutation=0):
    """A template's z is the sum of its filters run as one-filter templates."""
    bank = make_bank(1, 7, (0.9, 0.999), 50, seed=17)
    x = make_strain(1, 300, seed=18)
    z, _, _ = oracle.filter_bank(bank.off, bank.a, bank.b, bank.d, x, mutation=mutation)
    L = bank.n_filters
    zs, _, _ = oracle.filter_bank(np.arange(L + 1), bank.a, bank.b, bank.d, x,
                                  mutation=mutation)
    return rel_err(z[0, 0], zs[0].sum(axis=0)) < 1e-12


def pin_peak_bruteforce(mutation=0):
    """Peak = first argmax of |z|^2, including exact ties.  With a = 0 each
    filter is a pure delayed gain, z[k] = sum_l b_l x[k-d_l], so repeated
    input values give exactly tied peaks."""
    ok = True
    x = np.zeros((1, 64))
    x[0, [5, 20, 41]] = 3.0            # three equal maxima
    x[0, [9, 30]] = -2.0
    z, pa, pi = oracle.filter_bank([0, 1], [0j], [0.5 + 0.5j], [4], x, mutation=mutation)
    p = z[0, 0].real ** 2 + z[0, 0].imag ** 2
    ok &= pi[0, 0] == int(np.argmax(p)) == 9 and pa[0, 0] == p.max()
    bank = make_bank(4, 8, (0.9, 0.999), 30, seed=19)
    xs = make_strain(1, 700, seed=20)
    z, pa, pi = oracle.filter_bank(bank.off, bank.a, bank.b, bank.d, xs, mutation=mutation)
    p = z[0].real ** 2 + z[0].imag ** 2
    ok &= np.array_equal(pi[0], np.argmax(p, axis=1))
    ok &= np.array_equal(pa[0], p.max(axis=1))
    return ok


PINS = [pin_hand_example, pin_impulse, pin_step, pin_direct_convolution,
        pin_exact_rational, pin_time_shift, pin_linearity, pin_superposition,
        pin_peak_bruteforce]


@pytest.mark.parametrize("pin", PINS, ids=lambda p: p.__name__)
def test_pin(pin):
    assert pin()


@pytest.mark.parametrize("name", sorted(oracle.MUTATIONS))
def test_planted_mistake_is_caught(name):
    """Each planted slip in the oracle makes at least one pin fail."""
    m = oracle.MUTATIONS[name]
    failed = [p.__name__ for p in PINS if not p(mutation=m)]
    assert failed, f"mutation {name} slipped past every pin"


# ------------------------------------------------------- noise variance ---

def test_noise_variance_closed_form():
    """For unit white noise the stationary E|z|^2 is
    sum_{l,m} b_l conj(b_m) a_l^(D-d_l) conj(a_m)^(D-d_m) / (1 - a_l conj(a_m)),
    D = max(d_l, d_m).  Checked statistically over many templates."""
    T, L, n, burn = 64, 4, 40000, 2000
    bank = make_bank(T, L, (0.5, 0.9), 12, seed=21)
    x = make_strain(1, n, seed=22)
    z, _, _ = oracle.filter_bank(bank.off, bank.a, bank.b, bank.d, x)
    a = bank.a.astype(np.complex128)
    b = bank.b.astype(np.complex128)
    for t in range(T):
        sl = slice(bank.off[t], bank.off[t + 1])
        at, bt, dt = a[sl], b[sl], bank.d[sl].astype(np.int64)
        D = np.maximum(dt[:, None], dt[None, :])
        num = bt[:, None] * np.conj(bt)[None, :] * at[:, None] ** (D - dt[:, None]) \
            * np.conj(at)[None, :] ** (D - dt[None, :])
        var = float(np.real(np.sum(num / (1 - at[:, None] * np.conj(at)[None, :]))))
        est = float(np.mean(np.abs(z[0, t, burn:]) ** 2))
        # correlation time <= 1/(1-0.9) = 10 samples; allow 6 standard errors
        se = var * np.sqrt(2 * 20.0 / (n - burn))
        assert abs(est - var) < 6 * se, (t, est, var)


# ------------------------------------------------------------ multirate ---

def test_multirate_single_band_is_plain_filter():
    bank = make_multirate_bank(3, (6,), (1,), (0.9, 0.999), 20, seed=23)
    x = make_strain(1, 500, seed=24)
    z1, p1, i1 = oracle.filter_multirate(bank.off, bank.a, bank.b, bank.d, bank.band_of,
                                         bank.decim, x)
    z0, p0, i0 = oracle.filter_bank(bank.off, bank.a, bank.b, bank.d, x)
    assert np.array_equal(z1, z0) and np.array_equal(i1, i0)


@pytest.mark.parametrize("n", [512, 509])
def test_multirate_matches_subsample_and_interp(n):
    """Each band = plain filter on x[::R], brought to the top rate by
    numpy.interp (which holds the last value past the end)."""
    bank = make_multirate_bank(2, (3, 4, 5), (1, 4, 16), (0.9, 0.999), 10, seed=25)
    x = make_strain(1, n, seed=26)
    z, pa, pi = oracle.filter_multirate(bank.off, bank.a, bank.b, bank.d, bank.band_of,
                                        bank.decim, x)
    m = np.arange(n)
    for t in range(2):
        want = np.zeros(n, np.complex128)
        for j, R in enumerate(bank.decim):
            sel = [l for l in range(bank.off[t], bank.off[t + 1]) if bank.band_of[l] == j]
            xb = x[:, ::R]
            zb, _, _ = oracle.filter_bank([0, len(sel)], bank.a[sel], bank.b[sel],
                                          bank.d[sel], xb)
            zb = zb[0, 0]
            nb = np.arange(zb.shape[0])
            want += np.interp(m / R, nb, zb.real) + 1j * np.interp(m / R, nb, zb.imag)
        assert rel_err(z[0, t], want) < 1e-12
        p = np.abs(z[0, t]) ** 2
        assert pi[0, t] == np.argmax(p)


# -------------------------------------------------------------- adjoint ---

def _loss(bank_off, a, b, d, x, target):
    z, _, _ = oracle.filter_bank(bank_off, a, b, d, x)
    return float(np.sum(np.abs(z - target) ** 2)), z


def test_adjoint_central_differences():
    """g_a, g_b, g_x of L = sum |z - z_t|^2 against central differences
    (h = 1e-6, FP64) on sampled coordinates."""
    bank = make_bank(3, 5, (0.9, 0.995), 25, seed=27, n_det=2)
    x = make_strain(2, 300, seed=28).astype(np.float64)
    a = bank.a.astype(np.complex128)
    b = bank.b.astype(np.complex128)
    rng = np.random.default_rng(29)
    target = 0.05 * (rng.standard_normal((2, 3, 300)) + 1j * rng.standard_normal((2, 3, 300)))
    L0, z = _loss(bank.off, a, b, bank.d, x, target)
    ga, gb, gx = oracle.adjoint(bank.off, a, b, bank.d, x, 2 * (z - target))
    h = 1e-6
    for l in rng.choice(bank.n_filters, 6, replace=False):
        for unit, g in [(1.0, ga[l].real), (1j, ga[l].imag)]:
            ap, am = a.copy(), a.copy()
            ap[l] += unit * h
            am[l] -= unit * h
            fd = (_loss(bank.off, ap, b, bank.d, x, target)[0]
                  - _loss(bank.off, am, b, bank.d, x, target)[0]) / (2 * h)
            assert abs(fd - g) <= 1e-6 * max(1.0, abs(g)), (l, unit, fd, g)
        for unit, g in [(1.0, gb[l].real), (1j, gb[l].imag)]:
            bp, bm = b.copy(), b.copy()
            bp[l] += unit * h
            bm[l] -= unit * h
            fd = (_loss(bank.off, a, bp, bank.d, x, target)[0]
                  - _loss(bank.off, a, bm, bank.d, x, target)[0]) / (2 * h)
            assert abs(fd - g) <= 1e-6 * max(1.0, abs(g)), (l, unit, fd, g)
    for det, m in [(0, 0), (0, 150), (1, 299), (1, 17)]:
        xp, xm = x.copy(), x.copy()
        xp[det, m] += h
        xm[det, m] -= h
        fd = (_loss(bank.off, a, b, bank.d, xp, target)[0]
              - _loss(bank.off, a, b, bank.d, xm, target)[0]) / (2 * h)
        assert abs(fd - gx[det, m]) <= 1e-6 * max(1.0, abs(gx[det, m]))


def test_adjoint_transpose_identity():
    """x -> z is linear (z = A x), so for any G and x':
    Re <G, A x'> = <x', g_x>, where g_x is the adjoint's input gradient."""
    bank = make_bank(4, 6, (0.9, 0.999), 40, seed=30, n_det=2)
    x = make_strain(2, 400, seed=31)
    rng = np.random.default_rng(32)
    G = rng.standard_normal((2, 4, 400)) + 1j * rng.standard_normal((2, 4, 400))
    xp = rng.standard_normal((2, 400))
    _, _, gx = oracle.adjoint(bank.off, bank.a, bank.b, bank.d, x, G)
    Axp, _, _ = oracle.filter_bank(bank.off, bank.a, bank.b, bank.d, xp)
    lhs = float(np.real(np.sum(np.conj(G) * Axp)))
    rhs = float(np.sum(xp * gx))
    assert abs(lhs - rhs) <= 1e-11 * max(abs(lhs), 1.0)


# ------------------------------------------------- network peak (coincidence) ---
# The network statistic maximises, per template, the sum over detectors of
# |z|^2 over arrival-time offsets allowed by the detector separations
# (reference detector 0; |u| <= w_d for detector d).  Pins: the single-
# detector case is the plain argmax of |z|, a planted event with known
# offsets gives the closed-form value, a pure-Python loop over every (t, d,
# u) on tiny inputs (with exact ties), and shift invariance.

def _net_brute(z, window):
    """Every t, d, u by plain loops, float32 scalars in the kernel's order."""
    z = np.asarray(z, np.complex64)
    D, T, n = z.shape
    f32 = np.float32

    def p(d, k, t):
        v = z[d, k, t]
        return f32(f32(f32(v.real) * f32(v.real)) + f32(f32(v.imag) * f32(v.imag)))
    rho = np.zeros(T, np.float32)
    tt = np.zeros(T, np.int64)
    sh = np.zeros((T, D), np.int32)
    for k in range(T):
        best, best_t, best_u = None, 0, None
        for t in range(n):
            s = p(0, k, t)
            us = [0]
            for d in range(1, D):
                m, mu = None, 0
                for u in range(-int(window[d]), int(window[d]) + 1):
                    if 0 <= t + u < n and (m is None or p(d, k, t + u) > m):
                        m, mu = p(d, k, t + u), u
                s = f32(s + m)
                us.append(mu)
            if best is None or s > best:
                best, best_t, best_u = s, t, us
        rho[k] = np.sqrt(f32(best))
        tt[k] = best_t
        sh[k] = best_u
    return rho, tt, sh


def pin_network_single_detector(mutation=None):
    rng = np.random.default_rng(140)
    z = (rng.standard_normal((1, 5, 300)) + 1j * rng.standard_normal((1, 5, 300))).astype(
        np.complex64)
    rho, t, sh = oracle.network_peak(z, [0], mutation=mutation)
    mag = np.abs(z[0].astype(np.complex128))
    assert np.array_equal(t, np.argmax(mag, axis=1))
    assert np.allclose(rho, mag[np.arange(5), t], rtol=1e-6, atol=0)
    assert not sh.any()


def pin_network_planted_event(mutation=None):
    """Zero series with one spike per detector at t0 + offset_d: the peak is
    at t0 with the offsets as shifts and rho = sqrt(sum of squared spikes);
    an offset at the window's edge still counts, one past it does not."""
    z = np.zeros((3, 2, 120), np.complex64)
    z[0, 0, 50], z[1, 0, 57], z[2, 0, 45] = 3, 4j, 12            # offsets +7, -5
    z[0, 1, 60], z[1, 1, 69], z[2, 1, 60] = 6, 8, 0.5             # +9: outside w = 7
    rho, t, sh = oracle.network_peak(z, [0, 7, 5], mutation=mutation)
    assert t[0] == 50 and list(sh[0]) == [0, 7, -5] and rho[0] == np.float32(13.0)
    # template 1: detector 1's spike is out of reach of t = 60, but t = 62
    # sees both it (u = +7) and detector 2's spike (u = -2)
    s60 = 36 + 0 + 0.25
    s62 = 0 + 64 + 0.25
    assert s62 > s60
    assert t[1] == 62 and list(sh[1]) == [0, 7, -2]
    assert rho[1] == np.sqrt(np.float32(64.25))


def pin_network_brute_force(mutation=None):
    rng = np.random.default_rng(141)
    # small integers: many exact ties in |z|^2 and in s
    z = (rng.integers(-2, 3, (3, 4, 37)) + 1j * rng.integers(-2, 3, (3, 4, 37))).astype(
        np.complex64)
    window = [0, 2, 5]
    got = oracle.network_peak(z, window, mutation=mutation)
    want = _net_brute(z, window)
    for g, w in zip(got, want):
        assert np.array_equal(g, w)
    zr = (rng.standard_normal((2, 3, 64)) + 1j * rng.standard_normal((2, 3, 64))).astype(
        np.complex64)
    for g, w in zip(oracle.network_peak(zr, [0, 3], mutation=mutation), _net_brute(zr, [0, 3])):
        assert np.array_equal(g, w)


def pin_network_shift_invariance(mutation=None):
    """Delaying detector 2 by s samples adds s to its shift and leaves the
    peak, when the offsets stay within the window and away from the ends."""
    rng = np.random.default_rng(142)
    z = 0.1 * (rng.standard_normal((3, 3, 400)) + 1j * rng.standard_normal((3, 3, 400)))
    z = z.astype(np.complex64)
    for k, t0 in enumerate((100, 200, 300)):
        z[0, k, t0], z[1, k, t0 + 2], z[2, k, t0 - 1] = 5, 4, 3
    window = [0, 6, 6]
    rho, t, sh = oracle.network_peak(z, window, mutation=mutation)
    z2 = z.copy()
    z2[2] = np.roll(z[2], 3, axis=1)
    rho2, t2, sh2 = oracle.network_peak(z2, window, mutation=mutation)
    assert np.array_equal(t, t2) and np.array_equal(rho, rho2)
    assert np.array_equal(sh2[:, 2], sh[:, 2] + 3) and np.array_equal(sh2[:, 1], sh[:, 1])
    assert list(t) == [100, 200, 300] and list(sh[:, 1]) == [2, 2, 2]


NETWORK_PINS = [pin_network_single_detector, pin_network_planted_event, pin_network_brute_force,
                pin_network_shift_invariance]


@pytest.mark.parametrize("pin", NETWORK_PINS, ids=lambda f: f.__name__)
def test_network_peak_pins(pin):
    pin()


@pytest.mark.parametrize("mutation", oracle.NETWORK_MUTATIONS)
def test_network_mutations_are_caught(mutation):
    failed = 0
    for pin in NETWORK_PINS:
        try:
            pin(mutation)
        except AssertionError:
            failed += 1
    assert failed > 0, mutation


# ------------------------------------------------- band front-end FIR ---
# Band j's input becomes sum_i h_j[i] x[R_j k - i] instead of x[R_j k].

def test_band_fir_identity_taps_are_plain_subsampling():
    bank = make_multirate_bank(3, (3, 4, 2), (1, 4, 8), (0.95, 0.999), 20, seed=160, n_det=2)
    x = make_strain(2, 640, seed=161)
    z0, _, _ = oracle.filter_multirate(bank.off, bank.a, bank.b, bank.d, bank.band_of,
                                       bank.decim, x)
    z1 = oracle.filter_multirate_fir(bank.off, bank.a, bank.b, bank.d, bank.band_of,
                                     bank.decim, x, [[1.0], None, [1.0]])
    assert np.allclose(z1, z0, rtol=0, atol=1e-12 * np.abs(z0).max())


def test_band_fir_single_tap_is_a_delay_and_scale():
    """taps = c at lag m: band j sees c x[R k - m], i.e. the plain band of
    the strain delayed by m and scaled by c (closed form, one band)."""
    bank = make_multirate_bank(2, (0, 5, 0), (1, 4, 8), (0.95, 0.999), 10, seed=162)
    x = make_strain(1, 400, seed=163).astype(np.float64)
    m, c = 3, -2.5
    taps = np.zeros(m + 1)
    taps[m] = c
    z1 = oracle.filter_multirate_fir(bank.off, bank.a, bank.b, bank.d, bank.band_of,
                                     bank.decim, x, [None, taps, None])
    xd = np.zeros_like(x)
    xd[:, m:] = c * x[:, :-m]
    z0, _, _ = oracle.filter_multirate(bank.off, bank.a, bank.b, bank.d, bank.band_of,
                                       bank.decim, xd)
    assert np.allclose(z1, z0, rtol=0, atol=1e-12 * np.abs(z0).max())


def test_band_input_is_direct_convolution():
    rng = np.random.default_rng(164)
    x = rng.standard_normal((2, 50))
    taps = rng.standard_normal(7)
    got = oracle.band_input(x, taps)
    for dd in range(2):
        for k in range(50):
            want = sum(taps[i] * x[dd, k - i] for i in range(7) if k - i >= 0)
            assert abs(got[dd, k] - want) <= 1e-12


# ------------------------------------------------- gain fit (bank design) ---

def test_ls_gains_columns_are_filter_impulse_responses():
    """The least-squares matrix's columns are the filters' unit-gain impulse
    responses: the fitted response equals the oracle filter bank run on an
    impulse with the fitted gains."""
    rng = np.random.default_rng(180)
    L, N = 9, 300
    a = (rng.uniform(0.9, 0.99, L) * np.exp(1j * rng.uniform(0, np.pi, L))).astype(np.complex64)
    d = rng.integers(0, 60, L).astype(np.int32)
    t = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    b, resp = oracle.ls_gains(a, d, t)
    x = np.zeros((1, N))
    x[0, 0] = 1.0
    z, _, _ = oracle.filter_bank(np.array([0, L]), a, b, d, x)
    assert np.allclose(z[0, 0], resp, rtol=0, atol=1e-10 * np.abs(resp).max())


def test_ls_gains_recovers_gains_in_the_span_and_leaves_an_orthogonal_residual():
    """Least-squares facts, with the filters' responses from the oracle
    filter bank on an impulse: a target the bank can produce gives back its
    gains, and the residual of any target is orthogonal to every filter's
    response (the normal equations)."""
    rng = np.random.default_rng(181)
    L, N = 12, 400
    a = (rng.uniform(0.8, 0.98, L) * np.exp(1j * rng.uniform(0, np.pi, L))).astype(np.complex64)
    d = rng.integers(0, 100, L).astype(np.int32)
    x = np.zeros((1, N))
    x[0, 0] = 1.0

    def response(gains):
        return oracle.filter_bank(np.array([0, L]), a, gains, d, x)[0][0, 0]
    b0 = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    b, _ = oracle.ls_gains(a, d, response(b0))
    assert np.allclose(b, b0, rtol=0, atol=1e-9 * np.abs(b0).max())
    t = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    b, resp = oracle.ls_gains(a, d, t)
    cols = np.stack([response(np.eye(L)[l]) for l in range(L)], axis=1)
    assert np.abs(cols.conj().T @ (t - resp)).max() <= 1e-9 * np.linalg.norm(t) * np.linalg.norm(cols)


# ------------------------------------------------- chi^2 veto ---
# Allen's discriminator with the bins read as frequency groups of a
# template's filters: chi^2 = p sum_i |z_i - z / p|^2 at the peak.

def chi2_golden():
    g = json.load(open(os.path.join(HERE, "golden", "chi2_bins_hand.json")))
    a = np.array([complex(*v) for v in g["a"]], np.complex64)
    b = np.array([complex(*v) for v in g["b"]], np.complex64)
    return g, np.array(g["off"], np.int64), a, b, np.array(g["d"], np.int32)


def pin_chi2_energy(mutation=None):
    """A filter's bin weight is the energy of its impulse response: the sum
    of |y[k]|^2 over the output of the (separately pinned) filter bank run
    on an impulse, long enough that |a|^(2N) is below 1e-17."""
    bank = make_bank(40, 1, (0.2, 0.99), 30, seed=199)
    n = 30 + int(np.ceil(np.log(1e-17) / (2 * np.log(0.99)))) + 1
    x = np.zeros((1, n))
    x[0, 0] = 1.0
    y, _, _ = oracle.filter_bank(bank.off, bank.a, bank.b, bank.d, x)
    measured = np.sum(np.abs(y[0]) ** 2, axis=-1)
    e = oracle.chi2_energy(bank.a, bank.b, mutation=mutation)
    return bool(np.all(np.abs(e - measured) <= 1e-12 * measured))


def pin_chi2_hand(mutation=None):
    """The hand-worked grouping of tests/golden/chi2_bins_hand.json."""
    g, off, a, b, _ = chi2_golden()
    return all(oracle.chi2_groups(off, a, b, p, mutation=mutation).tolist() == g["groups"][str(p)]
               for p in (2, 3))


CHI2_PINS = [pin_chi2_energy, pin_chi2_hand]


@pytest.mark.parametrize("pin", CHI2_PINS, ids=lambda p: p.__name__)
def test_chi2_pin(pin):
    assert pin()


@pytest.mark.parametrize("name", oracle.CHI2_MUTATIONS)
def test_chi2_planted_mistake_is_caught(name):
    """A wrong energy weight (no |b|^2, or 1 - |a| for 1 - |a|^2) or the end
    of a filter's share instead of its midpoint fails a chi^2 pin."""
    failed = [p.__name__ for p in CHI2_PINS if not p(mutation=name)]
    assert failed, f"chi^2 mutation {name} slipped past every pin"


def test_chi2_groups_are_contiguous_in_frequency_and_balanced():
    bank = make_bank(5, (40, 120), (0.95, 0.999), 100, seed=190)
    p = 4
    g = oracle.chi2_groups(bank.off, bank.a, bank.b, p)
    for t in range(5):
        idx = np.arange(bank.off[t], bank.off[t + 1])
        order = idx[np.argsort(np.angle(bank.a[idx].astype(np.complex128)), kind="stable")]
        assert np.all(np.diff(g[order]) >= 0)            # contiguous in frequency
        e = np.abs(bank.b[idx].astype(np.complex128)) ** 2 / (
            1 - np.abs(bank.a[idx].astype(np.complex128)) ** 2)
        share = np.array([e[g[idx] == i].sum() for i in range(p)]) / e.sum()
        assert np.all(np.abs(share - 1 / p) <= e.max() / e.sum())   # within one filter


def test_chi2_vanishes_when_the_groups_agree_and_matches_a_hand_case():
    z = np.zeros((1, 1, 3, 10), np.complex128)
    z[0, 0, :, 4] = [2 + 1j, 2 + 1j, 2 + 1j]             # equal groups: chi^2 = 0
    _, t, chi2 = oracle.chi2_at_peak(z, 3)
    assert t[0, 0] == 4 and chi2[0, 0] == 0.0
    z[0, 0, :, 4] = [3, 0, 0]                            # one group carries it all
    pk, t, chi2 = oracle.chi2_at_peak(z, 3)
    # z = 3, z/p = 1: 3 * ((3-1)^2 + 1 + 1) = 18
    assert t[0, 0] == 4 and pk[0, 0] == 3.0 and abs(chi2[0, 0] - 18.0) < 1e-12


def test_chi2_groups_sum_to_the_template():
    """Filtering each group as its own template and adding the groups gives
    the template's z (the bank is linear in its filters)."""
    bank = make_bank(3, (20, 60), (0.95, 0.999), 50, seed=191)
    x = make_strain(1, 500, seed=192)
    p = 3
    g = oracle.chi2_groups(bank.off, bank.a, bank.b, p)
    z, _, _ = oracle.filter_bank(bank.off, bank.a, bank.b, bank.d, x)
    for t in range(3):
        total = 0
        for i in range(p):
            sel = np.arange(bank.off[t], bank.off[t + 1])
            sel = sel[g[sel] == i]
            zi, _, _ = oracle.filter_bank(np.array([0, sel.size]), bank.a[sel], bank.b[sel],
                                          bank.d[sel], x)
            total = total + zi[0, 0]
        assert np.allclose(total, z[0, t], rtol=0, atol=1e-12 * np.abs(z[0, t]).max())
