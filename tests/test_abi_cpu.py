"""C-ABI checks that need no GPU: the library loads, exports every function
include/spiir.h declares, validates banks, and builds a correct slot layout
(host-only plans, device = -1)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1602_05573_b300 as sp
from spiir_inputs import Bank, make_bank, workload_bank

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(spiir_\w+)\s*\(", src)
    return sorted(set(names))


def test_every_declared_function_is_exported():
    lib = sp.library()
    names = declared_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(names) <= set(sp.SYMBOLS) | set(names)


def test_probe_library_loads_and_exports_its_entry():
    """The measurement probe (bench.py --workload ceiling) is a library of its
    own, outside the filter ABI: it builds, loads without a GPU and exports
    spiir_probe_step (argument checks only; no kernel runs here)."""
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "_spiir_build", os.path.join(ROOT, "paper_1602_05573_b300", "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    lib = ctypes.CDLL(b.build_probe())
    f = lib.spiir_probe_step
    f.restype = ctypes.c_int
    ms, fr = ctypes.c_double(), ctypes.c_double()
    # unsupported combinations are refused before any CUDA call
    assert f(11, 32, 4, 10, ctypes.byref(ms), ctypes.byref(fr)) == -1
    assert f(7, 8, 4, 10, ctypes.byref(ms), ctypes.byref(fr)) == -1
    assert f(7, 32, 4, 0, ctypes.byref(ms), ctypes.byref(fr)) == -1


def test_status_strings():
    lib = sp.library()
    for st in range(6):
        assert lib.spiir_status_str(st)


def bank_of(off, a, b, d, n_det=1):
    return Bank(np.asarray(off, np.int64), np.asarray(a, np.complex64),
                np.asarray(b, np.complex64), np.asarray(d, np.int32), n_det)


@pytest.mark.parametrize("bad,status", [
    (dict(a=[1.0 + 0j]), sp.EINVAL),           # |a| = 1
    (dict(a=[0.8 + 0.7j]), sp.EINVAL),         # |a| > 1
    (dict(d=[-1]), sp.EINVAL),                 # negative delay
    (dict(b=[np.nan + 0j]), sp.EINVAL),        # non-finite gain
    (dict(off=[0, 2]), None),                  # CSR inconsistent with arrays -> below
])
def test_invalid_banks_rejected(bad, status):
    kw = dict(off=[0, 1], a=[0.5 + 0j], b=[1 + 0j], d=[0])
    kw.update(bad)
    if status is None:
        kw = dict(off=[0, 1, 0], a=[0.5 + 0j], b=[1 + 0j], d=[0])  # decreasing offsets
        status = sp.EINVAL
    with pytest.raises(sp.SpiirError) as e:
        sp.Plan(bank_of(**kw), device=-1)
    assert e.value.status == status


def test_template_too_large_is_unsupported():
    """A template spans at most 8 warps of 32 lanes x max_filters_per_lane."""
    bank = make_bank(1, 32 * 4 * 8 + 1, (0.9, 0.99), 10, seed=1)
    with pytest.raises(sp.SpiirError) as e:
        sp.Plan(bank, device=-1, max_filters_per_lane=4)
    assert e.value.status == sp.EUNSUPPORTED
    sp.Plan(make_bank(1, 32 * 4 * 8, (0.9, 0.99), 10, seed=1), device=-1,
            max_filters_per_lane=4)
    sp.Plan(make_bank(1, 32 * 10 * 8, (0.9, 0.99), 10, seed=1), device=-1)
    with pytest.raises(sp.SpiirError):
        sp.Plan(make_bank(1, 32 * 10 * 8 + 1, (0.9, 0.99), 10, seed=1), device=-1)
    with pytest.raises(sp.SpiirError):
        sp.Plan(make_bank(1, 321, (0.9, 0.99), 10, seed=1), device=-1, warps_per_cta=2,
                max_filters_per_lane=4)


def test_bad_options_rejected():
    bank = make_bank(2, 8, (0.9, 0.99), 10, seed=1)
    for kw in [dict(block_len=48), dict(ring_copies=3), dict(warps_per_cta=9),
               dict(max_filters_per_lane=11)]:
        with pytest.raises(sp.SpiirError) as e:
            sp.Plan(bank, device=-1, **kw)
        assert e.value.status in (sp.EINVAL, sp.EUNSUPPORTED)


def test_chunked_tc_and_projection_options():
    bank = make_bank(3, 300, (0.9, 0.99), 10, seed=1)
    info = sp.Plan(bank, device=-1, precision="chunked_tc").info()
    assert info["max_filters_per_lane"] <= 8      # the anchored kernel's cap
    with pytest.raises(sp.SpiirError) as e:
        sp.Plan(bank, device=-1, precision="chunked_tc", chunk_len=128)
    assert e.value.status == sp.EINVAL
    opt = sp.Options()
    sp.library().spiir_options_default(ctypes.byref(opt))
    opt.projection = 3
    desc, keep = sp.bank_desc(bank)
    h = ctypes.c_void_p()
    assert sp.library().spiir_plan_create(ctypes.byref(desc), ctypes.byref(opt),
                                          ctypes.byref(h)) == sp.EINVAL


def test_kernel_times_of_an_idle_plan_are_zero():
    p = sp.Plan(make_bank(2, 8, (0.9, 0.99), 10, seed=1), device=-1, kernel_timing=True)
    t = p.kernel_times()
    assert all(ms == 0.0 and n == 0 for ms, n in t.values())


def test_host_only_plan_refuses_compute():
    bank = make_bank(2, 8, (0.9, 0.99), 10, seed=1)
    p = sp.Plan(bank, device=-1)
    lib = sp.library()
    assert lib.spiir_filter(p.handle, None, 16, None, None) == sp.EINVAL
    assert lib.spiir_reset(p.handle, None) == sp.EINVAL


@pytest.mark.parametrize("counts,W,C,Fcap,tail", [
    ([1, 31, 32, 33, 64, 65, 100, 320], 0, 4, 0, 0),
    ([5] * 37, 4, 2, 1, 0),
    ([0, 3, 200, 17], 2, 1, 4, 0),
    ([1000, 129, 7, 640], 8, 4, 4, 0),
    ([300, 257, 100], 0, 2, 10, 0),
    ([300, 257, 100, 70, 130, 64], 4, 1, 10, 200),
    ([1, 31, 32, 33, 64, 65, 100, 320] * 5, 0, 1, 0, -1),
])
def test_slot_layout_covers_every_filter_once(counts, W, C, Fcap, tail):
    rng = np.random.default_rng(3)
    off = np.zeros(len(counts) + 1, np.int64)
    off[1:] = np.cumsum(counts)
    L = int(off[-1])
    a = (rng.uniform(0.5, 0.99, L) * np.exp(1j * rng.uniform(0, np.pi, L))).astype(np.complex64)
    b = (rng.standard_normal(L) + 1j * rng.standard_normal(L)).astype(np.complex64)
    d = rng.integers(0, 700, L).astype(np.int32)
    p = sp.Plan(Bank(off, a, b, d, 2), device=-1, warps_per_cta=W, ring_copies=C,
                max_filters_per_lane=Fcap, tail_split=tail)
    sf, st = p.slots()
    if tail > 0:    # the smallest splittable templates took twice their warps
        assert p.info()["tail_templates"] > 0
    real = sf[sf >= 0]
    assert np.array_equal(np.sort(real), np.arange(L))
    # every real slot serves the template that owns the filter
    tmpl_of = np.repeat(np.arange(len(counts)), counts)
    assert np.array_equal(st[sf >= 0], tmpl_of[sf[sf >= 0]])
    info = p.info()
    per_warp = 32 // info["lanes_per_template"]
    assert info["n_units"] * info["warps_per_cta"] * per_warp >= len(counts) * 2
    assert info["max_filters_per_lane"] <= (Fcap or 10)
    assert info["history_len"] >= int(d.max())
    assert info["history_len"] % info["block_len"] == 0
    assert 1.0 <= info["bank_conflict_ratio"] <= 4.0


def test_batched_layout_statistics():
    """The 4096-template bank packs with modest padding and few bank
    conflicts: ~8% padding at 10 filters per lane (one warp per template),
    more at 4 (templates split over warps); 4 ring copies keep conflicts
    low."""
    bank = workload_bank("batched")
    for cap, pad in [(4, 1.25), (10, 1.10)]:
        info = sp.Plan(bank, device=-1, max_filters_per_lane=cap, ring_copies=4).info()
        assert info["n_slots"] / info["n_filters"] < pad
        assert info["bank_conflict_ratio"] < 1.4
        assert info["smem_bytes"] <= 227 * 1024


def test_default_ring_copies_follow_filters_per_lane():
    """With ring_copies = 0 a full-warp layout of at most 4 filters per lane
    takes two bank-skewed ring copies (fewer conflicts where the strain
    reads bound the shared-memory pipe), larger ones one; an explicit count
    is kept as given."""
    from spiir_inputs import make_bank
    few = make_bank(16, 64, (0.99, 0.9995), 1024, seed=5)      # 2 filters per lane
    many = make_bank(16, 300, (0.99, 0.9995), 1024, seed=5)    # 10 filters per lane
    info = sp.Plan(few, device=-1).info()
    assert (info["lanes_per_template"], info["max_filters_per_lane"]) == (32, 2)
    assert info["ring_copies"] == 2
    assert sp.Plan(few, device=-1, ring_copies=1).info()["ring_copies"] == 1
    assert sp.Plan(few, device=-1, ring_copies=4).info()["ring_copies"] == 4
    assert sp.Plan(few, device=-1, lanes_per_template=16).info()["ring_copies"] == 1
    assert sp.Plan(many, device=-1).info()["ring_copies"] == 1
    # the second copy spreads each round over more banks
    assert (sp.Plan(few, device=-1).info()["bank_conflict_ratio"]
            < sp.Plan(few, device=-1, ring_copies=1).info()["bank_conflict_ratio"])


def test_multirate_plan_layout_and_validation():
    from spiir_inputs import make_multirate_bank
    bank = make_multirate_bank(5, (7, 40, 3), (1, 4, 16), (0.9, 0.99), 50, seed=9)
    p = sp.Plan(bank, device=-1)
    sf, st = p.slots()
    assert np.array_equal(np.sort(sf[sf >= 0]), np.arange(bank.n_filters))
    bad = make_multirate_bank(2, (3, 3), (2, 4), (0.9, 0.99), 5, seed=9)  # no top-rate band
    with pytest.raises(sp.SpiirError) as e:
        sp.Plan(bad, device=-1)
    assert e.value.status == sp.EINVAL
    bad = make_multirate_bank(2, (3, 3), (1, 4), (0.9, 0.99), 5, seed=9)
    bad.band_of = bad.band_of.copy()
    bad.band_of[0] = 5
    with pytest.raises(sp.SpiirError):
        sp.Plan(bad, device=-1)


def test_half_warp_mode_for_small_templates():
    """In a large bank, templates of <= 96 filters (3 rounds of 32) pair up
    in a warp (16 lanes each), so each lane holds twice the filters; larger
    ones keep 32 lanes."""
    many = make_bank(4800, (20, 64), (0.9, 0.99), 100, seed=5)
    assert sp.Plan(many, device=-1).info()["lanes_per_template"] == 16
    # few templates: keep one per warp (latency-bound, needs warps)
    few = make_bank(10, (20, 64), (0.9, 0.99), 100, seed=5)
    assert sp.Plan(few, device=-1).info()["lanes_per_template"] == 32
    assert sp.Plan(few, device=-1, lanes_per_template=16).info()["lanes_per_template"] == 16
    edge = make_bank(4800, (20, 96), (0.9, 0.99), 100, seed=5)
    assert sp.Plan(edge, device=-1).info()["lanes_per_template"] == 16
    assert sp.Plan(edge, device=-1, max_filters_per_lane=5).info()["lanes_per_template"] == 32
    big = make_bank(4800, (20, 97), (0.9, 0.99), 100, seed=5)
    assert sp.Plan(big, device=-1).info()["lanes_per_template"] == 32


# ------------------------------------------------- chi^2 bins (host) ---

def _golden_chi2_bank():
    import json
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "chi2_bins_hand.json")))
    bank = bank_of(g["off"], [complex(*v) for v in g["a"]], [complex(*v) for v in g["b"]],
                   g["d"])
    return g, bank


@pytest.mark.parametrize("p", [2, 3])
def test_chi2_split_matches_the_hand_worked_bins(p):
    """spiir_chi2_split on the hand-worked bank: the regrouped bank's
    filters and offsets exactly as derived by hand."""
    g, bank = _golden_chi2_bank()
    sb = sp.chi2_split(bank, p)
    want = g["regrouped"][str(p)]
    assert sb.filter_of.tolist() == want["filter_of"]
    assert sb.off.tolist() == want["group_off"]
    assert np.array_equal(sb.a, bank.a[sb.filter_of])
    assert np.array_equal(sb.b, bank.b[sb.filter_of])
    assert np.array_equal(sb.d, bank.d[sb.filter_of])


@pytest.mark.parametrize("p,seed", [(1, 3), (4, 5), (7, 6), (64, 8)])
def test_chi2_split_matches_the_oracle_groups(p, seed):
    """The library's bins are the oracle's (oracle.chi2_groups), template by
    template, each bin's filters in frequency order."""
    import oracle
    bank = make_bank(23, (0, 140), (0.9, 0.9999), 50, seed=seed, n_det=2)
    sb = sp.chi2_split(bank, p)
    grp = oracle.chi2_groups(bank.off, bank.a, bank.b, p)
    T = bank.n_templates
    assert sb.off.shape == (T * p + 1,) and sb.off[-1] == bank.n_filters
    for t in range(T):
        idx = np.arange(bank.off[t], bank.off[t + 1])
        ang = np.angle(bank.a[idx].astype(np.complex128))
        for i in range(p):
            got = sb.filter_of[sb.off[t * p + i]:sb.off[t * p + i + 1]]
            sel = idx[grp[idx] == i]
            want = sel[np.argsort(ang[grp[idx] == i], kind="stable")]
            assert got.tolist() == want.tolist(), (t, i)


def test_chi2_split_rejects_bad_arguments():
    _, bank = _golden_chi2_bank()
    for p in (0, 65):
        with pytest.raises(sp.SpiirError) as e:
            sp.chi2_split(bank, p)
        assert e.value.status == sp.EINVAL
    from spiir_inputs import make_multirate_bank
    mb = make_multirate_bank(2, (3, 4), (1, 4), (0.9, 0.99), 5, seed=2)
    with pytest.raises(sp.SpiirError) as e:
        sp.chi2_split(mb, 2)
    assert e.value.status == sp.EUNSUPPORTED
    desc, keep = sp.bank_desc(bank)
    lib = sp.library()
    assert lib.spiir_chi2_split(ctypes.byref(desc), 2, None, None, None, None, None) == sp.EINVAL


def test_tail_split_halves_the_smallest_templates_filters_per_lane():
    """Forced tail split on the batched bank: the split templates (100..128
    filters, 4 rounds) run on two warps of 2 filters per lane; the slot
    count stays the same (no new padding rounds for even round counts) and
    the unit count grows."""
    bank = workload_bank("batched")
    base = sp.Plan(bank, device=-1).info()
    split = sp.Plan(bank, device=-1, tail_split=30).info()
    assert split["tail_templates"] > 0
    assert split["n_units"] > base["n_units"]
    assert split["n_slots"] == base["n_slots"]
