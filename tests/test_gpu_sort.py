"""Parity of the CUDA hot path with the CPU oracle, through the C ABI.

Integer work throughout, so every comparison is bit-exact.  Sizes span several
tiles plus a ragged tail; edge cases cover n = 0/1, sub-vector sizes, all-equal
keys (every pass trivial), reduced precision, every key width, in-place and
out-of-place, keys-only and key/value, and the full 512 MB workload of five
distributions.
"""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU-only machines, never run there
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2605_10390_gb300 as fs  # noqa: E402

TILE = {16: 8192, 32: 6144, 64: 4096}        # chained scatter form
TABLE_TILE = {16: 11264, 32: 8192, 64: 6144}  # scatter form over the tile-offset table
DISTS = ["uniform", "zipf1.1", "gauss", "presorted", "equal"]


def gen(dist, n, kb, stream=0):
    return workloads.generate(dist, n, kb, seed=0, stream=stream)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.cpu().numpy()


def sizes(kb):
    t, u = TILE[kb], TABLE_TILE[kb]
    near = sorted({t - 1, t, t + 1, u - 1, u, u + 1, 2 * u + 1})
    return [1, 7, 8, 100] + near + [3 * t + 123, (1 << 18) + 5]


@pytest.fixture(scope="module")
def plans():
    made = {}

    def get(kb, vals, max_n=1 << 22, flags=0):
        key = (kb, vals, max_n, flags)
        if key not in made:
            made[key] = fs.Plan(max_n, kb, has_values=vals, flags=flags)
        return made[key]

    yield get
    for p in made.values():
        p.close()


# ---- K1: histograms -------------------------------------------------------------

@pytest.mark.parametrize("kb,p", [(16, 16), (16, 13), (16, 1), (32, 32), (32, 21), (64, 64), (64, 40), (64, 16)])
@pytest.mark.parametrize("dist", ["uniform", "zipf1.1", "equal"])
def test_histogram_matches_oracle(plans, kb, p, dist):
    plan = plans(kb, False)
    for n in [1, 7, TILE[kb] * 3 + 123, (1 << 19) + 3]:
        keys = gen(dist, n, kb)
        want = oracle.digit_histograms(keys, kb, p, 8)
        out = torch.zeros(want.size, dtype=torch.uint64, device="cuda")
        fs.fsort_histogram(plan.handle, dev(keys), out, key_bits=kb, precision_bits=p, digit_bits=8)
        plan.sync()
        assert np.array_equal(host(out).reshape(want.shape), want), n


@pytest.mark.parametrize("dist", DISTS)
def test_leaf_histogram_matches_oracle(plans, dist):
    """65,536-bin histogram with 16-bit tapered counters; all-equal and Zipf
    inputs drive counters through many overflow spills."""
    plan = plans(16, False, 1 << 23)
    for n in [5, 32768 * 3 + 11, (1 << 23) - 1]:
        keys = gen(dist, n, 16, stream=3)
        want = oracle.digit_histograms(keys, 16, 16, 16)[0]
        out = torch.zeros(65536, dtype=torch.uint64, device="cuda")
        fs.fsort_histogram(plan.handle, dev(keys), out, key_bits=16, precision_bits=16, digit_bits=16)
        plan.sync()
        assert np.array_equal(host(out), want), n


@pytest.mark.parametrize("dist", ["zipf1.1", "presorted", "equal", "uniform"])
def test_leaf_histogram_frequent_keys_matches_oracle(plans, dist):
    """2^26 keys: every CTA counts many rounds, so on skewed inputs a drain
    spills and the warps then count their frequent key in a register."""
    n = (1 << 26) + 12345
    plan = plans(16, False, n)
    keys = gen(dist, n, 16, stream=4)
    want = oracle.digit_histograms(keys, 16, 16, 16)[0]
    out = torch.zeros(65536, dtype=torch.uint64, device="cuda")
    fs.fsort_histogram(plan.handle, dev(keys), out, key_bits=16, precision_bits=16, digit_bits=16)
    plan.sync()
    assert np.array_equal(host(out), want)


# ---- K2: scan ------------------------------------------------------------------

@pytest.mark.parametrize("rows,bins", [(1, 256), (7, 256), (1, 65536), (3, 65536)])
def test_exclusive_scan_matches_oracle(plans, rows, bins):
    plan = plans(16, True)
    rng = np.random.default_rng(rows * bins)
    counts = rng.integers(0, 1 << 40, size=(rows, bins), dtype=np.uint64)
    counts[:, ::7] = 0
    out = torch.empty(rows * bins, dtype=torch.uint64, device="cuda")
    fs.fsort_exclusive_scan(plan.handle, dev(counts.reshape(-1)), rows, bins, out)
    plan.sync()
    want = np.stack([oracle.exclusive_scan(r) for r in counts])
    assert np.array_equal(host(out).reshape(rows, bins), want)


# ---- K3: one scatter pass ----------------------------------------------------------

@pytest.mark.parametrize("kb,shift,width", [(16, 0, 8), (16, 8, 8), (16, 3, 5), (32, 24, 8), (32, 7, 1),
                                            (64, 56, 8), (64, 13, 8)])
@pytest.mark.parametrize("with_vals", [True, False])
def test_scatter_pass_matches_oracle(plans, kb, shift, width, with_vals):
    plan = plans(kb, with_vals)
    for n in sizes(kb):
        keys = gen("zipf1.1" if shift % 2 else "uniform", n, kb, stream=5)
        vals = np.arange(n, dtype=np.uint32) * np.uint32(3) if with_vals else None
        wk, wv = oracle.scatter_pass(keys, vals, kb, shift, width)
        ko = torch.empty(n, dtype=getattr(torch, f"uint{kb}"), device="cuda")
        vo = torch.empty(n, dtype=torch.uint32, device="cuda") if with_vals else None
        fs.fsort_scatter_pass(plan.handle, dev(keys), dev(vals) if with_vals else None, ko, vo, shift, width,
                              key_bits=kb)
        plan.sync()
        assert np.array_equal(host(ko), wk), n
        if with_vals:
            assert np.array_equal(host(vo), wv), n


# ---- K4: expand ---------------------------------------------------------------------

@pytest.mark.parametrize("dist", ["uniform", "zipf1.1", "equal", "gauss"])
def test_expand_matches_oracle(plans, dist):
    plan = plans(16, False)
    for n in [1, 9, 12345, (1 << 20) + 3]:
        keys = gen(dist, n, 16, stream=7)
        counts = oracle.digit_histograms(keys, 16, 16, 16)[0]
        want = oracle.expand(counts, 16)
        out = torch.empty(n, dtype=torch.uint16, device="cuda")
        fs.fsort_expand(plan.handle, dev(counts), out)
        plan.sync()
        assert np.array_equal(host(out), want), n


# ---- the whole sort ---------------------------------------------------------------

PRECISIONS = {16: [16, 13, 9, 8, 3, 1], 32: [32, 21, 16, 9], 64: [64, 40, 32, 16, 1]}


# The two forms of the scatter passes: over fixed blocks of tiles (the default
# below 2^32 keys) and chained by decoupled look-back.
FORMS = {"blocks": 0, "chained": fs.FSORT_FLAG_CHAINED_SCATTER}


@pytest.mark.parametrize("kb", [16, 32, 64])
@pytest.mark.parametrize("with_vals", [True, False])
@pytest.mark.parametrize("in_place", [True, False])
@pytest.mark.parametrize("form", list(FORMS))
def test_sort_matches_oracle(plans, kb, with_vals, in_place, form):
    plan = plans(kb, with_vals, flags=FORMS[form])
    rng = np.random.default_rng(kb)
    for p in PRECISIONS[kb]:
        for n in sizes(kb):
            dist = DISTS[int(rng.integers(0, len(DISTS)))]
            keys = gen(dist, n, kb, stream=p)
            vals = rng.integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32) if with_vals else None
            wk, wv = oracle.sort(keys, vals, kb, p)
            dk = dev(keys)
            dv = dev(vals) if with_vals else None
            if in_place:
                fs.fsort_sort_pairs(plan.handle, dk, dv, key_bits=kb, precision_bits=p)
                ok, ov = dk, dv
            else:
                ok = torch.empty_like(dk)
                ov = torch.empty_like(dv) if with_vals else None
                fs.fsort_sort_pairs_out(plan.handle, dk, dv, ok, ov, key_bits=kb, precision_bits=p)
            plan.sync()
            assert np.array_equal(host(ok), wk), (p, n, dist)
            if with_vals:
                assert np.array_equal(host(ov), wv), (p, n, dist)


@pytest.mark.parametrize("dist", DISTS)
@pytest.mark.parametrize("form", list(FORMS))
def test_every_distribution_kv16(plans, dist, form):
    plan = plans(16, True, flags=FORMS[form])
    n = (1 << 21) + 17
    keys = gen(dist, n, 16, stream=11)
    idx = np.arange(n, dtype=np.uint32)
    wk, wv = oracle.sort(keys, idx, 16, 16)
    dk, dv = dev(keys), dev(idx)
    plan.sort(dk, dv, precision_bits=16)
    plan.sync()
    assert np.array_equal(host(dk), wk) and np.array_equal(host(dv), wv)


def test_plain_sort_small_config():
    """2^20 uint16 keys uniform on [0, 65535] from seed 0, uint32 values =
    original index, stable ascending on all 16 bits."""
    n = 1 << 20
    keys = workloads.generate("uniform", n, 16, seed=0, stream=0)
    idx = np.arange(n, dtype=np.uint32)
    wk, wv = oracle.sort(keys, idx, 16, 16)
    oracle.check_sorted_stable(keys, wk, wv, 16, 16)
    with fs.Plan(n, 16, has_values=True) as plan:
        dk, dv = dev(keys), dev(idx)
        plan.sort(dk, dv, precision_bits=16)
        plan.sync()
        assert np.array_equal(host(dk), wk) and np.array_equal(host(dv), wv)


@pytest.mark.parametrize("dist", DISTS)
def test_512mb_workload_full_size(dist):
    """2^28 uint16 keys + uint32 index values at 16-bit precision, out of place
    (the benchmark's launch configuration), every element compared."""
    n = 1 << 28
    stream = DISTS.index(dist)
    keys = workloads.generate(dist, n, 16, seed=0, stream=stream)
    idx = np.arange(n, dtype=np.uint32)
    wk, wv = oracle.sort(keys, idx, 16, 16)
    with fs.Plan(n, 16, has_values=True) as plan:
        dk, dv = dev(keys), dev(idx)
        ok, ov = torch.empty_like(dk), torch.empty_like(dv)
        plan.sort_out(dk, dv, ok, ov, precision_bits=16)
        plan.sync()
        assert np.array_equal(host(ok), wk)
        assert np.array_equal(host(ov), wv)
        assert np.array_equal(host(dk), keys)  # input untouched


def test_beyond_2pow30_keys_both_forms():
    """More keys than one look-back chunk holds (< 2^30): in the chained form
    the chunk bases carry the counts across chunks; in the block form output
    positions pass 2^30.  Keys only, 12-bit precision (radix path)."""
    n = (1 << 30) + 4099
    keys = workloads.generate("zipf1.1", n, 16, seed=0, stream=9)
    wk, _ = oracle.sort(keys, None, 16, 12)
    for flags in FORMS.values():
        with fs.Plan(n, 16, has_values=False, flags=flags) as plan:
            info = plan.describe(n, precision_bits=12)
            assert info["chunk_keys"] < n
            dk = dev(keys)
            plan.sort(dk, None, precision_bits=12)
            plan.sync()
            assert np.array_equal(host(dk), wk)
            del dk


def test_beyond_2pow31_keys_table_form():
    """More than 2^31 keys (output positions past the signed 32-bit range) in
    the default scatter form, whose offsets are 32-bit: keys only, 12-bit
    precision."""
    n = (1 << 31) + 4099
    keys = workloads.generate("uniform", n, 16, seed=0, stream=12)
    want, _ = oracle.sort(keys, None, 16, 12)
    with fs.Plan(n, 16, has_values=False) as plan:
        dk = dev(keys)
        plan.sort(dk, None, precision_bits=12)
        plan.sync()
        got = host(dk)
    assert np.array_equal(got, want)


def test_empty_input_and_describe(plans):
    plan = plans(16, True)
    k = torch.empty(0, dtype=torch.uint16, device="cuda")
    fs.fsort_sort_pairs(plan.handle, k, None, key_bits=16, precision_bits=16)
    info = plan.describe(1 << 20, precision_bits=16, has_values=True)
    assert info["passes"] == 2 and info["digit_bits"] == 8 and info["expand_path"] == 0
    assert info["algorithmic_bytes"] == 26 * (1 << 20)
    assert info["scatter_form"] == 0 and info["tile_keys"] == TABLE_TILE[16]  # table form below 2^32 keys
    assert info["num_tiles"] == -(-(1 << 20) // TABLE_TILE[16])
    chained = plans(16, True, flags=FORMS["chained"]).describe(1 << 20, precision_bits=16, has_values=True)
    assert chained["scatter_form"] == 1 and chained["tile_keys"] == TILE[16]
    info = plan.describe(1 << 20, precision_bits=16, has_values=False)
    assert info["expand_path"] == 1 and info["algorithmic_bytes"] == 4 * (1 << 20)


def test_invalid_arguments(plans):
    plan = plans(16, False, 1000)
    k = torch.zeros(2000, dtype=torch.uint16, device="cuda")
    v = torch.zeros(2000, dtype=torch.uint32, device="cuda")
    c = torch.zeros(1024, dtype=torch.int64, device="cuda")
    c2 = torch.zeros(1024, dtype=torch.int64, device="cuda")
    bad = [
        lambda: fs.fsort_sort_pairs(plan.handle, k, None, n=1001, key_bits=16, precision_bits=16),  # n > max_n
        lambda: fs.fsort_sort_pairs(plan.handle, k, None, n=10, key_bits=32, precision_bits=16),    # width
        lambda: fs.fsort_sort_pairs(plan.handle, k, None, n=10, key_bits=16, precision_bits=0),
        lambda: fs.fsort_sort_pairs(plan.handle, k, None, n=10, key_bits=16, precision_bits=17),
        lambda: fs.fsort_sort_pairs(plan.handle, k, v, n=10, key_bits=16, precision_bits=16),       # no values
        lambda: fs.fsort_sort_pairs(plan.handle, k.data_ptr() + 2, None, n=10, key_bits=16, precision_bits=16),
        lambda: fs.fsort_sort_pairs_out(plan.handle, k, None, k.data_ptr() + 16, None, n=100, key_bits=16,
                                        precision_bits=16),  # overlap
        lambda: fs.fsort_sort_pairs_host(plan.handle, np.zeros(10, np.uint16), None, key_bits=16,
                                         precision_bits=16),  # plan without host buffers
        # count and offset arrays off their 8-byte alignment: refused on the host
        lambda: fs.fsort_histogram(plan.handle, k, c.data_ptr() + 4, n=100, key_bits=16, precision_bits=16),
        lambda: fs.fsort_exclusive_scan(plan.handle, c.data_ptr() + 4, 1, 256, c2),
        lambda: fs.fsort_exclusive_scan(plan.handle, c, 1, 256, c2.data_ptr() + 2),
        lambda: fs.fsort_expand(plan.handle, c.data_ptr() + 4, k, n=10, key_bits=16),
    ]
    for f in bad:
        with pytest.raises(fs.FsortError) as e:
            f()
        assert e.value.status == 1
    with pytest.raises(fs.FsortError):
        fs.fsort_plan_create(0, 16)
    with pytest.raises(fs.FsortError):
        fs.fsort_plan_create(10, 24)
    plan.sync()


def test_host_buffer_entry_point():
    n = 300001
    keys = gen("gauss", n, 16, stream=2)
    idx = np.arange(n, dtype=np.uint32)
    wk, wv = oracle.sort(keys, idx, 16, 16)
    with fs.Plan(n, 16, has_values=True, flags=fs.FSORT_FLAG_HOST_IO) as plan:
        hk = torch.from_numpy(keys.copy()).pin_memory()
        hv = torch.from_numpy(idx.copy()).pin_memory()
        fs.fsort_sort_pairs_host(plan.handle, hk, hv, key_bits=16, precision_bits=16)
        assert np.array_equal(hk.numpy(), wk) and np.array_equal(hv.numpy(), wv)


def test_repeated_sorts_reuse_plan_state(plans):
    """Plan scratch (histogram accumulators, look-back regions, counters) must
    come back clean after every call."""
    plan = plans(32, True)
    for rep in range(4):
        n = [5000, 123457, 77, 1 << 20][rep]
        keys = gen(DISTS[rep], n, 32, stream=rep)
        idx = np.arange(n, dtype=np.uint32)
        wk, wv = oracle.sort(keys, idx, 32, 32 - rep * 5)
        dk, dv = dev(keys), dev(idx)
        fs.fsort_sort_pairs(plan.handle, dk, dv, key_bits=32, precision_bits=32 - rep * 5)
        plan.sync()
        assert np.array_equal(host(dk), wk) and np.array_equal(host(dv), wv)


def test_allocation_failure_is_reported_and_the_device_stays_usable():
    """A plan or a server whose device memory cannot exist (2^36 64-bit keys
    with values need over 1 TB of scratch) returns FSORT_ERR_OOM from its one
    allocation; nothing is left behind and the next plan sorts as usual."""
    with pytest.raises(fs.FsortError) as e:
        fs.fsort_plan_create(1 << 36, 64, has_values=True)
    assert e.value.status == 2
    with pytest.raises(fs.FsortError) as e:
        fs.fsort_serve_create(1 << 20, 32, True, hbm_budget_bytes=1 << 41)
    assert e.value.status == 2
    keys = gen("uniform", 100_003, 32, stream=13)
    want, _ = oracle.sort(keys, None, 32, 32)
    with fs.Plan(keys.size, 32, has_values=False) as plan:
        dk = dev(keys)
        plan.sort(dk, None, precision_bits=32)
        plan.sync()
        assert np.array_equal(host(dk), want)
