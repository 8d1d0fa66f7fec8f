"""Batched sorts (fsort_sort_batch) against the CPU oracle, segment by segment.

Segments of every size class: empty, on-chip (<= the small-segment capacity),
one tile, many tiles with a ragged tail; mixed distributions; every key width;
with and without values; 6-, 7- and 8-bit digits; graph replay with new data
of the same shape; the autotuner.  Integer data: bit-exact.
"""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2605_10390_gb300 as fs  # noqa: E402

DT = {16: torch.uint16, 32: torch.uint32, 64: torch.uint64}
DISTS = ["uniform", "zipf1.1", "gauss", "presorted", "equal"]


def make_batch(kb, sizes, with_vals, seed):
    rng = np.random.default_rng(seed)
    host, dev = [], []
    for i, n in enumerate(sizes):
        k = workloads.generate(DISTS[int(rng.integers(0, 5))], n, kb, seed=seed, stream=i)
        v = rng.integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32) if with_vals else None
        host.append((k, v))
        dk = torch.from_numpy(k).cuda() if n else torch.empty(0, dtype=DT[kb], device="cuda")
        dv = (torch.from_numpy(v).cuda() if n else torch.empty(0, dtype=torch.uint32, device="cuda")) if with_vals \
            else None
        dev.append((dk, dv, n))
    return host, dev


def check_batch(kb, p, host, dev):
    for (k, v), (dk, dv, n) in zip(host, dev):
        wk, wv = oracle.sort(k, v, kb, p)
        assert np.array_equal(dk.cpu().numpy(), wk), n
        if v is not None:
            assert np.array_equal(dv.cpu().numpy(), wv), n


SIZES = [0, 1, 7, 100, 1024, 1025, 2048, 4095, 4096, 4097, 6144, 8192, 30011, 100000, 262145, 5, 3000]


FORMS = {"table": 1, "chained": 0}  # how the larger segments' passes scatter (fsort_batch_config::large_form)


def set_form(plan, form):
    cfg = fs.fsort_batch_get_config(plan.handle)
    fs.fsort_batch_set_config(plan.handle, cfg["small_capacity"], cfg["small_ctas_per_sm"], FORMS[form])


@pytest.mark.parametrize("kb,p", [(16, 16), (16, 11), (32, 32), (32, 17), (64, 64), (64, 24)])
@pytest.mark.parametrize("with_vals", [True, False])
@pytest.mark.parametrize("form", list(FORMS))
def test_batch_matches_oracle(kb, p, with_vals, form):
    host, dev = make_batch(kb, SIZES, with_vals, seed=kb + p)
    total = sum(SIZES) + 8 * len(SIZES)
    with fs.Plan(total, kb, has_values=with_vals, max_segments=64) as plan:
        set_form(plan, form)
        plan.sort_batch(dev, precision_bits=p)
        plan.sync()
        check_batch(kb, p, host, dev)


@pytest.mark.parametrize("cap", [0, 1024, 2048, 4096])
@pytest.mark.parametrize("form", list(FORMS))
def test_batch_every_small_capacity(cap, form):
    kb, p = 32, 32
    host, dev = make_batch(kb, SIZES, True, seed=cap)
    with fs.Plan(sum(SIZES) + 8 * len(SIZES), kb, has_values=True, max_segments=64) as plan:
        fs.fsort_batch_set_config(plan.handle, cap, 1, FORMS[form])
        plan.sort_batch(dev, precision_bits=p)
        plan.sync()
        check_batch(kb, p, host, dev)


@pytest.mark.parametrize("kb,p", [(16, 16), (16, 11), (32, 32), (32, 17)])
@pytest.mark.parametrize("width", [6, 7])
@pytest.mark.parametrize("form", list(FORMS))
def test_batch_narrower_digits_match_oracle(kb, p, width, form):
    """Digit widths 6 and 7 (more passes, fewer distinct digits each) give the same output."""
    host, dev = make_batch(kb, SIZES, True, seed=kb * p + width)
    with fs.Plan(sum(SIZES) + 8 * len(SIZES), kb, has_values=True, max_segments=64) as plan:
        cfg = fs.fsort_batch_get_config(plan.handle)
        fs.fsort_batch_set_config(plan.handle, cfg["small_capacity"], cfg["small_ctas_per_sm"], FORMS[form], width)
        assert fs.fsort_batch_get_config(plan.handle)["digit_bits"] == width
        plan.sort_batch(dev, precision_bits=p)
        plan.sync()
        check_batch(kb, p, host, dev)


def test_batch_digit_width_is_checked():
    with fs.Plan(1 << 16, 32, has_values=True, max_segments=4) as plan:
        for bad in (5, 9, 16):
            with pytest.raises(fs.FsortError):
                fs.fsort_batch_set_config(plan.handle, 4096, 1, 1, bad)
    with fs.Plan(1 << 16, 64, has_values=False, max_segments=4) as plan:
        for bad in (6, 7):  # 64-bit keys would need more passes than the batch buffers hold
            with pytest.raises(fs.FsortError):
                fs.fsort_batch_set_config(plan.handle, 1024, 1, 1, bad)
        fs.fsort_batch_set_config(plan.handle, 1024, 1, 1, 8)


def test_batch_graph_is_recaptured_for_another_digit_width():
    kb, p = 32, 32
    sizes = [5000, 70000, 300, 4096, 12]
    stream = torch.cuda.Stream()
    with fs.Plan(sum(sizes) + 64, kb, has_values=True, flags=fs.FSORT_FLAG_GRAPH, max_segments=16) as plan:
        for rep, width in enumerate([8, 6, 7, 8]):  # same shape, another pass count each time
            cfg = fs.fsort_batch_get_config(plan.handle)
            fs.fsort_batch_set_config(plan.handle, cfg["small_capacity"], cfg["small_ctas_per_sm"],
                                      cfg["large_form"], width)
            host, dev = make_batch(kb, sizes, True, seed=200 + rep)
            torch.cuda.synchronize()
            with torch.cuda.stream(stream):
                plan.sort_batch(dev, precision_bits=p, stream=stream)
            plan.sync()
            stream.synchronize()
            check_batch(kb, p, host, dev)


def test_batch_graph_replay_with_new_data():
    kb, p = 32, 32
    sizes = [5000, 70000, 300, 4096, 123457, 12]
    stream = torch.cuda.Stream()
    with fs.Plan(sum(sizes) + 64, kb, has_values=True, flags=fs.FSORT_FLAG_GRAPH, max_segments=16) as plan:
        for rep in range(3):  # same shape each time: captured once, replayed
            host, dev = make_batch(kb, sizes, True, seed=100 + rep)
            torch.cuda.synchronize()
            with torch.cuda.stream(stream):
                plan.sort_batch(dev, precision_bits=p, stream=stream)
            plan.sync()
            stream.synchronize()
            check_batch(kb, p, host, dev)


def test_batch_autotune_sorts_and_picks_a_config():
    kb, p = 32, 32
    sizes = [2000, 4000, 9000, 50000, 800, 100000]
    host, dev = make_batch(kb, sizes, True, seed=7)
    with fs.Plan(sum(sizes) + 64, kb, has_values=True, max_segments=16) as plan:
        cfg, ms = fs.fsort_batch_autotune(plan.handle, dev, kb, p)
        assert cfg["small_capacity"] in (0, 1024, 2048, 4096) and cfg["large_form"] in (0, 1) and ms > 0
        assert cfg["digit_bits"] in (6, 7, 8)
        assert fs.fsort_batch_get_config(plan.handle) == cfg
        check_batch(kb, p, host, dev)


def test_autotune_cache_miss_then_hit(tmp_path):
    kb, p = 32, 32
    sizes = [2000, 4000, 9000, 50000, 800, 100000]
    path = str(tmp_path / "tune.json")
    host, dev = make_batch(kb, sizes, True, seed=8)
    with fs.Plan(sum(sizes) + 64, kb, has_values=True, max_segments=16) as plan:
        cfg, ms, hit = fs.autotune_cached(plan.handle, dev, kb, p, has_values=True, path=path)
        assert not hit and ms > 0
        check_batch(kb, p, host, dev)  # the timing runs leave the batch sorted
    host, dev = make_batch(kb, sizes, True, seed=9)
    with fs.Plan(sum(sizes) + 64, kb, has_values=True, max_segments=16) as plan:
        cfg2, _, hit = fs.autotune_cached(plan.handle, dev, kb, p, has_values=True, path=path)
        assert hit and cfg2 == cfg and fs.fsort_batch_get_config(plan.handle) == cfg
        plan.sort_batch(dev, precision_bits=p)
        plan.sync()
        check_batch(kb, p, host, dev)


def test_batch_invalid_arguments():
    k = torch.zeros(5000, dtype=torch.uint32, device="cuda")
    v = torch.zeros(5000, dtype=torch.uint32, device="cuda")
    with fs.Plan(10000, 32, has_values=True, max_segments=2) as plan:
        bad = [
            [(k, None, 10), (k, None, 10), (k, None, 10)],        # more segments than max_segments
            [(k, v, 10), (k, None, 10)],                          # values on some segments only
            [(k.data_ptr() + 4, None, 4990)],                     # large segment not 16-byte aligned
            [(k, None, 5000), (v, None, 5000), ],                 # scratch larger than max_n? (fits) -> valid
        ]
        for i, segs in enumerate(bad[:3]):
            with pytest.raises(fs.FsortError) as e:
                plan.sort_batch(segs, precision_bits=32)
            assert e.value.status == 1, i
    with fs.Plan(10000, 32, has_values=True) as plan:  # no batch tables
        with pytest.raises(fs.FsortError):
            plan.sort_batch([(k, None, 10)], precision_bits=32)
