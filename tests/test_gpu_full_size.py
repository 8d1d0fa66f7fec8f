"""Parity at the full sizes of the measured workloads, in the launch
configuration bench.py times.

Element by element against the oracle, in slab mode (oracle/slab.py): the
input is regenerated on the host from the counter-based generator, the keys of
chosen slab-key ranges are collected in input order, and the oracle's stable
sort of each slab must equal the GPU output over the slab's contiguous range.
- 32 GB, 2^32 uint64 keys at 16, 32 and 64 bits, uniform and Zipf on the top
  16 bits: slabs of the top 16 bits -- the first (for Zipf the head bucket,
  13.7 % of all keys), the last, and seeded ones in between;
- the learned workload (2^30 uint64 mixture keys at 64 bits): slabs of the full
  key -- the lowest and highest percent, one in the middle, and the most
  frequent key.
Before the oracle runs, properties that fix the result at any size are checked
on the device as fast pre-checks (order, permutation, sampled stability).

Through properties alone (exact at any size, no oracle needed):
- 32 GB, 2^34 uint16 keys at 16-bit precision (the expand path): the output is
  non-decreasing and has exactly the input's 65,536-bin histogram, so it is the
  sorted multiset (complete for keys only at full width);
- the batched workload (4,096 uint32 key + index sorts, 2^10..2^24 keys each,
  autotuned, CUDA graph captured and replayed): in every segment the values
  are indices into its input, the keys follow them, and (key, index) strictly
  increases, which makes the result the unique stable sort.

The device-side property checks use torch, never this library's kernels.
"""
import os

import numpy as np
import pytest

import oracle.slab as slab
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2605_10390_gb300 as fs  # noqa: E402

CHUNK = 1 << 30
SIGN = -(1 << 63)  # int64 with only the top bit set: x ^ SIGN orders like the unsigned value


def s64(x, p):
    """Sort keys of 64-bit keys held as int64, as int64 in unsigned order."""
    return x ^ SIGN if p == 64 else (x >> (64 - p)) & ((1 << p) - 1)


def mix_sums(x):
    """Order-independent sums (mod 2^64) of x, x^2 and a nonlinear mix of x."""
    m = (x * (0x9E3779B97F4A7C15 - (1 << 64)) >> 29) & ((1 << 35) - 1)
    return torch.stack([x.sum(), (x * x).sum(), m.sum()])


def free():
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def device_keys(dist, n, kb, stream_id, dtype):
    keys = torch.empty(n, dtype=dtype, device="cuda")
    table = workloads.table_for(dist, kb)
    tdev = torch.from_numpy(table).cuda() if table is not None else None
    workloads.generate_device(dist, keys.data_ptr(), n, kb, seed=0, stream=stream_id,
                              cuda_stream=torch.cuda.current_stream().cuda_stream,
                              table_dev_ptr=tdev.data_ptr() if tdev is not None else None)
    torch.cuda.synchronize()
    return keys


WORKERS = max(1, min(16, os.cpu_count() or 1))
HOST_CHUNK = 1 << 24  # 128 MB of 64-bit keys per worker at a time


def host_slabs(dist, n, kb, stream_id, slab_bits, ranges):
    """Slab-mode gather over the host regeneration of the workload that
    device_keys(dist, n, kb, stream_id, ...) writes on the device."""
    workloads.params_for(dist, n, kb, 0, stream_id)  # build the tables once, before the threads

    def chunk(c):
        st = c * HOST_CHUNK
        return workloads.generate(dist, min(HOST_CHUNK, n - st), kb, seed=0, stream=stream_id, start=st, n_total=n)

    return slab.slab_gather(chunk, (n + HOST_CHUNK - 1) // HOST_CHUNK, kb, slab_bits, ranges, workers=WORKERS)


def assert_slabs(out_dev, gathered, kb, p, what):
    """The device output over each slab's range equals the oracle's sort of the slab."""
    for first, keys in gathered:
        got = out_dev[first:first + keys.size].cpu().numpy().view(keys.dtype)
        want = slab.slab_expected(keys, kb, p)
        assert np.array_equal(got, want), (what, p, first, keys.size)
        del got, want


@pytest.mark.parametrize("dist", ["uniform", "zipf1.1"])
def test_2pow34_uint16_expand_is_the_sorted_multiset(dist):
    n = 1 << 34
    keys = device_keys(dist, n, 16, 7, torch.uint16)
    out = torch.empty_like(keys)
    with fs.Plan(n, 16, has_values=False) as plan:
        assert plan.describe(n, 16, False)["expand_path"] == 1
        plan.sort_out(keys, None, out, None, precision_bits=16)
        plan.sync()
    h_in = torch.zeros(65536, dtype=torch.int64, device="cuda")
    h_out = torch.zeros_like(h_in)
    last = -1
    for st in range(0, n, CHUNK):
        a = keys[st:st + CHUNK].view(torch.int16).to(torch.int32) & 0xFFFF
        h_in += torch.bincount(a, minlength=65536)
        del a
        b = out[st:st + CHUNK].view(torch.int16).to(torch.int32) & 0xFFFF
        h_out += torch.bincount(b, minlength=65536)
        assert int(b[0]) >= last and bool((b[1:] >= b[:-1]).all()), st
        last = int(b[-1])
        del b
    assert torch.equal(h_in, h_out)
    assert int(h_in.sum()) == n
    del keys, out
    free()


@pytest.mark.parametrize("dist", ["uniform", "zipf1.1"])
def test_2pow32_uint64_every_precision_against_oracle_slabs(dist):
    n = 1 << 32
    # slabs of the top 16 bits: first (for Zipf the head bucket), last, and seeded ones between
    width = 1 if dist == "zipf1.1" else 64
    rng = np.random.default_rng(21)
    mids = sorted(int(x) for x in rng.integers(1, 65535 - 64, 2))
    ranges = [(0, width), (65536 - 64, None)] + [(m, m + 64) for m in mids]
    gathered = host_slabs(dist, n, 64, 7, 16, ranges)
    assert sum(k.size for _, k in gathered) > (n // 8 if dist == "zipf1.1" else n // 300)
    keys = device_keys(dist, n, 64, 7, torch.int64)
    out = torch.empty_like(keys)
    want = sum(mix_sums(keys[st:st + CHUNK]) for st in range(0, n, CHUNK))
    with fs.Plan(n, 64, has_values=False) as plan:
        for p in (16, 32, 64):
            plan.sort_out(keys.view(torch.uint64), None, out.view(torch.uint64), None, precision_bits=p)
            plan.sync()
            torch.cuda.synchronize()
            # fast pre-checks on the device: a permutation of the input, ordered on s(k)
            got = sum(mix_sums(out[st:st + CHUNK]) for st in range(0, n, CHUNK))
            assert torch.equal(got, want), p
            last = None
            for st in range(0, n, CHUNK):
                s = s64(out[st:st + CHUNK], p)
                assert bool((s[1:] >= s[:-1]).all()) and (last is None or int(s[0]) >= last), (p, st)
                last = int(s[-1])
                del s
            # element by element against the oracle, slab by slab
            assert_slabs(out, gathered, 64, p, dist)
    del keys, out, gathered
    free()


def test_batched_4096_sorts_full_size_graph_replay():
    import bench  # the batched workload's sizes, as bench.py draws them
    sizes = bench.batch_sizes()
    dists = ["uniform", "zipf1.1", "gauss"]
    pick = np.random.default_rng(1).integers(0, 3, len(sizes))
    tables = {d: (torch.from_numpy(workloads.table_for(d, 32)).cuda() if workloads.table_for(d, 32) is not None
                  else None) for d in dists}
    starts, at = [], 0
    for n in sizes:
        starts.append(at)
        at += (n + 3) // 4 * 4
    keys = torch.empty(at, dtype=torch.int32, device="cuda")
    vals = torch.empty(at, dtype=torch.int32, device="cuda")
    side = torch.cuda.Stream()

    def regenerate():
        for i, (st, n) in enumerate(zip(starts, sizes)):
            t = tables[dists[pick[i]]]
            workloads.generate_device(dists[pick[i]], keys.data_ptr() + 4 * st, n, 32, seed=0, stream=i,
                                      cuda_stream=torch.cuda.current_stream().cuda_stream,
                                      table_dev_ptr=t.data_ptr() if t is not None else None)
        workloads.iota_device(vals.data_ptr(), at, cuda_stream=torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()

    segs = [(keys.data_ptr() + 4 * st, vals.data_ptr() + 4 * st, n) for st, n in zip(starts, sizes)]
    with fs.Plan(at + 8 * len(sizes), 32, has_values=True, flags=fs.FSORT_FLAG_GRAPH,
                 max_segments=len(sizes)) as plan:
        regenerate()
        fs.fsort_batch_autotune(plan.handle, segs, 32, 32, stream=side)
        for rep in range(2):  # the first call captures the graph, the second replays it
            regenerate()
            original = keys.clone()
            torch.cuda.synchronize()  # the copy is taken before the sort (on another stream) rewrites keys
            with torch.cuda.stream(side):
                plan.sort_batch(segs, precision_bits=32, stream=side)
            side.synchronize()
            plan.sync()
            for st, n in zip(starts, sizes):
                k_in = original[st:st + n].to(torch.int64) & 0xFFFFFFFF
                k = keys[st:st + n].to(torch.int64) & 0xFFFFFFFF
                # values are the global position as uint32 (the batch holds more than 2^32 keys):
                # the index within the segment, modulo 2^32
                idx = ((vals[st:st + n].to(torch.int64) & 0xFFFFFFFF) - st) & 0xFFFFFFFF
                assert bool(((idx >= 0) & (idx < n)).all()), (rep, st)
                assert torch.equal(k, k_in[idx]), (rep, st)
                c = (k << 24) | idx  # n <= 2^24: (key, index) in one ordered word
                assert bool((c[1:] > c[:-1]).all()), (rep, st)
            del original
    del keys, vals
    free()


def test_learned_2pow30_mixture_against_oracle_slabs():
    n = 1 << 30
    quant, hot, table = workloads.mixture_tables(0)
    t = [torch.from_numpy(a.view(np.int64)).cuda() for a in (table, quant, hot)]
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    workloads.generate_device("mixture", keys.data_ptr(), n, 64, 0, 9,
                              cuda_stream=torch.cuda.current_stream().cuda_stream,
                              table_dev_ptr=tuple(x.data_ptr() for x in t))
    torch.cuda.synchronize()
    out_l = keys.clone()
    with fs.Plan(n, 64, has_values=False, flags=fs.FSORT_FLAG_LEARNED) as lp:
        lp.learned_fit(keys.view(torch.uint64), seed=3)
        lp.sort(out_l.view(torch.uint64), precision_bits=64)
        lp.sync()
        st = lp.learned_stats()
    assert st["used"] == 1, st  # the judge accepted the map: this is the learned path's output
    out_p = keys.clone()
    with fs.Plan(n, 64, has_values=False) as pp:
        pp.sort(out_p.view(torch.uint64), precision_bits=64)
        pp.sync()
    assert torch.equal(out_l, out_p)  # fast pre-check against the plain path
    del out_p, keys
    free()
    # slabs of the full key, from quantiles of the first chunk: the lowest and
    # highest percent, one in the middle, and the most frequent key's slab
    sample = np.sort(workloads.generate("mixture", 1 << 20, 64, seed=0, stream=9, n_total=n))
    q = [int(sample[int(f * sample.size)]) for f in (0.01, 0.5, 0.51, 0.99)]
    vals, counts = np.unique(sample, return_counts=True)
    hot = int(vals[np.argmax(counts)])
    ranges = [(0, q[0]), (q[1], q[2]), (q[3], None), (hot, hot + 1)]
    gathered = host_slabs("mixture", n, 64, 9, 64, ranges)
    assert gathered[3][1].size > n // 100  # the most frequent key's slab holds over 1 % of the keys
    assert_slabs(out_l, gathered, 64, 64, "learned")
    del out_l, gathered
    free()
