"""The allocation-free scatter pass gives the same result as the plan-based one.

fsort_scatter_pass_noalloc is for callers that cannot call cudaMalloc where
they sort (another component owns the device memory budget, or the path must
not take cudaMalloc's implicit synchronisation): it keeps its scratch in a
fixed device array inside the library instead of a plan.  This file is named so
that pytest collects it last; it passes alone in a fresh process and after the
other tests.  Integer data, so "within tolerance" means bit-exact.
"""
import threading

import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2605_10390_gb300 as fs  # noqa: E402


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("key_bits,with_vals", [(16, True), (32, False), (64, True)])
def test_noalloc_matches_plan_based_pass_twice(key_bits, with_vals):
    n = 3 * 8192 + 4097
    plan = fs.Plan(n, key_bits, has_values=with_vals)
    try:
        # Two calls in a row with different inputs and digits: the shared
        # scratch must come back clean between them.
        for call, (dist, shift, width) in enumerate([("zipf1.1", key_bits - 8, 8), ("uniform", 3, 5)]):
            keys = workloads.generate(dist, n, key_bits, seed=0, stream=20 + call)
            vals = (np.arange(n, dtype=np.uint32) * np.uint32(7)) if with_vals else None
            dk = _dev(keys)
            dv = _dev(vals) if with_vals else None
            ref_k = torch.empty_like(dk)
            ref_v = torch.empty_like(dv) if with_vals else None
            fs.fsort_scatter_pass(plan.handle, dk, dv, ref_k, ref_v, shift, width, key_bits=key_bits)
            plan.sync()
            got_k = torch.empty_like(dk)
            got_v = torch.empty_like(dv) if with_vals else None
            fs.fsort_scatter_pass_noalloc(dk, dv, got_k, got_v, shift, width, key_bits=key_bits)
            torch.cuda.synchronize()
            assert torch.equal(got_k, ref_k), call
            if with_vals:
                assert torch.equal(got_v, ref_v), call
            # and both equal the oracle's pass on the same input
            want_k, want_v = oracle.scatter_pass(keys, vals, key_bits, shift, width)
            assert np.array_equal(got_k.cpu().numpy(), want_k), call
            if with_vals:
                assert np.array_equal(got_v.cpu().numpy(), want_v), call
    finally:
        plan.close()


def test_noalloc_at_its_largest_size_with_64_bit_keys_and_values():
    """n = FSORT_NOALLOC_MAX_KEYS with 64-bit keys: the look-back region of the
    fixed scratch is completely full (one row per 4,096-key tile) and abuts the
    histogram; the result must equal the plan-based pass bit for bit on two
    calls in a row, and satisfy the definition of a stable pass (checked on the
    device: digits non-decreasing, input positions increasing within a digit,
    every key taken from its position)."""
    n, kb, shift, width = fs.FSORT_NOALLOC_MAX_KEYS, 64, 56, 8
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    workloads.generate_device("uniform", keys.data_ptr(), n, kb, seed=1, stream=77,
                              cuda_stream=torch.cuda.current_stream().cuda_stream)
    vals = torch.arange(n, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    with fs.Plan(n, kb, has_values=True) as plan:
        ref_k, ref_v = torch.empty_like(keys), torch.empty_like(vals)
        fs.fsort_scatter_pass(plan.handle, keys.view(torch.uint64), vals, ref_k.view(torch.uint64), ref_v,
                              shift, width, key_bits=kb)
        plan.sync()
    got_k, got_v = torch.empty_like(keys), torch.empty_like(vals)
    for _ in range(2):
        got_k.zero_()
        got_v.zero_()
        fs.fsort_scatter_pass_noalloc(keys.view(torch.uint64), vals, got_k.view(torch.uint64), got_v, shift, width,
                                      key_bits=kb)
        torch.cuda.synchronize()
        assert torch.equal(got_k, ref_k) and torch.equal(got_v, ref_v)
    # the definition on the device: stable by the top byte, values are the input positions
    d = (got_k >> 56) & 0xFF
    assert bool((d[1:] >= d[:-1]).all())
    same = d[1:] == d[:-1]
    assert bool((got_v[1:][same] > got_v[:-1][same]).all())
    assert torch.equal(keys[got_v.long()], got_k)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    k = torch.empty(16, dtype=torch.uint16, device="cuda")
    with pytest.raises(fs.FsortError) as e:
        fs.fsort_scatter_pass_noalloc(k, None, torch.empty_like(k), None, 0, 8, n=fs.FSORT_NOALLOC_MAX_KEYS + 1,
                                      key_bits=16)
    assert e.value.status == 1


def test_noalloc_calls_from_several_threads_take_turns():
    """Four host threads, each on its own stream with its own data, call the
    pass at once: the library runs them one at a time on the shared array, so
    every result equals the oracle's pass on that thread's input."""
    n, kb = 2 * 8192 + 1001, 32
    cases = []
    for t in range(4):
        keys = workloads.generate(["uniform", "zipf1.1", "gauss", "presorted"][t], n, kb, seed=5, stream=40 + t)
        vals = np.arange(n, dtype=np.uint32) + np.uint32(t << 24)
        shift, width = [(0, 8), (24, 8), (13, 6), (5, 3)][t]
        cases.append((keys, vals, shift, width, oracle.scatter_pass(keys, vals, kb, shift, width)))
    results, errors = [None] * 4, []

    def worker(t):
        try:
            keys, vals, shift, width, _ = cases[t]
            stream = torch.cuda.Stream()
            with torch.cuda.stream(stream):
                dk, dv = _dev(keys), _dev(vals)
                ok, ov = torch.empty_like(dk), torch.empty_like(dv)
                stream.synchronize()
                for _ in range(3):  # repeated calls interleave with the other threads'
                    fs.fsort_scatter_pass_noalloc(dk, dv, ok, ov, shift, width, key_bits=kb, stream=stream)
                    results[t] = (ok.cpu().numpy(), ov.cpu().numpy())
        except Exception as e:  # reported below, on the main thread
            errors.append((t, e))

    threads = [threading.Thread(target=worker, args=(t,)) for t in range(4)]
    for th in threads:
        th.start()
    for th in threads:
        th.join(timeout=300)
    assert not errors, errors
    for t, (_, _, _, _, (wk, wv)) in enumerate(cases):
        assert np.array_equal(results[t][0], wk), t
        assert np.array_equal(results[t][1], wv), t
