"""The request loop (fsort_serve_*): continuous batching, admission by free
device memory, overlapping lanes.  Every result must be bit-identical to the
oracle's sort of that request alone, whatever mix it was served in.
"""
import time

import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2605_10390_gb300 as fs  # noqa: E402

DISTS = ["uniform", "zipf1.1", "gauss", "presorted", "equal"]


def pinned(a: np.ndarray):
    t = torch.from_numpy(a).pin_memory()
    return t


def make_requests(sizes, kb, with_vals, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for i, n in enumerate(sizes):
        k = workloads.generate(DISTS[int(rng.integers(0, 5))], n, kb, seed=seed, stream=i)
        v = rng.integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32) if with_vals else None
        reqs.append((k, v))
    return reqs


def check(reqs, outs, kb, p):
    for (k, v), (ok, ov) in zip(reqs, outs):
        wk, wv = oracle.sort(k, v, kb, p)
        assert np.array_equal(ok.numpy(), wk), k.size
        if v is not None:
            assert np.array_equal(ov.numpy(), wv), k.size


SIZES = [0, 1, 7, 100, 4096, 4097, 5000, 65_536, 70_001, 300_000, 1 << 20, (1 << 20) + 3, 2_000_000, 12, 999,
         40_000, 123_457, 3, 65_535, 250_000]


@pytest.mark.parametrize("kb,p", [(32, 32), (16, 16), (64, 40)])
def test_results_identical_alone_and_in_the_mix(kb, p):
    reqs = make_requests(SIZES * 2, kb, True, seed=kb)
    outs = [(pinned(k.copy()), pinned(v.copy())) for k, v in reqs]
    ins = [(pinned(k), pinned(v)) for k, v in reqs]
    with fs.Server(max(SIZES), kb, True, lanes=3, batch_keys=1 << 17, max_batch=16,
                   hbm_budget_bytes=256 << 20) as srv:
        tickets = [srv.submit(ik, iv, keys_out_host=ok, vals_out_host=ov, precision_bits=p)
                   for (ik, iv), (ok, ov) in zip(ins, outs)]
        results = [srv.wait(t) for t in tickets]
        st = srv.stats()
    assert all(r["status"] == 0 for r in results)
    check(reqs, outs, kb, p)
    assert st["completed"] == st["submitted"] == len(reqs)
    assert st["keys_completed"] == sum(SIZES) * 2
    assert st["max_inflight"] > 1            # work from several requests was on the device at once
    assert st["batches"] >= 1 and any(r["batched"] for r in results)
    assert st["peak_bytes"] <= st["budget_bytes"] and st["bytes_in_use"] == 0
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]


def test_admission_by_free_memory():
    # budget for about two of the largest requests at a time
    kb, n_big = 32, 1 << 21
    sizes = [n_big] * 6 + [5000] * 10
    reqs = make_requests(sizes, kb, True, seed=11)
    budget = 2 * (n_big * 8) + (1 << 20)
    outs = [(pinned(k.copy()), pinned(v.copy())) for k, v in reqs]
    ins = [(pinned(k), pinned(v)) for k, v in reqs]  # alive until every request is done
    with fs.Server(n_big, kb, True, lanes=4, hbm_budget_bytes=budget, batch_keys=8192) as srv:
        tickets = [srv.submit(ik, iv, keys_out_host=ok, vals_out_host=ov) for (ik, iv), (ok, ov)
                   in zip(ins, outs)]
        for t in tickets:
            assert srv.wait(t)["status"] == 0
        st = srv.stats()
    check(reqs, outs, kb, kb)
    assert st["peak_bytes"] <= budget
    with pytest.raises(fs.FsortError) as e:  # larger than the whole budget
        with fs.Server(1 << 22, kb, True, hbm_budget_bytes=1 << 20) as srv:
            srv.submit(np.zeros(1 << 20, np.uint32), np.zeros(1 << 20, np.uint32))
    assert e.value.status == 1


def test_queue_limit_poll_and_invalid_requests():
    kb = 32
    big = workloads.generate("uniform", 1 << 22, kb, seed=1)
    with fs.Server(1 << 22, kb, False, lanes=1, max_queue=2) as srv:
        k = [pinned(big.copy()) for _ in range(8)]
        tickets, busy, sent = [], 0, []
        for t in k:
            try:
                tickets.append(srv.submit(t))
                sent.append(t)
            except fs.FsortError as e:
                assert e.status == 5
                busy += 1
        assert busy >= 1  # one lane, two queue places: the burst overflows
        for t in tickets:
            r = srv.wait(t)
            assert r is not None and r["status"] == 0
        with pytest.raises(fs.FsortError):
            srv.poll(123456789)                                   # unknown ticket
        with pytest.raises(fs.FsortError):
            srv.submit(np.zeros((1 << 22) + 1, np.uint32))         # above max_request_keys
        with pytest.raises(fs.FsortError):
            srv.submit(np.zeros(10, np.uint32), precision_bits=33)
        assert srv.wait(srv.submit(np.zeros(0, np.uint32)))["n"] == 0
    want = np.sort(big)
    for t in sent:
        assert np.array_equal(t.numpy(), want)


def test_poisson_arrivals_report_latency():
    kb = 32
    rng = np.random.default_rng(3)
    sizes = np.exp(rng.uniform(np.log(1 << 12), np.log(1 << 21), 60)).astype(np.int64).tolist()
    reqs = make_requests(sizes, kb, True, seed=3)
    outs = [(pinned(k.copy()), pinned(v.copy())) for k, v in reqs]
    ins = [(pinned(k), pinned(v)) for k, v in reqs]
    gaps = rng.exponential(0.0005, len(reqs))
    with fs.Server(max(sizes), kb, True, lanes=4, hbm_budget_bytes=512 << 20) as srv:
        tickets = []
        for (ik, iv), (ok, ov), g in zip(ins, outs, gaps):
            time.sleep(float(g))
            tickets.append(srv.submit(ik, iv, keys_out_host=ok, vals_out_host=ov))
        lat = [srv.wait(t)["latency_ms"] for t in tickets]
        st = srv.stats()
    check(reqs, outs, kb, kb)
    assert st["completed"] == len(reqs) and st["keys_per_s"] > 0
    assert st["p50_ms"] == pytest.approx(sorted(lat)[(len(lat) + 1) // 2 - 1], rel=1e-6)


def test_learned_serving_on_the_mixture():
    n_fit = 1 << 22
    fit_keys = workloads.generate("mixture", n_fit, 64, seed=0, stream=1)
    sizes = [1 << 16, 200_000, 1 << 20, 3_000_000, 77_777, (1 << 22)]
    reqs = [(workloads.generate("mixture", n, 64, seed=5, stream=i), None) for i, n in enumerate(sizes)]
    outs = [(pinned(k.copy()), None) for k, _ in reqs]
    ins = [pinned(k) for k, _ in reqs]
    with fs.Plan(n_fit, 64, has_values=False, flags=fs.FSORT_FLAG_LEARNED) as plan:
        plan.learned_fit(torch.from_numpy(fit_keys).cuda(), seed=2)
        with fs.Server(max(sizes), 64, False, lanes=2, flags=fs.FSORT_FLAG_LEARNED, batch_keys=1 << 16) as srv:
            fs.fsort_serve_set_model(srv.handle, plan.handle)
            tickets = [srv.submit(ik, keys_out_host=ok) for ik, (ok, _) in zip(ins, outs)]
            for t in tickets:
                assert srv.wait(t)["status"] == 0
    check(reqs, outs, 64, 64)


def test_a_full_queue_refuses_with_busy():
    """One lane and room for one waiting request: the first request keeps the
    lane busy (64 MB copied in from pageable memory), so of the two requests
    submitted right after it at least one finds the queue full and gets
    FSORT_ERR_BUSY (whichever way the lane's thread is timed).  Every accepted
    request still completes with the oracle's result."""
    kb = 32
    src = [workloads.generate("uniform", 1 << 24, kb, seed=5, stream=0)]
    src += [workloads.generate("gauss", 1000, kb, seed=5, stream=i) for i in (1, 2)]
    bufs = [a.copy() for a in src]
    accepted, busy = [], 0
    with fs.Server(1 << 24, kb, False, lanes=1, max_queue=1) as srv:
        for i, b in enumerate(bufs):
            try:
                accepted.append((i, srv.submit(b)))
            except fs.FsortError as e:
                assert e.status == 5, e  # FSORT_ERR_BUSY
                busy += 1
        results = [(i, srv.wait(t)) for i, t in accepted]
    assert accepted[0][0] == 0 and busy >= 1
    for i, r in results:
        assert r["status"] == 0
        assert np.array_equal(bufs[i], oracle.sort(src[i], None, kb, kb)[0]), i
