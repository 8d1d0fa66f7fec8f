"""Streaming histogram (fsort_hist_*): batches accumulated one by one, never
re-read; counts, rank, select and the expanded sorted multiset against the
oracle's histogram tree (Alg. 1-3) and expand (Alg. 5) over the concatenation.
Integer results: bit-exact.
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

DISTS = ["uniform", "zipf1.1", "gauss", "presorted", "equal"]
BATCHES = [0, 1, 1000, 70_001, 1 << 20, 3, (1 << 18) + 5]


def batches(kb, seed):
    return [workloads.generate(DISTS[i % 5], n, kb, seed=seed, stream=i) for i, n in enumerate(BATCHES)]


def leaf_counts(tree, p):
    return tree[(1 << p) - 1:]  # level p of the tree (level l starts at 2^l - 1)


@pytest.mark.parametrize("kb,p", [(16, 16), (32, 20), (64, 24), (32, 8), (16, 1)])
def test_stream_counts_rank_select_expand(kb, p):
    bs = batches(kb, seed=p)
    allk = np.concatenate(bs)
    tree = oracle.tree_build(allk, kb, p)
    with fs.StreamHistogram(kb, p) as h:
        for b in bs:
            h.accumulate(torch.from_numpy(b).cuda() if b.size else torch.empty(0, device="cuda"))
        assert h.total() == allk.size
        counts = torch.empty(1 << p, dtype=torch.uint64, device="cuda")
        fs.fsort_hist_counts(h.handle, counts)
        torch.cuda.synchronize()
        assert np.array_equal(counts.cpu().numpy(), leaf_counts(tree, p))
        rng = np.random.default_rng(p)
        vals = np.concatenate([[0, 1, (1 << p) - 1, 1 << p, (1 << p) + 7], rng.integers(0, 1 << p, 500)])
        ranks = np.concatenate([[0, 1, allk.size - 1, allk.size, allk.size + 9], rng.integers(0, allk.size, 500)])
        rv = torch.empty(vals.size, dtype=torch.uint64, device="cuda")
        sv = torch.empty(ranks.size, dtype=torch.uint64, device="cuda")
        fs.fsort_hist_rank(h.handle, torch.from_numpy(vals.astype(np.uint64)).cuda(), rv)
        fs.fsort_hist_select(h.handle, torch.from_numpy(ranks.astype(np.uint64)).cuda(), sv)
        out = torch.empty(allk.size, dtype={16: torch.uint16, 32: torch.uint32, 64: torch.uint64}[kb], device="cuda")
        fs.fsort_hist_expand(h.handle, out)
        torch.cuda.synchronize()
    want_rank = [oracle.tree_rank(tree, p, int(v)) if v < (1 << p) else allk.size for v in vals]
    want_sel = [oracle.tree_select(tree, p, int(r)) for r in ranks]
    assert rv.cpu().numpy().tolist() == want_rank
    assert sv.cpu().numpy().tolist() == want_sel
    assert np.array_equal(out.cpu().numpy(), oracle.expand(leaf_counts(tree, p), kb))
    if p == kb:  # full precision: the expansion is the sorted stream itself
        assert np.array_equal(out.cpu().numpy(), oracle.sort(allk, None, kb, kb)[0])


def test_batches_equal_one_shot_and_reset():
    kb, p = 32, 24
    bs = batches(kb, seed=3)
    one = np.concatenate(bs)
    with fs.StreamHistogram(kb, p) as a, fs.StreamHistogram(kb, p) as b:
        for x in bs:
            if x.size:
                a.accumulate(torch.from_numpy(x).cuda())
        b.accumulate(torch.from_numpy(one).cuda())
        ca = torch.empty(1 << p, dtype=torch.uint64, device="cuda")
        cb = torch.empty_like(ca)
        fs.fsort_hist_counts(a.handle, ca)
        fs.fsort_hist_counts(b.handle, cb)
        torch.cuda.synchronize()
        assert torch.equal(ca, cb) and a.total() == b.total() == one.size
        fs.fsort_hist_reset(a.handle)
        assert a.total() == 0
        a.accumulate(torch.from_numpy(bs[2]).cuda())
        r = torch.empty(1, dtype=torch.uint64, device="cuda")
        fs.fsort_hist_rank(a.handle, torch.tensor([1 << p], dtype=torch.uint64, device="cuda"), r)
        torch.cuda.synchronize()
        assert int(r.item()) == bs[2].size
        with pytest.raises(fs.FsortError):  # n must equal the total
            fs.fsort_hist_expand(a.handle, torch.empty(5, dtype=torch.uint32, device="cuda"))
    with pytest.raises(fs.FsortError):
        fs.StreamHistogram(32, 25)  # more than 2^24 counters


def test_skewed_stream_all_equal_keys():
    kb, p = 64, 20
    x = np.full(3_000_000, 0xFEDCBA9876543210, np.uint64)
    with fs.StreamHistogram(kb, p) as h:
        for _ in range(3):
            h.accumulate(torch.from_numpy(x).cuda())
        out = torch.empty(3 * x.size, dtype=torch.uint64, device="cuda")
        fs.fsort_hist_expand(h.handle, out)
        torch.cuda.synchronize()
    assert torch.all(out == (0xFEDCBA9876543210 >> (64 - p)))


def test_misaligned_arrays_are_refused():
    """Arrays off their element alignment are refused on the host (status 1)."""
    k = torch.zeros(64, dtype=torch.uint32, device="cuda")
    v = torch.zeros(64, dtype=torch.int64, device="cuda")
    with fs.StreamHistogram(32, 12) as h:
        fs.fsort_hist_accumulate(h.handle, k, n=10)
        bad = [
            lambda: fs.fsort_hist_accumulate(h.handle, k.data_ptr() + 2, n=10),
            lambda: fs.fsort_hist_counts(h.handle, v.data_ptr() + 4),
            lambda: fs.fsort_hist_rank(h.handle, v.data_ptr() + 4, v, count=4),
            lambda: fs.fsort_hist_select(h.handle, v, v.data_ptr() + 4, count=4),
            lambda: fs.fsort_hist_expand(h.handle, k.data_ptr() + 2, n=10),
        ]
        for f in bad:
            with pytest.raises(fs.FsortError) as e:
                f()
            assert e.value.status == 1
        assert fs.fsort_hist_total(h.handle) == 10
