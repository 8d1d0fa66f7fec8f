"""Pins for the oracle's slab mode (oracle/slab.py), CPU only.

Slab mode checks a sort range by range: the keys whose slab key
t(k) = k >> (kb - b) lies in [lo, hi) must sit, in the oracle's stable order,
at output positions #{t < lo} onwards.  These tests pin that decomposition
against a library routine (numpy's stable argsort on the top-p-bit sort key
of the whole input), on inputs small enough to sort whole, with ranges that
include the first and last slab and the most frequent key's slab.
"""
import numpy as np
import pytest

import oracle
from oracle import slab

KEY_DT = {16: np.uint16, 32: np.uint32, 64: np.uint64}


def _whole_sorted(keys, kb, p):
    s = keys.astype(np.uint64) >> np.uint64(kb - p)
    return keys[np.argsort(s, kind="stable")]


@pytest.mark.parametrize("kb,b,p", [(64, 16, 16), (64, 16, 32), (64, 16, 64), (32, 8, 20), (16, 4, 16), (64, 64, 64)])
def test_slabs_equal_the_whole_sort_restricted(kb, b, p):
    rng = np.random.default_rng(kb * 100 + b + p)
    n = 50_000
    keys = rng.integers(0, 1 << kb, n, dtype=np.uint64).astype(KEY_DT[kb])
    keys[rng.integers(0, n, n // 5)] = keys[7]  # one heavy key, plus equal top bits for many others
    keys[: n // 10] &= KEY_DT[kb]((1 << (kb - 2)) - 1)  # a low-valued block
    t = slab.slab_key(keys, kb, b)
    heavy = int(slab.slab_key(keys[7:8], kb, b)[0])
    top = (1 << b) - 1 if b < 64 else int(t.max())
    ranges = [(0, max(1, top // 50)), (heavy, heavy + 1), (max(0, top - top // 50), None), (top // 3, top // 3 + top // 40)]
    chunks = 7
    bounds = np.linspace(0, n, chunks + 1).astype(int)
    got = slab.slab_gather(lambda c: keys[bounds[c]:bounds[c + 1]], chunks, kb, b, ranges, workers=3)
    whole = _whole_sorted(keys, kb, p)
    for (lo, hi), (first, sk) in zip(ranges, got):
        sel = (t >= np.uint64(lo)) if hi is None else (t >= np.uint64(lo)) & (t < np.uint64(hi))
        assert first == int(np.count_nonzero(t < np.uint64(lo)))
        assert np.array_equal(sk, keys[sel])  # the slab's keys, in input order
        exp = slab.slab_expected(sk, kb, p)
        assert np.array_equal(exp, whole[first:first + sk.size]), (lo, hi)


def test_a_slab_key_finer_than_the_precision_is_refused_by_the_argument():
    # b > p breaks the contiguity the decomposition needs: the slab of t in [lo, hi)
    # is then not one output range.  Shown on a case where it visibly fails.
    keys = np.array([0x12, 0x11, 0x21, 0x13], dtype=np.uint16) << np.uint16(8)
    whole = _whole_sorted(keys, 16, 4)  # orders by the top 4 bits only
    (first, sk), = slab.slab_gather(lambda c: keys, 1, 16, 8, [(0x12, 0x13)], workers=1)
    assert first == 1 and sk.tolist() == [0x1200]
    assert whole[first] != 0x1200  # position 1 holds 0x1100: top-8 slabs are not contiguous at p = 4


def test_empty_slab():
    keys = np.arange(100, dtype=np.uint32)
    (first, sk), = slab.slab_gather(lambda c: keys, 1, 32, 32, [(1000, 2000)], workers=1)
    assert first == 100 and sk.size == 0
    assert slab.slab_expected(sk, 32, 32).size == 0
