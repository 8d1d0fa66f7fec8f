"""Slab mode of the CPU oracle: checking sorts too large for host memory.

TEST INFRASTRUCTURE ONLY (like the rest of this package): used by ``tests/``
to check full-size GPU sorts against the oracle without holding the whole input
or output on the host.  It imports neither the product nor the workload
generators; the caller passes a function that regenerates any chunk of the
input.

Why a slab can be checked on its own.  The sort (Sec. II's histogram, prefix
sum and stable scatter, read with R2: order by the top p bits s(k) =
k >> (kb - p); and R3: ties keep input order) outputs the unique permutation
ordered by (s(k), input index).  Take a slab key t(k) = k >> (kb - b) with
b <= p, so t is a prefix of s and t(a) < t(c) implies s(a) < s(c).  Then the
keys with lo <= t(k) < hi occupy one contiguous output range starting at
#{k : t(k) < lo}, and inside it they appear in (s(k), input index) order --
which is the oracle's stable sort of just those keys, taken in input order.
So each slab is checked element by element by sorting only the slab.
"""
from __future__ import annotations

import concurrent.futures
from typing import Callable, Sequence

import numpy as np

from . import sort as oracle_sort

_KEY_DTYPES = {16: np.uint16, 32: np.uint32, 64: np.uint64}


def slab_key(keys: np.ndarray, key_bits: int, slab_bits: int) -> np.ndarray:
    """t(k) = k >> (key_bits - slab_bits), as uint64."""
    return keys.astype(np.uint64, copy=False) >> np.uint64(key_bits - slab_bits)


def slab_gather(chunk_fn: Callable[[int], np.ndarray], nchunks: int, key_bits: int, slab_bits: int,
                ranges: Sequence[tuple], workers: int = 8):
    """One ordered pass over the input, regenerated chunk by chunk.

    chunk_fn(c) returns chunk c of the input (chunks in input order).  ranges
    holds (lo, hi) pairs of slab-key values; hi = None means no upper bound.
    Returns, per range, (first, keys): first = #{k : t(k) < lo} (the slab's
    first output position) and the slab's keys in input order.  Chunks are
    produced and filtered by `workers` threads; results are combined in chunk
    order, so the keys stay in input order.
    """
    def work(c):
        k = chunk_fn(c)
        t = slab_key(k, key_bits, slab_bits)
        below, parts = [], []
        for lo, hi in ranges:
            lo64 = np.uint64(lo)
            below.append(int(np.count_nonzero(t < lo64)))
            sel = t >= lo64 if hi is None else (t >= lo64) & (t < np.uint64(hi))
            parts.append(k[sel])
        return below, parts

    first = [0] * len(ranges)
    collected = [[] for _ in ranges]
    with concurrent.futures.ThreadPoolExecutor(max_workers=workers) as ex:
        for below, parts in ex.map(work, range(nchunks)):
            for r in range(len(ranges)):
                first[r] += below[r]
                if parts[r].size:
                    collected[r].append(parts[r])
    dtype = _KEY_DTYPES[key_bits]
    out = []
    for r in range(len(ranges)):
        keys = np.concatenate(collected[r]) if collected[r] else np.empty(0, dtype=dtype)
        collected[r] = None
        out.append((first[r], keys))
    return out


def slab_expected(slab_keys: np.ndarray, key_bits: int, precision_bits: int) -> np.ndarray:
    """The output the sort must hold over a slab's range: the oracle's stable
    sort of the slab's keys (in input order) on the top precision_bits bits."""
    return oracle_sort(slab_keys, None, key_bits, precision_bits)[0]
