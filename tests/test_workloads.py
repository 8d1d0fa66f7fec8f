"""The shared input generators against the published SplitMix64 definition."""
import numpy as np
import pytest

import workloads as wl


def test_splitmix64_published_sequence():
    # SplitMix64 seeded with 0 (Steele, Lea & Flood 2014; Vigna's reference code)
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [wl.raw(0, i) for i in range(3)] == want
    assert [wl.py_raw(0, i) for i in range(3)] == want


@pytest.mark.parametrize("key_bits", [16, 32, 64])
def test_uniform_matches_python_statement(key_bits):
    n = 257
    k = wl.generate("uniform", n, key_bits, seed=3, stream=2, start=1000)
    base = wl.stream_base(3, 2, 0)
    want = [wl.py_raw(base, 1000 + i) >> (64 - key_bits) for i in range(n)]
    assert k.tolist() == want


@pytest.mark.parametrize("name", ["zipf1.1", "gauss"])
def test_table_lookup_matches_searchsorted(name):
    n = 2000
    k = wl.generate(name, n, 16, seed=0, stream=1)
    base = wl.stream_base(0, 1, 0)
    u = np.array([wl.py_raw(base, i) for i in range(n)], dtype=np.uint64)
    want = np.searchsorted(wl.table_for(name, 16), u, side="right")
    assert np.array_equal(k.astype(np.int64), want)


def test_slices_are_consistent():
    full = wl.generate("presorted", 5000, 32, seed=1, stream=3)
    part = wl.generate("presorted", 1000, 32, seed=1, stream=3, start=2000, n_total=5000)
    assert np.array_equal(full[2000:3000], part)


def test_distribution_shapes():
    n = 1 << 18
    z = wl.generate("zipf1.1", n, 16)
    p0 = np.mean(z == 0)
    pmf = wl.zipf_pmf(1.1)
    assert abs(p0 - pmf[0] / pmf.sum()) < 0.01          # about 13.7 % on key 0
    g = wl.generate("gauss", n, 16).astype(np.float64)
    assert abs(g.mean() - 32768) < 20 and abs(g.std() - 1024) < 20
    e = wl.generate("equal", 100, 16)
    assert (e == 0xA5A5).all()
    s = wl.generate("presorted", n, 16).astype(np.int64)
    frac_up = np.mean(np.diff(s) >= 0)
    assert frac_up > 0.8
    u = wl.generate("uniform", n, 16)
    assert abs(u.astype(np.float64).mean() - 32767.5) < 300
