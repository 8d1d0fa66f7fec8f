"""Pins for the CPU oracle, independent of the oracle itself.

Each test checks the oracle against something other than its own code: a
hand-worked example (tests/golden), a library routine (Python's stable
``sorted``, numpy's stable argsort, bincount, cumsum, repeat), brute force on
tiny inputs, or an invariant of the definition.  ``test_planted_mutants``
plants plausible mistakes in copies of the oracle source and shows that these
pins catch every one of them.
"""
import ctypes
import itertools
import os
import subprocess

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_example.txt")
KEY_DT = {16: np.uint16, 32: np.uint32, 64: np.uint64}


def _golden():
    out = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, *rest = line.split()
        out[name] = rest
    return out


def _ref_order(keys, key_bits, p):
    """Library routine: numpy's stable argsort on the top-p-bit sort key."""
    s = keys.astype(np.uint64) >> np.uint64(key_bits - p)
    return np.argsort(s, kind="stable")


def _rand_keys(rng, n, key_bits, top_values=None):
    if key_bits == 64:
        k = rng.integers(0, 2 ** 63, size=n, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, size=n,
                                                                                                dtype=np.uint64)
    else:
        k = rng.integers(0, 2 ** key_bits, size=n, dtype=np.uint64)
    if top_values is not None:  # force duplicates in the top bits
        k = (k & np.uint64((1 << (key_bits - 4)) - 1)) | (
            rng.integers(0, top_values, size=n, dtype=np.uint64) << np.uint64(key_bits - 4))
    return k.astype(KEY_DT[key_bits])


# ---- the paper's definition, worked by hand ---------------------------------

def test_golden_worked_example():
    g = _golden()
    keys = np.array([int(x, 16) for x in g["keys"]], dtype=np.uint16)
    idx = np.arange(keys.size, dtype=np.uint32)
    ko, vo = oracle.sort(keys, idx, 16, 16)
    assert vo.tolist() == [int(x) for x in g["p16_idx"]]
    assert ko.tolist() == [int(x, 16) for x in g["p16_keys"]]
    ko, vo = oracle.sort(keys, idx, 16, 8)
    assert vo.tolist() == [int(x) for x in g["p8_idx"]]
    assert ko.tolist() == [int(x, 16) for x in g["p8_keys"]]
    h = oracle.digit_histograms(keys, 16, 16, 8)
    for j, name in enumerate(["p16_hist_pass0", "p16_hist_pass1"]):
        want = np.zeros(256, dtype=np.uint64)
        for item in g[name]:
            d, c = item.split(":")
            want[int(d, 16)] = int(c)
        assert np.array_equal(h[j], want)
    tree = oracle.tree_build(keys, 16, 8)
    for item in g["p8_rank"]:
        v, r = item.split(":")
        assert oracle.tree_rank(tree, 8, int(v, 16)) == int(r)
    for item in g["p8_select"]:
        r, v = item.split(":")
        assert oracle.tree_select(tree, 8, int(r)) == int(v, 16)


# ---- brute force on tiny inputs ---------------------------------------------

@pytest.mark.parametrize("key_bits,p,alphabet", [
    (16, 16, [0x0000, 0x00FF, 0xFF00, 0x0100]),
    (16, 8, [0x0001, 0x0000, 0x0100, 0x01FF]),       # equal top byte, different low byte
    (32, 9, [0x00000000, 0x00800000, 0x00FFFFFF, 0xFF800000]),
    (64, 1, [0, 1, 1 << 63, (1 << 64) - 1]),
])
def test_exhaustive_tiny(key_bits, p, alphabet):
    """Every input of length <= 6 over a 4-key alphabet vs Python's stable sorted()."""
    dt = KEY_DT[key_bits]
    for n in range(0, 7):
        for combo in itertools.product(range(4), repeat=n):
            keys = np.array([alphabet[c] for c in combo], dtype=dt)
            idx = np.arange(n, dtype=np.uint32)
            ko, vo = oracle.sort(keys, idx, key_bits, p)
            want = sorted(range(n), key=lambda i: (int(keys[i]) >> (key_bits - p), i))
            assert vo.tolist() == want
            assert ko.tolist() == [int(keys[i]) for i in want]


@pytest.mark.parametrize("key_bits", [16, 32, 64])
@pytest.mark.parametrize("n", [0, 1, 2, 255, 1000, 4097])
def test_random_vs_numpy_stable_argsort(key_bits, n):
    rng = np.random.default_rng(1234 + n + key_bits)
    for p in sorted({1, 7, 8, 9, 15, 16, key_bits - 1, key_bits}):
        for dup in (None, 3):
            keys = _rand_keys(rng, n, key_bits, dup)
            idx = np.arange(n, dtype=np.uint32)
            ko, vo = oracle.sort(keys, idx, key_bits, p)
            order = _ref_order(keys, key_bits, p)
            assert np.array_equal(vo, order.astype(np.uint32)), (p, dup)
            assert np.array_equal(ko, keys[order])
            ko2, vo2 = oracle.sort(keys, None, key_bits, p)
            assert vo2 is None and np.array_equal(ko2, keys[order])


def test_special_cases():
    n = 5000
    idx = np.arange(n, dtype=np.uint32)
    eq = np.full(n, 0xA5A5, dtype=np.uint16)
    ko, vo = oracle.sort(eq, idx, 16, 16)
    assert np.array_equal(vo, idx) and np.array_equal(ko, eq)          # all-equal: identity
    asc = np.sort(np.random.default_rng(0).integers(0, 65536, n).astype(np.uint16))
    ko, vo = oracle.sort(asc, idx, 16, 16)
    assert np.array_equal(vo, idx)                                      # presorted: identity
    desc = np.arange(n, dtype=np.uint16)[::-1].copy()
    ko, vo = oracle.sort(desc, idx, 16, 16)
    assert np.array_equal(vo, idx[::-1])                                # distinct descending: reversal


def test_invalid_args():
    k = np.zeros(4, dtype=np.uint16)
    with pytest.raises(ValueError):
        oracle.sort(k, None, 16, 0)
    with pytest.raises(ValueError):
        oracle.sort(k, None, 16, 17)


# ---- one pass, histograms, scan ----------------------------------------------

@pytest.mark.parametrize("key_bits,shift,width", [(16, 0, 8), (16, 8, 8), (32, 5, 11), (64, 56, 8), (64, 0, 16)])
def test_scatter_pass_vs_numpy(key_bits, shift, width):
    rng = np.random.default_rng(shift * 100 + width)
    keys = _rand_keys(rng, 3001, key_bits, 5)
    vals = rng.integers(0, 2 ** 32, size=3001, dtype=np.uint64).astype(np.uint32)
    ko, vo = oracle.scatter_pass(keys, vals, key_bits, shift, width)
    d = (keys.astype(np.uint64) >> np.uint64(shift)) & np.uint64((1 << width) - 1)
    order = np.argsort(d, kind="stable")
    assert np.array_equal(ko, keys[order]) and np.array_equal(vo, vals[order])


@pytest.mark.parametrize("key_bits,p,d", [(16, 16, 8), (16, 13, 8), (32, 32, 11), (64, 64, 8), (16, 16, 16),
                                          (64, 20, 8)])
def test_digit_histograms_vs_bincount(key_bits, p, d):
    rng = np.random.default_rng(p * d)
    keys = _rand_keys(rng, 7777, key_bits, 2)
    h = oracle.digit_histograms(keys, key_bits, p, d)
    s = keys.astype(np.uint64) >> np.uint64(key_bits - p)
    assert h.shape == (-(-p // d), 1 << d)
    for j in range(h.shape[0]):
        width = min(d, p - j * d)
        dig = (s >> np.uint64(j * d)) & np.uint64((1 << width) - 1)
        want = np.bincount(dig.astype(np.int64), minlength=1 << d).astype(np.uint64)
        assert np.array_equal(h[j], want)
        assert int(h[j].sum()) == keys.size


def test_exclusive_scan_vs_cumsum():
    rng = np.random.default_rng(7)
    c = rng.integers(0, 1000, size=65536, dtype=np.uint64)
    b = oracle.exclusive_scan(c)
    want = np.concatenate([[0], np.cumsum(c)[:-1]]).astype(np.uint64)
    assert np.array_equal(b, want)


# ---- histogram tree: rank / select / count ----------------------------------

@pytest.mark.parametrize("p", [1, 4, 8, 12])
def test_tree_rank_select_bruteforce(p):
    rng = np.random.default_rng(p)
    keys = _rand_keys(rng, 999, 16, 3)
    tree = oracle.tree_build(keys, 16, p)
    s = (keys.astype(np.int64) >> (16 - p))
    for l in range(p + 1):
        for x in range(1 << l):
            assert oracle.tree_count(tree, p, l, x) == int(np.sum((s >> (p - l)) == x))
    for v in range(1 << p):
        assert oracle.tree_rank(tree, p, v) == int(np.sum(s < v))
    srt = np.sort(s)
    for r in range(keys.size):
        assert oracle.tree_select(tree, p, r) == int(srt[r])
    assert oracle.tree_select(tree, p, keys.size) == (1 << 64) - 1


def test_tree_rank_is_exclusive_scan_of_leaves():
    rng = np.random.default_rng(3)
    keys = rng.integers(0, 65536, 20000).astype(np.uint16)
    tree = oracle.tree_build(keys, 16, 10)
    leaves = tree[(1 << 10) - 1:]
    b = oracle.exclusive_scan(leaves)
    for v in range(0, 1 << 10, 37):
        assert oracle.tree_rank(tree, 10, v) == int(b[v])


def test_tree_levels_sum_to_n_and_uniform_expectation():
    """Every level counts all n keys; on uniform keys a level-l node holds
    about n / 2^l of them (Sec. III-B-1)."""
    n, p = 1 << 16, 16
    keys = np.random.default_rng(11).integers(0, 65536, n).astype(np.uint16)
    tree = oracle.tree_build(keys, 16, p)
    for l in range(p + 1):
        level = tree[(1 << l) - 1:(1 << (l + 1)) - 1]
        assert int(level.sum()) == n
        if l <= 6:
            exp = n / (1 << l)
            assert np.all(np.abs(level.astype(np.float64) - exp) < 6 * np.sqrt(exp) + 1)


# ---- expand (Alg. 5, no trailing bits) ----------------------------------------

def test_expand_vs_repeat():
    rng = np.random.default_rng(5)
    c = rng.integers(0, 5, size=65536, dtype=np.uint64)
    k = oracle.expand(c, 16)
    assert np.array_equal(k, np.repeat(np.arange(65536, dtype=np.uint16), c.astype(np.int64)))
    keys = rng.integers(0, 65536, 10000).astype(np.uint16)
    h = oracle.digit_histograms(keys, 16, 16, 16)[0]
    assert np.array_equal(oracle.expand(h, 16), np.sort(keys))


# ---- invariant checkers catch corrupted outputs -------------------------------

def test_checkers_catch_corruption():
    rng = np.random.default_rng(9)
    keys = rng.integers(0, 64, 2000).astype(np.uint16)
    idx = np.arange(keys.size, dtype=np.uint32)
    ko, vo = oracle.sort(keys, idx, 16, 16)
    oracle.check_sorted_stable(keys, ko, vo, 16, 16)
    oracle.check_sorted_multiset(keys, ko, 16, 16)
    eq = np.nonzero(ko[:-1] == ko[1:])[0][0]
    bad = vo.copy(); bad[eq], bad[eq + 1] = bad[eq + 1], bad[eq]           # stability
    badk = ko.copy()
    with pytest.raises(AssertionError):
        oracle.check_sorted_stable(keys, badk, bad, 16, 16)
    ne = np.nonzero(ko[:-1] != ko[1:])[0][0]
    bad = vo.copy(); bad[ne], bad[ne + 1] = bad[ne + 1], bad[ne]           # order
    badk = ko.copy(); badk[ne], badk[ne + 1] = badk[ne + 1], badk[ne]
    with pytest.raises(AssertionError):
        oracle.check_sorted_stable(keys, badk, bad, 16, 16)
    with pytest.raises(AssertionError):
        oracle.check_sorted_multiset(keys, badk, 16, 16)
    bad = vo.copy(); bad[5] = bad[6]                                        # not a permutation
    with pytest.raises(AssertionError):
        oracle.check_sorted_stable(keys, ko, bad, 16, 16)
    badk = ko.copy(); badk[-1] ^= 1                                         # key changed
    with pytest.raises(AssertionError):
        oracle.check_sorted_stable(keys, badk, vo, 16, 16)


# ---- planted mistakes in the oracle are caught by the pins --------------------

_MUTANTS = {
    "inclusive_scan": ("out[v] = running;\n    running += c;", "running += c;\n    out[v] = running;"),
    "digit_base_dropped": ("base + lo, width", "lo, width"),
    "one_pass_short": ("for (int j = 0; j < passes; ++j) {\n    const int lo", "for (int j = 1; j < passes; ++j) {\n    const int lo"),
    "unstable_reverse": ("for (uint64_t i = 0; i < n; ++i) {\n    const uint64_t k = get_key(keys_in, key_bits, i);",
                         "for (uint64_t i = n; i-- > 0;) {\n    const uint64_t k = get_key(keys_in, key_bits, i);"),
    "select_off_by_one": ("if (r < left) {", "if (r <= left) {"),
    "rank_wrong_child": ("if (bit) idx += tree[level_base(l + 1) + (prefix << 1)];",
                         "if (bit) idx += tree[level_base(l + 1) + (prefix << 1) + 1];"),
    "sort_key_shift": ("return k >> (key_bits - p);", "return k >> (key_bits - p + 1);"),
    # the step functions on their own (histograms, one pass, expand, tree build)
    "hist_one_row_for_all_passes": ("counts[(uint64_t)j * bins + digit_of(s, precision_bits, digit_bits, j)] += 1",
                                    "counts[digit_of(s, precision_bits, digit_bits, j)] += 1"),
    "hist_raw_key": ("const uint64_t s = sort_key(get_key(keys, key_bits, i), key_bits, precision_bits);\n    for (int j",
                     "const uint64_t s = get_key(keys, key_bits, i);\n    for (int j"),
    "hist_digit_low_bit": ("return (s >> lo) & mask;", "return (s >> (lo + 1)) & mask;"),
    "pass_mask_off_by_one": ("const uint64_t bins = 1ULL << width, mask = bins - 1;",
                             "const uint64_t bins = 1ULL << width, mask = (bins >> 1) - 1;"),
    "expand_drops_last_bin": ("for (uint64_t b = 0; b < bins; ++b)\n", "for (uint64_t b = 0; b + 1 < bins; ++b)\n"),
    "tree_build_skips_root": ("for (int l = 0; l <= p; ++l) tree", "for (int l = 1; l <= p; ++l) tree"),
    "tree_build_skips_leaves": ("for (int l = 0; l <= p; ++l) tree", "for (int l = 0; l < p; ++l) tree"),
}


def _bind(so_path):
    lib = ctypes.CDLL(str(so_path))
    vp, u64, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int
    lib.oracle_sort.argtypes = [vp, vp, vp, vp, u64, i32, i32]
    lib.oracle_scatter_pass.argtypes = [vp, vp, vp, vp, u64, i32, i32, i32]
    lib.oracle_digit_histograms.argtypes = [vp, u64, i32, i32, i32, vp]
    lib.oracle_exclusive_scan.argtypes = [vp, u64, vp]
    lib.oracle_exclusive_scan.restype = None
    lib.oracle_expand.argtypes = [vp, u64, i32, vp]
    lib.oracle_tree_build.argtypes = [vp, u64, i32, i32, vp]
    lib.oracle_tree_rank.argtypes = [vp, i32, u64]
    lib.oracle_tree_rank.restype = u64
    lib.oracle_tree_select.argtypes = [vp, i32, u64]
    lib.oracle_tree_select.restype = u64
    return lib


def _mutant_lib(tmp_path, name):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    old, new = _MUTANTS[name]
    assert src.count(old) == 1, name
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new, 1))
    so = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-o", str(so), str(path)])
    return _bind(so)


def _pins_pass(lib):
    """The pins above (worked example, stable argsort, bincount, cumsum,
    repeat, brute-force rank and select), run against a given library."""
    g = _golden()
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    keys = np.array([int(x, 16) for x in g["keys"]], dtype=np.uint16)
    cases = [(keys, 16, 16), (keys, 16, 8)]
    rng = np.random.default_rng(0)
    cases += [(_rand_keys(rng, 500, 32, 3), 32, 12), (_rand_keys(rng, 500, 64, 2), 64, 64)]
    for k, kb, pb in cases:
        idx = np.arange(k.size, dtype=np.uint32)
        ko, vo = np.zeros_like(k), np.zeros_like(idx)
        if lib.oracle_sort(p(k), p(idx), p(ko), p(vo), k.size, kb, pb) != 0:
            return False
        order = _ref_order(k, kb, pb)
        if not np.array_equal(vo, order.astype(np.uint32)):
            return False
    # histograms against bincount, for a precision below the key width and two digit widths
    for kb, pb, d in [(16, 13, 8), (32, 20, 11)]:
        k = _rand_keys(rng, 3000, kb, 2)
        passes = -(-pb // d)
        h = np.zeros((passes, 1 << d), dtype=np.uint64)
        if lib.oracle_digit_histograms(p(k), k.size, kb, pb, d, p(h)) != 0:
            return False
        s = k.astype(np.uint64) >> np.uint64(kb - pb)
        for j in range(passes):
            dig = (s >> np.uint64(j * d)) & np.uint64((1 << min(d, pb - j * d)) - 1)
            if not np.array_equal(h[j], np.bincount(dig.astype(np.int64), minlength=1 << d).astype(np.uint64)):
                return False
    # scan against cumsum
    c = rng.integers(0, 1000, size=4096, dtype=np.uint64)
    b = np.zeros_like(c)
    lib.oracle_exclusive_scan(p(c), c.size, p(b))
    if not np.array_equal(b, np.concatenate([[0], np.cumsum(c)[:-1]]).astype(np.uint64)):
        return False
    # one pass against numpy's stable argsort on the digit
    k = _rand_keys(rng, 3000, 32, 5)
    v = rng.integers(0, 2 ** 32, size=3000, dtype=np.uint64).astype(np.uint32)
    ko, vo = np.zeros_like(k), np.zeros_like(v)
    if lib.oracle_scatter_pass(p(k), p(v), p(ko), p(vo), k.size, 32, 5, 11) != 0:
        return False
    order = np.argsort((k.astype(np.uint64) >> np.uint64(5)) & np.uint64(2047), kind="stable")
    if not (np.array_equal(ko, k[order]) and np.array_equal(vo, v[order])):
        return False
    # expand against repeat (the last bin non-empty)
    c = rng.integers(0, 4, size=65536, dtype=np.uint64)
    c[-1] = 2
    out = np.zeros(int(c.sum()), dtype=np.uint16)  # not np.empty: unwritten tail must not hold the answer
    if lib.oracle_expand(p(c), c.size, 16, p(out)) != 0:
        return False
    if not np.array_equal(out, np.repeat(np.arange(65536, dtype=np.uint16), c.astype(np.int64))):
        return False
    # tree rank and select against brute force
    k = _rand_keys(rng, 300, 16, 3)
    tree = np.zeros((1 << 9) - 1, dtype=np.uint64)
    lib.oracle_tree_build(p(k), k.size, 16, 8, p(tree))
    s = k.astype(np.int64) >> 8
    for val in range(256):
        if lib.oracle_tree_rank(p(tree), 8, val) != int(np.sum(s < val)):
            return False
    srt = np.sort(s)
    for r in range(k.size):
        if lib.oracle_tree_select(p(tree), 8, r) != int(srt[r]):
            return False
    return True


def test_pins_accept_unmutated_oracle(tmp_path):
    src = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")
    so = tmp_path / "clean.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-o", str(so), src])
    assert _pins_pass(_bind(so))


@pytest.mark.parametrize("name", sorted(_MUTANTS))
def test_planted_mutants(tmp_path, name):
    assert not _pins_pass(_mutant_lib(tmp_path, name)), f"mutant {name} survived the pins"
