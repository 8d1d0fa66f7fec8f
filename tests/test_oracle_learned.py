"""Pins of the learned-mapping oracle (oracle/learned.py) against facts fixed
outside it: a library routine (torch's BF16 cast), closed forms of degenerate
networks, central finite differences of the loss, brute-force enumeration of
the key grid, and hand-computed maps.  A dropped term, a transposed weight
matrix, a wrong sign or an off-by-one cell fails one of these.
"""
import math

import numpy as np
import pytest

from oracle import learned as ol

torch = pytest.importorskip("torch")


def rand_params(seed, scale=0.5):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, scale, ol.PARAMS)


def test_bf16_round_matches_library_cast():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(0, 3, 20000), rng.uniform(-1e-3, 1e-3, 2000)]).astype(np.float32)
    # exact ties: low 16 bits 0x8000, both parities of bit 16
    ties = (np.arange(64, dtype=np.uint32) << 16 | 0x3F800000 | 0x8000).view(np.float32)
    x = np.concatenate([x, ties, -ties])
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(ol.bf16_round(x), want)


def single_path(a, c, d, g, e, f):
    """Parameters of a network with one path: W1[0], b1[0], W2[0][0], b2[0], W3[0], b3."""
    p = np.zeros(ol.PARAMS)
    p[0], p[64], p[128], p[128 + 4096], p[128 + 4096 + 64], p[-1] = a, c, d, g, e, f
    return p


def single_path_value(x, a, c, d, g, e, f):
    return 1.0 / (1.0 + math.exp(-(e * max(0.0, d * max(0.0, a * x + c) + g) + f)))


@pytest.mark.parametrize("d,g", [(0.9, 0.2), (-0.9, 0.2), (0.9, -0.5)])
def test_forward_single_path_closed_form(d, g):
    # d < 0 or g < 0 drives layer 2 below zero for some x: its ReLU must clip there
    a, c, e, f = 1.7, -0.3, 2.5, -0.4
    xs = np.linspace(-2, 2, 41)
    want = [single_path_value(x, a, c, d, g, e, f) for x in xs]
    assert np.allclose(ol.forward(single_path(a, c, d, g, e, f), xs), want, rtol=0, atol=1e-15)


@pytest.mark.parametrize("d,g", [(0.9, 0.2), (-0.9, 0.2), (0.9, -0.5)])
def test_loss_single_path_closed_form(d, g):
    a, c, e, f = 1.7, -0.3, 2.5, -0.4
    x = np.array([-1.5, -0.2, 0.1, 0.4, 0.9, 1.6])
    y = np.array([0.1, 0.3, 0.5, 0.7, 0.2, 0.9])
    want = 0.5 * np.mean([(single_path_value(xi, a, c, d, g, e, f) - yi) ** 2 for xi, yi in zip(x, y)])
    loss, _ = ol.loss_and_grad(single_path(a, c, d, g, e, f), x, y)
    assert loss == pytest.approx(want, rel=1e-13)


def test_forward_uses_row_j_of_w2_for_unit_j():
    # unit 1 of layer 1 feeds unit 2 of layer 2 through W2[2][1] only
    p = np.zeros(ol.PARAMS)
    p[1], p[64 + 1] = 1.0, 0.0           # h1_1 = relu(x)
    p[128 + 2 * 64 + 1] = 3.0            # W2[2][1]
    p[128 + 4096 + 64 + 2] = 1.0         # W3[2]
    x = np.array([0.5, -0.5])
    assert np.allclose(ol.forward(p, x), [1 / (1 + math.exp(-1.5)), 0.5])
    p[128 + 2 * 64 + 1], p[128 + 1 * 64 + 2] = 0.0, 3.0  # the transpose position: no path
    assert np.allclose(ol.forward(p, x), [0.5, 0.5])


def test_grad_zero_network_closed_form():
    p = np.zeros(ol.PARAMS)
    p[-1] = 0.3
    x = np.array([0.1, -0.7, 1.2])
    y = np.array([0.2, 0.9, 0.5])
    s = 1 / (1 + math.exp(-0.3))
    loss, g = ol.loss_and_grad(p, x, y)
    assert loss == pytest.approx(0.5 * np.mean((s - y) ** 2), rel=1e-14)
    assert g[-1] == pytest.approx(np.mean(s - y) * s * (1 - s), rel=1e-14)
    assert np.all(g[:-1] == 0)


@pytest.mark.parametrize("seed", [1, 2])
def test_grad_matches_central_differences(seed):
    p = rand_params(seed)
    rng = np.random.default_rng(100 + seed)
    x = rng.uniform(-1.2, 1.2, 9)
    y = rng.uniform(0, 1, 9)
    _, g = ol.loss_and_grad(p, x, y)
    idx = list(range(0, 128)) + list(range(128 + 4096, ol.PARAMS)) + list(rng.choice(np.arange(128, 4224), 300))
    h = 1e-6
    for i in idx:
        q = p.copy()
        q[i] += h
        lp, _ = ol.loss_and_grad(q, x, y)
        q[i] -= 2 * h
        lm, _ = ol.loss_and_grad(q, x, y)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(g[i])), (i, fd, g[i])


def test_cell_grid_brute_force():
    keys = [0, 1, 2, 1023, 1024, 2047, 2048, 2049, 4095, 4096, (1 << 64) - 1, (1 << 63), (1 << 63) - 1]
    keys += list(range(0, 5000, 7))
    for e in range(11, 64):
        keys += [(1 << e) - 1, 1 << e, (1 << e) + 1, (1 << e) + (1 << (e - 10)) - 1, (1 << e) + (1 << (e - 10))]
    rng = np.random.default_rng(3)
    keys += [int(v) for v in rng.integers(0, 1 << 63, 2000, dtype=np.uint64)]
    keys = sorted(set(keys))
    idx, frac = ol.cell_of(np.array(keys, dtype=np.uint64))
    starts = [int(v) for v in ol.cell_start(np.arange(ol.CELLS, dtype=np.uint64))]
    starts.append(1 << 64)
    for k, i, f in zip(keys, idx.tolist(), frac.tolist()):
        lo, hi = starts[i], starts[i + 1]
        assert lo <= k < hi, (k, i)
        assert f == (k - lo) * 65536 // (hi - lo), (k, i, f)
    assert np.all(np.diff(idx) >= 0)
    assert idx[-1] == ol.CELLS - 1
    # cell widths: 1 below 2048, then 2^(e-10) for the 1024 cells of exponent e
    assert starts[2048] == 2048 and starts[3072] == 4096 and starts[ol.CELLS - 1] == 2047 << 53


def test_table_monotone_with_heavy_counts():
    p = rand_params(5, scale=0.3)
    heavy = np.array([5, 3000, 10 ** 9, 10 ** 9 + 1, 2 ** 40], dtype=np.uint64)
    t = ol.table(p, heavy, center=0.6, half=0.3)
    assert np.all(np.diff(t[:, 0].astype(np.int64)) >= 0)
    assert tuple(t[-1]) == (0xFFFFFFFF, heavy.size)
    starts = ol.cell_start(np.arange(ol.CELLS, dtype=np.uint64))
    for i in [0, 5, 6, 2999, 3000, 3001, 20000, 40000, ol.CELLS - 1]:
        assert t[i, 1] == sum(1 for h in heavy.tolist() if h < int(starts[i])), i


def test_bucket_ids_monotone_and_heavy_alone():
    p = rand_params(7, scale=0.3)
    rng = np.random.default_rng(8)
    base = np.exp(rng.uniform(18, 44, 20000)).astype(np.uint64)
    heavy = np.unique(base[:300])
    t = ol.table(p, heavy, center=0.6, half=0.3)
    keys = np.sort(np.concatenate([base, heavy - np.uint64(1), heavy + np.uint64(1), heavy]))
    ids = ol.bucket_ids(keys, t, heavy, n_sort=1 << 24)
    assert np.all(np.diff(ids) >= 0)
    ih = ol.bucket_ids(heavy, t, heavy, n_sort=1 << 24)
    assert np.all(ol.bucket_ids(heavy - np.uint64(1), t, heavy, 1 << 24) < ih)
    assert np.all(ol.bucket_ids(heavy + np.uint64(1), t, heavy, 1 << 24) > ih)
    assert ids.max() < ol.buckets_for(1 << 24) + 2 * heavy.size


def test_bucket_ids_hand_case():
    # G_i = i * 2^21 below 2048 (single-key cells), saturating above
    t = np.zeros((ol.CELLS + 1, 2), dtype=np.uint32)
    g = np.minimum(np.arange(ol.CELLS + 1, dtype=np.uint64) << np.uint64(21), 0xFFFFFFFF)
    t[:, 0] = g
    heavy = np.array([10], dtype=np.uint64)
    starts = ol.cell_start(np.arange(ol.CELLS, dtype=np.uint64))
    t[:ol.CELLS, 1] = (starts > 10).astype(np.uint32)
    t[ol.CELLS] = (0xFFFFFFFF, 1)
    k = np.arange(2048, dtype=np.uint64)
    ids = ol.bucket_ids(k, t, heavy, n_sort=1000)  # B = 256: shift 24 -> k >> 3
    want = [(v >> 3) + 2 * (v > 10) + (v == 10) for v in range(2048)]
    assert ids.tolist() == want


def test_judge_rule():
    t = np.zeros((ol.CELLS + 1, 2), dtype=np.uint32)
    t[:, 0] = np.minimum(np.arange(ol.CELLS + 1, dtype=np.uint64) << np.uint64(21), 0xFFFFFFFF)
    t[ol.CELLS] = (0xFFFFFFFF, 0)
    keys = np.repeat(np.arange(0, 800, dtype=np.uint64), 4)  # n = 3200, B = 256, limit = 8 * 3200 / 256
    ok, mx, limit, b = ol.judge(keys, t, np.zeros(0, np.uint64))
    assert (b, limit) == (256, 100) and mx == 32 and ok  # 8 keys per bucket x 4 copies
    keys = np.concatenate([keys, np.full(80, 3, np.uint64)])  # bucket 0 grows to 112 > 8 * 3280 // 256
    ok, mx, limit, _ = ol.judge(keys, t, np.zeros(0, np.uint64))
    assert not ok and mx == 112 and limit == 102


def test_judge_ignores_heavy_buckets():
    # heavy key 10 sits alone in its bucket; its 504 copies must not count as imbalance
    t = np.zeros((ol.CELLS + 1, 2), dtype=np.uint32)
    t[:, 0] = np.minimum(np.arange(ol.CELLS + 1, dtype=np.uint64) << np.uint64(21), 0xFFFFFFFF)
    t[ol.CELLS] = (0xFFFFFFFF, 1)
    keys = np.concatenate([np.repeat(np.arange(0, 800, dtype=np.uint64), 4), np.full(500, 10, np.uint64)])
    heavy = np.array([10], dtype=np.uint64)
    ids = ol.bucket_ids(np.array([9, 10, 11], dtype=np.uint64), t, heavy, keys.size)
    assert ids.tolist() == [1, 2, 3]  # (k >> 3) + 2 [k > 10] + [k == 10]
    ok, mx, limit, b = ol.judge(keys, t, heavy)
    assert (b, limit) == (256, 8 * 3700 // 256) and mx == 32 and ok


def test_feature_closed_form():
    # log2(k + 1) is exact for k + 1 a power of two
    c, h = 0.25, 0.5
    k = np.array([0, 1, 3, (1 << 32) - 1, (1 << 64) - 1], dtype=np.uint64)
    want = [(e / 64 - c) / h for e in (0, 1, 2, 32, 64)]
    assert np.allclose(ol.feature(k, c, h), want, rtol=0, atol=1e-12)


def test_table_of_a_decreasing_network_is_flat():
    # F(x) = sigmoid(-x) for x >= 0 decreases along the cells; its running maximum stays at
    # F(x_0) = 1/2.  With center 0 and half 1/64 the feature is log2(start + 1), so the
    # uniform term is 1/2 at cell 0 and 1 elsewhere: G_0 = 2^32 (15/32 + 1/32) = 2^31 and
    # G_i = 2^32 (15/32 + 2/32) = 17 * 2^27 for every later cell.
    p = np.zeros(ol.PARAMS)
    p[0] = 1.0                     # W1[0]
    p[128] = 1.0                   # W2[0][0]
    p[128 + 4096 + 64] = -1.0      # W3[0]
    t = ol.table(p, np.zeros(0, np.uint64), center=0.0, half=1.0 / 64.0)
    assert t[0, 0] == 1 << 31
    assert np.all(t[1:ol.CELLS, 0] == 17 << 27)
    assert tuple(t[ol.CELLS]) == (0xFFFFFFFF, 0)


def test_buckets_for_rounds_up_and_clamps():
    # B = the smallest power of two >= n / 1024, clamped to [2^8, 2^22]
    assert ol.buckets_for(1) == 256 and ol.buckets_for(256 * 1024) == 256
    assert ol.buckets_for(256 * 1024 + 1) == 512
    assert ol.buckets_for(1 << 30) == 1 << 20 and ol.buckets_for((1 << 30) + 1) == 1 << 21
    assert ol.buckets_for(1 << 40) == 1 << 22
