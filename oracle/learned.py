"""CPU oracle for the learned bucket mapping.

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and nothing else.  It never
imports the product library and shares no code with it.

The paper has no learned component; the mapping serves the skewed inputs the
paper leaves open (Sec. IV-A).  What it computes is fixed by the library's
interface definition (the learned section of ``include/fsort.h``), restated
here plainly, float64 unless stated:

  model    F(x) = sigmoid(W3 . relu(W2 relu(W1 x + b1) + b2) + b3); flat
           parameter order W1[64], b1[64], W2[64][64] (row j feeds hidden unit
           j of layer 2), b2[64], W3[64], b3.  The library evaluates it with
           BF16-rounded weights, so callers pass those weights here.
  loss     L = 1/(2m) sum_i (F(x_i) - y_i)^2; gradient by the chain rule,
           layer by layer (``loss_and_grad``).
  feature  x(k) = (log2(k + 1) / 64 - center) / half.
  grid     cell of key k: k itself below 2048, else (e - 9) * 1024 + the 10
           bits below the leading one, e = floor(log2 k); a cell of width 2^w
           holds the keys whose bits below w are free; frac16 = position inside
           the cell in 1/65536 units.
  table    G_i = floor(2^32 * ((1 - eps) max_{j <= i} F(x(start_j)) +
           eps * clamp((x(start_i) + 1) / 2, 0, 1))) for the 56,320 cells (all
           ones in the closing entry), eps = 1/16; H_i = heavy keys below
           start_i.
  map      id(k) = (PLA(k) >> shift) + 2 c(k) + e(k), PLA(k) = G_i +
           floor((G_{i+1} - G_i) * frac16 / 2^16), c(k) = heavy keys below k,
           e(k) = [k is heavy], shift = 32 - log2(B), B = the power of two >= n /
           1024 clamped to [2^8, 2^22].
  judge    accept iff max over non-heavy ids of their counts <= floor(8 n / B).

The sort built on the map returns the sorted multiset of the keys, so its
expected output is ``oracle.sort`` at full precision.
"""
from __future__ import annotations

import math

import numpy as np

H = 64
PARAMS = 4353
CELLS = 56320
EPS = 1.0 / 16.0
TAU = 8
CAPACITY = 8192
KEYS_PER_BUCKET = 1024

_W1, _B1, _W2, _B2, _W3, _B3 = 0, H, 2 * H, 2 * H + H * H, 3 * H + H * H, 4 * H + H * H


def unpack(params):
    p = np.asarray(params, dtype=np.float64)
    if p.shape != (PARAMS,):
        raise ValueError(f"expected {PARAMS} parameters")
    return (p[_W1:_B1], p[_B1:_W2], p[_W2:_B2].reshape(H, H), p[_B2:_W3], p[_W3:_B3], p[_B3])


def bf16_round(a) -> np.ndarray:
    """float32 values rounded to the nearest BF16 (ties to even), as float32."""
    bits = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    bias = 0x7FFF + ((bits >> 16) & 1)
    return ((bits + bias) & 0xFFFF0000).astype(np.uint32).view(np.float32)


def _sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def forward(params, x) -> np.ndarray:
    """F(x) for every x (float64)."""
    w1, b1, w2, b2, w3, b3 = unpack(params)
    x = np.asarray(x, dtype=np.float64)
    h1 = np.maximum(0.0, np.outer(x, w1) + b1)        # m x 64
    h2 = np.maximum(0.0, h1 @ w2.T + b2)              # m x 64
    return _sigmoid(h2 @ w3 + b3)


def loss_and_grad(params, x, y):
    """(L, dL/dparams) for L = 1/(2m) sum (F(x) - y)^2."""
    w1, b1, w2, b2, w3, b3 = unpack(params)
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    m = x.shape[0]
    a1 = np.outer(x, w1) + b1
    h1 = np.maximum(0.0, a1)
    a2 = h1 @ w2.T + b2
    h2 = np.maximum(0.0, a2)
    f = _sigmoid(h2 @ w3 + b3)
    err = f - y
    loss = 0.5 * np.sum(err * err) / m
    dz = err * f * (1.0 - f) / m                        # dL/dz per input
    g_w3 = h2.T @ dz
    g_b3 = np.sum(dz)
    d2 = np.outer(dz, w3) * (a2 > 0)                    # dL/da2
    g_w2 = d2.T @ h1                                    # [j][i] = sum d2_j h1_i
    g_b2 = d2.sum(axis=0)
    d1 = (d2 @ w2) * (a1 > 0)                           # dL/da1
    g_w1 = d1.T @ x
    g_b1 = d1.sum(axis=0)
    grad = np.concatenate([g_w1, g_b1, g_w2.ravel(), g_b2, g_w3, [g_b3]])
    return loss, grad


def feature(keys, center: float, half: float) -> np.ndarray:
    k = np.asarray(keys, dtype=np.uint64).astype(np.float64)
    return (np.log2(k + 1.0) / 64.0 - center) / half


def cell_start(i) -> np.ndarray:
    """First key of each cell index i (0 <= i < CELLS)."""
    i = np.asarray(i, dtype=np.uint64)
    e = (i >> np.uint64(10)) + np.uint64(9)
    big = (np.uint64(1024) + (i & np.uint64(1023))) << np.maximum(e, np.uint64(10)) - np.uint64(10)
    return np.where(i < 2048, i, big)


def cell_of(keys):
    """(cell index, frac16) of every key."""
    k = np.asarray(keys, dtype=np.uint64)
    small = k < 2048
    kk = np.where(small, np.uint64(2048), k)
    e = np.zeros(k.shape, dtype=np.uint64)  # floor(log2 k) by bisection on the bit position
    for step in (32, 16, 8, 4, 2, 1):
        up = (kk >> (e + np.uint64(step))) != 0
        e = np.where(up, e + np.uint64(step), e)
    e = e.astype(np.int64)
    w = (e - 10).astype(np.uint64)
    idx = (e - 9).astype(np.uint64) * np.uint64(1024) + ((kk >> w) & np.uint64(1023))
    rem = kk & ((np.uint64(1) << w) - np.uint64(1))
    frac = np.where(w >= 16, rem >> np.maximum(w, np.uint64(16)) - np.uint64(16),
                    rem << np.uint64(16) - np.minimum(w, np.uint64(16)))
    idx = np.where(small, k, idx)
    frac = np.where(small, np.uint64(0), frac)
    return idx.astype(np.int64), frac.astype(np.uint64)


def table(params, heavy, center: float, half: float) -> np.ndarray:
    """The (G, H) table of a model: uint32 array of shape (CELLS + 1, 2)."""
    heavy = np.asarray(heavy, dtype=np.uint64)
    starts = cell_start(np.arange(CELLS, dtype=np.uint64))
    x = feature(starts, center, half)
    run = np.maximum.accumulate(np.clip(forward(params, x), 0.0, 1.0))
    v = (1.0 - EPS) * run + EPS * np.clip(0.5 * (x + 1.0), 0.0, 1.0)
    g = np.where(v >= 1.0, 0xFFFFFFFF, np.floor(v * 2.0 ** 32)).astype(np.uint64)
    out = np.zeros((CELLS + 1, 2), dtype=np.uint32)
    out[:CELLS, 0] = np.minimum(g, 0xFFFFFFFF)
    out[:CELLS, 1] = np.searchsorted(heavy, starts, side="left")
    out[CELLS] = (0xFFFFFFFF, heavy.size)
    return out


def buckets_for(n: int) -> int:
    want = -(-n // KEYS_PER_BUCKET)
    b = 256
    while b < want and b < (1 << 22):
        b <<= 1
    return b


def bucket_ids(keys, cells, heavy, n_sort: int) -> np.ndarray:
    """id(k) of every key under the table, with the B of a sort of n_sort keys."""
    k = np.asarray(keys, dtype=np.uint64)
    cells = np.asarray(cells, dtype=np.uint64)
    heavy = np.asarray(heavy, dtype=np.uint64)
    shift = np.uint64(32 - int(math.log2(buckets_for(n_sort))))
    idx, frac = cell_of(k)
    g0, g1 = cells[idx, 0], cells[idx + 1, 0]
    pla = g0 + (((g1 - g0) * frac) >> np.uint64(16))
    c = np.searchsorted(heavy, k, side="left").astype(np.uint64)
    hit = np.zeros(k.shape, dtype=bool)
    if heavy.size:
        at = np.minimum(c, heavy.size - 1).astype(np.int64)
        hit = heavy[at] == k
    return ((pla >> shift) + np.uint64(2) * c + hit.astype(np.uint64)).astype(np.int64)


def judge(keys, cells, heavy):
    """(accept, max non-heavy bucket, limit, B) for a sort of these keys."""
    k = np.asarray(keys, dtype=np.uint64)
    n = k.size
    b = buckets_for(n)
    ids = bucket_ids(k, cells, heavy, n)
    heavy = np.asarray(heavy, dtype=np.uint64)
    nonheavy = ~np.isin(k, heavy)
    counts = np.bincount(ids[nonheavy]) if nonheavy.any() else np.zeros(1, np.int64)
    mx = int(counts.max()) if counts.size else 0
    limit = TAU * n // b
    return mx <= limit and mx <= CAPACITY, mx, limit, b
