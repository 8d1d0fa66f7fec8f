"""CPU oracle for the compressed radix sort hot path (arXiv 2605.10390).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The product library never imports,
links or runs anything in this package, and this package never imports the
product.  The arithmetic lives in ``oracle.c`` (plain single-threaded C, each
function citing the paper passage it follows); this module only marshals numpy
arrays into it, plus invariant checkers written with numpy.

Function map (paper passage -> function):
  Sec. II (histogram, prefix sum, stable scatter) ........ sort, scatter_pass
  Sec. III-A/B (per-key counter updates) ................. digit_histograms
  Alg. 3 (GetIndex = rank of a leaf) ..................... exclusive_scan, tree_rank
  Alg. 2 (GetItem = select) .............................. tree_select
  Alg. 1 + Sec. III-B-1 (Fractal RMW, every path node) ... tree_build
  Alg. 5 with no trailing bits ........................... expand
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_KEY_DTYPES = {16: np.uint16, 32: np.uint32, 64: np.uint64}


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (plain C, no SIMD flags)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            u64, i32, vp = ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p
            lib.oracle_sort.argtypes = [vp, vp, vp, vp, u64, i32, i32]
            lib.oracle_sort.restype = i32
            lib.oracle_scatter_pass.argtypes = [vp, vp, vp, vp, u64, i32, i32, i32]
            lib.oracle_scatter_pass.restype = i32
            lib.oracle_digit_histograms.argtypes = [vp, u64, i32, i32, i32, vp]
            lib.oracle_digit_histograms.restype = i32
            lib.oracle_exclusive_scan.argtypes = [vp, u64, vp]
            lib.oracle_exclusive_scan.restype = None
            lib.oracle_num_passes.argtypes = [i32, i32]
            lib.oracle_num_passes.restype = i32
            lib.oracle_tree_size.argtypes = [i32]
            lib.oracle_tree_size.restype = u64
            lib.oracle_tree_build.argtypes = [vp, u64, i32, i32, vp]
            lib.oracle_tree_build.restype = i32
            lib.oracle_tree_count.argtypes = [vp, i32, i32, u64]
            lib.oracle_tree_count.restype = u64
            lib.oracle_tree_rank.argtypes = [vp, i32, u64]
            lib.oracle_tree_rank.restype = u64
            lib.oracle_tree_select.argtypes = [vp, i32, u64]
            lib.oracle_tree_select.restype = u64
            lib.oracle_expand.argtypes = [vp, u64, i32, vp]
            lib.oracle_expand.restype = i32
            _lib = lib
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _keys(keys: np.ndarray, key_bits: int) -> np.ndarray:
    dt = _KEY_DTYPES[key_bits]
    if keys.dtype != dt:
        raise TypeError(f"keys must be {np.dtype(dt).name} for key_bits={key_bits}")
    return np.ascontiguousarray(keys)


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


def sort(keys: np.ndarray, vals: np.ndarray | None, key_bits: int, precision_bits: int):
    """Stable ascending sort on the top ``precision_bits`` bits (Sec. II)."""
    lib = _load()
    keys = _keys(keys, key_bits)
    n = keys.shape[0]
    ko = np.empty_like(keys)
    vo = None
    if vals is not None:
        vals = np.ascontiguousarray(vals, dtype=np.uint32)
        if vals.shape[0] != n:
            raise ValueError("vals length differs from keys")
        vo = np.empty_like(vals)
    _check(lib.oracle_sort(_ptr(keys), _ptr(vals), _ptr(ko), _ptr(vo), n, key_bits, precision_bits), "sort")
    return ko, vo


def scatter_pass(keys: np.ndarray, vals: np.ndarray | None, key_bits: int, shift: int, width: int):
    """One stable counting pass on raw key bits [shift, shift+width)."""
    lib = _load()
    keys = _keys(keys, key_bits)
    ko = np.empty_like(keys)
    vo = None
    if vals is not None:
        vals = np.ascontiguousarray(vals, dtype=np.uint32)
        vo = np.empty_like(vals)
    _check(lib.oracle_scatter_pass(_ptr(keys), _ptr(vals), _ptr(ko), _ptr(vo), keys.shape[0], key_bits, shift,
                                   width), "scatter_pass")
    return ko, vo


def num_passes(precision_bits: int, digit_bits: int) -> int:
    return int(_load().oracle_num_passes(precision_bits, digit_bits))


def digit_histograms(keys: np.ndarray, key_bits: int, precision_bits: int, digit_bits: int) -> np.ndarray:
    """counts[j, v] = number of keys whose pass-j digit equals v."""
    lib = _load()
    keys = _keys(keys, key_bits)
    passes = num_passes(precision_bits, digit_bits)
    out = np.zeros((passes, 1 << digit_bits), dtype=np.uint64)
    _check(lib.oracle_digit_histograms(_ptr(keys), keys.shape[0], key_bits, precision_bits, digit_bits, _ptr(out)),
           "digit_histograms")
    return out


def exclusive_scan(counts: np.ndarray) -> np.ndarray:
    lib = _load()
    c = np.ascontiguousarray(counts, dtype=np.uint64).reshape(-1)
    out = np.empty_like(c)
    lib.oracle_exclusive_scan(_ptr(c), c.shape[0], _ptr(out))
    return out.reshape(np.shape(counts))


def tree_build(keys: np.ndarray, key_bits: int, precision_bits: int) -> np.ndarray:
    lib = _load()
    keys = _keys(keys, key_bits)
    tree = np.zeros(int(lib.oracle_tree_size(precision_bits)), dtype=np.uint64)
    _check(lib.oracle_tree_build(_ptr(keys), keys.shape[0], key_bits, precision_bits, _ptr(tree)), "tree_build")
    return tree


def tree_count(tree: np.ndarray, precision_bits: int, level: int, prefix: int) -> int:
    return int(_load().oracle_tree_count(_ptr(tree), precision_bits, level, prefix))


def tree_rank(tree: np.ndarray, precision_bits: int, v: int) -> int:
    return int(_load().oracle_tree_rank(_ptr(tree), precision_bits, v))


def tree_select(tree: np.ndarray, precision_bits: int, r: int) -> int:
    return int(_load().oracle_tree_select(_ptr(tree), precision_bits, r))


def expand(counts: np.ndarray, key_bits: int) -> np.ndarray:
    lib = _load()
    c = np.ascontiguousarray(counts, dtype=np.uint64).reshape(-1)
    out = np.empty(int(c.sum()), dtype=_KEY_DTYPES[key_bits])
    _check(lib.oracle_expand(_ptr(c), c.shape[0], key_bits, _ptr(out)), "expand")
    return out


# ---- invariant checkers (numpy) ---------------------------------------------
# With vals = original index, these three facts pin the unique stable result:
#   (1) vals_out is a permutation of 0..n-1;
#   (2) keys_out[i] == keys_in[vals_out[i]];
#   (3) (s(keys_out[i]), vals_out[i]) strictly increases with i.

def sort_key(keys: np.ndarray, key_bits: int, precision_bits: int) -> np.ndarray:
    return (keys.astype(np.uint64) >> np.uint64(key_bits - precision_bits))


def check_sorted_stable(keys_in: np.ndarray, keys_out: np.ndarray, idx_out: np.ndarray, key_bits: int,
                        precision_bits: int) -> None:
    """Raise AssertionError unless (keys_out, idx_out) is the stable sort of
    keys_in on the top precision_bits bits, idx_out holding original indices."""
    n = keys_in.shape[0]
    if keys_out.shape[0] != n or idx_out.shape[0] != n:
        raise AssertionError("length mismatch")
    idx = idx_out.astype(np.int64)
    if n == 0:
        return
    if idx.min() < 0 or idx.max() >= n:
        raise AssertionError("index out of range")
    seen = np.zeros(n, dtype=bool)
    seen[idx] = True
    if not seen.all():
        raise AssertionError("indices are not a permutation")
    if not np.array_equal(keys_out, keys_in[idx]):
        raise AssertionError("keys_out[i] != keys_in[idx_out[i]]")
    s = sort_key(keys_out, key_bits, precision_bits)
    s_prev, s_next = s[:-1], s[1:]
    i_prev, i_next = idx[:-1], idx[1:]
    ok = (s_prev < s_next) | ((s_prev == s_next) & (i_prev < i_next))
    if not ok.all():
        bad = int(np.argmin(ok))
        raise AssertionError(f"order or stability broken at position {bad}")


def check_sorted_multiset(keys_in: np.ndarray, keys_out: np.ndarray, key_bits: int, precision_bits: int) -> None:
    """Keys-only check: same multiset and non-decreasing on the sort key.  For
    precision_bits == key_bits this pins the output uniquely."""
    if keys_out.shape != keys_in.shape:
        raise AssertionError("length mismatch")
    s = sort_key(keys_out, key_bits, precision_bits)
    if s.shape[0] > 1 and not (s[:-1] <= s[1:]).all():
        raise AssertionError("not sorted")
    if not np.array_equal(np.sort(keys_in, kind="stable"), np.sort(keys_out, kind="stable")):
        raise AssertionError("multiset differs")
