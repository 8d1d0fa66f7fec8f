"""Seeded synthetic workloads shaped like the paper's inputs.

The paper's test bed fills batches of keys from a random number generator
(Sec. IV-A); its keys are uniformly distributed and skew is named as future
work.  The workloads here add the skewed shapes the sort must survive: Zipf,
a clamped discretised Gaussian, mostly-presorted input and all-equal keys.

This module holds none of the sort's arithmetic.  It is shared by the oracle's
tests, the CUDA parity tests and the benchmark, and it imports neither the
oracle nor the product.  The recipe (see wl_gen.h) is counter-based: element i
depends only on (seed, stream, i), the host (C) and device (CUDA) versions give
identical bytes, and inverse-CDF tables are plain data built here once.

Named distributions (16-bit top part; wider keys get uniform low bits):
  uniform    every bit uniform
  zipf1.1    P(top = r - 1) proportional to r^-1.1, r = 1..65536
  gauss      N(32768, 1024) over the top 16 bits, rounded to the nearest value
             and clamped to [0, 65535]  (sigma 1024 for 16-bit keys; 256 in
             top-16 units for 32-bit keys, i.e. sigma = 2^24 on the full key)
  presorted  ascending ramp on the top 16 bits with 10 % of elements replaced
             by uniform draws
  equal      every key 0xA5A5...
  mixture    (64-bit keys) 90 % from 8 lognormal clusters (ln-means U[20,40], ln-sigmas
             U[0.1,1], Dirichlet(1) weights) through a 65,537-point piecewise-linear
             inverse CDF, 10 % Zipf s=1.3 over 65,536 hot values drawn from the mixture
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_HOST_SRC = os.path.join(_HERE, "wl_gen.c")
_DEV_SRC = os.path.join(_HERE, "wl_gen_device.cu")
_HDR = os.path.join(_HERE, "wl_gen.h")
_HOST_LIB = os.path.join(_HERE, "libwl_host.so")
_DEV_LIB = os.path.join(_HERE, "libwl_device.so")

WL_UNIFORM, WL_TABLE, WL_PRESORTED, WL_CONSTANT, WL_QUANTILE, WL_HOTSET = 0, 1, 2, 3, 4, 5
GAMMA = 0x9E3779B97F4A7C15
MASK64 = (1 << 64) - 1

DISTRIBUTIONS = ("uniform", "zipf1.1", "gauss", "presorted", "equal")
_KEY_DTYPES = {16: np.uint16, 32: np.uint32, 64: np.uint64}

_lock = threading.Lock()
_host = None
_dev = None
_table_cache: dict = {}


class WlParams(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64), ("stream", ctypes.c_uint64), ("n_total", ctypes.c_uint64),
        ("dist", ctypes.c_int32), ("key_bits", ctypes.c_int32), ("hot_prob", ctypes.c_uint32),
        ("pad", ctypes.c_uint32), ("table", ctypes.c_void_p), ("quant", ctypes.c_void_p), ("hot", ctypes.c_void_p),
    ]


def _stale(lib: str, *srcs: str) -> bool:
    return not os.path.exists(lib) or any(os.path.getmtime(lib) < os.path.getmtime(s) for s in srcs)


def build_host(force: bool = False) -> str:
    if force or _stale(_HOST_LIB, _HOST_SRC, _HDR):
        tmp = _HOST_LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _HOST_SRC])
        os.replace(tmp, _HOST_LIB)
    return _HOST_LIB


def device_build_cmd(out: str) -> list:
    return ["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-shared", "-Xcompiler", "-fPIC",
            "-o", out, _DEV_SRC]


def build_device(force: bool = False) -> str:
    if force or _stale(_DEV_LIB, _DEV_SRC, _HDR):
        tmp = _DEV_LIB + f".tmp{os.getpid()}"
        subprocess.check_call(device_build_cmd(tmp))
        os.replace(tmp, _DEV_LIB)
    return _DEV_LIB


def _host_lib():
    global _host
    with _lock:
        if _host is None:
            build_host()
            lib = ctypes.CDLL(_HOST_LIB)
            lib.wl_fill.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.POINTER(WlParams)]
            lib.wl_fill.restype = ctypes.c_int
            lib.wl_raw.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.wl_raw.restype = ctypes.c_uint64
            lib.wl_stream_base.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
            lib.wl_stream_base.restype = ctypes.c_uint64
            _host = lib
    return _host


def _dev_lib():
    global _dev
    with _lock:
        if _dev is None:
            if not os.path.exists(_DEV_LIB):
                raise RuntimeError("workloads device generator not built (run __graft_entry__.build())")
            lib = ctypes.CDLL(_DEV_LIB)
            lib.wl_fill_device.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                           ctypes.POINTER(WlParams), ctypes.c_void_p]
            lib.wl_fill_device.restype = ctypes.c_int
            lib.wl_iota_device.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p]
            lib.wl_iota_device.restype = ctypes.c_int
            _dev = lib
    return _dev


# ---- inverse-CDF tables (plain data) ----------------------------------------

def thresholds_from_pmf(pmf: np.ndarray) -> np.ndarray:
    """65,535 ascending u64 thresholds T so that key t is drawn with
    probability pmf[t] when key = smallest t with u < T[t] (u uniform 64-bit)."""
    pmf = np.asarray(pmf, dtype=np.float64)
    if pmf.shape != (65536,):
        raise ValueError("pmf must have 65536 entries")
    cdf = np.cumsum(pmf / pmf.sum())[:-1]
    scaled = np.minimum(cdf * 2.0 ** 64, 2.0 ** 64 - 4096.0)
    return scaled.astype(np.uint64)


def zipf_pmf(s: float) -> np.ndarray:
    r = np.arange(1, 65537, dtype=np.float64)
    return r ** (-s)


def gaussian_pmf(mu: float, sigma: float) -> np.ndarray:
    """Rounded to the nearest integer and clamped to [0, 65535]."""
    edges = (np.arange(0, 65537, dtype=np.float64) - 0.5 - mu) / (sigma * math.sqrt(2.0))
    cdf = 0.5 * (1.0 + np.array([math.erf(x) for x in edges]))
    cdf[0], cdf[-1] = 0.0, 1.0
    return np.diff(cdf)


def table_for(name: str, key_bits: int):
    key = (name, key_bits)
    if key not in _table_cache:
        if name == "zipf1.1":
            _table_cache[key] = thresholds_from_pmf(zipf_pmf(1.1))
        elif name == "gauss":
            sigma = 1024.0 if key_bits == 16 else 256.0
            _table_cache[key] = thresholds_from_pmf(gaussian_pmf(32768.0, sigma))
        else:
            _table_cache[key] = None
    return _table_cache[key]


_MIX_CACHE: dict = {}


def lognormal_mixture(seed: int = 0, clusters: int = 8):
    """Mixture of `clusters` lognormal clusters: ln-means ~ U[20, 40], ln-sigmas
    ~ U[0.1, 1], weights ~ Dirichlet(1), all from `seed`.  Returns (mu, sigma, w)."""
    rng = np.random.default_rng(1000 + seed)
    mu = rng.uniform(20.0, 40.0, clusters)
    sigma = rng.uniform(0.1, 1.0, clusters)
    w = rng.dirichlet(np.ones(clusters))
    return mu, sigma, w


def _mixture_cdf(logx: np.ndarray, mu, sigma, w) -> np.ndarray:
    z = (logx[:, None] - mu[None, :]) / (sigma[None, :] * math.sqrt(2.0))
    erf = np.vectorize(math.erf)
    return (w[None, :] * 0.5 * (1.0 + erf(z))).sum(axis=1)


def mixture_tables(seed: int = 0):
    """Plain data for the learned-sort workload: 65,537 ascending u64 quantile
    points of the lognormal mixture (piecewise-linear inverse CDF), 65,536
    hot values drawn from the mixture, and the Zipf s=1.3 threshold table over
    their ranks.  Computed in float64 by bisection on ln(key)."""
    if seed in _MIX_CACHE:
        return _MIX_CACHE[seed]
    mu, sigma, w = lognormal_mixture(seed)
    probs = np.arange(65537, dtype=np.float64) / 65536.0
    probs[0], probs[-1] = 1e-9, 1.0 - 1e-9
    lo = np.full(probs.shape, float((mu - 8 * sigma).min()))
    hi = np.full(probs.shape, min(float((mu + 8 * sigma).max()), 44.0))
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        below = _mixture_cdf(mid, mu, sigma, w) < probs
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
    keys = np.minimum(np.exp(hi), 2.0 ** 64 - 4096.0)
    quant = np.maximum.accumulate(keys.astype(np.uint64))
    rng = np.random.default_rng(2000 + seed)
    u = rng.random(65536)
    idx = np.minimum((u * 65536).astype(np.int64), 65535)
    frac = u * 65536 - idx
    hot = (quant[idx] + (quant[idx + 1] - quant[idx]) * frac).astype(np.uint64)
    table = thresholds_from_pmf(zipf_pmf(1.3))
    _MIX_CACHE[seed] = (quant, hot, table)
    return _MIX_CACHE[seed]


MIXTURE_HOT_PROB = int(0.1 * 2 ** 32)


def params_for(name: str, n_total: int, key_bits: int, seed: int, stream: int):
    """(WlParams, table) for a named distribution; the table (or None) must be
    kept alive, and for device use copied to the device and its pointer set."""
    if key_bits not in _KEY_DTYPES:
        raise ValueError("key_bits must be 16, 32 or 64")
    if name == "mixture":
        quant, hot, table = mixture_tables(0)
        p = WlParams(seed=seed, stream=stream, n_total=n_total, dist=WL_HOTSET, key_bits=key_bits,
                     hot_prob=MIXTURE_HOT_PROB, pad=0, table=None, quant=None, hot=None)
        return p, (table, quant, hot)
    dist = {"uniform": WL_UNIFORM, "zipf1.1": WL_TABLE, "gauss": WL_TABLE, "presorted": WL_PRESORTED,
            "equal": WL_CONSTANT}.get(name)
    if dist is None:
        raise ValueError(f"unknown distribution {name!r}; known: {DISTRIBUTIONS + ('mixture',)}")
    table = table_for(name, key_bits)
    p = WlParams(seed=seed, stream=stream, n_total=n_total, dist=dist, key_bits=key_bits, hot_prob=0, pad=0,
                 table=None, quant=None, hot=None)
    return p, table


def generate(name: str, n: int, key_bits: int = 16, seed: int = 0, stream: int = 0, start: int = 0,
             n_total: int | None = None) -> np.ndarray:
    """Keys start..start+n-1 of a workload of n_total (default n) keys, on the host."""
    lib = _host_lib()
    p, table = params_for(name, n if n_total is None else n_total, key_bits, seed, stream)
    if isinstance(table, tuple):
        p.table, p.quant, p.hot = (t.ctypes.data_as(ctypes.c_void_p).value for t in table)
    elif table is not None:
        p.table = table.ctypes.data_as(ctypes.c_void_p).value
    out = np.empty(n, dtype=_KEY_DTYPES[key_bits])
    rc = lib.wl_fill(out.ctypes.data_as(ctypes.c_void_p), start, n, ctypes.byref(p))
    if rc:
        raise RuntimeError(f"wl_fill failed ({rc})")
    return out


def generate_device(name: str, out_ptr: int, n: int, key_bits: int, seed: int = 0, stream: int = 0,
                    start: int = 0, n_total: int | None = None, cuda_stream: int = 0, table_dev_ptr: int | None = None):
    """Same keys written straight into device memory at out_ptr.  For table
    distributions, table_dev_ptr must point at a device copy of table_for()."""
    lib = _dev_lib()
    p, table = params_for(name, n if n_total is None else n_total, key_bits, seed, stream)
    if isinstance(table, tuple):
        if not isinstance(table_dev_ptr, (tuple, list)) or len(table_dev_ptr) != 3:
            raise ValueError("the mixture needs (table, quantiles, hot values) device pointers")
        p.table, p.quant, p.hot = table_dev_ptr
    elif table is not None:
        if table_dev_ptr is None:
            raise ValueError("table distribution needs table_dev_ptr")
        p.table = table_dev_ptr
    rc = lib.wl_fill_device(ctypes.c_void_p(out_ptr), start, n, ctypes.byref(p), ctypes.c_void_p(cuda_stream))
    if rc:
        raise RuntimeError(f"wl_fill_device failed ({rc})")


def iota_device(out_ptr: int, n: int, start: int = 0, cuda_stream: int = 0):
    rc = _dev_lib().wl_iota_device(ctypes.c_void_p(out_ptr), start, n, ctypes.c_void_p(cuda_stream))
    if rc:
        raise RuntimeError(f"wl_iota_device failed ({rc})")


# ---- pure-Python statement of the random source, for pinning the C code ----

def py_mix(z: int) -> int:
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def py_raw(base: int, i: int) -> int:
    return py_mix((base + (i + 1) * GAMMA) & MASK64)


def raw(base: int, i: int) -> int:
    return int(_host_lib().wl_raw(base, i))


def stream_base(seed: int, stream: int, sub: int) -> int:
    return int(_host_lib().wl_stream_base(seed, stream, sub))
