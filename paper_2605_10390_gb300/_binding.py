"""ctypes binding of libfsort (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB = os.path.join(_PKG, "libfsort.so")
_lock = threading.Lock()
_lib = None

FSORT_FLAG_HOST_IO = 0x4
FSORT_FLAG_GRAPH = 0x2
FSORT_FLAG_LEARNED = 0x8
FSORT_FLAG_CHAINED_SCATTER = 0x10
FSORT_MLP_PARAMS = 4353
FSORT_LEARN_CELLS = 56320
FSORT_LEARN_MAX_HEAVY = 8192

STATUS = {
    0: "FSORT_OK", 1: "FSORT_ERR_INVALID_ARG", 2: "FSORT_ERR_OOM", 3: "FSORT_ERR_CUDA", 4: "FSORT_ERR_TIMEOUT",
    5: "FSORT_ERR_BUSY", 6: "FSORT_NOT_READY", 7: "FSORT_ERR_INTERNAL", 8: "FSORT_ERR_UNSUPPORTED",
}


class FsortError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}")


class FsortPlanDesc(ctypes.Structure):
    _fields_ = [("max_n", ctypes.c_uint64), ("key_bits", ctypes.c_int32), ("has_values", ctypes.c_int32),
                ("digit_bits", ctypes.c_int32), ("flags", ctypes.c_uint32), ("max_segments", ctypes.c_uint32)]


class FsortSegment(ctypes.Structure):
    _fields_ = [("keys", ctypes.c_void_p), ("vals", ctypes.c_void_p), ("n", ctypes.c_uint64)]


class FsortBatchConfig(ctypes.Structure):
    _fields_ = [("small_capacity", ctypes.c_int32), ("small_ctas_per_sm", ctypes.c_int32),
                ("large_form", ctypes.c_int32), ("digit_bits", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {"small_capacity": self.small_capacity, "small_ctas_per_sm": self.small_ctas_per_sm,
                "large_form": self.large_form, "digit_bits": self.digit_bits or 8}


class FsortPlanInfo(ctypes.Structure):
    _fields_ = [("passes", ctypes.c_int32), ("digit_bits", ctypes.c_int32), ("expand_path", ctypes.c_int32),
                ("tile_keys", ctypes.c_int32), ("num_tiles", ctypes.c_uint64), ("chunk_keys", ctypes.c_uint64),
                ("workspace_bytes", ctypes.c_uint64), ("algorithmic_bytes", ctypes.c_uint64),
                ("scatter_form", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class FsortKernelTime(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("pass_", ctypes.c_int32), ("active", ctypes.c_int32),
                ("call", ctypes.c_int32), ("n", ctypes.c_uint64), ("ms", ctypes.c_float), ("reserved", ctypes.c_float)]


class FsortLearnedOpts(ctypes.Structure):
    _fields_ = [("sample_keys", ctypes.c_uint32), ("steps", ctypes.c_uint32), ("batch", ctypes.c_uint32),
                ("lr", ctypes.c_float), ("seed", ctypes.c_uint64)]


class FsortLearnedStats(ctypes.Structure):
    _fields_ = [("fitted", ctypes.c_int32), ("used", ctypes.c_int32), ("buckets", ctypes.c_uint32),
                ("heavy_keys", ctypes.c_uint32), ("max_bucket", ctypes.c_uint32), ("limit", ctypes.c_uint32),
                ("imbalance", ctypes.c_double), ("tau", ctypes.c_double), ("sample_keys", ctypes.c_uint32),
                ("train_keys", ctypes.c_uint32), ("steps", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("loss_first", ctypes.c_float), ("loss_last", ctypes.c_float)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class FsortServeDesc(ctypes.Structure):
    _fields_ = [("max_request_keys", ctypes.c_uint64), ("hbm_budget_bytes", ctypes.c_uint64),
                ("key_bits", ctypes.c_int32), ("has_values", ctypes.c_int32), ("lanes", ctypes.c_uint32),
                ("max_queue", ctypes.c_uint32), ("batch_keys", ctypes.c_uint32), ("max_batch", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class FsortRequest(ctypes.Structure):
    _fields_ = [("keys_host", ctypes.c_void_p), ("vals_host", ctypes.c_void_p), ("keys_out_host", ctypes.c_void_p),
                ("vals_out_host", ctypes.c_void_p), ("n", ctypes.c_uint64), ("precision_bits", ctypes.c_int32),
                ("reserved", ctypes.c_uint32)]


class FsortResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("batched", ctypes.c_int32), ("n", ctypes.c_uint64),
                ("latency_ms", ctypes.c_double), ("queue_ms", ctypes.c_double), ("run_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class FsortServeStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("keys_completed", ctypes.c_uint64),
                ("batches", ctypes.c_uint64), ("bytes_in_use", ctypes.c_uint64), ("peak_bytes", ctypes.c_uint64),
                ("budget_bytes", ctypes.c_uint64), ("max_inflight", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("span_s", ctypes.c_double), ("keys_per_s", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


KERNEL_KINDS = {1: "histogram", 2: "scan", 3: "scatter", 4: "copy", 5: "leaf_hist", 6: "leaf_reduce",
                7: "leaf_scan", 8: "expand", 9: "learn_count1", 10: "learn_scatter1", 11: "learn_count2",
                12: "learn_judge", 13: "learn_scatter2", 14: "learn_fill", 15: "learn_buckets", 16: "tile_count",
                17: "tile_scan"}


def lib_path() -> str:
    return _LIB


def load_library():
    """Load libfsort.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB):
            raise RuntimeError(f"libfsort.so is not built ({_LIB}); run __graft_entry__.build() first")
        lib = ctypes.CDLL(_LIB)
        vp, u64, i32, st = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_int
        sig = {
            "fsort_plan_create": ([ctypes.POINTER(FsortPlanDesc), ctypes.POINTER(vp)], st),
            "fsort_plan_destroy": ([vp], st),
            "fsort_plan_sync": ([vp], st),
            "fsort_plan_describe": ([vp, u64, i32, i32, i32, ctypes.POINTER(FsortPlanInfo)], st),
            "fsort_sort_pairs": ([vp, vp, vp, u64, i32, i32, vp], st),
            "fsort_sort_pairs_out": ([vp, vp, vp, vp, vp, u64, i32, i32, vp], st),
            "fsort_sort_pairs_host": ([vp, vp, vp, u64, i32, i32, vp], st),
            "fsort_histogram": ([vp, vp, u64, i32, i32, i32, vp, vp], st),
            "fsort_exclusive_scan": ([vp, vp, u64, u64, vp, vp], st),
            "fsort_scatter_pass": ([vp, vp, vp, vp, vp, u64, i32, i32, i32, vp], st),
            "fsort_expand": ([vp, vp, vp, u64, i32, vp], st),
            "fsort_plan_set_timing": ([vp, i32], st),
            "fsort_plan_timing_report": ([vp, ctypes.POINTER(FsortKernelTime), ctypes.c_uint32,
                                          ctypes.POINTER(ctypes.c_uint32)], st),
            "fsort_plan_device_flags": ([vp], ctypes.c_uint32),
            "fsort_plan_set_fault_hook": ([vp, ctypes.c_uint32, ctypes.c_uint64], st),
            "fsort_scatter_pass_noalloc": ([vp, vp, vp, vp, u64, i32, i32, i32, vp], st),
            "fsort_sort_batch": ([vp, ctypes.POINTER(FsortSegment), ctypes.c_uint32, i32, i32, vp], st),
            "fsort_batch_set_config": ([vp, ctypes.POINTER(FsortBatchConfig)], st),
            "fsort_batch_get_config": ([vp, ctypes.POINTER(FsortBatchConfig)], st),
            "fsort_batch_autotune": ([vp, ctypes.POINTER(FsortSegment), ctypes.c_uint32, i32, i32, vp,
                                      ctypes.POINTER(FsortBatchConfig), ctypes.POINTER(ctypes.c_float)], st),
            "fsort_learned_fit": ([vp, vp, u64, ctypes.POINTER(FsortLearnedOpts), vp], st),
            "fsort_learned_fit_ecdf": ([vp, vp, u64, ctypes.POINTER(FsortLearnedOpts), vp], st),
            "fsort_learned_get_stats": ([vp, ctypes.POINTER(FsortLearnedStats)], st),
            "fsort_learned_get_model": ([vp, vp, vp, vp, ctypes.POINTER(ctypes.c_uint32), vp], st),
            "fsort_learned_bucket_ids": ([vp, vp, u64, vp, vp], st),
            "fsort_learned_set_model": ([vp, vp, vp, vp, ctypes.c_uint32, vp, vp], st),
            "fsort_mlp_forward": ([vp, vp, ctypes.c_uint32, vp, vp], st),
            "fsort_mlp_grad": ([vp, vp, vp, ctypes.c_uint32, vp, vp, vp], st),
            "fsort_serve_create": ([ctypes.POINTER(FsortServeDesc), ctypes.POINTER(vp)], st),
            "fsort_serve_destroy": ([vp], st),
            "fsort_serve_submit": ([vp, ctypes.POINTER(FsortRequest), ctypes.POINTER(ctypes.c_uint64)], st),
            "fsort_serve_poll": ([vp, ctypes.c_uint64, ctypes.POINTER(FsortResult)], st),
            "fsort_serve_wait": ([vp, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(FsortResult)], st),
            "fsort_serve_stats_get": ([vp, ctypes.POINTER(FsortServeStats)], st),
            "fsort_serve_set_model": ([vp, vp], st),
            "fsort_hist_create": ([i32, i32, ctypes.POINTER(vp)], st),
            "fsort_hist_destroy": ([vp], st),
            "fsort_hist_reset": ([vp, vp], st),
            "fsort_hist_accumulate": ([vp, vp, u64, vp], st),
            "fsort_hist_total": ([vp, ctypes.POINTER(ctypes.c_uint64)], st),
            "fsort_hist_counts": ([vp, vp, vp], st),
            "fsort_hist_rank": ([vp, vp, u64, vp, vp], st),
            "fsort_hist_select": ([vp, vp, u64, vp, vp], st),
            "fsort_hist_expand": ([vp, vp, u64, vp], st),
            "fsort_status_string": ([i32], ctypes.c_char_p),
            "fsort_version": ([], i32),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


# ---- marshalling helpers ------------------------------------------------------

def _ptr(x) -> int | None:
    """Device (or host) address of a torch tensor, numpy array or int; None -> NULL.

    The library reads every array as dense elements from its address, so a
    strided view (``keys[::2]``, a column of a row-major matrix) is refused:
    passing its address would sort the wrong elements without an error."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor is not contiguous; pass .contiguous() or a dense copy")
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array is not C-contiguous; pass np.ascontiguousarray(...)")
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x).__name__}")


def _stream(stream) -> int | None:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(status: int, where: str) -> None:
    if status != 0:
        raise FsortError(status, where)


_BITS = {"torch.uint16": 16, "torch.uint32": 32, "torch.uint64": 64, "torch.int16": 16, "torch.int32": 32,
         "torch.int64": 64, "uint16": 16, "uint32": 32, "uint64": 64}


def _key_bits_of(t, key_bits):
    if key_bits is not None:
        return key_bits
    kb = _BITS.get(str(getattr(t, "dtype", "")))
    if kb is None:
        raise TypeError("key_bits not given and not inferable from the key array's dtype")
    return kb


def _numel(t, n):
    if n is not None:
        return n
    if hasattr(t, "numel"):
        return int(t.numel())
    if hasattr(t, "size"):
        return int(t.size)
    raise TypeError("n not given and not inferable")


# ---- C ABI, same names -----------------------------------------------------------

def fsort_plan_create(max_n: int, key_bits: int, has_values: bool = True, digit_bits: int = 0, flags: int = 0,
                      max_segments: int = 0):
    lib = load_library()
    desc = FsortPlanDesc(max_n=max_n, key_bits=key_bits, has_values=int(bool(has_values)), digit_bits=digit_bits,
                         flags=flags, max_segments=max_segments)
    h = ctypes.c_void_p()
    _check(lib.fsort_plan_create(ctypes.byref(desc), ctypes.byref(h)), "fsort_plan_create")
    return h.value


def fsort_plan_destroy(plan) -> None:
    _check(load_library().fsort_plan_destroy(plan), "fsort_plan_destroy")


def fsort_plan_sync(plan) -> None:
    lib = load_library()
    st = lib.fsort_plan_sync(plan)
    if st != 0:
        raise FsortError(st, f"fsort_plan_sync (device flags {lib.fsort_plan_device_flags(plan):#x})")


def fsort_plan_device_flags(plan) -> int:
    return int(load_library().fsort_plan_device_flags(plan))


def fsort_plan_set_fault_hook(plan, withhold_tile: int, wait_limit_ns: int = 0) -> None:
    """Failure-detection test hook: chained-form scatter tile `withhold_tile`
    never publishes its look-back words (0xFFFFFFFF removes the hook); device
    waits of the plan give up after wait_limit_ns (0: the default bound)."""
    _check(load_library().fsort_plan_set_fault_hook(plan, withhold_tile & 0xFFFFFFFF, int(wait_limit_ns)),
           "fsort_plan_set_fault_hook")


def fsort_plan_describe(plan, n: int, key_bits: int, precision_bits: int, has_values: bool) -> dict:
    info = FsortPlanInfo()
    _check(load_library().fsort_plan_describe(plan, n, key_bits, precision_bits, int(bool(has_values)),
                                              ctypes.byref(info)), "fsort_plan_describe")
    return info.as_dict()


def fsort_sort_pairs(plan, keys, vals=None, n=None, key_bits=None, precision_bits=None, stream=None) -> None:
    kb = _key_bits_of(keys, key_bits)
    _check(load_library().fsort_sort_pairs(plan, _ptr(keys), _ptr(vals), _numel(keys, n), kb,
                                           kb if precision_bits is None else precision_bits, _stream(stream)),
           "fsort_sort_pairs")


def fsort_sort_pairs_out(plan, keys_in, vals_in, keys_out, vals_out, n=None, key_bits=None, precision_bits=None,
                         stream=None) -> None:
    kb = _key_bits_of(keys_in, key_bits)
    _check(load_library().fsort_sort_pairs_out(plan, _ptr(keys_in), _ptr(vals_in), _ptr(keys_out), _ptr(vals_out),
                                               _numel(keys_in, n), kb, kb if precision_bits is None else precision_bits,
                                               _stream(stream)), "fsort_sort_pairs_out")


def fsort_sort_pairs_host(plan, keys_host, vals_host=None, n=None, key_bits=None, precision_bits=None,
                          stream=None) -> None:
    kb = _key_bits_of(keys_host, key_bits)
    _check(load_library().fsort_sort_pairs_host(plan, _ptr(keys_host), _ptr(vals_host), _numel(keys_host, n), kb,
                                                kb if precision_bits is None else precision_bits, _stream(stream)),
           "fsort_sort_pairs_host")


def fsort_histogram(plan, keys, counts_out, n=None, key_bits=None, precision_bits=None, digit_bits=8,
                    stream=None) -> None:
    kb = _key_bits_of(keys, key_bits)
    _check(load_library().fsort_histogram(plan, _ptr(keys), _numel(keys, n), kb,
                                          kb if precision_bits is None else precision_bits, digit_bits,
                                          _ptr(counts_out), _stream(stream)), "fsort_histogram")


def fsort_exclusive_scan(plan, counts, rows: int, bins: int, offsets_out, stream=None) -> None:
    _check(load_library().fsort_exclusive_scan(plan, _ptr(counts), rows, bins, _ptr(offsets_out), _stream(stream)),
           "fsort_exclusive_scan")


def fsort_scatter_pass(plan, keys_in, vals_in, keys_out, vals_out, shift: int, width: int, n=None, key_bits=None,
                       stream=None) -> None:
    kb = _key_bits_of(keys_in, key_bits)
    _check(load_library().fsort_scatter_pass(plan, _ptr(keys_in), _ptr(vals_in), _ptr(keys_out), _ptr(vals_out),
                                             _numel(keys_in, n), kb, shift, width, _stream(stream)),
           "fsort_scatter_pass")


FSORT_NOALLOC_MAX_KEYS = 1 << 24


def fsort_scatter_pass_noalloc(keys_in, vals_in, keys_out, vals_out, shift: int, width: int, n=None, key_bits=None,
                               stream=None) -> None:
    """One stable scatter pass without any allocation: its scratch is a fixed
    device array owned by the library (for callers that cannot cudaMalloc).
    Synchronous; n <= FSORT_NOALLOC_MAX_KEYS; concurrent calls take turns."""
    kb = _key_bits_of(keys_in, key_bits)
    _check(load_library().fsort_scatter_pass_noalloc(_ptr(keys_in), _ptr(vals_in), _ptr(keys_out), _ptr(vals_out),
                                                     _numel(keys_in, n), kb, shift, width, _stream(stream)),
           "fsort_scatter_pass_noalloc")


def fsort_expand(plan, counts, keys_out, n=None, key_bits=16, stream=None) -> None:
    _check(load_library().fsort_expand(plan, _ptr(counts), _ptr(keys_out), _numel(keys_out, n), key_bits,
                                       _stream(stream)), "fsort_expand")


def fsort_plan_set_timing(plan, enable: bool) -> None:
    _check(load_library().fsort_plan_set_timing(plan, int(bool(enable))), "fsort_plan_set_timing")


def fsort_plan_timing_report(plan, capacity: int = 8192) -> list:
    """Per-launch device times of the calls recorded since timing was enabled
    (or last reported), as dicts."""
    buf = (FsortKernelTime * capacity)()
    count = ctypes.c_uint32()
    _check(load_library().fsort_plan_timing_report(plan, buf, capacity, ctypes.byref(count)),
           "fsort_plan_timing_report")
    return [{"kind": KERNEL_KINDS.get(r.kind, r.kind), "pass": r.pass_, "active": bool(r.active), "call": r.call,
             "n": r.n, "ms": r.ms} for r in buf[:count.value]]


def _segments(segments):
    """List of (keys, vals, n) (tensors or device addresses; vals may be None;
    n may be None for tensors) -> ctypes array."""
    arr = (FsortSegment * max(1, len(segments)))()
    for i, seg in enumerate(segments):
        keys, vals = seg[0], seg[1]
        n = seg[2] if len(seg) > 2 and seg[2] is not None else _numel(keys, None)
        arr[i] = FsortSegment(_ptr(keys), _ptr(vals), n)
    return arr


def fsort_sort_batch(plan, segments, key_bits: int, precision_bits=None, stream=None) -> None:
    arr = _segments(segments)
    _check(load_library().fsort_sort_batch(plan, arr, len(segments), key_bits,
                                           key_bits if precision_bits is None else precision_bits, _stream(stream)),
           "fsort_sort_batch")


def fsort_batch_set_config(plan, small_capacity: int, small_ctas_per_sm: int, large_form: int = 1,
                           digit_bits: int = 8) -> None:
    """large_form: 1 = the larger segments' passes scatter from a table of per-tile offsets, 0 = chained;
    digit_bits: width of the batch's radix digits (8, or 7 / 6 for 16- and 32-bit keys)."""
    cfg = FsortBatchConfig(small_capacity=small_capacity, small_ctas_per_sm=small_ctas_per_sm, large_form=large_form,
                           digit_bits=digit_bits)
    _check(load_library().fsort_batch_set_config(plan, ctypes.byref(cfg)), "fsort_batch_set_config")


def fsort_batch_get_config(plan) -> dict:
    cfg = FsortBatchConfig()
    _check(load_library().fsort_batch_get_config(plan, ctypes.byref(cfg)), "fsort_batch_get_config")
    return cfg.as_dict()


def fsort_batch_autotune(plan, segments, key_bits: int, precision_bits=None, stream=None):
    """Returns (best config dict, its time in ms)."""
    arr = _segments(segments)
    cfg = FsortBatchConfig()
    ms = ctypes.c_float()
    _check(load_library().fsort_batch_autotune(plan, arr, len(segments), key_bits,
                                               key_bits if precision_bits is None else precision_bits,
                                               _stream(stream), ctypes.byref(cfg), ctypes.byref(ms)),
           "fsort_batch_autotune")
    return cfg.as_dict(), ms.value


def fsort_learned_fit(plan, keys, n=None, sample_keys: int = 0, steps: int = 0, batch: int = 0, lr: float = 0.0,
                      seed: int = 0, stream=None) -> None:
    o = FsortLearnedOpts(sample_keys, steps, batch, lr, seed)
    _check(load_library().fsort_learned_fit(plan, _ptr(keys), _numel(keys, n), ctypes.byref(o), _stream(stream)),
           "fsort_learned_fit")


def fsort_learned_fit_ecdf(plan, keys, n=None, sample_keys: int = 0, seed: int = 0, stream=None) -> None:
    """Model-free map from the sorted sample's empirical CDF (no training)."""
    o = FsortLearnedOpts(sample_keys, 0, 0, 0.0, seed)
    _check(load_library().fsort_learned_fit_ecdf(plan, _ptr(keys), _numel(keys, n), ctypes.byref(o), _stream(stream)),
           "fsort_learned_fit_ecdf")


def fsort_learned_get_stats(plan) -> dict:
    out = FsortLearnedStats()
    _check(load_library().fsort_learned_get_stats(plan, ctypes.byref(out)), "fsort_learned_get_stats")
    return out.as_dict()


def fsort_learned_get_model(plan) -> dict:
    """The fitted model as numpy arrays: params (FP32), cells (G, H) pairs,
    frequent keys, and the feature normalisation (center, half)."""
    import numpy as np
    params = np.zeros(FSORT_MLP_PARAMS, np.float32)
    cells = np.zeros((FSORT_LEARN_CELLS + 1, 2), np.uint32)
    heavy = np.zeros(FSORT_LEARN_MAX_HEAVY, np.uint64)
    norm = np.zeros(2, np.float32)
    m = ctypes.c_uint32(0)
    _check(load_library().fsort_learned_get_model(plan, params.ctypes.data, cells.ctypes.data, heavy.ctypes.data,
                                                  ctypes.byref(m), norm.ctypes.data), "fsort_learned_get_model")
    return {"params": params, "cells": cells, "heavy": heavy[:m.value].copy(), "center": float(norm[0]),
            "half": float(norm[1])}


def fsort_learned_set_model(plan, params=None, cells=None, heavy=None, center: float = 0.0, half: float = 1.0,
                            stream=None) -> None:
    """Install a model: numpy float32 params[4353] and/or uint32 cells[(56321, 2)],
    uint64 heavy keys ascending, and the feature normalisation."""
    import numpy as np
    p = None if params is None else np.ascontiguousarray(params, np.float32)
    c = None if cells is None else np.ascontiguousarray(cells, np.uint32)
    h = np.ascontiguousarray(np.zeros(0, np.uint64) if heavy is None else heavy, np.uint64)
    # the library reads exactly these many elements from the host arrays
    if p is not None and p.size != FSORT_MLP_PARAMS:
        raise ValueError(f"params must hold {FSORT_MLP_PARAMS} values, not {p.size}")
    if c is not None and c.shape != (FSORT_LEARN_CELLS + 1, 2):
        raise ValueError(f"cells must have shape ({FSORT_LEARN_CELLS + 1}, 2), not {c.shape}")
    if h.ndim != 1 or h.size > FSORT_LEARN_MAX_HEAVY:
        raise ValueError(f"heavy must be 1-D with at most {FSORT_LEARN_MAX_HEAVY} keys")
    norm = np.array([center, half], np.float32)
    _check(load_library().fsort_learned_set_model(plan, None if p is None else p.ctypes.data,
                                                  None if c is None else c.ctypes.data,
                                                  h.ctypes.data if h.size else None, h.size, norm.ctypes.data,
                                                  _stream(stream)), "fsort_learned_set_model")


def fsort_learned_bucket_ids(plan, keys, ids, n=None, stream=None) -> None:
    _check(load_library().fsort_learned_bucket_ids(plan, _ptr(keys), _numel(keys, n), _ptr(ids), _stream(stream)),
           "fsort_learned_bucket_ids")


def fsort_mlp_forward(w_bf16, x, out, m=None, stream=None) -> None:
    _check(load_library().fsort_mlp_forward(_ptr(w_bf16), _ptr(x), _numel(x, m), _ptr(out), _stream(stream)),
           "fsort_mlp_forward")


def fsort_mlp_grad(w_bf16, x, y, grads, loss=None, m=None, stream=None) -> None:
    _check(load_library().fsort_mlp_grad(_ptr(w_bf16), _ptr(x), _ptr(y), _numel(x, m), _ptr(grads), _ptr(loss),
                                         _stream(stream)), "fsort_mlp_grad")


def fsort_serve_create(max_request_keys: int, key_bits: int, has_values: bool = True, hbm_budget_bytes: int = 0,
                       lanes: int = 0, max_queue: int = 0, batch_keys: int = 0, max_batch: int = 0, flags: int = 0):
    d = FsortServeDesc(max_request_keys, hbm_budget_bytes, key_bits, int(bool(has_values)), lanes, max_queue,
                       batch_keys, max_batch, flags, 0)
    h = ctypes.c_void_p()
    _check(load_library().fsort_serve_create(ctypes.byref(d), ctypes.byref(h)), "fsort_serve_create")
    return h.value


def fsort_serve_destroy(server) -> None:
    _check(load_library().fsort_serve_destroy(server), "fsort_serve_destroy")


def fsort_serve_submit(server, keys_host, vals_host=None, keys_out_host=None, vals_out_host=None, n=None,
                       precision_bits=None, key_bits=None) -> int:
    """Queue a sort of host arrays (numpy or pinned torch tensors); the
    result lands in keys_out_host/vals_out_host (default: in place)."""
    kb = _key_bits_of(keys_host, key_bits)
    r = FsortRequest(_ptr(keys_host), _ptr(vals_host), _ptr(keys_host if keys_out_host is None else keys_out_host),
                     _ptr(vals_host if vals_out_host is None else vals_out_host), _numel(keys_host, n),
                     kb if precision_bits is None else precision_bits, 0)
    t = ctypes.c_uint64()
    _check(load_library().fsort_serve_submit(server, ctypes.byref(r), ctypes.byref(t)), "fsort_serve_submit")
    return t.value


def fsort_serve_poll(server, ticket: int):
    """The result dict once the request is done, else None."""
    out = FsortResult()
    st = load_library().fsort_serve_poll(server, ticket, ctypes.byref(out))
    if st == 6:
        return None
    _check(st, "fsort_serve_poll")
    return out.as_dict()


def fsort_serve_wait(server, ticket: int, timeout_ms: float = -1.0):
    out = FsortResult()
    st = load_library().fsort_serve_wait(server, ticket, timeout_ms, ctypes.byref(out))
    if st == 6:
        return None
    _check(st, "fsort_serve_wait")
    return out.as_dict()


def fsort_serve_stats_get(server) -> dict:
    out = FsortServeStats()
    _check(load_library().fsort_serve_stats_get(server, ctypes.byref(out)), "fsort_serve_stats_get")
    return out.as_dict()


def fsort_serve_set_model(server, plan) -> None:
    _check(load_library().fsort_serve_set_model(server, plan), "fsort_serve_set_model")


def fsort_hist_create(key_bits: int, precision_bits: int):
    h = ctypes.c_void_p()
    _check(load_library().fsort_hist_create(key_bits, precision_bits, ctypes.byref(h)), "fsort_hist_create")
    return h.value


def fsort_hist_destroy(hist) -> None:
    _check(load_library().fsort_hist_destroy(hist), "fsort_hist_destroy")


def fsort_hist_reset(hist, stream=None) -> None:
    _check(load_library().fsort_hist_reset(hist, _stream(stream)), "fsort_hist_reset")


def fsort_hist_accumulate(hist, keys, n=None, stream=None) -> None:
    _check(load_library().fsort_hist_accumulate(hist, _ptr(keys), _numel(keys, n), _stream(stream)),
           "fsort_hist_accumulate")


def fsort_hist_total(hist) -> int:
    t = ctypes.c_uint64()
    _check(load_library().fsort_hist_total(hist, ctypes.byref(t)), "fsort_hist_total")
    return t.value


def fsort_hist_counts(hist, counts_out, stream=None) -> None:
    _check(load_library().fsort_hist_counts(hist, _ptr(counts_out), _stream(stream)), "fsort_hist_counts")


def fsort_hist_rank(hist, values, ranks, count=None, stream=None) -> None:
    _check(load_library().fsort_hist_rank(hist, _ptr(values), _numel(values, count), _ptr(ranks), _stream(stream)),
           "fsort_hist_rank")


def fsort_hist_select(hist, ranks, values, count=None, stream=None) -> None:
    _check(load_library().fsort_hist_select(hist, _ptr(ranks), _numel(ranks, count), _ptr(values), _stream(stream)),
           "fsort_hist_select")


def fsort_hist_expand(hist, keys_out, n=None, stream=None) -> None:
    _check(load_library().fsort_hist_expand(hist, _ptr(keys_out), _numel(keys_out, n), _stream(stream)),
           "fsort_hist_expand")


class StreamHistogram:
    """Owns an fsort_hist handle (see the streaming-histogram section of fsort.h)."""

    def __init__(self, key_bits: int, precision_bits: int):
        self.key_bits, self.precision_bits = key_bits, precision_bits
        self.handle = fsort_hist_create(key_bits, precision_bits)

    def close(self) -> None:
        if self.handle:
            fsort_hist_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def accumulate(self, keys, stream=None) -> None:
        fsort_hist_accumulate(self.handle, keys, stream=stream)

    def total(self) -> int:
        return fsort_hist_total(self.handle)


class Server:
    """Owns an fsort_server handle (see the serving section of fsort.h)."""

    def __init__(self, max_request_keys: int, key_bits: int, has_values: bool = True, **kw):
        self.handle = fsort_serve_create(max_request_keys, key_bits, has_values, **kw)

    def close(self) -> None:
        if self.handle:
            fsort_serve_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, keys_host, vals_host=None, **kw) -> int:
        return fsort_serve_submit(self.handle, keys_host, vals_host, **kw)

    def poll(self, ticket: int):
        return fsort_serve_poll(self.handle, ticket)

    def wait(self, ticket: int, timeout_ms: float = -1.0):
        return fsort_serve_wait(self.handle, ticket, timeout_ms)

    def stats(self) -> dict:
        return fsort_serve_stats_get(self.handle)


def fsort_status_string(status: int) -> str:
    return load_library().fsort_status_string(status).decode()


def fsort_version() -> int:
    return int(load_library().fsort_version())


class Plan:
    """Owns a libfsort plan; sorts torch tensors on the current CUDA stream."""

    def __init__(self, max_n: int, key_bits: int, has_values: bool = True, digit_bits: int = 0, flags: int = 0,
                 max_segments: int = 0):
        self.key_bits = key_bits
        self.has_values = has_values
        self.handle = fsort_plan_create(max_n, key_bits, has_values, digit_bits, flags, max_segments)

    def close(self) -> None:
        if self.handle:
            fsort_plan_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sort(self, keys, vals=None, precision_bits=None, stream=None) -> None:
        fsort_sort_pairs(self.handle, keys, vals, None, self.key_bits, precision_bits, stream)

    def sort_out(self, keys_in, vals_in, keys_out, vals_out, precision_bits=None, stream=None) -> None:
        fsort_sort_pairs_out(self.handle, keys_in, vals_in, keys_out, vals_out, None, self.key_bits, precision_bits,
                             stream)

    def sync(self) -> None:
        fsort_plan_sync(self.handle)

    def sort_batch(self, segments, precision_bits=None, stream=None) -> None:
        fsort_sort_batch(self.handle, segments, self.key_bits, precision_bits, stream)

    def learned_fit(self, keys, n=None, **opts) -> None:
        fsort_learned_fit(self.handle, keys, n, **opts)

    def learned_fit_ecdf(self, keys, n=None, **opts) -> None:
        fsort_learned_fit_ecdf(self.handle, keys, n, **opts)

    def learned_stats(self) -> dict:
        return fsort_learned_get_stats(self.handle)

    def describe(self, n: int, precision_bits=None, has_values=None) -> dict:
        return fsort_plan_describe(self.handle, n, self.key_bits,
                                   self.key_bits if precision_bits is None else precision_bits,
                                   self.has_values if has_values is None else has_values)
