"""The C-ABI library loads and exports every symbol include/fsort.h declares.
No compute: only calls that return before touching the GPU."""
import ctypes
import os
import re

import pytest

import paper_2605_10390_gb300 as fs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if hdr.endswith(".h"):
            text = open(os.path.join(ROOT, "include", hdr)).read()
            names += re.findall(r"FSORT_API\s+[\w\s\*]*?\b(fsort_\w+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["fsort_plan_create", "fsort_plan_destroy", "fsort_plan_sync", "fsort_sort_pairs",
                     "fsort_sort_pairs_out", "fsort_sort_pairs_host", "fsort_histogram", "fsort_exclusive_scan",
                     "fsort_scatter_pass", "fsort_expand", "fsort_status_string"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(fs.lib_path())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    missing = [n for n in declared_functions() if not hasattr(fs, n)]
    assert not missing, missing


def test_calls_without_gpu_work():
    assert fs.fsort_status_string(0) == "FSORT_OK"
    assert fs.fsort_status_string(4) == "FSORT_ERR_TIMEOUT"
    assert fs.fsort_status_string(99) == "FSORT_UNKNOWN_STATUS"
    assert fs.fsort_version() >= 100
    lib = fs.load_library()
    assert lib.fsort_plan_create(None, None) == 1
    h = ctypes.c_void_p()
    for desc in [fs.FsortPlanDesc(max_n=0, key_bits=16, has_values=1, digit_bits=0, flags=0),
                 fs.FsortPlanDesc(max_n=10, key_bits=24, has_values=1, digit_bits=0, flags=0),
                 fs.FsortPlanDesc(max_n=10, key_bits=16, has_values=2, digit_bits=0, flags=0),
                 fs.FsortPlanDesc(max_n=10, key_bits=16, has_values=1, digit_bits=0, flags=0x100)]:
        assert lib.fsort_plan_create(ctypes.byref(desc), ctypes.byref(h)) == 1
    desc = fs.FsortPlanDesc(max_n=10, key_bits=16, has_values=1, digit_bits=5, flags=0)
    assert lib.fsort_plan_create(ctypes.byref(desc), ctypes.byref(h)) == 8
    assert lib.fsort_plan_destroy(None) == 0
    assert lib.fsort_plan_sync(None) == 1
    assert lib.fsort_sort_pairs(None, None, None, 10, 16, 16, None) == 1


def test_misaligned_model_arrays_are_refused_before_any_launch():
    # every call below has one array off its element alignment, so the host
    # check refuses it (status 1) before anything reaches a device
    lib = fs.load_library()
    w, f, odd = 0x10000, 0x20000, 0x30001  # 0x30001: not 2- or 4-byte aligned
    fwd = lib.fsort_mlp_forward
    assert fwd(ctypes.c_void_p(odd), ctypes.c_void_p(f), 8, ctypes.c_void_p(f), None) == 1
    assert fwd(ctypes.c_void_p(w), ctypes.c_void_p(f + 2), 8, ctypes.c_void_p(f), None) == 1
    assert fwd(ctypes.c_void_p(w), ctypes.c_void_p(f), 8, ctypes.c_void_p(f + 1), None) == 1
    grad = lib.fsort_mlp_grad
    for bad in range(5):
        ptrs = [w, f, f, f, f]
        ptrs[bad] = odd
        args = [ctypes.c_void_p(p) for p in ptrs]
        assert grad(args[0], args[1], args[2], 8, args[3], args[4], None) == 1, bad


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2605_10390_gb300 import _binding
    monkeypatch.setattr(_binding, "_LIB", str(tmp_path / "nope.so"))
    monkeypatch.setattr(_binding, "_lib", None)
    with pytest.raises(RuntimeError):
        _binding.load_library()


def test_strided_arrays_are_refused_before_any_call():
    """A strided view's address would be read as dense elements: the binding
    refuses it (no library call is made)."""
    import numpy as np
    import torch
    from paper_2605_10390_gb300 import _binding as b
    a = np.arange(64, dtype=np.uint32)
    t = torch.arange(64, dtype=torch.int32)
    assert b._ptr(a) == a.ctypes.data and b._ptr(t) == t.data_ptr()
    assert b._ptr(a[8:16]) == a[8:].ctypes.data  # a dense slice is fine
    assert b._ptr(np.zeros((4, 3), np.uint32)) is not None
    for bad in (a[::2], np.zeros((4, 3), np.uint32)[:, 1], t[::2], torch.zeros(4, 3)[:, 1]):
        with pytest.raises(ValueError):
            b._ptr(bad)
    with pytest.raises(ValueError):  # through a public entry point: refused before the library is called
        fs.fsort_sort_pairs(None, a[::2], None, key_bits=32, precision_bits=32)


def test_model_arrays_of_the_wrong_shape_are_refused():
    """fsort_learned_set_model reads fixed-size host arrays: the binding checks
    their shapes before the library is called."""
    import numpy as np
    cells = np.zeros((fs.FSORT_LEARN_CELLS + 1, 2), np.uint32)
    bad = [dict(params=np.zeros(fs.FSORT_MLP_PARAMS - 1, np.float32)),
           dict(cells=cells[:-1]),
           dict(cells=cells.reshape(-1)),
           dict(cells=cells, heavy=np.arange(fs.FSORT_LEARN_MAX_HEAVY + 1, dtype=np.uint64))]
    for kw in bad:
        with pytest.raises(ValueError):
            fs.fsort_learned_set_model(None, **kw)
