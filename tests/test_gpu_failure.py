"""Failure detection on the GPU: a device-side wait that runs out.

A test hook makes one tile of a chained-form scatter pass withhold its
look-back publication, so the tiles after it wait for a flag that nothing
sets.  Every such wait is bounded (here to 1 ms of the device's global timer);
the first to give up sets status bit 1 and the others then give up at once.
The sort must report FSORT_ERR_TIMEOUT through fsort_plan_sync with bit 1 in
fsort_plan_device_flags, end quickly, leave the CUDA context usable, and the
next sort (hook removed, or on a new plan) must be exact.  Nothing here traps,
faults or waits without a bound.
"""
import time

import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2605_10390_gb300 as fs  # noqa: E402

TIMEOUT = 4  # FSORT_ERR_TIMEOUT
BIT_LOOKBACK_TIMEOUT = 1
BIT_OUTPUT_SKIPPED = 16


@pytest.mark.parametrize("kb,withhold", [(32, 1), (16, 2), (64, 0)])
def test_withheld_lookback_times_out_and_the_plan_recovers(kb, withhold):
    n = 6 * 8192 + 777  # several chained tiles in one look-back chunk, ragged tail
    keys = workloads.generate("uniform", n, kb, seed=5, stream=kb)
    idx = np.arange(n, dtype=np.uint32)
    want_k, want_v = oracle.sort(keys, idx, kb, kb)
    with fs.Plan(n, kb, has_values=True, flags=fs.FSORT_FLAG_CHAINED_SCATTER) as plan:
        fs.fsort_plan_set_fault_hook(plan.handle, withhold, 1_000_000)  # 1 ms bound
        dk = torch.from_numpy(keys).cuda()
        dv = torch.from_numpy(idx).cuda()
        t0 = time.monotonic()
        plan.sort(dk, dv, precision_bits=kb)
        with pytest.raises(fs.FsortError) as e:
            plan.sync()
        elapsed = time.monotonic() - t0
        assert e.value.status == TIMEOUT
        flags = fs.fsort_plan_device_flags(plan.handle)
        assert flags & BIT_LOOKBACK_TIMEOUT, hex(flags)
        assert flags & BIT_OUTPUT_SKIPPED, hex(flags)  # the tiles that gave up wrote nothing
        assert elapsed < 2.0, elapsed  # every pass ends within about one 1 ms bound, not 2 s per tile
        torch.cuda.synchronize()  # the context is still usable
        # hook removed: the same plan sorts exactly again
        fs.fsort_plan_set_fault_hook(plan.handle, 0xFFFFFFFF, 0)
        dk.copy_(torch.from_numpy(keys))
        dv.copy_(torch.from_numpy(idx))
        plan.sort(dk, dv, precision_bits=kb)
        plan.sync()
        assert np.array_equal(dk.cpu().numpy(), want_k) and np.array_equal(dv.cpu().numpy(), want_v)
    # and so does a new plan
    with fs.Plan(n, kb, has_values=True, flags=fs.FSORT_FLAG_CHAINED_SCATTER) as plan:
        dk = torch.from_numpy(keys).cuda()
        dv = torch.from_numpy(idx).cuda()
        plan.sort(dk, dv, precision_bits=kb)
        plan.sync()
        assert np.array_equal(dk.cpu().numpy(), want_k) and np.array_equal(dv.cpu().numpy(), want_v)


def test_hook_with_no_withheld_tile_changes_nothing():
    n = 3 * 8192 + 5
    keys = workloads.generate("zipf1.1", n, 32, seed=6, stream=1)
    want, _ = oracle.sort(keys, None, 32, 32)
    with fs.Plan(n, 32, has_values=False, flags=fs.FSORT_FLAG_CHAINED_SCATTER) as plan:
        fs.fsort_plan_set_fault_hook(plan.handle, 0xFFFFFFFF, 1_000_000)  # short bound, nothing withheld
        dk = torch.from_numpy(keys).cuda()
        plan.sort(dk, None, precision_bits=32)
        plan.sync()
        assert np.array_equal(dk.cpu().numpy(), want)
