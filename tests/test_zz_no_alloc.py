"""The allocation-free scatter pass gives the same result as the plan-based one.

fsort_scatter_pass_noalloc is for callers that cannot call cudaMalloc where
they sort (another component owns the device memory budget, or the path must
not take cudaMalloc's implicit synchronisation): it keeps its scratch in a
fixed device array inside the library instead of a plan.  This file is named so
that pytest collects it last; it passes alone in a fresh process and after the
other tests.  Integer data, so "within tolerance" means bit-exact.
"""
import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2605_10390_gb300 as fs  # noqa: E402


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("key_bits,with_vals", [(16, True), (32, False), (64, True)])
def test_noalloc_matches_plan_based_pass_twice(key_bits, with_vals):
    n = 3 * 8192 + 4097
    plan = fs.Plan(n, key_bits, has_values=with_vals)
    try:
        # Two calls in a row with different inputs and digits: the shared
        # scratch must come back clean between them.
        for call, (dist, shift, width) in enumerate([("zipf1.1", key_bits - 8, 8), ("uniform", 3, 5)]):
            keys = workloads.generate(dist, n, key_bits, seed=0, stream=20 + call)
            vals = (np.arange(n, dtype=np.uint32) * np.uint32(7)) if with_vals else None
            dk = _dev(keys)
            dv = _dev(vals) if with_vals else None
            ref_k = torch.empty_like(dk)
            ref_v = torch.empty_like(dv) if with_vals else None
            fs.fsort_scatter_pass(plan.handle, dk, dv, ref_k, ref_v, shift, width, key_bits=key_bits)
            plan.sync()
            got_k = torch.empty_like(dk)
            got_v = torch.empty_like(dv) if with_vals else None
            fs.fsort_scatter_pass_noalloc(dk, dv, got_k, got_v, shift, width, key_bits=key_bits)
            torch.cuda.synchronize()
            assert torch.equal(got_k, ref_k), call
            if with_vals:
                assert torch.equal(got_v, ref_v), call
    finally:
        plan.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    k = torch.empty(16, dtype=torch.uint16, device="cuda")
    with pytest.raises(fs.FsortError) as e:
        fs.fsort_scatter_pass_noalloc(k, None, torch.empty_like(k), None, 0, 8, n=fs.FSORT_NOALLOC_MAX_KEYS + 1,
                                      key_bits=16)
    assert e.value.status == 1
