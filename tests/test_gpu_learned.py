"""Learned bucket mapping on the GPU against the CPU oracle.

- the model's forward and backward kernels against the float64 oracle on the
  same BF16-rounded weights (fp32-accumulation tolerance);
- the map table a model produces on the GPU against the oracle's table;
- bucket ids of a given table: bit-exact;
- sorts through the learned path (accepted and rejected by the judge, fitted
  on the GPU or given): bit-exact with the oracle's sort;
- what the trained network gains: the learned path beats the plain path on
  the lognormal-mixture workload at identical output.
"""
import time

import numpy as np
import pytest

import oracle
import workloads
from oracle import learned as ol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2605_10390_gb300 as fs  # noqa: E402


def bf16_params(seed, scale=0.4):
    p = np.random.default_rng(seed).normal(0.0, scale, ol.PARAMS).astype(np.float32)
    return p, torch.from_numpy(p).to(torch.bfloat16).cuda()


def learned_plan(max_n):
    return fs.Plan(max_n, 64, has_values=False, flags=fs.FSORT_FLAG_LEARNED)


def mixture(n, seed=0, stream=0):
    return workloads.generate("mixture", n, 64, seed=seed, stream=stream)


def heavy_of(keys, min_count):
    u, c = np.unique(keys, return_counts=True)
    return u[c >= min_count][: fs.FSORT_LEARN_MAX_HEAVY]


def empirical_table(keys, heavy, warp=None):
    """A map table from the data's own CDF (non-heavy keys): balanced by construction,
    unless `warp` (a monotone map of [0, 1] onto itself) is applied to the CDF."""
    nh = np.sort(keys[~np.isin(keys, heavy)])
    starts = ol.cell_start(np.arange(ol.CELLS, dtype=np.uint64))
    t = np.zeros((ol.CELLS + 1, 2), np.uint32)
    frac = np.searchsorted(nh, starts, side="left") / max(nh.size, 1)
    if warp is not None:
        frac = warp(frac)
    t[:ol.CELLS, 0] = np.minimum(np.floor(frac * 2.0 ** 32), 0xFFFFFFFF).astype(np.uint64)
    t[:ol.CELLS, 1] = np.searchsorted(heavy, starts, side="left")
    t[ol.CELLS] = (0xFFFFFFFF, heavy.size)
    return t


def sort_and_check(plan, keys):
    d = torch.from_numpy(keys).cuda()
    plan.sort(d, precision_bits=64)
    plan.sync()
    want, _ = oracle.sort(keys, None, 64, 64)
    assert np.array_equal(d.cpu().numpy(), want)


# ---------------------------------------------------------------- model ----

def test_mlp_forward_matches_oracle():
    p, wb = bf16_params(1)
    x = np.random.default_rng(2).uniform(-1.5, 1.5, 4099).astype(np.float32)
    out = torch.empty(x.size, dtype=torch.float32, device="cuda")
    fs.fsort_mlp_forward(wb, torch.from_numpy(x).cuda(), out)
    torch.cuda.synchronize()
    want = ol.forward(ol.bf16_round(p), x)
    assert np.max(np.abs(out.cpu().numpy() - want)) < 1e-5


@pytest.mark.parametrize("m", [1, 63, 64, 4099])
def test_mlp_grad_matches_oracle(m):
    p, wb = bf16_params(3 + m)
    rng = np.random.default_rng(m)
    x = rng.uniform(-1.2, 1.2, m).astype(np.float32)
    y = rng.uniform(0.0, 1.0, m).astype(np.float32)
    g = torch.zeros(ol.PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    fs.fsort_mlp_grad(wb, xt, yt, g, loss)
    torch.cuda.synchronize()
    lw, gw = ol.loss_and_grad(ol.bf16_round(p), x, y)
    gg = g.cpu().numpy().astype(np.float64)
    scale = np.max(np.abs(gw))
    assert np.max(np.abs(gg - gw)) <= 1e-3 * scale + 1e-8
    assert float(loss.item()) == pytest.approx(lw, rel=1e-4)
    # the kernel accumulates into grads
    fs.fsort_mlp_grad(wb, xt, yt, g, None)
    torch.cuda.synchronize()
    assert np.max(np.abs(g.cpu().numpy() - 2 * gw)) <= 2e-3 * scale + 1e-8


def test_table_from_model_matches_oracle():
    p, _ = bf16_params(11, scale=0.3)
    heavy = np.unique(np.exp(np.random.default_rng(4).uniform(18, 44, 500)).astype(np.uint64))
    center, half = np.float32(0.6), np.float32(0.3)
    with learned_plan(1 << 16) as plan:
        fs.fsort_learned_set_model(plan.handle, params=p, heavy=heavy, center=center, half=half)
        m = fs.fsort_learned_get_model(plan.handle)
    want = ol.table(ol.bf16_round(p), heavy, float(center), float(half))
    got = m["cells"]
    assert np.array_equal(got[:, 1], want[:, 1])
    assert np.all(np.diff(got[:, 0].astype(np.int64)) >= 0) and got[-1, 0] == 0xFFFFFFFF
    assert np.max(np.abs(got[:, 0].astype(np.int64) - want[:, 0].astype(np.int64))) <= 3e-5 * 2 ** 32
    assert np.array_equal(m["heavy"], heavy)


@pytest.mark.parametrize("n", [1000, 100_003, 1 << 20])
def test_bucket_ids_of_a_given_table_are_exact(n):
    keys = mixture(n, stream=n % 7)
    heavy = heavy_of(keys, 3)
    table = ol.table(ol.bf16_round(bf16_params(5, 0.3)[0]), heavy, 0.6, 0.3)
    edge = np.array([0, 1, 2047, 2048, 2049, (1 << 63), (1 << 64) - 1], np.uint64)
    keys = np.concatenate([keys[: n - 7 - 3 * min(heavy.size, 50)], edge,
                           heavy[:50], heavy[:50] + np.uint64(1), heavy[:50] - np.uint64(1)])
    assert keys.size == n
    with learned_plan(n) as plan:
        fs.fsort_learned_set_model(plan.handle, cells=table, heavy=heavy, center=0.6, half=0.3)
        ids = torch.empty(n, dtype=torch.int32, device="cuda")
        fs.fsort_learned_bucket_ids(plan.handle, torch.from_numpy(keys).cuda(), ids)
        torch.cuda.synchronize()
    want = ol.bucket_ids(keys, table, heavy, n)
    assert np.array_equal(ids.cpu().numpy().astype(np.int64), want)


# ----------------------------------------------------------------- sorts ----

@pytest.mark.parametrize("n", [1, 2, 1000, 70_001, (1 << 20) + 77])
def test_sort_with_balanced_table_matches_oracle(n):
    keys = mixture(n, stream=3)
    heavy = heavy_of(keys, max(2, n // 4096))
    table = empirical_table(keys, heavy)
    ok, mx, limit, b = ol.judge(keys, table, heavy)
    with learned_plan(n) as plan:
        fs.fsort_learned_set_model(plan.handle, cells=table, heavy=heavy, center=0.6, half=0.3)
        sort_and_check(plan, keys)
        st = plan.learned_stats()
    assert st["used"] == (1 if ok else 0)
    assert (st["max_bucket"], st["limit"], st["buckets"]) == (mx, limit, b)
    if n >= 70_001:
        assert ok  # the data's own CDF balances the buckets


def test_buckets_above_the_narrow_unit_capacity_sort_exactly():
    """A CDF squeezed five-fold over a band of 16 bucket widths: a dozen buckets of 4,600 to
    4,750 keys, above the 4,096 keys a narrow unit holds but within the judge's limit (8 x 1,024),
    so they take the wide bucket sort while the rest are packed into narrow units."""
    n = 1 << 20
    keys = mixture(n, stream=6)
    heavy = heavy_of(keys, n // 4096)
    d = 16 / 1024
    table = empirical_table(keys, heavy, lambda f: np.interp(f, [0.0, 0.1, 0.1 + 5 * d, 1.0],
                                                             [0.0, 0.1, 0.1 + d, 1.0]))
    ok, mx, limit, b = ol.judge(keys, table, heavy)
    ids = ol.bucket_ids(keys, table, heavy, n)
    wide = int((np.bincount(ids[~np.isin(keys, heavy)]) > 4096).sum())
    assert ok and wide >= 8 and 4096 < mx <= limit
    with learned_plan(n) as plan:
        fs.fsort_learned_set_model(plan.handle, cells=table, heavy=heavy, center=0.6, half=0.3)
        sort_and_check(plan, keys)
        st = plan.learned_stats()
    assert st["used"] == 1 and (st["max_bucket"], st["limit"], st["buckets"]) == (mx, limit, b)


def test_sort_rejected_by_judge_falls_back_exactly():
    n = 300_000
    keys = mixture(n, stream=4)
    table = ol.table(ol.bf16_round(bf16_params(9, 0.3)[0]), np.zeros(0, np.uint64), 0.2, 0.05)
    ok, mx, _, _ = ol.judge(keys, table, np.zeros(0, np.uint64))
    assert not ok
    with learned_plan(n) as plan:
        fs.fsort_learned_set_model(plan.handle, cells=table, center=0.2, half=0.05)
        sort_and_check(plan, keys)
        st = plan.learned_stats()
    assert st["used"] == 0 and st["max_bucket"] == mx


def test_out_of_place_learned_sort():
    n = 200_000
    keys = mixture(n, stream=5)
    heavy = heavy_of(keys, 64)
    with learned_plan(n) as plan:
        fs.fsort_learned_set_model(plan.handle, cells=empirical_table(keys, heavy), heavy=heavy)
        src = torch.from_numpy(keys).cuda()
        dst = torch.empty_like(src)
        plan.sort_out(src, None, dst, None, precision_bits=64)
        plan.sync()
        assert plan.learned_stats()["used"] == 1
    assert np.array_equal(src.cpu().numpy(), keys)
    assert np.array_equal(dst.cpu().numpy(), oracle.sort(keys, None, 64, 64)[0])


def test_fit_on_mixture_trains_and_sorts_exactly():
    n = 1 << 22
    keys = mixture(n, stream=6)
    with learned_plan(n) as plan:
        d = torch.from_numpy(keys).cuda()
        plan.learned_fit(d, seed=1)
        st = plan.learned_stats()
        assert st["fitted"] == 1 and st["sample_keys"] == n and st["heavy_keys"] > 0
        assert st["train_keys"] + st["heavy_keys"] <= n
        assert st["loss_last"] < 0.2 * st["loss_first"]
        sort_and_check(plan, keys)
        st = plan.learned_stats()
        assert st["used"] == 1, st
        # a fresh draw of the same distribution: the model carries over
        sort_and_check(plan, mixture(n, seed=1, stream=6))
        assert plan.learned_stats()["used"] == 1
        # a different distribution: the judge rejects, the plain path sorts
        uni = workloads.generate("uniform", n, 64, seed=2)
        sort_and_check(plan, uni)
        assert plan.learned_stats()["used"] == 0


def test_fit_on_equal_keys():
    n = 100_000
    keys = np.full(n, 0xA5A5A5A5A5A5A5A5, np.uint64)
    with learned_plan(n) as plan:
        plan.learned_fit(torch.from_numpy(keys).cuda(), steps=20)
        st = plan.learned_stats()
        assert st["heavy_keys"] == 1 and st["train_keys"] == 0
        sort_and_check(plan, keys)
        assert plan.learned_stats()["used"] == 1  # every key in its heavy bucket
        for m in (1, 2, 3, 999):
            sort_and_check(plan, mixture(m, stream=m))


def test_values_or_reduced_precision_take_the_plain_path():
    n = 50_000
    keys = mixture(n, stream=8)
    with fs.Plan(n, 64, has_values=True, flags=fs.FSORT_FLAG_LEARNED) as plan:
        heavy = heavy_of(keys, 16)
        fs.fsort_learned_set_model(plan.handle, cells=empirical_table(keys, heavy), heavy=heavy)
        vals = np.arange(n, dtype=np.uint32)
        dk, dv = torch.from_numpy(keys).cuda(), torch.from_numpy(vals).cuda()
        plan.sort(dk, dv, precision_bits=64)
        plan.sync()
        wk, wv = oracle.sort(keys, vals, 64, 64)
        assert np.array_equal(dk.cpu().numpy(), wk) and np.array_equal(dv.cpu().numpy(), wv)
        assert plan.learned_stats()["used"] == -1  # never judged
        dk = torch.from_numpy(keys).cuda()
        plan.sort(dk, None, precision_bits=40)
        plan.sync()
        assert np.array_equal(dk.cpu().numpy(), oracle.sort(keys, None, 64, 40)[0])
        assert plan.learned_stats()["used"] == -1


def _time_sorts(plan, keys_dev, reps=3):
    work = torch.empty_like(keys_dev)
    ms = []
    for _ in range(reps + 1):
        work.copy_(keys_dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.sort(work, precision_bits=64)
        plan.sync()
        torch.cuda.synchronize()
        ms.append((time.perf_counter() - t0) * 1e3)
    return min(ms[1:]), work


def mixture_device(n, seed=0, stream=9):
    quant, hot, table = workloads.mixture_tables(0)
    t = [torch.from_numpy(a.view(np.int64)).cuda() for a in (table, quant, hot)]
    d = torch.empty(n, dtype=torch.int64, device="cuda")
    workloads.generate_device("mixture", d.data_ptr(), n, 64, seed, stream,
                              cuda_stream=torch.cuda.current_stream().cuda_stream,
                              table_dev_ptr=tuple(x.data_ptr() for x in t))
    torch.cuda.synchronize()
    return d.view(torch.uint64)


def test_learned_beats_plain_on_the_mixture():
    """What the trained network gains: on 2^28 keys of the lognormal mixture
    the judged learned path is faster than the plain radix path, with the
    identical output (the learned path's parity with the oracle is covered
    above; here the two GPU paths must agree bit for bit, and sampled output
    positions are checked against the definition of the sorted order)."""
    n = 1 << 28
    d = mixture_device(n)
    with learned_plan(n) as lp, fs.Plan(n, 64, has_values=False) as pp:
        lp.learned_fit(d, seed=3)
        t_learned, out_l = _time_sorts(lp, d)
        st = lp.learned_stats()
        assert st["used"] == 1, st
        t_plain, out_p = _time_sorts(pp, d)
    assert torch.equal(out_l, out_p)
    # sampled positions against the definition of the sorted multiset:
    # out[i] = v iff #{keys < v} <= i < #{keys <= v}
    keys = d.cpu().numpy()
    out = out_l.cpu().numpy()
    for i in np.random.default_rng(5).integers(0, n, 12).tolist() + [0, n - 1]:
        v = out[i]
        below = int(np.count_nonzero(keys < v))
        assert below <= i < below + int(np.count_nonzero(keys == v)), i
    print(f"learned {t_learned:.2f} ms  plain {t_plain:.2f} ms  ({t_plain / t_learned:.2f}x) imbalance "
          f"{st['imbalance']:.2f}")
    assert t_learned < t_plain


def test_network_against_the_model_free_table():
    """Ablation: the same partition with the map tabulated from the sorted
    sample's empirical CDF instead of the trained network (same sample, same
    frequent keys, same floor and judge).  Both judged sorts must be exact;
    the judge's largest bucket and the time of each are reported, so what the
    network itself adds is measured (bench.py reports the same at 2^30)."""
    n = 1 << 24
    d = mixture_device(n, stream=12)
    fresh = mixture(1 << 20, stream=13)
    with learned_plan(n) as lp, learned_plan(n) as ep:
        lp.learned_fit(d, seed=3)
        ep.learned_fit_ecdf(d, seed=3)
        for plan in (lp, ep):
            sort_and_check(plan, fresh)  # exact on keys the map was not fitted on
        t_net, out_n = _time_sorts(lp, d)
        st_net = lp.learned_stats()
        t_ecdf, out_e = _time_sorts(ep, d)
        st_ecdf = ep.learned_stats()
    assert st_net["used"] == 1 and st_ecdf["used"] == 1, (st_net, st_ecdf)
    assert st_ecdf["steps"] == 0 and st_ecdf["heavy_keys"] == st_net["heavy_keys"]
    assert torch.equal(out_n, out_e)
    print(f"network {t_net:.2f} ms (largest bucket {st_net['max_bucket']}), "
          f"empirical CDF {t_ecdf:.2f} ms (largest bucket {st_ecdf['max_bucket']})")


def test_saved_model_resumes_in_a_new_plan(tmp_path):
    """Checkpoint / resume: a model fitted once, saved to a file and installed
    in a fresh plan, makes the same judged sort as the plan that fitted it."""
    n = 1 << 20
    keys = mixture(n, stream=10)
    path = str(tmp_path / "map.fsm")
    with learned_plan(n) as plan:
        plan.learned_fit(torch.from_numpy(keys).cuda(), steps=300, seed=2)
        fs.save_plan_model(plan.handle, path)
        sort_and_check(plan, keys)
        st0 = plan.learned_stats()
    with learned_plan(n) as plan:
        fs.load_plan_model(plan.handle, path)
        assert plan.learned_stats()["fitted"] == 1
        sort_and_check(plan, keys)
        st1 = plan.learned_stats()
    assert (st1["used"], st1["buckets"], st1["max_bucket"]) == (st0["used"], st0["buckets"], st0["max_bucket"])
