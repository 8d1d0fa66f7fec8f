#!/usr/bin/env python3
"""Throughput of libfsort on the 512 MB workload, with its HBM roofline.

Workload (one step): five out-of-place stable sorts of 2^28 uint16 keys with
uint32 values (the original index) at 16-bit precision, one per seeded
distribution (uniform, Zipf s=1.1, Gaussian N(32768, 1024), 90 % presorted,
all-equal): 512 MB of keys+values per sort, 7.5 GB per step.  Inputs are
generated in HBM before timing and are far larger than L2 (1.5 GiB per sort vs
129 MB), so no L2 flush is needed.

Printed JSON line (rank 0): value = whole-job Gkeys/s (keys sorted by all ranks
/ max-over-ranks device time), plus
  roofline      the dominant kernel (the scatter pass): algorithmic bytes per
                launch (read + write of keys and values, 12 n) / its average
                CUDA-event duration over the timed region, against the measured
                HBM copy peak; traffic = DRAM bytes per launch from an ncu
                capture of the same kernel source, or null
  job_hbm       the whole step's algorithmic bytes over its time
  cpu_baseline  the CPU oracle on this machine's host cores, on a bounded sample
  e2e           the same metric end to end from pinned host buffers (copies in
                and out inside the timed region) through the request loop
                (fsort_serve_*, lanes overlapping copies in and out), with
                the synchronous single call fsort_sort_pairs_host beside it
  clocks        nvidia-smi samples taken during the timed region

--impl reference times the CPU oracle as the reference arm (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DISTS = ["uniform", "zipf1.1", "gauss", "presorted", "equal"]
LOG2N = 28
NOMINAL_HBM_GBS = 8000.0  # nominal HBM3e bandwidth of the part, for the second roofline fraction
KEY_BITS = 16
PRECISION = 16
WORKLOAD = ("512 MB: 2^28 uint16 keys + uint32 index values, stable, 16-bit precision, out of place; "
            "5 distributions per step (uniform, zipf s=1.1, gauss mu=32768 sigma=1024, 90% presorted, all-equal)")
METRIC = "Gkeys/s (16-bit keys + 32-bit values, 512 MB per sort, 5 distributions)"
SCATTER_SRC = [os.path.join(ROOT, "paper_2605_10390_gb300", "csrc", f)
               for f in ("fsort_blocks.cu", "fsort_dev.cuh", "fsort_rank.cuh")]


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="fsort", choices=["fsort", "reference"])
    ap.add_argument("--log2n", type=int, default=LOG2N, help="keys per sort (log2); the workload is 28")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the 32 GB arbitrary-precision configurations")
    ap.add_argument("--only", choices=["secondary", "expand", "batched", "learned", "serving", "serving_small"],
                    help="run one secondary section alone and print its JSON (profiling and debugging); "
                         "expand: the expand-path cases of the secondary section at --expand-log2n keys")
    ap.add_argument("--expand-log2n", type=int, default=34, help="keys of the expand-path cases (log2)")
    ap.add_argument("--reps", type=int, default=3, help="timed repetitions per case of --only sections")
    ap.add_argument("--learned-log2n", type=int, default=30, help="keys of the learned section (log2)")
    return ap.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, STREAM-style copy)"
    return 6800.0, "fallback (6.8 TB/s, earlier GB300 measurement)"


def max_over_ranks(torch, dist, values, device):
    """Element-wise maximum over the ranks of per-rank times (a step of the
    whole job ends when its slowest rank does); the values themselves on one
    rank.  Replicas only: this is the one collective, outside the data path."""
    vals = [float(v) for v in values]
    if not dist:
        return vals
    t = torch.tensor(vals, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def job_gkeys_per_s(world: int, keys_per_rank: int, seconds: float) -> float:
    """Whole-job throughput: the keys all ranks sorted over the max-over-ranks time."""
    return world * keys_per_rank / seconds / 1e9


def source_hash(paths) -> str:
    h = hashlib.sha256()
    for p in paths:
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def ncu_traffic(n, path=None):
    """DRAM bytes per scatter launch from the committed ncu summary, if it was
    taken on the current kernel source; scaled to n keys if taken smaller."""
    path = path or os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None, "no ncu capture committed"
    with open(path) as f:
        d = json.load(f).get("scatter")
    if not d or d.get("source_sha256") != source_hash(SCATTER_SRC):
        return None, "kernel changed since the ncu capture"
    return d["bytes_per_launch"] * n / d["n"], d.get("note", "")


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        return parse_clock_samples(out)


def parse_clock_samples(text: str) -> dict:
    """Summary of `nvidia-smi --query-gpu=<ClockSampler.FIELDS> --format=csv,noheader,nounits`
    rows: median SM clock, highest max clock, and every throttle reason seen
    Active in any sample.  Rows without numeric clocks ([N/A], a header) are skipped."""
    rows = [[c.strip() for c in line.split(",")] for line in text.strip().splitlines() if line.count(",") >= 8]
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for r in rows:
        try:
            sm.append(float(r[1]))
            mx.append(float(r[2]))
        except ValueError:
            continue
        for name, v in zip(names, r[5:9]):
            if v.lower() == "active":
                reasons.add(name)
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "reasons": sorted(reasons), "samples": len(sm)}


def run_e2e(fs, workloads, torch, n, rank, world, dist, kb, vb, steps):
    """The step's metric end to end from pinned host memory: every sort copies
    its keys and values in, sorts, and copies them back, inside the timed
    region.  Measured through the request loop (fsort_serve_*: several lanes,
    so one sort's copy back overlaps the next sort's copy in on the host link),
    and, for reference, through the synchronous single call
    fsort_sort_pairs_host."""
    import numpy as np
    pristine = [(torch.from_numpy(workloads.generate(d, n, KEY_BITS, seed=rank, stream=i)).pin_memory(),
                 torch.from_numpy(np.arange(n, dtype=np.uint32)).pin_memory()) for i, d in enumerate(DISTS)]
    # one output set: step k's sort of input i writes it once step k - 1's sort of input i is done
    # (five sorts later in submission order, so the lanes never wait on it)
    outs = [[(torch.empty(n, dtype=torch.uint16).pin_memory(), torch.empty(n, dtype=torch.uint32).pin_memory())
             for _ in DISTS]]
    lanes = 2  # measured best: three lanes contend for the host link and ran slower
    budget = lanes * n * (kb + vb) + (64 << 20)
    with fs.Server(n, KEY_BITS, True, lanes=lanes, hbm_budget_bytes=budget, batch_keys=1 << 16) as srv:
        def run(nsteps):
            pending = {}
            for k in range(nsteps):
                for i, (pk, pv) in enumerate(pristine):
                    if (k - 1, i) in pending:
                        r = srv.wait(pending.pop((k - 1, i)))
                        if r["status"] != 0:
                            raise RuntimeError(f"e2e request failed: {r}")
                    ok, ov = outs[0][i]
                    pending[(k, i)] = srv.submit(pk, pv, keys_out_host=ok, vals_out_host=ov, precision_bits=PRECISION)
            for t in pending.values():
                if srv.wait(t)["status"] != 0:
                    raise RuntimeError("e2e request failed")
        run(1)  # warm-up: plans, arena, page-ins
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        run(steps)
        total = time.perf_counter() - t0
    # the last step's outputs: keys non-decreasing, the same multiset as the input, values a key's own index
    sorted_ok = True
    for i, (pk, _) in enumerate(pristine):
        ok_, ov_ = outs[0][i]
        k_out, k_in = ok_.numpy(), pk.numpy()
        sorted_ok &= bool(np.all(k_out[1:] >= k_out[:-1]))
        sorted_ok &= bool(np.array_equal(np.bincount(k_out, minlength=65536), np.bincount(k_in, minlength=65536)))
        sorted_ok &= bool(np.array_equal(k_in[ov_.numpy()[:4096]], k_out[:4096]))
    # the synchronous single call, for reference
    hplan = fs.Plan(n, KEY_BITS, has_values=True, flags=fs.FSORT_FLAG_HOST_IO)
    wk = torch.empty(n, dtype=torch.uint16).pin_memory()
    wv = torch.empty(n, dtype=torch.uint32).pin_memory()
    sync_total = 0.0
    sync_steps = max(1, min(steps, 3))
    for st in range(sync_steps + 1):
        for pk, pv in pristine:
            wk.copy_(pk)
            wv.copy_(pv)
            t1 = time.perf_counter()
            fs.fsort_sort_pairs_host(hplan.handle, wk, wv, key_bits=KEY_BITS, precision_bits=PRECISION)
            if st > 0:
                sync_total += time.perf_counter() - t1
    hplan.close()
    total, sync_total = max_over_ranks(torch, dist, [total, sync_total], "cuda")
    return {"value": job_gkeys_per_s(world, steps * len(DISTS) * n, total), "unit": "Gkeys/s",
            "h2d_bytes_per_step": len(DISTS) * n * (kb + vb), "d2h_bytes_per_step": len(DISTS) * n * (kb + vb),
            "steps": steps, "output_checked": sorted_ok,
            "api": f"fsort_serve_submit / fsort_serve_wait ({lanes} lanes, pinned host buffers in and out)",
            "sync_single_call": {"value": job_gkeys_per_s(world, sync_steps * len(DISTS) * n, sync_total),
                                 "unit": "Gkeys/s",
                                 "api": "fsort_sort_pairs_host (pinned host buffers, synchronous)"},
            "host_link": "copies measured at ~211 GB/s host to device and ~194 GB/s back; ~343 GB/s both at once"}


def cpu_baseline(seconds: float = 10.0, log2n: int = 24):
    """The CPU oracle (single-threaded C) on a bounded sample of the same
    workload: 2^log2n keys of each distribution, repeated for >= `seconds`."""
    import numpy as np

    import oracle
    import workloads

    samples = [(workloads.generate(d, 1 << log2n, KEY_BITS, seed=0, stream=i),
                np.arange(1 << log2n, dtype=np.uint32)) for i, d in enumerate(DISTS)]
    oracle.sort(samples[0][0][:1000], samples[0][1][:1000], KEY_BITS, PRECISION)  # load + warm
    keys = 0
    t0 = time.perf_counter()
    while True:
        for k, v in samples:
            oracle.sort(k, v, KEY_BITS, PRECISION)
            keys += k.size
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return {"value": keys / el / 1e9, "unit": "Gkeys/s", "cores": 1, "kind": "oracle",
            "sample": f"5 distributions x 2^{log2n} keys (uint16 + uint32 index, p=16), repeated for {el:.1f} s, "
                      f"single-threaded C LSD counting sort on {os.cpu_count()} host cores (1 used)"}


def run_secondary(fs, workloads, torch, stream, peak, reps: int = 3, expand_log2n: int = 34, u64: bool = True):
    """The 32 GB arbitrary-precision configurations, keys only, out of place:
    2^34 uint16 keys at 16-bit precision (the expand path), and 2^32 uint64 keys
    at 16, 32 and 64 bits, each uniform and Zipf s=1.1 on the top 16 bits.
    expand_log2n and u64 shrink it for profiling (the expand cases alone)."""
    out = []
    cases = [(16, expand_log2n, 16, d) for d in ("uniform", "zipf1.1")]
    if u64:
        cases += [(64, 32, p, d) for p in (16, 32, 64) for d in ("uniform", "zipf1.1")]
    dtypes = {16: torch.uint16, 64: torch.uint64}
    cur = None
    for kb, log2n, p, dist in cases:
        n = 1 << log2n
        if cur is None or cur[0] != (kb, log2n, dist):
            cur = None
            torch.cuda.empty_cache()
            keys = torch.empty(n, dtype=dtypes[kb], device="cuda")
            table = workloads.table_for(dist, kb)
            tdev = torch.from_numpy(table).cuda() if table is not None else None
            workloads.generate_device(dist, keys.data_ptr(), n, kb, seed=0, stream=7,
                                      cuda_stream=stream.cuda_stream,
                                      table_dev_ptr=tdev.data_ptr() if tdev is not None else None)
            kout = torch.empty_like(keys)
            torch.cuda.synchronize()
            cur = ((kb, log2n, dist), keys, kout)
        _, keys, kout = cur
        plan = fs.Plan(n, kb, has_values=False)
        info = plan.describe(n, p, False)
        plan.sort_out(keys, None, kout, None, precision_bits=p)  # warm-up
        plan.sync()
        fs.fsort_plan_set_timing(plan.handle, True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            plan.sort_out(keys, None, kout, None, precision_bits=p)
        e1.record(stream)
        torch.cuda.synchronize()
        plan.sync()
        ms = e0.elapsed_time(e1) / reps
        recs = fs.fsort_plan_timing_report(plan.handle, 4096)
        kernels = {}
        for r in recs:
            k = r["kind"] + ("" if r["active"] else "_skipped")
            kernels.setdefault(k, 0.0)
            kernels[k] += r["ms"] / reps
        plan.close()
        alg = info["algorithmic_bytes"]
        out.append({"workload": f"2^{log2n} uint{kb} keys-only, {p}-bit precision, {dist}, out of place",
                    "gkeys_per_s": n / ms / 1e6, "ms": ms, "algorithmic_bytes": alg,
                    "achieved_gbs": alg / ms / 1e6, "frac": alg / ms / 1e6 / peak,
                    "path": "expand" if info["expand_path"] else f"{info['passes']} scatter passes",
                    "kernel_ms": kernels})
    del cur
    torch.cuda.empty_cache()
    return out


def batch_sizes(count: int = 4096, lo: int = 10, hi: int = 24, seed: int = 0):
    """Segment lengths log-uniform in [2^lo, 2^hi] (seeded)."""
    import numpy as np
    u = np.random.default_rng(seed).random(count)
    return [int(2 ** (lo + (hi - lo) * x)) for x in u]


def run_batched(fs, workloads, torch, stream, peak, reps: int = 2):
    """4096 independent uint32 key + uint32 value sorts (32-bit precision),
    lengths log-uniform 1K-16M, each segment's distribution drawn from
    uniform / Zipf s=1.1 / Gaussian: the batched path (one call, CUDA graph
    replay, autotuned) against the plain path (one fsort_sort_pairs per
    segment), same data, same exact output."""
    import numpy as np
    sizes = batch_sizes()
    dists = ["uniform", "zipf1.1", "gauss"]
    pick = np.random.default_rng(1).integers(0, 3, len(sizes))
    total = sum(sizes)
    tables = {d: (torch.from_numpy(workloads.table_for(d, 32)).cuda() if workloads.table_for(d, 32) is not None
                  else None) for d in dists}
    # every segment starts 16-byte aligned in one allocation
    starts, at = [], 0
    for n in sizes:
        starts.append(at)
        at += (n + 3) // 4 * 4
    need = at
    keys = torch.empty(need, dtype=torch.uint32, device="cuda")
    vals = torch.empty(need, dtype=torch.uint32, device="cuda")

    def regenerate():
        for i, (st, n) in enumerate(zip(starts, sizes)):
            d = dists[pick[i]]
            t = tables[d]
            workloads.generate_device(d, keys.data_ptr() + 4 * st, n, 32, seed=0, stream=i,
                                      cuda_stream=stream.cuda_stream, table_dev_ptr=t.data_ptr() if t is not None else None)
        workloads.iota_device(vals.data_ptr(), need, cuda_stream=stream.cuda_stream)
        torch.cuda.synchronize()

    segs = [(keys.data_ptr() + 4 * st, vals.data_ptr() + 4 * st, n) for st, n in zip(starts, sizes)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"workload": f"{len(sizes)} uint32 key + uint32 value sorts, 32-bit precision, lengths log-uniform "
                       f"2^10..2^24 (total {total} keys), uniform/zipf1.1/gauss per segment",
           "total_keys": total}
    # batched: autotune once on this batch, then time graph replays on fresh data
    side = torch.cuda.Stream()
    bplan = fs.Plan(need + 8 * len(sizes), 32, has_values=True, flags=fs.FSORT_FLAG_GRAPH, max_segments=len(sizes))
    regenerate()
    cfg, _ = fs.fsort_batch_autotune(bplan.handle, segs, 32, 32, stream=side)
    times = []
    for _ in range(reps + 1):
        regenerate()
        with torch.cuda.stream(side):
            e0.record(side)
            bplan.sort_batch(segs, precision_bits=32, stream=side)
            e1.record(side)
        side.synchronize()
        times.append(e0.elapsed_time(e1))
    bms = float(np.median(times[1:]))
    # the same batch at each digit width (the tuner's third coordinate), one warm-up and one timed run each
    width_ms = {}
    for width in (8, 7, 6):
        if isinstance(cfg, dict) and width == cfg.get("digit_bits"):
            width_ms[width] = bms
            continue
        fs.fsort_batch_set_config(bplan.handle, cfg["small_capacity"], cfg["small_ctas_per_sm"], cfg["large_form"],
                                  width)
        for rep in range(2):
            regenerate()
            with torch.cuda.stream(side):
                e0.record(side)
                bplan.sort_batch(segs, precision_bits=32, stream=side)
                e1.record(side)
            side.synchronize()
        width_ms[width] = e0.elapsed_time(e1)
    bplan.sync()
    bplan.close()
    # plain: one sort per segment
    pplan = fs.Plan(max(sizes), 32, has_values=True)
    times = []
    for _ in range(reps + 1):
        regenerate()
        e0.record(stream)
        for kp, vp, n in segs:
            fs.fsort_sort_pairs(pplan.handle, kp, vp, n=n, key_bits=32, precision_bits=32, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    pplan.sync()
    pplan.close()
    pms = float(np.median(times[1:]))
    alg = sum(4 * n + 4 * 2 * 8 * n for n in sizes)  # plain path's bytes: key read + 4 passes of keys+values
    # the batched path's own algorithmic bytes: segments sorted on chip move their keys and
    # values once in and once out (16 n); the others take the plain path's 68 n
    cap = int(cfg.get("small_capacity", 0)) if isinstance(cfg, dict) else 0
    balg = sum(16 * n if n <= cap else 68 * n for n in sizes)
    out.update({"batched_ms": bms, "batched_gkeys_per_s": total / bms / 1e6, "plain_ms": pms,
                "plain_gkeys_per_s": total / pms / 1e6, "speedup": pms / bms, "autotuned": cfg,
                "ms_by_digit_bits": width_ms,
                "plain_path_algorithmic_bytes": alg, "plain_path_frac": alg / pms / 1e6 / peak,
                "batched_algorithmic_bytes": balg, "batched_frac": balg / bms / 1e6 / peak})
    del keys, vals
    torch.cuda.empty_cache()
    return out


def mixture_device(workloads, torch, n: int, stream, seed: int = 0, stream_id: int = 9):
    """n uint64 keys of the lognormal mixture with Zipf s=1.3 hot keys, generated on the device."""
    import numpy as np
    quant, hot, table = workloads.mixture_tables(0)
    t = [torch.from_numpy(a.view(np.int64)).cuda() for a in (table, quant, hot)]
    d = torch.empty(n, dtype=torch.int64, device="cuda")
    workloads.generate_device("mixture", d.data_ptr(), n, 64, seed, stream_id, cuda_stream=stream.cuda_stream,
                              table_dev_ptr=tuple(x.data_ptr() for x in t))
    torch.cuda.synchronize()
    return d.view(torch.uint64)


def time_plan(fs, torch, plan, src, reps: int):
    """Median ms of in-place keys-only 64-bit sorts of fresh copies of src, and
    the per-kernel device times (library timing) averaged over the reps."""
    import numpy as np
    work = torch.empty_like(src)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times, kernels = [], {}
    for r in range(reps + 1):
        work.copy_(src)
        torch.cuda.synchronize()
        if r == 1:
            fs.fsort_plan_set_timing(plan.handle, True)
        e0.record()
        plan.sort(work, precision_bits=64)
        e1.record()
        plan.sync()
        torch.cuda.synchronize()
        if r > 0:
            times.append(e0.elapsed_time(e1))
    for rec in fs.fsort_plan_timing_report(plan.handle, 8192):
        k = rec["kind"] + ("" if rec["active"] else "_skipped")
        kernels[k] = kernels.get(k, 0.0) + rec["ms"] / reps
    fs.fsort_plan_set_timing(plan.handle, False)
    return float(np.median(times)), {k: round(v, 3) for k, v in kernels.items()}, work


def run_learned(fs, workloads, torch, stream, peak, log2n: int = 30, reps: int = 3):
    """2^30 uint64 keys (lognormal mixture + Zipf s=1.3 hot keys), keys only,
    64-bit precision: the learned path (model trained once on the GPU from a
    sample the plain sort sorted; every call judged by the exact bucket
    histogram) against the plain radix path on the same keys; outputs must be
    identical."""
    n = 1 << log2n
    src = mixture_device(workloads, torch, n, stream)
    lp = fs.Plan(n, 64, has_values=False, flags=fs.FSORT_FLAG_LEARNED)
    t0 = time.perf_counter()
    lp.learned_fit(src, seed=3)
    lp.sync()
    torch.cuda.synchronize()
    fit_s = time.perf_counter() - t0
    lms, lkern, out_l = time_plan(fs, torch, lp, src, reps)
    st = lp.learned_stats()
    # ablation: the same partition from the sorted sample's empirical CDF (no network)
    t0 = time.perf_counter()
    lp.learned_fit_ecdf(src, seed=3)
    lp.sync()
    torch.cuda.synchronize()
    ecdf_fit_s = time.perf_counter() - t0
    ems, _, out_e = time_plan(fs, torch, lp, src, reps)
    st_e = lp.learned_stats()
    same_e = bool(torch.equal(out_e, out_l))
    del out_e
    lp.close()
    out_l = out_l.clone()
    torch.cuda.empty_cache()
    pp = fs.Plan(n, 64, has_values=False)
    pms, pkern, out_p = time_plan(fs, torch, pp, src, reps)
    pp.close()
    same = bool(torch.equal(out_l, out_p))
    del src, out_l, out_p
    torch.cuda.empty_cache()
    plain_bytes = 8 * n + 8 * 16 * n
    return {"workload": f"2^{log2n} uint64 keys-only, 64-bit precision, 90% lognormal mixture (8 clusters) + "
                        f"10% Zipf s=1.3 over 65,536 hot keys",
            "learned_ms": lms, "plain_ms": pms, "learned_gkeys_per_s": n / lms / 1e6,
            "plain_gkeys_per_s": n / pms / 1e6, "speedup": pms / lms, "identical_output": same,
            "fit_s": fit_s,
            "break_even_sorts": (fit_s * 1e3 / (pms - lms)) if pms > lms else None,
            "model_free_ms": ems, "vs_model_free": ems / lms, "model_free_fit_s": ecdf_fit_s,
            "model_free": {"used": st_e["used"], "max_bucket": st_e["max_bucket"], "imbalance": st_e["imbalance"],
                           "identical_output": same_e,
                           "table": "empirical CDF of the sorted sample at the same cells, same floor and judge"},
            "judge": {k: st[k] for k in ("used", "imbalance", "tau", "buckets", "max_bucket",
                                                         "limit", "heavy_keys")},
            "training": {k: st[k] for k in ("sample_keys", "train_keys", "steps", "loss_first", "loss_last")},
            "learned_kernel_ms": lkern, "plain_kernel_ms": pkern,
            "plain_algorithmic_bytes": plain_bytes, "plain_frac": plain_bytes / pms / 1e6 / peak}


def run_serving(fs, workloads, torch, stream, requests: int = 48, lo: int = 16, hi: int = 28, util: float = 0.7,
                seed: int = 0):
    """Poisson stream of uint64 keys-only sorts (64-bit precision) of the same
    mixture, sizes log-uniform 2^16..2^28 keys, through the serving loop with
    learned lanes.  A calibration pass (requests one at a time, after one
    untimed pass) gives the mean service time; arrivals then come at ~70% of
    that service rate.  Latency is
    submit -> result in pinned host memory (copies included)."""
    import gc
    import numpy as np
    gc.collect()  # what earlier sections left in the caching allocator and pinned pools
    torch.cuda.empty_cache()
    rng = np.random.default_rng(seed)
    sizes = [int(2 ** (lo + (hi - lo) * u)) for u in rng.random(requests)]
    maxn = 1 << hi
    pool = torch.from_numpy(workloads.generate("mixture", maxn, 64, seed=1, stream=11)).pin_memory()
    ring = 6
    outs = [torch.empty(maxn, dtype=torch.uint64).pin_memory() for _ in range(ring)]
    offs = [int(rng.integers(0, maxn - n + 1)) for n in sizes]
    plan = fs.Plan(1 << 26, 64, has_values=False, flags=fs.FSORT_FLAG_LEARNED)
    plan.learned_fit(pool[: 1 << 26].cuda(), seed=4)
    plan.sync()
    lanes = 3
    budget = 3 * maxn * 8 + (64 << 20)
    srv = fs.Server(maxn, 64, False, lanes=lanes, hbm_budget_bytes=budget, flags=fs.FSORT_FLAG_LEARNED)
    fs.fsort_serve_set_model(srv.handle, plan.handle)
    plan.close()
    torch.cuda.empty_cache()

    def submit(i, slot):
        n, o = sizes[i], offs[i]
        return srv.submit(pool[o:o + n], keys_out_host=outs[slot][:n], n=n, key_bits=64, precision_bits=64)

    cal = list(range(min(8, requests)))
    for j, i in enumerate(cal):  # untimed: first use of every lane's kernels and buffers
        srv.wait(submit(i, j % ring))
    t0 = time.perf_counter()
    for j, i in enumerate(cal):
        srv.wait(submit(i, j % ring))
    per_key = (time.perf_counter() - t0) / sum(sizes[i] for i in cal)
    rate = util / (per_key * float(np.mean(sizes)))
    gaps = rng.exponential(1.0 / rate, requests)
    tickets, results = [], {}
    start = time.perf_counter()
    at = 0.0
    for i in range(requests):
        at += float(gaps[i])
        if i >= ring:  # the output slot must be free again
            results[i - ring] = srv.wait(tickets[i - ring])
        delay = start + at - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        tickets.append(submit(i, i % ring))
    for i in range(max(0, requests - ring), requests):
        results[i] = srv.wait(tickets[i])
    span = time.perf_counter() - start
    st = srv.stats()
    srv.close()
    ok = all(bool(np.all(np.diff(outs[i % ring][:sizes[i]].numpy()[:: max(1, sizes[i] // 65536)]
                                  .astype(np.float64)) >= 0)) for i in range(max(0, requests - ring), requests))
    lat = sorted(r["latency_ms"] for r in results.values())
    rank = lambda p: lat[max(0, min(len(lat), int(np.ceil(p * len(lat)))) - 1)]  # nearest rank
    del pool, outs
    return {"workload": f"{requests} requests, uint64 keys-only 64-bit sorts of the mixture, sizes log-uniform "
                        f"2^{lo}..2^{hi} (total {sum(sizes)} keys), Poisson arrivals at {rate:.1f}/s "
                        f"(~{int(util * 100)}% of the calibrated service rate)",
            "requests": requests, "lanes": lanes, "hbm_budget_bytes": budget, "p50_ms": rank(0.50), "p99_ms": rank(0.99),
            "mean_ms": float(np.mean(lat)), "max_ms": lat[-1], "keys_per_s": sum(sizes) / span, "span_s": span,
            "queue_ms_mean": float(np.mean([r["queue_ms"] for r in results.values()])),
            # where the tail's time went: the slowest requests split into waiting for a lane and running
            # (copies in, sort, copies out), and the running time per key by size
            "slowest": [{"n": int(r["n"]), "latency_ms": r["latency_ms"], "queue_ms": r["queue_ms"],
                         "run_ms": r["run_ms"], "run_ns_per_key": 1e6 * r["run_ms"] / max(1, int(r["n"]))}
                        for r in sorted(results.values(), key=lambda r: -r["latency_ms"])[:3]],
            "run_ns_per_key_by_size": {f"2^{b}..2^{b + 4}": float(np.median(v)) for b, v in (
                (b, [1e6 * r["run_ms"] / int(r["n"]) for r in results.values()
                     if b <= np.log2(max(1, int(r["n"]))) < b + 4]) for b in range(lo, hi, 4)) if v},
            "batched_requests": sum(1 for r in results.values() if r["batched"]),
            "max_inflight": st["max_inflight"], "peak_bytes": st["peak_bytes"], "outputs_sorted": ok,
            "api": "fsort_serve_submit / fsort_serve_wait (pinned host buffers; copies in the latency)"}


def run_serving_small(fs, workloads, torch, requests: int = 1024, lo: int = 10, hi: int = 16, load: float = 4.0,
                      seed: int = 1, lanes: int = 2):
    """Many small requests (uint64 keys-only 64-bit sorts of the mixture, sizes
    log-uniform 2^10..2^16 keys) arriving as a Poisson stream at `load` times the
    rate the loop serves them one at a time (calibrated first, one request in
    flight): the queue holds several requests whenever a lane frees up, and the
    loop must batch them to keep up.  Reports the share of requests served in
    batches and the latency against the single-request service time."""
    import numpy as np
    rng = np.random.default_rng(seed)
    sizes = [int(2 ** (lo + (hi - lo) * u)) for u in rng.random(requests)]
    maxn = 1 << hi
    pool = torch.from_numpy(workloads.generate("mixture", 1 << 22, 64, seed=2, stream=11)).pin_memory()
    ring = 256
    outs = [torch.empty(maxn, dtype=torch.uint64).pin_memory() for _ in range(ring)]
    offs = [int(rng.integers(0, pool.numel() - n + 1)) for n in sizes]
    srv = fs.Server(maxn, 64, False, lanes=lanes, hbm_budget_bytes=64 << 20, batch_keys=maxn, max_batch=64)

    def submit(i, slot):
        n, o = sizes[i], offs[i]
        return srv.submit(pool[o:o + n], keys_out_host=outs[slot][:n], n=n, key_bits=64, precision_bits=64)

    cal = list(range(64))
    for j, i in enumerate(cal):  # untimed: every lane's kernels and buffers in use once
        srv.wait(submit(i, j % ring))
    t0 = time.perf_counter()
    for j, i in enumerate(cal):
        srv.wait(submit(i, j % ring))
    service_ms = (time.perf_counter() - t0) * 1e3 / len(cal)
    rate = load * 1e3 / service_ms
    gaps = rng.exponential(1.0 / rate, requests)
    tickets, results = [], {}
    start = time.perf_counter()
    at = 0.0
    for i in range(requests):
        at += float(gaps[i])
        if i >= ring:
            results[i - ring] = srv.wait(tickets[i - ring])
        delay = start + at - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        tickets.append(submit(i, i % ring))
    for i in range(max(0, requests - ring), requests):
        results[i] = srv.wait(tickets[i])
    span = time.perf_counter() - start
    st = srv.stats()
    srv.close()
    ok = all(bool(np.all(np.diff(outs[i % ring][:sizes[i]].numpy().astype(np.float64)) >= 0))
             for i in range(max(0, requests - ring), requests))
    lat = sorted(r["latency_ms"] for r in results.values())
    rank = lambda q: lat[max(0, min(len(lat), int(np.ceil(q * len(lat)))) - 1)]  # nearest rank
    batched = sum(1 for r in results.values() if r["batched"])
    del pool, outs
    return {"workload": f"{requests} requests, uint64 keys-only 64-bit sorts of the mixture, sizes log-uniform "
                        f"2^{lo}..2^{hi} (total {sum(sizes)} keys), Poisson arrivals at {rate:.0f}/s "
                        f"({load:.1f}x the one-at-a-time service rate)",
            "requests": requests, "lanes": lanes, "single_request_service_ms": service_ms,
            "p50_ms": rank(0.50), "p99_ms": rank(0.99), "p99_over_service": rank(0.99) / service_ms,
            "mean_ms": float(np.mean(lat)), "batched_requests": batched, "batched_share": batched / requests,
            "batches": st.get("batches"), "keys_per_s": sum(sizes) / span, "requests_per_s": requests / span,
            "outputs_sorted": ok,
            "api": "fsort_serve_submit / fsort_serve_wait (pinned host buffers; copies in the latency)"}


def summary(result: dict) -> dict:
    """The headline and every secondary section in a few hundred characters,
    placed last on the JSON line so that a reader that keeps only its tail
    still has them."""
    r = lambda x, d=3: None if x is None else round(float(x), d)
    out = {"gkeys_per_s": r(result["value"], 2), "scatter_frac": r(result["roofline"]["frac"])}
    sec = result.get("secondary") or []
    if sec:
        out["gb32"] = {f"{'u16e' if 'uint16' in c['workload'] else 'u64'}"
                       f"{'' if 'uint16' in c['workload'] else '-p' + c['workload'].split('-bit')[0].split()[-1]}"
                       f"-{'zipf' if 'zipf' in c['workload'] else 'unif'}": [r(c["gkeys_per_s"], 1), r(c["frac"])]
                       for c in sec}
    b = result.get("batched")
    if b:
        out["batched"] = {"ms": r(b["batched_ms"], 1), "speedup": r(b["speedup"], 2), "frac": r(b.get("batched_frac")),
                          "cfg": b.get("autotuned")}
    lr = result.get("learned")
    if lr:
        out["learned"] = {"ms": r(lr["learned_ms"], 2), "plain_ms": r(lr["plain_ms"], 2), "speedup": r(lr["speedup"], 2),
                          "fit_s": r(lr["fit_s"], 2), "break_even": r(lr.get("break_even_sorts"), 1),
                          "identical": lr["identical_output"]}
        for k in ("model_free_ms", "vs_model_free"):
            if k in lr:
                out["learned"][k] = r(lr[k], 3)
    sv = result.get("serving")
    if sv:
        out["serving"] = {"p50_ms": r(sv["p50_ms"], 1), "p99_ms": r(sv["p99_ms"], 1),
                          "batched": sv["batched_requests"], "requests": sv.get("requests"),
                          "gkeys_per_s": r(sv["keys_per_s"] / 1e9, 2)}
    ss = result.get("serving_small")
    if ss:
        out["serving_small"] = {"p50_ms": r(ss["p50_ms"], 2), "p99_ms": r(ss["p99_ms"], 2),
                                "service_ms": r(ss["single_request_service_ms"], 2),
                                "batched_share": r(ss["batched_share"], 2), "requests": ss["requests"]}
    return out


def run_reference(args, rank: int):
    """Reference arm: the CPU oracle, timed per step on a bounded sample."""
    if rank != 0:
        return
    import numpy as np

    import oracle
    import workloads

    total_steps = args.steps + args.warmup
    log2n = 26
    while log2n > 18 and total_steps * 5 * (1 << log2n) * 9e-9 > 120:  # keep the run to about two minutes
        log2n -= 1
    n = 1 << log2n
    samples = [(workloads.generate(d, n, KEY_BITS, seed=0, stream=i), np.arange(n, dtype=np.uint32))
               for i, d in enumerate(DISTS)]
    for _ in range(args.warmup):
        for k, v in samples:
            oracle.sort(k, v, KEY_BITS, PRECISION)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for k, v in samples:
            oracle.sort(k, v, KEY_BITS, PRECISION)
    el = time.perf_counter() - t0
    value = args.steps * 5 * n / el / 1e9
    sample = f"each step: 5 distributions x 2^{log2n} keys (bounded sample of the 2^28-key workload)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Gkeys/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u16", "data": "synthetic",
            "config": {"workload": WORKLOAD, "reference": "CPU oracle (single-threaded C LSD counting sort)",
                       "sample": sample},
            "cpu_baseline": {"value": value, "unit": "Gkeys/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "Gkeys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import numpy as np
    import torch

    import workloads
    import paper_2605_10390_gb300 as fs

    torch.cuda.set_device(local_rank)
    if args.only:
        stream = torch.cuda.current_stream()
        peak = measured_peaks()[0]
        if args.only == "secondary":
            out = run_secondary(fs, workloads, torch, stream, peak)
        elif args.only == "expand":
            out = run_secondary(fs, workloads, torch, stream, peak, reps=args.reps, expand_log2n=args.expand_log2n,
                                u64=False)
        elif args.only == "batched":
            out = run_batched(fs, workloads, torch, stream, peak)
        elif args.only == "learned":
            out = run_learned(fs, workloads, torch, stream, peak, log2n=args.learned_log2n)
        elif args.only == "serving_small":
            out = run_serving_small(fs, workloads, torch)
        else:
            out = run_serving(fs, workloads, torch, stream)
        print(json.dumps({"section": args.only, "result": out}), flush=True)
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    n = 1 << args.log2n
    stream = torch.cuda.current_stream()

    # Inputs in HBM (generated on the device by the shared workload generator).
    inputs = []
    for i, d in enumerate(DISTS):
        keys = torch.empty(n, dtype=torch.uint16, device="cuda")
        vals = torch.empty(n, dtype=torch.uint32, device="cuda")
        table = workloads.table_for(d, KEY_BITS)
        tdev = torch.from_numpy(table).cuda() if table is not None else None
        workloads.generate_device(d, keys.data_ptr(), n, KEY_BITS, seed=rank, stream=i,
                                  cuda_stream=stream.cuda_stream, table_dev_ptr=tdev.data_ptr() if tdev is not None else None)
        workloads.iota_device(vals.data_ptr(), n, cuda_stream=stream.cuda_stream)
        inputs.append((keys, vals))
    keys_out = torch.empty(n, dtype=torch.uint16, device="cuda")
    vals_out = torch.empty(n, dtype=torch.uint32, device="cuda")
    torch.cuda.synchronize()

    plan = fs.Plan(n, KEY_BITS, has_values=True)
    info = plan.describe(n, PRECISION, True)

    def step():
        for k, v in inputs:
            plan.sort_out(k, v, keys_out, vals_out, precision_bits=PRECISION)

    for _ in range(args.warmup):
        step()
    plan.sync()
    fs.fsort_plan_set_timing(plan.handle, True)

    sampler = ClockSampler(local_rank) if rank == 0 else None
    if sampler:
        sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    plan.sync()
    ms = max_over_ranks(torch, dist, [ev0.elapsed_time(ev1)], "cuda")[0]
    recs = fs.fsort_plan_timing_report(plan.handle, 1 << 14)
    fs.fsort_plan_set_timing(plan.handle, False)

    value = job_gkeys_per_s(world, args.steps * len(DISTS) * n, ms / 1e3)

    # Roofline of the dominant kernel (scatter): algorithmic 12 n bytes per active launch.
    kb, vb = KEY_BITS // 8, 4
    sc = [r for r in recs if r["kind"] == "scatter" and r["active"]]
    sc_ms = sum(r["ms"] for r in sc)
    per_launch = 2 * (kb + vb) * n
    peak, peak_src = measured_peaks()
    achieved = (per_launch * len(sc) / (sc_ms / 1e3) / 1e9) if sc_ms > 0 else None
    traffic, traffic_note = ncu_traffic(n)
    kernels = {}
    for r in recs:
        key = r["kind"] + ("" if r["active"] else "_skipped")
        kk = kernels.setdefault(key, {"launches": 0, "ms": 0.0})
        kk["launches"] += 1
        kk["ms"] += r["ms"]
    total_kernel_ms = sum(v["ms"] for v in kernels.values()) or 1.0
    for v in kernels.values():
        v["share"] = v["ms"] / total_kernel_ms
        v["avg_us"] = v["ms"] / v["launches"] * 1e3
    # Whole-step algorithmic bytes: one key read for the histogram, read+write of
    # keys+values per executed pass, and read+write for a final copy when run.
    calls = {}
    for r in recs:
        c = calls.setdefault(r["call"], {"ms": 0.0, "bytes": kb * n})
        c["ms"] += r["ms"]
        if r["kind"] in ("scatter", "copy") and r["active"]:
            c["bytes"] += 2 * (kb + vb) * n
    job_bytes = sum(c["bytes"] for c in calls.values()) / max(1, args.steps)
    per_dist = {}
    passes_run = {}  # executed scatter passes per sort of each distribution (trivial passes are skipped)
    for idx, c in calls.items():
        per_dist.setdefault(DISTS[idx % len(DISTS)], []).append(c["ms"])
    for r in recs:
        if r["kind"] == "scatter" and r["active"]:
            d = DISTS[r["call"] % len(DISTS)]
            passes_run[d] = passes_run.get(d, 0) + 1
    passes_run = {d: passes_run.get(d, 0) / max(1, len(per_dist.get(d, []))) for d in DISTS}
    per_dist_gkeys = {d: n / (statistics.mean(v) / 1e3) / 1e9 for d, v in per_dist.items()}

    result = None
    if rank == 0:
        ms_per_step = ms / args.steps
        result = {
            "metric": METRIC, "value": value, "unit": "Gkeys/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u16", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_per_sort": n, "key_bits": KEY_BITS, "precision_bits": PRECISION,
                       "values": "uint32 original index", "sorts_per_step": len(DISTS), "digit_bits": info["digit_bits"],
                       "tile_keys": info["tile_keys"], "l2": "inputs larger than L2 (1.5 GiB per sort), no flush",
                       "parallelism": f"{world} independent replicas" if world > 1 else "single GPU"},
            "roofline": {"bound": "hbm", "kernel": "table scatter pass (KT3, tile_scatter_kernel)", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                         "algorithmic_bytes_per_launch": per_launch, "launches": len(sc),
                         "avg_launch_ms": sc_ms / len(sc) if sc else None, "peak_source": peak_src,
                         "traffic_note": traffic_note,
                         # Eq. 1's b_eff: algorithmic bytes over the DRAM bytes ncu measured for the launch
                         "b_eff": (per_launch / traffic) if traffic else None,
                         "frac_of_nominal": (achieved / NOMINAL_HBM_GBS) if achieved else None,
                         "nominal_gbs": NOMINAL_HBM_GBS, "passes_run": passes_run},
            "job_hbm": {"algorithmic_bytes_per_step": job_bytes,
                        "achieved_gbs": job_bytes / (ms_per_step / 1e3) / 1e9,
                        "frac": job_bytes / (ms_per_step / 1e3) / 1e9 / peak},
            "per_distribution_gkeys": per_dist_gkeys,
            "kernels": kernels,
            "gpu_launches": len(recs),
            "clocks": clocks,
        }
    plan.close()
    del inputs, keys_out, vals_out
    torch.cuda.empty_cache()

    if rank == 0 and not args.no_extra:
        result["secondary"] = run_secondary(fs, workloads, torch, stream, peak)
        result["batched"] = run_batched(fs, workloads, torch, stream, peak)
        result["learned"] = run_learned(fs, workloads, torch, stream, peak)
        result["serving"] = run_serving(fs, workloads, torch, stream)
        result["serving_small"] = run_serving_small(fs, workloads, torch)

    # End to end through the public host-buffer entry point (rank-local).
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(fs, workloads, torch, n, rank, world, dist, kb, vb, max(1, min(args.steps, 10)))
    if rank == 0:
        result["e2e"] = e2e
        if world == 1 and not args.no_cpu_baseline:
            result["cpu_baseline"] = cpu_baseline()
        else:
            result["cpu_baseline"] = None
        result["summary"] = summary(result)  # last key: kept by readers of the line's tail
        print(json.dumps(result), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
