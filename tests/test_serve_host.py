"""Host-only parts of the serving loop, compiled with the system C++ compiler
(no GPU): the first-fit device-memory arena that admission draws on, and the
latency log behind p50/p99.

The arena is checked against a granule bitmap: first fit with coalesced free
ranges must return the start of the lowest-addressed run of free granules
that holds the request, and used / peak / number of free ranges follow from
the bitmap.  The latency log is checked against nearest-rank percentiles of
the last W recorded values and the mean and maximum of all of them.
"""
import math
import os
import random
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
G = 256  # granule bytes


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("serve_host") / "serve_host_check")
    subprocess.run([cxx, "-std=c++17", "-O1", "-Wall", "-Werror", "-o", exe,
                    os.path.join(HERE, "serve_host_check.cc")], check=True)

    def run(lines):
        p = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, timeout=120)
        assert p.returncode == 0, p.stderr
        return p.stdout.split("\n")[:-1]
    return run


class BitmapArena:
    def __init__(self, size):
        self.busy = [False] * (size // G)
        self.used = self.peak = 0

    def runs(self):
        out, i = [], 0
        while i < len(self.busy):
            if self.busy[i]:
                i += 1
                continue
            j = i
            while j < len(self.busy) and not self.busy[j]:
                j += 1
            out.append((i, j - i))
            i = j
        return out

    def alloc(self, b):
        g = -(-b // G)
        for start, length in self.runs():
            if length >= g:
                for k in range(start, start + g):
                    self.busy[k] = True
                self.used += g * G
                self.peak = max(self.peak, self.used)
                return start * G
        return -1

    def free(self, off, b):
        g = -(-b // G)
        for k in range(off // G, off // G + g):
            assert self.busy[k]
            self.busy[k] = False
        self.used -= g * G


@pytest.mark.parametrize("seed", range(4))
def test_arena_matches_bitmap_first_fit(driver, seed):
    rng = random.Random(seed)
    size = 64 * 1024 + 100  # not a whole number of granules: floored
    model = BitmapArena(size // G * G)
    cmds, expect, live = [f"reset {size}"], [], []
    # build the command list against the model, then compare the driver's answers
    for _ in range(600):
        if live and rng.random() < 0.45:
            off, b = live.pop(rng.randrange(len(live)))
            model.free(off, b)
            cmds.append(f"free {off} {b}")
        else:
            b = rng.choice([1, 255, 256, 257, 1000, 4096, 9000, 20000, 70000])
            off = model.alloc(b)
            cmds.append(f"alloc {b}")
            expect.append(str(off))
            if off >= 0:
                live.append((off, b))
        if rng.random() < 0.1:
            cmds.append("stat")
            expect.append(f"{size // G * G} {model.used} {model.peak} {len(model.runs())}")
    for off, b in live:  # everything returned: one free range again
        model.free(off, b)
        cmds.append(f"free {off} {b}")
    cmds.append("stat")
    expect.append(f"{size // G * G} 0 {model.peak} 1")
    assert driver(cmds) == expect


def test_arena_coalesces_both_neighbours(driver):
    out = driver(["reset 4096", "alloc 1024", "alloc 1024", "alloc 1024", "stat",
                  "free 0 1024", "free 2048 1024", "stat", "free 1024 1024", "stat", "alloc 4096", "alloc 1"])
    assert out == ["0", "1024", "2048", "4096 3072 3072 1",   # [3072, 4096) free
                   "4096 1024 3072 2",                          # [0,1024) and [2048,4096)
                   "4096 0 3072 1",                             # middle joins both sides
                   "0", "-1"]


def nearest_rank(values, p):
    v = sorted(values)
    i = min(max(math.ceil(p * len(v) - 1e-9), 1), len(v))
    return v[i - 1]


@pytest.mark.parametrize("window,count", [(1, 5), (7, 3), (7, 7), (7, 50), (1000, 999)])
def test_latency_window_percentiles_and_totals(driver, window, count):
    rng = random.Random(window * 1000 + count)
    vals = [round(rng.uniform(0.0, 100.0), 3) for _ in range(count)]
    ps = [0.01, 0.5, 0.99, 1.0]
    cmds = [f"log {window}"] + [f"rec {x!r}" for x in vals] + [f"pct {p}" for p in ps] + ["mean", "max"]
    out = [float(x) for x in driver(cmds)]
    last = vals[-window:]
    assert out[:len(ps)] == [nearest_rank(last, p) for p in ps]
    assert out[-2] == pytest.approx(sum(vals) / len(vals), rel=1e-12)
    assert out[-1] == max(vals)


def test_empty_latency_log(driver):
    assert [float(x) for x in driver(["log 4", "pct 0.5", "mean", "max"])] == [0.0, 0.0, 0.0]
