"""Persistent cache of the batched path's autotuned configuration.

``fsort_batch_autotune`` times the candidate configurations of the batched
sort (the larger segments' form, on-chip segment capacity x CTAs per SM, digit
width) on the caller's batch and keeps the fastest in the plan.  Batch stream sorting is tuned per batch size
(Sec. III-C and IV-D); the choice depends on the device and on the
batch's shape, not on its data, so this module stores it in a JSON file keyed
by both.  A later process with a batch of the same shape class sets the stored
configuration with ``fsort_batch_set_config`` instead of timing again.

Shape class: the key and value widths, the precision, and for each size class
of the batched path (segments sorted whole on chip at capacities 1,024 /
2,048 / 4,096 keys, and larger segments) the segment count rounded up to a
power of two, plus the total keys rounded up to a power of two.  Batches in
one class run the same kernels on about the same amount of work.

The file holds ``{"version": 3, "entries": {"<device>|<class>": {...}}}``
(files of another version are ignored).
It is replaced atomically (write to a temporary file, then rename), so a
reader sees either the old or the new file.  Entries that do not name a valid
configuration are ignored, as is an unreadable file.
"""
from __future__ import annotations

import json
import os
import tempfile

from ._binding import _numel, fsort_batch_autotune, fsort_batch_set_config

VERSION = 3  # entries carry the digit width
CAPACITIES = (0, 1024, 2048, 4096)  # 0: no on-chip path
MAX_CTAS_PER_SM = 8
SIZE_CLASSES = (1024, 2048, 4096)   # upper bounds of the on-chip classes; larger segments form the last class


def _pow2_ceil(x: int) -> int:
    return 0 if x <= 0 else 1 << (int(x) - 1).bit_length()


def batch_class(sizes, key_bits: int, has_values: bool, precision_bits: int | None = None) -> str:
    """The shape class of a batch with these segment sizes (see the module docstring)."""
    p = key_bits if precision_bits is None else precision_bits
    counts = [0] * (len(SIZE_CLASSES) + 1)
    total = 0
    for n in sizes:
        n = int(n)
        if n < 0:
            raise ValueError("segment size must be >= 0")
        total += n
        if n == 0:
            continue  # empty segments launch nothing
        c = 0
        while c < len(SIZE_CLASSES) and n > SIZE_CLASSES[c]:
            c += 1
        counts[c] += 1
    parts = [f"k{key_bits}", f"v{1 if has_values else 0}", f"p{p}"]
    parts += [f"s{b}:{_pow2_ceil(c)}" for b, c in zip(list(SIZE_CLASSES) + ["big"], counts)]
    parts.append(f"n:{_pow2_ceil(total)}")
    return ",".join(parts)


def device_key(name: str, sm_count: int, major: int, minor: int) -> str:
    return f"{name}/sm{major}{minor}/{sm_count}sms"


def current_device_key() -> str:
    import torch
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    return device_key(props.name, props.multi_processor_count, props.major, props.minor)


CONFIG_KEYS = ("small_capacity", "small_ctas_per_sm", "large_form", "digit_bits")
DIGIT_BITS = (6, 7, 8)


def valid_config(cfg) -> bool:
    if not isinstance(cfg, dict):
        return False
    cap, ctas, form = cfg.get("small_capacity"), cfg.get("small_ctas_per_sm"), cfg.get("large_form")
    width = cfg.get("digit_bits")
    if any(not isinstance(v, int) or isinstance(v, bool) for v in (cap, ctas, form, width)):
        return False
    return cap in CAPACITIES and 1 <= ctas <= MAX_CTAS_PER_SM and form in (0, 1) and width in DIGIT_BITS


class TuneCache:
    """The JSON file of tuned batch configurations, one entry per (device, class)."""

    def __init__(self, path: str):
        self.path = path
        self.entries = self._load()

    def _load(self) -> dict:
        try:
            with open(self.path) as f:
                d = json.load(f)
        except (OSError, ValueError):
            return {}
        if not isinstance(d, dict) or d.get("version") != VERSION or not isinstance(d.get("entries"), dict):
            return {}
        return {k: v for k, v in d["entries"].items() if isinstance(k, str) and valid_config(v)}

    def get(self, device: str, cls: str) -> dict | None:
        e = self.entries.get(f"{device}|{cls}")
        return None if e is None else {k: e[k] for k in CONFIG_KEYS}

    def put(self, device: str, cls: str, cfg: dict, ms: float | None = None) -> None:
        if not valid_config(cfg):
            raise ValueError(f"not a batch configuration: {cfg!r}")
        e = {k: cfg[k] for k in CONFIG_KEYS}
        if ms is not None:
            e["ms"] = float(ms)
        self.entries[f"{device}|{cls}"] = e
        self.save()

    def save(self) -> None:
        folder = os.path.dirname(os.path.abspath(self.path))
        os.makedirs(folder, exist_ok=True)
        fd, tmp = tempfile.mkstemp(prefix=".tune-", suffix=".json", dir=folder)
        try:
            with os.fdopen(fd, "w") as f:
                json.dump({"version": VERSION, "entries": self.entries}, f, indent=1, sort_keys=True)
                f.write("\n")
            os.replace(tmp, self.path)
        except BaseException:
            if os.path.exists(tmp):
                os.unlink(tmp)
            raise


def segment_sizes(segments) -> list[int]:
    """Sizes of (keys, vals[, n]) segments, as fsort_sort_batch reads them."""
    return [int(s[2]) if len(s) > 2 and s[2] is not None else _numel(s[0], None) for s in segments]


def autotune_cached(plan, segments, key_bits: int, precision_bits=None, *, has_values: bool, path: str,
                    device: str | None = None, stream=None):
    """Set the plan's batch configuration from the cache, or tune and store it.

    Returns ``(config, ms, hit)``.  On a hit the stored configuration is set
    and nothing runs on the GPU (``ms`` is the time stored with it, or None).
    On a miss ``fsort_batch_autotune`` times the candidates on these segments
    (which leaves them sorted) and the winner is stored.
    """
    dev = current_device_key() if device is None else device
    cls = batch_class(segment_sizes(segments), key_bits, has_values, precision_bits)
    cache = TuneCache(path)
    cfg = cache.get(dev, cls)
    if cfg is not None:
        fsort_batch_set_config(plan, cfg["small_capacity"], cfg["small_ctas_per_sm"], cfg["large_form"],
                               cfg["digit_bits"])
        return cfg, cache.entries[f"{dev}|{cls}"].get("ms"), True
    cfg, ms = fsort_batch_autotune(plan, segments, key_bits, precision_bits, stream)
    cache.put(dev, cls, cfg, ms)
    return cfg, ms, False
