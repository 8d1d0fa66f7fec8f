"""Save and load a fitted learned bucket map (checkpoint / resume).

A plan's learned map is the fitted model: its FP32 parameters, the (G, H) map
table, the frequent keys and the feature normalisation.  ``fsort_learned_get_model``
reads it from a plan and ``fsort_learned_set_model`` installs it in another
one, so a model fitted once can serve later processes without refitting.

File format: a magic line, one JSON header line, then the arrays as raw
little-endian bytes in the order the header lists them:

    FSORTMODEL\\n
    {"version": 1, "center": c, "half": h, "arrays": [{"name": "params",
     "dtype": "<f4", "shape": [4353]}, ...], "sha256": "<digest of the payload>"}\\n
    <params f32[4353]> <cells u32[56321][2]> <heavy u64[m]>

The header's digest covers the payload, so a truncated or altered file is
refused.  The file is replaced atomically (written to a temporary file, then
renamed).
"""
from __future__ import annotations

import hashlib
import json
import os
import tempfile

import numpy as np

from ._binding import (FSORT_LEARN_CELLS, FSORT_LEARN_MAX_HEAVY, FSORT_MLP_PARAMS, fsort_learned_get_model,
                       fsort_learned_set_model)

MAGIC = b"FSORTMODEL\n"
VERSION = 1
_LAYOUT = (("params", "<f4"), ("cells", "<u4"), ("heavy", "<u8"))


def _check_model(model: dict) -> dict:
    params = np.ascontiguousarray(model["params"], np.float32)
    cells = np.ascontiguousarray(model["cells"], np.uint32)
    heavy = np.ascontiguousarray(model["heavy"], np.uint64)
    if params.shape != (FSORT_MLP_PARAMS,):
        raise ValueError(f"params must have shape ({FSORT_MLP_PARAMS},), not {params.shape}")
    if cells.shape != (FSORT_LEARN_CELLS + 1, 2):
        raise ValueError(f"cells must have shape ({FSORT_LEARN_CELLS + 1}, 2), not {cells.shape}")
    if heavy.ndim != 1 or heavy.size > FSORT_LEARN_MAX_HEAVY:
        raise ValueError(f"heavy must be 1-D with at most {FSORT_LEARN_MAX_HEAVY} keys")
    if heavy.size > 1 and not np.all(heavy[1:] > heavy[:-1]):
        raise ValueError("heavy keys must be strictly ascending")
    center, half = float(model["center"]), float(model["half"])
    if not (half > 0.0) or not np.isfinite(center):
        raise ValueError("the normalisation needs a finite center and half > 0")
    return {"params": params, "cells": cells, "heavy": heavy, "center": center, "half": half}


def save(path: str, model: dict) -> None:
    """Write a model (the dict ``fsort_learned_get_model`` returns) to path."""
    m = _check_model(model)
    arrays = [np.ascontiguousarray(m[name], dtype=np.dtype(dt)) for name, dt in _LAYOUT]
    payload = b"".join(a.tobytes() for a in arrays)
    header = {"version": VERSION, "center": m["center"], "half": m["half"],
              "arrays": [{"name": name, "dtype": dt, "shape": list(a.shape)} for (name, dt), a in zip(_LAYOUT, arrays)],
              "sha256": hashlib.sha256(payload).hexdigest()}
    folder = os.path.dirname(os.path.abspath(path))
    os.makedirs(folder, exist_ok=True)
    fd, tmp = tempfile.mkstemp(prefix=".model-", dir=folder)
    try:
        with os.fdopen(fd, "wb") as f:
            f.write(MAGIC)
            f.write(json.dumps(header, sort_keys=True).encode() + b"\n")
            f.write(payload)
        os.replace(tmp, path)
    except BaseException:
        if os.path.exists(tmp):
            os.unlink(tmp)
        raise


def load(path: str) -> dict:
    """Read a model written by save(); raises ValueError if the file is not one."""
    with open(path, "rb") as f:
        data = f.read()
    if not data.startswith(MAGIC):
        raise ValueError(f"{path}: not a libfsort model file")
    end = data.find(b"\n", len(MAGIC))
    if end < 0:
        raise ValueError(f"{path}: header line missing")
    try:
        header = json.loads(data[len(MAGIC):end])
    except ValueError as e:
        raise ValueError(f"{path}: unreadable header") from e
    if header.get("version") != VERSION:
        raise ValueError(f"{path}: unsupported version {header.get('version')!r}")
    payload = data[end + 1:]
    if hashlib.sha256(payload).hexdigest() != header.get("sha256"):
        raise ValueError(f"{path}: payload does not match its digest (truncated or altered)")
    specs = header.get("arrays", [])
    if [s.get("name") for s in specs] != [name for name, _ in _LAYOUT]:
        raise ValueError(f"{path}: unexpected arrays")
    out, at = {}, 0
    for (name, dt), spec in zip(_LAYOUT, specs):
        if spec.get("dtype") != dt:
            raise ValueError(f"{path}: {name} has dtype {spec.get('dtype')!r}, expected {dt}")
        shape = tuple(int(x) for x in spec["shape"])
        nbytes = int(np.prod(shape, dtype=np.int64)) * np.dtype(dt).itemsize
        if at + nbytes > len(payload):
            raise ValueError(f"{path}: payload shorter than its header says")
        out[name] = np.frombuffer(payload, dtype=np.dtype(dt), count=nbytes // np.dtype(dt).itemsize,
                                  offset=at).reshape(shape).copy()
        at += nbytes
    if at != len(payload):
        raise ValueError(f"{path}: payload longer than its header says")
    out["center"], out["half"] = float(header["center"]), float(header["half"])
    return _check_model(out)


def save_plan_model(plan, path: str) -> None:
    """Write the model fitted on (or installed in) a plan."""
    save(path, fsort_learned_get_model(plan))


def load_plan_model(plan, path: str, stream=None) -> None:
    """Install a saved model in a plan with FSORT_FLAG_LEARNED; its next
    eligible sorts take the learned path (judged as usual)."""
    m = load(path)
    fsort_learned_set_model(plan, params=m["params"], cells=m["cells"], heavy=m["heavy"], center=m["center"],
                            half=m["half"], stream=stream)
