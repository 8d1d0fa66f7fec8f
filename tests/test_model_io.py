"""Checkpoint / resume of a learned bucket map (no GPU): the file round-trips
every array bit for bit, and a truncated, altered or foreign file, or a model
of the wrong shape, is refused."""
import os

import numpy as np
import pytest

from oracle import learned as ol
from paper_2605_10390_gb300 import model_io


def model(seed=0, heavy_n=40):
    rng = np.random.default_rng(seed)
    params = rng.normal(0, 0.3, ol.PARAMS).astype(np.float32)
    heavy = np.unique(rng.integers(1, 1 << 62, heavy_n, dtype=np.uint64))
    cells = ol.table(ol.bf16_round(params), heavy, 0.6, 0.3)
    return {"params": params, "cells": cells, "heavy": heavy, "center": 0.6, "half": 0.3}


def same(a, b):
    return (all(np.array_equal(a[k], b[k]) and a[k].dtype == b[k].dtype for k in ("params", "cells", "heavy"))
            and np.float32(a["center"]) == np.float32(b["center"]) and a["half"] == b["half"])


@pytest.mark.parametrize("heavy_n", [0, 1, 40])
def test_round_trip_is_exact(tmp_path, heavy_n):
    m = model(heavy_n, heavy_n)
    path = str(tmp_path / "sub" / "map.fsm")
    model_io.save(path, m)
    got = model_io.load(path)
    assert got["params"].dtype == np.float32 and got["cells"].dtype == np.uint32 and got["heavy"].dtype == np.uint64
    assert same({**m, "params": m["params"].astype(np.float32), "cells": m["cells"].astype(np.uint32)}, got)
    assert os.listdir(tmp_path / "sub") == ["map.fsm"]  # no temporary file left behind


def test_damaged_or_foreign_files_are_refused(tmp_path):
    path = tmp_path / "map.fsm"
    model_io.save(str(path), model())
    data = path.read_bytes()
    cases = {
        "truncated": data[:-8],
        "flipped byte": data[:-100] + bytes([data[-100] ^ 1]) + data[-99:],
        "extra bytes": data + b"\0" * 8,
        "foreign": b"PK\x03\x04" + data[4:],
        "no header": model_io.MAGIC,
    }
    header_end = data.index(b"\n", len(model_io.MAGIC))
    hdr = data[len(model_io.MAGIC):header_end]
    cases["version"] = model_io.MAGIC + hdr.replace(b'"version": 1', b'"version": 2') + data[header_end:]
    cases["dtype"] = model_io.MAGIC + hdr.replace(b'"<f4"', b'"<f8"') + data[header_end:]
    for name, bad in cases.items():
        path.write_bytes(bad)
        with pytest.raises(ValueError):
            model_io.load(str(path))
        assert name


def test_models_of_the_wrong_shape_are_not_written(tmp_path):
    m = model()
    bad = [dict(m, params=m["params"][:-1]), dict(m, cells=m["cells"][:-1]), dict(m, heavy=m["heavy"][::-1].copy()),
           dict(m, heavy=np.arange(9000, dtype=np.uint64)), dict(m, half=0.0), dict(m, center=float("nan"))]
    for i, b in enumerate(bad):
        with pytest.raises(ValueError):
            model_io.save(str(tmp_path / f"m{i}.fsm"), b)
    assert not os.listdir(tmp_path)
