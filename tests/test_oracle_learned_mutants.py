"""The learned-mapping oracle's pins catch plausible mistakes: each mutant
below is oracle/learned.py with one plausible slip planted (a transposed
matrix, a dropped term, an off-by-one, a wrong rounding), and every mutant
must fail at least one pin of tests/test_oracle_learned.py.  The unmutated
source must pass them all.  CPU only."""
import importlib.util
import inspect
import os
import types

import pytest

pytest.importorskip("torch")  # the BF16 pin compares against torch's cast

HERE = os.path.dirname(os.path.abspath(__file__))
SRC_PATH = os.path.join(os.path.dirname(HERE), "oracle", "learned.py")

MUTANTS = {
    "bf16_truncates": ("bias = 0x7FFF + ((bits >> 16) & 1)", "bias = 0 * bits"),
    "bf16_ties_away": ("bias = 0x7FFF + ((bits >> 16) & 1)", "bias = 0x8000 + 0 * bits"),
    "forward_w2_transposed": ("h2 = np.maximum(0.0, h1 @ w2.T + b2)              # m x 64",
                              "h2 = np.maximum(0.0, h1 @ w2 + b2)"),
    "forward_relu2_dropped": ("h2 = np.maximum(0.0, h1 @ w2.T + b2)              # m x 64", "h2 = h1 @ w2.T + b2"),
    "grad_sigmoid_slope_dropped": ("dz = err * f * (1.0 - f) / m", "dz = err / m"),
    "grad_mean_dropped": ("dz = err * f * (1.0 - f) / m", "dz = err * f * (1.0 - f)"),
    "grad_w2_transposed": ("g_w2 = d2.T @ h1", "g_w2 = h1.T @ d2"),
    "grad_relu1_mask_dropped": ("d1 = (d2 @ w2) * (a1 > 0)", "d1 = (d2 @ w2)"),
    "grad_b2_dropped": ("g_b2 = d2.sum(axis=0)", "g_b2 = 0 * d2.sum(axis=0)"),
    "feature_sign": ("(np.log2(k + 1.0) / 64.0 - center) / half", "(np.log2(k + 1.0) / 64.0 + center) / half"),
    "cell_start_exponent": ("e = (i >> np.uint64(10)) + np.uint64(9)", "e = (i >> np.uint64(10)) + np.uint64(10)"),
    "cell_of_index": ("idx = (e - 9).astype(np.uint64) * np.uint64(1024)",
                      "idx = (e - 10).astype(np.uint64) * np.uint64(1024)"),
    "frac_scale": ("rem << np.uint64(16) - np.minimum(w, np.uint64(16))",
                   "rem << np.uint64(15) - np.minimum(w, np.uint64(15))"),
    "table_running_max_dropped": ("run = np.maximum.accumulate(np.clip(forward(params, x), 0.0, 1.0))",
                                  "run = np.clip(forward(params, x), 0.0, 1.0)"),
    "table_uniform_term_dropped": ("v = (1.0 - EPS) * run + EPS * np.clip(0.5 * (x + 1.0), 0.0, 1.0)", "v = run"),
    "heavy_count_inclusive": ('out[:CELLS, 1] = np.searchsorted(heavy, starts, side="left")',
                              'out[:CELLS, 1] = np.searchsorted(heavy, starts, side="right")'),
    "id_heavy_not_doubled": ("(pla >> shift) + np.uint64(2) * c + hit", "(pla >> shift) + c + hit"),
    "id_shift_off_by_one": ("shift = np.uint64(32 - int(math.log2(buckets_for(n_sort))))",
                            "shift = np.uint64(31 - int(math.log2(buckets_for(n_sort))))"),
    "buckets_round_down": ("want = -(-n // KEYS_PER_BUCKET)", "want = n // KEYS_PER_BUCKET"),
    "judge_counts_heavy": ("counts = np.bincount(ids[nonheavy]) if nonheavy.any() else np.zeros(1, np.int64)",
                           "counts = np.bincount(ids)"),
    "judge_limit_off_by_one": ("limit = TAU * n // b", "limit = TAU * n // b + 1"),
    # two sites changed together, so that the loss and its gradient stay consistent
    "loss_relu2_dropped_consistently": [("h2 = np.maximum(0.0, a2)", "h2 = a2"),
                                        ("d2 = np.outer(dz, w3) * (a2 > 0)", "d2 = np.outer(dz, w3)")],
    "loss_b1_dropped_consistently": [("a1 = np.outer(x, w1) + b1", "a1 = np.outer(x, w1)"),
                                     ("g_b1 = d1.sum(axis=0)", "g_b1 = 0 * d1.sum(axis=0)")],
}


def _pins():
    spec = importlib.util.spec_from_file_location("learned_pins", os.path.join(HERE, "test_oracle_learned.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    calls = []
    for name, fn in sorted(vars(mod).items()):
        if not name.startswith("test_") or not callable(fn):
            continue
        params = inspect.signature(fn).parameters
        if "seed" in params:
            calls += [(f"{name}[{s}]", lambda fn=fn, s=s: fn(s)) for s in (1, 2)]
        elif "d" in params and "g" in params:
            cases = [(0.9, 0.2), (-0.9, 0.2), (0.9, -0.5)]
            calls += [(f"{name}[{d},{g}]", lambda fn=fn, d=d, g=g: fn(d, g)) for d, g in cases]
        else:
            calls.append((name, fn))
    # the finite-difference pins are the slowest: run them last
    calls.sort(key=lambda c: "central_differences" in c[0])
    return mod, calls


def _oracle_from(src: str) -> types.ModuleType:
    m = types.ModuleType("learned_under_test")
    exec(compile(src, "learned_under_test.py", "exec"), m.__dict__)
    return m


def _first_failing_pin(src: str):
    pins, calls = _pins()
    pins.ol = _oracle_from(src)
    for name, fn in calls:
        try:
            fn()
        except Exception:  # an assertion, or the mutant breaking the code outright
            return name
    return None


def test_pins_pass_on_the_unmutated_oracle():
    with open(SRC_PATH) as f:
        assert _first_failing_pin(f.read()) is None


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mutant_fails_a_pin(name):
    with open(SRC_PATH) as f:
        src = f.read()
    sites = MUTANTS[name]
    for old, new in [sites] if isinstance(sites, tuple) else sites:
        assert src.count(old) == 1, f"mutation site of {name} not found once: {old}"
        src = src.replace(old, new)
    caught = _first_failing_pin(src)
    assert caught is not None, f"mutant {name} survived every pin"
