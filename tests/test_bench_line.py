"""bench.py's result line is strict JSON (no GPU): a strict parser accepts it even when the
result carries NaN and infinities (failed search candidates, a blown-up storage experiment),
which it writes as null, and it stays one line."""
import json
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _strict_loads(line):
    def reject(token):
        raise ValueError(f"non-standard JSON token {token}")
    return json.loads(line, parse_constant=reject)


def test_line_with_non_finite_numbers_is_strict_json():
    result = {
        "metric": bench.METRIC, "value": 2.5, "unit": "s",
        "candidates": [{"method": "faber", "time_to_T_s": float("nan")},
                       {"method": "hork", "time_to_T_s": float("inf")}],
        "bf16_storage": [{"seismo_rel_err": float("-inf")}],
        "nested": {"a": (1.0, float("nan"), np.float64("inf"), np.float32(0.5), np.int64(7))},
        "flag": True, "none": None, "text": "x",
    }
    line = bench.json_line(result)
    assert "\n" not in line
    d = _strict_loads(line)
    assert d["candidates"][0]["time_to_T_s"] is None
    assert d["candidates"][1]["time_to_T_s"] is None
    assert d["bf16_storage"][0]["seismo_rel_err"] is None
    assert d["nested"]["a"] == [1.0, None, None, 0.5, 7]
    assert d["flag"] is True and d["none"] is None and d["text"] == "x"
    assert d["value"] == 2.5 and math.isfinite(d["value"])


def test_finite_or_none_keeps_finite_values():
    obj = {"x": [0.0, -1.5, 3], "y": {"z": 1e300}}
    assert bench.finite_or_none(obj) == obj


def test_parse_defaults_finish_in_minutes():
    a = bench.parse([])
    assert a.gpus == 1 and a.steps >= 1 and a.warmup >= 3
    assert a.check3d == 0 and a.detail_out is None
