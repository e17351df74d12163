"""The autotuner's bookkeeping (no GPU): the fastest fitting candidate is
chosen, a shape is measured once and read from the JSON cache afterwards,
and a shape where nothing fits is an error."""
import json
import threading

import pytest

from paper_2203_02096_gb300 import autotune


def _bare_tuner(path):
    t = autotune.Tuner.__new__(autotune.Tuner)
    t.ctx, t.path, t.reps, t.device_name = None, str(path), 1, "test-device"
    t._lock = threading.Lock()
    t.entries = {}
    return t


def test_pick_measures_once_and_caches(tmp_path):
    path = tmp_path / "tune.json"
    t = _bare_tuner(path)
    calls = []

    def measure(cand):
        calls.append(tuple(cand))
        return [3.0, -1.0, 1.5, 2.0]   # 64 does not fit; 128 is fastest

    assert t._pick("k", (32, 64, 128, 256), measure) == 128
    assert t._pick("k", (32, 64, 128, 256), measure) == 128
    assert len(calls) == 1
    saved = json.loads(path.read_text())
    assert saved["k"]["choice"] == 128 and saved["k"]["ms"]["64"] == -1.0
    t2 = _bare_tuner(path)
    t2.entries = json.loads(path.read_text())
    assert t2._pick("k", (32, 64, 128, 256), measure) == 128 and len(calls) == 1


def test_nothing_fits_is_an_error(tmp_path):
    t = _bare_tuner(tmp_path / "tune.json")
    with pytest.raises(RuntimeError):
        t._pick("k", (1, 2, 4), lambda c: [-1.0, -1.0, -1.0])
