"""bench.py's reference arm on the CPU: the FP64 oracle timed on the host
cores prints one JSON line with the headline metric and config, the
cpu_baseline describing the run and an end-to-end entry with no copies;
under several ranks only rank 0 works and prints."""
import contextlib
import io
import json
import os

import pytest

import bench


@pytest.fixture
def rank_env(monkeypatch):
    def set_rank(rank, world):
        monkeypatch.setenv("RANK", str(rank))
        monkeypatch.setenv("WORLD_SIZE", str(world))
        monkeypatch.setenv("LOCAL_RANK", str(rank))
    return set_rank


def _run(argv):
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        rc = bench.main(argv)
    return rc, buf.getvalue()


def test_reference_arm_line(rank_env):
    rank_env(0, 1)
    rc, out = _run(["--impl", "reference", "--steps", "1", "--warmup", "3"])
    assert rc == 0
    lines = [l for l in out.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    # the same workload as the GPU arm's line (only the L2 note differs)
    want = bench.config_dict(bench.workload(), "")
    assert {k: v for k, v in d["config"].items() if k != "l2"} == {k: v for k, v in want.items() if k != "l2"}
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] == (os.cpu_count() or 1)
    assert "evaluations" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_do_nothing(rank_env):
    rank_env(1, 2)
    rc, out = _run(["--impl", "reference", "--steps", "1", "--warmup", "3"])
    assert rc == 0 and out.strip() == ""
