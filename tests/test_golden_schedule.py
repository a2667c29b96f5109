"""The staggered KNN schedule against the values the paper prints (Table 1,
tests/golden/table1_knn_schedule.txt).

  * the training workload (6.3 M photons: 2^20 per light per phase, two
    lights, three phases) uses Table 1's 6M row and its stage starts;
  * the stage rule of the training loop (step s is in stage i once
    s >= ceil(start_i * steps)) reproduces the table's percentage columns:
    of 100 steps, stages of 37, 27, 27 and 9 steps;
  * radii grow stage by stage in every row (the schedule coarsens).
"""
import math
import os

import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_knn_schedule.txt")


def _read():
    starts, rows = None, {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if line.startswith("# stage starts"):
                starts = [float(v) for v in line.split(":")[1].split()]
            if not line or line.startswith("#") or line.startswith("photons"):
                continue
            name, *r = line.split()
            rows[name] = [float(v) for v in r]
    return starts, rows


def _stage(s, steps, starts):
    i = 0
    for j in range(1, len(starts)):
        if s >= math.ceil(starts[j] * steps):
            i = j
    return i


def test_training_workload_uses_the_6m_row():
    bench = pytest.importorskip("bench")
    starts, rows = _read()
    assert [b for b, _ in bench.KNN_STAGES] == starts
    assert [r for _, r in bench.KNN_STAGES] == rows["6M"]
    photons = 2 * 3 * (1 << 20)
    assert min(rows, key=lambda k: abs(float(k[:-1]) * 1e6 - photons)) == "6M"


def test_stage_rule_matches_the_percentage_columns():
    starts, _ = _read()
    counts = [0] * len(starts)
    for s in range(100):
        counts[_stage(s, 100, starts)] += 1
    assert counts == [37, 27, 27, 9]      # 0-36 %, 37-63 %, 64-90 %, 91-100 %
    # and at the workload's 2000 steps the boundaries fall on the same percentages
    first = [min(s for s in range(2000) if _stage(s, 2000, starts) == i) for i in range(4)]
    assert first == [0, 740, 1280, 1820]


def test_radii_grow_stage_by_stage():
    _, rows = _read()
    assert set(rows) == {"1M", "3M", "6M", "12M"}
    for r in rows.values():
        assert len(r) == 4 and all(a < b for a, b in zip(r, r[1:]))
    # more photons, smaller final radius
    assert rows["1M"][3] > rows["3M"][3] > rows["6M"][3] > rows["12M"][3]
