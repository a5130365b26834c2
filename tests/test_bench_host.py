"""Host logic of bench.py that needs no GPU: the end-to-end pipeline schedule
and the clock-sample filter."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


@pytest.mark.parametrize("ne", [1, 2, 3, 4, 7, 16])
@pytest.mark.parametrize("H", [1, 2, 3, 4])
def test_pipeline_schedule(ne, H):
    ops = bench.pipeline_schedule(ne, H)
    issued = [j for op, j in ops if op == "issue"]
    stored = [j for op, j in ops if op == "store"]
    # every step issued once and stored once, both in step order
    assert issued == list(range(ne)) and stored == list(range(ne))
    pos = {op: i for i, op in enumerate(ops)}
    for j in range(ne):
        assert pos[("issue", j)] < pos[("store", j)]
        # a handle takes a new step only after its previous step was stored
        if j >= H:
            assert pos[("store", j - H)] < pos[("issue", j)]
        # at most H - 1 steps queued beyond the one being waited on
        ahead = sum(1 for i in range(ne) if pos[("issue", i)] < pos[("store", j)]) - (j + 1)
        assert ahead <= H - 1
    # and, where there are enough steps, exactly H - 1 while the pipeline is full
    if ne > H:
        j = 0
        ahead = sum(1 for i in range(ne) if pos[("issue", i)] < pos[("store", j)]) - 1
        assert ahead == H - 1


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        pass


class _FakeThread:
    def join(self, timeout=None):
        pass


def _sampler(lines, bus):
    c = bench.ClockSampler.__new__(bench.ClockSampler)
    c.lines, c.bus, c.proc, c.th = lines, bus, _FakeProc(), _FakeThread()
    return c.stop()


ROWS = ["0, 00000009:01:00.0, 2070, 2070, 500, 0x0, Not Active, Not Active, Not Active, Active",
        "1, 00000009:02:00.0, 1000, 2070, 500, 0x0, Active, Not Active, Not Active, Active"]


def test_clock_rows_by_bus_number():
    a = _sampler(ROWS, 1)
    assert a["sm_mhz"] == 2070.0 and a["samples"] == 1 and a["reasons"] == ["sw_power_cap"]
    b = _sampler(ROWS, 2)
    assert b["sm_mhz"] == 1000.0 and "hw_slowdown" in b["reasons"]


def test_clock_rows_unknown_bus():
    # two GPUs visible and no row on the process's bus: no clock record
    assert _sampler(ROWS, 7) is None
    # one GPU visible: its rows, whatever bus number torch reports
    one = _sampler(ROWS[:1], 0)
    assert one["sm_mhz"] == 2070.0
    assert _sampler([], 1) is None
