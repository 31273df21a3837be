"""Host logic of the benchmark's allocation refinement (no GPU): which
allocations it measures and which it keeps."""
import os
import sys
import types

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402


class _FakeWorkload:
    """Stands in for bench.Workload: records the allocations created and
    returns a saturated-trace duration from a given rate table."""

    def __init__(self, rate, sms=148):
        self.sms = sms
        self.rate = rate
        self.made = []
        self.cm = types.SimpleNamespace(camelot_pipeline_destroy=lambda p: None)

    def pipeline(self, mode, inst, quota):
        assert mode == 0
        self.made.append((tuple(inst), tuple(quota)))
        return len(self.made) - 1

    def trace(self, p, offsets):
        inst, quota = self.made[p]
        return None, len(offsets) / self.rate(inst, quota) * 1e3


def _total(inst, quota):
    return sum(a * q for a, q in zip(inst, quota))


def test_refine_neighbours_within_sm_budget():
    # the rate grows with stage 1's SMs
    wl = _FakeWorkload(lambda i, q: 1.0 + i[1] * q[1])
    inst, quota, table = bench.Workload.refine(wl, [3, 12, 3], [8, 8, 8])
    allocs = {(tuple(r["instances"]), tuple(r["sm_quota"])) for r in table}
    assert len(allocs) == len(table)                     # each measured once
    assert ((3, 12, 3), (8, 8, 8)) in allocs             # the allocator's own choice
    assert all(_total(a, q) <= 148 for a, q in allocs)   # 37 units of 4 SMs on 148 SMs
    # the first round: moves of one instance between stages, and the same SMs
    # as 4-SM instances
    assert {((2, 13, 3), (8, 8, 8)), ((4, 11, 3), (8, 8, 8)), ((3, 11, 4), (8, 8, 8)),
            ((6, 24, 6), (4, 4, 4)), ((3, 24, 3), (8, 4, 8))} <= allocs
    # then the neighbours of each new best: stage 1 ends with nearly all SMs
    assert _total(inst, quota) <= 148 and inst[1] * quota[1] >= 128


def test_refine_climbs_past_a_one_move_optimum():
    # a 3-stage pipeline whose rate is its slowest stage, on 8-SM instances
    # only (4-SM ones run badly here): from 6 / 9 / 3 the best one-instance
    # move is 5 / 10 / 3, and 4 / 11 / 3 (two moves away) is faster still
    rates = (0.75, 0.26, 1.2)
    wl = _FakeWorkload(lambda i, q: min(a * r for a, r in zip(i, rates)) if all(w == 8 for w in q) else 0.1)
    inst, quota, table = bench.Workload.refine(wl, [6, 9, 3], [8, 8, 8])
    allocs = {tuple(r["instances"]) for r in table}
    assert (5, 10, 3) in allocs
    assert (inst, quota) == ([4, 11, 3], [8, 8, 8])


def test_refine_adds_to_two_stages_at_once():
    # two stages limit the rate together: adding to either alone gains nothing
    rates = (1.0, 0.5, 0.5)
    wl = _FakeWorkload(lambda i, q: min(a * r for a, r in zip(i, rates)) if all(w == 8 for w in q) else 0.1)
    inst, quota, table = bench.Workload.refine(wl, [3, 4, 4], [8, 8, 8])
    assert quota == [8, 8, 8] and inst[1] > 4 and inst[2] > 4


def test_refine_tries_the_8_sm_split_of_wide_instances():
    # a pipeline in which two 8-SM instances beat one 16-SM instance
    wl = _FakeWorkload(lambda i, q: 1.0 + sum(a for a, w in zip(i, q) if w == 8))
    inst, quota, table = bench.Workload.refine(wl, [1, 16], [16, 8])
    allocs = {(tuple(r["instances"]), tuple(r["sm_quota"])) for r in table}
    assert ((1, 16), (16, 8)) in allocs and ((2, 16), (8, 8)) in allocs
    assert all(_total(a, q) <= 148 for a, q in allocs)
    assert quota == [8, 8] and _total(inst, quota) <= 148


def test_studies_report_failures_instead_of_failing(monkeypatch):
    # the compact study after the headline: its summary on success, its error
    # (and no exception) on failure
    def fake_ok(args, emit=True):
        assert args.diurnal == 12.0 and emit is False
        return {"value": 0.4, "unit": "fraction", "peak_qps": 1.0, "saturation_qps": 1.0, "static_alloc": {},
                "allocator_measured_over_predicted": 1.0, "sm_seconds": {"eq3": 1, "static": 2},
                "qos_violating_windows": {"eq3": 0, "static": 0}, "p99_ms_max": {"eq3": 0.1, "static": 0.1},
                "queries": 10, "clocks": {}, "config": {"load": "day"}, "windows_eq3": [1, 2, 3]}

    monkeypatch.setattr(bench, "run_diurnal", fake_ok)
    out = bench.run_studies()
    assert out["diurnal_fp8"]["value"] == 0.4 and out["diurnal_fp8"]["load"] == "day"
    assert "windows_eq3" not in out["diurnal_fp8"] and out["diurnal_fp8"]["seconds"] >= 0

    def fake_fail(args, emit=True):
        raise TimeoutError("trace did not drain")

    monkeypatch.setattr(bench, "run_diurnal", fake_fail)
    out = bench.run_studies()
    assert out["diurnal_fp8"]["error"] == "TimeoutError: trace did not drain"
