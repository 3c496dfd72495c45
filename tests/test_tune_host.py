"""Host logic of the autotuners, without a GPU: a fake context and a fake
timing rig stand in for the library, so the schedule tuner's coordinate
descent, noise margin and persisted choice, and the plan tuner's search over
the library's admissible baby-step splits, are checked on the CPU."""
import json

import pytest

pytest.importorskip("torch")
from paper_2408_17063_gb300 import tune  # noqa: E402


class FakeCtx:
    N, L, K, ndigits, t, moduli, log_n = 1 << 15, 8, 2, 4, 65537, [97], 15

    def __init__(self):
        self.sched = {k: 0 for k in tune.SCHEDULE_KNOBS}
        self.calls = []

    def set_schedule(self, **kw):
        self.sched = {k: kw.get(k, 0) for k in tune.SCHEDULE_KNOBS}
        self.calls.append(dict(self.sched))

    def schedule(self):
        return dict(self.sched)


def fake_rig(costs):
    """AnswerRig stand-in whose time is the default plus per-knob deltas."""
    class Rig:
        def __init__(self, ctx, n, s, B=0, stream=None):
            self.ctx = ctx

        def time(self, reps=3):
            return 10.0 + sum(costs.get((k, v), 0.0) for k, v in self.ctx.sched.items())

        def close(self):
            pass
    return Rig


def test_descent_keeps_gains_above_the_margin_and_persists(tmp_path, monkeypatch):
    # row bits 8 saves 0.5 (5%), tiles 2 saves 0.05 (0.5%: noise), bc 8 costs
    costs = {("ntt_row_bits", 8): -0.5, ("mac_tiles", 2): -0.05, ("mac_bc", 8): 0.3}
    monkeypatch.setattr(tune, "AnswerRig", fake_rig(costs))
    ctx = FakeCtx()
    path = tmp_path / "s.json"
    hit = tune.ScheduleTuner(str(path), reps=1).best(ctx, 1 << 20, 256, 32)
    assert hit["schedule"] == {"ntt_row_bits": 8, "mac_tiles": 0, "mac_bc": 0, "ntt_chunk": 0}
    assert hit["default_ms"] == 10.0 and hit["ms"] == pytest.approx(9.5)
    assert ctx.schedule() == hit["schedule"]
    # every knob's candidates were tried once each (no repeats of a schedule)
    assert len(hit["tried"]) == len(set(hit["tried"]))
    assert len(hit["tried"]) == 1 + sum(len(tune.schedule_candidates(ctx, k)) - 1
                                        for k in tune.SCHEDULE_KNOBS)
    saved = json.loads(path.read_text())
    assert list(saved.values())[0]["schedule"] == hit["schedule"]
    # a second tuner reads the file and sets the context without timing
    monkeypatch.setattr(tune, "AnswerRig", None)
    ctx2 = FakeCtx()
    assert tune.ScheduleTuner(str(path)).best(ctx2, 1 << 20, 256, 32)["schedule"] == hit["schedule"]
    assert ctx2.schedule() == hit["schedule"]


def test_row_split_candidates_follow_the_ring():
    ctx = FakeCtx()
    assert tune.schedule_candidates(ctx, "ntt_row_bits") == [0, 8, 9, 10]
    ctx.log_n = 12                      # both phases at most 2^11: row levels 1..11 of 12
    assert tune.schedule_candidates(ctx, "ntt_row_bits") == [0, 8, 9, 10]
    ctx.log_n = 9                       # one-phase transforms: no split to tune
    assert tune.schedule_candidates(ctx, "ntt_row_bits") == [0]


class FakePlanCtx(FakeCtx):
    def plan(self, n, s, B=0):
        from paper_2408_17063_gb300 import pdq
        return pdq.plan_make_client(self.t, self.log_n, n, s, B)


def test_plan_candidates_are_the_library_admissible_splits():
    """The tuner searches exactly the B the library accepts for a shape: the
    powers of two that divide s', at most 128, with at most 32 giant steps."""
    from paper_2408_17063_gb300 import pdq
    ctx = FakePlanCtx()
    for s in (1, 3, 16, 100, 256, 1024, 4096, 16384):
        sp = 1 << (s - 1).bit_length()
        accepted = []
        for b in (1 << i for i in range(sp.bit_length())):
            try:
                pdq.plan_make_client(ctx.t, ctx.log_n, 1 << 20, s, b)
                accepted.append(b)
            except pdq.PdqError:
                pass
        assert tune.candidates(ctx, 1 << 20, s) == accepted, s


def test_plan_tuner_keeps_the_fastest_split_and_persists(tmp_path, monkeypatch):
    ms = {1: 9.0, 2: 7.0, 4: 5.0, 8: 5.0, 16: 6.0, 32: 8.0}   # a tie: the smaller B wins
    timed = []

    def fake_time(self, ctx, n, s, B, stream=None):
        timed.append(B)
        return ms[B]

    monkeypatch.setattr(tune.PlanTuner, "time_answer", fake_time)
    ctx = FakePlanCtx()
    path = tmp_path / "plans.json"
    tuner = tune.PlanTuner(str(path))
    assert tuner.best(ctx, 1 << 16, 32) == 4
    assert sorted(timed) == tune.candidates(ctx, 1 << 16, 32) == [1, 2, 4, 8, 16, 32]
    entry = json.loads(path.read_text())[tune.shape_key(ctx, 1 << 16, 32)]
    assert entry["B"] == 4 and entry["default_B"] == ctx.plan(1 << 16, 32).B
    # a new tuner on the same file answers without timing
    timed.clear()
    assert tune.PlanTuner(str(path)).best(ctx, 1 << 16, 32) == 4 and timed == []
    # another sparsity with the same padded s' is the same shape
    assert tune.PlanTuner(str(path)).best(ctx, 1 << 16, 20) == 4 and timed == []
