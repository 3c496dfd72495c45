"""Host logic of the schedule autotuner, without a GPU: a fake context and a
fake timing rig stand in for the library, so the coordinate descent, the
noise margin and the persisted choice are checked on the CPU."""
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
