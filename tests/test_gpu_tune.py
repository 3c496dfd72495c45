"""The plan autotuner: it times every admissible baby-step split of a shape
through the C ABI, keeps the fastest, persists the choice, and the tuned plan
answers queries exactly."""
import json

import pytest

from paper_2408_17063_gb300 import tune
from tests.gpu_common import Setup

pytestmark = pytest.mark.gpu


def test_tuner_picks_the_fastest_admissible_split_and_persists_it(tmp_path):
    st = Setup("small")
    ctx, cfg = st.ctx, st.cfg
    cands = tune.candidates(ctx, cfg.n, cfg.s)
    assert cands == [1, 2, 4, 8, 16, 32]                  # s' = 32: every power of two
    path = tmp_path / "plans.json"
    tuner = tune.PlanTuner(str(path), reps=2)
    best = tuner.best(ctx, cfg.n, cfg.s)
    entry = json.loads(path.read_text())[tune.shape_key(ctx, cfg.n, cfg.s)]
    assert entry["B"] == best and set(entry["ms"]) == {str(b) for b in cands}
    assert entry["ms"][str(best)] == min(entry["ms"].values())
    # a second tuner reads the file instead of timing again
    again = tune.PlanTuner(str(path))
    again.time_answer = None
    assert again.best(ctx, cfg.n, cfg.s) == best
    # the tuned plan answers the query exactly
    tuned = Setup("small", B=best)
    slots = tuned.ctx.decrypt(tuned.sk, tuned.answer()).cpu().numpy()
    assert tuned.ctx.decomp(tuned.plan, slots) == [(int(i), int(tuned.q.db[i]))
                                                   for i in tuned.q.positions]


@pytest.mark.parametrize("cfg_name", ["c1", "grouped"])
def test_every_schedule_gives_the_same_bits(cfg_name):
    """The schedule knobs (transform phase split, multiply-accumulate tiles and
    staged baby steps) change launches, never results."""
    st = Setup(cfg_name)
    ctx = st.ctx
    ctx.set_schedule()
    want = st.answer().clone()
    rows = [r for r in tune.schedule_candidates(ctx, "ntt_row_bits") if r] or [0]
    for rb in rows:
        for mt in (1, 2, 8):
            for bc in (1, 4, 16):
                ctx.set_schedule(ntt_row_bits=rb, mac_tiles=mt, mac_bc=bc)
                assert ctx.schedule() == {"ntt_row_bits": rb, "mac_tiles": mt, "mac_bc": bc,
                                          "ntt_chunk": 0}
                assert st.answer().equal(want), (rb, mt, bc)
    for ch in (64, 100, 4096):                 # transforms in chunks (ragged last one)
        ctx.set_schedule(ntt_chunk=ch)
        assert st.answer().equal(want), ch
    ctx.set_schedule()


def test_schedules_at_the_large_ring_give_the_same_bits():
    """At N = 2^15 (8 + 2 primes, 4 digits) the raise and ModDown conversions
    ride on the transforms; chunked transforms and other splits keep the bits."""
    st = Setup("c3", n=1 << 16, s=64)
    ctx = st.ctx
    ctx.set_schedule()
    want = st.answer().clone()
    for kw in ({"ntt_chunk": 64}, {"ntt_chunk": 300}, {"ntt_row_bits": 8, "ntt_chunk": 1024},
               {"ntt_row_bits": 10}, {"mac_tiles": 1, "mac_bc": 2}):
        ctx.set_schedule(**kw)
        assert st.answer().equal(want), kw
    ctx.set_schedule()


def test_schedule_refuses_bad_knobs():
    from paper_2408_17063_gb300 import pdq
    ctx = Setup("c1").ctx
    for kw in ({"ntt_row_bits": 6}, {"ntt_row_bits": 12}, {"mac_tiles": 3}, {"mac_bc": 32},
               {"ntt_chunk": 8}):
        with pytest.raises(pdq.PdqError):
            ctx.set_schedule(**kw)
    ctx.set_schedule()


def test_schedule_tuner_keeps_the_fastest_and_persists_it(tmp_path):
    st = Setup("c1")
    ctx, cfg = st.ctx, st.cfg
    path = tmp_path / "sched.json"
    tuner = tune.ScheduleTuner(str(path), reps=2)
    hit = tuner.best(ctx, cfg.n, cfg.s)
    # the kept schedule is within the tuner's noise margin of the fastest tried
    assert hit["ms"] <= hit["default_ms"]
    assert min(hit["tried"].values()) >= hit["ms"] * (1 - tuner.min_gain) ** 3
    assert ctx.schedule() == hit["schedule"]
    saved = json.loads(path.read_text())
    assert [v["schedule"] for v in saved.values()] == [hit["schedule"]]
    ctx.set_schedule()
    again = tune.ScheduleTuner(str(path))
    assert again.best(ctx, cfg.n, cfg.s)["schedule"] == hit["schedule"]
    assert ctx.schedule() == hit["schedule"]
    ctx.set_schedule()
