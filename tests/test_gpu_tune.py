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
