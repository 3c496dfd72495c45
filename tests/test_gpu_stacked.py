"""Queries of one plan answered together (pdq_answer_stacked): every step of
Mask and Comp is one launch over all queries' ciphertexts, with each query's
own rotation keys and the shared database and plan constants (Sec. 5.2's
schedule unchanged per query).  Each query's output must be bit-identical to
its pdq_answer alone and decrypt and decompress to its matches; the call
writes nothing outside its output and workspace."""
import numpy as np
import pytest
import torch

from oracle import pdq as opdq
from tests.gpu_common import Setup, library

pytestmark = pytest.mark.gpu


def _queries(cfg_name, Q, **kw):
    base = Setup(cfg_name, **kw)
    rest = [Setup(cfg_name, seed=base.seed + 101 * i, ctx=base.ctx, **kw) for i in range(1, Q)]
    return base, [base] + rest


@pytest.mark.parametrize("cfg_name,Q,kw", [
    ("tiny", 2, {}),                      # ring below one rotation tile (per-rotation path)
    ("tiny2", 3, {}),
    ("small", 4, {}),
    ("c1", 2, {}),
    ("grouped", 3, {}),                   # 8 record groups, two outputs per query
    ("grouped", 2, {"n": 1700}),          # a partial last group and a partial output
    ("small", 8, {}),
])
def test_stacked_answers_equal_alone(cfg_name, Q, kw):
    base, sets = _queries(cfg_name, Q, **kw)
    ctx, plan = base.ctx, base.plan
    v = torch.cat([st.v_cts.reshape(-1) for st in sets])
    got = ctx.answer_stacked(plan, v, base.db, [st.keys for st in sets], base.galois, base.consts)
    assert tuple(got.shape) == (Q, plan.n_out, 2, ctx.L, ctx.N)
    for i, st in enumerate(sets):
        alone = ctx.answer(plan, st.v_cts, base.db, st.keys, base.galois, base.consts)
        assert torch.equal(got[i], alone), f"query {i} differs from its answer alone"
        dec = ctx.decrypt(st.sk, got[i]).cpu().numpy()
        # every query is answered over base's database
        truth = [(int(p), int(base.q.db[p])) for p in st.q.positions]
        assert ctx.decomp(plan, dec) == truth
        exp = opdq.expected_slots(base.par, base.oplan, st.q.v, base.q.db)
        assert all(np.array_equal(a, b) for a, b in zip(dec, exp))


def test_stacked_writes_only_its_buffers():
    lib = library().load()
    base, sets = _queries("grouped", 3)
    ctx, plan = base.ctx, base.plan
    guard, pattern = 1 << 14, 0x1234_5678_9ABC_DEF0
    Q = len(sets)
    wsn = lib.pdq_answer_stacked_workspace_bytes(ctx.h, plan, Q) // 8
    ws = torch.full((wsn + 2 * guard,), pattern, dtype=torch.int64, device="cuda")
    out = torch.full((Q * plan.n_out * ctx.ct_elems + 2 * guard,), pattern, dtype=torch.int64,
                     device="cuda")
    v = torch.cat([st.v_cts.reshape(-1) for st in sets])
    before = [t.clone() for t in (v, base.db, base.consts, *[st.keys for st in sets])]
    got = ctx.answer_stacked(plan, v, base.db, [st.keys for st in sets], base.galois,
                             base.consts, ws=ws[guard:guard + wsn].view(torch.uint8),
                             out=out[guard:-guard])
    torch.cuda.synchronize()
    for t in (ws, out):
        assert bool((t[:guard] == pattern).all()) and bool((t[-guard:] == pattern).all())
    after = (v, base.db, base.consts, *[st.keys for st in sets])
    assert all(torch.equal(a, b) for a, b in zip(before, after))
    for i, st in enumerate(sets):
        alone = ctx.answer(plan, st.v_cts, base.db, st.keys, base.galois, base.consts)
        assert torch.equal(got[i], alone)


def test_stacked_refuses_bad_arguments():
    pdq = library()
    base, sets = _queries("tiny2", 2)
    ctx, plan = base.ctx, base.plan
    v = torch.cat([st.v_cts.reshape(-1) for st in sets])
    keys = [st.keys for st in sets]
    with pytest.raises(pdq.PdqError, match="null key"):
        ctx.answer_stacked(plan, v, base.db, [keys[0], None], base.galois, base.consts)
    with pytest.raises(pdq.PdqError, match="1 to 64"):
        ctx.answer_stacked(plan, v, base.db, keys * 33, base.galois, base.consts,
                           ws=ctx.answer_stacked_workspace(plan, 2))
    small = ctx.answer_stacked_workspace(plan, 1)
    with pytest.raises(pdq.PdqError, match="workspace"):
        ctx.answer_stacked(plan, v, base.db, keys, base.galois, base.consts, ws=small)


def test_stacked_under_rotation_budget_and_schedule():
    """Stacked queries with the baby-step rotations made a prime at a time (a
    rotation budget) and a non-default launch schedule: still each query's
    answer alone (taken with the defaults)."""
    base, sets = _queries("c1", 3)
    ctx, plan = base.ctx, base.plan
    want = [ctx.answer(plan, st.v_cts, base.db, st.keys, base.galois, base.consts).clone()
            for st in sets]
    v = torch.cat([st.v_cts.reshape(-1) for st in sets])
    try:
        ctx.set_rotation_budget(1)            # one prime's rotations at a time
        ctx.set_schedule(ntt_row_bits=8, mac_tiles=1, mac_bc=4)
        got = ctx.answer_stacked(plan, v, base.db, [st.keys for st in sets], base.galois,
                                 base.consts)
        for i in range(len(sets)):
            assert torch.equal(got[i], want[i]), f"query {i}"
    finally:
        ctx.set_rotation_budget(0)
        ctx.set_schedule()
