"""The Answer on an unencrypted database (Sec. 5.2 remark, [C; C diag(DB)] v
with no Mask) on the GPU against the oracle, through the C ABI: bit for bit
on configurations with one and several giant steps and record groups, and
the answers decrypt and decompress to the matches."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import bfv, pdq as opdq
from tests.gpu_common import Setup, coeff, library, to_dev

pytestmark = pytest.mark.gpu


def _keys(st, galois):
    ctx = st.ctx
    rand = W.rotation_key_randomness(st.par.ext, st.par.N, len(st.par.digits), galois, st.seed)
    keys = ctx._u64(len(galois) * ctx.key_elems)
    kv = keys.view(len(galois), -1)
    for i, k in enumerate(galois):
        a, e = rand[k]
        ctx.rotkey_gen(st.sk, k, to_dev(a), torch.from_numpy(e).cuda(), out=kv[i])
    o_keys = {k: bfv.rotation_key(st.par, st.q.sk, k, *rand[k]) for k in galois}
    return keys, o_keys


@pytest.mark.parametrize("cfg_name,B", [("tiny", 0), ("tiny2", 2), ("grouped", 2), ("c1", 4),
                                        ("small", 0)])
def test_answer_plain_db_bit_exact_and_decompresses(cfg_name, B):
    st = Setup(cfg_name)
    cfg, par, ctx = st.cfg, st.par, st.ctx
    plan = ctx.plan_plain_db(cfg.n, cfg.s, B)
    oplan = opdq.make_plan_plain_db(par, cfg.n, cfg.s, B or None)
    assert (plan.B, plan.giants, plan.G, plan.n_out, plan.plain_db) == (
        oplan.B, oplan.giants, oplan.G, oplan.n_out, 1)
    galois = ctx.plan_galois(plan)
    assert galois == opdq.plain_db_galois_elements(par, oplan)
    keys, o_keys = _keys(st, galois)
    consts = ctx.db_diagonals(plan, torch.from_numpy(st.q.db.astype(np.int32)))
    out = ctx.answer_plain_db(plan, st.v_cts, keys, galois, consts)
    got = coeff(ctx, out.contiguous(), par.L)
    want = opdq.answer_plain_db(par, st.o_v_cts, st.q.db, o_keys, oplan)
    for c, w in enumerate(want):
        assert np.array_equal(got[c], w), c
    slots = ctx.decrypt(st.sk, out).cpu().numpy()
    truth = [(int(i), int(st.q.db[i])) for i in st.q.positions]
    assert ctx.decomp(plan, slots) == truth


def test_answer_plain_db_refuses_other_plans_and_missing_keys():
    pdq = library()
    st = Setup("tiny2")
    ctx = st.ctx
    plan = ctx.plan_plain_db(st.cfg.n, st.cfg.s, 2)
    galois = ctx.plan_galois(plan)
    keys, _ = _keys(st, galois)
    consts = ctx.db_diagonals(plan, torch.from_numpy(st.q.db.astype(np.int32)))
    with pytest.raises(pdq.PdqError) as e:               # a plan of the masked Answer
        ctx.answer_plain_db(st.plan, st.v_cts, keys, galois, consts)
    assert e.value.code == pdq.PDQ_E_PARAM
    with pytest.raises(pdq.PdqError) as e:               # the folded Rot_col key missing
        k = [g for g in galois if g not in ctx.plan_galois(ctx.plan(st.cfg.n, st.cfg.s, 2))]
        assert k
        drop = galois.index(k[0])
        kv = keys.view(len(galois), -1)
        sub = torch.cat([kv[:drop], kv[drop + 1:]]).contiguous()
        ctx.answer_plain_db(plan, st.v_cts, sub, galois[:drop] + galois[drop + 1:], consts)
    assert e.value.code == pdq.PDQ_E_KEY
