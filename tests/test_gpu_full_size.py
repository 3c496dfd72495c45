"""GPU checks at the full benchmark size (N = 2^15, n = 2^20 records, s = 256
clustered matches, the launch configuration the benchmark times) and edge
cases.  The whole oracle answer is too slow at this size, so the answer is
checked through properties that hold at any size (it decrypts to C v and C d
from Eq. 1, computed straight in Z_t, and decompresses to exactly the
matches), and single steps are compared bit for bit with the oracle on
sampled ciphertexts."""
import numpy as np
import pytest
import torch

from oracle import bfv, pdq as opdq
from tests.gpu_common import Setup, coeff, library

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c3():
    return Setup("c3")


def test_c3_answer_decrypts_to_closed_form_and_decompresses(c3):
    out = c3.answer()
    slots = c3.ctx.decrypt(c3.sk, out).cpu().numpy()
    exp = opdq.expected_slots(c3.par, c3.oplan, c3.q.v, c3.q.db)
    assert slots.shape[0] == len(exp) == 1
    assert np.array_equal(slots[0].astype(np.uint64), exp[0])
    truth = [(int(i), int(c3.q.db[i])) for i in c3.q.positions]
    assert c3.ctx.decomp(c3.plan, slots) == truth
    # deterministic: a second run gives the same bits
    assert torch.equal(out, c3.answer())


def test_c3_sampled_steps_bit_exact(c3):
    ctx, par = c3.ctx, c3.par
    # the first index ciphertext, its four masked ciphertexts and a rotation
    v0 = c3.o_v_cts[0]
    assert np.array_equal(coeff(ctx, c3.v_cts[:1].contiguous(), par.L)[0], v0)
    masked = ctx.mask(c3.plan, c3.v_cts, c3.db)
    got = coeff(ctx, masked[:4].contiguous(), par.L)
    top, bot = opdq.row_mask_slots(par, 0), opdq.row_mask_slots(par, 1)
    dbs = opdq.record_slots(par, c3.q.db, 0)
    pts = [top, bot, dbs * top, dbs * bot]
    for i in range(4):
        assert np.array_equal(got[i], bfv.pt_mul(par, v0, opdq.lifted_pt(par, pts[i])))
    k = 2 * par.N - 1
    i = c3.galois.index(k)
    key_o = bfv.rotation_key(par, c3.q.sk, k, *c3.key_rand[k])
    out = ctx.rotate(c3.v_cts[:1].contiguous(), k, c3.keys.view(len(c3.galois), -1)[i])
    assert np.array_equal(coeff(ctx, out, par.L)[0], bfv.rotate(par, v0, k, key_o))


@pytest.mark.parametrize("kw", [
    dict(cfg_name="tiny2", s=1),                 # s' = 1: one giant, no baby rotations
    dict(cfg_name="tiny2", s=32),                # s' = m: no rotate-and-sum
    dict(cfg_name="tiny2", s=5, B=8),            # one giant step, all baby steps
    dict(cfg_name="tiny2", s=5, B=1),            # no baby steps
    dict(cfg_name="tiny", n=1, s=1),             # a single record
    dict(cfg_name="grouped", n=257, s=2),        # a second group with one record
    dict(cfg_name="tiny2", n=300, s=32, B=32),   # 320 products per accumulator (wide fold)
    dict(cfg_name="small", n=2000, s=9),         # 4 half-blocks: rotation CTAs of 4
    dict(cfg_name="small", n=3500, s=9),         # 8 half-blocks: rotation CTAs of 8
    dict(cfg_name="c1", n=8000, s=20),           # 4 half-blocks at a two-phase ring
])
def test_edge_cases_bit_exact(kw):
    name = kw.pop("cfg_name")
    B = kw.pop("B", 0)
    st = Setup(name, B=B, **kw)
    par = st.par
    got = coeff(st.ctx, st.answer(), par.L)
    want = opdq.answer(par, st.o_v_cts, st.q.db, st.o_keys, st.oplan)
    for c, w in enumerate(want):
        assert np.array_equal(got[c], w)
    slots = st.ctx.decrypt(st.sk, st.answer()).cpu().numpy()
    truth = [(int(i), int(st.q.db[i])) for i in st.q.positions]
    assert st.ctx.decomp(st.plan, slots) == truth


def test_errors_are_reported():
    pdq = library()
    st = Setup("tiny")
    ctx = st.ctx
    with pytest.raises(pdq.PdqError) as e:
        ctx.answer(st.plan, st.v_cts, st.db, st.keys, st.galois[1:], st.consts)
    assert e.value.code == pdq.PDQ_E_KEY
    with pytest.raises(pdq.PdqError) as e:
        ctx.answer(st.plan, st.v_cts, st.db, st.keys, st.galois, st.consts,
                   ws=torch.empty(16, dtype=torch.uint8, device="cuda"))
    assert e.value.code == pdq.PDQ_E_NOMEM
    with pytest.raises(pdq.PdqError) as e:
        ctx.plan(100, ctx.m + 1)
    assert e.value.code == pdq.PDQ_E_PARAM
    with pytest.raises(pdq.PdqError):
        pdq.Context(12, 40960, 54, 2, 1, 2)      # t not prime
    # decomp rejects inconsistent slots
    bad = np.zeros((st.plan.n_out, ctx.N), dtype=np.uint32)
    bad[0, 0] = 5
    bad[0, ctx.m] = 1
    bad[0, 1] = 7
    with pytest.raises(pdq.PdqError) as e:
        ctx.decomp(st.plan, bad)
    assert e.value.code == pdq.PDQ_E_DECODE
