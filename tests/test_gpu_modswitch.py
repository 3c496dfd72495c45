"""Modulus switching (pdq_mod_switch) and the Answer with Comp on smaller
parameters: the switched ciphertexts and the whole switched answer bit for
bit against the oracle, and at the full benchmark size (N = 2^15, 8 primes
switched to 2) a switched ciphertext bit for bit and an answer that decrypts
to C v, C d and decompresses to exactly the matches."""
import numpy as np
import pytest

from oracle import bfv, pdq as opdq
from tests.gpu_common import Setup, coeff, library

pytestmark = pytest.mark.gpu


def _low(cfg_name, hi, L2):
    # digits no wider than P: dnum = ceil(L2 / K)
    return Setup(cfg_name, L=L2, dnum=-(-L2 // hi.par.K))


@pytest.mark.parametrize("cfg_name,L2", [("tiny2", 1), ("tiny2", 2), ("small", 2), ("c1", 1)])
def test_mod_switch_bit_exact(cfg_name, L2):
    hi = Setup(cfg_name)
    lo = _low(cfg_name, hi, L2)
    assert lo.ctx.moduli[:L2] == hi.ctx.moduli[:L2]
    sw = hi.ctx.mod_switch(lo.ctx, hi.v_cts)
    got = coeff(lo.ctx, sw, L2)
    for j, v in enumerate(hi.o_v_cts):
        assert np.array_equal(got[j], bfv.mod_switch(hi.par, lo.par, v)), j
    assert np.array_equal(lo.ctx.decrypt(lo.sk, sw).cpu().numpy(),
                          hi.ctx.decrypt(hi.sk, hi.v_cts).cpu().numpy())


@pytest.mark.parametrize("cfg_name", ["tiny2", "small"])
def test_switched_answer_bit_exact(cfg_name):
    hi = Setup(cfg_name)
    lo = _low(cfg_name, hi, 2)
    sw = hi.ctx.mod_switch(lo.ctx, hi.v_cts)
    out = lo.ctx.answer(lo.plan, sw, lo.db, lo.keys, lo.galois, lo.consts)
    want = opdq.answer_switched(hi.par, lo.par, hi.o_v_cts, hi.q.db, lo.o_keys, lo.oplan)
    got = coeff(lo.ctx, out, 2)
    assert got.shape[0] == len(want)
    for c, w in enumerate(want):
        assert np.array_equal(got[c], w), c
    slots = lo.ctx.decrypt(lo.sk, out).cpu().numpy()
    truth = [(int(i), int(hi.q.db[i])) for i in hi.q.positions]
    assert lo.ctx.decomp(lo.plan, slots) == truth
    # the answer switched to one prime before it leaves the server
    one = _low(cfg_name, hi, 1)
    out1 = lo.ctx.mod_switch(one.ctx, out)
    got1 = coeff(one.ctx, out1, 1)
    for c, w in enumerate(want):
        assert np.array_equal(got1[c], bfv.mod_switch(lo.par, one.par, w)), c
    assert one.ctx.decomp(one.plan, one.ctx.decrypt(one.sk, out1).cpu().numpy()) == truth


def test_mod_switch_refuses_unrelated_contexts():
    pdq = library()
    hi = Setup("tiny2")
    lo = _low("tiny2", hi, 2)
    with pytest.raises(pdq.PdqError):
        lo.ctx.mod_switch(hi.ctx, lo.v_cts)            # more primes
    other = Setup("tiny")                              # another ring
    with pytest.raises(pdq.PdqError):
        hi.ctx.mod_switch(other.ctx, hi.v_cts)


def test_c3_switched_answer():
    hi = Setup("c3")
    lo = Setup("c3", L=2, dnum=1)
    sw = hi.ctx.mod_switch(lo.ctx, hi.v_cts)
    got = coeff(lo.ctx, sw[:1].contiguous(), 2)[0]
    assert np.array_equal(got, bfv.mod_switch(hi.par, lo.par, hi.o_v_cts[0]))
    out = lo.ctx.answer(lo.plan, sw, lo.db, lo.keys, lo.galois, lo.consts)
    slots = lo.ctx.decrypt(lo.sk, out).cpu().numpy()
    exp = opdq.expected_slots(lo.par, lo.oplan, lo.q.v, lo.q.db)
    for c in range(len(exp)):
        assert np.array_equal(slots[c].astype(np.uint64), exp[c]), c
    truth = [(int(i), int(lo.q.db[i])) for i in lo.q.positions]
    assert lo.ctx.decomp(lo.plan, slots) == truth
    one = Setup("c3", L=1, dnum=1)
    out1 = lo.ctx.mod_switch(one.ctx, out)
    assert one.ctx.decomp(one.plan, one.ctx.decrypt(one.sk, out1).cpu().numpy()) == truth
