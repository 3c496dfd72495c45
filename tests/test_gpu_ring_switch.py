"""Ring switching on the GPU (Sec. 5.3) against the oracle, through the C ABI:
the switching key, the switched parts of a ciphertext and whole Answers with
Comp in the subring (Mask in the big ring, pdq_ring_switch with group 4,
pdq_comp on the subring with a switched plan) bit for bit; the answers
decrypt and decompress to the matches."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import bfv, pdq as opdq
from tests.gpu_common import Setup, coeff, library, to_dev

pytestmark = pytest.mark.gpu

SEED = 0x5B


class Switched:
    """A Setup of the big ring plus its subring, keys made from the same
    draws on both sides."""

    def __init__(self, cfg_name, log_small, **kw):
        self.st = st = Setup(cfg_name, **kw)
        self.big = st.par
        self.small = bfv.Params.subring(self.big, log_small)
        self.sctx = st.ctx.subring(log_small)
        self.sk_small = W.draw_ternary(self.small.N, W.rng_for(SEED, 11))
        self.rs_rand = W.rotation_key_randomness(self.big.ext, self.big.N, len(self.big.digits),
                                                 [1], SEED, stream=12)[1]
        self.rsk = st.ctx.ring_switch_key_gen(self.sctx, st.sk,
                                              torch.from_numpy(self.sk_small),
                                              to_dev(self.rs_rand[0]),
                                              torch.from_numpy(self.rs_rand[1]))
        cfg = st.cfg
        self.plan = self.sctx.plan_switched(self.big.log_n, cfg.n, cfg.s)
        self.oplan = opdq.make_switched_plan(self.big, self.small, cfg.n, cfg.s)
        self.galois = self.sctx.plan_galois(self.plan)
        assert self.galois == opdq.galois_elements(self.small, self.oplan)
        self.key_rand = W.rotation_key_randomness(self.small.ext, self.small.N,
                                                  len(self.small.digits), self.galois, SEED,
                                                  stream=13)
        self.ssk = self.sctx.secret_prepare(torch.from_numpy(self.sk_small))
        keys = self.sctx._u64(len(self.galois) * self.sctx.key_elems)
        kv = keys.view(len(self.galois), -1)
        for i, k in enumerate(self.galois):
            a, e = self.key_rand[k]
            self.sctx.rotkey_gen(self.ssk, k, to_dev(a), torch.from_numpy(e).cuda(), out=kv[i])
        self.keys = keys
        self.consts = self.sctx.plan_constants(self.plan)
        torch.cuda.synchronize()

    def o_rsk(self):
        return bfv.ring_switch_key(self.big, self.st.q.sk, self.sk_small, *self.rs_rand)

    def o_keys(self):
        return {k: bfv.rotation_key(self.small, self.sk_small, k, *self.key_rand[k])
                for k in self.galois}

    def answer(self):
        st = self.st
        masked = st.ctx.mask(st.plan, st.v_cts, st.db)
        ms = st.ctx.ring_switch(self.sctx, masked, self.rsk, group=4)
        return self.sctx.comp(self.plan, ms, self.keys, self.galois, self.consts)


@pytest.mark.parametrize("cfg_name,log_small", [("tiny2", 5), ("tiny2", 4)])
def test_switching_key_and_parts_bit_exact(cfg_name, log_small):
    sw = Switched(cfg_name, log_small)
    st, big, small = sw.st, sw.big, sw.small
    got_key = coeff(st.ctx, sw.rsk.contiguous(), big.L + big.K)
    assert np.array_equal(got_key, sw.o_rsk())
    parts = st.ctx.ring_switch(sw.sctx, st.v_cts, sw.rsk)
    R = big.N // small.N
    got = coeff(sw.sctx, parts.contiguous(), small.L)
    for j, v in enumerate(st.o_v_cts):
        want = bfv.ring_switch(big, small, v, sw.o_rsk())
        for r in range(R):
            assert np.array_equal(got[j * R + r], want[r]), (j, r)
    # part r decrypts in the subring to the coefficients r mod R of the plaintext
    m = bfv.decrypt_coeffs(big, st.q.sk, st.o_v_cts[0])
    slots = sw.sctx.decrypt(sw.ssk, parts[:R].contiguous()).cpu().numpy()
    for r in range(R):
        assert np.array_equal(slots[r].astype(np.uint64), bfv.decode(small, m[r::R]))


@pytest.mark.parametrize("cfg_name,log_small,kw", [
    ("tiny2", 5, {}),
    ("tiny2", 4, {}),
    ("grouped", 4, {}),                 # several record groups and output ciphertexts
    ("tiny2", 4, dict(n=130, s=1)),     # s' = 1, ragged n
])
def test_switched_answer_bit_exact_and_decompresses(cfg_name, log_small, kw):
    sw = Switched(cfg_name, log_small, **kw)
    st = sw.st
    out = sw.answer()
    got = coeff(sw.sctx, out, sw.small.L)
    want = opdq.answer_ring_switched(sw.big, sw.small, st.o_v_cts, st.q.db, sw.o_rsk(),
                                     sw.o_keys(), sw.oplan)
    assert got.shape[0] == len(want)
    for c, w in enumerate(want):
        assert np.array_equal(got[c], w), c
    slots = sw.sctx.decrypt(sw.ssk, out).cpu().numpy()
    truth = [(int(i), int(st.q.db[i])) for i in st.q.positions]
    assert sw.sctx.decomp(sw.plan, slots) == truth


def test_ring_switch_refuses_unrelated_contexts():
    pdq = library()
    sw = Switched("tiny2", 4)
    other = pdq.Context(4, 12289, 60, 3, 2, 2)          # a ring of its own primes
    with pytest.raises(pdq.PdqError) as e:
        sw.st.ctx.ring_switch(other, sw.st.v_cts, sw.rsk)
    assert e.value.code == pdq.PDQ_E_PARAM
    with pytest.raises(pdq.PdqError):
        sw.st.ctx.subring(sw.st.ctx.log_n)
    with pytest.raises(pdq.PdqError):                   # 3 ciphertexts in groups of 4
        sw.st.ctx.ring_switch(sw.sctx, sw.st.v_cts[:1].repeat(3, 1, 1, 1).contiguous(), sw.rsk,
                              group=4)
