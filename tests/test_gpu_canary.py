"""Out-of-bounds writes, checked without a sanitizer: every buffer the library
writes (the Answer's output and workspace, the ring switch's and the
unencrypted-database Answer's) sits inside a larger allocation whose guard
regions before and after it hold a known pattern, and every input (index
ciphertexts, database plaintexts, keys, plan constants) is compared with a
copy taken before the call.  A write past either end of a buffer, or into an
input, changes a guard or an input and fails the test."""
import numpy as np
import pytest
import torch

from tests.gpu_common import Setup, library

pytestmark = pytest.mark.gpu

GUARD = 1 << 16             # uint64 words before and after each written buffer
PATTERN = 0x5A5A_C3C3_0F0F_A5A5


class Guarded:
    """A buffer of n words with guard regions on both sides."""

    def __init__(self, n: int):
        self.full = torch.full((int(n) + 2 * GUARD,), PATTERN, dtype=torch.int64, device="cuda")
        self.buf = self.full[GUARD:GUARD + int(n)]

    def intact(self) -> bool:
        torch.cuda.synchronize()
        return bool((self.full[:GUARD] == PATTERN).all()) and \
            bool((self.full[-GUARD:] == PATTERN).all())


def _snap(*ts):
    return [t.clone() for t in ts]


@pytest.mark.parametrize("cfg_name", ["tiny2", "grouped", "c1"])
def test_answer_writes_only_its_output_and_workspace(cfg_name):
    lib = library().load()
    st = Setup(cfg_name)
    ctx, plan = st.ctx, st.plan
    want = st.answer().clone()
    ws = Guarded(lib.pdq_answer_workspace_bytes(ctx.h, plan) // 8)
    out = Guarded(plan.n_out * ctx.ct_elems)
    inputs = [st.v_cts, st.db, st.keys, st.consts]
    before = _snap(*inputs)
    ctx.answer(plan, st.v_cts, st.db, st.keys, st.galois, st.consts,
               ws=ws.buf.view(torch.uint8), out=out.buf)
    assert ws.intact() and out.intact()
    assert all(torch.equal(a, b) for a, b in zip(inputs, before))
    assert torch.equal(out.buf.view(want.shape), want)


def test_ring_switch_and_plain_db_write_only_their_buffers():
    lib = library().load()
    st = Setup("tiny2")
    ctx = st.ctx
    small = ctx.subring(4)
    rsk = torch.zeros(ctx.key_elems, dtype=torch.int64, device="cuda")     # any key: bounds only
    n = st.v_cts.numel() // ctx.ct_elems
    R = ctx.N // small.N
    ws = Guarded(lib.pdq_ring_switch_workspace_bytes(ctx.h, n) // 8)
    out = Guarded(n * R * small.ct_elems)
    before = _snap(st.v_cts, rsk)
    ctx.ring_switch(small, st.v_cts, rsk, out=out.buf, ws=ws.buf.view(torch.uint8))
    assert ws.intact() and out.intact()
    assert all(torch.equal(a, b) for a, b in zip([st.v_cts, rsk], before))
    # the Answer on an unencrypted database
    plan = ctx.plan_plain_db(st.cfg.n, st.cfg.s, 2)
    galois = ctx.plan_galois(plan)
    keys = torch.zeros(len(galois) * ctx.key_elems, dtype=torch.int64, device="cuda")
    consts = ctx.db_diagonals(plan, torch.from_numpy(st.q.db.astype(np.int32)))
    ws = Guarded(lib.pdq_answer_plain_db_workspace_bytes(ctx.h, plan) // 8)
    out = Guarded(plan.n_out * ctx.ct_elems)
    before = _snap(st.v_cts, keys, consts)
    ctx.answer_plain_db(plan, st.v_cts, keys, galois, consts, ws=ws.buf.view(torch.uint8),
                        out=out.buf)
    assert ws.intact() and out.intact()
    assert all(torch.equal(a, b) for a, b in zip([st.v_cts, keys, consts], before))
