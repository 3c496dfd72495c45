"""Baby-step rotations under a memory budget: made and consumed a chunk of
primes at a time (pdq_ctx_set_rotation_budget), the Answer is the same bits
as with every rotation held at once, and its workspace is smaller."""
import pytest
import torch

from tests.gpu_common import Setup, library

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cfg_name,primes_per_chunk", [("small", 1), ("c1", 2), ("grouped", 1),
                                                       ("c2", 3)])
def test_budgeted_answer_is_bit_exact(cfg_name, primes_per_chunk):
    lib = library().load()
    st = Setup(cfg_name)
    ctx, plan = st.ctx, st.plan
    assert plan.B > 1
    full_ws = lib.pdq_answer_workspace_bytes(ctx.h, plan)
    want = st.answer().clone()
    one_prime = plan.H * plan.B * 2 * ctx.N * 8
    ctx.set_rotation_budget(primes_per_chunk * one_prime)
    try:
        ws = lib.pdq_answer_workspace_bytes(ctx.h, plan)
        # the rotations' region: [H][B][2][primes][N], at least 8 G ciphertexts over Q u P
        E, unit = ctx.E, 2 * ctx.N * 8
        region = lambda k: max(plan.H * plan.B * k, 8 * plan.G * E) * unit
        assert full_ws - ws == region(E) - region(primes_per_chunk) > 0
        got = st.answer()
        torch.cuda.synchronize()
        assert torch.equal(got, want)
        masked = ctx.mask(plan, st.v_cts, st.db)
        ctx.set_rotation_budget(0)
        ref = ctx.comp(plan, masked, st.keys, st.galois, st.consts)
        ctx.set_rotation_budget(primes_per_chunk * one_prime)
        assert torch.equal(ctx.comp(plan, masked, st.keys, st.galois, st.consts), ref)
    finally:
        ctx.set_rotation_budget(0)
