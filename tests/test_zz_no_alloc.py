"""pdq_rotate_noalloc: the rotation for callers that cannot allocate device
memory at the call site (external memory managers, hard memory budgets,
serving loops that must not synchronise on an allocation).  Its scratch is a
fixed library-owned device array, so the call allocates nothing; it must give
exactly the bits of pdq_rotate, call after call.  This file is collected last
so that a failure here comes after every other test has run."""
import numpy as np
import pytest
import torch

import workloads as W
from tests.gpu_common import library, to_dev

pytestmark = pytest.mark.gpu


def _one_key_setup(cfg_name, count):
    pdq = library()
    cfg = W.CONFIGS[cfg_name]
    ctx = pdq.Context.from_config(cfg)
    sk = ctx.secret_prepare(torch.from_numpy(W.draw_ternary(ctx.N, W.rng_for(cfg.seed, 3))))
    k = 2 * ctx.N - 1 if count % 2 else pow(3, 5, 2 * ctx.N)
    a, e = W.rotation_key_randomness(ctx.moduli, ctx.N, ctx.ndigits, [k], cfg.seed)[k]
    key = ctx.rotkey_gen(sk, k, to_dev(a), torch.from_numpy(e).cuda())
    ea, ee = W.encryption_randomness(ctx.moduli[:ctx.L], ctx.N, count, cfg.seed)
    slots = W.rng_for(cfg.seed, 9).integers(0, ctx.t, size=(count, ctx.N)).astype(np.int32)
    ct = ctx.encrypt(sk, torch.from_numpy(slots).cuda(), to_dev(ea), torch.from_numpy(ee).cuda())
    return pdq, ctx, sk, k, key, ct, slots


@pytest.mark.parametrize("cfg_name,count", [("c1", 4), ("c3", 1)])
def test_noalloc_rotation_matches_workspace_rotation(cfg_name, count):
    pdq, ctx, sk, k, key, ct, slots = _one_key_setup(cfg_name, count)
    want = ctx.rotate(ct, k, key)
    out = torch.empty_like(ct)
    for _ in range(2):                       # two calls in a row share the scratch
        out.zero_()
        ctx.rotate_noalloc(ct, k, key, out=out)
        torch.cuda.synchronize()
        assert torch.equal(out, want)
    # and it decrypts to the rotated slots
    dec = ctx.decrypt(sk, out).cpu().numpy().reshape(count, 2, ctx.m)
    rows = slots.reshape(count, 2, ctx.m)
    if k == 2 * ctx.N - 1:
        assert np.array_equal(dec, rows[:, ::-1, :])
    else:
        assert np.array_equal(dec, np.roll(rows, -5, axis=2))


def test_noalloc_rejects_oversize_batches():
    pdq, ctx, sk, k, key, ct, slots = _one_key_setup("c3", 1)
    lib = pdq.load()
    limit = lib.pdq_rotate_noalloc_max_bytes()
    assert limit == 32 << 20
    too_many = 1
    while lib.pdq_rotate_workspace_bytes(ctx.h, too_many) <= limit:
        too_many += 1
    big = ct.repeat(too_many, 1, 1, 1).contiguous()
    with pytest.raises(pdq.PdqError) as e:
        ctx.rotate_noalloc(big, k, key)
    assert e.value.code == pdq.PDQ_E_PARAM
    assert "scratch" in str(e.value)
