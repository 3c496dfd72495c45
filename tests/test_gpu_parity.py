"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle on
identical seeded inputs.  Integer work, so every comparison is bit-exact
(coefficient form, canonical residues)."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import bfv, pdq as opdq
from tests.gpu_common import Setup, coeff, library, to_dev, to_np

pytestmark = pytest.mark.gpu

SMALL = ["tiny", "tiny2", "grouped", "small", "c1"]


def brv(x, bits):
    return int(format(x, f"0{bits}b")[::-1], 2) if bits else 0


@pytest.fixture(scope="module", params=SMALL + ["c2", "paper", "tiny40"])
def setup(request):
    return Setup(request.param)


def test_prime_chain_matches_oracle(setup):
    par, ctx = setup.par, setup.ctx
    assert ctx.moduli == par.ext
    assert ctx.zeta == par.zeta
    for i, r in enumerate(par.ext):
        assert pow(ctx.psi[i], par.N, r) == r - 1
    plan = setup.plan.as_dict()
    op = setup.oplan
    for f in ("s_prime", "B", "J", "H", "G_sz", "hpg", "G", "per_out", "n_out"):
        assert plan[f] == getattr(op, f), f
    assert setup.galois == opdq.galois_elements(par, op)


def test_paper_table_shapes_plan_matches_oracle():
    """The library's plan for every shape of Tables II and III (Sec. 6.2;
    fixture paper_answer_size.txt) equals the oracle's, one output
    ciphertext each, with the same rotations."""
    from tests.test_oracle_pdq import golden_rows
    cfg = W.CONFIGS["paper"]
    par = bfv.Params.from_config(cfg)
    ctx = library().Context.from_config(cfg)
    for _, n, s, _ in golden_rows("paper_answer_size.txt"):
        op = opdq.make_plan(par, int(n), int(s))
        plan = ctx.plan(int(n), int(s))
        got = plan.as_dict()
        for f in ("s_prime", "B", "J", "H", "G_sz", "hpg", "G", "per_out", "n_out"):
            assert got[f] == getattr(op, f), (n, s, f)
        assert got["n_out"] == 1
        assert ctx.plan_galois(plan) == opdq.galois_elements(par, op)


# every transform decomposition: one CTA (N <= 2^12), column + row phases of
# 5..8 column levels (2^13 .. 2^16)
RINGS = {"tiny": W.CONFIGS["tiny"], "c1": W.CONFIGS["c1"], "c3": W.CONFIGS["c3"],
         "n13": (13, 65537, 60, 3, 1, 3), "n14": (14, 65537, 60, 4, 2, 2),
         "n16": (16, 786433, 60, 2, 1, 2)}


@pytest.mark.parametrize("cfg_name", list(RINGS))
def test_ntt_is_evaluation_in_bit_reversed_order(cfg_name):
    pdq = library()
    cfg = RINGS[cfg_name]
    if isinstance(cfg, tuple):
        par = bfv.Params(*cfg)
        ctx = pdq.Context(*cfg)
        cfg = type("Ring", (), {"log_n": cfg[0]})
    else:
        par = bfv.Params.from_config(cfg)
        ctx = pdq.Context.from_config(cfg)
    rng = np.random.default_rng(1)
    mods = par.ext + [par.t]
    a = np.stack([rng.integers(0, r, size=par.N, dtype=np.uint64) for r in mods])
    d = to_dev(a)
    ctx.ntt_forward(d, 1, len(mods))
    got = to_np(d).reshape(len(mods), par.N)
    perm = np.array([brv(k, cfg.log_n) for k in range(par.N)])
    from oracle import ring
    for l, r in enumerate(mods):
        want = ring.ntt_forward(a[l], r, ctx.psi[l])
        assert np.array_equal(got[l], want[perm]), l
    ctx.ntt_inverse(d, 1, len(mods))
    assert np.array_equal(to_np(d).reshape(a.shape), a)


def test_encode_matches_oracle(setup):
    par, ctx = setup.par, setup.ctx
    rng = np.random.default_rng(2)
    slots = rng.integers(0, par.t, size=(3, par.N)).astype(np.int32)
    pt = ctx.encode(torch.from_numpy(slots).cuda(), nlimbs=par.L + par.K)
    got = coeff(ctx, pt, par.L + par.K)
    for i in range(3):
        want = bfv.lift(par, bfv.encode(par, slots[i]), par.ext)
        assert np.array_equal(got[i], want)


def test_encryption_and_keys_bit_exact(setup):
    ctx = setup.ctx
    got = coeff(ctx, setup.v_cts, setup.par.L)
    for j, want in enumerate(setup.o_v_cts):
        assert np.array_equal(got[j], want)
    E = setup.par.L + setup.par.K
    keys = coeff(ctx, setup.keys.view(len(setup.galois), ctx.ndigits, 2, E, ctx.N), E)
    for i, k in enumerate(setup.galois[:4]):
        assert np.array_equal(keys[i], setup.o_keys[k]), k


def test_decrypt_matches_slots(setup):
    got = setup.ctx.decrypt(setup.sk, setup.v_cts).cpu().numpy()
    assert np.array_equal(got, setup.v_slots)


def test_rotations_bit_exact(setup):
    ctx, par = setup.ctx, setup.par
    ct = setup.v_cts[:1].contiguous()
    for k in setup.galois[:3] + setup.galois[-2:]:
        i = setup.galois.index(k)
        key = setup.keys.view(len(setup.galois), -1)[i]
        out = ctx.rotate(ct, k, key)
        want = bfv.rotate(par, setup.o_v_cts[0], k, setup.o_keys[k])
        assert np.array_equal(coeff(ctx, out, par.L)[0], want), k


def test_mask_bit_exact(setup):
    ctx, par = setup.ctx, setup.par
    got = coeff(ctx, ctx.mask(setup.plan, setup.v_cts, setup.db), par.L)
    want = opdq.mask(par, setup.o_v_cts, setup.q.db, setup.oplan)
    assert len(want) == got.shape[0]
    for i, w in enumerate(want):
        assert np.array_equal(got[i], w), i


def test_literal_mask_and_comp_bit_exact(setup):
    """The remark's literal order (d = v.DB, then the row masks) and Comp on
    its output, against the oracle's mask_literal and comp."""
    ctx, par = setup.ctx, setup.par
    dbp = ctx.db_encode_plain(torch.from_numpy(setup.q.db.astype(np.int32)).cuda())
    lit = ctx.mask_literal(setup.plan, setup.v_cts, dbp)
    want = opdq.mask_literal(par, setup.o_v_cts, setup.q.db, setup.oplan)
    got = coeff(ctx, lit, par.L)
    for i, w in enumerate(want):
        assert np.array_equal(got[i], w), i
    out = ctx.comp(setup.plan, lit, setup.keys, setup.galois, setup.consts)
    wc = opdq.comp(par, want, setup.o_keys, setup.oplan)
    gc = coeff(ctx, out, par.L)
    for c, w in enumerate(wc):
        assert np.array_equal(gc[c], w), c


def test_answer_bit_exact_and_decompresses(setup):
    ctx, par = setup.ctx, setup.par
    out = setup.answer()
    got = coeff(ctx, out, par.L)
    want = opdq.answer(par, setup.o_v_cts, setup.q.db, setup.o_keys, setup.oplan)
    assert got.shape[0] == len(want)
    for c, w in enumerate(want):
        assert np.array_equal(got[c], w), c
    slots = ctx.decrypt(setup.sk, out).cpu().numpy()
    exp = opdq.expected_slots(par, setup.oplan, setup.q.v, setup.q.db)
    for c in range(len(exp)):
        assert np.array_equal(slots[c].astype(np.uint64), exp[c])
    truth = [(int(i), int(setup.q.db[i])) for i in setup.q.positions]
    assert ctx.decomp(setup.plan, slots) == truth


def test_comp_alone_bit_exact(setup):
    """Comp on the masked ciphertexts (the pack of Sec. 5.2) against the
    oracle's comp; it decrypts to the same slots as the Answer, whose fused
    Mask and pack give other ciphertexts."""
    ctx, par = setup.ctx, setup.par
    masked = ctx.mask(setup.plan, setup.v_cts, setup.db)
    a = ctx.comp(setup.plan, masked, setup.keys, setup.galois, setup.consts)
    o_masked = opdq.mask(par, setup.o_v_cts, setup.q.db, setup.oplan)
    want = opdq.comp(par, o_masked, setup.o_keys, setup.oplan)
    got = coeff(ctx, a, par.L)
    for c, w in enumerate(want):
        assert np.array_equal(got[c], w), c
    sa = ctx.decrypt(setup.sk, a).cpu().numpy()
    sb = ctx.decrypt(setup.sk, setup.answer()).cpu().numpy()
    assert np.array_equal(sa, sb)


def test_answer_host_matches_device(setup):
    ctx, par = setup.ctx, setup.par
    v_host = torch.from_numpy(coeff(ctx, setup.v_cts, par.L).view(np.int64).copy()).pin_memory()
    out_host = torch.empty(setup.plan.n_out * ctx.ct_elems, dtype=torch.int64).pin_memory()
    ctx.answer_host(setup.plan, v_host, setup.db, setup.keys, setup.galois, setup.consts,
                    out_host)
    dev = coeff(ctx, setup.answer(), par.L)
    assert np.array_equal(out_host.numpy().view(np.uint64).reshape(dev.shape), dev)
