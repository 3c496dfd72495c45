"""Pins for the oracle's Answer on an unencrypted database (Sec. 5.2, remark:
C (DB . v) = (C diag(DB)) v, so the server compresses v alone with
[C; C diag(DB)] and skips Mask).  The two diagonal sets, the row exchange
folded into the giant steps and the rotate-and-sum are pinned in the clear
against the power sums of Eq. 1 with Python integers; whole Answers against
the closed form and Decomp, with one and with several giant steps."""
import numpy as np
import pytest

import workloads as W
from oracle import bfv, pdq


def test_plan_cost_rule_by_hand():
    # c3: J = 32, G = 16, s' = 256; J(B-1) + 8G(2s'/B - 1) + 6G s'/B:
    #   B=32: 992 + 1920 + 768 = 3680, B=64: 2016 + 896 + 384 = 3296,
    #   B=128: 4064 + 384 + 192 = 4640  ->  B = 64, 4 giant steps
    cfg = W.CONFIGS["c3"]
    par = bfv.Params.from_config(cfg)
    plan = pdq.make_plan_plain_db(par, cfg.n, cfg.s)
    assert (plan.J, plan.G, plan.s_prime, plan.B, plan.giants) == (32, 16, 256, 64, 4)


def test_galois_elements_include_the_folded_column_rotation():
    cfg = W.CONFIGS["tiny2"]
    par = bfv.Params.from_config(cfg)
    plan = pdq.make_plan_plain_db(par, cfg.n, cfg.s, 2)
    ks = pdq.plain_db_galois_elements(par, plan)
    col = 2 * par.N - 1
    for g in range(1, plan.giants):
        r = pow(3, g * plan.B, 2 * par.N)
        assert r in ks and r * col % (2 * par.N) in ks
    assert col in ks and pow(3, 1, 2 * par.N) in ks


def _swap(par, x):
    return np.asarray(x).reshape(2, par.m)[::-1].reshape(-1)


@pytest.mark.parametrize("cfg_name,B", [("tiny", None), ("tiny2", 2), ("grouped", 2)])
def test_plain_db_bsgs_in_the_clear(cfg_name, B):
    """Both diagonal sets, the giant steps (set 1 through Rot_col) and the
    rotate-and-sum applied to random index slots give, per group, the power
    sums of v (row 0) and of DB . v (row 1) over its records."""
    cfg = W.CONFIGS[cfg_name]
    par = bfv.Params.from_config(cfg)
    plan = pdq.make_plan_plain_db(par, cfg.n, cfg.s, B)
    t, m, sp = par.t, par.m, plan.s_prime
    rng = np.random.default_rng(11)
    db = rng.integers(0, t, size=cfg.n, dtype=np.uint64)
    v = [rng.integers(0, t, size=par.N, dtype=np.uint64) for _ in range(plan.J)]
    jpg = plan.hpg // 2
    for gamma in range(plan.G):
        y = np.zeros(par.N, dtype=np.uint64)
        for sigma in range(2):
            for g in range(plan.giants):
                acc = np.zeros(par.N, dtype=np.uint64)
                for j in range(gamma * jpg, min((gamma + 1) * jpg, plan.J)):
                    for a in range(plan.B):
                        d = pdq.rot_slots(par, pdq.plain_db_diagonal_slots(
                            par, plan, db, j, sigma, g * plan.B + a), -g * plan.B)
                        acc = (acc + d * pdq.rot_slots(par, v[j], a)) % t
                term = pdq.rot_slots(par, acc, g * plan.B)
                y = (y + (_swap(par, term) if sigma else term)) % t
        for l, r in pdq.rotsum_levels(par, plan):
            y = sum(pdq.rot_slots(par, y, jj * l) for jj in range(r)) % t
        wv, wd = [0] * sp, [0] * sp
        for i in range(gamma * plan.G_sz, min((gamma + 1) * plan.G_sz, plan.J * par.N)):
            val = int(v[i // par.N][i % par.N])
            dbi = int(db[i]) if i < cfg.n else 0
            node = i % plan.G_sz + 1
            for k in range(sp):
                p = pow(node, k + 1, t)
                wv[k] = (wv[k] + p * val) % t
                wd[k] = (wd[k] + p * val * dbi) % t
        assert y[:sp].tolist() == wv
        assert y[m:m + sp].tolist() == wd


@pytest.mark.parametrize("cfg_name,B", [("tiny", None), ("tiny2", None), ("tiny2", 2),
                                        ("grouped", 2), ("c1", 4)])
def test_answer_plain_db_decrypts_and_decompresses(cfg_name, B):
    cfg = W.CONFIGS[cfg_name]
    par = bfv.Params.from_config(cfg)
    q = W.draw_query(cfg)
    plan = pdq.make_plan_plain_db(par, cfg.n, cfg.s, B)
    a, e = W.encryption_randomness(par.q, par.N, plan.J, cfg.seed)
    v = pdq.encrypt_index(par, q.sk, q.v, plan, a, e)
    gal = pdq.plain_db_galois_elements(par, plan)
    kr = W.rotation_key_randomness(par.ext, par.N, len(par.digits), gal, cfg.seed)
    keys = {k: bfv.rotation_key(par, q.sk, k, *kr[k]) for k in gal}
    out = pdq.answer_plain_db(par, v, q.db, keys, plan)
    slots = [bfv.decrypt(par, q.sk, o) for o in out]
    for got, want in zip(slots, pdq.expected_slots(par, plan, q.v, q.db)):
        assert np.array_equal(got, want)
    assert pdq.decomp_slots(par, plan, slots) == [(int(i), int(q.db[i])) for i in q.positions]
    assert min(bfv.noise_budget_bits(par, q.sk, o) for o in out) > 10
