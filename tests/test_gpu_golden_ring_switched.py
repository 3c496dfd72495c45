"""Bit-exact ring-switched Answer at the full-size rings.

The oracle's Answer with Comp in the subring (Mask in the ring 2^15, ring
switching to 2^13, Comp there; Sec. 5.2, 5.3) over 2 + 2 primes with one
digit, n = 2^17, s = 256 is stored in
``tests/golden/answer_ring_switched_15to13_L2K2_n131072_s256.txt`` (written by
``tests/golden/make_answer_ring_switched.py`` from the oracle alone).  These
are the ring dimensions and kernels of the benchmark's ring-switched leg:
the ring-switching key switch and split at R = 4, the switched diagonals of
16 half-block classes, hoisted rotations and the multiply-accumulate at
N' = 2^13.  The library's answer on the same seeded inputs must have the
same digests and sampled residues and decompress to the matches."""
from __future__ import annotations

import dataclasses
import hashlib
import os

import numpy as np
import pytest
import torch

import workloads as W
from tests.gpu_common import coeff, library, to_dev
from tests.test_gpu_golden_ring15 import load_fixture

FIXTURE = os.path.join(os.path.dirname(__file__), "golden",
                       "answer_ring_switched_15to13_L2K2_n131072_s256.txt")


def test_fixture_is_complete():
    fx = load_fixture(FIXTURE)
    cfg, plan = fx["config"], fx["plan"]
    assert (cfg["log_n"], cfg["log_small"], cfg["L"], cfg["K"], cfg["dnum"]) == (15, 13, 2, 2, 1)
    assert len(fx["digest"]) == plan["n_out"] * 2 * cfg["L"]
    assert len(fx["sample"]) >= 1000


@pytest.mark.gpu
def test_ring_switched_answer_bit_exact_at_full_rings():
    pdq = library()
    fx = load_fixture(FIXTURE)
    c, fplan = fx["config"], fx["plan"]
    cfg = dataclasses.replace(W.CONFIGS["c3"], n=c["n"], L=c["L"], dnum=c["dnum"])
    assert cfg.seed == c["seed"] and cfg.K == c["K"] and cfg.s == c["s"]
    big = pdq.Context.from_config(cfg)
    small = big.subring(c["log_small"])
    q = W.draw_query(cfg)
    bplan = big.plan(cfg.n, cfg.s)
    plan = small.plan_switched(cfg.log_n, cfg.n, cfg.s)
    for k in ("s_prime", "B", "giants", "J", "H", "G", "n_out"):
        assert getattr(plan, k) == fplan[k], k
    sk = big.secret_prepare(torch.from_numpy(q.sk))
    a, e = W.encryption_randomness(big.moduli[:big.L], big.N, bplan.J, cfg.seed)
    slots = np.zeros(bplan.J * big.N, dtype=np.int32)
    slots[:cfg.n] = q.v
    v_cts = big.encrypt(sk, torch.from_numpy(slots), to_dev(a), torch.from_numpy(e))
    s_small = W.draw_ternary(small.N, W.rng_for(c["seed_small"], 11))
    ka, ke = W.rotation_key_randomness(big.moduli, big.N, big.ndigits, [1], c["seed_small"],
                                       stream=12)[1]
    rsk = big.ring_switch_key_gen(small, sk, torch.from_numpy(s_small), to_dev(ka),
                                  torch.from_numpy(ke))
    galois = small.plan_galois(plan)
    assert len(galois) == fplan["galois"]
    ssk = small.secret_prepare(torch.from_numpy(s_small))
    rand = W.rotation_key_randomness(small.moduli, small.N, small.ndigits, galois,
                                     c["seed_small"], stream=13)
    keys = small._u64(len(galois) * small.key_elems)
    kv = keys.view(len(galois), -1)
    for i, k in enumerate(galois):
        ra, re_ = rand[k]
        small.rotkey_gen(ssk, k, to_dev(ra), torch.from_numpy(re_).cuda(), out=kv[i])
    db = big.db_encode(torch.from_numpy(q.db.astype(np.int32)))
    consts = small.plan_constants(plan)
    masked = big.mask(bplan, v_cts, db)
    ms = big.ring_switch(small, masked, rsk, group=4)
    out = small.comp(plan, ms, keys, galois, consts)
    got = coeff(small, out, small.L)
    bad_rows = [key for key, h in sorted(fx["digest"].items())
                if hashlib.sha256(np.ascontiguousarray(got[key], dtype="<u8").tobytes())
                .hexdigest() != h]
    bad = [(cc, p, l, x, v, int(got[cc][p][l][x])) for cc, p, l, x, v in fx["sample"]
           if int(got[cc][p][l][x]) != v]
    assert not bad_rows and not bad, (f"{len(bad_rows)} rows differ (first {bad_rows[:4]}); "
                                      f"{len(bad)} sampled residues differ (first {bad[:4]})")
    dec = small.decrypt(ssk, out).cpu().numpy()
    assert small.decomp(plan, dec) == [(int(i), int(q.db[i])) for i in q.positions]
