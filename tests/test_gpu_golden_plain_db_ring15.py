"""Bit-exact Answer on an unencrypted database at the full-size ring.

The oracle's Answer [C; C diag(DB)] v (Sec. 5.2, remark on an unencrypted
database) at N = 2^15, 8 + 2 primes, 4 digits, s' = 256 with B = 64 x 4 giant
steps per diagonal set and two record groups is stored in
``tests/golden/answer_plain_db_ring15_L8K2d4_n131072_s256_B64.txt`` (written by
``tests/golden/make_answer_plain_db_ring15.py`` from the oracle alone).  These
are the kernel shapes of the benchmark's unencrypted-database leg: hoisted
baby rotations of the index ciphertexts with 4 digits, the database-specific
multiply-accumulate with 4 giant steps per thread over both sets, the giant
steps of both sets in one launch (Rot_col folded into set 1's), and the
raise's and ModDown's conversions in the transforms.  The library's answer on
the same seeded inputs must have the same digests and sampled residues and
decompress to the matches."""
from __future__ import annotations

import hashlib
import os

import numpy as np
import pytest
import torch

import workloads as W
from tests.gpu_common import Setup, coeff, to_dev
from tests.test_gpu_golden_ring15 import load_fixture

FIXTURE = os.path.join(os.path.dirname(__file__), "golden",
                       "answer_plain_db_ring15_L8K2d4_n131072_s256_B64.txt")


def test_fixture_is_complete():
    fx = load_fixture(FIXTURE)
    cfg, plan = fx["config"], fx["plan"]
    assert (cfg["log_n"], cfg["L"], cfg["K"], cfg["dnum"]) == (15, 8, 2, 4)
    assert (plan["B"], plan["giants"], plan["G"]) == (64, 4, 2)
    assert len(fx["digest"]) == plan["n_out"] * 2 * cfg["L"]
    assert len(fx["sample"]) >= 1000


@pytest.mark.gpu
def test_plain_db_answer_bit_exact_at_full_ring_shape():
    fx = load_fixture(FIXTURE)
    cfg, fplan = fx["config"], fx["plan"]
    st = Setup("c3", n=cfg["n"], s=cfg["s"], pattern=cfg["pattern"])
    assert st.cfg.seed == cfg["seed"]
    ctx = st.ctx
    plan = ctx.plan_plain_db(cfg["n"], cfg["s"], cfg["B"])
    for k in ("s_prime", "B", "giants", "J", "H", "G", "n_out"):
        assert getattr(plan, k) == fplan[k], k
    galois = ctx.plan_galois(plan)
    assert len(galois) == fplan["galois"]
    rand = W.rotation_key_randomness(st.par.ext, st.par.N, len(st.par.digits), galois, st.seed)
    keys = ctx._u64(len(galois) * ctx.key_elems)
    kv = keys.view(len(galois), -1)
    for i, k in enumerate(galois):
        a, e = rand[k]
        ctx.rotkey_gen(st.sk, k, to_dev(a), torch.from_numpy(e).cuda(), out=kv[i])
    consts = ctx.db_diagonals(plan, torch.from_numpy(st.q.db.astype(np.int32)))
    out = ctx.answer_plain_db(plan, st.v_cts, keys, galois, consts)
    got = coeff(ctx, out.contiguous(), st.par.L)
    bad_rows = [key for key, h in sorted(fx["digest"].items())
                if hashlib.sha256(np.ascontiguousarray(got[key], dtype="<u8").tobytes())
                .hexdigest() != h]
    bad = [(c, p, l, x, v, int(got[c][p][l][x])) for c, p, l, x, v in fx["sample"]
           if int(got[c][p][l][x]) != v]
    assert not bad_rows and not bad, (f"{len(bad_rows)} rows differ (first {bad_rows[:4]}); "
                                      f"{len(bad)} sampled residues differ (first {bad[:4]})")
    slots = ctx.decrypt(st.sk, out).cpu().numpy()
    truth = [(int(i), int(st.q.db[i])) for i in st.q.positions]
    assert ctx.decomp(plan, slots) == truth
