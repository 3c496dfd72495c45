"""Bit-exact Answer at the full-size ring and key-switching shape.

The oracle's Answer (Mask then Comp, Alg. 7 in the SIMD form of Sec. 5.2) at
N = 2^15, 8 + 2 primes, 4 digits, s' = 256 with B = 32 x 8 giant steps and two
record groups is stored in ``tests/golden/answer_ring15_L8K2d4_n131072_s256_B32.txt``
(written by ``tests/golden/make_answer_ring15.py`` from the oracle alone).
These are the kernel shapes of the full-size workload: 4-digit key
switching, hoisted baby rotations with 4 digits, the multiply-accumulate
with 16 baby steps per staged chunk and 4 giant steps per thread, and the
128-bit single fold of each accumulator.  The library's coefficient-form
answer on the same seeded inputs must have the same SHA-256 digest per
(ciphertext, polynomial, prime) row and the same residues at the sampled
positions."""
from __future__ import annotations

import hashlib
import os

import numpy as np
import pytest

from tests.gpu_common import Setup, coeff

FIXTURE = os.path.join(os.path.dirname(__file__), "golden",
                       "answer_ring15_L8K2d4_n131072_s256_B32.txt")


def load_fixture(path: str = FIXTURE) -> dict:
    fx = {"digest": {}, "sample": []}
    with open(path) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            kind, *rest = line.split()
            if kind in ("config", "plan"):
                fx[kind] = {k: int(v, 0) if v[0].isdigit() else v
                            for k, v in (x.split("=") for x in rest)}
            elif kind == "digest":
                c, p, l, h = rest
                fx["digest"][(int(c), int(p), int(l))] = h
            elif kind == "sample":
                fx["sample"].append(tuple(int(x) for x in rest))
    return fx


def test_fixture_is_complete():
    """The fixture names the shapes it pins and covers every row (CPU)."""
    fx = load_fixture()
    cfg, plan = fx["config"], fx["plan"]
    assert (cfg["log_n"], cfg["L"], cfg["K"], cfg["dnum"]) == (15, 8, 2, 4)
    assert (plan["B"], plan["giants"], plan["G"]) == (32, 8, 2)
    assert len(fx["digest"]) == plan["n_out"] * 2 * cfg["L"]
    assert len(fx["sample"]) >= 1000


@pytest.mark.gpu
def test_answer_bit_exact_at_full_ring_shape():
    fx = load_fixture()
    cfg, fplan = fx["config"], fx["plan"]
    st = Setup("c3", n=cfg["n"], s=cfg["s"], B=cfg["B"], pattern=cfg["pattern"])
    assert st.cfg.seed == cfg["seed"]
    for k in ("s_prime", "B", "giants", "J", "H", "G", "n_out"):
        assert getattr(st.plan, k) == fplan[k], k
    assert len(st.galois) == fplan["galois"]
    got = coeff(st.ctx, st.answer(), st.par.L)
    bad_rows = [key for key, h in sorted(fx["digest"].items())
                if hashlib.sha256(np.ascontiguousarray(got[key], dtype="<u8").tobytes())
                .hexdigest() != h]
    bad_samples = [(c, p, l, x, v, int(got[c][p][l][x])) for c, p, l, x, v in fx["sample"]
                   if int(got[c][p][l][x]) != v]
    assert not bad_rows and not bad_samples, (
        f"{len(bad_rows)} rows differ (first {bad_rows[:4]}); "
        f"{len(bad_samples)} sampled residues differ (first {bad_samples[:4]})")
    slots = st.ctx.decrypt(st.sk, st.answer()).cpu().numpy()
    truth = [(int(i), int(st.q.db[i])) for i in st.q.positions]
    assert st.ctx.decomp(st.plan, slots) == truth
