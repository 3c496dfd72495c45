"""Write the oracle's Answer on an unencrypted database at the full-size ring.

The fixture pins the GPU path of the Answer on a database held in the clear
(Sec. 5.2, remark on an unencrypted database: [C; C diag(DB)] v, no Mask) at
the kernel shapes the full-size workload runs: ring N = 2^15, 8 x 60-bit
ciphertext primes + 2 special primes, 4 key-switching digits, s' = 256 with
B = 64 baby steps and 4 giant steps per diagonal set (the benchmark leg's
split), on a database small enough for the oracle: n = 2^17 records (J = 4
index ciphertexts, two record groups), s = 256 clustered matches, seed 0xC3.
Oracle only (``oracle/`` and the seeded draws of ``workloads/``),
single-threaded, about half an hour.

The Answer is ``oracle.pdq.answer_plain_db``; its coefficient-form output is
stored as one SHA-256 digest per (ciphertext, polynomial, prime) row plus
sampled residues.

Usage:  python tests/golden/make_answer_plain_db_ring15.py
"""
from __future__ import annotations

import dataclasses
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as W                          # noqa: E402
from oracle import bfv, pdq as opdq            # noqa: E402

OUT = os.path.join(HERE, "answer_plain_db_ring15_L8K2d4_n131072_s256_B64.txt")
N_RECORDS = 1 << 17
B = 64
SAMPLES = 1024
SAMPLE_SEED = 0x5A19


def config():
    return dataclasses.replace(W.CONFIGS["c3"], n=N_RECORDS)


def row_digest(row: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(row, dtype="<u8").tobytes()).hexdigest()


def main() -> None:
    cfg = config()
    par = bfv.Params.from_config(cfg)
    plan = opdq.make_plan_plain_db(par, cfg.n, cfg.s, B)
    q = W.draw_query(cfg)
    enc_a, enc_e = W.encryption_randomness(par.q, par.N, plan.J, cfg.seed)
    v_cts = opdq.encrypt_index(par, q.sk, q.v, plan, enc_a, enc_e)
    galois = opdq.plain_db_galois_elements(par, plan)
    rand = W.rotation_key_randomness(par.ext, par.N, len(par.digits), galois, cfg.seed)
    t0 = time.time()
    keys = {k: bfv.rotation_key(par, q.sk, k, *rand[k]) for k in galois}
    t1 = time.time()
    outs = opdq.answer_plain_db(par, v_cts, q.db, keys, plan)
    t2 = time.time()
    # written only for an answer that meets the closed form and decompresses
    slots = [bfv.decrypt(par, q.sk, o) for o in outs]
    exp = opdq.expected_slots(par, plan, q.v, q.db)
    assert all(np.array_equal(a, b) for a, b in zip(slots, exp)), "answer misses the closed form"
    truth = [(int(i), int(q.db[i])) for i in q.positions]
    assert opdq.decomp_slots(par, plan, slots) == truth, "answer does not decompress"
    lines = [
        "# Oracle Answer on an unencrypted database ([C; C diag(DB)] v, Sec. 5.2 remark) at",
        "# ring N = 2^15 with 8 x 60-bit ciphertext primes, 2 special primes and 4",
        "# key-switching digits; written by tests/golden/make_answer_plain_db_ring15.py",
        "# (oracle only).",
        f"config log_n={cfg.log_n} t={cfg.t} prime_bits={cfg.prime_bits} L={cfg.L} K={cfg.K} "
        f"dnum={cfg.dnum} n={cfg.n} s={cfg.s} pattern={cfg.pattern} seed={cfg.seed:#x} B={B}",
        f"plan s_prime={plan.s_prime} B={plan.B} giants={plan.giants} J={plan.J} H={plan.H} "
        f"G={plan.G} n_out={plan.n_out} galois={len(galois)}",
        f"# oracle time: keys {t1 - t0:.0f} s, answer {t2 - t1:.0f} s",
    ]
    for c, o in enumerate(outs):
        for p in range(2):
            for l in range(par.L):
                lines.append(f"digest {c} {p} {l} {row_digest(o[p][l])}")
    rng = np.random.Generator(np.random.PCG64(SAMPLE_SEED))
    for _ in range(SAMPLES):
        c, p, l, x = (int(rng.integers(0, len(outs))), int(rng.integers(0, 2)),
                      int(rng.integers(0, par.L)), int(rng.integers(0, par.N)))
        lines.append(f"sample {c} {p} {l} {x} {int(outs[c][p][l][x])}")
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")
    print(f"wrote {OUT}: keys {t1 - t0:.0f} s, answer {t2 - t1:.0f} s")


if __name__ == "__main__":
    main()
