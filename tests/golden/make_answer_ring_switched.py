"""Write the oracle's ring-switched Answer at the full-size rings.

The fixture pins the GPU path of Comp in a subring (Sec. 5.3) at the ring
dimensions the benchmark's ring-switched leg uses: the query's ring N = 2^15
and the subring N' = 2^13 (R = 4), over 2 x 60-bit ciphertext primes and the
2 special primes of the full-size chain (one key-switching digit), t = 65537,
n = 2^17 records (4 big index ciphertexts -> 16 subring quadruples, two
record groups), s = 256 clustered matches, seed 0xC3.  Oracle only (``oracle/``
and the seeded draws of ``workloads/``), single-threaded, a few minutes.

The Answer is Mask in the big ring, ring switching of the masked
ciphertexts, and Comp in the subring (``oracle.pdq.answer_ring_switched``);
its coefficient-form output is stored as one SHA-256 digest per
(ciphertext, polynomial, prime) row plus sampled residues.

Usage:  python tests/golden/make_answer_ring_switched.py
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

OUT = os.path.join(HERE, "answer_ring_switched_15to13_L2K2_n131072_s256.txt")
N_RECORDS = 1 << 17
LOG_SMALL = 13
SEED_SMALL = 0x5B          # draws of the subring secret and keys
SAMPLES = 1024
SAMPLE_SEED = 0x5A18


def config():
    return dataclasses.replace(W.CONFIGS["c3"], n=N_RECORDS, L=2, dnum=1)


def row_digest(row: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(row, dtype="<u8").tobytes()).hexdigest()


def main() -> None:
    cfg = config()
    big = bfv.Params.from_config(cfg)
    small = bfv.Params.subring(big, LOG_SMALL)
    q = W.draw_query(cfg)
    bplan = opdq.make_plan(big, cfg.n, cfg.s)
    plan = opdq.make_switched_plan(big, small, cfg.n, cfg.s)
    enc_a, enc_e = W.encryption_randomness(big.q, big.N, bplan.J, cfg.seed)
    v_cts = opdq.encrypt_index(big, q.sk, q.v, bplan, enc_a, enc_e)
    sk_small = W.draw_ternary(small.N, W.rng_for(SEED_SMALL, 11))
    ka, ke = W.rotation_key_randomness(big.ext, big.N, len(big.digits), [1], SEED_SMALL,
                                       stream=12)[1]
    t0 = time.time()
    rsk = bfv.ring_switch_key(big, q.sk, sk_small, ka, ke)
    galois = opdq.galois_elements(small, plan)
    rand = W.rotation_key_randomness(small.ext, small.N, len(small.digits), galois, SEED_SMALL,
                                     stream=13)
    keys = {k: bfv.rotation_key(small, sk_small, k, *rand[k]) for k in galois}
    t1 = time.time()
    outs = opdq.answer_ring_switched(big, small, v_cts, q.db, rsk, keys, plan)
    t2 = time.time()
    slots = [bfv.decrypt(small, sk_small, o) for o in outs]
    exp = opdq.expected_slots(small, plan, q.v, q.db)
    assert all(np.array_equal(a, b) for a, b in zip(slots, exp)), "answer misses the closed form"
    truth = [(int(i), int(q.db[i])) for i in q.positions]
    assert opdq.decomp_slots(small, plan, slots) == truth, "answer does not decompress"
    lines = [
        "# Oracle ring-switched Answer (Mask in the ring 2^15, ring switching to the subring",
        "# 2^13, Comp there: Sec. 5.2 and 5.3) over 2 x 60-bit primes + 2 special primes;",
        "# written by tests/golden/make_answer_ring_switched.py (oracle only).",
        f"config log_n={cfg.log_n} log_small={LOG_SMALL} t={cfg.t} prime_bits={cfg.prime_bits} "
        f"L={cfg.L} K={cfg.K} dnum={cfg.dnum} n={cfg.n} s={cfg.s} pattern={cfg.pattern} "
        f"seed={cfg.seed:#x} seed_small={SEED_SMALL:#x}",
        f"plan s_prime={plan.s_prime} B={plan.B} giants={plan.giants} J={plan.J} H={plan.H} "
        f"G={plan.G} n_out={plan.n_out} galois={len(galois)}",
        f"# oracle time: keys {t1 - t0:.0f} s, answer {t2 - t1:.0f} s",
    ]
    for c, o in enumerate(outs):
        for p in range(2):
            for l in range(small.L):
                lines.append(f"digest {c} {p} {l} {row_digest(o[p][l])}")
    rng = np.random.Generator(np.random.PCG64(SAMPLE_SEED))
    for _ in range(SAMPLES):
        c, p, l, x = (int(rng.integers(0, len(outs))), int(rng.integers(0, 2)),
                      int(rng.integers(0, small.L)), int(rng.integers(0, small.N)))
        lines.append(f"sample {c} {p} {l} {x} {int(outs[c][p][l][x])}")
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")
    print(f"wrote {OUT}: keys {t1 - t0:.0f} s, answer {t2 - t1:.0f} s")


if __name__ == "__main__":
    main()
