"""Pins for the oracle's ring switching (Sec. 5.3) and Comp in the subring
(no GPU).

Ring switching is pinned against the definitions it rests on: the switching
key against its equation with Python integers; the split against the big
ring's own decryption (part r decrypts to the plaintext coefficients of index
r mod R); the slot fold against the plaintext decomposition
m(X) = sum_r X^r m_r(X^R) evaluated at the roots; the switched diagonals in
the clear against the power sums of Eq. 1 over the original records; and the
whole switched Answer against the closed form and Decomp."""
import numpy as np
import pytest

import workloads as W
from oracle import bfv, pdq
from tests.test_oracle_ring import py_negacyclic


def _setup(cfg_name, log_small, seed=0x5B):
    cfg = W.CONFIGS[cfg_name]
    big = bfv.Params.from_config(cfg)
    small = bfv.Params.subring(big, log_small)
    q = W.draw_query(cfg)
    sk_small = W.draw_ternary(small.N, W.rng_for(seed, 11))
    ka, ke = W.rotation_key_randomness(big.ext, big.N, len(big.digits), [1], seed, stream=12)[1]
    rsk = bfv.ring_switch_key(big, q.sk, sk_small, ka, ke)
    return cfg, big, small, q, sk_small, rsk, (ka, ke)


def test_subring_shares_primes_and_slot_root():
    big = bfv.Params.from_config(W.CONFIGS["tiny2"])
    small = bfv.Params.subring(big, 4)
    assert (small.q, small.p, small.t, small.N) == (big.q, big.p, big.t, 16)
    assert small.zeta == pow(big.zeta, 4, big.t)          # zeta' = zeta^R
    assert all((r - 1) % (2 * small.N) == 0 for r in small.ext)
    with pytest.raises(ValueError):
        bfv.Params.subring(big, big.log_n)


def test_ring_switch_key_equation():
    """b + a s' = e + [q_i in digit] P s limb by limb, s'(X) = s_small(X^R)."""
    cfg, big, small, q, sk_small, rsk, (ka, ke) = _setup("tiny", 3)
    R = big.N // small.N
    s_to = [0] * big.N
    for i, v in enumerate(sk_small):
        s_to[R * i] = int(v)
    for b_idx, digit in enumerate(big.digits):
        for l, r in enumerate(big.ext):
            lhs = [(int(x) + y) % r for x, y in
                   zip(rsk[b_idx][0][l],
                       py_negacyclic([int(v) for v in rsk[b_idx][1][l]], [v % r for v in s_to], r))]
            extra = big.P % r if (l < big.L and l in digit) else 0
            rhs = [(int(ev) + extra * int(sv)) % r for ev, sv in zip(ke[b_idx], q.sk)]
            assert lhs == rhs


@pytest.mark.parametrize("cfg_name,log_small", [("tiny2", 5), ("tiny2", 4), ("grouped", 3)])
def test_parts_decrypt_to_coefficients_of_their_residue(cfg_name, log_small):
    """Part r of a switched ciphertext decrypts in the subring to the big
    plaintext's coefficients r, r + R, r + 2R, ... (and keeps noise budget)."""
    cfg, big, small, q, sk_small, rsk, _ = _setup(cfg_name, log_small)
    R = big.N // small.N
    plan = pdq.make_plan(big, cfg.n, cfg.s)
    a, e = W.encryption_randomness(big.q, big.N, plan.J, cfg.seed)
    ct = pdq.encrypt_index(big, q.sk, q.v, plan, a, e)[0]
    m = bfv.decrypt_coeffs(big, q.sk, ct)
    parts = bfv.ring_switch(big, small, ct, rsk)
    assert len(parts) == R
    for r, part in enumerate(parts):
        assert part.shape == (2, big.L, small.N)
        assert np.array_equal(bfv.decrypt_coeffs(small, sk_small, part), m[r::R])
        assert bfv.noise_budget_bits(small, sk_small, part) > 20


@pytest.mark.parametrize("log_small", [5, 4])
def test_slot_fold(log_small):
    """With m(X) = sum_r X^r m_r(X^R): m(zeta^e) = sum_r zeta^(e r) m_r(zeta'^e')
    for every big slot exponent e, e' = e mod 2N' (Python integers)."""
    big = bfv.Params.from_config(W.CONFIGS["tiny2"])
    small = bfv.Params.subring(big, log_small)
    R, t = big.N // small.N, big.t
    rng = np.random.default_rng(7)
    coeffs = rng.integers(0, t, size=big.N, dtype=np.uint64)
    big_slots = bfv.decode(big, coeffs)
    small_slots = [bfv.decode(small, coeffs[r::R]) for r in range(R)]
    e_big, e_small = big.slot_exponents(), small.slot_exponents()
    where = {int(e): i for i, e in enumerate(e_small)}
    for i, e in enumerate(e_big):
        ip = where[int(e) % (2 * small.N)]
        want = sum(pow(big.zeta, int(e) * r, t) * int(small_slots[r][ip]) for r in range(R)) % t
        assert int(big_slots[i]) == want


@pytest.mark.parametrize("cfg_name,log_small", [("tiny2", 4), ("grouped", 4)])
def test_switched_diagonals_in_the_clear(cfg_name, log_small):
    """Switched diagonals, baby/giant split and rotate-and-sum applied in the
    clear to the folded small-ring slots give the power sums of Eq. 1 over
    the original records of each group."""
    cfg = W.CONFIGS[cfg_name]
    big = bfv.Params.from_config(cfg)
    small = bfv.Params.subring(big, log_small)
    R, t, m = big.N // small.N, big.t, small.m
    plan = pdq.make_switched_plan(big, small, cfg.n, cfg.s)
    sp, B = plan.s_prime, plan.B
    rng = np.random.default_rng(3)
    Jb = plan.J // R
    recs = rng.integers(0, t, size=Jb * big.N, dtype=np.uint64)
    # fold each big ciphertext's slots into R small plaintexts (coefficient split)
    u = []
    for j in range(Jb):
        coeffs = bfv.encode(big, recs[j * big.N:(j + 1) * big.N])
        for r in range(R):
            ys = bfv.decode(small, coeffs[r::R])
            for rho in range(2):          # half-block 2(Rj + r) + rho: that row on both rows
                row = ys[rho * m:(rho + 1) * m]
                u.append(np.concatenate([row, row]))
    for gamma in range(plan.G):
        y = np.zeros(small.N, dtype=np.uint64)
        for g in range(plan.giants):
            acc = np.zeros(small.N, dtype=np.uint64)
            for h in pdq.group_halfblocks(plan, gamma):
                for a in range(B):
                    d = pdq.rot_slots(small, pdq.switched_diagonal_slots(big, small, plan, h,
                                                                         g * B + a), -g * B)
                    acc = (acc + d * pdq.rot_slots(small, u[h], a)) % t
            y = (y + pdq.rot_slots(small, acc, g * B)) % t
        for l, r in pdq.rotsum_levels(small, plan):
            y = sum(pdq.rot_slots(small, y, jj * l) for jj in range(r)) % t
        want = [0] * sp
        lo, hi = gamma * plan.G_sz, min((gamma + 1) * plan.G_sz, recs.size)
        for i in range(lo, hi):
            node = i % plan.G_sz + 1
            for k in range(sp):
                want[k] = (want[k] + pow(node, k + 1, t) * int(recs[i])) % t
        assert y[:sp].tolist() == want
        assert y[m:m + sp].tolist() == want


@pytest.mark.parametrize("cfg_name,log_small", [("tiny2", 5), ("tiny2", 4), ("grouped", 4)])
def test_answer_ring_switched_decrypts_and_decompresses(cfg_name, log_small):
    cfg, big, small, q, sk_small, rsk, _ = _setup(cfg_name, log_small)
    plan = pdq.make_switched_plan(big, small, cfg.n, cfg.s)
    bplan = pdq.make_plan(big, cfg.n, cfg.s)
    assert plan.J == bplan.J * (big.N // small.N) and plan.G == bplan.G
    a, e = W.encryption_randomness(big.q, big.N, bplan.J, cfg.seed)
    v = pdq.encrypt_index(big, q.sk, q.v, bplan, a, e)
    gal = pdq.galois_elements(small, plan)
    kr = W.rotation_key_randomness(small.ext, small.N, len(small.digits), gal, cfg.seed, stream=13)
    keys = {k: bfv.rotation_key(small, sk_small, k, *kr[k]) for k in gal}
    out = pdq.answer_ring_switched(big, small, v, q.db, rsk, keys, plan)
    assert len(out) == plan.n_out
    slots = [bfv.decrypt(small, sk_small, o) for o in out]
    for got, want in zip(slots, pdq.expected_slots(small, plan, q.v, q.db)):
        assert np.array_equal(got, want)
    assert pdq.decomp_slots(small, plan, slots) == [(int(i), int(q.db[i])) for i in q.positions]
    assert min(bfv.noise_budget_bits(small, sk_small, o) for o in out) > 10
