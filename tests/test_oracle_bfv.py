"""Pins for the oracle's scheme layer: slot encoding, encryption, key
switching and rotations (no GPU).  Big-integer and brute-force checks only."""
import math
import random

import numpy as np
import pytest

import workloads as W
from oracle import bfv, ring
from tests.test_oracle_ring import py_negacyclic


@pytest.fixture(scope="module")
def tiny():
    return bfv.Params.from_config(W.CONFIGS["tiny"])


@pytest.fixture(scope="module")
def tiny2():
    return bfv.Params.from_config(W.CONFIGS["tiny2"])


def test_slot_exponents_cover_odd_residues(tiny):
    e = tiny.slot_exponents()
    assert sorted(e.tolist()) == list(range(1, 2 * tiny.N, 2))


def test_encode_is_interpolation(tiny):
    rnd = random.Random(1)
    slots = [rnd.randrange(tiny.t) for _ in range(tiny.N)]
    m = bfv.encode(tiny, slots).tolist()
    e = tiny.slot_exponents()
    for idx in range(tiny.N):
        x = pow(tiny.zeta, int(e[idx]), tiny.t)
        assert sum(c * pow(x, j, tiny.t) for j, c in enumerate(m)) % tiny.t == slots[idx]
    assert bfv.decode(tiny, m).tolist() == slots
    assert pow(tiny.zeta, tiny.N, tiny.t) == tiny.t - 1


def test_encode_is_multiplicative(tiny):
    """encode(x) * encode(y) mod (X^N+1, t) = encode(x . y)."""
    rnd = random.Random(2)
    x = [rnd.randrange(tiny.t) for _ in range(tiny.N)]
    y = [rnd.randrange(tiny.t) for _ in range(tiny.N)]
    mx = bfv.encode(tiny, x).tolist()
    my = bfv.encode(tiny, y).tolist()
    prod = py_negacyclic(mx, my, tiny.t)
    xy = [(a * b) % tiny.t for a, b in zip(x, y)]
    assert prod == bfv.encode(tiny, xy).tolist()


def test_automorphisms_rotate_slots(tiny):
    """sigma_{3^r} = Rot_row(.; r) (left rotation of both rows), sigma_{2N-1}
    swaps the rows (Sec. 5.1)."""
    rnd = random.Random(3)
    slots = np.array([rnd.randrange(tiny.t) for _ in range(tiny.N)], dtype=np.uint64)
    m = bfv.encode(tiny, slots)
    rows = slots.reshape(2, tiny.m)
    for r in (1, 2, 5, tiny.m - 1, -3):
        got = bfv.decode(tiny, ring.automorphism(m, tiny.galois_rot(r), tiny.t))
        assert np.array_equal(got.reshape(2, tiny.m), np.roll(rows, -r, axis=1))
    got = bfv.decode(tiny, ring.automorphism(m, tiny.galois_col, tiny.t))
    assert np.array_equal(got.reshape(2, tiny.m), rows[::-1])


def test_lift_is_centred(tiny):
    c = np.arange(tiny.t, dtype=np.uint64)[: tiny.N * 0 + tiny.t]
    par = tiny
    for chunk in range(0, par.t, par.N):
        cc = np.zeros(par.N, dtype=np.uint64)
        part = c[chunk:chunk + par.N]
        cc[:part.size] = part
        out = bfv.lift(par, cc, par.q)
        for i, q in enumerate(par.q):
            v = [int(x) if int(x) < q // 2 else int(x) - q for x in out[i]]
            assert all(-(par.t // 2) <= x <= par.t // 2 for x in v)
            assert all((x - int(y)) % par.t == 0 for x, y in zip(v, cc))


def _key_material(par, seed=11):
    sk = W.draw_ternary(par.N, W.rng_for(seed, 3))
    return sk


def test_encrypt_decrypt_roundtrip(tiny2):
    par = tiny2
    sk = _key_material(par)
    a, e = W.encryption_randomness(par.q, par.N, 3, seed=5)
    for j in range(3):
        slots = W.rng_for(9, j).integers(0, par.t, size=par.N, dtype=np.uint64)
        ct = bfv.encrypt(par, sk, bfv.encode(par, slots), a[j], e[j])
        assert np.array_equal(bfv.decrypt(par, sk, ct), slots)
        assert bfv.noise_budget_bits(par, sk, ct) > 100


def test_decrypt_against_bigint_definition(tiny):
    """x = c0 + c1*s computed over Z_Q with Python integers (CRT first, then
    the ring product by definition), m = round(t x / Q) mod t."""
    par = tiny
    sk = _key_material(par, 4)
    a, e = W.encryption_randomness(par.q, par.N, 1, seed=6)
    slots = W.rng_for(10).integers(0, par.t, size=par.N, dtype=np.uint64)
    ct = bfv.encrypt(par, sk, bfv.encode(par, slots), a[0], e[0])
    Q = math.prod(par.q)

    def crt(limbs):
        out = []
        for c in range(par.N):
            x = 0
            for i, q in enumerate(par.q):
                hat = Q // q
                x += int(limbs[i][c]) * hat * pow(hat, -1, q)
            out.append(x % Q)
        return out
    c0, c1 = crt(ct[0]), crt(ct[1])
    s = [int(v) % Q for v in sk]
    x = [(u + w) % Q for u, w in zip(c0, py_negacyclic(c1, s, Q))]
    m = [((par.t * xv + Q // 2) // Q) % par.t for xv in x]
    assert bfv.decode(par, m).tolist() == slots.tolist()
    assert m == bfv.decrypt_coeffs(par, sk, ct).tolist()


def test_encryption_scale_is_floor_Q_over_t(tiny, tiny2):
    """BFV scales the message by Delta = floor(Q/t): a noise-free encryption
    (e = 0) of the constant plaintext m(X) = 1 has c0 + c1*s = Delta exactly
    over Z_Q (Python integers, ring product by definition), and that Delta is
    the largest integer with Delta*t <= Q."""
    for par in (tiny, tiny2):
        sk = _key_material(par, 7)
        a, _ = W.encryption_randomness(par.q, par.N, 1, seed=8)
        one = np.zeros(par.N, dtype=np.uint64)
        one[0] = 1
        ct = bfv.encrypt(par, sk, one, a[0], np.zeros(par.N, dtype=np.int64))
        Q = math.prod(par.q)
        crt = [[sum(int(ct[p][i][c]) * (Q // q) * pow(Q // q, -1, q)
                    for i, q in enumerate(par.q)) % Q for c in range(par.N)] for p in range(2)]
        s = [int(v) % Q for v in sk]
        x = [(u + w) % Q for u, w in zip(crt[0], py_negacyclic(crt[1], s, Q))]
        assert x[1:] == [0] * (par.N - 1)
        assert x[0] * par.t <= Q < (x[0] + 1) * par.t


def test_mod_up_against_crt(tiny2):
    par = tiny2
    rng = np.random.default_rng(3)
    X = [int(v) for v in rng.integers(0, 2**62, size=par.N)]
    for digit in par.digits:
        Qb = math.prod(par.q[i] for i in digit)
        Xd = [v % Qb for v in X]
        x = np.zeros((par.L, par.N), dtype=np.uint64)
        for i in digit:
            x[i] = [v % par.q[i] for v in Xd]
        y = bfv.mod_up(par, x, digit)
        for l, r in enumerate(par.ext):
            for c in range(par.N):
                ok = [(Xd[c] + u * Qb) % r for u in range(len(digit))]
                assert int(y[l][c]) in ok


def test_mod_down_is_floor_division_by_P(tiny2):
    par = tiny2
    rng = np.random.default_rng(4)
    QP = par.Q * par.P
    Y = [int.from_bytes(rng.bytes(32), "little") % QP for _ in range(par.N)]
    y = np.array([[v % r for v in Y] for r in par.ext], dtype=np.uint64)
    out = bfv.mod_down(par, y)
    for c in range(par.N):
        # conv = sum_k [y_k (P/p_k)^{-1}]_{p_k} (P/p_k), an integer = Y mod P (+ u P)
        conv = 0
        for pk in par.p:
            hat = par.P // pk
            conv += (Y[c] % pk) * pow(hat, -1, pk) % pk * hat
        assert (Y[c] - conv) % par.P == 0
        z = (Y[c] - conv) // par.P
        assert [int(out[i][c]) for i in range(par.L)] == [z % q for q in par.q]
        assert 0 <= conv < par.K * par.P


def test_rotation_key_equation(tiny):
    """b + a*s = e + [q_i in digit] P sigma_k(s) limb by limb (definition)."""
    par = tiny
    sk = _key_material(par, 5)
    k = par.galois_rot(1)
    kr = W.rotation_key_randomness(par.ext, par.N, len(par.digits), [k], seed=1)
    key = bfv.rotation_key(par, sk, k, *kr[k])
    from tests.test_oracle_ring import py_substitute
    for b_idx, digit in enumerate(par.digits):
        e = kr[k][1][b_idx]
        for l, r in enumerate(par.ext):
            s = [int(v) % r for v in sk]
            lhs = [(int(x) + y) % r for x, y in
                   zip(key[b_idx][0][l], py_negacyclic([int(v) for v in key[b_idx][1][l]], s, r))]
            sig = py_substitute(s, k, r)
            extra = par.P % r if (l < par.L and l in digit) else 0
            rhs = [(int(ev) + extra * sv) % r for ev, sv in zip(e, sig)]
            assert lhs == rhs


@pytest.mark.parametrize("cfg", ["tiny", "tiny2"])
def test_rotations_decrypt_to_rotated_slots(cfg):
    par = bfv.Params.from_config(W.CONFIGS[cfg])
    sk = _key_material(par, 8)
    a, e = W.encryption_randomness(par.q, par.N, 1, seed=8)
    slots = W.rng_for(12).integers(0, par.t, size=par.N, dtype=np.uint64)
    ct = bfv.encrypt(par, sk, bfv.encode(par, slots), a[0], e[0])
    rows = slots.reshape(2, par.m)
    ks = [par.galois_rot(r) for r in (1, 3)] + [par.galois_col]
    kr = W.rotation_key_randomness(par.ext, par.N, len(par.digits), ks, seed=2)
    keys = {k: bfv.rotation_key(par, sk, k, *kr[k]) for k in ks}
    for r in (1, 3):
        out = bfv.rotate(par, ct, par.galois_rot(r), keys[par.galois_rot(r)])
        assert np.array_equal(bfv.decrypt(par, sk, out).reshape(2, par.m),
                              np.roll(rows, -r, axis=1))
    col = bfv.rotate(par, ct, par.galois_col, keys[par.galois_col])
    assert np.array_equal(bfv.decrypt(par, sk, col).reshape(2, par.m), rows[::-1])
    back = bfv.rotate(par, col, par.galois_col, keys[par.galois_col])
    assert np.array_equal(bfv.decrypt(par, sk, back), slots)
    # the hoisted form with shared raised digits gives the same bits
    raised = bfv.mod_up_all(par, ct[1])
    k = par.galois_rot(3)
    assert np.array_equal(bfv.rotate_hoisted(par, ct, raised, k, keys[k]),
                          bfv.rotate(par, ct, k, keys[k]))


def test_plaintext_product_decrypts(tiny2):
    par = tiny2
    sk = _key_material(par, 9)
    a, e = W.encryption_randomness(par.q, par.N, 1, seed=9)
    x = W.rng_for(13).integers(0, par.t, size=par.N, dtype=np.uint64)
    y = W.rng_for(14).integers(0, par.t, size=par.N, dtype=np.uint64)
    ct = bfv.encrypt(par, sk, bfv.encode(par, x), a[0], e[0])
    out = bfv.pt_mul(par, ct, bfv.lift(par, bfv.encode(par, y), par.q))
    assert np.array_equal(bfv.decrypt(par, sk, out), x * y % par.t)


@pytest.mark.parametrize("cfg", ["tiny", "tiny2"])
def test_extended_rotation_lowers_to_the_rotation(cfg):
    """Keeping a rotation in Q u P and lowering it later gives the same bits:
    ModDown(P sigma(c0) + A0) = sigma(c0) + ModDown(A0) because P sigma(c0)
    vanishes modulo the special primes; and ModDown(P x) = x."""
    par = bfv.Params.from_config(W.CONFIGS[cfg])
    sk = _key_material(par, 21)
    a, e = W.encryption_randomness(par.q, par.N, 1, seed=21)
    slots = W.rng_for(22).integers(0, par.t, size=par.N, dtype=np.uint64)
    ct = bfv.encrypt(par, sk, bfv.encode(par, slots), a[0], e[0])
    k = par.galois_rot(2)
    kr = W.rotation_key_randomness(par.ext, par.N, len(par.digits), [k], seed=23)
    key = bfv.rotation_key(par, sk, k, *kr[k])
    ext = bfv.rotate_ext(par, ct, bfv.mod_up_all(par, ct[1]), k, key)
    assert np.array_equal(bfv.ct_mod_down(par, ext), bfv.rotate(par, ct, k, key))
    assert np.array_equal(bfv.ct_mod_down(par, bfv.ct_times_P(par, ct)), ct)


@pytest.mark.parametrize("cfg", ["tiny", "tiny2"])
def test_lazy_extended_rotation(cfg):
    """rotate_ext_lazy (c0 from Q u P, c1 lowered for the key switch) equals
    rotate_ext when c0 = P x, and on a genuine extended ciphertext (special
    limbs of c0 nonzero) lowers to a ciphertext of the rotated slots."""
    par = bfv.Params.from_config(W.CONFIGS[cfg])
    sk = _key_material(par, 25)
    a, e = W.encryption_randomness(par.q, par.N, 1, seed=25)
    slots = W.rng_for(26).integers(0, par.t, size=par.N, dtype=np.uint64)
    ct = bfv.encrypt(par, sk, bfv.encode(par, slots), a[0], e[0])
    ks = [par.galois_rot(1), par.galois_rot(3), par.galois_col]
    kr = W.rotation_key_randomness(par.ext, par.N, len(par.digits), ks, seed=27)
    keys = {k: bfv.rotation_key(par, sk, k, *kr[k]) for k in ks}
    raised = bfv.mod_up_all(par, ct[1])
    k1 = par.galois_rot(1)
    x = bfv.rotate_ext_lazy(par, bfv.ct_times_P(par, ct), raised, k1, keys[k1])
    assert np.array_equal(x, bfv.rotate_ext(par, ct, raised, k1, keys[k1]))
    assert np.any(x[0][par.L:] != 0)
    rows = slots.reshape(2, par.m)
    for k2, want in ((par.galois_rot(3), np.roll(rows, -4, axis=1)),
                     (par.galois_col, np.roll(rows, -1, axis=1)[::-1])):
        r2 = bfv.mod_up_all(par, bfv.mod_down(par, x[1]))
        y = bfv.ct_mod_down(par, bfv.rotate_ext_lazy(par, x, r2, k2, keys[k2]))
        assert np.array_equal(bfv.decrypt(par, sk, y).reshape(2, par.m), want)


@pytest.mark.parametrize("cfg,L2", [("tiny2", 1), ("tiny2", 2), ("small", 1)])
def test_mod_switch(cfg, L2):
    """Modulus switching keeps the slots, and every coefficient is
    floor(X / D) - u mod Q' for the coefficient X over Q, D the product of
    the dropped primes and 0 <= u < (number of dropped primes) (the
    base conversion without overflow correction), checked with Python
    integers."""
    import dataclasses
    c = W.CONFIGS[cfg]
    par = bfv.Params.from_config(c)
    low = bfv.Params.from_config(dataclasses.replace(c, L=L2, dnum=1))
    assert low.q == par.q[:L2]
    sk = _key_material(par, 41)
    a, e = W.encryption_randomness(par.q, par.N, 1, seed=41)
    slots = W.rng_for(42).integers(0, par.t, size=par.N, dtype=np.uint64)
    ct = bfv.encrypt(par, sk, bfv.encode(par, slots), a[0], e[0])
    sw = bfv.mod_switch(par, low, ct)
    assert np.array_equal(bfv.decrypt(low, sk, sw), slots)
    D = math.prod(par.q[L2:])
    Qp = math.prod(low.q)
    nd = par.L - L2
    for p in range(2):
        X = bfv.crt_compose(par, ct[p])
        Y = bfv.crt_compose(low, sw[p])
        for x, y in zip(X, Y):
            assert any((x // D - u - y) % Qp == 0 for u in range(nd))


def test_mod_switch_needs_a_prefix_of_the_primes(tiny, tiny2):
    """The smaller parameters must share the ring, the plaintext modulus and
    a proper prefix of the ciphertext primes; anything else is refused."""
    import dataclasses
    c = W.CONFIGS["tiny2"]
    low = bfv.Params.from_config(dataclasses.replace(c, L=1, dnum=1))
    ct = np.zeros((2, tiny2.L, tiny2.N), dtype=np.uint64)
    assert bfv.mod_switch(tiny2, low, ct).shape == (2, 1, tiny2.N)
    with pytest.raises(ValueError):
        bfv.mod_switch(low, tiny2, ct[:, :1])             # more primes
    with pytest.raises(ValueError):
        bfv.mod_switch(tiny2, tiny2, ct)                  # nothing dropped
    with pytest.raises(ValueError):
        bfv.mod_switch(tiny2, tiny, ct)                   # another ring
    other = bfv.Params(tiny2.log_n, tiny2.t, tiny2.bits - 1, 1, 1, 1)
    with pytest.raises(ValueError):
        bfv.mod_switch(tiny2, other, ct)                  # other primes
