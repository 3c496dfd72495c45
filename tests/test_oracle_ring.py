"""Pins for the oracle's ring arithmetic (no GPU).

Each check compares the oracle with something other than itself: the
definition written with Python big integers, brute force on small rings,
algebraic laws, or an independent library (sympy's primality test)."""
import random

import numpy as np
import pytest

from oracle import bfv, ring


def py_negacyclic(a, b, q):
    """Ring product in Z_q[X]/(X^N+1) from the definition, Python integers."""
    N = len(a)
    c = [0] * N
    for i in range(N):
        for j in range(N):
            k = i + j
            if k < N:
                c[k] += a[i] * b[j]
            else:
                c[k - N] -= a[i] * b[j]
    return [x % q for x in c]


def py_eval(a, x, q):
    """a(x) mod q by Horner."""
    r = 0
    for c in reversed(a):
        r = (r * x + c) % q
    return r


def py_substitute(a, k, q):
    """a(X^k) reduced modulo X^N + 1 by repeated X^N -> -1."""
    N = len(a)
    out = [0] * N
    for j, c in enumerate(a):
        e = j * k
        sign = -1 if (e // N) % 2 else 1
        out[e % N] += sign * c
    return [x % q for x in out]


PRIMES = [bfv.ntt_primes(64, 54, 2)[1], bfv.ntt_primes(64, 60, 1)[0], 12289, 65537]


@pytest.mark.parametrize("q", PRIMES)
@pytest.mark.parametrize("N", [4, 16, 64])
def test_ntt_is_evaluation_at_odd_powers(q, N):
    if (q - 1) % (2 * N):
        pytest.skip("q != 1 mod 2N")
    rnd = random.Random(q + N)
    psi = bfv.primitive_2n_root(q, N)
    assert pow(psi, N, q) == q - 1
    a = [rnd.randrange(q) for _ in range(N)]
    got = ring.ntt_forward(np.array(a, dtype=np.uint64), q, psi).tolist()
    want = [py_eval(a, pow(psi, 2 * j + 1, q), q) for j in range(N)]
    assert got == want


@pytest.mark.parametrize("logN", [1, 5, 10, 12])
def test_ntt_inverse_roundtrip(logN):
    N = 1 << logN
    q = bfv.ntt_primes(N, 60, 1)[0]
    psi = bfv.primitive_2n_root(q, N)
    rng = np.random.default_rng(logN)
    a = rng.integers(0, q, size=N, dtype=np.uint64)
    b = ring.ntt_inverse(ring.ntt_forward(a, q, psi), q, psi)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("N", [2, 8, 32, 64])
def test_product_matches_definition(N):
    q = bfv.ntt_primes(N, 60, 1)[0]
    psi = bfv.primitive_2n_root(q, N)
    rnd = random.Random(N)
    a = [rnd.randrange(q) for _ in range(N)]
    b = [rnd.randrange(q) for _ in range(N)]
    b[0] = q - 1
    want = py_negacyclic(a, b, q)
    assert ring.negacyclic_mul(np.array(a, dtype=np.uint64), np.array(b, dtype=np.uint64),
                               q, psi).tolist() == want
    assert ring.schoolbook(np.array(a, dtype=np.uint64), np.array(b, dtype=np.uint64),
                           q).tolist() == want


def test_transform_product_equals_schoolbook_n256():
    N = 256
    q = bfv.ntt_primes(N, 54, 3)[2]
    psi = bfv.primitive_2n_root(q, N)
    rng = np.random.default_rng(7)
    a = rng.integers(0, q, size=N, dtype=np.uint64)
    b = rng.integers(0, q, size=N, dtype=np.uint64)
    assert np.array_equal(ring.negacyclic_mul(a, b, q, psi), ring.schoolbook(a, b, q))


def test_modular_ops_edge_operands():
    q = bfv.ntt_primes(1024, 60, 1)[0]
    vals = [0, 1, 2, q - 2, q - 1, q // 2, (q + 1) // 2, 1 << 59]
    a = np.array([x for x in vals for _ in vals], dtype=np.uint64)
    b = np.array([y for _ in vals for y in vals], dtype=np.uint64)
    assert ring.vec_mul(a, b, q).tolist() == [x * y % q for x in vals for y in vals]
    assert ring.vec_add(a, b, q).tolist() == [(x + y) % q for x in vals for y in vals]
    assert ring.vec_sub(a, b, q).tolist() == [(x - y) % q for x in vals for y in vals]
    assert ring.powmod(3, q - 1, q) == 1
    assert ring.invmod(12345, q) * 12345 % q == 1


@pytest.mark.parametrize("N", [8, 32])
def test_automorphism_definition_and_laws(N):
    q = bfv.ntt_primes(N, 60, 1)[0]
    psi = bfv.primitive_2n_root(q, N)
    rnd = random.Random(3 * N)
    a = [rnd.randrange(q) for _ in range(N)]
    b = [rnd.randrange(q) for _ in range(N)]
    A = np.array(a, dtype=np.uint64)
    B = np.array(b, dtype=np.uint64)
    for k in range(1, 2 * N, 2):
        sk = ring.automorphism(A, k, q)
        assert sk.tolist() == py_substitute(a, k, q)
        # ring homomorphism: sigma(ab) = sigma(a) sigma(b)
        lhs = ring.automorphism(ring.negacyclic_mul(A, B, q, psi), k, q)
        rhs = ring.negacyclic_mul(sk, ring.automorphism(B, k, q), q, psi)
        assert np.array_equal(lhs, rhs)
    assert np.array_equal(ring.automorphism(A, 1, q), A)
    for k1 in (3, 5, 2 * N - 1):
        for k2 in (3, 9, 2 * N - 3):
            lhs = ring.automorphism(ring.automorphism(A, k2, q), k1, q)
            rhs = ring.automorphism(A, k1 * k2 % (2 * N), q)
            assert np.array_equal(lhs, rhs)


@pytest.mark.parametrize("ns", [1, 2, 3])
def test_basis_conversion_against_crt(ns):
    N = 64
    chain = bfv.ntt_primes(N, 60, ns + 2)
    src, dst = chain[:ns], chain[ns:]
    S = 1
    for s in src:
        S *= s
    rng = np.random.default_rng(ns)
    X = [int(x) for x in rng.integers(0, 2**62, size=N)]
    X = [x % S for x in X]
    xs = np.array([[x % s for x in X] for s in src], dtype=np.uint64)
    for r in dst:
        y = ring.basis_convert(xs, src, r).tolist()
        for c in range(N):
            # result is X + u*S for some 0 <= u < ns (no overflow correction)
            diffs = [(X[c] + u * S) % r for u in range(ns)]
            assert y[c] in diffs


def test_prime_chain_against_sympy():
    sympy = pytest.importorskip("sympy")
    for N, bits, count in [(1 << 12, 54, 3), (1 << 13, 60, 4), (1 << 15, 60, 10)]:
        got = bfv.ntt_primes(N, bits, count)
        # brute force with an independent primality test: walk down every
        # candidate = 1 mod 2N below 2^bits
        want, p = [], ((1 << bits) - 2) // (2 * N) * (2 * N) + 1
        while len(want) < count:
            if sympy.isprime(p):
                want.append(p)
            p -= 2 * N
        assert got == want
        assert all(x < (1 << bits) and x % (2 * N) == 1 for x in got)
    # the largest 60-bit prime = 1 mod 2^16
    assert bfv.ntt_primes(1 << 15, 60, 1)[0] == 0xffffffffffc0001


def test_slot_root_and_generator():
    sympy = pytest.importorskip("sympy")
    for t in (40961, 65537, 12289, 257):
        assert bfv.smallest_generator(t) == sympy.primitive_root(t)
    assert bfv.smallest_generator(65537) == 3 and bfv.smallest_generator(40961) == 3
