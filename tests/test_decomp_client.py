"""Client-side layout, rotation list and Decomp of the library without a
context or a GPU (pdq_plan_make_client, pdq_plan_galois_client,
pdq_decomp_client: host code of libpdq.so): the library's plans and Galois
elements equal the oracle's for every kind of plan, and its Decomp recovers
exactly the matching records from the closed-form answer slots of Eq. 1
(Alg. 6), as the oracle's Decomp does, with the same refusals."""
import ctypes
import functools

import numpy as np
import pytest

from oracle import bfv
from oracle import pdq as opdq
from paper_2408_17063_gb300 import pdq

FIELDS = ("n", "s", "s_prime", "B", "J", "H", "G_sz", "hpg", "G", "per_out", "n_out")


@functools.lru_cache(maxsize=None)
def ring(t, log_n):
    # an oracle parameter set with a short chain: the layout, the Galois
    # elements and the closed form read only its ring and t
    return bfv.Params(log_n=log_n, t=t, bits=40, L=1, K=1, dnum=1)


def to_struct(op, kind="answer", R=1):
    pl = pdq.Plan()
    for f in FIELDS:
        setattr(pl, f, getattr(op, f))
    pl.giants = op.giants
    pl.hclass = min(op.hpg, op.H)
    pl.ring_ratio = R
    pl.plain_db = 1 if kind == "plain_db" else 0
    return pl


def same_plan(lib_pl, op):
    return (all(getattr(lib_pl, f) == getattr(op, f) for f in FIELDS)
            and lib_pl.giants == op.giants and lib_pl.hclass == min(op.hpg, op.H)
            and lib_pl.ring_ratio == 1 and lib_pl.plain_db == 0)


SHAPES = [  # (t, log_n, n, s, B)
    (257, 3, 1, 1, 0), (257, 4, 7, 3, 0), (257, 7, 1000, 5, 0), (257, 7, 129, 64, 0),
    (40961, 6, 5000, 4, 0), (40961, 10, 2 ** 17, 16, 0), (40961, 12, 40960, 64, 8),
    (65537, 8, 65280, 2, 1), (65537, 8, 65281, 2, 2), (65537, 13, 16384, 16, 0),
    (65537, 13, 2 ** 17, 128, 0), (65537, 15, 2 ** 20, 256, 0), (65537, 15, 2 ** 20, 256, 32),
    (65537, 15, 2 ** 17, 1, 0), (65537, 15, 3, 4096, 128), (65537, 15, 2 ** 20, 1000, 0),
]


@pytest.mark.parametrize("t,log_n,n,s,B", SHAPES)
def test_client_plan_equals_oracle_plan(t, log_n, n, s, B):
    op = opdq.make_plan(ring(t, log_n), n, s, B or None)
    assert same_plan(pdq.plan_make_client(t, log_n, n, s, B), op)


@pytest.mark.parametrize("t,log_n,n,s,B", SHAPES)
def test_client_galois_elements_equal_the_oracle(t, log_n, n, s, B):
    """The rotations the schedule of Sec. 5.2 uses (Rot_col, baby and giant
    steps, the rotate-and-sum levels): the keys the client must send."""
    par = ring(t, log_n)
    op = opdq.make_plan(par, n, s, B or None)
    pl = pdq.plan_make_client(t, log_n, n, s, B)
    assert pdq.plan_galois_client(t, log_n, pl) == opdq.galois_elements(par, op)
    db = opdq.make_plan_plain_db(par, n, s, B or None)
    assert pdq.plan_galois_client(t, log_n, to_struct(db, kind="plain_db")) == \
        opdq.plain_db_galois_elements(par, db)


def test_client_galois_elements_of_a_switched_plan_and_refusals():
    big, small = ring(65537, 15), ring(65537, 13)
    op = opdq.make_switched_plan(big, small, 2 ** 17, 256)
    pl = to_struct(op, R=4)
    assert pdq.plan_galois_client(65537, 13, pl) == opdq.galois_elements(small, op)
    lib = pdq.load()
    cnt = ctypes.c_uint32()
    out = np.zeros(2, dtype=np.uint64)
    rc = lib.pdq_plan_galois_client(65537, 13, ctypes.byref(pl), out.ctypes.data, 2,
                                    ctypes.byref(cnt))
    assert rc == pdq.PDQ_E_NOMEM and cnt.value == len(opdq.galois_elements(small, op))
    pl.hpg += 1
    with pytest.raises(pdq.PdqError) as e:
        pdq.plan_galois_client(65537, 13, pl)
    assert e.value.code == pdq.PDQ_E_PARAM


def test_client_plan_refusals():
    lib = pdq.load()
    pl = pdq.Plan()
    bad = [(65537, 8, 10, 129, 0),      # s' = 256 > m = 128
           (257, 8, 10, 2, 0),          # t != 1 mod 2N
           (65539, 4, 10, 2, 0),        # t = 1 mod 2N is needed and t must be prime
           (65537, 2, 10, 1, 0),        # ring below 2^3
           (65537, 17, 10, 1, 0),       # ring above 2^16
           (65537, 10, 10, 16, 3),      # B does not divide s'
           (65537, 10, 10, 256, 256),   # B > 128
           (65537, 10, 10, 256, 4),     # 64 giant steps
           (65537, 10, 0, 1, 0), (65537, 10, 1, 0, 0)]
    for args in bad:
        assert lib.pdq_plan_make_client(*args, ctypes.byref(pl)) == pdq.PDQ_E_PARAM, args
        assert lib.pdq_last_error()
    assert lib.pdq_plan_make_client(65537, 10, 1, 1, 0, None) == pdq.PDQ_E_PARAM


def _case(t, log_n, n, s, seed, pattern="random", per_group=None):
    """Seeded index vector with at most s matches per record group, database
    values uniform in [0, t) (zeros included)."""
    par = ring(t, log_n)
    op = opdq.make_plan(par, n, s)
    rng = np.random.default_rng(seed)
    v = np.zeros(n, dtype=np.uint64)
    for gamma in range(op.G):
        lo, hi = gamma * op.G_sz, min((gamma + 1) * op.G_sz, n)
        if lo >= hi:
            continue
        k = min(hi - lo, s if per_group is None else per_group)
        k = int(rng.integers(0, k + 1)) if per_group is None else k
        if pattern == "clustered":
            start = int(rng.integers(lo, hi - k + 1))
            pos = np.arange(start, start + k)
        else:
            pos = rng.choice(np.arange(lo, hi), size=k, replace=False)
        v[pos] = 1
    db = rng.integers(0, t, size=n, dtype=np.uint64)
    db[rng.random(n) < 0.05] = 0
    truth = [(int(i), int(db[i])) for i in np.flatnonzero(v)]
    return par, op, v, db, truth


CASES = [  # (t, log_n, n, s, seed, pattern)
    (257, 3, 8, 1, 1, "random"), (257, 4, 16, 8, 2, "random"), (257, 6, 1000, 5, 3, "random"),
    (257, 7, 700, 64, 4, "clustered"), (40961, 6, 3000, 4, 5, "random"),
    (40961, 9, 90000, 16, 6, "clustered"), (65537, 8, 65280 * 2 + 17, 3, 7, "random"),
    (65537, 13, 16384, 16, 8, "random"), (65537, 13, 2 ** 17, 128, 9, "clustered"),
    (65537, 15, 2 ** 17, 256, 10, "clustered"), (65537, 15, 70000, 1, 11, "random"),
]


@pytest.mark.parametrize("t,log_n,n,s,seed,pattern", CASES)
def test_client_decomp_recovers_the_matches(t, log_n, n, s, seed, pattern):
    par, op, v, db, truth = _case(t, log_n, n, s, seed, pattern)
    slots = np.stack(opdq.expected_slots(par, op, v, db)).astype(np.uint32)
    pl = pdq.plan_make_client(t, log_n, n, s)
    got = pdq.decomp_client(t, log_n, pl, slots)
    assert got == truth
    assert got == opdq.decomp_slots(par, op, slots)


def test_client_decomp_full_groups_and_no_matches():
    # every group holding exactly s' matches, then none at all
    par, op, v, db, truth = _case(65537, 10, 3 * 65536 + 100, 8, 12, per_group=8)
    assert op.G == 4 and len(truth) == 8 * op.G
    pl = pdq.plan_make_client(65537, 10, v.size, 8)
    slots = np.stack(opdq.expected_slots(par, op, v, db)).astype(np.uint32)
    assert pdq.decomp_client(65537, 10, pl, slots) == truth
    zero = np.zeros_like(slots)
    assert pdq.decomp_client(65537, 10, pl, zero) == [] == opdq.decomp_slots(par, op, zero)


def test_client_decomp_refuses_what_the_oracle_refuses():
    t, log_n = 40961, 8
    par, op, v, db, _ = _case(t, log_n, 20000, 4, 13)
    pl = pdq.plan_make_client(t, log_n, 20000, 4)
    # one more match in a group than s' power sums can hold
    v2 = v.copy()
    v2[:] = 0
    v2[[3, 50, 77, 100, 129]] = 1
    over = np.stack(opdq.expected_slots(par, op, v2, db)).astype(np.uint32)
    with pytest.raises(opdq.DecodeError):
        opdq.decomp_slots(par, op, over)
    with pytest.raises(pdq.PdqError) as e:
        pdq.decomp_client(t, log_n, pl, over)
    assert e.value.code == pdq.PDQ_E_DECODE
    # values without indices: e-rows set, w-rows zero
    bad = np.zeros((op.n_out, par.N), dtype=np.uint32)
    bad[0, par.m] = 5
    with pytest.raises(opdq.DecodeError):
        opdq.decomp_slots(par, op, bad)
    with pytest.raises(pdq.PdqError) as e:
        pdq.decomp_client(t, log_n, pl, bad)
    assert e.value.code == pdq.PDQ_E_DECODE
    # a plan that is not the library's for this ring, a ring it would refuse
    tampered = pdq.plan_make_client(t, log_n, 20000, 4)
    tampered.G_sz += 1
    good = np.stack(opdq.expected_slots(par, op, v, db)).astype(np.uint32)
    for args in [(t, log_n, tampered), (t, log_n + 1, pl), (t + 2, log_n, pl), (t, 2, pl)]:
        with pytest.raises(pdq.PdqError) as e:
            pdq.decomp_client(*args, good)
        assert e.value.code == pdq.PDQ_E_PARAM


def test_client_decomp_reports_the_total_when_the_output_is_too_small():
    t, log_n = 65537, 9
    par, op, v, db, truth = _case(t, log_n, 4000, 16, 14, per_group=16)
    pl = pdq.plan_make_client(t, log_n, 4000, 16)
    slots = np.ascontiguousarray(np.stack(opdq.expected_slots(par, op, v, db)).astype(np.uint32))
    lib = pdq.load()
    cnt = ctypes.c_uint64()
    idx = np.zeros(4, dtype=np.uint64)
    val = np.zeros(4, dtype=np.uint32)
    rc = lib.pdq_decomp_client(t, log_n, ctypes.byref(pl), slots.ctypes.data, idx.ctypes.data,
                               val.ctypes.data, 4, ctypes.byref(cnt))
    assert rc == pdq.PDQ_E_NOMEM and cnt.value == len(truth) == 16
    assert [(int(i), int(x)) for i, x in zip(idx, val)] == truth[:4]
    rc = lib.pdq_decomp_client(t, log_n, ctypes.byref(pl), slots.ctypes.data, None, None, 0,
                               ctypes.byref(cnt))
    assert rc == pdq.PDQ_E_NOMEM and cnt.value == 16


@pytest.mark.parametrize("big_log_n,log_n,n,s", [(15, 13, 2 ** 17, 256), (12, 9, 10000, 8),
                                                 (8, 5, 700, 2)])
def test_client_decomp_of_ring_switched_answers(big_log_n, log_n, n, s):
    """A ring-switched answer (Sec. 5.3) keeps the big ring's record groups in
    the subring's slots: the library accepts the oracle's switched plan (so
    the two layouts agree) and decodes the closed form laid out by it."""
    t = 65537
    big, small = ring(t, big_log_n), ring(t, log_n)
    op = opdq.make_switched_plan(big, small, n, s)
    pl = to_struct(op, R=big.N // small.N)
    rng = np.random.default_rng(big_log_n * 100 + log_n)
    v = np.zeros(n, dtype=np.uint64)
    for gamma in range(op.G):
        lo, hi = gamma * op.G_sz, min((gamma + 1) * op.G_sz, n)
        if lo < hi:
            v[rng.choice(np.arange(lo, hi), size=min(s, hi - lo), replace=False)] = 1
    db = rng.integers(1, t, size=n, dtype=np.uint64)
    slots = np.stack(opdq.expected_slots(small, op, v, db)).astype(np.uint32)
    truth = [(int(i), int(db[i])) for i in np.flatnonzero(v)]
    assert pdq.decomp_client(t, log_n, pl, slots) == truth == opdq.decomp_slots(small, op, slots)


def test_client_decomp_of_unencrypted_database_answers():
    """The Answer on an unencrypted database has the masked Answer's layout
    with its own choice of B: the library accepts the oracle's plan."""
    t, log_n, n, s = 65537, 11, 50000, 32
    par = ring(t, log_n)
    op = opdq.make_plan_plain_db(par, n, s)
    pl = to_struct(op, kind="plain_db")
    _, _, v, db, truth = _case(t, log_n, n, s, 15)
    slots = np.stack(opdq.expected_slots(par, op, v, db)).astype(np.uint32)
    assert pdq.decomp_client(t, log_n, pl, slots) == truth
    # any admissible B is a plan of this kind (B changes the server's work, not
    # the layout); a changed layout is not
    other = to_struct(op, kind="plain_db")
    other.B = op.B * 2 if op.B * 2 <= op.s_prime else op.B // 2
    other.giants = op.s_prime // other.B
    assert pdq.decomp_client(t, log_n, other, slots) == truth
    other.per_out //= 2
    with pytest.raises(pdq.PdqError) as e:
        pdq.decomp_client(t, log_n, other, slots)
    assert e.value.code == pdq.PDQ_E_PARAM


BIG_T = 2013265921          # 15 * 2^27 + 1: a prime = 1 mod 2N for every ring up to 2^16


@pytest.mark.parametrize("log_n,n,s,seed", [(4, 16, 8, 21), (10, 5000, 64, 22), (13, 70000, 16, 23),
                                            (15, 2 ** 17, 128, 24)])
def test_client_decomp_with_a_large_plaintext_prime(log_n, n, s, seed):
    """With t near 2^31 a group holds t - 1 records, far too many nodes to try
    one by one: the roots come from gcd(g, X^t - X) and its splitting (the
    Cantor-Zassenhaus route of Sec. 3.1), and the matches are recovered
    exactly, as the closed form of Eq. 1 lays them out."""
    par, op, v, db, truth = _case(BIG_T, log_n, n, s, seed, per_group=s)
    assert op.G == 1 and op.G_sz == BIG_T - 1
    pl = pdq.plan_make_client(BIG_T, log_n, n, s)
    slots = np.stack(opdq.expected_slots(par, op, v, db)).astype(np.uint32)
    assert pdq.decomp_client(BIG_T, log_n, pl, slots) == truth
    # one match more than s' power sums can hold is refused
    if s < n:
        v2 = v.copy()
        v2[np.flatnonzero(v2 == 0)[:1]] = 1
        if int(v2.sum()) > op.s_prime:
            over = np.stack(opdq.expected_slots(par, op, v2, db)).astype(np.uint32)
            with pytest.raises(pdq.PdqError) as e:
                pdq.decomp_client(BIG_T, log_n, pl, over)
            assert e.value.code == pdq.PDQ_E_DECODE


def test_client_decomp_of_many_groups_and_the_first_failing_group():
    """Groups decode independently (on several host threads): 40 groups give
    the oracle's answer; an overflow planted in group 7 and values without
    indices in group 23 are reported as group 7's error, the first in group
    order, with its own message."""
    t, log_n = 257, 5                     # G_sz = 256 records per group, 16 slots per row
    n = 40 * 256 - 3
    par, op, v, db, truth = _case(t, log_n, n, 2, 31)
    assert op.G == 40 and op.n_out == 5
    pl = pdq.plan_make_client(t, log_n, n, 2)
    slots = np.stack(opdq.expected_slots(par, op, v, db)).astype(np.uint32)
    assert pdq.decomp_client(t, log_n, pl, slots) == truth == opdq.decomp_slots(par, op, slots)
    v2 = v.copy()
    lo = 7 * op.G_sz
    v2[lo:lo + op.G_sz] = 0
    v2[[lo + 3, lo + 40, lo + 99]] = 1    # three matches, s' = 2
    bad = np.stack(opdq.expected_slots(par, op, v2, db)).astype(np.uint32)
    with pytest.raises(opdq.DecodeError):
        opdq.decomp_slots(par, op, bad)
    c, o = divmod(23, op.per_out)
    bad[c, par.m + o * op.s_prime] = 5     # group 23: an e-row value, its w-rows zeroed
    bad[c, o * op.s_prime:(o + 1) * op.s_prime] = 0
    with pytest.raises(pdq.PdqError) as e:
        pdq.decomp_client(t, log_n, pl, bad)
    assert e.value.code == pdq.PDQ_E_DECODE
    assert "values without indices" not in str(e.value)
    # group 23's error alone is its own
    only23 = slots.copy()
    only23[c, par.m + o * op.s_prime] = 5
    only23[c, o * op.s_prime:(o + 1) * op.s_prime] = 0
    with pytest.raises(pdq.PdqError) as e:
        pdq.decomp_client(t, log_n, pl, only23)
    assert e.value.code == pdq.PDQ_E_DECODE and "values without indices" in str(e.value)


@pytest.mark.parametrize("seed", range(6))
def test_client_decomp_repeats_exactly(seed):
    """The same answer decoded again and again (threads racing on shared
    state would show here) gives the same records every time."""
    t, log_n, n, s = 65537, 9, 65536 * 3 + 700, 16
    par, op, v, db, truth = _case(t, log_n, n, s, 40 + seed, pattern="clustered")
    pl = pdq.plan_make_client(t, log_n, n, s)
    slots = np.stack(opdq.expected_slots(par, op, v, db)).astype(np.uint32)
    for _ in range(5):
        assert pdq.decomp_client(t, log_n, pl, slots) == truth
