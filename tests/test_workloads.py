"""The seeded input recipes that the oracle, the parity tests and the
benchmark share: each draw has the shape, range and structure its docstring
states (the paper's workloads are unspecified synthetic databases, Sec. 6),
and a seed always gives the same draw."""
import numpy as np
import pytest

import workloads as W


def _runs(pos):
    """Maximal runs of consecutive positions, as (start, length)."""
    runs, start = [], pos[0]
    for a, b in zip(pos[:-1], pos[1:]):
        if b != a + 1:
            runs.append((start, a - start + 1))
            start = b
    runs.append((start, pos[-1] - start + 1))
    return runs


@pytest.mark.parametrize("n,s,seed", [(1 << 20, 256, 0xC3), (4096, 100, 1), (64, 20, 2),
                                      (50, 1, 3)])
def test_clustered_matches(n, s, seed):
    pos = W.draw_matches_clustered(n, s, W.rng_for(seed, 2))
    assert pos.size == s and np.all(np.diff(pos) > 0) and pos[0] >= 0 and pos[-1] < n
    # runs of 1..8 records; a run never touches another, so the maximal runs
    # of the positions are the drawn runs themselves
    assert all(1 <= length <= 8 for _, length in _runs(pos))
    assert np.array_equal(pos, W.draw_matches_clustered(n, s, W.rng_for(seed, 2)))


def test_clustered_matches_are_clustered_at_c3():
    cfg = W.CONFIGS["c3"]
    q = W.draw_query(cfg)
    runs = _runs(q.positions)
    assert q.positions.size == 256 and cfg.pattern == "clustered"
    assert len(runs) < 256 / 2            # mean run length U{1..8} is 4.5 (the last cut)
    assert np.array_equal(np.flatnonzero(q.v), q.positions)


@pytest.mark.parametrize("name", ["c1", "c2", "tiny", "grouped", "paper"])
def test_uniform_queries(name):
    cfg = W.CONFIGS[name]
    q = W.draw_query(cfg)
    assert q.positions.size == cfg.s and len(set(q.positions.tolist())) == cfg.s
    assert np.all(np.diff(q.positions) > 0) and q.positions[-1] < cfg.n
    assert q.db.dtype == np.uint32 and q.db.size == cfg.n and int(q.db.max()) < cfg.t
    assert q.v.dtype == np.uint32 and int(q.v.sum()) == cfg.s
    assert set(np.unique(q.sk).tolist()) <= {-1, 0, 1} and q.sk.size == cfg.N
    again = W.draw_query(cfg)
    assert all(np.array_equal(a, b) for a, b in zip(
        (q.db, q.positions, q.sk), (again.db, again.positions, again.sk)))
    other = W.draw_query(cfg, seed=cfg.seed + 1)
    assert not np.array_equal(q.db, other.db)


def test_database_values_cover_the_plaintext_ring():
    db = W.draw_database(200_000, 65537, W.rng_for(5, 1))
    assert int(db.min()) < 10 and 65526 < int(db.max()) <= 65536
    assert abs(float(db.mean()) - 32768) < 300


def test_error_and_uniform_draws():
    e = W.draw_gaussian((64, 4096), W.rng_for(6, 0))
    assert e.dtype == np.int32 and int(np.abs(e).max()) <= W.TAIL
    assert abs(float(e.std()) - W.SIGMA) < 0.05 and abs(float(e.mean())) < 0.05
    moduli = [97, 2 ** 61 - 1, 65537]
    u = W.draw_uniform_mod(moduli, 1024, 3, W.rng_for(7, 0))
    assert u.shape == (3, 3, 1024) and u.dtype == np.uint64
    for i, q in enumerate(moduli):
        assert int(u[:, i].max()) < q
    assert float(u[:, 1].astype(np.float64).mean()) / (2 ** 61) == pytest.approx(0.5, abs=0.05)
    a, e2 = W.encryption_randomness(moduli, 1024, 2, seed=9)
    a2, e3 = W.encryption_randomness(moduli, 1024, 2, seed=9)
    assert np.array_equal(a, a2) and np.array_equal(e2, e3) and a.shape == (2, 3, 1024)
    keys = W.rotation_key_randomness(moduli, 64, 2, [3, 127], seed=9)
    assert set(keys) == {3, 127} and keys[3][0].shape == (2, 3, 64)
    assert not np.array_equal(keys[3][0], keys[127][0])
    # one element's draw does not depend on which other elements are drawn
    alone = W.rotation_key_randomness(moduli, 64, 2, [127], seed=9)
    assert np.array_equal(alone[127][0], keys[127][0])


def test_batched_mix_recipe():
    mix = W.batched_mix(64)
    assert len(mix) == 64 and mix == W.batched_mix(64)
    assert {q.log_n for q in mix} == {13, 14, 15}
    for q in mix:
        lg = q.n.bit_length() - 1
        assert q.n == 1 << lg and 12 <= lg <= 20
        assert 1 <= q.s <= min(1024, q.n // 16)
    assert [q.seed for q in mix] == [0xB0 + i for i in range(64)]
    for lg, p in W.RING_PARAMS.items():
        assert p["log_n"] == lg and (p["t"] - 1) % (2 << lg) == 0


def test_poisson_arrivals():
    arr = W.poisson_arrivals(500.0, 20_000, seed=3)
    assert np.all(np.diff(arr) > 0) and arr[0] > 0
    assert float(np.diff(arr).mean()) == pytest.approx(1 / 500.0, rel=0.03)
    assert np.array_equal(arr, W.poisson_arrivals(500.0, 20_000, seed=3))
