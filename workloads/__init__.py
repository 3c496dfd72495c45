"""Seeded synthetic inputs for the private-database-query hot path.

This module is shared by the CPU oracle and the CUDA library's tests and
benchmark.  It holds none of the method's arithmetic: it only draws random
numbers (database values, match positions, secret-key coefficients, error
samples and uniform polynomial coefficients below moduli that the caller
supplies) from ``numpy.random.Generator(PCG64(seed))``.

The workload shapes follow the paper's experiments (Sec. 6: unspecified
synthetic databases, sparsity s, database length n) and the parameter sets
used for this implementation:

* ``c1``  ring N=2^12, t=40961, 2 ciphertext primes of 54 bits + 1 special
  prime, n=4096 records, s=16 matches at uniform positions.
* ``c2``  N=2^13, t=65537, 3 x 60-bit + 1 special, n=2^16, s=64 uniform.
* ``c3``  N=2^15, t=65537, 8 x 60-bit + 2 special (4 key-switching digits),
  n=2^20, s=256 clustered matches (runs of 1..8 records).
* ``tiny*``, ``small``, ``grouped`` small rings for exhaustive CPU checks and
  GPU edge cases (ragged record counts, several record groups).

Notation: ``N`` is the ring dimension (the paper's n) and ``n`` the number
of database records (the paper's N); ``t`` is the plaintext prime (the
paper's p).
"""
from __future__ import annotations

import dataclasses

import numpy as np

SIGMA = 3.2          # discrete Gaussian error width
TAIL = 19            # |e| <= TAIL (about 6 sigma)


@dataclasses.dataclass(frozen=True)
class Config:
    name: str
    log_n: int         # ring dimension N = 2^log_n
    t: int             # plaintext prime, t = 1 mod 2N
    prime_bits: int    # bit size of every RNS prime
    L: int             # ciphertext primes
    K: int             # special primes (hybrid key switching)
    dnum: int          # key-switching digits
    n: int             # database records
    s: int             # number of matches (sparsity)
    pattern: str       # "uniform" or "clustered"
    seed: int

    @property
    def N(self) -> int:
        return 1 << self.log_n


CONFIGS = {
    "c1": Config("c1", 12, 40961, 54, 2, 1, 2, 4096, 16, "uniform", 0xC1),
    "c2": Config("c2", 13, 65537, 60, 3, 1, 3, 1 << 16, 64, "uniform", 0xC2),
    "c3": Config("c3", 15, 65537, 60, 8, 2, 4, 1 << 20, 256, "clustered", 0xC3),
    # small rings for exhaustive CPU checks and fast GPU edge cases
    "tiny": Config("tiny", 5, 12289, 54, 2, 1, 2, 40, 3, "uniform", 0x71),
    "tiny2": Config("tiny2", 6, 12289, 60, 3, 2, 2, 200, 5, "uniform", 0x72),
    "small": Config("small", 10, 12289, 60, 3, 1, 3, 5000, 20, "uniform", 0x73),
    # several record groups (n > t-1) and two output ciphertexts
    "grouped": Config("grouped", 6, 257, 60, 2, 1, 2, 2000, 5, "uniform", 0x74),
    # the ring and modulus of the paper's experiments (2^13, t = 65537, two
    # 54-bit primes; one special prime of the same size), Table III's n = 2^13
    "paper": Config("paper", 13, 65537, 54, 2, 1, 2, 1 << 13, 16, "uniform", 0x2408),
    # 40-bit primes: far from a power of two (the library's generic reduction)
    "tiny40": Config("tiny40", 6, 12289, 40, 3, 2, 2, 200, 5, "uniform", 0x75),
}


def rng_for(seed: int, stream: int = 0) -> np.random.Generator:
    """Independent generator for (seed, stream)."""
    return np.random.Generator(np.random.PCG64([int(seed), int(stream)]))


def draw_database(n: int, t: int, rng: np.random.Generator) -> np.ndarray:
    """n record values uniform in [0, t) as uint32."""
    return rng.integers(0, t, size=n, dtype=np.uint64).astype(np.uint32)


def draw_matches_uniform(n: int, s: int, rng: np.random.Generator) -> np.ndarray:
    """s distinct record positions uniform in [0, n), sorted."""
    return np.sort(rng.choice(n, size=s, replace=False)).astype(np.int64)


def draw_matches_clustered(n: int, s: int, rng: np.random.Generator,
                           max_run: int = 8) -> np.ndarray:
    """Exactly s match positions made of runs of 1..max_run consecutive records
    at uniform starts.  A run overlapping or touching an earlier run is
    redrawn; the last run is cut so that the total is s."""
    taken = np.zeros(n + 2, dtype=bool)
    out = []
    remaining = s
    guard = 0
    while remaining > 0:
        guard += 1
        if guard > 1_000_000:
            raise RuntimeError("cannot place clustered matches")
        run = int(rng.integers(1, max_run + 1))
        run = min(run, remaining)
        start = int(rng.integers(0, n - run + 1))
        lo, hi = start, start + run          # [lo, hi)
        # reject overlap or adjacency (positions lo-1 .. hi inclusive)
        if taken[max(lo - 1, 0):hi + 1].any():
            continue
        taken[lo:hi] = True
        out.extend(range(lo, hi))
        remaining -= run
    return np.sort(np.asarray(out, dtype=np.int64))


def index_vector(n: int, positions: np.ndarray) -> np.ndarray:
    """0/1 vector of length n with ones at positions (uint32)."""
    v = np.zeros(n, dtype=np.uint32)
    v[positions] = 1
    return v


def draw_ternary(N: int, rng: np.random.Generator) -> np.ndarray:
    """Secret-key coefficients uniform in {-1, 0, 1} (int8)."""
    return rng.integers(-1, 2, size=N, dtype=np.int64).astype(np.int8)


_GAUSS_SUPPORT = np.arange(-TAIL, TAIL + 1)
_GAUSS_P = np.exp(-(_GAUSS_SUPPORT.astype(np.float64) ** 2) / (2 * SIGMA * SIGMA))
_GAUSS_P /= _GAUSS_P.sum()


def draw_gaussian(shape, rng: np.random.Generator) -> np.ndarray:
    """Discrete Gaussian samples (sigma 3.2, |x| <= 19) as int32."""
    return rng.choice(_GAUSS_SUPPORT, size=shape, p=_GAUSS_P).astype(np.int32)


def draw_uniform_mod(moduli, N: int, count: int, rng: np.random.Generator) -> np.ndarray:
    """uint64 array [count][len(moduli)][N]; limb i uniform in [0, moduli[i])."""
    out = np.empty((count, len(moduli), N), dtype=np.uint64)
    for i, q in enumerate(moduli):
        out[:, i, :] = rng.integers(0, int(q), size=(count, N), dtype=np.uint64)
    return out


@dataclasses.dataclass
class QueryInputs:
    """Everything random that one query instance needs."""
    db: np.ndarray          # [n] uint32 record values
    positions: np.ndarray   # [s] sorted match positions
    v: np.ndarray           # [n] uint32 0/1 index vector
    sk: np.ndarray          # [N] int8 ternary secret


def draw_query(cfg: Config, seed: int | None = None) -> QueryInputs:
    seed = cfg.seed if seed is None else seed
    db = draw_database(cfg.n, cfg.t, rng_for(seed, 1))
    if cfg.pattern == "clustered":
        pos = draw_matches_clustered(cfg.n, cfg.s, rng_for(seed, 2))
    else:
        pos = draw_matches_uniform(cfg.n, cfg.s, rng_for(seed, 2))
    sk = draw_ternary(cfg.N, rng_for(seed, 3))
    return QueryInputs(db=db, positions=pos, v=index_vector(cfg.n, pos), sk=sk)


def encryption_randomness(moduli_q, N: int, count: int, seed: int, stream: int = 4):
    """(a, e) for `count` symmetric encryptions: a uniform over the ciphertext
    primes [count][L][N] uint64, e Gaussian [count][N] int32."""
    rng = rng_for(seed, stream)
    a = draw_uniform_mod(moduli_q, N, count, rng)
    e = draw_gaussian((count, N), rng)
    return a, e


def rotation_key_randomness(moduli_ext, N: int, digits: int, galois_elts, seed: int,
                            stream: int = 5):
    """Per Galois element (in the order given): (a, e) with a uniform over the
    extended basis [digits][L+K][N] uint64 and e Gaussian [digits][N] int32."""
    out = {}
    for idx, k in enumerate(galois_elts):
        rng = rng_for(seed, stream * 1_000_003 + int(k))
        a = draw_uniform_mod(moduli_ext, N, digits, rng)
        e = draw_gaussian((digits, N), rng)
        out[int(k)] = (a, e)
    return out



# Parameter sets of the mixed-ring workloads, by log2 N (the N = 2^14 chain
# is this implementation's choice: 4 x 60-bit + 2 special primes, 2 digits).
RING_PARAMS = {
    13: dict(log_n=13, t=65537, prime_bits=60, L=3, K=1, dnum=3),
    14: dict(log_n=14, t=65537, prime_bits=60, L=4, K=2, dnum=2),
    15: dict(log_n=15, t=65537, prime_bits=60, L=8, K=2, dnum=4),
}


@dataclasses.dataclass(frozen=True)
class MixQuery:
    log_n: int      # ring dimension 2^log_n
    n: int          # records
    s: int          # matches
    seed: int


def batched_mix(count: int = 64, base_seed: int = 0xB0) -> list[MixQuery]:
    """Independent queries of the batched / served workloads: ring dimension
    uniform over {2^13, 2^14, 2^15}, log2 n uniform over the integers 12..20,
    s uniform in [1, min(1024, n/16)], query q seeded with base_seed + q."""
    out = []
    for q in range(count):
        rng = rng_for(base_seed + q, 0)
        log_n = int(rng.integers(13, 16))
        n = 1 << int(rng.integers(12, 21))
        s = int(rng.integers(1, min(1024, n // 16) + 1))
        out.append(MixQuery(log_n, n, s, base_seed + q))
    return out


def poisson_arrivals(rate_per_s: float, count: int, seed: int) -> np.ndarray:
    """Arrival times (seconds from 0) of a Poisson process."""
    rng = rng_for(seed, 7)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))
