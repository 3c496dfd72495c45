"""Oracle for the RLWE scheme under the private database query: parameters,
SIMD slot encoding, symmetric BFV encryption/decryption, Galois
automorphisms and hybrid key switching.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper runs HElib's BGV (Sec. 5.1) with ring dimension a power of two and
plaintext prime t = 1 mod 2N, so that the plaintext ring Z_t[X]/(X^N+1) is
the slot algebra Z_t^{2 x N/2}; Rot_row(.; r) is the automorphism X -> X^{3^r}
and Rot_col the automorphism X -> X^{2N-1} (Sec. 5.1).  This oracle uses the
BFV flavour of the same ring and slot algebra.  Every choice the paper leaves
open (prime chain, slot order, lift, key-switching method) is fixed here and
listed with its reason in the design notes; the GPU library must reproduce
these bits exactly.

Polynomials are uint64 arrays [limbs][N] in coefficient form, canonical
residues; a ciphertext is [2][L][N].
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import ring


# ---------------------------------------------------------------- primes ----

_MR_BASES = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)


def is_prime(n: int) -> bool:
    """Deterministic Miller-Rabin for n < 3.3e24 (fixed witness set)."""
    if n < 2:
        return False
    for p in _MR_BASES:
        if n % p == 0:
            return n == p
    d, r = n - 1, 0
    while d % 2 == 0:
        d //= 2
        r += 1
    for a in _MR_BASES:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(r - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def ntt_primes(N: int, bits: int, count: int) -> list[int]:
    """The `count` largest primes p < 2^bits with p = 1 mod 2N, descending."""
    step = 2 * N
    p = ((1 << bits) - 2) // step * step + 1
    out = []
    while len(out) < count:
        if p < step:
            raise ValueError("not enough NTT primes")
        if is_prime(p):
            out.append(p)
        p -= step
    return out


def primitive_2n_root(q: int, N: int) -> int:
    """Some element of multiplicative order exactly 2N modulo the prime q."""
    assert (q - 1) % (2 * N) == 0
    for x in range(2, q):
        c = pow(x, (q - 1) // (2 * N), q)
        if pow(c, N, q) == q - 1:
            return c
    raise ValueError("no root")


def smallest_generator(t: int) -> int:
    """Smallest g whose powers give every nonzero residue mod the prime t."""
    n = t - 1
    factors, f, x = [], 2, n
    while f * f <= x:
        if x % f == 0:
            factors.append(f)
            while x % f == 0:
                x //= f
        f += 1
    if x > 1:
        factors.append(x)
    for g in range(2, t):
        if all(pow(g, n // f, t) != 1 for f in factors):
            return g
    raise ValueError("no generator")


# ------------------------------------------------------------ parameters ----

@dataclass
class Params:
    """One parameter set.  Special primes are the K largest NTT primes below
    2^bits, ciphertext primes q_0 > ... > q_{L-1} the next L.  The extended
    basis is ordered Q limbs first, then P limbs."""
    log_n: int
    t: int
    bits: int
    L: int
    K: int
    dnum: int
    chain: tuple | None = None   # (special primes, then ciphertext primes) instead of the search
    N: int = field(init=False)
    m: int = field(init=False)
    q: list = field(init=False)
    p: list = field(init=False)
    ext: list = field(init=False)
    psi: list = field(init=False)
    zeta: int = field(init=False)
    Q: int = field(init=False)
    P: int = field(init=False)
    delta: int = field(init=False)
    digits: list = field(init=False)

    def __post_init__(self):
        self.N = 1 << self.log_n
        self.m = self.N // 2
        if (self.t - 1) % (2 * self.N) or not is_prime(self.t):
            raise ValueError("t must be a prime = 1 mod 2N")
        if self.chain is None:
            chain = ntt_primes(self.N, self.bits, self.K + self.L)
        else:
            chain = [int(r) for r in self.chain]
            if len(chain) != self.K + self.L or any(
                    (r - 1) % (2 * self.N) or r >= 1 << self.bits or not is_prime(r) for r in chain):
                raise ValueError("chain: need K + L primes = 1 mod 2N below 2^bits")
        self.p = chain[:self.K]
        self.q = chain[self.K:]
        self.ext = self.q + self.p
        self.psi = [primitive_2n_root(r, self.N) for r in self.ext]
        # Slot root: zeta = g^{(t-1)/2N} with g the smallest generator of
        # Z_t^* (g = 3 for t = 40961 and t = 65537).
        self.zeta = pow(smallest_generator(self.t), (self.t - 1) // (2 * self.N), self.t)
        self.Q = math.prod(self.q)
        self.P = math.prod(self.p)
        self.delta = self.Q // self.t
        alpha = -(-self.L // self.dnum)
        self.digits = [list(range(b, min(b + alpha, self.L)))
                       for b in range(0, self.L, alpha)]

    @classmethod
    def from_config(cls, cfg) -> "Params":
        return cls(cfg.log_n, cfg.t, cfg.prime_bits, cfg.L, cfg.K, cfg.dnum)

    @classmethod
    def subring(cls, par: "Params", log_n: int) -> "Params":
        """The parameters of the subring Z[Y]/(Y^N'+1), Y = X^(N/N'), of
        par's ring (ring switching, Sec. 5.3): the same t, digits and primes
        (each = 1 mod 2N, hence 1 mod 2N'), ring dimension N' = 2^log_n."""
        if not 3 <= log_n < par.log_n:
            raise ValueError("subring: need a smaller ring dimension")
        return cls(log_n, par.t, par.bits, par.L, par.K, par.dnum, chain=tuple(par.p + par.q))

    # slot (row rho, column c) <-> evaluation exponent (-1)^rho 3^c mod 2N
    def slot_exponents(self) -> np.ndarray:
        """[2*m] exponents e(rho, c); slot index rho*m + c."""
        e = np.empty(self.N, dtype=np.int64)
        g = 1
        for c in range(self.m):
            e[c] = g
            e[self.m + c] = (2 * self.N - g) % (2 * self.N)
            g = g * 3 % (2 * self.N)
        return e

    def galois_rot(self, r: int) -> int:
        """Galois element of Rot_row(.; r): 3^r mod 2N (r may be negative)."""
        return pow(3, r % self.m, 2 * self.N)

    @property
    def galois_col(self) -> int:
        """Galois element of Rot_col: X -> X^{2N-1}."""
        return 2 * self.N - 1


# ---------------------------------------------------------------- encoding ---

def encode(par: Params, slots) -> np.ndarray:
    """Slots (length N, index rho*m + c) -> plaintext coefficients in [0, t).

    The plaintext m(X) is the unique polynomial of degree < N with
    m(zeta^{e(rho,c)}) = slot(rho, c); it is obtained by interpolation (the
    inverse of the negacyclic transform mod t)."""
    slots = np.asarray(slots, dtype=np.uint64) % par.t
    vals = np.zeros(par.N, dtype=np.uint64)
    vals[(par.slot_exponents() - 1) // 2] = slots
    return ring.ntt_inverse(vals, par.t, par.zeta)


def decode(par: Params, coeffs) -> np.ndarray:
    """Plaintext coefficients -> slot values (uint64, index rho*m + c)."""
    vals = ring.ntt_forward(np.asarray(coeffs, dtype=np.uint64) % par.t, par.t, par.zeta)
    return vals[(par.slot_exponents() - 1) // 2]


def lift(par: Params, coeffs, moduli) -> np.ndarray:
    """Centred lift of a plaintext (coefficients in [0,t)) to the given RNS
    primes: c <= (t-1)/2 stays c, larger c becomes c - t."""
    c = np.asarray(coeffs, dtype=np.uint64)
    neg = c > (par.t - 1) // 2
    out = np.empty((len(moduli), par.N), dtype=np.uint64)
    for i, r in enumerate(moduli):
        out[i] = np.where(neg, np.uint64(r) - (np.uint64(par.t) - c), c)
    return out


def signed_to_rns(x, moduli) -> np.ndarray:
    """Small signed integer polynomial -> residues [len(moduli)][N]."""
    x = np.asarray(x, dtype=np.int64)
    out = np.empty((len(moduli), x.shape[-1]), dtype=np.uint64)
    for i, r in enumerate(moduli):
        out[i] = np.where(x < 0, np.uint64(r) - (-x).astype(np.uint64), x.astype(np.uint64))
    return out


# ------------------------------------------------------- limb-wise ring ops -

def poly_mul(par: Params, a, b, limbs) -> np.ndarray:
    """Ring product limb by limb; `limbs` are indices into the extended basis."""
    return np.stack([ring.negacyclic_mul(a[i], b[i], par.ext[l], par.psi[l])
                     for i, l in enumerate(limbs)])


def poly_add(par: Params, a, b, limbs) -> np.ndarray:
    return np.stack([ring.vec_add(a[i], b[i], par.ext[l]) for i, l in enumerate(limbs)])


def poly_sub(par: Params, a, b, limbs) -> np.ndarray:
    return np.stack([ring.vec_sub(a[i], b[i], par.ext[l]) for i, l in enumerate(limbs)])


def poly_neg(par: Params, a, limbs) -> np.ndarray:
    z = np.zeros_like(a[0])
    return np.stack([ring.vec_sub(z, a[i], par.ext[l]) for i, l in enumerate(limbs)])


def poly_automorphism(par: Params, a, k: int, limbs) -> np.ndarray:
    return np.stack([ring.automorphism(a[i], k, par.ext[l]) for i, l in enumerate(limbs)])


def qlimbs(par: Params) -> list[int]:
    return list(range(par.L))


def extlimbs(par: Params) -> list[int]:
    return list(range(par.L + par.K))


# --------------------------------------------------------- encrypt/decrypt --

def encrypt(par: Params, sk, m_coeffs, a, e) -> np.ndarray:
    """Symmetric BFV encryption of plaintext m (coefficients in [0,t)):
    c1 = a, c0 = -a*s + e + Delta*m  (mod each q_i), Delta = floor(Q/t).
    a: [L][N] uniform residues, e: [N] small integers (both supplied)."""
    ql = qlimbs(par)
    s = signed_to_rns(sk, par.q)
    a = np.asarray(a, dtype=np.uint64)
    as_ = poly_mul(par, a, s, ql)
    e_r = signed_to_rns(e, par.q)
    m = np.asarray(m_coeffs, dtype=np.uint64)
    dm = np.stack([ring.vec_scale(ring.vec_reduce(m, par.q[i]), par.delta % par.q[i], par.q[i])
                   for i in ql])
    c0 = poly_add(par, poly_sub(par, e_r, as_, ql), dm, ql)
    return np.stack([c0, a.copy()])


def crt_compose(par: Params, x) -> list[int]:
    """Residues [L][N] modulo q_0..q_{L-1} -> the integers in [0, Q)."""
    terms = []
    for i, qi in enumerate(par.q):
        hat = par.Q // qi
        coef = hat * pow(hat % qi, -1, qi)
        terms.append((coef, x[i].tolist()))
    out = []
    Q = par.Q
    for c in range(par.N):
        out.append(sum(coef * xs[c] for coef, xs in terms) % Q)
    return out


def decrypt_coeffs(par: Params, sk, ct, with_noise: bool = False):
    """x = [c0 + c1*s]_Q in [0,Q); m = floor((t*x + floor(Q/2)) / Q) mod t.
    With with_noise also returns max |t*x - Q*round(t*x/Q)| / Q (the invariant
    noise; decryption is correct while it is below 1/2)."""
    ql = qlimbs(par)
    s = signed_to_rns(sk, par.q)
    x = poly_add(par, ct[0], poly_mul(par, ct[1], s, ql), ql)
    X = crt_compose(par, x)
    Q, t = par.Q, par.t
    m = np.array([((t * xv + Q // 2) // Q) % t for xv in X], dtype=np.uint64)
    if not with_noise:
        return m
    worst = 0
    for xv in X:
        r = (t * xv) % Q
        r = min(r, Q - r)
        worst = max(worst, r)
    return m, worst / Q


def decrypt(par: Params, sk, ct) -> np.ndarray:
    """Decrypt and decode to slots (index rho*m + c)."""
    return decode(par, decrypt_coeffs(par, sk, ct))


def noise_budget_bits(par: Params, sk, ct) -> float:
    """-log2(2 * invariant noise): bits left before decryption fails."""
    _, v = decrypt_coeffs(par, sk, ct, with_noise=True)
    return float("inf") if v == 0 else -math.log2(2 * v)


def pt_mul(par: Params, ct, pt_lifted) -> np.ndarray:
    """Plaintext-ciphertext product: each ciphertext polynomial times the
    lifted plaintext ([L][N]) in R_Q."""
    ql = qlimbs(par)
    return np.stack([poly_mul(par, ct[0], pt_lifted, ql), poly_mul(par, ct[1], pt_lifted, ql)])


def ct_add(par: Params, a, b) -> np.ndarray:
    ql = qlimbs(par)
    return np.stack([poly_add(par, a[0], b[0], ql), poly_add(par, a[1], b[1], ql)])


# ------------------------------------------------------------ key switching -

def rotation_key(par: Params, sk, k: int, a, e) -> np.ndarray:
    """Hybrid key-switching key from sigma_k(s) to s, one pair per digit beta:
      b_beta = -a_beta*s + e_beta + [q_i in digit beta] * P * sigma_k(s)  (mod each prime)
    over the extended basis Q u P.  a: [digits][L+K][N], e: [digits][N].
    Returns [digits][2][L+K][N] holding (b_beta, a_beta)."""
    el = extlimbs(par)
    s = signed_to_rns(sk, par.ext)
    sk_k = poly_automorphism(par, s, k, el)
    out = []
    for b_idx, digit in enumerate(par.digits):
        a_b = np.asarray(a[b_idx], dtype=np.uint64)
        e_b = signed_to_rns(e[b_idx], par.ext)
        b = poly_sub(par, e_b, poly_mul(par, a_b, s, el), el)
        for i in digit:
            qi = par.q[i]
            b[i] = ring.vec_add(b[i], ring.vec_scale(sk_k[i], par.P % qi, qi), qi)
        out.append(np.stack([b, a_b.copy()]))
    return np.stack(out)


def mod_up(par: Params, x, digit) -> np.ndarray:
    """Raise the digit's residues of x ([L][N], coefficient form) to the whole
    extended basis: limbs of the digit are copied, every other prime r gets
    sum_{i in digit} [x_i (Q_b/q_i)^{-1}]_{q_i} (Q_b/q_i) mod r."""
    src = [par.q[i] for i in digit]
    xs = np.stack([x[i] for i in digit])
    out = np.empty((par.L + par.K, par.N), dtype=np.uint64)
    for l, r in enumerate(par.ext):
        if l < par.L and l in digit:
            out[l] = x[l]
        else:
            out[l] = ring.basis_convert(xs, src, r)
    return out


def mod_down(par: Params, y) -> np.ndarray:
    """Divide an extended-basis polynomial by P (floor-like, no rounding):
    out_i = (y_i - sum_k [y_{p_k} (P/p_k)^{-1}]_{p_k} (P/p_k)) * P^{-1}  mod q_i."""
    yp = np.stack([y[par.L + k] for k in range(par.K)])
    out = np.empty((par.L, par.N), dtype=np.uint64)
    for i, qi in enumerate(par.q):
        conv = ring.basis_convert(yp, par.p, qi)
        out[i] = ring.vec_scale(ring.vec_sub(y[i], conv, qi), pow(par.P % qi, -1, qi), qi)
    return out


def mod_switch(par: Params, low: Params, ct) -> np.ndarray:
    """Modulus switching to smaller parameters (the paper runs Comp with
    smaller parameters than the query, Sec. 6): a ciphertext over
    Q = q_0..q_{L-1} ([2][L][N], coefficient form) to Q' = q_0..q_{L'-1}, the
    ciphertext primes of `low` (the first L' of par's), dividing by the
    dropped primes D = q_{L'}..q_{L-1} with the ModDown formula (floor-like):
      c'_i = (c_i - sum_k [c_{d_k} (D/d_k)^{-1}]_{d_k} (D/d_k)) D^{-1}  mod q_i.
    c0 + c1 s = Delta m + e over Q becomes Delta' m + e' over Q'."""
    if (low.N, low.t) != (par.N, par.t) or low.L >= par.L or low.q != par.q[:low.L]:
        raise ValueError("mod_switch: the smaller parameters must keep a prefix of the primes")
    dropped = par.q[low.L:]
    D = math.prod(dropped)
    out = np.empty((2, low.L, par.N), dtype=np.uint64)
    for p_idx in range(2):
        yd = np.stack([ct[p_idx][low.L + k] for k in range(len(dropped))])
        for i, qi in enumerate(low.q):
            conv = ring.basis_convert(yd, dropped, qi)
            out[p_idx][i] = ring.vec_scale(ring.vec_sub(ct[p_idx][i], conv, qi), pow(D % qi, -1, qi), qi)
    return out


def mod_up_all(par: Params, c1) -> list[np.ndarray]:
    """The hoistable part of a key switch: one raised polynomial per digit."""
    return [mod_up(par, c1, d) for d in par.digits]


def rotate_hoisted(par: Params, ct, raised, k: int, key) -> np.ndarray:
    """sigma_k followed by key switching, with the digits of c1 raised BEFORE
    the automorphism (so the raised digits can be shared by all rotations of
    the same ciphertext):
      (A0, A1) = sum_beta sigma_k(raised_beta) * (b_beta, a_beta)  over Q u P
      Rot(ct) = (sigma_k(c0) + ModDown(A0), ModDown(A1))."""
    el = extlimbs(par)
    ql = qlimbs(par)
    A0 = np.zeros((par.L + par.K, par.N), dtype=np.uint64)
    A1 = np.zeros_like(A0)
    for b_idx, _ in enumerate(par.digits):
        d = poly_automorphism(par, raised[b_idx], k, el)
        A0 = poly_add(par, A0, poly_mul(par, d, key[b_idx][0], el), el)
        A1 = poly_add(par, A1, poly_mul(par, d, key[b_idx][1], el), el)
    c0 = poly_add(par, poly_automorphism(par, ct[0], k, ql), mod_down(par, A0), ql)
    c1 = mod_down(par, A1)
    return np.stack([c0, c1])


def rotate_ext(par: Params, ct, raised, k: int, key) -> np.ndarray:
    """The rotation of rotate_hoisted before its ModDown, kept in the
    extended basis Q u P: (P sigma_k(c0) + A0, A1), [2][L+K][N].  P sigma_k(c0)
    is 0 modulo the special primes."""
    el = extlimbs(par)
    A0 = np.zeros((par.L + par.K, par.N), dtype=np.uint64)
    A1 = np.zeros_like(A0)
    for b_idx, _ in enumerate(par.digits):
        d = poly_automorphism(par, raised[b_idx], k, el)
        A0 = poly_add(par, A0, poly_mul(par, d, key[b_idx][0], el), el)
        A1 = poly_add(par, A1, poly_mul(par, d, key[b_idx][1], el), el)
    pc0 = times_P(par, poly_automorphism(par, ct[0], k, qlimbs(par)))
    return np.stack([poly_add(par, A0, pc0, el), A1])


def rotate_ext_lazy(par: Params, ct_ext, raised, k: int, key) -> np.ndarray:
    """Rotation of an extended-basis ciphertext (c0, c1) over Q u P whose c1
    was lowered for its key switch (raised = mod_up_all(mod_down(c1))) while
    c0 stays in Q u P: (sigma_k(c0) + A0, A1), [2][L+K][N].  Since
    c0 = P ModDown(c0) + r with |r| < K P, a later ModDown gives the rotation
    of the lowered ciphertext up to less than K + 1 per coefficient; for
    c0 = P x (special limbs 0) it is rotate_ext exactly."""
    el = extlimbs(par)
    A0 = np.zeros((par.L + par.K, par.N), dtype=np.uint64)
    A1 = np.zeros_like(A0)
    for b_idx, _ in enumerate(par.digits):
        d = poly_automorphism(par, raised[b_idx], k, el)
        A0 = poly_add(par, A0, poly_mul(par, d, key[b_idx][0], el), el)
        A1 = poly_add(par, A1, poly_mul(par, d, key[b_idx][1], el), el)
    return np.stack([poly_add(par, A0, poly_automorphism(par, ct_ext[0], k, el), el), A1])


def times_P(par: Params, x) -> np.ndarray:
    """P x over the extended basis for x over Q ([L][N] -> [L+K][N]); the
    special-prime limbs are 0."""
    out = np.zeros((par.L + par.K, par.N), dtype=np.uint64)
    for i, qi in enumerate(par.q):
        out[i] = ring.vec_scale(x[i], par.P % qi, qi)
    return out


def ct_times_P(par: Params, ct) -> np.ndarray:
    """A ciphertext over Q lifted to Q u P as (P c0, P c1)."""
    return np.stack([times_P(par, ct[0]), times_P(par, ct[1])])


def ct_mod_down(par: Params, ct_ext) -> np.ndarray:
    """ModDown of both polynomials of an extended-basis ciphertext."""
    return np.stack([mod_down(par, ct_ext[0]), mod_down(par, ct_ext[1])])


def rotate(par: Params, ct, k: int, key) -> np.ndarray:
    """Homomorphic automorphism sigma_k (Rot_row for k = 3^r, Rot_col for
    k = 2N-1), Sec. 5.1."""
    return rotate_hoisted(par, ct, mod_up_all(par, ct[1]), k, key)


# ---------------------------------------------------------- ring switching --

def embed_secret(sk_small, R: int) -> np.ndarray:
    """s'(X) = s_small(X^R): a secret of the subring as an element of the
    ring of dimension R N' (every R-th coefficient)."""
    s = np.asarray(sk_small, dtype=np.int64)
    out = np.zeros(s.size * R, dtype=np.int64)
    out[::R] = s
    return out


def ring_switch_key(par: Params, sk, sk_small, a, e) -> np.ndarray:
    """Hybrid key-switching key from s (par's ring) to s'(X) = s_small(X^R),
    R = N / N' (ring switching, Sec. 5.3, after Gentry-Halevi-Peikert-Smart):
      b_beta = -a_beta s' + e_beta + [q_i in digit beta] P s  over Q u P,
    the rotation key's equation with the target secret s' and the source
    s in place of sigma_k(s).  a: [digits][L+K][N], e: [digits][N];
    returns [digits][2][L+K][N] holding (b_beta, a_beta)."""
    el = extlimbs(par)
    R = par.N // len(sk_small)
    s_to = signed_to_rns(embed_secret(sk_small, R), par.ext)
    s_from = signed_to_rns(sk, par.ext)
    out = []
    for b_idx, digit in enumerate(par.digits):
        a_b = np.asarray(a[b_idx], dtype=np.uint64)
        e_b = signed_to_rns(e[b_idx], par.ext)
        b = poly_sub(par, e_b, poly_mul(par, a_b, s_to, el), el)
        for i in digit:
            qi = par.q[i]
            b[i] = ring.vec_add(b[i], ring.vec_scale(s_from[i], par.P % qi, qi), qi)
        out.append(np.stack([b, a_b.copy()]))
    return np.stack(out)


def ring_switch(par: Params, small: Params, ct, key) -> list[np.ndarray]:
    """Ring switching (Sec. 5.3) of a ciphertext of par's ring to R = N/N'
    ciphertexts of small's ring over the same primes.  The key switch to
    s'(X) = s_small(X^R) is the hybrid key switch of rotate() with the
    identity automorphism; then, with c0 + c1 s' = sum_r X^r
    (c0_r + c1_r s_small)(X^R) for c_p(X) = sum_r X^r c_{p,r}(X^R), part r
    = (c0[r::R], c1[r::R]) decrypts under s_small to m_r, where the
    plaintext is m(X) = sum_r X^r m_r(X^R) (noise split the same way).
    Returns R ciphertexts [2][L][N'] in coefficient form."""
    if (small.q, small.p, small.t) != (par.q, par.p, par.t) or par.N % small.N or small.N >= par.N:
        raise ValueError("ring_switch: small must be a subring with the same primes")
    R = par.N // small.N
    sw = rotate(par, ct, 1, key)
    return [np.ascontiguousarray(sw[:, :, r::R]) for r in range(R)]
