"""Oracle for the server-side hot path of the private database query (PDQ):
Mask followed by the SIMD-aware homomorphic compression Comp, plus the
client-side Decomp and the plaintext closed form that pins the result.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Paper anchors:
* Answer = Match -> Mask -> Comp, with the Match output v reused as the index
  vector (Alg. 7, Sec. 4.2.2).  Match depends on the query and is not given in
  the paper; the client's encrypted 0/1 index vector stands in for it.
* The compression matrix C[j][i] = i^j, j = 1..s (Eq. 1); Comp returns
  ctxt(Cv) and ctxt(Cd) (Alg. 5 and Alg. 7).
* SIMD form: u = [v; d] packed with row masks and Rot_col (Remark in
  Sec. 5.2), Pegasus-style diagonal matrix-vector product with baby-step /
  giant-step rotations on both rows at once, blocks summed before a single
  rotate-and-sum (Sec. 5.2).
* Decomp: Dec, Newton's identity (Lem. 1, Alg. 1 step 1), strip the factors
  of X and find the roots (Alg. 1 step 2), solve the Vandermonde system on
  the recovered columns (Alg. 4), scatter (Alg. 6).

Readings where the paper is silent (all mirrored by the GPU library):
* s' = 2^ceil(log2 s) rows of C (the diagonal method needs s' | N/2).
* The paper requires t > n (Eq. 1 remark).  Records are split into groups of
  G_sz = N*floor((t-1)/N) consecutive records; group gamma uses nodes
  alpha(i) = (i mod G_sz) + 1, and its (w, e) block sits in output ciphertext
  floor(gamma/(m/s')) at slot offset (gamma mod (m/s'))*s'.  With one group
  this is exactly the paper's C.
* The row masks of the u-packing remark are folded into the Mask plaintexts:
  (v.DB).[1;0] = v.(DB.[1;0]) (same slots, one multiplicative level less).
* Key switching is placed for speed without changing any slot: the baby-step
  rotations stay in the extended basis Q u P (no ModDown), the diagonal
  products are summed there and each accumulator is lowered once; the
  giant-step rotations of a group are summed in Q u P and lowered once.
* In the Answer (Mask then Comp) the pack's column rotation is applied to
  each index ciphertext before the Mask products (mask_pack): the same
  slots, half the pack's key switches.  Comp on its own packs the masked
  ciphertexts as Sec. 5.2 describes.
* Rotate-and-sum (sum of Rot(y; i s') over i < m/s', Sec. 5.2) runs in levels
  of radix r <= 8 instead of log2(m/s') doublings: each level sums
  Rot(y; j l), j < r, from one raise of y, in Q u P; the slots are the same.
* A ciphertext over Q u P that is only rotated next keeps c0 in Q u P: only
  c1 is lowered for the key switch (giant-step accumulators, giant-step
  sums, rotate-and-sum levels); the result is lowered once at the end.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import ring
from .bfv import (Params, ct_add, ct_mod_down, ct_times_P, decrypt, encode, encrypt, lift,
                  mod_down, mod_up_all, poly_add, pt_mul, ring_switch, rotate, rotate_ext,
                  rotate_ext_lazy)


# ------------------------------------------------------------------ plan ----

@dataclass(frozen=True)
class Plan:
    n: int          # records
    s: int          # sparsity bound
    s_prime: int    # padded compressed length per row
    B: int          # baby steps
    J: int          # index-vector ciphertexts
    H: int          # half-blocks (u ciphertexts) = 2J
    G_sz: int       # records per group
    hpg: int        # half-blocks per group
    G: int          # groups
    per_out: int    # groups per output ciphertext = m / s'
    n_out: int      # output ciphertexts

    @property
    def giants(self) -> int:
        return self.s_prime // self.B


def make_plan(par: Params, n: int, s: int, B: int | None = None) -> Plan:
    if n < 1 or s < 1:
        raise ValueError("n and s must be positive")
    s_prime = 1 << math.ceil(math.log2(s))
    if s_prime > par.m or s_prime >= par.t:
        raise ValueError("sparsity too large for the ring")
    J = -(-n // par.N)
    H = 2 * J
    G_sz = par.N * ((par.t - 1) // par.N)
    hpg = G_sz // par.m
    G = -(-H // hpg)
    B = _baby_steps(H, G, s_prime) if B is None else B
    if B < 1 or s_prime % B:
        raise ValueError("B must divide s'")
    per_out = par.m // s_prime
    n_out = -(-G // per_out)
    return Plan(n, s, s_prime, B, J, H, G_sz, hpg, G, per_out, n_out)


def _baby_steps(H: int, G: int, s_prime: int) -> int:
    """Baby/giant split (the paper leaves it open): among the powers of two
    B <= min(s', 128) with at most 32 giant steps, the one with the least work
    H(B-1) + 8 G(s'/B - 1) + 3 G s'/B (hoisted baby rotations, giant-step key
    switches, accumulator ModDowns); ties to the smaller B."""
    costs = {}
    b = 1
    while b <= min(s_prime, 128):
        if s_prime // b <= 32:
            costs[b] = H * (b - 1) + 8 * G * (s_prime // b - 1) + 3 * G * (s_prime // b)
        b *= 2
    return min(costs, key=lambda k: (costs[k], k))


def make_switched_plan(big: Params, small: Params, n: int, s: int, B: int | None = None) -> Plan:
    """Plan of Comp in the subring on a ring-switched query (Sec. 5.3): each
    of the ceil(n/N) ciphertexts of the big ring becomes R = N/N' ciphertexts
    of the small ring (part r of big ciphertext j at index R j + r, 2R
    half-blocks), and the records keep the groups of the big ring (G_sz =
    N floor((t-1)/N) records, nodes alpha(i) = (i mod G_sz) + 1), so
    hpg = G_sz / m' small half-blocks per group."""
    if n < 1 or s < 1:
        raise ValueError("n and s must be positive")
    R = big.N // small.N
    s_prime = 1 << math.ceil(math.log2(s))
    if s_prime > small.m or s_prime >= small.t:
        raise ValueError("sparsity too large for the ring")
    J = R * -(-n // big.N)
    H = 2 * J
    G_sz = big.N * ((big.t - 1) // big.N)
    hpg = G_sz // small.m
    G = -(-H // hpg)
    B = _baby_steps(H, G, s_prime) if B is None else B
    if B < 1 or s_prime % B:
        raise ValueError("B must divide s'")
    per_out = small.m // s_prime
    return Plan(n, s, s_prime, B, J, H, G_sz, hpg, G, per_out, -(-G // per_out))


def rotsum_levels(par: Params, plan: Plan) -> list[tuple[int, int]]:
    """Levels (l, r) of the rotate-and-sum: level i sums Rot(.; j l) for
    j < r, l the product of s' and the earlier radices.  The log2(m/s') bits
    are split into ceil(bits/3) chunks as evenly as possible, larger first,
    so every radix is at most 8."""
    bits = int(math.log2(par.m // plan.s_prime))
    if bits == 0:
        return []
    nlev = -(-bits // 3)
    base, extra = divmod(bits, nlev)
    levels, l = [], plan.s_prime
    for i in range(nlev):
        r = 1 << (base + (1 if i < extra else 0))
        levels.append((l, r))
        l *= r
    return levels


def galois_elements(par: Params, plan: Plan) -> list[int]:
    """Every automorphism the schedule uses, ascending."""
    ks = {par.galois_col}
    ks.update(par.galois_rot(a) for a in range(1, plan.B))
    ks.update(par.galois_rot(g * plan.B) for g in range(1, plan.giants))
    for l, r in rotsum_levels(par, plan):
        ks.update(par.galois_rot(j * l) for j in range(1, r))
    return sorted(ks)


# ---------------------------------------------------------------- layout ----

def record_slots(par: Params, values, j: int) -> np.ndarray:
    """Slots of ciphertext j: record i = j*N + rho*m + c sits at row rho,
    column c (slot index rho*m + c); records past the end are 0."""
    out = np.zeros(par.N, dtype=np.uint64)
    chunk = np.asarray(values[j * par.N:(j + 1) * par.N], dtype=np.uint64)
    out[:chunk.size] = chunk
    return out


def encrypt_index(par: Params, sk, v, plan: Plan, a, e) -> list[np.ndarray]:
    """Query: the client encrypts its 0/1 index vector, N records per
    ciphertext.  a: [J][L][N], e: [J][N] supplied randomness."""
    return [encrypt(par, sk, encode(par, record_slots(par, v, j)), a[j], e[j])
            for j in range(plan.J)]


def row_mask_slots(par: Params, rho: int) -> np.ndarray:
    s = np.zeros(par.N, dtype=np.uint64)
    s[rho * par.m:(rho + 1) * par.m] = 1
    return s


def lifted_pt(par: Params, slots) -> np.ndarray:
    return lift(par, encode(par, slots), par.q)


# ------------------------------------------------------------------ Mask ----

def mask(par: Params, v_cts, db, plan: Plan) -> list[np.ndarray]:
    """Mask with the row split folded in (4 ciphertexts per index ciphertext):
    vT = v.[1;0], vB = v.[0;1], dT = v.(DB.[1;0]), dB = v.(DB.[0;1])."""
    top = row_mask_slots(par, 0)
    bot = row_mask_slots(par, 1)
    pt_top, pt_bot = lifted_pt(par, top), lifted_pt(par, bot)
    out = []
    for j in range(plan.J):
        dbs = record_slots(par, db, j)
        out.append(pt_mul(par, v_cts[j], pt_top))
        out.append(pt_mul(par, v_cts[j], pt_bot))
        out.append(pt_mul(par, v_cts[j], lifted_pt(par, dbs * top)))
        out.append(pt_mul(par, v_cts[j], lifted_pt(par, dbs * bot)))
    return out


def mask_literal(par: Params, v_cts, db, plan: Plan) -> list[np.ndarray]:
    """Mask as the u-packing remark writes it (Sec. 5.2, remark (ii)): the
    masked database d = v . DB first, then the row masks on v and on d:
    vT = v.[1;0], vB = v.[0;1], dT = d.[1;0], dB = d.[0;1] -- one plaintext
    product more on d than mask(), the same slots."""
    pt_top = lifted_pt(par, row_mask_slots(par, 0))
    pt_bot = lifted_pt(par, row_mask_slots(par, 1))
    out = []
    for j in range(plan.J):
        d = pt_mul(par, v_cts[j], lifted_pt(par, record_slots(par, db, j)))
        out.append(pt_mul(par, v_cts[j], pt_top))
        out.append(pt_mul(par, v_cts[j], pt_bot))
        out.append(pt_mul(par, d, pt_top))
        out.append(pt_mul(par, d, pt_bot))
    return out


# ------------------------------------------------------------------ Comp ----

def pack(par: Params, masked, keys, plan: Plan) -> list[np.ndarray]:
    """u_{2j} = vT_j + Rot_col(dT_j), u_{2j+1} = Rot_col(vB_j) + dB_j, so that
    u_h = [v_h; d_h] for half-block h (u-packing remark, Sec. 5.2)."""
    kc = par.galois_col
    u = []
    for j in range(plan.J):
        vT, vB, dT, dB = masked[4 * j:4 * j + 4]
        u.append(ct_add(par, vT, rotate(par, dT, kc, keys[kc])))
        u.append(ct_add(par, rotate(par, vB, kc, keys[kc]), dB))
    return u


def swap_rows(par: Params, slots) -> np.ndarray:
    """The slot permutation of Rot_col: the two rows exchanged (Sec. 5.1)."""
    return np.asarray(slots).reshape(2, par.m)[::-1].reshape(-1)


def mask_pack(par: Params, v_cts, db, keys, plan: Plan) -> list[np.ndarray]:
    """Mask followed by the pack of Comp, with the column rotation moved in
    front of the Mask products.  Rot_col is a ring automorphism, so
    Rot_col(v . P) = Rot_col(v) . sigma_col(P) and, with w_j = Rot_col(v_j),
      u_{2j}   = v_j . [1;0] + w_j . sigma_col(DB_j . [1;0])
      u_{2j+1} = w_j . [1;0] + v_j . (DB_j . [0;1])
    hold the same slots as pack(mask(v)): one key switch per index
    ciphertext instead of two.  sigma_col of an encoded plaintext is the
    encoding of its row-swapped slots (t odd, so the centred lift commutes)."""
    kc = par.galois_col
    top, bot = row_mask_slots(par, 0), row_mask_slots(par, 1)
    pt_top = lifted_pt(par, top)
    u = []
    for j in range(plan.J):
        dbs = record_slots(par, db, j)
        w = rotate(par, v_cts[j], kc, keys[kc])
        u.append(ct_add(par, pt_mul(par, v_cts[j], pt_top),
                        pt_mul(par, w, lifted_pt(par, swap_rows(par, dbs * top)))))
        u.append(ct_add(par, pt_mul(par, w, pt_top),
                        pt_mul(par, v_cts[j], lifted_pt(par, dbs * bot))))
    return u


def node_row(par: Params, plan: Plan, h: int) -> np.ndarray:
    """alpha(i) = (i mod G_sz) + 1 for the m records i = h*m + x of half-block h."""
    x = np.arange(par.m, dtype=np.int64)
    return ((h * par.m + x) % plan.G_sz + 1).astype(np.uint64)


def powmod_vec(base: np.ndarray, exp: np.ndarray, t: int) -> np.ndarray:
    """Element-wise base^exp mod t (t < 2^31), square and multiply."""
    r = np.ones_like(base, dtype=np.uint64)
    b = base.astype(np.uint64) % np.uint64(t)
    e = exp.astype(np.int64).copy()
    while (e > 0).any():
        odd = (e & 1) == 1
        r = np.where(odd, r * b % np.uint64(t), r)
        b = b * b % np.uint64(t)
        e >>= 1
    return r


def diagonal_slots(par: Params, plan: Plan, h: int, k: int) -> np.ndarray:
    """k-th extended diagonal of the block of C acting on half-block h, the
    same on both rows (C "encoded twice", Sec. 5.2):
      D_{h,k}[c] = alpha(h*m + ((c + k) mod m))^{(c mod s') + 1}  mod t."""
    m = par.m
    c = np.arange(m)
    nodes = node_row(par, plan, h)[(c + k) % m]
    row = powmod_vec(nodes, (c % plan.s_prime) + 1, par.t)
    return np.concatenate([row, row])


def switched_nodes(big: Params, small: Params, plan: Plan, h: int):
    """The records behind half-block h = 2(R j + r) + rho' of a ring-switched
    query (part r of big ciphertext j, row rho'): small slot (rho', c') with
    exponent e' = (-1)^rho' 3^c' mod 2N' holds
      y_r(e') = m_r(zeta'^e') = (1/R) sum_u zeta^(-e_u r) m(zeta^(e_u)),
    e_u = e' + 2N' u (u < R), zeta' = zeta^R, because m(X) = sum_r X^r
    m_r(X^R); so the big slots are m(zeta^(e_u)) = sum_r zeta^(e_u r) y_r(e').
    Returns, per column c' < m' and u < R, the node alpha of the record in
    big slot e_u of ciphertext j and the factor zeta^(e_u r) mod t."""
    R = big.N // small.N
    i, rho = divmod(h, 2)
    j, r = divmod(i, R)
    e_small = small.slot_exponents()[rho * small.m:(rho + 1) * small.m].astype(np.int64)
    e_big = e_small[:, None] + 2 * small.N * np.arange(R, dtype=np.int64)[None, :]
    slot_of = np.empty(2 * big.N, dtype=np.int64)
    slot_of[big.slot_exponents()] = np.arange(big.N)
    rec = j * big.N + slot_of[e_big]
    alpha = (rec % plan.G_sz + 1).astype(np.uint64)
    factor = powmod_vec(np.full(e_big.shape, big.zeta, dtype=np.uint64),
                        (e_big * r) % (2 * big.N), big.t)
    return alpha, factor


def switched_diagonal_slots(big: Params, small: Params, plan: Plan, h: int, k: int) -> np.ndarray:
    """k-th extended diagonal for half-block h of a ring-switched query.
    With the fold of switched_nodes, sum over the records of
    alpha^kk v = sum over (r, e') of y_r(e') W_kk[r][e'],
    W_kk[r][e'] = sum_u alpha(e_u)^kk zeta^(e_u r): the block of half-block h
    is M[kk][c'] = W_{kk+1}[r][e'(rho', c')] and, as in diagonal_slots,
    D_{h,k}[c] = M[c mod s'][(c + k) mod m'] on both rows."""
    m, t = small.m, small.t
    alpha, factor = switched_nodes(big, small, plan, h)
    c = np.arange(m)
    cc = (c + k) % m
    kk = (c % plan.s_prime) + 1
    row = np.zeros(m, dtype=np.uint64)
    for u in range(alpha.shape[1]):
        row = (row + powmod_vec(alpha[cc, u], kk, t) * factor[cc, u]) % np.uint64(t)
    return np.concatenate([row, row])


def rot_slots(par: Params, slots, r: int) -> np.ndarray:
    """Rot(.; r) on both rows: [v_1..v_m] -> [v_{1+r}, ..., v_r] (Sec. 5.1)."""
    s = np.asarray(slots).reshape(2, par.m)
    return np.roll(s, -r, axis=1).reshape(-1)


def ring_dot(par: Params, pts, cts) -> np.ndarray:
    """sum_i pts[i] * cts[i] in R_Q (plaintext-ciphertext products, summed).
    Each product is a negacyclic product limb by limb; it is computed through
    the oracle's transform as INTT(sum_i NTT(pt_i) .* NTT(ct_i)), which equals
    the sum of the individual products because the transform is linear."""
    L, N = par.L, par.N
    acc = np.zeros((2, L, N), dtype=np.uint64)
    for pt, ct in zip(pts, cts):
        for i in range(L):
            q, psi = par.q[i], par.psi[i]
            fp = ring.ntt_forward(pt[i], q, psi)
            for p in range(2):
                fc = ring.ntt_forward(ct[p][i], q, psi)
                acc[p][i] = ring.vec_add(acc[p][i], ring.vec_mul(fp, fc, q), q)
    for p in range(2):
        for i in range(L):
            acc[p][i] = ring.ntt_inverse(acc[p][i], par.q[i], par.psi[i])
    return acc


def group_halfblocks(plan: Plan, gamma: int) -> range:
    return range(gamma * plan.hpg, min((gamma + 1) * plan.hpg, plan.H))


def baby_steps(par: Params, u, keys, plan: Plan):
    """R[h][a] = Rot_row(u_h; a) for a = 0..B-1, kept in the extended basis
    Q u P before its ModDown (a = 0: (P c0, P c1)); the digits of c1 are
    raised once per u_h and shared by all its rotations."""
    R = []
    for uh in u:
        raised = mod_up_all(par, uh[1])
        row = [ct_times_P(par, uh)]
        for a in range(1, plan.B):
            k = par.galois_rot(a)
            row.append(rotate_ext(par, uh, raised, k, keys[k]))
        R.append(row)
    return R


def ring_dot_ext(par: Params, pts, cts) -> np.ndarray:
    """ring_dot over the extended basis: sum_i pts[i] * cts[i] in R_{QP}
    (pts [L+K][N], cts [2][L+K][N]), through the oracle's transform."""
    E, N = par.L + par.K, par.N
    acc = np.zeros((2, E, N), dtype=np.uint64)
    for pt, ct in zip(pts, cts):
        for i in range(E):
            q, psi = par.ext[i], par.psi[i]
            fp = ring.ntt_forward(pt[i], q, psi)
            for p in range(2):
                fc = ring.ntt_forward(ct[p][i], q, psi)
                acc[p][i] = ring.vec_add(acc[p][i], ring.vec_mul(fp, fc, q), q)
    for p in range(2):
        for i in range(E):
            acc[p][i] = ring.ntt_inverse(acc[p][i], par.ext[i], par.psi[i])
    return acc


def giant_accumulators(par: Params, R, plan: Plan, diag=None):
    """acc[gamma][g] = sum_{h in gamma} sum_{a<B} Rot(D_{h,gB+a}; -gB) . R[h][a],
    the products summed over Q u P (diagonals lifted to every prime); the
    accumulators stay in Q u P (giant_steps lowers the ones it rotates).
    diag(par, plan, h, k) gives D_{h,k} (default: diagonal_slots)."""
    diag = diag or diagonal_slots
    acc = []
    for gamma in range(plan.G):
        row = []
        for g in range(plan.giants):
            pts, cts = [], []
            for h in group_halfblocks(plan, gamma):
                for a in range(plan.B):
                    d = rot_slots(par, diag(par, plan, h, g * plan.B + a), -g * plan.B)
                    pts.append(lift(par, encode(par, d), par.ext))
                    cts.append(R[h][a])
            row.append(ring_dot_ext(par, pts, cts))
        acc.append(row)
    return acc


def giant_steps(par: Params, acc, keys, plan: Plan):
    """y_gamma = acc[gamma][0] + sum_{g>=1} Rot(acc[gamma][g]; gB) over Q u P:
    the unrotated accumulator joins the sum as it is; of the others only c1 is
    lowered to Q (for its key switch), c0 enters the rotation from Q u P
    (rotate_ext_lazy).  The sums stay in Q u P for the rotate-and-sum."""
    el = list(range(par.L + par.K))
    ys = []
    for gamma in range(plan.G):
        y = acc[gamma][0]
        for g in range(1, plan.giants):
            k = par.galois_rot(g * plan.B)
            raised = mod_up_all(par, mod_down(par, acc[gamma][g][1]))
            r = rotate_ext_lazy(par, acc[gamma][g], raised, k, keys[k])
            y = np.stack([poly_add(par, y[0], r[0], el), poly_add(par, y[1], r[1], el)])
        ys.append(y)
    return ys


def rotate_and_sum(par: Params, y, keys, plan: Plan):
    """sum_{i < m/s'} Rot(y; i s') (once, after the blocks were summed,
    Sec. 5.2) for y over Q u P, level by level: y <- sum_{j<r} Rot(y; j l)
    with the rotations hoisted (one raise of the lowered c1) and kept in
    Q u P (j = 0: y itself; c0 enters each rotation from Q u P), lowered to Q
    after the last level.  The levels multiply out to every i < m/s' exactly
    once."""
    el = list(range(par.L + par.K))
    for l, r in rotsum_levels(par, plan):
        raised = mod_up_all(par, mod_down(par, y[1]))
        acc = y
        for j in range(1, r):
            k = par.galois_rot(j * l)
            rj = rotate_ext_lazy(par, y, raised, k, keys[k])
            acc = np.stack([poly_add(par, acc[0], rj[0], el), poly_add(par, acc[1], rj[1], el)])
        y = acc
    return ct_mod_down(par, y)


def group_mask_slots(par: Params, plan: Plan, o: int) -> np.ndarray:
    s = np.zeros(par.N, dtype=np.uint64)
    for rho in range(2):
        s[rho * par.m + o * plan.s_prime: rho * par.m + (o + 1) * plan.s_prime] = 1
    return s


def combine_groups(par: Params, ys, plan: Plan):
    """One group: the result as is (its block repeats every s' slots).
    Several groups: Out_c = sum_{gamma in c} M_{gamma mod (m/s')} . y_gamma."""
    if plan.G == 1:
        return [ys[0]]
    outs = []
    for c in range(plan.n_out):
        gs = range(c * plan.per_out, min((c + 1) * plan.per_out, plan.G))
        pts = [lifted_pt(par, group_mask_slots(par, plan, g - c * plan.per_out)) for g in gs]
        outs.append(ring_dot(par, pts, [ys[g] for g in gs]))
    return outs


def comp_packed(par: Params, u, keys, plan: Plan, diag=None) -> list[np.ndarray]:
    """Comp from the packed u_h on: baby steps, diagonal products, giant
    steps, rotate-and-sum, group masks."""
    R = baby_steps(par, u, keys, plan)
    acc = giant_accumulators(par, R, plan, diag)
    ys = giant_steps(par, acc, keys, plan)
    ys = [rotate_and_sum(par, y, keys, plan) for y in ys]
    return combine_groups(par, ys, plan)


def comp(par: Params, masked, keys, plan: Plan, diag=None) -> list[np.ndarray]:
    """Comp of Alg. 7 in SIMD form: returns the output ciphertexts holding
    ctxt(Cv) in row 0 and ctxt(Cd) in row 1."""
    return comp_packed(par, pack(par, masked, keys, plan), keys, plan, diag)


def answer(par: Params, v_cts, db, keys, plan: Plan) -> list[np.ndarray]:
    """Server side of the query: Mask then Comp (Alg. 7 without Match), with
    the pack's column rotation applied to v before the Mask products
    (mask_pack): the same slots as comp(mask(v)), one key switch per index
    ciphertext fewer."""
    return comp_packed(par, mask_pack(par, v_cts, db, keys, plan), keys, plan)


def answer_switched(par: Params, low: Params, v_cts, db, keys, plan: Plan) -> list[np.ndarray]:
    """The Answer with Comp on smaller parameters (Sec. 6): the index
    ciphertexts are switched from par's modulus to low's (mod_switch), then
    Mask and Comp run over low's primes with low's keys (plan made for low)."""
    from .bfv import mod_switch
    return answer(low, [mod_switch(par, low, v) for v in v_cts], db, keys, plan)


def ring_switch_masked(big: Params, small: Params, masked, rs_key) -> list[np.ndarray]:
    """The Mask outputs of the big ring (4 per index ciphertext, mask())
    switched to the subring: part r of masked[4j + q] becomes small
    ciphertext 4(R j + r) + q.  A small slot of row rho' folds only big slots
    of row rho' (their exponents agree mod 8), so the row masks survive."""
    R = big.N // small.N
    out = [None] * (len(masked) * R)
    for i, ct in enumerate(masked):
        j, q = divmod(i, 4)
        for r, part in enumerate(ring_switch(big, small, ct, rs_key)):
            out[4 * (R * j + r) + q] = part
    return out


def answer_ring_switched(big: Params, small: Params, v_cts, db, rs_key, keys,
                         plan: Plan) -> list[np.ndarray]:
    """The Answer with Comp in a subring (Sec. 5.3: ring switching after Mask,
    Comp with the smaller parameters): Mask in the big ring (mask()), every
    masked ciphertext switched to R ciphertexts of small's ring
    (ring_switch_masked), then Comp there (pack, baby steps, the diagonals of
    switched_diagonal_slots, giant steps, rotate-and-sum, group masks) with
    small-ring rotation keys.  plan from make_switched_plan.  The output
    decrypts under s_small to the same closed form as answer()."""
    R = big.N // small.N
    big_plan = Plan(plan.n, plan.s, plan.s_prime, plan.B, plan.J // R, plan.H // R, plan.G_sz,
                    plan.hpg, plan.G, plan.per_out, plan.n_out)
    masked = ring_switch_masked(big, small, mask(big, v_cts, db, big_plan), rs_key)
    return comp(small, masked, keys, plan,
                lambda par, pl, h, k: switched_diagonal_slots(big, par, pl, h, k))


# --------------------------------------------------- unencrypted database ---
#
# When the database is known in the clear, C (DB . v) = (C diag(DB)) v, so the
# server can skip Mask and compress v alone with the stacked matrix
# [C; C diag(DB)] (Sec. 5.2, remark on an unencrypted database).  Here index
# ciphertext j holds half-block 2j in row 0 and 2j+1 in row 1, and two sets of
# diagonals put C on one row and C diag(DB) on the other:
#   set 0: row 0 = C on half-block 2j,        row 1 = C diag(DB) on 2j+1
#   set 1: row 0 = C diag(DB) on half-block 2j, row 1 = C on 2j+1
# so after the BSGS products, giant steps and rotate-and-sum set 0 holds
# (C v_2j, C d_2j+1) and set 1 (C d_2j, C v_2j+1), and set 0 + Rot_col(set 1)
# = (C v, C d).  Rot_col commutes with the row rotations, so it is folded into
# the giant steps of set 1 (Galois element 3^(gB) (2N - 1), also for g = 0).

def make_plan_plain_db(par: Params, n: int, s: int, B: int | None = None) -> Plan:
    """Plan of the Answer on an unencrypted database: the layout of make_plan;
    by default B is the power of two B <= min(s', 128) with at most 32 giant
    steps that minimises J(B-1) + 8 G(2 s'/B - 1) + 6 G s'/B (hoisted baby
    rotations of the J index ciphertexts, giant-step key switches of both
    sets, accumulator ModDowns), ties to the smaller B."""
    if B is None:
        lay = make_plan(par, n, s, 1 << math.ceil(math.log2(s)))
        costs = {}
        b = 1
        while b <= min(lay.s_prime, 128):
            gi = lay.s_prime // b
            if gi <= 32:
                costs[b] = lay.J * (b - 1) + 8 * lay.G * (2 * gi - 1) + 6 * lay.G * gi
            b *= 2
        B = min(costs, key=lambda k: (costs[k], k))
    return make_plan(par, n, s, B)


def plain_db_diagonal_slots(par: Params, plan: Plan, db, j: int, sigma: int, k: int) -> np.ndarray:
    """k-th extended diagonal of set sigma for index ciphertext j: row rho is
    the diagonal of half-block h = 2j + rho (diagonal_slots), times the
    database records it meets on the row rho != sigma (row 1 for set 0, row 0
    for set 1):
      D[rho][c] = alpha(h m + c')^((c mod s')+1) (DB[h m + c'] if rho != sigma),
    c' = (c + k) mod m."""
    m, t = par.m, par.t
    c = np.arange(m)
    cc = (c + k) % m
    rows = []
    for rho in range(2):
        h = 2 * j + rho
        row = diagonal_slots(par, plan, h, k)[:m]
        if rho != sigma:
            dbh = np.zeros(m, dtype=np.uint64)
            chunk = np.asarray(db[h * m:(h + 1) * m], dtype=np.uint64) % np.uint64(t)
            dbh[:chunk.size] = chunk
            row = row * dbh[cc] % np.uint64(t)
        rows.append(row)
    return np.concatenate(rows)


def plain_db_galois_elements(par: Params, plan: Plan) -> list[int]:
    """Every automorphism of the unencrypted-database Answer, ascending."""
    col = par.galois_col
    ks = {col}
    ks.update(par.galois_rot(a) for a in range(1, plan.B))
    ks.update(par.galois_rot(g * plan.B) for g in range(1, plan.giants))
    ks.update(par.galois_rot(g * plan.B) * col % (2 * par.N) for g in range(1, plan.giants))
    for l, r in rotsum_levels(par, plan):
        ks.update(par.galois_rot(jj * l) for jj in range(1, r))
    return sorted(ks)


def answer_plain_db(par: Params, v_cts, db, keys, plan: Plan) -> list[np.ndarray]:
    """The Answer on an unencrypted database (no Mask): baby steps of the J
    index ciphertexts (baby_steps), per group gamma, set sigma and giant step g
      acc[sigma][g] = sum_{j in gamma} sum_{a<B} Rot(D^sigma_{j,gB+a}; -gB) . R[j][a]
    over Q u P, then y = sum_g Rot(acc[0][g]; gB) + sum_g Rot_col(Rot(acc[1][g]; gB))
    (acc[0][0] as it is; the others rotated from their lowered c1 as in
    giant_steps, set 1 with Galois element 3^(gB) (2N - 1)), rotate-and-sum,
    group masks.  Decrypts to the closed form of answer()."""
    el = list(range(par.L + par.K))
    R = baby_steps(par, v_cts, keys, plan)
    jpg = plan.hpg // 2                      # index ciphertexts per group
    col = par.galois_col
    ys = []
    for gamma in range(plan.G):
        js = range(gamma * jpg, min((gamma + 1) * jpg, plan.J))
        y = None
        for sigma in range(2):
            for g in range(plan.giants):
                pts, cts = [], []
                for j in js:
                    for a in range(plan.B):
                        d = rot_slots(par, plain_db_diagonal_slots(par, plan, db, j, sigma,
                                                                   g * plan.B + a), -g * plan.B)
                        pts.append(lift(par, encode(par, d), par.ext))
                        cts.append(R[j][a])
                acc = ring_dot_ext(par, pts, cts)
                if sigma == 0 and g == 0:
                    term = acc
                else:
                    k = par.galois_rot(g * plan.B) * (col if sigma else 1) % (2 * par.N)
                    raised = mod_up_all(par, mod_down(par, acc[1]))
                    term = rotate_ext_lazy(par, acc, raised, k, keys[k])
                y = term if y is None else np.stack(
                    [poly_add(par, y[0], term[0], el), poly_add(par, y[1], term[1], el)])
        ys.append(rotate_and_sum(par, y, keys, plan))
    return combine_groups(par, ys, plan)


# ------------------------------------------------------- closed form ------

def closed_form(par: Params, plan: Plan, v, db):
    """The plaintext result: per group gamma, for k = 1..s'
      w_k = sum_{i in gamma} alpha(i)^k v_i,   e_k = sum_{i in gamma} alpha(i)^k v_i DB_i  (mod t)
    i.e. C v and C d with d = v.DB (Eq. 1, Alg. 7).  Returns [G][2][s']."""
    t = np.uint64(par.t)
    v = np.asarray(v, dtype=np.uint64)
    d = v * np.asarray(db, dtype=np.uint64) % t
    out = np.zeros((plan.G, 2, plan.s_prime), dtype=np.uint64)
    n = v.size
    for gamma in range(plan.G):
        lo = gamma * plan.G_sz
        hi = min(lo + plan.G_sz, n)
        if lo >= hi:
            continue
        alpha = (np.arange(lo, hi, dtype=np.int64) % plan.G_sz + 1).astype(np.uint64)
        pw = np.ones_like(alpha)
        vv, dd = v[lo:hi], d[lo:hi]
        for k in range(plan.s_prime):
            pw = pw * alpha % t
            out[gamma, 0, k] = int((pw * vv % t).sum() % t)
            out[gamma, 1, k] = int((pw * dd % t).sum() % t)
    return out


def expected_slots(par: Params, plan: Plan, v, db) -> list[np.ndarray]:
    """Decrypted slots every output ciphertext must hold."""
    blocks = closed_form(par, plan, v, db)
    outs = []
    for c in range(plan.n_out):
        s = np.zeros(par.N, dtype=np.uint64)
        if plan.G == 1:
            for o in range(plan.per_out):
                for rho in range(2):
                    base = rho * par.m + o * plan.s_prime
                    s[base:base + plan.s_prime] = blocks[0, rho]
        else:
            for gamma in range(c * plan.per_out, min((c + 1) * plan.per_out, plan.G)):
                o = gamma - c * plan.per_out
                for rho in range(2):
                    base = rho * par.m + o * plan.s_prime
                    s[base:base + plan.s_prime] = blocks[gamma, rho]
        outs.append(s)
    return outs


# ---------------------------------------------------------------- Decomp ----

class DecodeError(Exception):
    pass


def newton_coefficients(w, t: int) -> list[int]:
    """Alg. 1 step 1: a_0 = 1, a_k = k^{-1} sum_{i=1}^{k} (-1)^{i-1} a_{k-i} w_i
    (mod t), from the power sums w_1..w_s (Lem. 1)."""
    s = len(w)
    a = [1]
    for k in range(1, s + 1):
        acc = 0
        for i in range(1, k + 1):
            term = a[k - i] * int(w[i - 1])
            acc += term if i % 2 == 1 else -term
        a.append(acc * pow(k, -1, t) % t)
    return a


def f_from_coefficients(a, t: int) -> list[int]:
    """f(X) = sum_{k=0}^{s} (-1)^k a_k X^{s-k}; returned lowest degree first."""
    s = len(a) - 1
    f = [0] * (s + 1)
    for k in range(s + 1):
        f[s - k] = (a[k] if k % 2 == 0 else -a[k]) % t
    return f


def strip_x(f) -> list[int]:
    """Divide by X while X divides f (Alg. 1 step 2)."""
    i = 0
    while i < len(f) - 1 and f[i] == 0:
        i += 1
    return list(f[i:])


def roots_bruteforce(g, lo: int, hi: int, t: int) -> list[int]:
    """All x in [lo, hi] with g(x) = 0 mod t, by evaluating g everywhere."""
    x = np.arange(lo, hi + 1, dtype=np.uint64)
    acc = np.zeros_like(x)
    tt = np.uint64(t)
    for c in reversed(g):
        acc = (acc * x + np.uint64(c)) % tt
    return [int(r) for r in x[acc == 0]]


def solve_mod(A, b, t: int):
    """Gaussian elimination mod t for a square nonsingular system."""
    n = len(A)
    M = [[int(A[i][j]) % t for j in range(n)] + [int(b[i]) % t] for i in range(n)]
    for col in range(n):
        piv = next((r for r in range(col, n) if M[r][col]), None)
        if piv is None:
            raise DecodeError("singular system")
        M[col], M[piv] = M[piv], M[col]
        inv = pow(M[col][col], -1, t)
        M[col] = [x * inv % t for x in M[col]]
        for r in range(n):
            if r != col and M[r][col]:
                f = M[r][col]
                M[r] = [(x - f * y) % t for x, y in zip(M[r], M[col])]
    return [M[i][n] for i in range(n)]


def reconst_idx(w, t: int, max_node: int) -> list[int]:
    """Alg. 1: the nodes whose power sums are w."""
    g = strip_x(f_from_coefficients(newton_coefficients(w, t), t))
    deg = len(g) - 1
    if deg == 0:
        return []
    roots = roots_bruteforce(g, 1, max_node, t)
    if len(roots) != deg:
        raise DecodeError(f"found {len(roots)} roots for degree {deg}")
    return roots


def reconst(e, nodes, t: int) -> list[int]:
    """Alg. 4: solve C_hat x = e on the recovered columns (rows 1..l square,
    the remaining rows must agree)."""
    l = len(nodes)
    if l == 0:
        if any(int(x) % t for x in e):
            raise DecodeError("nonzero values without indices")
        return []
    A = [[pow(a, j + 1, t) for a in nodes] for j in range(l)]
    x = solve_mod(A, [int(v) for v in e[:l]], t)
    for j in range(l, len(e)):
        if sum(pow(a, j + 1, t) * xi for a, xi in zip(nodes, x)) % t != int(e[j]) % t:
            raise DecodeError("inconsistent compressed values")
    return x


def decomp_slots(par: Params, plan: Plan, out_slots) -> list[tuple[int, int]]:
    """Alg. 6 on decrypted output slots: sorted (record index, value) pairs."""
    res = []
    for gamma in range(plan.G):
        c, o = divmod(gamma, plan.per_out) if plan.G > 1 else (0, 0)
        s = out_slots[c]
        w = s[o * plan.s_prime:(o + 1) * plan.s_prime]
        e = s[par.m + o * plan.s_prime: par.m + (o + 1) * plan.s_prime]
        nodes = reconst_idx(w, par.t, plan.G_sz)
        vals = reconst(e, nodes, par.t)
        res.extend((gamma * plan.G_sz + a - 1, int(x)) for a, x in zip(nodes, vals))
    return sorted(res)


def decomp(par: Params, sk, plan: Plan, outs) -> list[tuple[int, int]]:
    """Client-side Recover: decrypt the answer, then decompress."""
    return decomp_slots(par, plan, [decrypt(par, sk, ct) for ct in outs])
