"""Pins for the oracle's Mask / Comp / Decomp (no GPU).

The Comp ciphertext is not unique, so its slots are pinned: they must decrypt
to C v and C d computed straight from Eq. 1 with Python integers.  The
diagonal (Pegasus) algebra is pinned in the clear against an explicit matrix
product, Newton's identity against brute-force elementary symmetric
polynomials, and Decomp by exhaustive enumeration on tiny inputs."""
import itertools
import pathlib
import random

import numpy as np
import pytest

import workloads as W
from oracle import bfv, pdq


def build(cfg_name, seed=None):
    cfg = W.CONFIGS[cfg_name]
    par = bfv.Params.from_config(cfg)
    qi = W.draw_query(cfg, seed)
    plan = pdq.make_plan(par, cfg.n, cfg.s)
    ks = pdq.galois_elements(par, plan)
    kr = W.rotation_key_randomness(par.ext, par.N, len(par.digits), ks, cfg.seed)
    keys = {k: bfv.rotation_key(par, qi.sk, k, *kr[k]) for k in ks}
    a, e = W.encryption_randomness(par.q, par.N, plan.J, cfg.seed)
    v_cts = pdq.encrypt_index(par, qi.sk, qi.v, plan, a, e)
    return cfg, par, qi, plan, keys, v_cts


def matrix_C(s_prime, nodes, t):
    """Eq. 1: C[j][i] = nodes[i]^(j+1) mod t."""
    return [[pow(int(a), j + 1, t) for a in nodes] for j in range(s_prime)]


def test_plan_shapes_match_cost_model():
    # (config) -> (s', B, J, half-blocks, groups, outputs, #galois); B by hand
    # from the split cost H(B-1) + 8G(s'/B-1) + 3Gs'/B:
    #   c1 (H=2, G=1, s'=16): B=4: 42, B=8: 28, B=16: 33 -> 8
    #   c2 (H=16, G=1, s'=64): B=4: 216, B=8: 192, B=16: 276 -> 8
    #   c3 (H=64, G=16, s'=256): B=16: 3648, B=32: 3264, B=64: 4608 -> 32
    # #galois = Rot_col + (B-1) baby + (s'/B-1) giant + sum over the
    # rotate-and-sum levels of (r-1): c1 m/s' = 2^7 -> radices 8,4,4 (13),
    # c2 2^6 -> 8,8 (14), c3 2^6 -> 8,8 (14)
    want = {"c1": (16, 8, 1, 2, 1, 1, 22), "c2": (64, 8, 8, 16, 1, 1, 29),
            "c3": (256, 32, 32, 64, 16, 1, 53)}
    for name, w in want.items():
        cfg = W.CONFIGS[name]
        par = bfv.Params.from_config(cfg)
        plan = pdq.make_plan(par, cfg.n, cfg.s)
        got = (plan.s_prime, plan.B, plan.J, plan.H, plan.G, plan.n_out,
               len(pdq.galois_elements(par, plan)))
        assert got == w, name


def test_rotsum_levels_cover_every_shift_once():
    """The levels' shifts sum_i j_i l_i (j_i < r_i) are exactly the multiples
    i s' for i < m/s', each once (brute force), with every radix at most 8,
    ceil(log2(m/s')/3) levels and the larger radices first (the schedule the
    library runs, so that both use the same rotation keys)."""
    from types import SimpleNamespace
    for bits in range(0, 11):
        for s_prime in (1, 4, 16):
            par = SimpleNamespace(m=s_prime << bits)
            plan = SimpleNamespace(s_prime=s_prime)
            lv = pdq.rotsum_levels(par, plan)
            assert len(lv) == -(-bits // 3)
            assert all(2 <= r <= 8 and r & (r - 1) == 0 for _, r in lv)
            assert [r for _, r in lv] == sorted((r for _, r in lv), reverse=True)
            shifts = [0]
            for l, r in lv:
                shifts = [x + j * l for x in shifts for j in range(r)]
            assert sorted(shifts) == [i * s_prime for i in range(1 << bits)]


def test_rotate_and_sum_is_the_sum_of_rotations():
    """Decrypting the hoisted rotate-and-sum gives sum_{i < m/s'} Rot(y; i s')
    on both rows, computed here from the slots with numpy rolls (two levels:
    m/s' = 16 on the N = 64 ring)."""
    par = bfv.Params.from_config(W.CONFIGS["tiny2"])
    plan = pdq.make_plan(par, 100, 2)
    assert par.m // plan.s_prime == 16 and len(pdq.rotsum_levels(par, plan)) == 2
    sk = W.draw_ternary(par.N, W.rng_for(31, 3))
    a, e = W.encryption_randomness(par.q, par.N, 1, seed=31)
    slots = W.rng_for(32).integers(0, par.t, size=par.N, dtype=np.uint64)
    ct = bfv.encrypt(par, sk, bfv.encode(par, slots), a[0], e[0])
    ks = sorted({par.galois_rot(j * l) for l, r in pdq.rotsum_levels(par, plan)
                 for j in range(1, r)})
    kr = W.rotation_key_randomness(par.ext, par.N, len(par.digits), ks, seed=33)
    keys = {k: bfv.rotation_key(par, sk, k, *kr[k]) for k in ks}
    y = pdq.rotate_and_sum(par, bfv.ct_times_P(par, ct), keys, plan)
    got = bfv.decrypt(par, sk, y).reshape(2, par.m)
    rows = slots.reshape(2, par.m).astype(np.int64)
    want = sum(np.roll(rows, -i * plan.s_prime, axis=1) for i in range(16)) % par.t
    assert np.array_equal(got.astype(np.int64), want)


def golden_rows(name):
    """Rows of a fixture under tests/golden/ ('#' starts a comment)."""
    rows = []
    for line in (pathlib.Path(__file__).parent / "golden" / name).read_text().splitlines():
        f = line.split("#", 1)[0].split()
        if f:
            rows.append(f)
    return rows


def test_paper_single_ciphertext_answer():
    """Sec. 6.2, Tables II and III (Size column; fixture paper_answer_size.txt):
    on the ring and modulus of Sec. 6.1 every answer is one ciphertext of
    110.6 KB.  The plan has one output ciphertext for every row (both record
    groups of the 2^17-record row share it), and that ciphertext switched to
    the first ciphertext prime is 2 polynomials of N coefficients of 54 bits.
    Footnote of Sec. 6.2: one ciphertext unless s exceeds N/2 = 4096."""
    par = bfv.Params.from_config(W.CONFIGS["paper"])
    assert (par.N, par.t, par.L, [q.bit_length() for q in par.q]) == (8192, 65537, 2, [54, 54])
    low = bfv.Params(par.log_n, par.t, par.bits, 1, par.K, 1)
    assert low.q == par.q[:1]
    rows = golden_rows("paper_answer_size.txt")
    assert len(rows) == 10
    for table, n, s, kb in rows:
        plan = pdq.make_plan(par, int(n), int(s))
        assert plan.n_out == 1, (table, n, s)
        assert plan.G == (2 if int(n) > 65536 else 1)
        size = plan.n_out * 2 * low.L * par.N * low.q[0].bit_length() // 8
        assert size == 110592 and round(size / 1000, 1) == float(kb), (table, n, s)
    assert pdq.make_plan(par, 1 << 14, 4096).n_out == 1
    with pytest.raises(ValueError):
        pdq.make_plan(par, 1 << 14, 4097)


@pytest.mark.parametrize("cfg_name", ["tiny", "tiny2", "grouped", "small"])
def test_closed_form_is_matrix_C(cfg_name):
    cfg = W.CONFIGS[cfg_name]
    par = bfv.Params.from_config(cfg)
    qi = W.draw_query(cfg)
    plan = pdq.make_plan(par, cfg.n, cfg.s)
    cf = pdq.closed_form(par, plan, qi.v, qi.db)
    t = par.t
    for gamma in range(plan.G):
        lo, hi = gamma * plan.G_sz, min((gamma + 1) * plan.G_sz, cfg.n)
        nodes = list(range(1, hi - lo + 1))
        C = matrix_C(plan.s_prime, nodes, t)
        v = [int(x) for x in qi.v[lo:hi]]
        d = [int(x) * int(y) % t for x, y in zip(qi.v[lo:hi], qi.db[lo:hi])]
        assert cf[gamma, 0].tolist() == [sum(c * x for c, x in zip(row, v)) % t for row in C]
        assert cf[gamma, 1].tolist() == [sum(c * x for c, x in zip(row, d)) % t for row in C]


@pytest.mark.parametrize("cfg_name", ["tiny", "grouped"])
def test_diagonal_bsgs_in_the_clear(cfg_name):
    """The extended diagonals, baby/giant split and rotate-and-sum reproduce
    C u in the clear (Sec. 5.2), for every half-block and group."""
    cfg = W.CONFIGS[cfg_name]
    par = bfv.Params.from_config(cfg)
    plan = pdq.make_plan(par, cfg.n, cfg.s)
    t, m, sp, B = par.t, par.m, plan.s_prime, plan.B
    rng = np.random.default_rng(5)
    u = [rng.integers(0, t, size=par.N, dtype=np.uint64) for _ in range(plan.H)]
    for gamma in range(plan.G):
        y = np.zeros(par.N, dtype=np.uint64)
        for g in range(plan.giants):
            acc = np.zeros(par.N, dtype=np.uint64)
            for h in pdq.group_halfblocks(plan, gamma):
                for a in range(B):
                    d = pdq.rot_slots(par, pdq.diagonal_slots(par, plan, h, g * B + a), -g * B)
                    acc = (acc + d * pdq.rot_slots(par, u[h], a)) % t
            y = (y + pdq.rot_slots(par, acc, g * B)) % t
        for l, r in pdq.rotsum_levels(par, plan):
            y = sum(pdq.rot_slots(par, y, j * l) for j in range(r)) % t
        # explicit product with the group's block of C, both rows
        for rho in range(2):
            want = [0] * sp
            for h in pdq.group_halfblocks(plan, gamma):
                for x in range(m):
                    node = (h * m + x) % plan.G_sz + 1
                    val = int(u[h][rho * m + x])
                    for j in range(sp):
                        want[j] = (want[j] + pow(node, j + 1, t) * val) % t
            row = y[rho * m:(rho + 1) * m]
            for o in range(m // sp):
                assert row[o * sp:(o + 1) * sp].tolist() == want


@pytest.mark.parametrize("cfg_name", ["tiny", "tiny2"])
def test_mask_and_pack_decrypt(cfg_name):
    cfg, par, qi, plan, keys, v_cts = build(cfg_name)
    masked = pdq.mask(par, v_cts, qi.db, plan)
    t = par.t
    for j in range(plan.J):
        v = pdq.record_slots(par, qi.v, j)
        d = v * pdq.record_slots(par, qi.db, j) % t
        top, bot = pdq.row_mask_slots(par, 0), pdq.row_mask_slots(par, 1)
        want = [v * top, v * bot, d * top, d * bot]
        for idx in range(4):
            assert np.array_equal(bfv.decrypt(par, qi.sk, masked[4 * j + idx]), want[idx])
    u = pdq.pack(par, masked, keys, plan)
    for h in range(plan.H):
        rec = np.arange(h * par.m, (h + 1) * par.m)
        vh = np.zeros(par.m, dtype=np.uint64)
        dh = np.zeros(par.m, dtype=np.uint64)
        ok = rec < cfg.n
        vh[ok] = qi.v[rec[ok]]
        dh[ok] = qi.v[rec[ok]].astype(np.uint64) * qi.db[rec[ok]] % t
        assert np.array_equal(bfv.decrypt(par, qi.sk, u[h]), np.concatenate([vh, dh]))


@pytest.mark.parametrize("cfg_name", ["tiny", "tiny2", "grouped"])
def test_mask_pack_decrypts_to_packed_halfblocks(cfg_name):
    """The fused Mask and pack (column rotation of v first) gives u_h with
    the slots [v_h; d_h] of the half-block, like pack(mask(v))."""
    cfg, par, qi, plan, keys, v_cts = build(cfg_name)
    u = pdq.mask_pack(par, v_cts, qi.db, keys, plan)
    assert len(u) == plan.H
    t = par.t
    for h in range(plan.H):
        rec = np.arange(h * par.m, (h + 1) * par.m)
        vh = np.zeros(par.m, dtype=np.uint64)
        dh = np.zeros(par.m, dtype=np.uint64)
        ok = rec < cfg.n
        vh[ok] = qi.v[rec[ok]]
        dh[ok] = qi.v[rec[ok]].astype(np.uint64) * qi.db[rec[ok]] % t
        assert np.array_equal(bfv.decrypt(par, qi.sk, u[h]), np.concatenate([vh, dh]))


@pytest.mark.parametrize("cfg_name", ["tiny", "grouped"])
def test_mask_pack_with_every_record_matching(cfg_name):
    """Every record a match (v = 1 everywhere): each slot of every half-block
    must come through Mask and the pack, so a row split that drops or moves a
    column shows.  The expected slots are read off the records directly."""
    cfg, par, qi, plan, keys, _ = build(cfg_name)
    v = np.ones(cfg.n, dtype=np.uint32)
    a, e = W.encryption_randomness(par.q, par.N, plan.J, cfg.seed + 7)
    v_cts = pdq.encrypt_index(par, qi.sk, v, plan, a, e)
    t = par.t
    for name, u in (("pack(mask)", pdq.pack(par, pdq.mask(par, v_cts, qi.db, plan), keys, plan)),
                    ("mask_pack", pdq.mask_pack(par, v_cts, qi.db, keys, plan))):
        for h in range(plan.H):
            rec = np.arange(h * par.m, (h + 1) * par.m)
            ok = rec < cfg.n
            vh = ok.astype(np.uint64)
            dh = np.zeros(par.m, dtype=np.uint64)
            dh[ok] = qi.db[rec[ok]].astype(np.uint64) % t
            got = bfv.decrypt(par, qi.sk, u[h])
            assert np.array_equal(got, np.concatenate([vh, dh])), (name, h)


@pytest.mark.parametrize("cfg_name", ["tiny", "grouped"])
def test_sigma_col_of_a_lifted_plaintext_swaps_its_rows(cfg_name):
    """sigma_{2N-1} applied limb by limb to a lifted plaintext equals the lift
    of the row-swapped slots (the identity mask_pack relies on)."""
    from oracle import ring
    par = bfv.Params.from_config(W.CONFIGS[cfg_name])
    slots = W.rng_for(41).integers(0, par.t, size=par.N, dtype=np.uint64)
    lifted = pdq.lifted_pt(par, slots)
    want = pdq.lifted_pt(par, pdq.swap_rows(par, slots))
    for i, q in enumerate(par.q):
        assert np.array_equal(ring.automorphism(lifted[i], par.galois_col, q), want[i])


@pytest.mark.parametrize("cfg_name", ["tiny2", "grouped"])
def test_comp_of_mask_decrypts_to_closed_form(cfg_name):
    """Comp on the masked ciphertexts (pack as Sec. 5.2 describes) gives the
    same slots as the Answer's fused schedule."""
    cfg, par, qi, plan, keys, v_cts = build(cfg_name)
    outs = pdq.comp(par, pdq.mask(par, v_cts, qi.db, plan), keys, plan)
    for ct, want in zip(outs, pdq.expected_slots(par, plan, qi.v, qi.db)):
        assert np.array_equal(bfv.decrypt(par, qi.sk, ct), want)


@pytest.mark.parametrize("cfg_name", ["tiny2", "grouped", "c1"])
def test_literal_mask_schedule(cfg_name):
    """The remark's literal schedule (row masks after d = v . DB): its four
    products decrypt to v.[1;0], v.[0;1], d.[1;0], d.[0;1], and Comp on them
    decrypts to the closed form with noise budget to spare (the extra
    plaintext product costs budget, pinned against the folded masks)."""
    cfg, par, qi, plan, keys, v_cts = build(cfg_name)
    lit = pdq.mask_literal(par, v_cts, qi.db, plan)
    t = par.t
    top, bot = pdq.row_mask_slots(par, 0), pdq.row_mask_slots(par, 1)
    for j in range(plan.J):
        v = pdq.record_slots(par, qi.v, j)
        d = v * pdq.record_slots(par, qi.db, j) % t
        for idx, want in enumerate([v * top, v * bot, d * top, d * bot]):
            assert np.array_equal(bfv.decrypt(par, qi.sk, lit[4 * j + idx]), want)
    outs = pdq.comp(par, lit, keys, plan)
    folded = pdq.comp(par, pdq.mask(par, v_cts, qi.db, plan), keys, plan)
    for ct, ref, want in zip(outs, folded, pdq.expected_slots(par, plan, qi.v, qi.db)):
        assert np.array_equal(bfv.decrypt(par, qi.sk, ct), want)
        assert bfv.noise_budget_bits(par, qi.sk, ct) > 5
        assert bfv.noise_budget_bits(par, qi.sk, ct) <= bfv.noise_budget_bits(par, qi.sk, ref) + 1


@pytest.mark.parametrize("cfg_name", ["tiny", "tiny2", "grouped", "small", "c1"])
def test_answer_decrypts_to_closed_form_and_decompresses(cfg_name):
    cfg, par, qi, plan, keys, v_cts = build(cfg_name)
    outs = pdq.answer(par, v_cts, qi.db, keys, plan)
    assert len(outs) == plan.n_out
    exp = pdq.expected_slots(par, plan, qi.v, qi.db)
    for ct, want in zip(outs, exp):
        assert np.array_equal(bfv.decrypt(par, qi.sk, ct), want)
        assert bfv.noise_budget_bits(par, qi.sk, ct) > 10
    got = pdq.decomp(par, qi.sk, plan, outs)
    assert got == [(int(i), int(qi.db[i])) for i in qi.positions]


@pytest.mark.parametrize("cfg_name", ["tiny2", "small"])
def test_answer_after_mod_switch(cfg_name):
    """Comp on smaller parameters: the query switched from 3 primes to 2,
    keys and plan for the 2-prime parameters (digits no wider than P:
    dnum = ceil(2 / K)); the answer decrypts to C v, C d and decompresses."""
    import dataclasses
    cfg, par, qi, plan, keys, v_cts = build(cfg_name)
    lcfg = dataclasses.replace(cfg, L=2, dnum=-(-2 // cfg.K))
    low = bfv.Params.from_config(lcfg)
    lplan = pdq.make_plan(low, cfg.n, cfg.s)
    ks = pdq.galois_elements(low, lplan)
    kr = W.rotation_key_randomness(low.ext, low.N, len(low.digits), ks, cfg.seed + 1)
    lkeys = {k: bfv.rotation_key(low, qi.sk, k, *kr[k]) for k in ks}
    outs = pdq.answer_switched(par, low, v_cts, qi.db, lkeys, lplan)
    for ct, want in zip(outs, pdq.expected_slots(low, lplan, qi.v, qi.db)):
        assert np.array_equal(bfv.decrypt(low, qi.sk, ct), want)
        assert bfv.noise_budget_bits(low, qi.sk, ct) > 10
    assert pdq.decomp(low, qi.sk, lplan, outs) == [(int(i), int(qi.db[i])) for i in qi.positions]
    # the answer switched to one prime before it leaves the server
    one = bfv.Params.from_config(dataclasses.replace(cfg, L=1, dnum=1))
    outs1 = [bfv.mod_switch(low, one, ct) for ct in outs]
    for ct, want in zip(outs1, pdq.expected_slots(one, lplan, qi.v, qi.db)):
        assert np.array_equal(bfv.decrypt(one, qi.sk, ct), want)
    assert pdq.decomp(one, qi.sk, lplan, outs1) == [(int(i), int(qi.db[i])) for i in qi.positions]


def test_newton_against_elementary_symmetric_bruteforce():
    t = 65537
    rnd = random.Random(4)
    for size in range(0, 9):
        xs = rnd.sample(range(1, 2000), size)
        s = 12
        w = [sum(pow(x, k, t) for x in xs) % t for k in range(1, s + 1)]
        a = pdq.newton_coefficients(w, t)
        for k in range(s + 1):
            ek = sum(np.prod([x for x in c], dtype=object) for c in itertools.combinations(xs, k)) \
                if k <= size else 0
            assert a[k] == int(ek) % t
        f = pdq.f_from_coefficients(a, t)          # prod over the multiset (X - x) X^{s-size}
        for x in xs + [0]:
            assert sum(c * pow(x, i, t) for i, c in enumerate(f)) % t == 0
        assert sorted(pdq.reconst_idx(w, t, 2000)) == sorted(xs)


def test_decomp_exhaustive_tiny():
    """Every s-sparse (v, d) with s <= 3 on n = 16 records decodes uniquely
    (records may hold the value 0)."""
    t, n, sp = 257, 16, 4
    rnd = random.Random(5)
    for size in range(0, 4):
        for idx in itertools.combinations(range(n), size):
            vals = [rnd.randrange(t) for _ in idx]
            nodes = [i + 1 for i in idx]
            w = [sum(pow(a, j + 1, t) for a in nodes) % t for j in range(sp)]
            e = [sum(pow(a, j + 1, t) * x for a, x in zip(nodes, vals)) % t for j in range(sp)]
            got_nodes = pdq.reconst_idx(w, t, n)
            assert got_nodes == nodes
            assert pdq.reconst(e, got_nodes, t) == vals


def test_decomp_single_match_closed_form():
    """s' = 1: the index is w_1 and the value e_1 / w_1."""
    t = 65537
    for node, val in [(1, 0), (7, 5), (65536, 65536), (300, 12)]:
        w = [node % t]
        e = [node * val % t]
        assert pdq.reconst_idx(w, t, 65536) == [node]
        assert pdq.reconst(e, [node], t) == [val * 1 % t]


def test_decomp_rejects_inconsistent_values():
    """Alg. 4 solves the square system on the first l rows; the rows l+1..s'
    of C d must agree with that solution, so a compressed value changed in
    one of them is reported instead of decoded (brute force over every
    extra row)."""
    t, sp = 65537, 8
    nodes, vals = [3, 10, 4000], [5, 0, 65536]
    w = [sum(pow(a, j + 1, t) for a in nodes) % t for j in range(sp)]
    e = [sum(pow(a, j + 1, t) * x for a, x in zip(nodes, vals)) % t for j in range(sp)]
    got = pdq.reconst_idx(w, t, 65536)
    assert got == nodes
    assert pdq.reconst(e, got, t) == vals
    for j in range(len(nodes), sp):
        bad = list(e)
        bad[j] = (bad[j] + 1) % t
        with pytest.raises(pdq.DecodeError):
            pdq.reconst(bad, got, t)


def test_decomp_detects_overflow():
    """More matches than s' do not decode to a wrong answer silently."""
    t, sp = 65537, 4
    nodes = [3, 10, 77, 1000, 5000, 12345]
    w = [sum(pow(a, j + 1, t) for a in nodes) % t for j in range(sp)]
    with pytest.raises(pdq.DecodeError):
        pdq.reconst_idx(w, t, 65536)
