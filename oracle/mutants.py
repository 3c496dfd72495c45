"""Planted mistakes in the oracle, to show that its pins catch them.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Each mutant is one small edit of one oracle source (a flipped sign, an index
off by one, a dropped factor or term, a swapped operand, a skipped check),
the kind of slip a reader of the paper could make.  ``run`` applies each to a
fresh copy of the oracle, its pins (``tests/test_oracle_*.py``) and the input
module, and runs those pins: a mutant is killed when they fail.  Every mutant
must be killed; one that survives means a pin is missing.

    python -m oracle.mutants [-j JOBS] [name ...]
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import dataclasses
import os
import shutil
import subprocess
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@dataclasses.dataclass(frozen=True)
class Mutant:
    name: str
    path: str        # relative to the repository root
    find: str        # occurs exactly once in the file
    replace: str
    what: str


def _m(name, path, find, replace, what):
    return Mutant(name, path, find, replace, what)


C, RING, BFV, PDQ = "oracle/ref_ring.c", "oracle/ring.py", "oracle/bfv.py", "oracle/pdq.py"

MUTANTS = [
    # ---- C core: modular arithmetic, transform, product, automorphism, conversion
    _m("powmod_square", C, "if (e & 1) r = mulmod(r, a, q);", "if (e & 1) r = mulmod(r, r, q);",
       "square-and-multiply multiplies by the wrong operand"),
    _m("invmod_exponent", C, "ref_powmod(a, q - 2, q)", "ref_powmod(a, q - 1, q)",
       "Fermat inverse with exponent q-1"),
    _m("vec_sub_swapped", C, "c[i] = submod(a[i], b[i], q);", "c[i] = submod(b[i], a[i], q);",
       "subtraction operands swapped"),
    _m("vec_scale_off", C, "c[i] = mulmod(a[i], w % q, q);", "c[i] = mulmod(a[i], (w + 1) % q, q);",
       "scalar off by one"),
    _m("schoolbook_cyclic", C, "else c[k - N] = submod(c[k - N], p, q);",
       "else c[k - N] = addmod(c[k - N], p, q);", "cyclic instead of negacyclic wrap"),
    _m("bitrev_wrong_bit", C, "r = (r << 1) | (x & 1);", "r = (r << 1) | ((x >> 1) & 1);",
       "bit reversal reads the wrong bit"),
    _m("dft_root_power", C, "ref_powmod(omega, N / len, q);", "ref_powmod(omega, N / len + 1, q);",
       "butterfly root of the wrong order"),
    _m("dft_butterfly_sign", C, "a[start + k + len / 2] = submod(u, v, q);",
       "a[start + k + len / 2] = addmod(u, v, q);", "butterfly difference added"),
    _m("ntt_no_twist", C, "cyclic_dft(a, logN, q, mulmod(psi, psi, q));",
       "cyclic_dft(a, logN, q, psi);", "forward transform with psi for omega"),
    _m("intt_no_ninv", C, "u64 n_inv = ref_invmod(N % q, q);", "u64 n_inv = 1;",
       "inverse transform without 1/N"),
    _m("automorphism_no_sign", C, "u64 wraps = (u64)((e / N) & 1);", "u64 wraps = 0;",
       "X^N = -1 ignored by the automorphism"),
    _m("automorphism_index", C, "u64 dst = (u64)(e % N);", "u64 dst = (u64)((e + 1) % N);",
       "automorphism target index off by one"),
    _m("convert_no_hat_inv", C, "u64 v = mulmod(x[i * N + c], hat_inv[i], src[i]);",
       "u64 v = x[i * N + c];", "basis conversion drops (S/s_i)^-1"),
    _m("convert_subtracts", C, "acc = addmod(acc, mulmod(v % r, hat_mod_r[i], r), r);",
       "acc = submod(acc, mulmod(v % r, hat_mod_r[i], r), r);", "conversion terms subtracted"),
    # ---- limb helpers
    _m("hat_inv_not_inverted", RING, "hat_inv = _u([invmod((S // s) % s, s) for s in src])",
       "hat_inv = _u([((S // s) % s) for s in src])", "hat not inverted"),
    _m("automorphism_mod_N", RING, "k % (2 * a.shape[-1])", "k % (a.shape[-1])",
       "Galois element reduced mod N instead of 2N"),
    # ---- scheme: primes, slots, encoding, encryption, keys, key switching
    _m("primes_minus_one", BFV, "p = ((1 << bits) - 2) // step * step + 1",
       "p = ((1 << bits) - 2) // step * step - 1", "prime candidates = -1 mod 2N"),
    _m("root_order_N", BFV, "if pow(c, N, q) == q - 1:", "if pow(c, N, q) == 1:",
       "root of order dividing N, not 2N"),
    _m("zeta_order", BFV, "(self.t - 1) // (2 * self.N), self.t)", "(self.t - 1) // self.N, self.t)",
       "slot root of order N"),
    _m("slot_rows_same", BFV, "e[self.m + c] = (2 * self.N - g) % (2 * self.N)",
       "e[self.m + c] = g", "both slot rows at the same exponents"),
    _m("slot_generator_5", BFV, "g = g * 3 % (2 * self.N)", "g = g * 5 % (2 * self.N)",
       "slot order generated by 5 instead of 3"),
    _m("galois_rot_off", BFV, "return pow(3, r % self.m, 2 * self.N)",
       "return pow(3, (r + 1) % self.m, 2 * self.N)", "row rotation by one step more"),
    _m("galois_col_N", BFV, "return 2 * self.N - 1", "return self.N - 1",
       "column swap element N-1"),
    _m("decode_reversed", BFV, "return vals[(par.slot_exponents() - 1) // 2]",
       "return vals[(par.slot_exponents() - 1) // 2][::-1]", "decoded slots reversed"),
    _m("lift_not_centred", BFV, "neg = c > (par.t - 1) // 2", "neg = c > par.t",
       "plaintext lifted without centring"),
    _m("signed_drops_sign", BFV,
       "out[i] = np.where(x < 0, np.uint64(r) - (-x).astype(np.uint64), x.astype(np.uint64))",
       "out[i] = np.where(x < 0, (-x).astype(np.uint64), x.astype(np.uint64))",
       "negative coefficients lose their sign"),
    _m("encrypt_plus_as", BFV, "c0 = poly_add(par, poly_sub(par, e_r, as_, ql), dm, ql)",
       "c0 = poly_add(par, poly_add(par, e_r, as_, ql), dm, ql)", "c0 = +a s + e + Delta m"),
    _m("delta_off_by_one", BFV, "par.delta % par.q[i], par.q[i])", "(par.delta + 1) % par.q[i], par.q[i])",
       "Delta = floor(Q/t) + 1"),
    _m("crt_no_inverse", BFV, "coef = hat * pow(hat % qi, -1, qi)", "coef = hat",
       "CRT without the hat inverse"),
    _m("decrypt_floor", BFV, "m = np.array([((t * xv + Q // 2) // Q) % t for xv in X], dtype=np.uint64)",
       "m = np.array([((t * xv) // Q) % t for xv in X], dtype=np.uint64)",
       "decryption floors instead of rounding"),
    _m("key_plus_as", BFV, "        b = poly_sub(par, e_b, poly_mul(par, a_b, s, el), el)",
       "        b = poly_add(par, e_b, poly_mul(par, a_b, s, el), el)", "key b = +a s + e"),
    _m("key_unrotated_secret", BFV,
       "b[i] = ring.vec_add(b[i], ring.vec_scale(sk_k[i], par.P % qi, qi), qi)",
       "b[i] = ring.vec_add(b[i], ring.vec_scale(s[i], par.P % qi, qi), qi)",
       "key encrypts s instead of sigma_k(s)"),
    _m("mod_up_copies_all", BFV, "if l < par.L and l in digit:", "if l < par.L:",
       "raise copies every Q limb instead of converting"),
    _m("mod_down_adds", BFV,
       "out[i] = ring.vec_scale(ring.vec_sub(y[i], conv, qi), pow(par.P % qi, -1, qi), qi)",
       "out[i] = ring.vec_scale(ring.vec_add(y[i], conv, qi), pow(par.P % qi, -1, qi), qi)",
       "ModDown adds the converted special part"),
    _m("mod_down_no_pinv", BFV,
       "out[i] = ring.vec_scale(ring.vec_sub(y[i], conv, qi), pow(par.P % qi, -1, qi), qi)",
       "out[i] = ring.vec_sub(y[i], conv, qi)", "ModDown without P^-1"),
    _m("mod_switch_no_dinv", BFV, "pow(D % qi, -1, qi), qi)", "1, qi)",
       "modulus switch without D^-1"),
    _m("mod_switch_wrong_limbs", BFV, "yd = np.stack([ct[p_idx][low.L + k] for k in range(len(dropped))])",
       "yd = np.stack([ct[p_idx][k] for k in range(len(dropped))])", "switch converts kept limbs"),
    _m("rotate_c0_unrotated", BFV,
       "c0 = poly_add(par, poly_automorphism(par, ct[0], k, ql), mod_down(par, A0), ql)",
       "c0 = poly_add(par, ct[0], mod_down(par, A0), ql)", "rotation leaves c0 unrotated"),
    _m("rotate_ext_c0_unrotated", BFV, "pc0 = times_P(par, poly_automorphism(par, ct[0], k, qlimbs(par)))",
       "pc0 = times_P(par, ct[0])", "extended rotation leaves c0 unrotated"),
    _m("lazy_c0_unrotated", BFV,
       "return np.stack([poly_add(par, A0, poly_automorphism(par, ct_ext[0], k, el), el), A1])",
       "return np.stack([poly_add(par, A0, ct_ext[0], el), A1])", "lazy rotation leaves c0 unrotated"),
    _m("times_P_dropped", BFV, "out[i] = ring.vec_scale(x[i], par.P % qi, qi)", "out[i] = x[i].copy()",
       "P x without P"),
    _m("embed_negated", BFV, "out[::R] = s", "out[::R] = -s", "subring secret embedded negated"),
    _m("ring_parts_reversed", BFV, "sw[:, :, r::R]) for r in range(R)]",
       "sw[:, :, r::R]) for r in reversed(range(R))]", "ring-switched parts in reverse order"),
    _m("switch_key_target", BFV,
       "b[i] = ring.vec_add(b[i], ring.vec_scale(s_from[i], par.P % qi, qi), qi)",
       "b[i] = ring.vec_add(b[i], ring.vec_scale(s_to[i], par.P % qi, qi), qi)",
       "ring-switching key encrypts the target secret"),
    # ---- the method: plan, layout, Mask, pack, diagonals, BSGS, rotate-and-sum, groups
    _m("group_size_short", PDQ, "    G_sz = par.N * ((par.t - 1) // par.N)\n",
       "    G_sz = par.N * ((par.t - 1) // par.N) - par.m\n", "record groups half a row short"),
    _m("baby_cost_weight", PDQ, "H * (b - 1) + 8 * G * (s_prime // b - 1)",
       "H * (b - 1) + G * (s_prime // b - 1)", "giant-step key switches under-weighted in the B rule"),
    _m("rotsum_radix_order", PDQ, "r = 1 << (base + (1 if i < extra else 0))",
       "r = 1 << (base + (1 if i > extra else 0))", "rotate-and-sum radices do not cover m/s'"),
    _m("record_shift", PDQ, "chunk = np.asarray(values[j * par.N:(j + 1) * par.N], dtype=np.uint64)",
       "chunk = np.asarray(values[j * par.N + 1:(j + 1) * par.N + 1], dtype=np.uint64)",
       "records shifted by one slot"),
    _m("row_mask_short", PDQ, "s[rho * par.m:(rho + 1) * par.m] = 1", "s[rho * par.m:(rho + 1) * par.m - 1] = 1",
       "row mask misses the last column"),
    _m("mask_wrong_row", PDQ, "out.append(pt_mul(par, v_cts[j], lifted_pt(par, dbs * top)))",
       "out.append(pt_mul(par, v_cts[j], lifted_pt(par, dbs * bot)))", "dT masked with the bottom row"),
    _m("pack_no_rot_col", PDQ, "u.append(ct_add(par, vT, rotate(par, dT, kc, keys[kc])))",
       "u.append(ct_add(par, vT, dT))", "pack without Rot_col"),
    _m("mask_pack_no_swap", PDQ, "pt_mul(par, w, lifted_pt(par, swap_rows(par, dbs * top)))",
       "pt_mul(par, w, lifted_pt(par, dbs * top))", "sigma_col of the plaintext not applied"),
    _m("nodes_from_zero", PDQ, "return ((h * par.m + x) % plan.G_sz + 1).astype(np.uint64)",
       "return ((h * par.m + x) % plan.G_sz).astype(np.uint64)", "nodes start at 0"),
    _m("diag_power_off", PDQ, "row = powmod_vec(nodes, (c % plan.s_prime) + 1, par.t)",
       "row = powmod_vec(nodes, (c % plan.s_prime), par.t)", "diagonal powers 0..s'-1"),
    _m("diag_index_sign", PDQ, "nodes = node_row(par, plan, h)[(c + k) % m]",
       "nodes = node_row(par, plan, h)[(c - k) % m]", "diagonal index c - k"),
    _m("rot_slots_direction", PDQ, "return np.roll(s, -r, axis=1).reshape(-1)",
       "return np.roll(s, r, axis=1).reshape(-1)", "slot rotation to the right"),
    _m("ring_dot_root", PDQ, "q, psi = par.q[i], par.psi[i]", "q, psi = par.q[i], par.psi[(i + 1) % L]",
       "plaintext product with another prime's root"),
    _m("baby_step_off", PDQ, "            k = par.galois_rot(a)\n", "            k = par.galois_rot(a + 1)\n",
       "baby step a rotates by a + 1"),
    _m("giant_prerot_sign", PDQ, "d = rot_slots(par, diag(par, plan, h, g * plan.B + a), -g * plan.B)",
       "d = rot_slots(par, diag(par, plan, h, g * plan.B + a), g * plan.B)",
       "diagonal pre-rotated the wrong way"),
    _m("giant_lowers_c0", PDQ, "raised = mod_up_all(par, mod_down(par, acc[gamma][g][1]))",
       "raised = mod_up_all(par, mod_down(par, acc[gamma][g][0]))", "giant step raises c0"),
    _m("giant_drops_g0", PDQ, "        y = acc[gamma][0]\n", "        y = np.zeros_like(acc[gamma][0])\n",
       "unrotated accumulator dropped"),
    _m("rotsum_drops_j0", PDQ, "        acc = y\n", "        acc = np.zeros_like(y)\n",
       "rotate-and-sum drops Rot(y; 0)"),
    _m("group_mask_one_row", PDQ,
       "s[rho * par.m + o * plan.s_prime: rho * par.m + (o + 1) * plan.s_prime] = 1",
       "s[o * plan.s_prime:(o + 1) * plan.s_prime] = 1", "group mask on row 0 only"),
    _m("combine_drops_last", PDQ, "        gs = range(c * plan.per_out, min((c + 1) * plan.per_out, plan.G))\n",
       "        gs = range(c * plan.per_out, min((c + 1) * plan.per_out, plan.G) - 1)\n",
       "last group of an output dropped"),
    _m("closed_form_d_is_db", PDQ, "d = v * np.asarray(db, dtype=np.uint64) % t",
       "d = np.asarray(db, dtype=np.uint64) % t", "closed form uses DB for v.DB"),
    _m("closed_form_nodes", PDQ,
       "alpha = (np.arange(lo, hi, dtype=np.int64) % plan.G_sz + 1).astype(np.uint64)",
       "alpha = (np.arange(lo, hi, dtype=np.int64) % plan.G_sz + 2).astype(np.uint64)",
       "closed form with nodes from 2"),
    _m("switched_hpg", PDQ, "    hpg = G_sz // small.m\n", "    hpg = G_sz // big.m\n",
       "switched plan counts big half-blocks per group"),
    _m("switched_exponent_step", PDQ,
       "e_big = e_small[:, None] + 2 * small.N * np.arange(R, dtype=np.int64)[None, :]",
       "e_big = e_small[:, None] + small.N * np.arange(R, dtype=np.int64)[None, :]",
       "fold of the slot exponents by N' instead of 2N'"),
    _m("switched_no_factor", PDQ,
       "row = (row + powmod_vec(alpha[cc, u], kk, t) * factor[cc, u]) % np.uint64(t)",
       "row = (row + powmod_vec(alpha[cc, u], kk, t)) % np.uint64(t)", "fold factor zeta^(e r) dropped"),
    _m("plain_db_rows_swapped", PDQ, "        if rho != sigma:\n", "        if rho == sigma:\n",
       "database multiplied into the wrong row"),
    _m("plain_db_no_col", PDQ, "k = par.galois_rot(g * plan.B) * (col if sigma else 1) % (2 * par.N)",
       "k = par.galois_rot(g * plan.B)", "set 1 without Rot_col"),
    # ---- Decomp
    _m("newton_sign", PDQ, "acc += term if i % 2 == 1 else -term", "acc += term",
       "Newton's identity without alternating signs"),
    _m("newton_no_kinv", PDQ, "a.append(acc * pow(k, -1, t) % t)", "a.append(acc % t)",
       "Newton's identity without 1/k"),
    _m("f_reversed", PDQ, "f[s - k] = (a[k] if k % 2 == 0 else -a[k]) % t",
       "f[k] = (a[k] if k % 2 == 0 else -a[k]) % t", "f's coefficients reversed"),
    _m("strip_once", PDQ, "while i < len(f) - 1 and f[i] == 0:", "while i < min(len(f) - 1, 1) and f[i] == 0:",
       "at most one factor of X stripped"),
    _m("vandermonde_power", PDQ, "A = [[pow(a, j + 1, t) for a in nodes] for j in range(l)]",
       "A = [[pow(a, j, t) for a in nodes] for j in range(l)]", "Vandermonde rows from power 0"),
    _m("no_consistency_rows", PDQ,
       "if sum(pow(a, j + 1, t) * xi for a, xi in zip(nodes, x)) % t != int(e[j]) % t:",
       "if False:", "remaining rows not checked"),
    _m("decomp_index_off", PDQ, "res.extend((gamma * plan.G_sz + a - 1, int(x)) for a, x in zip(nodes, vals))",
       "res.extend((gamma * plan.G_sz + a, int(x)) for a, x in zip(nodes, vals))",
       "record index off by one"),
]

PIN_FILES = ["tests/test_oracle_bfv.py", "tests/test_oracle_pdq.py", "tests/test_oracle_plain_db.py",
             "tests/test_oracle_ring.py", "tests/test_oracle_ring_switch.py"]


def check(m: Mutant, root: str = ROOT) -> None:
    """Raise unless the mutant applies to the current source exactly once."""
    text = open(os.path.join(root, m.path)).read()
    n = text.count(m.find)
    if n != 1:
        raise ValueError(f"{m.name}: the text to replace occurs {n} times in {m.path}")
    if m.find == m.replace:
        raise ValueError(f"{m.name}: replacement equals the original")


def _copy_tree(dst: str) -> None:
    ignore = shutil.ignore_patterns("_build", "__pycache__", "*.so", "*.pyc")
    for d in ("oracle", "workloads"):
        shutil.copytree(os.path.join(ROOT, d), os.path.join(dst, d), ignore=ignore)
    os.makedirs(os.path.join(dst, "tests", "golden"))
    for f in PIN_FILES + ["tests/conftest.py"]:
        shutil.copy(os.path.join(ROOT, f), os.path.join(dst, f))
    for f in os.listdir(os.path.join(ROOT, "tests", "golden")):
        if f.endswith(".txt"):
            shutil.copy(os.path.join(ROOT, "tests", "golden", f), os.path.join(dst, "tests", "golden", f))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), os.path.join(dst, "pytest.ini"))


def run_one(m: Mutant, timeout: int = 600) -> tuple[str, str]:
    """('killed' | 'survived' | 'invalid' | 'timeout', detail) for one mutant."""
    check(m)
    with tempfile.TemporaryDirectory(prefix="pdq_mutant_") as tmp:
        _copy_tree(tmp)
        p = os.path.join(tmp, m.path)
        text = open(p).read()
        open(p, "w").write(text.replace(m.find, m.replace, 1))
        if m.path.endswith(".c"):
            cc = subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o",
                                 os.path.join(tmp, "check.so"), p], capture_output=True, text=True)
            if cc.returncode != 0:
                return "invalid", cc.stderr.strip().splitlines()[-1] if cc.stderr else "gcc failed"
        cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
               *PIN_FILES]
        try:
            r = subprocess.run(cmd, cwd=tmp, capture_output=True, text=True, timeout=timeout)
        except subprocess.TimeoutExpired:
            return "timeout", f"pins did not finish in {timeout} s"
        if r.returncode == 0:
            return "survived", r.stdout.strip().splitlines()[-1]
        if r.returncode in (2, 3, 4):
            return "invalid", (r.stdout + r.stderr).strip().splitlines()[-1]
        failed = [ln for ln in r.stdout.splitlines() if ln.startswith("FAILED")]
        return "killed", failed[0] if failed else r.stdout.strip().splitlines()[-1]


def run(names=None, jobs: int = 4) -> dict[str, tuple[str, str]]:
    chosen = [m for m in MUTANTS if not names or m.name in names]
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        res = dict(zip([m.name for m in chosen], ex.map(run_one, chosen)))
    return res


def main() -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("-j", "--jobs", type=int, default=max(1, (os.cpu_count() or 2) // 2))
    ap.add_argument("names", nargs="*")
    args = ap.parse_args()
    res = run(args.names, args.jobs)
    what = {m.name: m for m in MUTANTS}
    for name, (verdict, detail) in res.items():
        print(f"{verdict:8s} {name:26s} {what[name].what}  [{detail}]")
    counts = {v: sum(1 for r in res.values() if r[0] == v) for v in ("killed", "survived", "invalid", "timeout")}
    print(" ".join(f"{k} {v}" for k, v in counts.items()), f"of {len(res)}")
    return 0 if counts["survived"] == counts["invalid"] == 0 else 1


if __name__ == "__main__":
    sys.exit(main())
