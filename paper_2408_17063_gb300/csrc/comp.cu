// Comp and Answer (Alg. 7) in the SIMD form of Sec. 5.2, plus the C ABI
// entry points of the library's device-side calls.
//
// Schedule (every key switch raises the digits of c1 before the
// automorphism; additions are exact, so their order is free):
//   1. pack   u_{2j} = vT_j + Rot_col(dT_j),  u_{2j+1} = Rot_col(vB_j) + dB_j;
//             the Answer rotates v_j instead and masks after:
//             u_{2j} = v_j.[1;0] + Rot_col(v_j).sigma_col(DB_j.[1;0]),
//             u_{2j+1} = Rot_col(v_j).[1;0] + v_j.(DB_j.[0;1])
//   2. baby   R[h][a] = Rot(u_h; a), a < B, digits of u_h raised once
//   3. MAC    acc[gamma][g] = sum_{h in gamma} sum_a Rot(D_{h,gB+a}; -gB) . R[h][a]
//   4. giant  y_gamma = sum_g Rot(acc[gamma][g]; gB)
//   5. sum    y <- sum_{j<r} Rot(y; j l) per level (l, r) of rotsum_levels:
//             all i s', i < m/s', each once; one raise per level
// Ciphertexts over Q u P that are only rotated next (accumulators, giant
// sums, rotate-and-sum levels) lower only c1 for the key switch; c0 joins the
// rotation from Q u P, and the result is lowered once at the end.
//   6. groups out_c = sum_o M_o . y_{c per_out + o}   (one group: out = y)
#include <algorithm>
#include <cstring>
#include <initializer_list>

#include "pdq_internal.h"
#include "pdq_ops.h"

namespace pdq {

namespace {

const Ctx& C(const pdq_ctx* p) { return *reinterpret_cast<const Ctx*>(p); }

u32 ceil_log2(u64 x) {
    u32 r = 0;
    while ((1ull << r) < x) ++r;
    return r;
}

// the power of two minimising the work of the baby/giant split:
// H (B-1) hoisted baby rotations, G (s'/B - 1) giant-step key switches and
// G s'/B accumulator ModDowns, weighted 1 : 8 : 3
u32 default_baby_steps(u64 H, u64 G, u64 sp) {
    u64 best = ~0ull;
    u32 B = 1;
    for (u64 b = 1; b <= sp && b <= 128; b *= 2) {
        const u64 gi = sp / b;
        if (gi > 32) continue;
        const u64 cost = H * (b - 1) + 8 * G * (gi - 1) + 3 * G * gi;
        if (cost < best) { best = cost; B = (u32)b; }
    }
    return B;
}

int plan_make(const Ctx& c, u64 n, u32 s, u32 B, pdq_plan* pl) {
    if (n == 0 || s == 0) return fail(PDQ_E_PARAM, "plan: n and s must be positive");
    std::memset(pl, 0, sizeof(*pl));
    const u64 sp = 1ull << ceil_log2(s);
    if (sp > c.m || sp >= c.t) return fail(PDQ_E_PARAM, "plan: sparsity too large for the ring");
    const u64 J = (n + c.N - 1) / c.N;
    if (J > (1u << 20)) return fail(PDQ_E_PARAM, "plan: too many records");
    const u64 G_sz = (u64)c.N * ((c.t - 1) / c.N);
    const u64 hpg = G_sz / c.m;
    const u64 H = 2 * J;
    const u64 G = (H + hpg - 1) / hpg;
    if (B == 0) B = default_baby_steps(H, G, sp);
    if (sp % B != 0 || B > 128) return fail(PDQ_E_PARAM, "plan: B must divide s' and be at most 128");
    const u64 per_out = c.m / sp;
    pl->n = n;
    pl->s = s;
    pl->s_prime = (u32)sp;
    pl->B = B;
    pl->giants = (u32)(sp / B);
    pl->J = (u32)J;
    pl->H = (u32)H;
    pl->G_sz = (u32)G_sz;
    pl->hpg = (u32)hpg;
    pl->G = (u32)G;
    pl->hclass = (u32)std::min(hpg, H);
    pl->per_out = (u32)per_out;
    pl->n_out = (u32)((G + per_out - 1) / per_out);
    pl->ring_ratio = 1;
    if (pl->giants > 32) return fail(PDQ_E_PARAM, "plan: at most 32 giant steps (choose a larger B)");
    return PDQ_OK;
}

}  // namespace

// Comp in the subring c (dimension N) of a ring of dimension Nbig = 2^big_log_n
// after ring switching (Sec. 5.3): big ciphertext j becomes R = Nbig/N small
// ciphertexts R j + r, and the records keep the big ring's groups of
// G_sz = Nbig floor((t-1)/Nbig) records, i.e. G_sz/m small half-blocks each.
int plan_make_switched(const Ctx& c, u32 big_log_n, u64 n, u32 s, u32 B, pdq_plan* pl) {
    if (big_log_n <= c.log_n || big_log_n > 16) return fail(PDQ_E_PARAM, "plan: the big ring must be larger (at most 2^16)");
    const u64 Nbig = 1ull << big_log_n, R = Nbig / c.N;
    if ((c.t - 1) % (2 * Nbig) != 0) return fail(PDQ_E_PARAM, "plan: t must be 1 mod 2 N_big");
    if (n == 0 || s == 0) return fail(PDQ_E_PARAM, "plan: n and s must be positive");
    std::memset(pl, 0, sizeof(*pl));
    const u64 sp = 1ull << ceil_log2(s);
    if (sp > c.m || sp >= c.t) return fail(PDQ_E_PARAM, "plan: sparsity too large for the ring");
    const u64 J = R * ((n + Nbig - 1) / Nbig);
    if (J > (1u << 20)) return fail(PDQ_E_PARAM, "plan: too many records");
    const u64 G_sz = Nbig * ((c.t - 1) / Nbig);
    const u64 hpg = G_sz / c.m;
    const u64 H = 2 * J;
    const u64 G = (H + hpg - 1) / hpg;
    if (B == 0) B = default_baby_steps(H, G, sp);
    if (sp % B != 0 || B > 128) return fail(PDQ_E_PARAM, "plan: B must divide s' and be at most 128");
    const u64 per_out = c.m / sp;
    pl->n = n;
    pl->s = s;
    pl->s_prime = (u32)sp;
    pl->B = B;
    pl->giants = (u32)(sp / B);
    pl->J = (u32)J;
    pl->H = (u32)H;
    pl->G_sz = (u32)G_sz;
    pl->hpg = (u32)hpg;
    pl->G = (u32)G;
    pl->hclass = (u32)std::min(hpg, H);
    pl->per_out = (u32)per_out;
    pl->n_out = (u32)((G + per_out - 1) / per_out);
    pl->ring_ratio = (u32)R;
    if (pl->giants > 32) return fail(PDQ_E_PARAM, "plan: at most 32 giant steps (choose a larger B)");
    return PDQ_OK;
}

// The Answer on an unencrypted database (Sec. 5.2 remark): the layout of
// plan_make; B = 0 minimises J (B-1) + 8 G (2 s'/B - 1) + 6 G s'/B (baby
// rotations of the J index ciphertexts, giant-step key switches of both
// diagonal sets, accumulator ModDowns).
int plan_make_plain_db(const Ctx& c, u64 n, u32 s, u32 B, pdq_plan* pl) {
    PDQ_TRY(plan_make(c, n, s, B, pl));
    if (B == 0) {
        u64 best = ~0ull;
        u32 bb = pl->B;
        for (u64 b = 1; b <= pl->s_prime && b <= 128; b *= 2) {
            const u64 gi = pl->s_prime / b;
            if (gi > 32) continue;
            const u64 cost = (u64)pl->J * (b - 1) + 8ull * pl->G * (2 * gi - 1) + 6ull * pl->G * gi;
            if (cost < best) { best = cost; bb = (u32)b; }
        }
        PDQ_TRY(plan_make(c, n, s, bb, pl));
    }
    pl->plain_db = 1;
    return PDQ_OK;
}

namespace {

u64 galois_rot(const Ctx& c, long long r) {
    const long long m = c.m;
    long long rr = ((r % m) + m) % m;
    return host_powmod(3, (u64)rr, 2ull * c.N);
}

// Levels (l, r) of the rotate-and-sum (Sec. 5.2 sums Rot(y; i s') over
// i < m/s'): level i sums Rot(.; j l), j < r, l = s' times the earlier radices.
// The log2(m/s') bits are split into ceil(bits/3) chunks as evenly as
// possible, larger first (radix <= 8: one raise and one ModDown per level
// instead of per doubling, at most 7 hoisted rotations each).
std::vector<std::pair<u64, u32>> rotsum_levels(const Ctx& c, const pdq_plan& pl) {
    std::vector<std::pair<u64, u32>> lv;
    const u32 bits = ceil_log2(c.m / pl.s_prime);
    if (bits == 0) return lv;
    const u32 nlev = (bits + 2) / 3, base = bits / nlev, extra = bits % nlev;
    u64 l = pl.s_prime;
    for (u32 i = 0; i < nlev; ++i) {
        const u32 r = 1u << (base + (i < extra ? 1 : 0));
        lv.emplace_back(l, r);
        l *= r;
    }
    return lv;
}

std::vector<u64> plan_galois(const Ctx& c, const pdq_plan& pl) {
    std::vector<u64> ks;
    ks.push_back(2ull * c.N - 1);
    for (u32 a = 1; a < pl.B; ++a) ks.push_back(galois_rot(c, a));
    for (u32 g = 1; g < pl.giants; ++g) ks.push_back(galois_rot(c, (long long)g * pl.B));
    if (pl.plain_db)           // set 1 of the giant steps goes through Rot_col
        for (u32 g = 1; g < pl.giants; ++g)
            ks.push_back(galois_rot(c, (long long)g * pl.B) * (2ull * c.N - 1) % (2ull * c.N));
    for (const auto& [l, r] : rotsum_levels(c, pl))
        for (u32 j = 1; j < r; ++j) ks.push_back(galois_rot(c, (long long)(j * l)));
    std::sort(ks.begin(), ks.end());
    ks.erase(std::unique(ks.begin(), ks.end()), ks.end());
    return ks;
}

}  // namespace

bool valid_plan(const Ctx& c, const pdq_plan* pl) {
    if (!pl) return false;
    pdq_plan chk;
    int rc;
    if (pl->ring_ratio > 1) {
        const u32 R = pl->ring_ratio;
        if ((R & (R - 1)) != 0 || R > (1u << 13)) return false;
        rc = plan_make_switched(c, c.log_n + log2_exact(R), pl->n, pl->s, pl->B, &chk);
    } else if (pl->plain_db) {
        rc = plan_make_plain_db(c, pl->n, pl->s, pl->B, &chk);
    } else {
        rc = plan_make(c, pl->n, pl->s, pl->B, &chk);
    }
    if (rc != PDQ_OK) return false;
    return std::memcmp(&chk, pl, sizeof(chk)) == 0;
}

namespace {

struct Keys {
    const u64* base;
    const u64* galois;
    u32 n;
    u64 keysz;
    const u64* find(u64 k) const {
        for (u32 i = 0; i < n; ++i)
            if (galois[i] == k) return base + (u64)i * keysz;
        return nullptr;
    }
};

// Workspace of Comp, in uint64 elements from its start; the one place that
// fixes both the size and the placement of every region.
struct CompLayout {
    u64 U;      // packed u_h over Q, [H]
    u64 Rx;     // baby steps over Q u P [H][B], later the rotations of one
                // rotate-and-sum level (at most 8 per group)
    u64 accx;   // accumulators g >= 1 over Q u P, [G][giants-1]
    u64 acc;    // ... their c1 lowered to Q, [G][giants-1][L][N]
    u64 yx;     // giant-step sums over Q u P (from g = 0), [G]
    u64 Y0, Y1; // rotate-and-sum: the lowered c1 of a level, the output over Q
    u64 rws;    // key-switch raise scratch
    u64 aws;    // key-switch apply / ModDown scratch
    u64 end;
};

// Primes of the baby-step rotations held at once: all of them, or as many
// as the context's rotation budget allows (at least one).
u32 rotation_chunk(const Ctx& c, const pdq_plan& pl, u32 Q = 1) {
    const u32 E = c.L + c.K;
    if (c.rotation_budget == 0 || pl.B == 1 || !rotations_chunkable(c)) return E;
    const u64 per_prime = (u64)pl.H * Q * pl.B * 2 * c.N * sizeof(u64);
    const u64 k = c.rotation_budget / per_prime;
    return (u32)std::max<u64>(1, std::min<u64>(E, k));
}

// (Q queries of plan pl answered together: Q times the half-blocks and groups)
CompLayout comp_layout(const Ctx& c, const pdq_plan& pl, u32 Q = 1) {
    const u64 cts = ct_elems(c), ects = 2ull * (c.L + c.K) * c.N;
    const u64 G = (u64)pl.G * Q, GI = pl.giants, H = (u64)pl.H * Q;
    // raises: every u_h (baby steps), every lowered accumulator at once
    // (giant steps), every y (rotate-and-sum levels)
    const u32 cnt = (u32)std::max({H, G, G * (GI - 1)});
    const u64 scratch = std::max({apply_ws(c, cnt), mod_down_ws(c, (u32)G),
                                  mod_down_polys_ws(c, (u32)std::max<u64>(1, G * (GI - 1))),
                                  mod_down_polys_ws(c, (u32)G)}) / sizeof(u64);
    CompLayout lo;
    lo.U = 0;
    lo.Rx = lo.U + H * cts;
    const u64 echunk = 2ull * rotation_chunk(c, pl, Q) * c.N;
    lo.accx = lo.Rx + std::max<u64>(H * pl.B * echunk, G * 8 * ects);
    lo.acc = lo.accx + G * (GI - 1) * ects;
    lo.yx = lo.acc + G * (GI - 1) * cts;
    lo.Y0 = lo.yx + G * ects;
    lo.Y1 = lo.Y0 + G * cts;
    lo.rws = lo.Y1 + G * cts;
    lo.aws = lo.rws + raise_ws(c, cnt) / sizeof(u64);
    lo.end = lo.aws + scratch;
    return lo;
}

size_t comp_ws_bytes(const Ctx& c, const pdq_plan& pl, u32 Q = 1) {
    return comp_layout(c, pl, Q).end * sizeof(u64);
}

// The Answer's first stage for the jn index ciphertexts at v (NTT form):
// w_j = Rot_col(v_j), then the Mask products fused with the pack into
// u_{2j}, u_{2j+1}.  v, db, w and U point at the run's first j; rws and aws
// are Comp's key-switch scratch.
// (sk: jn = Q Jq index ciphertexts of the stacked queries, Jq each, every
// query masked by the same Jq database plaintexts and rotated with its keys)
int answer_pack(const Ctx& c, const Keys& keys, const u64* v, const u64* db, u64* w, u64* U,
                u32 jn, u64* rws, u64* aws, cudaStream_t st, const Stack* sk = nullptr,
                u32 Jq = 0) {
    const long long cts = (long long)ct_elems(c);
    const u64 kc = 2ull * c.N - 1;
    const u64* kp = keys.find(kc);
    if (!kp) return fail(PDQ_E_KEY, "answer: missing rotation key for Galois element " + std::to_string(kc));
    const CtSet vin = ct_set(v, cts);
    u64* D = nullptr;
    PDQ_TRY(ks_raise(c, vin, jn, rws, &D, st));
    const KeyTable kt = sk ? sk->table(Jq) : single_keys(keys.base);
    PDQ_TRY(ks_apply(c, D, vin, jn, (u32)kc, kp, ct_set(w, cts), CtSet{}, aws, st, &kt));
    prof_mark(c, PDQ_STAGE_MASK, st);
    return mask_pack(c, jn, v, w, db, U, st, Jq);
}

// Steps 5 and 6 of Comp on the giant-step sums yx ([G][2][L+K][N]): the
// rotate-and-sum on y over Q u P (per level the lowered c1 of every y, into
// Y1, is raised once, the r rotations (a = 0: y itself) go to Rx and are
// summed back into yx; the last level's sum is lowered to Y0), then the group
// masks (one group: the result as it is).
int rotsum_and_combine(const Ctx& c, const pdq_plan& pl, const Keys& keys, u64* yx, u64* Rx,
                       u64* Y0, u64* Y1, u64* rws, u64* aws, const u64* masks, u64* out,
                       cudaStream_t st, const Stack* sk = nullptr) {
    const long long cts = (long long)ct_elems(c);
    const long long ects = 2LL * (c.L + c.K) * c.N;
    const u64 EN = (u64)(c.L + c.K) * c.N, LN = (u64)c.L * c.N;
    const u32 Q = sk ? sk->Q : 1;
    const u32 G = pl.G * Q;                       // groups of every query
    const KeyTable kt = sk ? sk->table(pl.G) : single_keys(keys.base);
    u64* D = nullptr;
    prof_mark(c, PDQ_STAGE_ROTSUM, st);
    const CtSet y_ext = ct_set(yx, ects);
    for (const auto& [l, r] : rotsum_levels(c, pl)) {
        std::vector<u64> gal(r, 1), koff(r, 0);
        for (u32 j = 1; j < r; ++j) {
            gal[j] = galois_rot(c, (long long)(j * l));
            const u64* kp = keys.find(gal[j]);
            if (!kp) return fail(PDQ_E_KEY, "comp: missing rotation key for Galois element " + std::to_string(gal[j]));
            koff[j] = (u64)(kp - keys.base);
        }
        PDQ_TRY(mod_down_polys(c, yx + EN, 2 * EN, G, Y1, LN, aws, st));
        PDQ_TRY(ks_raise(c, ct_set(Y1, (long long)LN), G, rws, &D, st, 0));
        PDQ_TRY(hoisted_rotations_ext(c, D, y_ext, G, r, gal, keys.base, koff, Rx, st, true, 0, 0,
                                      &kt));
        PDQ_TRY(sum_rotations(c, Rx, G, r, yx, st));
    }
    PDQ_TRY(mod_down_batch(c, yx, G, ct_set(Y0, cts), aws, st));
    prof_mark(c, PDQ_STAGE_COMBINE, st);
    if (pl.G == 1) {                              // one group per query: y is the output
        if (cudaMemcpyAsync(out, Y0, (size_t)cts * Q * sizeof(u64), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return fail(PDQ_E_CUDA, "comp: output copy failed");
        return PDQ_OK;
    }
    return group_combine(c, pl, Y0, masks, out, st, Q);
}

// Comp from the masked ciphertexts (masked != nullptr: [J][4] as pdq_mask
// writes them), or the Answer from the index ciphertexts v_cts and the
// database db (masked == nullptr: the Mask fused with the pack, w holding J
// ciphertexts of scratch).
// (sk: the Answer of sk->Q queries of plan pl together, every step one
// launch over all of them; their index ciphertexts one after the other in
// v_cts, w the same size, outputs in out)
int comp_run(const Ctx& c, const pdq_plan& pl, const u64* masked, const Keys& keys,
             const u64* consts, u64* out, void* ws, size_t ws_bytes, cudaStream_t st,
             const u64* v_cts = nullptr, const u64* db = nullptr, u64* w = nullptr,
             bool prepacked = false, const Stack* sk = nullptr) {
    const u32 Q = sk ? sk->Q : 1;
    if (Q == 0 || Q > kMaxStack) return fail(PDQ_E_PARAM, "answer: 1 to 64 stacked queries");
    if (sk && masked) return fail(PDQ_E_PARAM, "comp: stacked queries take index ciphertexts");
    if (ws_bytes < comp_ws_bytes(c, pl, Q)) return fail(PDQ_E_NOMEM, "comp: workspace too small");
    const long long cts = (long long)ct_elems(c);
    const long long ects = 2LL * (c.L + c.K) * c.N;
    const u32 H = pl.H * Q, B = pl.B, G = pl.G * Q, GI = pl.giants;
    const CompLayout lo = comp_layout(c, pl, Q);
    u64* const base = reinterpret_cast<u64*>(ws);
    u64* U = base + lo.U;
    u64* Rx = base + lo.Rx;
    u64* accx = base + lo.accx;
    u64* acc = base + lo.acc;
    u64* yx = base + lo.yx;
    u64* Y0 = base + lo.Y0;
    u64* Y1 = base + lo.Y1;
    u64* rws = base + lo.rws;
    u64* aws = base + lo.aws;
    const u64* Dg = consts;
    const u64* masks = consts + (u64)pl.hclass * GI * B * (c.L + c.K) * c.N;

    auto key_for = [&](u64 k, const u64** kp) -> int {
        *kp = keys.find(k);
        if (!*kp) return fail(PDQ_E_KEY, "comp: missing rotation key for Galois element " + std::to_string(k));
        return PDQ_OK;
    };
    const CtSet none{};
    u64* D = nullptr;

    // 1. pack: i = 2j + which; which 0: dT_j (+vT_j), which 1: vB_j (+dB_j);
    // in the Answer Rot_col(v_j) once per j and the Mask products after it
    prof_mark(c, PDQ_STAGE_PACK, st);
    if (!masked) {
        // prepacked: the caller ran answer_pack into U already
        if (!prepacked) {
            if (!v_cts || !db || !w) return fail(PDQ_E_PARAM, "answer: null buffer");
            PDQ_TRY(answer_pack(c, keys, v_cts, db, w, U, pl.J * Q, rws, aws, st, sk, pl.J));
        }
    } else {
        CtSet in;  in.base = masked + 2 * cts;  in.outer = 4 * cts;  in.per = 2;  in.inner = -cts;
        CtSet add; add.base = masked;           add.outer = 4 * cts; add.per = 2; add.inner = 3 * cts;
        const u64* kp;
        PDQ_TRY(key_for(2ull * c.N - 1, &kp));
        PDQ_TRY(ks_raise(c, in, H, rws, &D, st));
        PDQ_TRY(ks_apply(c, D, in, H, (u32)(2ull * c.N - 1), kp, ct_set(U, cts), add, aws, st));
    }
    // 2. baby steps in the extended basis, the digits of every u_h raised once
    prof_mark(c, PDQ_STAGE_BABY, st);
    const CtSet u = ct_set(U, cts);
    // 3. diagonal multiply-accumulate over Q u P: the unrotated accumulators
    // (g = 0) start the giant-step sums yx; of the others only c1 is lowered
    // (into acc, [G][GI-1][L][N]), c0 stays in Q u P.  Steps 2 and 3 work
    // prime by prime, so under a rotation budget they alternate on chunks of
    // primes and only one chunk of rotations is held at a time.
    if (B == 1) {
        PDQ_TRY(times_P(c, u, H, ct_set(Rx, (long long)B * ects), true, st));
        prof_mark(c, PDQ_STAGE_MAC, st);
        PDQ_TRY(diag_mac(c, pl, Rx, Dg, yx, accx, st, 0, 0, Q));
    } else {
        PDQ_TRY(ks_raise(c, u, H, rws, &D, st));
        std::vector<u64> koff(B, 0);
        for (u32 a = 1; a < B; ++a) {
            const u64* kp;
            PDQ_TRY(key_for(galois_rot(c, a), &kp));
            koff[a] = (u64)(kp - keys.base);
        }
        const u32 E = c.L + c.K, ec = rotation_chunk(c, pl, Q);
        const KeyTable kth = sk ? sk->table(pl.H) : single_keys(keys.base);
        for (u32 l0 = 0; l0 < E; l0 += ec) {
            const u32 el = std::min(ec, E - l0);
            if (l0 > 0) prof_mark(c, PDQ_STAGE_BABY, st);
            PDQ_TRY(baby_steps_ext(c, D, u, H, B, keys.base, koff, Rx, st, l0, el, &kth));
            prof_mark(c, PDQ_STAGE_MAC, st);
            PDQ_TRY(diag_mac(c, pl, Rx, Dg, yx, accx, st, l0, el, Q));
        }
    }
    prof_mark(c, PDQ_STAGE_ACC_MODDOWN, st);
    const u64 EN = (u64)(c.L + c.K) * c.N, LN = (u64)c.L * c.N;
    if (GI > 1) PDQ_TRY(mod_down_polys(c, accx + EN, 2 * EN, G * (GI - 1), acc, LN, aws, st));
    // 4. giant steps: Rot(acc_g; gB) = (sigma(c0) + A0, A1) over Q u P, the
    // key switch raising the lowered c1, summed into yx.  The lowered c1 of
    // every (g, gamma) are raised in one call, ordered g-major, so that the
    // digits of giant step g are the contiguous run g - 1 of G ciphertexts.
    prof_mark(c, PDQ_STAGE_GIANT, st);
    if (GI > 1) {
        CtSet c1all;
        c1all.base = acc;
        c1all.outer = (long long)LN;                  // g
        c1all.per = G;
        c1all.inner = (long long)(GI - 1) * LN;       // gamma
        PDQ_TRY(ks_raise(c, c1all, G * (GI - 1), rws, &D, st, 0));
    }
    // all giant steps in one launch: term g - 1 rotates accumulator g of
    // every group (c0 over Q u P at accx[gamma][g - 1]) into yx[gamma]
    if (GI > 1) {
        std::vector<u64> gal(GI - 1), koff(GI - 1);
        for (u32 g = 1; g < GI; ++g) {
            gal[g - 1] = galois_rot(c, (long long)g * B);
            const u64* kp;
            PDQ_TRY(key_for(gal[g - 1], &kp));
            koff[g - 1] = (u64)(kp - keys.base);
        }
        const KeyTable ktg = sk ? sk->table(pl.G) : single_keys(keys.base);
        PDQ_TRY(ks_apply_giants(c, D, G, GI - 1, gal.data(), ktg, koff.data(), accx,
                                (u64)ects, (u64)(GI - 1) * ects, yx, (u64)ects, st));
    }
    PDQ_TRY(rotsum_and_combine(c, pl, keys, yx, Rx, Y0, Y1, rws, aws, masks, out, st, sk));
    prof_mark(c, -1, st);
    (void)none;
    return PDQ_OK;
}

// Workspace of the Answer on an unencrypted database, in uint64 elements.
struct PlainDbLayout {
    u64 Rx;     // baby steps of the index ciphertexts over Q u P [J][B], later
                // the rotations of one rotate-and-sum level
    u64 yx;     // giant-step sums over Q u P (from set 0, giant 0), [G]
    u64 accx;   // the other accumulators over Q u P, [G][2 giants - 1]
    u64 acc;    // ... their c1 lowered to Q, [G][2 giants - 1][L][N]
    u64 Y0, Y1; // rotate-and-sum: the output over Q, the lowered c1 of a level
    u64 rws;    // key-switch raise scratch
    u64 aws;    // ModDown scratch
    u64 end;
};

PlainDbLayout plain_db_layout(const Ctx& c, const pdq_plan& pl) {
    const u64 cts = ct_elems(c), ects = 2ull * (c.L + c.K) * c.N;
    const u64 G = pl.G, NA = 2ull * pl.giants - 1;
    const u32 cnt = std::max({pl.J, pl.G, (u32)(G * NA)});
    const u64 scratch = std::max({mod_down_ws(c, pl.G), mod_down_polys_ws(c, (u32)(G * NA)),
                                  apply_ws(c, pl.G)}) / sizeof(u64);
    PlainDbLayout lo;
    lo.Rx = 0;
    lo.yx = lo.Rx + std::max<u64>((u64)pl.J * pl.B, G * 8) * ects;
    lo.accx = lo.yx + G * ects;
    lo.acc = lo.accx + G * NA * ects;
    lo.Y0 = lo.acc + G * NA * (u64)c.L * c.N;
    lo.Y1 = lo.Y0 + G * cts;
    lo.rws = lo.Y1 + G * cts;
    lo.aws = lo.rws + raise_ws(c, cnt) / sizeof(u64);
    lo.end = lo.aws + scratch;
    return lo;
}

// The Answer on an unencrypted database (Sec. 5.2 remark): no Mask; baby
// steps of the J index ciphertexts; per group both diagonal sets and every
// giant step accumulated over Q u P (diag_mac_db); the accumulators other
// than (set 0, giant 0) rotated from their lowered c1 with Galois element
// 3^(gB) (set 0) or 3^(gB) (2N - 1) (set 1: Rot_col folded in), summed into
// yx; then rotate-and-sum and the group masks.
int answer_plain_db_run(const Ctx& c, const pdq_plan& pl, const u64* v_cts, const Keys& keys,
                        const u64* consts, u64* out, void* ws, cudaStream_t st) {
    const long long cts = (long long)ct_elems(c);
    const long long ects = 2LL * (c.L + c.K) * c.N;
    const u64 EN = (u64)(c.L + c.K) * c.N, LN = (u64)c.L * c.N;
    const u32 J = pl.J, B = pl.B, G = pl.G, GI = pl.giants, NA = 2 * GI - 1;
    const PlainDbLayout lo = plain_db_layout(c, pl);
    u64* const base = reinterpret_cast<u64*>(ws);
    u64* Rx = base + lo.Rx;
    u64* yx = base + lo.yx;
    u64* accx = base + lo.accx;
    u64* acc = base + lo.acc;
    u64* rws = base + lo.rws;
    u64* aws = base + lo.aws;
    const u64* Dd = consts;
    const u64* masks = consts + 2ull * J * B * GI * EN;
    u64* D = nullptr;
    // 1. baby steps of the index ciphertexts in the extended basis
    prof_mark(c, PDQ_STAGE_BABY, st);
    const CtSet v = ct_set(v_cts, cts);
    if (B == 1) PDQ_TRY(times_P(c, v, J, ct_set(Rx, (long long)B * ects), true, st));
    else {
        PDQ_TRY(ks_raise(c, v, J, rws, &D, st));
        std::vector<u64> koff(B, 0);
        for (u32 a = 1; a < B; ++a) {
            const u64 k = galois_rot(c, a);
            const u64* kp = keys.find(k);
            if (!kp) return fail(PDQ_E_KEY, "answer_plain_db: missing rotation key for Galois element " + std::to_string(k));
            koff[a] = (u64)(kp - keys.base);
        }
        PDQ_TRY(baby_steps_ext(c, D, v, J, B, keys.base, koff, Rx, st));
    }
    // 2. both diagonal sets, every giant step
    prof_mark(c, PDQ_STAGE_MAC, st);
    PDQ_TRY(diag_mac_db(c, pl, Rx, Dd, yx, accx, st));
    // 3. lower c1 of the accumulators to be rotated, raise them all at once
    // (ordered by (set, giant) first, so each key's digits are one run of G)
    prof_mark(c, PDQ_STAGE_ACC_MODDOWN, st);
    if (NA > 0) PDQ_TRY(mod_down_polys(c, accx + EN, 2 * EN, G * NA, acc, LN, aws, st));
    prof_mark(c, PDQ_STAGE_GIANT, st);
    if (NA > 0) {
        CtSet c1all;
        c1all.base = acc;
        c1all.outer = (long long)LN;
        c1all.per = G;
        c1all.inner = (long long)NA * LN;
        PDQ_TRY(ks_raise(c, c1all, G * NA, rws, &D, st, 0));
    }
    // every (set, giant) term in one launch
    if (NA > 0) {
        std::vector<u64> gal(NA), koff(NA);
        for (u32 i = 0; i < NA; ++i) {
            const u32 sigma = (i + 1) / GI, g = (i + 1) % GI;
            u64 k = galois_rot(c, (long long)g * B);
            if (sigma) k = k * (2ull * c.N - 1) % (2ull * c.N);
            const u64* kp = keys.find(k);
            if (!kp) return fail(PDQ_E_KEY, "answer_plain_db: missing rotation key for Galois element " + std::to_string(k));
            gal[i] = k;
            koff[i] = (u64)(kp - keys.base);
        }
        PDQ_TRY(ks_apply_giants(c, D, G, NA, gal.data(), single_keys(keys.base), koff.data(),
                                accx, (u64)ects, (u64)NA * ects, yx, (u64)ects, st));
    }
    // 4. rotate-and-sum and group masks
    PDQ_TRY(rotsum_and_combine(c, pl, keys, yx, Rx, base + lo.Y0, base + lo.Y1, rws, aws, masks,
                               out, st));
    prof_mark(c, -1, st);
    return PDQ_OK;
}

}  // namespace

}  // namespace pdq

using namespace pdq;

#define PDQ_CHECK_CTX(ctx) \
    if (!(ctx)) return fail(PDQ_E_PARAM, "null context")

extern "C" {

int pdq_ntt_forward(const pdq_ctx* ctx, uint64_t* data, uint32_t count, uint32_t nlimbs,
                    uint32_t limb0, uint64_t stride, void* stream) {
    PDQ_CHECK_CTX(ctx);
    if (count && !data) return fail(PDQ_E_PARAM, "ntt_forward: null buffer");
    return ntt_forward(C(ctx), data, count, nlimbs, limb0, stride, (cudaStream_t)stream);
}

int pdq_ntt_inverse(const pdq_ctx* ctx, uint64_t* data, uint32_t count, uint32_t nlimbs,
                    uint32_t limb0, uint64_t stride, void* stream) {
    PDQ_CHECK_CTX(ctx);
    if (count && !data) return fail(PDQ_E_PARAM, "ntt_inverse: null buffer");
    return ntt_inverse(C(ctx), data, count, nlimbs, limb0, stride, (cudaStream_t)stream);
}

int pdq_encode(const pdq_ctx* ctx, const uint32_t* slots, uint32_t count, uint32_t nlimbs,
               uint64_t* pt_out, void* stream) {
    PDQ_CHECK_CTX(ctx);
    if (count && (!slots || !pt_out)) return fail(PDQ_E_PARAM, "encode: null buffer");
    return encode_slots(C(ctx), slots, count, nlimbs, pt_out, (cudaStream_t)stream);
}

int pdq_secret_prepare(const pdq_ctx* ctx, const int8_t* s, uint64_t* sk_out, void* stream) {
    PDQ_CHECK_CTX(ctx);
    if (!s || !sk_out) return fail(PDQ_E_PARAM, "secret_prepare: null buffer");
    return secret_prepare(C(ctx), s, sk_out, (cudaStream_t)stream);
}

int pdq_encrypt(const pdq_ctx* ctx, const uint64_t* sk, const uint32_t* slots, uint32_t count,
                const uint64_t* a, const int32_t* e, uint64_t* ct_out, void* stream) {
    PDQ_CHECK_CTX(ctx);
    if (count && (!sk || !slots || !a || !e || !ct_out))
        return fail(PDQ_E_PARAM, "encrypt: null buffer");
    return encrypt(C(ctx), sk, slots, count, a, e, ct_out, (cudaStream_t)stream);
}

int pdq_rotkey_gen(const pdq_ctx* ctx, const uint64_t* sk, uint64_t galois, const uint64_t* a,
                   const int32_t* e, uint64_t* key_out, void* stream) {
    PDQ_CHECK_CTX(ctx);
    if (!sk || !a || !e || !key_out) return fail(PDQ_E_PARAM, "rotkey_gen: null buffer");
    return rotkey_gen(C(ctx), sk, galois, a, e, key_out, (cudaStream_t)stream);
}

size_t pdq_decrypt_workspace_bytes(const pdq_ctx* ctx, uint32_t count) {
    return ctx ? decrypt_ws(C(ctx), count) : 0;
}

int pdq_decrypt(const pdq_ctx* ctx, const uint64_t* sk, const uint64_t* ct, uint32_t count,
                uint32_t* slots_out, void* ws, size_t ws_bytes, void* stream) {
    PDQ_CHECK_CTX(ctx);
    if (ws_bytes < decrypt_ws(C(ctx), count)) return fail(PDQ_E_NOMEM, "decrypt: workspace too small");
    if (count && (!sk || !ct || !slots_out || !ws)) return fail(PDQ_E_PARAM, "decrypt: null buffer");
    return decrypt(C(ctx), sk, ct, count, slots_out, reinterpret_cast<u64*>(ws), (cudaStream_t)stream);
}

size_t pdq_rotate_workspace_bytes(const pdq_ctx* ctx, uint32_t count) {
    return ctx ? raise_ws(C(ctx), count) + apply_ws(C(ctx), count) : 0;
}

int pdq_rotate(const pdq_ctx* ctx, const uint64_t* ct_in, uint32_t count, uint64_t galois,
               const uint64_t* key, uint64_t* ct_out, void* ws, size_t ws_bytes, void* stream) {
    PDQ_CHECK_CTX(ctx);
    const Ctx& c = C(ctx);
    if (count == 0) return PDQ_OK;
    if (!ct_in || !key || !ct_out || !ws) return fail(PDQ_E_PARAM, "rotate: null buffer");
    if (galois % 2 == 0 || galois >= 2ull * c.N) return fail(PDQ_E_PARAM, "rotate: bad Galois element");
    if (ws_bytes < pdq_rotate_workspace_bytes(ctx, count)) return fail(PDQ_E_NOMEM, "rotate: workspace too small");
    const long long cts = (long long)ct_elems(c);
    u64* rws = reinterpret_cast<u64*>(ws);
    u64* aws = rws + raise_ws(c, count) / sizeof(u64);
    u64* D = nullptr;
    const CtSet in = ct_set(ct_in, cts);
    PDQ_TRY(ks_raise(c, in, count, rws, &D, (cudaStream_t)stream));
    return ks_apply(c, D, in, count, (u32)galois, key, ct_set(ct_out, cts), CtSet{}, aws,
                    (cudaStream_t)stream);
}

size_t pdq_mod_switch_workspace_bytes(const pdq_ctx* from, uint32_t count) {
    return from ? mod_switch_ws(C(from), count) : 0;
}

int pdq_mod_switch(const pdq_ctx* from, const pdq_ctx* to, const uint64_t* cts, uint32_t count,
                   uint64_t* out, void* ws, size_t ws_bytes, void* stream) {
    if (!from || !to) return fail(PDQ_E_PARAM, "mod_switch: null context");
    const Ctx& a = C(from);
    const Ctx& b = C(to);
    if (a.N != b.N || a.t != b.t || b.L >= a.L)
        return fail(PDQ_E_PARAM, "mod_switch: the target needs the same ring and fewer primes");
    for (u32 i = 0; i < b.L; ++i)
        if (a.mods[i] != b.mods[i])
            return fail(PDQ_E_PARAM, "mod_switch: the target's primes must be a prefix of the source's");
    if (count == 0) return PDQ_OK;
    if (!cts || !out || !ws) return fail(PDQ_E_PARAM, "mod_switch: null buffer");
    if (ws_bytes < mod_switch_ws(a, count)) return fail(PDQ_E_NOMEM, "mod_switch: workspace too small");
    return mod_switch(a, b.L, cts, count, out, reinterpret_cast<u64*>(ws), (cudaStream_t)stream);
}

int pdq_ctx_set_schedule(pdq_ctx* ctx, const pdq_schedule* sched) {
    PDQ_CHECK_CTX(ctx);
    if (!sched) return fail(PDQ_E_PARAM, "schedule: null");
    Ctx& c = *reinterpret_cast<Ctx*>(ctx);
    const u32 rb = sched->ntt_row_bits, mt = sched->mac_tiles, bc = sched->mac_bc;
    if (rb && (rb < 7 || rb > 11 || rb >= c.log_n))
        return fail(PDQ_E_PARAM, "schedule: row levels must be 7..11 and below log N");
    if (mt && (mt > 8 || (mt & (mt - 1)))) return fail(PDQ_E_PARAM, "schedule: 1, 2, 4 or 8 tiles");
    if (bc && (bc > 16 || (bc & (bc - 1)))) return fail(PDQ_E_PARAM, "schedule: 1..16 baby steps, a power of two");
    if (sched->ntt_chunk && (sched->ntt_chunk < 64 || sched->ntt_chunk > (1u << 20)))
        return fail(PDQ_E_PARAM, "schedule: 64..2^20 polynomials per transform launch");
    c.sched = *sched;
    return PDQ_OK;
}

int pdq_ctx_get_schedule(const pdq_ctx* ctx, pdq_schedule* sched) {
    PDQ_CHECK_CTX(ctx);
    if (!sched) return fail(PDQ_E_PARAM, "schedule: null");
    *sched = C(ctx).sched;
    return PDQ_OK;
}

int pdq_ctx_set_rotation_budget(pdq_ctx* ctx, uint64_t bytes) {
    if (!ctx) return fail(PDQ_E_PARAM, "null context");
    reinterpret_cast<Ctx*>(ctx)->rotation_budget = bytes;
    return PDQ_OK;
}

int pdq_plan_make(const pdq_ctx* ctx, uint64_t n, uint32_t s, uint32_t B, pdq_plan* plan) {
    PDQ_CHECK_CTX(ctx);
    if (!plan) return fail(PDQ_E_PARAM, "null plan");
    return plan_make(C(ctx), n, s, B, plan);
}

int pdq_plan_make_client(uint64_t t, uint32_t log_n, uint64_t n, uint32_t s, uint32_t B,
                         pdq_plan* plan) {
    if (!plan) return fail(PDQ_E_PARAM, "null plan");
    Ctx c;
    PDQ_TRY(host_ring(t, log_n, &c));
    return plan_make(c, n, s, B, plan);
}

int pdq_plan_galois(const pdq_ctx* ctx, const pdq_plan* plan, uint64_t* out, uint32_t cap,
                    uint32_t* count) {
    PDQ_CHECK_CTX(ctx);
    if (!valid_plan(C(ctx), plan) || !count) return fail(PDQ_E_PARAM, "plan_galois: invalid plan");
    auto ks = plan_galois(C(ctx), *plan);
    *count = (uint32_t)ks.size();
    if (out) {
        if (cap < ks.size()) return fail(PDQ_E_NOMEM, "plan_galois: output too small");
        std::copy(ks.begin(), ks.end(), out);
    }
    return PDQ_OK;
}

int pdq_plan_galois_client(uint64_t t, uint32_t log_n, const pdq_plan* plan, uint64_t* out,
                           uint32_t cap, uint32_t* count) {
    Ctx c;
    PDQ_TRY(host_ring(t, log_n, &c));
    if (!valid_plan(c, plan) || !count) return fail(PDQ_E_PARAM, "plan_galois: invalid plan");
    auto ks = plan_galois(c, *plan);
    *count = (uint32_t)ks.size();
    if (out) {
        if (cap < ks.size()) return fail(PDQ_E_NOMEM, "plan_galois: output too small");
        std::copy(ks.begin(), ks.end(), out);
    }
    return PDQ_OK;
}

size_t pdq_plan_constants_bytes(const pdq_ctx* ctx, const pdq_plan* plan) {
    if (!ctx || !valid_plan(C(ctx), plan)) return 0;
    const Ctx& c = C(ctx);
    const u64 diag = (u64)plan->hclass * plan->giants * plan->B * (c.L + c.K);
    const u64 masks = plan->G > 1 ? (u64)plan->per_out * c.L : 0;
    return (diag + masks) * c.N * sizeof(u64);
}

int pdq_plan_constants_build(const pdq_ctx* ctx, const pdq_plan* plan, uint64_t* out,
                             void* stream) {
    PDQ_CHECK_CTX(ctx);
    const Ctx& c = C(ctx);
    if (!valid_plan(c, plan)) return fail(PDQ_E_PARAM, "plan_constants_build: invalid plan");
    if (!out) return fail(PDQ_E_PARAM, "plan_constants_build: null buffer");
    PDQ_TRY(build_diagonals(c, *plan, out, (cudaStream_t)stream));
    if (plan->G > 1) {
        u64* masks = out + (u64)plan->hclass * plan->giants * plan->B * (c.L + c.K) * c.N;
        PDQ_TRY(build_group_masks(c, *plan, masks, (cudaStream_t)stream));
    }
    return PDQ_OK;
}

size_t pdq_db_bytes(const pdq_ctx* ctx, uint64_t n) {
    if (!ctx) return 0;
    const Ctx& c = C(ctx);
    const u64 J = (n + c.N - 1) / c.N;
    return J * ct_elems(c) * sizeof(u64);
}

int pdq_db_encode(const pdq_ctx* ctx, const uint32_t* values, uint64_t n, uint64_t* db_out,
                  void* stream) {
    PDQ_CHECK_CTX(ctx);
    const Ctx& c = C(ctx);
    if (n == 0) return fail(PDQ_E_PARAM, "db_encode: empty database");
    if (!values || !db_out) return fail(PDQ_E_PARAM, "db_encode: null buffer");
    const u64 J = (n + c.N - 1) / c.N;
    return build_db(c, values, n, (u32)J, db_out, (cudaStream_t)stream);
}

size_t pdq_db_plain_bytes(const pdq_ctx* ctx, uint64_t n) {
    if (!ctx) return 0;
    const Ctx& c = C(ctx);
    return (n + c.N - 1) / c.N * (u64)c.L * c.N * sizeof(u64);
}

int pdq_db_encode_plain(const pdq_ctx* ctx, const uint32_t* values, uint64_t n, uint64_t* db_out,
                        void* stream) {
    PDQ_CHECK_CTX(ctx);
    const Ctx& c = C(ctx);
    if (n == 0) return fail(PDQ_E_PARAM, "db_encode_plain: empty database");
    if (!values || !db_out) return fail(PDQ_E_PARAM, "db_encode_plain: null buffer");
    return build_db_plain(c, values, n, (u32)((n + c.N - 1) / c.N), db_out, (cudaStream_t)stream);
}

int pdq_mask_literal(const pdq_ctx* ctx, const pdq_plan* plan, const uint64_t* v_cts,
                     const uint64_t* db_plain, uint64_t* masked_out, void* stream) {
    PDQ_CHECK_CTX(ctx);
    if (!valid_plan(C(ctx), plan)) return fail(PDQ_E_PARAM, "mask_literal: invalid plan");
    if (!v_cts || !db_plain || !masked_out) return fail(PDQ_E_PARAM, "mask_literal: null buffer");
    return mask_literal(C(ctx), plan->J, v_cts, db_plain, masked_out, (cudaStream_t)stream);
}

int pdq_mask(const pdq_ctx* ctx, const pdq_plan* plan, const uint64_t* v_cts, const uint64_t* db,
             uint64_t* masked_out, void* stream) {
    PDQ_CHECK_CTX(ctx);
    if (!valid_plan(C(ctx), plan)) return fail(PDQ_E_PARAM, "mask: invalid plan");
    if (!v_cts || !db || !masked_out) return fail(PDQ_E_PARAM, "mask: null buffer");
    return mask(C(ctx), plan->J, v_cts, db, masked_out, (cudaStream_t)stream);
}

size_t pdq_comp_workspace_bytes(const pdq_ctx* ctx, const pdq_plan* plan) {
    if (!ctx || !valid_plan(C(ctx), plan)) return 0;
    return comp_ws_bytes(C(ctx), *plan);
}

int pdq_comp(const pdq_ctx* ctx, const pdq_plan* plan, const uint64_t* masked,
             const uint64_t* keys, const uint64_t* galois, uint32_t nkeys,
             const uint64_t* consts, uint64_t* out, void* ws, size_t ws_bytes, void* stream) {
    PDQ_CHECK_CTX(ctx);
    const Ctx& c = C(ctx);
    if (!valid_plan(c, plan)) return fail(PDQ_E_PARAM, "comp: invalid plan");
    if (!masked || !keys || !galois || !consts || !out || !ws) return fail(PDQ_E_PARAM, "comp: null buffer");
    Keys k{keys, galois, nkeys, (u64)c.ndigits * 2 * (c.L + c.K) * c.N};
    return comp_run(c, *plan, masked, k, consts, out, ws, ws_bytes, (cudaStream_t)stream);
}

size_t pdq_answer_workspace_bytes(const pdq_ctx* ctx, const pdq_plan* plan) {
    if (!ctx || !valid_plan(C(ctx), plan)) return 0;
    const Ctx& c = C(ctx);
    return (size_t)plan->J * ct_elems(c) * sizeof(u64) + comp_ws_bytes(c, *plan);
}

int pdq_answer(const pdq_ctx* ctx, const pdq_plan* plan, const uint64_t* v_cts,
               const uint64_t* db, const uint64_t* keys, const uint64_t* galois,
               uint32_t nkeys, const uint64_t* consts, uint64_t* out, void* ws,
               size_t ws_bytes, void* stream) {
    PDQ_CHECK_CTX(ctx);
    const Ctx& c = C(ctx);
    if (!valid_plan(c, plan)) return fail(PDQ_E_PARAM, "answer: invalid plan");
    if (ws_bytes < pdq_answer_workspace_bytes(ctx, plan)) return fail(PDQ_E_NOMEM, "answer: workspace too small");
    if (!v_cts || !db || !keys || !galois || !consts || !out || !ws)
        return fail(PDQ_E_PARAM, "answer: null buffer");
    u64* w = reinterpret_cast<u64*>(ws);                  // Rot_col(v_j), J ciphertexts
    const size_t wbytes = (size_t)plan->J * ct_elems(c) * sizeof(u64);
    Keys k{keys, galois, nkeys, (u64)c.ndigits * 2 * (c.L + c.K) * c.N};
    return comp_run(c, *plan, nullptr, k, consts, out, reinterpret_cast<char*>(ws) + wbytes,
                    ws_bytes - wbytes, (cudaStream_t)stream, v_cts, db, w);
}

size_t pdq_answer_stacked_workspace_bytes(const pdq_ctx* ctx, const pdq_plan* plan, uint32_t Q) {
    if (!ctx || !plan || Q == 0 || Q > kMaxStack) return 0;
    const Ctx& c = C(ctx);
    return (size_t)plan->J * Q * ct_elems(c) * sizeof(u64) + comp_ws_bytes(c, *plan, Q);
}

int pdq_answer_stacked(const pdq_ctx* ctx, const pdq_plan* plan, uint32_t Q,
                       const uint64_t* v_cts, const uint64_t* db,
                       const uint64_t* const* keys, const uint64_t* galois, uint32_t nkeys,
                       const uint64_t* consts, uint64_t* out, void* ws, size_t ws_bytes,
                       void* stream) {
    PDQ_CHECK_CTX(ctx);
    const Ctx& c = C(ctx);
    if (Q == 0 || Q > kMaxStack) return fail(PDQ_E_PARAM, "answer_stacked: 1 to 64 queries");
    if (!valid_plan(c, plan) || plan->plain_db || plan->ring_ratio > 1)
        return fail(PDQ_E_PARAM, "answer_stacked: invalid plan");
    if (!v_cts || !db || !keys || !galois || !consts || !out || !ws)
        return fail(PDQ_E_PARAM, "answer_stacked: null buffer");
    Stack sk;
    sk.Q = Q;
    for (u32 q = 0; q < Q; ++q) {
        if (!keys[q]) return fail(PDQ_E_PARAM, "answer_stacked: null key set");
        sk.keys[q] = keys[q];
    }
    if (ws_bytes < pdq_answer_stacked_workspace_bytes(ctx, plan, Q))
        return fail(PDQ_E_NOMEM, "answer_stacked: workspace too small");
    u64* w = reinterpret_cast<u64*>(ws);              // Rot_col(v_j), Q J ciphertexts
    const size_t wbytes = (size_t)plan->J * Q * ct_elems(c) * sizeof(u64);
    Keys k{keys[0], galois, nkeys, (u64)c.ndigits * 2 * (c.L + c.K) * c.N};
    return comp_run(c, *plan, nullptr, k, consts, out, reinterpret_cast<char*>(ws) + wbytes,
                    ws_bytes - wbytes, (cudaStream_t)stream, v_cts, db, w, false, &sk);
}

size_t pdq_answer_host_workspace_bytes(const pdq_ctx* ctx, const pdq_plan* plan) {
    if (!ctx || !valid_plan(C(ctx), plan)) return 0;
    const Ctx& c = C(ctx);
    return ((size_t)plan->J + plan->n_out) * ct_elems(c) * sizeof(u64) +
           pdq_answer_workspace_bytes(ctx, plan);
}

int pdq_answer_host(const pdq_ctx* ctx, const pdq_plan* plan, const uint64_t* v_host,
                    const uint64_t* db, const uint64_t* keys, const uint64_t* galois,
                    uint32_t nkeys, const uint64_t* consts, uint64_t* out_host, void* ws,
                    size_t ws_bytes, void* stream) {
    PDQ_CHECK_CTX(ctx);
    const Ctx& c = C(ctx);
    if (!valid_plan(c, plan)) return fail(PDQ_E_PARAM, "answer_host: invalid plan");
    if (!v_host || !out_host) return fail(PDQ_E_PARAM, "answer_host: null host buffer");
    if (!db || !keys || !galois || !consts || !ws) return fail(PDQ_E_PARAM, "answer_host: null buffer");
    if (ws_bytes < pdq_answer_host_workspace_bytes(ctx, plan)) return fail(PDQ_E_NOMEM, "answer_host: workspace too small");
    cudaStream_t st = (cudaStream_t)stream;
    const u64 cts = ct_elems(c);
    const u32 J = plan->J;
    // workspace: v [J] | answer [n_out] | w = Rot_col(v) [J] | Comp
    u64* v = reinterpret_cast<u64*>(ws);
    u64* o = v + (u64)J * cts;
    u64* w = o + (u64)plan->n_out * cts;
    u64* cws = w + (u64)J * cts;
    const size_t cws_bytes = ws_bytes - ((size_t)2 * J + plan->n_out) * cts * sizeof(u64);
    const CompLayout lo = comp_layout(c, *plan);
    u64* U = cws + lo.U;
    Keys k{keys, galois, nkeys, (u64)c.ndigits * 2 * (c.L + c.K) * c.N};

    // The index ciphertexts go up in (at most) four runs on a second stream;
    // each run is transformed and packed on `stream` while the next one is
    // copied.  The copies start after the work already queued on `stream`.
    struct Runs {
        cudaStream_t cs = nullptr;
        std::vector<cudaEvent_t> ev;
        ~Runs() {
            if (cs) cudaStreamSynchronize(cs);   // no copy outlives the call
            for (cudaEvent_t e : ev) cudaEventDestroy(e);
            if (cs) cudaStreamDestroy(cs);
        }
    } runs;
    const u32 per = (J + 3) / 4, nrun = (J + per - 1) / per;
    if (cudaStreamCreateWithFlags(&runs.cs, cudaStreamNonBlocking) != cudaSuccess) {
        runs.cs = nullptr;
        return cuda_check("answer_host: copy stream");
    }
    for (u32 r = 0; r <= nrun; ++r) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
            return cuda_check("answer_host: events");
        runs.ev.push_back(e);
    }
    if (cudaEventRecord(runs.ev[nrun], st) != cudaSuccess ||
        cudaStreamWaitEvent(runs.cs, runs.ev[nrun], 0) != cudaSuccess)
        return cuda_check("answer_host: stream order");
    for (u32 r = 0; r < nrun; ++r) {
        const u64 j0 = (u64)r * per, jn = std::min<u64>(per, J - j0);
        if (cudaMemcpyAsync(v + j0 * cts, v_host + j0 * cts, jn * cts * sizeof(u64),
                            cudaMemcpyHostToDevice, runs.cs) != cudaSuccess ||
            cudaEventRecord(runs.ev[r], runs.cs) != cudaSuccess)
            return fail(PDQ_E_CUDA, "answer_host: upload failed");
    }
    prof_mark(c, PDQ_STAGE_PACK, st);
    for (u32 r = 0; r < nrun; ++r) {
        const u64 j0 = (u64)r * per, jn = std::min<u64>(per, J - j0);
        if (cudaStreamWaitEvent(st, runs.ev[r], 0) != cudaSuccess) return cuda_check("answer_host: wait");
        PDQ_TRY(ntt_forward(c, v + j0 * cts, 2 * (u32)jn, c.L, 0, (u64)c.L * c.N, st));
        PDQ_TRY(answer_pack(c, k, v + j0 * cts, db + j0 * cts, w + j0 * cts, U + 2 * j0 * cts,
                            (u32)jn, cws + lo.rws, cws + lo.aws, st));
    }
    PDQ_TRY(comp_run(c, *plan, nullptr, k, consts, o, cws, cws_bytes, st, v, db, w, true));
    PDQ_TRY(ntt_inverse(c, o, 2 * plan->n_out, c.L, 0, (u64)c.L * c.N, st));
    const size_t obytes = (size_t)plan->n_out * cts * sizeof(u64);
    if (cudaMemcpyAsync(out_host, o, obytes, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return fail(PDQ_E_CUDA, "answer_host: download failed");
    if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_check("answer_host");
    return PDQ_OK;
}

int pdq_plan_make_plain_db(const pdq_ctx* ctx, uint64_t n, uint32_t s, uint32_t B,
                           pdq_plan* plan) {
    PDQ_CHECK_CTX(ctx);
    if (!plan) return fail(PDQ_E_PARAM, "null plan");
    return plan_make_plain_db(C(ctx), n, s, B, plan);
}

size_t pdq_db_diagonals_bytes(const pdq_ctx* ctx, const pdq_plan* plan) {
    if (!ctx || !valid_plan(C(ctx), plan) || !plan->plain_db) return 0;
    const Ctx& c = C(ctx);
    return ((size_t)2 * plan->J * plan->B * plan->giants * (c.L + c.K) * c.N +
            (size_t)plan->per_out * c.L * c.N) * sizeof(u64);
}

int pdq_db_diagonals_build(const pdq_ctx* ctx, const pdq_plan* plan, const uint32_t* values,
                           uint64_t* out, void* stream) {
    PDQ_CHECK_CTX(ctx);
    const Ctx& c = C(ctx);
    if (!valid_plan(c, plan) || !plan->plain_db) return fail(PDQ_E_PARAM, "db_diagonals_build: invalid plan");
    if (!values || !out) return fail(PDQ_E_PARAM, "db_diagonals_build: null buffer");
    cudaStream_t st = (cudaStream_t)stream;
    PDQ_TRY(build_db_diagonals(c, *plan, values, out, st));
    if (plan->G > 1)
        PDQ_TRY(build_group_masks(c, *plan,
                                  out + (u64)2 * plan->J * plan->B * plan->giants * (c.L + c.K) * c.N,
                                  st));
    return PDQ_OK;
}

size_t pdq_answer_plain_db_workspace_bytes(const pdq_ctx* ctx, const pdq_plan* plan) {
    if (!ctx || !valid_plan(C(ctx), plan) || !plan->plain_db) return 0;
    return plain_db_layout(C(ctx), *plan).end * sizeof(u64);
}

int pdq_answer_plain_db(const pdq_ctx* ctx, const pdq_plan* plan, const uint64_t* v_cts,
                        const uint64_t* keys, const uint64_t* galois, uint32_t nkeys,
                        const uint64_t* consts, uint64_t* out, void* ws, size_t ws_bytes,
                        void* stream) {
    PDQ_CHECK_CTX(ctx);
    const Ctx& c = C(ctx);
    if (!valid_plan(c, plan) || !plan->plain_db) return fail(PDQ_E_PARAM, "answer_plain_db: invalid plan");
    if (!v_cts || !keys || !galois || !consts || !out || !ws)
        return fail(PDQ_E_PARAM, "answer_plain_db: null buffer");
    if (ws_bytes < plain_db_layout(c, *plan).end * sizeof(u64))
        return fail(PDQ_E_NOMEM, "answer_plain_db: workspace too small");
    const Keys k{keys, galois, nkeys, (u64)c.ndigits * 2 * (c.L + c.K) * c.N};
    return answer_plain_db_run(c, *plan, v_cts, k, consts, out, ws, (cudaStream_t)stream);
}

}  // extern "C"
