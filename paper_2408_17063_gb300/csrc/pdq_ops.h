// Launchers of the element-wise kernels (ops.cu), used by the Comp
// orchestration (comp.cu) and the C ABI.
#pragma once

#include "pdq_internal.h"

namespace pdq {

// A strided set of ciphertexts: ciphertext i starts at
// base + (i / per) * outer + (i % per) * inner  (uint64 elements).
struct CtSet {
    const u64* base = nullptr;
    long long outer = 0;
    u32 per = 1;
    long long inner = 0;

    __host__ __device__ __forceinline__ u64* at(u64 i) const {
        // ciphertext counts fit in 32 bits; per is 1 or 2 on the hot paths
        const u32 j = (u32)i;
        u32 hi, lo;
        if (per == 1) { hi = j; lo = 0; }
        else if (per == 2) { hi = j >> 1; lo = j & 1; }
        else { hi = j / per; lo = j - hi * per; }
        return const_cast<u64*>(base) + (long long)hi * outer + (long long)lo * inner;
    }
};

inline CtSet ct_set(const u64* base, long long stride) {
    CtSet s;
    s.base = base;
    s.outer = stride;
    return s;
}

// Queries answered together in one launch per step (at most kMaxStack).
constexpr u32 kMaxStack = 64;

// Key sets of the queries of a launch: the key of ciphertext ct of the
// launch is read from p[ct / per] plus the key's offset inside a set (every
// set holds the same Galois elements in the same order).  One query: p[0]
// and per = ~0u.
struct KeyTable {
    const u64* p[kMaxStack];
    u32 per;
    u64 magic;      // ceil(2^32 / per): ct / per = (ct magic) >> 32 for ct, per < 2^16
    // key set of ciphertext ct of the launch (a multiply instead of a
    // division, which would cost the kernels registers)
    __host__ __device__ __forceinline__ const u64* of(u32 ct) const {
        return p[(u32)(((u64)ct * magic) >> 32)];
    }
};

inline KeyTable key_table(u32 per) {
    KeyTable t{};
    t.per = per;
    t.magic = ((1ull << 32) + per - 1) / per;
    return t;
}

inline KeyTable single_keys(const u64* base) {
    KeyTable t = key_table(~0u);       // (ct magic) >> 32 = 0 for ct < 2^31
    t.p[0] = base;
    return t;
}

// Q queries with one plan answered together: query q's ciphertexts follow
// query q-1's in every buffer of the Answer (index ciphertexts, half-blocks,
// groups, outputs), its key set at keys[q].
struct Stack {
    u32 Q = 1;
    const u64* keys[kMaxStack] = {};
    // the table for a launch over `per` ciphertexts of each query
    KeyTable table(u32 per) const {
        KeyTable t = key_table(Q == 1 ? ~0u : per);
        for (u32 q = 0; q < Q && q < kMaxStack; ++q) t.p[q] = keys[q];
        return t;
    }
};

struct DigitBounds {
    u32 lo[32];
    u32 hi[32];
};

int encode_finish(const Ctx& c, u64* out, u32 count, u32 nlimbs, cudaStream_t st);
int encode_slots(const Ctx& c, const u32* slots, u32 count, u32 nlimbs, u64* out, cudaStream_t st);
int build_diagonals(const Ctx& c, const pdq_plan& pl, u64* out, cudaStream_t st);
int build_group_masks(const Ctx& c, const pdq_plan& pl, u64* out, cudaStream_t st);
int build_db(const Ctx& c, const u32* values, u64 n, u32 J, u64* out, cudaStream_t st);
int secret_prepare(const Ctx& c, const int8_t* s, u64* out, cudaStream_t st);
int encrypt(const Ctx& c, const u64* sk, const u32* slots, u32 count, const u64* a,
            const int32_t* e, u64* ct, cudaStream_t st);
int rotkey_gen(const Ctx& c, const u64* sk, u64 galois, const u64* a, const int32_t* e, u64* key,
               cudaStream_t st);
// key-switching key from sigma_galois(s_from) to s (rotation keys: s_from = s)
int keygen(const Ctx& c, const u64* sk, const u64* sk_from, u64 galois, const u64* a,
           const int32_t* e, u64* key, cudaStream_t st);
// key-switching key from s (big's ring) to s_small(X^R) (ring switching)
int ring_switch_keygen(const Ctx& big, const u64* sk, const int8_t* s_small, u32 R, const u64* a,
                       const int32_t* e, u64* key, cudaStream_t st);
// part r of coefficient-form ciphertext i (big ring, [2][L][R N']) into
// out at index (i / group) group R + r group + i mod group ([2][L][N'])
int ring_split(const Ctx& small, const u64* in, u32 count, u32 R, u32 group, u64* out,
               cudaStream_t st);
size_t decrypt_ws(const Ctx& c, u32 count);
int decrypt(const Ctx& c, const u64* sk, const u64* ct, u32 count, u32* slots, u64* ws,
            cudaStream_t st);
int mask(const Ctx& c, u32 J, const u64* v, const u64* db, u64* out, cudaStream_t st);
// the remark's order: DB_j plaintexts without row masks ([J][L][N]), then
// out[j] = (v.[1;0], v.[0;1], (v.DB).[1;0], (v.DB).[0;1])
int build_db_plain(const Ctx& c, const u32* values, u64 n, u32 J, u64* out, cudaStream_t st);
int mask_literal(const Ctx& c, u32 J, const u64* v, const u64* dbp, u64* out, cudaStream_t st);
// u[2j] = v_j.[1;0] + w_j.sigma_col(DB_j.[1;0]), u[2j+1] = w_j.[1;0] + v_j.(DB_j.[0;1])
// with w_j = Rot_col(v_j): the packed u of Comp straight from the index
// ciphertexts (u [2J][2][L][N])
// (Jq > 0: the J index ciphertexts are queries of Jq each, all masked by
// the same Jq database plaintexts)
int mask_pack(const Ctx& c, u32 J, const u64* v, const u64* w, const u64* db, u64* u,
              cudaStream_t st, u32 Jq = 0);

// the Answer on an unencrypted database: diagonals [J][2][B][L+K][N][giants]
// (split layout) and their multiply-accumulate into y0 ([G][2][L+K][N], set 0
// giant 0) and acc ([G][2 giants - 1][2][L+K][N], the other (set, giant))
int build_db_diagonals(const Ctx& c, const pdq_plan& pl, const u32* values, u64* out,
                       cudaStream_t st);
int diag_mac_db(const Ctx& c, const pdq_plan& pl, const u64* R, const u64* Dd, u64* y0, u64* acc,
                cudaStream_t st);

// plans: valid_plan recomputes a plan (any kind) and compares it
bool valid_plan(const Ctx& c, const pdq_plan* pl);
int plan_make_switched(const Ctx& c, u32 big_log_n, u64 n, u32 s, u32 B, pdq_plan* pl);
inline u32 log2_exact(u32 x) {
    u32 r = 0;
    while ((1u << r) < x) ++r;
    return r;
}

// Hybrid key switching, split so that the raised digits of c1 can be shared
// by every rotation of the same ciphertexts (hoisting):
//   ks_raise: D[i][beta] = raise of digit beta of c1(in[i]) to Q u P (NTT form)
//   ks_apply: out[i] = sigma_k(c0) + ModDown(sum_beta sigma_k(D[i][beta]) * key[beta][0]),
//             ModDown(sum_beta sigma_k(D[i][beta]) * key[beta][1])   (+ add[i])
size_t raise_ws(const Ctx& c, u32 cnt);   // holds D (returned) and a scratch copy of c1
size_t apply_ws(const Ctx& c, u32 cnt);
// (c1 of ciphertext i at in.at(i) + c1_off; default L N, c1 of a ciphertext
// over Q; 0 raises a set of polynomials)
int ks_raise(const Ctx& c, CtSet in, u32 cnt, u64* ws, u64** D_out, cudaStream_t st,
             u64 c1_off = ~0ull);
// (kt: ciphertexts of several queries; `key` points into query 0's set and
// query q's key is at the same offset in kt->p[q])
int ks_apply(const Ctx& c, const u64* D, CtSet in, u32 cnt, u32 galois, const u64* key,
             CtSet out, CtSet add, u64* ws, cudaStream_t st, const KeyTable* kt = nullptr);

// Extended-basis rotation (no ModDown): out (+)= (P sigma(c0) + A0, A1) over
// Q u P, out ciphertexts [2][L+K][N]
// (`split`: residues stored as v0 | v1 << 32, v = v0 + v1 2^30, the operand
// layout of diag_mac; not combinable with `accumulate`)
// (c0_ext: c0src holds ciphertexts over Q u P and sigma(c0) joins on every
// limb as it is, instead of P sigma(c0) of a c0 over Q)
int ks_apply_ext(const Ctx& c, const u64* D, CtSet c0src, u32 cnt, u32 galois, const u64* key,
                 CtSet out, bool accumulate, bool split, cudaStream_t st, bool c0_ext = false,
                 const KeyTable* kt = nullptr);
constexpr u32 kMaxGiantTerms = 64;

// Every giant step in one launch, over Q u P: for ciphertext ct < cnt,
//   out[ct] += sum_{i < terms} Rot_i(c0_i[ct], c1_i[ct])
// where Rot_i is the extended-basis rotation with Galois element galois[i]
// and the key at keys + key_offsets[i], the raised digits of c1_i[ct] are
// D[i][ct] ([terms][cnt][ndigits][L+K][N], as ks_raise writes them for the
// c1 ordered term-major) and c0_i[ct] (over Q u P) starts at
// c0 + i c0_term + ct c0_ct.  out ciphertexts [2][L+K][N], ct-th at
// out + ct out_ct.  At most kMaxGiantTerms terms; ciphertext ct's keys are
// those of the set kt.p[ct / kt.per].
int ks_apply_giants(const Ctx& c, const u64* D, u32 cnt, u32 terms, const u64* galois,
                    const KeyTable& kt, const u64* key_offsets, const u64* c0, u64 c0_term,
                    u64 c0_ct, u64* out, u64 out_ct, cudaStream_t st);
// All baby-step rotations a = 0..B-1 of the H ciphertexts u (raised digits
// D; a = 0 is (P c0, P c1)) written to Rx[h][a] in the split operand layout;
// key a at keys + key_offsets[a] (B >= 2).  Only the primes l0 .. l0+el-1
// (el = 0: to the last), stored as Rx [H][B][2][el][N] (a chunk of primes).
// (kt: the H ciphertexts are queries of kt->per each, with their own keys)
int baby_steps_ext(const Ctx& c, const u64* D, CtSet u, u32 H, u32 B, const u64* keys,
                   const std::vector<u64>& key_offsets, u64* Rx, cudaStream_t st, u32 l0 = 0,
                   u32 el = 0, const KeyTable* kt = nullptr);
// whether the hoisted rotations can run on a chunk of primes (their fused
// kernel applies)
bool rotations_chunkable(const Ctx& c);
// The same for any Galois elements: Rx[h][a] = sigma_{galois[a]}(u_h) with
// key a (a = 1..B-1; a = 0 is (P c0, P c1)), split operand layout.  With
// `ext` the u_h are over Q u P ([2][L+K][N], D raised from their lowered c1):
// rotation a is (sigma(c0) + A0, A1) and a = 0 is u_h itself.
int hoisted_rotations_ext(const Ctx& c, const u64* D, CtSet u, u32 H, u32 B,
                          const std::vector<u64>& galois, const u64* keys,
                          const std::vector<u64>& key_offsets, u64* Rx, cudaStream_t st,
                          bool ext = false, u32 l0 = 0, u32 el = 0,
                          const KeyTable* kt = nullptr);
// out[h] = sum_{a<R} Rx[h][a] (Rx [cnt][R][2][L+K][N] split, out [cnt][2][L+K][N]
// canonical), R <= 8
int sum_rotations(const Ctx& c, const u64* Rx, u32 cnt, u32 R, u64* out, cudaStream_t st);
// (P c0, P c1) over Q u P
int times_P(const Ctx& c, CtSet in, u32 cnt, CtSet out, bool split, cudaStream_t st,
            bool ext = false);   // ext: copy of a ciphertext over Q u P
// ModDown of cnt extended-basis ciphertexts A ([cnt][2][L+K][N], special limbs
// clobbered) into out (Q basis)
size_t mod_down_ws(const Ctx& c, u32 cnt);
int mod_down_batch(const Ctx& c, u64* A, u32 cnt, CtSet out, u64* ws, cudaStream_t st);
// ModDown of npolys polynomials over Q u P (polynomial i at A + i a_stride,
// [L+K][N], left unchanged) into out + i out_stride ([L][N])
// Modulus switching of cnt ciphertexts [cnt][2][L][N] (NTT form) to the
// first L2 primes, out [cnt][2][L2][N]: the ModDown formula with the dropped
// primes q_{L2} .. q_{L-1} in the role of P (input unchanged)
size_t mod_switch_ws(const Ctx& c, u32 cnt);
int mod_switch(const Ctx& c, u32 L2, const u64* cts, u32 cnt, u64* out, u64* ws, cudaStream_t st);
size_t mod_down_polys_ws(const Ctx& c, u32 npolys);
int mod_down_polys(const Ctx& c, const u64* A, u64 a_stride, u32 npolys, u64* out,
                   u64 out_stride, u64* ws, cudaStream_t st);

int gather_rows(CtSet src, long long src_off, u32 cnt, u64 len, u64* dst, u64 dst_stride,
                cudaStream_t st);
// R and Dg in the split operand layout; outputs canonical over Q u P:
// giant index 0 to acc0 [G][2][L+K][N], the others to acc [G][giants-1][2][L+K][N].
// Only the primes l0 .. l0+el-1 (el = 0: to the last); R holds those primes
// ([H][B][2][el][N]).
// (Q > 1: Q queries of plan pl, their half-blocks and groups one after the
// other in R, acc0 and acc)
int diag_mac(const Ctx& c, const pdq_plan& pl, const u64* R, const u64* Dg, u64* acc0, u64* acc,
             cudaStream_t st, u32 l0 = 0, u32 el = 0, u32 Q = 1);
int ct_add(const Ctx& c, CtSet y, CtSet x, u32 cnt, cudaStream_t st);
int group_combine(const Ctx& c, const pdq_plan& pl, const u64* y, const u64* masks, u64* out,
                  cudaStream_t st, u32 Q = 1);

}  // namespace pdq
