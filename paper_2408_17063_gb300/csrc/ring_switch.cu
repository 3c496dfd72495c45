// Ring switching (Sec. 5.3): Comp needs one multiplicative level, so after
// Mask the query moves to a ring of smaller dimension, N' = N / R, where Comp
// is cheaper and the answer shorter (the paper switches 2^15/2^16 -> 2^13 and
// adopts the technique of Gentry, Halevi, Peikert and Smart for it).
//
// A ciphertext (c0, c1) of the big ring under s is key-switched to the secret
// s'(X) = s_small(X^R) of the subring (the hybrid key switch of the rotations
// with the identity automorphism and a key from s to s'), then both
// polynomials are split by coefficient index mod R: with
// c_p(X) = sum_r X^r c_{p,r}(X^R),
//   c0 + c1 s' = sum_r X^r (c0_r + c1_r s_small)(X^R),
// so (c0_r, c1_r) is a ciphertext of the subring, over the same primes, that
// decrypts to m_r, where the plaintext is m(X) = sum_r X^r m_r(X^R).  In the
// slots, m(zeta^e_u) = sum_r zeta^(e_u r) m_r(zeta'^e') for the R exponents
// e_u = e' + 2N'u that fold into small slot e': the diagonals of Comp in the
// subring (plan_make_switched, k_diag_slots_sw) undo that fold, so the answer
// holds the power sums of Eq. 1 over the original records.
#include <cstring>

#include "pdq_internal.h"
#include "pdq_ops.h"

namespace pdq {
namespace {

const Ctx& C(const pdq_ctx* p) { return *reinterpret_cast<const Ctx*>(p); }

int check_pair(const Ctx& b, const Ctx& s) {
    if (s.N >= b.N || b.N % s.N != 0 || s.t != b.t || s.L != b.L || s.K != b.K ||
        s.ndigits != b.ndigits)
        return fail(PDQ_E_PARAM, "ring switch: the small context must be a subring of the big one "
                                 "(pdq_ctx_create_subring)");
    for (u32 i = 0; i < b.L + b.K; ++i)
        if (b.mods[i] != s.mods[i]) return fail(PDQ_E_PARAM, "ring switch: the primes differ");
    return PDQ_OK;
}

size_t rs_ws(const Ctx& b, u32 count) {
    return raise_ws(b, count) + apply_ws(b, count) + (size_t)count * ct_elems(b) * sizeof(u64);
}

}  // namespace
}  // namespace pdq

using namespace pdq;

extern "C" {

int pdq_plan_make_switched(const pdq_ctx* small, uint32_t big_log_n, uint64_t n, uint32_t s,
                           uint32_t B, pdq_plan* plan) {
    if (!small || !plan) return fail(PDQ_E_PARAM, "null argument");
    return plan_make_switched(C(small), big_log_n, n, s, B, plan);
}

int pdq_ring_switch_key_gen(const pdq_ctx* big, const pdq_ctx* small, const uint64_t* sk,
                            const int8_t* s_small, const uint64_t* a, const int32_t* e,
                            uint64_t* key_out, void* stream) {
    if (!big || !small || !sk || !s_small || !a || !e || !key_out)
        return fail(PDQ_E_PARAM, "ring_switch_key_gen: null argument");
    PDQ_TRY(check_pair(C(big), C(small)));
    return ring_switch_keygen(C(big), sk, s_small, C(big).N / C(small).N, a, e, key_out,
                              (cudaStream_t)stream);
}

size_t pdq_ring_switch_workspace_bytes(const pdq_ctx* big, uint32_t count) {
    return big ? rs_ws(C(big), count) : 0;
}

int pdq_ring_switch(const pdq_ctx* big, const pdq_ctx* small, const uint64_t* cts, uint32_t count,
                    uint32_t group, const uint64_t* key, uint64_t* out, void* ws, size_t ws_bytes,
                    void* stream) {
    if (!big || !small) return fail(PDQ_E_PARAM, "ring_switch: null context");
    const Ctx& b = C(big);
    const Ctx& sm = C(small);
    PDQ_TRY(check_pair(b, sm));
    if (count == 0) return PDQ_OK;
    if (!cts || !key || !out || !ws) return fail(PDQ_E_PARAM, "ring_switch: null buffer");
    if (group == 0 || count % group != 0)
        return fail(PDQ_E_PARAM, "ring_switch: count must be a multiple of group");
    if (ws_bytes < rs_ws(b, count)) return fail(PDQ_E_NOMEM, "ring_switch: workspace too small");
    cudaStream_t st = (cudaStream_t)stream;
    const long long cts_b = (long long)ct_elems(b);
    u64* rws = reinterpret_cast<u64*>(ws);
    u64* aws = rws + raise_ws(b, count) / sizeof(u64);
    u64* tmp = aws + apply_ws(b, count) / sizeof(u64);
    const CtSet in = ct_set(cts, cts_b);
    u64* D = nullptr;
    // key switch to s_small(X^R): the identity automorphism with the ring-switching key
    PDQ_TRY(ks_raise(b, in, count, rws, &D, st));
    PDQ_TRY(ks_apply(b, D, in, count, 1u, key, ct_set(tmp, cts_b), CtSet{}, aws, st));
    // split by coefficient index mod R (coefficient form), back to the subring's transform
    PDQ_TRY(ntt_inverse(b, tmp, 2 * count, b.L, 0, (u64)b.L * b.N, st));
    const u32 R = b.N / sm.N;
    PDQ_TRY(ring_split(sm, tmp, count, R, group, out, st));
    return ntt_forward(sm, out, 2 * count * R, sm.L, 0, (u64)sm.L * sm.N, st);
}

}  // extern "C"
