// Internal declarations of the PDQ library (not part of the C ABI).
//
// Residues are uint64 in [0, q) with every prime q < 2^60, so lazy values up
// to 4q fit in 62 bits and sums of up to 2^7 products of two residues fit in
// an unsigned 128-bit accumulator.
#pragma once

#include <cstddef>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "pdq.h"

namespace pdq {

using u64 = uint64_t;
using u32 = uint32_t;
using u128 = unsigned __int128;

// ---------------------------------------------------------------- errors ----
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_check(const char* where);  // PDQ_OK or PDQ_E_CUDA with the message
int launched(const char* where);    // counts one kernel launch, then cuda_check

#define PDQ_TRY(expr)                   \
    do {                                \
        int _rc = (expr);               \
        if (_rc != PDQ_OK) return _rc;  \
    } while (0)

// ------------------------------------------------------- modulus constants --
// One prime with the constants every kernel needs.
struct Mod {
    u64 q;
    u64 ratio;       // floor(2^64 / q)
    u64 r64;         // 2^64 mod q
    u64 r64_shoup;   // floor(r64 * 2^64 / q)
    u64 qinv;        // -q^{-1} mod 2^64 (Montgomery reduction)
};

// ------------------------------------------------------------ device math --
__host__ __device__ __forceinline__ u64 mulhi64(u64 a, u64 b) {
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (u64)(((u128)a * b) >> 64);
#endif
}

// w * x mod q in [0, 2q) with wp = floor(w 2^64 / q), any x < 2^64 (Shoup).
__host__ __device__ __forceinline__ u64 mul_shoup_lazy(u64 x, u64 w, u64 wp, u64 q) {
    return x * w - mulhi64(x, wp) * q;
}

__host__ __device__ __forceinline__ u64 csub(u64 x, u64 q) { return x >= q ? x - q : x; }

// x mod q for any x < 2^64, via the estimate floor(x * floor(2^64/q) / 2^64).
__host__ __device__ __forceinline__ u64 reduce64(u64 x, const Mod& m) {
    return csub(x - mulhi64(x, m.ratio) * m.q, m.q);
}

// (hi * 2^64 + lo) mod q for any 128-bit value: hi * (2^64 mod q) by Shoup,
// lo by the single-word estimate, then two conditional subtractions.
__host__ __device__ __forceinline__ u64 reduce128(u64 hi, u64 lo, const Mod& m) {
    u64 a = mul_shoup_lazy(hi, m.r64, m.r64_shoup, m.q);      // [0, 2q)
    u64 b = lo - mulhi64(lo, m.ratio) * m.q;                  // [0, 2q)
    u64 s = a + b;                                            // [0, 4q)
    s = csub(s, 2 * m.q);
    return csub(s, m.q);
}

// Montgomery reduction of T = hi 2^64 + lo < q 2^64: T 2^-64 mod q, canonical.
// With m = lo (-q^-1) mod 2^64, T + m q is a multiple of 2^64; its quotient
// is hi + hi(m q) + [lo != 0] < 2q.
__host__ __device__ __forceinline__ u64 redc128(u64 hi, u64 lo, const Mod& md) {
    const u64 m = lo * md.qinv;
    const u64 t = hi + mulhi64(m, md.q) + (lo != 0 ? 1 : 0);
    return csub(t, md.q);
}

__host__ __device__ __forceinline__ u64 mulmod(u64 a, u64 b, const Mod& m) {
    u64 lo = a * b;
    u64 hi = mulhi64(a, b);
    return reduce128(hi, lo, m);
}

__host__ __device__ __forceinline__ u64 addmod(u64 a, u64 b, u64 q) { return csub(a + b, q); }
__host__ __device__ __forceinline__ u64 submod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }

// 128-bit accumulator: (hi, lo) += a * b, one carry chain.
__host__ __device__ __forceinline__ void mac128(u64& hi, u64& lo, u64 a, u64 b) {
#ifdef __CUDA_ARCH__
    asm("mad.lo.cc.u64 %0, %2, %3, %0;\n\t"
        "madc.hi.u64 %1, %2, %3, %1;"
        : "+l"(lo), "+l"(hi)
        : "l"(a), "l"(b));
#else
    u64 plo = a * b;
    u64 phi = mulhi64(a, b);
    lo += plo;
    hi += phi + (lo < plo ? 1 : 0);
#endif
}

// --------------------------------------------------------------- context ----
struct Ctx {
    u32 log_n = 0, N = 0, m = 0;
    u64 t = 0;
    u32 L = 0, K = 0, dnum = 0, alpha = 0, ndigits = 0, bits = 0;
    u32 nmod = 0;                 // L + K + 1 (the last is t)
    std::vector<u64> mods;        // q_0..q_{L-1}, p_0..p_{K-1}, t
    std::vector<Mod> hmods;
    u64 gen = 0;                  // smallest generator of Z_t^*
    u64 zeta = 0;                 // slot root mod t, gen^((t-1)/2N)
    std::vector<u64> psi;         // transform root per modulus
    // device tables, each [nmod][N] unless noted
    Mod* d_mods = nullptr;        // [nmod]
    u64* d_fw2 = nullptr;         // [nmod][N][2] forward twiddles psi^{brv(i)} + Shoup
    u64* d_iw2 = nullptr;         // [nmod][N][2] inverse twiddles psi^{-brv(i)} + Shoup
    u64* d_ninv = nullptr;        // [nmod][4]: N^-1, shoup, N^-1 * iw[1], shoup
    u32* d_slot_pos = nullptr;    // [N] transform position of slot rho*m + c
    u64* d_rowmask = nullptr;     // [2][L][N] NTT-form plaintexts [1;0], [0;1]
    // key-switching constants
    // ModUp, digit beta: for i in digit, hat_inv (Q_b/q_i)^-1 mod q_i + shoup;
    // for every ext prime r: (Q_b/q_i) mod r.   Layout:
    u64* d_up_hatinv = nullptr;   // [L] (q_i's own digit), value
    u64* d_up_hatinv_shoup = nullptr;
    u64* d_up_hatmod = nullptr;   // [L][L+K]: (Q_{digit(i)}/q_i) mod r
    u64* d_up_hatmod_shoup = nullptr;
    // the same scaled by R = 2^64 mod r (raised digits are kept multiplied by
    // R so that the key inner products end with one Montgomery reduction)
    u64* d_up_hatmod_mont = nullptr;
    u64* d_up_hatmod_mont_shoup = nullptr;
    // the raise with the conversion folded into the transforms: the inverse
    // transform's last-level constants times hat_inv_i ([nmod][4], as d_ninv),
    // and (hatmod R, Shoup) pairs [L][L+K][2]
    u64* d_ninv_up = nullptr;
    u64* d_up_mont2 = nullptr;
    // ModDown likewise: last-level constants times (P/p_k)^-1 on the special
    // primes ([nmod][4]) and ((P/p_k) mod q_i, Shoup) pairs [K][L][2]
    u64* d_ninv_dn = nullptr;
    u64* d_dn_pair = nullptr;
    // ModDown: (P/p_k)^-1 mod p_k (+shoup); (P/p_k) mod q_i; P^-1 mod q_i (+shoup)
    u64* d_dn_hatinv = nullptr;   // [K]
    u64* d_dn_hatinv_shoup = nullptr;
    u64* d_dn_hatmod = nullptr;   // [K][L]
    u64* d_dn_hatmod_shoup = nullptr;
    u64* d_dn_pinv = nullptr;     // [L]
    u64* d_dn_pinv_shoup = nullptr;
    // P mod q_i (keygen), Delta mod q_i (encryption)
    std::vector<u64> P_mod_q, delta_mod_q;
    u64* d_P_mod_q = nullptr;
    u64* d_P_mod_q_shoup = nullptr;
    u64* d_P_mont = nullptr;      // [L] P 2^64 mod q_i
    u64* d_delta_mod_q = nullptr;
    // decryption: per q_i, omega_i = (Q/q_i)^-1 mod q_i (+shoup), and
    // t * b / q_i split for rounding is done with 128-bit arithmetic.
    u64* d_ckar = nullptr;        // [nmod][8]: 1 - 2^30, 2^30, 2^60 - 2^30 (mod q), each + Shoup
    u64* d_dec_omega = nullptr;
    u64* d_dec_omega_shoup = nullptr;
    std::vector<std::vector<u32>> digit_limbs;   // limbs of each digit
    // modulus switching to the first L' ciphertext primes (L' = 1..L-1),
    // dividing by D = q_{L'} .. q_{L-1} (K' = L - L' primes): one block per
    // L' at d_ms + ms_off[L']: (D/d_k)^-1 mod d_k [K'] and Shoup [K'],
    // (D/d_k) mod q_i [K'][L'] and Shoup [K'][L'], D^-1 mod q_i [L'] and Shoup [L']
    u64* d_ms = nullptr;
    std::vector<u64> ms_off;
    // stage profiling: events recorded on the caller's stream when enabled
    struct Prof {
        bool on = false;
        bool nvtx_open = false;
        std::vector<cudaEvent_t> ev;
        std::vector<int> stage;
        size_t used = 0;
    };
    mutable Prof prof;
    // streams of pdq_answer_batch, created on first use
    struct Lanes {
        std::vector<cudaStream_t> streams;
        std::vector<cudaEvent_t> joins;
        cudaEvent_t fork = nullptr;
    };
    mutable Lanes lanes;
    mutable std::mutex lanes_mu;
    // bytes of baby-step rotations the Answer holds at once (0: all of
    // them); smaller budgets produce and consume them a chunk of primes at a
    // time (pdq_ctx_set_rotation_budget)
    u64 rotation_budget = 0;
    // launch schedule knobs (pdq_ctx_set_schedule; 0: the library's rule)
    pdq_schedule sched{};
};

void lanes_release(Ctx* c);

// uint64 elements of one ciphertext over the ciphertext primes, [2][L][N]
inline u64 ct_elems(const Ctx& c) { return 2ull * c.L * c.N; }

// Record a stage boundary (stage < 0 closes the current stage) when
// profiling is enabled on the context.
void prof_mark(const Ctx& c, int stage, cudaStream_t st);

// ---------------------------------------------------------- host helpers ---
u64 host_powmod(u64 a, u64 e, u64 q);
u64 host_invmod(u64 a, u64 q);
u64 shoup_of(u64 w, u64 q);
Mod make_mod(u64 q);
bool host_is_prime(u64 n);
// The ring X^N + 1 (N = 2^log_n) and the plaintext prime t alone, checked as
// a context checks them, into c: no primes, tables or device memory.  Enough
// for the plan arithmetic and Decomp, which a client runs without a GPU.
int host_ring(u64 t, u32 log_n, Ctx* c);
u32 bitrev(u32 x, u32 bits);

// ------------------------------------------------------------- transforms --
// Forward / inverse negacyclic transform of `count` groups of `nlimbs` limbs,
// group g limb l at data + g*stride + l*N, modulus index limb0 + l.
int ntt_forward(const Ctx& c, u64* data, u32 count, u32 nlimbs, u32 limb0, u64 stride,
                cudaStream_t st);
int ntt_inverse(const Ctx& c, u64* data, u32 count, u32 nlimbs, u32 limb0, u64 stride,
                cudaStream_t st, const u64* ninv_tab = nullptr);
// Forward transform of raised digits D[count][nd][nlimbs][N] except each
// digit's own limbs (digit b owns limbs b alpha .. b alpha + alpha - 1; every
// digit the same size)
int ntt_forward_digits(const Ctx& c, u64* D, u32 count, u32 nd, u32 alpha, u32 nlimbs,
                       cudaStream_t st);
// Inverse transform of `count` groups of nlimbs limbs (moduli limb0 ..)
// read from a strided set (group g at src + (g / src_per) src_outer +
// (g % src_per) src_inner + src_off, limb l at + l N), written to
// data + g stride.
// (ninv_tab: the last level's constants [nmod][4] instead of N^-1's, e.g.
// c.d_ninv_up, which leaves limb i scaled by hat_inv_i)
// (own_out: also write the raise's own limbs, c1_r R for r in digit r /
// alpha, into raised digits [count][ndigits][L+K][N], as the first phase reads
// c1; two-phase rings, nlimbs = L, limb0 = 0)
int ntt_inverse_from(const Ctx& c, const u64* src, long long src_outer, u32 src_per,
                     long long src_inner, u64 src_off, u64* data, u32 count, u32 nlimbs,
                     u64 stride, cudaStream_t st, u32 limb0 = 0, const u64* ninv_tab = nullptr,
                     u64* own_out = nullptr);
// The raised digits' forward transform with the basis conversion folded into
// its first phase: D[ct][b][r] (r outside digit b's alpha <= 2 limbs) =
// NTT(sum_{k < alpha} y[ct][b alpha + k] (Q_b/q_{b alpha+k}) R mod q_r), where
// Y [count][L][N] holds y_i = c1_i hat_inv_i (coefficient form); the digits'
// own limbs are left as they are.
int ntt_forward_digits_modup(const Ctx& c, u64* D, const u64* Y, u32 count, u32 nd, u32 alpha,
                             u32 nlimbs, cudaStream_t st);
// ModDown's conversion folded into a forward transform: Cv[g][i] (i < L) =
// NTT(sum_{k < K} y_k(g) (P/p_k) mod q_i) for the K <= 2 special limbs y_k(g)
// at S + g s_stride + k N, coefficient form scaled by (P/p_k)^-1 (an inverse
// transform with c.d_ninv_dn); Cv [count][L][N].
// With A: ModDown's last step in the transform's output, out[g][i] = (A[g][i]
// - Cv[g][i]) P^-1 mod q_i (A at A + g a_stride, out at out + g out_stride,
// limb i at + i N); Cv then only holds the intermediate of the two phases.
int ntt_forward_moddown(const Ctx& c, u64* Cv, const u64* S, u64 s_stride, u32 count,
                        cudaStream_t st, const u64* A = nullptr, u64 a_stride = 0,
                        u64* out = nullptr, u64 out_stride = 0);

}  // namespace pdq
