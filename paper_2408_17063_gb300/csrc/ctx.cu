// Parameter set, prime chain and device-resident tables.
//
// Prime chain (a reading, since the paper only names "two 54-bit primes",
// Sec. 6.1): every prime is below 2^bits and = 1 mod 2N; the K special primes
// are the K largest such primes, the L ciphertext primes the next L, in
// descending order.  The slot root is zeta = g^{(t-1)/2N} mod t with g the
// smallest generator of Z_t^*, and slot (row rho, column c) holds the value of
// the plaintext at zeta^{(-1)^rho 3^c} (Sec. 5.1), so that X -> X^{3^r} is
// Rot_row(.; r) and X -> X^{2N-1} is Rot_col.
#include <cstdio>
#include <cstring>
#include <atomic>
#include <mutex>

#include <nvtx3/nvToolsExt.h>

#include "pdq_internal.h"

namespace pdq {

// ---------------------------------------------------------------- errors ----
static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

int fail(int code, const std::string& msg) {
    set_error(msg);
    return code;
}

int cuda_check(const char* where) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(PDQ_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
    return PDQ_OK;
}

static std::atomic<unsigned long long> g_launches{0};

int launched(const char* where) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cuda_check(where);
}

// Stage names of the NVTX ranges (the order of PDQ_STAGE_*).
static const char* const kStageNames[PDQ_NSTAGES] = {"mask", "pack", "baby", "mac",
                                                     "giant", "rotsum", "combine", "acc_moddown"};

void prof_mark(const Ctx& c, int stage, cudaStream_t st) {
    Ctx::Prof& p = c.prof;
    if (!p.on) return;
    // an NVTX range per stage on the calling thread, so that profilers can
    // select a stage's launches (e.g. ncu --nvtx-include "timed/mac/")
    if (p.nvtx_open) {
        nvtxRangePop();
        p.nvtx_open = false;
    }
    if (stage >= 0 && stage < PDQ_NSTAGES) {
        nvtxRangePushA(kStageNames[stage]);
        p.nvtx_open = true;
    }
    if (p.used == p.ev.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        p.ev.push_back(e);
        p.stage.push_back(0);
    }
    p.stage[p.used] = stage;
    cudaEventRecord(p.ev[p.used], st);
    ++p.used;
}

// ------------------------------------------------------------ host math ----
u64 host_powmod(u64 a, u64 e, u64 q) {
    u128 r = 1 % q, b = a % q;
    while (e) {
        if (e & 1) r = r * b % q;
        b = b * b % q;
        e >>= 1;
    }
    return (u64)r;
}

u64 host_invmod(u64 a, u64 q) {
    // extended Euclid on signed 128-bit values
    __int128 t0 = 0, t1 = 1, r0 = q, r1 = a % q;
    while (r1 != 0) {
        __int128 qt = r0 / r1;
        __int128 tmp = r0 - qt * r1; r0 = r1; r1 = tmp;
        tmp = t0 - qt * t1; t0 = t1; t1 = tmp;
    }
    if (t0 < 0) t0 += q;
    return (u64)t0;
}

u64 shoup_of(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }

Mod make_mod(u64 q) {
    Mod m;
    m.q = q;
    m.ratio = (u64)(((u128)1 << 64) / q);
    m.r64 = (u64)(((u128)1 << 64) % q);
    m.r64_shoup = shoup_of(m.r64, q);
    u64 inv = q;                                   // q^-1 mod 2^64 by Newton (q odd)
    for (int i = 0; i < 6; ++i) inv *= 2 - q * inv;
    m.qinv = (u64)0 - inv;
    return m;
}

static u64 mulmod_h(u64 a, u64 b, u64 q) { return (u64)((u128)a * b % q); }

bool host_is_prime(u64 n) {
    if (n < 2) return false;
    static const u64 small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    for (u64 p : small) {
        if (n % p == 0) return n == p;
    }
    u64 d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; ++s; }
    for (u64 a : small) {
        u64 x = host_powmod(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int r = 1; r < s; ++r) {
            x = mulmod_h(x, x, n);
            if (x == n - 1) { comp = false; break; }
        }
        if (comp) return false;
    }
    return true;
}

u32 bitrev(u32 x, u32 bits) {
    u32 r = 0;
    for (u32 i = 0; i < bits; ++i) { r = (r << 1) | (x & 1); x >>= 1; }
    return r;
}

// distinct prime factors of n (trial division; n < 2^40 here)
static std::vector<u64> prime_factors(u64 n) {
    std::vector<u64> f;
    for (u64 d = 2; d * d <= n; ++d) {
        if (n % d == 0) {
            f.push_back(d);
            while (n % d == 0) n /= d;
        }
    }
    if (n > 1) f.push_back(n);
    return f;
}

// Element of order exactly 2N modulo q (q = 1 mod 2N, N a power of two):
// x^{(q-1)/2N} for the first x giving psi^N = -1.
static u64 root_2n(u64 q, u64 N) {
    for (u64 x = 2; x < q; ++x) {
        u64 c = host_powmod(x, (q - 1) / (2 * N), q);
        if (host_powmod(c, N, q) == q - 1) return c;
    }
    return 0;
}

int host_ring(u64 t, u32 log_n, Ctx* c) {
    if (log_n < 3 || log_n > 16) return fail(PDQ_E_PARAM, "log_n must be in [3, 16]");
    const u64 twoN = 2ull << log_n;
    if (t < 3 || t >= (1ull << 31) || (t - 1) % twoN != 0 || !host_is_prime(t))
        return fail(PDQ_E_PARAM, "t must be a prime < 2^31 with t = 1 mod 2N");
    c->log_n = log_n;
    c->N = 1u << log_n;
    c->m = c->N / 2;
    c->t = t;
    return PDQ_OK;
}

template <class T>
static int upload(T** dst, const std::vector<T>& src) {
    if (cudaMalloc((void**)dst, src.size() * sizeof(T)) != cudaSuccess)
        return fail(PDQ_E_NOMEM, "cudaMalloc of a device table failed");
    if (cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(PDQ_E_CUDA, "upload of a device table failed");
    return PDQ_OK;
}

static void free_ctx(Ctx* c) {
    if (!c) return;
    void* ptrs[] = {c->d_mods, c->d_fw2, c->d_iw2, c->d_ninv,
                    c->d_slot_pos, c->d_rowmask, c->d_up_hatinv, c->d_up_hatinv_shoup,
                    c->d_up_hatmod, c->d_up_hatmod_shoup, c->d_dn_hatinv,
                    c->d_dn_hatinv_shoup, c->d_dn_hatmod, c->d_dn_hatmod_shoup,
                    c->d_dn_pinv, c->d_dn_pinv_shoup, c->d_P_mod_q, c->d_P_mod_q_shoup, c->d_delta_mod_q,
                    c->d_dec_omega, c->d_dec_omega_shoup, c->d_ckar,
                    c->d_up_hatmod_mont, c->d_up_hatmod_mont_shoup, c->d_P_mont, c->d_ms,
                    c->d_ninv_up, c->d_up_mont2, c->d_ninv_dn, c->d_dn_pair};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (cudaEvent_t e : c->prof.ev) cudaEventDestroy(e);
    lanes_release(c);
    delete c;
}

int encode_slots(const Ctx& c, const u32* slots, u32 count, u32 nlimbs, u64* out,
                 cudaStream_t st);  // ops.cu

// chain (optional): the K special primes, then the L ciphertext primes, to
// use instead of the search (a subring shares its parent's primes)
static int build_ctx(const pdq_params& p, Ctx* c, const std::vector<u64>* given = nullptr) {
    if (p.log_n < 3 || p.log_n > 16) return fail(PDQ_E_PARAM, "log_n must be in [3, 16]");
    if (p.prime_bits < 20 || p.prime_bits > 60) return fail(PDQ_E_PARAM, "prime_bits must be in [20, 60]");
    if (p.L < 1 || p.L > 30 || p.K < 1 || p.K > 8) return fail(PDQ_E_PARAM, "need 1 <= L <= 30, 1 <= K <= 8");
    if (p.dnum < 1 || p.dnum > p.L) return fail(PDQ_E_PARAM, "need 1 <= dnum <= L");
    c->log_n = p.log_n;
    c->N = 1u << p.log_n;
    c->m = c->N / 2;
    c->t = p.t;
    c->L = p.L;
    c->K = p.K;
    c->dnum = p.dnum;
    c->bits = p.prime_bits;
    const u64 N = c->N, twoN = 2 * N;
    if (p.t < 3 || p.t >= (1ull << 31) || (p.t - 1) % twoN != 0 || !host_is_prime(p.t))
        return fail(PDQ_E_PARAM, "t must be a prime < 2^31 with t = 1 mod 2N");

    // prime chain: descending candidates = 1 mod 2N below 2^bits
    std::vector<u64> chain;
    if (given) {
        chain = *given;
        if (chain.size() != p.K + p.L) return fail(PDQ_E_PARAM, "prime chain of the wrong length");
        for (u64 q : chain)
            if ((q - 1) % twoN != 0 || !host_is_prime(q) || q >= (1ull << p.prime_bits))
                return fail(PDQ_E_PARAM, "prime chain: every prime must be = 1 mod 2N");
    }
    u64 cand = ((1ull << p.prime_bits) - 2) / twoN * twoN + 1;
    while (chain.size() < p.K + p.L) {
        if (cand <= twoN) return fail(PDQ_E_PARAM, "not enough NTT-friendly primes");
        if (host_is_prime(cand)) chain.push_back(cand);
        cand -= twoN;
    }
    for (u32 i = 0; i < p.L; ++i) c->mods.push_back(chain[p.K + i]);
    for (u32 k = 0; k < p.K; ++k) c->mods.push_back(chain[k]);
    c->mods.push_back(p.t);
    c->nmod = p.L + p.K + 1;
    for (u64 q : c->mods) c->hmods.push_back(make_mod(q));

    // digits
    c->alpha = (p.L + p.dnum - 1) / p.dnum;
    for (u32 b = 0; b < p.L; b += c->alpha) {
        std::vector<u32> d;
        for (u32 i = b; i < p.L && i < b + c->alpha; ++i) d.push_back(i);
        c->digit_limbs.push_back(d);
    }
    c->ndigits = (u32)c->digit_limbs.size();
    if (c->alpha > 8) return fail(PDQ_E_PARAM, "at most 8 primes per key-switching digit");
    // key inner products sum ndigits + 1 products below q^2 and end with a
    // Montgomery reduction, which needs the sum below q 2^64
    for (u32 i = 0; i < p.L + p.K; ++i)
        if ((u128)(c->ndigits + 1) * c->mods[i] >= ((u128)1 << 64))
            return fail(PDQ_E_PARAM, "too many key-switching digits for the prime size");

    // slot root
    u64 g = 0;
    {
        auto f = prime_factors(p.t - 1);
        for (u64 x = 2; x < p.t && !g; ++x) {
            bool ok = true;
            for (u64 pf : f)
                if (host_powmod(x, (p.t - 1) / pf, p.t) == 1) { ok = false; break; }
            if (ok) g = x;
        }
    }
    c->gen = g;
    c->zeta = host_powmod(g, (p.t - 1) / twoN, p.t);

    // twiddles
    const u32 nm = c->nmod;
    std::vector<u64> fw(nm * N), fws(nm * N), iw(nm * N), iws(nm * N), ninv(nm * 4);
    for (u32 mi = 0; mi < nm; ++mi) {
        const u64 q = c->mods[mi];
        const u64 psi = (mi == nm - 1) ? c->zeta : root_2n(q, N);
        if (!psi || host_powmod(psi, N, q) != q - 1) return fail(PDQ_E_PARAM, "no 2N-th root of unity");
        c->psi.push_back(psi);
        const u64 ipsi = host_invmod(psi, q);
        std::vector<u64> pw(N), ipw(N);
        pw[0] = 1;
        ipw[0] = 1;
        for (u64 i = 1; i < N; ++i) {
            pw[i] = mulmod_h(pw[i - 1], psi, q);
            ipw[i] = mulmod_h(ipw[i - 1], ipsi, q);
        }
        for (u32 i = 0; i < N; ++i) {
            const u32 r = bitrev(i, p.log_n);
            fw[mi * N + i] = pw[r];
            fws[mi * N + i] = shoup_of(pw[r], q);
            iw[mi * N + i] = ipw[r];
            iws[mi * N + i] = shoup_of(ipw[r], q);
        }
        const u64 ni = host_invmod(N % q, q);
        const u64 n1 = mulmod_h(ni, iw[mi * N + 1], q);
        ninv[4 * mi + 0] = ni;
        ninv[4 * mi + 1] = shoup_of(ni, q);
        ninv[4 * mi + 2] = n1;
        ninv[4 * mi + 3] = shoup_of(n1, q);
    }
    PDQ_TRY(upload(&c->d_mods, c->hmods));
    std::vector<u64> fw2(2 * (size_t)nm * N), iw2(2 * (size_t)nm * N);
    for (size_t i = 0; i < (size_t)nm * N; ++i) {
        fw2[2 * i] = fw[i];
        fw2[2 * i + 1] = fws[i];
        iw2[2 * i] = iw[i];
        iw2[2 * i + 1] = iws[i];
    }
    PDQ_TRY(upload(&c->d_fw2, fw2));
    PDQ_TRY(upload(&c->d_iw2, iw2));
    PDQ_TRY(upload(&c->d_ninv, ninv));
    std::vector<u64> ckar(nm * 8, 0);
    for (u32 mi = 0; mi < nm; ++mi) {
        const u64 q = c->mods[mi];
        const u64 p30 = (u64)(((u128)1 << 30) % q), p60 = (u64)(((u128)1 << 60) % q);
        const u64 k[3] = {(1 % q + q - p30) % q, p30, (p60 + q - p30) % q};
        for (int j = 0; j < 3; ++j) {
            ckar[8 * mi + 2 * j] = k[j];
            ckar[8 * mi + 2 * j + 1] = shoup_of(k[j], q);
        }
    }
    PDQ_TRY(upload(&c->d_ckar, ckar));

    // slot position in the transform output: slot (rho, c) is the value at
    // zeta^e with e = (-1)^rho 3^c mod 2N, found at position brv((e-1)/2)
    std::vector<u32> pos(N);
    u64 e = 1;
    for (u32 col = 0; col < c->m; ++col) {
        const u64 e_top = e, e_bot = twoN - e;
        pos[col] = bitrev((u32)((e_top - 1) / 2), p.log_n);
        pos[c->m + col] = bitrev((u32)((e_bot - 1) / 2), p.log_n);
        e = e * 3 % twoN;
    }
    PDQ_TRY(upload(&c->d_slot_pos, pos));

    const u32 L = p.L, K = p.K, E = L + K;
    // ModUp constants
    std::vector<u64> up_inv(L), up_inv_s(L), up_mod((size_t)L * E);
    for (const auto& d : c->digit_limbs) {
        for (u32 i : d) {
            const u64 qi = c->mods[i];
            u64 hat_i = 1;
            for (u32 j : d)
                if (j != i) hat_i = mulmod_h(hat_i, c->mods[j] % qi, qi);
            up_inv[i] = host_invmod(hat_i, qi);
            up_inv_s[i] = shoup_of(up_inv[i], qi);
            for (u32 r = 0; r < E; ++r) {
                const u64 qr = c->mods[r];
                u64 h = 1 % qr;
                for (u32 j : d)
                    if (j != i) h = mulmod_h(h, c->mods[j] % qr, qr);
                up_mod[(size_t)i * E + r] = h;
            }
        }
    }
    PDQ_TRY(upload(&c->d_up_hatinv, up_inv));
    PDQ_TRY(upload(&c->d_up_hatinv_shoup, up_inv_s));
    PDQ_TRY(upload(&c->d_up_hatmod, up_mod));
    std::vector<u64> up_mod_s(up_mod.size());
    for (u32 i = 0; i < L; ++i)
        for (u32 r = 0; r < E; ++r)
            up_mod_s[(size_t)i * E + r] = shoup_of(up_mod[(size_t)i * E + r], c->mods[r]);
    PDQ_TRY(upload(&c->d_up_hatmod_shoup, up_mod_s));
    std::vector<u64> up_mont(up_mod.size()), up_mont_s(up_mod.size());
    for (u32 i = 0; i < L; ++i)
        for (u32 r = 0; r < E; ++r) {
            const u64 qr = c->mods[r];
            const u64 R = (u64)(((u128)1 << 64) % qr);
            up_mont[(size_t)i * E + r] = mulmod_h(up_mod[(size_t)i * E + r], R, qr);
            up_mont_s[(size_t)i * E + r] = shoup_of(up_mont[(size_t)i * E + r], qr);
        }
    PDQ_TRY(upload(&c->d_up_hatmod_mont, up_mont));
    PDQ_TRY(upload(&c->d_up_hatmod_mont_shoup, up_mont_s));
    // the raise with the conversion folded into the transforms: limb i's
    // inverse transform ends scaled by hat_inv_i, the forward transform of a
    // raised digit reads (hatmod R, Shoup) pairs
    std::vector<u64> ninv_up(ninv), up_mont2(2 * up_mont.size());
    for (u32 i = 0; i < L; ++i) {
        const u64 q = c->mods[i];
        ninv_up[4 * i + 0] = mulmod_h(ninv[4 * i + 0], up_inv[i], q);
        ninv_up[4 * i + 1] = shoup_of(ninv_up[4 * i + 0], q);
        ninv_up[4 * i + 2] = mulmod_h(ninv[4 * i + 2], up_inv[i], q);
        ninv_up[4 * i + 3] = shoup_of(ninv_up[4 * i + 2], q);
    }
    for (size_t k = 0; k < up_mont.size(); ++k) {
        up_mont2[2 * k] = up_mont[k];
        up_mont2[2 * k + 1] = up_mont_s[k];
    }
    PDQ_TRY(upload(&c->d_ninv_up, ninv_up));
    PDQ_TRY(upload(&c->d_up_mont2, up_mont2));

    // ModDown constants
    std::vector<u64> dn_inv(K), dn_inv_s(K), dn_mod((size_t)K * L), pinv(L), pinv_s(L);
    for (u32 k = 0; k < K; ++k) {
        const u64 pk = c->mods[L + k];
        u64 hat = 1;
        for (u32 j = 0; j < K; ++j)
            if (j != k) hat = mulmod_h(hat, c->mods[L + j] % pk, pk);
        dn_inv[k] = host_invmod(hat, pk);
        dn_inv_s[k] = shoup_of(dn_inv[k], pk);
        for (u32 i = 0; i < L; ++i) {
            const u64 qi = c->mods[i];
            u64 h = 1;
            for (u32 j = 0; j < K; ++j)
                if (j != k) h = mulmod_h(h, c->mods[L + j] % qi, qi);
            dn_mod[(size_t)k * L + i] = h;
        }
    }
    c->P_mod_q.resize(L);
    for (u32 i = 0; i < L; ++i) {
        const u64 qi = c->mods[i];
        u64 P = 1;
        for (u32 k = 0; k < K; ++k) P = mulmod_h(P, c->mods[L + k] % qi, qi);
        c->P_mod_q[i] = P;
        pinv[i] = host_invmod(P, qi);
        pinv_s[i] = shoup_of(pinv[i], qi);
    }
    PDQ_TRY(upload(&c->d_dn_hatinv, dn_inv));
    PDQ_TRY(upload(&c->d_dn_hatinv_shoup, dn_inv_s));
    PDQ_TRY(upload(&c->d_dn_hatmod, dn_mod));
    std::vector<u64> dn_mod_s(dn_mod.size());
    for (u32 k = 0; k < K; ++k)
        for (u32 i = 0; i < L; ++i)
            dn_mod_s[(size_t)k * L + i] = shoup_of(dn_mod[(size_t)k * L + i], c->mods[i]);
    PDQ_TRY(upload(&c->d_dn_hatmod_shoup, dn_mod_s));
    // ModDown with the conversion folded into the transforms: special limb
    // k's inverse transform ends scaled by (P/p_k)^-1, the forward transform
    // of the converted limbs reads ((P/p_k) mod q_i, Shoup) pairs [K][L]
    {
        std::vector<u64> ninv_dn(ninv), dn_pair(2 * dn_mod.size());
        for (u32 k = 0; k < K; ++k) {
            const u32 mi = L + k;
            const u64 pk = c->mods[mi];
            ninv_dn[4 * mi + 0] = mulmod_h(ninv[4 * mi + 0], dn_inv[k], pk);
            ninv_dn[4 * mi + 1] = shoup_of(ninv_dn[4 * mi + 0], pk);
            ninv_dn[4 * mi + 2] = mulmod_h(ninv[4 * mi + 2], dn_inv[k], pk);
            ninv_dn[4 * mi + 3] = shoup_of(ninv_dn[4 * mi + 2], pk);
        }
        for (size_t i = 0; i < dn_mod.size(); ++i) {
            dn_pair[2 * i] = dn_mod[i];
            dn_pair[2 * i + 1] = dn_mod_s[i];
        }
        PDQ_TRY(upload(&c->d_ninv_dn, ninv_dn));
        PDQ_TRY(upload(&c->d_dn_pair, dn_pair));
    }
    PDQ_TRY(upload(&c->d_dn_pinv, pinv));
    PDQ_TRY(upload(&c->d_dn_pinv_shoup, pinv_s));
    PDQ_TRY(upload(&c->d_P_mod_q, c->P_mod_q));
    std::vector<u64> pq_s(L);
    for (u32 i = 0; i < L; ++i) pq_s[i] = shoup_of(c->P_mod_q[i], c->mods[i]);
    PDQ_TRY(upload(&c->d_P_mod_q_shoup, pq_s));
    std::vector<u64> pm(L);
    for (u32 i = 0; i < L; ++i)
        pm[i] = mulmod_h(c->P_mod_q[i], (u64)(((u128)1 << 64) % c->mods[i]), c->mods[i]);
    PDQ_TRY(upload(&c->d_P_mont, pm));

    // modulus switching tables, every target level L' < L
    c->ms_off.assign(L + 1, 0);
    std::vector<u64> ms;
    for (u32 L2 = 1; L2 < L; ++L2) {
        const u32 K2 = L - L2;
        c->ms_off[L2] = ms.size();
        std::vector<u64> hinv(K2), hinv_s(K2), hmod((size_t)K2 * L2), hmod_s((size_t)K2 * L2),
            dinv(L2), dinv_s(L2);
        for (u32 k = 0; k < K2; ++k) {
            const u64 dk = c->mods[L2 + k];
            u64 hat = 1;
            for (u32 j = 0; j < K2; ++j)
                if (j != k) hat = mulmod_h(hat, c->mods[L2 + j] % dk, dk);
            hinv[k] = host_invmod(hat, dk);
            hinv_s[k] = shoup_of(hinv[k], dk);
            for (u32 i = 0; i < L2; ++i) {
                const u64 qi = c->mods[i];
                u64 h = 1;
                for (u32 j = 0; j < K2; ++j)
                    if (j != k) h = mulmod_h(h, c->mods[L2 + j] % qi, qi);
                hmod[(size_t)k * L2 + i] = h;
                hmod_s[(size_t)k * L2 + i] = shoup_of(h, qi);
            }
        }
        for (u32 i = 0; i < L2; ++i) {
            const u64 qi = c->mods[i];
            u64 D = 1;
            for (u32 j = 0; j < K2; ++j) D = mulmod_h(D, c->mods[L2 + j] % qi, qi);
            dinv[i] = host_invmod(D, qi);
            dinv_s[i] = shoup_of(dinv[i], qi);
        }
        for (const auto* v : {&hinv, &hinv_s, &hmod, &hmod_s, &dinv, &dinv_s})
            ms.insert(ms.end(), v->begin(), v->end());
    }
    if (!ms.empty()) PDQ_TRY(upload(&c->d_ms, ms));

    // Delta = floor(Q/t): Q = t*Delta + (Q mod t) and Q = 0 mod q_i, so
    // Delta = -(Q mod t) * t^{-1} mod q_i.
    u64 Qmodt = 1;
    for (u32 i = 0; i < L; ++i) Qmodt = mulmod_h(Qmodt, c->mods[i] % p.t, p.t);
    c->delta_mod_q.resize(L);
    for (u32 i = 0; i < L; ++i) {
        const u64 qi = c->mods[i];
        const u64 v = mulmod_h(Qmodt % qi, host_invmod(p.t % qi, qi), qi);
        c->delta_mod_q[i] = v == 0 ? 0 : qi - v;
    }
    PDQ_TRY(upload(&c->d_delta_mod_q, c->delta_mod_q));

    // decryption: omega_i = ((Q/q_i) mod q_i)^{-1}
    std::vector<u64> om(L), oms(L);
    for (u32 i = 0; i < L; ++i) {
        const u64 qi = c->mods[i];
        u64 h = 1;
        for (u32 j = 0; j < L; ++j)
            if (j != i) h = mulmod_h(h, c->mods[j] % qi, qi);
        om[i] = host_invmod(h, qi);
        oms[i] = shoup_of(om[i], qi);
    }
    PDQ_TRY(upload(&c->d_dec_omega, om));
    PDQ_TRY(upload(&c->d_dec_omega_shoup, oms));

    // row masks [1;0], [0;1] in NTT form over the L ciphertext primes
    std::vector<u32> rm(2 * N, 0);
    for (u32 i = 0; i < c->m; ++i) {
        rm[i] = 1;
        rm[N + c->m + i] = 1;
    }
    u32* d_rm = nullptr;
    PDQ_TRY(upload(&d_rm, rm));
    if (cudaMalloc((void**)&c->d_rowmask, 2 * (size_t)L * N * sizeof(u64)) != cudaSuccess) {
        cudaFree(d_rm);
        return fail(PDQ_E_NOMEM, "cudaMalloc of row masks failed");
    }
    int rc = encode_slots(*c, d_rm, 2, L, c->d_rowmask, 0);
    cudaError_t e2 = cudaDeviceSynchronize();
    cudaFree(d_rm);
    if (rc != PDQ_OK) return rc;
    if (e2 != cudaSuccess) return fail(PDQ_E_CUDA, std::string("ctx setup: ") + cudaGetErrorString(e2));
    return PDQ_OK;
}

}  // namespace pdq

using namespace pdq;

extern "C" {

const char* pdq_last_error(void) { return g_last_error.c_str(); }

int pdq_ctx_create(const pdq_params* params, pdq_ctx** out) {
    if (!params || !out) return fail(PDQ_E_PARAM, "null argument");
    *out = nullptr;
    Ctx* c = new Ctx();
    int rc = build_ctx(*params, c);
    if (rc != PDQ_OK) {
        std::string msg = g_last_error;
        free_ctx(c);
        set_error(msg);
        return rc;
    }
    *out = reinterpret_cast<pdq_ctx*>(c);
    return PDQ_OK;
}

int pdq_ctx_create_subring(const pdq_ctx* big, uint32_t log_n, pdq_ctx** out) {
    if (!big || !out) return fail(PDQ_E_PARAM, "null argument");
    *out = nullptr;
    const Ctx& b = *reinterpret_cast<const Ctx*>(big);
    if (log_n < 3 || log_n >= b.log_n) return fail(PDQ_E_PARAM, "subring: need 3 <= log_n < the parent's");
    pdq_params p{};
    p.log_n = log_n;
    p.prime_bits = b.bits;
    p.L = b.L;
    p.K = b.K;
    p.dnum = b.dnum;
    p.t = b.t;
    std::vector<u64> chain;
    for (u32 k = 0; k < b.K; ++k) chain.push_back(b.mods[b.L + k]);
    for (u32 i = 0; i < b.L; ++i) chain.push_back(b.mods[i]);
    Ctx* c = new Ctx();
    int rc = build_ctx(p, c, &chain);
    if (rc == PDQ_OK && c->ndigits != b.ndigits) rc = fail(PDQ_E_PARAM, "subring: digit layout differs");
    if (rc != PDQ_OK) {
        std::string msg = g_last_error;
        free_ctx(c);
        set_error(msg);
        return rc;
    }
    *out = reinterpret_cast<pdq_ctx*>(c);
    return PDQ_OK;
}

int pdq_ctx_destroy(pdq_ctx* ctx) {
    free_ctx(reinterpret_cast<Ctx*>(ctx));
    return PDQ_OK;
}

unsigned long long pdq_launch_count(void) { return g_launches.load(); }

int pdq_profile_enable(pdq_ctx* ctx, int enable) {
    if (!ctx) return fail(PDQ_E_PARAM, "null context");
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    c->prof.on = enable != 0;
    c->prof.used = 0;
    return PDQ_OK;
}

int pdq_profile_read(pdq_ctx* ctx, float* ms, uint32_t* calls, uint32_t nstages) {
    if (!ctx || !ms) return fail(PDQ_E_PARAM, "null argument");
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    for (uint32_t i = 0; i < nstages; ++i) { ms[i] = 0.f; if (calls) calls[i] = 0; }
    Ctx::Prof& p = c->prof;
    for (size_t i = 0; i + 1 < p.used; ++i) {
        const int sidx = p.stage[i];
        if (sidx < 0 || (uint32_t)sidx >= nstages) continue;
        float t = 0.f;
        if (cudaEventSynchronize(p.ev[i + 1]) != cudaSuccess ||
            cudaEventElapsedTime(&t, p.ev[i], p.ev[i + 1]) != cudaSuccess)
            return fail(PDQ_E_CUDA, "profile_read: event query failed");
        ms[sidx] += t;
        if (calls) calls[sidx] += 1;
    }
    p.used = 0;
    return PDQ_OK;
}

int pdq_ctx_info(const pdq_ctx* ctx, pdq_info* info) {
    if (!ctx || !info) return fail(PDQ_E_PARAM, "null argument");
    const Ctx* c = reinterpret_cast<const Ctx*>(ctx);
    std::memset(info, 0, sizeof(*info));
    info->N = c->N;
    info->L = c->L;
    info->K = c->K;
    info->ndigits = c->ndigits;
    info->t = c->t;
    info->zeta = c->zeta;
    for (u32 i = 0; i < c->L + c->K && i < PDQ_MAX_MODULI; ++i) info->moduli[i] = c->mods[i];
    for (u32 i = 0; i < c->nmod && i < PDQ_MAX_MODULI; ++i) info->psi[i] = c->psi[i];
    return PDQ_OK;
}

}  // extern "C"
