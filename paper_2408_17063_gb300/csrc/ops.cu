// Element-wise kernels of the PDQ path: slot encoding, key generation,
// encryption and decryption (client side), Mask, the pieces of hybrid key
// switching (raise, inner product with the automorphism, lower), the
// diagonal multiply-accumulate of Comp and the group combine.
//
// All kernels read and write canonical residues.  Products of two residues
// are formed as 128-bit values and reduced once (reduce128), or summed
// unreduced in a 128-bit accumulator first when several products meet.
#include "pdq_internal.h"
#include "pdq_ops.h"

namespace pdq {

namespace {

constexpr u32 kBlock = 256;

inline dim3 grid_for(u64 total) {
    u64 b = (total + kBlock - 1) / kBlock;
    if (b > (1u << 20)) b = 1u << 20;
    if (b == 0) b = 1;
    return dim3((u32)b);
}

// Position holding a(psi^{e k}) for the position x that holds a(psi^e):
// sigma_k in the bit-reversed evaluation domain.
__device__ __forceinline__ u32 auto_index(u32 x, u32 k, u32 logN) {
    const u32 twoN_mask = (2u << logN) - 1;
    const u32 e = 2 * (__brev(x) >> (32 - logN)) + 1;
    const u32 e2 = (u32)(((u64)e * k) & twoN_mask);
    return __brev((e2 - 1) >> 1) >> (32 - logN);
}

// ------------------------------------------------------------- encoding ----

__global__ void k_scatter_slots(const u32* __restrict__ slots, u32 count, u32 N, u64 lstride,
                                const u32* __restrict__ pos, u64 t, u64* __restrict__ out) {
    const u64 total = (u64)count * N;
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < total;
         i += (u64)gridDim.x * blockDim.x) {
        const u64 c = i / N, idx = i % N;
        out[c * lstride + pos[idx]] = slots[i] % t;
    }
}

__global__ void k_lift(u64* __restrict__ out, u32 count, u32 N, u32 nlimbs,
                       const Mod* __restrict__ mods, u64 t) {
    const u64 total = (u64)count * N;
    const u64 half = (t - 1) / 2;
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < total;
         i += (u64)gridDim.x * blockDim.x) {
        const u64 c = i / N, x = i % N;
        u64* base = out + c * nlimbs * (u64)N + x;
        const u64 v = base[0];
        for (int l = (int)nlimbs - 1; l >= 0; --l) {
            const u64 q = mods[l].q;
            base[(u64)l * N] = v > half ? q - (t - v) : v;
        }
    }
}

// diagonal slot values, rotated by -gB, scattered to transform positions
__global__ void k_diag_slots(u64* __restrict__ out, u32 hclass, u32 giants, u32 B, u32 s_prime,
                             u32 m, u32 N, u32 L, const u32* __restrict__ pos, u64 t) {
    const u64 total = (u64)hclass * giants * B * N;
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < total;
         i += (u64)gridDim.x * blockDim.x) {
        const u64 pt = i / N;
        const u32 idx = (u32)(i % N);
        const u32 a = (u32)(pt % B);
        const u32 g = (u32)((pt / B) % giants);
        const u32 cls = (u32)(pt / ((u64)B * giants));
        const u32 col = idx % m;
        const u32 k = g * B + a;
        const u32 cp = (col + m - (g * B) % m) % m;        // Rot(.; -gB)
        const u64 node = (u64)cls * m + (cp + k) % m + 1;
        u32 e = cp % s_prime + 1;
        u64 r = 1, b = node % t;
        while (e) {
            if (e & 1) r = r * b % t;
            b = b * b % t;
            e >>= 1;
        }
        out[pt * (u64)L * N + pos[idx]] = r;
    }
}

// database plaintexts: for ciphertext j, [DB.[1;0], DB.[0;1]]
__global__ void k_db_slots(u64* __restrict__ out, const u32* __restrict__ values, u64 n, u32 J,
                           u32 m, u32 N, u32 L, const u32* __restrict__ pos, u64 t) {
    const u64 total = (u64)J * 2 * N;
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < total;
         i += (u64)gridDim.x * blockDim.x) {
        const u64 pt = i / N;               // j*2 + half
        const u32 idx = (u32)(i % N);
        const u64 j = pt / 2, half = pt % 2;
        const u64 rec = j * N + idx;
        const bool row_ok = (idx >= m) == (half == 1);
        const u64 v = (row_ok && rec < n) ? (u64)values[rec] % t : 0;
        out[pt * (u64)L * N + pos[idx]] = v;
    }
}

// group mask o: ones at slots [o s', (o+1) s') of both rows
__global__ void k_groupmask_slots(u64* __restrict__ out, u32 per_out, u32 s_prime, u32 m, u32 N,
                                  u32 L, const u32* __restrict__ pos) {
    const u64 total = (u64)per_out * N;
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < total;
         i += (u64)gridDim.x * blockDim.x) {
        const u64 o = i / N;
        const u32 idx = (u32)(i % N);
        const u32 col = idx % m;
        out[o * (u64)L * N + pos[idx]] = (col / s_prime == o) ? 1 : 0;
    }
}

// ------------------------------------------------------- keys / encryption -

__global__ void k_signed_to_rns(const int8_t* __restrict__ s, u32 N, u32 nl,
                                const Mod* __restrict__ mods, u64* __restrict__ out) {
    const u64 total = (u64)nl * N;
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < total;
         i += (u64)gridDim.x * blockDim.x) {
        const u32 l = (u32)(i / N), x = (u32)(i % N);
        const int v = s[x];
        const u64 q = mods[l].q;
        out[i] = v < 0 ? q - (u64)(-v) : (u64)v;
    }
}

// c0 = e + Delta * m (coefficient form); m read from limb 0 of c1's slot
__global__ void k_enc_c0(u64* __restrict__ ct, const int32_t* __restrict__ e, u32 count, u32 N,
                         u32 L, const Mod* __restrict__ mods, const u64* __restrict__ delta) {
    const u64 total = (u64)count * N;
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < total;
         i += (u64)gridDim.x * blockDim.x) {
        const u64 c = i / N, x = i % N;
        u64* c0 = ct + c * 2 * L * (u64)N;
        const u64 m = c0[(u64)L * N + x];         // c1 limb 0 holds m mod t
        const int ev = e[i];
        for (u32 l = 0; l < L; ++l) {
            const Mod md = mods[l];
            const u64 ee = ev < 0 ? md.q - (u64)(-ev) : (u64)ev;
            c0[(u64)l * N + x] = addmod(mulmod(m, delta[l], md), ee, md.q);
        }
    }
}

__global__ void k_copy_rows(u64* __restrict__ dst, u64 dst_stride, const u64* __restrict__ src,
                            u64 src_stride, u32 count, u64 len) {
    const u64 total = (u64)count * len;
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < total;
         i += (u64)gridDim.x * blockDim.x) {
        const u64 c = i / len, x = i % len;
        dst[c * dst_stride + x] = src[c * src_stride + x];
    }
}

// c0 -= c1 * s (NTT form)
__global__ void k_enc_finish(u64* __restrict__ ct, const u64* __restrict__ sk, u32 count, u32 N,
                             u32 L, const Mod* __restrict__ mods) {
    const u64 total = (u64)count * L * N;
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < total;
         i += (u64)gridDim.x * blockDim.x) {
        const u64 c = i / ((u64)L * N), r = i % ((u64)L * N);
        const u32 l = (u32)(r / N);
        const Mod md = mods[l];
        u64* c0 = ct + c * 2 * L * (u64)N;
        const u64 as = mulmod(c0[(u64)L * N + r], sk[r], md);
        c0[r] = submod(c0[r], as, md.q);
    }
}

// key: b = b(e) - a*s + [l in digit] P sigma_k(s), all NTT form
__global__ void k_key_finish(u64* __restrict__ key, const u64* __restrict__ sk, u32 nd, u32 E,
                             u32 N, u32 logN, u32 galois, const Mod* __restrict__ mods,
                             const u64* __restrict__ Pmodq, DigitBounds db) {
    const u64 total = (u64)nd * E * N;
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < total;
         i += (u64)gridDim.x * blockDim.x) {
        const u32 b = (u32)(i / ((u64)E * N));
        const u64 r = i % ((u64)E * N);
        const u32 l = (u32)(r / N), x = (u32)(r % N);
        const Mod md = mods[l];
        u64* kb = key + (u64)b * 2 * E * N;
        const u64 av = kb[(u64)E * N + r];
        u64 v = submod(kb[r], mulmod(av, sk[r], md), md.q);
        if (l >= db.lo[b] && l < db.hi[b]) {
            const u64 sv = sk[(u64)l * N + auto_index(x, galois, logN)];
            v = addmod(v, mulmod(sv, Pmodq[l], md), md.q);
        }
        kb[r] = v;
    }
}

// decryption: x = c0 + c1 s (NTT form) into ws
__global__ void k_dec_inner(const u64* __restrict__ ct, const u64* __restrict__ sk, u32 count,
                            u32 N, u32 L, const Mod* __restrict__ mods, u64* __restrict__ out) {
    const u64 total = (u64)count * L * N;
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < total;
         i += (u64)gridDim.x * blockDim.x) {
        const u64 c = i / ((u64)L * N), r = i % ((u64)L * N);
        const Mod md = mods[r / N];
        const u64* c0 = ct + c * 2 * L * (u64)N;
        out[i] = addmod(c0[r], mulmod(c0[(u64)L * N + r], sk[r], md), md.q);
    }
}

// m = round(sum_i [x_i omega_i]_{q_i} t / q_i) mod t, written to limb 0 of
// a [count][1][N] buffer (mod t)
__global__ void k_dec_round(const u64* __restrict__ x, u32 count, u32 N, u32 L,
                            const Mod* __restrict__ mods, const u64* __restrict__ om,
                            const u64* __restrict__ oms, u64 t, u64* __restrict__ out) {
    const u64 total = (u64)count * N;
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < total;
         i += (u64)gridDim.x * blockDim.x) {
        const u64 c = i / N, xi = i % N;
        u64 ip = 0;        // integer part (mod t accumulation, < L t)
        u128 fr = 0;       // fractional part, 64-bit fixed point
        for (u32 l = 0; l < L; ++l) {
            const u64 q = mods[l].q;
            const u64 v = x[(c * L + l) * (u64)N + xi];
            const u64 b = csub(mul_shoup_lazy(v, om[l], oms[l], q), q);
            const u128 bt = (u128)b * t;
            const u64 quo = (u64)(bt / q);
            const u64 rem = (u64)(bt % q);
            ip += quo % t;
            fr += (u128)(u64)(((u128)rem << 64) / q);
        }
        const u64 whole = (u64)(fr >> 64);
        const u64 lo = (u64)fr;
        const u64 r = (ip + whole + (lo >> 63)) % t;
        out[i] = r;
    }
}

__global__ void k_gather_slots(const u64* __restrict__ in, u32 count, u32 N,
                               const u32* __restrict__ pos, u32* __restrict__ slots) {
    const u64 total = (u64)count * N;
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < total;
         i += (u64)gridDim.x * blockDim.x) {
        const u64 c = i / N, idx = i % N;
        slots[i] = (u32)in[c * N + pos[idx]];
    }
}

// ------------------------------------------------------------------ Mask ----

// out[j] = (v.[1;0], v.[0;1], v.(DB.[1;0]), v.(DB.[0;1]))
__global__ void k_mask(const u64* __restrict__ v, const u64* __restrict__ db,
                       const u64* __restrict__ rowmask, u32 J, u32 L, u32 N,
                       const Mod* __restrict__ mods, u64* __restrict__ out) {
    const u64 LN = (u64)L * N;
    const u64 total = (u64)J * LN;
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < total;
         i += (u64)gridDim.x * blockDim.x) {
        const u64 j = i / LN, r = i % LN;
        const Mod md = mods[r / N];
        const u64 v0 = v[j * 2 * LN + r], v1 = v[j * 2 * LN + LN + r];
        const u64 pt[4] = {rowmask[r], rowmask[LN + r], db[j * 2 * LN + r], db[j * 2 * LN + LN + r]};
        u64* o = out + j * 8 * LN;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            o[(2 * k) * LN + r] = mulmod(v0, pt[k], md);
            o[(2 * k + 1) * LN + r] = mulmod(v1, pt[k], md);
        }
    }
}

// ---------------------------------------------------------- key switching --

// Raise every digit of c1 (coefficient form X [cnt][L][N]) to the extended
// basis: D[ct][beta][r] for r outside the digit (coefficient form, to be
// transformed), and for r inside the digit the NTT-form c1 limb is copied.
__global__ void k_modup(const u64* __restrict__ X, CtSet c1ntt, u32 cnt, u32 N, u32 L, u32 E,
                        u32 nd, u32 alpha, const Mod* __restrict__ mods,
                        const u64* __restrict__ hinv, const u64* __restrict__ hinvs,
                        const u64* __restrict__ hmod, u64* __restrict__ D) {
    const u64 total = (u64)cnt * nd * N;
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < total;
         i += (u64)gridDim.x * blockDim.x) {
        const u64 ct = i / ((u64)nd * N);
        const u32 b = (u32)((i / N) % nd);
        const u32 x = (u32)(i % N);
        const u32 lo = b * alpha, hi = min(lo + alpha, L);
        u64 y[8];
        const u64* Xc = X + ct * (u64)L * N;
        for (u32 l = lo; l < hi; ++l) {
            const u64 q = mods[l].q;
            y[l - lo] = csub(mul_shoup_lazy(Xc[(u64)l * N + x], hinv[l], hinvs[l], q), q);
        }
        u64* Dc = D + (ct * nd + b) * (u64)E * N;
        const u64* src = c1ntt.at(ct) + (u64)L * N;    // c1 of the input (NTT form)
        for (u32 r = 0; r < E; ++r) {
            if (r >= lo && r < hi) {
                Dc[(u64)r * N + x] = src[(u64)r * N + x];
                continue;
            }
            const Mod md = mods[r];
            u64 ah = 0, al = 0;
            for (u32 l = lo; l < hi; ++l) mac128(ah, al, y[l - lo], hmod[(u64)l * E + r]);
            Dc[(u64)r * N + x] = reduce128(ah, al, md);
        }
    }
}

// A[ct][p][r][x] = sum_beta D[ct][beta][r][sigma(x)] * key[beta][p][r][x]
__global__ void k_ks_inner(const u64* __restrict__ D, const u64* __restrict__ key, u32 cnt, u32 N,
                           u32 logN, u32 E, u32 nd, u32 galois, const Mod* __restrict__ mods,
                           u64* __restrict__ A) {
    const u64 EN = (u64)E * N;
    const u64 total = (u64)cnt * EN;
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < total;
         i += (u64)gridDim.x * blockDim.x) {
        const u64 ct = i / EN, r = i % EN;
        const u32 l = (u32)(r / N), x = (u32)(r % N);
        const u32 sx = auto_index(x, galois, logN);
        u64 h0 = 0, l0 = 0, h1 = 0, l1 = 0;
        for (u32 b = 0; b < nd; ++b) {
            const u64 d = D[(ct * nd + b) * EN + (u64)l * N + sx];
            mac128(h0, l0, d, key[(u64)b * 2 * EN + r]);
            mac128(h1, l1, d, key[(u64)b * 2 * EN + EN + r]);
        }
        const Mod md = mods[l];
        A[ct * 2 * EN + r] = reduce128(h0, l0, md);
        A[ct * 2 * EN + EN + r] = reduce128(h1, l1, md);
    }
}

// Conv[ct][p][i] = sum_k [y_k (P/p_k)^-1]_{p_k} (P/p_k) mod q_i from the
// special limbs of A (coefficient form)
__global__ void k_moddown_conv(const u64* __restrict__ A, u32 cnt, u32 N, u32 L, u32 K,
                               const Mod* __restrict__ mods, const u64* __restrict__ hinv,
                               const u64* __restrict__ hinvs, const u64* __restrict__ hmod,
                               u64* __restrict__ Cv) {
    const u32 E = L + K;
    const u64 total = (u64)cnt * 2 * N;
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < total;
         i += (u64)gridDim.x * blockDim.x) {
        const u64 cp = i / N;      // ct*2 + p
        const u32 x = (u32)(i % N);
        const u64* a = A + cp * (u64)E * N;
        u64 y[8];
        for (u32 k = 0; k < K; ++k) {
            const u64 pk = mods[L + k].q;
            y[k] = csub(mul_shoup_lazy(a[(u64)(L + k) * N + x], hinv[k], hinvs[k], pk), pk);
        }
        u64* o = Cv + cp * (u64)L * N;
        for (u32 l = 0; l < L; ++l) {
            u64 ah = 0, al = 0;
            for (u32 k = 0; k < K; ++k) mac128(ah, al, y[k], hmod[(u64)k * L + l]);
            o[(u64)l * N + x] = reduce128(ah, al, mods[l]);
        }
    }
}

// out = (A - Conv) * P^-1 (+ sigma(c0) for p = 0) (+ addend), NTT form
__global__ void k_moddown_final(const u64* __restrict__ A, const u64* __restrict__ Cv,
                                CtSet in, CtSet out, CtSet add, u32 cnt, u32 N, u32 logN, u32 L,
                                u32 K, u32 galois, const Mod* __restrict__ mods,
                                const u64* __restrict__ pinv, const u64* __restrict__ pinvs) {
    const u32 E = L + K;
    const u64 LN = (u64)L * N;
    const u64 total = (u64)cnt * 2 * LN;
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < total;
         i += (u64)gridDim.x * blockDim.x) {
        const u64 ct = i / (2 * LN);
        const u64 rr = i % (2 * LN);
        const u32 p = (u32)(rr / LN);
        const u64 r = rr % LN;
        const u32 l = (u32)(r / N), x = (u32)(r % N);
        const u64 q = mods[l].q;
        const u64 a = A[(ct * 2 + p) * (u64)E * N + r];
        const u64 cv = Cv[(ct * 2 + p) * LN + r];
        u64 v = csub(mul_shoup_lazy(submod(a, cv, q), pinv[l], pinvs[l], q), q);
        if (p == 0) v = addmod(v, in.at(ct)[(u64)l * N + auto_index(x, galois, logN)], q);
        if (add.base) v = addmod(v, add.at(ct)[rr], q);
        out.at(ct)[rr] = v;
    }
}

// ----------------------------------------------------------- Comp kernels --

// acc[gamma][g][p] = sum_{hh} sum_{a<B} Dg[cls(h)][g][a] * R[h][a][p], h = gamma*hpg + hh
template <int GI>
__global__ void k_diag_mac(const u64* __restrict__ R, const u64* __restrict__ Dg, u32 G, u32 hpg,
                           u32 H, u32 B, u32 L, u32 N, const Mod* __restrict__ mods,
                           u64* __restrict__ acc) {
    const u64 LN = (u64)L * N;
    const u64 total = (u64)G * 2 * LN;
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < total;
         i += (u64)gridDim.x * blockDim.x) {
        const u64 r = i % LN;
        const u32 p = (u32)((i / LN) % 2);
        const u32 gamma = (u32)(i / (2 * LN));
        u64 ah[GI], al[GI];
#pragma unroll
        for (int g = 0; g < GI; ++g) { ah[g] = 0; al[g] = 0; }
        const u32 h0 = gamma * hpg;
        const u32 h1 = min(h0 + hpg, H);
        const Mod md = mods[r / N];
        u32 terms = 0;   // products since the last fold (each < 2^120; 255 of them fit)
        for (u32 h = h0; h < h1; ++h) {
            if (terms + B > 255) {
#pragma unroll
                for (int g = 0; g < GI; ++g) { al[g] = reduce128(ah[g], al[g], md); ah[g] = 0; }
                terms = 0;
            }
            terms += B;
            const u32 cls = h % hpg;
            const u64* Rh = R + (u64)h * B * 2 * LN + (u64)p * LN + r;
            const u64* Dh = Dg + (u64)cls * GI * B * LN + r;
            for (u32 a = 0; a < B; ++a) {
                const u64 rv = Rh[(u64)a * 2 * LN];
#pragma unroll
                for (int g = 0; g < GI; ++g) mac128(ah[g], al[g], Dh[((u64)g * B + a) * LN], rv);
            }
        }
        u64* o = acc + (u64)gamma * GI * 2 * LN + (u64)p * LN + r;
#pragma unroll
        for (int g = 0; g < GI; ++g) o[(u64)g * 2 * LN] = reduce128(ah[g], al[g], md);
    }
}

// y[cnt] += x[cnt] (ciphertexts)
__global__ void k_ct_add(CtSet y, CtSet x, u32 cnt, u32 L, u32 N, const Mod* __restrict__ mods) {
    const u64 LN = (u64)L * N;
    const u64 total = (u64)cnt * 2 * LN;
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < total;
         i += (u64)gridDim.x * blockDim.x) {
        const u64 c = i / (2 * LN), r = i % (2 * LN);
        const u64 q = mods[(r % LN) / N].q;
        u64* yp = y.at(c);
        yp[r] = addmod(yp[r], x.at(c)[r], q);
    }
}

// out[c] = sum_{o} M_o * y[c*per_out + o]
__global__ void k_group_combine(const u64* __restrict__ y, const u64* __restrict__ masks, u32 G,
                                u32 per_out, u32 n_out, u32 L, u32 N, const Mod* __restrict__ mods,
                                u64* __restrict__ out) {
    const u64 LN = (u64)L * N;
    const u64 total = (u64)n_out * 2 * LN;
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < total;
         i += (u64)gridDim.x * blockDim.x) {
        const u64 c = i / (2 * LN), rr = i % (2 * LN);
        const u64 r = rr % LN;
        const Mod md = mods[r / N];
        u64 ah = 0, al = 0;
        for (u32 o = 0; o < per_out; ++o) {
            const u64 gamma = c * per_out + o;
            if (gamma >= G) break;
            if ((o & 127) == 127) { al = reduce128(ah, al, md); ah = 0; }
            mac128(ah, al, masks[(u64)o * LN + r], y[gamma * 2 * LN + rr]);
        }
        out[i] = reduce128(ah, al, md);
    }
}

}  // namespace

// ================================================================ launchers ==

int encode_finish(const Ctx& c, u64* out, u32 count, u32 nlimbs, cudaStream_t st) {
    const u64 N = c.N;
    PDQ_TRY(ntt_inverse(c, out, count, 1, c.nmod - 1, (u64)nlimbs * N, st));
    k_lift<<<grid_for((u64)count * N), kBlock, 0, st>>>(out, count, c.N, nlimbs, c.d_mods, c.t);
    PDQ_TRY(launched("k_lift"));
    return ntt_forward(c, out, count, nlimbs, 0, (u64)nlimbs * N, st);
}

int encode_slots(const Ctx& c, const u32* slots, u32 count, u32 nlimbs, u64* out,
                 cudaStream_t st) {
    if (count == 0) return PDQ_OK;
    if (nlimbs < 1 || nlimbs > c.L + c.K) return fail(PDQ_E_PARAM, "encode: bad limb count");
    k_scatter_slots<<<grid_for((u64)count * c.N), kBlock, 0, st>>>(
        slots, count, c.N, (u64)nlimbs * c.N, c.d_slot_pos, c.t, out);
    PDQ_TRY(launched("k_scatter_slots"));
    return encode_finish(c, out, count, nlimbs, st);
}

int build_diagonals(const Ctx& c, const pdq_plan& pl, u64* out, cudaStream_t st) {
    const u32 count = pl.hclass * pl.giants * pl.B;
    k_diag_slots<<<grid_for((u64)count * c.N), kBlock, 0, st>>>(
        out, pl.hclass, pl.giants, pl.B, pl.s_prime, c.m, c.N, c.L, c.d_slot_pos, c.t);
    PDQ_TRY(launched("k_diag_slots"));
    return encode_finish(c, out, count, c.L, st);
}

int build_group_masks(const Ctx& c, const pdq_plan& pl, u64* out, cudaStream_t st) {
    k_groupmask_slots<<<grid_for((u64)pl.per_out * c.N), kBlock, 0, st>>>(
        out, pl.per_out, pl.s_prime, c.m, c.N, c.L, c.d_slot_pos);
    PDQ_TRY(launched("k_groupmask_slots"));
    return encode_finish(c, out, pl.per_out, c.L, st);
}

int build_db(const Ctx& c, const u32* values, u64 n, u32 J, u64* out, cudaStream_t st) {
    k_db_slots<<<grid_for((u64)J * 2 * c.N), kBlock, 0, st>>>(out, values, n, J, c.m, c.N, c.L,
                                                               c.d_slot_pos, c.t);
    PDQ_TRY(launched("k_db_slots"));
    return encode_finish(c, out, 2 * J, c.L, st);
}

int secret_prepare(const Ctx& c, const int8_t* s, u64* out, cudaStream_t st) {
    const u32 E = c.L + c.K;
    k_signed_to_rns<<<grid_for((u64)E * c.N), kBlock, 0, st>>>(s, c.N, E, c.d_mods, out);
    PDQ_TRY(launched("k_signed_to_rns"));
    return ntt_forward(c, out, 1, E, 0, (u64)E * c.N, st);
}

int encrypt(const Ctx& c, const u64* sk, const u32* slots, u32 count, const u64* a,
            const int32_t* e, u64* ct, cudaStream_t st) {
    if (count == 0) return PDQ_OK;
    const u64 N = c.N, L = c.L, LN = L * N;
    // m mod t (coefficient form) into limb 0 of each c1
    k_scatter_slots<<<grid_for((u64)count * N), kBlock, 0, st>>>(slots, count, c.N, 2 * LN,
                                                                 c.d_slot_pos, c.t, ct + LN);
    PDQ_TRY(launched("k_scatter_slots"));
    PDQ_TRY(ntt_inverse(c, ct + LN, count, 1, c.nmod - 1, 2 * LN, st));
    k_enc_c0<<<grid_for((u64)count * N), kBlock, 0, st>>>(ct, e, count, c.N, c.L, c.d_mods,
                                                          c.d_delta_mod_q);
    PDQ_TRY(launched("k_enc_c0"));
    k_copy_rows<<<grid_for((u64)count * LN), kBlock, 0, st>>>(ct + LN, 2 * LN, a, LN, count, LN);
    PDQ_TRY(launched("k_copy_rows"));
    PDQ_TRY(ntt_forward(c, ct, 2 * count, c.L, 0, LN, st));
    k_enc_finish<<<grid_for((u64)count * LN), kBlock, 0, st>>>(ct, sk, count, c.N, c.L, c.d_mods);
    return launched("k_enc_finish");
}

namespace {
__global__ void k_signed32_to_rns(const int32_t* __restrict__ e, u32 N, u32 nl,
                                  const Mod* __restrict__ mods, u64* __restrict__ out) {
    const u64 total = (u64)nl * N;
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < total;
         i += (u64)gridDim.x * blockDim.x) {
        const u32 l = (u32)(i / N), x = (u32)(i % N);
        const long long v = e[x];
        const u64 q = mods[l].q;
        out[i] = v < 0 ? q - (u64)(-v) : (u64)v;
    }
}

__global__ void k_gather_set(CtSet src, long long off, u32 cnt, u64 len, u64* __restrict__ dst,
                             u64 dst_stride) {
    const u64 total = (u64)cnt * len;
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < total;
         i += (u64)gridDim.x * blockDim.x) {
        const u64 c = i / len, x = i % len;
        dst[c * dst_stride + x] = src.at(c)[off + (long long)x];
    }
}
}  // namespace

int gather_rows(CtSet src, long long src_off, u32 cnt, u64 len, u64* dst, u64 dst_stride,
                cudaStream_t st) {
    k_gather_set<<<grid_for((u64)cnt * len), kBlock, 0, st>>>(src, src_off, cnt, len, dst, dst_stride);
    return launched("k_gather_set");
}

int rotkey_gen(const Ctx& c, const u64* sk, u64 galois, const u64* a, const int32_t* e, u64* key,
               cudaStream_t st) {
    const u32 E = c.L + c.K, nd = c.ndigits;
    const u64 EN = (u64)E * c.N;
    if (galois % 2 == 0 || galois >= 2ull * c.N) return fail(PDQ_E_PARAM, "galois element must be odd and < 2N");
    if (nd > 32) return fail(PDQ_E_PARAM, "at most 32 digits");
    // a into the second half of every digit, e (as residues) into the first
    k_copy_rows<<<grid_for((u64)nd * EN), kBlock, 0, st>>>(key + EN, 2 * EN, a, EN, nd, EN);
    PDQ_TRY(launched("k_copy_rows"));
    for (u32 b = 0; b < nd; ++b) {
        k_signed32_to_rns<<<grid_for(EN), kBlock, 0, st>>>(e + (u64)b * c.N, c.N, E, c.d_mods,
                                                           key + (u64)b * 2 * EN);
        PDQ_TRY(launched("k_signed32_to_rns"));
    }
    PDQ_TRY(ntt_forward(c, key, 2 * nd, E, 0, EN, st));
    DigitBounds db{};
    for (u32 b = 0; b < nd; ++b) {
        db.lo[b] = c.digit_limbs[b].front();
        db.hi[b] = c.digit_limbs[b].back() + 1;
    }
    k_key_finish<<<grid_for((u64)nd * EN), kBlock, 0, st>>>(key, sk, nd, E, c.N, c.log_n,
                                                            (u32)galois, c.d_mods, c.d_P_mod_q, db);
    return launched("k_key_finish");
}

size_t decrypt_ws(const Ctx& c, u32 count) { return (size_t)count * (c.L + 1) * c.N * sizeof(u64); }

int decrypt(const Ctx& c, const u64* sk, const u64* ct, u32 count, u32* slots, u64* ws,
            cudaStream_t st) {
    if (count == 0) return PDQ_OK;
    const u64 LN = (u64)c.L * c.N;
    u64* x = ws;
    u64* m = ws + count * LN;
    k_dec_inner<<<grid_for(count * LN), kBlock, 0, st>>>(ct, sk, count, c.N, c.L, c.d_mods, x);
    PDQ_TRY(launched("k_dec_inner"));
    PDQ_TRY(ntt_inverse(c, x, count, c.L, 0, LN, st));
    k_dec_round<<<grid_for((u64)count * c.N), kBlock, 0, st>>>(
        x, count, c.N, c.L, c.d_mods, c.d_dec_omega, c.d_dec_omega_shoup, c.t, m);
    PDQ_TRY(launched("k_dec_round"));
    PDQ_TRY(ntt_forward(c, m, count, 1, c.nmod - 1, c.N, st));
    k_gather_slots<<<grid_for((u64)count * c.N), kBlock, 0, st>>>(m, count, c.N, c.d_slot_pos, slots);
    return launched("k_gather_slots");
}

int mask(const Ctx& c, u32 J, const u64* v, const u64* db, u64* out, cudaStream_t st) {
    k_mask<<<grid_for((u64)J * c.L * c.N), kBlock, 0, st>>>(v, db, c.d_rowmask, J, c.L, c.N,
                                                             c.d_mods, out);
    return launched("k_mask");
}

// ---- key switching pieces ---------------------------------------------------

size_t raise_ws(const Ctx& c, u32 cnt) {
    const u64 E = c.L + c.K;
    return (size_t)cnt * ((u64)c.L + (u64)c.ndigits * E) * c.N * sizeof(u64);
}

int ks_raise(const Ctx& c, CtSet in, u32 cnt, u64* ws, u64** D_out, cudaStream_t st) {
    const u64 N = c.N, L = c.L, E = c.L + c.K, nd = c.ndigits;
    u64* X = ws;
    u64* D = ws + cnt * L * N;
    // c1 of every ciphertext -> X, then coefficient form
    PDQ_TRY(gather_rows(in, (long long)(L * N), cnt, L * N, X, L * N, st));
    PDQ_TRY(ntt_inverse(c, X, cnt, c.L, 0, L * N, st));
    k_modup<<<grid_for((u64)cnt * nd * N), kBlock, 0, st>>>(
        X, in, cnt, c.N, c.L, (u32)E, (u32)nd, c.alpha, c.d_mods, c.d_up_hatinv,
        c.d_up_hatinv_shoup, c.d_up_hatmod, D);
    PDQ_TRY(launched("k_modup"));
    for (u32 b = 0; b < nd; ++b) {
        const u32 lo = c.digit_limbs[b].front(), hi = c.digit_limbs[b].back() + 1;
        u64* Db = D + (u64)b * E * N;
        if (lo > 0) PDQ_TRY(ntt_forward(c, Db, cnt, lo, 0, nd * E * N, st));
        PDQ_TRY(ntt_forward(c, Db + (u64)hi * N, cnt, (u32)(E - hi), hi, nd * E * N, st));
    }
    *D_out = D;
    return PDQ_OK;
}

size_t apply_ws(const Ctx& c, u32 cnt) {
    const u64 E = c.L + c.K;
    return (size_t)cnt * (2 * E + 2 * (u64)c.L) * c.N * sizeof(u64);
}

int ks_apply(const Ctx& c, const u64* D, CtSet in, u32 cnt, u32 galois, const u64* key,
             CtSet out, CtSet add, u64* ws, cudaStream_t st) {
    const u64 N = c.N, L = c.L, K = c.K, E = L + K;
    u64* A = ws;
    u64* Cv = ws + cnt * 2 * E * N;
    k_ks_inner<<<grid_for((u64)cnt * E * N), kBlock, 0, st>>>(D, key, cnt, c.N, c.log_n, (u32)E,
                                                              c.ndigits, galois, c.d_mods, A);
    PDQ_TRY(launched("k_ks_inner"));
    PDQ_TRY(ntt_inverse(c, A + L * N, 2 * cnt, c.K, c.L, E * N, st));
    k_moddown_conv<<<grid_for((u64)cnt * 2 * N), kBlock, 0, st>>>(
        A, cnt, c.N, c.L, c.K, c.d_mods, c.d_dn_hatinv, c.d_dn_hatinv_shoup, c.d_dn_hatmod, Cv);
    PDQ_TRY(launched("k_moddown_conv"));
    PDQ_TRY(ntt_forward(c, Cv, 2 * cnt, c.L, 0, L * N, st));
    k_moddown_final<<<grid_for((u64)cnt * 2 * L * N), kBlock, 0, st>>>(
        A, Cv, in, out, add, cnt, c.N, c.log_n, c.L, c.K, galois, c.d_mods, c.d_dn_pinv,
        c.d_dn_pinv_shoup);
    return launched("k_moddown_final");
}

int diag_mac(const Ctx& c, const pdq_plan& pl, const u64* R, const u64* Dg, u64* acc,
             cudaStream_t st) {
    const dim3 grid = grid_for((u64)pl.G * 2 * c.L * c.N);
    switch (pl.giants) {
#define PDQ_GI(n) case n: k_diag_mac<n><<<grid, kBlock, 0, st>>>(R, Dg, pl.G, pl.hpg, pl.H, pl.B, c.L, c.N, c.d_mods, acc); break;
        PDQ_GI(1) PDQ_GI(2) PDQ_GI(4) PDQ_GI(8) PDQ_GI(16) PDQ_GI(32)
#undef PDQ_GI
        default: return fail(PDQ_E_PARAM, "diag_mac: giant-step count must be a power of two <= 32");
    }
    return launched("k_diag_mac");
}

int ct_add(const Ctx& c, CtSet y, CtSet x, u32 cnt, cudaStream_t st) {
    k_ct_add<<<grid_for((u64)cnt * 2 * c.L * c.N), kBlock, 0, st>>>(y, x, cnt, c.L, c.N, c.d_mods);
    return launched("k_ct_add");
}

int group_combine(const Ctx& c, const pdq_plan& pl, const u64* y, const u64* masks, u64* out,
                  cudaStream_t st) {
    k_group_combine<<<grid_for((u64)pl.n_out * 2 * c.L * c.N), kBlock, 0, st>>>(
        y, masks, pl.G, pl.per_out, pl.n_out, c.L, c.N, c.d_mods, out);
    return launched("k_group_combine");
}

}  // namespace pdq
