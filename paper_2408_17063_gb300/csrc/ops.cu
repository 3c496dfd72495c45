// Element-wise kernels of the PDQ path: slot encoding, key generation,
// encryption and decryption (client side), Mask, the pieces of hybrid key
// switching (raise, inner product with the automorphism, lower), the
// diagonal multiply-accumulate of Comp and the group combine.
//
// All kernels read and write canonical residues.  Products of two residues
// are formed as 128-bit values and reduced once (reduce128), or summed
// unreduced in a 128-bit accumulator first when several products meet.
// Launch shape: a 2-D (or 3-D) grid whose x dimension walks the N (or L*N,
// E*N) positions of one polynomial block in 256-thread CTAs and whose y/z
// dimensions enumerate ciphertexts, limbs or digits, so that every index is
// a shift or a mask of 32-bit values.
#include "pdq_internal.h"
#include "pdq_ops.h"

namespace pdq {

namespace {

constexpr u32 kBlock = 256;

inline dim3 grid2(u64 xlen, u32 y, u32 z = 1) {
    return dim3((u32)((xlen + kBlock - 1) / kBlock), y, z);
}

inline int check_y(u64 y, const char* what) {
    if (y == 0 || y > 65535) return fail(PDQ_E_PARAM, std::string(what) + ": batch size out of range");
    return PDQ_OK;
}

// Position holding a(psi^{e k}) for the position x that holds a(psi^e):
// sigma_k in the bit-reversed evaluation domain.  Aligned tiles of 2^i
// consecutive positions map onto aligned tiles (k is odd), so warps gather
// from one contiguous 256-byte span.
__device__ __forceinline__ u32 auto_index(u32 x, u32 k, u32 logN) {
    const u32 twoN_mask = (2u << logN) - 1;
    const u32 e = 2 * (__brev(x) >> (32 - logN)) + 1;
    const u32 e2 = (e * k) & twoN_mask;
    return __brev((e2 - 1) >> 1) >> (32 - logN);
}

// v -> v0 | v1 << 32 with v = v0 + v1 2^30 (the operand layout of k_diag_mac)
__device__ __forceinline__ u64 split30(u64 v) { return (v & 0x3fffffffull) | ((v >> 30) << 32); }

// asynchronous global -> shared copies (valid == false: zero fill)
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
    const u32 s = (u32)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem),
                 "r"(valid ? 16 : 0));
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const u32 s = (u32)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// ------------------------------------------------------------- encoding ----

// out[c][0][pos[idx]] = slots[c][idx] mod t
__global__ void k_scatter_slots(const u32* __restrict__ slots, u32 logN, u64 lstride,
                                const u32* __restrict__ pos, u64 t, u64* __restrict__ out) {
    const u32 idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (1u << logN)) return;
    const u32 c = blockIdx.y;
    out[c * lstride + pos[idx]] = slots[((u64)c << logN) + idx] % t;
}

// centred lift of limb 0 (mod t) to limbs 0..nlimbs-1 (limb 0 written last)
__global__ void k_lift(u64* __restrict__ out, u32 logN, u32 nlimbs, const Mod* __restrict__ mods,
                       u64 t) {
    const u32 x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= (1u << logN)) return;
    u64* base = out + (((u64)blockIdx.y * nlimbs) << logN) + x;
    const u64 v = base[0];
    const u64 half = (t - 1) / 2;
    for (int l = (int)nlimbs - 1; l >= 0; --l) {
        const u64 q = mods[l].q;
        base[(u64)l << logN] = v > half ? q - (t - v) : v;
    }
}

// Diagonal slot values D_{h,gB+a} rotated by -gB (both rows), scattered to
// transform positions; one plaintext (cls, g, a) per grid row.
// (plaintext pt = pt_base + y pt_stride goes to row y)
__global__ void k_diag_slots(u64* __restrict__ out, u32 giants, u32 B, u32 s_prime, u32 logN,
                             u32 L, const u32* __restrict__ pos, u64 t, u32 pt_base,
                             u32 pt_stride) {
    const u32 idx = blockIdx.x * blockDim.x + threadIdx.x;
    const u32 N = 1u << logN, m = N / 2;
    if (idx >= N) return;
    const u32 pt = pt_base + blockIdx.y * pt_stride;
    const u32 a = pt % B;
    const u32 g = (pt / B) % giants;
    const u32 cls = pt / (B * giants);
    const u32 col = idx & (m - 1);
    const u32 k = g * B + a;
    const u32 cp = (col + m - (g * B) % m) & (m - 1);        // Rot(.; -gB)
    const u64 node = (u64)cls * m + ((cp + k) & (m - 1)) + 1;
    u32 e = (cp & (s_prime - 1)) + 1;
    u64 r = 1, b = node % t;
    while (e) {
        if (e & 1) r = r * b % t;
        b = b * b % t;
        e >>= 1;
    }
    out[(((u64)blockIdx.y * L) << logN) + pos[idx]] = r;
}

// Diagonals of Comp in a subring after ring switching (ring ratio R): the
// block of half-block class cls = 2(R jj + r) + rho (part r of the jj-th big
// ciphertext of a group, row rho) is M[kk][c'] = W_{kk+1}[r][e'], with small
// slot exponent e' = (-1)^rho 3^c' mod 2N, e_u = e' + 2N u (u < R) and
// W_kk = sum_u alpha(jj Nbig + slot_of[e_u])^kk zeta_big^(e_u r): the power
// sums of Eq. 1 over the big ring's records, read through the fold
// m(zeta^e_u) = sum_r zeta^(e_u r) m_r(zeta'^e') of the split.
// slot_of[e]: big slot index of odd exponent e; zpow[i] = zeta_big^i mod t.
__global__ void k_diag_slots_sw(u64* __restrict__ out, u32 giants, u32 B, u32 s_prime, u32 logN,
                                u32 L, const u32* __restrict__ pos, u64 t, u32 pt_base,
                                u32 pt_stride, u32 R, const u32* __restrict__ slot_of,
                                const u32* __restrict__ zpow) {
    const u32 idx = blockIdx.x * blockDim.x + threadIdx.x;
    const u32 N = 1u << logN, m = N / 2;
    if (idx >= N) return;
    const u32 pt = pt_base + blockIdx.y * pt_stride;
    const u32 a = pt % B;
    const u32 g = (pt / B) % giants;
    const u32 cls = pt / (B * giants);
    const u32 col = idx & (m - 1);
    const u32 k = g * B + a;
    const u32 cp = (col + m - (g * B) % m) & (m - 1);        // Rot(.; -gB)
    const u32 cc = (cp + k) & (m - 1);
    const u32 kk = (cp & (s_prime - 1)) + 1;
    const u32 rho = cls & 1, i = cls >> 1, r = i % R, jj = i / R;
    const u64 twoN = 2ull * N, Nbig = (u64)N * R, twoNbig = 2 * Nbig;
    u64 e = 1, b3 = 3;
    for (u32 x = cc; x; x >>= 1) {
        if (x & 1) e = e * b3 % twoN;
        b3 = b3 * b3 % twoN;
    }
    if (rho) e = twoN - e;
    u64 acc = 0;
    for (u32 u = 0; u < R; ++u) {
        const u64 eu = e + twoN * u;
        const u64 node = ((u64)jj * Nbig + slot_of[eu] + 1) % t;
        u64 p = 1, bb = node;
        for (u32 x = kk; x; x >>= 1) {
            if (x & 1) p = p * bb % t;
            bb = bb * bb % t;
        }
        acc += p * zpow[(eu * r) % twoNbig] % t;
    }
    out[(((u64)blockIdx.y * L) << logN) + pos[idx]] = acc % t;
}

// Diagonals of the Answer on an unencrypted database, one plaintext (j,
// sigma, g, a) per grid row (pt = pt_base + y B, pt = ((2j + sigma) giants +
// g) B + a): row rho is the diagonal of
// half-block h = 2j + rho rotated by -gB, times the database record it meets
// on the row rho != sigma:
//   D[rho][c] = alpha(h m + c')^((cp mod s')+1) (DB[h m + c'] if rho != sigma),
// cp = (c - gB) mod m, c' = (cp + gB + a) mod m, alpha(i) = (i mod G_sz) + 1.
__global__ void k_diag_slots_db(u64* __restrict__ out, u32 giants, u32 B, u32 s_prime, u32 logN,
                                u32 L, const u32* __restrict__ pos, u64 t, u32 G_sz,
                                const u32* __restrict__ values, u64 n, u64 pt_base) {
    const u32 idx = blockIdx.x * blockDim.x + threadIdx.x;
    const u32 N = 1u << logN, m = N / 2;
    if (idx >= N) return;
    const u64 pt = pt_base + (u64)blockIdx.y * B;
    const u32 a = (u32)(pt % B);
    const u32 g = (u32)((pt / B) % giants);
    const u32 sigma = (u32)((pt / ((u64)B * giants)) & 1);
    const u64 j = pt / (2ull * B * giants);
    const u32 rho = idx >= m ? 1 : 0;
    const u32 col = idx & (m - 1);
    const u32 k = g * B + a;
    const u32 cp = (col + m - (g * B) % m) & (m - 1);
    const u64 rec = (2 * j + rho) * m + ((cp + k) & (m - 1));
    u32 e = (cp & (s_prime - 1)) + 1;
    u64 r = 1, b = (rec % G_sz + 1) % t;
    while (e) {
        if (e & 1) r = r * b % t;
        b = b * b % t;
        e >>= 1;
    }
    if (rho != sigma) r = r * (rec < n ? (u64)values[rec] % t : 0) % t;
    out[(((u64)blockIdx.y * L) << logN) + pos[idx]] = r;
}

// database plaintexts: row pt = 2j + half holds DB_j.[1;0] (half 0) or DB_j.[0;1]
__global__ void k_db_slots(u64* __restrict__ out, const u32* __restrict__ values, u64 n, u32 logN,
                           u32 L, const u32* __restrict__ pos, u64 t) {
    const u32 idx = blockIdx.x * blockDim.x + threadIdx.x;
    const u32 N = 1u << logN, m = N / 2;
    if (idx >= N) return;
    const u32 pt = blockIdx.y;
    const u64 j = pt >> 1;
    const u32 half = pt & 1;
    const u64 rec = (j << logN) + idx;
    const bool row_ok = (idx >= m) == (half == 1);
    const u64 v = (row_ok && rec < n) ? (u64)values[rec] % t : 0;
    out[(((u64)pt * L) << logN) + pos[idx]] = v;
}

// database plaintexts without row masks: plaintext j holds DB_j on both rows
__global__ void k_db_plain_slots(u64* __restrict__ out, const u32* __restrict__ values, u64 n,
                                 u32 logN, u32 L, const u32* __restrict__ pos, u64 t) {
    const u32 idx = blockIdx.x * blockDim.x + threadIdx.x;
    const u32 N = 1u << logN;
    if (idx >= N) return;
    const u64 j = blockIdx.y;
    const u64 rec = (j << logN) + idx;
    out[((j * L) << logN) + pos[idx]] = rec < n ? (u64)values[rec] % t : 0;
}

// group mask o: ones at slots [o s', (o+1) s') of both rows
__global__ void k_groupmask_slots(u64* __restrict__ out, u32 s_prime, u32 logN, u32 L,
                                  const u32* __restrict__ pos) {
    const u32 idx = blockIdx.x * blockDim.x + threadIdx.x;
    const u32 N = 1u << logN, m = N / 2;
    if (idx >= N) return;
    const u32 o = blockIdx.y;
    const u32 col = idx & (m - 1);
    out[(((u64)o * L) << logN) + pos[idx]] = (col / s_prime == o) ? 1 : 0;
}

// ------------------------------------------------------- keys / encryption -

// out[l][x] = s[x] mod (prime l), s small signed
template <class T>
__global__ void k_signed_to_rns(const T* __restrict__ s, u32 logN, const Mod* __restrict__ mods,
                                u64* __restrict__ out) {
    const u32 x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= (1u << logN)) return;
    const u32 l = blockIdx.y;
    const long long v = s[x];
    const u64 q = mods[l].q;
    out[((u64)l << logN) + x] = v < 0 ? q - (u64)(-v) : (u64)v;
}

// c0 = e + Delta * m (coefficient form); m read from limb 0 of c1
__global__ void k_enc_c0(u64* __restrict__ ct, const int32_t* __restrict__ e, u32 logN, u32 L,
                         const Mod* __restrict__ mods, const u64* __restrict__ delta) {
    const u32 x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= (1u << logN)) return;
    const u32 c = blockIdx.y;
    u64* c0 = ct + (((u64)c * 2 * L) << logN);
    const u64 m = c0[((u64)L << logN) + x];
    const int ev = e[((u64)c << logN) + x];
    for (u32 l = 0; l < L; ++l) {
        const Mod md = mods[l];
        const u64 ee = ev < 0 ? md.q - (u64)(-ev) : (u64)ev;
        c0[((u64)l << logN) + x] = addmod(mulmod(m, delta[l], md), ee, md.q);
    }
}

__global__ void k_copy_rows(u64* __restrict__ dst, u64 dst_stride, const u64* __restrict__ src,
                            u64 src_stride, u32 len) {
    const u32 x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= len) return;
    const u32 c = blockIdx.y;
    dst[c * dst_stride + x] = src[c * src_stride + x];
}

// c0 -= c1 * s (NTT form)
__global__ void k_enc_finish(u64* __restrict__ ct, const u64* __restrict__ sk, u32 logN, u32 L,
                             const Mod* __restrict__ mods) {
    const u32 r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= (L << logN)) return;
    const Mod md = mods[r >> logN];
    u64* c0 = ct + (((u64)blockIdx.y * 2 * L) << logN);
    const u64 as = mulmod(c0[((u64)L << logN) + r], sk[r], md);
    c0[r] = submod(c0[r], as, md.q);
}

// key: b = b(e) - a*s_to + [l in digit] P sigma_k(s_from), all NTT form
// (a rotation key: s_to = s_from = s; a ring-switching key: k = 1, s_from = s,
// s_to the subring's secret embedded)
__global__ void k_key_finish(u64* __restrict__ key, const u64* __restrict__ sk,
                             const u64* __restrict__ sk_from, u32 E, u32 logN,
                             u32 galois, const Mod* __restrict__ mods,
                             const u64* __restrict__ Pmodq, DigitBounds db) {
    const u32 r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= (E << logN)) return;
    const u32 b = blockIdx.y;
    const u32 l = r >> logN, x = r & ((1u << logN) - 1);
    const Mod md = mods[l];
    u64* kb = key + (((u64)b * 2 * E) << logN);
    const u64 av = kb[((u64)E << logN) + r];
    u64 v = submod(kb[r], mulmod(av, sk[r], md), md.q);
    if (l >= db.lo[b] && l < db.hi[b]) {
        const u64 sv = sk_from[((u64)l << logN) + auto_index(x, galois, logN)];
        v = addmod(v, mulmod(sv, Pmodq[l], md), md.q);
    }
    kb[r] = v;
}

// decryption: x = c0 + c1 s (NTT form) into ws
__global__ void k_dec_inner(const u64* __restrict__ ct, const u64* __restrict__ sk, u32 logN,
                            u32 L, const Mod* __restrict__ mods, u64* __restrict__ out) {
    const u32 r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= (L << logN)) return;
    const Mod md = mods[r >> logN];
    const u64* c0 = ct + (((u64)blockIdx.y * 2 * L) << logN);
    out[(((u64)blockIdx.y * L) << logN) + r] =
        addmod(c0[r], mulmod(c0[((u64)L << logN) + r], sk[r], md), md.q);
}

// m = round(sum_i [x_i omega_i]_{q_i} t / q_i) mod t  (x in coefficient form)
__global__ void k_dec_round(const u64* __restrict__ x, u32 logN, u32 L,
                            const Mod* __restrict__ mods, const u64* __restrict__ om,
                            const u64* __restrict__ oms, u64 t, u64* __restrict__ out) {
    const u32 xi = blockIdx.x * blockDim.x + threadIdx.x;
    if (xi >= (1u << logN)) return;
    const u64 c = blockIdx.y;
    u64 ip = 0;        // integer part
    u128 fr = 0;       // fractional part, 64-bit fixed point
    for (u32 l = 0; l < L; ++l) {
        const u64 q = mods[l].q;
        const u64 v = x[((c * L + l) << logN) + xi];
        const u64 b = csub(mul_shoup_lazy(v, om[l], oms[l], q), q);
        const u128 bt = (u128)b * t;
        const u64 quo = (u64)(bt / q);
        const u64 rem = (u64)(bt % q);
        ip += quo % t;
        fr += (u128)(u64)(((u128)rem << 64) / q);
    }
    const u64 whole = (u64)(fr >> 64);
    const u64 lo = (u64)fr;
    out[(c << logN) + xi] = (ip + whole + (lo >> 63)) % t;
}

__global__ void k_gather_slots(const u64* __restrict__ in, u32 logN, const u32* __restrict__ pos,
                               u32* __restrict__ slots) {
    const u32 idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (1u << logN)) return;
    const u64 c = blockIdx.y;
    slots[(c << logN) + idx] = (u32)in[(c << logN) + pos[idx]];
}

// ------------------------------------------------------------------ Mask ----

// out[j] = (v.[1;0], v.[0;1], v.(DB.[1;0]), v.(DB.[0;1]))
__global__ void k_mask(const u64* __restrict__ v, const u64* __restrict__ db,
                       const u64* __restrict__ rowmask, u32 L, u32 logN,
                       const Mod* __restrict__ mods, u64* __restrict__ out) {
    const u32 r = blockIdx.x * blockDim.x + threadIdx.x;
    const u64 LN = (u64)L << logN;
    if (r >= LN) return;
    const u64 j = blockIdx.y;
    const Mod md = mods[r >> logN];
    const u64 v0 = v[j * 2 * LN + r], v1 = v[j * 2 * LN + LN + r];
    const u64 pt[4] = {rowmask[r], rowmask[LN + r], db[j * 2 * LN + r], db[j * 2 * LN + LN + r]};
    u64* o = out + j * 8 * LN;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        o[(2 * k) * LN + r] = mulmod(v0, pt[k], md);
        o[(2 * k + 1) * LN + r] = mulmod(v1, pt[k], md);
    }
}

// Mask in the order of the u-packing remark: d = v.DB first, then the row
// masks: out[j] = (v.[1;0], v.[0;1], d.[1;0], d.[0;1])
__global__ void k_mask_literal(const u64* __restrict__ v, const u64* __restrict__ dbp,
                               const u64* __restrict__ rowmask, u32 L, u32 logN,
                               const Mod* __restrict__ mods, u64* __restrict__ out) {
    const u32 r = blockIdx.x * blockDim.x + threadIdx.x;
    const u64 LN = (u64)L << logN;
    if (r >= LN) return;
    const u64 j = blockIdx.y;
    const Mod md = mods[r >> logN];
    const u64 v0 = v[j * 2 * LN + r], v1 = v[j * 2 * LN + LN + r];
    const u64 pd = dbp[j * LN + r], top = rowmask[r], bot = rowmask[LN + r];
    const u64 d0 = mulmod(v0, pd, md), d1 = mulmod(v1, pd, md);
    u64* o = out + j * 8 * LN;
    o[0 * LN + r] = mulmod(v0, top, md);
    o[1 * LN + r] = mulmod(v1, top, md);
    o[2 * LN + r] = mulmod(v0, bot, md);
    o[3 * LN + r] = mulmod(v1, bot, md);
    o[4 * LN + r] = mulmod(d0, top, md);
    o[5 * LN + r] = mulmod(d1, top, md);
    o[6 * LN + r] = mulmod(d0, bot, md);
    o[7 * LN + r] = mulmod(d1, bot, md);
}

// Mask fused with the pack (w_j = Rot_col(v_j), NTT form):
//   u[2j]   = v_j.[1;0] + w_j.sigma_col(DB_j.[1;0])
//   u[2j+1] = w_j.[1;0] + v_j.(DB_j.[0;1])
// sigma_col of the NTT-form plaintext is a gather: position x takes the
// value at the position that holds the conjugate evaluation point.
__global__ void k_mask_pack(const u64* __restrict__ v, const u64* __restrict__ w,
                            const u64* __restrict__ db, const u64* __restrict__ rowmask, u32 L,
                            u32 logN, const Mod* __restrict__ mods, u32 Jq,
                            u64* __restrict__ u) {
    const u32 r = blockIdx.x * blockDim.x + threadIdx.x;
    const u64 LN = (u64)L << logN;
    if (r >= LN) return;
    const u64 j = blockIdx.y;
    const u64 jd = Jq == gridDim.y ? j : (u32)j % Jq;   // j's database plaintext in its query
    const u32 N = 1u << logN;
    const u32 l = r >> logN, x = r & (N - 1);
    const Mod md = mods[l];
    const u64 top = rowmask[r];
    const u64 pb = db[jd * 2 * LN + ((u64)l << logN) + auto_index(x, 2 * N - 1, logN)];
    const u64 pd = db[jd * 2 * LN + LN + r];
    u64* o = u + j * 4 * LN;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const u64 vp = v[j * 2 * LN + p * LN + r], wp = w[j * 2 * LN + p * LN + r];
        o[p * LN + r] = addmod(mulmod(vp, top, md), mulmod(wp, pb, md), md.q);
        o[(2 + p) * LN + r] = addmod(mulmod(wp, top, md), mulmod(vp, pd, md), md.q);
    }
}

// ---------------------------------------------------------- key switching --

// Raise digit b = blockIdx.y of c1 (coefficient form X [cnt][L][N]) of
// ciphertext blockIdx.z to the extended basis, multiplied by R = 2^64 mod r
// (so that the key inner products end with a Montgomery reduction): D[ct][b][r]
// for r outside the digit (coefficient form, transformed afterwards; hmod
// carries the factor R); inside the digit the NTT-form c1 limb times R.  Two adjacent positions per thread
// (16-byte accesses); the digit's conversion constants (Q_b/q_i) mod r and
// the target moduli are staged in shared memory.  ALPHA: primes per digit
// (0: read from `alpha` at run time, at most 8).
template <int ALPHA>
__global__ void __launch_bounds__(256) k_modup(const u64* __restrict__ X, CtSet c1ntt, u64 c1_off,
                                               u32 logN, u32 L, u32 E, u32 alpha,
                                               const Mod* __restrict__ mods,
                                               const u64* __restrict__ hinv,
                                               const u64* __restrict__ hinvs,
                                               const u64* __restrict__ hmod,
                                               const u64* __restrict__ hmods,
                                               u64* __restrict__ D) {
    __shared__ ulonglong2 sh[8 * 32];     // (hmod, Shoup) [l - lo][r]
    __shared__ ulonglong2 sq[32];         // (q, floor(2^64/q)) of target r
    const u32 b = blockIdx.y, nd = gridDim.y;
    const u32 lo = b * alpha, hi = min(lo + alpha, L);
    const u32 na = hi - lo;
    for (u32 i = threadIdx.x; i < na * E; i += blockDim.x) {
        const u32 l = lo + i / E, r = i - (i / E) * E;
        sh[(l - lo) * 32 + r] = make_ulonglong2(hmod[(u64)l * E + r], hmods[(u64)l * E + r]);
    }
    for (u32 r = threadIdx.x; r < E; r += blockDim.x) sq[r] = make_ulonglong2(mods[r].q, mods[r].ratio);
    __syncthreads();
    const u32 x = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (x >= (1u << logN)) return;
    const u64 ct = blockIdx.z;
    u64 y0[8], y1[8];
    const u64* Xc = X + ((ct * L) << logN) + x;
#pragma unroll
    for (u32 k = 0; k < (ALPHA ? (u32)ALPHA : 8u); ++k) {
        if (k < na) {
            const u32 l = lo + k;
            const u64 q = sq[l].x;
            const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(Xc + ((u64)l << logN));
            y0[k] = csub(mul_shoup_lazy(v.x, hinv[l], hinvs[l], q), q);
            y1[k] = csub(mul_shoup_lazy(v.y, hinv[l], hinvs[l], q), q);
        }
    }
    u64* Dc = D + (((ct * nd + b) * E) << logN) + x;
    const u64* src = c1ntt.at(ct) + c1_off + x;             // c1 of the input (NTT form)
    for (u32 r = 0; r < E; ++r) {
        u64* o = Dc + ((u64)r << logN);
        if (r >= lo && r < hi) {
            // the digit's own limb, multiplied by R = 2^64 mod q_r like the
            // converted ones (whose constants carry the factor)
            const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(src + ((u64)r << logN));
            const Mod mr = mods[r];
            *reinterpret_cast<ulonglong2*>(o) =
                make_ulonglong2(csub(mul_shoup_lazy(v.x, mr.r64, mr.r64_shoup, mr.q), mr.q),
                                csub(mul_shoup_lazy(v.y, mr.r64, mr.r64_shoup, mr.q), mr.q));
            continue;
        }
        // products by the constants (Q_b/q_i) mod r, Shoup: each in [0, 2r),
        // at most 8 of them, so the sums stay below 2^64
        const ulonglong2 m = sq[r];
        u64 s0 = 0, s1 = 0;
#pragma unroll
        for (u32 k = 0; k < (ALPHA ? (u32)ALPHA : 8u); ++k) {
            if (k < na) {
                const ulonglong2 h = sh[k * 32 + r];
                s0 += mul_shoup_lazy(y0[k], h.x, h.y, m.x);
                s1 += mul_shoup_lazy(y1[k], h.x, h.y, m.x);
            }
        }
        Mod md;
        md.q = m.x;
        md.ratio = m.y;
        *reinterpret_cast<ulonglong2*>(o) = make_ulonglong2(reduce64(s0, md), reduce64(s1, md));
    }
}

// A[ct][p][r][x] = sum_beta D[ct][beta][r][sigma(x)] * key[beta][p][r][x]
// Two adjacent positions per thread (16-byte loads and stores): sigma maps
// the aligned pair {x, x+1} onto an aligned pair, possibly swapped.
__global__ void k_ks_inner(const u64* __restrict__ D, const KeyTable kt, u64 koff, u32 logN,
                           u32 E, u32 nd, u32 galois, const Mod* __restrict__ mods,
                           u64* __restrict__ A) {
    const u32 r = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const u64 EN = (u64)E << logN;
    if (r >= EN) return;
    const u64 ct = blockIdx.y;
    const u64* __restrict__ key = kt.of((u32)ct) + koff;
    const u32 l = r >> logN, x = r & ((1u << logN) - 1);
    const u32 sx = auto_index(x, galois, logN);
    const bool swap = (sx & 1) != 0;                 // sigma(x) odd -> sigma(x+1) = sigma(x) - 1
    const u32 sr = (l << logN) + (sx & ~1u);
    u64 h0a = 0, l0a = 0, h1a = 0, l1a = 0, h0b = 0, l0b = 0, h1b = 0, l1b = 0;
    const u64* Dc = D + ct * nd * EN;
    for (u32 b = 0; b < nd; ++b) {
        const ulonglong2 dv = *reinterpret_cast<const ulonglong2*>(Dc + b * EN + sr);
        const u64 da = swap ? dv.y : dv.x, db = swap ? dv.x : dv.y;
        const ulonglong2 k0 = __ldg(reinterpret_cast<const ulonglong2*>(key + b * 2 * EN + r));
        const ulonglong2 k1 = __ldg(reinterpret_cast<const ulonglong2*>(key + b * 2 * EN + EN + r));
        mac128(h0a, l0a, da, k0.x);
        mac128(h0b, l0b, db, k0.y);
        mac128(h1a, l1a, da, k1.x);
        mac128(h1b, l1b, db, k1.y);
    }
    // the digits carry the factor R: one Montgomery reduction per output
    const Mod md = mods[l];
    *reinterpret_cast<ulonglong2*>(A + ct * 2 * EN + r) =
        make_ulonglong2(redc128(h0a, l0a, md), redc128(h0b, l0b, md));
    *reinterpret_cast<ulonglong2*>(A + ct * 2 * EN + EN + r) =
        make_ulonglong2(redc128(h1a, l1a, md), redc128(h1b, l1b, md));
}

// The rotation before its ModDown, in the extended basis: for output
// ciphertext ct, limb r < E, position x (two positions per thread)
//   out[ct][0][r] (+)= sum_beta D[ct][beta][r][s(x)] key[beta][0][r][x] + [r < L] P c0[ct][r][s(x)]
//   out[ct][1][r] (+)= sum_beta D[ct][beta][r][s(x)] key[beta][1][r][x]
// with s = sigma_k; `accumulate` adds into out instead of overwriting it.
__global__ void k_ks_inner_ext(const u64* __restrict__ D, const KeyTable kt, u64 koff, u32 logN,
                               u32 E, u32 c0_limbs, u32 nd, u32 galois,
                               const Mod* __restrict__ mods, CtSet c0src,
                               const u64* __restrict__ Pm, CtSet out, u32 accumulate, u32 split) {
    const u32 r = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const u64 EN = (u64)E << logN;
    if (r >= EN) return;
    const u64 ct = blockIdx.y;
    const u64* __restrict__ key = kt.of((u32)ct) + koff;
    const u32 l = r >> logN, x = r & ((1u << logN) - 1);
    const u32 sx = auto_index(x, galois, logN);
    const bool swap = (sx & 1) != 0;
    const u32 sr = (l << logN) + (sx & ~1u);
    u64 h0a = 0, l0a = 0, h1a = 0, l1a = 0, h0b = 0, l0b = 0, h1b = 0, l1b = 0;
    const u64* Dc = D + ct * nd * EN;
    for (u32 b = 0; b < nd; ++b) {
        const ulonglong2 dv = *reinterpret_cast<const ulonglong2*>(Dc + b * EN + sr);
        const u64 da = swap ? dv.y : dv.x, db = swap ? dv.x : dv.y;
        const ulonglong2 k0 = __ldg(reinterpret_cast<const ulonglong2*>(key + b * 2 * EN + r));
        const ulonglong2 k1 = __ldg(reinterpret_cast<const ulonglong2*>(key + b * 2 * EN + EN + r));
        mac128(h0a, l0a, da, k0.x);
        mac128(h0b, l0b, db, k0.y);
        mac128(h1a, l1a, da, k1.x);
        mac128(h1b, l1b, db, k1.y);
    }
    // P sigma(c0) joins the sum as c0 times P R (the digits carry R), then one
    // Montgomery reduction per output; a c0 over Q u P (Pm == nullptr, all
    // limbs) joins as c0 times R
    const Mod md = mods[l];
    if (l < c0_limbs) {
        const ulonglong2 cv = *reinterpret_cast<const ulonglong2*>(c0src.at(ct) + sr);
        const u64 ca = swap ? cv.y : cv.x, cb = swap ? cv.x : cv.y;
        const u64 cm = Pm ? Pm[l] : md.r64;
        mac128(h0a, l0a, ca, cm);
        mac128(h0b, l0b, cb, cm);
    }
    u64 a0 = redc128(h0a, l0a, md), b0 = redc128(h0b, l0b, md);
    u64 a1 = redc128(h1a, l1a, md), b1 = redc128(h1b, l1b, md);
    ulonglong2* o0 = reinterpret_cast<ulonglong2*>(out.at(ct) + r);
    ulonglong2* o1 = reinterpret_cast<ulonglong2*>(out.at(ct) + EN + r);
    if (accumulate) {
        const ulonglong2 p0 = *o0, p1 = *o1;
        a0 = addmod(a0, p0.x, md.q);
        b0 = addmod(b0, p0.y, md.q);
        a1 = addmod(a1, p1.x, md.q);
        b1 = addmod(b1, p1.y, md.q);
    }
    if (split) {
        a0 = split30(a0); b0 = split30(b0); a1 = split30(a1); b1 = split30(b1);
    }
    *o0 = make_ulonglong2(a0, b0);
    *o1 = make_ulonglong2(a1, b1);
}

// Galois elements and key offsets of the terms of one giant-step launch
struct GiantTerms {
    u64 koff[kMaxGiantTerms];   // element offset of term i's key in the key buffer
    u32 galois[kMaxGiantTerms];
};

// Every giant step of the BSGS sum in one launch, in the extended basis: for
// ciphertext ct (a record group), limb r < E, position x (two per thread)
//   out[ct][p][r][x] += sum_i ( sum_beta D_i[ct][beta][r][s_i(x)] key_i[beta][p][r][x]
//                               + [p = 0] c0_i[ct][r][s_i(x)] )
// with s_i = sigma_{galois_i}, c0 over Q u P and the raised digits carrying R.
// Each term is reduced once (Montgomery) and the reduced terms added mod q,
// so the result equals the one-launch-per-term accumulation bit for bit.
// Record groups are the fastest grid index: the groups at a position run
// together and read each term's key there once from DRAM.
__global__ void k_ks_giants(const u64* __restrict__ D, u64 d_term, u64 d_ct,
                            const KeyTable kt, GiantTerms tm, u32 T, u32 logN, u32 E,
                            u32 nd, const Mod* __restrict__ mods, const u64* __restrict__ c0,
                            u64 c0_term, u64 c0_ct, u64* __restrict__ out, u64 out_ct) {
    const u32 r = 2 * (blockIdx.y * blockDim.x + threadIdx.x);
    const u64 EN = (u64)E << logN;
    if (r >= EN) return;
    const u64 ct = blockIdx.x;
    const u32 l = r >> logN, x = r & ((1u << logN) - 1);
    const Mod md = mods[l];
    const u64* __restrict__ keys = kt.of((u32)ct);
    u64 s0a = 0, s0b = 0, s1a = 0, s1b = 0;
#pragma unroll 2
    for (u32 i = 0; i < T; ++i) {
        const u32 sx = auto_index(x, tm.galois[i], logN);
        const bool swap = (sx & 1) != 0;
        const u32 sr = (l << logN) + (sx & ~1u);
        const u64* Dc = D + i * d_term + ct * d_ct;
        const u64* key = keys + tm.koff[i];
        u64 h0a = 0, l0a = 0, h1a = 0, l1a = 0, h0b = 0, l0b = 0, h1b = 0, l1b = 0;
        for (u32 b = 0; b < nd; ++b) {
            const ulonglong2 dv = *reinterpret_cast<const ulonglong2*>(Dc + b * EN + sr);
            const u64 da = swap ? dv.y : dv.x, db = swap ? dv.x : dv.y;
            const ulonglong2 k0 = __ldg(reinterpret_cast<const ulonglong2*>(key + b * 2 * EN + r));
            const ulonglong2 k1 = __ldg(reinterpret_cast<const ulonglong2*>(key + b * 2 * EN + EN + r));
            mac128(h0a, l0a, da, k0.x);
            mac128(h0b, l0b, db, k0.y);
            mac128(h1a, l1a, da, k1.x);
            mac128(h1b, l1b, db, k1.y);
        }
        const ulonglong2 cv =
            *reinterpret_cast<const ulonglong2*>(c0 + i * c0_term + ct * c0_ct + sr);
        mac128(h0a, l0a, swap ? cv.y : cv.x, md.r64);
        mac128(h0b, l0b, swap ? cv.x : cv.y, md.r64);
        s0a = addmod(s0a, redc128(h0a, l0a, md), md.q);
        s0b = addmod(s0b, redc128(h0b, l0b, md), md.q);
        s1a = addmod(s1a, redc128(h1a, l1a, md), md.q);
        s1b = addmod(s1b, redc128(h1b, l1b, md), md.q);
    }
    ulonglong2* o0 = reinterpret_cast<ulonglong2*>(out + ct * out_ct + r);
    ulonglong2* o1 = reinterpret_cast<ulonglong2*>(out + ct * out_ct + EN + r);
    const ulonglong2 p0 = *o0, p1 = *o1;
    *o0 = make_ulonglong2(addmod(s0a, p0.x, md.q), addmod(s0b, p0.y, md.q));
    *o1 = make_ulonglong2(addmod(s1a, p1.x, md.q), addmod(s1b, p1.y, md.q));
}

// All hoisted baby-step rotations a = 1..B-1 of H ciphertexts in one launch,
// in the extended basis (the rotation before its ModDown), written in the
// split operand layout of the multiply-accumulate:
//   R[h][a][0][r][x] = sum_beta D[h][beta][r][s(x)] key_a[beta][0][r][x] + [r < L] P c0_h[r][s(x)]
//   R[h][a][1][r][x] = sum_beta D[h][beta][r][s(x)] key_a[beta][1][r][x],   s = sigma_{3^a}.
// A CTA owns the aligned input tile Y = [y0, y0+T) of limb r for HC
// ciphertexts: it stages their raised digits (and c0) at Y in shared memory
// once; sigma_{3^a} maps the aligned output tile X_a = sigma^{-1}(Y) onto Y,
// so for every a it reads the key tile at X_a, computes all outputs of X_a
// and writes them as contiguous runs.
// Exact sums of up to 8 products of 60-bit operands from their 30-bit halves
// (v = v0 + v1 2^30), Karatsuba: S00 = sum a0 b0, S11 = sum a1 b1 and
// Sm = sum (a0 + a1)(b0 + b1) mod 2^64, each a 64-bit sum of 32x32-bit
// products (one mad.lo.cc / madc.hi carry chain each).  With at most 8
// terms S00, S11 < 8 2^60 = 2^63 and the cross sum Sm - S00 - S11 =
// sum (a0 b1 + a1 b0) < 16 (2^30 - 1)^2 < 2^64, so all three are exact.
struct Kara64 {
    u32 l00, h00, lm, hm, l11, h11;
};

__device__ __forceinline__ void kmac(Kara64& s, u32 a0, u32 a1, u32 as, u32 b0, u32 b1, u32 bs) {
    asm("mad.lo.cc.u32 %0, %6, %9, %0;\n\t"
        "madc.hi.u32 %1, %6, %9, %1;\n\t"
        "mad.lo.cc.u32 %2, %8, %11, %2;\n\t"
        "madc.hi.u32 %3, %8, %11, %3;\n\t"
        "mad.lo.cc.u32 %4, %7, %10, %4;\n\t"
        "madc.hi.u32 %5, %7, %10, %5;"
        : "+r"(s.l00), "+r"(s.h00), "+r"(s.lm), "+r"(s.hm), "+r"(s.l11), "+r"(s.h11)
        : "r"(a0), "r"(a1), "r"(as), "r"(b0), "r"(b1), "r"(bs));
}

// The summed products as the 128-bit value S00 + (Sm - S00 - S11) 2^30 + S11 2^60.
__device__ __forceinline__ void kara_value(const Kara64& s, u64& hi, u64& lo) {
    const u64 s00 = ((u64)s.h00 << 32) | s.l00;
    const u64 sm = ((u64)s.hm << 32) | s.lm;
    const u64 s11 = ((u64)s.h11 << 32) | s.l11;
    const u64 c = sm - s00 - s11;
    lo = s00;
    hi = c >> 34;
    asm("add.cc.u64 %0, %0, %2;\n\t"
        "addc.u64 %1, %1, %3;\n\t"
        "add.cc.u64 %0, %0, %4;\n\t"
        "addc.u64 %1, %1, 0;"
        : "+l"(lo), "+l"(hi)
        : "l"(c << 30), "l"(s11 >> 4), "l"(s11 << 60));
}

struct BabyParams {
    u32 k[128];       // Galois element of Rot(.; a)
    u32 kinv[128];    // its inverse mod 2N
    u64 koff[128];    // element offset of key a in the key buffer
};

template <int T, int HC, int CPT, int ND>
__global__ void __launch_bounds__(T * HC / CPT) k_baby_ext(
        const u64* __restrict__ D, CtSet u, const KeyTable kt, u32 Hq, u32 zper, u64 zmagic,
        u32 B, u32 logN,
        u32 E, u32 L, u32 c1_limb, const Mod* __restrict__ mods, const u64* __restrict__ Pm,
        u64* __restrict__ Rx, const BabyParams bp, u32 ER) {
    // Rx holds ER limbs per polynomial ([..][2][ER][N]): a chunk of primes
    // when the caller advanced every other pointer to the chunk's first prime.
    // L: limbs of c0 (L for ciphertexts over Q, whose c0 joins as P c0 with
    // Pm = P R; L + K for ciphertexts over Q u P, Pm == nullptr: c0 joins as
    // c0 R, and a = 0 is the input itself); c1 starts at limb c1_limb
    // The digit tile (and c0) of HC ciphertexts is staged in shared memory
    // once and only read afterwards; every thread keeps the 2 ND key values of
    // its position in registers, loaded one rotation ahead, so the rotation
    // loop has no barrier.
    extern __shared__ __align__(16) u64 sm[];
    u64* Ds = sm;                       // [HC][ND][T]
    u64* Cs = Ds + HC * ND * T;         // [HC][T]: c0
    u64* C1s = Cs + HC * T;             // [HC][T]: c1 (for a = 0)
    // blockIdx.z: chunk of HC ciphertexts of one query (queries of Hq
    // ciphertexts each, zper chunks per query); the chunk's rotations use
    // that query's keys.  blockIdx.z / zper by the multiplier
    // zmagic = ceil(2^32 / zper), exact below 2^16 (a hardware division here
    // costs the kernel half its registers' worth of unrolling)
    const u32 qz = (u32)(((u64)blockIdx.z * zmagic) >> 32), chunk = blockIdx.z - qz * zper;
    const u32 y0 = blockIdx.x * T, r = blockIdx.y, h0 = qz * Hq + chunk * HC;
    const u32 H = qz * Hq + min(Hq, chunk * HC + HC);   // end of the chunk
    const u64* __restrict__ keys = kt.p[qz];
    const u64 EN = (u64)E << logN, ERN = (u64)ER << logN;
    const u32 nthreads = T * HC / CPT;
    constexpr u32 TP = T / 2;           // 16-byte chunks per row of a tile

    for (u32 e = threadIdx.x; e < HC * ND * TP; e += nthreads) {
        const u32 yy = (e % TP) * 2, rest = e / TP, b = rest % ND, ct = rest / ND;
        const u32 h = h0 + ct;
        cp_async16(Ds + (ct * ND + b) * T + yy,
                   D + ((u64)(h < H ? h : h0) * ND + b) * EN + ((u64)r << logN) + y0 + yy, h < H);
    }
    if (r < L) {
        for (u32 e = threadIdx.x; e < HC * TP; e += nthreads) {
            const u32 yy = (e % TP) * 2, ct = e / TP, h = h0 + ct;
            const u64* src = u.at(h < H ? h : h0) + ((u64)r << logN) + y0 + yy;
            cp_async16(Cs + ct * T + yy, src, h < H);
            cp_async16(C1s + ct * T + yy, src + ((u64)c1_limb << logN), h < H);
        }
    }
    cp_async_commit();

    const Mod md = mods[r];
    const u64 PR = r < L ? (Pm ? Pm[r] : md.r64) : 0;   // P 2^64 (or 2^64) mod q_r
    const u32 xi = threadIdx.x % T, hg = threadIdx.x / T;
    // key values of rotation a at this thread's position (the position whose
    // source lies in this tile)
    auto load_keys = [&](u32 a, u64 (&kv)[ND][2], u32& x) {
        x = (auto_index(y0, bp.kinv[a], logN) & ~(T - 1)) + xi;
        const u64* key = keys + bp.koff[a] + ((u64)r << logN) + x;
#pragma unroll
        for (int b = 0; b < ND; ++b) {
            kv[b][0] = __ldg(key + (u64)(2 * b) * EN);
            kv[b][1] = __ldg(key + (u64)(2 * b + 1) * EN);
        }
    };
    u64 kc[ND][2], kn[ND][2];
    u32 xc, xn = 0;
    load_keys(1, kc, xc);
    cp_async_wait<0>();
    __syncthreads();
    // a = 0: (P c0, P c1) over Q u P (zero on the special primes), or the
    // input itself when it is over Q u P (PR = R); each thread keeps the
    // P c0 it computed in the c0 tile, which every rotation adds after its
    // reduction
#pragma unroll
    for (int i = 0; i < CPT; ++i) {
        const u32 ct = hg * CPT + i, h = h0 + ct;
        if (h >= H) continue;
        u64 v0 = 0, v1 = 0;
        if (r < L) {
            u64 hi = 0, lo = 0;
            mac128(hi, lo, Cs[ct * T + xi], PR);
            v0 = redc128(hi, lo, md);
            hi = lo = 0;
            mac128(hi, lo, C1s[ct * T + xi], PR);
            v1 = redc128(hi, lo, md);
            Cs[ct * T + xi] = v0;
        }
        u64* o = Rx + ((u64)h * B * 2) * ERN + ((u64)r << logN) + y0 + xi;
        o[0] = split30(v0);
        o[ERN] = split30(v1);
    }
    // The rotations take Karatsuba sums of the 30-bit halves (at most 8
    // digit-key products per output): the digit tile goes to the split layout
    // in shared memory once, the keys once per rotation in registers.
    for (u32 e = threadIdx.x; e < HC * ND * T; e += nthreads) Ds[e] = split30(Ds[e]);
    __syncthreads();
    for (u32 a = 1; a < B; ++a) {
        if (a + 1 < B) load_keys(a + 1, kn, xn);
        const u32 y = auto_index(xc, bp.k[a], logN) - y0;  // in [0, T)
        u32 k0[ND][2], k1[ND][2], ks[ND][2];
#pragma unroll
        for (int b = 0; b < ND; ++b)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                k0[b][j] = (u32)kc[b][j] & 0x3fffffffu;
                k1[b][j] = (u32)(kc[b][j] >> 30);
                ks[b][j] = k0[b][j] + k1[b][j];
            }
#pragma unroll
        for (int i = 0; i < CPT; ++i) {
            const u32 ct = hg * CPT + i, h = h0 + ct;
            if (h >= H) continue;
            Kara64 s0 = {0, 0, 0, 0, 0, 0}, s1 = {0, 0, 0, 0, 0, 0};
#pragma unroll
            for (int b = 0; b < ND; ++b) {
                const u64 d = Ds[(ct * ND + b) * T + y];
                const u32 d0 = (u32)d, d1 = (u32)(d >> 32), ds = d0 + d1;
                kmac(s0, d0, d1, ds, k0[b][0], k1[b][0], ks[b][0]);
                kmac(s1, d0, d1, ds, k0[b][1], k1[b][1], ks[b][1]);
            }
            u64 hi, lo;
            kara_value(s0, hi, lo);
            u64 v0 = redc128(hi, lo, md);
            if (r < L) v0 = addmod(v0, Cs[ct * T + y], md.q);     // + P sigma(c0)
            kara_value(s1, hi, lo);
            const u64 v1 = redc128(hi, lo, md);
            u64* o = Rx + (((u64)h * B + a) * 2) * ERN + ((u64)r << logN) + xc;
            o[0] = split30(v0);
            o[ERN] = split30(v1);
        }
#pragma unroll
        for (int b = 0; b < ND; ++b) { kc[b][0] = kn[b][0]; kc[b][1] = kn[b][1]; }
        xc = xn;
    }
}

// (P c0, P c1) over Q u P from a ciphertext over Q (special limbs 0); with
// `ext` the input is over Q u P already and is copied
__global__ void k_times_P(CtSet in, u32 logN, u32 L, u32 E, const Mod* __restrict__ mods,
                          const u64* __restrict__ Pq, const u64* __restrict__ Pqs, CtSet out,
                          u32 split, u32 ext) {
    const u32 rr = blockIdx.x * blockDim.x + threadIdx.x;     // over [2][E][N]
    const u32 EN = E << logN;
    if (rr >= 2 * EN) return;
    const u64 ct = blockIdx.y;
    const u32 p = rr >= EN ? 1 : 0;
    const u32 r = rr - p * EN;
    const u32 l = r >> logN;
    u64 v = 0;
    if (ext) {
        v = in.at(ct)[rr];
    } else if (l < L) {
        const u64 q = mods[l].q;
        v = csub(mul_shoup_lazy(in.at(ct)[(u64)p * (L << logN) + r], Pq[l], Pqs[l], q), q);
    }
    out.at(ct)[rr] = split ? split30(v) : v;
}

// out[h] = sum_{a < R} Rx[h][a] over Q u P, Rx in the split operand layout
// (v = v0 + v1 2^30 stored as v0 | v1 << 32), out canonical.  Two adjacent
// positions per thread; R <= 8, so the sum of R residues stays below 2^63.
__global__ void k_sum_split(const u64* __restrict__ Rx, u32 R, u32 logN, u32 E,
                            const Mod* __restrict__ mods, u64* __restrict__ out) {
    const u32 EN = E << logN;
    const u32 x = 2 * (blockIdx.x * blockDim.x + threadIdx.x);     // over [2][E][N]
    if (x >= 2 * EN) return;
    const u64 h = blockIdx.y;
    const u32 l = (x >= EN ? x - EN : x) >> logN;
    const u64* src = Rx + h * R * 2 * (u64)EN + x;
    u64 s0 = 0, s1 = 0;
    for (u32 a = 0; a < R; ++a) {
        const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(src + (u64)a * 2 * EN);
        s0 += (v.x & 0xffffffffull) + ((v.x >> 32) << 30);
        s1 += (v.y & 0xffffffffull) + ((v.y >> 32) << 30);
    }
    const Mod md = mods[l];
    *reinterpret_cast<ulonglong2*>(out + h * 2 * (u64)EN + x) =
        make_ulonglong2(reduce64(s0, md), reduce64(s1, md));
}

// Conv[cp][i] = sum_k [y_k (P/p_k)^-1]_{p_k} (P/p_k) mod q_i from the special
// limbs of A (coefficient form); cp = blockIdx.y = ct*2 + p
template <int KK>
__global__ void __launch_bounds__(256) k_moddown_conv(const u64* __restrict__ Asp, u64 sp_stride,
                                                      u32 logN, u32 L,
                                                      u32 K, const Mod* __restrict__ mods,
                                                      const u64* __restrict__ hinv,
                                                      const u64* __restrict__ hinvs,
                                                      const u64* __restrict__ hmod,
                                                      const u64* __restrict__ hmods,
                                                      u64* __restrict__ Cv) {
    // KK: special primes (0: K at run time, at most 8); two positions per
    // thread; constants (P/p_k) mod q_l and the moduli staged in shared memory
    __shared__ ulonglong2 sh[8 * 32];
    __shared__ ulonglong2 sq[40];
    const u32 E = L + K;
    for (u32 i = threadIdx.x; i < K * L; i += blockDim.x)
        sh[(i / L) * 32 + (i % L)] = make_ulonglong2(hmod[i], hmods[i]);
    for (u32 r = threadIdx.x; r < E; r += blockDim.x) sq[r] = make_ulonglong2(mods[r].q, mods[r].ratio);
    __syncthreads();
    const u32 x = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (x >= (1u << logN)) return;
    const u64 cp = blockIdx.y;
    const u64* a = Asp + cp * sp_stride + x;     // special limb k at a + k N
    u64 y0[8], y1[8];
#pragma unroll
    for (u32 k = 0; k < (KK ? (u32)KK : 8u); ++k) {
        if (k < K) {
            const u64 pk = sq[L + k].x;
            const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(a + ((u64)k << logN));
            y0[k] = csub(mul_shoup_lazy(v.x, hinv[k], hinvs[k], pk), pk);
            y1[k] = csub(mul_shoup_lazy(v.y, hinv[k], hinvs[k], pk), pk);
        }
    }
    u64* o = Cv + ((cp * L) << logN) + x;
    for (u32 l = 0; l < L; ++l) {
        const ulonglong2 m = sq[l];
        u64 s0 = 0, s1 = 0;
#pragma unroll
        for (u32 k = 0; k < (KK ? (u32)KK : 8u); ++k) {
            if (k < K) {
                const ulonglong2 h = sh[k * 32 + l];
                s0 += mul_shoup_lazy(y0[k], h.x, h.y, m.x);
                s1 += mul_shoup_lazy(y1[k], h.x, h.y, m.x);
            }
        }
        Mod md;
        md.q = m.x;
        md.ratio = m.y;
        *reinterpret_cast<ulonglong2*>(o + ((u64)l << logN)) =
            make_ulonglong2(reduce64(s0, md), reduce64(s1, md));
    }
}

__global__ void k_moddown_final(const u64* __restrict__ A, const u64* __restrict__ Cv,
                                CtSet in, CtSet out, CtSet add, u32 logN, u32 L, u32 K,
                                u32 galois, const Mod* __restrict__ mods,
                                const u64* __restrict__ pinv, const u64* __restrict__ pinvs) {
    // two adjacent positions per thread; sigma maps the aligned pair {x, x+1}
    // onto an aligned pair, possibly swapped
    const u32 rr = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const u32 LN = L << logN;
    if (rr >= 2 * LN) return;
    const u64 ct = blockIdx.y;
    const u32 E = L + K;
    const u32 p = rr >= LN ? 1 : 0;
    const u32 r = rr - p * LN;
    const u32 l = r >> logN, x = r & ((1u << logN) - 1);
    const u64 q = mods[l].q;
    const u64 pv = pinv[l], pvs = pinvs[l];
    const ulonglong2 a = *reinterpret_cast<const ulonglong2*>(A + (((ct * 2 + p) * E) << logN) + r);
    const ulonglong2 cv = *reinterpret_cast<const ulonglong2*>(Cv + (ct * 2 + p) * LN + r);
    u64 v0 = csub(mul_shoup_lazy(submod(a.x, cv.x, q), pv, pvs, q), q);
    u64 v1 = csub(mul_shoup_lazy(submod(a.y, cv.y, q), pv, pvs, q), q);
    if (p == 0 && in.base) {
        const u32 sx = auto_index(x, galois, logN);
        const ulonglong2 iv =
            *reinterpret_cast<const ulonglong2*>(in.at(ct) + ((u64)l << logN) + (sx & ~1u));
        const bool swap = (sx & 1) != 0;
        v0 = addmod(v0, swap ? iv.y : iv.x, q);
        v1 = addmod(v1, swap ? iv.x : iv.y, q);
    }
    if (add.base) {
        const ulonglong2 dv = *reinterpret_cast<const ulonglong2*>(add.at(ct) + rr);
        v0 = addmod(v0, dv.x, q);
        v1 = addmod(v1, dv.y, q);
    }
    *reinterpret_cast<ulonglong2*>(out.at(ct) + rr) = make_ulonglong2(v0, v1);
}

// out[i] = (A[i] - Cv[i]) P^-1 over Q for polynomials A[i] = A + i a_stride
// (NTT form, Q limbs first); two adjacent positions per thread
__global__ void k_moddown_final_poly(const u64* __restrict__ A, u64 a_stride,
                                     const u64* __restrict__ Cv, u64* __restrict__ out,
                                     u64 out_stride, u32 logN, u32 L,
                                     const Mod* __restrict__ mods, const u64* __restrict__ pinv,
                                     const u64* __restrict__ pinvs) {
    const u32 r = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const u32 LN = L << logN;
    if (r >= LN) return;
    const u64 i = blockIdx.y;
    const u32 l = r >> logN;
    const u64 q = mods[l].q;
    const u64 pv = pinv[l], pvs = pinvs[l];
    const ulonglong2 a = *reinterpret_cast<const ulonglong2*>(A + i * a_stride + r);
    const ulonglong2 cv = *reinterpret_cast<const ulonglong2*>(Cv + i * LN + r);
    *reinterpret_cast<ulonglong2*>(out + i * out_stride + r) =
        make_ulonglong2(csub(mul_shoup_lazy(submod(a.x, cv.x, q), pv, pvs, q), q),
                        csub(mul_shoup_lazy(submod(a.y, cv.y, q), pv, pvs, q), q));
}

// ----------------------------------------------------------- Comp kernels --

// Diagonal multiply-accumulate (the Pegasus inner sum):
//   acc[gamma][g][p][l][x] = sum_{hh} sum_{a<B} Dg[hh][a][l][x][g] * R[gamma hpg + hh][a][p][l][x]
// (giant index g = 0 is written to acc0[gamma][p], the others to acc[gamma][g-1][p])
//
// Arithmetic: residues are < 2^60, split into 30-bit halves v = v0 + v1 2^30
// (both operands arrive stored as v0 | v1 << 32, see split30).  A product
// a b = a0 b0 + (a0 b1 + a1 b0) 2^30 + a1 b1 2^60 takes three 32x32-bit
// products (Karatsuba): a0 b0, a1 b1 and (a0 + a1)(b0 + b1) < 2^62, whose
// difference from the other two is the middle term.  Each is accumulated as
// a carry chain into a 96-bit sum (low and high 32-bit halves, then a
// count of 64-bit overflows), so no sum needs renormalising within a tile;
// at the end of a position tile the sums are folded to
//   S00 + (Smid - S00 - S11) 2^30 + S11 2^60
// formed exactly in 128 bits and reduced once when an output sums at most
// 256 products (fold1), else as
//   S00 (1 - 2^30) + Smid 2^30 + S11 (2^60 - 2^30)   (mod q)
// from the three sums reduced separately (foldk).
//
// Work split: one CTA owns limb l = blockIdx.y, X consecutive positions and
// the (gamma, p) combinations of its z-slice; thread (xi, gs, ct) (position
// in the lowest bits) handles
// position x0 + xi, giant indices gs*GT .. gs*GT+GT-1 and the two
// polynomials p = 0, 1 of group gamma = (cbase + 2ct) / 2.  Per step
// (hh, a-chunk of BC) the CTA stages the diagonal tile
// Dg[hh][a0:a0+BC][l][x0:x0+X][:] (giant index innermost, rows padded by two
// words so that the 16-byte loads of a quarter warp hit distinct banks) and
// the rotated-ciphertext tile R[gamma hpg + hh][a0:a0+BC][p][l][x0:x0+X] of
// its combinations (stored [combination][a][x]) in shared memory with
// asynchronous 16-byte copies, double-buffered so that the next step's copies
// overlap this step's arithmetic; each diagonal value leaves DRAM once per
// z-slice and each rotated value once.
struct AccK {
    u32 x0, y0, z0;     // S00 = sum a0 b0
    u32 x1, y1, z1;     // Smid = sum (a0 + a1)(b0 + b1)
    u32 x2, y2, z2;     // S11 = sum a1 b1
};

__device__ __forceinline__ void mack(AccK& A, u32 a0, u32 a1, u32 as, u32 b0, u32 b1, u32 bs) {
    asm("mad.lo.cc.u32 %0, %9, %12, %0;\n\t"
        "madc.hi.cc.u32 %1, %9, %12, %1;\n\t"
        "addc.u32 %2, %2, 0;\n\t"
        "mad.lo.cc.u32 %3, %11, %14, %3;\n\t"
        "madc.hi.cc.u32 %4, %11, %14, %4;\n\t"
        "addc.u32 %5, %5, 0;\n\t"
        "mad.lo.cc.u32 %6, %10, %13, %6;\n\t"
        "madc.hi.cc.u32 %7, %10, %13, %7;\n\t"
        "addc.u32 %8, %8, 0;"
        : "+r"(A.x0), "+r"(A.y0), "+r"(A.z0), "+r"(A.x1), "+r"(A.y1), "+r"(A.z1), "+r"(A.x2),
          "+r"(A.y2), "+r"(A.z2)
        : "r"(a0), "r"(a1), "r"(as), "r"(b0), "r"(b1), "r"(bs));
}

// The accumulated value mod q; ck = (1 - 2^30, 2^30, 2^60 - 2^30) mod q with
// Shoup companions.
__device__ __forceinline__ u64 foldk(const AccK& A, const Mod& md, const u64* __restrict__ ck) {
    const u64 q = md.q;
    const u64 v00 = reduce128(A.z0, ((u64)A.y0 << 32) | A.x0, md);
    const u64 vm = reduce128(A.z1, ((u64)A.y1 << 32) | A.x1, md);
    const u64 v11 = reduce128(A.z2, ((u64)A.y2 << 32) | A.x2, md);
    u64 v = mul_shoup_lazy(v00, ck[0], ck[1], q);                  // [0, 2q)
    v += mul_shoup_lazy(vm, ck[2], ck[3], q);                       // [0, 4q)
    v += mul_shoup_lazy(v11, ck[4], ck[5], q);                      // [0, 6q) < 2^63
    return reduce64(v, md);
}

// The accumulated value mod q when it sums at most 256 products of residues
// below 2^60: S = S00 + (Smid - S00 - S11) 2^30 + S11 2^60 < 256 (2^60)^2 =
// 2^128 is formed exactly in 128 bits and reduced once.
__device__ __forceinline__ u64 fold1(const AccK& A, const Mod& md) {
    const u128 s00 = ((u128)A.z0 << 64) | ((u128)A.y0 << 32) | A.x0;
    const u128 sm = ((u128)A.z1 << 64) | ((u128)A.y1 << 32) | A.x1;
    const u128 s11 = ((u128)A.z2 << 64) | ((u128)A.y2 << 32) | A.x2;
    const u128 s = s00 + ((sm - s00 - s11) << 30) + (s11 << 60);
    return reduce128((u64)(s >> 64), (u64)s, md);
}

struct MacArgs {
    u32 G, hpg, H, B, GI, E, logN;  // G: groups of the launch; H: half-blocks per query
    u32 Gq;                        // groups per query (queries answered together)
    u64 Gq_magic;                  // ceil(2^32 / Gq): gm / Gq = (gm Gq_magic) >> 32
    u32 ER;                        // primes per polynomial in R (a chunk, or E)
    u32 logX, logGS, logGI, CPC;   // CPC: combinations per CTA (even)
    u32 tiles_per_cta, achunks;
    u32 fold_one;                  // at most 256 products per output: fold1
};

// STACKED: the groups belong to several queries (of a.Gq groups and a.H
// half-blocks each); one query's launch keeps the plain index arithmetic.
template <int GT, int BC, int PC, bool STACKED>
__global__ void __launch_bounds__(256, 2) k_diag_mac(const u64* __restrict__ R,
                                                  const u64* __restrict__ Dg, MacArgs a,
                                                  const Mod* __restrict__ mods,
                                                  const u64* __restrict__ ckar,
                                                  u64* __restrict__ acc0,
                                                  u64* __restrict__ acc) {
    extern __shared__ __align__(16) u64 smem[];
    const u32 X = 1u << a.logX, GI = a.GI, GIp = GI + 2, CPC = a.CPC;
    const u32 l = blockIdx.y;
    // position in the low thread bits: the 8 threads of a quarter-warp read
    // the diagonal rows of 8 positions (row stride GI + 2 words), whose
    // 16-byte loads fall in distinct banks, and write 8 consecutive outputs
    const u32 xi = threadIdx.x & (X - 1);
    const u32 gs = (threadIdx.x >> a.logX) & ((1u << a.logGS) - 1);
    const u32 ct = threadIdx.x >> (a.logGS + a.logX);
    const u32 cbase = blockIdx.z * CPC;
    const u64 N = 1ull << a.logN;
    const u64 LN = (u64)a.E << a.logN;
    const u32 hpg_eff = min(a.hpg, a.H);
    const u32 g0 = gs * GT;

    const u32 RB = BC * X + 2;                     // words per combination block (padded)
    const u32 dwords = BC * X * GIp, rwords = CPC * RB;
    const u32 stage = dwords + rwords;

    const u32 c0 = PC * ct;                        // first combination of this thread (in slice)

    const u32 spt = hpg_eff * a.achunks;           // steps per position tile
    const u32 steps = spt * a.tiles_per_cta;
    // position tiles blockIdx.x, blockIdx.x + gridDim.x, ... (round robin)

    // copies of step (tt, hh, ac) into stage buffer `buf`
    auto issue = [&](u32 tt, u32 hh, u32 ac, u32 buf) {
        const u32 a0 = ac * BC;
        const u64 x0 = (u64)(blockIdx.x + tt * gridDim.x) << a.logX;
        u64* D = smem + buf * stage;
        const u64* dsrc = Dg + (((u64)hh * a.B + a0) * a.E + l) * N * GI + x0 * GI;
        if (GI >= 2) {
            const u32 halfGI = GI >> 1;
            for (u32 e = threadIdx.x; e < BC * X * halfGI; e += blockDim.x) {
                const u32 gp = e & (halfGI - 1);
                const u32 x = (e >> (a.logGI - 1)) & (X - 1);
                const u32 ai = e >> (a.logGI - 1 + a.logX);
                cp_async16(D + (ai * X + x) * GIp + 2 * gp,
                           dsrc + (u64)ai * LN * GI + (u64)x * GI + 2 * gp, true);
            }
        } else {
            for (u32 e = threadIdx.x; e < BC * X; e += blockDim.x) {
                const u32 x = e & (X - 1), ai = e >> a.logX;
                cp_async8(D + (ai * X + x) * GIp, dsrc + (u64)ai * LN + x);
            }
        }
        u64* Rt = D + dwords;
        const u32 halfX = X >> 1;
        for (u32 e = threadIdx.x; e < BC * CPC * halfX; e += blockDim.x) {
            const u32 xp = e & (halfX - 1);
            const u32 row = e >> (a.logX - 1);     // cb * BC + ai
            const u32 cb = row / BC, ai = row & (BC - 1);
            const u32 combo = cbase + cb;
            const u32 gm = combo >> 1, p = combo & 1;
            // group gm is group gl of query qz, whose half-blocks start at qz H
            u32 h;
            bool valid;
            if constexpr (!STACKED) {
                h = gm * a.hpg + hh;
                valid = gm < a.G && h < a.H;
            } else {
                const u32 qz = (u32)(((u64)gm * a.Gq_magic) >> 32), gl = gm - qz * a.Gq;
                const u32 hl = gl * a.hpg + hh;
                valid = gm < a.G && hl < a.H;
                h = qz * a.H + hl;
            }
            const u64* src = R + ((((u64)(valid ? h : 0) * a.B + a0 + ai) * 2 + p) * a.ER + l) * N +
                             x0 + 2 * xp;
            cp_async16(Rt + cb * RB + ai * X + 2 * xp, src, valid);
        }
        cp_async_commit();
    };

    AccK A[PC][GT];
#pragma unroll
    for (int p = 0; p < PC; ++p)
#pragma unroll
        for (int g = 0; g < GT; ++g) A[p][g] = AccK{0, 0, 0, 0, 0, 0, 0, 0, 0};

    u32 itt = 0, ihh = 0, iac = 0;                 // next step to issue
    auto advance = [&](u32& tt, u32& hh, u32& ac) {
        if (++ac == a.achunks) {
            ac = 0;
            if (++hh == hpg_eff) { hh = 0; ++tt; }
        }
    };
    u32 chh = 0, cac = 0, ctt = 0;                 // step being computed
    issue(itt, ihh, iac, 0);
    advance(itt, ihh, iac);
    for (u32 st = 0; st < steps; ++st) {
        const u32 buf = st & 1;
        if (st + 1 < steps) {
            issue(itt, ihh, iac, buf ^ 1);
            advance(itt, ihh, iac);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const u64* D = smem + buf * stage + xi * GIp + g0;
        const u64* Rt = smem + buf * stage + dwords + c0 * RB + xi;
#pragma unroll
        for (int ai = 0; ai < BC; ++ai) {
            u64 d[GT];
            if (GT >= 2) {
#pragma unroll
                for (int g = 0; g < GT; g += 2) {
                    const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(D + ai * X * GIp + g);
                    d[g] = v.x;
                    d[g + 1] = v.y;
                }
            } else {
                d[0] = D[ai * X * GIp];
            }
            u32 rl[PC], rh[PC], rs[PC];
#pragma unroll
            for (int p = 0; p < PC; ++p) {
                const u64 r = Rt[p * RB + ai * X];
                rl[p] = (u32)r;
                rh[p] = (u32)(r >> 32);
                rs[p] = rl[p] + rh[p];
            }
#pragma unroll
            for (int g = 0; g < GT; ++g) {
                const u32 d0 = (u32)d[g], d1 = (u32)(d[g] >> 32), ds = d0 + d1;
#pragma unroll
                for (int p = 0; p < PC; ++p) mack(A[p][g], rl[p], rh[p], rs[p], d0, d1, ds);
            }
        }
        const bool tile_end = (cac + 1 == a.achunks) && (chh + 1 == hpg_eff);
        if (tile_end) {                            // last step of this position tile
#pragma unroll
            for (int p = 0; p < PC; ++p) {
                const u32 combo = cbase + c0 + p;          // (gamma, polynomial)
                const u32 gam = combo >> 1, poly = combo & 1;
                if (c0 + p < CPC && gam < a.G) {
                    const Mod md = mods[l];
                    const u64 pos = ((u64)l << a.logN) + ((u64)(blockIdx.x + ctt * gridDim.x) << a.logX) + xi;
#pragma unroll
                    for (int g = 0; g < GT; ++g) {
                        const u32 gi = g0 + g;
                        u64* o = gi == 0 ? acc0 + ((u64)gam * 2 + poly) * LN + pos
                                         : acc + (((u64)gam * (GI - 1) + gi - 1) * 2 + poly) * LN + pos;
                        *o = a.fold_one ? fold1(A[p][g], md) : foldk(A[p][g], md, ckar + 8 * l);
                    }
                }
            }
#pragma unroll
            for (int p = 0; p < PC; ++p)
#pragma unroll
                for (int g = 0; g < GT; ++g) A[p][g] = AccK{0, 0, 0, 0, 0, 0, 0, 0, 0};
        }
        advance(ctt, chh, cac);
        __syncthreads();                 // buffer `buf` is refilled by the next issue
    }
}

// out[l][x][g] = split30(in[g][l][x]) for the GI diagonals of one (class, a)
__global__ void k_diag_layout(const u64* __restrict__ in, u64* __restrict__ out, u32 GI,
                              u64 LN) {
    const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= LN) return;
    for (u32 g = 0; g < GI; ++g) out[i * GI + g] = split30(in[(u64)g * LN + i]);
}

// y[ct] += x[ct] (ciphertexts)
__global__ void k_ct_add(CtSet y, CtSet x, u32 L, u32 logN, const Mod* __restrict__ mods) {
    const u32 rr = blockIdx.x * blockDim.x + threadIdx.x;
    const u32 LN = L << logN;
    if (rr >= 2 * LN) return;
    const u64 c = blockIdx.y;
    const u64 q = mods[(rr >= LN ? rr - LN : rr) >> logN].q;
    u64* yp = y.at(c);
    yp[rr] = addmod(yp[rr], x.at(c)[rr], q);
}

// out[c] = sum_o M_o * y[c per_out + o]
__global__ void k_group_combine(const u64* __restrict__ y, const u64* __restrict__ masks, u32 G,
                                u32 per_out, u32 n_out, u32 L, u32 logN,
                                const Mod* __restrict__ mods, u64* __restrict__ out) {
    // output c is output cl of query qz (n_out outputs and G groups per query)
    const u32 rr = blockIdx.x * blockDim.x + threadIdx.x;
    const u32 LN = L << logN;
    if (rr >= 2 * LN) return;
    const u64 c = blockIdx.y;
    const u64 qz = c / n_out, cl = c - qz * n_out;
    const u32 r = rr >= LN ? rr - LN : rr;
    const Mod md = mods[r >> logN];
    u64 ah = 0, al = 0;
    for (u32 o = 0; o < per_out; ++o) {
        const u64 gl = cl * per_out + o;
        if (gl >= G) break;
        const u64 gamma = qz * G + gl;
        if ((o & 127) == 127) { al = reduce128(ah, al, md); ah = 0; }
        mac128(ah, al, masks[(u64)o * LN + r], y[gamma * 2 * LN + rr]);
    }
    out[c * 2 * LN + rr] = reduce128(ah, al, md);
}

__global__ void k_gather_set(CtSet src, long long off, u64 len, u64* __restrict__ dst,
                             u64 dst_stride) {
    const u64 x = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= len) return;
    const u64 c = blockIdx.y;
    dst[c * dst_stride + x] = src.at(c)[off + (long long)x];
}

}  // namespace

// ================================================================ launchers ==

int encode_finish(const Ctx& c, u64* out, u32 count, u32 nlimbs, cudaStream_t st) {
    const u64 N = c.N;
    PDQ_TRY(check_y(count, "encode"));
    PDQ_TRY(ntt_inverse(c, out, count, 1, c.nmod - 1, (u64)nlimbs * N, st));
    k_lift<<<grid2(N, count), kBlock, 0, st>>>(out, c.log_n, nlimbs, c.d_mods, c.t);
    PDQ_TRY(launched("k_lift"));
    return ntt_forward(c, out, count, nlimbs, 0, (u64)nlimbs * N, st);
}

int encode_slots(const Ctx& c, const u32* slots, u32 count, u32 nlimbs, u64* out,
                 cudaStream_t st) {
    if (count == 0) return PDQ_OK;
    if (nlimbs < 1 || nlimbs > c.L + c.K) return fail(PDQ_E_PARAM, "encode: bad limb count");
    PDQ_TRY(check_y(count, "encode"));
    k_scatter_slots<<<grid2(c.N, count), kBlock, 0, st>>>(slots, c.log_n, (u64)nlimbs * c.N,
                                                          c.d_slot_pos, c.t, out);
    PDQ_TRY(launched("k_scatter_slots"));
    return encode_finish(c, out, count, nlimbs, st);
}

int build_diagonals(const Ctx& c, const pdq_plan& pl, u64* out, cudaStream_t st) {
    // over every prime of Q u P: the products are taken in the extended basis.
    // Plaintext (cls, g, a) is encoded in a temporary, then stored at
    // out[cls][a][l][x][g] in the operand format of the multiply-accumulate.
    const u32 GI = pl.giants, B = pl.B, E = c.L + c.K;
    PDQ_TRY(check_y(GI, "diagonals"));
    const u64 LN = (u64)E * c.N;
    const u32 R = pl.ring_ratio;
    u64* tmp = nullptr;
    u32* sw = nullptr;           // ring-switched plans: slot_of, then zpow ([2 Nbig] each)
    const u64 twoNbig = 2ull * c.N * R;
    if (cudaMallocAsync((void**)&tmp, (size_t)GI * LN * sizeof(u64), st) != cudaSuccess ||
        (R > 1 && cudaMallocAsync((void**)&sw, 2 * twoNbig * sizeof(u32), st) != cudaSuccess)) {
        cudaGetLastError();
        if (tmp) cudaFreeAsync(tmp, st);
        return fail(PDQ_E_NOMEM, "diagonals: temporary allocation failed");
    }
    if (R > 1) {
        // the big ring's slot index per odd exponent and the powers of its slot root
        std::vector<u32> tab(2 * twoNbig, 0);
        const u64 mbig = twoNbig / 4;
        u64 e = 1;
        for (u64 col = 0; col < mbig; ++col) {
            tab[e] = (u32)col;
            tab[twoNbig - e] = (u32)(mbig + col);
            e = e * 3 % twoNbig;
        }
        const u64 zb = host_powmod(c.gen, (c.t - 1) / twoNbig, c.t);
        u64 z = 1;
        for (u64 i = 0; i < twoNbig; ++i) {
            tab[twoNbig + i] = (u32)z;
            z = z * zb % c.t;
        }
        if (cudaMemcpyAsync(sw, tab.data(), tab.size() * sizeof(u32), cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            cudaFreeAsync(tmp, st);
            cudaFreeAsync(sw, st);
            return fail(PDQ_E_CUDA, "diagonals: table upload failed");
        }
    }
    int rc = PDQ_OK;
    for (u32 cls = 0; cls < pl.hclass && rc == PDQ_OK; ++cls) {
        for (u32 a = 0; a < B && rc == PDQ_OK; ++a) {
            if (R > 1) {
                k_diag_slots_sw<<<grid2(c.N, GI), kBlock, 0, st>>>(
                    tmp, GI, B, pl.s_prime, c.log_n, E, c.d_slot_pos, c.t, cls * GI * B + a, B, R,
                    sw, sw + twoNbig);
                rc = launched("k_diag_slots_sw");
            } else {
                k_diag_slots<<<grid2(c.N, GI), kBlock, 0, st>>>(tmp, GI, B, pl.s_prime, c.log_n, E,
                                                                c.d_slot_pos, c.t, cls * GI * B + a,
                                                                B);
                rc = launched("k_diag_slots");
            }
            if (rc == PDQ_OK) rc = encode_finish(c, tmp, GI, E, st);
            if (rc == PDQ_OK) {
                k_diag_layout<<<(u32)((LN + kBlock - 1) / kBlock), kBlock, 0, st>>>(
                    tmp, out + ((u64)cls * B + a) * GI * LN, GI, LN);
                rc = launched("k_diag_layout");
            }
        }
    }
    cudaFreeAsync(tmp, st);
    if (sw) cudaFreeAsync(sw, st);
    return rc;
}

int build_group_masks(const Ctx& c, const pdq_plan& pl, u64* out, cudaStream_t st) {
    PDQ_TRY(check_y(pl.per_out, "group masks"));
    k_groupmask_slots<<<grid2(c.N, pl.per_out), kBlock, 0, st>>>(out, pl.s_prime, c.log_n, c.L,
                                                                 c.d_slot_pos);
    PDQ_TRY(launched("k_groupmask_slots"));
    return encode_finish(c, out, pl.per_out, c.L, st);
}

int build_db_plain(const Ctx& c, const u32* values, u64 n, u32 J, u64* out, cudaStream_t st) {
    PDQ_TRY(check_y(J, "database"));
    k_db_plain_slots<<<grid2(c.N, J), kBlock, 0, st>>>(out, values, n, c.log_n, c.L, c.d_slot_pos,
                                                       c.t);
    PDQ_TRY(launched("k_db_plain_slots"));
    return encode_finish(c, out, J, c.L, st);
}

int mask_literal(const Ctx& c, u32 J, const u64* v, const u64* dbp, u64* out, cudaStream_t st) {
    PDQ_TRY(check_y(J, "mask"));
    k_mask_literal<<<grid2((u64)c.L * c.N, J), kBlock, 0, st>>>(v, dbp, c.d_rowmask, c.L, c.log_n,
                                                                c.d_mods, out);
    return launched("k_mask_literal");
}

int build_db(const Ctx& c, const u32* values, u64 n, u32 J, u64* out, cudaStream_t st) {
    PDQ_TRY(check_y(2ull * J, "database"));
    k_db_slots<<<grid2(c.N, 2 * J), kBlock, 0, st>>>(out, values, n, c.log_n, c.L, c.d_slot_pos,
                                                     c.t);
    PDQ_TRY(launched("k_db_slots"));
    return encode_finish(c, out, 2 * J, c.L, st);
}

int secret_prepare(const Ctx& c, const int8_t* s, u64* out, cudaStream_t st) {
    const u32 E = c.L + c.K;
    k_signed_to_rns<int8_t><<<grid2(c.N, E), kBlock, 0, st>>>(s, c.log_n, c.d_mods, out);
    PDQ_TRY(launched("k_signed_to_rns"));
    return ntt_forward(c, out, 1, E, 0, (u64)E * c.N, st);
}

int encrypt(const Ctx& c, const u64* sk, const u32* slots, u32 count, const u64* a,
            const int32_t* e, u64* ct, cudaStream_t st) {
    if (count == 0) return PDQ_OK;
    PDQ_TRY(check_y(count, "encrypt"));
    const u64 N = c.N, L = c.L, LN = L * N;
    // m mod t (coefficient form) into limb 0 of each c1
    k_scatter_slots<<<grid2(N, count), kBlock, 0, st>>>(slots, c.log_n, 2 * LN, c.d_slot_pos, c.t,
                                                        ct + LN);
    PDQ_TRY(launched("k_scatter_slots"));
    PDQ_TRY(ntt_inverse(c, ct + LN, count, 1, c.nmod - 1, 2 * LN, st));
    k_enc_c0<<<grid2(N, count), kBlock, 0, st>>>(ct, e, c.log_n, c.L, c.d_mods, c.d_delta_mod_q);
    PDQ_TRY(launched("k_enc_c0"));
    k_copy_rows<<<grid2(LN, count), kBlock, 0, st>>>(ct + LN, 2 * LN, a, LN, (u32)LN);
    PDQ_TRY(launched("k_copy_rows"));
    PDQ_TRY(ntt_forward(c, ct, 2 * count, c.L, 0, LN, st));
    k_enc_finish<<<grid2(LN, count), kBlock, 0, st>>>(ct, sk, c.log_n, c.L, c.d_mods);
    return launched("k_enc_finish");
}

int gather_rows(CtSet src, long long src_off, u32 cnt, u64 len, u64* dst, u64 dst_stride,
                cudaStream_t st) {
    PDQ_TRY(check_y(cnt, "gather"));
    k_gather_set<<<grid2(len, cnt), kBlock, 0, st>>>(src, src_off, len, dst, dst_stride);
    return launched("k_gather_set");
}

int rotkey_gen(const Ctx& c, const u64* sk, u64 galois, const u64* a, const int32_t* e, u64* key,
               cudaStream_t st) {
    return keygen(c, sk, sk, galois, a, e, key, st);
}

// s'(X) = s_small(X^R): out[R i] = s_small[i], zero elsewhere
__global__ void k_embed_secret(const int8_t* __restrict__ s_small, u32 R, u32 Nbig,
                               int8_t* __restrict__ out) {
    const u32 x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= Nbig) return;
    out[x] = (x % R == 0) ? s_small[x / R] : (int8_t)0;
}

int ring_switch_keygen(const Ctx& big, const u64* sk, const int8_t* s_small, u32 R, const u64* a,
                       const int32_t* e, u64* key, cudaStream_t st) {
    const u32 E = big.L + big.K;
    int8_t* emb = nullptr;
    u64* sk_to = nullptr;
    if (cudaMallocAsync((void**)&emb, big.N, st) != cudaSuccess ||
        cudaMallocAsync((void**)&sk_to, (size_t)E * big.N * sizeof(u64), st) != cudaSuccess) {
        cudaGetLastError();
        if (emb) cudaFreeAsync(emb, st);
        return fail(PDQ_E_NOMEM, "ring_switch_keygen: temporary allocation failed");
    }
    k_embed_secret<<<(big.N + kBlock - 1) / kBlock, kBlock, 0, st>>>(s_small, R, big.N, emb);
    int rc = launched("k_embed_secret");
    if (rc == PDQ_OK) rc = secret_prepare(big, emb, sk_to, st);
    if (rc == PDQ_OK) rc = keygen(big, sk_to, sk, 1, a, e, key, st);
    cudaFreeAsync(sk_to, st);
    cudaFreeAsync(emb, st);
    return rc;
}

// small ciphertext (i / group) group R + r group + i mod group, polynomial p,
// limb l, coefficient y = big ciphertext i, p, l, coefficient R y + r
__global__ void k_ring_split(const u64* __restrict__ in, u32 R, u32 logNs, u32 L, u32 group,
                             u64* __restrict__ out) {
    const u64 Ns = 1ull << logNs, per = 2ull * L * Ns;
    const u64 idx = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= per) return;
    const u32 i = blockIdx.y / R, r = blockIdx.y % R;
    const u64 pl = idx >> logNs, y = idx & (Ns - 1);
    const u64 o = (u64)(i / group) * group * R + (u64)r * group + i % group;
    out[o * per + idx] = in[(u64)i * per * R + pl * Ns * R + y * R + r];
}

int ring_split(const Ctx& small, const u64* in, u32 count, u32 R, u32 group, u64* out,
               cudaStream_t st) {
    if (group == 0 || count % group != 0) return fail(PDQ_E_PARAM, "ring_split: count must be a multiple of group");
    PDQ_TRY(check_y((u64)count * R, "ring_split"));
    k_ring_split<<<grid2(2ull * small.L * small.N, count * R), kBlock, 0, st>>>(in, R, small.log_n,
                                                                               small.L, group, out);
    return launched("k_ring_split");
}

int keygen(const Ctx& c, const u64* sk, const u64* sk_from, u64 galois, const u64* a,
           const int32_t* e, u64* key, cudaStream_t st) {
    const u32 E = c.L + c.K, nd = c.ndigits;
    const u64 EN = (u64)E * c.N;
    if (galois % 2 == 0 || galois >= 2ull * c.N) return fail(PDQ_E_PARAM, "galois element must be odd and < 2N");
    if (nd > 32) return fail(PDQ_E_PARAM, "at most 32 digits");
    // a into the second half of every digit, e (as residues) into the first
    k_copy_rows<<<grid2(EN, nd), kBlock, 0, st>>>(key + EN, 2 * EN, a, EN, (u32)EN);
    PDQ_TRY(launched("k_copy_rows"));
    for (u32 b = 0; b < nd; ++b) {
        k_signed_to_rns<int32_t><<<grid2(c.N, E), kBlock, 0, st>>>(e + (u64)b * c.N, c.log_n,
                                                                   c.d_mods, key + (u64)b * 2 * EN);
        PDQ_TRY(launched("k_signed_to_rns"));
    }
    PDQ_TRY(ntt_forward(c, key, 2 * nd, E, 0, EN, st));
    DigitBounds db{};
    for (u32 b = 0; b < nd; ++b) {
        db.lo[b] = c.digit_limbs[b].front();
        db.hi[b] = c.digit_limbs[b].back() + 1;
    }
    k_key_finish<<<grid2(EN, nd), kBlock, 0, st>>>(key, sk, sk_from, E, c.log_n, (u32)galois,
                                                   c.d_mods, c.d_P_mod_q, db);
    return launched("k_key_finish");
}

size_t decrypt_ws(const Ctx& c, u32 count) { return (size_t)count * (c.L + 1) * c.N * sizeof(u64); }

int decrypt(const Ctx& c, const u64* sk, const u64* ct, u32 count, u32* slots, u64* ws,
            cudaStream_t st) {
    if (count == 0) return PDQ_OK;
    PDQ_TRY(check_y(count, "decrypt"));
    const u64 LN = (u64)c.L * c.N;
    u64* x = ws;
    u64* m = ws + count * LN;
    k_dec_inner<<<grid2(LN, count), kBlock, 0, st>>>(ct, sk, c.log_n, c.L, c.d_mods, x);
    PDQ_TRY(launched("k_dec_inner"));
    PDQ_TRY(ntt_inverse(c, x, count, c.L, 0, LN, st));
    k_dec_round<<<grid2(c.N, count), kBlock, 0, st>>>(x, c.log_n, c.L, c.d_mods, c.d_dec_omega,
                                                      c.d_dec_omega_shoup, c.t, m);
    PDQ_TRY(launched("k_dec_round"));
    PDQ_TRY(ntt_forward(c, m, count, 1, c.nmod - 1, c.N, st));
    k_gather_slots<<<grid2(c.N, count), kBlock, 0, st>>>(m, c.log_n, c.d_slot_pos, slots);
    return launched("k_gather_slots");
}

int mask_pack(const Ctx& c, u32 J, const u64* v, const u64* w, const u64* db, u64* u,
              cudaStream_t st, u32 Jq) {
    PDQ_TRY(check_y(J, "mask"));
    k_mask_pack<<<grid2((u64)c.L * c.N, J), kBlock, 0, st>>>(v, w, db, c.d_rowmask, c.L, c.log_n,
                                                             c.d_mods, Jq ? Jq : J, u);
    return launched("k_mask_pack");
}

int mask(const Ctx& c, u32 J, const u64* v, const u64* db, u64* out, cudaStream_t st) {
    PDQ_TRY(check_y(J, "mask"));
    k_mask<<<grid2((u64)c.L * c.N, J), kBlock, 0, st>>>(v, db, c.d_rowmask, c.L, c.log_n, c.d_mods,
                                                        out);
    return launched("k_mask");
}

// ---- key switching pieces ---------------------------------------------------

// Cv[cp][l] = sum_k [A[cp][L+k] (P/p_k)^-1]_{p_k} (P/p_k) mod q_l (coefficient form)
// Conv of cps polynomials whose special limbs (coefficient form) start at
// Asp + cp * sp_stride, limb k at + k N
int moddown_conv(const Ctx& c, const u64* Asp, u64 sp_stride, u32 cps, u64* Cv, cudaStream_t st);

// whether ModDown's conversion rides on the forward transform (two-phase
// transforms, N > 2^11; at most 2 special primes)
bool moddown_fused(const Ctx& c) { return c.log_n > 11 && c.K >= 1 && c.K <= 2; }

// Cv [cps][L][N] (NTT form) = the conversion of the special limbs of cps
// polynomials (limb k of polynomial g at Sp + g sp_stride + k N) to the
// ciphertext primes.  inverse: Sp holds the special limbs in NTT form and
// is transformed in place first (else: coefficient form already, from an
// inverse transform with c.d_ninv_dn when moddown_fused(c)).
int moddown_to_ntt(const Ctx& c, u64* Sp, u64 sp_stride, u32 cps, u64* Cv, bool inverse,
                   cudaStream_t st) {
    const bool fuse = moddown_fused(c);
    if (inverse)
        PDQ_TRY(ntt_inverse(c, Sp, cps, c.K, c.L, sp_stride, st, fuse ? c.d_ninv_dn : nullptr));
    if (fuse) return ntt_forward_moddown(c, Cv, Sp, sp_stride, cps, st);
    PDQ_TRY(moddown_conv(c, Sp, sp_stride, cps, Cv, st));
    return ntt_forward(c, Cv, cps, c.L, 0, (u64)c.L * c.N, st);
}

int moddown_conv(const Ctx& c, const u64* Asp, u64 sp_stride, u32 cps, u64* Cv, cudaStream_t st) {
    if (c.K > 8 || c.L + c.K > 40 || c.L > 32) return fail(PDQ_E_PARAM, "ModDown: too many primes");
    PDQ_TRY(check_y(cps, "ModDown"));
    const dim3 grid((c.N / 2 + kBlock - 1) / kBlock, cps);
#define PDQ_CONV(KK)                                                                              \
    k_moddown_conv<KK><<<grid, kBlock, 0, st>>>(Asp, sp_stride, c.log_n, c.L, c.K, c.d_mods,       \
                                                c.d_dn_hatinv,                                     \
                                                c.d_dn_hatinv_shoup, c.d_dn_hatmod,                \
                                                c.d_dn_hatmod_shoup, Cv)
    switch (c.K) {
        case 1: PDQ_CONV(1); break;
        case 2: PDQ_CONV(2); break;
        case 3: PDQ_CONV(3); break;
        default: PDQ_CONV(0); break;
    }
#undef PDQ_CONV
    return launched("k_moddown_conv");
}

size_t raise_ws(const Ctx& c, u32 cnt) {
    const u64 E = c.L + c.K;
    return (size_t)cnt * ((u64)c.L + (u64)c.ndigits * E) * c.N * sizeof(u64);
}

int ks_raise(const Ctx& c, CtSet in, u32 cnt, u64* ws, u64** D_out, cudaStream_t st, u64 c1_off) {
    const u64 N = c.N, L = c.L, E = c.L + c.K, nd = c.ndigits;
    PDQ_TRY(check_y(cnt, "key switch"));
    if (c1_off == ~0ull) c1_off = L * N;
    u64* X = ws;
    u64* D = ws + cnt * L * N;
    if (c.log_n > 11 && c.alpha <= 2 && c.L % c.alpha == 0) {
        // the conversion folded into the transforms: the inverse transform of
        // c1 ends scaled by hat_inv_i (y_i into X), the digits' own limbs are
        // c1 R, and the forward transform of the other limbs converts from y
        // in its first phase (no converted copy of the digits is written)
        // (the own limbs, c1 R, written by the inverse transform as it reads c1)
        PDQ_TRY(ntt_inverse_from(c, in.base, in.outer, in.per, in.inner, c1_off, X, cnt, c.L,
                                 L * N, st, 0, c.d_ninv_up, D));
        PDQ_TRY(ntt_forward_digits_modup(c, D, X, cnt, (u32)nd, c.alpha, (u32)E, st));
        *D_out = D;
        return PDQ_OK;
    }
    // c1 of every ciphertext, coefficient form, into X (the transform reads
    // the set directly)
    PDQ_TRY(ntt_inverse_from(c, in.base, in.outer, in.per, in.inner, c1_off, X, cnt, c.L, L * N,
                             st));
    if (E > 32 || c.alpha > 8) return fail(PDQ_E_PARAM, "key switch: too many primes per digit");
    const dim3 grid((c.N / 2 + kBlock - 1) / kBlock, (u32)nd, cnt);
#define PDQ_MODUP(A)                                                                              \
    k_modup<A><<<grid, kBlock, 0, st>>>(X, in, c1_off, c.log_n, c.L, (u32)E, c.alpha, c.d_mods,    \
                                        c.d_up_hatinv, c.d_up_hatinv_shoup, c.d_up_hatmod_mont,    \
                                        c.d_up_hatmod_mont_shoup, D)
    switch (c.alpha) {
        case 1: PDQ_MODUP(1); break;
        case 2: PDQ_MODUP(2); break;
        case 3: PDQ_MODUP(3); break;
        case 4: PDQ_MODUP(4); break;
        default: PDQ_MODUP(0); break;
    }
#undef PDQ_MODUP
    PDQ_TRY(launched("k_modup"));
    if (c.L % c.alpha == 0) {
        // every digit alpha primes: one transform over all (ciphertext, digit)
        PDQ_TRY(ntt_forward_digits(c, D, cnt, (u32)nd, c.alpha, (u32)E, st));
    } else {
        for (u32 b = 0; b < nd; ++b) {
            const u32 lo = c.digit_limbs[b].front(), hi = c.digit_limbs[b].back() + 1;
            u64* Db = D + (u64)b * E * N;
            if (lo > 0) PDQ_TRY(ntt_forward(c, Db, cnt, lo, 0, nd * E * N, st));
            PDQ_TRY(ntt_forward(c, Db + (u64)hi * N, cnt, (u32)(E - hi), hi, nd * E * N, st));
        }
    }
    *D_out = D;
    return PDQ_OK;
}

size_t apply_ws(const Ctx& c, u32 cnt) {
    const u64 E = c.L + c.K;
    return (size_t)cnt * (2 * E + 2 * (u64)c.L) * c.N * sizeof(u64);
}

int ks_apply(const Ctx& c, const u64* D, CtSet in, u32 cnt, u32 galois, const u64* key,
             CtSet out, CtSet add, u64* ws, cudaStream_t st, const KeyTable* kt) {
    const u64 N = c.N, L = c.L, K = c.K, E = L + K;
    PDQ_TRY(check_y(2ull * cnt, "key switch"));
    u64* A = ws;
    u64* Cv = ws + cnt * 2 * E * N;
    const KeyTable t = kt ? *kt : single_keys(key);
    const u64 koff = kt ? (u64)(key - kt->p[0]) : 0;
    k_ks_inner<<<grid2(E * N / 2, cnt), kBlock, 0, st>>>(D, t, koff, c.log_n, (u32)E, c.ndigits,
                                                         galois, c.d_mods, A);
    PDQ_TRY(launched("k_ks_inner"));
    PDQ_TRY(moddown_to_ntt(c, A + L * N, E * N, 2 * cnt, Cv, true, st));
    k_moddown_final<<<grid2(L * N, cnt), kBlock, 0, st>>>(A, Cv, in, out, add, c.log_n, c.L,
                                                              c.K, galois, c.d_mods, c.d_dn_pinv,
                                                              c.d_dn_pinv_shoup);
    return launched("k_moddown_final");
}

int ks_apply_ext(const Ctx& c, const u64* D, CtSet c0src, u32 cnt, u32 galois, const u64* key,
                 CtSet out, bool accumulate, bool split, cudaStream_t st, bool c0_ext,
                 const KeyTable* kt) {
    const u64 N = c.N, E = c.L + c.K;
    PDQ_TRY(check_y(cnt, "key switch"));
    if (accumulate && split) return fail(PDQ_E_PARAM, "ks_apply_ext: cannot accumulate split output");
    const KeyTable t = kt ? *kt : single_keys(key);
    const u64 koff = kt ? (u64)(key - kt->p[0]) : 0;
    k_ks_inner_ext<<<grid2(E * N / 2, cnt), kBlock, 0, st>>>(
        D, t, koff, c.log_n, (u32)E, c0_ext ? (u32)E : c.L, c.ndigits, galois, c.d_mods, c0src,
        c0_ext ? nullptr : c.d_P_mont, out, accumulate ? 1u : 0u, split ? 1u : 0u);
    return launched("k_ks_inner_ext");
}

int ks_apply_giants(const Ctx& c, const u64* D, u32 cnt, u32 terms, const u64* galois,
                    const KeyTable& kt, const u64* key_offsets, const u64* c0, u64 c0_term,
                    u64 c0_ct, u64* out, u64 out_ct, cudaStream_t st) {
    if (terms == 0) return PDQ_OK;
    if (terms > kMaxGiantTerms) return fail(PDQ_E_PARAM, "giant steps: too many terms");
    if (cnt == 0 || cnt > 0x7fffffffu || (kt.per != ~0u && (cnt > 65535 || kt.per > 65535)))
        return fail(PDQ_E_PARAM, "giant steps: bad ciphertext count");
    const u64 N = c.N, E = c.L + c.K;
    const u64 dstride = (u64)c.ndigits * E * N;
    if ((E * N / 2 + 127) / 128 > 65535) return fail(PDQ_E_PARAM, "giant steps: ring too large");
    GiantTerms tm{};
    for (u32 i = 0; i < terms; ++i) {
        tm.koff[i] = key_offsets[i];
        tm.galois[i] = (u32)galois[i];
    }
    // 128-thread CTAs: at 90 registers a thread, five per SM (20 warps)
    // instead of two of 256 (16 warps) for this latency-bound gather
    constexpr u32 kGiantBlock = 128;
    const dim3 grid(cnt, (u32)((E * N / 2 + kGiantBlock - 1) / kGiantBlock));
    k_ks_giants<<<grid, kGiantBlock, 0, st>>>(D, (u64)cnt * dstride, dstride, kt, tm, terms, c.log_n,
                                          (u32)E, c.ndigits, c.d_mods, c0, c0_term, c0_ct, out,
                                          out_ct);
    return launched("k_ks_giants");
}

namespace {

// HC ciphertexts per CTA, CPT per thread: 16 and 8, or 2/4/8 and 1/2/4 for
// queries of at most that many ciphertexts (a CTA holds one query's, which
// share a key set)
template <int ND, u32 HC = 16, u32 CPT = 8>
int launch_baby(const Ctx& c, const u64* D, CtSet u, u32 H, u32 B, const KeyTable& kt,
                const BabyParams& bp, u64* Rx, cudaStream_t st, bool ext, u32 l0, u32 el) {
    constexpr u32 T = 64;
    const u32 E = c.L + c.K;
    const size_t smem = ((size_t)HC * ND * T + 2 * HC * T) * sizeof(u64);
    // set once per process (thread-safe static initialisation; the server's
    // workers launch concurrently)
    static const cudaError_t configured = cudaFuncSetAttribute(
        k_baby_ext<T, HC, CPT, ND>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 << 10);
    if (configured != cudaSuccess)
        return fail(PDQ_E_CUDA, std::string("k_baby_ext attribute: ") + cudaGetErrorString(configured));
    // the chunk of primes l0 .. l0+el-1: every per-prime pointer advanced to l0
    const u32 nc0 = ext ? E : c.L;                   // limbs of c0 (from limb 0)
    const u64 off = (u64)l0 * c.N;
    CtSet uc = u;
    uc.base = u.base + off;
    BabyParams bpc = bp;
    for (u32 a = 1; a < B; ++a) bpc.koff[a] += off;
    // chunks of HC ciphertexts never span two queries (one key set each)
    const u32 Hq = kt.per == ~0u ? H : kt.per;
    if (Hq == 0 || H % Hq != 0) return fail(PDQ_E_PARAM, "hoisted rotations: ragged query stack");
    const u32 zper = (Hq + HC - 1) / HC;
    const u64 zs = (u64)(H / Hq) * zper;
    if (zs > 65535) return fail(PDQ_E_PARAM, "hoisted rotations: too many ciphertexts");
    const u64 zmagic = ((1ull << 32) + zper - 1) / zper;
    const dim3 grid(c.N / T, el, (u32)zs);
    k_baby_ext<T, HC, CPT, ND><<<grid, T * HC / CPT, smem, st>>>(
        D + off, uc, kt, Hq, zper, zmagic, B, c.log_n, E, nc0 > l0 ? nc0 - l0 : 0, nc0, c.d_mods + l0,
        ext ? nullptr : c.d_P_mont + l0, Rx, bpc, el);
    return launched("k_baby_ext");
}

}  // namespace

int baby_steps_ext(const Ctx& c, const u64* D, CtSet u, u32 H, u32 B, const u64* keys,
                   const std::vector<u64>& key_offsets, u64* Rx, cudaStream_t st, u32 l0,
                   u32 el, const KeyTable* kt) {
    std::vector<u64> galois(B, 1);
    for (u32 a = 1; a < B; ++a) galois[a] = host_powmod(3, a, 2ull * c.N);
    return hoisted_rotations_ext(c, D, u, H, B, galois, keys, key_offsets, Rx, st, false, l0, el,
                                 kt);
}

bool rotations_chunkable(const Ctx& c) { return c.N >= 64 && c.ndigits <= 8; }

int hoisted_rotations_ext(const Ctx& c, const u64* D, CtSet u, u32 H, u32 B,
                          const std::vector<u64>& galois, const u64* keys,
                          const std::vector<u64>& key_offsets, u64* Rx, cudaStream_t st,
                          bool ext, u32 l0, u32 el, const KeyTable* kt) {
    constexpr u32 T = 64;
    const u32 E = c.L + c.K;
    if (el == 0) el = E - l0;
    if (l0 + el > E || (el != E && !rotations_chunkable(c)))
        return fail(PDQ_E_PARAM, "hoisted rotations: bad prime range");
    if (B > 128) return fail(PDQ_E_PARAM, "hoisted rotations: at most 128");
    if (galois.size() < B || key_offsets.size() < B)
        return fail(PDQ_E_PARAM, "hoisted rotations: one Galois element and key per rotation");
    for (u32 a = 1; a < B; ++a)
        if (galois[a] % 2 == 0 || galois[a] >= 2ull * c.N)
            return fail(PDQ_E_PARAM, "hoisted rotations: bad Galois element");
    if (c.N < T || c.ndigits > 8) {
        // rings below one tile, or more digits than the fused kernel keeps
        // in registers: one rotation at a time
        PDQ_TRY(times_P(c, u, H, ct_set(Rx, (long long)B * 2 * (c.L + c.K) * c.N), true, st, ext));
        for (u32 a = 1; a < B; ++a) {
            PDQ_TRY(ks_apply_ext(c, D, u, H, (u32)galois[a], keys + key_offsets[a],
                                 ct_set(Rx + (u64)a * 2 * (c.L + c.K) * c.N,
                                        (long long)B * 2 * (c.L + c.K) * c.N),
                                 false, true, st, ext, kt));
        }
        return PDQ_OK;
    }
    BabyParams bp{};
    for (u32 a = 1; a < B; ++a) {
        bp.k[a] = (u32)galois[a];
        bp.kinv[a] = (u32)host_invmod(galois[a], 2ull * c.N);
        bp.koff[a] = key_offsets[a];
    }
    const KeyTable t = kt ? *kt : single_keys(keys);
    const u32 Hq = t.per == ~0u ? H : t.per;
    // CTAs of 4 or 8 ciphertexts for queries of that many (up to 4 digits)
    if (Hq > 2 && Hq <= 8 && c.ndigits <= 4) {
        if (Hq <= 4) {
            switch (c.ndigits) {
                case 1: return launch_baby<1, 4, 2>(c, D, u, H, B, t, bp, Rx, st, ext, l0, el);
                case 2: return launch_baby<2, 4, 2>(c, D, u, H, B, t, bp, Rx, st, ext, l0, el);
                case 3: return launch_baby<3, 4, 2>(c, D, u, H, B, t, bp, Rx, st, ext, l0, el);
                default: return launch_baby<4, 4, 2>(c, D, u, H, B, t, bp, Rx, st, ext, l0, el);
            }
        }
        switch (c.ndigits) {
            case 1: return launch_baby<1, 8, 4>(c, D, u, H, B, t, bp, Rx, st, ext, l0, el);
            case 2: return launch_baby<2, 8, 4>(c, D, u, H, B, t, bp, Rx, st, ext, l0, el);
            case 3: return launch_baby<3, 8, 4>(c, D, u, H, B, t, bp, Rx, st, ext, l0, el);
            default: return launch_baby<4, 8, 4>(c, D, u, H, B, t, bp, Rx, st, ext, l0, el);
        }
    }
    if (Hq <= 2) {
        switch (c.ndigits) {
            case 1: return launch_baby<1, 2, 1>(c, D, u, H, B, t, bp, Rx, st, ext, l0, el);
            case 2: return launch_baby<2, 2, 1>(c, D, u, H, B, t, bp, Rx, st, ext, l0, el);
            case 3: return launch_baby<3, 2, 1>(c, D, u, H, B, t, bp, Rx, st, ext, l0, el);
            case 4: return launch_baby<4, 2, 1>(c, D, u, H, B, t, bp, Rx, st, ext, l0, el);
            case 5: return launch_baby<5, 2, 1>(c, D, u, H, B, t, bp, Rx, st, ext, l0, el);
            case 6: return launch_baby<6, 2, 1>(c, D, u, H, B, t, bp, Rx, st, ext, l0, el);
            case 7: return launch_baby<7, 2, 1>(c, D, u, H, B, t, bp, Rx, st, ext, l0, el);
            default: return launch_baby<8, 2, 1>(c, D, u, H, B, t, bp, Rx, st, ext, l0, el);
        }
    }
    switch (c.ndigits) {
        case 1: return launch_baby<1>(c, D, u, H, B, t, bp, Rx, st, ext, l0, el);
        case 2: return launch_baby<2>(c, D, u, H, B, t, bp, Rx, st, ext, l0, el);
        case 3: return launch_baby<3>(c, D, u, H, B, t, bp, Rx, st, ext, l0, el);
        case 4: return launch_baby<4>(c, D, u, H, B, t, bp, Rx, st, ext, l0, el);
        case 5: return launch_baby<5>(c, D, u, H, B, t, bp, Rx, st, ext, l0, el);
        case 6: return launch_baby<6>(c, D, u, H, B, t, bp, Rx, st, ext, l0, el);
        case 7: return launch_baby<7>(c, D, u, H, B, t, bp, Rx, st, ext, l0, el);
        default: return launch_baby<8>(c, D, u, H, B, t, bp, Rx, st, ext, l0, el);
    }
}

int sum_rotations(const Ctx& c, const u64* Rx, u32 cnt, u32 R, u64* out, cudaStream_t st) {
    const u64 E = c.L + c.K;
    if (R == 0 || R > 8) return fail(PDQ_E_PARAM, "sum of rotations: 1 to 8 terms");
    PDQ_TRY(check_y(cnt, "sum of rotations"));
    k_sum_split<<<grid2(E * c.N, cnt), kBlock, 0, st>>>(Rx, R, c.log_n, (u32)E, c.d_mods, out);
    return launched("k_sum_split");
}

int times_P(const Ctx& c, CtSet in, u32 cnt, CtSet out, bool split, cudaStream_t st, bool ext) {
    const u64 E = c.L + c.K;
    PDQ_TRY(check_y(cnt, "times_P"));
    k_times_P<<<grid2(2 * E * c.N, cnt), kBlock, 0, st>>>(in, c.log_n, c.L, (u32)E, c.d_mods,
                                                         c.d_P_mod_q, c.d_P_mod_q_shoup, out,
                                                         split ? 1u : 0u, ext ? 1u : 0u);
    return launched("k_times_P");
}

size_t mod_down_ws(const Ctx& c, u32 cnt) { return (size_t)cnt * 2 * c.L * c.N * sizeof(u64); }

size_t mod_switch_ws(const Ctx& c, u32 cnt) { return (size_t)2 * cnt * c.L * c.N * sizeof(u64); }

int mod_switch(const Ctx& c, u32 L2, const u64* cts, u32 cnt, u64* out, u64* ws, cudaStream_t st) {
    const u64 N = c.N, L = c.L;
    if (L2 == 0 || L2 >= c.L) return fail(PDQ_E_PARAM, "mod_switch: target level out of range");
    const u32 K2 = c.L - L2;
    if (K2 > 8) return fail(PDQ_E_PARAM, "mod_switch: at most 8 dropped primes");
    PDQ_TRY(check_y(2ull * cnt, "mod_switch"));
    const u64* T = c.d_ms + c.ms_off[L2];
    const u64* hinv = T;
    const u64* hinv_s = hinv + K2;
    const u64* hmod = hinv_s + K2;
    const u64* hmod_s = hmod + (u64)K2 * L2;
    const u64* dinv = hmod_s + (u64)K2 * L2;
    const u64* dinv_s = dinv + L2;
    u64* S = ws;                                   // dropped limbs, coefficient form [2cnt][K2][N]
    u64* Cv = ws + 2ull * cnt * K2 * N;            // [2cnt][L2][N]
    PDQ_TRY(ntt_inverse_from(c, cts, (long long)(L * N), 1, 0, (u64)L2 * N, S, 2 * cnt, K2,
                             (u64)K2 * N, st, L2));
    const dim3 grid((c.N / 2 + kBlock - 1) / kBlock, 2 * cnt);
#define PDQ_MSCONV(KK)                                                                            \
    k_moddown_conv<KK><<<grid, kBlock, 0, st>>>(S, (u64)K2 * N, c.log_n, L2, K2, c.d_mods, hinv,   \
                                                hinv_s, hmod, hmod_s, Cv)
    switch (K2) {
        case 1: PDQ_MSCONV(1); break;
        case 2: PDQ_MSCONV(2); break;
        case 3: PDQ_MSCONV(3); break;
        default: PDQ_MSCONV(0); break;
    }
#undef PDQ_MSCONV
    PDQ_TRY(launched("k_moddown_conv"));
    PDQ_TRY(ntt_forward(c, Cv, 2 * cnt, L2, 0, (u64)L2 * N, st));
    k_moddown_final_poly<<<grid2((u64)L2 * N / 2, 2 * cnt), kBlock, 0, st>>>(
        cts, L * N, Cv, out, (u64)L2 * N, c.log_n, L2, c.d_mods, dinv, dinv_s);
    return launched("k_moddown_final_poly");
}

size_t mod_down_polys_ws(const Ctx& c, u32 npolys) {
    return (size_t)npolys * (c.L + c.K) * c.N * sizeof(u64);
}

int mod_down_polys(const Ctx& c, const u64* A, u64 a_stride, u32 npolys, u64* out,
                   u64 out_stride, u64* ws, cudaStream_t st) {
    const u64 N = c.N, L = c.L, K = c.K;
    PDQ_TRY(check_y(npolys, "mod_down"));
    u64* S = ws;                      // special limbs, coefficient form [npolys][K][N]
    u64* Cv = ws + (u64)npolys * K * N;
    const bool fuse = moddown_fused(c);
    PDQ_TRY(ntt_inverse_from(c, A, (long long)a_stride, 1, 0, L * N, S, npolys, c.K, K * N, st,
                             c.L, fuse ? c.d_ninv_dn : nullptr));
    // fused: the conversion in the forward transform's first phase and the
    // final (A - Cv) P^-1 in its last
    if (fuse) return ntt_forward_moddown(c, Cv, S, K * N, npolys, st, A, a_stride, out, out_stride);
    PDQ_TRY(moddown_to_ntt(c, S, K * N, npolys, Cv, false, st));
    k_moddown_final_poly<<<grid2(L * N / 2, npolys), kBlock, 0, st>>>(
        A, a_stride, Cv, out, out_stride, c.log_n, c.L, c.d_mods, c.d_dn_pinv, c.d_dn_pinv_shoup);
    return launched("k_moddown_final_poly");
}

int mod_down_batch(const Ctx& c, u64* A, u32 cnt, CtSet out, u64* ws, cudaStream_t st) {
    const u64 N = c.N, L = c.L, E = c.L + c.K;
    PDQ_TRY(check_y(2ull * cnt, "mod_down"));
    u64* Cv = ws;
    PDQ_TRY(moddown_to_ntt(c, A + L * N, E * N, 2 * cnt, Cv, true, st));
    k_moddown_final<<<grid2(L * N, cnt), kBlock, 0, st>>>(A, Cv, CtSet{}, out, CtSet{}, c.log_n,
                                                              c.L, c.K, 0, c.d_mods, c.d_dn_pinv,
                                                              c.d_dn_pinv_shoup);
    return launched("k_moddown_final");
}

namespace {

struct MacShape {
    u32 GT, logGS, logX, Bc, zslices, combos_per_cta, threads, tiles_per_cta;
    size_t smem;
};

u32 log2u(u32 x) {
    u32 r = 0;
    while ((1u << (r + 1)) <= x) ++r;
    return r;
}

// Launch shape of k_diag_mac: up to 4 giant indices and kMacPC polynomials
// of a group per thread (two: each staged value feeds 8 products; one
// polynomial per thread, with three CTAs per SM, measured 9% slower), up to
// 32 combinations per CTA (more go to further z-slices), X >= 2 positions so
// that a CTA has up to 256 threads (two CTAs per SM; one CTA of 512 threads
// with 16-position tiles measured 2.5% slower), and an a-chunk BC (up to 16)
// that keeps the two staged (diagonal + rotated) tiles within kMacSmem of
// shared memory.  Position tiles are dealt to CTAs round robin, so the two
// 64-byte halves of a 128-byte line of rotated operands are read by
// neighbouring CTAs of the same wave (dealt in consecutive runs per CTA,
// the second half was evicted before use and fetched again: 1.76x the
// algorithmic DRAM reads).
constexpr u32 kMacThreads = 256;
constexpr u32 kMacPC = 2;                // polynomials (of one group) per thread
constexpr u32 kMacSmem = 100u << 10;     // two CTAs per SM
constexpr u32 kMacMinX = 2;

MacShape mac_shape(const pdq_plan& pl, u32 logN, u32 Q = 1, const pdq_schedule* sc = nullptr) {
    MacShape s{};
    const u32 GI = pl.giants, combos = 2 * pl.G * Q;
    s.GT = GI < 4 ? GI : 4;
    const u32 GS = GI / s.GT;
    s.logGS = log2u(GS);
    const u32 minX = std::min(kMacMinX, 1u << logN);
    u32 ct = (combos + kMacPC - 1) / kMacPC;       // threads along the combinations
    u32 ct_max = kMacThreads / minX / GS;
    if (ct_max < 1) ct_max = 1;
    if (ct_max > 32 / kMacPC) ct_max = 32 / kMacPC;
    if (ct > ct_max) ct = 1u << log2u(ct_max);
    s.combos_per_cta = ct * kMacPC;
    s.zslices = (combos + s.combos_per_cta - 1) / s.combos_per_cta;
    u32 logX = 1;
    while (((ct * GS) << (logX + 1)) <= kMacThreads && logX < 8) ++logX;
    if (logX > logN) logX = logN;
    u32 Bc = pl.B < 16 ? pl.B : 16;
    if (sc && sc->mac_bc && sc->mac_bc < Bc) Bc = sc->mac_bc;
    auto bytes = [&](u32 bc, u32 lx) {
        return 2 * ((size_t)bc * (1u << lx) * (GI + 2 + s.combos_per_cta) + 2 * s.combos_per_cta) * 8;
    };
    while (bytes(Bc, logX) > kMacSmem) {
        if (Bc > 1) Bc /= 2; else if (logX > 1) --logX; else break;
    }
    s.logX = logX;
    s.Bc = Bc;
    s.threads = (ct * GS) << logX;
    s.smem = bytes(Bc, logX);
    // several position tiles per CTA so that the copy pipeline runs long
    const u32 tiles = 1u << (logN - logX);
    s.tiles_per_cta = 1;
    if (sc && sc->mac_tiles) {
        while (s.tiles_per_cta < sc->mac_tiles && tiles / (s.tiles_per_cta * 2) >= 1)
            s.tiles_per_cta *= 2;
    } else {
        while (s.tiles_per_cta < 8 && tiles / (s.tiles_per_cta * 2) >= 64) s.tiles_per_cta *= 2;
    }
    return s;
}

template <int GT, int BC, bool STACKED>
int launch_mac(const Ctx& c, const pdq_plan& pl, const MacShape& s, const u64* R, const u64* Dg,
               u64* acc0, u64* acc, cudaStream_t st, u32 l0, u32 el, u32 Q) {
    static const cudaError_t configured = cudaFuncSetAttribute(
        k_diag_mac<GT, BC, kMacPC, STACKED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
        (int)kMacSmem);
    if (configured != cudaSuccess)
        return fail(PDQ_E_CUDA, std::string("k_diag_mac attribute: ") + cudaGetErrorString(configured));
    MacArgs a;
    a.G = pl.G * Q;
    a.Gq = pl.G;
    a.Gq_magic = ((1ull << 32) + pl.G - 1) / pl.G;
    a.hpg = pl.hpg;
    a.H = pl.H;
    a.B = pl.B;
    a.GI = pl.giants;
    a.E = c.L + c.K;
    a.ER = el;
    a.logN = c.log_n;
    a.logX = s.logX;
    a.logGS = s.logGS;
    a.logGI = log2u(pl.giants);
    a.CPC = s.combos_per_cta;
    a.tiles_per_cta = s.tiles_per_cta;
    a.achunks = pl.B / BC;
    a.fold_one = (u64)std::min(pl.hpg, pl.H) * pl.B <= 256 ? 1u : 0u;
    const dim3 grid((c.N >> s.logX) / s.tiles_per_cta, el, s.zslices);
    // the chunk of primes l0 .. l0+el-1: per-prime pointers advanced to l0
    const u64 off = (u64)l0 * c.N;
    k_diag_mac<GT, BC, kMacPC, STACKED><<<grid, s.threads, s.smem, st>>>(R, Dg + off * pl.giants, a,
                                                                 c.d_mods + l0, c.d_ckar + 8 * l0,
                                                                 acc0 + off, acc + off);
    return launched("k_diag_mac");
}

template <int GT>
int launch_mac_bc(const Ctx& c, const pdq_plan& pl, const MacShape& s, const u64* R,
                  const u64* Dg, u64* acc0, u64* acc, cudaStream_t st, u32 l0, u32 el, u32 Q) {
    switch (s.Bc) {
        case 1: return Q > 1 ? launch_mac<GT, 1, true>(c, pl, s, R, Dg, acc0, acc, st, l0, el, Q)
                          : launch_mac<GT, 1, false>(c, pl, s, R, Dg, acc0, acc, st, l0, el, Q);
        case 2: return Q > 1 ? launch_mac<GT, 2, true>(c, pl, s, R, Dg, acc0, acc, st, l0, el, Q)
                          : launch_mac<GT, 2, false>(c, pl, s, R, Dg, acc0, acc, st, l0, el, Q);
        case 4: return Q > 1 ? launch_mac<GT, 4, true>(c, pl, s, R, Dg, acc0, acc, st, l0, el, Q)
                          : launch_mac<GT, 4, false>(c, pl, s, R, Dg, acc0, acc, st, l0, el, Q);
        case 8: return Q > 1 ? launch_mac<GT, 8, true>(c, pl, s, R, Dg, acc0, acc, st, l0, el, Q)
                          : launch_mac<GT, 8, false>(c, pl, s, R, Dg, acc0, acc, st, l0, el, Q);
        case 16: return Q > 1 ? launch_mac<GT, 16, true>(c, pl, s, R, Dg, acc0, acc, st, l0, el, Q)
                          : launch_mac<GT, 16, false>(c, pl, s, R, Dg, acc0, acc, st, l0, el, Q);
        default: return fail(PDQ_E_PARAM, "diag_mac: baby-step count must be a power of two");
    }
}

}  // namespace

int diag_mac(const Ctx& c, const pdq_plan& pl, const u64* R, const u64* Dg, u64* acc0, u64* acc,
             cudaStream_t st, u32 l0, u32 el, u32 Q) {
    // (the kernel divides group indices by pl.G with a multiplier: exact
    // while every group index times pl.G stays below 2^32)
    if (Q == 0 || pl.G == 0 || (u64)pl.G * Q * pl.G >= (1ull << 32))
        return fail(PDQ_E_PARAM, "diag_mac: too many groups for one launch");
    const MacShape s = mac_shape(pl, c.log_n, Q, &c.sched);
    if (el == 0) el = c.L + c.K - l0;
    if (l0 + el > c.L + c.K) return fail(PDQ_E_PARAM, "diag_mac: bad prime range");
    if (s.zslices > 65535) return fail(PDQ_E_PARAM, "diag_mac: too many groups");
    if (s.logX < 1 || s.smem > kMacSmem) return fail(PDQ_E_PARAM, "diag_mac: plan too large for one tile");
    switch (s.GT) {
        case 1: return launch_mac_bc<1>(c, pl, s, R, Dg, acc0, acc, st, l0, el, Q);
        case 2: return launch_mac_bc<2>(c, pl, s, R, Dg, acc0, acc, st, l0, el, Q);
        case 4: return launch_mac_bc<4>(c, pl, s, R, Dg, acc0, acc, st, l0, el, Q);
        default: return fail(PDQ_E_PARAM, "diag_mac: giant-step count must be a power of two");
    }
}

namespace {

// Multiply-accumulate of the Answer on an unencrypted database:
//   acc[gamma][sigma][g][p] = sum_{j in gamma} sum_{a<B} D[j][sigma][a][l][x][g] * R[j][a][p][l][x]
// over Q u P.  The diagonals are different for every index ciphertext (the
// database is in them), so each is used by one thread (for both
// polynomials) and streamed from DRAM once; the kernel is bound by that
// stream.  Thread = position x, set sigma and GT giant steps of one group
// and prime; its GT diagonal values are contiguous (giant index innermost,
// a warp reads one contiguous run) and the rotated operands R (split layout)
// are shared through L2 with the threads of the other sets and giant slices.
// Every thread streams its own operands through a private ring of kDbStages
// shared-memory slots with asynchronous copies, kDbStages - 1 steps ahead
// of its arithmetic (no block barrier: a thread reads only what it copied).
// Output (sigma, g) = (0, 0) goes to y0[gamma][p], the others to
// acc[gamma][sigma GI + g - 1][p].
constexpr u32 kDbStages = 4;
constexpr u32 kDbThreads = 256;

template <int GT>
__global__ void __launch_bounds__(kDbThreads, 2) k_diag_mac_db(
        const u64* __restrict__ R, const u64* __restrict__ Dd, u32 J, u32 jpg, u32 B, u32 GI,
        u32 GS, u32 E, u32 logN, const Mod* __restrict__ mods, const u64* __restrict__ ckar,
        u32 fold_one, u64* __restrict__ y0, u64* __restrict__ acc) {
    constexpr u32 W = GT + 2;                        // words per thread and stage
    extern __shared__ __align__(16) u64 sring[];     // [kDbStages][threads][W]
    const u64 N = 1ull << logN, EN = (u64)E << logN;
    const u32 tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
    const u64 x = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    const u32 sigma = threadIdx.y / GS, g0 = (threadIdx.y % GS) * GT;
    const u32 l = blockIdx.y, gamma = blockIdx.z;
    const bool live = x < N;
    const u64 loff = ((u64)l << logN) + (live ? x : 0);
    const u64 j0 = (u64)gamma * jpg;
    const u32 jn = (u32)(j0 >= J ? 0 : (J - j0 < jpg ? J - j0 : jpg));
    const u32 steps = jn * B;
    auto slot = [&](u32 st) { return sring + ((u64)(st % kDbStages) * nth + tid) * W; };
    auto issue = [&](u32 st) {
        if (st < steps) {
            const u64 j = j0 + st / B, a = st % B;
            u64* sl = slot(st);
            const u64* dp = Dd + ((((j * 2 + sigma) * B + a) * E) << logN) * GI + loff * GI + g0;
            if (GT >= 2) {
#pragma unroll
                for (int g = 0; g < GT; g += 2) cp_async16(sl + g, dp + g, live);
            } else {
                cp_async8(sl, dp);
            }
            const u64* rp = R + ((j * B + a) * 2) * EN + loff;
            cp_async8(sl + GT, rp);
            cp_async8(sl + GT + 1, rp + EN);
        }
        cp_async_commit();
    };
    AccK A[2][GT];
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int g = 0; g < GT; ++g) A[p][g] = AccK{0, 0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
    for (u32 st = 0; st + 1 < kDbStages; ++st) issue(st);
    for (u32 st = 0; st < steps; ++st) {
        cp_async_wait<kDbStages - 2>();
        const u64* sl = slot(st);
        u64 d[GT];
#pragma unroll
        for (int g = 0; g < GT; ++g) d[g] = sl[g];
        const u64 r0 = sl[GT], r1 = sl[GT + 1];
        issue(st + kDbStages - 1);                   // refills the slot read last step
        const u32 rl0 = (u32)r0, rh0 = (u32)(r0 >> 32), rs0 = rl0 + rh0;
        const u32 rl1 = (u32)r1, rh1 = (u32)(r1 >> 32), rs1 = rl1 + rh1;
#pragma unroll
        for (int g = 0; g < GT; ++g) {
            const u32 d0 = (u32)d[g], d1 = (u32)(d[g] >> 32), ds = d0 + d1;
            mack(A[0][g], rl0, rh0, rs0, d0, d1, ds);
            mack(A[1][g], rl1, rh1, rs1, d0, d1, ds);
        }
    }
    cp_async_wait<0>();
    if (!live) return;
    const Mod md = mods[l];
#pragma unroll
    for (int g = 0; g < GT; ++g) {
        const u32 gi = g0 + g;
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const u64 v = fold_one ? fold1(A[p][g], md) : foldk(A[p][g], md, ckar + 8 * l);
            u64* o = (sigma == 0 && gi == 0)
                         ? y0 + ((u64)gamma * 2 + p) * EN + loff
                         : acc + (((u64)gamma * (2 * GI - 1) + sigma * GI + gi - 1) * 2 + p) * EN + loff;
            *o = v;
        }
    }
}

}  // namespace

int build_db_diagonals(const Ctx& c, const pdq_plan& pl, const u32* values, u64* out,
                       cudaStream_t st) {
    const u32 GI = pl.giants, B = pl.B, E = c.L + c.K;
    PDQ_TRY(check_y(GI, "diagonals"));
    const u64 LN = (u64)E * c.N;
    u64* tmp = nullptr;
    if (cudaMallocAsync((void**)&tmp, (size_t)GI * LN * sizeof(u64), st) != cudaSuccess) {
        cudaGetLastError();
        return fail(PDQ_E_NOMEM, "diagonals: temporary allocation failed");
    }
    int rc = PDQ_OK;
    // plaintext (j, sigma, g, a) is encoded in tmp[g], then stored at
    // out[j][sigma][a][l][x][g] in the operand layout of the multiply-accumulate
    for (u64 js = 0; js < 2ull * pl.J && rc == PDQ_OK; ++js) {
        for (u32 a = 0; a < B && rc == PDQ_OK; ++a) {
            // row g of tmp: plaintext (js, g, a), pt = (js GI + g) B + a
            k_diag_slots_db<<<grid2(c.N, GI), kBlock, 0, st>>>(
                tmp, GI, B, pl.s_prime, c.log_n, E, c.d_slot_pos, c.t, pl.G_sz, values, pl.n,
                js * GI * B + a);
            rc = launched("k_diag_slots_db");
            if (rc == PDQ_OK) rc = encode_finish(c, tmp, GI, E, st);
            if (rc == PDQ_OK) {
                k_diag_layout<<<(u32)((LN + kBlock - 1) / kBlock), kBlock, 0, st>>>(
                    tmp, out + (js * B + a) * GI * LN, GI, LN);
                rc = launched("k_diag_layout");
            }
        }
    }
    cudaFreeAsync(tmp, st);
    return rc;
}

int diag_mac_db(const Ctx& c, const pdq_plan& pl, const u64* R, const u64* Dd, u64* y0, u64* acc,
                cudaStream_t st) {
    const u32 GI = pl.giants, E = c.L + c.K;
    const u32 GT = GI < 4 ? GI : 4, GS = GI / GT;
    if (2 * GS > kDbThreads / 32) return fail(PDQ_E_PARAM, "diag_mac_db: too many giant steps");
    const u32 X = kDbThreads / (2 * GS);
    const u32 jpg = pl.hpg / 2;
    const u32 fold_one = (u64)std::min(jpg, pl.J) * pl.B <= 256 ? 1u : 0u;
    if (pl.G > 65535) return fail(PDQ_E_PARAM, "diag_mac_db: too many groups");
    const dim3 block(X, 2 * GS), grid((c.N + X - 1) / X, E, pl.G);
    const size_t smem = (size_t)kDbStages * kDbThreads * (GT + 2) * sizeof(u64);
    switch (GT) {
        case 1:
            k_diag_mac_db<1><<<grid, block, smem, st>>>(R, Dd, pl.J, jpg, pl.B, GI, GS, E, c.log_n,
                                                        c.d_mods, c.d_ckar, fold_one, y0, acc);
            break;
        case 2:
            k_diag_mac_db<2><<<grid, block, smem, st>>>(R, Dd, pl.J, jpg, pl.B, GI, GS, E, c.log_n,
                                                        c.d_mods, c.d_ckar, fold_one, y0, acc);
            break;
        case 4:
            k_diag_mac_db<4><<<grid, block, smem, st>>>(R, Dd, pl.J, jpg, pl.B, GI, GS, E, c.log_n,
                                                        c.d_mods, c.d_ckar, fold_one, y0, acc);
            break;
        default: return fail(PDQ_E_PARAM, "diag_mac_db: giant-step count must be a power of two");
    }
    return launched("k_diag_mac_db");
}

int ct_add(const Ctx& c, CtSet y, CtSet x, u32 cnt, cudaStream_t st) {
    PDQ_TRY(check_y(cnt, "ct_add"));
    k_ct_add<<<grid2(2ull * c.L * c.N, cnt), kBlock, 0, st>>>(y, x, c.L, c.log_n, c.d_mods);
    return launched("k_ct_add");
}

int group_combine(const Ctx& c, const pdq_plan& pl, const u64* y, const u64* masks, u64* out,
                  cudaStream_t st, u32 Q) {
    PDQ_TRY(check_y((u64)pl.n_out * Q, "group_combine"));
    k_group_combine<<<grid2(2ull * c.L * c.N, pl.n_out * Q), kBlock, 0, st>>>(
        y, masks, pl.G, pl.per_out, pl.n_out, c.L, c.log_n, c.d_mods, out);
    return launched("k_group_combine");
}

}  // namespace pdq
