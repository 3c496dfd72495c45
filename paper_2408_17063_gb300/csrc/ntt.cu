// Negacyclic number-theoretic transform over 60-bit primes for sm_103a.
//
// The forward transform maps a(X) in Z_q[X]/(X^N+1) to its values at the
// odd powers of a primitive 2N-th root psi, stored in bit-reversed order
// (position k holds a(psi^{2 brv(k) + 1})); the inverse undoes it.  Both use
// the merged-twiddle radix-2 formulation: Cooley-Tukey butterflies forward,
// Gentleman-Sande butterflies inverse, Shoup multiplication by
// precomputed twiddles and Harvey's lazy ranges ([0,4q) forward, [0,2q)
// inverse), with N^{-1} folded into the last inverse level.  Outputs are
// canonical residues.
//
// Work decomposition: for log N <= 11 one CTA transforms one polynomial in
// shared memory.  Larger rings split the log N levels into a column phase
// (levels 0..S1-1: independent length-2^S1 transforms over elements spaced
// 2^9 apart) and a row phase (levels S1..logN-1: independent contiguous
// length-2^9 transforms), each CTA holding a 2048-element tile (16 KB) of
// consecutive columns or rows so that every global access is coalesced.
// Inside a tile, each thread runs up to three levels on eight elements in
// registers between shared-memory exchanges.
#include "pdq_internal.h"

namespace pdq {

namespace {

constexpr u32 kTileBits = 11;
constexpr u32 kTile = 1u << kTileBits;   // elements per CTA tile
constexpr u32 kRowBits = 9;       // row length 2^9 in the two-phase split
constexpr u32 kThreads = 256;     // 8 elements per thread and pass
constexpr int kMaxRadixBits = 3;  // levels per register pass (four, with 128
                                  // registers and half the resident warps,
                                  // measured 4-6% slower)

struct NttArgs {
    u64* data;
    u64 stride;        // elements between consecutive groups
    u32 nlimbs;        // limbs per group
    u32 limb0;         // modulus index of the first limb
    const Mod* mods;
    const ulonglong2* tw;  // [nmod][N] (twiddle, Shoup companion), forward or inverse
    const u64* ninv4;  // [nmod][4]
    u32 logN;
    u32 S1;            // levels done by the column phase (0: single phase)
    u32 logC;          // log2(sub-transforms per CTA)
    u32 last;          // 1: this phase writes canonical output
    // first phase only: read group g from src + (g / per) outer + (g % per)
    // inner + off (limb l at + l N) instead of data (src == nullptr: in place)
    const u64* src;
    long long src_outer, src_inner;
    u32 src_per;
    u64 src_off;
    // raised digits (skip_alpha > 0): group g is digit g % skip_nd of a
    // ciphertext, and its limbs skip the digit's own skip_alpha limbs
    u32 skip_nd, skip_alpha;
    // a basis conversion in the first (column) phase of a forward transform
    // (the raise's and ModDown's): transform group g takes source group
    // s = g / up_div and first source limb i0 = (g % up_div) up_i0_step;
    // element = sum_{k < up_n} y_k hm_k (Shoup), y_k at up_src + s
    // up_src_stride + (i0 + k) N, hm_k = up_hm[(i0 + k) up_E + prime]
    const u64* up_src;
    const ulonglong2* up_hm;
    u64 up_src_stride;
    u32 up_div, up_i0_step, up_n, up_E;
    // ModDown's last step in the last (row) phase of a forward transform of
    // converted limbs: instead of the transform, group g limb l writes
    // (A - NTT(conv)) P^-1 mod q to epi_out + g epi_out_stride + l N, A read at
    // epi_a + g epi_a_stride + l N
    const u64* epi_a;
    u64* epi_out;
    u64 epi_a_stride, epi_out_stride;
    const u64* epi_pinv;
    const u64* epi_pinvs;
    // the raise's own limbs from the first (row) phase of the inverse
    // transform of c1: as it reads limb r (NTT form) of ciphertext g it also
    // writes c1_r R mod q_r to own_out + ((g own_nd + r / own_alpha) own_E + r) N
    u64* own_out;
    u32 own_nd, own_alpha, own_E;
};

__device__ __forceinline__ void bf_fwd(u64& x, u64& y, u64 w, u64 wp, u64 q) {
    const u64 a = csub(x, 2 * q);
    const u64 t = mul_shoup_lazy(y, w, wp, q);
    x = a + t;
    y = a - t + 2 * q;
}

__device__ __forceinline__ void bf_inv(u64& x, u64& y, u64 w, u64 wp, u64 q) {
    const u64 a = x, b = y;
    x = csub(a + b, 2 * q);
    y = mul_shoup_lazy(a - b + 2 * q, w, wp, q);
}

// Shared-memory word of element l of sub-transform c.  Column tiles hold
// rows of C >= 16 consecutive columns (conflict-free as is).  Row tiles XOR
// bits 3..6 of the word index into bits 0..3: a bijection inside every
// aligned run of 16 words that makes the contiguous accesses and the
// stride-8 and stride-64 accesses of the register passes all hit distinct
// banks.
template <int S, bool COLS>
__device__ __forceinline__ u32 smem_index(u32 c, u32 l, u32 logC) {
    if (COLS) return (l << logC) + c;
    const u32 w = (c << S) + l;
    return w ^ ((w >> 3) & 15);
}

template <bool FWD, int S, bool COLS, bool SINGLE, bool MODUP = false, bool EPI = false,
          bool OWN = false>
struct Phase {
    static constexpr u32 GS = 1u << S;
    // sub-transforms per CTA: one whole polynomial in the single-phase case,
    // else as many as fill a tile
    static constexpr u32 LOGC = SINGLE ? 0 : kTileBits - S;
    static constexpr u32 C = 1u << LOGC;

    u64* sm;
    const ulonglong2* tw;
    u64 q;
    u64 n0, n0s, n1, n1s;  // N^-1 and psi^-1 N^-1 (with Shoup) for level 0
    u32 logN, sub0, S2;
    const u64* gin;        // tile input (global), read by a direct first pass
    u64* gout;             // tile output (global), written by a direct last pass
    bool canon;            // the last pass writes canonical residues
    // MODUP: the first pass converts from these sources (at most 2 limbs)
    const u64* ysrc0;
    const u64* ysrc1;
    u64 hm0, hm0s, hm1, hm1s;
    bool two;
    // EPI: the last pass writes (A - x) P^-1 to eout instead of x to gout
    const u64* ea;
    u64* eout;
    u64 pv, pvs;
    // OWN: the first pass also writes the loaded values times R to own
    u64* own;
    u64 rv, rvs;

    // global index of element l of sub-transform c
    __device__ __forceinline__ u32 gidx(u32 c, u32 l) const {
        return COLS ? (l << S2) + sub0 + c : ((sub0 + c) << S) + l;
    }

    // pair bits of the first and the last register pass
    static constexpr int first_lb() { return FWD ? S - (S >= kMaxRadixBits ? kMaxRadixBits : S) : 0; }
    static constexpr int last_lb() {
        if (FWD) return 0;
        int lo = 0;
        while (S - lo > kMaxRadixBits) lo += kMaxRadixBits;
        return lo;
    }
    // A first or last pass reads or writes global memory directly, instead
    // of staging the tile through shared memory, where its accesses coalesce:
    // every column pass and row passes whose pair bits start at 5 or above
    // (consecutive threads on consecutive elements), and row passes whose
    // pair bits start at 0 (each thread holds 2^R consecutive elements, moved
    // as 16-byte pairs).
    static constexpr bool direct(int lb) { return COLS || lb >= 5 || lb == 0; }
    static constexpr bool DIRECT_IN = direct(first_lb());
    static constexpr bool DIRECT_OUT = direct(last_lb());

    // One pass over the R local levels whose pair bits are LB .. LB+R-1:
    // every thread item holds the 2^R elements that these levels combine.
    // All shifts and masks of the local index are compile-time constants.
    template <int R, int LB, bool FIRST, bool LAST>
    __device__ __forceinline__ void pass() const {
        constexpr bool IN_G = FIRST && DIRECT_IN;
        constexpr bool OUT_G = LAST && DIRECT_OUT;
        constexpr u32 NE = 1u << R;
        constexpr u32 items = (C * GS) >> R;
        constexpr u32 lowmask = (1u << LB) - 1;
        const u32 gsh = LB + (COLS ? S2 : 0u);   // global position of pass bit 0
#pragma unroll 1
        for (u32 w = threadIdx.x; w < items; w += blockDim.x) {
            u32 c, fixed;
            if (COLS) {
                c = w & (C - 1);
                fixed = w >> LOGC;
            } else {
                fixed = w & ((GS >> R) - 1);
                c = w >> (S - R);
            }
            const u32 lbase = (fixed & lowmask) | ((fixed >> LB) << (LB + R));
            const u32 jbase = gidx(c, lbase);
            u64 x[NE];
            if constexpr (IN_G && !COLS && LB == 0) {
#pragma unroll
                for (u32 k = 0; k < NE; k += 2) {
                    const u32 pos = gidx(c, lbase + k);
                    const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(gin + pos);
                    x[k] = v.x;
                    x[k + 1] = v.y;
                    if constexpr (OWN)
                        *reinterpret_cast<ulonglong2*>(own + pos) =
                            make_ulonglong2(csub(mul_shoup_lazy(v.x, rv, rvs, q), q),
                                            csub(mul_shoup_lazy(v.y, rv, rvs, q), q));
                }
            } else {
#pragma unroll
                for (u32 k = 0; k < NE; ++k) {
                    if constexpr (IN_G && MODUP) {
                        // each Shoup product in [0, 2q): the sum within the
                        // forward transform's input range [0, 4q)
                        const u32 pos = gidx(c, lbase | (k << LB));
                        u64 v = mul_shoup_lazy(ysrc0[pos], hm0, hm0s, q);
                        if (two) v += mul_shoup_lazy(ysrc1[pos], hm1, hm1s, q);
                        x[k] = v;
                    } else if constexpr (IN_G) {
                        x[k] = gin[gidx(c, lbase | (k << LB))];
                    } else {
                        x[k] = sm[smem_index<S, COLS>(c, lbase | (k << LB), LOGC)];
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int kb = FWD ? R - 1 - r : r;          // pair bit inside the item
                const u32 P = gsh + kb;                      // pair bit in the global index
                const u32 st = logN - 1 - P;                 // radix-2 level
                const u32 ti0 = (1u << st) + (jbase >> (P + 1));
                const bool level0 = !FWD && st == 0;
                ulonglong2 wv[NE / 2];
                if (!level0) {
#pragma unroll
                    for (int id = 0; id < (int)(NE >> (kb + 1)); ++id) wv[id] = __ldg(tw + ti0 + id);
                }
#pragma unroll
                for (int id = 0; id < (int)(NE >> (kb + 1)); ++id) {
#pragma unroll
                    for (int low = 0; low < (1 << kb); ++low) {
                        const int k = (id << (kb + 1)) | low;
                        if (level0) {
                            const u64 xa = x[k], xb = x[k + (1 << kb)];
                            x[k] = mul_shoup_lazy(xa + xb, n0, n0s, q);
                            x[k + (1 << kb)] = mul_shoup_lazy(xa - xb + 2 * q, n1, n1s, q);
                        } else if (FWD) {
                            bf_fwd(x[k], x[k + (1 << kb)], wv[id].x, wv[id].y, q);
                        } else {
                            bf_inv(x[k], x[k + (1 << kb)], wv[id].x, wv[id].y, q);
                        }
                    }
                }
            }
            if constexpr (OUT_G) {
                if (canon) {
#pragma unroll
                    for (u32 k = 0; k < NE; ++k) x[k] = FWD ? csub(csub(x[k], 2 * q), q) : csub(x[k], q);
                }
                if constexpr (EPI && !COLS && LB == 0) {
#pragma unroll
                    for (u32 k = 0; k < NE; k += 2) {
                        const u32 pos = gidx(c, lbase + k);
                        const ulonglong2 av = *reinterpret_cast<const ulonglong2*>(ea + pos);
                        *reinterpret_cast<ulonglong2*>(eout + pos) = make_ulonglong2(
                            csub(mul_shoup_lazy(submod(av.x, x[k], q), pv, pvs, q), q),
                            csub(mul_shoup_lazy(submod(av.y, x[k + 1], q), pv, pvs, q), q));
                    }
                } else if constexpr (EPI) {
#pragma unroll
                    for (u32 k = 0; k < NE; ++k) {
                        const u32 pos = gidx(c, lbase | (k << LB));
                        eout[pos] = csub(mul_shoup_lazy(submod(ea[pos], x[k], q), pv, pvs, q), q);
                    }
                } else if constexpr (!COLS && LB == 0) {
#pragma unroll
                    for (u32 k = 0; k < NE; k += 2)
                        *reinterpret_cast<ulonglong2*>(gout + gidx(c, lbase + k)) = make_ulonglong2(x[k], x[k + 1]);
                } else {
#pragma unroll
                    for (u32 k = 0; k < NE; ++k) gout[gidx(c, lbase | (k << LB))] = x[k];
                }
            } else {
#pragma unroll
                for (u32 k = 0; k < NE; ++k) sm[smem_index<S, COLS>(c, lbase | (k << LB), LOGC)] = x[k];
            }
        }
        if constexpr (!OUT_G) __syncthreads();
    }

    // forward: pair bits from the top down, up to three at a time
    template <int TOP, bool FIRST>
    __device__ __forceinline__ void run_fwd() const {
        if constexpr (TOP > 0) {
            constexpr int R = TOP >= kMaxRadixBits ? kMaxRadixBits : TOP;
            pass<R, TOP - R, FIRST, TOP - R == 0>();
            run_fwd<TOP - R, false>();
        }
    }
    // inverse: pair bits from the bottom up
    template <int LO, bool FIRST>
    __device__ __forceinline__ void run_inv() const {
        if constexpr (LO < S) {
            constexpr int R = (S - LO) >= kMaxRadixBits ? kMaxRadixBits : (S - LO);
            pass<R, LO, FIRST, LO + R == S>();
            run_inv<LO + R, false>();
        }
    }
    __device__ __forceinline__ void run() const {
        if constexpr (FWD) run_fwd<S, true>();
        else run_inv<0, true>();
    }
};

template <bool FWD, int S, bool COLS, bool SINGLE, bool MODUP = false, bool EPI = false,
          bool OWN = false>
__global__ void __launch_bounds__(kThreads, 5) ntt_phase_kernel(NttArgs a) {
    __shared__ __align__(16) u64 sm[kTile];
    const u32 p = blockIdx.x;
    const u32 grp = p / a.nlimbs;
    u32 limb = p - grp * a.nlimbs;
    if (a.skip_alpha) {
        const u32 own = (grp % a.skip_nd) * a.skip_alpha;
        if (limb >= own) limb += a.skip_alpha;
    }
    const u32 mi = a.limb0 + limb;
    const u32 N = 1u << a.logN;
    u64* base = a.data + (u64)grp * a.stride + (u64)limb * N;
    const u64* inb = base;
    if (a.src) {
        const u32 hi = grp / a.src_per, lo = grp - hi * a.src_per;
        inb = a.src + (long long)hi * a.src_outer + (long long)lo * a.src_inner + a.src_off +
              (u64)limb * N;
    }

    Phase<FWD, S, COLS, SINGLE, MODUP, EPI, OWN> ph;
    if constexpr (OWN) {
        const u32 b = mi / a.own_alpha;
        ph.own = a.own_out + (((u64)grp * a.own_nd + b) * a.own_E + mi) * N;
        ph.rv = a.mods[mi].r64;
        ph.rvs = a.mods[mi].r64_shoup;
    }
    if constexpr (EPI) {
        ph.ea = a.epi_a + (u64)grp * a.epi_a_stride + (u64)limb * N;
        ph.eout = a.epi_out + (u64)grp * a.epi_out_stride + (u64)limb * N;
        ph.pv = a.epi_pinv[mi];
        ph.pvs = a.epi_pinvs[mi];
    }
    if constexpr (MODUP) {
        // group grp takes source group sg from its first source limb i0 (a
        // raised digit: its ciphertext and the digit's limbs); the constants
        // are those of prime mi
        const u32 sg = grp / a.up_div, i0 = (grp - sg * a.up_div) * a.up_i0_step;
        const u64 N2 = 1ull << a.logN;
        ph.ysrc0 = a.up_src + (u64)sg * a.up_src_stride + (u64)i0 * N2;
        ph.ysrc1 = ph.ysrc0 + N2;
        const ulonglong2 h0 = a.up_hm[(u64)i0 * a.up_E + mi];
        ph.hm0 = h0.x;
        ph.hm0s = h0.y;
        ph.two = a.up_n > 1;
        if (ph.two) {
            const ulonglong2 h1 = a.up_hm[(u64)(i0 + 1) * a.up_E + mi];
            ph.hm1 = h1.x;
            ph.hm1s = h1.y;
        }
    }
    ph.sm = sm;
    ph.q = a.mods[mi].q;
    ph.tw = a.tw + (u64)mi * N;
    ph.n0 = a.ninv4[4 * mi + 0];
    ph.n0s = a.ninv4[4 * mi + 1];
    ph.n1 = a.ninv4[4 * mi + 2];
    ph.n1s = a.ninv4[4 * mi + 3];
    ph.logN = a.logN;
    ph.sub0 = blockIdx.y << Phase<FWD, S, COLS, SINGLE>::LOGC;
    ph.S2 = a.logN - S;               // column phase: stride of the column elements
    ph.gin = inb;
    ph.gout = base;
    ph.canon = a.last != 0;

    using Ph = Phase<FWD, S, COLS, SINGLE, MODUP, EPI, OWN>;
    constexpr u32 GS = 1u << S;
    constexpr u32 LOGC = Ph::LOGC;
    constexpr u32 T = Ph::C * GS;
    // Staging (when the first or the last pass cannot access global memory
    // directly): adjacent element pairs are adjacent in global memory (C >= 2
    // columns, or rows of >= 2 elements) and in shared memory (the row
    // swizzle keeps aligned pairs together, possibly swapped), so tiles move
    // with 16-byte accesses on both sides.
    if constexpr (!Ph::DIRECT_IN) {
        for (u32 e = 2 * threadIdx.x; e < T; e += 2 * blockDim.x) {
            u32 c, l;
            if (COLS) { l = e >> LOGC; c = e & ((1u << LOGC) - 1); }
            else { c = e >> S; l = e & (GS - 1); }
            const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(inb + ph.gidx(c, l));
            const u32 w = smem_index<S, COLS>(c, l, LOGC);
            *reinterpret_cast<ulonglong2*>(sm + (w & ~1u)) = (w & 1) ? make_ulonglong2(v.y, v.x) : v;
        }
        __syncthreads();
    }
    ph.run();
    if constexpr (Ph::DIRECT_OUT) return;
    const u64 q = ph.q;
    for (u32 e = 2 * threadIdx.x; e < T; e += 2 * blockDim.x) {
        u32 c, l;
        if (COLS) { l = e >> LOGC; c = e & ((1u << LOGC) - 1); }
        else { c = e >> S; l = e & (GS - 1); }
        const u32 w = smem_index<S, COLS>(c, l, LOGC);
        const ulonglong2 sv = *reinterpret_cast<const ulonglong2*>(sm + (w & ~1u));
        u64 v0 = (w & 1) ? sv.y : sv.x, v1 = (w & 1) ? sv.x : sv.y;
        if (a.last) {
            v0 = FWD ? csub(csub(v0, 2 * q), q) : csub(v0, q);
            v1 = FWD ? csub(csub(v1, 2 * q), q) : csub(v1, q);
        }
        *reinterpret_cast<ulonglong2*>(base + ph.gidx(c, l)) = make_ulonglong2(v0, v1);
    }
}

template <bool FWD, bool COLS, bool SINGLE, bool MODUP = false>
int launch_phase(int S, dim3 grid, u32 threads, const NttArgs& a, cudaStream_t st) {
    switch (S) {
#define PDQ_CASE(s) case s: ntt_phase_kernel<FWD, s, COLS, SINGLE, MODUP><<<grid, threads, 0, st>>>(a); break;
        PDQ_CASE(1) PDQ_CASE(2) PDQ_CASE(3) PDQ_CASE(4) PDQ_CASE(5) PDQ_CASE(6)
        PDQ_CASE(7) PDQ_CASE(8) PDQ_CASE(9) PDQ_CASE(10) PDQ_CASE(11)
        // (column phases use S = log N - 9 <= 7 for the supported rings)
#undef PDQ_CASE
        default: return fail(PDQ_E_PARAM, "ntt: unsupported phase size");
    }
    return launched("ntt_phase_kernel");
}

// the row phase of a two-phase transform, R = 7..11 levels (EPI: ModDown's
// last step in its output; OWN: the raise's own limbs from its input)
template <bool FWD, bool EPI = false, bool OWN = false>
int launch_rows(u32 R, dim3 grid, const NttArgs& a, cudaStream_t st) {
    switch (R) {
        case 7: ntt_phase_kernel<FWD, 7, false, false, false, EPI, OWN><<<grid, kThreads, 0, st>>>(a); break;
        case 8: ntt_phase_kernel<FWD, 8, false, false, false, EPI, OWN><<<grid, kThreads, 0, st>>>(a); break;
        case 9: ntt_phase_kernel<FWD, 9, false, false, false, EPI, OWN><<<grid, kThreads, 0, st>>>(a); break;
        case 10: ntt_phase_kernel<FWD, 10, false, false, false, EPI, OWN><<<grid, kThreads, 0, st>>>(a); break;
        case 11: ntt_phase_kernel<FWD, 11, false, false, false, EPI, OWN><<<grid, kThreads, 0, st>>>(a); break;
        default: return fail(PDQ_E_PARAM, "ntt: unsupported row phase");
    }
    return launched("ntt_phase_kernel");
}

template <bool FWD>
int ntt_run(const Ctx& c, u64* data, u32 count, u32 nlimbs, u32 limb0, u64 stride,
            cudaStream_t st, const NttArgs* from = nullptr, u32 skip_nd = 0, u32 skip_alpha = 0,
            const u64* ninv_tab = nullptr, const NttArgs* conv = nullptr,
            const NttArgs* epi = nullptr, const NttArgs* own = nullptr) {
    if (count == 0 || nlimbs == 0) return PDQ_OK;
    if (limb0 + nlimbs + skip_alpha > c.nmod) return fail(PDQ_E_PARAM, "ntt: limb range out of bounds");
    const u64 polys = (u64)count * nlimbs;
    if (polys > 0x7fffffffULL) return fail(PDQ_E_PARAM, "ntt: too many polynomials");
    NttArgs a{};
    a.data = data;
    a.stride = stride;
    a.nlimbs = nlimbs;
    a.limb0 = limb0;
    a.mods = c.d_mods;
    a.tw = reinterpret_cast<const ulonglong2*>(FWD ? c.d_fw2 : c.d_iw2);
    a.ninv4 = ninv_tab ? ninv_tab : c.d_ninv;
    a.logN = c.log_n;
    a.skip_nd = skip_nd;
    a.skip_alpha = skip_alpha;
    const u64* up_src = conv ? conv->up_src : nullptr;
    if (conv) {
        // the conversion rides on the forward column phase
        if (!FWD || c.log_n <= kTileBits || conv->up_n == 0 || conv->up_n > 2 || conv->up_div == 0)
            return fail(PDQ_E_PARAM, "ntt: the fused conversion needs a two-phase forward transform of at most 2 sources");
        a.up_src = conv->up_src;
        a.up_hm = conv->up_hm;
        a.up_src_stride = conv->up_src_stride;
        a.up_div = conv->up_div;
        a.up_i0_step = conv->up_i0_step;
        a.up_n = conv->up_n;
        a.up_E = conv->up_E;
    }
    if (epi) {
        if (!FWD || c.log_n <= kTileBits) return fail(PDQ_E_PARAM, "ntt: the fused ModDown needs a two-phase forward transform");
        a.epi_a = epi->epi_a;
        a.epi_out = epi->epi_out;
        a.epi_a_stride = epi->epi_a_stride;
        a.epi_out_stride = epi->epi_out_stride;
        a.epi_pinv = epi->epi_pinv;
        a.epi_pinvs = epi->epi_pinvs;
    }
    if (own) {
        if (FWD || c.log_n <= kTileBits || limb0 != 0 || own->own_alpha == 0)
            return fail(PDQ_E_PARAM, "ntt: own limbs need a two-phase inverse transform of c1");
        a.own_out = own->own_out;
        a.own_nd = own->own_nd;
        a.own_alpha = own->own_alpha;
        a.own_E = own->own_E;
    }
    if (from) {
        a.src = from->src;
        a.src_outer = from->src_outer;
        a.src_inner = from->src_inner;
        a.src_per = from->src_per;
        a.src_off = from->src_off;
    }
    if (c.log_n <= kTileBits) {
        a.S1 = 0;
        a.logC = 0;
        a.last = 1;
        u32 threads = c.N / 8 < 32 ? 32 : (c.N / 8 > kThreads ? kThreads : c.N / 8);
        return launch_phase<FWD, false, true>((int)c.log_n, dim3((u32)polys, 1), threads, a, st);
    }
    // row phase: R levels (the schedule's, else kRowBits), column phase the rest
    const u32 R = c.sched.ntt_row_bits ? c.sched.ntt_row_bits : kRowBits;
    if (R < 7 || R > kTileBits || R >= c.log_n || c.log_n - R > kTileBits)
        return fail(PDQ_E_PARAM, "ntt: unsupported phase split");
    const u32 S1 = c.log_n - R;
    a.S1 = S1;
    NttArgs cols = a, rows = a;
    (FWD ? rows : cols).src = nullptr;        // the second phase works in place
    cols.logC = kTileBits - S1;                // 2^S1 * C = tile
    rows.logC = kTileBits - R;                 // 2^(11-R) rows of 2^R
    // (first phase: FWD columns, else rows; its `src` is the strided set)
    cols.last = FWD ? 0 : 1;
    rows.last = FWD ? 1 : 0;
    // Groups go in chunks of the schedule's polynomials per launch pair (0:
    // all at once), so that a chunk's intermediate between the two phases
    // can stay in L2.  A chunk starts on a whole ciphertext (digits,
    // conversion sources, strided input set).
    u32 unit = 1;
    if (skip_alpha) unit = skip_nd;
    if (conv) unit = std::max(unit, conv->up_div);
    if (from) unit = std::max(unit, from->src_per);
    u64 chunk = count;
    if (c.sched.ntt_chunk) {
        chunk = std::max<u64>(1, c.sched.ntt_chunk / nlimbs) / unit * unit;
        if (chunk == 0) chunk = unit;
    }
    for (u64 g0 = 0; g0 < count; g0 += chunk) {
        const u64 gn = std::min<u64>(chunk, count - g0);
        NttArgs cc = cols, rr = rows;
        cc.data = rr.data = data + g0 * stride;
        if (from) {
            // (the first phase of an inverse transform reads the set)
            const u64 hi = g0 / from->src_per;
            (FWD ? cc : rr).src = from->src + (long long)hi * from->src_outer;
        }
        if (conv) cc.up_src = conv->up_src + (g0 / conv->up_div) * conv->up_src_stride;
        if (epi) {
            rr.epi_a = epi->epi_a + g0 * epi->epi_a_stride;
            rr.epi_out = epi->epi_out + g0 * epi->epi_out_stride;
        }
        if (own) rr.own_out = own->own_out + g0 * own->own_nd * own->own_E * c.N;
        const u32 pc = (u32)(gn * nlimbs);
        const dim3 gcols(pc, (1u << R) >> cols.logC);
        const dim3 grows(pc, (1u << S1) >> rows.logC);
        if (FWD) {
            if (up_src) PDQ_TRY((launch_phase<true, true, false, true>((int)S1, gcols, kThreads, cc, st)));
            else PDQ_TRY((launch_phase<FWD, true, false>((int)S1, gcols, kThreads, cc, st)));
            if (epi) PDQ_TRY((launch_rows<true, true>(R, grows, rr, st)));
            else PDQ_TRY(launch_rows<FWD>(R, grows, rr, st));
        } else {
            if (own) PDQ_TRY((launch_rows<false, false, true>(R, grows, rr, st)));
            else PDQ_TRY(launch_rows<FWD>(R, grows, rr, st));
            PDQ_TRY((launch_phase<FWD, true, false>((int)S1, gcols, kThreads, cc, st)));
        }
    }
    return PDQ_OK;
}

}  // namespace

int ntt_forward(const Ctx& c, u64* data, u32 count, u32 nlimbs, u32 limb0, u64 stride,
                cudaStream_t st) {
    return ntt_run<true>(c, data, count, nlimbs, limb0, stride, st);
}

int ntt_inverse(const Ctx& c, u64* data, u32 count, u32 nlimbs, u32 limb0, u64 stride,
                cudaStream_t st, const u64* ninv_tab) {
    return ntt_run<false>(c, data, count, nlimbs, limb0, stride, st, nullptr, 0, 0, ninv_tab);
}

int ntt_forward_digits(const Ctx& c, u64* D, u32 count, u32 nd, u32 alpha, u32 nlimbs,
                       cudaStream_t st) {
    if (nd == 0 || alpha == 0) return fail(PDQ_E_PARAM, "ntt: bad digit layout");
    return ntt_run<true>(c, D, count * nd, nlimbs - alpha, 0, (u64)nlimbs * c.N, st, nullptr, nd,
                         alpha);
}

int ntt_forward_digits_modup(const Ctx& c, u64* D, const u64* Y, u32 count, u32 nd, u32 alpha,
                             u32 nlimbs, cudaStream_t st) {
    if (nd == 0 || alpha == 0 || !Y) return fail(PDQ_E_PARAM, "ntt: bad digit layout");
    NttArgs cv{};
    cv.up_src = Y;
    cv.up_hm = reinterpret_cast<const ulonglong2*>(c.d_up_mont2);
    cv.up_src_stride = (u64)c.L * c.N;     // y of one ciphertext, [L][N]
    cv.up_div = nd;                        // digits per ciphertext
    cv.up_i0_step = alpha;                 // digit b's limbs start at b alpha
    cv.up_n = alpha;
    cv.up_E = c.L + c.K;
    return ntt_run<true>(c, D, count * nd, nlimbs - alpha, 0, (u64)nlimbs * c.N, st, nullptr, nd,
                         alpha, nullptr, &cv);
}

int ntt_forward_moddown(const Ctx& c, u64* Cv, const u64* S, u64 s_stride, u32 count,
                        cudaStream_t st, const u64* A, u64 a_stride, u64* out, u64 out_stride) {
    if (!S || c.K == 0 || c.K > 2) return fail(PDQ_E_PARAM, "ntt: the fused ModDown takes 1 or 2 special primes");
    NttArgs cv{};
    cv.up_src = S;
    cv.up_hm = reinterpret_cast<const ulonglong2*>(c.d_dn_pair);
    cv.up_src_stride = s_stride;
    cv.up_div = 1;
    cv.up_i0_step = 0;
    cv.up_n = c.K;
    cv.up_E = c.L;                         // pairs [K][L]
    if (!A) return ntt_run<true>(c, Cv, count, c.L, 0, (u64)c.L * c.N, st, nullptr, 0, 0, nullptr, &cv);
    NttArgs ep{};
    ep.epi_a = A;
    ep.epi_a_stride = a_stride;
    ep.epi_out = out;
    ep.epi_out_stride = out_stride;
    ep.epi_pinv = c.d_dn_pinv;
    ep.epi_pinvs = c.d_dn_pinv_shoup;
    return ntt_run<true>(c, Cv, count, c.L, 0, (u64)c.L * c.N, st, nullptr, 0, 0, nullptr, &cv, &ep);
}

int ntt_inverse_from(const Ctx& c, const u64* src, long long src_outer, u32 src_per,
                     long long src_inner, u64 src_off, u64* data, u32 count, u32 nlimbs,
                     u64 stride, cudaStream_t st, u32 limb0, const u64* ninv_tab, u64* own_out) {
    if (src_per == 0) return fail(PDQ_E_PARAM, "ntt: bad source set");
    NttArgs from{};
    from.src = src;
    from.src_outer = src_outer;
    from.src_inner = src_inner;
    from.src_per = src_per;
    from.src_off = src_off;
    if (own_out) {
        NttArgs ow{};
        ow.own_out = own_out;
        ow.own_nd = c.ndigits;
        ow.own_alpha = c.alpha;
        ow.own_E = c.L + c.K;
        return ntt_run<false>(c, data, count, nlimbs, limb0, stride, st, &from, 0, 0, ninv_tab,
                              nullptr, nullptr, &ow);
    }
    return ntt_run<false>(c, data, count, nlimbs, limb0, stride, st, &from, 0, 0, ninv_tab);
}

}  // namespace pdq
