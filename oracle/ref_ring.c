/*
 * Plain reference arithmetic for the ring R_q = Z_q[X]/(X^N + 1).
 *
 * TEST INFRASTRUCTURE ONLY.  This file belongs to the CPU oracle that the
 * parity tests compare the CUDA library against.  Only tests/, the smoke
 * check and the benchmark's CPU-baseline leg may load it; the library never
 * does, and it shares no source with the library.
 *
 * Everything here is the textbook definition written out with 128-bit
 * integer division for every modular product ("a*b % q"): no Shoup or
 * Barrett tricks, no lazy reduction, no blocking.  Values are canonical
 * residues in [0, q) on entry and on exit of every function.
 *
 * Ring of the BGV/BFV schemes (Sec. 5.1): ciphertexts live in R_q^2 with
 * q a product of primes; one "limb" is one polynomial modulo one prime.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef uint64_t u64;
typedef unsigned __int128 u128;

static u64 mulmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }
static u64 addmod(u64 a, u64 b, u64 q) { u64 s = a + b; return s >= q ? s - q : s; }
static u64 submod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }

u64 ref_powmod(u64 a, u64 e, u64 q) {
    u64 r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = mulmod(r, a, q);
        a = mulmod(a, a, q);
        e >>= 1;
    }
    return r;
}

/* Inverse by Fermat's little theorem (q prime). */
u64 ref_invmod(u64 a, u64 q) { return ref_powmod(a, q - 2, q); }

/* Slot-wise (coefficient-wise) product c = a .* b mod q, n entries. */
void ref_vec_mul(const u64 *a, const u64 *b, u64 *c, u64 n, u64 q) {
    for (u64 i = 0; i < n; i++) c[i] = mulmod(a[i], b[i], q);
}

/* c += a .* b mod q. */
void ref_vec_mac(const u64 *a, const u64 *b, u64 *c, u64 n, u64 q) {
    for (u64 i = 0; i < n; i++) c[i] = addmod(c[i], mulmod(a[i], b[i], q), q);
}

void ref_vec_add(const u64 *a, const u64 *b, u64 *c, u64 n, u64 q) {
    for (u64 i = 0; i < n; i++) c[i] = addmod(a[i], b[i], q);
}

void ref_vec_sub(const u64 *a, const u64 *b, u64 *c, u64 n, u64 q) {
    for (u64 i = 0; i < n; i++) c[i] = submod(a[i], b[i], q);
}

/* c = a * w mod q for a scalar w. */
void ref_vec_scale(const u64 *a, u64 w, u64 *c, u64 n, u64 q) {
    for (u64 i = 0; i < n; i++) c[i] = mulmod(a[i], w % q, q);
}

/*
 * Negacyclic product by its definition:  c = a * b in Z_q[X]/(X^N + 1),
 *   c_k = sum_{i+j=k} a_i b_j  -  sum_{i+j=k+N} a_i b_j.
 * O(N^2); used to pin the transform-based product on small N.
 */
void ref_negacyclic_schoolbook(const u64 *a, const u64 *b, u64 *c, u64 N, u64 q) {
    for (u64 k = 0; k < N; k++) c[k] = 0;
    for (u64 i = 0; i < N; i++) {
        if (a[i] == 0) continue;
        for (u64 j = 0; j < N; j++) {
            u64 p = mulmod(a[i], b[j], q);
            u64 k = i + j;
            if (k < N) c[k] = addmod(c[k], p, q);
            else c[k - N] = submod(c[k - N], p, q);
        }
    }
}

/* Bit reversal of the low `bits` bits of x. */
static u64 bitrev(u64 x, int bits) {
    u64 r = 0;
    for (int i = 0; i < bits; i++) { r = (r << 1) | (x & 1); x >>= 1; }
    return r;
}

/*
 * Cyclic DFT over Z_q of length N = 2^logN with root omega, natural order
 * in and out:  A_j = sum_i a_i omega^{ij}.  Textbook iterative radix-2
 * Cooley-Tukey: bit-reversal permutation, then log N butterfly levels.
 */
static void cyclic_dft(u64 *a, int logN, u64 q, u64 omega) {
    u64 N = (u64)1 << logN;
    for (u64 i = 0; i < N; i++) {
        u64 r = bitrev(i, logN);
        if (r > i) { u64 tmp = a[i]; a[i] = a[r]; a[r] = tmp; }
    }
    for (u64 len = 2; len <= N; len <<= 1) {
        u64 wlen = ref_powmod(omega, N / len, q); /* primitive len-th root */
        for (u64 start = 0; start < N; start += len) {
            u64 w = 1;
            for (u64 k = 0; k < len / 2; k++) {
                u64 u = a[start + k];
                u64 v = mulmod(a[start + k + len / 2], w, q);
                a[start + k] = addmod(u, v, q);
                a[start + k + len / 2] = submod(u, v, q);
                w = mulmod(w, wlen, q);
            }
        }
    }
}

/*
 * Negacyclic transform: evaluation of a(X) at the odd powers of a primitive
 * 2N-th root psi, natural order:  out_j = a(psi^{2j+1}) = sum_i a_i psi^i omega^{ij}
 * with omega = psi^2.  In place.
 */
void ref_ntt_forward(u64 *a, int logN, u64 q, u64 psi) {
    u64 N = (u64)1 << logN;
    u64 pw = 1;
    for (u64 i = 0; i < N; i++) { a[i] = mulmod(a[i], pw, q); pw = mulmod(pw, psi, q); }
    cyclic_dft(a, logN, q, mulmod(psi, psi, q));
}

/* Inverse of ref_ntt_forward: interpolation from the values at psi^{2j+1}. */
void ref_ntt_inverse(u64 *a, int logN, u64 q, u64 psi) {
    u64 N = (u64)1 << logN;
    u64 psi_inv = ref_invmod(psi, q);
    cyclic_dft(a, logN, q, mulmod(psi_inv, psi_inv, q));
    u64 n_inv = ref_invmod(N % q, q);
    u64 pw = n_inv;
    for (u64 i = 0; i < N; i++) { a[i] = mulmod(a[i], pw, q); pw = mulmod(pw, psi_inv, q); }
}

/* Negacyclic product through the transform: c = INTT(NTT(a) .* NTT(b)). */
void ref_negacyclic_mul(const u64 *a, const u64 *b, u64 *c, int logN, u64 q, u64 psi) {
    u64 N = (u64)1 << logN;
    u64 *ta = (u64 *)malloc(N * sizeof(u64));
    u64 *tb = (u64 *)malloc(N * sizeof(u64));
    memcpy(ta, a, N * sizeof(u64));
    memcpy(tb, b, N * sizeof(u64));
    ref_ntt_forward(ta, logN, q, psi);
    ref_ntt_forward(tb, logN, q, psi);
    for (u64 i = 0; i < N; i++) c[i] = mulmod(ta[i], tb[i], q);
    ref_ntt_inverse(c, logN, q, psi);
    free(ta);
    free(tb);
}

/*
 * Galois automorphism sigma_k : a(X) -> a(X^k) on R_q, k odd (Sec. 5.1:
 * the row rotations are k = 3^r, the column swap is k = 2N-1).  Since
 * X^N = -1, the coefficient a_j moves to X^{jk mod N} with sign
 * (-1)^{floor(jk / N)}.
 */
void ref_automorphism(const u64 *a, u64 *out, u64 N, u64 k, u64 q) {
    for (u64 j = 0; j < N; j++) {
        u128 e = (u128)j * k;
        u64 dst = (u64)(e % N);
        u64 wraps = (u64)((e / N) & 1);
        out[dst] = wraps ? submod(0, a[j], q) : a[j];
    }
}

/*
 * Fast basis conversion of one polynomial from the primes src[0..ns) to a
 * prime r (coefficient form):
 *   y = sum_i [x_i * hat_inv_i]_{src_i} * hat_mod_r_i  mod r,
 * where hat = (prod src)/src_i, hat_inv_i = hat^{-1} mod src_i and
 * hat_mod_r_i = hat mod r.  x is laid out [ns][N].  No overflow correction
 * (the result may exceed the exact CRT value by a multiple of prod src).
 */
void ref_basis_convert(const u64 *x, const u64 *src, const u64 *hat_inv, u64 ns,
                       const u64 *hat_mod_r, u64 r, u64 *y, u64 N) {
    for (u64 c = 0; c < N; c++) {
        u64 acc = 0;
        for (u64 i = 0; i < ns; i++) {
            u64 v = mulmod(x[i * N + c], hat_inv[i], src[i]);
            acc = addmod(acc, mulmod(v % r, hat_mod_r[i], r), r);
        }
        y[c] = acc;
    }
}

/* x mod r for residues given modulo another prime (values < 2^64). */
void ref_vec_reduce(const u64 *x, u64 *y, u64 n, u64 r) {
    for (u64 i = 0; i < n; i++) y[i] = x[i] % r;
}
