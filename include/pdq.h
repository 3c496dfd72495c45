/*
 * pdq.h -- C ABI of the GB300 library for the server-side hot path of the
 * HE-based private database query of "SIMD-Aware Homomorphic Compression and
 * Application to Private Database Query" (arXiv 2408.17063).
 *
 * The path is Answer = Mask -> Comp (Alg. 7): the client's encrypted 0/1
 * index vector v (the output of Match) is multiplied slot-wise with the
 * database, and the masked ciphertexts are compressed by the homomorphic
 * matrix-vector product with the power-sum matrix C[j][i] = i^j (Eq. 1) in
 * the SIMD form of Sec. 5.2: u = [v; d] packing, Pegasus diagonals with
 * baby-step/giant-step rotations on both rows, blocks summed before one
 * rotate-and-sum.  The client decompresses with Newton's identity, root
 * finding and a Vandermonde solve (Alg. 1, 4, 6).
 *
 * Notation: N is the ring dimension (the paper's n), n the number of records
 * (the paper's N), t the plaintext prime (the paper's p), m = N/2 slots per
 * row, s' = 2^ceil(log2 s) the compressed length per row.
 *
 * Conventions for every call:
 *  - Return value: PDQ_OK (0) or an error code; pdq_last_error() gives a
 *    message for the calling thread.  No call throws across the ABI.
 *  - "dev" pointers are CUDA device pointers, "host" pointers host memory.
 *    The caller owns every buffer it passes; the library never frees them.
 *    A NULL buffer that a call would touch is refused with PDQ_E_PARAM
 *    before any work is queued (a zero count touches none).
 *    The context owns only its own tables (allocated in pdq_ctx_create).
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *    enqueued asynchronously on it unless a call says otherwise; buffers must
 *    stay valid until the stream reaches that point.
 *  - Residues are uint64 in [0, q).  A polynomial over the ciphertext primes
 *    is [L][N] (limb-major); over the extended basis [L+K][N] (the L
 *    ciphertext primes first, then the K special primes).  A ciphertext is
 *    [2][L][N]; J ciphertexts are contiguous, [J][2][L][N].  Device-side
 *    ciphertexts, keys and plaintexts are in the library's transform
 *    (evaluation) domain ("NTT form"); pdq_ntt_inverse gives coefficient
 *    form, which is what is compared with other implementations.
 *  - Slots of one plaintext are [N] uint32 with slot (row rho, column c) at
 *    index rho*m + c; record i of a database sits in ciphertext floor(i/N),
 *    slot i mod N.
 */
#ifndef PDQ_H
#define PDQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PDQ_OK 0
#define PDQ_E_PARAM 1    /* invalid argument or unsupported size */
#define PDQ_E_NOMEM 2    /* workspace too small or allocation failed */
#define PDQ_E_CUDA 3     /* CUDA runtime error (message has the detail) */
#define PDQ_E_DECODE 4   /* Decomp found no consistent sparse answer */
#define PDQ_E_KEY 5      /* a needed rotation key is missing */
#define PDQ_E_TIMEOUT 6  /* a wait ran out */
#define PDQ_E_BUSY 7     /* the server's queue is full */

#define PDQ_MAX_MODULI 40

typedef struct pdq_ctx pdq_ctx;

/* Parameter set (Sec. 5.1: ring X^N+1 with N a power of two, t = 1 mod 2N). */
typedef struct {
    uint32_t log_n;       /* N = 2^log_n, 3 <= log_n <= 16 */
    uint32_t prime_bits;  /* every RNS prime is < 2^prime_bits (<= 60) */
    uint32_t L;           /* ciphertext primes */
    uint32_t K;           /* special primes for hybrid key switching */
    uint32_t dnum;        /* key-switching digits: ceil(L / ceil(L/dnum)) */
    uint32_t reserved;
    uint64_t t;           /* plaintext prime, t = 1 mod 2N, t < 2^31 */
} pdq_params;

typedef struct {
    uint32_t N, L, K, ndigits;
    uint64_t t;
    uint64_t zeta;                      /* slot root mod t */
    uint64_t moduli[PDQ_MAX_MODULI];    /* q_0..q_{L-1}, p_0..p_{K-1} */
    uint64_t psi[PDQ_MAX_MODULI];       /* transform root (order 2N) per
                                           modulus; index L+K is t (= zeta) */
} pdq_info;

/* Layout of one query's compression (Sec. 5.2 with the readings below).
 * Records are split into groups of G_sz = N*floor((t-1)/N) consecutive
 * records so that the nodes 1..G_sz of Eq. 1 stay distinct mod t (the paper
 * assumes t > n); group gamma's (Cv, Cd) block lands in output ciphertext
 * floor(gamma/per_out) at slot offset (gamma mod per_out)*s'. */
typedef struct {
    uint64_t n;          /* records */
    uint32_t s;          /* sparsity bound (matches per group) */
    uint32_t s_prime;    /* 2^ceil(log2 s) */
    uint32_t B;          /* baby steps (divides s') */
    uint32_t giants;     /* s'/B */
    uint32_t J;          /* index-vector ciphertexts ceil(n/N) */
    uint32_t H;          /* half-blocks = u ciphertexts = 2J */
    uint32_t G_sz;       /* records per group */
    uint32_t hpg;        /* half-blocks per group */
    uint32_t G;          /* groups */
    uint32_t hclass;     /* distinct diagonal sets = min(hpg, H) */
    uint32_t per_out;    /* groups per output ciphertext = m/s' */
    uint32_t n_out;      /* output ciphertexts */
    uint32_t ring_ratio; /* 1; R = N_big/N for Comp in a subring after ring
                            switching (pdq_plan_make_switched) */
    uint32_t plain_db;   /* 1 for the Answer on an unencrypted database
                            (pdq_plan_make_plain_db), else 0 */
} pdq_plan;

/* ---------------------------------------------------------------- context */

/* Build the prime chain, transform tables, slot permutation and key-switching
 * constants of one parameter set on the current device: the ring and the
 * plaintext prime of Sec. 5.1, the modulus chain of Sec. 6.1 (there: two
 * 54-bit primes) extended by K special primes for hybrid key switching.
 * Synchronous.  *out is owned by the caller and released with
 * pdq_ctx_destroy.  Errors: PDQ_E_PARAM for unsupported sizes, PDQ_E_NOMEM /
 * PDQ_E_CUDA on device failures. */
int pdq_ctx_create(const pdq_params* params, pdq_ctx** out);
/* Release a context and its device tables (no operation of the paper; the
 * caller's buffers are untouched).  NULL is accepted. */
int pdq_ctx_destroy(pdq_ctx* ctx);
/* The parameters a context derived (the primes and roots of Sec. 5.1's ring
 * and slot structure) into host *info. */
int pdq_ctx_info(const pdq_ctx* ctx, pdq_info* info);
/* Message of the calling thread's last error (library bookkeeping; never
 * NULL, owned by the library until the thread's next failing call). */
const char* pdq_last_error(void);

/* Memory of the baby-step rotations (Sec. 5.2: Rot(u_h; a), a < B, for every
 * half-block, consumed by the diagonal products).  By default pdq_answer and
 * pdq_comp hold all of them at once (at N = 2^15, n = 2^20, B = 32: 10 GiB
 * of the 13.9 GiB workspace).  With a budget of `bytes` > 0 they are made
 * and consumed a chunk of primes at a time (each prime's rotations and
 * products are independent), holding at most max(bytes, one prime's
 * rotations); the results are the same bits, and
 * pdq_answer_workspace_bytes / pdq_comp_workspace_bytes shrink accordingly.
 * Set it before sizing workspaces; not while a call on the context runs. */
int pdq_ctx_set_rotation_budget(pdq_ctx* ctx, uint64_t bytes);

/* Launch schedule of the transforms and of the diagonal multiply-accumulate
 * (Sec. 5.2's products): the knobs an autotuner searches; every schedule
 * gives the same bits.  ntt_row_bits: levels in the row phase of a transform
 * of N > 2^11, 7..11 and below log N (the column phase takes the other
 * levels); mac_tiles: position tiles per multiply-accumulate CTA, 1, 2, 4 or
 * 8; mac_bc: baby steps staged per copy step, 1, 2, 4, 8 or 16 (fewer where
 * shared memory requires); ntt_chunk: polynomials per launch pair of a
 * two-phase transform (a call over more runs in chunks, so that a chunk's
 * intermediate between the phases can stay in L2; rounded to whole
 * ciphertexts), 0 or 64..2^20.  0 keeps the library's rule for a knob (9 row
 * levels; 8 tiles while 64 CTAs per prime remain; 16 baby steps; no chunks).
 * Errors: PDQ_E_PARAM for other values.  Set it before the calls it should
 * affect, not while a call on the context runs. */
typedef struct {
    uint32_t ntt_row_bits;
    uint32_t mac_tiles;
    uint32_t mac_bc;
    uint32_t ntt_chunk;
} pdq_schedule;
int pdq_ctx_set_schedule(pdq_ctx* ctx, const pdq_schedule* sched);
int pdq_ctx_get_schedule(const pdq_ctx* ctx, pdq_schedule* sched);

/* ------------------------------------------------------------- transforms
 * Negacyclic transform of polynomials in Z_q[X]/(X^N+1) (the ring of
 * Sec. 5.1), in place on `count` groups of `nlimbs` limbs: group g, limb l is
 * at data + g*stride + l*N (uint64 elements) and uses extended-basis modulus
 * limb0 + l (index L+K is the plaintext prime t).  dev data. */
int pdq_ntt_forward(const pdq_ctx* ctx, uint64_t* data, uint32_t count, uint32_t nlimbs,
                    uint32_t limb0, uint64_t stride, void* stream);
int pdq_ntt_inverse(const pdq_ctx* ctx, uint64_t* data, uint32_t count, uint32_t nlimbs,
                    uint32_t limb0, uint64_t stride, void* stream);

/* ------------------------------------------------------- encode / keys
 * Encode `count` slot vectors (dev [count][N] uint32, values < t) into
 * NTT-form plaintexts over the first nlimbs extended-basis primes (dev
 * pt_out [count][nlimbs][N]): interpolation mod t at the slot roots
 * (Sec. 5.1), centred lift to (-t/2, t/2], forward transform. */
int pdq_encode(const pdq_ctx* ctx, const uint32_t* slots, uint32_t count, uint32_t nlimbs,
               uint64_t* pt_out, void* stream);

/* The secret key s of HE KeyGen (Sec. 2.2), a ternary polynomial: dev [N]
 * int8 in {-1,0,1} -> NTT form over the extended basis (dev sk_out
 * [L+K][N]), the form pdq_encrypt, pdq_rotkey_gen and pdq_decrypt take.
 * PDQ_E_PARAM for a null pointer; coefficients outside {-1,0,1} are not
 * checked here (pdq_sk_export refuses them). */
int pdq_secret_prepare(const pdq_ctx* ctx, const int8_t* s, uint64_t* sk_out, void* stream);

/* Symmetric BFV encryption of `count` slot vectors (HE Enc, Sec. 2.2):
 * c1 = a, c0 = -a*s + e + floor(Q/t)*m.  The caller supplies the
 * randomness: a = dev [count][L][N] uniform residues in coefficient form,
 * e = dev [count][N] small integers.  ct_out: dev [count][2][L][N]. */
int pdq_encrypt(const pdq_ctx* ctx, const uint64_t* sk, const uint32_t* slots, uint32_t count,
                const uint64_t* a, const int32_t* e, uint64_t* ct_out, void* stream);

/* Hybrid key-switching key from sigma_k(s) to s (an evaluation key of HE
 * KeyGen, Sec. 2.2, for the rotations of Sec. 5.1) for the Galois element
 * `galois` (k odd, < 2N; Rot_row(.; r) is k = 3^r, Rot_col is k = 2N-1):
 * per digit beta, b = -a*s + e + [q_i in beta] * P * sigma_k(s).  a: dev
 * [ndigits][L+K][N] uniform coefficient form, e: dev [ndigits][N].
 * key_out: dev [ndigits][2][L+K][N] NTT form. */
int pdq_rotkey_gen(const pdq_ctx* ctx, const uint64_t* sk, uint64_t galois, const uint64_t* a,
                   const int32_t* e, uint64_t* key_out, void* stream);

/* HE Dec + decode (Sec. 2.2, Alg. 6 first line): m = round(t [c0 + c1 s]_Q / Q)
 * mod t, then the slot values.  ct: dev [count][2][L][N]; slots_out: dev
 * [count][N] uint32.  pdq_decrypt_workspace_bytes(count) is the dev scratch
 * this needs (smaller -> PDQ_E_NOMEM). */
size_t pdq_decrypt_workspace_bytes(const pdq_ctx* ctx, uint32_t count);
int pdq_decrypt(const pdq_ctx* ctx, const uint64_t* sk, const uint64_t* ct, uint32_t count,
                uint32_t* slots_out, void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------- homomorphic rotation
 * ct_out[i] = sigma_k(ct_in[i]) followed by hybrid key switching with `key`
 * (the key for `galois`), for i < count (Rot_row / Rot_col of Sec. 5.1).
 * The raised digits of c1 are computed before the automorphism.  ct_in and
 * ct_out: dev [count][2][L][N], may not overlap.  Workspace (dev):
 * pdq_rotate_workspace_bytes(count) bytes, the raised digits of Sec. 5.1's
 * key switching and the inner-product scratch; smaller -> PDQ_E_NOMEM. */
size_t pdq_rotate_workspace_bytes(const pdq_ctx* ctx, uint32_t count);
int pdq_rotate(const pdq_ctx* ctx, const uint64_t* ct_in, uint32_t count, uint64_t galois,
               const uint64_t* key, uint64_t* ct_out, void* ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------------ modulus switching
 * Comp needs one multiplicative level, so it can run with smaller HE
 * parameters than the query (Sec. 5.3 switches to a smaller parameter set
 * after Match and Mask; here the modulus is switched in the same ring).
 * Ciphertexts over Q = q_0..q_{L-1} of `from` ([count][2][L][N], NTT form)
 * become ciphertexts over Q' = q_0..q_{L'-1} of `to` ([count][2][L'][N]): the
 * ModDown formula with the dropped primes D = q_{L'}..q_{L-1} in the role of P,
 *   c'_i = (c_i - sum_k [c_{d_k} (D/d_k)^-1]_{d_k} (D/d_k)) D^-1  mod q_i,
 * so c0 + c1 s = Delta m + e becomes Delta' m + e'.  `to` must have the same
 * N and t and fewer primes, its ciphertext primes the first L' of `from`
 * (contexts with the same K and prime size have that), else PDQ_E_PARAM; at
 * most 8 primes dropped.  cts is not modified; out may not overlap it.
 * Workspace: pdq_mod_switch_workspace_bytes(from, count), else PDQ_E_NOMEM. */
size_t pdq_mod_switch_workspace_bytes(const pdq_ctx* from, uint32_t count);
int pdq_mod_switch(const pdq_ctx* from, const pdq_ctx* to, const uint64_t* cts, uint32_t count,
                   uint64_t* out, void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------- ring switching
 * Comp needs one multiplicative level, so the paper switches the query to a
 * ring of smaller dimension after Match and Mask (Sec. 5.3, the ring-switching
 * technique of Gentry, Halevi, Peikert and Smart): Comp is cheaper there and
 * the answer shorter.  A big-ring ciphertext under s is key-switched to the
 * subring secret s'(X) = s_small(X^R), R = N_big/N_small, then split by
 * coefficient index mod R into R subring ciphertexts over the same primes:
 * part r decrypts under s_small to m_r, where the plaintext is
 * m(X) = sum_r X^r m_r(X^R).
 * pdq_ctx_create_subring: the context of the subring of dimension 2^log_n
 *   (3 <= log_n < the parent's) with the parent's t, primes and digits.
 *   Synchronous; released with pdq_ctx_destroy.
 * pdq_ring_switch_key_gen (client): the key from s (sk: big-ring
 *   pdq_secret_prepare form) to s_small(X^R) (s_small: dev [N_small] int8
 *   ternary), b = -a s' + e + [q_i in digit] P s per digit; a: dev
 *   [ndigits][L+K][N_big] uniform coefficient form, e: dev [ndigits][N_big];
 *   key_out: dev [ndigits][2][L+K][N_big] NTT form.  Allocates temporaries.
 * pdq_ring_switch: cts dev [count][2][L][N_big] (NTT form, unchanged); part r
 *   of ciphertext i is written (NTT form of the subring) to out at index
 *   (i / group) group R + r group + i mod group, each [2][L][N_small]: group 1
 *   gives [count][R], group 4 turns pdq_mask's output ([J][4]) into a valid
 *   pdq_comp input of the subring ([R J][4]; a subring row folds only slots
 *   of the same big row, so the row masks carry over).  count must be a
 *   multiple of group.  Workspace: pdq_ring_switch_workspace_bytes(big, count)
 *   (dev), else PDQ_E_NOMEM.  PDQ_E_PARAM if small is not a subring of big. */
int pdq_ctx_create_subring(const pdq_ctx* big, uint32_t log_n, pdq_ctx** out);
int pdq_ring_switch_key_gen(const pdq_ctx* big, const pdq_ctx* small, const uint64_t* sk,
                            const int8_t* s_small, const uint64_t* a, const int32_t* e,
                            uint64_t* key_out, void* stream);
size_t pdq_ring_switch_workspace_bytes(const pdq_ctx* big, uint32_t count);
int pdq_ring_switch(const pdq_ctx* big, const pdq_ctx* small, const uint64_t* cts, uint32_t count,
                    uint32_t group, const uint64_t* key, uint64_t* out, void* ws, size_t ws_bytes,
                    void* stream);

/* ----------------------------------------------------------------- plans
 * Fill the layout for n records and sparsity s (s' = 2^ceil(log2 s), the
 * Pegasus baby-step/giant-step split k = gB + a of Sec. 5.2).  B = 0 picks
 * the power of two B <= min(s', 128) with at most 32 giant steps that
 * minimises H (B - 1) + 8 G (s'/B - 1) + 3 G s'/B (hoisted baby rotations,
 * giant-step key switches and accumulator ModDowns, weighted by their
 * measured costs), ties to the smaller B.  Errors: PDQ_E_PARAM if s' > N/2,
 * s' >= t, B does not divide s', B > 128 or s'/B > 32. */
int pdq_plan_make(const pdq_ctx* ctx, uint64_t n, uint32_t s, uint32_t B, pdq_plan* plan);
/* The same plan without a context, from the plaintext prime t and the ring
 * X^N + 1, N = 2^log_n, alone (the layout of Sec. 5.2 depends on nothing
 * else): for a client that computes the answer's layout on a machine with no
 * GPU.  Host only, synchronous; nothing is allocated.  Errors as
 * pdq_plan_make's, and PDQ_E_PARAM unless 3 <= log_n <= 16 and t is a prime
 * < 2^31 with t = 1 mod 2N (the checks of pdq_ctx_create). */
int pdq_plan_make_client(uint64_t t, uint32_t log_n, uint64_t n, uint32_t s, uint32_t B,
                         pdq_plan* plan);

/* The plan of Comp in the subring `small` on a query ring-switched from the
 * ring of dimension 2^big_log_n (Sec. 5.3): J = R ceil(n / N_big) subring
 * ciphertexts (part r of big ciphertext j at R j + r, as pdq_ring_switch
 * writes them with group 4 after pdq_mask), the big ring's record groups
 * (G_sz = N_big floor((t-1)/N_big)), the slot layout of the subring, and
 * ring_ratio = R.  pdq_plan_constants_build then makes the diagonals that
 * undo the slot fold of the split, so the answer holds the same power sums
 * of Eq. 1 as pdq_answer's and pdq_decomp (with this plan and the subring
 * context) recovers the matches.  Errors as pdq_plan_make, and PDQ_E_PARAM
 * unless N < 2^big_log_n <= 2^16 and t = 1 mod 2^(big_log_n+1). */
int pdq_plan_make_switched(const pdq_ctx* small, uint32_t big_log_n, uint64_t n, uint32_t s,
                           uint32_t B, pdq_plan* plan);

/* The Galois elements of every rotation the plan uses, ascending (host
 * out[cap]); *count receives how many there are (PDQ_E_NOMEM if cap is
 * smaller).  These are Rot_col of the u-packing remark (2N-1) and the row
 * rotations 3^r of Sec. 5.2's baby steps (r = 1..B-1), giant steps (r = gB)
 * and rotate-and-sum (r = j l per level); the client makes one key per
 * element (pdq_rotkey_gen).  The key buffer passed to pdq_comp holds one key
 * per element in this order. */
int pdq_plan_galois(const pdq_ctx* ctx, const pdq_plan* plan, uint64_t* out, uint32_t cap,
                    uint32_t* count);
/* The same list without a context, from t and the ring X^N + 1, N = 2^log_n
 * (the plan's ring: the subring for a ring-switched plan), as
 * pdq_plan_make_client: the client learns which rotation keys (Sec. 5.2) to
 * make and send on a machine with no GPU.  Host only; errors as
 * pdq_plan_galois's, and PDQ_E_PARAM for a ring or prime that
 * pdq_ctx_create would refuse. */
int pdq_plan_galois_client(uint64_t t, uint32_t log_n, const pdq_plan* plan, uint64_t* out,
                           uint32_t cap, uint32_t* count);

/* Query-independent constants of a plan: the extended diagonals
 *   D_{h,k}[c] = alpha(h m + ((c+k) mod m))^{(c mod s')+1} mod t,
 * alpha(i) = (i mod G_sz) + 1, rotated by -gB for k = gB + a, encoded on both
 * rows (Sec. 5.2: "encoding C twice") over every prime of Q u P, for the
 * hclass distinct half-block classes; then the group masks.  The layout is
 * internal to the library (the diagonals are stored in the operand format of
 * its multiply-accumulate).  dev out of pdq_plan_constants_bytes. */
size_t pdq_plan_constants_bytes(const pdq_ctx* ctx, const pdq_plan* plan);
int pdq_plan_constants_build(const pdq_ctx* ctx, const pdq_plan* plan, uint64_t* out,
                             void* stream);

/* Database plaintexts: for each index ciphertext j, DB_j . [1;0] and
 * DB_j . [0;1] (the row masks of the u-packing remark of Sec. 5.2 folded
 * into the database), NTT form.  values: dev [n] uint32 (< t).  db_out: dev
 * [J][2][L][N] (pdq_db_bytes). */
size_t pdq_db_bytes(const pdq_ctx* ctx, uint64_t n);
int pdq_db_encode(const pdq_ctx* ctx, const uint32_t* values, uint64_t n, uint64_t* db_out,
                  void* stream);

/* The u-packing remark's literal order (Sec. 5.2, remark (ii)): the masked
 * database d = v.DB first, then the row masks, one plaintext product more on
 * d than pdq_mask (the same slots, more noise).  pdq_db_encode_plain writes
 * DB_j on both rows without masks, dev [J][L][N] (pdq_db_plain_bytes;
 * values < t, else reduced mod t); pdq_mask_literal writes, for each index
 * ciphertext j, (v_j.[1;0], v_j.[0;1], (v_j.DB_j).[1;0], (v_j.DB_j).[0;1]) in
 * the layout of pdq_mask (dev [J][4][2][L][N]), a valid input of pdq_comp. */
size_t pdq_db_plain_bytes(const pdq_ctx* ctx, uint64_t n);
int pdq_db_encode_plain(const pdq_ctx* ctx, const uint32_t* values, uint64_t n, uint64_t* db_out,
                        void* stream);
int pdq_mask_literal(const pdq_ctx* ctx, const pdq_plan* plan, const uint64_t* v_cts,
                     const uint64_t* db_plain, uint64_t* masked_out, void* stream);

/* ------------------------------------------------------------ hot path
 * Mask (Alg. 7 step 2, with the row split of the u-packing remark): for each
 * index ciphertext j, vT = v_j.[1;0], vB = v_j.[0;1], dT = v_j.(DB_j.[1;0]),
 * dB = v_j.(DB_j.[0;1]).  v_cts: dev [J][2][L][N]; db from pdq_db_encode;
 * masked_out: dev [J][4][2][L][N]. */
int pdq_mask(const pdq_ctx* ctx, const pdq_plan* plan, const uint64_t* v_cts,
             const uint64_t* db, uint64_t* masked_out, void* stream);

/* Comp (Alg. 7 step 3 in the SIMD form of Sec. 5.2): pack u_h = [v_h; d_h]
 * with Rot_col, baby-step rotations of every u_h, diagonal multiply-
 * accumulate per group and giant step, giant-step rotations, rotate-and-sum,
 * group masks.  masked: dev output of pdq_mask; keys: dev, one key per
 * element of pdq_plan_galois in that order ([nkeys][ndigits][2][L+K][N]);
 * galois: host [nkeys]; consts from pdq_plan_constants_build.  out: dev
 * [n_out][2][L][N], row 0 of group gamma's block = Cv, row 1 = Cd.
 * Workspace: pdq_comp_workspace_bytes; too small -> PDQ_E_NOMEM. */
size_t pdq_comp_workspace_bytes(const pdq_ctx* ctx, const pdq_plan* plan);
int pdq_comp(const pdq_ctx* ctx, const pdq_plan* plan, const uint64_t* masked,
             const uint64_t* keys, const uint64_t* galois, uint32_t nkeys,
             const uint64_t* consts, uint64_t* out, void* ws, size_t ws_bytes, void* stream);

/* Answer = Mask then Comp on device buffers (Alg. 7 without Match).  The
 * pack's column rotation is applied to each index ciphertext before the Mask
 * products (Rot_col is a ring automorphism: Rot_col(v.P) = Rot_col(v).
 * sigma_col(P)), so u_{2j} = v_j.[1;0] + Rot_col(v_j).sigma_col(DB_j.[1;0])
 * and u_{2j+1} = Rot_col(v_j).[1;0] + v_j.(DB_j.[0;1]): one key switch per
 * index ciphertext instead of two.  The output decrypts to the same slots as
 * pdq_comp(pdq_mask(...)); the ciphertexts differ (other key-switching
 * noise).  Workspace: pdq_answer_workspace_bytes (holds J rotated index
 * ciphertexts too). */
size_t pdq_answer_workspace_bytes(const pdq_ctx* ctx, const pdq_plan* plan);
int pdq_answer(const pdq_ctx* ctx, const pdq_plan* plan, const uint64_t* v_cts,
               const uint64_t* db, const uint64_t* keys, const uint64_t* galois,
               uint32_t nkeys, const uint64_t* consts, uint64_t* out, void* ws,
               size_t ws_bytes, void* stream);

/* The Answer of Q queries (1 <= Q <= 64) with the same plan, e.g. clients of
 * one database asking for the same number of records and matches, in one
 * launch sequence: every step of Mask and Comp (Alg. 7 with the SIMD form of
 * Sec. 5.2) runs as one launch over the index ciphertexts, half-blocks and
 * record groups of all Q queries, reading the database plaintexts and the
 * plan constants once for all of them; each query's rotations use its own
 * keys.  v_cts: dev [Q][J][2][L][N] (query q's index ciphertexts after
 * query q-1's); keys: HOST array of Q device pointers, keys[q] = query q's key
 * set laid out as for pdq_answer (the same galois list and order for every
 * query); db, galois, nkeys, consts as for pdq_answer; out: dev
 * [Q][n_out][2][L][N].  Each query's output is bit-identical to its
 * pdq_answer alone.  Workspace: pdq_answer_stacked_workspace_bytes (about Q
 * times pdq_answer's); too small -> PDQ_E_NOMEM; Q out of range or a NULL
 * pointer -> PDQ_E_PARAM; a missing key -> PDQ_E_KEY. */
size_t pdq_answer_stacked_workspace_bytes(const pdq_ctx* ctx, const pdq_plan* plan, uint32_t Q);
int pdq_answer_stacked(const pdq_ctx* ctx, const pdq_plan* plan, uint32_t Q,
                       const uint64_t* v_cts, const uint64_t* db,
                       const uint64_t* const* keys, const uint64_t* galois, uint32_t nkeys,
                       const uint64_t* consts, uint64_t* out, void* ws, size_t ws_bytes,
                       void* stream);

/* Answer (Alg. 7 without Match, as pdq_answer) with host buffers, end to
 * end: copies the query ciphertexts (host [J][2][L][N], coefficient form) to
 * the device, transforms them, runs Mask and Comp, transforms the answer
 * back and copies it to out_host ([n_out][2][L][N], coefficient form).  The
 * query goes up in at most four runs of index ciphertexts on a stream of the
 * call's own, ordered after the work already queued on `stream`; each run is
 * transformed and packed on `stream` while the next one is copied.
 * Synchronises `stream` (and its own copy stream) before returning, also on
 * errors after the copies started.  Host buffers should be pinned for the
 * copies to overlap.  Workspace: pdq_answer_host_workspace_bytes (device). */
size_t pdq_answer_host_workspace_bytes(const pdq_ctx* ctx, const pdq_plan* plan);
int pdq_answer_host(const pdq_ctx* ctx, const pdq_plan* plan, const uint64_t* v_host,
                    const uint64_t* db, const uint64_t* keys, const uint64_t* galois,
                    uint32_t nkeys, const uint64_t* consts, uint64_t* out_host, void* ws,
                    size_t ws_bytes, void* stream);

/* ---------------------------------------------------- unencrypted database
 * When the server holds the database in the clear, C (DB . v) =
 * (C diag(DB)) v, so it can skip Mask and compress the index vector alone
 * with the stacked matrix [C; C diag(DB)] (Sec. 5.2, remark on an
 * unencrypted database).  Index ciphertext j holds half-block 2j in row 0
 * and 2j+1 in row 1; two diagonal sets carry C on one row and C diag(DB) on
 * the other (set 0: C on row 0, C diag(DB) on row 1; set 1 the reverse), so
 * set 0 + Rot_col(set 1) holds (C v, C d) with d = DB . v, and Rot_col is
 * folded into the giant steps of set 1 (Galois element 3^(gB) (2N-1)).
 * pdq_plan_make_plain_db: the layout of pdq_plan_make, plain_db = 1; B = 0
 *   picks the power of two B <= min(s', 128) with at most 32 giant steps that
 *   minimises J (B-1) + 8 G (2 s'/B - 1) + 6 G s'/B, ties to the smaller B.
 *   pdq_plan_galois lists its Galois elements (Rot_col, 3^a, 3^(gB),
 *   3^(gB) (2N-1), the rotate-and-sum levels).
 * pdq_db_diagonals_build: the database-specific diagonals of both sets for
 *   every index ciphertext, over every prime of Q u P, then the group masks
 *   (dev out of pdq_db_diagonals_bytes; J 2 s' (L+K) N words plus the masks:
 *   at N = 2^15, n = 2^20, s' = 256, 43 GB).  values: dev [n] uint32 (< t,
 *   else reduced mod t), n = plan->n.  Allocates temporaries.
 * pdq_answer_plain_db: v_cts dev [J][2][L][N]; keys, galois, nkeys as for
 *   pdq_answer with the elements of this plan; consts from
 *   pdq_db_diagonals_build; out dev [n_out][2][L][N] decrypting to the same
 *   slots as pdq_answer's.  Workspace: pdq_answer_plain_db_workspace_bytes
 *   (dev), else PDQ_E_NOMEM; PDQ_E_PARAM for a plan without plain_db,
 *   PDQ_E_KEY for a missing key. */
int pdq_plan_make_plain_db(const pdq_ctx* ctx, uint64_t n, uint32_t s, uint32_t B,
                           pdq_plan* plan);
size_t pdq_db_diagonals_bytes(const pdq_ctx* ctx, const pdq_plan* plan);
int pdq_db_diagonals_build(const pdq_ctx* ctx, const pdq_plan* plan, const uint32_t* values,
                           uint64_t* out, void* stream);
size_t pdq_answer_plain_db_workspace_bytes(const pdq_ctx* ctx, const pdq_plan* plan);
int pdq_answer_plain_db(const pdq_ctx* ctx, const pdq_plan* plan, const uint64_t* v_cts,
                        const uint64_t* keys, const uint64_t* galois, uint32_t nkeys,
                        const uint64_t* consts, uint64_t* out, void* ws, size_t ws_bytes,
                        void* stream);

/* ------------------------------------------------------ batches, serving
 * One query of a batch or of the server: the buffers of pdq_answer.  plan
 * and galois are host pointers, the rest device pointers. */
typedef struct {
    const pdq_plan* plan;
    const uint64_t* v_cts;    /* dev [J][2][L][N] encrypted index vector */
    const uint64_t* db;       /* dev pdq_db_encode output (>= n records) */
    const uint64_t* keys;     /* dev keys, one per element of galois */
    const uint64_t* galois;   /* host [nkeys] */
    uint32_t nkeys;
    uint32_t reserved;
    const uint64_t* consts;   /* dev pdq_plan_constants_build output */
    uint64_t* out;            /* dev [n_out][2][L][N] answer */
} pdq_query;

/* Answer nq queries of one parameter set (Alg. 7 per query).  Query i runs
 * on lane i mod lanes, a stream owned by the context, with workspace
 * lane_ws[i mod lanes] (dev, lane_ws_bytes[...] >= pdq_answer_workspace_bytes
 * of every query of that lane); queries of one lane run in order, lanes run
 * concurrently.  The lanes fork from `stream` and join back into it (events
 * only), so the whole batch can be captured into a CUDA graph on `stream`.
 * Stage profiling is suspended during the call.  1 <= lanes <= 32. */
int pdq_answer_batch(const pdq_ctx* ctx, const pdq_query* queries, uint32_t nq,
                     void* const* lane_ws, const size_t* lane_ws_bytes, uint32_t lanes,
                     void* stream);

/* Continuous-batching server of Answer requests (each one Alg. 7 without
 * Match, as pdq_answer; the serving loop itself is not part of the paper's
 * method).  `arena` (dev, arena_bytes) is the device memory the server may
 * use for workspaces: a request is admitted when one of the `lanes` worker
 * threads is idle and the arena has room for its workspace (first fit), in
 * arrival order; it then runs on that worker's stream, concurrently with the
 * other admitted requests.  max_queue (0 = unbounded) caps the number of
 * waiting requests (PDQ_E_BUSY beyond).  A request whose workspace exceeds
 * the whole arena is refused with PDQ_E_NOMEM.  The caller keeps every
 * buffer of a request alive until it is done and must not enable stage
 * profiling while a server runs.  The workers' streams do not wait on any
 * stream of the caller: the arena and every buffer of a request must hold no
 * pending work from other streams when they are handed over.  Times are host
 * steady-clock nanoseconds. */
typedef struct pdq_server pdq_server;
#define PDQ_REQ_QUEUED 0
#define PDQ_REQ_RUNNING 1
#define PDQ_REQ_DONE 2
typedef struct {
    int32_t state;           /* PDQ_REQ_* */
    int32_t status;          /* result code once done */
    uint64_t t_submit_ns, t_start_ns, t_done_ns;
    uint32_t stacked;        /* requests answered in the same launches (1: alone) */
    uint32_t reserved;
} pdq_ticket_info;
int pdq_server_create(void* arena, size_t arena_bytes, uint32_t lanes, uint32_t max_queue,
                      pdq_server** out);
int pdq_server_submit(pdq_server* srv, const pdq_ctx* ctx, const pdq_query* q,
                      uint64_t* ticket);
int pdq_server_status(pdq_server* srv, uint64_t ticket, pdq_ticket_info* info);
/* Stacking (continuous batching of requests of one shape; each request is
 * still Alg. 7's Answer, and stacking is a launch schedule that is not part
 * of the paper's method): with max_stack >= 2, a worker that admits the
 * oldest request also takes up to max_stack - 1 queued requests of the same
 * context, database, plan constants, Galois list and plan shape (every plan
 * field but the record and match counts, which only the client's Decomp
 * reads), as many as the arena has room for, and answers them with one
 * pdq_answer_stacked call (their index ciphertexts gathered into the
 * workspace first, the outputs copied to each request's buffer after); each
 * result is the same bits as the request alone.  0 or 1 turns it off (the
 * default); at most 64.  Affects requests admitted after the call. */
int pdq_server_set_stacking(pdq_server* srv, uint32_t max_stack);
int pdq_server_wait(pdq_server* srv, uint64_t ticket, uint32_t timeout_ms);
int pdq_server_drain(pdq_server* srv, uint32_t timeout_ms);
int pdq_server_destroy(pdq_server* srv);

/* ---------------------------------------------------------------- Decomp
 * Client-side Decomp (Alg. 6) on decrypted answer slots (host [n_out][N]
 * uint32): per group, Newton's identity on w (Alg. 1 step 1), strip the
 * factors of X and find the roots among the nodes 1..G_sz (Alg. 1 step 2),
 * solve the Vandermonde system on the recovered columns (Alg. 4) and check
 * the remaining rows.  Writes up to cap (record index, value) pairs sorted by
 * index to idx_out / val_out (host) and the total to *count.  Errors:
 * PDQ_E_DECODE if a group's power sums are not those of at most s' nodes or
 * the values are inconsistent, PDQ_E_NOMEM if cap is too small.  Host only,
 * synchronous. */
int pdq_decomp(const pdq_ctx* ctx, const pdq_plan* plan, const uint32_t* slots,
               uint64_t* idx_out, uint32_t* val_out, uint64_t cap, uint64_t* count);
/* Decomp (Alg. 6) without a context: the client decrypts and decompresses
 * on its own machine, which needs no GPU.  t and log_n give the plaintext
 * prime and the answer's ring (for a ring-switched answer, the subring's);
 * the plan is checked against a fresh plan of its kind for that ring, as
 * pdq_decomp checks it against its context's.  Same results and errors as
 * pdq_decomp, and PDQ_E_PARAM for a ring or prime that pdq_ctx_create would
 * refuse.  Host only, synchronous. */
int pdq_decomp_client(uint64_t t, uint32_t log_n, const pdq_plan* plan, const uint32_t* slots,
                      uint64_t* idx_out, uint32_t* val_out, uint64_t cap, uint64_t* count);

/* ---------------------------------------------------------- serialise
 * Exchange format between client and server (Alg. 7 sends the query
 * ciphertexts to the server and the answer back; the paper fixes no format).
 * Little-endian bytes: a 64-byte header (u32 magic "PDQC" for ciphertexts or
 * "PDQS" for a secret key, u32 version 1, u32 N, u32 limbs per polynomial,
 * u32 level (= limbs), u32 count, u64 t, u64 first ciphertext prime, 24 zero
 * bytes), then for ciphertexts count x 2 x L x N uint64 in coefficient form
 * (canonical residues, [ct][poly][limb][coeff]) and for a secret key its N
 * int8 coefficients in {-1, 0, 1}.  All four calls synchronise `stream`.
 * pdq_cts_export: cts dev [count][2][L][N] (NTT form, unchanged); out_host
 *   of at least pdq_cts_serialized_bytes(count) bytes; ws dev, count*2*L*N
 *   words of scratch.  Too small output -> PDQ_E_NOMEM.
 * pdq_cts_import: in_host as written by pdq_cts_export; cts_out dev room for
 *   cap ciphertexts (NTT form on return); *count = the header's count.
 *   PDQ_E_PARAM for a wrong magic, version, N, L, t or first prime, a short
 *   buffer or a non-canonical residue; PDQ_E_NOMEM if count > cap.
 * pdq_sk_export: sk dev [L+K][N] from pdq_secret_prepare; ws dev, N words.
 *   PDQ_E_PARAM if the secret is not ternary.
 * pdq_sk_import: sk_out dev [L+K][N], the pdq_secret_prepare form. */
size_t pdq_cts_serialized_bytes(const pdq_ctx* ctx, uint32_t count);
int pdq_cts_export(const pdq_ctx* ctx, const uint64_t* cts, uint32_t count, void* out_host,
                   size_t out_bytes, uint64_t* ws, void* stream);
int pdq_cts_import(const pdq_ctx* ctx, const void* in_host, size_t in_bytes, uint64_t* cts_out,
                   uint32_t cap, uint32_t* count, void* stream);
size_t pdq_sk_serialized_bytes(const pdq_ctx* ctx);
int pdq_sk_export(const pdq_ctx* ctx, const uint64_t* sk, void* out_host, size_t out_bytes,
                  uint64_t* ws, void* stream);
int pdq_sk_import(const pdq_ctx* ctx, const void* in_host, size_t in_bytes, uint64_t* sk_out,
                  void* stream);

/* Rotation keys (the hybrid key-switching keys of the rotations of Sec. 5.1
 * that Comp's baby steps, giant steps and rotate-and-sum use, Sec. 5.2): the
 * client makes them once per key set and the server keeps them resident.
 * Header as above with magic "PDQK", limbs = L+K, level = L and the digit
 * count in the first 4 reserved bytes; then count uint64 Galois elements;
 * then count x ndigits x 2 x (L+K) x N uint64 in coefficient form,
 * [key][digit][poly][limb][coeff] (poly 0 = b, 1 = a of pdq_rotkey_gen).
 * Both calls synchronise `stream`.
 * pdq_rotkeys_export: keys dev [count][ndigits][2][L+K][N] (NTT form, as
 *   pdq_rotkey_gen writes them; unchanged), galois host [count]; out_host of
 *   at least pdq_rotkeys_serialized_bytes(count) bytes (else PDQ_E_NOMEM);
 *   ws dev, ndigits*2*(L+K)*N words of scratch.  PDQ_E_PARAM for an even or
 *   out-of-range Galois element.
 * pdq_rotkeys_import: in_host as written by pdq_rotkeys_export (or by any
 *   client holding the same prime chain); keys_out dev room for cap keys (NTT
 *   form on return, the layout pdq_answer takes), galois_out host [cap];
 *   *count = the header's count.  PDQ_E_PARAM for a wrong magic, version, N,
 *   L, K, digit count, t or first prime, a truncated buffer, an even,
 *   out-of-range or repeated Galois element or a non-canonical residue;
 *   PDQ_E_NOMEM if count > cap. */
size_t pdq_rotkeys_serialized_bytes(const pdq_ctx* ctx, uint32_t count);
int pdq_rotkeys_export(const pdq_ctx* ctx, const uint64_t* keys, const uint64_t* galois,
                       uint32_t count, void* out_host, size_t out_bytes, uint64_t* ws,
                       void* stream);
int pdq_rotkeys_import(const pdq_ctx* ctx, const void* in_host, size_t in_bytes,
                       uint64_t* keys_out, uint64_t* galois_out, uint32_t cap, uint32_t* count,
                       void* stream);

/* ------------------------------------------------- rotation without alloc
 * The paper has no counterpart to this call: it exists for callers that
 * cannot allocate device memory where they rotate (an external memory
 * manager owns every byte, a hard device-memory budget, or a serving loop
 * that must not risk an allocation synchronising the device).
 * Same result as pdq_rotate (bit for bit), but the key-switching scratch is
 * a fixed array of pdq_rotate_noalloc_max_bytes() bytes (32 MiB) that the
 * library reserves on every GPU that loads it, until the process exits; the
 * call itself allocates nothing.  The first call on a device looks up that
 * array's address (once per device), so make it before any stream capture;
 * the address stays cached for the life of the process, so do not call this
 * again on a device after cudaDeviceReset has ended its context.
 * Calls share the array: two calls that overlap on the GPU race.  Every
 * scratch byte is written before it is read, so nothing needs clearing.
 * Errors: PDQ_E_PARAM if `count` ciphertexts need more scratch than the
 * array holds (pdq_rotate_workspace_bytes(count) > the maximum), PDQ_E_CUDA
 * if the address look-up fails. */
size_t pdq_rotate_noalloc_max_bytes(void);
int pdq_rotate_noalloc(const pdq_ctx* ctx, const uint64_t* ct_in, uint32_t count,
                       uint64_t galois, const uint64_t* key, uint64_t* ct_out, void* stream);

/* -------------------------------------------------------- instrumentation
 * Not part of the paper's method: counters for measuring the library.
 * pdq_launch_count: kernels this library has launched in this process.
 * pdq_profile_enable: when on, pdq_answer / pdq_comp record a CUDA event on
 * their stream at every stage boundary (stages PDQ_STAGE_*); enabling resets
 * the record.  pdq_profile_read waits for the recorded events, writes per
 * stage the summed milliseconds (ms[nstages]) and call counts (calls, may be
 * NULL), and clears the record. */
#define PDQ_STAGE_MASK 0
#define PDQ_STAGE_PACK 1
#define PDQ_STAGE_BABY 2
#define PDQ_STAGE_MAC 3           /* the diagonal multiply-accumulate kernel alone */
#define PDQ_STAGE_GIANT 4
#define PDQ_STAGE_ROTSUM 5
#define PDQ_STAGE_COMBINE 6
#define PDQ_STAGE_ACC_MODDOWN 7   /* ModDown of the multiply-accumulate outputs */
#define PDQ_NSTAGES 8
unsigned long long pdq_launch_count(void);
int pdq_profile_enable(pdq_ctx* ctx, int enable);
int pdq_profile_read(pdq_ctx* ctx, float* ms, uint32_t* calls, uint32_t nstages);

#ifdef __cplusplus
}
#endif

#endif /* PDQ_H */
