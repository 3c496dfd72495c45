// Exchange format for ciphertexts, secret keys and rotation keys (host bytes
// <-> device NTT-form buffers).  Not an operation of the paper: the query and
// the answer of Alg. 7 travel between client and server, and the client's
// key-switching keys for the rotations of Sec. 5.1 reach the server once per
// key set; the format fixes how.
//
//   header (64 bytes, little-endian): u32 magic ("PDQC" ciphertexts, "PDQS"
//   secret key, "PDQK" rotation keys), u32 version (1), u32 N, u32 limbs per
//   polynomial, u32 level (the ciphertext primes L), u32 count, u64 t, u64
//   first ciphertext prime, 24 reserved bytes (zero, except that rotation
//   keys keep their digit count in the first 4);
//   ciphertexts: count x 2 x limbs x N uint64, coefficient form, canonical
//   residues, [ct][poly][limb][coeff];
//   secret key: N int8 coefficients in {-1, 0, 1};
//   rotation keys (limbs = L + K): count uint64 Galois elements, then
//   count x digits x 2 x (L+K) x N uint64 in coefficient form,
//   [key][digit][poly][limb][coeff], poly 0 = b, poly 1 = a.
#include <cstring>
#include <vector>

#include "pdq_internal.h"
#include "pdq_ops.h"

namespace pdq {
namespace {

constexpr u32 kMagicCts = 0x43514450u;   // "PDQC"
constexpr u32 kMagicSk = 0x53514450u;    // "PDQS"
constexpr u32 kMagicKeys = 0x4b514450u;  // "PDQK"
constexpr u32 kVersion = 1;
constexpr size_t kHeader = 64;

struct Header {
    u32 magic, version, N, limbs, level, count;
    u64 t, q0;
    uint8_t zero[24];
};
static_assert(sizeof(Header) == kHeader, "header layout");

Header make_header(const Ctx& c, u32 magic, u32 count) {
    Header h;
    std::memset(&h, 0, sizeof(h));
    h.magic = magic;
    h.version = kVersion;
    h.N = c.N;
    h.limbs = c.L;
    h.level = c.L;
    h.count = count;
    h.t = c.t;
    h.q0 = c.mods[0];
    return h;
}

int check_header(const Ctx& c, const void* in, size_t in_bytes, u32 magic, Header* h) {
    if (!in || in_bytes < kHeader) return fail(PDQ_E_PARAM, "import: buffer shorter than the header");
    std::memcpy(h, in, kHeader);
    if (h->magic != magic) return fail(PDQ_E_PARAM, "import: wrong magic");
    if (h->version != kVersion) return fail(PDQ_E_PARAM, "import: unsupported version");
    const u32 limbs = magic == kMagicKeys ? c.L + c.K : c.L;
    if (h->N != c.N || h->limbs != limbs || h->level != c.L || h->t != c.t || h->q0 != c.mods[0])
        return fail(PDQ_E_PARAM, "import: parameters differ from the context");
    if (magic == kMagicKeys) {
        u32 nd;
        std::memcpy(&nd, h->zero, sizeof(nd));
        if (nd != c.ndigits) return fail(PDQ_E_PARAM, "import: digit count differs from the context");
    }
    return PDQ_OK;
}

u64 key_words(const Ctx& c) { return (u64)c.ndigits * 2 * (c.L + c.K) * c.N; }

}  // namespace
}  // namespace pdq

using namespace pdq;

extern "C" {

size_t pdq_cts_serialized_bytes(const pdq_ctx* ctx, uint32_t count) {
    if (!ctx) return 0;
    const Ctx& c = *reinterpret_cast<const Ctx*>(ctx);
    return kHeader + (size_t)count * 2 * c.L * c.N * sizeof(u64);
}

int pdq_cts_export(const pdq_ctx* ctx, const uint64_t* cts, uint32_t count, void* out_host,
                   size_t out_bytes, uint64_t* ws, void* stream) {
    if (!ctx || !out_host) return fail(PDQ_E_PARAM, "cts_export: null argument");
    const Ctx& c = *reinterpret_cast<const Ctx*>(ctx);
    if (out_bytes < pdq_cts_serialized_bytes(ctx, count)) return fail(PDQ_E_NOMEM, "cts_export: output too small");
    const Header h = make_header(c, kMagicCts, count);
    std::memcpy(out_host, &h, kHeader);
    if (count == 0) return PDQ_OK;
    if (!cts || !ws) return fail(PDQ_E_PARAM, "cts_export: null device buffer");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)count * 2 * c.L * c.N * sizeof(u64);
    if (cudaMemcpyAsync(ws, cts, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return fail(PDQ_E_CUDA, "cts_export: copy failed");
    PDQ_TRY(ntt_inverse(c, ws, 2 * count, c.L, 0, (u64)c.L * c.N, st));
    if (cudaMemcpyAsync(static_cast<char*>(out_host) + kHeader, ws, bytes, cudaMemcpyDeviceToHost,
                        st) != cudaSuccess)
        return fail(PDQ_E_CUDA, "cts_export: download failed");
    if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_check("cts_export");
    return PDQ_OK;
}

int pdq_cts_import(const pdq_ctx* ctx, const void* in_host, size_t in_bytes, uint64_t* cts_out,
                   uint32_t cap, uint32_t* count, void* stream) {
    if (!ctx || !count) return fail(PDQ_E_PARAM, "cts_import: null argument");
    const Ctx& c = *reinterpret_cast<const Ctx*>(ctx);
    Header h;
    PDQ_TRY(check_header(c, in_host, in_bytes, kMagicCts, &h));
    if (in_bytes < pdq_cts_serialized_bytes(ctx, h.count)) return fail(PDQ_E_PARAM, "cts_import: truncated payload");
    *count = h.count;
    if (h.count > cap) return fail(PDQ_E_NOMEM, "cts_import: output holds fewer ciphertexts");
    if (h.count == 0) return PDQ_OK;
    if (!cts_out) return fail(PDQ_E_PARAM, "cts_import: null device buffer");
    // every residue must be canonical
    const u64* p = reinterpret_cast<const u64*>(static_cast<const char*>(in_host) + kHeader);
    const u64 LN = (u64)c.L * c.N;
    for (u64 i = 0; i < (u64)h.count * 2 * LN; ++i)
        if (p[i] >= c.mods[(i % LN) / c.N]) return fail(PDQ_E_PARAM, "cts_import: residue out of range");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)h.count * 2 * LN * sizeof(u64);
    if (cudaMemcpyAsync(cts_out, p, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return fail(PDQ_E_CUDA, "cts_import: upload failed");
    PDQ_TRY(ntt_forward(c, cts_out, 2 * h.count, c.L, 0, LN, st));
    if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_check("cts_import");
    return PDQ_OK;
}

size_t pdq_sk_serialized_bytes(const pdq_ctx* ctx) {
    if (!ctx) return 0;
    return kHeader + reinterpret_cast<const Ctx*>(ctx)->N;
}

int pdq_sk_export(const pdq_ctx* ctx, const uint64_t* sk, void* out_host, size_t out_bytes,
                  uint64_t* ws, void* stream) {
    if (!ctx || !sk || !out_host || !ws) return fail(PDQ_E_PARAM, "sk_export: null argument");
    const Ctx& c = *reinterpret_cast<const Ctx*>(ctx);
    if (out_bytes < pdq_sk_serialized_bytes(ctx)) return fail(PDQ_E_NOMEM, "sk_export: output too small");
    cudaStream_t st = (cudaStream_t)stream;
    // limb 0 in coefficient form determines the ternary coefficients
    if (cudaMemcpyAsync(ws, sk, (size_t)c.N * sizeof(u64), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return fail(PDQ_E_CUDA, "sk_export: copy failed");
    PDQ_TRY(ntt_inverse(c, ws, 1, 1, 0, c.N, st));
    std::vector<u64> coeff(c.N);
    if (cudaMemcpyAsync(coeff.data(), ws, (size_t)c.N * sizeof(u64), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return fail(PDQ_E_CUDA, "sk_export: download failed");
    if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_check("sk_export");
    const u64 q = c.mods[0];
    int8_t* s = reinterpret_cast<int8_t*>(static_cast<char*>(out_host) + kHeader);
    for (u32 i = 0; i < c.N; ++i) {
        if (coeff[i] == 0) s[i] = 0;
        else if (coeff[i] == 1) s[i] = 1;
        else if (coeff[i] == q - 1) s[i] = -1;
        else return fail(PDQ_E_PARAM, "sk_export: secret is not ternary");
    }
    const Header h = make_header(c, kMagicSk, 1);
    std::memcpy(out_host, &h, kHeader);
    return PDQ_OK;
}

int pdq_sk_import(const pdq_ctx* ctx, const void* in_host, size_t in_bytes, uint64_t* sk_out,
                  void* stream) {
    if (!ctx || !sk_out) return fail(PDQ_E_PARAM, "sk_import: null argument");
    const Ctx& c = *reinterpret_cast<const Ctx*>(ctx);
    Header h;
    PDQ_TRY(check_header(c, in_host, in_bytes, kMagicSk, &h));
    if (in_bytes < pdq_sk_serialized_bytes(ctx)) return fail(PDQ_E_PARAM, "sk_import: truncated payload");
    const int8_t* s = reinterpret_cast<const int8_t*>(static_cast<const char*>(in_host) + kHeader);
    const u32 E = c.L + c.K;
    std::vector<u64> res((size_t)E * c.N);
    for (u32 i = 0; i < c.N; ++i) {
        if (s[i] < -1 || s[i] > 1) return fail(PDQ_E_PARAM, "sk_import: secret is not ternary");
        for (u32 l = 0; l < E; ++l)
            res[(size_t)l * c.N + i] = s[i] < 0 ? c.mods[l] - 1 : (u64)s[i];
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(sk_out, res.data(), res.size() * sizeof(u64), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return fail(PDQ_E_CUDA, "sk_import: upload failed");
    PDQ_TRY(ntt_forward(c, sk_out, 1, E, 0, (u64)E * c.N, st));
    if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_check("sk_import");
    return PDQ_OK;
}

size_t pdq_rotkeys_serialized_bytes(const pdq_ctx* ctx, uint32_t count) {
    if (!ctx) return 0;
    const Ctx& c = *reinterpret_cast<const Ctx*>(ctx);
    return kHeader + (size_t)count * sizeof(u64) + (size_t)count * key_words(c) * sizeof(u64);
}

int pdq_rotkeys_export(const pdq_ctx* ctx, const uint64_t* keys, const uint64_t* galois,
                       uint32_t count, void* out_host, size_t out_bytes, uint64_t* ws,
                       void* stream) {
    if (!ctx || !out_host) return fail(PDQ_E_PARAM, "rotkeys_export: null argument");
    const Ctx& c = *reinterpret_cast<const Ctx*>(ctx);
    if (out_bytes < pdq_rotkeys_serialized_bytes(ctx, count))
        return fail(PDQ_E_NOMEM, "rotkeys_export: output too small");
    if (count && (!keys || !galois || !ws)) return fail(PDQ_E_PARAM, "rotkeys_export: null buffer");
    for (u32 i = 0; i < count; ++i)
        if (galois[i] % 2 == 0 || galois[i] >= 2ull * c.N)
            return fail(PDQ_E_PARAM, "rotkeys_export: bad Galois element");
    Header h = make_header(c, kMagicKeys, count);
    h.limbs = c.L + c.K;
    std::memcpy(h.zero, &c.ndigits, sizeof(c.ndigits));
    char* out = static_cast<char*>(out_host);
    std::memcpy(out, &h, kHeader);
    std::memcpy(out + kHeader, galois, (size_t)count * sizeof(u64));
    char* payload = out + kHeader + (size_t)count * sizeof(u64);
    cudaStream_t st = (cudaStream_t)stream;
    const u64 kw = key_words(c), EN = (u64)(c.L + c.K) * c.N;
    // one key at a time through the caller's scratch (key_words words)
    for (u32 i = 0; i < count; ++i) {
        if (cudaMemcpyAsync(ws, keys + (u64)i * kw, kw * sizeof(u64), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return fail(PDQ_E_CUDA, "rotkeys_export: copy failed");
        PDQ_TRY(ntt_inverse(c, ws, 2 * c.ndigits, c.L + c.K, 0, EN, st));
        if (cudaMemcpyAsync(payload + (size_t)i * kw * sizeof(u64), ws, kw * sizeof(u64),
                            cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return fail(PDQ_E_CUDA, "rotkeys_export: download failed");
        if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_check("rotkeys_export");
    }
    return PDQ_OK;
}

int pdq_rotkeys_import(const pdq_ctx* ctx, const void* in_host, size_t in_bytes,
                       uint64_t* keys_out, uint64_t* galois_out, uint32_t cap, uint32_t* count,
                       void* stream) {
    if (!ctx || !count) return fail(PDQ_E_PARAM, "rotkeys_import: null argument");
    const Ctx& c = *reinterpret_cast<const Ctx*>(ctx);
    Header h;
    PDQ_TRY(check_header(c, in_host, in_bytes, kMagicKeys, &h));
    if (in_bytes < pdq_rotkeys_serialized_bytes(ctx, h.count))
        return fail(PDQ_E_PARAM, "rotkeys_import: truncated payload");
    *count = h.count;
    if (h.count > cap) return fail(PDQ_E_NOMEM, "rotkeys_import: output holds fewer keys");
    if (h.count == 0) return PDQ_OK;
    if (!keys_out || !galois_out) return fail(PDQ_E_PARAM, "rotkeys_import: null output buffer");
    const char* in = static_cast<const char*>(in_host);
    std::vector<u64> gal(h.count);
    std::memcpy(gal.data(), in + kHeader, (size_t)h.count * sizeof(u64));
    for (u32 i = 0; i < h.count; ++i) {
        if (gal[i] % 2 == 0 || gal[i] >= 2ull * c.N)
            return fail(PDQ_E_PARAM, "rotkeys_import: bad Galois element");
        for (u32 j = 0; j < i; ++j)
            if (gal[j] == gal[i]) return fail(PDQ_E_PARAM, "rotkeys_import: Galois element repeated");
    }
    const u64* p = reinterpret_cast<const u64*>(in + kHeader + (size_t)h.count * sizeof(u64));
    const u32 E = c.L + c.K;
    const u64 kw = key_words(c), total = (u64)h.count * kw;
    for (u64 i = 0; i < total; ++i)
        if (p[i] >= c.mods[(i / c.N) % E]) return fail(PDQ_E_PARAM, "rotkeys_import: residue out of range");
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(keys_out, p, total * sizeof(u64), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return fail(PDQ_E_CUDA, "rotkeys_import: upload failed");
    PDQ_TRY(ntt_forward(c, keys_out, h.count * 2 * c.ndigits, E, 0, (u64)E * c.N, st));
    if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_check("rotkeys_import");
    std::memcpy(galois_out, gal.data(), (size_t)h.count * sizeof(u64));
    return PDQ_OK;
}

}  // extern "C"
