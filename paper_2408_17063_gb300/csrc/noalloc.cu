// Homomorphic rotation that allocates nothing: the key-switching scratch
// lives in a fixed device array of this file instead of a caller workspace.
//
// Who needs it: callers that cannot call cudaMalloc / cudaFree or ask a
// framework allocator for memory at the point where they rotate, e.g. code
// running under an external memory manager that owns every byte of device
// memory, a process held to a hard device-memory budget, or a latency-
// critical serving loop where an allocation may synchronise the device.
//
// The array below is reserved on every GPU that loads this library and
// stays reserved until the process exits.  Its device address is looked up
// once per device (cudaGetSymbolAddress, with that device current) on the
// first call made on that device, so that first call should come before any
// stream capture.  The cached address belongs to the device's context at
// the time of the look-up: after cudaDeviceReset (which ends that context)
// it is stale, so a process that resets a device must not call this entry
// point on it again.  All calls share the array: the scratch keeps whatever the
// previous call left, which is fine because every byte the rotation reads is
// first written by the same call; but two calls that overlap on the GPU (on
// different streams, or from different threads) race on it.
#include <mutex>

#include "pdq_internal.h"
#include "pdq_ops.h"

#define PDQ_STATIC_SCRATCH_BYTES (32ull << 20)   /* 32 MiB per GPU */

static __device__ __align__(256) unsigned char g_rotate_scratch[PDQ_STATIC_SCRATCH_BYTES];

namespace pdq {
namespace {

constexpr size_t kStaticScratchBytes = PDQ_STATIC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_rotate_scratch on the current device (set-up once).
int scratch_address(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(PDQ_E_CUDA, "rotate_noalloc: no usable current device");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_rotate_scratch);
        if (e != cudaSuccess || !p)
            return fail(PDQ_E_CUDA, std::string("rotate_noalloc: cudaGetSymbolAddress failed: ") +
                                        cudaGetErrorString(e));
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return PDQ_OK;
}

}  // namespace
}  // namespace pdq

using namespace pdq;

extern "C" size_t pdq_rotate_noalloc_max_bytes(void) { return kStaticScratchBytes; }

extern "C" int pdq_rotate_noalloc(const pdq_ctx* ctx, const uint64_t* ct_in, uint32_t count,
                                  uint64_t galois, const uint64_t* key, uint64_t* ct_out,
                                  void* stream) {
    if (!ctx) return fail(PDQ_E_PARAM, "null context");
    const Ctx& c = *reinterpret_cast<const Ctx*>(ctx);
    if (count == 0) return PDQ_OK;
    if (!ct_in || !key || !ct_out) return fail(PDQ_E_PARAM, "rotate_noalloc: null buffer");
    if (galois % 2 == 0 || galois >= 2ull * c.N)
        return fail(PDQ_E_PARAM, "rotate_noalloc: bad Galois element");
    const size_t need = raise_ws(c, count) + apply_ws(c, count);
    if (need > kStaticScratchBytes)
        return fail(PDQ_E_PARAM, "rotate_noalloc: " + std::to_string(count) +
                                     " ciphertexts need " + std::to_string(need) +
                                     " bytes of scratch, more than the fixed " +
                                     std::to_string(kStaticScratchBytes) + " bytes");
    void* base = nullptr;
    PDQ_TRY(scratch_address(&base));
    cudaStream_t st = (cudaStream_t)stream;
    const long long cts = (long long)ct_elems(c);
    u64* rws = reinterpret_cast<u64*>(base);
    u64* aws = rws + raise_ws(c, count) / sizeof(u64);
    u64* D = nullptr;
    const CtSet in = ct_set(ct_in, cts);
    PDQ_TRY(ks_raise(c, in, count, rws, &D, st));
    return ks_apply(c, D, in, count, (u32)galois, key, ct_set(ct_out, cts), CtSet{}, aws, st);
}
