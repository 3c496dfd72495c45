// Register-only throughput ceilings of the two arithmetic primitives of the
// library on the current GPU, used as the ALU roofline denominators:
//   * a modular multiply-accumulate of 60-bit residues in the form the
//     diagonal multiply-accumulate uses (30-bit halves, Karatsuba: three
//     32x32->64-bit products, each a mad.lo.cc / madc.hi.cc / addc chain into
//     a 96-bit sum), in the schoolbook form (four mad.wide.u32 into 64-bit
//     partial sums), and in the 128-bit carry-chain form the key-switching
//     inner products use;
//   * the forward NTT butterfly (Harvey's lazy Cooley-Tukey butterfly with a
//     Shoup twiddle multiplication);
//   * plain 32x32->32-bit multiply-adds (mad.lo.u32) and 32x32->64-bit
//     multiply-adds (mad.wide.u32), for the per-SM issue rates of the
//     integer multiply pipe.
// No memory traffic inside the timed loops; CUDA events around each kernel.
#include <cstdint>
#include <cstdio>

typedef uint64_t u64;
typedef uint32_t u32;

__device__ __forceinline__ void mac128(u64& hi, u64& lo, u64 a, u64 b) {
    asm("mad.lo.cc.u64 %0, %2, %3, %0;\n\tmadc.hi.u64 %1, %2, %3, %1;"
        : "+l"(lo), "+l"(hi) : "l"(a), "l"(b));
}
__device__ __forceinline__ void mac30(u64* s, u32 a0, u32 a1, u32 b0, u32 b1) {
    asm("mad.wide.u32 %0, %4, %6, %0;\n\tmad.wide.u32 %1, %4, %7, %1;\n\t"
        "mad.wide.u32 %2, %5, %6, %2;\n\tmad.wide.u32 %3, %5, %7, %3;"
        : "+l"(s[0]), "+l"(s[1]), "+l"(s[2]), "+l"(s[3]) : "r"(a0), "r"(a1), "r"(b0), "r"(b1));
}
// one Karatsuba product step: three 96-bit sums s[0..2], s[3..5], s[6..8]
__device__ __forceinline__ void mack(u32* s, u32 a0, u32 a1, u32 as, u32 b0, u32 b1, u32 bs) {
    asm("mad.lo.cc.u32 %0, %9, %12, %0;\n\tmadc.hi.cc.u32 %1, %9, %12, %1;\n\taddc.u32 %2, %2, 0;\n\t"
        "mad.lo.cc.u32 %3, %11, %14, %3;\n\tmadc.hi.cc.u32 %4, %11, %14, %4;\n\taddc.u32 %5, %5, 0;\n\t"
        "mad.lo.cc.u32 %6, %10, %13, %6;\n\tmadc.hi.cc.u32 %7, %10, %13, %7;\n\taddc.u32 %8, %8, 0;"
        : "+r"(s[0]), "+r"(s[1]), "+r"(s[2]), "+r"(s[3]), "+r"(s[4]), "+r"(s[5]), "+r"(s[6]),
          "+r"(s[7]), "+r"(s[8])
        : "r"(a0), "r"(a1), "r"(as), "r"(b0), "r"(b1), "r"(bs));
}
__device__ __forceinline__ u64 csub(u64 x, u64 q) { return x >= q ? x - q : x; }
__device__ __forceinline__ void bf(u64& x, u64& y, u64 w, u64 wp, u64 q) {
    const u64 a = csub(x, 2 * q);
    const u64 t = y * w - __umul64hi(y, wp) * q;
    x = a + t;
    y = a - t + 2 * q;
}

// V = 0: mac128, 1: mac30 (four 64-bit partial sums), 2: mad.lo.u32 stream,
// 3: Karatsuba (three 96-bit sums; the operand half-sums are formed once per
// operand, as in the kernel, where each is shared by several products)
template <int V>
__global__ void k_mac(const u64* in, u64* out, int iters) {
    u64 a = in[threadIdx.x & 31], b = in[(threadIdx.x + 7) & 31];
    u64 acc[8][4] = {};
    u32 k[8][9] = {};
    for (int it = 0; it < iters; ++it) {
        const u32 a0 = (u32)a & 0x3fffffffu, a1 = (u32)(a >> 30) & 0x3fffffffu, as = a0 + a1;
#pragma unroll
        for (int g = 0; g < 8; ++g) {
            const u64 bb = b + g;
            if (V == 3) {
                const u32 b0 = (u32)bb & 0x3fffffffu, b1 = (u32)(bb >> 30) & 0x3fffffffu;
                mack(k[g], a0, a1, as, b0, b1, b0 + b1);
            } else if (V == 0) mac128(acc[g][0], acc[g][1], a, bb);
            else if (V == 1) mac30(acc[g], (u32)a & 0x3fffffffu, (u32)(a >> 30), (u32)bb & 0x3fffffffu,
                                   (u32)(bb >> 30));
            else {
                u32 x = (u32)acc[g][0];
                const u32 a0 = (u32)a, a1 = (u32)(a >> 32), b0 = (u32)bb, b1 = (u32)(bb >> 32);
                asm("mad.lo.u32 %0, %1, %2, %0;\n\tmad.lo.u32 %0, %3, %4, %0;\n\t"
                    "mad.lo.u32 %0, %1, %4, %0;\n\tmad.lo.u32 %0, %3, %2, %0;"
                    : "+r"(x) : "r"(a0), "r"(b0), "r"(a1), "r"(b1));
                acc[g][0] = x;
            }
        }
        a += 3;
    }
    u64 r = 0;
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 4; ++j) r ^= acc[i][j];
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 9; ++j) r ^= k[i][j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

__global__ void k_bf(const u64* in, u64* out, int iters, u64 q) {
    u64 x[8];
    for (int i = 0; i < 8; ++i) x[i] = in[(threadIdx.x + i) & 31];
    u64 w = in[5], wp = in[6];
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 4; ++i) bf(x[i], x[i + 4], w, wp, q);
#pragma unroll
        for (int i = 0; i < 8; i += 4) {
            bf(x[i], x[i + 2], w, wp, q);
            bf(x[i + 1], x[i + 3], w, wp, q);
        }
#pragma unroll
        for (int i = 0; i < 8; i += 2) bf(x[i], x[i + 1], w, wp, q);
        w += 1;
    }
    u64 r = 0;
    for (int i = 0; i < 8; ++i) r ^= x[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

int main() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * 8, threads = 256, iters = 4096;
    u64 *in, *out;
    cudaMalloc(&in, 32 * sizeof(u64));
    cudaMalloc(&out, (size_t)blocks * threads * sizeof(u64));
    const u64 q = 0x0fffffffffc0001ull;
    u64 h[32];
    for (int i = 0; i < 32; ++i) h[i] = (q - 977ull * i) % q;
    h[6] = (u64)(((unsigned __int128)h[5] << 64) / q);
    cudaMemcpy(in, h, sizeof(h), cudaMemcpyHostToDevice);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const double work = (double)blocks * threads * iters;
    float ms = 0;
    for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(e0);
        k_mac<1><<<blocks, threads>>>(in, out, iters);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
    }
    cudaEventElapsedTime(&ms, e0, e1);
    printf("{\"mac30_per_s\": %.4e, \"imad_wide_per_s\": %.4e, ", work * 8 / (ms * 1e-3),
           work * 8 * 4 / (ms * 1e-3));
    for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(e0);
        k_mac<0><<<blocks, threads>>>(in, out, iters);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
    }
    cudaEventElapsedTime(&ms, e0, e1);
    printf("\"mac128_per_s\": %.4e, ", work * 8 / (ms * 1e-3));
    for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(e0);
        k_mac<2><<<blocks, threads>>>(in, out, iters);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
    }
    cudaEventElapsedTime(&ms, e0, e1);
    printf("\"imad32_per_s\": %.4e, ", work * 8 * 4 / (ms * 1e-3));
    for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(e0);
        k_mac<3><<<blocks, threads>>>(in, out, iters);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
    }
    cudaEventElapsedTime(&ms, e0, e1);
    printf("\"mac_karatsuba_per_s\": %.4e, ", work * 8 / (ms * 1e-3));
    for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(e0);
        k_bf<<<blocks, threads>>>(in, out, iters, q);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
    }
    cudaEventElapsedTime(&ms, e0, e1);
    printf("\"butterfly_per_s\": %.4e, \"sms\": %d, \"status\": \"%s\"}\n", work * 12 / (ms * 1e-3),
           sms, cudaGetErrorString(cudaGetLastError()));
    return 0;
}
