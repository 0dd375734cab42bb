// ff_peaks.cuh - microbenchmarks of the ceilings the matching kernels are
// measured against on the running GPU: integer and dp4a throughput, the
// throughput of the matching error's own per-dimension arithmetic, L2 read
// bandwidth, and the dependent latencies of the instructions on a wavefront
// step's critical path.  Every loop runs a fixed number of iterations; no
// kernel waits on another.
#pragma once
#include "ff_kernels.cuh"

namespace ffk {

constexpr int kPeakThreads = 256;
constexpr int kPeakChains = 8;

// Throughput of one integer instruction kind: kPeakChains independent
// dependency chains per thread, full occupancy.  OP 0: dp4a (4 multiply-adds
// of bytes into an int32), 1: three-input add, 2: 32-bit multiply-add.
template <int OP>
__global__ void __launch_bounds__(kPeakThreads) k_peak_int(uint32_t *out, int iters, uint32_t s) {
    uint32_t a[kPeakChains];
#pragma unroll
    for (int j = 0; j < kPeakChains; j++) a[j] = s * (threadIdx.x + 1) + 0x9E3779B9u * (j + 1);
    const uint32_t b = s ^ 0x01020304u, c = s ^ 0x7F3A1B2Cu;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int j = 0; j < kPeakChains; j++) {
            if constexpr (OP == 0) a[j] = (uint32_t)__dp4a((int)a[j], (int)(b + j), (int)a[j]);
            else if constexpr (OP == 1) a[j] = a[j] + a[(j + 4) % kPeakChains] + c;
            else a[j] = a[j] * b + a[(j + 4) % kPeakChains];
        }
    }
    uint32_t r = 0;
#pragma unroll
    for (int j = 0; j < kPeakChains; j++) r ^= a[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

// Throughput of the matching error's arithmetic per feature dimension, from
// registers: the byte transpose of four taps, one dp4a per dimension (the
// bilinear interpolation minus 64 q), absolute value and accumulation --
// sad_word, as the sweep computes it.  kPeakChains words (4 dimensions
// each) per iteration; the taps change every iteration.
__global__ void __launch_bounds__(kPeakThreads) k_peak_sad(uint32_t *out, int iters, uint32_t s) {
    uint32_t t0 = s * (threadIdx.x + 1), t1 = t0 ^ 0x5A5A5A5Au, t2 = t0 + 0x01234567u,
             t3 = t0 * 3u;
    const uint32_t w = 0x10203040u ^ (s & 0x0F0F0F0Fu);
    const int4 na = make_int4(-64, 128, -192, 256);
    int acc[kPeakChains];
#pragma unroll
    for (int j = 0; j < kPeakChains; j++) acc[j] = j;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int j = 0; j < kPeakChains; j++)
            acc[j] += sad_word(t0 + j, t1 ^ j, t2 + 2 * j, t3 ^ (3 * j), w, na);
        t0 += 0x01010101u;
        t1 ^= t0;
        t2 += t1;
        t3 ^= t2;
    }
    int r = 0;
#pragma unroll
    for (int j = 0; j < kPeakChains; j++) r ^= acc[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = (uint32_t)r;
}

// L2 read bandwidth: `passes` grid-stride passes of 16-byte loads that skip
// L1 (ld.global.cg) over a buffer small enough to stay in L2.
__global__ void __launch_bounds__(kPeakThreads) k_peak_l2(const uint4 *buf, size_t n16, int passes,
                                                          uint32_t *out) {
    uint32_t x = 0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (int p = 0; p < passes; p++)
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) {
            const uint4 v = __ldcg(buf + i);
            x ^= v.x ^ v.y ^ v.z ^ v.w;
        }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x;
}

// Dependent latencies, one warp: each measured chain is `iters` instructions
// long, each instruction consuming the previous one's result.
// out[k] = clock cycles per instruction of chain k:
//   0 integer add / xor, 1 byte permute, 2 dp4a, 3 warp shuffle, 4 shared load,
//   5 global load hitting L1, 6 global load hitting L2 (L1 skipped),
//   7 clock read itself (subtracted from none; for reference)
__global__ void k_peak_latency(const uint32_t *chase_l1, const uint32_t *chase_l2, int iters,
                               uint32_t s, double *out) {
    __shared__ uint32_t sh[1024];
    for (int j = threadIdx.x; j < 1024; j += 32) sh[j] = (uint32_t)((j * 97 + 31) & 1023);
    __syncwarp();
    uint32_t a = s + threadIdx.x, b = s ^ 0x1234u, c = 0x9E37u ^ s;
    long long t0, t1;
    double r[8];
    // 0: integer add and xor alternating (inline PTX: no two of them can be
    // fused into one instruction, and the chain cannot be folded)
    t0 = clock64();
#pragma unroll 16
    for (int i = 0; i < iters; i++)
        asm volatile("add.u32 %0, %0, %1;\n\txor.b32 %0, %0, %2;" : "+r"(a) : "r"(b), "r"(c));
    t1 = clock64();
    r[0] = (double)(t1 - t0) / (2.0 * iters);
    // 1: byte permute
    t0 = clock64();
#pragma unroll 16
    for (int i = 0; i < iters; i++) asm volatile("prmt.b32 %0, %0, %1, 0x5140;" : "+r"(a) : "r"(b));
    t1 = clock64();
    r[1] = (double)(t1 - t0) / iters;
    // 2: dp4a
    t0 = clock64();
#pragma unroll 16
    for (int i = 0; i < iters; i++) asm volatile("dp4a.s32.s32 %0, %0, %1, %0;" : "+r"(a) : "r"(b));
    t1 = clock64();
    r[2] = (double)(t1 - t0) / iters;
    // 3: SHFL
    t0 = clock64();
    for (int i = 0; i < iters; i++) a = __shfl_xor_sync(0xffffffffu, a, 1);
    t1 = clock64();
    r[3] = (double)(t1 - t0) / iters;
    // 4: LDS (pointer chase)
    uint32_t p = a & 1023;
    t0 = clock64();
    for (int i = 0; i < iters; i++) p = *(volatile uint32_t *)&sh[p];
    t1 = clock64();
    r[4] = (double)(t1 - t0) / iters;
    // 5: LDG, L1 hit (a 4 KB chase, warmed first)
    uint32_t q = 0;
    for (int i = 0; i < 1024; i++) q = __ldca(chase_l1 + q);
    t0 = clock64();
    for (int i = 0; i < iters; i++) q = __ldca(chase_l1 + q);
    t1 = clock64();
    r[5] = (double)(t1 - t0) / iters;
    // 6: LDG, L2 hit (a chase through a buffer warmed into L2, L1 skipped)
    uint32_t z = 0;
    t0 = clock64();
    for (int i = 0; i < iters; i++) z = __ldcg(chase_l2 + z);
    t1 = clock64();
    r[6] = (double)(t1 - t0) / iters;
    t0 = clock64();
    t1 = clock64();
    r[7] = (double)(t1 - t0);
    if (threadIdx.x == 0) {
        for (int k = 0; k < 8; k++) out[k] = r[k];
        out[8] = (double)(a ^ p ^ q ^ z);   // keeps every chain live
    }
}

// a permutation cycle over n words with the given step (odd step, n a power
// of two: one cycle through every word)
__global__ void k_peak_chase_init(uint32_t *buf, uint32_t n, uint32_t step) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        buf[i] = (i + step) & (n - 1);
}

}  // namespace ffk
