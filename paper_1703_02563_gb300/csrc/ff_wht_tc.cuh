// Sec. 3.1 WHT features on the bf16 tensor cores (mma.sync m16n8k16, FP32
// accumulation): per level pixel, the 9 lowest-sequency Walsh coefficients
// per channel are one row of (8x8 window, flattened to 64) x (64 x 9 basis).
//
// Exactness: level-image values are integers 0..255 and the basis entries
// are +-1 (or 0 in the padding columns), all exact in bf16; every partial
// sum of 64 such products is an integer of magnitude <= 16320 < 2^24, so the
// FP32 accumulation is exact in any order and the coefficients equal the
// integer ones.  The int8 codes are then quantised exactly as in k_features.
//
// The precision form (IN = 1, 2) feeds the FP32 scale-space image instead:
// the level's area average without rounding (Sec. 3.6; exact in FP32, a sum
// of at most 255 4^L < 2^24 divided by 4^L), rounded to bf16 (IN = 1) or
// fp16 (IN = 2), and returns the FP32 coefficients.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace ffk {

// Walsh function u in sequency order at sample i of 8: ++++++++, ++++----, ++----++
__device__ __forceinline__ int walsh8(int u, int i) {
    if (u == 0) return 1;
    if (u == 1) return i < 4 ? 1 : -1;
    return (i < 2 || i >= 6) ? 1 : -1;
}

__device__ __forceinline__ uint32_t bf16_pair(uint16_t lo, uint16_t hi) {
    return (uint32_t)lo | ((uint32_t)hi << 16);
}

// bf16 bits of a basis entry: +1, -1 or 0
__device__ __forceinline__ uint16_t bf16_sign(int v) {
    return v > 0 ? (uint16_t)0x3F80 : (v < 0 ? (uint16_t)0xBF80 : (uint16_t)0);
}

// basis B[k][n], k = 8 i + j over the 8x8 window, n = 3u + v (0 for n >= 9)
__device__ __forceinline__ int wht_basis(int k, int n) {
    if (n >= 9) return 0;
    return walsh8(n / 3, k >> 3) * walsh8(n % 3, k & 7);
}

// fp16 bits of a basis entry: +1, -1 or 0
__device__ __forceinline__ uint16_t f16_sign(int v) {
    return v > 0 ? (uint16_t)0x3C00 : (v < 0 ? (uint16_t)0xBC00 : (uint16_t)0);
}

__device__ __forceinline__ void mma_f16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                              uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// One CTA: a 16x16 tile of level pixels, 4 warps x 4 tile rows; each tile
// row is one m16 fragment (16 pixels), K = 64 in 4 k-steps of two window
// rows, N = 9 coefficients padded to 16 (two n8 fragments).
// FLOAT_OUT: write the raw FP32 coefficients [HL][WL][9C] to fout instead
// of the int8 features.  IN: 0 the rounded integer level image in bf16; 1,
// 2 the unrounded FP32 scale-space image rounded to bf16, fp16 (FLOAT_OUT).
template <int C, bool FLOAT_OUT, int IN = 0>
__global__ void __launch_bounds__(128)
    k_features_tc(const uint8_t *__restrict__ img, int pitch, int W, int H, int L, int WL, int HL,
                  uint8_t *__restrict__ out, float *__restrict__ fout) {
    static_assert(IN == 0 || FLOAT_OUT, "the precision form returns coefficients");
    constexpr int TS = 16, TW = TS + 7, P = Geo<C>::P;
    __shared__ uint16_t sD[C][TW][TW + 1];                  // bf16 bits of D_n (tile + halo)
    __shared__ __align__(16) uint8_t sOut[TS * TS][P];     // int8 codes of the tile
    const int n = 1 << L;
    const int bx = blockIdx.x * TS, by = blockIdx.y * TS;
    const int half = (n * n) >> 1;
    for (int k = threadIdx.x; k < C * TW * TW; k += blockDim.x) {
        const int c = k / (TW * TW), rem = k - c * (TW * TW);
        const int ty = rem / TW, tx = rem - ty * TW;
        const int gx = clampi(bx - 3 + tx, 0, WL - 1);
        const int gy = clampi(by - 3 + ty, 0, HL - 1);
        const uint8_t *plane = img + (size_t)c * H * pitch;
        int sum = 0;
        for (int i = 0; i < n; i++) {
            const uint8_t *row = plane + (size_t)min(gy * n + i, H - 1) * pitch;
            for (int j = 0; j < n; j++) sum += row[min(gx * n + j, W - 1)];
        }
        if constexpr (IN == 0) {
            sD[c][ty][tx] = __bfloat16_as_ushort(__int2bfloat16_rn((sum + half) >> (2 * L)));
        } else {
            const float avg = (float)sum / (float)(n * n);   // exact
            sD[c][ty][tx] = IN == 1 ? __bfloat16_as_ushort(__float2bfloat16_rn(avg))
                                    : __half_as_ushort(__float2half_rn(avg));
        }
    }
    if (!FLOAT_OUT)
        for (int k = threadIdx.x; k < TS * TS * P / 16; k += blockDim.x)
            reinterpret_cast<uint4 *>(&sOut[0][0])[k] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    // B fragments: reg 0 holds k = 2t, 2t+1 of window row 2s, reg 1 the same
    // columns of window row 2s+1; column n = 8 nf + g
    uint32_t bfr[4][2][2];
#pragma unroll
    for (int s = 0; s < 4; s++)
#pragma unroll
        for (int nf = 0; nf < 2; nf++)
#pragma unroll
            for (int r = 0; r < 2; r++) {
                const int k0 = 8 * (2 * s + r) + 2 * t, col = 8 * nf + g;
                if constexpr (IN == 2)
                    bfr[s][nf][r] = bf16_pair(f16_sign(wht_basis(k0, col)),
                                              f16_sign(wht_basis(k0 + 1, col)));
                else
                    bfr[s][nf][r] = bf16_pair(bf16_sign(wht_basis(k0, col)),
                                              bf16_sign(wht_basis(k0 + 1, col)));
            }
#pragma unroll 1
    for (int rr = 0; rr < 4; rr++) {
        const int ty = warp * 4 + rr;
#pragma unroll
        for (int c = 0; c < C; c++) {
            float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
            for (int s = 0; s < 4; s++) {
                const uint16_t *r0 = &sD[c][ty + 2 * s][0];
                const uint16_t *r1 = &sD[c][ty + 2 * s + 1][0];
                // A: row = pixel (g or g+8), column k = 2t, 2t+1 (+8: next window row)
                uint32_t a[4];
                a[0] = bf16_pair(r0[g + 2 * t], r0[g + 2 * t + 1]);
                a[1] = bf16_pair(r0[g + 8 + 2 * t], r0[g + 8 + 2 * t + 1]);
                a[2] = bf16_pair(r1[g + 2 * t], r1[g + 2 * t + 1]);
                a[3] = bf16_pair(r1[g + 8 + 2 * t], r1[g + 8 + 2 * t + 1]);
                if constexpr (IN == 2) {
                    mma_f16_16816(acc[0], a, bfr[s][0][0], bfr[s][0][1]);
                    mma_f16_16816(acc[1], a, bfr[s][1][0], bfr[s][1][1]);
                } else {
                    mma_bf16_16816(acc[0], a, bfr[s][0][0], bfr[s][0][1]);
                    mma_bf16_16816(acc[1], a, bfr[s][1][0], bfr[s][1][1]);
                }
            }
            // acc[nf][h * 2 + e]: pixel g + 8h, coefficient 8 nf + 2t + e
#pragma unroll
            for (int nf = 0; nf < 2; nf++)
#pragma unroll
                for (int h = 0; h < 2; h++)
#pragma unroll
                    for (int e = 0; e < 2; e++) {
                        const int coef = 8 * nf + 2 * t + e, px = g + 8 * h;
                        if (coef >= 9) continue;
                        const float v = acc[nf][h * 2 + e];
                        if (FLOAT_OUT) {
                            const int x = bx + px, y = by + ty;
                            if (x < WL && y < HL)
                                fout[((size_t)y * WL + x) * 9 * C + c * 9 + coef] = v;
                        } else {
                            const int iv = (int)v;   // an exact integer
                            const int q = coef == 0 ? ((iv + 32) >> 6) - 128 : ((iv + 8) >> 4);
                            sOut[ty * TS + px][c * 9 + coef] = (uint8_t)(clampi(q, -128, 127) & 0xff);
                        }
                    }
        }
    }
    if (FLOAT_OUT) return;
    __syncthreads();
    constexpr int V = P / 16;   // 16-byte words per pixel
    for (int k = threadIdx.x; k < TS * TS * V; k += blockDim.x) {
        const int p = k / V, w = k - p * V;
        const int x = bx + (p & (TS - 1)), y = by + p / TS;
        if (x < WL && y < HL)
            reinterpret_cast<uint4 *>(out + ((size_t)y * WL + x) * P)[w] =
                reinterpret_cast<const uint4 *>(&sOut[p][0])[w];
    }
}

}  // namespace ffk
