// ff_seed_tc.cuh - the seeding search's full pass on the 5th-generation
// tensor cores (tcgen05, accumulators in tensor memory).  Same contraction
// and output as k_seed_mma (Sec. 3.1 Eq. 1 / Sec. 3.2 Eq. 4 read as an exact
// top-8 by (|q - c|^2, index)); only the machinery differs.
#pragma once

#include <cuda_bf16.h>

#include "ff_kernels.cuh"
#include "ff_seed.cuh"   // key_less, reg_insert

namespace ffk {

constexpr int kTcRows = 128;    // queries per CTA (MMA M) and candidates per tile (MMA N)
constexpr int kTcStages = 4;    // candidate tiles in flight in shared memory

// Byte offset of element (r, k) in a tile of 128 rows x K bf16 laid out for
// the tensor core without swizzling: 8-row x 16-byte core matrices, the K
// direction's core matrices 128 bytes apart, 8-row groups K * 16 bytes apart.
__host__ __device__ constexpr int tc_tile_offset(int r, int k, int K) {
    return (r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// Row-major bf16 rows of K (n of them) -> 128-row tiles in the layout above.
// Rows n .. to the next multiple of 128 are padding: zeros, or for
// candidates a +inf at position dh2, so that their keys are +inf.
template <int K>
__global__ void k_seed_tile(const __nv_bfloat16 *__restrict__ rows, int n, int dh2,
                            uint8_t *__restrict__ tiles) {
    const int npad = (n + kTcRows - 1) / kTcRows * kTcRows;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;   // one 16-byte piece
    if (j >= npad * (K / 8)) return;
    const int r = j / (K / 8), kg = j - r * (K / 8);
    uint4 v = make_uint4(0, 0, 0, 0);
    if (r < n) {
        v = reinterpret_cast<const uint4 *>(rows + (size_t)r * K)[kg];
    } else if (dh2 >= 0 && dh2 / 8 == kg) {
        __align__(16) __nv_bfloat16 z[8];
#pragma unroll
        for (int e = 0; e < 8; e++)
            z[e] = (kg * 8 + e == dh2) ? __float2bfloat16(__int_as_float(0x7f800000))
                                       : __int2bfloat16_rn(0);
        v = *reinterpret_cast<const uint4 *>(z);
    }
    uint8_t *tile = tiles + (size_t)(r / kTcRows) * kTcRows * K * 2;
    *reinterpret_cast<uint4 *>(tile + tc_tile_offset(r % kTcRows, kg * 8, K)) = v;
}

__device__ __forceinline__ uint32_t tc_smem(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
// shared-memory matrix descriptor (no swizzle): start, K-direction core
// matrix offset, 8-row group offset, descriptor version 1
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
__device__ __forceinline__ void mbar_init(uint64_t *m, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_smem(m)), "r"(count));
}
__device__ __forceinline__ bool mbar_test(uint64_t *m, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(ok)
        : "r"(tc_smem(m)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for phase `parity` of m: false when the CTA's abort flag is up
// or wait_ns passed (then the error word gets FF_ETIMEOUT and the flag rises).
__device__ __forceinline__ bool mbar_wait(uint64_t *m, uint32_t parity, unsigned long long wait_ns,
                                          volatile int *abort_flag, int *err) {
    if (mbar_test(m, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    while (!mbar_test(m, parity)) {
        if (*abort_flag) return false;
        if (globaltimer_ns() - t0 > wait_ns) {
            atomicCAS(err, 0, kErrTimeout);
            *abort_flag = 1;
            return false;
        }
    }
    return true;
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *m, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc_smem(m)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *m) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc_smem(m)) : "memory");
}
// one contiguous global -> shared copy, completing on mbarrier m
__device__ __forceinline__ void bulk_copy(void *dst, const void *src, uint32_t bytes, uint64_t *m) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(tc_smem(dst)),
        "l"(src), "r"(bytes), "r"(tc_smem(m))
        : "memory");
}

template <int KS>
__host__ __device__ constexpr int tc_seed_smem_bytes() {
    return kTcRows * 16 * KS * 2 * (1 + kTcStages) + 8 * 32 * 32 * 4;
}

// 64 consecutive 32-bit columns of this warp's 32 tensor-memory lanes
__device__ __forceinline__ void tmem_ld64(uint32_t *r, uint32_t taddr) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%64];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
        : "r"(taddr));
}

// Per CTA: 128 queries (tensor-memory lanes; epilogue thread = query row)
// against one chunk of candidates, 128 per tile.  Warp 8 allocates tensor
// memory and streams candidate tiles into a 4-stage ring with bulk copies;
// warp 9 issues the K/16 MMAs of each tile into one of two 128-column
// accumulators; warps 0-7 read their rows' keys per tile with tcgen05.ld
// (warps w and w + 4: the same rows, the first and the second 64 columns)
// and keep each query's top-8 by (key, index) in registers, key
// entering only at or below min(the query's bound t0, its 8th key) (a key
// equal to it only while the list's 8th key is larger; keys are exact
// integers).  All waits are bounded.  Output as k_seed_mma, with two lists
// per chunk (chunk slots 2 blockIdx.y and 2 blockIdx.y + 1).
template <int KS>
__global__ void __launch_bounds__(320)
    k_seed_tc(const uint8_t *__restrict__ qtile, const int *__restrict__ qn,
              const uint8_t *__restrict__ ctile, int NQ, int NC, int chunk, int W, int stride,
              int Wc, const float *__restrict__ t0, int t0_chunks, int2 *__restrict__ part,
              int *err, unsigned long long wait_ns) {
    constexpr int K = 16 * KS;
    constexpr uint32_t TILE_BYTES = kTcRows * K * 2;
    constexpr float kEmpty = 3.0e38f;
    // dynamic shared memory (tc_seed_smem_bytes<KS>()): the query tile, the
    // candidate ring and each epilogue warp's 32 x 32 key scratch
    extern __shared__ __align__(1024) uint8_t tc_dyn[];
    uint8_t *sA = tc_dyn;
    uint8_t(*sB)[TILE_BYTES] = reinterpret_cast<uint8_t(*)[TILE_BYTES]>(tc_dyn + TILE_BYTES);
    float(*scr)[32][32] =
        reinterpret_cast<float(*)[32][32]>(tc_dyn + TILE_BYTES * (1 + kTcStages));   // [8][32][32]
    __shared__ __align__(8) uint64_t bar_a, full[kTcStages], empty[kTcStages], accf[2], acce[2];
    __shared__ uint32_t taddr_slot;
    __shared__ int abort_flag;
    volatile int *v_abort = &abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int qt = blockIdx.x;
    const int c0 = blockIdx.y * chunk, c1 = min(c0 + chunk, NC);
    const int ntiles = (c1 - c0 + kTcRows - 1) / kTcRows;   // chunk is a multiple of 128
    if (tid == 0) {
        abort_flag = 0;
        mbar_init(&bar_a, 1);
        for (int s = 0; s < kTcStages; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], 8);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 8) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(
            tc_smem(&taddr_slot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = taddr_slot;

    if (warp == 8) {
        // ---------------- producer: queries once, then candidate tiles
        if (lane == 0) {
            mbar_expect_tx(&bar_a, TILE_BYTES);
            bulk_copy(sA, qtile + (size_t)qt * TILE_BYTES, TILE_BYTES, &bar_a);
            const int tile0 = c0 / kTcRows;
            for (int t = 0; t < ntiles; t++) {
                const int s = t % kTcStages;
                if (t >= kTcStages &&
                    !mbar_wait(&empty[s], ((t / kTcStages) - 1) & 1, wait_ns, v_abort, err))
                    break;
                mbar_expect_tx(&full[s], TILE_BYTES);
                bulk_copy(sB[s], ctile + (size_t)(tile0 + t) * TILE_BYTES, TILE_BYTES, &full[s]);
            }
        }
    } else if (warp == 9) {
        // ---------------- MMA issuer
        if (lane == 0 && mbar_wait(&bar_a, 0, wait_ns, v_abort, err)) {
            // kind::f16, bf16 x bf16 -> f32, both K-major, N = 128, M = 128
            constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) |
                                       ((uint32_t)(kTcRows >> 3) << 17) |
                                       ((uint32_t)(kTcRows >> 4) << 24);
            for (int t = 0; t < ntiles; t++) {
                const int s = t % kTcStages, b = t & 1;
                if (!mbar_wait(&full[s], (t / kTcStages) & 1, wait_ns, v_abort, err)) break;
                if (t >= 2 && !mbar_wait(&acce[b], ((t >> 1) - 1) & 1, wait_ns, v_abort, err)) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = taddr + (uint32_t)(b * kTcRows);
#pragma unroll
                for (int ks = 0; ks < KS; ks++) {
                    const uint64_t da = tc_desc(tc_smem(sA) + ks * 256, 128, K * 16);
                    const uint64_t db = tc_desc(tc_smem(sB[s]) + ks * 256, 128, K * 16);
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                        "l"(da), "l"(db), "r"(idesc), "r"(ks));
                }
                asm volatile(
                    "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::
                        "r"(tc_smem(&empty[s]))
                    : "memory");
                asm volatile(
                    "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::
                        "r"(tc_smem(&accf[b]))
                    : "memory");
            }
        }
    } else {
        // ---------------- epilogue: warps w and w + 4 share tensor-memory lanes
        // 32 (w mod 4) .. +31 (thread = query row) and take the first and the
        // second 64 keys of each tile: two lists per query, merged later
        const int quarter = warp & 3, half = warp >> 2;
        const int row = quarter * 32 + lane, q = qt * kTcRows + row;
        float tinit = kEmpty;
        if (t0 && q < NQ)
            for (int c = 0; c < t0_chunks; c++) tinit = fminf(tinit, __ldg(t0 + (size_t)c * NQ + q));
        float lk[8];
        int li[8];
#pragma unroll
        for (int e = 0; e < 8; e++) {
            lk[e] = kEmpty;
            li[e] = 0x7fffffff;
        }
        for (int t = 0; t < ntiles; t++) {
            const int b = t & 1;
            if (!mbar_wait(&accf[b], (t >> 1) & 1, wait_ns, v_abort, err)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int base = c0 + t * kTcRows;
            // this warp's 64 keys of the tile for its row
            uint32_t r[64];
            const uint32_t ta = taddr + ((uint32_t)(quarter * 32) << 16) +
                                (uint32_t)(b * kTcRows + half * 64);
            tmem_ld64(r, ta);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            // bound of this row: a key equal to it counts only while the list's
            // 8th key is larger
            float tq = fminf(lk[7], tinit);
            float thr = lk[7] > tq ? tq + 1.0f : tq;
#pragma unroll
            for (int cc = 0; cc < 64; cc += 32) {
                float mn = __uint_as_float(r[cc]);
#pragma unroll
                for (int j = 1; j < 32; j++) mn = fminf(mn, __uint_as_float(r[cc + j]));
                if (mn < thr) {
                    // rare: the hits of these 32 keys, in column order, through
                    // this lane's scratch column
                    uint32_t mask = 0;
#pragma unroll
                    for (int j = 0; j < 32; j++) {
                        const float key = __uint_as_float(r[cc + j]);
                        scr[warp][j][lane] = key;
                        mask |= (key < thr ? 1u : 0u) << j;
                    }
                    while (mask) {
                        const int j = __ffs(mask) - 1;
                        mask &= mask - 1;
                        const float key = scr[warp][j][lane];
                        if (key < thr) {
                            const int ord = base + half * 64 + cc + j;
                            if (key_less(key, ord, lk[7], li[7])) reg_insert(lk, li, key, ord);
                            tq = fminf(lk[7], tinit);
                            thr = lk[7] > tq ? tq + 1.0f : tq;
                        }
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce[b]);
        }
        if (q < NQ && !*v_abort) {
            const int qq = qn[q];
            int2 *dst = part + ((size_t)(2 * blockIdx.y + half) * NQ + q) * 8;
#pragma unroll
            for (int e = 0; e < 8; e++) {
                if (li[e] == 0x7fffffff) {
                    dst[e] = make_int2(0x7fffffff, 0x7fffffff);
                } else {
                    const int ci = li[e];
                    const int idx = (ci / Wc) * stride * W + (ci % Wc) * stride;
                    dst[e] = make_int2((int)lk[e] + qq, idx);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 8) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(taddr));
    }
}

}  // namespace ffk
