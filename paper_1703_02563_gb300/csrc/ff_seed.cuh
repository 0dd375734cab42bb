// ff_seed.cuh - seeding search on the tensor cores (arXiv 1703.02563, Sec. 3.1
// Eq. 1 and Sec. 3.2 Eq. 4: the l candidates of every coarsest-grid point).
//
// The exact top-l nearest neighbours of a query vector q among candidate
// vectors c (squared Euclidean distance of int8 WHT codes) only need, per
// query, the ranking of key(c) = |c|^2 - 2 q.c, since |q|^2 is common.  The
// keys of all (query, candidate) pairs are one matrix product -- the one
// dense contraction of the method -- computed exactly on the bf16 tensor
// cores with FP32 accumulation:
//   query row     = (-2 q_1 .. -2 q_D, 65536, 256, 1, 0 ..)
//   candidate row = (  c_1 ..   c_D,  h2,  h1, h0, 0 ..),  |c|^2 = h2 65536 + h1 256 + h0
// Every entry is an integer of magnitude <= 256 or a power of two (exact in
// bf16), every product is exact, and every partial sum stays below 2^24 in
// magnitude, so FP32 accumulation in any order returns the key exactly.
#pragma once
#include <cuda_bf16.h>

#include "ff_kernels.cuh"

namespace ffk {

// Gathers the level-0 feature vectors of an (outW x outH) grid with spacing
// `step` (the coarsest-grid queries, or the stride-sigma candidates) into the
// bf16 rows above (K = 16 for gray, 32 for Lab).  Queries also get |q|^2.
template <int C, int K, bool QUERY>
__global__ void k_seed_prep(const uint8_t *__restrict__ feat, int W, int step, int outW, int outH,
                            __nv_bfloat16 *__restrict__ out, int *__restrict__ qnorm) {
    constexpr int D = 9 * C;
    static_assert(D + 3 <= K, "no room for the norm digits");
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= outW * outH) return;
    const int oy = o / outW, ox = o - oy * outW;
    const int8_t *src = reinterpret_cast<const int8_t *>(feat) +
                        ((size_t)oy * step * W + (size_t)ox * step) * Geo<C>::P;
    __align__(16) __nv_bfloat16 row[K];
    int nn = 0;
#pragma unroll
    for (int d = 0; d < D; d++) {
        const int v = (int)src[d];
        nn += v * v;
        row[d] = __int2bfloat16_rn(QUERY ? -2 * v : v);
    }
    if (QUERY) {
        row[D] = __int2bfloat16_rn(65536);
        row[D + 1] = __int2bfloat16_rn(256);
        row[D + 2] = __int2bfloat16_rn(1);
    } else {
        row[D] = __int2bfloat16_rn(nn >> 16);
        row[D + 1] = __int2bfloat16_rn((nn >> 8) & 255);
        row[D + 2] = __int2bfloat16_rn(nn & 255);
    }
#pragma unroll
    for (int d = D + 3; d < K; d++) row[d] = __int2bfloat16_rn(0);
    uint4 *dst = reinterpret_cast<uint4 *>(out + (size_t)o * K);
    const uint4 *s4 = reinterpret_cast<const uint4 *>(row);
#pragma unroll
    for (int k = 0; k < K / 8; k++) dst[k] = s4[k];
    if (QUERY) qnorm[o] = nn;
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                               uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldmatrix_x4(uint32_t (&r)[4], const void *smem_row) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_row);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(s));
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ bool key_less(float k, int i, float K2, int I2) {
    return k < K2 || (k == K2 && i < I2);
}

// insert (key, ordinal) into a register list of 8 ascending by (key,
// ordinal), dropping the last entry; the displaced entries move down in the
// same order, so equal keys keep their ordinal order
__device__ __forceinline__ void reg_insert(float (&lk)[8], int (&li)[8], float key, int ord) {
#pragma unroll
    for (int e = 0; e < 8; e++) {
        const bool sw = key_less(key, ord, lk[e], li[e]);
        const float tk = lk[e];
        const int ti = li[e];
        lk[e] = sw ? key : tk;
        li[e] = sw ? ord : ti;
        key = sw ? tk : key;
        ord = sw ? ti : ord;
    }
}

// Per CTA: 64 queries (4 warps x one m16 tile of 16 queries, whose A
// fragments stay in registers) against one chunk of candidates, 64 at a time
// through a 3-stage cp.async ring in shared memory (rows padded so ldmatrix
// is free of bank conflicts; one barrier per tile).  In the m16n8
// accumulator layout each lane holds two query rows and, per n8 tile, two
// candidate columns; it keeps its own top-8 list for each of its rows over
// the columns it sees.  A key enters only if it is at most the row's bound:
// the smallest of the query's initial bound (t0: 8th keys of subsets of the
// candidates) and the quad's threshold (the smallest 8th key among the four
// lanes of the row; that lane alone holds 8 keys at or below it), so no key
// of the final top 8 is ever filtered out; keys equal to the bound go
// through the exact (key, index) insertion.  Tiles without any such key in a
// warp cost only the matrix product and a min tree.  At the end the four
// lists of each row are merged in shared memory and the chunk's top-8 of
// every query is written as (|q|^2 + key, linear index) for k_seed_merge --
// or, when t0_out is given, only the chunk's 8th key (a bound pass).
// Candidate ordinal ci of a launch is candidate ci * cstep of the grid; t0 has
// t0_chunks bounds per query (t0[c * NQ + q]).
template <int KS>
__global__ void __launch_bounds__(128)
    k_seed_mma(const __nv_bfloat16 *__restrict__ qf, const int *__restrict__ qn,
               const __nv_bfloat16 *__restrict__ cf, int NQ, int NC, int chunk, int cstep,
               int W, int stride, int Wc, const float *__restrict__ t0, int t0_chunks,
               float *__restrict__ t0_out, int2 *__restrict__ part) {
    constexpr int K = 16 * KS, BM = 64, BN = 64, NT = BN / 8, NSTAGE = 3, NPOS = 4 * NT;
    constexpr int SROW = K + 8;                      // padded smem row (bf16)
    constexpr int DH2 = KS == 1 ? 9 : 27;            // position of the h2 digit
    constexpr float kEmpty = 3.0e38f;
    __shared__ __align__(16) __nv_bfloat16 sB[NSTAGE][BN][SROW];
    // per-warp scratch of the slow path; reused for the final merge
    __shared__ __align__(16) float scr[4][NPOS][32];
    float(*mkey)[4][8] = reinterpret_cast<float(*)[4][8]>(&scr[0][0][0]);
    __shared__ int mord[BM][4][8];
    static_assert(sizeof(scr) >= sizeof(float) * BM * 4 * 8, "merge buffer too small");

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q0 = blockIdx.x * BM;
    const int c0 = blockIdx.y * chunk, c1 = min(c0 + chunk, NC);
    const int ntiles = (c1 - c0 + BN - 1) / BN;

    // A fragments of this warp's 16 query rows (m16n8k16, row-major A)
    uint32_t a[KS][4];
    {
        const int r = q0 + warp * 16 + (lane >> 2);
#pragma unroll
        for (int ks = 0; ks < KS; ks++) {
            const int c = ks * 16 + (lane & 3) * 2;
            const uint32_t *p0 = reinterpret_cast<const uint32_t *>(qf + (size_t)r * K + c);
            const uint32_t *p1 = reinterpret_cast<const uint32_t *>(qf + (size_t)(r + 8) * K + c);
            a[ks][0] = r < NQ ? __ldg(p0) : 0u;
            a[ks][1] = r + 8 < NQ ? __ldg(p1) : 0u;
            a[ks][2] = r < NQ ? __ldg(p0 + 4) : 0u;
            a[ks][3] = r + 8 < NQ ? __ldg(p1 + 4) : 0u;
        }
    }
    float tinit[2];
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int r = q0 + warp * 16 + (lane >> 2) + h * 8;
        float v = kEmpty;
        if (t0 && r < NQ)
            for (int c = 0; c < t0_chunks; c++) v = fminf(v, __ldg(t0 + (size_t)c * NQ + r));
        tinit[h] = v;
    }
    float lk[2][8];
    int li[2][8];
#pragma unroll
    for (int h = 0; h < 2; h++)
#pragma unroll
        for (int e = 0; e < 8; e++) {
            lk[h][e] = kEmpty;
            li[h][e] = 0x7fffffff;
        }

    // stage tile t into its ring slot; a missing candidate is a zero row whose
    // h2 digit is +inf, so its key is +inf and it is never inserted
    auto stage = [&](int t) {
        if (t < ntiles) {
            const int b = t % NSTAGE, base = c0 + t * BN;
            for (int j = tid; j < BN * (K / 8); j += 128) {
                const int cc = j / (K / 8), p16 = j - cc * (K / 8);
                const int ci = base + cc;
                __nv_bfloat16 *dst = &sB[b][cc][p16 * 8];
                if (ci < c1) {
                    cp_async16(dst, cf + (size_t)ci * cstep * K + p16 * 8);
                } else {
                    __align__(16) __nv_bfloat16 z[8];
#pragma unroll
                    for (int e = 0; e < 8; e++)
                        z[e] = (p16 * 8 + e == DH2) ? __float2bfloat16(__int_as_float(0x7f800000))
                                                    : __int2bfloat16_rn(0);
                    *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(z);
                }
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");   // (possibly empty) group
    };
    stage(0);
    stage(1);

    for (int t = 0; t < ntiles; t++) {
        const int b = t % NSTAGE;
        asm volatile("cp.async.wait_group 1;" ::: "memory");   // tile t has landed
        __syncthreads();   // ... for every thread; and slot (t+2)%3 = (t-1)%3 is free
        stage(t + 2);
        float acc[NT][4];
#pragma unroll
        for (int nt = 0; nt < NT; nt++)
#pragma unroll
            for (int j = 0; j < 4; j++) acc[nt][j] = 0.f;
        // B fragments by ldmatrix.x4: matrices (nt, k 0-7), (nt, k 8-15),
        // (nt+1, k 0-7), (nt+1, k 8-15), rows = candidates
#pragma unroll
        for (int ks = 0; ks < KS; ks++) {
#pragma unroll
            for (int nt = 0; nt < NT; nt += 2) {
                const int mat = lane >> 3, rr = lane & 7;
                const int n = (nt + (mat >> 1)) * 8 + rr;
                const int kk = ks * 16 + (mat & 1) * 8;
                uint32_t bb[4];
                ldmatrix_x4(bb, &sB[b][n][kk]);
                mma_bf16_16816(acc[nt], a[ks], bb[0], bb[1]);
                mma_bf16_16816(acc[nt + 1], a[ks], bb[2], bb[3]);
            }
        }
        // acc[nt] = keys of rows (lane>>2), (lane>>2)+8 and columns
        // nt*8 + 2*(lane&3) + {0, 1}: position p = 4 nt + j, row j>>1
        // A key equal to the bound can only enter this lane's list while the
        // list's own 8th key is larger: once the lane holds 8 keys at the
        // bound, a later candidate of this lane (a larger index) at the same
        // key loses the (key, index) order.  So equality counts only while
        // lk[h][7] > tq[h]; in flat image regions, where thousands of
        // candidates share one key, this keeps them off the slow path.  Keys
        // are exact integers, so "key <= tq" is "key < tq + 1".
        float tq[2], thr[2], mn[2];
#pragma unroll
        for (int h = 0; h < 2; h++) {
            float v = lk[h][7];
            v = fminf(v, __shfl_xor_sync(0xffffffffu, v, 1));
            v = fminf(v, __shfl_xor_sync(0xffffffffu, v, 2));
            tq[h] = fminf(v, tinit[h]);
            thr[h] = lk[h][7] > tq[h] ? tq[h] + 1.0f : tq[h];
            float m[NT];
#pragma unroll
            for (int nt = 0; nt < NT; nt++) m[nt] = fminf(acc[nt][2 * h], acc[nt][2 * h + 1]);
#pragma unroll
            for (int w2 = NT / 2; w2 > 0; w2 >>= 1)
#pragma unroll
                for (int nt = 0; nt < w2; nt++) m[nt] = fminf(m[nt], m[nt + w2]);
            mn[h] = m[0];
        }
        if (__any_sync(0xffffffffu, mn[0] < thr[0] || mn[1] < thr[1])) {
            // slow path: the lane's candidate keys in positions, then only its hits
            float *my = &scr[warp][0][lane];
            uint32_t mask = 0;
#pragma unroll
            for (int nt = 0; nt < NT; nt++)
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    my[(4 * nt + j) * 32] = acc[nt][j];
                    mask |= (acc[nt][j] < thr[j >> 1] ? 1u : 0u) << (4 * nt + j);
                }
            const int base = c0 + t * BN + (lane & 3) * 2;
            while (mask) {
                const int pos = __ffs(mask) - 1;
                mask &= mask - 1;
                const float key = my[pos * 32];
                const int ord = (base + (pos >> 2) * 8 + (pos & 1)) * cstep;
                if ((pos & 2) == 0) {
                    if (key_less(key, ord, lk[0][7], li[0][7])) reg_insert(lk[0], li[0], key, ord);
                } else {
                    if (key_less(key, ord, lk[1][7], li[1][7])) reg_insert(lk[1], li[1], key, ord);
                }
            }
            __syncwarp();
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();   // scr becomes the merge buffer

    // merge the four lists of each row (the lanes of a quad) in shared memory
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int row = warp * 16 + (lane >> 2) + h * 8;
#pragma unroll
        for (int e = 0; e < 8; e++) {
            mkey[row][lane & 3][e] = lk[h][e];
            mord[row][lane & 3][e] = li[h][e];
        }
    }
    __syncthreads();
    for (int row = tid; row < BM; row += 128) {
        const int q = q0 + row;
        if (q >= NQ) continue;
        float bk[8];
        int bi[8];
#pragma unroll
        for (int e = 0; e < 8; e++) {
            bk[e] = kEmpty;
            bi[e] = 0x7fffffff;
        }
        for (int s = 0; s < 4; s++)
            for (int e = 0; e < 8; e++) {
                const float key = mkey[row][s][e];
                const int ord = mord[row][s][e];
                if (ord == 0x7fffffff || !key_less(key, ord, bk[7], bi[7])) break;
                float ck = key;
                int cx = ord;
#pragma unroll
                for (int f = 0; f < 8; f++) {
                    const bool sw = key_less(ck, cx, bk[f], bi[f]);
                    const float tk = bk[f];
                    const int tx = bi[f];
                    bk[f] = sw ? ck : tk;
                    bi[f] = sw ? cx : tx;
                    ck = sw ? tk : ck;
                    cx = sw ? tx : cx;
                }
            }
        if (t0_out) {   // bound pass: this chunk's 8th key, +inf when fewer than 8
            t0_out[(size_t)blockIdx.y * NQ + q] =
                bi[7] == 0x7fffffff ? __int_as_float(0x7f800000) : bk[7];
            continue;
        }
        const int qq = qn[q];
        int2 *dst = part + ((size_t)blockIdx.y * NQ + q) * 8;
#pragma unroll
        for (int e = 0; e < 8; e++) {
            if (bi[e] == 0x7fffffff) {
                dst[e] = make_int2(0x7fffffff, 0x7fffffff);
            } else {
                const int ci = bi[e];
                const int idx = (ci / Wc) * stride * W + (ci % Wc) * stride;
                dst[e] = make_int2((int)bk[e] + qq, idx);
            }
        }
    }
}

}  // namespace ffk
