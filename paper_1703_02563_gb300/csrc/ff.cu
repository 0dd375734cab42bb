// ff.cu - GB300 (sm_103a) kernels and C ABI of the Flow Fields
// patch-matching loop (arXiv 1703.02563, Sec. 3).  The ABI is declared in
// include/ff.h.
#include <cuda.h>   // CUcontext / CUresult types only; the driver is reached through the runtime
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <deque>
#include <mutex>
#include <string>
#include <vector>

#include "ff.h"
#include "ff_kernels.cuh"

using namespace ffk;

// ============================================================================
// kernels
// ============================================================================

// Sec. 3.6 + 3.1: level image D_n (n x n area average rounded half up,
// replicate border) and its 9 lowest-sequency Walsh coefficients per channel
// over the 8x8 window at offsets -3..+4, quantised to int8:
//   DC: round(c/64) - 128, others: round(c/16), both saturated.
// One thread per level pixel; a 16x16 tile plus its 7-pixel halo of D_n is
// built in shared memory straight from the frame, then the coefficients come
// from separable +-1 row and column sums.  One launch covers every level of
// a frame (the levels are independent: each is computed from the frame), its
// blocks listed coarsest level first, since a coarse tile sums the most frame
// pixels per level pixel.
struct FeatLevels {
    int n;                                    // levels in this launch
    int L[FF_MAX_SCALES], WL[FF_MAX_SCALES], HL[FF_MAX_SCALES];
    int tiles_x[FF_MAX_SCALES];               // 16-pixel tiles across the level
    int first[FF_MAX_SCALES + 1];             // first block of each level
    uint8_t *out[FF_MAX_SCALES];
};
template <int C>
__global__ void __launch_bounds__(256)
    k_features(const uint8_t *__restrict__ img, int pitch, int W, int H, const FeatLevels lv) {
    constexpr int TS = 16, TW = TS + 7, P = Geo<C>::P;
    __shared__ int16_t sD[C][TW][TW];
    int li = 0;
    while (li + 1 < lv.n && (int)blockIdx.x >= lv.first[li + 1]) li++;
    const int b = (int)blockIdx.x - lv.first[li];
    const int L = lv.L[li], WL = lv.WL[li], HL = lv.HL[li];
    uint8_t *__restrict__ out = lv.out[li];
    const int n = 1 << L;
    const int bx = (b % lv.tiles_x[li]) * TS, by = (b / lv.tiles_x[li]) * TS;
    const int tid = threadIdx.y * TS + threadIdx.x;
    const int half = (n * n) >> 1;
    for (int k = tid; k < C * TW * TW; k += TS * TS) {
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
        sD[c][ty][tx] = (int16_t)((sum + half) >> (2 * L));
    }
    __syncthreads();
    const int x = bx + threadIdx.x, y = by + threadIdx.y;
    if (x >= WL || y >= HL) return;
    uint32_t words[P / 4];
#pragma unroll
    for (int k = 0; k < P / 4; k++) words[k] = 0;
#pragma unroll
    for (int c = 0; c < C; c++) {
        int r0[8], r1[8], r2[8];
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const int16_t *row = &sD[c][threadIdx.y + i][threadIdx.x];
            const int a0 = row[0], a1 = row[1], a2 = row[2], a3 = row[3];
            const int a4 = row[4], a5 = row[5], a6 = row[6], a7 = row[7];
            r0[i] = (a0 + a1 + a2 + a3) + (a4 + a5 + a6 + a7);
            r1[i] = (a0 + a1 + a2 + a3) - (a4 + a5 + a6 + a7);
            r2[i] = (a0 + a1 + a6 + a7) - (a2 + a3 + a4 + a5);
        }
        int coef[9];
#pragma unroll
        for (int v = 0; v < 3; v++) {
            const int *r = v == 0 ? r0 : (v == 1 ? r1 : r2);
            coef[0 * 3 + v] = (r[0] + r[1] + r[2] + r[3]) + (r[4] + r[5] + r[6] + r[7]);
            coef[1 * 3 + v] = (r[0] + r[1] + r[2] + r[3]) - (r[4] + r[5] + r[6] + r[7]);
            coef[2 * 3 + v] = (r[0] + r[1] + r[6] + r[7]) - (r[2] + r[3] + r[4] + r[5]);
        }
#pragma unroll
        for (int k = 0; k < 9; k++) {
            const int q = k == 0 ? ((coef[0] + 32) >> 6) - 128 : ((coef[k] + 8) >> 4);
            const int b = clampi(q, -128, 127) & 0xff;
            const int dim = c * 9 + k;
            words[dim >> 2] |= (uint32_t)b << (8 * (dim & 3));
        }
    }
    uint4 *dst = reinterpret_cast<uint4 *>(out + ((size_t)y * WL + x) * P);
#pragma unroll
    for (int k = 0; k < P / 16; k++)
        dst[k] = make_uint4(words[4 * k], words[4 * k + 1], words[4 * k + 2], words[4 * k + 3]);
}

// dense copy [H_L][W_L][9C] of a level's features (for inspection)
template <int C>
__global__ void k_dense(const uint8_t *__restrict__ feat, int N, int8_t *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    for (int d = 0; d < 9 * C; d++)
        out[(size_t)i * 9 * C + d] = (int8_t)feat[(size_t)i * Geo<C>::P + d];
}

// ---------------------------------------------------------------------------
// seeding: exact top-8 by (squared distance, linear index) of level-0 WHT
// vectors (Sec. 3.1 Eq. 1, Sec. 3.2 Eq. 4; kd-tree leaf replaced by the exact
// nearest neighbours it approximates)
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool lex_less(int d, int i, int D, int I) {
    return d < D || (d == D && i < I);
}

// insert (d, i) into the ascending list (D, I) of 8, dropping the last entry
__device__ __forceinline__ void list_insert(int (&D)[8], int (&I)[8], int d, int i) {
#pragma unroll
    for (int k = 0; k < 8; k++) {
        const bool sw = lex_less(d, i, D[k], I[k]);
        const int td = D[k], ti = I[k];
        D[k] = sw ? d : td;
        I[k] = sw ? i : ti;
        d = sw ? td : d;
        i = sw ? ti : i;
    }
}

// Phase 1: QPT queries per thread (a tile of 128*QPT queries per CTA), one
// candidate chunk per blockIdx.y.  Candidates of the chunk are staged 256 at
// a time in shared memory with their squared norms.  Since
// |q - c|^2 = |q|^2 + |c|^2 - 2 q.c and |q|^2 is fixed per query, the lists
// are kept on the key |c|^2 - 2 q.c (one dp4a per 4 dimensions for q.c) and
// |q|^2 is added on output.  Within a chunk candidates arrive in increasing
// linear index, so a strict compare against the list's worst key keeps the
// (distance, index) order.
template <int C, int QPT>
__global__ void __launch_bounds__(128)
    k_seed_scan(const uint8_t *__restrict__ f1, const uint8_t *__restrict__ f2, int W, int N,
                int WS, int NQ, int stride, int Wc, int ncand, int chunk, int2 *__restrict__ part) {
    constexpr int P = Geo<C>::P, NV = P / 16, NW = Geo<C>::NW, TILE = 256;
    __shared__ uint4 s_w[TILE][NV];
    __shared__ int2 s_ni[TILE];   // (norm, linear index)
    uint32_t qw[QPT][NW];
    int thr[QPT];
    int D[QPT][8], I[QPT][8];
#pragma unroll
    for (int j = 0; j < QPT; j++) {
        const int q = min((blockIdx.x * QPT + j) * 128 + threadIdx.x, NQ - 1);
        const int gy = q / WS, gx = q - gy * WS;
        const uint32_t *src =
            reinterpret_cast<const uint32_t *>(f1 + ((size_t)gy * N * W + gx * N) * P);
        int qn = 0;
#pragma unroll
        for (int w = 0; w < NW; w++) {
            qw[j][w] = __ldg(src + w);
            qn = __dp4a((int)qw[j][w], (int)qw[j][w], qn);
        }
        (void)qn;
        thr[j] = 0x7fffffff;   // the list's worst key; INT32_MAX while not full
#pragma unroll
        for (int k = 0; k < 8; k++) D[j][k] = I[j][k] = 0x7fffffff;
    }
    const int c0 = blockIdx.y * chunk, c1 = min(c0 + chunk, ncand);
    for (int base = c0; base < c1; base += TILE) {
        __syncthreads();
        for (int k = threadIdx.x; k < TILE; k += 128) {
            const int ci = base + k;
            if (ci < c1) {
                const int cy = (ci / Wc) * stride, cx = (ci % Wc) * stride;
                const uint4 *src = reinterpret_cast<const uint4 *>(f2 + ((size_t)cy * W + cx) * P);
                int nn = 0;
#pragma unroll
                for (int v = 0; v < NV; v++) {
                    const uint4 x = __ldg(src + v);
                    s_w[k][v] = x;
                    nn = __dp4a((int)x.x, (int)x.x, nn);
                    nn = __dp4a((int)x.y, (int)x.y, nn);
                    nn = __dp4a((int)x.z, (int)x.z, nn);
                    nn = __dp4a((int)x.w, (int)x.w, nn);
                }
                s_ni[k] = make_int2(nn, cy * W + cx);
            }
        }
        __syncthreads();
        const int cnt = min(TILE, c1 - base);
        for (int k = 0; k < cnt; k++) {
            uint32_t cw[NV * 4];
#pragma unroll
            for (int v = 0; v < NV; v++) {
                const uint4 x = s_w[k][v];
                cw[4 * v] = x.x;
                cw[4 * v + 1] = x.y;
                cw[4 * v + 2] = x.z;
                cw[4 * v + 3] = x.w;
            }
            const int2 ni = s_ni[k];
#pragma unroll
            for (int j = 0; j < QPT; j++) {
                int dot = 0;
#pragma unroll
                for (int w = 0; w < NW; w++) dot = __dp4a((int)qw[j][w], (int)cw[w], dot);
                const int key = ni.x - 2 * dot;
                if (key < thr[j]) {
                    // the list stores |c|^2 - 2 q.c; |q|^2 is added on output
                    list_insert(D[j], I[j], key, ni.y);
                    thr[j] = D[j][7];
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < QPT; j++) {
        const int q = (blockIdx.x * QPT + j) * 128 + threadIdx.x;
        if (q >= NQ) continue;
        int qn = 0;
#pragma unroll
        for (int w = 0; w < NW; w++) qn = __dp4a((int)qw[j][w], (int)qw[j][w], qn);
        int2 *dst = part + ((size_t)blockIdx.y * NQ + q) * 8;
#pragma unroll
        for (int k = 0; k < 8; k++)
            dst[k] = make_int2(I[j][k] == 0x7fffffff ? 0x7fffffff : D[j][k] + qn, I[j][k]);
    }
}

// Phase 2: merge the per-chunk lists of each query into its top-l.
__global__ void k_seed_merge(const int2 *__restrict__ part, int nchunks, int NQ, int leaf,
                             int *__restrict__ knn_idx, int *__restrict__ knn_dist) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= NQ) return;
    int D[8], I[8];
#pragma unroll
    for (int k = 0; k < 8; k++) D[k] = I[k] = 0x7fffffff;
    for (int c = 0; c < nchunks; c++) {
        const int2 *src = part + ((size_t)c * NQ + q) * 8;
        for (int k = 0; k < 8; k++) {
            const int2 e = src[k];
            if (e.y == 0x7fffffff) break;
            if (!lex_less(e.x, e.y, D[7], I[7])) break;
            list_insert(D, I, e.x, e.y);
        }
    }
    for (int k = 0; k < leaf; k++) {
        const bool ok = I[k] != 0x7fffffff;
        knn_idx[(size_t)q * leaf + k] = ok ? I[k] : -1;
        knn_dist[(size_t)q * leaf + k] = ok ? D[k] : -1;
    }
}

// Phase 3 (Eq. 1 rerank): each candidate p2 gives F = 8 (p2 - p); keep the
// lowest E at the coarsest scale, the earlier rank on ties.
template <int C>
__global__ void k_seed_rerank(const int *__restrict__ knn_idx, int leaf, const uint8_t *f1L,
                              const uint8_t *f2L, int W, int H, int L, int WL, int HL,
                              uint32_t *__restrict__ flow, int *__restrict__ cost) {
    constexpr int P = Geo<C>::P;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= WL * HL) return;
    const int gy = q / WL, gx = q - gy * WL;
    const int px = gx << L, py = gy << L;
    uint32_t qw[P / 4];
#pragma unroll
    for (int w = 0; w < P / 4; w++) qw[w] = ldg32(f1L + (size_t)q * P + 4 * w);
    uint32_t bf = kFlowInvalid;
    int bc = kCostInvalid;
    for (int r = 0; r < leaf; r++) {
        const int idx = knn_idx[(size_t)q * leaf + r];
        if (idx < 0) break;
        int fx = 8 * (idx % W - px), fy = 8 * (idx / W - py);
        clamp_flow(W, H, px, py, fx, fy);
        const int e = sad_full<C>(f2L, make_tap<P>(px, py, fx, fy, L, WL, HL), qw);
        if (e < bc) {
            bc = e;
            bf = pack_flow(fx, fy);
        }
    }
    flow[q] = bf;
    cost[q] = bc;
}

// caller-supplied seeds on the coarsest grid: clamp and evaluate
template <int C>
__global__ void k_seed_given(const uint32_t *__restrict__ seeds, const uint8_t *f1L,
                             const uint8_t *f2L, int W, int H, int L, int WL, int HL,
                             uint32_t *__restrict__ flow, int *__restrict__ cost) {
    constexpr int P = Geo<C>::P;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= WL * HL) return;
    const uint32_t s = seeds[q];
    if (flow_x(s) == -32768 || flow_y(s) == -32768) {
        flow[q] = kFlowInvalid;
        cost[q] = kCostInvalid;
        return;
    }
    const int gy = q / WL, gx = q - gy * WL;
    const int px = gx << L, py = gy << L;
    uint32_t qw[P / 4];
#pragma unroll
    for (int w = 0; w < P / 4; w++) qw[w] = ldg32(f1L + (size_t)q * P + 4 * w);
    int fx = flow_x(s), fy = flow_y(s);
    clamp_flow(W, H, px, py, fx, fy);
    flow[q] = pack_flow(fx, fy);
    cost[q] = sad_full<C>(f2L, make_tap<P>(px, py, fx, fy, L, WL, HL), qw);
}

// Sec. 3.2 coarse to fine: points of level L that are points of level L+1
// (both grid coordinates even) keep their flow, re-evaluated at scale n; the
// other points start unset.
template <int C>
__global__ void k_upsample(const uint32_t *__restrict__ pflow, int WP, const uint8_t *f1L,
                           const uint8_t *f2L, int W, int H, int L, int WL, int HL,
                           uint32_t *__restrict__ flow, int *__restrict__ cost) {
    constexpr int P = Geo<C>::P;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= WL * HL) return;
    const int gy = q / WL, gx = q - gy * WL;
    uint32_t f = kFlowInvalid;
    if (((gx | gy) & 1) == 0) f = pflow[(gy >> 1) * WP + (gx >> 1)];
    if (f == kFlowInvalid) {
        flow[q] = kFlowInvalid;
        cost[q] = kCostInvalid;
        return;
    }
    uint32_t qw[P / 4];
#pragma unroll
    for (int w = 0; w < P / 4; w++) qw[w] = ldg32(f1L + (size_t)q * P + 4 * w);
    const int px = gx << L, py = gy << L;
    flow[q] = f;
    cost[q] = sad_full<C>(f2L, make_tap<P>(px, py, flow_x(f), flow_y(f), L, WL, HL), qw);
}

#include "ff_sweep.cuh"
#include "ff_peaks.cuh"
#include "ff_seed.cuh"
#include "ff_wht_tc.cuh"
#include "ff_seed_tc.cuh"

// ---- region filter (Sec. 3.7) ------------------------------------------
// Kept points are joined into regions by a lock-free union-find: a root only
// ever gets a smaller parent (atomicMin), so every tree's root is the
// smallest index of its region and no thread waits on another.
__device__ __forceinline__ bool rf_close(uint32_t a, uint32_t b) {
    const int dx = flow_x(a) - flow_x(b), dy = flow_y(a) - flow_y(b);
    return dx * dx + dy * dy < 24 * 24;   // below 3 px
}

__device__ __forceinline__ int rf_find(const int *parent, int x) {
    int p;
    while ((p = __ldcg(parent + x)) != x) x = p;
    return x;
}

// find with path halving: each visited point is re-linked to its
// grandparent (an ancestor, so the trees stay valid under concurrent
// linking; atomicMin keeps every parent pointer non-increasing)
__device__ __forceinline__ int rf_find_halve(int *parent, int x) {
    int p = __ldcg(parent + x);
    while (p != x) {
        const int gp = __ldcg(parent + p);
        if (gp != p) atomicMin(parent + x, gp);
        x = p;
        p = gp;
    }
    return x;
}

__device__ void rf_unite(int *parent, int a, int b) {
    for (;;) {
        a = rf_find_halve(parent, a);
        b = rf_find_halve(parent, b);
        if (a == b) return;
        if (a > b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicMin(parent + b, a);   // link the larger root under the smaller
        if (old == b) return;
        b = old;                                     // b got another parent meanwhile: retry
    }
}

__global__ void k_rf_init(const uint8_t *__restrict__ mask, int N, int *parent, int *size,
                          uint8_t *flag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    parent[i] = mask[i] ? i : -1;
    size[i] = 0;
    flag[i] = 0;
}

__global__ void k_rf_union(const uint32_t *__restrict__ flow, const uint8_t *__restrict__ mask,
                           int W, int H, int *parent) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= W * H || !mask[i]) return;
    const int y = i / W, x = i - y * W;
    const uint32_t f = flow[i];
    if (x + 1 < W && mask[i + 1] && rf_close(f, flow[i + 1])) rf_unite(parent, i, i + 1);
    if (y + 1 < H && mask[i + W] && rf_close(f, flow[i + W])) rf_unite(parent, i, i + W);
}

// region sizes, and whether a region touches a joinable removed point
__global__ void k_rf_count(const uint32_t *__restrict__ flow, const uint8_t *__restrict__ mask,
                           int W, int H, int *parent, int *size, uint8_t *flag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= W * H || !mask[i]) return;
    const int y = i / W, x = i - y * W;
    const int r = rf_find_halve(parent, i);
    atomicMin(parent + i, r);
    atomicAdd(size + r, 1);
    const uint32_t f = flow[i];
    const int nb[4] = {x + 1 < W ? i + 1 : -1, x > 0 ? i - 1 : -1, y + 1 < H ? i + W : -1,
                       y > 0 ? i - W : -1};
    bool join = false;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        if (nb[k] < 0 || mask[nb[k]]) continue;
        const uint32_t g = flow[nb[k]];
        if (flow_x(g) != -32768 && flow_y(g) != -32768 && rf_close(f, g)) join = true;
    }
    if (join) flag[r] = 1;
}

__global__ void k_rf_apply(const uint8_t *mask_in, int N, int s, const int *__restrict__ parent,
                           const int *__restrict__ size, const uint8_t *__restrict__ flag,
                           uint8_t *mask_out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    uint8_t m = mask_in[i];
    if (m) {
        const int r = parent[i];
        if (size[r] < s && flag[r]) m = 0;
    }
    mask_out[i] = m;
}

// ---- sparsification (Sec. 3.7-3.8) -------------------------------------
// consistency error |F(p) + F_b(q)| in 1/8 px, q the final-grid point nearest
// to p + F(p); infinite when a flow is unset or q is off the grid
__device__ __forceinline__ double sp_error(uint32_t f, const uint32_t *__restrict__ bwd, int x,
                                           int y, int W, int H, int L) {
    if (flow_x(f) == -32768 || flow_y(f) == -32768) return CUDART_INF;
    const int half = 4 << L, sh = 3 + L;
    const int qx = x + ((flow_x(f) + half) >> sh), qy = y + ((flow_y(f) + half) >> sh);
    if (qx < 0 || qx >= W || qy < 0 || qy >= H) return CUDART_INF;
    const uint32_t b = bwd[qy * W + qx];
    if (flow_x(b) == -32768 || flow_y(b) == -32768) return CUDART_INF;
    const long long dx = flow_x(f) + flow_x(b), dy = flow_y(f) + flow_y(b);
    return sqrt((double)(dx * dx + dy * dy));
}

// one thread per q x q cell: keep the kept point of smallest summed error
// (first in raster order on ties) if the cell holds at least e kept points
__global__ void k_sparsify(const uint32_t *__restrict__ fwd, const uint32_t *__restrict__ b1,
                           const uint32_t *__restrict__ b2, const uint8_t *mask_in, int W, int H,
                           int L, int q, int e, int cells_x, int ncells, uint8_t *mask_out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    const int cy = (c / cells_x) * q, cx = (c % cells_x) * q;
    const int y1 = min(cy + q, H), x1 = min(cx + q, W);
    int count = 0, best = -1;
    double best_err = 0.0;
    for (int y = cy; y < y1; y++)
        for (int x = cx; x < x1; x++) {
            const int i = y * W + x;
            if (!mask_in[i]) continue;
            count++;
            const uint32_t f = fwd[i];
            double err = sp_error(f, b1, x, y, W, H, L);
            if (b2) err = err + sp_error(f, b2, x, y, W, H, L);
            if (best < 0 || err < best_err) {
                best = i;
                best_err = err;
            }
        }
    if (count < e) best = -1;
    for (int y = cy; y < y1; y++)
        for (int x = cx; x < x1; x++) mask_out[y * W + x] = (y * W + x == best) ? 1 : 0;
}

// level state -> caller's flow / cost arrays
__global__ void k_export(const uint32_t *__restrict__ flow, const int *__restrict__ cost, int N,
                         uint32_t *__restrict__ flow_out, int *__restrict__ cost_out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    flow_out[i] = flow[i];
    if (cost_out) cost_out[i] = cost[i];
}

// Sec. 3.7 forward/backward consistency: keep p iff |F(p) + F_b(q)|^2 < eps^2
// Sec. 3.7 on the final grid (points (x 2^L, y 2^L)): keep p iff
// |F(p) + F_b(q)| < eps for each of the NB backward flows, q the grid point
// nearest to p + F(p) (half up); an INVALID flow or a q off the grid rejects p.
template <int NB>
__global__ void k_filter(const uint32_t *__restrict__ fwd, const uint32_t *__restrict__ b1,
                         const uint32_t *__restrict__ b2, int W, int H, int L, int eps,
                         uint8_t *__restrict__ mask) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= W * H) return;
    const int y = i / W, x = i - y * W;
    const uint32_t f = fwd[i];
    uint8_t m = 0;
    if (flow_x(f) != -32768 && flow_y(f) != -32768) {
        const int half = 4 << L, sh = 3 + L;
        const int qx = x + ((flow_x(f) + half) >> sh), qy = y + ((flow_y(f) + half) >> sh);
        if (qx >= 0 && qx < W && qy >= 0 && qy < H) {
            m = 1;
#pragma unroll
            for (int j = 0; j < NB; j++) {
                const uint32_t b = (j == 0 ? b1 : b2)[qy * W + qx];
                if (flow_x(b) == -32768 || flow_y(b) == -32768) {
                    m = 0;
                } else {
                    const long long dx = flow_x(f) + flow_x(b), dy = flow_y(f) + flow_y(b);
                    if (!(dx * dx + dy * dy < (long long)eps * eps)) m = 0;
                }
            }
        }
    }
    mask[i] = m;
}

// ============================================================================
// host side
// ============================================================================
namespace {

constexpr int kMaxIters = 64;
constexpr int kNumDirs = 3;   // forward, backward, second backward
constexpr int kMaxChunks = 64;
constexpr int kCtasPerSm = 8;     // seeding grids: about this many CTAs per SM
constexpr int kSeedQpt = 2;
constexpr int kSeedSample = 16;   // candidate subsampling of the bound pass
constexpr int kSeedQueriesPerCta = 128 * kSeedQpt;

struct DirState {
    uint32_t *flow[2] = {nullptr, nullptr};   // ping-pong level state
    int *cost[2] = {nullptr, nullptr};
    unsigned long long *edge = nullptr;
    unsigned int *ticket = nullptr;           // [FF_MAX_SCALES * kMaxIters]
    int *knn_idx = nullptr;
    int *knn_dist = nullptr;
    int2 *part = nullptr;                     // seeding scratch: per-chunk lists
    __nv_bfloat16 *qbf = nullptr;             // seeding queries, bf16 rows of K
    int *qnorm = nullptr;                     //   their squared norms
    float *t0 = nullptr;                      //   upper bounds of their 8th key
    __nv_bfloat16 *cbf = nullptr;             // seeding candidates, bf16 rows of K
    uint8_t *qtile = nullptr, *ctile = nullptr;   // the same in 128-row tensor-core tiles
    int *err = nullptr;
};

}  // namespace

struct ff_ctx {
    ff_config cfg;
    int device = 0;
    int sms = 152;                // SMs of the device (grid sizes of the seeding)
    cudaStream_t stream = nullptr;
    cudaStream_t side = nullptr, side2 = nullptr;   // backward flows 1 and 2
    cudaEvent_t ev_a = nullptr, ev_b = nullptr, ev_c = nullptr;
    int C = 1, P = 16, S = 4, I = 4;
    int maxW = 0, maxH = 0;
    size_t feat_cap = 0;
    uint8_t *feat[2] = {nullptr, nullptr};
    int fw[2] = {0, 0}, fh[2] = {0, 0};
    bool have[2] = {false, false};
    DirState dir[kNumDirs];
    size_t nq_cap = 0;
    size_t edge_cap = 0;
    // staging for ff_pair_host
    uint8_t *img_dev[2] = {nullptr, nullptr};
    uint32_t *pair_flow[3] = {nullptr, nullptr, nullptr};   // fwd, bwd, second bwd
    uint8_t *pair_mask = nullptr;
    // region filter scratch: union-find parents, region sizes, join flags
    int *rf_parent = nullptr, *rf_size = nullptr;
    uint8_t *rf_flag = nullptr;
    unsigned long long wait_ns = 2000000000ull;
    int sweep_lanes = 4;   // propagation-warp lanes per grid point in the sweep: 2, 4 or 8
    int seed_tc = 1;       // seeding full pass on tcgen05 (0: mma.sync)
    int force_timeout = 0;
    long long launches = 0;
    std::string last_error;
    // launch timing (ff_profile): event pairs recorded on the launch stream,
    // one per launch (FF_PROFILE_LAUNCHES) or one per run of consecutive
    // sweep launches on a stream (FF_PROFILE_SWEEP_RUNS)
    int prof_mode = 0;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    struct ProfRec {
        int kernel, launches;
        size_t ev0, ev1;   // indices into ev_pool
    };
    std::vector<ProfRec> prof;
    const char *pending_kernel = nullptr;
    size_t pending_ev = 0;
    struct SweepRun {
        cudaStream_t stream;
        size_t ev0;
        int launches;
    };
    std::vector<SweepRun> runs;   // open runs, at most one per stream
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

ff_status fail(ff_ctx *ctx, ff_status s, const std::string &msg) {
    if (ctx) ctx->last_error = msg;
    return s;
}

ff_status check_cuda(ff_ctx *ctx, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return FF_OK;
    return fail(ctx, FF_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

const char *const kKernelNames[] = {"k_features", "k_seed_prep", "k_seed_scan", "k_seed_merge",
                                    "k_seed_rerank", "k_seed_given", "k_upsample",
                                    "k_sweep", "k_export", "k_filter", "k_dense", "k_region",
                                    "k_sparsify"};
constexpr int kNumKernels = sizeof(kKernelNames) / sizeof(kKernelNames[0]);

int kernel_id(const char *name) {
    for (int i = 0; i < kNumKernels; i++)
        if (strcmp(kKernelNames[i], name) == 0) return i;
    return -1;
}

cudaEvent_t pool_event(ff_ctx *c) {
    if (c->ev_used == c->ev_pool.size()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        c->ev_pool.push_back(e);
    }
    return c->ev_pool[c->ev_used++];
}

// ends open sweep run r: its end event on its own stream, one record
void close_run(ff_ctx *c, size_t r) {
    const ff_ctx::SweepRun run = c->runs[r];
    c->runs.erase(c->runs.begin() + (long)r);
    cudaEvent_t e = pool_event(c);
    if (!e) return;   // (the run is dropped)
    cudaEventRecord(e, run.stream);
    c->prof.push_back({kernel_id("k_sweep"), run.launches, run.ev0, c->ev_used - 1});
}

// Called before each launch while profiling.  Per launch: the start event.
// Sweep runs: a sweep launch opens a run on its stream (or extends the open
// one); any other launch on that stream closes it first.
void prof_begin(ff_ctx *c, const char *kernel) {
    if (c->prof_mode == 0) return;
    if (c->prof_mode == FF_PROFILE_SWEEP_RUNS) {
        const bool sweep = strcmp(kernel, "k_sweep") == 0;
        for (size_t r = 0; r < c->runs.size(); r++) {
            if (c->runs[r].stream != c->stream) continue;
            if (sweep) {
                c->pending_kernel = kernel;
                return;
            }
            close_run(c, r);
            break;
        }
        if (!sweep) return;
        cudaEvent_t e = pool_event(c);
        if (!e) return;
        cudaEventRecord(e, c->stream);
        c->runs.push_back({c->stream, c->ev_used - 1, 0});
        c->pending_kernel = kernel;
        return;
    }
    cudaEvent_t e = pool_event(c);
    if (!e) return;
    cudaEventRecord(e, c->stream);
    c->pending_kernel = kernel;
    c->pending_ev = c->ev_used - 1;
}

ff_status check_launch(ff_ctx *ctx, const char *what) {
    ctx->launches++;
    const ff_status s = check_cuda(ctx, cudaGetLastError(), what);
    if (ctx->prof_mode != 0 && ctx->pending_kernel) {
        if (ctx->prof_mode == FF_PROFILE_SWEEP_RUNS) {
            for (auto &r : ctx->runs)
                if (r.stream == ctx->stream) {
                    r.launches++;
                    break;
                }
        } else {
            cudaEvent_t e = pool_event(ctx);
            if (e) {
                cudaEventRecord(e, ctx->stream);
                ctx->prof.push_back(
                    {kernel_id(ctx->pending_kernel), 1, ctx->pending_ev, ctx->ev_used - 1});
            }
        }
        ctx->pending_kernel = nullptr;
    }
    return s;
}

void level_dims(int W, int H, int L, int *WL, int *HL) {
    const int n = 1 << L;
    *WL = (W + n - 1) / n;
    *HL = (H + n - 1) / n;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t level_offset(int W, int H, int P, int L) {
    size_t off = 0;
    for (int l = 0; l < L; l++) {
        int wl, hl;
        level_dims(W, H, l, &wl, &hl);
        off += align256((size_t)wl * hl * P);
    }
    return off;
}

// rows of one sweep strip for `lanes` propagation-warp lanes per grid point
// (8 gives the smallest strips)
int rows_per_strip(int lanes) {
    return lanes == 2 ? SweepGeo<1, 1>::RW : (lanes == 8 ? SweepGeo<1, 4>::RW : SweepGeo<1, 2>::RW);
}

template <typename T>
cudaError_t alloc(T **p, size_t count) {
    return cudaMalloc((void **)p, count * sizeof(T) + 16);
}

void free_all(ff_ctx *c) {
    for (int s = 0; s < 2; s++) {
        cudaFree(c->feat[s]);
        cudaFree(c->img_dev[s]);
        cudaFree(c->pair_flow[s]);
        if (s == 1) cudaFree(c->pair_flow[2]);
    }
    for (int s = 0; s < kNumDirs; s++) {
        DirState &d = c->dir[s];
        cudaFree(d.flow[0]);
        cudaFree(d.flow[1]);
        cudaFree(d.cost[0]);
        cudaFree(d.cost[1]);
        cudaFree(d.edge);
        cudaFree(d.ticket);
        cudaFree(d.knn_idx);
        cudaFree(d.knn_dist);
        cudaFree(d.part);
        cudaFree(d.qbf);
        cudaFree(d.qnorm);
        cudaFree(d.t0);
        cudaFree(d.cbf);
        cudaFree(d.qtile);
        cudaFree(d.ctile);
        cudaFree(d.err);
    }
    cudaFree(c->pair_mask);
    cudaFree(c->rf_parent);
    cudaFree(c->rf_size);
    cudaFree(c->rf_flag);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    c->ev_pool.clear();
    if (c->side) cudaStreamDestroy(c->side);
    if (c->side2) cudaStreamDestroy(c->side2);
    if (c->ev_a) cudaEventDestroy(c->ev_a);
    if (c->ev_b) cudaEventDestroy(c->ev_b);
    if (c->ev_c) cudaEventDestroy(c->ev_c);
}

ff_status validate_config(const ff_config *c, std::string *why) {
    if (c->patch != 8) return *why = "patch must be 8", FF_EINVAL;
    if (c->n_coeffs != 9) return *why = "n_coeffs must be 9", FF_EINVAL;
    if (c->channels != 1 && c->channels != 3) return *why = "channels must be 1 or 3", FF_EINVAL;
    if (c->scales < 1 || c->scales > FF_MAX_SCALES) return *why = "scales must be 1..8", FF_EINVAL;
    if (c->iters < 1 || c->iters > kMaxIters) return *why = "iters must be 1..64", FF_EINVAL;
    if (c->radius_q3 < 0 || c->radius_q3 > 255) return *why = "radius_q3 must be 0..255", FF_EINVAL;
    if (c->seed_leaf < 1 || c->seed_leaf > FF_MAX_LEAF) return *why = "seed_leaf must be 1..8", FF_EINVAL;
    if (c->seed_stride < 1 || c->seed_stride > 64) return *why = "seed_stride must be 1..64", FF_EINVAL;
    if (c->eps_q3 < 0 || c->eps_q3 > 65535) return *why = "eps_q3 out of range", FF_EINVAL;
    if (c->schedule < FF_SCHED_BASIC || c->schedule > FF_SCHED_PLUS_FAST_X2)
        return *why = "unknown schedule", FF_EINVAL;
    if (c->wht_tensor_cores != 0 && c->wht_tensor_cores != 1)
        return *why = "wht_tensor_cores must be 0 or 1", FF_EINVAL;
    if (c->region_min < 0 || c->region_min > (1 << 24))
        return *why = "region_min out of range", FF_EINVAL;
    if (c->schedule == FF_SCHED_PLUS_FAST_X2 && c->scales < 2)
        return *why = "the Fast x2 schedule needs at least 2 scales", FF_EINVAL;
    if (c->max_width < 1 || c->max_width > FF_MAX_DIM || c->max_height < 1 ||
        c->max_height > FF_MAX_DIM)
        return *why = "max_width/max_height must be 1..4096", FF_EINVAL;
    return FF_OK;
}

// seeding launch geometry: queries in tiles of 128, candidates split so the
// grid holds about kCtasPerSm CTAs per SM of the device (sms)
void seed_geometry(int nq, int ncand, int sms, int *nchunks, int *chunk) {
    const int qt = (nq + kSeedQueriesPerCta - 1) / kSeedQueriesPerCta;
    int nc = (kCtasPerSm * sms + qt - 1) / qt;
    nc = nc < 1 ? 1 : (nc > kMaxChunks ? kMaxChunks : nc);
    int ch = (ncand + nc - 1) / nc;
    if (ch < 512) ch = 512;
    *chunk = ch;
    *nchunks = (ncand + ch - 1) / ch;
}

// seeding geometry of the mma.sync scan: 64 queries per CTA, candidates
// split into chunks (whole 64-candidate tiles) so the grid holds about four
// CTAs per SM of the device (sms): long chunks, few restarts
void seed_geometry_mma(int nq, int ncand, int sms, int *nchunks, int *chunk) {
    const int qt = (nq + 63) / 64;
    int nc = (4 * sms + qt - 1) / qt;
    nc = nc < 1 ? 1 : (nc > kMaxChunks ? kMaxChunks : nc);
    int ch = (ncand + nc - 1) / nc;
    ch = ((ch + 63) / 64) * 64;
    if (ch < 512) ch = 512;
    *chunk = ch;
    *nchunks = (ncand + ch - 1) / ch;
}

ff_status launch_seed_knn(ff_ctx *c, int d, const uint8_t *fs, const uint8_t *fd, int W, int H) {
    DirState &st = c->dir[d];
    const int S = c->S, N = 1 << (S - 1);
    int WS, HS;
    level_dims(W, H, S - 1, &WS, &HS);
    const int nq = WS * HS;
    const int stride = c->cfg.seed_stride;
    const int Wc = (W + stride - 1) / stride, Hc = (H + stride - 1) / stride;
    const int ncand = Wc * Hc;
    // bf16 rows of the queries (coarsest grid) and candidates (stride grid)
    prof_begin(c, "k_seed_prep");
    if (c->C == 1)
        k_seed_prep<1, 16, true><<<(nq + 127) / 128, 128, 0, c->stream>>>(fs, W, N, WS, HS, st.qbf,
                                                                         st.qnorm);
    else
        k_seed_prep<3, 32, true><<<(nq + 127) / 128, 128, 0, c->stream>>>(fs, W, N, WS, HS, st.qbf,
                                                                         st.qnorm);
    ff_status s = check_launch(c, "k_seed_prep");
    if (s) return s;
    prof_begin(c, "k_seed_prep");
    if (c->C == 1)
        k_seed_prep<1, 16, false><<<(ncand + 127) / 128, 128, 0, c->stream>>>(
            fd, W, stride, Wc, Hc, st.cbf, nullptr);
    else
        k_seed_prep<3, 32, false><<<(ncand + 127) / 128, 128, 0, c->stream>>>(
            fd, W, stride, Wc, Hc, st.cbf, nullptr);
    s = check_launch(c, "k_seed_prep");
    if (s) return s;
    // bound pass over every kSeedSample-th candidate: the 8th key of each
    // chunk of the sample bounds the query's final 8th key from above
    const int ns = (ncand + kSeedSample - 1) / kSeedSample;
    int nchunks1, chunk1;
    seed_geometry_mma(nq, ns, c->sms, &nchunks1, &chunk1);
    {
        dim3 grid1((nq + 63) / 64, nchunks1);
        prof_begin(c, "k_seed_scan");
        if (c->C == 1)
            k_seed_mma<1><<<grid1, 128, 0, c->stream>>>(st.qbf, st.qnorm, st.cbf, nq, ns, chunk1,
                                                        kSeedSample, W, stride, Wc, nullptr, 0,
                                                        st.t0, st.part);
        else
            k_seed_mma<2><<<grid1, 128, 0, c->stream>>>(st.qbf, st.qnorm, st.cbf, nq, ns, chunk1,
                                                        kSeedSample, W, stride, Wc, nullptr, 0,
                                                        st.t0, st.part);
        s = check_launch(c, "k_seed_scan");
        if (s) return s;
    }
    int nchunks, chunk;
    if (c->seed_tc) {
        // full pass on tcgen05: 128-row tiles of queries and candidates
        const int K = c->C == 1 ? 16 : 32, DH2 = 9 * c->C;
        const int nq_t = (nq + kTcRows - 1) / kTcRows;
        const int nc_pad = (ncand + kTcRows - 1) / kTcRows * kTcRows;
        prof_begin(c, "k_seed_prep");
        if (K == 16) {
            k_seed_tile<16><<<(nq_t * kTcRows * 2 + 255) / 256, 256, 0, c->stream>>>(st.qbf, nq, -1,
                                                                                 st.qtile);
        } else {
            k_seed_tile<32><<<(nq_t * kTcRows * 4 + 255) / 256, 256, 0, c->stream>>>(st.qbf, nq, -1,
                                                                                 st.qtile);
        }
        if ((s = check_launch(c, "k_seed_prep"))) return s;
        prof_begin(c, "k_seed_prep");
        if (K == 16)
            k_seed_tile<16><<<(nc_pad * 2 + 255) / 256, 256, 0, c->stream>>>(st.cbf, ncand, DH2,
                                                                          st.ctile);
        else
            k_seed_tile<32><<<(nc_pad * 4 + 255) / 256, 256, 0, c->stream>>>(st.cbf, ncand, DH2,
                                                                          st.ctile);
        if ((s = check_launch(c, "k_seed_prep"))) return s;
        // one wave of two CTAs per SM (tensor memory holds two): split the
        // candidates into 128-aligned chunks
        int nc = (2 * c->sms) / nq_t;
        nc = nc < 1 ? 1 : (nc > kMaxChunks / 2 ? kMaxChunks / 2 : nc);
        chunk = (ncand + nc - 1) / nc;
        chunk = (chunk + kTcRows - 1) / kTcRows * kTcRows;
        nchunks = (ncand + chunk - 1) / chunk;
        prof_begin(c, "k_seed_scan");
        if (c->C == 1)
            k_seed_tc<1><<<dim3(nq_t, nchunks), 320, tc_seed_smem_bytes<1>(), c->stream>>>(
                st.qtile, st.qnorm, st.ctile, nq, ncand, chunk, W, stride, Wc, st.t0, nchunks1,
                st.part, st.err, c->wait_ns);
        else
            k_seed_tc<2><<<dim3(nq_t, nchunks), 320, tc_seed_smem_bytes<2>(), c->stream>>>(
                st.qtile, st.qnorm, st.ctile, nq, ncand, chunk, W, stride, Wc, st.t0, nchunks1,
                st.part, st.err, c->wait_ns);
        if ((s = check_launch(c, "k_seed_scan"))) return s;
        nchunks *= 2;   // two lists per chunk
    } else {
        seed_geometry_mma(nq, ncand, c->sms, &nchunks, &chunk);
        dim3 grid((nq + 63) / 64, nchunks);
        prof_begin(c, "k_seed_scan");
        if (c->C == 1)
            k_seed_mma<1><<<grid, 128, 0, c->stream>>>(st.qbf, st.qnorm, st.cbf, nq, ncand, chunk,
                                                       1, W, stride, Wc, st.t0, nchunks1, nullptr,
                                                       st.part);
        else
            k_seed_mma<2><<<grid, 128, 0, c->stream>>>(st.qbf, st.qnorm, st.cbf, nq, ncand, chunk,
                                                       1, W, stride, Wc, st.t0, nchunks1, nullptr,
                                                       st.part);
        if ((s = check_launch(c, "k_seed_scan"))) return s;
    }
    prof_begin(c, "k_seed_merge");
    k_seed_merge<<<(nq + 127) / 128, 128, 0, c->stream>>>(st.part, nchunks, nq, c->cfg.seed_leaf,
                                                         st.knn_idx, st.knn_dist);
    return check_launch(c, "k_seed_merge");
}

// Sweep schedule of one level (Sec. 3.1-3.2 basic; Sec. 3.3 Flow Fields+:
// 4 sweeps with 2R then 8 with R, a random search after every sweep of a
// phase but its last; Sec. 3.4 Fast: the finest scale runs 4 sweeps with R).
bool plus_level(const ff_config &cfg, int L) {
    return cfg.schedule == FF_SCHED_PLUS || (cfg.schedule == FF_SCHED_PLUS_FAST && L > 0) ||
           (cfg.schedule == FF_SCHED_PLUS_FAST_X2 && L > 1);
}
// Fast x2 (Sec. 3.4) never runs the finest scale: its matches are the
// 2nd-finest scale's, one per 2x2 region
int final_level(const ff_config &cfg) { return cfg.schedule == FF_SCHED_PLUS_FAST_X2 ? 1 : 0; }
int level_sweeps(const ff_config &cfg, int L) {
    if (plus_level(cfg, L)) return 12;
    if (L < final_level(cfg)) return 0;
    if (cfg.schedule == FF_SCHED_PLUS_FAST || cfg.schedule == FF_SCHED_PLUS_FAST_X2) return 4;
    return cfg.iters;
}
bool search_after(const ff_config &cfg, int L, int t) {
    const int n = level_sweeps(cfg, L);
    if (plus_level(cfg, L)) return t != 3 && t != n - 1;
    return t < n - 1;
}
int search_radius(const ff_config &cfg, int L, int t) {
    return (plus_level(cfg, L) && t < 4) ? 2 * cfg.radius_q3 : cfg.radius_q3;
}

ff_status launch_sweep(ff_ctx *c, int d, const uint8_t *f1L, const uint8_t *f2L, uint32_t *flow,
                       int *cost, int W, int H, int L, int t, uint32_t pair_id) {
    DirState &st = c->dir[d];
    int WL, HL;
    level_dims(W, H, L, &WL, &HL);
    SweepArgs a;
    a.f1L = f1L;
    a.f2L = f2L;
    a.flow = flow;
    a.cost = cost;
    a.edge = st.edge;
    a.ticket = st.ticket + (size_t)L * kMaxIters + t;
    a.err = st.err;
    a.W = W;
    a.H = H;
    a.L = L;
    a.WL = WL;
    a.HL = HL;
    a.d = t & 3;
    a.t = t;
    a.dir = d;
    a.do_rs = search_after(c->cfg, L, t) ? 1 : 0;
    a.radius_q3 = search_radius(c->cfg, L, t);
    a.seed = c->cfg.seed;
    a.pair_id = pair_id;
    // boundary-row tags: unique per (level, sweep) within a match (the rows
    // are cleared when a match starts), never 0, below bit 31; the same in
    // every replay of a captured graph
    a.epoch = 1u + (uint32_t)(L * kMaxIters + t);
    a.wait_ns = c->wait_ns;
    a.force_timeout = c->force_timeout;
    const int R = rows_per_strip(c->sweep_lanes);
    const int nstrips = (HL + R - 1) / R;
    prof_begin(c, "k_sweep");
#define FF_LAUNCH_SWEEP(CC, LPC) \
    k_sweep<CC, LPC><<<nstrips, SweepGeo<CC, LPC>::THREADS, 0, c->stream>>>(a)
    if (c->C == 1) {
        if (c->sweep_lanes == 2)
            k_sweep_many<1><<<nstrips, SweepGeo<1, 1>::THREADS, 0, c->stream>>>(a);
        else if (c->sweep_lanes == 8) FF_LAUNCH_SWEEP(1, 4);
        else FF_LAUNCH_SWEEP(1, 2);
    } else {
        if (c->sweep_lanes == 2)
            k_sweep_many<3><<<nstrips, SweepGeo<3, 1>::THREADS, 0, c->stream>>>(a);
        else if (c->sweep_lanes == 8) FF_LAUNCH_SWEEP(3, 4);
        else FF_LAUNCH_SWEEP(3, 2);
    }
#undef FF_LAUNCH_SWEEP
    return check_launch(c, "k_sweep");
}

template <int C>
void launch_rerank(ff_ctx *c, int d, const uint8_t *f1L, const uint8_t *f2L, int W, int H, int L,
                   int WL, int HL, uint32_t *flow, int *cost) {
    const int nq = WL * HL;
    prof_begin(c, "k_seed_rerank");
    k_seed_rerank<C><<<(nq + 127) / 128, 128, 0, c->stream>>>(
        c->dir[d].knn_idx, c->cfg.seed_leaf, f1L, f2L, W, H, L, WL, HL, flow, cost);
}

template <int C>
void launch_given(ff_ctx *c, const uint32_t *seeds, const uint8_t *f1L, const uint8_t *f2L, int W,
                  int H, int L, int WL, int HL, uint32_t *flow, int *cost) {
    const int nq = WL * HL;
    prof_begin(c, "k_seed_given");
    k_seed_given<C><<<(nq + 127) / 128, 128, 0, c->stream>>>(seeds, f1L, f2L, W, H, L, WL, HL, flow,
                                                          cost);
}

template <int C>
void launch_upsample(ff_ctx *c, const uint32_t *pflow, int WP, const uint8_t *f1L,
                     const uint8_t *f2L, int W, int H, int L, int WL, int HL, uint32_t *flow,
                     int *cost) {
    const int nq = WL * HL;
    prof_begin(c, "k_upsample");
    k_upsample<C><<<(nq + 255) / 256, 256, 0, c->stream>>>(pflow, WP, f1L, f2L, W, H, L, WL, HL,
                                                        flow, cost);
}

ff_status check_pair(ff_ctx *c) {
    if (!c->have[0] || !c->have[1])
        return fail(c, FF_ESTATE, "both frames need features (ff_features slot 0 and 1)");
    if (c->fw[0] != c->fw[1] || c->fh[0] != c->fh[1])
        return fail(c, FF_ESTATE, "the two frames have different sizes");
    return FF_OK;
}

ff_status run_match(ff_ctx *c, ff_dir dir, uint32_t pair_id, const int16_t *seeds_in,
                    int until_level, int until_sweeps, int16_t *flow_out, int32_t *cost_out) {
    ff_status s = check_pair(c);
    if (s) return s;
    if (dir != FF_FWD && dir != FF_BWD && dir != FF_BWD2)
        return fail(c, FF_EINVAL, "dir must be FF_FWD, FF_BWD or FF_BWD2");
    if (until_level < final_level(c->cfg) || until_level >= c->S || until_sweeps < 0 ||
        until_sweeps > level_sweeps(c->cfg, until_level))
        return fail(c, FF_EINVAL, "until_level/until_sweeps out of range");
    if (!flow_out) return fail(c, FF_EINVAL, "flow_out is NULL");
    if (((uintptr_t)flow_out & 3) || ((uintptr_t)cost_out & 3) || ((uintptr_t)seeds_in & 3))
        return fail(c, FF_EINVAL, "flow_out, cost_out and seeds_in must be 4-byte aligned");
    const int d = (int)dir;
    const int W = c->fw[0], H = c->fh[0];
    const uint8_t *fsrc = c->feat[d == 0 ? 0 : 1];
    const uint8_t *fdst = c->feat[d == 0 ? 1 : 0];
    DirState &st = c->dir[d];
    s = check_cuda(c, cudaMemsetAsync(st.ticket, 0, sizeof(unsigned) * FF_MAX_SCALES * kMaxIters,
                                      c->stream),
                   "memset tickets");
    if (s) return s;
    s = check_cuda(c, cudaMemsetAsync(st.edge, 0, c->edge_cap * sizeof(unsigned long long),
                                      c->stream),
                   "clear boundary rows");
    if (s) return s;
    int cur = 0, WP = 0;
    for (int L = c->S - 1; L >= until_level; L--) {
        int WL, HL;
        level_dims(W, H, L, &WL, &HL);
        const size_t off = level_offset(W, H, c->P, L);
        const uint8_t *f1L = fsrc + off, *f2L = fdst + off;
        uint32_t *flow = st.flow[cur];
        int *cost = st.cost[cur];
        if (L == c->S - 1) {
            if (seeds_in) {
                if (c->C == 1)
                    launch_given<1>(c, (const uint32_t *)seeds_in, f1L, f2L, W, H, L, WL, HL, flow,
                                    cost);
                else
                    launch_given<3>(c, (const uint32_t *)seeds_in, f1L, f2L, W, H, L, WL, HL, flow,
                                    cost);
                s = check_launch(c, "k_seed_given");
            } else {
                s = launch_seed_knn(c, d, fsrc, fdst, W, H);
                if (s) return s;
                if (c->C == 1)
                    launch_rerank<1>(c, d, f1L, f2L, W, H, L, WL, HL, flow, cost);
                else
                    launch_rerank<3>(c, d, f1L, f2L, W, H, L, WL, HL, flow, cost);
                s = check_launch(c, "k_seed_rerank");
            }
        } else {
            if (c->C == 1)
                launch_upsample<1>(c, st.flow[cur ^ 1], WP, f1L, f2L, W, H, L, WL, HL, flow, cost);
            else
                launch_upsample<3>(c, st.flow[cur ^ 1], WP, f1L, f2L, W, H, L, WL, HL, flow, cost);
            s = check_launch(c, "k_upsample");
        }
        if (s) return s;
        const int sweeps = (L == until_level) ? until_sweeps : level_sweeps(c->cfg, L);
        for (int t = 0; t < sweeps; t++) {
            s = launch_sweep(c, d, f1L, f2L, flow, cost, W, H, L, t, pair_id);
            if (s) return s;
        }
        WP = WL;
        if (L > until_level) cur ^= 1;
    }
    int WL, HL;
    level_dims(W, H, until_level, &WL, &HL);
    const int N = WL * HL;
    prof_begin(c, "k_export");
    k_export<<<(N + 255) / 256, 256, 0, c->stream>>>(st.flow[cur], st.cost[cur], N,
                                                     (uint32_t *)flow_out, (int *)cost_out);
    return check_launch(c, "k_export");
}

ff_status filter_into(ff_ctx *c, const int16_t *fwd, const int16_t *b1, const int16_t *b2,
                      uint8_t *mask);
ff_status region_into(ff_ctx *c, const int16_t *fwd, const uint8_t *mask_in, int s,
                      uint8_t *mask_out);

// One whole pair on device buffers, enqueued without waiting: features on
// the context's stream, the backward flow(s) on the side stream(s)
// overlapping the forward flow, the filter after all of them.  The next
// work on the context's stream is ordered after every part.
ff_status enqueue_pair(ff_ctx *c, const uint8_t *img1, const uint8_t *img2, int w, int h,
                       int pitch, uint32_t pair_id, int16_t *fwd, int16_t *bwd, int16_t *bwd2,
                       uint8_t *mask) {
    const int Lf = final_level(c->cfg);
    const int n = level_sweeps(c->cfg, Lf);
    cudaStream_t main = c->stream;
    ff_status s;
    // the two frames' features on the two streams (the side stream starts
    // after what main holds so far), then each stream waits for the other's
    if ((s = check_cuda(c, cudaEventRecord(c->ev_a, main), "event"))) return s;
    if ((s = check_cuda(c, cudaStreamWaitEvent(c->side, c->ev_a, 0), "wait"))) return s;
    if ((s = ff_features(c, 0, img1, w, h, pitch))) return s;
    c->stream = c->side;
    s = ff_features(c, 1, img2, w, h, pitch);
    c->stream = main;
    if (s) return s;
    if ((s = check_cuda(c, cudaEventRecord(c->ev_a, main), "event"))) return s;
    if ((s = check_cuda(c, cudaEventRecord(c->ev_c, c->side), "event"))) return s;
    if ((s = check_cuda(c, cudaStreamWaitEvent(c->side, c->ev_a, 0), "wait"))) return s;
    if ((s = check_cuda(c, cudaStreamWaitEvent(main, c->ev_c, 0), "wait"))) return s;
    c->stream = c->side;
    s = run_match(c, FF_BWD, pair_id, nullptr, Lf, n, bwd, nullptr);
    c->stream = main;
    if (s) return s;
    if (bwd2) {
        if ((s = check_cuda(c, cudaStreamWaitEvent(c->side2, c->ev_a, 0), "wait"))) return s;
        if ((s = check_cuda(c, cudaStreamWaitEvent(c->side2, c->ev_c, 0), "wait"))) return s;
        c->stream = c->side2;
        s = run_match(c, FF_BWD2, pair_id, nullptr, Lf, n, bwd2, nullptr);
        c->stream = main;
        if (s) return s;
    }
    if ((s = run_match(c, FF_FWD, pair_id, nullptr, Lf, n, fwd, nullptr))) return s;
    if ((s = check_cuda(c, cudaEventRecord(c->ev_b, c->side), "event"))) return s;
    if ((s = check_cuda(c, cudaStreamWaitEvent(main, c->ev_b, 0), "wait"))) return s;
    if (bwd2) {
        if ((s = check_cuda(c, cudaEventRecord(c->ev_c, c->side2), "event"))) return s;
        if ((s = check_cuda(c, cudaStreamWaitEvent(main, c->ev_c, 0), "wait"))) return s;
    }
    if (!mask) return FF_OK;
    if ((s = filter_into(c, fwd, bwd, bwd2, mask))) return s;
    if (c->cfg.region_min > 0) return region_into(c, fwd, mask, c->cfg.region_min, mask);
    return FF_OK;
}

// reads and clears the context's device error words (after a synchronize)
ff_status take_error_words(ff_ctx *c) {
    int err[kNumDirs] = {0, 0, 0};
    ff_status s;
    for (int d = 0; d < kNumDirs; d++)
        if ((s = check_cuda(c, cudaMemcpy(&err[d], c->dir[d].err, sizeof(int),
                                          cudaMemcpyDeviceToHost), "read error word")))
            return s;
    if (err[0] || err[1] || err[2]) {
        for (int d = 0; d < kNumDirs; d++) cudaMemset(c->dir[d].err, 0, sizeof(int));
        cudaDeviceSynchronize();
        return fail(c, FF_ETIMEOUT, "a bounded device wait expired during matching");
    }
    return FF_OK;
}

// Sec. 3.7 on the schedule's final grid, against one or two backward flows
ff_status filter_into(ff_ctx *c, const int16_t *fwd, const int16_t *b1, const int16_t *b2,
                      uint8_t *mask) {
    const int Lf = final_level(c->cfg);
    int W, H;
    level_dims(c->fw[0], c->fh[0], Lf, &W, &H);
    const int N = W * H;
    prof_begin(c, "k_filter");
    if (b2)
        k_filter<2><<<(N + 255) / 256, 256, 0, c->stream>>>(
            (const uint32_t *)fwd, (const uint32_t *)b1, (const uint32_t *)b2, W, H, Lf,
            c->cfg.eps_q3, mask);
    else
        k_filter<1><<<(N + 255) / 256, 256, 0, c->stream>>>(
            (const uint32_t *)fwd, (const uint32_t *)b1, nullptr, W, H, Lf, c->cfg.eps_q3, mask);
    return check_launch(c, "k_filter");
}

// Sec. 3.7 region filter on the final grid (mask_in may equal mask_out)
ff_status region_into(ff_ctx *c, const int16_t *fwd, const uint8_t *mask_in, int s,
                      uint8_t *mask_out) {
    const int Lf = final_level(c->cfg);
    int W, H;
    level_dims(c->fw[0], c->fh[0], Lf, &W, &H);
    const int N = W * H, nb = (N + 255) / 256;
    const uint32_t *f = (const uint32_t *)fwd;
    ff_status st;
    prof_begin(c, "k_region");
    k_rf_init<<<nb, 256, 0, c->stream>>>(mask_in, N, c->rf_parent, c->rf_size, c->rf_flag);
    if ((st = check_launch(c, "k_region"))) return st;
    prof_begin(c, "k_region");
    k_rf_union<<<nb, 256, 0, c->stream>>>(f, mask_in, W, H, c->rf_parent);
    if ((st = check_launch(c, "k_region"))) return st;
    prof_begin(c, "k_region");
    k_rf_count<<<nb, 256, 0, c->stream>>>(f, mask_in, W, H, c->rf_parent, c->rf_size, c->rf_flag);
    if ((st = check_launch(c, "k_region"))) return st;
    prof_begin(c, "k_region");
    k_rf_apply<<<nb, 256, 0, c->stream>>>(mask_in, N, s, c->rf_parent, c->rf_size, c->rf_flag,
                                          mask_out);
    return check_launch(c, "k_region");
}

}  // namespace

// ============================================================================
// allocation-free seeding search (ff_seed_knn_static)
// ============================================================================
namespace {

// Scratch of the allocation-free seeding search: the per-chunk partial top-8
// lists, 8 MiB.  It lives in this file's static device memory, so every GPU
// that loads the library holds it until the process exits.  Every call
// shares it; calls that overlap on a GPU race on it.
constexpr size_t kStaticScratchInt2 = (size_t)1 << 20;   // 8 MiB of int2
static __device__ __align__(256) int2 g_seed_scratch[kStaticScratchInt2];

// In host code g_seed_scratch names a host-side stand-in, not device memory:
// the kernels get the device address from cudaGetSymbolAddress, called with
// the device current.  The address is cached per CUDA context, keyed by the
// context's process-unique id (cuCtxGetId), so a context that is torn down
// and created again (cudaDeviceReset, a released primary context) gets a
// fresh lookup instead of a stale address.  Where the driver does not offer
// those entry points the address is looked up on every call.
typedef CUresult (*PfnCtxGetCurrent)(CUcontext *);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long *);

struct ScratchEntry {
    int device;
    unsigned long long ctx_id;
    int2 *ptr;
};
std::mutex g_scratch_mutex;
ScratchEntry g_scratch_cache[64];
int g_scratch_entries = 0;
bool g_ctx_api_tried = false;
PfnCtxGetCurrent g_ctx_get_current = nullptr;
PfnCtxGetId g_ctx_get_id = nullptr;

void load_ctx_api() {
    if (g_ctx_api_tried) return;
    g_ctx_api_tried = true;
    void *f1 = nullptr, *f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) ==
            cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) ==
            cudaSuccess &&
        q2 == cudaDriverEntryPointSuccess) {
        g_ctx_get_current = (PfnCtxGetCurrent)f1;
        g_ctx_get_id = (PfnCtxGetId)f2;
    }
}

// id of the calling thread's current context, 0 if there is none or it
// cannot be read
unsigned long long current_ctx_id() {
    if (!g_ctx_get_current || !g_ctx_get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
    if (g_ctx_get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

cudaError_t static_scratch(int device, int2 **out) {
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    load_ctx_api();
    const unsigned long long id = current_ctx_id();
    if (id != 0)
        for (int i = 0; i < g_scratch_entries; i++)
            if (g_scratch_cache[i].device == device && g_scratch_cache[i].ctx_id == id) {
                *out = g_scratch_cache[i].ptr;
                return cudaSuccess;
            }
    void *ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_seed_scratch);
    if (e != cudaSuccess) return e;
    *out = (int2 *)ptr;
    // the lookup makes the device's primary context current if none was
    const unsigned long long id2 = id != 0 ? id : current_ctx_id();
    if (id2 != 0) {
        int slot = -1;
        for (int i = 0; i < g_scratch_entries; i++)
            if (g_scratch_cache[i].device == device) slot = i;   // replaces a torn-down context's
        if (slot < 0) slot = g_scratch_entries < 64 ? g_scratch_entries++ : device & 63;
        g_scratch_cache[slot] = {device, id2, (int2 *)ptr};
    }
    return cudaSuccess;
}

}  // namespace

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

ff_status ff_config_default(ff_config *cfg) {
    if (!cfg) return FF_EINVAL;
    memset(cfg, 0, sizeof(*cfg));
    cfg->patch = 8;
    cfg->n_coeffs = 9;
    cfg->channels = 1;
    cfg->scales = 4;
    cfg->iters = 4;
    cfg->radius_q3 = 8;
    cfg->seed_leaf = 8;
    cfg->seed_stride = 1;
    cfg->eps_q3 = 8;
    cfg->seed = 20261203u;
    cfg->max_width = 1024;
    cfg->max_height = 1024;
    cfg->schedule = FF_SCHED_BASIC;
    return FF_OK;
}

ff_status ff_create(const ff_config *cfg, int device, void *cuda_stream, ff_ctx **out) {
    if (!cfg || !out) return FF_EINVAL;
    *out = nullptr;
    std::string why;
    if (validate_config(cfg, &why) != FF_OK) return FF_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return FF_ECUDA;
    DeviceGuard guard(device);
    // the tensor-core seeding kernel takes more than 48 KB of shared memory
    if (cudaFuncSetAttribute(k_seed_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             tc_seed_smem_bytes<1>()) != cudaSuccess ||
        cudaFuncSetAttribute(k_seed_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             tc_seed_smem_bytes<2>()) != cudaSuccess) {
        cudaGetLastError();
        return FF_ECUDA;
    }
    ff_ctx *c = new ff_ctx();
    c->cfg = *cfg;
    c->device = device;
    if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return FF_ECUDA;
    }
    c->stream = (cudaStream_t)cuda_stream;
    c->C = cfg->channels;
    c->P = cfg->channels == 1 ? 16 : 32;
    c->sweep_lanes = 4;   // the shortest step chain, for one pair at a time
    c->S = cfg->scales;
    c->I = cfg->iters;
    c->maxW = cfg->max_width;
    c->maxH = cfg->max_height;
    c->feat_cap = level_offset(c->maxW, c->maxH, c->P, c->S);
    int WS, HS;
    level_dims(c->maxW, c->maxH, c->S - 1, &WS, &HS);
    c->nq_cap = (size_t)WS * HS;
    const size_t npix = (size_t)c->maxW * c->maxH;
    const int R = rows_per_strip(8);   // the smallest strip
    c->edge_cap = (size_t)((c->maxH + R - 1) / R) * c->maxW;
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < 2 && e == cudaSuccess; s++) {
        e = alloc(&c->feat[s], c->feat_cap);
        if (e == cudaSuccess) e = alloc(&c->img_dev[s], npix * c->C);
        if (e == cudaSuccess) e = alloc(&c->pair_flow[s], npix);
        if (e == cudaSuccess && s == 1) e = alloc(&c->pair_flow[2], npix);
    }
    for (int s = 0; s < kNumDirs && e == cudaSuccess; s++) {
        DirState &d = c->dir[s];
        if (e == cudaSuccess) e = alloc(&d.flow[0], npix);
        if (e == cudaSuccess) e = alloc(&d.flow[1], npix);
        if (e == cudaSuccess) e = alloc(&d.cost[0], npix);
        if (e == cudaSuccess) e = alloc(&d.cost[1], npix);
        if (e == cudaSuccess) e = alloc(&d.edge, c->edge_cap);
        if (e == cudaSuccess) e = cudaMemset(d.edge, 0, c->edge_cap * sizeof(unsigned long long));
        if (e == cudaSuccess) e = alloc(&d.ticket, (size_t)FF_MAX_SCALES * kMaxIters);
        if (e == cudaSuccess) e = alloc(&d.knn_idx, c->nq_cap * FF_MAX_LEAF);
        if (e == cudaSuccess) e = alloc(&d.knn_dist, c->nq_cap * FF_MAX_LEAF);
        if (e == cudaSuccess) e = alloc(&d.part, c->nq_cap * kMaxChunks * 8);
        const size_t K = c->C == 1 ? 16 : 32;
        if (e == cudaSuccess) e = alloc(&d.qbf, c->nq_cap * K);
        if (e == cudaSuccess) e = alloc(&d.qnorm, c->nq_cap);
        if (e == cudaSuccess) e = alloc(&d.t0, c->nq_cap * kMaxChunks);
        if (e == cudaSuccess) e = alloc(&d.cbf, npix * K);
        const size_t pad = kTcRows;
        if (e == cudaSuccess) e = alloc(&d.qtile, (c->nq_cap + pad - 1) / pad * pad * K * 2);
        if (e == cudaSuccess) e = alloc(&d.ctile, (npix + pad - 1) / pad * pad * K * 2);
        if (e == cudaSuccess) e = alloc(&d.err, 1);
        if (e == cudaSuccess) e = cudaMemset(d.err, 0, sizeof(int));
    }
    if (e == cudaSuccess) e = alloc(&c->pair_mask, npix);
    if (e == cudaSuccess) e = alloc(&c->rf_parent, npix);
    if (e == cudaSuccess) e = alloc(&c->rf_size, npix);
    if (e == cudaSuccess) e = alloc(&c->rf_flag, npix);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->side2, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_a, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_b, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_c, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        const ff_status s = (e == cudaErrorMemoryAllocation) ? FF_ENOMEM : FF_ECUDA;
        free_all(c);
        delete c;
        cudaGetLastError();
        return s;
    }
    *out = c;
    return FF_OK;
}

ff_status ff_set_stream(ff_ctx *c, void *cuda_stream) {
    if (!c) return FF_EINVAL;
    c->stream = (cudaStream_t)cuda_stream;
    return FF_OK;
}

ff_status ff_features(ff_ctx *c, int slot, const uint8_t *img, int w, int h, int pitch) {
    if (!c) return FF_EINVAL;
    if (slot != 0 && slot != 1) return fail(c, FF_EINVAL, "slot must be 0 or 1");
    if (!img) return fail(c, FF_EINVAL, "img is NULL");
    if (w < 1 || h < 1 || w > c->maxW || h > c->maxH)
        return fail(c, FF_EINVAL, "frame size exceeds the context's max_width/max_height");
    if (pitch < w) return fail(c, FF_EINVAL, "pitch < width");
    DeviceGuard guard(c->device);
    c->have[slot] = false;
    if (c->cfg.wht_tensor_cores) {
        for (int L = 0; L < c->S; L++) {
            int WL, HL;
            level_dims(w, h, L, &WL, &HL);
            uint8_t *out = c->feat[slot] + level_offset(w, h, c->P, L);
            dim3 grid((WL + 15) / 16, (HL + 15) / 16);
            prof_begin(c, "k_features");
            if (c->C == 1)
                k_features_tc<1, false><<<grid, 128, 0, c->stream>>>(img, pitch, w, h, L, WL, HL,
                                                                     out, nullptr);
            else
                k_features_tc<3, false><<<grid, 128, 0, c->stream>>>(img, pitch, w, h, L, WL, HL,
                                                                     out, nullptr);
            ff_status s = check_launch(c, "k_features");
            if (s) return s;
        }
    } else {
        // every level in one launch, coarsest first
        FeatLevels lv{};
        lv.n = c->S;
        int blocks = 0;
        for (int k = 0; k < c->S; k++) {
            const int L = c->S - 1 - k;
            int WL, HL;
            level_dims(w, h, L, &WL, &HL);
            lv.L[k] = L;
            lv.WL[k] = WL;
            lv.HL[k] = HL;
            lv.tiles_x[k] = (WL + 15) / 16;
            lv.first[k] = blocks;
            lv.out[k] = c->feat[slot] + level_offset(w, h, c->P, L);
            blocks += lv.tiles_x[k] * ((HL + 15) / 16);
        }
        lv.first[c->S] = blocks;
        prof_begin(c, "k_features");
        if (c->C == 1)
            k_features<1><<<blocks, dim3(16, 16), 0, c->stream>>>(img, pitch, w, h, lv);
        else
            k_features<3><<<blocks, dim3(16, 16), 0, c->stream>>>(img, pitch, w, h, lv);
        ff_status s = check_launch(c, "k_features");
        if (s) return s;
    }
    c->fw[slot] = w;
    c->fh[slot] = h;
    c->have[slot] = true;
    return FF_OK;
}

ff_status ff_match(ff_ctx *c, ff_dir dir, uint32_t pair_id, const int16_t *seeds_in,
                   int16_t *flow_out, int32_t *cost_out) {
    if (!c) return FF_EINVAL;
    DeviceGuard guard(c->device);
    return run_match(c, dir, pair_id, seeds_in, final_level(c->cfg),
                     level_sweeps(c->cfg, final_level(c->cfg)), flow_out, cost_out);
}

ff_status ff_match_until(ff_ctx *c, ff_dir dir, uint32_t pair_id, const int16_t *seeds_in,
                         int until_level, int until_sweeps, int16_t *flow_out,
                         int32_t *cost_out) {
    if (!c) return FF_EINVAL;
    DeviceGuard guard(c->device);
    return run_match(c, dir, pair_id, seeds_in, until_level, until_sweeps, flow_out, cost_out);
}

ff_status ff_filter(ff_ctx *c, const int16_t *flow_fwd, const int16_t *flow_bwd,
                    uint8_t *mask_out) {
    if (!c) return FF_EINVAL;
    if (!flow_fwd || !flow_bwd || !mask_out) return fail(c, FF_EINVAL, "NULL argument");
    if (((uintptr_t)flow_fwd & 3) || ((uintptr_t)flow_bwd & 3))
        return fail(c, FF_EINVAL, "flows must be 4-byte aligned");
    ff_status s = check_pair(c);
    if (s) return s;
    DeviceGuard guard(c->device);
    return filter_into(c, flow_fwd, flow_bwd, nullptr, mask_out);
}

ff_status ff_filter_2way(ff_ctx *c, const int16_t *flow_fwd, const int16_t *flow_bwd1,
                         const int16_t *flow_bwd2, uint8_t *mask_out) {
    if (!c) return FF_EINVAL;
    if (!flow_fwd || !flow_bwd1 || !flow_bwd2 || !mask_out)
        return fail(c, FF_EINVAL, "NULL argument");
    if (((uintptr_t)flow_fwd & 3) || ((uintptr_t)flow_bwd1 & 3) || ((uintptr_t)flow_bwd2 & 3))
        return fail(c, FF_EINVAL, "flows must be 4-byte aligned");
    ff_status s = check_pair(c);
    if (s) return s;
    DeviceGuard guard(c->device);
    return filter_into(c, flow_fwd, flow_bwd1, flow_bwd2, mask_out);
}

ff_status ff_region_filter(ff_ctx *c, const int16_t *flow_fwd, const uint8_t *mask_in,
                           int min_region, uint8_t *mask_out) {
    if (!c) return FF_EINVAL;
    if (!flow_fwd || !mask_in || !mask_out) return fail(c, FF_EINVAL, "NULL argument");
    if ((uintptr_t)flow_fwd & 3) return fail(c, FF_EINVAL, "flow must be 4-byte aligned");
    if (min_region < 0) return fail(c, FF_EINVAL, "min_region < 0");
    ff_status s = check_pair(c);
    if (s) return s;
    DeviceGuard guard(c->device);
    return region_into(c, flow_fwd, mask_in, min_region, mask_out);
}

ff_status ff_wht_coeffs_tc(const uint8_t *img, int w, int h, int pitch, int channels, int level,
                           float *coeffs_out, void *cuda_stream) {
    if (!img || !coeffs_out) return FF_EINVAL;
    if (w < 1 || h < 1 || w > FF_MAX_DIM || h > FF_MAX_DIM || pitch < w) return FF_EINVAL;
    if ((channels != 1 && channels != 3) || level < 0 || level >= FF_MAX_SCALES) return FF_EINVAL;
    int WL, HL;
    level_dims(w, h, level, &WL, &HL);
    dim3 grid((WL + 15) / 16, (HL + 15) / 16);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (channels == 1)
        k_features_tc<1, true><<<grid, 128, 0, st>>>(img, pitch, w, h, level, WL, HL, nullptr,
                                                     coeffs_out);
    else
        k_features_tc<3, true><<<grid, 128, 0, st>>>(img, pitch, w, h, level, WL, HL, nullptr,
                                                     coeffs_out);
    return cudaGetLastError() == cudaSuccess ? FF_OK : FF_ECUDA;
}

ff_status ff_wht_coeffs_scalespace_tc(const uint8_t *img, int w, int h, int pitch, int channels,
                                      int level, int fp16, float *coeffs_out, void *cuda_stream) {
    if (!img || !coeffs_out) return FF_EINVAL;
    if (w < 1 || h < 1 || w > FF_MAX_DIM || h > FF_MAX_DIM || pitch < w) return FF_EINVAL;
    if ((channels != 1 && channels != 3) || level < 0 || level >= FF_MAX_SCALES) return FF_EINVAL;
    if (fp16 != 0 && fp16 != 1) return FF_EINVAL;
    int WL, HL;
    level_dims(w, h, level, &WL, &HL);
    dim3 grid((WL + 15) / 16, (HL + 15) / 16);
    cudaStream_t st = (cudaStream_t)cuda_stream;
#define FF_LAUNCH_TCS(CC, IN) \
    k_features_tc<CC, true, IN><<<grid, 128, 0, st>>>(img, pitch, w, h, level, WL, HL, nullptr, \
                                                      coeffs_out)
    if (channels == 1) {
        if (fp16) FF_LAUNCH_TCS(1, 2);
        else FF_LAUNCH_TCS(1, 1);
    } else {
        if (fp16) FF_LAUNCH_TCS(3, 2);
        else FF_LAUNCH_TCS(3, 1);
    }
#undef FF_LAUNCH_TCS
    return cudaGetLastError() == cudaSuccess ? FF_OK : FF_ECUDA;
}

ff_status ff_sparsify(ff_ctx *c, const int16_t *flow_fwd, const int16_t *flow_bwd1,
                      const int16_t *flow_bwd2, const uint8_t *mask_in, int q, int e,
                      uint8_t *mask_out) {
    if (!c) return FF_EINVAL;
    if (!flow_fwd || !flow_bwd1 || !mask_in || !mask_out)
        return fail(c, FF_EINVAL, "NULL argument");
    if (((uintptr_t)flow_fwd & 3) || ((uintptr_t)flow_bwd1 & 3) || ((uintptr_t)flow_bwd2 & 3))
        return fail(c, FF_EINVAL, "flows must be 4-byte aligned");
    if (q < 1 || q > 64 || e < 0) return fail(c, FF_EINVAL, "q must be 1..64 and e >= 0");
    ff_status s = check_pair(c);
    if (s) return s;
    DeviceGuard guard(c->device);
    const int Lf = final_level(c->cfg);
    int W, H;
    level_dims(c->fw[0], c->fh[0], Lf, &W, &H);
    const int cells_x = (W + q - 1) / q, ncells = cells_x * ((H + q - 1) / q);
    prof_begin(c, "k_sparsify");
    k_sparsify<<<(ncells + 127) / 128, 128, 0, c->stream>>>(
        (const uint32_t *)flow_fwd, (const uint32_t *)flow_bwd1, (const uint32_t *)flow_bwd2,
        mask_in, W, H, Lf, q, e, cells_x, ncells, mask_out);
    return check_launch(c, "k_sparsify");
}

ff_status ff_pair_host(ff_ctx *c, const uint8_t *img1_host, const uint8_t *img2_host, int w,
                       int h, uint32_t pair_id, int16_t *flow_fwd_host, int16_t *flow_bwd_host,
                       uint8_t *mask_host) {
    if (!c) return FF_EINVAL;
    if (!img1_host || !img2_host) return fail(c, FF_EINVAL, "NULL image");
    if (w < 1 || h < 1 || w > c->maxW || h > c->maxH)
        return fail(c, FF_EINVAL, "frame size exceeds the context's max_width/max_height");
    DeviceGuard guard(c->device);
    const size_t ibytes = (size_t)w * h * c->C;
    const int Lf = final_level(c->cfg);
    int WL, HL;
    level_dims(w, h, Lf, &WL, &HL);
    const size_t npix = (size_t)WL * HL;   // points of the final grid
    cudaStream_t main = c->stream;
    ff_status s;
    if ((s = check_cuda(c, cudaMemcpyAsync(c->img_dev[0], img1_host, ibytes,
                                           cudaMemcpyHostToDevice, main), "copy img1")))
        return s;
    if ((s = check_cuda(c, cudaMemcpyAsync(c->img_dev[1], img2_host, ibytes,
                                           cudaMemcpyHostToDevice, main), "copy img2")))
        return s;
    if ((s = enqueue_pair(c, c->img_dev[0], c->img_dev[1], w, h, w, pair_id,
                          (int16_t *)c->pair_flow[0], (int16_t *)c->pair_flow[1], nullptr,
                          c->pair_mask)))
        return s;
    if (flow_fwd_host &&
        (s = check_cuda(c, cudaMemcpyAsync(flow_fwd_host, c->pair_flow[0], npix * 4,
                                           cudaMemcpyDeviceToHost, main), "copy flow_fwd")))
        return s;
    if (flow_bwd_host &&
        (s = check_cuda(c, cudaMemcpyAsync(flow_bwd_host, c->pair_flow[1], npix * 4,
                                           cudaMemcpyDeviceToHost, main), "copy flow_bwd")))
        return s;
    if (mask_host &&
        (s = check_cuda(c, cudaMemcpyAsync(mask_host, c->pair_mask, npix, cudaMemcpyDeviceToHost,
                                           main), "copy mask")))
        return s;
    if ((s = check_cuda(c, cudaStreamSynchronize(main), "synchronize"))) return s;
    return take_error_words(c);
}

ff_status ff_get_features(ff_ctx *c, int slot, int level, int8_t *dst) {
    if (!c) return FF_EINVAL;
    if (slot != 0 && slot != 1) return fail(c, FF_EINVAL, "slot must be 0 or 1");
    if (level < 0 || level >= c->S) return fail(c, FF_EINVAL, "level out of range");
    if (!c->have[slot]) return fail(c, FF_ESTATE, "slot has no features");
    if (!dst) return fail(c, FF_EINVAL, "dst is NULL");
    DeviceGuard guard(c->device);
    int WL, HL;
    level_dims(c->fw[slot], c->fh[slot], level, &WL, &HL);
    const uint8_t *src = c->feat[slot] + level_offset(c->fw[slot], c->fh[slot], c->P, level);
    const int N = WL * HL;
    prof_begin(c, "k_dense");
    if (c->C == 1)
        k_dense<1><<<(N + 255) / 256, 256, 0, c->stream>>>(src, N, dst);
    else
        k_dense<3><<<(N + 255) / 256, 256, 0, c->stream>>>(src, N, dst);
    return check_launch(c, "k_dense");
}

ff_status ff_seed_knn(ff_ctx *c, ff_dir dir, int32_t *idx_out, int32_t *dist_out) {
    if (!c) return FF_EINVAL;
    ff_status s = check_pair(c);
    if (s) return s;
    if (dir != FF_FWD && dir != FF_BWD && dir != FF_BWD2)
        return fail(c, FF_EINVAL, "dir must be FF_FWD, FF_BWD or FF_BWD2");
    if (!idx_out || !dist_out) return fail(c, FF_EINVAL, "NULL output");
    DeviceGuard guard(c->device);
    const int d = (int)dir, W = c->fw[0], H = c->fh[0];
    s = launch_seed_knn(c, d, c->feat[d == 0 ? 0 : 1], c->feat[d == 0 ? 1 : 0], W, H);
    if (s) return s;
    int WS, HS;
    level_dims(W, H, c->S - 1, &WS, &HS);
    const size_t bytes = (size_t)WS * HS * c->cfg.seed_leaf * sizeof(int);
    if ((s = check_cuda(c, cudaMemcpyAsync(idx_out, c->dir[d].knn_idx, bytes,
                                           cudaMemcpyDeviceToDevice, c->stream), "copy knn")))
        return s;
    return check_cuda(c, cudaMemcpyAsync(dist_out, c->dir[d].knn_dist, bytes,
                                         cudaMemcpyDeviceToDevice, c->stream), "copy knn");
}

ff_status ff_seed_knn_static(const int8_t *feat_src0, const int8_t *feat_dst0, int w, int h,
                             int channels, int scales, int leaf, int stride, int32_t *idx_out,
                             int32_t *dist_out, void *cuda_stream, const char **why) {
    const char *dummy = nullptr;
    const char **msg = why ? why : &dummy;
    *msg = "";
    if (!feat_src0 || !feat_dst0 || !idx_out || !dist_out)
        return *msg = "a pointer argument is NULL", FF_EINVAL;
    if (channels != 1 && channels != 3) return *msg = "channels must be 1 or 3", FF_EINVAL;
    if (w < 1 || h < 1 || w > FF_MAX_DIM || h > FF_MAX_DIM)
        return *msg = "frame size must be 1..4096 in each direction", FF_EINVAL;
    if (scales < 1 || scales > FF_MAX_SCALES) return *msg = "scales must be 1..8", FF_EINVAL;
    if (leaf < 1 || leaf > FF_MAX_LEAF) return *msg = "leaf must be 1..8", FF_EINVAL;
    if (stride < 1 || stride > 64) return *msg = "stride must be 1..64", FF_EINVAL;
    if (((uintptr_t)feat_src0 & 15) || ((uintptr_t)feat_dst0 & 15))
        return *msg = "feature arrays must be 16-byte aligned", FF_EINVAL;
    if (((uintptr_t)idx_out & 3) || ((uintptr_t)dist_out & 3))
        return *msg = "outputs must be 4-byte aligned", FF_EINVAL;
    int WS, HS;
    level_dims(w, h, scales - 1, &WS, &HS);
    const size_t nq = (size_t)WS * HS;
    const size_t max_slots = kStaticScratchInt2 / 8;   // (chunk, query) lists that fit
    if (nq > max_slots)
        return *msg = "too many coarsest-grid points for the static scratch (limit 131072)",
               FF_EINVAL;
    // an error left pending by earlier work on this thread is reported as
    // such, not as this call's
    if (cudaPeekAtLastError() != cudaSuccess)
        return *msg = "a CUDA error from earlier work is pending; nothing launched", FF_ECUDA;
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    int2 *scratch = nullptr;
    if (e == cudaSuccess) e = static_scratch(device, &scratch);
    if (e != cudaSuccess) return *msg = "device set-up failed", FF_ECUDA;
    const int N = 1 << (scales - 1);
    const int Wc = (w + stride - 1) / stride, Hc = (h + stride - 1) / stride;
    const int ncand = Wc * Hc;
    int nchunks, chunk, sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return *msg = "device query failed", FF_ECUDA;
    seed_geometry((int)nq, ncand, sms, &nchunks, &chunk);
    const int cap = (int)(max_slots / nq);
    if (nchunks > cap) {
        chunk = (ncand + cap - 1) / cap;
        nchunks = (ncand + chunk - 1) / chunk;
    }
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    const uint8_t *fs = (const uint8_t *)feat_src0, *fd = (const uint8_t *)feat_dst0;
    dim3 grid((unsigned)((nq + kSeedQueriesPerCta - 1) / kSeedQueriesPerCta), nchunks);
    if (channels == 1)
        k_seed_scan<1, kSeedQpt><<<grid, 128, 0, stream>>>(fs, fd, w, N, WS, (int)nq, stride, Wc,
                                                          ncand, chunk, scratch);
    else
        k_seed_scan<3, kSeedQpt><<<grid, 128, 0, stream>>>(fs, fd, w, N, WS, (int)nq, stride, Wc,
                                                          ncand, chunk, scratch);
    if (cudaGetLastError() != cudaSuccess) return *msg = "k_seed_scan launch failed", FF_ECUDA;
    k_seed_merge<<<(unsigned)((nq + 127) / 128), 128, 0, stream>>>(scratch, nchunks, (int)nq, leaf,
                                                                  idx_out, dist_out);
    if (cudaGetLastError() != cudaSuccess) return *msg = "k_seed_merge launch failed", FF_ECUDA;
    return FF_OK;
}

ff_status ff_measure_peaks(int device, ff_peaks *out) {
    if (!out) return FF_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return FF_EINVAL;
    DeviceGuard guard(device);
    memset(out, 0, sizeof(*out));
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return FF_ECUDA;
    out->sm_count = sms;
    const int blocks = sms * 8;                          // 2048 threads per SM
    const size_t nthreads = (size_t)blocks * kPeakThreads;
    const size_t l2_bytes = (size_t)48 << 20;            // resident in the L2
    const uint32_t n_l1 = 1024, n_l2 = (uint32_t)(16u << 20) / 4;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    uint32_t *sink = nullptr, *chase1 = nullptr, *chase2 = nullptr;
    uint4 *l2buf = nullptr;
    double *lat = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMalloc((void **)&sink, nthreads * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc((void **)&l2buf, l2_bytes);
    if (e == cudaSuccess) e = cudaMalloc((void **)&chase1, n_l1 * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc((void **)&chase2, (size_t)n_l2 * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc((void **)&lat, 16 * sizeof(double));
    if (e == cudaSuccess) e = cudaMemsetAsync(l2buf, 1, l2_bytes, st);
    // times one launch (after an untimed one) in ms
    auto timed = [&](auto launch) -> float {
        float ms = 0.f;
        launch();
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        launch();
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        return ms;
    };
    if (e == cudaSuccess) {
        const int it_int = 65536, it_sad = 8192;
        const double n_int = (double)nthreads * it_int * kPeakChains;
        const float t_dp4a = timed([&] { k_peak_int<0><<<blocks, kPeakThreads, 0, st>>>(sink, it_int, 7u); });
        const float t_add = timed([&] { k_peak_int<1><<<blocks, kPeakThreads, 0, st>>>(sink, it_int, 7u); });
        const float t_mad = timed([&] { k_peak_int<2><<<blocks, kPeakThreads, 0, st>>>(sink, it_int, 7u); });
        const float t_sad = timed([&] { k_peak_sad<<<blocks, kPeakThreads, 0, st>>>(sink, it_sad, 7u); });
        const int passes = 20;
        const float t_l2 = timed([&] {
            k_peak_l2<<<blocks, kPeakThreads, 0, st>>>(l2buf, l2_bytes / 16, passes, sink);
        });
        if (e == cudaSuccess) {
            out->dp4a_per_s = n_int / (t_dp4a * 1e-3);
            out->iadd3_per_s = n_int / (t_add * 1e-3);
            out->imad_per_s = n_int / (t_mad * 1e-3);
            out->sad_dims_per_s = (double)nthreads * it_sad * kPeakChains * 4 / (t_sad * 1e-3);
            out->l2_read_gbs = (double)l2_bytes * passes / (t_l2 * 1e-3) / 1e9;
        }
    }
    if (e == cudaSuccess) {
        // latency chains: a 4 KB cycle for L1 hits, a 16 MB cycle (warmed into L2) for L2 hits
        k_peak_chase_init<<<64, 256, 0, st>>>(chase1, n_l1, 33u);
        k_peak_chase_init<<<sms * 4, 256, 0, st>>>(chase2, n_l2, 4099u);
        k_peak_l2<<<blocks, kPeakThreads, 0, st>>>((const uint4 *)chase2, (size_t)n_l2 / 4, 2, sink);
        k_peak_latency<<<1, 32, 0, st>>>(chase1, chase2, 4096, 7u, lat);
        e = cudaGetLastError();
        double h[16];
        if (e == cudaSuccess) e = cudaMemcpyAsync(h, lat, 9 * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) {
            out->lat_alu = h[0];
            out->lat_prmt = h[1];
            out->lat_dp4a = h[2];
            out->lat_shfl = h[3];
            out->lat_lds = h[4];
            out->lat_ldg_l1 = h[5];
            out->lat_ldg_l2 = h[6];
        }
    }
    cudaFree(lat);
    cudaFree(chase2);
    cudaFree(chase1);
    cudaFree(l2buf);
    cudaFree(sink);
    if (e1) cudaEventDestroy(e1);
    if (e0) cudaEventDestroy(e0);
    if (st) cudaStreamDestroy(st);
    return e == cudaSuccess ? FF_OK : FF_ECUDA;
}

ff_status ff_sync(ff_ctx *c) {
    if (!c) return FF_EINVAL;
    DeviceGuard guard(c->device);
    ff_status s = check_cuda(c, cudaDeviceSynchronize(), "synchronize");
    if (s) return s;
    return take_error_words(c);
}

ff_status ff_debug_set(ff_ctx *c, ff_debug_key key, long long value) {
    if (!c) return FF_EINVAL;
    switch (key) {
        case FF_DEBUG_WAIT_LIMIT_NS:
            if (value < 1000 || value > 60000000000LL)
                return fail(c, FF_EINVAL, "wait limit must be 1 us .. 60 s");
            c->wait_ns = (unsigned long long)value;
            return FF_OK;
        case FF_DEBUG_FORCE_TIMEOUT:
            c->force_timeout = value != 0;
            return FF_OK;
        case FF_DEBUG_SEED_TC:
            c->seed_tc = value != 0;
            return FF_OK;
        case FF_DEBUG_SWEEP_LANES:
            if (value != 2 && value != 4 && value != 8)
                return fail(c, FF_EINVAL, "sweep lanes per grid point must be 2, 4 or 8");
            c->sweep_lanes = (int)value;
            return FF_OK;
    }
    return fail(c, FF_EINVAL, "unknown debug key");
}

ff_status ff_profile(ff_ctx *c, int mode) {
    if (!c) return FF_EINVAL;
    if (mode != 0 && mode != FF_PROFILE_LAUNCHES && mode != FF_PROFILE_SWEEP_RUNS)
        return fail(c, FF_EINVAL, "profile mode must be 0, FF_PROFILE_LAUNCHES or "
                                  "FF_PROFILE_SWEEP_RUNS");
    DeviceGuard guard(c->device);
    while (!c->runs.empty()) close_run(c, 0);   // runs still open end here
    if (mode != 0) {
        c->ev_used = 0;
        c->prof.clear();
    }
    c->prof_mode = mode;
    c->pending_kernel = nullptr;
    return FF_OK;
}

ff_status ff_kernel_stats(ff_ctx *c, const char *kernel, long long *launches, double *total_ms) {
    if (!c || !kernel || !launches || !total_ms) return FF_EINVAL;
    const int id = kernel_id(kernel);
    if (id < 0) return fail(c, FF_EINVAL, std::string("unknown kernel ") + kernel);
    DeviceGuard guard(c->device);
    long long n = 0;
    double ms = 0.0;
    for (const auto &r : c->prof) {
        if (r.kernel != id) continue;
        float t = 0.f;
        const cudaError_t e = cudaEventElapsedTime(&t, c->ev_pool[r.ev0], c->ev_pool[r.ev1]);
        if (e != cudaSuccess) return check_cuda(c, e, "cudaEventElapsedTime");
        n += r.launches;
        ms += t;
    }
    *launches = n;
    *total_ms = ms;
    return FF_OK;
}

long long ff_launch_count(const ff_ctx *c) { return c ? c->launches : 0; }

const char *ff_last_error(const ff_ctx *c) { return c ? c->last_error.c_str() : "NULL context"; }

const char *ff_status_string(ff_status s) {
    switch (s) {
        case FF_OK: return "FF_OK";
        case FF_EINVAL: return "FF_EINVAL";
        case FF_ENOMEM: return "FF_ENOMEM";
        case FF_ECUDA: return "FF_ECUDA";
        case FF_ETIMEOUT: return "FF_ETIMEOUT";
        case FF_ESTATE: return "FF_ESTATE";
    }
    return "unknown status";
}

void ff_destroy(ff_ctx *c) {
    if (!c) return;
    {
        DeviceGuard guard(c->device);
        cudaDeviceSynchronize();
        free_all(c);
    }
    delete c;
}

}  // extern "C"

// ============================================================================
// batched form
// ============================================================================
struct ff_batch {
    ff_config cfg;
    int device = 0;
    cudaStream_t stream = nullptr;              // the caller's stream
    std::vector<ff_ctx *> slot;
    std::vector<cudaStream_t> slot_stream;      // one per slot, owned
    std::vector<cudaEvent_t> ev_join;           // one per slot
    cudaEvent_t ev_fork = nullptr;
    cudaStream_t capture = nullptr;             // graphs are captured here, owned
    // the last captured graph and the descriptors it was captured for
    cudaGraphExec_t exec = nullptr;
    std::vector<ff_pair_desc> exec_desc;
    long long exec_launches = 0;
    long long launches = 0;
    std::string last_error;
};

namespace {

ff_status bfail(ff_batch *b, ff_status s, const std::string &msg) {
    b->last_error = msg;
    return s;
}

void batch_free(ff_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (ff_ctx *c : b->slot) ff_destroy(c);
    for (cudaStream_t s : b->slot_stream)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->ev_join)
        if (e) cudaEventDestroy(e);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->capture) cudaStreamDestroy(b->capture);
}

long long slot_launches(const ff_batch *b) {
    long long n = 0;
    for (const ff_ctx *c : b->slot) n += c->launches;
    return n;
}

bool same_desc(const ff_pair_desc &x, const ff_pair_desc &y) {
    return x.img1 == y.img1 && x.img2 == y.img2 && x.w == y.w && x.h == y.h &&
           x.pitch == y.pitch && x.pair_id == y.pair_id && x.flow_fwd == y.flow_fwd &&
           x.flow_bwd == y.flow_bwd && x.flow_bwd2 == y.flow_bwd2 && x.mask == y.mask;
}

// fork from `origin` to the used slots, enqueue every pair on its slot,
// join back into `origin`
ff_status batch_enqueue(ff_batch *b, cudaStream_t origin, int n, const ff_pair_desc *pairs) {
    const int used = n < (int)b->slot.size() ? n : (int)b->slot.size();
    ff_status s;
    if (used == 0) return FF_OK;
    if ((s = check_cuda(b->slot[0], cudaEventRecord(b->ev_fork, origin), "event")))
        return bfail(b, s, b->slot[0]->last_error);
    for (int j = 0; j < used; j++)
        if ((s = check_cuda(b->slot[j], cudaStreamWaitEvent(b->slot_stream[j], b->ev_fork, 0),
                            "wait")))
            return bfail(b, s, b->slot[j]->last_error);
    for (int i = 0; i < n; i++) {
        const ff_pair_desc &p = pairs[i];
        ff_ctx *c = b->slot[i % used];
        if ((s = enqueue_pair(c, p.img1, p.img2, p.w, p.h, p.pitch, p.pair_id, p.flow_fwd,
                              p.flow_bwd, p.flow_bwd2, p.mask)))
            return bfail(b, s, "pair " + std::to_string(i) + ": " + c->last_error);
    }
    for (int j = 0; j < used; j++) {
        if ((s = check_cuda(b->slot[j], cudaEventRecord(b->ev_join[j], b->slot_stream[j]),
                            "event")))
            return bfail(b, s, b->slot[j]->last_error);
        if ((s = check_cuda(b->slot[j], cudaStreamWaitEvent(origin, b->ev_join[j], 0),
                            "wait")))
            return bfail(b, s, b->slot[j]->last_error);
    }
    return FF_OK;
}

}  // namespace

extern "C" {

ff_status ff_batch_create(const ff_config *cfg, int device, int slots, void *cuda_stream,
                          ff_batch **out) {
    if (!cfg || !out) return FF_EINVAL;
    *out = nullptr;
    if (slots < 1 || slots > 256) return FF_EINVAL;
    std::string why;
    if (validate_config(cfg, &why) != FF_OK) return FF_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return FF_ECUDA;
    DeviceGuard guard(device);
    ff_batch *b = new ff_batch();
    b->cfg = *cfg;
    b->device = device;
    b->stream = (cudaStream_t)cuda_stream;
    ff_status s = FF_OK;
    cudaError_t e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
    for (int i = 0; i < slots && e == cudaSuccess && s == FF_OK; i++) {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        b->slot_stream.push_back(st);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        b->ev_join.push_back(ev);
        if (e != cudaSuccess) break;
        ff_ctx *c = nullptr;
        s = ff_create(cfg, device, st, &c);
        if (s == FF_OK) {
            // many pairs in flight: one lane per candidate (16 rows per strip,
            // fewer instructions per grid point than the 4-lane layout)
            c->sweep_lanes = 2;
            b->slot.push_back(c);
        }
    }
    if (e != cudaSuccess || s != FF_OK) {
        batch_free(b);
        delete b;
        cudaGetLastError();
        return s != FF_OK ? s : (e == cudaErrorMemoryAllocation ? FF_ENOMEM : FF_ECUDA);
    }
    *out = b;
    return FF_OK;
}

ff_status ff_batch_run(ff_batch *b, int n, const ff_pair_desc *pairs, int use_graph) {
    if (!b) return FF_EINVAL;
    if (n < 0 || (n > 0 && !pairs)) return bfail(b, FF_EINVAL, "bad pair count or array");
    for (int i = 0; i < n; i++) {
        const ff_pair_desc &p = pairs[i];
        const std::string at = "pair " + std::to_string(i) + ": ";
        if (!p.img1 || !p.img2 || !p.flow_fwd || !p.flow_bwd)
            return bfail(b, FF_EINVAL, at + "NULL image or flow");
        if (p.w < 1 || p.h < 1 || p.w > b->cfg.max_width || p.h > b->cfg.max_height)
            return bfail(b, FF_EINVAL, at + "frame size exceeds max_width/max_height");
        if (p.pitch < p.w) return bfail(b, FF_EINVAL, at + "pitch < width");
        if (((uintptr_t)p.flow_fwd & 3) || ((uintptr_t)p.flow_bwd & 3) ||
            ((uintptr_t)p.flow_bwd2 & 3))
            return bfail(b, FF_EINVAL, at + "flows must be 4-byte aligned");
    }
    DeviceGuard guard(b->device);
    if (use_graph && b->exec && (int)b->exec_desc.size() == n) {
        bool same = true;
        for (int i = 0; i < n && same; i++) same = same_desc(b->exec_desc[i], pairs[i]);
        if (same) {
            const cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
            if (e != cudaSuccess)
                return bfail(b, FF_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
            b->launches += b->exec_launches;
            return FF_OK;
        }
    }
    const long long l0 = slot_launches(b);
    if (!use_graph) {
        const ff_status s = batch_enqueue(b, b->stream, n, pairs);
        b->launches += slot_launches(b) - l0;
        return s;
    }
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
        b->exec_desc.clear();
    }
    // captured on the batch's own stream (the caller's may be the legacy
    // default stream, which cannot be captured), launched into the caller's
    cudaError_t e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess)
        return bfail(b, FF_ECUDA, std::string("begin capture: ") + cudaGetErrorString(e));
    const ff_status s = batch_enqueue(b, b->capture, n, pairs);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(b->capture, &graph);
    if (s != FF_OK) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return s;
    }
    if (e != cudaSuccess)
        return bfail(b, FF_ECUDA, std::string("end capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        b->exec = nullptr;
        return bfail(b, FF_ECUDA, std::string("instantiate: ") + cudaGetErrorString(e));
    }
    b->exec_desc.assign(pairs, pairs + n);
    b->exec_launches = slot_launches(b) - l0;
    e = cudaGraphLaunch(b->exec, b->stream);
    if (e != cudaSuccess)
        return bfail(b, FF_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
    b->launches += b->exec_launches;
    return FF_OK;
}

ff_status ff_batch_set_stream(ff_batch *b, void *cuda_stream) {
    if (!b) return FF_EINVAL;
    b->stream = (cudaStream_t)cuda_stream;
    return FF_OK;
}

ff_status ff_batch_sync(ff_batch *b) {
    if (!b) return FF_EINVAL;
    DeviceGuard guard(b->device);
    const cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess)
        return bfail(b, FF_ECUDA, std::string("synchronize: ") + cudaGetErrorString(e));
    for (ff_ctx *c : b->slot) {
        const ff_status s = take_error_words(c);
        if (s) return bfail(b, s, c->last_error);
    }
    return FF_OK;
}

ff_status ff_batch_debug_set(ff_batch *b, ff_debug_key key, long long value) {
    if (!b) return FF_EINVAL;
    for (ff_ctx *c : b->slot) {
        const ff_status s = ff_debug_set(c, key, value);
        if (s) return bfail(b, s, c->last_error);
    }
    if (b->exec) {   // the captured graph holds the old launches
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
        b->exec_desc.clear();
    }
    return FF_OK;
}

long long ff_batch_launch_count(const ff_batch *b) { return b ? b->launches : 0; }

const char *ff_batch_last_error(const ff_batch *b) { return b ? b->last_error.c_str() : ""; }

void ff_batch_destroy(ff_batch *b) {
    if (!b) return;
    {
        DeviceGuard guard(b->device);
        cudaDeviceSynchronize();
        batch_free(b);
    }
    delete b;
}

}  // extern "C"

// ============================================================================
// serving loop
// ============================================================================
namespace {

struct ServerSlot {
    ff_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    int *err_host = nullptr;        // pinned: the three error words after the pair
    long long ticket = -1;          // -1: free
};

struct Pending {
    ff_host_pair p;
    long long ticket;
};

}  // namespace

struct ff_server {
    ff_config cfg;
    int device = 0;
    size_t slot_bytes = 0;
    std::vector<ServerSlot> slot;
    std::deque<Pending> queue;
    long long next_ticket = 0;
    long long launches = 0;
    std::string last_error;
};

namespace {

ff_status sfail(ff_server *v, ff_status s, const std::string &msg) {
    v->last_error = msg;
    return s;
}

// device bytes ff_create allocates for one context (and so one slot)
size_t context_bytes(const ff_config &cfg) {
    const int C = cfg.channels, P = C == 1 ? 16 : 32, K = C == 1 ? 16 : 32;
    const size_t npix = (size_t)cfg.max_width * cfg.max_height;
    int WS, HS;
    level_dims(cfg.max_width, cfg.max_height, cfg.scales - 1, &WS, &HS);
    const size_t nq = (size_t)WS * HS;
    (void)C;
    const int R = rows_per_strip(8);
    const size_t edge = (size_t)((cfg.max_height + R - 1) / R) * cfg.max_width;
    size_t b = 2 * level_offset(cfg.max_width, cfg.max_height, P, cfg.scales);   // features
    b += 2 * npix * C + 3 * npix * 4 + npix;                                    // staging
    b += npix * (4 + 4 + 1);                                                    // region scratch
    const size_t pad = kTcRows;
    const size_t dir = npix * 4 * 4 + edge * 8 + FF_MAX_SCALES * kMaxIters * 4 +
                       nq * FF_MAX_LEAF * 8 + nq * kMaxChunks * 8 * 8 + nq * K * 2 + nq * 4 +
                       nq * kMaxChunks * 4 + npix * K * 2 + 4 +
                       ((nq + pad - 1) / pad + (npix + pad - 1) / pad) * pad * K * 2;   // tiles
    return b + kNumDirs * dir;
}

// enqueue one request on a free slot: frames in, the pair, results out,
// error words out, completion event
ff_status server_start(ff_server *v, ServerSlot &sl, const Pending &q) {
    ff_ctx *c = sl.ctx;
    const ff_host_pair &p = q.p;
    const int C = c->C;
    ff_status s;
    for (int k = 0; k < C; k++) {
        if ((s = check_cuda(c, cudaMemcpy2DAsync(c->img_dev[0] + (size_t)k * p.w * p.h, p.w,
                                                 p.img1 + (size_t)k * p.plane, p.pitch, p.w, p.h,
                                                 cudaMemcpyHostToDevice, sl.stream),
                            "copy img1")))
            return s;
        if ((s = check_cuda(c, cudaMemcpy2DAsync(c->img_dev[1] + (size_t)k * p.w * p.h, p.w,
                                                 p.img2 + (size_t)k * p.plane, p.pitch, p.w, p.h,
                                                 cudaMemcpyHostToDevice, sl.stream),
                            "copy img2")))
            return s;
    }
    if ((s = enqueue_pair(c, c->img_dev[0], c->img_dev[1], p.w, p.h, p.w, p.pair_id,
                          (int16_t *)c->pair_flow[0], (int16_t *)c->pair_flow[1],
                          p.two_way ? (int16_t *)c->pair_flow[2] : nullptr, c->pair_mask)))
        return s;
    int WL, HL;
    level_dims(p.w, p.h, final_level(c->cfg), &WL, &HL);
    const size_t n = (size_t)WL * HL;
    const struct {
        void *dst;
        const void *src;
        size_t bytes;
    } out[4] = {{p.flow_fwd, c->pair_flow[0], n * 4},
                {p.flow_bwd, c->pair_flow[1], n * 4},
                {p.two_way ? p.flow_bwd2 : nullptr, c->pair_flow[2], n * 4},
                {p.mask, c->pair_mask, n}};
    for (const auto &o : out)
        if (o.dst && (s = check_cuda(c, cudaMemcpyAsync(o.dst, o.src, o.bytes,
                                                        cudaMemcpyDeviceToHost, sl.stream),
                                     "copy result")))
            return s;
    for (int d = 0; d < kNumDirs; d++)
        if ((s = check_cuda(c, cudaMemcpyAsync(sl.err_host + d, c->dir[d].err, sizeof(int),
                                               cudaMemcpyDeviceToHost, sl.stream),
                            "copy error word")))
            return s;
    if ((s = check_cuda(c, cudaEventRecord(sl.done, sl.stream), "event"))) return s;
    sl.ticket = q.ticket;
    return FF_OK;
}

// move queued requests into free slots, in arrival order
ff_status server_admit(ff_server *v) {
    for (ServerSlot &sl : v->slot) {
        if (v->queue.empty()) break;
        if (sl.ticket >= 0) continue;
        const long long l0 = sl.ctx->launches;
        const ff_status s = server_start(v, sl, v->queue.front());
        v->launches += sl.ctx->launches - l0;
        if (s) return sfail(v, s, sl.ctx->last_error);
        v->queue.pop_front();
    }
    return FF_OK;
}

void server_free(ff_server *v) {
    for (ServerSlot &sl : v->slot) {
        if (sl.ctx) ff_destroy(sl.ctx);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.err_host) cudaFreeHost(sl.err_host);
    }
}

}  // namespace

extern "C" {

size_t ff_slot_bytes(const ff_config *cfg) { return cfg ? context_bytes(*cfg) : 0; }

ff_status ff_server_create(const ff_config *cfg, int device, size_t mem_budget, int max_slots,
                           ff_server **out) {
    if (!cfg || !out) return FF_EINVAL;
    *out = nullptr;
    std::string why;
    if (validate_config(cfg, &why) != FF_OK || max_slots < 1 || max_slots > 1024)
        return FF_EINVAL;
    const size_t per = context_bytes(*cfg);
    size_t nslots = mem_budget / per;
    if (nslots < 1) return FF_ENOMEM;
    if (nslots > (size_t)max_slots) nslots = (size_t)max_slots;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return FF_ECUDA;
    DeviceGuard guard(device);
    ff_server *v = new ff_server();
    v->cfg = *cfg;
    v->device = device;
    v->slot_bytes = per;
    v->slot.resize(nslots);
    ff_status s = FF_OK;
    cudaError_t e = cudaSuccess;
    for (ServerSlot &sl : v->slot) {
        e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocHost((void **)&sl.err_host, kNumDirs * sizeof(int));
        if (e == cudaSuccess) s = ff_create(cfg, device, sl.stream, &sl.ctx);
        if (s == FF_OK && sl.ctx) sl.ctx->sweep_lanes = 2;   // as in ff_batch
        if (e != cudaSuccess || s != FF_OK) break;
    }
    if (e != cudaSuccess || s != FF_OK) {
        server_free(v);
        delete v;
        cudaGetLastError();
        return s != FF_OK ? s : (e == cudaErrorMemoryAllocation ? FF_ENOMEM : FF_ECUDA);
    }
    *out = v;
    return FF_OK;
}

int ff_server_slots(const ff_server *v) { return v ? (int)v->slot.size() : 0; }

ff_status ff_server_submit(ff_server *v, const ff_host_pair *p, long long *ticket) {
    if (!v) return FF_EINVAL;
    if (!p || !p->img1 || !p->img2) return sfail(v, FF_EINVAL, "NULL request or image");
    if (p->w < 1 || p->h < 1 || p->w > v->cfg.max_width || p->h > v->cfg.max_height)
        return sfail(v, FF_EINVAL, "frame size exceeds max_width/max_height");
    if (p->pitch < p->w || p->plane < (long long)(p->h - 1) * p->pitch + p->w)
        return sfail(v, FF_EINVAL, "pitch < width or plane too small");
    DeviceGuard guard(v->device);
    const long long t = v->next_ticket++;
    v->queue.push_back(Pending{*p, t});
    if (ticket) *ticket = t;
    return server_admit(v);
}

ff_status ff_server_poll(ff_server *v, long long *tickets, int *status, int cap, int *n_done) {
    if (!v || !n_done || cap < 0 || (cap > 0 && (!tickets || !status))) return FF_EINVAL;
    DeviceGuard guard(v->device);
    *n_done = 0;
    for (ServerSlot &sl : v->slot) {
        if (sl.ticket < 0 || *n_done >= cap) continue;
        const cudaError_t e = cudaEventQuery(sl.done);
        if (e == cudaErrorNotReady) continue;
        int st = FF_OK;
        if (e != cudaSuccess) {
            v->last_error = std::string("pair failed: ") + cudaGetErrorString(e);
            st = FF_ECUDA;
        } else if (sl.err_host[0] || sl.err_host[1] || sl.err_host[2]) {
            for (int d = 0; d < kNumDirs; d++)
                cudaMemsetAsync(sl.ctx->dir[d].err, 0, sizeof(int), sl.stream);
            v->last_error = "a bounded device wait expired during matching";
            st = FF_ETIMEOUT;
        }
        tickets[*n_done] = sl.ticket;
        status[*n_done] = st;
        (*n_done)++;
        sl.ticket = -1;
    }
    return server_admit(v);
}

int ff_server_pending(const ff_server *v) {
    if (!v) return 0;
    int n = (int)v->queue.size();
    for (const ServerSlot &sl : v->slot) n += sl.ticket >= 0;
    return n;
}

long long ff_server_launch_count(const ff_server *v) { return v ? v->launches : 0; }

const char *ff_server_last_error(const ff_server *v) { return v ? v->last_error.c_str() : ""; }

void ff_server_destroy(ff_server *v) {
    if (!v) return;
    {
        DeviceGuard guard(v->device);
        cudaDeviceSynchronize();
        server_free(v);
    }
    delete v;
}

}  // extern "C"
