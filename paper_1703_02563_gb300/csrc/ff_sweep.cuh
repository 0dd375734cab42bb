// ff_sweep.cuh - propagation sweep + random search kernel (arXiv 1703.02563,
// Sec. 3.1 Eq. 2 and the random search step; Sec. 3.2 for R_n = R n).
#pragma once
#include "ff_kernels.cuh"

namespace ffk {

struct SweepArgs {
    const uint8_t *f1L;
    const uint8_t *f2L;
    uint32_t *flow;                // level state, updated in place
    int *cost;
    unsigned long long *edge;      // [nstrips][WL] boundary rows: (epoch << 32) | flow
    unsigned int *ticket;          // strip counter of this launch (zeroed before)
    int *err;                      // error word of this direction
    int W, H, L, WL, HL;
    int d, t, dir, do_rs, radius_q3;
    uint32_t seed, pair_id, epoch;
    unsigned long long wait_ns;
    int force_timeout;
};

// Lane layout: G lanes per grid point, WPL 4-dimension feature words per
// lane; RW = 32/G rows per warp; NP propagation warps per strip, each paired
// with a helper warp and a warming warp; one loader warp.
template <int C, int NP_, int WPL_ = 2> struct SweepGeo {
    static constexpr int P = Geo<C>::P;
    static constexpr int WPL = WPL_;     // feature words per lane: 1, 2 or 4
    static constexpr int G = P / (4 * WPL);   // lanes per point
    static_assert(G >= 1 && G <= 32 && G * 4 * WPL == P, "lane layout");
    static constexpr int RW = 32 / G;    // rows per warp
    static constexpr int NP = NP_;       // propagation warps (and as many helpers)
    static constexpr int R = NP * RW;    // rows per strip
    static constexpr int DI = 16;        // staged-input ring depth (steps)
    static constexpr int DO = 16;        // result ring depth (steps)
    static constexpr int A = 8;          // staging distance (steps ahead)
    static constexpr int RING = 64;      // propagation warp -> warp ring
    static constexpr int LRING = 128;    // previous strip -> this strip ring
    static constexpr int NB = 8 / G;     // random-search offsets per lane per 8 steps
    static constexpr int PD = 1;         // L1 warming distance (level pixels)
    static constexpr int PF_COLS = 4;    // feature columns warmed from the target on
    static constexpr int PF_ROWS = WPL == 4 ? 4 : 6;   // feature rows warmed around the target
    static constexpr int THREADS = (3 * NP + 1) * 32;   // + loader, + NP warming warps
};

template <int WPL> struct QWords {
    uint32_t w[WPL];
};
template <> struct __align__(8) QWords<2> {
    uint32_t w[2];
};
template <> struct __align__(16) QWords<4> {
    uint32_t w[4];
};

template <int C, int NP, int WPL> struct SweepShared {
    using SG = SweepGeo<C, NP, WPL>;
    uint32_t in_flow[NP][SG::DI][SG::RW];
    int in_cost[NP][SG::DI][SG::RW];
    QWords<WPL> in_q[NP][SG::DI][32];
    unsigned long long out[NP][SG::DO][SG::RW];   // (tag:12 | cost:20) << 32 | flow
    unsigned long long ring[NP][SG::RING];        // (column + 1) << 32 | flow
    unsigned long long lring[SG::LRING];          // (column + 1) << 32 | flow
    int in_ready[NP], out_cons[NP], cons[NP];
    int lcons, abort, strip;
    uint32_t pf_sink[NP][32];                     // destination of L1-warming copies
};

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16ca(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ unsigned long long lds64(const unsigned long long *p) {
    return *(const volatile unsigned long long *)p;
}
__device__ __forceinline__ void sts64(unsigned long long *p, unsigned long long v) {
    *(volatile unsigned long long *)p = v;
}

__device__ __forceinline__ uint2 ldg64(const uint8_t *p) {
    return __ldg(reinterpret_cast<const uint2 *>(p));
}

// bilinear taps of a target already clamped into the frame (1/8 px, full res)
template <int P>
__device__ __forceinline__ Tap tap_at(int tx, int ty, int L, int WL, int HL) {
    const int half = (1 << L) >> 1;
    const int sx = (tx + half) >> L, sy = (ty + half) >> L;
    const int ix = sx >> 3, ax = sx & 7, iy = sy >> 3, ay = sy & 7;
    const int x0 = min(ix, WL - 1), x1 = min(ix + 1, WL - 1);
    const int y0 = min(iy, HL - 1), y1 = min(iy + 1, HL - 1);
    Tap t;
    t.o00 = (y0 * WL + x0) * P;
    t.o10 = (y0 * WL + x1) * P;
    t.o01 = (y1 * WL + x0) * P;
    t.o11 = (y1 * WL + x1) * P;
    t.w = (uint32_t)((8 - ax) * (8 - ay)) | ((uint32_t)(ax * (8 - ay)) << 8) |
          ((uint32_t)((8 - ax) * ay) << 16) | ((uint32_t)(ax * ay) << 24);
    return t;
}

// WPL words of one feature vector (dimensions 4 WPL g .. 4 WPL g + 4 WPL - 1)
template <int WPL>
__device__ __forceinline__ QWords<WPL> ldg_words(const uint8_t *p) {
    QWords<WPL> r;
    if constexpr (WPL == 4) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p));
        r.w[0] = v.x, r.w[1] = v.y, r.w[2] = v.z, r.w[3] = v.w;
    } else if constexpr (WPL == 2) {
        const uint2 v = __ldg(reinterpret_cast<const uint2 *>(p));
        r.w[0] = v.x, r.w[1] = v.y;
    } else {
        r.w[0] = __ldg(reinterpret_cast<const unsigned int *>(p));
    }
    return r;
}
// the same words staged in shared memory (written by cp.async, read volatile)
template <int WPL>
__device__ __forceinline__ QWords<WPL> lds_words(const QWords<WPL> *p) {
    QWords<WPL> r;
    if constexpr (WPL == 4) {
        uint32_t x, y, z, w;
        asm volatile("ld.volatile.shared.v4.u32 {%0,%1,%2,%3}, [%4];"
                     : "=r"(x), "=r"(y), "=r"(z), "=r"(w)
                     : "r"((unsigned)__cvta_generic_to_shared(p)));
        r.w[0] = x, r.w[1] = y, r.w[2] = z, r.w[3] = w;
    } else if constexpr (WPL == 2) {
        const unsigned long long v = *(const volatile unsigned long long *)p;
        r.w[0] = (uint32_t)v, r.w[1] = (uint32_t)(v >> 32);
    } else {
        r.w[0] = *(const volatile uint32_t *)p;
    }
    return r;
}
template <int WPL>
__device__ __forceinline__ void cp_async_words(QWords<WPL> *smem, const uint8_t *gmem) {
    if constexpr (WPL == 4) cp_async16ca(smem, gmem);
    else if constexpr (WPL == 2) cp_async8(smem, gmem);
    else cp_async4(smem, gmem);
}

// the 4 taps of one lane's WPL words
template <int WPL> struct Taps {
    QWords<WPL> t00, t10, t01, t11;
};
template <int WPL>
__device__ __forceinline__ Taps<WPL> load_taps(const uint8_t *f2L, const Tap &t, int g) {
    const uint8_t *b = f2L + 4 * WPL * g;
    Taps<WPL> r;
    r.t00 = ldg_words<WPL>(b + t.o00);
    r.t10 = ldg_words<WPL>(b + t.o10);
    r.t01 = ldg_words<WPL>(b + t.o01);
    r.t11 = ldg_words<WPL>(b + t.o11);
    return r;
}
// -64 x the query words, the seeds of the interpolation dot products
template <int WPL> struct NegQ {
    int4 na[WPL];
};
template <int WPL>
__device__ __forceinline__ NegQ<WPL> neg_query(const QWords<WPL> &q) {
    NegQ<WPL> r;
#pragma unroll
    for (int j = 0; j < WPL; j++) r.na[j] = neg64(q.w[j]);
    return r;
}
template <int WPL>
__device__ __forceinline__ int sad_words(const Taps<WPL> &x, uint32_t w, const NegQ<WPL> &nq) {
    int e = 0;
#pragma unroll
    for (int j = 0; j < WPL; j++)
        e += sad_word(x.t00.w[j], x.t10.w[j], x.t01.w[j], x.t11.w[j], w, nq.na[j]);
    return e;
}

// target (1/8 px) of flow f at grid point (px, py), clamped into the frame
__device__ __forceinline__ void target_of(uint32_t f, int px, int py, int W, int H, int &tx,
                                          int &ty) {
    tx = clampi(8 * px + flow_x(f), 0, 8 * (W - 1));
    ty = clampi(8 * py + flow_y(f), 0, 8 * (H - 1));
}

__device__ __forceinline__ unsigned long long pack_out(int tag, int cost, uint32_t flow) {
    const uint32_t c = cost == kCostInvalid ? 0xFFFFFu : (uint32_t)cost;
    return ((unsigned long long)(((uint32_t)(tag & 0xFFF) << 20) | c) << 32) | flow;
}

// Slow path of a warp-uniform wait: returns true when the warp must give up
// (the CTA's abort flag is up, or nothing changed for wait_ns, in which case
// the error word gets FF_ETIMEOUT and the abort flag is raised).  t0 == 0
// on the first call of a wait.
__device__ __forceinline__ bool wait_expired(unsigned long long &t0, unsigned long long wait_ns,
                                             volatile int *abort_flag, int *err) {
    const unsigned long long now = globaltimer_ns();
    if (t0 == 0) t0 = now;
    int stop = *abort_flag;
    if (!stop && now - t0 > wait_ns) {
        atomicCAS(err, 0, kErrTimeout);
        *abort_flag = 1;
        stop = 1;
    }
    return __any_sync(0xffffffffu, stop) != 0;
}

// One sweep in direction d, followed (when do_rs) by the random search.
//
// The sweep runs in its own frame (u, v): u follows the sweep's x order, v
// its y order, so every direction has sources (u-1, v) and (u, v-1) and a
// v-major raster order.  Point (u, v) depends only on those two sources, so
// the points of one anti-diagonal are independent, and the kernel reproduces
// the raster order exactly as a skewed wavefront: row r handles column
// u = i - (r mod RW) at local step i of its warp.
//
//  * A CTA owns a strip of R rows.  Each of its NP propagation warps owns RW
//    consecutive rows (G lanes per point, two feature words per lane) and does
//    only the dependent chain: sources -> candidate targets -> tap loads ->
//    SAD -> argmin -> hand-down.  Inside a warp the vertical source is the
//    previous step's result of the lane group above (a shuffle); between
//    warps it travels through a shared ring of tagged 64-bit slots, and
//    between strips through tagged 64-bit words in global memory that a
//    loader warp copies into a shared ring ahead of use.  A consumer polls
//    the slot's tag itself, so no fence or counter sits on the critical path.
//    Strips are handed out by a ticket counter, so a strip only waits on a
//    strip that is already running.
//  * Each propagation warp has a helper warp.  The helper stages the
//    pre-sweep state and the query words of every point into a shared ring A
//    steps ahead (cp.async), and, a few steps behind, takes each sweep
//    result, runs the random search of that point (Philox4x32-10, counter
//    (y*W + x, t, L, dir), key (seed, pair_id); accepted only if strictly
//    better) and writes the final flow and cost to memory.  Neighbours in
//    this sweep see only the sweep value, never the random-search result.
//  * Each propagation warp has a warming warp too.  It follows the result
//    slots and warms L1 with the feature sectors around the target of each
//    decided flow two points further on, where the next loads of that row
//    will most likely fall.
//  * A candidate equal to the current flow has exactly the cached cost, and
//    equal candidates have equal costs, so such evaluations are skipped
//    (warp-uniformly) without changing any result.
// Every wait is bounded and warp-uniform: a warp that sees no progress for
// wait_ns sets the error word to FF_ETIMEOUT, raises the CTA's abort flag and
// returns; every other wait in the CTA checks that flag on its slow path.
// DIR >= 0 fixes the direction at compile time (it must equal a.d); -1
// reads it from a.d.
template <int C, int NP, int WPL, int DIR = -1>
__global__ void __launch_bounds__(SweepGeo<C, NP, WPL>::THREADS) k_sweep(const SweepArgs a) {
    using SG = SweepGeo<C, NP, WPL>;
    constexpr int P = SG::P, G = SG::G, RW = SG::RW, R = SG::R;
    constexpr int DI = SG::DI, DO = SG::DO, A = SG::A, RING = SG::RING, LRING = SG::LRING;
    constexpr int NB = SG::NB, PD = SG::PD, PF_ROWS = SG::PF_ROWS;
    constexpr int PF_COLS = SG::PF_COLS;
    constexpr unsigned FULL = 0xffffffffu;
    __shared__ SweepShared<C, NP, WPL> sm;
    volatile int *v_in_ready = sm.in_ready;
    volatile int *v_out_cons = sm.out_cons;
    volatile int *v_cons = sm.cons;
    volatile int *v_lcons = &sm.lcons;
    volatile int *v_abort = &sm.abort;

    const int tid = threadIdx.x;
    const int U = a.WL, V = a.HL;
    const int nstrips = (V + R - 1) / R;
    if (tid == 0) {
        sm.strip = (int)atomicAdd(a.ticket, 1u);
        sm.lcons = 0;
        sm.abort = 0;
    }
    if (tid < NP) {
        sm.in_ready[tid] = 0;
        sm.out_cons[tid] = 0;
        sm.cons[tid] = 0;
    }
    // ring tags start at 0 (no column has tag 0); result slots at tag 0xFFF
    for (int j = tid; j < NP * RING; j += blockDim.x) (&sm.ring[0][0])[j] = 0ull;
    for (int j = tid; j < LRING; j += blockDim.x) sm.lring[j] = 0ull;
    for (int j = tid; j < NP * DO * RW; j += blockDim.x) (&sm.out[0][0][0])[j] = ~0ull;
    __syncthreads();
    const int strip = sm.strip;
    if (strip >= nstrips) return;
    const int v0 = strip * R;
    const int warp = tid >> 5, lane = tid & 31;

    if (warp == 2 * NP) {
        // ---------------- loader warp: previous strip's last row -> lring
        if (strip == 0) return;
        const unsigned long long *src = a.edge + (size_t)(strip - 1) * U;
        const uint32_t want = (a.force_timeout && strip == 1) ? (a.epoch ^ 0x80000000u) : a.epoch;
        int base = 0;
        unsigned long long t0 = globaltimer_ns();
        while (base < U) {
            const int col = base + lane;
            const int limit = *v_lcons + LRING;
            bool ready = col >= U;
            uint32_t val = 0;
            if (col < U && col < limit) {
                const unsigned long long e = ld_relaxed_u64(src + col);
                ready = (uint32_t)(e >> 32) == want;
                val = (uint32_t)e;
            }
            const unsigned m = __ballot_sync(FULL, ready);
            int nready = (m == FULL) ? 32 : (__ffs(~m) - 1);
            nready = min(nready, U - base);
            if (lane < nready)
                sts64(&sm.lring[col & (LRING - 1)], ((unsigned long long)(col + 1) << 32) | val);
            if (nready > 0) {
                base += nready;
                t0 = globaltimer_ns();
            } else {
                int stop = 0;
                if (lane == 0) {
                    const bool late = globaltimer_ns() - t0 > a.wait_ns;
                    if (late) atomicCAS(a.err, 0, kErrTimeout);
                    stop = late || *v_abort || ld_relaxed_i32(a.err) != 0;
                    if (stop) *v_abort = 1;
                }
                if (__shfl_sync(FULL, stop, 0)) return;
                __nanosleep(32);
            }
        }
        return;
    }

    const bool warmer = warp > 2 * NP;
    const bool helper = !warmer && warp >= NP;
    const int w = warmer ? warp - 2 * NP - 1 : (helper ? warp - NP : warp);
    if (v0 + w * RW >= V) return;                         // no valid row in this warp
    const int k = lane / G, g = lane - (lane / G) * G;
    const int r = w * RW + k, v = v0 + r;
    const bool row_ok = v < V;
    const int L = a.L, n = 1 << L, W = a.W, H = a.H;
    const int sd = DIR >= 0 ? DIR : a.d;
    const bool flipx = (sd == 1 || sd == 2), flipy = (sd == 1 || sd == 3);
    const int gy = row_ok ? (flipy ? V - 1 - v : v) : 0;
    const int py = gy * n;
    const int NS = U + RW - 1;                            // local steps of this warp
    const uint8_t *f1L = a.f1L, *f2L = a.f2L;
    const size_t rowbase = (size_t)gy * U;

    if (warmer) {
        // ================= warming warp =================
        // Warms L1 with the feature sectors its propagation warp will read two
        // points after each decision: rows iy-2 .. iy+3 around the target of
        // the decided flow at that point (a row per lane), columns ix ..
        // ix+PF_COLS-1, one sector (one point's feature vector) each, by
        // asynchronous 4-byte copies into a scratch word.  Features are read
        // in 32-byte sectors, so each step needs new ones; one step of lead
        // covers the L2 latency, and the nearer the point, the likelier the
        // decided flow is still the latest one (measured: 1 step and 4
        // columns beat 16 steps and 1 column by 18%).  It follows the tagged
        // result slots the propagation warp publishes every step, so the
        // propagation warp spends no instruction on it; a slot holding a
        // later step than expected (this warp fell a ring behind) is taken
        // as it is.
        const int sxdir = flipx ? -1 : 1;
        const int half = n >> 1;
        int i = 0;
        unsigned long long t0 = 0;
        while (i < NS) {
            const unsigned long long e = lds64(&sm.out[w][i & (DO - 1)][k]);
            const uint32_t d = ((uint32_t)(e >> 52) - (uint32_t)i) & 0xFFFu;   // its step - i
            if (!__all_sync(FULL, d < 0x800u)) {
                if (wait_expired(t0, a.wait_ns, v_abort, a.err)) break;
                continue;
            }
            t0 = 0;
            const int u = i + (int)d - k;                 // the point decided in that step
            const uint32_t f = (uint32_t)e;
            if (row_ok && u >= 0 && u < U && f != kFlowInvalid && g < PF_ROWS) {
                const int gx = flipx ? U - 1 - u : u;
                int tx, ty;
                target_of(f, (gx + sxdir * (PD + 1)) * n, py, W, H, tx, ty);
                const int ix = min((tx + half) >> (L + 3), U - 1);
                const int iy0 = ((ty + half) >> (L + 3)) - (PF_ROWS / 2 - 1);
#pragma unroll
                for (int rr = 0; rr < (PF_ROWS + G - 1) / G; rr++) {
                    const int row = g + rr * G;
                    if (row < PF_ROWS) {
                        const uint8_t *rowp = f2L + (size_t)clampi(iy0 + row, 0, V - 1) * U * P;
#pragma unroll
                        for (int cc = 0; cc < PF_COLS; cc++)
                            cp_async4(&sm.pf_sink[w][lane],
                                      rowp + (size_t)min(ix + cc, U - 1) * P);
                    }
                }
            }
            i += 1 + (int)__reduce_min_sync(FULL, d);
        }
        cp_async_commit();
        cp_async_wait<0>();
        return;
    }

    if (helper) {
        // ================= helper warp =================
        const int Rq = a.radius_q3 * n;
        const uint32_t span = 2u * (uint32_t)Rq + 1u;
        auto stage = [&](int j) {   // this row's point of local step j -> input ring
            const int uj = j - k;
            if (row_ok && uj >= 0 && uj < U) {
                const int gx = flipx ? U - 1 - uj : uj;
                const size_t pi = rowbase + gx;
                const int slot = j & (DI - 1);
                if (g == 0) cp_async4(&sm.in_flow[w][slot][k], a.flow + pi);
                if (g == G - 1) cp_async4(&sm.in_cost[w][slot][k], a.cost + pi);
                cp_async_words<WPL>(&sm.in_q[w][slot][lane], f1L + pi * P + 4 * WPL * g);
            }
        };
        for (int j = 0; j < A; j++) {
            stage(j);
            cp_async_commit();
        }
        cp_async_wait<0>();
        __threadfence_block();
        __syncwarp();
        if (lane == 0) v_in_ready[w] = A;
        int offs[NB];
#pragma unroll
        for (int j = 0; j < NB; j++) offs[j] = 0;
        for (int i = 0; i < NS; i++) {
            // stage step i + A; the inputs of steps < i + A - 2 are then complete
            stage(i + A);
            cp_async_commit();
            cp_async_wait<3>();
            __threadfence_block();
            __syncwarp();
            if (lane == 0) v_in_ready[w] = max(A, i + A - 2);
            // random-search offsets of this row's points of steps i .. i+7
            const int phase = i & 7;
            if (phase == 0 && a.do_rs) {
#pragma unroll
                for (int j = 0; j < NB; j++) {
                    const int up = i + g * NB + j - k;
                    const int gxp = flipx ? U - 1 - up : up;
                    const uint4 rnd = philox4x32_10(
                        make_uint4((uint32_t)(py * W + gxp * n), (uint32_t)a.t, (uint32_t)L,
                                   (uint32_t)a.dir),
                        a.seed, a.pair_id);
                    const int ox = (int)(rnd.x % span) - Rq, oy = (int)(rnd.y % span) - Rq;
                    offs[j] = (ox & 0xffff) | (oy << 16);
                }
            }
            // the propagation result of step i (tagged slot)
            const unsigned long long *oslot = &sm.out[w][i & (DO - 1)][k];
            unsigned long long e;
            unsigned long long t0 = 0;
            while (true) {
                e = lds64(oslot);
                const bool ok = (uint32_t)(e >> 52) == (uint32_t)(i & 0xFFF);
                if (__all_sync(FULL, ok)) break;
                if (wait_expired(t0, a.wait_ns, v_abort, a.err)) {
                    cp_async_wait<0>();
                    return;
                }
            }
            const QWords<WPL> q = lds_words<WPL>(&sm.in_q[w][i & (DI - 1)][lane]);
            __syncwarp();
            if (lane == 0) v_out_cons[w] = i + 1;
            const uint32_t best = (uint32_t)e;
            const uint32_t c20 = (uint32_t)(e >> 32) & 0xFFFFFu;
            const int bcost = c20 == 0xFFFFFu ? kCostInvalid : (int)c20;
            const int u = i - k;
            const bool valid = row_ok && u >= 0 && u < U;
            const int gx = flipx ? U - 1 - u : u;
            const int px = gx * n;
            uint32_t fflow = best;
            int fcost = bcost;
            if (a.do_rs) {
                int mine = offs[0];
#pragma unroll
                for (int j = 1; j < NB; j++)
                    if (phase % NB == j) mine = offs[j];
                const int off = __shfl_sync(FULL, mine, (lane & ~(G - 1)) + phase / NB);
                const int ox = (int)(int16_t)(off & 0xffff), oy = off >> 16;
                const int rtx = clampi(8 * px + flow_x(best) + ox, 0, 8 * (W - 1));
                const int rty = clampi(8 * py + flow_y(best) + oy, 0, 8 * (H - 1));
                const uint32_t cR = pack_flow(rtx - 8 * px, rty - 8 * py);
                const bool nR = valid && best != kFlowInvalid && cR != best;
                int er = 0;
                if (__any_sync(FULL, nR)) {
                    const Tap tR = tap_at<P>(rtx, rty, L, U, V);
                    er = sad_words<WPL>(load_taps<WPL>(f2L, tR, g), tR.w, neg_query<WPL>(q));
                }
#pragma unroll
                for (int o = G / 2; o > 0; o >>= 1) er += __shfl_xor_sync(FULL, er, o);
                if (nR && er < bcost) {
                    fflow = cR;
                    fcost = er;
                }
            }
            if (valid && g == 0) {
                a.flow[rowbase + gx] = fflow;
                a.cost[rowbase + gx] = fcost;
            }
        }
        cp_async_wait<0>();
        return;
    }

    // ================= propagation warp =================
    const bool ring_out = (w < NP - 1) && (v0 + (w + 1) * RW < V);
    const bool edge_out = (w == NP - 1) && (k == RW - 1) && (strip + 1 < nstrips);
    const bool top_src = (v0 + w * RW) > 0;     // group 0 has a row above it
    uint32_t last = kFlowInvalid;       // this row's sweep value at the previous step
    int ready = 0;                      // cached in_ready
    int ocons = 0;                      // cached out_cons
    int ncons = 0;                      // cached consumption of our ring by warp w + 1
    for (int i = 0; i < NS; i++) {
        const int u = i - k;
        const bool active = row_ok && u >= 0 && u < U;
        const int gx = flipx ? U - 1 - u : u;
        const int px = gx * n;
        const uint32_t above = __shfl_up_sync(FULL, last, G);
        // staged inputs of step i, and (group 0) the vertical source of column i
        const bool need_top = top_src && i < U && k == 0;
        const unsigned long long *tslot =
            (w > 0) ? &sm.ring[w - 1][i & (RING - 1)] : &sm.lring[i & (LRING - 1)];
        unsigned long long te = 0;
        unsigned long long t0 = 0;
        while (true) {
            if (ready <= i) ready = v_in_ready[w];
            bool ok = ready > i;
            if (need_top) {
                te = lds64(tslot);
                ok = ok && (uint32_t)(te >> 32) == (uint32_t)(i + 1);
            }
            if (__all_sync(FULL, ok)) break;
            if (wait_expired(t0, a.wait_ns, v_abort, a.err)) return;
        }
        if (need_top && g == 0) {
            if (w > 0)
                v_cons[w] = i + 1;
            else
                *v_lcons = i + 1;
        }
        uint32_t vflow = kFlowInvalid;
        if (active && v > 0) vflow = (k > 0) ? above : (uint32_t)te;
        const int islot = i & (DI - 1);
        uint32_t cur = kFlowInvalid;
        int ccost = kCostInvalid;
        if (active) {
            cur = ((volatile uint32_t *)sm.in_flow[w][islot])[k];
            ccost = ((volatile int *)sm.in_cost[w][islot])[k];
        }
        const QWords<WPL> q = lds_words<WPL>(&sm.in_q[w][islot][lane]);
        const uint32_t hflow = (active && u > 0) ? last : kFlowInvalid;
        const bool vv = vflow != kFlowInvalid, hv = hflow != kFlowInvalid;
        int vtx, vty, htx, hty;
        target_of(vflow, px, py, W, H, vtx, vty);
        target_of(hflow, px, py, W, H, htx, hty);
        const uint32_t cV = pack_flow(vtx - 8 * px, vty - 8 * py);
        const uint32_t cH = pack_flow(htx - 8 * px, hty - 8 * py);
        const bool nV = active && vv && cV != cur;
        const bool nH = active && hv && cH != cur && !(vv && cH == cV);
        // each candidate is evaluated when some row of the warp needs it
        const bool anyV = __any_sync(FULL, nV), anyH = __any_sync(FULL, nH);
        int ev = 0, eh = 0;
        if (anyV && anyH) {
            const Tap tV = tap_at<P>(vtx, vty, L, U, V), tH = tap_at<P>(htx, hty, L, U, V);
            const Taps<WPL> xV = load_taps<WPL>(f2L, tV, g), xH = load_taps<WPL>(f2L, tH, g);
            const NegQ<WPL> nq = neg_query<WPL>(q);
            ev = sad_words<WPL>(xV, tV.w, nq);
            eh = sad_words<WPL>(xH, tH.w, nq);
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) {
                ev += __shfl_xor_sync(FULL, ev, o);
                eh += __shfl_xor_sync(FULL, eh, o);
            }
        } else if (anyV || anyH) {
            const Tap t1 = anyV ? tap_at<P>(vtx, vty, L, U, V) : tap_at<P>(htx, hty, L, U, V);
            const Taps<WPL> x1 = load_taps<WPL>(f2L, t1, g);
            int e1 = sad_words<WPL>(x1, t1.w, neg_query<WPL>(q));
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) e1 += __shfl_xor_sync(FULL, e1, o);
            if (anyV)
                ev = e1;
            else
                eh = e1;
        }
        // [current, vertical, horizontal]: lowest cost, the later one on ties
        uint32_t best = cur;
        int bcost = ccost;
        const int EV = (cV == cur) ? ccost : ev;
        if (active && vv && EV <= bcost) {
            best = cV;
            bcost = EV;
        }
        const int EH = (cH == cur) ? ccost : ((vv && cH == cV) ? EV : eh);
        if (active && hv && EH <= bcost) {
            best = cH;
            bcost = EH;
        }
        if (active) last = best;
        // hand the last row's value down (next warp, next strip)
        if constexpr (NP > 1) {
            const bool pub = ring_out && active && k == RW - 1;
            if (__any_sync(FULL, pub && ncons <= u - RING)) {
                unsigned long long t1 = 0;
                while (true) {
                    if (pub && ncons <= u - RING) ncons = v_cons[w + 1];
                    if (__all_sync(FULL, !pub || ncons > u - RING)) break;
                    if (wait_expired(t1, a.wait_ns, v_abort, a.err)) return;
                }
            }
            if (pub && g == 0)
                sts64(&sm.ring[w][u & (RING - 1)], ((unsigned long long)(u + 1) << 32) | best);
        }
        if (edge_out && active && g == 0)
            st_relaxed_u64(a.edge + (size_t)strip * U + u,
                           ((unsigned long long)a.epoch << 32) | best);
        // result -> helper (tagged slot); room for the next 4 steps is checked
        // at once (ocons is warp-uniform: every lane loads the same word)
        if ((i & 3) == 0 && ocons <= i + 3 - DO) {
            unsigned long long t2 = 0;
            while (true) {
                ocons = v_out_cons[w];
                if (__all_sync(FULL, ocons > i + 3 - DO)) break;
                if (wait_expired(t2, a.wait_ns, v_abort, a.err)) return;
            }
        }
        if (g == 0) sts64(&sm.out[w][i & (DO - 1)][k], pack_out(i, bcost, best));
    }
}

}  // namespace ffk
