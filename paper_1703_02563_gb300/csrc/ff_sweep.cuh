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

// Geometry of a sweep CTA.  A CTA owns a strip of RW rows and has five warps:
// propagation (warp 0), random search (1), input stager (2), L1 warmer (3)
// and boundary-row loader (4), so the propagation warp shares its SM
// sub-partition only with the loader, which mostly sleeps.  The layout for
// many pairs in flight (LPC = 1) has no warmer (the loader is warp 3): with
// several CTAs per SM the warming copies cost more issue slots than the L1
// hits they buy (measured on the 32- and 64-pair batches).
//
// A grid point is handled by G = 2 LPC lanes of the propagation warp: lanes
// 0..LPC-1 evaluate the vertical candidate, lanes LPC..2 LPC-1 the horizontal
// one, each over WPC of the NWU feature words (4 dimensions each) that hold
// codes (7 for Lab, 3 for gray; the rest of the P bytes is zero on both
// sides, so a lane may include a padding word: it adds |0 - 0| = 0).
template <int C, int LPC> struct SweepGeo {
    static constexpr int P = Geo<C>::P;              // bytes per feature vector: 16, 32
    static constexpr int NW = P / 4;                 // words per feature vector: 4, 8
    static constexpr int NWU = C == 3 ? 7 : 3;       // words holding codes
    static constexpr int G = 2 * LPC;                // lanes per grid point
    static constexpr int RW = 32 / G;                // rows per strip
    static constexpr int WPC = (NWU + LPC - 1) / LPC;              // words per lane and candidate
    static constexpr int LWP = WPC <= 1 ? 1 : (WPC <= 2 ? 2 : (WPC <= 4 ? 4 : 8));  // words loaded
    static_assert(LPC * LWP <= NW || LPC == 1, "lane words");
    static constexpr int WPH = NW >= G ? NW / G : 1; // words per lane in the random search
    static constexpr int HL_ = NW / WPH;             // random-search lanes holding words
    static constexpr int QB = P / G >= 4 ? P / G : 4;  // query bytes a stager lane copies
    static constexpr int QL = P / QB;                // stager lanes holding query bytes
    // One lane per candidate is the layout for many pairs in flight: a
    // shorter input ring (8 steps, staged 4 ahead) and a register bound let
    // six CTAs share an SM, whose other CTAs hide the staging latency.
    static constexpr int DI = LPC == 1 ? 8 : 16;     // staged-input ring depth (steps)
    static constexpr int DO = 16;                    // result ring depth (steps)
    static constexpr int A = LPC == 1 ? 4 : 8;       // staging distance (steps ahead)
    static constexpr int MIN_CTAS = 8;               // CTAs per SM the registers allow (LPC 1)
    static constexpr bool WARM = LPC != 1;           // an L1-warming warp
    static constexpr int LOADER = WARM ? 4 : 3;      // the loader's warp
    static constexpr int LRING = 128;                // previous strip -> this strip ring
    static constexpr int NB = 8 / G;                 // random-search offsets per lane per 8 steps
    static constexpr int PD = 1;                     // L1 warming distance (level pixels)
    static constexpr int PF_COLS = 4;                // feature columns warmed from the target on
    static constexpr int PF_ROWS = LPC == 2 ? 6 : 4; // feature rows warmed around the target
    // Lab: the staged pre-sweep flow of the point PDS steps ahead is warmed too
    // (1.7% faster on the Sintel-shaped pair; on gray frames it cost 10%)
    static constexpr int PDS = C == 3 ? 6 : 0;
    static constexpr int THREADS = (WARM ? 5 : 4) * 32;
};

template <int C, int LPC> struct SweepShared {
    using SG = SweepGeo<C, LPC>;
    // -64 x query, per word (4 dimensions).  The batch layout's rows are
    // padded by one word so that its 16 rows' loads spread over the banks
    // (6.7% faster on the Sintel-shaped pair; neutral for the one-pair layouts)
    int4 in_nq[SG::DI][SG::RW][SG::NW + (LPC == 1 ? 1 : 0)];
    uint8_t in_raw[SG::DI][SG::RW][SG::P];        // query bytes as copied
    uint32_t in_flow[SG::DI][SG::RW];
    int in_cost[SG::DI][SG::RW];
    unsigned long long out[SG::DO][SG::RW];       // (tag:12 | cost:20) << 32 | flow
    unsigned long long lring[SG::LRING];          // (column + 1) << 32 | flow
    int in_ready, out_cons, lcons, abort, strip;
    uint32_t pf_sink[32];                         // destination of L1-warming copies
};

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16ca(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
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
__device__ __forceinline__ int4 lds128v(const int4 *p) {
    int4 r;
    asm volatile("ld.volatile.shared.v4.s32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "r"((unsigned)__cvta_generic_to_shared(p)));
    return r;
}

// per-half-word signed clamp of a packed (x, y) int16 pair
__device__ __forceinline__ uint32_t clamp_s16x2(uint32_t v, uint32_t lo, uint32_t hi) {
    uint32_t r;
    asm("min.s16x2 %0, %1, %2;" : "=r"(r) : "r"(v), "r"(hi));
    asm("max.s16x2 %0, %0, %1;" : "+r"(r) : "r"(lo));
    return r;
}

// Bilinear read position of a flow already clamped into the frame, at grid
// point (gx, gy) of level L: the target 8 p + F in 1/8 px divided by n = 2^L
// with rounding half up (8 n gx + fx + n/2) >> L = 8 gx + ((fx + n/2) >> L);
// taps at the integer part and +1, clamped to the level (replicative
// border); weights (8-a)(8-b), a(8-b), (8-a)b, ab packed as bytes in tap
// order x0y0, x1y0, x0y1, x1y1, which is (8 + 255 a)(8 + 65535 b) (no byte
// of it carries into the next: each weight is at most 64).
struct TapRows {
    int r0, r1;      // byte offsets of rows y0, y1
    int c0, c1;      // byte offsets of columns x0, x1 within a row
    uint32_t w;
};
template <int P>
__device__ __forceinline__ TapRows taps_of(uint32_t f, int gx, int gy, int L, int half, int WL,
                                           int HL) {
    const int fx = (int)(int16_t)(f & 0xffffu), fy = (int)f >> 16;
    const int sx = 8 * gx + ((fx + half) >> L), sy = 8 * gy + ((fy + half) >> L);
    const int ix = sx >> 3, ax = sx & 7, iy = sy >> 3, ay = sy & 7;
    TapRows t;
    t.c0 = min(ix, WL - 1) * P;
    t.c1 = min(ix + 1, WL - 1) * P;
    t.r0 = min(iy, HL - 1) * WL * P;
    t.r1 = min(iy + 1, HL - 1) * WL * P;
    t.w = (uint32_t)(8 + 255 * ax) * (uint32_t)(8 + 65535 * ay);
    return t;
}

// NWL consecutive feature words of one tap (NWL = 1, 2, 4 or 8)
template <int NWL> struct Words {
    uint32_t w[NWL];
};
template <int NWL>
__device__ __forceinline__ Words<NWL> ldg_words(const uint8_t *p) {
    Words<NWL> r;
    if constexpr (NWL == 8) {
        const uint4 a = __ldg(reinterpret_cast<const uint4 *>(p));
        const uint4 b = __ldg(reinterpret_cast<const uint4 *>(p + 16));
        r.w[0] = a.x, r.w[1] = a.y, r.w[2] = a.z, r.w[3] = a.w;
        r.w[4] = b.x, r.w[5] = b.y, r.w[6] = b.z, r.w[7] = b.w;
    } else if constexpr (NWL == 4) {
        const uint4 a = __ldg(reinterpret_cast<const uint4 *>(p));
        r.w[0] = a.x, r.w[1] = a.y, r.w[2] = a.z, r.w[3] = a.w;
    } else if constexpr (NWL == 2) {
        const uint2 a = __ldg(reinterpret_cast<const uint2 *>(p));
        r.w[0] = a.x, r.w[1] = a.y;
    } else {
        r.w[0] = __ldg(reinterpret_cast<const unsigned int *>(p));
    }
    return r;
}

// Partial matching error over NC words of one lane: the 4 taps of each word
// are byte-transposed and one dp4a per dimension forms sum_taps w tap[d] -
// 64 q[d] (the query enters as the accumulator).
template <int NWL, int NC>
__device__ __forceinline__ int sad_taps(const uint8_t *base, const TapRows &t, const int4 *nq) {
    const Words<NWL> a = ldg_words<NWL>(base + t.r0 + t.c0);
    const Words<NWL> b = ldg_words<NWL>(base + t.r0 + t.c1);
    const Words<NWL> c = ldg_words<NWL>(base + t.r1 + t.c0);
    const Words<NWL> d = ldg_words<NWL>(base + t.r1 + t.c1);
    int e = 0;
#pragma unroll
    for (int j = 0; j < NC; j++) e += sad_word(a.w[j], b.w[j], c.w[j], d.w[j], t.w, nq[j]);
    return e;
}

// A result slot: tag (the step, 12 bits), cost (20 bits; a cost is at most
// 27 x 255 x 64 = 440640 < 2^20, 0xFFFFF marks an unset one) and flow.
__device__ __forceinline__ unsigned long long pack_out(int tag, int cost, uint32_t flow) {
    const uint32_t c = cost == kCostInvalid ? 0xFFFFFu : ((uint32_t)cost & 0xFFFFFu);
    return ((unsigned long long)(((uint32_t)(tag & 0xFFF) << 20) | c) << 32) | flow;
}

// target (1/8 px) of flow f at grid point (px, py), clamped into the frame
__device__ __forceinline__ void target_of(uint32_t f, int px, int py, int W, int H, int &tx,
                                          int &ty) {
    tx = clampi(8 * px + flow_x(f), 0, 8 * (W - 1));
    ty = clampi(8 * py + flow_y(f), 0, 8 * (H - 1));
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
// the raster order exactly as a skewed wavefront: row r of a strip handles
// column u = i - r at step i.
//
//  * Propagation warp: only the dependent chain.  Each step takes the
//    vertical source (the row above's last decision by a shuffle, or for the
//    strip's first row the previous strip's last row through a ring the
//    loader fills) and the horizontal source (the row's own last decision),
//    clamps both into the frame, evaluates each on its own lanes, exchanges
//    the two costs by a shuffle and keeps, among [current, vertical,
//    horizontal], the lowest cost, the later candidate on ties.  Both
//    candidates are always evaluated: a candidate equal to the current flow
//    has exactly the cached cost, so this changes no result.  The decision
//    goes into a tagged result slot and, for the strip's last row, into the
//    boundary row in global memory.  The step's inputs are read at the end
//    of the step before and checked at once (one branch per step).
//  * Stager warp: copies each point's pre-sweep flow, cost and query bytes
//    into a shared ring A steps ahead (cp.async) and turns the query into
//    -64 q per dimension, the accumulator seed of the cost's dot products.
//  * Random-search warp: a few steps behind, takes each result, draws the
//    point's offset (Philox4x32-10, counter (y*W + x, t, L, dir), key (seed,
//    pair_id)), keeps it only if strictly better, and writes the final flow
//    and cost.  Neighbours in this sweep see only the sweep value.
//  * Warming warp: follows the result slots and pulls into L1 the feature
//    sectors around each decided flow's target two points further on, where
//    the row's next loads most likely fall (for Lab frames also those of the
//    staged pre-sweep flows a few steps ahead).
//  * Loader warp: copies the previous strip's boundary row into the ring.
// Strips are handed out by a ticket counter, so a strip only waits on a
// strip that is already running.  Every wait is bounded and warp-uniform: a
// warp that sees no progress for wait_ns sets the error word to FF_ETIMEOUT,
// raises the CTA's abort flag and returns; every other wait in the CTA
// checks that flag on its slow path.
template <int C, int LPC>
__device__ __forceinline__ void sweep_body(const SweepArgs &a) {
    using SG = SweepGeo<C, LPC>;
    constexpr int P = SG::P, G = SG::G, RW = SG::RW;
    constexpr int DI = SG::DI, DO = SG::DO, A = SG::A, LRING = SG::LRING;
    constexpr int WPC = SG::WPC, LWP = SG::LWP, WPH = SG::WPH, NB = SG::NB;
    constexpr int PD = SG::PD, PF_ROWS = SG::PF_ROWS, PF_COLS = SG::PF_COLS;
    constexpr unsigned FULL = 0xffffffffu;
    __shared__ __align__(16) SweepShared<C, LPC> sm;
    volatile int *v_in_ready = &sm.in_ready;
    volatile int *v_out_cons = &sm.out_cons;
    volatile int *v_lcons = &sm.lcons;
    volatile int *v_abort = &sm.abort;

    const int tid = threadIdx.x;
    const int U = a.WL, V = a.HL;
    const int nstrips = (V + RW - 1) / RW;
    if (tid == 0) {
        sm.strip = (int)atomicAdd(a.ticket, 1u);
        sm.lcons = 0;
        sm.abort = 0;
        sm.in_ready = 0;
        sm.out_cons = 0;
    }
    // ring tags start at 0 (no column has tag 0); result slots at tag 0xFFF
    for (int j = tid; j < LRING; j += blockDim.x) sm.lring[j] = 0ull;
    for (int j = tid; j < DO * RW; j += blockDim.x) (&sm.out[0][0])[j] = ~0ull;
    __syncthreads();
    const int strip = sm.strip;
    if (strip >= nstrips) return;
    const int v0 = strip * RW;
    const int warp = tid >> 5, lane = tid & 31;

    if (warp == SG::LOADER) {
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

    const int k = lane / G, g = lane - (lane / G) * G;
    const int v = v0 + k;
    const bool row_ok = v < V;
    const int L = a.L, n = 1 << L, W = a.W, H = a.H, half = n >> 1;
    const int sd = a.d;
    const bool flipx = (sd == 1 || sd == 2), flipy = (sd == 1 || sd == 3);
    const int gy = row_ok ? (flipy ? V - 1 - v : v) : 0;
    const int py = gy * n;
    const int NS = U + RW - 1;                            // local steps of a warp
    const uint8_t *f1L = a.f1L, *f2L = a.f2L;
    const size_t rowbase = (size_t)gy * U;

    if (SG::WARM && warp == 3) {
        // ================= warming warp =================
        // Warms L1 with the feature sectors the propagation warp will read two
        // points after each decision: rows iy-2 .. iy+3 around the target of
        // the decided flow at that point, columns ix .. ix+PF_COLS-1, one
        // sector (one point's feature vector) each, by asynchronous 4-byte
        // copies into a scratch word.  It follows the tagged result slots,
        // so the propagation warp spends no instruction on it; a slot holding
        // a later step than expected (this warp fell a ring behind) is taken
        // as it is.  For Lab frames it also warms, PDS steps ahead, the 3 x 3
        // sectors around the target of a point's staged pre-sweep flow at the
        // next point: in a settled field that flow is the likely value of the
        // next point's horizontal source and of the point below's vertical one.
        const int sxdir = flipx ? -1 : 1;
        int i = 0, wready = 0;
        unsigned long long t0 = 0;
        while (i < NS) {
            const unsigned long long e = lds64(&sm.out[i & (DO - 1)][k]);
            const uint32_t dd = ((uint32_t)(e >> 52) - (uint32_t)i) & 0xFFFu;   // its step - i
            if (!__all_sync(FULL, dd < 0x800u)) {
                if (wait_expired(t0, a.wait_ns, v_abort, a.err)) break;
                continue;
            }
            t0 = 0;
            const int u = i + (int)dd - k;                // the point decided in that step
            const uint32_t f = (uint32_t)e;
            if (row_ok && u >= 0 && u < U && f != kFlowInvalid) {
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
                            cp_async4(&sm.pf_sink[lane], rowp + (size_t)min(ix + cc, U - 1) * P);
                    }
                }
            }
            if (SG::PDS > 0) {
                const int j = i + (int)dd + SG::PDS;
                if (wready <= j) wready = *v_in_ready;
                const int uj = j - k;
                if (j < wready && row_ok && uj >= 0 && uj + 1 < U && g < 3) {
                    const uint32_t fj = ((volatile uint32_t *)sm.in_flow[j & (DI - 1)])[k];
                    if (fj != kFlowInvalid) {
                        const int gxn = flipx ? U - 1 - (uj + 1) : uj + 1;
                        int tx, ty;
                        target_of(fj, gxn * n, py, W, H, tx, ty);
                        const int ixn = tx >> (L + 3), iyn = (ty >> (L + 3)) + g;
                        const uint8_t *rowp = f2L + (size_t)clampi(iyn, 0, V - 1) * U * P;
#pragma unroll
                        for (int cc = -1; cc <= 1; cc++)
                            cp_async4(&sm.pf_sink[lane],
                                      rowp + (size_t)clampi(ixn + cc, 0, U - 1) * P);
                    }
                }
            }
            i += 1 + (int)__reduce_min_sync(FULL, dd);
        }
        cp_async_commit();
        cp_async_wait<0>();
        return;
    }

    if (warp == 2) {
        // ================= stager warp =================
        // step j's inputs -> ring slot j mod DI: flow and cost, the query's
        // bytes (P / G per lane), then -64 q per dimension.  A slot is reused
        // only after the random-search warp (the last reader) took its step.
        constexpr int QB = SG::QB, QL = SG::QL;            // query bytes per lane, lanes used
        auto stage = [&](int j) {
            const int uj = j - k;
            if (row_ok && uj >= 0 && uj < U) {
                const int gx = flipx ? U - 1 - uj : uj;
                const size_t pi = rowbase + gx;
                const int slot = j & (DI - 1);
                if (g == 0) cp_async4(&sm.in_flow[slot][k], a.flow + pi);
                if (g == G - 1) cp_async4(&sm.in_cost[slot][k], a.cost + pi);
                if (g < QL) {
                    uint8_t *dst = &sm.in_raw[slot][k][QB * g];
                    const uint8_t *srcq = f1L + pi * P + QB * g;
                    if constexpr (QB == 16) cp_async16ca(dst, srcq);
                    else if constexpr (QB == 8) cp_async8(dst, srcq);
                    else cp_async4(dst, srcq);
                }
            }
        };
        auto convert = [&](int j) {
            if (g >= QL) return;
            const int slot = j & (DI - 1);
            const uint32_t *raw = reinterpret_cast<const uint32_t *>(&sm.in_raw[slot][k][QB * g]);
#pragma unroll
            for (int ww = 0; ww < QB / 4; ww++) sm.in_nq[slot][k][(QB / 4) * g + ww] = neg64(raw[ww]);
        };
        for (int j = 0; j < A; j++) {
            stage(j);
            cp_async_commit();
        }
        cp_async_wait<0>();
        for (int j = 0; j < A; j++) convert(j);
        __threadfence_block();
        __syncwarp();
        if (lane == 0) *v_in_ready = A;
        int ocons = 0;
        for (int i = 0; i + A < NS + 3; i++) {
            const int j = i + A;
            if (j < NS && ocons <= j - DI) {
                unsigned long long t0 = 0;
                while (true) {
                    ocons = *v_out_cons;
                    if (__all_sync(FULL, ocons > j - DI)) break;
                    if (wait_expired(t0, a.wait_ns, v_abort, a.err)) {
                        cp_async_wait<0>();
                        return;
                    }
                }
            }
            if (j < NS) stage(j);
            cp_async_commit();
            cp_async_wait<3>();
            if (j - 3 >= A) convert(j - 3);                // its copies have landed
            __threadfence_block();
            __syncwarp();
            if (lane == 0) *v_in_ready = max(A, j - 2);
        }
        cp_async_wait<0>();
        return;
    }

    if (warp == 1) {
        // ================= random-search warp =================
        const int Rq = a.radius_q3 * n;
        const uint32_t span = 2u * (uint32_t)Rq + 1u;
        int offs[NB];
#pragma unroll
        for (int j = 0; j < NB; j++) offs[j] = 0;
        for (int i = 0; i < NS; i++) {
            const int phase = i & 7;
            if (phase == 0 && a.do_rs) {
                // offsets of this row's points of steps i .. i+7
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
            const unsigned long long *oslot = &sm.out[i & (DO - 1)][k];
            unsigned long long e;
            unsigned long long t0 = 0;
            while (true) {
                e = lds64(oslot);
                const bool ok = (uint32_t)(e >> 52) == (uint32_t)(i & 0xFFF);
                if (__all_sync(FULL, ok)) break;
                if (wait_expired(t0, a.wait_ns, v_abort, a.err)) return;
            }
            constexpr int HLW = SG::HL_;
            const int gw = g < HLW ? g : 0;              // lanes past the words evaluate nothing
            int4 nq[WPH];
#pragma unroll
            for (int j = 0; j < WPH; j++) nq[j] = lds128v(&sm.in_nq[i & (DI - 1)][k][WPH * gw + j]);
            __syncwarp();
            if (lane == 0) *v_out_cons = i + 1;
            const uint32_t best = (uint32_t)e;
            const uint32_t c20 = (uint32_t)(e >> 32) & 0xFFFFFu;
            const int bcost = c20 == 0xFFFFFu ? kCostInvalid : (int)c20;
            const int u = i - k;
            const bool valid = row_ok && u >= 0 && u < U;
            // an in-frame column for every lane keeps every tap address in bounds
            const int uc = min(max(u, 0), U - 1);
            const int gx = flipx ? U - 1 - uc : uc;
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
                    const TapRows t = taps_of<P>(cR, gx, gy, L, half, U, V);
                    er = sad_taps<WPH, WPH>(f2L + 4 * WPH * gw, t, nq);
                    if (g >= HLW) er = 0;
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
        return;
    }

    // ================= propagation warp =================
    const int cand = g / LPC;                    // 0: vertical candidate, 1: horizontal
    const int hw = g - cand * LPC;               // which words of the candidate
    const bool edge_out = (k == RW - 1) && (strip + 1 < nstrips);
    const bool top_src = v0 > 0;                 // row 0 has a row above it
    const uint8_t *f2w = f2L + 4 * LWP * hw;     // this lane's words of every feature vector
    const int loy = -8 * py, hiy = 8 * (H - 1) - 8 * py;
    uint32_t last = kFlowInvalid;       // this row's sweep value at the previous step
    // The step has one branch besides the loop's: its inputs are checked at
    // once, from values read at the end of the step before (the stager's and
    // the random-search warp's progress, row 0's ring entry), and only a step
    // that finds one of them short takes the slow path and reads them again.
    // Every other condition is a select or a predicate (each branch on this
    // chain cost about 2% of the sweep, measured).
    int ready = 0;                      // in_ready as read at the end of the step before
    int ocons = 0;                      // out_cons as read at the end of the step before
    unsigned long long te_next = lds64(&sm.lring[0]);
    for (int i = 0; i < NS; i++) {
        const int u = i - k;
        const bool active = row_ok && u >= 0 && u < U;
        const int uc = min(max(u, 0), U - 1);
        const int gx = flipx ? U - 1 - uc : uc;
        const uint32_t above = __shfl_up_sync(FULL, last, G);
        // staged inputs of step i, (row 0) the vertical source of column i,
        // and room in the result ring (the random-search warp took step i - DO)
        const bool need_top = top_src && i < U && k == 0;
        unsigned long long te = te_next;
        bool ok = ready > i && ocons > i - DO;
        if (need_top) ok = ok && (uint32_t)(te >> 32) == (uint32_t)(i + 1);
        if (!__all_sync(FULL, ok)) {
            unsigned long long t0 = 0;
            while (true) {
                if (wait_expired(t0, a.wait_ns, v_abort, a.err)) return;
                ready = *v_in_ready;
                ocons = *v_out_cons;
                ok = ready > i && ocons > i - DO;
                if (need_top) {
                    te = lds64(&sm.lring[i & (LRING - 1)]);
                    ok = ok && (uint32_t)(te >> 32) == (uint32_t)(i + 1);
                }
                if (__all_sync(FULL, ok)) break;
            }
        }
        if (need_top && g == 0) *v_lcons = i + 1;
        const int islot = i & (DI - 1);
        // (a row before or past its columns holds no staged point: unset)
        const uint32_t sflow = ((volatile uint32_t *)sm.in_flow[islot])[k];
        const int scost = ((volatile int *)sm.in_cost[islot])[k];
        const uint32_t cur = active ? sflow : kFlowInvalid;
        const int ccost = active ? scost : kCostInvalid;
        int4 nq[WPC];
#pragma unroll
        for (int j = 0; j < WPC; j++) nq[j] = lds128v(&sm.in_nq[islot][k][LWP * hw + j]);
        const uint32_t vflow = (active && v > 0) ? ((k > 0) ? above : (uint32_t)te) : kFlowInvalid;
        const uint32_t hflow = (active && u > 0) ? last : kFlowInvalid;
        // both candidates clamped into the frame: 8 p + F in [0, 8(W-1)] x [0, 8(H-1)]
        const int lox = -8 * gx * n;
        const uint32_t lo = ((uint32_t)loy << 16) | ((uint32_t)lox & 0xffffu);
        const uint32_t hi = ((uint32_t)hiy << 16) | ((uint32_t)(lox + 8 * (W - 1)) & 0xffffu);
        const uint32_t cV = clamp_s16x2(vflow, lo, hi);
        const uint32_t cH = clamp_s16x2(hflow, lo, hi);
        const TapRows t = taps_of<P>(cand == 0 ? cV : cH, gx, gy, L, half, U, V);
        int e = sad_taps<LWP, WPC>(f2w, t, nq);
        // this candidate's cost and the other one's (eo); with two lanes per
        // candidate, three independent shuffles instead of two in a row
        int eo;
        if constexpr (LPC == 2) {
            const int x1 = __shfl_xor_sync(FULL, e, 1), x2 = __shfl_xor_sync(FULL, e, 2),
                      x3 = __shfl_xor_sync(FULL, e, 3);
            e += x1;
            eo = x2 + x3;
        } else {
#pragma unroll
            for (int o = 1; o < LPC; o <<= 1) e += __shfl_xor_sync(FULL, e, o);
            eo = __shfl_xor_sync(FULL, e, LPC);
        }
        const int ev = cand == 0 ? e : eo, eh = cand == 0 ? eo : e;
        // [current, vertical, horizontal]: lowest cost, the later one on ties
        uint32_t best = cur;
        int bcost = ccost;
        if (vflow != kFlowInvalid && ev <= bcost) {
            best = cV;
            bcost = ev;
        }
        if (hflow != kFlowInvalid && eh <= bcost) {
            best = cH;
            bcost = eh;
        }
        if (active) last = best;
        // the strip's last row -> the next strip (a predicated store)
        st_relaxed_u64_if(a.edge + (size_t)strip * U + uc, ((unsigned long long)a.epoch << 32) | best,
                          edge_out && active && g == 0);
        // result -> random-search and warming warps (tagged slot)
        if (g == 0) sts64(&sm.out[i & (DO - 1)][k], pack_out(i, bcost, best));
        // the next step's inputs, read now (checked at its start)
        te_next = lds64(&sm.lring[(i + 1) & (LRING - 1)]);
        ready = *v_in_ready;
        ocons = *v_out_cons;
    }
}

// The sweep kernel.  One lane per candidate (LPC = 1) is bounded to the
// registers that let MIN_CTAS CTAs share an SM; the other layouts run one CTA
// per SM for a single pair, so they are compiled for one (the compiler then
// takes 79 instead of 64 registers: 2% faster on both single-pair workloads).
template <int C, int LPC>
__global__ void __launch_bounds__(SweepGeo<C, LPC>::THREADS, 1) k_sweep(const SweepArgs a) {
    sweep_body<C, LPC>(a);
}
template <int C>
__global__ void __launch_bounds__(SweepGeo<C, 1>::THREADS, SweepGeo<C, 1>::MIN_CTAS)
    k_sweep_many(const SweepArgs a) {
    sweep_body<C, 1>(a);
}

}  // namespace ffk
