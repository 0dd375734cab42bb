// ff_kernels.cuh - device code of the Flow Fields matching loop for sm_103a.
//
// Data layout in device memory (all row-major):
//   features   uint8 [H_L][W_L][P] per level, P = 16 (gray) or 32 (Lab);
//              the 9 (27) int8 WHT codes fill bytes 0..8 (0..26), the rest
//              is zero, so one 4-byte word holds 4 dimensions.
//   flow       uint32 per grid point: x in the low int16, y in the high int16
//              (1/8 px); 0x80008000 marks an unset flow.
//   cost       int32 per grid point, INT32_MAX when unset.
//
// Arithmetic is exact integer throughout; see the comments at each kernel
// for the step of the paper (arXiv 1703.02563) it computes.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ffk {

constexpr uint32_t kFlowInvalid = 0x80008000u;
constexpr int kCostInvalid = 0x7fffffff;
constexpr int kErrTimeout = 4;   // matches FF_ETIMEOUT

template <int C> struct Geo;
template <> struct Geo<1> { static constexpr int P = 16, NW = 3, G = 4; };
template <> struct Geo<3> { static constexpr int P = 32, NW = 7, G = 8; };

__device__ __forceinline__ uint32_t pack_flow(int fx, int fy) {
    return (uint32_t)(uint16_t)(int16_t)fx | ((uint32_t)(uint16_t)(int16_t)fy << 16);
}
__device__ __forceinline__ int flow_x(uint32_t f) { return (int)(int16_t)(f & 0xffffu); }
__device__ __forceinline__ int flow_y(uint32_t f) { return (int)(int16_t)(f >> 16); }

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

// A candidate flow whose target 8p + F leaves the frame is moved to the
// nearest target inside it; the moved flow is the one kept.
__device__ __forceinline__ void clamp_flow(int W, int H, int px, int py, int &fx, int &fy) {
    fx = clampi(8 * px + fx, 0, 8 * (W - 1)) - 8 * px;
    fy = clampi(8 * py + fy, 0, 8 * (H - 1)) - 8 * py;
}

// Bilinear read position of candidate F at grid point p on level L: the
// target in 1/8 px is divided by n = 2^L with rounding half up; taps at the
// integer part and +1 (clamped to the level), weights (8-f)(8-g), f(8-g),
// (8-f)g, fg packed as bytes in tap order (x0y0, x1y0, x0y1, x1y1).
struct Tap {
    int o00, o10, o01, o11;   // byte offsets of the 4 tap pixels
    uint32_t w;               // packed weights
};

template <int P>
__device__ __forceinline__ Tap make_tap(int px, int py, int fx, int fy, int L, int WL, int HL) {
    const int half = (1 << L) >> 1;
    const int sx = (8 * px + fx + half) >> L;
    const int sy = (8 * py + fy + half) >> L;
    const int ix = sx >> 3, ax = sx & 7;
    const int iy = sy >> 3, ay = sy & 7;
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

// -64 * (the 4 signed bytes of a query word), the accumulator seeds of the
// interpolation dot products
__device__ __forceinline__ int4 neg64(uint32_t q) {
    return make_int4(-64 * (int)(int8_t)(q & 0xff), -64 * (int)(int8_t)((q >> 8) & 0xff),
                     -64 * (int)(int8_t)((q >> 16) & 0xff), -64 * (int)(int8_t)(q >> 24));
}

// Sum over the 4 dimensions of one feature word of
// | sum_taps w * tap[d] - 64 * query[d] |.  The 4 taps are transposed so that
// each dimension's 4 tap bytes share a word, then one dp4a per dimension
// forms the interpolation and subtracts the query.
__device__ __forceinline__ int sad_word(uint32_t t00, uint32_t t10, uint32_t t01, uint32_t t11,
                                        uint32_t w, int4 na) {
    const uint32_t lo01 = __byte_perm(t00, t10, 0x5140);
    const uint32_t hi01 = __byte_perm(t00, t10, 0x7362);
    const uint32_t lo23 = __byte_perm(t01, t11, 0x5140);
    const uint32_t hi23 = __byte_perm(t01, t11, 0x7362);
    const int e0 = __dp4a((int)__byte_perm(lo01, lo23, 0x5410), (int)w, na.x);
    const int e1 = __dp4a((int)__byte_perm(lo01, lo23, 0x7632), (int)w, na.y);
    const int e2 = __dp4a((int)__byte_perm(hi01, hi23, 0x5410), (int)w, na.z);
    const int e3 = __dp4a((int)__byte_perm(hi01, hi23, 0x7632), (int)w, na.w);
    return abs(e0) + abs(e1) + abs(e2) + abs(e3);
}

__device__ __forceinline__ uint32_t ldg32(const uint8_t *p) {
    return __ldg(reinterpret_cast<const unsigned int *>(p));
}

// Partial matching error of one word (lane g of a point's lane group).
__device__ __forceinline__ int sad_lane(const uint8_t *f2L, const Tap &t, int g, int4 na) {
    const uint8_t *b = f2L + 4 * g;
    return sad_word(ldg32(b + t.o00), ldg32(b + t.o10), ldg32(b + t.o01), ldg32(b + t.o11), t.w,
                    na);
}

// Full matching error by one thread (all words of the query).
template <int C>
__device__ __forceinline__ int sad_full(const uint8_t *f2L, const Tap &t, const uint32_t *q) {
    int e = 0;
#pragma unroll
    for (int g = 0; g < Geo<C>::NW; g++) e += sad_lane(f2L, t, g, neg64(q[g]));
    return e;
}

// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64-bit
// products; the key advances by the Weyl constants after every round.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; r++) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// the same, under a predicate (no branch around the store)
__device__ __forceinline__ void st_relaxed_u64_if(unsigned long long *p, unsigned long long v,
                                                  bool pred) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.s32 p, %2, 0;\n\t@p st.relaxed.gpu.global.b64 [%0], %1;\n\t}"
        ::"l"(p), "l"(v), "r"((int)pred)
        : "memory");
}

__device__ __forceinline__ int ld_relaxed_i32(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// named barrier 1 over `n` threads with an OR-reduction of `pred`
__device__ __forceinline__ int bar_or(int pred, int n) {
    int out;
    asm volatile(
        "{\n\t.reg .pred pi, po;\n\t"
        "setp.ne.s32 pi, %1, 0;\n\t"
        "bar.red.or.pred po, 1, %2, pi;\n\t"
        "selp.s32 %0, 1, 0, po;\n\t}"
        : "=r"(out)
        : "r"(pred), "r"(n)
        : "memory");
    return out;
}

}  // namespace ffk
