/*
 * ffo.c - CPU oracle of the Flow Fields multi-scale patch-matching loop.
 *
 * TEST INFRASTRUCTURE ONLY: tests, the smoke check and the benchmark's CPU
 * baseline call this; the product path never does.  Plain, sequential C in
 * exact integer arithmetic, one function per step of the method, in the
 * paper's order (arXiv 1703.02563):
 *
 *   level images      Sec. 3.6 (area downsampling) + replicative border
 *   WHT features      Sec. 3.1 (first 9 Walsh-Hadamard bases per channel)
 *   seeding           Sec. 3.1 Eq. 1 (candidates + rerank by E_d), Sec. 3.2 Eq. 4
 *   propagation       Sec. 3.1 Eq. 2 (sources processed before the point)
 *   random search     Sec. 3.1 (uniform offset of at most R, accept if E drops)
 *   directions        Sec. 3.1 (4 propagations alternating with 3 searches)
 *   coarse to fine    Sec. 3.2 (grid points p^n, R_n = R n, seeds from scale 2n)
 *   consistency       Sec. 3.7 (|F(p) + F_b(p + F(p))| < eps)
 *
 * Where the paper leaves a choice open, the reading taken is stated at the
 * function that makes it.
 */
#include "ffo.h"

#include <limits.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define INVALID_F (-32768)
#define INVALID_COST INT32_MAX

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* floor(a / b) for b > 0, independent of how C rounds negative quotients */
static int floor_div(int a, int b) {
    int q = a / b;
    if ((a % b != 0) && (a < 0)) q -= 1;
    return q;
}

void ffo_level_dims(int W, int H, int L, int *WL, int *HL) {
    int n = 1 << L;
    *WL = (W + n - 1) / n;
    *HL = (H + n - 1) / n;
}

long ffo_feature_offset(int W, int H, int C, int L) {
    long off = 0;
    for (int l = 0; l < L; l++) {
        int wl, hl;
        ffo_level_dims(W, H, l, &wl, &hl);
        off += (long)wl * hl * 9 * C;
    }
    return off;
}

long ffo_feature_bytes(int W, int H, int C, int S) { return ffo_feature_offset(W, H, C, S); }

/* Sec. 3.6: "downsampling ... by a factor of n with area based downsampling";
 * pixels outside the image take the colour of the nearest visible pixel.
 * Reading: the average is rounded half up to an integer (n*n/2 added before
 * the division by n*n). */
void ffo_level_image(const uint8_t *img, int C, int W, int H, int L, uint8_t *out) {
    int n = 1 << L, WL, HL;
    ffo_level_dims(W, H, L, &WL, &HL);
    for (int c = 0; c < C; c++)
        for (int y = 0; y < HL; y++)
            for (int x = 0; x < WL; x++) {
                int sum = 0;
                for (int i = 0; i < n; i++)
                    for (int j = 0; j < n; j++) {
                        int yy = clampi(n * y + i, 0, H - 1);
                        int xx = clampi(n * x + j, 0, W - 1);
                        sum += img[((long)c * H + yy) * W + xx];
                    }
                out[((long)c * HL + y) * WL + x] = (uint8_t)((sum + n * n / 2) / (n * n));
            }
}

/* Sec. 3.1: WHT of the patch around each pixel, first 9 bases per channel.
 * Reading: the 9 bases are the 2-D Walsh functions w_u (x) w_v with u, v in
 * {0,1,2}, the three lowest-sequency 1-D Walsh functions of length 8 (0, 1 and
 * 2 sign changes).  The 8x8 window is split in the middle as the footnote
 * says: offsets -3..+4 around the pixel in each direction.  u runs down the
 * rows, v along the columns; dimension index ch*9 + 3u + v. */
static const int WALSH[3][8] = {
    {1, 1, 1, 1, 1, 1, 1, 1},
    {1, 1, 1, 1, -1, -1, -1, -1},
    {1, 1, -1, -1, -1, -1, 1, 1},
};

void ffo_wht_coeffs(const uint8_t *D, int C, int WL, int HL, int32_t *out) {
    for (int y = 0; y < HL; y++)
        for (int x = 0; x < WL; x++)
            for (int c = 0; c < C; c++)
                for (int u = 0; u < 3; u++)
                    for (int v = 0; v < 3; v++) {
                        int32_t acc = 0;
                        for (int i = 0; i < 8; i++)
                            for (int j = 0; j < 8; j++) {
                                int yy = clampi(y - 3 + i, 0, HL - 1);
                                int xx = clampi(x - 3 + j, 0, WL - 1);
                                acc += WALSH[u][i] * WALSH[v][j] *
                                       (int32_t)D[((long)c * HL + yy) * WL + xx];
                            }
                        out[((long)y * WL + x) * 9 * C + c * 9 + 3 * u + v] = acc;
                    }
}

/* int8 code of one coefficient.  The paper keeps WHT vectors in floating
 * point; this quantiser is the library's definition: the DC term becomes the
 * window mean minus 128, every other term is divided by 16; both are rounded
 * half up (floor of x + 1/2) and saturated to [-128, 127]. */
int ffo_quantise(int32_t c, int uv_is_dc) {
    int q = uv_is_dc ? floor_div(c + 32, 64) - 128 : floor_div(c + 8, 16);
    return clampi(q, -128, 127);
}

void ffo_wht_features(const uint8_t *D, int C, int WL, int HL, int8_t *out) {
    long n = (long)WL * HL * 9 * C;
    int32_t *coef = (int32_t *)malloc(sizeof(int32_t) * n);
    ffo_wht_coeffs(D, C, WL, HL, coef);
    for (long k = 0; k < n; k++) out[k] = (int8_t)ffo_quantise(coef[k], (k % 9) == 0);
    free(coef);
}

/* Features of every level.  F2-style ordering (Sec. 3.6): the image is
 * downsampled first and the features are computed on the downsampled level. */
void ffo_features_all(const uint8_t *img, int C, int W, int H, int S, int8_t *out) {
    for (int L = 0; L < S; L++) {
        int WL, HL;
        ffo_level_dims(W, H, L, &WL, &HL);
        uint8_t *D = (uint8_t *)malloc((size_t)C * WL * HL);
        ffo_level_image(img, C, W, H, L, D);
        ffo_wht_features(D, C, WL, HL, out + ffo_feature_offset(W, H, C, L));
        free(D);
    }
}

/* Philox4x32-10, from Salmon, Moraes, Dror, Shaw, "Parallel random numbers:
 * as easy as 1, 2, 3" (SC'11): ten rounds of two 32x32->64 multiplications;
 * the key is bumped by the Weyl constants (golden ratio, sqrt(3)-1) between
 * rounds. */
void ffo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* Reading: a candidate whose target 8p + F leaves the image is moved to the
 * nearest target inside it, and the moved flow is the one kept.  The paper
 * only fixes the replicative border for pixel values (Sec. 3.6). */
void ffo_clamp_flow(int W, int H, int px, int py, int32_t *Fx, int32_t *Fy) {
    int tx = clampi(8 * px + *Fx, 0, 8 * (W - 1));
    int ty = clampi(8 * py + *Fy, 0, 8 * (H - 1));
    *Fx = tx - 8 * px;
    *Fy = ty - 8 * py;
}

/* Matching error E_d (Sec. 3.1; subsampled patch of Eq. 3 realised by the
 * level features).  Reading: the data term compares single feature vectors
 * (a pixel-wise feature, r = 0, as for the paper's pixel-wise SIFT term) with
 * the sum of absolute differences; the matched position is read with
 * bilinear interpolation in 1/8 pixel, as the paper prescribes for subpixel
 * positions.  Everything is scaled by 64 = 8*8 so it stays integer:
 *
 *   q = 8p + F (1/8 px, full resolution); s = round_half_up(q / n) on level L;
 *   taps at floor(s/8) and +1 (clamped to the level: replicative border),
 *   weights (8 - f)(8 - g), f(8 - g), (8 - f)g, fg with f, g = s mod 8;
 *   E = sum_d | 64 f1[p/n][d] - sum_taps w f2[tap][d] |.
 */
int32_t ffo_cost(const int8_t *f1L, const int8_t *f2L, int C, int W, int H, int L,
                 int px, int py, int32_t Fx, int32_t Fy) {
    int n = 1 << L, WL, HL;
    ffo_level_dims(W, H, L, &WL, &HL);
    int D = 9 * C;
    int qx = 8 * px + Fx, qy = 8 * py + Fy;
    int sx = floor_div(2 * qx + n, 2 * n); /* round half up of qx / n */
    int sy = floor_div(2 * qy + n, 2 * n);
    int ix = floor_div(sx, 8), fx = sx - 8 * ix;
    int iy = floor_div(sy, 8), fy = sy - 8 * iy;
    int x0 = clampi(ix, 0, WL - 1), x1 = clampi(ix + 1, 0, WL - 1);
    int y0 = clampi(iy, 0, HL - 1), y1 = clampi(iy + 1, 0, HL - 1);
    int w00 = (8 - fx) * (8 - fy), w10 = fx * (8 - fy), w01 = (8 - fx) * fy, w11 = fx * fy;
    const int8_t *a = f1L + ((long)(py / n) * WL + (px / n)) * D;
    const int8_t *t00 = f2L + ((long)y0 * WL + x0) * D;
    const int8_t *t10 = f2L + ((long)y0 * WL + x1) * D;
    const int8_t *t01 = f2L + ((long)y1 * WL + x0) * D;
    const int8_t *t11 = f2L + ((long)y1 * WL + x1) * D;
    int32_t E = 0;
    for (int d = 0; d < D; d++) {
        int interp = w00 * t00[d] + w10 * t10[d] + w01 * t01[d] + w11 * t11[d];
        int diff = 64 * a[d] - interp;
        E += diff < 0 ? -diff : diff;
    }
    return E;
}

/* Sec. 3.1: the kd-tree leaf of the query's WHT vector gives l candidates.
 * Reading: the exact l nearest neighbours (squared Euclidean distance of the
 * level-0 vectors) that the kd-tree approximates, ties broken by the smaller
 * linear index y2*W + x2; candidates are all image-2 pixels on the stride
 * grid (stride 1 in the paper; stride 2 is its Fast x2 option, Sec. 3.4.1).
 * Sec. 3.2: queries are the grid points p^N of the coarsest scale, using
 * non-subsampled (level-0) vectors. */
int ffo_seed_knn(const int8_t *f1_0, const int8_t *f2_0, int C, int W, int H, int S,
                 int leaf, int stride, int32_t *knn_idx, int32_t *knn_dist) {
    int WS, HS;
    ffo_level_dims(W, H, S - 1, &WS, &HS);
    return ffo_seed_knn_rows(f1_0, f2_0, C, W, H, S, leaf, stride, 0, HS, knn_idx, knn_dist);
}

int ffo_seed_knn_rows(const int8_t *f1_0, const int8_t *f2_0, int C, int W, int H, int S,
                      int leaf, int stride, int gy0, int gy1, int32_t *knn_idx,
                      int32_t *knn_dist) {
    int D = 9 * C, N = 1 << (S - 1), WS, HS, filled_max = 0;
    ffo_level_dims(W, H, S - 1, &WS, &HS);
    if (gy0 < 0) gy0 = 0;
    if (gy1 > HS) gy1 = HS;
    for (int gy = gy0; gy < gy1; gy++)
        for (int gx = 0; gx < WS; gx++) {
            int px = gx * N, py = gy * N;
            const int8_t *q = f1_0 + ((long)py * W + px) * D;
            int32_t *bi = knn_idx + ((long)gy * WS + gx) * leaf;
            int32_t *bd = knn_dist + ((long)gy * WS + gx) * leaf;
            int filled = 0;
            for (int y2 = 0; y2 < H; y2 += stride)
                for (int x2 = 0; x2 < W; x2 += stride) {
                    const int8_t *c = f2_0 + ((long)y2 * W + x2) * D;
                    int32_t dist = 0;
                    for (int d = 0; d < D; d++) {
                        int e = (int)q[d] - (int)c[d];
                        dist += e * e;
                    }
                    int32_t idx = y2 * W + x2;
                    /* insert into the ascending list ordered by (dist, idx);
                     * candidates arrive in increasing idx, so an equal
                     * distance goes after the entries already there */
                    if (filled == leaf && dist >= bd[leaf - 1]) continue;
                    int pos = (filled < leaf) ? filled : leaf - 1;
                    while (pos > 0 && bd[pos - 1] > dist) {
                        bd[pos] = bd[pos - 1];
                        bi[pos] = bi[pos - 1];
                        pos--;
                    }
                    bd[pos] = dist;
                    bi[pos] = idx;
                    if (filled < leaf) filled++;
                }
            for (int k = filled; k < leaf; k++) {
                bi[k] = -1;
                bd[k] = -1;
            }
            if (filled > filled_max) filled_max = filled;
        }
    return filled_max;
}

/* Sweep schedules.
 * basic (Sec. 3.1-3.2): `iters` sweeps with radius R, a random search after
 *   each but the last.
 * Flow Fields+ (Sec. 3.3): 4 sweeps with R+ = 2R (3 random searches), then 8
 *   sweeps with R (7 random searches); the four directions repeat every 4.
 * Flow Fields+ Fast (Sec. 3.4): as Flow Fields+, but the finest scale runs
 *   only 4 sweeps with R (3 random searches).
 * Flow Fields+ Fast x2 (Sec. 3.4): the finest scale is not run at all (its
 *   matches are the 2nd-finest scale's, one per 2x2 region); the 2nd-finest
 *   runs 4 sweeps with R, the coarser ones 4 with R+ and 8 with R. */
static int plus_level(int schedule, int L) {
    return schedule == 1 || (schedule == 2 && L > 0) || (schedule == 3 && L > 1);
}

int ffo_schedule_final_level(int schedule) { return schedule == 3 ? 1 : 0; }

int ffo_schedule_sweeps(int schedule, int iters, int L) {
    if (plus_level(schedule, L)) return 12;
    if (L < ffo_schedule_final_level(schedule)) return 0;
    if (schedule == 2 || schedule == 3) return 4;
    return iters;
}

int ffo_schedule_radius_mult(int schedule, int L, int t) {
    return (plus_level(schedule, L) && t < 4) ? 2 : 1;
}

int ffo_schedule_rs_after(int schedule, int iters, int L, int t) {
    const int n = ffo_schedule_sweeps(schedule, iters, L);
    if (plus_level(schedule, L)) return t != 3 && t != n - 1;
    return t < n - 1;
}

typedef struct {
    int16_t *fx, *fy;
    int32_t *cost;
} state_t;

static void set_invalid(state_t *s, long i) {
    s->fx[i] = INVALID_F;
    s->fy[i] = INVALID_F;
    s->cost[i] = INVALID_COST;
}

static int is_valid(const state_t *s, long i) { return s->fx[i] != INVALID_F; }

/* Sec. 3.1 Eq. 2 with the four directions of Sec. 3.1 (repeating every four
 * sweeps, Sec. 3.3).  Direction d = t mod 4; sweep 0 goes right and down so
 * that every new point gets a value (Sec. 3.1, 3.2).  Reading for the other
 * three (their figure is lost): d=1 left/up from the bottom-right corner,
 * d=2 from the top-right corner (sources right and above), d=3 from the
 * bottom-left corner (sources left and below).  At each point the candidates
 * are [current, vertical source, horizontal source] with the sources' values
 * already updated in this sweep; the lowest cost wins, and on equal cost the
 * later candidate wins, so horizontal propagation is preferred (Sec. 4.5). */
static void sweep(const int8_t *f1L, const int8_t *f2L, int C, int W, int H, int L, int d,
                  state_t *st, int64_t *evals) {
    int n = 1 << L, WL, HL;
    ffo_level_dims(W, H, L, &WL, &HL);
    int dx = (d == 0 || d == 3) ? 1 : -1; /* +1: left to right */
    int dy = (d == 0 || d == 2) ? 1 : -1; /* +1: top to bottom */
    for (int k = 0; k < HL; k++) {
        int gy = dy > 0 ? k : HL - 1 - k;
        for (int m = 0; m < WL; m++) {
            int gx = dx > 0 ? m : WL - 1 - m;
            long i = (long)gy * WL + gx;
            int px = gx * n, py = gy * n;
            int32_t bestx = st->fx[i], besty = st->fy[i], bestc = st->cost[i];
            int vy = gy - dy, hx = gx - dx; /* vertical / horizontal source */
            if (vy >= 0 && vy < HL) {
                long j = (long)vy * WL + gx;
                if (is_valid(st, j)) {
                    int32_t Fx = st->fx[j], Fy = st->fy[j];
                    ffo_clamp_flow(W, H, px, py, &Fx, &Fy);
                    int32_t E = ffo_cost(f1L, f2L, C, W, H, L, px, py, Fx, Fy);
                    (*evals)++;
                    if (E <= bestc) {
                        bestx = Fx;
                        besty = Fy;
                        bestc = E;
                    }
                }
            }
            if (hx >= 0 && hx < WL) {
                long j = (long)gy * WL + hx;
                if (is_valid(st, j)) {
                    int32_t Fx = st->fx[j], Fy = st->fy[j];
                    ffo_clamp_flow(W, H, px, py, &Fx, &Fy);
                    int32_t E = ffo_cost(f1L, f2L, C, W, H, L, px, py, Fx, Fy);
                    (*evals)++;
                    if (E <= bestc) {
                        bestx = Fx;
                        besty = Fy;
                        bestc = E;
                    }
                }
            }
            st->fx[i] = (int16_t)bestx;
            st->fy[i] = (int16_t)besty;
            st->cost[i] = bestc;
        }
    }
}

/* Sec. 3.1 random search: one uniformly distributed offset of at most R_n =
 * R n (Sec. 3.2), accepted only if the error decreases.  Each point depends
 * only on itself.  Readings: the offset is uniform over the square
 * [-R_n, R_n]^2 in 1/8 px, drawn per component as r mod (2R_n + 1) - R_n from
 * Philox4x32-10 with counter (y*W + x, t, L, dir) and key (seed, pair_id),
 * where (x, y) is the grid point's full-resolution position and t the sweep
 * the search follows. */
static void random_search(const int8_t *f1L, const int8_t *f2L, int C, int W, int H, int L,
                          int t, int dir, int radius_q3, uint32_t seed, uint32_t pair_id,
                          state_t *st, int64_t *evals) {
    int n = 1 << L, WL, HL;
    ffo_level_dims(W, H, L, &WL, &HL);
    uint32_t R = (uint32_t)(radius_q3 * n);
    uint32_t span = 2 * R + 1;
    for (int gy = 0; gy < HL; gy++)
        for (int gx = 0; gx < WL; gx++) {
            long i = (long)gy * WL + gx;
            if (!is_valid(st, i)) continue;
            int px = gx * n, py = gy * n;
            uint32_t ctr[4] = {(uint32_t)(py * W + px), (uint32_t)t, (uint32_t)L, (uint32_t)dir};
            uint32_t key[2] = {seed, pair_id};
            uint32_t r[4];
            ffo_philox4x32_10(ctr, key, r);
            int32_t ox = (int32_t)(r[0] % span) - (int32_t)R;
            int32_t oy = (int32_t)(r[1] % span) - (int32_t)R;
            int32_t Fx = st->fx[i] + ox, Fy = st->fy[i] + oy;
            ffo_clamp_flow(W, H, px, py, &Fx, &Fy);
            int32_t E = ffo_cost(f1L, f2L, C, W, H, L, px, py, Fx, Fy);
            (*evals)++;
            if (E < st->cost[i]) {
                st->fx[i] = (int16_t)Fx;
                st->fy[i] = (int16_t)Fy;
                st->cost[i] = E;
            }
        }
}

/* one propagation sweep / one random-search pass on a level's state
 * (flow interleaved int16 [HL][WL][2]); used by the tests to check a
 * single step of the method */
static void split_state(const int16_t *flow, const int32_t *cost, long NL, state_t *st) {
    st->fx = (int16_t *)malloc(sizeof(int16_t) * NL);
    st->fy = (int16_t *)malloc(sizeof(int16_t) * NL);
    st->cost = (int32_t *)malloc(sizeof(int32_t) * NL);
    for (long i = 0; i < NL; i++) {
        st->fx[i] = flow[2 * i];
        st->fy[i] = flow[2 * i + 1];
        st->cost[i] = cost[i];
    }
}

static void join_state(state_t *st, long NL, int16_t *flow, int32_t *cost) {
    for (long i = 0; i < NL; i++) {
        flow[2 * i] = st->fx[i];
        flow[2 * i + 1] = st->fy[i];
        cost[i] = st->cost[i];
    }
    free(st->fx);
    free(st->fy);
    free(st->cost);
}

void ffo_sweep_level(const int8_t *f1L, const int8_t *f2L, int C, int W, int H, int L, int d,
                     int16_t *flow, int32_t *cost, int64_t *evals) {
    int WL, HL;
    ffo_level_dims(W, H, L, &WL, &HL);
    state_t st;
    split_state(flow, cost, (long)WL * HL, &st);
    sweep(f1L, f2L, C, W, H, L, d & 3, &st, evals);
    join_state(&st, (long)WL * HL, flow, cost);
}

void ffo_random_search_level(const int8_t *f1L, const int8_t *f2L, int C, int W, int H, int L,
                             int t, int dir, int radius_q3, uint32_t seed, uint32_t pair_id,
                             int16_t *flow, int32_t *cost, int64_t *evals) {
    int WL, HL;
    ffo_level_dims(W, H, L, &WL, &HL);
    state_t st;
    split_state(flow, cost, (long)WL * HL, &st);
    random_search(f1L, f2L, C, W, H, L, t, dir, radius_q3, seed, pair_id, &st, evals);
    join_state(&st, (long)WL * HL, flow, cost);
}

/* Eq. 1 / Eq. 4 at the coarsest scale: each of the l seeding candidates p2
 * gives F = 8 (p2 - p); the one with the lowest E at scale N is kept, and on
 * equal E the earlier rank (the nearer WHT vector) stays. */
static void rerank(const ffo_params *prm, const int8_t *f1L, const int8_t *f2L, int W, int H,
                   int L, const int32_t *knn_idx, state_t *cur, int64_t *evals) {
    int n = 1 << L, WL, HL, C = prm->channels, l = prm->seed_leaf;
    ffo_level_dims(W, H, L, &WL, &HL);
    long NL = (long)WL * HL;
    for (long i = 0; i < NL; i++) {
        int gx = (int)(i % WL), gy = (int)(i / WL);
        int px = gx * n, py = gy * n;
        set_invalid(cur, i);
        for (int r = 0; r < l; r++) {
            int32_t idx = knn_idx[i * l + r];
            if (idx < 0) break;
            int32_t Fx = 8 * (idx % W - px), Fy = 8 * (idx / W - py);
            ffo_clamp_flow(W, H, px, py, &Fx, &Fy);
            int32_t E = ffo_cost(f1L, f2L, C, W, H, L, px, py, Fx, Fy);
            (*evals)++;
            if (E < cur->cost[i]) { /* ties: the earlier rank stays */
                cur->fx[i] = (int16_t)Fx;
                cur->fy[i] = (int16_t)Fy;
                cur->cost[i] = E;
            }
        }
    }
}

static int match_impl(const ffo_params *prm, const int8_t *fsrc, const int8_t *fdst,
                      int W, int H, int dir, uint32_t pair_id, const int16_t *seeds_in,
                      const int32_t *knn_in, int until_level, int until_sweeps,
                      int16_t *flow_out, int32_t *cost_out, int64_t *evals_out) {
    int C = prm->channels, S = prm->scales, I = prm->iters, sch = prm->schedule;
    if (W < 1 || H < 1 || W > 4096 || H > 4096 || (C != 1 && C != 3) || S < 1 || S > 8 ||
        I < 1 || prm->seed_leaf < 1 || prm->seed_stride < 1 || prm->radius_q3 < 0 ||
        sch < 0 || sch > 3 || until_level < ffo_schedule_final_level(sch) ||
        until_level >= S || until_sweeps < 0 ||
        until_sweeps > ffo_schedule_sweeps(sch, I, until_level))
        return 1;
    int64_t evals = 0;
    int WL, HL, WP = 0, HP = 0;
    state_t cur = {0}, prev = {0};
    for (int L = S - 1; L >= until_level; L--) {
        int n = 1 << L;
        ffo_level_dims(W, H, L, &WL, &HL);
        long NL = (long)WL * HL;
        const int8_t *f1L = fsrc + ffo_feature_offset(W, H, C, L);
        const int8_t *f2L = fdst + ffo_feature_offset(W, H, C, L);
        cur.fx = (int16_t *)malloc(sizeof(int16_t) * NL);
        cur.fy = (int16_t *)malloc(sizeof(int16_t) * NL);
        cur.cost = (int32_t *)malloc(sizeof(int32_t) * NL);
        if (L == S - 1) {
            if (seeds_in) {
                /* caller-supplied seeds on the coarsest grid */
                for (long i = 0; i < NL; i++) {
                    int gx = (int)(i % WL), gy = (int)(i / WL);
                    int32_t Fx = seeds_in[2 * i], Fy = seeds_in[2 * i + 1];
                    if (Fx == INVALID_F || Fy == INVALID_F) {
                        set_invalid(&cur, i);
                        continue;
                    }
                    ffo_clamp_flow(W, H, gx * n, gy * n, &Fx, &Fy);
                    cur.fx[i] = (int16_t)Fx;
                    cur.fy[i] = (int16_t)Fy;
                    cur.cost[i] = ffo_cost(f1L, f2L, C, W, H, L, gx * n, gy * n, Fx, Fy);
                    evals++;
                }
            } else if (knn_in) {
                /* seeding lists computed beforehand (by ffo_seed_knn_rows) */
                rerank(prm, f1L, f2L, W, H, L, knn_in, &cur, &evals);
            } else {
                int l = prm->seed_leaf;
                int32_t *ki = (int32_t *)malloc(sizeof(int32_t) * NL * l);
                int32_t *kd = (int32_t *)malloc(sizeof(int32_t) * NL * l);
                ffo_seed_knn(fsrc, fdst, C, W, H, S, l, prm->seed_stride, ki, kd);
                rerank(prm, f1L, f2L, W, H, L, ki, &cur, &evals);
                free(ki);
                free(kd);
            }
        } else {
            /* Sec. 3.2: grid points of scale 2n keep their flow as seeds (its
             * error re-evaluated at scale n); the new points start empty */
            for (long i = 0; i < NL; i++) {
                int gx = (int)(i % WL), gy = (int)(i / WL);
                set_invalid(&cur, i);
                if (gx % 2 == 0 && gy % 2 == 0) {
                    long j = (long)(gy / 2) * WP + gx / 2;
                    if (prev.fx[j] != INVALID_F) {
                        int32_t Fx = prev.fx[j], Fy = prev.fy[j];
                        cur.fx[i] = (int16_t)Fx;
                        cur.fy[i] = (int16_t)Fy;
                        cur.cost[i] = ffo_cost(f1L, f2L, C, W, H, L, gx * n, gy * n, Fx, Fy);
                        evals++;
                    }
                }
            }
            free(prev.fx);
            free(prev.fy);
            free(prev.cost);
        }
        int sweeps = (L == until_level) ? until_sweeps : ffo_schedule_sweeps(sch, I, L);
        for (int t = 0; t < sweeps; t++) {
            sweep(f1L, f2L, C, W, H, L, t % 4, &cur, &evals);
            if (ffo_schedule_rs_after(sch, I, L, t))
                random_search(f1L, f2L, C, W, H, L, t, dir,
                              prm->radius_q3 * ffo_schedule_radius_mult(sch, L, t), prm->seed,
                              pair_id, &cur, &evals);
        }
        prev = cur;
        WP = WL;
        HP = HL;
    }
    long NL = (long)WP * HP;
    for (long i = 0; i < NL; i++) {
        flow_out[2 * i] = prev.fx[i];
        flow_out[2 * i + 1] = prev.fy[i];
        if (cost_out) cost_out[i] = prev.cost[i];
    }
    free(prev.fx);
    free(prev.fy);
    free(prev.cost);
    if (evals_out) *evals_out = evals;
    return 0;
}

int ffo_match_features(const ffo_params *prm, const int8_t *fsrc, const int8_t *fdst,
                       int W, int H, int dir, uint32_t pair_id, const int16_t *seeds_in,
                       int until_level, int until_sweeps,
                       int16_t *flow_out, int32_t *cost_out, int64_t *evals_out) {
    return match_impl(prm, fsrc, fdst, W, H, dir, pair_id, seeds_in, NULL, until_level,
                      until_sweeps, flow_out, cost_out, evals_out);
}

int ffo_match_features_knn(const ffo_params *prm, const int8_t *fsrc, const int8_t *fdst,
                           int W, int H, int dir, uint32_t pair_id, const int32_t *knn_idx,
                           int until_level, int until_sweeps,
                           int16_t *flow_out, int32_t *cost_out, int64_t *evals_out) {
    if (!knn_idx) return 1;
    return match_impl(prm, fsrc, fdst, W, H, dir, pair_id, NULL, knn_idx, until_level,
                      until_sweeps, flow_out, cost_out, evals_out);
}

int ffo_match(const ffo_params *prm, const uint8_t *src, const uint8_t *dst, int W, int H,
              int dir, uint32_t pair_id, const int16_t *seeds_in,
              int until_level, int until_sweeps,
              int16_t *flow_out, int32_t *cost_out, int64_t *evals) {
    int C = prm->channels, S = prm->scales;
    if (C != 1 && C != 3) return 1;
    if (S < 1 || S > 8 || W < 1 || H < 1 || W > 4096 || H > 4096) return 1;
    long nb = ffo_feature_bytes(W, H, C, S);
    int8_t *fs = (int8_t *)malloc((size_t)nb);
    int8_t *fd = (int8_t *)malloc((size_t)nb);
    ffo_features_all(src, C, W, H, S, fs);
    ffo_features_all(dst, C, W, H, S, fd);
    int rc = ffo_match_features(prm, fs, fd, W, H, dir, pair_id, seeds_in, until_level,
                                until_sweeps, flow_out, cost_out, evals);
    free(fs);
    free(fd);
    return rc;
}

/* Sec. 3.7: keep p iff |F(p) + F_b(p + F(p))| < eps.  Reading: F_b is read at
 * the nearest point of the flows' grid to p + F(p) (rounded half up); a
 * target outside the grid or an INVALID flow rejects the point.  The grid is
 * the pixel grid, or the level-L grid (points (x n, y n), n = 2^L) for flows
 * that end on a coarser scale (Fast x2, Sec. 3.4). */
void ffo_filter_grid(const int16_t *fwd, const int16_t *bwd, int WL, int HL, int L, int eps_q3,
                     uint8_t *mask) {
    const int n = 1 << L;
    for (int y = 0; y < HL; y++)
        for (int x = 0; x < WL; x++) {
            long i = (long)y * WL + x;
            int Fx = fwd[2 * i], Fy = fwd[2 * i + 1];
            mask[i] = 0;
            if (Fx == INVALID_F || Fy == INVALID_F) continue;
            /* nearest grid point to (x n + Fx / 8) / n */
            int qx = x + floor_div(Fx + 4 * n, 8 * n), qy = y + floor_div(Fy + 4 * n, 8 * n);
            if (qx < 0 || qx >= WL || qy < 0 || qy >= HL) continue;
            long j = (long)qy * WL + qx;
            int Bx = bwd[2 * j], By = bwd[2 * j + 1];
            if (Bx == INVALID_F || By == INVALID_F) continue;
            long ddx = Fx + Bx, ddy = Fy + By;
            mask[i] = (ddx * ddx + ddy * ddy < (long)eps_q3 * eps_q3) ? 1 : 0;
        }
}

void ffo_filter(const int16_t *fwd, const int16_t *bwd, int W, int H, int eps_q3,
                uint8_t *mask) {
    ffo_filter_grid(fwd, bwd, W, H, 0, eps_q3, mask);
}

/* Sec. 3.7: with two backward flows (different random streams), a pixel is
 * deleted if it is not consistent with either of them. */
void ffo_filter2(const int16_t *fwd, const int16_t *bwd1, const int16_t *bwd2, int WL, int HL,
                 int L, int eps_q3, uint8_t *mask) {
    long n = (long)WL * HL;
    uint8_t *m2 = (uint8_t *)malloc((size_t)n);
    ffo_filter_grid(fwd, bwd1, WL, HL, L, eps_q3, mask);
    ffo_filter_grid(fwd, bwd2, WL, HL, L, eps_q3, m2);
    for (long i = 0; i < n; i++) mask[i] = (uint8_t)(mask[i] & m2[i]);
    free(m2);
}

/* Sec. 3.7, region filter.  Kept points (mask_in = 1) are segmented into
 * regions: two 4-neighbours belong to the same region when their flows
 * differ by less than 3 px (|F(p) - F(q)| < 24 in Q3; only neighbours'
 * differences count, so a region's flow may drift).  A region of fewer than
 * s points is removed when one of its points has a 4-neighbour that the
 * consistency check removed (mask_in = 0, flow set) and that the same rule
 * would join to it.  Regions are found by breadth-first search from each
 * unvisited kept point in raster order. */
static int close3(const int16_t *f, long a, long b) {
    long dx = (long)f[2 * a] - f[2 * b], dy = (long)f[2 * a + 1] - f[2 * b + 1];
    return dx * dx + dy * dy < 24L * 24L;
}

void ffo_region_filter(const int16_t *fwd, const uint8_t *mask_in, int W, int H, int s,
                       uint8_t *mask_out) {
    const long n = (long)W * H;
    long *queue = (long *)malloc(sizeof(long) * (size_t)(n > 0 ? n : 1));
    long *region = (long *)malloc(sizeof(long) * (size_t)(n > 0 ? n : 1));
    uint8_t *seen = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    const int ox[4] = {1, -1, 0, 0}, oy[4] = {0, 0, 1, -1};
    memcpy(mask_out, mask_in, (size_t)n);
    for (long start = 0; start < n; start++) {
        if (!mask_in[start] || seen[start]) continue;
        long head = 0, tail = 0, size = 0;
        int joins_outlier = 0;
        queue[tail++] = start;
        seen[start] = 1;
        while (head < tail) {
            long p = queue[head++];
            region[size++] = p;
            int x = (int)(p % W), y = (int)(p / W);
            for (int k = 0; k < 4; k++) {
                int qx = x + ox[k], qy = y + oy[k];
                if (qx < 0 || qx >= W || qy < 0 || qy >= H) continue;
                long q = (long)qy * W + qx;
                if (!close3(fwd, p, q)) continue;
                if (mask_in[q]) {
                    if (!seen[q]) {
                        seen[q] = 1;
                        queue[tail++] = q;
                    }
                } else if (fwd[2 * q] != INVALID_F && fwd[2 * q + 1] != INVALID_F) {
                    joins_outlier = 1;
                }
            }
        }
        if (size < s && joins_outlier)
            for (long i = 0; i < size; i++) mask_out[region[i]] = 0;
    }
    free(queue);
    free(region);
    free(seen);
}

/* Sec. 3.7-3.8 sparsification.  The grid is cut into q x q cells from the
 * origin (the last row and column of cells may be partial).  A cell that
 * still holds at least e kept points (mask_in = 1) keeps exactly one: the
 * point whose consistency errors |F(p) + F_b(p + F(p))|, summed over the
 * given backward flows (bwd2 may be NULL), are smallest; ties go to the
 * first point in raster order.  Errors are Euclidean lengths in 1/8 px,
 * each an IEEE double square root, summed in the order bwd1, bwd2.  The
 * backward flows are read at the grid point nearest to p + F(p), as in the
 * consistency check on the level-L grid; an unset flow or a target off the
 * grid (possible only for masks not made by the check) counts as infinite. */
static double check_error(const int16_t *fwd, const int16_t *bwd, int WL, int HL, int L, long i) {
    const int n = 1 << L;
    const int x = (int)(i % WL), y = (int)(i / WL);
    const int Fx = fwd[2 * i], Fy = fwd[2 * i + 1];
    if (Fx == INVALID_F || Fy == INVALID_F) return HUGE_VAL;
    const int qx = x + floor_div(Fx + 4 * n, 8 * n), qy = y + floor_div(Fy + 4 * n, 8 * n);
    if (qx < 0 || qx >= WL || qy < 0 || qy >= HL) return HUGE_VAL;
    const long j = (long)qy * WL + qx;
    const int Bx = bwd[2 * j], By = bwd[2 * j + 1];
    if (Bx == INVALID_F || By == INVALID_F) return HUGE_VAL;
    const long dx = (long)Fx + Bx, dy = (long)Fy + By;
    return sqrt((double)(dx * dx + dy * dy));
}

void ffo_sparsify(const int16_t *fwd, const int16_t *bwd1, const int16_t *bwd2,
                  const uint8_t *mask_in, int WL, int HL, int L, int q, int e,
                  uint8_t *mask_out) {
    memset(mask_out, 0, (size_t)WL * HL);
    for (int cy = 0; cy < HL; cy += q)
        for (int cx = 0; cx < WL; cx += q) {
            int count = 0;
            long best = -1;
            double best_err = 0.0;
            for (int y = cy; y < cy + q && y < HL; y++)
                for (int x = cx; x < cx + q && x < WL; x++) {
                    const long i = (long)y * WL + x;
                    if (!mask_in[i]) continue;
                    count++;
                    double err = check_error(fwd, bwd1, WL, HL, L, i);
                    if (bwd2) err = err + check_error(fwd, bwd2, WL, HL, L, i);
                    if (best < 0 || err < best_err) {
                        best = i;
                        best_err = err;
                    }
                }
            if (count >= e && best >= 0) mask_out[best] = 1;
        }
}
