/*
 * ffo.h - CPU oracle of the Flow Fields multi-scale patch-matching loop.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, sequential definition
 * of what the CUDA library computes; it exists so tests, the smoke check and
 * the CPU baseline of the benchmark can compare against it.  The product
 * path never links, loads or calls it, and it shares no code with the CUDA
 * sources (not even headers or constants).
 *
 * Method: Bailer, Taetz, Stricker, "Flow Fields: Dense Correspondence Fields
 * for Highly Accurate Large Displacement Optical Flow Estimation" (TPAMI
 * extension, arXiv 1703.02563), Sec. 3.1 (basic Flow Fields: WHT vectors,
 * seeding + reranking Eq. 1, propagation Eq. 2, random search), Sec. 3.2
 * (multi-scale scheme, Eqs. 3-4), Sec. 3.6 (area downsampling, replicative
 * border) and Sec. 3.7 (forward/backward consistency check).
 *
 * All buffers are host memory owned by the caller.  Images are planar uint8
 * [C][H][W]; features are int8 [H_L][W_L][9C] per level (dense, dim index
 * ch*9 + 3u + v); flows are int16 pairs (x, y) in 1/8 pixel (Q3); costs are
 * int32.  INVALID flow = (-32768, -32768) with cost INT32_MAX.
 */
#ifndef FFO_H
#define FFO_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int channels;     /* 1 or 3                                  */
    int scales;       /* S: number of levels, coarsest n = 2^(S-1) */
    int iters;        /* I: propagation sweeps per level           */
    int radius_q3;    /* random-search radius R in 1/8 px          */
    int seed_leaf;    /* l: candidates kept by the seeding search  */
    int seed_stride;  /* sigma: candidate grid stride in image 2   */
    uint32_t seed;    /* Philox key word 0                         */
    int schedule;     /* 0 basic, 1 Flow Fields+, 2 Flow Fields+ Fast, 3 Fast x2 */
} ffo_params;

/* The sweep schedule of one level: number of sweeps, and for sweep t the
 * random-search radius multiplier (1 or 2) and whether a random search
 * follows it. */
int ffo_schedule_sweeps(int schedule, int iters, int L);
/* the finest level a schedule runs (1 for Fast x2, else 0) */
int ffo_schedule_final_level(int schedule);
int ffo_schedule_radius_mult(int schedule, int L, int t);
int ffo_schedule_rs_after(int schedule, int iters, int L, int t);

/* level grid size for scale n = 2^L: ceil(W/n) x ceil(H/n) */
void ffo_level_dims(int W, int H, int L, int *WL, int *HL);
/* byte offset of level L inside the concatenated feature buffer of all levels */
long ffo_feature_offset(int W, int H, int C, int L);
long ffo_feature_bytes(int W, int H, int C, int S);

/* D_n: n x n area average (round half up) with replicate border, n = 2^L */
void ffo_level_image(const uint8_t *img, int C, int W, int H, int L, uint8_t *out);
/* raw 3x3 lowest-sequency Walsh coefficients c_uv, int32 [HL][WL][9C] */
void ffo_wht_coeffs(const uint8_t *D, int C, int WL, int HL, int32_t *out);
/* quantise one coefficient (u,v) to int8 */
int ffo_quantise(int32_t c, int uv_is_dc);
/* quantised features of one level, int8 [HL][WL][9C] */
void ffo_wht_features(const uint8_t *D, int C, int WL, int HL, int8_t *out);
/* all S levels of one image, concatenated (offsets from ffo_feature_offset) */
void ffo_features_all(const uint8_t *img, int C, int W, int H, int S, int8_t *out);

/* Philox4x32 with 10 rounds (Salmon et al., SC'11) */
void ffo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* clamp flow (in place) so that 8p + F lies inside [0,8(W-1)] x [0,8(H-1)] */
void ffo_clamp_flow(int W, int H, int px, int py, int32_t *Fx, int32_t *Fy);
/* matching error E of grid point p (full-res px,py; level L) under flow F (Q3) */
int32_t ffo_cost(const int8_t *f1L, const int8_t *f2L, int C, int W, int H, int L,
                 int px, int py, int32_t Fx, int32_t Fy);

/* exact top-l seeding search for every coarsest-grid point (level S-1).
 * knn_idx / knn_dist: [N_{S-1}][l], linear index y2*W + x2 / squared distance,
 * ascending by (dist, index); unused slots get -1.  Returns the slots filled. */
int ffo_seed_knn(const int8_t *f1_0, const int8_t *f2_0, int C, int W, int H, int S,
                 int leaf, int stride, int32_t *knn_idx, int32_t *knn_dist);

/* the same search restricted to coarsest-grid rows gy0 <= gy < gy1 (the
 * outputs are still indexed by the full grid) */
int ffo_seed_knn_rows(const int8_t *f1_0, const int8_t *f2_0, int C, int W, int H, int S,
                      int leaf, int stride, int gy0, int gy1, int32_t *knn_idx,
                      int32_t *knn_dist);

/* single steps on one level's state: flow int16 [HL][WL][2], cost int32
 * [HL][WL], both updated in place; d = direction 0..3, t = sweep index */
void ffo_sweep_level(const int8_t *f1L, const int8_t *f2L, int C, int W, int H, int L, int d,
                     int16_t *flow, int32_t *cost, int64_t *evals);
void ffo_random_search_level(const int8_t *f1L, const int8_t *f2L, int C, int W, int H, int L,
                             int t, int dir, int radius_q3, uint32_t seed, uint32_t pair_id,
                             int16_t *flow, int32_t *cost, int64_t *evals);

/* Full matching of src -> dst features (all levels, concatenated).
 * dir: 0 forward, 1 backward, 2 second backward (Philox counter word 3;
 * Sec. 3.7's second backward flow differs from the first only in its random
 * stream).  seeds_in: NULL or int16 [H_{S-1}][W_{S-1}][2] flows replacing the
 * seeding search.  Stops at level until_level after until_sweeps sweeps (each
 * followed by its random search when one follows it); the defaults are 0 and
 * the schedule's sweep count of level 0.  Writes
 * that level's grid: flow_out int16 [HL][WL][2], cost_out int32 [HL][WL].
 * evals (may be NULL) receives the number of cost evaluations performed.
 * Returns 0 on success, nonzero on bad arguments. */
int ffo_match_features(const ffo_params *prm, const int8_t *fsrc, const int8_t *fdst,
                       int W, int H, int dir, uint32_t pair_id, const int16_t *seeds_in,
                       int until_level, int until_sweeps,
                       int16_t *flow_out, int32_t *cost_out, int64_t *evals);

/* the same with the seeding search's lists given: knn_idx [N_{S-1}][l] as
 * ffo_seed_knn (or ffo_seed_knn_rows over all rows) writes them; the Eq. 1
 * rerank and everything after it run here */
int ffo_match_features_knn(const ffo_params *prm, const int8_t *fsrc, const int8_t *fdst,
                           int W, int H, int dir, uint32_t pair_id, const int32_t *knn_idx,
                           int until_level, int until_sweeps,
                           int16_t *flow_out, int32_t *cost_out, int64_t *evals);

/* same, computing the features of both images first */
int ffo_match(const ffo_params *prm, const uint8_t *src, const uint8_t *dst, int W, int H,
              int dir, uint32_t pair_id, const int16_t *seeds_in,
              int until_level, int until_sweeps,
              int16_t *flow_out, int32_t *cost_out, int64_t *evals);

/* forward/backward consistency check: mask 1 keeps a pixel */
void ffo_filter(const int16_t *fwd, const int16_t *bwd, int W, int H, int eps_q3,
                uint8_t *mask);
/* the same on the level-L grid [HL][WL] (points (x 2^L, y 2^L)) */
void ffo_filter_grid(const int16_t *fwd, const int16_t *bwd, int WL, int HL, int L, int eps_q3,
                     uint8_t *mask);
/* two backward flows on the level-L grid: a point is kept only if consistent
 * with both */
void ffo_filter2(const int16_t *fwd, const int16_t *bwd1, const int16_t *bwd2, int WL, int HL,
                 int L, int eps_q3, uint8_t *mask);

/* Sec. 3.7 region filter on a grid [H][W]: mask_out = mask_in minus every
 * region (4-neighbours with flows less than 3 px apart) of fewer than s
 * points that the same rule would join to a point the consistency check
 * removed (mask_in = 0, flow set). */
void ffo_region_filter(const int16_t *fwd, const uint8_t *mask_in, int W, int H, int s,
                       uint8_t *mask_out);

/* Sec. 3.7-3.8 sparsification on the level-L grid [HL][WL]: in each q x q
 * cell with at least e kept points, keep the one with the smallest summed
 * consistency error over bwd1 and bwd2 (NULL: bwd1 only). */
void ffo_sparsify(const int16_t *fwd, const int16_t *bwd1, const int16_t *bwd2,
                  const uint8_t *mask_in, int WL, int HL, int L, int q, int e,
                  uint8_t *mask_out);

#ifdef __cplusplus
}
#endif
#endif
