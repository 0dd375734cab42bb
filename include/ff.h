/*
 * ff.h - C ABI of the GB300 Flow Fields patch-matching library (libff.so).
 *
 * Flow Fields (Bailer, Taetz, Stricker; arXiv 1703.02563) computes, for two
 * images I1 and I2, a correspondence field F(p) = M(p) - p for every pixel p
 * of I1 (Sec. 3, problem statement).  This library runs the method's
 * multi-scale patch-matching loop on one GPU:
 *
 *   ff_features  level images + WHT features of one frame     Sec. 3.1, 3.6
 *   ff_match     seeding, then per scale (coarse to fine)      Sec. 3.1 Eq. 1-2,
 *                propagation sweeps + random search            Sec. 3.2 Eq. 3-4
 *   ff_filter    forward/backward consistency check            Sec. 3.7
 *
 * Conventions shared by every call:
 *  - Every pointer argument is DEVICE memory unless the name ends in _host.
 *    The caller owns inputs and outputs and keeps them alive until the work
 *    is done; the context owns features, per-level state and scratch.
 *  - Calls are asynchronous on the context's current stream (ff_create /
 *    ff_set_stream) unless stated otherwise.  A device-side failure (a
 *    bounded wait that ran out) is recorded in the context and reported by
 *    ff_sync().
 *  - Flows are int16 pairs (x, y) in 1/8 pixel, row-major [H][W][2]; the
 *    value (-32768, -32768) marks an unset flow.  Costs are int32 [H][W]
 *    (sum of absolute feature differences scaled by 64; unset = INT32_MAX).
 *  - Status codes: FF_OK on success; FF_EINVAL for bad arguments (nothing is
 *    launched); FF_ENOMEM when device memory runs out in ff_create; FF_ECUDA
 *    when a CUDA call fails; FF_ETIMEOUT when a bounded device wait expired;
 *    FF_ESTATE when a call comes in the wrong order (e.g. ff_match before
 *    both frames have features).  ff_last_error() gives a message.
 *  - Results are bit-exact integers: the same inputs and config give the
 *    same flows, costs and masks on every run and in every call order.
 */
#ifndef FF_H
#define FF_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ff_ctx ff_ctx;

typedef enum {
    FF_OK = 0,
    FF_EINVAL = 1,
    FF_ENOMEM = 2,
    FF_ECUDA = 3,
    FF_ETIMEOUT = 4,
    FF_ESTATE = 5
} ff_status;

/* FF_BWD2: a second backward flow (slot 1 -> 0) with its own random stream,
 * for the two-way consistency check of Sec. 3.7. */
typedef enum { FF_FWD = 0, FF_BWD = 1, FF_BWD2 = 2 } ff_dir;

/* Sweep schedules per scale.
 * FF_SCHED_BASIC (Sec. 3.1-3.2): `iters` sweeps with radius R, a random
 *   search after each but the last.
 * FF_SCHED_PLUS (Flow Fields+, Sec. 3.3): 4 sweeps with R+ = 2R (3 random
 *   searches), then 8 sweeps with R (7 random searches); `iters` is unused.
 * FF_SCHED_PLUS_FAST (Flow Fields+ Fast, Sec. 3.4): as FF_SCHED_PLUS, but
 *   the finest scale runs only 4 sweeps with R (3 random searches).
 * FF_SCHED_PLUS_FAST_X2 (Flow Fields+ Fast x2, Sec. 3.4): the finest scale
 *   is not run; the 2nd-finest runs 4 sweeps with R and the coarser ones as
 *   FF_SCHED_PLUS.  Matches come on the level-1 grid, one per 2x2 region:
 *   the "final grid" below is [ceil(H/2)][ceil(W/2)] (points (2x, 2y)) for
 *   this schedule and the pixel grid [H][W] for the others.  The paper pairs
 *   it with seed_stride = 2.  Needs scales >= 2. */
typedef enum {
    FF_SCHED_BASIC = 0,
    FF_SCHED_PLUS = 1,
    FF_SCHED_PLUS_FAST = 2,
    FF_SCHED_PLUS_FAST_X2 = 3
} ff_schedule;

#define FF_MAX_SCALES 8
#define FF_MAX_LEAF 8
#define FF_MAX_DIM 4096

/* Parameters of the method (Sec. 4.1 gives the paper's values). */
typedef struct {
    int patch;        /* WHT window side, must be 8 (offsets -3..+4, Sec. 3.1 footnote) */
    int n_coeffs;     /* WHT bases per channel, must be 9 (Sec. 3.1)                     */
    int channels;     /* 1 (gray) or 3 (8-bit CIELab, Sec. 3.1)                          */
    int scales;       /* S levels; the coarsest scale is n = 2^(S-1) (k = S-1, Sec. 3.2) */
    int iters;        /* I propagation sweeps per level, I-1 random searches (Sec. 3.1)  */
    int radius_q3;    /* random-search radius R in 1/8 px; R_n = R n (Sec. 3.2)          */
    int seed_leaf;    /* l seeding candidates kept per point, 1..8 (Sec. 3.1, l = 8)     */
    int seed_stride;  /* candidate grid stride in I2 (1; 2 = the Fast x2 option)         */
    int eps_q3;       /* consistency threshold eps in 1/8 px (Sec. 3.7)                  */
    uint32_t seed;    /* random-search key word 0                                        */
    int max_width;    /* largest frame the context must hold, 1..4096                     */
    int max_height;
    int schedule;     /* an ff_schedule value                                             */
    int region_min;   /* s of the region filter (Sec. 3.7) applied after the consistency  */
                      /* check by ff_pair_host and ff_batch_run; 0 = off (default)        */
    int wht_tensor_cores; /* 1: ff_features computes the WHT on the bf16 tensor cores     */
                      /* (FP32 accumulation; exact, so the int8 features are identical)  */
} ff_config;

/* Fills the paper's defaults: patch 8, 9 coefficients, 1 channel, S = 4,
 * I = 4, R = 1 px, l = 8, stride 1, eps = 1 px, max 1024 x 1024, basic schedule. */
ff_status ff_config_default(ff_config *cfg);

/* Creates a context on `device` and allocates all its device memory for
 * frames up to max_width x max_height.  cuda_stream: a cudaStream_t (NULL =
 * the legacy default stream).  *out receives the context. */
ff_status ff_create(const ff_config *cfg, int device, void *cuda_stream, ff_ctx **out);

/* Makes later calls enqueue on another stream.  Features and matching state
 * of the two slots / directions are separate buffers, so ff_features of
 * slot 0 and of slot 1 may run concurrently on two streams, and so may
 * ff_match(FF_FWD) and ff_match(FF_BWD) once both frames' features are
 * complete (ordering them is the caller's job). */
ff_status ff_set_stream(ff_ctx *ctx, void *cuda_stream);

/* Sec. 3.1 + 3.6: builds the S level images of one frame (n x n area
 * average, replicate border) and their int8 WHT features into the
 * context.  slot 0 = I1, slot 1 = I2.  img: device uint8, planar
 * [channels][h][pitch], pitch >= w.  1 <= w <= max_width, 1 <= h <= max_height. */
ff_status ff_features(ff_ctx *ctx, int slot, const uint8_t *img, int w, int h, int pitch);

/* Sec. 3.1-3.2: matches slot 0 -> 1 (FF_FWD) or 1 -> 0 (FF_BWD, FF_BWD2).  Each
 * direction has its own state, so the three may run on three streams.  Both slots
 * must hold features of the same size.  pair_id: random-search key word 1.
 * seeds_in: NULL (seed by the exact top-l WHT search, Eq. 1/4) or int16
 * [H_c][W_c][2] flows on the coarsest grid (H_c = ceil(h / 2^(S-1))).
 * flow_out: int16 [h][w][2]; cost_out: int32 [h][w] or NULL (the final grid
 * of the schedule: [ceil(h/2)][ceil(w/2)] for Fast x2).  Both 4-byte
 * aligned. */
ff_status ff_match(ff_ctx *ctx, ff_dir dir, uint32_t pair_id, const int16_t *seeds_in,
                   int16_t *flow_out, int32_t *cost_out);

/* As ff_match, but stops at level `until_level` after `until_sweeps` sweeps
 * (each followed by its random search when one follows it) and writes that
 * level's grid: flow_out int16 [H_L][W_L][2], cost_out int32 [H_L][W_L].
 * until_sweeps = 0 returns the level's initial state (seeds or upsampled
 * flows).  until_level >= 1 under Fast x2.  Used to check each stage of the
 * method. */
ff_status ff_match_until(ff_ctx *ctx, ff_dir dir, uint32_t pair_id, const int16_t *seeds_in,
                         int until_level, int until_sweeps, int16_t *flow_out,
                         int32_t *cost_out);

/* Sec. 3.7: mask[p] = 1 iff |F(p) + F_b(q)| < eps, q = the point of the
 * final grid nearest to p + F(p) (rounded half up); 0 when q is outside the
 * grid or a flow is unset.  flow_fwd / flow_bwd: int16 [h][w][2] of the last
 * ff_features size ([ceil(h/2)][ceil(w/2)][2] for Fast x2); mask_out: uint8
 * of the same grid. */
ff_status ff_filter(ff_ctx *ctx, const int16_t *flow_fwd, const int16_t *flow_bwd,
                    uint8_t *mask_out);

/* Sec. 3.7, two backward flows: mask[p] = 1 iff p passes the check of
 * ff_filter against flow_bwd1 and against flow_bwd2 (a pixel inconsistent
 * with either backward flow is deleted).  Same layouts as ff_filter. */
ff_status ff_filter_2way(ff_ctx *ctx, const int16_t *flow_fwd, const int16_t *flow_bwd1,
                         const int16_t *flow_bwd2, uint8_t *mask_out);

/* Sec. 3.7 region filter.  Kept points of mask_in are segmented into
 * regions: 4-neighbours whose forward flows differ by less than 3 px
 * (squared Q3 distance < 24^2) share a region.  A region of fewer than
 * min_region points is deleted when one of its points has a 4-neighbour that
 * mask_in rejects, whose flow is set, and that the same rule would join to
 * it.  flow_fwd: int16 final grid [..][..][2]; mask_in / mask_out: uint8 on
 * the same grid (they may be the same buffer).  Uses context scratch, so
 * calls on one context run in stream order. */
ff_status ff_region_filter(ff_ctx *ctx, const int16_t *flow_fwd, const uint8_t *mask_in,
                           int min_region, uint8_t *mask_out);

/* Sec. 3.7-3.8 sparsification before dense interpolation.  The final grid
 * is cut into q x q cells from its origin (border cells may be partial).  A
 * cell holding at least e points of mask_in keeps exactly one in mask_out:
 * the one whose consistency errors |F(p) + F_b(q)| (q as in ff_filter),
 * summed over flow_bwd1 and flow_bwd2, are smallest (flow_bwd2 NULL: one
 * backward flow).  Errors are IEEE double lengths in 1/8 px added in that
 * order; an unset flow or q off the grid counts as infinite; ties go to the
 * first point in raster order.  Other points get 0.  1 <= q <= 64, e >= 0.
 * mask_in and mask_out may be the same buffer. */
ff_status ff_sparsify(ff_ctx *ctx, const int16_t *flow_fwd, const int16_t *flow_bwd1,
                      const int16_t *flow_bwd2, const uint8_t *mask_in, int q, int e,
                      uint8_t *mask_out);

/* Whole pair with HOST buffers (blocking): copies both frames in (planar
 * uint8 [channels][h][w]), builds features, matches forward and backward
 * concurrently, filters (and region-filters when cfg.region_min > 0), and
 * copies the results out: flow_fwd_host and
 * flow_bwd_host int16 [h][w][2], mask_host uint8 [h][w] (on the final grid
 * of the schedule; any may be NULL to skip its copy).  Pinned host memory makes the copies asynchronous.
 * Returns after the results are on the host. */
ff_status ff_pair_host(ff_ctx *ctx, const uint8_t *img1_host, const uint8_t *img2_host,
                       int w, int h, uint32_t pair_id, int16_t *flow_fwd_host,
                       int16_t *flow_bwd_host, uint8_t *mask_host);

/* The WHT of ff_features on the bf16 tensor cores, before quantisation:
 * coeffs_out float [H_L][W_L][9 * channels] (dimension ch*9 + 3u + v) of
 * level `level` of a device frame img (planar [channels][h][pitch]).  With
 * 8-bit level images and +-1 bases every product and partial sum is an
 * integer below 2^24, so the values are exact.  Stateless; enqueued on
 * cuda_stream.  No paper counterpart: it exposes the intermediate for the
 * precision check against an FP64 transform. */
ff_status ff_wht_coeffs_tc(const uint8_t *img, int w, int h, int pitch, int channels, int level,
                           float *coeffs_out, void *cuda_stream);

/* The precision form of the WHT: the transform of the FP32 scale-space
 * image, i.e. level `level`'s n x n area average without rounding (Sec. 3.6,
 * replicative border; exact in FP32), rounded to bf16 (fp16 = 0) or fp16
 * (fp16 = 1) and multiplied with the +-1 Walsh basis on the tensor cores
 * with FP32 accumulation.  coeffs_out float [H_L][W_L][9 * channels]
 * (dimension ch*9 + 3u + v); img planar [channels][h][pitch] on the device.
 * At level 0 the inputs are 8-bit integers, exact in both formats, so the
 * result equals the exact transform; at level >= 1 each input is rounded to
 * the nearest value of its format, at most half a unit in the last place
 * (below 256: 0.5 for bf16, 1/16 for fp16), so a coefficient is within 64
 * such half-units (32 and 4) plus the FP32 accumulation error of the FP64
 * transform.  Matching never uses these values: ff_features quantises the
 * rounded integer level image.  Stateless; enqueued on cuda_stream.  No
 * paper counterpart: the paper's WHT is floating point on the CPU; this
 * measures what the tensor-core formats lose against FP64. */
ff_status ff_wht_coeffs_scalespace_tc(const uint8_t *img, int w, int h, int pitch, int channels,
                                      int level, int fp16, float *coeffs_out, void *cuda_stream);

/* Copies level `level` of slot `slot`'s features to dst: int8
 * [H_L][W_L][9 * channels] (dense, dimension index ch*9 + 3u + v). */
ff_status ff_get_features(ff_ctx *ctx, int slot, int level, int8_t *dst);

/* Runs only the seeding search of ff_match(dir) and writes, per coarsest
 * grid point, the l nearest I2 pixels: idx_out int32 [H_c][W_c][l] (linear
 * index y*w + x, -1 if fewer candidates exist) and dist_out int32
 * [H_c][W_c][l] (squared feature distance), ascending by (dist, idx). */
ff_status ff_seed_knn(ff_ctx *ctx, ff_dir dir, int32_t *idx_out, int32_t *dist_out);

/* Allocation-free seeding search.  The paper has no counterpart: this is an
 * interface for callers that cannot allocate device memory, for example a
 * plug-in running inside a host application that owns every allocation and
 * hands libraries a fixed budget, or a real-time loop that must never wait
 * on the allocator (cudaMalloc and cudaFree can synchronise the device and
 * stall every stream).  It computes what ff_seed_knn computes, without a
 * context, and allocates nothing: its scratch (the per-chunk partial lists)
 * is an 8 MiB array in the library's static device memory, which every GPU
 * that loads the library holds until the process exits.
 *  feat_src0 / feat_dst0: level-0 features of the query and the candidate
 *    frame, int8 [h][w][P] (P = 16 for 1 channel, 32 for 3: the 9*channels
 *    codes of ff_get_features, then zero bytes), 16-byte aligned.
 *  idx_out / dist_out: int32 [H_c][W_c][leaf], as ff_seed_knn.
 *  cuda_stream: the stream to enqueue on (NULL = legacy default stream).
 *  why: NULL, or receives a static message when the call is rejected.
 * The first call on a device, and the first after that device's context was
 * re-created, looks up the scratch's device address with that device
 * current; make that first call before any stream capture.  Every call
 * shares the scratch, which keeps the last call's contents, so calls that
 * overlap on a GPU race: order them on one stream.  Nothing in the scratch
 * needs clearing: each call writes every list it reads.  Returns FF_EINVAL
 * (nothing launched) for bad arguments, including more than 131072
 * coarsest-grid points, which is the scratch limit, and FF_ECUDA if a CUDA
 * error from earlier work is still pending (nothing launched), if the
 * set-up fails or if a launch fails. */
ff_status ff_seed_knn_static(const int8_t *feat_src0, const int8_t *feat_dst0, int w, int h,
                             int channels, int scales, int leaf, int stride, int32_t *idx_out,
                             int32_t *dist_out, void *cuda_stream, const char **why);

/* Ceilings of the running GPU, measured by microbenchmarks, for quoting the
 * matching kernels against what this device can do (no counterpart in the
 * paper, which reports CPU runtimes only).  Throughputs are whole-GPU rates
 * at full occupancy: dp4a instructions (each 4 byte multiply-adds into an
 * int32), three-input adds and 32-bit multiply-adds per second; the matching
 * error's own arithmetic per feature dimension (byte transpose of the four
 * bilinear taps, one dp4a forming the interpolation minus 64 q, absolute
 * value, accumulation) in dimensions per second, from registers; and the
 * read bandwidth of a 48 MB buffer resident in L2 (loads that skip L1).
 * Latencies are SM clock cycles per instruction of a dependent chain run by
 * one warp: integer add or xor, byte permute, dp4a, warp shuffle, shared load,
 * global load hitting L1, global load hitting L2.  The call allocates its
 * own buffers and stream, runs for a few tens of milliseconds and returns
 * when done.  FF_EINVAL for a NULL out or a bad device, FF_ECUDA if a CUDA
 * call fails. */
typedef struct {
    int sm_count;
    double dp4a_per_s, iadd3_per_s, imad_per_s, sad_dims_per_s, l2_read_gbs;
    double lat_alu, lat_prmt, lat_dp4a, lat_shfl, lat_lds, lat_ldg_l1, lat_ldg_l2;
} ff_peaks;
ff_status ff_measure_peaks(int device, ff_peaks *out);

/* Blocks until the context's work is done; returns FF_ETIMEOUT if a bounded
 * device wait expired since the last ff_sync (and clears the record). */
ff_status ff_sync(ff_ctx *ctx);

/* Test and tuning hooks.  FF_DEBUG_WAIT_LIMIT_NS: upper bound of every
 * device-side wait (default 2 s).  FF_DEBUG_FORCE_TIMEOUT: when nonzero, the
 * next propagation sweeps wait for a boundary row that is never written, so
 * the bounded wait runs out and ff_sync reports FF_ETIMEOUT.
 * FF_DEBUG_SWEEP_LANES: lanes of the sweep's propagation warp per grid point,
 * 4 (default: each candidate's cost split over two lanes, 8 rows per strip)
 * or 2 (one lane per candidate, 16 rows per strip: fewer instructions per
 * point, a longer step).  FF_DEBUG_SEED_TC: 1 (default) runs the seeding
 * search's full pass on the tcgen05 tensor cores, 0 on mma.sync.  Every value
 * gives the same results. */
typedef enum {
    FF_DEBUG_WAIT_LIMIT_NS = 1,
    FF_DEBUG_FORCE_TIMEOUT = 2,
    FF_DEBUG_SWEEP_LANES = 4,
    FF_DEBUG_SEED_TC = 5
} ff_debug_key;
ff_status ff_debug_set(ff_ctx *ctx, ff_debug_key key, long long value);

/* Launch timing for measurement, with CUDA events on the stream each kernel
 * is launched on.  FF_PROFILE_LAUNCHES brackets every kernel launch with an
 * event pair.  FF_PROFILE_SWEEP_RUNS records only the sweep kernel, with one
 * pair around each run of consecutive sweep launches on a stream (a level's
 * sweeps), so that timing the dominant kernel adds a few events per match
 * instead of two per launch (per-launch events cost about 2% of a pair's
 * time); a run's time includes the launch gaps inside it.  ff_profile(ctx,
 * mode) clears the record and starts recording; ff_profile(ctx, 0) stops (an
 * open run ends there).  Any other mode: FF_EINVAL.  ff_kernel_stats (call
 * after ff_sync) returns, for the kernel named `kernel` ("k_features",
 * "k_seed_prep", "k_seed_scan", "k_seed_merge", "k_seed_rerank",
 * "k_seed_given", "k_upsample", "k_sweep", "k_export", "k_filter", "k_dense",
 * "k_region", "k_sparsify"), the number of recorded launches and their summed
 * device time in milliseconds. */
typedef enum { FF_PROFILE_LAUNCHES = 1, FF_PROFILE_SWEEP_RUNS = 2 } ff_profile_mode;
ff_status ff_profile(ff_ctx *ctx, int mode);
ff_status ff_kernel_stats(ff_ctx *ctx, const char *kernel, long long *launches,
                          double *total_ms);

/* Number of kernel launches this context has made so far. */
long long ff_launch_count(const ff_ctx *ctx);

const char *ff_last_error(const ff_ctx *ctx);
const char *ff_status_string(ff_status s);
void ff_destroy(ff_ctx *ctx);

/* ---- Batched form --------------------------------------------------------
 * Many frame pairs of mixed sizes in flight at once.  The paper matches one
 * pair at a time (Sec. 3); this form has no counterpart there.  It changes
 * nothing in what a pair computes: every pair's flows and mask equal those of
 * ff_features + ff_match + ff_filter (or ff_filter_2way) on one context with
 * the same config and pair_id.
 *
 * A batch owns `slots` matching slots; each holds its own features, states
 * and streams for frames up to cfg.max_width x cfg.max_height.  ff_batch_run
 * deals pairs round-robin to the slots: pairs in different slots overlap on
 * the device, so their sweeps' wavefronts share the SMs; pairs in one slot
 * run in order. */
typedef struct ff_batch ff_batch;

typedef struct {
    const uint8_t *img1;  /* device, planar uint8 [channels][h][pitch]; read only     */
    const uint8_t *img2;
    int w, h, pitch;      /* 1 <= w <= max_width, 1 <= h <= max_height, pitch >= w     */
    uint32_t pair_id;     /* random-search key word 1                                  */
    int16_t *flow_fwd;    /* device, final grid [..][..][2] (see ff_schedule); required */
    int16_t *flow_bwd;    /* device, final grid; required                              */
    int16_t *flow_bwd2;   /* device, final grid, or NULL: one backward flow            */
    uint8_t *mask;        /* device, final grid, or NULL: no filter                    */
} ff_pair_desc;

/* Creates a batch of `slots` (1..256) slots on `device`; the work of each
 * ff_batch_run joins back into cuda_stream (NULL = legacy default stream).
 * Allocates all device memory up front: per slot, what ff_create allocates,
 * plus one stream. */
ff_status ff_batch_create(const ff_config *cfg, int device, int slots, void *cuda_stream,
                          ff_batch **out);

/* Enqueues n pairs (n >= 0) and returns without waiting; the batch's stream
 * is ordered after all of them.  The caller owns every buffer and keeps it
 * alive until that point; output buffers of different pairs must not
 * overlap.  Descriptors are checked before anything is enqueued (FF_EINVAL,
 * nothing launched).  use_graph != 0: the whole enqueue is captured as one
 * CUDA graph and launched; a later call with the same n and identical
 * descriptors relaunches that graph without capturing again. */
ff_status ff_batch_run(ff_batch *b, int n, const ff_pair_desc *pairs, int use_graph);

/* Makes later ff_batch_run calls join into another stream. */
ff_status ff_batch_set_stream(ff_batch *b, void *cuda_stream);

/* Waits for the device and reports FF_ETIMEOUT if a bounded wait of any
 * slot expired (the words are cleared). */
ff_status ff_batch_sync(ff_batch *b);

/* ff_debug_set on every slot (a captured graph is dropped). */
ff_status ff_batch_debug_set(ff_batch *b, ff_debug_key key, long long value);

/* Kernel launches made by this batch so far (graph relaunches included). */
long long ff_batch_launch_count(const ff_batch *b);

const char *ff_batch_last_error(const ff_batch *b);
void ff_batch_destroy(ff_batch *b);

/* ---- Serving loop ---------------------------------------------------------
 * Continuous admission of frame-pair requests with HOST buffers.  Like the
 * batched form it has no counterpart in the paper and changes nothing in
 * what a pair computes.  A server owns as many slots as its device-memory
 * budget holds (ff_slot_bytes each, at most max_slots); each slot keeps its
 * pyramids, states and staging resident on the device.  A request goes into
 * the first free slot as soon as there is one, so requests that arrive while
 * others run overlap with them on the device; the rest wait in arrival
 * order.  Calls are not thread-safe: one host thread drives a server. */
typedef struct ff_server ff_server;

typedef struct {
    const uint8_t *img1;  /* host, planar uint8: channel k, row y, column x at        */
    const uint8_t *img2;  /*   img[k * plane + y * pitch + x]; read until completion  */
    int w, h, pitch;      /* 1 <= w <= max_width, 1 <= h <= max_height, pitch >= w     */
    long long plane;      /* elements between channel planes, >= (h - 1) * pitch + w  */
    uint32_t pair_id;     /* random-search key word 1                                  */
    int two_way;          /* nonzero: second backward flow and two-way check          */
    int16_t *flow_fwd;    /* host, final grid [..][..][2], or NULL                     */
    int16_t *flow_bwd;    /* host or NULL                                              */
    int16_t *flow_bwd2;   /* host or NULL (used when two_way)                          */
    uint8_t *mask;        /* host, final grid, or NULL; region-filtered when           */
                          /*   cfg.region_min > 0                                      */
} ff_host_pair;

/* Device bytes one slot (one context) of this config holds. */
size_t ff_slot_bytes(const ff_config *cfg);

/* Creates min(max_slots, mem_budget / ff_slot_bytes(cfg)) slots on `device`
 * (FF_ENOMEM if not even one fits). */
ff_status ff_server_create(const ff_config *cfg, int device, size_t mem_budget, int max_slots,
                           ff_server **out);
int ff_server_slots(const ff_server *srv);

/* Queues a request (the descriptor is copied; the buffers it points to must
 * live until the request completes), admits what fits and returns at once.
 * *ticket (may be NULL) receives its number: 0, 1, 2, ... in submit order. */
ff_status ff_server_submit(ff_server *srv, const ff_host_pair *req, long long *ticket);

/* Retires finished requests without waiting: writes up to cap (ticket,
 * status) pairs, *n_done of them (status FF_OK, FF_ETIMEOUT when a bounded
 * device wait expired, FF_ECUDA), then admits queued requests into the
 * freed slots.  A retired request's outputs are on the host. */
ff_status ff_server_poll(ff_server *srv, long long *tickets, int *status, int cap, int *n_done);

/* Requests submitted and not yet retired. */
int ff_server_pending(const ff_server *srv);

long long ff_server_launch_count(const ff_server *srv);
const char *ff_server_last_error(const ff_server *srv);
/* Waits for the device, then frees everything (unretired results are lost). */
void ff_server_destroy(ff_server *srv);

#ifdef __cplusplus
}
#endif
#endif
