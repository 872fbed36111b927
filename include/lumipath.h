/*
 * lumipath.h -- C ABI of the GB300 light-field sampling library.
 *
 * The library samples the light field of LumiPath (Fink et al., arXiv
 * 1903.03837, Section 2). A bounding sphere S (radius R, centre O) carries two
 * spherical-Fibonacci (SF) point sets: M ray origins P_o and N "directions"
 * P_d (exit points on S). The radiance table L^(i,j) holds one texel per
 * origin/exit pair. For each camera ray the library
 *   1. intersects the ray with S (front hit h_o, back hit h_d; tangential rays
 *      are discarded),
 *   2. finds the 5 nearest points of P_o to h_o and of P_d to h_d (the inverse
 *      SF mapping, extended to five neighbours),
 *   3. weights each neighbour with the distance filter kernel of radius
 *      R*5^(1/4)*sqrt(4*pi/(sqrt(5)*n)) (= R*sqrt(4*pi/n)), tent-shaped,
 *   4. blends the 25 texels L^(i_a, j_b) with the product weights.
 *
 * All entry points are plain C: device pointers are CUDA global-memory
 * addresses on the current device, host pointers are ordinary memory, and
 * `stream` is a cudaStream_t (NULL = legacy default stream). Every call
 * returns an lf_status and never aborts; lf_last_error() gives the message of
 * the calling thread's last failure. Work is enqueued on `stream` and is
 * asynchronous unless stated otherwise.
 */
#ifndef LUMIPATH_H
#define LUMIPATH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum lf_status {
    LF_OK = 0,
    LF_ERR_INVALID_ARG = 1,    /* a null pointer, a size out of range, a bad enum */
    LF_ERR_OUT_OF_MEMORY = 2,  /* a device allocation failed */
    LF_ERR_CUDA = 3,           /* a CUDA runtime call or launch failed */
    LF_ERR_UNSUPPORTED = 4,    /* valid but not implemented combination */
    LF_ERR_TIMEOUT = 5,        /* a bounded device wait gave up */
    LF_ERR_DEVICE_CHECK = 6    /* a device-side check set the table's status word */
} lf_status;

/* Storage type of the radiance table. FP16 and E4M3 tables carry one FP32
 * scale per origin row: texel value = scale[i] * decode(code). */
typedef enum lf_dtype {
    LF_DTYPE_F32 = 0,
    LF_DTYPE_F16 = 1,          /* IEEE 754 binary16 */
    LF_DTYPE_E4M3 = 2          /* OCP FP8 E4M3FN (bias 7, max 448, no inf) */
} lf_dtype;

/* lf_table_desc.flags */
#define LF_TABLE_BORROW 0x1u   /* keep the caller's device pointers instead of copying */
/* Only the origin rows of the upper hemisphere are stored (Section 3: z_i > 0,
 * i.e. i < M/2): the table has floor(M/2) rows (and scales). Origin neighbours
 * outside the stored rows are dropped and the remaining origin weights
 * renormalised; a ray whose 5 origin neighbours are all unstored is masked
 * (written as a miss). */
#define LF_TABLE_UPPER_HEMISPHERE 0x2u

/* Description of a light-field table (Section 2: sphere S with radius R and
 * origin O; point counts M and N; the texture L^(i,j) of M x N texels). */
typedef struct lf_table_desc {
    double radius;             /* R > 0, finite */
    double center[3];          /* O, finite */
    uint32_t n_origins;        /* M, 1 <= M <= 2^24 */
    uint32_t n_directions;     /* N, 1 <= N <= 2^24 */
    uint32_t channels;         /* C in {3, 4} */
    int32_t dtype;             /* lf_dtype */
    uint32_t flags;            /* LF_TABLE_* */
    uint32_t k_nearest;        /* neighbours per hit: 5 (0 means 5), 1 for nearest sampling, or 9
                                  (the "up to nine" of Section 2: 9 x 9 = 81 taps per ray) */
} lf_table_desc;

/* A pinhole camera. Pixel (x, y) of a W x H image looks along
 *   v = forward + ((x+0.5) * s_w - 1) * tan_half_x * right
 *               + (1 - (y+0.5) * s_h) * tan_half_y * up,
 *   d = v * (1 / sqrt(v.v)),
 * from `eye`, where s_w = 2/W and s_h = 2/H are rounded to FP32 once; every
 * other operation is one FP32 IEEE operation in exactly this order (no fused
 * multiply-add). Row 0 is the top of the image. The pixel's output goes to
 * out[out_offset + y*W + x]. */
typedef struct lf_view {
    float eye[3];
    float right[3];
    float up[3];
    float forward[3];
    float tan_half_x;
    float tan_half_y;
    uint32_t width;            /* 1 <= W <= 65536 */
    uint32_t height;           /* 1 <= H <= 65536 */
    uint64_t out_offset;       /* in pixels */
} lf_view;

/* Launch shape of the render and backward kernels (chosen by the autotuner).
 * block = tile_w * tile_h threads (at most 256); one thread per ray; each warp
 * covers a warp_w x (32/warp_w) pixel sub-tile. tile_w and tile_h are powers
 * of two. */
typedef struct lf_launch {
    uint32_t tile_w;           /* pixels per CTA tile in x; power of two, multiple of warp_w */
    uint32_t tile_h;           /* pixels per CTA tile in y; power of two, multiple of 32/warp_w */
    uint32_t warp_w;           /* 1, 2, 4, 8, 16 or 32 */
    uint32_t order;            /* 0: tiles in raster order per view; 1: strips of 4 tile rows, column by column */
    uint32_t persistent;       /* 0: one CTA per tile; 1: CTAs pull tiles from a queue */
    uint32_t ctas_per_sm;      /* persistent grid = SMs * ctas_per_sm (0: occupancy) */
} lf_launch;

typedef struct lf_table lf_table;

/* Create a table on the current device.
 * radiance_dev: device array [M'][N][C] in row-major order (origin row i,
 *   direction column j, channel c), M' = M, or floor(M/2) with
 *   LF_TABLE_UPPER_HEMISPHERE; element type per dtype (float, uint16 binary16
 *   bits, uint8 E4M3 bits).
 * row_scales_dev: device array [M'] of FP32 scales; required for F16/E4M3,
 *   ignored (may be NULL) for F32.
 * Without LF_TABLE_BORROW the table and scales are copied (FP16/E4M3 texels
 *   padded to 4 channels) and the caller may free its arrays once the stream
 *   reaches this call. With LF_TABLE_BORROW the caller's arrays are used in
 *   place (F32 with C in {3,4}, or F16/E4M3 with C = 4) and must outlive the
 *   table; the caller may update their contents between renders (table fitting).
 * Also builds the SF point caches of both sets on `stream`.
 * Errors: LF_ERR_INVALID_ARG (null desc/out/radiance, bad sizes, R <= 0 or
 *   non-finite, missing scales, unsupported channel count), LF_ERR_UNSUPPORTED
 *   (k_nearest other than 0, 1, 5 or 9),
 *   LF_ERR_OUT_OF_MEMORY, LF_ERR_CUDA. On error *out is NULL. */
lf_status lf_create_table(const lf_table_desc *desc, const void *radiance_dev,
                          const float *row_scales_dev, void *stream, lf_table **out);

/* Render n_views views (Section 2, image synthesis by sampling L^).
 * views_host: host array of n_views lf_view (read during the call only).
 * out_dev: device FP32 [P][C], P = max(out_offset + W*H) over the views; rays
 *   that miss S get all C channels 0.
 * idx_dev: optional device int32 [P][2K]: the K origin indices then the K
 *   direction indices of each ray, each set in ascending (squared chord
 *   distance, index) order; -1 for a miss. NULL to skip.
 * With k_nearest = 1 (nearest sampling, Section 2 and Fig. 2) each hit maps to
 * its nearest SF point and the pixel takes the single texel L^(i, j).
 * Views must not overlap in the output. n_views <= 65536.
 * Errors: LF_ERR_INVALID_ARG, LF_ERR_CUDA. */
lf_status lf_render(const lf_table *t, const lf_view *views_host, uint32_t n_views,
                    float *out_dev, int32_t *idx_dev, void *stream);

/* lf_render with the image stored as IEEE binary16 (out_dev: device uint16
 * [P][C], each value the FP32 result of lf_render rounded once to nearest
 * even): half the bytes for a caller that reads the image back to the host.
 * Alignment: 8 bytes for C = 4, 2 for C = 3. Errors as lf_render, and
 * LF_ERR_UNSUPPORTED for a table with k_nearest = 9. */
lf_status lf_render_f16(const lf_table *t, const lf_view *views_host, uint32_t n_views,
                        uint16_t *out_dev, int32_t *idx_dev, void *stream);

/* Gradient of the render with respect to the table: for every hit ray and
 * every tap (a, b), grad_table[i_a][j_b][c] += W_ab * grad_out[ray][c]
 * (the adjoint of the linear blend). grad_out_dev: device FP32 [P][C];
 * grad_table_dev: device FP32 [M'][N][C], accumulated (not cleared) with
 * warp-aggregated atomic adds, so the summation order is not fixed.
 * Errors: LF_ERR_INVALID_ARG, LF_ERR_CUDA. */
lf_status lf_render_backward(const lf_table *t, const lf_view *views_host, uint32_t n_views,
                             const float *grad_out_dev, float *grad_table_dev, void *stream);

/* The same gradient from the sample indices a render of the same views wrote
 * (idx_dev: device int32 [P][2K] as lf_render writes them, [P][2] with nearest
 * sampling), instead of a new index step: the hits, the unit hits and the
 * double-float distances of these indices are recomputed, the same distances by
 * the same function as the index step's, so the weights are identical and a
 * fit that keeps its forward indices skips the search in the backward. A miss
 * (index -1) contributes nothing; an index out of range counts as missing and
 * makes the next lf_sync_status report LF_ERR_DEVICE_CHECK.
 * Errors: LF_ERR_INVALID_ARG, LF_ERR_CUDA. */
lf_status lf_render_backward_idx(const lf_table *t, const lf_view *views_host, uint32_t n_views,
                                 const float *grad_out_dev, const int32_t *idx_dev, float *grad_table_dev,
                                 void *stream);

/* Destroy a table (NULL-safe). Synchronises the device before freeing. */
void lf_destroy(lf_table *t);

/* Message of the calling thread's last error ("" if none). */
const char *lf_last_error(void);

/* Launch shape used by lf_render / lf_render_backward on this table.
 * Errors: LF_ERR_INVALID_ARG for an inconsistent shape. */
lf_status lf_set_launch(lf_table *t, const lf_launch *cfg);
lf_status lf_get_launch(const lf_table *t, lf_launch *cfg);

/* Synchronise `stream` and report the table's device status word: LF_OK, or
 * LF_ERR_DEVICE_CHECK if a kernel recorded a failed check since the last
 * call (the word is then cleared). */
lf_status lf_sync_status(lf_table *t, void *stream);

/* Per-row quantisation of an FP32 table for storage (not part of the paper;
 * the storage forms of the precision study). src_dev [M][N][C] FP32;
 * codes_dev [M][N][4] (uint16 binary16 bits or uint8 E4M3 bits; channel 3 is 0
 * when C = 3); scales_dev [M]. scale = amax (F16) or amax/448 (E4M3) over the
 * row's N*C values, 1 if amax = 0; code = RNE(x / scale), E4M3 saturating.
 * Errors: LF_ERR_INVALID_ARG, LF_ERR_CUDA. */
lf_status lf_quantize_table(const float *src_dev, uint32_t M, uint32_t N, uint32_t C,
                            int32_t dtype, void *codes_dev, float *scales_dev, void *stream);

/* Synthetic radiance field (a stand-in for the path-traced light field of
 * Section 2, which needs scenes that are not available):
 *   T(i,j,c) = sum_l col[l][c] * exp(kp[l] (p^o_i . ap[l] - 1))
 *                              * exp(kd[l] (dhat_ij . ad[l] - 1)) + 0.01 u(i,j,c)
 * with dhat_ij the unit ray direction from p^o_i to p^d_j (the ray r_k of
 * Section 2) and u the SplitMix64 uniform of counter (i<<32 | j<<4 | c) in the
 * stream seeded by `noise_seed`. Evaluated in FP64, stored as FP32
 * out_dev [M][N][C]. Host arrays: ap, ad [L][3]; kp, kd [L]; col [L][C]; L <= 64.
 * Errors: LF_ERR_INVALID_ARG, LF_ERR_OUT_OF_MEMORY, LF_ERR_CUDA. */
lf_status lf_fill_lobe_table(uint32_t M, uint32_t N, uint32_t C, uint32_t L,
                             const double *ap, const double *ad, const double *kp,
                             const double *kd, const double *col, uint64_t noise_seed,
                             float *out_dev, void *stream);

/* ---------------------------------------------------------------------------
 * Light-field precompute (Section 2): fill L^(i,j) by tracing every ray
 *   r_k = (O + R p^o_i) + t d_ij,  d_ij = (p^d_j - p^o_i) / |p^d_j - p^o_i|
 * (-p^o_i if the two points coincide) through an analytic scene inside S, with
 * the origin of each of `spp` samples jittered uniformly on the disk of area
 * A_S / M = 4 pi R^2 / M tangent to S at O + R p^o_i; the texel is the mean of
 * the samples. The scene is an emission-absorption volume of Gaussian blobs
 * (a stand-in for the paper's path-traced CT data, which is not available):
 *   density  sigma(x) = sum_b kappa_b exp(-|x - mu_b|^2 / (2 s_b^2)),
 *   emission q(x)     = sum_b kappa_b exp(...) emit_b        (per unit length),
 * integrated from the origin (t = 0) to the far intersection of the line with
 * S by the midpoint rule with `steps` steps of constant sigma and q:
 *   L += T (1 - exp(-sigma dt)) / sigma * q,   T *= exp(-sigma dt),
 * plus T times the background bg0 + bg1 (1 + d_z) / 2 of the ray's direction.
 * Channel 3 (channels = 4) holds the mean opacity 1 - T.
 * Jitter of sample s of texel (i, j): u1, u2 = the top 24 bits of
 * SplitMix64(seed, 2 ((i N + j) spp + s)) and of the next counter, times 2^-24;
 * offset = (2R / sqrt(M)) sqrt(u1) (cos(2 pi u2) e_phi + sin(2 pi u2) e_theta)
 * with e_phi = (-p_y, p_x, 0) / rho, e_theta = (p_x p_z, p_y p_z, -rho^2) / rho,
 * rho = sqrt(p_x^2 + p_y^2). SplitMix64(seed, c): z = seed + (c + 1) *
 * 0x9e3779b97f4a7c15, then the published SplitMix64 finaliser.
 * ------------------------------------------------------------------------- */
typedef struct {
    float center[3];     /* mu_b */
    float width;         /* s_b > 0 */
    float density;       /* kappa_b >= 0, per unit length */
    float emit[3];       /* emitted colour per unit density (RGB) */
} lf_blob;               /* 32 bytes */

#define LF_PRECOMPUTE_MAX_BLOBS 16u

typedef struct {
    double radius;             /* R > 0 */
    double center[3];          /* O */
    uint32_t n_origins;        /* M, 1 .. 2^24 */
    uint32_t n_directions;     /* N, 1 .. 2^24 */
    uint32_t channels;         /* 3 (RGB) or 4 (RGB + opacity) */
    uint32_t rows;             /* origin rows filled, 1 .. M: rows [0, rows), e.g. M/2 for an
                                  upper-hemisphere table (z_i > 0 exactly for i < M/2) */
    uint32_t spp;              /* jittered samples per texel, 1 .. 1024 */
    uint32_t steps;            /* midpoint steps per sample, 1 .. 4096 */
    uint32_t jitter;           /* 1: jitter the origins; 0: every sample starts at O + R p^o_i */
    uint32_t n_blobs;          /* 0 .. LF_PRECOMPUTE_MAX_BLOBS */
    uint64_t seed;             /* generator seed of the jitter */
    float bg0[3], bg1[3];      /* background */
} lf_precompute_desc;          /* 96 bytes */

/* Fill out_dev [rows][N][channels] FP32 (device, caller-owned, row-major,
 * j fastest) with the precomputed light field of the scene `blobs_host`
 * (n_blobs host structs, read during the call). FP32 arithmetic; the library
 * allocates and frees a (M + N) x 32-byte point scratch in stream order.
 * Errors: LF_ERR_INVALID_ARG (NULL, ranges, non-finite or non-positive sizes),
 * LF_ERR_OUT_OF_MEMORY, LF_ERR_CUDA. Asynchronous on `stream`. */
lf_status lf_precompute_table(const lf_precompute_desc *desc, const lf_blob *blobs_host,
                              float *out_dev, void *stream);

/* Direct render of the same volume: the ground truth that a light-field render
 * of the precomputed table approximates (the paper compares its renders with
 * path-traced images of the scene, Section 3). For every pixel of the views the
 * camera ray and its front hit h_o on S are the FP32 steps of lf_render; the
 * ray is then integrated as above from h_o along its direction to the far
 * intersection with S (that length computed in FP64), one sample, no jitter.
 * out_dev [pixels][channels] FP32 (device, caller-owned; RGB, plus opacity
 * 1 - T for channels = 4), written at each view's out_offset; misses store 0.
 * Reads radius, center, channels, steps, n_blobs and the background of
 * `desc`; n_origins, n_directions, rows, spp, jitter and seed are ignored.
 * out_dev must be 16-byte aligned for 4 channels, 4-byte for 3. One kernel
 * launch per view; allocates nothing. Errors: LF_ERR_INVALID_ARG (NULL,
 * ranges, non-finite values, views as for lf_render), LF_ERR_CUDA.
 * Asynchronous on `stream`. */
lf_status lf_render_volume(const lf_precompute_desc *desc, const lf_blob *blobs_host,
                           const lf_view *views_host, uint32_t n_views, float *out_dev, void *stream);

/* ---------------------------------------------------------------------------
 * Learned post-filter of a light-field image (Section 2, post-processing: a
 * network removes the interpolation artifacts of the rendered image). Only the
 * image-to-image filter is provided, not the paper's adversarial training: for
 * each view, three 3x3 convolution layers (4 -> 16 -> 16 -> 3 channels, ReLU
 * after the first two, zero padding of 1 before each, cross-correlation as in
 * the common deep-learning frameworks) on the features (R, G, B, hit), where
 * hit = 1 if the pixel's ray meets the sphere (radius, center) by the FP32 test
 * of lf_render, else 0; the result is added to the input RGB of hit pixels,
 * other pixels are set to 0, and channel 3 (channels = 4) is copied.
 * Arithmetic: the layers run on the tensor cores with FP16 operands (the input
 * colour clamped to +-65504, the hidden activations and the weights each
 * rounded once to FP16) and FP32 accumulation; the residual adds the FP32
 * input colour.
 * weights_host: LF_POST_WEIGHTS FP32 values (host, read during the call; they
 * travel in the kernel's parameters as FP16), in this order and each in
 * [out][in][row][column] layout: W1 [16][4][3][3], b1 [16], W2 [16][16][3][3],
 * b2 [16], W3 [3][16][3][3], b3 [3]. in_dev / out_dev: [pixels][channels] FP32
 * (device; views laid out as for lf_render, channels 3 or 4; 4-byte aligned);
 * out_dev must not overlap in_dev. One launch per 32 views; allocates nothing.
 * Errors: LF_ERR_INVALID_ARG (NULL, channels, radius, non-finite weights,
 * views as for lf_render, overlapping buffers), LF_ERR_CUDA. Asynchronous on
 * `stream`.
 * ------------------------------------------------------------------------- */
#define LF_POST_WEIGHTS 3347u
lf_status lf_post_filter(double radius, const double center[3], uint32_t channels, const float *weights_host,
                         const lf_view *views_host, uint32_t n_views, const float *in_dev, float *out_dev,
                         void *stream);

/* Largest M + N that lf_render_noalloc accepts, and the number of rays of one
 * launch (one call's views, in chunks of 64) whose nearest-neighbour order the
 * render kernel leaves to the exact pass it queues them for: past this many the
 * exact pass renders every ray of that launch (the same image, more slowly). */
#define LF_NOALLOC_MAX_POINTS 278528u
#define LF_NOALLOC_MAX_DEFERRED 16384u

/* Render without allocating any device memory. The paper has no counterpart:
 * this exists for callers that cannot call cudaMalloc -- a process whose
 * device memory is already fully reserved by another runtime's pool (an
 * allocation would fail), or a frame-paced loop that must not call
 * cudaMalloc/cudaFree because they synchronise the device and take unbounded
 * time. Instead of a table object, the call takes the table description and
 * the caller's device arrays directly (radiance [M][N][C] FP32 with C in
 * {3,4}, or FP16/E4M3 codes [M][N][4] with row_scales_dev [M]; views, out_dev
 * and idx_dev as for lf_render; launch may be NULL for the default shape). It
 * writes the same image and indices as lf_create_table + lf_render.
 * The SF point caches, the status/queue words and the queue of rays left to
 * the exact pass live in one fixed device array inside the library (32 B per
 * point for up to LF_NOALLOC_MAX_POINTS points plus 8 B per queued ray for up
 * to LF_NOALLOC_MAX_DEFERRED rays, about 8.6 MiB), which every GPU that loads
 * the library keeps until the process exits. Each call rebuilds that content
 * on `stream` and leaves the last call's contents behind; calls that overlap
 * on the GPU (other streams or threads) race on it. Every call looks up the
 * array's device address (cudaGetSymbolAddress, with the caller's device
 * current; it allocates nothing, and the address is valid only for the
 * context that looked it up); the first call on a device may load the
 * library's device code, so make it before any stream capture.
 * Allocates nothing: no cudaMalloc, cudaFree or allocating library routine.
 * Device-side checks (an index out of range) are recorded in the array's
 * status word; lf_noalloc_sync_status reads them.
 * Errors: LF_ERR_INVALID_ARG (including M + N > LF_NOALLOC_MAX_POINTS, with a
 * message saying so), LF_ERR_UNSUPPORTED, LF_ERR_CUDA. */
lf_status lf_render_noalloc(const lf_table_desc *desc, const void *radiance_dev,
                            const float *row_scales_dev, const lf_view *views_host,
                            uint32_t n_views, const lf_launch *launch, float *out_dev,
                            int32_t *idx_dev, void *stream);

/* Synchronise `stream` and report the status word of lf_render_noalloc's
 * device array on the current device, as lf_sync_status does for a table:
 * LF_OK, or LF_ERR_DEVICE_CHECK if a kernel of the last lf_render_noalloc call
 * on this device recorded a failed check (the word is then cleared; every
 * lf_render_noalloc call clears it when it starts). Allocates nothing; no
 * counterpart in the paper. Errors: LF_ERR_CUDA, LF_ERR_DEVICE_CHECK. */
lf_status lf_noalloc_sync_status(void *stream);

/* Number of SMs of the current device (0 without one) and the library
 * version string. */
int lf_device_sm_count(void);
const char *lf_version(void);

/* sizeof of the ABI structures as compiled into the library, for bindings to
 * check their layouts: which = 0 lf_table_desc, 1 lf_view, 2 lf_launch, 3 lf_precompute_desc, 4 lf_blob;
 * 0 for any other value. */
size_t lf_struct_size(int which);

#ifdef __cplusplus
}
#endif

#endif /* LUMIPATH_H */
