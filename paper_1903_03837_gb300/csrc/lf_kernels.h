// lf_kernels.h -- kernel parameter blocks and launchers (host <-> device).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lf_internal.h"

namespace lfk {

constexpr int kSmallViews = 2;     // one view or a stereo pair per launch
constexpr int kLargeViews = 64;    // batches are split into launches of <= 64 views
constexpr int kMaxBlock = 256;     // threads per CTA (tile_w * tile_h)
constexpr uint32_t kStripTiles = 4;

// Device words of a table or of a no-allocation render: [0] status, [1] tile
// queue, [2] finished render CTAs, [3] finished fixup CTAs, bytes 16..23 the
// count of queued rays; the queued rays follow at byte kWordsBytes.
constexpr uint32_t kWordsBytes = 256;
constexpr uint32_t kDeferCap = 1u << 18;         // queued rays a table holds per launch
constexpr unsigned kFixupCtas = 304, kFixupThreads = 256;   // the fixup grid when the occupancy query fails
constexpr uint32_t kFixupWarps = kFixupThreads / 32;

struct RenderParamsBase {
    SphereK sphere;
    PointSetK po, pd;
    const void *texels;            // [M][N][Cs]
    const float *scales;           // [M] (F16 / E4M3)
    uint32_t N;                    // texels per origin row
    uint32_t C;                    // output / gradient channels (3 or 4)
    float *out;                    // forward: [P][C] FP32, or binary16 when out_f16
    uint32_t out_f16;              // 1: the image is stored as binary16 (round to nearest even)
    int32_t *idx;                  // forward: [P][2K] or NULL
    const int32_t *idx_in;         // backward: the forward's [P][2K] indices, or NULL (search again)
    const float *grad_out;         // backward: [P][C]
    float *grad;                   // backward: [M][N][C]
    uint32_t *status, *queue, *done;
    // Rays whose fast-path order was not certain: the render kernel queues
    // them here and the fixup kernel that follows it on the stream renders
    // them (more than defer_cap in one launch: the fixup renders every ray).
    unsigned long long *defer_count;   // rays queued in this launch (reset by the fixup kernel)
    uint32_t *defer_done;              // fixup CTAs finished
    unsigned long long *defer_items;   // [defer_cap]: view << 32 | y << 16 | x
    uint32_t defer_cap;
    uint64_t total_pixels;             // pixels of all views of the launch
    uint32_t n_views, total_tiles;
    uint32_t tile_w, tile_h, warp_w, order, persistent;
    uint32_t tw_log, th_log, ww_log;   // log2 of tile_w, tile_h, warp_w
    uint32_t rows_stored;              // origin rows present (upper hemisphere), 0: all
    uint32_t rows_valid;               // rows of the table (M or rows_stored)
    uint32_t nearest_only;             // 1: nearest sampling (K = 1), else 5 or 9 neighbours
    uint32_t nine;                     // 1: 9 neighbours per hit (81 taps)
};

template <int MAXV>
struct RenderParams : RenderParamsBase {
    uint32_t tile_prefix[MAXV + 1];
    ViewK views[MAXV];
};

cudaError_t launch_render_small(int kind, bool bwd, const RenderParams<kSmallViews> &p, unsigned grid,
                                unsigned block, cudaStream_t st);
cudaError_t launch_render_large(int kind, bool bwd, const RenderParams<kLargeViews> &p, unsigned grid,
                                unsigned block, cudaStream_t st);
int render_occupancy(int kind, bool bwd, bool large, bool nine, unsigned block);

// lf_table.cu
cudaError_t launch_build_points(uint32_t n, float4 *hi, float4 *lo, cudaStream_t st);
cudaError_t launch_pad_codes(const void *src, uint32_t M, uint32_t N, int bytes, void *dst, cudaStream_t st);
cudaError_t launch_quantize(const float *src, uint32_t M, uint32_t N, uint32_t C, int dtype, void *codes,
                            float *scales, cudaStream_t st);

constexpr int kMaxLobes = 64;
struct LobeParams {
    uint32_t L, C;
    uint64_t seed;
    double ap[kMaxLobes][3], ad[kMaxLobes][3], kp[kMaxLobes], kd[kMaxLobes], col[kMaxLobes][4];
};
cudaError_t launch_fill_lobe(const LobeParams &P, const float4 *po_hi, const float4 *po_lo,
                             const float4 *pd_hi, const float4 *pd_lo, uint32_t M, uint32_t N,
                             float *out, cudaStream_t st);

// SplitMix64 (Steele, Lea, Flood 2014): output number ctr+1 of the stream
// seeded with `seed` (the counter-based generator of the synthetic inputs).
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t ctr)
{
    uint64_t z = seed + (ctr + 1ull) * 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// lf_precompute.cu: the light-field precompute of Section 2 (volume scene).
constexpr int kMaxBlobs = 16;
struct PrecomputeParams {
    const float4 *po_hi, *po_lo, *pd_hi, *pd_lo;   // SF points (hi + lo parts)
    float *out;                                     // [rows][N][C]
    float Ox, Oy, Oz, R;                            // sphere S
    float disk_r;                                   // 2R / sqrt(M): disk of area 4 pi R^2 / M
    uint32_t N, C, rows, spp, steps, jitter, nb;
    uint64_t seed;
    float bg0[3], bg1[3];
    float4 blob_pos[kMaxBlobs];    // centre xyz, log2(kappa_b) (-inf for kappa_b = 0)
    float4 blob_col[kMaxBlobs];    // emit rgb, a_b = sqrt(log2(e) / 2) / s_b
};
cudaError_t launch_precompute(const PrecomputeParams &p, cudaStream_t st);
// Direct render of the precompute's volume along the pixel rays of one view
// (out at the view's out_offset; p.out, p.C and the volume fields are used;
// R is the radius in FP64 for the far end of each ray).
cudaError_t launch_volume_direct(const PrecomputeParams &p, const ViewK &v, const SphereK &S, double R,
                                 cudaStream_t st);

// lf_post.cu: the learned post-filter of the light-field image. Weights in
// framework (OIHW) order, FP32: W1 [16][4][3][3], b1 [16], W2 [16][16][3][3],
// b2 [16], W3 [3][16][3][3], b3 [3]; launch_post_filter lays them out as the
// FP16 B operands of the kernel's MMAs, which travel in its parameter block.
constexpr int kPostHidden = 16;
constexpr int kPostW1 = 0;
constexpr int kPostB1 = kPostW1 + kPostHidden * 4 * 9;
constexpr int kPostW2 = kPostB1 + kPostHidden;
constexpr int kPostB2 = kPostW2 + kPostHidden * kPostHidden * 9;
constexpr int kPostW3 = kPostB2 + kPostHidden;
constexpr int kPostB3 = kPostW3 + 3 * kPostHidden * 9;
constexpr int kPostWeights = kPostB3 + 3;
constexpr int kPostMaxViews = 32;       // views per launch
struct PostParams {
    SphereK sphere;                     // the hit mask of each pixel's ray
    const float *in;                    // [P][C] light-field image
    float *out;                         // [P][C] filtered image (must not overlap `in`)
    uint32_t C;                         // 3 or 4 (channel 3 is copied)
    uint32_t n_views;
    ViewK views[kPostMaxViews];         // cameras
    float w[kPostWeights];
};
// Splits the views (at most kPostMaxViews) into strips and chunks and launches the filter.
cudaError_t launch_post_filter(const PostParams &p, cudaStream_t st);

// Fills the conservative-miss constants of a view for sphere (R, O) (lf_abi.cu).
void fill_view_miss_consts(ViewK &k, double R, const double O[3]);

// Host-side constants of sphere S (lf_abi.cu): FP32 radius and centre for the
// ray/sphere step, the centre as a hi/lo float pair and in FP64, and for the
// unit-hit step 1/R and R^2 as hi/lo float pairs, 1/R^2 and whether O is the
// origin.
void fill_sphere_consts(SphereK &S, double R, const double O[3]);

// Sets the calling thread's lf_last_error() message (lf_abi.cu).
void set_last_error(const char *msg);

}  // namespace lfk
