// lf_internal.h -- structures shared by the host side of the C ABI and the
// kernels of the light-field sampling library.
#pragma once

#include <stdint.h>

#include "lumipath.h"

namespace lfk {

// Bits of a table's device status word (read back by lf_sync_status).
constexpr uint32_t kStatusIndex = 1u;        // a search returned an index out of range (recorded, replaced by 0)
constexpr uint32_t kStatusIdxInput = 2u;     // given indices disagree with the ray (backward from indices)
constexpr uint32_t kStatusDebugPoint = 4u;   // debug build: a point index about to be read is out of range
constexpr uint32_t kStatusDebugTexel = 8u;   // debug build: a texel index about to be read is out of range
constexpr uint32_t kStatusDebugGrad = 16u;   // debug build: a gradient index about to be written is out of range

// Debug builds (-DLF_DEBUG_CHECKS), in place of a sanitizer: every index the
// kernels are about to dereference is checked against its bound; a failure
// sets a status bit and the access goes to index 0 instead (recorded, never a
// trap or a fault). Release builds: the index as it is (in range by construction).
#ifdef LF_DEBUG_CHECKS
#define LF_DINDEX(idx, bound, status, bit) \
    (((uint64_t)(idx) < (uint64_t)(bound)) ? (idx) : (atomicOr((status), (bit)), decltype(+(idx))(0)))
#else
#define LF_DINDEX(idx, bound, status, bit) (idx)
#endif

// Storage forms the kernels read (texel type x channel count).
enum TexelKind { kF32C4 = 0, kF32C3 = 1, kF16C4 = 2, kE4M3C4 = 3 };

// A view as the kernels read it (kernel-parameter space).
struct ViewK {
    float eye[3], right[3], up[3], fwd[3];
    float tan_x, tan_y;
    uint32_t width, height;
    uint64_t out_offset;
    uint32_t tiles_x, tiles_y;
    // Conservative miss test: e - O, |e - O|^2 - R^2, |e - O|^2, 2/W, 2/H
    // (host FP64, rounded), and whether the eye is clearly outside S.
    float f0[3], c0, ff0, inv2w, inv2h;
    uint32_t outside;
};

// Sphere S: FP32 centre and radius for the ray/sphere step, the centre as a
// hi/lo float pair and in FP64 for the unit hit vectors.
struct SphereK {
    float o32[3];
    float r32;
    float o_hi[3], o_lo[3];
    double o64[3];
    float ir_h, ir_l;        // 1/R as a hi/lo pair
    float r2_h, r2_l;        // R^2 as a hi/lo pair
    float inv_r2;            // 1/R^2
    uint32_t centred;        // O == (0, 0, 0)
};

// One SF point set: p_i as hi/lo float4 pairs (w unused), n, n as float and
// the reciprocal kernel radius 1/sqrt(4*pi/n).
struct PointSetK {
    const float4 *hi;
    const float4 *lo;
    uint32_t n;
    float nf;
    float inv_sigma;
};

// Argument checks and view set-up shared by the entry points (lf_abi.cu): a
// failed check sets the calling thread's lf_last_error() message.
lf_status check_desc(const lf_table_desc *d);
lf_status check_launch(const lf_launch *c);
lf_status check_views(const lf_view *views, uint32_t n);
ViewK camera_of(const lf_view &w);                  // the camera only (no tiling, no miss constants)
ViewK view_params(const lf_view &w, const lf_launch &L, double R, const double O[3]);

}  // namespace lfk

struct lf_table {
    lf_table_desc desc;
    int device;
    int texel_kind;                  // lfk::TexelKind
    uint32_t C;                      // logical channels (3 or 4)
    uint32_t rows;                   // origin rows stored (M, or M/2 for the upper hemisphere)
    const void *texels;              // [M][N][Cs]
    const float *scales;             // [M] or NULL (F32)
    void *owned_texels;              // non-NULL if the library owns the copy
    float *owned_scales;
    float4 *points;                  // [2M + 2N]: origins hi, lo, then directions hi, lo
    uint32_t *scratch;               // device words and the queue of deferred rays (layout: lf_kernels.h)
    lfk::SphereK sphere;
    lfk::PointSetK po, pd;
    lf_launch launch;
    int sm_count;
};
