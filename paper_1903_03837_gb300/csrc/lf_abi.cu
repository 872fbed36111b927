// lf_abi.cu -- host side of the C ABI declared in include/lumipath.h:
// argument validation, table ownership, the view/tile bookkeeping of each
// launch and the thread-local error message. No arithmetic of the sampling
// path runs here; every step of it is a kernel.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "lf_kernels.h"
#include "lumipath.h"

namespace {

thread_local std::string g_err;

lf_status fail(lf_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

// An NVTX range around one entry point (for nsys/ncu timelines; a no-op when
// no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

// Vector loads, stores and atomics need their natural alignment; a misaligned
// caller pointer is an argument error, never a device fault.
bool misaligned(const void *p, uintptr_t a) { return p && ((uintptr_t)p & (a - 1)); }

lf_status cuda_fail(cudaError_t e, const char *what)
{
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(LF_ERR_OUT_OF_MEMORY, "%s: %s", what, cudaGetErrorString(e));
    }
    return fail(LF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool finite3(const float *v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }
bool finite3(const double *v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

lf_launch default_launch()
{
    lf_launch l;
    l.tile_w = 16;
    l.tile_h = 16;
    l.warp_w = 8;
    l.order = 0;
    l.persistent = 0;
    l.ctas_per_sm = 0;
    return l;
}

// Volume fields of a precompute description (radius, centre, channels,
// steps, blobs, background) checked and turned into kernel parameters; the
// SF-set fields are left to the caller.
lf_status volume_params(const lf_precompute_desc *d, const lf_blob *blobs, float *out_dev,
                        lfk::PrecomputeParams &P)
{
    if (!(d->radius > 0.0) || !std::isfinite(d->radius) || !std::isfinite(d->center[0]) ||
        !std::isfinite(d->center[1]) || !std::isfinite(d->center[2]))
        return fail(LF_ERR_INVALID_ARG, "R must be positive and finite, O finite");
    if (d->channels != 3 && d->channels != 4) return fail(LF_ERR_INVALID_ARG, "channels must be 3 or 4");
    if (d->steps == 0 || d->steps > 4096) return fail(LF_ERR_INVALID_ARG, "steps must be in [1, 4096]");
    if (d->n_blobs > LF_PRECOMPUTE_MAX_BLOBS)
        return fail(LF_ERR_INVALID_ARG, "at most %u blobs", LF_PRECOMPUTE_MAX_BLOBS);
    if (d->n_blobs && !blobs) return fail(LF_ERR_INVALID_ARG, "blobs is NULL");
    if (misaligned(out_dev, d->channels == 4 ? 16 : 4))
        return fail(LF_ERR_INVALID_ARG, "out must be %u-byte aligned for %u channels",
                    d->channels == 4 ? 16u : 4u, d->channels);
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(d->bg0[k]) || !std::isfinite(d->bg1[k]))
            return fail(LF_ERR_INVALID_ARG, "non-finite background");
    memset(&P, 0, sizeof P);
    for (uint32_t b = 0; b < d->n_blobs; ++b) {
        const lf_blob &B = blobs[b];
        bool ok = B.width > 0.0f && std::isfinite(B.width) && B.density >= 0.0f && std::isfinite(B.density);
        for (int k = 0; k < 3; ++k) ok = ok && std::isfinite(B.center[k]) && std::isfinite(B.emit[k]);
        if (!ok) return fail(LF_ERR_INVALID_ARG, "blob %u: non-finite value, width <= 0 or density < 0", b);
        // density kappa exp(-r^2 / (2 s^2)) = exp2(log2(kappa) - (a r)^2), a^2 = log2(e) / (2 s^2)
        const double a = std::sqrt(1.4426950408889634 / 2.0) / (double)B.width;
        P.blob_pos[b] = make_float4(B.center[0], B.center[1], B.center[2],
                                    B.density > 0.0f ? (float)std::log2((double)B.density) : -INFINITY);
        P.blob_col[b] = make_float4(B.emit[0], B.emit[1], B.emit[2], (float)a);
    }
    P.out = out_dev;
    P.Ox = (float)d->center[0];
    P.Oy = (float)d->center[1];
    P.Oz = (float)d->center[2];
    P.R = (float)d->radius;
    P.C = d->channels;
    P.steps = d->steps;
    P.nb = d->n_blobs;
    for (int k = 0; k < 3; ++k) {
        P.bg0[k] = d->bg0[k];
        P.bg1[k] = d->bg1[k];
    }
    return LF_OK;
}


}  // namespace

namespace lfk {

lf_status check_launch(const lf_launch *c)
{
    if (!c) return fail(LF_ERR_INVALID_ARG, "launch config is NULL");
    uint32_t ww = c->warp_w;
    if (!(ww == 1 || ww == 2 || ww == 4 || ww == 8 || ww == 16 || ww == 32))
        return fail(LF_ERR_INVALID_ARG, "warp_w must be 1, 2, 4, 8, 16 or 32 (got %u)", ww);
    uint32_t wh = 32 / ww;
    if (c->tile_w == 0 || c->tile_h == 0 || (c->tile_w & (c->tile_w - 1)) || (c->tile_h & (c->tile_h - 1)))
        return fail(LF_ERR_INVALID_ARG, "tile %ux%u: both sides must be powers of two", c->tile_w, c->tile_h);
    if (c->tile_w % ww || c->tile_h % wh)
        return fail(LF_ERR_INVALID_ARG, "tile %ux%u is not a whole number of %ux%u warp tiles",
                    c->tile_w, c->tile_h, ww, wh);
    if (c->tile_w * c->tile_h > (uint32_t)kMaxBlock)
        return fail(LF_ERR_INVALID_ARG, "tile %ux%u exceeds %d threads", c->tile_w, c->tile_h, kMaxBlock);
    if (c->order > 1 || c->persistent > 1)
        return fail(LF_ERR_INVALID_ARG, "order must be 0/1 and persistent 0/1");
    if (c->ctas_per_sm > 64) return fail(LF_ERR_INVALID_ARG, "ctas_per_sm > 64");
    return LF_OK;
}

lf_status check_views(const lf_view *views, uint32_t n)
{
    if (!views) return fail(LF_ERR_INVALID_ARG, "views is NULL");
    if (n == 0 || n > 65536) return fail(LF_ERR_INVALID_ARG, "n_views must be in [1, 65536] (got %u)", n);
    for (uint32_t v = 0; v < n; ++v) {
        const lf_view &w = views[v];
        if (w.width == 0 || w.height == 0 || w.width > 65536 || w.height > 65536)
            return fail(LF_ERR_INVALID_ARG, "view %u: size %ux%u out of range", v, w.width, w.height);
        if (!finite3(w.eye) || !finite3(w.right) || !finite3(w.up) || !finite3(w.forward) ||
            !std::isfinite(w.tan_half_x) || !std::isfinite(w.tan_half_y))
            return fail(LF_ERR_INVALID_ARG, "view %u: non-finite camera", v);
        uint64_t end = w.out_offset + (uint64_t)w.width * w.height;
        if (end < w.out_offset || end > (1ull << 40))
            return fail(LF_ERR_INVALID_ARG, "view %u: output range overflows", v);
    }
    return LF_OK;
}

// The camera of a view (no tiling, no miss constants).
ViewK camera_of(const lf_view &w)
{
    ViewK k;
    memset(&k, 0, sizeof k);
    for (int i = 0; i < 3; ++i) {
        k.eye[i] = w.eye[i];
        k.right[i] = w.right[i];
        k.up[i] = w.up[i];
        k.fwd[i] = w.forward[i];
    }
    k.tan_x = w.tan_half_x;
    k.tan_y = w.tan_half_y;
    k.width = w.width;
    k.height = w.height;
    k.out_offset = w.out_offset;
    k.inv2w = (float)(2.0 / w.width);        // the camera ray's pixel scale, and the miss test's
    k.inv2h = (float)(2.0 / w.height);
    return k;
}

ViewK view_params(const lf_view &w, const lf_launch &L, double R, const double O[3])
{
    ViewK k = camera_of(w);
    k.tiles_x = (w.width + L.tile_w - 1) / L.tile_w;
    k.tiles_y = (w.height + L.tile_h - 1) / L.tile_h;
    fill_view_miss_consts(k, R, O);
    return k;
}

// Checks of a table description shared by lf_create_table and
// lf_render_noalloc: radius and centre, point counts, channels, storage type,
// neighbour count and flags.
lf_status check_desc(const lf_table_desc *d)
{
    if (!d) return fail(LF_ERR_INVALID_ARG, "desc is NULL");
    if (!(std::isfinite(d->radius) && d->radius > 0.0))
        return fail(LF_ERR_INVALID_ARG, "radius must be finite and > 0");
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(d->center[k])) return fail(LF_ERR_INVALID_ARG, "center must be finite");
    const uint32_t M = d->n_origins, N = d->n_directions, C = d->channels;
    if (M == 0 || N == 0 || M > (1u << 24) || N > (1u << 24))
        return fail(LF_ERR_INVALID_ARG, "point counts must be in [1, 2^24] (M=%u, N=%u)", M, N);
    if (C != 3 && C != 4) return fail(LF_ERR_INVALID_ARG, "channels must be 3 or 4 (got %u)", C);
    if (d->dtype != LF_DTYPE_F32 && d->dtype != LF_DTYPE_F16 && d->dtype != LF_DTYPE_E4M3)
        return fail(LF_ERR_INVALID_ARG, "unknown dtype %d", d->dtype);
    if (d->k_nearest != 0 && d->k_nearest != 1 && d->k_nearest != 5 && d->k_nearest != 9)
        return fail(LF_ERR_UNSUPPORTED, "k_nearest=%u: 1, 5 or 9 neighbours per hit are built", d->k_nearest);
    if (d->flags & ~(LF_TABLE_BORROW | LF_TABLE_UPPER_HEMISPHERE))
        return fail(LF_ERR_INVALID_ARG, "unknown flags 0x%x", d->flags);
    if ((d->flags & LF_TABLE_UPPER_HEMISPHERE) && M < 2)
        return fail(LF_ERR_INVALID_ARG, "an upper-hemisphere table needs M >= 2");
    return LF_OK;
}

}  // namespace lfk

namespace {

template <int MAXV>
lf_status run_chunk(const lf_table *t, const lfk::RenderParamsBase &base, const lf_view *views,
                    uint32_t nv, bool bwd, cudaStream_t st)
{
    // RenderParams<64> is a few KB: keep it off the stack of deep callers.
    static thread_local lfk::RenderParams<MAXV> p;
    static_cast<lfk::RenderParamsBase &>(p) = base;
    const lf_launch &L = t->launch;
    uint64_t tiles = 0;
    for (uint32_t v = 0; v < nv; ++v) {
        p.views[v] = lfk::view_params(views[v], L, t->desc.radius, t->desc.center);
        p.tile_prefix[v] = (uint32_t)tiles;
        tiles += (uint64_t)p.views[v].tiles_x * p.views[v].tiles_y;
    }
    if (tiles >= (1ull << 31)) return fail(LF_ERR_INVALID_ARG, "too many tiles in one launch");
    p.tile_prefix[nv] = (uint32_t)tiles;
    p.n_views = nv;
    p.total_tiles = (uint32_t)tiles;
    p.total_pixels = 0;
    for (uint32_t v = 0; v < nv; ++v) p.total_pixels += (uint64_t)views[v].width * views[v].height;
    unsigned block = L.tile_w * L.tile_h;
    unsigned grid = (unsigned)tiles;
    if (L.persistent) {
        int per_sm = L.ctas_per_sm ? (int)L.ctas_per_sm
                                   : lfk::render_occupancy(t->texel_kind, bwd, MAXV != lfk::kSmallViews,
                                                           p.nine != 0, block);
        uint64_t g = (uint64_t)t->sm_count * (uint64_t)per_sm;
        grid = (unsigned)(g < tiles ? g : tiles);
    }
    if (grid == 0) return LF_OK;
    cudaError_t e;
    if constexpr (MAXV == lfk::kSmallViews)
        e = lfk::launch_render_small(t->texel_kind, bwd, p, grid, block, st);
    else
        e = lfk::launch_render_large(t->texel_kind, bwd, p, grid, block, st);
    if (e != cudaSuccess) return cuda_fail(e, bwd ? "backward launch" : "render launch");
    return LF_OK;
}

lf_status run(const lf_table *t, const lf_view *views, uint32_t n_views, float *out, int32_t *idx,
              const float *grad_out, float *grad, void *stream, const int32_t *idx_in = nullptr,
              bool out_f16 = false)
{
    lf_status s = lfk::check_views(views, n_views);
    if (s != LF_OK) return s;
    const uintptr_t va = t->C == 4 ? 16 : 4;      // float4 image / gradient accesses for 4 channels
    const uintptr_t oa = out_f16 ? (t->C == 4 ? 8 : 2) : va;
    if (misaligned(out, oa) || misaligned(grad_out, va) || misaligned(grad, va))
        return fail(LF_ERR_INVALID_ARG, "image and gradient buffers must be %u-byte aligned", (unsigned)va);
    if (misaligned(idx, 8)) return fail(LF_ERR_INVALID_ARG, "idx must be 8-byte aligned");
    if (misaligned(idx_in, 4)) return fail(LF_ERR_INVALID_ARG, "idx must be 4-byte aligned");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != t->device) return fail(LF_ERR_INVALID_ARG, "table lives on device %d, current is %d", t->device, dev);
    lfk::RenderParamsBase b;
    memset(&b, 0, sizeof b);
    b.sphere = t->sphere;
    b.po = t->po;
    b.pd = t->pd;
    b.texels = t->texels;
    b.scales = t->scales;
    b.N = t->desc.n_directions;
    b.C = t->C;
    b.out = out;
    b.idx = idx;
    b.idx_in = idx_in;
    b.out_f16 = out_f16 ? 1u : 0u;
    b.grad_out = grad_out;
    b.grad = grad;
    b.status = t->scratch;
    b.queue = t->scratch + 1;
    b.done = t->scratch + 2;
    b.defer_done = t->scratch + 3;
    b.defer_count = reinterpret_cast<unsigned long long *>(t->scratch + 4);
    b.defer_items = reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(t->scratch) + lfk::kWordsBytes);
    b.defer_cap = lfk::kDeferCap;
    b.tile_w = t->launch.tile_w;
    b.tile_h = t->launch.tile_h;
    b.warp_w = t->launch.warp_w;
    b.order = t->launch.order;
    b.persistent = t->launch.persistent;
    b.tw_log = (uint32_t)__builtin_ctz(t->launch.tile_w);
    b.th_log = (uint32_t)__builtin_ctz(t->launch.tile_h);
    b.ww_log = (uint32_t)__builtin_ctz(t->launch.warp_w);
    b.rows_valid = t->rows;
    b.nearest_only = t->desc.k_nearest == 1 ? 1u : 0u;
    b.nine = t->desc.k_nearest == 9 ? 1u : 0u;
    b.rows_stored = (t->desc.flags & LF_TABLE_UPPER_HEMISPHERE) ? t->rows : 0u;
    const bool bwd = grad != nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    if (n_views <= (uint32_t)lfk::kSmallViews) return run_chunk<lfk::kSmallViews>(t, b, views, n_views, bwd, st);
    for (uint32_t v0 = 0; v0 < n_views; v0 += lfk::kLargeViews) {
        uint32_t nv = n_views - v0 < (uint32_t)lfk::kLargeViews ? n_views - v0 : (uint32_t)lfk::kLargeViews;
        s = run_chunk<lfk::kLargeViews>(t, b, views + v0, nv, bwd, st);
        if (s != LF_OK) return s;
    }
    return LF_OK;
}

size_t code_bytes(int dtype) { return dtype == LF_DTYPE_F32 ? 4 : (dtype == LF_DTYPE_F16 ? 2 : 1); }

}  // namespace

namespace lfk {
void set_last_error(const char *msg) { g_err = msg ? msg : ""; }

void fill_view_miss_consts(ViewK &k, double R, const double O[3])
{
    double f[3] = {(double)k.eye[0] - O[0], (double)k.eye[1] - O[1], (double)k.eye[2] - O[2]};
    double ff = f[0] * f[0] + f[1] * f[1] + f[2] * f[2];
    for (int i = 0; i < 3; ++i) k.f0[i] = (float)f[i];
    k.ff0 = (float)ff;
    k.c0 = (float)(ff - R * R);
    k.outside = (ff - R * R) > 1e-3 * ff ? 1u : 0u;
}

void fill_sphere_consts(SphereK &S, double R, const double O[3])
{
    double ir = 1.0 / R, r2 = R * R;
    S.ir_h = (float)ir;
    S.ir_l = (float)(ir - (double)S.ir_h);
    S.r2_h = (float)r2;
    S.r2_l = (float)(r2 - (double)S.r2_h);
    S.inv_r2 = (float)(1.0 / r2);
    S.centred = (O[0] == 0.0 && O[1] == 0.0 && O[2] == 0.0) ? 1u : 0u;
    S.r32 = (float)R;
    for (int k = 0; k < 3; ++k) {
        S.o32[k] = (float)O[k];
        S.o_hi[k] = (float)O[k];
        S.o_lo[k] = (float)(O[k] - (double)S.o_hi[k]);
        S.o64[k] = O[k];
    }
}
}  // namespace lfk

extern "C" {

const char *lf_last_error(void) { return g_err.c_str(); }

const char *lf_version(void) { return "lumipath-gb300 0.1 (sm_103a)"; }

size_t lf_struct_size(int which)
{
    switch (which) {
    case 0: return sizeof(lf_table_desc);
    case 1: return sizeof(lf_view);
    case 2: return sizeof(lf_launch);
    case 3: return sizeof(lf_precompute_desc);
    case 4: return sizeof(lf_blob);
    default: return 0;
    }
}

int lf_device_sm_count(void)
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return n;
}

lf_status lf_create_table(const lf_table_desc *d, const void *radiance_dev, const float *row_scales_dev,
                          void *stream, lf_table **out)
{
    NvtxRange nvtx_("lf_create_table");
    g_err.clear();
    if (!out) return fail(LF_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    lf_status ds = lfk::check_desc(d);
    if (ds != LF_OK) return ds;
    if (!radiance_dev) return fail(LF_ERR_INVALID_ARG, "radiance is NULL");
    const uint32_t M = d->n_origins, N = d->n_directions, C = d->channels;
    const bool upper = (d->flags & LF_TABLE_UPPER_HEMISPHERE) != 0;
    const uint32_t rows = upper ? M / 2 : M;
    const bool quant = d->dtype != LF_DTYPE_F32;
    if (quant && !row_scales_dev) return fail(LF_ERR_INVALID_ARG, "F16/E4M3 tables need row scales");
    const bool borrow = (d->flags & LF_TABLE_BORROW) != 0;
    if (borrow && quant && C != 4)
        return fail(LF_ERR_INVALID_ARG, "a borrowed F16/E4M3 table must have 4 channels");
    if (borrow) {
        // texel loads: float4 (F32, 4 channels), float2 + float (F32, 3), uint2 (F16), uint32 (E4M3)
        const uintptr_t a = !quant ? (C == 4 ? 16 : 8) : (d->dtype == LF_DTYPE_F16 ? 8 : 4);
        if (misaligned(radiance_dev, a))
            return fail(LF_ERR_INVALID_ARG, "a borrowed table must be %u-byte aligned", (unsigned)a);
        if (misaligned(row_scales_dev, 4)) return fail(LF_ERR_INVALID_ARG, "row scales must be 4-byte aligned");
    }
    const uint64_t texels = (uint64_t)rows * N;
    if (texels > (1ull << 40)) return fail(LF_ERR_INVALID_ARG, "table too large");

    lf_table *t = new (std::nothrow) lf_table;
    if (!t) return fail(LF_ERR_OUT_OF_MEMORY, "host allocation failed");
    memset(t, 0, sizeof *t);
    t->desc = *d;
    t->C = C;
    t->rows = rows;
    t->launch = default_launch();
    cudaGetDevice(&t->device);
    t->sm_count = lf_device_sm_count();
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    auto bail = [&](lf_status s) { lf_destroy(t); return s; };

    e = cudaMalloc(&t->points, sizeof(float4) * 2ull * ((uint64_t)M + N));
    if (e != cudaSuccess) return bail(cuda_fail(e, "point cache allocation"));
    e = cudaMalloc(&t->scratch, lfk::kWordsBytes + sizeof(unsigned long long) * (size_t)lfk::kDeferCap);
    if (e != cudaSuccess) return bail(cuda_fail(e, "scratch allocation"));
    e = cudaMemsetAsync(t->scratch, 0, lfk::kWordsBytes, st);
    if (e != cudaSuccess) return bail(cuda_fail(e, "scratch clear"));
    e = lfk::launch_build_points(M, t->points, t->points + M, st);
    if (e == cudaSuccess) e = lfk::launch_build_points(N, t->points + 2 * (uint64_t)M, t->points + 2 * (uint64_t)M + N, st);
    if (e != cudaSuccess) return bail(cuda_fail(e, "point cache build"));

    if (!quant) t->texel_kind = C == 4 ? lfk::kF32C4 : lfk::kF32C3;
    else t->texel_kind = d->dtype == LF_DTYPE_F16 ? lfk::kF16C4 : lfk::kE4M3C4;

    if (borrow) {
        t->texels = radiance_dev;
        t->scales = quant ? row_scales_dev : nullptr;
    } else {
        const size_t cb = code_bytes(d->dtype);
        const uint32_t Cs = quant ? 4 : C;
        e = cudaMalloc(&t->owned_texels, texels * Cs * cb);
        if (e != cudaSuccess) return bail(cuda_fail(e, "table allocation"));
        if (quant && C == 3)
            e = lfk::launch_pad_codes(radiance_dev, rows, N, (int)cb, t->owned_texels, st);
        else
            e = cudaMemcpyAsync(t->owned_texels, radiance_dev, texels * Cs * cb, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return bail(cuda_fail(e, "table copy"));
        t->texels = t->owned_texels;
        if (quant) {
            e = cudaMalloc(&t->owned_scales, sizeof(float) * rows);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(t->owned_scales, row_scales_dev, sizeof(float) * rows, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return bail(cuda_fail(e, "scale copy"));
            t->scales = t->owned_scales;
        }
    }

    lfk::SphereK &S = t->sphere;
    lfk::fill_sphere_consts(S, d->radius, d->center);
    const double four_pi = 12.566370614359172953850573533118;
    t->po = {t->points, t->points + M, M, (float)M, (float)(1.0 / std::sqrt(four_pi / (double)M))};
    t->pd = {t->points + 2 * (uint64_t)M, t->points + 2 * (uint64_t)M + N, N, (float)N,
             (float)(1.0 / std::sqrt(four_pi / (double)N))};
    *out = t;
    return LF_OK;
}

void lf_destroy(lf_table *t)
{
    if (!t) return;
    if (t->points || t->scratch || t->owned_texels || t->owned_scales) cudaDeviceSynchronize();
    if (t->points) cudaFree(t->points);
    if (t->scratch) cudaFree(t->scratch);
    if (t->owned_texels) cudaFree(t->owned_texels);
    if (t->owned_scales) cudaFree(t->owned_scales);
    delete t;
}

lf_status lf_set_launch(lf_table *t, const lf_launch *cfg)
{
    if (!t) return fail(LF_ERR_INVALID_ARG, "table is NULL");
    lf_status s = lfk::check_launch(cfg);
    if (s != LF_OK) return s;
    t->launch = *cfg;
    return LF_OK;
}

lf_status lf_get_launch(const lf_table *t, lf_launch *cfg)
{
    if (!t || !cfg) return fail(LF_ERR_INVALID_ARG, "NULL argument");
    *cfg = t->launch;
    return LF_OK;
}

lf_status lf_render(const lf_table *t, const lf_view *views, uint32_t n_views, float *out_dev,
                    int32_t *idx_dev, void *stream)
{
    NvtxRange nvtx_("lf_render");
    g_err.clear();
    if (!t) return fail(LF_ERR_INVALID_ARG, "table is NULL");
    if (!out_dev) return fail(LF_ERR_INVALID_ARG, "out is NULL");
    return run(t, views, n_views, out_dev, idx_dev, nullptr, nullptr, stream);
}

lf_status lf_render_f16(const lf_table *t, const lf_view *views, uint32_t n_views, uint16_t *out_dev,
                        int32_t *idx_dev, void *stream)
{
    NvtxRange nvtx_("lf_render_f16");
    g_err.clear();
    if (!t) return fail(LF_ERR_INVALID_ARG, "table is NULL");
    if (!out_dev) return fail(LF_ERR_INVALID_ARG, "out is NULL");
    if (t->desc.k_nearest == 9) return fail(LF_ERR_UNSUPPORTED, "a binary16 image with 9 neighbours is not built");
    return run(t, views, n_views, reinterpret_cast<float *>(out_dev), idx_dev, nullptr, nullptr, stream, nullptr,
               true);
}

lf_status lf_render_backward(const lf_table *t, const lf_view *views, uint32_t n_views,
                             const float *grad_out_dev, float *grad_table_dev, void *stream)
{
    NvtxRange nvtx_("lf_render_backward");
    g_err.clear();
    if (!t) return fail(LF_ERR_INVALID_ARG, "table is NULL");
    if (!grad_out_dev || !grad_table_dev) return fail(LF_ERR_INVALID_ARG, "gradient buffer is NULL");
    return run(t, views, n_views, nullptr, nullptr, grad_out_dev, grad_table_dev, stream);
}

lf_status lf_render_backward_idx(const lf_table *t, const lf_view *views, uint32_t n_views,
                                 const float *grad_out_dev, const int32_t *idx_dev, float *grad_table_dev,
                                 void *stream)
{
    NvtxRange nvtx_("lf_render_backward_idx");
    g_err.clear();
    if (!t) return fail(LF_ERR_INVALID_ARG, "table is NULL");
    if (!grad_out_dev || !grad_table_dev) return fail(LF_ERR_INVALID_ARG, "gradient buffer is NULL");
    if (!idx_dev) return fail(LF_ERR_INVALID_ARG, "idx is NULL");
    return run(t, views, n_views, nullptr, nullptr, grad_out_dev, grad_table_dev, stream, idx_dev);
}

lf_status lf_sync_status(lf_table *t, void *stream)
{
    if (!t) return fail(LF_ERR_INVALID_ARG, "table is NULL");
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    uint32_t w = 0;
    e = cudaMemcpy(&w, t->scratch, sizeof w, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    if (w) {
        cudaMemset(t->scratch, 0, sizeof w);
        return fail(LF_ERR_DEVICE_CHECK, "device check failed (status word 0x%x)", w);
    }
    return LF_OK;
}

lf_status lf_quantize_table(const float *src_dev, uint32_t M, uint32_t N, uint32_t C, int32_t dtype,
                            void *codes_dev, float *scales_dev, void *stream)
{
    NvtxRange nvtx_("lf_quantize_table");
    g_err.clear();
    if (!src_dev || !codes_dev || !scales_dev) return fail(LF_ERR_INVALID_ARG, "NULL buffer");
    if (M == 0 || N == 0 || M > (1u << 24) || N > (1u << 24)) return fail(LF_ERR_INVALID_ARG, "bad M/N");
    if (C != 3 && C != 4) return fail(LF_ERR_INVALID_ARG, "channels must be 3 or 4");
    if (dtype != LF_DTYPE_F16 && dtype != LF_DTYPE_E4M3)
        return fail(LF_ERR_INVALID_ARG, "dtype must be F16 or E4M3");
    cudaError_t e = lfk::launch_quantize(src_dev, M, N, C, dtype, codes_dev, scales_dev, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "quantize launch");
    return LF_OK;
}

lf_status lf_fill_lobe_table(uint32_t M, uint32_t N, uint32_t C, uint32_t L, const double *ap,
                             const double *ad, const double *kp, const double *kd, const double *col,
                             uint64_t noise_seed, float *out_dev, void *stream)
{
    NvtxRange nvtx_("lf_fill_lobe_table");
    g_err.clear();
    if (!out_dev) return fail(LF_ERR_INVALID_ARG, "out is NULL");
    if (M == 0 || N == 0 || M > (1u << 24) || N > (1u << 24)) return fail(LF_ERR_INVALID_ARG, "bad M/N");
    if (C != 3 && C != 4) return fail(LF_ERR_INVALID_ARG, "channels must be 3 or 4");
    if (L > (uint32_t)lfk::kMaxLobes) return fail(LF_ERR_INVALID_ARG, "at most %d lobes", lfk::kMaxLobes);
    if (L && (!ap || !ad || !kp || !kd || !col)) return fail(LF_ERR_INVALID_ARG, "NULL lobe array");
    static thread_local lfk::LobeParams P;
    memset(&P, 0, sizeof P);
    P.L = L;
    P.C = C;
    P.seed = noise_seed;
    for (uint32_t l = 0; l < L; ++l) {
        for (int k = 0; k < 3; ++k) {
            P.ap[l][k] = ap[3 * l + k];
            P.ad[l][k] = ad[3 * l + k];
        }
        P.kp[l] = kp[l];
        P.kd[l] = kd[l];
        for (uint32_t c = 0; c < C; ++c) P.col[l][c] = col[C * l + c];
    }
    cudaStream_t st = (cudaStream_t)stream;
    float4 *pts = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&pts, sizeof(float4) * 2ull * ((uint64_t)M + N), st);
    if (e != cudaSuccess) return cuda_fail(e, "point allocation");
    e = lfk::launch_build_points(M, pts, pts + M, st);
    if (e == cudaSuccess) e = lfk::launch_build_points(N, pts + 2 * (uint64_t)M, pts + 2 * (uint64_t)M + N, st);
    if (e == cudaSuccess)
        e = lfk::launch_fill_lobe(P, pts, pts + M, pts + 2 * (uint64_t)M, pts + 2 * (uint64_t)M + N, M, N,
                                  out_dev, st);
    cudaError_t e2 = cudaFreeAsync(pts, st);
    if (e != cudaSuccess) return cuda_fail(e, "lobe fill");
    if (e2 != cudaSuccess) return cuda_fail(e2, "point free");
    return LF_OK;
}

lf_status lf_precompute_table(const lf_precompute_desc *d, const lf_blob *blobs, float *out_dev,
                              void *stream)
{
    NvtxRange nvtx_("lf_precompute_table");
    g_err.clear();
    if (!d) return fail(LF_ERR_INVALID_ARG, "desc is NULL");
    if (!out_dev) return fail(LF_ERR_INVALID_ARG, "out is NULL");
    const uint32_t M = d->n_origins, N = d->n_directions;
    if (M == 0 || N == 0 || M > (1u << 24) || N > (1u << 24)) return fail(LF_ERR_INVALID_ARG, "bad M/N");
    if (d->rows == 0 || d->rows > M) return fail(LF_ERR_INVALID_ARG, "rows must be in [1, M] (got %u)", d->rows);
    if (d->spp == 0 || d->spp > 1024) return fail(LF_ERR_INVALID_ARG, "spp must be in [1, 1024]");
    if (d->jitter > 1) return fail(LF_ERR_INVALID_ARG, "jitter must be 0 or 1");
    static thread_local lfk::PrecomputeParams P;
    lf_status s = volume_params(d, blobs, out_dev, P);
    if (s != LF_OK) return s;
    P.disk_r = (float)(2.0 * d->radius / std::sqrt((double)M));
    P.N = N;
    P.rows = d->rows;
    P.spp = d->spp;
    P.jitter = d->jitter;
    P.seed = d->seed;
    cudaStream_t st = (cudaStream_t)stream;
    float4 *pts = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&pts, sizeof(float4) * 2ull * ((uint64_t)M + N), st);
    if (e != cudaSuccess) return cuda_fail(e, "point allocation");
    P.po_hi = pts;
    P.po_lo = pts + M;
    P.pd_hi = pts + 2 * (uint64_t)M;
    P.pd_lo = pts + 2 * (uint64_t)M + N;
    e = lfk::launch_build_points(M, pts, pts + M, st);
    if (e == cudaSuccess) e = lfk::launch_build_points(N, pts + 2 * (uint64_t)M, pts + 2 * (uint64_t)M + N, st);
    if (e == cudaSuccess) e = lfk::launch_precompute(P, st);
    cudaError_t e2 = cudaFreeAsync(pts, st);
    if (e != cudaSuccess) return cuda_fail(e, "precompute");
    if (e2 != cudaSuccess) return cuda_fail(e2, "point free");
    return LF_OK;
}

lf_status lf_render_volume(const lf_precompute_desc *d, const lf_blob *blobs, const lf_view *views,
                           uint32_t n_views, float *out_dev, void *stream)
{
    NvtxRange nvtx_("lf_render_volume");
    g_err.clear();
    if (!d) return fail(LF_ERR_INVALID_ARG, "desc is NULL");
    if (!out_dev) return fail(LF_ERR_INVALID_ARG, "out is NULL");
    static thread_local lfk::PrecomputeParams P;
    lf_status s = volume_params(d, blobs, out_dev, P);
    if (s != LF_OK) return s;
    s = lfk::check_views(views, n_views);
    if (s != LF_OK) return s;
    lfk::SphereK S{};
    lfk::fill_sphere_consts(S, d->radius, d->center);
    cudaStream_t st = (cudaStream_t)stream;
    for (uint32_t v = 0; v < n_views; ++v) {
        cudaError_t e = lfk::launch_volume_direct(P, lfk::camera_of(views[v]), S, d->radius, st);
        if (e != cudaSuccess) return cuda_fail(e, "direct volume render");
    }
    return LF_OK;
}

lf_status lf_post_filter(double radius, const double center[3], uint32_t channels, const float *weights_host,
                         const lf_view *views, uint32_t n_views, const float *in_dev, float *out_dev,
                         void *stream)
{
    NvtxRange nvtx_("lf_post_filter");
    g_err.clear();
    static_assert(lfk::kPostWeights == (int)LF_POST_WEIGHTS, "post-filter weight count");
    if (!center || !weights_host || !in_dev || !out_dev)
        return fail(LF_ERR_INVALID_ARG, "center, weights, in and out must not be NULL");
    if (!(radius > 0.0) || !std::isfinite(radius) || !finite3(center))
        return fail(LF_ERR_INVALID_ARG, "R must be positive and finite, O finite");
    if (channels != 3 && channels != 4) return fail(LF_ERR_INVALID_ARG, "channels must be 3 or 4");
    if (misaligned(in_dev, 4) || misaligned(out_dev, 4))
        return fail(LF_ERR_INVALID_ARG, "in and out must be 4-byte aligned");
    lf_status s = lfk::check_views(views, n_views);
    if (s != LF_OK) return s;
    uint64_t P = 0;
    for (uint32_t v = 0; v < n_views; ++v) {
        const uint64_t end = views[v].out_offset + (uint64_t)views[v].width * views[v].height;
        P = end > P ? end : P;
    }
    const uintptr_t a = (uintptr_t)in_dev, b = (uintptr_t)out_dev, bytes = (uintptr_t)(P * channels * 4);
    if (a < b + bytes && b < a + bytes) return fail(LF_ERR_INVALID_ARG, "out must not overlap in");
    for (uint32_t k = 0; k < LF_POST_WEIGHTS; ++k)
        if (!std::isfinite(weights_host[k])) return fail(LF_ERR_INVALID_ARG, "weight %u is not finite", k);
    // PostParams holds 13 KB of weights: keep it off the stack
    static thread_local lfk::PostParams p;
    memset(&p, 0, sizeof p);
    lfk::fill_sphere_consts(p.sphere, radius, center);
    memcpy(p.w, weights_host, sizeof p.w);
    p.in = in_dev;
    p.out = out_dev;
    p.C = channels;
    cudaStream_t st = (cudaStream_t)stream;
    for (uint32_t v0 = 0; v0 < n_views; v0 += lfk::kPostMaxViews) {
        const uint32_t nv = n_views - v0 < (uint32_t)lfk::kPostMaxViews ? n_views - v0 : (uint32_t)lfk::kPostMaxViews;
        for (uint32_t v = 0; v < nv; ++v) {
            p.views[v] = lfk::camera_of(views[v0 + v]);
            lfk::fill_view_miss_consts(p.views[v], radius, center);   // the certain hit/miss tests of the mask
        }
        p.n_views = nv;
        cudaError_t e = lfk::launch_post_filter(p, st);
        if (e != cudaSuccess) return cuda_fail(e, "post-filter");
    }
    return LF_OK;
}

}  // extern "C"
