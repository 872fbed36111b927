// lf_noalloc.cu -- lf_render_noalloc: a render that allocates no device memory.
//
// lf_create_table allocates the SF point caches, a copy of the table and a
// few status/queue words with cudaMalloc. Some callers cannot do that: a
// process whose device memory is already fully reserved by another runtime's
// memory pool (cudaMalloc would fail), or a frame-paced render loop that must
// not call cudaMalloc/cudaFree because they synchronise the device and have
// unbounded latency. For them this entry point keeps everything it needs
// beyond the caller's inputs and outputs in one file-scope device array of
// fixed size, g_lf_noalloc_scratch, which every GPU that loads the library
// holds until the process exits.
//
// Layout of the array: the hi/lo point caches of both SF sets (M + N points,
// 32 B each), then 256 B of words (status, tile queue, finished CTAs, the
// count of rays queued for the exact fixup pass), then the queue itself
// (kNoAllocDeferCap entries of 8 B). Every call rebuilds the point caches and
// clears the words on its stream, so the array only ever holds the last
// call's contents; calls that overlap on the GPU (different streams, or
// another thread) race on it.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "lf_kernels.h"
#include "lumipath.h"

namespace {

constexpr uint64_t kNoAllocMaxPoints = LF_NOALLOC_MAX_POINTS;     // M + N
constexpr uint64_t kWordsFloat4 = lfk::kWordsBytes / 16;             // 256 B of words
constexpr uint32_t kNoAllocDeferCap = LF_NOALLOC_MAX_DEFERRED;       // queued rays per launch
constexpr uint64_t kQueueFloat4 = kNoAllocDeferCap / 2;              // 8 B per queued ray

static __device__ __align__(256) float4 g_lf_noalloc_scratch[2 * kNoAllocMaxPoints + kWordsFloat4 + kQueueFloat4];

lf_status na_fail(lf_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    lfk::set_last_error(buf);
    return s;
}

// Host code must not use g_lf_noalloc_scratch directly: on the host it names a
// stand-in object, not device memory. Its device address is looked up on every
// call, with the caller's device current: the lookup allocates nothing, and an
// address kept from an earlier call could belong to a context that has since
// been torn down (cudaDeviceReset), where it would no longer be valid.
lf_status scratch_address(float4 **out)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_lf_noalloc_scratch);
    if (e != cudaSuccess || !p)
        return na_fail(LF_ERR_CUDA, "cudaGetSymbolAddress of the no-allocation scratch: %s", cudaGetErrorString(e));
    *out = (float4 *)p;
    return LF_OK;
}

template <int MAXV>
lf_status launch_views(const lfk::RenderParamsBase &base, const lf_launch &L, int kind, int sm_count,
                       const lf_view *views, uint32_t nv, const lf_table_desc *d, cudaStream_t st)
{
    static thread_local lfk::RenderParams<MAXV> p;
    static_cast<lfk::RenderParamsBase &>(p) = base;
    uint64_t tiles = 0;
    p.total_pixels = 0;
    for (uint32_t v = 0; v < nv; ++v) {
        p.views[v] = lfk::view_params(views[v], L, d->radius, d->center);
        p.tile_prefix[v] = (uint32_t)tiles;
        tiles += (uint64_t)p.views[v].tiles_x * p.views[v].tiles_y;
        p.total_pixels += (uint64_t)views[v].width * views[v].height;
    }
    if (tiles >= (1ull << 31)) return na_fail(LF_ERR_INVALID_ARG, "too many tiles in one launch");
    p.tile_prefix[nv] = (uint32_t)tiles;
    p.n_views = nv;
    p.total_tiles = (uint32_t)tiles;
    unsigned block = L.tile_w * L.tile_h;
    unsigned grid = (unsigned)tiles;
    if (L.persistent) {
        int per_sm = L.ctas_per_sm ? (int)L.ctas_per_sm
                                   : lfk::render_occupancy(kind, false, MAXV != lfk::kSmallViews, false, block);
        uint64_t g = (uint64_t)sm_count * (uint64_t)per_sm;
        grid = (unsigned)(g < tiles ? g : tiles);
    }
    if (grid == 0) return LF_OK;
    cudaError_t e;
    if constexpr (MAXV == lfk::kSmallViews)
        e = lfk::launch_render_small(kind, false, p, grid, block, st);
    else
        e = lfk::launch_render_large(kind, false, p, grid, block, st);
    if (e != cudaSuccess) return na_fail(LF_ERR_CUDA, "render launch: %s", cudaGetErrorString(e));
    return LF_OK;
}

}  // namespace

extern "C" {

lf_status lf_render_noalloc(const lf_table_desc *d, const void *radiance_dev, const float *row_scales_dev,
                            const lf_view *views, uint32_t n_views, const lf_launch *launch,
                            float *out_dev, int32_t *idx_dev, void *stream)
{
    lfk::set_last_error("");
    lf_status s = lfk::check_desc(d);
    if (s != LF_OK) return s;
    if (!radiance_dev || !out_dev) return na_fail(LF_ERR_INVALID_ARG, "NULL argument");
    const uint32_t M = d->n_origins, N = d->n_directions, C = d->channels;
    if ((uint64_t)M + N > kNoAllocMaxPoints)
        return na_fail(LF_ERR_INVALID_ARG,
                       "M + N = %llu exceeds the no-allocation scratch limit of %llu points",
                       (unsigned long long)M + N, (unsigned long long)kNoAllocMaxPoints);
    const bool quant = d->dtype != LF_DTYPE_F32;
    if (quant && (C != 4 || !row_scales_dev))
        return na_fail(LF_ERR_INVALID_ARG, "F16/E4M3 tables need 4 channels and row scales here");
    if (d->k_nearest == 9) return na_fail(LF_ERR_UNSUPPORTED, "1 or 5 neighbours per hit here (9: lf_render)");
    {
        // natural alignment of the vector accesses (a misaligned pointer is an argument error)
        const uintptr_t ta = !quant ? (C == 4 ? 16 : 8) : (d->dtype == LF_DTYPE_F16 ? 8 : 4);
        const uintptr_t oa = C == 4 ? 16 : 4;
        if (((uintptr_t)radiance_dev & (ta - 1)) || ((uintptr_t)out_dev & (oa - 1)) ||
            ((uintptr_t)idx_dev & 7u) || ((uintptr_t)row_scales_dev & 3u))
            return na_fail(LF_ERR_INVALID_ARG, "misaligned table, scale, image or index buffer");
    }
    s = lfk::check_views(views, n_views);
    if (s != LF_OK) return s;
    lf_launch L = {16, 16, 8, 0, 0, 0};
    if (launch) {
        s = lfk::check_launch(launch);
        if (s != LF_OK) return s;
        L = *launch;
    }

    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(LF_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    float4 *base = nullptr;
    s = scratch_address(&base);
    if (s != LF_OK) return s;
    int sm_count = 0;
    e = cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || sm_count <= 0)
        return na_fail(LF_ERR_CUDA, "SM count of device %d: %s", dev, cudaGetErrorString(e));
    cudaStream_t st = (cudaStream_t)stream;
    float4 *po_hi = base, *po_lo = base + M, *pd_hi = base + 2 * (uint64_t)M, *pd_lo = pd_hi + N;
    uint32_t *words = reinterpret_cast<uint32_t *>(base + 2 * kNoAllocMaxPoints);
    e = cudaMemsetAsync(words, 0, kWordsFloat4 * sizeof(float4), st);
    if (e == cudaSuccess) e = lfk::launch_build_points(M, po_hi, po_lo, st);
    if (e == cudaSuccess) e = lfk::launch_build_points(N, pd_hi, pd_lo, st);
    if (e != cudaSuccess) return na_fail(LF_ERR_CUDA, "scratch set-up: %s", cudaGetErrorString(e));

    lfk::RenderParamsBase b;
    memset(&b, 0, sizeof b);
    lfk::fill_sphere_consts(b.sphere, d->radius, d->center);
    const double four_pi = 12.566370614359172953850573533118;
    b.po = {po_hi, po_lo, M, (float)M, (float)(1.0 / std::sqrt(four_pi / (double)M))};
    b.pd = {pd_hi, pd_lo, N, (float)N, (float)(1.0 / std::sqrt(four_pi / (double)N))};
    b.texels = radiance_dev;
    b.scales = quant ? row_scales_dev : nullptr;
    b.N = N;
    b.C = C;
    b.out = out_dev;
    b.idx = idx_dev;
    b.status = words;
    b.queue = words + 1;
    b.done = words + 2;
    b.defer_done = words + 3;
    b.defer_count = reinterpret_cast<unsigned long long *>(words + 4);
    b.defer_items = reinterpret_cast<unsigned long long *>(base + 2 * kNoAllocMaxPoints + kWordsFloat4);
    b.defer_cap = kNoAllocDeferCap;
    b.tile_w = L.tile_w;
    b.tile_h = L.tile_h;
    b.warp_w = L.warp_w;
    b.order = L.order;
    b.persistent = L.persistent;
    b.tw_log = (uint32_t)__builtin_ctz(L.tile_w);
    b.th_log = (uint32_t)__builtin_ctz(L.tile_h);
    b.ww_log = (uint32_t)__builtin_ctz(L.warp_w);
    const bool upper = (d->flags & LF_TABLE_UPPER_HEMISPHERE) != 0;
    b.rows_valid = upper ? M / 2 : M;
    b.nearest_only = d->k_nearest == 1 ? 1u : 0u;
    b.rows_stored = upper ? M / 2 : 0u;
    int kind = !quant ? (C == 4 ? lfk::kF32C4 : lfk::kF32C3) : (d->dtype == LF_DTYPE_F16 ? lfk::kF16C4 : lfk::kE4M3C4);
    if (n_views <= (uint32_t)lfk::kSmallViews)
        return launch_views<lfk::kSmallViews>(b, L, kind, sm_count, views, n_views, d, st);
    for (uint32_t v0 = 0; v0 < n_views; v0 += lfk::kLargeViews) {
        uint32_t nv = n_views - v0 < (uint32_t)lfk::kLargeViews ? n_views - v0 : (uint32_t)lfk::kLargeViews;
        s = launch_views<lfk::kLargeViews>(b, L, kind, sm_count, views + v0, nv, d, st);
        if (s != LF_OK) return s;
    }
    return LF_OK;
}

lf_status lf_noalloc_sync_status(void *stream)
{
    lfk::set_last_error("");
    float4 *base = nullptr;
    lf_status s = scratch_address(&base);
    if (s != LF_OK) return s;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return na_fail(LF_ERR_CUDA, "stream synchronize: %s", cudaGetErrorString(e));
    uint32_t *words = reinterpret_cast<uint32_t *>(base + 2 * kNoAllocMaxPoints);
    uint32_t w = 0;
    e = cudaMemcpy(&w, words, sizeof w, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return na_fail(LF_ERR_CUDA, "status read: %s", cudaGetErrorString(e));
    if (w) {
        e = cudaMemset(words, 0, sizeof w);
        if (e != cudaSuccess) return na_fail(LF_ERR_CUDA, "status clear: %s", cudaGetErrorString(e));
        return na_fail(LF_ERR_DEVICE_CHECK, "device check failed (status word 0x%x)", w);
    }
    return LF_OK;
}

}  // extern "C"
