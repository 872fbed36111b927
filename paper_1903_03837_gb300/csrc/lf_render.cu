// lf_render.cu -- forward render and backward scatter kernels of the
// light-field sampling path (LumiPath, arXiv 1903.03837, Section 2).
//
// One thread per camera ray. A CTA renders a tile of tile_w x tile_h pixels of
// one view; each warp covers a warp_w x (32/warp_w) sub-tile so that its rays
// hit neighbouring SF cells and share texels in L1. Tiles of all views of a
// call are numbered consecutively (view-major); a CTA either takes tile
// blockIdx.x (static grid) or pulls tiles from a queue word (persistent grid
// of SMs x occupancy CTAs; the last CTA to leave resets the queue, so the
// launch is replayable, e.g. from a CUDA graph). Views live in the kernel's
// parameter space (no device copy, graph friendly).
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "lf_device.cuh"
#include "lf_kernels.h"

// Resident CTAs of kMaxBlock threads per SM the register budget is cut for:
// 4 -> 64 registers, 32 warps per SM (forward and backward).
#ifndef LF_MIN_BLOCKS
#define LF_MIN_BLOCKS 4
#endif

namespace lfk {

// Tile t of the launch -> (view, tile column, tile row). Runs in one thread
// per CTA; the result is shared through shared memory.
__device__ __forceinline__ void tile_of(const RenderParamsBase &p, const ViewK *views,
                                        const uint32_t *prefix, uint32_t nv, uint32_t t,
                                        uint32_t &v, uint32_t &tx, uint32_t &ty)
{
    uint32_t lo = 0, hi = nv;          // largest v with prefix[v] <= t
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (prefix[mid] <= t) lo = mid; else hi = mid;
    }
    v = lo;
    uint32_t lt = t - prefix[v];
    uint32_t tiles_x = views[v].tiles_x;
    if (p.order == 0) {
        ty = lt / tiles_x;
        tx = lt - ty * tiles_x;
    } else {                           // strips of kStripTiles tile rows, column by column
        uint32_t strip = lt / (tiles_x * kStripTiles);
        uint32_t r = lt - strip * tiles_x * kStripTiles;
        uint32_t hs = min(kStripTiles, views[v].tiles_y - strip * kStripTiles);
        tx = r / hs;
        ty = strip * kStripTiles + (r - tx * hs);
    }
}

// Pixel of this thread in tile (tx, ty): tile and warp shapes are powers of
// two, so the mapping is shifts and masks.
__device__ __forceinline__ void pixel_of(const RenderParamsBase &p, uint32_t tx, uint32_t ty,
                                         uint32_t &px, uint32_t &py)
{
    uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t wx_log = p.tw_log - p.ww_log;              // log2(warps per tile row)
    px = (tx << p.tw_log) + ((warp & ((1u << wx_log) - 1u)) << p.ww_log) + (lane & ((1u << p.ww_log) - 1u));
    py = (ty << p.th_log) + ((warp >> wx_log) << (5u - p.ww_log)) + (lane >> p.ww_log);
}

// Weights of one set's neighbours r (set 0: origins, 1: directions) by the
// sampling mode; false when the ray is masked (an upper-hemisphere table with
// no stored origin neighbour).
template <int K>
__device__ __forceinline__ bool set_weights(const RenderParamsBase &p, int s, float inv_sigma, TopK<K> &r,
                                            float (&w)[K])
{
    if (p.nearest_only) {
        // nearest sampling: the nearest point alone (Section 2, Fig. 2)
        if (s == 0 && p.rows_stored && (uint32_t)r.i[0] >= p.rows_stored) return false;
#pragma unroll
        for (int m = 0; m < K; ++m) w[m] = m == 0 ? 1.0f : 0.0f;
#pragma unroll
        for (int m = 1; m < K; ++m) r.i[m] = -1;
        return true;
    }
    if (s == 0 && p.rows_stored) return tent_weights_kept(r.d2, r.i, r.cnt, inv_sigma, p.rows_stored, w);
    tent_weights(r.d2, r.cnt, inv_sigma, w);
    return true;
}

__device__ __forceinline__ PointSetK point_set(const RenderParamsBase &p, int s)
{
    PointSetK P;
    P.hi = s ? p.pd.hi : p.po.hi;
    P.lo = s ? p.pd.lo : p.po.lo;
    P.n = s ? p.pd.n : p.po.n;
    P.nf = s ? p.pd.nf : p.po.nf;
    P.inv_sigma = s ? p.pd.inv_sigma : p.po.inv_sigma;
    return P;
}

// Indices and normalised weights of one ray of unit direction d (K = 5 or 9
// neighbours per hit); false for a miss. With five neighbours, a set whose tier-1 order was not
// certain sets bit s of `pend` and leaves its samples empty; resolve_pending
// fills them in once the warp has reconverged.
template <int K>
__device__ __forceinline__ bool ray_samples(const RenderParamsBase &p, const ViewK &v, float3 d,
                                            int32_t (&io)[K], int32_t (&jd)[K], float (&wo)[K],
                                            float (&wd)[K], uint32_t &pend)
{
    // The origin set's indices and weights wait in shared memory (one slot per
    // thread, no synchronisation) while the direction set is searched: 2K
    // fewer live registers across the second search.
    __shared__ int s_stash[2 * K * kMaxBlock];
    float3 ho, hd;
    if (!intersect_sphere(p.sphere, v.eye, d, ho, hd)) return false;
    // One copy of the index step serves both sets (instruction-cache footprint).
#pragma unroll 1
    for (int s = 0; s < 2; ++s) {
        const PointSetK P = point_set(p, s);
        TopK<K> r;
        bool unc = false;
        if constexpr (K == 9)
            r = knn9(P, p.sphere, s ? hd : ho, p.status);
        else
            r = knn5(P, p.sphere, s ? hd : ho, p.status, unc);
        float w[K];
        if (unc) {
            pend |= 1u << s;
#pragma unroll
            for (int m = 0; m < K; ++m) w[m] = 0.0f;
        } else if (!set_weights<K>(p, s, P.inv_sigma, r, w)) {
            pend = 0;
            return false;
        }
        if (s == 0) {
#pragma unroll
            for (int m = 0; m < K; ++m) {
                s_stash[m * kMaxBlock + threadIdx.x] = r.i[m];
                s_stash[(K + m) * kMaxBlock + threadIdx.x] = __float_as_int(w[m]);
            }
        } else {
#pragma unroll
            for (int m = 0; m < K; ++m) {
                jd[m] = r.i[m];
                wd[m] = w[m];
            }
        }
    }
#pragma unroll
    for (int m = 0; m < K; ++m) {
        io[m] = s_stash[m * kMaxBlock + threadIdx.x];
        wo[m] = __int_as_float(s_stash[(K + m) * kMaxBlock + threadIdx.x]);
    }
    return true;
}

// Queues ray (view vi, pixel px, py) for the fixup kernel; bit s of pend marks
// a set whose search was not certain. When the queue is full the count still
// grows past defer_cap, which tells the fixup kernel to render every ray.
__device__ __forceinline__ void defer_push(const RenderParamsBase &p, uint32_t vi, uint32_t px, uint32_t py,
                                           uint32_t pend)
{
    const unsigned long long slot = atomicAdd(p.defer_count, 1ull);
    if (slot < p.defer_cap)
        p.defer_items[slot] = ((unsigned long long)pend << 48) | ((unsigned long long)vi << 32) |
                              ((unsigned long long)py << 16) | px;
}

// The samples of one ray from the indices a forward pass wrote for it (idx_in:
// [P][2K], or [P][2] with nearest sampling): the hits and unit hits are
// recomputed and the weights formed from the double-float distances of these
// indices -- the same distances, by the same function, as the index step's, so
// the weights are identical. An index out of range counts as missing and sets
// bit 0 of the status word; a ray the indices call a hit but that misses S sets
// bit 1.
template <int K>
__device__ __forceinline__ bool samples_from_idx(const RenderParamsBase &p, const ViewK &v, uint32_t px,
                                                 uint32_t py, uint64_t pix, int32_t (&io)[K], int32_t (&jd)[K],
                                                 float (&wo)[K], float (&wd)[K])
{
    const int32_t *q = p.idx_in + pix * (uint64_t)(p.nearest_only ? 2 : 2 * K);
#pragma unroll
    for (int m = 0; m < K; ++m) io[m] = jd[m] = -1;
    if (p.nearest_only) {
        io[0] = __ldg(q);
        jd[0] = __ldg(q + 1);
    } else {
#pragma unroll
        for (int m = 0; m < K; ++m) {
            io[m] = __ldg(q + m);
            jd[m] = __ldg(q + K + m);
        }
    }
    if (io[0] < 0) return false;
    float3 d = camera_dir(v, px, py);
    float3 ho, hd;
    if (!intersect_sphere(p.sphere, v.eye, d, ho, hd)) {
        atomicOr(p.status, kStatusIdxInput);
        return false;
    }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        PointSetK P;
        P.hi = s ? p.pd.hi : p.po.hi;
        P.lo = s ? p.pd.lo : p.po.lo;
        P.n = s ? p.pd.n : p.po.n;
        P.inv_sigma = s ? p.pd.inv_sigma : p.po.inv_sigma;
        int32_t (&ix)[K] = s ? jd : io;
        float(&w)[K] = s ? wd : wo;
        float3 qh, ql;
        unit_hit_df(p.sphere, s ? hd : ho, qh, ql);
        float d2[K];
        int cnt = 0;
#pragma unroll
        for (int m = 0; m < K; ++m) {
            const bool ok = (uint32_t)ix[m] < P.n;
            if (!ok && ix[m] >= 0) {
                atomicOr(p.status, kStatusIndex);
                ix[m] = -1;
            }
            d2[m] = ok ? dist2_df(P, ok ? ix[m] : 0, qh, ql) : 0.0f;
            cnt += ok ? 1 : 0;
        }
        if (p.nearest_only) {
#pragma unroll
            for (int m = 0; m < K; ++m) w[m] = m == 0 ? 1.0f : 0.0f;
        } else if (s == 0 && p.rows_stored) {
            if (!tent_weights_kept(d2, ix, cnt, P.inv_sigma, p.rows_stored, w)) return false;
        } else {
            tent_weights(d2, cnt, P.inv_sigma, w);
        }
    }
    return true;
}

// binary16 image: the FP32 result rounded once (half the bytes to read back).
__device__ __forceinline__ void store_f16(float *out, uint32_t C, uint64_t pix, float4 acc)
{
    const __half2 xy = __floats2half2_rn(acc.x, acc.y), zw = __floats2half2_rn(acc.z, acc.w);
    if (C == 4) {
        uint2 v;
        v.x = *reinterpret_cast<const uint32_t *>(&xy);
        v.y = *reinterpret_cast<const uint32_t *>(&zw);
        __stcs(reinterpret_cast<uint2 *>(out) + pix, v);
    } else {
        unsigned short *o = reinterpret_cast<unsigned short *>(out) + pix * 3;
        __stcs(o, __half_as_ushort(__low2half(xy)));
        __stcs(o + 1, __half_as_ushort(__high2half(xy)));
        __stcs(o + 2, __half_as_ushort(__low2half(zw)));
    }
}

// Packed FP32 pair FMA (one instruction for two lanes of a texel).
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c)
{
    unsigned long long ra = *reinterpret_cast<unsigned long long *>(&a);
    unsigned long long rb = *reinterpret_cast<unsigned long long *>(&b);
    unsigned long long rc = *reinterpret_cast<unsigned long long *>(&c);
    unsigned long long rd;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(rd) : "l"(ra), "l"(rb), "l"(rc));
    return *reinterpret_cast<float2 *>(&rd);
}

// Image and index output of one ray.
template <int K, bool F16>
__device__ __forceinline__ void store_ray(const RenderParamsBase &p, const ViewK &v, uint32_t px, uint32_t py,
                                          float4 acc, const int32_t (&io)[K], const int32_t (&jd)[K])
{
    const uint64_t pix = v.out_offset + (uint64_t)py * v.width + px;
    if constexpr (F16) {
        store_f16(p.out, p.C, pix, acc);
    } else if (p.C == 4) {
        __stcs(reinterpret_cast<float4 *>(p.out) + pix, acc);
    } else {
        float *o = p.out + pix * 3;
        __stcs(o, acc.x);
        __stcs(o + 1, acc.y);
        __stcs(o + 2, acc.z);
    }
    if (p.idx) {
        if constexpr (K == 9) {
            int2 *q = reinterpret_cast<int2 *>(p.idx + pix * 18);
#pragma unroll
            for (int m = 0; m < 9; ++m) {
                const int e0 = 2 * m, e1 = 2 * m + 1;
                q[m] = make_int2(e0 < 9 ? io[e0] : jd[e0 - 9], e1 < 9 ? io[e1] : jd[e1 - 9]);
            }
        } else if (p.nearest_only) {
            reinterpret_cast<int2 *>(p.idx)[pix] = make_int2(io[0], jd[0]);
        } else {
            int2 *q = reinterpret_cast<int2 *>(p.idx + pix * 10);
            q[0] = make_int2(io[0], io[1]);
            q[1] = make_int2(io[2], io[3]);
            q[2] = make_int2(io[4], jd[0]);
            q[3] = make_int2(jd[1], jd[2]);
            q[4] = make_int2(jd[3], jd[4]);
        }
    }
}

// Tap (i, j) of the blend: weight-scaled texel accumulated in FP32 pairs.
template <int DT>
__device__ __forceinline__ void blend_tap(const RenderParamsBase &p, size_t row, int32_t j, float w, bool live,
                                          int32_t j0, float2 &in_xy, float2 &in_zw)
{
    // a dead tap reads column j0 of its row (finite) with weight 0: a branch
    // around the load costs more than the load; j0 is the lane's nearest
    // direction, so in a live row that texel is loaded anyway (an L1 hit)
    const float4 t = texel<DT>(p.texels, LF_DINDEX(row + (uint32_t)(live ? j : j0), (uint64_t)p.rows_valid * p.N,
                                                   p.status, kStatusDebugTexel));
    w = live ? w : 0.0f;
    const float2 w2 = make_float2(w, w);
    in_xy = ffma2(w2, make_float2(t.x, t.y), in_xy);
    in_zw = ffma2(w2, make_float2(t.z, t.w), in_zw);
}

template <int DT, int K, bool F16>
__device__ __forceinline__ void render_ray(const RenderParamsBase &p, const ViewK &v, uint32_t vi, bool active,
                                           uint32_t px, uint32_t py)
{
    // initialised even though every path writes them before use: measured 1.6%
    // faster than leaving them undefined on the miss path
    int32_t io[K], jd[K];
    float wo[K], wd[K];
#pragma unroll
    for (int m = 0; m < K; ++m) {
        io[m] = jd[m] = -1;
        wo[m] = wd[m] = 0.0f;
    }
    float2 acc_xy = make_float2(0.f, 0.f), acc_zw = make_float2(0.f, 0.f);
    uint32_t pend = 0;
    const bool hit = active && !certain_miss(v, px, py) && ray_samples<K>(p, v, camera_dir(v, px, py), io, jd, wo, wd, pend);
    // Origin rows past every lane's last tap of weight > 0 are skipped. The
    // neighbours of a set are sorted by distance and the tent gives every one
    // beyond the kernel radius weight 0, so the nonzero weights of a set sit in
    // a prefix (nearest sampling: the first; unstored rows of an upper-hemisphere
    // table may leave zeros inside it). The loop over origin neighbours runs to
    // the longest such prefix of the warp -- a bound every lane shares, reached
    // by all 32 lanes (every lane of a tile calls this function); within it a
    // lane's taps of weight 0 read, without a branch, its nearest direction
    // column of the row (the direction taps are not cut short: a bound there
    // measured slower). Every texel is finite (the FP32 table is the caller's
    // promise; the FP16 and E4M3 codes are finite by construction), so a dead
    // tap adds exactly the 0 that its weight gives.
    int no = 0;
#pragma unroll
    for (int m = 0; m < K; ++m) no = wo[m] != 0.0f ? m + 1 : no;
    const int no_w = (int)__reduce_max_sync(0xffffffffu, (unsigned)no);
    // The 81 taps of K = 9 keep the outer loop rolled (instruction-cache footprint).
#pragma unroll(K == 5 ? 5 : 1)
    for (int a = 0; a < K; ++a) {
        if (a >= no_w) break;
        // origin neighbour a by a select chain: with the loop rolled (K = 9) a
        // run-time index would move the arrays to local memory; unrolled (K = 5)
        // the chain folds away
        int32_t ia = io[0];
        float wa = wo[0];
#pragma unroll
        for (int m = 1; m < K; ++m) {
            ia = (a == m) ? io[m] : ia;
            wa = (a == m) ? wo[m] : wa;
        }
        const bool la = wa != 0.0f;
        // a missing or unstored neighbour has weight 0 and reads within row 0
        const int32_t i = la ? ia : 0;
        float s = wa;
        if constexpr (DT == kF16C4 || DT == kE4M3C4) s *= la ? __ldg(p.scales + i) : 0.0f;
        const size_t row = (size_t)i * p.N;
        float2 in_xy = make_float2(0.f, 0.f), in_zw = make_float2(0.f, 0.f);
#pragma unroll
        for (int b = 0; b < K; ++b)
            blend_tap<DT>(p, row, jd[b], wd[b], la && wd[b] != 0.0f, max(jd[0], 0), in_xy, in_zw);
        const float2 s2 = make_float2(s, s);
        acc_xy = ffma2(s2, in_xy, acc_xy);
        acc_zw = ffma2(s2, in_zw, acc_zw);
    }
    if (!active) return;
    if (pend) {
        // the fixup kernel renders this ray (the weights of its uncertain set
        // were 0 above, so it read nothing)
        defer_push(p, vi, px, py, pend);
        return;
    }
    if (!hit) {
#pragma unroll
        for (int a = 0; a < K; ++a) io[a] = jd[a] = -1;
    }
    store_ray<K, F16>(p, v, px, py, make_float4(acc_xy.x, acc_xy.y, acc_zw.x, acc_zw.y), io, jd);
}

// Position of the n-th (0-based) set bit of m (m has more than n set bits).
__device__ __forceinline__ int nth_set_bit(unsigned m, int n)
{
    int pos = 0, c;
    c = __popc(m & 0xffffu); if (n >= c) { n -= c; m >>= 16; pos += 16; }
    c = __popc(m & 0xffu);   if (n >= c) { n -= c; m >>= 8;  pos += 8; }
    c = __popc(m & 0xfu);    if (n >= c) { n -= c; m >>= 4;  pos += 4; }
    c = __popc(m & 0x3u);    if (n >= c) { n -= c; m >>= 2;  pos += 2; }
    c = (int)(m & 1u);       if (n >= c) { pos += 1; }
    return pos;
}

// Sum of `val` over the lanes of this lane's group `grp` (lanes holding the
// same texel key), delivered to the group's lowest lane: a binary tree over the
// members' ranks, log2(largest group) rounds. Every lane of the warp calls it.
__device__ __forceinline__ float4 group_sum_tree(float4 val, unsigned grp, unsigned lane)
{
    const int rank = __popc(grp & ((1u << lane) - 1u));
    const int size = __popc(grp);
    const int maxsize = (int)__reduce_max_sync(0xffffffffu, (unsigned)size);
    for (int off = 1; off < maxsize; off <<= 1) {
        bool recv = (rank & (2 * off - 1)) == 0 && rank + off < size;
        int src = recv ? nth_set_bit(grp, rank + off) : (int)lane;
        float4 o;
        o.x = __shfl_sync(0xffffffffu, val.x, src);
        o.y = __shfl_sync(0xffffffffu, val.y, src);
        o.z = __shfl_sync(0xffffffffu, val.z, src);
        o.w = __shfl_sync(0xffffffffu, val.w, src);
        if (recv) {
            val.x += o.x; val.y += o.y; val.z += o.z; val.w += o.w;
        }
    }
    return val;
}

__device__ __forceinline__ void add_to_grad(const RenderParamsBase &p, uint64_t key, float4 sum)
{
    key = LF_DINDEX(key, (uint64_t)p.rows_valid * p.N, p.status, kStatusDebugGrad);
    if (p.C == 4) {
        atomicAdd(reinterpret_cast<float4 *>(p.grad) + key, sum);
    } else {
        float *q = p.grad + key * 3;
        atomicAdd(q, sum.x);
        atomicAdd(q + 1, sum.y);
        atomicAdd(q + 2, sum.z);
    }
}

// dL/d(image) of pixel pix.
__device__ __forceinline__ float4 grad_of(const RenderParamsBase &p, uint64_t pix)
{
    if (p.C == 4) return __ldg(reinterpret_cast<const float4 *>(p.grad_out) + pix);
    const float *q = p.grad_out + pix * 3;
    return make_float4(__ldg(q), __ldg(q + 1), __ldg(q + 2), 0.f);
}

// The warp-aggregated scatter of the taps of one warp's rays (every lane of
// the warp calls it; lanes without a hit contribute nothing).
template <int K>
__device__ __forceinline__ void backward_taps(const RenderParamsBase &p, bool hit, const int32_t (&io)[K],
                                              const int32_t (&jd)[K], const float (&wo)[K], const float (&wd)[K],
                                              float4 g)
{
    const unsigned lane = threadIdx.x & 31;
    // Both neighbour sets wait in a per-thread shared-memory slot during the tap
    // loop (no synchronisation: each thread reads only its own slot): twenty
    // registers fewer than keeping them live, 8% faster.
    __shared__ int s_bw[4 * K * kMaxBlock];
#pragma unroll
    for (int m = 0; m < K; ++m) {
        s_bw[m * kMaxBlock + threadIdx.x] = io[m];
        s_bw[(K + m) * kMaxBlock + threadIdx.x] = __float_as_int(wo[m]);
        s_bw[(2 * K + m) * kMaxBlock + threadIdx.x] = jd[m];
        s_bw[(3 * K + m) * kMaxBlock + threadIdx.x] = __float_as_int(wd[m]);
    }
#pragma unroll 1
    for (int a = 0; a < K; ++a) {
        const int32_t ia = s_bw[a * kMaxBlock + threadIdx.x];
        const float wa = __int_as_float(s_bw[(K + a) * kMaxBlock + threadIdx.x]);
#pragma unroll
        for (int b = 0; b < K; ++b) {
            const int32_t jb = s_bw[(2 * K + b) * kMaxBlock + threadIdx.x];
            const float wb = __int_as_float(s_bw[(3 * K + b) * kMaxBlock + threadIdx.x]);
            // a tap of weight 0 (beyond the kernel radius in either set) would add
            // exactly 0: it takes no atomic
            bool live = hit && (uint32_t)ia < p.rows_valid && jb >= 0 && wa != 0.0f && wb != 0.0f;
            uint64_t key = live ? (uint64_t)ia * p.N + (uint64_t)jb : 0ull;
            float W = live ? wa * wb : 0.f;
            float4 val = make_float4(W * g.x, W * g.y, W * g.z, W * g.w);
            unsigned live_mask = __ballot_sync(0xffffffffu, live);
            if (live_mask == 0u) continue;
            const int leader = __ffs(live_mask) - 1;
            uint64_t lkey = __shfl_sync(0xffffffffu, key, leader);
            if (__all_sync(0xffffffffu, !live || key == lkey)) {
#pragma unroll
                for (int s = 16; s >= 1; s >>= 1) {
                    val.x += __shfl_xor_sync(0xffffffffu, val.x, s);
                    val.y += __shfl_xor_sync(0xffffffffu, val.y, s);
                    val.z += __shfl_xor_sync(0xffffffffu, val.z, s);
                    val.w += __shfl_xor_sync(0xffffffffu, val.w, s);
                }
                if ((int)lane == leader) add_to_grad(p, lkey, val);
            } else {
                unsigned grp = __match_any_sync(0xffffffffu, live ? key : ~0ull - lane);
                float4 sum = group_sum_tree(val, grp, lane);
                if (live && (__ffs(grp) - 1) == (int)lane) add_to_grad(p, key, sum);
            }
        }
    }
}
// Backward of one ray: grad[i_a][j_b] += W_ab * g for the K x K taps. Lanes that
// hold the same texel key are summed first (warp aggregation): when every live
// lane of the warp has the same key, a butterfly over the warp and one atomic;
// otherwise __match_any_sync groups and a tree sum per group, one atomic per
// group. The loop over origin neighbours stays rolled (instruction-cache
// footprint) and the K direction taps inside it unrolled; both read the
// neighbours from shared memory (a run-time index into register arrays would
// move them to local memory).
template <int K>
__device__ __forceinline__ void backward_ray(const RenderParamsBase &p, const ViewK *v, uint32_t vi, bool active,
                                             uint32_t px, uint32_t py)
{
    int32_t io[K], jd[K];
    float wo[K], wd[K];
#pragma unroll
    for (int m = 0; m < K; ++m) {
        io[m] = jd[m] = -1;
        wo[m] = wd[m] = 0.0f;
    }
    bool hit = false;
    uint32_t pend = 0;
    float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
    if (active) {
        uint64_t pix = v->out_offset + (uint64_t)py * v->width + px;
        hit = p.idx_in ? samples_from_idx<K>(p, *v, px, py, pix, io, jd, wo, wd)
                       : (!certain_miss(*v, px, py) &&
                          ray_samples<K>(p, *v, camera_dir(*v, px, py), io, jd, wo, wd, pend));
        g = grad_of(p, pix);
    }
    if (pend) {
        defer_push(p, vi, px, py, pend);   // scattered by the fixup kernel
        hit = false;
    }
    if (__any_sync(0xffffffffu, hit)) backward_taps<K>(p, hit, io, jd, wo, wd, g);
}



template <int DT, int MAXV, bool BWD, int K, bool F16 = false>
__global__ void __launch_bounds__(kMaxBlock, K == 5 ? LF_MIN_BLOCKS : 2)
    render_kernel(const __grid_constant__ RenderParams<MAXV> p)
{
    __shared__ uint32_t s_tile[4];     // view, tile column, tile row, valid
    const uint32_t nv = p.n_views;
    for (;;) {
        if (threadIdx.x == 0) {
            uint32_t t = p.persistent ? atomicAdd(p.queue, 1u) : blockIdx.x;
            uint32_t v = 0, tx = 0, ty = 0;
            bool ok = t < p.total_tiles;
            if (ok) tile_of(p, p.views, p.tile_prefix, nv, t, v, tx, ty);
            s_tile[0] = v;
            s_tile[1] = tx;
            s_tile[2] = ty;
            s_tile[3] = ok;
        }
        __syncthreads();
        const uint32_t v = s_tile[0], tx = s_tile[1], ty = s_tile[2];
        if (!s_tile[3]) break;
        const ViewK &vw = p.views[v];
        uint32_t px, py;
        pixel_of(p, tx, ty, px, py);
        bool active = px < vw.width && py < vw.height;
        if constexpr (BWD) {
            backward_ray<K>(p, &vw, v, active, px, py);
        } else {
            render_ray<DT, K, F16>(p, vw, v, active, px, py);
        }
        if (!p.persistent) break;
        __syncthreads();               // everyone has read s_tile before it is rewritten
    }
    if (p.persistent && threadIdx.x == 0) {
        __threadfence();
        uint32_t done = atomicAdd(p.done, 1u);
        if (done == gridDim.x - 1) {                  // last CTA out: re-arm the queue
            atomicExch(p.queue, 0u);
            atomicExch(p.done, 0u);
        }
    }
}

// One ray rendered (or its gradient scattered) by a whole warp: the sets
// marked in pend ranked exactly by coop_knn5, weights as in the render kernel,
// then lane 0 blends or scatters the taps of nonzero weight. Every lane of the
// warp calls it with the same pixel (pend = 3 when the queue overflowed).
template <int DT, bool BWD, bool F16>
__device__ __forceinline__ void exact_ray(const RenderParamsBase &p, const ViewK &v, uint32_t px, uint32_t py,
                                          uint32_t pend)
{
    int32_t io[5], jd[5];
    float wo[5], wd[5];
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        io[m] = jd[m] = -1;
        wo[m] = wd[m] = 0.0f;
    }
    float3 ho, hd;
    bool hit = intersect_sphere(p.sphere, v.eye, camera_dir(v, px, py), ho, hd);
    if (hit) {
        const PointSetK Po = point_set(p, 0), Pd = point_set(p, 1);
        // a set the render kernel settled gives the same samples by its search
        // again (in every lane alike); the other is ranked by the whole warp
        bool unc = false;
        TopK<5> ro = (pend & 1u) ? coop_knn5(Po, p.sphere, ho) : knn5(Po, p.sphere, ho, p.status, unc);
        TopK<5> rd = (pend & 2u) ? coop_knn5(Pd, p.sphere, hd) : knn5(Pd, p.sphere, hd, p.status, unc);
        hit = set_weights<5>(p, 0, Po.inv_sigma, ro, wo) && set_weights<5>(p, 1, Pd.inv_sigma, rd, wd);
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            io[m] = hit ? ro.i[m] : -1;
            jd[m] = hit ? rd.i[m] : -1;
            wo[m] = hit ? wo[m] : 0.0f;
            wd[m] = hit ? wd[m] : 0.0f;
        }
    }
    if ((threadIdx.x & 31u) != 0u) return;
    if constexpr (BWD) {
        if (!hit) return;
        const float4 g = grad_of(p, v.out_offset + (uint64_t)py * v.width + px);
#pragma unroll
        for (int a = 0; a < 5; ++a) {
            if (wo[a] == 0.0f || (uint32_t)io[a] >= p.rows_valid) continue;
#pragma unroll
            for (int b = 0; b < 5; ++b) {
                if (wd[b] == 0.0f || jd[b] < 0) continue;
                const float W = wo[a] * wd[b];
                add_to_grad(p, (uint64_t)io[a] * p.N + (uint64_t)jd[b], make_float4(W * g.x, W * g.y, W * g.z, W * g.w));
            }
        }
    } else {
        float2 acc_xy = make_float2(0.f, 0.f), acc_zw = make_float2(0.f, 0.f);
#pragma unroll
        for (int a = 0; a < 5; ++a) {
            const bool la = wo[a] != 0.0f;
            const int32_t i = la ? io[a] : 0;
            float s = wo[a];
            if constexpr (DT == kF16C4 || DT == kE4M3C4) s *= la ? __ldg(p.scales + i) : 0.0f;
            const size_t row = (size_t)i * p.N;
            float2 in_xy = make_float2(0.f, 0.f), in_zw = make_float2(0.f, 0.f);
#pragma unroll
            for (int b = 0; b < 5; ++b)
                blend_tap<DT>(p, row, jd[b], wd[b], la && wd[b] != 0.0f, max(jd[0], 0), in_xy, in_zw);
            const float2 s2 = make_float2(s, s);
            acc_xy = ffma2(s2, in_xy, acc_xy);
            acc_zw = ffma2(s2, in_zw, acc_zw);
        }
        store_ray<5, F16>(p, v, px, py, make_float4(acc_xy.x, acc_xy.y, acc_zw.x, acc_zw.y), io, jd);
    }
}

// The rays the render kernel queued, one warp per ray; when more were queued
// than the queue holds, every ray of the launch (the exact path gives the same
// result for the rays the render kernel finished). The last CTA to finish
// resets the queue for the next launch (replayable, e.g. from a CUDA graph).
template <int DT, int MAXV, bool BWD, bool F16>
__global__ void __launch_bounds__(kFixupThreads) fixup_kernel(const __grid_constant__ RenderParams<MAXV> p)
{
    const unsigned long long queued = *reinterpret_cast<volatile unsigned long long *>(p.defer_count);
    const bool all = queued > p.defer_cap;
    const unsigned long long total = all ? p.total_pixels : queued;
    const unsigned long long nw = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    for (unsigned long long e = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < total; e += nw) {
        uint32_t vi = 0, px, py, pend = 3u;
        if (!all) {
            const unsigned long long it = p.defer_items[e];
            pend = (uint32_t)(it >> 48) & 3u;
            vi = (uint32_t)(it >> 32) & 0xffffu;
            py = (uint32_t)(it >> 16) & 0xffffu;
            px = (uint32_t)it & 0xffffu;
        } else {
            unsigned long long r = e;
            while (r >= (unsigned long long)p.views[vi].width * p.views[vi].height) {
                r -= (unsigned long long)p.views[vi].width * p.views[vi].height;
                ++vi;
            }
            py = (uint32_t)(r / p.views[vi].width);
            px = (uint32_t)(r - (unsigned long long)py * p.views[vi].width);
        }
        exact_ray<DT, BWD, F16>(p, p.views[vi], px, py, pend);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(p.defer_done, 1u) == gridDim.x - 1) {
            atomicExch(p.defer_count, 0ull);
            atomicExch(p.defer_done, 0u);
        }
    }
}

// Grid of a fixup kernel: as many CTAs as its registers let the SMs hold at
// once (a few queued rays per warp at most), found once per device and thread.
template <int DT, int MAXV, bool BWD, bool F16>
static unsigned fixup_grid()
{
    static thread_local int dev_cached = -1;
    static thread_local unsigned grid = kFixupCtas;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return kFixupCtas;
    if (dev != dev_cached) {
        int sms = 0, per_sm = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fixup_kernel<DT, MAXV, BWD, F16>,
                                                          (int)kFixupThreads, 0) == cudaSuccess &&
            sms > 0 && per_sm > 0)
            grid = (unsigned)(sms * per_sm);
        dev_cached = dev;
    }
    return grid;
}

template <int MAXV, int K, bool F16>
static cudaError_t launch_k(int kind, bool bwd, const RenderParams<MAXV> &p, unsigned grid, unsigned block,
                            cudaStream_t st)
{
    // five neighbours: the fixup kernel follows on the same stream (nine never defer)
    const unsigned fb = kFixupThreads;
    if (bwd) {
        render_kernel<kF32C4, MAXV, true, K><<<grid, block, 0, st>>>(p);
        if (K == 5) fixup_kernel<kF32C4, MAXV, true, false><<<fixup_grid<kF32C4, MAXV, true, false>(), fb, 0, st>>>(p);
    } else {
        switch (kind) {
        case kF32C4:
            render_kernel<kF32C4, MAXV, false, K, F16><<<grid, block, 0, st>>>(p);
            if (K == 5) fixup_kernel<kF32C4, MAXV, false, F16><<<fixup_grid<kF32C4, MAXV, false, F16>(), fb, 0, st>>>(p);
            break;
        case kF32C3:
            render_kernel<kF32C3, MAXV, false, K, F16><<<grid, block, 0, st>>>(p);
            if (K == 5) fixup_kernel<kF32C3, MAXV, false, F16><<<fixup_grid<kF32C3, MAXV, false, F16>(), fb, 0, st>>>(p);
            break;
        case kF16C4:
            render_kernel<kF16C4, MAXV, false, K, F16><<<grid, block, 0, st>>>(p);
            if (K == 5) fixup_kernel<kF16C4, MAXV, false, F16><<<fixup_grid<kF16C4, MAXV, false, F16>(), fb, 0, st>>>(p);
            break;
        default:
            render_kernel<kE4M3C4, MAXV, false, K, F16><<<grid, block, 0, st>>>(p);
            if (K == 5) fixup_kernel<kE4M3C4, MAXV, false, F16><<<fixup_grid<kE4M3C4, MAXV, false, F16>(), fb, 0, st>>>(p);
            break;
        }
    }
    return cudaGetLastError();
}

// Five neighbours: FP32 or binary16 image; nine neighbours: FP32 image (the
// host refuses a binary16 image with nine).
template <int MAXV>
static cudaError_t launch_t(int kind, bool bwd, const RenderParams<MAXV> &p, unsigned grid,
                            unsigned block, cudaStream_t st)
{
    if (p.nine) return launch_k<MAXV, 9, false>(kind, bwd, p, grid, block, st);
    return p.out_f16 && !bwd ? launch_k<MAXV, 5, true>(kind, bwd, p, grid, block, st)
                             : launch_k<MAXV, 5, false>(kind, bwd, p, grid, block, st);
}

template <int MAXV, int K, bool F16>
static int occupancy_k(int kind, bool bwd, unsigned block)
{
    int n = 0;
    const void *f;
    if (bwd) f = (const void *)render_kernel<kF32C4, MAXV, true, K>;
    else if (kind == kF32C4) f = (const void *)render_kernel<kF32C4, MAXV, false, K, F16>;
    else if (kind == kF32C3) f = (const void *)render_kernel<kF32C3, MAXV, false, K, F16>;
    else if (kind == kF16C4) f = (const void *)render_kernel<kF16C4, MAXV, false, K, F16>;
    else f = (const void *)render_kernel<kE4M3C4, MAXV, false, K, F16>;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, (int)block, 0) != cudaSuccess) n = 1;
    return n > 0 ? n : 1;
}

cudaError_t launch_render_small(int kind, bool bwd, const RenderParams<kSmallViews> &p, unsigned grid,
                                unsigned block, cudaStream_t st)
{
    return launch_t<kSmallViews>(kind, bwd, p, grid, block, st);
}
cudaError_t launch_render_large(int kind, bool bwd, const RenderParams<kLargeViews> &p, unsigned grid,
                                unsigned block, cudaStream_t st)
{
    return launch_t<kLargeViews>(kind, bwd, p, grid, block, st);
}
int render_occupancy(int kind, bool bwd, bool large, bool nine, unsigned block)
{
    if (nine)
        return large ? occupancy_k<kLargeViews, 9, false>(kind, bwd, block)
                     : occupancy_k<kSmallViews, 9, false>(kind, bwd, block);
    return large ? occupancy_k<kLargeViews, 5, false>(kind, bwd, block)
                 : occupancy_k<kSmallViews, 5, false>(kind, bwd, block);
}

}  // namespace lfk
