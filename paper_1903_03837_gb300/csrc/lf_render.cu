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

// Indices and normalised weights of one ray (K = 5 or 9 neighbours per hit);
// false for a miss.
template <int K>
__device__ __forceinline__ bool ray_samples(const RenderParamsBase &p, const ViewK &v, uint32_t px,
                                            uint32_t py, int32_t (&io)[K], int32_t (&jd)[K], float (&wo)[K],
                                            float (&wd)[K])
{
    // The origin set's indices and weights wait in shared memory (one slot per
    // thread, no synchronisation) while the direction set is searched: 2K
    // fewer live registers across the second search.
    __shared__ int s_stash[2 * K * kMaxBlock];
    float3 d = camera_dir(v, px, py);
    float3 ho, hd;
    if (!intersect_sphere(p.sphere, v.eye, d, ho, hd)) return false;
    // One copy of the index step serves both sets (instruction-cache footprint).
#pragma unroll 1
    for (int s = 0; s < 2; ++s) {
        PointSetK P;
        P.hi = s ? p.pd.hi : p.po.hi;
        P.lo = s ? p.pd.lo : p.po.lo;
        P.n = s ? p.pd.n : p.po.n;
        P.nf = s ? p.pd.nf : p.po.nf;
        P.inv_sigma = s ? p.pd.inv_sigma : p.po.inv_sigma;
        TopK<K> r;
        if constexpr (K == 9)
            r = knn9(P, p.sphere, s ? hd : ho, p.status);
        else
            r = knn5(P, p.sphere, s ? hd : ho, p.status);
        float w[K];
        if (p.nearest_only) {
            // nearest sampling: the nearest point alone (Section 2, Fig. 2)
            if (s == 0 && p.rows_stored && (uint32_t)r.i[0] >= p.rows_stored) return false;
#pragma unroll
            for (int m = 0; m < K; ++m) w[m] = m == 0 ? 1.0f : 0.0f;
#pragma unroll
            for (int m = 1; m < K; ++m) r.i[m] = -1;
        } else if (s == 0 && p.rows_stored) {
            if (!tent_weights_kept(r.d2, r.i, r.cnt, P.inv_sigma, p.rows_stored, w)) return false;
        } else {
            tent_weights(r.d2, r.cnt, P.inv_sigma, w);
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

template <int DT, int K, bool F16>
__device__ __forceinline__ void render_ray(const RenderParamsBase &p, const ViewK &v, uint32_t px,
                                           uint32_t py)
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
    bool hit = !certain_miss(v, px, py) && ray_samples(p, v, px, py, io, jd, wo, wd);
    if (hit) {
        // All K x K taps in every mode: with nearest sampling the other 24 have
        // weight 0 and index -1 (row 0, texel 0, an L1 hit), which costs less
        // than a second copy of the loop. The 81 taps of K = 9 keep the outer
        // loop rolled (instruction-cache footprint).
#pragma unroll(K == 5 ? 5 : 1)
        for (int a = 0; a < K; ++a) {
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
            // Nine neighbours: the tent gives the outer ones weight 0 almost always;
            // their taps are skipped (a branch that whole warps take together).
            if constexpr (K == 9) {
                if (wa == 0.0f) continue;
            }
            // a missing or unstored neighbour has weight 0 and reads row 0
            int32_t i = (uint32_t)ia < p.rows_valid ? ia : 0;
            float s = wa;
            if constexpr (DT == kF16C4 || DT == kE4M3C4) s *= __ldg(p.scales + i);
            size_t row = (size_t)i * p.N;
            float2 in_xy = make_float2(0.f, 0.f), in_zw = make_float2(0.f, 0.f);
#pragma unroll
            for (int b = 0; b < K; ++b) {
                if constexpr (K == 9) {
                    if (wd[b] == 0.0f) continue;
                }
                float4 t = texel<DT>(p.texels, LF_DINDEX(row + (uint32_t)max(jd[b], 0), (uint64_t)p.rows_valid * p.N,
                                                          p.status, kStatusDebugTexel));
                float2 w2 = make_float2(wd[b], wd[b]);
                in_xy = ffma2(w2, make_float2(t.x, t.y), in_xy);
                in_zw = ffma2(w2, make_float2(t.z, t.w), in_zw);
            }
            float2 s2 = make_float2(s, s);
            acc_xy = ffma2(s2, in_xy, acc_xy);
            acc_zw = ffma2(s2, in_zw, acc_zw);
        }
    } else {
#pragma unroll
        for (int a = 0; a < K; ++a) io[a] = jd[a] = -1;
    }
    const float4 acc = make_float4(acc_xy.x, acc_xy.y, acc_zw.x, acc_zw.y);
    uint64_t pix = v.out_offset + (uint64_t)py * v.width + px;
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

// Backward of one ray: grad[i_a][j_b] += W_ab * g for the K x K taps. Lanes that
// hold the same texel key are summed first (warp aggregation): when every live
// lane of the warp has the same key, a butterfly over the warp and one atomic;
// otherwise __match_any_sync groups and a tree sum per group, one atomic per
// group. The loop over origin neighbours stays rolled (instruction-cache
// footprint) and the K direction taps inside it unrolled; both read the
// neighbours from shared memory (a run-time index into register arrays would
// move them to local memory).
template <int K>
__device__ __forceinline__ void backward_ray(const RenderParamsBase &p, const ViewK *v, bool active,
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
    float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
    if (active) {
        uint64_t pix = v->out_offset + (uint64_t)py * v->width + px;
        hit = p.idx_in ? samples_from_idx<K>(p, *v, px, py, pix, io, jd, wo, wd)
                       : (!certain_miss(*v, px, py) && ray_samples<K>(p, *v, px, py, io, jd, wo, wd));
        if (p.C == 4) {
            g = __ldg(reinterpret_cast<const float4 *>(p.grad_out) + pix);
        } else {
            const float *q = p.grad_out + pix * 3;
            g = make_float4(__ldg(q), __ldg(q + 1), __ldg(q + 2), 0.f);
        }
    }
    const unsigned lane = threadIdx.x & 31;
    if (!__any_sync(0xffffffffu, hit)) return;
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
            bool live = hit && (uint32_t)ia < p.rows_valid && jb >= 0;
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
        uint32_t px, py;
        pixel_of(p, tx, ty, px, py);
        const ViewK &vw = p.views[v];
        bool active = px < vw.width && py < vw.height;
        if constexpr (BWD) {
            backward_ray<K>(p, &vw, active, px, py);
        } else {
            if (active) render_ray<DT, K, F16>(p, vw, px, py);
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

template <int MAXV, int K, bool F16>
static cudaError_t launch_k(int kind, bool bwd, const RenderParams<MAXV> &p, unsigned grid, unsigned block,
                            cudaStream_t st)
{
    if (bwd) {
        render_kernel<kF32C4, MAXV, true, K><<<grid, block, 0, st>>>(p);
    } else {
        switch (kind) {
        case kF32C4: render_kernel<kF32C4, MAXV, false, K, F16><<<grid, block, 0, st>>>(p); break;
        case kF32C3: render_kernel<kF32C3, MAXV, false, K, F16><<<grid, block, 0, st>>>(p); break;
        case kF16C4: render_kernel<kF16C4, MAXV, false, K, F16><<<grid, block, 0, st>>>(p); break;
        default: render_kernel<kE4M3C4, MAXV, false, K, F16><<<grid, block, 0, st>>>(p); break;
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
