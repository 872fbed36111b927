// lf_post.cu -- learned post-filter of the light-field render (Section 2,
// post-processing: a network that removes the interpolation artifacts of the
// light-field image). Only the image-to-image filter is built -- three 3x3
// convolution layers, 4 -> 16 -> 16 -> 3 channels with ReLU after the first
// two, added to the input colour (residual) -- not the adversarial training of
// the paper. Input features per pixel: the light-field RGB and the hit mask of
// the pixel's ray (1 if the ray meets S); pixels whose ray misses S stay 0, as
// the render leaves them. Zero padding at the view border before every layer,
// the same semantics as a framework convolution with padding 1.
//
// One CTA of 256 threads per 14x30 output tile of one view (the tiles of all
// views of a launch numbered consecutively), FP32 on the CUDA cores. The 20x36
// input tile with its mask, the 18x34 first-layer and the 16x32 second-layer
// activations live in shared memory. The first and third layers (14% of the
// multiply-adds) take their weights from the kernel's parameter block as
// constant-bank operands, fully unrolled. The second layer (86%) computes two
// vertically adjacent positions per thread, loops over its 16 input channels
// without unrolling (a small loop body for the instruction cache) and reads the
// weights of each input channel as 16-byte shared-memory broadcasts, each used
// for both positions. The layers are 16 channels wide: too narrow to fill a
// tensor-core tile.
#include <cuda_runtime.h>

#include "lf_device.cuh"
#include "lf_kernels.h"

namespace lfk {

constexpr int kPW = 14, kPHt = 30;                 // output tile (width x height)
constexpr int kL2W = kPW + 2, kL2H = kPHt + 2;     // 16 x 32 second-layer activations
constexpr int kL1W = kPW + 4, kL1H = kPHt + 4;     // 18 x 34 first-layer activations
constexpr int kInW = kPW + 6, kInH = kPHt + 6;     // 20 x 36 input tile
constexpr int kL1S = 24;                           // row stride of the first-layer tile: two rows
                                                   // apart (the lanes' position pairs) = 16 banks
constexpr int kW2S = 12;                           // 9 weights of (i, o) padded to three float4
constexpr size_t kPostSmem = sizeof(float) * (4 * kInW * kInH + kPostHidden * kL1H * kL1S +
                                              kPostHidden * kL2W * kL2H + kPostHidden * kPostHidden * kW2S);

__global__ void __launch_bounds__(256, 2) post_filter_kernel(const __grid_constant__ PostParams p)
{
    extern __shared__ float4 sm4[];
    float *s_w2 = reinterpret_cast<float *>(sm4);              // [i][o][12]
    float *s_in = s_w2 + kPostHidden * kPostHidden * kW2S;      // [4][kInH][kInW]: R, G, B, hit mask
    float *s_h1 = s_in + 4 * kInW * kInH;                       // [16][kL1H][kL1S]
    float *s_h2 = s_h1 + kPostHidden * kL1H * kL1S;             // [16][kL2H][kL2W]
    __shared__ uint32_t s_tile[3];
    const int tid = threadIdx.x;
    if (tid == 0) {
        uint32_t lo = 0, hi = p.n_views;                 // largest v with tile_prefix[v] <= blockIdx.x
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (p.tile_prefix[mid] <= blockIdx.x) lo = mid; else hi = mid;
        }
        const uint32_t lt = blockIdx.x - p.tile_prefix[lo];
        s_tile[0] = lo;
        s_tile[1] = lt % p.views[lo].tiles_x;
        s_tile[2] = lt / p.views[lo].tiles_x;
    }
    for (int k = tid; k < kPostHidden * kPostHidden * kW2S; k += blockDim.x) {
        const int i = k / (kPostHidden * kW2S), r = k - i * (kPostHidden * kW2S);
        const int o = r / kW2S, t = r - o * kW2S;
        s_w2[k] = t < 9 ? p.w[kPostW2 + (o * kPostHidden + i) * 9 + t] : 0.0f;
    }
    __syncthreads();
    const ViewK &v = p.views[s_tile[0]];
    const int x0 = (int)s_tile[1] * kPW, y0 = (int)s_tile[2] * kPHt;
    const int W = (int)v.width, H = (int)v.height;

    for (int k = tid; k < kInW * kInH; k += blockDim.x) {
        const int ty = k / kInW, tx = k - ty * kInW;
        const int x = x0 - 3 + tx, y = y0 - 3 + ty;
        float r = 0.0f, g = 0.0f, b = 0.0f, m = 0.0f;
        if (x >= 0 && y >= 0 && x < W && y < H) {
            const float *q = p.in + (v.out_offset + (uint64_t)y * W + x) * p.C;
            r = __ldg(q);
            g = __ldg(q + 1);
            b = __ldg(q + 2);
            const float3 d = camera_dir(v, (uint32_t)x, (uint32_t)y);
            float3 ho, hd;
            m = intersect_sphere(p.sphere, v.eye, d, ho, hd) ? 1.0f : 0.0f;
        }
        s_in[k] = r;
        s_in[kInW * kInH + k] = g;
        s_in[2 * kInW * kInH + k] = b;
        s_in[3 * kInW * kInH + k] = m;
    }
    __syncthreads();

    // layer 1: 4 -> 16 channels on the 18x34 tile (weights as constant operands)
    for (int k = tid; k < kL1W * kL1H; k += blockDim.x) {
        const int ty = k / kL1W, tx = k - ty * kL1W;
        const int x = x0 - 2 + tx, y = y0 - 2 + ty;
        const bool inside = x >= 0 && y >= 0 && x < W && y < H;
        float acc[kPostHidden];
#pragma unroll
        for (int o = 0; o < kPostHidden; ++o) acc[o] = p.w[kPostB1 + o];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float in[9];
#pragma unroll
            for (int t = 0; t < 9; ++t) in[t] = s_in[i * kInW * kInH + (ty + t / 3) * kInW + tx + t % 3];
#pragma unroll
            for (int o = 0; o < kPostHidden; ++o)
#pragma unroll
                for (int t = 0; t < 9; ++t) acc[o] = fmaf(p.w[kPostW1 + (o * 4 + i) * 9 + t], in[t], acc[o]);
        }
#pragma unroll
        for (int o = 0; o < kPostHidden; ++o) s_h1[o * kL1H * kL1S + ty * kL1S + tx] = inside ? fmaxf(acc[o], 0.0f) : 0.0f;
    }
    __syncthreads();

    // layer 2: 16 -> 16 channels on the 16x32 tile, rows 2r and 2r + 1 of column c per thread
    {
        const int c = tid % kL2W, r2 = 2 * (tid / kL2W);
        const int x = x0 - 1 + c, ya = y0 - 1 + r2;
        const bool in_x = x >= 0 && x < W;
        const bool inside_a = in_x && ya >= 0 && ya < H, inside_b = in_x && ya + 1 >= 0 && ya + 1 < H;
        float acc_a[kPostHidden], acc_b[kPostHidden];
#pragma unroll
        for (int o = 0; o < kPostHidden; ++o) acc_a[o] = acc_b[o] = p.w[kPostB2 + o];
#pragma unroll 1
        for (int i = 0; i < kPostHidden; ++i) {
            float in[4][3];
            const float *src = s_h1 + i * kL1H * kL1S + r2 * kL1S + c;
#pragma unroll
            for (int rr = 0; rr < 4; ++rr)
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) in[rr][cc] = src[rr * kL1S + cc];
            const float4 *wrow = reinterpret_cast<const float4 *>(s_w2 + i * kPostHidden * kW2S);
#pragma unroll
            for (int o = 0; o < kPostHidden; ++o) {
                const float4 w0 = wrow[o * 3], w1 = wrow[o * 3 + 1], w2 = wrow[o * 3 + 2];
                const float w[9] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w, w2.x};
#pragma unroll
                for (int t = 0; t < 9; ++t) {
                    acc_a[o] = fmaf(w[t], in[t / 3][t % 3], acc_a[o]);
                    acc_b[o] = fmaf(w[t], in[t / 3 + 1][t % 3], acc_b[o]);
                }
            }
        }
#pragma unroll
        for (int o = 0; o < kPostHidden; ++o) {
            s_h2[o * kL2W * kL2H + r2 * kL2W + c] = inside_a ? fmaxf(acc_a[o], 0.0f) : 0.0f;
            s_h2[o * kL2W * kL2H + (r2 + 1) * kL2W + c] = inside_b ? fmaxf(acc_b[o], 0.0f) : 0.0f;
        }
    }
    __syncthreads();

    // layer 3: 16 -> 3 channels (weights as constant operands), added to the input
    // colour of hit pixels
    for (int k = tid; k < kPW * kPHt; k += blockDim.x) {
        const int ty = k / kPW, tx = k - ty * kPW;
        const int x = x0 + tx, y = y0 + ty;
        if (x >= W || y >= H) continue;
        float acc[3] = {p.w[kPostB3], p.w[kPostB3 + 1], p.w[kPostB3 + 2]};
#pragma unroll
        for (int i = 0; i < kPostHidden; ++i) {
            float in[9];
#pragma unroll
            for (int t = 0; t < 9; ++t) in[t] = s_h2[i * kL2W * kL2H + (ty + t / 3) * kL2W + tx + t % 3];
#pragma unroll
            for (int o = 0; o < 3; ++o)
#pragma unroll
                for (int t = 0; t < 9; ++t)
                    acc[o] = fmaf(p.w[kPostW3 + (o * kPostHidden + i) * 9 + t], in[t], acc[o]);
        }
        const int ci = (ty + 3) * kInW + tx + 3;
        const bool hit = s_in[3 * kInW * kInH + ci] != 0.0f;
        const uint64_t pix = v.out_offset + (uint64_t)y * W + x;
        float *o = p.out + pix * p.C;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) o[ch] = hit ? s_in[ch * kInW * kInH + ci] + acc[ch] : 0.0f;
        if (p.C == 4) o[3] = __ldg(p.in + pix * 4 + 3);
    }
}

// The views' tile counts and prefix sums for the 14x30 output tiles (at most
// 32 views of at most 65536 x 65536 pixels: fewer than 2^31 tiles).
cudaError_t launch_post_filter(const PostParams &p0, cudaStream_t st)
{
    static thread_local PostParams p;
    p = p0;
    uint64_t tiles = 0;
    for (uint32_t v = 0; v < p.n_views; ++v) {
        p.views[v].tiles_x = (p.views[v].width + kPW - 1) / kPW;
        p.views[v].tiles_y = (p.views[v].height + kPHt - 1) / kPHt;
        p.tile_prefix[v] = (uint32_t)tiles;
        tiles += (uint64_t)p.views[v].tiles_x * p.views[v].tiles_y;
    }
    p.tile_prefix[p.n_views] = (uint32_t)tiles;
    if (tiles == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(post_filter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kPostSmem);
    if (e != cudaSuccess) return e;
    post_filter_kernel<<<(unsigned)tiles, 256, kPostSmem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace lfk
