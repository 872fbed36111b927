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
// One CTA of 256 threads per 14x14 output tile of one view (the tiles of all
// views of a launch numbered consecutively), FP32 on the CUDA cores: the 20x20
// input tile with its mask, the 18x18 first-layer and the 16x16 second-layer
// activations live in shared memory (43.5 KB); the second layer, 86% of the
// multiply-adds, is exactly one output position per thread. The weights are
// part of the kernel's parameter block and every loop over them is unrolled,
// so each multiply-add takes its weight as a constant-bank operand: one
// instruction per multiply-add, and the activations are read from shared
// memory once per tap for all 16 (or 3) output channels. The layers are 16
// channels wide: too narrow to fill a tensor-core tile.
#include <cuda_runtime.h>

#include "lf_device.cuh"
#include "lf_kernels.h"

namespace lfk {

constexpr int kPT = kPostTile;          // 14: output tile side
constexpr int kPH2 = kPT + 2;           // 16: second-layer activations
constexpr int kPH1 = kPT + 4;           // 18: first-layer activations
constexpr int kPIn = kPT + 6;           // 20: input tile (3 layers of radius 1)

__global__ void __launch_bounds__(256) post_filter_kernel(const __grid_constant__ PostParams p)
{
    __shared__ float s_in[4 * kPIn * kPIn];              // R, G, B, hit mask
    __shared__ float s_h1[kPostHidden * kPH1 * kPH1];
    __shared__ float s_h2[kPostHidden * kPH2 * kPH2];
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
    __syncthreads();
    const ViewK &v = p.views[s_tile[0]];
    const int x0 = (int)s_tile[1] * kPT, y0 = (int)s_tile[2] * kPT;
    const int W = (int)v.width, H = (int)v.height;

    for (int k = tid; k < kPIn * kPIn; k += blockDim.x) {
        const int ty = k / kPIn, tx = k - ty * kPIn;
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
        s_in[kPIn * kPIn + k] = g;
        s_in[2 * kPIn * kPIn + k] = b;
        s_in[3 * kPIn * kPIn + k] = m;
    }
    __syncthreads();

    // layer 1: 4 -> 16 channels on the 18x18 tile
    for (int k = tid; k < kPH1 * kPH1; k += blockDim.x) {
        const int ty = k / kPH1, tx = k - ty * kPH1;
        const int x = x0 - 2 + tx, y = y0 - 2 + ty;
        const bool inside = x >= 0 && y >= 0 && x < W && y < H;
        float acc[kPostHidden];
#pragma unroll
        for (int o = 0; o < kPostHidden; ++o) acc[o] = p.w[kPostB1 + o];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float in[9];
#pragma unroll
            for (int t = 0; t < 9; ++t) in[t] = s_in[i * kPIn * kPIn + (ty + t / 3) * kPIn + tx + t % 3];
#pragma unroll
            for (int o = 0; o < kPostHidden; ++o)
#pragma unroll
                for (int t = 0; t < 9; ++t) acc[o] = fmaf(p.w[kPostW1 + (o * 4 + i) * 9 + t], in[t], acc[o]);
        }
#pragma unroll
        for (int o = 0; o < kPostHidden; ++o) s_h1[o * kPH1 * kPH1 + k] = inside ? fmaxf(acc[o], 0.0f) : 0.0f;
    }
    __syncthreads();

    // layer 2: 16 -> 16 channels on the 16x16 tile, one position per thread
    {
        const int ty = tid / kPH2, tx = tid - ty * kPH2;
        const int x = x0 - 1 + tx, y = y0 - 1 + ty;
        const bool inside = x >= 0 && y >= 0 && x < W && y < H;
        float acc[kPostHidden];
#pragma unroll
        for (int o = 0; o < kPostHidden; ++o) acc[o] = p.w[kPostB2 + o];
#pragma unroll
        for (int i = 0; i < kPostHidden; ++i) {
            float in[9];
#pragma unroll
            for (int t = 0; t < 9; ++t) in[t] = s_h1[i * kPH1 * kPH1 + (ty + t / 3) * kPH1 + tx + t % 3];
#pragma unroll
            for (int o = 0; o < kPostHidden; ++o)
#pragma unroll
                for (int t = 0; t < 9; ++t)
                    acc[o] = fmaf(p.w[kPostW2 + (o * kPostHidden + i) * 9 + t], in[t], acc[o]);
        }
#pragma unroll
        for (int o = 0; o < kPostHidden; ++o) s_h2[o * kPH2 * kPH2 + tid] = inside ? fmaxf(acc[o], 0.0f) : 0.0f;
    }
    __syncthreads();

    // layer 3: 16 -> 3 channels, added to the input colour of hit pixels
    if (tid < kPT * kPT) {
        const int ty = tid / kPT, tx = tid - ty * kPT;
        const int x = x0 + tx, y = y0 + ty;
        if (x < W && y < H) {
            float acc[3] = {p.w[kPostB3], p.w[kPostB3 + 1], p.w[kPostB3 + 2]};
#pragma unroll
            for (int i = 0; i < kPostHidden; ++i) {
                float in[9];
#pragma unroll
                for (int t = 0; t < 9; ++t) in[t] = s_h2[i * kPH2 * kPH2 + (ty + t / 3) * kPH2 + tx + t % 3];
#pragma unroll
                for (int o = 0; o < 3; ++o)
#pragma unroll
                    for (int t = 0; t < 9; ++t)
                        acc[o] = fmaf(p.w[kPostW3 + (o * kPostHidden + i) * 9 + t], in[t], acc[o]);
            }
            const int c = (ty + 3) * kPIn + tx + 3;
            const bool hit = s_in[3 * kPIn * kPIn + c] != 0.0f;
            const uint64_t pix = v.out_offset + (uint64_t)y * W + x;
            float *o = p.out + pix * p.C;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) o[ch] = hit ? s_in[ch * kPIn * kPIn + c] + acc[ch] : 0.0f;
            if (p.C == 4) o[3] = __ldg(p.in + pix * 4 + 3);
        }
    }
}

cudaError_t launch_post_filter(const PostParams &p, unsigned tiles, cudaStream_t st)
{
    post_filter_kernel<<<tiles, 256, 0, st>>>(p);
    return cudaGetLastError();
}

}  // namespace lfk
