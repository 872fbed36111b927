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
// One CTA per 16x16 output tile of one view, FP32 on the CUDA cores: the
// 22x22 input tile (with its mask), the 20x20 first-layer and the 18x18
// second-layer activations and the 3,347 weights live in shared memory (66 KB),
// so each layer reads the previous one from shared memory once per tap. The
// layers are 16 channels wide: too narrow to fill a tensor-core tile.
#include <cuda_runtime.h>

#include "lf_device.cuh"
#include "lf_kernels.h"

namespace lfk {

constexpr int kPT = 16;                 // output tile side
constexpr int kPIn = kPT + 6;           // input tile side (3 layers of radius 1)
constexpr int kPH1 = kPT + 4;           // first-layer activations
constexpr int kPH2 = kPT + 2;           // second-layer activations
constexpr int kPostWeightsPad = (kPostWeights + 3) & ~3;
constexpr size_t kPostSmem =
    sizeof(float) * (kPostWeightsPad + 4 * kPIn * kPIn + kPostHidden * kPH1 * kPH1 + kPostHidden * kPH2 * kPH2);

__global__ void __launch_bounds__(256) post_filter_kernel(const __grid_constant__ PostParams p,
                                                          const __grid_constant__ ViewK v)
{
    extern __shared__ float sm[];
    float *s_w = sm;
    float *s_in = s_w + kPostWeightsPad;                 // [4][kPIn][kPIn]: R, G, B, hit mask
    float *s_h1 = s_in + 4 * kPIn * kPIn;                // [16][kPH1][kPH1]
    float *s_h2 = s_h1 + kPostHidden * kPH1 * kPH1;      // [16][kPH2][kPH2]
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * kPT, y0 = blockIdx.y * kPT;
    const int W = (int)v.width, H = (int)v.height;

    for (int k = tid; k < kPostWeights; k += blockDim.x) s_w[k] = __ldg(p.w + k);
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

    // layer 1: 4 -> 16 channels on the 20x20 ring-extended tile
    for (int k = tid; k < kPH1 * kPH1; k += blockDim.x) {
        const int ty = k / kPH1, tx = k - ty * kPH1;
        const int x = x0 - 2 + tx, y = y0 - 2 + ty;
        const bool inside = x >= 0 && y >= 0 && x < W && y < H;
        float in[36];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int t = 0; t < 9; ++t) in[i * 9 + t] = s_in[i * kPIn * kPIn + (ty + t / 3) * kPIn + tx + t % 3];
#pragma unroll 4
        for (int o = 0; o < kPostHidden; ++o) {
            float acc = s_w[kPostB1 + o];
#pragma unroll
            for (int j = 0; j < 36; ++j) acc = fmaf(s_w[kPostW1 + o * 36 + j], in[j], acc);
            s_h1[o * kPH1 * kPH1 + k] = inside ? fmaxf(acc, 0.0f) : 0.0f;
        }
    }
    __syncthreads();

    // layer 2: 16 -> 16 channels on the 18x18 tile
    for (int k = tid; k < kPH2 * kPH2; k += blockDim.x) {
        const int ty = k / kPH2, tx = k - ty * kPH2;
        const int x = x0 - 1 + tx, y = y0 - 1 + ty;
        const bool inside = x >= 0 && y >= 0 && x < W && y < H;
        float acc[kPostHidden];
#pragma unroll
        for (int o = 0; o < kPostHidden; ++o) acc[o] = s_w[kPostB2 + o];
        for (int i = 0; i < kPostHidden; ++i) {
            float in[9];
#pragma unroll
            for (int t = 0; t < 9; ++t) in[t] = s_h1[i * kPH1 * kPH1 + (ty + t / 3) * kPH1 + tx + t % 3];
#pragma unroll
            for (int o = 0; o < kPostHidden; ++o)
#pragma unroll
                for (int t = 0; t < 9; ++t) acc[o] = fmaf(s_w[kPostW2 + (o * kPostHidden + i) * 9 + t], in[t], acc[o]);
        }
#pragma unroll
        for (int o = 0; o < kPostHidden; ++o) s_h2[o * kPH2 * kPH2 + k] = inside ? fmaxf(acc[o], 0.0f) : 0.0f;
    }
    __syncthreads();

    // layer 3: 16 -> 3 channels, added to the input colour of hit pixels
    for (int k = tid; k < kPT * kPT; k += blockDim.x) {
        const int ty = k / kPT, tx = k - ty * kPT;
        const int x = x0 + tx, y = y0 + ty;
        if (x >= W || y >= H) continue;
        float acc[3] = {s_w[kPostB3], s_w[kPostB3 + 1], s_w[kPostB3 + 2]};
        for (int i = 0; i < kPostHidden; ++i) {
            float in[9];
#pragma unroll
            for (int t = 0; t < 9; ++t) in[t] = s_h2[i * kPH2 * kPH2 + (ty + t / 3) * kPH2 + tx + t % 3];
#pragma unroll
            for (int o = 0; o < 3; ++o)
#pragma unroll
                for (int t = 0; t < 9; ++t) acc[o] = fmaf(s_w[kPostW3 + (o * kPostHidden + i) * 9 + t], in[t], acc[o]);
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

cudaError_t launch_post_filter(const PostParams &p, const ViewK &v, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(post_filter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kPostSmem);
    if (e != cudaSuccess) return e;
    const dim3 grid((v.width + kPT - 1) / kPT, (v.height + kPT - 1) / kPT);
    post_filter_kernel<<<grid, 256, kPostSmem, st>>>(p, v);
    return cudaGetLastError();
}

}  // namespace lfk
