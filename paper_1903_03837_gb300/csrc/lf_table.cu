// lf_table.cu -- table-side kernels: the SF point caches, the per-row
// FP16/E4M3 quantiser, 3->4 channel padding of codes, and the synthetic lobe
// radiance field.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "lf_kernels.h"

namespace lfk {

// round(2^128 * (Phi - 1)) split into two 64-bit words: frac(i/Phi) =
// frac(i*(Phi-1)) is (i * G mod 2^128) / 2^128 up to i * 2^-129.
constexpr uint64_t kGoldHi = 0x9e3779b97f4a7c15ull;
constexpr uint64_t kGoldLo = 0xf39cc0605cedc834ull;
constexpr double kTwoPi = 6.283185307179586476925286766559;

// SF point p_i of a set of n points (Section 2, SF point set equation):
// phi_i = 2*pi*frac(i/Phi) (phase truncated to 53 bits), z_i = 1 - (2i+1)/n,
// p_i = (cos(phi_i) sin(theta_i), sin(phi_i) sin(theta_i), z_i) with
// sin(theta_i) = sqrt((1 - z_i)(1 + z_i)); FP64, stored as hi/lo floats.
__global__ void build_points_kernel(uint32_t n, float4 *hi, float4 *lo)
{
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t ii = i;
    uint64_t top = ii * kGoldHi + __umul64hi(ii, kGoldLo);
    double t = (double)(top >> 11) * 0x1p-53;
    double phi = __dmul_rn(kTwoPi, t);
    double z = __dsub_rn(1.0, __ddiv_rn((double)(2ull * ii + 1ull), (double)n));
    double s = __dsqrt_rn(__dmul_rn(__dsub_rn(1.0, z), __dadd_rn(1.0, z)));
    double sp, cp;
    sincos(phi, &sp, &cp);
    double p[3] = {__dmul_rn(cp, s), __dmul_rn(sp, s), z};
    float h[3], l[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        h[k] = __double2float_rn(p[k]);
        l[k] = __double2float_rn(__dsub_rn(p[k], (double)h[k]));
    }
    hi[i] = make_float4(h[0], h[1], h[2], 0.0f);
    lo[i] = make_float4(l[0], l[1], l[2], 0.0f);
}

cudaError_t launch_build_points(uint32_t n, float4 *hi, float4 *lo, cudaStream_t st)
{
    build_points_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, hi, lo);
    return cudaGetLastError();
}

// [M][N][3] codes -> [M][N][4] codes with channel 3 = 0.
template <typename T>
__global__ void pad_codes_kernel(const T *src, uint64_t texels, T *dst)
{
    uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= texels) return;
    dst[4 * t] = src[3 * t];
    dst[4 * t + 1] = src[3 * t + 1];
    dst[4 * t + 2] = src[3 * t + 2];
    dst[4 * t + 3] = T(0);
}

cudaError_t launch_pad_codes(const void *src, uint32_t M, uint32_t N, int bytes, void *dst, cudaStream_t st)
{
    uint64_t texels = (uint64_t)M * N;
    unsigned grid = (unsigned)((texels + 255) / 256);
    if (bytes == 2)
        pad_codes_kernel<<<grid, 256, 0, st>>>((const uint16_t *)src, texels, (uint16_t *)dst);
    else
        pad_codes_kernel<<<grid, 256, 0, st>>>((const uint8_t *)src, texels, (uint8_t *)dst);
    return cudaGetLastError();
}

// Per-row quantisation: one CTA per origin row. amax over the row's N*C
// values; scale = amax (F16) or amax/448 (E4M3), 1 if amax = 0; codes of
// RNE(x / scale) (E4M3 saturating to +-448), 4 channels per texel.
__device__ __forceinline__ uint16_t e4m3x2(float a_hi, float b_lo)
{
    uint16_t r;
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(r) : "f"(a_hi), "f"(b_lo));
    return r;
}

template <int DTYPE>
__global__ void quantize_rows_kernel(const float *src, uint32_t N, uint32_t C, void *codes, float *scales)
{
    __shared__ float red[32];
    const uint32_t i = blockIdx.x;
    const size_t rowlen = (size_t)N * C;
    const float *r = src + (size_t)i * rowlen;
    float amax = 0.0f;
    for (size_t k = threadIdx.x; k < rowlen; k += blockDim.x) amax = fmaxf(amax, fabsf(r[k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = amax;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0) red[0] = v;
    }
    __syncthreads();
    amax = red[0];
    const float s = amax == 0.0f ? 1.0f : (DTYPE == LF_DTYPE_E4M3 ? __fdiv_rn(amax, 448.0f) : amax);
    if (threadIdx.x == 0) scales[i] = s;
    for (uint32_t j = threadIdx.x; j < N; j += blockDim.x) {
        float x[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) x[c] = (uint32_t)c < C ? __fdiv_rn(r[(size_t)j * C + c], s) : 0.0f;
        size_t t = (size_t)i * N + j;
        if (DTYPE == LF_DTYPE_E4M3) {
            uint32_t v = (uint32_t)e4m3x2(x[1], x[0]) | ((uint32_t)e4m3x2(x[3], x[2]) << 16);
            reinterpret_cast<uint32_t *>(codes)[t] = v;
        } else {
            __half2 a = __floats2half2_rn(x[0], x[1]), b = __floats2half2_rn(x[2], x[3]);
            uint2 v = make_uint2(*reinterpret_cast<uint32_t *>(&a), *reinterpret_cast<uint32_t *>(&b));
            reinterpret_cast<uint2 *>(codes)[t] = v;
        }
    }
}

cudaError_t launch_quantize(const float *src, uint32_t M, uint32_t N, uint32_t C, int dtype, void *codes,
                            float *scales, cudaStream_t st)
{
    if (dtype == LF_DTYPE_E4M3)
        quantize_rows_kernel<LF_DTYPE_E4M3><<<M, 256, 0, st>>>(src, N, C, codes, scales);
    else
        quantize_rows_kernel<LF_DTYPE_F16><<<M, 256, 0, st>>>(src, N, C, codes, scales);
    return cudaGetLastError();
}

__device__ __forceinline__ double dot3(const double a[3], const double b[3])
{
    return __dadd_rn(__dadd_rn(__dmul_rn(a[0], b[0]), __dmul_rn(a[1], b[1])), __dmul_rn(a[2], b[2]));
}

// Lobe field, one thread per texel (i, j); a CTA covers 256 columns of one row
// and shares that row's position factors. FP64, rounded once to FP32.
__global__ void fill_lobe_kernel(const __grid_constant__ LobeParams P, const float4 *po_hi,
                                 const float4 *po_lo, const float4 *pd_hi, const float4 *pd_lo,
                                 uint32_t N, uint32_t blocks_per_row, float *out)
{
    __shared__ double s_ep[kMaxLobes];
    const uint32_t i = blockIdx.x / blocks_per_row;
    const uint32_t j = (blockIdx.x % blocks_per_row) * blockDim.x + threadIdx.x;
    float4 a = po_hi[i], b = po_lo[i];
    const double po[3] = {__dadd_rn((double)a.x, (double)b.x), __dadd_rn((double)a.y, (double)b.y),
                          __dadd_rn((double)a.z, (double)b.z)};
    if (threadIdx.x < P.L) {
        double cp = dot3(po, P.ap[threadIdx.x]);
        s_ep[threadIdx.x] = exp(__dmul_rn(P.kp[threadIdx.x], __dsub_rn(cp, 1.0)));
    }
    __syncthreads();
    if (j >= N) return;
    float4 c = pd_hi[j], e = pd_lo[j];
    double d[3] = {__dsub_rn(__dadd_rn((double)c.x, (double)e.x), po[0]),
                   __dsub_rn(__dadd_rn((double)c.y, (double)e.y), po[1]),
                   __dsub_rn(__dadd_rn((double)c.z, (double)e.z), po[2])};
    double l = __dsqrt_rn(dot3(d, d));
    if (l < 1e-12) {
        d[0] = -po[0]; d[1] = -po[1]; d[2] = -po[2];
    } else {
        d[0] = __ddiv_rn(d[0], l); d[1] = __ddiv_rn(d[1], l); d[2] = __ddiv_rn(d[2], l);
    }
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (uint32_t k = 0; k < P.L; ++k) {
        double cd = dot3(d, P.ad[k]);
        double g = __dmul_rn(s_ep[k], exp(__dmul_rn(P.kd[k], __dsub_rn(cd, 1.0))));
        for (uint32_t ch = 0; ch < P.C; ++ch) acc[ch] = __dadd_rn(acc[ch], __dmul_rn(P.col[k][ch], g));
    }
    float *o = out + ((size_t)i * N + j) * P.C;
    for (uint32_t ch = 0; ch < P.C; ++ch) {
        uint64_t ctr = ((uint64_t)i << 32) | ((uint64_t)j << 4) | ch;
        double u = (double)(splitmix64(P.seed, ctr) >> 11) * 0x1p-53;
        o[ch] = __double2float_rn(__dadd_rn(acc[ch], __dmul_rn(0.01, u)));
    }
}

cudaError_t launch_fill_lobe(const LobeParams &P, const float4 *po_hi, const float4 *po_lo,
                             const float4 *pd_hi, const float4 *pd_lo, uint32_t M, uint32_t N,
                             float *out, cudaStream_t st)
{
    uint32_t bpr = (N + 255) / 256;
    fill_lobe_kernel<<<(unsigned)((uint64_t)M * bpr), 256, 0, st>>>(P, po_hi, po_lo, pd_hi, pd_lo, N, bpr, out);
    return cudaGetLastError();
}

}  // namespace lfk
