// lf_precompute.cu -- the light-field precompute of Section 2: every ray
// r_k = (O + R p^o_i) + t d_ij of the two SF point sets, with its origin
// jittered on the disk of area A_S / M tangent to S, traced through an
// analytic emission-absorption volume of Gaussian blobs; L^(i,j) is the mean
// over the jittered samples.
//
// One thread per texel, FP32. Per sample the blobs are re-expressed along the
// ray: with f_b = o - mu_b and a_b^2 = log2(e) / (2 s_b^2), the density of blob
// b at step k (t_k = (k + 1/2) dt) is
//   exp2(la_b - y_k^2),  la_b = log2(kappa_b) - a_b^2 |f_b x d|^2,
//                        y_k  = a_b (f_b . d + 1/2 dt) + k (a_b dt),
// two fma and one ex2 per blob-step (with blobs taken in pairs: one packed
// fma, mul and sub per pair and two ex2). The cross product keeps the distance of
// the ray from a narrow blob's centre accurate (|f|^2 - (f.d)^2 would cancel).
// The emission is accumulated per blob, G_b += w_k g_bk with w_k the step's
// compositing weight, and turned into colour once per sample: sum_b G_b emit_b
// (the same sum as sum_k w_k sum_b g_bk emit_b, one fma per blob-step instead
// of three).
#include <cuda_runtime.h>
#include <math.h>

#include "lf_device.cuh"
#include "lf_kernels.h"

namespace lfk {

constexpr float kLog2e = 1.4426950408889634f;

// 2^x by the hardware approximation (relative error below 2^-22; results
// below 2^-126 flush to zero, far below any contribution that matters here).
__device__ __forceinline__ float ex2_approx(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Packed FP32 pairs (one instruction for two blobs).
__device__ __forceinline__ unsigned long long pk(float2 a) { return *reinterpret_cast<unsigned long long *>(&a); }
__device__ __forceinline__ float2 upk(unsigned long long r) { return *reinterpret_cast<float2 *>(&r); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)), "l"(pk(c)));
    return upk(d);
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b)
{
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
    return upk(d);
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
    return upk(d);
}
__device__ __forceinline__ float2 add2(float2 a, float2 b)
{
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
    return upk(d);
}

// (1 - exp(-x)) / x for x >= 0, given E = exp(-x): the Taylor series of the
// left side below x = 1/16 (truncation < x^5/720 < 2^-29 relative), the
// quotient above (cancellation in 1 - E costs at most 16 ulp there). Both are
// evaluated and one selected, so that a warp does not diverge.
__device__ __forceinline__ float one_minus_exp_over_x(float x, float E)
{
    const float series = fmaf(x, fmaf(x, fmaf(x, fmaf(x, 1.0f / 120.0f, -1.0f / 24.0f), 1.0f / 6.0f), -0.5f), 1.0f);
    const float quot = __fdividef(1.0f - E, x);
    return x < 0.0625f ? series : quot;
}

// CTAs of 256 threads per SM the register budget of the 8-blob kernel is cut
// for, and the unroll of the step loop (measured with the packed blob loop:
// 2 CTAs and 2 steps were fastest).
#ifndef LF_PRE_MIN_BLOCKS
#define LF_PRE_MIN_BLOCKS 2
#endif

// 1: the blob loop in packed FP32 pairs (fma/mul/sub/add .f32x2); 0: scalar.
#ifndef LF_PRE_PACKED
#define LF_PRE_PACKED 1
#endif
#ifndef LF_PRE_STEP_UNROLL
#define LF_PRE_STEP_UNROLL 2
#endif
constexpr int kPreStepUnroll = LF_PRE_STEP_UNROLL;

// Radiance collected along o + t d, t in [0, t_end], by the midpoint rule with
// p.steps steps of constant density and emission (see the top of the file):
// (RGB including the background seen through the final transmittance T, and
// 1 - T).
template <int BMAX>
__device__ __forceinline__ float4 march(const PrecomputeParams &p, float ox, float oy, float oz, float dx,
                                        float dy, float dz, float t_end)
{
    const float dt = t_end / (float)p.steps;
    // per-blob constants of this ray
    float y0[BMAX], dy0[BMAX], la[BMAX], G[BMAX];
#pragma unroll
    for (int k = 0; k < BMAX; ++k) {
        const float4 bp = p.blob_pos[k];
        const float a = p.blob_col[k].w;
        const float fx = ox - bp.x, fy = oy - bp.y, fz = oz - bp.z;
        const float along = fmaf(fx, dx, fmaf(fy, dy, fz * dz));
        const float cx = fy * dz - fz * dy, cy = fz * dx - fx * dz, cz = fx * dy - fy * dx;
        const float perp = fmaf(cx, cx, fmaf(cy, cy, cz * cz));
        y0[k] = a * fmaf(0.5f, dt, along);
        dy0[k] = a * dt;
        la[k] = (k < (int)p.nb) ? fmaf(-a * a, perp, bp.w) : -INFINITY;
        G[k] = 0.0f;
    }

    float T = 1.0f;
    if (dt > 0.0f) {
        // dt folded into the densities: g' = g dt = 2^(la + log2 dt - y^2), so the
        // step's optical depth is sum g' and its weight T (1 - e^-x) / x
        const float l2dt = __log2f(dt);
#pragma unroll
        for (int k = 0; k < BMAX; ++k) la[k] += l2dt;
#if LF_PRE_PACKED
        // blobs in pairs: y, y^2, the exponent, the density sum and the
        // per-blob weights in packed FP32 pairs
        constexpr int BP = BMAX / 2;
        float2 Y0[BP], DY[BP], LA[BP], G2[BP];
#pragma unroll
        for (int q = 0; q < BP; ++q) {
            Y0[q] = make_float2(y0[2 * q], y0[2 * q + 1]);
            DY[q] = make_float2(dy0[2 * q], dy0[2 * q + 1]);
            LA[q] = make_float2(la[2 * q], la[2 * q + 1]);
            G2[q] = make_float2(0.0f, 0.0f);
        }
        float kf = 0.0f;
#pragma unroll kPreStepUnroll
        for (uint32_t st = 0; st < p.steps; ++st, kf += 1.0f) {
            const float2 kf2 = make_float2(kf, kf);
            float2 g2[BP], sig2 = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int q = 0; q < BP; ++q) {
                const float2 y = fma2(kf2, DY[q], Y0[q]);
                const float2 arg = sub2(LA[q], mul2(y, y));
                g2[q] = make_float2(ex2_approx(arg.x), ex2_approx(arg.y));
                sig2 = add2(sig2, g2[q]);
            }
            // step of constant density: x = sigma dt, weight T (1 - e^-x) / x per g'
            const float xs = sig2.x + sig2.y;
            const float E = ex2_approx(-xs * kLog2e);
            const float w = T * one_minus_exp_over_x(xs, E);
            const float2 w2 = make_float2(w, w);
#pragma unroll
            for (int q = 0; q < BP; ++q) G2[q] = fma2(w2, g2[q], G2[q]);
            T *= E;
        }
#pragma unroll
        for (int q = 0; q < BP; ++q) {
            G[2 * q] = G2[q].x;
            G[2 * q + 1] = G2[q].y;
        }
#else
        float kf = 0.0f;
#pragma unroll kPreStepUnroll
        for (uint32_t st = 0; st < p.steps; ++st, kf += 1.0f) {
            float g[BMAX], sig = 0.0f;
#pragma unroll
            for (int k = 0; k < BMAX; ++k) {
                const float y = fmaf(kf, dy0[k], y0[k]);
                g[k] = ex2_approx(fmaf(-y, y, la[k]));
                sig += g[k];
            }
            // step of constant density: x = sigma dt, weight T (1 - e^-x) / x per g'
            const float xs = sig;
            const float E = ex2_approx(-xs * kLog2e);
            const float w = T * one_minus_exp_over_x(xs, E);
#pragma unroll
            for (int k = 0; k < BMAX; ++k) G[k] = fmaf(w, g[k], G[k]);
            T *= E;
        }
#endif
    }
    float L0 = 0.0f, L1 = 0.0f, L2 = 0.0f;
#pragma unroll
    for (int k = 0; k < BMAX; ++k) {
        const float4 bc = p.blob_col[k];
        L0 = fmaf(G[k], bc.x, L0);
        L1 = fmaf(G[k], bc.y, L1);
        L2 = fmaf(G[k], bc.z, L2);
    }
    const float bgw = 0.5f * (1.0f + dz);
    return make_float4(fmaf(T, fmaf(p.bg1[0], bgw, p.bg0[0]), L0), fmaf(T, fmaf(p.bg1[1], bgw, p.bg0[1]), L1),
                       fmaf(T, fmaf(p.bg1[2], bgw, p.bg0[2]), L2), 1.0f - T);
}

template <int BMAX>
__global__ void __launch_bounds__(256, BMAX <= 8 ? LF_PRE_MIN_BLOCKS : 1)
    precompute_kernel(const __grid_constant__ PrecomputeParams p)
{
    const uint64_t total = (uint64_t)p.rows * p.N;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
        const uint32_t i = (uint32_t)(t / p.N);
        const uint32_t j = (uint32_t)(t - (uint64_t)i * p.N);
        const float4 ph = __ldg(p.po_hi + i), pl = __ldg(p.po_lo + i);
        const float4 qh = __ldg(p.pd_hi + j), ql = __ldg(p.pd_lo + j);
        const float px = ph.x + pl.x, py = ph.y + pl.y, pz = ph.z + pl.z;

        // chord direction d_ij from the hi/lo parts (-p if the points coincide)
        float dx = (qh.x - ph.x) + (ql.x - pl.x);
        float dy = (qh.y - ph.y) + (ql.y - pl.y);
        float dz = (qh.z - ph.z) + (ql.z - pl.z);
        const float l2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        if (l2 < 1e-24f) {
            dx = -px; dy = -py; dz = -pz;
        } else {
            const float il = rsqrtf(l2);
            dx *= il; dy *= il; dz *= il;
        }

        // unit tangents of S at p along azimuth and polar angle
        const float rho2 = fmaf(px, px, py * py);
        const float irho = rsqrtf(rho2);
        const float ephx = -py * irho, ephy = px * irho;
        const float ethx = px * pz * irho, ethy = py * pz * irho, ethz = -rho2 * irho;
        const float pd = fmaf(px, dx, fmaf(py, dy, pz * dz));    // p . d

        float acc0 = 0.0f, acc1 = 0.0f, acc2 = 0.0f, acc3 = 0.0f;
        for (uint32_t s = 0; s < p.spp; ++s) {
            // origin o = O + R p + off, off in the tangent plane (|off| <= disk_r)
            float offx = 0.0f, offy = 0.0f, offz = 0.0f;
            if (p.jitter) {
                const uint64_t ctr = 2ull * (((uint64_t)i * p.N + j) * p.spp + s);
                const float u1 = (float)(uint32_t)(splitmix64(p.seed, ctr) >> 40) * 0x1p-24f;
                const float u2 = (float)(uint32_t)(splitmix64(p.seed, ctr + 1) >> 40) * 0x1p-24f;
                const float r = p.disk_r * sqrtf(u1);
                float sa, ca;
                sincospif(2.0f * u2, &sa, &ca);
                offx = r * fmaf(ca, ephx, sa * ethx);
                offy = r * fmaf(ca, ephy, sa * ethy);
                offz = r * (sa * ethz);
            }
            const float ox = fmaf(p.R, px, p.Ox) + offx;
            const float oy = fmaf(p.R, py, p.Oy) + offy;
            const float oz = fmaf(p.R, pz, p.Oz) + offz;

            // far end of the segment inside S: with f = o - O = R p + off and off . p = 0,
            // b = f . d and |f|^2 - R^2 = |off|^2
            const float b = fmaf(p.R, pd, fmaf(offx, dx, fmaf(offy, dy, offz * dz)));
            const float c = fmaf(offx, offx, fmaf(offy, offy, offz * offz));
            const float disc = fmaf(b, b, -c);
            const float t_end = disc > 0.0f ? fmaxf(0.0f, sqrtf(disc) - b) : 0.0f;

            const float4 r = march<BMAX>(p, ox, oy, oz, dx, dy, dz, t_end);
            acc0 += r.x;
            acc1 += r.y;
            acc2 += r.z;
            acc3 += r.w;
        }
        const float inv = 1.0f / (float)p.spp;
        if (p.C == 4) {
            reinterpret_cast<float4 *>(p.out)[t] = make_float4(acc0 * inv, acc1 * inv, acc2 * inv, acc3 * inv);
        } else {
            float *o = p.out + 3 * t;
            o[0] = acc0 * inv;
            o[1] = acc1 * inv;
            o[2] = acc2 * inv;
        }
    }
}

// Direct render of the same volume, one thread per pixel of one view: the
// pixel's camera ray and its front hit h_o on S (the FP32 steps of the
// light-field render), the far end of the ray inside S from h_o in FP64 (the
// FP32 form of |h_o - O|^2 - R^2 cancels for grazing rays), then the
// integral of the precompute along that ray (one sample, no jitter). Misses
// store 0.
template <int BMAX>
__global__ void __launch_bounds__(256, BMAX <= 8 ? LF_PRE_MIN_BLOCKS : 1)
    volume_direct_kernel(const __grid_constant__ PrecomputeParams p, const __grid_constant__ ViewK v,
                         const __grid_constant__ SphereK S, double R)
{
    const uint64_t total = (uint64_t)v.width * v.height;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
        const uint32_t y = (uint32_t)(t / v.width), x = (uint32_t)(t - (uint64_t)y * v.width);
        const float3 d = camera_dir(v, x, y);
        float3 ho, hd;
        float4 r = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (intersect_sphere(S, v.eye, d, ho, hd)) {
            const double f0 = __dsub_rn((double)ho.x, S.o64[0]);
            const double f1 = __dsub_rn((double)ho.y, S.o64[1]);
            const double f2 = __dsub_rn((double)ho.z, S.o64[2]);
            const double b = __dadd_rn(__dadd_rn(__dmul_rn(f0, (double)d.x), __dmul_rn(f1, (double)d.y)),
                                       __dmul_rn(f2, (double)d.z));
            const double c = __dsub_rn(__dadd_rn(__dadd_rn(__dmul_rn(f0, f0), __dmul_rn(f1, f1)), __dmul_rn(f2, f2)),
                                       __dmul_rn(R, R));
            const double disc = __dsub_rn(__dmul_rn(b, b), c);
            const double te = disc > 0.0 ? __dadd_rn(-b, __dsqrt_rn(disc)) : 0.0;
            r = march<BMAX>(p, ho.x, ho.y, ho.z, d.x, d.y, d.z, te > 0.0 ? (float)te : 0.0f);
        }
        const uint64_t pix = v.out_offset + t;
        if (p.C == 4) {
            reinterpret_cast<float4 *>(p.out)[pix] = r;
        } else {
            float *o = p.out + 3 * pix;
            o[0] = r.x;
            o[1] = r.y;
            o[2] = r.z;
        }
    }
}

cudaError_t launch_volume_direct(const PrecomputeParams &p, const ViewK &v, const SphereK &S, double R,
                                 cudaStream_t st)
{
    const uint64_t total = (uint64_t)v.width * v.height;
    const uint64_t blocks = (total + 255) / 256;
    const unsigned grid = (unsigned)(blocks < (1ull << 20) ? blocks : (1ull << 20));
    if (p.nb <= 8)
        volume_direct_kernel<8><<<grid, 256, 0, st>>>(p, v, S, R);
    else
        volume_direct_kernel<kMaxBlobs><<<grid, 256, 0, st>>>(p, v, S, R);
    return cudaGetLastError();
}

cudaError_t launch_precompute(const PrecomputeParams &p, cudaStream_t st)
{
    const uint64_t total = (uint64_t)p.rows * p.N;
    const uint64_t blocks = (total + 255) / 256;
    const unsigned grid = (unsigned)(blocks < (1ull << 20) ? blocks : (1ull << 20));
    if (p.nb <= 8)
        precompute_kernel<8><<<grid, 256, 0, st>>>(p);
    else
        precompute_kernel<kMaxBlobs><<<grid, 256, 0, st>>>(p);
    return cudaGetLastError();
}

}  // namespace lfk
