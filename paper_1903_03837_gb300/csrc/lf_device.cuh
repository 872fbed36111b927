// lf_device.cuh -- device-side steps of the light-field sampling path
// (LumiPath, arXiv 1903.03837, Section 2), written for sm_103a.
//
// Per ray: pinhole ray (fixed FP32 operation order), ray/sphere hits, unit hit
// vectors in double-float, the 5 nearest SF points of each hit through the
// inverse SF lattice, tent weights of the distance filter kernel, and the
// texel decoders of the three storage types.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lf_internal.h"

namespace lfk {

// ---------------------------------------------------------------------------
// Fibonacci numbers and the signed lattice offsets eps_k = F_k/Phi - F_{k-1}
// = (-1)^(k+1) Phi^-k (Binet). The lattice of SF points in (turns, index)
// coordinates has basis (eps_k, F_k), (eps_{k+1}, F_{k+1}).
// ---------------------------------------------------------------------------
constexpr int kFibN = 40;
struct FibTables {
    int32_t F[kFibN];
    float eps[kFibN];
};
constexpr FibTables make_fib() {
    FibTables t{};
    long long a = 0, b = 1;
    double g = 0.61803398874989484820, gk = 1.0;
    for (int k = 0; k < kFibN; ++k) {
        t.F[k] = (int32_t)a;
        long long c = a + b;
        a = b;
        b = c;
        t.eps[k] = (float)((k % 2 == 1) ? gk : -gk);   // (-1)^(k+1) g^k
        gk *= g;
    }
    return t;
}
__constant__ constexpr FibTables kFib = make_fib();

// log2(Phi^2), used by the zone number k = floor(log_{Phi^2}(sqrt5*pi*n*(1-z^2))).
constexpr float kInvLog2Phi2 = 0.72021234840458929f;    // 1 / log2(Phi^2)
constexpr float kSqrt5Pi = 7.0248147310407731f;          // sqrt(5)*pi
constexpr float kInv2Pi = 0.15915494309189535f;

// Certification margins of the FP32 ranking (see knn5): relative gap needed
// between consecutive keys for the order to be exact, by slot-bit count.
__device__ __forceinline__ float tau_for_bits(int bits) { return __int_as_float((127 + bits - 21) << 23); }
constexpr float kTauAbs = 3.637978807091713e-12f;      // 2^-38

// ---------------------------------------------------------------------------
// Camera ray and sphere intersection: IEEE FP32, fixed order, no contraction.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float3 camera_dir(const ViewK &v, uint32_t x, uint32_t y)
{
    float px = __fadd_rn(__uint2float_rn(x), 0.5f);
    float py = __fadd_rn(__uint2float_rn(y), 0.5f);
    float sx = __fdiv_rn(__fadd_rn(px, px), __uint2float_rn(v.width));
    float sy = __fdiv_rn(__fadd_rn(py, py), __uint2float_rn(v.height));
    float nx = __fmul_rn(__fsub_rn(sx, 1.0f), v.tan_x);
    float ny = __fmul_rn(__fsub_rn(1.0f, sy), v.tan_y);
    float vx = __fadd_rn(__fadd_rn(v.fwd[0], __fmul_rn(nx, v.right[0])), __fmul_rn(ny, v.up[0]));
    float vy = __fadd_rn(__fadd_rn(v.fwd[1], __fmul_rn(nx, v.right[1])), __fmul_rn(ny, v.up[1]));
    float vz = __fadd_rn(__fadd_rn(v.fwd[2], __fmul_rn(nx, v.right[2])), __fmul_rn(ny, v.up[2]));
    float l2 = __fadd_rn(__fadd_rn(__fmul_rn(vx, vx), __fmul_rn(vy, vy)), __fmul_rn(vz, vz));
    float l = __fsqrt_rn(l2);
    return make_float3(__fdiv_rn(vx, l), __fdiv_rn(vy, l), __fdiv_rn(vz, l));
}

// Front hit h_o and back hit h_d; false if the discriminant is <= 0 (tangential
// rays are discarded) or the front hit lies behind the eye.
__device__ __forceinline__ bool intersect_sphere(const SphereK &S, const float e[3], float3 d,
                                                 float3 &ho, float3 &hd)
{
    float fx = __fsub_rn(e[0], S.o32[0]);
    float fy = __fsub_rn(e[1], S.o32[1]);
    float fz = __fsub_rn(e[2], S.o32[2]);
    float b = __fadd_rn(__fadd_rn(__fmul_rn(fx, d.x), __fmul_rn(fy, d.y)), __fmul_rn(fz, d.z));
    float c = __fsub_rn(__fadd_rn(__fadd_rn(__fmul_rn(fx, fx), __fmul_rn(fy, fy)), __fmul_rn(fz, fz)),
                        __fmul_rn(S.r32, S.r32));
    float disc = __fsub_rn(__fmul_rn(b, b), c);
    if (!(disc > 0.0f)) return false;
    float sq = __fsqrt_rn(disc);
    float tn = __fsub_rn(-b, sq), tf = __fadd_rn(-b, sq);
    if (!(tn > 0.0f)) return false;
    ho = make_float3(__fadd_rn(e[0], __fmul_rn(tn, d.x)), __fadd_rn(e[1], __fmul_rn(tn, d.y)),
                     __fadd_rn(e[2], __fmul_rn(tn, d.z)));
    hd = make_float3(__fadd_rn(e[0], __fmul_rn(tf, d.x)), __fadd_rn(e[1], __fmul_rn(tf, d.y)),
                     __fadd_rn(e[2], __fmul_rn(tf, d.z)));
    return true;
}

// ---------------------------------------------------------------------------
// Double-float arithmetic (value = hi + lo, about 48 significant bits).
// ---------------------------------------------------------------------------
struct df { float h, l; };
__device__ __forceinline__ df two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ df fast_two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df df_add(df x, df y)
{
    df s = two_sum(x.h, y.h);
    return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(x.l, y.l)));
}
__device__ __forceinline__ df df_mul(df x, df y)
{
    float p = __fmul_rn(x.h, y.h);
    float e = __fmaf_rn(x.h, y.h, -p);
    e = __fmaf_rn(x.h, y.l, __fmaf_rn(x.l, y.h, e));
    return fast_two_sum(p, e);
}

// Unit vector (h - O)/|h - O| as hi/lo float3 pairs; |error| about 2^-44.
__device__ __forceinline__ void unit_hit_df(const SphereK &S, float3 h, float3 &qh, float3 &ql)
{
    df f[3];
    const float hv[3] = {h.x, h.y, h.z};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        df s = two_sum(hv[k], -S.o_hi[k]);
        f[k] = fast_two_sum(s.h, __fsub_rn(s.l, S.o_lo[k]));
    }
    df r2 = df_add(df_add(df_mul(f[0], f[0]), df_mul(f[1], f[1])), df_mul(f[2], f[2]));
    float y0 = rsqrtf(r2.h);
    df t = df_mul(r2, df{__fmul_rn(y0, y0), __fmaf_rn(y0, y0, -__fmul_rn(y0, y0))});
    float e = __fsub_rn(__fsub_rn(1.0f, t.h), t.l);
    df y = fast_two_sum(y0, __fmul_rn(__fmul_rn(0.5f, y0), e));
    df q0 = df_mul(f[0], y), q1 = df_mul(f[1], y), q2 = df_mul(f[2], y);
    qh = make_float3(q0.h, q1.h, q2.h);
    ql = make_float3(q0.l, q1.l, q2.l);
}

// FP64 unit hit vector in the operation order of the FP64 definition.
__device__ __forceinline__ void unit_hit_fp64(const SphereK &S, float3 h, double q[3])
{
    double f0 = __dsub_rn((double)h.x, S.o64[0]);
    double f1 = __dsub_rn((double)h.y, S.o64[1]);
    double f2 = __dsub_rn((double)h.z, S.o64[2]);
    double l = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(f0, f0), __dmul_rn(f1, f1)), __dmul_rn(f2, f2)));
    q[0] = __ddiv_rn(f0, l);
    q[1] = __ddiv_rn(f1, l);
    q[2] = __ddiv_rn(f2, l);
}

// Squared chord distance to SF point i from the hi/lo point cache (FP32
// result, relative error <= 2^-21 plus 2^-42 |d|).
__device__ __forceinline__ float dist2_df(const PointSetK &P, int32_t i, float3 qh, float3 ql)
{
    float4 a = __ldg(P.hi + i);
    float4 b = __ldg(P.lo + i);
    float dx = __fadd_rn(__fsub_rn(qh.x, a.x), __fsub_rn(ql.x, b.x));
    float dy = __fadd_rn(__fsub_rn(qh.y, a.y), __fsub_rn(ql.y, b.y));
    float dz = __fadd_rn(__fsub_rn(qh.z, a.z), __fsub_rn(ql.z, b.z));
    return __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmul_rn(dz, dz)));
}

__device__ __forceinline__ double dist2_fp64(const PointSetK &P, int32_t i, const double q[3])
{
    float4 a = __ldg(P.hi + i);
    float4 b = __ldg(P.lo + i);
    double p0 = __dadd_rn((double)a.x, (double)b.x);
    double p1 = __dadd_rn((double)a.y, (double)b.y);
    double p2 = __dadd_rn((double)a.z, (double)b.z);
    double u = __dsub_rn(q[0], p0), v = __dsub_rn(q[1], p1), w = __dsub_rn(q[2], p2);
    return __dadd_rn(__dadd_rn(__dmul_rn(u, u), __dmul_rn(v, v)), __dmul_rn(w, w));
}

// ---------------------------------------------------------------------------
// Inverse SF mapping, extended to the 5 nearest points (Section 2).
//
// Candidate sources:
//   FULL   n <= 128: every point (slot = index, 7 slot bits).
//   POLE   the continuous index (n(1-z)-1)/2 of the hit lies within 16 of a
//          pole: the 64 points nearest that pole (slot = offset, 6 bits).
//   WINDOW otherwise: the 4x4 lattice cells around floor(u, v), where (u, v)
//          are the hit's coordinates in the local Fibonacci basis of zone k
//          (slot = 4*(du+1) + (dv+1), 4 bits).
// Each candidate's squared distance becomes a 32-bit key (float bits with the
// low slot bits replaced by the slot); the 6 smallest keys are kept sorted.
// The FP32 order is accepted when every consecutive gap among those 6 exceeds
// the combined rounding and packing error; otherwise the same candidates are
// ranked again in FP64 by (distance, index).
// ---------------------------------------------------------------------------
#define LF_CS(a, b)                          \
    {                                        \
        uint32_t lo_ = min(k[a], k[b]);      \
        k[b] = max(k[a], k[b]);              \
        k[a] = lo_;                          \
    }

__device__ __forceinline__ void select6_of16(uint32_t k[16])
{
    // Batcher odd-even merge sort of 16 keys, pruned to the comparators that
    // reach outputs 0..5 (54 comparators).
    LF_CS(0, 1) LF_CS(2, 3) LF_CS(0, 2) LF_CS(1, 3) LF_CS(1, 2) LF_CS(4, 5) LF_CS(6, 7)
    LF_CS(4, 6) LF_CS(5, 7) LF_CS(5, 6) LF_CS(0, 4) LF_CS(2, 6) LF_CS(2, 4) LF_CS(1, 5)
    LF_CS(3, 7) LF_CS(3, 5) LF_CS(1, 2) LF_CS(3, 4) LF_CS(5, 6) LF_CS(8, 9) LF_CS(10, 11)
    LF_CS(8, 10) LF_CS(9, 11) LF_CS(9, 10) LF_CS(12, 13) LF_CS(14, 15) LF_CS(12, 14)
    LF_CS(13, 15) LF_CS(13, 14) LF_CS(8, 12) LF_CS(10, 14) LF_CS(10, 12) LF_CS(9, 13)
    LF_CS(11, 15) LF_CS(11, 13) LF_CS(9, 10) LF_CS(11, 12) LF_CS(13, 14) LF_CS(0, 8)
    LF_CS(4, 12) LF_CS(4, 8) LF_CS(2, 10) LF_CS(6, 14) LF_CS(6, 10) LF_CS(2, 4) LF_CS(6, 8)
    LF_CS(1, 9) LF_CS(5, 13) LF_CS(5, 9) LF_CS(3, 11) LF_CS(3, 5) LF_CS(1, 2) LF_CS(3, 4)
    LF_CS(5, 6)
}

__device__ __forceinline__ void insert6(uint32_t s[6], uint32_t key)
{
#pragma unroll
    for (int m = 0; m < 6; ++m) {
        uint32_t lo = min(key, s[m]);
        key = max(key, s[m]);
        s[m] = lo;
    }
}

// FP64 insertion by (d2, index); idx/dd hold `cnt` sorted entries (cnt <= 5).
__device__ __forceinline__ void insert5_exact(int32_t idx[5], double dd[5], int &cnt, int32_t i, double d)
{
    if (cnt == 5 && !(d < dd[4] || (d == dd[4] && i < idx[4]))) return;
    int s = cnt < 5 ? cnt++ : 4;
    while (s > 0 && (d < dd[s - 1] || (d == dd[s - 1] && i < idx[s - 1]))) {
        dd[s] = dd[s - 1];
        idx[s] = idx[s - 1];
        --s;
    }
    dd[s] = d;
    idx[s] = i;
}

struct Window {
    int32_t base, F0, F1;
};

__device__ __forceinline__ Window lattice_window(const PointSetK &P, float3 qh)
{
    float z = qh.z;
    float omz2 = __fmul_rn(__fsub_rn(1.0f, z), __fadd_rn(1.0f, z));
    float t = atan2f(qh.y, qh.x) * kInv2Pi;                        // turns
    float ic = (P.nf * (1.0f - z) - 1.0f) * 0.5f;                  // continuous index
    int k = __float2int_rd(__log2f(kSqrt5Pi * P.nf * omz2) * kInvLog2Phi2);
    k = max(2, min(k, kFibN - 3));
    int32_t F0 = kFib.F[k], F1 = kFib.F[k + 1];
    float e0 = kFib.eps[k], e1 = kFib.eps[k + 1];
    float sg = (k & 1) ? -1.0f : 1.0f;
    float u = sg * __fmaf_rn(-(float)F1, t, e1 * ic);
    float v = sg * __fmaf_rn((float)F0, t, -e0 * ic);
    int32_t u0 = __float2int_rd(u), v0 = __float2int_rd(v);
    return {u0 * F0 + v0 * F1, F0, F1};
}

__device__ __forceinline__ int32_t window_index(const Window &w, int slot)
{
    return w.base + ((slot >> 2) - 1) * w.F0 + ((slot & 3) - 1) * w.F1;
}

// Result: idx[0..cnt) in (distance, index) order and their FP32 squared
// distances d2 (recomputed in double-float). cnt = min(5, n).
__device__ __forceinline__ void knn5(const PointSetK &P, const SphereK &S, float3 h, int32_t idx[5],
                                  float d2[5], int &cnt, uint32_t *status)
{
    float3 qh, ql;
    unit_hit_df(S, h, qh, ql);
    const int32_t n = (int32_t)P.n;
    int src;            // 0 window, 1 scan
    int32_t scan_base = 0, scan_cnt = 0;
    int bits;
    Window w{0, 0, 0};
    if (n <= 128) {
        src = 1; scan_cnt = n; bits = 7;
    } else {
        float icn = (P.nf * (1.0f - qh.z) - 1.0f) * 0.5f;
        float ics = (P.nf * (1.0f + qh.z) - 1.0f) * 0.5f;
        if (icn < 16.0f) { src = 1; scan_cnt = 64; bits = 6; }
        else if (ics < 16.0f) { src = 1; scan_base = n - 64; scan_cnt = 64; bits = 6; }
        else { src = 0; bits = 4; w = lattice_window(P, qh); }
    }
    const uint32_t mask = (1u << bits) - 1u;
    uint32_t s6[6];
    if (src == 0) {
        uint32_t k[16];
#pragma unroll
        for (int s = 0; s < 16; ++s) {
            int32_t i = window_index(w, s);
            bool ok = (i >= 0) & (i < n);
            float dd = ok ? dist2_df(P, i, qh, ql) : 0.0f;
            k[s] = ok ? ((__float_as_uint(dd) & ~mask) | (uint32_t)s) : 0xffffffffu;
        }
        select6_of16(k);
#pragma unroll
        for (int m = 0; m < 6; ++m) s6[m] = k[m];
    } else {
#pragma unroll
        for (int m = 0; m < 6; ++m) s6[m] = 0xffffffffu;
        for (int s = 0; s < scan_cnt; ++s) {
            float dd = dist2_df(P, scan_base + s, qh, ql);
            insert6(s6, (__float_as_uint(dd) & ~mask) | (uint32_t)s);
        }
    }
    // Certification of the FP32 order (including the 5th/6th boundary).
    const float tau = tau_for_bits(bits);
    bool exact = true;
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        if (s6[m + 1] != 0xffffffffu) {
            float a = __uint_as_float(s6[m] & ~mask), b = __uint_as_float(s6[m + 1] & ~mask);
            exact &= (b - a) > __fmaf_rn(tau, b, kTauAbs);
        }
    }
    cnt = 0;
    if (exact) {
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            if (s6[m] != 0xffffffffu) {
                int slot = (int)(s6[m] & mask);
                idx[m] = src == 0 ? window_index(w, slot) : scan_base + slot;
                cnt = m + 1;
            } else {
                idx[m] = -1;
            }
        }
    } else {
        double q[3], dd[5];
        unit_hit_fp64(S, h, q);
        if (src == 0) {
            for (int s = 0; s < 16; ++s) {
                int32_t i = window_index(w, s);
                if (i >= 0 && i < n) insert5_exact(idx, dd, cnt, i, dist2_fp64(P, i, q));
            }
        } else {
            for (int s = 0; s < scan_cnt; ++s)
                insert5_exact(idx, dd, cnt, scan_base + s, dist2_fp64(P, scan_base + s, q));
        }
        for (int m = cnt; m < 5; ++m) idx[m] = -1;
    }
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        if (m < cnt) {
            if ((uint32_t)idx[m] >= (uint32_t)n) {   // impossible by construction; recorded, never trapped
                atomicOr(status, 1u);
                idx[m] = 0;
            }
            d2[m] = dist2_df(P, idx[m], qh, ql);
        } else {
            d2[m] = 0.0f;
        }
    }
}

// Tent weights of one set, normalised to sum 1 (nearest takes all if none is
// inside the kernel radius).
__device__ __forceinline__ void tent_weights(const float d2[5], int cnt, float inv_sigma, float w[5])
{
    float S = 0.0f;
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        float v = m < cnt ? fmaxf(0.0f, 1.0f - sqrtf(d2[m]) * inv_sigma) : 0.0f;
        w[m] = v;
        S += v;
    }
    if (S > 0.0f) {
        float r = 1.0f / S;
#pragma unroll
        for (int m = 0; m < 5; ++m) w[m] *= r;
    } else {
#pragma unroll
        for (int m = 0; m < 5; ++m) w[m] = (m == 0) ? 1.0f : 0.0f;
    }
}

// ---------------------------------------------------------------------------
// Texel decoders: 4 channels to FP32.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float4 texel_f32x4(const void *base, size_t t)
{
    return __ldg(reinterpret_cast<const float4 *>(base) + t);
}
__device__ __forceinline__ float4 texel_f32x3(const void *base, size_t t)
{
    const float *p = reinterpret_cast<const float *>(base) + 3 * t;
    return make_float4(__ldg(p), __ldg(p + 1), __ldg(p + 2), 0.0f);
}
__device__ __forceinline__ float4 texel_f16x4(const void *base, size_t t)
{
    uint2 v = __ldg(reinterpret_cast<const uint2 *>(base) + t);
    __half2 a = *reinterpret_cast<__half2 *>(&v.x), b = *reinterpret_cast<__half2 *>(&v.y);
    float2 fa = __half22float2(a), fb = __half22float2(b);
    return make_float4(fa.x, fa.y, fb.x, fb.y);
}
__device__ __forceinline__ float4 texel_e4m3x4(const void *base, size_t t)
{
    uint32_t v = __ldg(reinterpret_cast<const uint32_t *>(base) + t);
    uint32_t h01, h23;
    asm("{\n\t.reg .b16 lo, hi;\n\tmov.b32 {lo, hi}, %2;\n\t"
        "cvt.rn.f16x2.e4m3x2 %0, lo;\n\tcvt.rn.f16x2.e4m3x2 %1, hi;\n\t}"
        : "=r"(h01), "=r"(h23) : "r"(v));
    float2 fa = __half22float2(*reinterpret_cast<__half2 *>(&h01));
    float2 fb = __half22float2(*reinterpret_cast<__half2 *>(&h23));
    return make_float4(fa.x, fa.y, fb.x, fb.y);
}

template <int DT>
__device__ __forceinline__ float4 texel(const void *base, size_t t)
{
    if constexpr (DT == kF32C4) return texel_f32x4(base, t);
    else if constexpr (DT == kF32C3) return texel_f32x3(base, t);
    else if constexpr (DT == kF16C4) return texel_f16x4(base, t);
    else return texel_e4m3x4(base, t);
}

}  // namespace lfk
