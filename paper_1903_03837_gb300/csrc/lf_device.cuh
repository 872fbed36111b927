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

// Azimuth of (x, y) in turns, for choosing the lattice cell only. atan on
// [0, 1] is a degree-15 odd polynomial, minimax over [0, 1] (Lawson's
// reweighted least squares on Chebyshev nodes, rounded to float32; written by
// fit_atan.py beside this file): 3.7e-8 rad in exact arithmetic, 1.5e-7 rad
// evaluated in float32. Any value congruent modulo whole turns gives the same
// cell, and the window tolerates 2e-3 cells (1.9e-6 rad at n = 2^24).
__device__ __forceinline__ float azimuth_turns(float y, float x)
{
    constexpr float kAtanC[8] = {0.9999993443489075f, -0.33329859375953674f, 0.19946566224098206f,
                                 -0.1390862911939621f, 0.0964219719171524f, -0.0559123270213604f,
                                 0.021862957626581192f, -0.004054567310959101f};
    float ax = fabsf(x), ay = fabsf(y);
    float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
    float a = __fdividef(mn, fmaxf(mx, 1e-30f));
    float a2 = a * a;
    float p = kAtanC[7];
#pragma unroll
    for (int k = 6; k >= 0; --k) p = __fmaf_rn(p, a2, kAtanC[k]);
    float r = a * p;                                   // atan(mn/mx) in [0, pi/4]
    r = ay > ax ? 1.57079632679f - r : r;
    r = x < 0.0f ? 3.14159265359f - r : r;
    r = y < 0.0f ? -r : r;
    return r * kInv2Pi;
}

// ---------------------------------------------------------------------------
// Camera ray and sphere intersection: IEEE FP32, fixed order, no contraction.
// ---------------------------------------------------------------------------
// The camera ray's direction before normalisation is the column term
// fwd + nx*right of pixel column x plus the row term ny*up of pixel row y (in
// this operation order), so a tile can compute its columns and rows once. The
// pixel centre x + 1/2 is scaled by 2/W rounded to FP32 once per view
// (ViewK::inv2w; 2/H likewise), and the direction is normalised by one
// correctly rounded reciprocal of its length: every step an IEEE FP32
// operation, so a CPU reproduces the ray bit for bit.
__device__ __forceinline__ float3 camera_col(const ViewK &v, uint32_t x)
{
    float px = __fadd_rn(__uint2float_rn(x), 0.5f);
    float sx = __fmul_rn(px, v.inv2w);
    float nx = __fmul_rn(__fsub_rn(sx, 1.0f), v.tan_x);
    return make_float3(__fadd_rn(v.fwd[0], __fmul_rn(nx, v.right[0])), __fadd_rn(v.fwd[1], __fmul_rn(nx, v.right[1])),
                       __fadd_rn(v.fwd[2], __fmul_rn(nx, v.right[2])));
}
__device__ __forceinline__ float3 camera_row(const ViewK &v, uint32_t y)
{
    float py = __fadd_rn(__uint2float_rn(y), 0.5f);
    float sy = __fmul_rn(py, v.inv2h);
    float ny = __fmul_rn(__fsub_rn(1.0f, sy), v.tan_y);
    return make_float3(__fmul_rn(ny, v.up[0]), __fmul_rn(ny, v.up[1]), __fmul_rn(ny, v.up[2]));
}
// Unit ray direction from a column term and a row term.
__device__ __forceinline__ float3 camera_dir_cr(float3 c, float3 r)
{
    float vx = __fadd_rn(c.x, r.x), vy = __fadd_rn(c.y, r.y), vz = __fadd_rn(c.z, r.z);
    float l2 = __fadd_rn(__fadd_rn(__fmul_rn(vx, vx), __fmul_rn(vy, vy)), __fmul_rn(vz, vz));
    float il = __frcp_rn(__fsqrt_rn(l2));
    return make_float3(__fmul_rn(vx, il), __fmul_rn(vy, il), __fmul_rn(vz, il));
}
__device__ __forceinline__ float3 camera_dir(const ViewK &v, uint32_t x, uint32_t y)
{
    return camera_dir_cr(camera_col(v, x), camera_row(v, y));
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

// True only for rays that certainly miss S: an approximate ray (FMA, no IEEE
// division) whose line passes outside S, or points away from it, by a
// relative margin of 1e-4 -- far beyond the ~1e-6 difference between this
// approximation and the exact FP32 ray, so the exact step would also report a
// miss. Anything else takes the exact path.
__device__ __forceinline__ bool certain_miss(const ViewK &v, uint32_t x, uint32_t y)
{
    if (!v.outside) return false;
    float nx = __fmaf_rn(__uint2float_rn(x) + 0.5f, v.inv2w, -1.0f) * v.tan_x;
    float ny = __fmaf_rn(-(__uint2float_rn(y) + 0.5f), v.inv2h, 1.0f) * v.tan_y;
    float vx = __fmaf_rn(ny, v.up[0], __fmaf_rn(nx, v.right[0], v.fwd[0]));
    float vy = __fmaf_rn(ny, v.up[1], __fmaf_rn(nx, v.right[1], v.fwd[1]));
    float vz = __fmaf_rn(ny, v.up[2], __fmaf_rn(nx, v.right[2], v.fwd[2]));
    float b = __fmaf_rn(v.f0[0], vx, __fmaf_rn(v.f0[1], vy, v.f0[2] * vz));
    float vv = __fmaf_rn(vx, vx, __fmaf_rn(vy, vy, vz * vz));
    float b2 = b * b, vc = vv * v.c0;
    bool no_disc = (b2 - vc) < -1e-4f * (b2 + vc);
    // b > 1e-4 |v| |f0|, compared in squares (no square root)
    bool away = b > 0.0f && b2 > 1e-8f * (vv * v.ff0);
    return no_disc || away;
}

// The hit mask of a pixel's ray by the approximate ray of certain_miss, where
// it is certain: 0 if the ray certainly misses S, 1 if it certainly hits S in
// front of the eye (discriminant above 0 and direction towards the centre,
// both by the relative margin 1e-4, so the exact step would report the same),
// -1 if only the exact ray/sphere step can tell.
__device__ __forceinline__ int approx_mask(const ViewK &v, uint32_t x, uint32_t y)
{
    if (!v.outside) return -1;
    float nx = __fmaf_rn(__uint2float_rn(x) + 0.5f, v.inv2w, -1.0f) * v.tan_x;
    float ny = __fmaf_rn(-(__uint2float_rn(y) + 0.5f), v.inv2h, 1.0f) * v.tan_y;
    float vx = __fmaf_rn(ny, v.up[0], __fmaf_rn(nx, v.right[0], v.fwd[0]));
    float vy = __fmaf_rn(ny, v.up[1], __fmaf_rn(nx, v.right[1], v.fwd[1]));
    float vz = __fmaf_rn(ny, v.up[2], __fmaf_rn(nx, v.right[2], v.fwd[2]));
    float b = __fmaf_rn(v.f0[0], vx, __fmaf_rn(v.f0[1], vy, v.f0[2] * vz));
    float vv = __fmaf_rn(vx, vx, __fmaf_rn(vy, vy, vz * vz));
    float b2 = b * b, vc = vv * v.c0, m = 1e-4f * sqrtf(vv * v.ff0);
    if ((b2 - vc) < -1e-4f * (b2 + vc) || b > m) return 0;
    if ((b2 - vc) > 1e-4f * (b2 + vc) && b < -m) return 1;
    return -1;
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

// Unit vector (h - O)/|h - O| as hi/lo float3 pairs by a double-float Newton
// step from rsqrt (|error| about 2^-44); used when h lies far off the sphere.
__device__ __forceinline__ void unit_hit_df_newton(df f[3], float3 &qh, float3 &ql)
{
    df r2 = df_add(df_add(df_mul(f[0], f[0]), df_mul(f[1], f[1])), df_mul(f[2], f[2]));
    float y0 = rsqrtf(r2.h);
    df t = df_mul(r2, df{__fmul_rn(y0, y0), __fmaf_rn(y0, y0, -__fmul_rn(y0, y0))});
    float e = __fsub_rn(__fsub_rn(1.0f, t.h), t.l);
    df y = fast_two_sum(y0, __fmul_rn(__fmul_rn(0.5f, y0), e));
    df q0 = df_mul(f[0], y), q1 = df_mul(f[1], y), q2 = df_mul(f[2], y);
    qh = make_float3(q0.h, q1.h, q2.h);
    ql = make_float3(q0.l, q1.l, q2.l);
}

// Unit vector (h - O)/|h - O| as hi/lo float3 pairs. The hit h lies on S up to
// FP32 rounding, so |h - O|^2 = R^2 (1 + eps) with tiny eps, and
// 1/|h - O| = (1/R)(1 - eps/2 + 3 eps^2/8 - 5 eps^3/16 + ...). eps is formed
// from an error-free expansion of |h - O|^2 - R^2; for |eps| <= 2^-12 the
// result is within about 2^-37 of the exact unit vector (2^-45 for the
// |eps| ~ 1e-6 of cameras a few radii away), otherwise the Newton form runs.
__device__ __forceinline__ void unit_hit_df(const SphereK &S, float3 h, float3 &qh, float3 &ql)
{
    df f[3];
    const float hv[3] = {h.x, h.y, h.z};
    if (S.centred) {
#pragma unroll
        for (int k = 0; k < 3; ++k) f[k] = df{hv[k], 0.0f};
    } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            df s = two_sum(hv[k], -S.o_hi[k]);
            f[k] = fast_two_sum(s.h, __fsub_rn(s.l, S.o_lo[k]));
        }
    }
    // |f|^2 - R^2 = sum_k (fh^2 + err(fh^2) + 2 fh fl) - (r2_h + r2_l), cancellation-free
    float p0 = __fmul_rn(f[0].h, f[0].h), p1 = __fmul_rn(f[1].h, f[1].h), p2 = __fmul_rn(f[2].h, f[2].h);
    float small = __fmaf_rn(f[0].h, f[0].h, -p0);
    small = __fadd_rn(small, __fmaf_rn(f[1].h, f[1].h, -p1));
    small = __fadd_rn(small, __fmaf_rn(f[2].h, f[2].h, -p2));
    small = __fmaf_rn(2.0f * f[0].h, f[0].l, small);
    small = __fmaf_rn(2.0f * f[1].h, f[1].l, small);
    small = __fmaf_rn(2.0f * f[2].h, f[2].l, small);
    df a = two_sum(p0, p1);
    df b = two_sum(a.h, p2);
    df c = two_sum(b.h, -S.r2_h);
    float d = __fadd_rn(__fadd_rn(__fadd_rn(c.h, c.l), __fadd_rn(a.l, b.l)), __fsub_rn(small, S.r2_l));
    float eps = __fmul_rn(d, S.inv_r2);
    if (!(fabsf(eps) <= 0x1p-12f)) {
        unit_hit_df_newton(f, qh, ql);
        return;
    }
    float delta = eps * __fmaf_rn(eps, __fmaf_rn(-0.3125f, eps, 0.375f), -0.5f);
    const float s_h = S.ir_h, s_l = __fmaf_rn(S.ir_h, delta, S.ir_l);
    float qhv[3], qlv[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float pr = __fmul_rn(f[k].h, s_h);
        float er = __fmaf_rn(f[k].h, s_h, -pr);
        er = __fmaf_rn(f[k].h, s_l, __fmaf_rn(f[k].l, s_h, er));
        df q = fast_two_sum(pr, er);
        qhv[k] = q.h;
        qlv[k] = q.l;
    }
    qh = make_float3(qhv[0], qhv[1], qhv[2]);
    ql = make_float3(qlv[0], qlv[1], qlv[2]);
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
//   FULL   n <= 128: every point.
//   POLE   the continuous index (n(1-z)-1)/2 of the hit lies within 16 of a
//          pole: the 64 points nearest that pole.
//   WINDOW otherwise: 12 lattice corners around round(u, v) (below), where
//          (u, v) are the hit's coordinates in the local Fibonacci basis of zone k.
// Every source numbers its candidates by a slot s, and candidate s has index
// b0 + (s & 3) G0 + (s >> 2) G1 (a scan takes G0 = 1, G1 = 4: index b0 + s).
//
// Tier 1 ranks every candidate by an FP32 squared distance from the hi parts
// only (key = float bits with the low bits replaced by the slot) and keeps the
// 7 smallest keys, sorted. With the rigorous error bound e1 of that distance,
// the tier-1 order of the top 5 is the exact one when each of the top 6 keys'
// upper bound lies below the next key's lower bound by more than any FP64
// rounding (the order certificate): the common case, which needs double-float
// distances of those 5 only (for the weights). Otherwise (out of line) the
// true 5 nearest still lie among the tier-1 top 6 when the 5th key's upper
// bound is below the 7th key's lower bound; tier 2 recomputes those 6 in
// double-float, sorts them and accepts the order when every consecutive gap
// exceeds the tier-2 error. Anything uncertain is ranked again in FP64 by
// (distance, index) over all candidates.
// ---------------------------------------------------------------------------
#define LF_CS(a, b)                          \
    {                                        \
        uint32_t lo_ = min(k[a], k[b]);      \
        k[b] = max(k[a], k[b]);              \
        k[a] = lo_;                          \
    }

// The 7 smallest of 12 keys, sorted into k[0..6]: Batcher's odd-even merge
// sort of 16 inputs with inputs 12..15 fixed at +inf, pruned to the
// comparators that reach outputs 0..6 (37 comparators; the compiler drops the
// max of the 7 whose larger output is never read).
__device__ __forceinline__ void select7_of12(uint32_t k[12])
{
    LF_CS(0, 1) LF_CS(2, 3) LF_CS(0, 2) LF_CS(1, 3) LF_CS(1, 2) LF_CS(4, 5) LF_CS(6, 7)
    LF_CS(4, 6) LF_CS(5, 7) LF_CS(5, 6) LF_CS(0, 4) LF_CS(2, 6) LF_CS(2, 4) LF_CS(1, 5)
    LF_CS(3, 7) LF_CS(3, 5) LF_CS(1, 2) LF_CS(3, 4) LF_CS(5, 6) LF_CS(8, 9) LF_CS(10, 11)
    LF_CS(8, 10) LF_CS(9, 11) LF_CS(9, 10) LF_CS(0, 8) LF_CS(4, 8) LF_CS(2, 10) LF_CS(6, 10)
    LF_CS(2, 4) LF_CS(6, 8) LF_CS(1, 9) LF_CS(5, 9) LF_CS(3, 11) LF_CS(3, 5) LF_CS(1, 2)
    LF_CS(3, 4) LF_CS(5, 6)
}

// Optimal 12-comparator network sorting 6 keys.
__device__ __forceinline__ void sort6(uint32_t k[6])
{
    LF_CS(1, 2) LF_CS(4, 5) LF_CS(0, 2) LF_CS(3, 5) LF_CS(0, 1) LF_CS(3, 4) LF_CS(1, 4)
    LF_CS(0, 3) LF_CS(2, 5) LF_CS(1, 3) LF_CS(2, 4) LF_CS(2, 3)
}

// The 10 smallest of 25 keys, sorted into k[0..9]: Batcher's odd-even merge
// sort of 32 inputs with inputs 25..31 fixed at +inf, pruned to the
// comparators that reach outputs 0..9 (119 comparators, against 250
// compare-exchanges for inserting the 25 keys into a sorted list of 10).
__device__ __forceinline__ void select10_of25(uint32_t k[25])
{
    LF_CS(0, 1) LF_CS(2, 3) LF_CS(0, 2) LF_CS(1, 3) LF_CS(1, 2) LF_CS(4, 5) LF_CS(6, 7)
    LF_CS(4, 6) LF_CS(5, 7) LF_CS(5, 6) LF_CS(0, 4) LF_CS(2, 6) LF_CS(2, 4) LF_CS(1, 5)
    LF_CS(3, 7) LF_CS(3, 5) LF_CS(1, 2) LF_CS(3, 4) LF_CS(5, 6) LF_CS(8, 9) LF_CS(10, 11)
    LF_CS(8, 10) LF_CS(9, 11) LF_CS(9, 10) LF_CS(12, 13) LF_CS(14, 15) LF_CS(12, 14) LF_CS(13, 15)
    LF_CS(13, 14) LF_CS(8, 12) LF_CS(10, 14) LF_CS(10, 12) LF_CS(9, 13) LF_CS(11, 15) LF_CS(11, 13)
    LF_CS(9, 10) LF_CS(11, 12) LF_CS(13, 14) LF_CS(0, 8) LF_CS(4, 12) LF_CS(4, 8) LF_CS(2, 10)
    LF_CS(6, 14) LF_CS(6, 10) LF_CS(2, 4) LF_CS(6, 8) LF_CS(10, 12) LF_CS(1, 9) LF_CS(5, 13)
    LF_CS(5, 9) LF_CS(3, 11) LF_CS(7, 15) LF_CS(7, 11) LF_CS(3, 5) LF_CS(7, 9) LF_CS(11, 13)
    LF_CS(1, 2) LF_CS(3, 4) LF_CS(5, 6) LF_CS(7, 8) LF_CS(9, 10) LF_CS(11, 12) LF_CS(16, 17)
    LF_CS(18, 19) LF_CS(16, 18) LF_CS(17, 19) LF_CS(17, 18) LF_CS(20, 21) LF_CS(22, 23) LF_CS(20, 22)
    LF_CS(21, 23) LF_CS(21, 22) LF_CS(16, 20) LF_CS(18, 22) LF_CS(18, 20) LF_CS(17, 21) LF_CS(19, 23)
    LF_CS(19, 21) LF_CS(17, 18) LF_CS(19, 20) LF_CS(21, 22) LF_CS(16, 24) LF_CS(20, 24) LF_CS(18, 20)
    LF_CS(22, 24) LF_CS(19, 21) LF_CS(17, 18) LF_CS(19, 20) LF_CS(21, 22) LF_CS(23, 24) LF_CS(0, 16)
    LF_CS(8, 24) LF_CS(8, 16) LF_CS(4, 20) LF_CS(12, 20) LF_CS(4, 8) LF_CS(12, 16) LF_CS(2, 18)
    LF_CS(10, 18) LF_CS(6, 22) LF_CS(6, 10) LF_CS(2, 4) LF_CS(6, 8) LF_CS(10, 12) LF_CS(1, 17)
    LF_CS(9, 17) LF_CS(5, 21) LF_CS(5, 9) LF_CS(3, 19) LF_CS(11, 19) LF_CS(7, 23) LF_CS(7, 11)
    LF_CS(3, 5) LF_CS(7, 9) LF_CS(1, 2) LF_CS(3, 4) LF_CS(5, 6) LF_CS(7, 8) LF_CS(9, 10)
}

__device__ __forceinline__ void insert7(uint32_t s[7], uint32_t key)
{
#pragma unroll
    for (int m = 0; m < 7; ++m) {
        uint32_t lo = min(key, s[m]);
        key = max(key, s[m]);
        s[m] = lo;
    }
}

// Candidate source of one query: slot s -> index b0 + (s & 3) G0 + (s >> 2) G1.
struct Source {
    int32_t b0, G0, G1;
    int32_t scan_cnt;        // 0: lattice window, else the number of scanned points
    int bits;                // tier-1 slot bits
    bool interior;           // every window candidate lies in [0, n)
};

__device__ __forceinline__ int32_t source_index(const Source &s, uint32_t slot)
{
    return s.b0 + (int32_t)(slot & 3u) * s.G0 + (int32_t)(slot >> 2) * s.G1;
}

// Lattice window. (u, v) rounded to the nearest cell corner (ru, rv) = c; the
// candidates are the 3x3 corners around c plus three corners on the side of
// the sign quadrant of (u - ru, v - rv): with (du, dv) the offsets from c,
//   (+,+): (1,2) (2,-1) (2,0)      (-,-): (-2,0) (-1,-2) (-2,1)
//   (+,-): (-1,-2) (0,-2) (2,-1)   (-,+): (-2,1) (0,2) (1,2).
// The four quadrant sets are one set turned by quarter turns of the lattice
// (du, dv) -> (-dv, du), under which the 3x3 block is invariant, so the
// window is the fixed offsets {-1,0,1}^2 + {(1,2), (2,-1), (2,0)} in the basis
// (G0, G1) = (F0, F1), (-F0, -F1), (-F1, F0) or (F1, -F0) of the quadrant
// (+,+), (-,-), (+,-), (-,+). In slots s = (du + 1) + 4 (dv + 1) these are
// s = 0..10 and 14, and candidate s has index c - G0 - G1 + (s & 3) G0 +
// (s >> 2) G1. The window is complete for the 5 nearest (tests/
// test_window_study.py: brute force against this window for n = 256 ... 2^24
// with the lattice coordinates and the zone perturbed by more than their FP32
// error). Outside the pole scan the zone is k >= 6 (F_k >= 8), so the 12
// corners have distinct indices.
__device__ __forceinline__ Source lattice_window(const PointSetK &P, float3 qh)
{
    float z = qh.z;
    float omz2 = __fmul_rn(__fsub_rn(1.0f, z), __fadd_rn(1.0f, z));
    float t = azimuth_turns(qh.y, qh.x);                            // turns
    float ic = (P.nf * (1.0f - z) - 1.0f) * 0.5f;                  // continuous index
    int k = __float2int_rd(__log2f(kSqrt5Pi * P.nf * omz2) * kInvLog2Phi2);
    k = max(2, min(k, kFibN - 3));
    int32_t F0 = kFib.F[k], F1 = kFib.F[k + 1];
    float e0 = kFib.eps[k], e1 = kFib.eps[k + 1];
    float sg = (k & 1) ? -1.0f : 1.0f;
    float u = sg * __fmaf_rn(-(float)F1, t, e1 * ic);
    float v = sg * __fmaf_rn((float)F0, t, -e0 * ic);
    float ru = rintf(u), rv = rintf(v);
    bool pu = u >= ru, pv = v >= rv;
    Source s;
    const int32_t base = (int32_t)ru * F0 + (int32_t)rv * F1;
    s.G0 = pu ? (pv ? F0 : -F1) : (pv ? F1 : -F0);
    s.G1 = pu ? (pv ? F1 : F0) : (pv ? -F0 : -F1);
    s.b0 = base - s.G0 - s.G1;
    const int32_t reach = 2 * (F0 + F1);
    s.interior = (base - reach >= 0) && (base + reach < (int32_t)P.n);
    s.scan_cnt = 0;
    s.bits = 4;
    return s;
}

constexpr int kWindow = 12;

// Slot of window candidate j (0..11).
__device__ __forceinline__ constexpr uint32_t slot5(int j) { return j < 11 ? (uint32_t)j : 14u; }

// Candidate source of one query (see above).
__device__ __forceinline__ Source candidate_source(const PointSetK &P, float3 qh)
{
    const int32_t n = (int32_t)P.n;
    Source s;
    s.b0 = 0;
    s.G0 = 1;
    s.G1 = 4;
    s.interior = true;
    if (n <= 128) {
        s.scan_cnt = n;
        s.bits = 7;
        return s;
    }
    float icn = (P.nf * (1.0f - qh.z) - 1.0f) * 0.5f;
    float ics = (P.nf * (1.0f + qh.z) - 1.0f) * 0.5f;
    s.scan_cnt = 64;
    s.bits = 6;
    if (icn < 16.0f) return s;
    s.b0 = n - 64;
    if (ics < 16.0f) return s;
    return lattice_window(P, qh);
}

// Tier-1 squared distance from the hi parts only.
__device__ __forceinline__ float dist2_hi(const PointSetK &P, int32_t i, float3 qh)
{
    float4 a = __ldg(P.hi + i);
    float dx = __fsub_rn(qh.x, a.x), dy = __fsub_rn(qh.y, a.y), dz = __fsub_rn(qh.z, a.z);
    return __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmul_rn(dz, dz)));
}

// Bound of |dist2_hi - d^2| as a function of the computed d1 = dist2_hi. The
// hi parts lie within 2^-25 (+ the 2^-37 of the unit hit) of q and p per
// component, so each difference is off by at most 2^-24 (1 + 2^-12) plus one
// rounding; squaring and the three roundings of the sum give
// |d1 - d^2| <= 5u d^2 + 2 sqrt(3) 2^-24 d + 3 * 2^-46 (u = 2^-24), which
// 2^-21 d1 + 2^-21 sqrt(d1) + 2^-42 exceeds by a factor of two or more in each
// term (also for d^2 up to d1 + e1, and with the few ulps of rsqrtf).
__device__ __forceinline__ float tier1_err(float d2)
{
    float d = d2 * rsqrtf(fmaxf(d2, 0x1p-100f));          // sqrt(d2) to a few ulps
    return __fmaf_rn(0x1p-21f, d2, __fmaf_rn(0x1p-21f, d, 0x1p-42f));
}

template <int K>
struct TopK {
    int32_t i[K];
    float d2[K];
    int cnt;
};
using Top5 = TopK<5>;

// The 5 nearest points of the unit hit of h (qh + ql) in (distance, index)
// order, with their double-float squared distances; cnt = min(5, n). This is
// the render kernels' fast path: tier 1 and its order certificate, and when
// that fails a short tier 2 over the tier-1 top 6. When tier 2 cannot settle
// the order either, `uncertain` is set and the result is meaningless; the
// render kernel queues the ray for the exact pass (coop_knn5 in a kernel of
// its own). Neither the exact ranking nor any FP64 code sits in the render
// kernel: a rarely taken path there costs the common path registers (spills),
// and run by one lane it holds its warp and CTA for tens of thousands of
// cycles (FP64 division and square root alone take hundreds of cycles each on
// this GPU).
__device__ __forceinline__ Top5 knn5(const PointSetK &P, const SphereK &S, float3 h, uint32_t *status,
                                     bool &uncertain)
{
    float3 qh, ql;
    unit_hit_df(S, h, qh, ql);
    const int32_t n = (int32_t)P.n;
    const Source src = candidate_source(P, qh);
    const uint32_t mask1 = (1u << src.bits) - 1u;
    constexpr uint32_t kNone = 0xffffffffu;

    // Tier 1: the 7 smallest keys, sorted.
    uint32_t s7[7];
    if (src.scan_cnt == 0 && src.interior) {
        // the common case: 12 window corners, all in range, unrolled
        uint32_t k[12];
#pragma unroll
        for (int j = 0; j < kWindow; ++j) {
            const uint32_t s = slot5(j);
            const int32_t i = source_index(src, s);
            const float dd = dist2_hi(P, LF_DINDEX(i, P.n, status, kStatusDebugPoint), qh);
            k[j] = (__float_as_uint(dd) & ~15u) | s;
        }
        select7_of12(k);
#pragma unroll
        for (int m = 0; m < 7; ++m) s7[m] = k[m];
    } else {
        // pole and full scans, windows that reach past either end of the index range
#pragma unroll
        for (int m = 0; m < 7; ++m) s7[m] = kNone;
        const int total = src.scan_cnt ? src.scan_cnt : kWindow;
#pragma unroll 1
        for (int j = 0; j < total; ++j) {
            const uint32_t s = src.scan_cnt ? (uint32_t)j : slot5(j);
            const int32_t i = source_index(src, s);
            if ((uint32_t)i >= (uint32_t)n) continue;
            insert7(s7, (__float_as_uint(dist2_hi(P, LF_DINDEX(i, P.n, status, kStatusDebugPoint), qh)) & ~mask1) | s);
        }
    }

    // Order certificate at tier 1. The keys lost their low `bits` bits to the
    // slot, and one bound e1 serves all of them (tier1_err grows with the
    // distance; taken at the 6th key, and at 4.5 > any squared chord when that
    // slot is empty). Each of the top 6 lying below the next by more than
    // 2^-40 (far above any FP64 rounding of the oracle's distances) makes the
    // order and the membership of the 5 those of the exact ranking: every
    // candidate past the 6th has a key, hence a lower bound, at least the 6th's.
    const float e1 = tier1_err(fminf(__uint_as_float(s7[5] | mask1), 4.5f));
    const float gap = __fmaf_rn(2.0f, e1, 0x1p-40f);
    bool order1 = true;
#pragma unroll
    for (int m = 0; m < 5; ++m)   // no branches here or below: they cost more than the work they skip
        order1 &= (s7[m + 1] == kNone) |
                  (__fsub_rn(__uint_as_float(s7[m + 1] & ~mask1), __uint_as_float(s7[m] | mask1)) > gap);
    // Double-float distances of the tier-1 top 5: the result's weights when the
    // certificate holds, tier 2's input otherwise (an empty slot reads point 0
    // and discards it)
    Top5 r;
    r.cnt = 0;
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        const bool ok = s7[m] != kNone;
        const int32_t i = ok ? source_index(src, s7[m] & mask1) : 0;
        const float d2 = dist2_df(P, LF_DINDEX(i, P.n, status, kStatusDebugPoint), qh, ql);
        r.i[m] = ok ? i : -1;
        r.d2[m] = ok ? d2 : 0.0f;
        r.cnt += ok ? 1 : 0;
    }
    if (order1) return r;
    {
        // Tier 2: the top 6 in double-float, sorted, when the tier-1 bounds put
        // the true 5 nearest among them (the 5th's upper bound below the 7th's
        // lower bound, with the error bound taken at the 7th key). Accepted when
        // every consecutive gap of the 6 exceeds the tier-2 error (2^-21 relative
        // per distance, 2^-20 for the 3 slot bits of the keys, 2^-40 absolute);
        // otherwise the hit is left to the exact pass.
        const float e7 = tier1_err(fminf(__uint_as_float(s7[6] | mask1), 4.5f));
        bool ok2 = s7[6] == kNone ||
                   __fsub_rn(__uint_as_float(s7[6] & ~mask1), e7) > __fadd_rn(__uint_as_float(s7[4] | mask1), e7);
        const int32_t i5 = s7[5] != kNone ? source_index(src, s7[5] & mask1) : 0;
        const float d5 = dist2_df(P, LF_DINDEX(i5, P.n, status, kStatusDebugPoint), qh, ql);
        uint32_t k6[6];
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            const float dm = m < 5 ? r.d2[m] : d5;
            k6[m] = s7[m] != kNone ? ((__float_as_uint(dm) & ~7u) | (uint32_t)m) : kNone;
        }
        sort6(k6);
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            if (k6[m + 1] != kNone) {
                const float a = __uint_as_float(k6[m] & ~7u), b = __uint_as_float(k6[m + 1] & ~7u);
                ok2 &= (b - a) > __fmaf_rn(0x1p-18f, b, 0x1p-40f);
            }
        }
        if (!ok2) {
            uncertain = true;
            return r;
        }
        // the order of the 5 by their tier-2 distances
        Top5 t;
        t.cnt = r.cnt;
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            const int sl = (int)(k6[m] & 7u);
            int32_t i = sl == 5 ? i5 : r.i[0];
            float dd = sl == 5 ? d5 : r.d2[0];
#pragma unroll
            for (int c = 1; c < 5; ++c) {
                i = sl == c ? r.i[c] : i;
                dd = sl == c ? r.d2[c] : dd;
            }
            t.i[m] = k6[m] != kNone ? i : -1;
            t.d2[m] = k6[m] != kNone ? dd : 0.0f;
        }
        return t;
    }
}

// ---------------------------------------------------------------------------
// Warp-cooperative exact ranking (the rare hits whose tier-1 order was not
// certain). All 32 lanes of a warp call it with the same hit h; lane l takes
// candidates l, l + 32, l + 64, l + 96 of the source, each lane computes its
// candidates' squared distances in double-float (tier 2), and six rounds of a
// warp-wide minimum by (distance, index) pick the nearest in order. The order
// is accepted when each of the top 6 lies below the next by more than the
// tier-2 error; otherwise the same rounds run on FP64 distances computed in
// the FP64 definition's operation order (ties to the smaller index). The
// latency is that of a handful of loads and shuffles, not of a long serial
// path in one lane.
// ---------------------------------------------------------------------------

// Squared distance |q - p|^2 in double-float (q = qh + ql, p = hi + lo of
// point i): each difference exact up to 2^-47 (two_sum of the hi parts plus
// the lo parts), squares and sums as double-float products and sums.
__device__ __forceinline__ df dist2_dd(const PointSetK &P, int32_t i, float3 qh, float3 ql)
{
    const float4 a = __ldg(P.hi + i);
    const float4 b = __ldg(P.lo + i);
    const float qv[3] = {qh.x, qh.y, qh.z}, lv[3] = {ql.x, ql.y, ql.z};
    const float av[3] = {a.x, a.y, a.z}, bv[3] = {b.x, b.y, b.z};
    df acc{0.0f, 0.0f};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const df s = two_sum(qv[k], -av[k]);
        const df dx = fast_two_sum(s.h, __fadd_rn(s.l, __fsub_rn(lv[k], bv[k])));
        acc = df_add(acc, df_mul(dx, dx));
    }
    return acc;
}

// Bound of |dist2_dd - d^2| for the exact unit hit and point: the unit hit's
// own error (2^-37 per component at worst) and the differences' 2^-47 give
// 2 sqrt(3) (2^-37 + 2^-47) d, the double-float squares and sums 2^-44 d^2;
// this exceeds both by a factor of two.
__device__ __forceinline__ float tier2_err(float d2)
{
    const float d = d2 * rsqrtf(fmaxf(d2, 0x1p-100f));
    return __fmaf_rn(0x1p-43f, d2, __fmaf_rn(0x1p-34f, d, 0x1p-70f));
}

// (a, ia) < (b, ib) for double-float distances, ties to the smaller index.
__device__ __forceinline__ bool dd_less(df a, int32_t ia, df b, int32_t ib)
{
    return a.h < b.h || (a.h == b.h && (a.l < b.l || (a.l == b.l && ia < ib)));
}

__device__ __forceinline__ Top5 coop_knn5(const PointSetK &P, const SphereK &S, float3 h)
{
    constexpr int kPer = 4;                       // candidates per lane (scans have at most 128)
    constexpr int32_t kNoIdx = 0x7fffffff;
    const unsigned full = 0xffffffffu;
    const int lane = (int)(threadIdx.x & 31u);
    float3 qh, ql;
    unit_hit_df(S, h, qh, ql);
    const int32_t n = (int32_t)P.n;
    const Source src = candidate_source(P, qh);
    const int total = src.scan_cnt ? src.scan_cnt : kWindow;
    df kd[kPer];
    int32_t ki[kPer];
#pragma unroll
    for (int c = 0; c < kPer; ++c) {
        kd[c] = df{INFINITY, 0.0f};
        ki[c] = kNoIdx;
        if (32 * c >= total) continue;            // warp-uniform: windows fill lanes 0..11 only
        const int j = lane + 32 * c;
        const int32_t i = j < total ? source_index(src, src.scan_cnt ? (uint32_t)j : slot5(j)) : -1;
        if ((uint32_t)i < (uint32_t)n) {
            kd[c] = dist2_dd(P, i, qh, ql);
            ki[c] = i;
        }
    }
    // six rounds of a warp-wide minimum; the lane holding the winner retires it
    df wd6[6];
    int32_t wi6[6];
#pragma unroll
    for (int r = 0; r < 6; ++r) {
        df bd = kd[0];
        int32_t bi = ki[0];
#pragma unroll
        for (int c = 1; c < kPer; ++c)
            if (dd_less(kd[c], ki[c], bd, bi)) {
                bd = kd[c];
                bi = ki[c];
            }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            const df od{__shfl_xor_sync(full, bd.h, o), __shfl_xor_sync(full, bd.l, o)};
            const int32_t oi = __shfl_xor_sync(full, bi, o);
            if (dd_less(od, oi, bd, bi)) {
                bd = od;
                bi = oi;
            }
        }
#pragma unroll
        for (int c = 0; c < kPer; ++c)
            if (ki[c] == bi) {
                kd[c] = df{INFINITY, 0.0f};
                ki[c] = kNoIdx;
            }
        wd6[r] = bd;
        wi6[r] = bi;
    }
    bool exact = true;
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        if (wi6[m + 1] != kNoIdx) {
            const float g = __fadd_rn(__fsub_rn(wd6[m + 1].h, wd6[m].h), __fsub_rn(wd6[m + 1].l, wd6[m].l));
            exact &= g > 2.0f * tier2_err(wd6[m + 1].h);
        }
    }
    if (!exact) {
        // FP64 in the definition's operation order, over the same candidates
        double q[3];
        unit_hit_fp64(S, h, q);
        double kq[kPer];
#pragma unroll
        for (int c = 0; c < kPer; ++c) {
            const int j = lane + 32 * c;
            const int32_t i = j < total ? source_index(src, src.scan_cnt ? (uint32_t)j : slot5(j)) : -1;
            const bool ok = (uint32_t)i < (uint32_t)n;
            kq[c] = ok ? dist2_fp64(P, i, q) : INFINITY;
            ki[c] = ok ? i : kNoIdx;
        }
#pragma unroll
        for (int r = 0; r < 5; ++r) {
            double bd = kq[0];
            int32_t bi = ki[0];
#pragma unroll
            for (int c = 1; c < kPer; ++c)
                if (kq[c] < bd || (kq[c] == bd && ki[c] < bi)) {
                    bd = kq[c];
                    bi = ki[c];
                }
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) {
                const double od = __shfl_xor_sync(full, bd, o);
                const int32_t oi = __shfl_xor_sync(full, bi, o);
                if (od < bd || (od == bd && oi < bi)) {
                    bd = od;
                    bi = oi;
                }
            }
#pragma unroll
            for (int c = 0; c < kPer; ++c)
                if (ki[c] == bi) {
                    kq[c] = INFINITY;
                    ki[c] = kNoIdx;
                }
            wi6[r] = bi;
        }
    }
    Top5 res;
    res.cnt = 0;
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        const bool ok = wi6[m] != kNoIdx;
        res.i[m] = ok ? wi6[m] : -1;
        res.d2[m] = ok ? dist2_df(P, wi6[m], qh, ql) : 0.0f;
        res.cnt += ok ? 1 : 0;
    }
    return res;
}

// ---------------------------------------------------------------------------
// The 9 nearest points (the paper's "up to nine" neighbours per hit point).
// Candidates: FULL and POLE as for 5; away from the poles the 5x5 lattice
// corners around round(u, v). A brute-force study over n = 256 ... 262,144
// (600,000 random queries per n, (u, v) perturbed by +-2e-3 and the zone
// number by +-0.02) found the true 9 nearest always within 20 corners per
// sign quadrant of (u - ru, v - rv), all inside this block (the study grew to
// 21 when queries within 12 indices of a pole were admitted, so the pole scan
// keeps its threshold of 16). Ranking: tier-1 keys (5 slot bits) of all
// candidates into a sorted list of the 10 smallest; when each of the top 10
// lies below the next by more than the tier-1 error plus 2^-40, the order and
// membership of the top 9 are exact; otherwise tier 2 re-ranks the top 10 in
// double-float, and FP64 settles what is still uncertain.
// ---------------------------------------------------------------------------
constexpr int kWindow9 = 25;

// The 5x5 corners around the rounded corner c = b0 + G0 + G1 (the block is
// invariant under the quadrant's quarter turns of the basis).
__device__ __forceinline__ int32_t window_index25(const Source &s, int slot)
{
    return s.b0 + (slot / 5 - 1) * s.G0 + (slot % 5 - 1) * s.G1;
}

__device__ __forceinline__ int32_t source_index9(const Source &s, int slot)
{
    return s.scan_cnt ? s.b0 + slot : window_index25(s, slot);
}

template <int N>
__device__ __forceinline__ void insert_sorted(uint32_t (&s)[N], uint32_t key)
{
#pragma unroll
    for (int m = 0; m < N; ++m) {
        uint32_t lo = min(key, s[m]);
        key = max(key, s[m]);
        s[m] = lo;
    }
}

static __device__ __noinline__ TopK<9> knn9_fp64(const PointSetK P, const SphereK S, float3 h, const Source src,
                                          float3 qh, float3 ql)
{
    double q[3];
    unit_hit_fp64(S, h, q);
    int32_t idx[9];
    double dd[9];
    int cnt = 0;
    const int32_t n = (int32_t)P.n;
    const int total = src.scan_cnt ? src.scan_cnt : kWindow9;
    for (int s = 0; s < total; ++s) {
        int32_t i = source_index9(src, s);
        if (i < 0 || i >= n) continue;
        double d = dist2_fp64(P, i, q);
        if (cnt == 9 && !(d < dd[8] || (d == dd[8] && i < idx[8]))) continue;
        int m = cnt < 9 ? cnt++ : 8;
        while (m > 0 && (d < dd[m - 1] || (d == dd[m - 1] && i < idx[m - 1]))) {
            dd[m] = dd[m - 1];
            idx[m] = idx[m - 1];
            --m;
        }
        dd[m] = d;
        idx[m] = i;
    }
    TopK<9> r;
    for (int m = 0; m < 9; ++m) {
        r.i[m] = m < cnt ? idx[m] : -1;
        r.d2[m] = m < cnt ? dist2_df(P, idx[m], qh, ql) : 0.0f;
    }
    r.cnt = cnt;
    return r;
}

// Tier 2 of the 9 nearest (rare: the tier-1 order was not certain): the top 10
// in double-float, sorted (4 slot bits), accepted when every consecutive gap of
// the top 10 exceeds the tier-2 error (2^-18 d^2 + 2^-40, as for 5 neighbours);
// otherwise FP64 by (distance, index). Out of line: the common path keeps its
// registers.
struct Keys10 {
    uint32_t k[10];
};

static __device__ __noinline__ TopK<9> knn9_rerank(const PointSetK P, const SphereK S, float3 h, const Source src,
                                            float3 qh, float3 ql, const Keys10 s10, uint32_t mask1)
{
    constexpr uint32_t kNone = 0xffffffffu;
    uint32_t k10[10];
    int32_t id10[10];
    float dd10[10];
#pragma unroll
    for (int m = 0; m < 10; ++m) {
        bool ok = s10.k[m] != kNone;
        int32_t i = ok ? source_index9(src, (int)(s10.k[m] & mask1)) : 0;
        id10[m] = i;
        dd10[m] = dist2_df(P, i, qh, ql);
        k10[m] = kNone;
    }
#pragma unroll
    for (int m = 0; m < 10; ++m)
        insert_sorted(k10, s10.k[m] != kNone ? ((__float_as_uint(dd10[m]) & ~15u) | (uint32_t)m) : kNone);
    bool exact = true;
#pragma unroll
    for (int m = 0; m < 9; ++m) {
        if (k10[m + 1] != kNone) {
            float a = __uint_as_float(k10[m] & ~15u), b = __uint_as_float(k10[m + 1] & ~15u);
            exact &= (b - a) > __fmaf_rn(0x1p-18f, b, 0x1p-40f);
        }
    }
    if (!exact) return knn9_fp64(P, S, h, src, qh, ql);
    TopK<9> r;
    r.cnt = 0;
#pragma unroll
    for (int m = 0; m < 9; ++m) {
        bool ok = k10[m] != kNone;
        int sl = (int)(k10[m] & 15u);
        int32_t i = id10[0];
        float dd = dd10[0];
#pragma unroll
        for (int c = 1; c < 10; ++c) {
            i = (sl == c) ? id10[c] : i;
            dd = (sl == c) ? dd10[c] : dd;
        }
        r.i[m] = ok ? i : -1;
        r.d2[m] = ok ? dd : 0.0f;
        r.cnt += ok ? 1 : 0;
    }
    return r;
}

// The 9 nearest points of the unit hit in (distance, index) order with their
// double-float squared distances; cnt = min(9, n).
__device__ __forceinline__ TopK<9> knn9(const PointSetK &P, const SphereK &S, float3 h, uint32_t *status)
{
    float3 qh, ql;
    unit_hit_df(S, h, qh, ql);
    const int32_t n = (int32_t)P.n;
    const Source src = candidate_source(P, qh);
    const int bits = src.scan_cnt ? src.bits : 5;
    const uint32_t mask1 = (1u << bits) - 1u;
    constexpr uint32_t kNone = 0xffffffffu;

    uint32_t s10[10];
#pragma unroll
    for (int m = 0; m < 10; ++m) s10[m] = kNone;
    if (src.scan_cnt == 0) {
        uint32_t k[kWindow9];
#pragma unroll
        for (int s = 0; s < kWindow9; ++s) {
            const int32_t i = window_index25(src, s);
            const bool ok = (uint32_t)i < (uint32_t)n;
            const float dd = dist2_hi(P, ok ? i : 0, qh);
            k[s] = ok ? ((__float_as_uint(dd) & ~mask1) | (uint32_t)s) : kNone;
        }
        select10_of25(k);
#pragma unroll
        for (int m = 0; m < 10; ++m) s10[m] = k[m];
    } else {
        for (int s = 0; s < src.scan_cnt; ++s)
            insert_sorted(s10, (__float_as_uint(dist2_hi(P, src.b0 + s, qh)) & ~mask1) | (uint32_t)s);
    }

    // one tier-1 error bound for all keys, taken at the 10th (4.5 for an empty slot)
    const float e = tier1_err(fminf(__uint_as_float(s10[9] | mask1), 4.5f));
    bool order1 = true;
#pragma unroll
    for (int m = 0; m < 9; ++m) {   // no branches here or below (as in knn5)
        const float lb = __uint_as_float(s10[m + 1] & ~mask1) - e;
        const float ub = __uint_as_float(s10[m] | mask1) + e;
        order1 &= (s10[m + 1] == kNone) | ((lb - ub) > 0x1p-40f);
    }
    TopK<9> r;
    r.cnt = 0;
#pragma unroll
    for (int m = 0; m < 9; ++m) {
        const bool ok = s10[m] != kNone;
        const int32_t i = ok ? source_index9(src, (int)(s10[m] & mask1)) : 0;
        const float d2 = dist2_df(P, i, qh, ql);
        r.i[m] = ok ? i : -1;
        r.d2[m] = ok ? d2 : 0.0f;
        r.cnt += ok ? 1 : 0;
    }
    if (!order1) {
        Keys10 keys;
#pragma unroll
        for (int m = 0; m < 10; ++m) keys.k[m] = s10[m];
        r = knn9_rerank(P, S, h, src, qh, ql, keys, mask1);
    }
#pragma unroll
    for (int m = 0; m < 9; ++m) {
        if (m < r.cnt && (uint32_t)r.i[m] >= (uint32_t)n) {   // impossible by construction; recorded, never trapped
            atomicOr(status, 1u);
            r.i[m] = 0;
        }
    }
    return r;
}

// 1/x by the hardware approximation (within 1 ulp; x here is a sum of tent
// weights, in (0, 9]): the weights carry a tolerance, not the bits of an IEEE
// division.
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Tent weights of one set of K neighbours, normalised to sum 1 (nearest takes
// all if none is inside the kernel radius).
template <int K>
__device__ __forceinline__ void tent_weights(const float (&d2)[K], int cnt, float inv_sigma, float (&w)[K])
{
    float S = 0.0f;
#pragma unroll
    for (int m = 0; m < K; ++m) {
        float d = d2[m] * rsqrtf(fmaxf(d2[m], 1e-37f));
        float v = m < cnt ? fmaxf(0.0f, 1.0f - d * inv_sigma) : 0.0f;
        w[m] = v;
        S += v;
    }
    if (S > 0.0f) {
        const float r = rcp_approx(S);
#pragma unroll
        for (int m = 0; m < K; ++m) w[m] *= r;
    } else {
#pragma unroll
        for (int m = 0; m < K; ++m) w[m] = (m == 0) ? 1.0f : 0.0f;
    }
}

// Tent weights over the neighbours with index < rows only (the stored origin
// rows of an upper-hemisphere table), normalised over those; if all of them
// are 0 the nearest kept neighbour takes weight 1. Returns false when no
// neighbour is kept (the ray is masked).
template <int K>
__device__ __forceinline__ bool tent_weights_kept(const float (&d2)[K], const int32_t (&idx)[K], int cnt,
                                                  float inv_sigma, uint32_t rows, float (&w)[K])
{
    float S = 0.0f;
    int first = -1;
#pragma unroll
    for (int m = 0; m < K; ++m) {
        bool keep = m < cnt && (uint32_t)idx[m] < rows;
        first = (keep && first < 0) ? m : first;
        float d = d2[m] * rsqrtf(fmaxf(d2[m], 1e-37f));
        w[m] = keep ? fmaxf(0.0f, 1.0f - d * inv_sigma) : 0.0f;
        S += w[m];
    }
    if (first < 0) return false;
    if (S > 0.0f) {
        const float r = rcp_approx(S);
#pragma unroll
        for (int m = 0; m < K; ++m) w[m] *= r;
    } else {
#pragma unroll
        for (int m = 0; m < K; ++m) w[m] = (m == first) ? 1.0f : 0.0f;
    }
    return true;
}

// ---------------------------------------------------------------------------
// Texel decoders: 4 channels to FP32.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float4 texel_f32x4(const void *base, size_t t)
{
    return __ldg(reinterpret_cast<const float4 *>(base) + t);
}
// 12-byte texels in two loads: the texel's 8-byte-aligned pair (its first two
// floats for even t, its last two for odd t; the table is 8-byte aligned) and
// the remaining float.
__device__ __forceinline__ float4 texel_f32x3(const void *base, size_t t)
{
    const float *p = reinterpret_cast<const float *>(base) + 3 * t;
    const bool odd = (t & 1) != 0;
    const float2 pair = __ldg(reinterpret_cast<const float2 *>(p + (odd ? 1 : 0)));
    const float one = __ldg(p + (odd ? 0 : 2));
    return odd ? make_float4(one, pair.x, pair.y, 0.0f) : make_float4(pair.x, pair.y, one, 0.0f);
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
