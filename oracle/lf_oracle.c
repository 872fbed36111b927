/*
 * lf_oracle.c -- plain, slow CPU oracle for the LumiPath light-field sampling
 * path (Fink et al., "LumiPath -- Towards Real-time Physically-based Rendering
 * on Embedded Devices", arXiv 1903.03837).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark use this file. It shares no code, header, table or
 * constant generator with the CUDA library; it is written from the paper and
 * from the plain definitions of the quantities it computes.
 *
 * What it computes, step by step, each citing the passage it follows:
 *   - spherical-Fibonacci (SF) points p_i            (Section 2, SF point set equation)
 *   - the pinhole camera ray of a pixel               (Section 2, "rasterization ray")
 *   - the front/back hits h_o, h_d on the sphere S    (Section 2, Fig. 2; tangential rays discarded)
 *   - the K nearest SF points of each normalised hit  (Section 2: nearest neighbour of the
 *     inverse mapping, extended to "five neighbours for each point"). The oracle takes
 *     the plain definition: brute force over all n points, ordered by (squared chord
 *     distance, index).
 *   - the distance filter kernel (Section 2, kernel size R*5^(1/4)*sqrt(4*pi/(sqrt(5)*N)),
 *     which equals R*sqrt(4*pi/N) exactly); shape read as a tent of that radius.
 *   - the 25-tap blend of L^(i,j) (Section 2, "25 samples of L^ per pixel").
 *   - the adjoint of that blend with respect to the table (gradient of a linear map).
 *   - the synthetic lobe radiance field used as input, and the FP16 / FP8-E4M3
 *     per-row quantisers written from the IEEE 754 binary16 and OCP E4M3FN definitions.
 *   - the light-field precompute (Section 2, equation of r_k; origins jittered on a
 *     disk of area A_S/M): every ray r_k traced through an analytic emission-absorption
 *     volume (Gaussian blobs), midpoint rule, mean over jittered samples.
 *
 * Everything that decides a neighbour is FP64; the camera ray and the sphere
 * intersection are FP32 with one fixed operation order and no contraction
 * (compile with -ffp-contract=off), so that the hit points are fixed bit patterns.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define LFO_PI 3.14159265358979323846
#define LFO_KMAX 16

/* ------------------------------------------------------------------------- */
/* SF point set (Section 2, SF point set equation).                           */
/* phi_i = 2*pi*frac(i/Phi), z_i = 1 - (2i+1)/n, p_i = C(phi_i, acos z_i).     */
/* frac(i/Phi) = frac(i*(Phi-1)); (Phi-1) is held as the 128-bit fixed-point   */
/* number G = round(2^128 (Phi-1)), so frac(i*(Phi-1)) = (i*G mod 2^128)/2^128 */
/* up to i*2^-129. The phase is then truncated to 53 bits.                     */
/* ------------------------------------------------------------------------- */
static const uint64_t LFO_GOLD_HI = 0x9e3779b97f4a7c15ULL;
static const uint64_t LFO_GOLD_LO = 0xf39cc0605cedc834ULL;

double lfo_sf_phase(uint64_t i)
{
    unsigned __int128 lo = (unsigned __int128)i * LFO_GOLD_LO;
    uint64_t hi = i * LFO_GOLD_HI + (uint64_t)(lo >> 64);
    return ldexp((double)(hi >> 11), -53);
}

void lfo_sf_point(uint32_t n, uint32_t i, double p[3])
{
    double t = lfo_sf_phase(i);
    double phi = (2.0 * LFO_PI) * t;
    double z = 1.0 - (double)(2ull * i + 1ull) / (double)n;
    double s = sqrt((1.0 - z) * (1.0 + z));          /* sin(acos z) */
    p[0] = cos(phi) * s;
    p[1] = sin(phi) * s;
    p[2] = z;
}

void lfo_sf_points(uint32_t n, double *out /* [n][3] */)
{
    for (uint32_t i = 0; i < n; ++i) lfo_sf_point(n, i, out + 3ull * i);
}

/* ------------------------------------------------------------------------- */
/* Camera ray (pinhole), FP32, fixed order. A view is 14 floats:              */
/* eye[3], right[3], up[3], forward[3], tan_half_x, tan_half_y.               */
/* Pixel centres at +0.5; row 0 is the top of the image (+up). The paper      */
/* only asks for one rasterisation ray per pixel (Section 2); this library    */
/* fixes its arithmetic: the pixel centre times 2/W (2/H) rounded to FP32     */
/* once, the direction times the rounded reciprocal of its length.            */
/* ------------------------------------------------------------------------- */
void lfo_camera_ray(const float *vw, uint32_t W, uint32_t H, uint32_t x, uint32_t y,
                    float dir[3])
{
    const float *right = vw + 3, *up = vw + 6, *fwd = vw + 9;
    const float s2w = (float)(2.0 / (double)W), s2h = (float)(2.0 / (double)H);
    float px = (float)x + 0.5f, py = (float)y + 0.5f;
    float sx = px * s2w;
    float sy = py * s2h;
    float nx = (sx - 1.0f) * vw[12];
    float ny = (1.0f - sy) * vw[13];
    float v[3];
    for (int k = 0; k < 3; ++k) v[k] = (fwd[k] + nx * right[k]) + ny * up[k];
    float l2 = (v[0] * v[0] + v[1] * v[1]) + v[2] * v[2];
    float il = 1.0f / sqrtf(l2);
    for (int k = 0; k < 3; ++k) dir[k] = v[k] * il;
}

/* Ray / sphere S (Section 2): front hit h_o and back hit h_d. Returns 0 for a */
/* miss: discriminant <= 0 (tangential rays are discarded) or t_near <= 0.     */
int lfo_intersect(float R, const float O[3], const float e[3], const float d[3],
                  float ho[3], float hd[3])
{
    float f[3] = {e[0] - O[0], e[1] - O[1], e[2] - O[2]};
    float b = (f[0] * d[0] + f[1] * d[1]) + f[2] * d[2];
    float c = ((f[0] * f[0] + f[1] * f[1]) + f[2] * f[2]) - R * R;
    float disc = b * b - c;
    if (!(disc > 0.0f)) return 0;
    float sq = sqrtf(disc);
    float tn = -b - sq, tf = -b + sq;
    if (!(tn > 0.0f)) return 0;
    for (int k = 0; k < 3; ++k) {
        ho[k] = e[k] + tn * d[k];
        hd[k] = e[k] + tf * d[k];
    }
    return 1;
}

/* Hit point on S -> unit vector about the centre, FP64. */
void lfo_normalize_hit(const float h[3], const double O[3], double q[3])
{
    double f0 = (double)h[0] - O[0], f1 = (double)h[1] - O[1], f2 = (double)h[2] - O[2];
    double l = sqrt((f0 * f0 + f1 * f1) + f2 * f2);
    q[0] = f0 / l; q[1] = f1 / l; q[2] = f2 / l;
}

/* ------------------------------------------------------------------------- */
/* K nearest SF points of q by brute force over all n points (the definition */
/* the inverse mapping of Section 2 reaches). Order: (d^2, index) ascending;  */
/* equal distances go to the smaller index. Returns the number found.        */
/* ------------------------------------------------------------------------- */
int lfo_knn(const double *P, uint32_t n, const double q[3], int K, int32_t *idx, double *d2)
{
    int cnt = 0;
    if (K > LFO_KMAX) K = LFO_KMAX;
    for (uint32_t i = 0; i < n; ++i) {
        const double *p = P + 3ull * i;
        double a = q[0] - p[0], b = q[1] - p[1], c = q[2] - p[2];
        double dd = (a * a + b * b) + c * c;
        if (cnt == K && !(dd < d2[K - 1])) continue;   /* later i never wins a tie */
        int s = (cnt < K) ? cnt++ : K - 1;
        while (s > 0 && dd < d2[s - 1]) { d2[s] = d2[s - 1]; idx[s] = idx[s - 1]; --s; }
        d2[s] = dd; idx[s] = (int32_t)i;
    }
    return cnt;
}

/* Filter kernel (Section 2): radius sigma_n = sqrt(4*pi/n) on the unit sphere */
/* (the printed size divided by R), tent shape; weights of one set normalised  */
/* to sum 1; if all are zero the nearest point takes weight 1.                  */
double lfo_kernel_sigma(uint32_t n) { return sqrt(4.0 * LFO_PI / (double)n); }

void lfo_tent_weights(const double *d2, int cnt, uint32_t n, double *w)
{
    double sigma = lfo_kernel_sigma(n), S = 0.0;
    for (int a = 0; a < cnt; ++a) {
        double v = 1.0 - sqrt(d2[a]) / sigma;
        w[a] = v > 0.0 ? v : 0.0;
        S += w[a];
    }
    if (S > 0.0) {
        for (int a = 0; a < cnt; ++a) w[a] /= S;
    } else {
        for (int a = 0; a < cnt; ++a) w[a] = (a == 0) ? 1.0 : 0.0;
    }
}

/* Tent weights over the neighbours with index < rows only (others weigh 0),  */
/* normalised over those; if all of them are 0 the nearest kept one takes 1.   */
void lfo_tent_weights_kept(const double *d2, const int32_t *idx, int cnt, uint32_t n, int32_t rows,
                           double *w)
{
    double sigma = lfo_kernel_sigma(n), S = 0.0;
    int first = -1;
    for (int a = 0; a < cnt; ++a) {
        int keep = idx[a] < rows;
        if (keep && first < 0) first = a;
        double v = keep ? 1.0 - sqrt(d2[a]) / sigma : 0.0;
        w[a] = v > 0.0 ? v : 0.0;
        S += w[a];
    }
    if (S > 0.0) {
        for (int a = 0; a < cnt; ++a) w[a] /= S;
    } else {
        for (int a = 0; a < cnt; ++a) w[a] = (a == first) ? 1.0 : 0.0;
    }
}

/* ------------------------------------------------------------------------- */
/* Quantisers.                                                                */
/* IEEE 754 binary16: 1 sign, 5 exponent (bias 15), 10 fraction bits.         */
/* OCP FP8 E4M3FN: 1 sign, 4 exponent (bias 7), 3 fraction bits, no infinity, */
/* S.1111.111 is NaN, largest finite 448. Both round to nearest, ties to even; */
/* E4M3 saturates to +-448.                                                     */
/* ------------------------------------------------------------------------- */
double lfo_f16_decode(uint16_t h)
{
    int s = h >> 15, e = (h >> 10) & 31, m = h & 1023;
    double v;
    if (e == 0) v = ldexp((double)m, -24);
    else if (e == 31) v = m ? NAN : INFINITY;
    else v = ldexp(1024.0 + m, e - 25);
    return s ? -v : v;
}

uint16_t lfo_f16_encode(float xf)
{
    double x = (double)xf;
    uint16_t sign = (signbit(x) ? 0x8000 : 0);
    double a = fabs(x);
    if (isnan(x)) return 0x7e00;
    if (a == 0.0) return sign;
    int e;
    frexp(a, &e);                 /* a = f * 2^e, f in [0.5, 1) -> unbiased exponent e-1 */
    int ue = e - 1;
    if (ue < -14) {               /* subnormal range: multiples of 2^-24 */
        double m = nearbyint(ldexp(a, 24));
        return (uint16_t)(sign | (uint16_t)m);   /* m == 1024 is the smallest normal */
    }
    double m = nearbyint(ldexp(a, -ue) * 1024.0 - 1024.0);
    if (m == 1024.0) { m = 0.0; ++ue; }
    if (ue > 15) return (uint16_t)(sign | 0x7c00);
    return (uint16_t)(sign | (uint16_t)((ue + 15) << 10) | (uint16_t)m);
}

double lfo_e4m3_decode(uint8_t b)
{
    int s = b >> 7, e = (b >> 3) & 15, m = b & 7;
    double v;
    if (e == 15 && m == 7) v = NAN;
    else if (e == 0) v = ldexp((double)m, -9);
    else v = ldexp(8.0 + m, e - 10);
    return s ? -v : v;
}

uint8_t lfo_e4m3_encode(float xf)
{
    double x = (double)xf;
    uint8_t sign = (signbit(x) ? 0x80 : 0);
    double a = fabs(x);
    if (isnan(x)) return 0x7f;
    if (a >= 448.0) return (uint8_t)(sign | 0x7e);
    if (a == 0.0) return sign;
    int e;
    frexp(a, &e);
    int ue = e - 1;
    if (ue < -6) {                /* subnormal: multiples of 2^-9 */
        double m = nearbyint(ldexp(a, 9));
        return (uint8_t)(sign | (uint8_t)m);     /* m == 8 is the smallest normal */
    }
    double m = nearbyint(ldexp(a, -ue) * 8.0 - 8.0);
    if (m == 8.0) { m = 0.0; ++ue; }
    if (ue > 8) return (uint8_t)(sign | 0x7e);
    return (uint8_t)(sign | (uint8_t)((ue + 7) << 3) | (uint8_t)m);
}

/* Per-row quantisation of an FP32 table [M][N][C]. dtype 1 = FP16 (scale =   */
/* amax), dtype 2 = E4M3 (scale = amax/448). amax over all texels and channels */
/* of the row; amax == 0 gives scale 1. q = fl32(x / scale), then encode.      */
void lfo_quantize_rows(const float *T, uint32_t M, uint32_t N, uint32_t C, int dtype,
                       void *codes, float *scales)
{
    size_t row = (size_t)N * C;
    for (uint32_t i = 0; i < M; ++i) {
        const float *r = T + (size_t)i * row;
        float amax = 0.0f;
        for (size_t k = 0; k < row; ++k) { float a = fabsf(r[k]); if (a > amax) amax = a; }
        float s = (amax == 0.0f) ? 1.0f : (dtype == 2 ? amax / 448.0f : amax);
        scales[i] = s;
        for (size_t k = 0; k < row; ++k) {
            float q = r[k] / s;
            if (dtype == 2) ((uint8_t *)codes)[(size_t)i * row + k] = lfo_e4m3_encode(q);
            else ((uint16_t *)codes)[(size_t)i * row + k] = lfo_f16_encode(q);
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Synthetic lobe radiance field (input recipe, not part of the paper).       */
/* T(i,j,c) = sum_l col[l][c] * exp(kp_l (p^o_i . ap_l - 1))                  */
/*                             * exp(kd_l (dhat_ij . ad_l - 1))               */
/*            + 0.01 * u(seed, i, j, c),                                      */
/* dhat_ij = (p^d_j - p^o_i)/|p^d_j - p^o_i| (the ray direction of r_k,       */
/* Section 2), -p^o_i if that length is below 1e-12. u is SplitMix64 (Steele, */
/* Lea, Flood 2014): output number (ctr+1) of the stream seeded with `seed`,  */
/* ctr = i<<32 | j<<4 | c, mapped to [0,1) by its top 53 bits.                */
/* ------------------------------------------------------------------------- */
uint64_t lfo_splitmix64(uint64_t seed, uint64_t ctr)
{
    uint64_t z = seed + (ctr + 1ull) * 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

typedef struct {
    uint32_t L, C;
    uint64_t seed;
    const double *ap, *ad;   /* [L][3] unit axes (position, direction) */
    const double *kp, *kd;   /* [L] sharpness */
    const double *col;       /* [L][C] colour */
} lfo_lobes;

void lfo_lobe_texel(const lfo_lobes *lb, const double *Po, const double *Pd,
                    uint32_t i, uint32_t j, double *out /* [C] */)
{
    const double *po = Po + 3ull * i, *pd = Pd + 3ull * j;
    double d[3] = {pd[0] - po[0], pd[1] - po[1], pd[2] - po[2]};
    double l = sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]);
    if (l < 1e-12) { d[0] = -po[0]; d[1] = -po[1]; d[2] = -po[2]; }
    else { d[0] /= l; d[1] /= l; d[2] /= l; }
    for (uint32_t c = 0; c < lb->C; ++c) out[c] = 0.0;
    for (uint32_t k = 0; k < lb->L; ++k) {
        const double *a = lb->ap + 3 * k, *b = lb->ad + 3 * k;
        double cp = (po[0] * a[0] + po[1] * a[1]) + po[2] * a[2];
        double cd = (d[0] * b[0] + d[1] * b[1]) + d[2] * b[2];
        double g = exp(lb->kp[k] * (cp - 1.0)) * exp(lb->kd[k] * (cd - 1.0));
        for (uint32_t c = 0; c < lb->C; ++c) out[c] += lb->col[k * lb->C + c] * g;
    }
    for (uint32_t c = 0; c < lb->C; ++c) {
        uint64_t ctr = ((uint64_t)i << 32) | ((uint64_t)j << 4) | (uint64_t)c;
        double u = ldexp((double)(lfo_splitmix64(lb->seed, ctr) >> 11), -53);
        out[c] += 0.01 * u;
    }
}

/* FP32 table rows [i0, i1) of the lobe field (FP64 evaluation, rounded once). */
void lfo_lobe_table_rows(const lfo_lobes *lb, const double *Po, const double *Pd,
                         uint32_t N, uint32_t i0, uint32_t i1, float *out /* [(i1-i0)][N][C] */)
{
    double v[16];
    for (uint32_t i = i0; i < i1; ++i)
        for (uint32_t j = 0; j < N; ++j) {
            lfo_lobe_texel(lb, Po, Pd, i, j, v);
            for (uint32_t c = 0; c < lb->C; ++c)
                out[(((size_t)(i - i0)) * N + j) * lb->C + c] = (float)v[c];
        }
}

static void lfo_chord_dir(const double p[3], const double q[3], double d[3]);

/* The lobe field as a continuous function of an origin q on the unit sphere
   and a unit direction d: the texel formula with p^o_i -> q and d_ij -> d,
   without the per-texel noise. The table samples this function at the SF
   points; rendering interpolates it, so it is the reference of image quality
   for a given neighbour count. */
void lfo_lobe_continuous(const lfo_lobes *lb, const double q[3], const double d[3],
                         double *out /* [C] */)
{
    for (uint32_t c = 0; c < lb->C; ++c) out[c] = 0.0;
    for (uint32_t k = 0; k < lb->L; ++k) {
        const double *a = lb->ap + 3 * k, *b = lb->ad + 3 * k;
        double cp = (q[0] * a[0] + q[1] * a[1]) + q[2] * a[2];
        double cd = (d[0] * b[0] + d[1] * b[1]) + d[2] * b[2];
        double g = exp(lb->kp[k] * (cp - 1.0)) * exp(lb->kd[k] * (cd - 1.0));
        for (uint32_t c = 0; c < lb->C; ++c) out[c] += lb->col[k * lb->C + c] * g;
    }
}

/* Reference pixels: the continuous lobe field at the pixel's normalised front
   hit and the unit chord direction from the front to the back hit (the ray's
   own direction inside S); hit[p] = 0 and out 0 for a miss. */
int64_t lfo_lobe_reference_pixels(const lfo_lobes *lb, double R, const double O[3], const float *views,
                                  const uint32_t *wh, const uint32_t *pix, int64_t np, double *out,
                                  uint8_t *hit)
{
    int64_t hits = 0;
    float O32[3] = {(float)O[0], (float)O[1], (float)O[2]};
    for (int64_t p = 0; p < np; ++p) {
        uint32_t v = pix[3 * p], x = pix[3 * p + 1], y = pix[3 * p + 2];
        const float *vw = views + 14 * v;
        float d[3], ho[3], hd[3];
        for (uint32_t c = 0; c < lb->C; ++c) out[p * lb->C + c] = 0.0;
        hit[p] = 0;
        lfo_camera_ray(vw, wh[2 * v], wh[2 * v + 1], x, y, d);
        if (!lfo_intersect((float)R, O32, vw, d, ho, hd)) continue;
        double qo[3], qd[3], u[3];
        lfo_normalize_hit(ho, O, qo);
        lfo_normalize_hit(hd, O, qd);
        lfo_chord_dir(qo, qd, u);
        lfo_lobe_continuous(lb, qo, u, out + p * lb->C);
        hit[p] = 1;
        ++hits;
    }
    return hits;
}

/* ------------------------------------------------------------------------- */
/* Rendering (Section 2): per pixel, ray -> hits -> K-NN of each hit ->       */
/* tent weights -> sum_ab W_ab * L^(i_a, j_b).                                */
/* ------------------------------------------------------------------------- */
typedef struct {
    double R, O[3];
    uint32_t M, N, C;
    int K;
    const double *Po, *Pd;   /* SF points [M][3], [N][3] */
    int dtype;               /* 0 FP32, 1 FP16 codes, 2 E4M3 codes, 3 lobe field in FP64 */
    const void *table;       /* [M][N][C] FP32 or codes */
    const float *scales;     /* [M] for dtype 1, 2 */
    const lfo_lobes *lobes;  /* dtype 3 */
    const int32_t *rowmap;   /* optional [M]: table/scale row holding origin row i (-1: absent) */
    int upper;               /* 1: only the upper-hemisphere origin rows (z_i > 0, i < M/2) exist */
} lfo_scene;

static void lfo_fetch(const lfo_scene *S, uint32_t i, uint32_t j, double *v)
{
    int64_t r = S->rowmap ? (int64_t)S->rowmap[i] : (int64_t)i;
    if (S->dtype != 3 && r < 0) {
        for (uint32_t c = 0; c < S->C; ++c) v[c] = NAN;
        return;
    }
    size_t base = ((size_t)r * S->N + j) * S->C;
    switch (S->dtype) {
    case 0:
        for (uint32_t c = 0; c < S->C; ++c) v[c] = (double)((const float *)S->table)[base + c];
        break;
    case 1:
        for (uint32_t c = 0; c < S->C; ++c)
            v[c] = (double)S->scales[r] * lfo_f16_decode(((const uint16_t *)S->table)[base + c]);
        break;
    case 2:
        for (uint32_t c = 0; c < S->C; ++c)
            v[c] = (double)S->scales[r] * lfo_e4m3_decode(((const uint8_t *)S->table)[base + c]);
        break;
    default:
        lfo_lobe_texel(S->lobes, S->Po, S->Pd, i, j, v);
        break;
    }
}

/* One pixel: indices (K origin, K direction; -1 on a miss), weights, hit flag. */
static int lfo_pixel_samples(const lfo_scene *S, const float *vw, uint32_t W, uint32_t H,
                             uint32_t x, uint32_t y, int32_t *io, int32_t *jd,
                             double *wo, double *wd, int *ko, int *kd)
{
    float d[3], ho[3], hd[3];
    float O32[3] = {(float)S->O[0], (float)S->O[1], (float)S->O[2]};
    lfo_camera_ray(vw, W, H, x, y, d);
    if (!lfo_intersect((float)S->R, O32, vw, d, ho, hd)) return 0;
    double qo[3], qd[3], d2o[LFO_KMAX], d2d[LFO_KMAX];
    lfo_normalize_hit(ho, S->O, qo);
    lfo_normalize_hit(hd, S->O, qd);
    *ko = lfo_knn(S->Po, S->M, qo, S->K, io, d2o);
    *kd = lfo_knn(S->Pd, S->N, qd, S->K, jd, d2d);
    if (S->upper) {
        /* Section 3: only origins of the upper hemisphere are stored. Origin
         * neighbours outside the stored rows are dropped and the remaining
         * weights renormalised; a pixel with none left is masked (as a miss). */
        int kept = 0;
        for (int a = 0; a < *ko; ++a) kept += io[a] < (int32_t)(S->M / 2);
        if (!kept) return 0;
        lfo_tent_weights_kept(d2o, io, *ko, S->M, (int32_t)(S->M / 2), wo);
    } else {
        lfo_tent_weights(d2o, *ko, S->M, wo);
    }
    lfo_tent_weights(d2d, *kd, S->N, wd);
    return 1;
}

/* Render a list of pixels. views: [nv][14] floats, wh: [nv][2], pix: [np][3]  */
/* (view, x, y). out: [np][C] FP64; idx (optional): [np][2K]. Returns hits.    */
int64_t lfo_render_pixels(const lfo_scene *S, const float *views, const uint32_t *wh,
                          const uint32_t *pix, int64_t np, double *out, int32_t *idx)
{
    int64_t hits = 0;
    int K = S->K;
    for (int64_t p = 0; p < np; ++p) {
        uint32_t v = pix[3 * p], x = pix[3 * p + 1], y = pix[3 * p + 2];
        int32_t io[LFO_KMAX], jd[LFO_KMAX];
        double wo[LFO_KMAX], wd[LFO_KMAX], t[16];
        int ko = 0, kd = 0;
        int hit = lfo_pixel_samples(S, views + 14 * v, wh[2 * v], wh[2 * v + 1], x, y,
                                    io, jd, wo, wd, &ko, &kd);
        for (uint32_t c = 0; c < S->C; ++c) out[p * S->C + c] = 0.0;
        if (idx) for (int k = 0; k < 2 * K; ++k) idx[p * 2 * K + k] = -1;
        if (!hit) continue;
        ++hits;
        for (int a = 0; a < ko; ++a)
            for (int b = 0; b < kd; ++b) {
                if (S->upper && io[a] >= (int32_t)(S->M / 2)) continue;   /* not stored */
                double W = wo[a] * wd[b];
                lfo_fetch(S, (uint32_t)io[a], (uint32_t)jd[b], t);
                for (uint32_t c = 0; c < S->C; ++c) out[p * S->C + c] += W * t[c];
            }
        if (idx) {
            for (int a = 0; a < ko; ++a) idx[p * 2 * K + a] = io[a];
            for (int b = 0; b < kd; ++b) idx[p * 2 * K + K + b] = jd[b];
        }
    }
    return hits;
}

/* Adjoint of the blend with respect to the table: G[i_a][j_b][c] += W_ab g_c. */
void lfo_render_backward_pixels(const lfo_scene *S, const float *views, const uint32_t *wh,
                                const uint32_t *pix, int64_t np, const double *g, double *G)
{
    for (int64_t p = 0; p < np; ++p) {
        uint32_t v = pix[3 * p], x = pix[3 * p + 1], y = pix[3 * p + 2];
        int32_t io[LFO_KMAX], jd[LFO_KMAX];
        double wo[LFO_KMAX], wd[LFO_KMAX];
        int ko = 0, kd = 0;
        if (!lfo_pixel_samples(S, views + 14 * v, wh[2 * v], wh[2 * v + 1], x, y,
                               io, jd, wo, wd, &ko, &kd))
            continue;
        for (int a = 0; a < ko; ++a)
            for (int b = 0; b < kd; ++b) {
                if (S->upper && io[a] >= (int32_t)(S->M / 2)) continue;   /* not stored */
                double W = wo[a] * wd[b];
                size_t base = ((size_t)io[a] * S->N + (size_t)jd[b]) * S->C;
                for (uint32_t c = 0; c < S->C; ++c) G[base + c] += W * g[p * S->C + c];
            }
    }
}

/* Pixel-level pieces for the tests: ray, hits and normalised hits of pixels. */
int lfo_trace_pixel(double R, const double O[3], const float *vw, uint32_t W, uint32_t H,
                    uint32_t x, uint32_t y, float dir[3], float ho[3], float hd[3],
                    double qo[3], double qd[3])
{
    float O32[3] = {(float)O[0], (float)O[1], (float)O[2]};
    lfo_camera_ray(vw, W, H, x, y, dir);
    if (!lfo_intersect((float)R, O32, vw, dir, ho, hd)) return 0;
    lfo_normalize_hit(ho, O, qo);
    lfo_normalize_hit(hd, O, qd);
    return 1;
}

/* ------------------------------------------------------------------------- */
/* Light-field precompute (Section 2): L^(i,j) is the radiance a camera ray   */
/* r_k = (O + R p^o_i) + t d_ij, d_ij = (p^d_j - p^o_i)/|p^d_j - p^o_i|,       */
/* collects inside S; each of `spp` samples moves the origin uniformly on a   */
/* disk of area A_S / M = 4 pi R^2 / M tangent to S at O + R p^o_i, and the   */
/* texel is the mean of the samples. The scene here is an emission-absorption */
/* volume of Gaussian blobs (density kappa_b exp(-|x - mu_b|^2 / (2 s_b^2)),  */
/* emitted radiance per unit length = density times the blob's colour) in    */
/* front of a background that depends on the direction only. Each sample     */
/* integrates, from the origin (t = 0) to the far intersection with S, the    */
/* emission-absorption equation by the midpoint rule with `steps` steps of    */
/* constant density and emission: L += T (1 - exp(-sigma dt)) / sigma * q,    */
/* T *= exp(-sigma dt); the background is seen through the final T.           */
/* ------------------------------------------------------------------------- */
typedef struct {
    uint32_t B, C;              /* blobs; channels 3 (RGB) or 4 (RGB + opacity 1 - T) */
    uint32_t spp, steps;        /* samples per texel; midpoint steps per sample */
    uint32_t jitter;            /* 1: origins jittered on the disk; 0: at O + R p^o_i */
    uint32_t pad_;
    uint64_t seed;              /* counter-based generator (SplitMix64) seed */
    double R, O[3];
    const double *mu;           /* [B][3] blob centres */
    const double *width;        /* [B] s_b > 0 */
    const double *dens;         /* [B] kappa_b >= 0 (per unit length) */
    const double *emit;         /* [B][3] emitted colour */
    double bg0[3], bg1[3];      /* background bg0 + bg1 (1 + d_z) / 2 */
} lfo_volume;

/* Uniform in [0, 1) on a 2^-24 grid: the top 24 bits of SplitMix64(seed, ctr). */
static double lfo_u24(uint64_t seed, uint64_t ctr)
{
    return ldexp((double)(lfo_splitmix64(seed, ctr) >> 40), -24);
}

/* Unit direction of the chord from p (origin point) to q (direction point);
   -p if the two coincide (same convention as the lobe field). */
static void lfo_chord_dir(const double p[3], const double q[3], double d[3])
{
    double v[3] = {q[0] - p[0], q[1] - p[1], q[2] - p[2]};
    double l = sqrt((v[0] * v[0] + v[1] * v[1]) + v[2] * v[2]);
    if (l < 1e-12) { d[0] = -p[0]; d[1] = -p[1]; d[2] = -p[2]; return; }
    d[0] = v[0] / l; d[1] = v[1] / l; d[2] = v[2] / l;
}

/* Origin of sample s of texel (i, j): O + R p + r (cos a e_phi + sin a e_theta),
   r = (2R / sqrt(M)) sqrt(u1), a = 2 pi u2, with e_phi, e_theta the unit
   tangents of the sphere at p along azimuth and polar angle. */
void lfo_volume_origin(const lfo_volume *V, uint32_t M, uint32_t N, const double p[3],
                       uint32_t i, uint32_t j, uint32_t s, double o[3])
{
    for (int k = 0; k < 3; ++k) o[k] = V->O[k] + V->R * p[k];
    if (!V->jitter) return;
    uint64_t ctr = 2ull * (((uint64_t)i * N + j) * V->spp + s);
    double u1 = lfo_u24(V->seed, ctr), u2 = lfo_u24(V->seed, ctr + 1);
    double rho = sqrt(p[0] * p[0] + p[1] * p[1]);
    double ephi[3] = {1.0, 0.0, 0.0}, eth[3] = {0.0, 1.0, 0.0};
    if (rho > 0.0) {
        ephi[0] = -p[1] / rho; ephi[1] = p[0] / rho; ephi[2] = 0.0;
        eth[0] = p[0] * p[2] / rho; eth[1] = p[1] * p[2] / rho; eth[2] = -rho;
    }
    double r = 2.0 * V->R / sqrt((double)M) * sqrt(u1), a = 2.0 * LFO_PI * u2;
    for (int k = 0; k < 3; ++k) o[k] += r * (cos(a) * ephi[k] + sin(a) * eth[k]);
}

/* Far end of the segment inside S: max(0, -b + sqrt(b^2 - c)), 0 if the line misses. */
double lfo_volume_tend(const lfo_volume *V, const double o[3], const double d[3])
{
    double f[3] = {o[0] - V->O[0], o[1] - V->O[1], o[2] - V->O[2]};
    double b = (f[0] * d[0] + f[1] * d[1]) + f[2] * d[2];
    double c = ((f[0] * f[0] + f[1] * f[1]) + f[2] * f[2]) - V->R * V->R;
    double disc = b * b - c;
    if (disc <= 0.0) return 0.0;
    double t = -b + sqrt(disc);
    return t > 0.0 ? t : 0.0;
}

/* One ray: radiance rgb[3] (background included) and final transmittance. */
void lfo_volume_ray(const lfo_volume *V, const double o[3], const double d[3], double rgb[3],
                    double *T_out)
{
    double t_end = lfo_volume_tend(V, o, d);
    double dt = t_end / (double)V->steps;
    double T = 1.0, L[3] = {0.0, 0.0, 0.0};
    for (uint32_t k = 0; k < V->steps && dt > 0.0; ++k) {
        double t = ((double)k + 0.5) * dt;
        double x[3] = {o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2]};
        double sigma = 0.0, q[3] = {0.0, 0.0, 0.0};
        for (uint32_t b = 0; b < V->B; ++b) {
            const double *m = V->mu + 3 * b;
            double r2 = ((x[0] - m[0]) * (x[0] - m[0]) + (x[1] - m[1]) * (x[1] - m[1])) +
                        (x[2] - m[2]) * (x[2] - m[2]);
            double g = V->dens[b] * exp(-r2 / (2.0 * V->width[b] * V->width[b]));
            sigma += g;
            for (int c = 0; c < 3; ++c) q[c] += g * V->emit[3 * b + c];
        }
        if (sigma > 0.0) {
            double phi = -expm1(-sigma * dt) / sigma;     /* integral of exp(-sigma t) over the step */
            for (int c = 0; c < 3; ++c) L[c] += T * phi * q[c];
            T *= exp(-sigma * dt);
        }
    }
    double w = 0.5 * (1.0 + d[2]);
    for (int c = 0; c < 3; ++c) rgb[c] = L[c] + T * (V->bg0[c] + V->bg1[c] * w);
    *T_out = T;
}

/* Texel (i, j): mean over the samples; channel 3 (if C = 4) is the mean opacity. */
void lfo_volume_texel(const lfo_volume *V, const double *Po, const double *Pd, uint32_t M,
                      uint32_t N, uint32_t i, uint32_t j, double *out /* [C] */)
{
    const double *p = Po + 3ull * i, *q = Pd + 3ull * j;
    double d[3], acc[4] = {0.0, 0.0, 0.0, 0.0};
    lfo_chord_dir(p, q, d);
    for (uint32_t s = 0; s < V->spp; ++s) {
        double o[3], rgb[3], T;
        lfo_volume_origin(V, M, N, p, i, j, s, o);
        lfo_volume_ray(V, o, d, rgb, &T);
        for (int c = 0; c < 3; ++c) acc[c] += rgb[c];
        acc[3] += 1.0 - T;
    }
    for (uint32_t c = 0; c < V->C; ++c) out[c] = acc[c] / (double)V->spp;
}

/* FP32 table rows [i0, i1) of the volume scene (FP64 evaluation, rounded once). */
void lfo_volume_table_rows(const lfo_volume *V, const double *Po, const double *Pd, uint32_t M,
                           uint32_t N, uint32_t i0, uint32_t i1, float *out /* [(i1-i0)][N][C] */)
{
    double v[4];
    for (uint32_t i = i0; i < i1; ++i)
        for (uint32_t j = 0; j < N; ++j) {
            lfo_volume_texel(V, Po, Pd, M, N, i, j, v);
            for (uint32_t c = 0; c < V->C; ++c)
                out[(((size_t)(i - i0)) * N + j) * V->C + c] = (float)v[c];
        }
}

/* Direct render of the volume (the ground truth a light-field render of the  */
/* precomputed table approximates): each pixel's camera ray and front hit     */
/* h_o on S as above (FP32), then the same emission-absorption integral from   */
/* h_o along the ray's direction to the far intersection with S (one sample,   */
/* no jitter). out: [np][C] FP64, RGB (+ opacity 1 - T); misses store 0.       */
/* Returns the number of hits.                                                 */
int64_t lfo_volume_pixels(const lfo_volume *V, const float *views, const uint32_t *wh,
                          const uint32_t *pix, int64_t np, double *out)
{
    int64_t hits = 0;
    float O32[3] = {(float)V->O[0], (float)V->O[1], (float)V->O[2]};
    for (int64_t p = 0; p < np; ++p) {
        uint32_t v = pix[3 * p], x = pix[3 * p + 1], y = pix[3 * p + 2];
        const float *vw = views + 14 * v;
        float dir[3], ho[3], hd[3];
        for (uint32_t c = 0; c < V->C; ++c) out[p * V->C + c] = 0.0;
        lfo_camera_ray(vw, wh[2 * v], wh[2 * v + 1], x, y, dir);
        if (!lfo_intersect((float)V->R, O32, vw, dir, ho, hd)) continue;
        ++hits;
        double o[3] = {ho[0], ho[1], ho[2]}, d[3] = {dir[0], dir[1], dir[2]}, rgb[3], T;
        lfo_volume_ray(V, o, d, rgb, &T);
        for (int c = 0; c < 3; ++c) out[p * V->C + c] = rgb[c];
        if (V->C == 4) out[p * V->C + 3] = 1.0 - T;
    }
    return hits;
}
