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
// All three layers run on the tensor cores (tcgen05.mma kind::f16: FP16
// operands, FP32 accumulation in tensor memory); the CUDA cores only build the
// input rows and apply bias, ReLU and the border of each layer. Each layer is
// an implicit GEMM whose M is one row of 128 positions and whose K is 16 input
// values of one position (the 16 channels of a hidden layer; for the input,
// (R, G, B, hit, four zeros) of two neighbouring positions). One MMA takes one
// row of the layer below at one horizontal tap (or tap pair) dx and all three
// kernel rows: its N = 48 columns are the 16 output channels of the three
// output rows that this operand row feeds (through taps dy = 2, 1, 0), which
// lie side by side in tensor memory, so the MMAs accumulate each output row's
// nine taps in place and read every operand row once per dx. The operands are
// read straight from shared memory in their canonical layout (K-major, no
// swizzle: 16 contiguous bytes hold eight FP16 channels of one position), so a
// tap's shift is just another start address; the input's second K chunk is the
// next position (leading byte offset 16), so one MMA takes the taps dx and
// dx + 1 (dx = 0, 2; the weights of dx = 3 are zero). The third layer has 3
// output channels: its one MMA per operand row holds all three horizontal taps
// in N (16 columns per output row: 3 dx x 3 channels, 9 used) on the unshifted
// row, and its epilogue adds the taps dx = 1, 2 from the next positions' lanes.
//
// A CTA of 256 threads walks down one strip of 124 output columns of one view
// over a chunk of its rows. Every step adds kBand rows to each layer: it loads
// kBand input rows, and each layer computes the kBand rows whose 3 x 3
// neighbourhood in the layer below is now complete -- two rows behind the
// layer below (the input rows of a step are its rows t .. t + kBand - 1, the
// first layer's t - 2 .., the second's t - 4 .., the output's t - 6 ..). Each
// layer keeps its last rows in a ring in shared memory, so no row is computed
// twice except the six rows before the chunk; the rows of the first step
// that lie before it are computed from rows never loaded and are only ever
// read for outputs before the chunk, which are not stored. A CTA needs 95 KB
// of shared memory and 256 tensor-memory columns (half an SM's), so two share
// an SM and each runs its loads and epilogues while the other's MMAs run. The MMAs of each
// row produce 128 positions and the valid width shrinks by 2 per layer (130
// input positions, 128 first-layer, 126 second-layer, 124 output columns).
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "lf_device.cuh"
#include "lf_kernels.h"

namespace lfk {

constexpr int kPW = 124;                            // output columns per strip
constexpr int kBand = 6;                            // rows each layer adds per step
constexpr int kRow = 130;                           // positions stored per ring row
constexpr int kInRing = kBand + 3;                  // the kBand + 2 rows of layer 1's taps, and the row of the masks of the outputs
constexpr int kHRing = kBand + 2;                   // the kBand + 2 rows of the next layer's taps
constexpr int kInBytes = (kInRing * kRow + 1) * 16; // FP16 [row][position][8], one zero position after the last
constexpr int kHChunk = kHRing * kRow * 16;         // one 8-channel chunk of a hidden layer's ring
constexpr int kWGroup = 1536;                       // one MMA's 48 x 16 FP16 weights: [K chunk][n 48][8 k]
constexpr int kWBytes = 6 * kWGroup;                // layer 1: 2 tap pairs; layer 2: 3 taps; layer 3: 1
constexpr size_t kOffH1 = (kInBytes + 127) / 128 * 128, kOffH2 = kOffH1 + 2 * kHChunk, kOffW = kOffH2 + 2 * kHChunk;
constexpr size_t kPostSmem = kOffW + kWBytes;
constexpr int kBlocks = kBand + 4;                  // accumulator blocks: output rows -2 .. kBand + 1 of a layer
constexpr uint32_t kTmemCols = 256;                 // kBlocks blocks of 16 columns, rounded to a power of two
constexpr int kWaitTries = 1 << 22;                 // bounded wait on the MMAs (about a second at most)
constexpr int kPostThreads = 256;
constexpr int kRowsPerWarp = (kBand + 1) / 2;       // epilogue rows of a warp: two groups of four warps
constexpr int kBandPix = kBand * kRow;              // input positions loaded per step
constexpr int kLoadIters = (kBandPix + kPostThreads - 1) / kPostThreads;
static_assert(kBlocks * 16 <= (int)kTmemCols && kHRing >= 7 && kBand + 1 < kInRing, "ring and tensor-memory sizes");
static_assert(2 * (kPostSmem + 1024) <= 228 * 1024, "two CTAs per SM");
static_assert(kBand == 2 * kRowsPerWarp, "every warp takes kRowsPerWarp rows of a step");

// The kernel's parameters: the launch's views split into strips and chunks,
// the biases and the FP16 B operands of the MMAs (post_weight_image).
struct PostK {
    SphereK sphere;
    const float *in;
    float *out;
    uint32_t C, n_views;
    uint32_t vec4;                              // C == 4 and in, out 16-byte aligned
    uint32_t chunk_rows;                        // output rows per CTA
    uint32_t tile_prefix[kPostMaxViews + 1];    // CTAs before each view
    ViewK views[kPostMaxViews];                 // tiles_x = strips, tiles_y = chunks
    float bias[2 * kPostHidden + 3];            // b1, b2, b3
    uint4 wimg[kWBytes / 16];
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Ring slot of layer row t (t >= -2n: the first step's rows reach back to -6).
__device__ __forceinline__ int ring(int t, int n) { return (t + 2 * n) % n; }

// Shared-memory matrix descriptor of a K-major operand without swizzle: start
// address, leading byte offset (between the two 8-element K chunks), stride
// byte offset (between groups of 8 rows), the fixed version field 0b001.
__device__ __forceinline__ uint64_t kmajor_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, FP16 A and B, both
// K-major, N = 48, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | ((48u >> 3) << 17) | ((128u >> 4) << 24);

// D += A B (the accumulator's blocks start at zero: see tmem_zero16).
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 ::"r"(d_tmem), "l"(a), "l"(b), "r"(kIdesc), "r"(1u));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar));
}

// Waits (bounded) for phase `parity` of the mbarrier; false on timeout.
__device__ __forceinline__ bool wait_phase(uint32_t mbar, uint32_t parity)
{
    uint32_t done = 0;
    for (int it = 0; it < kWaitTries && !done; ++it)
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.b32 %0, 1, 0, p;\n\t}" : "=r"(done) : "r"(mbar), "r"(parity));
    return done != 0;
}

// The threads' shared-memory writes become visible to the MMAs, and tensor
// memory is handed over between the MMAs and the threads, across a barrier
// that also ANDs `ok` over the CTA.
__device__ __forceinline__ bool handover_sync(bool ok)
{
    asm volatile("tcgen05.fence::before_thread_sync;");
    asm volatile("fence.proxy.async.shared::cta;");
    ok = __syncthreads_and(ok) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;");
    return ok;
}

// Starts a load of 16 (or 4) consecutive accumulator columns of this warp's
// 32 lanes; tmem_wait completes every load started and ties their registers
// to it, so no use of them is scheduled before the wait.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&r)[4])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(taddr));
}

// Writes zeros to 16 accumulator columns of this warp's 32 lanes (completed
// by tcgen05.wait::st before the next handover).
__device__ __forceinline__ void tmem_zero16(uint32_t taddr)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};"
                 ::"r"(taddr), "r"(0u));
}

template <int N, int ROWS>
__device__ __forceinline__ void tmem_wait(uint32_t (&r)[ROWS][N])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int i = 0; i < ROWS; ++i)
#pragma unroll
        for (int k = 0; k < N; ++k) asm volatile("" : "+r"(r[i][k]));
}

__device__ __forceinline__ uint32_t pack_h2(float a, float b)
{
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// The colour as a network input: FP16, clamped to its finite range (a zero
// weight times an infinity would make NaN).
__device__ __forceinline__ float fp16_range(float c) { return fminf(fmaxf(c, -65504.0f), 65504.0f); }

// Epilogue of a 16-channel layer for its rows t0 .. t0 + kBand - 1 (row t0 + r
// in accumulator block r + 2, position = lane): bias, ReLU, zero where the
// pixel (xo + pos, yo + t0 + r) lies outside the view; FP16 into the ring of
// the next layer's operand, and the block back to zero for the next layer.
// Warp w reads tensor-memory lanes 32 (w % 4) .. + 31 of rows w / 4,
// w / 4 + 2, ... one row at a time (a batch of three rows' 48 registers spills).
__device__ __forceinline__ void epilogue16(uint32_t taddr, int t0, const float *bias, int xo, int yo, int W,
                                           int H, bool ok, uint8_t *dst)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, q = warp & 3, pos = 32 * q + lane;
    const int x = xo + pos;
#pragma unroll 1
    for (int r = warp >> 2; r < kBand; r += 2) {
        uint32_t h[1][16];
        const uint32_t blk = taddr + ((uint32_t)(32 * q) << 16) + 16 * (r + 2);
        tmem_ld16(blk, h[0]);
        tmem_wait<16, 1>(h);
        tmem_zero16(blk);
        const int y = yo + t0 + r;
        const bool inside = ok && x >= 0 && y >= 0 && x < W && y < H;
        uint32_t pk[8];
#pragma unroll
        for (int o = 0; o < 8; ++o) {
            const float a = fmaxf(__uint_as_float(h[0][2 * o]) + bias[2 * o], 0.0f);
            const float b = fmaxf(__uint_as_float(h[0][2 * o + 1]) + bias[2 * o + 1], 0.0f);
            pk[o] = inside ? pack_h2(a, b) : 0u;
        }
        uint8_t *row = dst + (ring(t0 + r, kHRing) * kRow + pos) * 16;
        *reinterpret_cast<uint4 *>(row) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        *reinterpret_cast<uint4 *>(row + kHChunk) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
    }
    asm volatile("tcgen05.wait::st.sync.aligned;");
}

// Issues one layer's MMAs: operand row rho (0 .. kBand + 1, the layer below's
// row t0 + rho, ring slot s0 + rho of a ring of n rows) at tap group gr into
// accumulator blocks rho .. rho + 2 (N = 48). GROUPS = 3: gr = dx; GROUPS = 2
// (the input): gr = the tap pair dx = 2 gr, 2 gr + 1; GROUPS = 1 (the third
// layer): the row unshifted, its three taps dx in the B operand's columns. The rows go 0, 3, 6, 1,
// 4, 7, 2, 5, so consecutive MMAs write disjoint blocks. The descriptors'
// start addresses advance in 16-byte units.
template <int GROUPS>
__device__ __forceinline__ void issue_layer(uint32_t taddr, uint64_t a0, uint64_t b0, int s0, int n)
{
    static_assert(kBand + 2 == 8, "row order");
    constexpr int kOrder[8] = {0, 3, 6, 1, 4, 7, 2, 5};
#pragma unroll
    for (int gr = 0; gr < GROUPS; ++gr) {
        const int dx = GROUPS == 3 ? gr : 2 * gr;
#pragma unroll
        for (int k = 0; k < kBand + 2; ++k) {
            const int rho = kOrder[k], sr = s0 + rho;
            const int slot = (sr >= n ? sr - n : sr) * kRow;
            mma_f16(taddr + 16 * rho, a0 + (uint64_t)(slot + dx), b0 + (uint64_t)(gr * (kWGroup / 16)));
        }
    }
}

// Loads the colours of input rows y_first .. y_first + kBand - 1 of the strip
// (pixels x0 - 3 + position) into c and returns their hit masks, one bit per
// pixel (a rolled loop, so the exact ray step is inlined once): the render's
// FP32 ray test, which the approximate ray settles for all but the pixels next
// to the silhouette. Pixels outside the view are 0 with mask 0.
__device__ __forceinline__ uint32_t load_input_band(const PostK &p, const ViewK &v, int x0, int y_first, int W,
                                                    int H, float3 (&c)[kLoadIters])
{
#pragma unroll
    for (int i = 0; i < kLoadIters; ++i) {
        const int k = threadIdx.x + i * kPostThreads, rr = k / kRow, x = x0 - 3 + (k - rr * kRow), y = y_first + rr;
        c[i] = make_float3(0.0f, 0.0f, 0.0f);
        if (k < kBandPix && x >= 0 && y >= 0 && x < W && y < H) {
            const float *in = p.in + (v.out_offset + (uint64_t)y * W + x) * p.C;
            if (p.vec4) {
                const float4 a = __ldg(reinterpret_cast<const float4 *>(in));
                c[i] = make_float3(a.x, a.y, a.z);
            } else {
                c[i] = make_float3(__ldg(in), __ldg(in + 1), __ldg(in + 2));
            }
        }
    }
    uint32_t mbits = 0;
#pragma unroll 1
    for (int i = 0; i < kLoadIters; ++i) {
        const int k = threadIdx.x + i * kPostThreads, rr = k / kRow;
        const int x = x0 - 3 + (k - rr * kRow), y = y_first + rr;
        if (k >= kBandPix || x < 0 || y < 0 || x >= W || y >= H) continue;
        int a = approx_mask(v, (uint32_t)x, (uint32_t)y);
        if (a < 0) {
            const float3 d = camera_dir(v, (uint32_t)x, (uint32_t)y);
            float3 ho, hd;
            a = intersect_sphere(p.sphere, v.eye, d, ho, hd) ? 1 : 0;
        }
        mbits |= (uint32_t)a << i;
    }
    return mbits;
}

__global__ void __launch_bounds__(kPostThreads, 2) post_filter_kernel(const __grid_constant__ PostK p)
{
    extern __shared__ __align__(128) uint8_t sm[];
    uint8_t *s_in = sm, *s_h1 = sm + kOffH1, *s_h2 = sm + kOffH2, *s_w = sm + kOffW;
    __shared__ uint32_t s_tile[3];
    __shared__ uint32_t s_taddr;
    __shared__ __align__(8) uint64_t s_mbar;
    __shared__ float s_edge[2][kRowsPerWarp][4][9];   // third layer: lanes 0, 1 of each 32 positions
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t mbar = smem_addr(&s_mbar);
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
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_taddr)),
                     "n"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // the rings start at zero: positions 128, 129 of the hidden rows and the
    // position after the input ring are read (by taps of zero weight, or for
    // positions not stored) and never written
    for (int k = tid; k < (int)(kOffW / 16); k += kPostThreads)
        reinterpret_cast<uint4 *>(sm)[k] = make_uint4(0u, 0u, 0u, 0u);
    for (int k = tid; k < kWBytes / 16; k += kPostThreads) reinterpret_cast<uint4 *>(s_w)[k] = p.wimg[k];
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t taddr = s_taddr;
    const int q = warp & 3, g = warp >> 2, pos = 32 * q + lane;
    // the accumulator blocks of the output rows start at zero; each epilogue
    // returns its blocks to zero (the MMAs only accumulate)
    for (int r = g; r < kBand; r += 2) tmem_zero16(taddr + ((uint32_t)(32 * q) << 16) + 16 * (r + 2));
    asm volatile("tcgen05.wait::st.sync.aligned;");
    bool ok = handover_sync(true);
    const ViewK &v = p.views[s_tile[0]];
    const int W = (int)v.width, H = (int)v.height;
    const int x0 = (int)s_tile[1] * kPW, ya = (int)(s_tile[2] * p.chunk_rows);
    const int rows = min((int)p.chunk_rows, H - ya);
    const int steps = (rows + 6 + kBand - 1) / kBand;
    const int xout = x0 + pos;
    const bool col_ok = pos < kPW && xout < W;
    uint32_t phase = 0;

    const uint64_t a_in = kmajor_desc(smem_addr(s_in), 16, 128), a_h1 = kmajor_desc(smem_addr(s_h1), kHChunk, 128),
                   a_h2 = kmajor_desc(smem_addr(s_h2), kHChunk, 128),
                   b_w1 = kmajor_desc(smem_addr(s_w), 768, 128),
                   b_w2 = kmajor_desc(smem_addr(s_w + 2 * kWGroup), 768, 128),
                   b_w3 = kmajor_desc(smem_addr(s_w + 5 * kWGroup), 768, 128);
    float3 c[kLoadIters];
    uint32_t mbits = load_input_band(p, v, x0, ya - 3, W, H, c);

    for (int j = 0; j < steps; ++j) {
        const int tin = j * kBand, t1 = tin - 2, t2 = tin - 4, t3 = tin - 6;
        // the previous step's last epilogue has read the masks of the rows replaced now
        ok = __syncthreads_and(ok) != 0;
        // input rows tin .. tin + kBand - 1, FP16 (R, G, B, hit, 0, 0, 0, 0)
#pragma unroll
        for (int i = 0; i < kLoadIters; ++i) {
            const int k = tid + i * kPostThreads, rr = k / kRow, tx = k - rr * kRow;
            if (k >= kBandPix) break;
            const float m = (float)((mbits >> i) & 1u);
            *reinterpret_cast<uint4 *>(s_in + (ring(tin + rr, kInRing) * kRow + tx) * 16) =
                make_uint4(pack_h2(fp16_range(c[i].x), fp16_range(c[i].y)), pack_h2(fp16_range(c[i].z), m), 0u, 0u);
        }
        ok = handover_sync(ok);

        // layer 1: rows t1 .. t1 + kBand - 1 from input rows t1 .. t1 + kBand + 1
        if (tid == 0 && ok) {
            issue_layer<2>(taddr, a_in, b_w1, ring(t1, kInRing), kInRing);
            mma_commit(mbar);
        }
        // while the MMAs run: the next step's input rows and masks, and the FP32
        // colour of this step's output pixels for the residual
        if (j + 1 < steps) mbits = load_input_band(p, v, x0, ya - 3 + tin + kBand, W, H, c);
        float4 res[kRowsPerWarp];
#pragma unroll
        for (int i = 0; i < kRowsPerWarp; ++i) {
            const int t = t3 + g + 2 * i;
            res[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (g + 2 * i < kBand && col_ok && t >= 0 && t < rows) {
                const float *in = p.in + (v.out_offset + (uint64_t)(ya + t) * W + xout) * p.C;
                if (p.vec4) {
                    res[i] = __ldg(reinterpret_cast<const float4 *>(in));
                } else {
                    res[i].x = __ldg(in);
                    res[i].y = __ldg(in + 1);
                    res[i].z = __ldg(in + 2);
                    if (p.C == 4) res[i].w = __ldg(in + 3);
                }
            }
        }
        bool done = ok && wait_phase(mbar, phase);
        phase ^= ok ? 1u : 0u;
        asm volatile("tcgen05.fence::after_thread_sync;");
        epilogue16(taddr, t1, p.bias, x0 - 2, ya - 2, W, H, done, s_h1);
        ok = handover_sync(done);

        // layer 2: rows t2 .. from first-layer rows t2 .. t2 + kBand + 1
        if (tid == 0 && ok) {
            issue_layer<3>(taddr, a_h1, b_w2, ring(t2, kHRing), kHRing);
            mma_commit(mbar);
        }
        done = ok && wait_phase(mbar, phase);
        phase ^= ok ? 1u : 0u;
        asm volatile("tcgen05.fence::after_thread_sync;");
        epilogue16(taddr, t2, p.bias + kPostHidden, x0 - 1, ya - 1, W, H, done, s_h2);
        ok = handover_sync(done);

        // layer 3: output rows t3 .. from second-layer rows t3 .. t3 + kBand + 1, one MMA per
        // operand row: its 16 columns per output row are (dx, channel), 9 used, unshifted
        if (tid == 0 && ok) {
            issue_layer<1>(taddr, a_h2, b_w3, ring(t3, kHRing), kHRing);
            mma_commit(mbar);
        }
        done = ok && wait_phase(mbar, phase);
        phase ^= ok ? 1u : 0u;
        ok = done;
        asm volatile("tcgen05.fence::after_thread_sync;");
        // The third layer's accumulator row of position p holds, in column
        // 3 dx + c, channel c of tap dx applied at position p; the output at p
        // sums column 3 dx + c of position p + dx (dx = 0, 1, 2). Within a warp
        // the shifted columns come by shuffles; lanes 30 and 31 take them from
        // lanes 0 and 1 of the next 32 positions through shared memory (a
        // barrier of the row group's four warps). Then the bias, added to the
        // input colour of hit pixels; NaN if the MMAs never completed; the
        // blocks back to zero for the next step's first layer.
#pragma unroll
        for (int i = 0; i < kRowsPerWarp; ++i) {
            const int r = g + 2 * i, t = t3 + r;
            uint32_t hv[1][16];
            const uint32_t blk = taddr + ((uint32_t)(32 * q) << 16) + 16 * (r + 2);
            tmem_ld16(blk, hv[0]);
            tmem_wait<16, 1>(hv);
            tmem_zero16(blk);
            float f[9];
#pragma unroll
            for (int c = 0; c < 9; ++c) f[c] = __uint_as_float(hv[0][c]);
            float *edge = s_edge[g][i][q];
            if (lane == 0) {
#pragma unroll
                for (int c = 3; c < 9; ++c) edge[c] = f[c];
            } else if (lane == 1) {
#pragma unroll
                for (int c = 0; c < 3; ++c) edge[c] = f[6 + c];
            }
            if (g == 0)
                asm volatile("bar.sync 1, 128;" ::: "memory");
            else
                asm volatile("bar.sync 2, 128;" ::: "memory");
            float o1[3], o2[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                o1[c] = __shfl_down_sync(0xffffffffu, f[3 + c], 1);
                o2[c] = __shfl_down_sync(0xffffffffu, f[6 + c], 2);
            }
            if (q < 3 && lane >= 30) {
                const float *next = s_edge[g][i][q + 1];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    o1[c] = lane == 31 ? next[3 + c] : o1[c];
                    o2[c] = lane == 31 ? next[c] : next[6 + c];
                }
            }
            if (!col_ok || t < 0 || t >= rows) continue;
            const __half2 bm = *reinterpret_cast<const __half2 *>(s_in + (ring(t + 3, kInRing) * kRow + pos + 3) * 16 + 4);
            const bool hit = __high2float(bm) != 0.0f;
            float a3[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) a3[c] = __fadd_rn(__fadd_rn(f[c], o1[c]), o2[c]) + p.bias[2 * kPostHidden + c];
            float4 o;
            o.x = hit ? res[i].x + a3[0] : 0.0f;
            o.y = hit ? res[i].y + a3[1] : 0.0f;
            o.z = hit ? res[i].z + a3[2] : 0.0f;
            o.w = res[i].w;
            if (!done) o.x = o.y = o.z = __int_as_float(0x7fc00000);
            float *out = p.out + (v.out_offset + (uint64_t)(ya + t) * W + xout) * p.C;
            if (p.vec4) {
                *reinterpret_cast<float4 *>(out) = o;
            } else {
                out[0] = o.x;
                out[1] = o.y;
                out[2] = o.z;
                if (p.C == 4) out[3] = o.w;
            }
        }
        asm volatile("tcgen05.wait::st.sync.aligned;");
        asm volatile("tcgen05.fence::before_thread_sync;");
    }
    ok = handover_sync(ok);
    // after a timeout: one more bounded wait for the MMAs still in flight (the
    // last commit, of parity phase ^ 1) before their tensor memory is freed
    if (!ok) wait_phase(mbar, phase ^ 1u);
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "n"(kTmemCols));
}

// The B operands of the kernel's MMAs, FP16, [group][K chunk c][n][k] with
// n = 16 s + o (output channel o of the output row fed through kernel row
// dy = 2 - s): layer 1 (groups 0, 1: the tap pair dx = 2 gr + c, input
// channel k < 4, zero for dx = 3 and k >= 4), layer 2 (groups 2..4: tap
// dx = group, input channel 8 c + k) and layer 3 (group 5: column o = 3 dx +
// output channel, all three taps dx, zero for o >= 9).
static void post_weight_image(const float *w, uint4 *img)
{
    uint16_t *h = reinterpret_cast<uint16_t *>(img);
    for (int gr = 0; gr < 6; ++gr)
        for (int c = 0; c < 2; ++c)
            for (int n = 0; n < 48; ++n)
                for (int k = 0; k < 8; ++k) {
                    const int s = n >> 4, o = n & 15, dy = 2 - s;
                    float x = 0.0f;
                    if (gr < 2) {
                        const int dx = 2 * gr + c;
                        if (k < 4 && dx < 3) x = w[kPostW1 + ((o * 4 + k) * 3 + dy) * 3 + dx];
                    } else if (gr < 5) {
                        x = w[kPostW2 + ((o * kPostHidden + 8 * c + k) * 3 + dy) * 3 + (gr - 2)];
                    } else if (o < 9) {
                        const int dx = o / 3, ch = o - 3 * dx;
                        x = w[kPostW3 + ((ch * kPostHidden + 8 * c + k) * 3 + dy) * 3 + dx];
                    }
                    const __half hx = __float2half_rn(x);
                    memcpy(&h[(gr * kWGroup + c * 768 + n * 16 + k * 2) / 2], &hx, 2);
                }
}

// Strips of 124 columns, chunks of chunk_rows rows (a multiple of kBand): the
// chunks are as short as keeps the CTAs within one wave of the resident slots
// (two per SM), at most 32 views of at most 65536 x 65536 pixels (fewer than
// 2^31 CTAs).
cudaError_t launch_post_filter(const PostParams &p0, cudaStream_t st)
{
    static thread_local PostK p;
    static thread_local int cached_dev = -1, cached_slots = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev != cached_dev) {
        e = cudaFuncSetAttribute(post_filter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPostSmem);
        if (e != cudaSuccess) return e;
        // all of the unified L1 as shared memory: room for two CTAs per SM
        e = cudaFuncSetAttribute(post_filter_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        // resident CTAs per SM from the kernel's resources: shared memory
        // (dynamic, static and the per-CTA reservation), registers, threads and
        // tensor-memory columns (512 per SM, which the occupancy API does not
        // count)
        int sms = 0, smem_sm = 0, rsv = 0, regs_sm = 0, threads_sm = 0;
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, post_filter_kernel);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&threads_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
        if (e != cudaSuccess) return e;
        const int smem_cta = (int)kPostSmem + (int)fa.sharedSizeBytes + rsv;
        const int regs_cta = ((fa.numRegs + 7) / 8 * 8) * kPostThreads;
        int per_sm = 512 / (int)kTmemCols;
        per_sm = std::min(per_sm, smem_sm / smem_cta);
        per_sm = std::min(per_sm, regs_sm / std::max(regs_cta, 1));
        per_sm = std::min(per_sm, threads_sm / kPostThreads);
        cached_slots = sms * std::max(per_sm, 1);
        cached_dev = dev;
    }
    p.sphere = p0.sphere;
    p.in = p0.in;
    p.out = p0.out;
    p.C = p0.C;
    p.n_views = p0.n_views;
    p.vec4 = p.C == 4 && ((uintptr_t)p.in % 16) == 0 && ((uintptr_t)p.out % 16) == 0;
    for (int k = 0; k < kPostHidden; ++k) {
        p.bias[k] = p0.w[kPostB1 + k];
        p.bias[kPostHidden + k] = p0.w[kPostB2 + k];
    }
    for (int k = 0; k < 3; ++k) p.bias[2 * kPostHidden + k] = p0.w[kPostB3 + k];
    // the FP16 layout of the weights, rebuilt only when they change (the
    // conversion costs more host time than the kernel's launch)
    static thread_local float last_w[kPostWeights];
    static thread_local bool have_image = false;
    if (!have_image || memcmp(last_w, p0.w, sizeof last_w) != 0) {
        post_weight_image(p0.w, p.wimg);
        memcpy(last_w, p0.w, sizeof last_w);
        have_image = true;
    }
    uint64_t bands = 0, max_vb = 0, ctas = 0;
    for (uint32_t v = 0; v < p.n_views; ++v) {
        p.views[v] = p0.views[v];
        p.views[v].tiles_x = (p.views[v].width + kPW - 1) / kPW;
        const uint64_t vb = (p.views[v].height + kBand - 1) / kBand;
        bands += (uint64_t)p.views[v].tiles_x * vb;
        max_vb = vb > max_vb ? vb : max_vb;
    }
    if (bands == 0) return cudaSuccess;
    uint64_t per_chunk = (bands + cached_slots - 1) / cached_slots;
    for (; per_chunk < max_vb; ++per_chunk) {
        ctas = 0;
        for (uint32_t v = 0; v < p.n_views; ++v)
            ctas += (uint64_t)p.views[v].tiles_x * ((p.views[v].height + kBand * per_chunk - 1) / (kBand * per_chunk));
        if (ctas <= (uint64_t)cached_slots) break;
    }
    p.chunk_rows = (uint32_t)(per_chunk * kBand);
    ctas = 0;
    for (uint32_t v = 0; v < p.n_views; ++v) {
        p.views[v].tiles_y = (p.views[v].height + p.chunk_rows - 1) / p.chunk_rows;
        p.tile_prefix[v] = (uint32_t)ctas;
        ctas += (uint64_t)p.views[v].tiles_x * p.views[v].tiles_y;
    }
    p.tile_prefix[p.n_views] = (uint32_t)ctas;
    post_filter_kernel<<<(unsigned)ctas, kPostThreads, kPostSmem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace lfk
