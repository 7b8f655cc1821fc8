// fv_closure.cu -- the level-1 solver with the learned closure of the level-4 moments.
//
// Model (the paper's model hierarchy, Eq. (sme) / Sec. 3.4, with a learned per-cell "material
// closure" for the truncated moments): the level-4 system restricted to the rows of the level-1
// variables (h, h alpha_0, h beta_0, h alpha_1, h beta_1).  The moments alpha_2..4, beta_2..4 are
// not transported: at every stage input a per-cell MLP predicts them from
// (h, u_m, v_m, alpha_1, beta_1, lambda).  Fluxes, the nonconservative product (path integral over
// the closed profiles), the Newtonian source and the wave speed use the closed level-4 profile; the
// bottom stress is implicit in the two prognostic moments with the closed ones frozen.
//
// The MLP (6 -> 64 -> 64 -> 6, tanh-form GELU, BF16 weights and layer inputs, FP32 accumulation)
// runs inside the stage kernel on the tensor cores: the warp that marches a row holds 32 cells, the
// batch of two m16 tiles of mma.sync.m16n8k16 BF16 operations; the accumulator fragments of layer 1
// and 2 are re-packed in registers as the A operands of the next layer, and the weight fragments sit
// pre-swizzled in shared memory.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "closure_stage.cuh"
#include "f32x2.cuh"
#include "fv_common.cuh"
#include "tcgen05.cuh"
#include "zoomy_internal.h"
#include "zoomy_kernels.h"

namespace zoomy {

// weight fragments in the layout of the mma.sync B operand (per lane), then FP32 biases
struct ClosureDev {
    uint32_t w1[8][32];     // layer 1: n-tile, lane -> b0 (rows 2t,2t+1 of the padded 16-row W1)
    uint2 w2[4][8][32];     // layer 2: k-chunk, n-tile, lane -> (b0, b1)
    uint2 w3[4][32];        // layer 3: k-chunk, lane -> (b0, b1) (outputs padded 6 -> 8)
    float b1[64], b2[64], b3[8];
    float in_scale[6], out_scale[6];
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __float22bfloat162_rn(make_float2(lo, hi));
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ void mma_bf16(float *d, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float tanh_approx(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// GELU, tanh form: z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3)))
__device__ __forceinline__ float gelu(float z)
{
    const float u = 0.7978845608028654f * z * fmaf(0.044715f, z * z, 1.0f);
    const float hz = 0.5f * z;
    return fmaf(hz, tanh_approx(u), hz);
}

// GELU of a pair in terms of h = z/2 without the SFU: GELU(z) = h + h tanh(h (2c + 8 * 0.044715 c
// h^2)) = h + E(h^2), with E(s) approximated by s P(s), P of degree 6, fitted (least squares with
// Lawson's reweighting towards the minimax error) on Chebyshev nodes of s in [0, 4]; for |h| > 2 the
// tanh is 1 to 4e-5 and E = |h|.  Largest error against the tanh form: 2.1e-4 absolute, below the
// error of tanh.approx.f32 there (|h| 2^-11) and of the BF16 rounding that follows.
__device__ __forceinline__ F2 gelu_poly2(F2 h)
{
    const F2 s = h * h;
    F2 p = fma2(F2(3.9228369132615626e-04f), s, F2(-6.8186875432729721e-03f));
    p = fma2(p, s, F2(5.0590563565492630e-02f));
    p = fma2(p, s, F2(-2.1221332252025604e-01f));
    p = fma2(p, s, F2(5.6576108932495117e-01f));
    p = fma2(p, s, F2(-1.0342786312103271e+00f));
    p = fma2(p, s, F2(1.5909816026687622e+00f));
    const F2 e = s * p;
    return h + F2(s.x() > 4.0f ? fabsf(h.x()) : e.x(), s.y() > 4.0f ? fabsf(h.y()) : e.y());
}

// Warp-cooperative MLP of the 32 cells held by the lanes (one cell per lane).
// xs / ys: this warp's shared tiles (32 x 4 u32 features, 32 x 8 floats outputs).
__device__ __forceinline__ void mlp_warp(const ClosureDev *net, const float *feat, float *out, uint32_t *xs,
                                         float *ys, int lane)
{
    const int g = lane >> 2, t = lane & 3;
    // features -> BF16 pairs in this lane's row of the input tile (columns 6, 7 are zero padding)
    xs[lane * 4 + 0] = pack_bf16(feat[0] * net->in_scale[0], feat[1] * net->in_scale[1]);
    xs[lane * 4 + 1] = pack_bf16(feat[2] * net->in_scale[2], feat[3] * net->in_scale[3]);
    xs[lane * 4 + 2] = pack_bf16(feat[4] * net->in_scale[4], feat[5] * net->in_scale[5]);
    xs[lane * 4 + 3] = 0u;
    __syncwarp();
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        const uint32_t a0 = xs[(mt * 16 + g) * 4 + t], a1 = xs[(mt * 16 + g + 8) * 4 + t];
        // layer 1: [16 x 16] x [16 x 64]
        float c1[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const float2 bb = *reinterpret_cast<const float2 *>(&net->b1[nt * 8 + 2 * t]);
            c1[nt][0] = bb.x;
            c1[nt][1] = bb.y;
            c1[nt][2] = bb.x;
            c1[nt][3] = bb.y;
            mma_bf16(c1[nt], a0, a1, 0u, 0u, net->w1[nt][lane], 0u);
        }
        uint32_t A[4][4];
#pragma unroll
        for (int kc = 0; kc < 4; ++kc) {
            A[kc][0] = pack_bf16(gelu(c1[2 * kc][0]), gelu(c1[2 * kc][1]));
            A[kc][1] = pack_bf16(gelu(c1[2 * kc][2]), gelu(c1[2 * kc][3]));
            A[kc][2] = pack_bf16(gelu(c1[2 * kc + 1][0]), gelu(c1[2 * kc + 1][1]));
            A[kc][3] = pack_bf16(gelu(c1[2 * kc + 1][2]), gelu(c1[2 * kc + 1][3]));
        }
        // layer 2: [16 x 64] x [64 x 64]
        float c2[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const float2 bb = *reinterpret_cast<const float2 *>(&net->b2[nt * 8 + 2 * t]);
            c2[nt][0] = bb.x;
            c2[nt][1] = bb.y;
            c2[nt][2] = bb.x;
            c2[nt][3] = bb.y;
#pragma unroll
            for (int kc = 0; kc < 4; ++kc) {
                const uint2 w = net->w2[kc][nt][lane];
                mma_bf16(c2[nt], A[kc][0], A[kc][1], A[kc][2], A[kc][3], w.x, w.y);
            }
        }
#pragma unroll
        for (int kc = 0; kc < 4; ++kc) {
            A[kc][0] = pack_bf16(gelu(c2[2 * kc][0]), gelu(c2[2 * kc][1]));
            A[kc][1] = pack_bf16(gelu(c2[2 * kc][2]), gelu(c2[2 * kc][3]));
            A[kc][2] = pack_bf16(gelu(c2[2 * kc + 1][0]), gelu(c2[2 * kc + 1][1]));
            A[kc][3] = pack_bf16(gelu(c2[2 * kc + 1][2]), gelu(c2[2 * kc + 1][3]));
        }
        // layer 3: [16 x 64] x [64 x 8]
        float c3[4];
        const float2 bb = *reinterpret_cast<const float2 *>(&net->b3[2 * t]);
        c3[0] = bb.x;
        c3[1] = bb.y;
        c3[2] = bb.x;
        c3[3] = bb.y;
#pragma unroll
        for (int kc = 0; kc < 4; ++kc) {
            const uint2 w = net->w3[kc][lane];
            mma_bf16(c3, A[kc][0], A[kc][1], A[kc][2], A[kc][3], w.x, w.y);
        }
        ys[(mt * 16 + g) * 8 + 2 * t] = c3[0];
        ys[(mt * 16 + g) * 8 + 2 * t + 1] = c3[1];
        ys[(mt * 16 + g + 8) * 8 + 2 * t] = c3[2];
        ys[(mt * 16 + g + 8) * 8 + 2 * t + 1] = c3[3];
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 6; ++j) out[j] = ys[lane * 8 + j] * net->out_scale[j];
    __syncwarp();
}

// Wave speed of the closed profile of a cell: state x, predictions p (the level-4 bound R3).
__device__ __forceinline__ float closed_speed(const float *x, const float *p, float g, float hdry)
{
    SideC r;
    float ih;
    make_side_c(r, x, 0.0f, p, false, false, g, hdry, ih);
    return r.sc;
}

__device__ __forceinline__ void features(const float *q, float lambda, float hdry, float *f)
{
    const float h = q[0];
    const float ih = h > hdry ? __frcp_rn(h) : 0.0f;
    f[0] = h;
    f[1] = q[1] * ih;
    f[2] = q[2] * ih;
    f[3] = q[3] * ih;
    f[4] = q[4] * ih;
    f[5] = lambda;
}

// The FV stage of the closed model (closure_stage.cuh): one warp per CTA marches a 30-column strip.
template <int STAGE>
__global__ void __launch_bounds__(32) k_stage_closure(ClosureArgs ca)
{
    const StageArgs<float> &a = ca.s;
    pdl_enter();  // programmatic dependent launch: the prediction of this stage's input first
    if (*(volatile unsigned int *)&a.ctl->status) return;
    float dt;
    if (!step_dt(a, dt)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&a.ctl->status, DEV_NOWAVE);
        return;
    }
    if (STAGE == 1 && blockIdx.x == 0 && threadIdx.x == 0) step_bookkeeping(a, dt);
    unsigned flag = 0;
    march_strip_c<STAGE>(ca, blockIdx.x % a.nstrips, blockIdx.x / a.nstrips, threadIdx.x, dt, flag);
    if (STAGE == 2 && flag) atomicOr(&a.ctl->status, flag);
}

// The closure of every cell of the stage input X: predicted moments into ca.pred, and (WS) the
// maximum wave speed of the closed profiles into the control slot a.slot_out, plus the
// non-finite / negative-depth flags of X.  The stage kernels then read the predictions of their
// cells and of the halo cells.
template <bool WS>
__global__ void __launch_bounds__(128) k_closure_predict(ClosureArgs ca)
{
    const StageArgs<float> &a = ca.s;
    __shared__ ClosureDev net;
    __shared__ uint32_t xs_all[4][32 * 4];
    __shared__ float ys_all[4][32 * 8];
    {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(ca.net);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&net);
        for (int i = threadIdx.x; i < (int)(sizeof(ClosureDev) / 4); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    if (*(volatile unsigned int *)&a.ctl->status) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t nc = (int64_t)a.nx * a.ny;
    float smax = 0.0f;
    unsigned flag = 0;
    // warps stride over groups of 32 cells (the MLP needs all lanes)
    for (int64_t base = ((int64_t)blockIdx.x * 4 + warp) * 32; base < nc; base += (int64_t)gridDim.x * 4 * 32) {
        const int64_t i = base + lane;
        const int64_t ic = i < nc ? i : nc - 1;
        float x[CL_NV];
#pragma unroll
        for (int v = 0; v < CL_NV; ++v) x[v] = __ldg(a.X + v * a.ld + ic);
        float f[6], p[6];
        features(x, ca.lambda, a.hdry, f);
        mlp_warp(&net, f, p, xs_all[warp], ys_all[warp], lane);
        if (i < nc) {
#pragma unroll
            for (int j = 0; j < 6; ++j) ca.pred[j * ca.pstride + i] = p[j];
        }
        if (WS) {
            const float s = closed_speed(x, p, a.g, a.hdry);
            if (i < nc) {
                if (!(s <= 3.0e38f)) flag |= DEV_NAN;
                if (!(x[0] >= 0.0f)) flag |= (x[0] < 0.0f) ? DEV_NEGDEPTH : DEV_NAN;
                smax = (s > smax || s != s) ? s : smax;
            }
        }
    }
    if (WS) {
        if (flag) atomicOr(&a.ctl->status, flag);
        reduce_smax<float>(a.ctl, a.slot_out, smax);
    }
}

// The closure MLP alone on n feature vectors (SoA [6][n] -> [6][n]), same device code as in the stage.
__global__ void __launch_bounds__(128) k_closure_eval(const ClosureDev *gnet, const float *feat, float *out, int64_t n)
{
    __shared__ ClosureDev net;
    __shared__ uint32_t xs_all[4][32 * 4];
    __shared__ float ys_all[4][32 * 8];
    {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(gnet);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&net);
        for (int i = threadIdx.x; i < (int)(sizeof(ClosureDev) / 4); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t base = ((int64_t)blockIdx.x * 4 + warp) * 32; base < n; base += (int64_t)gridDim.x * 4 * 32) {
        const int64_t i = base + lane;
        const int64_t ic = i < n ? i : n - 1;
        float f[6], y[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) f[j] = feat[j * n + ic];
        mlp_warp(&net, f, y, xs_all[warp], ys_all[warp], lane);
        if (i < n) {
#pragma unroll
            for (int j = 0; j < 6; ++j) out[j * n + i] = y[j];
        }
    }
}

// ------------------------------------------------------------------------------------------
// The same network on the 5th-generation tensor cores: a CTA of 4 warps takes 128 cells per tile
// (cell i of the tile = row i of the MMA = tensor-memory lane i, owned by thread i).  Per layer one
// thread issues tcgen05.mma (M = 128, N = 64 or 16, K = 16 per instruction) from BF16 operands in
// shared memory into FP32 accumulators in tensor memory; the threads read their row back with
// tcgen05.ld, add the bias, apply the GELU and write the BF16 row of the next layer's A operand.
// Every completion wait is bounded; a wait that gives up raises DEV_TIMEOUT, waits once more for
// the outstanding MMAs and frees the tensor memory before returning.
// ------------------------------------------------------------------------------------------

// Weights in the K-major no-swizzle operand layout (B operands are the transposed weights).
// B3 comes first so that even a mis-read LBO/SBO pair would stay inside the structure.
// The biases ride on the tensor core: columns 6 and 7 of every layer-1 input row hold 1.0, and
// the matching columns of B1 / Bb2 / Bb3 hold the bias split into two BF16 parts (hi + lo, ~16
// bits), so a K = 16 step with the layer-1 tile as A adds the bias of layers 2 and 3.  Layers 1
// and 2 are scaled by 1/2 (exact in BF16): the accumulator holds z/2, and the GELU
// z/2 (1 + tanh(c (z + 0.044715 z^3))) is evaluated in terms of z/2.
struct ClosureTC {
    uint16_t B3[16 * 64];   // W3^T: 6 outputs (padded to 16) x 64
    uint16_t Bb3[16 * 16];  // b3 in columns 6, 7
    uint16_t B1[64 * 16];   // W1^T / 2 (6 inputs, padded to 16), b1 / 2 in columns 6, 7
    uint16_t B2[64 * 64];   // W2^T / 2
    uint16_t Bb2[64 * 16];  // b2 / 2 in columns 6, 7
    float in_scale[8], out_scale[8];
};
static_assert(sizeof(ClosureTC) % 16 == 0, "ClosureTC is copied in 16-byte words");

// Tiles in flight per CTA.  With one, a CTA's epilogue waits for its own MMA and the other CTAs on
// the SM fill that time (6 CTAs of 32 KB and 80 registers per thread, 24 warps per SM); with two,
// each tile's epilogue overlaps the other tile's MMA (4 CTAs of 53 KB, 128 registers, 16 warps).
constexpr int TC_TILES = 1;
constexpr int TC_CHUNK = 16;  // accumulator columns read back per tensor-memory load batch
// Every TC_POLY_EVERY-th pair of hidden activations takes its GELU from gelu_poly2 on the FMA pipe
// instead of two tanh.approx on the SFU (0: none), balancing the two pipes.
constexpr int TC_POLY_EVERY = 3;

struct TCSmem {
    ClosureTC net;
    alignas(128) uint16_t A1[TC_TILES][128 * 16];  // layer-1 input tiles (K = 16), one per tile in flight
    alignas(128) uint16_t A2[TC_TILES][128 * 64];  // layer-2 and layer-3 input tiles (K = 64)
    uint64_t bar[TC_TILES];
    uint32_t tmem;
};

// Each tile owns a 64-column accumulator region that serves its three layers in turn (a layer's
// accumulator is read back completely before the next MMA into it is issued).
constexpr uint32_t TC_COLS = 64 * TC_TILES;
constexpr long long TC_WAIT = 2000000000LL;    // ~1 s at 2 GHz
constexpr int TC_DYN_SMEM = (int)sizeof(TCSmem);
constexpr int TC_THREADS = 128;
constexpr int TC_CTAS_PER_SM = TC_TILES == 1 ? 6 : 4;
constexpr uint32_t TC_IDESC64 = tc::idesc_bf16_f32(128, 64);
constexpr uint32_t TC_IDESC16 = tc::idesc_bf16_f32(128, 16);

// MODE 0: predict from the stage input (ca.s.X) into ca.pred; MODE 1: the same plus the closed wave
// speed into slot a.slot_out; MODE 2: evaluate feat [6][n] (unscaled features) into out [6][n].
// Thread r owns row r of both tiles in flight (tensor-memory lane r).
template <int MODE>
__global__ void __launch_bounds__(TC_THREADS, TC_CTAS_PER_SM) k_closure_tc(ClosureArgs ca, const ClosureTC *gnet,
                                                                           const float *feat, float *out, int64_t n)
{
    extern __shared__ __align__(1024) uint8_t tc_smem[];  // sizeof(TCSmem) bytes (above the static limit)
    TCSmem &sm = *reinterpret_cast<TCSmem *>(tc_smem);
    const StageArgs<float> &a = ca.s;
    const int tid = threadIdx.x, warp = tid >> 5;
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(gnet);
        uint4 *dst = reinterpret_cast<uint4 *>(&sm.net);
        for (int i = tid; i < (int)(sizeof(ClosureTC) / 16); i += TC_THREADS) dst[i] = src[i];
        // columns 8..15 of the layer-1 inputs are zero padding for every tile
#pragma unroll
        for (int b = 0; b < TC_TILES; ++b)
            *reinterpret_cast<uint4 *>(&sm.A1[b][tc::kmajor_index(tid, 8, 16)]) = make_uint4(0u, 0u, 0u, 0u);
    }
    if (warp == 0) tc::tmem_alloc(&sm.tmem, TC_COLS);
    if (tid == 0) {
#pragma unroll
        for (int b = 0; b < TC_TILES; ++b) tc::mbar_init(&sm.bar[b], 1);
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = sm.tmem;
    const uint32_t tlane = (uint32_t)(warp * 32) << 16;  // this warp's 32 lanes
    // inside a step the launch is programmatic: the set-up above overlaps the previous kernel, whose
    // results (the stage output, the control block) are read only after this
    if (MODE != 2) pdl_enter();
    const bool skip = MODE != 2 && __syncthreads_or(tid == 0 && *(volatile unsigned int *)&a.ctl->status != 0u);
    const uint32_t sb1 = tc::smem_u32(sm.net.B1), sb2 = tc::smem_u32(sm.net.B2), sb3 = tc::smem_u32(sm.net.B3);
    const uint32_t sbb2 = tc::smem_u32(sm.net.Bb2), sbb3 = tc::smem_u32(sm.net.Bb3);
    const int64_t nc = MODE == 2 ? n : (int64_t)a.nx * a.ny;
    const int64_t ntiles = (nc + 127) / 128;
    uint32_t phase[TC_TILES];
#pragma unroll
    for (int b = 0; b < TC_TILES; ++b) phase[b] = 0u;
    bool failed = false;
    float smax = 0.0f;
    unsigned flag = 0;
    float x[TC_TILES][CL_NV];  // the stage input of this thread's cells (wave speed)

    auto load = [&](int64_t tile, float *dst) {
        const int64_t i = tile * 128 + tid;
        const int64_t ic = i < nc ? i : nc - 1;
#pragma unroll
        for (int v = 0; v < (MODE == 2 ? 6 : CL_NV); ++v)
            dst[v] = MODE == 2 ? __ldg(feat + v * n + ic) : __ldg(a.X + v * a.ld + ic);
    };
    // features of this thread's cell -> BF16 row of the layer-1 tile b
    auto prep = [&](int b, const float *in) {
        float f[6];
        if (MODE == 2) {
#pragma unroll
            for (int j = 0; j < 6; ++j) f[j] = in[j];
        } else {
#pragma unroll
            for (int v = 0; v < CL_NV; ++v) x[b][v] = in[v];
            features(x[b], ca.lambda, a.hdry, f);
        }
        const float *is = sm.net.in_scale;
        uint4 w;
        w.x = pack_bf16(f[0] * is[0], f[1] * is[1]);
        w.y = pack_bf16(f[2] * is[2], f[3] * is[3]);
        w.z = pack_bf16(f[4] * is[4], f[5] * is[5]);
        w.w = 0x3F803F80u;  // 1.0, 1.0: the bias columns
        *reinterpret_cast<uint4 *>(&sm.A1[b][tc::kmajor_index(tid, 0, 16)]) = w;
    };
    // the operand tiles written by all threads -> the tensor core; then one thread issues layer L of tile b
    // the operand tiles written by all threads -> the tensor core; then one thread issues layer L of
    // tile b.  The barrier also carries the outcome of the completion waits since the last one
    // (false: some thread's wait gave up, stop).
    bool lost = false;
    auto issue = [&](int b, int L) {
        tc::fence_async_smem();
        tc::fence_before_sync();
        if (__syncthreads_or(lost)) return false;
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t d = tmem + 64 * b;
            const uint32_t sa1 = tc::smem_u32(sm.A1[b]), sa2 = tc::smem_u32(sm.A2[b]);
            if (L == 1) {
                tc::mma_bf16(d, tc::smem_desc(sa1, 128, 256), tc::smem_desc(sb1, 128, 256), TC_IDESC64, 0u);
            } else {
                // the bias (layer-1 tile's ones columns x Bb), then the four K = 16 steps of the layer
                const uint32_t sb = L == 2 ? sb2 : sb3, idesc = L == 2 ? TC_IDESC64 : TC_IDESC16;
                tc::mma_bf16(d, tc::smem_desc(sa1, 128, 256), tc::smem_desc(L == 2 ? sbb2 : sbb3, 128, 256), idesc, 0u);
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    tc::mma_bf16(d, tc::smem_desc(sa2 + 256 * k, 128, 1024), tc::smem_desc(sb + 256 * k, 128, 1024),
                                 idesc, 1u);
            }
            tc::commit(&sm.bar[b]);
        }
        return true;
    };
    // Every thread waits for its tile's MMAs itself (no barrier); a wait that gives up is recorded
    // and stops the loop at the next barrier (its phase is kept for the final wait).
    auto wait = [&](int b) {
        if (tc::mbar_wait(&sm.bar[b], phase[b], TC_WAIT))
            phase[b] ^= 1u;
        else
            lost = true;
        tc::fence_after_sync();
    };
    // GELU of the 64 accumulator columns of tile b (which hold z/2, bias included) -> BF16 row of its
    // A2 tile.  The four loads are issued back to back and waited for once; with h = z/2,
    // GELU(z) = h (1 + tanh(h (2c + 8 * 0.044715 c h^2))), evaluated on packed FP32 pairs.
    auto hidden = [&](int b) {
        const F2 kb(2.0f * 0.7978845608028654f), ka(8.0f * 0.044715f * 0.7978845608028654f);
#pragma unroll
        for (int c0 = 0; c0 < 64; c0 += TC_CHUNK) {
            uint32_t r[TC_CHUNK];
#pragma unroll
            for (int c = 0; c < TC_CHUNK / 16; ++c) tc::tmem_ld16_nowait(tmem + tlane + 64 * b + c0 + 16 * c, r + 16 * c);
            tc::wait_ld();
#pragma unroll
            for (int g = 0; g < TC_CHUNK / 8; ++g) {
                uint32_t w[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int j = 8 * g + 2 * q;
                    const F2 h(__uint_as_float(r[j]), __uint_as_float(r[j + 1]));
                    F2 gz;
                    if (TC_POLY_EVERY > 0 && (j / 2) % TC_POLY_EVERY == TC_POLY_EVERY - 1) {
                        gz = gelu_poly2(h);  // this pair on the FMA pipe
                    } else {
                        const F2 u = h * fma2(ka, h * h, kb);
                        const F2 t(tanh_approx(u.x()), tanh_approx(u.y()));
                        gz = fma2(h, t, h);
                    }
                    w[q] = pack_bf16(gz.x(), gz.y());
                }
                *reinterpret_cast<uint4 *>(&sm.A2[b][tc::kmajor_index(tid, c0 + 8 * g, 64)]) =
                    make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
    };
    // layer-3 accumulator of tile b -> outputs of this thread's cell
    auto output = [&](int b, int64_t tile) {
        float y[8], p[6];
        tc::tmem_ld8(tmem + tlane + 64 * b, y);
#pragma unroll
        for (int j = 0; j < 6; ++j) p[j] = y[j] * sm.net.out_scale[j];
        const int64_t i = tile * 128 + tid;
        if (i < nc) {
            float *dst = MODE == 2 ? out : ca.pred;
            const int64_t stride = MODE == 2 ? n : ca.pstride;
#pragma unroll
            for (int j = 0; j < 6; ++j) dst[j * stride + i] = p[j];
        }
        if (MODE == 1) {
            const float sp = closed_speed(x[b], p, a.g, a.hdry);
            if (i < nc) {
                if (!(sp <= 3.0e38f)) flag |= DEV_NAN;
                if (!(x[b][0] >= 0.0f)) flag |= (x[b][0] < 0.0f) ? DEV_NEGDEPTH : DEV_NAN;
                smax = (sp > smax || sp != sp) ? sp : smax;
            }
        }
    };

    if constexpr (TC_TILES == 1) {
        float in[6];
        if (!skip && blockIdx.x < ntiles) load(blockIdx.x, in);
        for (int64_t tile = blockIdx.x; tile < ntiles && !skip; tile += gridDim.x) {
            prep(0, in);
            if (!issue(0, 1)) break;
            if (tile + gridDim.x < ntiles) load(tile + gridDim.x, in);  // the next tile's inputs
            wait(0);
            hidden(0);
            if (!issue(0, 2)) break;
            wait(0);
            hidden(0);
            if (!issue(0, 3)) break;
            wait(0);
            output(0, tile);
            // every accumulator row is read before the next tile's layer-1 MMA overwrites the region
            tc::fence_before_sync();
            if (__syncthreads_or(lost)) break;
        }
    } else {
        float inA[6], inB[6];
        const int64_t npairs = (ntiles + 1) / 2;
        if (!skip && blockIdx.x < npairs) load(2 * blockIdx.x, inA);
        for (int64_t pr = blockIdx.x; pr < npairs && !skip; pr += gridDim.x) {
            const int64_t tA = 2 * pr, tB = 2 * pr + 1;
            const bool hasB = tB < ntiles;  // uniform across the CTA
            if (hasB) load(tB, inB);
            prep(0, inA);
            if (!issue(0, 1)) break;
            if (hasB) {
                prep(1, inB);
                if (!issue(1, 1)) break;
            }
            if (pr + gridDim.x < npairs) load(2 * (pr + gridDim.x), inA);  // next pair's first tile
            // layer 1 -> 2 -> 3 of both tiles, each epilogue overlapping the other tile's MMA
            wait(0);
            hidden(0);
            if (!issue(0, 2)) break;
            if (hasB) {
                wait(1);
                hidden(1);
                if (!issue(1, 2)) break;
            }
            wait(0);
            hidden(0);
            if (!issue(0, 3)) break;
            if (hasB) {
                wait(1);
                hidden(1);
                if (!issue(1, 3)) break;
            }
            wait(0);
            output(0, tA);
            if (hasB) {
                wait(1);
                output(1, tB);
            }
            tc::fence_before_sync();
            if (__syncthreads_or(lost)) break;
        }
    }
    failed = __syncthreads_or(lost);
    if (failed) {
        if (tid == 0) atomicOr(&a.ctl->status, DEV_TIMEOUT);
        // the MMAs still in flight, once more with a limit
#pragma unroll
        for (int b = 0; b < TC_TILES; ++b) tc::mbar_wait(&sm.bar[b], phase[b], TC_WAIT);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, TC_COLS);
    }
    if (MODE == 1) {
        if (flag) atomicOr(&a.ctl->status, flag);
        reduce_smax<float>(a.ctl, a.slot_out, smax);
    }
}

// ------------------------------------------------------------------------------------------
// Host side
// ------------------------------------------------------------------------------------------

static uint16_t to_bf16(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    const uint32_t lsb = (u >> 16) & 1u;
    u = u + 0x7fffu + lsb;
    return (uint16_t)(u >> 16);
}

static uint32_t pair_bf16(float lo, float hi) { return (uint32_t)to_bf16(lo) | ((uint32_t)to_bf16(hi) << 16); }

// params: W1 [6][64] (row = input), b1 [64], W2 [64][64], b2 [64], W3 [64][6], b3 [6] (FP32)
static void build_closure_dev(const float *p, const float *in_scale, const float *out_scale, ClosureDev &d)
{
    const float *W1 = p, *b1 = W1 + 6 * 64, *W2 = b1 + 64, *b2 = W2 + 64 * 64, *W3 = b2 + 64, *b3 = W3 + 64 * 6;
    auto w1 = [&](int k, int n) { return k < 6 ? W1[k * 64 + n] : 0.0f; };
    auto w3 = [&](int k, int n) { return n < 6 ? W3[k * 6 + n] : 0.0f; };
    memset(&d, 0, sizeof(d));
    for (int lane = 0; lane < 32; ++lane) {
        const int g = lane >> 2, t = lane & 3;
        for (int nt = 0; nt < 8; ++nt) d.w1[nt][lane] = pair_bf16(w1(2 * t, nt * 8 + g), w1(2 * t + 1, nt * 8 + g));
        for (int kc = 0; kc < 4; ++kc) {
            for (int nt = 0; nt < 8; ++nt) {
                const int n = nt * 8 + g, k0 = 16 * kc + 2 * t;
                d.w2[kc][nt][lane].x = pair_bf16(W2[k0 * 64 + n], W2[(k0 + 1) * 64 + n]);
                d.w2[kc][nt][lane].y = pair_bf16(W2[(k0 + 8) * 64 + n], W2[(k0 + 9) * 64 + n]);
            }
            const int k0 = 16 * kc + 2 * t;
            d.w3[kc][lane].x = pair_bf16(w3(k0, g), w3(k0 + 1, g));
            d.w3[kc][lane].y = pair_bf16(w3(k0 + 8, g), w3(k0 + 9, g));
        }
    }
    memcpy(d.b1, b1, sizeof(float) * 64);
    memcpy(d.b2, b2, sizeof(float) * 64);
    for (int j = 0; j < 6; ++j) d.b3[j] = b3[j];
    memcpy(d.in_scale, in_scale, sizeof(float) * 6);
    memcpy(d.out_scale, out_scale, sizeof(float) * 6);
}

// The network in the tcgen05 operand layout (weights rounded to BF16 like the mma.sync image).
static float from_bf16(uint16_t h)
{
    const uint32_t u = (uint32_t)h << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

static void build_closure_tc(const float *p, const float *in_scale, const float *out_scale, ClosureTC &d)
{
    const float *W1 = p, *b1 = W1 + 6 * 64, *W2 = b1 + 64, *b2 = W2 + 64 * 64, *W3 = b2 + 64, *b3 = W3 + 64 * 6;
    memset(&d, 0, sizeof(d));
    // a bias value as two BF16 parts in columns 6 (hi) and 7 (lo) of a K = 16 row
    auto bias = [&](uint16_t *B, int n, float v) {
        const uint16_t hi = to_bf16(v);
        B[tc::kmajor_index(n, 6, 16)] = hi;
        B[tc::kmajor_index(n, 7, 16)] = to_bf16(v - from_bf16(hi));
    };
    for (int n = 0; n < 64; ++n) {
        for (int k = 0; k < 6; ++k) d.B1[tc::kmajor_index(n, k, 16)] = to_bf16(0.5f * W1[k * 64 + n]);
        bias(d.B1, n, 0.5f * b1[n]);
        for (int k = 0; k < 64; ++k) d.B2[tc::kmajor_index(n, k, 64)] = to_bf16(0.5f * W2[k * 64 + n]);
        bias(d.Bb2, n, 0.5f * b2[n]);
    }
    for (int n = 0; n < 6; ++n) {
        for (int k = 0; k < 64; ++k) d.B3[tc::kmajor_index(n, k, 64)] = to_bf16(W3[k * 6 + n]);
        bias(d.Bb3, n, b3[n]);
    }
    for (int j = 0; j < 6; ++j) {
        d.in_scale[j] = in_scale[j];
        d.out_scale[j] = out_scale[j];
    }
}

static cudaError_t launch_predict(zoomy_ctx *c, const ClosureArgs &ca, bool ws)
{
    if (c->closure_engine == 0) {
        const unsigned grid = (unsigned)(TC_CTAS_PER_SM * c->nsm);
        const ClosureTC *net = (const ClosureTC *)c->closure_tc;
        const float *nof = nullptr;
        float *noo = nullptr;
        return ws ? launch_pdl_dyn(k_closure_tc<1>, grid, TC_THREADS, TC_DYN_SMEM, c->stream, ca, net, nof, noo,
                                   (int64_t)0)
                  : launch_pdl_dyn(k_closure_tc<0>, grid, TC_THREADS, TC_DYN_SMEM, c->stream, ca, net, nof, noo,
                                   (int64_t)0);
    } else {
        const unsigned pgrid = (unsigned)(4 * c->nsm);
        if (ws)
            k_closure_predict<true><<<pgrid, 128, 0, c->stream>>>(ca);
        else
            k_closure_predict<false><<<pgrid, 128, 0, c->stream>>>(ca);
    }
    return cudaGetLastError();
}

zoomy_status closure_run_steps(zoomy_ctx *c, float *Q, int64_t ld, double dt, int nsteps)
{
    ClosureArgs ca;
    memset(&ca, 0, sizeof(ca));
    StageArgs<float> &a = ca.s;
    a.bed = (const float *)c->bed_dev;
    a.ld = ld;
    a.nx = (int)c->nx;
    a.ny = (int)c->ny;
    a.inv_dx = (float)(1.0 / c->dx);
    a.inv_dy = (float)(1.0 / c->dy);
    for (int i = 0; i < 4; ++i) a.bc[i] = c->bc[i];
    a.g = (float)c->g;
    a.hdry = (float)c->hdry;
    a.fric = c->fric.kind;
    a.nu_rho = c->fric.kind == ZOOMY_FRICTION_SLIP_NEWTONIAN ? (float)(c->fric.nu / c->fric.rho) : 0.0f;
    a.C_rho = (float)(c->fric.C / c->fric.rho);
    a.gn2 = (float)(c->g * c->fric.manning_n * c->fric.manning_n);
    a.cfl = c->cfl;
    a.dmin = c->min_delta;
    a.dt_fixed = dt;
    a.ctl = c->ctl;
    a.nstrips = (int)((c->nx + 29) / 30);
    if (c->rows_per_warp > 0) {
        a.H = c->rows_per_warp;
    } else {  // segments of one wave of one-warp CTAs
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_stage_closure<2>, 32, 0) != cudaSuccess || nb < 1)
            nb = 1;
        const int64_t segs = std::max<int64_t>(1, (int64_t)c->nsm * nb / a.nstrips);
        a.H = (int)std::max<int64_t>(1, (c->ny + segs - 1) / segs);
    }
    a.nsegs = (int)((c->ny + a.H - 1) / a.H);
    ca.net = (const ClosureDev *)c->closure_d;
    ca.pred = (float *)c->closure_pred;
    ca.pstride = c->nx * c->ny;
    ca.lambda = (float)c->closure_lambda;
    float *Q1 = (float *)c->q1;
    const dim3 grid((unsigned)(a.nstrips * a.nsegs)), block(32);
    for (int k = 0; k < nsteps; ++k) {
        // closure of Q^n and its wave speed (this step's dt) into slot k & 1, cleared by the previous
        // step's first stage (or at the start of the call)
        a.X = Q;
        a.slot_out = k & 1;
        zoomy_status ps = prof_mark(c, 3, true);
        if (ps != ZOOMY_OK) return ps;
        cudaError_t e = launch_predict(c, ca, true);
        if (e != cudaSuccess) return cuda_fail(e, "closure prediction launch");
        if ((ps = prof_mark(c, 3, false)) != ZOOMY_OK) return ps;
        a.slot_in = k & 1;
        a.slot_out = (k + 1) & 1;
        a.Qn = Q;
        a.out = Q1;
        if ((ps = prof_mark(c, 1, true)) != ZOOMY_OK) return ps;
        if ((e = launch_pdl(k_stage_closure<1>, grid, block, c->stream, ca)) != cudaSuccess)
            return cuda_fail(e, "closure stage 1 launch");
        if ((ps = prof_mark(c, 1, false)) != ZOOMY_OK) return ps;
        a.X = Q1;
        if (c->closure_schedule == 0) {  // schedule 1 keeps the predictions made on Q^n
            if ((ps = prof_mark(c, 3, true)) != ZOOMY_OK) return ps;
            if ((e = launch_predict(c, ca, false)) != cudaSuccess) return cuda_fail(e, "closure prediction launch");
            if ((ps = prof_mark(c, 3, false)) != ZOOMY_OK) return ps;
        }
        a.Qn = Q;
        a.out = Q;
        if ((ps = prof_mark(c, 2, true)) != ZOOMY_OK) return ps;
        if ((e = launch_pdl(k_stage_closure<2>, grid, block, c->stream, ca)) != cudaSuccess)
            return cuda_fail(e, "closure stage 2 launch");
        if ((ps = prof_mark(c, 2, false)) != ZOOMY_OK) return ps;
    }
    return ZOOMY_OK;
}

// Maximum wave speed of the closed profiles of Q (the speed the closed solver's CFL step uses): the
// prediction kernel with its wave-speed reduction into the auxiliary control block.
zoomy_status closure_max_wavespeed(zoomy_ctx *c, const float *Q, int64_t ld, double *out)
{
    ClosureArgs ca;
    memset(&ca, 0, sizeof(ca));
    StageArgs<float> &a = ca.s;
    a.X = Q;
    a.ld = ld;
    a.nx = (int)c->nx;
    a.ny = (int)c->ny;
    a.g = (float)c->g;
    a.hdry = (float)c->hdry;
    a.ctl = c->ctl_aux;
    a.slot_out = 0;
    ca.net = (const ClosureDev *)c->closure_d;
    ca.pred = (float *)c->closure_pred;
    ca.pstride = c->nx * c->ny;
    ca.lambda = (float)c->closure_lambda;
    cudaError_t e = cudaMemsetAsync(c->ctl_aux, 0, sizeof(DevCtl), c->stream);
    if (e == cudaSuccess) e = launch_predict(c, ca, true);
    DevCtl h;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, c->ctl_aux, sizeof(DevCtl), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "closure wave speed");
    float v;
    memcpy(&v, &h.smax_f[0], 4);
    *out = v;
    if (h.status & DEV_NAN) return set_error(ZOOMY_ENAN, "non-finite state");
    if (h.status & DEV_TIMEOUT) return set_error(ZOOMY_ETIMEOUT, "a device-side wait exceeded its limit");
    return ZOOMY_OK;
}

zoomy_status closure_upload(zoomy_ctx *c, const float *params, const float *in_scale, const float *out_scale)
{
    ClosureDev d;
    build_closure_dev(params, in_scale, out_scale, d);
    if (!c->closure_d) {
        cudaError_t e = cudaMalloc(&c->closure_d, sizeof(ClosureDev));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    }
    if (!c->closure_pred) {
        cudaError_t e = cudaMalloc(&c->closure_pred, sizeof(float) * 6 * (size_t)(c->nx * c->ny));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    }
    if (!c->closure_tc) {
        cudaError_t e = cudaMalloc(&c->closure_tc, sizeof(ClosureTC));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
        // the two-tile operand buffers exceed the default 48 KB of shared memory per CTA
        if ((e = cudaFuncSetAttribute(k_closure_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_DYN_SMEM)) !=
                cudaSuccess ||
            (e = cudaFuncSetAttribute(k_closure_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_DYN_SMEM)) !=
                cudaSuccess ||
            (e = cudaFuncSetAttribute(k_closure_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_DYN_SMEM)) !=
                cudaSuccess)
            return cuda_fail(e, "cudaFuncSetAttribute");
    }
    ClosureTC t;
    build_closure_tc(params, in_scale, out_scale, t);
    cudaError_t e = cudaMemcpy(c->closure_d, &d, sizeof(ClosureDev), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->closure_tc, &t, sizeof(ClosureTC), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
    return ZOOMY_OK;
}

}  // namespace zoomy

using namespace zoomy;

extern "C" zoomy_status zoomy_closure_eval(zoomy_ctx *c, const float *feat, float *out, int64_t n)
{
    if (!c || !feat || !out || n < 0) return set_error(ZOOMY_EINVAL, "zoomy_closure_eval: bad arguments");
    if (!c->closure_d) return set_error(ZOOMY_ESTATE, "zoomy_closure_eval: no closure set");
    if (n == 0) return ZOOMY_OK;
    int64_t blocks = (n + 127) / 128;
    if (c->closure_engine == 0) {
        if (blocks > (int64_t)TC_CTAS_PER_SM * c->nsm) blocks = (int64_t)TC_CTAS_PER_SM * c->nsm;
        ClosureArgs ca;
        memset(&ca, 0, sizeof(ca));
        ca.s.ctl = c->ctl;  // a timed-out completion wait is reported by the next synchronising call
        k_closure_tc<2><<<(unsigned)blocks, TC_THREADS, TC_DYN_SMEM, c->stream>>>(ca, (const ClosureTC *)c->closure_tc,
                                                                         feat, out, n);
    } else {
        if (blocks > 8LL * c->nsm) blocks = 8LL * c->nsm;
        k_closure_eval<<<(unsigned)blocks, 128, 0, c->stream>>>((const ClosureDev *)c->closure_d, feat, out, n);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "closure eval launch");
    return ZOOMY_OK;
}

extern "C" zoomy_status zoomy_closure_schedule(zoomy_ctx *c, int32_t schedule)
{
    if (!c || schedule < 0 || schedule > 1) return set_error(ZOOMY_EINVAL, "zoomy_closure_schedule: schedule is 0 or 1");
    c->closure_schedule = schedule;
    return ZOOMY_OK;
}

extern "C" zoomy_status zoomy_closure_engine(zoomy_ctx *c, int32_t engine)
{
    if (!c || engine < 0 || engine > 1) return set_error(ZOOMY_EINVAL, "zoomy_closure_engine: engine is 0 or 1");
    c->closure_engine = engine;
    return ZOOMY_OK;
}
