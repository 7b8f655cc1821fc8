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
#include <cstdint>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "f32x2.cuh"
#include "fv_common.cuh"
#include "tcgen05.cuh"
#include "zoomy_internal.h"
#include "zoomy_kernels.h"

namespace zoomy {

constexpr int CL_M = 5;   // moments of the closed profile (level 4)
constexpr int CL_NV = 5;  // prognostic variables (level 1, 2D)

// weight fragments in the layout of the mma.sync B operand (per lane), then FP32 biases
struct ClosureDev {
    uint32_t w1[8][32];     // layer 1: n-tile, lane -> b0 (rows 2t,2t+1 of the padded 16-row W1)
    uint2 w2[4][8][32];     // layer 2: k-chunk, n-tile, lane -> (b0, b1)
    uint2 w3[4][32];        // layer 3: k-chunk, lane -> (b0, b1) (outputs padded 6 -> 8)
    float b1[64], b2[64], b3[8];
    float in_scale[6], out_scale[6];
};

struct ClosureArgs {
    StageArgs<float> s;
    const ClosureDev *net;
    float *pred;      // predicted closed moments of the stage input, SoA [6][pstride]
    int64_t pstride;  // nx * ny
    float lambda;
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

// Closed cell record (scalar FP32).
struct CRec {
    float h, b;
    float a[CL_M], c[CL_M];       // alpha_k, beta_k of the closed profile (zero where dry)
    float um, s2, s1;
    float gaa[2], gab[2], gbb[2];  // flux products of rows k = 0, 1
    float sa, sb;                  // sum_{k>=2} alpha_k, beta_k (closed part, for the bottom stress)
};

__device__ __forceinline__ void make_crec(CRec &r, float h, float b, const float *q, const float *pred, bool xwall,
                                          bool ywall, float hdry)
{
    const bool wet = h > hdry;
    const float ih = wet ? __frcp_rn(h) : 0.0f;
    r.h = h;
    r.b = b;
    r.a[0] = q[1] * ih;
    r.c[0] = q[2] * ih;
    r.a[1] = q[3] * ih;
    r.c[1] = q[4] * ih;
#pragma unroll
    for (int k = 2; k < CL_M; ++k) {
        r.a[k] = wet ? pred[k - 2] : 0.0f;
        r.c[k] = wet ? pred[k + 1] : 0.0f;
    }
#pragma unroll
    for (int k = 0; k < CL_M; ++k) {
        if (xwall) r.a[k] = -r.a[k];
        if (ywall) r.c[k] = -r.c[k];
    }
    r.sa = r.a[2] + r.a[3] + r.a[4];
    r.sb = r.c[2] + r.c[3] + r.c[4];
    r.um = sqrtf(r.a[0] * r.a[0] + r.c[0] * r.c[0]);
    float s2 = 0.f, s1 = 0.f;
#pragma unroll
    for (int k = 1; k < CL_M; ++k) {
        const float q2 = r.a[k] * r.a[k] + r.c[k] * r.c[k];
        s2 += q2;
        if (k >= 2) s1 += sqrtf(q2);
    }
    r.s2 = s2;
    r.s1 = s1;
    static_for<0, 2>([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        float saa = 0.f, sab = 0.f, sbb = 0.f;
        static_for<0, CL_M>([&](auto ii) {
            constexpr int i = decltype(ii)::value;
            static_for<0, CL_M>([&](auto jj) {
                constexpr int j = decltype(jj)::value;
                constexpr double w = fluxA(i, j, k);
                if constexpr (w != 0.0) {
                    if constexpr (j >= i) {
                        constexpr double w2 = (i == j) ? w : 2.0 * w;
                        saa += float(w2) * r.a[i] * r.a[j];
                        sbb += float(w2) * r.c[i] * r.c[j];
                    }
                    sab += float(w) * r.a[i] * r.c[j];
                }
            });
        });
        r.gaa[k] = saa;
        r.gab[k] = sab;
        r.gbb[k] = sbb;
    });
}

// Face terms of the restricted model in a face frame (n, t): rows mass, n_0, n_1, t_0, t_1.
// out: fc[5] (mass, n0, n1, t0, t1) and nc[5] (only n1, t1 are non-zero), pd on n0.
template <bool YDIR>
__device__ __forceinline__ void face_closure(const CRec &L, const CRec &R, float g, float hdry, float *fc, float &pd,
                                             float *nc)
{
    const float *nL = YDIR ? L.c : L.a, *tL = YDIR ? L.a : L.c;
    const float *nR = YDIR ? R.c : R.a, *tR = YDIR ? R.a : R.c;
    const float *gnnL = YDIR ? L.gbb : L.gaa, *gnnR = YDIR ? R.gbb : R.gaa;
    const float bf = fmaxf(L.b, R.b);
    const HPair pl = hr_depth(L.h, L.b, bf), pr = hr_depth(R.h, R.b, bf);
    const float hl = hp_val(pl), hr = hp_val(pr), dh = hp_diff(pr, pl);
    const bool wl = hl > hdry, wr = hr > hdry;
    const float sl = wl ? L.um + sqrtf(g * hl + L.s2) + L.s1 : sqrtf(g * hl);
    const float sr = wr ? R.um + sqrtf(g * hr + R.s2) + R.s1 : sqrtf(g * hr);
    const float hs = 0.5f * fmaxf(sl, sr);
    const float el = wl ? hl : 0.0f, er = wr ? hr : 0.0f;
    float dn[CL_M], dtv[2];
#pragma unroll
    for (int k = 0; k < CL_M; ++k) dn[k] = er * nR[k] - el * nL[k];
    dtv[0] = er * tR[0] - el * tL[0];
    dtv[1] = er * tR[1] - el * tL[1];
    fc[0] = 0.5f * (el * nL[0] + er * nR[0]) - hs * dh;
    fc[1] = 0.5f * (el * gnnL[0] + er * gnnR[0]) - hs * dn[0];
    fc[2] = 0.5f * (el * gnnL[1] + er * gnnR[1]) - hs * dn[1];
    fc[3] = 0.5f * (el * L.gab[0] + er * R.gab[0]) - hs * dtv[0];
    fc[4] = 0.5f * (el * L.gab[1] + er * R.gab[1]) - hs * dtv[1];
    pd = 0.25f * g * dh * (hr + hl);
    // path-averaged closed profiles (3-point Gauss-Legendre, weights W0/W1 as in the structured kernels)
    constexpr float sq15 = 0.38729833462074168852f;
    const float sn[3] = {0.5f - sq15, 0.5f, 0.5f + sq15};
    const float wq[3] = {5.0f / 18.0f, 8.0f / 18.0f, 5.0f / 18.0f};
    float W0 = 0.f, W1 = 0.f;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float hq = fmaf(sn[q], dh, hl);
        const float iw = hq > hdry ? wq[q] * __frcp_rn(hq) : 0.0f;
        W0 += iw;
        W1 = fmaf(sn[q], iw, W1);
    }
    float nb[CL_M], tb[CL_M];
#pragma unroll
    for (int k = 0; k < CL_M; ++k) {
        nb[k] = el * nL[k] * W0 + dn[k] * W1;
        tb[k] = el * tL[k] * W0 + (er * tR[k] - el * tL[k]) * W1;
    }
    float rn = 0.f, rt = 0.f;
    static_for<1, CL_M>([&](auto ll) {
        constexpr int l = decltype(ll)::value;
        float en = 0.f, et = 0.f;
        static_for<0, CL_M>([&](auto jj) {
            constexpr int j = decltype(jj)::value;
            constexpr double w = ncB(1, j, l);
            if constexpr (w != 0.0) {
                en += float(w) * nb[j];
                et += float(w) * tb[j];
            }
        });
        rn += en * dn[l];
        rt += et * dn[l];
    });
    nc[0] = nc[1] = nc[3] = 0.0f;
    nc[2] = 0.5f * rn;
    nc[4] = 0.5f * rt;
}

__device__ __forceinline__ CRec shfl_up_crec(const CRec &r)
{
    constexpr unsigned F = 0xffffffffu;
    CRec o;
    o.h = __shfl_up_sync(F, r.h, 1);
    o.b = __shfl_up_sync(F, r.b, 1);
    o.um = __shfl_up_sync(F, r.um, 1);
    o.s2 = __shfl_up_sync(F, r.s2, 1);
    o.s1 = __shfl_up_sync(F, r.s1, 1);
#pragma unroll
    for (int k = 0; k < CL_M; ++k) {
        o.a[k] = __shfl_up_sync(F, r.a[k], 1);
        o.c[k] = __shfl_up_sync(F, r.c[k], 1);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        o.gaa[k] = __shfl_up_sync(F, r.gaa[k], 1);
        o.gab[k] = __shfl_up_sync(F, r.gab[k], 1);
        o.gbb[k] = 0.0f;
    }
    o.sa = o.sb = 0.0f;
    return o;
}

// frame row (mass, n0, n1, t0, t1) -> variable (h, hA0, hB0, hA1, hB1)
template <bool YDIR>
__device__ __forceinline__ int cl_var(int row)
{
    // x-face: n = alpha, t = beta;  y-face: n = beta, t = alpha
    const int xmap[5] = {0, 1, 3, 2, 4};
    const int ymap[5] = {0, 2, 4, 1, 3};
    return YDIR ? ymap[row] : xmap[row];
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

template <int STAGE>
__global__ void __launch_bounds__(128) k_stage_closure(ClosureArgs ca)
{
    const StageArgs<float> &a = ca.s;
    constexpr unsigned F = 0xffffffffu;
    if (*(volatile unsigned int *)&a.ctl->status) return;
    float dt;
    if (!step_dt(a, dt)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&a.ctl->status, DEV_NOWAVE);
        return;
    }
    if (STAGE == 1 && blockIdx.x == 0 && threadIdx.x == 0) step_bookkeeping(a, dt);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wg = blockIdx.x * 4 + warp;
    const int strip = wg % a.nstrips, seg = wg / a.nstrips;
    if (seg >= a.nsegs) return;
    const int col = strip * 30 - 1 + lane;
    const bool owned = lane >= 1 && lane <= 30 && col < a.nx;
    const int csrc = col < 0 ? 0 : (col >= a.nx ? a.nx - 1 : col);
    const bool xwall = (col < 0 && a.bc[0] == 1) || (col >= a.nx && a.bc[1] == 1);
    const int r0 = seg * a.H, r1 = min(r0 + a.H, a.ny);
    const float g = a.g, hdry = a.hdry;

    CRec prev, cur;
    {
        const float z[6] = {0, 0, 0, 0, 0, 0};
        const float q0[5] = {0, 0, 0, 0, 0};
        make_crec(prev, 0.0f, 0.0f, q0, z, false, false, hdry);
    }
    float xprev[CL_NV] = {0, 0, 0, 0, 0}, accp[CL_NV] = {0, 0, 0, 0, 0};
    unsigned flag = 0;
    // the next row's state, bed and predictions are loaded one iteration ahead
    float xn[CL_NV], bn, pn[6];
    auto load_row = [&](int rr) {
        const int rs = rr < 0 ? 0 : (rr >= a.ny ? a.ny - 1 : rr);
        const int64_t idx = (int64_t)rs * a.nx + csrc;
#pragma unroll
        for (int v = 0; v < CL_NV; ++v) xn[v] = __ldg(a.X + v * a.ld + idx);
        bn = __ldg(a.bed + idx);
#pragma unroll
        for (int j = 0; j < 6; ++j) pn[j] = __ldg(ca.pred + j * ca.pstride + idx);
    };
    load_row(r0 - 1);
    for (int r = r0 - 1; r <= r1; ++r) {
        const bool ywall = (r < 0 && a.bc[2] == 1) || (r >= a.ny && a.bc[3] == 1);
        float x[CL_NV], pred[6];
#pragma unroll
        for (int v = 0; v < CL_NV; ++v) x[v] = xn[v];
        const float bed = bn;
        // closure of this row's cells (predicted from the unreflected state; ghosts reflect it)
#pragma unroll
        for (int j = 0; j < 6; ++j) pred[j] = pn[j];
        if (r < r1) load_row(r + 1);
        // Q^n of the row finished in this iteration (stage 2), requested before the face work
        float qn[CL_NV];
        if (STAGE == 2) {
            const int64_t qidx = (int64_t)(r - 1 >= r0 ? r - 1 : r0) * a.nx + csrc;
#pragma unroll
            for (int v = 0; v < CL_NV; ++v) qn[v] = __ldg(a.Qn + v * a.ld + qidx);
        }
        float q[CL_NV];
#pragma unroll
        for (int v = 0; v < CL_NV; ++v) q[v] = x[v];
        make_crec(cur, x[0], bed, q, pred, xwall, ywall, hdry);

        float accc[CL_NV] = {0, 0, 0, 0, 0};
        float fc[5], nc[5], pd;
        const bool xrow = r >= r0 && r < r1;
        if (xrow) {
            const CRec left = shfl_up_crec(cur);
            face_closure<false>(left, cur, g, hdry, fc, pd, nc);
            float tl[CL_NV];
#pragma unroll
            for (int row = 0; row < 5; ++row) {
                const int v = cl_var<false>(row);
                const float pdr = row == 1 ? pd : 0.0f;
                accc[v] += a.inv_dx * (fc[row] - pdr - nc[row]);
                tl[v] = a.inv_dx * (fc[row] + pdr + nc[row]);
            }
#pragma unroll
            for (int v = 0; v < CL_NV; ++v) accc[v] -= __shfl_down_sync(F, tl[v], 1);
        }
        if (r > r0 - 1) {
            face_closure<true>(prev, cur, g, hdry, fc, pd, nc);
#pragma unroll
            for (int row = 0; row < 5; ++row) {
                const int v = cl_var<true>(row);
                const float pdr = row == 1 ? pd : 0.0f;
                accp[v] -= a.inv_dy * (fc[row] + pdr + nc[row]);
                accc[v] += a.inv_dy * (fc[row] - pdr - nc[row]);
            }
            const bool fin = r - 1 >= r0;
            if (fin) {  // row r-1 is complete (all lanes compute; owners store)
                // Newtonian bulk stress of the closed profile, rows k = 0, 1
                const float f0 = prev.h > 0.0f ? a.nu_rho / prev.h : 0.0f;
                float sa[2], sb[2];
                static_for<0, 2>([&](auto kk) {
                    constexpr int k = decltype(kk)::value;
                    float xa = 0.f, xb = 0.f;
                    static_for<0, CL_M>([&](auto ii) {
                        constexpr int i = decltype(ii)::value;
                        constexpr double w = visC(i, k);
                        if constexpr (w != 0.0) {
                            xa += float(w) * prev.a[i];
                            xb += float(w) * prev.c[i];
                        }
                    });
                    sa[k] = -f0 * xa;
                    sb[k] = -f0 * xb;
                });
                float y[CL_NV];
                y[0] = xprev[0] + dt * accp[0];
                y[1] = xprev[1] + dt * accp[1] + dt * sa[0];
                y[2] = xprev[2] + dt * accp[2] + dt * sb[0];
                y[3] = xprev[3] + dt * accp[3] + dt * sa[1];
                y[4] = xprev[4] + dt * accp[4] + dt * sb[1];
                // bottom stress: implicit in (alpha_0, alpha_1), closed moments frozen at the stage input
                const float h = y[0];
                const bool wet = h > hdry;
                const float ih = __frcp_rn(h);
                const float sah = h * prev.sa, sbh = h * prev.sb;
                float cc = 0.0f;
                if (a.fric == 1) {
                    cc = a.C_rho * ih;
                } else if (a.fric == 2) {
                    const float ub = (y[1] + y[3] + sah) * ih, vb = (y[2] + y[4] + sbh) * ih;
                    cc = a.gn2 * sqrtf(ub * ub + vb * vb) * ih / cbrtf(h);
                }
                const float dc = dt * cc;
                const float ra0 = y[1] - dc * sah, ra1 = y[3] - 3.0f * dc * sah;
                const float rb0 = y[2] - dc * sbh, rb1 = y[4] - 3.0f * dc * sbh;
                const float den = 1.0f + 4.0f * dc;
                const float fa = dc * (ra0 + ra1) / den, fb = dc * (rb0 + rb1) / den;
                y[1] = wet ? ra0 - fa : 0.0f;
                y[3] = wet ? ra1 - 3.0f * fa : 0.0f;
                y[2] = wet ? rb0 - fb : 0.0f;
                y[4] = wet ? rb1 - 3.0f * fb : 0.0f;
                const int64_t oidx = (int64_t)(r - 1) * a.nx + (owned ? col : csrc);
                if (STAGE == 2) {
#pragma unroll
                    for (int v = 0; v < CL_NV; ++v) y[v] = 0.5f * (qn[v] + y[v]);
                    // (the next step's prediction kernel takes the new state's wave speed)
                    if (owned) {
                        bool bad = false;
#pragma unroll
                        for (int v = 0; v < CL_NV; ++v) bad |= !(fabsf(y[v]) <= 3.0e38f);
                        if (bad) flag |= DEV_NAN;
                        if (y[0] < 0.0f) flag |= DEV_NEGDEPTH;
                    }
                }
                if (owned) {
#pragma unroll
                    for (int v = 0; v < CL_NV; ++v) a.out[v * a.ld + oidx] = y[v];
                }
            }
        }
        prev = cur;
#pragma unroll
        for (int v = 0; v < CL_NV; ++v) {
            xprev[v] = x[v];
            accp[v] = accc[v];
        }
    }
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
            CRec r;
            make_crec(r, x[0], 0.0f, x, p, false, false, a.hdry);
            const float s = r.um + sqrtf(a.g * fmaxf(x[0], 0.0f) + r.s2) + r.s1;
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

struct TCSmem {
    ClosureTC net;
    alignas(128) uint16_t A1[2][128 * 16];  // layer-1 input tiles (K = 16), one per tile in flight
    alignas(128) uint16_t A2[2][128 * 64];  // layer-2 and layer-3 input tiles (K = 64)
    uint64_t bar[2];
    uint32_t tmem;
};

// Two tiles are in flight per CTA: while the tensor core runs one tile's layer, the threads apply
// the GELU to the other tile's previous layer.  Each tile owns a 64-column accumulator region that
// serves its three layers in turn (a layer's accumulator is read back completely before the next
// MMA into it is issued): 128 columns per CTA, 4 CTAs per SM (53 KB of shared memory each).
constexpr uint32_t TC_COLS = 128;
constexpr long long TC_WAIT = 2000000000LL;    // ~1 s at 2 GHz
constexpr int TC_DYN_SMEM = (int)sizeof(TCSmem);
constexpr int TC_THREADS = 128;
constexpr int TC_CTAS_PER_SM = 4;
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
        *reinterpret_cast<uint4 *>(&sm.A1[0][tc::kmajor_index(tid, 8, 16)]) = make_uint4(0u, 0u, 0u, 0u);
        *reinterpret_cast<uint4 *>(&sm.A1[1][tc::kmajor_index(tid, 8, 16)]) = make_uint4(0u, 0u, 0u, 0u);
    }
    if (warp == 0) tc::tmem_alloc(&sm.tmem, TC_COLS);
    if (tid == 0) {
        tc::mbar_init(&sm.bar[0], 1);
        tc::mbar_init(&sm.bar[1], 1);
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = sm.tmem;
    const uint32_t tlane = (uint32_t)(warp * 32) << 16;  // this warp's 32 lanes
    const bool skip = MODE != 2 && __syncthreads_or(tid == 0 && *(volatile unsigned int *)&a.ctl->status != 0u);
    const uint32_t sb1 = tc::smem_u32(sm.net.B1), sb2 = tc::smem_u32(sm.net.B2), sb3 = tc::smem_u32(sm.net.B3);
    const uint32_t sbb2 = tc::smem_u32(sm.net.Bb2), sbb3 = tc::smem_u32(sm.net.Bb3);
    const int64_t nc = MODE == 2 ? n : (int64_t)a.nx * a.ny;
    const int64_t ntiles = (nc + 127) / 128;
    uint32_t phase[2] = {0u, 0u};
    bool failed = false;
    float smax = 0.0f;
    unsigned flag = 0;
    float x[2][CL_NV];  // the stage input of this thread's cells (wave speed)

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
    auto issue = [&](int b, int L) {
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
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
    };
    auto wait = [&](int b) {
        const bool ok = tc::mbar_wait(&sm.bar[b], phase[b], TC_WAIT);
        if (__syncthreads_or(!ok)) return false;
        phase[b] ^= 1u;
        tc::fence_after_sync();
        return true;
    };
    // GELU of the 64 accumulator columns of tile b (which hold z/2, bias included) -> BF16 row of its
    // A2 tile.  The four loads are issued back to back and waited for once; with h = z/2,
    // GELU(z) = h (1 + tanh(h (2c + 8 * 0.044715 c h^2))), evaluated on packed FP32 pairs.
    auto hidden = [&](int b) {
        uint32_t r[64];
#pragma unroll
        for (int c = 0; c < 4; ++c) tc::tmem_ld16_nowait(tmem + tlane + 64 * b + 16 * c, r + 16 * c);
        tc::wait_ld();
        const F2 kb(2.0f * 0.7978845608028654f), ka(8.0f * 0.044715f * 0.7978845608028654f);
#pragma unroll
        for (int g = 0; g < 8; ++g) {
            uint32_t w[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int j = 8 * g + 2 * q;
                const F2 h(__uint_as_float(r[j]), __uint_as_float(r[j + 1]));
                const F2 u = h * fma2(ka, h * h, kb);
                const F2 t(tanh_approx(u.x()), tanh_approx(u.y()));
                const F2 gz = fma2(h, t, h);
                w[q] = pack_bf16(gz.x(), gz.y());
            }
            *reinterpret_cast<uint4 *>(&sm.A2[b][tc::kmajor_index(tid, 8 * g, 64)]) = make_uint4(w[0], w[1], w[2], w[3]);
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
            CRec r;
            make_crec(r, x[b][0], 0.0f, x[b], p, false, false, a.hdry);
            const float sp = r.um + sqrtf(a.g * fmaxf(x[b][0], 0.0f) + r.s2) + r.s1;
            if (i < nc) {
                if (!(sp <= 3.0e38f)) flag |= DEV_NAN;
                if (!(x[b][0] >= 0.0f)) flag |= (x[b][0] < 0.0f) ? DEV_NEGDEPTH : DEV_NAN;
                smax = (sp > smax || sp != sp) ? sp : smax;
            }
        }
    };

    float inA[6], inB[6];
    const int64_t npairs = (ntiles + 1) / 2;
    if (!skip && blockIdx.x < npairs) load(2 * blockIdx.x, inA);
    for (int64_t pr = blockIdx.x; pr < npairs && !skip; pr += gridDim.x) {
        const int64_t tA = 2 * pr, tB = 2 * pr + 1;
        const bool hasB = tB < ntiles;  // uniform across the CTA
        if (hasB) load(tB, inB);
        prep(0, inA);
        issue(0, 1);
        if (hasB) {
            prep(1, inB);
            issue(1, 1);
        }
        if (pr + gridDim.x < npairs) load(2 * (pr + gridDim.x), inA);  // next pair's first tile
        // layer 1 -> 2 -> 3 of both tiles, each epilogue overlapping the other tile's MMA
        if (!wait(0)) { failed = true; break; }
        hidden(0);
        issue(0, 2);
        if (hasB) {
            if (!wait(1)) { failed = true; break; }
            hidden(1);
            issue(1, 2);
        }
        if (!wait(0)) { failed = true; break; }
        hidden(0);
        issue(0, 3);
        if (hasB) {
            if (!wait(1)) { failed = true; break; }
            hidden(1);
            issue(1, 3);
        }
        if (!wait(0)) { failed = true; break; }
        output(0, tA);
        if (hasB) {
            if (!wait(1)) { failed = true; break; }
            output(1, tB);
        }
        // every accumulator row is read before the next pair's layer-1 MMAs overwrite the regions
        tc::fence_before_sync();
        __syncthreads();
    }
    if (failed) {
        if (tid == 0) atomicOr(&a.ctl->status, DEV_TIMEOUT);
        // the MMAs still in flight, once more with a limit
        tc::mbar_wait(&sm.bar[0], phase[0], TC_WAIT);
        tc::mbar_wait(&sm.bar[1], phase[1], TC_WAIT);
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
        if (ws)
            k_closure_tc<1><<<grid, TC_THREADS, TC_DYN_SMEM, c->stream>>>(ca, (const ClosureTC *)c->closure_tc, nullptr,
                                                                   nullptr, 0);
        else
            k_closure_tc<0><<<grid, TC_THREADS, TC_DYN_SMEM, c->stream>>>(ca, (const ClosureTC *)c->closure_tc, nullptr,
                                                                   nullptr, 0);
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
    a.H = c->rows_per_warp > 0 ? c->rows_per_warp : rows_per_warp_for(c->nx, c->ny, c->nsm, 16);
    a.nsegs = (int)((c->ny + a.H - 1) / a.H);
    ca.net = (const ClosureDev *)c->closure_d;
    ca.pred = (float *)c->closure_pred;
    ca.pstride = c->nx * c->ny;
    ca.lambda = (float)c->closure_lambda;
    float *Q1 = (float *)c->q1;
    const int nwarps = a.nstrips * a.nsegs;
    dim3 grid((nwarps + 3) / 4), block(128);
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
        k_stage_closure<1><<<grid, block, 0, c->stream>>>(ca);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "closure stage 1 launch");
        if ((ps = prof_mark(c, 1, false)) != ZOOMY_OK) return ps;
        a.X = Q1;
        if ((ps = prof_mark(c, 3, true)) != ZOOMY_OK) return ps;
        if ((e = launch_predict(c, ca, false)) != cudaSuccess) return cuda_fail(e, "closure prediction launch");
        if ((ps = prof_mark(c, 3, false)) != ZOOMY_OK) return ps;
        a.Qn = Q;
        a.out = Q;
        if ((ps = prof_mark(c, 2, true)) != ZOOMY_OK) return ps;
        k_stage_closure<2><<<grid, block, 0, c->stream>>>(ca);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "closure stage 2 launch");
        if ((ps = prof_mark(c, 2, false)) != ZOOMY_OK) return ps;
    }
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

extern "C" zoomy_status zoomy_closure_engine(zoomy_ctx *c, int32_t engine)
{
    if (!c || engine < 0 || engine > 1) return set_error(ZOOMY_EINVAL, "zoomy_closure_engine: engine is 0 or 1");
    c->closure_engine = engine;
    return ZOOMY_OK;
}
