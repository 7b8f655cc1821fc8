// closure_stage.cuh -- FV stage of the learned-closure model (level-1 state, level-4 profile) in the
// packed row-marching form of struct2d_f32.cuh.
//
// Model (fv_closure.cu): the level-4 system restricted to the rows of (h, h alpha_0, h beta_0,
// h alpha_1, h beta_1); alpha_2..4, beta_2..4 come from the network's predictions (velocity moments,
// zero where the stage input is dry, reflected with the state in wall ghosts).  The face terms are the
// level-4 ones (Eq. (sme), 2D SME of Sec. 3.4) on the closed profiles projected on those rows: the
// flux rows mass, n_0, n_1, t_0, t_1, the path-conservative Rusanov dissipation, the hydrostatic
// reconstruction with the FP64-grade depth difference (hr_faces), and the nonconservative product of
// row 1 summed over the four closed columns.  The Newtonian source of row 1 sums over all five
// moments; the bottom stress is implicit in (alpha_0, alpha_1) with the closed moments frozen at the
// stage input.
//
// Kernel structure as in struct2d_f32.cuh: one warp marches a 30-column strip (lanes 0 and 31 are
// halo columns) down a segment of rows with the previous row in registers; the x-face on the left
// of a cell and the y-face below it are the two halves of packed f32x2 operations; face terms are
// pre-scaled by dt and accumulate onto X + dt S(X); rows strictly inside the segment run one
// branch-free body.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "f32x2.cuh"
#include "fv_common.cuh"
#include "model.cuh"
#include "struct2d_f32.cuh"

namespace zoomy {

constexpr int CL_M = 5;   // moments of the closed profile (level 4)
constexpr int CL_NV = 5;  // prognostic variables (level 1, 2D)

struct ClosureArgs {
    StageArgs<float> s;
    const struct ClosureDev *net;
    float *pred;      // predicted closed moments, SoA [6][pstride]: alpha_2..4, beta_2..4
    int64_t pstride;  // nx * ny
    float lambda;
};

// A cell of the closed profile as seen by its two faces: the pairs hold the x-face frame in .x and
// the y-face frame in .y.
struct SideC {
    float h, b, um, s2, s1, sc;  // depth, bed, |u_mean|, sum_{k>=1}|a_k|^2, sum_{k>=2}|a_k|, wave speed
    F2 n[CL_M], t[CL_M];         // (alpha_k, beta_k), (beta_k, alpha_k)
    F2 gnn[2], gnt[2];           // flux products of rows k = 0, 1: (aa, bb), (ab, ab)
    F2 sig;                      // closed part of the bottom velocity: sum_{k>=2} (alpha_k, beta_k)
};

struct RowC {
    SideC s;
    float acc[CL_NV];  // X + dt S_newton(X) + dt * (face terms so far)
};

// Closed profile of a cell from its raw state q (h, h alpha_0, h beta_0, h alpha_1, h beta_1), bed b
// and predictions p; wall ghosts reflect every moment of the normal direction.
__device__ __forceinline__ void make_side_c(SideC &r, const float *q, float b, const float *p, bool xwall, bool ywall,
                                            float g, float hdry, float &ih)
{
    const float h = q[0];
    const bool wet = h > hdry;
    ih = wet ? rcpa(h) : 0.0f;
    float a[CL_M], c[CL_M];
    a[0] = q[1] * ih;
    c[0] = q[2] * ih;
    a[1] = q[3] * ih;
    c[1] = q[4] * ih;
#pragma unroll
    for (int k = 2; k < CL_M; ++k) {
        a[k] = wet ? p[k - 2] : 0.0f;
        c[k] = wet ? p[k + 1] : 0.0f;
    }
#pragma unroll
    for (int k = 0; k < CL_M; ++k) {
        a[k] = xwall ? -a[k] : a[k];
        c[k] = ywall ? -c[k] : c[k];
    }
    r.h = h;
    r.b = b;
    r.um = sqrtf(fmaf(a[0], a[0], c[0] * c[0]));
    float s2 = 0.f, s1 = 0.f;
#pragma unroll
    for (int k = 1; k < CL_M; ++k) {
        const float qq = fmaf(a[k], a[k], c[k] * c[k]);
        s2 += qq;
        if (k >= 2) s1 += sqrtf(qq);
    }
    r.s2 = s2;
    r.s1 = s1;
    r.sc = r.um + sqrtf(fmaf(g, fmaxf(h, 0.0f), s2)) + s1;
#pragma unroll
    for (int k = 0; k < CL_M; ++k) {
        r.n[k] = F2(a[k], c[k]);
        r.t[k] = F2(c[k], a[k]);
    }
    r.sig = F2(a[2] + a[3] + a[4], c[2] + c[3] + c[4]);
    static_for<0, 2>([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        F2 sq(0.0f);
        float sab = 0.f;
        static_for<0, CL_M>([&](auto ii) {
            constexpr int i = decltype(ii)::value;
            static_for<0, CL_M>([&](auto jj) {
                constexpr int j = decltype(jj)::value;
                constexpr double w = fluxA(i, j, k);
                if constexpr (w != 0.0) {
                    if constexpr (j >= i) {
                        constexpr double w2 = (i == j) ? w : 2.0 * w;
                        if constexpr (w2 == 1.0)
                            sq = fma2(r.n[i], r.n[j], sq);
                        else
                            sq = fma2(F2(float(w2)) * r.n[i], r.n[j], sq);
                    }
                    sab = fmaf(float(w) * a[i], c[j], sab);
                }
            });
        });
        r.gnn[k] = sq;
        r.gnt[k] = F2(sab);
    });
}

// Face terms of the restricted model for the pair of faces (x-face .x, y-face .y):
//   pr = dt/|Omega| |e| (fc - nc) (row n_0 also - pd)   : contribution to the right cell
//   mi = dt/|Omega| |e| (fc + nc) (row n_0 also + pd)   : minus the contribution to the left cell
// Rows: [0] mass, [1] n_0, [2] n_1, [3] t_0, [4] t_1.  The left side comes as face-frame pairs with
// its scalars packed in the spare slots as in face2: Ln[M] = depth, Lt[M] = bed, Lgnn[2] = (um_x,
// s2_x), Lgnt[2] = (s1_x, um_y), Ln[M+1] = (s2_y, s1_y), Lt[M+1] = wave speeds.
__device__ __forceinline__ void face_c(const F2 *Ln, const F2 *Lt, const F2 *Lgnn, const F2 *Lgnt, const SideC &R,
                                       float g, float hdry, F2 scale, F2 *pr, F2 *mi)
{
    constexpr int m = CL_M;
    F2 hl, hr, dh;
    bool lowLx, lowLy;
    hr_faces(Ln[m], Lt[m], R.h, R.b, hl, hr, dh, lowLx, lowLy);
    const float hlx = hl.x(), hly = hl.y(), hrx = hr.x(), hry = hr.y();
    auto lower_speed = [&](float hs, float um, float s2, float s1) {
        const bool w = hs > hdry;
        const float t = sqrtf(fmaf(g, hs, w ? s2 : 0.0f));
        return t + (w ? um + s1 : 0.0f);
    };
    const float slowx = lower_speed(lowLx ? hlx : hrx, lowLx ? Lgnn[2].x() : R.um, lowLx ? Lgnn[2].y() : R.s2,
                                    lowLx ? Lgnt[2].x() : R.s1);
    const float slowy = lower_speed(lowLy ? hly : hry, lowLy ? Lgnt[2].y() : R.um, lowLy ? Ln[m + 1].x() : R.s2,
                                    lowLy ? Ln[m + 1].y() : R.s1);
    const float slx = lowLx ? slowx : Lt[m + 1].x(), srx = lowLx ? R.sc : slowx;
    const float sly = lowLy ? slowy : Lt[m + 1].y(), sry = lowLy ? R.sc : slowy;
    const F2 half = F2(0.5f) * scale;
    const F2 hs = half * F2(fmaxf(slx, srx), fmaxf(sly, sry));
    const F2 el(hlx > hdry ? hlx : 0.0f, hly > hdry ? hly : 0.0f);
    const F2 er(hrx > hdry ? hrx : 0.0f, hry > hdry ? hry : 0.0f);
    F2 qln[m], qlt[m], dn[m], dtv[m];
#pragma unroll
    for (int k = 0; k < m; ++k) {
        qln[k] = el * Ln[k];
        qlt[k] = el * Lt[k];
        dn[k] = er * R.n[k] - qln[k];
        dtv[k] = er * R.t[k] - qlt[k];
    }
    F2 fc[5];
    fc[0] = half * fma2(er, R.n[0], qln[0]) - hs * dh;
    fc[1] = half * fma2(el, Lgnn[0], er * R.gnn[0]) - hs * dn[0];
    fc[2] = half * fma2(el, Lgnn[1], er * R.gnn[1]) - hs * dn[1];
    fc[3] = half * fma2(el, Lgnt[0], er * R.gnt[0]) - hs * dtv[0];
    fc[4] = half * fma2(el, Lgnt[1], er * R.gnt[1]) - hs * dtv[1];
    const F2 pd = (F2(0.25f * g) * scale) * dh * (hr + hl);
    // 3-point Gauss-Legendre path integral of the closed profiles (weights W0, W1 as in face2)
    constexpr float sq15 = 0.38729833462074168852f;
    const float sn[3] = {0.5f - sq15, 0.5f, 0.5f + sq15};
    const float wq[3] = {5.0f / 18.0f, 8.0f / 18.0f, 5.0f / 18.0f};
    F2 W0(0.0f), W1(0.0f);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const F2 hq = fma2(F2(sn[q]), dh, hl);
        const F2 iw(hq.x() > hdry ? wq[q] * rcpa(hq.x()) : 0.0f, hq.y() > hdry ? wq[q] * rcpa(hq.y()) : 0.0f);
        W0 = W0 + iw;
        W1 = fma2(F2(sn[q]), iw, W1);
    }
    F2 nb[m], tb[m];
#pragma unroll
    for (int k = 0; k < m; ++k) {
        nb[k] = fma2(qln[k], W0, dn[k] * W1);
        tb[k] = fma2(qlt[k], W0, dtv[k] * W1);
    }
    // row 1 of the nonconservative product: sum over the columns l >= 1 of the closed profile
    F2 rn(0.0f), rt(0.0f);
    static_for<1, m>([&](auto ll) {
        constexpr int l = decltype(ll)::value;
        F2 en(0.0f), et(0.0f);
        static_for<0, m>([&](auto jj) {
            constexpr int j = decltype(jj)::value;
            constexpr double w = ncB(1, j, l);
            if constexpr (w != 0.0) {
                en = fma2(F2(float(w)), nb[j], en);
                et = fma2(F2(float(w)), tb[j], et);
            }
        });
        rn = fma2(en, dn[l], rn);
        rt = fma2(et, dn[l], rt);
    });
    const F2 nc2 = half * rn, nc4 = half * rt;
    pr[0] = fc[0];
    mi[0] = fc[0];
    pr[1] = fc[1] - pd;
    mi[1] = fc[1] + pd;
    pr[2] = fc[2] - nc2;
    mi[2] = fc[2] + nc2;
    pr[3] = fc[3];
    mi[3] = fc[3];
    pr[4] = fc[4] - nc4;
    mi[4] = fc[4] + nc4;
}

// Variable of frame row (mass, n_0, n_1, t_0, t_1) for the x-face (n = alpha) and the y-face (n = beta).
__device__ __forceinline__ constexpr int cl_xvar(int row) { return row == 0 ? 0 : row == 1 ? 1 : row == 2 ? 3 : row == 3 ? 2 : 4; }
__device__ __forceinline__ constexpr int cl_yvar(int row) { return row == 0 ? 0 : row == 1 ? 2 : row == 2 ? 4 : row == 3 ? 1 : 3; }

struct RowCtxC {
    const float *xcol, *bcol, *pcol;  // X, bed and predictions at the source column
    int ld, nx, ny, csrc, lane;
    int64_t pstride;
    bool owned, xwall;
};

// raw row: 5 state values, bed, 6 predictions
constexpr int CL_RAW = CL_NV + 1 + 6;

__device__ __forceinline__ void load_row_c(const RowCtxC &c, int r, float *dst, unsigned *status)
{
    const int rs = r < 0 ? 0 : (r >= c.ny ? c.ny - 1 : r);
    const int off = (int)bounds_idx(rs * c.nx + c.csrc, (int64_t)c.nx * c.ny, status) - c.csrc;
#pragma unroll
    for (int v = 0; v < CL_NV; ++v) dst[v] = __ldg(c.xcol + (off + v * c.ld));
    dst[CL_NV] = __ldg(c.bcol + off);
#pragma unroll
    for (int j = 0; j < 6; ++j) dst[CL_NV + 1 + j] = __ldg(c.pcol + ((int64_t)off + j * c.pstride));
}

template <int STAGE, bool STEADY = false>
__device__ __forceinline__ void row_body_c(const StageArgs<float> &a, const RowCtxC &c, int r, int r0, int r1, float dt,
                                           float *nxt, RowC &P, RowC &C, unsigned &flag)
{
    constexpr int m = CL_M;
    constexpr unsigned F = 0xffffffffu;
    const float g = a.g, hdry = a.hdry;
    const bool ywall = (r < 0 && a.bc[2] == 1) || (r >= c.ny && a.bc[3] == 1);
    float ih;
    make_side_c(C.s, nxt, nxt[CL_NV], nxt + CL_NV + 1, c.xwall, ywall, g, hdry, ih);
    {  // X + dt S_newton(X): rows 0 carry no bulk stress (phi_0' = 0); row 1 sums the closed moments
        const float f = -a.nu_rho * ih;
        float xa = 0.f, xb = 0.f;
        static_for<0, m>([&](auto ii) {
            constexpr int i = decltype(ii)::value;
            constexpr double w = visC(i, 1);
            if constexpr (w != 0.0) {
                xa = fmaf(float(w), C.s.n[i].x(), xa);
                xb = fmaf(float(w), C.s.n[i].y(), xb);
            }
        });
        C.acc[0] = nxt[0];
        C.acc[1] = nxt[1];
        C.acc[2] = nxt[2];
        C.acc[3] = fmaf(dt * f, xa, nxt[3]);
        C.acc[4] = fmaf(dt * f, xb, nxt[4]);
    }
    if (STEADY || r < r1) load_row_c(c, r + 1, nxt, &a.ctl->status);
    const bool xrow = STEADY || (r >= r0 && r < r1);
    const bool fin = STEADY || (r - 1 >= r0 && r - 1 < r1);
    // stage 2 updates Q^n in place: Q^n of the finished row comes from the addresses it is stored to
    float qn[CL_NV];
    float *const orow = a.out + (unsigned)((fin ? r - 1 : r0) * c.nx + c.csrc);
    if (STAGE == 2) {
#pragma unroll
        for (int v = 0; v < CL_NV; ++v) qn[v] = orow[(unsigned)(v * c.ld)];
    }
    F2 Ln[m + 2], Lt[m + 2], Lgnn[3], Lgnt[3];
#pragma unroll
    for (int k = 0; k < m; ++k) {
        Ln[k] = P.s.n[k];
        Ln[k].v.x = __shfl_up_sync(F, C.s.n[k].x(), 1);
        Lt[k] = P.s.t[k];
        Lt[k].v.x = __shfl_up_sync(F, C.s.t[k].x(), 1);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        Lgnn[k] = P.s.gnn[k];
        Lgnn[k].v.x = __shfl_up_sync(F, C.s.gnn[k].x(), 1);
        Lgnt[k] = P.s.gnt[k];
        Lgnt[k].v.x = __shfl_up_sync(F, C.s.gnt[k].x(), 1);
    }
    Ln[m] = F2(__shfl_up_sync(F, C.s.h, 1), P.s.h);
    Lt[m] = F2(__shfl_up_sync(F, C.s.b, 1), P.s.b);
    Lgnn[2] = F2(__shfl_up_sync(F, C.s.um, 1), __shfl_up_sync(F, C.s.s2, 1));
    Lgnt[2] = F2(__shfl_up_sync(F, C.s.s1, 1), P.s.um);
    Ln[m + 1] = F2(P.s.s2, P.s.s1);
    Lt[m + 1] = F2(__shfl_up_sync(F, C.s.sc, 1), P.s.sc);
    F2 pr[5], mi[5];
    face_c(Ln, Lt, Lgnn, Lgnt, C.s, g, hdry, F2(dt * a.inv_dx, dt * a.inv_dy), pr, mi);
    if (xrow) {
        float tl[CL_NV];
#pragma unroll
        for (int row = 0; row < 5; ++row) {
            C.acc[cl_xvar(row)] += pr[row].x();
            tl[cl_xvar(row)] = mi[row].x();
        }
#pragma unroll
        for (int v = 0; v < CL_NV; ++v) C.acc[v] -= __shfl_down_sync(F, tl[v], 1);
    }
    if (STEADY || r > r0 - 1) {
#pragma unroll
        for (int row = 0; row < 5; ++row) {
            C.acc[cl_yvar(row)] += pr[row].y();
            P.acc[cl_yvar(row)] -= mi[row].y();
        }
        if (fin) {
            // bottom stress, implicit in (alpha_0, alpha_1) with the closed moments frozen at the stage
            // input: rows (h alpha_0, h alpha_1) with weights (1, 3), Sherman-Morrison on the 2x2 rank-1
            const float h = P.acc[0];
            const bool wet = h > hdry;
            const float ihf = rcpa(h);
            const F2 sh = F2(h) * P.s.sig;  // closed momenta (h sum alpha_k, h sum beta_k)
            F2 y0(P.acc[1], P.acc[2]), y1(P.acc[3], P.acc[4]);
            float cc = 0.0f;
            if (a.fric == 1) {
                cc = a.C_rho * ihf;
            } else if (a.fric == 2) {
                const F2 ub = (y0 + y1 + sh) * F2(ihf);
                cc = a.gn2 * sqrtf(fmaf(ub.x(), ub.x(), ub.y() * ub.y())) * ihf * rcpa(cbrtf(h));
            }
            const float dc = dt * cc;
            const F2 r0v = y0 - F2(dc) * sh, r1v = y1 - F2(3.0f * dc) * sh;
            const float f = dc * rcpa(fmaf(dc, 4.0f, 1.0f));
            const F2 fab = F2(f) * (r0v + r1v);
            y0 = r0v - fab;
            y1 = r1v - F2(3.0f) * fab;
            float y[CL_NV];
            y[0] = h;
            y[1] = wet ? y0.x() : 0.0f;
            y[2] = wet ? y0.y() : 0.0f;
            y[3] = wet ? y1.x() : 0.0f;
            y[4] = wet ? y1.y() : 0.0f;
            if (STAGE == 2) {
                unsigned fl = 0;
#pragma unroll
                for (int v = 0; v < CL_NV; ++v) {
                    y[v] = 0.5f * (qn[v] + y[v]);
                    if (!(fabsf(y[v]) <= 3.0e38f)) fl |= DEV_NAN;
                }
                if (y[0] < 0.0f) fl |= DEV_NEGDEPTH;
                flag |= c.owned ? fl : 0u;
            }
            if (c.owned) {
#pragma unroll
                for (int v = 0; v < CL_NV; ++v) orow[(unsigned)(v * c.ld)] = y[v];
            }
        }
    }
}

__device__ __forceinline__ void zero_row_c(RowC &S)
{
    S.s.h = S.s.b = S.s.um = S.s.s2 = S.s.s1 = S.s.sc = 0.0f;
#pragma unroll
    for (int k = 0; k < CL_M; ++k) S.s.n[k] = S.s.t[k] = F2(0.0f);
#pragma unroll
    for (int k = 0; k < 2; ++k) S.s.gnn[k] = S.s.gnt[k] = F2(0.0f);
    S.s.sig = F2(0.0f);
#pragma unroll
    for (int v = 0; v < CL_NV; ++v) S.acc[v] = 0.0f;
}

// One warp marches its strip over the rows of segment seg (see march_strip in struct2d_f32.cuh).
template <int STAGE>
__device__ __forceinline__ void march_strip_c(const ClosureArgs &ca, int strip, int seg, int lane, float dt,
                                              unsigned &flag)
{
    const StageArgs<float> &a = ca.s;
    RowCtxC c;
    c.lane = lane;
    const int col = strip * 30 - 1 + lane;
    c.nx = a.nx;
    c.ny = a.ny;
    c.ld = (int)a.ld;
    c.pstride = ca.pstride;
    c.owned = lane >= 1 && lane <= 30 && col < a.nx;
    c.csrc = col < 0 ? 0 : (col >= a.nx ? a.nx - 1 : col);
    c.xwall = (col < 0 && a.bc[0] == 1) || (col >= a.nx && a.bc[1] == 1);
    c.xcol = a.X + c.csrc;
    c.bcol = a.bed + c.csrc;
    c.pcol = ca.pred + c.csrc;
    const int r0 = seg * a.H;
    const int r1 = min(r0 + a.H, a.ny);
    RowC A, B;
    zero_row_c(A);
    zero_row_c(B);
    float nxt[CL_RAW];
    load_row_c(c, r0 - 1, nxt, &a.ctl->status);
    int r = r0 - 1;
    while (true) {  // general pairs at both ends of the segment, branch-free pairs inside it
        row_body_c<STAGE>(a, c, r, r0, r1, dt, nxt, B, A, flag);
        if (r + 1 <= r1) row_body_c<STAGE>(a, c, r + 1, r0, r1, dt, nxt, A, B, flag);
        r += 2;
        if (r > r1) break;
        for (; r + 1 < r1; r += 2) {
            row_body_c<STAGE, true>(a, c, r, r0, r1, dt, nxt, B, A, flag);
            row_body_c<STAGE, true>(a, c, r + 1, r0, r1, dt, nxt, A, B, flag);
        }
    }
}

}  // namespace zoomy
