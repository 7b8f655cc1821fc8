// struct2d_f32.cuh -- device code of the FP32 structured-grid stage (row-marching warps with
// packed f32x2 face pairs), shared by the single-grid kernel (fv_struct2d_f32.cu) and the batched
// ensemble kernel (fv_ensemble.cu).  See fv_struct2d_f32.cu for the design.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "f32x2.cuh"
#include "fv_common.cuh"
#include "model.cuh"

namespace zoomy {

// 1/x from the MUFU reciprocal (about 1 ulp, no slow path for special values).
__device__ __forceinline__ float rcpa(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// A cell as seen by its two faces.  Scalars are frame-free; the pairs hold the x-face frame
// (n = alpha, t = beta) in .x and the y-face frame (n = beta, t = alpha) in .y.
template <int N>
struct Side2 {
    static constexpr int m = N + 1;
    float h, b, um, s2, s1, sc;  // depth, bed, |u_mean|, sum_{k>=1}|a_k|^2, sum_{k>=2}|a_k|, wave speed
    F2 n[m], t[m], gnn[m], gnt[m];
};

template <int N>
struct RowState {
    static constexpr int nv = 3 + 2 * N;
    Side2<N> s;
    float acc[nv];  // X + dt S_newton(X) + dt * (face terms so far)
};

// Primitive recovery, wave-speed parts and flux products of a cell, packed for its faces.
template <int N>
__device__ __forceinline__ void make_side(Side2<N> &r, float h, float b, const float *ha, const float *hb, float g,
                                          float hdry, float &ih)
{
    constexpr int m = N + 1;
    ih = h > hdry ? rcpa(h) : 0.0f;
    float a[m], c[m];
#pragma unroll
    for (int k = 0; k < m; ++k) {
        a[k] = ha[k] * ih;
        c[k] = hb[k] * ih;
    }
    r.h = h;
    r.b = b;
    r.um = sqrtf(fmaf(a[0], a[0], c[0] * c[0]));
    float s2 = 0.f, s1 = 0.f;
#pragma unroll
    for (int k = 1; k < m; ++k) {
        const float q = fmaf(a[k], a[k], c[k] * c[k]);
        s2 += q;
        if (k >= 2) s1 += sqrtf(q);
    }
    r.s2 = s2;
    r.s1 = s1;
    r.sc = r.um + sqrtf(fmaf(g, fmaxf(h, 0.0f), s2)) + s1;
#pragma unroll
    for (int k = 0; k < m; ++k) {
        r.n[k] = F2(a[k], c[k]);
        r.t[k] = F2(c[k], a[k]);
    }
    // per unit depth flux products, (aa, bb) packed and ab duplicated
    static_for<0, m>([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        F2 sq(0.0f);
        float sab = 0.f;
        static_for<0, m>([&](auto ii) {
            constexpr int i = decltype(ii)::value;
            static_for<0, m>([&](auto jj) {
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

// Hydrostatic depths of both faces (branch-free): hl, hr and hR* - hL*, with the FP64-grade
// bed/surface difference: h + (b - bf) of the lower side is formed by two TwoSums (the exact pair of
// model.cuh's hr_depth), evaluated for the x- and the y-face at once with packed additions.
__device__ __forceinline__ void hr_faces(F2 hL, F2 bL, float hR, float bR, F2 &hl, F2 &hr, F2 &dh, bool &lowLx,
                                         bool &lowLy)
{
    lowLx = bL.x() < bR;
    lowLy = bL.y() < bR;
    const F2 bf(fmaxf(bL.x(), bR), fmaxf(bL.y(), bR));
    const F2 h(lowLx ? hL.x() : hR, lowLy ? hL.y() : hR);
    const F2 b(lowLx ? bL.x() : bR, lowLy ? bL.y() : bR);
    const F2 s = b - bf;
    const F2 bb = s - b;
    const F2 e = (b - (s - bb)) - (bf + bb);
    const F2 r = h + s;
    const F2 bb2 = r - h;
    const F2 e2 = (h - (r - bb2)) + (s - bb2);
    F2 lo = e2 + e;
    F2 hi = r + lo;
    lo = lo - (hi - r);
    const bool px = hi.x() > 0.0f, py = hi.y() > 0.0f;
    hi = F2(px ? hi.x() : 0.0f, py ? hi.y() : 0.0f);
    lo = F2(px ? lo.x() : 0.0f, py ? lo.y() : 0.0f);
    const F2 hh(fmaxf(lowLx ? hR : hL.x(), 0.0f), fmaxf(lowLy ? hR : hL.y(), 0.0f));  // higher side
    hl = F2(lowLx ? hi.x() : hh.x(), lowLy ? hi.y() : hh.y());
    hr = F2(lowLx ? hh.x() : hi.x(), lowLy ? hh.y() : hi.y());
    const F2 sl(lowLx ? -lo.x() : lo.x(), lowLy ? -lo.y() : lo.y());
    dh = (hr - hl) + sl;
}

// Face terms for the pair of faces (formulas of face_term in model.cuh), returned as
//   pr = dt/|Omega| |e| (fc - nc) (row n_0 also - pd)   : contribution to the right cell
//   mi = dt/|Omega| |e| (fc + nc) (row n_0 also + pd)   : minus the contribution to the left cell
// Layout: [0] mass, [1+k] row n_k, [1+m+k] row t_k.
// The left side arrives as face-frame pairs Ln/Lt/Lgnn/Lgnt[0..N] plus its scalars packed in the
// spare slots: Ln[m] = depth, Lt[m] = bed, Lgnn[m] = (um_x, s2_x), Lgnt[m] = (s1_x, um_y),
// Ln[m+1] = (s2_y, s1_y), Lt[m+1] = wave speed.
template <int N>
__device__ __forceinline__ void face2(const F2 *Ln, const F2 *Lt, const F2 *Lgnn, const F2 *Lgnt, const Side2<N> &R,
                                      float g, float hdry, F2 scale, F2 *pr, F2 *mi)
{
    constexpr int m = N + 1;
    F2 hl, hr, dh;
    bool lowLx, lowLy;
    hr_faces(Ln[m], Lt[m], R.h, R.b, hl, hr, dh, lowLx, lowLy);
    const float hlx = hl.x(), hly = hl.y(), hrx = hr.x(), hry = hr.y();
    // wave speed of the lower side at its reconstructed depth; the higher side keeps its own
    auto lower_speed = [&](float hs, float um, float s2, float s1) {
        const bool w = hs > hdry;
        const float t = sqrtf(fmaf(g, hs, w ? s2 : 0.0f));
        return t + (w ? um + s1 : 0.0f);
    };
    const float slowx = lower_speed(lowLx ? hlx : hrx, lowLx ? Lgnn[m].x() : R.um, lowLx ? Lgnn[m].y() : R.s2,
                                    lowLx ? Lgnt[m].x() : R.s1);
    const float slowy = lower_speed(lowLy ? hly : hry, lowLy ? Lgnt[m].y() : R.um, lowLy ? Ln[m + 1].x() : R.s2,
                                    lowLy ? Ln[m + 1].y() : R.s1);
    const float slx = lowLx ? slowx : Lt[m + 1].x(), srx = lowLx ? R.sc : slowx;
    const float sly = lowLy ? slowy : Lt[m + 1].y(), sry = lowLy ? R.sc : slowy;
    // every face term is multiplied by scale = dt |e| / |Omega|: fold it into the constants
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
    F2 fc[1 + 2 * m];
    fc[0] = half * fma2(er, R.n[0], qln[0]) - hs * dh;
#pragma unroll
    for (int k = 0; k < m; ++k) {
        fc[1 + k] = half * fma2(el, Lgnn[k], er * R.gnn[k]) - hs * dn[k];
        fc[1 + m + k] = half * fma2(el, Lgnt[k], er * R.gnt[k]) - hs * dtv[k];
    }
    const F2 pd = (F2(0.25f * g) * scale) * dh * (hr + hl);
    F2 nc[1 + 2 * m];
    if constexpr (N >= 1) {
        // sum_q w_q (QL* + s_q dQ)/h(s_q) = QL* W0 + dQ W1 (wet nodes only), 3-point Gauss-Legendre
        constexpr float sq15 = 0.38729833462074168852f;
        const float sn[3] = {0.5f - sq15, 0.5f, 0.5f + sq15};
        const float wq[3] = {5.0f / 18.0f, 8.0f / 18.0f, 5.0f / 18.0f};
        F2 W0(0.0f), W1(0.0f);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const F2 hq = fma2(F2(sn[q]), dh, hl);
            const F2 iw(hq.x() > hdry ? wq[q] * rcpa(hq.x()) : 0.0f,
                        hq.y() > hdry ? wq[q] * rcpa(hq.y()) : 0.0f);
            W0 = W0 + iw;
            W1 = fma2(F2(sn[q]), iw, W1);
        }
        F2 nb[m], tb[m];
#pragma unroll
        for (int k = 0; k < m; ++k) {
            nb[k] = fma2(qln[k], W0, dn[k] * W1);
            tb[k] = fma2(qlt[k], W0, dtv[k] * W1);
        }
        static_for<1, m>([&](auto kk) {
            constexpr int k = decltype(kk)::value;
            F2 rn(0.0f), rt(0.0f);
            static_for<1, m>([&](auto ll) {
                constexpr int l = decltype(ll)::value;
                F2 en(0.0f), et(0.0f);
                static_for<0, m>([&](auto jj) {
                    constexpr int j = decltype(jj)::value;
                    constexpr double w = ncB(k, j, l);
                    if constexpr (w != 0.0) {
                        en = fma2(F2(float(w)), nb[j], en);
                        et = fma2(F2(float(w)), tb[j], et);
                    }
                });
                rn = fma2(en, dn[l], rn);
                rt = fma2(et, dn[l], rt);
            });
            nc[1 + k] = half * rn;
            nc[1 + m + k] = half * rt;
        });
    }
#pragma unroll
    for (int k = 0; k < 1 + 2 * m; ++k) {
        const bool has_nc = (N >= 1) && ((k >= 2 && k <= m) || k >= m + 2);
        if (has_nc) {
            pr[k] = fc[k] - nc[k];
            mi[k] = fc[k] + nc[k];
        } else {
            pr[k] = fc[k];
            mi[k] = fc[k];
        }
    }
    pr[1] = pr[1] - pd;
    mi[1] = mi[1] + pd;
}

// Bottom stress (implicit, rank-1 Sherman-Morrison) and dry cut, branch-free (see
// bottom_friction in model.cuh).
template <int N>
__device__ __forceinline__ void friction32(float h, float *ya, float *yb, int fric, float C_rho, float gn2, float dt,
                                           float hdry)
{
    constexpr int m = N + 1;
    const bool wet = h > hdry;
    float sa = 0.f, sb = 0.f;
#pragma unroll
    for (int k = 0; k < m; ++k) {
        sa += ya[k];
        sb += yb[k];
    }
    const float ih = rcpa(h);
    float c = 0.0f;
    if (fric == 1) {
        c = C_rho * ih;
    } else if (fric == 2) {
        const float ub = sa * ih, vb = sb * ih;
        c = gn2 * sqrtf(fmaf(ub, ub, vb * vb)) * ih * rcpa(cbrtf(h));
    }
    const float dc = dt * c;
    const float f = dc * rcpa(fmaf(dc, float(m * m), 1.0f));
    const float fa = __fmul_rn(f, sa), fb = __fmul_rn(f, sb);  // never contracted into the update below
#pragma unroll
    for (int k = 0; k < m; ++k) {
        ya[k] = wet ? fmaf(-float(2 * k + 1), fa, ya[k]) : 0.0f;
        yb[k] = wet ? fmaf(-float(2 * k + 1), fb, yb[k]) : 0.0f;
    }
}

struct RowCtx {
    const float *xcol;   // X + csrc
    const float *bcol;   // bed + csrc (or nullptr)
    int ld, nx, ny, csrc, col, lane;
    bool owned, xwall;
};

template <int N, int STAGE>
__device__ __forceinline__ void load_row(const StageArgs<float> &a, const RowCtx &c, int r, float *dst)
{
    constexpr int nv = 3 + 2 * N;
    const int rs = r < 0 ? 0 : (r >= c.ny ? c.ny - 1 : r);
    const int off = (int)bounds_idx(rs * c.nx + c.csrc, (int64_t)c.nx * c.ny, &a.ctl->status) - c.csrc;
#pragma unroll
    for (int v = 0; v < nv; ++v) dst[v] = __ldg(c.xcol + (off + v * c.ld));
    dst[nv] = __ldg(c.bcol + off);
}

// Process row r with the previous row state P and the current row state C.  IMP: the friction
// (bulk + bottom stress) by backward Euler after the stage instead of the default treatment.
template <int N, int STAGE, bool IMP = false, bool STEADY = false>
__device__ __forceinline__ void row_body(const StageArgs<float> &a, const RowCtx &c, int r, int r0, int r1, float dt,
                                         float *nxt, RowState<N> &P, RowState<N> &C, float &smax, unsigned &flag)
{
    constexpr int m = N + 1, nv = 3 + 2 * N;
    constexpr unsigned F = 0xffffffffu;
    const float g = a.g, hdry = a.hdry;
    // ---- the cell of this row (raw values were prefetched into nxt) -------------------------
    const bool ywall = (r < 0 && a.bc[2] == 1) || (r >= c.ny && a.bc[3] == 1);
    float ha[m], hb[m];
#pragma unroll
    for (int k = 0; k < m; ++k) {
        ha[k] = c.xwall ? -nxt[var_a<N, 2>(k)] : nxt[var_a<N, 2>(k)];
        hb[k] = ywall ? -nxt[var_b<N>(k)] : nxt[var_b<N>(k)];
    }
    float ih;
    make_side<N>(C.s, nxt[0], nxt[nv], ha, hb, g, hdry, ih);
    // accumulator starts at X + dt S_newton(X): -(nu/rho) / h^2 sum_i C_ik / M_k (h alpha_i)
    {
        const float f = -a.nu_rho * ih * ih;
        C.acc[0] = nxt[0];
        static_for<0, m>([&](auto kk) {
            constexpr int k = decltype(kk)::value;
            float xa = 0.f, xb = 0.f;
            static_for<0, m>([&](auto ii) {
                constexpr int i = decltype(ii)::value;
                constexpr double w = visC(i, k);
                if constexpr (w != 0.0) {
                    xa = fmaf(float(w), ha[i], xa);
                    xb = fmaf(float(w), hb[i], xb);
                }
            });
            C.acc[var_a<N, 2>(k)] = fmaf(dt * f, xa, ha[k]);
            C.acc[var_b<N>(k)] = fmaf(dt * f, xb, hb[k]);
        });
    }
    // ---- prefetch the next row, and Q^n of the row finished in this step --------------------
    // STEADY: a row strictly inside the segment (r0 < r < r1): every flag below is true
    if (STEADY || r < r1) load_row<N, STAGE>(a, c, r + 1, nxt);
    const bool xrow = STEADY || (r >= r0 && r < r1);
    const bool fin = STEADY || (r - 1 >= r0 && r - 1 < r1);  // row r-1 is finished by this step
    // Stage 2 updates Q^n in place (the launcher checks out == Qn): Q^n of the finished row is read
    // from the addresses its result is stored to.
    float qn[nv];
    float *const orow = a.out + (unsigned)((fin ? r - 1 : r0) * c.nx + c.csrc);
    if (STAGE == 2) {
#pragma unroll
        for (int v = 0; v < nv; ++v) qn[v] = orow[(unsigned)(v * c.ld)];
        if (xrow) {  // bring Q^n of this row into L2; it is read when the row is finished
#pragma unroll
            for (int v = 0; v < nv; ++v)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(orow + (unsigned)(c.nx + v * c.ld)));
        }
    }
    // ---- left neighbour (x-face) from the lane on the left, lower neighbour (y-face) from P ----
    // Ln/Lt/Lgnn/Lgnt carry the face-frame pairs; index m / m+1 carry (h, b), (um, s2), (s1, sc).
    // The x halves of P's pairs are dead (P's own x-face is done), so each pair is reused with the
    // shuffled value written into its x half.
    F2 Ln[m + 2], Lt[m + 2], Lgnn[m + 1], Lgnt[m + 1];
#pragma unroll
    for (int k = 0; k < m; ++k) {
        Ln[k] = P.s.n[k];
        Ln[k].v.x = __shfl_up_sync(F, C.s.n[k].x(), 1);
        Lt[k] = P.s.t[k];
        Lt[k].v.x = __shfl_up_sync(F, C.s.t[k].x(), 1);
        Lgnn[k] = P.s.gnn[k];
        Lgnn[k].v.x = __shfl_up_sync(F, C.s.gnn[k].x(), 1);
        Lgnt[k] = P.s.gnt[k];
        Lgnt[k].v.x = __shfl_up_sync(F, C.s.gnt[k].x(), 1);
    }
    Ln[m] = F2(__shfl_up_sync(F, C.s.h, 1), P.s.h);      // depth
    Lt[m] = F2(__shfl_up_sync(F, C.s.b, 1), P.s.b);      // bed
    Lgnn[m] = F2(__shfl_up_sync(F, C.s.um, 1), __shfl_up_sync(F, C.s.s2, 1));  // x-face: um, s2
    Lgnt[m] = F2(__shfl_up_sync(F, C.s.s1, 1), P.s.um);  // x: s1, y: um
    Ln[m + 1] = F2(P.s.s2, P.s.s1);                      // y: s2, s1
    Lt[m + 1] = F2(__shfl_up_sync(F, C.s.sc, 1), P.s.sc);  // wave speeds
    F2 pr[1 + 2 * m], mi[1 + 2 * m];
    face2<N>(Ln, Lt, Lgnn, Lgnt, C.s, g, hdry, F2(dt * a.inv_dx, dt * a.inv_dy), pr, mi);
    // ---- scatter: x-face (.x) frame rows (alpha, beta); y-face (.y) frame rows (beta, alpha) ----
    const bool yrow = STEADY || r > r0 - 1;
    if (xrow) {
        float tl[nv];
        C.acc[0] += pr[0].x();
        tl[0] = mi[0].x();
#pragma unroll
        for (int k = 0; k < m; ++k) {
            C.acc[var_a<N, 2>(k)] += pr[1 + k].x();
            C.acc[var_b<N>(k)] += pr[1 + m + k].x();
            tl[var_a<N, 2>(k)] = mi[1 + k].x();
            tl[var_b<N>(k)] = mi[1 + m + k].x();
        }
#pragma unroll
        for (int v = 0; v < nv; ++v) C.acc[v] -= __shfl_down_sync(F, tl[v], 1);
    }
    if (yrow) {
        C.acc[0] += pr[0].y();
        P.acc[0] -= mi[0].y();
#pragma unroll
        for (int k = 0; k < m; ++k) {
            C.acc[var_b<N>(k)] += pr[1 + k].y();
            C.acc[var_a<N, 2>(k)] += pr[1 + m + k].y();
            P.acc[var_b<N>(k)] -= mi[1 + k].y();
            P.acc[var_a<N, 2>(k)] -= mi[1 + m + k].y();
        }
        // ---- the row below is complete: bottom stress, dry cut, SSP-RK2 average, store -------
        // (computed by every lane; only the lanes that own a cell store it)
        if (fin) {
            float ya[m], yb[m];
#pragma unroll
            for (int k = 0; k < m; ++k) {
                ya[k] = P.acc[var_a<N, 2>(k)];
                yb[k] = P.acc[var_b<N>(k)];
            }
            const float h = P.acc[0];
            if constexpr (IMP)
                friction_implicit<N, 2, float>(h, ya, yb, a.fric, a.C_rho, a.nu_imp, a.gn2, dt, hdry);
            else
                friction32<N>(h, ya, yb, a.fric, a.C_rho, a.gn2, dt, hdry);
            float y[nv];
            y[0] = h;
#pragma unroll
            for (int k = 0; k < m; ++k) {
                y[var_a<N, 2>(k)] = ya[k];
                y[var_b<N>(k)] = yb[k];
            }
            if (STAGE == 2) {
#pragma unroll
                for (int v = 0; v < nv; ++v) y[v] = 0.5f * (qn[v] + y[v]);
                const float hy = y[0];
                const float ihh = hy > hdry ? rcpa(hy) : 0.0f;
                const float u0 = y[var_a<N, 2>(0)] * ihh, v0 = y[var_b<N>(0)] * ihh;
                float s2 = 0.f, s1 = 0.f;
#pragma unroll
                for (int k = 1; k < m; ++k) {
                    const float ak = y[var_a<N, 2>(k)] * ihh, bk = y[var_b<N>(k)] * ihh;
                    const float q = fmaf(ak, ak, bk * bk);
                    s2 += q;
                    if (k >= 2) s1 += sqrtf(q);
                }
                const float s = sqrtf(fmaf(u0, u0, v0 * v0)) + sqrtf(fmaf(g, fmaxf(hy, 0.0f), s2)) + s1;
                unsigned fl = 0;
                if (!(s <= 3.0e38f)) fl |= DEV_NAN;
                if (!(hy >= 0.0f)) fl |= (hy < 0.0f) ? DEV_NEGDEPTH : DEV_NAN;
                flag |= c.owned ? fl : 0u;
                const float so = c.owned ? s : 0.0f;
                smax = (so > smax || so != so) ? so : smax;
            }
            if (c.owned) {  // (fin: orow is row r - 1; an owned lane's column is its source column)
#pragma unroll
                for (int v = 0; v < nv; ++v) orow[(unsigned)(v * c.ld)] = y[v];
            }
        }
    }
}

template <int N>
__device__ __forceinline__ void zero_state(RowState<N> &S)
{
    constexpr int m = N + 1, nv = 3 + 2 * N;
    S.s.h = S.s.b = S.s.um = S.s.s2 = S.s.s1 = S.s.sc = 0.0f;
#pragma unroll
    for (int k = 0; k < m; ++k) S.s.n[k] = S.s.t[k] = S.s.gnn[k] = S.s.gnt[k] = F2(0.0f);
#pragma unroll
    for (int v = 0; v < nv; ++v) S.acc[v] = 0.0f;
}

// One warp marches its strip (30 columns) over the rows of segment seg: the whole stage for those
// cells.  smax / flag accumulate the wave speed and status of the cells the lane finishes (stage 2).
template <int N, int STAGE, bool IMP = false, bool PEEL = true>
__device__ __forceinline__ void march_strip(const StageArgs<float> &a, int strip, int seg, int lane, float dt,
                                            float &smax, unsigned &flag)
{
    constexpr int nv = 3 + 2 * N;
    RowCtx c;
    c.lane = lane;
    c.col = strip * 30 - 1 + lane;
    c.nx = a.nx;
    c.ny = a.ny;
    c.ld = (int)a.ld;
    c.owned = lane >= 1 && lane <= 30 && c.col < a.nx;
    c.csrc = c.col < 0 ? 0 : (c.col >= a.nx ? a.nx - 1 : c.col);
    c.xwall = (c.col < 0 && a.bc[0] == 1) || (c.col >= a.nx && a.bc[1] == 1);
    c.xcol = a.X + c.csrc;
    c.bcol = a.bed + c.csrc;  // the host always provides a bed array (zeros for a flat bed)
    const int r0 = seg * a.H;
    const int r1 = min(r0 + a.H, a.ny);

    RowState<N> A, B;
    zero_state<N>(A);
    zero_state<N>(B);
    float nxt[nv + 1];
    load_row<N, STAGE>(a, c, r0 - 1, nxt);
    if constexpr (PEEL) {
        // pairs of rows with the general flags at both ends of the segment (rows r0 - 1 and r0, then
        // the last one or two), pairs strictly inside it without any test (one straight block per
        // pair, so consecutive rows' independent work can overlap).  Row r uses A as its current state
        // when r - r0 is odd.
        int r = r0 - 1;
        while (true) {
            row_body<N, STAGE, IMP>(a, c, r, r0, r1, dt, nxt, B, A, smax, flag);
            if (r + 1 <= r1) row_body<N, STAGE, IMP>(a, c, r + 1, r0, r1, dt, nxt, A, B, smax, flag);
            r += 2;
            if (r > r1) break;
            for (; r + 1 < r1; r += 2) {
                row_body<N, STAGE, IMP, true>(a, c, r, r0, r1, dt, nxt, B, A, smax, flag);
                row_body<N, STAGE, IMP, true>(a, c, r + 1, r0, r1, dt, nxt, A, B, smax, flag);
            }
        }
    } else {
        for (int r = r0 - 1; r <= r1; r += 2) {
            row_body<N, STAGE, IMP>(a, c, r, r0, r1, dt, nxt, B, A, smax, flag);
            if (r + 1 <= r1) row_body<N, STAGE, IMP>(a, c, r + 1, r0, r1, dt, nxt, A, B, smax, flag);
        }
    }
}

}  // namespace zoomy
