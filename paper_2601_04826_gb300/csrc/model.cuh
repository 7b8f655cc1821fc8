// model.cuh -- device form of the level-N shallow-moment model and its face terms.
//
// Model: Eq. (sme) (Sec. 1) and the 2D SME system of Sec. 3.4, written as
//   d_t Q + div F(Q) + B(Q) grad Q = S(Q)                       (Eq. (PDE-structure))
// with Q = (h, h alpha_0, h beta_0, h alpha_1..h alpha_N, h beta_1..h beta_N) in 2D and
// Q = (h, h alpha_0..h alpha_N) in 1D.
//
// All face work is done in the frame of the face: "n" moments are the velocity
// moments along the face normal and "t" moments the transverse ones.  The model is
// rotation- and reflection-invariant, so an x-face uses (n, t) = (alpha, beta) and a
// y-face (n, t) = (beta, alpha).  In that frame, per unit depth,
//   F_n = h * ( n_0,  sum_ij n_i n_j A_ijk/M_k,  sum_ij n_i t_j A_ijk/M_k ) + g h^2/2 on row n_0,
// and the nonconservative product has rows k >= 1 and columns l >= 1 only:
//   (B_n dQ)_{n_k} = sum_{j>=0} n_j B_kjl/M_k d(h n_l),  (B_n dQ)_{t_k} = sum_{j>=0} t_j B_kjl/M_k d(h n_l),
// whose j = 0 term is the -u_m d(h n_k) of Eq. (sme) (B_k0l/M_k = -delta_kl).
#pragma once
#include <cuda_runtime.h>

#include "basis.cuh"

namespace zoomy {

template <typename T>
__device__ __forceinline__ T dev_div(T a, T b);
template <>
__device__ __forceinline__ float dev_div<float>(float a, float b)
{
    return __fdividef(a, b);
}
template <>
__device__ __forceinline__ double dev_div<double>(double a, double b)
{
    return a / b;
}

template <typename T>
__device__ __forceinline__ T dev_sqrt(T a)
{
    return sqrt(a);
}

// Hydrostatic reconstruction depth h* = max(0, h + b - bf) (Audusse et al.), the bed/surface
// difference the method needs in FP64 precision.  In FP32 it is returned as an unevaluated pair
// hi + lo equal to h + b - bf up to about 2^-46 relative: the sum is formed by two error-free
// additions (Knuth's TwoSum), so the face differences hR* - hL* that drive the pressure and mass
// terms keep the accuracy of an FP64 evaluation even where they are far below the FP32
// resolution of h.  On the higher side (b == bf) h* = h exactly.
struct HPair {
    float hi, lo;
};
__device__ __forceinline__ HPair hr_depth(float h, float b, float bf)
{
    if (b >= bf) return {fmaxf(h, 0.0f), 0.0f};
    float s = b - bf;
    float bb = s - b;
    float e = (b - (s - bb)) + (-bf - bb);
    float r = h + s;
    float bb2 = r - h;
    float e2 = (h - (r - bb2)) + (s - bb2);
    float lo = e2 + e;
    float hi = r + lo;             // rounded depth
    lo = lo - (hi - r);            // remainder, |lo| <= ulp(hi)/2 (Fast2Sum, |r| >= |lo|)
    if (hi <= 0.0f) return {0.0f, 0.0f};
    return {hi, lo};
}
__device__ __forceinline__ float hp_diff(HPair r, HPair l) { return (r.hi - l.hi) + (r.lo - l.lo); }
__device__ __forceinline__ float hp_val(HPair a) { return a.hi; }

struct DPair {
    double hi;
};
__device__ __forceinline__ DPair hr_depth(double h, double b, double bf)
{
    double hs = (h + b) - bf;
    return {hs > 0.0 ? hs : 0.0};
}
__device__ __forceinline__ double hp_diff(DPair r, DPair l) { return r.hi - l.hi; }
__device__ __forceinline__ double hp_val(DPair a) { return a.hi; }

// One cell, primitive form, with the per-unit-depth flux products it contributes to faces.
template <int N, int D, typename T>
struct CellRec {
    static constexpr int m = N + 1;
    static constexpr int mt = (D == 2) ? N + 1 : 1;
    T h, b;
    T a[m];      // alpha_k (x moments), zero if dry
    T c[mt];     // beta_k (y moments), zero if dry
    T um, s2, s1;  // |mean velocity|, sum_{k>=1} |a_k|^2, sum_{k>=2} |a_k|
    T ih;          // 1/h if wet, else 0 (FP64 records; the Newtonian source reuses it)
    T gaa[m];    // sum_ij alpha_i alpha_j A_ijk / M_k
    T gab[mt];   // sum_ij alpha_i beta_j A_ijk / M_k
    T gbb[mt];   // sum_ij beta_i beta_j A_ijk / M_k
};

// Primitive recovery (velocities zero where h <= h_dry), wave-speed parts, flux products.
template <int N, int D, typename T>
__device__ __forceinline__ void make_cell(CellRec<N, D, T> &r, T h, T b, const T *ha, const T *hb, T hdry)
{
    constexpr int m = N + 1;
    r.h = h;
    r.b = b;
    const bool wet = h > hdry;
    if constexpr (sizeof(T) == 8) {
        // FP64: one division per cell (the FP64 path is bound by its division chains on GB300); the
        // moments are within an ulp of h alpha_k / h
        const T ih = wet ? T(1) / h : T(0);
        r.ih = ih;
#pragma unroll
        for (int k = 0; k < m; ++k) r.a[k] = ha[k] * ih;
        if constexpr (D == 2) {
#pragma unroll
            for (int k = 0; k < m; ++k) r.c[k] = hb[k] * ih;
        }
    } else {
        r.ih = T(0);  // not used in FP32
#pragma unroll
        for (int k = 0; k < m; ++k) r.a[k] = wet ? dev_div(ha[k], h) : T(0);
        if constexpr (D == 2) {
#pragma unroll
            for (int k = 0; k < m; ++k) r.c[k] = wet ? dev_div(hb[k], h) : T(0);
        }
    }
    if constexpr (D == 2)
        r.um = dev_sqrt(r.a[0] * r.a[0] + r.c[0] * r.c[0]);
    else
        r.um = fabs(r.a[0]);
    T s2 = 0, s1 = 0;
#pragma unroll
    for (int k = 1; k < m; ++k) {
        T q = r.a[k] * r.a[k];
        if constexpr (D == 2) q += r.c[k] * r.c[k];
        s2 += q;
        if (k >= 2) {
            if constexpr (D == 2)
                s1 += dev_sqrt(q);
            else
                s1 += fabs(r.a[k]);
        }
    }
    r.s2 = s2;
    r.s1 = s1;
    static_for<0, m>([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        T saa = 0;
        [[maybe_unused]] T sab = 0, sbb = 0;  // 2D only
        static_for<0, m>([&](auto ii) {
            constexpr int i = decltype(ii)::value;
            static_for<0, m>([&](auto jj) {
                constexpr int j = decltype(jj)::value;
                constexpr double w = fluxA(i, j, k);
                if constexpr (w != 0.0) {
                    if constexpr (j >= i) {  // A is symmetric in i, j: pair the terms of alpha_i alpha_j
                        constexpr double w2 = (i == j) ? w : 2.0 * w;
                        saa += T(w2) * r.a[i] * r.a[j];
                        if constexpr (D == 2) sbb += T(w2) * r.c[i] * r.c[j];
                    }
                    if constexpr (D == 2) sab += T(w) * r.a[i] * r.c[j];
                }
            });
        });
        r.gaa[k] = saa;
        if constexpr (D == 2) {
            r.gab[k] = sab;
            r.gbb[k] = sbb;
        }
    });
}

// View of a cell in a face frame.
template <int N, int D, typename T>
struct FrameView {
    const T *n, *t, *gnn, *gnt;
};

template <int N, int D, typename T, bool YDIR>
__device__ __forceinline__ FrameView<N, D, T> frame(const CellRec<N, D, T> &r)
{
    if constexpr (YDIR)
        return {r.c, r.a, r.gbb, r.gab};
    else
        return {r.a, r.c, r.gaa, r.gab};
}

// Face term of the path-conservative Rusanov scheme with hydrostatic reconstruction, in the
// frame of a face whose normal points from L to R (Eq. (PDE-hyperbolic); Sec. 2.1.2, the
// path-conservative FV scheme for nonconservative systems; Audusse et al. reconstruction):
//   fc = 1/2 (F_n(QL*) + F_n(QR*)) - 1/2 s_f (QR* - QL*)   without the pressure g h^2/2
//   pd = 1/2 (P(hR*) - P(hL*)),  P(h) = g h^2 / 2           (row n_0 only)
//   nc = 1/2 Btilde (QR* - QL*), Btilde = sum_q w_q B_n(QL* + s_q (QR* - QL*)), 3-point Gauss
// Cell L receives -(fc + pd + nc) and cell R receives +(fc - pd - nc), times |e|/|Omega|.
// Layout of fc / nc: [0] mass, [1 + k] row n_k, [1 + m + k] row t_k (2D only).
template <int N, int D, typename T>
__device__ __forceinline__ void face_term(const CellRec<N, D, T> &L, const FrameView<N, D, T> &FL,
                                          const CellRec<N, D, T> &R, const FrameView<N, D, T> &FR, T g, T hdry,
                                          T *fc, T &pd, T *nc)
{
    constexpr int m = N + 1;
    const T bf = L.b > R.b ? L.b : R.b;
    const auto hpl = hr_depth(L.h, L.b, bf);
    const auto hpr = hr_depth(R.h, R.b, bf);
    const T hl = hp_val(hpl), hr = hp_val(hpr);
    const T dh = hp_diff(hpr, hpl);  // hR* - hL* with the bed/surface difference kept exact
    const bool wl = hl > hdry, wr = hr > hdry;
    // wave speeds of the reconstructed states
    const T sl = wl ? L.um + dev_sqrt(g * hl + L.s2) + L.s1 : dev_sqrt(g * hl);
    const T sr = wr ? R.um + dev_sqrt(g * hr + R.s2) + R.s1 : dev_sqrt(g * hr);
    const T sf = sl > sr ? sl : sr;
    const T el = wl ? hl : T(0), er = wr ? hr : T(0);  // depth that carries velocity
    const T hs = T(0.5) * sf;
    // conserved differences dQ = QR* - QL*
    T dn[m], dt_[D == 2 ? m : 1];
#pragma unroll
    for (int k = 0; k < m; ++k) dn[k] = er * FR.n[k] - el * FL.n[k];
    if constexpr (D == 2) {
#pragma unroll
        for (int k = 0; k < m; ++k) dt_[k] = er * FR.t[k] - el * FL.t[k];
    }
    fc[0] = T(0.5) * (el * FL.n[0] + er * FR.n[0]) - hs * dh;
#pragma unroll
    for (int k = 0; k < m; ++k) fc[1 + k] = T(0.5) * (el * FL.gnn[k] + er * FR.gnn[k]) - hs * dn[k];
    if constexpr (D == 2) {
#pragma unroll
        for (int k = 0; k < m; ++k) fc[1 + m + k] = T(0.5) * (el * FL.gnt[k] + er * FR.gnt[k]) - hs * dt_[k];
    }
    pd = T(0.25) * g * dh * (hr + hl);

#pragma unroll
    for (int k = 0; k < 1 + (D == 2 ? 2 : 1) * m; ++k) nc[k] = T(0);
    if constexpr (N >= 1) {
        // path-averaged velocity moments along Psi(s) = QL* + s dQ (3-point Gauss-Legendre)
        T nbar[m], tbar[D == 2 ? m : 1];
#pragma unroll
        for (int k = 0; k < m; ++k) nbar[k] = T(0);
        if constexpr (D == 2) {
#pragma unroll
            for (int k = 0; k < m; ++k) tbar[k] = T(0);
        }
        constexpr double sq15 = 0.38729833462074168852;  // sqrt(15)/10
        const T sn[3] = {T(0.5 - sq15), T(0.5), T(0.5 + sq15)};
        const T wq[3] = {T(5.0 / 18.0), T(8.0 / 18.0), T(5.0 / 18.0)};
        // FP64: the three reciprocals from one division of the product of the wet depths (dry nodes
        // count as 1 and get weight 0)
        T hqs[3], rp = T(1);
        if constexpr (sizeof(T) == 8) {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                hqs[q] = hl + sn[q] * dh;
                if (!(hqs[q] > hdry)) hqs[q] = T(1);
            }
            rp = T(1) / (hqs[0] * hqs[1] * hqs[2]);
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const T hq = hl + sn[q] * dh;
            const bool wet = hq > hdry;
            T iw;
            if constexpr (sizeof(T) == 8)
                iw = wet ? wq[q] * (rp * hqs[(q + 1) % 3] * hqs[(q + 2) % 3]) : T(0);
            else
                iw = wet ? dev_div(wq[q], hq) : T(0);
#pragma unroll
            for (int k = 0; k < m; ++k) nbar[k] += iw * (el * FL.n[k] + sn[q] * dn[k]);
            if constexpr (D == 2) {
#pragma unroll
                for (int k = 0; k < m; ++k) tbar[k] += iw * (el * FL.t[k] + sn[q] * dt_[k]);
            }
        }
        static_for<1, m>([&](auto kk) {
            constexpr int k = decltype(kk)::value;
            T rn = 0;
            [[maybe_unused]] T rt = 0;  // 2D only
            static_for<1, m>([&](auto ll) {
                constexpr int l = decltype(ll)::value;
                T en = 0;
                [[maybe_unused]] T et = 0;  // 2D only
                static_for<0, m>([&](auto jj) {
                    constexpr int j = decltype(jj)::value;
                    constexpr double w = ncB(k, j, l);
                    if constexpr (w != 0.0) {
                        en += T(w) * nbar[j];
                        if constexpr (D == 2) et += T(w) * tbar[j];
                    }
                });
                rn += en * dn[l];
                if constexpr (D == 2) rt += et * dn[l];
            });
            nc[1 + k] = T(0.5) * rn;
            if constexpr (D == 2) nc[1 + m + k] = T(0.5) * rt;
        });
    }
}

// Newtonian bulk friction, explicit part of the source (Sec. 3.4 closure sigma = nu d_z u):
//   S_{alpha_k} = -(nu/(rho h)) sum_i alpha_i C_ik / M_k,  C_ik = <phi_i', phi_k'>.
template <int N, int D, typename T>
__device__ __forceinline__ void newtonian(const CellRec<N, D, T> &r, T nu_rho, T *sa, T *sb)
{
    constexpr int m = N + 1;
    // FP64: the record's 1/h (0 where dry, where the velocity moments are 0 too), no second division
    T f;
    if constexpr (sizeof(T) == 8)
        f = nu_rho * r.ih;
    else
        f = r.h > T(0) ? dev_div(nu_rho, r.h) : T(0);
    static_for<0, m>([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        T xa = 0;
        [[maybe_unused]] T xb = 0;  // 2D only
        static_for<0, m>([&](auto ii) {
            constexpr int i = decltype(ii)::value;
            constexpr double w = visC(i, k);
            if constexpr (w != 0.0) {
                xa += T(w) * r.a[i];
                if constexpr (D == 2) xb += T(w) * r.c[i];
            }
        });
        sa[k] = -f * xa;
        if constexpr (D == 2) sb[k] = -f * xb;
    });
}

// Bottom stress, linearly implicit, then the dry cut, on the stage output y (in place).
// Stress on row k: -(2k+1) c sum_i y_i with c = C/(rho h) (Navier slip, Sec. 3.4) or
// c = g n^2 |u_b| / h^(4/3) (Manning), frozen at y; solved by Sherman-Morrison:
//   y <- y - dt c w (1^T y) / (1 + dt c 1^T w),  w_k = phi_k(0)/M_k = 2k+1.
// fric: 0 none, 1 slip (+ Newtonian elsewhere), 2 Manning.
template <int N, int D, typename T>
__device__ __forceinline__ void bottom_friction(T h, T *ya, T *yb, int fric, T C_rho, T gn2, T dt, T hdry)
{
    constexpr int m = N + 1;
    if (!(h > hdry)) {
#pragma unroll
        for (int k = 0; k < m; ++k) {
            ya[k] = T(0);
            if constexpr (D == 2) yb[k] = T(0);
        }
        return;
    }
    if (fric == 0) return;
    T sa = 0, sb = 0;
#pragma unroll
    for (int k = 0; k < m; ++k) {
        sa += ya[k];
        if constexpr (D == 2) sb += yb[k];
    }
    constexpr T sw = T(m * m);  // sum_k (2k+1)
    T f;
    if (sizeof(T) == 8 && fric == 1) {
        // FP64 slip: f = dt c / (1 + dt c sw) with c = C/(rho h) is dt C/rho / (h + dt C/rho sw), one
        // division instead of two (the FP64 path is bound by its division chains)
        const T dC = dt * C_rho;
        f = dC / (h + dC * sw);
    } else {
        T c;
        if (fric == 1) {
            c = dev_div(C_rho, h);
        } else {
            T ub = dev_div(sa, h), vb = dev_div(sb, h);
            T sp = (D == 2) ? dev_sqrt(ub * ub + vb * vb) : fabs(ub);
            // h^(4/3) = h * cbrt(h)
            c = dev_div(gn2 * sp, h * cbrt(h));
        }
        f = dev_div(dt * c, T(1) + dt * c * sw);
    }
    const T fa = f * sa, fb = f * sb;
#pragma unroll
    for (int k = 0; k < m; ++k) {
        ya[k] -= T(2 * k + 1) * fa;
        if constexpr (D == 2) yb[k] -= T(2 * k + 1) * fb;
    }
}

// Friction fully implicit (the paper's step_source_implicit for the friction ODE of Eq. (PDE-source)):
// backward Euler (I + dt K) z = y on the moment rows with K_ki = (2k+1) c + (nu/rho)/h^2 C_ik/M_k,
// the bottom stress (c as in bottom_friction) and the Newtonian bulk stress, h and c frozen at y;
// then the dry cut.  K = D (c 1 1^T + (nu/rho)/h^2 C), D = diag(2k+1), C positive semi-definite:
// I + dt K is similar to a symmetric positive-definite matrix, so elimination needs no pivoting.
template <int N, int D, typename T>
__device__ __forceinline__ void friction_implicit(T h, T *ya, T *yb, int fric, T C_rho, T nu_rho, T gn2, T dt,
                                                  T hdry)
{
    constexpr int m = N + 1;
    if (!(h > hdry)) {
#pragma unroll
        for (int k = 0; k < m; ++k) {
            ya[k] = T(0);
            if constexpr (D == 2) yb[k] = T(0);
        }
        return;
    }
    if (fric == 0) return;
    T sa = 0, sb = 0;
#pragma unroll
    for (int k = 0; k < m; ++k) {
        sa += ya[k];
        if constexpr (D == 2) sb += yb[k];
    }
    T c;
    if (fric == 1) {
        c = dev_div(C_rho, h);
    } else {
        T ub = dev_div(sa, h), vb = dev_div(sb, h);
        T sp = (D == 2) ? dev_sqrt(ub * ub + vb * vb) : fabs(ub);
        c = dev_div(gn2 * sp, h * cbrt(h));
    }
    const T nuh = fric == 1 ? dev_div(nu_rho, h * h) : T(0);
    T A[m][m];
    static_for<0, m>([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        static_for<0, m>([&](auto ii) {
            constexpr int i = decltype(ii)::value;
            A[k][i] = (k == i ? T(1) : T(0)) + dt * (T(bedW(k)) * c + nuh * T(visC(i, k)));
        });
    });
#pragma unroll
    for (int col = 0; col < m; ++col) {
        const T piv = dev_div(T(1), A[col][col]);
#pragma unroll
        for (int r = col + 1; r < m; ++r) {
            const T f = A[r][col] * piv;
#pragma unroll
            for (int j = col + 1; j < m; ++j) A[r][j] -= f * A[col][j];
            ya[r] -= f * ya[col];
            if constexpr (D == 2) yb[r] -= f * yb[col];
        }
    }
#pragma unroll
    for (int k = m - 1; k >= 0; --k) {
        T za = ya[k], zb = D == 2 ? yb[k] : T(0);
#pragma unroll
        for (int j = k + 1; j < m; ++j) {
            za -= A[k][j] * ya[j];
            if constexpr (D == 2) zb -= A[k][j] * yb[j];
        }
        const T inv = dev_div(T(1), A[k][k]);
        ya[k] = za * inv;
        if constexpr (D == 2) yb[k] = zb * inv;
    }
}

// Cell wave-speed bound s = |u_mean| + sqrt(g h + sum_{k>=1}|a_k|^2) + sum_{k>=2}|a_k|.
template <int N, int D, typename T>
__device__ __forceinline__ T wavespeed(const CellRec<N, D, T> &r, T g)
{
    T h = r.h > T(0) ? r.h : T(0);
    return r.um + dev_sqrt(g * h + r.s2) + r.s1;
}

}  // namespace zoomy
