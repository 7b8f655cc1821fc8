// fv_order2.cu -- second order in space on 1D and structured 2D grids (MUSCL).
//
// Per direction d, a cell's reconstruction variables w = (h, eta = h + b, alpha_0..N, beta_0..N)
// get the minmod-limited slope sigma = minmod(w_i - w_{i-1}, w_{i+1} - w_i) (zero for every variable
// when one of the three cells is dry); its face states are w +- sigma/2 with the bed
// b +- (sigma_eta - sigma_h)/2, so that a lake at rest keeps a flat surface at every face.  Every
// face is the first-order face term (hydrostatic reconstruction, path-conservative Rusanov flux,
// pressure difference, 3-point path integral of the nonconservative product) between the two
// reconstructed face states, and every cell adds per direction the interior terms
//   g (h_+ + h_-)/2 (eta_+ - eta_-)          on the normal mean-momentum row,
//   Btilde(Q_- -> Q_+) (Q_+ - Q_-)            (path integral across the cell),
// which vanish for zero slopes (first order) and for a lake at rest.  Sources, bottom stress, dry
// cut and SSP-RK2 averaging are those of the first-order stages.
//
// 1D lines: one thread per cell (k_stage_order2): the stencil of radius 2 is loaded, the cell's slopes
// and those of its neighbours are computed, and each face is evaluated from the side of the cell being
// updated.  Structured 2D grids: row-marching warps (k_stage_order2_march, below) that turn each cell
// into its primitive vector once and evaluate each face once.
#include <cstdint>

#include <cuda_runtime.h>

#include "fv_common.cuh"
#include "model.cuh"
#include "zoomy_kernels.h"

namespace zoomy {

template <int N, int D>
struct O2 {
    static constexpr int m = N + 1;
    static constexpr int nv = D == 1 ? 1 + m : 1 + 2 * m;
    static constexpr int nw = D == 1 ? 2 + m : 2 + 2 * m;
};

// State and bed of cell (ix, iy); outside the grid the ghost of the boundary cell (copy, or the
// moment vectors reflected at a wall).
template <int N, int D, typename T>
__device__ __forceinline__ void state_at(const StageArgs<T> &a, int ix, int iy, T *q)
{
    constexpr int m = N + 1, nv = O2<N, D>::nv;
    const int cx = ix < 0 ? 0 : (ix >= a.nx ? a.nx - 1 : ix);
    const int cy = D == 1 ? 0 : (iy < 0 ? 0 : (iy >= a.ny ? a.ny - 1 : iy));
    const int64_t idx = bounds_idx((int64_t)cy * a.nx + cx, (int64_t)a.nx * (D == 1 ? 1 : a.ny), &a.ctl->status);
#pragma unroll
    for (int v = 0; v < nv; ++v) q[v] = a.X[(int64_t)v * a.ld + idx];
    q[nv] = a.bed[idx];
    const bool xwall = (ix < 0 && a.bc[0] == 1) || (ix >= a.nx && a.bc[1] == 1);
    const bool ywall = D == 2 && ((iy < 0 && a.bc[2] == 1) || (iy >= a.ny && a.bc[3] == 1));
#pragma unroll
    for (int k = 0; k < m; ++k) {
        if (xwall) q[var_a<N, D>(k)] = -q[var_a<N, D>(k)];
        if constexpr (D == 2)
            if (ywall) q[var_b<N>(k)] = -q[var_b<N>(k)];
    }
}

template <int N, int D, typename T>
__device__ __forceinline__ void prim(const T *q, T hdry, T *w)
{
    constexpr int m = N + 1, nv = O2<N, D>::nv;
    const T h = q[0];
    const bool wet = h > hdry;
    w[0] = h;
    w[1] = h + q[nv];
    if constexpr (sizeof(T) == 8) {
        // FP64: one division per cell (the FP64 path is bound by its division chains)
        const T rh = wet ? T(1) / h : T(0);
#pragma unroll
        for (int k = 0; k < m; ++k) {
            w[2 + k] = q[var_a<N, D>(k)] * rh;
            if constexpr (D == 2) w[2 + m + k] = q[var_b<N>(k)] * rh;
        }
    } else {
#pragma unroll
        for (int k = 0; k < m; ++k) {
            w[2 + k] = wet ? q[var_a<N, D>(k)] / h : T(0);
            if constexpr (D == 2) w[2 + m + k] = wet ? q[var_b<N>(k)] / h : T(0);
        }
    }
}

__host__ __device__ __forceinline__ double mmod(double x, double y)
{
    return (x > 0.0 && y > 0.0) ? (x < y ? x : y) : ((x < 0.0 && y < 0.0) ? (x > y ? x : y) : 0.0);
}
__host__ __device__ __forceinline__ float mmod(float x, float y)
{
    return (x > 0.0f && y > 0.0f) ? fminf(x, y) : ((x < 0.0f && y < 0.0f) ? fmaxf(x, y) : 0.0f);
}

// Limited slopes of the cell with states qc (centre), ql, qr (its neighbours along the direction).
template <int N, int D, typename T>
__device__ __forceinline__ void slopes(const T *ql, const T *qc, const T *qr, T hdry, T *sig)
{
    constexpr int nw = O2<N, D>::nw;
    T wl[nw], wc[nw], wr[nw];
    prim<N, D, T>(ql, hdry, wl);
    prim<N, D, T>(qc, hdry, wc);
    prim<N, D, T>(qr, hdry, wr);
    const bool dry = !(ql[0] > hdry) || !(qc[0] > hdry) || !(qr[0] > hdry);
#pragma unroll
    for (int v = 0; v < nw; ++v) sig[v] = dry ? T(0) : mmod(wc[v] - wl[v], wr[v] - wc[v]);
}

// Cell record of the face state on side s (-1 / +1) of a cell with primitive vector wc = prim(qc),
// bed bc and slopes sig; reflect: the state is the ghost across a wall of direction d (the normal
// moment components change sign).
template <int N, int D, typename T>
__device__ __forceinline__ void face_rec_w(const T *wc, T bc, const T *sig, int s, int d, bool reflect, T hdry,
                                           CellRec<N, D, T> &r)
{
    constexpr int m = N + 1, nw = O2<N, D>::nw;
    T w[nw];
    const T hs = T(0.5) * T(s);
#pragma unroll
    for (int v = 0; v < nw; ++v) w[v] = wc[v] + hs * sig[v];
    const T bf = bc + hs * (sig[1] - sig[0]);
    T ha[m], hb[m];
#pragma unroll
    for (int k = 0; k < m; ++k) {
        ha[k] = w[0] * w[2 + k];
        hb[k] = D == 2 ? w[0] * w[2 + m + k] : T(0);
        if (reflect) {
            if (d == 0) ha[k] = -ha[k];
            else hb[k] = -hb[k];
        }
    }
    make_cell<N, D, T>(r, w[0], bf, ha, hb, hdry);
}

template <int N, int D, typename T>
__device__ __forceinline__ void face_rec(const T *qc, const T *sig, int s, int d, bool reflect, T hdry,
                                         CellRec<N, D, T> &r)
{
    constexpr int nv = O2<N, D>::nv, nw = O2<N, D>::nw;
    T w[nw];
    prim<N, D, T>(qc, hdry, w);
    face_rec_w<N, D, T>(w, qc[nv], sig, s, d, reflect, hdry, r);
}

// Adds the face terms and the interior terms of direction d (YD: the y direction) to acc; st[0..4]:
// the states at offsets -2..+2 along d; lowb / highb: the cell lies on the low / high boundary.
template <int N, int D, typename T, bool YD>
__device__ __forceinline__ void direction_terms(const StageArgs<T> &a, const T (*st)[O2<N, D>::nv + 1], bool lowb,
                                                bool highb, T inv_d, T *acc)
{
    constexpr int m = N + 1, nw = O2<N, D>::nw;
    const int d = YD ? 1 : 0;
    T sc[nw], sl[nw], sr[nw];
    slopes<N, D, T>(st[1], st[2], st[3], a.hdry, sc);
    CellRec<N, D, T> cm, cp, nl, nr;
    face_rec<N, D, T>(st[2], sc, -1, d, false, a.hdry, cm);
    face_rec<N, D, T>(st[2], sc, +1, d, false, a.hdry, cp);
    // low-side neighbour: its high face state, or the ghost of this cell's low face state
    if (lowb) {
        face_rec<N, D, T>(st[2], sc, -1, d, a.bc[2 * d] == 1, a.hdry, nl);
    } else {
        slopes<N, D, T>(st[0], st[1], st[2], a.hdry, sl);
        face_rec<N, D, T>(st[1], sl, +1, d, false, a.hdry, nl);
    }
    if (highb) {
        face_rec<N, D, T>(st[2], sc, +1, d, a.bc[2 * d + 1] == 1, a.hdry, nr);
    } else {
        slopes<N, D, T>(st[2], st[3], st[4], a.hdry, sr);
        face_rec<N, D, T>(st[3], sr, -1, d, false, a.hdry, nr);
    }
    constexpr int nr_ = D == 2 ? 1 + 2 * m : 1 + m;
    T fc[nr_], nc[nr_], pd;
    // row of the face frame -> variable of the state
    auto var = [&](int row) {
        if (row == 0) return 0;
        if constexpr (D == 1) return var_a<N, 1>(row - 1);
        const int k = row <= m ? row - 1 : row - 1 - m;
        const bool normal = row <= m;
        return (normal != YD) ? var_a<N, 2>(k) : var_b<N>(k);
    };
    const int n0 = YD ? var_b<N>(0) : var_a<N, D>(0);
    // low face: this cell is R
    face_term<N, D, T>(nl, frame<N, D, T, YD>(nl), cm, frame<N, D, T, YD>(cm), a.g, a.hdry, fc, pd, nc);
#pragma unroll
    for (int row = 0; row < nr_; ++row) acc[var(row)] += inv_d * (fc[row] - nc[row]);
    acc[n0] -= inv_d * pd;
    // high face: this cell is L
    face_term<N, D, T>(cp, frame<N, D, T, YD>(cp), nr, frame<N, D, T, YD>(nr), a.g, a.hdry, fc, pd, nc);
#pragma unroll
    for (int row = 0; row < nr_; ++row) acc[var(row)] -= inv_d * (fc[row] + nc[row]);
    acc[n0] -= inv_d * pd;
    // cell interior: pressure against the surface slope, and the full path integral from the low to
    // the high face state (the bed is left out so the depths are the reconstructed ones)
    const T etam = cm.h + cm.b, etap = cp.h + cp.b;
    acc[n0] -= inv_d * (T(0.5) * a.g * (cp.h + cm.h) * (etap - etam));
    cm.b = T(0);
    cp.b = T(0);
    face_term<N, D, T>(cm, frame<N, D, T, YD>(cm), cp, frame<N, D, T, YD>(cp), a.g, a.hdry, fc, pd, nc);
#pragma unroll
    for (int row = 0; row < nr_; ++row) acc[var(row)] -= inv_d * (T(2) * nc[row]);
}

template <int N, int D, typename T, int STAGE>
__global__ void __launch_bounds__(128) k_stage_order2(StageArgs<T> a)
{
    constexpr int m = N + 1, nv = O2<N, D>::nv;
    if (*(volatile unsigned int *)&a.ctl->status) return;
    T dt;
    if (!step_dt(a, dt)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&a.ctl->status, DEV_NOWAVE);
        return;
    }
    if (STAGE == 1 && blockIdx.x == 0 && threadIdx.x == 0) step_bookkeeping(a, dt);
    const int64_t nc = (int64_t)a.nx * (D == 2 ? a.ny : 1);
    T smax = T(0);
    unsigned flag = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nc; i += (int64_t)gridDim.x * blockDim.x) {
        const int ix = (int)(i % a.nx), iy = D == 2 ? (int)(i / a.nx) : 0;
        T acc[nv];
#pragma unroll
        for (int v = 0; v < nv; ++v) acc[v] = T(0);
        T st[5][nv + 1];
#pragma unroll
        for (int o = 0; o < 5; ++o) state_at<N, D, T>(a, ix + o - 2, iy, st[o]);
        direction_terms<N, D, T, false>(a, st, ix == 0, ix == a.nx - 1, a.inv_dx, acc);
        if constexpr (D == 2) {
#pragma unroll
            for (int o = 0; o < 5; ++o) state_at<N, D, T>(a, ix, iy + o - 2, st[o]);
            direction_terms<N, D, T, true>(a, st, iy == 0, iy == a.ny - 1, a.inv_dy, acc);
        }
        // sources at the stage input, bottom stress / full implicit friction, dry cut
        const T *x = st[2];  // the centre cell (index 2 of either direction's stencil)
        T ha[m], hb[m];
#pragma unroll
        for (int k = 0; k < m; ++k) {
            ha[k] = x[var_a<N, D>(k)];
            hb[k] = D == 2 ? x[var_b<N>(k)] : T(0);
        }
        CellRec<N, D, T> me;
        make_cell<N, D, T>(me, x[0], x[nv], ha, hb, a.hdry);
        T sa[m], sb[m];
        newtonian<N, D, T>(me, a.nu_rho, sa, D == 2 ? sb : nullptr);
        T y[nv], ya[m], yb[m];
        y[0] = x[0] + dt * acc[0];
#pragma unroll
        for (int k = 0; k < m; ++k) {
            ya[k] = ha[k] + dt * (acc[var_a<N, D>(k)] + sa[k]);
            yb[k] = D == 2 ? hb[k] + dt * (acc[var_b<N>(k)] + sb[k]) : T(0);
        }
        if (a.src_implicit)
            friction_implicit<N, D, T>(y[0], ya, D == 2 ? yb : nullptr, a.fric, a.C_rho, a.nu_imp, a.gn2, dt, a.hdry);
        else
            bottom_friction<N, D, T>(y[0], ya, D == 2 ? yb : nullptr, a.fric, a.C_rho, a.gn2, dt, a.hdry);
#pragma unroll
        for (int k = 0; k < m; ++k) {
            y[var_a<N, D>(k)] = ya[k];
            if constexpr (D == 2) y[var_b<N>(k)] = yb[k];
        }
        if (STAGE == 2) {
#pragma unroll
            for (int v = 0; v < nv; ++v) y[v] = T(0.5) * (a.Qn[(int64_t)v * a.ld + i] + y[v]);
#pragma unroll
            for (int k = 0; k < m; ++k) {
                ya[k] = y[var_a<N, D>(k)];
                yb[k] = D == 2 ? y[var_b<N>(k)] : T(0);
            }
            CellRec<N, D, T> co;
            make_cell<N, D, T>(co, y[0], T(0), ya, yb, a.hdry);
            const T s = wavespeed<N, D, T>(co, a.g);
            if (!(s <= T(3.0e38))) flag |= DEV_NAN;
            if (!(y[0] >= T(0))) flag |= (y[0] < T(0)) ? DEV_NEGDEPTH : DEV_NAN;
            smax = (s > smax || s != s) ? s : smax;
        }
#pragma unroll
        for (int v = 0; v < nv; ++v) a.out[(int64_t)v * a.ld + i] = y[v];
    }
    if (STAGE == 2) {
        if (flag) atomicOr(&a.ctl->status, flag);
        // block maximum (NaN wins), then one atomic per CTA
        __shared__ T wmax[4];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const T v = __shfl_xor_sync(0xffffffffu, smax, o);
            smax = (v > smax || v != v) ? v : smax;
        }
        if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = smax;
        __syncthreads();
        if (threadIdx.x < 32) {
            smax = threadIdx.x < 4 ? wmax[threadIdx.x] : T(0);
            reduce_smax<T>(a.ctl, a.slot_out, smax);
        }
    }
}

// ------------------------------------------------------------------------------------------
// Structured 2D: row-marching warps, each face once
// ------------------------------------------------------------------------------------------
//
// A warp takes a strip of 28 columns (lanes 2..29; lanes 0, 1, 30, 31 hold the two neighbour columns
// on each side) and marches down the rows of a segment.  Each lane turns the state of its cell into
// the primitive vector once; the x-slopes come from the neighbour lanes (shuffles), the y-slopes from
// the three rows kept in registers.  Step M (the lead row M + 1 loaded) does row M: its x-faces (lane
// l evaluates the face on its low side; the lane past the last column evaluates the high boundary
// face), its x and y interior terms and the y-face below it, whose upper-side record was kept from
// step M - 1.  That face completes row M - 1, which is finished (sources, bottom stress, SSP-RK2
// average, store).  Every face sees the same face states as in the cell-centric kernel, and a
// boundary face sees the ghost of the cell's own face state (copy, or wall reflection).

constexpr int O2_COLS = 28;

template <int N, typename T>
struct O2Row {
    T w[O2<N, 2>::nw];
    T b;
};

// Raw state and bed of (col, row), clamped into the grid (the loads only: a row is fetched one step
// before it is used, and the ghost reflection is applied when it is used, in o2_make)
template <int N, typename T>
__device__ __forceinline__ void o2_fetch(const StageArgs<T> &a, int col, int row, T *q)
{
    constexpr int nv = O2<N, 2>::nv;
    const int cx = col < 0 ? 0 : (col >= a.nx ? a.nx - 1 : col);
    const int cy = row < 0 ? 0 : (row >= a.ny ? a.ny - 1 : row);
    const int64_t idx = bounds_idx((int64_t)cy * a.nx + cx, (int64_t)a.nx * a.ny, &a.ctl->status);
#pragma unroll
    for (int v = 0; v < nv; ++v) q[v] = a.X[(int64_t)v * a.ld + idx];
    q[nv] = a.bed[idx];
}

// The fetched state as state_at gives it (the moment vectors reflected at a wall ghost), then its
// primitive vector and bed
template <int N, typename T>
__device__ __forceinline__ void o2_make(const StageArgs<T> &a, int col, int row, T *q, O2Row<N, T> &P)
{
    constexpr int m = N + 1, nv = O2<N, 2>::nv;
    const bool xwall = (col < 0 && a.bc[0] == 1) || (col >= a.nx && a.bc[1] == 1);
    const bool ywall = (row < 0 && a.bc[2] == 1) || (row >= a.ny && a.bc[3] == 1);
#pragma unroll
    for (int k = 0; k < m; ++k) {
        if (xwall) q[var_a<N, 2>(k)] = -q[var_a<N, 2>(k)];
        if (ywall) q[var_b<N>(k)] = -q[var_b<N>(k)];
    }
    prim<N, 2, T>(q, a.hdry, P.w);
    P.b = q[nv];
}

// Reflection of a face-state record across a wall of direction d: the normal moments and the mixed
// flux products change sign (bitwise the record of the reflected state).
template <int N, typename T>
__device__ __forceinline__ void reflect_rec(CellRec<N, 2, T> &r, int d)
{
#pragma unroll
    for (int k = 0; k <= N; ++k) {
        if (d == 0)
            r.a[k] = -r.a[k];
        else
            r.c[k] = -r.c[k];
        r.gab[k] = -r.gab[k];
    }
}

template <int N, typename T>
__device__ __forceinline__ void shfl_up_rec(CellRec<N, 2, T> &o, const CellRec<N, 2, T> &r)
{
    constexpr unsigned F = 0xffffffffu;
    o.h = __shfl_up_sync(F, r.h, 1);
    o.b = __shfl_up_sync(F, r.b, 1);
    o.um = __shfl_up_sync(F, r.um, 1);
    o.s2 = __shfl_up_sync(F, r.s2, 1);
    o.s1 = __shfl_up_sync(F, r.s1, 1);
#pragma unroll
    for (int k = 0; k <= N; ++k) {
        o.a[k] = __shfl_up_sync(F, r.a[k], 1);
        o.c[k] = __shfl_up_sync(F, r.c[k], 1);
        o.gaa[k] = __shfl_up_sync(F, r.gaa[k], 1);
        o.gab[k] = __shfl_up_sync(F, r.gab[k], 1);
        o.gbb[k] = T(0);  // not used in the x frame
    }
}

// Face-frame row -> state variable, direction YD
template <int N, bool YD>
__device__ __forceinline__ int o2_var(int row)
{
    constexpr int m = N + 1;
    if (row == 0) return 0;
    const int k = row <= m ? row - 1 : row - 1 - m;
    const bool normal = row <= m;
    return (normal != YD) ? var_a<N, 2>(k) : var_b<N>(k);
}

// Interior terms of a cell in direction YD from its two face states (cm, cp are changed)
template <int N, typename T, bool YD>
__device__ __forceinline__ void o2_interior(const StageArgs<T> &a, CellRec<N, 2, T> &cm, CellRec<N, 2, T> &cp,
                                            T inv_d, T *acc)
{
    constexpr int m = N + 1, nr = 1 + 2 * m;
    const int n0 = YD ? var_b<N>(0) : var_a<N, 2>(0);
    const T etam = cm.h + cm.b, etap = cp.h + cp.b;
    acc[n0] -= inv_d * (T(0.5) * a.g * (cp.h + cm.h) * (etap - etam));
    cm.b = T(0);
    cp.b = T(0);
    T fc[nr], nc[nr], pd;
    face_term<N, 2, T>(cm, frame<N, 2, T, YD>(cm), cp, frame<N, 2, T, YD>(cp), a.g, a.hdry, fc, pd, nc);
#pragma unroll
    for (int row = 0; row < nr; ++row) acc[o2_var<N, YD>(row)] -= inv_d * (T(2) * nc[row]);
}

// FP32 up to level 2: held to 128 registers (16 one-warp CTAs per SM), measured faster than the 142-154
// registers the prefetching kernel takes on its own (0.526 against 0.594 ms per 2048^2 level-2 step);
// the other instantiations are left at their own counts (a cap spills them)
template <int N, typename T>
constexpr int O2_MIN_CTAS = (sizeof(T) == 4 && N <= 2) ? 16 : 1;

template <int N, typename T, int STAGE>
__global__ void __launch_bounds__(32, O2_MIN_CTAS<N, T>) k_stage_order2_march(StageArgs<T> a, int nstrips, int H)
{
    constexpr int m = N + 1, nv = O2<N, 2>::nv, nw = O2<N, 2>::nw, nr = 1 + 2 * m;
    constexpr unsigned F = 0xffffffffu;
    pdl_enter();
    if (*(volatile unsigned int *)&a.ctl->status) return;
    T dt;
    if (!step_dt(a, dt)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&a.ctl->status, DEV_NOWAVE);
        return;
    }
    if (STAGE == 1 && blockIdx.x == 0 && threadIdx.x == 0) step_bookkeeping(a, dt);
    const int lane = threadIdx.x;
    const int strip = blockIdx.x % nstrips, seg = blockIdx.x / nstrips;
    const int col = strip * O2_COLS - 2 + lane;
    const bool owned = lane >= 2 && lane < 2 + O2_COLS && col < a.nx;
    const int r0 = seg * H, r1 = min(r0 + H, a.ny);
    const int n0x = var_a<N, 2>(0), n0y = var_b<N>(0);
    const T hdry = a.hdry;
    T smax = T(0);
    unsigned flag = 0;

    O2Row<N, T> P2, P1, P0;  // rows M - 1, M, M + 1
    T nxt[nv + 1];           // fetched raw state of row M + 1
    o2_fetch<N, T>(a, col, r0 - 2, nxt);
    o2_make<N, T>(a, col, r0 - 2, nxt, P2);
    o2_fetch<N, T>(a, col, r0 - 1, nxt);
    o2_make<N, T>(a, col, r0 - 1, nxt, P1);
    o2_fetch<N, T>(a, col, r0, nxt);
    CellRec<N, 2, T> cpy_prev;  // upper y face state of row M - 1 (set at step M - 1)
    T accM[nv], accP[nv];        // rows M and M - 1
#pragma unroll
    for (int v = 0; v < nv; ++v) accM[v] = accP[v] = T(0);
    for (int M = r0 - 1; M <= r1; ++M) {
        o2_make<N, T>(a, col, M + 1, nxt, P0);
        if (M < r1) o2_fetch<N, T>(a, col, M + 2, nxt);  // in flight during this step
        // the stage input and Q^n of row M - 1, finished at the end of this step
        const bool fin = M - 1 >= r0 && owned;
        const int64_t fi = (int64_t)(fin ? M - 1 : r0) * a.nx + (owned ? col : 0);
        T xf[nv], qf[nv];
        if (fin) {
#pragma unroll
            for (int v = 0; v < nv; ++v) {
                xf[v] = a.X[(int64_t)v * a.ld + fi];
                if (STAGE == 2) qf[v] = a.Qn[(int64_t)v * a.ld + fi];
            }
        }
        const bool inner = M >= r0 && M < r1;  // warp-uniform
        T fc[nr], nc[nr], pd;
        // ---- x direction of row M -------------------------------------------------------
        if (inner) {
            T sig[nw];
            const T wl0 = __shfl_up_sync(F, P1.w[0], 1), wr0 = __shfl_down_sync(F, P1.w[0], 1);
            const bool dry = !(wl0 > hdry) || !(P1.w[0] > hdry) || !(wr0 > hdry);
#pragma unroll
            for (int v = 0; v < nw; ++v) {
                const T wl = __shfl_up_sync(F, P1.w[v], 1), wr = __shfl_down_sync(F, P1.w[v], 1);
                sig[v] = dry ? T(0) : mmod(P1.w[v] - wl, wr - P1.w[v]);
            }
            CellRec<N, 2, T> cm, cp, L;
            face_rec_w<N, 2, T>(P1.w, P1.b, sig, -1, 0, false, hdry, cm);
            face_rec_w<N, 2, T>(P1.w, P1.b, sig, +1, 0, false, hdry, cp);
            // the face on this column's low side: L = the upper state of the column on the left, or at
            // column 0 the ghost of this cell's lower state; past the last column, R = the ghost of L
            shfl_up_rec<N, T>(L, cp);
            if (col == 0) {
                L = cm;
                if (a.bc[0] == 1) reflect_rec<N, T>(L, 0);
            }
            if (col == a.nx) {
                CellRec<N, 2, T> R = L;
                if (a.bc[1] == 1) reflect_rec<N, T>(R, 0);
                face_term<N, 2, T>(L, frame<N, 2, T, false>(L), R, frame<N, 2, T, false>(R), a.g, hdry, fc, pd, nc);
            } else {
                face_term<N, 2, T>(L, frame<N, 2, T, false>(L), cm, frame<N, 2, T, false>(cm), a.g, hdry, fc, pd, nc);
            }
            // this cell is R of its low face and L of its high face (the next lane's)
#pragma unroll
            for (int row = 0; row < nr; ++row) accM[o2_var<N, false>(row)] += a.inv_dx * (fc[row] - nc[row]);
            accM[n0x] -= a.inv_dx * pd;
#pragma unroll
            for (int row = 0; row < nr; ++row)
                accM[o2_var<N, false>(row)] -= a.inv_dx * __shfl_down_sync(F, fc[row] + nc[row], 1);
            accM[n0x] -= a.inv_dx * __shfl_down_sync(F, pd, 1);
            o2_interior<N, T, false>(a, cm, cp, a.inv_dx, accM);
        }
        // ---- y direction of row M: the face below it, the interior terms ----------------
        {
            T sig[nw];
            const bool dry = !(P2.w[0] > hdry) || !(P1.w[0] > hdry) || !(P0.w[0] > hdry);
#pragma unroll
            for (int v = 0; v < nw; ++v) sig[v] = dry ? T(0) : mmod(P1.w[v] - P2.w[v], P0.w[v] - P1.w[v]);
            CellRec<N, 2, T> cm, cp;
            face_rec_w<N, 2, T>(P1.w, P1.b, sig, -1, 1, false, hdry, cm);
            face_rec_w<N, 2, T>(P1.w, P1.b, sig, +1, 1, false, hdry, cp);
            if (M >= r0) {
                CellRec<N, 2, T> L = cpy_prev, R = cm;
                if (M == 0) {
                    L = cm;
                    if (a.bc[2] == 1) reflect_rec<N, T>(L, 1);
                }
                if (M == a.ny) {
                    R = cpy_prev;
                    if (a.bc[3] == 1) reflect_rec<N, T>(R, 1);
                }
                face_term<N, 2, T>(L, frame<N, 2, T, true>(L), R, frame<N, 2, T, true>(R), a.g, hdry, fc, pd, nc);
#pragma unroll
                for (int row = 0; row < nr; ++row) {
                    accM[o2_var<N, true>(row)] += a.inv_dy * (fc[row] - nc[row]);
                    accP[o2_var<N, true>(row)] -= a.inv_dy * (fc[row] + nc[row]);
                }
                accM[n0y] -= a.inv_dy * pd;
                accP[n0y] -= a.inv_dy * pd;
            }
            cpy_prev = cp;
            if (inner) o2_interior<N, T, true>(a, cm, cp, a.inv_dy, accM);
        }
        // ---- row M - 1 is complete: sources, bottom stress, dry cut, SSP-RK2 average ------
        if (fin) {
            const int64_t i = fi;
            const T *x = xf;
            CellRec<N, 2, T> me;  // the Newtonian source needs h and the velocity moments (P2 = row M - 1)
            me.h = x[0];
            me.ih = x[0] > a.hdry ? T(1) / x[0] : T(0);
#pragma unroll
            for (int k = 0; k < m; ++k) {
                me.a[k] = P2.w[2 + k];
                me.c[k] = P2.w[2 + m + k];
            }
            T sa[m], sb[m];
            newtonian<N, 2, T>(me, a.nu_rho, sa, sb);
            T y[nv], ya[m], yb[m];
            y[0] = x[0] + dt * accP[0];
#pragma unroll
            for (int k = 0; k < m; ++k) {
                ya[k] = x[var_a<N, 2>(k)] + dt * (accP[var_a<N, 2>(k)] + sa[k]);
                yb[k] = x[var_b<N>(k)] + dt * (accP[var_b<N>(k)] + sb[k]);
            }
            if (a.src_implicit)
                friction_implicit<N, 2, T>(y[0], ya, yb, a.fric, a.C_rho, a.nu_imp, a.gn2, dt, a.hdry);
            else
                bottom_friction<N, 2, T>(y[0], ya, yb, a.fric, a.C_rho, a.gn2, dt, a.hdry);
#pragma unroll
            for (int k = 0; k < m; ++k) {
                y[var_a<N, 2>(k)] = ya[k];
                y[var_b<N>(k)] = yb[k];
            }
            if (STAGE == 2) {
#pragma unroll
                for (int v = 0; v < nv; ++v) y[v] = T(0.5) * (qf[v] + y[v]);
#pragma unroll
                for (int k = 0; k < m; ++k) {
                    ya[k] = y[var_a<N, 2>(k)];
                    yb[k] = y[var_b<N>(k)];
                }
                CellRec<N, 2, T> co;
                make_cell<N, 2, T>(co, y[0], T(0), ya, yb, a.hdry);
                const T sp = wavespeed<N, 2, T>(co, a.g);
                if (!(sp <= T(3.0e38))) flag |= DEV_NAN;
                if (!(y[0] >= T(0))) flag |= (y[0] < T(0)) ? DEV_NEGDEPTH : DEV_NAN;
                smax = (sp > smax || sp != sp) ? sp : smax;
            }
#pragma unroll
            for (int v = 0; v < nv; ++v) a.out[(int64_t)v * a.ld + i] = y[v];
        }
        P2 = P1;
        P1 = P0;
#pragma unroll
        for (int v = 0; v < nv; ++v) {
            accP[v] = accM[v];
            accM[v] = T(0);
        }
    }
    if (STAGE == 2) {
        if (flag) atomicOr(&a.ctl->status, flag);
        reduce_smax<T>(a.ctl, a.slot_out, smax);
    }
}

// One-warp CTAs, one wave: the segment height H spreads the strips' rows over the resident warps.
template <int N, typename T>
static cudaError_t launch_o2_march(const StageArgs<T> &a, int stage, int nsm, cudaStream_t st)
{
    const int nstrips = (a.nx + O2_COLS - 1) / O2_COLS;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, stage == 1 ? k_stage_order2_march<N, T, 1> : k_stage_order2_march<N, T, 2>, 32, 0);
    if (e != cudaSuccess) return e;
    const long long slots = (long long)nsm * (per_sm > 0 ? per_sm : 1);
    long long H = ((long long)nstrips * a.ny + slots - 1) / slots;
    if (H < 8) H = 8;
    if (H > a.ny) H = a.ny;
    const long long nsegs = (a.ny + H - 1) / H;
    const dim3 grid((unsigned)(nstrips * nsegs)), block(32);
    const int h = (int)H;
    if (stage == 1) return launch_pdl(k_stage_order2_march<N, T, 1>, grid, block, st, a, nstrips, h);
    return launch_pdl(k_stage_order2_march<N, T, 2>, grid, block, st, a, nstrips, h);
}

template <int N, int D, typename T>
static cudaError_t launch_o2(const StageArgs<T> &a, int stage, int nsm, cudaStream_t st)
{
    const int64_t nc = (int64_t)a.nx * (D == 2 ? a.ny : 1);
    int64_t blocks = (nc + 127) / 128;
    if (blocks > (int64_t)nsm * 8) blocks = (int64_t)nsm * 8;
    const dim3 grid((unsigned)(blocks > 0 ? blocks : 1)), block(128);
    if (stage == 1)
        k_stage_order2<N, D, T, 1><<<grid, block, 0, st>>>(a);
    else
        k_stage_order2<N, D, T, 2><<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_stage_order2(int dim, int level, const StageArgs<T> &a, int stage, int nsm, cudaStream_t st)
{
    if (dim == 1) {
        switch (level) {
            case 0: return launch_o2<0, 1, T>(a, stage, nsm, st);
            case 1: return launch_o2<1, 1, T>(a, stage, nsm, st);
            case 2: return launch_o2<2, 1, T>(a, stage, nsm, st);
            case 3: return launch_o2<3, 1, T>(a, stage, nsm, st);
            case 4: return launch_o2<4, 1, T>(a, stage, nsm, st);
        }
    } else {
        switch (level) {
            case 0: return launch_o2_march<0, T>(a, stage, nsm, st);
            case 1: return launch_o2_march<1, T>(a, stage, nsm, st);
            case 2: return launch_o2_march<2, T>(a, stage, nsm, st);
            case 3: return launch_o2_march<3, T>(a, stage, nsm, st);
            case 4: return launch_o2_march<4, T>(a, stage, nsm, st);
        }
    }
    return cudaErrorInvalidValue;
}

template cudaError_t launch_stage_order2<float>(int, int, const StageArgs<float> &, int, int, cudaStream_t);
template cudaError_t launch_stage_order2<double>(int, int, const StageArgs<double> &, int, int, cudaStream_t);

}  // namespace zoomy
