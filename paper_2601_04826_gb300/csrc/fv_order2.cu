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
// One thread per cell: the cross stencil of radius 2 is loaded, the cell's slopes and those of its
// neighbours are computed, and each face is evaluated from the side of the cell being updated
// (every face twice overall: simple, and the stencil stays in L1/L2).
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
#pragma unroll
    for (int k = 0; k < m; ++k) {
        w[2 + k] = wet ? q[var_a<N, D>(k)] / h : T(0);
        if constexpr (D == 2) w[2 + m + k] = wet ? q[var_b<N>(k)] / h : T(0);
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

// Cell record of the face state on side s (-1 / +1) of a cell (state qc, slopes sig); reflect: the
// state is the ghost across a wall of direction d (the normal moment components change sign).
template <int N, int D, typename T>
__device__ __forceinline__ void face_rec(const T *qc, const T *sig, int s, int d, bool reflect, T hdry,
                                         CellRec<N, D, T> &r)
{
    constexpr int m = N + 1, nv = O2<N, D>::nv, nw = O2<N, D>::nw;
    T w[nw];
    prim<N, D, T>(qc, hdry, w);
    const T hs = T(0.5) * T(s);
#pragma unroll
    for (int v = 0; v < nw; ++v) w[v] += hs * sig[v];
    const T bf = qc[nv] + hs * (sig[1] - sig[0]);
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
            case 0: return launch_o2<0, 2, T>(a, stage, nsm, st);
            case 1: return launch_o2<1, 2, T>(a, stage, nsm, st);
            case 2: return launch_o2<2, 2, T>(a, stage, nsm, st);
            case 3: return launch_o2<3, 2, T>(a, stage, nsm, st);
            case 4: return launch_o2<4, 2, T>(a, stage, nsm, st);
        }
    }
    return cudaErrorInvalidValue;
}

template cudaError_t launch_stage_order2<float>(int, int, const StageArgs<float> &, int, int, cudaStream_t);
template cudaError_t launch_stage_order2<double>(int, int, const StageArgs<double> &, int, int, cudaStream_t);

}  // namespace zoomy
