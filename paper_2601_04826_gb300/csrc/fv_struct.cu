// fv_struct.cu -- fused SSP-RK2 stage kernels on uniform 1D and structured 2D grids.
//
// One launch performs one stage of the SSP-RK2 step (reading of the time integrator):
//   stage 1:  Q1      = R(Q^n + dt L(Q^n))
//   stage 2:  Q^{n+1} = 1/2 (Q^n + R(Q1 + dt L(Q1)))     and  s_max(Q^{n+1}) for the next dt
// where L is the path-conservative Rusanov operator with hydrostatic reconstruction plus the
// Newtonian source (Eq. (PDE-hyperbolic), Sec. 2.1.2) and R the implicit bottom stress and
// dry cut (Eq. (PDE-source)).  Each stage reads its input once and writes Q once.
#include <cstdint>
#include <cuda_runtime.h>

#include "fv_common.cuh"
#include "zoomy_kernels.h"

namespace zoomy {

// ----------------------------------------------------------------------------------------
// 1D: one thread per cell; the thread evaluates its two faces (cell-centric).
// ----------------------------------------------------------------------------------------

template <int N, typename T>
__device__ __forceinline__ void load_cell_1d(const StageArgs<T> &a, int i, CellRec<N, 1, T> &r, T *raw)
{
    constexpr int m = N + 1;
    const int src = (int)bounds_idx(i < 0 ? 0 : (i >= a.nx ? a.nx - 1 : i), a.nx, &a.ctl->status);
    bool wall = (i < 0 && a.bc[0] == 1) || (i >= a.nx && a.bc[1] == 1);
    T h = a.X[src];
    T ha[m];
#pragma unroll
    for (int k = 0; k < m; ++k) {
        ha[k] = a.X[(int64_t)(1 + k) * a.ld + src];
        if (wall) ha[k] = -ha[k];
    }
    T b = a.bed ? a.bed[src] : T(0);
    make_cell<N, 1, T>(r, h, b, ha, nullptr, a.hdry);
    if (raw) {
        raw[0] = h;
#pragma unroll
        for (int k = 0; k < m; ++k) raw[1 + k] = ha[k];
    }
}

template <int N, typename T, int STAGE>
__global__ void __launch_bounds__(256) k_stage_1d(StageArgs<T> a)
{
    constexpr int m = N + 1, nv = 1 + m;
    pdl_enter();
    if (*(volatile unsigned int *)&a.ctl->status) return;
    T dt;
    if (!step_dt(a, dt)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&a.ctl->status, DEV_NOWAVE);
        return;
    }
    if (STAGE == 1 && blockIdx.x == 0 && threadIdx.x == 0) step_bookkeeping(a, dt);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    T s = T(0);
    if (i < a.nx) {
        CellRec<N, 1, T> cl, cc, cr;
        T raw[nv];
        load_cell_1d<N, T>(a, i - 1, cl, nullptr);
        load_cell_1d<N, T>(a, i, cc, raw);
        load_cell_1d<N, T>(a, i + 1, cr, nullptr);
        T acc[nv];
#pragma unroll
        for (int v = 0; v < nv; ++v) acc[v] = T(0);
        T fc[nv], nc[nv], pd;
        // left face (i-1 | i): this cell is R
        face_term<N, 1, T>(cl, frame<N, 1, T, false>(cl), cc, frame<N, 1, T, false>(cc), a.g, a.hdry, fc, pd, nc);
#pragma unroll
        for (int v = 0; v < nv; ++v) acc[v] += fc[v] - nc[v];
        acc[1] -= pd;
        // right face (i | i+1): this cell is L
        face_term<N, 1, T>(cc, frame<N, 1, T, false>(cc), cr, frame<N, 1, T, false>(cr), a.g, a.hdry, fc, pd, nc);
#pragma unroll
        for (int v = 0; v < nv; ++v) acc[v] -= fc[v] + nc[v];
        acc[1] -= pd;
        T sa[m];
        newtonian<N, 1, T>(cc, a.nu_rho, sa, nullptr);
        T y[nv];
        y[0] = raw[0] + dt * (a.inv_dx * acc[0]);
#pragma unroll
        for (int k = 0; k < m; ++k) y[1 + k] = raw[1 + k] + dt * (a.inv_dx * acc[1 + k]) + dt * sa[k];
        if (a.src_implicit)
            friction_implicit<N, 1, T>(y[0], y + 1, nullptr, a.fric, a.C_rho, a.nu_imp, a.gn2, dt, a.hdry);
        else
            bottom_friction<N, 1, T>(y[0], y + 1, nullptr, a.fric, a.C_rho, a.gn2, dt, a.hdry);
        if (STAGE == 2) {
#pragma unroll
            for (int v = 0; v < nv; ++v) y[v] = T(0.5) * (a.Qn[(int64_t)v * a.ld + i] + y[v]);
            CellRec<N, 1, T> co;
            make_cell<N, 1, T>(co, y[0], T(0), y + 1, nullptr, a.hdry);
            s = wavespeed<N, 1, T>(co, a.g);
            unsigned int flag = 0;
            if (!(s <= T(1e300))) flag |= DEV_NAN;
            if (!(y[0] >= T(0))) flag |= (y[0] < T(0)) ? DEV_NEGDEPTH : DEV_NAN;
            if (flag) atomicOr(&a.ctl->status, flag);
        }
#pragma unroll
        for (int v = 0; v < nv; ++v) a.out[(int64_t)v * a.ld + i] = y[v];
    }
    if (STAGE == 2) reduce_smax<T>(a.ctl, a.slot_out, s);
}

// ----------------------------------------------------------------------------------------
// 2D: row-marching warps.  A warp owns a strip of 30 columns and H rows; lane l holds
// column c0 - 1 + l (lanes 0 and 31 are the halo columns).  The warp walks down its rows
// keeping the previous row in registers, so every y-face is evaluated once with no data
// exchange and every x-face once with a register shuffle; each cell is loaded once per
// stage (plus one halo row per segment and two halo columns per strip).
// ----------------------------------------------------------------------------------------

constexpr int STRIP = 30;

template <int N, typename T>
__device__ __forceinline__ CellRec<N, 2, T> shfl_up_rec(const CellRec<N, 2, T> &r)
{
    constexpr int m = N + 1;
    constexpr unsigned F = 0xffffffffu;
    CellRec<N, 2, T> o;
    o.h = __shfl_up_sync(F, r.h, 1);
    o.b = __shfl_up_sync(F, r.b, 1);
    o.um = __shfl_up_sync(F, r.um, 1);
    o.s2 = __shfl_up_sync(F, r.s2, 1);
    o.s1 = __shfl_up_sync(F, r.s1, 1);
#pragma unroll
    for (int k = 0; k < m; ++k) {
        o.a[k] = __shfl_up_sync(F, r.a[k], 1);
        o.c[k] = __shfl_up_sync(F, r.c[k], 1);
        o.gaa[k] = __shfl_up_sync(F, r.gaa[k], 1);
        o.gab[k] = __shfl_up_sync(F, r.gab[k], 1);
    }
    return o;
}

template <int N, typename T, int STAGE>
__global__ void __launch_bounds__(128) k_stage_2d(StageArgs<T> a)
{
    constexpr int m = N + 1, nv = 3 + 2 * N;
    constexpr unsigned F = 0xffffffffu;
    if (*(volatile unsigned int *)&a.ctl->status) return;
    T dt;
    if (!step_dt(a, dt)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&a.ctl->status, DEV_NOWAVE);
        return;
    }
    if (STAGE == 1 && blockIdx.x == 0 && threadIdx.x == 0) step_bookkeeping(a, dt);

    const int lane = threadIdx.x & 31;
    const int wg = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int strip = wg % a.nstrips, seg = wg / a.nstrips;
    if (seg >= a.nsegs) return;  // whole warp leaves together
    const int col = strip * STRIP - 1 + lane;
    const bool owned = lane >= 1 && lane <= STRIP && col < a.nx;
    const int csrc = col < 0 ? 0 : (col >= a.nx ? a.nx - 1 : col);
    const bool xwall = (col < 0 && a.bc[0] == 1) || (col >= a.nx && a.bc[1] == 1);
    const int r0 = seg * a.H;
    const int r1 = min(r0 + a.H, a.ny);

    CellRec<N, 2, T> prev, cur;
    T xprev[nv], xcur[nv], accp[nv], accc[nv];
    // loop-carried values start defined (the first row is a halo row whose faces are unused)
    {
        T zero[m];
#pragma unroll
        for (int k = 0; k < m; ++k) zero[k] = T(0);
        make_cell<N, 2, T>(prev, T(0), T(0), zero, zero, a.hdry);
#pragma unroll
        for (int v = 0; v < nv; ++v) xprev[v] = accp[v] = T(0);
    }
    T smax = T(0);
    unsigned int flag = 0;

    for (int r = r0 - 1; r <= r1; ++r) {
        const int rsrc = r < 0 ? 0 : (r >= a.ny ? a.ny - 1 : r);
        const bool ywall = (r < 0 && a.bc[2] == 1) || (r >= a.ny && a.bc[3] == 1);
        const int64_t cidx = bounds_idx((int64_t)rsrc * a.nx + csrc, (int64_t)a.nx * a.ny, &a.ctl->status);
        // load the stage input of this row (ghost rows/columns mirror the boundary cell)
#pragma unroll
        for (int v = 0; v < nv; ++v) xcur[v] = a.X[(int64_t)v * a.ld + cidx];
        const T bcur = a.bed ? a.bed[cidx] : T(0);
        T ha[m], hb[m];
#pragma unroll
        for (int k = 0; k < m; ++k) {
            ha[k] = xcur[var_a<N, 2>(k)];
            hb[k] = xcur[var_b<N>(k)];
            if (xwall) ha[k] = -ha[k];
            if (ywall) hb[k] = -hb[k];
        }
        make_cell<N, 2, T>(cur, xcur[0], bcur, ha, hb, a.hdry);
#pragma unroll
        for (int v = 0; v < nv; ++v) accc[v] = T(0);

        T fc[1 + 2 * m], nc[1 + 2 * m], pd;
        if (r >= r0 && r < r1) {
            // x-face (col-1 | col), evaluated by the lane on its right
            CellRec<N, 2, T> left = shfl_up_rec<N, T>(cur);
            face_term<N, 2, T>(left, frame<N, 2, T, false>(left), cur, frame<N, 2, T, false>(cur), a.g, a.hdry,
                               fc, pd, nc);
            T tl[nv];
            tl[0] = -(fc[0] + nc[0]);
            accc[0] += fc[0] - nc[0];
#pragma unroll
            for (int k = 0; k < m; ++k) {
                const int ia = var_a<N, 2>(k), ib = var_b<N>(k);
                tl[ia] = -(fc[1 + k] + nc[1 + k]);
                tl[ib] = -(fc[1 + m + k] + nc[1 + m + k]);
                accc[ia] += fc[1 + k] - nc[1 + k];
                accc[ib] += fc[1 + m + k] - nc[1 + m + k];
            }
            tl[var_a<N, 2>(0)] -= pd;
            accc[var_a<N, 2>(0)] -= pd;
#pragma unroll
            for (int v = 0; v < nv; ++v) {
                accc[v] *= a.inv_dx;
                accc[v] += a.inv_dx * __shfl_down_sync(F, tl[v], 1);
            }
        }
        if (r > r0 - 1) {
            // y-face (r-1 | r): prev is below (L), cur above (R); frame (n, t) = (beta, alpha)
            face_term<N, 2, T>(prev, frame<N, 2, T, true>(prev), cur, frame<N, 2, T, true>(cur), a.g, a.hdry, fc,
                               pd, nc);
            accp[0] -= a.inv_dy * (fc[0] + nc[0]);
            accc[0] += a.inv_dy * (fc[0] - nc[0]);
#pragma unroll
            for (int k = 0; k < m; ++k) {
                const int ib = var_b<N>(k), ia = var_a<N, 2>(k);
                accp[ib] -= a.inv_dy * (fc[1 + k] + nc[1 + k]);
                accp[ia] -= a.inv_dy * (fc[1 + m + k] + nc[1 + m + k]);
                accc[ib] += a.inv_dy * (fc[1 + k] - nc[1 + k]);
                accc[ia] += a.inv_dy * (fc[1 + m + k] - nc[1 + m + k]);
            }
            accp[var_b<N>(0)] -= a.inv_dy * pd;
            accc[var_b<N>(0)] -= a.inv_dy * pd;

            if (r - 1 >= r0 && owned) {
                // finalize cell (r-1, col)
                const int64_t oidx = (int64_t)(r - 1) * a.nx + col;
                T sa[m], sb[m];
                newtonian<N, 2, T>(prev, a.nu_rho, sa, sb);
                T y[nv];
                y[0] = xprev[0] + dt * accp[0];
                T ya[m], yb[m];
#pragma unroll
                for (int k = 0; k < m; ++k) {
                    const int ia = var_a<N, 2>(k), ib = var_b<N>(k);
                    ya[k] = xprev[ia] + dt * accp[ia] + dt * sa[k];
                    yb[k] = xprev[ib] + dt * accp[ib] + dt * sb[k];
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
                    for (int v = 0; v < nv; ++v) y[v] = T(0.5) * (a.Qn[(int64_t)v * a.ld + oidx] + y[v]);
                    CellRec<N, 2, T> co;
#pragma unroll
                    for (int k = 0; k < m; ++k) {
                        ya[k] = y[var_a<N, 2>(k)];
                        yb[k] = y[var_b<N>(k)];
                    }
                    make_cell<N, 2, T>(co, y[0], T(0), ya, yb, a.hdry);
                    T s = wavespeed<N, 2, T>(co, a.g);
                    if (!(s <= T(3.0e38))) flag |= DEV_NAN;
                    if (!(y[0] >= T(0))) flag |= (y[0] < T(0)) ? DEV_NEGDEPTH : DEV_NAN;
                    smax = (s > smax || s != s) ? s : smax;
                }
#pragma unroll
                for (int v = 0; v < nv; ++v) a.out[(int64_t)v * a.ld + oidx] = y[v];
            }
        }
        prev = cur;
#pragma unroll
        for (int v = 0; v < nv; ++v) {
            xprev[v] = xcur[v];
            accp[v] = accc[v];
        }
    }
    if (STAGE == 2) {
        if (flag) atomicOr(&a.ctl->status, flag);
        reduce_smax<T>(a.ctl, a.slot_out, smax);
    }
}

// ----------------------------------------------------------------------------------------
// Host launchers
// ----------------------------------------------------------------------------------------

template <int N, typename T>
static cudaError_t launch_1d(const StageArgs<T> &a, int stage, cudaStream_t st)
{
    // small lines (the work is FP64-rate bound, not memory bound): one-warp CTAs spread the cells
    // over as many SMs as possible; large lines use 256-thread CTAs
    // (programmatic dependent launch: each stage's launch overlaps the previous kernel's tail)
    const int bs = a.nx < 65536 ? 32 : 256;
    dim3 grid((a.nx + bs - 1) / bs), block(bs);
    if (stage == 1) return launch_pdl(k_stage_1d<N, T, 1>, grid, block, st, a);
    return launch_pdl(k_stage_1d<N, T, 2>, grid, block, st, a);
}

template <int N, typename T>
static cudaError_t launch_2d(const StageArgs<T> &a, int stage, int warps_per_block, cudaStream_t st)
{
    const int nwarps = a.nstrips * a.nsegs;
    dim3 grid((nwarps + warps_per_block - 1) / warps_per_block), block(32 * warps_per_block);
    if (stage == 1)
        k_stage_2d<N, T, 1><<<grid, block, 0, st>>>(a);
    else
        k_stage_2d<N, T, 2><<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_stage_struct(int dim, int level, const StageArgs<T> &a, int stage, int warps_per_block,
                                cudaStream_t st)
{
    if (dim == 1) {
        switch (level) {
            case 0: return launch_1d<0, T>(a, stage, st);
            case 1: return launch_1d<1, T>(a, stage, st);
            case 2: return launch_1d<2, T>(a, stage, st);
            case 3: return launch_1d<3, T>(a, stage, st);
            case 4: return launch_1d<4, T>(a, stage, st);
        }
    } else {
        switch (level) {
            case 0: return launch_2d<0, T>(a, stage, warps_per_block, st);
            case 1: return launch_2d<1, T>(a, stage, warps_per_block, st);
            case 2: return launch_2d<2, T>(a, stage, warps_per_block, st);
            case 3: return launch_2d<3, T>(a, stage, warps_per_block, st);
            case 4: return launch_2d<4, T>(a, stage, warps_per_block, st);
        }
    }
    return cudaErrorInvalidValue;
}

template cudaError_t launch_stage_struct<float>(int, int, const StageArgs<float> &, int, int, cudaStream_t);
template cudaError_t launch_stage_struct<double>(int, int, const StageArgs<double> &, int, int, cudaStream_t);

}  // namespace zoomy
