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
// 1D: face-centric warps.  Lane l of a warp takes the face (c-1 | c), c = base + l, and lanes 0..30
// update the cells base..base+30 (31 cells per warp) with their own face on the left and the next
// lane's face on the right.  Each face is evaluated once (twice at warp seams) instead of once for
// each of its two cells: the FP64 line is bound by the instruction stream of each warp.
// ----------------------------------------------------------------------------------------

constexpr int CELLS_PER_WARP_1D = 31;

// Loads of the state go through L2 only (ld.global.cg) in every 1D kernel: the persistent kernel reads
// data other CTAs of the same launch wrote before a grid barrier, which L1 may hold stale.
template <int N, typename T>
__device__ __forceinline__ void load_cell_1d(const StageArgs<T> &a, const T *X, int i, CellRec<N, 1, T> &r, T *raw)
{
    constexpr int m = N + 1;
    const int src = (int)bounds_idx(i < 0 ? 0 : (i >= a.nx ? a.nx - 1 : i), a.nx, &a.ctl->status);
    bool wall = (i < 0 && a.bc[0] == 1) || (i >= a.nx && a.bc[1] == 1);
    T h = __ldcg(X + src);
    T ha[m];
#pragma unroll
    for (int k = 0; k < m; ++k) {
        ha[k] = __ldcg(X + (int64_t)(1 + k) * a.ld + src);
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

// One stage of the 31 cells base.. of a 1D line, called by all 32 lanes of a warp (the shuffles need the
// full warp): each lane evaluates its face, then the lanes with a cell c < nx add both faces, the
// source and the bottom stress, (stage 2) take the SSP-RK2 average with Q^n, write the cell to out
// and return (stage 2) its wave speed.  Faces beyond the line (c > nx) read clamped cells and are not
// used.  Kept out of line: the per-stage kernels and the persistent kernel call this one compiled body,
// so both launch shapes execute the same instructions (inlined into different kernels, the compiler
// may contract multiplies and adds into FMAs differently, which changes the last bit).
template <int N, typename T, int STAGE>
__device__ __noinline__ T stage_1d_warp(const StageArgs<T> &a, const T *X, const T *Qn, T *out, T dt, int base)
{
    constexpr int m = N + 1, nv = 1 + m;
    const int lane = threadIdx.x & 31, c = base + lane;
    CellRec<N, 1, T> cl, cc;
    T raw[nv];
    load_cell_1d<N, T>(a, X, c - 1, cl, nullptr);
    load_cell_1d<N, T>(a, X, c, cc, raw);
    T fl[nv], nl[nv], pl;
    face_term<N, 1, T>(cl, frame<N, 1, T, false>(cl), cc, frame<N, 1, T, false>(cc), a.g, a.hdry, fl, pl, nl);
    // the right face (c | c+1) is the next lane's
    T fr[nv], nr[nv];
#pragma unroll
    for (int v = 0; v < nv; ++v) {
        fr[v] = __shfl_down_sync(0xffffffffu, fl[v], 1);
        nr[v] = __shfl_down_sync(0xffffffffu, nl[v], 1);
    }
    const T pr = __shfl_down_sync(0xffffffffu, pl, 1);
    T s = T(0);
    if (lane < CELLS_PER_WARP_1D && c < a.nx) {
        T acc[nv];
#pragma unroll
        for (int v = 0; v < nv; ++v) acc[v] = T(0);
        // left face: this cell is R; right face: this cell is L
#pragma unroll
        for (int v = 0; v < nv; ++v) acc[v] += fl[v] - nl[v];
        acc[1] -= pl;
#pragma unroll
        for (int v = 0; v < nv; ++v) acc[v] -= fr[v] + nr[v];
        acc[1] -= pr;
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
            for (int v = 0; v < nv; ++v) y[v] = T(0.5) * (__ldcg(Qn + (int64_t)v * a.ld + c) + y[v]);
            CellRec<N, 1, T> co;
            make_cell<N, 1, T>(co, y[0], T(0), y + 1, nullptr, a.hdry);
            s = wavespeed<N, 1, T>(co, a.g);
            unsigned int flag = 0;
            if (!(s <= T(1e300))) flag |= DEV_NAN;
            if (!(y[0] >= T(0))) flag |= (y[0] < T(0)) ? DEV_NEGDEPTH : DEV_NAN;
            if (flag) atomicOr(&a.ctl->status, flag);
        }
#pragma unroll
        for (int v = 0; v < nv; ++v) out[(int64_t)v * a.ld + c] = y[v];
    }
    return s;
}

// One stage, one warp per 31 cells (warp-uniform exit past the line).
template <int N, typename T, int STAGE>
__global__ void __launch_bounds__(256) k_stage_1d(const __grid_constant__ StageArgs<T> a)
{
    pdl_enter();
    if (*(volatile unsigned int *)&a.ctl->status) return;
    T dt;
    if (!step_dt(a, a.slot_in, dt)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&a.ctl->status, DEV_NOWAVE);
        return;
    }
    if (STAGE == 1 && blockIdx.x == 0 && threadIdx.x == 0) step_bookkeeping(a, a.slot_out, dt);
    const int base = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * CELLS_PER_WARP_1D;
    if (base >= a.nx) return;
    const T s = stage_1d_warp<N, T, STAGE>(a, a.X, a.Qn, a.out, dt, base);
    if (STAGE == 2) reduce_smax<T>(a.ctl, a.slot_out, s);
}

// Grid barrier of a cooperative launch on bar = DevCtl::bar (arrivals, generation, status snapshot;
// zero at the launch).  Thread 0 of each CTA arrives; the last one copies the sticky status into the
// snapshot before it releases the others, so every CTA takes the same decision.  Returns true when the
// CTA is to stop: the snapshot shows a device-detected error (the per-stage kernels skip their work
// then too), or this CTA's bounded wait ran out (DEV_TIMEOUT).
__device__ __forceinline__ bool grid_barrier_1d(unsigned *bar, unsigned nbar, unsigned *status, long long spin_limit)
{
    __shared__ unsigned stop;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vb = bar;
        const unsigned g0 = vb[1];
        __threadfence();
        if (atomicAdd(bar, 1u) == nbar - 1) {
            vb[0] = 0u;
            vb[2] = *(volatile unsigned *)status;
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long long it = 0;
            while (vb[1] == g0) {
                if (++it > spin_limit) {
                    atomicOr(status, DEV_TIMEOUT);
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        stop = vb[1] == g0 || vb[2] != 0u;
    }
    __syncthreads();
    return stop != 0u;
}

// Every step of a zoomy_step call on a short 1D line in one cooperative launch: stage 1 (Q -> Q1),
// grid barrier, stage 2 (Q1 and Q^n = Q -> Q, wave-speed maximum), grid barrier.  The stages are the
// per-stage kernels' warp body (stage_1d_warp, the same compiled function); the step size, the time
// and wave-speed slot bookkeeping and the skip after a device-detected error are those of two
// launches per step, so the state is bitwise the same.
template <int N, typename T>
__global__ void __launch_bounds__(256) k_steps_1d(const __grid_constant__ StageArgs<T> a, T *Q, T *Q1, int nsteps,
                                                  unsigned nbar, long long spin_limit)
{
    const int base = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * CELLS_PER_WARP_1D;
    unsigned *bar = a.ctl->bar;
    // an error left by an earlier call of this context skips the call (as in the per-stage kernels);
    // taken from the barrier's snapshot so that every CTA decides alike
    if (grid_barrier_1d(bar, nbar, &a.ctl->status, spin_limit)) return;
    for (int k = 0; k < nsteps; ++k) {
        const int slot_in = k & 1, slot_out = (k + 1) & 1;
        T dt;
        // every CTA reads the same s_max (final before the last barrier), so all of them stop here
        if (!step_dt(a, slot_in, dt)) {
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&a.ctl->status, DEV_NOWAVE);
            return;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) step_bookkeeping(a, slot_out, dt);
        T s = T(0);
        if (base < a.nx) stage_1d_warp<N, T, 1>(a, Q, Q, Q1, dt, base);
        if (grid_barrier_1d(bar, nbar, &a.ctl->status, spin_limit)) return;
        if (base < a.nx) s = stage_1d_warp<N, T, 2>(a, Q1, Q, Q, dt, base);
        reduce_smax<T>(a.ctl, slot_out, s);
        if (grid_barrier_1d(bar, nbar, &a.ctl->status, spin_limit)) return;
    }
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
static cudaError_t launch_1d(const StageArgs<T> &a, int stage, int warps_per_cta, cudaStream_t st)
{
    // programmatic dependent launch: each stage's launch overlaps the previous kernel's tail
    const int nwarps = (a.nx + CELLS_PER_WARP_1D - 1) / CELLS_PER_WARP_1D;
    dim3 grid((nwarps + warps_per_cta - 1) / warps_per_cta), block(32 * warps_per_cta);
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
cudaError_t launch_stage_struct(int dim, int level, const StageArgs<T> &a, int stage, int block_shape,
                                cudaStream_t st)
{
    if (dim == 1) {
        const int warps_per_cta = block_shape;
        switch (level) {
            case 0: return launch_1d<0, T>(a, stage, warps_per_cta, st);
            case 1: return launch_1d<1, T>(a, stage, warps_per_cta, st);
            case 2: return launch_1d<2, T>(a, stage, warps_per_cta, st);
            case 3: return launch_1d<3, T>(a, stage, warps_per_cta, st);
            case 4: return launch_1d<4, T>(a, stage, warps_per_cta, st);
        }
    } else {
        switch (level) {
            case 0: return launch_2d<0, T>(a, stage, block_shape, st);
            case 1: return launch_2d<1, T>(a, stage, block_shape, st);
            case 2: return launch_2d<2, T>(a, stage, block_shape, st);
            case 3: return launch_2d<3, T>(a, stage, block_shape, st);
            case 4: return launch_2d<4, T>(a, stage, block_shape, st);
        }
    }
    return cudaErrorInvalidValue;
}

template <int N, typename T>
static cudaError_t launch_steps_1d_n(const StageArgs<T> &a, T *Q, T *Q1, int nsteps, int warps_per_cta, int nsm,
                                     cudaStream_t st)
{
    const int nwarps = (a.nx + CELLS_PER_WARP_1D - 1) / CELLS_PER_WARP_1D;
    const unsigned nb = (unsigned)((nwarps + warps_per_cta - 1) / warps_per_cta);
    const int bs = 32 * warps_per_cta;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_steps_1d<N, T>, bs, 0);
    if (e != cudaSuccess) return e;
    if ((long long)nb > (long long)per_sm * nsm) return cudaErrorCooperativeLaunchTooLarge;
    long long spin = 20000000LL;  // at least 0.6 s of 32 ns naps
    void *args[] = {(void *)&a, (void *)&Q, (void *)&Q1, (void *)&nsteps, (void *)&nb, (void *)&spin};
    return cudaLaunchCooperativeKernel((const void *)k_steps_1d<N, T>, dim3(nb), dim3(bs), args, 0, st);
}

template <typename T>
cudaError_t launch_steps_1d(int level, const StageArgs<T> &a, T *Q, T *Q1, int nsteps, int warps_per_cta, int nsm,
                            cudaStream_t st)
{
    if (warps_per_cta < 1 || warps_per_cta > 8) return cudaErrorInvalidValue;
    switch (level) {
        case 0: return launch_steps_1d_n<0, T>(a, Q, Q1, nsteps, warps_per_cta, nsm, st);
        case 1: return launch_steps_1d_n<1, T>(a, Q, Q1, nsteps, warps_per_cta, nsm, st);
        case 2: return launch_steps_1d_n<2, T>(a, Q, Q1, nsteps, warps_per_cta, nsm, st);
        case 3: return launch_steps_1d_n<3, T>(a, Q, Q1, nsteps, warps_per_cta, nsm, st);
        case 4: return launch_steps_1d_n<4, T>(a, Q, Q1, nsteps, warps_per_cta, nsm, st);
    }
    return cudaErrorInvalidValue;
}

template cudaError_t launch_steps_1d<float>(int, const StageArgs<float> &, float *, float *, int, int, int,
                                            cudaStream_t);
template cudaError_t launch_steps_1d<double>(int, const StageArgs<double> &, double *, double *, int, int, int,
                                             cudaStream_t);

template cudaError_t launch_stage_struct<float>(int, int, const StageArgs<float> &, int, int, cudaStream_t);
template cudaError_t launch_stage_struct<double>(int, int, const StageArgs<double> &, int, int, cudaStream_t);

}  // namespace zoomy
