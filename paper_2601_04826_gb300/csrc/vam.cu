// vam.cu -- the non-hydrostatic VAM predictor-corrector in 1D (Sec. "Unsteady Vertically Averaged
// Momentum Equations in 1D"; the splitting of Eq. (PDE-hyperbolic) - Eq. (PDE-source)), FP64, flat bed.
//
//   Q = (h, h u0, h u1, h w0, h w1), w2 = -(w0 + w1)
//   predictor: Q* = Q^n - dt/dx (D+_{i-1/2} + D-_{i+1/2}), path-conservative Rusanov fluctuations
//     D-+ = (F(QR) - F(QL))/2 + Btilde (QR - QL)/2 -+ s_f (QR - QL)/2 with
//     F = (h u0, h u0^2 + h u1^2/3, 2 h u0 u1, h u0 w0 + h u1 w1/3, h u0 w1 + u1 (h w0 + 2/5 h w2)),
//     B: row h u0 g h on h; row h u1 -u0 on h u1; row h w1 (w2/5 - w0) on h u1 (3-point Gauss-Legendre
//     average on the straight segment), s = |u0| + sqrt(g h + u1^2) + |u1|;
//   corrector: the pressure (p0, p1) per cell such that Q** = Q* - dt S(p),
//     S = (0, d(h p0)/dx, d(h p1)/dx - (3 p0 - p1) dh/dx, -2 p1, 6 (p0 - p1)),
//     satisfies R0 = h du0/dx + d(h u1)/dx/3 + u1 dh/dx/3 + 2 w0 = 0 and R1 = h du0/dx + u1 dh/dx - 2 w1 = 0
//     with central differences and mirrored ghosts (u0, u1 and their momenta change sign at walls).
//
// The constraints are linear in p with a stencil of two cells on each side, so the matrix is banded
// (unknowns interleaved (p0_i, p1_i): 5 sub- and 5 super-diagonals).  It is assembled without any
// symbolic derivation: probing with the 10 vectors that are 1 on one component of every fifth cell
// (cells five apart never share a row) gives every band entry as R(probe) - R(0).  The banded system
// is solved by Gaussian elimination with partial pivoting in one warp (1D problems are small).
#include <cmath>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/zoomy.h"
#include "fv_common.cuh"
#include "zoomy_internal.h"

namespace zoomy {

constexpr int VKL = 5, VKU = 5, VW = 2 * VKL + VKU + 1;  // band half-widths, stored row width (with fill)

struct VamArgs {
    double *Q;        // state [5][ld] (in: Q^n, out: Q^{n+1})
    double *Qs;       // predictor result Q* [5][ld]
    double *band;     // [2 nc][VW]: A(r, c) at band[r * VW + (c - r + VKL)]
    double *rhs;      // [2 nc]: -R(0), then the solution p
    int64_t ld, nc;
    double dx, g, cfl;
    int bcl, bcr;     // 1 wall, 0 transmissive
    DevCtl *ctl;
    double dt_fixed;
    int slot_in, slot_out;
};

__device__ __forceinline__ double vq(const VamArgs &a, const double *Q, int v, int64_t j)
{
    // state with mirrored ghosts; walls change the sign of the horizontal momenta (v = 1, 2)
    if (j < 0) return (v == 1 || v == 2) && a.bcl == 1 ? -Q[v * a.ld] : Q[v * a.ld];
    if (j >= a.nc) return (v == 1 || v == 2) && a.bcr == 1 ? -Q[v * a.ld + a.nc - 1] : Q[v * a.ld + a.nc - 1];
    return Q[v * a.ld + j];
}

__device__ __forceinline__ double vspeed(const double *q, double g)
{
    const double u0 = q[1] / q[0], u1 = q[2] / q[0];
    return fabs(u0) + sqrt(g * q[0] + u1 * u1) + fabs(u1);
}

__device__ __forceinline__ void vflux(const double *q, double *F)
{
    const double h = q[0], u0 = q[1] / h, u1 = q[2] / h, w0 = q[3] / h, w1 = q[4] / h, w2 = -(w0 + w1);
    F[0] = h * u0;
    F[1] = h * u0 * u0 + h * u1 * u1 / 3.0;
    F[2] = 2.0 * h * u0 * u1;
    F[3] = h * u0 * w0 + h * u1 * w1 / 3.0;
    F[4] = h * u0 * w1 + u1 * (h * w0 + 0.4 * h * w2);
}

// Fluctuations of the face between states qL, qR: dm (to the left cell), dp (to the right cell).
__device__ __forceinline__ void vface(const double *qL, const double *qR, double g, double *dm, double *dp)
{
    double FL[5], FR[5], dq[5], bt[5] = {0, 0, 0, 0, 0};
    vflux(qL, FL);
    vflux(qR, FR);
    for (int v = 0; v < 5; ++v) dq[v] = qR[v] - qL[v];
    const double sq[3] = {0.5 - 0.38729833462074168852, 0.5, 0.5 + 0.38729833462074168852};
    const double wq[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
    for (int k = 0; k < 3; ++k) {
        double p[5];
        for (int v = 0; v < 5; ++v) p[v] = qL[v] + sq[k] * dq[v];
        const double h = p[0], u0 = p[1] / h, w0 = p[3] / h, w1 = p[4] / h, w2 = -(w0 + w1);
        bt[1] += wq[k] * g * h * dq[0];
        bt[2] += wq[k] * (-u0) * dq[2];
        bt[4] += wq[k] * (w2 / 5.0 - w0) * dq[2];
    }
    const double sL = vspeed(qL, g), sR = vspeed(qR, g), sf = sL > sR ? sL : sR;
    for (int v = 0; v < 5; ++v) {
        const double c = 0.5 * (FR[v] - FL[v]) + 0.5 * bt[v];
        dm[v] = c - 0.5 * sf * dq[v];
        dp[v] = c + 0.5 * sf * dq[v];
    }
}

__device__ __forceinline__ double vam_dt(const VamArgs &a)
{
    if (a.dt_fixed > 0.0) return a.dt_fixed;
    const double smax = __longlong_as_double((long long)*(volatile unsigned long long *)&a.ctl->smax_d[a.slot_in]);
    return (smax > 0.0 && smax < 1e300) ? a.cfl * a.dx / smax : 0.0;
}

// max s over Q^n into the slot of this step
__global__ void __launch_bounds__(128) k_vam_wavespeed(VamArgs a)
{
    double s = 0.0;
    unsigned flag = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.nc; i += (int64_t)gridDim.x * blockDim.x) {
        double q[5];
        for (int v = 0; v < 5; ++v) q[v] = a.Q[v * a.ld + i];
        const double si = vspeed(q, a.g);
        if (!(q[0] > 0.0)) flag |= q[0] < 0.0 ? DEV_NEGDEPTH : DEV_NAN;
        s = (si > s || si != si) ? si : s;
    }
    if (flag) atomicOr(&a.ctl->status, flag);
    reduce_smax<double>(a.ctl, a.slot_out, s);
}

__global__ void __launch_bounds__(128) k_vam_predict(VamArgs a)
{
    if (*(volatile unsigned int *)&a.ctl->status) return;
    const double dt = vam_dt(a);
    if (!(dt > 0.0)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&a.ctl->status, DEV_NOWAVE);
        return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctl->t += dt;
        a.ctl->dt_last = dt;
        a.ctl->smax_d[a.slot_out] = 0ull;  // the next step's slot
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.nc; i += (int64_t)gridDim.x * blockDim.x) {
        double ql[5], qc[5], qr[5], dm[5], dp[5], dml[5], dpl[5];
        for (int v = 0; v < 5; ++v) {
            ql[v] = vq(a, a.Q, v, i - 1);
            qc[v] = vq(a, a.Q, v, i);
            qr[v] = vq(a, a.Q, v, i + 1);
        }
        vface(ql, qc, a.g, dml, dpl);  // face i-1/2: this cell is on the right
        vface(qc, qr, a.g, dm, dp);    // face i+1/2: this cell is on the left
        for (int v = 0; v < 5; ++v) a.Qs[v * a.ld + i] = qc[v] - dt / a.dx * (dpl[v] + dm[v]);
    }
}

// Probe pattern: component `comp` of every cell j with j % 5 == color is 1 (color < 0: p = 0).
struct Probe {
    int color, comp;
    const double *p;  // or, when non-null, an explicit pressure [2 nc]
    __device__ __forceinline__ double get(int64_t j, int c) const
    {
        if (p) return p[2 * j + c];
        return (color >= 0 && c == comp && (int)(j % 5) == color) ? 1.0 : 0.0;
    }
};

// Q** = Q* - dt S(p) at real cell j (mirrored ghosts for the differences inside S).
__device__ __forceinline__ void vcorrected(const VamArgs &a, const Probe &pr, int64_t j, double dt, double *q)
{
    const int64_t jl = j > 0 ? j - 1 : 0, jr = j + 1 < a.nc ? j + 1 : a.nc - 1;
    const double h = a.Qs[j], hl = a.Qs[jl], hr = a.Qs[jr];
    const double i2dx = 0.5 / a.dx;
    const double p0 = pr.get(j, 0), p1 = pr.get(j, 1);
    const double dhp0 = (hr * pr.get(jr, 0) - hl * pr.get(jl, 0)) * i2dx;
    const double dhp1 = (hr * pr.get(jr, 1) - hl * pr.get(jl, 1)) * i2dx;
    const double dh = (hr - hl) * i2dx;
    q[0] = h;
    q[1] = a.Qs[a.ld + j] - dt * dhp0;
    q[2] = a.Qs[2 * a.ld + j] - dt * (dhp1 - (3.0 * p0 - p1) * dh);
    q[3] = a.Qs[3 * a.ld + j] + dt * 2.0 * p1;
    q[4] = a.Qs[4 * a.ld + j] - dt * 6.0 * (p0 - p1);
}

__device__ __forceinline__ void vresidual(const VamArgs &a, const Probe &pr, int64_t i, double dt, double *R)
{
    double qc[5], ql[5], qr[5];
    vcorrected(a, pr, i, dt, qc);
    if (i > 0) {
        vcorrected(a, pr, i - 1, dt, ql);
    } else {
        for (int v = 0; v < 5; ++v) ql[v] = qc[v];
        if (a.bcl == 1) ql[1] = -ql[1], ql[2] = -ql[2];
    }
    if (i + 1 < a.nc) {
        vcorrected(a, pr, i + 1, dt, qr);
    } else {
        for (int v = 0; v < 5; ++v) qr[v] = qc[v];
        if (a.bcr == 1) qr[1] = -qr[1], qr[2] = -qr[2];
    }
    const double i2dx = 0.5 / a.dx;
    const double h = qc[0], u1 = qc[2] / h, w0 = qc[3] / h, w1 = qc[4] / h;
    const double dh = (qr[0] - ql[0]) * i2dx;
    const double du0 = (qr[1] / qr[0] - ql[1] / ql[0]) * i2dx;
    const double dhu1 = (qr[2] - ql[2]) * i2dx;
    R[0] = h * du0 + dhu1 / 3.0 + u1 * dh / 3.0 + 2.0 * w0;
    R[1] = h * du0 + u1 * dh - 2.0 * w1;
}

// Band entries by probing, and the right-hand side -R(0); the fill columns start at zero.
__global__ void __launch_bounds__(128) k_vam_assemble(VamArgs a)
{
    if (*(volatile unsigned int *)&a.ctl->status) return;
    const double dt = *(volatile double *)&a.ctl->dt_last;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.nc; i += (int64_t)gridDim.x * blockDim.x) {
        double r0[2];
        vresidual(a, Probe{-1, 0, nullptr}, i, dt, r0);
        for (int r = 0; r < 2; ++r) {
            double *row = a.band + (2 * i + r) * VW;
            for (int w = 0; w < VW; ++w) row[w] = 0.0;
            a.rhs[2 * i + r] = -r0[r];
        }
        for (int color = 0; color < 5; ++color)
            for (int comp = 0; comp < 2; ++comp) {
                // the one cell of this color within the stencil i-2..i+2 of row i
                const int64_t j = i - 2 + (((color - (int)((i - 2 + 10 * 5) % 5)) % 5 + 5) % 5);
                if (j < 0 || j >= a.nc) continue;
                double rp[2];
                vresidual(a, Probe{color, comp, nullptr}, i, dt, rp);
                for (int r = 0; r < 2; ++r) {
                    const int64_t row = 2 * i + r, col = 2 * j + comp;
                    a.band[row * VW + (col - row + VKL)] = rp[r] - r0[r];
                }
            }
    }
}

// Gaussian elimination with partial pivoting on the band by one warp; the solution overwrites rhs.
// The elimination is a chain over the columns, so its working set stays in shared memory: the six
// rows k..k+5 that column k touches (row r in slot r % 6, column c at index c % 16; every row covers
// 16 consecutive columns from r - 5, entries left of the current column are kept at zero), the next
// row prefetched into registers during each step, the finished row k written back for the back
// substitution, which keeps the last solution values in a ring of 16.
__global__ void __launch_bounds__(32) k_vam_solve(VamArgs a)
{
    if (*(volatile unsigned int *)&a.ctl->status) return;
    constexpr unsigned F = 0xffffffffu;
    __shared__ double win[6][16];
    __shared__ double rw[6];
    __shared__ double xs[16];
    const int lane = threadIdx.x;
    const int64_t n = 2 * a.nc;
    double *band = a.band, *rhs = a.rhs;
    // row r of the band (offsets 0..15 = columns r-5..r+10) into its window slot
    auto load = [&](int64_t r, double &val, double &rv) {
        val = 0.0;
        rv = 0.0;
        if (r < n) {
            if (lane < 16) val = band[r * VW + lane];
            if (lane == 16) rv = rhs[r];
        }
    };
    auto put = [&](int64_t r, double val, double rv) {
        if (r < n) {
            if (lane < 16) win[r % 6][(r - 5 + lane) & 15] = val;
            if (lane == 16) rw[r % 6] = rv;
        }
    };
    for (int64_t r = 0; r < 6; ++r) {
        double val, rv;
        load(r, val, rv);
        put(r, val, rv);
    }
    __syncwarp();
    for (int64_t k = 0; k < n; ++k) {
        double nval, nrv;
        load(k + 6, nval, nrv);  // in flight during this step
        const int64_t rmax = k + VKL < n ? k + VKL : n - 1;
        const int64_t cmax = k + VKL + VKU < n ? k + VKL + VKU : n - 1;
        const int kc = (int)(k & 15);
        // pivot: the largest |A(r, k)|, r = k..rmax (lowest row on ties)
        double v = -1.0;
        int best = lane;
        if (lane <= rmax - k) v = fabs(win[(k + lane) % 6][kc]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(F, v, o);
            const int ob = __shfl_xor_sync(F, best, o);
            if (ov > v || (ov == v && ob < best)) {
                v = ov;
                best = ob;
            }
        }
        if (!(v > 0.0)) {
            if (lane == 0) atomicOr(&a.ctl->status, DEV_NAN);  // singular pressure system
            return;
        }
        const int sk = (int)(k % 6), sb = (int)((k + best) % 6);
        if (best != 0) {
            if (lane < 16) {
                const double t = win[sk][lane];
                win[sk][lane] = win[sb][lane];
                win[sb][lane] = t;
            }
            if (lane == 16) {
                const double t = rw[sk];
                rw[sk] = rw[sb];
                rw[sb] = t;
            }
        }
        __syncwarp();
        const double inv = 1.0 / win[sk][kc];
        const int nr = (int)(rmax - k), ncol = (int)(cmax - k);
        // multipliers of the rows below (read before any of them changes)
        double l = 0.0;
        if (lane < nr) l = win[(k + 1 + lane) % 6][kc] * inv;
        __syncwarp();
        for (int idx = lane; idx < nr * ncol; idx += 32) {
            const int rr = idx / ncol, cc = 1 + idx % ncol;
            const double lr = win[(k + 1 + rr) % 6][kc] * inv;  // column k is not written in this loop
            win[(k + 1 + rr) % 6][(k + cc) & 15] -= lr * win[sk][(k + cc) & 15];
        }
        __syncwarp();
        if (lane < nr) {
            rw[(k + 1 + lane) % 6] -= l * rw[sk];
            win[(k + 1 + lane) % 6][kc] = 0.0;  // eliminated
        }
        // the finished row k (columns k..cmax) and its right-hand side go back for the substitution
        if (lane <= ncol) band[k * VW + VKL + lane] = win[sk][(k + lane) & 15];
        if (lane == 16) rhs[k] = rw[sk];
        __syncwarp();
        put(k + 6, nval, nrv);  // slot of row k is free now
        __syncwarp();
    }
    // back substitution; the next row of U and its right-hand side are loaded during each step
    auto loadu = [&](int64_t r, double &bv, double &rv) {
        bv = 0.0;
        rv = 0.0;
        if (r >= 0) {
            if (lane <= VKL + VKU) bv = band[r * VW + VKL + lane];
            if (lane == 16) rv = rhs[r];
        }
    };
    double bv, rv;
    loadu(n - 1, bv, rv);
    for (int64_t k = n - 1; k >= 0; --k) {
        double nbv, nrv;
        loadu(k - 1, nbv, nrv);
        const int64_t cmax = k + VKL + VKU < n ? k + VKL + VKU : n - 1;
        const int ncol = (int)(cmax - k);
        double s = 0.0;
        if (lane >= 1 && lane <= ncol) s = bv * xs[(k + lane) & 15];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(F, s, o);
        const double rk = __shfl_sync(F, rv, 16);
        if (lane == 0) {
            const double x = (rk - s) / bv;  // lane 0 holds the diagonal
            xs[k & 15] = x;
            rhs[k] = x;
        }
        __syncwarp();
        bv = nbv;
        rv = nrv;
    }
}

__global__ void __launch_bounds__(128) k_vam_correct(VamArgs a)
{
    if (*(volatile unsigned int *)&a.ctl->status) return;
    const double dt = *(volatile double *)&a.ctl->dt_last;
    unsigned flag = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.nc; i += (int64_t)gridDim.x * blockDim.x) {
        double q[5];
        vcorrected(a, Probe{-1, 0, a.rhs}, i, dt, q);
        for (int v = 0; v < 5; ++v) {
            if (!(fabs(q[v]) <= 1e300)) flag |= DEV_NAN;
            a.Q[v * a.ld + i] = q[v];
        }
        if (q[0] <= 0.0) flag |= DEV_NEGDEPTH;
    }
    if (flag) atomicOr(&a.ctl->status, flag);
}

zoomy_status vam_run_steps(zoomy_ctx *c, double *Q, int64_t ld, double dt, int nsteps)
{
    VamArgs a;
    a.Q = Q;
    a.Qs = (double *)c->q1;
    a.band = c->vam_band;
    a.rhs = c->vam_rhs;
    a.ld = ld;
    a.nc = c->nc;
    a.dx = c->dx;
    a.g = c->g;
    a.cfl = c->cfl;
    a.bcl = c->bc[0];
    a.bcr = c->bc[1];
    a.ctl = c->ctl;
    a.dt_fixed = dt;
    int64_t blocks = (c->nc + 127) / 128;
    if (blocks > (int64_t)c->nsm * 4) blocks = (int64_t)c->nsm * 4;
    const unsigned grid = (unsigned)blocks;
    for (int k = 0; k < nsteps; ++k) {
        a.slot_in = k & 1;
        a.slot_out = k & 1;  // the wave-speed reduction of step k fills the slot its predictor reads
        k_vam_wavespeed<<<grid, 128, 0, c->stream>>>(a);
        a.slot_out = (k + 1) & 1;  // the predictor clears the next step's slot
        k_vam_predict<<<grid, 128, 0, c->stream>>>(a);
        k_vam_assemble<<<grid, 128, 0, c->stream>>>(a);
        k_vam_solve<<<1, 32, 0, c->stream>>>(a);
        k_vam_correct<<<grid, 128, 0, c->stream>>>(a);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "VAM step launch");
    }
    return ZOOMY_OK;
}

}  // namespace zoomy

using namespace zoomy;

extern "C" zoomy_status zoomy_vam_set(zoomy_ctx *c, int32_t enable)
{
    if (!c) return set_error(ZOOMY_EINVAL, "zoomy_vam_set: NULL context");
    if (enable != 0 && enable != 1) return set_error(ZOOMY_EINVAL, "zoomy_vam_set: enable is 0 or 1");
    if (enable) {
        if (c->kind != ZOOMY_MESH_1D || !c->model_ok || c->dtype != ZOOMY_FP64)
            return set_error(ZOOMY_EINVAL, "zoomy_vam_set: needs a 1D FP64 context after zoomy_model_set");
        if (c->closure_on || c->order != 1 || c->src_implicit)
            return set_error(ZOOMY_EINVAL, "zoomy_vam_set: not with the closure, order 2 or implicit friction");
        if (!c->vam_band) {
            cudaError_t e = cudaMalloc(&c->vam_band, sizeof(double) * (size_t)(2 * c->nc) * VW);
            if (e == cudaSuccess) e = cudaMalloc(&c->vam_rhs, sizeof(double) * (size_t)(2 * c->nc));
            if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
        }
        c->vam = 1;
        c->nv = 5;
    } else {
        c->vam = 0;
        c->nv = c->level + 2;
    }
    return ZOOMY_OK;
}
