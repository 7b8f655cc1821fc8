// vam.cu -- the non-hydrostatic VAM predictor-corrector in 1D (Sec. "Unsteady Vertically Averaged
// Momentum Equations in 1D"; the splitting of Eq. (PDE-hyperbolic) - Eq. (PDE-source)), FP64, over a
// bed b(x) with b_x the central difference per cell (bed ghosts copy the boundary cell).
//
//   Q = (h, h u0, h u1, h w0, h w1), w2 = -(w0 + w1) + (u0 + u1) b_x
//   predictor: hydrostatic reconstruction per face (b_f = max(b_L, b_R), h* = max(0, h + b - b_f),
//     velocities kept), Phi = (F(L*) + F(R*))/2 - s_f (R* - L*)/2 with
//     F = (h u0, h u0^2 + h u1^2/3 + g h^2/2, 2 h u0 u1, h u0 w0 + h u1 w1/3, h u0 w1 + u1 (h w0 + 2/5 h w2)),
//     the path integral Btilde (R* - L*) of B (row h u1: -u0 on h u1; row h w1: (w2/5 - w0) on h u1) by
//     3-point Gauss-Legendre on the straight segment, and
//     Q*_i = Q_i - dt/dx [(Phi - P(h*_i) e1 + Btilde dQ/2)_{i+1/2} - (Phi - P(h*_i) e1 - Btilde dQ/2)_{i-1/2}],
//     P(h) = g h^2/2, s = |u0| + sqrt(g h* + u1^2) + |u1|; in a flux the cell's own b_x, along a path
//     the mean of both cells' (a wall ghost's slope changes sign);
//   corrector: the pressure (p0, p1) per cell such that Q** = Q* - dt S(p),
//     S = (0, d(h p0)/dx + 2 p1 b_x, d(h p1)/dx - (3 p0 - p1) dh/dx - 6 (p0 - p1) b_x, -2 p1, 6 (p0 - p1)),
//     satisfies R0 = h du0/dx + d(h u1)/dx/3 + u1 dh/dx/3 + 2 (w0 - u0 b_x) = 0 and
//     R1 = h du0/dx + u1 dh/dx + 2 (u1 b_x - w1) = 0 with central differences and mirrored ghosts
//     (u0, u1 and their momenta change sign at walls).
//
// The constraints are linear in p with a stencil of two cells on each side.  Grouping two cells per
// block (unknowns (p0, p1) of cells 2I and 2I+1) makes the system block tridiagonal with 4 x 4 blocks
//   A_I x_{I-1} + D_I x_I + C_I x_{I+1} = f_I,  I = 0 .. N-1,  N = ceil(nc / 2)
// (an odd line gets one dummy cell with p = 0).  The entries come without any symbolic derivation:
// probing with the 10 vectors that are 1 on one component of every fifth cell (cells five apart never
// share a row) gives every entry as R(probe) - R(0), one thread per cell and probe.  The system is
// solved by parallel cyclic reduction: with Y_J = D_J^{-1} (A_J | C_J | f_J), level s replaces
//   D_I <- D_I - A_I YC_{I-s} - C_I YA_{I+s},  A_I <- -A_I YA_{I-s},  C_I <- -C_I YC_{I+s},
//   f_I <- f_I - A_I Yf_{I-s} - C_I Yf_{I+s}
// (row I then couples to I -+ 2s); after ceil(log2 N) levels no coupling is left and x_I = Yf_I.
// Every level is one launch with a half-warp per block row (lane = entry (r, c)): the update, then
// Gauss-Jordan elimination with partial pivoting inside the 4 x 4 block for the new Y_I.  No pivoting
// across blocks: the constraint operator is close to symmetric positive definite once each cell's two
// rows are combined (3 R0 + R1, R0), so elimination in any order is stable, and the probed 4 x 4 blocks
// keep their own pivoting.
#include <cmath>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/zoomy.h"
#include "fv_common.cuh"
#include "zoomy_internal.h"

namespace zoomy {

constexpr int RS = 64;  // block row: A [16] at 0, C [16] at 16, D [16] at 32, f [4] at 48 (entry r * 4 + c)
constexpr int YS = 48;  // Y_J: YA [16] at 0, YC [16] at 16, Yf [4] at 32
constexpr int PCR_ROWS = 8;  // block rows per 128-thread CTA of the reduction

struct VamArgs {
    double *Q;        // state [5][ld] (in: Q^n, out: Q^{n+1})
    const double *bed;  // b per cell [nc]
    double *Qs;       // predictor result Q* [5][ld]
    double *rows;     // [N][RS] block rows of the pressure system (updated in place by the reduction)
    double *Y[2];     // [N][YS] ping-pong Y of the reduction levels
    double *rhs;      // [4 N]: the solution p, unknown 2 j + comp for cell j
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
    return Q[v * a.ld + bounds_idx(j, a.nc, &a.ctl->status)];
}

// b_x of cell j (0 <= j < nc): central difference with copied bed ghosts
__device__ __forceinline__ double vbx_cell(const VamArgs &a, int64_t j)
{
    const int64_t jl = j > 0 ? j - 1 : 0, jr = j + 1 < a.nc ? j + 1 : a.nc - 1;
    return (a.bed[jr] - a.bed[jl]) * (0.5 / a.dx);
}

// b and b_x of cell or ghost j (-1 <= j <= nc); a wall ghost's slope changes sign
__device__ __forceinline__ void vbed(const VamArgs &a, int64_t j, double &b, double &bx)
{
    if (j < 0) {
        b = a.bed[0];
        bx = a.bcl == 1 ? -vbx_cell(a, 0) : vbx_cell(a, 0);
    } else if (j >= a.nc) {
        b = a.bed[a.nc - 1];
        bx = a.bcr == 1 ? -vbx_cell(a, a.nc - 1) : vbx_cell(a, a.nc - 1);
    } else {
        b = a.bed[j];
        bx = vbx_cell(a, j);
    }
}

__device__ __forceinline__ double vspeed(const double *q, double rh, double g)
{
    const double u0 = q[1] * rh, u1 = q[2] * rh;
    return fabs(u0) + sqrt(g * q[0] + u1 * u1) + fabs(u1);
}

// F(q); rh = 1 / h, or 0 for a dry reconstructed state (the velocities as products)
__device__ __forceinline__ void vflux(const double *q, double rh, double bx, double g, double *F)
{
    const double h = q[0], u0 = q[1] * rh, u1 = q[2] * rh, w0 = q[3] * rh, w1 = q[4] * rh;
    const double w2 = -(w0 + w1) + (u0 + u1) * bx;
    F[0] = h * u0;
    F[1] = h * u0 * u0 + h * u1 * u1 * (1.0 / 3.0) + 0.5 * g * h * h;
    F[2] = 2.0 * h * u0 * u1;
    F[3] = h * u0 * w0 + h * u1 * w1 * (1.0 / 3.0);
    F[4] = h * u0 * w1 + u1 * (h * w0 + 0.4 * h * w2);
}

__device__ __forceinline__ double vrh(double h) { return h > 0.0 ? 1.0 / h : 0.0; }

// Face between the states qL, qR over beds (bL, bxL), (bR, bxR): gm to the left cell (its right
// face), gp to the right cell (its left face).
__device__ __forceinline__ void vface(const double *qL, const double *qR, double bL, double bxL, double bR,
                                      double bxR, double g, double *gm, double *gp)
{
    const double bf = fmax(bL, bR);
    const double hLs = fmax(0.0, qL[0] + bL - bf), hRs = fmax(0.0, qR[0] + bR - bf);
    // f = h* / h and 1/h* of each side from one division: 1/(h h*) (both zero where h* = 0)
    const bool wL = qL[0] > 0.0 && hLs > 0.0, wR = qR[0] > 0.0 && hRs > 0.0;
    const double rL = wL ? 1.0 / (qL[0] * hLs) : 0.0, rR = wR ? 1.0 / (qR[0] * hRs) : 0.0;
    const double fL = hLs * hLs * rL, fR = hRs * hRs * rR;
    double Ls[5], Rs[5], FL[5], FR[5], dq[5], bt[5] = {0, 0, 0, 0, 0};
    Ls[0] = hLs;
    Rs[0] = hRs;
    for (int v = 1; v < 5; ++v) {
        Ls[v] = qL[v] * fL;
        Rs[v] = qR[v] * fR;
    }
    const double rhL = qL[0] * rL, rhR = qR[0] * rR;
    vflux(Ls, rhL, bxL, g, FL);
    vflux(Rs, rhR, bxR, g, FR);
    for (int v = 0; v < 5; ++v) dq[v] = Rs[v] - Ls[v];
    const double bxf = 0.5 * (bxL + bxR);
    const double sq[3] = {0.5 - 0.38729833462074168852, 0.5, 0.5 + 0.38729833462074168852};
    const double wq[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
    // 1/h at the three nodes from one division of the product of the wet depths (dry: 1, weight 0);
    // FP64 divisions are long dependent chains on GB300, and constant divisors become products
    double hq[3];
    for (int k = 0; k < 3; ++k) {
        hq[k] = Ls[0] + sq[k] * dq[0];
        if (!(hq[k] > 0.0)) hq[k] = 1.0;
    }
    const double rp = 1.0 / (hq[0] * hq[1] * hq[2]);
    for (int k = 0; k < 3; ++k) {
        double p[5];
        for (int v = 0; v < 5; ++v) p[v] = Ls[v] + sq[k] * dq[v];
        const double rh = p[0] > 0.0 ? rp * hq[(k + 1) % 3] * hq[(k + 2) % 3] : 0.0;
        const double u0 = p[1] * rh, u1 = p[2] * rh, w0 = p[3] * rh, w1 = p[4] * rh;
        const double w2 = -(w0 + w1) + (u0 + u1) * bxf;
        bt[2] += wq[k] * (-u0) * dq[2];
        bt[4] += wq[k] * (w2 * 0.2 - w0) * dq[2];
    }
    const double sL = vspeed(Ls, rhL, g), sR = vspeed(Rs, rhR, g), sf = sL > sR ? sL : sR;
    for (int v = 0; v < 5; ++v) {
        const double phi = 0.5 * (FL[v] + FR[v]) - 0.5 * sf * dq[v];
        gm[v] = phi + 0.5 * bt[v];
        gp[v] = phi - 0.5 * bt[v];
    }
    gm[1] -= 0.5 * g * hLs * hLs;
    gp[1] -= 0.5 * g * hRs * hRs;
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
    pdl_enter();
    double s = 0.0;
    unsigned flag = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.nc; i += (int64_t)gridDim.x * blockDim.x) {
        double q[5];
        for (int v = 0; v < 5; ++v) q[v] = a.Q[v * a.ld + i];
        const double si = vspeed(q, 1.0 / q[0], a.g);
        if (!(q[0] > 0.0)) flag |= q[0] < 0.0 ? DEV_NEGDEPTH : DEV_NAN;
        s = (si > s || si != si) ? si : s;
    }
    if (flag) atomicOr(&a.ctl->status, flag);
    reduce_smax<double>(a.ctl, a.slot_out, s);
}

__global__ void __launch_bounds__(128) k_vam_predict(VamArgs a)
{
    pdl_enter();
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
    // a warp per 31 cells: lane j evaluates the face between cells i-1 and i (i = 31 w + j) once;
    // cell i (j < 31) takes that face's gp and, from lane j+1, the gm of its right face
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * blockDim.x / 32;
    for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; w * 31 < a.nc; w += nw) {
        const int64_t i = 31 * w + lane;
        double ql[5], qr[5], gm[5], gp[5];
        if (i <= a.nc) {
            double bL, bxL, bR, bxR;
            for (int v = 0; v < 5; ++v) {
                ql[v] = vq(a, a.Q, v, i - 1);
                qr[v] = vq(a, a.Q, v, i);
            }
            vbed(a, i - 1, bL, bxL);
            vbed(a, i, bR, bxR);
            vface(ql, qr, bL, bxL, bR, bxR, a.g, gm, gp);
        } else {
            for (int v = 0; v < 5; ++v) qr[v] = gm[v] = gp[v] = 0.0;
        }
        for (int v = 0; v < 5; ++v) {
            const double gmr = __shfl_down_sync(0xffffffffu, gm[v], 1);  // the right face of cell i
            if (lane < 31 && i < a.nc) a.Qs[v * a.ld + i] = qr[v] - dt / a.dx * (gmr - gp[v]);
        }
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
    const double bx = vbx_cell(a, j);
    q[0] = h;
    q[1] = a.Qs[a.ld + j] - dt * (dhp0 + 2.0 * p1 * bx);
    q[2] = a.Qs[2 * a.ld + j] - dt * (dhp1 - (3.0 * p0 - p1) * dh - 6.0 * (p0 - p1) * bx);
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
    const double h = qc[0], rh = 1.0 / h, u0 = qc[1] * rh, u1 = qc[2] * rh, w0 = qc[3] * rh, w1 = qc[4] * rh;
    const double bx = vbx_cell(a, i);
    const double dh = (qr[0] - ql[0]) * i2dx;
    const double du0 = (qr[1] * ql[0] - ql[1] * qr[0]) / (qr[0] * ql[0]) * i2dx;
    const double dhu1 = (qr[2] - ql[2]) * i2dx;
    R[0] = h * du0 + (dhu1 + u1 * dh) * (1.0 / 3.0) + 2.0 * (w0 - u0 * bx);
    R[1] = h * du0 + u1 * dh + 2.0 * (u1 * bx - w1);
}

// Block rows by probing: thread (i, q) of cell i evaluates R(0) (q = 0, which also writes f = -R(0)
// and the zero entries outside the stencil) or R(probe q) - R(0) for the q-th (color, component).
__global__ void __launch_bounds__(128) k_vam_assemble(VamArgs a)
{
    pdl_enter();
    if (*(volatile unsigned int *)&a.ctl->status) return;
    const double dt = *(volatile double *)&a.ctl->dt_last;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < 11 * a.nc; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / 11, I = i >> 1;
        const int q = (int)(t - 11 * i);
        double *blk = a.rows + I * RS;
        const int r0w = 2 * (int)(i & 1);  // this cell's two rows within the block
        double r0[2];
        vresidual(a, Probe{-1, 0, nullptr}, i, dt, r0);
        // column within the 12 of the block row (A | D | C) for unknown (cell j, comp)
        auto put = [&](int64_t j, int comp, int r, double v) {
            const int col = 2 * (int)(j - 2 * (I - 1)) + comp;
            blk[16 * (col < 4 ? 0 : col < 8 ? 2 : 1) + 4 * (r0w + r) + (col & 3)] = v;
        };
        if (q == 0) {
            for (int r = 0; r < 2; ++r) blk[48 + r0w + r] = -r0[r];
            const int64_t jout = (i & 1) ? 2 * I - 2 : 2 * I + 3;  // the one cell of the block row outside the stencil
            for (int r = 0; r < 2; ++r)
                for (int comp = 0; comp < 2; ++comp) put(jout, comp, r, 0.0);
            if (i == a.nc - 1 && !(i & 1)) {
                // odd line: the dummy cell 2I+1 has rows p = 0
                for (int e = 0; e < 8; ++e) {
                    blk[8 + e] = 0.0;
                    blk[16 + 8 + e] = 0.0;
                    blk[32 + 8 + e] = 0.0;
                }
                blk[32 + 10] = 1.0;
                blk[32 + 15] = 1.0;
                blk[48 + 2] = 0.0;
                blk[48 + 3] = 0.0;
            }
            continue;
        }
        const int color = (q - 1) >> 1, comp = (q - 1) & 1;
        // the one cell of this color within the stencil i-2..i+2 of row i
        const int64_t j = i - 2 + (((color - (int)((i - 2 + 10 * 5) % 5)) % 5 + 5) % 5);
        if (j < 0 || j >= a.nc) {
            for (int r = 0; r < 2; ++r) put(j, comp, r, 0.0);
            continue;
        }
        double rp[2];
        vresidual(a, Probe{color, comp, nullptr}, i, dt, rp);
        for (int r = 0; r < 2; ++r) put(j, comp, r, rp[r] - r0[r]);
    }
}

// One level of the block cyclic reduction over the block rows I = j * step (s = 0: only
// Y_I = D_I^{-1} (A_I | C_I | f_I)); `last` writes the solution of those rows.  step = 1 and s = 1, 2, 4, ...:
// parallel cyclic reduction of all rows; step = 2s: a cyclic-reduction level (the rows at odd multiples
// of s are eliminated from the system of the rows at multiples of 2s; their Y are kept for the
// back-substitution; Yin may be Yout since the rows read and the rows written are disjoint).  A
// half-warp per block row; lane l holds entry (r, c) = (l / 4, l % 4).
__global__ void __launch_bounds__(128) k_vam_pcr(VamArgs a, int64_t N, int64_t s, int64_t step, const double *Yin,
                                                 double *Yout, int last)
{
    pdl_enter();
    if (*(volatile unsigned int *)&a.ctl->status) return;
    __shared__ double S[PCR_ROWS][4][16];
    const int hw = threadIdx.x >> 4, l = threadIdx.x & 15, r = l >> 2, c = l & 3;
    const int64_t I = ((int64_t)blockIdx.x * PCR_ROWS + hw) * step;
    if (I >= N) return;  // the whole half-warp
    const unsigned mask = 0xffffu << (threadIdx.x & 16);
    double *row = a.rows + I * RS;
    double D, A, C, F;
    if (s > 0) {
        double arow[4], crow[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            arow[k] = row[4 * r + k];
            crow[k] = row[16 + 4 * r + k];
        }
        D = row[32 + l];
        F = row[48 + r];
        A = 0.0;
        C = 0.0;
        if (I - s >= 0) {
            const double *Ym = Yin + bounds_idx(I - s, N, &a.ctl->status) * YS;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                D -= arow[k] * Ym[16 + 4 * k + c];
                A -= arow[k] * Ym[4 * k + c];
                F -= arow[k] * Ym[32 + k];
            }
        }
        if (I + s < N) {
            const double *Yp = Yin + bounds_idx(I + s, N, &a.ctl->status) * YS;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                D -= crow[k] * Yp[4 * k + c];
                C -= crow[k] * Yp[16 + 4 * k + c];
                F -= crow[k] * Yp[32 + k];
            }
        }
        __syncwarp(mask);  // every lane has read the old row
        row[l] = A;
        row[16 + l] = C;
        row[32 + l] = D;
        if (c == 0) row[48 + r] = F;
    } else {
        A = row[l];
        C = row[16 + l];
        D = row[32 + l];
        F = row[48 + r];
    }
    // Gauss-Jordan elimination with partial pivoting on [D | A | C | f], fraction-free: every row but
    // the pivot row becomes pk * row - m * pivot row, and each row is divided by its diagonal at the
    // end (one division per lane instead of one per step); magnitudes compare as bit patterns
    double(*M)[16] = S[hw];
    bool singular = false;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        M[r][c] = D;
        M[r][4 + c] = A;
        M[r][8 + c] = C;
        if (c == 0) M[r][12] = F;
        __syncwarp(mask);
        constexpr unsigned long long MAG = 0x7fffffffffffffffull;
        int piv = k;
        unsigned long long best = (unsigned long long)__double_as_longlong(M[k][k]) & MAG;
#pragma unroll
        for (int q = k + 1; q < 4; ++q) {
            const unsigned long long v = (unsigned long long)__double_as_longlong(M[q][k]) & MAG;
            if (v > best) {
                best = v;
                piv = q;
            }
        }
        singular |= best == 0ull || best >= 0x7ff0000000000000ull;  // zero, infinite or NaN pivot
        const int rs = r == k ? piv : (r == piv ? k : r);  // the row that lands in row r after the swap
        const double pk = M[piv][k];
        const double P0 = M[piv][c], P1 = M[piv][4 + c], P2 = M[piv][8 + c], Pf = M[piv][12];
        if (r == k) {
            D = P0;
            A = P1;
            C = P2;
            F = Pf;
        } else {
            const double m = M[rs][k];
            D = pk * M[rs][c] - m * P0;
            A = pk * M[rs][4 + c] - m * P1;
            C = pk * M[rs][8 + c] - m * P2;
            F = pk * M[rs][12] - m * Pf;
        }
        __syncwarp(mask);
    }
    if (singular && l == 0) atomicOr(&a.ctl->status, DEV_NAN);  // singular pressure block
    const double ip = 1.0 / __shfl_sync(mask, D, 5 * r, 16);  // row r's diagonal, lane (r, r)
    A *= ip;
    C *= ip;
    F *= ip;
    double *y = Yout + I * YS;
    y[l] = A;
    y[16 + l] = C;
    if (c == 0) {
        y[32 + r] = F;
        if (last) a.rhs[4 * I + r] = F;  // (a dummy cell's unknowns are 0 and never read)
    }
}

// Back-substitution of a cyclic-reduction level: the rows I = s + 2 s j, eliminated at that level, from
// x_I = Yf_I - YA_I x_{I-s} - YC_I x_{I+s} with their Y of that level (x_{I+s} = 0 past the last row);
// x lives in rhs, 4 unknowns per block row.  A thread per (row, component).
__global__ void __launch_bounds__(128) k_vam_backsub(VamArgs a, int64_t N, int64_t s, const double *Y)
{
    pdl_enter();
    if (*(volatile unsigned int *)&a.ctl->status) return;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t I = s + 2 * s * (t >> 2);
    const int r = (int)(t & 3);
    if (I >= N) return;
    const double *y = Y + I * YS;
    const double *xm = a.rhs + 4 * (I - s);
    double x = y[32 + r];
#pragma unroll
    for (int c = 0; c < 4; ++c) x -= y[4 * r + c] * xm[c];
    if (I + s < N) {
        const double *xp = a.rhs + 4 * (I + s);
#pragma unroll
        for (int c = 0; c < 4; ++c) x -= y[16 + 4 * r + c] * xp[c];
    }
    a.rhs[4 * I + r] = x;
}

__global__ void __launch_bounds__(128) k_vam_correct(VamArgs a)
{
    pdl_enter();
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
    const int64_t N = (c->nc + 1) / 2;
    a.Q = Q;
    a.bed = (const double *)c->bed_dev;
    a.Qs = (double *)c->q1;
    a.rows = c->vam_sys;
    a.Y[0] = c->vam_sys + N * RS;
    a.Y[1] = a.Y[0] + N * YS;
    a.rhs = c->vam_p;
    a.ld = ld;
    a.nc = c->nc;
    a.dx = c->dx;
    a.g = c->g;
    a.cfl = c->cfl;
    a.bcl = c->bc[0];
    a.bcr = c->bc[1];
    a.ctl = c->ctl;
    a.dt_fixed = dt;
    // FP64 work per cell: one-warp CTAs spread short lines over more SMs
    const int threads = c->nc < 65536 ? 32 : 128;
    auto grid_for = [&](int64_t work) {
        int64_t b = (work + threads - 1) / threads;
        const int64_t cap = (int64_t)c->nsm * (threads == 32 ? 16 : 4);
        return (unsigned)(b < cap ? b : cap);
    };
    const unsigned grid = grid_for(c->nc), grid_asm = grid_for(11 * c->nc);
    const unsigned grid_pred = grid_for((c->nc + 30) / 31 * 32);  // a warp per 31 cells
    const unsigned grid_pcr = (unsigned)((N + PCR_ROWS - 1) / PCR_ROWS);
    // cyclic-reduction levels before the parallel reduction (each halves the rows left): two measured
    // fastest at 2000 cells (97.9 us per step against 102.8 with none, 100.3 / 102.4 / 104.3 with 3 / 4 / 6;
    // the levels are latency-bound, so the work saved per level gains little against the added launches)
    const int cr = 2;
    const cudaStream_t st = c->stream;
    for (int k = 0; k < nsteps; ++k) {
        a.slot_in = k & 1;
        a.slot_out = k & 1;  // the wave-speed reduction of step k fills the slot its predictor reads
        cudaError_t e = launch_pdl(k_vam_wavespeed, grid, threads, st, a);
        a.slot_out = (k + 1) & 1;  // the predictor clears the next step's slot
        if (e == cudaSuccess) e = launch_pdl(k_vam_predict, grid_pred, threads, st, a);
        if (e == cudaSuccess) e = launch_pdl(k_vam_assemble, grid_asm, threads, st, a);
        const unsigned bp = 16 * PCR_ROWS;
        auto grid_rows = [&](int64_t step) {
            const int64_t rows = (N + step - 1) / step;
            return (unsigned)((rows + PCR_ROWS - 1) / PCR_ROWS);
        };
        if (e == cudaSuccess)
            e = launch_pdl(k_vam_pcr, grid_pcr, bp, st, a, N, (int64_t)0, (int64_t)1, (const double *)a.Y[1], a.Y[0],
                           (int)(N == 1));
        // cyclic-reduction levels: the system of the rows at multiples of st, st = 2, 4, ..., 2^cr
        int64_t sr = 1;
        for (int q = 0; q < cr && 2 * sr < N && e == cudaSuccess; ++q, sr *= 2)
            e = launch_pdl(k_vam_pcr, grid_rows(2 * sr), bp, st, a, N, sr, 2 * sr, (const double *)a.Y[0], a.Y[0], 0);
        // parallel cyclic reduction of that system
        int cur = 0;
        for (int64_t s = sr; s < N && e == cudaSuccess; s *= 2) {
            e = launch_pdl(k_vam_pcr, grid_rows(sr), bp, st, a, N, s, sr, (const double *)a.Y[cur], a.Y[cur ^ 1],
                           (int)(2 * s >= N));
            cur ^= 1;
        }
        // back-substitution of the eliminated rows (their Y are in Y[0])
        for (int64_t s = sr / 2; s >= 1 && e == cudaSuccess; s /= 2) {
            const int64_t rows = (N - s + 2 * s - 1) / (2 * s);
            e = launch_pdl(k_vam_backsub, (unsigned)((4 * rows + 127) / 128), 128u, st, a, N, s, (const double *)a.Y[0]);
        }
        if (e == cudaSuccess) e = launch_pdl(k_vam_correct, grid, threads, st, a);
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
        if (!c->vam_sys) {
            const size_t N = (size_t)(c->nc + 1) / 2;
            cudaError_t e = cudaMalloc(&c->vam_sys, sizeof(double) * N * (RS + 2 * YS));
            if (e == cudaSuccess) e = cudaMalloc(&c->vam_p, sizeof(double) * 4 * N);
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
