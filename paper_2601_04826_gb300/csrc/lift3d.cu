// lift3d.cu -- lifting of the depth-averaged moment state to three-dimensional fields at sigma
// levels (the paper's interpolate_3d postprocessing, Sec. "Postprocessing").
//
// At level zeta_j in [0, 1] of a cell (elevation z = b + zeta h):
//   u = sum_k alpha_k phi_k(zeta),  v = sum_k beta_k phi_k(zeta)
//   w = -sum_k [d_x(h alpha_k) + d_y(h beta_k)] Phi_k(zeta) + u (d_x b + zeta d_x h) + v (d_y b + zeta d_y h)
//   p = g h (1 - zeta)
// (continuity integrated upwards from the bed, where w = u.grad b; horizontal derivatives at fixed z;
// hydrostatic pressure with rho = 1).  Level 0 on a flat bed gives w(1) = -h (d_x u + d_y v), the
// paper's SWE lifting.  Horizontal derivatives are Green-Gauss over the cell's faces with face value
// (q_i + q_j)/2 and q_j = q_i on boundary faces (central differences on uniform grids).  Dry cells get
// u = v = w = 0.
//
// One thread per cell (grid-stride), the basis values phi_k(zeta_j), Phi_k(zeta_j) in a small table
// evaluated on the host in double precision; the 4 K output planes are written coalesced.
#include <cmath>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/zoomy.h"
#include "fv_common.cuh"
#include "zoomy_internal.h"

namespace zoomy {

constexpr int LIFT_MAXK = 64;

template <typename T>
struct LiftArgs {
    const T *Q, *bed;
    T *out;
    int64_t ld, ldo, nc, nx, ny;
    T inv_dx, inv_dy, g, hdry;
    const T *tab;  // [K][2][m]: phi_k(zeta_j), Phi_k(zeta_j)
    const T *zeta;
    const int32_t *nbr;  // triangles: [3][nc]
    const float *geo;    // triangles: nx[3][nc], ny[3][nc], |e|/|Omega| [3][nc]
    int K;
    unsigned *status;    // bounds-checking build: the context's status word
};

// MESH 0: 1D uniform, 1: 2D structured, 2: triangles
template <int N, int MESH, typename T>
__global__ void __launch_bounds__(128) k_lift3d(LiftArgs<T> a)
{
    constexpr int m = N + 1, nv = (MESH == 0) ? 1 + m : 1 + 2 * m;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.nc; i += (int64_t)gridDim.x * blockDim.x) {
        T q[nv + 1];
#pragma unroll
        for (int v = 0; v < nv; ++v) q[v] = a.Q[v * a.ld + i];
        q[nv] = a.bed[i];
        T gx[nv + 1], gy[nv + 1];
#pragma unroll
        for (int v = 0; v <= nv; ++v) gx[v] = gy[v] = T(0);
        auto val = [&](int64_t j, int v) {
            j = bounds_idx(j, a.nc, a.status);
            return v < nv ? a.Q[v * a.ld + j] : a.bed[j];
        };
        if (MESH == 0 || MESH == 1) {
            const int64_t ix = MESH == 0 ? i : i % a.nx;
            const int64_t iw = ix > 0 ? i - 1 : i, ie = ix + 1 < a.nx ? i + 1 : i;
#pragma unroll
            for (int v = 0; v <= nv; ++v) gx[v] = T(0.5) * (val(ie, v) - val(iw, v)) * a.inv_dx;
            if (MESH == 1) {
                const int64_t iy = i / a.nx;
                const int64_t is = iy > 0 ? i - a.nx : i, in = iy + 1 < a.ny ? i + a.nx : i;
#pragma unroll
                for (int v = 0; v <= nv; ++v) gy[v] = T(0.5) * (val(in, v) - val(is, v)) * a.inv_dy;
            }
        } else {
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                const int32_t j = a.nbr[f * a.nc + i];
                const T wx = T(a.geo[(6 + f) * a.nc + i]) * T(a.geo[f * a.nc + i]);
                const T wy = T(a.geo[(6 + f) * a.nc + i]) * T(a.geo[(3 + f) * a.nc + i]);
#pragma unroll
                for (int v = 0; v <= nv; ++v) {
                    const T fv = T(0.5) * (q[v] + (j >= 0 ? val(j, v) : q[v]));
                    gx[v] += wx * fv;
                    gy[v] += wy * fv;
                }
            }
        }
        const T h = q[0];
        const bool wet = h > a.hdry;
        const T ih = wet ? T(1) / h : T(0);
        T al[m], be[m], gk[m];
#pragma unroll
        for (int k = 0; k < m; ++k) {
            al[k] = q[var_a<N, (MESH == 0 ? 1 : 2)>(k)] * ih;
            be[k] = MESH == 0 ? T(0) : q[var_b<N>(k)] * ih;
            gk[k] = gx[var_a<N, (MESH == 0 ? 1 : 2)>(k)] + (MESH == 0 ? T(0) : gy[var_b<N>(k)]);
        }
        for (int jz = 0; jz < a.K; ++jz) {
            const T *ph = a.tab + jz * 2 * m, *Ph = ph + m;
            const T zt = a.zeta[jz];
            T u = T(0), v = T(0), G = T(0);
#pragma unroll
            for (int k = 0; k < m; ++k) {
                u += al[k] * ph[k];
                v += be[k] * ph[k];
                G += gk[k] * Ph[k];
            }
            T w = -G + u * (gx[nv] + zt * gx[0]) + v * (gy[nv] + zt * gy[0]);
            if (!wet) u = v = w = T(0);
            T *o = a.out + (int64_t)jz * a.ldo + i;
            o[0] = u;
            o[(int64_t)a.K * a.ldo] = v;
            o[(int64_t)2 * a.K * a.ldo] = w;
            o[(int64_t)3 * a.K * a.ldo] = a.g * h * (T(1) - zt);
        }
    }
}

template <int MESH, typename T>
static cudaError_t launch_lift_mesh(int level, const LiftArgs<T> &a, int nsm, cudaStream_t st)
{
    int64_t blocks = (a.nc + 127) / 128;
    if (blocks > (int64_t)nsm * 16) blocks = (int64_t)nsm * 16;
    const dim3 grid((unsigned)(blocks > 0 ? blocks : 1)), block(128);
    switch (level) {
        case 0: k_lift3d<0, MESH, T><<<grid, block, 0, st>>>(a); break;
        case 1: k_lift3d<1, MESH, T><<<grid, block, 0, st>>>(a); break;
        case 2: k_lift3d<2, MESH, T><<<grid, block, 0, st>>>(a); break;
        case 3: k_lift3d<3, MESH, T><<<grid, block, 0, st>>>(a); break;
        case 4: k_lift3d<4, MESH, T><<<grid, block, 0, st>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// phi_k(z) = P_k(1 - 2z) by the Legendre recurrence; Phi_k(z) = int_0^z phi_k = z (k = 0) and
// -(P_{k+1}(x) - P_{k-1}(x)) / (2 (2k + 1)) at x = 1 - 2z (k >= 1), from int P_k = (P_{k+1} - P_{k-1})/(2k+1).
static void lift_basis(int N, double z, double *phi, double *Phi)
{
    double P[ZOOMY_MAX_LEVEL + 2];
    const double x = 1.0 - 2.0 * z;
    P[0] = 1.0;
    P[1] = x;
    for (int k = 1; k <= N; ++k) P[k + 1] = ((2.0 * k + 1.0) * x * P[k] - k * P[k - 1]) / (k + 1.0);
    for (int k = 0; k <= N; ++k) {
        phi[k] = P[k];
        Phi[k] = k == 0 ? z : -(P[k + 1] - P[k - 1]) / (2.0 * (2.0 * k + 1.0));
    }
}

template <typename T>
static zoomy_status lift_run(zoomy_ctx *c, const T *Q, int64_t ld, int K, const double *zeta, T *out, int64_t ldo)
{
    const int m = c->level + 1;
    std::vector<T> tab((size_t)K * 2 * m + K);
    for (int j = 0; j < K; ++j) {
        double phi[ZOOMY_MAX_LEVEL + 1], Phi[ZOOMY_MAX_LEVEL + 1];
        lift_basis(c->level, zeta[j], phi, Phi);
        for (int k = 0; k < m; ++k) {
            tab[(size_t)j * 2 * m + k] = T(phi[k]);
            tab[(size_t)j * 2 * m + m + k] = T(Phi[k]);
        }
        tab[(size_t)K * 2 * m + j] = T(zeta[j]);
    }
    // the table lives in the context's reduction scratch (2 * 64 * 5 + 64 values fit its 1024 doubles)
    const size_t bytes = sizeof(T) * tab.size();
    if (bytes > sizeof(double) * NPARTIAL) return set_error(ZOOMY_EINVAL, "zoomy_lift3d: table too large");
    // (a copy from pageable memory has read the host buffer when the call returns)
    cudaError_t e = cudaMemcpyAsync(c->partials, tab.data(), bytes, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "zoomy_lift3d table upload");
    LiftArgs<T> a;
    a.Q = Q;
    a.bed = (const T *)c->bed_dev;
    a.out = out;
    a.ld = ld;
    a.ldo = ldo;
    a.nc = c->nc;
    a.nx = c->nx;
    a.ny = c->ny;
    a.inv_dx = T(1.0 / c->dx);
    a.inv_dy = T(1.0 / c->dy);
    a.g = T(c->g);
    a.hdry = T(c->hdry);
    a.tab = (const T *)c->partials;
    a.zeta = (const T *)c->partials + (size_t)K * 2 * m;
    a.nbr = c->tri_nbr_d;
    a.geo = c->tri_geo_d;
    a.K = K;
    a.status = &c->ctl->status;
    if (c->kind == ZOOMY_MESH_1D)
        e = launch_lift_mesh<0, T>(c->level, a, c->nsm, c->stream);
    else if (c->kind == ZOOMY_MESH_2D)
        e = launch_lift_mesh<1, T>(c->level, a, c->nsm, c->stream);
    else
        e = launch_lift_mesh<2, T>(c->level, a, c->nsm, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "zoomy_lift3d launch");
#ifdef ZOOMY_BOUNDS_CHECK
    return read_status(c, nullptr);  // the bounds-checking build reports a bad index right away
#else
    return ZOOMY_OK;
#endif
}

}  // namespace zoomy

using namespace zoomy;

extern "C" zoomy_status zoomy_lift3d(zoomy_ctx *c, const void *Q, int64_t ld, int32_t K, const double *zeta, void *out,
                                     int64_t ldo)
{
    zoomy_status st = check_step_args(c, Q, ld, 0.0, 0, "zoomy_lift3d");
    if (st != ZOOMY_OK) return st;
    if (c->vam) return set_error(ZOOMY_EINVAL, "zoomy_lift3d: not defined for the VAM model");
    if (c->kind == ZOOMY_MESH_ENSEMBLE) return set_error(ZOOMY_EINVAL, "zoomy_lift3d: not for ensemble contexts");
    if (!out || !zeta) return set_error(ZOOMY_EINVAL, "zoomy_lift3d: NULL output or levels");
    if (K < 1 || K > LIFT_MAXK) return set_error(ZOOMY_EINVAL, "zoomy_lift3d: K in [1, %d]", LIFT_MAXK);
    if (ldo < c->nc) return set_error(ZOOMY_EINVAL, "zoomy_lift3d: ldo < ncells");
    for (int j = 0; j < K; ++j)
        if (!(zeta[j] >= 0.0 && zeta[j] <= 1.0)) return set_error(ZOOMY_EINVAL, "zoomy_lift3d: zeta outside [0, 1]");
    return c->dtype == ZOOMY_FP64 ? lift_run<double>(c, (const double *)Q, ld, K, zeta, (double *)out, ldo)
                                  : lift_run<float>(c, (const float *)Q, ld, K, zeta, (float *)out, ldo);
}
