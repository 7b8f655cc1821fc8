// fv_tri.cu -- triangle meshes: host mesh builder (orientation, neighbours, geometry, Morton
// order) and the cell-centric fused SSP-RK2 stage kernel.
//
// The paper's numerical layer runs the path-conservative FV scheme on unstructured meshes
// (Sec. 2.1.2, "hyperbolic_step" on 1D/2D/3D unstructured grids).  Here one thread owns one cell:
// it gathers its (up to) three neighbours through a neighbour table, evaluates each face in the
// frame of the face's outward normal (velocity moments rotated to normal / transverse components,
// the same face term as the structured kernels), rotates the result back and writes its own cell
// once.  Every face is evaluated from both sides: no atomics, deterministic results, and exact
// antisymmetry of the conservative fluxes.  Cells are renumbered along a Morton curve of their
// centroids so that neighbour gathers hit the same cache lines.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <vector>

#include <cuda_runtime.h>

#include "fv_common.cuh"
#include "zoomy_internal.h"
#include "zoomy_kernels.h"

namespace zoomy {

// ------------------------------------------------------------------------------------------
// Host: mesh construction
// ------------------------------------------------------------------------------------------

static uint32_t spread16(uint32_t v)
{
    v &= 0xffffu;
    v = (v | (v << 8)) & 0x00ff00ffu;
    v = (v | (v << 4)) & 0x0f0f0f0fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}

zoomy_status create_tri_mesh(const zoomy_mesh_desc *d, void *stream, zoomy_ctx **out)
{
    if (d->ntris < 1 || d->nverts < 3 || !d->verts_xy || !d->tris)
        return set_error(ZOOMY_EINVAL, "zoomy_mesh_create: triangle mesh needs verts_xy, tris, nverts >= 3");
    if (d->ntris > (1LL << 30)) return set_error(ZOOMY_EINVAL, "zoomy_mesh_create: too many triangles");
    if (d->bc[0] != ZOOMY_BC_TRANSMISSIVE && d->bc[0] != ZOOMY_BC_WALL)
        return set_error(ZOOMY_EINVAL, "zoomy_mesh_create: bc[0] must be 0 or 1");
    const int64_t nt = d->ntris, nvx = d->nverts;
    const double *xy = d->verts_xy;
    for (int64_t t = 0; t < 3 * nt; ++t)
        if (d->tris[t] < 0 || d->tris[t] >= nvx)
            return set_error(ZOOMY_EINVAL, "zoomy_mesh_create: triangle vertex index out of range");

    // orientation, area, centroid
    std::vector<int32_t> tv(3 * nt);
    std::vector<double> area(nt), cx(nt), cy(nt);
    for (int64_t t = 0; t < nt; ++t) {
        int32_t a = d->tris[3 * t], b = d->tris[3 * t + 1], c = d->tris[3 * t + 2];
        double A2 = (xy[2 * b] - xy[2 * a]) * (xy[2 * c + 1] - xy[2 * a + 1]) -
                    (xy[2 * c] - xy[2 * a]) * (xy[2 * b + 1] - xy[2 * a + 1]);
        if (A2 < 0) std::swap(b, c), A2 = -A2;
        if (!(A2 > 0)) return set_error(ZOOMY_EINVAL, "zoomy_mesh_create: degenerate triangle %lld", (long long)t);
        tv[3 * t] = a;
        tv[3 * t + 1] = b;
        tv[3 * t + 2] = c;
        area[t] = 0.5 * A2;
        cx[t] = (xy[2 * a] + xy[2 * b] + xy[2 * c]) / 3.0;
        cy[t] = (xy[2 * a + 1] + xy[2 * b + 1] + xy[2 * c + 1]) / 3.0;
    }
    // Morton order of the centroids: perm[new] = old
    std::vector<int64_t> perm(nt);
    std::iota(perm.begin(), perm.end(), 0);
    if (d->morton_reorder) {
        double x0 = *std::min_element(cx.begin(), cx.end()), x1 = *std::max_element(cx.begin(), cx.end());
        double y0 = *std::min_element(cy.begin(), cy.end()), y1 = *std::max_element(cy.begin(), cy.end());
        double sx = x1 > x0 ? 65535.0 / (x1 - x0) : 0.0, sy = y1 > y0 ? 65535.0 / (y1 - y0) : 0.0;
        std::vector<uint32_t> code(nt);
        for (int64_t t = 0; t < nt; ++t) {
            uint32_t ix = (uint32_t)((cx[t] - x0) * sx), iy = (uint32_t)((cy[t] - y0) * sy);
            code[t] = spread16(ix) | (spread16(iy) << 1);
        }
        std::stable_sort(perm.begin(), perm.end(), [&](int64_t a, int64_t b) { return code[a] < code[b]; });
    }
    std::vector<int64_t> inv(nt);
    for (int64_t i = 0; i < nt; ++i) inv[perm[i]] = i;

    // neighbours through sorted edge keys; face f of a cell is the edge (v_f, v_{f+1})
    struct HalfEdge {
        uint64_t key;
        int64_t cell;
        int face;
    };
    std::vector<HalfEdge> he(3 * nt);
    for (int64_t t = 0; t < nt; ++t)
        for (int f = 0; f < 3; ++f) {
            uint32_t p = (uint32_t)tv[3 * t + f], q = (uint32_t)tv[3 * t + (f + 1) % 3];
            uint64_t key = p < q ? ((uint64_t)p << 32) | q : ((uint64_t)q << 32) | p;
            he[3 * t + f] = {key, inv[t], f};
        }
    std::sort(he.begin(), he.end(), [](const HalfEdge &a, const HalfEdge &b) {
        return a.key < b.key || (a.key == b.key && a.cell < b.cell);
    });
    std::vector<int32_t> nbr(3 * nt, -1);
    for (size_t e = 0; e + 1 < he.size();) {
        if (he[e].key == he[e + 1].key) {
            if (e + 2 < he.size() && he[e + 2].key == he[e].key)
                return set_error(ZOOMY_EINVAL, "zoomy_mesh_create: an edge is shared by more than two triangles");
            nbr[he[e].face * nt + he[e].cell] = (int32_t)he[e + 1].cell;
            nbr[he[e + 1].face * nt + he[e + 1].cell] = (int32_t)he[e].cell;
            e += 2;
        } else {
            e += 1;
        }
    }
    // per (face, cell) geometry in the new order: outward unit normal, |e| / |Omega|
    std::vector<float> gnx(3 * nt), gny(3 * nt), glen(3 * nt);
    std::vector<double> area_new(nt);
    double dmin = 1e300;
    for (int64_t i = 0; i < nt; ++i) {
        const int64_t t = perm[i];
        double per = 0.0;
        for (int f = 0; f < 3; ++f) {
            int32_t p = tv[3 * t + f], q = tv[3 * t + (f + 1) % 3];
            double ex = xy[2 * q] - xy[2 * p], ey = xy[2 * q + 1] - xy[2 * p + 1];
            double len = std::sqrt(ex * ex + ey * ey);
            per += len;
            gnx[f * nt + i] = (float)(ey / len);
            gny[f * nt + i] = (float)(-ex / len);
            glen[f * nt + i] = (float)(len / area[t]);
        }
        area_new[i] = area[t];
        dmin = std::min(dmin, 2.0 * area[t] / per);
    }

    zoomy_ctx *c = new (std::nothrow) zoomy_ctx();
    if (!c) return set_error(ZOOMY_ENOMEM, "zoomy_mesh_create: host allocation");
    c->kind = ZOOMY_MESH_TRI;
    c->dim = 2;
    c->nx = nt;
    c->ny = 1;
    c->nc = nt;
    c->min_delta = dmin;
    c->bc[0] = d->bc[0];
    c->stream = (cudaStream_t)stream;
    c->perm = perm;
    if (d->bathymetry) c->bed_host.assign(d->bathymetry, d->bathymetry + nt);
    zoomy_status st = ctx_init_device(c);
    auto fail = [&](cudaError_t e, const char *w) {
        zoomy_status s2 = cuda_fail(e, w);
        zoomy_mesh_destroy(c);
        return s2;
    };
    if (st != ZOOMY_OK) {
        zoomy_mesh_destroy(c);
        return st;
    }
    cudaError_t e;
    if ((e = cudaMalloc(&c->tri_nbr_d, sizeof(int32_t) * 3 * nt)) != cudaSuccess) return fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&c->tri_geo_d, sizeof(float) * 9 * nt)) != cudaSuccess) return fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&c->tri_area_d, sizeof(double) * nt)) != cudaSuccess) return fail(e, "cudaMalloc");
    std::vector<float> geo(9 * nt);
    memcpy(geo.data(), gnx.data(), sizeof(float) * 3 * nt);
    memcpy(geo.data() + 3 * nt, gny.data(), sizeof(float) * 3 * nt);
    memcpy(geo.data() + 6 * nt, glen.data(), sizeof(float) * 3 * nt);
    if ((e = cudaMemcpy(c->tri_nbr_d, nbr.data(), sizeof(int32_t) * 3 * nt, cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail(e, "cudaMemcpy");
    if ((e = cudaMemcpy(c->tri_geo_d, geo.data(), sizeof(float) * 9 * nt, cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail(e, "cudaMemcpy");
    if ((e = cudaMemcpy(c->tri_area_d, area_new.data(), sizeof(double) * nt, cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail(e, "cudaMemcpy");
    *out = c;
    return ZOOMY_OK;
}

void tri_free(zoomy_ctx *c)
{
    cudaFree(c->tri_nbr_d);
    cudaFree(c->tri_geo_d);
    cudaFree(c->tri_area_d);
}

// ------------------------------------------------------------------------------------------
// Device: cell-centric stage kernel
// ------------------------------------------------------------------------------------------

struct TriArgs {
    StageArgs<float> s;      // X, Qn, out, bed, ld, physics, dt control (structured fields unused)
    const int32_t *nbr;      // [3][nc]
    const float *geo;        // nx[3][nc], ny[3][nc], |e|/|Omega| [3][nc]
    int64_t nc;
    int wall;                // boundary edges: 1 wall, 0 transmissive
    int nsm;                 // SMs of the device (grid size)
};

template <int N>
__device__ __forceinline__ void tri_load(const TriArgs &a, int64_t i, float *raw)
{
    constexpr int nv = 3 + 2 * N;
#pragma unroll
    for (int v = 0; v < nv; ++v) raw[v] = __ldg(a.s.X + v * a.s.ld + i);
    raw[nv] = __ldg(a.s.bed + i);
}

// Velocity moments of a raw state rotated into the face frame (n, t), then the cell record.
template <int N>
__device__ __forceinline__ void tri_cell(const float *raw, float nx, float ny, bool reflect, float hdry,
                                         CellRec<N, 2, float> &r)
{
    constexpr int m = N + 1;
    float hn[m], ht[m];
#pragma unroll
    for (int k = 0; k < m; ++k) {
        const float ha = raw[var_a<N, 2>(k)], hb = raw[var_b<N>(k)];
        hn[k] = ha * nx + hb * ny;
        ht[k] = hb * nx - ha * ny;
        if (reflect) hn[k] = -hn[k];
    }
    // in the face frame the x-moments are the normal ones: CellRec.a = n, CellRec.c = t
    make_cell<N, 2, float>(r, raw[0], raw[3 + 2 * N], hn, ht, hdry);
}

template <int N, int STAGE>
__global__ void __launch_bounds__(128) k_stage_tri(TriArgs a)
{
    constexpr int m = N + 1, nv = 3 + 2 * N;
    const StageArgs<float> &s = a.s;
    pdl_enter();  // the previous kernel's results (state, wave-speed slot, status) first
    if (*(volatile unsigned int *)&s.ctl->status) return;
    float dt;
    if (!step_dt(s, dt)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&s.ctl->status, DEV_NOWAVE);
        return;
    }
    if (STAGE == 1 && blockIdx.x == 0 && threadIdx.x == 0) step_bookkeeping(s, dt);
    float smax = 0.0f;
    unsigned flag = 0;
    // grid-stride over the cells: a bounded grid keeps the wave-speed reduction at one atomic per CTA
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.nc; i += (int64_t)gridDim.x * blockDim.x) {
        // every load of the cell is issued up front: its state, the neighbour indices, the face
        // geometry, the three neighbours' states (gathers) and, in stage 2, Q^n
        float raw[nv + 1];
        tri_load<N>(a, i, raw);
        int32_t jn[3];
#pragma unroll
        for (int f = 0; f < 3; ++f) jn[f] = __ldg(a.nbr + f * a.nc + i);
        float qn[nv];
        if (STAGE == 2) {
#pragma unroll
            for (int v = 0; v < nv; ++v) qn[v] = __ldg(s.Qn + v * s.ld + i);
        }
        float rawn[3][nv + 1];
#pragma unroll
        for (int f = 0; f < 3; ++f) tri_load<N>(a, bounds_idx(jn[f] >= 0 ? jn[f] : i, a.nc, &s.ctl->status), rawn[f]);
        float acc[nv];
#pragma unroll
        for (int v = 0; v < nv; ++v) acc[v] = 0.0f;
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            const int32_t j = jn[f];
            const float nx = __ldg(a.geo + f * a.nc + i), ny = __ldg(a.geo + (3 + f) * a.nc + i);
            const float lw = __ldg(a.geo + (6 + f) * a.nc + i);
            CellRec<N, 2, float> L, R;
            tri_cell<N>(raw, nx, ny, false, s.hdry, L);
            // neighbour, or the ghost of a boundary face: copy or wall reflection of this cell
            tri_cell<N>(rawn[f], nx, ny, j < 0 && a.wall != 0, s.hdry, R);
            float fc[1 + 2 * m], nc[1 + 2 * m], pd;
            face_term<N, 2, float>(L, frame<N, 2, float, false>(L), R, frame<N, 2, float, false>(R), s.g, s.hdry, fc,
                                   pd, nc);
            fc[1] += pd;
            // this cell is the left side: it receives -(fc + pd + nc) |e|/|Omega|, rotated back to (x, y)
            acc[0] -= lw * (fc[0] + nc[0]);
#pragma unroll
            for (int k = 0; k < m; ++k) {
                const float rn = fc[1 + k] + nc[1 + k], rt = fc[1 + m + k] + nc[1 + m + k];
                acc[var_a<N, 2>(k)] -= lw * (rn * nx - rt * ny);
                acc[var_b<N>(k)] -= lw * (rn * ny + rt * nx);
            }
        }
        // Newtonian source at the stage input, explicit
        CellRec<N, 2, float> me;
        {
            float ha[m], hb[m];
#pragma unroll
            for (int k = 0; k < m; ++k) {
                ha[k] = raw[var_a<N, 2>(k)];
                hb[k] = raw[var_b<N>(k)];
            }
            make_cell<N, 2, float>(me, raw[0], raw[nv], ha, hb, s.hdry);
        }
        float sa[m], sb[m];
        newtonian<N, 2, float>(me, s.nu_rho, sa, sb);
        float y[nv], ya[m], yb[m];
        y[0] = fmaf(dt, acc[0], raw[0]);
#pragma unroll
        for (int k = 0; k < m; ++k) {
            ya[k] = raw[var_a<N, 2>(k)] + dt * (acc[var_a<N, 2>(k)] + sa[k]);
            yb[k] = raw[var_b<N>(k)] + dt * (acc[var_b<N>(k)] + sb[k]);
        }
        if (s.src_implicit)
            friction_implicit<N, 2, float>(y[0], ya, yb, s.fric, s.C_rho, s.nu_imp, s.gn2, dt, s.hdry);
        else
            bottom_friction<N, 2, float>(y[0], ya, yb, s.fric, s.C_rho, s.gn2, dt, s.hdry);
#pragma unroll
        for (int k = 0; k < m; ++k) {
            y[var_a<N, 2>(k)] = ya[k];
            y[var_b<N>(k)] = yb[k];
        }
        if (STAGE == 2) {
#pragma unroll
            for (int v = 0; v < nv; ++v) y[v] = 0.5f * (qn[v] + y[v]);
            CellRec<N, 2, float> co;
#pragma unroll
            for (int k = 0; k < m; ++k) {
                ya[k] = y[var_a<N, 2>(k)];
                yb[k] = y[var_b<N>(k)];
            }
            make_cell<N, 2, float>(co, y[0], 0.0f, ya, yb, s.hdry);
            const float sp = wavespeed<N, 2, float>(co, s.g);
            if (!(sp <= 3.0e38f)) flag |= DEV_NAN;
            if (!(y[0] >= 0.0f)) flag |= (y[0] < 0.0f) ? DEV_NEGDEPTH : DEV_NAN;
            smax = (sp > smax || sp != sp) ? sp : smax;
        }
#pragma unroll
        for (int v = 0; v < nv; ++v) s.out[v * s.ld + i] = y[v];
    }
    if (STAGE == 2) {
        if (flag) atomicOr(&s.ctl->status, flag);
        // block maximum (NaN wins), then one atomic per CTA
        __shared__ float wmax[4];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float v = __shfl_xor_sync(0xffffffffu, smax, o);
            smax = (v > smax || v != v) ? v : smax;
        }
        if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = smax;
        __syncthreads();
        if (threadIdx.x < 32) {
            smax = threadIdx.x < 4 ? wmax[threadIdx.x] : 0.0f;
            reduce_smax<float>(s.ctl, s.slot_out, smax);
        }
    }
}

// ------------------------------------------------------------------------------------------
// Device: tiled face-centric stage kernel
// ------------------------------------------------------------------------------------------
//
// A CTA takes a tile of TRI_TILE consecutive (Morton-ordered) cells.  Each cell's record (primitive
// velocities, wave-speed parts and flux products) is built once, in the x/y frame, into shared
// memory.  A face is evaluated once when both of its cells are in the tile (by the lower cell, which
// writes both cells' contributions); a face to a cell outside the tile, or on the boundary, is
// evaluated by its tile's cell only.  The face frame needs the record rotated into (n, t): with
// alpha_n = alpha_x n_x + alpha_y n_y and alpha_t = alpha_y n_x - alpha_x n_y the flux products are
// quadratic forms, so
//   g_nn = g_xx n_x^2 + 2 g_xy n_x n_y + g_yy n_y^2,   g_nt = g_xy (n_x^2 - n_y^2) + (g_yy - g_xx) n_x n_y,
// and |u|, sum |alpha_k|^2 and sum |alpha_k| are invariant.  The three face contributions of a cell
// land in fixed slots and are added in face order: deterministic, no atomics.

constexpr int TRI_TILE = 128;

template <int N>
struct TriTileSmem {
    static constexpr int m = N + 1, nv = 3 + 2 * N, nrec = 5 + 5 * m;
    float rec[nrec][TRI_TILE];           // h, b, |u|, s2, s1, alpha_x[m], alpha_y[m], g_xx[m], g_xy[m], g_yy[m]
    float contrib[3][nv][TRI_TILE];      // face slot, variable, cell (x/y frame, times |e|/|Omega|)
    float geo[9][TRI_TILE];              // n_x[3], n_y[3], |e|/|Omega| [3]
    int32_t nbr[3][TRI_TILE];
    int32_t fj[3 * TRI_TILE];            // face list: neighbour
    uint16_t ftf[3 * TRI_TILE];          // face list: (tile cell << 2) | face
    int wsum[TRI_TILE / 32];
    float wmax[TRI_TILE / 32];
};

template <int N>
__device__ __forceinline__ void tile_store_rec(TriTileSmem<N> &S, int t, const CellRec<N, 2, float> &r)
{
    constexpr int m = N + 1;
    S.rec[0][t] = r.h;
    S.rec[1][t] = r.b;
    S.rec[2][t] = r.um;
    S.rec[3][t] = r.s2;
    S.rec[4][t] = r.s1;
#pragma unroll
    for (int k = 0; k < m; ++k) {
        S.rec[5 + k][t] = r.a[k];
        S.rec[5 + m + k][t] = r.c[k];
        S.rec[5 + 2 * m + k][t] = r.gaa[k];
        S.rec[5 + 3 * m + k][t] = r.gab[k];
        S.rec[5 + 4 * m + k][t] = r.gbb[k];
    }
}

// Record of x/y-frame values (h, b, |u|, s2, s1, alpha_x, alpha_y, g_xx, g_xy, g_yy) rotated into the
// frame of normal (nx, ny); reflect: the wall ghost (normal moments and g_nt change sign).
template <int N>
__device__ __forceinline__ void tile_rotate(float h, float b, float um, float s2, float s1, const float *ax,
                                            const float *ay, const float *gxx, const float *gxy, const float *gyy,
                                            float nx, float ny, bool reflect, CellRec<N, 2, float> &r)
{
    constexpr int m = N + 1;
    r.h = h;
    r.b = b;
    r.um = um;
    r.s2 = s2;
    r.s1 = s1;
    const float nxx = nx * nx, nyy = ny * ny, nxy = nx * ny;
#pragma unroll
    for (int k = 0; k < m; ++k) {
        const float an = fmaf(ax[k], nx, ay[k] * ny), at = fmaf(ay[k], nx, -ax[k] * ny);
        const float gnn = fmaf(gxx[k], nxx, fmaf(2.0f * gxy[k], nxy, gyy[k] * nyy));
        const float gnt = fmaf(gxy[k], nxx - nyy, (gyy[k] - gxx[k]) * nxy);
        r.a[k] = reflect ? -an : an;
        r.c[k] = at;
        r.gaa[k] = gnn;
        r.gab[k] = reflect ? -gnt : gnt;
        r.gbb[k] = 0.0f;
    }
}

template <int N>
__device__ __forceinline__ void tile_rotate_smem(const TriTileSmem<N> &S, int t, float nx, float ny, bool reflect,
                                                 CellRec<N, 2, float> &r)
{
    constexpr int m = N + 1;
    float ax[m], ay[m], gxx[m], gxy[m], gyy[m];
#pragma unroll
    for (int k = 0; k < m; ++k) {
        ax[k] = S.rec[5 + k][t];
        ay[k] = S.rec[5 + m + k][t];
        gxx[k] = S.rec[5 + 2 * m + k][t];
        gxy[k] = S.rec[5 + 3 * m + k][t];
        gyy[k] = S.rec[5 + 4 * m + k][t];
    }
    tile_rotate<N>(S.rec[0][t], S.rec[1][t], S.rec[2][t], S.rec[3][t], S.rec[4][t], ax, ay, gxx, gxy, gyy, nx, ny,
                   reflect, r);
}

template <int N>
__device__ __forceinline__ void tile_make_xy(const float *raw, float hdry, CellRec<N, 2, float> &r)
{
    constexpr int m = N + 1, nv = 3 + 2 * N;
    float ha[m], hb[m];
#pragma unroll
    for (int k = 0; k < m; ++k) {
        ha[k] = raw[var_a<N, 2>(k)];
        hb[k] = raw[var_b<N>(k)];
    }
    make_cell<N, 2, float>(r, raw[0], raw[nv], ha, hb, hdry);
}

template <int N, int STAGE>
__global__ void __launch_bounds__(TRI_TILE, 4) k_stage_tri_tile(TriArgs a)
{
    constexpr int m = N + 1, nv = 3 + 2 * N;
    __shared__ TriTileSmem<N> S;
    const StageArgs<float> &s = a.s;
    pdl_enter();
    if (*(volatile unsigned int *)&s.ctl->status) return;
    float dt;
    if (!step_dt(s, dt)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&s.ctl->status, DEV_NOWAVE);
        return;
    }
    if (STAGE == 1 && blockIdx.x == 0 && threadIdx.x == 0) step_bookkeeping(s, dt);
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    float smax = 0.0f;
    unsigned flag = 0;
    const int64_t ntiles = (a.nc + TRI_TILE - 1) / TRI_TILE;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t c0 = tile * TRI_TILE, i = c0 + t;
        const bool valid = i < a.nc;
        const int64_t ic = valid ? i : a.nc - 1;  // the tail's idle threads read a valid cell
        // phase A: the cell's state, neighbours, geometry (and Q^n) -> record and face ownership
        float raw[nv + 1];
        tri_load<N>(a, ic, raw);
        float qn[nv];
        if (STAGE == 2) {
#pragma unroll
            for (int v = 0; v < nv; ++v) qn[v] = __ldg(s.Qn + v * s.ld + ic);
        }
        int cnt = 0;
        int32_t jn[3];
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            jn[f] = __ldg(a.nbr + f * a.nc + ic);
            S.nbr[f][t] = jn[f];
            const int64_t j = jn[f];
            // owned faces by kind, packed 10 bits each: inside the tile, to a cell outside, boundary
            if (valid) cnt += j < 0 ? (1 << 20) : ((j < c0 || j >= c0 + TRI_TILE) ? (1 << 10) : (j > i ? 1 : 0));
        }
#pragma unroll
        for (int g = 0; g < 9; ++g) S.geo[g][t] = __ldg(a.geo + g * a.nc + ic);
        {
            CellRec<N, 2, float> xy;
            tile_make_xy<N>(raw, s.hdry, xy);
            tile_store_rec<N>(S, t, xy);
        }
        // block exclusive scan of the packed counts -> face list sorted by kind (inside faces first,
        // then faces to outside cells, then boundary faces), so that a warp mostly takes one branch
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) S.wsum[w] = incl;
        __syncthreads();
        int excl = incl - cnt, tot = 0;
#pragma unroll
        for (int q = 0; q < TRI_TILE / 32; ++q) {
            if (q < w) excl += S.wsum[q];
            tot += S.wsum[q];
        }
        const int n_in = tot & 1023, n_out = (tot >> 10) & 1023, nface = n_in + n_out + (tot >> 20);
        int pos[3] = {excl & 1023, n_in + ((excl >> 10) & 1023), n_in + n_out + (excl >> 20)};
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            const int64_t j = jn[f];
            const int kind = j < 0 ? 2 : ((j < c0 || j >= c0 + TRI_TILE) ? 1 : (j > i ? 0 : -1));
            if (valid && kind >= 0) {
                const int e = pos[kind]++;
                S.fj[e] = jn[f];
                S.ftf[e] = (uint16_t)((t << 2) | f);
            }
        }
        __syncthreads();
        // phase B: each listed face once
        for (int e = t; e < nface; e += TRI_TILE) {
            const int tl = S.ftf[e] >> 2, f = S.ftf[e] & 3;
            const int32_t j = S.fj[e];
            const float nx = S.geo[f][tl], ny = S.geo[3 + f][tl], lw = S.geo[6 + f][tl];
            const int64_t jl = (int64_t)j - c0;
            const bool inside = j >= 0 && jl >= 0 && jl < TRI_TILE;
            CellRec<N, 2, float> L, R;
            tile_rotate_smem<N>(S, tl, nx, ny, false, L);
            if (inside) {
                tile_rotate_smem<N>(S, (int)jl, nx, ny, false, R);
            } else if (j >= 0) {
                float rawj[nv + 1];
                tri_load<N>(a, bounds_idx(j, a.nc, &s.ctl->status), rawj);
                CellRec<N, 2, float> xy;
                tile_make_xy<N>(rawj, s.hdry, xy);
                tile_rotate<N>(xy.h, xy.b, xy.um, xy.s2, xy.s1, xy.a, xy.c, xy.gaa, xy.gab, xy.gbb, nx, ny, false, R);
            } else {
                // boundary: a copy of the cell, or its wall reflection
                tile_rotate_smem<N>(S, tl, nx, ny, a.wall != 0, R);
            }
            float fc[1 + 2 * m], nc[1 + 2 * m], pd;
            face_term<N, 2, float>(L, frame<N, 2, float, false>(L), R, frame<N, 2, float, false>(R), s.g, s.hdry, fc,
                                   pd, nc);
            // cell L receives -(fc + pd + nc), cell R +(fc - pd - nc) (pd on row n_0), rotated back to (x, y)
            S.contrib[f][0][tl] = -lw * (fc[0] + nc[0]);
#pragma unroll
            for (int k = 0; k < m; ++k) {
                const float rn = fc[1 + k] + nc[1 + k] + (k == 0 ? pd : 0.0f), rt = fc[1 + m + k] + nc[1 + m + k];
                S.contrib[f][var_a<N, 2>(k)][tl] = -lw * (rn * nx - rt * ny);
                S.contrib[f][var_b<N>(k)][tl] = -lw * (rn * ny + rt * nx);
            }
            if (inside) {
                const int tj = (int)jl;
                const int64_t ig = c0 + tl;
                const int fb = S.nbr[0][tj] == ig ? 0 : (S.nbr[1][tj] == ig ? 1 : 2);
                const float lwj = S.geo[6 + fb][tj];
                S.contrib[fb][0][tj] = lwj * (fc[0] - nc[0]);
#pragma unroll
                for (int k = 0; k < m; ++k) {
                    const float rn = fc[1 + k] - nc[1 + k] - (k == 0 ? pd : 0.0f), rt = fc[1 + m + k] - nc[1 + m + k];
                    S.contrib[fb][var_a<N, 2>(k)][tj] = lwj * (rn * nx - rt * ny);
                    S.contrib[fb][var_b<N>(k)][tj] = lwj * (rn * ny + rt * nx);
                }
            }
        }
        __syncthreads();
        // phase C: the cell update
        if (valid) {
            float acc[nv];
#pragma unroll
            for (int v = 0; v < nv; ++v) acc[v] = (S.contrib[0][v][t] + S.contrib[1][v][t]) + S.contrib[2][v][t];
            CellRec<N, 2, float> me;  // the x/y record, for the Newtonian source
            me.h = S.rec[0][t];
#pragma unroll
            for (int k = 0; k < m; ++k) {
                me.a[k] = S.rec[5 + k][t];
                me.c[k] = S.rec[5 + m + k][t];
            }
            float sa[m], sb[m];
            newtonian<N, 2, float>(me, s.nu_rho, sa, sb);
            float y[nv], ya[m], yb[m];
            y[0] = fmaf(dt, acc[0], raw[0]);
#pragma unroll
            for (int k = 0; k < m; ++k) {
                ya[k] = raw[var_a<N, 2>(k)] + dt * (acc[var_a<N, 2>(k)] + sa[k]);
                yb[k] = raw[var_b<N>(k)] + dt * (acc[var_b<N>(k)] + sb[k]);
            }
            if (s.src_implicit)
                friction_implicit<N, 2, float>(y[0], ya, yb, s.fric, s.C_rho, s.nu_imp, s.gn2, dt, s.hdry);
            else
                bottom_friction<N, 2, float>(y[0], ya, yb, s.fric, s.C_rho, s.gn2, dt, s.hdry);
#pragma unroll
            for (int k = 0; k < m; ++k) {
                y[var_a<N, 2>(k)] = ya[k];
                y[var_b<N>(k)] = yb[k];
            }
            if (STAGE == 2) {
#pragma unroll
                for (int v = 0; v < nv; ++v) y[v] = 0.5f * (qn[v] + y[v]);
                CellRec<N, 2, float> co;
#pragma unroll
                for (int k = 0; k < m; ++k) {
                    ya[k] = y[var_a<N, 2>(k)];
                    yb[k] = y[var_b<N>(k)];
                }
                make_cell<N, 2, float>(co, y[0], 0.0f, ya, yb, s.hdry);
                const float sp = wavespeed<N, 2, float>(co, s.g);
                if (!(sp <= 3.0e38f)) flag |= DEV_NAN;
                if (!(y[0] >= 0.0f)) flag |= (y[0] < 0.0f) ? DEV_NEGDEPTH : DEV_NAN;
                smax = (sp > smax || sp != sp) ? sp : smax;
            }
#pragma unroll
            for (int v = 0; v < nv; ++v) s.out[v * s.ld + i] = y[v];
        }
    }
    if (STAGE == 2) {
        if (flag) atomicOr(&s.ctl->status, flag);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float v = __shfl_xor_sync(0xffffffffu, smax, o);
            smax = (v > smax || v != v) ? v : smax;
        }
        if (lane == 0) S.wmax[w] = smax;
        __syncthreads();
        if (t < 32) {
            smax = t < TRI_TILE / 32 ? S.wmax[t] : 0.0f;
            reduce_smax<float>(s.ctl, s.slot_out, smax);
        }
    }
}

template <int N>
static cudaError_t launch_tri_tile(const TriArgs &a, int stage, cudaStream_t st)
{
    int64_t blocks = (a.nc + TRI_TILE - 1) / TRI_TILE;
    if (blocks > (int64_t)a.nsm * 4) blocks = (int64_t)a.nsm * 4;
    dim3 grid((unsigned)(blocks > 0 ? blocks : 1)), block(TRI_TILE);
    return stage == 1 ? launch_pdl(k_stage_tri_tile<N, 1>, grid, block, st, a)
                      : launch_pdl(k_stage_tri_tile<N, 2>, grid, block, st, a);
}

template <int N>
static cudaError_t launch_tri(const TriArgs &a, int stage, cudaStream_t st)
{
    int64_t blocks = (a.nc + 127) / 128;
    if (blocks > (int64_t)a.nsm * 16) blocks = (int64_t)a.nsm * 16;
    dim3 grid((unsigned)(blocks > 0 ? blocks : 1)), block(128);
    // programmatic dependent launch: the launch and CTA ramp overlap the previous kernel's tail
    return stage == 1 ? launch_pdl(k_stage_tri<N, 1>, grid, block, st, a) : launch_pdl(k_stage_tri<N, 2>, grid, block, st, a);
}

static cudaError_t launch_tri_level(int level, int tiled, const TriArgs &a, int stage, cudaStream_t st)
{
    if (tiled) {
        switch (level) {
            case 0: return launch_tri_tile<0>(a, stage, st);
            case 1: return launch_tri_tile<1>(a, stage, st);
            case 2: return launch_tri_tile<2>(a, stage, st);
            case 3: return launch_tri_tile<3>(a, stage, st);
            case 4: return launch_tri_tile<4>(a, stage, st);
        }
        return cudaErrorInvalidValue;
    }
    switch (level) {
        case 0: return launch_tri<0>(a, stage, st);
        case 1: return launch_tri<1>(a, stage, st);
        case 2: return launch_tri<2>(a, stage, st);
        case 3: return launch_tri<3>(a, stage, st);
        case 4: return launch_tri<4>(a, stage, st);
    }
    return cudaErrorInvalidValue;
}

zoomy_status tri_run_steps(zoomy_ctx *c, float *Q, int64_t ld, double dt, int nsteps)
{
    TriArgs a;
    memset(&a, 0, sizeof(a));
    StageArgs<float> &s = a.s;
    s.bed = (const float *)c->bed_dev;
    s.ld = ld;
    s.g = (float)c->g;
    s.hdry = (float)c->hdry;
    s.fric = c->fric.kind;
    s.nu_rho = c->fric.kind == ZOOMY_FRICTION_SLIP_NEWTONIAN ? (float)(c->fric.nu / c->fric.rho) : 0.0f;
    if (c->src_implicit) {  // friction by backward Euler after the stage: no explicit Newtonian term
        s.src_implicit = 1;
        s.nu_imp = s.nu_rho;
        s.nu_rho = 0.0f;
    }
    s.C_rho = (float)(c->fric.C / c->fric.rho);
    s.gn2 = (float)(c->g * c->fric.manning_n * c->fric.manning_n);
    s.cfl = c->cfl;
    s.dmin = c->min_delta;
    s.dt_fixed = dt;
    s.ctl = c->ctl;
    a.nbr = c->tri_nbr_d;
    a.geo = c->tri_geo_d;
    a.nc = c->nc;
    a.wall = c->bc[0] == ZOOMY_BC_WALL;
    a.nsm = c->nsm;
    float *Q1 = (float *)c->q1;
    for (int k = 0; k < nsteps; ++k) {
        s.slot_in = k & 1;
        s.slot_out = (k + 1) & 1;
        s.X = Q;
        s.Qn = Q;
        s.out = Q1;
        zoomy_status ps = prof_mark(c, 1, true);
        if (ps != ZOOMY_OK) return ps;
        const int tiled = c->tri_variant != ZOOMY_TRI_CELL;
        cudaError_t e = launch_tri_level(c->level, tiled, a, 1, c->stream);
        if (e != cudaSuccess) return cuda_fail(e, "triangle stage 1 launch");
        if ((ps = prof_mark(c, 1, false)) != ZOOMY_OK) return ps;
        s.X = Q1;
        s.Qn = Q;
        s.out = Q;
        if ((ps = prof_mark(c, 2, true)) != ZOOMY_OK) return ps;
        e = launch_tri_level(c->level, tiled, a, 2, c->stream);
        if (e != cudaSuccess) return cuda_fail(e, "triangle stage 2 launch");
        if ((ps = prof_mark(c, 2, false)) != ZOOMY_OK) return ps;
    }
    return ZOOMY_OK;
}

}  // namespace zoomy
