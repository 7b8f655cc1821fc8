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

template <int N>
static cudaError_t launch_tri(const TriArgs &a, int stage, cudaStream_t st)
{
    int64_t blocks = (a.nc + 127) / 128;
    if (blocks > (int64_t)a.nsm * 16) blocks = (int64_t)a.nsm * 16;
    dim3 grid((unsigned)(blocks > 0 ? blocks : 1)), block(128);
    // programmatic dependent launch: the launch and CTA ramp overlap the previous kernel's tail
    return stage == 1 ? launch_pdl(k_stage_tri<N, 1>, grid, block, st, a) : launch_pdl(k_stage_tri<N, 2>, grid, block, st, a);
}

static cudaError_t launch_tri_level(int level, const TriArgs &a, int stage, cudaStream_t st)
{
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
        cudaError_t e = launch_tri_level(c->level, a, 1, c->stream);
        if (e != cudaSuccess) return cuda_fail(e, "triangle stage 1 launch");
        if ((ps = prof_mark(c, 1, false)) != ZOOMY_OK) return ps;
        s.X = Q1;
        s.Qn = Q;
        s.out = Q;
        if ((ps = prof_mark(c, 2, true)) != ZOOMY_OK) return ps;
        e = launch_tri_level(c->level, a, 2, c->stream);
        if (e != cudaSuccess) return cuda_fail(e, "triangle stage 2 launch");
        if ((ps = prof_mark(c, 2, false)) != ZOOMY_OK) return ps;
    }
    return ZOOMY_OK;
}

}  // namespace zoomy
