// zoomy_api.cu -- the C ABI of include/zoomy.h: contexts, model selection, the SSP-RK2 step
// driver (Sec. 2.1.2 "HyperbolicSolver": boundary handling, hyperbolic step and source step
// inside a time loop with adaptive dt), reductions and error reporting.
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/zoomy.h"
#include "fv_common.cuh"
#include "zoomy_kernels.h"
#include "zoomy_internal.h"

using namespace zoomy;

static thread_local char g_err[512] = "no error";

zoomy_status zoomy::set_error(zoomy_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

zoomy_status zoomy::cuda_fail(cudaError_t e, const char *where)
{
    return set_error(e == cudaErrorMemoryAllocation ? ZOOMY_ENOMEM : ZOOMY_ECUDA, "%s: %s", where,
                     cudaGetErrorString(e));
}

#define ZCHECK(call)                                                    \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);             \
    } while (0)

extern "C" const char *zoomy_last_error(void) { return g_err; }

extern "C" int32_t zoomy_version(void) { return 10000; }

static size_t elem_size(int dtype) { return dtype == ZOOMY_FP64 ? 8 : 4; }

extern "C" zoomy_status zoomy_mesh_create(const zoomy_mesh_desc *d, void *stream, zoomy_ctx **out)
{
    if (!d || !out) return set_error(ZOOMY_EINVAL, "zoomy_mesh_create: NULL argument");
    *out = nullptr;
    if (d->kind == ZOOMY_MESH_1D || d->kind == ZOOMY_MESH_2D) {
        if (d->nx < 1 || (d->kind == ZOOMY_MESH_2D && d->ny < 1))
            return set_error(ZOOMY_EINVAL, "zoomy_mesh_create: nx, ny must be >= 1");
        if (d->nx > (1LL << 30) || d->ny > (1LL << 30) || (d->kind == ZOOMY_MESH_2D && d->nx * d->ny > (1LL << 40)))
            return set_error(ZOOMY_EINVAL, "zoomy_mesh_create: grid too large");
        if (!(d->x1 > d->x0) || (d->kind == ZOOMY_MESH_2D && !(d->y1 > d->y0)))
            return set_error(ZOOMY_EINVAL, "zoomy_mesh_create: empty domain");
        int nbc = d->kind == ZOOMY_MESH_1D ? 2 : 4;
        for (int i = 0; i < nbc; ++i)
            if (d->bc[i] != ZOOMY_BC_TRANSMISSIVE && d->bc[i] != ZOOMY_BC_WALL)
                return set_error(ZOOMY_EINVAL, "zoomy_mesh_create: bc[%d] must be 0 or 1", i);
    } else if (d->kind == ZOOMY_MESH_TRI) {
        return create_tri_mesh(d, stream, out);
    } else {
        return set_error(ZOOMY_EINVAL, "zoomy_mesh_create: unknown mesh kind %d", d->kind);
    }
    zoomy_ctx *c = new (std::nothrow) zoomy_ctx();
    if (!c) return set_error(ZOOMY_ENOMEM, "zoomy_mesh_create: host allocation");
    c->kind = d->kind;
    c->dim = d->kind == ZOOMY_MESH_1D ? 1 : 2;
    c->nx = d->nx;
    c->ny = d->kind == ZOOMY_MESH_1D ? 1 : d->ny;
    c->nc = c->nx * c->ny;
    c->dx = (d->x1 - d->x0) / (double)c->nx;
    c->dy = c->dim == 2 ? (d->y1 - d->y0) / (double)c->ny : 1.0;
    c->area_const = c->dim == 2 ? c->dx * c->dy : c->dx;
    // Delta = 2 |Omega| / P: dx in 1D, dx dy / (dx + dy) for a rectangle
    c->min_delta = c->dim == 2 ? 2.0 * c->dx * c->dy / (2.0 * c->dx + 2.0 * c->dy) : c->dx;
    for (int i = 0; i < 4; ++i) c->bc[i] = d->bc[i];
    c->stream = (cudaStream_t)stream;
    if (d->bathymetry) c->bed_host.assign(d->bathymetry, d->bathymetry + c->nc);
    zoomy_status st = ctx_init_device(c);
    if (st != ZOOMY_OK) {
        zoomy_mesh_destroy(c);
        return st;
    }
    *out = c;
    return ZOOMY_OK;
}

zoomy_status zoomy::ctx_init_device(zoomy_ctx *c)
{
    ZCHECK(cudaGetDevice(&c->device));
    ZCHECK(cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device));
    ZCHECK(cudaMalloc(&c->ctl, sizeof(DevCtl)));
    ZCHECK(cudaMalloc(&c->ctl_aux, sizeof(DevCtl)));
    ZCHECK(cudaMalloc(&c->partials, sizeof(double) * (NPARTIAL + 1)));
    ZCHECK(cudaMemsetAsync(c->ctl, 0, sizeof(DevCtl), c->stream));
    ZCHECK(cudaStreamSynchronize(c->stream));
    return ZOOMY_OK;
}

extern "C" zoomy_status zoomy_mesh_destroy(zoomy_ctx *c)
{
    if (!c) return ZOOMY_OK;
    if (c->stream || c->ctl) cudaStreamSynchronize(c->stream);
    cudaFree(c->ctl);
    cudaFree(c->ctl_aux);
    cudaFree(c->partials);
    cudaFree(c->bed_dev);
    cudaFree(c->q1);
    cudaFree(c->qdev_host);
    cudaFree(c->closure_d);
    cudaFree(c->closure_pred);
    cudaFree(c->vam_sys);
    cudaFree(c->vam_p);
    cudaFree(c->closure_tc);
    for (cudaEvent_t ev : c->prof_events) cudaEventDestroy(ev);
    tri_free(c);
    ens_free(c);
    delete c;
    return ZOOMY_OK;
}

extern "C" zoomy_status zoomy_set_stream(zoomy_ctx *c, void *stream)
{
    if (!c) return set_error(ZOOMY_EINVAL, "zoomy_set_stream: NULL context");
    c->stream = (cudaStream_t)stream;
    return ZOOMY_OK;
}

extern "C" zoomy_status zoomy_mesh_info(zoomy_ctx *c, int64_t *ncells, double *min_delta)
{
    if (!c) return set_error(ZOOMY_EINVAL, "zoomy_mesh_info: NULL context");
    if (ncells) *ncells = c->nc;
    if (min_delta) *min_delta = c->min_delta;
    return ZOOMY_OK;
}

extern "C" zoomy_status zoomy_mesh_permutation(zoomy_ctx *c, int64_t *perm)
{
    if (!c || !perm) return set_error(ZOOMY_EINVAL, "zoomy_mesh_permutation: NULL argument");
    if (c->kind == ZOOMY_MESH_TRI && !c->perm.empty()) {
        memcpy(perm, c->perm.data(), sizeof(int64_t) * c->nc);
    } else {
        for (int64_t i = 0; i < c->nc; ++i) perm[i] = i;
    }
    return ZOOMY_OK;
}

extern "C" zoomy_status zoomy_model_set(zoomy_ctx *c, int32_t level, const zoomy_friction *fr, double g, double cfl,
                                        double h_dry, int32_t dtype)
{
    if (!c) return set_error(ZOOMY_EINVAL, "zoomy_model_set: NULL context");
    if (level < 0 || level > ZOOMY_MAX_LEVEL)
        return set_error(ZOOMY_EINVAL, "zoomy_model_set: level %d outside [0, %d]", level, ZOOMY_MAX_LEVEL);
    if (!(g > 0.0) || !(cfl > 0.0 && cfl <= 1.0) || !(h_dry >= 0.0))
        return set_error(ZOOMY_EINVAL, "zoomy_model_set: need g > 0, 0 < cfl <= 1, h_dry >= 0");
    if (dtype != ZOOMY_FP32 && dtype != ZOOMY_FP64) return set_error(ZOOMY_EINVAL, "zoomy_model_set: bad dtype");
    zoomy_friction f = {ZOOMY_FRICTION_NONE, 0.0, 0.0, 1.0, 0.0};
    if (fr) f = *fr;
    if (!friction_ok(f)) return set_error(ZOOMY_EINVAL, "zoomy_model_set: bad friction parameters");
    if (c->kind == ZOOMY_MESH_TRI && dtype != ZOOMY_FP32)
        return set_error(ZOOMY_EINVAL, "zoomy_model_set: triangle meshes run the FP32 state path");
    c->level = level;
    c->fric = f;
    c->g = g;
    c->cfl = cfl;
    c->hdry = h_dry;
    c->nv = c->dim == 1 ? level + 2 : 2 * level + 3;
    c->vam = 0;  // a new model leaves the VAM mode
    if (c->dtype != dtype || !c->bed_dev) {
        cudaFree(c->bed_dev);
        c->bed_dev = nullptr;
        c->dtype = dtype;
        // a flat bed is stored as zeros so that the kernels read one layout
        {
            size_t es = elem_size(dtype);
            ZCHECK(cudaMalloc(&c->bed_dev, es * c->nc));
            std::vector<char> tmp(es * c->nc);
            for (int64_t i = 0; i < c->nc; ++i) {
                double b = c->bed_host.empty() ? 0.0
                                               : c->bed_host[c->kind == ZOOMY_MESH_TRI && !c->perm.empty() ? c->perm[i] : i];
                if (dtype == ZOOMY_FP64)
                    ((double *)tmp.data())[i] = b;
                else
                    ((float *)tmp.data())[i] = (float)b;
            }
            ZCHECK(cudaMemcpyAsync(c->bed_dev, tmp.data(), es * c->nc, cudaMemcpyHostToDevice, c->stream));
            ZCHECK(cudaStreamSynchronize(c->stream));
        }
    }
    c->model_ok = true;
    return ZOOMY_OK;
}

extern "C" zoomy_status zoomy_nvars(zoomy_ctx *c, int32_t *nv)
{
    if (!c || !nv) return set_error(ZOOMY_EINVAL, "zoomy_nvars: NULL argument");
    if (!c->model_ok) return set_error(ZOOMY_ESTATE, "zoomy_nvars: call zoomy_model_set first");
    *nv = c->nv;
    return ZOOMY_OK;
}

static zoomy_status ensure_stage_buffer(zoomy_ctx *c, int64_t ld)
{
    size_t need = elem_size(c->dtype) * (size_t)c->nv * (size_t)ld;
    if (c->q1 && c->q1_bytes >= need) return ZOOMY_OK;
    cudaFree(c->q1);
    c->q1 = nullptr;
    c->q1_bytes = 0;
    ZCHECK(cudaMalloc(&c->q1, need));
    c->q1_bytes = need;
    return ZOOMY_OK;
}

template <typename T>
static void fill_args(zoomy_ctx *c, StageArgs<T> &a, int64_t ld, double dt)
{
    memset(&a, 0, sizeof(a));
    a.bed = (const T *)c->bed_dev;
    a.ld = ld;
    a.nx = (int)c->nx;
    a.ny = (int)c->ny;
    a.inv_dx = T(1.0 / c->dx);
    a.inv_dy = T(1.0 / c->dy);
    for (int i = 0; i < 4; ++i) a.bc[i] = c->bc[i];
    a.g = T(c->g);
    a.hdry = T(c->hdry);
    a.fric = c->fric.kind;
    a.nu_rho = c->fric.kind == ZOOMY_FRICTION_SLIP_NEWTONIAN ? T(c->fric.nu / c->fric.rho) : T(0);
    if (c->src_implicit) {  // friction by backward Euler after the stage: no explicit Newtonian term
        a.src_implicit = 1;
        a.nu_imp = a.nu_rho;
        a.nu_rho = T(0);
    }
    a.C_rho = T(c->fric.C / c->fric.rho);
    a.gn2 = T(c->g * c->fric.manning_n * c->fric.manning_n);
    a.cfl = c->cfl;
    a.dmin = c->min_delta;
    a.dt_fixed = dt;
    a.ctl = c->ctl;
    a.H = c->rows_per_warp > 0 ? c->rows_per_warp : rows_per_warp_for(c->nx, c->ny, c->nsm, 24);
    a.nstrips = (int)((c->nx + 29) / 30);
    a.nsegs = (int)((c->ny + a.H - 1) / a.H);
}

// Warps per CTA of the first-order 1D kernels (zoomy_tune_1d, else automatic: lines shorter than
// 65536 cells spread one-warp CTAs over the SMs, longer ones use 8-warp CTAs).
static int warps_per_cta_1d(const zoomy_ctx *c)
{
    if (c->warps_per_cta_1d > 0) return c->warps_per_cta_1d;
    return c->nx < 65536 ? 1 : 8;
}

// The persistent 1D launch (first-order lines, stage profiling off) is taken only when zoomy_tune_1d
// asks for it: two launches per step with programmatic dependent launch measured faster on GB300.
static bool persistent_1d(const zoomy_ctx *c, int nsteps)
{
    if (c->dim != 1 || c->order != 1 || c->prof_on || nsteps < 1) return false;
    return c->launch_1d == ZOOMY_LAUNCH_PERSISTENT;
}

template <typename T>
static cudaError_t launch_stage(zoomy_ctx *c, const StageArgs<T> &a, int stage)
{
    if (c->order == 2) return launch_stage_order2<T>(c->dim, c->level, a, stage, c->nsm, c->stream);
    if constexpr (sizeof(T) == 4) {
        // the specialised FP32 kernel indexes with 32-bit offsets
        if (c->dim == 2 && (int64_t)c->nv * a.ld < (1LL << 31))
            return launch_stage_2d_f32(c->level, a, stage, c->warps_per_block, c->stream);
    }
    return launch_stage_struct<T>(c->dim, c->level, a, stage, c->dim == 1 ? warps_per_cta_1d(c) : c->warps_per_block,
                                  c->stream);
}

template <typename T>
static zoomy_status run_steps(zoomy_ctx *c, T *Q, int64_t ld, double dt, int nsteps)
{
    if constexpr (sizeof(T) == 4) {
        if (c->closure_on) return closure_run_steps(c, Q, ld, dt, nsteps);
    } else {
        if (c->vam) return vam_run_steps(c, Q, ld, dt, nsteps);
    }
    T *Q1 = (T *)c->q1;
    if (dt <= 0.0) {
        cudaError_t e = launch_wavespeed<T>(c->dim, c->level, Q, ld, c->nc, T(c->g), T(c->hdry), c->ctl, 0, c->nsm,
                                            c->stream);
        if (e != cudaSuccess) return cuda_fail(e, "wavespeed launch");
    }
    if (c->kind == ZOOMY_MESH_TRI) return tri_run_steps(c, (float *)Q, ld, dt, nsteps);
    StageArgs<T> a;
    fill_args<T>(c, a, ld, dt);
    if (persistent_1d(c, nsteps)) {
        // DevCtl::bar was zeroed with the wave-speed slots at the start of the call
        cudaError_t e = launch_steps_1d<T>(c->level, a, Q, Q1, nsteps, warps_per_cta_1d(c), c->nsm, c->stream);
        if (e == cudaSuccess) return ZOOMY_OK;
        if (e != cudaErrorCooperativeLaunchTooLarge) return cuda_fail(e, "persistent 1D launch");
    }
    for (int s = 0; s < nsteps; ++s) {
        a.slot_in = s & 1;
        a.slot_out = (s + 1) & 1;
        a.X = Q;
        a.Qn = Q;
        a.out = Q1;
        zoomy_status ps = prof_mark(c, 1, true);
        if (ps != ZOOMY_OK) return ps;
        cudaError_t e = launch_stage<T>(c, a, 1);
        if (e != cudaSuccess) return cuda_fail(e, "stage 1 launch");
        if ((ps = prof_mark(c, 1, false)) != ZOOMY_OK) return ps;
        a.X = Q1;
        a.Qn = Q;
        a.out = Q;
        if ((ps = prof_mark(c, 2, true)) != ZOOMY_OK) return ps;
        e = launch_stage<T>(c, a, 2);
        if (e != cudaSuccess) return cuda_fail(e, "stage 2 launch");
        if ((ps = prof_mark(c, 2, false)) != ZOOMY_OK) return ps;
    }
    return ZOOMY_OK;
}

zoomy_status zoomy::read_status(zoomy_ctx *c, double *t_total)
{
    DevCtl h;
    ZCHECK(cudaMemcpyAsync(&h, c->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, c->stream));
    ZCHECK(cudaStreamSynchronize(c->stream));
    // the time and the sticky status are consumed by this read
    ZCHECK(cudaMemsetAsync((char *)c->ctl + offsetof(DevCtl, t), 0, sizeof(DevCtl) - offsetof(DevCtl, t), c->stream));
    if (t_total) *t_total = h.t;
    if (h.status & DEV_NAN) return set_error(ZOOMY_ENAN, "a step produced a non-finite state");
    if (h.status & DEV_NEGDEPTH) return set_error(ZOOMY_ENEGDEPTH, "a step produced a negative depth");
    if (h.status & DEV_NOWAVE) return set_error(ZOOMY_ECFL, "no positive finite wave speed for the CFL step");
    if (h.status & DEV_TIMEOUT) return set_error(ZOOMY_ETIMEOUT, "a device-side wait exceeded its limit");
    if (h.status & DEV_BOUNDS) return set_error(ZOOMY_EBOUNDS, "a gather index fell outside its buffer");
    return ZOOMY_OK;
}

zoomy_status zoomy::check_step_args(zoomy_ctx *c, const void *Q, int64_t ld, double dt, int32_t nsteps,
                                    const char *who)
{
    if (!c) return set_error(ZOOMY_EINVAL, "%s: NULL context", who);
    if (!c->model_ok) return set_error(ZOOMY_ESTATE, "%s: call zoomy_model_set first", who);
    if (!Q) return set_error(ZOOMY_EINVAL, "%s: NULL state", who);
    if (ld < c->nc) return set_error(ZOOMY_EINVAL, "%s: ld = %lld < ncells = %lld", who, (long long)ld, (long long)c->nc);
    if (((uintptr_t)Q) % elem_size(c->dtype)) return set_error(ZOOMY_EINVAL, "%s: misaligned state pointer", who);
    if (nsteps < 0) return set_error(ZOOMY_EINVAL, "%s: nsteps < 0", who);
    if (!(dt >= 0.0) || dt > 1e300) return set_error(ZOOMY_EINVAL, "%s: dt must be >= 0 and finite", who);
    return ZOOMY_OK;
}

extern "C" zoomy_status zoomy_step(zoomy_ctx *c, void *Q, int64_t ld, double dt, int32_t nsteps, double *t_advanced)
{
    zoomy_status st = check_step_args(c, Q, ld, dt, nsteps, "zoomy_step");
    if (st != ZOOMY_OK) return st;
    if (c->kind == ZOOMY_MESH_ENSEMBLE) return set_error(ZOOMY_EINVAL, "zoomy_step: use zoomy_ensemble_step");
    st = ensure_stage_buffer(c, ld);
    if (st != ZOOMY_OK) return st;
    // reset the wave-speed slots; time and status accumulate until read (read_status)
    ZCHECK(cudaMemsetAsync(c->ctl, 0, offsetof(DevCtl, t), c->stream));
    st = c->dtype == ZOOMY_FP64 ? run_steps<double>(c, (double *)Q, ld, dt, nsteps)
                                : run_steps<float>(c, (float *)Q, ld, dt, nsteps);
    if (st != ZOOMY_OK) return st;
    if (t_advanced) return read_status(c, t_advanced);
    return ZOOMY_OK;
}

extern "C" zoomy_status zoomy_step_host(zoomy_ctx *c, void *Qh, int64_t ld, double dt, int32_t nsteps,
                                        double *t_advanced)
{
    zoomy_status st = check_step_args(c, Qh, ld, dt, nsteps, "zoomy_step_host");
    if (st != ZOOMY_OK) return st;
    size_t bytes = elem_size(c->dtype) * (size_t)c->nv * (size_t)ld;
    if (!c->qdev_host || c->qdev_host_bytes < bytes) {
        cudaFree(c->qdev_host);
        c->qdev_host = nullptr;
        ZCHECK(cudaMalloc(&c->qdev_host, bytes));
        c->qdev_host_bytes = bytes;
    }
    ZCHECK(cudaMemcpyAsync(c->qdev_host, Qh, bytes, cudaMemcpyHostToDevice, c->stream));
    double t = 0.0;
    st = zoomy_step(c, c->qdev_host, ld, dt, nsteps, nullptr);
    if (st != ZOOMY_OK) return st;
    ZCHECK(cudaMemcpyAsync(Qh, c->qdev_host, bytes, cudaMemcpyDeviceToHost, c->stream));
    st = read_status(c, &t);
    if (t_advanced) *t_advanced = t;
    return st;
}

extern "C" zoomy_status zoomy_sync(zoomy_ctx *c, double *t_total)
{
    if (!c) return set_error(ZOOMY_EINVAL, "zoomy_sync: NULL context");
    return read_status(c, t_total);
}

extern "C" zoomy_status zoomy_max_wavespeed(zoomy_ctx *c, const void *Q, int64_t ld, double *out)
{
    zoomy_status st = check_step_args(c, Q, ld, 0.0, 0, "zoomy_max_wavespeed");
    if (st != ZOOMY_OK) return st;
    if (c->vam) return set_error(ZOOMY_EINVAL, "zoomy_max_wavespeed: not defined for the VAM model");
    if (!out) return set_error(ZOOMY_EINVAL, "zoomy_max_wavespeed: NULL output");
    if (c->closure_on) return closure_max_wavespeed(c, (const float *)Q, ld, out);
    ZCHECK(cudaMemsetAsync(c->ctl_aux, 0, sizeof(DevCtl), c->stream));
    cudaError_t e = c->dtype == ZOOMY_FP64
                        ? launch_wavespeed<double>(c->dim, c->level, (const double *)Q, ld, c->nc, c->g, c->hdry,
                                                   c->ctl_aux, 0, c->nsm, c->stream)
                        : launch_wavespeed<float>(c->dim, c->level, (const float *)Q, ld, c->nc, (float)c->g,
                                                  (float)c->hdry, c->ctl_aux, 0, c->nsm, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "wavespeed launch");
    DevCtl h;
    ZCHECK(cudaMemcpyAsync(&h, c->ctl_aux, sizeof(DevCtl), cudaMemcpyDeviceToHost, c->stream));
    ZCHECK(cudaStreamSynchronize(c->stream));
    if (c->dtype == ZOOMY_FP64) {
        double v;
        memcpy(&v, &h.smax_d[0], 8);
        *out = v;
    } else {
        float v;
        memcpy(&v, &h.smax_f[0], 4);
        *out = v;
    }
    if (h.status & DEV_NAN) return set_error(ZOOMY_ENAN, "non-finite state");
    return ZOOMY_OK;
}

// Advance to t_end with CFL steps in chunks (one wave-speed read per chunk) and land on t_end exactly:
// once fewer than ~1.25 CFL steps remain, one or two fixed steps of equal length finish the run.
extern "C" zoomy_status zoomy_advance(zoomy_ctx *c, void *Q, int64_t ld, double t_end, int32_t chunk, double *t_out,
                                      int64_t *steps_out)
{
    zoomy_status st = check_step_args(c, Q, ld, 0.0, 0, "zoomy_advance");
    if (st != ZOOMY_OK) return st;
    if (!(t_end >= 0.0) || !(t_end < 1e300) || chunk < 1)
        return set_error(ZOOMY_EINVAL, "zoomy_advance: need a finite t_end >= 0 and chunk >= 1");
    double t = 0.0;
    int64_t steps = 0;
    while (t_end - t > 1e-12 * t_end) {
        const double rem = t_end - t;
        double smax = 0.0;
        if ((st = zoomy_max_wavespeed(c, Q, ld, &smax)) != ZOOMY_OK) return st;
        if (!(smax > 0.0)) return set_error(ZOOMY_ECFL, "zoomy_advance: no positive finite wave speed");
        const double dt_est = c->cfl * c->min_delta / smax;
        const double want = 0.8 * rem / dt_est - 1.0;
        const int n = want >= (double)chunk ? chunk : (int)want;
        double dt_sum = 0.0;
        if (n >= 1) {
            if ((st = zoomy_step(c, Q, ld, 0.0, n, &dt_sum)) != ZOOMY_OK) return st;
            t += dt_sum;
            steps += n;
        } else {
            const int k = rem <= dt_est ? 1 : 2;
            for (int i = 0; i < k; ++i) {
                if ((st = zoomy_step(c, Q, ld, rem / k, 1, &dt_sum)) != ZOOMY_OK) return st;
                t += dt_sum;
            }
            steps += k;
            break;
        }
    }
    if (t_out) *t_out = t;
    if (steps_out) *steps_out = steps;
    return ZOOMY_OK;
}

extern "C" zoomy_status zoomy_mass(zoomy_ctx *c, const void *Q, int64_t ld, double *out)
{
    zoomy_status st = check_step_args(c, Q, ld, 0.0, 0, "zoomy_mass");
    if (st != ZOOMY_OK) return st;
    if (!out) return set_error(ZOOMY_EINVAL, "zoomy_mass: NULL output");
    const double *area = c->kind == ZOOMY_MESH_TRI ? c->tri_area_d : nullptr;
    cudaError_t e = c->dtype == ZOOMY_FP64
                        ? launch_mass<double>((const double *)Q, c->nc, c->area_const, area, c->partials, NPARTIAL,
                                              c->partials + NPARTIAL, c->stream)
                        : launch_mass<float>((const float *)Q, c->nc, c->area_const, area, c->partials, NPARTIAL,
                                             c->partials + NPARTIAL, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "mass launch");
    ZCHECK(cudaMemcpyAsync(out, c->partials + NPARTIAL, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    ZCHECK(cudaStreamSynchronize(c->stream));
    return ZOOMY_OK;
}

extern "C" zoomy_status zoomy_tune_set(zoomy_ctx *c, int32_t rows_per_warp, int32_t warps_per_block)
{
    if (!c) return set_error(ZOOMY_EINVAL, "zoomy_tune_set: NULL context");
    if (rows_per_warp < 1 || rows_per_warp > 4096 || warps_per_block < 1 || warps_per_block > 32)
        return set_error(ZOOMY_EINVAL, "zoomy_tune_set: rows_per_warp in [1, 4096], warps_per_block in [1, 32]");
    c->rows_per_warp = rows_per_warp;
    c->warps_per_block = warps_per_block;
    return ZOOMY_OK;
}

extern "C" zoomy_status zoomy_tune_1d(zoomy_ctx *c, int32_t mode, int32_t warps_per_cta)
{
    if (!c) return set_error(ZOOMY_EINVAL, "zoomy_tune_1d: NULL context");
    if (mode < ZOOMY_LAUNCH_AUTO || mode > ZOOMY_LAUNCH_PERSISTENT)
        return set_error(ZOOMY_EINVAL, "zoomy_tune_1d: mode must be 0, 1 or 2");
    if (warps_per_cta < 0 || warps_per_cta > 8)
        return set_error(ZOOMY_EINVAL, "zoomy_tune_1d: warps_per_cta must be in [0, 8]");
    c->launch_1d = mode;
    c->warps_per_cta_1d = warps_per_cta;
    return ZOOMY_OK;
}

zoomy_status zoomy::prof_mark(zoomy_ctx *c, int stage, bool start)
{
    if (!c->prof_on) return ZOOMY_OK;
    if (c->prof_used == c->prof_events.size()) {
        cudaEvent_t ev;
        ZCHECK(cudaEventCreate(&ev));
        c->prof_events.push_back(ev);
    }
    if (start) c->prof_kind.push_back(stage);
    ZCHECK(cudaEventRecord(c->prof_events[c->prof_used++], c->stream));
    return ZOOMY_OK;
}

extern "C" zoomy_status zoomy_profile_enable(zoomy_ctx *c, int32_t on)
{
    if (!c) return set_error(ZOOMY_EINVAL, "zoomy_profile_enable: NULL context");
    c->prof_on = on != 0;
    c->prof_used = 0;
    c->prof_kind.clear();
    return ZOOMY_OK;
}

extern "C" zoomy_status zoomy_profile_read(zoomy_ctx *c, int64_t *launches, double *total_ms)
{
    if (!c || !launches || !total_ms) return set_error(ZOOMY_EINVAL, "zoomy_profile_read: NULL argument");
    ZCHECK(cudaStreamSynchronize(c->stream));
    launches[0] = launches[1] = launches[2] = 0;
    total_ms[0] = total_ms[1] = total_ms[2] = 0.0;
    for (size_t k = 0; k < c->prof_kind.size(); ++k) {
        float ms = 0.f;
        ZCHECK(cudaEventElapsedTime(&ms, c->prof_events[2 * k], c->prof_events[2 * k + 1]));
        int s = c->prof_kind[k] - 1;
        launches[s] += 1;
        total_ms[s] += ms;
    }
    c->prof_used = 0;
    c->prof_kind.clear();
    return ZOOMY_OK;
}

// ------------------------------------------------------------------------------------------
// Autotuner (structured 2D): rows per warp segment and warps per block
// ------------------------------------------------------------------------------------------

static std::string tune_key(zoomy_ctx *c)
{
    char buf[256];
    cudaDeviceProp p;
    cudaGetDeviceProperties(&p, c->device);
    snprintf(buf, sizeof(buf), "%s|sm%d|%lldx%lld|L%d|%s", p.name, p.multiProcessorCount, (long long)c->nx,
             (long long)c->ny, c->level, c->dtype == ZOOMY_FP64 ? "f64" : "f32");
    return buf;
}

static bool tune_cache_lookup(const char *path, const std::string &key, int *H, int *W, double *us)
{
    if (!path) return false;
    FILE *f = fopen(path, "r");
    if (!f) return false;
    char line[512];
    bool found = false;
    while (fgets(line, sizeof(line), f)) {
        const char *k = strstr(line, "\"key\": \"");
        if (!k) continue;
        k += 8;
        const char *e = strchr(k, '"');
        if (!e || std::string(k, e - k) != key) continue;
        const char *h = strstr(line, "\"rows_per_warp\": ");
        const char *w = strstr(line, "\"warps_per_block\": ");
        const char *u = strstr(line, "\"us_per_step\": ");
        if (h && w) {
            *H = atoi(h + 17);
            *W = atoi(w + 19);
            *us = u ? atof(u + 15) : 0.0;
            found = *H >= 1 && *W >= 1;
        }
    }
    fclose(f);
    return found;
}

template <typename T>
static zoomy_status tune_measure(zoomy_ctx *c, const T *Q, int64_t ld, int H, int W, T *tmp, double *us)
{
    StageArgs<T> a;
    int saveH = c->rows_per_warp, saveW = c->warps_per_block;
    c->rows_per_warp = H;
    c->warps_per_block = W;
    fill_args<T>(c, a, ld, 1e-9);  // a tiny fixed step: the timing does not depend on it
    a.slot_in = 0;
    a.slot_out = 1;
    cudaEvent_t e0, e1;
    ZCHECK(cudaEventCreate(&e0));
    ZCHECK(cudaEventCreate(&e1));
    const int reps = 4;
    float best = 1e30f;
    for (int rep = 0; rep < reps + 1; ++rep) {
        ZCHECK(cudaEventRecord(e0, c->stream));
        a.X = Q;
        a.Qn = Q;
        a.out = (T *)c->q1;
        cudaError_t e = launch_stage<T>(c, a, 1);
        if (e != cudaSuccess) return cuda_fail(e, "autotune stage 1");
        a.X = (const T *)c->q1;
        a.Qn = tmp;
        a.out = tmp;
        e = launch_stage<T>(c, a, 2);
        if (e != cudaSuccess) return cuda_fail(e, "autotune stage 2");
        ZCHECK(cudaEventRecord(e1, c->stream));
        ZCHECK(cudaEventSynchronize(e1));
        float ms;
        ZCHECK(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0 && ms < best) best = ms;  // the first repetition warms up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->rows_per_warp = saveH;
    c->warps_per_block = saveW;
    *us = best * 1e3;
    return ZOOMY_OK;
}

extern "C" zoomy_status zoomy_autotune(zoomy_ctx *c, const void *Q, int64_t ld, const char *cache_path,
                                       int32_t *rows_per_warp_out, double *us_per_step_out)
{
    zoomy_status st = check_step_args(c, Q, ld, 0.0, 0, "zoomy_autotune");
    if (st != ZOOMY_OK) return st;
    if (c->kind != ZOOMY_MESH_2D) {  // only the structured 2D kernels have a decomposition to tune
        if (rows_per_warp_out) *rows_per_warp_out = c->rows_per_warp;
        if (us_per_step_out) *us_per_step_out = 0.0;
        return ZOOMY_OK;
    }
    const std::string key = tune_key(c);
    int H = 0, W = 0;
    double us = 0.0;
    if (!tune_cache_lookup(cache_path, key, &H, &W, &us)) {
        if ((st = ensure_stage_buffer(c, ld)) != ZOOMY_OK) return st;
        size_t bytes = elem_size(c->dtype) * (size_t)c->nv * (size_t)ld;
        void *tmp = nullptr;
        ZCHECK(cudaMalloc(&tmp, bytes));
        ZCHECK(cudaMemcpyAsync(tmp, Q, bytes, cudaMemcpyDeviceToDevice, c->stream));
        const int Hs[] = {8, 12, 16, 20, 24, 32, 40, 48, 56, 64, 72, 80, 96, 112, 128, 160, 192, 256};
        const int Ws_generic[] = {1, 2, 4};
        const bool packed = c->dtype == ZOOMY_FP32 && (int64_t)c->nv * ld < (1LL << 31);
        double best = 1e300;
        for (int h : Hs) {
            if (h > c->ny && h != Hs[0]) continue;
            for (int w : Ws_generic) {
                if (packed && w != 1) continue;  // the FP32 kernel runs one warp per CTA
                double t;
                st = c->dtype == ZOOMY_FP64 ? tune_measure<double>(c, (const double *)Q, ld, h, w, (double *)tmp, &t)
                                            : tune_measure<float>(c, (const float *)Q, ld, h, w, (float *)tmp, &t);
                if (st != ZOOMY_OK) {
                    cudaFree(tmp);
                    return st;
                }
                if (t < best) {
                    best = t;
                    H = h;
                    W = w;
                }
            }
        }
        cudaFree(tmp);
        us = best;
        if (cache_path) {
            FILE *f = fopen(cache_path, "a");
            if (f) {
                fprintf(f, "{\"key\": \"%s\", \"rows_per_warp\": %d, \"warps_per_block\": %d, \"us_per_step\": %.3f}\n",
                        key.c_str(), H, W, us);
                fclose(f);
            }
        }
    }
    c->rows_per_warp = H;
    c->warps_per_block = W;
    if (rows_per_warp_out) *rows_per_warp_out = H;
    if (us_per_step_out) *us_per_step_out = us;
    return ZOOMY_OK;
}

extern "C" zoomy_status zoomy_closure_set(zoomy_ctx *c, const float *params, const float *in_scale,
                                          const float *out_scale, double lambda)
{
    if (!c || !params || !in_scale || !out_scale) return set_error(ZOOMY_EINVAL, "zoomy_closure_set: NULL argument");
    if (!c->model_ok || c->kind != ZOOMY_MESH_2D || c->level != 1 || c->dtype != ZOOMY_FP32)
        return set_error(ZOOMY_EINVAL, "zoomy_closure_set: needs a structured 2D level-1 FP32 model");
    if (!(lambda >= 0.0)) return set_error(ZOOMY_EINVAL, "zoomy_closure_set: lambda >= 0");
    if (c->src_implicit || c->order != 1)
        return set_error(ZOOMY_EINVAL, "zoomy_closure_set: needs the default source mode and first order");
    zoomy_status st = closure_upload(c, params, in_scale, out_scale);
    if (st != ZOOMY_OK) return st;
    c->closure_on = true;
    c->closure_lambda = lambda;
    return ZOOMY_OK;
}

extern "C" zoomy_status zoomy_source_mode(zoomy_ctx *c, int32_t mode)
{
    if (!c) return set_error(ZOOMY_EINVAL, "zoomy_source_mode: NULL context");
    if (mode < 0 || mode > 1) return set_error(ZOOMY_EINVAL, "zoomy_source_mode: mode is 0 or 1");
    if (c->kind == ZOOMY_MESH_ENSEMBLE || c->closure_on)
        return set_error(ZOOMY_EINVAL, "zoomy_source_mode: not available for ensembles or the learned closure");
    c->src_implicit = mode;
    return ZOOMY_OK;
}

extern "C" zoomy_status zoomy_space_order(zoomy_ctx *c, int32_t order)
{
    if (!c) return set_error(ZOOMY_EINVAL, "zoomy_space_order: NULL context");
    if (order < 1 || order > 2) return set_error(ZOOMY_EINVAL, "zoomy_space_order: order is 1 or 2");
    if (order == 2 && (c->kind == ZOOMY_MESH_TRI || c->kind == ZOOMY_MESH_ENSEMBLE || c->closure_on))
        return set_error(ZOOMY_EINVAL, "zoomy_space_order: order 2 needs a 1D or structured 2D context "
                                       "without the learned closure");
    c->order = order;
    return ZOOMY_OK;
}

extern "C" zoomy_status zoomy_closure_clear(zoomy_ctx *c)
{
    if (!c) return set_error(ZOOMY_EINVAL, "zoomy_closure_clear: NULL context");
    c->closure_on = false;
    return ZOOMY_OK;
}
