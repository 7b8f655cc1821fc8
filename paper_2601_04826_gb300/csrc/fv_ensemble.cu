// fv_ensemble.cu -- batched ensembles of independent structured 2D runs of uneven sizes.
//
// Each member is its own square grid (side s_m on [0,1]^2, walls), with its own slip coefficient
// and its own CFL step.  All members' states are concatenated in one SoA array Q[v][ld] (member m's
// cell (i, j) at offset_m + j s_m + i).  The work unit is one (member, 30-column strip, segment of H
// rows) item, marched by one warp with the same device code as the single-grid FP32 kernel.
//
// Persistent mode: one cooperative launch runs every step of every member.  Warps take items from a
// per-phase atomic work counter (dynamic load balance over ragged members); phases are the initial
// wave speeds, then stage 1 and stage 2 of each step, separated by grid-wide barriers.  Every
// barrier wait is bounded: after the spin limit the kernel records ETIMEOUT and returns, so a
// barrier that cannot complete never hangs the GPU.  The launch can be captured in a CUDA graph.
// Batched mode: one launch per phase over all items (2 nsteps + 1 launches, graph-capturable).
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "struct2d_f32.cuh"
#include "zoomy_internal.h"
#include "zoomy_kernels.h"

namespace zoomy {

struct EnsMember {
    int64_t off;   // offset of the member's cells in the concatenated state
    int side;      // cells per side
    float inv_dx;  // = side (unit square)
    float C_rho;   // slip coefficient / rho of the member
    double dmin;   // CFL length 2 |Omega| / P = dx / 2 (same formula as a single grid)
};

struct EnsArgs {
    StageArgs<float> base;  // bed, ld, physics shared by all members
    float *Q, *Q1;          // concatenated state and stage buffer
    const EnsMember *mem;
    const int4 *items;      // (member, strip, segment, -)
    int nitems, nmembers, nsteps;
    DevCtl *ctls;           // one control block per member
    unsigned *counters;     // per-phase work counters [2 nsteps + 1]
    unsigned *bar;          // grid barrier: [0] arrivals, [1] generation
    unsigned *gstatus;      // launch-wide status (timeout)
    unsigned nbar;          // participants of the barrier (grid size + extra, see zoomy_ensemble_set_barrier)
    int64_t ncells;         // cells of all members (the concatenated arrays' extent)
    long long spin_limit;   // barrier spin iterations before giving up
};


// Arguments of one member for one phase: 0 reads Q; stage 1 reads Q, writes Q1; stage 2 reads Q1 and
// Q^n = Q, writes Q in place.
__device__ __forceinline__ StageArgs<float> member_args(const EnsArgs &e, int m, int stage, int k)
{
    StageArgs<float> a = e.base;
    const EnsMember mb = e.mem[m];
    // the member's cells lie inside the concatenated arrays (its last cell is checked)
    (void)bounds_idx(mb.off + (int64_t)mb.side * mb.side - 1, e.ncells, &e.ctls[m].status);
    a.X = (stage == 2 ? e.Q1 : e.Q) + mb.off;
    a.Qn = e.Q + mb.off;
    a.out = (stage == 1 ? e.Q1 : e.Q) + mb.off;
    a.bed = e.base.bed + mb.off;
    a.nx = a.ny = mb.side;
    a.inv_dx = a.inv_dy = mb.inv_dx;
    a.C_rho = mb.C_rho;
    a.dmin = mb.dmin;
    a.ctl = e.ctls + m;
    a.slot_in = k & 1;
    a.slot_out = (k + 1) & 1;
    return a;
}

// Initial wave speeds of an item's owned cells into the member's slot 0.
template <int N>
__device__ __forceinline__ void item_wavespeed(const StageArgs<float> &a, int strip, int seg, int lane)
{
    constexpr int m = N + 1;
    const int col = strip * 30 - 1 + lane;
    const bool owned = lane >= 1 && lane <= 30 && col < a.nx;
    const int r0 = seg * a.H, r1 = min(r0 + a.H, a.ny);
    float smax = 0.0f;
    unsigned flag = 0;
    if (owned) {
        for (int r = r0; r < r1; ++r) {
            const float *p = a.X + ((int64_t)r * a.nx + col);
            float ha[m], hb[m];
#pragma unroll
            for (int k = 0; k < m; ++k) {
                ha[k] = p[(int64_t)var_a<N, 2>(k) * a.ld];
                hb[k] = p[(int64_t)var_b<N>(k) * a.ld];
            }
            CellRec<N, 2, float> rec;
            make_cell<N, 2, float>(rec, p[0], 0.0f, ha, hb, a.hdry);
            const float s = wavespeed<N, 2, float>(rec, a.g);
            if (!(s <= 3.0e38f)) flag |= DEV_NAN;
            if (!(p[0] >= 0.0f)) flag |= (p[0] < 0.0f) ? DEV_NEGDEPTH : DEV_NAN;
            smax = (s > smax || s != s) ? s : smax;
        }
    }
    if (flag) atomicOr(&a.ctl->status, flag);
    reduce_smax<float>(a.ctl, 0, smax);
}

// One phase for one item: 0 = initial wave speeds, 1 / 2 = SSP-RK2 stages of step k.
template <int N>
__device__ __forceinline__ void run_item(const EnsArgs &e, int idx, int phase, int k, int lane)
{
    const int4 it = e.items[idx];
    const int m = it.x;
    StageArgs<float> a = member_args(e, m, phase, k);
    if (phase == 0) {
        item_wavespeed<N>(a, it.y, it.z, lane);
        return;
    }
    if (*(volatile unsigned int *)&a.ctl->status) return;
    float dt;
    if (!step_dt(a, dt)) {
        if (lane == 0) atomicOr(&a.ctl->status, DEV_NOWAVE);
        return;
    }
    if (phase == 1) {
        if (it.y == 0 && it.z == 0 && lane == 0) step_bookkeeping(a, dt);
        float smax = 0.0f;
        unsigned flag = 0;
        march_strip<N, 1, false, false>(a, it.y, it.z, lane, dt, smax, flag);
    } else {
        float smax = 0.0f;
        unsigned flag = 0;
        march_strip<N, 2, false, false>(a, it.y, it.z, lane, dt, smax, flag);
        if (flag) atomicOr(&a.ctl->status, flag);
        reduce_smax<float>(a.ctl, a.slot_out, smax);
    }
}

// Bounded grid barrier (one warp per CTA; lane 0 arrives).  Returns false on timeout.
__device__ __forceinline__ bool grid_barrier(const EnsArgs &e)
{
    unsigned ok = 1;
    if (threadIdx.x == 0) {
        volatile unsigned *gen = e.bar + 1;
        const unsigned g0 = *gen;
        __threadfence();
        if (atomicAdd(e.bar, 1u) == e.nbar - 1) {
            *(volatile unsigned *)e.bar = 0u;
            __threadfence();
            atomicAdd(e.bar + 1, 1u);
        } else {
            long long it = 0;
            while (*gen == g0) {
                if (++it > e.spin_limit || *(volatile unsigned *)e.gstatus) {
                    ok = 0;
                    atomicOr(e.gstatus, DEV_TIMEOUT);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

template <int N>
__device__ __forceinline__ void phase_loop(const EnsArgs &e, int phase, int k, int ctr)
{
    const int lane = threadIdx.x;
    while (true) {
        unsigned idx = 0;
        if (lane == 0) idx = atomicAdd(e.counters + ctr, 1u);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx >= (unsigned)e.nitems) break;
        run_item<N>(e, (int)idx, phase, k, lane);
    }
}

// One-warp CTAs: at level 1 (the ensemble workload) the kernel is held to 128 registers, 16 warps per
// SM (its natural allocation, 152 registers, leaves 13); other levels take what they need.
template <int N>
constexpr int ENS_MIN_CTAS = N == 1 ? 16 : 1;

template <int N>
__global__ void __launch_bounds__(32, ENS_MIN_CTAS<N>) k_ensemble_persistent(EnsArgs e)
{
    phase_loop<N>(e, 0, 0, 0);
    if (!grid_barrier(e)) return;
    for (int k = 0; k < e.nsteps; ++k) {
        phase_loop<N>(e, 1, k, 1 + 2 * k);
        if (!grid_barrier(e)) return;
        phase_loop<N>(e, 2, k, 2 + 2 * k);
        if (!grid_barrier(e)) return;
    }
}

template <int N>
__global__ void __launch_bounds__(32, ENS_MIN_CTAS<N>) k_ensemble_phase(EnsArgs e, int phase, int k)
{
    run_item<N>(e, blockIdx.x, phase, k, threadIdx.x);
}

// ------------------------------------------------------------------------------------------
// Host side
// ------------------------------------------------------------------------------------------

struct EnsState {
    std::vector<EnsMember> mem;
    int H = 32;
    EnsMember *mem_d = nullptr;
    int4 *items_d = nullptr;
    int nitems = 0;
    DevCtl *ctls_d = nullptr;
    unsigned *counters_d = nullptr;
    int counters_cap = 0;
    unsigned *bar_d = nullptr;  // [0] arrivals, [1] generation, [2] launch status
    int extra_participants = 0;
    long long spin_limit = 20000000LL;  // x ~64 ns sleeps: about a second per wait
    int persistent_grid = 0;
    cudaStream_t cs = nullptr;          // private stream for graph capture (the caller's may be legacy)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
};

static EnsState *ens(zoomy_ctx *c) { return (EnsState *)c->ens; }

static zoomy_status ens_build_items(zoomy_ctx *c, int H)
{
    EnsState *E = ens(c);
    std::vector<int4> items;
    for (int m = 0; m < (int)E->mem.size(); ++m) {
        const int s = E->mem[m].side;
        const int ns = (s + 29) / 30, ng = (s + H - 1) / H;
        for (int g = 0; g < ng; ++g)
            for (int t = 0; t < ns; ++t) items.push_back(make_int4(m, t, g, 0));
    }
    cudaFree(E->items_d);
    E->items_d = nullptr;
    cudaError_t e = cudaMalloc(&E->items_d, sizeof(int4) * items.size());
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    e = cudaMemcpy(E->items_d, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
    E->nitems = (int)items.size();
    E->H = H;
    return ZOOMY_OK;
}

void ens_free(zoomy_ctx *c)
{
    EnsState *E = ens(c);
    if (!E) return;
    cudaFree(E->mem_d);
    cudaFree(E->items_d);
    cudaFree(E->ctls_d);
    cudaFree(E->counters_d);
    cudaFree(E->bar_d);
    if (E->cs) cudaStreamDestroy(E->cs);
    if (E->ev_in) cudaEventDestroy(E->ev_in);
    if (E->ev_out) cudaEventDestroy(E->ev_out);
    delete E;
    c->ens = nullptr;
}

typedef void (*PersistentFn)(EnsArgs);
static PersistentFn persistent_fn(int level)
{
    switch (level) {
        case 0: return k_ensemble_persistent<0>;
        case 1: return k_ensemble_persistent<1>;
        case 2: return k_ensemble_persistent<2>;
        case 3: return k_ensemble_persistent<3>;
        case 4: return k_ensemble_persistent<4>;
    }
    return nullptr;
}

static cudaError_t launch_phase(int level, const EnsArgs &a, int phase, int k, cudaStream_t st)
{
    dim3 grid(a.nitems), block(32);
    switch (level) {
        case 0: k_ensemble_phase<0><<<grid, block, 0, st>>>(a, phase, k); break;
        case 1: k_ensemble_phase<1><<<grid, block, 0, st>>>(a, phase, k); break;
        case 2: k_ensemble_phase<2><<<grid, block, 0, st>>>(a, phase, k); break;
        case 3: k_ensemble_phase<3><<<grid, block, 0, st>>>(a, phase, k); break;
        case 4: k_ensemble_phase<4><<<grid, block, 0, st>>>(a, phase, k); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

static EnsArgs ens_args(zoomy_ctx *c, float *Q, float *Q1, int64_t ld, int nsteps)
{
    EnsState *E = ens(c);
    EnsArgs a;
    memset(&a, 0, sizeof(a));
    a.Q = Q;
    a.Q1 = Q1;
    StageArgs<float> &s = a.base;
    s.bed = (const float *)c->bed_dev;
    s.ld = ld;
    s.bc[0] = s.bc[1] = s.bc[2] = s.bc[3] = 1;  // walls
    s.g = (float)c->g;
    s.hdry = (float)c->hdry;
    s.fric = c->fric.kind;
    s.nu_rho = c->fric.kind == ZOOMY_FRICTION_SLIP_NEWTONIAN ? (float)(c->fric.nu / c->fric.rho) : 0.0f;
    s.gn2 = (float)(c->g * c->fric.manning_n * c->fric.manning_n);
    s.cfl = c->cfl;
    s.dt_fixed = 0.0;
    s.H = E->H;
    a.mem = E->mem_d;
    a.items = E->items_d;
    a.nitems = E->nitems;
    a.nmembers = (int)E->mem.size();
    a.ncells = c->nc;
    a.nsteps = nsteps;
    a.ctls = E->ctls_d;
    a.counters = E->counters_d;
    a.bar = E->bar_d;
    a.gstatus = E->bar_d + 2;
    a.spin_limit = E->spin_limit;
    return a;
}

}  // namespace zoomy

using namespace zoomy;

extern "C" zoomy_status zoomy_ensemble_create(int32_t nmembers, const int64_t *sides, const double *C, int32_t level,
                                              double nu, double g, double cfl, double h_dry, void *stream,
                                              zoomy_ctx **out)
{
    if (!out || !sides || !C) return set_error(ZOOMY_EINVAL, "zoomy_ensemble_create: NULL argument");
    *out = nullptr;
    if (nmembers < 1) return set_error(ZOOMY_EINVAL, "zoomy_ensemble_create: nmembers < 1");
    if (level < 0 || level > ZOOMY_MAX_LEVEL) return set_error(ZOOMY_EINVAL, "zoomy_ensemble_create: bad level");
    if (!(g > 0.0) || !(cfl > 0.0 && cfl <= 1.0) || !(h_dry >= 0.0) || nu < 0.0)
        return set_error(ZOOMY_EINVAL, "zoomy_ensemble_create: need g > 0, 0 < cfl <= 1, h_dry >= 0, nu >= 0");
    int64_t total = 0;
    for (int m = 0; m < nmembers; ++m) {
        if (sides[m] < 1 || sides[m] > 65536 || !(C[m] >= 0.0))
            return set_error(ZOOMY_EINVAL, "zoomy_ensemble_create: member %d: side in [1, 65536], C >= 0", m);
        total += sides[m] * sides[m];
    }
    if ((int64_t)(2 * level + 3) * total >= (1LL << 31))
        return set_error(ZOOMY_EINVAL, "zoomy_ensemble_create: more than 2^31 state values");
    zoomy_ctx *c = new (std::nothrow) zoomy_ctx();
    if (!c) return set_error(ZOOMY_ENOMEM, "zoomy_ensemble_create: host allocation");
    c->kind = ZOOMY_MESH_ENSEMBLE;
    c->dim = 2;
    c->nx = total;
    c->ny = 1;
    c->nc = total;
    c->stream = (cudaStream_t)stream;
    EnsState *E = new (std::nothrow) EnsState();
    c->ens = E;
    zoomy_status st = ctx_init_device(c);
    if (st != ZOOMY_OK) {
        zoomy_mesh_destroy(c);
        return st;
    }
    int64_t off = 0;
    double dmin = 1e300;
    for (int m = 0; m < nmembers; ++m) {
        EnsMember mb;
        mb.off = off;
        mb.side = (int)sides[m];
        mb.C_rho = (float)C[m];
        const double dx = 1.0 / (double)sides[m];
        mb.dmin = 2.0 * dx * dx / (2.0 * dx + 2.0 * dx);
        mb.inv_dx = (float)(1.0 / dx);
        E->mem.push_back(mb);
        off += sides[m] * sides[m];
        dmin = std::min(dmin, mb.dmin);
    }
    c->min_delta = dmin;
    zoomy_friction f = {ZOOMY_FRICTION_SLIP_NEWTONIAN, 0.0, nu, 1.0, 0.0};
    // the model of the members (their slip coefficients are per member)
    if ((st = zoomy_model_set(c, level, &f, g, cfl, h_dry, ZOOMY_FP32)) != ZOOMY_OK) {
        zoomy_mesh_destroy(c);
        return st;
    }
    cudaError_t e;
    auto fail = [&](cudaError_t er, const char *w) {
        zoomy_status s2 = cuda_fail(er, w);
        zoomy_mesh_destroy(c);
        return s2;
    };
    if ((e = cudaMalloc(&E->mem_d, sizeof(EnsMember) * nmembers)) != cudaSuccess) return fail(e, "cudaMalloc");
    if ((e = cudaMemcpy(E->mem_d, E->mem.data(), sizeof(EnsMember) * nmembers, cudaMemcpyHostToDevice)) !=
        cudaSuccess)
        return fail(e, "cudaMemcpy");
    if ((e = cudaMalloc(&E->ctls_d, sizeof(DevCtl) * nmembers)) != cudaSuccess) return fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&E->bar_d, sizeof(unsigned) * 4)) != cudaSuccess) return fail(e, "cudaMalloc");
    if ((e = cudaStreamCreateWithFlags(&E->cs, cudaStreamNonBlocking)) != cudaSuccess) return fail(e, "cudaStreamCreate");
    if ((e = cudaEventCreateWithFlags(&E->ev_in, cudaEventDisableTiming)) != cudaSuccess) return fail(e, "cudaEventCreate");
    if ((e = cudaEventCreateWithFlags(&E->ev_out, cudaEventDisableTiming)) != cudaSuccess) return fail(e, "cudaEventCreate");
    if ((st = ens_build_items(c, 32)) != ZOOMY_OK) {
        zoomy_mesh_destroy(c);
        return st;
    }
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)persistent_fn(level), 32, 0)) !=
        cudaSuccess)
        return fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    E->persistent_grid = per_sm * c->nsm;
    *out = c;
    return ZOOMY_OK;
}

extern "C" zoomy_status zoomy_ensemble_offsets(zoomy_ctx *c, int64_t *offsets)
{
    if (!c || !offsets || c->kind != ZOOMY_MESH_ENSEMBLE)
        return set_error(ZOOMY_EINVAL, "zoomy_ensemble_offsets: need an ensemble context and an output array");
    EnsState *E = ens(c);
    for (size_t m = 0; m < E->mem.size(); ++m) offsets[m] = E->mem[m].off;
    offsets[E->mem.size()] = c->nc;
    return ZOOMY_OK;
}

extern "C" zoomy_status zoomy_ensemble_set_barrier(zoomy_ctx *c, int64_t spin_limit, int32_t extra_participants)
{
    if (!c || c->kind != ZOOMY_MESH_ENSEMBLE || spin_limit < 1 || extra_participants < 0)
        return set_error(ZOOMY_EINVAL, "zoomy_ensemble_set_barrier: bad arguments");
    ens(c)->spin_limit = spin_limit;
    ens(c)->extra_participants = extra_participants;
    return ZOOMY_OK;
}

static zoomy_status ens_read(zoomy_ctx *c, double *t_members, unsigned launch_status)
{
    EnsState *E = ens(c);
    const int M = (int)E->mem.size();
    std::vector<DevCtl> h(M);
    cudaError_t e = cudaMemcpyAsync(h.data(), E->ctls_d, sizeof(DevCtl) * M, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    unsigned any = 0;
    for (int m = 0; m < M; ++m) {
        if (t_members) t_members[m] = h[m].t;
        any |= h[m].status;
    }
    if (launch_status & DEV_TIMEOUT) return set_error(ZOOMY_ETIMEOUT, "ensemble barrier wait exceeded its spin limit");
    if (any & DEV_NAN) return set_error(ZOOMY_ENAN, "an ensemble member produced a non-finite state");
    if (any & DEV_NEGDEPTH) return set_error(ZOOMY_ENEGDEPTH, "an ensemble member produced a negative depth");
    if (any & DEV_NOWAVE) return set_error(ZOOMY_ECFL, "an ensemble member has no positive finite wave speed");
    return ZOOMY_OK;
}

extern "C" zoomy_status zoomy_ensemble_step(zoomy_ctx *c, void *Qv, int64_t ld, int32_t nsteps, int32_t mode,
                                            double *t_members)
{
    if (!c || c->kind != ZOOMY_MESH_ENSEMBLE) return set_error(ZOOMY_EINVAL, "zoomy_ensemble_step: not an ensemble");
    zoomy_status st = check_step_args(c, Qv, ld, 0.0, nsteps, "zoomy_ensemble_step");
    if (st != ZOOMY_OK) return st;
    if (mode < 0 || mode > 3) return set_error(ZOOMY_EINVAL, "zoomy_ensemble_step: mode in [0, 3]");
    if ((int64_t)c->nv * ld >= (1LL << 31)) return set_error(ZOOMY_EINVAL, "zoomy_ensemble_step: ld too large");
    EnsState *E = ens(c);
    float *Q = (float *)Qv;
    // stage buffer with the caller's layout
    size_t need = sizeof(float) * (size_t)c->nv * (size_t)ld;
    if (!c->q1 || c->q1_bytes < need) {
        cudaFree(c->q1);
        c->q1 = nullptr;
        cudaError_t e = cudaMalloc(&c->q1, need);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
        c->q1_bytes = need;
    }
    float *Q1 = (float *)c->q1;
    const int nphase = 2 * nsteps + 1;
    if (E->counters_cap < nphase) {
        cudaFree(E->counters_d);
        E->counters_d = nullptr;
        cudaError_t e = cudaMalloc(&E->counters_d, sizeof(unsigned) * nphase);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
        E->counters_cap = nphase;
    }
    const int M = (int)E->mem.size();
    // all work runs on the context's private stream, ordered after and before the caller's stream
    cudaStream_t s = E->cs;
    cudaError_t e = cudaEventRecord(E->ev_in, c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, E->ev_in, 0);
    if (e != cudaSuccess) return cuda_fail(e, "stream ordering");
    const bool graph = mode == 0 || mode == 2;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    if (graph && (e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return cuda_fail(e, "cudaStreamBeginCapture");
    auto enqueue = [&]() -> cudaError_t {
        cudaError_t r;
        if ((r = cudaMemsetAsync(E->ctls_d, 0, sizeof(DevCtl) * M, s)) != cudaSuccess) return r;
        if ((r = cudaMemsetAsync(E->bar_d, 0, sizeof(unsigned) * 4, s)) != cudaSuccess) return r;
        if ((r = cudaMemsetAsync(E->counters_d, 0, sizeof(unsigned) * nphase, s)) != cudaSuccess) return r;
        EnsArgs a = ens_args(c, Q, Q1, ld, nsteps);
        if (mode <= 1) {
            a.nbar = (unsigned)(E->persistent_grid + E->extra_participants);
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(E->persistent_grid);
            cfg.blockDim = dim3(32);
            cfg.stream = s;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeCooperative;
            attr[0].val.cooperative = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            void *args[] = {&a};
            return cudaLaunchKernelExC(&cfg, (const void *)persistent_fn(c->level), args);
        }
        for (int ph = 0; ph < nphase; ++ph) {
            const int phase = ph == 0 ? 0 : (ph % 2 == 1 ? 1 : 2);
            const int k = ph == 0 ? 0 : (ph - 1) / 2;
            if ((r = launch_phase(c->level, a, phase, k, s)) != cudaSuccess) return r;
        }
        return cudaSuccess;
    };
    e = enqueue();
    if (graph) {
        cudaError_t e2 = cudaStreamEndCapture(s, &g);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
        if (e == cudaSuccess) e = cudaGraphLaunch(ge, s);
        if (ge) cudaGraphExecDestroy(ge);
        if (g) cudaGraphDestroy(g);
    }
    if (e != cudaSuccess) return cuda_fail(e, "ensemble launch");
    if ((e = cudaEventRecord(E->ev_out, s)) != cudaSuccess || (e = cudaStreamWaitEvent(c->stream, E->ev_out, 0)) != cudaSuccess)
        return cuda_fail(e, "stream ordering");
    unsigned hst[4];
    if ((e = cudaMemcpyAsync(hst, E->bar_d, sizeof(hst), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync");
    return ens_read(c, t_members, hst[2]);
}

extern "C" zoomy_status zoomy_ensemble_autotune(zoomy_ctx *c, void *Qv, int64_t ld, int32_t *rows_out,
                                                double *us_out)
{
    if (!c || c->kind != ZOOMY_MESH_ENSEMBLE) return set_error(ZOOMY_EINVAL, "zoomy_ensemble_autotune: not an ensemble");
    zoomy_status st = check_step_args(c, Qv, ld, 0.0, 1, "zoomy_ensemble_autotune");
    if (st != ZOOMY_OK) return st;
    // candidates are timed on a scratch copy of the state (the step modifies it)
    size_t bytes = sizeof(float) * (size_t)c->nv * (size_t)ld;
    void *tmp = nullptr;
    cudaError_t e = cudaMalloc(&tmp, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    const int Hs[] = {16, 24, 32, 48, 64, 96, 128};
    double best = 1e300;
    int bestH = ens(c)->H;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int H : Hs) {
        if ((st = ens_build_items(c, H)) != ZOOMY_OK) break;
        double tbest = 1e300;
        for (int rep = 0; rep < 3; ++rep) {
            cudaMemcpyAsync(tmp, Qv, bytes, cudaMemcpyDeviceToDevice, c->stream);
            cudaEventRecord(e0, c->stream);
            st = zoomy_ensemble_step(c, tmp, ld, 2, 1, nullptr);
            cudaEventRecord(e1, c->stream);
            cudaEventSynchronize(e1);
            if (st != ZOOMY_OK) break;
            float ms;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) tbest = std::min(tbest, (double)ms);
        }
        if (st != ZOOMY_OK) break;
        if (tbest < best) {
            best = tbest;
            bestH = H;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(tmp);
    if (st != ZOOMY_OK) return st;
    if ((st = ens_build_items(c, bestH)) != ZOOMY_OK) return st;
    if (rows_out) *rows_out = bestH;
    if (us_out) *us_out = best * 1e3 / 2.0;
    return ZOOMY_OK;
}
