// step_noalloc.cu -- an SSP-RK2 step of the structured 2D FP32 path that allocates no memory.
//
// Some callers cannot call cudaMalloc: code that runs where the allocator is off limits (inside a
// host callback or a driver hook, under an external memory manager that owns every device
// allocation, or in a real-time loop where an allocation's implicit synchronisation is not
// acceptable).  zoomy_step_noalloc serves them: the caller passes its state, bed and stream, and the
// stage buffer plus the step's control block live in a fixed device array compiled into this
// library.  That array is reserved on every GPU that loads the library and stays there until the
// process exits, which is why its size is capped at ZOOMY_NOALLOC_SCRATCH_BYTES.
#include <cstdint>
#include <cstring>

#include <cuda_runtime.h>

#include "../../include/zoomy.h"
#include "fv_common.cuh"
#include "zoomy_internal.h"
#include "zoomy_kernels.h"

using namespace zoomy;

namespace {

constexpr size_t kScratchBytes = ZOOMY_NOALLOC_SCRATCH_BYTES;
constexpr size_t kCtlBytes = 256;  // DevCtl, padded so that the stage buffer stays 256-byte aligned
static_assert(sizeof(DevCtl) <= kCtlBytes, "control block must fit its slot");

// The shared scratch: [DevCtl | stage buffer Q1].  Host code must not use this name as an address.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Look up the device address of the scratch array on the current device.  This runs on every
// call: the lookup allocates nothing, and an address cached across calls would dangle after a
// cudaDeviceReset (the library's device code is loaded again, possibly elsewhere).  The first call
// on a device loads that device code.
zoomy_status scratch_setup(void **ptr, int *nsm)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e == cudaSuccess ? cudaErrorInvalidSymbol : e, "cudaGetSymbolAddress");
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    *ptr = p;
    *nsm = n > 0 ? n : 1;
    return ZOOMY_OK;
}

}  // namespace

extern "C" zoomy_status zoomy_step_noalloc(int64_t nx, int64_t ny, double x0, double x1, double y0, double y1,
                                           const int32_t *bc, int32_t level, const zoomy_friction *friction,
                                           double g, double cfl, double h_dry, const float *bed, float *Q,
                                           int64_t ld, double dt, int32_t nsteps, void *stream, double *t_advanced)
{
    const char *who = "zoomy_step_noalloc";
    if (!bc || !bed || !Q) return set_error(ZOOMY_EINVAL, "%s: NULL argument (bc, bed and Q are required)", who);
    if (nx < 1 || ny < 1 || !(x1 > x0) || !(y1 > y0)) return set_error(ZOOMY_EINVAL, "%s: empty grid", who);
    for (int i = 0; i < 4; ++i)
        if (bc[i] != ZOOMY_BC_TRANSMISSIVE && bc[i] != ZOOMY_BC_WALL)
            return set_error(ZOOMY_EINVAL, "%s: bc[%d] must be 0 or 1", who, i);
    if (level < 0 || level > ZOOMY_MAX_LEVEL) return set_error(ZOOMY_EINVAL, "%s: level outside [0, 4]", who);
    if (!(g > 0.0) || !(cfl > 0.0 && cfl <= 1.0) || !(h_dry >= 0.0) || nsteps < 0 || !(dt >= 0.0) || dt > 1e300)
        return set_error(ZOOMY_EINVAL, "%s: need g > 0, 0 < cfl <= 1, h_dry >= 0, dt >= 0, nsteps >= 0", who);
    zoomy_friction f = {ZOOMY_FRICTION_NONE, 0.0, 0.0, 1.0, 0.0};
    if (friction) f = *friction;
    if (!friction_ok(f)) return set_error(ZOOMY_EINVAL, "%s: bad friction parameters", who);
    // the kernels index cells with 32-bit integers: reject sizes whose products would wrap
    if (nx > INT32_MAX || ny > INT32_MAX || nx > INT32_MAX / ny)
        return set_error(ZOOMY_EINVAL, "%s: nx = %lld, ny = %lld exceed the 32-bit cell index", who, (long long)nx,
                         (long long)ny);
    const int64_t nc = nx * ny;
    const int nv = 2 * level + 3;
    if (ld < nc) return set_error(ZOOMY_EINVAL, "%s: ld < nx * ny", who);
    if (((uintptr_t)Q) % sizeof(float) || ((uintptr_t)bed) % sizeof(float))
        return set_error(ZOOMY_EINVAL, "%s: Q and bed must be 4-byte aligned float arrays", who);
    // the stage buffer has the caller's layout [nv][ld] and must fit the fixed scratch
    if (ld > (int64_t)(kScratchBytes / sizeof(float)) ||
        kCtlBytes + sizeof(float) * (size_t)nv * (size_t)ld > kScratchBytes)
        return set_error(ZOOMY_EINVAL,
                         "%s: state of %d x %lld floats needs %zu bytes of scratch; the fixed scratch holds %zu "
                         "(use zoomy_step for larger grids)",
                         who, nv, (long long)ld, kCtlBytes + sizeof(float) * (size_t)nv * (size_t)ld, kScratchBytes);
    void *scratch = nullptr;
    int nsm = 1;
    zoomy_status st = scratch_setup(&scratch, &nsm);
    if (st != ZOOMY_OK) return st;
    DevCtl *ctl = (DevCtl *)scratch;
    float *Q1 = (float *)((char *)scratch + kCtlBytes);
    cudaStream_t s = (cudaStream_t)stream;

    // the control block keeps the previous call's contents: clear it (wave-speed slots, time, status)
    cudaError_t e = cudaMemsetAsync(ctl, 0, sizeof(DevCtl), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    StageArgs<float> a;
    memset(&a, 0, sizeof(a));
    a.bed = bed;
    a.ld = ld;
    a.nx = (int)nx;
    a.ny = (int)ny;
    const double dx = (x1 - x0) / (double)nx, dy = (y1 - y0) / (double)ny;
    a.inv_dx = (float)(1.0 / dx);
    a.inv_dy = (float)(1.0 / dy);
    for (int i = 0; i < 4; ++i) a.bc[i] = bc[i];
    a.g = (float)g;
    a.hdry = (float)h_dry;
    a.fric = f.kind;
    a.nu_rho = f.kind == ZOOMY_FRICTION_SLIP_NEWTONIAN ? (float)(f.nu / f.rho) : 0.0f;
    a.C_rho = (float)(f.C / f.rho);
    a.gn2 = (float)(g * f.manning_n * f.manning_n);
    a.cfl = cfl;
    a.dmin = 2.0 * dx * dy / (2.0 * dx + 2.0 * dy);
    a.dt_fixed = dt;
    a.ctl = ctl;
    a.H = 64;
    a.nstrips = (int)((nx + 29) / 30);
    a.nsegs = (int)((ny + a.H - 1) / a.H);
    if (dt <= 0.0) {
        e = launch_wavespeed<float>(2, level, Q, ld, nc, (float)g, (float)h_dry, ctl, 0, nsm, s);
        if (e != cudaSuccess) return cuda_fail(e, "wavespeed launch");
    }
    for (int k = 0; k < nsteps; ++k) {
        a.slot_in = k & 1;
        a.slot_out = (k + 1) & 1;
        a.X = Q;
        a.Qn = Q;
        a.out = Q1;
        e = launch_stage_2d_f32(level, a, 1, 1, s);
        if (e != cudaSuccess) return cuda_fail(e, "stage 1 launch");
        a.X = Q1;
        a.Qn = Q;
        a.out = Q;
        e = launch_stage_2d_f32(level, a, 2, 1, s);
        if (e != cudaSuccess) return cuda_fail(e, "stage 2 launch");
    }
    if (!t_advanced) return ZOOMY_OK;
    DevCtl h;
    e = cudaMemcpyAsync(&h, ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    *t_advanced = h.t;
    if (h.status & DEV_NAN) return set_error(ZOOMY_ENAN, "%s: a step produced a non-finite state", who);
    if (h.status & DEV_NEGDEPTH) return set_error(ZOOMY_ENEGDEPTH, "%s: a step produced a negative depth", who);
    if (h.status & DEV_NOWAVE) return set_error(ZOOMY_ECFL, "%s: no positive finite wave speed", who);
    return ZOOMY_OK;
}
