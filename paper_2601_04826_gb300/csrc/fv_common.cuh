// fv_common.cuh -- device control block, variable layout and kernel arguments shared by the
// structured-grid kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "model.cuh"

namespace zoomy {

// Per-context device control block (one per zoomy_ctx, device memory).
struct DevCtl {
    unsigned int smax_f[2];          // max wave speed, FP32 bit pattern (s >= 0 orders like uint)
    unsigned long long smax_d[2];    // max wave speed, FP64 bit pattern
    unsigned int bar[4];             // grid barrier of the persistent 1D launch (arrivals, generation, status)
    double t;                        // time advanced by the steps of the current call
    double dt_last;                  // last step size
    unsigned int status;             // DEV_* flags, sticky until the host clears them
    unsigned int pad;
};

// DEV_TIMEOUT: a device-side wait gave up (grid barriers, tensor-core completion waits)
enum : unsigned int { DEV_NAN = 1u, DEV_NEGDEPTH = 2u, DEV_NOWAVE = 4u, DEV_TIMEOUT = 8u, DEV_BOUNDS = 16u };

// Bounds-checking build (compiled with -DZOOMY_BOUNDS_CHECK, build(debug=True)): every gather index
// of the stage, lifting and VAM kernels passes through bounds_idx before its access.  An index
// outside [0, n) sets DEV_BOUNDS in the control block (the host returns ZOOMY_EBOUNDS) and is replaced
// by 0, so the access itself stays inside the buffer.  Regular builds compile the check away.
#ifdef ZOOMY_BOUNDS_CHECK
__device__ __forceinline__ int64_t bounds_idx(int64_t i, int64_t n, unsigned *status)
{
    if (i >= 0 && i < n) return i;
    atomicOr(status, DEV_BOUNDS);
    return 0;
}
#else
__device__ __forceinline__ int64_t bounds_idx(int64_t i, int64_t, unsigned *) { return i; }
#endif

// Variable index of h alpha_k / h beta_k in the SoA state (Eq. (sme) variable order).
template <int N, int D>
__host__ __device__ constexpr int var_a(int k)
{
    return D == 1 ? 1 + k : (k == 0 ? 1 : 2 + k);
}
template <int N>
__host__ __device__ constexpr int var_b(int k)
{
    return k == 0 ? 2 : 2 + N + k;
}
template <int N, int D>
__host__ __device__ constexpr int nvars()
{
    return D == 1 ? 2 + N : 3 + 2 * N;
}

template <typename T>
struct StageArgs {
    const T *X;     // stage input [nv][ld]
    const T *Qn;    // Q^n for the final SSP-RK2 average (stage 2), else unused
    T *out;         // stage output [nv][ld] (stage 2 may alias Qn: pointwise read-then-write)
    const T *bed;   // [ncells] bed level, or nullptr for a flat bed
    int64_t ld;
    int nx, ny;
    T inv_dx, inv_dy;
    int bc[4];      // x-, x+, y-, y+ (1D: left, right): 0 transmissive, 1 wall
    T g, hdry;
    int fric;       // 0 none, 1 slip + Newtonian, 2 Manning
    T nu_rho, C_rho, gn2;        // nu_rho: the explicit Newtonian term (0 when the friction is implicit)
    int src_implicit;            // 1: friction by backward Euler after the stage (nu_imp = nu / rho)
    T nu_imp;
    double cfl, dmin, dt_fixed;  // dt_fixed > 0: fixed step; else CFL from ctl->smax[slot_in]
    int slot_in, slot_out;
    DevCtl *ctl;
    int nstrips, nsegs, H;       // 2D marching decomposition
};

// Step size of the current step: fixed, or dt = CFL * min Delta / max s (reading of the
// adaptive time stepping with CFL = 0.45 of Sec. 3.1), s_max taken over Q^n.
template <typename T>
__device__ __forceinline__ bool step_dt(const StageArgs<T> &a, int slot_in, T &dt)
{
    if (a.dt_fixed > 0.0) {
        dt = T(a.dt_fixed);
        return true;
    }
    double smax;
    if constexpr (sizeof(T) == 4)
        smax = (double)__uint_as_float(*(volatile unsigned int *)&a.ctl->smax_f[slot_in]);
    else
        smax = __longlong_as_double((long long)*(volatile unsigned long long *)&a.ctl->smax_d[slot_in]);
    if (!(smax > 0.0) || !(smax < 1e300)) return false;
    dt = T(a.cfl * a.dmin / smax);
    return true;
}

template <typename T>
__device__ __forceinline__ bool step_dt(const StageArgs<T> &a, T &dt)
{
    return step_dt(a, a.slot_in, dt);
}

// Bookkeeping done once per step by one thread of the first stage.
template <typename T>
__device__ __forceinline__ void step_bookkeeping(const StageArgs<T> &a, int slot_out, T dt)
{
    a.ctl->t += (double)dt;
    a.ctl->dt_last = (double)dt;
    if constexpr (sizeof(T) == 4)
        a.ctl->smax_f[slot_out] = 0u;
    else
        a.ctl->smax_d[slot_out] = 0ull;
}

template <typename T>
__device__ __forceinline__ void step_bookkeeping(const StageArgs<T> &a, T dt)
{
    step_bookkeeping(a, a.slot_out, dt);
}

// Programmatic dependent launch: a kernel launched with launch_pdl waits here for its predecessor on
// the stream to complete (with its memory visible), then lets the next kernel launch, so each launch
// and CTA ramp overlaps the kernel before it.
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
static inline cudaError_t launch_pdl_dyn(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                         Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

template <typename... KArgs, typename... Args>
static inline cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, Args... args)
{
    return launch_pdl_dyn(k, grid, block, 0, st, args...);
}

template <typename T>
__device__ __forceinline__ void reduce_smax(DevCtl *ctl, int slot, T s)
{
    // warp max, then one atomic per warp on the bit pattern (s >= 0, or NaN which wins)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        T v = __shfl_xor_sync(0xffffffffu, s, o);
        s = (v > s || v != v) ? v : s;
    }
    if ((threadIdx.x & 31) == 0) {
        if constexpr (sizeof(T) == 4)
            atomicMax(&ctl->smax_f[slot], __float_as_uint(s));
        else
            atomicMax(&ctl->smax_d[slot], (unsigned long long)__double_as_longlong(s));
    }
}

}  // namespace zoomy
