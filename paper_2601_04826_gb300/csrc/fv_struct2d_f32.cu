// fv_struct2d_f32.cu -- FP32-state fused SSP-RK2 stage on structured 2D grids.
//
// Same scheme and data flow as the generic row-marching kernel in fv_struct.cu (one warp per
// 30-column strip, marching down H rows with the previous row in registers), specialised for the
// FP32 state:
//  * the x-face on the left of a cell and the y-face below it are evaluated together as the two
//    halves of packed f32x2 operations (FADD2/FMUL2/FFMA2);
//  * the path integral of the nonconservative product reduces to two weights per face;
//  * only the lower side of a face needs a new wave speed;
//  * face contributions are pre-scaled by dt and accumulate onto X + dt S(X), so a finished row
//    needs no copy of its input;
//  * the row loop is unrolled by two with the previous/current row states swapping roles, and the
//    next row is prefetched while the current one is computed;
//  * dry-state handling and the bottom stress are branch-free.
#include <cstdint>
#include <cuda_runtime.h>

#include "struct2d_f32.cuh"
#include "zoomy_kernels.h"

namespace zoomy {

template <int N, int STAGE, bool IMP>
__global__ void __launch_bounds__(32) k_stage_2d_f32(StageArgs<float> a)
{
    pdl_enter();  // launched with programmatic dependent launch: the previous kernel's results first
    if (*(volatile unsigned int *)&a.ctl->status) return;
    float dt;
    if (!step_dt(a, dt)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&a.ctl->status, DEV_NOWAVE);
        return;
    }
    if (STAGE == 1 && blockIdx.x == 0 && threadIdx.x == 0) step_bookkeeping(a, dt);
    // one warp per CTA: the strip / segment indices and the row loop are uniform across the CTA
    float smax = 0.0f;
    unsigned flag = 0;
    march_strip<N, STAGE, IMP, !IMP>(a, blockIdx.x % a.nstrips, blockIdx.x / a.nstrips, threadIdx.x, dt, smax, flag);
    if (STAGE == 2) {
        if (flag) atomicOr(&a.ctl->status, flag);
        reduce_smax<float>(a.ctl, a.slot_out, smax);
    }
}

template <int N>
static cudaError_t launch_f32(const StageArgs<float> &a, int stage, int wpb, cudaStream_t st)
{
    (void)wpb;  // one warp per CTA
    if (!a.bed) return cudaErrorInvalidValue;
    if (stage == 2 && a.Qn != a.out) return cudaErrorInvalidValue;  // stage 2 updates Q^n in place
    dim3 grid(a.nstrips * a.nsegs), block(32);
    // each launch overlaps its ramp with the previous kernel's tail (programmatic dependent launch)
    if (a.src_implicit)
        return stage == 1 ? launch_pdl(k_stage_2d_f32<N, 1, true>, grid, block, st, a)
                          : launch_pdl(k_stage_2d_f32<N, 2, true>, grid, block, st, a);
    return stage == 1 ? launch_pdl(k_stage_2d_f32<N, 1, false>, grid, block, st, a)
                      : launch_pdl(k_stage_2d_f32<N, 2, false>, grid, block, st, a);
}

cudaError_t launch_stage_2d_f32(int level, const StageArgs<float> &a, int stage, int wpb, cudaStream_t st)
{
    switch (level) {
        case 0: return launch_f32<0>(a, stage, wpb, st);
        case 1: return launch_f32<1>(a, stage, wpb, st);
        case 2: return launch_f32<2>(a, stage, wpb, st);
        case 3: return launch_f32<3>(a, stage, wpb, st);
        case 4: return launch_f32<4>(a, stage, wpb, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace zoomy
