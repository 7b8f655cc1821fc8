// zoomy_kernels.h -- host-side entry points of the kernel translation units (internal).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace zoomy {

struct DevCtl;
template <typename T>
struct StageArgs;

// block_shape: warps per CTA (2D: row-marching warps; 1D: face-centric warps of 31 cells)
template <typename T>
cudaError_t launch_stage_struct(int dim, int level, const StageArgs<T> &a, int stage, int block_shape,
                                cudaStream_t st);

// second order in space (fv_order2.cu): 1D and structured 2D grids, FP32 / FP64
template <typename T>
cudaError_t launch_stage_order2(int dim, int level, const StageArgs<T> &a, int stage, int nsm, cudaStream_t st);
cudaError_t launch_stage_2d_f32(int level, const StageArgs<float> &a, int stage, int warps_per_block,
                                cudaStream_t st);

// every step of a call on a 1D line in one cooperative launch with grid barriers (fv_struct.cu):
// warps_per_cta in [1, 8]; DevCtl::bar zero at the launch; returns cudaErrorCooperativeLaunchTooLarge,
// without launching, when the CTAs cannot all be resident
template <typename T>
cudaError_t launch_steps_1d(int level, const StageArgs<T> &a, T *Q, T *Q1, int nsteps, int warps_per_cta, int nsm,
                            cudaStream_t st);

template <typename T>
cudaError_t launch_wavespeed(int dim, int level, const T *Q, int64_t ld, int64_t nc, T g, T hdry, DevCtl *ctl,
                             int slot, int nsm, cudaStream_t st);

template <typename T>
cudaError_t launch_mass(const T *h, int64_t nc, double area_const, const double *area, double *partial,
                        int npartial, double *out, cudaStream_t st);

}  // namespace zoomy
