// zoomy_kernels.h -- host-side entry points of the kernel translation units (internal).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace zoomy {

struct DevCtl;
template <typename T>
struct StageArgs;

template <typename T>
cudaError_t launch_stage_struct(int dim, int level, const StageArgs<T> &a, int stage, int warps_per_block,
                                cudaStream_t st);

// second order in space (fv_order2.cu): 1D and structured 2D grids, FP32 / FP64
template <typename T>
cudaError_t launch_stage_order2(int dim, int level, const StageArgs<T> &a, int stage, int nsm, cudaStream_t st);
cudaError_t launch_stage_2d_f32(int level, const StageArgs<float> &a, int stage, int warps_per_block,
                                cudaStream_t st);

template <typename T>
cudaError_t launch_wavespeed(int dim, int level, const T *Q, int64_t ld, int64_t nc, T g, T hdry, DevCtl *ctl,
                             int slot, int nsm, cudaStream_t st);

template <typename T>
cudaError_t launch_mass(const T *h, int64_t nc, double area_const, const double *area, double *partial,
                        int npartial, double *out, cudaStream_t st);

}  // namespace zoomy
