// reduce.cu -- whole-mesh reductions: the maximum wave speed that sets the CFL step
// (adaptive time stepping of Sec. 3.1) and the FP64 mass sum_i |Omega_i| h_i.
#include <cstdint>
#include <cuda_runtime.h>

#include "fv_common.cuh"
#include "zoomy_kernels.h"

namespace zoomy {

template <int N, int D, typename T>
__global__ void __launch_bounds__(256) k_wavespeed(const T *Q, int64_t ld, int64_t nc, T g, T hdry, DevCtl *ctl,
                                                   int slot)
{
    constexpr int m = N + 1;
    T smax = T(0);
    unsigned int flag = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nc; i += (int64_t)gridDim.x * blockDim.x) {
        T ha[m], hb[m];
#pragma unroll
        for (int k = 0; k < m; ++k) {
            ha[k] = Q[(int64_t)var_a<N, D>(k) * ld + i];
            if constexpr (D == 2) hb[k] = Q[(int64_t)var_b<N>(k) * ld + i];
        }
        CellRec<N, D, T> r;
        make_cell<N, D, T>(r, Q[i], T(0), ha, hb, hdry);
        T s = wavespeed<N, D, T>(r, g);
        if (!(s <= T(3.0e38))) flag |= DEV_NAN;
        if (!(Q[i] >= T(0))) flag |= (Q[i] < T(0)) ? DEV_NEGDEPTH : DEV_NAN;
        smax = (s > smax || s != s) ? s : smax;
    }
    if (flag) atomicOr(&ctl->status, flag);
    reduce_smax<T>(ctl, slot, smax);
}

template <typename T>
__global__ void __launch_bounds__(256) k_mass_partial(const T *h, int64_t nc, double area_const, const double *area,
                                                      double *partial)
{
    __shared__ double sh[256];
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nc; i += (int64_t)gridDim.x * blockDim.x)
        s += (area ? area[i] : area_const) * (double)h[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(256) k_sum_partials(const double *partial, int n, double *out)
{
    __shared__ double sh[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

template <int N, int D, typename T>
static cudaError_t ws(const T *Q, int64_t ld, int64_t nc, T g, T hdry, DevCtl *ctl, int slot, int nsm,
                      cudaStream_t st)
{
    int64_t blocks = (nc + 255) / 256;
    if (blocks > 8LL * nsm) blocks = 8LL * nsm;
    if (blocks < 1) blocks = 1;
    k_wavespeed<N, D, T><<<(unsigned)blocks, 256, 0, st>>>(Q, ld, nc, g, hdry, ctl, slot);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_wavespeed(int dim, int level, const T *Q, int64_t ld, int64_t nc, T g, T hdry, DevCtl *ctl,
                             int slot, int nsm, cudaStream_t st)
{
#define ZW(NN)                                                             \
    case NN:                                                               \
        return dim == 1 ? ws<NN, 1, T>(Q, ld, nc, g, hdry, ctl, slot, nsm, st) \
                        : ws<NN, 2, T>(Q, ld, nc, g, hdry, ctl, slot, nsm, st);
    switch (level) {
        ZW(0)
        ZW(1)
        ZW(2)
        ZW(3)
        ZW(4)
    }
#undef ZW
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_mass(const T *h, int64_t nc, double area_const, const double *area, double *partial,
                        int npartial, double *out, cudaStream_t st)
{
    k_mass_partial<T><<<npartial, 256, 0, st>>>(h, nc, area_const, area, partial);
    k_sum_partials<<<1, 256, 0, st>>>(partial, npartial, out);
    return cudaGetLastError();
}

template cudaError_t launch_wavespeed<float>(int, int, const float *, int64_t, int64_t, float, float, DevCtl *, int,
                                             int, cudaStream_t);
template cudaError_t launch_wavespeed<double>(int, int, const double *, int64_t, int64_t, double, double, DevCtl *,
                                              int, int, cudaStream_t);
template cudaError_t launch_mass<float>(const float *, int64_t, double, const double *, double *, int, double *,
                                        cudaStream_t);
template cudaError_t launch_mass<double>(const double *, int64_t, double, const double *, double *, int, double *,
                                         cudaStream_t);

}  // namespace zoomy
