// mlp_train.cu -- training of the closure MLP on the GPU with hand-written kernels, and the
// extraction of training samples from level-N states.
//
// Network: 6 -> 64 -> 64 -> 6, tanh-form GELU, loss = mean over the batch and the six outputs of
// (y - t)^2 in the scaled output space; Adam (Kingma & Ba) on FP32 master weights.  The inference
// kernel (fv_closure.cu) later rounds the weights to BF16.
//   forward:   one thread per sample; the weights sit in shared memory; activations a1, a2 and the
//              GELU derivatives are stored SoA [64][n] for the backward pass
//   backward:  one thread per sample for the activation gradients dz2, dz1 (SoA)
//   weights:   dW = A^T dZ over the batch as a split-K reduction (per-block partials summed in a
//              fixed order: deterministic)
//   update:    Adam, element-wise
#include <cmath>
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/zoomy.h"
#include "fv_common.cuh"
#include "zoomy_internal.h"

namespace zoomy {

constexpr int NI = 6, NH = 64, NO = 6;
constexpr int NPARAM = NI * NH + NH + NH * NH + NH + NH * NO + NO;  // 4998
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NI * NH, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NH * NO;
constexpr int KCHUNK = 512;  // samples per split-K block

__device__ __forceinline__ void gelu_and_grad(float z, float &g, float &dg)
{
    const float c = 0.7978845608028654f, k = 0.044715f;
    const float u = c * (z + k * z * z * z);
    const float t = tanhf(u);
    g = 0.5f * z * (1.0f + t);
    dg = 0.5f * (1.0f + t) + 0.5f * z * (1.0f - t * t) * c * (1.0f + 3.0f * k * z * z);
}

// X: [n][6] scaled inputs, T: [n][6] scaled targets.  Writes a1, g1 (= gelu'(z1)), a2, g2 [64][n],
// dy [6][n] = 2 (y - t) / (6 n), and per-block partial sums of (y - t)^2.
__global__ void __launch_bounds__(128) k_mlp_forward(const float *P, const float *X, const float *T, int64_t n,
                                                     float *a1, float *g1, float *a2, float *g2, float *dy,
                                                     float *loss_part)
{
    __shared__ float w[NPARAM];
    __shared__ float red[128];
    for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) w[i] = P[i];
    __syncthreads();
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    float sq = 0.0f;
    if (s < n) {
        float x[NI], h1[NH], y[NO];
#pragma unroll
        for (int i = 0; i < NI; ++i) x[i] = X[s * NI + i];
#pragma unroll
        for (int j = 0; j < NH; ++j) {
            float z = w[OFF_B1 + j];
#pragma unroll
            for (int i = 0; i < NI; ++i) z = fmaf(x[i], w[OFF_W1 + i * NH + j], z);
            float g, dg;
            gelu_and_grad(z, g, dg);
            h1[j] = g;
            a1[j * n + s] = g;
            g1[j * n + s] = dg;
        }
#pragma unroll
        for (int o = 0; o < NO; ++o) y[o] = w[OFF_B3 + o];
        for (int j = 0; j < NH; ++j) {
            float z = w[OFF_B2 + j];
#pragma unroll
            for (int i = 0; i < NH; ++i) z = fmaf(h1[i], w[OFF_W2 + i * NH + j], z);
            float g, dg;
            gelu_and_grad(z, g, dg);
            a2[j * n + s] = g;
            g2[j * n + s] = dg;
#pragma unroll
            for (int o = 0; o < NO; ++o) y[o] = fmaf(g, w[OFF_W3 + j * NO + o], y[o]);
        }
        const float inv = 2.0f / (float)(NO * n);
#pragma unroll
        for (int o = 0; o < NO; ++o) {
            const float d = y[o] - T[s * NO + o];
            sq = fmaf(d, d, sq);
            dy[o * n + s] = inv * d;
        }
    }
    red[threadIdx.x] = sq;
    __syncthreads();
    for (int o = 64; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss_part[blockIdx.x] = red[0];
}

// dz2 = (dy W3^T) * g2, dz1 = (dz2 W2^T) * g1 (one thread per sample).
__global__ void __launch_bounds__(128) k_mlp_backward(const float *P, int64_t n, const float *g1, const float *g2,
                                                      const float *dy, float *dz1, float *dz2)
{
    __shared__ float w[NPARAM];
    for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) w[i] = P[i];
    __syncthreads();
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    float d[NO], e2[NH];
#pragma unroll
    for (int o = 0; o < NO; ++o) d[o] = dy[o * n + s];
#pragma unroll
    for (int j = 0; j < NH; ++j) {
        float v = 0.0f;
#pragma unroll
        for (int o = 0; o < NO; ++o) v = fmaf(d[o], w[OFF_W3 + j * NO + o], v);
        e2[j] = v * g2[j * n + s];
        dz2[j * n + s] = e2[j];
    }
    for (int i = 0; i < NH; ++i) {
        float v = 0.0f;
#pragma unroll
        for (int j = 0; j < NH; ++j) v = fmaf(e2[j], w[OFF_W2 + i * NH + j], v);
        dz1[i * n + s] = v * g1[i * n + s];
    }
}

// Split-K reduction C[i][j] = sum_s A[i][s] B[j][s] (A: [M][n] SoA, or the [n][M] sample-major
// inputs when a_rows_major = 0), plus column sums of B (bias gradients) when bias_part != nullptr.
// One block per chunk of KCHUNK samples; 256 threads cover the M x N outputs.
__global__ void __launch_bounds__(256) k_grad_chunk(const float *A, int a_soa, const float *B, int M, int N,
                                                    int64_t n, float *part, float *bias_part)
{
    __shared__ float As[64][65];
    __shared__ float Bs[64][65];
    const int64_t s0 = (int64_t)blockIdx.x * KCHUNK;
    const int64_t s1 = s0 + KCHUNK < n ? s0 + KCHUNK : n;
    float acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = 0.0f;
    float bacc = 0.0f;
    for (int64_t sb = s0; sb < s1; sb += 64) {
        const int cnt = (int)((s1 - sb) < 64 ? (s1 - sb) : 64);
        for (int idx = threadIdx.x; idx < 64 * 64; idx += 256) {
            const int r = idx / 64, k = idx % 64;  // row r, sample k of the tile
            float av = 0.0f, bv = 0.0f;
            if (k < cnt) {
                if (r < M) av = a_soa ? A[(int64_t)r * n + sb + k] : A[(sb + k) * M + r];
                if (r < N) bv = B[(int64_t)r * n + sb + k];
            }
            As[r][k] = av;
            Bs[r][k] = bv;
        }
        __syncthreads();
        // thread -> 16 outputs: i = (tid / 16) * 4 + qi, j = (tid % 16) * 4 + qj
        const int ib = (threadIdx.x / 16) * 4, jb = (threadIdx.x % 16) * 4;
        for (int k = 0; k < cnt; ++k) {
#pragma unroll
            for (int qi = 0; qi < 4; ++qi)
#pragma unroll
                for (int qj = 0; qj < 4; ++qj) acc[qi * 4 + qj] = fmaf(As[ib + qi][k], Bs[jb + qj][k], acc[qi * 4 + qj]);
        }
        if (bias_part && threadIdx.x < N)
            for (int k = 0; k < cnt; ++k) bacc += Bs[threadIdx.x][k];
        __syncthreads();
    }
    const int ib = (threadIdx.x / 16) * 4, jb = (threadIdx.x % 16) * 4;
#pragma unroll
    for (int qi = 0; qi < 4; ++qi)
#pragma unroll
        for (int qj = 0; qj < 4; ++qj) {
            const int i = ib + qi, j = jb + qj;
            if (i < M && j < N) part[(int64_t)blockIdx.x * M * N + i * N + j] = acc[qi * 4 + qj];
        }
    if (bias_part && threadIdx.x < N) bias_part[(int64_t)blockIdx.x * N + threadIdx.x] = bacc;
}

// out[k] = sum over chunks of part[c][k] (fixed order)
__global__ void k_sum_chunks(const float *part, int nchunks, int len, float *out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= len) return;
    float s = 0.0f;
    for (int c = 0; c < nchunks; ++c) s += part[(int64_t)c * len + k];
    out[k] = s;
}

__global__ void k_adam(float *P, const float *G, float *m, float *v, int len, float lr, float b1, float b2,
                       float eps, float c1, float c2)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= len) return;
    const float g = G[k];
    const float mk = b1 * m[k] + (1.0f - b1) * g;
    const float vk = b2 * v[k] + (1.0f - b2) * g * g;
    m[k] = mk;
    v[k] = vk;
    P[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
}

// Training samples from a level-N state: X = features (h, u_m, v_m, alpha_1, beta_1, lambda) * in_scale,
// T = (alpha_2, alpha_3, alpha_4, beta_2, beta_3, beta_4) / out_scale for the listed cells.
__global__ void k_closure_samples(const float *Q, int64_t ld, int level, const int64_t *cells, int64_t n,
                                  float lambda, float hdry, const float *in_scale, const float *out_scale, float *X,
                                  float *T)
{
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int64_t c = cells[s];
    const float h = Q[c];
    const float ih = h > hdry ? 1.0f / h : 0.0f;
    auto va = [&](int k) { return k == 0 ? 1 : 2 + k; };
    auto vb = [&](int k) { return k == 0 ? 2 : 2 + level + k; };
    const float f[6] = {h, Q[va(0) * ld + c] * ih, Q[vb(0) * ld + c] * ih, Q[va(1) * ld + c] * ih,
                        Q[vb(1) * ld + c] * ih, lambda};
    for (int i = 0; i < 6; ++i) X[s * 6 + i] = f[i] * in_scale[i];
    for (int k = 2; k <= 4; ++k) {
        const float a = k <= level ? Q[va(k) * ld + c] * ih : 0.0f;
        const float b = k <= level ? Q[vb(k) * ld + c] * ih : 0.0f;
        T[s * 6 + (k - 2)] = a / out_scale[k - 2];
        T[s * 6 + (k + 1)] = b / out_scale[k + 1];
    }
}

}  // namespace zoomy

using namespace zoomy;

struct zoomy_mlp {
    cudaStream_t stream = nullptr;
    float *P = nullptr, *G = nullptr, *m = nullptr, *v = nullptr;
    int64_t cap = 0;                 // samples the workspace holds
    float *work = nullptr;           // a1, g1, a2, g2 [64][cap], dy [6][cap], dz1, dz2 [64][cap]
    float *part = nullptr;           // split-K partials
    float *loss_part = nullptr;
    int64_t step = 0;
};

static zoomy_status mlp_reserve(zoomy_mlp *M, int64_t n)
{
    if (n <= M->cap) return ZOOMY_OK;
    cudaFree(M->work);
    cudaFree(M->part);
    cudaFree(M->loss_part);
    M->work = M->part = M->loss_part = nullptr;
    M->cap = 0;
    const int64_t nchunks = (n + KCHUNK - 1) / KCHUNK;
    cudaError_t e;
    if ((e = cudaMalloc(&M->work, sizeof(float) * (size_t)n * (6 * 64 + 6))) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&M->part, sizeof(float) * (size_t)nchunks * (64 * 64 + 64))) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&M->loss_part, sizeof(float) * (size_t)((n + 127) / 128))) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc");
    M->cap = n;
    return ZOOMY_OK;
}

extern "C" zoomy_status zoomy_mlp_create(const float *params, void *stream, zoomy_mlp **out)
{
    if (!params || !out) return set_error(ZOOMY_EINVAL, "zoomy_mlp_create: NULL argument");
    zoomy_mlp *M = new (std::nothrow) zoomy_mlp();
    if (!M) return set_error(ZOOMY_ENOMEM, "zoomy_mlp_create: host allocation");
    M->stream = (cudaStream_t)stream;
    cudaError_t e;
    if ((e = cudaMalloc(&M->P, sizeof(float) * NPARAM * 4)) != cudaSuccess) {
        delete M;
        return cuda_fail(e, "cudaMalloc");
    }
    M->G = M->P + NPARAM;
    M->m = M->G + NPARAM;
    M->v = M->m + NPARAM;
    if ((e = cudaMemset(M->G, 0, sizeof(float) * NPARAM * 3)) != cudaSuccess ||
        (e = cudaMemcpy(M->P, params, sizeof(float) * NPARAM, cudaMemcpyHostToDevice)) != cudaSuccess) {
        cudaFree(M->P);
        delete M;
        return cuda_fail(e, "zoomy_mlp_create upload");
    }
    *out = M;
    return ZOOMY_OK;
}

extern "C" zoomy_status zoomy_mlp_destroy(zoomy_mlp *M)
{
    if (!M) return ZOOMY_OK;
    cudaStreamSynchronize(M->stream);
    cudaFree(M->P);
    cudaFree(M->work);
    cudaFree(M->part);
    cudaFree(M->loss_part);
    delete M;
    return ZOOMY_OK;
}

extern "C" zoomy_status zoomy_mlp_get_params(zoomy_mlp *M, float *params)
{
    if (!M || !params) return set_error(ZOOMY_EINVAL, "zoomy_mlp_get_params: NULL argument");
    cudaError_t e = cudaMemcpyAsync(params, M->P, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, M->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(M->stream);
    return e == cudaSuccess ? ZOOMY_OK : cuda_fail(e, "zoomy_mlp_get_params");
}

// loss and full-batch gradient into M->G
static zoomy_status mlp_loss_grad(zoomy_mlp *M, const float *X, const float *T, int64_t n, float *loss)
{
    zoomy_status st = mlp_reserve(M, n);
    if (st != ZOOMY_OK) return st;
    const size_t cap = (size_t)M->cap;
    float *a1 = M->work, *g1 = a1 + 64 * cap, *a2 = g1 + 64 * cap, *g2 = a2 + 64 * cap, *dy = g2 + 64 * cap,
          *dz1 = dy + 6 * cap, *dz2 = dz1 + 64 * cap;
    const unsigned nb = (unsigned)((n + 127) / 128);
    cudaStream_t s = M->stream;
    // activations stored with the workspace stride n (not cap): kernels index [j * n + s]
    k_mlp_forward<<<nb, 128, 0, s>>>(M->P, X, T, n, a1, g1, a2, g2, dy, M->loss_part);
    k_mlp_backward<<<nb, 128, 0, s>>>(M->P, n, g1, g2, dy, dz1, dz2);
    const int nch = (int)((n + KCHUNK - 1) / KCHUNK);
    float *bias_part = M->part + (size_t)nch * 64 * 64;
    // W3 = a2^T dy (64 x 6), b3 = sum dy
    k_grad_chunk<<<nch, 256, 0, s>>>(a2, 1, dy, 64, 6, n, M->part, bias_part);
    k_sum_chunks<<<(64 * 6 + 255) / 256, 256, 0, s>>>(M->part, nch, 64 * 6, M->G + OFF_W3);
    k_sum_chunks<<<1, 256, 0, s>>>(bias_part, nch, 6, M->G + OFF_B3);
    // W2 = a1^T dz2 (64 x 64), b2 = sum dz2
    k_grad_chunk<<<nch, 256, 0, s>>>(a1, 1, dz2, 64, 64, n, M->part, bias_part);
    k_sum_chunks<<<(64 * 64 + 255) / 256, 256, 0, s>>>(M->part, nch, 64 * 64, M->G + OFF_W2);
    k_sum_chunks<<<1, 256, 0, s>>>(bias_part, nch, 64, M->G + OFF_B2);
    // W1 = x^T dz1 (6 x 64), b1 = sum dz1
    k_grad_chunk<<<nch, 256, 0, s>>>(X, 0, dz1, 6, 64, n, M->part, bias_part);
    k_sum_chunks<<<(6 * 64 + 255) / 256, 256, 0, s>>>(M->part, nch, 6 * 64, M->G + OFF_W1);
    k_sum_chunks<<<1, 256, 0, s>>>(bias_part, nch, 64, M->G + OFF_B1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "mlp gradient launches");
    if (loss) {
        std::vector<float> lp(nb);
        if ((e = cudaMemcpyAsync(lp.data(), M->loss_part, sizeof(float) * nb, cudaMemcpyDeviceToHost, s)) !=
                cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return cuda_fail(e, "loss read");
        double tot = 0.0;
        for (float x : lp) tot += x;
        *loss = (float)(tot / (double)(6 * n));
    }
    return ZOOMY_OK;
}

extern "C" zoomy_status zoomy_mlp_grad(zoomy_mlp *M, const float *X, const float *T, int64_t n, float *loss,
                                       float *grad)
{
    if (!M || !X || !T || n < 1) return set_error(ZOOMY_EINVAL, "zoomy_mlp_grad: bad arguments");
    zoomy_status st = mlp_loss_grad(M, X, T, n, loss);
    if (st != ZOOMY_OK) return st;
    if (grad) {
        cudaError_t e = cudaMemcpyAsync(grad, M->G, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, M->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(M->stream);
        if (e != cudaSuccess) return cuda_fail(e, "gradient read");
    }
    return ZOOMY_OK;
}

extern "C" zoomy_status zoomy_mlp_train_step(zoomy_mlp *M, const float *X, const float *T, int64_t n, float lr,
                                             float *loss)
{
    if (!M || !X || !T || n < 1 || !(lr > 0.0f)) return set_error(ZOOMY_EINVAL, "zoomy_mlp_train_step: bad arguments");
    zoomy_status st = mlp_loss_grad(M, X, T, n, loss);
    if (st != ZOOMY_OK) return st;
    M->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)M->step), c2 = 1.0f - powf(b2, (float)M->step);
    k_adam<<<(NPARAM + 255) / 256, 256, 0, M->stream>>>(M->P, M->G, M->m, M->v, NPARAM, lr, b1, b2, 1e-8f, c1, c2);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ZOOMY_OK : cuda_fail(e, "adam launch");
}

extern "C" zoomy_status zoomy_closure_samples(const float *Q, int64_t ld, int32_t level, const int64_t *cells, int64_t n,
                                              double lambda, double h_dry, const float *in_scale,
                                              const float *out_scale, float *X, float *T, void *stream)
{
    if (!Q || !cells || !in_scale || !out_scale || !X || !T || n < 0 || level < 1 || level > ZOOMY_MAX_LEVEL)
        return set_error(ZOOMY_EINVAL, "zoomy_closure_samples: bad arguments");
    if (n == 0) return ZOOMY_OK;
    k_closure_samples<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        Q, ld, level, cells, n, (float)lambda, (float)h_dry, in_scale, out_scale, X, T);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ZOOMY_OK : cuda_fail(e, "closure samples launch");
}

// Per-column maxima of |X| and |T| ([n][6] each) into max_x / max_t (device [6], zeroed by the
// caller): the bit patterns of non-negative floats order like unsigned integers.
__global__ void k_sample_absmax(const float *X, const float *T, int64_t n, unsigned *max_x, unsigned *max_t)
{
    __shared__ unsigned sx[6], st[6];
    if (threadIdx.x < 6) sx[threadIdx.x] = st[threadIdx.x] = 0u;
    __syncthreads();
    unsigned mx[6] = {0, 0, 0, 0, 0, 0}, mt[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            mx[j] = max(mx[j], __float_as_uint(fabsf(X[i * 6 + j])));
            mt[j] = max(mt[j], __float_as_uint(fabsf(T[i * 6 + j])));
        }
    }
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        atomicMax(&sx[j], mx[j]);
        atomicMax(&st[j], mt[j]);
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        atomicMax(&max_x[threadIdx.x], sx[threadIdx.x]);
        atomicMax(&max_t[threadIdx.x], st[threadIdx.x]);
    }
}

__global__ void k_sample_scale(float *X, float *T, int64_t n, const float *in_scale, const float *out_scale)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n * 6; i += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(i % 6);
        X[i] = __fmul_rn(X[i], in_scale[j]);
        T[i] = __fdiv_rn(T[i], out_scale[j]);  // IEEE division (the library builds with fast math)
    }
}

extern "C" zoomy_status zoomy_sample_scales(const float *X, const float *T, int64_t n, float *in_scale,
                                            float *out_scale, void *stream)
{
    if (!X || !T || !in_scale || !out_scale || n < 1) return set_error(ZOOMY_EINVAL, "zoomy_sample_scales: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned *d = nullptr;
    cudaError_t e = cudaMallocAsync(&d, 12 * sizeof(unsigned), st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
    unsigned h[12];
    if ((e = cudaMemsetAsync(d, 0, 12 * sizeof(unsigned), st)) == cudaSuccess) {
        const int64_t blocks = std::min<int64_t>((n + 255) / 256, 1024);
        k_sample_absmax<<<(unsigned)blocks, 256, 0, st>>>(X, T, n, d, d + 6);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    cudaFreeAsync(d, st);
    if (e != cudaSuccess) return cuda_fail(e, "zoomy_sample_scales");
    for (int j = 0; j < 6; ++j) {
        float mx, mt;
        memcpy(&mx, &h[j], 4);
        memcpy(&mt, &h[6 + j], 4);
        in_scale[j] = 1.0f / std::max(mx, 1e-12f);
        out_scale[j] = std::max(mt, 1e-12f);
    }
    return ZOOMY_OK;
}

extern "C" zoomy_status zoomy_sample_scale(float *X, float *T, int64_t n, const float *in_scale, const float *out_scale,
                                           void *stream)
{
    if (!X || !T || !in_scale || !out_scale || n < 0) return set_error(ZOOMY_EINVAL, "zoomy_sample_scale: bad arguments");
    if (n == 0) return ZOOMY_OK;
    const int64_t blocks = std::min<int64_t>((6 * n + 255) / 256, 4096);
    k_sample_scale<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(X, T, n, in_scale, out_scale);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ZOOMY_OK : cuda_fail(e, "sample scale launch");
}

