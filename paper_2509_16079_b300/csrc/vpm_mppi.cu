// MPPI reweighting of §IV-A (Eq. 25) on the device. Reductions run in binary64 over a fixed
// thread-to-element mapping and a fixed tree, so results do not depend on timing.
#include <math.h>

#include "vpm_device.cuh"

namespace vpm {

constexpr int kMppiThreads = 1024;

template <class T, class Op>
__device__ T block_reduce(T v, Op op, T identity, T *scratch)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = (lane < (int)(blockDim.x >> 5)) ? scratch[lane] : identity;
        for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) scratch[0] = v;
    }
    __syncthreads();
    T r = scratch[0];
    __syncthreads();
    return r;
}

struct MinOp {
    __device__ float operator()(float a, float b) const { return fminf(a, b); }
};
struct SumOp {
    __device__ double operator()(double a, double b) const { return a + b; }
};

// w_i = exp(-(J_i - J_min) / lambda) / sum_j exp(-(J_j - J_min) / lambda), J_min and the sum
// over the finite costs. A cost that is not finite (a rollout that diverged; the rollout kernel
// stores NaN) takes the limit of Eq. 25 as J_i -> +inf: weight 0. With no finite cost every
// weight is NaN. One block.
__global__ void __launch_bounds__(kMppiThreads) mppi_weights_kernel(const float *J, int K,
                                                                   double lambda, float *w)
{
    __shared__ double sd[32];
    __shared__ float sf[32];
    float m = INFINITY;
    for (int i = threadIdx.x; i < K; i += blockDim.x)
        if (isfinite(J[i])) m = fminf(m, J[i]);
    m = block_reduce(m, MinOp(), (float)INFINITY, sf);
    if (!isfinite(m)) {
        for (int i = threadIdx.x; i < K; i += blockDim.x) w[i] = __int_as_float(0x7fc00000);
        return;
    }
    const double jmin = (double)m;
    double s = 0.0;
    for (int i = threadIdx.x; i < K; i += blockDim.x)
        if (isfinite(J[i])) s += exp(-((double)J[i] - jmin) / lambda);
    s = block_reduce(s, SumOp(), 0.0, sd);
    const double eta = 1.0 / s;
    for (int i = threadIdx.x; i < K; i += blockDim.x)
        w[i] = isfinite(J[i]) ? (float)(exp(-((double)J[i] - jmin) / lambda) * eta) : 0.f;
}

// mu[k] = sum_i w_i xi[i, k]. Block (32, 32): x indexes k (coalesced rows), y strides over i.
__global__ void __launch_bounds__(1024) mppi_update_kernel(const float *w, const float *xi, int K,
                                                           int H, float *mu)
{
    __shared__ double part[32][33];
    const int k = blockIdx.x * 32 + threadIdx.x;
    double s = 0.0;
    if (k < H)
        for (int i = threadIdx.y; i < K; i += 32) s = fma((double)w[i], (double)xi[(size_t)i * H + k], s);
    part[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && k < H) {
        double t = 0.0;
        for (int r = 0; r < 32; ++r) t += part[r][threadIdx.x];
        mu[k] = (float)t;
    }
}

__global__ void mppi_perturb_kernel(const float *mu, const float *eps, int K, int H, float *out)
{
    const size_t total = (size_t)K * H;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x)
        out[e] = mu[e % H] + eps[e];
}

cudaError_t launch_mppi_weights(const float *J, int K, double lambda, float *w, cudaStream_t s)
{
    mppi_weights_kernel<<<1, kMppiThreads, 0, s>>>(J, K, lambda, w);
    return cudaGetLastError();
}

cudaError_t launch_mppi_update(const float *w, const float *xi, int K, int H, float *mu,
                               cudaStream_t s)
{
    mppi_update_kernel<<<(H + 31) / 32, dim3(32, 32), 0, s>>>(w, xi, K, H, mu);
    return cudaGetLastError();
}

cudaError_t launch_mppi_perturb(const float *mu, const float *eps, int K, int H, float *out,
                                cudaStream_t s)
{
    const size_t total = (size_t)K * H;
    size_t blocks = (total + 255) / 256;
    if (blocks > 148 * 16) blocks = 148 * 16;
    if (blocks < 1) blocks = 1;
    mppi_perturb_kernel<<<(unsigned)blocks, 256, 0, s>>>(mu, eps, K, H, out);
    return cudaGetLastError();
}

}  // namespace vpm
