// Throughput probe: achievable rates of the FP32 FMA pipe, of the MUFU reciprocal square root
// and base-2 exponential, and of the rollout kernel's binary32 pair loop on this device. The
// paper has no counterpart; the rates state the ceiling the pair kernels are measured against.
#include <cstdio>
#include <vector>

#include "vpm_rollout.cuh"

namespace vpm {
vpm_status report_error(vpm_status st, const char *msg);
}

namespace {

constexpr int kChains = 8;       // independent dependency chains per thread
constexpr int kProbeThreads = 128;

__global__ void __launch_bounds__(kProbeThreads) ffma_probe(float *out, int iters, float b, float c)
{
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1e-3f * (float)threadIdx.x + (float)k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == 1234.5f) out[blockIdx.x] = s;     // keeps the chains live
}

__device__ __forceinline__ float mufu_rsqrt(float x)
{
    float y;
    asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float mufu_ex2_neg(float x)
{
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x));
    return y;
}

// x <- 1/sqrt(x) stays finite (fixed point 1); x <- 2^-x stays in (0.5, 1).
template <int KIND>
__global__ void __launch_bounds__(kProbeThreads) mufu_probe(float *out, int iters)
{
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 0.5f + 1e-4f * (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = KIND == 0 ? mufu_rsqrt(a[k]) : mufu_ex2_neg(a[k]);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == 1234.5f) out[blockIdx.x] = s;
}

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    Timer() { cudaEventCreate(&a); cudaEventCreate(&b); }
    ~Timer() { cudaEventDestroy(a); cudaEventDestroy(b); }
};

}  // namespace

extern "C" vpm_status vpm_probe_rate(int probe, int blocks_per_sm, double *h_rate)
{
    using vpm::report_error;
    char msg[160];
    if (!h_rate) return report_error(VPM_ERR_INVALID, "vpm_probe_rate: null rate pointer");
    if (probe < VPM_PROBE_FFMA || probe > VPM_PROBE_PAIRS_SYM)
        return report_error(VPM_ERR_INVALID, "vpm_probe_rate: unknown probe");
    if (blocks_per_sm < 1 || blocks_per_sm > 7)
        return report_error(VPM_ERR_INVALID, "vpm_probe_rate: blocks_per_sm must lie in 1..7");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (!e) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e) {
        snprintf(msg, sizeof msg, "vpm_probe_rate: %s", cudaGetErrorString(e));
        return report_error(VPM_ERR_CUDA, msg);
    }
    const int grid = sms * blocks_per_sm;
    Timer t;
    float ms = 0.f;
    double work = 0.0;
    if (probe <= VPM_PROBE_EX2) {
        float *d_out = nullptr;
        e = cudaMalloc(&d_out, sizeof(float) * grid);
        const int iters = probe == VPM_PROBE_FFMA ? 1 << 16 : 1 << 15;
        for (int pass = 0; pass < 2 && !e; ++pass) {   // pass 0 warms up
            if (pass == 1) cudaEventRecord(t.a);
            if (probe == VPM_PROBE_FFMA)
                ffma_probe<<<grid, kProbeThreads>>>(d_out, iters, 0.999f, 1e-3f);
            else if (probe == VPM_PROBE_RSQRT)
                mufu_probe<0><<<grid, kProbeThreads>>>(d_out, iters);
            else
                mufu_probe<1><<<grid, kProbeThreads>>>(d_out, iters);
            e = cudaGetLastError();
            if (pass == 1) cudaEventRecord(t.b);
        }
        if (!e) e = cudaEventSynchronize(t.b);
        if (!e) e = cudaEventElapsedTime(&ms, t.a, t.b);
        cudaFree(d_out);
        work = (double)grid * kProbeThreads * kChains * iters;
    } else {
        const int n = 1024, reps = 16;
        const int tpl = probe == VPM_PROBE_PAIRS_T4 ? 4 : (probe == VPM_PROBE_PAIRS_T2 ? 2 : 1);
        std::vector<float4> h(n);
        unsigned long long x = 0x9E3779B97F4A7C15ull;       // splitmix64 field: box [0, 6] x [-1.5, 1.5]
        auto next = [&x]() {
            x += 0x9E3779B97F4A7C15ull;
            unsigned long long z = x;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            return (double)((z ^ (z >> 31)) >> 11) * (1.0 / 9007199254740992.0);
        };
        for (int i = 0; i < n; ++i)
            h[i] = make_float4((float)(6.0 * next()), (float)(3.0 * next() - 1.5),
                               (float)(0.02 * next() - 0.01), 0.f);
        const bool sym = probe == VPM_PROBE_PAIRS_SYM;
        float4 *d_src = nullptr;
        float2 *d_out = nullptr, *d_scr = nullptr;
        e = cudaMalloc(&d_src, sizeof(float4) * n);
        if (!e) e = cudaMalloc(&d_out, sizeof(float2) * (size_t)n * grid);
        if (!e && sym) e = cudaMalloc(&d_scr, sizeof(float2) * (size_t)vpm::rollout_rev_slots(VPM_FP32, n) * grid);
        if (!e) e = cudaMemcpy(d_src, h.data(), sizeof(float4) * n, cudaMemcpyHostToDevice);
        for (int pass = 0; pass < 2 && !e; ++pass) {
            if (pass == 1) cudaEventRecord(t.a);
            e = sym ? vpm::launch_pair_probe_sym(grid, n, pass ? reps : 1, 0.05, d_src, d_out, d_scr, 0)
                    : vpm::launch_pair_probe(tpl, grid, n, pass ? reps : 1, 0.05, d_src, d_out, 0);
            if (pass == 1) cudaEventRecord(t.b);
        }
        if (!e) e = cudaEventSynchronize(t.b);
        if (!e) e = cudaEventElapsedTime(&ms, t.a, t.b);
        cudaFree(d_src);
        cudaFree(d_out);
        cudaFree(d_scr);
        work = (double)grid * reps * (double)n * n;
    }
    if (e) {
        snprintf(msg, sizeof msg, "vpm_probe_rate: %s", cudaGetErrorString(e));
        return report_error(VPM_ERR_CUDA, msg);
    }
    *h_rate = ms > 0.f ? work / (ms * 1e-3) : 0.0;
    return VPM_OK;
}
