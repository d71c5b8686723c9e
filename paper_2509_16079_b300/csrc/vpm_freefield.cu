// Free-field Biot-Savart velocities (Eq. 3 with the kernels of Eqs. 4-5) for large fields and
// their Heun time stepping. Each thread holds two targets in registers; a block stages source
// tiles in shared memory with coalesced float4 loads, every thread then reads each source by a
// broadcast shared-memory load. Plain binary32 sums within a tile are added into
// Kahan-compensated totals across tiles.
#include "vpm_device.cuh"

namespace vpm {

constexpr int kFfThreads = 256;
constexpr int kFfTile = 512;   // sources staged per tile (8 KB)

// Epilogue modes of one velocity evaluation.
enum FfMode : int {
    kFfVelocity = 0,   // vel = V(src)
    kFfHeunStage1 = 1, // vel = V(src); mid = src + dt vel
    kFfHeunStage2 = 2  // out = out + dt/2 (vel + V(src)), src being the stage-1 positions
};

struct FfArgs {
    const float4 *src;   // sources and targets (x, z, Gamma, unused)
    int n;
    float rc4, inv_rc2;
    float dt;
    float2 *vel;         // velocity mode and stage 1: output; stage 2: v1 input
    float4 *mid;         // stage 1 output
    float4 *out;         // stage 2 output (in place over the base positions)
};

template <int KER, int MODE>
__global__ void __launch_bounds__(kFfThreads) freefield_kernel(const FfArgs a)
{
    __shared__ float4 tile[kFfTile];
    const int ia = blockIdx.x * (2 * kFfThreads) + threadIdx.x;
    const int ib = ia + kFfThreads;
    const int n = a.n;
    const float4 pa = a.src[ia < n ? ia : 0];
    const float4 pb = a.src[ib < n ? ib : 0];
    float sua = 0.f, cua = 0.f, swa = 0.f, cwa = 0.f;
    float sub = 0.f, cub = 0.f, swb = 0.f, cwb = 0.f;
    for (int j0 = 0; j0 < n; j0 += kFfTile) {
        const int cnt = min(kFfTile, n - j0);
        __syncthreads();
        for (int t = threadIdx.x; t < cnt; t += kFfThreads) tile[t] = a.src[j0 + t];
        __syncthreads();
        float ua = 0.f, wa = 0.f, ub = 0.f, wb = 0.f;
#pragma unroll 8
        for (int j = 0; j < cnt; ++j) {
            const float4 s = tile[j];
            const float dxa = pa.x - s.x, dza = pa.y - s.y;
            const float dxb = pb.x - s.x, dzb = pb.y - s.y;
            const float ga = s.z * PairF32<KER>::q(fmaf(dxa, dxa, dza * dza), a.rc4, a.inv_rc2);
            const float gb = s.z * PairF32<KER>::q(fmaf(dxb, dxb, dzb * dzb), a.rc4, a.inv_rc2);
            ua = fmaf(-dza, ga, ua);
            wa = fmaf(dxa, ga, wa);
            ub = fmaf(-dzb, gb, ub);
            wb = fmaf(dxb, gb, wb);
        }
        kahan_add(sua, cua, ua);
        kahan_add(swa, cwa, wa);
        kahan_add(sub, cub, ub);
        kahan_add(swb, cwb, wb);
    }
    const float inv2pi = (float)kInv2Pi;
    const float va_u = (sua - cua) * inv2pi, va_w = (swa - cwa) * inv2pi;
    const float vb_u = (sub - cub) * inv2pi, vb_w = (swb - cwb) * inv2pi;
    if (MODE == kFfVelocity) {
        if (ia < n) a.vel[ia] = make_float2(va_u, va_w);
        if (ib < n) a.vel[ib] = make_float2(vb_u, vb_w);
    } else if (MODE == kFfHeunStage1) {
        if (ia < n) {
            a.vel[ia] = make_float2(va_u, va_w);
            a.mid[ia] = make_float4(fmaf(a.dt, va_u, pa.x), fmaf(a.dt, va_w, pa.y), pa.z, 0.f);
        }
        if (ib < n) {
            a.vel[ib] = make_float2(vb_u, vb_w);
            a.mid[ib] = make_float4(fmaf(a.dt, vb_u, pb.x), fmaf(a.dt, vb_w, pb.y), pb.z, 0.f);
        }
    } else {
        const float h = 0.5f * a.dt;
        if (ia < n) {
            const float2 v1 = a.vel[ia];
            float4 q = a.out[ia];
            q.x = fmaf(h, v1.x + va_u, q.x);
            q.y = fmaf(h, v1.y + va_w, q.y);
            a.out[ia] = q;
        }
        if (ib < n) {
            const float2 v1 = a.vel[ib];
            float4 q = a.out[ib];
            q.x = fmaf(h, v1.x + vb_u, q.x);
            q.y = fmaf(h, v1.y + vb_w, q.y);
            a.out[ib] = q;
        }
    }
}

template <int MODE>
static cudaError_t launch_mode(int kernel, const FfArgs &a, cudaStream_t s)
{
    const int grid = (a.n + 2 * kFfThreads - 1) / (2 * kFfThreads);
    if (grid == 0) return cudaSuccess;
    if (kernel == VPM_KERNEL_GAUSSIAN)
        freefield_kernel<VPM_KERNEL_GAUSSIAN, MODE><<<grid, kFfThreads, 0, s>>>(a);
    else if (kernel == VPM_KERNEL_SINGULAR)
        freefield_kernel<VPM_KERNEL_SINGULAR, MODE><<<grid, kFfThreads, 0, s>>>(a);
    else
        freefield_kernel<VPM_KERNEL_VATISTAS, MODE><<<grid, kFfThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_freefield_velocity(const float *p, int n, int kernel, double r_core,
                                      float *vel, cudaStream_t s)
{
    FfArgs a{};
    a.src = reinterpret_cast<const float4 *>(p);
    a.n = n;
    a.rc4 = (float)(r_core * r_core * r_core * r_core);
    a.inv_rc2 = r_core > 0 ? (float)(1.0 / (r_core * r_core)) : 0.f;
    a.vel = reinterpret_cast<float2 *>(vel);
    return launch_mode<kFfVelocity>(kernel, a, s);
}

// Heun steps with caller-provided scratch: mid[n] float4 and v1[n] float2.
cudaError_t launch_freefield_heun(float *p, int n, int kernel, double r_core, double dt,
                                  int steps, float *scratch_mid, float *scratch_v1,
                                  cudaStream_t s)
{
    FfArgs a{};
    a.n = n;
    a.rc4 = (float)(r_core * r_core * r_core * r_core);
    a.inv_rc2 = r_core > 0 ? (float)(1.0 / (r_core * r_core)) : 0.f;
    a.dt = (float)dt;
    a.vel = reinterpret_cast<float2 *>(scratch_v1);
    a.mid = reinterpret_cast<float4 *>(scratch_mid);
    a.out = reinterpret_cast<float4 *>(p);
    for (int k = 0; k < steps; ++k) {
        a.src = reinterpret_cast<const float4 *>(p);
        cudaError_t e = launch_mode<kFfHeunStage1>(kernel, a, s);
        if (e != cudaSuccess) return e;
        a.src = a.mid;
        e = launch_mode<kFfHeunStage2>(kernel, a, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace vpm
