// Device-side building blocks of the VPM library: the parameter block every kernel receives,
// particle storage for the binary32 and binary64 paths, and compensated arithmetic.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/vpm.h"

namespace vpm {

constexpr int kMaxB = 32;                 // largest N_b accepted by the library
constexpr int kMaxC = kMaxB + 1;          // collocation points
constexpr int kMaxS = kMaxB + 2;          // surface unknowns (bound + LEV + TEV)
constexpr int kThreads = 128;             // threads of a rollout block on the default path
constexpr int kMaxWarps = 16;             // largest rollout block: 512 threads
constexpr double kInv2Pi = 0.15915494309189533577;

// Device status bits of a rollout launch (latched in the state's status word).
enum Status : int { kStOk = 0, kStNonFinite = 1, kStCapacity = 2 };

// Everything a rollout kernel needs to know about the model, prepared on the host.
struct DevParams {
    int n_b, n_c;
    int kernel;            // vpm_kernel of wake and shed vortices
    int shed_gate;
    int n_wake_max;
    int fixed_plate;
    double chord, lb, span, rho;
    double r_core, rc4, inv_rc2;   // r_core^4 (Vatistas), 1/r_core^2 (Gaussian)
    double shed_dist;      // delta_s (absolute)
    double decay;          // exp(-gamma dt)
    double alpha_crit;
    double u_inf_x, u_inf_z;
    double dt;
    double mass, inertia, g, l, l_w, l_e, s_e;
    double inv_dt, inv_lb, inv_mass, inv_inertia;   // reciprocals: no divisions on the plate path
    double q[7], x_d[7];
    // Inverses of the body-frame surface matrix (Eq. 8) for the four shedding variants,
    // index (lev * 2 + tev); each is m x m row-major with m = n_b + lev + tev, stored with a
    // row stride of kMaxS.
    const double *kinv;
};

// ------------------------------------------------------------------ compensated arithmetic

// Error-free sum a + b = s + e (Knuth's TwoSum, six additions, no magnitude condition).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    float bp = s - a;
    float ap = s - bp;
    e = (a - ap) + (b - bp);
}

// Kahan compensated accumulation of one term into (sum, comp).
__device__ __forceinline__ void kahan_add(float &sum, float &comp, float x)
{
    float y = x - comp;
    float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

// ------------------------------------------------------------------ particle storage

// Binary32 path: (x_hi, z_hi, Gamma, lo) where lo packs the bfloat16 residues of x and z so
// that x = x_hi + x_lo to about 34 significant bits. The pair sums read x_hi and z_hi only.
__device__ __forceinline__ float pack_lo(float xl, float zl)
{
    __nv_bfloat16 a = __float2bfloat16_rn(xl), b = __float2bfloat16_rn(zl);
    uint32_t u = (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
    return __uint_as_float(u);
}

__device__ __forceinline__ void unpack_lo(float w, float &xl, float &zl)
{
    uint32_t u = __float_as_uint(w);
    xl = __bfloat162float(__ushort_as_bfloat16((unsigned short)(u & 0xffffu)));
    zl = __bfloat162float(__ushort_as_bfloat16((unsigned short)(u >> 16)));
}

__device__ __forceinline__ float4 make_part_f32(double x, double z, float g)
{
    float xh = (float)x, zh = (float)z;
    float xl = (float)(x - (double)xh), zl = (float)(z - (double)zh);
    return make_float4(xh, zh, g, pack_lo(xl, zl));
}

__device__ __forceinline__ void part_xz(const float4 &p, double &x, double &z)
{
    float xl, zl;
    unpack_lo(p.w, xl, zl);
    x = (double)p.x + (double)xl;
    z = (double)p.y + (double)zl;
}

// Binary64 path.
struct alignas(16) Part64 {
    double x, z, g, pad;
};

__device__ __forceinline__ Part64 make_part_f64(double x, double z, double g)
{
    Part64 p;
    p.x = x; p.z = z; p.g = g; p.pad = 0.0;
    return p;
}

// Record type, velocity type and accessors of each path. On the binary32 path a float4 record
// is (x_hi, z_hi, Gamma, lo): Gamma is the record's third component.
template <class R> struct Store;
template <> struct Store<float> {
    using P = float4;
    using V = float2;
    __device__ static P make(double x, double z, double g) { return make_part_f32(x, z, (float)g); }
    __device__ static void xz(const P &p, double &x, double &z) { part_xz(p, x, z); }
    __device__ static double gam(const P &p) { return (double)p.z; }
};
template <> struct Store<double> {
    using P = Part64;
    using V = double2;
    __device__ static P make(double x, double z, double g) { return make_part_f64(x, z, g); }
    __device__ static void xz(const P &p, double &x, double &z) { x = p.x; z = p.z; }
    __device__ static double gam(const P &p) { return p.g; }
};

// ------------------------------------------------------------------ pair kernels

// Velocity factor q such that the unit-circulation velocity at displacement (dx, dz) is
// q * (-dz, dx) / (2 pi), for each kernel of §III-A (Eqs. 4-5) and the Gaussian core.
template <int KER> struct PairF32;
template <> struct PairF32<VPM_KERNEL_VATISTAS> {
    // 1 / sqrt(r^4 + r_core^4): Eq. 4 times Eq. 5 simplifies to this; 0 displacement gives 0.
    __device__ __forceinline__ static float q(float r2, float rc4, float) {
        return rsqrtf(fmaf(r2, r2, rc4));
    }
};
template <> struct PairF32<VPM_KERNEL_GAUSSIAN> {
    __device__ __forceinline__ static float q(float r2, float, float inv_rc2) {
        float r2s = fmaxf(r2, 1e-30f);
        return -expm1f(-r2s * inv_rc2) / r2s;
    }
};
template <> struct PairF32<VPM_KERNEL_SINGULAR> {
    __device__ __forceinline__ static float q(float r2, float, float) {
        return r2 > 0.f ? 1.0f / r2 : 0.f;
    }
};

template <int KER> struct PairF64;
template <> struct PairF64<VPM_KERNEL_VATISTAS> {
    __device__ __forceinline__ static double q(double r2, double rc4, double) {
        return 1.0 / sqrt(fma(r2, r2, rc4));
    }
};
template <> struct PairF64<VPM_KERNEL_GAUSSIAN> {
    // Beyond r^2 / delta^2 = 50, e^(-r^2/delta^2) < 2e-22 and 1 - e^(-r^2/delta^2) is 1 to binary64
    // precision: the exponential (the costly part on a narrow FP64 pipe) is skipped there.
    __device__ __forceinline__ static double q(double r2, double, double inv_rc2) {
        const double x = r2 * inv_rc2;
        if (x >= 50.0) return 1.0 / r2;
        return r2 > 0.0 ? -expm1(-x) / r2 : 0.0;
    }
};
template <> struct PairF64<VPM_KERNEL_SINGULAR> {
    __device__ __forceinline__ static double q(double r2, double, double) {
        return r2 > 0.0 ? 1.0 / r2 : 0.0;
    }
};

}  // namespace vpm
