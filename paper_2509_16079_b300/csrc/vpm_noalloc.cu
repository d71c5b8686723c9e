// Free-field Heun stepping that allocates nothing.
//
// vpm_freefield_heun asks the stream-ordered allocator for its scratch on every call (24 n bytes
// plus the pair-sum slots of its one-evaluation-per-pair kernel). Some callers cannot let a
// library allocate: a real-time control loop whose memory is fixed up front (an allocation can
// stall or fail in the middle of a control period), or a host process that hands the GPU over
// to code that owns all device memory. For them this file keeps the scratch in one statically
// sized device array, which the device gives to the library when its device code is loaded
// (lazily by default: on the first call on that device), and vpm_freefield_heun_noalloc uses
// it instead of allocating; it evaluates every pair once per target, which needs only the
// 24 n bytes.
#include <stdio.h>

#include "vpm_device.cuh"

namespace vpm {
cudaError_t launch_freefield_heun(float *p, int n, int kernel, double r_core, double dt,
                                  int steps, float *scratch_mid, float *scratch_v1,
                                  cudaStream_t s);
vpm_status report_error(vpm_status st, const char *msg);
}  // namespace vpm

// Largest field the entry point accepts, and its scratch: stage positions (4 floats) and the
// first-stage velocity (2 floats) per particle, 6 MiB in all. Every device that loads the
// library holds this array until the process exits.
static constexpr int kNoAllocMaxN = 262144;
static __device__ __align__(256) float g_heun_scratch[(size_t)kNoAllocMaxN * 6];

// Device address of g_heun_scratch on the current device. In host code the array's name only
// stands in for the symbol; it is not a device pointer. The address is looked up on every call
// (cheap once the module is loaded) rather than cached, so that a device reset, after which
// the module is loaded again at a possibly different address, cannot leave a stale pointer.
static vpm_status scratch_for_current_device(float **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0) {
        cudaGetLastError();
        return vpm::report_error(VPM_ERR_CUDA, "vpm_freefield_heun_noalloc: no usable current CUDA device");
    }
    void *ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_heun_scratch);
    if (e != cudaSuccess || !ptr) {
        cudaGetLastError();
        char msg[256];
        snprintf(msg, sizeof msg, "vpm_freefield_heun_noalloc: cudaGetSymbolAddress failed: %s",
                 cudaGetErrorString(e));
        return vpm::report_error(VPM_ERR_CUDA, msg);
    }
    *out = static_cast<float *>(ptr);
    return VPM_OK;
}

extern "C" vpm_status vpm_freefield_heun_noalloc(float *d_particles, int n, int kernel,
                                                 double r_core, double dt, int steps,
                                                 cudaStream_t stream)
{
    if (n < 0 || steps < 0 || (n > 0 && !d_particles) || !isfinite(dt))
        return vpm::report_error(VPM_ERR_INVALID, "vpm_freefield_heun_noalloc: bad arguments");
    if (kernel < 0 || kernel > 2 || (kernel != VPM_KERNEL_SINGULAR && !(r_core > 0)))
        return vpm::report_error(VPM_ERR_INVALID, "vpm_freefield_heun_noalloc: bad kernel or core radius");
    if (n > kNoAllocMaxN) {
        char msg[160];
        snprintf(msg, sizeof msg,
                 "vpm_freefield_heun_noalloc: n = %d exceeds the fixed scratch limit of %d particles "
                 "(use vpm_freefield_heun)", n, kNoAllocMaxN);
        return vpm::report_error(VPM_ERR_CAPACITY, msg);
    }
    if (n == 0 || steps == 0) return VPM_OK;
    float *scratch = nullptr;
    vpm_status st = scratch_for_current_device(&scratch);
    if (st != VPM_OK) return st;
    // Stage one of every step writes all n entries of both scratch parts before stage two
    // reads them, so nothing left by an earlier call is ever read and no clearing is needed.
    cudaError_t e = vpm::launch_freefield_heun(d_particles, n, kernel, r_core, dt, steps, scratch,
                                               scratch + (size_t)4 * n, stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        char msg[256];
        snprintf(msg, sizeof msg, "vpm_freefield_heun_noalloc: %s", cudaGetErrorString(e));
        return vpm::report_error(VPM_ERR_CUDA, msg);
    }
    return VPM_OK;
}
