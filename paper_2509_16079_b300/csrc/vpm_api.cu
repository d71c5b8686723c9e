// Host side of the C ABI declared in include/vpm.h: argument checks, the body-frame surface
// matrix inverse, resident state management, and kernel launches.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <string>

#include "vpm_rollout.cuh"
#include "vpm_trace.cuh"

namespace vpm {
cudaError_t launch_mppi_weights(const float *J, int K, double lambda, float *w, cudaStream_t s);
cudaError_t launch_mppi_update(const float *w, const float *xi, int K, int H, float *mu,
                               cudaStream_t s);
cudaError_t launch_mppi_perturb(const float *mu, const float *eps, int K, int H, float *out,
                                cudaStream_t s);
cudaError_t launch_freefield_heun(float *p, int n, int kernel, double r_core, double dt,
                                  int steps, float *scratch_mid, float *scratch_v1,
                                  cudaStream_t s);
size_t freefield_sym_scratch_bytes(int n);
int freefield_sym_max_n();
cudaError_t launch_freefield_sym_velocity(const float *p, int n, int kernel, double r_core,
                                          float *vel, void *scratch, cudaStream_t s);
cudaError_t launch_freefield_sym_heun(float *p, int n, int kernel, double r_core, double dt,
                                      int steps, float *scratch_mid, float *scratch_v1,
                                      void *scratch, cudaStream_t s);
}  // namespace vpm

using namespace vpm;

static thread_local std::string g_last_error;

namespace vpm {
// Records a failure message for vpm_last_error() from other translation units of the library.
vpm_status report_error(vpm_status st, const char *msg)
{
    g_last_error = msg;
    return st;
}
}  // namespace vpm

static vpm_status fail(vpm_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

static vpm_status cuda_fail(cudaError_t e, const char *what)
{
    cudaGetLastError();  // clear a non-sticky launch error of this thread
    return fail(VPM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CUDA_TRY(call, what)                                   \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);     \
    } while (0)

struct vpm_state {
    vpm_params params;
    DevParams dp;
    int capacity;
    int n_upper;          // host-side upper bound of the resident count
    int pair_slots;       // 2 once a disturbance pair was injected (kept after its termination)
    int device;
    size_t rec_bytes;     // bytes of one particle record
    void *d_part;
    int *d_n;
    double *d_glider;     // 7
    double *d_hist;       // kMaxB + 2
    double *d_kinv;       // 4 x kMaxS x kMaxS
    int *d_status;
};

extern "C" const char *vpm_last_error(void) { return g_last_error.c_str(); }
extern "C" const char *vpm_version(void) { return "vpm-b300 1.0 (sm_103a)"; }

// ------------------------------------------------------------------ parameters

static bool finite_all(const double *v, int n)
{
    for (int i = 0; i < n; ++i)
        if (!isfinite(v[i])) return false;
    return true;
}

static vpm_status check_params(const vpm_params *p)
{
    if (!p) return fail(VPM_ERR_INVALID, "params is null");
    if (p->n_b < 2 || p->n_b > kMaxB) return fail(VPM_ERR_INVALID, "n_b must be in [2, %d]", kMaxB);
    double scal[] = {p->chord, p->span, p->rho, p->r_core, p->shed_offset, p->gamma_decay,
                     p->alpha_crit, p->u_inf[0], p->u_inf[1], p->dt, p->mass, p->inertia,
                     p->g, p->l, p->l_w, p->l_e, p->s_e};
    if (!finite_all(scal, (int)(sizeof scal / sizeof scal[0])) || !finite_all(p->q, 7) ||
        !finite_all(p->x_d, 7))
        return fail(VPM_ERR_INVALID, "non-finite parameter");
    if (p->chord <= 0 || p->dt <= 0 || p->mass <= 0 || p->inertia <= 0)
        return fail(VPM_ERR_INVALID, "chord, dt, mass and inertia must be positive");
    if (p->wake_kernel < 0 || p->wake_kernel > 2) return fail(VPM_ERR_INVALID, "bad wake_kernel");
    if (p->wake_kernel != VPM_KERNEL_SINGULAR && p->r_core <= 0)
        return fail(VPM_ERR_INVALID, "r_core must be positive for a regularised kernel");
    if (p->shed_gate < 0 || p->shed_gate > 2) return fail(VPM_ERR_INVALID, "bad shed_gate");
    if (p->precision != VPM_FP32 && p->precision != VPM_FP64)
        return fail(VPM_ERR_INVALID, "bad precision");
    if (p->n_wake_max < 0) return fail(VPM_ERR_INVALID, "n_wake_max must be >= 0");
    return VPM_OK;
}

// Core factor f(r) of the wake kernel: Eq. 5 (Vatistas n = 2), the Gaussian core, or 1.
static double core_factor(int kernel, double r, double rc)
{
    if (kernel == VPM_KERNEL_VATISTAS) return r * r / sqrt(rc * rc * rc * rc + r * r * r * r);
    if (kernel == VPM_KERNEL_GAUSSIAN) return -expm1(-(r * r) / (rc * rc));
    return 1.0;
}

// In the body frame every plate point is s e_t, and the unit-circulation velocity of a vortex
// at sigma e_t, dotted with e_n, is -f(|s - sigma|) / (2 pi (s - sigma)) because
// e_z x e_t = -e_n. The matrix of Eq. 8 therefore does not depend on the plate's pose.
static double influence(int kernel, double rc, double s, double sigma)
{
    double d = s - sigma;
    return -core_factor(kernel, fabs(d), rc) / (2.0 * M_PI * d);
}

// Gauss-Jordan inversion with partial pivoting of an m x m matrix (row stride ld).
static bool invert(int m, const double *A, int ld, double *Ainv)
{
    double W[kMaxS][2 * kMaxS];
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < 2 * m; ++j)
            W[i][j] = j < m ? A[i * ld + j] : (j - m == i ? 1.0 : 0.0);
    for (int c = 0; c < m; ++c) {
        int piv = c;
        for (int r = c + 1; r < m; ++r)
            if (fabs(W[r][c]) > fabs(W[piv][c])) piv = r;
        if (W[piv][c] == 0.0) return false;
        if (piv != c)
            for (int j = 0; j < 2 * m; ++j) { double t = W[c][j]; W[c][j] = W[piv][j]; W[piv][j] = t; }
        double d = W[c][c];
        for (int j = 0; j < 2 * m; ++j) W[c][j] /= d;
        for (int r = 0; r < m; ++r) {
            if (r == c || W[r][c] == 0.0) continue;
            double f = W[r][c];
            for (int j = 0; j < 2 * m; ++j) W[r][j] -= f * W[c][j];
        }
    }
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) Ainv[i * ld + j] = W[i][m + j];
    return true;
}

// Inverses of the surface system for the four shedding variants (lev, tev).
static vpm_status surface_inverses(const vpm_params *p, double *kinv)
{
    const int nb = p->n_b, nc = nb + 1;
    const double c = p->chord, lb = c / nb, ds = p->shed_offset * c;
    memset(kinv, 0, sizeof(double) * 4 * kMaxS * kMaxS);
    for (int lev = 0; lev < 2; ++lev)
        for (int tev = 0; tev < 2; ++tev) {
            const int m = nb + lev + tev;
            double A[kMaxS * kMaxS];
            int r = 0;
            for (int i = 0; i < nc; ++i) {
                if ((i == 0 && !lev) || (i == nc - 1 && !tev)) continue;
                const double s = -0.5 * c + i * lb;
                int col = 0;
                for (int j = 0; j < nb; ++j)
                    A[r * kMaxS + col++] = influence(VPM_KERNEL_SINGULAR, 0.0, s, -0.5 * c + (j + 0.5) * lb);
                if (lev) A[r * kMaxS + col++] = influence(p->wake_kernel, p->r_core, s, -0.5 * c - ds);
                if (tev) A[r * kMaxS + col++] = influence(p->wake_kernel, p->r_core, s, 0.5 * c + ds);
                ++r;
            }
            for (int j = 0; j < m; ++j) A[r * kMaxS + j] = 1.0;   // Kelvin's row (Eq. 7)
            if (!invert(m, A, kMaxS, kinv + (size_t)(lev * 2 + tev) * kMaxS * kMaxS))
                return fail(VPM_ERR_SINGULAR, "surface system singular (lev=%d, tev=%d)", lev, tev);
        }
    return VPM_OK;
}

static void fill_dev_params(const vpm_params *p, DevParams &d)
{
    memset(&d, 0, sizeof d);
    d.n_b = p->n_b;
    d.n_c = p->n_b + 1;
    d.kernel = p->wake_kernel;
    d.shed_gate = p->shed_gate;
    d.n_wake_max = p->n_wake_max;
    d.fixed_plate = p->fixed_plate;
    d.chord = p->chord;
    d.lb = p->chord / p->n_b;
    d.inv_lb = p->n_b / p->chord;
    d.inv_dt = 1.0 / p->dt;
    d.inv_mass = 1.0 / p->mass;
    d.inv_inertia = 1.0 / p->inertia;
    d.span = p->span;
    d.rho = p->rho;
    d.r_core = p->r_core;
    d.rc4 = p->r_core * p->r_core * p->r_core * p->r_core;
    d.inv_rc2 = p->r_core > 0 ? 1.0 / (p->r_core * p->r_core) : 0.0;
    d.shed_dist = p->shed_offset * p->chord;
    d.decay = exp(-p->gamma_decay * p->dt);
    d.alpha_crit = p->alpha_crit;
    d.u_inf_x = p->u_inf[0];
    d.u_inf_z = p->u_inf[1];
    d.dt = p->dt;
    d.mass = p->mass; d.inertia = p->inertia; d.g = p->g;
    d.l = p->l; d.l_w = p->l_w; d.l_e = p->l_e; d.s_e = p->s_e;
    for (int i = 0; i < 7; ++i) { d.q[i] = p->q[i]; d.x_d[i] = p->x_d[i]; }
}

static vpm_status require_device(int *dev)
{
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || count == 0) {
        cudaGetLastError();
        return fail(VPM_ERR_CUDA, "no CUDA device available (%s)",
                    e == cudaSuccess ? "device count is 0" : cudaGetErrorString(e));
    }
    CUDA_TRY(cudaGetDevice(dev), "cudaGetDevice");
    return VPM_OK;
}

// ------------------------------------------------------------------ host packing of records

// Round-to-nearest-even binary32 -> bfloat16 bits (finite inputs).
static uint16_t host_bf16(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
    return (uint16_t)(u >> 16);
}

static float host_from_bf16(uint16_t h)
{
    uint32_t u = (uint32_t)h << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

static void pack_records(int precision, const double *h, int n, void *out)
{
    if (precision == VPM_FP64) {
        Part64 *o = static_cast<Part64 *>(out);
        for (int i = 0; i < n; ++i) { o[i].x = h[3 * i]; o[i].z = h[3 * i + 1]; o[i].g = h[3 * i + 2]; o[i].pad = 0; }
        return;
    }
    float4 *o = static_cast<float4 *>(out);
    for (int i = 0; i < n; ++i) {
        double x = h[3 * i], z = h[3 * i + 1];
        float xh = (float)x, zh = (float)z;
        float xl = (float)(x - (double)xh), zl = (float)(z - (double)zh);
        uint32_t w = (uint32_t)host_bf16(xl) | ((uint32_t)host_bf16(zl) << 16);
        float wf;
        memcpy(&wf, &w, 4);
        o[i] = make_float4(xh, zh, (float)h[3 * i + 2], wf);
    }
}

static void unpack_records(int precision, const void *in, int n, double *h)
{
    if (precision == VPM_FP64) {
        const Part64 *o = static_cast<const Part64 *>(in);
        for (int i = 0; i < n; ++i) { h[3 * i] = o[i].x; h[3 * i + 1] = o[i].z; h[3 * i + 2] = o[i].g; }
        return;
    }
    const float4 *o = static_cast<const float4 *>(in);
    for (int i = 0; i < n; ++i) {
        uint32_t w;
        memcpy(&w, &o[i].w, 4);
        h[3 * i] = (double)o[i].x + (double)host_from_bf16((uint16_t)(w & 0xffffu));
        h[3 * i + 1] = (double)o[i].y + (double)host_from_bf16((uint16_t)(w >> 16));
        h[3 * i + 2] = (double)o[i].z;
    }
}

// Entry points for the batch code in vpm_batch.cu.
namespace vpm {
vpm_status check_params_ext(const vpm_params *p) { return check_params(p); }
vpm_status surface_inverses_ext(const vpm_params *p, double *kinv) { return surface_inverses(p, kinv); }
void fill_dev_params_ext(const vpm_params *p, DevParams &d) { fill_dev_params(p, d); }
void pack_records_ext(int precision, const double *h, int n, void *out) { pack_records(precision, h, n, out); }
}  // namespace vpm

// ------------------------------------------------------------------ state

static size_t max_smem_optin()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        return 227 * 1024;
    }
    return (size_t)v;
}

// Static shared memory of the rollout kernel (workspace), kept out of the dynamic budget.
static size_t static_smem_reserve() { return 4 * 1024; }

extern "C" vpm_status vpm_state_create(const vpm_params *params, const double *h_particles,
                                       int n, int capacity, const double *h_glider7,
                                       vpm_state **out, cudaStream_t stream)
{
    vpm_status st = check_params(params);
    if (st) return st;
    if (!out || !h_glider7 || (n > 0 && !h_particles))
        return fail(VPM_ERR_INVALID, "null argument");
    if (n < 0 || capacity < n || capacity < 1)
        return fail(VPM_ERR_INVALID, "need 0 <= n <= capacity and capacity >= 1");
    if (!finite_all(h_glider7, 7) || (n > 0 && !finite_all(h_particles, 3 * n)))
        return fail(VPM_ERR_NONFINITE, "non-finite particle or glider value");
    int dev;
    if ((st = require_device(&dev))) return st;
    if (rollout_smem_bytes(params->precision, capacity) + static_smem_reserve() > max_smem_optin())
        return fail(VPM_ERR_CAPACITY, "capacity %d does not fit one block's shared memory", capacity);
    vpm_state *s = new vpm_state();
    s->params = *params;
    s->capacity = capacity;
    s->n_upper = n;
    s->device = dev;
    s->rec_bytes = params->precision == VPM_FP64 ? sizeof(Part64) : sizeof(float4);
    fill_dev_params(params, s->dp);
    double *kinv = (double *)malloc(sizeof(double) * 4 * kMaxS * kMaxS);
    if ((st = surface_inverses(params, kinv))) { free(kinv); delete s; return st; }
    void *host_rec = malloc(s->rec_bytes * (size_t)(n > 0 ? n : 1));
    pack_records(params->precision, h_particles, n, host_rec);
    double hist[kMaxB + 2] = {0};
    cudaError_t e = cudaSuccess;
    if ((e = cudaMalloc(&s->d_part, s->rec_bytes * capacity)) != cudaSuccess ||
        (e = cudaMalloc(&s->d_n, sizeof(int) * 2)) != cudaSuccess ||
        (e = cudaMalloc(&s->d_glider, sizeof(double) * 7)) != cudaSuccess ||
        (e = cudaMalloc(&s->d_hist, sizeof(double) * (kMaxB + 2))) != cudaSuccess ||
        (e = cudaMalloc(&s->d_kinv, sizeof(double) * 4 * kMaxS * kMaxS)) != cudaSuccess ||
        (e = cudaMalloc(&s->d_status, sizeof(int))) != cudaSuccess) {
        free(kinv); free(host_rec);
        cudaGetLastError();
        vpm_state_destroy(s);
        return fail(VPM_ERR_OOM, "cudaMalloc: %s", cudaGetErrorString(e));
    }
    s->dp.kinv = s->d_kinv;
    e = cudaMemcpyAsync(s->d_part, host_rec, s->rec_bytes * n, cudaMemcpyHostToDevice, stream);
    const int n_pair[2] = {n, 0};         // count, disturbance pair count
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_n, n_pair, sizeof n_pair, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_glider, h_glider7, sizeof(double) * 7, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_hist, hist, sizeof hist, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_kinv, kinv, sizeof(double) * 4 * kMaxS * kMaxS, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d_status, 0, sizeof(int), stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    free(kinv);
    free(host_rec);
    if (e != cudaSuccess) {
        vpm_state_destroy(s);
        return cuda_fail(e, "vpm_state_create upload");
    }
    *out = s;
    return VPM_OK;
}

extern "C" vpm_status vpm_state_destroy(vpm_state *s)
{
    if (!s) return VPM_OK;
    cudaDeviceSynchronize();
    cudaFree(s->d_part); cudaFree(s->d_n); cudaFree(s->d_glider); cudaFree(s->d_hist);
    cudaFree(s->d_kinv); cudaFree(s->d_status);
    cudaGetLastError();
    delete s;
    return VPM_OK;
}

extern "C" vpm_status vpm_state_set_history(vpm_state *s, const double *h_gb_prev,
                                            double glev_prev, int has_prev, cudaStream_t stream)
{
    if (!s || (has_prev && !h_gb_prev)) return fail(VPM_ERR_INVALID, "null argument");
    double hist[kMaxB + 2] = {0};
    for (int j = 0; j < s->params.n_b; ++j) hist[j] = h_gb_prev ? h_gb_prev[j] : 0.0;
    hist[s->params.n_b] = glev_prev;
    hist[s->params.n_b + 1] = has_prev ? 1.0 : 0.0;
    CUDA_TRY(cudaMemcpyAsync(s->d_hist, hist, sizeof hist, cudaMemcpyHostToDevice, stream), "set_history");
    CUDA_TRY(cudaStreamSynchronize(stream), "set_history sync");
    return VPM_OK;
}

extern "C" vpm_status vpm_state_set_glider(vpm_state *s, const double *h_x7, cudaStream_t stream)
{
    if (!s || !h_x7) return fail(VPM_ERR_INVALID, "null argument");
    if (!finite_all(h_x7, 7)) return fail(VPM_ERR_NONFINITE, "non-finite glider state");
    CUDA_TRY(cudaMemcpyAsync(s->d_glider, h_x7, sizeof(double) * 7, cudaMemcpyHostToDevice, stream), "set_glider");
    CUDA_TRY(cudaStreamSynchronize(stream), "set_glider sync");
    return VPM_OK;
}

extern "C" vpm_status vpm_state_get_glider(const vpm_state *s, double *h_x7, cudaStream_t stream)
{
    if (!s || !h_x7) return fail(VPM_ERR_INVALID, "null argument");
    CUDA_TRY(cudaMemcpyAsync(h_x7, s->d_glider, sizeof(double) * 7, cudaMemcpyDeviceToHost, stream), "get_glider");
    CUDA_TRY(cudaStreamSynchronize(stream), "get_glider sync");
    return VPM_OK;
}

extern "C" vpm_status vpm_state_copy(vpm_state *dst, const vpm_state *src, cudaStream_t stream)
{
    if (!dst || !src) return fail(VPM_ERR_INVALID, "null argument");
    if (dst == src) return VPM_OK;
    if (dst->params.precision != src->params.precision || dst->params.n_b != src->params.n_b ||
        dst->capacity < src->n_upper)
        return fail(VPM_ERR_INVALID, "states differ in precision or n_b, or the capacity is too small");
    CUDA_TRY(cudaMemcpyAsync(dst->d_part, src->d_part, src->rec_bytes * (size_t)src->capacity <
                             dst->rec_bytes * (size_t)dst->capacity ? src->rec_bytes * (size_t)src->capacity
                             : dst->rec_bytes * (size_t)dst->capacity,
                             cudaMemcpyDeviceToDevice, stream), "state copy");
    CUDA_TRY(cudaMemcpyAsync(dst->d_n, src->d_n, sizeof(int) * 2, cudaMemcpyDeviceToDevice, stream), "state copy");
    CUDA_TRY(cudaMemcpyAsync(dst->d_glider, src->d_glider, sizeof(double) * 7, cudaMemcpyDeviceToDevice, stream), "state copy");
    CUDA_TRY(cudaMemcpyAsync(dst->d_hist, src->d_hist, sizeof(double) * (kMaxB + 2), cudaMemcpyDeviceToDevice, stream), "state copy");
    dst->n_upper = src->n_upper;
    dst->pair_slots = src->pair_slots > dst->pair_slots ? src->pair_slots : dst->pair_slots;
    return VPM_OK;
}

extern "C" vpm_status vpm_state_inject_pair(vpm_state *s, const double *h_pair, cudaStream_t stream)
{
    if (!s || !h_pair) return fail(VPM_ERR_INVALID, "null argument");
    if (!finite_all(h_pair, 6)) return fail(VPM_ERR_NONFINITE, "non-finite disturbance pair");
    if (s->n_upper + 2 > s->capacity)
        return fail(VPM_ERR_CAPACITY, "no room for the pair: capacity %d", s->capacity);
    int cnt[2];
    CUDA_TRY(cudaMemcpyAsync(cnt, s->d_n, sizeof cnt, cudaMemcpyDeviceToHost, stream), "inject");
    CUDA_TRY(cudaStreamSynchronize(stream), "inject");
    if (cnt[1] != 0) return fail(VPM_ERR_INVALID, "a disturbance pair is already present");
    CUDA_TRY(launch_inject_pair(s->params.precision, s->d_part, s->d_n, s->capacity, h_pair, stream), "inject launch");
    s->n_upper += 2;
    s->pair_slots = 2;
    return VPM_OK;
}

extern "C" vpm_status vpm_state_disturbance(const vpm_state *s, int *h_n_dist, cudaStream_t stream)
{
    if (!s || !h_n_dist) return fail(VPM_ERR_INVALID, "null argument");
    CUDA_TRY(cudaMemcpyAsync(h_n_dist, s->d_n + 1, sizeof(int), cudaMemcpyDeviceToHost, stream), "disturbance");
    CUDA_TRY(cudaStreamSynchronize(stream), "disturbance");
    return VPM_OK;
}

static vpm_status take_status(vpm_state *s, cudaStream_t stream)
{
    int st = 0;
    CUDA_TRY(cudaMemcpyAsync(&st, s->d_status, sizeof(int), cudaMemcpyDeviceToHost, stream), "status read");
    CUDA_TRY(cudaStreamSynchronize(stream), "status sync");
    if (st) {
        CUDA_TRY(cudaMemsetAsync(s->d_status, 0, sizeof(int), stream), "status clear");
        CUDA_TRY(cudaStreamSynchronize(stream), "status clear sync");
        if (st & kStNonFinite) return fail(VPM_ERR_NONFINITE, "non-finite value in a rollout");
        return fail(VPM_ERR_CAPACITY, "device reported status %d", st);
    }
    return VPM_OK;
}

extern "C" vpm_status vpm_state_status(vpm_state *s, cudaStream_t stream)
{
    if (!s) return fail(VPM_ERR_INVALID, "null state");
    return take_status(s, stream);
}

extern "C" vpm_status vpm_state_read(const vpm_state *cs, double *h_particles, int *n_out,
                                     double *h_glider7, double *h_hist, cudaStream_t stream)
{
    vpm_state *s = const_cast<vpm_state *>(cs);
    if (!s || !h_particles || !n_out || !h_glider7) return fail(VPM_ERR_INVALID, "null argument");
    int n = 0;
    double hist[kMaxB + 2];
    void *rec = malloc(s->rec_bytes * s->capacity);
    cudaError_t e = cudaMemcpyAsync(&n, s->d_n, sizeof(int), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(rec, s->d_part, s->rec_bytes * s->capacity, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_glider7, s->d_glider, sizeof(double) * 7, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hist, s->d_hist, sizeof hist, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) { free(rec); return cuda_fail(e, "vpm_state_read"); }
    if (n < 0 || n > s->capacity) { free(rec); return fail(VPM_ERR_CAPACITY, "device count %d out of range", n); }
    unpack_records(s->params.precision, rec, n, h_particles);
    free(rec);
    *n_out = n;
    s->n_upper = n;
    if (h_hist)
        for (int j = 0; j < s->params.n_b + 2; ++j) h_hist[j] = hist[j];
    return take_status(s, stream);
}

// Serialised layout: header (magic, precision, n_b, capacity, n, glider, hist), then the
// capacity records of the particle array.
struct SaveHeader {
    uint32_t magic, precision, n_b, capacity;
    int32_t n, pad;          // count, disturbance pair count
    double glider[7];
    double hist[kMaxB + 2];
};
static const uint32_t kSaveMagic = 0x56504d31u;  // "VPM1"

extern "C" vpm_status vpm_state_save(const vpm_state *cs, void *h_buf, size_t *bytes,
                                     cudaStream_t stream)
{
    vpm_state *s = const_cast<vpm_state *>(cs);
    if (!s || !bytes) return fail(VPM_ERR_INVALID, "null argument");
    const size_t need = sizeof(SaveHeader) + s->rec_bytes * s->capacity;
    if (!h_buf) { *bytes = need; return VPM_OK; }
    if (*bytes < need) return fail(VPM_ERR_INVALID, "buffer of %zu bytes, need %zu", *bytes, need);
    SaveHeader h;
    memset(&h, 0, sizeof h);
    h.magic = kSaveMagic;
    h.precision = s->params.precision;
    h.n_b = s->params.n_b;
    h.capacity = s->capacity;
    char *dst = static_cast<char *>(h_buf);
    cudaError_t e = cudaMemcpyAsync(&h.n, s->d_n, sizeof(int) * 2, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.glider, s->d_glider, sizeof h.glider, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.hist, s->d_hist, sizeof h.hist, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst + sizeof h, s->d_part, s->rec_bytes * s->capacity, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "vpm_state_save");
    memcpy(dst, &h, sizeof h);
    *bytes = need;
    return VPM_OK;
}

extern "C" vpm_status vpm_state_load(vpm_state *s, const void *h_buf, size_t bytes,
                                     cudaStream_t stream)
{
    if (!s || !h_buf) return fail(VPM_ERR_INVALID, "null argument");
    SaveHeader h;
    if (bytes < sizeof h) return fail(VPM_ERR_INVALID, "buffer too small");
    memcpy(&h, h_buf, sizeof h);
    if (h.magic != kSaveMagic || h.precision != (uint32_t)s->params.precision ||
        h.n_b != (uint32_t)s->params.n_b || h.capacity != (uint32_t)s->capacity ||
        bytes < sizeof h + s->rec_bytes * s->capacity || h.n < 0 || h.n > s->capacity ||
        (h.pad != 0 && h.pad != 2))
        return fail(VPM_ERR_INVALID, "saved state does not match this state");
    const char *src = static_cast<const char *>(h_buf);
    CUDA_TRY(cudaMemcpyAsync(s->d_part, src + sizeof h, s->rec_bytes * s->capacity, cudaMemcpyHostToDevice, stream), "load records");
    CUDA_TRY(cudaMemcpyAsync(s->d_n, &h.n, sizeof(int) * 2, cudaMemcpyHostToDevice, stream), "load n");
    CUDA_TRY(cudaMemcpyAsync(s->d_glider, h.glider, sizeof h.glider, cudaMemcpyHostToDevice, stream), "load glider");
    CUDA_TRY(cudaMemcpyAsync(s->d_hist, h.hist, sizeof h.hist, cudaMemcpyHostToDevice, stream), "load hist");
    CUDA_TRY(cudaStreamSynchronize(stream), "load sync");
    s->n_upper = h.n;
    if (h.pad) s->pair_slots = 2;
    return VPM_OK;
}

// ------------------------------------------------------------------ stepping and rollouts

// Largest count a rollout of H steps can reach from the state's current upper bound. Merging
// holds the wake (the disturbance pair excluded) at n_wake_max after each step, and two records
// are appended before each merge.
static long long grown(const vpm_state *s, int H)
{
    long long n = (long long)s->n_upper + 2LL * H;
    if (s->params.n_wake_max > 0) {
        const long long lim = (long long)s->params.n_wake_max + s->pair_slots;
        long long cap = (lim > s->n_upper ? lim : s->n_upper) + 2;
        if (n > cap) n = cap;
    }
    return n;
}

// Upper bound of the count after `steps` committed steps (merging done).
static int after_steps(const vpm_state *s, int steps)
{
    long long g = (long long)s->n_upper + 2LL * steps;
    if (s->params.n_wake_max > 0) {
        const long long lim = (long long)s->params.n_wake_max + s->pair_slots;
        if (g > lim) g = lim > s->n_upper ? lim : s->n_upper;
    }
    return (int)g;
}

// Device bytes of the binary32 pair-sum scratch that a batch of K rollouts of H steps, taken
// after `advance` more committed steps, allocates while it runs (the serving loop's admission).
namespace vpm {
size_t rollout_scratch_bytes(const vpm_state *s, int K, int H, int advance)
{
    long long cap = grown(s, H + advance);
    if (cap > s->capacity) cap = s->capacity;
    return sizeof(float2) * (size_t)K * (size_t)rollout_rev_slots(s->params.precision, (int)cap);
}

// Pair interactions of K rollouts of H steps taken after `advance` more committed steps,
// estimated from the host's count bound at mid-horizon: K H n^2 (the serving loop's
// least-work-first admission).
double rollout_work_estimate(const vpm_state *s, int K, int H, int advance)
{
    long long n = grown(s, advance + H / 2);
    if (n > s->capacity) n = s->capacity;
    return (double)K * (double)H * (double)n * (double)n;
}
}  // namespace vpm

extern "C" vpm_status vpm_rollout_scratch_bytes_cap(int precision, int capacity, int K, size_t *bytes)
{
    if (!bytes || K < 1 || capacity < 0 || (precision != VPM_FP32 && precision != VPM_FP64))
        return fail(VPM_ERR_INVALID, "vpm_rollout_scratch_bytes_cap: null, K < 1, capacity < 0 or bad precision");
    *bytes = sizeof(float2) * (size_t)K * (size_t)rollout_rev_slots(precision, capacity);
    return VPM_OK;
}

extern "C" vpm_status vpm_rollout_scratch_slot(int capacity, int kind, int row, int particle,
                                               long long *slot)
{
    const int rows = (capacity + 127) / 128;
    const bool ok = slot && capacity > 0 && particle >= 0 && particle < capacity &&
                    ((kind == 0 && particle < 128 * (rows - 1)) ||
                     (kind == 1 && row >= 0 && row < rows - 1 && particle >= 128 * (row + 1)));
    if (!ok) return fail(VPM_ERR_INVALID, "vpm_rollout_scratch_slot: no such slot");
    *slot = rollout_scratch_slot(capacity, kind, row, particle);
    return VPM_OK;
}

extern "C" vpm_status vpm_rollout_scratch_bytes(const vpm_state *s, int K, int H, size_t *bytes)
{
    if (!s || !bytes || K < 1 || H < 1) return fail(VPM_ERR_INVALID, "vpm_rollout_scratch_bytes: null or K, H < 1");
    *bytes = vpm::rollout_scratch_bytes(s, K, H, 0);
    return VPM_OK;
}

static void base_args(const vpm_state *s, RolloutArgs &a)
{
    memset(&a, 0, sizeof a);
    a.p = s->dp;
    a.root_part = s->d_part;
    a.root_n = s->d_n;
    a.root_ndist = s->d_n + 1;
    a.root_glider = s->d_glider;
    a.root_hist = s->d_hist;
    a.status = s->d_status;
}

extern "C" vpm_status vpm_step(vpm_state *s, double u, double *d_fm, double *d_gamma_s,
                               double *d_vel, double *d_vtilde, cudaStream_t stream)
{
    vpm::TraceRange tr("vpm_step");
    if (!s) return fail(VPM_ERR_INVALID, "null state");
    if (!isfinite(u)) return fail(VPM_ERR_INVALID, "non-finite control");
    if (grown(s, 1) > s->capacity)
        return fail(VPM_ERR_CAPACITY, "step would exceed capacity %d", s->capacity);
    RolloutArgs a;
    base_args(s, a);
    a.H = 1; a.K = 1; a.cap = s->capacity;
    a.u_const = u;
    a.out_part = s->d_part; a.out_n = s->d_n; a.out_glider = s->d_glider; a.out_hist = s->d_hist;
    a.out_ndist = s->d_n + 1;
    a.probe_fm = d_fm; a.probe_gs = d_gamma_s; a.probe_vel = d_vel; a.probe_vt = d_vtilde;
    cudaError_t e = launch_rollout(s->params.precision, a, 1, stream);
    if (e != cudaSuccess) return cuda_fail(e, "vpm_step launch");
    s->n_upper = after_steps(s, 1);
    return VPM_OK;
}

static vpm_status rollout_batch(const vpm_state *s, int K, int H, const double *d_x0,
                                const float *d_controls, float *d_costs, double *d_final_glider,
                                double *d_traj, double *d_field, int *d_count, cudaStream_t stream)
{
    vpm::TraceRange tr("vpm_rollout_batch");
    if (!s || !d_controls || !d_costs) return fail(VPM_ERR_INVALID, "null argument");
    if (K < 1 || H < 1) return fail(VPM_ERR_INVALID, "K and H must be positive");
    const long long need = grown(s, H);
    if (need > s->capacity)
        return fail(VPM_ERR_CAPACITY, "rollout may reach %lld particles, capacity %d", need, s->capacity);
    RolloutArgs a;
    base_args(s, a);
    a.H = H; a.K = K;
    a.cap = (int)(need > 0 ? need : 1);
    a.x0 = d_x0;
    a.controls = d_controls; a.ctrl_stride = H;
    a.costs = d_costs; a.final_glider = d_final_glider; a.traj = d_traj;
    a.field = d_field; a.field_cap = s->capacity; a.count = d_count;
    cudaError_t e = launch_rollout(s->params.precision, a, K, stream);
    if (e != cudaSuccess) return cuda_fail(e, "vpm_rollout_batch launch");
    return VPM_OK;
}

extern "C" vpm_status vpm_rollout_batch(const vpm_state *s, int K, int H, const float *d_controls,
                                        float *d_costs, double *d_final_glider, double *d_traj,
                                        double *d_field, int *d_count, cudaStream_t stream)
{
    return rollout_batch(s, K, H, nullptr, d_controls, d_costs, d_final_glider, d_traj, d_field,
                         d_count, stream);
}

extern "C" vpm_status vpm_state_advance_policy(vpm_state *s, int steps, const double *d_gains,
                                                const double *d_xbar, const float *d_ubar,
                                                int offset, cudaStream_t stream)
{
    if (!s || !d_gains || !d_xbar || !d_ubar) return fail(VPM_ERR_INVALID, "null argument");
    if (steps < 0 || offset < 0) return fail(VPM_ERR_INVALID, "steps and offset must be >= 0");
    if (steps == 0) return VPM_OK;
    const long long need = grown(s, steps);
    if (need > s->capacity)
        return fail(VPM_ERR_CAPACITY, "advance may reach %lld particles, capacity %d", need, s->capacity);
    RolloutArgs a;
    base_args(s, a);
    a.H = steps; a.K = 1; a.cap = s->capacity;
    a.out_part = s->d_part; a.out_n = s->d_n; a.out_glider = s->d_glider; a.out_hist = s->d_hist;
    a.out_ndist = s->d_n + 1;
    a.pol_gains = d_gains; a.pol_xbar = d_xbar; a.pol_ubar = d_ubar; a.pol_offset = offset;
    cudaError_t e = launch_rollout(s->params.precision, a, 1, stream);
    if (e != cudaSuccess) return cuda_fail(e, "vpm_state_advance_policy launch");
    s->n_upper = after_steps(s, steps);
    return VPM_OK;
}

extern "C" vpm_status vpm_rollout_batch_policy(const vpm_state *s, int K, int H, const double *d_x0,
                                               const double *d_gains, const double *d_xbar,
                                               const float *d_ubar, int offset,
                                               const float *d_controls, float *d_costs,
                                               double *d_final_glider, double *d_traj,
                                               cudaStream_t stream)
{
    if (!s || !d_gains || !d_xbar || !d_ubar || !d_costs) return fail(VPM_ERR_INVALID, "null argument");
    if (K < 1 || H < 1 || offset < 0) return fail(VPM_ERR_INVALID, "K, H must be positive, offset >= 0");
    const long long need = grown(s, H);
    if (need > s->capacity)
        return fail(VPM_ERR_CAPACITY, "rollout may reach %lld particles, capacity %d", need, s->capacity);
    RolloutArgs a;
    base_args(s, a);
    a.H = H; a.K = K;
    a.cap = (int)(need > 0 ? need : 1);
    a.x0 = d_x0;
    a.controls = d_controls; a.ctrl_stride = H;
    a.pol_gains = d_gains; a.pol_xbar = d_xbar; a.pol_ubar = d_ubar; a.pol_offset = offset;
    a.costs = d_costs; a.final_glider = d_final_glider; a.traj = d_traj;
    cudaError_t e = launch_rollout(s->params.precision, a, K, stream);
    if (e != cudaSuccess) return cuda_fail(e, "vpm_rollout_batch_policy launch");
    return VPM_OK;
}

extern "C" vpm_status vpm_rollout_batch_x0(const vpm_state *s, int K, int H, const double *d_x0,
                                           const float *d_controls, float *d_costs,
                                           double *d_final_glider, double *d_traj,
                                           double *d_field, int *d_count, cudaStream_t stream)
{
    if (!d_x0) return fail(VPM_ERR_INVALID, "null initial states");
    return rollout_batch(s, K, H, d_x0, d_controls, d_costs, d_final_glider, d_traj, d_field,
                         d_count, stream);
}

// One-rollout-per-launch comparison form: the field of every rollout lives in global memory
// between launches; each launch advances one rollout by one step.
extern "C" vpm_status vpm_rollout_batch_per_launch(const vpm_state *s, int K, int H,
                                                   const float *d_controls, float *d_costs,
                                                   double *d_final_glider, cudaStream_t stream)
{
    if (!s || !d_controls || !d_costs) return fail(VPM_ERR_INVALID, "null argument");
    if (K < 1 || H < 1) return fail(VPM_ERR_INVALID, "K and H must be positive");
    const long long need = grown(s, H);
    if (need > s->capacity)
        return fail(VPM_ERR_CAPACITY, "rollout may reach %lld particles, capacity %d", need, s->capacity);
    const int cap = (int)(need > 0 ? need : 1);
    const size_t rec = s->rec_bytes;
    const int stride = kMaxB + 2;
    void *parts = nullptr;
    int *ns = nullptr;
    double *gl = nullptr, *hi = nullptr;
    CUDA_TRY(lib_malloc_async(&parts, rec * (size_t)cap * K, stream), "per-launch scratch");
    CUDA_TRY(lib_malloc_async((void **)&ns, sizeof(int) * 2 * K, stream), "per-launch scratch");
    CUDA_TRY(lib_malloc_async((void **)&gl, sizeof(double) * stride * K, stream), "per-launch scratch");
    CUDA_TRY(lib_malloc_async((void **)&hi, sizeof(double) * stride * K, stream), "per-launch scratch");
    // pair-sum scratch of the one block every launch runs, allocated once for all launches
    const long long rev_slots = rollout_rev_slots(s->params.precision, cap);
    float2 *rev = nullptr;
    if (rev_slots > 0)
        CUDA_TRY(lib_malloc_async((void **)&rev, sizeof(float2) * (size_t)rev_slots, stream), "per-launch scratch");
    // replicate the root into every rollout's slot (a zero-step launch of the rollout kernel)
    RolloutArgs a;
    base_args(s, a);
    a.H = 0; a.K = K; a.cap = cap;
    a.out_stride = cap; a.out_state_stride = stride;
    a.out_part = parts; a.out_n = ns; a.out_glider = gl; a.out_hist = hi;
    a.out_ndist = ns + K;
    cudaError_t e = launch_rollout(s->params.precision, a, K, stream);
    // then every step of every rollout is its own launch, state in global memory in between
    a.root_part = parts; a.root_n = ns; a.root_glider = gl; a.root_hist = hi;
    a.root_ndist = ns + K;
    a.root_stride = cap; a.state_stride = stride;
    a.H = 1;
    a.controls = d_controls; a.ctrl_stride = H;
    a.costs = d_costs;
    a.rev = rev; a.rev_stride = rev_slots;
    for (int k = 0; k < H && e == cudaSuccess; ++k) {
        a.step0 = k;
        for (int i = 0; i < K && e == cudaSuccess; ++i) {
            a.rid0 = i;
            e = launch_rollout(s->params.precision, a, 1, stream);
        }
    }
    if (e == cudaSuccess && d_final_glider) {
        for (int i = 0; i < K && e == cudaSuccess; ++i)
            e = cudaMemcpyAsync(d_final_glider + 7 * i, gl + (size_t)stride * i, sizeof(double) * 7, cudaMemcpyDeviceToDevice, stream);
    }
    cudaError_t e2 = cudaFreeAsync(parts, stream);
    if (e2 == cudaSuccess) e2 = cudaFreeAsync(ns, stream);
    if (e2 == cudaSuccess) e2 = cudaFreeAsync(gl, stream);
    if (e2 == cudaSuccess) e2 = cudaFreeAsync(hi, stream);
    if (e2 == cudaSuccess && rev) e2 = cudaFreeAsync(rev, stream);
    if (e != cudaSuccess) return cuda_fail(e, "per-launch rollout");
    if (e2 != cudaSuccess) return cuda_fail(e2, "per-launch scratch free");
    return VPM_OK;
}

// ------------------------------------------------------------------ MPPI

extern "C" vpm_status mppi_weights(const float *d_costs, int K, float lambda, float *d_weights,
                                   cudaStream_t stream)
{
    if (!d_costs || !d_weights) return fail(VPM_ERR_INVALID, "null argument");
    if (K < 1 || !(lambda > 0.f) || !isfinite(lambda)) return fail(VPM_ERR_INVALID, "need K >= 1 and lambda > 0");
    CUDA_TRY(launch_mppi_weights(d_costs, K, (double)lambda, d_weights, stream), "mppi_weights");
    return VPM_OK;
}

extern "C" vpm_status mppi_update(const float *d_weights, const float *d_controls, int K, int H,
                                  float *d_mu, cudaStream_t stream)
{
    if (!d_weights || !d_controls || !d_mu) return fail(VPM_ERR_INVALID, "null argument");
    if (K < 1 || H < 1) return fail(VPM_ERR_INVALID, "K and H must be positive");
    CUDA_TRY(launch_mppi_update(d_weights, d_controls, K, H, d_mu, stream), "mppi_update");
    return VPM_OK;
}

extern "C" vpm_status mppi_perturb(const float *d_mu, const float *d_eps, int K, int H,
                                   float *d_controls, cudaStream_t stream)
{
    if (!d_mu || !d_eps || !d_controls) return fail(VPM_ERR_INVALID, "null argument");
    if (K < 1 || H < 1) return fail(VPM_ERR_INVALID, "K and H must be positive");
    CUDA_TRY(launch_mppi_perturb(d_mu, d_eps, K, H, d_controls, stream), "mppi_perturb");
    return VPM_OK;
}

// ------------------------------------------------------------------ free field

extern "C" vpm_status vpm_freefield_scratch_bytes(int n, size_t *bytes)
{
    if (n < 0 || !bytes) return fail(VPM_ERR_INVALID, "vpm_freefield_scratch_bytes: n < 0 or null");
    *bytes = freefield_sym_scratch_bytes(n);
    return VPM_OK;
}

extern "C" vpm_status vpm_pool_trim(size_t *bytes_held)
{
    cudaMemPool_t pool = lib_pool();
    if (!pool) return fail(VPM_ERR_CUDA, "vpm_pool_trim: no library pool on the current device");
    CUDA_TRY(cudaMemPoolTrimTo(pool, 0), "vpm_pool_trim");
    if (bytes_held) {
        unsigned long long held = 0;
        CUDA_TRY(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &held), "vpm_pool_trim");
        *bytes_held = (size_t)held;
    }
    return VPM_OK;
}

extern "C" vpm_status vpm_freefield_velocity(const float *d_particles, int n, int kernel,
                                             double r_core, float *d_vel, cudaStream_t stream)
{
    if (n < 0 || (n > 0 && (!d_particles || !d_vel))) return fail(VPM_ERR_INVALID, "bad arguments");
    if (kernel < 0 || kernel > 2 || (kernel != VPM_KERNEL_SINGULAR && !(r_core > 0)))
        return fail(VPM_ERR_INVALID, "bad kernel or core radius");
    if (n > freefield_sym_max_n())
        return fail(VPM_ERR_CAPACITY, "vpm_freefield_velocity: n = %d exceeds %d particles", n, freefield_sym_max_n());
    if (n == 0) return VPM_OK;
    void *scratch = nullptr;
    CUDA_TRY(lib_malloc_async(&scratch, freefield_sym_scratch_bytes(n), stream), "freefield scratch");
    cudaError_t e = launch_freefield_sym_velocity(d_particles, n, kernel, r_core, d_vel, scratch, stream);
    cudaError_t e2 = cudaFreeAsync(scratch, stream);
    if (e != cudaSuccess) return cuda_fail(e, "freefield velocity");
    if (e2 != cudaSuccess) return cuda_fail(e2, "freefield scratch free");
    return VPM_OK;
}

extern "C" vpm_status vpm_freefield_heun(float *d_particles, int n, int kernel, double r_core,
                                         double dt, int steps, cudaStream_t stream)
{
    if (n < 0 || steps < 0 || (n > 0 && !d_particles) || !isfinite(dt))
        return fail(VPM_ERR_INVALID, "bad arguments");
    if (kernel < 0 || kernel > 2 || (kernel != VPM_KERNEL_SINGULAR && !(r_core > 0)))
        return fail(VPM_ERR_INVALID, "bad kernel or core radius");
    if (n > freefield_sym_max_n())
        return fail(VPM_ERR_CAPACITY, "vpm_freefield_heun: n = %d exceeds %d particles", n, freefield_sym_max_n());
    if (n == 0 || steps == 0) return VPM_OK;
    // stage positions (16 n bytes), first-stage velocities (8 n bytes), then the accumulators
    char *scratch = nullptr;
    CUDA_TRY(lib_malloc_async((void **)&scratch, (size_t)n * 24 + freefield_sym_scratch_bytes(n), stream),
             "heun scratch");
    cudaError_t e = launch_freefield_sym_heun(d_particles, n, kernel, r_core, dt, steps,
                                              reinterpret_cast<float *>(scratch),
                                              reinterpret_cast<float *>(scratch + (size_t)n * 16),
                                              scratch + (size_t)n * 24, stream);
    cudaError_t e2 = cudaFreeAsync(scratch, stream);
    if (e != cudaSuccess) return cuda_fail(e, "freefield heun");
    if (e2 != cudaSuccess) return cuda_fail(e2, "heun scratch free");
    return VPM_OK;
}
