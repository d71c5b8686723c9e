// Batches of rollouts from many different roots (uneven particle counts) in persistent
// launches: host-side grouping into shared-memory classes, longest-first ordering, the
// autotuner (block size, diagonal-unit size, CTAs per rollout, class launches or one launch
// for all), and
// capture of a whole horizon into a CUDA graph.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <string>
#include <vector>

#include "vpm_rollout.cuh"
#include "vpm_trace.cuh"

namespace vpm {
vpm_status report_error(vpm_status st, const char *msg);
}

using namespace vpm;

static vpm_status bfail(vpm_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return report_error(st, buf);
}

static vpm_status bcuda(cudaError_t e, const char *what)
{
    cudaGetLastError();
    return bfail(VPM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define BTRY(call, what)                                   \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return bcuda(e_, what);     \
    } while (0)

// Shared-memory classes: a rollout whose field can reach `cap` particles goes to the first
// class with cap <= limit. The limits are where the number of resident 128-thread blocks per
// SM changes (24 bytes per particle on the binary32 path): 7, 4, 3, 2, 1.
static const int kClassLimit[] = {1300, 2300, 3000, 4500, 9300};
static const int kNumClasses = 5;
static const int kStateStride = kMaxB + 2;

struct BatchClass {
    int cap = 0;                 // largest capacity in the class (shared-memory size)
    int nt = 128;                // threads per block (autotuned)
    int dt = 2;                  // targets per lane of the diagonal pair units (autotuned)
    int ctas = 1;                // CTAs per rollout: 1, or a cluster of 2 or 4 (autotuned)
    int grid = 0;                // persistent CTAs (resident blocks per SM x SMs, or resident
                                 // clusters x ctas)
    float tuned_ms = 0.f;
    std::vector<int> items;      // rollout indices, largest first
    int *d_order = nullptr;
    float2 *d_rev = nullptr;     // pair-sum scratch of the persistent blocks (binary32)
    size_t rev_blocks = 0;       // blocks it holds
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
};

struct vpm_batch {
    vpm_params params;
    DevParams dp;
    int R = 0, max_h = 0, device = 0, sms = 0;
    size_t rec_bytes = 0;
    std::vector<int> counts;
    void *d_part = nullptr;
    long long *d_offset = nullptr;
    int *d_n = nullptr;
    double *d_glider = nullptr, *d_hist = nullptr, *d_kinv = nullptr;
    int *d_counters = nullptr, *d_status = nullptr;
    BatchClass cls[kNumClasses + 1];   // the classes, then all rollouts as one class
    bool merged = false;               // run the last one (one launch) instead of the classes
    float split_ms = 0.f, merged_ms = 0.f;   // the tuner's whole-batch times of both schedules
    cudaEvent_t fork = nullptr;
    cudaStream_t capture_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    int g_h = -1;
    const void *g_ctrl = nullptr, *g_costs = nullptr, *g_count = nullptr, *g_final = nullptr;
};

// Defined in vpm_api.cu (parameter checks, body-frame surface inverses, record packing).
namespace vpm {
vpm_status check_params_ext(const vpm_params *p);
vpm_status surface_inverses_ext(const vpm_params *p, double *kinv);
void fill_dev_params_ext(const vpm_params *p, DevParams &d);
void pack_records_ext(int precision, const double *h, int n, void *out);
}

static void batch_free(vpm_batch *b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (auto &c : b->cls) {
        cudaFree(c.d_order);
        cudaFree(c.d_rev);
        if (c.stream) cudaStreamDestroy(c.stream);
        if (c.done) cudaEventDestroy(c.done);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    cudaFree(b->d_part); cudaFree(b->d_offset); cudaFree(b->d_n); cudaFree(b->d_glider);
    cudaFree(b->d_hist); cudaFree(b->d_kinv); cudaFree(b->d_counters); cudaFree(b->d_status);
    cudaGetLastError();
    delete b;
}

extern "C" vpm_status vpm_batch_create(const vpm_params *params, int R, const int *h_counts,
                                       const double *h_particles, const double *h_gliders,
                                       int max_horizon, vpm_batch **out, cudaStream_t stream)
{
    vpm_status st = check_params_ext(params);
    if (st) return st;
    if (!out || !h_counts || !h_gliders || R < 1 || max_horizon < 1)
        return bfail(VPM_ERR_INVALID, "vpm_batch_create: need R >= 1, max_horizon >= 1 and non-null arrays");
    long long total = 0;
    for (int i = 0; i < R; ++i) {
        if (h_counts[i] < 0) return bfail(VPM_ERR_INVALID, "vpm_batch_create: negative count");
        total += h_counts[i];
    }
    if (total > 0 && !h_particles) return bfail(VPM_ERR_INVALID, "vpm_batch_create: null particles");
    for (long long i = 0; i < 3 * total; ++i)
        if (!isfinite(h_particles[i])) return bfail(VPM_ERR_NONFINITE, "vpm_batch_create: non-finite particle");
    for (int i = 0; i < 7 * R; ++i)
        if (!isfinite(h_gliders[i])) return bfail(VPM_ERR_NONFINITE, "vpm_batch_create: non-finite glider");
    int dev = 0, count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) {
        cudaGetLastError();
        return bfail(VPM_ERR_CUDA, "no CUDA device available");
    }
    BTRY(cudaGetDevice(&dev), "cudaGetDevice");
    vpm_batch *b = new vpm_batch();
    b->params = *params;
    b->R = R;
    b->max_h = max_horizon;
    b->device = dev;
    b->counts.assign(h_counts, h_counts + R);
    BTRY(cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    b->rec_bytes = params->precision == VPM_FP64 ? sizeof(Part64) : sizeof(float4);
    fill_dev_params_ext(params, b->dp);
    // classes by capacity, longest first within a class; the merged class holds every rollout
    BatchClass &all = b->cls[kNumClasses];
    for (int i = 0; i < R; ++i) {
        long long cap = (long long)h_counts[i] + 2LL * max_horizon;
        if (params->n_wake_max > 0)
            cap = std::min<long long>(cap, std::max<long long>(params->n_wake_max, h_counts[i]) + 2);
        int c = 0;
        while (c < kNumClasses && cap > kClassLimit[c]) ++c;
        if (c == kNumClasses || (params->precision == VPM_FP64 && cap > 4500)) {
            batch_free(b);
            return bfail(VPM_ERR_CAPACITY, "rollout %d may reach %lld particles, beyond one block's shared memory", i, cap);
        }
        b->cls[c].items.push_back(i);
        b->cls[c].cap = std::max(b->cls[c].cap, (int)std::max<long long>(cap, 1));
        all.items.push_back(i);
        all.cap = std::max(all.cap, (int)std::max<long long>(cap, 1));
    }
    for (auto &c : b->cls)
        std::stable_sort(c.items.begin(), c.items.end(),
                         [&](int x, int y) { return h_counts[x] > h_counts[y]; });
    // device copies
    std::vector<long long> off(R);
    long long acc = 0;
    for (int i = 0; i < R; ++i) { off[i] = acc; acc += h_counts[i]; }
    std::vector<char> rec(b->rec_bytes * (size_t)std::max<long long>(total, 1));
    pack_records_ext(params->precision, h_particles, (int)total, rec.data());
    std::vector<double> gl((size_t)kStateStride * R, 0.0), hist((size_t)kStateStride * R, 0.0);
    for (int i = 0; i < R; ++i)
        for (int k = 0; k < 7; ++k) gl[(size_t)kStateStride * i + k] = h_gliders[7 * i + k];
    std::vector<double> kinv(4 * kMaxS * kMaxS);
    if ((st = surface_inverses_ext(params, kinv.data()))) { batch_free(b); return st; }
    cudaError_t e = cudaSuccess;
    if ((e = cudaMalloc(&b->d_part, rec.size())) != cudaSuccess ||
        (e = cudaMalloc((void **)&b->d_offset, sizeof(long long) * R)) != cudaSuccess ||
        (e = cudaMalloc((void **)&b->d_n, sizeof(int) * R)) != cudaSuccess ||
        (e = cudaMalloc((void **)&b->d_glider, sizeof(double) * gl.size())) != cudaSuccess ||
        (e = cudaMalloc((void **)&b->d_hist, sizeof(double) * hist.size())) != cudaSuccess ||
        (e = cudaMalloc((void **)&b->d_kinv, sizeof(double) * kinv.size())) != cudaSuccess ||
        (e = cudaMalloc((void **)&b->d_counters, sizeof(int) * (kNumClasses + 1))) != cudaSuccess ||
        (e = cudaMalloc((void **)&b->d_status, sizeof(int))) != cudaSuccess) {
        batch_free(b);
        cudaGetLastError();
        return bfail(VPM_ERR_OOM, "vpm_batch_create: %s", cudaGetErrorString(e));
    }
    b->dp.kinv = b->d_kinv;
    e = cudaMemcpyAsync(b->d_part, rec.data(), rec.size(), cudaMemcpyHostToDevice, stream);
    if (!e) e = cudaMemcpyAsync(b->d_offset, off.data(), sizeof(long long) * R, cudaMemcpyHostToDevice, stream);
    if (!e) e = cudaMemcpyAsync(b->d_n, h_counts, sizeof(int) * R, cudaMemcpyHostToDevice, stream);
    if (!e) e = cudaMemcpyAsync(b->d_glider, gl.data(), sizeof(double) * gl.size(), cudaMemcpyHostToDevice, stream);
    if (!e) e = cudaMemcpyAsync(b->d_hist, hist.data(), sizeof(double) * hist.size(), cudaMemcpyHostToDevice, stream);
    if (!e) e = cudaMemcpyAsync(b->d_kinv, kinv.data(), sizeof(double) * kinv.size(), cudaMemcpyHostToDevice, stream);
    if (!e) e = cudaMemsetAsync(b->d_status, 0, sizeof(int), stream);
    for (auto &c : b->cls) {
        if (c.items.empty() || e) continue;
        if (!e) e = cudaMalloc((void **)&c.d_order, sizeof(int) * c.items.size());
        if (!e) e = cudaMemcpyAsync(c.d_order, c.items.data(), sizeof(int) * c.items.size(), cudaMemcpyHostToDevice, stream);
        if (!e) e = cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking);
        if (!e) e = cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming);
        // default block size before tuning: more threads where fewer blocks fit per SM
        c.nt = c.cap <= kClassLimit[0] ? 128 : (c.cap <= kClassLimit[2] ? 256 : 512);
        if (params->precision == VPM_FP64) c.nt = 128;
    }
    if (!e) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (!e) e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
    if (!e) e = cudaStreamSynchronize(stream);
    if (e) { batch_free(b); return bcuda(e, "vpm_batch_create"); }
    *out = b;
    return VPM_OK;
}

extern "C" vpm_status vpm_batch_destroy(vpm_batch *b)
{
    batch_free(b);
    return VPM_OK;
}

static void batch_args(const vpm_batch *b, int H, const float *ctrl, float *costs, int *count,
                       double *final_glider, RolloutArgs &a)
{
    memset(&a, 0, sizeof a);
    a.p = b->dp;
    a.root_part = b->d_part;
    a.root_n = b->d_n;
    a.root_glider = b->d_glider;
    a.root_hist = b->d_hist;
    a.root_offset = b->d_offset;
    a.state_stride = kStateStride;
    a.H = H;
    a.K = b->R;
    a.controls = ctrl;
    a.ctrl_stride = H;
    a.costs = costs;
    a.count = count;
    a.final_glider = final_glider;
    a.status = b->d_status;
}

// Persistent grid of class c for nt threads per block and `ctas` CTAs per rollout; also sets
// the kernel's shared-memory limit, so it runs before any capture.
static cudaError_t prepare_class(vpm_batch *b, int c, int nt, int dt, int ctas)
{
    BatchClass &k = b->cls[c];
    const size_t smem = rollout_smem_bytes(b->params.precision, k.cap);
    if (ctas > 1) {
        const int clusters = uneven_max_clusters(b->params.precision, b->params.wake_kernel, nt, dt,
                                                 ctas, smem);
        if (clusters < 1) return cudaErrorInvalidConfiguration;
        k.grid = std::min<int>((int)k.items.size(), clusters) * ctas;
    } else {
        const int per_sm = uneven_blocks_per_sm(b->params.precision, b->params.wake_kernel, nt, dt, smem);
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        k.grid = std::min<int>((int)k.items.size(), per_sm * b->sms);
    }
    // scratch for the grid's blocks; a captured graph that holds the old buffer is dropped
    const long long slots = rollout_rev_slots(b->params.precision, k.cap);
    if (slots > 0 && (size_t)k.grid > k.rev_blocks) {
        if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return e;
        cudaFree(k.d_rev);
        k.d_rev = nullptr;
        k.rev_blocks = 0;
        e = cudaMalloc((void **)&k.d_rev, sizeof(float2) * (size_t)slots * (size_t)k.grid);
        if (e != cudaSuccess) return e;
        k.rev_blocks = (size_t)k.grid;
    }
    return cudaSuccess;
}

// The classes a schedule runs: the separate classes, or the merged one.
static bool runs_class(const vpm_batch *b, int c, bool merged)
{
    return !b->cls[c].items.empty() && (merged ? c == kNumClasses : c < kNumClasses);
}

// Enqueues the class launches on the class streams, forked from and joined back into s (the
// merged schedule: one launch). The classes must have been prepared for the sizes used.
static cudaError_t enqueue_classes(vpm_batch *b, int H, const float *ctrl, float *costs,
                                   int *count, double *final_glider, cudaStream_t s,
                                   int only_class = -1, int nt_override = 0, int dt_override = 0,
                                   int merged = -1, int ctas_override = 0)
{
    const bool mg = merged < 0 ? b->merged : merged != 0;
    cudaError_t e = cudaMemsetAsync(b->d_counters, 0, sizeof(int) * (kNumClasses + 1), s);
    if (!e) e = cudaEventRecord(b->fork, s);
    for (int c = 0; c <= kNumClasses && !e; ++c) {
        BatchClass &k = b->cls[c];
        if (only_class >= 0 ? (c != only_class || k.items.empty()) : !runs_class(b, c, mg)) continue;
        const int nt = nt_override ? nt_override : k.nt;
        const int dt = dt_override ? dt_override : k.dt;
        const int ctas = ctas_override ? ctas_override : k.ctas;
        const int grid = k.grid;
        RolloutArgs a;
        batch_args(b, H, ctrl, costs, count, final_glider, a);
        a.cap = k.cap;
        a.order = k.d_order;
        a.counter = b->d_counters + c;
        a.n_items = (int)k.items.size();
        a.rev = k.d_rev;
        a.rev_stride = rollout_rev_slots(b->params.precision, k.cap);
        e = cudaStreamWaitEvent(k.stream, b->fork, 0);
        if (!e) e = ctas > 1 ? launch_uneven_cluster(a, grid / ctas, nt, dt, ctas, k.stream)
                             : launch_uneven(b->params.precision, a, grid, nt, dt, k.stream);
        if (!e) e = cudaEventRecord(k.done, k.stream);
        if (!e) e = cudaStreamWaitEvent(s, k.done, 0);
    }
    return e;
}

extern "C" vpm_status vpm_batch_rollout(vpm_batch *b, int H, const float *d_controls,
                                        float *d_costs, int *d_count, double *d_final_glider,
                                        int use_graph, cudaStream_t stream)
{
    vpm::TraceRange tr("vpm_batch_rollout");
    if (!b || !d_controls || !d_costs) return bfail(VPM_ERR_INVALID, "vpm_batch_rollout: null argument");
    if (H < 1 || H > b->max_h) return bfail(VPM_ERR_INVALID, "vpm_batch_rollout: need 1 <= H <= %d", b->max_h);
    for (int c = 0; c <= kNumClasses; ++c)
        if (runs_class(b, c, b->merged))
            BTRY(prepare_class(b, c, b->cls[c].nt, b->cls[c].dt, b->cls[c].ctas), "prepare class");
    if (!use_graph) {
        cudaError_t e = enqueue_classes(b, H, d_controls, d_costs, d_count, d_final_glider, stream);
        if (e) return bcuda(e, "vpm_batch_rollout");
        return VPM_OK;
    }
    if (!b->graph || b->g_h != H || b->g_ctrl != d_controls || b->g_costs != d_costs ||
        b->g_count != d_count || b->g_final != d_final_glider) {
        if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
        cudaGraph_t g = nullptr;
        BTRY(cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        cudaError_t e = enqueue_classes(b, H, d_controls, d_costs, d_count, d_final_glider, b->capture_stream);
        cudaError_t e2 = cudaStreamEndCapture(b->capture_stream, &g);
        if (e || e2) {
            if (g) cudaGraphDestroy(g);
            return bcuda(e ? e : e2, "graph capture");
        }
        e = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (e) { b->graph = nullptr; return bcuda(e, "graph instantiate"); }
        b->g_h = H; b->g_ctrl = d_controls; b->g_costs = d_costs; b->g_count = d_count;
        b->g_final = d_final_glider;
    }
    BTRY(cudaGraphLaunch(b->graph, stream), "graph launch");
    return VPM_OK;
}

// Times one enqueue of the batch (or of one class) over Ht steps after one warm-up enqueue.
static cudaError_t time_enqueue(vpm_batch *b, int Ht, const float *ctrl, float *costs, cudaStream_t s,
                                cudaEvent_t t0, cudaEvent_t t1, float &ms, int only_class, int nt,
                                int dt, int merged, int ctas = 0)
{
    cudaError_t e = enqueue_classes(b, Ht, ctrl, costs, nullptr, nullptr, s, only_class, nt, dt, merged, ctas);
    if (!e) e = cudaEventRecord(t0, s);
    if (!e) e = enqueue_classes(b, Ht, ctrl, costs, nullptr, nullptr, s, only_class, nt, dt, merged, ctas);
    if (!e) e = cudaEventRecord(t1, s);
    if (!e) e = cudaEventSynchronize(t1);
    if (!e) e = cudaEventElapsedTime(&ms, t0, t1);
    return e;
}

// Median time of three replays of the whole batch over Ht steps in the schedule `merged`, captured
// into a CUDA graph as vpm_batch_rollout runs it (concurrent class launches vary from run to run,
// and their eager and graph forms differ by a few per cent).
static cudaError_t time_graph(vpm_batch *b, int Ht, const float *ctrl, float *costs, cudaStream_t s,
                              cudaEvent_t t0, cudaEvent_t t1, bool merged, float &ms)
{
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal);
    if (e) return e;
    e = enqueue_classes(b, Ht, ctrl, costs, nullptr, nullptr, b->capture_stream, -1, 0, 0, merged ? 1 : 0);
    const cudaError_t e2 = cudaStreamEndCapture(b->capture_stream, &g);
    if (!e) e = e2;
    if (!e) e = cudaGraphInstantiate(&ge, g, 0);
    if (g) cudaGraphDestroy(g);
    float t[3] = {0.f, 0.f, 0.f};
    if (!e) e = cudaGraphLaunch(ge, s);              // warm-up
    for (int r = 0; r < 3 && !e; ++r) {
        e = cudaEventRecord(t0, s);
        if (!e) e = cudaGraphLaunch(ge, s);
        if (!e) e = cudaEventRecord(t1, s);
        if (!e) e = cudaEventSynchronize(t1);
        if (!e) e = cudaEventElapsedTime(&t[r], t0, t1);
    }
    if (ge) cudaGraphExecDestroy(ge);
    std::sort(t, t + 3);
    ms = t[1];
    return e;
}

// Autotuner over the launch shape: for every class (and for the merged class that runs all
// rollouts in one persistent launch), one launch of the class alone over min(H, 3) steps is timed
// for each block size that fits (128, 256, 512 threads) and each diagonal-unit size (32, 64 or
// 128 targets: 1, 2 or 4 per lane; the Vatistas kernel only, others keep 2); each keeps its
// fastest. A class of fields above kClusterMinCap particles (Vatistas kernel) is then timed at
// that shape with each rollout spread over a cluster of 2 and of 4 CTAs, and keeps the fastest
// of 1, 2 and 4 CTAs per rollout. A class alone may leave SMs idle that clusters fill, while the
// classes side by side fill the GPU anyway, so cluster choices are kept only if the whole batch
// of class launches runs faster with them than with one CTA per rollout. Then the whole batch is
// timed as concurrent class launches and as the one merged launch, and the faster schedule is
// kept. The whole-batch timings run the whole horizon H as a CUDA graph (median of three
// replays): over 3 or 10 steps the class launches of the 4096-rollout batch looked 3-5 % faster
// than the merged launch and were 1-2 % slower over its 50 steps, and one eager timing of them
// came out 6 % below their graph replay.
// A rollout's result depends on none of these choices, so tuning changes speed only.
// Synchronises `stream`.
static const int kClusterMinCap = 2300;

extern "C" vpm_status vpm_batch_tune(vpm_batch *b, int H, const float *d_controls,
                                     cudaStream_t stream)
{
    if (!b || !d_controls) return bfail(VPM_ERR_INVALID, "vpm_batch_tune: null argument");
    if (H < 1 || H > b->max_h) return bfail(VPM_ERR_INVALID, "vpm_batch_tune: bad H");
    if (b->params.precision == VPM_FP64) return VPM_OK;
    const int Ht = std::min(H, 3);
    float *costs = nullptr;
    BTRY(lib_malloc_async((void **)&costs, sizeof(float) * b->R, stream), "tune scratch");
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    vpm_status st = VPM_OK;
    const bool vat = b->params.wake_kernel == VPM_KERNEL_VATISTAS;
    int nonempty = 0;
    for (int c = 0; c < kNumClasses; ++c) nonempty += !b->cls[c].items.empty();
    for (int c = 0; c <= kNumClasses && st == VPM_OK; ++c) {
        BatchClass &k = b->cls[c];
        if (k.items.empty() || (c == kNumClasses && nonempty < 2)) continue;
        const size_t smem = rollout_smem_bytes(b->params.precision, k.cap);
        float best = INFINITY;
        int best_nt = k.nt, best_dt = k.dt;
        for (int nt : {128, 256, 512}) {
            for (int dt : {1, 2, 4}) {
                if (dt != 2 && !vat) continue;
                if (uneven_blocks_per_sm(b->params.precision, b->params.wake_kernel, nt, dt, smem) < 1) continue;
                float ms = 0.f;
                cudaError_t e = prepare_class(b, c, nt, dt, 1);
                if (!e) e = time_enqueue(b, Ht, d_controls, costs, stream, t0, t1, ms, c, nt, dt, -1, 1);
                if (e) { st = bcuda(e, "vpm_batch_tune"); break; }
                if (ms < best) { best = ms; best_nt = nt; best_dt = dt; }
            }
            if (st != VPM_OK) break;
        }
        int best_ctas = 1;
        for (int ctas : {2, 4}) {
            if (st != VPM_OK || !vat || k.cap <= kClusterMinCap) break;
            if (uneven_max_clusters(b->params.precision, b->params.wake_kernel, best_nt, best_dt, ctas, smem) < 1)
                continue;
            float ms = 0.f;
            cudaError_t e = prepare_class(b, c, best_nt, best_dt, ctas);
            if (!e) e = time_enqueue(b, Ht, d_controls, costs, stream, t0, t1, ms, c, best_nt, best_dt, -1, ctas);
            if (e) { st = bcuda(e, "vpm_batch_tune"); break; }
            if (ms < best) { best = ms; best_ctas = ctas; }
        }
        k.nt = best_nt;
        k.dt = best_dt;
        k.ctas = best_ctas;
        k.tuned_ms = best;
        if (st == VPM_OK) {
            cudaError_t e = prepare_class(b, c, best_nt, best_dt, best_ctas);
            if (e) st = bcuda(e, "vpm_batch_tune");
        }
    }
    const int Hw = H;
    b->merged = false;
    // cluster choices made class by class, against one CTA per rollout for the whole batch
    bool clustered = false;
    for (int c = 0; c < kNumClasses; ++c) clustered |= !b->cls[c].items.empty() && b->cls[c].ctas > 1;
    if (st == VPM_OK && nonempty >= 2 && clustered) {
        float with = 0.f, without = 0.f;
        int chosen[kNumClasses];
        for (int c = 0; c < kNumClasses; ++c) chosen[c] = b->cls[c].ctas;
        cudaError_t e = time_graph(b, Hw, d_controls, costs, stream, t0, t1, false, with);
        for (int c = 0; c < kNumClasses && !e; ++c) {
            if (b->cls[c].items.empty() || chosen[c] == 1) continue;
            b->cls[c].ctas = 1;
            e = prepare_class(b, c, b->cls[c].nt, b->cls[c].dt, 1);
        }
        if (!e) e = time_graph(b, Hw, d_controls, costs, stream, t0, t1, false, without);
        if (!e && with < without) {
            for (int c = 0; c < kNumClasses && !e; ++c) {
                if (b->cls[c].items.empty() || chosen[c] == 1) continue;
                b->cls[c].ctas = chosen[c];
                e = prepare_class(b, c, b->cls[c].nt, b->cls[c].dt, chosen[c]);
            }
        }
        if (e) st = bcuda(e, "vpm_batch_tune");
    }
    // class launches side by side against the one merged launch
    if (st == VPM_OK && nonempty >= 2) {
        float split = 0.f, one = 0.f;
        cudaError_t e = time_graph(b, Hw, d_controls, costs, stream, t0, t1, false, split);
        if (!e) e = time_graph(b, Hw, d_controls, costs, stream, t0, t1, true, one);
        if (e) st = bcuda(e, "vpm_batch_tune");
        else { b->merged = one < split; b->split_ms = split; b->merged_ms = one; }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaFreeAsync(costs, stream);
    if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
    cudaError_t e = cudaStreamSynchronize(stream);
    if (st == VPM_OK && e) st = bcuda(e, "vpm_batch_tune sync");
    return st;
}

extern "C" vpm_status vpm_batch_schedule(const vpm_batch *b, int *h_nclasses, int *h_cap,
                                         int *h_nt, int *h_items, float *h_tuned_ms, int *h_diag_t,
                                         int *h_ctas, int *h_merged)
{
    if (!b || !h_nclasses) return bfail(VPM_ERR_INVALID, "vpm_batch_schedule: null argument");
    int m = 0;
    for (int c = 0; c <= kNumClasses; ++c) {
        if (!runs_class(b, c, b->merged)) continue;
        const BatchClass &k = b->cls[c];
        if (h_cap) h_cap[m] = k.cap;
        if (h_nt) h_nt[m] = k.nt;
        if (h_items) h_items[m] = (int)k.items.size();
        if (h_tuned_ms) h_tuned_ms[m] = k.tuned_ms;
        if (h_diag_t) h_diag_t[m] = k.dt;
        if (h_ctas) h_ctas[m] = k.ctas;
        ++m;
    }
    *h_nclasses = m;
    if (h_merged) *h_merged = b->merged ? 1 : 0;
    return VPM_OK;
}

extern "C" vpm_status vpm_batch_tuned_modes(const vpm_batch *b, float *h_split_ms, float *h_merged_ms)
{
    if (!b || !h_split_ms || !h_merged_ms) return bfail(VPM_ERR_INVALID, "vpm_batch_tuned_modes: null argument");
    *h_split_ms = b->split_ms;
    *h_merged_ms = b->merged_ms;
    return VPM_OK;
}

extern "C" vpm_status vpm_batch_set_schedule(vpm_batch *b, int merged, int cls, int nt, int diag_t)
{
    if (!b) return bfail(VPM_ERR_INVALID, "vpm_batch_set_schedule: null batch");
    if (nt != 128 && nt != 256 && nt != 512) return bfail(VPM_ERR_INVALID, "vpm_batch_set_schedule: threads must be 128, 256 or 512");
    if (diag_t != 1 && diag_t != 2 && diag_t != 4) return bfail(VPM_ERR_INVALID, "vpm_batch_set_schedule: diag_t must be 1, 2 or 4");
    if (b->params.precision == VPM_FP64 && (nt != 128 || diag_t != 2))
        return bfail(VPM_ERR_INVALID, "vpm_batch_set_schedule: binary64 batches run 128 threads, diag_t 2");
    if (b->params.wake_kernel != VPM_KERNEL_VATISTAS && diag_t != 2)
        return bfail(VPM_ERR_INVALID, "vpm_batch_set_schedule: diag_t other than 2 needs the Vatistas kernel");
    int m = 0, target = -1;
    for (int c = 0; c <= kNumClasses; ++c) {
        if (!runs_class(b, c, merged != 0)) continue;
        if (m++ == cls) target = c;
    }
    if (target < 0) return bfail(VPM_ERR_INVALID, "vpm_batch_set_schedule: class %d does not exist in that schedule", cls);
    const size_t smem = rollout_smem_bytes(b->params.precision, b->cls[target].cap);
    if (uneven_blocks_per_sm(b->params.precision, b->params.wake_kernel, nt, diag_t, smem) < 1)
        return bfail(VPM_ERR_INVALID, "vpm_batch_set_schedule: %d threads do not fit the class", nt);
    const int ctas = b->cls[target].ctas;
    if (ctas > 1 && uneven_max_clusters(b->params.precision, b->params.wake_kernel, nt, diag_t, ctas, smem) < 1)
        return bfail(VPM_ERR_INVALID, "vpm_batch_set_schedule: %d threads do not fit a cluster of %d", nt, ctas);
    b->merged = merged != 0;
    b->cls[target].nt = nt;
    b->cls[target].dt = diag_t;
    if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
    return VPM_OK;
}

extern "C" vpm_status vpm_batch_set_ctas(vpm_batch *b, int merged, int cls, int ctas)
{
    if (!b) return bfail(VPM_ERR_INVALID, "vpm_batch_set_ctas: null batch");
    if (ctas != 1 && ctas != 2 && ctas != 4) return bfail(VPM_ERR_INVALID, "vpm_batch_set_ctas: ctas must be 1, 2 or 4");
    if (ctas > 1 && (b->params.precision != VPM_FP32 || b->params.wake_kernel != VPM_KERNEL_VATISTAS))
        return bfail(VPM_ERR_INVALID, "vpm_batch_set_ctas: clusters need a binary32 batch with the Vatistas kernel");
    int m = 0, target = -1;
    for (int c = 0; c <= kNumClasses; ++c) {
        if (!runs_class(b, c, merged != 0)) continue;
        if (m++ == cls) target = c;
    }
    if (target < 0) return bfail(VPM_ERR_INVALID, "vpm_batch_set_ctas: class %d does not exist in that schedule", cls);
    BatchClass &k = b->cls[target];
    const size_t smem = rollout_smem_bytes(b->params.precision, k.cap);
    if (ctas > 1 && uneven_max_clusters(b->params.precision, b->params.wake_kernel, k.nt, k.dt, ctas, smem) < 1)
        return bfail(VPM_ERR_INVALID, "vpm_batch_set_ctas: a cluster of %d CTAs of %d threads does not fit", ctas, k.nt);
    b->merged = merged != 0;
    k.ctas = ctas;
    if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
    return VPM_OK;
}

extern "C" vpm_status vpm_batch_status(vpm_batch *b, cudaStream_t stream)
{
    if (!b) return bfail(VPM_ERR_INVALID, "null batch");
    int st = 0;
    BTRY(cudaMemcpyAsync(&st, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, stream), "status");
    BTRY(cudaStreamSynchronize(stream), "status sync");
    if (st) {
        BTRY(cudaMemsetAsync(b->d_status, 0, sizeof(int), stream), "status clear");
        return bfail(VPM_ERR_NONFINITE, "non-finite value in a batched rollout");
    }
    return VPM_OK;
}
