// Feedback NMPC of §IV-C: a tracking instance of the model follows the observed glider state;
// every P control steps a plan starts from a copy of it, projected L steps ahead under the
// current closed-loop policy (the replanning time), then MPPI reweightings warm-started from the
// previous nominal controls and the least-squares / TVLQR synthesis around the new nominal give
// the policy that takes effect L steps later. The control at step t is
// ubar_t - H_t (x_t - xbar_t) of the policy in effect. Planning runs inline (deterministic) or
// on its own thread and stream, the two-thread split of §IV-C.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/vpm.h"
#include "vpm_trace.cuh"

namespace vpm {
vpm_status report_error(vpm_status st, const char *msg);
}

namespace {

vpm_status fail(vpm_status st, const char *fmt, ...)
{
    char msg[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof msg, fmt, ap);
    va_end(ap);
    return vpm::report_error(st, msg);
}

// A tracking policy indexed by absolute step: rows t0 .. N-1 of gains and ubar, t0 .. N of xbar.
struct Policy {
    int t0 = -1;
    std::vector<float> ubar;      // N
    std::vector<double> xbar;     // (N + 1) x 7
    std::vector<double> gains;    // N x 7
};

}  // namespace

struct vpm_nmpc {
    vpm_nmpc_config cfg;
    vpm_params params;
    int N = 0, K = 0, device = 0;
    vpm_state *tracking = nullptr, *proj = nullptr;
    cudaStream_t ctl = nullptr, pln = nullptr;
    // random draws, per plan
    int n_plans = 0, next_plan = 0;
    std::vector<float> eps, zeta;
    std::vector<double> xi;
    // planner buffers (device)
    float *d_mu = nullptr, *d_noise = nullptr, *d_ctrl = nullptr, *d_costs = nullptr, *d_w = nullptr;
    double *d_traj = nullptr, *d_x0 = nullptr, *d_xbar = nullptr, *d_ahat = nullptr,
           *d_bhat = nullptr, *d_gains = nullptr;
    int *d_info = nullptr;
    // the policy the planner projects with (its own copy) and the control thread's copy
    double *d_pgains = nullptr, *d_pxbar = nullptr;
    float *d_pubar = nullptr;
    std::vector<float> mu;        // N, nominal controls by absolute step (planner-owned)
    Policy active, pending;
    bool has_pending = false;
    bool planned = false;         // the initial plan runs at the first control step
    // threading
    std::thread planner;
    std::mutex m;
    std::condition_variable cv;
    bool stop = false, busy = false, request = false;
    int req_t = 0;
    std::vector<double> req_x;
    Policy req_policy;
    vpm_status planner_error = VPM_OK;
    // statistics
    int plans_done = 0, plans_skipped = 0;
    double last_ms = 0.0, max_ms = 0.0;
};

namespace {

template <class T>
cudaError_t alloc(T **p, size_t n) { return cudaMalloc((void **)p, sizeof(T) * (n ? n : 1)); }

#define NTRY(expr)                                  \
    do {                                            \
        vpm_status st_ = (expr);                    \
        if (st_ != VPM_OK) return st_;              \
    } while (0)
#define NCUDA(expr, what)                                                                   \
    do {                                                                                    \
        cudaError_t e_ = (expr);                                                            \
        if (e_ != cudaSuccess) return fail(VPM_ERR_CUDA, "nmpc %s: %s", what, cudaGetErrorString(e_)); \
    } while (0)

// Device copy of a policy in absolute-step layout for vpm_state_advance_policy.
vpm_status upload_policy(vpm_nmpc *nm, const Policy &p, cudaStream_t s)
{
    NCUDA(cudaMemcpyAsync(nm->d_pgains, p.gains.data(), sizeof(double) * p.gains.size(), cudaMemcpyHostToDevice, s), "policy upload");
    NCUDA(cudaMemcpyAsync(nm->d_pxbar, p.xbar.data(), sizeof(double) * p.xbar.size(), cudaMemcpyHostToDevice, s), "policy upload");
    NCUDA(cudaMemcpyAsync(nm->d_pubar, p.ubar.data(), sizeof(float) * p.ubar.size(), cudaMemcpyHostToDevice, s), "policy upload");
    NCUDA(cudaStreamSynchronize(s), "policy upload");
    return VPM_OK;
}

// MPPI from nm->proj over steps t0 .. N-1, then the policy synthesis around the result, with
// the draws of plan `pi`. Runs on the planner stream; returns the new policy in *out.
vpm_status plan(vpm_nmpc *nm, int t0, int pi, Policy *out)
{
    vpm::TraceRange tr("nmpc: plan (MPPI + least squares + TVLQR)");
    const int N = nm->N, K = nm->K, Hr = N - t0, it_n = nm->cfg.iterations;
    cudaStream_t s = nm->pln;
    const double dt = nm->params.dt;
    std::vector<float> tile((size_t)K * Hr);
    auto upload_tile = [&](const float *src) -> vpm_status {      // rows of N -> rows of Hr
        for (int i = 0; i < K; ++i) memcpy(&tile[(size_t)i * Hr], src + (size_t)i * N, sizeof(float) * Hr);
        NCUDA(cudaMemcpyAsync(nm->d_noise, tile.data(), sizeof(float) * tile.size(), cudaMemcpyHostToDevice, s), "noise upload");
        NCUDA(cudaStreamSynchronize(s), "noise upload");
        return VPM_OK;
    };
    NCUDA(cudaMemcpyAsync(nm->d_mu, nm->mu.data(), sizeof(float) * N, cudaMemcpyHostToDevice, s), "mu upload");
    for (int it = 0; it < it_n; ++it) {
        NTRY(upload_tile(&nm->eps[(((size_t)pi * it_n + it) * K) * N]));
        NTRY(mppi_perturb(nm->d_mu + t0, nm->d_noise, K, Hr, nm->d_ctrl, s));
        NTRY(vpm_rollout_batch(nm->proj, K, Hr, nm->d_ctrl, nm->d_costs, nullptr, nullptr, nullptr, nullptr, s));
        NTRY(mppi_weights(nm->d_costs, K, nm->cfg.lambda, nm->d_w, s));
        NTRY(mppi_update(nm->d_w, nm->d_ctrl, K, Hr, nm->d_mu + t0, s));
    }
    // nominal trajectory: the projected state, then the rollout of the new nominal controls
    NTRY(vpm_rollout_batch(nm->proj, 1, Hr, nm->d_mu + t0, nm->d_costs, nullptr, nm->d_traj, nullptr, nullptr, s));
    double x0bar[7];
    NTRY(vpm_state_get_glider(nm->proj, x0bar, s));
    NCUDA(cudaMemcpyAsync(nm->d_xbar, x0bar, sizeof x0bar, cudaMemcpyHostToDevice, s), "xbar");
    NCUDA(cudaMemcpyAsync(nm->d_xbar + 7, nm->d_traj, sizeof(double) * 7 * Hr, cudaMemcpyDeviceToDevice, s), "xbar");
    // synthesis rollouts: perturbed initial states and controls
    std::vector<double> x0((size_t)K * 7);
    const double *xi = &nm->xi[(size_t)pi * K * 7];
    for (int i = 0; i < K; ++i)
        for (int c = 0; c < 7; ++c) x0[(size_t)i * 7 + c] = x0bar[c] + xi[(size_t)i * 7 + c];
    NCUDA(cudaMemcpyAsync(nm->d_x0, x0.data(), sizeof(double) * x0.size(), cudaMemcpyHostToDevice, s), "x0 upload");
    NTRY(upload_tile(&nm->zeta[(size_t)pi * K * N]));
    NTRY(mppi_perturb(nm->d_mu + t0, nm->d_noise, K, Hr, nm->d_ctrl, s));
    NTRY(vpm_rollout_batch_x0(nm->proj, K, Hr, nm->d_x0, nm->d_ctrl, nm->d_costs, nullptr, nm->d_traj, nullptr, nullptr, s));
    NTRY(vpm_ls_jacobians(K, Hr, dt, nm->d_x0, nm->d_traj, nm->d_ctrl, nm->d_xbar, nm->d_mu + t0,
                          nm->d_ahat, nm->d_bhat, nm->d_info, s));
    NTRY(vpm_tvlqr(Hr, dt, nm->d_ahat, nm->d_bhat, nm->cfg.qc, nm->cfg.qf, nm->cfg.rc, nm->d_gains, nullptr, s));
    // read back
    Policy p;
    p.t0 = t0;
    p.ubar.assign(N, 0.f);
    p.xbar.assign((size_t)(N + 1) * 7, 0.0);
    p.gains.assign((size_t)N * 7, 0.0);
    std::vector<int> info(Hr);
    NCUDA(cudaMemcpyAsync(nm->mu.data() + t0, nm->d_mu + t0, sizeof(float) * Hr, cudaMemcpyDeviceToHost, s), "read back");
    NCUDA(cudaMemcpyAsync(&p.xbar[(size_t)t0 * 7], nm->d_xbar, sizeof(double) * 7 * (Hr + 1), cudaMemcpyDeviceToHost, s), "read back");
    NCUDA(cudaMemcpyAsync(&p.gains[(size_t)t0 * 7], nm->d_gains, sizeof(double) * 7 * Hr, cudaMemcpyDeviceToHost, s), "read back");
    NCUDA(cudaMemcpyAsync(info.data(), nm->d_info, sizeof(int) * Hr, cudaMemcpyDeviceToHost, s), "read back");
    NCUDA(cudaStreamSynchronize(s), "plan");
    for (int k = 0; k < Hr; ++k)
        if (info[k]) return fail(VPM_ERR_SINGULAR, "nmpc: least squares singular at step %d of the plan from %d", k, t0);
    NTRY(vpm_state_status(nm->proj, s));
    p.ubar = nm->mu;
    *out = std::move(p);
    return VPM_OK;
}

// The planner's copy of the tracking instance (taken by the caller) gets the observed glider
// state, is projected L steps under `pol`, then a plan runs from step t + L with the draws of
// plan `pi`. *ms receives the wall time.
vpm_status replan(vpm_nmpc *nm, int t, const double *x_obs, const Policy &pol, int pi, Policy *out,
                  double *ms)
{
    vpm::TraceRange tr("nmpc: replan (projection + plan)");
    const auto t_start = std::chrono::steady_clock::now();
    const int L = nm->cfg.latency;
    NTRY(upload_policy(nm, pol, nm->pln));
    NTRY(vpm_state_set_glider(nm->proj, x_obs, nm->pln));
    NTRY(vpm_state_advance_policy(nm->proj, L, nm->d_pgains, nm->d_pxbar, nm->d_pubar, t, nm->pln));
    NTRY(plan(nm, t + L, pi, out));
    *ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    return VPM_OK;
}

void record_plan(vpm_nmpc *nm, double ms)
{
    nm->last_ms = ms;
    nm->max_ms = std::max(nm->max_ms, ms);
    nm->plans_done++;
}

void planner_loop(vpm_nmpc *nm)
{
    cudaSetDevice(nm->device);
    std::unique_lock<std::mutex> lk(nm->m);
    for (;;) {
        nm->cv.wait(lk, [nm] { return nm->stop || nm->request; });
        if (nm->stop) return;
        nm->request = false;
        const int t = nm->req_t, pi = nm->next_plan++;
        std::vector<double> x = nm->req_x;
        Policy pol = nm->req_policy;
        lk.unlock();
        Policy out;
        double ms = 0.0;
        vpm_status st = replan(nm, t, x.data(), pol, pi, &out, &ms);
        lk.lock();
        nm->busy = false;
        if (st != VPM_OK) {
            nm->planner_error = st;
        } else {
            nm->pending = std::move(out);
            nm->has_pending = true;
            record_plan(nm, ms);
        }
    }
}

// The pending policy becomes the active one once its first step is reached.
vpm_status take_due_plan(vpm_nmpc *nm, int t)
{
    std::unique_lock<std::mutex> lk(nm->m, std::defer_lock);
    if (nm->cfg.threaded) lk.lock();
    if (nm->cfg.threaded && nm->planner_error != VPM_OK) return nm->planner_error;
    if (nm->has_pending && t >= nm->pending.t0) {
        nm->active = std::move(nm->pending);
        nm->has_pending = false;
    }
    return VPM_OK;
}

bool due(const vpm_nmpc *nm, int t)
{
    return t > 0 && t % nm->cfg.replan_every == 0 && t + nm->cfg.latency < nm->N &&
           nm->next_plan < nm->n_plans;
}

}  // namespace

extern "C" vpm_status vpm_nmpc_create(const vpm_nmpc_config *cfg, const vpm_params *params,
                                      const double *h_particles, int n, int capacity,
                                      const double *h_x0, const float *h_mu0, int n_plans,
                                      const float *h_eps, const double *h_xi, const float *h_zeta,
                                      vpm_nmpc **out)
{
    if (!cfg || !params || !h_x0 || !h_mu0 || !h_eps || !h_xi || !h_zeta || !out)
        return fail(VPM_ERR_INVALID, "vpm_nmpc_create: null argument");
    if (cfg->horizon < 2 || cfg->replan_every < 1 || cfg->latency < 0 ||
        cfg->latency > cfg->replan_every || cfg->rollouts < 6 ||
        cfg->iterations < 1 || !(cfg->lambda > 0.f) || !(cfg->rc > 0.0) || n_plans < 1)
        return fail(VPM_ERR_INVALID, "vpm_nmpc_create: bad configuration");
    vpm_nmpc *nm = new vpm_nmpc();
    cudaGetDevice(&nm->device);
    nm->cfg = *cfg;
    nm->params = *params;
    nm->N = cfg->horizon;
    nm->K = cfg->rollouts;
    nm->n_plans = n_plans;
    const size_t N = nm->N, K = nm->K, it = cfg->iterations;
    nm->eps.assign(h_eps, h_eps + (size_t)n_plans * it * K * N);
    nm->xi.assign(h_xi, h_xi + (size_t)n_plans * K * 7);
    nm->zeta.assign(h_zeta, h_zeta + (size_t)n_plans * K * N);
    nm->mu.assign(h_mu0, h_mu0 + N);
    auto cleanup = [nm](vpm_status st) { vpm_nmpc_destroy(nm); return st; };
    cudaError_t e = cudaStreamCreateWithFlags(&nm->ctl, cudaStreamNonBlocking);
    if (!e) e = cudaStreamCreateWithFlags(&nm->pln, cudaStreamNonBlocking);
    if (!e) e = alloc(&nm->d_mu, N);
    if (!e) e = alloc(&nm->d_noise, K * N);
    if (!e) e = alloc(&nm->d_ctrl, K * N);
    if (!e) e = alloc(&nm->d_costs, K);
    if (!e) e = alloc(&nm->d_w, K);
    if (!e) e = alloc(&nm->d_traj, K * N * 7);
    if (!e) e = alloc(&nm->d_x0, K * 7);
    if (!e) e = alloc(&nm->d_xbar, (N + 1) * 7);
    if (!e) e = alloc(&nm->d_ahat, N * 15);
    if (!e) e = alloc(&nm->d_bhat, N * 3);
    if (!e) e = alloc(&nm->d_gains, N * 7);
    if (!e) e = alloc(&nm->d_info, N);
    if (!e) e = alloc(&nm->d_pgains, N * 7);
    if (!e) e = alloc(&nm->d_pxbar, (N + 1) * 7);
    if (!e) e = alloc(&nm->d_pubar, N);
    if (e) return cleanup(fail(VPM_ERR_OOM, "vpm_nmpc_create: %s", cudaGetErrorString(e)));
    vpm_status st = vpm_state_create(params, h_particles, n, capacity, h_x0, &nm->tracking, nm->ctl);
    if (st == VPM_OK) st = vpm_state_create(params, h_particles, n, capacity, h_x0, &nm->proj, nm->pln);
    if (st != VPM_OK) return cleanup(st);
    nm->next_plan = 1;
    if (cfg->threaded) nm->planner = std::thread(planner_loop, nm);
    *out = nm;
    return VPM_OK;
}

extern "C" vpm_status vpm_nmpc_control(vpm_nmpc *nm, int t, const double *h_x_obs, double *h_u)
{
    if (!nm || !h_x_obs || !h_u) return fail(VPM_ERR_INVALID, "vpm_nmpc_control: null argument");
    if (t < 0 || t >= nm->N) return fail(VPM_ERR_INVALID, "vpm_nmpc_control: step outside the horizon");
    vpm::TraceRange tr("nmpc: control step");
    if (!nm->planned) {
        // the first plan, from the tracking instance as it stands (with any injected pair),
        // with the draws of plan 0; a plan's projection needs none at step 0
        NCUDA(cudaStreamSynchronize(nm->ctl), "control stream");
        NTRY(vpm_state_copy(nm->proj, nm->tracking, nm->pln));
        NTRY(vpm_state_set_glider(nm->proj, h_x_obs, nm->pln));
        const auto t_start = std::chrono::steady_clock::now();
        Policy first;
        NTRY(plan(nm, t, 0, &first));
        std::unique_lock<std::mutex> lk(nm->m, std::defer_lock);
        if (nm->cfg.threaded) lk.lock();
        nm->active = std::move(first);
        nm->planned = true;
        record_plan(nm, std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count());
    }
    // a plan due at this step takes effect before this step's replan starts, so that the
    // replan projects under the policy that will be in effect (replan_every == latency), and
    // again after it, so that a plan made with no latency acts at once
    NTRY(take_due_plan(nm, t));
    if (due(nm, t)) {
        if (!nm->cfg.threaded) {
            NCUDA(cudaStreamSynchronize(nm->ctl), "control stream");
            NTRY(vpm_state_copy(nm->proj, nm->tracking, nm->pln));
            Policy out;
            double ms = 0.0;
            NTRY(replan(nm, t, h_x_obs, nm->active, nm->next_plan++, &out, &ms));
            nm->pending = std::move(out);
            nm->has_pending = true;
            record_plan(nm, ms);
        } else {
            std::lock_guard<std::mutex> lk(nm->m);
            if (nm->planner_error != VPM_OK) return nm->planner_error;
            if (nm->busy) {
                nm->plans_skipped++;
            } else {
                // snapshot now: the planner's copy of the tracking instance and of the policy
                cudaError_t e = cudaStreamSynchronize(nm->ctl);
                if (e) return fail(VPM_ERR_CUDA, "vpm_nmpc_control: %s", cudaGetErrorString(e));
                NTRY(vpm_state_copy(nm->proj, nm->tracking, nm->pln));
                e = cudaStreamSynchronize(nm->pln);
                if (e) return fail(VPM_ERR_CUDA, "vpm_nmpc_control: %s", cudaGetErrorString(e));
                nm->req_t = t;
                nm->req_x.assign(h_x_obs, h_x_obs + 7);
                nm->req_policy = nm->active;
                nm->request = true;
                nm->busy = true;
                nm->cv.notify_one();
            }
        }
    }
    NTRY(take_due_plan(nm, t));
    const Policy &p = nm->active;
    double u = (double)p.ubar[t];
    for (int c = 0; c < 7; ++c) u -= p.gains[(size_t)t * 7 + c] * (h_x_obs[c] - p.xbar[(size_t)t * 7 + c]);
    NTRY(vpm_state_set_glider(nm->tracking, h_x_obs, nm->ctl));
    NTRY(vpm_step(nm->tracking, u, nullptr, nullptr, nullptr, nullptr, nm->ctl));
    *h_u = u;
    return VPM_OK;
}

extern "C" vpm_status vpm_nmpc_inject_pair(vpm_nmpc *nm, const double *h_pair)
{
    if (!nm || !h_pair) return fail(VPM_ERR_INVALID, "vpm_nmpc_inject_pair: null argument");
    NCUDA(cudaStreamSynchronize(nm->ctl), "control stream");
    return vpm_state_inject_pair(nm->tracking, h_pair, nm->ctl);
}

extern "C" vpm_status vpm_nmpc_policy(vpm_nmpc *nm, int *t0, double *h_gains, double *h_xbar,
                                      float *h_ubar)
{
    if (!nm) return fail(VPM_ERR_INVALID, "vpm_nmpc_policy: null argument");
    std::unique_lock<std::mutex> lk(nm->m, std::defer_lock);
    if (nm->cfg.threaded) lk.lock();
    const Policy &p = nm->active;
    if (t0) *t0 = p.t0;
    if (h_gains) memcpy(h_gains, p.gains.data(), sizeof(double) * p.gains.size());
    if (h_xbar) memcpy(h_xbar, p.xbar.data(), sizeof(double) * p.xbar.size());
    if (h_ubar) memcpy(h_ubar, p.ubar.data(), sizeof(float) * p.ubar.size());
    return VPM_OK;
}

extern "C" vpm_status vpm_nmpc_stats(vpm_nmpc *nm, int *plans_done, int *plans_skipped,
                                     double *last_plan_ms, double *max_plan_ms)
{
    if (!nm) return fail(VPM_ERR_INVALID, "vpm_nmpc_stats: null argument");
    std::unique_lock<std::mutex> lk(nm->m, std::defer_lock);
    if (nm->cfg.threaded) lk.lock();
    if (plans_done) *plans_done = nm->plans_done;
    if (plans_skipped) *plans_skipped = nm->plans_skipped;
    if (last_plan_ms) *last_plan_ms = nm->last_ms;
    if (max_plan_ms) *max_plan_ms = nm->max_ms;
    return VPM_OK;
}

extern "C" vpm_status vpm_nmpc_destroy(vpm_nmpc *nm)
{
    if (!nm) return VPM_OK;
    if (nm->planner.joinable()) {
        {
            std::lock_guard<std::mutex> lk(nm->m);
            nm->stop = true;
        }
        nm->cv.notify_all();
        nm->planner.join();
    }
    if (nm->ctl) cudaStreamSynchronize(nm->ctl);
    if (nm->pln) cudaStreamSynchronize(nm->pln);
    if (nm->tracking) vpm_state_destroy(nm->tracking);
    if (nm->proj) vpm_state_destroy(nm->proj);
    void *bufs[] = {nm->d_mu, nm->d_noise, nm->d_ctrl, nm->d_costs, nm->d_w, nm->d_traj, nm->d_x0,
                    nm->d_xbar, nm->d_ahat, nm->d_bhat, nm->d_gains, nm->d_info, nm->d_pgains,
                    nm->d_pxbar, nm->d_pubar};
    for (void *b : bufs)
        if (b) cudaFree(b);
    if (nm->ctl) cudaStreamDestroy(nm->ctl);
    if (nm->pln) cudaStreamDestroy(nm->pln);
    delete nm;
    return VPM_OK;
}
