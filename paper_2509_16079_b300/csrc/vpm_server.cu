// Replanning server: resident scenario fields, requests admitted by free device memory and
// slots, overlapping on the device (continuous batching at the granularity of requests).
//
// A request asks for one MPPI iteration (§IV-A, Eq. 25) of K rollouts over H steps on one
// scenario's resident field, optionally after advancing that field by a few committed steps
// (the tracking instance of §IV-C). A worker thread owns all device work: it completes finished
// requests, then admits queued ones in arrival order while a slot is free, the scenario has no
// request on the device, the request's device memory (its buffers and its rollouts' pair-sum
// scratch) fits both the configured budget and the memory the device has free at that moment
// (read at each admission, less a reserve of max(1 GiB, 2 % of the device)), and its rollouts
// fit the rollout budget (beyond the rollout blocks the device holds at once, more concurrency
// adds latency without throughput). Each admitted
// request runs on its own stream, so requests that arrive while others are on the GPU overlap
// with them. A request for a scenario supersedes that scenario's older request still waiting
// in the queue. Every request is computed by the same deterministic kernels, so its result is
// the same alone and in a mix.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/vpm.h"
#include "vpm_trace.cuh"

namespace vpm {
vpm_status report_error(vpm_status st, const char *msg);
size_t rollout_scratch_bytes(const vpm_state *s, int K, int H, int advance);
double rollout_work_estimate(const vpm_state *s, int K, int H, int advance);
cudaError_t lib_malloc_async(void **p, size_t bytes, cudaStream_t s);
size_t lib_pool_idle_bytes();
}

static vpm_status sfail(vpm_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return vpm::report_error(st, buf);
}

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    long long ticket = 0;
    int scenario = 0, K = 0, H = 0, advance_steps = 0;
    float lambda = 1.f, advance_u = 0.f;
    std::vector<float> mu, eps;
    size_t bytes = 0;                 // device bytes the request holds while in flight
    size_t buf_bytes = 0;             // of which its own buffers (the rest: rollout scratch)
    double work = 0;                  // estimated pair interactions (least-work-first admission)
    double t_submit = 0, t_start = 0, t_done = 0;
};

struct Result {
    int status = VPM_OK;
    Request req;
    float j_min = 0.f;
    std::vector<float> mu;
};

struct Slot {
    bool busy = false;
    bool small = false;               // the current request runs on the small requests' lane
    cudaStream_t stream = nullptr;    // default priority
    cudaStream_t stream_hi = nullptr; // highest priority (the small requests' lane), if enabled
    cudaStream_t active = nullptr;    // the current request's stream
    cudaEvent_t done = nullptr;
    float *pinned = nullptr;          // eps + mu in, mu + costs out
    size_t pinned_floats = 0;
    float *d_buf = nullptr;           // eps, controls, costs, weights, mu (stream-ordered)
    Request req;
};

}  // namespace

struct vpm_server {
    vpm_server_config cfg;
    int device = 0;
    size_t budget = 0, in_flight_bytes = 0;   // budget: the configured cap (SIZE_MAX: none)
    size_t reserve = 0, total_mem = 0;       // device memory admission leaves free, and the total
    long long rollout_budget = 0, in_flight_rollouts = 0;
    long long in_flight_small = 0;            // of which on the small requests' lane
    Clock::time_point t0;
    std::vector<vpm_state *> scenarios;
    std::vector<int> scenario_busy;
    std::vector<Slot> slots;
    std::deque<Request> queue;
    std::map<long long, Result> done;
    long long next_ticket = 1;
    long long completed_rollouts = 0;
    std::mutex m;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::thread worker;

    double now_ms() const
    {
        return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
    }
};

static size_t request_bytes(int K, int H)
{
    // eps, controls (K x H each), costs, weights (K each), mu (H): binary32
    return sizeof(float) * (2 * (size_t)K * H + 2 * (size_t)K + (size_t)H);
}

// Enqueues one request on its slot's stream. Called by the worker with the lock held.
static vpm_status start_request(vpm_server *s, Slot &sl, const Request &r)
{
    vpm::TraceRange tr("server: start request");
    const int K = r.K, H = r.H;
    float *pin = sl.pinned;
    memcpy(pin, r.eps.data(), sizeof(float) * (size_t)K * H);
    memcpy(pin + (size_t)K * H, r.mu.data(), sizeof(float) * H);
    cudaError_t e = vpm::lib_malloc_async((void **)&sl.d_buf, r.buf_bytes, sl.active);
    if (e) { cudaGetLastError(); return sfail(VPM_ERR_OOM, "server: allocation: %s", cudaGetErrorString(e)); }
    float *d_eps = sl.d_buf, *d_ctrl = d_eps + (size_t)K * H, *d_costs = d_ctrl + (size_t)K * H;
    float *d_w = d_costs + K, *d_mu = d_w + K;
    e = cudaMemcpyAsync(d_eps, pin, sizeof(float) * (size_t)K * H, cudaMemcpyHostToDevice, sl.active);
    if (!e) e = cudaMemcpyAsync(d_mu, pin + (size_t)K * H, sizeof(float) * H, cudaMemcpyHostToDevice, sl.active);
    if (e) { cudaGetLastError(); return sfail(VPM_ERR_CUDA, "server: upload: %s", cudaGetErrorString(e)); }
    vpm_state *st = s->scenarios[r.scenario];
    vpm_status v = VPM_OK;
    for (int k = 0; k < r.advance_steps && v == VPM_OK; ++k)
        v = vpm_step(st, (double)r.advance_u, nullptr, nullptr, nullptr, nullptr, sl.active);
    if (v == VPM_OK) v = mppi_perturb(d_mu, d_eps, K, H, d_ctrl, sl.active);
    if (v == VPM_OK) v = vpm_rollout_batch(st, K, H, d_ctrl, d_costs, nullptr, nullptr, nullptr, nullptr, sl.active);
    if (v == VPM_OK) v = mppi_weights(d_costs, K, r.lambda, d_w, sl.active);
    if (v == VPM_OK) v = mppi_update(d_w, d_ctrl, K, H, d_mu, sl.active);
    if (v != VPM_OK) return v;
    e = cudaMemcpyAsync(pin, d_mu, sizeof(float) * H, cudaMemcpyDeviceToHost, sl.active);
    if (!e) e = cudaMemcpyAsync(pin + H, d_costs, sizeof(float) * K, cudaMemcpyDeviceToHost, sl.active);
    if (!e) e = cudaFreeAsync(sl.d_buf, sl.active);
    if (!e) e = cudaEventRecord(sl.done, sl.active);
    if (e) { cudaGetLastError(); return sfail(VPM_ERR_CUDA, "server: enqueue: %s", cudaGetErrorString(e)); }
    return VPM_OK;
}

static void finish(vpm_server *s, const Request &r, int status, const float *mu, float jmin)
{
    Result res;
    res.status = status;
    res.req = r;
    res.req.eps.clear();
    res.req.eps.shrink_to_fit();
    res.req.t_done = s->now_ms();
    res.j_min = jmin;
    if (mu) res.mu.assign(mu, mu + r.H);
    s->done[r.ticket] = std::move(res);
    s->cv_done.notify_all();
}

// Device memory a request can take now: what the device has free plus what the library's pool
// holds reserved and unused, less the reserve. Read at every admission, so memory that other
// code in the process allocates or frees after the server was made counts.
static size_t live_available(const vpm_server *s)
{
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const size_t avail = free_b + vpm::lib_pool_idle_bytes();
    return avail > s->reserve ? avail - s->reserve : 0;
}

static void worker_loop(vpm_server *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->m);
    while (!s->stop) {
        bool progressed = false;
        // completions
        for (auto &sl : s->slots) {
            if (!sl.busy) continue;
            cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) continue;
            const Request &r = sl.req;
            int status = VPM_OK;
            if (q != cudaSuccess) {
                cudaGetLastError();
                status = VPM_ERR_CUDA;
            } else if (vpm_state_status(s->scenarios[r.scenario], sl.active) != VPM_OK) {
                status = VPM_ERR_NONFINITE;
            }
            float jmin = INFINITY;
            for (int i = 0; i < r.K; ++i) jmin = fminf(jmin, sl.pinned[r.H + i]);
            s->completed_rollouts += r.K;
            finish(s, r, status, sl.pinned, jmin);
            s->in_flight_bytes -= r.bytes;
            s->in_flight_rollouts -= r.K;
            if (sl.small) s->in_flight_small -= r.K;
            s->scenario_busy[r.scenario] = 0;
            sl.busy = false;
            progressed = true;
        }
        // least work first: among the queued requests whose scenario is idle and whose bytes fit,
        // the one with the fewest estimated pair interactions, unless one has waited longer than
        // max_wait_ms (then the longest-waiting of those); admission stops at a request that would
        // overfill the device, as in arrival order
        while (s->cfg.policy == VPM_ADMIT_LEAST_WORK && !s->queue.empty()) {
            Slot *free_slot = nullptr;
            for (auto &sl : s->slots)
                if (!sl.busy) { free_slot = &sl; break; }
            if (!free_slot) break;
            const double now = s->now_ms();
            const size_t avail = live_available(s);
            auto least = s->queue.end(), aged = s->queue.end();
            for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
                if (s->scenario_busy[it->scenario] || s->in_flight_bytes + it->bytes > s->budget ||
                    it->bytes > avail)
                    continue;
                if (s->cfg.max_wait_ms > 0 && now - it->t_submit > s->cfg.max_wait_ms && aged == s->queue.end())
                    aged = it;                // the queue is in arrival order
                if (least == s->queue.end() || it->work < least->work) least = it;
            }
            // a request fits its lane: the small requests' lane (if enabled) by its own rollouts,
            // the others by theirs, whatever the other lane holds
            const long long normal = s->in_flight_rollouts - s->in_flight_small;
            auto is_small = [&](const Request &q) { return s->cfg.small_rollouts > 0 && q.K <= s->cfg.small_rollouts; };
            auto fits = [&](const Request &q) {
                if (is_small(q)) return s->in_flight_small == 0 || s->in_flight_small + q.K <= s->rollout_budget;
                return normal == 0 || normal + q.K <= s->rollout_budget;
            };
            auto it = aged != s->queue.end() ? aged : least;
            if (it == s->queue.end()) break;
            if (!fits(*it)) {
                // the small requests' lane still admits its least-work candidate
                auto sm = s->queue.end();
                for (auto q = s->queue.begin(); q != s->queue.end(); ++q) {
                    if (!is_small(*q) || s->scenario_busy[q->scenario] || s->in_flight_bytes + q->bytes > s->budget ||
                        q->bytes > avail)
                        continue;
                    if (sm == s->queue.end() || q->work < sm->work) sm = q;
                }
                if (sm == s->queue.end() || !fits(*sm)) break;
                it = sm;
            }
            const bool small = is_small(*it);
            Request r = std::move(*it);
            s->queue.erase(it);
            r.t_start = s->now_ms();
            free_slot->small = small;
            free_slot->active = small && free_slot->stream_hi ? free_slot->stream_hi : free_slot->stream;
            vpm_status v = start_request(s, *free_slot, r);
            if (v != VPM_OK) {
                finish(s, r, v, nullptr, 0.f);
                continue;
            }
            free_slot->req = std::move(r);
            free_slot->req.eps.clear();
            free_slot->busy = true;
            s->in_flight_bytes += free_slot->req.bytes;
            s->in_flight_rollouts += free_slot->req.K;
            if (small) s->in_flight_small += free_slot->req.K;
            s->scenario_busy[free_slot->req.scenario] = 1;
            progressed = true;
        }
        // admission in arrival order: free slot, idle scenario, memory budget
        for (auto it = s->queue.begin(); s->cfg.policy != VPM_ADMIT_LEAST_WORK && it != s->queue.end();) {
            Slot *free_slot = nullptr;
            for (auto &sl : s->slots)
                if (!sl.busy) { free_slot = &sl; break; }
            if (!free_slot) break;
            const bool fits_rollouts = s->in_flight_rollouts == 0 ||
                                       s->in_flight_rollouts + it->K <= s->rollout_budget;
            if (!fits_rollouts) break;        // keep arrival order for work that fills the device
            if (s->scenario_busy[it->scenario] || s->in_flight_bytes + it->bytes > s->budget ||
                it->bytes > live_available(s)) {
                ++it;
                continue;
            }
            Request r = std::move(*it);
            it = s->queue.erase(it);
            r.t_start = s->now_ms();
            free_slot->small = false;
            free_slot->active = free_slot->stream;
            vpm_status v = start_request(s, *free_slot, r);
            if (v != VPM_OK) {
                finish(s, r, v, nullptr, 0.f);
                continue;
            }
            free_slot->req = std::move(r);
            free_slot->req.eps.clear();
            free_slot->busy = true;
            s->in_flight_bytes += free_slot->req.bytes;
            s->in_flight_rollouts += free_slot->req.K;
            s->scenario_busy[free_slot->req.scenario] = 1;
            progressed = true;
        }
        bool any_busy = false;
        for (auto &sl : s->slots) any_busy |= sl.busy;
        if (!progressed) {
            // busy: poll the device again shortly; requests waiting for device memory that other
            // code holds: look again every half millisecond; idle: sleep until a submission
            if (any_busy)
                s->cv_work.wait_for(lk, std::chrono::microseconds(50));
            else if (!s->queue.empty())
                s->cv_work.wait_for(lk, std::chrono::microseconds(500));
            else
                s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty(); });
        }
    }
}

extern "C" vpm_status vpm_server_create(const vpm_server_config *cfg, vpm_server **out)
{
    if (!cfg || !out || cfg->max_inflight < 1 || cfg->max_rollouts < 1 || cfg->max_horizon < 1)
        return sfail(VPM_ERR_INVALID, "vpm_server_create: need max_inflight, max_rollouts, max_horizon >= 1");
    if (cfg->policy != VPM_ADMIT_ARRIVAL && cfg->policy != VPM_ADMIT_LEAST_WORK)
        return sfail(VPM_ERR_INVALID, "vpm_server_create: unknown admission policy %d", cfg->policy);
    if (cfg->small_rollouts < 0 || (cfg->small_rollouts > 0 && cfg->policy != VPM_ADMIT_LEAST_WORK))
        return sfail(VPM_ERR_INVALID, "vpm_server_create: small_rollouts needs VPM_ADMIT_LEAST_WORK and must be >= 0");
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) {
        cudaGetLastError();
        return sfail(VPM_ERR_CUDA, "no CUDA device available");
    }
    vpm_server *s = new vpm_server();
    s->cfg = *cfg;
    s->t0 = Clock::now();
    cudaGetDevice(&s->device);
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    s->total_mem = total_b;
    s->reserve = total_b / 50 > ((size_t)1 << 30) ? total_b / 50 : ((size_t)1 << 30);
    s->budget = cfg->hbm_budget ? cfg->hbm_budget : ~(size_t)0;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
    s->rollout_budget = cfg->max_inflight_rollouts > 0 ? cfg->max_inflight_rollouts : (long long)sms * 7;
    s->slots.resize(cfg->max_inflight);
    const size_t pf = (size_t)cfg->max_rollouts * cfg->max_horizon + cfg->max_horizon + cfg->max_rollouts;
    for (auto &sl : s->slots) {
        cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (!e && cfg->small_rollouts > 0) {
            int least = 0, greatest = 0;
            e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
            if (!e) e = cudaStreamCreateWithPriority(&sl.stream_hi, cudaStreamNonBlocking, greatest);
        }
        sl.active = sl.stream;
        if (!e) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (!e) e = cudaMallocHost((void **)&sl.pinned, sizeof(float) * pf);
        if (e) {
            cudaGetLastError();
            vpm_server_destroy(s);
            return sfail(VPM_ERR_OOM, "vpm_server_create: %s", cudaGetErrorString(e));
        }
        sl.pinned_floats = pf;
    }
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return VPM_OK;
}

extern "C" vpm_status vpm_server_add_scenario(vpm_server *s, const vpm_params *params,
                                              const double *h_particles, int n, int capacity,
                                              const double *h_glider7, int *scenario)
{
    if (!s || !scenario) return sfail(VPM_ERR_INVALID, "vpm_server_add_scenario: null argument");
    std::lock_guard<std::mutex> lk(s->m);
    vpm_state *st = nullptr;
    vpm_status v = vpm_state_create(params, h_particles, n, capacity, h_glider7, &st, nullptr);
    if (v != VPM_OK) return v;
    s->scenarios.push_back(st);
    s->scenario_busy.push_back(0);
    *scenario = (int)s->scenarios.size() - 1;
    return VPM_OK;
}

extern "C" vpm_status vpm_server_submit(vpm_server *s, int scenario, int K, int H,
                                        const float *h_mu, const float *h_eps, float lambda,
                                        int advance_steps, float advance_u, long long *ticket)
{
    if (!s || !h_eps || !ticket) return sfail(VPM_ERR_INVALID, "vpm_server_submit: null argument");
    if (K < 1 || H < 1 || K > s->cfg.max_rollouts || H > s->cfg.max_horizon || advance_steps < 0 ||
        !(lambda > 0.f))
        return sfail(VPM_ERR_INVALID, "vpm_server_submit: K, H outside the server's limits or lambda <= 0");
    Request r;
    r.K = K;
    r.H = H;
    r.scenario = scenario;
    r.lambda = lambda;
    r.advance_steps = advance_steps;
    r.advance_u = advance_u;
    r.buf_bytes = request_bytes(K, H);
    r.eps.assign(h_eps, h_eps + (size_t)K * H);
    r.mu.assign(H, 0.f);
    if (h_mu) r.mu.assign(h_mu, h_mu + H);
    std::lock_guard<std::mutex> lk(s->m);
    if (scenario < 0 || scenario >= (int)s->scenarios.size())
        return sfail(VPM_ERR_INVALID, "vpm_server_submit: unknown scenario %d", scenario);
    r.bytes = r.buf_bytes + vpm::rollout_scratch_bytes(s->scenarios[scenario], K, H, advance_steps);
    r.work = vpm::rollout_work_estimate(s->scenarios[scenario], K, H, advance_steps);
    if (r.bytes > s->budget || r.bytes + s->reserve > s->total_mem)
        return sfail(VPM_ERR_CAPACITY, "vpm_server_submit: request needs %zu bytes; budget %zu, device %zu less %zu "
                     "kept free", r.bytes, s->budget, s->total_mem, s->reserve);
    r.ticket = s->next_ticket++;
    r.t_submit = s->now_ms();
    // the newest request for a scenario supersedes the one still waiting in the queue
    for (auto it = s->queue.begin(); it != s->queue.end(); ++it)
        if (it->scenario == scenario) {
            finish(s, *it, VPM_ERR_BUSY, nullptr, 0.f);
            s->queue.erase(it);
            break;
        }
    s->queue.push_back(std::move(r));
    *ticket = s->next_ticket - 1;
    s->cv_work.notify_one();
    return VPM_OK;
}

extern "C" vpm_status vpm_server_poll(vpm_server *s, long long ticket, int timeout_ms,
                                      vpm_server_result *out, float *h_mu_out)
{
    if (!s || !out) return sfail(VPM_ERR_INVALID, "vpm_server_poll: null argument");
    std::unique_lock<std::mutex> lk(s->m);
    auto ready = [&] { return s->done.count(ticket) > 0; };
    if (!ready()) {
        if (timeout_ms == 0) return VPM_ERR_BUSY;
        if (timeout_ms < 0)
            s->cv_done.wait(lk, ready);
        else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
            return VPM_ERR_TIMEOUT;
    }
    Result &r = s->done[ticket];
    out->status = r.status;
    out->scenario = r.req.scenario;
    out->K = r.req.K;
    out->H = r.req.H;
    out->t_submit_ms = r.req.t_submit;
    out->t_start_ms = r.req.t_start;
    out->t_done_ms = r.req.t_done;
    out->j_min = r.j_min;
    if (h_mu_out && !r.mu.empty()) memcpy(h_mu_out, r.mu.data(), sizeof(float) * r.mu.size());
    s->done.erase(ticket);
    return VPM_OK;
}

extern "C" vpm_status vpm_server_request_bytes(vpm_server *s, int scenario, int K, int H,
                                               int advance_steps, size_t *bytes)
{
    if (!s || !bytes || K < 1 || H < 1 || advance_steps < 0)
        return sfail(VPM_ERR_INVALID, "vpm_server_request_bytes: null, K or H < 1, or advance_steps < 0");
    std::lock_guard<std::mutex> lk(s->m);
    if (scenario < 0 || scenario >= (int)s->scenarios.size())
        return sfail(VPM_ERR_INVALID, "vpm_server_request_bytes: unknown scenario %d", scenario);
    *bytes = request_bytes(K, H) + vpm::rollout_scratch_bytes(s->scenarios[scenario], K, H, advance_steps);
    return VPM_OK;
}

extern "C" vpm_status vpm_server_stats(vpm_server *s, long long *completed_rollouts,
                                       int *queued, int *in_flight, size_t *in_flight_bytes)
{
    if (!s) return sfail(VPM_ERR_INVALID, "null server");
    std::lock_guard<std::mutex> lk(s->m);
    if (completed_rollouts) *completed_rollouts = s->completed_rollouts;
    if (queued) *queued = (int)s->queue.size();
    int b = 0;
    for (auto &sl : s->slots) b += sl.busy;
    if (in_flight) *in_flight = b;
    if (in_flight_bytes) *in_flight_bytes = s->in_flight_bytes;
    return VPM_OK;
}

extern "C" vpm_status vpm_server_read_scenario(vpm_server *s, int scenario, double *h_particles,
                                               int *n_out, double *h_glider7)
{
    if (!s) return sfail(VPM_ERR_INVALID, "null server");
    std::unique_lock<std::mutex> lk(s->m);
    if (scenario < 0 || scenario >= (int)s->scenarios.size())
        return sfail(VPM_ERR_INVALID, "unknown scenario");
    s->cv_done.wait(lk, [&] { return !s->scenario_busy[scenario]; });
    for (auto &r : s->queue)
        if (r.scenario == scenario) return sfail(VPM_ERR_BUSY, "scenario has a queued request");
    return vpm_state_read(s->scenarios[scenario], h_particles, n_out, h_glider7, nullptr, nullptr);
}

extern "C" vpm_status vpm_server_destroy(vpm_server *s)
{
    if (!s) return VPM_OK;
    {
        std::lock_guard<std::mutex> lk(s->m);
        s->stop = true;
        s->cv_work.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    cudaDeviceSynchronize();
    for (auto &sl : s->slots) {
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.stream_hi) cudaStreamDestroy(sl.stream_hi);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.pinned) cudaFreeHost(sl.pinned);
    }
    for (auto *st : s->scenarios) vpm_state_destroy(st);
    cudaGetLastError();
    delete s;
    return VPM_OK;
}
