// Serving loop: uncertainty-evaluation requests admitted by device memory and
// run concurrently, each on its own slot (stream, workspace, library context),
// so that requests arriving while others run start as soon as a slot and
// memory are free and their kernels overlap on the GPU (continuous batching).
// Results go to caller-owned device buffers; latency is measured from submit
// to completion on the device.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/fastmc.h"
#include "api_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

// Deep copy of a scenario (the caller's arrays may go away after submit).
struct OwnedScenario {
    fmc_scenario s{};
    std::vector<double> G, B, Ginf, Binf, H, D, E, Pm, theta, sigma, inject;

    explicit OwnedScenario(const fmc_scenario& in) : s(in)
    {
        const size_t n = (size_t)in.n, d = (size_t)in.d;
        auto cp = [](std::vector<double>& dst, const double* src, size_t k) {
            if (src) dst.assign(src, src + k);
        };
        cp(G, in.G, n * n);
        cp(B, in.B, n * n);
        cp(H, in.H, n);
        cp(D, in.D, n);
        cp(E, in.E, n);
        cp(Pm, in.Pm, n);
        cp(theta, in.theta, d);
        cp(sigma, in.sigma, d);
        cp(inject, in.inject, n * d);
        if (in.has_inf_bus) {
            cp(Ginf, in.Ginf, n);
            cp(Binf, in.Binf, n);
        }
        auto ptr = [](const std::vector<double>& v) -> const double* { return v.empty() ? nullptr : v.data(); };
        s.G = ptr(G);
        s.B = ptr(B);
        s.H = ptr(H);
        s.D = ptr(D);
        s.E = ptr(E);
        s.Pm = ptr(Pm);
        s.theta = ptr(theta);
        s.sigma = ptr(sigma);
        s.inject = ptr(inject);
        s.Ginf = ptr(Ginf);
        s.Binf = ptr(Binf);
    }
};

struct Request {
    uint64_t id = 0;
    std::unique_ptr<OwnedScenario> scen;
    int32_t path = FMC_PATH_FUSED;
    double* mean = nullptr;
    double* var = nullptr;
    size_t bytes = 0;  // device memory charged against the budget
    int status = FMC_NOT_READY;
    bool started = false;
    std::string error;
    Clock::time_point t_submit, t_start, t_done;
};

// Device bytes a request's workspace needs (the design, basis, partials,
// equilibrium and the plain path's buffers), rounded up generously.
size_t request_bytes(const fmc_scenario& s, int32_t path)
{
    const double Nt = s.dt > 0 ? s.T / s.dt : 0.0;
    const size_t n = (size_t)s.n, d = (size_t)s.d, K = (size_t)s.K, N = (size_t)s.N;
    const size_t Ks = (K + 7) / 8 * 8, Kp = (K + 31) / 32 * 32;
    const size_t Nt1 = (size_t)Nt + 1;
    size_t b = 4096 + (2 * n * n + 9 * n) * 8;
    if (path == FMC_PATH_PLAIN) {
        b += N * d * K * 4 + K * (size_t)Nt * 4 + N * d * (size_t)Nt * 4 + N * Nt1 * 2 * n * 4;
    } else {
        b += 2 * N * d * Ks * 2 + 2 * (size_t)Nt * Kp * 2;
    }
    return b + b / 8;
}

}  // namespace

struct fmc_server {
    int device = 0;
    size_t budget = 0;
    size_t in_use = 0;
    bool stopping = false;
    uint64_t next_id = 1;
    std::mutex mu;
    std::condition_variable cv_work;   // workers: a request may be admissible
    std::condition_variable cv_done;   // waiters: a request finished
    std::deque<uint64_t> queue;        // FIFO of waiting requests
    std::map<uint64_t, std::unique_ptr<Request>> reqs;
    std::vector<std::thread> workers;
    std::vector<fmc_ctx*> ctxs;
    std::string err;
};

static void worker_loop(fmc_server* srv, int slot)
{
    fmc_ctx* ctx = srv->ctxs[slot];
    cudaSetDevice(srv->device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    for (;;) {
        Request* r = nullptr;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            // the head of the queue runs as soon as its memory fits (FIFO: no
            // overtaking, so large requests are not starved)
            srv->cv_work.wait(lk, [&] {
                if (srv->stopping) return true;
                if (srv->queue.empty()) return false;
                Request* h = srv->reqs[srv->queue.front()].get();
                return srv->in_use + h->bytes <= srv->budget;
            });
            if (srv->stopping) break;
            r = srv->reqs[srv->queue.front()].get();
            srv->queue.pop_front();
            srv->in_use += r->bytes;
            r->started = true;
            r->t_start = Clock::now();
        }
        // moments summed with FP64 atomics: no per-tile partial buffers to hold
        int rc = fmc::simulate_moments(ctx, &r->scen->s, r->path, r->mean, r->var, false, st);
        if (rc == FMC_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = FMC_ECUDA;
        if (rc == FMC_OK) {
            int it = 0, kerr = 0;
            rc = fmc_device_status(ctx, &it, &kerr);
        }
        // the workspace stays with the slot; the charge is released with the request
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            r->status = rc;
            if (rc != FMC_OK) r->error = fmc_last_error(ctx);
            r->t_done = Clock::now();
            srv->in_use -= r->bytes;
        }
        srv->cv_done.notify_all();
        srv->cv_work.notify_all();
    }
    cudaStreamDestroy(st);
}

extern "C" {

int fmc_server_create(int device, int32_t slots, size_t mem_budget_bytes, fmc_server** out)
{
    if (!out || slots < 1 || slots > 64) return FMC_EINVAL;
    *out = nullptr;
    fmc_server* srv = new fmc_server();
    srv->device = device;
    if (mem_budget_bytes == 0) {
        size_t fr = 0, tot = 0;
        if (cudaSetDevice(device) != cudaSuccess || cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            delete srv;
            return FMC_ECUDA;
        }
        mem_budget_bytes = fr / 10 * 8;
    }
    srv->budget = mem_budget_bytes;
    for (int i = 0; i < slots; ++i) {
        fmc_ctx* c = nullptr;
        int rc = fmc_create(&c, device, 0);
        if (rc != FMC_OK) {
            for (fmc_ctx* x : srv->ctxs) fmc_destroy(x);
            delete srv;
            return rc;
        }
        srv->ctxs.push_back(c);
    }
    for (int i = 0; i < slots; ++i) srv->workers.emplace_back(worker_loop, srv, i);
    *out = srv;
    return FMC_OK;
}

int fmc_server_destroy(fmc_server* srv)
{
    if (!srv) return FMC_EINVAL;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stopping = true;
        for (uint64_t id : srv->queue) {
            Request* r = srv->reqs[id].get();
            r->status = FMC_ECANCELLED;
            r->t_done = Clock::now();
        }
        srv->queue.clear();
    }
    srv->cv_work.notify_all();
    srv->cv_done.notify_all();
    for (std::thread& t : srv->workers) t.join();
    for (fmc_ctx* c : srv->ctxs) fmc_destroy(c);
    delete srv;
    return FMC_OK;
}

int fmc_submit(fmc_server* srv, const fmc_scenario* scen, int32_t path, double* mean_dev, double* var_dev,
               uint64_t* handle)
{
    if (!srv || !scen || !mean_dev || !var_dev || !handle) return FMC_EINVAL;
    if (path != FMC_PATH_FUSED && path != FMC_PATH_PLAIN) return FMC_EINVAL;
    if (scen->n < 1 || scen->d < 1 || scen->K < 1 || scen->N < 1 || !(scen->dt > 0) || !(scen->T > 0))
        return FMC_EINVAL;
    auto r = std::make_unique<Request>();
    r->scen = std::make_unique<OwnedScenario>(*scen);
    r->path = path;
    r->mean = mean_dev;
    r->var = var_dev;
    r->bytes = request_bytes(*scen, path);
    r->t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->stopping) return FMC_ECANCELLED;
    if (r->bytes > srv->budget) return FMC_ENOMEM;  // could never be admitted
    r->id = srv->next_id++;
    *handle = r->id;
    srv->queue.push_back(r->id);
    srv->reqs[r->id] = std::move(r);
    srv->cv_work.notify_all();
    return FMC_OK;
}

static void fill_result(const Request* r, fmc_result* out)
{
    if (!out) return;
    out->status = r->status;
    auto us = [](Clock::time_point a, Clock::time_point b) {
        return (double)std::chrono::duration_cast<std::chrono::nanoseconds>(b - a).count() * 1e-3;
    };
    out->latency_us = us(r->t_submit, r->t_done);
    out->queue_us = r->started ? us(r->t_submit, r->t_start) : out->latency_us;
    out->device_bytes = (uint64_t)r->bytes;
    snprintf(out->message, sizeof out->message, "%s", r->error.c_str());
}

int fmc_poll(fmc_server* srv, uint64_t handle, fmc_result* out)
{
    if (!srv) return FMC_EINVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(handle);
    if (it == srv->reqs.end()) return FMC_EINVAL;
    Request* r = it->second.get();
    if (r->status == FMC_NOT_READY) return FMC_NOT_READY;
    fill_result(r, out);
    srv->reqs.erase(it);  // a finished request is reported once
    return FMC_OK;
}

int fmc_wait(fmc_server* srv, uint64_t handle, int64_t timeout_us, fmc_result* out)
{
    if (!srv) return FMC_EINVAL;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(handle);
    if (it == srv->reqs.end()) return FMC_EINVAL;
    Request* r = it->second.get();
    const auto deadline = Clock::now() + std::chrono::microseconds(timeout_us < 0 ? 0 : timeout_us);
    bool ok = srv->cv_done.wait_until(lk, deadline, [&] { return r->status != FMC_NOT_READY; });
    if (!ok) return FMC_ETIMEOUT;
    fill_result(r, out);
    srv->reqs.erase(handle);
    return FMC_OK;
}

int fmc_cancel(fmc_server* srv, uint64_t handle)
{
    if (!srv) return FMC_EINVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(handle);
    if (it == srv->reqs.end()) return FMC_EINVAL;
    Request* r = it->second.get();
    if (r->started) return r->status == FMC_NOT_READY ? FMC_EBUSY : FMC_OK;
    for (auto q = srv->queue.begin(); q != srv->queue.end(); ++q)
        if (*q == handle) {
            srv->queue.erase(q);
            break;
        }
    r->status = FMC_ECANCELLED;
    r->t_done = Clock::now();
    srv->cv_done.notify_all();
    srv->cv_work.notify_all();
    return FMC_OK;
}

int fmc_server_stats(fmc_server* srv, int32_t* queued, int32_t* running, size_t* bytes_in_use)
{
    if (!srv) return FMC_EINVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    int run = 0;
    for (auto& kv : srv->reqs)
        if (kv.second->started && kv.second->status == FMC_NOT_READY) ++run;
    if (queued) *queued = (int32_t)srv->queue.size();
    if (running) *running = run;
    if (bytes_in_use) *bytes_in_use = srv->in_use;
    return FMC_OK;
}

}  // extern "C"
