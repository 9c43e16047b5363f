// Serving loop: uncertainty-evaluation requests admitted by device memory and
// run concurrently, each on its own slot (stream, workspace, library context),
// so that requests arriving while others run start as soon as a slot and
// memory are free and their kernels overlap on the GPU (continuous batching).
// Results go to caller-owned device buffers; latency is measured from submit
// to completion on the device.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
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

struct Request {
    uint64_t id = 0;
    std::unique_ptr<fmc::OwnedScenario> scen;
    int32_t path = FMC_PATH_FUSED;
    double* mean = nullptr;
    double* var = nullptr;
    size_t bytes = 0;  // device memory charged against the budget
    int status = FMC_NOT_READY;
    bool started = false;
    std::string error;
    Clock::time_point t_submit, t_start, t_done;
    // target-error requests (fmc_submit_target)
    double tol_E = 0.0, tol_Var = 0.0;
    int64_t max_N = 0;
    int replicates = 1;
    int64_t n_used = 0;
    double err_E = -1.0, err_Var = -1.0;
    int target_met = 0;
};

constexpr int kReplicates = 4;
// the largest per-tile partial buffer a request's merged replicate launches may use
constexpr int64_t kMergedPartBytes = (int64_t)2 << 30;

// Per-tile partial bytes of a merged launch of `samples` samples of s.
int64_t merged_part_bytes(const fmc_scenario& s, int64_t samples)
{
    const int64_t Nt = (int64_t)std::llround(s.T / s.dt);
    return (samples + 127) / 128 * (Nt + 1) * 6 * (int64_t)s.n * 4;
}

// The largest per-replicate design (N growing fourfold up to nb) whose round runs
// as one merged launch, or 0 when the request's rounds never merge: the fused
// path, a KL design without the correlation-reducing permutation, tile-aligned
// designs, and per-tile partials within kMergedPartBytes (separate launches add
// their sums with FP64 atomics and need no partials).
int64_t merge_limit(const fmc_scenario& s, int32_t path, int64_t nb)
{
    if (path != FMC_PATH_FUSED || s.sampling == FMC_SRS_EM || s.correlation == FMC_CORR_RANK || s.N < 128 ||
        s.N % 128 != 0)
        return 0;
    int64_t lim = 0;
    for (int64_t n = s.N; n <= nb; n *= 4)
        if (merged_part_bytes(s, kReplicates * n) <= kMergedPartBytes) lim = n;
    return lim;
}

// splitmix64: seeds of the replicate designs
uint64_t mix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// Runs a target-error request on the slot's contexts and streams (see
// fmc_submit_target): rounds of kReplicates independent designs, n growing
// fourfold until the replicate spread meets the targets or max_N is reached.
// A round's designs share one launch (one equilibrium, one design block of
// R n samples, per-replicate sums) where simulate_moments_replicates takes the
// request; otherwise each runs on its own context and stream, concurrently.
int run_target(fmc_ctx* const* rctx, const cudaStream_t* rst, Request* r)
{
    cudaStream_t st = rst[0];
    fmc_scenario s = r->scen->s;
    const int R = kReplicates;
    const int64_t Nt = (int64_t)std::llround(s.T / s.dt);
    const size_t cols = (size_t)(Nt + 1) * 2 * (size_t)s.n;
    double* dbuf = nullptr;
    if (cudaMallocAsync((void**)&dbuf, sizeof(double) * cols * 2 * R, st) != cudaSuccess) return FMC_ENOMEM;
    // the largest design a round of this request may draw, per replicate, and
    // the largest whose round runs as one merged launch (merge_limit)
    int64_t nb = s.N < 2 ? 2 : s.N;
    while (4 * (int64_t)R * nb <= r->max_N) nb *= 4;
    const int64_t n_mm = merge_limit(s, r->path, nb);
    // workspaces sized once for the largest round of each form, so that no round
    // grows (and reallocates) them: the merged rounds' on the first context; the
    // separate rounds' on every context, reserved (after the merged workspace is
    // released) when the first of them comes
    bool separate_ready = false;
    auto reserve_for = [&](int count, int64_t samples) -> int {
        fmc_scenario big = s;
        big.N = samples;
        for (int k = 0; k < count; ++k) {
            const int rc0 = fmc::reserve_workspace(rctx[k], &big, r->path, samples, rst[k]);
            if (rc0 != FMC_OK) {
                r->error = fmc_last_error(rctx[k]);
                return rc0;
            }
        }
        return FMC_OK;
    };
    {
        const int rc0 = n_mm > 0 ? reserve_for(1, (int64_t)R * n_mm) : reserve_for(R, nb);
        separate_ready = n_mm == 0;
        if (rc0 != FMC_OK) {
            cudaFreeAsync(dbuf, st);
            return rc0;
        }
    }
    std::vector<double> hm(cols * R), hv(cols * R), mbar(cols), vbar(cols);
    const uint64_t seed0 = s.seed;
    int64_t n = s.N < 2 ? 2 : s.N;
    int rc = FMC_OK;
    for (int round = 0;; ++round) {
        if (cudaStreamSynchronize(st) != cudaSuccess) {  // the scratch is ready for the replicates
            rc = FMC_ECUDA;
            break;
        }
        s.N = n;
        uint64_t seeds[kReplicates];
        for (int k = 0; k < R; ++k) seeds[k] = mix64(seed0 ^ ((uint64_t)(round * R + k + 1) << 32));
        const bool merged = n <= n_mm;
        if (!merged && !separate_ready) {
            if ((rc = fmc::release_workspace(rctx[0], rst[0])) == FMC_OK) rc = reserve_for(R, nb);
            separate_ready = true;
            if (rc != FMC_OK) break;
        }
        if (merged) {
            rc = fmc::simulate_moments_replicates(rctx[0], &s, r->path, R, seeds, dbuf, dbuf + (size_t)R * cols, st);
            if (rc != FMC_OK) r->error = fmc_last_error(rctx[0]);
        }
        for (int k = 0; k < R && rc == FMC_OK && !merged; ++k) {
            s.seed = seeds[k];
            rc = fmc::simulate_moments(rctx[k], &s, r->path, dbuf + (size_t)k * cols, dbuf + (size_t)(R + k) * cols,
                                       false, rst[k]);
            if (rc != FMC_OK) r->error = fmc_last_error(rctx[k]);
        }
        for (int k = 0; k < R; ++k)
            if (cudaStreamSynchronize(rst[k]) != cudaSuccess) rc = FMC_ECUDA;
        if (rc != FMC_OK) break;
        if (cudaMemcpyAsync(hm.data(), dbuf, sizeof(double) * cols * R, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(hv.data(), dbuf + cols * R, sizeof(double) * cols * R, cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            rc = FMC_ECUDA;
            break;
        }
        double sd_m = 0.0, sd_v = 0.0, scale_m = 0.0, scale_v = 0.0;
        for (size_t c = 0; c < cols; ++c) {
            double am = 0.0, av = 0.0;
            for (int k = 0; k < R; ++k) {
                am += hm[k * cols + c];
                av += hv[k * cols + c];
            }
            am /= R;
            av /= R;
            double qm = 0.0, qv = 0.0;
            for (int k = 0; k < R; ++k) {
                qm += (hm[k * cols + c] - am) * (hm[k * cols + c] - am);
                qv += (hv[k * cols + c] - av) * (hv[k * cols + c] - av);
            }
            mbar[c] = am;
            vbar[c] = av;
            sd_m = std::fmax(sd_m, std::sqrt(qm / (R - 1)));
            sd_v = std::fmax(sd_v, std::sqrt(qv / (R - 1)));
            scale_m = std::fmax(scale_m, std::sqrt(std::fmax(av, 0.0)));
            scale_v = std::fmax(scale_v, av);
        }
        r->err_E = scale_m > 0 ? sd_m / std::sqrt((double)R) / scale_m : 0.0;
        r->err_Var = scale_v > 0 ? sd_v / std::sqrt((double)R) / scale_v : 0.0;
        r->n_used = (int64_t)R * n;
        r->replicates = R;
        r->target_met = (r->tol_E <= 0 || r->err_E <= r->tol_E) && (r->tol_Var <= 0 || r->err_Var <= r->tol_Var);
        if (r->target_met || 4 * (int64_t)R * n > r->max_N) break;
        n *= 4;
    }
    if (rc == FMC_OK &&
        (cudaMemcpyAsync(r->mean, mbar.data(), sizeof(double) * cols, cudaMemcpyHostToDevice, st) != cudaSuccess ||
         cudaMemcpyAsync(r->var, vbar.data(), sizeof(double) * cols, cudaMemcpyHostToDevice, st) != cudaSuccess))
        rc = FMC_ECUDA;
    cudaFreeAsync(dbuf, st);
    return rc;
}

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
    std::vector<fmc_ctx*> ctxs;  // kReplicates per slot
    std::string err;
};

static void worker_loop(fmc_server* srv, int slot)
{
    fmc_ctx* const* rctx = &srv->ctxs[(size_t)slot * kReplicates];
    fmc_ctx* ctx = rctx[0];
    cudaSetDevice(srv->device);
    cudaStream_t rst[kReplicates];
    for (int k = 0; k < kReplicates; ++k) cudaStreamCreateWithFlags(&rst[k], cudaStreamNonBlocking);
    cudaStream_t st = rst[0];
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
        int rc;
        if (r->tol_E > 0 || r->tol_Var > 0) {
            rc = run_target(rctx, rst, r);
        } else {
            rc = fmc::simulate_moments(ctx, &r->scen->s, r->path, r->mean, r->var, false, st);
            r->n_used = r->scen->s.N;
        }
        if (rc == FMC_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = FMC_ECUDA;
        // status words of this slot's streams only (no device-wide wait)
        for (int k = 0; k < kReplicates && rc == FMC_OK; ++k) {
            rc = fmc::device_status_on(rctx[k], rst[k]);
            if (rc != FMC_OK) r->error = fmc_last_error(rctx[k]);
        }
        // the charge is released with the request, and so is the memory it paid
        // for: the slot's workspaces go back to the device's memory pool (in stream
        // order), where any slot's next allocation can reuse them
        for (int k = 0; k < kReplicates; ++k) fmc::release_workspace(rctx[k], rst[k]);
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            r->status = rc;
            if (rc != FMC_OK && r->error.empty()) r->error = fmc_last_error(ctx);
            r->t_done = Clock::now();
            srv->in_use -= r->bytes;
        }
        srv->cv_done.notify_all();
        srv->cv_work.notify_all();
    }
    for (int k = 0; k < kReplicates; ++k) cudaStreamDestroy(rst[k]);
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
    // keep freed workspace memory in the device's default pool for reuse by the
    // next requests instead of returning it to the driver at every synchronisation
    {
        cudaMemPool_t pool = nullptr;
        if (cudaSetDevice(device) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
            uint64_t keep = (uint64_t)mem_budget_bytes;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
    }
    for (int i = 0; i < slots * kReplicates; ++i) {
        fmc_ctx* c = nullptr;
        int rc = fmc_create(&c, device, 0);
        if (rc != FMC_OK) {
            for (fmc_ctx* x : srv->ctxs) fmc_destroy(x);
            delete srv;
            return rc;
        }
        fmc::set_stream_ordered(c, true);  // each is used on its worker's replicate stream only
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

static int submit_request(fmc_server* srv, const fmc_scenario* scen, int32_t path, double tol_E, double tol_Var,
                          int64_t max_N, double* mean_dev, double* var_dev, uint64_t* handle)
{
    if (!srv || !scen || !mean_dev || !var_dev || !handle) return FMC_EINVAL;
    if (path != FMC_PATH_FUSED && path != FMC_PATH_PLAIN) return FMC_EINVAL;
    if (scen->n < 1 || scen->d < 1 || scen->K < 1 || scen->N < 1 || !(scen->dt > 0) || !(scen->T > 0))
        return FMC_EINVAL;
    const bool target = tol_E > 0 || tol_Var > 0;
    if (target && (max_N < (int64_t)kReplicates * scen->N || !(tol_E >= 0) || !(tol_Var >= 0))) return FMC_EINVAL;
    auto r = std::make_unique<Request>();
    r->scen = std::make_unique<fmc::OwnedScenario>(*scen);
    r->path = path;
    r->mean = mean_dev;
    r->var = var_dev;
    r->tol_E = tol_E;
    r->tol_Var = tol_Var;
    r->max_N = max_N;
    // charged for the largest design it may draw, in each of its replicates, and
    // the per-tile partials of its largest merged round
    fmc_scenario largest = *scen;
    int64_t n_mm = 0;
    if (target) {
        int64_t n = scen->N;
        while (4 * (int64_t)kReplicates * n <= max_N) n *= 4;
        largest.N = n;
        n_mm = merge_limit(*scen, path, n);
    }
    r->bytes = request_bytes(largest, path) * (target ? (size_t)kReplicates : 1u) +
               (n_mm > 0 ? (size_t)merged_part_bytes(*scen, kReplicates * n_mm) : 0u);
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

int fmc_submit(fmc_server* srv, const fmc_scenario* scen, int32_t path, double* mean_dev, double* var_dev,
               uint64_t* handle)
{
    return submit_request(srv, scen, path, 0.0, 0.0, 0, mean_dev, var_dev, handle);
}

int fmc_submit_target(fmc_server* srv, const fmc_scenario* scen, int32_t path, double tol_E, double tol_Var,
                      int64_t max_N, double* mean_dev, double* var_dev, uint64_t* handle)
{
    if (!(tol_E > 0) && !(tol_Var > 0)) return FMC_EINVAL;
    return submit_request(srv, scen, path, tol_E, tol_Var, max_N, mean_dev, var_dev, handle);
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
    out->replicates = r->replicates;
    out->n_used = r->n_used;
    out->err_E = r->err_E;
    out->err_Var = r->err_Var;
    out->target_met = r->target_met;
    out->reserved = 0;
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
