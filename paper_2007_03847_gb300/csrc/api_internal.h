// Entry points shared between the library's own translation units.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "../../include/fastmc.h"

namespace fmc {

// Deep copy of a scenario, so that the caller's arrays may go away (requests of
// the server, scenarios of a batch).
struct OwnedScenario {
    fmc_scenario s{};
    std::vector<double> G, B, Ginf, Binf, H, D, E, Pm, theta, sigma, inject;
    std::vector<fmc_ito> ito;

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
        if (in.ito) {
            ito.assign(in.ito, in.ito + d);
            s.ito = ito.data();
        }
    }
};



// Contexts used on one stream only grow their workspace in stream order on it
// (no device-wide synchronisation); the server's contexts.
void set_stream_ordered(fmc_ctx* ctx, bool on);

// Frees the workspace buffers that scale with the samples or the horizon (in
// stream order on st for a stream-ordered context).
int release_workspace(fmc_ctx* ctx, cudaStream_t st);

// Grows ctx's workspace to what simulate_moments needs for `count` samples of s
// (without solving anything), on stream st when the context is stream-ordered.
int reserve_workspace(fmc_ctx* ctx, const fmc_scenario* s, int32_t path, int64_t count, cudaStream_t st);

// fmc_simulate with a choice of how the fused kernel combines its per-time sums:
// per_tile_partials = true writes FP32 partials per 128-sample tile and adds them
// in a fixed order (deterministic); false adds them with FP64 atomics (no
// partial buffer; the order of the FP64 additions is not fixed).
int simulate_moments(fmc_ctx* ctx, const fmc_scenario* s, int32_t path, double* mean_dev, double* var_dev,
                     bool per_tile_partials, cudaStream_t st);

// simulate_moments for R independent designs of the same scenario in one launch:
// replicate k draws its design of s->N samples from seeds[k]; its moments go to
// mean_dev + k (Nt+1) 2n and var_dev + k (Nt+1) 2n, equal to simulate_moments of
// the scenario with that seed (the same tiles reduced in the same order).
// FMC_EUNSUPPORTED unless the path is fused, the design a KL design without the
// correlation-reducing permutation and s->N a multiple of 128 (the caller then
// runs the replicates one by one).
int simulate_moments_replicates(fmc_ctx* ctx, const fmc_scenario* s, int32_t path, int R, const uint64_t* seeds,
                                double* mean_dev, double* var_dev, cudaStream_t st);

// fmc_device_status for the work enqueued on one stream: waits for that stream
// only (not the device), so concurrent requests of the server keep running.
int device_status_on(fmc_ctx* ctx, cudaStream_t st);

}  // namespace fmc
