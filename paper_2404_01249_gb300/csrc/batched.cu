// fa_register_batched: many independent registrations (pairs x parameter
// sets) in one call, run concurrently on internal streams forked from the
// caller's stream.  Each concurrent slot owns a slice of the workspace and
// runs its jobs one after another; slices are sized for the largest job.
//
// Registrations are independent (Algorithm 1 runs per pair), so there is no
// data exchange between jobs.  Concurrency matters because the coarse levels
// of one registration fill only part of the GPU: jobs on other streams run in
// the gaps.
#include <stdio.h>

#include <mutex>
#include <vector>

#include "ops.h"
#include "register.h"
#include "validate.h"

namespace fa {

namespace {

constexpr int kMaxConcurrency = 32;
constexpr int kMaxDevices = 64;

std::mutex g_stream_mu;
cudaStream_t g_streams[kMaxDevices][kMaxConcurrency];

// The first n internal streams of the current device (created once, kept
// for the life of the process).
fa_status internal_streams(int n, cudaStream_t *out) {
    int dev = -1;
    FA_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("fa_register_batched: device ordinal %d is not supported", dev);
        return FA_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_stream_mu);
    for (int k = 0; k < n; ++k) {
        if (!g_streams[dev][k]) {
            cudaStream_t st = nullptr;
            cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreateWithFlags");
            g_streams[dev][k] = st;
        }
        out[k] = g_streams[dev][k];
    }
    return FA_OK;
}

__global__ void k_copy_status(const WsHeader *h, unsigned *out) { *out = h->status; }

size_t slot_bytes(int32_t n_pairs, const fa_vol *fixed, int32_t n_cfg, const fa_params *cfgs) {
    size_t b = 0;
    for (int i = 0; i < n_pairs; ++i)
        for (int c = 0; c < n_cfg; ++c) {
            const size_t j = register_ws_bytes(fixed[i].D, fixed[i].H, fixed[i].W, &cfgs[c]);
            if (j == 0) return 0;
            b = j > b ? j : b;
        }
    return (b + 255) & ~size_t(255);
}

fa_status check_counts(int32_t n_pairs, const fa_vol *fixed, int32_t n_cfg, const fa_params *cfgs,
                       int32_t concurrency) {
    if (n_pairs < 1 || n_cfg < 1 || !fixed || !cfgs) {
        set_error("fa_register_batched: need n_pairs >= 1, n_cfg >= 1 and non-NULL arrays");
        return FA_ERR_INVALID;
    }
    if (concurrency < 1 || concurrency > kMaxConcurrency) {
        set_error("fa_register_batched: concurrency must be in 1..%d (got %d)", kMaxConcurrency,
                  (int)concurrency);
        return FA_ERR_INVALID;
    }
    return FA_OK;
}

}  // namespace

}  // namespace fa

extern "C" size_t fa_register_batched_workspace_size(int32_t n_pairs, const fa_vol *fixed,
                                                     int32_t n_cfg, const fa_params *cfgs,
                                                     int32_t concurrency) {
    using namespace fa;
    clear_error();
    if (check_counts(n_pairs, fixed, n_cfg, cfgs, concurrency) != FA_OK) return 0;
    const int jobs = n_pairs * n_cfg;
    const int conc = concurrency < jobs ? concurrency : jobs;
    return slot_bytes(n_pairs, fixed, n_cfg, cfgs) * (size_t)conc;
}

extern "C" fa_status fa_register_batched(int32_t n_pairs, const fa_vol *fixed,
                                         const fa_vol *moving, int32_t n_cfg,
                                         const fa_params *cfgs, fa_vol *u_out,
                                         float *final_loss_dev, uint32_t *status_dev,
                                         int32_t concurrency, void *ws, size_t ws_bytes,
                                         void *stream) {
    using namespace fa;
    clear_error();
    FA_TRY(check_counts(n_pairs, fixed, n_cfg, cfgs, concurrency));
    if (!moving || !u_out) {
        set_error("fa_register_batched: moving and u_out must not be NULL");
        return FA_ERR_INVALID;
    }
    const int jobs = n_pairs * n_cfg;
    // every job is checked before anything is enqueued
    for (int i = 0; i < n_pairs; ++i)
        for (int c = 0; c < n_cfg; ++c) {
            const fa_status st = register_check(&fixed[i], &moving[i], &cfgs[c], &u_out[i * n_cfg + c]);
            if (st != FA_OK) {
                char msg[512];
                snprintf(msg, sizeof(msg), "%s", fa_last_error());
                set_error("fa_register_batched: pair %d, parameter set %d: %s", i, c, msg);
                return st;
            }
        }
    const int conc = concurrency < jobs ? concurrency : jobs;
    const size_t slot = slot_bytes(n_pairs, fixed, n_cfg, cfgs);
    FA_TRY(check_ws(ws, ws_bytes, slot * (size_t)conc, "fa_register_batched"));
    cudaStream_t st[kMaxConcurrency];
    FA_TRY(internal_streams(conc, st));
    cudaStream_t s = (cudaStream_t)stream;

    // fork: every slot stream starts after the work already on `stream`
    cudaEvent_t fork;
    FA_CUDA_TRY(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    cudaError_t e = cudaEventRecord(fork, s);
    for (int k = 0; k < conc && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(st[k], fork, 0);
    cudaEventDestroy(fork);
    FA_CUDA_TRY(e);

    fa_status result = FA_OK;
    for (int j = 0; j < jobs && result == FA_OK; ++j) {
        const int i = j / n_cfg, c = j % n_cfg, k = j % conc;
        char *w = (char *)ws + slot * (size_t)k;
        // jobs on concurrent streams take the four fused kernels: a
        // persistent launch needs its CTAs resident together
        fa_params pc = cfgs[c];
        if (pc.mode == FA_MODE_PERSISTENT) pc.mode = FA_MODE_FUSED;
        result = register_impl(&fixed[i], &moving[i], &pc, nullptr, &u_out[j],
                               final_loss_dev ? final_loss_dev + j : nullptr, nullptr, w, slot,
                               st[k], nullptr);
        if (result == FA_OK && status_dev) {
            k_copy_status<<<1, 1, 0, st[k]>>>((const WsHeader *)w, status_dev + j);
            note_launch();
            const cudaError_t le = cudaGetLastError();
            if (le != cudaSuccess) result = cuda_fail(le, "k_copy_status");
        }
    }
    // join: `stream` continues after every slot's jobs (also after a failure,
    // so that nothing enqueued is left unordered)
    for (int k = 0; k < conc; ++k) {
        cudaEvent_t done;
        cudaError_t je = cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
        if (je == cudaSuccess) je = cudaEventRecord(done, st[k]);
        if (je == cudaSuccess) je = cudaStreamWaitEvent(s, done, 0);
        if (je == cudaSuccess) cudaEventDestroy(done);
        if (je != cudaSuccess && result == FA_OK) result = cuda_fail(je, "fa_register_batched join");
    }
    return result;
}

// ------------------------------------------------------------------ lockstep
// All jobs of a wave advance together: every iteration is one launch per
// fused kernel over the tiles of every job in the wave (one per Gaussian
// radius and compose variant for K3 and K4), so the coarse levels of many
// registrations fill the GPU together.  Waves of `jobs_per_wave` jobs run one
// after another in the same workspace slices.

namespace fa {
namespace {

fa_status check_wave(int32_t jobs_per_wave) {
    if (jobs_per_wave < 1 || jobs_per_wave > kMaxLockstepJobs) {
        set_error("fa_register_batched_lockstep: jobs_per_wave must be in 1..%d (got %d)",
                  kMaxLockstepJobs, (int)jobs_per_wave);
        return FA_ERR_INVALID;
    }
    return FA_OK;
}

}  // namespace
}  // namespace fa

extern "C" size_t fa_register_lockstep_workspace_size(int32_t n_pairs, const fa_vol *fixed,
                                                      int32_t n_cfg, const fa_params *cfgs,
                                                      int32_t jobs_per_wave) {
    using namespace fa;
    clear_error();
    if (check_counts(n_pairs, fixed, n_cfg, cfgs, 1) != FA_OK || check_wave(jobs_per_wave) != FA_OK)
        return 0;
    const int jobs = n_pairs * n_cfg;
    const int wave = jobs_per_wave < jobs ? jobs_per_wave : jobs;
    return slot_bytes(n_pairs, fixed, n_cfg, cfgs) * (size_t)wave;
}

extern "C" fa_status fa_register_batched_lockstep(int32_t n_pairs, const fa_vol *fixed,
                                                  const fa_vol *moving, int32_t n_cfg,
                                                  const fa_params *cfgs, fa_vol *u_out,
                                                  float *final_loss_dev, uint32_t *status_dev,
                                                  int32_t jobs_per_wave, void *ws,
                                                  size_t ws_bytes, void *stream) {
    using namespace fa;
    clear_error();
    FA_TRY(check_counts(n_pairs, fixed, n_cfg, cfgs, 1));
    FA_TRY(check_wave(jobs_per_wave));
    if (!moving || !u_out) {
        set_error("fa_register_batched_lockstep: moving and u_out must not be NULL");
        return FA_ERR_INVALID;
    }
    const int jobs = n_pairs * n_cfg;
    std::vector<LockstepArgs> a((size_t)jobs);
    for (int i = 0; i < n_pairs; ++i)
        for (int c = 0; c < n_cfg; ++c) {
            const int j = i * n_cfg + c;
            const fa_status st = register_check(&fixed[i], &moving[i], &cfgs[c], &u_out[j]);
            if (st != FA_OK) {
                char msg[512];
                snprintf(msg, sizeof(msg), "%s", fa_last_error());
                set_error("fa_register_batched_lockstep: pair %d, parameter set %d: %s", i, c, msg);
                return st;
            }
            a[(size_t)j] = LockstepArgs{&fixed[i], &moving[i], &cfgs[c], &u_out[j],
                                        final_loss_dev ? final_loss_dev + j : nullptr,
                                        status_dev ? status_dev + j : nullptr};
        }
    // every wave is checked before anything is enqueued
    const int wave = jobs_per_wave < jobs ? jobs_per_wave : jobs;
    for (int j0 = 0; j0 < jobs; j0 += wave) {
        const int n = jobs - j0 < wave ? jobs - j0 : wave;
        FA_TRY(lockstep_check(n, a.data() + j0));
    }
    const size_t slot = slot_bytes(n_pairs, fixed, n_cfg, cfgs);
    FA_TRY(check_ws(ws, ws_bytes, slot * (size_t)wave, "fa_register_batched_lockstep"));
    for (int j0 = 0; j0 < jobs; j0 += wave) {
        const int n = jobs - j0 < wave ? jobs - j0 : wave;
        FA_TRY(register_lockstep(n, a.data() + j0, ws, slot, (cudaStream_t)stream));
    }
    return FA_OK;
}
