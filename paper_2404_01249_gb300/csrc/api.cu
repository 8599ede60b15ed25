// Error reporting, parameter defaults and descriptor validation of libfa.
#include <stdarg.h>
#include <cuda.h>

#include <atomic>
#include <stdio.h>
#include <string.h>

#include "common.cuh"
#include "validate.h"

namespace fa {

static thread_local char g_err[512];
static std::atomic<unsigned long long> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(unsigned long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
unsigned long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void clear_error() { g_err[0] = 0; }

fa_status cuda_fail(cudaError_t e, const char *where) {
    set_error("%s: %s", where, cudaGetErrorString(e));
    return FA_ERR_CUDA;
}

cudaError_t current_context_id(unsigned long long *id) {
    using GetCurrent = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static const GetCurrent get_current = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return (GetCurrent)p;
    }();
    static const GetId get_id = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return (GetId)p;
    }();
    *id = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaSetDevice(dev)) != cudaSuccess) return e;  // makes the primary context current
    if (!get_current || !get_id) return cudaSuccess;
    CUcontext ctx = nullptr;
    unsigned long long v = 0;
    if (get_current(&ctx) == CUDA_SUCCESS && ctx && get_id(ctx, &v) == CUDA_SUCCESS) *id = v;
    return cudaSuccess;
}

fa_status check_vol(const fa_vol *v, const char *name, int C) {
    return check_vol_dtype(v, name, C, FA_F32);
}

fa_status check_vol_dtype(const fa_vol *v, const char *name, int C, int dtype) {
    if (!v) {
        set_error("%s: descriptor is NULL", name);
        return FA_ERR_INVALID;
    }
    if (!v->data) {
        set_error("%s: data pointer is NULL", name);
        return FA_ERR_INVALID;
    }
    if (v->dtype != dtype) {
        set_error("%s: dtype %d not supported here (expected %d)", name, (int)v->dtype, dtype);
        return FA_ERR_DTYPE;
    }
    if (v->C != C || v->D < 1 || v->H < 1 || v->W < 1) {
        set_error("%s: expected C=%d and positive D, H, W (got C=%d D=%d H=%d W=%d)", name, C,
                  (int)v->C, (int)v->D, (int)v->H, (int)v->W);
        return FA_ERR_SHAPE;
    }
    if ((long long)v->D * v->H * v->W >= (1ll << 31)) {
        set_error("%s: grid of %lld voxels exceeds 2^31 - 1", name,
                  (long long)v->D * v->H * v->W);
        return FA_ERR_SHAPE;
    }
    if (((uintptr_t)v->data & 15u) != 0) {
        set_error("%s: data pointer must be 16-byte aligned", name);
        return FA_ERR_INVALID;
    }
    return FA_OK;
}

fa_status same_grid(const fa_vol *a, const fa_vol *b, const char *an, const char *bn) {
    if (a->D != b->D || a->H != b->H || a->W != b->W) {
        set_error("%s (%dx%dx%d) and %s (%dx%dx%d) must share a grid", an, (int)a->D, (int)a->H,
                  (int)a->W, bn, (int)b->D, (int)b->H, (int)b->W);
        return FA_ERR_SHAPE;
    }
    return FA_OK;
}

fa_status check_ws(const void *ws, size_t have, size_t need, const char *who) {
    if (need == 0) return FA_OK;
    if (!ws) {
        set_error("%s: workspace is NULL (needs %zu bytes)", who, need);
        return FA_ERR_WORKSPACE;
    }
    if (((uintptr_t)ws & 255u) != 0) {
        set_error("%s: workspace must be 256-byte aligned", who);
        return FA_ERR_WORKSPACE;
    }
    if (have < need) {
        set_error("%s: workspace of %zu bytes is smaller than the %zu needed", who, have, need);
        return FA_ERR_WORKSPACE;
    }
    return FA_OK;
}

}  // namespace fa

extern "C" {

const char *fa_status_str(fa_status s) {
    switch (s) {
        case FA_OK: return "ok";
        case FA_ERR_INVALID: return "invalid argument";
        case FA_ERR_SHAPE: return "shape error";
        case FA_ERR_DTYPE: return "unsupported dtype";
        case FA_ERR_CUDA: return "CUDA error";
        case FA_ERR_NONFINITE: return "non-finite value detected on the device";
        case FA_ERR_TIMEOUT: return "device wait timed out";
        case FA_ERR_UNSUPPORTED: return "unsupported request";
        case FA_ERR_WORKSPACE: return "workspace error";
    }
    return "unknown status";
}

const char *fa_last_error(void) { return fa::g_err; }

uint64_t fa_launch_count(void) { return fa::g_launches.load(std::memory_order_relaxed); }

fa_status fa_params_default(fa_params *p) {
    if (!p) {
        fa::set_error("fa_params_default: NULL");
        return FA_ERR_INVALID;
    }
    memset(p, 0, sizeof(*p));
    p->n_levels = 3;
    p->scales[0] = 4; p->scales[1] = 2; p->scales[2] = 1;
    p->iters[0] = 200; p->iters[1] = 100; p->iters[2] = 50;
    p->lr = 0.5f;
    p->sigma_grad = 1.0f;
    p->sigma_warp = 0.5f;
    p->window = 5;
    p->loss = FA_LOSS_LNCC;
    p->beta1 = 0.9f;
    p->beta2 = 0.999f;
    p->adam_eps = 1e-8f;
    p->cc_eps = 1e-5f;
    p->c_lp = 2.0f;
    p->mode = FA_MODE_FUSED;
    p->storage = FA_F32;
    p->graph = 1;
    p->mi_bins = 32;
    return FA_OK;
}

fa_status fa_ws_status(const void *ws, void *stream) {
    if (!ws) {
        fa::set_error("fa_ws_status: workspace is NULL");
        return FA_ERR_INVALID;
    }
    FA_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    unsigned st = 0;
    FA_CUDA_TRY(cudaMemcpy(&st, ws, sizeof(st), cudaMemcpyDeviceToHost));
    if (st & fa::ST_NONFINITE) {
        fa::set_error("a kernel found a non-finite loss, step or field");
        return FA_ERR_NONFINITE;
    }
    if (st & fa::ST_TIMEOUT) {
        fa::set_error("a bounded device wait gave up");
        return FA_ERR_TIMEOUT;
    }
    return FA_OK;
}

}  // extern "C"
