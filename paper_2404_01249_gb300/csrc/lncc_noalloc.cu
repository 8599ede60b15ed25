// fa_lncc_fwd_bwd_noalloc: the LNCC forward/backward of fa_lncc_fwd_bwd for
// callers that cannot allocate device memory.
//
// Some callers cannot hand libfa a workspace: code running where
// cudaMalloc is forbidden or unavailable (inside a host callback or another
// library's allocation-free section, a plugin host that owns every device
// allocation, or a real-time loop that must never enter the allocator).
// This entry point takes only the inputs and outputs and runs the same
// kernels as fa_lncc_fwd_bwd on a scratch area that is part of the library
// image itself: a file-scope device array of kNoAllocScratchBytes (64 MiB)
// that every GPU which loads this library keeps until the process exits.
//
// Limits and rules for callers:
//  * the grid may hold at most as many voxels as fit the scratch (the
//    same bytes fa_lncc_workspace_size reports: at most 621,376 voxels, e.g.
//    80 x 96 x 80); larger grids are rejected with FA_ERR_SHAPE before
//    anything is launched;
//  * the first call on each device looks up the array's device address
//    (cudaGetSymbolAddress, with that device current); make that first call
//    before any stream capture.  The address is kept per device and CUDA
//    context: after a device reset the next call looks it up again (in the
//    new context) and must likewise come before any capture;
//  * all calls share the one array and it keeps the previous call's
//    contents (every call clears the fields that must start at zero); calls
//    that overlap on the GPU -- different streams, or several host threads
//    -- race on it, so serialise them;
//  * no cudaMalloc, cudaFree or allocating library routine is called.
#include <mutex>

#include "ops.h"
#include "validate.h"

namespace fa {

static constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;
static constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_mu;
struct NoAllocSlot {
    unsigned long long ctx;  // context id the address was looked up in
    void *ptr;
};
static NoAllocSlot g_noalloc_slot[kMaxDevices];

// Device address of the scratch array in the current device's context,
// looked up once per context: a device reset makes a new context (with a new
// id) in which the array has a new address, and the next call looks it up
// again.
static fa_status noalloc_scratch(void **out) {
    int dev = -1;
    FA_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("fa_lncc_fwd_bwd_noalloc: device ordinal %d is not supported", dev);
        return FA_ERR_UNSUPPORTED;
    }
    unsigned long long ctx = 0;
    FA_CUDA_TRY(current_context_id(&ctx));
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoAllocSlot &sl = g_noalloc_slot[dev];
    if (!sl.ptr || sl.ctx != ctx) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        sl.ptr = p;
        sl.ctx = ctx;
    }
    *out = sl.ptr;
    return FA_OK;
}

}  // namespace fa

extern "C" fa_status fa_lncc_fwd_bwd_noalloc(const fa_vol *fixed, const fa_vol *warped,
                                             int32_t window, float cc_eps, float *loss_dev,
                                             fa_vol *dL_dwarped_opt, fa_vol *dL_dfixed_opt,
                                             void *stream) {
    using namespace fa;
    clear_error();
    if (window < 1 || window > 15 || (window % 2) == 0) {
        set_error("fa_lncc_fwd_bwd_noalloc: window must be odd and in 1..15 (got %d)",
                  (int)window);
        return FA_ERR_INVALID;
    }
    if (!(cc_eps >= 0.0f) || !(cc_eps < 3.0e38f)) {
        set_error("fa_lncc_fwd_bwd_noalloc: cc_eps must be finite and >= 0");
        return FA_ERR_INVALID;
    }
    FA_TRY(check_vol(fixed, "fixed", 1));
    FA_TRY(check_vol(warped, "warped", 1));
    FA_TRY(same_grid(fixed, warped, "fixed", "warped"));
    if (dL_dwarped_opt) {
        FA_TRY(check_vol(dL_dwarped_opt, "dL_dwarped", 1));
        FA_TRY(same_grid(fixed, dL_dwarped_opt, "fixed", "dL_dwarped"));
    }
    if (dL_dfixed_opt) {
        FA_TRY(check_vol(dL_dfixed_opt, "dL_dfixed", 1));
        FA_TRY(same_grid(fixed, dL_dfixed_opt, "fixed", "dL_dfixed"));
    }
    Dims d{fixed->D, fixed->H, fixed->W};
    long long N = d.N();
    size_t need = lncc_plain_bytes(N);
    if (need > kNoAllocScratchBytes) {
        set_error("fa_lncc_fwd_bwd_noalloc: a %dx%dx%d grid needs %zu bytes of scratch but the "
                  "built-in scratch holds %zu (at most 621376 voxels); use fa_lncc_fwd_bwd with a "
                  "workspace",
                  d.D, d.H, d.W, need, kNoAllocScratchBytes);
        return FA_ERR_SHAPE;
    }
    void *scratch = nullptr;
    FA_TRY(noalloc_scratch(&scratch));
    cudaStream_t s = (cudaStream_t)stream;
    WsCarver c(scratch, kNoAllocScratchBytes);
    WsHeader *h = c.take<WsHeader>(1);
    LnccBuffers b = lncc_carve(c, N);
    const float *I = (const float *)fixed->data, *J = (const float *)warped->data;
    FA_CUDA_TRY(launch_header_reset(h, s));  // loss accumulator, maxima, status start at zero
    FA_CUDA_TRY(launch_absmax2(I, J, N, h, s));
    FA_CUDA_TRY(launch_lncc_forward(I, J, d, window, cc_eps, dL_dfixed_opt != nullptr, h, b, s));
    FA_CUDA_TRY(launch_loss_finalize(h, N, -1.0f, loss_dev, s));
    if (dL_dwarped_opt || dL_dfixed_opt)
        FA_CUDA_TRY(launch_lncc_backward(
            I, J, nullptr, d, window, h, b, dL_dwarped_opt ? (float *)dL_dwarped_opt->data : nullptr,
            dL_dfixed_opt ? (float *)dL_dfixed_opt->data : nullptr, nullptr, s));
    return FA_OK;
}
