// noalloc.cu -- svm_score_noalloc: RBF scoring on the tensor cores that allocates no device memory.
//
// svm_score keeps its partial sums in the context workspace, which it grows with cudaMalloc
// when a call needs more.  Some callers cannot allow that: real-time loops that cannot afford
// the device-wide synchronisation that cudaMalloc / cudaFree may cause in the middle of a
// frame, and processes whose free device memory is already owned by another allocator (a
// framework's pool, a fixed per-tenant budget).  This entry point keeps its scratch in one
// fixed-size array of device memory that belongs to the library's module instead.
#include <mutex>

#include "internal.h"

namespace {

// Scratch of svm_score_noalloc.  Every GPU that loads the library holds it until the process
// exits.  All calls on a device share it, and it keeps the last call's contents.
constexpr size_t kStaticScratchBytes = RGBD_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on `device` (which must be current).  In host code the
// array's name is only a host-side stand-in, so the address is looked up once per device.
int scratch_address(int device, void** out) {
    if (device < 0 || device >= kMaxDevices)
        return rgbd::set_error(RGBD_ERR_UNSUPPORTED, "svm_score_noalloc: device %d above %d", device, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return rgbd::cuda_error(e, "svm_score_noalloc: cudaGetSymbolAddress");
        g_scratch_addr[device] = p;
    }
    *out = g_scratch_addr[device];
    return RGBD_OK;
}

}  // namespace

extern "C" int svm_score_noalloc(rgbd_ctx* ctx, const rgbd_svm* model, const void* x, const float* xsq, int n,
                                 float x_scale, float* scores, int32_t* labels, void* stream) {
    rgbd::NvtxRange nvtx_range("svm_score_noalloc");
    using namespace rgbd;
    if (!ctx || !model) return set_error(RGBD_ERR_ARG, "svm_score_noalloc: ctx or model is NULL");
    if (!model->scorable) return set_error(RGBD_ERR_ARG, "svm_score_noalloc: model was packed without coefficients");
    if (model->kernel != RGBD_KERNEL_RBF || model->dtype == RGBD_DT_F32)
        return set_error(RGBD_ERR_UNSUPPORTED,
                         "svm_score_noalloc: only RBF models packed as BF16, BF16X3, FP8 or TF32 (tensor-core path)");
    if (n < 0) return set_error(RGBD_ERR_ARG, "svm_score_noalloc: n %d < 0", n);
    if (n == 0) return RGBD_OK;
    if (!x || !xsq || !scores) return set_error(RGBD_ERR_ARG, "svm_score_noalloc: NULL x, xsq or scores");
    if (model->device != ctx->props.device)
        return set_error(RGBD_ERR_ARG, "svm_score_noalloc: model and ctx on different devices");
    if (model->dtype == RGBD_DT_FP8 && !(x_scale > 0.f))
        return set_error(RGBD_ERR_ARG, "svm_score_noalloc: FP8 needs x_scale > 0");
    DeviceGuard g(ctx->props.device);
    void* scratch = nullptr;
    int rc = scratch_address(ctx->props.device, &scratch);
    if (rc) return rc;
    size_t need = 0;
    return score_rbf_tc_external_ws(ctx, model, x, xsq, n, x_scale, scores, labels, (cudaStream_t)stream, scratch,
                                    kStaticScratchBytes, &need);
}
