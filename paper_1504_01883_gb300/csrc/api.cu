// api.cu -- the extern "C" entry points: argument checks, context, dispatch.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "internal.h"

namespace rgbd {

static thread_local char g_last_error[1024] = "";

int set_error(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_error(cudaError_t e, const char* what) {
    if (e == cudaErrorMemoryAllocation)
        return set_error(RGBD_ERR_NOMEM, "%s: %s", what, cudaGetErrorString(e));
    return set_error(RGBD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int ensure_workspace(rgbd_ctx* ctx, size_t bytes, cudaStream_t stream) {
    if (bytes <= ctx->workspace_bytes) return RGBD_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (stream != nullptr && cudaStreamIsCapturing(stream, &cs) == cudaSuccess &&
        cs != cudaStreamCaptureStatusNone)
        return set_error(RGBD_ERR_ARG,
                         "workspace must grow to %zu bytes while the stream is capturing; "
                         "call rgbd_ctx_reserve() before capture",
                         bytes);
    if (ctx->workspace) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_error(e, "workspace resize sync");
        cudaFree(ctx->workspace);
        ctx->workspace = nullptr;
        ctx->workspace_bytes = 0;
    }
    size_t sz = (bytes + 0xFFFFF) & ~size_t(0xFFFFF);
    cudaError_t e = cudaMalloc(&ctx->workspace, sz);
    if (e != cudaSuccess) return cuda_error(e, "workspace cudaMalloc");
    ctx->workspace_bytes = sz;
    return RGBD_OK;
}

}  // namespace rgbd

using namespace rgbd;

#define CHECK_ARG(cond, ...)                                  \
    do {                                                      \
        if (!(cond)) return set_error(RGBD_ERR_ARG, __VA_ARGS__); \
    } while (0)

extern "C" {

int rgbd_version(void) { return (1 << 16) | 0; }

int rgbd_last_error(char* buf, size_t len) {
    size_t n = strlen(g_last_error);
    if (buf && len) {
        size_t c = n < len - 1 ? n : len - 1;
        memcpy(buf, g_last_error, c);
        buf[c] = 0;
    }
    return (int)n;
}

int rgbd_ctx_create(int device, rgbd_ctx** out) {
    CHECK_ARG(out != nullptr, "rgbd_ctx_create: out is NULL");
    *out = nullptr;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDeviceCount");
    CHECK_ARG(device >= 0 && device < count, "rgbd_ctx_create: device %d of %d", device, count);
    DeviceGuard g(device);
    rgbd_ctx* c = new (std::nothrow) rgbd_ctx();
    if (!c) return set_error(RGBD_ERR_NOMEM, "rgbd_ctx_create: host allocation");
    c->props.device = device;
    cudaDeviceGetAttribute(&c->props.sm_count, cudaDevAttrMultiProcessorCount, device);
    cudaDeviceGetAttribute(&c->props.cc_major, cudaDevAttrComputeCapabilityMajor, device);
    cudaDeviceGetAttribute(&c->props.cc_minor, cudaDevAttrComputeCapabilityMinor, device);
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    c->props.smem_optin = (size_t)optin;
    e = cudaMalloc(&c->d_status, sizeof(uint32_t) * (1 + kFaceCounters));
    if (e != cudaSuccess) {
        delete c;
        return cuda_error(e, "rgbd_ctx_create: status word");
    }
    c->d_counters = c->d_status + 1;
    e = cudaMemset(c->d_status, 0, sizeof(uint32_t) * (1 + kFaceCounters));
    if (e != cudaSuccess) {
        cudaFree(c->d_status);
        delete c;
        return cuda_error(e, "rgbd_ctx_create: status memset");
    }
    *out = c;
    return RGBD_OK;
}

int rgbd_ctx_destroy(rgbd_ctx* ctx) {
    if (!ctx) return RGBD_OK;
    DeviceGuard g(ctx->props.device);
    cudaDeviceSynchronize();
    if (ctx->workspace) cudaFree(ctx->workspace);
    if (ctx->d_status) cudaFree(ctx->d_status);
    delete ctx;
    return RGBD_OK;
}

int rgbd_ctx_reserve(rgbd_ctx* ctx, size_t bytes) {
    CHECK_ARG(ctx != nullptr, "rgbd_ctx_reserve: ctx is NULL");
    DeviceGuard g(ctx->props.device);
    return ensure_workspace(ctx, bytes, nullptr);
}

int rgbd_ctx_status(rgbd_ctx* ctx, uint32_t* flags, int clear) {
    CHECK_ARG(ctx != nullptr, "rgbd_ctx_status: ctx is NULL");
    DeviceGuard g(ctx->props.device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_error(e, "rgbd_ctx_status: synchronize");
    uint32_t v = 0;
    e = cudaMemcpy(&v, ctx->d_status, sizeof(v), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "rgbd_ctx_status: read");
    if (flags) *flags = v;
    if (clear) {
        e = cudaMemset(ctx->d_status, 0, sizeof(uint32_t));
        if (e != cudaSuccess) return cuda_error(e, "rgbd_ctx_status: clear");
    }
    return RGBD_OK;
}

int rgbd_ctx_set_tuning(rgbd_ctx* ctx, int key, int value) {
    CHECK_ARG(ctx != nullptr, "rgbd_ctx_set_tuning: ctx is NULL");
    CHECK_ARG(value >= 0, "rgbd_ctx_set_tuning: value %d < 0", value);
    switch (key) {
        case RGBD_TUNE_LBP_CTAS_PER_SM:
            CHECK_ARG(value <= 2, "rgbd_ctx_set_tuning: %d CTAs per SM (0, 1 or 2)", value);
            ctx->tune_lbp_ctas_per_sm = value;
            return RGBD_OK;
        case RGBD_TUNE_TC_SPLITS:
            ctx->tune_tc_splits = value;
            return RGBD_OK;
        case RGBD_TUNE_LBP_SHAPE:
            CHECK_ARG(value <= 3, "rgbd_ctx_set_tuning: fused-kernel shape %d (0..3)", value);
            ctx->tune_lbp_shape = value;
            return RGBD_OK;
        case RGBD_TUNE_TC_SPLITK:
            CHECK_ARG(value <= 4096, "rgbd_ctx_set_tuning: %d K ranges (at most 4096)", value);
            ctx->tune_tc_splitk = value;
            return RGBD_OK;
        case RGBD_TUNE_TC_PAIRING:
            CHECK_ARG(value == 0 || value == 2 || value == 3, "rgbd_ctx_set_tuning: CTA pairing %d (0, 2 or 3)", value);
            ctx->tune_tc_pairing = value;
            return RGBD_OK;
        default:
            return set_error(RGBD_ERR_ARG, "rgbd_ctx_set_tuning: unknown key %d", key);
    }
}

int rgbd_crop_affine(rgbd_ctx* ctx, const uint8_t* grey, const uint16_t* depth, int n_frames, int H,
                     int W, const rgbd_rect* rects, const int32_t* affine_q16, int n_rects,
                     int out_h, int out_w, uint8_t* out_grey, uint16_t* out_depth, void* stream) {
    rgbd::NvtxRange nvtx_range("rgbd_crop_affine");
    CHECK_ARG(ctx != nullptr, "rgbd_crop_affine: ctx is NULL");
    CHECK_ARG(n_rects >= 0, "rgbd_crop_affine: n_rects %d < 0", n_rects);
    if (n_rects == 0) return RGBD_OK;
    CHECK_ARG(grey && depth && rects && out_grey && out_depth,
              "rgbd_crop_affine: NULL data pointer");
    CHECK_ARG(n_frames > 0 && H > 0 && W > 0, "rgbd_crop_affine: frames %d x %d x %d", n_frames, H, W);
    CHECK_ARG(H <= 65535 && W <= 65535, "rgbd_crop_affine: frame side above 65535");
    CHECK_ARG(out_h > 0 && out_w > 0 && out_h <= 4096 && out_w <= 4096,
              "rgbd_crop_affine: crop %d x %d", out_h, out_w);
    DeviceGuard g(ctx->props.device);
    return launch_crop_affine(ctx, grey, depth, n_frames, H, W, rects, affine_q16, n_rects, out_h,
                              out_w, out_grey, out_depth, (cudaStream_t)stream);
}

static int check_x_out(const char* fn, int dim, int x_dtype, const void* x_out, int k_pad,
                       float x_scale) {
    if (x_dtype == 0) return RGBD_OK;
    CHECK_ARG(x_dtype == RGBD_DT_F32 || x_dtype == RGBD_DT_BF16 || x_dtype == RGBD_DT_FP8 ||
                  x_dtype == RGBD_DT_TF32 || x_dtype == RGBD_DT_BF16X3,
              "%s: unknown x_dtype %d", fn, x_dtype);
    CHECK_ARG(x_out != nullptr, "%s: x_out is NULL", fn);
    CHECK_ARG(k_pad >= dim && k_pad % kKAlign == 0, "%s: k_pad %d must be >= %d and a multiple of %d",
              fn, k_pad, dim, kKAlign);
    CHECK_ARG(x_dtype != RGBD_DT_FP8 || (x_scale > 0.f && x_scale < 1e30f),
              "%s: FP8 output needs a positive x_scale", fn);
    return RGBD_OK;
}

int lbp_fused_features(rgbd_ctx* ctx, const uint8_t* grey, const uint16_t* depth, int n_frames,
                       int H, int W, const rgbd_rect* rects, const int32_t* affine_q16, int n,
                       int crop, int cell, int mask_mm, int flags, uint16_t* feats, int x_dtype,
                       void* x_out, int k_pad, float x_scale, const float* x_centre, float* xsq_out,
                       void* stream) {
    rgbd::NvtxRange nvtx_range("lbp_fused_features");
    CHECK_ARG(ctx != nullptr, "lbp_fused_features: ctx is NULL");
    CHECK_ARG(n >= 0, "lbp_fused_features: n %d < 0", n);
    CHECK_ARG((flags & ~(RGBD_LBP_GE | RGBD_LBP_NBR_IGNORE_MASK | RGBD_LBP_FACE_HIST256)) == 0,
              "lbp_fused_features: unknown flags 0x%x", flags);
    const bool face256 = (flags & RGBD_LBP_FACE_HIST256) != 0;
    if (face256) {
        if (cell != crop)
            return set_error(RGBD_ERR_UNSUPPORTED, "lbp_fused_features: the 0-255 face histogram needs cell == crop");
        if (crop < 8 || crop > 255)
            return set_error(RGBD_ERR_UNSUPPORTED, "lbp_fused_features: crop %d (8..255 for the face histogram)", crop);
    } else {
        if (cell != kCell)
            return set_error(RGBD_ERR_UNSUPPORTED, "lbp_fused_features: cell %d (only 8)", cell);
        if (crop != 32 && crop != 64 && crop != 96 && crop != 128)
            return set_error(RGBD_ERR_UNSUPPORTED,
                             "lbp_fused_features: crop %d (32, 64, 96 or 128)", crop);
    }
    CHECK_ARG(mask_mm > 0, "lbp_fused_features: mask_mm %d", mask_mm);
    if (n == 0) return RGBD_OK;
    CHECK_ARG(grey && depth, "lbp_fused_features: NULL frame pointer");
    CHECK_ARG(feats || x_out, "lbp_fused_features: neither feats nor x_out given");
    const int dim = face256 ? 256 : (crop / kCell) * (crop / kCell) * kBins;
    int rc = check_x_out("lbp_fused_features", dim, x_dtype, x_out, k_pad, x_scale);
    if (rc) return rc;
    CHECK_ARG((reinterpret_cast<uintptr_t>(x_centre) & 15) == 0, "lbp_fused_features: x_centre not 16-byte aligned");
    if (rects == nullptr) {
        CHECK_ARG(affine_q16 == nullptr, "lbp_fused_features: affine needs rects");
        CHECK_ARG(n_frames == n && H == crop && W == crop,
                  "lbp_fused_features: pre-cut crops need n_frames == n and H == W == crop");
    } else {
        CHECK_ARG(n_frames > 0 && H > 0 && W > 0 && H <= 65535 && W <= 65535,
                  "lbp_fused_features: frames %d x %d x %d", n_frames, H, W);
    }
    DeviceGuard g(ctx->props.device);
    LbpArgs a;
    a.grey = grey;
    a.depth = depth;
    a.n_frames = n_frames;
    a.H = H;
    a.W = W;
    a.rects = rects;
    a.affine = affine_q16;
    a.n = n;
    a.crop = crop;
    a.mask_mm = mask_mm;
    a.flags = flags;
    a.feats = feats;
    a.x_dtype = x_dtype;
    a.x_out = x_out;
    a.k_pad = k_pad;
    a.x_scale = x_scale;
    a.x_centre = x_dtype ? x_centre : nullptr;
    a.x_plane = (size_t)n * k_pad;
    a.xsq = xsq_out;
    a.status = ctx->d_status;
    a.face_counter = ctx->d_counters + (ctx->counter_next++ % kFaceCounters);
    return launch_lbp_fused(ctx, a, (cudaStream_t)stream);
}

int lbp_normalize_features(rgbd_ctx* ctx, const uint16_t* feats, int n, int dim, int nbins,
                           int x_dtype, void* x_out, int k_pad, float x_scale, const float* x_centre,
                           float* xsq_out, void* stream) {
    rgbd::NvtxRange nvtx_range("lbp_normalize_features");
    CHECK_ARG(ctx != nullptr, "lbp_normalize_features: ctx is NULL");
    CHECK_ARG(n >= 0 && dim > 0 && nbins > 0 && dim % nbins == 0,
              "lbp_normalize_features: n %d dim %d nbins %d", n, dim, nbins);
    CHECK_ARG(nbins <= 256, "lbp_normalize_features: nbins %d > 256", nbins);
    CHECK_ARG(x_dtype != 0, "lbp_normalize_features: x_dtype 0");
    if (n == 0) return RGBD_OK;  // nothing to write: x_out may be NULL (an empty buffer)
    int rc = check_x_out("lbp_normalize_features", dim, x_dtype, x_out, k_pad, x_scale);
    if (rc) return rc;
    CHECK_ARG(feats != nullptr, "lbp_normalize_features: feats is NULL");
    DeviceGuard g(ctx->props.device);
    return launch_normalize(feats, n, dim, nbins, x_dtype, x_out, k_pad, x_scale, xsq_out, nullptr,
                            (cudaStream_t)stream, 0, x_centre);
}

int svm_score(rgbd_ctx* ctx, const rgbd_svm* model, const void* x, const float* xsq, int n,
              float x_scale, float* scores, int32_t* labels, void* stream) {
    rgbd::NvtxRange nvtx_range("svm_score");
    CHECK_ARG(ctx != nullptr && model != nullptr, "svm_score: ctx or model is NULL");
    CHECK_ARG(model->scorable, "svm_score: model was packed without coefficients");
    CHECK_ARG(n >= 0, "svm_score: n %d < 0", n);
    if (n == 0) return RGBD_OK;
    CHECK_ARG(x != nullptr && scores != nullptr, "svm_score: NULL x or scores");
    CHECK_ARG(model->device == ctx->props.device, "svm_score: model and ctx on different devices");
    DeviceGuard g(ctx->props.device);
    cudaStream_t s = (cudaStream_t)stream;
    if (model->kernel == RGBD_KERNEL_LINEAR)
        return score_linear(ctx, model, (const float*)x, n, scores, labels, s);
    CHECK_ARG(xsq != nullptr, "svm_score: RBF needs xsq");
    if (model->dtype == RGBD_DT_F32)
        return score_rbf_f32(ctx, model, (const float*)x, xsq, n, scores, labels, s);
    if (model->dtype == RGBD_DT_FP8)
        CHECK_ARG(x_scale > 0.f, "svm_score: FP8 needs x_scale > 0");
    return score_rbf_tc(ctx, model, x, xsq, n, x_scale, scores, labels, s);
}

}  // extern "C"
