// pack.cu -- svm_train_data_pack: turns a trained SVM (Section 2.5; trained on the host as in
// Section 3) into a device-resident model: support vectors normalised per cell and stored in
// the scoring dtype with their squared norms, coefficients in fp32 (SIMT path) and bf16
// (tensor-core path), per-class coefficient sums, and the TMA descriptors of the tensor path.
#include <string.h>

#include <cuda_bf16.h>

#include <algorithm>
#include <new>

#include "internal.h"

namespace rgbd {
namespace {

// Coefficients padded to [C][n_pad] fp32 and [C_pad][n_pad] bf16 (round to nearest even); with
// `split`, a second bf16 plane holds lo = bf16(a - hi).
__global__ void coef_pad_kernel(const float* __restrict__ coef, int C, int n, int n_pad, int C_pad,
                                float* __restrict__ out_f32, uint16_t* __restrict__ out_bf16, int split) {
    const size_t total = (size_t)C_pad * n_pad;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(idx / n_pad), i = (int)(idx - (size_t)c * n_pad);
        const float v = (c < C && i < n) ? coef[(size_t)c * n + i] : 0.f;
        if (c < C) out_f32[(size_t)c * n_pad + i] = v;
        if (out_bf16) {
            const __nv_bfloat16 hi = __float2bfloat16_rn(v);
            out_bf16[idx] = __bfloat16_as_ushort(hi);
            if (split) out_bf16[total + idx] = __bfloat16_as_ushort(__float2bfloat16_rn(v - __bfloat162float(hi)));
        }
    }
}

// asum[c] = sum_i a_ci in fp64; one warp per class.
__global__ void asum_kernel(const float* __restrict__ coef, int C, int n, float* __restrict__ asum) {
    const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (c >= C) return;
    double s = 0.0;
    for (int i = lane; i < n; i += 32) s += (double)coef[(size_t)c * n + i];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, off);
    if (lane == 0) asum[c] = (float)s;
}

// asum_tile[t][c] = sum of a_ci over the SVs of tile t (fp64); one warp per (tile, class),
// zero for the padded classes c >= C.
__global__ void asum_tile_kernel(const float* __restrict__ coef, int C, int C_pad, int n_pad,
                                 float* __restrict__ out) {
    const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const int nt = n_pad / kSvTile;
    if (w >= nt * C_pad) return;
    const int t = w / C_pad, c = w - t * C_pad;
    double s = 0.0;
    if (c < C)
        for (int i = lane; i < kSvTile; i += 32) s += (double)coef[(size_t)c * n_pad + t * kSvTile + i];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, off);
    if (lane == 0) out[w] = (float)s;
}

__global__ void copy_pad_rows_kernel(const float* __restrict__ src, int rows, int cols, int ld,
                                     float* __restrict__ dst) {
    const size_t total = (size_t)rows * ld;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(idx / ld), j = (int)(idx - (size_t)r * ld);
        dst[idx] = j < cols ? src[(size_t)r * cols + j] : 0.f;
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

void free_model(rgbd_svm* m) {
    if (!m) return;
    cudaFree(m->sv);
    cudaFree(m->sv_sq);
    cudaFree(m->coef);
    cudaFree(m->coef_bf16);
    cudaFree(m->asum);
    cudaFree(m->asum_tile);
    cudaFree(m->bias);
    cudaFree(m->centre);
    delete m;
}

}  // namespace

int encode_tmap_2d(CUtensorMap* map, CUtensorMapDataType dt, const void* base, uint64_t inner,
                   uint64_t outer, uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer,
                   CUtensorMapSwizzle swizzle) {
    EncodeTiledFn fn = get_encode_fn();
    if (!fn) return set_error(RGBD_ERR_CUDA, "cuTensorMapEncodeTiled entry point unavailable");
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {row_bytes};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(RGBD_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return RGBD_OK;
}

}  // namespace rgbd

using namespace rgbd;

// bytes per element of a packed row (RGBD_DT_BF16X3: two bf16 planes)
static size_t dtype_bytes(int dt) { return dt == RGBD_DT_BF16 ? 2 : (dt == RGBD_DT_FP8 ? 1 : 4); }

extern "C" {

int svm_train_data_pack(rgbd_ctx* ctx, const uint16_t* sv_feats, int n_sv, int dim, int nbins,
                        const float* coef, const float* bias, int n_classes, int kernel, float gamma,
                        int dtype, rgbd_svm** model_out, void* stream) {
    rgbd::NvtxRange nvtx_range("svm_train_data_pack");
    if (!ctx || !model_out) return set_error(RGBD_ERR_ARG, "svm_train_data_pack: ctx or model_out is NULL");
    *model_out = nullptr;
    if (kernel != RGBD_KERNEL_LINEAR && kernel != RGBD_KERNEL_RBF)
        return set_error(RGBD_ERR_ARG, "svm_train_data_pack: kernel %d", kernel);
    const bool centred = (dtype & RGBD_DT_CENTRED) != 0;
    dtype &= ~RGBD_DT_CENTRED;
    if (centred && kernel != RGBD_KERNEL_RBF)
        return set_error(RGBD_ERR_ARG, "svm_train_data_pack: RGBD_DT_CENTRED applies to RBF models only");
    if (dim <= 0 || nbins <= 0 || nbins > 256 || dim % nbins)
        return set_error(RGBD_ERR_ARG, "svm_train_data_pack: dim %d nbins %d", dim, nbins);
    if (coef && (n_classes <= 0 || n_classes > 256))
        return set_error(RGBD_ERR_ARG, "svm_train_data_pack: n_classes %d (1..256)", n_classes);
    if (kernel == RGBD_KERNEL_RBF) {
        if (!sv_feats || n_sv <= 0) return set_error(RGBD_ERR_ARG, "svm_train_data_pack: RBF needs support vectors");
        if (!(gamma > 0.f)) return set_error(RGBD_ERR_ARG, "svm_train_data_pack: gamma must be > 0");
        if (dtype != RGBD_DT_F32 && dtype != RGBD_DT_BF16 && dtype != RGBD_DT_FP8 && dtype != RGBD_DT_TF32 &&
            dtype != RGBD_DT_BF16X3)
            return set_error(RGBD_ERR_ARG, "svm_train_data_pack: dtype %d", dtype);
    } else {
        if (!coef) return set_error(RGBD_ERR_ARG, "svm_train_data_pack: a linear model needs coef (w)");
        dtype = RGBD_DT_F32;
    }
    DeviceGuard g(ctx->props.device);
    cudaStream_t s = (cudaStream_t)stream;
    rgbd_svm* m = new (std::nothrow) rgbd_svm();
    if (!m) return set_error(RGBD_ERR_NOMEM, "svm_train_data_pack: host allocation");
    m->device = ctx->props.device;
    m->kernel = kernel;
    m->dtype = dtype;
    m->dim = dim;
    m->nbins = nbins;
    m->k_pad = (dim + kKAlign - 1) / kKAlign * kKAlign;
    m->gamma = gamma;
    m->C = coef ? n_classes : 0;
    m->C_pad = std::max(16, (m->C + 15) / 16 * 16);
    m->scorable = coef != nullptr;
    cudaError_t e = cudaSuccess;
    int rc = RGBD_OK;
#define TRY_CUDA(call, what)                  \
    do {                                      \
        e = (call);                           \
        if (e != cudaSuccess) {               \
            rc = cuda_error(e, what);         \
            free_model(m);                    \
            return rc;                        \
        }                                     \
    } while (0)

    if (kernel == RGBD_KERNEL_LINEAR) {
        TRY_CUDA(cudaMalloc(&m->coef, sizeof(float) * (size_t)m->C * m->k_pad), "pack: w");
        copy_pad_rows_kernel<<<256, 256, 0, s>>>(coef, m->C, dim, m->k_pad, m->coef);
        TRY_CUDA(cudaGetLastError(), "pack: w copy");
    } else {
        m->n_sv = n_sv;
        m->n_pad = (n_sv + kSvTile - 1) / kSvTile * kSvTile;
        const size_t esz = dtype_bytes(dtype);
        TRY_CUDA(cudaMalloc(&m->sv, esz * (size_t)m->n_pad * m->k_pad), "pack: sv");
        TRY_CUDA(cudaMalloc(&m->sv_sq, sizeof(float) * (size_t)m->n_pad), "pack: sv_sq");
        TRY_CUDA(cudaMemsetAsync(m->sv, 0, esz * (size_t)m->n_pad * m->k_pad, s), "pack: sv clear");
        TRY_CUDA(cudaMemsetAsync(m->sv_sq, 0, sizeof(float) * (size_t)m->n_pad, s), "pack: sv_sq clear");
        if (centred) {
            // fp32 rows, their column means mu (fp64 sums), rows - mu, then the dtype conversion
            // (FP8: per-tensor scale 448 / max|sv - mu|) with the squared norms of the stored values.
            float* tmp = nullptr;
            float* d_max = nullptr;
            TRY_CUDA(cudaMalloc(&m->centre, sizeof(float) * (size_t)m->k_pad), "pack: centre");
            TRY_CUDA(cudaMalloc(&tmp, sizeof(float) * (size_t)n_sv * m->k_pad), "pack: centring staging");
            e = cudaMalloc(&d_max, sizeof(float));
            if (e != cudaSuccess) {
                cudaFree(tmp);
                rc = cuda_error(e, "pack: max");
                free_model(m);
                return rc;
            }
            cudaMemsetAsync(d_max, 0, sizeof(float), s);
            rc = launch_normalize(sv_feats, n_sv, dim, nbins, RGBD_DT_F32, tmp, m->k_pad, 1.f, nullptr, nullptr, s);
            if (!rc) rc = launch_centre_rows(tmp, n_sv, dim, m->k_pad, m->centre, d_max, s);
            float hmax = 0.f;
            if (!rc && dtype == RGBD_DT_FP8) {
                e = cudaMemcpyAsync(&hmax, d_max, sizeof(float), cudaMemcpyDeviceToHost, s);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                if (e != cudaSuccess) rc = cuda_error(e, "pack: max readback");
                m->sv_scale = hmax > 0.f ? 448.f / hmax : 1.f;
            }
            if (!rc)
                rc = launch_quantize_f32(tmp, n_sv, m->k_pad, dtype, m->sv, m->sv_scale, m->sv_sq, s,
                                         (size_t)m->n_pad * m->k_pad);
            cudaStreamSynchronize(s);
            cudaFree(tmp);
            cudaFree(d_max);
            if (rc) {
                free_model(m);
                return rc;
            }
        } else if (dtype == RGBD_DT_FP8) {
            // fp32 rows first, then the per-tensor scale 448 / max|sv|, then E4M3 codes.
            float* tmp = nullptr;
            float* d_max = nullptr;
            TRY_CUDA(cudaMalloc(&tmp, sizeof(float) * (size_t)n_sv * m->k_pad), "pack: fp8 staging");
            e = cudaMalloc(&d_max, sizeof(float));
            if (e != cudaSuccess) {
                cudaFree(tmp);
                rc = cuda_error(e, "pack: max");
                free_model(m);
                return rc;
            }
            cudaMemsetAsync(d_max, 0, sizeof(float), s);
            rc = launch_normalize(sv_feats, n_sv, dim, nbins, RGBD_DT_F32, tmp, m->k_pad, 1.f, nullptr, d_max, s);
            float hmax = 0.f;
            if (!rc) {
                e = cudaMemcpyAsync(&hmax, d_max, sizeof(float), cudaMemcpyDeviceToHost, s);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                if (e != cudaSuccess) rc = cuda_error(e, "pack: max readback");
            }
            if (!rc) {
                m->sv_scale = hmax > 0.f ? 448.f / hmax : 1.f;
                rc = launch_quantize_f32(tmp, n_sv, m->k_pad, RGBD_DT_FP8, m->sv, m->sv_scale, m->sv_sq, s);
            }
            cudaStreamSynchronize(s);
            cudaFree(tmp);
            cudaFree(d_max);
            if (rc) {
                free_model(m);
                return rc;
            }
        } else {
            rc = launch_normalize(sv_feats, n_sv, dim, nbins, dtype, m->sv, m->k_pad, 1.f, m->sv_sq, nullptr, s,
                                  (size_t)m->n_pad * m->k_pad);
            if (rc) {
                free_model(m);
                return rc;
            }
        }
        if (coef) {
            TRY_CUDA(cudaMalloc(&m->coef, sizeof(float) * (size_t)m->C * m->n_pad), "pack: coef");
            const int planes = dtype == RGBD_DT_BF16X3 ? 2 : 1;
            TRY_CUDA(cudaMalloc(&m->coef_bf16, sizeof(uint16_t) * planes * (size_t)m->C_pad * m->n_pad),
                     "pack: coef bf16");
            TRY_CUDA(cudaMalloc(&m->asum, sizeof(float) * (size_t)m->C), "pack: asum");
            coef_pad_kernel<<<512, 256, 0, s>>>(coef, m->C, n_sv, m->n_pad, m->C_pad, m->coef, m->coef_bf16,
                                                dtype == RGBD_DT_BF16X3);
            TRY_CUDA(cudaGetLastError(), "pack: coef launch");
            asum_kernel<<<(m->C + 7) / 8, 256, 0, s>>>(coef, m->C, n_sv, m->asum);
            TRY_CUDA(cudaGetLastError(), "pack: asum launch");
            const int tile_sums = m->n_pad / kSvTile * m->C_pad;
            TRY_CUDA(cudaMalloc(&m->asum_tile, sizeof(float) * (size_t)tile_sums), "pack: tile sums");
            asum_tile_kernel<<<(tile_sums + 7) / 8, 256, 0, s>>>(m->coef, m->C, m->C_pad, m->n_pad, m->asum_tile);
            TRY_CUDA(cudaGetLastError(), "pack: tile sums launch");
        }
    }
    if (coef) {
        TRY_CUDA(cudaMalloc(&m->bias, sizeof(float) * (size_t)m->C), "pack: bias");
        if (bias)
            TRY_CUDA(cudaMemcpyAsync(m->bias, bias, sizeof(float) * m->C, cudaMemcpyDeviceToDevice, s), "pack: bias copy");
        else
            TRY_CUDA(cudaMemsetAsync(m->bias, 0, sizeof(float) * m->C, s), "pack: bias clear");
    }
    TRY_CUDA(cudaStreamSynchronize(s), "pack: synchronize");
    if (kernel == RGBD_KERNEL_RBF && dtype != RGBD_DT_F32 && coef) {
        rc = pack_model_tensor_maps(m);
        if (rc) {
            free_model(m);
            return rc;
        }
    }
#undef TRY_CUDA
    *model_out = m;
    return RGBD_OK;
}

int rgbd_svm_free(rgbd_svm* model) {
    if (!model) return RGBD_OK;
    DeviceGuard g(model->device);
    cudaDeviceSynchronize();
    free_model(model);
    return RGBD_OK;
}

int rgbd_svm_get_info(const rgbd_svm* m, rgbd_svm_info* info) {
    if (!m || !info) return set_error(RGBD_ERR_ARG, "rgbd_svm_get_info: NULL argument");
    info->kernel = m->kernel;
    info->dtype = m->dtype;
    info->n_sv = m->n_sv;
    info->n_sv_pad = m->n_pad;
    info->dim = m->dim;
    info->k_pad = m->k_pad;
    info->n_classes = m->C;
    info->scorable = m->scorable ? 1 : 0;
    info->gamma = m->gamma;
    info->sv_scale = m->sv_scale;
    info->centred = m->centre != nullptr ? 1 : 0;
    return RGBD_OK;
}

int rgbd_svm_centre(const rgbd_svm* m, const float** centre) {
    if (!m || !centre) return set_error(RGBD_ERR_ARG, "rgbd_svm_centre: NULL argument");
    *centre = m->centre;
    return RGBD_OK;
}

int rgbd_svm_packed_sv(const rgbd_svm* m, const void** sv, const float** sv_sq) {
    if (!m) return set_error(RGBD_ERR_ARG, "rgbd_svm_packed_sv: model is NULL");
    if (sv) *sv = m->sv;
    if (sv_sq) *sv_sq = m->sv_sq;
    return RGBD_OK;
}

}  // extern "C"
