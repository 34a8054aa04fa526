// internal.h -- declarations shared by the library's translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "rgbd_lbp.h"
#include <nvtx3/nvToolsExt.h>

namespace rgbd {

// NVTX range over one C-ABI call (a no-op unless a profiler is attached): names each stage in
// nsys / ncu timelines.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

constexpr int kBins = 59;     // uniform-pattern bins per cell (58 uniform + 1)
constexpr int kCell = 8;      // cell side in pixels
constexpr int kKAlign = 128;  // k_pad granularity (elements)
constexpr int kSvTile = 256;  // SVs per tensor-core tile; n_pad is a multiple of it
constexpr int kFaceCounters = 256;  // face-queue counters per context (launches in flight at once)

// Sets the thread's last error message (printf-style) and returns `code`.
int set_error(int code, const char* fmt, ...);
int cuda_error(cudaError_t e, const char* what);

struct DeviceProps {
    int device = 0;
    int sm_count = 0;
    int cc_major = 0, cc_minor = 0;
    size_t smem_optin = 0;
};

}  // namespace rgbd

struct rgbd_ctx {
    rgbd::DeviceProps props;
    int tune_lbp_ctas_per_sm = 0;  // 0 = occupancy limit
    int tune_tc_splits = 0;        // 0 = cost model
    int tune_tc_pairing = 0;       // CTA pairing: 0 = auto, 2 = none, 3 = 2-CTA MMA pairs
    int tune_lbp_shape = 0;        // fused-kernel threads per cell: 0 = auto, 1 = one, 2 = two, 3 = four
    int tune_tc_splitk = 0;        // K ranges of one-block scoring: 0 = auto, 1 = off, >= 2 forced
    uint32_t* d_status = nullptr;  // device status word, followed by kFaceCounters face-queue counters
    uint32_t* d_counters = nullptr;
    uint32_t counter_next = 0;     // next counter of the pool (a launch takes one and zeroes it)
    void* workspace = nullptr;
    size_t workspace_bytes = 0;
};

struct rgbd_svm {
    int device = 0;
    int kernel = RGBD_KERNEL_RBF;
    int dtype = RGBD_DT_F32;
    int n_sv = 0, n_pad = 0, dim = 0, nbins = rgbd::kBins, k_pad = 0;
    int C = 0, C_pad = 0;
    float gamma = 0.f;
    float sv_scale = 1.f;
    bool scorable = false;
    float* centre = nullptr;  // RGBD_DT_CENTRED: mu [k_pad], else NULL
    void* sv = nullptr;       // [n_pad][k_pad] of dtype (float for F32 / TF32)
    float* sv_sq = nullptr;   // [n_pad]
    float* coef = nullptr;    // RBF: float [C][n_pad]; linear: float [C][k_pad]
    uint16_t* coef_bf16 = nullptr;  // RBF tensor path: bf16 bits [C_pad][n_pad] ([2][C_pad][n_pad]
                                    // hi, lo for RGBD_DT_BF16X3)
    float* asum = nullptr;    // [C] sum_i a_ci (accumulated in fp64)
    float* asum_tile = nullptr;  // RBF: [n_pad / kSvTile][C_pad] sum of a_ci over each SV tile (fp64)
    float* bias = nullptr;    // [C]
    CUtensorMap tm_sv;        // tensor-core path: TMA descriptors (a whole SV tile, ...
    CUtensorMap tm_sv_half;   // ... half of it, the share of each CTA of a 2-CTA MMA pair)
    CUtensorMap tm_sv_lo;     // RGBD_DT_BF16X3: the same two maps over the lo plane
    CUtensorMap tm_sv_lo_half;
    CUtensorMap tm_coef;
    CUtensorMap tm_coef_half; // half of the classes of a coefficient chunk (2-CTA MMA pairs)
    CUtensorMap tm_coef_lo;   // RGBD_DT_BF16X3: the same two maps over the lo coefficient plane
    CUtensorMap tm_coef_lo_half;
    bool has_tmaps = false;
};

namespace rgbd {

// RAII device selection: makes ctx's device current for the scope of a call.
struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
            changed = (cudaSetDevice(dev) == cudaSuccess);
        }
    }
    ~DeviceGuard() {
        if (changed) cudaSetDevice(prev);
    }
};

// Grows the workspace of ctx to `bytes`.  Refuses while `stream` is capturing.
int ensure_workspace(rgbd_ctx* ctx, size_t bytes, cudaStream_t stream);

// ---- launchers (each returns RGBD_OK or an error code with the message set) ----------
int launch_crop_affine(rgbd_ctx* ctx, const uint8_t* grey, const uint16_t* depth, int n_frames,
                       int H, int W, const rgbd_rect* rects, const int32_t* affine, int n,
                       int out_h, int out_w, uint8_t* og, uint16_t* od, cudaStream_t s);

struct LbpArgs {
    const uint8_t* grey;
    const uint16_t* depth;
    int n_frames, H, W;
    const rgbd_rect* rects;
    const int32_t* affine;
    int n;
    int crop;
    int mask_mm;
    int flags;
    uint16_t* feats;
    int x_dtype;
    void* x_out;
    int k_pad;
    float x_scale;
    const float* x_centre;  // NULL, or float [dim] subtracted from the normalised values
    size_t x_plane;  // RGBD_DT_BF16X3: elements from the hi plane to the lo plane
    float* xsq;
    uint32_t* status;
    uint32_t* face_counter;  // NULL: faces strided over CTAs; else a zeroed queue counter
};
int launch_lbp_fused(rgbd_ctx* ctx, const LbpArgs& a, cudaStream_t s);

// plane: RGBD_DT_BF16X3 offset (elements) of the lo plane; 0 means n * k_pad.
int launch_normalize(const uint16_t* feats, int n, int dim, int nbins, int x_dtype, void* x_out,
                     int k_pad, float x_scale, float* xsq, float* row_max, cudaStream_t s,
                     size_t plane = 0, const float* centre = nullptr);

// fp32 rows [n][k_pad] -> dtype rows (FP8 with `scale`), with the squared norms of the stored
// values; plane: RGBD_DT_BF16X3 offset of the lo plane (0 means n * k_pad).
int launch_quantize_f32(const float* src, int n, int k_pad, int x_dtype, void* dst, float scale,
                        float* sq, cudaStream_t s, size_t plane = 0);

// Column means of fp32 rows [n][k_pad] (fp64 sums in row order, rounded to fp32) into mu[k_pad]
// (zero past dim), then rows -= mu (fp32), and the largest |value| into *absmax (>= 0).
int launch_centre_rows(float* rows, int n, int dim, int k_pad, float* mu, float* absmax, cudaStream_t s);

// scoring
int score_linear(rgbd_ctx* ctx, const rgbd_svm* m, const float* x, int n, float* scores,
                 int32_t* labels, cudaStream_t s);
int score_rbf_f32(rgbd_ctx* ctx, const rgbd_svm* m, const float* x, const float* xsq, int n,
                  float* scores, int32_t* labels, cudaStream_t s);
// Workspace bytes a scoring call of n rows takes (0: none, or a model the path rejects).
size_t score_rbf_f32_bytes(rgbd_ctx* ctx, const rgbd_svm* m, int n);
size_t score_rbf_tc_bytes(rgbd_ctx* ctx, const rgbd_svm* m, int n);
int score_rbf_tc(rgbd_ctx* ctx, const rgbd_svm* m, const void* x, const float* xsq, int n,
                 float x_scale, float* scores, int32_t* labels, cudaStream_t s);

// Tensor-core RBF scoring with its scratch (partial sums) in a buffer the caller provides
// instead of the context workspace.  *need receives the bytes required; when ws_bytes is
// smaller the call launches nothing and returns RGBD_ERR_ARG.
int score_rbf_tc_external_ws(rgbd_ctx* ctx, const rgbd_svm* m, const void* x, const float* xsq, int n,
                             float x_scale, float* scores, int32_t* labels, cudaStream_t s, void* ws,
                             size_t ws_bytes, size_t* need);

// model packing helpers (pack.cu)
int pack_model_tensor_maps(rgbd_svm* m);

// Final reduction of per-split partial scores (svm_simt.cu), shared by both RBF paths.
//   part  [splits][n][C_stride] partial sums D_s[k][c]
//   ref   NULL, or [splits][n] per-split reference distances r_s (see svm_tc.cu)
//   asum_tile  with ref: [n_tiles][C_stride] coefficient sums per SV tile; split s covers
//              tiles [s * tiles_per_split, (s + 1) * tiles_per_split) clipped to n_tiles
int launch_reduce_scores(const float* part, const float* ref, int splits, int n, int C,
                         int C_stride, const float* asum, const float* asum_tile,
                         int tiles_per_split, int n_tiles, const float* bias, float gamma,
                         float* scores, int32_t* labels, cudaStream_t s);

// TMA descriptor encoding through the driver entry point (no libcuda link).
int encode_tmap_2d(CUtensorMap* map, CUtensorMapDataType dt, const void* base, uint64_t inner,
                   uint64_t outer, uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer,
                   CUtensorMapSwizzle swizzle);

}  // namespace rgbd
