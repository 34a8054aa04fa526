// roi.cu -- the depth-space region of a colour-detected face (Section 2.1): every depth pixel is
// mapped into the colour image (the camera mapping, here an exact integer calibration), the
// pixels landing inside the detected colour rect belong to the face, and the rect bounding them
// is the face region of the depth image.
#include <limits.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "internal.h"

namespace rgbd {
namespace {

constexpr int kRoiThreads = 256;

__device__ __forceinline__ long long floor_q16(long long v) { return v >> 16; }  // arithmetic shift = floor

// One CTA per face.  The scan covers a window that holds every depth pixel which can map inside
// the rect: with p(d) = 256 (parallax / d) between p_lo (at d_max) and p_hi (at d_min), a pixel
// inside needs A = a0 j + a1 i + a2 in [X0 - p_hi, X1 - p_lo) and B = a3 j + a4 i + a5 in [Y0, Y1)
// (X0, X1, Y0, Y1 the rect clipped to the colour image, in Q16.16), a parallelogram in (j, i)
// whose corners bound the window (computed in float, widened by 2 pixels; the per-pixel test
// below is exact, so the window only has to be large enough).
__global__ void __launch_bounds__(kRoiThreads) face_roi_kernel(const uint16_t* __restrict__ depth, int n_frames, int H,
                                                               int W, rgbd_calib c, const rgbd_rect* __restrict__ rects,
                                                               int n, rgbd_rect* __restrict__ out,
                                                               uint32_t* __restrict__ status) {
    __shared__ int red[4][kRoiThreads / 32];
    __shared__ int win[4];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const rgbd_rect r = rects[k];
        const bool bad = r.frame < 0 || r.frame >= n_frames || r.w <= 0 || r.h <= 0;
        if (tid == 0) {
            if (bad) atomicOr(status, RGBD_STATUS_BAD_RECT);
            const long long cx0 = max(0ll, (long long)r.x), cx1 = min((long long)c.colour_w, (long long)r.x + r.w);
            const long long cy0 = max(0ll, (long long)r.y), cy1 = min((long long)c.colour_h, (long long)r.y + r.h);
            int j0 = 0, j1 = -1, i0 = 0, i1 = -1;  // empty
            if (!bad && cx0 < cx1 && cy0 < cy1) {
                const long long p_lo = (long long)(c.parallax / c.d_max) * 256;
                const long long p_hi = (long long)(c.parallax / c.d_min) * 256;
                const float A[2] = {(float)(cx0 * 65536 - p_hi - c.a[2]), (float)(cx1 * 65536 - p_lo - c.a[2])};
                const float Bv[2] = {(float)(cy0 * 65536 - c.a[5]), (float)(cy1 * 65536 - c.a[5])};
                const float det = (float)c.a[0] * (float)c.a[4] - (float)c.a[1] * (float)c.a[3];
                if (fabsf(det) < 1.0f) {  // degenerate mapping: scan the whole frame
                    j0 = 0, j1 = W - 1, i0 = 0, i1 = H - 1;
                } else {
                    float jmn = 3e38f, jmx = -3e38f, imn = 3e38f, imx = -3e38f;
                    for (int u = 0; u < 2; ++u)
                        for (int v = 0; v < 2; ++v) {
                            const float jj = ((float)c.a[4] * A[u] - (float)c.a[1] * Bv[v]) / det;
                            const float ii = ((float)c.a[0] * Bv[v] - (float)c.a[3] * A[u]) / det;
                            jmn = fminf(jmn, jj), jmx = fmaxf(jmx, jj);
                            imn = fminf(imn, ii), imx = fmaxf(imx, ii);
                        }
                    j0 = (int)fmaxf(0.f, floorf(jmn) - 2.f), j1 = (int)fminf((float)(W - 1), ceilf(jmx) + 2.f);
                    i0 = (int)fmaxf(0.f, floorf(imn) - 2.f), i1 = (int)fminf((float)(H - 1), ceilf(imx) + 2.f);
                }
            }
            win[0] = j0, win[1] = j1, win[2] = i0, win[3] = i1;
        }
        __syncthreads();
        const int j0 = win[0], i0 = win[2];
        const int ww = win[1] - j0 + 1, wh = win[3] - i0 + 1;
        int xmin = INT_MAX, ymin = INT_MAX, xmax = -1, ymax = -1;
        if (ww > 0 && wh > 0) {
            const uint16_t* dp = depth + (size_t)r.frame * H * W;
            const long long X0 = (long long)max(r.x, 0) * 65536, X1 = min((long long)r.x + r.w, (long long)c.colour_w) * 65536;
            const long long Y0 = (long long)max(r.y, 0) * 65536, Y1 = min((long long)r.y + r.h, (long long)c.colour_h) * 65536;
            const int area = ww * wh;
            for (int idx = tid; idx < area; idx += kRoiThreads) {
                const int row = idx / ww;
                const int i = i0 + row, j = j0 + (idx - row * ww);
                {
                    const int d = dp[(size_t)i * W + j];
                    if (d < c.d_min || d > c.d_max) continue;
                    const long long X = (long long)c.a[0] * j + (long long)c.a[1] * i + c.a[2] +
                                        (long long)(c.parallax / d) * 256;
                    const long long Y = (long long)c.a[3] * j + (long long)c.a[4] * i + c.a[5];
                    // inside the clipped rect <=> floor(X / 2^16) in [max(x,0), min(x+w, cw)), same for Y
                    if (floor_q16(X) < X0 / 65536 || X >= X1 || floor_q16(Y) < Y0 / 65536 || Y >= Y1) continue;
                    xmin = min(xmin, j), xmax = max(xmax, j);
                    ymin = min(ymin, i), ymax = max(ymax, i);
                }
            }
        }
        // block reduction of the four extremes
        xmin = __reduce_min_sync(0xFFFFFFFFu, xmin);
        ymin = __reduce_min_sync(0xFFFFFFFFu, ymin);
        xmax = __reduce_max_sync(0xFFFFFFFFu, xmax);
        ymax = __reduce_max_sync(0xFFFFFFFFu, ymax);
        if (lane == 0) {
            red[0][warp] = xmin, red[1][warp] = ymin, red[2][warp] = xmax, red[3][warp] = ymax;
        }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < kRoiThreads / 32; ++w) {
                xmin = min(xmin, red[0][w]), ymin = min(ymin, red[1][w]);
                xmax = max(xmax, red[2][w]), ymax = max(ymax, red[3][w]);
            }
            rgbd_rect o;
            o.frame = r.frame;
            if (!bad && xmax >= 0) {
                o.x = xmin, o.y = ymin, o.w = xmax - xmin + 1, o.h = ymax - ymin + 1;
            } else {
                o.x = o.y = o.w = o.h = 0;
            }
            out[k] = o;
        }
        __syncthreads();  // win[] and red[] are reused by the next face
    }
}

}  // namespace
}  // namespace rgbd

using namespace rgbd;

extern "C" int rgbd_face_roi(rgbd_ctx* ctx, const uint16_t* depth, int n_frames, int H, int W, const rgbd_calib* calib,
                             const rgbd_rect* colour_rects, int n, rgbd_rect* depth_rects, void* stream) {
    rgbd::NvtxRange nvtx_range("rgbd_face_roi");
    if (!ctx) return set_error(RGBD_ERR_ARG, "rgbd_face_roi: ctx is NULL");
    if (!calib) return set_error(RGBD_ERR_ARG, "rgbd_face_roi: calib is NULL");
    if (n < 0 || n_frames <= 0 || H <= 0 || W <= 0)
        return set_error(RGBD_ERR_ARG, "rgbd_face_roi: n %d, frames %d, H %d, W %d", n, n_frames, H, W);
    const rgbd_calib c = *calib;
    if (c.d_min < 1 || c.d_max < c.d_min || c.parallax < 0 || c.colour_w <= 0 || c.colour_h <= 0)
        return set_error(RGBD_ERR_ARG, "rgbd_face_roi: calibration depth range %d..%d, parallax %d, colour %dx%d",
                         c.d_min, c.d_max, c.parallax, c.colour_w, c.colour_h);
    for (int i = 0; i < 6; ++i) {
        const int lim = (i == 2 || i == 5) ? (1 << 30) : (1 << 24);  // offsets, linear terms
        if (c.a[i] > lim || c.a[i] < -lim)
            return set_error(RGBD_ERR_ARG, "rgbd_face_roi: calibration entry a[%d] = %d out of range", i, c.a[i]);
    }
    if (n == 0) return RGBD_OK;
    if (!depth || !colour_rects || !depth_rects) return set_error(RGBD_ERR_ARG, "rgbd_face_roi: NULL pointer");
    DeviceGuard g(ctx->props.device);
    const int grid = std::min(n, ctx->props.sm_count * 8);
    face_roi_kernel<<<grid, kRoiThreads, 0, (cudaStream_t)stream>>>(depth, n_frames, H, W, c, colour_rects, n,
                                                                    depth_rects, ctx->d_status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "rgbd_face_roi: launch");
    return RGBD_OK;
}
