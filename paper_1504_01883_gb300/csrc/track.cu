// track.cu -- nearest-centre face tracking (Section 2.3): each face of the previous frame is
// followed to the face of the current frame whose rectangle centre is nearest to its own.
#include <stdint.h>

#include "internal.h"

namespace rgbd {
namespace {

// One thread per previous face; the current faces are scanned in index order so ties keep the
// lowest index.  Centres are compared in doubled integer coordinates (2x + w, 2y + h), exactly.
__global__ void track_nearest_kernel(const rgbd_rect* __restrict__ prev, int n_prev, const rgbd_rect* __restrict__ cur,
                                     int n_cur, int32_t* __restrict__ match) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_prev) return;
    const rgbd_rect p = prev[i];
    const int64_t px = 2 * (int64_t)p.x + p.w, py = 2 * (int64_t)p.y + p.h;
    int best = -1;
    int64_t best_d = 0;
    for (int j = 0; j < n_cur; ++j) {
        const rgbd_rect c = cur[j];
        if (c.frame != p.frame) continue;
        const int64_t dx = 2 * (int64_t)c.x + c.w - px, dy = 2 * (int64_t)c.y + c.h - py;
        const int64_t d = dx * dx + dy * dy;
        if (best < 0 || d < best_d) {
            best = j;
            best_d = d;
        }
    }
    match[i] = best;
}

}  // namespace
}  // namespace rgbd

using namespace rgbd;

extern "C" int rgbd_track_nearest(rgbd_ctx* ctx, const rgbd_rect* prev, int n_prev, const rgbd_rect* cur, int n_cur,
                                  int32_t* match, void* stream) {
    if (!ctx) return set_error(RGBD_ERR_ARG, "rgbd_track_nearest: ctx is NULL");
    if (n_prev < 0 || n_cur < 0) return set_error(RGBD_ERR_ARG, "rgbd_track_nearest: negative count");
    if (n_prev == 0) return RGBD_OK;
    if (!prev || !match || (n_cur > 0 && !cur)) return set_error(RGBD_ERR_ARG, "rgbd_track_nearest: NULL pointer");
    DeviceGuard g(ctx->props.device);
    track_nearest_kernel<<<(n_prev + 127) / 128, 128, 0, (cudaStream_t)stream>>>(prev, n_prev, cur, n_cur, match);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "rgbd_track_nearest: launch");
    return RGBD_OK;
}
