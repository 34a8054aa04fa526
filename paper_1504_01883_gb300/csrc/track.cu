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

constexpr int kTrackMaxFaces = 256;

// Per-stream tracking over a batch of frames: one warp per stream id walks the batch's frames
// in order and handles those of its stream (Section 2.3): every previous face picks its nearest
// current face; a current face picked by several takes the identity of the nearest of them
// (lowest index on ties), one picked by none its own label; the stream's state becomes the
// frame's faces.  Block 0 also passes labels through for frames whose stream id is out of range.
__global__ void __launch_bounds__(32) track_streams_kernel(
    rgbd_rect* __restrict__ state_rects, int32_t* __restrict__ state_ids, int32_t* __restrict__ state_count,
    int n_streams, int max_faces, int n_frames, const int32_t* __restrict__ frame_stream,
    const int32_t* __restrict__ frame_start, const rgbd_rect* __restrict__ rects, int n,
    const int32_t* __restrict__ labels, int32_t* __restrict__ ids, uint32_t* __restrict__ status) {
    __shared__ rgbd_rect prev[kTrackMaxFaces];
    __shared__ int32_t pid[kTrackMaxFaces], nid[kTrackMaxFaces], match[kTrackMaxFaces];
    __shared__ long long mdist[kTrackMaxFaces];
    const int s = blockIdx.x, lane = threadIdx.x;
    int np = state_count[s];
    np = np < 0 ? 0 : (np > max_faces ? max_faces : np);
    for (int j = lane; j < np; j += 32) {
        prev[j] = state_rects[(size_t)s * max_faces + j];
        pid[j] = state_ids[(size_t)s * max_faces + j];
    }
    __syncwarp();
    for (int f = 0; f < n_frames; ++f) {
        const int fs = frame_stream[f];
        const int k0 = frame_start[f], nf = frame_start[f + 1] - k0;
        const bool bad = k0 < 0 || nf < 0 || k0 + nf > n;
        if (bad) {
            if (s == 0 && lane == 0) atomicOr(status, RGBD_STATUS_BAD_RECT);
            continue;
        }
        if (fs < 0 || fs >= n_streams) {
            if (s == 0) {
                for (int k = lane; k < nf; k += 32) ids[k0 + k] = labels[k0 + k];
                if (lane == 0) atomicOr(status, RGBD_STATUS_BAD_RECT);
            }
            continue;
        }
        if (fs != s) continue;
        // step 1: nearest current face of every previous face (doubled centres, exact)
        for (int j = lane; j < np; j += 32) {
            const long long px = 2ll * prev[j].x + prev[j].w, py = 2ll * prev[j].y + prev[j].h;
            int best = -1;
            long long bd = 0;
            for (int k = 0; k < nf; ++k) {
                const rgbd_rect c = rects[k0 + k];
                const long long dx = 2ll * c.x + c.w - px, dy = 2ll * c.y + c.h - py;
                const long long d = dx * dx + dy * dy;
                if (best < 0 || d < bd) {
                    best = k;
                    bd = d;
                }
            }
            match[j] = best;
            mdist[j] = bd;
        }
        __syncwarp();
        // step 2: identities of the current faces
        for (int k = lane; k < nf; k += 32) {
            int bj = -1;
            long long bd = 0;
            for (int j = 0; j < np; ++j)
                if (match[j] == k && (bj < 0 || mdist[j] < bd)) {
                    bj = j;
                    bd = mdist[j];
                }
            const int id = bj >= 0 ? pid[bj] : labels[k0 + k];
            ids[k0 + k] = id;
            if (k < max_faces) nid[k] = id;
        }
        __syncwarp();
        // step 3: the stream's state becomes this frame's faces
        np = nf < max_faces ? nf : max_faces;
        for (int k = lane; k < np; k += 32) {
            prev[k] = rects[k0 + k];
            pid[k] = nid[k];
        }
        __syncwarp();
    }
    for (int j = lane; j < np; j += 32) {
        state_rects[(size_t)s * max_faces + j] = prev[j];
        state_ids[(size_t)s * max_faces + j] = pid[j];
    }
    if (lane == 0) state_count[s] = np;
}

}  // namespace
}  // namespace rgbd

using namespace rgbd;

extern "C" int rgbd_track_streams(rgbd_ctx* ctx, rgbd_rect* state_rects, int32_t* state_ids, int32_t* state_count,
                                  int n_streams, int max_faces, int n_frames, const int32_t* frame_stream,
                                  const int32_t* frame_start, const rgbd_rect* rects, int n, const int32_t* labels,
                                  int32_t* ids, void* stream) {
    rgbd::NvtxRange nvtx_range("rgbd_track_streams");
    if (!ctx) return set_error(RGBD_ERR_ARG, "rgbd_track_streams: ctx is NULL");
    if (n_streams < 1 || max_faces < 1 || max_faces > kTrackMaxFaces || n_frames < 0 || n < 0)
        return set_error(RGBD_ERR_ARG, "rgbd_track_streams: n_streams %d, max_faces %d (1..%d), n_frames %d, n %d",
                         n_streams, max_faces, kTrackMaxFaces, n_frames, n);
    if (!state_rects || !state_ids || !state_count || (n_frames > 0 && (!frame_stream || !frame_start)) ||
        (n > 0 && (!rects || !labels || !ids)))
        return set_error(RGBD_ERR_ARG, "rgbd_track_streams: NULL pointer");
    if (n_frames == 0) return RGBD_OK;
    DeviceGuard g(ctx->props.device);
    track_streams_kernel<<<n_streams, 32, 0, (cudaStream_t)stream>>>(state_rects, state_ids, state_count, n_streams,
                                                                    max_faces, n_frames, frame_stream, frame_start,
                                                                    rects, n, labels, ids, ctx->d_status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "rgbd_track_streams: launch");
    return RGBD_OK;
}

extern "C" int rgbd_track_nearest(rgbd_ctx* ctx, const rgbd_rect* prev, int n_prev, const rgbd_rect* cur, int n_cur,
                                  int32_t* match, void* stream) {
    rgbd::NvtxRange nvtx_range("rgbd_track_nearest");
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
