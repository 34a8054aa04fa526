// server.cu -- the native request loop (rgbd_server_*): continuous batching of camera frames.
//
// Callers submit frames (host buffers) from any thread.  One worker thread per server admits
// them into a pool of device frame slots, uploads them on a copy stream, and whenever fewer than
// two batches are on the GPU, turns every uploaded frame into one batch: all its faces go
// through one fused feature launch, one scoring launch and one per-stream tracking launch
// (Sections 2.3-2.5 of the paper, per frame), and the results come back to pinned staging and
// then to the caller's buffers.  Frames that arrive while a batch runs are uploaded meanwhile
// and form the next one, so uploads overlap compute and batches follow each other without a
// gap.  The worker polls (it spins with yields while work is in flight) so that a finished
// batch is seen within microseconds: a serving loop trades one host core for latency.
#include <string.h>
#include <time.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "internal.h"

namespace {

double now_s() {
    timespec t;
    clock_gettime(CLOCK_MONOTONIC, &t);
    return (double)t.tv_sec + 1e-9 * (double)t.tv_nsec;
}

struct Request {
    uint64_t id = 0;
    int32_t stream = 0;
    const uint8_t* grey = nullptr;
    const uint16_t* depth = nullptr;
    const rgbd_rect* rects = nullptr;
    int32_t n = 0;
    float* scores = nullptr;
    int32_t* labels = nullptr;
    int32_t* ids = nullptr;
    double t_submit = 0.0;
    int slot = -1;
    bool waited = false;  // found no free slot on its first admission attempt
};

// Buffers of one batch: device rows and outputs, pinned host staging.  Two of them let one batch
// be prepared while the other runs.
// Each direction moves in one copy: the input block holds the batch's rects (frame = slot)
// followed by its meta rows (stream of each frame, then the face starts), the output block its
// scores [faces][C], then labels [faces], then identities [faces] -- offsets that depend on the
// batch's face count.
struct BatchBuf {
    unsigned char* d_in = nullptr;   // device input block (rects, meta)
    unsigned char* h_in = nullptr;   // pinned
    void* d_x = nullptr;             // normalised rows in the model's type
    float* d_xsq = nullptr;
    float* d_out = nullptr;          // device output block (scores, labels, identities)
    float* h_out = nullptr;          // pinned
    uint32_t* h_status = nullptr;    // the context's status word after the batch
    cudaEvent_t done = nullptr;
    bool busy = false;
};
size_t in_bytes(int faces, int n_slots) {
    return sizeof(rgbd_rect) * (size_t)faces + sizeof(int32_t) * (size_t)(2 * n_slots + 1);
}

struct Batch {
    std::vector<Request> reqs;
    int buf = 0;
    bool owns_buf = false;  // holds s->buf[buf] (a request that failed before batching does not)
    int faces = 0;
    int status = RGBD_OK;
};

size_t x_elem_bytes(int dt) {
    if (dt == RGBD_DT_BF16) return 2;
    if (dt == RGBD_DT_FP8) return 1;
    if (dt == RGBD_DT_BF16X3) return 4;  // two bf16 planes
    return 4;
}

}  // namespace

struct rgbd_server {
    rgbd_server_config cfg{};
    const rgbd_svm* model = nullptr;
    rgbd_ctx* ctx = nullptr;
    int device = 0, C = 0, k_pad = 0, x_dtype = 0;
    const float* centre = nullptr;
    uint8_t* d_grey = nullptr;    // [n_slots][H][W]
    uint16_t* d_depth = nullptr;  // [n_slots][H][W]
    rgbd_rect* d_state_rects = nullptr;
    int32_t* d_state_ids = nullptr;
    int32_t* d_state_count = nullptr;
    BatchBuf buf[2];
    cudaStream_t compute = nullptr, copy = nullptr;
    std::vector<cudaEvent_t> slot_ev;  // upload of each slot done
    std::vector<int> free_slots;
    size_t frame_bytes = 0, face_bytes = 0;  // device bytes a frame holds while in flight
    size_t budget = 0, used = 0;              // admission: bytes of the pool frames draw on
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> incoming;      // submitted, not yet seen by the worker
    std::deque<rgbd_completion> done;  // finished, not yet polled
    std::atomic<int> pending{0};       // submitted and not finished
    bool stop = false;
    std::atomic<bool> stopping{false};  // stop, readable without the lock (the idle poll)
    uint64_t next_id = 1;
    std::atomic<uint64_t> frames{0}, faces{0}, batches{0}, waits{0};
    std::thread worker;
};

namespace {

using rgbd::set_error;

// Copies a frame into its slot on `st` and marks the slot's event: the copy stream while a batch
// runs (the upload overlaps it), the compute stream when the GPU is idle (the batch's kernels then
// follow the copy in stream order, without a wait on another stream's event).
int upload(rgbd_server* s, const Request& r, cudaStream_t st) {
    const size_t plane = (size_t)s->cfg.H * s->cfg.W;
    cudaError_t e = cudaMemcpyAsync(s->d_grey + (size_t)r.slot * plane, r.grey, plane, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->d_depth + (size_t)r.slot * plane, r.depth, 2 * plane, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(s->slot_ev[r.slot], st);
    return e == cudaSuccess ? RGBD_OK : rgbd::cuda_error(e, "rgbd_server: upload");
}

// Enqueues one batch (the uploaded frames in `b.reqs`) on the compute stream.
int launch(rgbd_server* s, Batch& b) {
    BatchBuf& bb = s->buf[b.buf];
    const rgbd_server_config& c = s->cfg;
    const int nf = (int)b.reqs.size();
    int faces = 0;
    for (const Request& r : b.reqs) faces += r.n;
    b.faces = faces;
    rgbd_rect* h_rects = reinterpret_cast<rgbd_rect*>(bb.h_in);
    int32_t* h_meta = reinterpret_cast<int32_t*>(bb.h_in + sizeof(rgbd_rect) * (size_t)faces);
    int at = 0;
    for (int f = 0; f < nf; ++f) {
        const Request& r = b.reqs[f];
        for (int i = 0; i < r.n; ++i) {
            rgbd_rect q = r.rects[i];
            q.frame = r.slot;
            h_rects[at + i] = q;
        }
        h_meta[f] = r.stream;
        h_meta[c.n_slots + f] = at;
        at += r.n;
        cudaError_t e = cudaStreamWaitEvent(s->compute, s->slot_ev[r.slot], 0);
        if (e != cudaSuccess) return rgbd::cuda_error(e, "rgbd_server: wait for upload");
    }
    h_meta[c.n_slots + nf] = faces;
    const rgbd_rect* d_rects = reinterpret_cast<const rgbd_rect*>(bb.d_in);
    const int32_t* d_meta = reinterpret_cast<const int32_t*>(bb.d_in + sizeof(rgbd_rect) * (size_t)faces);
    float* d_scores = bb.d_out;
    int32_t* d_labels = reinterpret_cast<int32_t*>(bb.d_out + (size_t)faces * s->C);
    int32_t* d_ids = d_labels + faces;
    cudaError_t e = cudaMemcpyAsync(bb.d_in, bb.h_in, in_bytes(faces, c.n_slots), cudaMemcpyHostToDevice, s->compute);
    if (e != cudaSuccess) return rgbd::cuda_error(e, "rgbd_server: batch upload");
    const size_t k_pad = (size_t)s->k_pad;
    int rc = lbp_fused_features(s->ctx, s->d_grey, s->d_depth, c.n_slots, c.H, c.W, d_rects, nullptr, faces,
                                c.crop, rgbd::kCell, c.mask_mm, c.flags, nullptr, s->x_dtype, bb.d_x, (int)k_pad,
                                c.x_scale, s->centre, bb.d_xsq, s->compute);
    if (!rc) rc = svm_score(s->ctx, s->model, bb.d_x, bb.d_xsq, faces, c.x_scale, d_scores, d_labels, s->compute);
    if (!rc)
        rc = rgbd_track_streams(s->ctx, s->d_state_rects, s->d_state_ids, s->d_state_count, c.n_streams, c.max_faces,
                                nf, d_meta, d_meta + c.n_slots, d_rects, faces, d_labels, d_ids, s->compute);
    if (rc) return rc;
    if (faces > 0) {
        e = cudaMemcpyAsync(bb.h_out, bb.d_out, sizeof(float) * (size_t)faces * (s->C + 2), cudaMemcpyDeviceToHost,
                            s->compute);
        if (e != cudaSuccess) return rgbd::cuda_error(e, "rgbd_server: result read-back");
    }
    // the batch's device status flags, read back and cleared for the next batch
    e = cudaMemcpyAsync(bb.h_status, s->ctx->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s->compute);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->ctx->d_status, 0, sizeof(uint32_t), s->compute);
    if (e != cudaSuccess) return rgbd::cuda_error(e, "rgbd_server: status read-back");
    return RGBD_OK;
}

// Results of a finished batch into the callers' buffers; its slots and buffers become free.
void finish(rgbd_server* s, Batch& b) {
    BatchBuf& bb = s->buf[b.buf];
    const float* h_scores = bb.h_out;
    const int32_t* h_labels = reinterpret_cast<const int32_t*>(bb.h_out + (size_t)b.faces * s->C);
    const int32_t* h_ids = h_labels + b.faces;
    int off = 0;
    std::vector<rgbd_completion> out;
    out.reserve(b.reqs.size());
    for (const Request& r : b.reqs) {
        if (b.status == RGBD_OK && r.n > 0) {
            memcpy(r.scores, h_scores + (size_t)off * s->C, sizeof(float) * (size_t)r.n * s->C);
            memcpy(r.labels, h_labels + off, sizeof(int32_t) * (size_t)r.n);
            if (r.ids) memcpy(r.ids, h_ids + off, sizeof(int32_t) * (size_t)r.n);
        }
        off += r.n;
        if (r.slot >= 0) s->used -= s->frame_bytes + (size_t)r.n * s->face_bytes;
        rgbd_completion c;
        c.request_id = r.id;
        c.status = b.status;
        c.flags = (b.owns_buf && b.status == RGBD_OK) ? *bb.h_status : 0u;
        c.n_faces = r.n;
        c.t_submit = r.t_submit;
        c.t_done = now_s();
        out.push_back(c);
        s->free_slots.push_back(r.slot);
    }
    if (b.owns_buf) bb.busy = false;
    s->frames += b.reqs.size();
    s->faces += (uint64_t)off;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (const rgbd_completion& c : out) s->done.push_back(c);
    }
    s->pending -= (int)b.reqs.size();
    s->cv_done.notify_all();
}

void worker_main(rgbd_server* s) {
    cudaSetDevice(s->device);
    std::deque<Request> waiting;   // seen, waiting for a slot
    std::deque<Request> admitted;  // in a slot (uploading or uploaded)
    std::deque<Batch> inflight;
    for (;;) {
        bool progress = false;
        if (waiting.empty() && admitted.empty() && inflight.empty() && s->cfg.idle_spin_us > 0) {
            // out of work: poll for a submission for a while before sleeping on the condition
            // variable (a sleeping thread wakes through the scheduler, which adds tens of
            // microseconds to the next frame)
            const double t_idle = now_s(), spin = 1e-6 * s->cfg.idle_spin_us;
            while (s->pending.load(std::memory_order_acquire) == 0 && !s->stopping.load(std::memory_order_acquire) &&
                   now_s() - t_idle < spin)
                std::this_thread::yield();
        }
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (waiting.empty() && admitted.empty() && inflight.empty() && s->incoming.empty()) {
                if (s->stop) break;
                s->cv_work.wait(lk, [&] { return s->stop || !s->incoming.empty(); });
            }
            while (!s->incoming.empty()) {
                waiting.push_back(s->incoming.front());
                s->incoming.pop_front();
                progress = true;
            }
        }
        // finished batches first: they free slots and buffers
        while (!inflight.empty()) {
            const cudaError_t q = cudaEventQuery(s->buf[inflight.front().buf].done);
            if (q == cudaErrorNotReady) break;
            if (q != cudaSuccess && inflight.front().status == RGBD_OK)
                inflight.front().status = rgbd::cuda_error(q, "rgbd_server: batch");
            finish(s, inflight.front());
            inflight.pop_front();
            progress = true;
        }
        // admission, in arrival order: a frame needs a free slot and its bytes (planes, and per
        // face the rows it occupies until done) within the pool's budget
        while (!waiting.empty() && !s->free_slots.empty() &&
               s->used + s->frame_bytes + (size_t)waiting.front().n * s->face_bytes <= s->budget) {
            Request r = waiting.front();
            waiting.pop_front();
            s->used += s->frame_bytes + (size_t)r.n * s->face_bytes;
            r.slot = s->free_slots.back();
            s->free_slots.pop_back();
            if (r.waited) s->waits++;
            const int rc = upload(s, r, inflight.empty() ? s->compute : s->copy);
            if (rc) {  // reported through the batch that carries it
                Batch bad;
                bad.reqs.push_back(r);
                bad.status = rc;
                finish(s, bad);
                continue;
            }
            admitted.push_back(r);
            progress = true;
        }
        for (Request& r : waiting) r.waited = true;
        // a new batch of all uploaded frames (up to the face limit) when a buffer set is free
        if (!admitted.empty() && inflight.size() < 2) {
            Batch b;
            b.buf = s->buf[0].busy ? 1 : 0;
            int faces = 0;
            while (!admitted.empty() && faces + admitted.front().n <= s->cfg.max_batch_faces) {
                faces += admitted.front().n;
                b.reqs.push_back(admitted.front());
                admitted.pop_front();
            }
            s->buf[b.buf].busy = true;
            b.owns_buf = true;
            b.status = launch(s, b);
            const cudaError_t e = cudaEventRecord(s->buf[b.buf].done, s->compute);
            if (e != cudaSuccess && b.status == RGBD_OK) b.status = rgbd::cuda_error(e, "rgbd_server: batch event");
            s->batches++;
            inflight.push_back(std::move(b));
            progress = true;
        }
        if (!progress) std::this_thread::yield();
    }
}

void free_server(rgbd_server* s) {
    for (BatchBuf& bb : s->buf) {
        cudaFree(bb.d_in);
        cudaFree(bb.d_x);
        cudaFree(bb.d_xsq);
        cudaFree(bb.d_out);
        cudaFreeHost(bb.h_in);
        cudaFreeHost(bb.h_out);
        cudaFreeHost(bb.h_status);
        if (bb.done) cudaEventDestroy(bb.done);
    }
    for (cudaEvent_t e : s->slot_ev)
        if (e) cudaEventDestroy(e);
    cudaFree(s->d_grey);
    cudaFree(s->d_depth);
    cudaFree(s->d_state_rects);
    cudaFree(s->d_state_ids);
    cudaFree(s->d_state_count);
    if (s->compute) cudaStreamDestroy(s->compute);
    if (s->copy) cudaStreamDestroy(s->copy);
    if (s->ctx) rgbd_ctx_destroy(s->ctx);
    delete s;
}

}  // namespace

extern "C" {

int rgbd_server_create(const rgbd_svm* model, const rgbd_server_config* cfg, rgbd_server** out) {
    rgbd::NvtxRange nvtx_range("rgbd_server_create");
    if (!model || !cfg || !out) return set_error(RGBD_ERR_ARG, "rgbd_server_create: NULL argument");
    *out = nullptr;
    const rgbd_server_config c = *cfg;
    if (!model->scorable) return set_error(RGBD_ERR_ARG, "rgbd_server_create: the model has no coefficients");
    if (c.n_slots < 1 || c.n_slots > 1024 || c.max_batch_faces < 1 || c.max_batch_faces > 65536)
        return set_error(RGBD_ERR_ARG, "rgbd_server_create: n_slots %d (1..1024), max_batch_faces %d (1..65536)",
                         c.n_slots, c.max_batch_faces);
    if (c.H < 1 || c.W < 1 || c.H > 65535 || c.W > 65535)
        return set_error(RGBD_ERR_ARG, "rgbd_server_create: frame %d x %d", c.H, c.W);
    if (c.crop != 32 && c.crop != 64 && c.crop != 96 && c.crop != 128)
        return set_error(RGBD_ERR_ARG, "rgbd_server_create: crop %d (32, 64, 96 or 128)", c.crop);
    if (model->dim != (c.crop / rgbd::kCell) * (c.crop / rgbd::kCell) * rgbd::kBins)
        return set_error(RGBD_ERR_ARG, "rgbd_server_create: model dim %d does not match crop %d", model->dim, c.crop);
    if (c.mask_mm < 1 || (c.flags & ~(RGBD_LBP_GE | RGBD_LBP_NBR_IGNORE_MASK)) != 0)
        return set_error(RGBD_ERR_ARG, "rgbd_server_create: mask_mm %d, flags 0x%x", c.mask_mm, c.flags);
    if (c.n_streams < 1 || c.n_streams > 65536 || c.max_faces < 1 || c.max_faces > 256)
        return set_error(RGBD_ERR_ARG, "rgbd_server_create: n_streams %d (1..65536), max_faces %d (1..256)",
                         c.n_streams, c.max_faces);
    if (c.idle_spin_us < 0 || c.idle_spin_us > 1000000)
        return set_error(RGBD_ERR_ARG, "rgbd_server_create: idle_spin_us %d (0..1000000)", c.idle_spin_us);
    if (model->dtype == RGBD_DT_FP8 && !(c.x_scale > 0.f && c.x_scale < 1e30f))
        return set_error(RGBD_ERR_ARG, "rgbd_server_create: FP8 models need x_scale > 0");
    rgbd_server* s = new (std::nothrow) rgbd_server();
    if (!s) return set_error(RGBD_ERR_NOMEM, "rgbd_server_create: host allocation");
    s->cfg = c;
    s->model = model;
    s->device = model->device;
    s->C = model->C;
    s->k_pad = model->k_pad;
    s->x_dtype = model->kernel == RGBD_KERNEL_LINEAR ? RGBD_DT_F32 : model->dtype;
    s->centre = model->centre;
    rgbd::DeviceGuard g(s->device);
    int rc = rgbd_ctx_create(s->device, &s->ctx);
    if (rc) {
        delete s;
        return rc;
    }
    const size_t plane = (size_t)c.H * c.W, nb = (size_t)c.max_batch_faces, ns = (size_t)c.n_slots;
    cudaError_t e = cudaSuccess;
    auto dev = [&](void** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, std::max<size_t>(bytes, 16));
    };
    auto pin = [&](void** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMallocHost(p, std::max<size_t>(bytes, 16));
    };
    dev((void**)&s->d_grey, ns * plane);
    dev((void**)&s->d_depth, 2 * ns * plane);
    dev((void**)&s->d_state_rects, sizeof(rgbd_rect) * (size_t)c.n_streams * c.max_faces);
    dev((void**)&s->d_state_ids, sizeof(int32_t) * (size_t)c.n_streams * c.max_faces);
    dev((void**)&s->d_state_count, sizeof(int32_t) * (size_t)c.n_streams);
    if (e == cudaSuccess) e = cudaMemset(s->d_state_count, 0, sizeof(int32_t) * (size_t)c.n_streams);
    for (BatchBuf& bb : s->buf) {
        dev((void**)&bb.d_in, in_bytes(c.max_batch_faces, c.n_slots));
        dev(&bb.d_x, x_elem_bytes(s->x_dtype) * nb * (size_t)s->k_pad);
        dev((void**)&bb.d_xsq, sizeof(float) * nb);
        dev((void**)&bb.d_out, sizeof(float) * nb * (s->C + 2));
        pin((void**)&bb.h_in, in_bytes(c.max_batch_faces, c.n_slots));
        pin((void**)&bb.h_out, sizeof(float) * nb * (s->C + 2));
        pin((void**)&bb.h_status, sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bb.done, cudaEventDisableTiming);
    }
    s->slot_ev.assign(ns, nullptr);
    for (size_t i = 0; i < ns && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&s->slot_ev[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->compute, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        rc = e == cudaErrorMemoryAllocation ? set_error(RGBD_ERR_NOMEM, "rgbd_server_create: device or pinned memory")
                                            : rgbd::cuda_error(e, "rgbd_server_create");
        free_server(s);
        return rc;
    }
    if (e == cudaSuccess && model->kernel == RGBD_KERNEL_RBF) {
        // the scoring workspace of the largest batch of either scoring path (at most 128 rows
        // split over K, more rows by SV tiles), reserved now: growing it during serving would
        // put a cudaFree / cudaMalloc pair, which wait for the device, in a frame's latency
        size_t ws = 0;
        for (int nq : {std::min(128, c.max_batch_faces), c.max_batch_faces})
            ws = std::max(ws, model->dtype == RGBD_DT_F32 ? rgbd::score_rbf_f32_bytes(s->ctx, model, nq)
                                                           : rgbd::score_rbf_tc_bytes(s->ctx, model, nq));
        rc = ws ? rgbd::ensure_workspace(s->ctx, ws, nullptr) : RGBD_OK;
        if (rc) {
            free_server(s);
            return rc;
        }
    }
    for (int i = c.n_slots - 1; i >= 0; --i) s->free_slots.push_back(i);
    s->frame_bytes = 3 * plane;
    s->face_bytes = x_elem_bytes(s->x_dtype) * (size_t)s->k_pad + sizeof(float) * (1 + (size_t)s->C) +
                    3 * sizeof(int32_t) + sizeof(rgbd_rect);
    s->budget = ns * s->frame_bytes + 2 * nb * s->face_bytes;
    try {
        s->worker = std::thread(worker_main, s);
    } catch (...) {
        free_server(s);
        return set_error(RGBD_ERR_NOMEM, "rgbd_server_create: worker thread");
    }
    *out = s;
    return RGBD_OK;
}

int rgbd_server_submit(rgbd_server* s, int32_t stream_id, const uint8_t* grey, const uint16_t* depth,
                       const rgbd_rect* rects, int32_t n_faces, float* scores, int32_t* labels, int32_t* ids,
                       uint64_t* request_id) {
    if (!s || !grey || !depth || !request_id) return set_error(RGBD_ERR_ARG, "rgbd_server_submit: NULL argument");
    if (stream_id < 0 || stream_id >= s->cfg.n_streams)
        return set_error(RGBD_ERR_ARG, "rgbd_server_submit: stream %d of %d", stream_id, s->cfg.n_streams);
    if (n_faces < 0 || n_faces > s->cfg.max_batch_faces)
        return set_error(RGBD_ERR_ARG, "rgbd_server_submit: %d faces (0..%d)", n_faces, s->cfg.max_batch_faces);
    if (n_faces > 0 && (!rects || !scores || !labels))
        return set_error(RGBD_ERR_ARG, "rgbd_server_submit: NULL rects, scores or labels");
    Request r;
    r.stream = stream_id;
    r.grey = grey;
    r.depth = depth;
    r.rects = rects;
    r.n = n_faces;
    r.scores = scores;
    r.labels = labels;
    r.ids = ids;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return set_error(RGBD_ERR_ARG, "rgbd_server_submit: the server is stopping");
        r.id = s->next_id++;
        r.t_submit = now_s();
        s->incoming.push_back(r);
        s->pending++;
    }
    s->cv_work.notify_one();
    *request_id = r.id;
    return RGBD_OK;
}

int rgbd_server_poll(rgbd_server* s, rgbd_completion* done, int32_t max, int32_t* n_done, int32_t wait_us) {
    if (!s || !n_done || (max > 0 && !done)) return set_error(RGBD_ERR_ARG, "rgbd_server_poll: NULL argument");
    *n_done = 0;
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->done.empty() && wait_us > 0)
        s->cv_done.wait_for(lk, std::chrono::microseconds(wait_us), [&] { return !s->done.empty(); });
    int k = 0;
    while (k < max && !s->done.empty()) {
        done[k++] = s->done.front();
        s->done.pop_front();
    }
    *n_done = k;
    return RGBD_OK;
}

int rgbd_server_stats(rgbd_server* s, uint64_t* frames, uint64_t* faces, uint64_t* batches, uint64_t* waits) {
    if (!s) return set_error(RGBD_ERR_ARG, "rgbd_server_stats: NULL server");
    if (frames) *frames = s->frames.load();
    if (faces) *faces = s->faces.load();
    if (batches) *batches = s->batches.load();
    if (waits) *waits = s->waits.load();
    return RGBD_OK;
}

int rgbd_server_destroy(rgbd_server* s) {
    if (!s) return RGBD_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->stopping.store(true, std::memory_order_release);
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    rgbd::DeviceGuard g(s->device);
    cudaDeviceSynchronize();
    free_server(s);
    return RGBD_OK;
}

}  // extern "C"
