/*
 * rgbd_lbp.h -- C ABI of the GB300 (sm_103a) depth-fused LBP + SVM library.
 *
 * The library implements the GPU hot path of Naik & Rathna, "Robust real time
 * face recognition and tracking on GPU using fusion of RGB and depth image"
 * (arXiv 1504.01883): for each face rectangle, an affine resample of the grey
 * and depth frames (Section 2.1, Eq. 1), a depth mask around the face's median
 * depth (the depth/grey fusion of Sections 1 and 2.5), 8-neighbour radius-1 LBP
 * codes (Section 2.4, Eq. 2, Fig. 7), per-cell uniform-pattern histograms
 * concatenated into the feature vector (Section 2.4, Eq. 3; Section 3), and
 * the SVM decision function that scores those vectors (Section 2.5).
 *
 * Conventions shared by every call:
 *  - Every call returns an int status: RGBD_OK (0) or a negative RGBD_ERR_*.
 *    rgbd_last_error() returns the calling thread's last message.  Nothing
 *    throws across this boundary.
 *  - Every data pointer is a DEVICE pointer owned by the caller, unless the
 *    argument says otherwise.  The library owns only rgbd_ctx and rgbd_svm.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is enqueued asynchronously on it; only argument checks
 *    run synchronously.  A call that must grow the context workspace
 *    allocates device memory first (synchronous); call rgbd_ctx_reserve()
 *    before capturing calls into a CUDA graph.
 *  - Sizes are int32 element counts; arrays are dense and row-major.
 *  - Problems that only the device can see (a descriptor whose frame index is
 *    out of range, a pipeline wait that ran out of time) do not abort the
 *    call: the affected output rows are written as zeros and a bit is set in
 *    the context's status word, read with rgbd_ctx_status().
 */
#ifndef RGBD_LBP_H
#define RGBD_LBP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------------------- */
#define RGBD_OK 0
#define RGBD_ERR_ARG (-1)         /* an argument is out of range or inconsistent */
#define RGBD_ERR_NOMEM (-2)       /* device allocation failed */
#define RGBD_ERR_CUDA (-3)        /* a CUDA runtime call or a launch failed */
#define RGBD_ERR_TIMEOUT (-4)     /* a device-side wait ran out of time */
#define RGBD_ERR_UNSUPPORTED (-5) /* a valid request this build does not implement */

/* ---- bits of the device status word (rgbd_ctx_status) ------------------------------- */
#define RGBD_STATUS_BAD_RECT 0x1u     /* a descriptor had frame out of range or w, h <= 0 */
#define RGBD_STATUS_WAIT_TIMEOUT 0x2u /* a bounded pipeline wait expired; outputs are invalid */

/* ---- element types of normalised feature rows and packed models ---------------------- */
#define RGBD_DT_F32 1  /* fp32 storage, scored with exact fp32 SIMT arithmetic */
#define RGBD_DT_BF16 2 /* bfloat16 storage, scored on tcgen05 tensor cores, fp32 accumulate */
#define RGBD_DT_FP8 3  /* FP8 E4M3 storage with a per-tensor scale, tcgen05, fp32 accumulate */
#define RGBD_DT_TF32 4 /* fp32 storage, scored on tcgen05 tensor cores as TF32 */
#define RGBD_DT_BF16X3 5 /* two bfloat16 planes, hi = bf16(x) and lo = bf16(x - hi), so x = hi + lo
                            to 2^-18; scored with three BF16 MMAs (hi.hi + hi.lo + lo.hi), fp32
                            accumulate.  A row buffer holds the hi plane [n][k_pad] followed by
                            the lo plane [n][k_pad]. */
#define RGBD_DT_CENTRED 0x100 /* svm_train_data_pack flag, OR-ed into an RBF model's dtype: the
                            support vectors are stored relative to their mean mu (a float per
                            feature column, computed in fp64 and rounded to fp32).  The RBF
                            kernel depends only on x - sv_i, so the scores are those of the
                            uncentred model up to rounding, while the centred values are about
                            half as large in magnitude and their bf16 / FP8 rounding error
                            shrinks with them.  Rows scored against such a model must be
                            centred at the same mu: pass rgbd_svm_centre()'s pointer as
                            x_centre to lbp_fused_features / lbp_normalize_features. */

/* ---- SVM kernels ------------------------------------------------------------------------- */
#define RGBD_KERNEL_LINEAR 0 /* S_c = w_c . x + b_c */
#define RGBD_KERNEL_RBF 1    /* S_c = sum_i a_ci exp(-gamma |x - sv_i|^2) + b_c */

/* ---- LBP option flags ------------------------------------------------------------------- */
#define RGBD_LBP_GE 0x1               /* s(g_p - g_c) = [g_p >= g_c] instead of [g_p > g_c] */
#define RGBD_LBP_NBR_IGNORE_MASK 0x2  /* neighbours compare on grey whatever their depth */
#define RGBD_LBP_FACE_HIST256 0x4     /* one 0-255 histogram of the raw codes per face (Section 3's
                                         form): cell must equal crop, crop 8..255, dim = 256 */

/* A face rectangle on frame `frame`: top-left (x, y), width w, height h, in
 * frame pixels.  It may extend past the frame border (taps are clamped). */
typedef struct rgbd_rect {
    int32_t frame, x, y, w, h;
} rgbd_rect;

typedef struct rgbd_ctx rgbd_ctx;
typedef struct rgbd_svm rgbd_svm;

/* Shape of a packed model (host struct filled by rgbd_svm_get_info). */
typedef struct rgbd_svm_info {
    int32_t kernel;    /* RGBD_KERNEL_* */
    int32_t dtype;     /* RGBD_DT_* of the packed support vectors */
    int32_t n_sv;      /* support vectors (0 for a linear model) */
    int32_t n_sv_pad;  /* rows of the packed SV matrix */
    int32_t dim;       /* feature length (cells * nbins) */
    int32_t k_pad;     /* row stride of packed vectors and of x given to svm_score */
    int32_t n_classes;
    int32_t scorable;  /* 0 when packed without coefficients */
    float gamma;
    float sv_scale;    /* FP8 per-tensor scale of the SVs (1 otherwise) */
    int32_t centred;   /* 1 when packed with RGBD_DT_CENTRED */
} rgbd_svm_info;

/* ======================================================================================= */
/* Context                                                                                 */
/* ======================================================================================= */

/* Library version, (major << 16) | minor. */
int rgbd_version(void);

/* Copies the calling thread's last error message (NUL-terminated, truncated to
 * len) into buf.  Returns the untruncated length.  buf: host memory. */
int rgbd_last_error(char* buf, size_t len);

/* Creates a context bound to CUDA device `device`: a device status word, the
 * workspace (grown on demand) and cached device properties.  *out receives a
 * library-owned handle, freed by rgbd_ctx_destroy.  Errors: RGBD_ERR_ARG (bad
 * device, out == NULL), RGBD_ERR_CUDA, RGBD_ERR_NOMEM. */
int rgbd_ctx_create(int device, rgbd_ctx** out);

/* Frees the context and its device memory.  Synchronises the device first. */
int rgbd_ctx_destroy(rgbd_ctx* ctx);

/* Grows the context workspace to at least `bytes` (synchronous).  Call it
 * before capturing library calls into a CUDA graph. */
int rgbd_ctx_reserve(rgbd_ctx* ctx, size_t bytes);

/* Reads the device status word (synchronises the device).  flags (host) may be
 * NULL; with clear != 0 the word is reset to 0 afterwards. */
int rgbd_ctx_status(rgbd_ctx* ctx, uint32_t* flags, int clear);

/* Launch-shape knobs of a context, set by an autotuner (0 restores the built-in choice).
 * They change only how work is laid out on the GPU, never a result bit of the integer
 * path; scores change within rounding (the split of the SV sum).
 *   RGBD_TUNE_LBP_CTAS_PER_SM   resident fused-kernel CTAs per SM (1 or 2)
 *   RGBD_TUNE_TC_SPLITS         SV-tile ranges per 128-row block in tensor-core scoring
 *   RGBD_TUNE_LBP_SHAPE         fused-kernel tile shape: 0 = default (2), 1 = one thread
 *                               per 8 x 8 cell (crops 64 and 128; CTAs of (crop/8)^2
 *                               threads), 2 = one thread per 4 x 8 half cell (CTAs of
 *                               2 (crop/8)^2 threads), 3 = one thread per 4 x 4 quarter
 *                               cell (crops 64 and 128; CTAs of 4 (crop/8)^2 threads)
 *   RGBD_TUNE_TC_PAIRING        CTA pairing of 128-row blocks in tensor-core scoring:
 *                               0 = default (3), 2 = no pairing, 3 = each pair runs one
 *                               256-row MMA (tcgen05 cta_group::2, each CTA holding half of
 *                               the SV tile)
 *   RGBD_TUNE_TC_SPLITK         tensor-core scoring of at most 128 rows: 0 = default (the K
 *                               extent of every SV tile is split over several CTAs when the
 *                               tiles alone would occupy fewer than half the SMs), 1 = never,
 *                               k >= 2 = always, in k ranges (at most one per 8 k-blocks)
 * Errors: RGBD_ERR_ARG for an unknown key, a negative value, a pairing other than 0, 2, 3 or
 * more than 4096 K ranges. */
#define RGBD_TUNE_LBP_CTAS_PER_SM 1
#define RGBD_TUNE_TC_SPLITS 2
#define RGBD_TUNE_TC_PAIRING 3
#define RGBD_TUNE_LBP_SHAPE 4
#define RGBD_TUNE_TC_SPLITK 5
int rgbd_ctx_set_tuning(rgbd_ctx* ctx, int key, int value);

/* ======================================================================================= */
/* Depth-space region of interest of a colour-detected face (Section 2.1)                   */
/* ======================================================================================= */

/* Depth-to-colour pixel mapping: a stand-in for the camera SDK's per-pixel mapping, exact in
 * integers.  A depth pixel (column j, row i) holding d millimetres, d_min <= d <= d_max, maps to
 * the colour image point
 *   X_q = a[0]*j + a[1]*i + a[2] + (parallax / d) * 256,   Y_q = a[3]*j + a[4]*i + a[5]
 * in Q16.16 (64-bit arithmetic; parallax / d is the integer quotient, parallax >= 0 in units of
 * 1/256 pixel x mm: the stereo shift that grows as the object comes nearer), i.e. colour pixel
 * (X_q >> 16, Y_q >> 16) (floor).  Depths outside [d_min, d_max] (holes included) do not map. */
typedef struct rgbd_calib {
    int32_t a[6];
    int32_t parallax;
    int32_t d_min, d_max;     /* millimetres, 1 <= d_min <= d_max */
    int32_t colour_w, colour_h;
} rgbd_calib;

/* For each face rect detected in the colour image, the bounding rect, in depth pixels, of all
 * depth pixels of its frame that map inside the colour image and inside that rect (Section 2.1:
 * the depth pixels of the face are found through the camera mapping, and the rectangle bounding
 * them is the face region of the depth image; a contour or an ellipse fitted to that point set
 * has the same bounding rect).
 *   depth        uint16 [n_frames][H][W] (device)
 *   calib        host pointer, copied at the call
 *   colour_rects rgbd_rect [n] (device): frame index and the rect in colour pixels
 *   depth_rects  rgbd_rect [n] (device, out): (frame, x_min, y_min, x_max - x_min + 1,
 *                y_max - y_min + 1) over the mapped pixels; (frame, 0, 0, 0, 0) when none maps
 * A rect with frame out of range or w, h <= 0 gives (frame, 0, 0, 0, 0) and
 * RGBD_STATUS_BAD_RECT.  Errors: RGBD_ERR_ARG (NULL pointers, sizes, a calibration with
 * d_min < 1, d_max < d_min, parallax < 0, colour sizes <= 0, |a[0]|, |a[1]|, |a[3]|, |a[4]|
 * above 2^24 or |a[2]|, |a[5]| above 2^30). */
int rgbd_face_roi(rgbd_ctx* ctx, const uint16_t* depth, int n_frames, int H, int W, const rgbd_calib* calib,
                  const rgbd_rect* colour_rects, int n, rgbd_rect* depth_rects, void* stream);

/* ======================================================================================= */
/* A1: affine crop (Section 2.1, Eq. 1 p' = x.u + y.v + t; Section 3: each face is      */
/* resized to a fixed square)                                                              */
/* ======================================================================================= */

/* Resamples n_rects rectangles of the registered grey / depth frames into
 * out_h x out_w crops.
 *   grey   uint8  [n_frames][H][W]
 *   depth  uint16 [n_frames][H][W], millimetres, 0 = hole
 *   rects  rgbd_rect [n_rects] (device)
 *   affine_q16  NULL, or int32 [n_rects][6] = (a00, a01, t0, a10, a11, t1) in
 *          Q16.16: crop pixel (u, v) reads source point
 *          (a00*u + a01*v + t0, a10*u + a11*v + t1) / 2^16 (Eq. 1 with basis
 *          vectors (a00, a10), (a01, a11) and origin (t0, t1)).  When NULL the
 *          rect maps pixel centres to pixel centres:
 *          X_q(u) = x*2^16 + floor((2u+1) * w * 2^16 / (2*out_w)) - 2^15.
 *   out_grey  uint8  [n_rects][out_h][out_w]: bilinear, Q8 weights, round half up
 *   out_depth uint16 [n_rects][out_h][out_w]: nearest, never interpolated
 * Taps outside the frame are clamped to the border.  A descriptor with frame
 * out of range or w, h <= 0 gives zero crops and RGBD_STATUS_BAD_RECT.
 * Errors: RGBD_ERR_ARG (NULL pointers, n_rects < 0, sizes <= 0). */
int rgbd_crop_affine(rgbd_ctx* ctx, const uint8_t* grey, const uint16_t* depth, int n_frames, int H,
                     int W, const rgbd_rect* rects, const int32_t* affine_q16, int n_rects,
                     int out_h, int out_w, uint8_t* out_grey, uint16_t* out_depth, void* stream);

/* ======================================================================================= */
/* A1-A5 fused: crop, median-depth mask, LBP codes, uniform-59 cell histograms and      */
/* the per-cell normalisation, in one persistent launch (Sections 2.1, 2.4, 3)            */
/* ======================================================================================= */

/* For each of n faces: the crop of A1 (crop x crop), the lower median m of the
 * crop's non-zero depths, the mask valid = (d != 0 && |d - m| < mask_mm), the
 * LBP code of every valid centre (ring p0..p7 clockwise from the top-left
 * neighbour, bit p set when neighbour p is valid and brighter; neighbours past
 * the crop edge replicate it), and one 59-bin histogram per cell x cell block
 * (bins: the 58 codes with at most two circular 0/1 transitions in ascending
 * code order, then one bin for all others).
 *   rects == NULL: the frames already are the crops (n_frames == n,
 *          H == W == crop) and affine_q16 must be NULL.
 *   crop   32, 64, 96 or 128; cell must be 8; mask_mm > 0.
 *   flags  RGBD_LBP_* bits.
 *   feats  uint16 [n][dim], dim = (crop/8)^2 * 59, cell-major, bin fastest;
 *          may be NULL when x_out is given.
 *   x_dtype / x_out / k_pad / x_scale: optional normalised rows
 *          x_j = H_j / n_valid(cell) (IEEE fp32 quotient, 0 for an empty cell),
 *          stored as RGBD_DT_F32 / RGBD_DT_TF32 (float), RGBD_DT_BF16 (round
 *          to nearest even) or RGBD_DT_FP8 (E4M3 of x * x_scale, round to
 *          nearest even, saturating); row stride k_pad >= dim, a multiple of
 *          128; columns dim..k_pad-1 are written as 0.  x_dtype 0 = none.
 *   x_centre  NULL, or device float [dim] (e.g. rgbd_svm_centre() of an
 *          RGBD_DT_CENTRED model): the rows hold x_j - x_centre[j] (fp32
 *          difference, round to nearest even) before the conversion above.
 *   xsq_out  NULL or float [n]: sum of squares of the values x_out represents
 *          (for FP8, of the decoded code / x_scale).
 * Errors: RGBD_ERR_ARG, RGBD_ERR_UNSUPPORTED (cell != 8, crop outside the
 * range), RGBD_ERR_CUDA. */
int lbp_fused_features(rgbd_ctx* ctx, const uint8_t* grey, const uint16_t* depth, int n_frames,
                       int H, int W, const rgbd_rect* rects, const int32_t* affine_q16, int n,
                       int crop, int cell, int mask_mm, int flags, uint16_t* feats, int x_dtype,
                       void* x_out, int k_pad, float x_scale, const float* x_centre, float* xsq_out,
                       void* stream);

/* With flags & RGBD_LBP_FACE_HIST256 the same call computes the paper's own face descriptor
 * (Section 3: one histogram of the raw 8-bit LBP codes, bins 0..255, per face): crop any size
 * 8..255 (the paper resizes faces to 200x200), cell == crop, and feats
 * is uint16 [n][256], bin = raw code.  Mask, codes and normalisation are as above (one cell). */

/* A5 alone: per-cell normalisation of count rows that came from elsewhere (a
 * stored database, synthetic counts).  feats uint16 [n][dim], dim a multiple
 * of nbins; other arguments as in lbp_fused_features. */
int lbp_normalize_features(rgbd_ctx* ctx, const uint16_t* feats, int n, int dim, int nbins,
                           int x_dtype, void* x_out, int k_pad, float x_scale, const float* x_centre,
                           float* xsq_out, void* stream);

/* ======================================================================================= */
/* A5-A7: the SVM (Section 2.5: one-vs-rest, "faces" vs "non-faces" per person)           */
/* ======================================================================================= */

/* Packs a trained SVM into a device-resident model (synchronous on `stream`).
 *   RBF:    sv_feats uint16 [n_sv][dim] are the support vectors' count rows
 *           (normalised per cell here); coef float [n_classes][n_sv] holds
 *           a_ci = alpha_ci * y_ci; gamma > 0.
 *   LINEAR: sv_feats NULL, n_sv 0; coef float [n_classes][dim] holds w_c.
 *   bias   float [n_classes] (NULL = zeros).
 *   dtype  RGBD_DT_*: how SVs are stored and scored (FP8: per-tensor scale
 *          448 / max|sv|, reported in rgbd_svm_info.sv_scale).  A linear
 *          model is always RGBD_DT_F32.  An RBF model may add
 *          RGBD_DT_CENTRED: mu_j = fp32(sum_i x_ij / n_sv), the sum over the
 *          fp32 normalised SV rows taken in fp64 in row order; the stored rows
 *          are fp32(x_ij - mu_j) (then the dtype conversion; FP8 scale 448 /
 *          max|x - mu|), and their squared norms are those of the stored
 *          values.
 *   coef == NULL packs only the normalised SV matrix (for a host trainer,
 *          Section 3 trains on the CPU); such a model is not scorable.
 * *model_out receives a library-owned handle (free with rgbd_svm_free).
 * Errors: RGBD_ERR_ARG, RGBD_ERR_NOMEM, RGBD_ERR_CUDA. */
int svm_train_data_pack(rgbd_ctx* ctx, const uint16_t* sv_feats, int n_sv, int dim, int nbins,
                        const float* coef, const float* bias, int n_classes, int kernel,
                        float gamma, int dtype, rgbd_svm** model_out, void* stream);

int rgbd_svm_free(rgbd_svm* model);

/* info: host struct. */
int rgbd_svm_get_info(const rgbd_svm* model, rgbd_svm_info* info);

/* Device pointers of the packed SV matrix ([n_sv_pad][k_pad], model dtype) and
 * of the squared norms of its rows (float [n_sv_pad]); either may be NULL. */
int rgbd_svm_packed_sv(const rgbd_svm* model, const void** sv, const float** sv_sq);

/* *centre receives the device pointer of an RGBD_DT_CENTRED model's mean mu
 * (float [k_pad], zero past dim; owned by the model), or NULL for a model
 * packed without centring.  Errors: RGBD_ERR_ARG (NULL arguments). */
int rgbd_svm_centre(const rgbd_svm* model, const float** centre);

/* Scores n normalised rows.
 *   x       [n][k_pad] in the model's dtype (float for F32 / TF32 / linear),
 *           as written by lbp_fused_features or lbp_normalize_features
 *           (with the model's centre as x_centre when it was packed with
 *           RGBD_DT_CENTRED).
 *   xsq     float [n], squared norms of the rows (RBF only; may be NULL for a
 *           linear model).
 *   x_scale FP8 per-tensor scale of x (ignored for other dtypes).
 *   scores  float [n][n_classes]: S_c = sum_i a_ci exp(-gamma |x - sv_i|^2) + b_c
 *           (RBF) or w_c . x + b_c (linear).
 *   labels  NULL or int32 [n]: argmax_c S_c, lowest index on ties.
 * Uses context workspace (partial sums), grown on demand.  Tensor-core models
 * score up to 128 rows by splitting the SV tiles' K extent over several CTAs
 * (two launches, the second a programmatic dependent of the first) when the
 * tiles alone would occupy few SMs (RGBD_TUNE_TC_SPLITK); larger batches by SV
 * tiles.  The two paths round differently within the model type's tolerance.
 * Errors: RGBD_ERR_ARG, RGBD_ERR_UNSUPPORTED, RGBD_ERR_NOMEM, RGBD_ERR_CUDA. */
int svm_score(rgbd_ctx* ctx, const rgbd_svm* model, const void* x, const float* xsq, int n,
              float x_scale, float* scores, int32_t* labels, void* stream);

/* ======================================================================================= */
/* SVM training (Section 2.5; the paper trains on the host)                                 */
/* ======================================================================================= */

/* One-vs-rest RBF SVM training of n_classes classifiers on the same n rows.  For class c,
 * y_t = +1 if labels[t] == c else -1, and with K_st = exp(-gamma |x_s - x_t|^2) the dual problem
 *   minimise 1/2 sum_st alpha_s alpha_t y_s y_t K_st - sum_t alpha_t,
 *   0 <= alpha_t <= cost, sum_t y_t alpha_t = 0
 * is solved by sequential minimal optimisation: each step takes the maximal violating pair
 * (i = argmax over the indices that may move up of -y_t G_t, j = argmin over those that may move
 * down, lowest index on ties; G the gradient), stops when the gap is at most eps or after
 * max_iter steps, and otherwise moves the pair along the constraint by the clipped Newton step.
 * The bias makes y_t f(x_t) = 1 on average over the free vectors (0 < alpha < cost), else it is
 * the midpoint of the last bounds.
 *   x        float [n][k_pad] normalised rows (lbp_normalize_features with RGBD_DT_F32)
 *   xsq      float [n] their squared norms
 *   labels   int32 [n], values in 0..n_classes-1 (others train as "rest" in every class)
 *   coef     float [n_classes][n] out: a_ct = y_t alpha_t (svm_train_data_pack's coefficients)
 *   bias     float [n_classes] out: b_c, so that f_c(x) = sum_t a_ct K(x_t, x) + b_c
 *   iters    int32 [n_classes] out: SMO steps taken (max_iter means the gap was not reached)
 * The kernel matrix (4 n^2 bytes, fp32) lives in the context workspace; n is 2..16384,
 * max_iter 0..2e6.  Asynchronous on stream.  Errors: RGBD_ERR_ARG, RGBD_ERR_NOMEM. */
int svm_train_rbf(rgbd_ctx* ctx, const float* x, const float* xsq, int n, int k_pad, const int32_t* labels,
                  int n_classes, float gamma, float cost, float eps, int max_iter, float* coef, float* bias,
                  int32_t* iters, void* stream);

/* ======================================================================================= */
/* Nearest-centre face tracking (Section 2.3)                                              */
/* ======================================================================================= */

/* For each face of the previous frame, the face of the current frame whose rect centre is
 * nearest to its own (Section 2.3: a person's face in the following frame is the detection
 * whose centre lies closest to that person's previous centre).  The `frame` field of each rect is the
 * camera stream id: faces only match faces of the same stream.
 *   prev  rgbd_rect [n_prev], cur rgbd_rect [n_cur] (device)
 *   match int32 [n_prev] (device): index into cur, or -1 when the stream has no current
 *         face.  Centres are compared exactly as (2x + w, 2y + h); ties go to the lowest index.
 * Each previous face is matched independently (two may pick the same current face).
 * Errors: RGBD_ERR_ARG. */
int rgbd_track_nearest(rgbd_ctx* ctx, const rgbd_rect* prev, int n_prev, const rgbd_rect* cur, int n_cur,
                       int32_t* match, void* stream);

/* Per-stream identities across a batch of frames (Section 2.3: each face is followed to the
 * nearest rectangle centre in the next frame of its camera, and the stream's data set is
 * updated at every frame).  The state of every stream -- the rects of its last served frame
 * and the identity of each of those faces -- stays on the device between calls.
 * For each frame f of the batch, in order:
 *   1. every previous face j of stream frame_stream[f] picks the current face of f whose
 *      centre is nearest (exact, as (2x + w, 2y + h); lowest index on ties);
 *   2. a current face picked by one or more previous faces takes the identity of the nearest
 *      of them (lowest j on ties); a face picked by none takes its own label;
 *   3. the stream's state becomes f's first min(faces, max_faces) faces and their identities.
 *   state_rects  rgbd_rect [n_streams][max_faces] (device, caller-owned, updated)
 *   state_ids    int32 [n_streams][max_faces]     (device, updated)
 *   state_count  int32 [n_streams]                (device, updated; zero = no previous frame)
 *   frame_stream int32 [n_frames] stream id of each frame (device)
 *   frame_start  int32 [n_frames + 1]: faces of frame f are rects/labels/ids
 *                [frame_start[f], frame_start[f + 1]) (device)
 *   rects        rgbd_rect [n] (device; the frame field is ignored)
 *   labels       int32 [n] classifier labels (device), ids int32 [n] identities (device, out)
 * max_faces is 1..256.  A frame whose stream id is out of range keeps its labels and leaves the
 * states alone; a frame whose face range is out of bounds is skipped; both set
 * RGBD_STATUS_BAD_RECT.  Asynchronous on stream.  Errors: RGBD_ERR_ARG. */
int rgbd_track_streams(rgbd_ctx* ctx, rgbd_rect* state_rects, int32_t* state_ids, int32_t* state_count,
                       int n_streams, int max_faces, int n_frames, const int32_t* frame_stream,
                       const int32_t* frame_start, const rgbd_rect* rects, int n, const int32_t* labels,
                       int32_t* ids, void* stream);

/* Size of the fixed scratch array behind svm_score_noalloc (16 MiB per GPU). */
#define RGBD_NOALLOC_SCRATCH_BYTES (16u << 20)

/* svm_score for callers that cannot allocate device memory.  The paper has no
 * counterpart: this is a deployment variant of the RBF scoring above.
 *
 * svm_score may grow the context workspace with cudaMalloc.  Some callers
 * cannot allow that: real-time loops that must not meet the device-wide
 * synchronisation that cudaMalloc / cudaFree can cause in the middle of a
 * frame, and processes whose device memory is already handed out by another
 * allocator (a framework's pool, a fixed budget per tenant), where a
 * library-side cudaMalloc can fail or steal memory that was promised
 * elsewhere.  This call allocates nothing: its partial sums live in one
 * file-scope device array of RGBD_NOALLOC_SCRATCH_BYTES that every GPU loading
 * the library holds until the process exits.
 *   - Arguments and results as in svm_score.  Only RBF models packed for the
 *     tensor-core path (RGBD_DT_BF16, RGBD_DT_BF16X3, RGBD_DT_FP8 or
 *     RGBD_DT_TF32); others give RGBD_ERR_UNSUPPORTED.
 *   - The scratch needed grows with n x classes (4 x n x C_pad bytes per SV
 *     split plus small terms); a call that would need more than
 *     RGBD_NOALLOC_SCRATCH_BYTES launches nothing and returns RGBD_ERR_ARG with
 *     the sizes in rgbd_last_error().
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress, which may load the module and so take longer than
 *     later calls); a latency-bound caller makes one warm-up call first.
 *   - Every call on a device shares the one array, which keeps the previous
 *     call's contents (each call overwrites what it reads).  Calls whose work
 *     overlaps on the GPU -- on different streams, or from different threads
 *     -- race on it and give wrong results; order them on one stream. */
int svm_score_noalloc(rgbd_ctx* ctx, const rgbd_svm* model, const void* x, const float* xsq, int n,
                      float x_scale, float* scores, int32_t* labels, void* stream);

/* ======================================================================================= */
/* Native request loop: continuous batching of camera frames (Sections 2.3-2.5 per frame)  */
/* ======================================================================================= */

/* A server runs the whole per-frame path -- upload of the frame, fused features of its faces,
 * scoring against a resident model, per-stream tracking of identities, read-back of the results
 * -- for frames submitted from any host thread, on a worker thread of its own.  Frames are
 * admitted, in submission order, into a pool of device frame slots while a slot is free and
 * their bytes (the planes, and per face the rows it occupies until done) fit the pool's budget
 * (the bytes of all slots and of two full batches); frames that
 * arrive while a batch is on the GPU are uploaded on a copy stream and form the next batch
 * (all their faces in one fused launch and one scoring launch), so uploads overlap compute and
 * batches follow each other without a gap.  While work is in flight the worker polls its
 * events (spinning with yields: one host core for latency); out of work, it keeps polling for
 * idle_spin_us, then sleeps until a submission.
 * The server owns its own context (workspace, face queues); the model must outlive it and is
 * only read. */
typedef struct rgbd_server_config {
    int32_t n_slots;          /* device frame slots (frames in flight), 1..1024 */
    int32_t max_batch_faces;  /* faces per batch, 1..65536; a frame with more is rejected */
    int32_t H, W;             /* frame size: uint8 grey and uint16 depth planes [H][W] */
    int32_t crop;             /* 32, 64, 96 or 128 */
    int32_t mask_mm;          /* depth window around the median, > 0 */
    int32_t flags;            /* RGBD_LBP_* (not RGBD_LBP_FACE_HIST256) */
    int32_t n_streams;        /* camera streams tracked, 1..65536 */
    int32_t max_faces;        /* faces remembered per stream for tracking, 1..256 */
    float x_scale;            /* FP8 per-tensor scale of the rows (FP8 models), else ignored */
    int32_t idle_spin_us;     /* 0..1000000: how long the worker keeps polling for submissions
                                 after it runs out of work before it sleeps (0: at once).  A
                                 sleeping worker wakes through the operating system's scheduler,
                                 tens of microseconds added to the next frame's latency */
} rgbd_server_config;

/* One finished request, as returned by rgbd_server_poll. */
typedef struct rgbd_completion {
    uint64_t request_id;
    int32_t status;           /* RGBD_OK, or the error code of the failed call */
    uint32_t flags;           /* RGBD_STATUS_* raised on the device by the request's batch (e.g. a
                                 bad rect, whose face gets zero features) */
    int32_t n_faces;
    double t_submit;          /* CLOCK_MONOTONIC seconds at submission ... */
    double t_done;            /* ... and when the results were in the caller's buffers */
} rgbd_completion;

typedef struct rgbd_server rgbd_server;

/* Creates a server on the model's device and starts its worker thread.  Allocates the frame
 * slots (3 H W bytes each), two sets of batch buffers and the tracking state (synchronous).
 * Errors: RGBD_ERR_ARG (sizes out of range, a model without coefficients), RGBD_ERR_NOMEM. */
int rgbd_server_create(const rgbd_svm* model, const rgbd_server_config* cfg, rgbd_server** out);

/* Queues one frame of camera stream `stream_id` (0 .. n_streams-1) and returns at once.
 *   grey uint8 [H][W], depth uint16 [H][W]: host memory (pinned memory lets the upload run
 *        asynchronously); rects rgbd_rect [n_faces] host memory, the frame field ignored.
 *   scores float [n_faces][n_classes], labels int32 [n_faces], ids int32 [n_faces] (identities
 *        after tracking): host memory the results are written to; ids may be NULL.
 * All buffers are caller-owned and must stay valid, unchanged, until the request completes.
 * Requests of one stream are served in submission order.  *request_id is its id.
 * Errors: RGBD_ERR_ARG (NULL pointers, stream id or face count out of range, a stopped server). */
int rgbd_server_submit(rgbd_server* s, int32_t stream_id, const uint8_t* grey, const uint16_t* depth,
                       const rgbd_rect* rects, int32_t n_faces, float* scores, int32_t* labels, int32_t* ids,
                       uint64_t* request_id);

/* Moves up to `max` finished requests into done[] (*n_done of them), waiting up to wait_us
 * microseconds for the first one when none is ready (0: do not wait). */
int rgbd_server_poll(rgbd_server* s, rgbd_completion* done, int32_t max, int32_t* n_done, int32_t wait_us);

/* Counters since creation: frames and faces completed, batches launched, admissions that had to
 * wait for a slot; any pointer may be NULL. */
int rgbd_server_stats(rgbd_server* s, uint64_t* frames, uint64_t* faces, uint64_t* batches, uint64_t* waits);

/* Serves every queued request, stops the worker and frees the server. */
int rgbd_server_destroy(rgbd_server* s);

/* ======================================================================================= */
/* Diagnostics                                                                              */
/* ======================================================================================= */

/* rgbd_debug_expm1 -- evaluates, for a test, the e^z - 1 the tensor-core RBF epilogue uses
 * (Section 2.5's kernel value relative to a reference distance, where |z| is small): a
 * degree-6 Taylor polynomial for |z| < 2^-5, expm1f otherwise.
 *   z, out   device fp32 [n] (caller-owned); out[i] = e^z[i] - 1.
 *   Asynchronous on stream.  Errors: RGBD_ERR_ARG for n < 0 or NULL pointers with n > 0. */
int rgbd_debug_expm1(const float* z, float* out, int n, void* stream);

/* rgbd_debug_wait_timeout -- runs, for a test of the failure path, the bounded barrier wait of
 * the tensor-core kernel on a phase that nothing completes: after limit_ns (1 us .. 100 ms) the
 * wait gives up, sets RGBD_STATUS_WAIT_TIMEOUT in the context status and the kernel returns, so
 * the context stays usable.  *result (device int) receives 1 when the wait gave up.
 * Errors: RGBD_ERR_ARG. */
int rgbd_debug_wait_timeout(rgbd_ctx* ctx, uint64_t limit_ns, int* result, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RGBD_LBP_H */
