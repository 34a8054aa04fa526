/*
 * rgbd_oracle.c -- plain, slow, single-threaded CPU oracle for the depth-fused
 * LBP + SVM hot path of "Robust real time face recognition and tracking on GPU
 * using fusion of RGB and depth image" (Naik & Rathna, arXiv 1504.01883).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no source, header, table or constant generator
 * with the CUDA library: every definition below is written out from the
 * paper's text and the readings listed beside each function.
 *
 * Precision: the integer steps (resample, median, mask, LBP codes, histograms)
 * are exact.  The per-cell normalisation has two forms: an fp64 one that feeds
 * the fp64 SVM, and the fp32 IEEE quotient the fused kernel must reproduce
 * bit for bit.  SVM scores are computed in fp64, directly from the definition
 * (sum of squared differences, no norm expansion).
 *
 * Pins (what ties this file to something other than itself) live in
 * tests/test_oracle_pins.py.  Every function here has at least one pin.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t frame, x, y, w, h;
} orc_rect;

/* ------------------------------------------------------------------ */
/* S1. Affine resample (Section 2.1, Eq. 1: p' = x.u + y.v + t).       */
/* ------------------------------------------------------------------ */

/* floor(a / b) for b > 0, on int64. */
static int64_t floor_div(int64_t a, int64_t b) {
    int64_t q = a / b;
    if ((a % b != 0) && (a < 0)) q -= 1;
    return q;
}

static int64_t clamp64(int64_t v, int64_t lo, int64_t hi) {
    return v < lo ? lo : (v > hi ? hi : v);
}

/* Source coordinate (Q16.16) of crop pixel index i when a rect side starting
 * at `origin` with length `len` is mapped onto `out_len` crop pixels, pixel
 * centre to pixel centre:  origin + (i + 1/2) * len / out_len - 1/2.
 * The fractional part is taken with floor division so CPU and GPU agree. */
int64_t orc_rect_coord_q16(int32_t origin, int32_t len, int32_t out_len, int32_t i) {
    int64_t num = (int64_t)(2 * (int64_t)i + 1) * (int64_t)len * 65536;
    return (int64_t)origin * 65536 + floor_div(num, 2 * (int64_t)out_len) - 32768;
}

/* Bilinear sample of an 8-bit image at Q16.16 (Xq, Yq); taps clamped to the
 * image (replicate edge), Q8 weights, result rounded half up. */
uint8_t orc_bilinear_u8(const uint8_t* img, int H, int W, int64_t Xq, int64_t Yq) {
    int64_t x0 = floor_div(Xq, 65536);
    int64_t y0 = floor_div(Yq, 65536);
    int64_t fx = (Xq - x0 * 65536) / 256; /* 0..255 */
    int64_t fy = (Yq - y0 * 65536) / 256;
    int64_t xa = clamp64(x0, 0, W - 1), xb = clamp64(x0 + 1, 0, W - 1);
    int64_t ya = clamp64(y0, 0, H - 1), yb = clamp64(y0 + 1, 0, H - 1);
    int64_t p00 = img[ya * W + xa], p01 = img[ya * W + xb];
    int64_t p10 = img[yb * W + xa], p11 = img[yb * W + xb];
    int64_t acc = (256 - fx) * (256 - fy) * p00 + fx * (256 - fy) * p01 +
                  (256 - fx) * fy * p10 + fx * fy * p11;
    return (uint8_t)((acc + 32768) / 65536);
}

/* Nearest-neighbour sample of a 16-bit depth image (never interpolated). */
uint16_t orc_nearest_u16(const uint16_t* img, int H, int W, int64_t Xq, int64_t Yq) {
    int64_t ix = clamp64(floor_div(Xq + 32768, 65536), 0, W - 1);
    int64_t iy = clamp64(floor_div(Yq + 32768, 65536), 0, H - 1);
    return img[iy * W + ix];
}

/* One crop.  With `affine` (6 x int32 Q16.16: a00 a01 t0 a10 a11 t1) the
 * source point is Xq = a00*u + a01*v + t0, Yq = a10*u + a11*v + t1 (Eq. 1
 * with basis vectors (a00,a10), (a01,a11) and origin (t0,t1)); otherwise the
 * rect's pixel-centre map above. */
void orc_crop(const uint8_t* grey, const uint16_t* depth, int H, int W,
              const orc_rect* r, const int32_t* affine, int out_h, int out_w,
              uint8_t* out_grey, uint16_t* out_depth) {
    for (int v = 0; v < out_h; ++v) {
        for (int u = 0; u < out_w; ++u) {
            int64_t Xq, Yq;
            if (affine) {
                Xq = (int64_t)affine[0] * u + (int64_t)affine[1] * v + affine[2];
                Yq = (int64_t)affine[3] * u + (int64_t)affine[4] * v + affine[5];
            } else {
                Xq = orc_rect_coord_q16(r->x, r->w, out_w, u);
                Yq = orc_rect_coord_q16(r->y, r->h, out_h, v);
            }
            out_grey[v * out_w + u] = orc_bilinear_u8(grey, H, W, Xq, Yq);
            out_depth[v * out_w + u] = orc_nearest_u16(depth, H, W, Xq, Yq);
        }
    }
}

/* ------------------------------------------------------------------ */
/* S2. Depth mask: the fusion region of interest (Sections 1 and 2.5). */
/* ------------------------------------------------------------------ */

static int cmp_u16(const void* a, const void* b) {
    int x = *(const uint16_t*)a, y = *(const uint16_t*)b;
    return (x > y) - (x < y);
}

/* Lower median of the non-zero depth values: sort them and take index
 * floor((n-1)/2).  Returns -1 when every value is a hole (zero). */
int32_t orc_median_nonzero(const uint16_t* d, int n) {
    uint16_t* buf = (uint16_t*)malloc(sizeof(uint16_t) * (size_t)(n > 0 ? n : 1));
    int m = 0;
    for (int i = 0; i < n; ++i)
        if (d[i] != 0) buf[m++] = d[i];
    int32_t med = -1;
    if (m > 0) {
        qsort(buf, (size_t)m, sizeof(uint16_t), cmp_u16);
        med = buf[(m - 1) / 2];
    }
    free(buf);
    return med;
}

/* valid = (d != 0) and |d - median| < mask_mm (strict). */
void orc_valid_mask(const uint16_t* d, int n, int32_t median, int mask_mm, uint8_t* valid) {
    for (int i = 0; i < n; ++i) {
        int32_t diff = (int32_t)d[i] - median;
        if (diff < 0) diff = -diff;
        valid[i] = (uint8_t)(median >= 0 && d[i] != 0 && diff < mask_mm);
    }
}

/* ------------------------------------------------------------------ */
/* S3. LBP code, Eq. 2 read as sum_{p=0}^{7} s(g_p - g_c) 2^p.         */
/* ------------------------------------------------------------------ */

/* Neighbour p of the 3x3 ring, clockwise from top-left, y pointing down. */
static const int RING_DX[8] = {-1, 0, 1, 1, 1, 0, -1, -1};
static const int RING_DY[8] = {-1, -1, -1, 0, 1, 1, 1, 0};

enum { ORC_LBP_GE = 1, ORC_LBP_NBR_IGNORE_MASK = 2 };

/* Code of centre (i = row, j = column).  Neighbours outside the crop are
 * replaced by the nearest crop pixel (replicate edge).  Bit p is set when the
 * neighbour is depth-valid and brighter than the centre (strict, or >= with
 * ORC_LBP_GE). */
int orc_lbp_code(const uint8_t* g, const uint8_t* valid, int h, int w, int i, int j, int flags) {
    int gc = g[i * w + j];
    int code = 0;
    for (int p = 0; p < 8; ++p) {
        int r = i + RING_DY[p], c = j + RING_DX[p];
        r = r < 0 ? 0 : (r > h - 1 ? h - 1 : r);
        c = c < 0 ? 0 : (c > w - 1 ? w - 1 : c);
        int gp = g[r * w + c];
        int nbr_ok = (flags & ORC_LBP_NBR_IGNORE_MASK) ? 1 : valid[r * w + c];
        int s = (flags & ORC_LBP_GE) ? (gp >= gc) : (gp > gc);
        if (nbr_ok && s) code |= 1 << p;
    }
    return code;
}

/* ------------------------------------------------------------------ */
/* S4. Histograms, Eq. 3, with the 59-bin uniform-pattern map.         */
/* ------------------------------------------------------------------ */

/* Number of 0/1 changes going once around the 8-bit ring. */
static int ring_transitions(int c) {
    int t = 0;
    for (int p = 0; p < 8; ++p) {
        int a = (c >> p) & 1;
        int b = (c >> ((p + 1) % 8)) & 1;
        t += (a != b);
    }
    return t;
}

/* lut[c] = rank of c among the codes with at most two transitions, in
 * ascending code order (0..57); every other code maps to 58. */
void orc_uniform_table(int32_t* lut) {
    int rank = 0;
    for (int c = 0; c < 256; ++c) {
        if (ring_transitions(c) <= 2)
            lut[c] = rank++;
        else
            lut[c] = -1;
    }
    for (int c = 0; c < 256; ++c)
        if (lut[c] < 0) lut[c] = rank; /* rank == 58 here */
}

/* Per-cell histograms of one crop.  feat has (h/cell)*(w/cell)*nbins entries,
 * cell-major row by row, bin fastest.  With nbins == 59 the uniform map is
 * used; with nbins == 256 the raw code (the paper's 0-255 histogram). */
void orc_histograms(const uint8_t* g, const uint8_t* valid, int h, int w, int cell,
                    int nbins, int flags, uint16_t* feat) {
    int32_t lut[256];
    orc_uniform_table(lut);
    int gx = w / cell, gy = h / cell;
    memset(feat, 0, sizeof(uint16_t) * (size_t)gx * gy * nbins);
    for (int i = 0; i < gy * cell; ++i) {
        for (int j = 0; j < gx * cell; ++j) {
            if (!valid[i * w + j]) continue;
            int code = orc_lbp_code(g, valid, h, w, i, j, flags);
            int bin = (nbins == 59) ? lut[code] : code;
            int k = (i / cell) * gx + (j / cell);
            feat[(size_t)k * nbins + bin] += 1;
        }
    }
}

/* Steps S1..S4 for a batch.  With rects == NULL the frames already are the
 * crops (n_frames == n, H == out_h, W == out_w).  Invalid descriptors (frame
 * out of range, non-positive side) give an all-zero feature row.  medians
 * (nullable) receives the lower median per crop, -1 for an all-hole crop or
 * an invalid descriptor. */
void orc_features_batch(const uint8_t* grey, const uint16_t* depth, int n_frames, int H, int W,
                        const orc_rect* rects, const int32_t* affine, int n, int out_h, int out_w,
                        int cell, int mask_mm, int nbins, int flags, uint16_t* feats,
                        int32_t* medians) {
    size_t npx = (size_t)out_h * out_w;
    size_t dim = (size_t)(out_h / cell) * (out_w / cell) * nbins;
    uint8_t* cg = (uint8_t*)malloc(npx);
    uint16_t* cd = (uint16_t*)malloc(npx * sizeof(uint16_t));
    uint8_t* valid = (uint8_t*)malloc(npx);
    for (int k = 0; k < n; ++k) {
        uint16_t* out = feats + (size_t)k * dim;
        if (rects) {
            const orc_rect* r = &rects[k];
            if (r->frame < 0 || r->frame >= n_frames || r->w <= 0 || r->h <= 0) {
                memset(out, 0, dim * sizeof(uint16_t));
                if (medians) medians[k] = -1;
                continue;
            }
            orc_crop(grey + (size_t)r->frame * H * W, depth + (size_t)r->frame * H * W, H, W, r,
                     affine ? affine + 6 * (size_t)k : NULL, out_h, out_w, cg, cd);
        } else {
            memcpy(cg, grey + (size_t)k * npx, npx);
            memcpy(cd, depth + (size_t)k * npx, npx * sizeof(uint16_t));
        }
        int32_t med = orc_median_nonzero(cd, (int)npx);
        if (medians) medians[k] = med;
        orc_valid_mask(cd, (int)npx, med, mask_mm, valid);
        orc_histograms(cg, valid, out_h, out_w, cell, nbins, flags, out);
    }
    free(cg);
    free(cd);
    free(valid);
}

/* ------------------------------------------------------------------ */
/* S5. Per-cell normalisation and the SVM decision function (2.5).     */
/* ------------------------------------------------------------------ */

/* x_j = H_j / n_valid(cell), 0 for an empty cell.  fp64 form. */
void orc_normalize_f64(const uint16_t* feats, int n, int cells, int nbins, double* x) {
    for (int k = 0; k < n; ++k) {
        for (int c = 0; c < cells; ++c) {
            const uint16_t* h = feats + ((size_t)k * cells + c) * nbins;
            double* o = x + ((size_t)k * cells + c) * nbins;
            long tot = 0;
            for (int b = 0; b < nbins; ++b) tot += h[b];
            for (int b = 0; b < nbins; ++b) o[b] = tot ? (double)h[b] / (double)tot : 0.0;
        }
    }
}

/* The same quotient as one IEEE single-precision division. */
void orc_normalize_f32(const uint16_t* feats, int n, int cells, int nbins, float* x) {
    for (int k = 0; k < n; ++k) {
        for (int c = 0; c < cells; ++c) {
            const uint16_t* h = feats + ((size_t)k * cells + c) * nbins;
            float* o = x + ((size_t)k * cells + c) * nbins;
            long tot = 0;
            for (int b = 0; b < nbins; ++b) tot += h[b];
            for (int b = 0; b < nbins; ++b) {
                volatile float num = (float)h[b], den = (float)tot;
                o[b] = tot ? num / den : 0.0f;
            }
        }
    }
}

/* fp32 -> bfloat16, round to nearest even (finite inputs). */
uint16_t orc_f32_to_bf16(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7FFFu + lsb;
    return (uint16_t)(u >> 16);
}

/* fp32 -> FP8 E4M3 (bias 7, max 448, no infinities), round to nearest even,
 * saturating.  Finite inputs. */
uint8_t orc_f32_to_e4m3(float f) {
    double v = f;
    uint8_t sign = 0;
    if (v < 0) {
        sign = 0x80;
        v = -v;
    }
    if (v >= 448.0) return sign | 0x7E;
    if (v == 0.0) return sign;
    int e;
    frexp(v, &e); /* v = m * 2^e, m in [0.5, 1): exponent of leading bit is e-1 */
    int lead = e - 1;
    if (lead < -6) lead = -6; /* subnormal range: quantum 2^-9 */
    double quantum = ldexp(1.0, lead - 3);
    double q = v / quantum; /* exact: power-of-two division */
    double fl = floor(q);
    double rem = q - fl;
    double m = fl;
    if (rem > 0.5 || (rem == 0.5 && fmod(fl, 2.0) != 0.0)) m = fl + 1.0;
    int mi = (int)m;
    int expf_field;
    if (mi >= 16) { /* carried into the next binade */
        mi = 8;
        lead += 1;
    }
    if (mi < 8) { /* subnormal: exponent field 0 */
        expf_field = 0;
    } else {
        expf_field = lead + 7;
        mi -= 8;
    }
    int code = (expf_field << 3) | mi;
    if (code > 0x7E) code = 0x7E;
    return sign | (uint8_t)code;
}

double orc_e4m3_to_f64(uint8_t b) {
    int s = b >> 7, e = (b >> 3) & 15, m = b & 7;
    double v = (e == 0) ? ldexp((double)m, -9) : ldexp(1.0 + m / 8.0, e - 7);
    return s ? -v : v;
}

/* RBF one-vs-rest decision: S[k][c] = sum_i a[c][i] exp(-gamma |x_k - sv_i|^2) + b[c],
 * with |.|^2 summed term by term in fp64. */
void orc_svm_rbf(const double* x, int n, const double* sv, int n_sv, int dim, const double* a,
                 const double* b, int n_classes, double gamma, double* scores) {
    double* kv = (double*)malloc(sizeof(double) * (size_t)(n_sv > 0 ? n_sv : 1));
    for (int k = 0; k < n; ++k) {
        const double* xk = x + (size_t)k * dim;
        for (int i = 0; i < n_sv; ++i) {
            const double* s = sv + (size_t)i * dim;
            double d2 = 0.0;
            for (int j = 0; j < dim; ++j) {
                double t = xk[j] - s[j];
                d2 += t * t;
            }
            kv[i] = exp(-gamma * d2);
        }
        for (int c = 0; c < n_classes; ++c) {
            double acc = 0.0;
            for (int i = 0; i < n_sv; ++i) acc += a[(size_t)c * n_sv + i] * kv[i];
            scores[(size_t)k * n_classes + c] = acc + b[c];
        }
    }
    free(kv);
}

/* Linear one-vs-rest decision: S[k][c] = w_c . x_k + b[c]. */
void orc_svm_linear(const double* x, int n, int dim, const double* w, const double* b,
                    int n_classes, double* scores) {
    for (int k = 0; k < n; ++k) {
        for (int c = 0; c < n_classes; ++c) {
            double acc = 0.0;
            for (int j = 0; j < dim; ++j) acc += w[(size_t)c * dim + j] * x[(size_t)k * dim + j];
            scores[(size_t)k * n_classes + c] = acc + b[c];
        }
    }
}

/* Label = argmax over classes, lowest index on ties. */
void orc_argmax(const double* scores, int n, int n_classes, int32_t* labels) {
    for (int k = 0; k < n; ++k) {
        int best = 0;
        for (int c = 1; c < n_classes; ++c)
            if (scores[(size_t)k * n_classes + c] > scores[(size_t)k * n_classes + best]) best = c;
        labels[k] = best;
    }
}

/* ------------------------------------------------------------------ */
/* Section 2.3: nearest-centre tracking.                               */
/* ------------------------------------------------------------------ */

/* For each previous face, the index of the current face (same stream id in `frame`) whose
 * rect centre (x + w/2, y + h/2) is nearest in Euclidean distance; -1 if the stream has no
 * current face; ties go to the lowest index.  Distances are compared in fp64 on the
 * half-pixel centres. */
/* One-vs-rest RBF SVM training (Section 2.5 trains the classifier on the face database; here
 * the dual problem is solved by sequential minimal optimisation with the maximal violating pair).
 * For class c, y_t = +1 if labels[t] == c else -1, and with K_st = exp(-gamma |x_s - x_t|^2):
 *   minimise f(alpha) = 1/2 sum_st alpha_s alpha_t y_s y_t K_st - sum_t alpha_t
 *   subject to 0 <= alpha_t <= cost, sum_t y_t alpha_t = 0.
 * G_t = y_t sum_s alpha_s y_s K_st - 1 is the gradient.  Each step takes
 *   i = argmax_{t in I_up} -y_t G_t,   j = argmin_{t in I_low} -y_t G_t
 * (I_up: y = +1 and alpha < cost, or y = -1 and alpha > 0; I_low: y = +1 and alpha > 0, or
 * y = -1 and alpha < cost; the lowest index on ties), stops when the gap m - M <= eps, and
 * otherwise moves alpha_i += y_i lambda, alpha_j -= y_j lambda with
 * lambda = min((m - M) / eta, the box limits), eta = K_ii + K_jj - 2 K_ij (at least 1e-12); then
 * G_t += y_t lambda (K_it - K_jt).  The bias b makes y_t f(x_t) = 1 on the free vectors: the mean
 * of -y_t G_t over 0 < alpha_t < cost, else the midpoint (m + M) / 2 of the last bounds (m alone,
 * M alone, or 0 when a side is empty).  Outputs a_ct = y_t alpha_t and b_c, so that the decision
 * function is f_c(x) = sum_t a_ct K(x_t, x) + b_c, and the steps taken per class. */
void orc_svm_train_rbf(const double* x, int n, int dim, const int32_t* labels, int n_classes, double gamma,
                       double cost, double eps, int max_iter, double* a_out, double* b_out, int32_t* iters) {
    double* K = (double*)malloc(sizeof(double) * (size_t)n * n);
    for (int s = 0; s < n; ++s)
        for (int t = 0; t < n; ++t) {
            double d2 = 0.0;
            for (int k = 0; k < dim; ++k) {
                const double df = x[(size_t)s * dim + k] - x[(size_t)t * dim + k];
                d2 += df * df;
            }
            K[(size_t)s * n + t] = exp(-gamma * d2);
        }
    double* alpha = (double*)malloc(sizeof(double) * (size_t)n);
    double* G = (double*)malloc(sizeof(double) * (size_t)n);
    int* y = (int*)malloc(sizeof(int) * (size_t)n);
    for (int c = 0; c < n_classes; ++c) {
        for (int t = 0; t < n; ++t) {
            y[t] = labels[t] == c ? 1 : -1;
            alpha[t] = 0.0;
            G[t] = -1.0;
        }
        int it = 0;
        double m = 0.0, M = 0.0;
        int have_up = 0, have_low = 0;
        for (;;) {
            int i = -1, j = -1;
            for (int t = 0; t < n; ++t) {
                const double v = -y[t] * G[t];
                const int up = (y[t] > 0 && alpha[t] < cost) || (y[t] < 0 && alpha[t] > 0.0);
                const int low = (y[t] > 0 && alpha[t] > 0.0) || (y[t] < 0 && alpha[t] < cost);
                if (up && (i < 0 || v > m)) {
                    i = t;
                    m = v;
                }
                if (low && (j < 0 || v < M)) {
                    j = t;
                    M = v;
                }
            }
            have_up = i >= 0;
            have_low = j >= 0;
            if (!have_up || !have_low || m - M <= eps || it >= max_iter) break;
            double eta = K[(size_t)i * n + i] + K[(size_t)j * n + j] - 2.0 * K[(size_t)i * n + j];
            if (eta < 1e-12) eta = 1e-12;
            double lam = (m - M) / eta;
            const double lim_i = y[i] > 0 ? cost - alpha[i] : alpha[i];
            const double lim_j = y[j] > 0 ? alpha[j] : cost - alpha[j];
            if (lam > lim_i) lam = lim_i;
            if (lam > lim_j) lam = lim_j;
            alpha[i] += y[i] * lam;
            alpha[j] -= y[j] * lam;
            /* snap the box edges exactly */
            if (alpha[i] < 0.0) alpha[i] = 0.0;
            if (alpha[i] > cost) alpha[i] = cost;
            if (alpha[j] < 0.0) alpha[j] = 0.0;
            if (alpha[j] > cost) alpha[j] = cost;
            if (lam == lim_i) alpha[i] = y[i] > 0 ? cost : 0.0;
            if (lam == lim_j) alpha[j] = y[j] > 0 ? 0.0 : cost;
            for (int t = 0; t < n; ++t) G[t] += y[t] * lam * (K[(size_t)i * n + t] - K[(size_t)j * n + t]);
            ++it;
        }
        double sum = 0.0;
        int nfree = 0;
        for (int t = 0; t < n; ++t)
            if (alpha[t] > 0.0 && alpha[t] < cost) {
                sum += -y[t] * G[t];
                ++nfree;
            }
        double b;
        if (nfree > 0)
            b = sum / nfree;
        else if (have_up && have_low)
            b = 0.5 * (m + M);
        else if (have_up)
            b = m;
        else if (have_low)
            b = M;
        else
            b = 0.0;
        for (int t = 0; t < n; ++t) a_out[(size_t)c * n + t] = y[t] * alpha[t];
        b_out[c] = b;
        iters[c] = it;
    }
    free(K);
    free(alpha);
    free(G);
    free(y);
}

/* Depth-to-colour mapping of the face region (Section 2.1): a depth pixel (column j, row i)
 * holding d mm, d_min <= d <= d_max, lands on colour point
 *   X = a0 j + a1 i + a2 + 256 (parallax / d),   Y = a3 j + a4 i + a5      (Q16.16, integers)
 * and the face's depth region is the bounding rect of the depth pixels landing inside the colour
 * image and inside the detected colour rect. */
typedef struct {
    int32_t a[6];
    int32_t parallax, d_min, d_max, colour_w, colour_h;
} orc_calib;

static int64_t floor_div_q16(int64_t v) { return v >= 0 ? v / 65536 : -((-v + 65535) / 65536); }

void orc_face_roi(const uint16_t* depth, int n_frames, int H, int W, const orc_calib* c, const orc_rect* rects,
                  int n, orc_rect* out) {
    for (int k = 0; k < n; ++k) {
        const orc_rect r = rects[k];
        out[k].frame = r.frame;
        out[k].x = out[k].y = out[k].w = out[k].h = 0;
        if (r.frame < 0 || r.frame >= n_frames || r.w <= 0 || r.h <= 0) continue;
        int xmin = W, ymin = H, xmax = -1, ymax = -1;
        for (int i = 0; i < H; ++i) {
            for (int j = 0; j < W; ++j) {
                const int d = depth[((size_t)r.frame * H + i) * W + j];
                if (d < c->d_min || d > c->d_max) continue;
                const int64_t X = (int64_t)c->a[0] * j + (int64_t)c->a[1] * i + c->a[2] +
                                  (int64_t)(c->parallax / d) * 256;
                const int64_t Y = (int64_t)c->a[3] * j + (int64_t)c->a[4] * i + c->a[5];
                const int64_t x = floor_div_q16(X), y = floor_div_q16(Y);
                if (x < 0 || x >= c->colour_w || y < 0 || y >= c->colour_h) continue;
                if (x < r.x || x >= (int64_t)r.x + r.w || y < r.y || y >= (int64_t)r.y + r.h) continue;
                if (j < xmin) xmin = j;
                if (j > xmax) xmax = j;
                if (i < ymin) ymin = i;
                if (i > ymax) ymax = i;
            }
        }
        if (xmax >= 0) {
            out[k].x = xmin;
            out[k].y = ymin;
            out[k].w = xmax - xmin + 1;
            out[k].h = ymax - ymin + 1;
        }
    }
}

void orc_track_nearest(const orc_rect* prev, int n_prev, const orc_rect* cur, int n_cur, int32_t* match) {
    for (int i = 0; i < n_prev; ++i) {
        double px = prev[i].x + prev[i].w / 2.0, py = prev[i].y + prev[i].h / 2.0;
        int best = -1;
        double bd = 0.0;
        for (int j = 0; j < n_cur; ++j) {
            if (cur[j].frame != prev[i].frame) continue;
            double cx = cur[j].x + cur[j].w / 2.0, cy = cur[j].y + cur[j].h / 2.0;
            double d = sqrt((cx - px) * (cx - px) + (cy - py) * (cy - py));
            if (best < 0 || d < bd) {
                best = j;
                bd = d;
            }
        }
        match[i] = best;
    }
}

/* Per-stream tracking over a batch of frames (Section 2.3: each face of the previous frame of
 * a stream is followed to the nearest face centre of the next frame, and the stream's data set
 * is updated at every frame).  For each frame f in batch order, with s = frame_stream[f]:
 *   1. every previous face j of s (state) is matched to its nearest current face of f
 *      (orc_track_nearest's rule: Euclidean distance of centres, lowest index on ties);
 *   2. a current face matched by some previous faces takes the identity of the nearest of
 *      them (lowest j on ties); every other current face takes its own classifier label;
 *   3. the state of s becomes f's first min(faces, max_faces) faces and their identities.
 * state_rects [n_streams][max_faces], state_ids [n_streams][max_faces], state_count
 * [n_streams] are updated in place; ids [n] receives each face's identity.  A frame whose
 * stream id is out of range leaves every state untouched and its faces keep their labels. */
void orc_track_streams(orc_rect* state_rects, int32_t* state_ids, int32_t* state_count, int n_streams,
                       int max_faces, int n_frames, const int32_t* frame_stream, const int32_t* frame_start,
                       const orc_rect* rects, const int32_t* labels, int32_t* ids) {
    for (int f = 0; f < n_frames; ++f) {
        const int s = frame_stream[f];
        const int k0 = frame_start[f], nf = frame_start[f + 1] - frame_start[f];
        for (int k = 0; k < nf; ++k) ids[k0 + k] = labels[k0 + k];
        if (s < 0 || s >= n_streams) continue;
        orc_rect* prev = state_rects + (size_t)s * max_faces;
        int32_t* prev_id = state_ids + (size_t)s * max_faces;
        const int np = state_count[s];
        /* step 1 on copies whose stream field is the same, so orc_track_nearest compares them */
        orc_rect* p = (orc_rect*)malloc(sizeof(orc_rect) * (size_t)(np > 0 ? np : 1));
        orc_rect* c = (orc_rect*)malloc(sizeof(orc_rect) * (size_t)(nf > 0 ? nf : 1));
        int32_t* m = (int32_t*)malloc(sizeof(int32_t) * (size_t)(np > 0 ? np : 1));
        for (int j = 0; j < np; ++j) {
            p[j] = prev[j];
            p[j].frame = 0;
        }
        for (int k = 0; k < nf; ++k) {
            c[k] = rects[k0 + k];
            c[k].frame = 0;
        }
        orc_track_nearest(p, np, c, nf, m);
        /* step 2: the nearest of the previous faces that chose current face k */
        for (int k = 0; k < nf; ++k) {
            int best = -1;
            double bd = 0.0;
            const double cx = c[k].x + c[k].w / 2.0, cy = c[k].y + c[k].h / 2.0;
            for (int j = 0; j < np; ++j) {
                if (m[j] != k) continue;
                const double px = p[j].x + p[j].w / 2.0, py = p[j].y + p[j].h / 2.0;
                const double d = sqrt((cx - px) * (cx - px) + (cy - py) * (cy - py));
                if (best < 0 || d < bd) {
                    best = j;
                    bd = d;
                }
            }
            if (best >= 0) ids[k0 + k] = prev_id[best];
        }
        /* step 3 */
        const int keep = nf < max_faces ? nf : max_faces;
        for (int k = 0; k < keep; ++k) {
            prev[k] = rects[k0 + k];
            prev_id[k] = ids[k0 + k];
        }
        state_count[s] = keep;
        free(p);
        free(c);
        free(m);
    }
}
