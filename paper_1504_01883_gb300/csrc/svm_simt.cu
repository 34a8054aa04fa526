// svm_simt.cu -- A6/A7 with exact fp32 SIMT arithmetic (Section 2.5: the SVM decision function):
//   linear   S_c = w_c . x + b_c
//   RBF      S_c = sum_i a_ci exp(-gamma d_i^2) + b_c,  d_i^2 = |x|^2 + |sv_i|^2 - 2 x.sv_i
// For RBF the kernel value is split as exp(-gamma d^2) = 1 + E with E = expm1(-gamma d^2),
// so S_c = asum_c + sum_i a_ci E_i + b_c.  With gamma = 1/dim on per-cell normalised
// histograms gamma*d^2 is ~2e-4, and E keeps the information that 1 + E would round away.
//
// Two fp32 kernels produce per-split partial sums D_s[k][c] = sum_{i in split s} a_ci E_ki:
//   rbf_smallm_kernel  n <= 8 rows: one warp per support vector, all rows at once (the
//                      one-frame workload, bound by reading the SV matrix once);
//   rbf_tiled_kernel   128 x 128 register-tiled SGEMM over (rows, SVs), E in the epilogue,
//                      then E x a^T accumulated per split.
// reduce_scores_kernel adds the splits, asum and the bias, and takes the argmax
// (reduce_scores_hoisted_kernel: the same with the row-independent sums shared by a block).
#include <algorithm>

#include "internal.h"

namespace rgbd {
namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;

// ---------------------------------------------------------------------------------------
// Linear SVM: one CTA (4 warps) per row, one warp per class.
// ---------------------------------------------------------------------------------------
__global__ void linear_kernel(const float* __restrict__ x, int n, int k_pad, const float* __restrict__ w,
                              const float* __restrict__ bias, int C, float* __restrict__ scores,
                              int32_t* __restrict__ labels) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int row = blockIdx.x; row < n; row += gridDim.x) {
        const float4* xr = reinterpret_cast<const float4*>(x + (size_t)row * k_pad);
        for (int c = warp; c < C; c += nw) {
            const float4* wr = reinterpret_cast<const float4*>(w + (size_t)c * k_pad);
            float acc = 0.f;
            for (int j = lane; j < k_pad / 4; j += 32) {
                const float4 a = __ldg(xr + j), b = __ldg(wr + j);
                acc = fmaf(a.x, b.x, acc);
                acc = fmaf(a.y, b.y, acc);
                acc = fmaf(a.z, b.z, acc);
                acc = fmaf(a.w, b.w, acc);
            }
            for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(FULL, acc, off);
            if (lane == 0) scores[(size_t)row * C + c] = acc + bias[c];
        }
        __syncthreads();
        if (labels && threadIdx.x == 0) {
            int best = 0;
            float bv = scores[(size_t)row * C];
            for (int c = 1; c < C; ++c) {
                const float v = scores[(size_t)row * C + c];
                if (v > bv) {
                    bv = v;
                    best = c;
                }
            }
            labels[row] = best;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------
// RBF, n <= 8 rows: warp-per-SV.  Each warp owns a contiguous SV range and keeps the partial
// class sums of all rows in registers (lane holds classes lane, lane+32, ...).
// ---------------------------------------------------------------------------------------
template <int MB, int CW>
__global__ void __launch_bounds__(256) rbf_smallm_kernel(const float* __restrict__ x, const float* __restrict__ xsq,
                                                         int n, int k_pad, const float* __restrict__ sv,
                                                         const float* __restrict__ svsq, int n_sv,
                                                         const float* __restrict__ coef, int n_pad, int C,
                                                         float gamma, int sv_per_warp,
                                                         float* __restrict__ part) {
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int i0 = gw * sv_per_warp, i1 = min(n_sv, i0 + sv_per_warp);
    float acc[MB][CW];
#pragma unroll
    for (int m = 0; m < MB; ++m)
#pragma unroll
        for (int cc = 0; cc < CW; ++cc) acc[m][cc] = 0.f;
    float xs[MB];
#pragma unroll
    for (int m = 0; m < MB; ++m) xs[m] = (m < n) ? xsq[m] : 0.f;

    for (int i = i0; i < i1; ++i) {
        const float4* s4 = reinterpret_cast<const float4*>(sv + (size_t)i * k_pad);
        float dot[MB];
#pragma unroll
        for (int m = 0; m < MB; ++m) dot[m] = 0.f;
        for (int j = lane; j < k_pad / 4; j += 32) {
            const float4 b = __ldg(s4 + j);
#pragma unroll
            for (int m = 0; m < MB; ++m) {
                if (m < n) {
                    const float4 a = __ldg(reinterpret_cast<const float4*>(x + (size_t)m * k_pad) + j);
                    dot[m] = fmaf(a.x, b.x, dot[m]);
                    dot[m] = fmaf(a.y, b.y, dot[m]);
                    dot[m] = fmaf(a.z, b.z, dot[m]);
                    dot[m] = fmaf(a.w, b.w, dot[m]);
                }
            }
        }
#pragma unroll
        for (int m = 0; m < MB; ++m)
            for (int off = 16; off > 0; off >>= 1) dot[m] += __shfl_xor_sync(FULL, dot[m], off);
        const float ss = svsq[i];
#pragma unroll
        for (int m = 0; m < MB; ++m) {
            const float d2 = fmaxf(xs[m] + ss - 2.f * dot[m], 0.f);
            const float e = expm1f(-gamma * d2);
#pragma unroll
            for (int cc = 0; cc < CW; ++cc) {
                const int c = lane + 32 * cc;
                if (c < C) acc[m][cc] = fmaf(coef[(size_t)c * n_pad + i], e, acc[m][cc]);
            }
        }
    }
    // part[gw][m][c]
#pragma unroll
    for (int m = 0; m < MB; ++m) {
        if (m >= n) break;
#pragma unroll
        for (int cc = 0; cc < CW; ++cc) {
            const int c = lane + 32 * cc;
            if (c < C) part[((size_t)gw * n + m) * C + c] = acc[m][cc];
        }
    }
}

// ---------------------------------------------------------------------------------------
// RBF, general n: 128 x 128 x 8 register-tiled fp32 GEMM of X . SV^T per (row tile, SV tile);
// each CTA walks the SV tiles of its split and accumulates E . a^T into part[split][row][c].
// ---------------------------------------------------------------------------------------
constexpr int TBM = 128, TBN = 128, TBK = 8;

struct TiledSmem {
    float As[2][TBK][TBM];
    float Bs[2][TBK][TBN];
    float Es[TBM][TBN + 4];
    float Cs[TBN][128];  // coefficients of the SV tile, [i][c], C <= 128
};

__global__ void __launch_bounds__(256, 1) rbf_tiled_kernel(const float* __restrict__ x, const float* __restrict__ xsq,
                                                           int n, int k_pad, const float* __restrict__ sv,
                                                           const float* __restrict__ svsq, int n_pad,
                                                           const float* __restrict__ coef, int C, float gamma,
                                                           int tiles_per_split, float* __restrict__ part) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TiledSmem& sm = *reinterpret_cast<TiledSmem*>(smem_raw);
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.x * TBM;
    const int split = blockIdx.y;
    const int n_tiles = n_pad / TBN;
    const int t0 = split * tiles_per_split, t1 = min(n_tiles, t0 + tiles_per_split);
    const int lr = tid >> 1, lk = (tid & 1) * 4;  // loader: row, k offset
    const bool arow_ok = (m0 + lr) < n;
    const float* arow = x + (size_t)(arow_ok ? m0 + lr : 0) * k_pad + lk;
    const int nk = k_pad / TBK;

    for (int t = t0; t < t1; ++t) {
        const int n0 = t * TBN;
        const float* brow = sv + (size_t)(n0 + lr) * k_pad + lk;
        float acc[8][8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

        float4 ra = arow_ok ? __ldg(reinterpret_cast<const float4*>(arow)) : make_float4(0, 0, 0, 0);
        float4 rb = __ldg(reinterpret_cast<const float4*>(brow));
        __syncthreads();  // previous tile's epilogue is done with shared memory
        sm.As[0][lk + 0][lr] = ra.x;
        sm.As[0][lk + 1][lr] = ra.y;
        sm.As[0][lk + 2][lr] = ra.z;
        sm.As[0][lk + 3][lr] = ra.w;
        sm.Bs[0][lk + 0][lr] = rb.x;
        sm.Bs[0][lk + 1][lr] = rb.y;
        sm.Bs[0][lk + 2][lr] = rb.z;
        sm.Bs[0][lk + 3][lr] = rb.w;
        __syncthreads();
        for (int kt = 0; kt < nk; ++kt) {
            const int cur = kt & 1;
            if (kt + 1 < nk) {
                ra = arow_ok ? __ldg(reinterpret_cast<const float4*>(arow + (size_t)(kt + 1) * TBK))
                             : make_float4(0, 0, 0, 0);
                rb = __ldg(reinterpret_cast<const float4*>(brow + (size_t)(kt + 1) * TBK));
            }
#pragma unroll
            for (int k = 0; k < TBK; ++k) {
                const float4 a0 = *reinterpret_cast<const float4*>(&sm.As[cur][k][ty * 4]);
                const float4 a1 = *reinterpret_cast<const float4*>(&sm.As[cur][k][64 + ty * 4]);
                const float4 b0 = *reinterpret_cast<const float4*>(&sm.Bs[cur][k][tx * 4]);
                const float4 b1 = *reinterpret_cast<const float4*>(&sm.Bs[cur][k][64 + tx * 4]);
                const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
            }
            if (kt + 1 < nk) {
                const int nx = cur ^ 1;
                sm.As[nx][lk + 0][lr] = ra.x;
                sm.As[nx][lk + 1][lr] = ra.y;
                sm.As[nx][lk + 2][lr] = ra.z;
                sm.As[nx][lk + 3][lr] = ra.w;
                sm.Bs[nx][lk + 0][lr] = rb.x;
                sm.Bs[nx][lk + 1][lr] = rb.y;
                sm.Bs[nx][lk + 2][lr] = rb.z;
                sm.Bs[nx][lk + 3][lr] = rb.w;
            }
            __syncthreads();
        }
        // epilogue 1: E = expm1(-gamma d^2) for the 8 x 8 block of this thread
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int rl = (i < 4) ? ty * 4 + i : 64 + ty * 4 + (i - 4);
            const int rg = m0 + rl;
            const float xs = (rg < n) ? xsq[rg] : 0.f;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int cl = (j < 4) ? tx * 4 + j : 64 + tx * 4 + (j - 4);
                const float d2 = fmaxf(xs + svsq[n0 + cl] - 2.f * acc[i][j], 0.f);
                sm.Es[rl][cl] = expm1f(-gamma * d2);
            }
        }
        for (int idx = tid; idx < TBN * C; idx += 256) {
            const int c = idx / TBN, i = idx - c * TBN;
            sm.Cs[i][c] = coef[(size_t)c * n_pad + n0 + i];
        }
        __syncthreads();
        // epilogue 2: part[split][row][c] (+)= sum_i E[row][i] a[c][i]
        for (int idx = tid; idx < TBM * C; idx += 256) {
            const int rl = idx / C, c = idx - rl * C;
            const int rg = m0 + rl;
            float s = 0.f;
#pragma unroll 8
            for (int i = 0; i < TBN; ++i) s = fmaf(sm.Es[rl][i], sm.Cs[i][c], s);
            if (rg < n) {
                float* p = part + ((size_t)split * n + rg) * C + c;
                *p = (t == t0) ? s : (*p + s);
            }
        }
    }
}

// ---------------------------------------------------------------------------------------
// Final reduction: one warp per row.
//   ref == NULL:  S_c = asum_c + sum_s D_s[c] + b_c
//   ref != NULL:  the partial sums of split s are relative to a reference distance r_s
//                 (D_s = sum_i a_ci expm1(-gamma (d_i^2 - r_s))); with r* = r_0 and
//                 delta_s = expm1(-gamma (r_s - r*)):
//                 S_c = exp(-gamma r*) (asum_c + sum_s [D_s + delta_s (asum_{c,s} + D_s)]) + b_c
// ---------------------------------------------------------------------------------------
__global__ void reduce_scores_kernel(const float* __restrict__ part, const float* __restrict__ ref,
                                     int splits, int n, int C, int C_stride, const float* __restrict__ asum,
                                     const float* __restrict__ asum_tile, int tps, int nt,
                                     const float* __restrict__ bias, float gamma, float* __restrict__ scores,
                                     int32_t* __restrict__ labels) {
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= n) return;
    float best = -INFINITY;
    int bi = 0x7FFFFFFF;
    const float rstar = ref ? ref[row] : 0.f;
    const float escale = ref ? expf(-gamma * rstar) : 1.f;
    for (int c = lane; c < C; c += 32) {
        float acc = 0.f;
        for (int s = 0; s < splits; ++s) {
            const float d = part[((size_t)s * n + row) * C_stride + c];
            if (ref) {
                float as = 0.f;  // sum of a_ci over the SVs of split s
                if (s > 0)
                    for (int t = s * tps; t < min(nt, (s + 1) * tps); ++t) as += asum_tile[(size_t)t * C_stride + c];
                const float delta = (s == 0) ? 0.f : expm1f(-gamma * (ref[(size_t)s * n + row] - rstar));
                acc += d + delta * (as + d);
            } else {
                acc += d;
            }
        }
        const float sc = escale * (asum[c] + acc) + bias[c];
        scores[(size_t)row * C + c] = sc;
        if (sc > best) {
            best = sc;
            bi = c;
        }
    }
    if (labels) {
        for (int off = 16; off > 0; off >>= 1) {
            const float ob = __shfl_xor_sync(FULL, best, off);
            const int oi = __shfl_xor_sync(FULL, bi, off);
            if (ob > best || (ob == best && oi < bi)) {
                best = ob;
                bi = oi;
            }
        }
        if (lane == 0) labels[row] = bi;
    }
}

// The same combination with the row-independent parts hoisted: a block of rows first sums, per
// split and class, the coefficients of the split's tiles (sum_{i in split s} a_ci) and, per row
// and split, delta_s = expm1(-gamma (r_s - r*)), into shared memory; then one warp per row adds
// the splits in the same order and with the same operations as reduce_scores_kernel, so the
// scores are bit-identical to it.  (reduce_scores_kernel repeats the tile sums per row and the
// expm1 per class, as a chain of dependent loads in every warp.)
__global__ void reduce_scores_hoisted_kernel(const float* __restrict__ part, const float* __restrict__ ref,
                                             int splits, int n, int C, int C_stride,
                                             const float* __restrict__ asum, const float* __restrict__ asum_tile,
                                             int tps, int nt, const float* __restrict__ bias, float gamma,
                                             float* __restrict__ scores, int32_t* __restrict__ labels) {
    extern __shared__ float sh[];
    const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* s_as = sh;                              // [splits][C]
    float* s_del = sh + (size_t)splits * C;        // [nw][splits]
    const int row = blockIdx.x * nw + warp;
    if (ref) {
        for (int i = threadIdx.x; i < splits * C; i += blockDim.x) {
            const int sp = i / C, c = i - sp * C;
            float as = 0.f;
            if (sp > 0)
                for (int t = sp * tps; t < min(nt, (sp + 1) * tps); ++t) as += asum_tile[(size_t)t * C_stride + c];
            s_as[i] = as;
        }
    }
    float escale = 1.f;
    if (ref && row < n) {
        const float rstar = ref[row];
        escale = expf(-gamma * rstar);
        for (int sp = lane; sp < splits; sp += 32)
            s_del[warp * splits + sp] = (sp == 0) ? 0.f : expm1f(-gamma * (ref[(size_t)sp * n + row] - rstar));
    }
    __syncthreads();
    if (row >= n) return;
    float best = -INFINITY;
    int bi = 0x7FFFFFFF;
    for (int c = lane; c < C; c += 32) {
        float acc = 0.f;
        for (int s = 0; s < splits; ++s) {
            const float d = part[((size_t)s * n + row) * C_stride + c];
            if (ref)
                acc += d + s_del[warp * splits + s] * (s_as[s * C + c] + d);
            else
                acc += d;
        }
        const float sc = escale * (asum[c] + acc) + bias[c];
        scores[(size_t)row * C + c] = sc;
        if (sc > best) {
            best = sc;
            bi = c;
        }
    }
    if (labels) {
        for (int off = 16; off > 0; off >>= 1) {
            const float ob = __shfl_xor_sync(FULL, best, off);
            const int oi = __shfl_xor_sync(FULL, bi, off);
            if (ob > best || (ob == best && oi < bi)) {
                best = ob;
                bi = oi;
            }
        }
        if (lane == 0) labels[row] = bi;
    }
}

}  // namespace

int launch_reduce_scores(const float* part, const float* ref, int splits, int n, int C, int C_stride,
                         const float* asum, const float* asum_tile, int tiles_per_split, int n_tiles,
                         const float* bias, float gamma, float* scores, int32_t* labels, cudaStream_t s) {
    constexpr int kRowsHoisted = 16;
    const size_t sh = sizeof(float) * ((size_t)splits * C + (size_t)kRowsHoisted * splits);
    if (ref && sh <= 32 * 1024) {
        reduce_scores_hoisted_kernel<<<(n + kRowsHoisted - 1) / kRowsHoisted, 32 * kRowsHoisted, sh, s>>>(
            part, ref, splits, n, C, C_stride, asum, asum_tile, tiles_per_split, n_tiles, bias, gamma, scores,
            labels);
    } else {
        const int rows_per_block = 8;
        reduce_scores_kernel<<<(n + rows_per_block - 1) / rows_per_block, 32 * rows_per_block, 0, s>>>(
            part, ref, splits, n, C, C_stride, asum, asum_tile, tiles_per_split, n_tiles, bias, gamma, scores,
            labels);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "svm_score: reduce launch");
    return RGBD_OK;
}

int score_linear(rgbd_ctx* ctx, const rgbd_svm* m, const float* x, int n, float* scores,
                 int32_t* labels, cudaStream_t s) {
    const int grid = std::min(n, ctx->props.sm_count * 16);
    linear_kernel<<<grid, 128, 0, s>>>(x, n, m->k_pad, m->coef, m->bias, m->C, scores, labels);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "svm_score: linear launch");
    return RGBD_OK;
}

template <int MB, int CW>
static void launch_smallm(int blocks, cudaStream_t s, const float* x, const float* xsq, int n, int k_pad,
                          const rgbd_svm* m, int spw, float* part) {
    rbf_smallm_kernel<MB, CW><<<blocks, 256, 0, s>>>(x, xsq, n, k_pad, (const float*)m->sv, m->sv_sq,
                                                     m->n_sv, m->coef, m->n_pad, m->C, m->gamma, spw, part);
}

// The workspace score_rbf_f32 takes for n rows (the same arithmetic as its two paths).
size_t score_rbf_f32_bytes(rgbd_ctx* ctx, const rgbd_svm* m, int n) {
    if (n <= 8) {
        const int warps_target = ctx->props.sm_count * 8 * 4;
        const int spw = std::max(1, (m->n_sv + warps_target - 1) / warps_target);
        const int nwarps = (m->n_sv + spw - 1) / spw;
        return sizeof(float) * (size_t)((nwarps + 7) / 8 * 8) * n * m->C;
    }
    const int mt = (n + TBM - 1) / TBM;
    const int nt = m->n_pad / TBN;
    int splits = std::max(1, std::min(nt, (ctx->props.sm_count + mt - 1) / mt));
    const int tps = (nt + splits - 1) / splits;
    splits = (nt + tps - 1) / tps;
    return sizeof(float) * (size_t)splits * n * m->C;
}

int score_rbf_f32(rgbd_ctx* ctx, const rgbd_svm* m, const float* x, const float* xsq, int n,
                  float* scores, int32_t* labels, cudaStream_t s) {
    if (m->C > 128) return set_error(RGBD_ERR_UNSUPPORTED, "svm_score: fp32 RBF supports up to 128 classes");
    cudaError_t e;
    if (n <= 8) {
        // one warp per SV range; enough warps to cover every SM a few times
        const int warps_target = ctx->props.sm_count * 8 * 4;
        const int spw = std::max(1, (m->n_sv + warps_target - 1) / warps_target);
        const int nwarps = (m->n_sv + spw - 1) / spw;
        const int blocks = (nwarps + 7) / 8;
        const int total_warps = blocks * 8;
        const size_t need = sizeof(float) * (size_t)total_warps * n * m->C;
        int rc = ensure_workspace(ctx, need, s);
        if (rc) return rc;
        float* part = (float*)ctx->workspace;
        const int cw = (m->C + 31) / 32;
        const int mb = n <= 1 ? 1 : (n <= 2 ? 2 : (n <= 4 ? 4 : 8));
#define SMALLM(MBV, CWV) \
    if (mb == MBV && cw == CWV) launch_smallm<MBV, CWV>(blocks, s, x, xsq, n, m->k_pad, m, spw, part);
        SMALLM(1, 1) SMALLM(1, 2) SMALLM(1, 3) SMALLM(1, 4)
        SMALLM(2, 1) SMALLM(2, 2) SMALLM(2, 3) SMALLM(2, 4)
        SMALLM(4, 1) SMALLM(4, 2) SMALLM(4, 3) SMALLM(4, 4)
        SMALLM(8, 1) SMALLM(8, 2) SMALLM(8, 3) SMALLM(8, 4)
#undef SMALLM
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_error(e, "svm_score: rbf small-n launch");
        // warps past n_sv wrote zeros (empty SV range), so every split is summed
        return launch_reduce_scores(part, nullptr, total_warps, n, m->C, m->C, m->asum, nullptr, 0, 0, m->bias,
                                    m->gamma, scores, labels, s);
    }
    static bool attr_set = false;
    const size_t smem = sizeof(TiledSmem);
    if (!attr_set) {
        e = cudaFuncSetAttribute(rbf_tiled_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_error(e, "svm_score: tiled smem attribute");
        attr_set = true;
    }
    const int mt = (n + TBM - 1) / TBM;
    const int nt = m->n_pad / TBN;
    int splits = std::max(1, std::min(nt, (ctx->props.sm_count + mt - 1) / mt));
    const int tps = (nt + splits - 1) / splits;
    splits = (nt + tps - 1) / tps;
    const size_t need = sizeof(float) * (size_t)splits * n * m->C;
    int rc = ensure_workspace(ctx, need, s);
    if (rc) return rc;
    float* part = (float*)ctx->workspace;
    dim3 grid(mt, splits);
    rbf_tiled_kernel<<<grid, 256, smem, s>>>(x, xsq, n, m->k_pad, (const float*)m->sv, m->sv_sq, m->n_pad,
                                             m->coef, m->C, m->gamma, tps, part);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "svm_score: rbf tiled launch");
    return launch_reduce_scores(part, nullptr, splits, n, m->C, m->C, m->asum, nullptr, 0, 0, m->bias, m->gamma,
                                scores, labels, s);
}

}  // namespace rgbd
