// train.cu -- one-vs-rest RBF SVM training on the GPU (Section 2.5 trains the classifier on the
// face database; the paper does it on the CPU).  The dual problem of every class is solved by
// sequential minimal optimisation with the maximal violating pair, on one kernel matrix that all
// classes share:
//   kernel_matrix_kernel  K_st = exp(-gamma max(0, |x_s|^2 + |x_t|^2 - 2 x_s . x_t)), fp32, a
//                         64 x 64 register-tiled product per CTA;
//   smo_kernel            one CTA per class; alpha and the gradient G stay in shared memory; each
//                         step reduces the two selections over the CTA, updates the pair on one
//                         thread, then G_t += y_t lambda (K_it - K_jt) with all threads.
#include <float.h>
#include <stdint.h>

#include <algorithm>

#include "internal.h"

namespace rgbd {
namespace {

constexpr int KM_TILE = 64, KM_K = 16;
constexpr int SMO_THREADS = 1024;

__global__ void __launch_bounds__(256) kernel_matrix_kernel(const float* __restrict__ x, const float* __restrict__ xsq,
                                                            int n, int k_pad, float gamma, float* __restrict__ K) {
    __shared__ float As[KM_K][KM_TILE + 4];
    __shared__ float Bs[KM_K][KM_TILE + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int s0 = blockIdx.y * KM_TILE, t0 = blockIdx.x * KM_TILE;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < k_pad; k0 += KM_K) {
        // 64 rows x 16 columns of each operand: 256 threads load 4 values each
        for (int e = threadIdx.x; e < KM_TILE * KM_K; e += 256) {
            const int r = e / KM_K, kk = e - r * KM_K;
            const int sr = s0 + r, tr = t0 + r;
            As[kk][r] = (sr < n && k0 + kk < k_pad) ? x[(size_t)sr * k_pad + k0 + kk] : 0.f;
            Bs[kk][r] = (tr < n && k0 + kk < k_pad) ? x[(size_t)tr * k_pad + k0 + kk] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < KM_K; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = As[kk][ty * 4 + u];
                b[u] = Bs[kk][tx * 4 + u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int s = s0 + ty * 4 + u;
        if (s >= n) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int t = t0 + tx * 4 + v;
            if (t >= n) continue;
            const float d2 = fmaxf(xsq[s] + xsq[t] - 2.f * acc[u][v], 0.f);
            K[(size_t)s * n + t] = (s == t) ? 1.f : expf(-gamma * d2);
        }
    }
}

// (value, index) pairs: the larger value wins (or the smaller, for the minimum), then the lower index
__device__ __forceinline__ void arg_better_max(float& v, int& i, float ov, int oi) {
    if (oi >= 0 && (i < 0 || ov > v || (ov == v && oi < i))) {
        v = ov;
        i = oi;
    }
}
__device__ __forceinline__ void arg_better_min(float& v, int& i, float ov, int oi) {
    if (oi >= 0 && (i < 0 || ov < v || (ov == v && oi < i))) {
        v = ov;
        i = oi;
    }
}

__global__ void __launch_bounds__(SMO_THREADS, 1) smo_kernel(const float* __restrict__ K, int n,
                                                            const int32_t* __restrict__ labels, float cost, float eps,
                                                            int max_iter, float* __restrict__ coef,
                                                            float* __restrict__ bias, int32_t* __restrict__ iters) {
    extern __shared__ float smo_smem[];
    float* alpha = smo_smem;
    float* G = smo_smem + n;
    int8_t* y = reinterpret_cast<int8_t*>(smo_smem + 2 * n);
    __shared__ float rv[2][32];
    __shared__ int ri[2][32];
    __shared__ int sel_i, sel_j, stop;
    __shared__ float sel_lam, sel_m, sel_M;
    const int c = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int t = tid; t < n; t += SMO_THREADS) {
        y[t] = labels[t] == c ? 1 : -1;
        alpha[t] = 0.f;
        G[t] = -1.f;
    }
    __syncthreads();
    int it = 0;
    for (;;) {
        // selection: i = argmax over I_up of -y G, j = argmin over I_low of -y G
        float mu = 0.f, ml = 0.f;
        int iu = -1, il = -1;
        for (int t = tid; t < n; t += SMO_THREADS) {
            const float v = -(float)y[t] * G[t];
            const bool up = (y[t] > 0 && alpha[t] < cost) || (y[t] < 0 && alpha[t] > 0.f);
            const bool low = (y[t] > 0 && alpha[t] > 0.f) || (y[t] < 0 && alpha[t] < cost);
            if (up) arg_better_max(mu, iu, v, t);
            if (low) arg_better_min(ml, il, v, t);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            arg_better_max(mu, iu, __shfl_xor_sync(0xFFFFFFFFu, mu, off), __shfl_xor_sync(0xFFFFFFFFu, iu, off));
            arg_better_min(ml, il, __shfl_xor_sync(0xFFFFFFFFu, ml, off), __shfl_xor_sync(0xFFFFFFFFu, il, off));
        }
        if (lane == 0) {
            rv[0][warp] = mu, ri[0][warp] = iu;
            rv[1][warp] = ml, ri[1][warp] = il;
        }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < SMO_THREADS / 32; ++w) {
                arg_better_max(mu, iu, rv[0][w], ri[0][w]);
                arg_better_min(ml, il, rv[1][w], ri[1][w]);
            }
            sel_m = mu, sel_M = ml;
            sel_i = iu, sel_j = il;
            int st = iu < 0 || il < 0 || mu - ml <= eps || it >= max_iter;
            if (!st) {
                const float kii = K[(size_t)iu * n + iu], kjj = K[(size_t)il * n + il], kij = K[(size_t)iu * n + il];
                float eta = kii + kjj - 2.f * kij;
                if (eta < 1e-12f) eta = 1e-12f;
                float lam = (mu - ml) / eta;
                const float lim_i = y[iu] > 0 ? cost - alpha[iu] : alpha[iu];
                const float lim_j = y[il] > 0 ? alpha[il] : cost - alpha[il];
                const bool hit_i = lam >= lim_i, hit_j = lam >= lim_j;
                lam = fminf(lam, fminf(lim_i, lim_j));
                float ai = alpha[iu] + (float)y[iu] * lam, aj = alpha[il] - (float)y[il] * lam;
                ai = fminf(fmaxf(ai, 0.f), cost);
                aj = fminf(fmaxf(aj, 0.f), cost);
                if (hit_i && lam == lim_i) ai = y[iu] > 0 ? cost : 0.f;  // snap the box edges exactly
                if (hit_j && lam == lim_j) aj = y[il] > 0 ? 0.f : cost;
                alpha[iu] = ai;
                alpha[il] = aj;
                sel_lam = lam;
            }
            stop = st;
        }
        __syncthreads();
        if (stop) break;
        const float lam = sel_lam;
        const float* Ki = K + (size_t)sel_i * n;
        const float* Kj = K + (size_t)sel_j * n;
        for (int t = tid; t < n; t += SMO_THREADS) G[t] += (float)y[t] * lam * (Ki[t] - Kj[t]);
        ++it;
        __syncthreads();
    }
    // bias: mean of -y G over the free vectors, else the midpoint of the last bounds
    float sum = 0.f;
    int cnt = 0;
    for (int t = tid; t < n; t += SMO_THREADS)
        if (alpha[t] > 0.f && alpha[t] < cost) {
            sum += -(float)y[t] * G[t];
            ++cnt;
        }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        sum += __shfl_xor_sync(0xFFFFFFFFu, sum, off);
        cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, off);
    }
    __syncthreads();
    if (lane == 0) {
        rv[0][warp] = sum;
        ri[0][warp] = cnt;
    }
    __syncthreads();
    if (tid == 0) {
        float s = 0.f;
        int k = 0;
        for (int w = 0; w < SMO_THREADS / 32; ++w) s += rv[0][w], k += ri[0][w];
        float b;
        if (k > 0)
            b = s / (float)k;
        else if (sel_i >= 0 && sel_j >= 0)
            b = 0.5f * (sel_m + sel_M);
        else if (sel_i >= 0)
            b = sel_m;
        else if (sel_j >= 0)
            b = sel_M;
        else
            b = 0.f;
        bias[c] = b;
        iters[c] = it;
    }
    for (int t = tid; t < n; t += SMO_THREADS) coef[(size_t)c * n + t] = (float)y[t] * alpha[t];
}

}  // namespace
}  // namespace rgbd

using namespace rgbd;

extern "C" int svm_train_rbf(rgbd_ctx* ctx, const float* x, const float* xsq, int n, int k_pad, const int32_t* labels,
                             int n_classes, float gamma, float cost, float eps, int max_iter, float* coef, float* bias,
                             int32_t* iters, void* stream) {
    rgbd::NvtxRange nvtx_range("svm_train_rbf");
    if (!ctx) return set_error(RGBD_ERR_ARG, "svm_train_rbf: ctx is NULL");
    if (n < 2 || n > 16384 || k_pad <= 0 || n_classes < 1 || !(gamma > 0.f) || !(cost > 0.f) || !(eps > 0.f) ||
        max_iter < 0 || max_iter > 2000000)
        return set_error(RGBD_ERR_ARG,
                         "svm_train_rbf: n %d (2..16384), k_pad %d, classes %d, gamma %g, cost %g, eps %g, max_iter %d (0..2e6)",
                         n, k_pad, n_classes, gamma, cost, eps, max_iter);
    if (!x || !xsq || !labels || !coef || !bias || !iters) return set_error(RGBD_ERR_ARG, "svm_train_rbf: NULL pointer");
    DeviceGuard g(ctx->props.device);
    cudaStream_t s = (cudaStream_t)stream;
    int rc = ensure_workspace(ctx, sizeof(float) * (size_t)n * n, s);
    if (rc) return rc;
    float* K = (float*)ctx->workspace;
    dim3 grid((n + KM_TILE - 1) / KM_TILE, (n + KM_TILE - 1) / KM_TILE);
    kernel_matrix_kernel<<<grid, 256, 0, s>>>(x, xsq, n, k_pad, gamma, K);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "svm_train_rbf: kernel matrix launch");
    const size_t smem = sizeof(float) * 2 * (size_t)n + (size_t)n;
    e = cudaFuncSetAttribute(smo_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_error(e, "svm_train_rbf: smem attribute");
    smo_kernel<<<n_classes, SMO_THREADS, smem, s>>>(K, n, labels, cost, eps, max_iter, coef, bias, iters);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "svm_train_rbf: SMO launch");
    return RGBD_OK;
}
