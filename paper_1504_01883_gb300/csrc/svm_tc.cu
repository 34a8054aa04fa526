// svm_tc.cu -- A6/A7 on the 5th-generation tensor cores (tcgen05, sm_103a): the RBF SVM decision
// function of Section 2.5, S_c = sum_i a_ci exp(-gamma |x - sv_i|^2) + b_c, for BF16, FP8 E4M3
// (per-tensor scales) and TF32 operands with fp32 accumulation in tensor memory.
//
// One CTA (11 warps) owns 128 feature rows and a contiguous range ("split") of 256-wide SV tiles:
//   warp 0      TMA producer of the main ring: per k-block (128 B of K per row, 128B-swizzled)
//               the 128-row X block and the 256-row SV block, 3 stages of 48 KB.
//   warp 1      TMEM owner and MMA issuer (one thread):
//                 G (128 x 256 fp32, TMEM)  = X . SV_t^T over all k-blocks   (N = 256 MMAs)
//                 D (128 x C_pad fp32, TMEM) += F_q . a_q^T  for every 64-column chunk q of F
//   warp 2      TMA producer of the bf16 coefficient chunks a[c][64 SVs] (2-slot ring).
//   warps 3-10  epilogue, two sets of four warps (one per TMEM lane quarter); set k handles the
//               64-column chunks k and k + 2 of every tile.  One thread per row reads G with
//               tcgen05.ld, forms d^2 = |x|^2 + |sv|^2 - 2 G and F = expm1(-gamma (d^2 - r)) in
//               bf16, and writes F into its slot of a 2-slot ring in the UMMA K-major 128B-swizzle
//               layout, which the second MMA reads.  r is the row's mean d^2 over chunks 0
//               and 2 of the split's first tile; since exp(-gamma d^2) = exp(-gamma r) (1 + F),
//                 S_c = sum_splits exp(-gamma r_s) (sum_{i in s} a_ci + D_s[c]) + b_c,
//               and F keeps the small per-SV variation at full relative precision (gamma d^2 is
//               ~2e-4 for gamma = 1/dim, so exp() itself is flat to 1e-4).
// The MMA thread services finished F chunks between main-loop k-blocks, so the second MMA and
// the epilogue overlap the next tile's main loop.  Partial sums D_s and r_s go to workspace;
// launch_reduce_scores combines the splits.
//
// Every wait on an mbarrier is bounded by a %globaltimer deadline; on expiry the CTA sets
// RGBD_STATUS_WAIT_TIMEOUT, stops issuing work, waits (bounded) for its own copies and MMAs
// in flight, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>

#include "internal.h"

namespace rgbd {
namespace {

constexpr int BM = 128;
constexpr int BN = 256;
constexpr int STAGES = 3;
constexpr int X_TILE = BM * 128;   // bytes of one X k-block
constexpr int SV_TILE = BN * 128;  // bytes of one SV k-block
constexpr int STAGE_BYTES = X_TILE + SV_TILE;
constexpr int F_CHUNK = BM * 64 * 2;               // one 64-column bf16 chunk of F (16 KB)
constexpr int F_OFF = STAGES * STAGE_BYTES;        // 2 slots
constexpr int MAX_CPAD = 128;
constexpr int COEF_CHUNK_MAX = MAX_CPAD * 64 * 2;  // one 64-SV chunk of a (C_pad rows)
constexpr int COEF_OFF = F_OFF + 2 * F_CHUNK;      // 2 slots
constexpr int BAR_OFF = COEF_OFF + 2 * COEF_CHUNK_MAX;
constexpr int SMEM_BYTES = BAR_OFF + 256 + 1024;   // + barriers + alignment slack
constexpr int NUM_WARPS = 11;
constexpr int NUM_THREADS = NUM_WARPS * 32;
constexpr uint32_t TMEM_COLS = 512;                // G: 256 columns, D: C_pad columns at 256
constexpr uint64_t WAIT_NS = 1000000000ull;        // 1 s: far above any legitimate wait

// barrier slots (8 bytes each) inside the barrier block
enum {
    B_FULL = 0,                   // STAGES
    B_EMPTY = B_FULL + STAGES,    // STAGES
    B_GFULL = B_EMPTY + STAGES,
    B_GEMPTY = B_GFULL + 1,
    B_FFULL = B_GEMPTY + 1,       // 2 (F chunk written + its coefficient chunk loaded)
    B_FEMPTY = B_FFULL + 2,       // 2 (second MMA of the chunk done)
    B_DFULL = B_FEMPTY + 2,
    B_DRAIN = B_DFULL + 1,
    B_COUNT = B_DRAIN + 1
};

struct TcParams {
    int n;            // feature rows
    int n_sv;         // real support vectors
    int C, C_pad;
    int k_blocks;     // k_pad * elem_size / 128
    int k_elems;      // elements per k-block
    int tiles_per_split;
    int n_tiles;
    float gamma;
    float gscale;     // 1 / (x_scale * sv_scale) for FP8, else 1
    const float* xsq;
    const float* svsq;
    float* part;      // [splits][n][C_pad]
    float* ref;       // [splits][n]
    uint32_t* status;
    uint32_t idesc_main;
    uint32_t idesc_second;
    int kind;         // 0 = f16 (bf16), 1 = f8f6f4 (e4m3), 2 = tf32
};

// ---------------------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void bar_init(uint32_t a, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint32_t a) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(a) : "memory");
}
__device__ __forceinline__ void bar_arrive_tx(uint32_t a, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(a),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool bar_try(uint32_t a, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait.  Returns false when the CTA is aborting (deadline passed here or elsewhere).
__device__ __noinline__ bool bar_wait(uint32_t a, uint32_t parity, volatile int* abort_flag, uint32_t* status) {
    const uint64_t t0 = globaltimer();
    while (!bar_try(a, parity)) {
        if (*abort_flag) return false;
        if (globaltimer() - t0 > WAIT_NS) {
            *abort_flag = 1;
            atomicOr(status, RGBD_STATUS_WAIT_TIMEOUT);
            return false;
        }
    }
    return true;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
// TMA load multicast to the CTAs of `mask` in the cluster: same CTA-relative destination offset
// and mbarrier in each of them.
__device__ __forceinline__ void tma_load_2d_mc(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar,
                                               uint16_t mask) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.multicast::cluster"
        " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar), "h"(mask)
        : "memory");
}
__device__ __forceinline__ void tc_commit_mc(uint32_t bar, uint16_t mask) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(bar),
        "h"(mask)
        : "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// UMMA shared-memory descriptor: K-major operand, 128-byte swizzle, 8-row atoms 1024 B apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(16u >> 4) << 16;    // leading byte offset (unused with 128B swizzle, K-major)
    d |= (uint64_t)(1024u >> 4) << 32;  // stride byte offset: next group of 8 rows
    d |= (uint64_t)1 << 46;             // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;             // 128-byte swizzle
    return d;
}
__device__ __forceinline__ void mma_issue(int kind, uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if (kind == 0) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    } else if (kind == 1) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    }
}
#define TC_LD_X32(taddr, v)                                                                                   \
    asm volatile(                                                                                             \
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"     \
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"                          \
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),     \
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),           \
          "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),         \
          "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),         \
          "=r"(v[29]), "=r"(v[30]), "=r"(v[31])                                                              \
        : "r"(taddr))
#define TC_LD_X16(taddr, v)                                                                                   \
    asm volatile(                                                                                             \
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "   \
        "[%16];"                                                                                              \
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),     \
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),           \
          "=r"(v[15])                                                                                        \
        : "r"(taddr))
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }


// ---------------------------------------------------------------------------------------
// The kernel
// ---------------------------------------------------------------------------------------
// MC: the CTA runs in a cluster of two along the rows.  Both CTAs use the same SV tiles, so each
// loads half of every SV k-block and multicasts it into both CTAs' stage, and each CTA's MMA
// releases the stage in both CTAs: the pair reads each SV k-block from L2 once.
template <bool MC>
__global__ void __launch_bounds__(NUM_THREADS, 1)
    rbf_tc_kernel(const __grid_constant__ CUtensorMap tm_x, const __grid_constant__ CUtensorMap tm_sv,
                  const __grid_constant__ CUtensorMap tm_coef, const TcParams p) {
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;  // 1024-byte aligned for the 128B swizzle atoms
    unsigned char* gbase = smem_raw + (base - raw);
    const uint32_t bars = base + BAR_OFF;
    auto bar = [&](int i) { return bars + 8u * (uint32_t)i; };
    volatile int* abort_flag = reinterpret_cast<volatile int*>(gbase + BAR_OFF + 8 * B_COUNT);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbase + BAR_OFF + 8 * B_COUNT + 8);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * BM;
    const int split = blockIdx.y;
    const int t0 = split * p.tiles_per_split;
    const int t1 = min(p.n_tiles, t0 + p.tiles_per_split);
    const int U = t1 - t0;   // tiles of this split (>= 1)
    const int Q = 4 * U;     // 64-column chunks of this split

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            bar_init(bar(B_FULL + s), 1);
            bar_init(bar(B_EMPTY + s), MC ? 2 : 1);  // both CTAs' MMAs read a multicast stage
        }
        bar_init(bar(B_GFULL), 1);
        bar_init(bar(B_GEMPTY), 8);
        for (int s = 0; s < 2; ++s) {
            bar_init(bar(B_FFULL + s), 4 + 1);  // 4 epilogue warps + the coefficient producer
            bar_init(bar(B_FEMPTY + s), 1);
        }
        bar_init(bar(B_DFULL), 1);
        bar_init(bar(B_DRAIN), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncwarp();
    if (MC)
        cluster_sync();  // the peer's barriers are initialised before any multicast reaches them
    else
        __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t crank = MC ? cluster_rank() : 0u;
    const uint32_t coef_chunk_bytes = (uint32_t)p.C_pad * 128u;

    if (warp == 0) {
        // ===================== TMA producer: X and SV k-blocks =====================
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tm_x) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tm_sv) : "memory");
            int stage = 0;
            uint32_t phase = 0, armed = 0, armed_par = 0;
            bool alive = true;
            for (int u = 0; u < U && alive; ++u) {
                const int n0 = (t0 + u) * BN;
                for (int kb = 0; kb < p.k_blocks; ++kb) {
                    if (!bar_wait(bar(B_EMPTY + stage), phase ^ 1u, abort_flag, p.status)) {
                        alive = false;
                        break;
                    }
                    const uint32_t sa = base + (uint32_t)stage * STAGE_BYTES;
                    bar_arrive_tx(bar(B_FULL + stage), STAGE_BYTES);
                    tma_load_2d(sa, &tm_x, kb * p.k_elems, m0, bar(B_FULL + stage));
                    if (MC)
                        tma_load_2d_mc(sa + X_TILE + crank * (SV_TILE / 2), &tm_sv, kb * p.k_elems,
                                       n0 + (int)crank * (BN / 2), bar(B_FULL + stage), (uint16_t)0x3);
                    else
                        tma_load_2d(sa + X_TILE, &tm_sv, kb * p.k_elems, n0, bar(B_FULL + stage));
                    armed |= 1u << stage;
                    armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!alive) {  // drain: wait (bounded) for the copies this thread issued
                const uint64_t tq = globaltimer();
                for (int s = 0; s < STAGES; ++s)
                    if (armed & (1u << s))
                        while (!bar_try(bar(B_FULL + s), (armed_par >> s) & 1u) && globaltimer() - tq < WAIT_NS) {
                        }
            }
        }
    } else if (warp == 2) {
        // ===================== TMA producer: coefficient chunks =====================
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tm_coef) : "memory");
            uint32_t armed = 0, armed_par = 0;
            bool alive = true;
            for (int q = 0; q < Q && alive; ++q) {
                const int slot = q & 1;
                if (q >= 2 && !bar_wait(bar(B_FEMPTY + slot), (uint32_t)(((q - 2) >> 1) & 1), abort_flag, p.status)) {
                    alive = false;
                    break;
                }
                const int n0 = (t0 + (q >> 2)) * BN + (q & 3) * 64;
                bar_arrive_tx(bar(B_FFULL + slot), coef_chunk_bytes);
                tma_load_2d(base + COEF_OFF + slot * COEF_CHUNK_MAX, &tm_coef, n0, 0, bar(B_FFULL + slot));
                armed |= 1u << slot;
                armed_par = (armed_par & ~(1u << slot)) | ((uint32_t)((q >> 1) & 1) << slot);
            }
            if (!alive && armed) {
                // the barrier cannot show these copies complete (the epilogue's arrivals are
                // missing once aborting), so give the copies in flight a bounded 200 us to land
                (void)armed_par;
                const uint64_t tq = globaltimer();
                while (globaltimer() - tq < 200000ull) {
                }
            }
        }
    } else if (warp == 1) {
        // ===================== MMA issuer =====================
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            bool alive = true;
            int q_next = 0, q_avail = 0;
            const uint32_t d_tmem = tmem + 256;  // second-MMA accumulator, C_pad columns
            // Issues the second MMA of the next finished F chunk; returns false if none is ready.
            auto service = [&]() -> bool {
                if (q_next >= q_avail) return false;
                const int slot = q_next & 1;
                if (!bar_try(bar(B_FFULL + slot), (uint32_t)((q_next >> 1) & 1))) return false;
                tc_fence_after();
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
                    const uint64_t a = sdesc(base + F_OFF + slot * F_CHUNK + ks * 32);
                    const uint64_t b = sdesc(base + COEF_OFF + slot * COEF_CHUNK_MAX + ks * 32);
                    mma_issue(0, d_tmem, a, b, p.idesc_second, (q_next > 0 || ks > 0) ? 1u : 0u);
                }
                tc_commit(bar(B_FEMPTY + slot));
                ++q_next;
                return true;
            };
            // Blocks (bounded) until barrier (a, parity) completes, servicing chunks meanwhile.
            auto wait_servicing = [&](uint32_t a, uint32_t parity) -> bool {
                const uint64_t tw = globaltimer();
                while (!bar_try(a, parity)) {
                    if (service()) continue;
                    if (*abort_flag) return false;
                    if (globaltimer() - tw > WAIT_NS) {
                        *abort_flag = 1;
                        atomicOr(p.status, RGBD_STATUS_WAIT_TIMEOUT);
                        return false;
                    }
                }
                return true;
            };
            for (int u = 0; u < U && alive; ++u) {
                if (u >= 1) {  // the epilogue has read G of the previous tile
                    if (!wait_servicing(bar(B_GEMPTY), (uint32_t)((u - 1) & 1))) {
                        alive = false;
                        break;
                    }
                    tc_fence_after();
                }
                for (int kb = 0; kb < p.k_blocks; ++kb) {
                    if (!wait_servicing(bar(B_FULL + stage), phase)) {
                        alive = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = base + (uint32_t)stage * STAGE_BYTES;
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint64_t a = sdesc(sa + ks * 32);
                        const uint64_t bd = sdesc(sa + X_TILE + ks * 32);
                        mma_issue(p.kind, tmem, a, bd, p.idesc_main, (kb > 0 || ks > 0) ? 1u : 0u);
                    }
                    if (MC)
                        tc_commit_mc(bar(B_EMPTY + stage), (uint16_t)0x3);
                    else
                        tc_commit(bar(B_EMPTY + stage));
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                    service();
                }
                if (!alive) break;
                tc_commit(bar(B_GFULL));
                q_avail = 4 * (u + 1);
            }
            // the chunks of the last tile
            while (alive && q_next < Q) {
                const uint64_t tw = globaltimer();
                while (!service()) {
                    if (*abort_flag || globaltimer() - tw > WAIT_NS) {
                        if (!*abort_flag) atomicOr(p.status, RGBD_STATUS_WAIT_TIMEOUT);
                        *abort_flag = 1;
                        alive = false;
                        break;
                    }
                }
            }
            if (alive) tc_commit(bar(B_DFULL));
            // drain: every MMA this thread issued has completed once B_DRAIN flips
            tc_commit(bar(B_DRAIN));
            const uint64_t tq = globaltimer();
            while (!bar_try(bar(B_DRAIN), 0)) {
                if (globaltimer() - tq > WAIT_NS) break;
            }
        }
    } else {
        // ===================== epilogue: warps 3..10, one thread per row =====================
        const int ew = warp - 3;           // 0..7
        const int set = ew >> 2;           // chunks set, set + 2 of every tile
        const int quarter = warp & 3;      // TMEM lanes this warp may access
        const int row = quarter * 32 + lane;
        const int grow = m0 + row;
        const bool row_ok = grow < p.n;
        const float xs = row_ok ? p.xsq[grow] : 0.f;
        const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
        float r = 0.f;
        bool alive = true;
        auto wait_warp = [&](uint32_t a, uint32_t parity) -> bool {
            bool ok = false;
            if (lane == 0) ok = bar_wait(a, parity, abort_flag, p.status);
            return __shfl_sync(0xFFFFFFFFu, ok ? 1 : 0, 0) != 0;
        };
        for (int u = 0; u < U && alive; ++u) {
            const int n0 = (t0 + u) * BN;
            if (!wait_warp(bar(B_GFULL), (uint32_t)(u & 1))) {
                alive = false;
                break;
            }
            tc_fence_after();
            const uint32_t g_tmem = tmem + lane_addr;
            if (u == 0) {
                // reference distance: mean d^2 over the valid columns of chunks 0 and 2 of the
                // split's first tile; both warp sets compute the same value independently
                float sum = 0.f;
                int cnt = 0;
#pragma unroll 1
                for (int h = 0; h < 2; ++h) {
                    const int c = 2 * h;
#pragma unroll 1
                    for (int half = 0; half < 2; ++half) {
                        uint32_t v[32];
                        TC_LD_X32(g_tmem + c * 64 + half * 32, v);
                        tc_wait_ld();
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const int col = c * 64 + half * 32 + j;
                            if (n0 + col < p.n_sv) {
                                sum += xs + __ldg(p.svsq + n0 + col) - 2.f * p.gscale * __uint_as_float(v[j]);
                                ++cnt;
                            }
                        }
                    }
                }
                r = sum / (float)max(cnt, 1);
            }
#pragma unroll 1
            for (int h = 0; h < 2; ++h) {
                const int c = set + 2 * h;  // chunk within the tile
                const int q = 4 * u + c;    // chunk index within the split
                uint32_t pk[32];
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    uint32_t v[32];
                    TC_LD_X32(g_tmem + c * 64 + half * 32, v);
                    tc_wait_ld();
#pragma unroll
                    for (int j = 0; j < 32; j += 2) {
                        const int col = n0 + c * 64 + half * 32 + j;
                        const float d0 = xs + __ldg(p.svsq + col) - 2.f * p.gscale * __uint_as_float(v[j]);
                        const float d1 = xs + __ldg(p.svsq + col + 1) - 2.f * p.gscale * __uint_as_float(v[j + 1]);
                        const __nv_bfloat162 hv = __floats2bfloat162_rn(expm1f(-p.gamma * (d0 - r)),
                                                                        expm1f(-p.gamma * (d1 - r)));
                        pk[half * 16 + (j >> 1)] = *reinterpret_cast<const uint32_t*>(&hv);
                    }
                }
                if (h == 1) {  // this set's last read of G for the tile
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) bar_arrive(bar(B_GEMPTY));
                }
                // the slot is free once the second MMA of chunk q - 2 is done
                if (q >= 2 && !wait_warp(bar(B_FEMPTY + set), (uint32_t)(((q - 2) >> 1) & 1))) {
                    alive = false;
                    break;
                }
                unsigned char* rowp = gbase + F_OFF + set * F_CHUNK + (row >> 3) * 1024 + (row & 7) * 128;
#pragma unroll
                for (int g = 0; g < 8; ++g)
                    *reinterpret_cast<uint4*>(rowp + ((g ^ (row & 7)) << 4)) =
                        make_uint4(pk[4 * g], pk[4 * g + 1], pk[4 * g + 2], pk[4 * g + 3]);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) bar_arrive(bar(B_FFULL + set));
            }
        }
        if (alive && set == 0 && wait_warp(bar(B_DFULL), 0)) {
            tc_fence_after();
            const uint32_t d_tmem = tmem + lane_addr + 256;
            float* prow = p.part + ((size_t)split * p.n + grow) * p.C_pad;
#pragma unroll 1
            for (int c0 = 0; c0 < p.C_pad; c0 += 16) {
                uint32_t v[16];
                TC_LD_X16(d_tmem + c0, v);
                tc_wait_ld();
                if (row_ok) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) prow[c0 + j] = __uint_as_float(v[j]);
                }
            }
            if (row_ok) p.ref[(size_t)split * p.n + grow] = r;
        }
    }

    tc_fence_before();
    __syncwarp();
    if (MC)
        cluster_sync();  // no CTA leaves while its peer may still multicast into it or arrive on it
    else
        __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// asum_split[s][c] = sum of a_ci over the SVs of split s (fp64 accumulation).
__global__ void asum_split_kernel(const float* __restrict__ coef, int C, int C_pad, int n_pad, int n_sv,
                                  int sv_per_split, float* __restrict__ out) {
    const int s = blockIdx.x;
    const int i0 = s * sv_per_split, i1 = min(n_sv, i0 + sv_per_split);
    for (int c = threadIdx.x; c < C_pad; c += blockDim.x) {
        double acc = 0.0;
        if (c < C)
            for (int i = i0; i < i1; ++i) acc += (double)coef[(size_t)c * n_pad + i];
        out[(size_t)s * C_pad + c] = (float)acc;
    }
}

// Number of SV-tile ranges ("splits") per 128-row block.  One CTA runs per SM, so the time
// is about waves x (tiles per CTA + 1): the +1 stands for the pipeline fill, the epilogue of
// the last tile and the partial-sum write that every CTA pays once.  Fewer splits win ties.
int choose_splits(int mt, int nt, int sms) {
    int best = 1;
    long long best_cost = -1;
    for (int sp = 1; sp <= nt; ++sp) {
        const int tps = (nt + sp - 1) / sp;
        if ((nt + tps - 1) / tps != sp) continue;
        const long long waves = ((long long)mt * sp + sms - 1) / sms;
        const long long cost = waves * (tps + 1);
        if (best_cost < 0 || cost * 100 < best_cost * 97) {
            best_cost = cost;
            best = sp;
        }
    }
    return best;
}

// Instruction descriptor of a dense tcgen05.mma: fp32 accumulator, K-major A and B.
uint32_t make_idesc(uint32_t a_fmt, uint32_t b_fmt, int M, int N) {
    uint32_t d = 0;
    d |= 1u << 4;                      // accumulator format: F32
    d |= (a_fmt & 7u) << 7;            // A format
    d |= (b_fmt & 7u) << 10;           // B format
    d |= (uint32_t)(N >> 3) << 17;     // N / 8
    d |= (uint32_t)(M >> 4) << 24;     // M / 16
    return d;
}

}  // namespace

int pack_model_tensor_maps(rgbd_svm* m) {
    if (m->C > MAX_CPAD) {
        m->has_tmaps = false;
        return RGBD_OK;  // scoring will report the class limit
    }
    CUtensorMapDataType dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    int esz = 2;
    if (m->dtype == RGBD_DT_FP8) {
        dt = CU_TENSOR_MAP_DATA_TYPE_UINT8;
        esz = 1;
    } else if (m->dtype == RGBD_DT_TF32) {
        dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
        esz = 4;
    }
    int rc = encode_tmap_2d(&m->tm_sv, dt, m->sv, (uint64_t)m->k_pad, (uint64_t)m->n_pad,
                            (uint64_t)m->k_pad * esz, 128u / esz, BN, CU_TENSOR_MAP_SWIZZLE_128B);
    if (rc) return rc;
    rc = encode_tmap_2d(&m->tm_sv_half, dt, m->sv, (uint64_t)m->k_pad, (uint64_t)m->n_pad,
                        (uint64_t)m->k_pad * esz, 128u / esz, BN / 2, CU_TENSOR_MAP_SWIZZLE_128B);
    if (rc) return rc;
    rc = encode_tmap_2d(&m->tm_coef, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, m->coef_bf16, (uint64_t)m->n_pad,
                        (uint64_t)m->C_pad, (uint64_t)m->n_pad * 2, 64u, (uint32_t)m->C_pad,
                        CU_TENSOR_MAP_SWIZZLE_128B);
    if (rc) return rc;
    m->has_tmaps = true;
    return RGBD_OK;
}

namespace {

struct TcPlan {
    int esz, kind, splits, tps, mt, nt;
    uint32_t fmt;
    CUtensorMapDataType dt;
    size_t off_ref, off_as, bytes;
};

int plan_tc(rgbd_ctx* ctx, const rgbd_svm* m, int n, TcPlan* pl) {
    if (m->C > MAX_CPAD || !m->has_tmaps)
        return set_error(RGBD_ERR_UNSUPPORTED, "svm_score: tensor-core RBF supports up to %d classes", MAX_CPAD);
    if (ctx->props.cc_major != 10)
        return set_error(RGBD_ERR_UNSUPPORTED, "svm_score: tensor-core path needs an sm_10x GPU");
    pl->esz = 2;
    pl->kind = 0;
    pl->fmt = 1;  // BF16
    pl->dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    if (m->dtype == RGBD_DT_FP8) {
        pl->esz = 1;
        pl->kind = 1;
        pl->fmt = 0;  // E4M3
        pl->dt = CU_TENSOR_MAP_DATA_TYPE_UINT8;
    } else if (m->dtype == RGBD_DT_TF32) {
        pl->esz = 4;
        pl->kind = 2;
        pl->fmt = 2;  // TF32
        pl->dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    }
    pl->mt = (n + BM - 1) / BM;
    pl->nt = m->n_pad / BN;
    pl->splits = ctx->tune_tc_splits > 0 ? std::min(ctx->tune_tc_splits, pl->nt)
                                         : choose_splits(pl->mt, pl->nt, ctx->props.sm_count);
    pl->tps = (pl->nt + pl->splits - 1) / pl->splits;
    pl->splits = (pl->nt + pl->tps - 1) / pl->tps;  // every split non-empty
    const size_t part_bytes = sizeof(float) * (size_t)pl->splits * n * m->C_pad;
    const size_t ref_bytes = sizeof(float) * (size_t)pl->splits * n;
    const size_t as_bytes = sizeof(float) * (size_t)pl->splits * m->C_pad;
    pl->off_ref = (part_bytes + 255) & ~size_t(255);
    pl->off_as = (pl->off_ref + ref_bytes + 255) & ~size_t(255);
    pl->bytes = pl->off_as + as_bytes;
    return RGBD_OK;
}

int launch_tc(rgbd_ctx* ctx, const rgbd_svm* m, const void* x, const float* xsq, int n, float x_scale,
              float* scores, int32_t* labels, cudaStream_t s, const TcPlan& pl, char* ws) {
    float* part = (float*)ws;
    float* ref = (float*)(ws + pl.off_ref);
    float* asplit = (float*)(ws + pl.off_as);
    CUtensorMap tm_x;
    int rc = encode_tmap_2d(&tm_x, pl.dt, x, (uint64_t)m->k_pad, (uint64_t)n, (uint64_t)m->k_pad * pl.esz,
                            128u / pl.esz, BM, CU_TENSOR_MAP_SWIZZLE_128B);
    if (rc) return rc;
    // pairs of 128-row blocks share their SV tiles, unless tuned off
    const bool mc = pl.mt >= 2 && ctx->tune_tc_multicast != 2;
    cudaError_t e = mc ? cudaFuncSetAttribute(rbf_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              SMEM_BYTES)
                       : cudaFuncSetAttribute(rbf_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              SMEM_BYTES);
    if (e != cudaSuccess) return cuda_error(e, "svm_score: tc smem attribute");
    TcParams p;
    p.n = n;
    p.n_sv = m->n_sv;
    p.C = m->C;
    p.C_pad = m->C_pad;
    p.k_blocks = m->k_pad * pl.esz / 128;
    p.k_elems = 128 / pl.esz;
    p.tiles_per_split = pl.tps;
    p.n_tiles = pl.nt;
    p.gamma = m->gamma;
    p.gscale = (m->dtype == RGBD_DT_FP8) ? 1.0f / (x_scale * m->sv_scale) : 1.0f;
    p.xsq = xsq;
    p.svsq = m->sv_sq;
    p.part = part;
    p.ref = ref;
    p.status = ctx->d_status;
    p.idesc_main = make_idesc(pl.fmt, pl.fmt, BM, BN);
    p.idesc_second = make_idesc(1, 1, BM, m->C_pad);
    p.kind = pl.kind;
    asum_split_kernel<<<pl.splits, 128, 0, s>>>(m->coef, m->C, m->C_pad, m->n_pad, m->n_sv, pl.tps * BN, asplit);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "svm_score: asum split launch");
    if (mc) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)((pl.mt + 1) / 2 * 2), (unsigned)pl.splits, 1);
        cfg.blockDim = dim3(NUM_THREADS, 1, 1);
        cfg.dynamicSmemBytes = SMEM_BYTES;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, rbf_tc_kernel<true>, tm_x, m->tm_sv_half, m->tm_coef, p);
    } else {
        dim3 grid(pl.mt, pl.splits);
        rbf_tc_kernel<false><<<grid, NUM_THREADS, SMEM_BYTES, s>>>(tm_x, m->tm_sv, m->tm_coef, p);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_error(e, "svm_score: tc launch");
    return launch_reduce_scores(part, ref, pl.splits, n, m->C, m->C_pad, m->asum, asplit, m->bias, m->gamma, scores,
                                labels, s);
}

}  // namespace

int score_rbf_tc(rgbd_ctx* ctx, const rgbd_svm* m, const void* x, const float* xsq, int n, float x_scale,
                 float* scores, int32_t* labels, cudaStream_t s) {
    TcPlan pl;
    int rc = plan_tc(ctx, m, n, &pl);
    if (rc) return rc;
    rc = ensure_workspace(ctx, pl.bytes, s);
    if (rc) return rc;
    return launch_tc(ctx, m, x, xsq, n, x_scale, scores, labels, s, pl, (char*)ctx->workspace);
}

int score_rbf_tc_external_ws(rgbd_ctx* ctx, const rgbd_svm* m, const void* x, const float* xsq, int n,
                             float x_scale, float* scores, int32_t* labels, cudaStream_t s, void* ws_ptr,
                             size_t ws_cap, size_t* need) {
    TcPlan pl;
    int rc = plan_tc(ctx, m, n, &pl);
    if (rc) return rc;
    if (need) *need = pl.bytes;
    if (pl.bytes > ws_cap)
        return set_error(RGBD_ERR_ARG, "scratch of %zu bytes needed for %d rows, %d classes, %d splits; only %zu available",
                         pl.bytes, n, m->C, pl.splits, ws_cap);
    return launch_tc(ctx, m, x, xsq, n, x_scale, scores, labels, s, pl, (char*)ws_ptr);
}

}  // namespace rgbd
