// svm_tc.cu -- A6/A7 on the 5th-generation tensor cores (tcgen05, sm_103a): the RBF SVM decision
// function of Section 2.5, S_c = sum_i a_ci exp(-gamma |x - sv_i|^2) + b_c, for BF16, FP8 E4M3
// (per-tensor scales) and TF32 operands with fp32 accumulation in tensor memory.
//
// One CTA (19 warps) owns 128 feature rows and a contiguous range ("split") of 256-wide SV tiles:
//   warp 0      TMA producer of the main ring: per k-block (128 B of K per row, 128B-swizzled)
//               the 128-row X block and the SV block (4 stages of 48 KB; 6 of 32 KB in 2-CTA pairs,
//               where each CTA holds half of the SV tile and stages are released two at a time).
//   warp 1      TMEM owner and MMA issuer (one thread; in 2-CTA pairs only CTA 0's):
//                 G (128 x 256 fp32, TMEM)  = X . SV_t^T over all k-blocks   (N = 256 MMAs)
//                 D (128 x C_pad fp32, TMEM) += F_q . a_q^T  for every 64-column chunk q of F,
//               with F read from tensor memory (A operand) and a from shared memory.
//   warp 2      TMA producer of the bf16 coefficient chunks a[c][64 SVs] (2-slot ring).
//   warps 3-18  epilogue, four sets of four warps (one per TMEM lane quarter); set k handles the
//               64-column chunk k of every tile.  One thread per row reads its chunk of G with
//               tcgen05.ld and releases G, then forms d^2 = |x|^2 + |sv|^2 - 2 G and
//               F = expm1(-gamma (d^2 - r)) in bf16, and stores F with tcgen05.st into its slot
//               (two slots of 32 packed columns) for the second MMA.  r is the row's mean d^2 over
//               chunks 0 and 2 of the split's first tile; since exp(-gamma d^2) = exp(-gamma r) (1 + F),
//                 S_c = sum_splits exp(-gamma r_s) (sum_{i in s} a_ci + D_s[c]) + b_c,
//               and F keeps the small per-SV variation at full relative precision (gamma d^2 is
//               ~2e-4 for gamma = 1/dim, so exp() itself is flat to 1e-4).
// The MMA thread services finished F chunks between main-loop k-blocks, so the second MMA and
// the epilogue overlap the next tile's main loop.  Partial sums D_s and r_s go to workspace;
// launch_reduce_scores combines the splits.
//
// Batches of one 128-row block whose SV tiles would fill few SMs take rbf_tc_splitk_kernel
// instead (the K extent of every tile split over several CTAs; see there).
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
constexpr int BN = kSvTile;
constexpr int X_TILE = BM * 128;   // bytes of one X k-block
constexpr int SV_TILE = BN * 128;  // bytes of one SV k-block
constexpr int MAX_CPAD = 128;
constexpr int COEF_CHUNK_MAX = MAX_CPAD * 64 * 2;  // one 64-SV chunk of a (C_pad rows)
constexpr int MAX_STAGES = 6;

// Launch modes of the kernel.
enum { MODE_SINGLE = 0,   // one CTA per (row block, split)
       MODE_PAIR = 1 };   // CTA pairs run one 256-row MMA (cta_group::2): each CTA holds its own
                          // 128 X rows and half of the SV tile (and of the coefficient chunk)

// Shared-memory layout of a mode: main ring, coefficient ring (2 slots), barriers.  (The F
// operand of the second MMA lives in tensor memory.)
// SPLIT2: split bf16 with the second product split too (hi and lo coefficient chunks per slot).
template <int MODE, bool SPLIT2 = false>
struct Lay {
    static constexpr int STAGES = MODE == MODE_PAIR ? 6 : (SPLIT2 ? 3 : 4);
    static constexpr int SV_BYTES = MODE == MODE_PAIR ? SV_TILE / 2 : SV_TILE;  // SV rows per stage
    static constexpr int STAGE = X_TILE + SV_BYTES;
    static constexpr int COEF_CHUNK = MODE == MODE_PAIR ? COEF_CHUNK_MAX / 2 : COEF_CHUNK_MAX;
    static constexpr int COEF_SLOT = SPLIT2 ? 2 * COEF_CHUNK : COEF_CHUNK;  // hi, then lo
    static constexpr int COEF_OFF = STAGES * STAGE;
    static constexpr int BAR_OFF = COEF_OFF + 2 * COEF_SLOT;
    static constexpr int SMEM = BAR_OFF + 256 + 1024;  // + barriers + alignment slack
    static_assert(STAGES <= MAX_STAGES, "barrier slots");
    static_assert(SMEM <= 227 * 1024, "shared memory per CTA");
};
constexpr int NUM_WARPS = 19;  // producer, MMA issuer, coefficient producer, 16 epilogue warps
constexpr int NUM_THREADS = NUM_WARPS * 32;
// Tensor memory: G at column 0 (256 columns), D at 256 (C_pad <= 128 columns), the two F slots
// (128 rows x 64 bf16, packed in pairs: 32 columns each) at 384 and 416 -- or, with the second
// product split, two slots of 64 columns (hi, then lo) at 384 and 448.
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t TMEM_D = 256;
constexpr uint32_t TMEM_F = 384;
constexpr uint64_t WAIT_NS = 1000000000ull;        // 1 s: far above any legitimate wait

// barrier slots (8 bytes each) inside the barrier block
enum {
    B_FULL = 0,                       // MAX_STAGES
    B_EMPTY = B_FULL + MAX_STAGES,    // MAX_STAGES
    B_GFULL = B_EMPTY + MAX_STAGES,
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
    int passes;       // 1, or 3 for split bf16 operands (RGBD_DT_BF16X3)
    // split combine inside the kernel (fuse = 1): the last CTA of each 128-row block to finish
    // adds the splits of its rows (counters[row block] counts finished splits, zeroed per launch)
    int fuse;
    uint32_t* counters;
    const float* asum;       // [C]
    const float* asum_tile;  // [n_tiles][C_pad]
    const float* bias;       // [C]
    float* scores;           // [n][C]
    int32_t* labels;         // [n] or NULL
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
// CL: acquire at cluster scope (the barrier also receives arrivals from the peer CTA).
template <bool CL = false>
__device__ __forceinline__ bool bar_try(uint32_t a, uint32_t parity) {
    uint32_t ok;
    if (CL)
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
    return ok != 0;
}
// Non-blocking test of a phase (try_wait may suspend the thread for a while when the phase is
// not complete, which must not happen to the MMA issuer between its k-blocks).
template <bool CL = false>
__device__ __forceinline__ bool bar_test(uint32_t a, uint32_t parity) {
    uint32_t ok;
    if (CL)
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
    return ok != 0;
}
// Bounded wait.  Returns false when the CTA is aborting (deadline passed here or elsewhere).
// The abort flag and the deadline clock (%globaltimer, slow to read) are consulted only once
// every 16 failed tests, so that neither sits on the critical path of a k-block handshake; the
// deadline counts from the first consultation.
// SPIN polls with test_wait instead of try_wait: a thread suspended in try_wait resumes late
// after the phase completes, which costs the ring producer ~8 % of the scoring kernel's time.
// (The ring producer spins inline first: see bar_spin.)
template <bool CL = false, bool SPIN = false>
__device__ __noinline__ bool bar_wait(uint32_t a, uint32_t parity, volatile int* abort_flag, uint32_t* status,
                                      uint64_t limit_ns = WAIT_NS) {
    uint64_t t0 = 0;
    for (uint32_t it = 0;; ++it) {
        if (SPIN ? bar_test<CL>(a, parity) : bar_try<CL>(a, parity)) return true;
        if ((it & 15u) != 15u) continue;
        if (*abort_flag) return false;
        const uint64_t now = globaltimer();
        if (t0 == 0) {
            t0 = now;
        } else if (now - t0 > limit_ns) {
            *abort_flag = 1;
            atomicOr(status, RGBD_STATUS_WAIT_TIMEOUT);
            return false;
        }
    }
}
// The ring producer's wait, on the critical path of every k-block: an inline test_wait spin
// (a call into bar_wait per k-block costs ~8 % of the scoring kernel), then the bounded wait.
template <bool CL>
__device__ __forceinline__ bool bar_spin(uint32_t a, uint32_t parity, volatile int* abort_flag, uint32_t* status) {
    for (int i = 0; i < 4096; ++i)
        if (bar_test<CL>(a, parity)) return true;
    return bar_wait<CL, true>(a, parity, abort_flag, status);
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
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
// The address of the same shared-memory object in cluster CTA 0 (the pair's MMA issuer).
__device__ __forceinline__ uint32_t map_rank0(uint32_t a) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, 0;" : "=r"(r) : "r"(a));
    return r;
}
// Arrive on an mbarrier given by its cluster address (possibly in the peer CTA).
__device__ __forceinline__ void bar_arrive_cluster(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
// TMA load into this CTA's shared memory whose completion is counted on an mbarrier of either
// CTA of the pair (cluster address).
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap* map, int x, int y,
                                                 uint32_t bar_cluster) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.cta_group::2"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar_cluster)
        : "memory");
}
__device__ __forceinline__ void tc_commit2(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// Commit of a 2-CTA MMA pair whose arrive lands on the same barrier in both CTAs of `mask`.
__device__ __forceinline__ void tc_commit2_pair(uint32_t bar, uint16_t mask) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(bar),
        "h"(mask)
        : "memory");
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
// KIND: 0 = kind::f16 (bf16 operands), 1 = kind::f8f6f4 (E4M3), 2 = kind::tf32, 3 = kind::f16 with
// split bf16 operands (three passes, and the second product split as well).
template <int CG, int KIND>
__device__ __forceinline__ void mma_issue(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
#define RGBD_MMA_SS(CGS, KS)                                                                          \
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"                                   \
                 "tcgen05.mma.cta_group::" CGS ".kind::" KS " [%0], %1, %2, %3, p;\n\t}" ::"r"(d), "l"(a), \
                 "l"(b), "r"(idesc), "r"(acc))
    if constexpr (CG == 1) {
        if constexpr (KIND == 0 || KIND == 3) RGBD_MMA_SS("1", "f16");
        else if constexpr (KIND == 1) RGBD_MMA_SS("1", "f8f6f4");
        else RGBD_MMA_SS("1", "tf32");
    } else {
        if constexpr (KIND == 0 || KIND == 3) RGBD_MMA_SS("2", "f16");
        else if constexpr (KIND == 1) RGBD_MMA_SS("2", "f8f6f4");
        else RGBD_MMA_SS("2", "tf32");
    }
#undef RGBD_MMA_SS
}
// D (+)= A B^T with A (bf16, 128 rows per CTA) in tensor memory and B in shared memory.
template <int CG>
__device__ __forceinline__ void mma_issue_ts(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc) {
    if (CG == 1)
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
            "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc));
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
            "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc));
}
#define TC_ST_X32(taddr, v)                                                                                   \
    asm volatile(                                                                                             \
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"   \
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),                 \
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]),      \
        "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]),         \
        "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]),        \
        "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])                     \
        : "memory")
__device__ __forceinline__ void tc_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
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
// e^z - 1.  The near-flat RBF gives |z| = gamma |d^2 - r| of order 1e-3, where the Taylor series
// z + z^2/2! + ... + z^6/6! (Horner form) is exact to fp32 rounding: for |z| < 2^-5 the first
// omitted term is below 2^-30 |z| / 5040.  Larger arguments use expm1f.
__device__ __forceinline__ float expm1_near0(float z) {
    if (fabsf(z) < 0.03125f) {
        float q = fmaf(z, 1.0f / 720.0f, 1.0f / 120.0f);
        q = fmaf(z, q, 1.0f / 24.0f);
        q = fmaf(z, q, 1.0f / 6.0f);
        q = fmaf(z, q, 0.5f);
        return fmaf(z * z, q, z);
    }
    return expm1f(z);
}
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }


// ---------------------------------------------------------------------------------------
// Split combine (A7), run by the last CTA of a 128-row block to finish: for each row and class
//   S_c = exp(-gamma r*) (asum_c + sum_s [D_s + delta_s (asum_{c,s} + D_s)]) + b_c,
// delta_s = expm1(-gamma (r_s - r*)), r* = r_0, asum_{c,s} the coefficient sum of split s's
// tiles -- the same terms in the same order as the split-combine kernels of
// launch_reduce_scores -- then the argmax (lowest class on ties).  The other splits' partial sums are read past L1 (__ldcg): their CTAs fenced
// them before counting themselves finished.  `work` is shared memory of combine_bytes().
// ---------------------------------------------------------------------------------------
__host__ __device__ inline size_t combine_bytes(int splits, int C_pad) {
    return sizeof(float) * ((size_t)splits * C_pad + (size_t)splits * BM + BM + (size_t)BM * C_pad);
}

__device__ __noinline__ void combine_splits(const TcParams& p, int m0, int splits, float* work) {
    const int C = p.C, Cs = p.C_pad, tid = threadIdx.x, nth = blockDim.x;
    float* s_as = work;                          // [splits][C_pad]
    float* s_delta = s_as + (size_t)splits * Cs;  // [splits][BM]
    float* s_esc = s_delta + (size_t)splits * BM;  // [BM]
    float* s_sc = s_esc + BM;                     // [BM][C_pad]
    for (int i = tid; i < splits * Cs; i += nth) {
        const int sp = i / Cs, c = i - sp * Cs;
        float v = 0.f;
        if (sp > 0 && c < C)
            for (int t = sp * p.tiles_per_split; t < min(p.n_tiles, (sp + 1) * p.tiles_per_split); ++t)
                v += __ldg(p.asum_tile + (size_t)t * Cs + c);
        s_as[i] = v;
    }
    for (int i = tid; i < splits * BM; i += nth) {
        const int sp = i / BM, rl = i - sp * BM, row = m0 + rl;
        float d = 0.f;
        if (row < p.n) {
            const float rstar = __ldcg(p.ref + row);
            if (sp > 0) d = expm1f(-p.gamma * (__ldcg(p.ref + (size_t)sp * p.n + row) - rstar));
            else s_esc[rl] = expf(-p.gamma * rstar);
        }
        s_delta[i] = d;
    }
    __syncthreads();
    for (int i = tid; i < BM * C; i += nth) {
        const int rl = i / C, c = i - rl * C, row = m0 + rl;
        if (row >= p.n) continue;
        float acc = 0.f;
        for (int sp = 0; sp < splits; ++sp) {
            const float d = __ldcg(p.part + ((size_t)sp * p.n + row) * Cs + c);
            acc += d + s_delta[sp * BM + rl] * (s_as[sp * Cs + c] + d);
        }
        const float sc = s_esc[rl] * (__ldg(p.asum + c) + acc) + __ldg(p.bias + c);
        p.scores[(size_t)row * C + c] = sc;
        s_sc[rl * Cs + c] = sc;
    }
    if (!p.labels) return;
    __syncthreads();
    const int lane = tid & 31;
    for (int rl = tid >> 5; rl < BM; rl += nth >> 5) {
        if (m0 + rl >= p.n) continue;
        float best = -INFINITY;
        int bi = 0x7FFFFFFF;
        for (int c = lane; c < C; c += 32) {
            const float v = s_sc[rl * Cs + c];
            if (v > best) {
                best = v;
                bi = c;
            }
        }
        for (int off = 16; off > 0; off >>= 1) {
            const float ob = __shfl_xor_sync(0xFFFFFFFFu, best, off);
            const int oi = __shfl_xor_sync(0xFFFFFFFFu, bi, off);
            if (ob > best || (ob == best && oi < bi)) {
                best = ob;
                bi = oi;
            }
        }
        if (lane == 0) p.labels[m0 + rl] = bi;
    }
}

// ---------------------------------------------------------------------------------------
// The kernel
// ---------------------------------------------------------------------------------------
// MODE_PAIR: the two CTAs of a cluster form one 256-row MMA (tcgen05 cta_group::2).  Each CTA
// loads its own 128 X rows and one half of the SV tile (CTA r: SVs r*128 .. r*128+127 of the
// tile) and one half of the classes of each coefficient chunk; CTA 0 issues every MMA, which
// reads the operands of both CTAs and writes G and D into both CTAs' tensor memory (each CTA
// holds its own rows).  All copies count on CTA 0's barriers, and CTA 0's commits arrive on
// both CTAs' barriers.  Per MMA each CTA supplies 8 KB of operands instead of 12 KB.
template <int MODE, int KIND>
__global__ void __launch_bounds__(NUM_THREADS, 1)
    rbf_tc_kernel(const __grid_constant__ CUtensorMap tm_x, const __grid_constant__ CUtensorMap tm_sv,
                  const __grid_constant__ CUtensorMap tm_coef, const __grid_constant__ CUtensorMap tm_x2,
                  const __grid_constant__ CUtensorMap tm_sv2, const __grid_constant__ CUtensorMap tm_coef2,
                  const TcParams p) {
    constexpr bool PAIR = MODE == MODE_PAIR;
    constexpr bool SPLIT2 = KIND == 3;
    constexpr int CG = PAIR ? 2 : 1;
    constexpr uint32_t F_SLOT = SPLIT2 ? 64u : 32u;  // TMEM columns per F slot
    using L = Lay<MODE, SPLIT2>;
    // Pairs fill and release ring stages two at a time (one FULL and one EMPTY barrier per
    // group): a 2-CTA commit per k-block cost ~5 % of the kernel (the ring turned over
    // slower than its copies land).  Single CTAs, with a 4-stage ring, keep one per stage.
    constexpr int GRP = (MODE == MODE_PAIR && L::STAGES % 2 == 0) ? 2 : 1;  // stages released per commit
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;  // 1024-byte aligned for the 128B swizzle atoms
    unsigned char* gbase = smem_raw + (base - raw);
    const uint32_t bars = base + L::BAR_OFF;
    auto bar = [&](int i) { return bars + 8u * (uint32_t)i; };
    volatile int* abort_flag = reinterpret_cast<volatile int*>(gbase + L::BAR_OFF + 8 * B_COUNT);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbase + L::BAR_OFF + 8 * B_COUNT + 8);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * BM;
    const int split = blockIdx.y;
    const int t0 = split * p.tiles_per_split;
    const int t1 = min(p.n_tiles, t0 + p.tiles_per_split);
    const int U = t1 - t0;   // tiles of this split (>= 1)
    const int Q = 4 * U;     // 64-column chunks of this split

    if (threadIdx.x == 0) {
        for (int s = 0; s < L::STAGES; ++s) {
            bar_init(bar(B_FULL + s), 1);
            bar_init(bar(B_EMPTY + s), 1);
        }
        bar_init(bar(B_GFULL), 1);
        bar_init(bar(B_GEMPTY), PAIR ? 32 : 16);  // the epilogue warps (of both CTAs of a pair)
        for (int s = 0; s < 2; ++s) {
            // 4 epilogue warps (per CTA of a pair) + the coefficient producer
            bar_init(bar(B_FFULL + s), PAIR ? 8 + 1 : 4 + 1);
            bar_init(bar(B_FEMPTY + s), 1);
        }
        bar_init(bar(B_DFULL), 1);
        bar_init(bar(B_DRAIN), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (PAIR) cluster_sync();  // both CTAs are running before they allocate together
    if (warp == 1) {
        if (PAIR) {
            // one warp of each CTA of the pair allocates collectively (same columns in both)
            asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(tmem_slot)),
                         "r"(TMEM_COLS)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
        } else {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(tmem_slot)),
                         "r"(TMEM_COLS)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
    }
    tc_fence_before();
    __syncwarp();
    if (PAIR)
        cluster_sync();  // the peer's barriers are initialised before any copy or commit reaches them
    else
        __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t crank = PAIR ? cluster_rank() : 0u;
    const uint32_t coef_chunk_bytes = (uint32_t)(PAIR ? p.C_pad / 2 : p.C_pad) * 128u;

    if (warp == 0) {
        // ===================== TMA producer: X and SV k-blocks =====================
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tm_x) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tm_sv) : "memory");
            int stage = 0;
            uint32_t phase = 0, armed = 0, armed_par = 0;
            bool alive = true;
            const int KT = p.passes * p.k_blocks;  // k-blocks per tile
            for (int u = 0; u < U && alive; ++u) {
                const int n0 = (t0 + u) * BN;
                for (int kt = 0; kt < KT; ++kt) {
                    // three passes for split bf16 operands: (x_hi, sv_hi), (x_hi, sv_lo), (x_lo, sv_hi)
                    const int pass = kt / p.k_blocks, kb = kt - pass * p.k_blocks;
                    const CUtensorMap* mx = (pass == 2) ? &tm_x2 : &tm_x;
                    const CUtensorMap* msv = (pass == 1) ? &tm_sv2 : &tm_sv;
                    // the first stage of a group waits for the group's release (EMPTY slot stage / GRP)
                    if ((GRP == 1 || stage % GRP == 0) &&
                        !bar_spin<PAIR>(bar(B_EMPTY + stage / GRP), phase ^ 1u, abort_flag, p.status)) {
                        alive = false;
                        break;
                    }
                    const uint32_t sa = base + (uint32_t)stage * L::STAGE;
                    if (PAIR) {
                        const uint32_t fb = map_rank0(bar(B_FULL + stage / GRP));
                        // one FULL barrier per group of stages: the group's first stage arms it
                        // for all the group's copies (fewer when the split's k-blocks run out)
                        if (crank == 0 && stage % GRP == 0) {
                            const int left = U * KT - (u * KT + kt);  // k-blocks still to load
                            const uint32_t nst = (uint32_t)min(GRP, left);
                            bar_arrive_tx(bar(B_FULL + stage / GRP), 2u * L::STAGE * nst);
                        }
                        tma_load_2d_pair(sa, mx, kb * p.k_elems, m0, fb);
                        tma_load_2d_pair(sa + X_TILE, msv, kb * p.k_elems, n0 + (int)crank * (BN / 2), fb);
                    } else {
                        bar_arrive_tx(bar(B_FULL + stage), L::STAGE);
                        tma_load_2d(sa, mx, kb * p.k_elems, m0, bar(B_FULL + stage));
                        tma_load_2d(sa + X_TILE, msv, kb * p.k_elems, n0, bar(B_FULL + stage));
                    }
                    armed |= 1u << stage;
                    armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
                    if (++stage == L::STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!alive && PAIR && crank != 0) {
                // this CTA's copies count on the peer's barriers: give those in flight a bounded
                // 200 us to land
                (void)armed;
                const uint64_t tq = globaltimer();
                while (globaltimer() - tq < 200000ull) {
                }
            } else if (!alive) {  // drain: wait (bounded) for the copies this thread issued
                const uint64_t tq = globaltimer();
                for (int s = 0; s < L::STAGES; ++s)
                    if (armed & (1u << s))
                        while (!bar_try<PAIR>(bar(B_FULL + s / GRP), (armed_par >> s) & 1u) &&
                               globaltimer() - tq < WAIT_NS) {
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
                if (q >= 2 &&
                    !bar_wait<PAIR>(bar(B_FEMPTY + slot), (uint32_t)(((q - 2) >> 1) & 1), abort_flag, p.status)) {
                    alive = false;
                    break;
                }
                const int n0 = (t0 + (q >> 2)) * BN + (q & 3) * 64;
                const uint32_t dst = base + L::COEF_OFF + slot * L::COEF_SLOT;
                const uint32_t nb = (SPLIT2 ? 2u : 1u) * coef_chunk_bytes;
                if (PAIR) {
                    const uint32_t fb = map_rank0(bar(B_FFULL + slot));
                    if (crank == 0) bar_arrive_tx(bar(B_FFULL + slot), 2u * nb);
                    tma_load_2d_pair(dst, &tm_coef, n0, (int)crank * (p.C_pad / 2), fb);
                    if (SPLIT2) tma_load_2d_pair(dst + L::COEF_CHUNK, &tm_coef2, n0, (int)crank * (p.C_pad / 2), fb);
                } else {
                    bar_arrive_tx(bar(B_FFULL + slot), nb);
                    tma_load_2d(dst, &tm_coef, n0, 0, bar(B_FFULL + slot));
                    if (SPLIT2) tma_load_2d(dst + L::COEF_CHUNK, &tm_coef2, n0, 0, bar(B_FFULL + slot));
                }
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
        // ===================== MMA issuer (CTA 0 of a pair) =====================
        if (lane == 0 && (!PAIR || crank == 0)) {
            int stage = 0;
            uint32_t phase = 0;
            bool alive = true;
            int q_next = 0, q_avail = 0;
            const uint32_t d_tmem = tmem + TMEM_D;  // second-MMA accumulator, C_pad columns
            // Issues the second MMA of the next finished F chunk; returns false if none is ready.
            auto service = [&]() -> bool {
                if (q_next >= q_avail) return false;
                const int slot = q_next & 1;
                if (!bar_test<PAIR>(bar(B_FFULL + slot), (uint32_t)((q_next >> 1) & 1))) return false;
                tc_fence_after();
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {  // K = 16 per MMA: 8 packed columns of F
                    const uint32_t a = tmem + TMEM_F + F_SLOT * slot + 8u * ks;
                    const uint32_t cb = base + L::COEF_OFF + slot * L::COEF_SLOT + ks * 32;
                    mma_issue_ts<CG>(d_tmem, a, sdesc(cb), p.idesc_second, (q_next > 0 || ks > 0) ? 1u : 0u);
                    if (SPLIT2) {  // + F_hi a_lo + F_lo a_hi
                        mma_issue_ts<CG>(d_tmem, a, sdesc(cb + L::COEF_CHUNK), p.idesc_second, 1u);
                        mma_issue_ts<CG>(d_tmem, a + 32u, sdesc(cb), p.idesc_second, 1u);
                    }
                }
                if (PAIR)
                    tc_commit2_pair(bar(B_FEMPTY + slot), (uint16_t)0x3);
                else
                    tc_commit(bar(B_FEMPTY + slot));
                ++q_next;
                return true;
            };
            // Blocks (bounded) until barrier (a, parity) completes, servicing chunks meanwhile:
            // while a chunk may still arrive the barrier is polled without suspending.
            auto wait_servicing = [&](uint32_t a, uint32_t parity) -> bool {
                uint64_t tw = 0;
                for (uint32_t it = 0; !(q_next < q_avail ? bar_test<PAIR>(a, parity) : bar_try<PAIR>(a, parity)); ++it) {
                    if (service()) continue;
                    if (*abort_flag) return false;
                    if ((it & 15u) != 0) continue;  // the deadline clock is slow to read
                    if (tw == 0) tw = globaltimer();
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
                for (int kt = 0; kt < p.passes * p.k_blocks; ++kt) {
                    // The issue loop must stay well under the 512 tensor-pipe cycles of a k-block,
                    // so the ready case costs one barrier test, the stage's TMA data needs no
                    // tcgen05 fence (the barrier orders it), and finished F chunks are serviced only
                    // every 8 k-blocks (the epilogue waits two chunks back).
                    // one wait per group of stages (its FULL barrier counts all its copies)
                    if (stage % GRP == 0 && !bar_try<PAIR>(bar(B_FULL + stage / GRP), phase) &&
                        !wait_servicing(bar(B_FULL + stage / GRP), phase)) {
                        alive = false;
                        break;
                    }
                    const uint32_t sa = base + (uint32_t)stage * L::STAGE;
                    const uint64_t a0 = sdesc(sa), b0 = sdesc(sa + X_TILE);
                    // K step ks starts 32 bytes further along the swizzled rows: +2 in the
                    // descriptor's address field (16-byte units)
                    mma_issue<CG, KIND>(tmem, a0, b0, p.idesc_main, kt > 0 ? 1u : 0u);
#pragma unroll
                    for (int ks = 1; ks < 4; ++ks)
                        mma_issue<CG, KIND>(tmem, a0 + 2u * ks, b0 + 2u * ks, p.idesc_main, 1u);
                    // release a group after its last stage (and after the split's last k-block)
                    if (GRP == 1 || stage % GRP == GRP - 1 || (u == U - 1 && kt == p.passes * p.k_blocks - 1)) {
                        if (PAIR)
                            tc_commit2_pair(bar(B_EMPTY + stage / GRP), (uint16_t)0x3);
                        else
                            tc_commit(bar(B_EMPTY + stage / GRP));
                    }
                    if (++stage == L::STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                    if ((kt & 7) == 7) service();
                }
                if (!alive) break;
                if (PAIR)
                    tc_commit2_pair(bar(B_GFULL), (uint16_t)0x3);
                else
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
            if (alive) {
                if (PAIR)
                    tc_commit2_pair(bar(B_DFULL), (uint16_t)0x3);
                else
                    tc_commit(bar(B_DFULL));
            }
            // drain: every MMA this thread issued has completed once B_DRAIN flips
            if (PAIR)
                tc_commit2(bar(B_DRAIN));
            else
                tc_commit(bar(B_DRAIN));
            const uint64_t tq = globaltimer();
            while (!bar_try(bar(B_DRAIN), 0)) {
                if (globaltimer() - tq > WAIT_NS) break;
            }
        }
    } else {
        // ===================== epilogue: warps 3..18, one thread per row =====================
        // Four sets of four warps; set s converts chunk s (columns 64 s .. 64 s + 63) of every
        // tile.  A thread first reads its whole chunk of G, so that the issuer may start the
        // next tile's G as soon as every set has read, and only then computes F.
        const int ew = warp - 3;           // 0..15
        const int set = ew >> 2;           // chunk of every tile
        const int slot = set & 1;          // F slot and coefficient slot of the chunk (q & 1)
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
            if (lane == 0) ok = bar_wait<PAIR>(a, parity, abort_flag, p.status);
            return __shfl_sync(0xFFFFFFFFu, ok ? 1 : 0, 0) != 0;
        };
        for (int u = 0; u < U && alive; ++u) {
            const int n0 = (t0 + u) * BN;
            // the tile's G: lane 0 polls with short sleeps (a thread suspended in try_wait wakes
            // late, and plain spinning takes issue slots from the warps computing F), then falls
            // back to the bounded wait
            bool g_ok = true;
            if (lane == 0) {
                int polls = 0;
                while (!bar_test<PAIR>(bar(B_GFULL), (uint32_t)(u & 1))) {
                    __nanosleep(64);
                    if (++polls > (1 << 20)) {
                        g_ok = bar_wait<PAIR>(bar(B_GFULL), (uint32_t)(u & 1), abort_flag, p.status);
                        break;
                    }
                }
            }
            if (!__shfl_sync(0xFFFFFFFFu, g_ok ? 1 : 0, 0)) {
                alive = false;
                break;
            }
            tc_fence_after();
            const uint32_t g_tmem = tmem + lane_addr;
            if (u == 0) {
                // reference distance: mean d^2 over the valid columns of chunks 0 and 2 of the
                // split's first tile; the four sets compute the same value independently
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
            {
                const int c = set;          // chunk within the tile
                const int q = 4 * u + c;    // chunk index within the split
                uint32_t pk[32], pl[SPLIT2 ? 32 : 1];
                uint32_t v[2][32];
                TC_LD_X32(g_tmem + c * 64, v[0]);
                TC_LD_X32(g_tmem + c * 64 + 32, v[1]);
                tc_wait_ld();
                // this set's only read of G for the tile
                tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    if (PAIR)
                        bar_arrive_cluster(map_rank0(bar(B_GEMPTY)));
                    else
                        bar_arrive(bar(B_GEMPTY));
                }
#pragma unroll
                for (int half = 0; half < 2; ++half) {
#pragma unroll
                    for (int j = 0; j < 32; j += 2) {
                        const int col = n0 + c * 64 + half * 32 + j;
                        const float d0 = xs + __ldg(p.svsq + col) - 2.f * p.gscale * __uint_as_float(v[half][j]);
                        const float d1 = xs + __ldg(p.svsq + col + 1) - 2.f * p.gscale * __uint_as_float(v[half][j + 1]);
                        const float f0 = expm1_near0(-p.gamma * (d0 - r)), f1 = expm1_near0(-p.gamma * (d1 - r));
                        const __nv_bfloat162 hv = __floats2bfloat162_rn(f0, f1);
                        pk[half * 16 + (j >> 1)] = *reinterpret_cast<const uint32_t*>(&hv);
                        if (SPLIT2) {  // lo = bf16(F - hi)
                            const __nv_bfloat162 lv = __floats2bfloat162_rn(f0 - __low2float(hv), f1 - __high2float(hv));
                            pl[SPLIT2 ? half * 16 + (j >> 1) : 0] = *reinterpret_cast<const uint32_t*>(&lv);
                        }
                    }
                }
                // the slot is free once the second MMA of chunk q - 2 is done
                if (q >= 2 && !wait_warp(bar(B_FEMPTY + slot), (uint32_t)(((q - 2) >> 1) & 1))) {
                    alive = false;
                    break;
                }
                // F of this warp's 32 rows into the slot's 32 columns (row = TMEM lane); the lo
                // part into the next 32 when the second product is split
                TC_ST_X32(tmem + lane_addr + TMEM_F + F_SLOT * (uint32_t)slot, pk);
                if constexpr (SPLIT2) TC_ST_X32(tmem + lane_addr + TMEM_F + F_SLOT * (uint32_t)slot + 32u, pl);
                tc_wait_st();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    if (PAIR)
                        bar_arrive_cluster(map_rank0(bar(B_FFULL + slot)));
                    else
                        bar_arrive(bar(B_FFULL + slot));
                }
            }
        }
        if (alive && set == 0 && wait_warp(bar(B_DFULL), 0)) {
            tc_fence_after();
            const uint32_t d_tmem = tmem + lane_addr + TMEM_D;
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
            if (p.fuse) __threadfence();  // this split's sums are visible before it counts as done
        }
    }

    tc_fence_before();
    __syncwarp();
    if (PAIR)
        cluster_sync();  // no CTA leaves while its peer's commits may still arrive on it
    else
        __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        if (PAIR)
            asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                         : "memory");
        else
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                         : "memory");
    }
    if (p.fuse) {
        // the last split of this row block to finish adds them all; the ring's shared memory is
        // free now (every copy and MMA of the CTA has completed)
        __shared__ int last;
        if (threadIdx.x == 0) {
            __threadfence();
            last = atomicAdd(p.counters + blockIdx.x, 1u) == gridDim.y - 1;
        }
        __syncthreads();
        if (last) {
            __threadfence();
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the ring was the async proxy's
            combine_splits(p, m0, (int)gridDim.y, reinterpret_cast<float*>(gbase));
        }
    }
}

// ---------------------------------------------------------------------------------------
// Small batches (one 128-row block): split over K.
// ---------------------------------------------------------------------------------------
// With at most 128 rows the kernel above runs one CTA per SV tile at most (32 CTAs for 8192
// SVs), and each streams a whole 7.7 MB SV tile through its ring: a one-frame serving batch
// takes as long as 4096 rows take per CTA.  Here the K extent (the k-blocks of every pass) of
// each SV tile is cut into `kz` ranges, one CTA per (tile, range), so that all SMs stream the
// SVs; each CTA writes its partial G = X . SV_t^T of the valid rows to `gpart`
// ([kz][n_pad][n]), and rbf_splitk_epilogue_kernel adds the ranges, finishes the tile and, in
// the last CTA of each row group, combines the tiles into scores and labels.
// Warps: 0 the TMA producer (4 stages of X and SV k-blocks), 1 the TMEM owner and MMA issuer,
// 2-5 the epilogue (one thread per row, TMEM lane quarter = warp % 4).  The X copies hold only
// the batch's rows (rounded up to 8, the swizzle atom's height): the MMA still reads 128 rows,
// but an output row depends only on its own A row, and rows past the batch are never written.
// G for one SV tile lives in 256 tensor-memory columns.
constexpr int SK_WARPS = 6;
constexpr int SK_STAGES = 4;
constexpr int SK_STAGE = X_TILE + SV_TILE;
constexpr int SK_BAR_OFF = SK_STAGES * SK_STAGE;
constexpr int SK_SMEM = SK_BAR_OFF + 256 + 1024;
enum { SK_FULL = 0, SK_EMPTY = SK_FULL + SK_STAGES, SK_GFULL = SK_EMPTY + SK_STAGES, SK_DRAIN = SK_GFULL + 1,
       SK_COUNT = SK_DRAIN + 1 };

struct SkParams {
    int n;          // rows (<= BM)
    int n_pad;      // SV rows of the model (a multiple of BN)
    int k_blocks;   // k-blocks per pass
    int k_elems;    // elements per k-block
    int passes;     // 1, or 3 for split bf16 operands
    int kpz;        // k-blocks (over all passes) per K range
    uint32_t x_bytes;  // bytes of one X k-block: only the valid rows, rounded up to 8, are copied
    uint32_t idesc;
    float* gpart;   // [kz][n_pad][n]
    uint32_t* counters;  // [n_groups]: finished tiles per row group of the epilogue, zeroed here
    int n_groups;
    uint32_t* status;
};

template <int KIND>
__global__ void __launch_bounds__(SK_WARPS * 32, 1)
    rbf_tc_splitk_kernel(const __grid_constant__ CUtensorMap tm_x, const __grid_constant__ CUtensorMap tm_sv,
                         const __grid_constant__ CUtensorMap tm_x2, const __grid_constant__ CUtensorMap tm_sv2,
                         const SkParams p) {
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char* gbase = smem_raw + (base - raw);
    const uint32_t bars = base + SK_BAR_OFF;
    auto bar = [&](int i) { return bars + 8u * (uint32_t)i; };
    volatile int* abort_flag = reinterpret_cast<volatile int*>(gbase + SK_BAR_OFF + 8 * SK_COUNT);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbase + SK_BAR_OFF + 8 * SK_COUNT + 8);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tile = blockIdx.x, z = blockIdx.y;
    const int KT = p.passes * p.k_blocks;
    const int kt0 = z * p.kpz, kt1 = min(KT, kt0 + p.kpz);  // non-empty: the host sizes kz so

    if (blockIdx.x == 0 && blockIdx.y == 0)  // the epilogue kernel that follows counts on these
        for (int i = threadIdx.x; i < p.n_groups; i += blockDim.x) p.counters[i] = 0u;
    // the epilogue kernel may be scheduled now: its CTAs wait (griddepcontrol.wait) for this grid
    // to complete, so its launch latency hides behind this kernel instead of following it
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (threadIdx.x == 0) {
        for (int s = 0; s < SK_STAGES; ++s) {
            bar_init(bar(SK_FULL + s), 1);
            bar_init(bar(SK_EMPTY + s), 1);
        }
        bar_init(bar(SK_GFULL), 1);
        bar_init(bar(SK_DRAIN), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"((uint32_t)BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ===================== TMA producer =====================
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0, armed = 0, armed_par = 0;
            for (int kt = kt0; kt < kt1; ++kt) {
                const int pass = kt / p.k_blocks, kb = kt - pass * p.k_blocks;
                const CUtensorMap* mx = (pass == 2) ? &tm_x2 : &tm_x;
                const CUtensorMap* msv = (pass == 1) ? &tm_sv2 : &tm_sv;
                if (!bar_spin<false>(bar(SK_EMPTY + stage), phase ^ 1u, abort_flag, p.status)) break;
                const uint32_t sa = base + (uint32_t)stage * SK_STAGE;
                bar_arrive_tx(bar(SK_FULL + stage), p.x_bytes + SV_TILE);
                tma_load_2d(sa, mx, kb * p.k_elems, 0, bar(SK_FULL + stage));
                tma_load_2d(sa + X_TILE, msv, kb * p.k_elems, tile * BN, bar(SK_FULL + stage));
                armed |= 1u << stage;
                armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
                if (++stage == SK_STAGES) {
                    stage = 0;
                    phase ^= 1u;
                }
            }
            if (*abort_flag) {  // drain: wait (bounded) for the copies this thread issued
                const uint64_t tq = globaltimer();
                for (int s = 0; s < SK_STAGES; ++s)
                    if (armed & (1u << s))
                        while (!bar_try(bar(SK_FULL + s), (armed_par >> s) & 1u) && globaltimer() - tq < WAIT_NS) {
                        }
            }
        }
    } else if (warp == 1) {
        // ===================== MMA issuer =====================
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            bool alive = true;
            for (int kt = kt0; kt < kt1; ++kt) {
                if (!bar_try(bar(SK_FULL + stage), phase) &&
                    !bar_wait<false, true>(bar(SK_FULL + stage), phase, abort_flag, p.status)) {
                    alive = false;
                    break;
                }
                const uint32_t sa = base + (uint32_t)stage * SK_STAGE;
                const uint64_t a0 = sdesc(sa), b0 = sdesc(sa + X_TILE);
                mma_issue<1, KIND>(tmem, a0, b0, p.idesc, kt > kt0 ? 1u : 0u);
#pragma unroll
                for (int ks = 1; ks < 4; ++ks) mma_issue<1, KIND>(tmem, a0 + 2u * ks, b0 + 2u * ks, p.idesc, 1u);
                tc_commit(bar(SK_EMPTY + stage));
                if (++stage == SK_STAGES) {
                    stage = 0;
                    phase ^= 1u;
                }
            }
            if (alive) tc_commit(bar(SK_GFULL));
            // drain: every MMA this thread issued has completed once SK_DRAIN flips
            tc_commit(bar(SK_DRAIN));
            const uint64_t tq = globaltimer();
            while (!bar_try(bar(SK_DRAIN), 0)) {
                if (globaltimer() - tq > WAIT_NS) break;
            }
        }
    } else {
        // ===================== epilogue: warps 2..5, one thread per row =====================
        const int quarter = warp & 3;
        const int row = quarter * 32 + lane;
        bool ok = false;
        if (lane == 0) ok = bar_wait<false>(bar(SK_GFULL), 0, abort_flag, p.status);
        if (__shfl_sync(0xFFFFFFFFu, ok ? 1 : 0, 0)) {
            tc_fence_after();
            const uint32_t g_tmem = tmem + ((uint32_t)(quarter * 32) << 16);
            float* out = p.gpart + ((size_t)z * p.n_pad + (size_t)tile * BN) * p.n + row;
#pragma unroll 1
            for (int c = 0; c < BN; c += 32) {
                uint32_t v[32];
                TC_LD_X32(g_tmem + c, v);
                tc_wait_ld();
                if (row < p.n) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) out[(size_t)(c + j) * p.n] = __uint_as_float(v[j]);
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)BN)
                     : "memory");
    }
}

// Finishes one SV tile for up to SKE_ROWS rows: G = the sum of the K ranges' partials,
// d^2 = |x|^2 + |sv|^2 - 2 G, the row's reference distance r (mean d^2 over the tile's real SVs),
// F = expm1(-gamma (d^2 - r)) and D_c = sum_i a_ci F_i with the fp32 coefficients.  Each tile
// is one split of the split combine (D and r per tile); the last CTA of a row group to finish
// (counters[row group], zeroed by the split-K kernel) adds the tiles of its rows and takes the
// argmax, with the terms of the combine kernels of launch_reduce_scores.  The loads of each step
// are issued together: the kernel is a short chain of dependent L2 round trips.
constexpr int SKE_ROWS = 16;
constexpr int SKE_THREADS = 256;
constexpr int SKE_CPW = 8;  // classes per warp and pass (their coefficients loaded at once)
__global__ void __launch_bounds__(SKE_THREADS) rbf_splitk_epilogue_kernel(
    const float* __restrict__ gpart, int kz, int n_pad, int n, const float* __restrict__ xsq,
    const float* __restrict__ svsq, int n_sv, const float* __restrict__ coef, int C, int C_pad, float gamma,
    float gscale, float* __restrict__ part, float* __restrict__ ref, uint32_t* __restrict__ counters, int nt,
    const float* __restrict__ asum, const float* __restrict__ asum_tile, const float* __restrict__ bias,
    float* __restrict__ scores, int32_t* __restrict__ labels) {
    __shared__ float F[SKE_ROWS][BN];
    __shared__ float r_row[SKE_ROWS];
    __shared__ int last;
    // launched as a programmatic dependent of the split-K kernel: wait for it to complete
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int tile = blockIdx.x, k0 = blockIdx.y * SKE_ROWS;
    const int rows = min(SKE_ROWS, n - k0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = SKE_THREADS / 32;
    static_assert(SKE_THREADS == BN, "one thread per SV column of the tile");
    {
        // thread = column: every K range's partial of every row, all loads issued together
        const int col = tile * BN + threadIdx.x;
        const size_t zs = (size_t)n_pad * n;
        const float* gp = gpart + (size_t)col * n + k0;
        float g[SKE_ROWS];
#pragma unroll
        for (int k = 0; k < SKE_ROWS; ++k) g[k] = 0.f;
        for (int zz = 0; zz < kz; ++zz) {
#pragma unroll
            for (int k = 0; k < SKE_ROWS; ++k)
                if (k < rows) g[k] += gp[zz * zs + k];
        }
        const bool real = col < n_sv;
        const float svs = real ? svsq[col] : 0.f;
#pragma unroll
        for (int k = 0; k < SKE_ROWS; ++k)
            if (k < rows) F[k][threadIdx.x] = real ? xsq[k0 + k] + svs - 2.f * gscale * g[k] : 0.f;
    }
    __syncthreads();
    const int valid = min(BN, n_sv - tile * BN);
    for (int k = warp; k < rows; k += nw) {
        float sum = 0.f;
        for (int i = lane; i < valid; i += 32) sum += F[k][i];
        for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, off);
        if (lane == 0) r_row[k] = sum / (float)max(valid, 1);
    }
    __syncthreads();
    for (int k = 0; k < rows; ++k) {
        const int i = threadIdx.x;
        F[k][i] = i < valid ? expm1_near0(-gamma * (F[k][i] - r_row[k])) : 0.f;
    }
    __syncthreads();
    for (int c0 = warp * SKE_CPW; c0 < C; c0 += nw * SKE_CPW) {
        float a[SKE_CPW][BN / 32];
#pragma unroll
        for (int cc = 0; cc < SKE_CPW; ++cc)
#pragma unroll
            for (int j = 0; j < BN / 32; ++j)
                a[cc][j] = c0 + cc < C ? coef[(size_t)(c0 + cc) * n_pad + tile * BN + lane + 32 * j] : 0.f;
        for (int k = 0; k < rows; ++k) {
            float sk[SKE_CPW];
#pragma unroll
            for (int cc = 0; cc < SKE_CPW; ++cc) {
                float t = 0.f;
#pragma unroll
                for (int j = 0; j < BN / 32; ++j) t = fmaf(F[k][lane + 32 * j], a[cc][j], t);
                sk[cc] = t;
            }
#pragma unroll
            for (int cc = 0; cc < SKE_CPW; ++cc)
                for (int off = 16; off > 0; off >>= 1) sk[cc] += __shfl_xor_sync(0xFFFFFFFFu, sk[cc], off);
            if (lane < SKE_CPW && c0 + lane < C) {
                float v = sk[0];
#pragma unroll
                for (int cc = 1; cc < SKE_CPW; ++cc) v = lane == cc ? sk[cc] : v;
                part[((size_t)tile * n + k0 + k) * C_pad + c0 + lane] = v;
            }
        }
    }
    if (threadIdx.x < rows) ref[(size_t)tile * n + k0 + threadIdx.x] = r_row[threadIdx.x];

    // ---- the last tile of this row group to finish adds the tiles ----
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(counters + blockIdx.y, 1u) == (uint32_t)nt - 1u;
    __syncthreads();
    if (!last) return;
    __threadfence();
    // shared memory (F reused): delta_s per row and tile, the tiles' coefficient sums when they
    // fit, then the scores of the group's rows
    float* s_del = &F[0][0];                       // [rows][nt] (nt <= 256)
    float* s_as = s_del + rows * nt;               // [nt][C] or unused
    const bool as_fit = rows * nt + nt * C + rows * C <= SKE_ROWS * BN;
    float* s_sc = as_fit ? s_as + nt * C : s_del + rows * nt;  // [rows][C]
    const bool sc_fit = (int)(s_sc - s_del) + rows * C <= SKE_ROWS * BN;
    for (int idx = threadIdx.x; idx < rows * nt; idx += SKE_THREADS) {
        const int k = idx / nt, t = idx - k * nt;
        s_del[idx] = t == 0 ? 0.f : expm1f(-gamma * (__ldcg(ref + (size_t)t * n + k0 + k) - __ldcg(ref + k0 + k)));
    }
    if (as_fit)
        for (int idx = threadIdx.x; idx < nt * C; idx += SKE_THREADS) {
            const int t = idx / C, c = idx - t * C;
            s_as[idx] = t == 0 ? 0.f : __ldg(asum_tile + (size_t)t * C_pad + c);
        }
    __syncthreads();
    // thread = (row, class), two of them at a time: the tiles' partial sums loaded 32 at a time
    // for both (one L2 round trip per chunk), then added in tile order
    const size_t ts = (size_t)n * C_pad;
    for (int i0 = threadIdx.x; i0 < rows * C; i0 += 2 * SKE_THREADS) {
        const int i1 = i0 + SKE_THREADS;
        const bool two = i1 < rows * C;
        const int ka = i0 / C, ca = i0 - ka * C;
        const int kb = two ? i1 / C : ka, cb = two ? i1 - kb * C : ca;
        const float* pa = part + (size_t)(k0 + ka) * C_pad + ca;
        const float* pb = part + (size_t)(k0 + kb) * C_pad + cb;
        float acc_a = 0.f, acc_b = 0.f;
        for (int t0 = 0; t0 < nt; t0 += 32) {
            float da[32], db[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                da[j] = t0 + j < nt ? __ldcg(pa + (t0 + j) * ts) : 0.f;
                db[j] = (two && t0 + j < nt) ? __ldcg(pb + (t0 + j) * ts) : 0.f;
            }
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                if (t0 + j < nt) {
                    const int t = t0 + j;
                    const float asa = as_fit ? s_as[t * C + ca] : (t == 0 ? 0.f : __ldg(asum_tile + (size_t)t * C_pad + ca));
                    const float asb = as_fit ? s_as[t * C + cb] : (t == 0 ? 0.f : __ldg(asum_tile + (size_t)t * C_pad + cb));
                    acc_a += da[j] + s_del[ka * nt + t] * (asa + da[j]);
                    acc_b += db[j] + s_del[kb * nt + t] * (asb + db[j]);
                }
            }
        }
        const float sa = expf(-gamma * __ldcg(ref + k0 + ka)) * (__ldg(asum + ca) + acc_a) + __ldg(bias + ca);
        scores[(size_t)(k0 + ka) * C + ca] = sa;
        if (sc_fit) s_sc[i0] = sa;
        if (two) {
            const float sb = expf(-gamma * __ldcg(ref + k0 + kb)) * (__ldg(asum + cb) + acc_b) + __ldg(bias + cb);
            scores[(size_t)(k0 + kb) * C + cb] = sb;
            if (sc_fit) s_sc[i1] = sb;
        }
    }
    if (!labels) return;
    __syncthreads();
    for (int k = warp; k < rows; k += nw) {
        float best = -INFINITY;
        int bi = 0x7FFFFFFF;
        for (int c = lane; c < C; c += 32) {
            const float v = sc_fit ? s_sc[k * C + c] : __ldcg(scores + (size_t)(k0 + k) * C + c);
            if (v > best) {
                best = v;
                bi = c;
            }
        }
        for (int off = 16; off > 0; off >>= 1) {
            const float ob = __shfl_xor_sync(0xFFFFFFFFu, best, off);
            const int oi = __shfl_xor_sync(0xFFFFFFFFu, bi, off);
            if (ob > best || (ob == best && oi < bi)) {
                best = ob;
                bi = oi;
            }
        }
        if (lane == 0) labels[k0 + k] = bi;
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
    // split bf16: the lo plane follows the hi plane (defaults to the hi maps otherwise)
    const void* lo = m->sv;
    if (m->dtype == RGBD_DT_BF16X3) lo = reinterpret_cast<const uint16_t*>(m->sv) + (size_t)m->n_pad * m->k_pad;
    rc = encode_tmap_2d(&m->tm_sv_lo, dt, lo, (uint64_t)m->k_pad, (uint64_t)m->n_pad, (uint64_t)m->k_pad * esz,
                        128u / esz, BN, CU_TENSOR_MAP_SWIZZLE_128B);
    if (rc) return rc;
    rc = encode_tmap_2d(&m->tm_sv_lo_half, dt, lo, (uint64_t)m->k_pad, (uint64_t)m->n_pad, (uint64_t)m->k_pad * esz,
                        128u / esz, BN / 2, CU_TENSOR_MAP_SWIZZLE_128B);
    if (rc) return rc;
    rc = encode_tmap_2d(&m->tm_coef, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, m->coef_bf16, (uint64_t)m->n_pad,
                        (uint64_t)m->C_pad, (uint64_t)m->n_pad * 2, 64u, (uint32_t)m->C_pad,
                        CU_TENSOR_MAP_SWIZZLE_128B);
    if (rc) return rc;
    rc = encode_tmap_2d(&m->tm_coef_half, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, m->coef_bf16, (uint64_t)m->n_pad,
                        (uint64_t)m->C_pad, (uint64_t)m->n_pad * 2, 64u, (uint32_t)m->C_pad / 2,
                        CU_TENSOR_MAP_SWIZZLE_128B);
    if (rc) return rc;
    // split bf16: the lo plane of the coefficients follows the hi plane (else the hi maps again)
    const uint16_t* coef_lo = m->coef_bf16;
    if (m->dtype == RGBD_DT_BF16X3) coef_lo += (size_t)m->C_pad * m->n_pad;
    rc = encode_tmap_2d(&m->tm_coef_lo, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, coef_lo, (uint64_t)m->n_pad,
                        (uint64_t)m->C_pad, (uint64_t)m->n_pad * 2, 64u, (uint32_t)m->C_pad,
                        CU_TENSOR_MAP_SWIZZLE_128B);
    if (rc) return rc;
    rc = encode_tmap_2d(&m->tm_coef_lo_half, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, coef_lo, (uint64_t)m->n_pad,
                        (uint64_t)m->C_pad, (uint64_t)m->n_pad * 2, 64u, (uint32_t)m->C_pad / 2,
                        CU_TENSOR_MAP_SWIZZLE_128B);
    if (rc) return rc;
    m->has_tmaps = true;
    return RGBD_OK;
}

namespace {

struct TcPlan {
    int esz, kind, passes, splits, tps, mt, nt;
    int kz, kpz;  // K ranges of the small-batch path (0: the tile kernel) and k-blocks per range
    uint32_t fmt;
    CUtensorMapDataType dt;
    size_t off_ref, off_cnt, off_gpart, bytes;  // (the small-batch path keeps its counters at off_cnt)
};

// ws_cap: the scratch a caller can offer; the small-batch path is planned only if it fits.
int plan_tc(rgbd_ctx* ctx, const rgbd_svm* m, int n, TcPlan* pl, size_t ws_cap = ~size_t(0)) {
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
    pl->passes = (m->dtype == RGBD_DT_BF16X3) ? 3 : 1;
    if (m->dtype == RGBD_DT_BF16X3) pl->kind = 3;  // split bf16, second product split too
    pl->mt = (n + BM - 1) / BM;
    pl->nt = m->n_pad / BN;
    // One 128-row block whose SV tiles cannot occupy half the SMs: split K instead (tuning value
    // 1 turns this off, >= 2 forces that many K ranges); every range holds >= 8 k-blocks.
    pl->kz = 0;
    pl->kpz = 0;
    if (pl->mt == 1 && pl->nt <= 256 && ctx->tune_tc_splitk != 1) {
        const int KT = pl->passes * (m->k_pad * pl->esz / 128);
        int kz = ctx->tune_tc_splitk >= 2 ? ctx->tune_tc_splitk
                                          : (2 * pl->nt <= ctx->props.sm_count ? ctx->props.sm_count / pl->nt : 0);
        // above 32 rows the partials' traffic (kz x n_pad x n floats, written and read back)
        // outweighs the wider spread: half the ranges measured faster at 64 and 128 rows
        if (ctx->tune_tc_splitk == 0 && n > 32) kz = std::max(2, kz / 2);
        kz = std::min(kz, std::max(1, KT / 8));
        if (kz >= 2) {
            pl->kpz = (KT + kz - 1) / kz;
            pl->kz = (KT + pl->kpz - 1) / pl->kpz;  // every range non-empty
            if (pl->kz < 2) pl->kz = 0;
        }
    }
    if (pl->kz) {
        // each SV tile is one split of the combine
        pl->splits = pl->nt;
        pl->tps = 1;
        const size_t part_bytes = sizeof(float) * (size_t)pl->nt * n * m->C_pad;
        const size_t ref_bytes = sizeof(float) * (size_t)pl->nt * n;
        pl->off_ref = (part_bytes + 255) & ~size_t(255);
        pl->off_cnt = (pl->off_ref + ref_bytes + 255) & ~size_t(255);
        pl->off_gpart = pl->off_cnt + 256;  // counters: one per group of SKE_ROWS rows (<= 8)
        pl->bytes = pl->off_gpart + sizeof(float) * (size_t)pl->kz * m->n_pad * n;
        if (pl->bytes <= ws_cap) return RGBD_OK;
        pl->kz = 0;  // too large for the caller's scratch: the tile kernel instead
    }
    pl->splits = ctx->tune_tc_splits > 0 ? std::min(ctx->tune_tc_splits, pl->nt)
                                         : choose_splits(pl->mt, pl->nt, ctx->props.sm_count);
    pl->tps = (pl->nt + pl->splits - 1) / pl->splits;
    pl->splits = (pl->nt + pl->tps - 1) / pl->tps;  // every split non-empty
    const size_t part_bytes = sizeof(float) * (size_t)pl->splits * n * m->C_pad;
    const size_t ref_bytes = sizeof(float) * (size_t)pl->splits * n;
    pl->off_ref = (part_bytes + 255) & ~size_t(255);
    pl->off_cnt = (pl->off_ref + ref_bytes + 255) & ~size_t(255);
    pl->bytes = pl->off_cnt + sizeof(uint32_t) * (size_t)((pl->mt + 1) / 2 * 2);  // one counter per row block
    pl->off_gpart = 0;
    return RGBD_OK;
}

// The small-batch path: K-range partials of G, their per-tile epilogue, the split combine.
template <int KIND>
cudaError_t launch_splitk(const TcPlan& pl, const SkParams& sp, const rgbd_svm* m, const CUtensorMap& tm_x,
                          const CUtensorMap& tm_x2, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(rbf_tc_splitk_kernel<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         SK_SMEM);
    if (e != cudaSuccess) return e;
    rbf_tc_splitk_kernel<KIND><<<dim3((unsigned)pl.nt, (unsigned)pl.kz), SK_WARPS * 32, SK_SMEM, s>>>(
        tm_x, m->tm_sv, tm_x2, m->tm_sv_lo, sp);
    return cudaGetLastError();
}

// Launches one instantiation: single CTAs on a (row blocks, splits) grid, pairs as clusters of
// two along the rows (the row-block count rounded up to even).
template <int MODE, int KIND>
cudaError_t launch_mode(const TcPlan& pl, const TcParams& p, const rgbd_svm* m, const CUtensorMap& tm_x,
                        const CUtensorMap& tm_x2, cudaStream_t s) {
    constexpr int smem = Lay<MODE, KIND == 3>::SMEM;
    cudaError_t e = cudaFuncSetAttribute(rbf_tc_kernel<MODE, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    if (MODE == MODE_SINGLE) {
        dim3 grid(pl.mt, pl.splits);
        rbf_tc_kernel<MODE, KIND><<<grid, NUM_THREADS, smem, s>>>(tm_x, m->tm_sv, m->tm_coef, tm_x2, m->tm_sv_lo,
                                                                  m->tm_coef_lo, p);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((pl.mt + 1) / 2 * 2), (unsigned)pl.splits, 1);
    cfg.blockDim = dim3(NUM_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, rbf_tc_kernel<MODE, KIND>, tm_x, m->tm_sv_half,
                              MODE == MODE_PAIR ? m->tm_coef_half : m->tm_coef, tm_x2, m->tm_sv_lo_half,
                              MODE == MODE_PAIR ? m->tm_coef_lo_half : m->tm_coef_lo, p);
}

int launch_tc(rgbd_ctx* ctx, const rgbd_svm* m, const void* x, const float* xsq, int n, float x_scale,
              float* scores, int32_t* labels, cudaStream_t s, const TcPlan& pl, char* ws) {
    float* part = (float*)ws;
    float* ref = (float*)(ws + pl.off_ref);
    CUtensorMap tm_x, tm_x2;
    const float gscale = (m->dtype == RGBD_DT_FP8) ? 1.0f / (x_scale * m->sv_scale) : 1.0f;
    // the small-batch path copies only the batch's rows of X (a multiple of 8)
    const uint32_t x_rows = pl.kz ? (uint32_t)std::min(BM, (n + 7) & ~7) : (uint32_t)BM;
    int rc = encode_tmap_2d(&tm_x, pl.dt, x, (uint64_t)m->k_pad, (uint64_t)n, (uint64_t)m->k_pad * pl.esz,
                            128u / pl.esz, x_rows, CU_TENSOR_MAP_SWIZZLE_128B);
    if (rc) return rc;
    const void* x_lo = x;  // split bf16: the lo plane of the rows follows their hi plane
    if (pl.passes == 3) x_lo = reinterpret_cast<const uint16_t*>(x) + (size_t)n * m->k_pad;
    rc = encode_tmap_2d(&tm_x2, pl.dt, x_lo, (uint64_t)m->k_pad, (uint64_t)n, (uint64_t)m->k_pad * pl.esz,
                        128u / pl.esz, x_rows, CU_TENSOR_MAP_SWIZZLE_128B);
    if (rc) return rc;
    if (pl.kz) {
        SkParams sp;
        sp.n = n;
        sp.n_pad = m->n_pad;
        sp.k_blocks = m->k_pad * pl.esz / 128;
        sp.k_elems = 128 / pl.esz;
        sp.passes = pl.passes;
        sp.kpz = pl.kpz;
        sp.x_bytes = x_rows * 128u;
        sp.idesc = make_idesc(pl.fmt, pl.fmt, BM, BN);
        sp.gpart = (float*)(ws + pl.off_gpart);
        sp.counters = reinterpret_cast<uint32_t*>(ws + pl.off_cnt);
        sp.n_groups = (n + SKE_ROWS - 1) / SKE_ROWS;
        sp.status = ctx->d_status;
        cudaError_t e;
        switch (pl.kind) {
            case 0: e = launch_splitk<0>(pl, sp, m, tm_x, tm_x2, s); break;
            case 1: e = launch_splitk<1>(pl, sp, m, tm_x, tm_x2, s); break;
            case 2: e = launch_splitk<2>(pl, sp, m, tm_x, tm_x2, s); break;
            default: e = launch_splitk<3>(pl, sp, m, tm_x, tm_x2, s); break;
        }
        if (e != cudaSuccess) return cuda_error(e, "svm_score: split-K launch");
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)pl.nt, (unsigned)sp.n_groups, 1);
        cfg.blockDim = dim3(SKE_THREADS, 1, 1);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, rbf_splitk_epilogue_kernel, (const float*)sp.gpart, pl.kz, m->n_pad, n, xsq,
                               (const float*)m->sv_sq, m->n_sv, (const float*)m->coef, m->C, m->C_pad, m->gamma,
                               gscale, part, ref, sp.counters, pl.nt, (const float*)m->asum,
                               (const float*)m->asum_tile, (const float*)m->bias, scores, labels);
        if (e != cudaSuccess) return cuda_error(e, "svm_score: split-K epilogue launch");
        return RGBD_OK;
    }
    // Mode: tuning value 2 = single CTAs, 3 = 2-CTA MMA pairs, 0 = auto (the 2-CTA pairs).
    // Pairs need at least two 128-row blocks.
    int mode = MODE_SINGLE;
    if (pl.mt >= 2) mode = (ctx->tune_tc_pairing == 2) ? MODE_SINGLE : MODE_PAIR;
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
    p.gscale = gscale;
    p.xsq = xsq;
    p.svsq = m->sv_sq;
    p.part = part;
    p.ref = ref;
    p.status = ctx->d_status;
    const int mma_m = mode == MODE_PAIR ? 2 * BM : BM;  // a pair's MMA covers both CTAs' rows
    p.idesc_main = make_idesc(pl.fmt, pl.fmt, mma_m, BN);
    p.idesc_second = make_idesc(1, 1, mma_m, m->C_pad);
    p.passes = pl.passes;
    // Small batches (up to 8 row blocks) combine their splits inside the kernel, in the last CTA
    // of each row block to finish, which saves a launch on the latency path of a serving batch;
    // larger ones leave it to the split-combine kernel, which spreads the work over every SM instead
    // of adding a tail to the last CTAs (on the 4096-row batch the fused combine cost ~9 us more).
    // The combine also needs its shared memory to fit the ring (every mode's holds >= 140 KB).
    p.fuse = (pl.mt <= 8 && combine_bytes(pl.splits, m->C_pad) <= (size_t)140 * 1024) ? 1 : 0;
    p.counters = reinterpret_cast<uint32_t*>(ws + pl.off_cnt);
    p.asum = m->asum;
    p.asum_tile = m->asum_tile;
    p.bias = m->bias;
    p.scores = scores;
    p.labels = labels;
    if (p.fuse) {
        const cudaError_t ez =
            cudaMemsetAsync(p.counters, 0, sizeof(uint32_t) * (size_t)((pl.mt + 1) / 2 * 2), s);
        if (ez != cudaSuccess) return cuda_error(ez, "svm_score: split counters");
    }
    cudaError_t e;
    switch (mode * 4 + pl.kind) {
        case MODE_SINGLE * 4 + 0: e = launch_mode<MODE_SINGLE, 0>(pl, p, m, tm_x, tm_x2, s); break;
        case MODE_SINGLE * 4 + 1: e = launch_mode<MODE_SINGLE, 1>(pl, p, m, tm_x, tm_x2, s); break;
        case MODE_SINGLE * 4 + 2: e = launch_mode<MODE_SINGLE, 2>(pl, p, m, tm_x, tm_x2, s); break;
        case MODE_SINGLE * 4 + 3: e = launch_mode<MODE_SINGLE, 3>(pl, p, m, tm_x, tm_x2, s); break;
        case MODE_PAIR * 4 + 0: e = launch_mode<MODE_PAIR, 0>(pl, p, m, tm_x, tm_x2, s); break;
        case MODE_PAIR * 4 + 1: e = launch_mode<MODE_PAIR, 1>(pl, p, m, tm_x, tm_x2, s); break;
        case MODE_PAIR * 4 + 2: e = launch_mode<MODE_PAIR, 2>(pl, p, m, tm_x, tm_x2, s); break;
        default: e = launch_mode<MODE_PAIR, 3>(pl, p, m, tm_x, tm_x2, s); break;
    }
    if (e != cudaSuccess) return cuda_error(e, "svm_score: tc launch");
    if (p.fuse) return RGBD_OK;
    return launch_reduce_scores(part, ref, pl.splits, n, m->C, m->C_pad, m->asum, m->asum_tile, pl.tps, pl.nt,
                                m->bias, m->gamma, scores, labels, s);
}

// The bounded wait of the scoring kernel on a barrier phase that nothing completes: after
// `limit_ns` it flags RGBD_STATUS_WAIT_TIMEOUT and returns (the path every stalled wait takes).
__global__ void wait_probe_kernel(uint32_t* status, uint64_t limit_ns, int* waited_out) {
    __shared__ __align__(8) uint64_t barrier;
    __shared__ int abort_flag;
    const uint32_t b = smem_u32(&barrier);
    bar_init(b, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    const bool ok = bar_wait<false>(b, 0, &abort_flag, status, limit_ns);
    *waited_out = ok ? 0 : (abort_flag ? 1 : 2);
}

__global__ void expm1_probe_kernel(const float* __restrict__ z, float* __restrict__ out, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = expm1_near0(z[i]);
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

size_t score_rbf_tc_bytes(rgbd_ctx* ctx, const rgbd_svm* m, int n) {
    TcPlan pl;
    return plan_tc(ctx, m, n, &pl) ? 0 : pl.bytes;
}

int score_rbf_tc_external_ws(rgbd_ctx* ctx, const rgbd_svm* m, const void* x, const float* xsq, int n,
                             float x_scale, float* scores, int32_t* labels, cudaStream_t s, void* ws_ptr,
                             size_t ws_cap, size_t* need) {
    TcPlan pl;
    int rc = plan_tc(ctx, m, n, &pl, ws_cap);
    if (rc) return rc;
    if (need) *need = pl.bytes;
    if (pl.bytes > ws_cap)
        return set_error(RGBD_ERR_ARG, "scratch of %zu bytes needed for %d rows, %d classes, %d splits; only %zu available",
                         pl.bytes, n, m->C, pl.splits, ws_cap);
    return launch_tc(ctx, m, x, xsq, n, x_scale, scores, labels, s, pl, (char*)ws_ptr);
}

}  // namespace rgbd

extern "C" int rgbd_debug_expm1(const float* z, float* out, int n, void* stream) {
    using namespace rgbd;
    if (n < 0 || (n > 0 && (!z || !out))) return set_error(RGBD_ERR_ARG, "rgbd_debug_expm1: n %d, z %p, out %p", n, z, out);
    if (n == 0) return RGBD_OK;
    expm1_probe_kernel<<<std::min((n + 255) / 256, 1024), 256, 0, (cudaStream_t)stream>>>(z, out, n);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? RGBD_OK : cuda_error(e, "rgbd_debug_expm1");
}

extern "C" int rgbd_debug_wait_timeout(rgbd_ctx* ctx, uint64_t limit_ns, int* result, void* stream) {
    using namespace rgbd;
    if (!ctx || !result) return set_error(RGBD_ERR_ARG, "rgbd_debug_wait_timeout: NULL pointer");
    if (limit_ns < 1000 || limit_ns > 100000000ull)
        return set_error(RGBD_ERR_ARG, "rgbd_debug_wait_timeout: limit %llu ns (1 us .. 100 ms)",
                         (unsigned long long)limit_ns);
    DeviceGuard g(ctx->props.device);
    wait_probe_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(ctx->d_status, limit_ns, result);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? RGBD_OK : cuda_error(e, "rgbd_debug_wait_timeout");
}
