// lbp.cu -- steps A1..A5 of the hot path on sm_103a:
//   A1 affine crop of each face rect (Section 2.1, Eq. 1; Section 3 resizes every face),
//   A2 median-depth mask (the depth/grey fusion of Sections 1 and 2.5),
//   A3 8-neighbour radius-1 LBP codes (Section 2.4, Eq. 2, Fig. 7),
//   A4 per-cell uniform-pattern histograms (Section 2.4, Eq. 3; Section 3),
//   A5 per-cell normalisation (and bf16 / FP8 quantisation) of the feature rows.
//
// The fused kernel is persistent: one CTA per half-SM slot walks over faces.  Per face:
//   P1  every thread resamples 8 groups of 4 crop pixels (grey bilinear, depth nearest;
//       for rects at most 2 S wide the grey taps of two neighbouring pixels come from one
//       aligned 8-byte window per source row, and each horizontal interpolation is one byte
//       permute and one 4-way byte dot product); grey and depth go to shared memory (the
//       depths share their space with the P5 histograms) and the depths are counted into a
//       coarse histogram of 1024 mm bins (eight 8-bit counters per thread in one 64-bit word,
//       summed over the warp with redux).
//   P2/P3  radix select of the lower median: the coarse bin holding rank (n-1)/2, then a
//       1 mm histogram restricted to that bin (bins are of d - 1, so holes fall outside).
//   P4  mask bytes (0x80 = valid) from the depths.
//   P5  one thread per half cell (4 x 8 pixels) walks down its 8 rows with a
//       3-row sliding window of packed words and computes four codes per step
//       with byte-SIMD compares; codes go through the uniform table into a
//       thread-private 8-bit histogram (no atomics, no bank conflicts).  Under the
//       default rule an invalid centre compares as grey 255 and so has code 0; P6
//       subtracts the cell's invalid centres from bin 0.
//   P6/P7  half-cell histograms are summed into a uint16 staging row, which is
//       written out coalesced together with the normalised row and its norm (bf16 rows
//       read each quotient h / n from a per-CTA table of the 65 x 65 possible values).
//       P7 first asks L2 for the next face's source rows (its rect was copied in during P5),
//       so that face's P1 gathers find them there.
// Everything up to A4 is exact integer arithmetic.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>

#include "internal.h"

namespace rgbd {
namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;

// ---------------------------------------------------------------------------------------
// A1 helpers: Q16.16 source coordinates, pixel centre to pixel centre.
// ---------------------------------------------------------------------------------------

// origin + (i + 1/2) * len / out_len - 1/2 in Q16.16 (len > 0, so the quotient is >= 0).
__device__ __forceinline__ int64_t rect_coord_q16(int origin, int len, int out_len, int i) {
    uint64_t num = (uint64_t)(2 * i + 1) * (uint64_t)len * 65536ull;
    return (int64_t)origin * 65536 + (int64_t)(num / (2ull * (uint64_t)out_len)) - 32768;
}

// Packs the taps of one coordinate: .x = a | (b - a) << 16 | frac << 24 (bilinear: clamped
// taps a = floor, b = floor + 1, Q8 fraction), .y = the clamped nearest index.
__device__ __forceinline__ uint2 make_tap(int64_t q, int lim) {
    const int64_t f0 = q >> 16;  // floor (arithmetic shift)
    const int frac = (int)((q >> 8) & 255);
    const int64_t nn = (q + 32768) >> 16;
    const int64_t hi = (int64_t)lim - 1;
    const int a = (int)(f0 < 0 ? 0 : (f0 > hi ? hi : f0));
    const int b = (int)(f0 + 1 < 0 ? 0 : (f0 + 1 > hi ? hi : f0 + 1));
    const int n = (int)(nn < 0 ? 0 : (nn > hi ? hi : nn));
    return make_uint2((uint32_t)a | ((uint32_t)(b - a) << 16) | ((uint32_t)frac << 24), (uint32_t)n);
}

// Asks L2 for the source rows of a face rect (grey and depth, each row's span widened by one
// pixel for the bilinear taps and clamped to the frame): one prefetch per 128 bytes, every
// address inside its row's span.  Threads pair up per row: even threads take the grey span,
// odd ones the depth span.
__device__ __forceinline__ void prefetch_rect_rows(const uint8_t* grey, const uint16_t* depth, int H, int W,
                                                   const rgbd_rect& rn, int tid, int nt) {
    const int x0 = max(rn.x - 1, 0), x1 = min(rn.x + rn.w + 1, W);
    const int y0 = max(rn.y - 1, 0), y1 = min(rn.y + rn.h + 1, H);
    if (x1 <= x0 || y1 <= y0) return;
    const size_t plane = (size_t)H * W;
    const bool dep = tid & 1;
    const uint8_t* base = dep ? reinterpret_cast<const uint8_t*>(depth + (size_t)rn.frame * plane)
                              : grey + (size_t)rn.frame * plane;
    const size_t esz = dep ? 2 : 1;
    for (int y = y0 + (tid >> 1); y < y1; y += nt >> 1) {
        const uint8_t* first = base + ((size_t)y * W + x0) * esz;
        const uint8_t* last = base + ((size_t)y * W + x1) * esz - 1;
        for (const uint8_t* pp = first;; pp += 128) {
            asm volatile("prefetch.global.L2 [%0];" ::"l"(pp < last ? pp : last));
            if (pp >= last - 127) break;
        }
    }
}

// Bilinear grey sample with Q8 weights (they sum to 2^16), rounded half up.
__device__ __forceinline__ uint32_t bilerp(const uint8_t* img, int W, uint32_t cx, uint32_t ry) {
    const uint32_t xa = cx & 0xFFFFu, dx = (cx >> 16) & 1u, fx = cx >> 24;
    const uint32_t ya = ry & 0xFFFFu, dy = (ry >> 16) & 1u, fy = ry >> 24;
    const uint8_t* r0 = img + (size_t)ya * W + xa;
    const uint8_t* r1 = r0 + (size_t)dy * W;
    const uint32_t p00 = __ldg(r0), p01 = __ldg(r0 + dx);
    const uint32_t p10 = __ldg(r1), p11 = __ldg(r1 + dx);
    const uint32_t acc = (256u - fy) * ((256u - fx) * p00 + fx * p01) + fy * ((256u - fx) * p10 + fx * p11);
    return (acc + 32768u) >> 16;
}

// ---------------------------------------------------------------------------------------
// A3 helper: byte-SIMD "a > b" (or >=) on four packed pixels.  cb = (b & 0x7f7f7f7f) + 1 per
// byte for the strict test, without the +1 for >=.  Result: 0x80 in each byte where it holds.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t cmp_msb(uint32_t a, uint32_t b, uint32_t cb) {
    const uint32_t d = (a | 0x80808080u) - cb;  // per byte: low 7 bits of a vs b, no borrows
    return ((a & ~b) | (~(a ^ b) & d)) & 0x80808080u;
}

// Slot of quotient-table entry i = 128 n + h: bits 1..5 of h are XOR-ed with the low bits of n.
// A warp's lanes read values of several cells at once; without the XOR the table's rows are
// 64 words apart, so equal counts h of different cells fall into the same bank.  The XOR stays
// inside the row of n.
__device__ __forceinline__ int qbf_slot(int i) { return i ^ (((i >> 7) & 31) << 1); }
// The same for two 16-bit indices (count | centres << 7) packed in one word.
__device__ __forceinline__ uint32_t qbf_slot2(uint32_t w) { return w ^ ((w >> 6) & 0x003E003Eu); }

// Tile shape of the fused kernel: TPC threads per 8 x 8 cell (2: one per 4 x 8 half cell, 1: one
// per cell, 4: one per 4 x 4 quarter cell), so a CTA of NT = TPC (S/8)^2 threads works on one
// face; each thread resamples IPT groups of 4 crop pixels.  Four threads per cell make 1024-thread
// CTAs for 128 x 128 crops: one per SM, twice the warps on a face.
template <int S, int TPC = 2>
struct Cfg {
    static constexpr int G = S / 8;          // cells per side
    static constexpr int NT = TPC * G * G;   // threads
    static constexpr int SW = S / 4;         // packed words per crop row
    static constexpr int IPT = S * S / 4 / NT;  // 4-pixel groups per thread
    static constexpr int DIM = G * G * kBins;
    static constexpr int HW = 15;            // histogram words per thread (60 bins / 4)
    static constexpr int MINB = (S == 128 && TPC <= 2) ? 2 : 1;
    static constexpr int RPT = TPC == 4 ? 4 : 8;        // cell rows a thread walks in P5
    static constexpr int WPT = (HW + TPC - 1) / TPC;    // histogram words a thread stages in P6
    static_assert(TPC == 1 || TPC == 2 || TPC == 4, "one, two or four threads per cell");
};

template <int S, int TPC = 2>
struct __align__(16) Smem {
    // grey words with a one-word / one-row clamp-to-edge border ((S + 2) rows of S / 4 + 2
    // words), then mask words; later the uint16 staging row
    uint32_t img[(S + 2) * (S / 4 + 2) + S * S / 4];
    union {
        uint32_t hist[Cfg<S, TPC>::HW * Cfg<S, TPC>::NT];  // P5-P6: thread-private 8-bit counts, word (bin/4)*NT + t
        uint32_t dep[S * S / 2];                 // P1-P4: the crop's depths, two per word, by item
    };
    uint2 colmap[S];                   // taps per crop column, read two at a time (uint4)
    uint2 rowmap[S];                   // taps per crop row
    unsigned long long ctab[65];       // coarse-histogram increment per key of d - 1 (64: a hole)
    uint16_t ncol[S];                  // nearest depth column per crop column (colmap order)
    uint32_t h1[64];                   // coarse depth histogram: key (d - 1) >> 10 (1024 mm bins)
    uint32_t h2[1024];                 // fine histogram ((d - 1) & 1023) inside the median's coarse bin
    uint32_t cnt[Cfg<S, TPC>::NT];     // valid centres per thread (half cell or cell)
    float nvf[Cfg<S>::G * Cfg<S>::G];  // valid centres per cell (as float) ...
    float rcp[Cfg<S>::G * Cfg<S>::G];  // ... and its IEEE reciprocal (0 for an empty cell)
    float red[Cfg<S, TPC>::NT / 32];
    uint32_t wsum[Cfg<S, TPC>::NT / 32];  // per-warp totals of the fine median histogram
    uint32_t sink[32];                 // target of the border stores of non-edge lanes
    int info[4];
    rgbd_rect nrect;                   // the next face's rect, copied in during the current face
    uint16_t lut[257];                 // byte offset of each code's counter in a thread's histogram
                                       // (entry 256: the unused bin 59, where invalid centres go
                                       // under the rules other than the default one)
    uint16_t qbf[65 * 128];            // bf16 bits of the quotient h / n, entry 128 n + h (n, h <= 64)
};

template <int S, int TPC>
__global__ void __launch_bounds__(Cfg<S, TPC>::NT, Cfg<S, TPC>::MINB) lbp_fused_kernel(LbpArgs a) {
    using C = Cfg<S, TPC>;
    constexpr int IPT = C::IPT;
    constexpr int NT = C::NT, SW = C::SW, G = C::G, DIM = C::DIM;
    constexpr int SP = SW + 2;               // words per row of the bordered grey plane
    constexpr int MW_OFF = (S + 2) * SP;     // the mask plane follows it
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<S, TPC>& sm = *reinterpret_cast<Smem<S, TPC>*>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // Uniform-pattern table: code c is uniform when it has at most two 0/1 changes around the
    // ring; uniform codes are ranked in ascending order (0..57), all others share bin 58.
    if (warp == 0) {
        int prefix = 0;
        for (int r = 0; r < 8; ++r) {
            const int c = r * 32 + lane;
            const int rot = ((c << 1) | (c >> 7)) & 0xFF;
            const bool uni = __popc(c ^ rot) <= 2;
            const unsigned m = __ballot_sync(FULL, uni);
            const int rank = prefix + __popc(m & ((1u << lane) - 1u));
            const int bin = uni ? rank : 58;
            // counters of one thread: byte (bin & 3) of word (bin / 4) * NT + thread
            sm.lut[c] = (uint16_t)(((bin >> 2) * NT) * 4 + (bin & 3));
            prefix += __popc(m);
        }
        if (lane == 0) sm.lut[256] = (uint16_t)(((59 >> 2) * NT) * 4 + (59 & 3));
    }
    // Quotient table of the bf16 output: a cell has at most 64 centres, so every normalised value
    // is one of the 65 x 65 quotients h / n (stored at qbf_slot(128 n + h)), computed once per
    // CTA exactly as the other output
    // types compute them (IEEE single quotient by the reciprocal and Markstein's one-fma
    // correction, then round to nearest even bf16).  Entry
    // 128 n + h, so that a staged count with its cell's centre count above it is the index.
    for (int i = tid; i < 65 * 128; i += NT) {
        const int n = i >> 7, hh = min(i & 127, 64);
        const float n_f = (float)n, r_f = n ? __frcp_rn(n_f) : 0.f, h_f = (float)hh;
        const float q0 = __fmul_rn(h_f, r_f);
        const float rem = __fmaf_rn(-q0, n_f, h_f);
        sm.qbf[qbf_slot(i)] = __bfloat16_as_ushort(__float2bfloat16_rn(__fmaf_rn(rem, r_f, q0)));
    }

    for (int i = tid; i < 65; i += NT) sm.ctab[i] = i < 8 ? 1ull << (8 * i) : 0ull;

    const bool strict = !(a.flags & RGBD_LBP_GE);
    const bool nbr_ignore = (a.flags & RGBD_LBP_NBR_IGNORE_MASK) != 0;
    const bool masked_grey = strict && !nbr_ignore;  // the default rule (readings c2, c7)
    const int x_dtype = a.x_out ? a.x_dtype : 0;

    // Faces: the first one by CTA index, then from the launch's queue counter (a CTA that
    // finishes early takes the next face), or strided over the CTAs when there is no counter.
    for (int face = blockIdx.x; face < a.n;) {
        __syncthreads();  // the previous face's output pass is done with shared memory

        // ---- P0: descriptor, tap maps, cleared histograms --------------------------------
        bool ok = true;
        rgbd_rect r = {0, 0, 0, S, S};
        bool pair_win = false;  // grey taps read as 8-byte windows (rects at most 2 S wide)
        const uint8_t* gsrc = a.grey;
        const uint16_t* dsrc = a.depth;
        int64_t aff[6] = {0, 0, 0, 0, 0, 0};
        if (a.rects) {
            r = face == (int)blockIdx.x ? a.rects[face] : sm.nrect;
            ok = r.frame >= 0 && r.frame < a.n_frames && r.w > 0 && r.h > 0;
            if (!ok && tid == 0) atomicOr(a.status, RGBD_STATUS_BAD_RECT);
            if (ok) {
                gsrc += (size_t)r.frame * a.H * a.W;
                dsrc += (size_t)r.frame * a.H * a.W;
                pair_win = !a.affine && r.w <= 2 * S && (a.W & 3) == 0 && a.W >= 8 &&
                           (reinterpret_cast<size_t>(a.grey) & 3) == 0;
            }
            if (ok && a.affine) {
#pragma unroll
                for (int i = 0; i < 6; ++i) aff[i] = a.affine[6 * (size_t)face + i];
            } else if (ok) {
                for (int i = tid; i < 2 * S; i += NT) {
                    if (i < S) {
                        uint2 t = make_tap(rect_coord_q16(r.x, r.w, S, i), a.W);
                        const int ci = (((i & 3) >> 1) * SW + (i >> 2)) * 2 + (i & 1);
                        if (pair_win) {
                            // grey taps of the column pair (4q + 2j, 4q + 2j + 1) inside one aligned
                            // 8-byte window starting at wb: .x = byte selector (o, o + dx, o) | wb << 16,
                            // .y = byte weights (255 - fx, fx, 1, 0), so that one byte permute and one
                            // 4-way byte dot product give 256 p(o) + fx (p(o + dx) - p(o)).
                            // The pair's first column is the previous lane (column threads form
                            // whole warps: S is a multiple of 32).  With at most 2 S source columns
                            // for S crop columns, neighbouring taps are at most 2 apart, so
                            // o, o + dx <= 7 (the window start is clamped to W - 8).
                            const uint32_t x_prev = __shfl_up_sync(FULL, t.x, 1);
                            const uint32_t x_first = (i & 1) ? x_prev : t.x;
                            const uint32_t wb = min((x_first & 0xFFFCu), (uint32_t)a.W - 8u);
                            const uint32_t xa = t.x & 0xFFFFu, dx = (t.x >> 16) & 1u, fx = t.x >> 24;
                            const uint32_t o = xa - wb, od = xa + dx - wb;
                            sm.ncol[ci] = (uint16_t)t.y;
                            t = make_uint2(o | (od << 4) | (o << 8) | (wb << 16), (255u - fx) | (fx << 8) | (1u << 16));
                        }
                        // column u = 4q + e lives at uint2 index ((e / 2) * SW + q) * 2 + e % 2
                        sm.colmap[ci] = t;
                    } else {
                        const int v = i - S;
                        sm.rowmap[v] = make_tap(rect_coord_q16(r.y, r.h, S, v), a.H);
                    }
                }
            }
        } else {
            gsrc += (size_t)face * S * S;
            dsrc += (size_t)face * S * S;
        }
        for (int i = tid; i < 1024; i += NT) {
            if (i < 64) sm.h1[i] = 0;
            sm.h2[i] = 0;
        }
        __syncthreads();

        // ---- P1: resample; grey and depth to shared memory, coarse depth histogram ----------
        // One group of 4 pixels per iteration, not unrolled: each group's gathers are
        // independent, other warps hide their latency, and the rolled loop keeps the group's
        // registers free of spills (unrolled, the loop ran 4.5 % slower at 64 registers).
        // The next face is claimed now (the atomic's latency hides behind P1) and published at
        // the end of P1; its rect is copied into shared memory asynchronously during P5.
        int next_face = 0;
        if (tid == 0)
            next_face = a.face_counter ? (int)gridDim.x + (int)atomicAdd(a.face_counter, 1u) : face + (int)gridDim.x;
        unsigned long long cnt8 = 0;  // coarse depth histogram, see below
#pragma unroll 1
        for (int k = 0; k < IPT; ++k) {
            const int item = tid + k * NT;  // = v * SW + q
            const int v = item / SW, q = item - v * SW;
            uint32_t gw = 0, d01 = 0, d23 = 0;
            if (ok) {
                if (!a.rects) {
                    gw = __ldg(reinterpret_cast<const uint32_t*>(gsrc) + item);
                    const uint2 dd = __ldg(reinterpret_cast<const uint2*>(dsrc) + item);
                    d01 = dd.x;
                    d23 = dd.y;
                } else if (!a.affine) {
                    const uint2 rm = sm.rowmap[v];
                    const uint32_t fy = rm.x >> 24;
                    const uint8_t* g0 = gsrc + (size_t)(rm.x & 0xFFFFu) * a.W;
                    const uint8_t* g1 = g0 + (size_t)((rm.x >> 16) & 1u) * a.W;
                    const uint16_t* drow = dsrc + (size_t)rm.y * a.W;
                    const uint4* cm4 = reinterpret_cast<const uint4*>(sm.colmap);
                    uint32_t dv[4];
                    uint32_t accv[4];  // pair windows: (acc + 2^15) per pixel, the rounded value in byte 2
                    if (pair_win) {
#pragma unroll
                    for (int e2 = 0; e2 < 2; ++e2) {
                        const uint4 cc = cm4[e2 * SW + q];  // taps of columns 4q + 2 e2 and + 1
                        const uint32_t nn = reinterpret_cast<const uint32_t*>(sm.ncol)[e2 * SW + q];
                        const uint32_t wb = cc.x >> 16;
                        const uint32_t* wa = reinterpret_cast<const uint32_t*>(g0 + wb);
                        const uint32_t* wv = reinterpret_cast<const uint32_t*>(g1 + wb);
                        const uint32_t a0 = __ldg(wa), a1 = __ldg(wa + 1), b0 = __ldg(wv), b1 = __ldg(wv + 1);
#pragma unroll
                        for (int j = 0; j < 2; ++j) {
                            const uint32_t sel = j ? cc.z : cc.x, wts = j ? cc.w : cc.y;
                            // h = 256 p0 + fx (p1 - p0) for the two source rows, then
                            // (256 - fy) h0 + fy h1 = 256 h0 + fy (h1 - h0), exactly
                            const uint32_t h0 = __dp4a(__byte_perm(a0, a1, sel), wts, 0u);
                            const uint32_t h1 = __dp4a(__byte_perm(b0, b1, sel), wts, 0u);
                            const int e = 2 * e2 + j;
                            accv[e] = h0 * (256u - fy) + (h1 * fy + 32768u);  // < 2^24
                            dv[e] = __ldg(drow + (j ? (nn >> 16) : (nn & 0xFFFFu)));
                        }
                    }
                    // byte 2 of each rounded sum is the pixel: gather the four with byte permutes
                    gw = __byte_perm(__byte_perm(accv[0], accv[1], 0x0062u), __byte_perm(accv[2], accv[3], 0x0062u),
                                     0x5410u);
                    } else {
#pragma unroll
                    for (int e2 = 0; e2 < 2; ++e2) {
                        const uint4 cc = cm4[e2 * SW + q];  // taps of columns 4q + 2 e2 and + 1
#pragma unroll
                        for (int j = 0; j < 2; ++j) {
                            const uint32_t cx = j ? cc.z : cc.x;
                            const uint32_t xa = cx & 0xFFFFu, dx = (cx >> 16) & 1u;
                            const int fx = (int)(cx >> 24);
                            const int p00 = __ldg(g0 + xa), p01 = __ldg(g0 + xa + dx);
                            const int p10 = __ldg(g1 + xa), p11 = __ldg(g1 + xa + dx);
                            // (256 - f) a + f b = 256 a + f (b - a), exactly
                            const int h0 = (p00 << 8) + fx * (p01 - p00);
                            const int h1 = (p10 << 8) + fx * (p11 - p10);
                            const int acc = (h0 << 8) + (int)fy * (h1 - h0);
                            const int e = 2 * e2 + j;
                            gw |= (uint32_t)((acc + 32768) >> 16) << (8 * e);
                            dv[e] = __ldg(drow + (j ? cc.w : cc.y));
                        }
                    }
                    }
                    d01 = dv[0] | (dv[1] << 16);
                    d23 = dv[2] | (dv[3] << 16);
                } else {
                    uint32_t dv[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int u = 4 * q + e;
                        const int64_t xq = aff[0] * u + aff[1] * v + aff[2];
                        const int64_t yq = aff[3] * u + aff[4] * v + aff[5];
                        const uint2 tx = make_tap(xq, a.W), ty = make_tap(yq, a.H);
                        gw |= bilerp(gsrc, a.W, tx.x, ty.x) << (8 * e);
                        dv[e] = __ldg(dsrc + (size_t)ty.y * a.W + tx.y);
                    }
                    d01 = dv[0] | (dv[1] << 16);
                    d23 = dv[2] | (dv[3] << 16);
                }
            }
            sm.img[(v + 1) * SP + q + 1] = gw;
            reinterpret_cast<uint2*>(sm.dep)[item] = make_uint2(d01, d23);
#pragma unroll
            for (int hh = 0; hh < 4; ++hh) {
                const uint32_t d = ((hh < 2 ? d01 : d23) >> (16 * (hh & 1))) & 0xFFFFu;
                const uint32_t key = min((d - 1u) >> 10, 64u);  // a hole (d = 0) wraps to 64
                cnt8 += sm.ctab[key];
                if (key - 8u < 56u) atomicAdd(&sm.h1[key], 1u);
            }
        }
        {
            // coarse histogram of the non-zero depths, keyed by (d - 1) >> 10 (bins of 1024 mm;
            // any monotone key serves the select, and this one needs no test for holes): a thread
            // holds 4 IPT <= 64 depths, so eight 8-bit counters in one 64-bit word count keys 0..7
            // (depths up to 8192 mm), added from a table; the warp sums them as 16-bit fields (at
            // most 2048 each) and lane 0 adds them to the histogram.  Rarer, larger depths count
            // with atomics.
            const unsigned long long ev = cnt8 & 0x00FF00FF00FF00FFull;          // keys 0, 2, 4, 6
            const unsigned long long od = (cnt8 >> 8) & 0x00FF00FF00FF00FFull;   // keys 1, 3, 5, 7
            const uint32_t s02 = __reduce_add_sync(FULL, (uint32_t)ev);
            const uint32_t s46 = __reduce_add_sync(FULL, (uint32_t)(ev >> 32));
            const uint32_t s13 = __reduce_add_sync(FULL, (uint32_t)od);
            const uint32_t s57 = __reduce_add_sync(FULL, (uint32_t)(od >> 32));
            if (lane == 0) {
                const uint32_t c8[8] = {s02 & 0xFFFFu, s13 & 0xFFFFu, s02 >> 16, s13 >> 16,
                                        s46 & 0xFFFFu, s57 & 0xFFFFu, s46 >> 16, s57 >> 16};
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    if (c8[k]) atomicAdd(&sm.h1[k], c8[k]);
            }
        }
        if (tid == 0) sm.info[3] = next_face;
        __syncthreads();

        // ---- P2: coarse bin of the lower median (rank (n-1)/2 of the non-zero depths) -----
        if (warp == 0) {
            uint32_t s8[2], lsum = 0;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                s8[j] = sm.h1[lane * 2 + j];
                lsum += s8[j];
            }
            uint32_t incl = lsum;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const uint32_t t = __shfl_up_sync(FULL, incl, off);
                if (lane >= off) incl += t;
            }
            const uint32_t total = __shfl_sync(FULL, incl, 31);
            int b1 = -1, k1 = 0;
            if (total > 0) {
                const uint32_t k = (total - 1) / 2;
                const uint32_t excl = incl - lsum;
                const unsigned m = __ballot_sync(FULL, k >= excl && k < incl);
                const int src = __ffs(m) - 1;
                if (lane == src) {
                    uint32_t c = excl;
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        if (b1 < 0 && k < c + s8[j]) {
                            b1 = lane * 2 + j;
                            k1 = (int)(k - c);
                        }
                        c += s8[j];
                    }
                }
                b1 = __shfl_sync(FULL, b1, src);
                k1 = __shfl_sync(FULL, k1, src);
            }
            if (lane == 0) {
                sm.info[0] = b1;
                sm.info[1] = k1;
            }
        }
        __syncthreads();
        const int b1 = sm.info[0];

        // ---- P3: the median's value inside coarse bin b1 (1 mm bins) ----------------------
        int med = -1;
        if (b1 >= 0) {
#pragma unroll
            for (int i = 0; i < 2 * IPT; ++i) {
                const uint32_t dw = sm.dep[2 * (tid + (i >> 1) * NT) + (i & 1)];
                const uint32_t lo = dw & 0xFFFFu, hi = dw >> 16;
                if (((lo - 1u) >> 10) == (uint32_t)b1) atomicAdd(&sm.h2[(lo - 1u) & 1023u], 1u);
                if (((hi - 1u) >> 10) == (uint32_t)b1) atomicAdd(&sm.h2[(hi - 1u) & 1023u], 1u);
            }
            __syncthreads();
            // rank k1 among the 1024 fine bins: every thread sums its 1024 / NT contiguous bins,
            // the warps scan their threads, every thread adds the totals of the warps before its
            // own, and the one thread whose bins hold rank k1 walks them
            constexpr int BPT = (1024 + NT - 1) / NT;
            const uint32_t k1 = (uint32_t)sm.info[1];
            uint32_t lsum = 0;
#pragma unroll
            for (int j = 0; j < BPT; ++j)
                if (tid * BPT + j < 1024) lsum += sm.h2[tid * BPT + j];
            uint32_t incl = lsum;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const uint32_t t = __shfl_up_sync(FULL, incl, off);
                if (lane >= off) incl += t;
            }
            if (lane == 31) sm.wsum[warp] = incl;
            __syncthreads();
            uint32_t base = 0;
            for (int w = 0; w < warp; ++w) base += sm.wsum[w];
            const uint32_t excl = base + incl - lsum;
            if (k1 >= excl && k1 < excl + lsum) {
                uint32_t c = excl;
                int b2 = -1;
#pragma unroll
                for (int j = 0; j < BPT; ++j) {
                    const uint32_t hj = tid * BPT + j < 1024 ? sm.h2[tid * BPT + j] : 0u;
                    if (b2 < 0 && k1 < c + hj) b2 = tid * BPT + j;
                    c += hj;
                }
                sm.info[2] = b1 * 1024 + b2 + 1;  // keys are of d - 1
            }
            __syncthreads();
            med = sm.info[2];
        }

        // ---- P4: depth mask, 0x80 per valid pixel ----------------------------------------
        {
            uint32_t* mw = sm.img + MW_OFF;
            // d != 0 and |d - med| < mask  <=>  d - lo < width as unsigned numbers, with
            // lo = max(med - mask + 1, 1) (a hole wraps around) and width = med + mask - lo, or 0
            // when there is no median (all |d - med| < 65536, so the mask is capped there)
            const int mk = min(a.mask_mm, 65536);
            const int lo_i = max(med - mk + 1, 1);
            const uint32_t lo = (uint32_t)lo_i;
            const uint32_t width = (med >= 0 && med + mk > lo_i) ? (uint32_t)(med + mk - lo_i) : 0u;
#pragma unroll
            for (int k = 0; k < IPT; ++k) {
                uint32_t m = 0;
                const uint2 dd = reinterpret_cast<const uint2*>(sm.dep)[tid + k * NT];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const uint32_t d = ((e < 2 ? dd.x : dd.y) >> (16 * (e & 1))) & 0xFFFFu;
                    m |= (d - lo < width) ? (0x80u << (8 * e)) : 0u;
                }
                mw[tid + k * NT] = m;
                const int item = tid + k * NT, v = item / SW, q = item - v * SW;
                uint32_t* gp = sm.img + (v + 1) * SP + q + 1;
                uint32_t g = *gp;
                // strict compares with masked neighbours: a grey of 0 never compares greater, so
                // zeroing the invalid pixels once replaces the per-neighbour masks of P5
                if (masked_grey) {
                    g &= (m >> 7) * 0xFFu;
                    *gp = g;
                }
                // the border repeats the edge pixels (clamp-to-edge neighbours); branch-free:
                // lanes away from the left and right edges store into a sink word
                {
                    const bool le = q == 0, re = q == SW - 1;
                    uint32_t* side = le ? gp - 1 : (re ? gp + 1 : sm.sink + lane);
                    const uint32_t pv = le ? (g << 24) : (g >> 24);
                    *side = pv;
                    if (v == 0 || v == S - 1) {  // the border rows
                        const int dv = v == 0 ? -SP : SP;
                        gp[dv] = g;
                        *((le || re) ? side + dv : sm.sink + lane) = pv;  // corner words
                    }
                }
            }
        }
        __syncthreads();

        // ---- P5: LBP codes and private histograms, one half cell per thread ---------------
        if (tid == 0 && a.rects && sm.info[3] < a.n) {
            const int* src = reinterpret_cast<const int*>(a.rects + sm.info[3]);
            const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&sm.nrect);
#pragma unroll
            for (int i = 0; i < 5; ++i)
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst + 4u * i), "l"(src + i) : "memory");
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
#pragma unroll
        for (int w = 0; w < C::HW; ++w) sm.hist[w * NT + tid] = 0;  // (the depths are no longer needed)
        {
            // the thread's half cell (TPC = 2), both halves of its cell in turn (TPC = 1), or a
            // quarter: the upper or lower four rows of a half (TPC = 4)
            const int c = tid / TPC;
            const int cy = c / G, cx = c - cy * G;
            const int r0 = 8 * cy + (TPC == 4 ? 4 * ((tid >> 1) & 1) : 0);
            constexpr int RPT = C::RPT;
            const uint32_t* GW = sm.img;
            const uint32_t* MW = sm.img + MW_OFF;
            uint32_t nvalid = 0;
            uint8_t* hb_t = reinterpret_cast<uint8_t*>(sm.hist) + 4 * tid;  // this thread's counters
#pragma unroll 1
            for (int hh = 0; hh < (TPC == 1 ? 2 : 1); ++hh) {
            const int h = TPC == 1 ? hh : (tid & 1);
            const int wc = 2 * cx + h;
            const bool le = wc == 0, re = wc == SW - 1;
            const int wl = le ? wc : wc - 1, wr = re ? wc : wc + 1;
            // Words holding pixels (x-1 .. x+2), (x .. x+3), (x+1 .. x+4) of a row; past the crop
            // edge a neighbour repeats the edge pixel (the grey plane's border holds the repeats).
            auto row3g = [&](int row, uint32_t& L, uint32_t& M, uint32_t& R) {
                const uint32_t* p = GW + (row + 1) * SP + wc + 1;
                const uint32_t c0 = p[0];
                L = __byte_perm(p[-1], c0, 0x6543);
                M = c0;
                R = __byte_perm(c0, p[1], 0x4321);
            };
            auto row3 = [&](const uint32_t* base, int row, uint32_t& L, uint32_t& M, uint32_t& R) {
                row = min(max(row, 0), S - 1);
                const uint32_t* p = base + row * SW;
                const uint32_t c0 = p[wc];
                const uint32_t l0 = le ? (c0 << 24) : p[wl];
                const uint32_t r1 = re ? (c0 >> 24) : p[wr];
                L = __byte_perm(l0, c0, 0x6543);
                M = c0;
                R = __byte_perm(c0, r1, 0x4321);
            };
            uint32_t gUL, gUC, gUR, gCL, gCC, gCR, gDL, gDC, gDR;
            if (masked_grey) {
                // invalid pixels read as grey 0 (P4): no neighbour masks, only the centre's
                row3g(r0 - 1, gUL, gUC, gUR);
                row3g(r0, gCL, gCC, gCR);
#pragma unroll 2
                for (int i = 0; i < RPT; ++i) {
                    row3g(r0 + i + 1, gDL, gDC, gDR);
                    const uint32_t mC = MW[(r0 + i) * SW + wc];
                    // an invalid centre compares as grey 255, so no neighbour is greater and its
                    // code is 0; P6 takes the invalid centres back out of bin U(0) = 0
                    const uint32_t inv = ~mC & 0x80808080u;
                    const uint32_t gc = gCC | inv | (inv - (inv >> 7));
                    const uint32_t cb = (gc & 0x7F7F7F7Fu) + 0x01010101u;
                    const uint32_t code = (cmp_msb(gUL, gc, cb) >> 7) | (cmp_msb(gUC, gc, cb) >> 6) |
                                          (cmp_msb(gUR, gc, cb) >> 5) | (cmp_msb(gCR, gc, cb) >> 4) |
                                          (cmp_msb(gDR, gc, cb) >> 3) | (cmp_msb(gDC, gc, cb) >> 2) |
                                          (cmp_msb(gDL, gc, cb) >> 1) | cmp_msb(gCL, gc, cb);
                    nvalid += __popc(mC);
#pragma unroll
                    for (int e = 0; e < 4; ++e) hb_t[sm.lut[(code >> (8 * e)) & 0xFFu]] += 1;
                    gUL = gCL; gUC = gCC; gUR = gCR; gCL = gDL; gCC = gDC; gCR = gDR;
                }
            } else {
            uint32_t mUL, mUC, mUR, mCL, mCC, mCR, mDL, mDC, mDR;
            row3g(r0 - 1, gUL, gUC, gUR);
            row3(MW, r0 - 1, mUL, mUC, mUR);
            row3g(r0, gCL, gCC, gCR);
            row3(MW, r0, mCL, mCC, mCR);
#pragma unroll 2
            for (int i = 0; i < RPT; ++i) {
                row3g(r0 + i + 1, gDL, gDC, gDR);
                row3(MW, r0 + i + 1, mDL, mDC, mDR);
                const uint32_t NM = 0x80808080u;
                const uint32_t cb = (gCC & 0x7F7F7F7Fu) + (strict ? 0x01010101u : 0u);
                const uint32_t code =
                    ((cmp_msb(gUL, gCC, cb) & (nbr_ignore ? NM : mUL)) >> 7) |
                    ((cmp_msb(gUC, gCC, cb) & (nbr_ignore ? NM : mUC)) >> 6) |
                    ((cmp_msb(gUR, gCC, cb) & (nbr_ignore ? NM : mUR)) >> 5) |
                    ((cmp_msb(gCR, gCC, cb) & (nbr_ignore ? NM : mCR)) >> 4) |
                    ((cmp_msb(gDR, gCC, cb) & (nbr_ignore ? NM : mDR)) >> 3) |
                    ((cmp_msb(gDC, gCC, cb) & (nbr_ignore ? NM : mDC)) >> 2) |
                    ((cmp_msb(gDL, gCC, cb) & (nbr_ignore ? NM : mDL)) >> 1) |
                    (cmp_msb(gCL, gCC, cb) & (nbr_ignore ? NM : mCL));
                // branch-free: an invalid centre counts into the unused bin 59
                nvalid += __popc(mCC);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const uint32_t idx = ((mCC >> (8 * e + 7)) & 1u) ? ((code >> (8 * e)) & 0xFFu) : 256u;
                    hb_t[sm.lut[idx]] += 1;
                }
                gUL = gCL; gUC = gCC; gUR = gCR; gCL = gDL; gCC = gDC; gCR = gDR;
                mUL = mCL; mUC = mCC; mUR = mCR; mCL = mDL; mCC = mDC; mCR = mDR;
            }
            }
            }
            sm.cnt[tid] = nvalid;
        }
        if (tid == 0 && a.rects) asm volatile("cp.async.wait_all;" ::: "memory");  // the next rect has landed
        __syncthreads();

        // ---- P6: each cell's histogram (the sum of its two halves) into a uint16 staging row
        uint16_t* stg = reinterpret_cast<uint16_t*>(sm.img);
        {
            // TPC = 2: the two threads of a cell split its words; TPC = 1: one thread per cell;
            // TPC = 4: four threads split them (C::WPT each) and add the four partial histograms
            // byte by byte (a byte holds at most 64 counts in all)
            const int c = tid / TPC, h = TPC == 1 ? 0 : (tid & (TPC - 1));
            uint32_t nv = TPC == 1 ? sm.cnt[c] : sm.cnt[TPC * c] + sm.cnt[TPC * c + 1];
            if (TPC == 4) nv += sm.cnt[TPC * c + 2] + sm.cnt[TPC * c + 3];
            if (h == 0) {
                sm.nvf[c] = (float)nv;
                sm.rcp[c] = nv ? __frcp_rn((float)nv) : 0.f;
            }
            const int w0 = TPC == 4 ? h * C::WPT : (h ? 8 : 0);
            const int w1 = TPC == 4 ? min(C::HW, w0 + C::WPT) : ((h || TPC == 1) ? C::HW : 8);
#pragma unroll 1  // rolled: 0.7 % faster than the compiler's unrolling
            for (int w = w0; w < w1; ++w) {
                uint32_t s = TPC == 1 ? sm.hist[w * NT + c] : sm.hist[w * NT + TPC * c] + sm.hist[w * NT + TPC * c + 1];
                if (TPC == 4) s += sm.hist[w * NT + TPC * c + 2] + sm.hist[w * NT + TPC * c + 3];
                if (masked_grey && w == 0) s -= 64u - nv;  // the invalid centres counted as code 0
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int b = 4 * w + e;
                    // the count (<= 64) with the cell's valid centres above it: the index of
                    // its quotient in qbf
                    if (b < kBins) stg[c * kBins + b] = (uint16_t)(((s >> (8 * e)) & 0xFFu) | (nv << 7));
                }
            }
        }
        __syncthreads();

        // ---- P7: coalesced output of counts, normalised row and its squared norm ----------
        // first ask L2 for the next face's source rows, a face ahead of its P1 gathers
        if (a.rects && !a.affine && sm.info[3] < a.n) {
            const rgbd_rect rn = sm.nrect;
            if (rn.frame >= 0 && rn.frame < a.n_frames && rn.w > 0 && rn.h > 0)
                prefetch_rect_rows(a.grey, a.depth, a.H, a.W, rn, tid, NT);
        }
        float sq = 0.f;
        const bool centred = a.x_centre != nullptr;
        const bool wide = x_dtype == RGBD_DT_BF16 && !centred && (a.k_pad & 7) == 0 && (DIM & 7) == 0 &&
                          ((reinterpret_cast<size_t>(a.feats) | reinterpret_cast<size_t>(a.x_out)) & 15) == 0;
        if (wide) {
            // bf16 rows, 8 values per thread step (16-byte loads and stores)
            for (int j8 = tid; j8 < a.k_pad / 8; j8 += NT) {
                const int j = 8 * j8;
                uint4 hv = make_uint4(0u, 0u, 0u, 0u);
                uint32_t pk[4] = {0u, 0u, 0u, 0u};
                if (j < DIM) {
                    hv = *reinterpret_cast<const uint4*>(stg + j);
                    if (a.feats)
                        *reinterpret_cast<uint4*>(a.feats + (size_t)face * DIM + j) =
                            make_uint4(hv.x & 0x007F007Fu, hv.y & 0x007F007Fu, hv.z & 0x007F007Fu, hv.w & 0x007F007Fu);
                    const uint32_t hw[4] = {qbf_slot2(hv.x), qbf_slot2(hv.y), qbf_slot2(hv.z), qbf_slot2(hv.w)};
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const uint32_t qb = sm.qbf[(hw[e >> 1] >> (16 * (e & 1))) & 0xFFFFu];
                        const float f = __uint_as_float(qb << 16);
                        sq = fmaf(f, f, sq);
                        pk[e >> 1] |= qb << (16 * (e & 1));
                    }
                }
                *reinterpret_cast<uint4*>(reinterpret_cast<uint16_t*>(a.x_out) + (size_t)face * a.k_pad + j) =
                    make_uint4(pk[0], pk[1], pk[2], pk[3]);
            }
        }
        const int len4 = wide ? 0 : (x_dtype ? a.k_pad : DIM) / 4;
        for (int j4 = tid; j4 < len4; j4 += NT) {
            const int j = 4 * j4;
            uint2 hv = make_uint2(0, 0);
            if (j < DIM) {
                hv = *reinterpret_cast<const uint2*>(stg + j);
                if (a.feats)
                    *reinterpret_cast<uint2*>(a.feats + (size_t)face * DIM + j) =
                        make_uint2(hv.x & 0x007F007Fu, hv.y & 0x007F007Fu);
            }
            if (x_dtype == RGBD_DT_BF16 && !centred) {
                // bf16 rows: one table read per value
                uint32_t pk[2] = {0u, 0u};
                if (j < DIM) {
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const uint32_t qb = sm.qbf[(qbf_slot2(e < 2 ? hv.x : hv.y) >> (16 * (e & 1))) & 0xFFFFu];
                        const float f = __uint_as_float(qb << 16);
                        sq = fmaf(f, f, sq);
                        pk[e >> 1] |= qb << (16 * (e & 1));
                    }
                }
                *reinterpret_cast<uint2*>(reinterpret_cast<uint16_t*>(a.x_out) + (size_t)face * a.k_pad + j) =
                    make_uint2(pk[0], pk[1]);
            } else if (x_dtype) {
                // x = h / n as the IEEE single quotient: q0 = h * (1/n), then Markstein's
                // correction step (P. Markstein, IBM J. Res. Dev. 34(1), 1990): the remainder
                // r = h - q0 n exactly by one fma, then q = q0 + r (1/n) rounded once.  For
                // 0 <= h <= n <= 64 (a cell has 64 pixels) this reproduces div.rn exactly
                // (checked exhaustively); an empty cell has h = 0 and rcp = 0, giving 0.
                float x[4] = {0.f, 0.f, 0.f, 0.f};
                if (j < DIM) {  // DIM is a multiple of 4, so the whole group is inside
                    const int c0 = j / kBins;
                    const int split = (c0 + 1) * kBins;  // first index of the next cell
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int cc = (j + e < split) ? c0 : c0 + 1;
                        const float n_f = sm.nvf[cc], r_f = sm.rcp[cc];
                        const float h_f = (float)(((e < 2 ? hv.x : hv.y) >> (16 * (e & 1))) & 0x7Fu);
                        const float q0 = __fmul_rn(h_f, r_f);
                        const float rem = __fmaf_rn(-q0, n_f, h_f);
                        x[e] = __fmaf_rn(rem, r_f, q0);
                    }
                    if (centred) {  // x - mu, one fp32 rounding
                        const float4 mu = *reinterpret_cast<const float4*>(a.x_centre + j);
                        x[0] = __fsub_rn(x[0], mu.x);
                        x[1] = __fsub_rn(x[1], mu.y);
                        x[2] = __fsub_rn(x[2], mu.z);
                        x[3] = __fsub_rn(x[3], mu.w);
                    }
                }
                if (x_dtype == RGBD_DT_BF16) {  // centred bf16 rows (round to nearest even)
                    uint32_t pk[2] = {0u, 0u};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const __nv_bfloat16 q = __float2bfloat16_rn(x[e]);
                        const float f = __bfloat162float(q);
                        sq = fmaf(f, f, sq);
                        pk[e >> 1] |= (uint32_t)__bfloat16_as_ushort(q) << (16 * (e & 1));
                    }
                    *reinterpret_cast<uint2*>(reinterpret_cast<uint16_t*>(a.x_out) + (size_t)face * a.k_pad + j) =
                        make_uint2(pk[0], pk[1]);
                } else if (x_dtype == RGBD_DT_BF16X3) {
                    // hi = bf16(x) into the first plane, lo = bf16(x - hi) into the second
                    uint32_t ph[2], pl[2];
#pragma unroll
                    for (int e = 0; e < 4; e += 2) {
                        const __nv_bfloat16 h0 = __float2bfloat16_rn(x[e]), h1 = __float2bfloat16_rn(x[e + 1]);
                        const float hf0 = __bfloat162float(h0), hf1 = __bfloat162float(h1);
                        const __nv_bfloat16 l0 = __float2bfloat16_rn(x[e] - hf0);
                        const __nv_bfloat16 l1 = __float2bfloat16_rn(x[e + 1] - hf1);
                        const float v0 = hf0 + __bfloat162float(l0), v1 = hf1 + __bfloat162float(l1);
                        sq = fmaf(v0, v0, sq);
                        sq = fmaf(v1, v1, sq);
                        ph[e >> 1] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
                        pl[e >> 1] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
                    }
                    uint16_t* xb = reinterpret_cast<uint16_t*>(a.x_out) + (size_t)face * a.k_pad + j;
                    *reinterpret_cast<uint2*>(xb) = make_uint2(ph[0], ph[1]);
                    *reinterpret_cast<uint2*>(xb + a.x_plane) = make_uint2(pl[0], pl[1]);
                } else if (x_dtype == RGBD_DT_FP8) {
                    uint32_t pk = 0;
                    const float inv = 1.0f / a.x_scale;
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const __nv_fp8_e4m3 q8(x[e] * a.x_scale);
                        const float f = static_cast<float>(q8) * inv;
                        sq = fmaf(f, f, sq);
                        pk |= (uint32_t)q8.__x << (8 * e);
                    }
                    *reinterpret_cast<uint32_t*>(reinterpret_cast<uint8_t*>(a.x_out) +
                                                 (size_t)face * a.k_pad + j) = pk;
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e) sq = fmaf(x[e], x[e], sq);
                    *reinterpret_cast<float4*>(reinterpret_cast<float*>(a.x_out) +
                                               (size_t)face * a.k_pad + j) =
                        make_float4(x[0], x[1], x[2], x[3]);
                }
            }
        }
        if (a.xsq) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) sq += __shfl_xor_sync(FULL, sq, off);
            if (lane == 0) sm.red[warp] = sq;
            __syncthreads();
            if (tid == 0) {
                float t = 0.f;
                for (int w = 0; w < NT / 32; ++w) t += sm.red[w];
                a.xsq[face] = t;
            }
        }
        __syncthreads();
        face = sm.info[3];
    }
}

// ---------------------------------------------------------------------------------------
// Section 3's own descriptor: one 0-255 histogram of the raw LBP codes per face (crop up to
// 255 x 255; the paper uses 200 x 200).  Same resample, median mask and codes as the fused
// kernel, written plainly (one pixel per thread step): this is the paper-literal variant, not
// the throughput path.  One CTA of 1024 threads per face, persistent over faces.
// ---------------------------------------------------------------------------------------
constexpr int F256_THREADS = 1024;
constexpr int F256_COPIES = 8;  // histogram copies (warp % 8) to spread same-code atomics

__global__ void __launch_bounds__(F256_THREADS, 1) lbp_face256_kernel(LbpArgs a) {
    const int S = a.crop, SS = S * S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint16_t* depth = reinterpret_cast<uint16_t*>(smem_raw);           // [SS], later the mask bytes
    uint8_t* grey = smem_raw + 2 * ((SS + 7) & ~7);                     // [SS]
    uint32_t* hist = reinterpret_cast<uint32_t*>(grey + ((SS + 15) & ~15));  // [COPIES][256]
    uint2* colmap = reinterpret_cast<uint2*>(hist + F256_COPIES * 256);     // [S]
    uint2* rowmap = colmap + S;                                             // [S]
    uint32_t* h1 = reinterpret_cast<uint32_t*>(rowmap + S);                 // [256]
    uint32_t* h2 = h1 + 256;                                                // [256]
    int* info = reinterpret_cast<int*>(h2 + 256);                           // [4]
    float* red = reinterpret_cast<float*>(info + 4);                        // [32]
    uint8_t* mask = reinterpret_cast<uint8_t*>(depth);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool strict = !(a.flags & RGBD_LBP_GE);
    const bool nbr_ignore = (a.flags & RGBD_LBP_NBR_IGNORE_MASK) != 0;
    const int x_dtype = a.x_out ? a.x_dtype : 0;
    const int iters = (SS + F256_THREADS - 1) / F256_THREADS;

    for (int face = blockIdx.x; face < a.n; face += gridDim.x) {
        __syncthreads();
        bool ok = true;
        rgbd_rect r = {0, 0, 0, S, S};
        const uint8_t* gsrc = a.grey;
        const uint16_t* dsrc = a.depth;
        int64_t aff[6] = {0, 0, 0, 0, 0, 0};
        if (a.rects) {
            r = a.rects[face];
            ok = r.frame >= 0 && r.frame < a.n_frames && r.w > 0 && r.h > 0;
            if (!ok && tid == 0) atomicOr(a.status, RGBD_STATUS_BAD_RECT);
            if (ok) {
                gsrc += (size_t)r.frame * a.H * a.W;
                dsrc += (size_t)r.frame * a.H * a.W;
                if (a.affine) {
                    for (int i = 0; i < 6; ++i) aff[i] = a.affine[6 * (size_t)face + i];
                } else {
                    for (int i = tid; i < 2 * S; i += F256_THREADS) {
                        if (i < S)
                            colmap[i] = make_tap(rect_coord_q16(r.x, r.w, S, i), a.W);
                        else
                            rowmap[i - S] = make_tap(rect_coord_q16(r.y, r.h, S, i - S), a.H);
                    }
                }
            }
        } else {
            gsrc += (size_t)face * SS;
            dsrc += (size_t)face * SS;
        }
        for (int i = tid; i < F256_COPIES * 256; i += F256_THREADS) hist[i] = 0;
        for (int i = tid; i < 256; i += F256_THREADS) {
            h1[i] = 0;
            h2[i] = 0;
        }
        __syncthreads();
        // resample and the depth high-byte histogram
        for (int it = 0; it < iters; ++it) {
            const int pidx = tid + it * F256_THREADS;
            uint32_t d = 0;
            if (pidx < SS && ok) {
                const int v = pidx / S, u = pidx - v * S;
                uint32_t g;
                if (!a.rects) {
                    g = gsrc[pidx];
                    d = dsrc[pidx];
                } else if (!a.affine) {
                    const uint2 tx = colmap[u], ty = rowmap[v];
                    g = bilerp(gsrc, a.W, tx.x, ty.x);
                    d = __ldg(dsrc + (size_t)ty.y * a.W + tx.y);
                } else {
                    const int64_t xq = aff[0] * u + aff[1] * v + aff[2];
                    const int64_t yq = aff[3] * u + aff[4] * v + aff[5];
                    const uint2 tx = make_tap(xq, a.W), ty = make_tap(yq, a.H);
                    g = bilerp(gsrc, a.W, tx.x, ty.x);
                    d = __ldg(dsrc + (size_t)ty.y * a.W + tx.y);
                }
                grey[pidx] = (uint8_t)g;
            }
            if (pidx < SS) depth[pidx] = (uint16_t)d;
            if (d) atomicAdd(&h1[d >> 8], 1u);
        }
        __syncthreads();
        // lower median of the non-zero depths (radix select over the high, then low byte)
        if (warp == 0) {
            uint32_t c = 0;
            for (int i = lane; i < 256; i += 32) c += h1[i];
            for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(FULL, c, off);
            if (lane == 0) {
                int b1 = -1, k1 = 0;
                if (c > 0) {
                    const uint32_t k = (c - 1) / 2;
                    uint32_t acc = 0;
                    for (int b = 0; b < 256; ++b) {
                        if (k < acc + h1[b]) {
                            b1 = b;
                            k1 = (int)(k - acc);
                            break;
                        }
                        acc += h1[b];
                    }
                }
                info[0] = b1;
                info[1] = k1;
            }
        }
        __syncthreads();
        const int b1 = info[0];
        int med = -1;
        if (b1 >= 0) {
            for (int pidx = tid; pidx < SS; pidx += F256_THREADS) {
                const uint32_t d = depth[pidx];
                if (d && (int)(d >> 8) == b1) atomicAdd(&h2[d & 255u], 1u);
            }
            __syncthreads();
            if (tid == 0) {
                const uint32_t k1 = (uint32_t)info[1];
                uint32_t acc = 0;
                int b2 = 0;
                for (int b = 0; b < 256; ++b) {
                    if (k1 < acc + h2[b]) {
                        b2 = b;
                        break;
                    }
                    acc += h2[b];
                }
                info[2] = b1 * 256 + b2;
            }
            __syncthreads();
            med = info[2];
        }
        // mask: valid bits to registers first, then bytes over the depth buffer
        uint32_t vbits[4] = {0, 0, 0, 0};  // up to 128 pixels per thread (255^2 / 1024 < 64)
        for (int it = 0; it < iters; ++it) {
            const int pidx = tid + it * F256_THREADS;
            if (pidx < SS) {
                const int d = depth[pidx];
                const int diff = d - med;
                if (med >= 0 && d != 0 && diff < a.mask_mm && -diff < a.mask_mm) vbits[it >> 5] |= 1u << (it & 31);
            }
        }
        __syncthreads();
        for (int it = 0; it < iters; ++it) {
            const int pidx = tid + it * F256_THREADS;
            if (pidx < SS) mask[pidx] = (uint8_t)((vbits[it >> 5] >> (it & 31)) & 1u);
        }
        __syncthreads();
        // codes and the 0-255 histogram
        uint32_t* myh = hist + (warp % F256_COPIES) * 256;
        for (int pidx = tid; pidx < SS; pidx += F256_THREADS) {
            if (!mask[pidx]) continue;
            const int i = pidx / S, j = pidx - i * S;
            const int gc = grey[pidx];
            int code = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                // ring p0..p7 clockwise from the top-left neighbour, y down
                const int dx = (q == 0 || q == 6 || q == 7) ? -1 : ((q == 1 || q == 5) ? 0 : 1);
                const int dy = (q <= 2) ? -1 : ((q == 3 || q == 7) ? 0 : 1);
                const int rr = min(max(i + dy, 0), S - 1), cc = min(max(j + dx, 0), S - 1);
                const int gp = grey[rr * S + cc];
                const bool nb = nbr_ignore || mask[rr * S + cc];
                if (nb && (strict ? gp > gc : gp >= gc)) code |= 1 << q;
            }
            atomicAdd(&myh[code], 1u);
        }
        __syncthreads();
        // merge the copies, write counts, the normalised row and its squared norm
        uint32_t cnt = 0;
        if (tid < 256) {
            for (int k = 0; k < F256_COPIES; ++k) cnt += hist[k * 256 + tid];
            hist[tid] = cnt;  // copy 0 now holds the totals (each thread owns its bin)
        }
        __syncthreads();
        if (warp == 0) {
            uint32_t t = 0;
            for (int i = lane; i < 256; i += 32) t += hist[i];
            for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(FULL, t, off);
            if (lane == 0) info[3] = (int)t;
        }
        __syncthreads();
        const uint32_t nvalid = (uint32_t)info[3];
        float sq = 0.f;
        const int len = x_dtype ? a.k_pad : 256;
        for (int j = tid; j < len; j += F256_THREADS) {
            const uint32_t h = j < 256 ? hist[j] : 0u;
            if (j < 256 && a.feats) a.feats[(size_t)face * 256 + j] = (uint16_t)h;
            if (x_dtype) {
                float x = (j < 256 && nvalid) ? (float)h / (float)nvalid : 0.f;
                if (a.x_centre && j < 256) x = __fsub_rn(x, a.x_centre[j]);
                const size_t idx = (size_t)face * a.k_pad + j;
                float qv = x;
                if (x_dtype == RGBD_DT_BF16) {
                    const __nv_bfloat16 b = __float2bfloat16_rn(x);
                    reinterpret_cast<uint16_t*>(a.x_out)[idx] = __bfloat16_as_ushort(b);
                    qv = __bfloat162float(b);
                } else if (x_dtype == RGBD_DT_BF16X3) {
                    const __nv_bfloat16 hi = __float2bfloat16_rn(x);
                    const __nv_bfloat16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
                    reinterpret_cast<uint16_t*>(a.x_out)[idx] = __bfloat16_as_ushort(hi);
                    reinterpret_cast<uint16_t*>(a.x_out)[idx + a.x_plane] = __bfloat16_as_ushort(lo);
                    qv = __bfloat162float(hi) + __bfloat162float(lo);
                } else if (x_dtype == RGBD_DT_FP8) {
                    const __nv_fp8_e4m3 b(x * a.x_scale);
                    reinterpret_cast<uint8_t*>(a.x_out)[idx] = b.__x;
                    qv = static_cast<float>(b) * (1.0f / a.x_scale);
                } else {
                    reinterpret_cast<float*>(a.x_out)[idx] = x;
                }
                sq = fmaf(qv, qv, sq);
            }
        }
        if (a.xsq) {
            for (int off = 16; off > 0; off >>= 1) sq += __shfl_xor_sync(FULL, sq, off);
            if (lane == 0) red[warp] = sq;
            __syncthreads();
            if (tid == 0) {
                float t = 0.f;
                for (int w = 0; w < F256_THREADS / 32; ++w) t += red[w];
                a.xsq[face] = t;
            }
        }
    }
}

size_t face256_smem(int S) {
    const size_t SS = (size_t)S * S;
    return 2 * ((SS + 7) & ~size_t(7)) + ((SS + 15) & ~size_t(15)) + 4 * F256_COPIES * 256 + 2 * 8 * (size_t)S +
           4 * 512 + 16 + 4 * 32;
}

// ---------------------------------------------------------------------------------------
// Plain crop (rgbd_crop_affine): one thread per crop pixel.
// ---------------------------------------------------------------------------------------
__global__ void crop_affine_kernel(const uint8_t* __restrict__ grey, const uint16_t* __restrict__ depth,
                                   int n_frames, int H, int W, const rgbd_rect* __restrict__ rects,
                                   const int32_t* __restrict__ affine, int n, int oh, int ow,
                                   uint8_t* __restrict__ og, uint16_t* __restrict__ od,
                                   uint32_t* status) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= oh * ow) return;
    const int v = p / ow, u = p - v * ow;
    for (int k = blockIdx.y; k < n; k += gridDim.y) {
        const rgbd_rect r = rects[k];
        const size_t o = (size_t)k * oh * ow + p;
        if (!(r.frame >= 0 && r.frame < n_frames && r.w > 0 && r.h > 0)) {
            og[o] = 0;
            od[o] = 0;
            if (p == 0) atomicOr(status, RGBD_STATUS_BAD_RECT);
            continue;
        }
        int64_t xq, yq;
        if (affine) {
            const int32_t* m = affine + 6 * (size_t)k;
            xq = (int64_t)m[0] * u + (int64_t)m[1] * v + m[2];
            yq = (int64_t)m[3] * u + (int64_t)m[4] * v + m[5];
        } else {
            xq = rect_coord_q16(r.x, r.w, ow, u);
            yq = rect_coord_q16(r.y, r.h, oh, v);
        }
        const uint2 tx = make_tap(xq, W), ty = make_tap(yq, H);
        const size_t base = (size_t)r.frame * H * W;
        og[o] = (uint8_t)bilerp(grey + base, W, tx.x, ty.x);
        od[o] = __ldg(depth + base + (size_t)ty.y * W + tx.y);
    }
}

// ---------------------------------------------------------------------------------------
// A5 alone: per-cell normalisation of count rows; one CTA per row.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ float store_x(void* out, int dtype, size_t idx, float x, float scale,
                                         size_t plane = 0) {
    if (dtype == RGBD_DT_BF16) {
        const __nv_bfloat16 q = __float2bfloat16_rn(x);
        reinterpret_cast<uint16_t*>(out)[idx] = __bfloat16_as_ushort(q);
        return __bfloat162float(q);
    } else if (dtype == RGBD_DT_BF16X3) {
        // hi = bf16(x), lo = bf16(x - hi): x = hi + lo to 2^-18 relative
        const __nv_bfloat16 hi = __float2bfloat16_rn(x);
        const float hf = __bfloat162float(hi);
        const __nv_bfloat16 lo = __float2bfloat16_rn(x - hf);
        reinterpret_cast<uint16_t*>(out)[idx] = __bfloat16_as_ushort(hi);
        reinterpret_cast<uint16_t*>(out)[idx + plane] = __bfloat16_as_ushort(lo);
        return hf + __bfloat162float(lo);
    } else if (dtype == RGBD_DT_FP8) {
        const __nv_fp8_e4m3 q(x * scale);
        reinterpret_cast<uint8_t*>(out)[idx] = q.__x;
        return static_cast<float>(q) * (1.0f / scale);
    }
    reinterpret_cast<float*>(out)[idx] = x;
    return x;
}

__global__ void normalize_kernel(const uint16_t* __restrict__ feats, int n, int dim, int nbins,
                                 int x_dtype, void* x_out, int k_pad, float x_scale, float* xsq,
                                 float* row_max, size_t plane, const float* __restrict__ centre) {
    extern __shared__ uint32_t nv[];  // [dim / nbins]
    __shared__ float red[2][32];
    const int cells = dim / nbins;
    for (int row = blockIdx.x; row < n; row += gridDim.x) {
        __syncthreads();
        const uint16_t* h = feats + (size_t)row * dim;
        for (int c = threadIdx.x; c < cells; c += blockDim.x) {
            uint32_t t = 0;
            for (int b = 0; b < nbins; ++b) t += h[c * nbins + b];
            nv[c] = t;
        }
        __syncthreads();
        float sq = 0.f, mx = 0.f;
        for (int j = threadIdx.x; j < k_pad; j += blockDim.x) {
            float x = 0.f;
            if (j < dim) {
                const uint32_t t = nv[j / nbins];
                x = t ? (float)h[j] / (float)t : 0.f;
                if (centre) x = __fsub_rn(x, centre[j]);
            }
            mx = fmaxf(mx, fabsf(x));
            const float q = store_x(x_out, x_dtype, (size_t)row * k_pad + j, x, x_scale, plane);
            sq = fmaf(q, q, sq);
        }
        for (int off = 16; off > 0; off >>= 1) {
            sq += __shfl_xor_sync(FULL, sq, off);
            mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, off));
        }
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        if (lane == 0) {
            red[0][warp] = sq;
            red[1][warp] = mx;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            float t = 0.f, m = 0.f;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                t += red[0][w];
                m = fmaxf(m, red[1][w]);
            }
            if (xsq) xsq[row] = t;
            if (row_max) atomicMax(reinterpret_cast<int*>(row_max), __float_as_int(m));  // m >= 0
        }
    }
}

// fp32 rows -> dtype rows (FP8 with `scale`), with squared norms of the stored values.
__global__ void quantize_kernel(const float* __restrict__ src, int n, int k_pad, int dtype, void* dst,
                                float scale, float* sq_out, size_t plane) {
    __shared__ float red[32];
    for (int row = blockIdx.x; row < n; row += gridDim.x) {
        __syncthreads();
        float sq = 0.f;
        for (int j = threadIdx.x; j < k_pad; j += blockDim.x) {
            const float q = store_x(dst, dtype, (size_t)row * k_pad + j, src[(size_t)row * k_pad + j], scale, plane);
            sq = fmaf(q, q, sq);
        }
        for (int off = 16; off > 0; off >>= 1) sq += __shfl_xor_sync(FULL, sq, off);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sq;
        __syncthreads();
        if (threadIdx.x == 0) {
            float t = 0.f;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
            if (sq_out) sq_out[row] = t;
        }
    }
}

// mu[j] = fp32(sum_i rows[i][j] / n), the sum in fp64 in row order (one thread per column, so
// the order and the result are fixed); mu[j] = 0 for j >= dim.
__global__ void column_mean_kernel(const float* __restrict__ rows, int n, int dim, int k_pad, float* __restrict__ mu) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= k_pad) return;
    double acc = 0.0;
    if (j < dim)
        for (int i = 0; i < n; ++i) acc += (double)rows[(size_t)i * k_pad + j];
    mu[j] = j < dim ? (float)(acc / (double)n) : 0.f;
}

// rows[i][j] -= mu[j] (fp32, round to nearest even); *absmax = max |result| (non-negative floats
// order like their bit patterns, so an integer max serves).
__global__ void centre_kernel(float* __restrict__ rows, int n, int k_pad, const float* __restrict__ mu,
                              float* absmax) {
    __shared__ float red[32];
    for (int row = blockIdx.x; row < n; row += gridDim.x) {
        float m = 0.f;
        for (int j = threadIdx.x; j < k_pad; j += blockDim.x) {
            const size_t idx = (size_t)row * k_pad + j;
            const float v = __fsub_rn(rows[idx], mu[j]);
            rows[idx] = v;
            m = fmaxf(m, fabsf(v));
        }
        for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(FULL, m, off));
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
            atomicMax(reinterpret_cast<int*>(absmax), __float_as_int(m));
        }
    }
}

template <int S, int TPC>
int launch_fused_t(rgbd_ctx* ctx, const LbpArgs& a, cudaStream_t s) {
    static int blocks_per_sm = -1;
    const size_t smem = sizeof(Smem<S, TPC>);
    if (blocks_per_sm < 0) {
        cudaError_t e = cudaFuncSetAttribute(lbp_fused_kernel<S, TPC>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_error(e, "lbp_fused_features: smem attribute");
        int b = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, lbp_fused_kernel<S, TPC>, Cfg<S, TPC>::NT, smem);
        if (e != cudaSuccess) return cuda_error(e, "lbp_fused_features: occupancy");
        blocks_per_sm = b > 0 ? b : 1;
    }
    const int per_sm = ctx->tune_lbp_ctas_per_sm > 0 ? std::min(ctx->tune_lbp_ctas_per_sm, blocks_per_sm) : blocks_per_sm;
    const int grid = (int)std::min<long long>((long long)a.n, (long long)per_sm * ctx->props.sm_count);
    LbpArgs la = a;
    if (grid >= a.n) {
        la.face_counter = nullptr;  // one face per CTA: no queue, and no reset launch for it
    } else if (la.face_counter) {
        cudaError_t e = cudaMemsetAsync(la.face_counter, 0, sizeof(uint32_t), s);
        if (e != cudaSuccess) return cuda_error(e, "lbp_fused_features: face queue reset");
    }
    lbp_fused_kernel<S, TPC><<<grid, Cfg<S, TPC>::NT, smem, s>>>(la);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "lbp_fused_features: launch");
    return RGBD_OK;
}

}  // namespace

int launch_lbp_fused(rgbd_ctx* ctx, const LbpArgs& a, cudaStream_t s) {
    if (a.flags & RGBD_LBP_FACE_HIST256) {
        const size_t smem = face256_smem(a.crop);
        cudaError_t e = cudaFuncSetAttribute(lbp_face256_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return cuda_error(e, "lbp_fused_features: 0-255 histogram smem attribute");
        const int grid = std::min(a.n, ctx->props.sm_count);
        lbp_face256_kernel<<<grid, F256_THREADS, smem, s>>>(a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_error(e, "lbp_fused_features: 0-255 histogram launch");
        return RGBD_OK;
    }
    // tile shape (crops 64 and 128): one thread per cell (tuning value 1), per half cell (2, the
    // default), per quarter cell (3: 1024-thread CTAs, measured 7 % slower even when every face
    // has an SM of its own, and 50 % slower on full batches)
    const int shape = ctx->tune_lbp_shape == 0 ? 2 : ctx->tune_lbp_shape;
    switch (a.crop) {
        case 32: return launch_fused_t<32, 2>(ctx, a, s);
        case 64:
            return shape == 1 ? launch_fused_t<64, 1>(ctx, a, s)
                              : (shape == 3 ? launch_fused_t<64, 4>(ctx, a, s) : launch_fused_t<64, 2>(ctx, a, s));
        case 96: return launch_fused_t<96, 2>(ctx, a, s);
        case 128:
            return shape == 1 ? launch_fused_t<128, 1>(ctx, a, s)
                              : (shape == 3 ? launch_fused_t<128, 4>(ctx, a, s) : launch_fused_t<128, 2>(ctx, a, s));
        default:
            return set_error(RGBD_ERR_UNSUPPORTED, "lbp_fused_features: crop %d (32, 64, 96 or 128)", a.crop);
    }
}

int launch_crop_affine(rgbd_ctx* ctx, const uint8_t* grey, const uint16_t* depth, int n_frames,
                       int H, int W, const rgbd_rect* rects, const int32_t* affine, int n,
                       int out_h, int out_w, uint8_t* og, uint16_t* od, cudaStream_t s) {
    const int px = out_h * out_w;
    dim3 grid((px + 255) / 256, std::min(n, 65535));
    crop_affine_kernel<<<grid, 256, 0, s>>>(grey, depth, n_frames, H, W, rects, affine, n, out_h,
                                            out_w, og, od, ctx->d_status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "rgbd_crop_affine: launch");
    return RGBD_OK;
}

int launch_normalize(const uint16_t* feats, int n, int dim, int nbins, int x_dtype, void* x_out,
                     int k_pad, float x_scale, float* xsq, float* row_max, cudaStream_t s, size_t plane,
                     const float* centre) {
    const int cells = dim / nbins;
    const size_t smem = sizeof(uint32_t) * (size_t)cells;
    if (smem > 48 * 1024) return set_error(RGBD_ERR_UNSUPPORTED, "normalize: %d cells", cells);
    const int grid = std::min(n, 8192);
    if (plane == 0) plane = (size_t)n * k_pad;
    normalize_kernel<<<grid, 256, smem, s>>>(feats, n, dim, nbins, x_dtype, x_out, k_pad, x_scale,
                                             xsq, row_max, plane, centre);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "lbp_normalize_features: launch");
    return RGBD_OK;
}

int launch_quantize_f32(const float* src, int n, int k_pad, int x_dtype, void* dst, float scale,
                        float* sq, cudaStream_t s, size_t plane) {
    const int grid = std::min(n, 8192);
    if (plane == 0) plane = (size_t)n * k_pad;
    quantize_kernel<<<grid, 256, 0, s>>>(src, n, k_pad, x_dtype, dst, scale, sq, plane);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "quantize: launch");
    return RGBD_OK;
}

int launch_centre_rows(float* rows, int n, int dim, int k_pad, float* mu, float* absmax, cudaStream_t s) {
    column_mean_kernel<<<(k_pad + 255) / 256, 256, 0, s>>>(rows, n, dim, k_pad, mu);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "centre: mean launch");
    centre_kernel<<<std::min(n, 8192), 256, 0, s>>>(rows, n, k_pad, mu, absmax);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "centre: launch");
    return RGBD_OK;
}

}  // namespace rgbd
