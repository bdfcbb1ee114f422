// Compile-time tile configurations of the bulk-copy (TMA) kernels, shared by
// the single-problem kernel (tsm2_stream.cu) and the batched kernel
// (tsm2_batched.cu).
#pragma once

#include "common.cuh"

namespace tsm2 {

#ifndef TSM2_PACKED_FMA
#define TSM2_PACKED_FMA 1
#endif
constexpr bool kPackedFma = TSM2_PACKED_FMA != 0;
#ifndef TSM2_CQ
#define TSM2_CQ 4
#endif

constexpr size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
constexpr int cmin(int a, int b) { return a < b ? a : b; }

template <typename T_, int KC_, int NV_, int WR_, int WC_, int WK_, int JW_, int STAGES_, bool BRES_, int NRES_,
          bool BT_ = false, int BOXM_ = 0, bool WHOLE_ = false, bool SEPI_ = false>
struct Cfg {
    using T = T_;
    using VT = Vec16<T>;
    using vec_t = typename VT::type;
    static constexpr int V = VT::n;          // elements per 16-byte vector
    static constexpr int KC = KC_;           // C columns per pass
    static constexpr int NV = NV_;           // 16-byte row vectors per lane
    static constexpr int WR = WR_;           // warps along rows
    static constexpr int WC = WC_;           // warps along the inner dimension
    static constexpr int WK = WK_;           // warps along the columns of C
    static constexpr int KCW = KC_ / WK_;    // C columns per warp
    static constexpr int JW = JW_;           // inner columns per warp per stage
    static constexpr int STAGES = STAGES_;
    static constexpr bool BRES = BRES_;      // B resident in shared memory
    static constexpr int NRES = NRES_;       // inner extent reserved for resident B
    // B in shared memory row-major (element (j, c) at j*KC + c) instead of
    // column-major: one 16-byte load gives two column pairs of one inner index,
    // so packed FMAs pair C columns and duplicate the A value (R per inner
    // index) instead of the B value (KCW per inner index).
    static constexpr bool BT = BT_;
    // Streamed B read row-major is loaded by the three otherwise idle warps
    // of the producer warpgroup, straight from the caller's column-major B
    // (in L2 after first use), a few stages ahead; they transpose it in
    // registers and store it as rows, so no packing pass over B runs before
    // the launch and B is not part of the bulk copy.  The rows are BROWS
    // elements apart; with one column warp (WK == 1) the 16-byte groups of
    // row j sit XOR-swizzled by (j & 3), which spreads the loaders' 16-byte
    // stores over the banks while every consumer address stays a
    // compile-time offset.
    static constexpr bool BLOAD = BT_ && !BRES_;
    static constexpr bool BSWZ = BLOAD && WK_ == 1;
    static constexpr int BROWS = BSWZ ? (KC_ <= 16 ? 16 : 32) : KC_;
    // Row blocks are never split between blocks (one group = one row block,
    // no partial sums): always with resident B, optionally with streamed B
    // (the TSM2L schedule for B too large to keep on chip).
    static constexpr bool WHOLE = BRES_ || WHOLE_;
    // Whole row blocks write C through shared memory (rounds of CC columns
    // of every column-warp group, then coalesced copies): storing 128
    // accumulators straight from registers costs spills in this kernel.
    static constexpr bool SEPI = SEPI_;
    static constexpr int R = NV * V;         // rows per lane
    static constexpr int BM = WR * 32 * R;   // rows per row block
    static constexpr int BNS = WC * JW;      // inner columns per stage
    static constexpr int NW = WR * WC * WK;  // consumer warps
    static constexpr int NT = NW * 32;       // consumer threads
    static constexpr int THREADS = NT + 128; // plus one producer warpgroup (one lane works)
    static_assert(NW == 8, "register split below assumes 2 consumer warpgroups");
    static constexpr int BOXM = BOXM_ > 0 ? BOXM_ : (BM < 256 ? BM : 256);
    static constexpr int NBOX = BM / BOXM;
    static constexpr int JV = V;             // inner columns per B vector
    static constexpr int CC = cmin(KC, 4);   // C columns per cross-warp reduction round
    static constexpr int CQ = cmin(KCW, TSM2_CQ);  // C columns per group of the inner loop
    static constexpr int A_STAGE = BM * BNS;                 // elements
    static constexpr int B_STAGE = (BRES || BLOAD) ? 0 : BNS * KC;  // elements copied with A (column-major)
    static constexpr int BROW_STAGE = BLOAD ? BNS * BROWS : 0;       // elements stored by the loaders (rows)
    static constexpr int RED = WC > 1 ? WC * CC * BM : (SEPI ? WK * CC * BM : 0);  // elements
    static constexpr int BRES_ELEMS = BRES ? KC * NRES : 0;  // elements
    static constexpr uint32_t TX_BYTES = (uint32_t)((A_STAGE + B_STAGE) * sizeof(T));
    static constexpr size_t OFF_A = 0;
    static constexpr size_t OFF_B = OFF_A + (size_t)STAGES * A_STAGE * sizeof(T);
    static constexpr size_t OFF_BROW = OFF_B + (size_t)STAGES * B_STAGE * sizeof(T);
    static constexpr size_t OFF_BRES = OFF_BROW + (size_t)STAGES * BROW_STAGE * sizeof(T);
    static constexpr size_t OFF_RED = OFF_BRES + (size_t)BRES_ELEMS * sizeof(T);
    static constexpr size_t OFF_BAR = align_up(OFF_RED + (size_t)RED * sizeof(T), 16);
    // full and empty barriers, STAGES each
    static constexpr int NBAR = 2;
    // Arrivals that complete a stage: the producer lane's (with the copy's
    // bytes) and, with loaded B, one loader warp's.
    static constexpr int FULL_ARRIVALS = BLOAD ? 2 : 1;
    static constexpr size_t OFF_FLAGS = OFF_BAR + NBAR * STAGES * sizeof(uint64_t);
    // Resident B without the staged epilogue: row blocks can be claimed at
    // run time, and meta[] holds the row block of every stage.
    static constexpr bool DYN = BRES_ && !SEPI_;
    static constexpr size_t OFF_META = OFF_FLAGS + 32;
    static constexpr size_t SMEM = OFF_META + (DYN ? align_up(STAGES * sizeof(int), 16) : 0) + 128;  // + slack for 128-byte alignment

    static_assert(BT || JW % JV == 0, "a warp's columns must be whole B vectors");
    static_assert((BNS * sizeof(T)) % 16 == 0, "TMA inner box extent must be 16-byte multiple");
    static_assert((A_STAGE * sizeof(T)) % 128 == 0, "stage buffers stay 128-byte aligned");
    static_assert((B_STAGE * sizeof(T)) % 128 == 0 || BRES, "stage buffers stay 128-byte aligned");
    static_assert(BM % BOXM == 0 && (32 * V) <= BOXM, "a warp's vector row group fits one box");
    static_assert(WC == 1 || (CC * BM) % NT == 0, "reduction rounds split evenly over threads");
    static_assert(!BRES || NRES % BNS == 0, "resident B covers whole stages");
    static_assert(KC % WK == 0 && (WK == 1 || (WC == 1 && WHOLE)), "C columns split only in the TSM2L schedules");
    static_assert(WC == 1 || !WHOLE, "whole row blocks need no cross-warp inner split");
    static_assert(!SEPI || (WHOLE && WC == 1 && KCW % CC == 0 && (WK * CC * BM) % (4 * NT) == 0 && BM % 4 == 0),
                  "staged epilogue: whole row blocks, column rounds of CC, whole 16-byte vectors per thread");
    static_assert(SMEM <= 227 * 1024, "shared memory per block");
    static_assert(!BT || (sizeof(T) == 4 && KCW % 4 == 0), "row-major B: binary32, whole 16-byte column groups");
    static_assert(!BSWZ || (JW % 4 == 0 && KC <= BROWS), "swizzle key j & 3 known per unrolled inner index");
    static_assert(!BLOAD || BNS % 4 == 0, "loaded B: whole 4 x 4 blocks");
    // A loader warp takes every third stage; with at least three stages the
    // empty-barrier parity it waits on cannot alias an older phase.
    static_assert(!BLOAD || STAGES >= 3, "loaded B needs three stages or more");
};

// Physical 16-byte group of logical group g (columns 4g .. 4g+3) in row j
// of a loaded B tile.
template <class K>
__device__ __forceinline__ int bgroup(int j, int g) {
    return K::BSWZ ? (g ^ (j & 3)) : g;
}

// One loader warp fills the B rows of a stage: rows j0 .. j0+BNS-1 of B
// (n x k, column-major, ldb; 16-byte aligned with ldb a multiple of 4),
// columns 0 .. KC-1, zero past n and k, as rows of BROWS elements: (j, c) at
// brow[(j-j0)*BROWS + 4*bgroup<K>(j-j0, c/4) + c%4].  Block u (a lane's, in
// steps of 32) covers rows 4(u/NG) .. +3 and columns 4(u%NG) .. +3: four
// 16-byte loads down its columns, a register transpose, four 16-byte row
// stores.
template <class K>
__device__ __forceinline__ void load_b_stage(const float *__restrict__ B, int64_t ldb, int64_t n, int k, int64_t j0,
                                             float *brow, int lane, unsigned *status) {
    constexpr int NG = K::KC >= 4 ? K::KC / 4 : 1;  // (instantiated, never run, for KC < 4)
    constexpr int NBLK = (K::BNS / 4) * NG;
#pragma unroll 1
    for (int u = lane; u < NBLK; u += 32) {
        const int q = u / NG, cg = u - (u / NG) * NG;
        const int64_t jr = j0 + 4 * q;  // first row of the block
        float4 v[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int c = 4 * cg + i;
            const float *col = B + jr + (int64_t)c * ldb;
            if (c >= k || !dbg_in_bounds(jr >= 0 && c < K::KC, status)) {
                v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            } else if (jr + 3 < n) {
                v[i] = __ldg(reinterpret_cast<const float4 *>(col));
            } else {
                v[i].x = jr + 0 < n ? __ldg(col + 0) : 0.f;
                v[i].y = jr + 1 < n ? __ldg(col + 1) : 0.f;
                v[i].z = jr + 2 < n ? __ldg(col + 2) : 0.f;
                v[i].w = jr + 3 < n ? __ldg(col + 3) : 0.f;
            }
        }
        const int j = 4 * q;
        float *row = brow + j * K::BROWS;
        *reinterpret_cast<float4 *>(row + 4 * bgroup<K>(j + 0, cg)) = make_float4(v[0].x, v[1].x, v[2].x, v[3].x);
        row += K::BROWS;
        *reinterpret_cast<float4 *>(row + 4 * bgroup<K>(j + 1, cg)) = make_float4(v[0].y, v[1].y, v[2].y, v[3].y);
        row += K::BROWS;
        *reinterpret_cast<float4 *>(row + 4 * bgroup<K>(j + 2, cg)) = make_float4(v[0].z, v[1].z, v[2].z, v[3].z);
        row += K::BROWS;
        *reinterpret_cast<float4 *>(row + 4 * bgroup<K>(j + 3, cg)) = make_float4(v[0].w, v[1].w, v[2].w, v[3].w);
    }
}

// One pipeline stage of one consumer warp (Alg. 2's inner update, with the
// warp's share of the stage): for j over the warp's JW inner indices,
// ascending, acc[r][c] += A(rbase + row(r), j) * B(j, kbase + c).
//   a_st:  the stage's A tile, NBOX boxes of BOXM rows x BNS inner columns,
//          rows contiguous;
//   b_st:  the stage's B, row-major (K::BT: element (j, c) at b_st[j*KC + c])
//          or column-major (column c at b_st + c*bstride);
//   rbase: first row of the lane's first 16-byte row vector (vector v covers
//          rows rbase + v*32*V .. + V-1).
// Every accumulator sees the same sequence of single-rounding FMAs in both
// layouts, so results do not depend on the layout.
template <class K>
__device__ __forceinline__ void consume_stage(const typename K::T *a_st, const typename K::T *b_st, int bstride,
                                              int wc, int kbase, int rbase, typename K::T (&acc)[K::R][K::KCW]) {
    using T = typename K::T;
    using vec_t = typename K::vec_t;
    if constexpr (K::BT) {
        // Per inner index: the lane's R values of A, then for each group of
        // four C columns one 16-byte broadcast load giving two column pairs,
        // each updated by a packed FMA with (a, a).
#pragma unroll
        for (int jj = 0; jj < K::JW; ++jj) {
            const int j = wc * K::JW + jj;
            float a[K::R];
#pragma unroll
            for (int v = 0; v < K::NV; ++v) {
                const int r = rbase + v * 32 * K::V;
                const int q = r / K::BOXM;
                const int rr = r - q * K::BOXM;
                const float4 x = *reinterpret_cast<const float4 *>(a_st + q * K::BOXM * K::BNS + j * K::BOXM + rr);
                a[v * 4 + 0] = x.x;
                a[v * 4 + 1] = x.y;
                a[v * 4 + 2] = x.z;
                a[v * 4 + 3] = x.w;
            }
            const T *brow = b_st + j * K::BROWS + kbase;
#pragma unroll
            for (int c0 = 0; c0 < K::KCW; c0 += 4) {
                // BSWZ: kbase = 0 and j & 3 = jj & 3 (JW % 4 == 0), so the
                // swizzled group offset is a constant.
                const int goff = K::BSWZ ? 4 * ((c0 >> 2) ^ (jj & 3)) : c0;
                const float4 bq = *reinterpret_cast<const float4 *>(brow + goff);
                const float2 b01 = make_float2(bq.x, bq.y);
                const float2 b23 = make_float2(bq.z, bq.w);
#pragma unroll
                for (int r = 0; r < K::R; ++r) {
                    const float2 aa = make_float2(a[r], a[r]);
                    const float2 t0 = __ffma2_rn(aa, b01, make_float2(acc[r][c0], acc[r][c0 + 1]));
                    const float2 t1 = __ffma2_rn(aa, b23, make_float2(acc[r][c0 + 2], acc[r][c0 + 3]));
                    acc[r][c0] = t0.x;
                    acc[r][c0 + 1] = t0.y;
                    acc[r][c0 + 2] = t1.x;
                    acc[r][c0 + 3] = t1.y;
                }
            }
        }
    } else {
        // Column-major B: one 16-byte load gives JV consecutive inner indices
        // of one C column; A for those JV indices is loaded first.
#pragma unroll
        for (int jj = 0; jj < K::JW; jj += K::JV) {
            const int j = wc * K::JW + jj;  // stage-local inner column of the first vector lane
            T a[K::JV][K::R];
#pragma unroll
            for (int jv = 0; jv < K::JV; ++jv)
#pragma unroll
                for (int v = 0; v < K::NV; ++v) {
                    const int r = rbase + v * 32 * K::V;
                    const int q = r / K::BOXM;
                    const int rr = r - q * K::BOXM;
                    const vec_t x =
                        *reinterpret_cast<const vec_t *>(a_st + q * K::BOXM * K::BNS + (j + jv) * K::BOXM + rr);
#pragma unroll
                    for (int e = 0; e < K::V; ++e) a[jv][v * K::V + e] = K::VT::get(x, e);
                }
            // C columns in groups of CQ: consecutive FMAs of a group hit
            // different accumulators, so no FMA waits on the previous one.
#pragma unroll
            for (int c0 = 0; c0 < K::KCW; c0 += K::CQ) {
                vec_t bv[K::CQ];
#pragma unroll
                for (int cq = 0; cq < K::CQ; ++cq)
                    bv[cq] = *reinterpret_cast<const vec_t *>(b_st + (kbase + c0 + cq) * bstride + j);
#pragma unroll
                for (int jv = 0; jv < K::JV; ++jv)
#pragma unroll
                    for (int cq = 0; cq < K::CQ; ++cq) {
                        const int c = c0 + cq;
                        const T b = K::VT::get(bv[cq], jv);
                        if constexpr (kPackedFma && sizeof(T) == 4) {
                            // Two rows per packed FFMA2: half the FMA issue slots.
                            const float2 bb = make_float2(b, b);
#pragma unroll
                            for (int r = 0; r < K::R; r += 2) {
                                const float2 t = __ffma2_rn(make_float2(a[jv][r], a[jv][r + 1]), bb,
                                                            make_float2(acc[r][c], acc[r + 1][c]));
                                acc[r][c] = t.x;
                                acc[r + 1][c] = t.y;
                            }
                        } else {
#pragma unroll
                            for (int r = 0; r < K::R; ++r) acc[r][c] = fma(a[jv][r], b, acc[r][c]);
                        }
                    }
            }
        }
    }
}

// Resident B (n <= NRES inner indices, KC columns) into shared memory by the
// NT consumer threads (tid 0 .. NT-1), zero beyond n and k so padded lanes
// contribute exact zeros: column c at sBres[c*NRES + j], or row-major
// (K::BT) (j, c) at sBres[j*KC + c].  All of a thread's loads are issued
// before its stores, so their DRAM round trips overlap (one after another,
// the eight loads per thread of KC = 32 delayed the first stage by ~5 us).
template <class K>
__device__ __forceinline__ void load_resident_b(typename K::T *sBres, const typename K::T *B, int64_t n, int k,
                                                int64_t ldb, int tid) {
    using T = typename K::T;
    constexpr int TOTAL = K::KC * K::NRES;
    constexpr int PER = (TOTAL + K::NT - 1) / K::NT;
    T v[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int t = tid + i * K::NT;
        const int j = K::BT ? t / K::KC : t % K::NRES;
        const int c = K::BT ? t % K::KC : t / K::NRES;
        v[i] = (t < TOTAL && j < n && c < k) ? B[j + (int64_t)c * ldb] : T(0);
    }
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int t = tid + i * K::NT;
        if (t < TOTAL) sBres[t] = v[i];
    }
}

// The part of resident B that pairs with stage jc (inner indices jc*BNS ..).
template <class K>
__device__ __forceinline__ const typename K::T *resident_b_stage(const typename K::T *sBres, int jc) {
    return K::BT ? sBres + (size_t)jc * K::BNS * K::KC : sBres + jc * K::BNS;
}

// Block index that owns group x under the partition gs(g) = floor(g*NG/G).
__device__ __forceinline__ int64_t owner_of(int64_t x, int64_t G, int64_t NG) {
    return ((x + 1) * G + NG - 1) / NG - 1;
}

// Register split (setmaxnreg): launched with 384 threads x 168 registers =
// 64512; the producer warpgroup drops to 40 and the two consumer warpgroups
// rise to 232: 4*32*40 + 8*32*232 = 64512, exactly the launch pool, and every
// SM sub-partition (one producer warp + two consumer warps) holds
// 32*(40 + 2*232) = 16128 <= 16384 registers.
constexpr int kProducerRegs = 40;
constexpr int kConsumerRegs = 232;
static_assert(4 * 32 * kProducerRegs + 8 * 32 * kConsumerRegs <= 384 * 168, "register split exceeds launch pool");

// TSM2R schedule: 1 x 8 warps split the inner columns of each stage.
//   binary32: R = 8 rows per lane (two float4), BM = 256, BNS = 32.
//   binary64: R = 4 rows per lane (two double2), BM = 128, BNS = 32.
//   KC >= 12 keeps B row-major in shared memory (fewer operand duplications).
#ifndef TSM2_R16_NV
#define TSM2_R16_NV 2
#endif
#ifndef TSM2_R16_JW
#define TSM2_R16_JW 4
#endif
#ifndef TSM2_R16_STAGES
#define TSM2_R16_STAGES 4
#endif
// Pipeline stages (measured on GB300, 30720^2 and 10240^2): four for 8..16
// C columns (k = 16: 0.6048 -> 0.5987 ms, k = 8: 0.5731 -> 0.5669 ms at
// 30720^2 against five; three is slower again), five for 2..4 columns.
#ifndef TSM2_R_STAGES
#define TSM2_R_STAGES 5
#endif
#ifndef TSM2_R8_STAGES
#define TSM2_R8_STAGES 4
#endif
template <int KC>
using R32 = Cfg<float, KC, (KC >= 16 ? TSM2_R16_NV : 2), 1, 8, 1, (KC >= 16 ? TSM2_R16_JW : 4),
                (KC >= 16 ? TSM2_R16_STAGES : (KC >= 8 ? TSM2_R8_STAGES : TSM2_R_STAGES)), false, 0, (KC >= 12),
                (KC >= 16 && TSM2_R16_NV == 3 ? 128 : 0)>;
template <int KC> using R64 = Cfg<double, KC, 2, 1, 8, 1, 4, 5, false, 0>;
// TSM2L: resident B row-major wherever a warp's C columns are whole groups of
// four (the B load at block start transposes; no packed copy needed).
#ifndef TSM2_L_BT
#define TSM2_L_BT 1
#endif
// TSM2L schedule: 8 x 1 warps split the rows; B (n <= 64) resident.
//   binary32: R = 4, BM = 1024, BNS = 8.   binary64: R = 2, BM = 512, BNS = 8.
//   KC = 32 splits the C columns over 2 x 4 warps (16 accumulated columns per
//   lane, BM halves) to keep the accumulators in registers.
#ifndef TSM2_L_STAGES
#define TSM2_L_STAGES 5
#endif
template <int KC>
using L32 = Cfg<float, KC, 1, (KC >= 32 ? 4 : 8), 1, (KC >= 32 ? 2 : 1), 8, TSM2_L_STAGES, true, 64,
                (TSM2_L_BT != 0 && (KC / (KC >= 32 ? 2 : 1)) % 4 == 0)>;
template <int KC> using L64 = Cfg<double, KC, 1, (KC >= 32 ? 4 : 8), 1, (KC >= 32 ? 2 : 1), 8, 5, true, 64>;
// TSM2L schedule for tall A and wide C (binary32, KC = 24 and 32): R = 8 rows
// per lane, so every B value read from shared memory (one wavefront per
// broadcast value) feeds twice the FMAs; the C columns are split over WK = 2
// warps.  Chosen when there are enough row blocks for an even spread over the
// SMs.  KC = 32: 16 C columns per lane (128 accumulators, 1024-row blocks),
// stored straight from registers.  n = k = 32 is FMA-bound on chip (32 FMAs
// per 8 bytes of A and C), and against 8 columns per lane this halves the
// shared-memory reads of A per FMA: 75% -> 92% of HBM at 2^23 rows.  (For KC
// <= 16 the 4-rows-per-lane schedule with row blocks claimed at run time
// measured equal or faster at every height, up to 9% at 2^23 x 16.)
struct WShape {
    int nv, wr, wk, jw, st;
    bool sepi;
};
#ifndef TSM2_W_STAGES
#define TSM2_W_STAGES 5
#endif
constexpr WShape w32_shape(int kc) {
    return kc >= 32 ? WShape{2, 4, 2, 8, TSM2_W_STAGES, false}   // 16 columns per lane
                    : WShape{2, 4, 2, 8, TSM2_W_STAGES, false};  // KC = 24: 12 columns per lane
}
template <int KC>
using W32 = Cfg<float, KC, w32_shape(KC).nv, w32_shape(KC).wr, 1, w32_shape(KC).wk, w32_shape(KC).jw,
                w32_shape(KC).st, true, 64, (TSM2_L_BT != 0 && (KC / w32_shape(KC).wk) % 4 == 0), 0, false,
                w32_shape(KC).sepi>;
// TSM2L with B staged instead of resident (Alg. 6's setting, Sec. 3.2.2: B
// too large to stay on chip, here n > 64): B rows arrive with each A stage,
// but every block still owns whole row blocks and keeps their C columns in
// registers across the inner loop, so C is written once and A is read once
// per 32 columns of C.  16 C columns per lane for KC >= 16 (C staged through
// shared memory), 8 inner columns per stage for KC = 32; C columns in groups
// of at least four (narrower k pads to KC = 4).
constexpr WShape t32_shape(int kc) {
    return kc >= 24   ? WShape{2, 4, 2, 8, 5, true}
           : kc >= 16 ? WShape{2, 8, 1, 4, 4, true}
                      : WShape{2, 8, 1, 8, 3, false};
}
template <int KC>
using T32 = Cfg<float, KC, t32_shape(KC).nv, t32_shape(KC).wr, 1, t32_shape(KC).wk, t32_shape(KC).jw, t32_shape(KC).st,
                false, 0, ((KC / t32_shape(KC).wk) % 4 == 0), 0, true, t32_shape(KC).sepi>;
template <int KC>
using T64 = Cfg<double, KC, 1, (KC >= 32 ? 4 : 8), 1, (KC >= 32 ? 2 : 1), 8, 5, false, 0, false, 0, true>;

}  // namespace tsm2
