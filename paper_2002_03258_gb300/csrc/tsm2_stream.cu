// Bulk-copy (TMA) path for TSM2R and TSM2L on sm_103a.
//
// What it computes: C(m x k) = A(m x n) B(n x k), column-major, for up to KC
// columns of C per launch (the host loops over column chunks, which is the
// t2 loop of Algorithm 4, Sec. 3.1.4).
//
// How it maps the paper's design onto GB300:
//  * Outer product, A read once (Algorithm 2, Sec. 3.1.2): every lane owns R
//    rows of C and keeps all KC accumulators of each row in registers; every
//    element of A that reaches the lane is multiplied into all KC of them.
//  * B staged on chip and read by broadcast (Algorithm 3, Sec. 3.1.3-3.1.4):
//    the rows of B that pair with the current A tile arrive in shared memory
//    with it, in column order; all lanes of a warp read the same 16 bytes at
//    once.  Configurations that read B row-major (two column pairs per
//    16-byte load) have the three otherwise idle producer warps load each
//    stage's B rows from global memory and store them transposed.
//  * Prefetching (Algorithm 4, Sec. 3.1.5) becomes a STAGES-deep ring of
//    shared-memory buffers filled by the tensor-memory accelerator: one
//    producer lane issues 2-D bulk tensor copies of A tiles (BM rows x BNS
//    columns) STAGES-1 tiles ahead of the consumer warps, signalling
//    completion on per-stage mbarriers; consumers release a stage through a
//    second mbarrier.  The bytes in flight per SM are set by Little's law
//    (Sec. 3.1.8) rather than by registers per thread.
//  * Fewer, longer-lived threads (Algorithm 5, Sec. 3.2.2): the grid is
//    persistent, one thread block per SM.  The work units (one pipeline
//    stage each, i.e. a BM x BNS tile of A) are numbered row block by row
//    block and every block takes a contiguous run of them, so all blocks get
//    the same amount of work whatever the shape.  With B resident (TSM2L),
//    whole row blocks are instead handed out at run time: each block starts
//    with its own and then claims the next from a counter, so blocks on SMs
//    that stream faster take more.
//  * When a block's run starts or ends inside a row block (TSM2R schedule),
//    its partial sums go to a workspace slot; the last block to finish a row
//    block (an atomic arrival counter, no waiting) adds the slots in a fixed
//    order and writes C.  Results are therefore bitwise reproducible.
//  * TSM2R schedule: the 8 consumer warps of a block share the rows of one
//    row block and split the inner-dimension columns of every stage; their
//    partial sums meet once per row block in shared memory (fixed warp
//    order).  TSM2L schedule: the warps split the rows (BM = 8 x 32 x R),
//    the whole of B (n <= 64) is loaded once per block, and runs are aligned
//    to row blocks, so no partial sums are ever needed.
//
// Every wait is bounded (mbar_wait_bounded); on timeout the block records it
// in the status word, stops consuming, lets its in-flight copies land and
// exits normally.
#include "common.cuh"
#include "internal.h"
#include "tsm2_cfg.cuh"

#include <climits>
#include <mutex>

namespace tsm2 {

namespace {

struct Params {
    int64_t m, n;
    int k;
    const void *B;  // raw B for the resident copy
    int64_t ldb;
    void *C;
    int64_t ldc;
    void *ws;
    // Split row blocks: one arrival counter per row block.  Resident-B
    // (TSM2L) schedules, which split nothing, use counters[0..1] to hand out
    // row blocks at run time instead: [0] counts the row blocks claimed
    // beyond the first one of every block, [1] the blocks that have claimed
    // their last.  Zero between launches; nullptr: the static partition.
    int *counters;
    unsigned *status;
    int64_t wait_ns;
    int64_t upr;      // units (stages) per row block
    int64_t gran;     // units per indivisible group
    int64_t ngroups;  // groups in total
    int c_vec;
    unsigned long long *trace;  // optional: 4 words per block (start, first data, end, units [| SM << 32])
};

template <class K>
__global__ void __launch_bounds__(384, 1)
stream_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, const Params p) {
    using T = typename K::T;
    using vec_t = typename K::vec_t;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = smem_aligned<128>(smem_raw);
    T *sA = reinterpret_cast<T *>(smem + K::OFF_A);
    T *sB = reinterpret_cast<T *>(smem + K::OFF_B);
    T *sBres = reinterpret_cast<T *>(smem + K::OFF_BRES);
    T *sRed = reinterpret_cast<T *>(smem + K::OFF_RED);
    T *sBrow = reinterpret_cast<T *>(smem + K::OFF_BROW);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + K::OFF_BAR);
    uint64_t *empty = full + K::STAGES;
    volatile int *flags = reinterpret_cast<volatile int *>(smem + K::OFF_FLAGS);  // [0] abort, [1] last
    // ldc re-read from shared memory in the epilogue, so the compiler cannot
    // hoist per-column address offsets out of the unit loop (they would sit in
    // registers next to the accumulators).
    volatile int64_t *s_ldc = reinterpret_cast<volatile int64_t *>(smem + K::OFF_FLAGS + 16);
    // Row block of every stage when row blocks are claimed at run time.
    volatile int *meta = reinterpret_cast<volatile int *>(smem + K::OFF_META);
    // (Not with the staged epilogue, whose consumer warps would have to agree
    // on every claimed row block at a barrier: a timed-out warp cannot follow
    // the claims.  Only staged-B TSM2L stages C, and it keeps static runs.)
    const bool dyn = K::DYN && p.counters != nullptr;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t G = gridDim.x;
    const int64_t g = blockIdx.x;
    const int64_t gs = g * p.ngroups / G;
    const int64_t ge = (g + 1) * p.ngroups / G;
    const int64_t u_begin = gs * p.gran;
    const int64_t u_end = ge * p.gran;

    if (threadIdx.x == 0) {
        if (p.trace) {
            p.trace[4 * g + 0] = globaltimer_ns();
            p.trace[4 * g + 3] = (unsigned long long)(u_end - u_begin);
        }
        for (int s = 0; s < K::STAGES; ++s) {
            mbar_init(&full[s], K::FULL_ARRIVALS);
            mbar_init(&empty[s], K::NW);
        }
        flags[0] = 0;
        flags[1] = 0;
        *s_ldc = p.ldc;
        fence_mbar_init();
    }
    __syncthreads();

    if (warp < 4) {
        // ---------------- producer warpgroup: one lane issues all bulk copies ----------------
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kProducerRegs));
        if (warp == 0 && lane == 0) {
            prefetch_tensormap(&mapA);
            if constexpr (!K::BRES) prefetch_tensormap(&mapB);
            const uint64_t policy = l2_policy_evict_first();
            int s = 0;
            uint32_t ph = 0;
            uint32_t issued = 0, last_par = 0;  // per-stage: issued at least once, parity of last issue
            const int upr = (int)p.upr;
            if constexpr (K::DYN) {
              if (dyn) {
                // Whole row blocks claimed at run time: block g starts with row
                // block g, then takes G + (the claim counter's old value) until
                // the row blocks run out.  Each claim is issued a row block
                // ahead of its use, so its round trip overlaps the copies.
                // Every stage carries its row block in meta[]; a final stage
                // with row block -1 and no bytes tells the consumers to stop.
                // The result does not depend on who computes a row block.
                // (Few live registers: this lane runs with the producer's 40.)
                int rb = (int)g;
                while (rb < (int)p.ngroups) {
                    const int claim = atomicAdd(&p.counters[0], 1);
                    for (int jc = 0; jc < upr; ++jc) {
                        if (flags[0] || !mbar_wait_bounded(&empty[s], ph ^ 1u, p.wait_ns, flags)) {
                            flags[0] = 1;
                            atomicOr(p.status, kStatusTimeout);
                            break;
                        }
                        meta[s] = rb;
                        mbar_arrive_expect_tx(&full[s], K::TX_BYTES);
                        T *dstA = sA + (size_t)s * K::A_STAGE;
#pragma unroll
                        for (int q = 0; q < K::NBOX; ++q)
                            tma_load_2d_hint(dstA + q * K::BOXM * K::BNS, &mapA, rb * K::BM + q * K::BOXM,
                                             jc * K::BNS, &full[s], policy);
                        issued |= 1u << s;
                        last_par = (last_par & ~(1u << s)) | (ph << s);
                        if (++s == K::STAGES) { s = 0; ph ^= 1u; }
                    }
                    rb = flags[0] ? INT_MAX : (int)G + claim;
                }
                if (!flags[0] && mbar_wait_bounded(&empty[s], ph ^ 1u, p.wait_ns, flags)) {
                    meta[s] = -1;
                    mbar_arrive(&full[s]);
                    issued |= 1u << s;
                    last_par = (last_par & ~(1u << s)) | (ph << s);
                } else {
                    flags[0] = 1;
                    atomicOr(p.status, kStatusTimeout);
                }
                // This block's claims are done; the last block to get here
                // rearms both counters for the next launch.
                __threadfence();
                if (atomicAdd(&p.counters[1], 1) == (int)G - 1) {
                    p.counters[0] = 0;
                    p.counters[1] = 0;
                }
              }
            }
            const int nunits = dyn ? 0 : (int)(u_end - u_begin);
            int rb = (int)(u_begin / p.upr);
            int jc = (int)(u_begin - (int64_t)rb * p.upr);
            for (int i = 0; i < nunits; ++i) {
                if (flags[0]) break;
                if (!mbar_wait_bounded(&empty[s], ph ^ 1u, p.wait_ns, flags)) {
                    flags[0] = 1;
                    atomicOr(p.status, kStatusTimeout);
                    break;
                }
                mbar_arrive_expect_tx(&full[s], K::TX_BYTES);
                T *dstA = sA + (size_t)s * K::A_STAGE;
                const int32_t x0 = (int32_t)(rb * K::BM);
                const int32_t y0 = (int32_t)(jc * K::BNS);
#pragma unroll
                for (int q = 0; q < K::NBOX; ++q)
                    tma_load_2d_hint(dstA + q * K::BOXM * K::BNS, &mapA, x0 + q * K::BOXM, y0, &full[s], policy);
                // B rows of the stage, column-major (BNS x KC box of B),
                // unless the loader warps bring them.
                if constexpr (!K::BRES && !K::BLOAD) tma_load_2d(sB + (size_t)s * K::B_STAGE, &mapB, y0, 0, &full[s]);
                issued |= 1u << s;
                last_par = (last_par & ~(1u << s)) | (ph << s);
                if (++s == K::STAGES) { s = 0; ph ^= 1u; }
                if (++jc == upr) { jc = 0; ++rb; }
            }
            // Let every copy this block started land before the block can exit.
            for (int t = 0; t < K::STAGES; ++t)
                if (issued & (1u << t)) (void)mbar_wait_bounded(&full[t], (last_par >> t) & 1u, 4000000000LL, nullptr);
        } else if (K::BLOAD && warp >= 1) {
            // Loader warps 1..3: B rows of every third stage, from global
            // memory, as soon as the stage is free again.
            const int nunits = (int)(u_end - u_begin);
            for (int i = warp - 1; i < nunits; i += 3) {
                const int s = i % K::STAGES;
                const uint32_t ph = (uint32_t)(i / K::STAGES) & 1u;
                bool ok = !flags[0] && mbar_wait_bounded(&empty[s], ph ^ 1u, p.wait_ns, flags);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) {
                    if (lane == 0) {
                        flags[0] = 1;
                        atomicOr(p.status, kStatusTimeout);
                    }
                    break;
                }
                const int64_t u = u_begin + i;
                const int64_t jc = u - (u / p.upr) * p.upr;
                load_b_stage<K>(static_cast<const float *>(p.B), p.ldb, p.n, p.k, jc * K::BNS,
                                reinterpret_cast<float *>(sBrow + (size_t)s * K::BROW_STAGE), lane, p.status);
                __syncwarp();
                if (lane == 0) mbar_arrive(&full[s]);
            }
        }
        return;
    }

    // ---------------- consumers ----------------
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kConsumerRegs));
    if constexpr (K::BRES) {
        // Whole of B (n <= NRES) once per block, loaded by the consumers
        // while the producer's first copies of A are already in flight.
        load_resident_b<K>(sBres, static_cast<const T *>(p.B), p.n, p.k, p.ldb, threadIdx.x - 128);
        named_bar_sync(1, K::NT);
    }
    const int cwarp = warp - 4;                 // consumer warp 0 .. NW-1
    const int wk = cwarp % K::WK;               // group of C columns
    const int wc = (cwarp / K::WK) % K::WC;     // inner-column group
    const int wr = cwarp / (K::WK * K::WC);     // row group
    const int kbase = wk * K::KCW;              // first C column of this warp
    T acc[K::R][K::KCW];
#pragma unroll
    for (int r = 0; r < K::R; ++r)
#pragma unroll
        for (int c = 0; c < K::KCW; ++c) acc[r][c] = T(0);

    // Rows of the row block owned by this lane: vector v covers rows
    // row_of(v) .. row_of(v) + V - 1.
    auto row_of = [&](int v) { return wr * 32 * K::R + v * 32 * K::V + lane * K::V; };

    int s = 0;
    uint32_t ph = 0;
    bool aborted = false;
    // Unit bookkeeping in 32 bits (a block's run is far below 2^31 units;
    // the host checks): registers are the scarce resource here.
    // With row blocks claimed at run time the count is open-ended: the
    // producer's end marker stops the loop.
    const int nunits = (K::DYN && dyn) ? INT_MAX : (int)(u_end - u_begin);
    const int upr = (int)p.upr;
    int rb = (K::DYN && dyn) ? 0 : (int)(u_begin / p.upr);
    int jc = (K::DYN && dyn) ? 0 : (int)(u_begin - (int64_t)rb * p.upr);
    bool piece_at_rb_start = (jc == 0);

    for (int i = 0; i < nunits; ++i) {
        if (!aborted) {
            // Warp-uniform decision: the warp consumes the stage only if every
            // lane saw it complete.
            bool ok = !flags[0] && mbar_wait_bounded(&full[s], ph, p.wait_ns, flags);
            ok = __all_sync(0xffffffffu, ok);
            if (p.trace && i == 0 && cwarp == 0 && lane == 0) p.trace[4 * g + 1] = globaltimer_ns();
            if (!ok) {
                aborted = true;
                if (lane == 0) {
                    flags[0] = 1;
                    atomicOr(p.status, kStatusTimeout);
                }
            }
        }
        if constexpr (K::DYN) {
          if (dyn) {
            // (No named barriers in the loop of these configurations: a warp
            // that gave up can leave at once.)
            if (aborted) break;
            if (jc == 0) {
                rb = meta[s];
                if (rb < 0) {
                    if (p.trace && threadIdx.x == 128)
                        p.trace[4 * g + 3] = (unsigned long long)i | ((unsigned long long)sm_id() << 32);
                    break;
                }
            }
          }
        }
        if (!aborted) {
            const T *a_st = sA + (size_t)s * K::A_STAGE;
            const T *b_st;
            int bstride;
            if constexpr (K::BRES) {
                b_st = resident_b_stage<K>(sBres, jc);
                bstride = K::NRES;
            } else if constexpr (K::BLOAD) {
                b_st = sBrow + (size_t)s * K::BROW_STAGE;
                bstride = K::BROWS;
            } else {
                b_st = sB + (size_t)s * K::B_STAGE;
                bstride = K::BNS;
            }
            consume_stage<K>(a_st, b_st, bstride, wc, kbase, row_of(0), acc);
        }
        // Release the stage to the producer.  A warp that gave up releases
        // nothing more: the producer then stops too, so no copy is ever issued
        // into a buffer whose previous copy may still be landing.
        if (!aborted) {
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
        }
        if (++s == K::STAGES) { s = 0; ph ^= 1u; }

        const bool rb_end = (jc == upr - 1);
        if (rb_end || i == nunits - 1) {
            // ---------------- epilogue of one piece of row block rb ----------------
            const int64_t rb64 = rb;
            const int64_t rb_u0 = rb64 * p.upr;
            // TSM2L runs are whole row blocks by construction (gran = upr).
            const bool whole = K::WHOLE || (piece_at_rb_start && rb_end);
            const int64_t row0 = rb64 * K::BM;
            T *C = static_cast<T *>(p.C);
            T *ws = static_cast<T *>(p.ws);
            const int64_t NG = p.ngroups;
            const int64_t gA = owner_of(rb_u0 / p.gran, G, NG);
            const int64_t gB = owner_of((rb_u0 + p.upr - 1) / p.gran, G, NG);
            const int64_t my_slot = g + rb64;
            const int tid = threadIdx.x - 128;  // 0 .. NT-1 for consumers

            if constexpr (K::SEPI) {
                // Whole row block, C through shared memory: for each round of
                // CC of its columns, every warp stores them at its rows of
                // sRed (slot wk*CC + cc); then all consumer threads copy the
                // WK*CC staged columns to C, 16 bytes per access where the
                // row block lies inside C and C allows it.
                const bool fast = p.c_vec && row0 + K::BM <= p.m;
                const int64_t ldc = *s_ldc;
#pragma unroll
                for (int r0 = 0; r0 < K::KCW; r0 += K::CC) {
                    named_bar_sync(1, K::NT);
                    if (!aborted) {
#pragma unroll
                        for (int cc = 0; cc < K::CC; ++cc)
#pragma unroll
                            for (int v = 0; v < K::NV; ++v) {
                                T tmp[K::V];
#pragma unroll
                                for (int e = 0; e < K::V; ++e) tmp[e] = acc[v * K::V + e][r0 + cc];
                                *reinterpret_cast<vec_t *>(sRed + (wk * K::CC + cc) * K::BM + row_of(v)) =
                                    K::VT::make(tmp);
                            }
                    }
                    named_bar_sync(1, K::NT);
                    if (!aborted) {
                        if (fast) {
#pragma unroll 2
                            for (int q = 0; q < (K::WK * K::CC * K::BM) / (4 * K::NT); ++q) {
                                const int e = 4 * (tid + q * K::NT);
                                const int slot = e / K::BM;
                                const int row = e - slot * K::BM;
                                const int c = (slot / K::CC) * K::KCW + r0 + (slot % K::CC);
                                if (c < p.k && dbg_in_bounds(row0 + row + 3 < p.m, p.status))
                                    *reinterpret_cast<float4 *>(C + row0 + row + (int64_t)c * ldc) =
                                        *reinterpret_cast<const float4 *>(sRed + e);
                            }
                        } else {
#pragma unroll 4
                            for (int q = 0; q < (K::WK * K::CC * K::BM) / K::NT; ++q) {
                                const int e = tid + q * K::NT;
                                const int slot = e / K::BM;
                                const int row = e - slot * K::BM;
                                const int c = (slot / K::CC) * K::KCW + r0 + (slot % K::CC);
                                if (c < p.k && row0 + row < p.m) C[row0 + row + (int64_t)c * ldc] = sRed[e];
                            }
                        }
                    }
                }
            } else if constexpr (K::WC == 1) {
                if (whole) {
                    // Not conditional on `aborted`: after a timeout C is undefined
                    // anyway (the host reports the error), both branches stay
                    // inside C, and a guard here makes ptxas spill the 128
                    // accumulators of the wide TSM2L shapes.
                    {
                        // Fast path: the row block lies inside C, all its columns are
                        // live and C allows 16-byte stores: unpredicated vector stores.
                        const bool vrows = p.c_vec && row0 + K::BM <= p.m;  // whole 16-byte row vectors
                        const bool fast = vrows && kbase + K::KCW <= p.k;
                        const int64_t ldc = *s_ldc;
                        T *cw = C + row0 + (int64_t)kbase * ldc;
                        if (fast) {
#pragma unroll
                            for (int c = 0; c < K::KCW; ++c) {
#pragma unroll
                                for (int v = 0; v < K::NV; ++v) {
                                    T tmp[K::V];
#pragma unroll
                                    for (int e = 0; e < K::V; ++e) tmp[e] = acc[v * K::V + e][c];
                                    if (dbg_in_bounds(row0 + row_of(v) + K::V - 1 < p.m && kbase + c < p.k, p.status))
                                        *reinterpret_cast<vec_t *>(cw + row_of(v)) = K::VT::make(tmp);
                                }
                                cw += ldc;
                            }
                        } else if (vrows) {
                            // Columns past k skipped, rows still whole vectors.
#pragma unroll
                            for (int c = 0; c < K::KCW; ++c) {
                                if (kbase + c < p.k) {
#pragma unroll
                                    for (int v = 0; v < K::NV; ++v) {
                                        T tmp[K::V];
#pragma unroll
                                        for (int e = 0; e < K::V; ++e) tmp[e] = acc[v * K::V + e][c];
                                        if (dbg_in_bounds(row0 + row_of(v) + K::V - 1 < p.m, p.status))
                                            *reinterpret_cast<vec_t *>(cw + row_of(v)) = K::VT::make(tmp);
                                    }
                                }
                                cw += ldc;
                            }
                        } else {
#pragma unroll
                            for (int c = 0; c < K::KCW; ++c) {
                                if (kbase + c < p.k) {
#pragma unroll
                                    for (int v = 0; v < K::NV; ++v)
#pragma unroll
                                        for (int e = 0; e < K::V; ++e)
                                            if (row0 + row_of(v) + e < p.m) cw[row_of(v) + e] = acc[v * K::V + e][c];
                                }
                                cw += ldc;
                            }
                        }
                    }
                } else if constexpr (!K::WHOLE) {
                    // Partial sums in registers -> slot [KC][BM] at this lane's rows.
                    T *slot = ws + my_slot * (int64_t)(K::KC * K::BM);
#pragma unroll
                    for (int v = 0; v < K::NV; ++v)
#pragma unroll
                        for (int c = 0; c < K::KC; ++c) {
                            T tmp[K::V];
#pragma unroll
                            for (int e = 0; e < K::V; ++e) tmp[e] = acc[v * K::V + e][c];
                            if (dbg_in_bounds(my_slot < G + (p.m + K::BM - 1) / K::BM, p.status))
                                __stcg(reinterpret_cast<vec_t *>(slot + c * K::BM + row_of(v)), K::VT::make(tmp));
                        }
                }
            } else {
                // Cross-warp reduction in shared memory, CC columns per round,
                // fixed order wc = 0 .. WC-1; output in the canonical layout
                // e = c * BM + row, element e handled by consumer thread e % NT.
                T *slot = ws + my_slot * (int64_t)(K::KC * K::BM);
#pragma unroll
                for (int c0 = 0; c0 < K::KC; c0 += K::CC) {
                    named_bar_sync(1, K::NT);
#pragma unroll
                    for (int cc = 0; cc < K::CC; ++cc)
#pragma unroll
                        for (int v = 0; v < K::NV; ++v) {
                            T tmp[K::V];
#pragma unroll
                            for (int e = 0; e < K::V; ++e) tmp[e] = acc[v * K::V + e][c0 + cc];
                            *reinterpret_cast<vec_t *>(sRed + (wc * K::CC + cc) * K::BM + row_of(v)) = K::VT::make(tmp);
                        }
                    named_bar_sync(1, K::NT);
#pragma unroll
                    for (int q = 0; q < (K::CC * K::BM) / K::NT; ++q) {
                        const int e = tid + q * K::NT;
                        const int cc = e / K::BM;
                        const int row = e - cc * K::BM;
                        T sum = sRed[cc * K::BM + row];
#pragma unroll
                        for (int w2 = 1; w2 < K::WC; ++w2) sum += sRed[(w2 * K::CC + cc) * K::BM + row];
                        const int c = c0 + cc;
                        if (whole) {
                            if (!aborted && c < p.k && row0 + row < p.m) C[row0 + row + (int64_t)c * p.ldc] = sum;
                        } else if (dbg_in_bounds(my_slot < G + (p.m + K::BM - 1) / K::BM, p.status)) {
                            __stcg(slot + c * K::BM + row, sum);
                        }
                    }
                }
            }

            if (!K::WHOLE && !whole) {
                // Publish this piece; the last arriving block of the row block
                // adds all pieces in block order and writes C.
                __threadfence();
                named_bar_sync(1, K::NT);
                if (tid == 0) {
                    int last = 0;
                    if (!flags[0] && dbg_in_bounds(rb64 < (p.m + K::BM - 1) / K::BM, p.status)) {
                        const int npieces = (int)(gB - gA + 1);
                        const int old = atomicAdd(&p.counters[rb], 1);
                        last = (old == npieces - 1);
                        if (last) p.counters[rb] = 0;  // ready for the next launch
                    }
                    flags[1] = last;
                }
                named_bar_sync(1, K::NT);
                if (flags[1] && dbg_in_bounds(gA >= 0 && gB + rb64 < G + (p.m + K::BM - 1) / K::BM, p.status)) {
                    __threadfence();
                    if constexpr (K::WC == 1) {
#pragma unroll
                        for (int v = 0; v < K::NV; ++v)
#pragma unroll
                            for (int c = 0; c < K::KC; ++c) {
                                T sum[K::V];
                                for (int64_t gp = gA; gp <= gB; ++gp) {
                                    const vec_t x = __ldcg(reinterpret_cast<const vec_t *>(
                                        ws + (gp + rb64) * (int64_t)(K::KC * K::BM) + c * K::BM + row_of(v)));
#pragma unroll
                                    for (int e = 0; e < K::V; ++e)
                                        sum[e] = (gp == gA) ? K::VT::get(x, e) : sum[e] + K::VT::get(x, e);
                                }
                                const int64_t r0 = row0 + row_of(v);
                                if (c < p.k)
#pragma unroll
                                    for (int e = 0; e < K::V; ++e)
                                        if (r0 + e < p.m) C[r0 + e + (int64_t)c * p.ldc] = sum[e];
                            }
                    } else {
                        // All of a piece's loads are issued together (independent
                        // L2 round trips in flight), pieces added in block order.
                        constexpr int E = (K::KC * K::BM) / K::NT;
                        T sum[E];
                        const T *src = ws + (gA + rb64) * (int64_t)(K::KC * K::BM) + tid;
#pragma unroll
                        for (int q = 0; q < E; ++q) sum[q] = __ldcg(src + q * K::NT);
                        for (int64_t gp = gA + 1; gp <= gB; ++gp) {
                            src += K::KC * K::BM;
                            T x[E];
#pragma unroll
                            for (int q = 0; q < E; ++q) x[q] = __ldcg(src + q * K::NT);
#pragma unroll
                            for (int q = 0; q < E; ++q) sum[q] += x[q];
                        }
#pragma unroll
                        for (int q = 0; q < E; ++q) {
                            const int e = tid + q * K::NT;
                            const int c = e / K::BM;
                            const int row = e - c * K::BM;
                            if (c < p.k && row0 + row < p.m) C[row0 + row + (int64_t)c * p.ldc] = sum[q];
                        }
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < K::R; ++r)
#pragma unroll
                for (int c = 0; c < K::KCW; ++c) acc[r][c] = T(0);
            piece_at_rb_start = true;
        }
        if (++jc == upr) { jc = 0; ++rb; }
    }
    if (p.trace && threadIdx.x == 128) p.trace[4 * g + 2] = globaltimer_ns();
}

// ---------------------------------------------------------------------------
// Host side: compiled configurations and launch.

template <class K>
cudaError_t launch_cfg(const StreamLaunch &L, cudaStream_t stream) {
    static std::mutex mu;
    static uint64_t attr_done = 0;  // one bit per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (dev < 64 && !(attr_done & (1ull << dev))) {
            e = cudaFuncSetAttribute(stream_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::SMEM);
            if (e != cudaSuccess) return e;
            attr_done |= 1ull << dev;
        }
    }
    Params p;
    p.m = L.g.m;
    p.n = L.g.n;
    p.k = L.g.k;
    p.B = L.g.B;
    p.ldb = L.g.ldb;
    p.C = L.g.C;
    p.ldc = L.g.ldc;
    p.ws = L.ws;
    p.counters = K::DYN ? L.claims : L.counters;
    p.status = L.status;
    p.wait_ns = L.wait_ns;
    const int64_t num_rb = (L.g.m + K::BM - 1) / K::BM;
    p.upr = (L.g.n + K::BNS - 1) / K::BNS;
    p.gran = K::WHOLE ? p.upr : 1;  // TSM2L schedules keep row blocks whole
    p.ngroups = num_rb * p.upr / p.gran;
    p.c_vec = L.c_vec ? 1 : 0;
    p.trace = L.trace;
    stream_kernel<K><<<L.grid, K::THREADS, K::SMEM, stream>>>(L.mapA, L.mapB, p);
    return cudaGetLastError();
}

template <class K>
StreamShape shape_of(const char *name) {
    StreamShape s;
    s.name = name;
    s.elem = (int)sizeof(typename K::T);
    s.KC = K::KC;
    s.BM = K::BM;
    s.BNS = K::BNS;
    s.BOXM = K::BOXM;
    s.gran_rows = K::WHOLE ? 0 : 1;
    s.b_resident = K::BRES;
    s.n_max_resident = K::NRES;
    s.smem_bytes = (int)K::SMEM;
    s.threads = K::THREADS;
    return s;
}

struct Entry {
    char op;  // 'r': TSM2R schedule, 'l': TSM2L, 'w': TSM2L with 8 rows per lane, 't': TSM2L with staged B
    StreamShape shape;
    cudaError_t (*launch)(const StreamLaunch &, cudaStream_t);
};

#define TSM2_ENTRY(OP, CFG, NAME) Entry{OP, shape_of<CFG>(NAME), &launch_cfg<CFG>}

const Entry kEntries[] = {
    TSM2_ENTRY('r', R32<2>, "r_f32_kc2"),    TSM2_ENTRY('r', R32<4>, "r_f32_kc4"),
    TSM2_ENTRY('r', R32<8>, "r_f32_kc8"),    TSM2_ENTRY('r', R32<12>, "r_f32_kc12"),
    TSM2_ENTRY('r', R32<16>, "r_f32_kc16"),  TSM2_ENTRY('r', R64<2>, "r_f64_kc2"),
    TSM2_ENTRY('r', R64<4>, "r_f64_kc4"),    TSM2_ENTRY('r', R64<8>, "r_f64_kc8"),
    TSM2_ENTRY('r', R64<12>, "r_f64_kc12"),  TSM2_ENTRY('r', R64<16>, "r_f64_kc16"),
    TSM2_ENTRY('l', L32<2>, "l_f32_kc2"),    TSM2_ENTRY('l', L32<4>, "l_f32_kc4"),
    TSM2_ENTRY('l', L32<8>, "l_f32_kc8"),    TSM2_ENTRY('l', L32<12>, "l_f32_kc12"),
    TSM2_ENTRY('l', L32<16>, "l_f32_kc16"),  TSM2_ENTRY('l', L32<24>, "l_f32_kc24"),
    TSM2_ENTRY('l', L32<32>, "l_f32_kc32"),  TSM2_ENTRY('l', L64<2>, "l_f64_kc2"),
    TSM2_ENTRY('l', L64<4>, "l_f64_kc4"),    TSM2_ENTRY('l', L64<8>, "l_f64_kc8"),
    TSM2_ENTRY('l', L64<12>, "l_f64_kc12"),  TSM2_ENTRY('l', L64<16>, "l_f64_kc16"),
    TSM2_ENTRY('l', L64<24>, "l_f64_kc24"),  TSM2_ENTRY('l', L64<32>, "l_f64_kc32"),
    TSM2_ENTRY('w', W32<24>, "lw_f32_kc24"), TSM2_ENTRY('w', W32<32>, "lw_f32_kc32"),
    TSM2_ENTRY('t', T32<4>, "lt_f32_kc4"),   TSM2_ENTRY('t', T32<8>, "lt_f32_kc8"),
    TSM2_ENTRY('t', T32<12>, "lt_f32_kc12"), TSM2_ENTRY('t', T32<16>, "lt_f32_kc16"),
    TSM2_ENTRY('t', T32<24>, "lt_f32_kc24"), TSM2_ENTRY('t', T32<32>, "lt_f32_kc32"),
    TSM2_ENTRY('t', T64<4>, "lt_f64_kc4"),   TSM2_ENTRY('t', T64<8>, "lt_f64_kc8"),
    TSM2_ENTRY('t', T64<12>, "lt_f64_kc12"), TSM2_ENTRY('t', T64<16>, "lt_f64_kc16"),
    TSM2_ENTRY('t', T64<24>, "lt_f64_kc24"), TSM2_ENTRY('t', T64<32>, "lt_f64_kc32"),
};


}  // namespace

const StreamShape *stream_shape(int elem, char op, int kc) {
    for (const Entry &en : kEntries)
        if (en.shape.elem == elem && en.op == op && en.shape.KC == kc) return &en.shape;
    return nullptr;
}

cudaError_t stream_launch(const StreamShape *shape, const StreamLaunch &L, cudaStream_t stream) {
    for (const Entry &en : kEntries)
        if (&en.shape == shape) return en.launch(L, stream);
    return cudaErrorInvalidValue;
}

}  // namespace tsm2
