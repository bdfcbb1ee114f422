// Persistent kernel for batches of uneven TSM2R / TSM2L problems (binary32),
// over a list of tile classes.
//
// A tile class (schedule and C-column width KC, a Cfg<> from tsm2_cfg.cuh)
// numbers the work groups of all of its problems end to end: a TSM2R problem
// contributes one group per pipeline stage (a BM x BNS tile of A), a TSM2L
// problem one group per row block.  For every class of the list, block g of
// the persistent grid takes the groups [g*NG/G, (g+1)*NG/G) of that class,
// crossing problem boundaries as it goes (the stream-K partition of the
// single-problem kernel applied to the whole batch); it then moves on to its
// share of the next class without waiting for the other blocks.  One launch
// with a list of several classes therefore runs a whole mixed batch; a list
// of one class is the per-class kernel.
//
// All classes of a list share one ring of shared-memory stages (the stage
// buffers are sized for the largest class) and one set of full / empty
// barriers; the producer lane, the three B-loader warps and the consumer
// warps walk the same sequence of stages, so a stage of the next class can be
// in flight while the consumers finish the previous class.  Partial sums of
// split row blocks go to per-class workspace slots and the last arriving
// block adds them in a fixed order: results do not depend on the grid's
// timing.
//
// This is Algorithm 5's idea (fewer, longer-lived threads walking over
// tiles, Sec. 3.2.2) taken across problems and across tile classes.
#pragma once

#include "common.cuh"
#include "internal.h"
#include "tsm2_cfg.cuh"

#include <mutex>

namespace tsm2 {

constexpr size_t smax() { return 0; }
template <class... X>
constexpr size_t smax(size_t a, X... rest) {
    const size_t b = smax(rest...);
    return a > b ? a : b;
}

template <class K0, class... Ks>
struct BatchLayout {
    static constexpr int STAGES = K0::STAGES;
    static_assert(((Ks::STAGES == STAGES) && ...), "the classes of one kernel share the stage ring");
    static_assert(sizeof(typename K0::T) == 4 && ((sizeof(typename Ks::T) == 4) && ...), "binary32 classes");
    static_assert(K0::NW == 8 && ((Ks::NW == 8) && ...), "eight consumer warps");
    static_assert(STAGES >= 3, "loader warps take every third stage");
    static constexpr size_t A_BYTES = align_up(smax(K0::A_STAGE * 4, Ks::A_STAGE * 4 ...), 128);
    static constexpr size_t B_BYTES = align_up(smax(K0::B_STAGE * 4, Ks::B_STAGE * 4 ...), 128);
    static constexpr size_t BROW_BYTES = align_up(smax(K0::BROW_STAGE * 4, Ks::BROW_STAGE * 4 ...), 16);
    static constexpr size_t BRES_BYTES = align_up(smax(K0::BRES_ELEMS * 4, Ks::BRES_ELEMS * 4 ...), 16);
    static constexpr size_t RED_BYTES = align_up(smax(K0::RED * 4, Ks::RED * 4 ...), 16);
    static constexpr size_t OFF_A = 0;
    static constexpr size_t OFF_B = OFF_A + STAGES * A_BYTES;
    static constexpr size_t OFF_BROW = OFF_B + STAGES * B_BYTES;
    static constexpr size_t OFF_BRES = OFF_BROW + STAGES * BROW_BYTES;
    static constexpr size_t OFF_RED = OFF_BRES + BRES_BYTES;
    static constexpr size_t OFF_BAR = align_up(OFF_RED + RED_BYTES, 16);
    // full, empty and meta barriers (STAGES each), then the stage records
    static constexpr size_t OFF_META = OFF_BAR + 3 * STAGES * sizeof(uint64_t);
    static constexpr size_t OFF_FLAGS = OFF_META + STAGES * 32;
    // This block's weighted share of the TSM2L classes: Q below, Q below +
    // own, Q total (0: equal shares), launch epoch.
    static constexpr size_t OFF_WSH = OFF_FLAGS + 32;
    static constexpr size_t SMEM = OFF_WSH + 32 + 128;  // + slack for 128-byte alignment
    static_assert(SMEM <= 227 * 1024, "shared memory per block");
};

// What the producer lane tells the loader warps about a stage: the class
// (its index in the kernel's list) and, for classes that load B, where the
// stage's rows of B start.
struct StageMeta {
    const float *b;  // B + j0 (first row of the stage), or nullptr: nothing to load
    int64_t ldb;
    int32_t rows;    // rows of B left from j0 (n - j0)
    int32_t k;
    int32_t cls;
    int32_t pad;
};
static_assert(sizeof(StageMeta) == 32, "stage record size");

// Block g's share of a class: groups [g*NG/Gc, (g+1)*NG/Gc) with
// Gc = min(grid, NG).  With more blocks than groups only the first NG blocks
// take one group each, so every block between the first and last owner of a
// split row block has written its partial sum (the fix-up adds them all).
// TSM2L classes (whole row blocks) with adaptive weights (wsh[2] > 0): groups
// [NG*Qb/Qt, NG*(Qb+Qg)/Qt), where Qb is the sum of the integer weights of the
// blocks before g; every block computes the same integer prefix sums, so the
// shares tile the class exactly.
__device__ __forceinline__ bool class_share(const ClassParams &cp, const int64_t *wsh, int64_t &Gc, int64_t &gs,
                                            int64_t &ge) {
    const int64_t G = gridDim.x, g = blockIdx.x;
    if (cp.whole && wsh[2] > 0) {
        Gc = G;
        gs = cp.ngroups * wsh[0] / wsh[2];
        ge = cp.ngroups * wsh[1] / wsh[2];
        return gs < ge;
    }
    Gc = G < cp.ngroups ? G : cp.ngroups;
    if (g >= Gc) return false;
    gs = g * cp.ngroups / Gc;
    ge = (g + 1) * cp.ngroups / Gc;
    return gs < ge;
}

__device__ __forceinline__ int find_problem(const ProbDesc *probs, int nprob, int64_t gidx) {
    int lo = 0, hi = nprob - 1;  // last problem with group_begin <= gidx
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (probs[mid].group_begin <= gidx) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Walk over one block's share of a class: problem, row block and stage of
// every unit, stepped unit by unit (the descriptor is read again only at a
// change of problem).
struct Walk {
    const ProbDesc *probs;
    int nprob;
    int64_t ngroups;
    int pi;
    const ProbDesc *pd;
    int64_t next_begin;
    int upr, gran, rb, jc;

    __device__ __forceinline__ void start(const ClassParams &cp, int64_t gs) {
        probs = cp.probs;
        nprob = cp.nprob;
        ngroups = cp.ngroups;
        pi = find_problem(probs, nprob, gs);
        pd = &probs[pi];
        next_begin = (pi + 1 < nprob) ? probs[pi + 1].group_begin : ngroups;
        upr = pd->upr;
        gran = pd->gran;
        rb = (int)(gs - pd->group_begin) * gran / upr;
        jc = (int)(gs - pd->group_begin) * gran - rb * upr;
    }
    // At the first unit of group gg: move to the problem that owns it.
    // Returns true when the problem changed.
    __device__ __forceinline__ bool enter(int64_t gg) {
        if (gg < next_begin) return false;
        do {
            ++pi;
            next_begin = (pi + 1 < nprob) ? probs[pi + 1].group_begin : ngroups;
        } while (gg >= next_begin);
        pd = &probs[pi];
        upr = pd->upr;
        gran = pd->gran;
        rb = 0;
        jc = 0;
        return true;
    }
    __device__ __forceinline__ void step() {
        if (++jc == upr) { jc = 0; ++rb; }
    }
};

struct Ring {
    int s = 0;
    uint32_t ph = 0;
    template <int STAGES>
    __device__ __forceinline__ void next() {
        if (++s == STAGES) { s = 0; ph ^= 1u; }
    }
};

template <class K, class LY>
__device__ __forceinline__ void produce_class(const ClassParams &cp, int cls, unsigned char *smem, uint64_t *full,
                                              uint64_t *empty, uint64_t *metab, volatile int *flags,
                                              const BatchKParams &p, Ring &ring, uint32_t &issued,
                                              uint32_t &last_par, bool &stop, uint64_t policy) {
    int64_t Gc, gs, ge;
    if (stop || !class_share(cp, reinterpret_cast<const int64_t *>(smem + LY::OFF_WSH), Gc, gs, ge)) return;
    Walk w;
    w.start(cp, gs);
    for (int64_t gg = gs; gg < ge && !stop; ++gg) {
        w.enter(gg);
        for (int t = 0; t < w.gran; ++t) {
            const int s = ring.s;
            if (flags[0] || !mbar_wait_bounded(&empty[s], ring.ph ^ 1u, p.wait_ns, flags)) {
                flags[0] = 1;
                atomicOr(p.status, kStatusTimeout);
                stop = true;
                break;
            }
            const int32_t x0 = w.rb * K::BM, y0 = w.jc * K::BNS;
            StageMeta *meta = reinterpret_cast<StageMeta *>(smem + LY::OFF_META) + s;
            meta->b = K::BLOAD ? static_cast<const float *>(w.pd->B) + y0 : nullptr;
            meta->ldb = w.pd->ldb;
            meta->rows = (int32_t)(w.pd->n - y0);
            meta->k = w.pd->k;
            meta->cls = cls;
            mbar_arrive(&metab[s]);  // publishes the record to the loader warp of this stage
            mbar_arrive_expect_tx(&full[s], K::TX_BYTES);
            float *dstA = reinterpret_cast<float *>(smem + LY::OFF_A + (size_t)s * LY::A_BYTES);
#pragma unroll
            for (int q = 0; q < K::NBOX; ++q)
                tma_load_2d_hint(dstA + q * K::BOXM * K::BNS, &w.pd->mapA, x0 + q * K::BOXM, y0, &full[s], policy);
            if constexpr (!K::BRES && !K::BLOAD)  // B rows of the stage, column-major
                tma_load_2d(smem + LY::OFF_B + (size_t)s * LY::B_BYTES, &w.pd->mapB, y0, 0, &full[s]);
            issued |= 1u << s;
            last_par = (last_par & ~(1u << s)) | (ring.ph << s);
            ring.next<LY::STAGES>();
            w.step();
        }
    }
}

// Stages a block runs in one class: whole groups of gran stages each.
__device__ __forceinline__ int64_t class_units(const ClassParams &cp, const int64_t *wsh) {
    int64_t Gc, gs, ge;
    if (!class_share(cp, wsh, Gc, gs, ge)) return 0;
    int64_t units = 0;
    for (int pi = find_problem(cp.probs, cp.nprob, gs); pi < cp.nprob; ++pi) {
        const ProbDesc &d = cp.probs[pi];
        const int64_t b0 = d.group_begin > gs ? d.group_begin : gs;
        const int64_t nb = pi + 1 < cp.nprob ? cp.probs[pi + 1].group_begin : cp.ngroups;
        const int64_t b1 = nb < ge ? nb : ge;
        if (b0 >= ge) break;
        if (b1 > b0) units += (b1 - b0) * d.gran;
    }
    return units;
}

template <class K>
__device__ __forceinline__ void load_if(bool hit, const StageMeta &m, float *brow, int lane, unsigned *status) {
    if constexpr (K::BLOAD)
        if (hit) load_b_stage<K>(m.b, m.ldb, m.rows, m.k, 0, brow, lane, status);
}

// Loader warps 1..3 of the producer warpgroup: warp w takes every third stage
// of the block's whole walk.  It waits for the producer lane's record of the
// stage, loads the stage's B rows when the class reads streamed B row-major,
// and arrives on the stage's full barrier (which takes the producer lane's
// copy and one loader arrival).
template <class LY, class... Ks>
__device__ __forceinline__ void loader_warp(const BatchKParams &p, unsigned char *smem, uint64_t *full,
                                            uint64_t *metab, volatile int *flags, int w, int lane) {
    int total = 0;  // a block's stages: far below 2^31
    int ci = 0;
    const int64_t *wsh = reinterpret_cast<const int64_t *>(smem + LY::OFF_WSH);
    ((total += (int)class_units(p.cls[ci++], wsh), (void)sizeof(Ks)), ...);
    int s = w, ph = 0;  // stage and parity of unit u, stepped by 3
    for (int u = w; u < total; u += 3) {
        bool ok = !flags[0] && mbar_wait_bounded(&metab[s], (uint32_t)ph, p.wait_ns, flags);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) {
            if (lane == 0) {
                flags[0] = 1;
                atomicOr(p.status, kStatusTimeout);
            }
            return;
        }
        const StageMeta &m = reinterpret_cast<const StageMeta *>(smem + LY::OFF_META)[s];
        if (m.b) {
            float *brow = reinterpret_cast<float *>(smem + LY::OFF_BROW + (size_t)s * LY::BROW_BYTES);
            int c = 0;
            (load_if<Ks>(c++ == m.cls, m, brow, lane, p.status), ...);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&full[s]);
        s += 3;
        if (s >= LY::STAGES) {
            s -= LY::STAGES;
            ph ^= 1;
        }
    }
}

template <class K, class LY>
__device__ __forceinline__ void consume_class(const ClassParams &cp, unsigned char *smem, uint64_t *full,
                                              uint64_t *empty, volatile int *flags, const BatchKParams &p,
                                              Ring &ring, bool &aborted, unsigned long long &lstart,
                                              long long &lunits) {
    using T = float;
    using vec_t = typename K::vec_t;
    if constexpr (K::BRES) {
        if (p.bal && lstart == 0) lstart = globaltimer_ns();  // the block reached its TSM2L work
    }
    int64_t G, gs, ge;  // G: the blocks that share this class
    if (!class_share(cp, reinterpret_cast<const int64_t *>(smem + LY::OFF_WSH), G, gs, ge)) return;
    if constexpr (K::BRES) lunits += class_units(cp, reinterpret_cast<const int64_t *>(smem + LY::OFF_WSH));
    const int64_t g = blockIdx.x;
    T *sBres = reinterpret_cast<T *>(smem + LY::OFF_BRES);
    T *sRed = reinterpret_cast<T *>(smem + LY::OFF_RED);
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int cwarp = warp - 4;
    const int wk = cwarp % K::WK;
    const int wc = (cwarp / K::WK) % K::WC;
    const int wr = cwarp / (K::WK * K::WC);
    const int kbase = wk * K::KCW;
    const int tid = threadIdx.x - 128;
    T acc[K::R][K::KCW];
#pragma unroll
    for (int r = 0; r < K::R; ++r)
#pragma unroll
        for (int c = 0; c < K::KCW; ++c) acc[r][c] = T(0);
    auto row_of = [&](int v) { return wr * 32 * K::R + v * 32 * K::V + lane * K::V; };

    Walk w;
    w.start(cp, gs);
    bool load_b = true;
    for (int64_t gg = gs; gg < ge; ++gg) {
        if (w.enter(gg)) load_b = true;
        if constexpr (K::BRES) {
            if (load_b) {
                // Resident B of this problem; every warp finished the previous
                // problem's last piece (its epilogue) before reaching here.
                named_bar_sync(1, K::NT);
                load_resident_b<K>(sBres, static_cast<const T *>(w.pd->B), w.pd->n, w.pd->k, w.pd->ldb, tid);
                named_bar_sync(1, K::NT);
            }
        }
        load_b = false;
        for (int t = 0; t < w.gran; ++t) {
            const int s = ring.s;
            if (!aborted) {
                bool ok = !flags[0] && mbar_wait_bounded(&full[s], ring.ph, p.wait_ns, flags);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) {
                    aborted = true;
                    if (lane == 0) {
                        flags[0] = 1;
                        atomicOr(p.status, kStatusTimeout);
                    }
                }
            }
            if (!aborted) {
                const T *a_st = reinterpret_cast<const T *>(smem + LY::OFF_A + (size_t)s * LY::A_BYTES);
                const T *b_st;
                int bstride;
                if constexpr (K::BRES) {
                    b_st = resident_b_stage<K>(sBres, w.jc);
                    bstride = K::NRES;
                } else if constexpr (K::BLOAD) {
                    b_st = reinterpret_cast<const T *>(smem + LY::OFF_BROW + (size_t)s * LY::BROW_BYTES);
                    bstride = K::BROWS;
                } else {
                    b_st = reinterpret_cast<const T *>(smem + LY::OFF_B + (size_t)s * LY::B_BYTES);
                    bstride = K::BNS;
                }
                consume_stage<K>(a_st, b_st, bstride, wc, kbase, row_of(0), acc);
            }
            if (!aborted) {
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[s]);
            }
            ring.next<LY::STAGES>();

            const bool rb_end = (w.jc == w.upr - 1);
            const bool last = (gg == ge - 1) && (t == w.gran - 1);
            if (rb_end || last) {
                // ---- epilogue of one piece of row block rb of problem pi ----
                const ProbDesc *pd = w.pd;
                const int upr = w.upr, gran = w.gran;
                const int64_t rb64 = w.rb;
                // First and last group of rb: a group is one stage (gran 1) or
                // a whole row block (gran upr).
                const int64_t rb_g0 = pd->group_begin + (gran == 1 ? rb64 * upr : rb64);
                const int64_t rb_g1 = pd->group_begin + (gran == 1 ? rb64 * upr + upr - 1 : rb64);
                // TSM2L classes (WC == 1) take whole row blocks only; saying
                // so at compile time also keeps ptxas from spilling their
                // wide accumulator tiles.
                const bool whole = K::WC == 1 || ((rb_g0 >= gs) && rb_end);
                const int64_t row0 = rb64 * K::BM;
                const int64_t m = pd->m;
                const int kk = pd->k;
                const int64_t ldc = pd->ldc;
                T *C = static_cast<T *>(pd->C);
                const int64_t rbg = pd->rb_begin + rb64;  // row block of the class: counters and slots
                T *ws = cp.ws;
                if constexpr (K::WC == 1) {
                    // Not conditional on `aborted`: after a timeout C is
                    // undefined anyway (the host reports the error), every
                    // store stays inside C, and the guard makes ptxas spill
                    // wide accumulator tiles.
                    if (whole) {
                        T *cw = C + row0 + (int64_t)kbase * ldc;
                        const bool vrows = pd->c_vec && row0 + K::BM <= m;  // whole 16-byte row vectors
                        const bool fast = vrows && kbase + K::KCW <= kk;
                        if (fast) {
#pragma unroll
                            for (int c = 0; c < K::KCW; ++c) {
#pragma unroll
                                for (int v = 0; v < K::NV; ++v) {
                                    T tmp[K::V];
#pragma unroll
                                    for (int e = 0; e < K::V; ++e) tmp[e] = acc[v * K::V + e][c];
                                    if (dbg_in_bounds(row0 + row_of(v) + K::V - 1 < m && kbase + c < kk, p.status))
                                        *reinterpret_cast<vec_t *>(cw + row_of(v)) = K::VT::make(tmp);
                                }
                                cw += ldc;
                            }
                        } else if (vrows) {
                            // Columns past k skipped, rows still whole vectors.
#pragma unroll
                            for (int c = 0; c < K::KCW; ++c) {
                                if (kbase + c < kk) {
#pragma unroll
                                    for (int v = 0; v < K::NV; ++v) {
                                        T tmp[K::V];
#pragma unroll
                                        for (int e = 0; e < K::V; ++e) tmp[e] = acc[v * K::V + e][c];
                                        if (dbg_in_bounds(row0 + row_of(v) + K::V - 1 < m, p.status))
                                            *reinterpret_cast<vec_t *>(cw + row_of(v)) = K::VT::make(tmp);
                                    }
                                }
                                cw += ldc;
                            }
                        } else {
#pragma unroll
                            for (int c = 0; c < K::KCW; ++c) {
                                if (kbase + c < kk) {
#pragma unroll
                                    for (int v = 0; v < K::NV; ++v)
#pragma unroll
                                        for (int e = 0; e < K::V; ++e)
                                            if (row0 + row_of(v) + e < m) cw[row_of(v) + e] = acc[v * K::V + e][c];
                                }
                                cw += ldc;
                            }
                        }
                    }
                } else {
                    T *slot = ws + (g + rbg) * (int64_t)(K::KC * K::BM);
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
                                *reinterpret_cast<vec_t *>(sRed + (wc * K::CC + cc) * K::BM + row_of(v)) =
                                    K::VT::make(tmp);
                            }
                        named_bar_sync(1, K::NT);
#pragma unroll
                        for (int q = 0; q < (K::CC * K::BM) / K::NT; ++q) {
                            const int e = tid + q * K::NT;
                            const int cc = e / K::BM, row = e - (e / K::BM) * K::BM;
                            T sum = sRed[cc * K::BM + row];
#pragma unroll
                            for (int w2 = 1; w2 < K::WC; ++w2) sum += sRed[(w2 * K::CC + cc) * K::BM + row];
                            const int c = c0 + cc;
                            if (whole) {
                                if (!aborted && c < kk && row0 + row < m) C[row0 + row + (int64_t)c * ldc] = sum;
                            } else if (dbg_in_bounds(g + rbg < G + cp.nrb, p.status)) {
                                __stcg(slot + c * K::BM + row, sum);
                            }
                        }
                    }
                    if (!whole) {
                        const int64_t gA = owner_of(rb_g0, G, cp.ngroups);
                        const int64_t gB = owner_of(rb_g1, G, cp.ngroups);
                        __threadfence();
                        named_bar_sync(1, K::NT);
                        if (tid == 0) {
                            int lastp = 0;
                            if (!flags[0] && dbg_in_bounds(rbg >= 0 && rbg < cp.nrb, p.status)) {
                                const int old = atomicAdd(&cp.counters[rbg], 1);
                                lastp = (old == (int)(gB - gA));
                                if (lastp) cp.counters[rbg] = 0;
                            }
                            flags[1] = lastp;
                        }
                        named_bar_sync(1, K::NT);
                        if (flags[1] && dbg_in_bounds(gA >= 0 && gB + rbg < G + cp.nrb, p.status)) {
                            __threadfence();
                            constexpr int E = (K::KC * K::BM) / K::NT;
                            T sum[E];
                            const T *src = ws + (gA + rbg) * (int64_t)(K::KC * K::BM) + tid;
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
                                const int c = e / K::BM, row = e - (e / K::BM) * K::BM;
                                if (c < kk && row0 + row < m) C[row0 + row + (int64_t)c * ldc] = sum[q];
                            }
                        }
                        named_bar_sync(1, K::NT);  // flags[1] is reused by the next piece
                    }
                }
#pragma unroll
                for (int r = 0; r < K::R; ++r)
#pragma unroll
                    for (int c = 0; c < K::KCW; ++c) acc[r][c] = T(0);
            }
            w.step();
        }
    }
}

// Integer share weight of a block (2^16 = an even share), from the float
// weight the previous launch left; bounded to [1/16, 16] of an even share.
__device__ __forceinline__ long long weight_q(float x) {
    if (!(x >= 0.0625f)) x = (x > 0.0f) ? 0.0625f : 1.0f;  // also NaN -> even share
    if (x > 16.0f) x = 16.0f;
    return (long long)(x * 65536.0f + 0.5f);
}

// Warp 1 of every block at launch: this block's share of the TSM2L classes
// from the weights of the running epoch (integer prefix sums, the same in
// every block).
__device__ __forceinline__ void balance_shares(const BatchKParams &p, int64_t *wsh, int lane) {
    const int G = gridDim.x, g = blockIdx.x;
    if (!p.bal || G > kBalanceMaxBlocks) {
        if (lane == 0) wsh[0] = wsh[1] = wsh[2] = wsh[3] = 0;
        return;
    }
    const int e = __ldcg(&p.bal->epoch);
    const float *w = p.bal->w[e & 1];
    long long below = 0, mine = 0, all = 0;
    for (int b = lane; b < G; b += 32) {
        const long long q = weight_q(__ldcg(&w[b]));
        all += q;
        if (b < g) below += q;
        if (b == g) mine = q;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        below += __shfl_xor_sync(0xffffffffu, below, o);
        mine += __shfl_xor_sync(0xffffffffu, mine, o);
        all += __shfl_xor_sync(0xffffffffu, all, o);
    }
    if (lane == 0) {
        wsh[0] = below;
        wsh[1] = below + mine;
        wsh[2] = all;
        wsh[3] = e;
    }
}

// The last block of a launch: weights for the next one.  Block b ran its
// TSM2L stages u_b at rate r_b = u_b / (end_b - start_b) from start_b; all
// blocks finish together at T if block b gets r_b (T - start_b) stages, with
// T fixed by the total.  The new weight is half the old (normalised) and half
// that target; blocks without TSM2L work count at the mean rate.  Warp 4's
// 32 lanes share the blocks.
__device__ __forceinline__ void balance_update(BatchBalance *bal, int e, int lane) {
    const int G = gridDim.x;
    const float *wo = bal->w[e & 1];
    float *wn = bal->w[(e + 1) & 1];
    unsigned long long l0 = ~0ull;
    double U = 0, rs = 0, nv = 0;
    for (int b = lane; b < G; b += 32) {
        const unsigned long long ls = __ldcg(&bal->t_lstart[b]), te = __ldcg(&bal->t_end[b]);
        const long long u = __ldcg(&bal->units[b]);
        l0 = ls < l0 ? ls : l0;
        U += (double)u;
        if (u > 0 && te > ls) {
            rs += (double)u / (double)(te - ls);
            nv += 1;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long x = __shfl_xor_sync(0xffffffffu, l0, o);
        l0 = x < l0 ? x : l0;
        U += __shfl_xor_sync(0xffffffffu, U, o);
        rs += __shfl_xor_sync(0xffffffffu, rs, o);
        nv += __shfl_xor_sync(0xffffffffu, nv, o);
    }
    const bool keep = __ldcg(&bal->bad) != 0 || U <= 0 || nv <= 0;
    const double rmean = nv > 0 ? rs / nv : 1.0;
    auto rate = [&](int b) {
        const unsigned long long ls = __ldcg(&bal->t_lstart[b]), te = __ldcg(&bal->t_end[b]);
        const long long u = __ldcg(&bal->units[b]);
        return (u > 0 && te > ls) ? (double)u / (double)(te - ls) : rmean;
    };
    double R = 0, RL = 0, W = 0;
    for (int b = lane; b < G; b += 32) {
        const double r = rate(b);
        R += r;
        RL += r * (double)(__ldcg(&bal->t_lstart[b]) - l0);
        W += (double)weight_q(__ldcg(&wo[b]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        R += __shfl_xor_sync(0xffffffffu, R, o);
        RL += __shfl_xor_sync(0xffffffffu, RL, o);
        W += __shfl_xor_sync(0xffffffffu, W, o);
    }
    const double Tend = (U + RL) / R;  // common end time (ns after the earliest start)
    const double floor_u = 0.02 * U / G;
    double S = 0;
    for (int b = lane; b < G; b += 32) {
        const double t = rate(b) * (Tend - (double)(__ldcg(&bal->t_lstart[b]) - l0));
        S += t > floor_u ? t : floor_u;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) S += __shfl_xor_sync(0xffffffffu, S, o);
    for (int b = lane; b < G; b += 32) {
        const double old = (double)weight_q(__ldcg(&wo[b])) * G / W;  // mean 1
        double x = old;
        if (!keep) {
            const double t = rate(b) * (Tend - (double)(__ldcg(&bal->t_lstart[b]) - l0));
            x = 0.5 * old + 0.5 * (t > floor_u ? t : floor_u) * G / S;
        }
        wn[b] = (float)x;
    }
}

// Register split of the batch kernel: the producer warpgroup (producer lane
// and loader warps) gets PREG registers per thread, the consumers the rest of
// the launch pool (384 x 168), rounded down to the multiple of 8 that
// setmaxnreg takes.
template <int PREG>
struct BatchRegs {
    static constexpr int P = PREG;
    static constexpr int C = ((384 * 168 - 4 * 32 * PREG) / (8 * 32)) / 8 * 8;
    static_assert(PREG % 8 == 0 && PREG >= 24, "setmaxnreg takes multiples of 8");
    static_assert(4 * 32 * P + 8 * 32 * C <= 384 * 168, "register split exceeds launch pool");
};

template <int PREG, class... Ks>
__global__ void __launch_bounds__(384, 1) batch_kernel(const __grid_constant__ BatchKParams p) {
    using LY = BatchLayout<Ks...>;
    using RG = BatchRegs<PREG>;
    static_assert(sizeof...(Ks) <= kMaxBatchMenu, "classes per kernel");
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = smem_aligned<128>(smem_raw);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + LY::OFF_BAR);
    uint64_t *empty = full + LY::STAGES;
    uint64_t *metab = empty + LY::STAGES;
    volatile int *flags = reinterpret_cast<volatile int *>(smem + LY::OFF_FLAGS);  // [0] abort, [1] last
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    if (warp == 1) balance_shares(p, reinterpret_cast<int64_t *>(smem + LY::OFF_WSH), lane);
    if (threadIdx.x == 0) {
        if (p.trace) p.trace[4 * blockIdx.x] = globaltimer_ns();
        for (int s = 0; s < LY::STAGES; ++s) {
            mbar_init(&full[s], 2);  // the producer lane's copy and one loader warp
            mbar_init(&empty[s], 8);
            mbar_init(&metab[s], 1);
        }
        flags[0] = 0;
        flags[1] = 0;
        fence_mbar_init();
    }
    __syncthreads();

    if (warp < 4) {
        // ---------------- producer warpgroup ----------------
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(RG::P));
        if (warp == 0 && lane == 0) {
            const uint64_t policy = l2_policy_evict_first();
            Ring ring;
            uint32_t issued = 0, last_par = 0;
            bool stop = false;
            int ci = 0;
            ((produce_class<Ks, LY>(p.cls[ci], ci, smem, full, empty, metab, flags, p, ring, issued, last_par,
                                    stop, policy),
              ++ci),
             ...);
            // Let every copy this block started land before the block can exit.
            for (int t = 0; t < LY::STAGES; ++t)
                if (issued & (1u << t)) (void)mbar_wait_bounded(&full[t], (last_par >> t) & 1u, 4000000000LL, nullptr);
        } else if (warp >= 1) {
            loader_warp<LY, Ks...>(p, smem, full, metab, flags, warp - 1, lane);
        }
        return;
    }

    // ---------------- consumers ----------------
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(RG::C));
    Ring ring;
    bool aborted = false;
    unsigned long long lstart = 0;
    long long lunits = 0;
    int ci = 0;
    (consume_class<Ks, LY>(p.cls[ci++], smem, full, empty, flags, p, ring, aborted, lstart, lunits), ...);
    const unsigned long long t_end = globaltimer_ns();
    if (p.trace && threadIdx.x == 128) p.trace[4 * blockIdx.x + 2] = t_end;
    if (p.bal && gridDim.x <= kBalanceMaxBlocks) {
        // Record this block's TSM2L timing; the last block to get here sets
        // the next launch's weights and rearms the counters.
        const int64_t *wsh = reinterpret_cast<const int64_t *>(smem + LY::OFF_WSH);
        named_bar_sync(1, 256);  // every consumer warp is done (flags[1] is free again)
        if (threadIdx.x == 128) {
            const int g = blockIdx.x;
            p.bal->t_lstart[g] = lstart ? lstart : t_end;
            p.bal->t_end[g] = t_end;
            p.bal->units[g] = lunits;
            if (flags[0]) atomicExch(&p.bal->bad, 1);
            __threadfence();
            flags[1] = atomicAdd(&p.bal->done, 1) == (int)gridDim.x - 1;
        }
        named_bar_sync(1, 256);
        if (flags[1] && warp == 4) {
            __threadfence();
            balance_update(p.bal, (int)wsh[3], lane);
            __syncwarp();
            if (lane == 0) {
                __threadfence();
                p.bal->bad = 0;
                p.bal->done = 0;
                p.bal->epoch = (int)wsh[3] + 1;
            }
        }
    }
}

template <int PREG, class... Ks>
cudaError_t launch_batch_kernel(const BatchKParams &p, int grid, cudaStream_t stream) {
    using LY = BatchLayout<Ks...>;
    static std::mutex mu;
    static uint64_t attr_done = 0;  // one bit per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (dev < 64 && !(attr_done & (1ull << dev))) {
            e = cudaFuncSetAttribute(batch_kernel<PREG, Ks...>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)LY::SMEM);
            if (e != cudaSuccess) return e;
            attr_done |= 1ull << dev;
        }
    }
    batch_kernel<PREG, Ks...><<<grid, 384, LY::SMEM, stream>>>(p);
    return cudaGetLastError();
}

// Host-side description of class K.
template <class K>
BatchClass class_of(char op, const char *name) {
    BatchClass c;
    c.op = op;
    c.name = name;
    c.KC = K::KC;
    c.BM = K::BM;
    c.BNS = K::BNS;
    c.BOXM = K::BOXM;
    c.stages = K::STAGES;
    c.rows_per_lane = K::R;
    return c;
}

}  // namespace tsm2
