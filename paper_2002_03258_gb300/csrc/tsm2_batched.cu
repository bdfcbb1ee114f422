// Batched TSM2R / TSM2L: many problems of uneven shape in one persistent
// kernel per tile class (binary32).
//
// The problems of one class (same schedule and C-column width KC) are laid
// end to end in a single numbering of work groups: a TSM2R problem
// contributes one group per pipeline stage (BM x BNS tile of A), a TSM2L
// problem one group per row block (B resident, all of its stages).  Block g of
// the persistent grid takes groups [g*NG/G, (g+1)*NG/G), crossing problem
// boundaries as it goes (the stream-K partition of the single-problem kernel
// applied to the whole batch), so every block gets the same amount of work
// however uneven the problems are.  Problem descriptors, including their
// tensor maps, live in device memory; row blocks are numbered globally, so
// the deterministic last-arriver fix-up of split row blocks works unchanged.
//
// This is Algorithm 5's idea (fewer, longer-lived threads walking over
// tiles, Sec. 3.2.2) taken across problems instead of across the rows of one.
#include "common.cuh"
#include "internal.h"
#include "tsm2_cfg.cuh"

#include <mutex>

namespace tsm2 {
namespace {

struct BatchParams {
    const ProbDesc *probs;
    int nprob;
    int64_t ngroups;  // groups of all problems of the class
    float *ws;
    int *counters;
    unsigned *status;
    int64_t wait_ns;
};

__device__ __forceinline__ int find_problem(const ProbDesc *probs, int nprob, int64_t gidx) {
    int lo = 0, hi = nprob - 1;  // last problem with group_begin <= gidx
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (probs[mid].group_begin <= gidx) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <class K>
__global__ void __launch_bounds__(384, 1) batched_kernel(const BatchParams p) {
    using T = typename K::T;
    using vec_t = typename K::vec_t;
    static_assert(sizeof(T) == 4, "the batched kernel is binary32");
    static_assert(K::WC > 1 || K::BRES, "row-split schedules run whole row blocks only (no partial-sum path)");
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = smem_aligned<128>(smem_raw);
    T *sA = reinterpret_cast<T *>(smem + K::OFF_A);
    T *sB = reinterpret_cast<T *>(smem + K::OFF_B);
    T *sBres = reinterpret_cast<T *>(smem + K::OFF_BRES);
    T *sRed = reinterpret_cast<T *>(smem + K::OFF_RED);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + K::OFF_BAR);
    uint64_t *empty = full + K::STAGES;
    volatile int *flags = reinterpret_cast<volatile int *>(smem + K::OFF_FLAGS);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t G = gridDim.x, g = blockIdx.x;
    const int64_t gs = g * p.ngroups / G;
    const int64_t ge = (g + 1) * p.ngroups / G;

    if (threadIdx.x == 0) {
        for (int s = 0; s < K::STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], K::NW);
        }
        flags[0] = 0;
        flags[1] = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (gs >= ge) return;
    const int pi0 = find_problem(p.probs, p.nprob, gs);

    if (warp < 4) {
        // ---------------- producer ----------------
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kProducerRegs));
        if (warp == 0 && lane == 0) {
            const uint64_t policy = l2_policy_evict_first();
            int s = 0;
            uint32_t ph = 0, issued = 0, last_par = 0;
            int pi = pi0;
            const ProbDesc *pd = &p.probs[pi];
            int64_t next_begin = (pi + 1 < p.nprob) ? p.probs[pi + 1].group_begin : p.ngroups;
            // Row block and stage of the current unit, stepped unit by unit;
            // the descriptor is read again only at a change of problem.
            int upr = pd->upr, gran = pd->gran;
            int rb = (int)(gs - pd->group_begin) * gran / upr;
            int jc = (int)(gs - pd->group_begin) * gran - rb * upr;
            bool stop = false;
            for (int64_t gg = gs; gg < ge && !stop; ++gg) {
                if (gg >= next_begin) {  // the next non-empty problem, from its first unit
                    do {
                        ++pi;
                        next_begin = (pi + 1 < p.nprob) ? p.probs[pi + 1].group_begin : p.ngroups;
                    } while (gg >= next_begin);
                    pd = &p.probs[pi];
                    upr = pd->upr;
                    gran = pd->gran;
                    rb = 0;
                    jc = 0;
                }
                for (int t = 0; t < gran; ++t) {
                    if (flags[0] || !mbar_wait_bounded(&empty[s], ph ^ 1u, p.wait_ns, flags)) {
                        flags[0] = 1;
                        atomicOr(p.status, kStatusTimeout);
                        stop = true;
                        break;
                    }
                    mbar_arrive_expect_tx(&full[s], K::TX_BYTES);
                    T *dstA = sA + (size_t)s * K::A_STAGE;
                    const int32_t x0 = rb * K::BM, y0 = jc * K::BNS;
#pragma unroll
                    for (int q = 0; q < K::NBOX; ++q)
                        tma_load_2d_hint(dstA + q * K::BOXM * K::BNS, &pd->mapA, x0 + q * K::BOXM, y0, &full[s], policy);
                    if constexpr (!K::BRES)  // row-major classes: the packed copy, inner coordinate 0
                        tma_load_2d(sB + (size_t)s * K::B_STAGE, &pd->mapB, K::BT ? 0 : y0, K::BT ? y0 : 0, &full[s]);
                    issued |= 1u << s;
                    last_par = (last_par & ~(1u << s)) | (ph << s);
                    if (++s == K::STAGES) { s = 0; ph ^= 1u; }
                    if (++jc == upr) { jc = 0; ++rb; }
                }
            }
            for (int t = 0; t < K::STAGES; ++t)
                if (issued & (1u << t)) (void)mbar_wait_bounded(&full[t], (last_par >> t) & 1u, 4000000000LL, nullptr);
        }
        return;
    }

    // ---------------- consumers ----------------
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kConsumerRegs));
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

    int s = 0;
    uint32_t ph = 0;
    bool aborted = false;
    int pi = pi0;
    const ProbDesc *pd = &p.probs[pi];
    int64_t next_begin = (pi + 1 < p.nprob) ? p.probs[pi + 1].group_begin : p.ngroups;
    bool load_b = true;
    int upr = pd->upr, gran = pd->gran;  // see the producer: stepped, not recomputed
    int rb = (int)(gs - pd->group_begin) * gran / upr;
    int jc = (int)(gs - pd->group_begin) * gran - rb * upr;
    for (int64_t gg = gs; gg < ge; ++gg) {
        if (gg >= next_begin) {  // the next non-empty problem, from its first unit
            do {
                ++pi;
                next_begin = (pi + 1 < p.nprob) ? p.probs[pi + 1].group_begin : p.ngroups;
            } while (gg >= next_begin);
            pd = &p.probs[pi];
            upr = pd->upr;
            gran = pd->gran;
            rb = 0;
            jc = 0;
            load_b = true;
        }
        if constexpr (K::BRES) {
            if (load_b) {
                // Resident B of this problem; every warp finished the previous
                // problem's last piece (its epilogue) before reaching here.
                named_bar_sync(1, K::NT);
                load_resident_b<K>(sBres, static_cast<const T *>(pd->B), pd->n, pd->k, pd->ldb, tid);
                named_bar_sync(1, K::NT);
            }
        }
        load_b = false;
        for (int t = 0; t < gran; ++t) {
            if (!aborted) {
                bool ok = !flags[0] && mbar_wait_bounded(&full[s], ph, p.wait_ns, flags);
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
                const T *a_st = sA + (size_t)s * K::A_STAGE;
                const T *b_st;
                int bstride;
                if constexpr (K::BRES) {
                    b_st = resident_b_stage<K>(sBres, jc);
                    bstride = K::NRES;
                } else {
                    b_st = sB + (size_t)s * K::B_STAGE;
                    bstride = K::BNS;
                }
                consume_stage<K>(a_st, b_st, bstride, wc, kbase, row_of(0), acc);
            }
            if (!aborted) {
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[s]);
            }
            if (++s == K::STAGES) { s = 0; ph ^= 1u; }

            const bool rb_end = (jc == upr - 1);
            const bool last = (gg == ge - 1) && (t == gran - 1);
            if (rb_end || last) {
                // ---- epilogue of one piece of row block rb of problem pi ----
                const int64_t rb64 = rb;
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
                const int64_t rbg = pd->rb_begin + rb64;  // global row block: counters and slots
                T *ws = p.ws;
                if constexpr (K::WC == 1) {
                    // Not conditional on `aborted`: after a timeout C is
                    // undefined anyway (the host reports the error), both
                    // branches stay inside C, and the guard makes ptxas spill
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
                                *reinterpret_cast<vec_t *>(sRed + (wc * K::CC + cc) * K::BM + row_of(v)) = K::VT::make(tmp);
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
                            } else {
                                __stcg(slot + c * K::BM + row, sum);
                            }
                        }
                    }
                    if (!whole) {
                        const int64_t gA = owner_of(rb_g0, G, p.ngroups);
                        const int64_t gB = owner_of(rb_g1, G, p.ngroups);
                        __threadfence();
                        named_bar_sync(1, K::NT);
                        if (tid == 0) {
                            int lastp = 0;
                            if (!flags[0]) {
                                const int old = atomicAdd(&p.counters[rbg], 1);
                                lastp = (old == (int)(gB - gA));
                                if (lastp) p.counters[rbg] = 0;
                            }
                            flags[1] = lastp;
                        }
                        named_bar_sync(1, K::NT);
                        if (flags[1]) {
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
                    }
                }
#pragma unroll
                for (int r = 0; r < K::R; ++r)
#pragma unroll
                    for (int c = 0; c < K::KCW; ++c) acc[r][c] = T(0);
            }
            if (++jc == upr) { jc = 0; ++rb; }
        }
    }
}

// Packed row-major copies of B for the problems of a row-major TSM2R class:
// Bt[j*kc + c] = B[j + c*ldb] for c < k, zero for k <= c < kc.  Run before
// every execution of the class, so the plan always sees the current B.
__global__ void batch_bt_pack_kernel(const ProbDesc *__restrict__ probs, int nprob, int kc) {
    for (int i = blockIdx.y; i < nprob; i += gridDim.y) {
        const ProbDesc &d = probs[i];
        const float *B = static_cast<const float *>(d.B);
        float *Bt = static_cast<float *>(d.Bt);
        const int64_t total = d.n * kc;
        for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
             t += (int64_t)gridDim.x * blockDim.x) {
            const int64_t j = t / kc;
            const int c = (int)(t - j * kc);
            Bt[t] = c < d.k ? B[j + (int64_t)c * d.ldb] : 0.0f;
        }
    }
}

template <class K>
cudaError_t launch_batched(const BatchLaunch &L, cudaStream_t stream) {
    static std::mutex mu;
    static uint64_t attr_done = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (dev < 64 && !(attr_done & (1ull << dev))) {
            e = cudaFuncSetAttribute(batched_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::SMEM);
            if (e != cudaSuccess) return e;
            attr_done |= 1ull << dev;
        }
    }
    BatchParams p;
    p.probs = L.probs;
    p.nprob = L.nprob;
    p.ngroups = L.ngroups;
    p.ws = static_cast<float *>(L.ws);
    p.counters = L.counters;
    p.status = L.status;
    p.wait_ns = L.wait_ns;
    if constexpr (K::BT && !K::BRES) {
        const dim3 pg(8, (unsigned)(L.nprob < 65535 ? L.nprob : 65535));
        batch_bt_pack_kernel<<<pg, 256, 0, stream>>>(L.probs, L.nprob, K::KC);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    batched_kernel<K><<<L.grid, 384, K::SMEM, stream>>>(p);
    return cudaGetLastError();
}

template <class K>
BatchClass class_of(char op, const char *name) {
    BatchClass c;
    c.op = op;
    c.name = name;
    c.KC = K::KC;
    c.BM = K::BM;
    c.BNS = K::BNS;
    c.BOXM = K::BOXM;
    c.b_rowmajor = K::BT && !K::BRES;
    c.launch = &launch_batched<K>;
    return c;
}

const BatchClass kClasses[] = {
    class_of<R32<2>>('r', "br_f32_kc2"),    class_of<R32<4>>('r', "br_f32_kc4"),
    class_of<R32<8>>('r', "br_f32_kc8"),    class_of<R32<12>>('r', "br_f32_kc12"),
    class_of<R32<16>>('r', "br_f32_kc16"),  class_of<L32<2>>('l', "bl_f32_kc2"),
    class_of<L32<4>>('l', "bl_f32_kc4"),    class_of<L32<8>>('l', "bl_f32_kc8"),
    class_of<L32<12>>('l', "bl_f32_kc12"),  class_of<L32<16>>('l', "bl_f32_kc16"),
    class_of<L32<24>>('l', "bl_f32_kc24"),  class_of<L32<32>>('l', "bl_f32_kc32"),
    class_of<W32N<2>>('w', "bw_f32_kc2"),   class_of<W32N<4>>('w', "bw_f32_kc4"),
    class_of<W32N<8>>('w', "bw_f32_kc8"),   class_of<W32N<12>>('w', "bw_f32_kc12"),
    class_of<W32N<16>>('w', "bw_f32_kc16"), class_of<W32N<24>>('w', "bw_f32_kc24"),
    class_of<W32N<32>>('w', "bw_f32_kc32"),
};


}  // namespace

const BatchClass *batch_class(char op, int kc) {
    for (const BatchClass &c : kClasses)
        if (c.op == op && c.KC == kc) return &c;
    return nullptr;
}

}  // namespace tsm2
