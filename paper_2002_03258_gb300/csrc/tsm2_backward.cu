// Kernels of the backward products of C = A B (A m x n, B n x k, column-major):
//
//   dB = A^T dC   (n x k)   -- "transposed TSM2R": the reduction runs along
//                             A's contiguous (row) dimension;
//   dA = dC B^T   (m x n)   -- a rank-k update, one streaming write of m*n.
//
// Both read their large operand (A, resp. write dA) exactly once, as the
// forward outer-product form does for A (Algorithm 2, Sec. 3.1.2).
//
// tsm2t_kernel: the same warp-specialised TMA pipeline as the forward path.
// A work unit is a BM x BNS tile of A plus the BM x KC tile of dC with the
// same rows; units are numbered column chunk by column chunk, so a block
// accumulates a chunk of dB over a contiguous run of row blocks in registers.
// Each lane owns R rows; warp w owns JW of the chunk's columns.  Products of
// row pairs go through packed FFMA2 into two partial sums (even/odd rows),
// which is operand-friendly (both pairs are adjacent rows of a 16-byte load).
// At the end of a run the 32 lanes are combined by a fixed butterfly; runs
// that start or end inside a column chunk go through the same deterministic
// last-arriver fix-up as the forward kernel.
#include "common.cuh"
#include "internal.h"

#include <mutex>

namespace tsm2 {
namespace {

constexpr int kProducerRegsT = 40;
constexpr int kConsumerRegsT = 232;

template <typename T_, int KC_, int NV_, int JW_, int STAGES_>
struct TCfg {
    using T = T_;
    using VT = Vec16<T>;
    using vec_t = typename VT::type;
    static constexpr int V = VT::n;
    static constexpr int KC = KC_;
    static constexpr int NV = NV_;
    static constexpr int R = NV * V;          // rows per lane
    static constexpr int BM = 32 * R;         // rows per unit
    static constexpr int JW = JW_;            // columns per warp
    static constexpr int NW = 8;
    static constexpr int BNS = NW * JW;       // columns per unit (chunk width)
    static constexpr int STAGES = STAGES_;
    static constexpr int BOXM = BM < 256 ? BM : 256;
    static constexpr int NBOX = BM / BOXM;
    static constexpr int A_STAGE = BM * BNS;
    static constexpr int D_STAGE = BM * KC;
    static constexpr uint32_t TX_BYTES = (uint32_t)((A_STAGE + D_STAGE) * sizeof(T));
    static constexpr size_t OFF_D = (size_t)STAGES * A_STAGE * sizeof(T);
    static constexpr size_t OFF_BAR = OFF_D + (size_t)STAGES * D_STAGE * sizeof(T);
    static constexpr size_t OFF_FLAGS = OFF_BAR + 2 * STAGES * sizeof(uint64_t);
    static constexpr size_t SMEM = OFF_FLAGS + 16 + 128;
    static constexpr int NOUT = JW * KC;      // outputs per warp per run
    static constexpr int NP = sizeof(T) == 4 ? 2 : 1;  // partial sums per output (even/odd rows for FFMA2)
    static_assert((A_STAGE * sizeof(T)) % 128 == 0 && (D_STAGE * sizeof(T)) % 128 == 0, "stage alignment");
    static_assert(R % 2 == 0, "row pairs");
    static_assert(SMEM <= 227 * 1024, "shared memory per block");
};

struct TParams {
    int64_t m, n;
    int k;
    void *dB;
    int64_t lddb;
    void *ws;
    int *counters;
    unsigned *status;
    int64_t wait_ns;
    int64_t nrb;      // row blocks (units per column chunk)
    int64_t nunits;   // total units
};

__device__ __forceinline__ int64_t owner_of_t(int64_t x, int64_t G, int64_t NG) {
    return ((x + 1) * G + NG - 1) / NG - 1;
}

template <class K>
__global__ void __launch_bounds__(384, 1)
tsm2t_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapD, const TParams p) {
    using T = typename K::T;
    using vec_t = typename K::vec_t;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = smem_aligned<128>(smem_raw);
    T *sA = reinterpret_cast<T *>(smem);
    T *sD = reinterpret_cast<T *>(smem + K::OFF_D);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + K::OFF_BAR);
    uint64_t *empty = full + K::STAGES;
    volatile int *flags = reinterpret_cast<volatile int *>(smem + K::OFF_FLAGS);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t G = gridDim.x;
    const int64_t g = blockIdx.x;
    const int64_t u_begin = g * p.nunits / G;
    const int64_t u_end = (g + 1) * p.nunits / G;
    const int nunits = (int)(u_end - u_begin);
    const int nrb = (int)p.nrb;

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

    if (warp < 4) {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kProducerRegsT));
        if (warp == 0 && lane == 0) {
            prefetch_tensormap(&mapA);
            prefetch_tensormap(&mapD);
            const uint64_t policy = l2_policy_evict_first();
            int s = 0;
            uint32_t ph = 0, issued = 0, last_par = 0;
            int jc = (int)(u_begin / p.nrb);
            int rb = (int)(u_begin - (int64_t)jc * p.nrb);
            for (int i = 0; i < nunits; ++i) {
                if (flags[0]) break;
                if (!mbar_wait_bounded(&empty[s], ph ^ 1u, p.wait_ns, flags)) {
                    flags[0] = 1;
                    atomicOr(p.status, kStatusTimeout);
                    break;
                }
                mbar_arrive_expect_tx(&full[s], K::TX_BYTES);
                const int32_t x0 = rb * K::BM;
                const int32_t y0 = jc * K::BNS;
#pragma unroll
                for (int q = 0; q < K::NBOX; ++q) {
                    tma_load_2d_hint(sA + (size_t)s * K::A_STAGE + q * K::BOXM * K::BNS, &mapA, x0 + q * K::BOXM, y0,
                                     &full[s], policy);
                    tma_load_2d(sD + (size_t)s * K::D_STAGE + q * K::BOXM * K::KC, &mapD, x0 + q * K::BOXM, 0,
                                &full[s]);
                }
                issued |= 1u << s;
                last_par = (last_par & ~(1u << s)) | (ph << s);
                if (++s == K::STAGES) { s = 0; ph ^= 1u; }
                if (++rb == nrb) { rb = 0; ++jc; }
            }
            for (int t = 0; t < K::STAGES; ++t)
                if (issued & (1u << t)) (void)mbar_wait_bounded(&full[t], (last_par >> t) & 1u, 4000000000LL, nullptr);
        }
        return;
    }

    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kConsumerRegsT));
    const int cw = warp - 4;
    T acc[K::JW][K::KC][K::NP];  // binary32: even / odd rows
#pragma unroll
    for (int jj = 0; jj < K::JW; ++jj)
#pragma unroll
        for (int c = 0; c < K::KC; ++c)
#pragma unroll
            for (int q = 0; q < K::NP; ++q) acc[jj][c][q] = T(0);

    auto row_of = [&](int v) { return v * 32 * K::V + lane * K::V; };  // first row of vector v in the unit

    int s = 0;
    uint32_t ph = 0;
    bool aborted = false;
    int jc = (int)(u_begin / p.nrb);
    int rb = (int)(u_begin - (int64_t)jc * p.nrb);
    bool piece_at_start = (rb == 0);

    for (int i = 0; i < nunits; ++i) {
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
            const T *d_st = sD + (size_t)s * K::D_STAGE;
            T a[K::JW][K::R];
#pragma unroll
            for (int jj = 0; jj < K::JW; ++jj)
#pragma unroll
                for (int v = 0; v < K::NV; ++v) {
                    const int r = row_of(v);
                    const int q = r / K::BOXM, rr = r - q * K::BOXM;
                    const vec_t x = *reinterpret_cast<const vec_t *>(a_st + q * K::BOXM * K::BNS +
                                                                     (cw * K::JW + jj) * K::BOXM + rr);
#pragma unroll
                    for (int e = 0; e < K::V; ++e) a[jj][v * K::V + e] = K::VT::get(x, e);
                }
#pragma unroll
            for (int c = 0; c < K::KC; ++c) {
                T d[K::R];
#pragma unroll
                for (int v = 0; v < K::NV; ++v) {
                    const int r = row_of(v);
                    const int q = r / K::BOXM, rr = r - q * K::BOXM;
                    const vec_t x = *reinterpret_cast<const vec_t *>(d_st + q * K::BOXM * K::KC + c * K::BOXM + rr);
#pragma unroll
                    for (int e = 0; e < K::V; ++e) d[v * K::V + e] = K::VT::get(x, e);
                }
#pragma unroll
                for (int jj = 0; jj < K::JW; ++jj)
#pragma unroll
                    for (int r = 0; r < K::R; r += 2) {
                        if constexpr (K::NP == 2) {
                            const float2 t = __ffma2_rn(make_float2(a[jj][r], a[jj][r + 1]), make_float2(d[r], d[r + 1]),
                                                        make_float2(acc[jj][c][0], acc[jj][c][K::NP - 1]));
                            acc[jj][c][0] = t.x;
                            acc[jj][c][K::NP - 1] = t.y;
                        } else {
                            acc[jj][c][0] = fma(a[jj][r], d[r], acc[jj][c][0]);
                            acc[jj][c][0] = fma(a[jj][r + 1], d[r + 1], acc[jj][c][0]);
                        }
                    }
            }
        }
        if (!aborted) {
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
        }
        if (++s == K::STAGES) { s = 0; ph ^= 1u; }

        const bool chunk_end = (rb == nrb - 1);
        if (chunk_end || i == nunits - 1) {
            // ---- end of a run over column chunk jc ----
            const bool whole = piece_at_start && chunk_end;
            // Lane partials -> warp totals: fixed butterfly; every lane ends
            // with every total, lane t keeps outputs t, t+32, ...
            T mine[(K::NOUT + 31) / 32];
#pragma unroll
            for (int o = 0; o < (K::NOUT + 31) / 32; ++o) mine[o] = T(0);
#pragma unroll
            for (int jj = 0; jj < K::JW; ++jj)
#pragma unroll
                for (int c = 0; c < K::KC; ++c) {
                    T v = acc[jj][c][0];
                    if constexpr (K::NP == 2) v += acc[jj][c][K::NP - 1];
#pragma unroll
                    for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
                    const int o = jj * K::KC + c;
                    if ((o & 31) == lane) mine[o >> 5] = v;
#pragma unroll
                    for (int q = 0; q < K::NP; ++q) acc[jj][c][q] = T(0);
                }
            T *dB = static_cast<T *>(p.dB);
            T *ws = static_cast<T *>(p.ws);
            const int64_t j0 = (int64_t)jc * K::BNS + cw * K::JW;
            if (whole) {
                if (!aborted)
#pragma unroll
                    for (int o0 = 0; o0 < K::NOUT; o0 += 32) {
                        const int o = o0 + lane;
                        if (o < K::NOUT) {
                            const int jj = o / K::KC, c = o - (o / K::KC) * K::KC;
                            if (j0 + jj < p.n && c < p.k) dB[j0 + jj + (int64_t)c * p.lddb] = mine[o0 >> 5];
                        }
                    }
            } else {
                // Partial: slot [BNS][KC] of (block g, chunk jc) = index g + jc.
                T *slot = ws + (g + jc) * (int64_t)(K::BNS * K::KC);
#pragma unroll
                for (int o0 = 0; o0 < K::NOUT; o0 += 32) {
                    const int o = o0 + lane;
                    if (o < K::NOUT && dbg_in_bounds(g + jc < G + p.nunits / p.nrb, p.status))
                        __stcg(slot + cw * K::NOUT + o, mine[o0 >> 5]);
                }
                __threadfence();
                named_bar_sync(1, 256);
                const int64_t cu0 = (int64_t)jc * p.nrb;
                const int64_t gA = owner_of_t(cu0, G, p.nunits);
                const int64_t gB = owner_of_t(cu0 + p.nrb - 1, G, p.nunits);
                if (threadIdx.x == 128) {
                    int last = 0;
                    if (!flags[0] && dbg_in_bounds(jc < p.nunits / p.nrb, p.status)) {
                        const int old = atomicAdd(&p.counters[jc], 1);
                        last = (old == (int)(gB - gA));
                        if (last) p.counters[jc] = 0;
                    }
                    flags[1] = last;
                }
                named_bar_sync(1, 256);
                if (flags[1] && dbg_in_bounds(gA >= 0 && gB + jc < G + p.nunits / p.nrb, p.status)) {
                    __threadfence();
                    for (int o0 = 0; o0 < K::NOUT; o0 += 32) {
                        const int o = o0 + lane;
                        if (o < K::NOUT) {
                            const T *src = ws + (gA + jc) * (int64_t)(K::BNS * K::KC) + cw * K::NOUT + o;
                            T sum = __ldcg(src);
                            for (int64_t gp = gA + 1; gp <= gB; ++gp) {
                                src += K::BNS * K::KC;
                                sum += __ldcg(src);
                            }
                            const int jj = o / K::KC, c = o - (o / K::KC) * K::KC;
                            if (j0 + jj < p.n && c < p.k) dB[j0 + jj + (int64_t)c * p.lddb] = sum;
                        }
                    }
                }
            }
            piece_at_start = true;
        }
        if (++rb == nrb) { rb = 0; ++jc; }
    }
}

template <class K>
cudaError_t launch_t_cfg(const TLaunch &L, cudaStream_t stream) {
    static std::mutex mu;
    static uint64_t attr_done = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (dev < 64 && !(attr_done & (1ull << dev))) {
            e = cudaFuncSetAttribute(tsm2t_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::SMEM);
            if (e != cudaSuccess) return e;
            attr_done |= 1ull << dev;
        }
    }
    TParams p;
    p.m = L.m;
    p.n = L.n;
    p.k = L.k;
    p.dB = L.dB;
    p.lddb = L.lddb;
    p.ws = L.ws;
    p.counters = L.counters;
    p.status = L.status;
    p.wait_ns = L.wait_ns;
    p.nrb = (L.m + K::BM - 1) / K::BM;
    p.nunits = p.nrb * ((L.n + K::BNS - 1) / K::BNS);
    tsm2t_kernel<K><<<L.grid, 384, K::SMEM, stream>>>(L.mapA, L.mapD, p);
    return cudaGetLastError();
}

// binary32: R = 8 rows per lane (BM = 256), 4 columns per warp (BNS = 32).
// binary64: R = 4 rows per lane (BM = 128), 4 columns per warp (BNS = 32).
// Stages for chunks below 16 columns, measured on GB300 at 16384^2 x 8:
// 5 / 4 / 3 stages 0.1748 / 0.1716 / 0.1707 ms.
#ifndef TSM2_T_STAGES
#define TSM2_T_STAGES 3
#endif
template <int KC> using T32 = TCfg<float, KC, 2, 4, (KC >= 16 ? 4 : TSM2_T_STAGES)>;
template <int KC> using T64 = TCfg<double, KC, 2, 4, (KC >= 16 ? 4 : 5)>;

struct TEntry {
    TShape shape;
    cudaError_t (*launch)(const TLaunch &, cudaStream_t);
};

template <class K>
TShape tshape_of(const char *name) {
    TShape s;
    s.name = name;
    s.elem = (int)sizeof(typename K::T);
    s.KC = K::KC;
    s.BM = K::BM;
    s.BNS = K::BNS;
    s.BOXM = K::BOXM;
    return s;
}

#define TSM2_TENTRY(CFG, NAME) TEntry{tshape_of<CFG>(NAME), &launch_t_cfg<CFG>}
const TEntry kTEntries[] = {
    TSM2_TENTRY(T32<2>, "t_f32_kc2"), TSM2_TENTRY(T32<4>, "t_f32_kc4"), TSM2_TENTRY(T32<8>, "t_f32_kc8"),
    TSM2_TENTRY(T32<16>, "t_f32_kc16"), TSM2_TENTRY(T64<2>, "t_f64_kc2"), TSM2_TENTRY(T64<4>, "t_f64_kc4"),
    TSM2_TENTRY(T64<8>, "t_f64_kc8"), TSM2_TENTRY(T64<16>, "t_f64_kc16"),
};

// ---------------------------------------------------------------------------
// Element-wise transposed product for operands the TMA engine cannot
// address: block per column of A, threads stride over rows, block tree sum.

template <typename T, int KC>
__global__ void __launch_bounds__(256) simple_t_kernel(int64_t m, int64_t n, int k, const T *__restrict__ A,
                                                       int64_t lda, const T *__restrict__ dC, int64_t lddc,
                                                       T *__restrict__ dB, int64_t lddb) {
    __shared__ T red[256][KC + 1];
    const int64_t j = blockIdx.x;
    T acc[KC];
#pragma unroll
    for (int c = 0; c < KC; ++c) acc[c] = T(0);
    for (int64_t i = threadIdx.x; i < m; i += 256) {
        const T a = A[i + j * lda];
#pragma unroll
        for (int c = 0; c < KC; ++c)
            if (c < k) acc[c] = fma(a, dC[i + (int64_t)c * lddc], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < KC; ++c) red[threadIdx.x][c] = acc[c];
    __syncthreads();
    for (int w = 128; w >= 1; w >>= 1) {
        if (threadIdx.x < w)
#pragma unroll
            for (int c = 0; c < KC; ++c) red[threadIdx.x][c] += red[threadIdx.x + w][c];
        __syncthreads();
    }
    if (threadIdx.x < k && threadIdx.x < KC) dB[j + (int64_t)threadIdx.x * lddb] = red[0][threadIdx.x];
}

// ---------------------------------------------------------------------------
// Rank-k update dA = dC B^T: each thread owns V consecutive rows of one
// column strip; dC rows stay in registers across the strip's columns, the
// strip's rows of B are staged in shared memory and read by broadcast.

template <typename T, int KC>
__global__ void __launch_bounds__(256) rankk_kernel(int64_t m, int64_t n, int k, const T *__restrict__ dC,
                                                    int64_t lddc, const T *__restrict__ B, int64_t ldb,
                                                    T *__restrict__ dA, int64_t ldda, int vec_ok, int64_t ncol_strips,
                                                    int strip, int accumulate) {
    using VT = Vec16<T>;
    using vec_t = typename VT::type;
    constexpr int V = VT::n;
    __shared__ T sBt[64][KC];  // strip rows of B (<= 64 columns of dA)
    const int64_t nrow_tiles = (m + 256 * V - 1) / (256 * V);
    const int64_t tiles = nrow_tiles * ncol_strips;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int64_t cs = t / nrow_tiles;
        const int64_t rt = t - cs * nrow_tiles;
        const int64_t j0 = cs * strip;
        const int jn = (int)((n - j0) < strip ? (n - j0) : strip);
        __syncthreads();
        for (int e = threadIdx.x; e < strip * KC; e += 256) {
            const int jj = e / KC, c = e - (e / KC) * KC;
            sBt[jj][c] = (jj < jn && c < k) ? B[j0 + jj + (int64_t)c * ldb] : T(0);
        }
        __syncthreads();
        const int64_t r0 = rt * 256 * V + (int64_t)threadIdx.x * V;
        if (r0 >= m) continue;
        T d[KC][V];
#pragma unroll
        for (int c = 0; c < KC; ++c)
#pragma unroll
            for (int e = 0; e < V; ++e)
                d[c][e] = (c < k && r0 + e < m) ? dC[r0 + e + (int64_t)c * lddc] : T(0);
        const bool full = vec_ok && r0 + V <= m;
        for (int jj = 0; jj < jn; ++jj) {
            T *dst = dA + r0 + (j0 + jj) * ldda;
            T out[V];
#pragma unroll
            for (int e = 0; e < V; ++e) out[e] = (accumulate && r0 + e < m) ? dst[e] : T(0);
#pragma unroll
            for (int c = 0; c < KC; ++c) {
                const T b = sBt[jj][c];
#pragma unroll
                for (int e = 0; e < V; ++e) out[e] = fma(d[c][e], b, out[e]);
            }
            if (full) {
                __stcs(reinterpret_cast<vec_t *>(dst), VT::make(out));  // streamed, written once
            } else {
#pragma unroll
                for (int e = 0; e < V; ++e)
                    if (r0 + e < m) dst[e] = out[e];
            }
        }
    }
}

}  // namespace

const TShape *tsm2t_shape(int elem, int kc) {
    for (const TEntry &en : kTEntries)
        if (en.shape.elem == elem && en.shape.KC == kc) return &en.shape;
    return nullptr;
}

cudaError_t tsm2t_launch(const TShape *shape, const TLaunch &L, cudaStream_t stream) {
    for (const TEntry &en : kTEntries)
        if (&en.shape == shape) return en.launch(L, stream);
    return cudaErrorInvalidValue;
}

cudaError_t simple_t_launch(int elem, int64_t m, int64_t n, int k, const void *A, int64_t lda, const void *dC,
                            int64_t lddc, void *dB, int64_t lddb, cudaStream_t stream) {
    if (n <= 0 || k <= 0) return cudaSuccess;
    if (elem == 8)
        simple_t_kernel<double, 16><<<(unsigned)n, 256, 0, stream>>>(m, n, k, static_cast<const double *>(A), lda,
                                                                     static_cast<const double *>(dC), lddc,
                                                                     static_cast<double *>(dB), lddb);
    else
        simple_t_kernel<float, 16><<<(unsigned)n, 256, 0, stream>>>(m, n, k, static_cast<const float *>(A), lda,
                                                                    static_cast<const float *>(dC), lddc,
                                                                    static_cast<float *>(dB), lddb);
    return cudaGetLastError();
}

cudaError_t rankk_launch(int elem, int64_t m, int64_t n, int k, const void *dC, int64_t lddc, const void *B,
                         int64_t ldb, void *dA, int64_t ldda, bool vec_ok, bool accumulate, int sm_count,
                         cudaStream_t stream) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    const int strip = 64;
    const int64_t ncs = (n + strip - 1) / strip;
    const int V = 16 / elem;
    const int64_t nrt = (m + 256 * V - 1) / (256 * V);
    int64_t grid = (int64_t)sm_count * 4;
    if (grid > nrt * ncs) grid = nrt * ncs;
#define TSM2_RK(TT, KCV)                                                                                          \
    rankk_kernel<TT, KCV><<<(unsigned)grid, 256, 0, stream>>>(m, n, k, static_cast<const TT *>(dC), lddc,        \
                                                              static_cast<const TT *>(B), ldb,                    \
                                                              static_cast<TT *>(dA), ldda, vec_ok ? 1 : 0, ncs,   \
                                                              strip, accumulate ? 1 : 0)
    if (elem == 8) {
        if (k <= 4) TSM2_RK(double, 4); else if (k <= 8) TSM2_RK(double, 8); else TSM2_RK(double, 16);
    } else {
        if (k <= 4) TSM2_RK(float, 4); else if (k <= 8) TSM2_RK(float, 8); else TSM2_RK(float, 16);
    }
#undef TSM2_RK
    return cudaGetLastError();
}

}  // namespace tsm2
