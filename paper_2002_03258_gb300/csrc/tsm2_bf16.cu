// TSM2R with A stored in bfloat16 (optionally as a hi + lo pair), B and C in
// binary32, binary32 accumulation -- on the tensor cores (tcgen05 + TMEM).
//
// The contraction C(m x k) = A(m x n) B(n x k) is the paper's TSM2R (Sec. 3.1)
// with A read once; with A in bfloat16 the FMA work per byte of A doubles,
// which the CUDA cores cannot sustain at HBM speed, so the products run on
// the tensor cores instead:
//
//  * B (binary32) is split exactly into three bfloat16 pieces, B = B1 + B2 + B3
//    (each piece the round-to-nearest-even of the remainder), by a small prep
//    kernel that also lays them out pre-tiled in the canonical K-major
//    no-swizzle layout of the MMA B operand (8 x 16-byte core matrices).
//  * A tiles (512 rows x BK inner columns per stage, eight 64-row boxes, so
//    DRAM sees 1 KB runs per column) arrive by TMA with the 128-byte swizzle,
//    i.e. in the canonical MN-major SW128 layout of the MMA A operand (A is
//    column-major, rows contiguous); each stage is four M = 128 row tiles.
//    BK = 64 for plain A (a 64 KB tile per stage) and 32 for hi+lo (two 32 KB
//    tiles): every stage hand-off (full/empty barriers, copy issue, MMA
//    commit) costs a fixed time, which 32 KB stages could not hide (79% of
//    HBM for plain A against 90% with 64 KB stages).
//  * One thread issues tcgen05.mma.kind::f16 (M = 128, K = 16, bf16 x bf16
//    -> f32) into TMEM, one MMA per A operand with the B pieces side by side
//    in N, each piece into its own 16 accumulator columns:
//        plain:  [D1 D2]    += A   * [B1 B2]     (N = 32; B to 16 bits: below
//                                                 the 2^-9 representation error of A)
//        hi+lo:  [D1 D2 D3] += Ahi * [B1 B2 B3]  (N = 48)
//                [D1 D2 D3] += Alo * [B1 B2 B3]
//    so each A tile is read from shared memory once per K step, not once per
//    piece (with N = 16 per piece the MMAs' A reads limited the kernel).
//    tcgen05.commit releases each shared-memory stage back to the producer.
//  * A group of stages accumulates into one of the TMEM buffers (4 for plain,
//    2 for hi+lo, so the MMAs can run groups ahead of the drain); four
//    epilogue warps drain it with tcgen05.ld after every group (one TMEM lane
//    = one row of C), add the pieces smallest first and carry the sum over
//    groups in registers with round-to-nearest binary32 adds.  hi+lo drains
//    after every stage (the tensor cores' own accumulation then covers one
//    stage's products only, which keeps hi+lo at binary32-like accuracy);
//    plain drains every 4 stages, far below its bfloat16 representation
//    error.
//    Groups never cross a row block.  Pieces end in C, or in a partial sum
//    for the same deterministic stream-K fix-up as the CUDA-core kernels.
// Every wait is bounded; TMEM is always released before the block exits.
#include "common.cuh"
#include "internal.h"

#include <cuda_bf16.h>

#include <mutex>

namespace tsm2 {
namespace {

constexpr int kMM = 128;          // MMA M = TMEM lanes
constexpr int kSub = 4;           // MMA row tiles per unit
constexpr int kBM = kSub * kMM;   // 512 rows per unit: 1 KB contiguous per column of A
constexpr int kKC = 16;           // C columns per B piece
constexpr int kMaxStages = 8;     // stages are sized at run time: 3 (plain and hi+lo)
constexpr int kMaxBuf = 4;        // TMEM accumulator buffers at most
constexpr int kTmemCols = 512;    // TMEM columns allocated per block
// Per-variant geometry: plain A (one bfloat16 matrix) or hi+lo (two).
template <bool HILO>
struct Variant {
    static constexpr int BK = HILO ? 32 : 64;                 // inner columns per stage
    static constexpr int KSteps = BK / 16;                    // MMA K steps per stage
    static constexpr int NP = HILO ? 3 : 2;                   // B pieces per MMA (N = 16 NP)
    static constexpr int Box = 64 * BK * 2;                   // one 64-row TMA box
    static constexpr int ATile = kBM * BK * 2;                // one A tile (8 boxes)
    static constexpr int BBlock = KSteps * NP * 512;          // B pieces per stage
    static constexpr int Stage = (HILO ? 2 : 1) * ATile + BBlock;
    static constexpr int SubCols = NP * kKC;                  // TMEM columns per row tile
    static constexpr int BufCols = kSub * SubCols;            // TMEM columns per buffer
    static constexpr int NBuf = HILO ? 2 : 4;
    // Instruction descriptor, kind::f16: D f32, A bf16, B bf16, A MN-major
    // (column-major A: rows contiguous), B K-major, N = 16 NP, M = 128.
    static constexpr uint32_t Idesc = (1u << 4)               // D format f32
                                      | (1u << 7)             // A format bf16
                                      | (1u << 10)            // B format bf16
                                      | (1u << 15)            // A major: MN
                                      | (0u << 16)            // B major: K
                                      | ((uint32_t)(SubCols >> 3) << 17)
                                      | ((uint32_t)(kMM >> 4) << 24);
    static_assert(NBuf <= kMaxBuf && NBuf * BufCols <= kTmemCols, "TMEM buffers");
    static_assert(Stage % 1024 == 0 && Box % 1024 == 0, "1 KB alignment of A boxes");
};
using VPlain = Variant<false>;
using VHiLo = Variant<true>;
constexpr int kSmemBudget = 210 * 1024;                // ring bytes (barriers follow)
static_assert(kSmemBudget / VHiLo::Stage >= 3 && kSmemBudget / VPlain::Stage >= 3 &&
                  kSmemBudget + 1024 + 512 <= 227 * 1024,
              "shared memory budget");


// Shared-memory matrix descriptor (tcgen05): start address, leading and
// stride byte offsets (all >> 4), fixed version 1 (bits 46-47), layout type
// (bits 61-63: 0 = no swizzle, 2 = 128-byte swizzle).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo, uint32_t layout) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)(layout & 7u) << 61;
    return d;
}

__device__ __forceinline__ void umma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive TMEM columns of this warp's 32 lanes; the caller waits
// (tmem_ld_wait) before using the registers, so several loads can be in
// flight at once.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

struct BParams {
    int64_t m, n;
    int k;
    const unsigned char *bpieces;  // [n/BK blocks][piece][kstep][512 B], device
    float *C;
    int64_t ldc;
    float *ws;
    int *counters;
    unsigned *status;
    int64_t wait_ns;
    int64_t upr;     // stages per row block
    int64_t ngroups; // units in total
    int group;        // stages summed in TMEM per drain (1 for hi+lo)
    int stages;       // ring depth
    int stage_bytes;  // ring stride (A_hi, [A_lo], B pieces)
};

__device__ __forceinline__ int64_t owner_b(int64_t x, int64_t G, int64_t NG) { return ((x + 1) * G + NG - 1) / NG - 1; }

template <bool HILO>
__global__ void __launch_bounds__(192, 1)
bf16_kernel(const __grid_constant__ CUtensorMap mapHi, const __grid_constant__ CUtensorMap mapLo, const BParams p) {
    using D = Variant<HILO>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = smem_aligned<1024>(smem_raw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kSmemBudget);
    uint64_t *full = bars;                   // [stages] TMA landed
    uint64_t *empty = bars + kMaxStages;     // [stages] MMAs done with the stage
    uint64_t *accf = bars + 2 * kMaxStages;  // [NBuf] stage sum complete in TMEM
    uint64_t *acce = accf + kMaxBuf;         // [NBuf] drained by the epilogue
    uint64_t *fin = acce + kMaxBuf;          // [1] all MMAs finished
    const int nst = p.stages;
    const int sbytes = p.stage_bytes;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(fin + 1);
    volatile int *flags = reinterpret_cast<volatile int *>(tmem_slot + 2);  // [0] abort, [1] last

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t G = gridDim.x, g = blockIdx.x;
    const int64_t u_begin = g * p.ngroups / G;
    const int64_t u_end = (g + 1) * p.ngroups / G;
    const int nunits = (int)(u_end - u_begin);
    const int upr = (int)p.upr;

    if (threadIdx.x == 0) {
        for (int s = 0; s < nst; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < D::NBuf; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], 4);
        }
        mbar_init(fin, 1);
        flags[0] = 0;
        flags[1] = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t *>(tmem_slot);

    if (warp == 0) {
        // ---------------- producer ----------------
        if (lane == 0) {
            prefetch_tensormap(&mapHi);
            if (HILO) prefetch_tensormap(&mapLo);
            const uint64_t policy = l2_policy_evict_first();
            const uint32_t tx = (uint32_t)D::Stage;
            int s = 0;
            uint32_t ph = 0, issued = 0, last_par = 0;
            int rb = (int)(u_begin / p.upr);
            int kc = (int)(u_begin - (int64_t)rb * p.upr);
            for (int i = 0; i < nunits; ++i) {
                if (flags[0]) break;
                if (!mbar_wait_bounded(&empty[s], ph ^ 1u, p.wait_ns, flags)) {
                    flags[0] = 1;
                    atomicOr(p.status, kStatusTimeout);
                    break;
                }
                unsigned char *st = smem + s * sbytes;
                mbar_arrive_expect_tx(&full[s], tx);
                const int32_t x0 = rb * kBM, y0 = kc * D::BK;
#pragma unroll
                for (int q = 0; q < kBM / 64; ++q) {
                    tma_load_2d_hint(st + q * D::Box, &mapHi, x0 + q * 64, y0, &full[s], policy);
                    if (HILO)
                        tma_load_2d_hint(st + D::ATile + q * D::Box, &mapLo, x0 + q * 64, y0, &full[s], policy);
                }
                bulk_g2s(st + sbytes - D::BBlock, p.bpieces + (size_t)kc * D::BBlock, D::BBlock, &full[s]);
                issued |= 1u << s;
                last_par = (last_par & ~(1u << s)) | (ph << s);
                if (++s == nst) { s = 0; ph ^= 1u; }
                if (++kc == upr) { kc = 0; ++rb; }
            }
            for (int t = 0; t < nst; ++t)
                if (issued & (1u << t)) (void)mbar_wait_bounded(&full[t], (last_par >> t) & 1u, 4000000000LL, nullptr);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            uint32_t acc_ph = 0;  // bit b: parity of buffer b
            int buf = 0;
            int gcnt = 0;         // stages already summed into the current buffer
            int kc = (int)(u_begin % p.upr);
            bool issued_any = false;
            for (int i = 0; i < nunits; ++i) {
                if (flags[0]) break;
                // Each group of stages accumulates into its own TMEM buffer,
                // which the epilogue must have drained (four buffers rotate).
                // A group ends after p.group stages, at the end of a row
                // block and at the block's last unit (the epilogue tracks the
                // same boundaries).
                const bool gstart = (gcnt == 0);
                const bool gend = (gcnt + 1 == p.group) || (kc == upr - 1) || (i == nunits - 1);
                if (gstart && !mbar_wait_bounded(&acce[buf], ((acc_ph >> buf) & 1u) ^ 1u, p.wait_ns, flags)) {
                    flags[0] = 1;
                    atomicOr(p.status, kStatusTimeout);
                    break;
                }
                if (!mbar_wait_bounded(&full[s], ph, p.wait_ns, flags)) {
                    flags[0] = 1;
                    atomicOr(p.status, kStatusTimeout);
                    break;
                }
                tc_fence_after();
                const uint32_t st = smem_u32(smem + s * sbytes);
#pragma unroll
                for (int ks = 0; ks < D::KSteps; ++ks) {
                    // B pieces of K step ks side by side in N: K-major, no
                    // swizzle, K-halves 128 B apart (LBO), 8-column groups
                    // 256 B apart (SBO); piece p covers N = 16p .. 16p + 15.
                    const uint64_t bdesc = sdesc(st + sbytes - D::BBlock + ks * D::NP * 512, 128, 256, 0);
#pragma unroll
                    for (int sub = 0; sub < kSub; ++sub) {
                        // A row tile sub: MN-major SW128, its two 64-row boxes
                        // one box apart (LBO), 8-column groups 1 KB apart (SBO).
                        const uint32_t aoff = sub * 2 * D::Box + ks * 2048;
                        const uint32_t d = tmem + (uint32_t)(buf * D::BufCols + sub * D::SubCols);
                        umma_f16(d, sdesc(st + aoff, D::Box, 1024, 2), bdesc, D::Idesc, (gstart && ks == 0) ? 0u : 1u);
                        if (HILO) umma_f16(d, sdesc(st + D::ATile + aoff, D::Box, 1024, 2), bdesc, D::Idesc, 1u);
                    }
                }
                issued_any = true;
                umma_commit(&empty[s]);  // stage s may be refilled once these MMAs are done
                if (gend) {
                    umma_commit(&accf[buf]);  // and the group's sum is ready for the epilogue
                    acc_ph ^= 1u << buf;
                    if (++buf == D::NBuf) buf = 0;
                    gcnt = 0;
                } else {
                    ++gcnt;
                }
                if (++s == nst) { s = 0; ph ^= 1u; }
                if (++kc == upr) kc = 0;
            }
            // Every MMA this thread issued has completed before TMEM is freed.
            if (issued_any) {
                umma_commit(fin);
                (void)mbar_wait_bounded(fin, 0, 4000000000LL, nullptr);
            }
        }
    } else {
        // ---------------- epilogue: warps 2..5, one TMEM lane quarter each ----------------
        const int quarter = warp & 3;          // TMEM lanes 32*quarter .. +31
        const int r = quarter * 32 + lane;     // row within each 128-row tile
        const int et = threadIdx.x - 64;       // 0 .. 127
        uint32_t acc_ph = 0;
        int buf = 0;
        bool aborted = false;
        int rb = (int)(u_begin / p.upr);
        int kc = (int)(u_begin - (int64_t)rb * p.upr);
        bool piece_at_start = (kc == 0);
        // The tensor cores sum one group of stages only; the long sum over
        // groups runs here in binary32 with round-to-nearest adds.
        float v[kSub][kKC];
#pragma unroll
        for (int sub = 0; sub < kSub; ++sub)
#pragma unroll
            for (int c = 0; c < kKC; ++c) v[sub][c] = 0.f;
        int gcnt = 0;
        for (int i = 0; i < nunits; ++i) {
            const bool rb_end = (kc == upr - 1);
            const bool gend = (gcnt + 1 == p.group) || rb_end || (i == nunits - 1);
            if (gend) {
                if (!aborted) {
                    bool ok = !flags[0] && mbar_wait_bounded(&accf[buf], (acc_ph >> buf) & 1u, p.wait_ns, flags);
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
                    tc_fence_after();
                    // Two row tiles' pieces in flight per wait; the pieces of
                    // each output are added smallest first.
#pragma unroll
                    for (int sub0 = 0; sub0 < kSub; sub0 += 2) {
                        uint32_t t[2][D::NP][16];
#pragma unroll
                        for (int h = 0; h < 2; ++h)
#pragma unroll
                            for (int pc = 0; pc < D::NP; ++pc)
                                tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) +
                                              (uint32_t)(buf * D::BufCols + (sub0 + h) * D::SubCols + pc * kKC),
                                          t[h][pc]);
                        tmem_ld_wait();
#pragma unroll
                        for (int h = 0; h < 2; ++h)
#pragma unroll
                            for (int c = 0; c < kKC; ++c) {
                                float x = __uint_as_float(t[h][D::NP - 1][c]);
#pragma unroll
                                for (int pc = D::NP - 2; pc >= 0; --pc) x += __uint_as_float(t[h][pc][c]);
                                v[sub0 + h][c] += x;
                            }
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&acce[buf]);
                }
                acc_ph ^= 1u << buf;
                if (++buf == D::NBuf) buf = 0;
                gcnt = 0;
            } else {
                ++gcnt;
            }
            if (rb_end || i == nunits - 1) {
                const bool whole = piece_at_start && rb_end;
                const int64_t rb64 = rb;
                const int64_t row0 = rb64 * kBM;
                if (whole) {
                    if (!aborted)
#pragma unroll
                        for (int sub = 0; sub < kSub; ++sub) {
                            const int64_t row = row0 + sub * kMM + r;
                            if (row < p.m)
#pragma unroll
                                for (int c = 0; c < kKC; ++c)
                                    if (c < p.k) p.C[row + (int64_t)c * p.ldc] = v[sub][c];
                        }
                } else {
                    const int64_t rb_u0 = rb64 * p.upr;
                    const int64_t gA = owner_b(rb_u0, G, p.ngroups);
                    const int64_t gB = owner_b(rb_u0 + p.upr - 1, G, p.ngroups);
                    float *slot = p.ws + (g + rb64) * (int64_t)(kKC * kBM);
#pragma unroll
                    for (int sub = 0; sub < kSub; ++sub)
#pragma unroll
                        for (int c = 0; c < kKC; ++c) __stcg(slot + c * kBM + sub * kMM + r, v[sub][c]);
                    __threadfence();
                    named_bar_sync(1, 128);
                    if (et == 0) {
                        int last = 0;
                        if (!flags[0]) {
                            const int old = atomicAdd(&p.counters[rb], 1);
                            last = (old == (int)(gB - gA));
                            if (last) p.counters[rb] = 0;
                        }
                        flags[1] = last;
                    }
                    named_bar_sync(1, 128);
                    if (flags[1]) {
                        __threadfence();
#pragma unroll 1
                        for (int sub = 0; sub < kSub; ++sub) {
                            float sum[kKC];
                            const float *src = p.ws + (gA + rb64) * (int64_t)(kKC * kBM) + sub * kMM + r;
#pragma unroll
                            for (int c = 0; c < kKC; ++c) sum[c] = __ldcg(src + c * kBM);
                            for (int64_t gp = gA + 1; gp <= gB; ++gp) {
                                src += kKC * kBM;
                                float x[kKC];
#pragma unroll
                                for (int c = 0; c < kKC; ++c) x[c] = __ldcg(src + c * kBM);
#pragma unroll
                                for (int c = 0; c < kKC; ++c) sum[c] += x[c];
                            }
                            const int64_t row = row0 + sub * kMM + r;
                            if (row < p.m)
#pragma unroll
                                for (int c = 0; c < kKC; ++c)
                                    if (c < p.k) p.C[row + (int64_t)c * p.ldc] = sum[c];
                        }
                    }
                    named_bar_sync(1, 128);  // flags[1] is reused by the next piece
                }
                piece_at_start = true;
#pragma unroll
                for (int sub = 0; sub < kSub; ++sub)
#pragma unroll
                    for (int c = 0; c < kKC; ++c) v[sub][c] = 0.f;
            }
            if (++kc == upr) { kc = 0; ++rb; }
        }
    }
    // Everyone (including idle lanes) meets here before the TMEM is freed.
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// Split binary32 B (n x k, k <= 16) into bfloat16 pieces b1 + b2 + b3 = b
// (each the round-to-nearest-even of the remainder), the first np of them
// written in the MMA B-operand layout [n/bk blocks][kstep][piece][core nb]
// [core kb][8][8] (bk inner columns per block, one block per pipeline stage;
// the pieces of one K step side by side form one N = 16 np operand).
__global__ void bsplit_kernel(int64_t n, int k, const float *__restrict__ B, int64_t ldb, __nv_bfloat16 *out,
                              int64_t nblocks, int bk, int np) {
    const int ksteps = bk / 16;
    const int64_t total = nblocks * ksteps * np * 256;  // bf16 elements
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t q = t;
        const int e = (int)(q % 8); q /= 8;
        const int rr = (int)(q % 8); q /= 8;
        const int kb = (int)(q % 2); q /= 2;
        const int nb = (int)(q % 2); q /= 2;
        const int piece = (int)(q % np); q /= np;
        const int ks = (int)(q % ksteps); q /= ksteps;
        const int64_t blk = q;
        const int64_t j = blk * bk + ks * 16 + kb * 8 + e;
        const int c = nb * 8 + rr;
        const float b = (j < n && c < k) ? B[j + (int64_t)c * ldb] : 0.f;
        const __nv_bfloat16 b1 = __float2bfloat16_rn(b);
        const float r1 = b - __bfloat162float(b1);
        const __nv_bfloat16 b2 = __float2bfloat16_rn(r1);
        const float r2 = r1 - __bfloat162float(b2);
        const __nv_bfloat16 b3 = __float2bfloat16_rn(r2);
        out[t] = piece == 0 ? b1 : piece == 1 ? b2 : b3;
    }
}

// Element-wise path (any alignment): one thread per row, bf16 -> f32 in
// registers, binary32 FMAs with B.
__global__ void __launch_bounds__(128) bf16_simple_kernel(int64_t m, int64_t n, int k, const __nv_bfloat16 *A_hi,
                                                          const __nv_bfloat16 *A_lo, int64_t lda, const float *B,
                                                          int64_t ldb, float *C, int64_t ldc) {
    __shared__ float Bs[64][kKC];
    const int64_t row = (int64_t)blockIdx.x * 128 + threadIdx.x;
    float acc[kKC];
#pragma unroll
    for (int c = 0; c < kKC; ++c) acc[c] = 0.f;
    for (int64_t j0 = 0; j0 < n; j0 += 64) {
        __syncthreads();
        for (int t = threadIdx.x; t < 64 * kKC; t += 128) {
            const int jj = t % 64, c = t / 64;
            Bs[jj][c] = (j0 + jj < n && c < k) ? B[j0 + jj + (int64_t)c * ldb] : 0.f;
        }
        __syncthreads();
        if (row < m) {
            const int jn = (int)((n - j0) < 64 ? (n - j0) : 64);
            for (int jj = 0; jj < jn; ++jj) {
                float a = __bfloat162float(A_hi[row + (j0 + jj) * lda]);
                if (A_lo) a += __bfloat162float(A_lo[row + (j0 + jj) * lda]);  // exact: 16 significant bits
#pragma unroll
                for (int c = 0; c < kKC; ++c) acc[c] = fmaf(a, Bs[jj][c], acc[c]);
            }
        }
    }
    if (row < m)
#pragma unroll
        for (int c = 0; c < kKC; ++c)
            if (c < k) C[row + (int64_t)c * ldc] = acc[c];
}

// x -> hi = RNE_bf16(x), lo = RNE_bf16(x - hi) (x - hi is exact in binary32).
__global__ void split_kernel(int64_t rows, int64_t cols, const float *X, int64_t ldx, __nv_bfloat16 *hi,
                             __nv_bfloat16 *lo, int64_t ldh) {
    const int64_t total = rows * cols;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = t / rows, i = t - (t / rows) * rows;
        const float x = X[i + j * ldx];
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        hi[i + j * ldh] = h;
        if (lo) lo[i + j * ldh] = __float2bfloat16_rn(x - __bfloat162float(h));
    }
}

}  // namespace

int bf16_bm() { return kBM; }
int bf16_bk(bool hilo) { return hilo ? VHiLo::BK : VPlain::BK; }
size_t bf16_bpieces_bytes(int64_t n, bool hilo) {
    const int bk = bf16_bk(hilo);
    return (size_t)((n + bk - 1) / bk) * (hilo ? VHiLo::BBlock : VPlain::BBlock);
}

cudaError_t bf16_prep_b(int64_t n, int k, const float *B, int64_t ldb, void *out, bool hilo, cudaStream_t stream) {
    const int bk = bf16_bk(hilo);
    const int64_t nblocks = (n + bk - 1) / bk;
    const int np = hilo ? VHiLo::NP : VPlain::NP;
    const int64_t total = nblocks * (bk / 16) * np * 256;
    int64_t grid = (total + 255) / 256;
    if (grid > 4096) grid = 4096;
    bsplit_kernel<<<(unsigned)grid, 256, 0, stream>>>(n, k, B, ldb, static_cast<__nv_bfloat16 *>(out), nblocks, bk,
                                                      np);
    return cudaGetLastError();
}

template <bool HILO>
cudaError_t bf16_set_smem(int smem) {
    static std::mutex mu;
    static uint64_t attr_done = 0;  // one bit per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 64 && !(attr_done & (1ull << dev))) {
        e = cudaFuncSetAttribute(bf16_kernel<HILO>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr_done |= 1ull << dev;
    }
    return cudaSuccess;
}

cudaError_t bf16_launch(const BF16Launch &L, cudaStream_t stream) {
    const int smem = kSmemBudget + 1024 + 512;  // ring + 1 KB alignment slack + barriers
    cudaError_t e = L.hilo ? bf16_set_smem<true>(smem) : bf16_set_smem<false>(smem);
    if (e != cudaSuccess) return e;
    BParams p;
    p.m = L.m;
    p.n = L.n;
    p.k = L.k;
    p.bpieces = static_cast<const unsigned char *>(L.bpieces);
    p.C = static_cast<float *>(L.C);
    p.ldc = L.ldc;
    p.ws = static_cast<float *>(L.ws);
    p.counters = L.counters;
    p.status = L.status;
    p.wait_ns = L.wait_ns;
    const int bk = bf16_bk(L.hilo);
    p.upr = (L.n + bk - 1) / bk;
    p.ngroups = ((L.m + kBM - 1) / kBM) * p.upr;
    // Plain: the tensor cores sum 4 stages (256 inner indices, 512 products
    // per output) before each drain, far inside the bfloat16 representation
    // error of A; hi+lo: one stage per drain, for binary32-like accuracy.
    p.group = L.hilo ? 1 : 4;
    p.stage_bytes = L.hilo ? VHiLo::Stage : VPlain::Stage;
    p.stages = kSmemBudget / p.stage_bytes;
    if (p.stages > kMaxStages) p.stages = kMaxStages;
    if (L.hilo)
        bf16_kernel<true><<<L.grid, 192, smem, stream>>>(L.mapHi, L.mapLo, p);
    else
        bf16_kernel<false><<<L.grid, 192, smem, stream>>>(L.mapHi, L.mapLo, p);
    return cudaGetLastError();
}

cudaError_t bf16_simple_launch(int64_t m, int64_t n, int k, const void *A_hi, const void *A_lo, int64_t lda,
                               const float *B, int64_t ldb, float *C, int64_t ldc, cudaStream_t stream) {
    if (m <= 0) return cudaSuccess;
    bf16_simple_kernel<<<(unsigned)((m + 127) / 128), 128, 0, stream>>>(
        m, n, k, static_cast<const __nv_bfloat16 *>(A_hi), static_cast<const __nv_bfloat16 *>(A_lo), lda, B, ldb, C,
        ldc);
    return cudaGetLastError();
}

cudaError_t split_bf16_launch(int64_t rows, int64_t cols, const float *X, int64_t ldx, void *hi, void *lo,
                              int64_t ldh, int sm_count, cudaStream_t stream) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    const int64_t total = rows * cols;
    int64_t grid = (total + 255) / 256;
    if (grid > (int64_t)sm_count * 32) grid = (int64_t)sm_count * 32;
    split_kernel<<<(unsigned)grid, 256, 0, stream>>>(rows, cols, X, ldx, static_cast<__nv_bfloat16 *>(hi),
                                                    static_cast<__nv_bfloat16 *>(lo), ldh);
    return cudaGetLastError();
}

}  // namespace tsm2
