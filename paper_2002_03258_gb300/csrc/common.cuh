// Device helpers shared by the kernels of the library: 16-byte vector types,
// mbarrier and bulk tensor copy (TMA) wrappers in inline PTX, and bounded
// waits that record a timeout in a status word instead of spinning forever.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace tsm2 {

// Status bits written to the device status word.
constexpr unsigned kStatusTimeout = 1u;
constexpr unsigned kStatusBounds = 2u;  // debug builds: an access outside its operand was skipped

// Debug builds (-DTSM2_DEBUG) check every hand-computed global address
// against the extents of the operand it belongs to (rows and columns of C or
// B, workspace slots, arrival counters) before the access.  dbg_in_bounds
// returns `ok`; when it is false it records kStatusBounds in the status word
// and the caller skips the access, so a wrong index shows up as a status
// instead of a fault.  Release builds compile it to `true`.
#ifdef TSM2_DEBUG
constexpr bool kDebugChecks = true;
#else
constexpr bool kDebugChecks = false;
#endif
__device__ __forceinline__ bool dbg_in_bounds(bool ok, unsigned *status) {
    if constexpr (kDebugChecks) {
        if (!ok) {
            atomicOr(status, kStatusBounds);
            return false;
        }
    }
    return true;
}

// 16-byte vector of T: float4 for binary32, double2 for binary64.
template <typename T> struct Vec16;
template <> struct Vec16<float> {
    using type = float4;
    static constexpr int n = 4;
    __device__ static inline float get(const float4 &v, int i) {
        return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
    }
    __device__ static inline float4 make(const float *x) { return make_float4(x[0], x[1], x[2], x[3]); }
};
template <> struct Vec16<double> {
    using type = double2;
    static constexpr int n = 2;
    __device__ static inline double get(const double2 &v, int i) { return i == 0 ? v.x : v.y; }
    __device__ static inline double2 make(const double *x) { return make_double2(x[0], x[1]); }
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Dynamic shared memory rounded up to `align` bytes.  The pad comes from the
// shared-window address and is added to the array pointer itself, so the
// result stays a shared-space pointer: loads through it compile to shared
// loads, not generic ones (an integer round trip would lose that).
template <unsigned kAlign>
__device__ __forceinline__ unsigned char *smem_aligned(unsigned char *raw) {
    static_assert((kAlign & (kAlign - 1)) == 0, "power of two");
    const uint32_t a = smem_u32(raw);
    return raw + ((kAlign - (a & (kAlign - 1))) & (kAlign - 1));
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t sm_id() {
    uint32_t s;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(s));
    return s;
}

// ---- mbarrier ---------------------------------------------------------------

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Make barrier initialisation visible to the async proxy (TMA) and the CTA.
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits until the phase with parity `parity` of `bar` has completed, for at
// most `budget_ns` nanoseconds (0: a single attempt, which the hardware may
// itself suspend for a short while), giving up early when `*abort` becomes
// non-zero.  A negative budget gives up at once without testing the barrier
// (a test hook: it drives every kernel's timeout path deterministically).
// Returns false on timeout or abort; the caller records it and stops using
// the pipeline.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int64_t budget_ns,
                                                  const volatile int *abort = nullptr) {
    if (budget_ns < 0) return false;
    if (mbar_try_wait(bar, parity)) return true;
    if (budget_ns <= 0) return false;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 0u) {
            if (abort && *abort) return false;
            if ((int64_t)(globaltimer_ns() - t0) > budget_ns) return false;
        }
    }
}

// ---- bulk tensor copies (TMA) -------------------------------------------------

// 2-D tiled load of the box at coordinates (x = innermost, y) of `map` into
// shared memory at `dst`; completion is signalled on `bar` as transaction
// bytes.  The caller guarantees x * sizeof(elem) is a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int32_t x, int32_t y,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Same, with an L2 eviction-priority hint (streamed operands read once).
__device__ __forceinline__ void tma_load_2d_hint(void *dst, const CUtensorMap *map, int32_t x, int32_t y,
                                                 uint64_t *bar, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

__device__ __forceinline__ uint64_t l2_policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap *map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// Named barrier over `nthreads` threads (a multiple of 32), id >= 1.
__device__ __forceinline__ void named_bar_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

}  // namespace tsm2
