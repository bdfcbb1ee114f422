// Copies of column-major blocks between page-locked host memory and device
// memory done by the SMs' own loads and stores (the host memory reached
// through its device-mapped address), for the host-operand entry points.
//
// On GB300 the copy engines' first pass over page-locked host buffers ran at
// 33 GB/s in a process started after many others had allocated and freed
// page-locked memory on the same host, against 211 GB/s on a freshly booted
// host, while SM loads of the same pages ran at 211 GB/s (the link rate) in
// both states.  Each copy block takes a whole SM (it reserves more than half of the
// SM's shared memory), so a copy kernel of G blocks leaves the other SMs to
// the product kernels running beside it.
#include "internal.h"

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace tsm2 {
namespace {

constexpr int kThreads = 1024;
constexpr int kUnroll = 4;                    // 16-byte loads in flight per thread
constexpr int kExclusiveSmem = 120 * 1024;    // > half of an SM: one copy block per SM

// Copies `cols` columns of `row_bytes` bytes: column c starts at
// src + c*lds and dst + c*ldd (bytes).  VEC: every column start of both sides
// is 16-byte aligned; the column body moves in 16-byte words and its last
// row_bytes % 16 bytes in 4-byte words.  Otherwise all of it moves in 4-byte
// words (column starts 4-byte aligned: elements are 4 or 8 bytes).
template <bool VEC>
__global__ void __launch_bounds__(kThreads, 1)
    copy2d_kernel(const char *__restrict__ src, int64_t lds, char *__restrict__ dst, int64_t ldd, int64_t row_bytes,
                  int64_t cols) {
    using W = typename std::conditional<VEC, uint4, unsigned>::type;
    constexpr int64_t WB = sizeof(W);
    const int64_t nw = row_bytes / WB;  // whole words per column
    const int64_t total = nw * cols;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; base < total; base += stride * kUnroll) {
        W r[kUnroll];
        int64_t off_d[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int64_t v = base + u * stride;
            off_d[u] = -1;
            if (v < total) {
                const int64_t c = v / nw, q = v - c * nw;
                r[u] = *reinterpret_cast<const W *>(src + c * lds + q * WB);
                off_d[u] = c * ldd + q * WB;
            }
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
            if (off_d[u] >= 0) *reinterpret_cast<W *>(dst + off_d[u]) = r[u];
    }
    if constexpr (VEC) {  // the last row_bytes % 16 bytes of every column, 4 bytes at a time
        const int64_t tw = (row_bytes - nw * WB) / 4;
        const int64_t ttot = tw * cols;
        for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < ttot; v += stride) {
            const int64_t c = v / tw, q = v - c * tw;
            const int64_t o = nw * WB + q * 4;
            *reinterpret_cast<unsigned *>(dst + c * ldd + o) = *reinterpret_cast<const unsigned *>(src + c * lds + o);
        }
    }
}

template <bool VEC>
cudaError_t launch(const char *src, int64_t lds, char *dst, int64_t ldd, int64_t row_bytes, int64_t cols, int grid,
                   cudaStream_t stream) {
    // Set on every launch: the attribute belongs to the current device.
    cudaError_t e = cudaFuncSetAttribute(copy2d_kernel<VEC>, cudaFuncAttributeMaxDynamicSharedMemorySize, kExclusiveSmem);
    if (e != cudaSuccess) return e;
    copy2d_kernel<VEC><<<grid, kThreads, kExclusiveSmem, stream>>>(src, lds, dst, ldd, row_bytes, cols);
    return cudaGetLastError();
}

}  // namespace

cudaError_t sm_copy2d_launch(const void *src, int64_t lds_bytes, void *dst, int64_t ldd_bytes, int64_t row_bytes,
                             int64_t cols, int grid, cudaStream_t stream) {
    if (row_bytes <= 0 || cols <= 0) return cudaSuccess;
    if (row_bytes % 4 || lds_bytes % 4 || ldd_bytes % 4 || (reinterpret_cast<uintptr_t>(src) & 3) ||
        (reinterpret_cast<uintptr_t>(dst) & 3))
        return cudaErrorInvalidValue;
    if (grid < 1) grid = 1;
    const bool vec = (reinterpret_cast<uintptr_t>(src) % 16 == 0) && (reinterpret_cast<uintptr_t>(dst) % 16 == 0) &&
                     lds_bytes % 16 == 0 && ldd_bytes % 16 == 0;
    const char *s = static_cast<const char *>(src);
    char *d = static_cast<char *>(dst);
    return vec ? launch<true>(s, lds_bytes, d, ldd_bytes, row_bytes, cols, grid, stream)
               : launch<false>(s, lds_bytes, d, ldd_bytes, row_bytes, cols, grid, stream);
}

}  // namespace tsm2
