// Element-wise path: any alignment of A, B, C and any leading dimensions.
//
// This follows Algorithm 3 of the paper (Sec. 3.1.3): one thread per row of A
// (outer-product accumulation of Algorithm 2, so each A element is loaded once
// per pass), with the rows of B for the current tile of the inner dimension
// staged in shared memory by the whole block and read back as broadcasts.
// It is the path for operands that the bulk-copy engine cannot address
// (unaligned base pointers or leading dimensions), and the first correct
// implementation the bulk-copy kernel is checked against.
#include "common.cuh"
#include "internal.h"

namespace tsm2 {

namespace {

constexpr int kSimpleThreads = 128;  // t1 of Algorithm 3: threads per block
constexpr int kSimpleTileB = 64;     // rows of B per shared-memory tile
constexpr int kSimpleKC = 16;        // t2: C columns per pass

template <typename T, int KC>
__global__ void __launch_bounds__(kSimpleThreads)
simple_kernel(int64_t m, int64_t n, int k, const T *__restrict__ A, int64_t lda,
              const T *__restrict__ B, int64_t ldb, T *__restrict__ C, int64_t ldc) {
    __shared__ T Bs[kSimpleTileB][KC];  // row-major tile: one row of B per j
    const int64_t row = (int64_t)blockIdx.x * kSimpleThreads + threadIdx.x;
    T acc[KC];
#pragma unroll
    for (int c = 0; c < KC; ++c) acc[c] = T(0);

    for (int64_t j0 = 0; j0 < n; j0 += kSimpleTileB) {
        __syncthreads();
        for (int t = threadIdx.x; t < kSimpleTileB * KC; t += kSimpleThreads) {
            const int jj = t % kSimpleTileB;
            const int c = t / kSimpleTileB;
            const int64_t j = j0 + jj;
            Bs[jj][c] = (j < n && c < k) ? B[j + (int64_t)c * ldb] : T(0);
        }
        __syncthreads();
        if (row < m) {
            const int jn = (int)((n - j0) < kSimpleTileB ? (n - j0) : kSimpleTileB);
            const T *a_col = A + row + j0 * lda;
            for (int jj = 0; jj < jn; ++jj) {
                const T a = a_col[(int64_t)jj * lda];
#pragma unroll
                for (int c = 0; c < KC; ++c) acc[c] = fma(a, Bs[jj][c], acc[c]);
            }
        }
    }
    if (row < m) {
#pragma unroll
        for (int c = 0; c < KC; ++c)
            if (c < k) C[row + (int64_t)c * ldc] = acc[c];
    }
}

template <typename T>
cudaError_t launch_t(const GemmArgs &g, cudaStream_t stream) {
    const int64_t blocks = (g.m + kSimpleThreads - 1) / kSimpleThreads;
    const T *A = static_cast<const T *>(g.A);
    const T *B = static_cast<const T *>(g.B);
    T *C = static_cast<T *>(g.C);
    // Narrow instantiations for small k keep registers (and occupancy) in line.
    if (g.k <= 2)
        simple_kernel<T, 2><<<(unsigned)blocks, kSimpleThreads, 0, stream>>>(g.m, g.n, g.k, A, g.lda, B, g.ldb, C, g.ldc);
    else if (g.k <= 4)
        simple_kernel<T, 4><<<(unsigned)blocks, kSimpleThreads, 0, stream>>>(g.m, g.n, g.k, A, g.lda, B, g.ldb, C, g.ldc);
    else if (g.k <= 8)
        simple_kernel<T, 8><<<(unsigned)blocks, kSimpleThreads, 0, stream>>>(g.m, g.n, g.k, A, g.lda, B, g.ldb, C, g.ldc);
    else
        simple_kernel<T, 16><<<(unsigned)blocks, kSimpleThreads, 0, stream>>>(g.m, g.n, g.k, A, g.lda, B, g.ldb, C, g.ldc);
    return cudaGetLastError();
}

}  // namespace

int simple_kc_max() { return kSimpleKC; }

cudaError_t simple_launch(int elem, const GemmArgs &g, unsigned * /*status*/, cudaStream_t stream) {
    if (g.m <= 0 || g.k <= 0) return cudaSuccess;
    if (elem == 8) return launch_t<double>(g, stream);
    return launch_t<float>(g, stream);
}

}  // namespace tsm2
