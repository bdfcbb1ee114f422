// Synthetic benchmark inputs generated in device memory.
//
// Same definition as the host-side generator (package tsm2_inputs):
// splitmix64 (Steele, Lea and Flood 2014) with stream key
// key = fmix(fmix(seed + G) + matrix_id * G), draw idx = fmix(key + (idx+1)*G),
// element (i, j) of a logical rows x cols matrix is draw i + j*rows.  Every
// distribution is formed with exact binary64 operations, so host and device
// agree bit for bit.  Not part of the multiply.
#include "tsm2.h"

#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;

__host__ __device__ inline uint64_t fmix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

inline uint64_t stream_key(uint64_t seed, uint64_t mid) { return fmix(fmix(seed + kGolden) + mid * kGolden); }

__device__ inline uint64_t draw(uint64_t key, uint64_t idx) { return fmix(key + (idx + 1) * kGolden); }

enum Dist { kUniform = 0, kIntSmall = 1, kNormalIH = 2, kLogMag = 3 };

__device__ inline double value_of(int dist, uint64_t key, uint64_t idx, double scale) {
    if (dist == kUniform) {
        const uint64_t x = draw(key, idx);
        return (double)(x >> 11) * 0x1p-52 - 1.0;
    }
    if (dist == kIntSmall) {
        const uint64_t x = draw(key, idx);
        return (double)((x >> 32) % 9ull) - 4.0;
    }
    if (dist == kNormalIH) {
        double s = 0.0;
        for (int t = 0; t < 12; ++t) {
            const double u = (double)(draw(key, idx * 12ull + (uint64_t)t) >> 11) * 0x1p-53;
            s = __dadd_rn(s, u);  // left to right, no reassociation
        }
        return __dmul_rn(__dadd_rn(s, -6.0), scale);
    }
    // kLogMag
    const uint64_t x = draw(key, idx);
    const int e = (int)((x >> 32) % 20ull) - 10;
    const double f = (double)((x >> 1) & 0x7FFFFFFFull);
    const double mag = ldexp(__dadd_rn(1.0, f * 0x1p-31), e);
    return (x & 1ull) ? -mag : mag;
}

template <typename T>
__global__ void fill_kernel(int64_t rows, int64_t cols, uint64_t key, int dist, double scale, T *X, int64_t ldx) {
    const int64_t total = rows * cols;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = t / rows;
        const int64_t i = t - j * rows;
        X[i + j * ldx] = (T)value_of(dist, key, (uint64_t)t, scale);  // binary32: round to nearest even
    }
}

template <typename T>
tsm2_status fill(int64_t rows, int64_t cols, uint64_t seed, uint64_t mid, int dist, double scale, T *X, int64_t ldx,
                 void *stream) {
    if (rows < 0 || cols < 0 || ldx < (rows > 1 ? rows : 1)) return TSM2_ERR_INVALID_VALUE;
    if (rows == 0 || cols == 0) return TSM2_SUCCESS;
    if (!X) return TSM2_ERR_INVALID_VALUE;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t total = rows * cols;
    int64_t blocks = (total + 255) / 256;
    const int64_t cap = (int64_t)(sms > 0 ? sms : 1) * 16;
    if (blocks > cap) blocks = cap;
    fill_kernel<T><<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(rows, cols, stream_key(seed, mid),
                                                                                    dist, scale, X, ldx);
    return cudaGetLastError() == cudaSuccess ? TSM2_SUCCESS : TSM2_ERR_CUDA;
}

// FMA throughput probe: every thread runs kChains independent multiply-add
// chains for `iters` steps (x <- x * a + c, no chain waits on another), so
// the FMA pipes, not latency, set the rate.  The values stay bounded (|a| < 1)
// and the chains' sum goes to `sink` so nothing is optimised away.
constexpr int kChains = 8;

__global__ void __launch_bounds__(256) fma_probe_f64(int64_t iters, double *sink) {
    double x[kChains];
    const double a = 0.999999 - 1e-9 * (threadIdx.x & 7), c = 1e-7 * (1 + (blockIdx.x & 3));
#pragma unroll
    for (int q = 0; q < kChains; ++q) x[q] = 0.5 + 0.01 * q + 1e-6 * threadIdx.x;
    for (int64_t it = 0; it < iters; ++it)
#pragma unroll
        for (int q = 0; q < kChains; ++q) x[q] = fma(x[q], a, c);
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kChains; ++q) s += x[q];
    sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// binary32 with packed FFMA2 (two lanes per instruction), as the kernels use.
__global__ void __launch_bounds__(256) fma_probe_f32(int64_t iters, float *sink) {
    float2 x[kChains];
    const float a = 0.9999f - 1e-6f * (threadIdx.x & 7), c = 1e-5f * (1 + (blockIdx.x & 3));
    const float2 aa = make_float2(a, a), cc = make_float2(c, c);
#pragma unroll
    for (int q = 0; q < kChains; ++q) x[q] = make_float2(0.5f + 0.01f * q, 0.25f + 1e-4f * threadIdx.x);
    for (int64_t it = 0; it < iters; ++it)
#pragma unroll
        for (int q = 0; q < kChains; ++q) x[q] = __ffma2_rn(x[q], aa, cc);
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < kChains; ++q) s += x[q].x + x[q].y;
    sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" {

tsm2_status tsm2_fma_probe(int elem, int blocks, int64_t iters, void *sink, void *stream) {
    if ((elem != 4 && elem != 8) || blocks < 1 || iters < 0 || !sink)
        return TSM2_ERR_INVALID_VALUE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (elem == 8)
        fma_probe_f64<<<blocks, 256, 0, st>>>(iters, static_cast<double *>(sink));
    else
        fma_probe_f32<<<blocks, 256, 0, st>>>(iters, static_cast<float *>(sink));
    return cudaGetLastError() == cudaSuccess ? TSM2_SUCCESS : TSM2_ERR_CUDA;
}

tsm2_status tsm2_fill_uniform_d(int64_t rows, int64_t cols, uint64_t seed, uint64_t mid, double *X, int64_t ldx,
                                void *stream) {
    return fill<double>(rows, cols, seed, mid, kUniform, 0.0, X, ldx, stream);
}
tsm2_status tsm2_fill_uniform_s(int64_t rows, int64_t cols, uint64_t seed, uint64_t mid, float *X, int64_t ldx,
                                void *stream) {
    return fill<float>(rows, cols, seed, mid, kUniform, 0.0, X, ldx, stream);
}
tsm2_status tsm2_fill_int_small_d(int64_t rows, int64_t cols, uint64_t seed, uint64_t mid, double *X, int64_t ldx,
                                  void *stream) {
    return fill<double>(rows, cols, seed, mid, kIntSmall, 0.0, X, ldx, stream);
}
tsm2_status tsm2_fill_int_small_s(int64_t rows, int64_t cols, uint64_t seed, uint64_t mid, float *X, int64_t ldx,
                                  void *stream) {
    return fill<float>(rows, cols, seed, mid, kIntSmall, 0.0, X, ldx, stream);
}
tsm2_status tsm2_fill_normal_ih_d(int64_t rows, int64_t cols, uint64_t seed, uint64_t mid, double scale, double *X,
                                  int64_t ldx, void *stream) {
    return fill<double>(rows, cols, seed, mid, kNormalIH, scale, X, ldx, stream);
}
tsm2_status tsm2_fill_normal_ih_s(int64_t rows, int64_t cols, uint64_t seed, uint64_t mid, double scale, float *X,
                                  int64_t ldx, void *stream) {
    return fill<float>(rows, cols, seed, mid, kNormalIH, scale, X, ldx, stream);
}
tsm2_status tsm2_fill_logmag_s(int64_t rows, int64_t cols, uint64_t seed, uint64_t mid, float *X, int64_t ldx,
                               void *stream) {
    return fill<float>(rows, cols, seed, mid, kLogMag, 0.0, X, ldx, stream);
}

}  // extern "C"
