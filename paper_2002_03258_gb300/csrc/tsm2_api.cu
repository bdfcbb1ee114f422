// C ABI of the library (declared in include/tsm2.h): argument checking,
// choice of kernel path and configuration, tensor-map encoding, workspace
// management and the device status word.
#include "common.cuh"
#include "internal.h"
#include "tsm2.h"

#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

namespace tsm2 {
namespace {

__device__ unsigned int g_status_word;  // per device; bits kStatusTimeout, kStatusBounds set by kernels

thread_local std::string t_last_error = "no error";
thread_local const char *t_last_config = "none";
thread_local const char *t_last_host_copy = "none";  // copy path of the last host-operand call

int64_t g_wait_ns = 1000000000LL;
int g_path = 0;
int g_grid_override = 0;
int g_host_copy = 0;               // 0: SM copies for device-mapped page-locked host buffers; 1: copy engines
int g_balance = 0;                 // 0: TSM2L row blocks claimed at run time; 1: static; 2: 0 + batched shares always adapted
thread_local int t_grid_cap = 0;   // > 0: upper bound of the product kernels' persistent grid (this thread)
unsigned long long *g_trace = nullptr;
int64_t g_trace_blocks = 0;

tsm2_status set_error(tsm2_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_last_error = buf;
    return s;
}

tsm2_status cuda_error(cudaError_t e, const char *what) {
    return set_error(TSM2_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

// ---- per-device state ------------------------------------------------------

struct DeviceState {
    bool init = false;
    int sm_count = 0;
    unsigned *status = nullptr;  // device address of g_status_word
};

std::mutex g_mu;
DeviceState g_dev[64];

struct Workspace {
    void *ptr = nullptr;
    size_t bytes = 0;
    size_t counter_bytes = 0;
};
std::map<std::pair<int, uintptr_t>, Workspace> g_ws;  // (device, stream) -> workspace

tsm2_status device_state(DeviceState **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return set_error(TSM2_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceState &d = g_dev[dev];
    if (!d.init) {
        e = cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_error(e, "cudaDeviceGetAttribute");
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_status_word);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(status)");
        d.status = static_cast<unsigned *>(p);
        d.init = true;
    }
    *out = &d;
    return TSM2_SUCCESS;
}

// Returns a workspace of at least `bytes` (256-byte aligned) whose first
// `counter_bytes` bytes are zero.  The counters return to zero after every
// completed launch, so they are only cleared when (re)allocated.
tsm2_status workspace(cudaStream_t stream, size_t counter_bytes, size_t slot_bytes, void **ws, int **counters) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    counter_bytes = (counter_bytes + 255) / 256 * 256;
    std::lock_guard<std::mutex> lk(g_mu);
    Workspace &w = g_ws[{dev, reinterpret_cast<uintptr_t>(stream)}];
    if (!w.ptr || w.counter_bytes < counter_bytes || w.bytes < w.counter_bytes + slot_bytes) {
        // Growing needs a synchronize and cudaMalloc, neither of which may
        // run while the stream is being captured into a graph.
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        e = cudaStreamIsCapturing(stream, &cap);
        if (e != cudaSuccess) return cuda_error(e, "cudaStreamIsCapturing");
        if (cap != cudaStreamCaptureStatusNone)
            return set_error(TSM2_ERR_UNSUPPORTED,
                             "the stream's workspace must grow, which cannot happen during stream capture: call the "
                             "largest shape once on this stream before capturing");
        const size_t cb = std::max(counter_bytes, w.counter_bytes);
        const size_t nb = std::max((cb + slot_bytes) * 5 / 4 + 4096, w.bytes);
        if (w.ptr) {
            // Pending work of this stream may still use the old buffer.
            e = cudaStreamSynchronize(stream);
            if (e != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize(workspace)");
            cudaFree(w.ptr);
            w = Workspace{};
        }
        void *p = nullptr;
        e = cudaMalloc(&p, nb);
        if (e != cudaSuccess) return cuda_error(e, "cudaMalloc(workspace)");
        e = cudaMemsetAsync(p, 0, cb, stream);
        if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync(workspace counters)");
        w.ptr = p;
        w.bytes = nb;
        w.counter_bytes = cb;
    }
    *counters = static_cast<int *>(w.ptr);
    *ws = static_cast<char *>(w.ptr) + w.counter_bytes;
    return TSM2_SUCCESS;
}

// Claim counters of the resident-B schedules: the first two counters of the
// stream's workspace (zero between launches; the kernel rearms them).  While
// the stream is being captured a workspace cannot be created, and the launch
// then keeps the static partition (nullptr).
tsm2_status claim_counters(cudaStream_t stream, int **claims) {
    *claims = nullptr;
    if (g_balance == 1) return TSM2_SUCCESS;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_ws.find({dev, reinterpret_cast<uintptr_t>(stream)});
        if (it != g_ws.end() && it->second.ptr && it->second.counter_bytes >= 2 * sizeof(int)) {
            *claims = static_cast<int *>(it->second.ptr);
            return TSM2_SUCCESS;
        }
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(stream, &cap);
    if (e != cudaSuccess) return cuda_error(e, "cudaStreamIsCapturing");
    if (cap != cudaStreamCaptureStatusNone) return TSM2_SUCCESS;
    void *ws = nullptr;
    return workspace(stream, 2 * sizeof(int), 0, &ws, claims);
}

// ---- tensor maps -----------------------------------------------------------

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

tsm2_status encode_2d_ex(CUtensorMap *map, CUtensorMapDataType dtype, int elem, const void *base, int64_t rows,
                         int64_t cols, int64_t ld, int box_rows, int box_cols, CUtensorMapSwizzle swizzle) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return set_error(TSM2_ERR_CUDA, "cuTensorMapEncodeTiled unavailable from the driver");
    const cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
    const cuuint64_t strides[1] = {(cuuint64_t)(ld * elem)};
    const cuuint32_t box[2] = {(cuuint32_t)box_rows, (cuuint32_t)box_cols};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(map, dtype, 2, const_cast<void *>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(TSM2_ERR_CUDA, "cuTensorMapEncodeTiled failed (CUresult %d)", (int)r);
    return TSM2_SUCCESS;
}

tsm2_status encode_2d(CUtensorMap *map, int elem, const void *base, int64_t rows, int64_t cols, int64_t ld,
                      int box_rows, int box_cols) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return set_error(TSM2_ERR_CUDA, "cuTensorMapEncodeTiled unavailable from the driver");
    const cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
    const cuuint64_t strides[1] = {(cuuint64_t)(ld * elem)};
    const cuuint32_t box[2] = {(cuuint32_t)box_rows, (cuuint32_t)box_cols};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(map, elem == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                          const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(TSM2_ERR_CUDA, "cuTensorMapEncodeTiled failed (CUresult %d)", (int)r);
    return TSM2_SUCCESS;
}

// ---- C-column widths --------------------------------------------------------

// Smallest compiled C-column width (KC) that holds a chunk of k columns: the
// kernels compute all KC columns (padding columns of B read as zero), so a
// close fit saves FMAs in the FMA-bound shapes.
int kc_for(int k) {
    static const int widths[] = {2, 4, 8, 12, 16, 24, 32};
    for (int w : widths)
        if (w >= k) return w;
    return 32;
}

// ---- argument checks ---------------------------------------------------------

bool ranges_overlap(const void *a, size_t abytes, const void *b, size_t bbytes) {
    if (!a || !b || !abytes || !bbytes) return false;
    const uintptr_t a0 = (uintptr_t)a, b0 = (uintptr_t)b;
    return a0 < b0 + bbytes && b0 < a0 + abytes;
}

size_t span_bytes(int64_t rows, int64_t cols, int64_t ld, int elem) {
    if (rows <= 0 || cols <= 0) return 0;
    return (size_t)(((cols - 1) * ld + rows) * elem);
}

tsm2_status check_args(const char *fn, int64_t m, int64_t n, int64_t k, const void *A, int64_t lda, const void *B,
                       int64_t ldb, const void *C, int64_t ldc, int elem) {
    if (m < 0 || n < 0 || k < 0)
        return set_error(TSM2_ERR_INVALID_VALUE, "%s: negative dimension (m=%lld n=%lld k=%lld)", fn, (long long)m,
                         (long long)n, (long long)k);
    if (lda < (m > 1 ? m : 1)) return set_error(TSM2_ERR_INVALID_VALUE, "%s: lda=%lld < max(1,m)", fn, (long long)lda);
    if (ldb < (n > 1 ? n : 1)) return set_error(TSM2_ERR_INVALID_VALUE, "%s: ldb=%lld < max(1,n)", fn, (long long)ldb);
    if (ldc < (m > 1 ? m : 1)) return set_error(TSM2_ERR_INVALID_VALUE, "%s: ldc=%lld < max(1,m)", fn, (long long)ldc);
    if (m > 0 && k > 0 && C == nullptr) return set_error(TSM2_ERR_INVALID_VALUE, "%s: C is NULL", fn);
    if (m > 0 && n > 0 && k > 0 && A == nullptr) return set_error(TSM2_ERR_INVALID_VALUE, "%s: A is NULL", fn);
    if (m > 0 && n > 0 && k > 0 && B == nullptr) return set_error(TSM2_ERR_INVALID_VALUE, "%s: B is NULL", fn);
    if (m > 0 && k > 0) {
        const size_t cb = span_bytes(m, k, ldc, elem);
        if ((n > 0 && ranges_overlap(C, cb, A, span_bytes(m, n, lda, elem))) ||
            (n > 0 && ranges_overlap(C, cb, B, span_bytes(n, k, ldb, elem))))
            return set_error(TSM2_ERR_INVALID_VALUE, "%s: C overlaps A or B", fn);
    }
    return TSM2_SUCCESS;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// ---- the multiply ------------------------------------------------------------

tsm2_status gemm(const char *fn, char op, int elem, int64_t m, int64_t n, int64_t k, const void *A, int64_t lda,
                 const void *B, int64_t ldb, void *C, int64_t ldc, void *stream_v) {
    tsm2_status st = check_args(fn, m, n, k, A, lda, B, ldb, C, ldc, elem);
    if (st != TSM2_SUCCESS) return st;
    if (m == 0 || k == 0) {
        t_last_config = "empty";
        return TSM2_SUCCESS;
    }
    cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
    if (n == 0) {
        t_last_config = "zero-fill";
        cudaError_t e = cudaMemset2DAsync(C, (size_t)ldc * elem, 0, (size_t)m * elem, (size_t)k, stream);
        return e == cudaSuccess ? TSM2_SUCCESS : cuda_error(e, "cudaMemset2DAsync");
    }
    DeviceState *dev = nullptr;
    st = device_state(&dev);
    if (st != TSM2_SUCCESS) return st;

    // TSM2L keeps B resident when n <= 64 and stages it with A otherwise
    // (whole row blocks either way).
    const bool staged_l = op == 'l' && n > 64;
    // The bulk-copy path needs 16-byte aligned bases and row strides, and
    // 32-bit tensor coordinates.  Resident B is read with ordinary loads, so
    // only A matters there.
    const bool a_ok = aligned16(A) && ((lda * elem) % 16 == 0) && m < (1ll << 31) - 4096 && n < (1ll << 31);
    const bool b_ok = (op == 'l' && !staged_l) || (aligned16(B) && ((ldb * elem) % 16 == 0));
    const bool use_stream = g_path != 1 && a_ok && b_ok;

    const int kc_max = use_stream ? (op == 'l' ? 32 : 16) : simple_kc_max();
    for (int64_t c0 = 0; c0 < k; c0 += kc_max) {
        GemmArgs g;
        g.m = m;
        g.n = n;
        g.k = (int)((k - c0) < kc_max ? (k - c0) : kc_max);
        g.A = A;
        g.lda = lda;
        g.B = static_cast<const char *>(B) + (size_t)c0 * ldb * elem;
        g.ldb = ldb;
        g.C = static_cast<char *>(C) + (size_t)c0 * ldc * elem;
        g.ldc = ldc;
        cudaError_t e;
        if (!use_stream) {
            t_last_config = elem == 8 ? "simple_f64" : "simple_f32";
            e = simple_launch(elem, g, dev->status, stream);
            if (e != cudaSuccess) return cuda_error(e, "simple kernel launch");
            continue;
        }
        int kc = kc_for(g.k);
        if (staged_l && kc < 4) kc = 4;  // staged-B TSM2L: C columns in groups of four
        const StreamShape *shape = stream_shape(elem, staged_l ? 't' : op, kc);
        if (op == 'l' && !staged_l) {
            // Tall A and wide C: the 8-rows-per-lane schedule (KC = 24, 32)
            // once every SM gets enough of its (larger) row blocks.  Measured
            // on GB300: KC = 24 wins from about 1.5 row blocks per SM (5-11%
            // at 2^18 .. 2^20 rows, a tie below), KC = 32 needs about 6.
            const StreamShape *wide = stream_shape(elem, 'w', kc);
            const int64_t min_rb_per_sm = kc == 24 ? 1 : 6;
            if (wide && (m + wide->BM - 1) / wide->BM >= min_rb_per_sm * (int64_t)dev->sm_count) shape = wide;
        }
        if (!shape) return set_error(TSM2_ERR_UNSUPPORTED, "%s: no kernel configuration for k chunk %d", fn, g.k);
        StreamLaunch L;
        std::memset(&L, 0, sizeof L);
        L.g = g;
        st = encode_2d(&L.mapA, elem, A, m, n, lda, shape->BOXM, shape->BNS);
        if (st != TSM2_SUCCESS) return st;
        if (!shape->b_resident) {
            st = encode_2d(&L.mapB, elem, g.B, n, g.k, ldb, shape->BNS, shape->KC);
            if (st != TSM2_SUCCESS) return st;
        }
        const int64_t num_rb = (m + shape->BM - 1) / shape->BM;
        const int64_t upr = (n + shape->BNS - 1) / shape->BNS;
        const bool whole = shape->gran_rows == 0;  // row blocks never split: no partial sums
        const int64_t ngroups = whole ? num_rb : num_rb * upr;
        int64_t grid = dev->sm_count;
        if (!whole) {
            // At least four stages per block so partial sums stay a small
            // fraction of the traffic.
            const int64_t cap = (num_rb * upr) / 4;
            if (cap < grid) grid = cap;
        }
        if (grid > ngroups) grid = ngroups;
        if (g_grid_override > 0) grid = g_grid_override < ngroups ? g_grid_override : ngroups;
        if (t_grid_cap > 0 && grid > t_grid_cap) grid = t_grid_cap;
        if (grid < 1) grid = 1;
        L.grid = (int)grid;
        void *ws = nullptr;
        int *counters = nullptr;
        if (!shape->b_resident && !whole) {
            const size_t slots = (size_t)(grid + num_rb) * shape->KC * shape->BM * elem;
            st = workspace(stream, (size_t)num_rb * sizeof(int), slots, &ws, &counters);
            if (st != TSM2_SUCCESS) return st;
        }
        L.ws = ws;
        L.counters = counters;
        if (shape->b_resident) {
            st = claim_counters(stream, &L.claims);
            if (st != TSM2_SUCCESS) return st;
        }
        L.status = dev->status;
        L.wait_ns = g_wait_ns;
        L.c_vec = aligned16(g.C) && ((ldc * elem) % 16 == 0);
        L.trace = (g_trace && g_trace_blocks >= grid) ? g_trace : nullptr;
        t_last_config = shape->name;
        e = stream_launch(shape, L, stream);
        if (e != cudaSuccess) return cuda_error(e, "stream kernel launch");
    }
    return TSM2_SUCCESS;
}

// ---- backward products ------------------------------------------------------

tsm2_status gemm_t(const char *fn, int elem, int64_t m, int64_t n, int64_t k, const void *A, int64_t lda,
                   const void *dC, int64_t lddc, void *dB, int64_t lddb, void *stream_v) {
    if (m < 0 || n < 0 || k < 0)
        return set_error(TSM2_ERR_INVALID_VALUE, "%s: negative dimension (m=%lld n=%lld k=%lld)", fn, (long long)m,
                         (long long)n, (long long)k);
    if (lda < (m > 1 ? m : 1)) return set_error(TSM2_ERR_INVALID_VALUE, "%s: lda=%lld < max(1,m)", fn, (long long)lda);
    if (lddc < (m > 1 ? m : 1))
        return set_error(TSM2_ERR_INVALID_VALUE, "%s: lddc=%lld < max(1,m)", fn, (long long)lddc);
    if (lddb < (n > 1 ? n : 1))
        return set_error(TSM2_ERR_INVALID_VALUE, "%s: lddb=%lld < max(1,n)", fn, (long long)lddb);
    if (n > 0 && k > 0 && dB == nullptr) return set_error(TSM2_ERR_INVALID_VALUE, "%s: dB is NULL", fn);
    if (m > 0 && n > 0 && k > 0 && (A == nullptr || dC == nullptr))
        return set_error(TSM2_ERR_INVALID_VALUE, "%s: A or dC is NULL", fn);
    if (n > 0 && k > 0 && m > 0) {
        const size_t ob = span_bytes(n, k, lddb, elem);
        if (ranges_overlap(dB, ob, A, span_bytes(m, n, lda, elem)) ||
            ranges_overlap(dB, ob, dC, span_bytes(m, k, lddc, elem)))
            return set_error(TSM2_ERR_INVALID_VALUE, "%s: dB overlaps A or dC", fn);
    }
    if (n == 0 || k == 0) {
        t_last_config = "empty";
        return TSM2_SUCCESS;
    }
    cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
    if (m == 0) {
        t_last_config = "zero-fill";
        cudaError_t e = cudaMemset2DAsync(dB, (size_t)lddb * elem, 0, (size_t)n * elem, (size_t)k, stream);
        return e == cudaSuccess ? TSM2_SUCCESS : cuda_error(e, "cudaMemset2DAsync");
    }
    DeviceState *dev = nullptr;
    tsm2_status st = device_state(&dev);
    if (st != TSM2_SUCCESS) return st;
    const bool ok = g_path != 1 && aligned16(A) && aligned16(dC) && (lda * elem) % 16 == 0 &&
                    (lddc * elem) % 16 == 0 && m < (1ll << 31) - 4096 && n < (1ll << 31);
    for (int64_t c0 = 0; c0 < k; c0 += 16) {
        const int kk = (int)((k - c0) < 16 ? (k - c0) : 16);
        const void *dCc = static_cast<const char *>(dC) + (size_t)c0 * lddc * elem;
        void *dBc = static_cast<char *>(dB) + (size_t)c0 * lddb * elem;
        cudaError_t e;
        if (!ok) {
            t_last_config = elem == 8 ? "simple_t_f64" : "simple_t_f32";
            e = simple_t_launch(elem, m, n, kk, A, lda, dCc, lddc, dBc, lddb, stream);
            if (e != cudaSuccess) return cuda_error(e, "simple_t kernel launch");
            continue;
        }
        int kc = 2;
        while (kc < kk) kc *= 2;
        const TShape *shape = tsm2t_shape(elem, kc);
        if (!shape) return set_error(TSM2_ERR_UNSUPPORTED, "%s: no configuration for k chunk %d", fn, kk);
        TLaunch L;
        std::memset(&L, 0, sizeof L);
        L.m = m;
        L.n = n;
        L.k = kk;
        st = encode_2d(&L.mapA, elem, A, m, n, lda, shape->BOXM, shape->BNS);
        if (st != TSM2_SUCCESS) return st;
        st = encode_2d(&L.mapD, elem, dCc, m, kk, lddc, shape->BOXM, shape->KC);
        if (st != TSM2_SUCCESS) return st;
        const int64_t nrb = (m + shape->BM - 1) / shape->BM;
        const int64_t nch = (n + shape->BNS - 1) / shape->BNS;
        const int64_t nunits = nrb * nch;
        int64_t grid = dev->sm_count;
        if (nunits / 4 < grid) grid = nunits / 4;
        if (g_grid_override > 0) grid = g_grid_override;
        if (grid > nunits) grid = nunits;
        if (grid < 1) grid = 1;
        void *ws = nullptr;
        int *counters = nullptr;
        st = workspace(stream, (size_t)nch * sizeof(int), (size_t)(grid + nch) * shape->BNS * shape->KC * elem, &ws,
                       &counters);
        if (st != TSM2_SUCCESS) return st;
        L.dB = dBc;
        L.lddb = lddb;
        L.ws = ws;
        L.counters = counters;
        L.status = dev->status;
        L.wait_ns = g_wait_ns;
        L.grid = (int)grid;
        t_last_config = shape->name;
        e = tsm2t_launch(shape, L, stream);
        if (e != cudaSuccess) return cuda_error(e, "transposed kernel launch");
    }
    return TSM2_SUCCESS;
}

tsm2_status rankk(const char *fn, int elem, int64_t m, int64_t n, int64_t k, const void *dC, int64_t lddc,
                  const void *B, int64_t ldb, void *dA, int64_t ldda, void *stream_v) {
    if (m < 0 || n < 0 || k < 0)
        return set_error(TSM2_ERR_INVALID_VALUE, "%s: negative dimension (m=%lld n=%lld k=%lld)", fn, (long long)m,
                         (long long)n, (long long)k);
    if (lddc < (m > 1 ? m : 1))
        return set_error(TSM2_ERR_INVALID_VALUE, "%s: lddc=%lld < max(1,m)", fn, (long long)lddc);
    if (ldb < (n > 1 ? n : 1)) return set_error(TSM2_ERR_INVALID_VALUE, "%s: ldb=%lld < max(1,n)", fn, (long long)ldb);
    if (ldda < (m > 1 ? m : 1))
        return set_error(TSM2_ERR_INVALID_VALUE, "%s: ldda=%lld < max(1,m)", fn, (long long)ldda);
    if (m > 0 && n > 0 && dA == nullptr) return set_error(TSM2_ERR_INVALID_VALUE, "%s: dA is NULL", fn);
    if (m > 0 && n > 0 && k > 0 && (dC == nullptr || B == nullptr))
        return set_error(TSM2_ERR_INVALID_VALUE, "%s: dC or B is NULL", fn);
    if (m > 0 && n > 0 && k > 0) {
        const size_t ob = span_bytes(m, n, ldda, elem);
        if (ranges_overlap(dA, ob, dC, span_bytes(m, k, lddc, elem)) ||
            ranges_overlap(dA, ob, B, span_bytes(n, k, ldb, elem)))
            return set_error(TSM2_ERR_INVALID_VALUE, "%s: dA overlaps dC or B", fn);
    }
    if (m == 0 || n == 0) {
        t_last_config = "empty";
        return TSM2_SUCCESS;
    }
    cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
    if (k == 0) {
        t_last_config = "zero-fill";
        cudaError_t e = cudaMemset2DAsync(dA, (size_t)ldda * elem, 0, (size_t)m * elem, (size_t)n, stream);
        return e == cudaSuccess ? TSM2_SUCCESS : cuda_error(e, "cudaMemset2DAsync");
    }
    DeviceState *dev = nullptr;
    tsm2_status st = device_state(&dev);
    if (st != TSM2_SUCCESS) return st;
    const bool vec_ok = aligned16(dA) && (ldda * elem) % 16 == 0;
    t_last_config = elem == 8 ? "rankk_f64" : "rankk_f32";
    for (int64_t c0 = 0; c0 < k; c0 += 16) {
        const int kk = (int)((k - c0) < 16 ? (k - c0) : 16);
        cudaError_t e = rankk_launch(elem, m, n, kk, static_cast<const char *>(dC) + (size_t)c0 * lddc * elem, lddc,
                                     static_cast<const char *>(B) + (size_t)c0 * ldb * elem, ldb, dA, ldda, vec_ok,
                                     c0 > 0, dev->sm_count, stream);
        if (e != cudaSuccess) return cuda_error(e, "rank-k kernel launch");
    }
    return TSM2_SUCCESS;
}

// ---- bfloat16 A (tensor cores) -------------------------------------------------

tsm2_status gemm_bf16(int64_t m, int64_t n, int64_t k, const void *A_hi, const void *A_lo, int64_t lda,
                      const float *B, int64_t ldb, float *C, int64_t ldc, void *stream_v) {
    const char *fn = "tsm2r_bf16";
    if (m < 0 || n < 0 || k < 0)
        return set_error(TSM2_ERR_INVALID_VALUE, "%s: negative dimension (m=%lld n=%lld k=%lld)", fn, (long long)m,
                         (long long)n, (long long)k);
    if (lda < (m > 1 ? m : 1)) return set_error(TSM2_ERR_INVALID_VALUE, "%s: lda=%lld < max(1,m)", fn, (long long)lda);
    if (ldb < (n > 1 ? n : 1)) return set_error(TSM2_ERR_INVALID_VALUE, "%s: ldb=%lld < max(1,n)", fn, (long long)ldb);
    if (ldc < (m > 1 ? m : 1)) return set_error(TSM2_ERR_INVALID_VALUE, "%s: ldc=%lld < max(1,m)", fn, (long long)ldc);
    if (m > 0 && k > 0 && C == nullptr) return set_error(TSM2_ERR_INVALID_VALUE, "%s: C is NULL", fn);
    if (m > 0 && n > 0 && k > 0 && (A_hi == nullptr || B == nullptr))
        return set_error(TSM2_ERR_INVALID_VALUE, "%s: A_hi or B is NULL", fn);
    if (m > 0 && n > 0 && k > 0) {
        const size_t cb = span_bytes(m, k, ldc, 4);
        const size_t ab = span_bytes(m, n, lda, 2);
        if (ranges_overlap(C, cb, A_hi, ab) || ranges_overlap(C, cb, A_lo, ab) ||
            ranges_overlap(C, cb, B, span_bytes(n, k, ldb, 4)))
            return set_error(TSM2_ERR_INVALID_VALUE, "%s: C overlaps A_hi, A_lo or B", fn);
    }
    if (m == 0 || k == 0) {
        t_last_config = "empty";
        return TSM2_SUCCESS;
    }
    cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
    if (n == 0) {
        t_last_config = "zero-fill";
        cudaError_t e = cudaMemset2DAsync(C, (size_t)ldc * 4, 0, (size_t)m * 4, (size_t)k, stream);
        return e == cudaSuccess ? TSM2_SUCCESS : cuda_error(e, "cudaMemset2DAsync");
    }
    DeviceState *dev = nullptr;
    tsm2_status st = device_state(&dev);
    if (st != TSM2_SUCCESS) return st;
    const bool ok = g_path != 1 && aligned16(A_hi) && (A_lo == nullptr || aligned16(A_lo)) && (lda * 2) % 16 == 0 &&
                    m < (1ll << 31) - 4096 && n < (1ll << 31);
    for (int64_t c0 = 0; c0 < k; c0 += 16) {
        const int kk = (int)((k - c0) < 16 ? (k - c0) : 16);
        const float *Bc = B + c0 * ldb;
        float *Cc = C + c0 * ldc;
        cudaError_t e;
        if (!ok) {
            t_last_config = "simple_bf16";
            e = bf16_simple_launch(m, n, kk, A_hi, A_lo, lda, Bc, ldb, Cc, ldc, stream);
            if (e != cudaSuccess) return cuda_error(e, "bf16 element-wise kernel launch");
            continue;
        }
        BF16Launch L;
        std::memset(&L, 0, sizeof L);
        L.m = m;
        L.n = n;
        L.k = kk;
        L.hilo = A_lo != nullptr;
        st = encode_2d_ex(&L.mapHi, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, A_hi, m, n, lda, 64, bf16_bk(L.hilo),
                          CU_TENSOR_MAP_SWIZZLE_128B);
        if (st != TSM2_SUCCESS) return st;
        if (L.hilo) {
            st = encode_2d_ex(&L.mapLo, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, A_lo, m, n, lda, 64, bf16_bk(L.hilo),
                              CU_TENSOR_MAP_SWIZZLE_128B);
            if (st != TSM2_SUCCESS) return st;
        }
        const int64_t num_rb = (m + bf16_bm() - 1) / bf16_bm();
        const int64_t upr = (n + bf16_bk(L.hilo) - 1) / bf16_bk(L.hilo);
        const int64_t ngroups = num_rb * upr;
        int64_t grid = dev->sm_count;
        if (ngroups / 4 < grid) grid = ngroups / 4;
        if (g_grid_override > 0) grid = g_grid_override;
        if (grid > ngroups) grid = ngroups;
        if (grid < 1) grid = 1;
        const size_t pieces = (bf16_bpieces_bytes(n, L.hilo) + 255) / 256 * 256;
        const size_t slots = (size_t)(grid + num_rb) * 16 * bf16_bm() * 4;
        void *ws = nullptr;
        int *counters = nullptr;
        st = workspace(stream, (size_t)num_rb * sizeof(int), pieces + slots, &ws, &counters);
        if (st != TSM2_SUCCESS) return st;
        e = bf16_prep_b(n, kk, Bc, ldb, ws, L.hilo, stream);
        if (e != cudaSuccess) return cuda_error(e, "bf16 B split kernel launch");
        L.bpieces = ws;
        L.ws = static_cast<char *>(ws) + pieces;
        L.counters = counters;
        L.C = Cc;
        L.ldc = ldc;
        L.status = dev->status;
        L.wait_ns = g_wait_ns;
        L.grid = (int)grid;
        t_last_config = L.hilo ? "tc_bf16_hilo" : "tc_bf16";
        e = bf16_launch(L, stream);
        if (e != cudaSuccess) return cuda_error(e, "bf16 tensor-core kernel launch");
    }
    return TSM2_SUCCESS;
}

// ---- batched problems ----------------------------------------------------------

}  // namespace
}  // namespace tsm2

struct tsm2_batch_plan_s {
    struct Cls {
        const tsm2::BatchClass *cls = nullptr;
        int slot = 0;             // slot of the class in the menu's kernel
        std::vector<tsm2::ProbDesc> host;
        int64_t ngroups = 0, nrb = 0;
        double bytes = 0;
        tsm2::ProbDesc *d_probs = nullptr;
        void *d_ws = nullptr;     // counters, then partial-sum slots
        size_t counter_bytes = 0;
        int grid = 1;             // blocks of the class in the concurrent mode
        cudaStream_t aux = nullptr;
        cudaEvent_t done = nullptr;
    };
    struct Zero {
        void *C;
        int64_t ldc, m, k;
    };
    int dev = 0;
    int sm_count = 0;
    int variant = 0;
    const tsm2::BatchMenu *menu = nullptr;
    int mode = TSM2_BATCH_SINGLE_LAUNCH;
    int single_grid = 0;             // blocks of the single launch
    std::vector<Cls> classes;
    std::vector<Zero> zeros;
    cudaEvent_t fork = nullptr;
    cudaGraphExec_t graph = nullptr;
    cudaStream_t capture = nullptr;  // private stream the graph is captured on
    double total_bytes = 0;
    tsm2::BatchBalance *d_bal = nullptr;  // adaptive TSM2L shares of the single launch
};

namespace tsm2 {
namespace {

// Live plans, so that a timeout can reset their arrival counters.
std::mutex g_plans_mu;
std::vector<tsm2_batch_plan_s *> g_plans;

void destroy_plan(tsm2_batch_plan_s *P) {
    if (!P) return;
    {
        std::lock_guard<std::mutex> lk(g_plans_mu);
        g_plans.erase(std::remove(g_plans.begin(), g_plans.end(), P), g_plans.end());
    }
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(P->dev);
    if (P->graph) cudaGraphExecDestroy(P->graph);
    for (auto &c : P->classes) {
        if (c.d_probs) cudaFree(c.d_probs);
        if (c.d_ws) cudaFree(c.d_ws);
        if (c.aux) cudaStreamDestroy(c.aux);
        if (c.done) cudaEventDestroy(c.done);
    }
    if (P->fork) cudaEventDestroy(P->fork);
    if (P->capture) cudaStreamDestroy(P->capture);
    if (P->d_bal) cudaFree(P->d_bal);
    cudaSetDevice(cur);
    delete P;
}

// Arrival counters of every live plan on device `dev` back to zero (after a
// launch that gave up, they may be left non-zero).
void reset_plan_counters(int dev) {
    std::lock_guard<std::mutex> lk(g_plans_mu);
    for (tsm2_batch_plan_s *P : g_plans)
        if (P->dev == dev) {
            for (auto &c : P->classes)
                if (c.d_ws) cudaMemset(c.d_ws, 0, c.counter_bytes);
            if (P->d_bal) cudaMemset(P->d_bal, 0, 4 * sizeof(int));  // epoch, done, bad
        }
}

void class_params(const tsm2_batch_plan_s::Cls &c, ClassParams &cp) {
    cp.probs = c.d_probs;
    cp.nprob = (int)c.host.size();
    cp.whole = c.cls->op == 'w' ? 1 : 0;
    cp.ngroups = c.ngroups;
    cp.counters = static_cast<int *>(c.d_ws);
    cp.ws = reinterpret_cast<float *>(static_cast<char *>(c.d_ws) + c.counter_bytes);
    cp.nrb = c.nrb;
}

// Adaptive TSM2L shares pay off when the TSM2L phase is long against the
// launch-to-launch noise of when blocks reach it.  Measured on GB300 (one
// launch, median of 15): the 512-problem batch (42.8 GB) 1.4-2.2% faster,
// its first 120 problems (9.3 GB) 0.4-1% slower, its first 40 (3.4 GB) 5%
// slower.  Plans below this size keep equal shares.
constexpr double kAdaptMinBytes = 16e9;

// One launch of the plan's batch kernel over the classes [lo, hi) (all
// other slots empty) on `grid` blocks; `adapt`: TSM2L shares from the plan's
// adaptive weights.
tsm2_status launch_classes(tsm2_batch_plan_s *P, int lo, int hi, int grid, cudaStream_t stream, bool adapt = false) {
    DeviceState *dev = nullptr;
    tsm2_status st = device_state(&dev);
    if (st != TSM2_SUCCESS) return st;
    BatchKParams kp;
    std::memset(&kp, 0, sizeof kp);
    for (int i = lo; i < hi; ++i) class_params(P->classes[i], kp.cls[P->classes[i].slot]);
    kp.status = dev->status;
    kp.wait_ns = g_wait_ns;
    kp.trace = (g_trace && g_trace_blocks >= grid) ? g_trace : nullptr;
    kp.bal = (adapt && g_balance != 1 && grid <= kBalanceMaxBlocks) ? P->d_bal : nullptr;
    const cudaError_t e = P->menu->launch(kp, grid < 1 ? 1 : grid, stream);
    return e == cudaSuccess ? TSM2_SUCCESS : cuda_error(e, "batch kernel launch");
}

int class_grid_alone(const tsm2_batch_plan_s *P, int i) {
    return (int)std::min<int64_t>(P->sm_count, P->classes[i].ngroups);
}

tsm2_status plan_execute(tsm2_batch_plan_s *P, cudaStream_t stream, int only) {
    cudaError_t e;
    const int nc = (int)P->classes.size();
    if (only >= 0) return launch_classes(P, only, only + 1, class_grid_alone(P, only), stream);
    for (const auto &z : P->zeros) {
        e = cudaMemset2DAsync(z.C, (size_t)z.ldc * 4, 0, (size_t)z.m * 4, (size_t)z.k, stream);
        if (e != cudaSuccess) return cuda_error(e, "cudaMemset2DAsync");
    }
    if (nc == 0) return TSM2_SUCCESS;
    if (P->mode == TSM2_BATCH_SINGLE_LAUNCH)
        return launch_classes(P, 0, nc, P->single_grid, stream, g_balance == 2 || P->total_bytes >= kAdaptMinBytes);
    if (P->mode == TSM2_BATCH_SERIAL) {
        for (int i = 0; i < nc; ++i) {
            tsm2_status s = launch_classes(P, i, i + 1, class_grid_alone(P, i), stream);
            if (s != TSM2_SUCCESS) return s;
        }
        return TSM2_SUCCESS;
    }
    // Concurrent: every class on its own SM share, forked onto the plan's
    // streams and joined back.
    if (nc > 1) {
        e = cudaEventRecord(P->fork, stream);
        if (e != cudaSuccess) return cuda_error(e, "cudaEventRecord");
    }
    for (int i = 0; i < nc; ++i) {
        auto &c = P->classes[i];
        cudaStream_t s = i == 0 ? stream : c.aux;
        if (i > 0) {
            e = cudaStreamWaitEvent(s, P->fork, 0);
            if (e != cudaSuccess) return cuda_error(e, "cudaStreamWaitEvent");
        }
        tsm2_status st = launch_classes(P, i, i + 1, c.grid, s);
        if (st != TSM2_SUCCESS) return st;
        if (i > 0) {
            e = cudaEventRecord(c.done, s);
            if (e != cudaSuccess) return cuda_error(e, "cudaEventRecord");
            e = cudaStreamWaitEvent(stream, c.done, 0);
            if (e != cudaSuccess) return cuda_error(e, "cudaStreamWaitEvent");
        }
    }
    return TSM2_SUCCESS;
}

// ---- allocation-free variant of the binary32 TSM2R bulk-copy path -----------
//
// Some callers cannot call cudaMalloc at all: a process whose device memory is
// entirely owned by another allocator (for example a framework's caching pool
// that has already reserved the free memory), or a latency-bound loop that
// must not pay cudaMalloc's cost and implicit synchronisation.  For them,
// tsm2r_s_noalloc keeps the partial sums of split row blocks and their
// arrival counters in this fixed, file-scope device array instead of the
// lazily allocated workspace.  Every GPU that loads the library holds these
// bytes until the process exits.

constexpr size_t kNoAllocScratchBytes = 16u << 20;     // 16 MiB
constexpr size_t kNoAllocCounterBytes = 64u << 10;     // first 64 KiB: arrival counters
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[64];  // device address of g_noalloc_scratch, per device

// Host code may not pass g_noalloc_scratch itself to a kernel: on the host
// that name is only a stand-in for the device array.  Its device address is
// looked up once per device, with that device current.
tsm2_status noalloc_scratch(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return set_error(TSM2_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(no-alloc scratch)");
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return TSM2_SUCCESS;
}

tsm2_status gemm_r32_noalloc(int64_t m, int64_t n, int64_t k, const float *A, int64_t lda, const float *B,
                             int64_t ldb, float *C, int64_t ldc, void *stream_v) {
    const char *fn = "tsm2r_s_noalloc";
    const int elem = 4;
    tsm2_status st = check_args(fn, m, n, k, A, lda, B, ldb, C, ldc, elem);
    if (st != TSM2_SUCCESS) return st;
    if (m == 0 || k == 0) {
        t_last_config = "empty";
        return TSM2_SUCCESS;
    }
    cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
    if (n == 0) {
        t_last_config = "zero-fill";
        cudaError_t e = cudaMemset2DAsync(C, (size_t)ldc * elem, 0, (size_t)m * elem, (size_t)k, stream);
        return e == cudaSuccess ? TSM2_SUCCESS : cuda_error(e, "cudaMemset2DAsync");
    }
    DeviceState *dev = nullptr;
    st = device_state(&dev);
    if (st != TSM2_SUCCESS) return st;
    const bool a_ok = aligned16(A) && ((lda * elem) % 16 == 0) && m < (1ll << 31) - 4096 && n < (1ll << 31);
    const bool b_ok = aligned16(B) && ((ldb * elem) % 16 == 0);
    const bool use_stream = g_path != 1 && a_ok && b_ok;
    void *scratch = nullptr;
    if (use_stream) {
        st = noalloc_scratch(&scratch);
        if (st != TSM2_SUCCESS) return st;
    }
    const int kc_max = use_stream ? 16 : simple_kc_max();
    for (int64_t c0 = 0; c0 < k; c0 += kc_max) {
        GemmArgs g;
        g.m = m;
        g.n = n;
        g.k = (int)((k - c0) < kc_max ? (k - c0) : kc_max);
        g.A = A;
        g.lda = lda;
        g.B = reinterpret_cast<const char *>(B) + (size_t)c0 * ldb * elem;
        g.ldb = ldb;
        g.C = reinterpret_cast<char *>(C) + (size_t)c0 * ldc * elem;
        g.ldc = ldc;
        cudaError_t e;
        if (!use_stream) {  // element-wise path: needs no scratch at all
            t_last_config = "simple_f32";
            e = simple_launch(elem, g, dev->status, stream);
            if (e != cudaSuccess) return cuda_error(e, "simple kernel launch");
            continue;
        }
        const int kc = kc_for(g.k);
        const StreamShape *shape = stream_shape(elem, 'r', kc);
        if (!shape) return set_error(TSM2_ERR_UNSUPPORTED, "%s: no kernel configuration for k chunk %d", fn, g.k);
        const int64_t num_rb = (m + shape->BM - 1) / shape->BM;
        const int64_t upr = (n + shape->BNS - 1) / shape->BNS;
        const int64_t ngroups = num_rb * upr;
        int64_t grid = dev->sm_count;
        const int64_t cap = ngroups / 4;
        if (cap < grid) grid = cap;
        if (g_grid_override > 0) grid = g_grid_override < ngroups ? g_grid_override : ngroups;
        if (grid > ngroups) grid = ngroups;
        if (grid < 1) grid = 1;
        const size_t counter_bytes = (size_t)num_rb * sizeof(int);
        // Partial-sum slots of split row blocks.
        const size_t slot_bytes = (size_t)(grid + num_rb) * shape->KC * shape->BM * elem;
        const size_t data_cap = kNoAllocScratchBytes - kNoAllocCounterBytes;
        if (counter_bytes > kNoAllocCounterBytes || slot_bytes > data_cap)
            return set_error(TSM2_ERR_UNSUPPORTED,
                             "%s: m=%lld n=%lld needs %zu bytes of counters and %zu bytes of partial sums; "
                             "the static scratch holds %zu and %zu; use tsm2r_s instead",
                             fn, (long long)m, (long long)n, counter_bytes, slot_bytes, kNoAllocCounterBytes,
                             data_cap);
        StreamLaunch L;
        std::memset(&L, 0, sizeof L);
        L.g = g;
        st = encode_2d(&L.mapA, elem, A, m, n, lda, shape->BOXM, shape->BNS);
        if (st != TSM2_SUCCESS) return st;
        st = encode_2d(&L.mapB, elem, g.B, n, g.k, ldb, shape->BNS, shape->KC);
        if (st != TSM2_SUCCESS) return st;
        // The array keeps whatever the previous call left; the arrival
        // counters must start at zero.
        e = cudaMemsetAsync(scratch, 0, counter_bytes, stream);
        if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync(no-alloc counters)");
        L.grid = (int)grid;
        L.counters = static_cast<int *>(scratch);
        L.ws = static_cast<char *>(scratch) + kNoAllocCounterBytes;
        L.status = dev->status;
        L.wait_ns = g_wait_ns;
        L.c_vec = aligned16(g.C) && ((ldc * elem) % 16 == 0);
        t_last_config = shape->name;
        e = stream_launch(shape, L, stream);
        if (e != cudaSuccess) return cuda_error(e, "stream kernel launch");
    }
    return TSM2_SUCCESS;
}

// ---- TSM2X: choice between the TSM2R and TSM2L schedules --------------------
//
// TSM2R streams A in stages of 32 inner columns per row block of 256 (128)
// rows and splits the inner dimension between blocks; with few inner columns
// a row block is one or two stages long and the kernel is bound by latency
// and per-row-block overheads (the paper's observation for small inner
// dimensions, Sec. 3.2.1).  TSM2L owns whole, taller row blocks and keeps B
// on chip (or stages it, n > 64); it needs enough row blocks to occupy the
// GPU.  Largest n for which TSM2L was faster in a GB300 sweep over m in
// {15360, 2^18, 2^20, 2^22, 2^23}, n in {2, 4, ..., 1024}, k in {16, 32}:
//   binary32: m >= 2^17: n <= 256; shorter: n <= 64 (k <= 16), 128 (k > 16)
//   binary64: m >= 2^17: n <= 64 (k <= 16), 256 (k > 16); shorter: 32, 64.
int64_t tsm2x_l_max_n(int elem, int64_t m, int64_t k) {
    const bool tall = m >= (int64_t(1) << 17);
    const bool wide_c = k > 16;
    if (elem == 4) return tall ? 256 : (wide_c ? 128 : 64);
    return tall ? (wide_c ? 256 : 64) : (wide_c ? 64 : 32);
}

char tsm2x_schedule(int elem, int64_t m, int64_t n, int64_t k) {
    return n <= tsm2x_l_max_n(elem, m, k) ? 'l' : 'r';
}

// ---- host-resident operands: row-chunk pipeline ---------------------------
//
// A is streamed to the device in chunks of whole rows (a 2-D copy: mc rows of
// each of the n columns) into one of two staging slots.  Three streams run
// the stages: the copy-in stream fills slot (c & 1) with chunk c, the compute
// stream runs the device product on it, the copy-out stream returns its C
// rows.  Copy-in of chunk c+1 overlaps the product and copy-out of chunk c,
// and copy-in of chunk c+2 waits only for copy-out of chunk c (which itself
// followed the product), so the link stays busy in both directions.
//
// Page-locked buffers that the device can address are copied by SM kernels
// (tsm2_hostcopy.cu) on kCopyInSMs + up to kCopyOutSMs whole SMs, and the
// product kernels' grid is capped to the remaining SMs, so all three stages
// still run at once; other host memory goes through the copy engines.

constexpr int kCopyInSMs = 24;   // ~64 KB of loads in flight per SM covers the host link's latency
constexpr int kCopyOutSMs = 16;

// Device address of host memory at `p` when the current device can load and
// store it directly (page-locked and mapped), else nullptr.
void *device_view(const void *p) {
    if (g_host_copy != 0 || (reinterpret_cast<uintptr_t>(p) & 3)) return nullptr;  // copy kernels move 4-byte words
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // clear the error state the failed query left
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer || !a.hostPointer) return nullptr;
    return static_cast<char *>(a.devicePointer) + (static_cast<const char *>(p) - static_cast<const char *>(a.hostPointer));
}

// Resets the calling thread's grid cap on scope exit.
struct GridCap {
    explicit GridCap(int cap) { t_grid_cap = cap; }
    ~GridCap() { t_grid_cap = 0; }
};

struct HostPipe {
    cudaStream_t in = nullptr, comp = nullptr, out = nullptr;
    cudaEvent_t entry = nullptr, b_ready = nullptr, done = nullptr;
    cudaEvent_t a_ready[2] = {}, c_ready[2] = {}, slot_free[2] = {};
    void *dA[2] = {}, *dC[2] = {}, *dB = nullptr;
    size_t a_bytes = 0, c_bytes = 0, b_bytes = 0;
    std::mutex mu;
};
std::mutex g_pipe_mu;
std::map<int, HostPipe *> g_pipes;

#ifndef TSM2_HOST_CHUNK_MB
#define TSM2_HOST_CHUNK_MB 256
#endif
#ifndef TSM2_HOST_MIN_SEGMENT_KB
#define TSM2_HOST_MIN_SEGMENT_KB 64
#endif
constexpr size_t kHostChunkBytes = (size_t)TSM2_HOST_CHUNK_MB << 20;        // target bytes of A per chunk
constexpr size_t kHostMinSegment = (size_t)TSM2_HOST_MIN_SEGMENT_KB << 10;  // least bytes per column piece

void pipe_free_buffers(HostPipe *P) {
    for (int i = 0; i < 2; ++i) {
        if (P->dA[i]) cudaFree(P->dA[i]);
        if (P->dC[i]) cudaFree(P->dC[i]);
        P->dA[i] = P->dC[i] = nullptr;
    }
    if (P->dB) cudaFree(P->dB);
    P->dB = nullptr;
    P->a_bytes = P->c_bytes = P->b_bytes = 0;
}

void pipe_destroy(HostPipe *P) {
    pipe_free_buffers(P);
    for (cudaStream_t s : {P->in, P->comp, P->out})
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : {P->entry, P->b_ready, P->done, P->a_ready[0], P->a_ready[1], P->c_ready[0], P->c_ready[1],
                          P->slot_free[0], P->slot_free[1]})
        if (e) cudaEventDestroy(e);
    delete P;
}

tsm2_status pipe_for_device(HostPipe **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lk(g_pipe_mu);
    auto it = g_pipes.find(dev);
    if (it != g_pipes.end()) {
        *out = it->second;
        return TSM2_SUCCESS;
    }
    HostPipe *P = new HostPipe();
    for (cudaStream_t *s : {&P->in, &P->comp, &P->out})
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(s, cudaStreamNonBlocking);
    for (cudaEvent_t *ev : {&P->entry, &P->b_ready, &P->done, &P->a_ready[0], &P->a_ready[1], &P->c_ready[0],
                            &P->c_ready[1], &P->slot_free[0], &P->slot_free[1]})
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        pipe_destroy(P);
        return cuda_error(e, "host pipeline set-up");
    }
    g_pipes[dev] = P;
    *out = P;
    return TSM2_SUCCESS;
}

// Grows a device buffer; the pipeline's streams are idle when this runs (the
// caller synchronises them first).
tsm2_status grow(void **p, size_t *have, size_t want) {
    if (*have >= want && *p) return TSM2_SUCCESS;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *have = 0;
    cudaError_t e = cudaMalloc(p, want);
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_error(e, "cudaMalloc(host pipeline staging)");
    }
    *have = want;
    return TSM2_SUCCESS;
}

tsm2_status gemm_host(const char *fn, char op, int elem, int64_t m, int64_t n, int64_t k, const void *hA, int64_t lda,
                      const void *hB, int64_t ldb, void *hC, int64_t ldc, void *stream_v) {
    tsm2_status st = check_args(fn, m, n, k, hA, lda, hB, ldb, hC, ldc, elem);
    if (st != TSM2_SUCCESS) return st;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
    cudaError_t e;
    if (m == 0 || k == 0) {
        t_last_config = "empty";
        return TSM2_SUCCESS;
    }
    if (n == 0) {  // C = 0 on the host, after the caller's pending work
        e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize");
        for (int64_t c = 0; c < k; ++c) std::memset(static_cast<char *>(hC) + (size_t)(c * ldc) * elem, 0, (size_t)m * elem);
        t_last_config = "zero-fill";
        return TSM2_SUCCESS;
    }
    HostPipe *P = nullptr;
    st = pipe_for_device(&P);
    if (st != TSM2_SUCCESS) return st;
    std::lock_guard<std::mutex> lk(P->mu);

    // Rows per chunk: about kHostChunkBytes of A but column pieces of at
    // least kHostMinSegment bytes (a 2-D copy moves one piece per column),
    // a multiple of 256 rows (whole row blocks of every schedule); the
    // staging leading dimension is the chunk height rounded to 16 bytes.
    const int64_t vec = 16 / elem;
    int64_t mc = (int64_t)(kHostChunkBytes / ((size_t)n * elem));
    if (mc < (int64_t)(kHostMinSegment / elem)) mc = (int64_t)(kHostMinSegment / elem);
    mc = mc / 256 * 256;
    if (mc < 256) mc = 256;
    if (mc > m) mc = m;
    const int64_t ldd = (mc + vec - 1) / vec * vec;
    const int64_t ldbd = (n + vec - 1) / vec * vec;
    const size_t a_need = (size_t)ldd * n * elem, c_need = (size_t)ldd * k * elem, b_need = (size_t)ldbd * k * elem;
    if (P->a_bytes < a_need || P->c_bytes < c_need || P->b_bytes < b_need) {
        for (cudaStream_t s : {P->in, P->comp, P->out}) {
            e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize(host pipeline)");
        }
        size_t ah = P->a_bytes, ch = P->c_bytes;
        for (int i = 0; i < 2; ++i) {
            size_t a_have = ah, c_have = ch;
            if ((st = grow(&P->dA[i], &a_have, a_need)) != TSM2_SUCCESS) return st;
            if ((st = grow(&P->dC[i], &c_have, c_need)) != TSM2_SUCCESS) return st;
            if (i == 1) {
                P->a_bytes = a_have;
                P->c_bytes = c_have;
            }
        }
        if ((st = grow(&P->dB, &P->b_bytes, b_need)) != TSM2_SUCCESS) return st;
    }

    // SM copies where the device can address the host buffers (section
    // comment above); the product kernels get the SMs the copies leave.
    DeviceState *dev = nullptr;
    if ((st = device_state(&dev)) != TSM2_SUCCESS) return st;
    const void *vA = device_view(hA), *vB = device_view(hB);
    void *vC = device_view(hC);
    const int in_sms = vA ? kCopyInSMs : 0;
    int out_sms = 0;
    if (vC) {  // scaled to the bytes of C per byte of A, at least 2
        out_sms = (int)std::min<int64_t>(kCopyOutSMs, std::max<int64_t>(2, (kCopyOutSMs * k + n - 1) / n));
    }
    GridCap cap(in_sms + out_sms > 0 ? std::max(dev->sm_count - in_sms - out_sms, 1) : 0);
    static const char *const kCopyNames[8] = {"A:engine B:engine C:engine", "A:sm B:engine C:engine",
                                              "A:engine B:sm C:engine",     "A:sm B:sm C:engine",
                                              "A:engine B:engine C:sm",     "A:sm B:engine C:sm",
                                              "A:engine B:sm C:sm",         "A:sm B:sm C:sm"};
    t_last_host_copy = kCopyNames[(vA ? 1 : 0) | (vB ? 2 : 0) | (vC ? 4 : 0)];

    // Everything starts after the caller's pending work on `stream`.
    if ((e = cudaEventRecord(P->entry, stream)) != cudaSuccess) return cuda_error(e, "cudaEventRecord");
    for (cudaStream_t s : {P->in, P->comp, P->out})
        if ((e = cudaStreamWaitEvent(s, P->entry, 0)) != cudaSuccess) return cuda_error(e, "cudaStreamWaitEvent");
    if (vB) {
        e = sm_copy2d_launch(vB, ldb * elem, P->dB, ldbd * elem, n * elem, k, kCopyInSMs, P->in);
        if (e != cudaSuccess) return cuda_error(e, "host copy kernel (B)");
    } else {
        e = cudaMemcpy2DAsync(P->dB, (size_t)ldbd * elem, hB, (size_t)ldb * elem, (size_t)n * elem, (size_t)k,
                              cudaMemcpyHostToDevice, P->in);
        if (e != cudaSuccess) return cuda_error(e, "cudaMemcpy2DAsync(B)");
    }
    if ((e = cudaEventRecord(P->b_ready, P->in)) != cudaSuccess) return cuda_error(e, "cudaEventRecord");
    if ((e = cudaStreamWaitEvent(P->comp, P->b_ready, 0)) != cudaSuccess) return cuda_error(e, "cudaStreamWaitEvent");

    const char *config = "";
    int64_t chunk = 0;
    for (int64_t i0 = 0; i0 < m; i0 += mc, ++chunk) {
        const int slot = (int)(chunk & 1);
        const int64_t rows = (m - i0) < mc ? (m - i0) : mc;
        if (chunk >= 2 && (e = cudaStreamWaitEvent(P->in, P->slot_free[slot], 0)) != cudaSuccess)
            return cuda_error(e, "cudaStreamWaitEvent");
        if (vA) {
            e = sm_copy2d_launch(static_cast<const char *>(vA) + (size_t)i0 * elem, lda * elem, P->dA[slot],
                                 ldd * elem, rows * elem, n, in_sms, P->in);
            if (e != cudaSuccess) return cuda_error(e, "host copy kernel (A chunk)");
        } else {
            e = cudaMemcpy2DAsync(P->dA[slot], (size_t)ldd * elem, static_cast<const char *>(hA) + (size_t)i0 * elem,
                                  (size_t)lda * elem, (size_t)rows * elem, (size_t)n, cudaMemcpyHostToDevice, P->in);
            if (e != cudaSuccess) return cuda_error(e, "cudaMemcpy2DAsync(A chunk)");
        }
        if ((e = cudaEventRecord(P->a_ready[slot], P->in)) != cudaSuccess) return cuda_error(e, "cudaEventRecord");
        if ((e = cudaStreamWaitEvent(P->comp, P->a_ready[slot], 0)) != cudaSuccess)
            return cuda_error(e, "cudaStreamWaitEvent");
        st = gemm(fn, op, elem, rows, n, k, P->dA[slot], ldd, P->dB, ldbd, P->dC[slot], ldd, P->comp);
        if (st != TSM2_SUCCESS) return st;
        config = t_last_config;
        if ((e = cudaEventRecord(P->c_ready[slot], P->comp)) != cudaSuccess) return cuda_error(e, "cudaEventRecord");
        if ((e = cudaStreamWaitEvent(P->out, P->c_ready[slot], 0)) != cudaSuccess)
            return cuda_error(e, "cudaStreamWaitEvent");
        if (vC) {
            e = sm_copy2d_launch(P->dC[slot], ldd * elem, static_cast<char *>(vC) + (size_t)i0 * elem, ldc * elem,
                                 rows * elem, k, out_sms, P->out);
            if (e != cudaSuccess) return cuda_error(e, "host copy kernel (C chunk)");
        } else {
            e = cudaMemcpy2DAsync(static_cast<char *>(hC) + (size_t)i0 * elem, (size_t)ldc * elem, P->dC[slot],
                                  (size_t)ldd * elem, (size_t)rows * elem, (size_t)k, cudaMemcpyDeviceToHost, P->out);
            if (e != cudaSuccess) return cuda_error(e, "cudaMemcpy2DAsync(C chunk)");
        }
        if ((e = cudaEventRecord(P->slot_free[slot], P->out)) != cudaSuccess) return cuda_error(e, "cudaEventRecord");
    }
    // The caller's stream resumes once the last C rows are on the host.
    if ((e = cudaEventRecord(P->done, P->out)) != cudaSuccess) return cuda_error(e, "cudaEventRecord");
    if ((e = cudaStreamWaitEvent(stream, P->done, 0)) != cudaSuccess) return cuda_error(e, "cudaStreamWaitEvent");
    t_last_config = config;
    return TSM2_SUCCESS;
}

}  // namespace
}  // namespace tsm2

using namespace tsm2;

extern "C" {

tsm2_status tsm2r_d(int64_t m, int64_t n, int64_t k, const double *A, int64_t lda, const double *B, int64_t ldb,
                    double *C, int64_t ldc, void *stream) {
    return gemm("tsm2r_d", 'r', 8, m, n, k, A, lda, B, ldb, C, ldc, stream);
}

tsm2_status tsm2r_s(int64_t m, int64_t n, int64_t k, const float *A, int64_t lda, const float *B, int64_t ldb,
                    float *C, int64_t ldc, void *stream) {
    return gemm("tsm2r_s", 'r', 4, m, n, k, A, lda, B, ldb, C, ldc, stream);
}

tsm2_status tsm2l_d(int64_t m, int64_t n, int64_t k, const double *A, int64_t lda, const double *B, int64_t ldb,
                    double *C, int64_t ldc, void *stream) {
    return gemm("tsm2l_d", 'l', 8, m, n, k, A, lda, B, ldb, C, ldc, stream);
}

tsm2_status tsm2l_s(int64_t m, int64_t n, int64_t k, const float *A, int64_t lda, const float *B, int64_t ldb,
                    float *C, int64_t ldc, void *stream) {
    return gemm("tsm2l_s", 'l', 4, m, n, k, A, lda, B, ldb, C, ldc, stream);
}

const char *tsm2_get_last_error_string(void) { return t_last_error.c_str(); }

const char *tsm2_last_config(void) { return t_last_config; }

const char *tsm2_last_host_copy(void) { return t_last_host_copy; }

tsm2_status tsm2_get_device_status(void *stream) {
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize");
    unsigned w = 0;
    e = cudaMemcpyFromSymbol(&w, g_status_word, sizeof w);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemcpyFromSymbol(status)");
    if (w == 0) return TSM2_SUCCESS;
    const unsigned zero = 0;
    e = cudaMemcpyToSymbol(g_status_word, &zero, sizeof zero);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemcpyToSymbol(status)");
    // An abandoned launch may leave arrival counters non-zero: clear them all
    // on this device (stream workspaces and batch plans).
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> lk(g_mu);
        for (auto &kv : g_ws)
            if (kv.first.first == dev && kv.second.ptr) cudaMemset(kv.second.ptr, 0, kv.second.counter_bytes);
    }
    reset_plan_counters(dev);
    cudaDeviceSynchronize();
    if (w & kStatusBounds)
        return set_error(TSM2_ERR_BOUNDS,
                         "debug build: a kernel computed an address outside its operand and skipped the access; the "
                         "output of that call is undefined");
    return set_error(TSM2_ERR_TIMEOUT, "a pipeline wait exceeded its bound; the output of that call is undefined");
}

int tsm2_debug_checks(void) { return kDebugChecks ? 1 : 0; }

void tsm2_shutdown(void) {
    int cur = 0;
    cudaGetDevice(&cur);
    {
        std::lock_guard<std::mutex> lk(g_pipe_mu);
        for (auto &kv : g_pipes) {
            cudaSetDevice(kv.first);
            for (cudaStream_t s : {kv.second->in, kv.second->comp, kv.second->out}) cudaStreamSynchronize(s);
            pipe_destroy(kv.second);
        }
        g_pipes.clear();
    }
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto &kv : g_ws) {
        if (!kv.second.ptr) continue;
        cudaSetDevice(kv.first.first);
        cudaFree(kv.second.ptr);
    }
    g_ws.clear();
    cudaSetDevice(cur);
}

tsm2_status tsm2x_s(int64_t m, int64_t n, int64_t k, const float *A, int64_t lda, const float *B, int64_t ldb, float *C,
                    int64_t ldc, void *stream) {
    return gemm("tsm2x_s", tsm2x_schedule(4, m, n, k), 4, m, n, k, A, lda, B, ldb, C, ldc, stream);
}

tsm2_status tsm2x_d(int64_t m, int64_t n, int64_t k, const double *A, int64_t lda, const double *B, int64_t ldb,
                    double *C, int64_t ldc, void *stream) {
    return gemm("tsm2x_d", tsm2x_schedule(8, m, n, k), 8, m, n, k, A, lda, B, ldb, C, ldc, stream);
}

char tsm2x_choice(int elem_bytes, int64_t m, int64_t n, int64_t k) {
    if ((elem_bytes != 4 && elem_bytes != 8) || m < 0 || n < 0 || k < 0) return 0;
    return tsm2x_schedule(elem_bytes, m, n, k);
}

tsm2_status tsm2r_s_host(int64_t m, int64_t n, int64_t k, const float *A, int64_t lda, const float *B, int64_t ldb,
                         float *C, int64_t ldc, void *stream) {
    return gemm_host("tsm2r_s_host", 'r', 4, m, n, k, A, lda, B, ldb, C, ldc, stream);
}

tsm2_status tsm2r_d_host(int64_t m, int64_t n, int64_t k, const double *A, int64_t lda, const double *B, int64_t ldb,
                         double *C, int64_t ldc, void *stream) {
    return gemm_host("tsm2r_d_host", 'r', 8, m, n, k, A, lda, B, ldb, C, ldc, stream);
}

tsm2_status tsm2l_s_host(int64_t m, int64_t n, int64_t k, const float *A, int64_t lda, const float *B, int64_t ldb,
                         float *C, int64_t ldc, void *stream) {
    return gemm_host("tsm2l_s_host", 'l', 4, m, n, k, A, lda, B, ldb, C, ldc, stream);
}

tsm2_status tsm2l_d_host(int64_t m, int64_t n, int64_t k, const double *A, int64_t lda, const double *B, int64_t ldb,
                         double *C, int64_t ldc, void *stream) {
    return gemm_host("tsm2l_d_host", 'l', 8, m, n, k, A, lda, B, ldb, C, ldc, stream);
}

tsm2_status tsm2r_t_d(int64_t m, int64_t n, int64_t k, const double *A, int64_t lda, const double *dC, int64_t lddc,
                      double *dB, int64_t lddb, void *stream) {
    return gemm_t("tsm2r_t_d", 8, m, n, k, A, lda, dC, lddc, dB, lddb, stream);
}

tsm2_status tsm2r_t_s(int64_t m, int64_t n, int64_t k, const float *A, int64_t lda, const float *dC, int64_t lddc,
                      float *dB, int64_t lddb, void *stream) {
    return gemm_t("tsm2r_t_s", 4, m, n, k, A, lda, dC, lddc, dB, lddb, stream);
}

tsm2_status tsm2_rankk_d(int64_t m, int64_t n, int64_t k, const double *dC, int64_t lddc, const double *B, int64_t ldb,
                         double *dA, int64_t ldda, void *stream) {
    return rankk("tsm2_rankk_d", 8, m, n, k, dC, lddc, B, ldb, dA, ldda, stream);
}

tsm2_status tsm2_rankk_s(int64_t m, int64_t n, int64_t k, const float *dC, int64_t lddc, const float *B, int64_t ldb,
                         float *dA, int64_t ldda, void *stream) {
    return rankk("tsm2_rankk_s", 4, m, n, k, dC, lddc, B, ldb, dA, ldda, stream);
}

tsm2_status tsm2r_bf16(int64_t m, int64_t n, int64_t k, const uint16_t *A_hi, const uint16_t *A_lo, int64_t lda,
                       const float *B, int64_t ldb, float *C, int64_t ldc, void *stream) {
    return gemm_bf16(m, n, k, A_hi, A_lo, lda, B, ldb, C, ldc, stream);
}

tsm2_status tsm2_split_bf16(int64_t rows, int64_t cols, const float *X, int64_t ldx, uint16_t *hi, uint16_t *lo,
                            int64_t ldh, void *stream) {
    if (rows < 0 || cols < 0) return set_error(TSM2_ERR_INVALID_VALUE, "tsm2_split_bf16: negative dimension");
    if (ldx < (rows > 1 ? rows : 1) || ldh < (rows > 1 ? rows : 1))
        return set_error(TSM2_ERR_INVALID_VALUE, "tsm2_split_bf16: leading dimension < max(1,rows)");
    if (rows == 0 || cols == 0) return TSM2_SUCCESS;
    if (!X || !hi) return set_error(TSM2_ERR_INVALID_VALUE, "tsm2_split_bf16: X or hi is NULL");
    DeviceState *dev = nullptr;
    tsm2_status st = device_state(&dev);
    if (st != TSM2_SUCCESS) return st;
    cudaError_t e = split_bf16_launch(rows, cols, X, ldx, hi, lo, ldh, dev->sm_count, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? TSM2_SUCCESS : cuda_error(e, "split kernel launch");
}

tsm2_status tsm2_batch_plan_create_s(int nprob, const tsm2_problem_s *probs, int flags, tsm2_batch_plan_t *out) {
    if (!out) return set_error(TSM2_ERR_INVALID_VALUE, "tsm2_batch_plan_create_s: out is NULL");
    *out = nullptr;
    if (nprob < 0 || (nprob > 0 && !probs))
        return set_error(TSM2_ERR_INVALID_VALUE, "tsm2_batch_plan_create_s: bad problem list");
    const int variant = (flags >> 8) & 0xFF;
    if (variant >= batch_menu_count())
        return set_error(TSM2_ERR_INVALID_VALUE, "tsm2_batch_plan_create_s: tile variant %d out of [0, %d)", variant,
                         batch_menu_count());
    DeviceState *dev = nullptr;
    tsm2_status st = device_state(&dev);
    if (st != TSM2_SUCCESS) return st;
    tsm2_batch_plan_s *P = new tsm2_batch_plan_s();
    cudaGetDevice(&P->dev);
    P->sm_count = dev->sm_count;
    P->single_grid = dev->sm_count;
    P->variant = variant;
    P->menu = batch_menu(variant);
    const bool merge_r = (flags & TSM2_BATCH_MERGE_R) != 0;
    const bool merge_l = (flags & TSM2_BATCH_MERGE_L) != 0;
    // Class of a column chunk: the narrowest slot of its schedule that holds
    // kk columns (the widest with the merge flag).
    auto slot_for = [&](char op, int kk) -> int {
        int best = -1;
        for (int t = 0; t < P->menu->nslots; ++t) {
            const BatchClass *c = P->menu->slots[t];
            if (c->op != op || c->KC < kk) continue;
            const bool merge = op == 'r' ? merge_r : merge_l;
            if (best < 0 || (merge ? c->KC > P->menu->slots[best]->KC : c->KC < P->menu->slots[best]->KC)) best = t;
        }
        return best;
    };
    std::map<int, int> index;  // slot -> class
    for (int i = 0; i < nprob; ++i) {
        const tsm2_problem_s &q = probs[i];
        const char op = q.op == 'l' ? 'l' : (q.op == 'r' ? 'r' : 0);
        if (!op) {
            destroy_plan(P);
            return set_error(TSM2_ERR_INVALID_VALUE, "batch problem %d: op must be 'r' or 'l'", i);
        }
        st = check_args("tsm2_batch_plan_create_s", q.m, q.n, q.k, q.A, q.lda, q.B, q.ldb, q.C, q.ldc, 4);
        if (st != TSM2_SUCCESS) {
            destroy_plan(P);
            return st;
        }
        if (q.m == 0 || q.k == 0) continue;
        if (q.n == 0) {
            P->zeros.push_back({q.C, q.ldc, q.m, q.k});
            continue;
        }
        if (op == 'l' && (q.n > 64 || q.k > 64)) {
            destroy_plan(P);
            return set_error(TSM2_ERR_UNSUPPORTED, "batch problem %d: TSM2L needs n, k <= 64", i);
        }
        if (!aligned16(q.A) || (q.lda * 4) % 16 != 0 || q.m >= (1ll << 31) - 4096 || q.n >= (1ll << 31) ||
            (op == 'r' && (!aligned16(q.B) || (q.ldb * 4) % 16 != 0))) {
            destroy_plan(P);
            return set_error(TSM2_ERR_UNSUPPORTED,
                             "batch problem %d: batched operands need 16-byte aligned bases and leading dimensions", i);
        }
        const int kcmax = op == 'l' ? 32 : 16;
        for (int64_t c0 = 0; c0 < q.k; c0 += kcmax) {
            const int kk = (int)std::min<int64_t>(kcmax, q.k - c0);
            const int slot = slot_for(op == 'l' ? 'w' : 'r', kk);
            if (slot < 0) {
                destroy_plan(P);
                return set_error(TSM2_ERR_UNSUPPORTED, "batch problem %d: no class for k chunk %d", i, kk);
            }
            const BatchClass *cls = P->menu->slots[slot];
            auto it = index.find(slot);
            if (it == index.end()) {
                it = index.emplace(slot, (int)P->classes.size()).first;
                P->classes.emplace_back();
                P->classes.back().cls = cls;
                P->classes.back().slot = slot;
            }
            auto &C = P->classes[it->second];
            ProbDesc d;
            std::memset(&d, 0, sizeof d);
            const float *Bc = q.B + c0 * q.ldb;
            st = encode_2d(&d.mapA, 4, q.A, q.m, q.n, q.lda, cls->BOXM, cls->BNS);
            if (st == TSM2_SUCCESS && op == 'r') st = encode_2d(&d.mapB, 4, Bc, q.n, kk, q.ldb, cls->BNS, cls->KC);
            if (st != TSM2_SUCCESS) {
                destroy_plan(P);
                return st;
            }
            const int64_t num_rb = (q.m + cls->BM - 1) / cls->BM;
            const int64_t upr = (q.n + cls->BNS - 1) / cls->BNS;
            d.m = q.m;
            d.n = q.n;
            d.ldb = q.ldb;
            d.ldc = q.ldc;
            d.B = Bc;
            d.C = q.C + c0 * q.ldc;
            d.k = kk;
            d.upr = (int32_t)upr;
            d.gran = op == 'l' ? (int32_t)upr : 1;
            d.c_vec = aligned16(d.C) && (q.ldc * 4) % 16 == 0;
            d.group_begin = C.ngroups;
            d.rb_begin = C.nrb;
            C.ngroups += op == 'l' ? num_rb : num_rb * upr;
            C.nrb += num_rb;
            C.bytes += 4.0 * ((double)q.m * q.n + (double)q.n * kk + (double)q.m * kk);
            C.host.push_back(d);
        }
    }
    // Classes in menu order: the single launch walks them in this order.
    std::sort(P->classes.begin(), P->classes.end(),
              [](const tsm2_batch_plan_s::Cls &a, const tsm2_batch_plan_s::Cls &b) { return a.slot < b.slot; });
    cudaError_t e = cudaSuccess;
    for (auto &C : P->classes) {
        P->total_bytes += C.bytes;
        C.counter_bytes = ((size_t)C.nrb * sizeof(int) + 255) / 256 * 256;
        // Partial-sum slots for grids of up to one block per SM (TSM2R
        // classes split row blocks; TSM2L classes never do).
        const size_t slots = C.cls->op == 'r' ? (size_t)(P->sm_count + C.nrb) * C.cls->KC * C.cls->BM * 4 : 0;
        if ((e = cudaMalloc(&C.d_ws, C.counter_bytes + slots + 256)) != cudaSuccess) break;
        if ((e = cudaMalloc(&C.d_probs, C.host.size() * sizeof(ProbDesc))) != cudaSuccess) break;
        if ((e = cudaMemcpy(C.d_probs, C.host.data(), C.host.size() * sizeof(ProbDesc), cudaMemcpyHostToDevice)) !=
            cudaSuccess)
            break;
        if ((e = cudaMemset(C.d_ws, 0, C.counter_bytes)) != cudaSuccess) break;
        if ((e = cudaStreamCreateWithFlags(&C.aux, cudaStreamNonBlocking)) != cudaSuccess) break;
        if ((e = cudaEventCreateWithFlags(&C.done, cudaEventDisableTiming)) != cudaSuccess) break;
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P->capture, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
        // Even shares for the first single launch.
        std::vector<BatchBalance> init(1);
        std::memset(init.data(), 0, sizeof(BatchBalance));
        for (int b = 0; b < kBalanceMaxBlocks; ++b) init[0].w[0][b] = init[0].w[1][b] = 1.0f;
        e = cudaMalloc(&P->d_bal, sizeof(BatchBalance));
        if (e == cudaSuccess) e = cudaMemcpy(P->d_bal, init.data(), sizeof(BatchBalance), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        destroy_plan(P);
        return cuda_error(e, "tsm2_batch_plan_create_s");
    }
    // Default SM shares of the concurrent mode: proportional to each class's
    // algorithmic bytes.
    const int nc = (int)P->classes.size();
    if (nc > 0) {
        int left = std::max(P->sm_count - nc, 0);
        double tot = 0;
        for (auto &C : P->classes) tot += C.bytes;
        for (auto &C : P->classes) {
            const int g = 1 + (int)((double)left * C.bytes / (tot > 0 ? tot : 1));
            C.grid = (int)std::min<int64_t>(g, C.ngroups);
        }
    }
    {
        std::lock_guard<std::mutex> lk(g_plans_mu);
        g_plans.push_back(P);
    }
    *out = P;
    return TSM2_SUCCESS;
}

tsm2_status tsm2_batch_plan_execute(tsm2_batch_plan_t plan, void *stream) {
    if (!plan) return set_error(TSM2_ERR_INVALID_VALUE, "tsm2_batch_plan_execute: NULL plan");
    return plan_execute(plan, static_cast<cudaStream_t>(stream), -1);
}

tsm2_status tsm2_batch_plan_execute_class(tsm2_batch_plan_t plan, int cls, void *stream) {
    if (!plan || cls < 0 || cls >= (int)plan->classes.size())
        return set_error(TSM2_ERR_INVALID_VALUE, "tsm2_batch_plan_execute_class: bad plan or class");
    return plan_execute(plan, static_cast<cudaStream_t>(stream), cls);
}

tsm2_status tsm2_batch_plan_graph_launch(tsm2_batch_plan_t plan, void *stream_v) {
    if (!plan) return set_error(TSM2_ERR_INVALID_VALUE, "tsm2_batch_plan_graph_launch: NULL plan");
    cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
    cudaError_t e;
    if (!plan->graph) {
        // Captured once on the plan's own stream (the legacy default stream
        // cannot be captured); the executable graph then runs on any stream.
        e = cudaStreamBeginCapture(plan->capture, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_error(e, "cudaStreamBeginCapture");
        tsm2_status st = plan_execute(plan, plan->capture, -1);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(plan->capture, &graph);
        if (st != TSM2_SUCCESS) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&plan->graph, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            plan->graph = nullptr;
            return cuda_error(e, "cudaGraphInstantiate");
        }
    }
    e = cudaGraphLaunch(plan->graph, stream);
    return e == cudaSuccess ? TSM2_SUCCESS : cuda_error(e, "cudaGraphLaunch");
}

int tsm2_batch_plan_num_classes(tsm2_batch_plan_t plan) { return plan ? (int)plan->classes.size() : 0; }

tsm2_status tsm2_batch_plan_class_info(tsm2_batch_plan_t plan, int cls, const char **name, double *bytes, int *grid,
                                       int *nprob) {
    if (!plan || cls < 0 || cls >= (int)plan->classes.size())
        return set_error(TSM2_ERR_INVALID_VALUE, "tsm2_batch_plan_class_info: bad plan or class");
    const auto &c = plan->classes[cls];
    if (name) *name = c.cls->name;
    if (bytes) *bytes = c.bytes;
    if (grid) *grid = c.grid;
    if (nprob) *nprob = (int)c.host.size();
    return TSM2_SUCCESS;
}

static void drop_graph(tsm2_batch_plan_t plan) {
    if (plan->graph) {
        cudaGraphExecDestroy(plan->graph);
        plan->graph = nullptr;
    }
}

tsm2_status tsm2_batch_plan_set_grids(tsm2_batch_plan_t plan, int ncls, const int *grids) {
    if (!plan || ncls != (int)plan->classes.size() || (ncls > 0 && !grids))
        return set_error(TSM2_ERR_INVALID_VALUE, "tsm2_batch_plan_set_grids: bad arguments");
    for (int i = 0; i < ncls; ++i) {
        if (grids[i] < 1 || grids[i] > plan->sm_count)
            return set_error(TSM2_ERR_INVALID_VALUE, "tsm2_batch_plan_set_grids: grid %d out of [1, %d]", grids[i],
                             plan->sm_count);
    }
    for (int i = 0; i < ncls; ++i)
        plan->classes[i].grid = (int)std::min<int64_t>(grids[i], plan->classes[i].ngroups);
    drop_graph(plan);
    return TSM2_SUCCESS;
}

tsm2_status tsm2_batch_plan_set_serial(tsm2_batch_plan_t plan, int serial) {
    if (!plan) return set_error(TSM2_ERR_INVALID_VALUE, "tsm2_batch_plan_set_serial: NULL plan");
    return tsm2_batch_plan_set_mode(plan, serial ? TSM2_BATCH_SERIAL : TSM2_BATCH_CONCURRENT);
}

tsm2_status tsm2_batch_plan_set_mode(tsm2_batch_plan_t plan, int mode) {
    if (!plan) return set_error(TSM2_ERR_INVALID_VALUE, "tsm2_batch_plan_set_mode: NULL plan");
    if (mode != TSM2_BATCH_CONCURRENT && mode != TSM2_BATCH_SERIAL && mode != TSM2_BATCH_SINGLE_LAUNCH)
        return set_error(TSM2_ERR_INVALID_VALUE, "tsm2_batch_plan_set_mode: unknown mode %d", mode);
    if (plan->mode != mode) drop_graph(plan);
    plan->mode = mode;
    return TSM2_SUCCESS;
}

tsm2_status tsm2_batch_plan_set_single_grid(tsm2_batch_plan_t plan, int grid) {
    if (!plan || grid < 1 || grid > plan->sm_count)
        return set_error(TSM2_ERR_INVALID_VALUE, "tsm2_batch_plan_set_single_grid: bad plan or grid");
    if (plan->single_grid != grid) drop_graph(plan);
    plan->single_grid = grid;
    return TSM2_SUCCESS;
}

int tsm2_batch_plan_num_launches(tsm2_batch_plan_t plan) {
    if (!plan || plan->classes.empty()) return 0;
    return plan->mode == TSM2_BATCH_SINGLE_LAUNCH ? 1 : (int)plan->classes.size();
}

int tsm2_batch_num_variants(void) { return batch_menu_count(); }

tsm2_status tsm2_batch_variant_info(int variant, const char **name, int *stages, int *rows_per_lane,
                                    int *inner_per_warp) {
    const BatchMenu *m = (variant >= 0) ? batch_menu(variant) : nullptr;
    if (!m) return set_error(TSM2_ERR_INVALID_VALUE, "tsm2_batch_variant_info: variant %d out of range", variant);
    if (name) *name = m->name;
    if (stages) *stages = m->stages;
    if (rows_per_lane) *rows_per_lane = m->rows_per_lane;
    if (inner_per_warp) *inner_per_warp = m->inner_per_warp;
    return TSM2_SUCCESS;
}

void tsm2_batch_plan_destroy(tsm2_batch_plan_t plan) { destroy_plan(plan); }

void tsm2_set_wait_budget_ns(int64_t ns) { g_wait_ns = ns < 0 ? -1 : ns; }

void tsm2_set_path(int path) { g_path = path; }

void tsm2_set_grid(int blocks) { g_grid_override = blocks < 0 ? 0 : blocks; }

void tsm2_set_host_copy(int mode) { g_host_copy = mode == 1 ? 1 : 0; }

void tsm2_set_balance(int mode) { g_balance = (mode == 1 || mode == 2) ? mode : 0; }

void tsm2_set_trace(unsigned long long *device_words, int64_t blocks) {
    g_trace = device_words;
    g_trace_blocks = device_words ? blocks : 0;
}

tsm2_status tsm2r_s_noalloc(int64_t m, int64_t n, int64_t k, const float *A, int64_t lda, const float *B,
                            int64_t ldb, float *C, int64_t ldc, void *stream) {
    return gemm_r32_noalloc(m, n, k, A, lda, B, ldb, C, ldc, stream);
}

}  // extern "C"
