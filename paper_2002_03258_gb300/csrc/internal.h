// Host-side declarations shared between the C ABI (tsm2_api.cu) and the
// translation units that hold the kernels.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace tsm2 {

// One launch of a multiply kernel on a column chunk of at most KC columns of
// C.  All pointers are device pointers; `k` is the number of live columns.
struct GemmArgs {
    int64_t m, n;
    int k;
    const void *A;
    int64_t lda;
    const void *B;
    int64_t ldb;
    void *C;
    int64_t ldc;
};

// Everything a stream (TMA) kernel launch needs besides the operands.
struct StreamLaunch {
    GemmArgs g;
    CUtensorMap mapA;   // A: dims {m, n}, box {BOXM, BNS}
    CUtensorMap mapB;   // B: dims {n, k}, box {BNS, KC} (unused when B is resident)
    void *ws;           // partial-sum slots, 256-byte aligned
    int *counters;      // one arrival counter per row block, zero between launches
    int *claims;        // resident-B schedules: row-block claim counters, zero between launches (nullptr: static)
    unsigned *status;   // device status word
    int64_t wait_ns;    // bound of every pipeline wait
    int grid;           // thread blocks of the persistent grid
    bool c_vec;         // C base and ldc allow 16-byte stores
    unsigned long long *trace;  // optional per-block timestamps (nullptr: off)
};

// Static description of a compiled stream-kernel configuration.
struct StreamShape {
    const char *name;
    int elem;        // bytes per element
    int KC;          // C columns per pass
    int BM;          // rows per row block
    int BNS;         // inner-dimension columns per pipeline stage
    int BOXM;        // rows per TMA box
    int gran_rows;   // 1: split inner dim at stage granularity; 0: whole row blocks
    bool b_resident; // B loaded once into shared memory (requires n <= n_max_resident)
    int n_max_resident;
    int smem_bytes;
    int threads;
};

// Kernel selectors: op 'r' (TSM2R schedule) or 'l' (TSM2L schedule).
// Returns nullptr if no compiled configuration covers (elem, op, kc).
const StreamShape *stream_shape(int elem, char op, int kc);
cudaError_t stream_launch(const StreamShape *shape, const StreamLaunch &L, cudaStream_t stream);

// Copies `cols` columns of `row_bytes` bytes (column c at src + c*lds_bytes,
// dst + c*ldd_bytes) with the SMs' loads and stores; either side may be a
// device-mapped address of page-locked host memory.  `grid` blocks, each
// holding a whole SM.  Requires 4-byte aligned starts and strides and
// row_bytes % 4 == 0 (cudaErrorInvalidValue otherwise).
cudaError_t sm_copy2d_launch(const void *src, int64_t lds_bytes, void *dst, int64_t ldd_bytes, int64_t row_bytes,
                             int64_t cols, int grid, cudaStream_t stream);

// Element-wise fallback (any alignment), Algorithm 3 style.
cudaError_t simple_launch(int elem, const GemmArgs &g, unsigned *status, cudaStream_t stream);
int simple_kc_max();

// ---- backward products ----------------------------------------------------

// dB = A^T dC with the bulk-copy pipeline (tsm2_backward.cu).
struct TLaunch {
    int64_t m, n;
    int k;           // live columns of dC / dB in this chunk (<= KC)
    CUtensorMap mapA;  // A: dims {m, n}, box {BOXM, BNS}
    CUtensorMap mapD;  // dC: dims {m, k}, box {BOXM, KC}
    void *dB;
    int64_t lddb;
    void *ws;
    int *counters;
    unsigned *status;
    int64_t wait_ns;
    int grid;
};
struct TShape {
    const char *name;
    int elem, KC, BM, BNS, BOXM;
};
const TShape *tsm2t_shape(int elem, int kc);
cudaError_t tsm2t_launch(const TShape *shape, const TLaunch &L, cudaStream_t stream);
cudaError_t simple_t_launch(int elem, int64_t m, int64_t n, int k, const void *A, int64_t lda, const void *dC,
                            int64_t lddc, void *dB, int64_t lddb, cudaStream_t stream);
cudaError_t rankk_launch(int elem, int64_t m, int64_t n, int k, const void *dC, int64_t lddc, const void *B,
                         int64_t ldb, void *dA, int64_t ldda, bool vec_ok, bool accumulate, int sm_count,
                         cudaStream_t stream);

// ---- bfloat16 A on the tensor cores (tsm2_bf16.cu) --------------------------

struct BF16Launch {
    int64_t m, n;
    int k;               // <= 16
    CUtensorMap mapHi;   // A_hi: bf16 dims {m, n}, box {64, bf16_bk(hilo)}, 128-byte swizzle
    CUtensorMap mapLo;   // A_lo (when hilo)
    bool hilo;
    const void *bpieces; // prepared B pieces (bf16_prep_b)
    void *C;
    int64_t ldc;
    void *ws;
    int *counters;
    unsigned *status;
    int64_t wait_ns;
    int grid;
};
int bf16_bm();
int bf16_bk(bool hilo);  // inner columns per pipeline stage
size_t bf16_bpieces_bytes(int64_t n, bool hilo);
cudaError_t bf16_prep_b(int64_t n, int k, const float *B, int64_t ldb, void *out, bool hilo, cudaStream_t stream);
cudaError_t bf16_launch(const BF16Launch &L, cudaStream_t stream);
cudaError_t bf16_simple_launch(int64_t m, int64_t n, int k, const void *A_hi, const void *A_lo, int64_t lda,
                               const float *B, int64_t ldb, float *C, int64_t ldc, cudaStream_t stream);
cudaError_t split_bf16_launch(int64_t rows, int64_t cols, const float *X, int64_t ldx, void *hi, void *lo,
                              int64_t ldh, int sm_count, cudaStream_t stream);

// ---- batched problems (tsm2_batched.cu) --------------------------------------

// Device-side descriptor of one problem of a batch class.
struct ProbDesc {  // aligned as its tensor maps
    CUtensorMap mapA;      // A: dims {m, n}, box {BOXM, BNS}
    CUtensorMap mapB;      // TSM2R classes: B dims {n, k}, box {BNS, KC} (column-major)
    int64_t m, n, ldb, ldc;
    const void *B;         // TSM2L classes read B with ordinary loads
    void *C;
    int64_t group_begin;   // first work group of the problem in the class numbering
    int64_t rb_begin;      // first row block (counters and partial-sum slots)
    int32_t k, upr, gran, c_vec;
};

// Classes per batch kernel (tsm2_batch_kernel.cuh) and its launch arguments.
constexpr int kMaxBatchMenu = 8;

// Per-class arguments of one batch-kernel launch.
struct ClassParams {
    const ProbDesc *probs;
    int nprob;
    int whole;        // TSM2L class: groups are whole row blocks (no partial sums)
    int64_t ngroups;  // 0: the class has no work in this launch
    float *ws;        // partial-sum slots: (grid + row blocks) x KC x BM
    int *counters;    // one arrival counter per row block, zero between launches
    int64_t nrb;      // row blocks of the class (counters; slots beyond the grid)
};

// Shares of the TSM2L classes in the single launch of a batch plan, adapted
// from launch to launch (plan-owned device memory).  Block b takes the
// fraction w[b] / sum(w) of every TSM2L class's row blocks; each launch
// records when every block reached its TSM2L work, when it finished and how
// many stages it consumed, and the last block to finish sets the weights of
// the next launch so that all blocks would have finished together.  Whole row
// blocks are computed the same way whoever owns them, so the results do not
// depend on the weights.
constexpr int kBalanceMaxBlocks = 1024;
struct BatchBalance {
    int epoch;  // launches completed: weights are read from w[epoch & 1]
    int done;   // blocks finished in the running launch (zero between launches)
    int bad;    // a block gave up in the running launch: keep the weights
    int pad;
    float w[2][kBalanceMaxBlocks];
    unsigned long long t_lstart[kBalanceMaxBlocks];  // first TSM2L class reached (ns)
    unsigned long long t_end[kBalanceMaxBlocks];     // consumers done (ns)
    long long units[kBalanceMaxBlocks];              // TSM2L stages consumed
};

struct BatchKParams {
    ClassParams cls[kMaxBatchMenu];  // slot i of the kernel's menu
    unsigned *status;
    int64_t wait_ns;
    unsigned long long *trace;  // optional: 4 words per block (start, 0, end, 0); nullptr: off
    BatchBalance *bal;          // adaptive TSM2L shares (single launch); nullptr: equal shares
};

struct BatchClass {
    char op;  // 'r' TSM2R schedule, 'w' TSM2L schedule (whole row blocks, B resident)
    const char *name;
    int KC, BM, BNS, BOXM;
    int stages, rows_per_lane;
};

// A tile variant: the classes one batch kernel holds (its "menu") and the
// launch of that kernel.  Every class of a plan is a slot of its menu; a
// launch runs any subset of the slots (empty slots have no work).
struct BatchMenu {
    const char *name;   // tile variant, e.g. "v0 stages5 rows8 inner4"
    int stages, rows_per_lane, inner_per_warp;
    int nslots;
    const BatchClass *slots[kMaxBatchMenu];
    cudaError_t (*launch)(const BatchKParams &, int grid, cudaStream_t);
};
int batch_menu_count();
const BatchMenu *batch_menu(int variant);

// Work partition of the persistent grid (shared by host sizing and kernels).
struct Partition {
    int64_t num_rb;  // row blocks
    int64_t upr;     // stages (units) per row block
    int64_t gran;    // units per indivisible group
    int64_t ngroups; // total groups
};

}  // namespace tsm2
