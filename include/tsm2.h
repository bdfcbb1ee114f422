/*
 * tsm2.h -- C ABI of the GB300 tall-and-skinny matrix-multiply library.
 *
 * Operation (Sec. 2.1 of Rivera et al., "TSM2X: High-Performance
 * Tall-and-Skinny Matrix-Matrix Multiplication on GPUs"):
 *
 *     C(m x k) = A(m x n) * B(n x k),  C(i,c) = sum_j A(i,j) B(j,c)
 *
 * Naming: A is m x n, B is n x k, C is m x k, so n is the inner (reduced)
 * dimension and k the skinny one.  (The paper calls the inner dimension k
 * and the skinny one n.)
 *
 *  - TSM2R (Sec. 3.1, Algorithms 2-4): a large, roughly square A times a
 *    tall-and-skinny B, m ~ n >> k.
 *  - TSM2L (Sec. 3.2, Algorithm 5): a tall-and-skinny A times a small
 *    square B, m >> n ~ k.
 *
 * Both entry points compute the same function; they differ in the kernel
 * schedule they select, and TSM2L limits n and k.
 *
 * Common conventions for every matrix entry point below:
 *  - Layout: column-major.  Element (i, j) of X is X[i + j * ldx].
 *  - Pointers: DEVICE pointers to caller-owned memory on the current CUDA
 *    device.  The library never frees or retains them.
 *  - stream: a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Calls are asynchronous with respect to the host; results are ready once
 *    the stream reaches the point of the call.
 *  - Semantics: C is overwritten (beta = 0); its previous contents are never
 *    read.  Rows m .. ldc-1 of C are never written.  C must not overlap A or
 *    B (checked on address ranges: TSM2_ERR_INVALID_VALUE).
 *  - Quick returns: m == 0 or k == 0 does nothing and returns SUCCESS;
 *    n == 0 sets C to zero (the empty sum).
 *  - Errors (checked before anything is launched; nothing is launched on
 *    error):
 *      TSM2_ERR_INVALID_VALUE  m, n or k negative; lda < max(1,m);
 *                              ldb < max(1,n); ldc < max(1,m); a NULL
 *                              pointer for a non-empty operand; overlap.
 *      TSM2_ERR_UNSUPPORTED    see each entry point.
 *      TSM2_ERR_CUDA           a CUDA runtime error at launch time; the
 *                              message is in tsm2_get_last_error_string().
 *    Faults during execution surface at the caller's next synchronisation,
 *    as for any CUDA kernel.  A pipeline wait that exceeds its time bound
 *    sets a device status word instead of hanging; tsm2_get_device_status()
 *    reports it as TSM2_ERR_TIMEOUT (and, in the debug build, a skipped
 *    out-of-bounds access as TSM2_ERR_BOUNDS; see tsm2_debug_checks).
 *  - Alignment: any alignment is accepted.  16-byte aligned base pointers
 *    with leading dimensions whose byte size is a multiple of 16 select the
 *    bulk-copy (TMA) path; anything else selects a slower path that loads
 *    element by element.  Both give results within the same error bound.
 *  - Accuracy: every C(i,c) is a sum of the n products computed with fused
 *    multiply-adds in the input precision; |C - AB| <= gamma_n |A||B|
 *    componentwise, gamma_n = n u / (1 - n u).  The summation order is fixed
 *    for a given (shape, device), so repeated calls are bitwise identical.
 *  - Scratch: kernels that split the inner dimension over several thread
 *    blocks combine partial sums through a per-(device, stream) workspace
 *    that the library allocates lazily with cudaMalloc on first use and
 *    grows when needed; tsm2_shutdown() frees it.  Two calls in flight at
 *    once on the SAME stream are ordered by the stream and never race.
 *    Growing synchronises the stream and calls cudaMalloc, which cannot
 *    happen while the stream is captured into a CUDA graph: a call that
 *    would grow the workspace during capture returns TSM2_ERR_UNSUPPORTED
 *    (the capture itself stays valid).  Call the largest shape once on the
 *    stream before capturing.  TSM2L with B on chip (n <= 64) hands out
 *    its row blocks at run time through two counters of the same workspace
 *    (allocated on the first such call on a stream); while a stream without
 *    a workspace is captured it uses the static partition instead.  Either
 *    way every row block is computed whole by one thread block in the same
 *    order, so the result is the same bits.
 */
#ifndef TSM2_H
#define TSM2_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum tsm2_status {
    TSM2_SUCCESS = 0,
    TSM2_ERR_INVALID_VALUE = 1,
    TSM2_ERR_UNSUPPORTED = 2,
    TSM2_ERR_CUDA = 3,
    TSM2_ERR_TIMEOUT = 4,
    TSM2_ERR_BOUNDS = 5  /* debug builds only: an access outside its operand was skipped */
} tsm2_status;

/* TSM2R, binary64.  A is streamed from device memory once per group of up
 * to 16 columns of C (Sec. 3.1.2, outer-product form of Algorithm 2; the
 * t2 loop of Algorithm 4 re-reads A ceil(k/16) times).  Any k >= 0. */
tsm2_status tsm2r_d(int64_t m, int64_t n, int64_t k,
                    const double *A, int64_t lda,
                    const double *B, int64_t ldb,
                    double *C, int64_t ldc, void *stream);

/* TSM2R, binary32.  Same contract as tsm2r_d. */
tsm2_status tsm2r_s(int64_t m, int64_t n, int64_t k,
                    const float *A, int64_t lda,
                    const float *B, int64_t ldb,
                    float *C, int64_t ldc, void *stream);

/* TSM2L, binary64 (Sec. 3.2, Algorithm 5: a persistent grid of thread
 * blocks strides over row blocks of the tall-and-skinny A).  Any n, k >= 0.
 * For n <= 64 B is held on chip for the whole call; for n > 64 B is staged
 * through shared memory beside each stage of A (the staged-B setting of
 * Algorithm 6, Sec. 3.2.2).  C is produced in groups of up to 32 columns, A
 * read once per group (ceil(k/32) times).  Same pointer, stream, alignment,
 * accuracy and error contract as tsm2r_d; TSM2_ERR_UNSUPPORTED is not
 * returned for any n or k. */
tsm2_status tsm2l_d(int64_t m, int64_t n, int64_t k,
                    const double *A, int64_t lda,
                    const double *B, int64_t ldb,
                    double *C, int64_t ldc, void *stream);

/* TSM2L, binary32.  Same contract as tsm2l_d. */
tsm2_status tsm2l_s(int64_t m, int64_t n, int64_t k,
                    const float *A, int64_t lda,
                    const float *B, int64_t ldb,
                    float *C, int64_t ldc, void *stream);

/* ---- Backward products of C = A B (gradients for a differentiable TSM2R) -- */

/* dB(n x k) = A^T dC, A m x n (lda >= max(1,m)), dC m x k (lddc >= max(1,m)),
 * dB n x k (lddb >= max(1,n)); dB is overwritten.  The reduction runs along
 * the m rows of A, each of which is read once per group of up to 16 columns
 * of dC (the outer-product principle of Algorithm 2, Sec. 3.1.2, applied to
 * the transposed product).  m == 0 sets dB to zero.  Same pointer, stream,
 * alignment, accuracy (gamma_m |A^T||dC|), scratch and error contract as
 * tsm2r_d. */
tsm2_status tsm2r_t_d(int64_t m, int64_t n, int64_t k, const double *A, int64_t lda,
                      const double *dC, int64_t lddc, double *dB, int64_t lddb, void *stream);
tsm2_status tsm2r_t_s(int64_t m, int64_t n, int64_t k, const float *A, int64_t lda,
                      const float *dC, int64_t lddc, float *dB, int64_t lddb, void *stream);

/* dA(m x n) = dC B^T, dC m x k (lddc >= max(1,m)), B n x k (ldb >= max(1,n)),
 * dA m x n (ldda >= max(1,m)); dA is overwritten (k == 0 sets it to zero).
 * A rank-k update: dA is written once, as a stream.  For k > 16 the columns of
 * dC and B are processed in groups of 16 and later groups add into dA. */
tsm2_status tsm2_rankk_d(int64_t m, int64_t n, int64_t k, const double *dC, int64_t lddc,
                         const double *B, int64_t ldb, double *dA, int64_t ldda, void *stream);
tsm2_status tsm2_rankk_s(int64_t m, int64_t n, int64_t k, const float *dC, int64_t lddc,
                         const float *B, int64_t ldb, float *dA, int64_t ldda, void *stream);

/* ---- bfloat16 storage of A (tensor cores) ---------------------------------- */

/* TSM2R with A stored in bfloat16: C(m x k, binary32) = A B, B n x k binary32,
 * binary32 accumulation.  A_hi holds bfloat16 bit patterns (column-major, lda),
 * A_lo (same layout and lda) the optional low parts of a hi + lo split (see
 * tsm2_split_bf16); NULL means A = A_hi.  The paper omits half precision
 * (Sec. 4.1); this extends TSM2R (Sec. 3.1): A is streamed once, at half the
 * bytes of binary32 (or the same bytes, with about 16 significant bits, for
 * hi + lo), and the products run on the tensor cores (B is split internally
 * into bfloat16 pieces b1 + b2 + b3 = b exactly; plain A uses b1 + b2, B to
 * 17 bits, hi + lo all three).  Error, componentwise against the product of
 * the bfloat16-represented A (A_eff = A_hi or A_hi + A_lo), with S = |A_eff||B|,
 * G inner indices summed on the tensor cores per drain (256 plain, 32 hi + lo)
 * in s = 16 (plain) or 4 (hi + lo) MMA steps, and P the stream-K partial sums
 * that cover one row block (at most ceil((U - 1) / u) + 1 for U pipeline stages
 * per row block and u >= 4 stages per thread block at the default grid; 4 at
 * 32768 x 32768):
 *   |C - A_eff B| <= 1.04 (e_B + 18 s 2^-23 + gamma_{NP-1} + gamma_{n/G + P}) S,
 * e_B = 2^-17 (plain) or 0 (hi + lo), NP = 2 or 3 pieces, gamma_j = j 2^-24 /
 * (1 - j 2^-24); the tensor-core term assumes the aligned, truncating sums
 * measured on earlier NVIDIA tensor cores.  About 5e-5 S (plain) and 7e-5 S
 * (hi + lo) at n = 32768.  The element-wise path: gamma_n S.  The bulk-copy
 * path needs 16-byte aligned A_hi/A_lo and lda a multiple of 8; otherwise an element-wise
 * CUDA-core path runs.  Uses the workspace (B pieces and split partial sums).
 * Same error contract as tsm2r_s. */
tsm2_status tsm2r_bf16(int64_t m, int64_t n, int64_t k, const uint16_t *A_hi, const uint16_t *A_lo,
                       int64_t lda, const float *B, int64_t ldb, float *C, int64_t ldc, void *stream);

/* hi = RNE_bf16(X), lo = RNE_bf16(X - hi) elementwise (X - hi is exact in
 * binary32), rows x cols column-major; lo may be NULL.  hi and lo share ldh. */
tsm2_status tsm2_split_bf16(int64_t rows, int64_t cols, const float *X, int64_t ldx,
                            uint16_t *hi, uint16_t *lo, int64_t ldh, void *stream);

/* TSM2X: the same product, C = A B (tsm2r_* semantics, any n and k), with
 * the schedule chosen from the shape: TSM2L (whole row blocks, B on chip or
 * staged) for small inner dimensions on tall A, TSM2R (inner dimension split
 * between blocks) otherwise.  The paper selects between its two kernels by
 * the shape regime (Sec. 2.1, Sec. 3.2.1: TSM2R is latency-bound when the
 * inner dimension is small); the thresholds here were measured on GB300:
 * TSM2L when n <= tsm2x_choice's bound, i.e.
 *   binary32: m >= 2^17: n <= 256; shorter A: n <= 64 (k <= 16), 128 (k > 16)
 *   binary64: m >= 2^17: n <= 64 (k <= 16), 256 (k > 16); shorter: 32, 64. */
tsm2_status tsm2x_s(int64_t m, int64_t n, int64_t k, const float *A, int64_t lda, const float *B, int64_t ldb,
                    float *C, int64_t ldc, void *stream);
tsm2_status tsm2x_d(int64_t m, int64_t n, int64_t k, const double *A, int64_t lda, const double *B, int64_t ldb,
                    double *C, int64_t ldc, void *stream);
/* The schedule tsm2x_s (elem_bytes 4) / tsm2x_d (8) runs for a shape: 'r' or
 * 'l'; 0 for invalid arguments.  Host-only, no device call. */
char tsm2x_choice(int elem_bytes, int64_t m, int64_t n, int64_t k);

/* Host-resident operands: the same products with A, B and C in host memory
 * (page-locked memory gives full copy/compute overlap; pageable memory works
 * at lower speed).  The paper keeps its operands in device memory; these are
 * a library convenience with no counterpart there.
 *  - Work: B is copied once; A streams to the device in chunks of whole rows
 *    (about 256 MiB, at least 64 KiB per column piece, multiples of 256 rows)
 *    through two device staging slots; each chunk's C rows are copied back
 *    as soon as its product is done.  Copy-in of the next chunk overlaps the
 *    product and copy-out of the current one.
 *  - Copies: a buffer in page-locked memory that the device can address
 *    (cudaHostAlloc / cudaMallocHost, or cudaHostRegister'ed and mapped) is
 *    read or written by copy kernels on the SMs (24 SMs in, 2-16 out; the
 *    product kernels then use the remaining SMs); any other buffer is copied
 *    by the copy engines (cudaMemcpy2DAsync).  See tsm2_set_host_copy.
 *  - Ordering: the work starts after everything already queued on `stream`,
 *    and `stream` waits for the last C rows to reach the host: synchronise
 *    `stream` before reading C.  The host buffers must stay valid until then.
 *  - Memory: the staging slots are device memory the library allocates on
 *    first use and grows as needed (held until tsm2_shutdown).  Calls on one
 *    device are serialised on one set of staging slots.
 *  - Errors: the argument rules of the device entry points (pointers are
 *    host pointers here); n == 0 waits for `stream` and zeroes C on the host. */
tsm2_status tsm2r_s_host(int64_t m, int64_t n, int64_t k, const float *A, int64_t lda, const float *B, int64_t ldb,
                         float *C, int64_t ldc, void *stream);
tsm2_status tsm2r_d_host(int64_t m, int64_t n, int64_t k, const double *A, int64_t lda, const double *B,
                         int64_t ldb, double *C, int64_t ldc, void *stream);
tsm2_status tsm2l_s_host(int64_t m, int64_t n, int64_t k, const float *A, int64_t lda, const float *B, int64_t ldb,
                         float *C, int64_t ldc, void *stream);
tsm2_status tsm2l_d_host(int64_t m, int64_t n, int64_t k, const double *A, int64_t lda, const double *B,
                         int64_t ldb, double *C, int64_t ldc, void *stream);

/* TSM2R, binary32, allocating nothing.  The paper has no counterpart: this
 * is a library convenience.  Same arguments, result and error contract as
 * tsm2r_s, for callers that cannot call cudaMalloc at all -- a process whose
 * device memory is wholly owned by another allocator (a framework's caching
 * pool that has reserved the free memory), or a latency-bound loop that
 * cannot pay for cudaMalloc and its implicit synchronisation.
 *  - Scratch: partial sums of row blocks split between thread blocks and
 *    their arrival counters live in a fixed 16 MiB array in device memory.
 *    The array belongs to the library's device code: it is reserved, with the
 *    library's status word, when that code is first loaded on a device, which
 *    is the first call of any tsm2 entry point there (CUDA loads modules
 *    lazily), and it stays reserved until the process exits.  No call of this
 *    function allocates or frees device memory after that.  A caller whose
 *    allocator reserves all free device memory should make one tsm2 call on
 *    each device first, or that first call can fail for lack of memory.
 *  - Limit: those must fit the array: m up to about 222,000 rows when a
 *    column chunk is 13..16 wide (KC = 16; the partial-sum slots grow with m,
 *    not with n), more for narrower chunks (the sizes are in the error
 *    message).  Larger problems return TSM2_ERR_UNSUPPORTED before anything
 *    is launched.
 *  - Set-up: the first call on each device looks up the array's device
 *    address (cudaGetSymbolAddress) with that device current; make that first
 *    call before any stream capture.
 *  - Sharing: every call on a device uses the same array and it keeps the
 *    previous call's contents; each call clears the counters it needs on its
 *    stream.  Calls that overlap on the GPU (different streams, or other
 *    host threads) race on the array and give undefined results; order them
 *    on one stream or synchronise between them. */
tsm2_status tsm2r_s_noalloc(int64_t m, int64_t n, int64_t k,
                            const float *A, int64_t lda,
                            const float *B, int64_t ldb,
                            float *C, int64_t ldc, void *stream);

/* ---- Batches of uneven problems (binary32) ----------------------------------
 *
 * Many TSM2R / TSM2L problems of different shapes executed as one unit.  The
 * problems are grouped into tile classes (schedule and C-column width KC:
 * TSM2R with 8, 12 or 16 columns, TSM2L with 8, 16, 24 or 32; each column chunk
 * goes to the narrowest class that holds it).  In every class the work units
 * of all its problems are numbered end to end and every block of a persistent
 * grid takes a contiguous share (equal; weighted for the TSM2L classes of
 * large plans, below), crossing problem boundaries
 * (Algorithm 5's persistent walk over tiles, Sec. 3.2.2, extended across
 * problems).  The tile parameters that the paper tunes offline (Sec. 3.1.9,
 * 3.2.2) come in compiled variants (pipeline stages, rows of C per lane,
 * inner columns per warp and stage), chosen per plan.  Execution modes:
 *  - TSM2_BATCH_SINGLE_LAUNCH (default): ONE persistent kernel whose blocks
 *    walk their share of every class in turn, through one pipeline.  In
 *    plans of 16 GB or more (algorithmic bytes) the shares of the TSM2L
 *    classes adapt from launch to launch: each launch
 *    records every block's TSM2L rate and start, and the last block to
 *    finish sets the next launch's shares so that all blocks would finish
 *    together (TSM2L row blocks are computed whole, so the bits do not
 *    change; tsm2_set_balance(1) keeps equal shares);
 *  - TSM2_BATCH_SERIAL: one launch per class, each on all SMs;
 *  - TSM2_BATCH_CONCURRENT: one launch per class, concurrently on SM shares
 *    (tsm2_batch_plan_set_grids; by default proportional to their bytes).
 * A whole batch can be replayed as one CUDA graph launch.  Results do not
 * depend on the mode, the variant's timing or the grid: every sum runs in a
 * fixed order. */

typedef struct tsm2_problem_s {
    char op;             /* 'r' (TSM2R schedule) or 'l' (TSM2L: n, k <= 64) */
    int64_t m, n, k;
    const float *A;      /* m x n, column-major, lda; device */
    int64_t lda;
    const float *B;      /* n x k, ldb */
    int64_t ldb;
    float *C;            /* m x k, ldc; overwritten */
    int64_t ldc;
} tsm2_problem_s;

typedef struct tsm2_batch_plan_s *tsm2_batch_plan_t;

/* Plan flags. */
#define TSM2_BATCH_WIDE_L 1   /* accepted and ignored (rows per lane come from the tile variant) */
#define TSM2_BATCH_MERGE_R 2  /* TSM2R column chunks all in the widest TSM2R class (16 columns) */
#define TSM2_BATCH_MERGE_L 4  /* TSM2L column chunks all in the widest TSM2L class (32 columns) */
#define TSM2_BATCH_VARIANT(v) ((v) << 8)  /* tile variant v in [0, tsm2_batch_num_variants()) */

/* Execution modes (tsm2_batch_plan_set_mode). */
#define TSM2_BATCH_CONCURRENT 0
#define TSM2_BATCH_SERIAL 1
#define TSM2_BATCH_SINGLE_LAUNCH 2

/* Validates the problems (argument rules of tsm2r_s; additionally every A,
 * and B of TSM2R problems, must be 16-byte aligned with 16-byte multiple
 * leading-dimension strides, and TSM2L problems need n <= 64 and k <= 64
 * because batched TSM2L classes hold B on chip: TSM2_ERR_UNSUPPORTED
 * otherwise; the single-problem tsm2l_s has no such limit;
 * TSM2_ERR_INVALID_VALUE for an unknown tile variant), encodes their tensor
 * maps and uploads the plan's tables and workspace (cudaMalloc: make plans
 * outside timed or captured regions).  The operand pointers are recorded:
 * the plan computes on whatever those buffers hold at execution.  Problems
 * with k > 16 (TSM2R) or k > 32 (TSM2L) are split into column groups.  *out
 * receives the plan (mode TSM2_BATCH_SINGLE_LAUNCH). */
tsm2_status tsm2_batch_plan_create_s(int nprob, const tsm2_problem_s *probs, int flags,
                                     tsm2_batch_plan_t *out);

/* Runs every problem of the plan on `stream` in the plan's mode.  Plans must
 * not run concurrently with themselves (their workspace is shared). */
tsm2_status tsm2_batch_plan_execute(tsm2_batch_plan_t plan, void *stream);

/* Runs only class `cls` on `stream`, on all SMs (used to measure classes). */
tsm2_status tsm2_batch_plan_execute_class(tsm2_batch_plan_t plan, int cls, void *stream);

/* Captures tsm2_batch_plan_execute once into a CUDA graph, on a stream the
 * plan owns (re-captured after any change of mode, grids or shares), and
 * launches the graph on `stream` (any stream, including the legacy default
 * stream 0). */
tsm2_status tsm2_batch_plan_graph_launch(tsm2_batch_plan_t plan, void *stream);

int tsm2_batch_plan_num_classes(tsm2_batch_plan_t plan);
tsm2_status tsm2_batch_plan_class_info(tsm2_batch_plan_t plan, int cls, const char **name, double *bytes,
                                       int *grid, int *nprob);

/* Sets the number of persistent blocks of every class in the concurrent mode
 * (each in [1, #SMs]). */
tsm2_status tsm2_batch_plan_set_grids(tsm2_batch_plan_t plan, int ncls, const int *grids);

/* serial != 0: mode TSM2_BATCH_SERIAL, else TSM2_BATCH_CONCURRENT. */
tsm2_status tsm2_batch_plan_set_serial(tsm2_batch_plan_t plan, int serial);

/* Execution mode: TSM2_BATCH_SINGLE_LAUNCH, TSM2_BATCH_SERIAL or
 * TSM2_BATCH_CONCURRENT (TSM2_ERR_INVALID_VALUE otherwise). */
tsm2_status tsm2_batch_plan_set_mode(tsm2_batch_plan_t plan, int mode);

/* Blocks of the single launch, in [1, #SMs] (default #SMs). */
tsm2_status tsm2_batch_plan_set_single_grid(tsm2_batch_plan_t plan, int grid);

/* Kernel launches of one execution in the plan's current mode. */
int tsm2_batch_plan_num_launches(tsm2_batch_plan_t plan);

/* Compiled tile variants and their parameters. */
int tsm2_batch_num_variants(void);
tsm2_status tsm2_batch_variant_info(int variant, const char **name, int *stages, int *rows_per_lane,
                                    int *inner_per_warp);

void tsm2_batch_plan_destroy(tsm2_batch_plan_t plan);

/* Message describing the last error returned to the calling host thread
 * (thread-local; valid until that thread's next call). Never NULL. */
const char *tsm2_get_last_error_string(void);

/* Synchronises `stream`, then reads and clears the current device's status
 * word.  Returns TSM2_ERR_TIMEOUT if a kernel of this library gave up on a
 * bounded pipeline wait since the previous call (its output is then
 * undefined), TSM2_ERR_CUDA if synchronisation failed, else SUCCESS. */
tsm2_status tsm2_get_device_status(void *stream);

/* Frees every workspace the library allocated (all devices).  Call with no
 * library work in flight.  The library stays usable; it reallocates lazily. */
void tsm2_shutdown(void);

/* 1 in the debug build of the library (libtsm2_debug.so, compiled with
 * -DTSM2_DEBUG), 0 otherwise.  The debug build checks every hand-computed
 * global address of the bulk-copy, batched and backward kernels against the
 * extents of its operand (rows and columns of C and B, workspace slots,
 * arrival counters) before the access; an access that would fall outside is
 * skipped and recorded, and tsm2_get_device_status then returns
 * TSM2_ERR_BOUNDS.  It stands in for a memory checker: nothing faults. */
int tsm2_debug_checks(void);

/* ---- Tuning and debugging knobs (process-wide, not thread-safe) ---------- */

/* Upper bound, in nanoseconds, of every pipeline wait inside the kernels
 * (default 1e9).  0 means a single attempt (which the hardware may suspend
 * briefly, so a wait can still succeed); a negative value makes every wait
 * give up at once without testing its barrier, which drives each kernel's
 * timeout path deterministically.  Both are for tests of the error path;
 * copies already issued are always waited for (up to 4 s) before a block
 * exits. */
void tsm2_set_wait_budget_ns(int64_t ns);

/* Kernel path selection: 0 = automatic (default), 1 = always the
 * element-wise path, 2 = the bulk-copy path when alignment allows. */
void tsm2_set_path(int path);

/* Number of thread blocks of the persistent grid (0 = automatic: one per
 * SM, limited so each block gets at least a few work units). */
void tsm2_set_grid(int blocks);

/* Work partition of TSM2L with B on chip (n <= 64): 0 = row blocks claimed
 * at run time from an atomic counter, each block starting with its own
 * (default: blocks on SMs that stream faster take more row blocks), and in
 * the single launch of a batch plan shares adapted from launch to launch;
 * 1 = a static partition, equal contiguous runs of row blocks; 2 = as 0,
 * with batch plans of any size adapting their shares (for tests).  Every
 * row block is computed whole by one thread block in the same order either
 * way, so the results are bitwise equal.  TSM2R and TSM2L with staged B
 * (n > 64) always use their static partitions. */
void tsm2_set_balance(int mode);

/* How the host-operand entry points move page-locked buffers: 0 = copy
 * kernels on the SMs where the device can address the buffer (default),
 * 1 = always the copy engines.  Other values select 0. */
void tsm2_set_host_copy(int mode);

/* Per-block timeline of the bulk-copy kernels and of the batched kernel,
 * for profiling.  When set, every later launch whose grid has at most
 * `blocks` blocks writes four 64-bit words per block b into device memory at
 * device_words[4b..4b+3] (the batched kernel writes only the start and end
 * times, the other two stay as they were):
 * start time, time the first stage arrived, end time (ns, %globaltimer),
 * and the number of work units the block processed (low 32 bits; with
 * TSM2L row blocks claimed at run time also the index of the SM the block
 * ran on in the high 32 bits, else 0 there).  NULL turns it off.
 * The buffer is caller-owned device memory. */
void tsm2_set_trace(unsigned long long *device_words, int64_t blocks);

/* Name of the kernel configuration the last call on this thread launched
 * (for reports and tests). */
const char *tsm2_last_config(void);

/* How the last host-operand call on this thread moved A, B and C: a string
 * "A:<p> B:<p> C:<p>" with <p> "sm" (copy kernels) or "engine" (copy
 * engines); "none" before the first such call (for reports and tests). */
const char *tsm2_last_host_copy(void);

/* ---- Synthetic inputs (definition in tsm2_inputs: splitmix64 counter
 * stream per (seed, matrix_id); element (i,j) of the logical rows x cols
 * matrix is draw i + j*rows).  Column-major, leading dimension ldx.  These
 * exist so that multi-gigabyte benchmark inputs can be generated in device
 * memory; they are not part of the multiply. ------------------------------ */
tsm2_status tsm2_fill_uniform_d(int64_t rows, int64_t cols, uint64_t seed, uint64_t matrix_id,
                                double *X, int64_t ldx, void *stream);
tsm2_status tsm2_fill_uniform_s(int64_t rows, int64_t cols, uint64_t seed, uint64_t matrix_id,
                                float *X, int64_t ldx, void *stream);
tsm2_status tsm2_fill_int_small_d(int64_t rows, int64_t cols, uint64_t seed, uint64_t matrix_id,
                                  double *X, int64_t ldx, void *stream);
tsm2_status tsm2_fill_int_small_s(int64_t rows, int64_t cols, uint64_t seed, uint64_t matrix_id,
                                  float *X, int64_t ldx, void *stream);
tsm2_status tsm2_fill_normal_ih_d(int64_t rows, int64_t cols, uint64_t seed, uint64_t matrix_id,
                                  double scale, double *X, int64_t ldx, void *stream);
tsm2_status tsm2_fill_normal_ih_s(int64_t rows, int64_t cols, uint64_t seed, uint64_t matrix_id,
                                  double scale, float *X, int64_t ldx, void *stream);
tsm2_status tsm2_fill_logmag_s(int64_t rows, int64_t cols, uint64_t seed, uint64_t matrix_id,
                               float *X, int64_t ldx, void *stream);

/* FMA throughput probe for the roofline denominators (not part of the
 * multiply; the paper's model takes the peak FMA rate as an input, Sec. 3.1.8).
 * Launches `blocks` blocks of 256 threads, each thread running 8 independent
 * multiply-add chains of `iters` steps in binary64 (elem = 8, DFMA) or packed
 * binary32 (elem = 4, FFMA2, two lanes per instruction), and writes one value
 * per thread to `sink` (device, blocks * 256 elements of the element type).
 * Work: 16 * iters flops per thread (elem 8) or 32 * iters (elem 4).  The
 * caller times it.  TSM2_ERR_INVALID_VALUE for a bad elem, blocks < 1,
 * iters < 0 or a NULL sink. */
tsm2_status tsm2_fma_probe(int elem, int blocks, int64_t iters, void *sink, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* TSM2_H */
