/*
 * ata.h -- C ABI of the GB300 library for the symmetric product C = A^t A.
 *
 * The operation is the one of Arrigoni & Massini, "Fast Strassen-based A^t A
 * Parallel Multiplication" (arXiv 1902.02104), Section 3, Algorithm 1:
 *
 *   input  A, a real m x n matrix (Algorithm 1, "Input");
 *   output one triangle of C = A^t A (Algorithm 1, "Output"; Section 3 keeps
 *          n(n+1)/2 entries because C is symmetric).
 *
 * The library computes it with the ATA recursion: the 2 x 2 block split of
 * Section 3 (Eq. "submatrices", ceil/floor halves), the block formulas of
 * Eq. "Cij" (diagonal blocks by recursion, the off-diagonal block by
 * Strassen products, Section 4.2.2), and the base case of Algorithm 1 with
 * the cutoff as a parameter.  C_21 is never computed: the library returns
 * C_12 = C_21^t, i.e. the upper triangle.
 *
 * Layouts
 *   A         row-major, m rows, n columns, leading dimension lda >= n
 *             (elements).  Element (k, i) is at A[k*lda + i].  FP64 for
 *             ATA_F64 and ATA_F64_OZAKI, FP32 for the FP32 modes.  Device
 *             memory for ata_execute / ata_execute_batched; host memory for
 *             ata_execute_host.  Never modified.
 *   C_packed  FP64, n(n+1)/2 entries, row-major packed upper triangle:
 *             C(i, j), i <= j, is at i*n - i*(i-1)/2 + (j - i).  This is the
 *             same memory order as LAPACK's column-major packed lower
 *             triangle ('L'), i.e. the paper's lower triangle read by
 *             columns.  Every entry is written (m == 0 writes zeros).
 *
 * Ownership
 *   The caller owns A and C_packed.  A plan owns its device workspace, its
 *   task tables and its CUDA graph; ata_plan_destroy frees them.  A plan
 *   runs one execution at a time (its workspace is reused): an execution
 *   queued on another stream than the plan's latest one first waits for it
 *   (an event the library records), in single, batched and prepared-batch
 *   calls alike, so executions of one plan never overlap on the device.
 *   Run independent products concurrently with separate plans.
 *
 * Errors
 *   Arguments are checked before any work is queued; a bad argument returns
 *   ATA_EINVAL and queues nothing.  Execution is asynchronous on the given
 *   stream: an error raised by the device surfaces as ATA_ECUDA from a later
 *   call on the same plan (or from ata_poll).  NaN and Inf in A propagate by
 *   IEEE rules; they are not checked.  ata_last_error_message() returns a
 *   thread-local description of the last failure.
 */
#ifndef ATA_H
#define ATA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ATA_OK = 0,
    ATA_EINVAL = 1,        /* bad argument; nothing was queued            */
    ATA_ENOMEM = 2,        /* device or host allocation failed            */
    ATA_EUNSUPPORTED = 3,  /* valid request this build cannot run         */
    ATA_ECUDA = 4,         /* CUDA runtime / device error                 */
    ATA_PENDING = 5,       /* ata_poll: request still running             */
    ATA_ETIMEOUT = 6,      /* ata_poll / ata_server_wait: time limit hit  */
    ATA_EBUSY = 7          /* admission refused: no slot or budget free   */
} ata_status;

/* Input type and leaf arithmetic. */
typedef enum {
    ATA_F64 = 0,           /* FP64 input, FP64 leaves (DFMA), FP64 sums       */
    ATA_F32_BF16X3 = 1,    /* FP32 input, leaves on bf16 tensor cores with a
                              3-way split of each operand; the leading part
                              products are summed exactly per 256-deep K
                              chunk, the chunks added into a pair of FP32
                              values, and the result written in FP64;
                              normwise error <= 1e-6                          */
    ATA_F32_TF32 = 2,      /* FP32 input rounded to TF32, tensor-core leaves
                              accumulating in FP32 over the whole K, the
                              result written in FP64; normwise error <= 1e-3 */
    ATA_F64_OZAKI = 3      /* FP64 input, FP64-accuracy leaves emulated on
                              bf16 tensor cores (exact slice products, FP64
                              Strassen sums and final accumulation).  Each
                              column of a leaf operand is held in 48-bit
                              fixed point below the column's largest entry
                              M_i, and the low-order part products add in
                              FP32, so the bound that holds for every input
                              is |C_ij - (A^t A)_ij| <= 2^-35 K M_i M_j for
                              classical leaves (K = m).  Componentwise
                              |dC_ij| <= 1e-11 (|A|^t|A|)_ij is measured on
                              inputs whose columns keep their weight within a
                              bounded range of the column maximum: i.i.d.
                              entries, columns scaled over 2^+-200, row bands
                              scaled over 2^+-20.  It does not hold when a
                              column has a few entries far above its others
                              in rows where another column is small (one
                              entry 2^30 above the rest gives about 1e-7 on
                              the pair); ATA_F64 meets it for every input.
                              With Strassen levels the error is bounded
                              normwise.                                      */
} ata_dtype;

/* Strassen form used for the off-diagonal products. */
typedef enum {
    ATA_STRASSEN = 0,      /* Strassen 1969, the form of Section 4.2.2        */
    ATA_WINOGRAD = 1       /* Winograd's variant (Section 1)                  */
} ata_variant;

typedef struct ata_plan_s* ata_plan;

/* Planner statistics (host-only; see ata_plan_query). */
typedef struct {
    int64_t m, n;
    int32_t dtype, cutoff;      /* cutoff actually used                    */
    int32_t depth;              /* levels of the ATA column recursion      */
    int32_t n_diag_leaves;      /* base-case (diagonal) blocks             */
    int32_t n_nodes;            /* off-diagonal products C_12, one per node*/
    int32_t max_strassen_levels;
    int32_t n_leaf_products;    /* products run by the leaf kernel         */
    int32_t n_leaf_tiles;       /* output tiles of the leaf launch          */
    int32_t n_sum_tasks;        /* materialised Strassen operand sums       */
    int32_t n_combine_tasks;    /* Strassen output combines                 */
    int32_t n_launches;         /* kernels per execution                    */
    int64_t mults;              /* scalar multiplications of the tree (on
                                   padded sizes; Section 3.1 recurrence)    */
    int64_t classical_mults;    /* m * n (n + 1) / 2                        */
    int64_t adds;               /* scalar additions of Strassen sums/combines*/
    int64_t workspace_bytes;    /* device workspace the plan allocates      */
    int32_t leaf_tile_rows;     /* output tile of the leaf kernel: rows ... */
    int32_t leaf_tile_cols;     /* ... and columns.  Tensor-core leaves use
                                   CTA-pair tiles (two SMs per tile; 256 x
                                   256 for TF32, 256 x 128 otherwise) when
                                   every leaf is padded to them and they add
                                   at most 1/8 to the tile area;
                                   ata_plan_query reports the planned shape,
                                   ata_plan_get_info the one that runs on
                                   the plan's device                        */
    int64_t r;                  /* general product X^t Y: columns of Y (and
                                   n = columns of X, m = rows of both);
                                   0 for A^t A plans                        */
} ata_plan_info;

/* Status text ("ATA_OK", ...).  Never NULL. */
const char* ata_status_string(ata_status s);

/* Thread-local description of the last failure in this thread. */
const char* ata_last_error_message(void);

/* Device memory the library holds for its own buffers (plan workspaces, task
 * tables, staging buffers of the host-memory calls, batched bindings), in
 * bytes: what every live plan, batch and server holds together.  Destroying
 * them returns it to zero; a value that stays above zero afterwards is a
 * leak.
 *
 * Allocation failures can be injected from the host for tests: with the
 * environment variable ATA_FAULT=alloc@N, the N-th of these allocations
 * after the variable takes that value fails as if the device were out of
 * memory (the call returns ATA_ENOMEM and frees what it had allocated).
 * Every device allocation the library makes goes through this count except
 * the static array of ata_execute_static_scratch. */
int64_t ata_device_bytes_held(void);

/* Run the planner only (no device call): fills *out for the plan that
 * ata_plan_create(m, n, dtype, cutoff) would build.  cutoff must be in
 * [16, 4096]; 0 selects it by the planner's cost model (as ata_plan_create).
 * Errors: ATA_EINVAL for m < 0, n < 0, a bad dtype or cutoff, n > 2^31-1. */
ata_status ata_plan_query(int64_t m, int64_t n, ata_dtype dtype, int cutoff,
                          ata_plan_info* out);

/* Build a plan for an m x n input: the recursion tree of Algorithm 1 (base
 * case min(rows, cols) <= cutoff), the Strassen products of every
 * off-diagonal block, the task tables, and the device workspace (allocated
 * here, on the current device).  cutoff in [16, 4096]; 0 = autotune: the
 * cutoff minimising the planner's cost model of this part (leaf
 * multiply-adds, Strassen additions and workspace traffic at the measured
 * rates, workspace capped at 48 GiB), cached per shape and dtype.  Each
 * Strassen level holds the operand sums and outputs of all its products at
 * once; when no cutoff fits the cap, the autotune lowers the Strassen level
 * cap (unless max_strassen_levels fixes it) until one does, and when none
 * fits even without Strassen levels it takes the plan with the smallest
 * workspace.
 * Errors: ATA_EINVAL (bad sizes, dtype or cutoff, NULL out), ATA_ENOMEM,
 * ATA_ECUDA. */
ata_status ata_plan_create(ata_plan* out, int64_t m, int64_t n,
                           ata_dtype dtype, int cutoff);

/* Planner options beyond the cutoff.  Fields set to -1 take the default. */
typedef struct {
    int32_t cutoff;              /* as in ata_plan_create (0 = autotune)      */
    int32_t variant;             /* ata_variant (-1 = ATA_STRASSEN)            */
    int32_t fuse_levels;         /* bottom Strassen levels whose operand sums
                                    are formed inside the leaf loads instead of
                                    materialised (-1 = dtype default: 0 for
                                    ATA_F64; for ATA_F64_OZAKI 1 (sums formed
                                    in fixed point while slicing), 0 with
                                    Winograd's variant; 1 for the FP32 modes) */
    int32_t max_strassen_levels; /* cap on Strassen levels per product
                                    (-1 = none, or what fits the workspace
                                    cap when the cutoff is autotuned; 0 =
                                    classical products)                       */
    int32_t cta_pair;            /* tensor-core leaves: 1 = output tiles
                                    computed by CTA pairs (two SMs, tcgen05
                                    cta_group::2; 256 x 256 for TF32, 256 x
                                    128 otherwise) when every leaf is wider
                                    than 128 rows and the pair tiles add at
                                    most 1/8 to the tile area; 0 = 128 x 128 tiles
                                    on single CTAs; -1 = the mode's default
                                    (pairs for TF32, single CTAs otherwise) */
    int32_t wait_limit_us;       /* tensor-core leaves: limit of each wait of
                                    the leaf kernel's pipeline (TMA producer,
                                    MMA issuer, epilogue) in microseconds, in
                                    [1, 1000000]; -1 or 0 = 1 s.  A wait that
                                    runs out records its code in the plan's
                                    device status word (ata_plan_device_status)
                                    and the kernel returns without finishing;
                                    the waits for copies and MMAs still in
                                    flight before the kernel exits keep 1 s.
                                    For tests of that failure path: a limit
                                    shorter than the pipeline's latency makes
                                    the waits run out on purpose */
} ata_plan_options;

/* Same as ata_plan_create with explicit options (opts may not be NULL).
 * Errors: as ata_plan_create; ATA_EUNSUPPORTED if the fused operands would
 * exceed the kernels' 32 terms per operand. */
ata_status ata_plan_create_opts(ata_plan* out, int64_t m, int64_t n,
                                ata_dtype dtype, const ata_plan_options* opts);

/* Host-side check of the plan ata_plan_create_opts(m, n, dtype, opts) would
 * build (no device call): every read and write of every task stays inside
 * A (m x n), the workspace and C, and the tasks write every entry of the
 * packed triangle exactly once (the latter for n <= 4096).  Returns ATA_OK,
 * or ATA_EINVAL with the first violation in ata_last_error_message(). */
ata_status ata_plan_check(int64_t m, int64_t n, ata_dtype dtype,
                          const ata_plan_options* opts);

/* ata_plan_query with explicit options. */
ata_status ata_plan_query_opts(int64_t m, int64_t n, ata_dtype dtype,
                               const ata_plan_options* opts,
                               ata_plan_info* out);

/* Measured tuning: chooses the cutoff (and, when base->cta_pair is -1 in a
 * tensor-core mode, single-CTA or CTA-pair tiles) for an m x n product by
 * timing on the current device.  The planner's cost model ranks the
 * cutoffs; its best `candidates` (1..8), each with both tile forms where
 * they are tuned, run on a synthetic input of the exact shape (device
 * buffers allocated and freed here): one untimed execution, then three
 * timed with CUDA events on a stream of the call's own; the median decides.
 * Fills *out with base's options and the winning cutoff and cta_pair, and
 * *best_ms (may be NULL) with the winner's median time.  Results are cached
 * per (device, m, n, dtype, base options) for the process, so a second call
 * returns at once.  base may be NULL (all defaults; its cutoff is ignored).  Runs
 * work on the device and synchronises with it: call it before the timed or
 * captured part of an application.
 * Errors: as ata_plan_query_opts, ATA_ENOMEM (no candidate fits), ATA_ECUDA. */
ata_status ata_tune(int64_t m, int64_t n, ata_dtype dtype,
                    const ata_plan_options* base, int candidates,
                    ata_plan_options* out, float* best_ms);

/* Statistics of a created plan. */
ata_status ata_plan_get_info(ata_plan plan, ata_plan_info* out);

/* Device workspace held by the plan, in bytes. */
ata_status ata_plan_workspace_size(ata_plan plan, size_t* bytes);

/* C_packed = A^t A, queued on `stream` (a cudaStream_t; NULL = legacy
 * default stream).  A and C_packed are device pointers (layouts above).
 * The first call on a plan captures its CUDA graph; later calls replay it.
 * Returns once the work is queued.
 * Inside a stream capture (the caller building its own CUDA graph) the
 * plan's kernels are recorded into that capture themselves, since a graph
 * launch cannot be captured: the same kernels and parameters.  The captured
 * graph then reads A and writes C_packed at those pointers.  The plan must
 * outlive it, and the caller orders its replays with the plan's other
 * executions.  The plan's tables must already be those of this lda (a call
 * outside the capture with it, or lda = n); otherwise the call returns
 * ATA_EINVAL and queues nothing (the capture stays valid).
 * Errors: ATA_EINVAL (NULL plan, lda < n, NULL A with m*n > 0, NULL
 * C_packed with n > 0, A or C_packed not 8-byte aligned), ATA_ECUDA. */
ata_status ata_execute(ata_plan plan, const void* A, int64_t lda,
                       double* C_packed, void* stream);

/* End-to-end convenience: A and C_packed in HOST memory.  Copies A to the
 * device, runs ata_execute on `stream`, copies C back and waits for the
 * stream.  Device staging buffers are owned by the plan (allocated on first
 * use).  Not on a capturing stream (host copies cannot be recorded).
 * Errors: as ata_execute (ATA_EINVAL also for a capturing stream), plus
 * ATA_ENOMEM. */
ata_status ata_execute_host(ata_plan plan, const void* A_host, int64_t lda,
                            double* C_packed_host, void* stream);

/* Pipelined end-to-end execution for a stream of inputs: queues the copy of
 * A_host (host memory, leading dimension lda) to the device, the execution
 * and the copy of the packed result to C_packed_host on streams the plan
 * owns, and returns without waiting.  Successive calls alternate between two
 * device staging sets (allocated on first use: 2 x (m n + n(n+1)/2)
 * elements), so that the copies of one call overlap the executions of its
 * neighbours; executions run one at a time in call order.  Host buffers
 * should be pinned (page-locked) for the copies to overlap.  A_host may not
 * be modified, and C_packed_host not read, until ata_plan_wait returns; a
 * plan's pipelined calls come from one thread at a time and are not mixed
 * with other executions of the same plan before ata_plan_wait.
 * Errors: as ata_execute_host; errors of the queued work are reported by
 * ata_plan_wait. */
ata_status ata_execute_host_async(ata_plan plan, const void* A_host,
                                  int64_t lda, double* C_packed_host);

/* Waits until every call queued by ata_execute_host_async on plan has
 * finished (ATA_OK at once if there was none).  Errors: ATA_EINVAL (NULL
 * plan), ATA_ECUDA (a queued copy or execution failed). */
ata_status ata_plan_wait(ata_plan plan);

/* Many independent products in one queued batch: plans[i] (each built for
 * its own m_i x n_i and dtype) applied to A[i] (device, leading dimension
 * lda[i]) into C_packed[i].  All leaf tiles of all instances run in one
 * persistent launch, heaviest first; sums and combines are grouped per
 * level across instances.  Plans may not repeat within one call.  Not on
 * a capturing stream (the batch's graph is launched and its bindings may be
 * uploaded from host memory): capture ata_execute per plan instead.
 * Errors: ATA_EINVAL (count < 0, NULL arrays, a repeated plan, mixed dtype
 * families, a capturing stream), ATA_ENOMEM, ATA_ECUDA. */
ata_status ata_execute_batched(const ata_plan* plans, int count,
                               const void* const* A, const int64_t* lda,
                               double* const* C_packed, void* stream);

/* A prepared batch: the same execution as ata_execute_batched, with the
 * plans bound once to one packed layout, so that a call passes two device
 * pointers.  Instance i reads its A at element offset a_off[i] of the input
 * buffer (leading dimension lda[i]; elements of the plans' input type) and
 * writes its packed C at element offset c_off[i] of one FP64 output buffer.
 * The caller sizes both buffers to cover every instance and keeps the
 * instances' C ranges disjoint.  The merged task tables are built here; the
 * batch's graph is captured on the first execution, and when A or C moves
 * only the instances' bindings (a device array the kernels read) are
 * uploaded again.  The plans must stay alive: destroying one of
 * them retires the batch (its executions then fail with ATA_EINVAL).
 * Errors: ATA_EINVAL (NULL out, count < 0, NULL arrays with count > 0, a
 * NULL or repeated plan, mixed dtype families, lda[i] < max(n_i, 1), a
 * negative offset), ATA_ENOMEM, ATA_ECUDA. */
typedef struct ata_batch_s* ata_batch;
ata_status ata_batch_create(ata_batch* out, const ata_plan* plans, int count,
                            const int64_t* lda, const int64_t* a_off,
                            const int64_t* c_off);

/* Queue one execution of the batch on `stream`: A and C are the device
 * buffers of the layout above (A aligned to its element size, C to 8 bytes).
 * Returns once the work is queued.  Not on a capturing stream (as
 * ata_execute_batched).  Errors: ATA_EINVAL (NULL batch, NULL or misaligned
 * A or C with count > 0, a plan of the batch destroyed, a capturing stream),
 * ATA_ECUDA. */
ata_status ata_batch_execute(ata_batch batch, const void* A, double* C,
                             void* stream);

/* Kernel launches one execution of the batch makes (the kernel nodes of its
 * graph).  Errors: ATA_EINVAL (NULL argument, not executed yet, a
 * plan destroyed). */
ata_status ata_batch_graph_kernels(ata_batch batch, int32_t* kernels);

/* Release the batch (waits for the device first).  The plans stay. */
void ata_batch_destroy(ata_batch batch);

/* Stage timing.  With enable != 0 the plan's graph also records CUDA events
 * on the execution stream around its stages (the graph is re-captured on the
 * next ata_execute).  ata_plan_stage_times fills ms[4] for the most recent
 * execution (which must have completed): the Strassen operand-split
 * launches, the leaf operand preparation (tensor-core modes; 0 for FP64),
 * the leaf product kernel, and the Strassen combine launches.
 * Errors: ATA_EINVAL (NULL arguments, timing not enabled, no execution yet),
 * ATA_ECUDA. */
ata_status ata_plan_enable_stage_timing(ata_plan plan, int enable);
ata_status ata_plan_stage_times(ata_plan plan, float* ms);

/* Kernel launches one execution of the plan makes: the kernel nodes of its
 * captured CUDA graph (the graph of its most recent ata_execute).  Errors:
 * ATA_EINVAL (NULL argument, or the plan has not been executed yet). */
ata_status ata_plan_graph_kernels(ata_plan plan, int32_t* kernels);

/* The same for ata_execute_batched(plans, count, ..., lda, ...): the kernel
 * nodes of its graph.  Errors: ATA_EINVAL
 * (NULL or invalid argument, or the batch has not been executed yet). */
ata_status ata_batched_graph_kernels(const ata_plan* plans, int count,
                                     const int64_t* lda, int32_t* kernels);

/* Error word of the plan's tensor-core kernels (0 = none).  Their waits on
 * pipeline barriers are bounded (1 s); a wait that gives up records a
 * nonzero code (1 TMA producer, 2 MMA issuer, 3 epilogue), the kernel
 * returns without finishing, and the word stays set for the plan.
 * Synchronises with the device.  Errors: ATA_EINVAL, ATA_ECUDA. */
ata_status ata_plan_device_status(ata_plan plan, int* code);

/* Release the plan (waits for its queued work first). */
void ata_plan_destroy(ata_plan plan);

/* ---------------------------------------------------------------------------
 * General product C = X^t Y: the HASA step of Section 4.2.2 as an entry point
 * of its own (the off-diagonal block C_12 = A_L^t A_R of the recursion is one
 * such product).  X is m x p and Y is m x r, row-major with leading
 * dimensions ldx >= p and ldy >= r (FP64 for ATA_F64 / ATA_F64_OZAKI, FP32
 * for ATA_F32_BF16X3 / ATA_F32_TF32, as A above); C is p x r, row-major FP64
 * with ldc >= r, every entry written.  Strassen levels (Section 4.2.2, with
 * the corrected M1 and M7, or Winograd's variant) run while min(p, m, r) >
 * cutoff, halving all three with ceil/floor and implicit zero padding; the
 * leaves are the same kernels as A^t A's off-diagonal products.  Plans are
 * ata_plan objects: ata_plan_get_info, ata_plan_workspace_size, stage
 * timing, ata_plan_device_status and ata_plan_destroy apply; ata_execute,
 * ata_execute_host and ata_execute_batched reject them (ATA_EINVAL).
 * opts may be NULL (all defaults, cutoff autotuned).
 * -------------------------------------------------------------------------*/

/* Planner only (no device call); info.n = p, info.r = r,
 * info.classical_mults = m p r.  Errors: ATA_EINVAL (negative sizes, a size
 * >= 2^31, bad dtype or options, NULL out). */
ata_status ata_gemm_query(int64_t m, int64_t p, int64_t r, ata_dtype dtype,
                          const ata_plan_options* opts, ata_plan_info* out);

/* Host check of the plan's tables: every term inside X, Y or the workspace,
 * every workspace range inside the workspace, every entry of C written
 * exactly once (checked up to 2^24 entries).  Errors: ATA_EINVAL with the
 * first violation in ata_last_error_message(). */
ata_status ata_gemm_plan_check(int64_t m, int64_t p, int64_t r, ata_dtype dtype,
                               const ata_plan_options* opts);

/* Build a general-product plan on the current device (workspace allocated
 * here).  Errors: as ata_gemm_query, plus ATA_ENOMEM, ATA_ECUDA. */
ata_status ata_gemm_plan_create(ata_plan* out, int64_t m, int64_t p, int64_t r,
                                ata_dtype dtype, const ata_plan_options* opts);

/* C = X^t Y, queued on `stream` (device pointers; layouts above; X and Y
 * not modified).  The first call, and a call with other leading dimensions,
 * captures the plan's graph.  Inside a stream capture the kernels are
 * recorded into it, as for ata_execute (the tables must already be those of
 * ldx, ldy and ldc).  Errors: ATA_EINVAL (an A^t A plan, ldx < p,
 * ldy < r, ldc < r, NULL X or Y with m p r > 0, NULL C with p r > 0,
 * pointers not aligned to their element size), ATA_ECUDA. */
ata_status ata_gemm_tn(ata_plan plan, const void* X, int64_t ldx,
                       const void* Y, int64_t ldy, double* C, int64_t ldc,
                       void* stream);

/* C_packed = A^t A (FP64, as ata_execute with ATA_F64 and the given
 * cutoff) without allocating any device memory.  The paper has no
 * counterpart: this entry point exists for callers that may not allocate
 * while they run -- code that is about to capture a CUDA graph, services
 * that fix their device-memory footprint at start-up, and hosts whose device
 * memory belongs to another allocator.  The task tables, the tile counter
 * and the Strassen workspace live in a static device array of 64 MiB built
 * into the library (every GPU that loads the library holds it until the
 * process exits); the caller passes A and C_packed (device pointers,
 * layouts as above).
 * The first call on a device looks up the array's device address (once per
 * device); make that first call before any stream capture.  Every call
 * shares the one array and overwrites what the previous call left there, so
 * calls whose work overlaps on the GPU (other streams, other host threads)
 * race; calls queued on one stream are ordered.  The host task tables are
 * copied into the array with cudaMemcpyAsync on `stream` from a host buffer
 * that lives only for the call, so a call on a stream that is capturing is
 * refused (ATA_EINVAL) rather than recorded.
 * Errors: ATA_EINVAL (bad sizes or pointers, cutoff outside [16, 4096], a
 * capturing stream, or a problem whose tables and workspace exceed the
 * 64 MiB array -- use ata_execute or a larger cutoff), ATA_ECUDA. */
ata_status ata_execute_static_scratch(int64_t m, int64_t n, const double* A,
                                      int64_t lda, double* C_packed,
                                      int cutoff, void* stream);

/* ------------------------------------------------------------------ */
/* Serving: continuous batching of independent requests.               */
/* ------------------------------------------------------------------ */

typedef struct ata_server_s* ata_server;
typedef uint64_t ata_ticket;

/* Start a server on the current device: a host scheduler thread, up to
 * max_inflight concurrent requests on their own streams, and a device-memory
 * budget (bytes) that bounds the plans' workspaces and staging buffers held
 * at once.  Plans are created on first use of a shape and stay resident
 * while the budget allows.  A request is admitted when a stream slot is
 * free, its plan fits the budget, and the device reports that much memory
 * free plus a 256 MiB reserve (cudaMemGetInfo); otherwise idle plans are
 * evicted, least recently used first, once no request is in flight, or the
 * request waits.  A request that cannot fit even then fails with ATA_EBUSY.
 * Each request's kernels are launched directly on its slot's stream (no
 * graph capture on the scheduler thread).  The server's streams do not wait
 * for the caller's streams: A must be complete, and C free, when a request
 * is submitted.  Errors: ATA_EINVAL, ATA_ENOMEM, ATA_ECUDA. */
ata_status ata_server_create(ata_server* out, size_t device_budget_bytes,
                             ata_dtype dtype, int max_inflight);

/* Submit one request: A (device pointer, m x n, lda) -> C_packed (device).
 * The buffers must stay valid until the ticket completes.  Returns at once
 * with a ticket; the request is admitted when a slot and budget bytes are
 * free.  Errors: ATA_EINVAL (bad sizes or pointers), ATA_EBUSY (the request
 * alone exceeds the budget). */
ata_status ata_submit(ata_server srv, int64_t m, int64_t n, const void* A,
                      int64_t lda, double* C_packed, ata_ticket* ticket);

/* Completion check.  timeout_us = 0 polls once; > 0 waits up to that long.
 * Returns ATA_OK (done; the ticket is released), ATA_PENDING (timeout_us ==
 * 0 and not done), ATA_ETIMEOUT (waited and not done), ATA_EINVAL (unknown
 * ticket), or the request's own error. */
ata_status ata_poll(ata_server srv, ata_ticket ticket, int timeout_us);

/* Latency statistics of completed requests (submit to completion seen by
 * the scheduler), in microseconds, and the count. */
ata_status ata_server_stats(ata_server srv, double* p50_us, double* p99_us,
                            int64_t* completed);

/* Forget the latencies recorded so far (e.g. after a warm-up phase), and
 * the kernel count below. */
ata_status ata_server_reset_stats(ata_server srv);

/* Kernel launches of the executions the server has queued since it was
 * created or its statistics were reset (each execution: the kernel nodes of
 * its plan's graph, as ata_plan_graph_kernels).  Errors: ATA_EINVAL. */
ata_status ata_server_kernels(ata_server srv, int64_t* kernels);

/* Stop the scheduler after draining queued work, then free everything. */
void ata_server_destroy(ata_server srv);

#ifdef __cplusplus
}
#endif

#endif /* ATA_H */
