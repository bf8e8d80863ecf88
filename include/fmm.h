/*
 * fmm.h -- C ABI of the GB300 (sm_103a) recursive Strassen-Winograd SGEMM.
 *
 * The operation is C <- alpha * A * B + beta * C on single-precision matrices,
 * computed by `depth` levels of Winograd's variant of Strassen's recursion
 * (7 sub-products and 15 quadrant additions per level) over dense classical
 * tensor-core leaves.  Background: D'Alberto, "A Heterogeneous Accelerated
 * Matrix Multiplication: OpenCL + APU + GPU + Fast Matrix Multiply"
 * (arXiv 1205.2927): the quadrant division of any m x n matrix is Eq. 1,
 * the recursive C = AB / C += AB skeleton is Table 1, the leaf is an SGEMM
 * (Sec. 3.2), and the fast recursion based on Winograd's algorithm is the
 * optimisation named at the end of Sec. 4.3.  Throughput is reported as
 * 2MNK / wall-clock (Sec. 4), with transfers included for host operands.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Layout.     Row-major with leading dimensions in ELEMENTS: element (i, j)
 *             of A is A[i * lda + j]; A is M x K, B is K x N, C is M x N.
 *             Column-major callers compute C^T = B^T A^T by swapping A/B and
 *             M/N.
 * Semantics.  Netlib SGEMM: beta == 0 writes C without reading it (NaN in C
 *             is not propagated); alpha == 0 or K == 0 reads neither A nor B
 *             and sets C <- beta * C; M == 0 or N == 0 is a no-op.
 * Ownership.  The caller owns A, B, C and the workspace; the library never
 *             frees caller memory.  A plan owns only small host state.
 * Streams.    Every device operation is enqueued on the caller's stream; no
 *             entry point synchronises the device unless stated.
 * Errors.     Every entry point returns a status and never aborts.  Invalid
 *             arguments are rejected before any device work.  Kernel-side
 *             faults that the kernels detect (a bounded wait that ran out,
 *             an inconsistent descriptor) are recorded in a device status
 *             word, read with fmm_get_device_status().
 * No fallback. There is no CPU path: without a CUDA device every compute
 *             call returns FMM_ERR_NO_DEVICE.
 */
#ifndef FMM_GB300_H
#define FMM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* fmm_stream_t; /* == cudaStream_t; NULL = legacy default stream */

typedef enum {
    FMM_OK = 0,
    FMM_ERR_INVALID_ARG = 1,     /* null pointer, negative size, ld < row length, bad option */
    FMM_ERR_ALIGNMENT = 2,       /* operand alignment the plan cannot handle */
    FMM_ERR_SHAPE_MISMATCH = 3,  /* plan used with other sizes / leading dimensions */
    FMM_ERR_OOM = 4,             /* host allocation failed */
    FMM_ERR_CUDA = 5,            /* a CUDA runtime call failed (message: fmm_last_error()) */
    FMM_ERR_UNSUPPORTED = 6,     /* option combination not implemented */
    FMM_ERR_TIMEOUT = 7,         /* a bounded device wait ran out (device status word) */
    FMM_ERR_NO_DEVICE = 8,       /* no CUDA device, or not an sm_103 device */
    FMM_ERR_WORKSPACE = 9        /* workspace missing or smaller than required */
} fmm_status_t;

typedef enum {
    FMM_PREC_FP32 = 0,   /* 3 x TF32: hi*hi + hi*lo + lo*hi, fp32 accumulate (FP32-class) */
    FMM_PREC_TF32 = 1,   /* one TF32 product, fp32 accumulate */
    FMM_PREC_BF16X3 = 2, /* bfloat16 hi/lo split, 3 products, fp32 accumulate */
    FMM_PREC_FP16X3 = 3  /* IEEE half hi/lo split with power-of-two scaling, 3 products */
} fmm_precision_t;

typedef enum {
    FMM_ODD_PAD = 0,  /* virtual zero padding of the bottom/right quadrants (Eq. 1) */
    FMM_ODD_PEEL = 1, /* even core through the recursion + classical border fix-ups */
    FMM_ODD_TILE = 2, /* peeling with whole leaf tiles: the recursion covers the largest
                         multiple of (leaf tile x 2^depth) in M and N (256 x 2^depth for CTA
                         pairs), so every leaf is a whole number of tiles; the border rows and
                         columns (and K's remainder modulo 4 x 2^depth) run as classical leaves */
    FMM_ODD_AUTO = 3  /* TILE when each of M and N leaves a remainder of at most an eighth
                         of its whole-tile granule, and some remainder; else PAD.
                         Host-resident and batched plans pad.
                         fmm_plan_info reports the mode taken */
} fmm_odd_t;

typedef enum {
    FMM_PLANNER_FIXED = 0,      /* fixed size thresholds (the paper's Table 2 style) */
    FMM_PLANNER_EXHAUSTIVE = 1, /* time every candidate plan on the device, keep the best */
    FMM_PLANNER_MLP = 2         /* score candidates with the registered cost-model network */
} fmm_planner_t;

typedef enum {
    FMM_ALGO_WINOGRAD = 0,   /* 7-product Winograd recursion */
    FMM_ALGO_CLASSICAL = 1   /* 8-product quadrant recursion of Table 1 (RMUL): C_ij = sum_k
                                A_ik B_kj.  The independent (i, j) blocks share one leaf
                                launch; the k-blocks (Eq. 1's halves of K per level, rounded
                                up to 8 elements) are accumulated in order, the first with
                                the caller's beta, the rest with beta = 1.  Depth 0 equals
                                Winograd depth 0.  The fixed rule picks the depth; host-
                                resident, batched and autotuned plans return
                                FMM_ERR_UNSUPPORTED */
} fmm_algo_t;

typedef struct {
    int depth;                 /* recursion levels; -1 = chosen by the planner */
    int cutoff;                /* planner: smallest leaf dimension worth a level (elements) */
    int leaf_tile;             /* leaf tile: 128 or 256 (128 x N tile on one SM), 512 (256 x 256
                                  tile on a pair of SMs; TF32 batched plans and a peeled border
                                  use 256 instead); 0 = chosen with the depth (batched: 512,
                                  or 256 for TF32) */
    fmm_precision_t precision;
    fmm_odd_t odd;
    fmm_planner_t planner;
    fmm_algo_t algo;
    int host_operands;         /* 1: A, B, C may be pinned host memory (streamed in/out) */
    int refine_fp64;           /* reserved: residual refinement in float64 (fmm_residual) */
    int fuse_last;             /* last Winograd level inside the leaf launch: the seven products
                                  of each last-level node are folded into the node's output
                                  quadrants as they complete (the U-chain in its own order, so
                                  the result is bitwise that of the separate post-addition
                                  pass) and never stored.  Applies to depth-2 to depth-4 plans
                                  on CTA-pair tiles with split-plane leaves (FP32, BF16X3,
                                  FP16X3; device operands).  1 on, -1 off, 0 library default
                                  (on at depths 2 and 3 when every leaf is whole 256 x 256
                                  tiles in M and N, off otherwise and at depth 4) */
    int host_copy;             /* host-resident plans: how A, B, C cross the host link.
                                  1: copy engines (cudaMemcpy2DAsync); 2: SM loads and stores
                                  on the device mapping of the pinned memory (32 blocks; the
                                  same link rate one way, no duplex, but no stall where the
                                  copy engines stall; copy engines for memory without a device
                                  mapping); 0: library default: copy engines until a call's
                                  input transfers (at least 64 MiB, not the plan's first call)
                                  ran at under half of the link's rate, SM copies from the
                                  first call after that judgement (fmm_plan_host_copy) */
} fmm_options_t;

typedef struct fmm_plan_s* fmm_plan_t;

/* Fill *opt with defaults: depth -1, cutoff 2048, leaf_tile 0, FP32, AUTO odd
 * sizes, FIXED planner, Winograd, device operands, fuse_last 0 (the library's
 * choice).  Returns FMM_ERR_INVALID_ARG on NULL. */
fmm_status_t fmm_options_default(fmm_options_t* opt);

/* Build a plan for one (M, N, K, lda, ldb, ldc, options) problem.
 *   out              receives the plan; if NULL, only *workspace_needed is set.
 *   workspace        device memory owned by the caller, 256-byte aligned, at
 *                    least *workspace_needed bytes; it must outlive the plan
 *                    and must not be shared by plans running concurrently.
 *   workspace_needed optional; receives the byte count this plan requires.
 * The planner runs here (FMM_PLANNER_EXHAUSTIVE times candidates on `stream`
 * and synchronises it).  Requires ld >= row length (lda >= K, ldb >= N,
 * ldc >= N).  Errors: INVALID_ARG, WORKSPACE, UNSUPPORTED, NO_DEVICE, CUDA. */
fmm_status_t fmm_plan(fmm_plan_t* out, int64_t M, int64_t N, int64_t K,
                      int64_t lda, int64_t ldb, int64_t ldc, const fmm_options_t* opt,
                      void* workspace, size_t workspace_bytes, size_t* workspace_needed,
                      fmm_stream_t stream);

/* Run the plan: C <- alpha * A * B + beta * C.  A, B, C are device pointers,
 * or pinned host pointers when the plan was made with host_operands = 1 (then
 * the call streams A and B in and C out on internal copy streams ordered
 * after `stream`; C is complete in host memory once `stream` has reached this
 * point, e.g. after cudaStreamSynchronize(stream)).  Pageable host memory is
 * rejected with FMM_ERR_INVALID_ARG.  Asynchronous in both cases.
 * A plan serves one call at a time: calls on one stream are ordered by the
 * stream; calls of one plan on different streams must be ordered by the
 * caller, since they share the plan's workspace temporaries and its
 * tile-scheduling area. */
fmm_status_t fmm_gemm(fmm_plan_t plan, float alpha, const float* A, const float* B,
                      float beta, float* C, fmm_stream_t stream);

/* Many independent products C_i <- alpha_i A_i B_i + beta_i C_i of uneven
 * sizes in one persistent tensor-core launch.  All arrays have `count`
 * entries and live in host memory; the matrices are device pointers.  With
 * workspace == NULL only *workspace_needed is set.  The plan (each size
 * class's depth, the launch's leaf tile) follows opt->planner as in
 * fmm_batched_plan.  Asynchronous unless the planner times candidates. */
fmm_status_t fmm_gemm_batched(int count, const int64_t* M, const int64_t* N, const int64_t* K,
                              const float* const* A, const int64_t* lda,
                              const float* const* B, const int64_t* ldb,
                              float* const* C, const int64_t* ldc,
                              const float* alpha, const float* beta,
                              const fmm_options_t* opt, void* workspace, size_t workspace_bytes,
                              size_t* workspace_needed, fmm_stream_t stream);

/* Batched plan: the same products as fmm_gemm_batched, split so that the
 * launches can be captured in a CUDA graph and replayed.  fmm_batched_plan
 * picks the depths and the leaf tile, encodes every tensor map and leaf
 * descriptor and copies the tables into the workspace (synchronously).
 * Problems fall into size classes (smallest and largest dimension, each
 * rounded to a power of two); the launch has one leaf tile (opt->leaf_tile,
 * or chosen):
 *   opt->depth >= 0 or FMM_PLANNER_FIXED: the fixed rule per problem, tile
 *     512 (CTA pairs) for the split-plane precisions, 256 for TF32;
 *   FMM_PLANNER_EXHAUSTIVE: per leaf tile, one pass of coordinate descent over
 *     the classes, largest work first, timing each class's candidate depths as
 *     whole-batch launches on scratch outputs in the workspace (the caller's
 *     A and B are read, C is not touched; synchronises `stream`);
 *   FMM_PLANNER_MLP: the registered cost model scores every problem at every
 *     candidate (depth, tile) in one inference launch; each class takes the
 *     depth of least predicted sum, the launch the tile of least predicted
 *     total; that proposal and the fixed rule's plan are then timed as
 *     whole-batch launches (as EXHAUSTIVE does) and the faster is kept, since
 *     the model predicts problems run alone (without a model: EXHAUSTIVE).
 * A problem's depth never exceeds 4 or leaves below 64 wide.
 * fmm_batched_run then only launches kernels: one
 * batched transpose/copy launch, the pre-additions of the problems that
 * recurse, ONE persistent leaf launch over every leaf product of every problem
 * (longest tiles first), and the post-additions; FP16x3 first derives every
 * problem's own power-of-two operand scales (two launches).  The operand
 * pointers are bound at plan time.  With out == NULL only *workspace_needed is
 * set.  Errors: UNSUPPORTED for opt->odd = PEEL or opt->algo = CLASSICAL. */
typedef struct fmm_batched_s* fmm_batched_t;
fmm_status_t fmm_batched_plan(fmm_batched_t* out, int count, const int64_t* M, const int64_t* N,
                              const int64_t* K, const float* const* A, const int64_t* lda,
                              const float* const* B, const int64_t* ldb, float* const* C,
                              const int64_t* ldc, const float* alpha, const float* beta,
                              const fmm_options_t* opt, void* workspace, size_t workspace_bytes,
                              size_t* workspace_needed, fmm_stream_t stream);
fmm_status_t fmm_batched_run(fmm_batched_t plan, fmm_stream_t stream);
void fmm_batched_free(fmm_batched_t plan);
/* depths: `count` ints (-1 for problems with no product to compute); any
 * pointer may be NULL.  launches: kernels launched by all runs so far. */
fmm_status_t fmm_batched_info(fmm_batched_t plan, int* depths, int64_t* total_tiles, int64_t* launches);
/* classes: `count` ints, each problem's size class index (0 .. *nclasses - 1,
 * -1 for problems with no product); *leaf_tile: the launch's leaf tile (512 =
 * CTA pairs).  Any pointer may be NULL. */
fmm_status_t fmm_batched_classes(fmm_batched_t plan, int* classes, int* nclasses, int* leaf_tile);

/* Release a plan (NULL-safe).  Never frees the caller's workspace. */
void fmm_free(fmm_plan_t plan);

/* Static string naming a status code. */
const char* fmm_status_string(fmm_status_t s);

/* Text of the last CUDA error seen by this thread's calls (static storage). */
const char* fmm_last_error(void);

/* Synchronise the plan's last stream and read its device status word:
 * FMM_OK, or FMM_ERR_TIMEOUT when a kernel's bounded wait ran out.  The word
 * is cleared by the read. */
fmm_status_t fmm_get_device_status(fmm_plan_t plan);

/* Algorithmic bytes of the plan's last call (device-operand plans; 0 for
 * host-resident ones): every read and write the addition passes need, counted
 * once, without cache or padding effects.  pre_bytes covers the passes before
 * the leaf launch (FP16X3 operand scales, operand splits into hi / lo planes,
 * transposes, the S / T pre-additions of the Winograd recursion); post_bytes
 * the passes after it (the U post-additions, alpha / beta into C, and for peeled
 * plans the border's operand copies).  Dividing by the phase times of
 * fmm_plan_profile_read gives the addition kernels' achieved HBM bandwidth.
 * Either pointer may be NULL. */
fmm_status_t fmm_plan_phase_bytes(fmm_plan_t plan, double* pre_bytes, double* post_bytes);

/* Failure-path self-test of the device waits.  Launches one block on `stream`
 * whose thread waits, with the bounded wait every kernel pipeline of the
 * library uses but a limit of limit_ns (1e6 .. 1e10 ns), on a barrier that
 * nothing signals.  The wait runs out, sets the timeout bit of the plan's
 * device status word and the kernel returns, so the context stays usable:
 * fmm_get_device_status then reports FMM_ERR_TIMEOUT (and clears the word).
 * FMM_ERR_INVALID_ARG for a NULL plan or a limit out of range.  Asynchronous. */
fmm_status_t fmm_wait_selftest(fmm_plan_t plan, int64_t limit_ns, fmm_stream_t stream);

/* Plan inspection: depth, leaf tile width, precision and odd mode the plan
 * uses (after the planner ran); any pointer may be NULL. */
fmm_status_t fmm_plan_info(fmm_plan_t plan, int* depth, int* leaf_tile, int* precision,
                           int* odd, int* algo);

/* Whether the plan's leaf launches fold the last Winograd level into the node
 * outputs (fmm_options_t.fuse_last after the planner ran; for host-resident
 * plans, their device-resident child plan): *fused = 1 or 0. */
fmm_status_t fmm_plan_fuse_last(fmm_plan_t plan, int* fused);

/* How a host-resident plan moves its next call's operands: *mode = 1 (copy
 * engines) or 2 (SM loads and stores); 0 for device-resident plans.  Under the
 * library default (fmm_options_t.host_copy = 0) the answer turns from 1 to 2
 * once a call's input transfers ran at under half of the host link's rate
 * (judged at the following call, from calls moving at least 64 MiB in). */
fmm_status_t fmm_plan_host_copy(fmm_plan_t plan, int* mode);

/* Freivalds residual of a computed product: r = C x - A (B x) for a probe
 * vector x (N entries, device; +-1 entries make a single wrong C entry show up
 * exactly in r).  A (M x K), B (K x N), C (M x N) row-major device matrices;
 * r: M doubles (device).  fp64 = 0 accumulates in fp32, fp64 = 1 in float64
 * (the optional one-step fp64 refinement of the residual).  workspace: device
 * memory of *workspace_needed bytes (K + M doubles); with workspace and r both
 * NULL only *workspace_needed is set.  Asynchronous; one pass over A, B, C. */
fmm_status_t fmm_residual(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda,
                          const float* B, int64_t ldb, const float* C, int64_t ldc,
                          const float* x, double* r, void* workspace, size_t workspace_bytes,
                          size_t* workspace_needed, int fp64, fmm_stream_t stream);

/* ---------------------------------------------------------------- planner
 * Candidate plans of a problem: depth 0..4 (a level only while every leaf
 * dimension stays >= 128) x leaf tile {128, 256, 512} (512 only for leaves
 * of at least 256 x 256), restricted by
 * opt->depth / opt->leaf_tile when those are set.  The paper's fixed
 * thresholds (Table 2, the recursion point of Sec. 3.1) never ask whether one
 * more split would pay on the machine at hand; these planners measure or
 * predict it.
 *
 * fmm_autotune times every candidate on the caller's device buffers A, B, C
 * (C is overwritten) with CUDA events on `stream` (1 warm-up + reps timed
 * runs, median) and synchronises.  depths/tiles/times_ms receive up to 16
 * entries, *count their number; any may be NULL.  workspace: at least
 * *workspace_needed bytes (the largest candidate); with workspace == NULL
 * only *workspace_needed is set. */
fmm_status_t fmm_autotune(int64_t M, int64_t N, int64_t K, const fmm_options_t* opt,
                          const float* A, const float* B, float* C,
                          void* workspace, size_t workspace_bytes, size_t* workspace_needed,
                          int* depths, int* tiles, float* times_ms, int* count, int reps,
                          fmm_stream_t stream);

/* Cost-model network used by FMM_PLANNER_MLP: 6 -> 64 -> 64 -> 1, ReLU, fp32,
 * FMM_MLP_NPARAM parameters laid out W1[64][6], b1[64], W2[64][64], b2[64],
 * W3[1][64], b3[1] (weights row-major [out][in]).  Input features of a
 * candidate (see fmm_plan_features) are standardised with the given mean and
 * std (6 floats each); the output predicts log(milliseconds). */
#define FMM_MLP_NPARAM 4673

/* Raw features of a candidate: log2 M, log2 K, log2 N, depth, leaf_tile/128,
 * precision id.  Host only. */
fmm_status_t fmm_plan_features(int64_t M, int64_t N, int64_t K, int depth, int leaf_tile, int precision,
                               float* out6);

/* Network inference: Y[i] = f(X[i, 0:6]) for `batch` standardised feature
 * rows.  params, X, Y: device pointers.  Asynchronous, one launch. */
fmm_status_t fmm_mlp_forward(const float* params, const float* X, float* Y, int batch, fmm_stream_t stream);

/* One full-batch training step of 0.5 * mean((f(X) - T)^2) with Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected; `step` counts from 1;
 * lr == 0 computes gradients without updating).  params, adam_m, adam_v:
 * FMM_MLP_NPARAM device floats each, updated in place.  grad_out (nullable,
 * FMM_MLP_NPARAM device floats) receives the gradient; loss_out (nullable,
 * one device float) the loss before the update.  workspace: device memory,
 * *workspace_needed bytes (activations of the batch); with workspace and
 * params NULL only the size is returned.  Deterministic summation order. */
fmm_status_t fmm_mlp_train_step(float* params, float* adam_m, float* adam_v, int step, float lr,
                                const float* X, const float* T, int batch,
                                void* workspace, size_t workspace_bytes, size_t* workspace_needed,
                                float* grad_out, float* loss_out, fmm_stream_t stream);

/* Register the cost model for FMM_PLANNER_MLP (host pointers, copied).  The
 * parameters are uploaded to each device on first use.  params == NULL
 * unregisters; without a model FMM_PLANNER_MLP falls back to the exhaustive
 * autotuner. */
fmm_status_t fmm_set_cost_model(const float* params, const float* mean6, const float* std6);

/* Allocation-free variant of fmm_gemm.  The paper has no counterpart; this is
 * a deployment convenience for callers that cannot allocate device memory when
 * they multiply: a host runtime whose device memory is reserved up front by
 * another allocator (so a cudaMalloc would fail or break its accounting),
 * embeddings that hand this library no allocator and no workspace, and
 * latency-bound paths that must not pay for an allocation or a
 * synchronising free.
 *
 * Computes C <- alpha * A * B + beta * C (row-major device pointers, the same
 * conventions as fmm_gemm) with one Winograd level over 3xTF32 tensor-core
 * leaves.  Its temporaries live in a device array of 22,020,352 bytes compiled
 * into the library (held by every GPU that loads it until the process exits),
 * so M, N and K must each be <= 1024; larger sizes return FMM_ERR_INVALID_ARG
 * with the limit in fmm_last_error().  The call allocates nothing (no
 * cudaMalloc/cudaFree, no host heap, no allocating library routine).  The
 * first call on a device looks up the array's device address (once per device,
 * with that device current); make that first call before any stream capture.
 * Every call clears the status word it uses, so fmm_gemm_static_status reports
 * on the last call.  All calls share the one array, which keeps the last
 * call's contents: calls that overlap on the GPU (different streams, or
 * different threads on the same device) race and must be serialised by the
 * caller. */
fmm_status_t fmm_gemm_static(int64_t M, int64_t N, int64_t K, float alpha, const float* A, int64_t lda,
                             const float* B, int64_t ldb, float beta, float* C, int64_t ldc,
                             fmm_stream_t stream);

/* Device status of the last fmm_gemm_static call on the current device:
 * synchronises `stream` (the stream of that call), reads the status word in
 * the library's fixed array and clears it.  FMM_OK, FMM_ERR_TIMEOUT when one
 * of the call's bounded device waits ran out (C is then incomplete), or
 * FMM_ERR_CUDA for any other device-side error bit.  Allocates nothing. */
fmm_status_t fmm_gemm_static_status(fmm_stream_t stream);

/* Measurement helper, not part of the method: the tensor-pipe rate of this
 * GPU, the ceiling the leaf launches are measured against.  Launches, on
 * `stream`, one CTA pair per two SMs that issues tcgen05.mma back to back on
 * operand tiles held in shared memory, in the leaf kernel's instruction shape
 * (cta_group::2, M = 256, N = 256, K-major operands with 128-byte swizzle):
 * kind = 0 kind::tf32 (K = 8 per instruction), kind = 1 kind::f16 on bf16
 * operands (K = 16).  Each pair issues batches x 64 instructions, at most two
 * batches queued.  fill: device buffer of at least 16384 floats (16-byte
 * aligned) copied into every CTA's tiles (use random values: the tensor core's
 * power draw, hence its clock under the power cap, depends on them).  One
 * untimed launch, then one launch timed with CUDA events; synchronises.
 * *tflops = 2 * 256 * 256 * K * 64 * batches * pairs / time; *ms (nullable) the
 * timed launch.  Errors: INVALID_ARG (kind, batches outside 1 .. 2^24, NULL),
 * ALIGNMENT, NO_DEVICE, CUDA, TIMEOUT (a bounded wait ran out). */
fmm_status_t fmm_tensor_peak(int kind, int64_t batches, const float* fill, double* tflops, double* ms,
                             fmm_stream_t stream);

/* Phase profiling.  fmm_plan_profile(plan, 1) resets the counters and makes
 * every later fmm_gemm on the plan record CUDA events (on the call's stream)
 * around three phases: pre-additions (plus operand copies), the leaf launch,
 * and post-additions.  fmm_plan_profile_read synchronises on the recorded
 * events and returns the summed milliseconds per phase, the number of kernel
 * launches the library made and the number of calls since the reset (any
 * pointer may be NULL).  Profiling adds no device work beyond event records. */
fmm_status_t fmm_plan_profile(fmm_plan_t plan, int enable);
fmm_status_t fmm_plan_profile_read(fmm_plan_t plan, double* pre_ms, double* leaf_ms, double* post_ms,
                                   int64_t* launches, int64_t* calls);

#ifdef __cplusplus
}
#endif
#endif /* FMM_GB300_H */
