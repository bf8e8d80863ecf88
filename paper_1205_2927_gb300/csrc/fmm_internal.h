// fmm_internal.h -- structures shared by the host scheduler and the kernels.
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace fmm {

constexpr unsigned FMM_DEV_TIMEOUT_BIT = 1u;  // device status word: a bounded wait ran out
constexpr unsigned FMM_DEV_BADDESC_BIT = 2u;  // device status word: inconsistent descriptor
constexpr int kMaxMaps = 16;
constexpr int kMaxGroups = 8;
constexpr int kBM = 128;  // leaf tile rows (one TMEM lane per row)
constexpr int kBK = 32;   // fp32 elements per 128-byte swizzled row

// One group of leaf products: `batch` independent C_b = alpha * A_b * B_b^T
// (+ beta * C_b) sharing sizes.  A_b is M x K (K-major), B_b is N x K
// (K-major, i.e. the transposed right operand), read through 3-D tensor maps
// whose third coordinate is the batch index (plus an offset).
struct GemmGroup {
    int M, N, K;
    int batch;
    int tiles_m, tiles_n;
    long long tile_begin;   // first linear tile index of this group
    float* C;
    long long ldc;
    long long c_batch_stride;
    float alpha, beta;
    int map_a, map_b;       // tensor-map indices
    int a_batch_off, b_batch_off;
    int vec_ok;             // C, ldc and the batch stride allow 16-byte stores
    int pad_;
    const float* scale;     // 16-bit split leaves: device {s_a, s_b} power-of-two operand scales, or null
    int map_a_lo, map_b_lo; // pre-split 16-bit leaves: maps of the lo planes (map_a / map_b hold hi)
};

struct GemmArgs {
    CUtensorMap maps[kMaxMaps];    // used when ext_maps == nullptr
    GemmGroup groups[kMaxGroups];  // used when ext_groups == nullptr
    const CUtensorMap* ext_maps;   // device-memory tables (batched launches)
    const GemmGroup* ext_groups;
    int num_groups;
    int raster_m;                  // tile rows per raster band
    long long total_tiles;
    unsigned* status;              // device status word
    // dynamic tile order of a leaf launch (null: static round robin): the next
    // free tile (zero before the launch), and one ring per CTA (per pair for
    // CTA-pair launches) of kPairSeqSlots 64-bit slots ((index + 1) << 32 | tile;
    // zero before the launch)
    int* tile_counter;
    unsigned long long* tile_seq;
    // fused last Winograd level (CTA-pair launches): per-CTA running tiles, two
    // of 128 x 256 floats per CTA (kFuseBytesPerPair per pair), or null
    float* fuse_scratch;
};
constexpr int kFuseMaxPairs = 128;    // pairs a fused launch may use
constexpr size_t kFuseBytesPerPair = 2 * 2 * 128 * 256 * sizeof(float);
constexpr int kPairSeqSlots = 64;     // ring slots per CTA / pair (its roles stay within ~10 tiles)
constexpr int kMaxSeqRings = 256;     // CTAs / pairs a dynamically scheduled launch may use
constexpr size_t kTileSchedBytes = 256 + (size_t)kMaxSeqRings * kPairSeqSlots * 8;   // counter, then the rings

// precision of a leaf launch
// kLeafBF16x3 / kLeafFP16x3 split fp32 tiles in shared memory; the *P modes
// read operands already split into 16-bit hi / lo planes in global memory.
enum LeafMode : int { kLeafTF32 = 0, kLeaf3xTF32 = 1, kLeafBF16x3 = 2, kLeafFP16x3 = 3, kLeafBF16x3P = 4,
                      kLeafFP16x3P = 5, kLeaf3xTF32P = 6 };

// Launch the persistent tensor-core leaf kernel.  Returns a cudaError_t.
cudaError_t launch_leaf_gemm(const GemmArgs& args, int mode, int bn, int num_sms, cudaStream_t stream);
size_t leaf_smem_bytes(int mode, int bn);
// CTA-pair variant (pre-split modes only): 256 x 256 tiles (group tiles_m /
// tiles_n must be counted in 256-row / 256-column units, B maps with 128-row
// boxes).
cudaError_t launch_leaf_gemm_pair(const GemmArgs& args, int mode, int num_sms, cudaStream_t stream);
// One bounded wait on a barrier nothing signals: sets the timeout bit of *status
// after limit_ns and returns (the failure path of every pipeline wait).
cudaError_t launch_wait_selftest(unsigned* status, unsigned long long limit_ns, cudaStream_t stream);

// ------------------------------------------------------------ additions
// A matrix operand view: `nodes` matrices of rows x cols, node i at
// ptr + i * node_stride, row stride ld (elements).  Reads outside
// valid_rows x valid_cols are zero (virtual padding of the root).
struct View {
    const float* ptr;
    long long ld;
    long long node_stride;
    long long rows, cols;
    long long valid_rows, valid_cols;
};
// Output stack of children: child c of node p is at
// ptr + (p * nchild + c) * child_stride, row stride ld.
struct Stack {
    float* ptr;
    long long ld;
    long long child_stride;
    int nchild;
};

// Pre-additions of one level, A side (S1..S4) or transposed-B side (T1..T4
// transposed).  full = 1 writes all 7 child operands (quadrant copies
// included); full = 0 writes only the 4 sums.
cudaError_t launch_pre_add(const View& parent, long long nodes, const Stack& out, int side_b, int full,
                           cudaStream_t stream);
// Root B side: reads row-major B (K x N) and writes transposed children.
cudaError_t launch_pre_add_b_root(const float* B, long long ldb, long long K, long long N, long long kh,
                                  long long nh, const Stack& out, int full, cudaStream_t stream);
// Post-additions of one level: children outputs (stack of 7 per node, each h x w,
// row stride ld_in) -> node outputs (2h x 2w).  At the root: C = alpha*U + beta*C
// restricted to valid rows/cols.
cudaError_t launch_post_add(const float* P, long long ld_in, long long child_stride, long long nodes, long long h,
                            long long w, float* out, long long ld_out, long long out_node_stride,
                            long long valid_rows, long long valid_cols, float alpha, float beta,
                            cudaStream_t stream);
// Transposed copy: B (K x N, ldb) -> Bt (N x K, ldt).  With rows_out x cols_out
// given (>= N x K), the whole padded extent is written, zeros outside N x K.
cudaError_t launch_transpose(const float* B, long long ldb, long long K, long long N, float* Bt, long long ldt,
                             cudaStream_t stream, long long rows_out = -1, long long cols_out = -1);
// Plain copy of an M x K matrix into a buffer with another leading dimension.
cudaError_t launch_copy2d(const float* A, long long lda, long long M, long long K, float* dst, long long ldd,
                          cudaStream_t stream);
// Batched copies for many problems in one launch: transpose = 1 writes
// src^T (src: rows x cols, row stride lds) into dst (cols x rows, row stride
// ldd); transpose = 0 copies src into dst with another row stride.  32 x 32
// tiles; tile_begin is the job's first tile in the launch.
struct CopyJob {
    const float* src;
    long long lds;
    long long rows, cols;
    float* dst;
    long long ldd;
    long long tile_begin;
    int tiles_c;
    int transpose;
};
cudaError_t launch_batched_copy(const CopyJob* jobs, int njobs, long long total_tiles, cudaStream_t stream);
// Batched split into planes: like the copy jobs, but `dst` / `lo` are the hi /
// lo planes of split `kind` (SplitKind; no operand scaling) and ldd is the
// planes' row stride in elements.
struct SplitJob {
    const float* src;
    long long lds;
    long long rows, cols;
    void* dst;
    void* lo;
    long long ldd;
    long long tile_begin;   // first 32 x 128 block of the job in the launch
    int tiles_c;            // 128-column blocks per 32-row band of the source
    int transpose;
    const float* scale;     // FP16x3: the problem's device {s_a, s_b} (the job uses scale[transpose]), or null
};
cudaError_t launch_batched_split(const SplitJob* jobs, int njobs, long long total_tiles, int kind,
                                 cudaStream_t stream);
// FP16x3 in a batched launch: the largest |x| of every operand (rows x cols,
// row stride lds) is folded into its problem's slot, one launch over 32 x 128
// blocks of all operands; then every problem's scales {s_a, s_b} from its two
// maxima times its bound (4^depth), by the rule of launch_fp16_scales.
struct AbsJob {
    const float* src;
    long long lds;
    long long rows, cols;
    unsigned* slot;         // float bits of the running maximum (starts at 0)
    long long tile_begin;
    int tiles_c;
};
cudaError_t launch_batched_absmax(const AbsJob* jobs, int njobs, long long total_tiles, cudaStream_t stream);
cudaError_t launch_batched_fp16_scales(const unsigned* maxima, const float* bound, float* scales, int count,
                                       cudaStream_t stream);
// FP16x3 operand scales: scale[0] = 2^e_a, scale[1] = 2^e_b with the largest
// e such that bound_mult * max|X| * 2^e <= 2^14 (1 when X is all zero); the
// maxima are taken over the M x K / K x N operands (any leading dimension).
cudaError_t launch_fp16_scales(const float* A, long long lda, long long M, long long K, const float* B,
                               long long ldb, long long N, float bound_mult, float* scale, unsigned* scratch,
                               cudaStream_t stream);
// Host-streamed root level: quadrant buffers are separate (h x w, row stride
// ld, all multiples of 4 floats, 16-byte aligned).
struct QuadPre {
    const float* in[4];   // Q0..Q3
    float* out[4];        // the four sums, in order 1..4
    long long ld, h, w;
};
struct QuadPost {
    const float* p[7];    // P1..P7
    float* c[4];          // C11, C12, C21, C22 quadrant buffers
    long long ld, h, w;
    float alpha, beta;
};
cudaError_t launch_quad_pre(const QuadPre& q, int side_b, cudaStream_t stream);
cudaError_t launch_quad_post(const QuadPost& q, int part, cudaStream_t stream);
// ------------------------------------------------------------ split hi/lo planes
// Kinds of split: bf16 (x*s = hi + lo, 16-bit), fp16 (same, 16-bit), tf32
// (fp32 planes: hi = x itself -- the tensor core reads trunc_tf32(x) -- and
// lo = rn_tf32(x - trunc_tf32(x))).
enum SplitKind : int { kSplitBF16 = 0, kSplitFP16 = 1, kSplitTF32 = 2 };
// A stack of split matrices: child c of node p at plane + (p * nchild + c) *
// child_stride elements, row stride ld (elements, multiple of 8 so rows start
// on 16 bytes); element size 2 (bf16, fp16) or 4 (tf32).
struct Stack16 {
    void* hi;
    void* lo;
    long long ld;
    long long child_stride;
    int nchild;
};
// Pre-additions of one level writing all 7 children as split 16-bit planes
// (the last level of a split-precision plan); scale = device {s_a, s_b} or null.
cudaError_t launch_pre_add16(const View& parent, long long nodes, const Stack16& out, int side_b, int kind,
                             const float* scale, cudaStream_t stream);
cudaError_t launch_pre_add16_b_root(const float* B, long long ldb, long long K, long long N, long long kh,
                                    long long nh, const Stack16& out, int kind, const float* scale,
                                    cudaStream_t stream);
// Plain split of an M x K matrix (transpose = 0) or of B^T for a K x N matrix
// B (transpose = 1, rows = K, cols = N) into 16-bit planes; which = 0 uses
// scale[0], 1 uses scale[1].
cudaError_t launch_split16(const float* X, long long ldx, long long rows, long long cols, const Stack16& out,
                           int transpose, int kind, const float* scale, int which, cudaStream_t stream);
// Two consecutive levels in one pass (middle level never stored; identical
// arithmetic).  pre: node operands (4h x 4w, uniform stack `node`, reads
// outside its valid window are zero) -> the 49 grandchildren as split planes
// (child stride, ld of `out`); w must be a multiple of 4.  post: 49 grandchild
// products per node (h x w, row stride ld_in, child stride) -> node outputs
// (4h x 4w, row stride ld_out, node stride); valid_rows >= 0 marks the root:
// C <- alpha * U + beta * C inside valid_rows x valid_cols.
cudaError_t launch_pre_add2(const View& node, long long nodes, const Stack16& out, int side_b, int kind,
                            const float* scale, cudaStream_t stream);
// Root B side of a depth-2 plan: the caller's row-major B (K x N valid) straight
// into the 49 leaf operands of B^T (h = N0 / 4 rows, w = K0 / 4 columns each).
cudaError_t launch_pre_add2_b_root(const float* B, long long ldb, long long K, long long N, long long h, long long w,
                                   const Stack16& out, int kind, const float* scale, cudaStream_t stream);
// Root B side of a depth-3 plan straight from row-major B (valid K x N) into
// the 343 leaf operands of B^T (h x w each, h a multiple of 4), split planes.
cudaError_t launch_pre_add3_bt(const float* B, long long ldb, long long K, long long N, long long h, long long w,
                               const Stack16& out, int kind, const float* scale, cudaStream_t stream);
// Three levels at once (a depth-3 plan's whole recursion): node operands
// (8h x 8w) -> 343 split leaf operands each; and 343 products per node -> the
// node output (alpha / beta and the valid window at the root, valid_rows >= 0).
cudaError_t launch_pre_add3(const View& node, long long nodes, const Stack16& out, int side_b, int kind,
                            const float* scale, cudaStream_t stream);
cudaError_t launch_post_add3(const float* P, long long ld_in, long long child_stride, long long nodes, long long h,
                             long long w, float* out, long long ld_out, long long out_node_stride,
                             long long valid_rows, long long valid_cols, float alpha, float beta,
                             cudaStream_t stream);
cudaError_t launch_post_add2(const float* P, long long ld_in, long long child_stride, long long nodes, long long h,
                             long long w, float* out, long long ld_out, long long out_node_stride,
                             long long valid_rows, long long valid_cols, float alpha, float beta,
                             cudaStream_t stream);
// Deterministic pseudo-random fill of n floats in [-1, 1) (autotuner scratch).
cudaError_t launch_fill(float* p, size_t n, unsigned seed, cudaStream_t stream);
// Cost-model inference (mlp.cu): Y = f(X), `batch` rows of 6 features.
cudaError_t mlp_forward(const float* params, const float* X, float* Y, int batch, cudaStream_t s);
// C <- beta * C (beta == 0 writes zeros).
cudaError_t launch_scale(float* C, long long ldc, long long M, long long N, float beta, cudaStream_t stream);
// rows x cols block copy by SM loads/stores; either side may be the device
// mapping of pinned host memory (row strides lds, ldd in elements)
cudaError_t launch_host_copy2d(const float* src, long long lds, float* dst, long long ldd, long long rows,
                               long long cols, cudaStream_t stream);

}  // namespace fmm
