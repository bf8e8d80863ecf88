// residual.cu -- Freivalds residual r = C x - A (B x) of a computed product.
//
// Three row-times-vector passes, each one warp per matrix row with coalesced
// reads along the row: y = B x (K entries), z = A y (M), w = C x (M), r = w - z.
// Accumulation in fp32, or in fp64 for the optional refinement (O(mn + mk + kn)
// fp64 operations, cheap despite the low fp64 rate).  One pass over A, B and C:
// bandwidth-bound.
#include "../../include/fmm.h"
#include "fmm_internal.h"

namespace fmm {
namespace {

template <typename Acc, typename Vec>
__global__ void __launch_bounds__(256) rowdot_kernel(const float* __restrict__ X, long long ld, long long rows,
                                                     long long cols, const Vec* __restrict__ v,
                                                     double* __restrict__ out, const double* __restrict__ sub) {
    const long long row = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= rows) return;
    const float* xr = X + row * ld;
    Acc acc = 0;
    for (long long c = lane; c < cols; c += 32) acc += (Acc)xr[c] * (Acc)v[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[row] = sub ? (double)acc - sub[row] : (double)acc;
}

template <typename Acc>
cudaError_t residual_impl(long long M, long long N, long long K, const float* A, long long lda, const float* B,
                          long long ldb, const float* C, long long ldc, const float* x, double* r, double* y,
                          double* z, cudaStream_t s) {
    // y = B x ; z = A y ; r = C x - z
    if (K > 0) rowdot_kernel<Acc, float><<<(unsigned)((K + 7) / 8), 256, 0, s>>>(B, ldb, K, N, x, y, nullptr);
    rowdot_kernel<Acc, double><<<(unsigned)((M + 7) / 8), 256, 0, s>>>(A, lda, M, K, y, z, nullptr);
    rowdot_kernel<Acc, float><<<(unsigned)((M + 7) / 8), 256, 0, s>>>(C, ldc, M, N, x, r, z);
    return cudaGetLastError();
}

}  // namespace
}  // namespace fmm

extern "C" fmm_status_t fmm_residual(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda, const float* B,
                                     int64_t ldb, const float* C, int64_t ldc, const float* x, double* r,
                                     void* workspace, size_t workspace_bytes, size_t* workspace_needed, int fp64,
                                     fmm_stream_t stream) {
    if (M < 0 || N < 0 || K < 0) return FMM_ERR_INVALID_ARG;
    if (lda < (K > 0 ? K : 1) || ldb < (N > 0 ? N : 1) || ldc < (N > 0 ? N : 1)) return FMM_ERR_INVALID_ARG;
    const size_t need = ((size_t)(K > 0 ? K : 1) + (size_t)(M > 0 ? M : 1)) * sizeof(double) + 256;
    if (workspace_needed) *workspace_needed = need;
    if (!workspace && !r) return FMM_OK;  // size query
    if (M == 0) return FMM_OK;
    if (!A || !B || !C || !x || !r) return FMM_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < need) return FMM_ERR_WORKSPACE;
    double* y = static_cast<double*>(workspace);
    double* z = y + (K > 0 ? K : 1);
    cudaError_t e = fp64 ? fmm::residual_impl<double>(M, N, K, A, lda, B, ldb, C, ldc, x, r, y, z, (cudaStream_t)stream)
                         : fmm::residual_impl<float>(M, N, K, A, lda, B, ldb, C, ldc, x, r, y, z, (cudaStream_t)stream);
    return e == cudaSuccess ? FMM_OK : FMM_ERR_CUDA;
}
