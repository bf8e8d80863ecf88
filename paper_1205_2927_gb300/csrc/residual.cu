// residual.cu -- Freivalds residual r = C x - A (B x) of a computed product.
//
// Three row-times-vector passes, each one block per matrix row with coalesced
// reads along the row: y = B x (K entries), z = A y (M), w = C x (M), r = w - z.
// Accumulation in fp32, or in fp64 for the optional refinement (O(mn + mk + kn)
// fp64 operations: at n = 16384 the fp64 pipe, not HBM, sets its time).  One
// pass over A, B and C: bandwidth-bound in fp32.
#include "../../include/fmm.h"
#include "fmm_internal.h"

#include <cstdint>
#include <type_traits>

namespace fmm {
namespace {

// One block of 256 threads per row: out[row] = sum_c X[row][c] v[c] (minus
// sub[row]).  When the rows and v are 16-byte aligned, thread t reads columns
// 4g .. 4g + 3 for g = t, t + 256, ... (a block-wide coalesced sweep of the
// row, several 16-byte loads in flight per thread) into four independent
// partial sums; the last cols % 4 columns, or every column of unaligned rows,
// go one at a time.  Warp sums, then the 8 warp sums in a fixed order.  One
// row per block keeps the grid many waves deep (16384 rows: 13.5 waves).
template <typename Acc, typename Vec, typename Out>
__global__ void __launch_bounds__(256) rowdot_kernel(const float* __restrict__ X, long long ld, long long rows,
                                                     long long cols, const Vec* __restrict__ v,
                                                     Out* __restrict__ out, const double* __restrict__ sub,
                                                     int vec4) {
    __shared__ Acc warp_sum[8];
    const long long row = blockIdx.x;
    const int t = threadIdx.x;
    const float* xr = X + row * ld;
    Acc a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    long long c0 = 0;
    if (vec4) {
        const long long groups = cols >> 2;
        const float4* x4 = reinterpret_cast<const float4*>(xr);
#pragma unroll 4
        for (long long g = t; g < groups; g += 256) {
            const float4 xv = __ldg(x4 + g);
            Acc v0, v1, v2, v3;
            if constexpr (std::is_same<Vec, float>::value) {
                const float4 q = __ldg(reinterpret_cast<const float4*>(v) + g);
                v0 = q.x; v1 = q.y; v2 = q.z; v3 = q.w;
            } else {
                const double2 q0 = __ldg(reinterpret_cast<const double2*>(v) + 2 * g);
                const double2 q1 = __ldg(reinterpret_cast<const double2*>(v) + 2 * g + 1);
                v0 = (Acc)q0.x; v1 = (Acc)q0.y; v2 = (Acc)q1.x; v3 = (Acc)q1.y;
            }
            a0 += (Acc)xv.x * v0;
            a1 += (Acc)xv.y * v1;
            a2 += (Acc)xv.z * v2;
            a3 += (Acc)xv.w * v3;
        }
        c0 = groups << 2;
    }
    for (long long c = c0 + t; c < cols; c += 256) a0 += (Acc)xr[c] * (Acc)v[c];
    Acc acc = (a0 + a1) + (a2 + a3);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((t & 31) == 0) warp_sum[t >> 5] = acc;
    __syncthreads();
    if (t == 0) {
        Acc s = warp_sum[0];
#pragma unroll
        for (int w = 1; w < 8; ++w) s += warp_sum[w];
        if (sub) out[row] = (Out)((double)s - sub[row]);
        else out[row] = (Out)s;
    }
}

inline int aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0 ? 1 : 0; }

// y = B x ; z = A y ; r = C x - z.  y is kept in the accumulation type: an
// fp32 sum is exactly representable either way, and a float y keeps the
// middle pass off the FP64 pipe (a double-to-float conversion per element).
template <typename Acc>
cudaError_t residual_impl(long long M, long long N, long long K, const float* A, long long lda, const float* B,
                          long long ldb, const float* C, long long ldc, const float* x, double* r, double* y_ws,
                          double* z, cudaStream_t s) {
    Acc* y = reinterpret_cast<Acc*>(y_ws);   // K entries (the workspace holds K doubles)
    const int vx = aligned16(x), vy = aligned16(y);
    if (K > 0)
        rowdot_kernel<Acc, float, Acc><<<(unsigned)K, 256, 0, s>>>(B, ldb, K, N, x, y, nullptr,
                                                                   vx & aligned16(B) & (ldb % 4 == 0));
    rowdot_kernel<Acc, Acc, double><<<(unsigned)M, 256, 0, s>>>(A, lda, M, K, y, z, nullptr,
                                                                vy & aligned16(A) & (lda % 4 == 0));
    rowdot_kernel<Acc, float, double><<<(unsigned)M, 256, 0, s>>>(C, ldc, M, N, x, r, z,
                                                                  vx & aligned16(C) & (ldc % 4 == 0));
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
