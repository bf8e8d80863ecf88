// addsub.cu -- bandwidth-bound kernels of the recursion: the 8 pre-additions
// (S1..S4 on A, T1..T4 on B) and the 7 post-additions (U1..U7) of Winograd's
// variant of Strassen's algorithm, plus the copies the leaves need (transposed
// right operand, aligned left operand) and C <- beta*C.
//
// Quadrant naming follows Eq. 1: Q0 = X11 (top-left), Q1 = X12, Q2 = X21,
// Q3 = X22.  The right operand is kept transposed (Y = B^T, K-major) below the
// root, so B11 = Y11^T, B12 = Y21^T, B21 = Y12^T, B22 = Y22^T and
//   T1^T = Y21 - Y11,  T2^T = Y22 - T1^T,  T3^T = Y22 - Y21,  T4^T = T2^T - Y12.
// Child order (one child per product P1..P7):
//   A side: Q0, Q1, S4, Q3, S1, S2, S3        (sums only: S1, S2, S3, S4)
//   B side: Y0, Y1, Y3, T4, T1, T2, T3        (sums only: T1, T2, T3, T4)
// All streaming kernels move 16-byte vectors when the view allows it.
#include "fmm_internal.h"
#include "ptx.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace fmm {

namespace {

__device__ __forceinline__ float4 f4(float a, float b, float c, float d) { return make_float4(a, b, c, d); }
__device__ __forceinline__ float4 add4(float4 a, float4 b) { return f4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); }
__device__ __forceinline__ float4 sub4(float4 a, float4 b) { return f4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w); }

// 4 consecutive elements (r, c..c+3) of quadrant q of node view `base`,
// zero outside valid rows/cols.
template <bool VEC>
__device__ __forceinline__ float4 load_q(const View& v, const float* base, long long r, long long c) {
    if (VEC) {
        if (r < v.valid_rows && c + 3 < v.valid_cols) return __ldg(reinterpret_cast<const float4*>(base + r * v.ld + c));
    }
    float t[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) t[j] = (r < v.valid_rows && c + j < v.valid_cols) ? __ldg(base + r * v.ld + c + j) : 0.0f;
    return f4(t[0], t[1], t[2], t[3]);
}

__device__ __forceinline__ void store4(float* p, float4 v, bool vec, long long nvalid) {
    if (vec && nvalid >= 4) { *reinterpret_cast<float4*>(p) = v; return; }
    if (nvalid > 0) p[0] = v.x;
    if (nvalid > 1) p[1] = v.y;
    if (nvalid > 2) p[2] = v.z;
    if (nvalid > 3) p[3] = v.w;
}

// grid: x over column groups of 4, y over rows (strided), z over nodes.
template <bool VEC, int SIDE_B, bool FULL>
__global__ void __launch_bounds__(128) pre_add_kernel(View P, long long h, long long w, Stack out) {
    const long long c = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (c >= w) return;
    const long long node = blockIdx.z;
    const float* base = P.ptr + node * P.node_stride;
    const float* q1p = base + w;
    const float* q2p = base + h * P.ld;
    const float* q3p = q2p + w;
    // quadrant views share the node's validity window, shifted
    View v0 = P, v1 = P, v2 = P, v3 = P;
    v1.valid_cols = P.valid_cols - w;
    v2.valid_rows = P.valid_rows - h;
    v3.valid_rows = P.valid_rows - h;
    v3.valid_cols = P.valid_cols - w;
    const long long nvalid = w - c;
    for (long long r = blockIdx.y; r < h; r += gridDim.y) {
        const float4 Q0 = load_q<VEC>(v0, base, r, c);
        const float4 Q1 = load_q<VEC>(v1, q1p, r, c);
        const float4 Q2 = load_q<VEC>(v2, q2p, r, c);
        const float4 Q3 = load_q<VEC>(v3, q3p, r, c);
        float4 X1, X2, X3, X4;  // S1..S4 or T1^T..T4^T
        if (!SIDE_B) {
            X1 = add4(Q2, Q3);   // S1 = A21 + A22
            X2 = sub4(X1, Q0);   // S2 = S1 - A11
            X3 = sub4(Q0, Q2);   // S3 = A11 - A21
            X4 = sub4(Q1, X2);   // S4 = A12 - S2
        } else {
            X1 = sub4(Q2, Q0);   // T1^T = Y21 - Y11  (B12 - B11)
            X2 = sub4(Q3, X1);   // T2^T = Y22 - T1^T (B22 - T1)
            X3 = sub4(Q3, Q2);   // T3^T = Y22 - Y21  (B22 - B12)
            X4 = sub4(X2, Q1);   // T4^T = T2^T - Y12 (T2 - B21)
        }
        float* o = out.ptr + (node * out.nchild) * out.child_stride + r * out.ld + c;
        const long long cs = out.child_stride;
        if (FULL) {
            store4(o + 0 * cs, Q0, VEC, nvalid);
            store4(o + 1 * cs, Q1, VEC, nvalid);
            if (!SIDE_B) {
                store4(o + 2 * cs, X4, VEC, nvalid);  // P3 = S4 B22
                store4(o + 3 * cs, Q3, VEC, nvalid);  // P4 = A22 T4
            } else {
                store4(o + 2 * cs, Q3, VEC, nvalid);  // P3: B22
                store4(o + 3 * cs, X4, VEC, nvalid);  // P4: T4
            }
            store4(o + 4 * cs, X1, VEC, nvalid);
            store4(o + 5 * cs, X2, VEC, nvalid);
            store4(o + 6 * cs, X3, VEC, nvalid);
        } else {
            store4(o + 0 * cs, X1, VEC, nvalid);
            store4(o + 1 * cs, X2, VEC, nvalid);
            store4(o + 2 * cs, X3, VEC, nvalid);
            store4(o + 3 * cs, X4, VEC, nvalid);
        }
    }
}

// Root B side: B is K x N row-major (ldb).  Tile of 32 (k) x 32 (n) in the
// half domain; reads the four quadrants coalesced along n, writes the
// transposed children coalesced along k.  blockDim = (32, 8).
template <bool FULL>
__global__ void __launch_bounds__(256) pre_add_b_root_kernel(const float* __restrict__ B, long long ldb, long long K,
                                                             long long N, long long kh, long long nh, Stack out) {
    constexpr int NC = FULL ? 7 : 4;
    __shared__ float tile[NC][32][33];
    const long long k0 = (long long)blockIdx.y * 32, n0 = (long long)blockIdx.x * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int kl = ty + 8 * i;
        const long long k = k0 + kl, n = n0 + tx;
        float b11 = 0.f, b12 = 0.f, b21 = 0.f, b22 = 0.f;
        if (k < kh && n < nh) {
            const long long kk2 = k + kh, nn2 = n + nh;
            if (k < K && n < N) b11 = B[k * ldb + n];
            if (k < K && nn2 < N) b12 = B[k * ldb + nn2];
            if (kk2 < K && n < N) b21 = B[kk2 * ldb + n];
            if (kk2 < K && nn2 < N) b22 = B[kk2 * ldb + nn2];
        }
        const float t1 = b12 - b11;  // T1 = B12 - B11
        const float t2 = b22 - t1;   // T2 = B22 - T1
        const float t3 = b22 - b12;  // T3 = B22 - B12
        const float t4 = t2 - b21;   // T4 = T2 - B21
        if (FULL) {
            tile[0][kl][tx] = b11; tile[1][kl][tx] = b21; tile[2][kl][tx] = b22; tile[3][kl][tx] = t4;
            tile[4][kl][tx] = t1;  tile[5][kl][tx] = t2;  tile[6][kl][tx] = t3;
        } else {
            tile[0][kl][tx] = t1; tile[1][kl][tx] = t2; tile[2][kl][tx] = t3; tile[3][kl][tx] = t4;
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int nl = ty + 8 * i;
        const long long n = n0 + nl, k = k0 + tx;
        if (n < nh && k < kh) {
#pragma unroll
            for (int c = 0; c < NC; ++c) out.ptr[c * out.child_stride + n * out.ld + k] = tile[c][tx][nl];
        }
    }
}

// Post-additions: per node, children P1..P7 (h x w each) -> node output.
template <bool VEC, bool ROOT>
__global__ void __launch_bounds__(128) post_add_kernel(const float* __restrict__ P, long long ld_in, long long cs,
                                                       long long h, long long w, float* out, long long ld_out,
                                                       long long out_ns, long long valid_rows, long long valid_cols,
                                                       float alpha, float beta) {
    const long long c = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (c >= w) return;
    const long long node = blockIdx.z;
    const float* base = P + node * 7 * cs;
    float* o = out + node * out_ns;
    for (long long r = blockIdx.y; r < h; r += gridDim.y) {
        const float* pr = base + r * ld_in + c;
        float4 p[7];
        if (VEC) {
#pragma unroll
            for (int i = 0; i < 7; ++i) p[i] = __ldg(reinterpret_cast<const float4*>(pr + i * cs));
        } else {
#pragma unroll
            for (int i = 0; i < 7; ++i) {
                float t[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) t[j] = (c + j < w) ? __ldg(pr + i * cs + j) : 0.0f;
                p[i] = f4(t[0], t[1], t[2], t[3]);
            }
        }
        const float4 U1 = add4(p[0], p[1]);   // P1 + P2
        const float4 U2 = add4(p[0], p[5]);   // P1 + P6
        const float4 U3 = add4(U2, p[6]);     // U2 + P7
        const float4 U4 = add4(U2, p[4]);     // U2 + P5
        const float4 U5 = add4(U4, p[2]);     // U4 + P3
        const float4 U6 = sub4(U3, p[3]);     // U3 - P4
        const float4 U7 = add4(U3, p[4]);     // U3 + P5
        const float4 quad[4] = {U1, U5, U6, U7};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const long long rr = r + (q >> 1) * h;
            const long long cc = c + (q & 1) * w;
            float4 v = quad[q];
            if (!ROOT) {
                store4(o + rr * ld_out + cc, v, VEC, w - c);
            } else {
                if (rr >= valid_rows || cc >= valid_cols) continue;
                const long long nv = min(min(4LL, w - c), valid_cols - cc);
                float* dst = o + rr * ld_out + cc;
                const bool vec = VEC && nv == 4 && ((reinterpret_cast<uintptr_t>(dst) & 15) == 0);
                if (vec) {
                    float4 r4 = f4(alpha * v.x, alpha * v.y, alpha * v.z, alpha * v.w);
                    if (beta != 0.0f) {
                        const float4 old = *reinterpret_cast<const float4*>(dst);
                        r4.x += beta * old.x; r4.y += beta * old.y; r4.z += beta * old.z; r4.w += beta * old.w;
                    }
                    *reinterpret_cast<float4*>(dst) = r4;
                } else {
                    const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        if (j < nv) {
                            float x = alpha * vv[j];
                            if (beta != 0.0f) x += beta * dst[j];
                            dst[j] = x;
                        }
                    }
                }
            }
        }
    }
}

// Bt (rows_out x cols_out, >= N x K) = B^T, zeros outside the N x K valid part.
__global__ void __launch_bounds__(256) transpose_kernel(const float* __restrict__ B, long long ldb, long long K,
                                                        long long N, float* __restrict__ Bt, long long ldt,
                                                        long long rows_out, long long cols_out) {
    // one 128 (k) x 32 (n) block of B per CTA: 16 loads in flight per thread,
    // then 32 rows of B^T written as 512 contiguous bytes each
    __shared__ float tile[32][129];   // [n][k]
    const long long k0 = (long long)blockIdx.y * 128, n0 = (long long)blockIdx.x * 32;
    const int lane = threadIdx.x, warp = threadIdx.y, tid = warp * 32 + lane;
    float x[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const long long k = k0 + warp + 8 * i, n = n0 + lane;
        x[i] = (k < K && n < N) ? __ldg(B + k * ldb + n) : 0.0f;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) tile[lane][warp + 8 * i] = x[i];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int v = tid + 256 * j;   // row v / 128 of the B^T block, column v % 128
        const long long n = n0 + (v >> 7), k = k0 + (v & 127);
        if (n < rows_out && k < cols_out) Bt[n * ldt + k] = tile[v >> 7][v & 127];
    }
}

__global__ void copy2d_kernel(const float* __restrict__ A, long long lda, long long M, long long K, float* dst,
                              long long ldd) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (long long r = blockIdx.y; r < M; r += gridDim.y)
        if (c < K) dst[r * ldd + c] = A[r * lda + c];
}

__global__ void scale_kernel(float* C, long long ldc, long long M, long long N, float beta) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (long long r = blockIdx.y; r < M; r += gridDim.y)
        if (c < N) C[r * ldc + c] = (beta == 0.0f) ? 0.0f : beta * C[r * ldc + c];
}

__global__ void __launch_bounds__(256) batched_copy_kernel(const CopyJob* __restrict__ jobs, int njobs) {
    __shared__ float tile[32][33];
    const long long t = blockIdx.x;
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
    }
    const CopyJob J = jobs[lo];
    const long long local = t - J.tile_begin;
    const long long r0 = (local / J.tiles_c) * 32, c0 = (local % J.tiles_c) * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    if (!J.transpose) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const long long r = r0 + ty + 8 * i, c = c0 + tx;
            if (r < J.rows && c < J.cols) J.dst[r * J.ldd + c] = J.src[r * J.lds + c];
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const long long r = r0 + ty + 8 * i, c = c0 + tx;
        tile[ty + 8 * i][tx] = (r < J.rows && c < J.cols) ? J.src[r * J.lds + c] : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const long long c = c0 + ty + 8 * i, r = r0 + tx;
        if (c < J.cols && r < J.rows) J.dst[c * J.ldd + r] = tile[tx][ty + 8 * i];
    }
}

__global__ void fill_kernel(float* p, size_t n, unsigned seed) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        unsigned x = (unsigned)i * 2654435761u ^ seed;   // integer hash (xorshift-multiply)
        x ^= x >> 16; x *= 0x7feb352du; x ^= x >> 15; x *= 0x846ca68bu; x ^= x >> 16;
        p[i] = (float)(x >> 8) * (2.0f / 16777216.0f) - 1.0f;
    }
}

// max |x| over a rows x cols matrix, folded into *out (float bits; non-negative
// floats order like unsigned integers)
// max |X| over a rows x cols operand (row stride ld): rows grid-strided over
// blockIdx.y, columns over blockIdx.x; 16-byte loads when the rows allow;
// one atomic per block.
__global__ void __launch_bounds__(256) absmax_kernel(const float* __restrict__ X, long long ld, long long rows,
                                                     long long cols, unsigned* out) {
    __shared__ float warp_max[8];
    const bool vec = (reinterpret_cast<uintptr_t>(X) & 15) == 0 && (ld & 3) == 0;
    const long long step = (long long)gridDim.x * blockDim.x;
    float m = 0.f;
    for (long long r = blockIdx.y; r < rows; r += gridDim.y) {
        const float* xr = X + r * ld;
        if (vec) {
            const long long groups = cols >> 2;
            for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < groups; g += step) {
                const float4 v = __ldg(reinterpret_cast<const float4*>(xr) + g);
                m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
            }
            for (long long c = (groups << 2) + (long long)blockIdx.x * blockDim.x + threadIdx.x; c < cols; c += step)
                m = fmaxf(m, fabsf(__ldg(xr + c)));
        } else {
            for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < cols; c += step)
                m = fmaxf(m, fabsf(__ldg(xr + c)));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) warp_max[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int w = 1; w < 8; ++w) m = fmaxf(m, warp_max[w]);
        atomicMax(out, __float_as_uint(m));
    }
}

// Largest power of two s with m * s <= 2^14 (1 for m = 0 or not finite).
__device__ __forceinline__ float fp16_scale_of(float m) {
    if (!(m > 0.f) || !isfinite(m)) return 1.0f;
    int x;
    frexpf(m, &x);                   // m = f * 2^x, 0.5 <= f < 1
    int e = 14 - x;                  // largest e with m * 2^e <= 2^14
    e = max(-100, min(100, e));
    return ldexpf(1.0f, e);
}

__global__ void fp16_scale_kernel(const unsigned* mx, float bound_mult, float* scale) {
    const int i = threadIdx.x;
    if (i > 1) return;
    scale[i] = fp16_scale_of(__uint_as_float(mx[i]) * bound_mult);
}

// Batched maxima: one 32 x 128 block of one operand per CTA (the job found by
// binary search on its first block); 16-byte loads when the rows allow, every
// load issued before the first compare; one atomic per CTA into the job's slot.
__global__ void __launch_bounds__(256) batched_absmax_kernel(const AbsJob* __restrict__ jobs, int njobs) {
    __shared__ float warp_max[8];
    const long long t = blockIdx.x;
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
    }
    const AbsJob J = jobs[lo];
    const long long local = t - J.tile_begin;
    const long long r0 = (local / J.tiles_c) * 32, c0 = (local % J.tiles_c) * 128;
    const bool vec = (reinterpret_cast<uintptr_t>(J.src) & 15) == 0 && (J.lds & 3) == 0;
    float4 v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int g = threadIdx.x + 256 * j;   // row g / 32 of the block, columns 4 (g % 32) .. + 3
        const long long r = r0 + (g >> 5), c = c0 + 4 * (g & 31);
        v[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r >= J.rows || c >= J.cols) continue;
        const float* src = J.src + r * J.lds + c;
        if (vec && c + 3 < J.cols) {
            v[j] = __ldg(reinterpret_cast<const float4*>(src));
        } else {
            v[j].x = __ldg(src);
            if (c + 1 < J.cols) v[j].y = __ldg(src + 1);
            if (c + 2 < J.cols) v[j].z = __ldg(src + 2);
            if (c + 3 < J.cols) v[j].w = __ldg(src + 3);
        }
    }
    float m = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) m = fmaxf(fmaxf(m, fmaxf(fabsf(v[j].x), fabsf(v[j].y))), fmaxf(fabsf(v[j].z), fabsf(v[j].w)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) warp_max[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int w = 1; w < 8; ++w) m = fmaxf(m, warp_max[w]);
        atomicMax(J.slot, __float_as_uint(m));
    }
}

__global__ void batched_fp16_scale_kernel(const unsigned* __restrict__ maxima, const float* __restrict__ bound,
                                          float* __restrict__ scales, int count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * count) return;
    scales[i] = fp16_scale_of(__uint_as_float(maxima[i]) * bound[i >> 1]);
}

// Root pre-additions of the host-streamed schedule: the four quadrants are
// separate row-major buffers (h x w, row stride ld); writes the four sums.
//   A side: S1 = Q2 + Q3, S2 = S1 - Q0, S3 = Q0 - Q2, S4 = Q1 - S2
//   B side: T1 = Q1 - Q0, T2 = Q3 - T1, T3 = Q3 - Q1, T4 = T2 - Q2
template <int SIDE_B>
__global__ void __launch_bounds__(128) quad_pre_kernel(QuadPre q) {
    const long long c = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (c >= q.w) return;
    for (long long r = blockIdx.y; r < q.h; r += gridDim.y) {
        const long long o = r * q.ld + c;
        const float4 Q0 = *reinterpret_cast<const float4*>(q.in[0] + o);
        const float4 Q1 = *reinterpret_cast<const float4*>(q.in[1] + o);
        const float4 Q2 = *reinterpret_cast<const float4*>(q.in[2] + o);
        const float4 Q3 = *reinterpret_cast<const float4*>(q.in[3] + o);
        float4 X1, X2, X3, X4;
        if (!SIDE_B) {
            X1 = add4(Q2, Q3); X2 = sub4(X1, Q0); X3 = sub4(Q0, Q2); X4 = sub4(Q1, X2);
        } else {
            X1 = sub4(Q1, Q0); X2 = sub4(Q3, X1); X3 = sub4(Q3, Q1); X4 = sub4(X2, Q2);
        }
        *reinterpret_cast<float4*>(q.out[0] + o) = X1;
        *reinterpret_cast<float4*>(q.out[1] + o) = X2;
        *reinterpret_cast<float4*>(q.out[2] + o) = X3;
        *reinterpret_cast<float4*>(q.out[3] + o) = X4;
    }
}

// Root post-additions of the host-streamed schedule from the seven product
// buffers (h x w, row stride ld) into one quadrant buffer of C (same layout),
// with the U-chain's operation order, so each quadrant can be formed (and
// copied out) as soon as its products exist:
//   part 0: C11 = alpha * U1 + beta * C11, U1 = P1 + P2
//   part 1: C12 = alpha * U5 + beta * C12, U5 = ((P1 + P6) + P5) + P3
//   part 2: C21 = alpha * U6 + beta * C21, U6 = ((P1 + P6) + P7) - P4
//   part 3: C22 = alpha * U7 + beta * C22, U7 = ((P1 + P6) + P7) + P5
template <int PART>
__global__ void __launch_bounds__(128) quad_post_kernel(QuadPost q) {
    const long long c = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (c >= q.w) return;
    for (long long r = blockIdx.y; r < q.h; r += gridDim.y) {
        const long long o = r * q.ld + c;
        auto P = [&](int i) { return *reinterpret_cast<const float4*>(q.p[i] + o); };
        auto put = [&](float* dst, float4 u) {
            float4 v = f4(q.alpha * u.x, q.alpha * u.y, q.alpha * u.z, q.alpha * u.w);
            if (q.beta != 0.0f) {
                const float4 old = *reinterpret_cast<const float4*>(dst + o);
                v.x += q.beta * old.x; v.y += q.beta * old.y; v.z += q.beta * old.z; v.w += q.beta * old.w;
            }
            *reinterpret_cast<float4*>(dst + o) = v;
        };
        if (PART == 0) {
            put(q.c[0], add4(P(0), P(1)));
        } else {
            const float4 U2 = add4(P(0), P(5));
            if (PART == 1) {
                put(q.c[1], add4(add4(U2, P(4)), P(2)));   // U5 = U4 + P3, U4 = U2 + P5
            } else {
                const float4 U3 = add4(U2, P(6));
                if (PART == 2) put(q.c[2], sub4(U3, P(3)));   // U6 = U3 - P4
                else put(q.c[3], add4(U3, P(4)));             // U7 = U3 + P5
            }
        }
    }
}

// ---------------------------------------------------------------- 16-bit hi/lo planes
// Split four consecutive values into the planes at element offset o.
//   bf16 / fp16: x * s = hi + lo (+ residual), hi = rn16(x s), lo = rn16(x s - hi)
//   tf32:        hi = x (the tensor core reads trunc_tf32(x)), lo = rn_tf32(x - trunc_tf32(x))
// The planes are written with evict-first (streaming) stores: they are read by
// the leaf launch only after far more data than L2 holds has passed, and they
// must not push out the operand lines a fused pass reads again.
template <int KIND>
__device__ __forceinline__ void split_store(void* hi_plane, void* lo_plane, long long o, float4 v, float sc) {
    if constexpr (KIND == kSplitTF32) {
        float4 l;
        l.x = tf32_round_rne(v.x - tf32_trunc(v.x));
        l.y = tf32_round_rne(v.y - tf32_trunc(v.y));
        l.z = tf32_round_rne(v.z - tf32_trunc(v.z));
        l.w = tf32_round_rne(v.w - tf32_trunc(v.w));
        // no hi plane: the leaves read the raw operand itself (hi = x)
        if (hi_plane) __stcs(reinterpret_cast<float4*>(static_cast<float*>(hi_plane) + o), v);
        __stcs(reinterpret_cast<float4*>(static_cast<float*>(lo_plane) + o), l);
        return;
    }
    uint16_t* hi = static_cast<uint16_t*>(hi_plane) + o;
    uint16_t* lo = static_cast<uint16_t*>(lo_plane) + o;
    const float x0 = v.x * sc, x1 = v.y * sc, x2 = v.z * sc, x3 = v.w * sc;
    uint32_t h01, h23, l01, l23;
    if constexpr (KIND == kSplitBF16) {
        const __nv_bfloat162 a = __floats2bfloat162_rn(x0, x1), b = __floats2bfloat162_rn(x2, x3);
        const float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
        const __nv_bfloat162 c = __floats2bfloat162_rn(x0 - fa.x, x1 - fa.y), d = __floats2bfloat162_rn(x2 - fb.x, x3 - fb.y);
        h01 = *reinterpret_cast<const uint32_t*>(&a); h23 = *reinterpret_cast<const uint32_t*>(&b);
        l01 = *reinterpret_cast<const uint32_t*>(&c); l23 = *reinterpret_cast<const uint32_t*>(&d);
    } else {
        const __half2 a = __floats2half2_rn(x0, x1), b = __floats2half2_rn(x2, x3);
        const float2 fa = __half22float2(a), fb = __half22float2(b);
        const __half2 c = __floats2half2_rn(x0 - fa.x, x1 - fa.y), d = __floats2half2_rn(x2 - fb.x, x3 - fb.y);
        h01 = *reinterpret_cast<const uint32_t*>(&a); h23 = *reinterpret_cast<const uint32_t*>(&b);
        l01 = *reinterpret_cast<const uint32_t*>(&c); l23 = *reinterpret_cast<const uint32_t*>(&d);
    }
    __stcs(reinterpret_cast<uint2*>(hi), make_uint2(h01, h23));
    __stcs(reinterpret_cast<uint2*>(lo), make_uint2(l01, l23));
}

// Same arithmetic as pre_add_kernel (all 7 children), output split into planes.
template <bool VEC, int SIDE_B, int KIND>
__global__ void __launch_bounds__(128) pre_add16_kernel(View P, long long h, long long w, Stack16 out,
                                                        const float* __restrict__ scale) {
    const long long c = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (c >= w) return;
    const float sc = scale ? scale[SIDE_B] : 1.0f;
    const long long node = blockIdx.z;
    const float* base = P.ptr + node * P.node_stride;
    const float* q1p = base + w;
    const float* q2p = base + h * P.ld;
    const float* q3p = q2p + w;
    View v0 = P, v1 = P, v2 = P, v3 = P;
    v1.valid_cols = P.valid_cols - w;
    v2.valid_rows = P.valid_rows - h;
    v3.valid_rows = P.valid_rows - h;
    v3.valid_cols = P.valid_cols - w;
    for (long long r = blockIdx.y; r < h; r += gridDim.y) {
        const float4 Q0 = load_q<VEC>(v0, base, r, c);
        const float4 Q1 = load_q<VEC>(v1, q1p, r, c);
        const float4 Q2 = load_q<VEC>(v2, q2p, r, c);
        const float4 Q3 = load_q<VEC>(v3, q3p, r, c);
        float4 X1, X2, X3, X4;
        if (!SIDE_B) {
            X1 = add4(Q2, Q3); X2 = sub4(X1, Q0); X3 = sub4(Q0, Q2); X4 = sub4(Q1, X2);
        } else {
            X1 = sub4(Q2, Q0); X2 = sub4(Q3, X1); X3 = sub4(Q3, Q2); X4 = sub4(X2, Q1);
        }
        const float4 ch[7] = {Q0, Q1, SIDE_B ? Q3 : X4, SIDE_B ? X4 : Q3, X1, X2, X3};
        const long long o = (node * out.nchild) * out.child_stride + r * out.ld + c;
#pragma unroll
        for (int i = 0; i < 7; ++i) split_store<KIND>(out.hi, out.lo, o + i * out.child_stride, ch[i], sc);
    }
}

// Root B side into 16-bit planes (transposing), children in product order.
template <int KIND>
__global__ void __launch_bounds__(256) pre_add16_b_root_kernel(const float* __restrict__ B, long long ldb, long long K,
                                                               long long N, long long kh, long long nh, Stack16 out,
                                                               const float* __restrict__ scale) {
    __shared__ float tile[7][32][33];
    const float sc = scale ? scale[1] : 1.0f;
    const long long k0 = (long long)blockIdx.y * 32, n0 = (long long)blockIdx.x * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int kl = ty + 8 * i;
        const long long k = k0 + kl, n = n0 + tx;
        float b11 = 0.f, b12 = 0.f, b21 = 0.f, b22 = 0.f;
        if (k < kh && n < nh) {
            const long long kk2 = k + kh, nn2 = n + nh;
            if (k < K && n < N) b11 = B[k * ldb + n];
            if (k < K && nn2 < N) b12 = B[k * ldb + nn2];
            if (kk2 < K && n < N) b21 = B[kk2 * ldb + n];
            if (kk2 < K && nn2 < N) b22 = B[kk2 * ldb + nn2];
        }
        const float t1 = b12 - b11, t2 = b22 - t1, t3 = b22 - b12, t4 = t2 - b21;
        tile[0][kl][tx] = b11; tile[1][kl][tx] = b21; tile[2][kl][tx] = b22; tile[3][kl][tx] = t4;
        tile[4][kl][tx] = t1;  tile[5][kl][tx] = t2;  tile[6][kl][tx] = t3;
    }
    __syncthreads();
    // each thread: 4 consecutive k of one n row, for the 7 children
    const int t = ty * 32 + tx;          // 0..255
    const int nl = t >> 3, kq = (t & 7) * 4;
    const long long n = n0 + nl, k = k0 + kq;
    if (n < nh && k < kh) {
#pragma unroll
        for (int c = 0; c < 7; ++c) {
            const float4 v = make_float4(tile[c][kq][nl], tile[c][kq + 1][nl], tile[c][kq + 2][nl], tile[c][kq + 3][nl]);
            split_store<KIND>(out.hi, out.lo, c * out.child_stride + n * out.ld + k, v, sc);
        }
    }
}

// Plain split (transpose = 0: rows x cols -> rows x ld planes) or transposed
// split (transpose = 1: X is rows(K) x cols(N), planes are cols x ld).  Every
// thread issues all of its loads before its first store.  Plain: one 32 x 128
// block per CTA, 16-byte loads straight to the planes.  Transposed: one
// 128 (row) x 32 (column) block staged in a shared tile, left as 32 plane rows
// of 128 elements (512 contiguous bytes each).
template <int KIND, bool TRANS>
__global__ void __launch_bounds__(256) split16_kernel(const float* __restrict__ X, long long ldx, long long rows,
                                                      long long cols, Stack16 out, const float* __restrict__ scale,
                                                      int which) {
    const float sc = scale ? scale[which] : 1.0f;
    const int lane = threadIdx.x, warp = threadIdx.y, tid = warp * 32 + lane;
    if (!TRANS) {
        const long long r0 = (long long)blockIdx.y * 32, c0 = (long long)blockIdx.x * 128;
        const bool vec = (reinterpret_cast<uintptr_t>(X) & 15) == 0 && (ldx & 3) == 0;
        float4 v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int g = tid + 256 * j;   // row g / 32 of the block, columns 4 (g % 32) .. + 3
            const long long r = r0 + (g >> 5), c = c0 + 4 * (g & 31);
            v[j] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (r >= rows || c >= cols) continue;
            const float* src = X + r * ldx + c;
            if (vec && c + 3 < cols) {
                v[j] = __ldg(reinterpret_cast<const float4*>(src));
            } else {
                v[j].x = __ldg(src);
                if (c + 1 < cols) v[j].y = __ldg(src + 1);
                if (c + 2 < cols) v[j].z = __ldg(src + 2);
                if (c + 3 < cols) v[j].w = __ldg(src + 3);
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int g = tid + 256 * j;
            const long long r = r0 + (g >> 5), c = c0 + 4 * (g & 31);
            // ld is a multiple of 8, so a group of 4 never crosses a row: padding columns get zeros
            if (r < rows && c < cols) split_store<KIND>(out.hi, out.lo, r * out.ld + c, v[j], sc);
        }
        return;
    }
    __shared__ float tile[32][129];   // [column of X][row of X]
    const long long r0 = (long long)blockIdx.y * 128, c0 = (long long)blockIdx.x * 32;
    float x[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const long long r = r0 + warp + 8 * i, c = c0 + lane;
        x[i] = (r < rows && c < cols) ? __ldg(X + r * ldx + c) : 0.0f;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) tile[lane][warp + 8 * i] = x[i];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int g = tid + 256 * j;   // plane row g / 32 (a column of X), 4 consecutive plane columns
        const int a = g >> 5, q = (g & 31) * 4;
        const long long orow = c0 + a, ocol = r0 + q;
        if (orow < cols && ocol < rows) {
            const float4 v = make_float4(tile[a][q], tile[a][q + 1], tile[a][q + 2], tile[a][q + 3]);
            split_store<KIND>(out.hi, out.lo, orow * out.ld + ocol, v, sc);
        }
    }
}

// ---------------------------------------------------------------- two levels at once
// The 7 children of an operand from its 4 quadrants, in product order, with
// the same fp32 operations as pre_add_kernel (A: S1..S4; B^T: T1..T4).
template <int SIDE_B>
__device__ __forceinline__ void children7(const float4 (&Q)[4], float4 (&ch)[7]) {
    float4 X1, X2, X3, X4;
    if (!SIDE_B) {
        X1 = add4(Q[2], Q[3]); X2 = sub4(X1, Q[0]); X3 = sub4(Q[0], Q[2]); X4 = sub4(Q[1], X2);
    } else {
        X1 = sub4(Q[2], Q[0]); X2 = sub4(Q[3], X1); X3 = sub4(Q[3], Q[2]); X4 = sub4(X2, Q[1]);
    }
    ch[0] = Q[0]; ch[1] = Q[1];
    ch[2] = SIDE_B ? Q[3] : X4;
    ch[3] = SIDE_B ? X4 : Q[3];
    ch[4] = X1; ch[5] = X2; ch[6] = X3;
}

// Pre-additions of two consecutive levels in one pass: each node operand
// (4h x 4w, a uniform stack) -> its 49 grandchildren (h x w), written as split
// planes at stack index (node * 7 + i) * 7 + j.  Identical arithmetic to two
// pre_add passes; the middle level is never stored.
// 4 consecutive elements at (row, col) of a view, zero outside its valid window.
template <bool VEC>
__device__ __forceinline__ float4 load_sub(const View& v, const float* base, long long row, long long col) {
    if (VEC && row < v.valid_rows && col + 3 < v.valid_cols)
        return __ldg(reinterpret_cast<const float4*>(base + row * v.ld + col));
    float t[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) t[j] = (row < v.valid_rows && col + j < v.valid_cols) ? __ldg(base + row * v.ld + col + j) : 0.0f;
    return f4(t[0], t[1], t[2], t[3]);
}

template <bool VEC, int SIDE_B, int KIND>
__global__ void __launch_bounds__(128) pre_add2_kernel(View P, long long h, long long w, Stack16 out,
                                                       const float* __restrict__ scale) {
    const long long c = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (c >= w) return;
    const float sc = scale ? scale[SIDE_B] : 1.0f;
    const long long node = blockIdx.z;
    const float* base = P.ptr + node * P.node_stride;
    for (long long r = blockIdx.y; r < h; r += gridDim.y) {
        // sub-block (a, b) of the node: quadrant (a / 2, b / 2), sub-quadrant (a % 2, b % 2)
        float4 X[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b)
                X[a][b] = load_sub<VEC>(P, base, a * h + r, b * w + c);
        // quadrant q of the node, sub-quadrant t: X[(q / 2) * 2 + t / 2][(q % 2) * 2 + t % 2]
        const long long o0 = (node * 49) * out.child_stride + r * out.ld + c;
        float4 C[4][7];   // child i's quadrant t (t = sub-quadrant position)
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const float4 Qt[4] = {X[(t >> 1)][(t & 1)], X[(t >> 1)][2 + (t & 1)], X[2 + (t >> 1)][(t & 1)],
                                  X[2 + (t >> 1)][2 + (t & 1)]};
            float4 ch[7];
            children7<SIDE_B>(Qt, ch);
#pragma unroll
            for (int i = 0; i < 7; ++i) C[t][i] = ch[i];
        }
#pragma unroll
        for (int i = 0; i < 7; ++i) {
            const float4 Qi[4] = {C[0][i], C[1][i], C[2][i], C[3][i]};
            float4 g[7];
            children7<SIDE_B>(Qi, g);
#pragma unroll
            for (int j = 0; j < 7; ++j) split_store<KIND>(out.hi, out.lo, o0 + (i * 7 + j) * out.child_stride, g[j], sc);
        }
    }
}

// Child i (product order) of an operand from its four quadrants, one element at
// a time: the same fp32 operations as children7 computing only that child.
template <int SIDE_B>
__device__ __forceinline__ float child_of1(int i, float Q0, float Q1, float Q2, float Q3) {
    if (!SIDE_B) {
        switch (i) {
            case 0: return Q0;
            case 1: return Q1;
            case 2: return Q1 - ((Q2 + Q3) - Q0);   // S4 = Q1 - S2
            case 3: return Q3;
            case 4: return Q2 + Q3;                 // S1
            case 5: return (Q2 + Q3) - Q0;          // S2 = S1 - Q0
            default: return Q0 - Q2;                // S3
        }
    }
    switch (i) {
        case 0: return Q0;
        case 1: return Q1;
        case 2: return Q3;
        case 3: return (Q3 - (Q2 - Q0)) - Q1;       // T4 = T2 - Q1, T2 = Q3 - T1
        case 4: return Q2 - Q0;                     // T1
        case 5: return Q3 - (Q2 - Q0);              // T2
        default: return Q3 - Q2;                    // T3
    }
}

// One value into the planes at element offset o (evict-first stores).
template <int KIND>
__device__ __forceinline__ void split_store1(void* hi_plane, void* lo_plane, long long o, float v, float sc) {
    if constexpr (KIND == kSplitTF32) {
        __stcs(static_cast<float*>(hi_plane) + o, v);
        __stcs(static_cast<float*>(lo_plane) + o, tf32_round_rne(v - tf32_trunc(v)));
        return;
    }
    const float x = v * sc;
    unsigned short h, l;
    if constexpr (KIND == kSplitBF16) {
        const __nv_bfloat16 a = __float2bfloat16_rn(x);
        const __nv_bfloat16 b = __float2bfloat16_rn(x - __bfloat162float(a));
        h = __bfloat16_as_ushort(a);
        l = __bfloat16_as_ushort(b);
    } else {
        const __half a = __float2half_rn(x);
        const __half b = __float2half_rn(x - __half2float(a));
        h = __half_as_ushort(a);
        l = __half_as_ushort(b);
    }
    __stcs(static_cast<unsigned short*>(hi_plane) + o, h);
    __stcs(static_cast<unsigned short*>(lo_plane) + o, l);
}

// Pre-additions of three consecutive levels in one pass (the whole recursion
// of a depth-3 plan): each node operand (8h x 8w, read through its view with
// zero outside the valid window) -> its 343 great-grandchildren (h x w), split
// planes at stack index node * 343 + (i * 7 + j) * 7 + l.  One element per
// thread: the node's 64 sub-block values are loaded once, level-1 child i's
// 4 x 4 sub-block values are formed from them, then level-2 child j's
// quadrants, then its 7 children; the fp32 operations are those of three
// pre_add passes.
template <int SIDE_B, int KIND>
__global__ void __launch_bounds__(256, 2) pre_add3_kernel(View P, long long h, long long w, Stack16 out,
                                                       const float* __restrict__ scale) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= w) return;
    const float sc = scale ? scale[SIDE_B] : 1.0f;
    const long long node = blockIdx.z;
    const float* base = P.ptr + node * P.node_stride;
    for (long long r = blockIdx.y; r < h; r += gridDim.y) {
        const long long o0 = (node * 343) * out.child_stride + r * out.ld + c;
        float X[8][8];   // sub-block (a, b) of the node
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const long long row = a * h + r, col = b * w + c;
                X[a][b] = (row < P.valid_rows && col < P.valid_cols) ? __ldg(base + row * P.ld + col) : 0.0f;
            }
#pragma unroll 1
        for (int i = 0; i < 7; ++i) {
            float Y[4][4];   // level-1 child i, sub-block (a, b)
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    Y[a][b] = child_of1<SIDE_B>(i, X[a][b], X[a][4 + b], X[4 + a][b], X[4 + a][4 + b]);
#pragma unroll 1
            for (int j = 0; j < 7; ++j) {
                float Cj[4];   // level-2 child (i, j), quadrant t
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    Cj[t] = child_of1<SIDE_B>(j, Y[(t >> 1)][(t & 1)], Y[(t >> 1)][2 + (t & 1)],
                                              Y[2 + (t >> 1)][(t & 1)], Y[2 + (t >> 1)][2 + (t & 1)]);
#pragma unroll
                for (int l = 0; l < 7; ++l)
                    split_store1<KIND>(out.hi, out.lo, o0 + (i * 49 + j * 7 + l) * out.child_stride,
                                       child_of1<SIDE_B>(l, Cj[0], Cj[1], Cj[2], Cj[3]), sc);
            }
        }
    }
}

// Root B side of a depth-3 plan in one pass, straight from the caller's
// row-major B (valid K x N, zero outside) into the 343 leaf operands of B^T,
// split into planes.  Leaf position (n, k) of B^T sub-block (a, b) is
// B[b * w + k][a * h + n] (h = N0 / 8, w = K0 / 8).  A block takes an 8 (n) x
// 32 (k) patch of positions: it stages the 64 sub-block tiles of B that the
// patch needs (32 rows of k by 8 columns of n, one 32-byte sector per row) in
// shared memory, every load issued before the first store; each thread then
// reads its position's 64 values from there (rows padded to 9 floats, so the
// 32 lanes of a warp -- 32 consecutive k -- hit 32 banks) and runs
// pre_add3_kernel's chain, its leaf stores running along k, coalesced.  The
// fp32 operations are those of pre_add3_kernel<1> on a transposed copy.
constexpr int kBtN = 8, kBtK = 32, kBtPitch = 9;
constexpr size_t kBtSmem = (size_t)64 * kBtK * kBtPitch * sizeof(float);   // 73,728 bytes

template <int KIND>
__global__ void __launch_bounds__(256, 2) pre_add3_bt_kernel(const float* __restrict__ B, long long ldb, long long K,
                                                          long long N, long long h, long long w, long long tiles_n,
                                                          Stack16 out, const float* __restrict__ scale) {
    extern __shared__ float bt_tile[];   // [64 sub-blocks][kBtK rows of k][kBtPitch]
    const float sc = scale ? scale[1] : 1.0f;
    const int t = threadIdx.x;
    const long long n0 = (long long)(blockIdx.x % tiles_n) * kBtN, k0 = (long long)(blockIdx.x / tiles_n) * kBtK;
    const bool vec = (reinterpret_cast<uintptr_t>(B) & 15) == 0 && (ldb & 3) == 0;
    // 64 tiles x 32 rows x 2 float4 = 4096 float4, 16 per thread
    float4 v[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int L = t + 256 * j;   // sub-block L / 64 = 8 a + b, row (L % 64) / 2, half L % 2
        const int ab = L >> 6, kr = (L & 63) >> 1, q = L & 1;
        const long long k = k0 + kr, n = n0 + 4 * q;   // h is a multiple of 4: n < h covers n + 3
        const long long row = (ab & 7) * w + k, col = (ab >> 3) * h + n;
        v[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (k < w && n < h && row < K && col < N) {
            const float* src = B + row * ldb + col;
            if (vec && col + 3 < N) {
                v[j] = __ldg(reinterpret_cast<const float4*>(src));
            } else {
                v[j].x = __ldg(src);
                if (col + 1 < N) v[j].y = __ldg(src + 1);
                if (col + 2 < N) v[j].z = __ldg(src + 2);
                if (col + 3 < N) v[j].w = __ldg(src + 3);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int L = t + 256 * j;
        float* d = bt_tile + ((L >> 6) * kBtK + ((L & 63) >> 1)) * kBtPitch + 4 * (L & 1);
        d[0] = v[j].x; d[1] = v[j].y; d[2] = v[j].z; d[3] = v[j].w;
    }
    __syncthreads();
    const int tn = t >> 5, tk = t & 31;
    const long long n = n0 + tn, k = k0 + tk;
    if (n >= h || k >= w) return;
    float X[8][8];   // sub-block (a, b) of B^T at position (n, k)
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) X[a][b] = bt_tile[((a * 8 + b) * kBtK + tk) * kBtPitch + tn];
    const long long o0 = n * out.ld + k;
#pragma unroll 1
    for (int i = 0; i < 7; ++i) {
        float Y[4][4];   // level-1 child i, sub-block (a, b)
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) Y[a][b] = child_of1<1>(i, X[a][b], X[a][4 + b], X[4 + a][b], X[4 + a][4 + b]);
#pragma unroll 1
        for (int j = 0; j < 7; ++j) {
            float Cj[4];   // level-2 child (i, j), quadrant t
#pragma unroll
            for (int q = 0; q < 4; ++q)
                Cj[q] = child_of1<1>(j, Y[(q >> 1)][(q & 1)], Y[(q >> 1)][2 + (q & 1)], Y[2 + (q >> 1)][(q & 1)],
                                     Y[2 + (q >> 1)][2 + (q & 1)]);
#pragma unroll
            for (int l = 0; l < 7; ++l)
                split_store1<KIND>(out.hi, out.lo, o0 + (i * 49 + j * 7 + l) * out.child_stride,
                                   child_of1<1>(l, Cj[0], Cj[1], Cj[2], Cj[3]), sc);
        }
    }
}

// Root B side of a depth-2 plan in one pass, straight from the caller's
// row-major B (valid K x N, zero outside) into the 49 leaf operands of B^T,
// split into planes.  Leaf position (n, k) of B^T sub-block (a, b) is
// B[b * w + k][a * h + n] (h = N0 / 4, w = K0 / 4).  A 32 (k) x 32 (n) block of
// positions is loaded coalesced along n; each thread keeps 4 rows (k) packed in
// the lanes of a float4, so the chain is pre_add2_kernel's, element for
// element.  Grandchildren leave through a shared tile, transposed, 7 at a time.
template <int KIND>
__global__ void __launch_bounds__(256) pre_add2_b_root_kernel(const float* __restrict__ B, long long ldb, long long K,
                                                              long long N, long long h, long long w, Stack16 out,
                                                              const float* __restrict__ scale) {
    __shared__ float tile[7][32][33];
    const float sc = scale ? scale[1] : 1.0f;
    const long long k0 = (long long)blockIdx.y * 32, n0 = (long long)blockIdx.x * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const long long n = n0 + tx;
    float4 X[4][4];   // X[a][b]: sub-block (a, b) of B^T; lane l = row k0 + ty + 8 l
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            float t[4];
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                const long long k = k0 + ty + 8 * l;
                const long long row = b * w + k, col = a * h + n;
                t[l] = (k < w && n < h && row < K && col < N) ? __ldg(B + row * ldb + col) : 0.0f;
            }
            X[a][b] = f4(t[0], t[1], t[2], t[3]);
        }
    const int t = ty * 32 + tx;
    const int nl = t >> 3, kq = (t & 7) * 4;   // store role: 4 consecutive k of row n0 + nl
    const long long on = n0 + nl, ok = k0 + kq;
    const bool store = on < h && ok < w;
#pragma unroll 1
    for (int i = 0; i < 7; ++i) {
        float4 Ci[4];   // child i's quadrant t
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 Qt[4] = {X[(q >> 1)][(q & 1)], X[(q >> 1)][2 + (q & 1)], X[2 + (q >> 1)][(q & 1)],
                                  X[2 + (q >> 1)][2 + (q & 1)]};
            float4 ch[7];
            children7<1>(Qt, ch);
            Ci[q] = ch[i];
        }
        float4 g[7];
        children7<1>(Ci, g);
#pragma unroll
        for (int j = 0; j < 7; ++j) {
            tile[j][ty][tx] = g[j].x;
            tile[j][ty + 8][tx] = g[j].y;
            tile[j][ty + 16][tx] = g[j].z;
            tile[j][ty + 24][tx] = g[j].w;
        }
        __syncthreads();
        if (store) {
#pragma unroll
            for (int j = 0; j < 7; ++j) {
                const float4 v = make_float4(tile[j][kq][nl], tile[j][kq + 1][nl], tile[j][kq + 2][nl], tile[j][kq + 3][nl]);
                split_store<KIND>(out.hi, out.lo, (i * 7 + j) * out.child_stride + on * out.ld + ok, v, sc);
            }
        }
        __syncthreads();
    }
}

// Post-additions of two consecutive levels in one pass: for each node, its 49
// grandchild products P[(node * 7 + i) * 7 + j] (h x w, row stride ld_in) ->
// the node output (4h x 4w).  The children's quadrant values are formed with
// the same U-chain as post_add_kernel, then the node's; results are identical
// to two post_add passes and the middle level is never stored.
__device__ __forceinline__ float uchain_quadrant(int q, float P1, float P2, float P3, float P4, float P5, float P6,
                                                 float P7) {
    if (q == 0) return P1 + P2;                               // U1
    const float U2 = P1 + P6;
    if (q == 1) return (U2 + P5) + P3;                        // U5 = U4 + P3, U4 = U2 + P5
    const float U3 = U2 + P7;
    if (q == 2) return U3 - P4;                               // U6
    return U3 + P5;                                           // U7
}

// One element per thread: the 49 products of a position are loaded once.
// ROOT: out is the caller's C: alpha / beta and the valid window apply.
template <bool ROOT>
__global__ void __launch_bounds__(128) post_add2_kernel(const float* __restrict__ P, long long ld_in, long long cs,
                                                        long long h, long long w, float* out, long long ld_out,
                                                        long long out_ns, long long valid_rows, long long valid_cols,
                                                        float alpha, float beta) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= w) return;
    const long long node = blockIdx.z;
    const float* base = P + node * 49 * cs;
    float* o = out + node * out_ns;
    for (long long r = blockIdx.y; r < h; r += gridDim.y) {
        const float* pr = base + r * ld_in + c;
        float p[7][7];
#pragma unroll
        for (int i = 0; i < 7; ++i)
#pragma unroll
            for (int j = 0; j < 7; ++j) p[i][j] = __ldg(pr + (i * 7 + j) * cs);
#pragma unroll
        for (int t = 0; t < 4; ++t) {            // sub-quadrant of every child quadrant
            float Ct[7];                          // child i's quadrant t
#pragma unroll
            for (int i = 0; i < 7; ++i)
                Ct[i] = uchain_quadrant(t, p[i][0], p[i][1], p[i][2], p[i][3], p[i][4], p[i][5], p[i][6]);
#pragma unroll
            for (int q = 0; q < 4; ++q) {        // node quadrant q, its sub-quadrant t
                const long long rr = (long long)((q >> 1) * 2 + (t >> 1)) * h + r;
                const long long cc = (long long)((q & 1) * 2 + (t & 1)) * w + c;
                const float v = uchain_quadrant(q, Ct[0], Ct[1], Ct[2], Ct[3], Ct[4], Ct[5], Ct[6]);
                if (!ROOT) {
                    o[rr * ld_out + cc] = v;
                } else if (rr < valid_rows && cc < valid_cols) {
                    float* dst = o + rr * ld_out + cc;
                    *dst = (beta != 0.0f) ? alpha * v + beta * *dst : alpha * v;
                }
            }
        }
    }
}

// Post-additions of three consecutive levels in one pass (the whole recursion
// of a depth-3 plan, ROOT) or of a node's bottom three levels: for each node,
// its 343 great-grandchild products P[node * 343 + (i * 7 + j) * 7 + l] (h x w,
// row stride ld_in) -> the node output (8h x 8w).  One element per thread,
// every product loaded once.  Level-2 outputs (the U-chain over l), then each
// level-1 child's 16 values (the U-chain over j), then the node's 64 values
// (the U-chain over i): the fp32 operations of three post_add passes.
//
// The level-1 children are visited in the order P1, P6, P7, P5, P3, P4, P2, in
// which the node's U-chain needs them; the chain keeps three running values per
// position (P1, U2 then U4, U3) and each node quadrant is stored as soon as it
// is final (C22 = U7 after P5, C12 = U5 after P3, C21 = U6 after P4, C11 = U1
// after P2).  48 live values instead of the seven children's 112 leave room
// for four blocks per SM, i.e. twice the loads in flight.

// Level-1 child I's 16 values at (quadrant q1, sub-quadrant q2): o1[q1 * 4 + q2].
template <int I>
__device__ __forceinline__ void post3_child(const float* __restrict__ pr, long long cs, float (&o1)[16]) {
    float o2[7][4];   // level-2 child (I, j), quadrant q2
#pragma unroll
    for (int j = 0; j < 7; ++j) {
        float p[7];
#pragma unroll
        for (int l = 0; l < 7; ++l) p[l] = __ldg(pr + ((I * 7 + j) * 7 + l) * cs);
#pragma unroll
        for (int q2 = 0; q2 < 4; ++q2) o2[j][q2] = uchain_quadrant(q2, p[0], p[1], p[2], p[3], p[4], p[5], p[6]);
    }
#pragma unroll
    for (int q1 = 0; q1 < 4; ++q1)
#pragma unroll
        for (int q2 = 0; q2 < 4; ++q2)
            o1[q1 * 4 + q2] = uchain_quadrant(q1, o2[0][q2], o2[1][q2], o2[2][q2], o2[3][q2], o2[4][q2], o2[5][q2],
                                              o2[6][q2]);
}

template <bool ROOT>
__global__ void __launch_bounds__(128, 4) post_add3_kernel(const float* __restrict__ P, long long ld_in, long long cs,
                                                        long long h, long long w, float* out, long long ld_out,
                                                        long long out_ns, long long valid_rows, long long valid_cols,
                                                        float alpha, float beta) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= w) return;
    const long long node = blockIdx.z;
    const float* base = P + node * 343 * cs;
    float* o = out + node * out_ns;
    for (long long r = blockIdx.y; r < h; r += gridDim.y) {
        const float* pr = base + r * ld_in + c;
        // node quadrant q0 at position s = (q1, q2)
        auto put = [&](int q0, int s, float v) {
            const int q1 = s >> 2, q2 = s & 3;
            const long long rr = (long long)(4 * (q0 >> 1) + 2 * (q1 >> 1) + (q2 >> 1)) * h + r;
            const long long cc = (long long)(4 * (q0 & 1) + 2 * (q1 & 1) + (q2 & 1)) * w + c;
            if (!ROOT) {
                o[rr * ld_out + cc] = v;
            } else if (rr < valid_rows && cc < valid_cols) {
                float* dst = o + rr * ld_out + cc;
                *dst = (beta != 0.0f) ? alpha * v + beta * *dst : alpha * v;
            }
        };
        float o1[16], a1[16], u2[16], u3[16];
        post3_child<0>(pr, cs, o1);                                  // P1
#pragma unroll
        for (int s = 0; s < 16; ++s) a1[s] = o1[s];
        post3_child<5>(pr, cs, o1);                                  // P6: U2 = P1 + P6
#pragma unroll
        for (int s = 0; s < 16; ++s) u2[s] = a1[s] + o1[s];
        post3_child<6>(pr, cs, o1);                                  // P7: U3 = U2 + P7
#pragma unroll
        for (int s = 0; s < 16; ++s) u3[s] = u2[s] + o1[s];
        post3_child<4>(pr, cs, o1);                                  // P5: U4 = U2 + P5, C22 = U7 = U3 + P5
#pragma unroll
        for (int s = 0; s < 16; ++s) {
            u2[s] = u2[s] + o1[s];
            put(3, s, u3[s] + o1[s]);
        }
        post3_child<2>(pr, cs, o1);                                  // P3: C12 = U5 = U4 + P3
#pragma unroll
        for (int s = 0; s < 16; ++s) put(1, s, u2[s] + o1[s]);
        post3_child<3>(pr, cs, o1);                                  // P4: C21 = U6 = U3 - P4
#pragma unroll
        for (int s = 0; s < 16; ++s) put(2, s, u3[s] - o1[s]);
        post3_child<1>(pr, cs, o1);                                  // P2: C11 = U1 = P1 + P2
#pragma unroll
        for (int s = 0; s < 16; ++s) put(0, s, a1[s] + o1[s]);
    }
}

// Split jobs of a batched launch: one 32 x 128 block of the source per CTA
// (jobs found by binary search on their first block).  Every thread issues all
// of its loads before its first store.  Untransposed jobs go straight from
// 16-byte loads to the planes (a warp covers 512 contiguous bytes of a row);
// transposed jobs stage the block in a 32 x 129 shared tile (conflict-free both
// ways) and leave it as 128 rows of 32 elements.
template <int KIND>
__global__ void __launch_bounds__(256) batched_split_kernel(const SplitJob* __restrict__ jobs, int njobs) {
    __shared__ float tile[32][129];
    const long long t = blockIdx.x;
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
    }
    const SplitJob J = jobs[lo];
    const float sc = J.scale ? J.scale[J.transpose] : 1.0f;
    const long long local = t - J.tile_begin;
    const long long r0 = (local / J.tiles_c) * 32, c0 = (local % J.tiles_c) * 128;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    if (!J.transpose) {
        const bool vec = (reinterpret_cast<uintptr_t>(J.src) & 15) == 0 && (J.lds & 3) == 0;
        float4 v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int g = tid + 256 * j;   // row g / 32 of the block, columns 4 (g % 32) .. + 3
            const long long r = r0 + (g >> 5), c = c0 + 4 * (g & 31);
            v[j] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (r >= J.rows || c >= J.cols) continue;
            const float* src = J.src + r * J.lds + c;
            if (vec && c + 3 < J.cols) {
                v[j] = __ldg(reinterpret_cast<const float4*>(src));
            } else {
                v[j].x = __ldg(src);
                if (c + 1 < J.cols) v[j].y = __ldg(src + 1);
                if (c + 2 < J.cols) v[j].z = __ldg(src + 2);
                if (c + 3 < J.cols) v[j].w = __ldg(src + 3);
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int g = tid + 256 * j;
            const long long r = r0 + (g >> 5), c = c0 + 4 * (g & 31);
            // ld is a multiple of 8, so a group of 4 never crosses a row: padding columns get zeros
            if (r < J.rows && c < J.cols) split_store<KIND>(J.dst, J.lo, r * J.ldd + c, v[j], sc);
        }
        return;
    }
    // source rows r0 + i (i = warp + 8 s), columns c0 + lane + 32 q
    const int lane = threadIdx.x, warp = threadIdx.y;
    float x[4][4];
#pragma unroll
    for (int sI = 0; sI < 4; ++sI)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const long long r = r0 + warp + 8 * sI, c = c0 + lane + 32 * q;
            x[sI][q] = (r < J.rows && c < J.cols) ? __ldg(J.src + r * J.lds + c) : 0.0f;
        }
#pragma unroll
    for (int sI = 0; sI < 4; ++sI)
#pragma unroll
        for (int q = 0; q < 4; ++q) tile[warp + 8 * sI][lane + 32 * q] = x[sI][q];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int g = tid + 256 * j;   // output row a (a source column), 4 consecutive output columns
        const int a = g >> 3, q = (g & 7) * 4;
        const long long orow = c0 + a, ocol = r0 + q;
        if (orow < J.cols && ocol < J.rows) {
            const float4 v = make_float4(tile[q][a], tile[q + 1][a], tile[q + 2][a], tile[q + 3][a]);
            split_store<KIND>(J.dst, J.lo, orow * J.ldd + ocol, v, sc);
        }
    }
}

inline unsigned gy(long long rows) { return (unsigned)(rows < 65535 ? (rows > 0 ? rows : 1) : 65535); }
inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

}  // namespace

cudaError_t launch_pre_add(const View& parent, long long nodes, const Stack& out, int side_b, int full,
                           cudaStream_t stream) {
    const long long h = parent.rows / 2, w = parent.cols / 2;
    if (h <= 0 || w <= 0 || nodes <= 0) return cudaSuccess;
    const bool vec = aligned16(parent.ptr) && aligned16(out.ptr) && parent.ld % 4 == 0 && w % 4 == 0 &&
                     parent.node_stride % 4 == 0 && out.ld % 4 == 0 && out.child_stride % 4 == 0;
    dim3 grid((unsigned)((w + 4 * 128 - 1) / (4 * 128)), gy(h), (unsigned)nodes);
#define FMM_PRE(V, S, F) pre_add_kernel<V, S, F><<<grid, 128, 0, stream>>>(parent, h, w, out)
    if (vec) {
        if (side_b) { if (full) FMM_PRE(true, 1, true); else FMM_PRE(true, 1, false); }
        else        { if (full) FMM_PRE(true, 0, true); else FMM_PRE(true, 0, false); }
    } else {
        if (side_b) { if (full) FMM_PRE(false, 1, true); else FMM_PRE(false, 1, false); }
        else        { if (full) FMM_PRE(false, 0, true); else FMM_PRE(false, 0, false); }
    }
#undef FMM_PRE
    return cudaGetLastError();
}

cudaError_t launch_pre_add_b_root(const float* B, long long ldb, long long K, long long N, long long kh,
                                  long long nh, const Stack& out, int full, cudaStream_t stream) {
    if (kh <= 0 || nh <= 0) return cudaSuccess;
    dim3 grid((unsigned)((nh + 31) / 32), (unsigned)((kh + 31) / 32));
    dim3 block(32, 8);
    if (full) pre_add_b_root_kernel<true><<<grid, block, 0, stream>>>(B, ldb, K, N, kh, nh, out);
    else pre_add_b_root_kernel<false><<<grid, block, 0, stream>>>(B, ldb, K, N, kh, nh, out);
    return cudaGetLastError();
}

cudaError_t launch_post_add(const float* P, long long ld_in, long long child_stride, long long nodes, long long h,
                            long long w, float* out, long long ld_out, long long out_node_stride,
                            long long valid_rows, long long valid_cols, float alpha, float beta,
                            cudaStream_t stream) {
    if (h <= 0 || w <= 0 || nodes <= 0) return cudaSuccess;
    const bool root = valid_rows >= 0;
    const bool vec = aligned16(P) && ld_in % 4 == 0 && child_stride % 4 == 0 && w % 4 == 0 &&
                     (root || (aligned16(out) && ld_out % 4 == 0 && out_node_stride % 4 == 0));
    dim3 grid((unsigned)((w + 4 * 128 - 1) / (4 * 128)), gy(h), (unsigned)nodes);
#define FMM_POST(V, R)                                                                                         \
    post_add_kernel<V, R><<<grid, 128, 0, stream>>>(P, ld_in, child_stride, h, w, out, ld_out, out_node_stride, \
                                                   valid_rows, valid_cols, alpha, beta)
    if (root) { if (vec) FMM_POST(true, true); else FMM_POST(false, true); }
    else      { if (vec) FMM_POST(true, false); else FMM_POST(false, false); }
#undef FMM_POST
    return cudaGetLastError();
}

cudaError_t launch_transpose(const float* B, long long ldb, long long K, long long N, float* Bt, long long ldt,
                             cudaStream_t stream, long long rows_out, long long cols_out) {
    if (rows_out < 0) rows_out = N;
    if (cols_out < 0) cols_out = K;
    if (rows_out <= 0 || cols_out <= 0) return cudaSuccess;
    dim3 grid((unsigned)((rows_out + 31) / 32), (unsigned)((cols_out + 127) / 128));
    transpose_kernel<<<grid, dim3(32, 8), 0, stream>>>(B, ldb, K, N, Bt, ldt, rows_out, cols_out);
    return cudaGetLastError();
}

cudaError_t launch_copy2d(const float* A, long long lda, long long M, long long K, float* dst, long long ldd,
                          cudaStream_t stream) {
    if (M <= 0 || K <= 0) return cudaSuccess;
    dim3 grid((unsigned)((K + 255) / 256), gy(M));
    copy2d_kernel<<<grid, 256, 0, stream>>>(A, lda, M, K, dst, ldd);
    return cudaGetLastError();
}

cudaError_t launch_batched_copy(const CopyJob* jobs, int njobs, long long total_tiles, cudaStream_t stream) {
    if (njobs <= 0 || total_tiles <= 0) return cudaSuccess;
    batched_copy_kernel<<<(unsigned)total_tiles, dim3(32, 8), 0, stream>>>(jobs, njobs);
    return cudaGetLastError();
}

cudaError_t launch_fp16_scales(const float* A, long long lda, long long M, long long K, const float* B,
                               long long ldb, long long N, float bound_mult, float* scale, unsigned* scratch,
                               cudaStream_t stream) {
    cudaError_t e = cudaMemsetAsync(scratch, 0, 2 * sizeof(unsigned), stream);
    if (e != cudaSuccess) return e;
    if (M > 0 && K > 0) absmax_kernel<<<dim3(4, gy(M < 1024 ? M : 1024)), 256, 0, stream>>>(A, lda, M, K, scratch);
    if (K > 0 && N > 0) absmax_kernel<<<dim3(4, gy(K < 1024 ? K : 1024)), 256, 0, stream>>>(B, ldb, K, N, scratch + 1);
    fp16_scale_kernel<<<1, 32, 0, stream>>>(scratch, bound_mult, scale);
    return cudaGetLastError();
}

cudaError_t launch_quad_pre(const QuadPre& q, int side_b, cudaStream_t stream) {
    if (q.h <= 0 || q.w <= 0) return cudaSuccess;
    dim3 grid((unsigned)((q.w + 511) / 512), gy(q.h));
    if (side_b) quad_pre_kernel<1><<<grid, 128, 0, stream>>>(q);
    else quad_pre_kernel<0><<<grid, 128, 0, stream>>>(q);
    return cudaGetLastError();
}

cudaError_t launch_quad_post(const QuadPost& q, int part, cudaStream_t stream) {
    if (q.h <= 0 || q.w <= 0) return cudaSuccess;
    dim3 grid((unsigned)((q.w + 511) / 512), gy(q.h));
    switch (part) {
        case 0: quad_post_kernel<0><<<grid, 128, 0, stream>>>(q); break;
        case 1: quad_post_kernel<1><<<grid, 128, 0, stream>>>(q); break;
        case 2: quad_post_kernel<2><<<grid, 128, 0, stream>>>(q); break;
        case 3: quad_post_kernel<3><<<grid, 128, 0, stream>>>(q); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_pre_add16(const View& parent, long long nodes, const Stack16& out, int side_b, int kind,
                             const float* scale, cudaStream_t stream) {
    const long long h = parent.rows / 2, w = parent.cols / 2;
    if (h <= 0 || w <= 0 || nodes <= 0) return cudaSuccess;
    const bool vec = aligned16(parent.ptr) && parent.ld % 4 == 0 && w % 4 == 0 && parent.node_stride % 4 == 0;
    dim3 grid((unsigned)((w + 4 * 128 - 1) / (4 * 128)), gy(h), (unsigned)nodes);
#define FMM_PRE16(V, S, K) pre_add16_kernel<V, S, K><<<grid, 128, 0, stream>>>(parent, h, w, out, scale)
#define FMM_PRE16K(V, S)                                                    \
    switch (kind) {                                                          \
        case kSplitBF16: FMM_PRE16(V, S, kSplitBF16); break;                \
        case kSplitFP16: FMM_PRE16(V, S, kSplitFP16); break;                \
        default: FMM_PRE16(V, S, kSplitTF32); break;                        \
    }
    if (vec) { if (side_b) { FMM_PRE16K(true, 1) } else { FMM_PRE16K(true, 0) } }
    else     { if (side_b) { FMM_PRE16K(false, 1) } else { FMM_PRE16K(false, 0) } }
#undef FMM_PRE16K
#undef FMM_PRE16
    return cudaGetLastError();
}

cudaError_t launch_pre_add16_b_root(const float* B, long long ldb, long long K, long long N, long long kh,
                                    long long nh, const Stack16& out, int kind, const float* scale,
                                    cudaStream_t stream) {
    if (kh <= 0 || nh <= 0) return cudaSuccess;
    dim3 grid((unsigned)((nh + 31) / 32), (unsigned)((kh + 31) / 32));
    switch (kind) {
        case kSplitBF16:
            pre_add16_b_root_kernel<kSplitBF16><<<grid, dim3(32, 8), 0, stream>>>(B, ldb, K, N, kh, nh, out, scale);
            break;
        case kSplitFP16:
            pre_add16_b_root_kernel<kSplitFP16><<<grid, dim3(32, 8), 0, stream>>>(B, ldb, K, N, kh, nh, out, scale);
            break;
        default:
            pre_add16_b_root_kernel<kSplitTF32><<<grid, dim3(32, 8), 0, stream>>>(B, ldb, K, N, kh, nh, out, scale);
    }
    return cudaGetLastError();
}

cudaError_t launch_split16(const float* X, long long ldx, long long rows, long long cols, const Stack16& out,
                           int transpose, int kind, const float* scale, int which, cudaStream_t stream) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    // plain: 32 x 128 blocks; transposed: 128 (row) x 32 (column) blocks
    const dim3 grid = transpose ? dim3((unsigned)((cols + 31) / 32), (unsigned)((rows + 127) / 128))
                                : dim3((unsigned)((cols + 127) / 128), (unsigned)((rows + 31) / 32));
#define FMM_SPLIT(K, T) split16_kernel<K, T><<<grid, dim3(32, 8), 0, stream>>>(X, ldx, rows, cols, out, scale, which)
#define FMM_SPLITK(T)                                   \
    switch (kind) {                                      \
        case kSplitBF16: FMM_SPLIT(kSplitBF16, T); break; \
        case kSplitFP16: FMM_SPLIT(kSplitFP16, T); break; \
        default: FMM_SPLIT(kSplitTF32, T); break;         \
    }
    if (transpose) { FMM_SPLITK(true) } else { FMM_SPLITK(false) }
#undef FMM_SPLITK
#undef FMM_SPLIT
    return cudaGetLastError();
}

cudaError_t launch_pre_add2(const View& node, long long nodes, const Stack16& out, int side_b, int kind,
                            const float* scale, cudaStream_t stream) {
    const long long h = node.rows / 4, w = node.cols / 4;
    if (h <= 0 || w <= 0 || nodes <= 0) return cudaSuccess;
    if (w % 4) return cudaErrorInvalidValue;
    const bool vec = aligned16(node.ptr) && node.ld % 4 == 0 && node.node_stride % 4 == 0;
    dim3 grid((unsigned)((w + 511) / 512), gy(h), (unsigned)nodes);
#define FMM_PRE2(V, S, K) pre_add2_kernel<V, S, K><<<grid, 128, 0, stream>>>(node, h, w, out, scale)
#define FMM_PRE2K(V, S)                                        \
    switch (kind) {                                             \
        case kSplitBF16: FMM_PRE2(V, S, kSplitBF16); break;    \
        case kSplitFP16: FMM_PRE2(V, S, kSplitFP16); break;    \
        default: FMM_PRE2(V, S, kSplitTF32); break;            \
    }
    if (vec) { if (side_b) { FMM_PRE2K(true, 1) } else { FMM_PRE2K(true, 0) } }
    else     { if (side_b) { FMM_PRE2K(false, 1) } else { FMM_PRE2K(false, 0) } }
#undef FMM_PRE2K
#undef FMM_PRE2
    return cudaGetLastError();
}

cudaError_t launch_pre_add2_b_root(const float* B, long long ldb, long long K, long long N, long long h, long long w,
                                   const Stack16& out, int kind, const float* scale, cudaStream_t stream) {
    if (h <= 0 || w <= 0) return cudaSuccess;
    if (w % 4) return cudaErrorInvalidValue;
    dim3 grid((unsigned)((h + 31) / 32), (unsigned)((w + 31) / 32));
    dim3 block(32, 8);
    switch (kind) {
        case kSplitBF16: pre_add2_b_root_kernel<kSplitBF16><<<grid, block, 0, stream>>>(B, ldb, K, N, h, w, out, scale); break;
        case kSplitFP16: pre_add2_b_root_kernel<kSplitFP16><<<grid, block, 0, stream>>>(B, ldb, K, N, h, w, out, scale); break;
        default: pre_add2_b_root_kernel<kSplitTF32><<<grid, block, 0, stream>>>(B, ldb, K, N, h, w, out, scale); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_pre_add3(const View& node, long long nodes, const Stack16& out, int side_b, int kind,
                            const float* scale, cudaStream_t stream) {
    const long long h = node.rows / 8, w = node.cols / 8;
    if (h <= 0 || w <= 0 || nodes <= 0) return cudaSuccess;
    dim3 grid((unsigned)((w + 255) / 256), gy(h), (unsigned)nodes);
#define FMM_PRE3(S, K) pre_add3_kernel<S, K><<<grid, 256, 0, stream>>>(node, h, w, out, scale)
#define FMM_PRE3K(S)                                        \
    switch (kind) {                                          \
        case kSplitBF16: FMM_PRE3(S, kSplitBF16); break;    \
        case kSplitFP16: FMM_PRE3(S, kSplitFP16); break;    \
        default: FMM_PRE3(S, kSplitTF32); break;            \
    }
    if (side_b) { FMM_PRE3K(1) } else { FMM_PRE3K(0) }
#undef FMM_PRE3K
#undef FMM_PRE3
    return cudaGetLastError();
}

template <int KIND>
static cudaError_t launch_pre_add3_bt_impl(const float* B, long long ldb, long long K, long long N, long long h,
                                           long long w, const Stack16& out, const float* scale,
                                           cudaStream_t stream) {
    // once per device and instantiation (keeps later launches free of other API calls)
    static bool attr_done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !attr_done[dev]) {
        e = cudaFuncSetAttribute(pre_add3_bt_kernel<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBtSmem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_done[dev] = true;
    }
    const long long tiles_n = (h + kBtN - 1) / kBtN, tiles = tiles_n * ((w + kBtK - 1) / kBtK);
    pre_add3_bt_kernel<KIND><<<(unsigned)tiles, 256, kBtSmem, stream>>>(B, ldb, K, N, h, w, tiles_n, out, scale);
    return cudaGetLastError();
}

cudaError_t launch_pre_add3_bt(const float* B, long long ldb, long long K, long long N, long long h, long long w,
                               const Stack16& out, int kind, const float* scale, cudaStream_t stream) {
    if (h <= 0 || w <= 0) return cudaSuccess;
    if ((h & 3) != 0) return cudaErrorInvalidValue;   // float4 staging along n
    switch (kind) {
        case kSplitBF16: return launch_pre_add3_bt_impl<kSplitBF16>(B, ldb, K, N, h, w, out, scale, stream);
        case kSplitFP16: return launch_pre_add3_bt_impl<kSplitFP16>(B, ldb, K, N, h, w, out, scale, stream);
        default: return launch_pre_add3_bt_impl<kSplitTF32>(B, ldb, K, N, h, w, out, scale, stream);
    }
}

cudaError_t launch_post_add3(const float* P, long long ld_in, long long child_stride, long long nodes, long long h,
                             long long w, float* out, long long ld_out, long long out_node_stride,
                             long long valid_rows, long long valid_cols, float alpha, float beta,
                             cudaStream_t stream) {
    if (h <= 0 || w <= 0 || nodes <= 0) return cudaSuccess;
    dim3 grid((unsigned)((w + 127) / 128), gy(h), (unsigned)nodes);
    if (valid_rows >= 0)
        post_add3_kernel<true><<<grid, 128, 0, stream>>>(P, ld_in, child_stride, h, w, out, ld_out, out_node_stride,
                                                         valid_rows, valid_cols, alpha, beta);
    else
        post_add3_kernel<false><<<grid, 128, 0, stream>>>(P, ld_in, child_stride, h, w, out, ld_out, out_node_stride,
                                                          -1, -1, 1.f, 0.f);
    return cudaGetLastError();
}

cudaError_t launch_post_add2(const float* P, long long ld_in, long long child_stride, long long nodes, long long h,
                             long long w, float* out, long long ld_out, long long out_node_stride,
                             long long valid_rows, long long valid_cols, float alpha, float beta,
                             cudaStream_t stream) {
    if (h <= 0 || w <= 0 || nodes <= 0) return cudaSuccess;
    dim3 grid((unsigned)((w + 127) / 128), gy(h), (unsigned)nodes);
    if (valid_rows >= 0)
        post_add2_kernel<true><<<grid, 128, 0, stream>>>(P, ld_in, child_stride, h, w, out, ld_out, out_node_stride,
                                                         valid_rows, valid_cols, alpha, beta);
    else
        post_add2_kernel<false><<<grid, 128, 0, stream>>>(P, ld_in, child_stride, h, w, out, ld_out, out_node_stride,
                                                          -1, -1, 1.f, 0.f);
    return cudaGetLastError();
}

cudaError_t launch_batched_split(const SplitJob* jobs, int njobs, long long total_tiles, int kind,
                                 cudaStream_t stream) {
    if (njobs <= 0 || total_tiles <= 0) return cudaSuccess;
    switch (kind) {
        case kSplitBF16: batched_split_kernel<kSplitBF16><<<(unsigned)total_tiles, dim3(32, 8), 0, stream>>>(jobs, njobs); break;
        case kSplitFP16: batched_split_kernel<kSplitFP16><<<(unsigned)total_tiles, dim3(32, 8), 0, stream>>>(jobs, njobs); break;
        default: batched_split_kernel<kSplitTF32><<<(unsigned)total_tiles, dim3(32, 8), 0, stream>>>(jobs, njobs);
    }
    return cudaGetLastError();
}

cudaError_t launch_batched_absmax(const AbsJob* jobs, int njobs, long long total_tiles, cudaStream_t stream) {
    if (njobs <= 0 || total_tiles <= 0) return cudaSuccess;
    batched_absmax_kernel<<<(unsigned)total_tiles, 256, 0, stream>>>(jobs, njobs);
    return cudaGetLastError();
}

cudaError_t launch_batched_fp16_scales(const unsigned* maxima, const float* bound, float* scales, int count,
                                       cudaStream_t stream) {
    if (count <= 0) return cudaSuccess;
    batched_fp16_scale_kernel<<<(unsigned)((2 * count + 255) / 256), 256, 0, stream>>>(maxima, bound, scales, count);
    return cudaGetLastError();
}

cudaError_t launch_fill(float* p, size_t n, unsigned seed, cudaStream_t stream) {
    if (n == 0) return cudaSuccess;
    fill_kernel<<<1024, 256, 0, stream>>>(p, n, seed);
    return cudaGetLastError();
}

// 2-D copy of a rows x cols block between pinned host memory (through its
// device mapping) and device memory, by SM loads and stores: the host-resident
// plan's alternative to the copy engines.  float4 when both blocks allow it,
// four of them in flight per thread, so that a few blocks fill the host link
// (32 blocks of 512 threads: 211 GB/s in, 193 GB/s out) and the other SMs stay
// with the compute running beside the copy.
constexpr int kHostCopyBlocks = 32;
constexpr int kHostCopyUnroll = 4;
__global__ void __launch_bounds__(512) host_copy2d_kernel(const float* __restrict__ src, long long lds,
                                                          float* __restrict__ dst, long long ldd, long long rows,
                                                          long long cols, int vec) {
    const long long step = (long long)gridDim.x * blockDim.x;
    if (vec) {
        const long long c4 = cols >> 2, total = rows * c4;
        long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
        for (; i + (kHostCopyUnroll - 1) * step < total; i += kHostCopyUnroll * step) {
            float4 v[kHostCopyUnroll];
#pragma unroll
            for (int j = 0; j < kHostCopyUnroll; ++j) {
                const long long e = i + j * step, r = e / c4, c = e - r * c4;
                v[j] = reinterpret_cast<const float4*>(src + r * lds)[c];
            }
#pragma unroll
            for (int j = 0; j < kHostCopyUnroll; ++j) {
                const long long e = i + j * step, r = e / c4, c = e - r * c4;
                reinterpret_cast<float4*>(dst + r * ldd)[c] = v[j];
            }
        }
        for (; i < total; i += step) {
            const long long r = i / c4, c = i - r * c4;
            reinterpret_cast<float4*>(dst + r * ldd)[c] = reinterpret_cast<const float4*>(src + r * lds)[c];
        }
    } else {
        const long long total = rows * cols;
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += step) {
            const long long r = i / cols, c = i - r * cols;
            dst[r * ldd + c] = src[r * lds + c];
        }
    }
}

cudaError_t launch_host_copy2d(const float* src, long long lds, float* dst, long long ldd, long long rows,
                               long long cols, cudaStream_t stream) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    const int vec = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0 &&
                    lds % 4 == 0 && ldd % 4 == 0 && cols % 4 == 0;
    host_copy2d_kernel<<<kHostCopyBlocks, 512, 0, stream>>>(src, lds, dst, ldd, rows, cols, vec);
    return cudaGetLastError();
}

cudaError_t launch_scale(float* C, long long ldc, long long M, long long N, float beta, cudaStream_t stream) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    dim3 grid((unsigned)((N + 255) / 256), gy(M));
    scale_kernel<<<grid, 256, 0, stream>>>(C, ldc, M, N, beta);
    return cudaGetLastError();
}

}  // namespace fmm
