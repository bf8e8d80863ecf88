// peak.cu -- tensor-pipe throughput probe of this GPU.
//
// Issues tcgen05.mma back to back on operand tiles that stay in shared memory,
// with the instruction shape of the CTA-pair leaf kernel (cta_group::2,
// M = 256, N = 256, both operands K-major with 128-byte swizzle), one pair per
// two SMs, so that no operand traffic, epilogue or pipeline wait limits the
// rate: the measured flop rate is the ceiling the leaf launches are held
// against.  Operands are uniform random values (the tensor core's power, and
// so its clock under the power cap, depends on the data).  Measurement only:
// the multiply itself never runs this code.
#include "../../include/fmm.h"
#include "fmm_internal.h"
#include "ptx.cuh"

#include <cstdio>

namespace fmm {
namespace {

constexpr int kProbeTileBytes = 128 * 128;            // 128 rows x 128 bytes per CTA and operand
constexpr int kProbeStages = 2;                       // A | B pairs at distinct addresses
constexpr int kProbeBytes = kProbeStages * 2 * kProbeTileBytes;
// more shared memory than two CTAs of an SM could share: one probe CTA per SM
constexpr int kProbeSmem = 120 * 1024;
static_assert(1024 + kProbeBytes + 64 <= kProbeSmem, "probe shared memory");
constexpr int kProbeBatch = 64;                       // MMAs per commit

__device__ unsigned g_probe_status;

// KIND 0: kind::tf32 (K = 8 per instruction); 1: kind::f16 with bf16 operands (K = 16).
template <int KIND>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(128, 1)
    mma_probe_kernel(const float* __restrict__ fill, long long batches) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw_addr = smem_u32(smem_raw);
    const uint32_t base = (raw_addr + 1023u) & ~1023u;
    uint8_t* base_ptr = smem_raw + (base - raw_addr);
    const uint32_t bar0 = base + kProbeBytes;             // two commit barriers
    uint8_t* bar_ptr = base_ptr + kProbeBytes;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar_ptr + 16);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(bar_ptr + 24);
    const uint32_t rank = cluster_ctarank();
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    // operand tiles: the same random words in every CTA (the tile contents
    // only matter for the tensor core's power draw)
    {
        float4* dst = reinterpret_cast<float4*>(base_ptr);
        const float4* src = reinterpret_cast<const float4*>(fill);
        for (int i = threadIdx.x; i < kProbeBytes / 16; i += blockDim.x) dst[i] = src[i];
    }
    fence_proxy_async_smem();   // generic-proxy writes, read by the tensor core (async proxy)
    if (threadIdx.x == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar0 + 8, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc_pair(smem_u32(tmem_slot), 256);
        tmem_relinquish_pair();
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0 && rank == 0) {
        constexpr uint32_t idesc = make_idesc(KIND == 0 ? 2u : 1u, 256, 256);
        for (long long j = 0; j < batches; ++j) {
            for (int i = 0; i < kProbeBatch; i += 4) {
                const uint32_t st = base + (uint32_t)(((i >> 2) & (kProbeStages - 1)) * 2 * kProbeTileBytes);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint64_t ad = sdesc_kmajor_sw128(st + kk * 32);
                    const uint64_t bd = sdesc_kmajor_sw128(st + kProbeTileBytes + kk * 32);
                    const uint32_t acc = (j == 0 && i == 0 && kk == 0) ? 0u : 1u;
                    if constexpr (KIND == 0) mma_tf32_pair(tmem, ad, bd, idesc, acc);
                    else mma_f16_pair(tmem, ad, bd, idesc, acc);
                }
            }
            // batch j completes on barrier j % 2 (its (j / 2)-th phase); wait for
            // batch j - 1 before issuing more, so at most two batches are queued
            // and no barrier receives a commit before its previous phase was seen
            mma_commit_pair(bar0 + 8u * (uint32_t)(j & 1), (uint16_t)0x1);
            if (j >= 1) {
                const long long p = j - 1;
                if (!mbar_wait(bar0 + 8u * (uint32_t)(p & 1), (uint32_t)((p >> 1) & 1), abort_flag, &g_probe_status))
                    break;
            }
        }
        if (!*abort_flag && batches >= 1) {
            const long long p = batches - 1;
            mbar_wait(bar0 + 8u * (uint32_t)(p & 1), (uint32_t)((p >> 1) & 1), abort_flag, &g_probe_status);
        }
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync();   // every pair MMA of CTA 0 is complete (or the wait gave up)
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc_pair(tmem, 256);
    }
}

template <int KIND>
cudaError_t launch_probe(const float* fill, long long batches, int clusters, cudaStream_t s) {
    auto kern = mma_probe_kernel<KIND>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kProbeSmem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)(2 * clusters), 128, kProbeSmem, s>>>(fill, batches);
    return cudaGetLastError();
}

}  // namespace
}  // namespace fmm

using namespace fmm;

extern "C" fmm_status_t fmm_tensor_peak(int kind, int64_t batches, const float* fill, double* tflops, double* ms,
                                        fmm_stream_t stream_) {
    if ((kind != 0 && kind != 1) || batches < 1 || batches > (int64_t)1 << 24 || !fill || !tflops)
        return FMM_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(fill) & 15) != 0) return FMM_ERR_ALIGNMENT;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) {
        cudaGetLastError();
        return FMM_ERR_NO_DEVICE;
    }
    int dev = 0, major = 0, minor = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FMM_ERR_CUDA;
    if (!(major == 10 && minor == 3)) return FMM_ERR_NO_DEVICE;
    cudaStream_t s = (cudaStream_t)stream_;
    // as many pairs as can be resident at once (a cluster's CTAs share a GPC)
    int clusters = sms / 2;
    {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr;
        attr.id = cudaLaunchAttributeClusterDimension;
        attr.val.clusterDim.x = 2;
        attr.val.clusterDim.y = 1;
        attr.val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)(sms & ~1));
        cfg.blockDim = dim3(128);
        cfg.dynamicSmemBytes = kProbeSmem;
        cfg.attrs = &attr;
        cfg.numAttrs = 1;
        int n = 0;
        cudaError_t e = kind == 0 ? cudaFuncSetAttribute(mma_probe_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                         kProbeSmem)
                                  : cudaFuncSetAttribute(mma_probe_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                         kProbeSmem);
        if (e != cudaSuccess) return FMM_ERR_CUDA;
        e = cudaOccupancyMaxActiveClusters(&n, kind == 0 ? (void*)mma_probe_kernel<0> : (void*)mma_probe_kernel<1>,
                                           &cfg);
        if (e == cudaSuccess && n > 0 && n < clusters) clusters = n;
        cudaGetLastError();
    }
    unsigned zero = 0;
    if (cudaMemcpyToSymbolAsync(g_probe_status, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return FMM_ERR_CUDA;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return FMM_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return FMM_ERR_CUDA; }
    cudaError_t e = kind == 0 ? launch_probe<0>(fill, batches, clusters, s) : launch_probe<1>(fill, batches, clusters, s);
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = kind == 0 ? launch_probe<0>(fill, batches, clusters, s)
                                        : launch_probe<1>(fill, batches, clusters, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    unsigned w = 0;
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&w, g_probe_status, sizeof(w));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return FMM_ERR_CUDA;
    if (w & FMM_DEV_TIMEOUT_BIT) return FMM_ERR_TIMEOUT;
    const double k_per_mma = kind == 0 ? 8.0 : 16.0;
    const double flops = 2.0 * 256.0 * 256.0 * k_per_mma * (double)kProbeBatch * (double)batches * (double)clusters;
    *tflops = flops / ((double)t * 1e-3) / 1e12;
    if (ms) *ms = t;
    return FMM_OK;
}
