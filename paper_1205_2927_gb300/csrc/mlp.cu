// mlp.cu -- the planner's cost model: a 6 -> 64 -> 64 -> 1 ReLU network in fp32
// that predicts log(run time) of a candidate plan from
// (log2 M, log2 K, log2 N, depth, leaf tile / 128, precision), standardised.
//
// Parameter vector (flat, NPARAM floats): W1[64][6], b1[64], W2[64][64], b2[64],
// W3[1][64], b3[1]; weights row-major [out][in].
//
// Kernels: forward (one thread per sample, weights in shared memory);
// training step = per-sample forward/backward writing activations and deltas,
// then one thread per parameter summing its gradient over the batch in a fixed
// order (deterministic) and applying Adam in place.
#include "../../include/fmm.h"
#include "fmm_internal.h"

namespace fmm {
namespace {

constexpr int IN = 6, HID = 64;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + HID * IN, OFF_W2 = OFF_B1 + HID, OFF_B2 = OFF_W2 + HID * HID,
              OFF_W3 = OFF_B2 + HID, OFF_B3 = OFF_W3 + HID, NPARAM = OFF_B3 + 1;
static_assert(NPARAM == FMM_MLP_NPARAM, "parameter count");

__device__ __forceinline__ void load_params(float* sp, const float* __restrict__ params) {
    for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) sp[i] = params[i];
    __syncthreads();
}

__global__ void __launch_bounds__(128) mlp_forward_kernel(const float* __restrict__ params,
                                                          const float* __restrict__ X, float* __restrict__ Y,
                                                          int batch) {
    __shared__ float sp[NPARAM];
    load_params(sp, params);
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= batch) return;
    float x[IN], h1[HID];
#pragma unroll
    for (int j = 0; j < IN; ++j) x[j] = X[s * IN + j];
#pragma unroll 4
    for (int i = 0; i < HID; ++i) {
        float z = sp[OFF_B1 + i];
#pragma unroll
        for (int j = 0; j < IN; ++j) z += sp[OFF_W1 + i * IN + j] * x[j];
        h1[i] = z > 0.f ? z : 0.f;
    }
    float y = sp[OFF_B3];
    for (int i = 0; i < HID; ++i) {
        float z = sp[OFF_B2 + i];
#pragma unroll 8
        for (int j = 0; j < HID; ++j) z += sp[OFF_W2 + i * HID + j] * h1[j];
        y += sp[OFF_W3 + i] * (z > 0.f ? z : 0.f);
    }
    Y[s] = y;
}

// Per sample: activations h1, h2 and deltas dz1, dz2 (all [batch][64]), dy and (y - t)^2.
__global__ void __launch_bounds__(128) mlp_fwdbwd_kernel(const float* __restrict__ params,
                                                         const float* __restrict__ X, const float* __restrict__ T,
                                                         int batch, float* __restrict__ H1, float* __restrict__ H2,
                                                         float* __restrict__ DZ1, float* __restrict__ DZ2,
                                                         float* __restrict__ DY, float* __restrict__ SQ) {
    __shared__ float sp[NPARAM];
    load_params(sp, params);
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= batch) return;
    float x[IN], h1[HID], z2[HID];
#pragma unroll
    for (int j = 0; j < IN; ++j) x[j] = X[s * IN + j];
#pragma unroll 4
    for (int i = 0; i < HID; ++i) {
        float z = sp[OFF_B1 + i];
#pragma unroll
        for (int j = 0; j < IN; ++j) z += sp[OFF_W1 + i * IN + j] * x[j];
        h1[i] = z > 0.f ? z : 0.f;  // z1 > 0 <=> h1 > 0
        H1[(size_t)s * HID + i] = h1[i];
    }
    float y = sp[OFF_B3];
    for (int i = 0; i < HID; ++i) {
        float z = sp[OFF_B2 + i];
#pragma unroll 8
        for (int j = 0; j < HID; ++j) z += sp[OFF_W2 + i * HID + j] * h1[j];
        z2[i] = z;
        const float h2 = z > 0.f ? z : 0.f;
        H2[(size_t)s * HID + i] = h2;
        y += sp[OFF_W3 + i] * h2;
    }
    const float r = y - T[s];
    const float dy = r / (float)batch;  // d(0.5 mean r^2)/dy
    DY[s] = dy;
    SQ[s] = r * r;
    float dz2[HID];
#pragma unroll 8
    for (int i = 0; i < HID; ++i) {
        dz2[i] = z2[i] > 0.f ? dy * sp[OFF_W3 + i] : 0.f;
        DZ2[(size_t)s * HID + i] = dz2[i];
    }
    for (int j = 0; j < HID; ++j) {
        float dh = 0.f;
#pragma unroll 8
        for (int i = 0; i < HID; ++i) dh += sp[OFF_W2 + i * HID + j] * dz2[i];
        DZ1[(size_t)s * HID + j] = h1[j] > 0.f ? dh : 0.f;
    }
}

// One thread per parameter (plus one for the loss): gradient summed over the
// batch in sample order, then Adam (bias-corrected) in place.
__global__ void __launch_bounds__(128) mlp_grad_adam_kernel(float* __restrict__ params, float* __restrict__ m,
                                                            float* __restrict__ v, const float* __restrict__ X,
                                                            const float* __restrict__ H1,
                                                            const float* __restrict__ H2,
                                                            const float* __restrict__ DZ1,
                                                            const float* __restrict__ DZ2,
                                                            const float* __restrict__ DY,
                                                            const float* __restrict__ SQ, int batch, int step,
                                                            float lr, float beta1, float beta2, float eps,
                                                            float* __restrict__ grad_out,
                                                            float* __restrict__ loss_out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > NPARAM) return;
    if (p == NPARAM) {
        if (loss_out) {
            float acc = 0.f;
            for (int s = 0; s < batch; ++s) acc += SQ[s];
            *loss_out = 0.5f * acc / (float)batch;
        }
        return;
    }
    float g = 0.f;
    if (p < OFF_B1) {
        const int i = p / IN, j = p % IN;
        for (int s = 0; s < batch; ++s) g += DZ1[(size_t)s * HID + i] * X[s * IN + j];
    } else if (p < OFF_W2) {
        const int i = p - OFF_B1;
        for (int s = 0; s < batch; ++s) g += DZ1[(size_t)s * HID + i];
    } else if (p < OFF_B2) {
        const int i = (p - OFF_W2) / HID, j = (p - OFF_W2) % HID;
        for (int s = 0; s < batch; ++s) g += DZ2[(size_t)s * HID + i] * H1[(size_t)s * HID + j];
    } else if (p < OFF_W3) {
        const int i = p - OFF_B2;
        for (int s = 0; s < batch; ++s) g += DZ2[(size_t)s * HID + i];
    } else if (p < OFF_B3) {
        const int j = p - OFF_W3;
        for (int s = 0; s < batch; ++s) g += DY[s] * H2[(size_t)s * HID + j];
    } else {
        for (int s = 0; s < batch; ++s) g += DY[s];
    }
    if (grad_out) grad_out[p] = g;
    if (lr != 0.f) {
        const float mi = beta1 * m[p] + (1.f - beta1) * g;
        const float vi = beta2 * v[p] + (1.f - beta2) * g * g;
        m[p] = mi;
        v[p] = vi;
        const float mhat = mi / (1.f - powf(beta1, (float)step));
        const float vhat = vi / (1.f - powf(beta2, (float)step));
        params[p] -= lr * mhat / (sqrtf(vhat) + eps);
    }
}

}  // namespace

cudaError_t mlp_forward(const float* params, const float* X, float* Y, int batch, cudaStream_t s) {
    if (batch <= 0) return cudaSuccess;
    mlp_forward_kernel<<<(batch + 127) / 128, 128, 0, s>>>(params, X, Y, batch);
    return cudaGetLastError();
}

}  // namespace fmm

extern "C" fmm_status_t fmm_mlp_forward(const float* params, const float* X, float* Y, int batch, fmm_stream_t s) {
    if (batch < 0 || (batch > 0 && (!params || !X || !Y))) return FMM_ERR_INVALID_ARG;
    return fmm::mlp_forward(params, X, Y, batch, (cudaStream_t)s) == cudaSuccess ? FMM_OK : FMM_ERR_CUDA;
}

extern "C" fmm_status_t fmm_mlp_train_step(float* params, float* adam_m, float* adam_v, int step, float lr,
                                           const float* X, const float* T, int batch, void* workspace,
                                           size_t workspace_bytes, size_t* workspace_needed, float* grad_out,
                                           float* loss_out, fmm_stream_t stream) {
    using namespace fmm;
    if (batch < 0) return FMM_ERR_INVALID_ARG;
    const size_t per = (size_t)(batch > 0 ? batch : 1);
    const size_t need = (4 * per * HID + 2 * per) * sizeof(float) + 256;
    if (workspace_needed) *workspace_needed = need;
    if (!workspace && !params) return FMM_OK;  // size query
    if (batch == 0) return FMM_OK;
    if (!params || !adam_m || !adam_v || !X || !T || step < 1) return FMM_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < need) return FMM_ERR_WORKSPACE;
    float* H1 = static_cast<float*>(workspace);
    float* H2 = H1 + per * HID;
    float* DZ1 = H2 + per * HID;
    float* DZ2 = DZ1 + per * HID;
    float* DY = DZ2 + per * HID;
    float* SQ = DY + per;
    cudaStream_t s = (cudaStream_t)stream;
    mlp_fwdbwd_kernel<<<(batch + 127) / 128, 128, 0, s>>>(params, X, T, batch, H1, H2, DZ1, DZ2, DY, SQ);
    mlp_grad_adam_kernel<<<(NPARAM + 1 + 127) / 128, 128, 0, s>>>(params, adam_m, adam_v, X, H1, H2, DZ1, DZ2, DY, SQ,
                                                                 batch, step, lr, 0.9f, 0.999f, 1e-8f, grad_out,
                                                                 loss_out);
    return cudaGetLastError() == cudaSuccess ? FMM_OK : FMM_ERR_CUDA;
}
