// leaf_gemm.cu -- persistent, warp-specialised tcgen05 leaf GEMM for sm_103a.
//
// Computes, for every group g and batch entry b of a launch,
//     C_b = alpha * A_b * B_b^T + beta * C_b      (A_b: M x K, B_b: N x K, both K-major)
// i.e. the dense classical leaf products of the recursion (the SGEMM leaf of
// Sec. 3.2; c_ij = sum_k a_ik b_kj, Sec. 3.3), all leaves of one level in a
// single launch.
//
// Pipeline per CTA (one CTA per SM, 1 tile of 128 x BN outputs at a time):
//   warp 0        TMA producer: A and B tiles (128 x 32 and BN x 32 fp32,
//                 128-byte swizzle) into a ring of shared-memory stages
//   warp 1        MMA issuer: tcgen05.mma kind::tf32 (M = 128, N = BN, K = 8)
//                 into a double-buffered TMEM accumulator (2 x BN columns)
//   warp 2        TMEM allocation / release
//   warps 4..7    epilogue: tcgen05.ld -> alpha/beta -> global stores
//   warps 8..11   (3xTF32 only) write lo = tf32_rn(x - trunc_tf32(x)) of each
//                 landed stage into a second buffer; the tensor core reads
//                 the raw fp32 tile as hi (kind::tf32 truncates its operands
//                 to 10 mantissa bits on sm_103a, which the GPU tests pin), so
//                 the MMA warp issues lo*hi + hi*lo + hi*hi, fp32 accumulate.
// Every mbarrier wait is bounded (ptx.cuh): a broken pipeline records a
// timeout in the status word and the kernel returns.
#include "fmm_internal.h"
#include "ptx.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace fmm {

template <int BN, int MODE>
struct LeafCfg {
    static constexpr bool kPre32 = MODE == kLeaf3xTF32P;                         // fp32 raw / lo planes via TMA
    static constexpr bool kPre = MODE == kLeafBF16x3P || MODE == kLeafFP16x3P || kPre32;  // split planes via TMA
    // pre-split stages hold A hi|lo and B hi|lo tiles with 64-byte rows: as many bytes as one fp32 stage
    static constexpr int kStages = (MODE == kLeafTF32 || kPre)
                                       ? (BN == 256 ? 4 : 6)
                                       : (BN == 256 ? 2 : 3);
    static constexpr int kABytes = kBM * 128;
    static constexpr int kBBytes = BN * 128;
    static constexpr int kStageBytes = kABytes + kBBytes;
    static constexpr int kKB = kPre32 ? 16 : 32;   // K elements per stage (one 64- or 128-byte row)
    static constexpr bool kSplit = MODE != kLeafTF32 && !kPre;   // split warps + a second buffer per stage
    static constexpr bool k16 = MODE == kLeafBF16x3 || MODE == kLeafFP16x3 || MODE == kLeafBF16x3P ||
                                MODE == kLeafFP16x3P;
    static constexpr int kLoBytes = kSplit ? kStageBytes : 0;
    static constexpr int kTmemCols = 2 * BN;
    static constexpr int kThreads = kSplit ? 384 : 256;
    static constexpr int kBarBytes = 256;
    static constexpr size_t kSmem = 1024 + (size_t)kStages * (kStageBytes + kLoBytes) + kBarBytes;
    static_assert((3 * kStages + 4) * 8 + 16 <= kBarBytes, "barrier area");
    static_assert(kSmem <= 227 * 1024, "shared memory");
    static_assert(kTmemCols == 256 || kTmemCols == 512, "TMEM columns");
};

// hi = rn16(x), lo = rn16(x - hi) for four values, packed as 4 x 16 bits.
template <bool BF16>
__device__ __forceinline__ void split16(float x0, float x1, float x2, float x3, uint2& hi, uint2& lo) {
    if constexpr (BF16) {
        const __nv_bfloat162 h01 = __floats2bfloat162_rn(x0, x1), h23 = __floats2bfloat162_rn(x2, x3);
        const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
        const __nv_bfloat162 l01 = __floats2bfloat162_rn(x0 - f01.x, x1 - f01.y);
        const __nv_bfloat162 l23 = __floats2bfloat162_rn(x2 - f23.x, x3 - f23.y);
        hi = make_uint2(*reinterpret_cast<const uint32_t*>(&h01), *reinterpret_cast<const uint32_t*>(&h23));
        lo = make_uint2(*reinterpret_cast<const uint32_t*>(&l01), *reinterpret_cast<const uint32_t*>(&l23));
    } else {
        const __half2 h01 = __floats2half2_rn(x0, x1), h23 = __floats2half2_rn(x2, x3);
        const float2 f01 = __half22float2(h01), f23 = __half22float2(h23);
        const __half2 l01 = __floats2half2_rn(x0 - f01.x, x1 - f01.y);
        const __half2 l23 = __floats2half2_rn(x2 - f23.x, x3 - f23.y);
        hi = make_uint2(*reinterpret_cast<const uint32_t*>(&h01), *reinterpret_cast<const uint32_t*>(&h23));
        lo = make_uint2(*reinterpret_cast<const uint32_t*>(&l01), *reinterpret_cast<const uint32_t*>(&l23));
    }
}

__device__ __forceinline__ void decode_tile(const GemmGroup* groups, int ng, int raster_m, long long t, int& g,
                                            int& b, int& tm, int& tn) {
    int lo = 0, hi = ng - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (groups[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
    }
    g = lo;
    const GemmGroup& G = groups[g];
    const long long local = t - G.tile_begin;
    const long long per = (long long)G.tiles_m * G.tiles_n;
    b = (int)(local / per);
    const int r = (int)(local - (long long)b * per);
    const int band = raster_m * G.tiles_n;
    const int sr = r / band;
    const int rr = r - sr * band;
    const int gm = min(raster_m, G.tiles_m - sr * raster_m);
    tn = rr / gm;
    tm = sr * raster_m + (rr - tn * gm);
}

// Dynamic tile order of a leaf launch.  The producer (CTA 0's, for a CTA pair)
// takes tiles from the launch-wide counter and publishes its i-th tile in slot i
// of its ring; every other role (MMA issuer, epilogue and split warps, and the
// peer CTA's producer and epilogue warps of a pair) reads the same sequence, so
// all of them walk the same tiles while the CTAs together stay on neighbouring
// tiles (operand panels shared in L2) however their speeds drift, and uneven
// tiles (a batched launch) balance as they are taken.
__device__ __forceinline__ void seq_publish(unsigned long long* slot, unsigned i, long long t) {
    const unsigned long long v = ((unsigned long long)(i + 1) << 32) | (unsigned long long)(unsigned)t;
    asm volatile("st.release.gpu.global.b64 [%0], %1;" ::"l"(slot), "l"(v) : "memory");
}
// The pair's i-th tile, or -1 when the block is aborting or the bounded wait ran
// out (then the status word and the block's abort flag are set).
__device__ __forceinline__ long long seq_read(const unsigned long long* slot, unsigned i, volatile int* abort_flag,
                                              unsigned* status) {
    const unsigned long long want = (unsigned long long)(i + 1);
    unsigned long long t0 = 0;
    for (uint32_t it = 0;; ++it) {
        unsigned long long v;
        asm volatile("ld.acquire.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(slot) : "memory");
        if ((v >> 32) == want) return (long long)(unsigned)(v & 0xffffffffull);
        if ((it & 63u) == 0) {
            if (*abort_flag) return -1;
            const unsigned long long now = global_ns();
            if (it == 0) t0 = now;
            else if (now - t0 > FMM_WAIT_LIMIT_NS) {
                atomicOr(status, FMM_DEV_TIMEOUT_BIT);
                *abort_flag = 1;
                return -1;
            }
        }
    }
}

template <int BN, int MODE>
__global__ void __launch_bounds__(LeafCfg<BN, MODE>::kThreads, 1) leaf_gemm_kernel(const __grid_constant__ GemmArgs args) {
    using Cfg = LeafCfg<BN, MODE>;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw_addr = smem_u32(smem_raw);
    const uint32_t base = (raw_addr + 1023u) & ~1023u;
    uint8_t* base_ptr = smem_raw + (base - raw_addr);
    const uint32_t stage0 = base;                                       // raw stages
    const uint32_t lo0 = base + Cfg::kStages * Cfg::kStageBytes;        // lo copies (3xTF32)
    const uint32_t bar0 = lo0 + Cfg::kStages * Cfg::kLoBytes;
    uint8_t* bar_ptr = base_ptr + (bar0 - base);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar_ptr + 8 * (3 * Cfg::kStages + 4));
    volatile int* abort_flag = reinterpret_cast<volatile int*>(bar_ptr + 8 * (3 * Cfg::kStages + 4) + 8);
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (Cfg::kStages + s); };
    auto ready_bar = [&](int s) { return bar0 + 8u * (2 * Cfg::kStages + s); };
    auto tfull_bar = [&](int a) { return bar0 + 8u * (3 * Cfg::kStages + a); };
    auto tempty_bar = [&](int a) { return bar0 + 8u * (3 * Cfg::kStages + 2 + a); };

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const CUtensorMap* maps = args.ext_maps ? args.ext_maps : args.maps;
    const GemmGroup* groups = args.ext_groups ? args.ext_groups : args.groups;
    const int ng = args.num_groups;
    const long long total = args.total_tiles;
    unsigned* status = args.status;
    const bool dyn = args.tile_counter != nullptr;   // dynamic tile order (this CTA's ring)
    unsigned long long* seq = dyn ? args.tile_seq + (long long)blockIdx.x * kPairSeqSlots : nullptr;

    if (threadIdx.x == 0) {
        for (int s = 0; s < Cfg::kStages; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
            mbar_init(ready_bar(s), 128);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(tfull_bar(a), 1);
            mbar_init(tempty_bar(a), 128);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 2) {
        tmem_alloc(smem_u32(tmem_slot), Cfg::kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true;
            long long issued = 0;
            long long t_next = dyn ? (long long)atomicAdd(args.tile_counter, 1) : 0;
            for (unsigned i = 0; ok; ++i) {
                long long t = blockIdx.x + (long long)i * gridDim.x;
                if (dyn) {   // take the next tile (one ahead) and publish it to this CTA's roles
                    t = t_next;
                    seq_publish(seq + (i % kPairSeqSlots), i, t < total ? t : total);
                    if (t < total) t_next = atomicAdd(args.tile_counter, 1);
                }
                if (t >= total) break;
                int g, b, tm, tn;
                decode_tile(groups, ng, args.raster_m, t, g, b, tm, tn);
                const GemmGroup& G = groups[g];
                const CUtensorMap* ma = maps + G.map_a;
                const CUtensorMap* mb = maps + G.map_b;
                const int nk = (G.K + Cfg::kKB - 1) / Cfg::kKB;
                for (int kb = 0; kb < nk; ++kb) {
                    if (!mbar_wait(empty_bar(stage), phase ^ 1u, abort_flag, status)) { ok = false; break; }
                    mbar_arrive_expect_tx(full_bar(stage), Cfg::kStageBytes);
                    const uint32_t sa = stage0 + stage * Cfg::kStageBytes;
                    if constexpr (Cfg::kPre) {
                        // A hi | B hi | A lo | B lo, 64-byte rows (32 16-bit or 16 fp32 elements of K)
                        const uint32_t bh = sa + kBM * 64, al = bh + BN * 64, bl = al + kBM * 64;
                        const int a0 = tm * kBM, b0 = tn * BN, ab = b + G.a_batch_off, bb = b + G.b_batch_off;
                        tma_load_3d(sa, ma, full_bar(stage), kb * Cfg::kKB, a0, ab);
                        tma_load_3d(bh, mb, full_bar(stage), kb * Cfg::kKB, b0, bb);
                        tma_load_3d(al, maps + G.map_a_lo, full_bar(stage), kb * Cfg::kKB, a0, ab);
                        tma_load_3d(bl, maps + G.map_b_lo, full_bar(stage), kb * Cfg::kKB, b0, bb);
                    } else {
                        tma_load_3d(sa, ma, full_bar(stage), kb * Cfg::kKB, tm * kBM, b + G.a_batch_off);
                        tma_load_3d(sa + Cfg::kABytes, mb, full_bar(stage), kb * Cfg::kKB, tn * BN, b + G.b_batch_off);
                    }
                    ++issued;
                    if (++stage == Cfg::kStages) { stage = 0; phase ^= 1u; }
                }
            }
            if (!ok || *abort_flag) drain_fills(full_bar(0), stage, phase, issued, Cfg::kStages);
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc_full = make_idesc(2u, kBM, BN);
            constexpr uint32_t idesc16_full = make_idesc((MODE == kLeafBF16x3 || MODE == kLeafBF16x3P) ? 1u : 0u, kBM, BN);
            static_assert(idesc_with_n(idesc_full, BN) == idesc_full, "N field of the instruction descriptor");
            int stage = 0;
            uint32_t phase = 0;
            int acc = 0;
            uint32_t acc_phase = 0;
            bool ok = true;
            for (unsigned i = 0; ok; ++i) {
                const long long t = dyn ? seq_read(seq + (i % kPairSeqSlots), i, abort_flag, status)
                                        : blockIdx.x + (long long)i * gridDim.x;
                if (t < 0 || t >= total) break;
                int g, b, tm, tn;
                decode_tile(groups, ng, args.raster_m, t, g, b, tm, tn);
                const int nk = (groups[g].K + Cfg::kKB - 1) / Cfg::kKB;
                // under the dynamic tile order the last tile column runs narrower
                // MMAs; under static round robin a cheaper tile lets its CTA drift
                // off its neighbours' operand panels, which costs more than it saves
                const uint32_t ncols = dyn ? tile_cols(groups[g].N, tn, BN) : (uint32_t)BN;
                const uint32_t idesc = idesc_with_n(idesc_full, ncols);
                const uint32_t idesc16 = idesc_with_n(idesc16_full, ncols);
                if (!mbar_wait(tempty_bar(acc), acc_phase ^ 1u, abort_flag, status)) break;
                tc_fence_after();
                const uint32_t d = tmem_base + (uint32_t)(acc * BN);
                for (int kb = 0; kb < nk; ++kb) {
                    const uint32_t wb = Cfg::kSplit ? ready_bar(stage) : full_bar(stage);
                    if (!mbar_wait(wb, phase, abort_flag, status)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t sa = stage0 + stage * Cfg::kStageBytes;
                    const uint32_t sb = sa + Cfg::kABytes;
                    if constexpr (Cfg::kPre32) {
                        // fp32 raw | lo tiles with 64-byte rows (16 elements of K): A raw | B raw | A lo | B lo
                        const uint32_t ah = stage0 + stage * Cfg::kStageBytes;
                        const uint32_t bh = ah + kBM * 64;
                        const uint32_t al = bh + BN * 64;
                        const uint32_t bl = al + kBM * 64;
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk) {
                            const uint32_t first = (kb == 0 && kk == 0) ? 0u : 1u;
                            const uint64_t ahd = sdesc_kmajor_sw64(ah + kk * 32);
                            const uint64_t bhd = sdesc_kmajor_sw64(bh + kk * 32);
                            mma_tf32(d, sdesc_kmajor_sw64(al + kk * 32), bhd, idesc, first);  // lo_a * hi_b
                            mma_tf32(d, ahd, sdesc_kmajor_sw64(bl + kk * 32), idesc, 1u);     // hi_a * lo_b
                            mma_tf32(d, ahd, bhd, idesc, 1u);                                 // hi_a * hi_b
                        }
                    } else if constexpr (Cfg::k16) {
                        // 16-bit hi/lo tiles, 64-byte rows: A hi | B hi | A lo | B lo (in the
                        // split buffer, or straight from TMA in the stage for pre-split planes)
                        const uint32_t ah = (Cfg::kPre ? stage0 : lo0) + stage * Cfg::kStageBytes;
                        const uint32_t bh = ah + kBM * 64;
                        const uint32_t al = bh + BN * 64;
                        const uint32_t bl = al + kBM * 64;
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk) {
                            const uint32_t first = (kb == 0 && kk == 0) ? 0u : 1u;
                            const uint64_t ahd = sdesc_kmajor_sw64(ah + kk * 32);
                            const uint64_t bhd = sdesc_kmajor_sw64(bh + kk * 32);
                            mma_f16(d, sdesc_kmajor_sw64(al + kk * 32), bhd, idesc16, first);  // lo_a * hi_b
                            mma_f16(d, ahd, sdesc_kmajor_sw64(bl + kk * 32), idesc16, 1u);     // hi_a * lo_b
                            mma_f16(d, ahd, bhd, idesc16, 1u);                                 // hi_a * hi_b
                        }
                    } else {
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint64_t ad = sdesc_kmajor_sw128(sa + kk * 32);
                            const uint64_t bd = sdesc_kmajor_sw128(sb + kk * 32);
                            const uint32_t first = (kb == 0 && kk == 0) ? 0u : 1u;
                            if constexpr (MODE == kLeaf3xTF32) {
                                const uint32_t la = lo0 + stage * Cfg::kStageBytes;
                                const uint64_t ald = sdesc_kmajor_sw128(la + kk * 32);
                                const uint64_t bld = sdesc_kmajor_sw128(la + Cfg::kABytes + kk * 32);
                                mma_tf32(d, ald, bd, idesc, first);  // lo_a * hi_b
                                mma_tf32(d, ad, bld, idesc, 1u);     // hi_a * lo_b
                                mma_tf32(d, ad, bd, idesc, 1u);      // hi_a * hi_b
                            } else {
                                mma_tf32(d, ad, bd, idesc, first);
                            }
                        }
                    }
                    mma_commit(empty_bar(stage));
                    if (++stage == Cfg::kStages) { stage = 0; phase ^= 1u; }
                }
                if (!ok) break;
                mma_commit(tfull_bar(acc));
                acc ^= 1;
                if (acc == 0) acc_phase ^= 1u;
            }
        }
    } else if (warp >= 4 && warp < 8) {
        // ------------------------------------------------ epilogue
        const int q = warp & 3;
        int acc = 0;
        uint32_t acc_phase = 0;
        for (unsigned i = 0;; ++i) {
            long long t = blockIdx.x + (long long)i * gridDim.x;
            if (dyn) {
                if (lane == 0) t = seq_read(seq + (i % kPairSeqSlots), i, abort_flag, status);
                t = __shfl_sync(0xffffffffu, t, 0);
            }
            if (t < 0 || t >= total) break;
            int g, b, tm, tn;
            decode_tile(groups, ng, args.raster_m, t, g, b, tm, tn);
            const GemmGroup& G = groups[g];
            bool ok = mbar_wait(tfull_bar(acc), acc_phase, abort_flag, status);
            if (!__all_sync(0xffffffffu, ok)) break;
            tc_fence_after();
            const int row = tm * kBM + q * 32 + lane;
            const bool row_ok = row < G.M;
            float* crow = G.C + (long long)b * G.c_batch_stride + (long long)(row_ok ? row : 0) * G.ldc;
            float alpha = G.alpha;
            const float beta = G.beta;
            if (Cfg::k16 && G.scale) alpha = alpha / (G.scale[0] * G.scale[1]);  // undo the operand scaling
#pragma unroll 1
            for (int c = 0; c < BN / 32; ++c) {
                uint32_t r[32];
                tmem_ld_32x32b_x32(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * BN + c * 32), r);
                tmem_ld_wait();
                const int col0 = tn * BN + c * 32;
                if (row_ok && col0 < G.N) {
                    float* cp = crow + col0;
                    if (G.vec_ok && col0 + 32 <= G.N) {
#pragma unroll
                        for (int j = 0; j < 32; j += 4) {
                            float4 v;
                            v.x = alpha * __uint_as_float(r[j + 0]);
                            v.y = alpha * __uint_as_float(r[j + 1]);
                            v.z = alpha * __uint_as_float(r[j + 2]);
                            v.w = alpha * __uint_as_float(r[j + 3]);
                            if (beta != 0.0f) {
                                const float4 o = *reinterpret_cast<const float4*>(cp + j);
                                v.x += beta * o.x; v.y += beta * o.y; v.z += beta * o.z; v.w += beta * o.w;
                            }
                            // evict-first: the products are read only after the
                            // whole launch, and must not push operand lines out of L2
                            __stcs(reinterpret_cast<float4*>(cp + j), v);
                        }
                    } else {
                        const int lim = min(32, G.N - col0);
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            if (j < lim) {
                                float v = alpha * __uint_as_float(r[j]);
                                if (beta != 0.0f) v += beta * cp[j];
                                cp[j] = v;
                            }
                        }
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(tempty_bar(acc));
            acc ^= 1;
            if (acc == 0) acc_phase ^= 1u;
        }
    } else if (Cfg::k16 && !Cfg::kPre && warp >= 8) {  // in-kernel 16-bit split
        // ------------------------------------------------ fp32 -> 16-bit hi/lo
        // Reads the 128-byte-swizzled fp32 stage and writes hi = rn16(s*x),
        // lo = rn16(s*x - hi) into 64-byte-swizzled K-major tiles (16-byte chunk
        // j of row r sits at chunk j ^ ((r >> 1) & 3)); s is the group's
        // power-of-two operand scale (1 without one).
        const int tid = threadIdx.x - 256;
        int stage = 0;
        uint32_t phase = 0;
        bool ok = true;
        for (unsigned i = 0; ok; ++i) {
            long long t = blockIdx.x + (long long)i * gridDim.x;
            if (dyn) {
                if (lane == 0) t = seq_read(seq + (i % kPairSeqSlots), i, abort_flag, status);
                t = __shfl_sync(0xffffffffu, t, 0);
            }
            if (t < 0 || t >= total) break;
            int g, b, tm, tn;
            decode_tile(groups, ng, args.raster_m, t, g, b, tm, tn);
            const GemmGroup& G = groups[g];
            const int nk = (G.K + Cfg::kKB - 1) / Cfg::kKB;
            const float s_a = G.scale ? G.scale[0] : 1.0f;
            const float s_b = G.scale ? G.scale[1] : 1.0f;
            for (int kb = 0; kb < nk; ++kb) {
                bool w = mbar_wait(full_bar(stage), phase, abort_flag, status);
                if (!__all_sync(0xffffffffu, w)) { ok = false; break; }
                const float4* src = reinterpret_cast<const float4*>(base_ptr + stage * Cfg::kStageBytes);
                uint8_t* cv = base_ptr + (lo0 - base) + stage * Cfg::kStageBytes;
#pragma unroll 4
                for (int i = tid; i < Cfg::kStageBytes / 16; i += 128) {
                    const bool is_a = i < kBM * 8;
                    const int r = is_a ? (i >> 3) : ((i - kBM * 8) >> 3);
                    const int c = (i & 7) ^ (r & 7);                    // logical 16-byte chunk of the fp32 row
                    const float sc = is_a ? s_a : s_b;
                    const float4 v = src[i];
                    uint2 hi, lo;
                    split16<MODE == kLeafBF16x3>(v.x * sc, v.y * sc, v.z * sc, v.w * sc, hi, lo);
                    const int off = r * 64 + ((((c >> 1) ^ ((r >> 1) & 3))) << 4) + ((c & 1) << 3);
                    uint8_t* hbase = cv + (is_a ? 0 : kBM * 64);
                    uint8_t* lbase = cv + kBM * 64 + BN * 64 + (is_a ? 0 : kBM * 64);
                    *reinterpret_cast<uint2*>(hbase + off) = hi;
                    *reinterpret_cast<uint2*>(lbase + off) = lo;
                }
                fence_proxy_async_smem();
                mbar_arrive(ready_bar(stage));
                if (++stage == Cfg::kStages) { stage = 0; phase ^= 1u; }
            }
        }
    } else if (MODE == kLeaf3xTF32 && warp >= 8) {
        // ------------------------------------------------ hi/lo split
        const int tid = threadIdx.x - 256;
        int stage = 0;
        uint32_t phase = 0;
        bool ok = true;
        for (unsigned i = 0; ok; ++i) {
            long long t = blockIdx.x + (long long)i * gridDim.x;
            if (dyn) {
                if (lane == 0) t = seq_read(seq + (i % kPairSeqSlots), i, abort_flag, status);
                t = __shfl_sync(0xffffffffu, t, 0);
            }
            if (t < 0 || t >= total) break;
            int g, b, tm, tn;
            decode_tile(groups, ng, args.raster_m, t, g, b, tm, tn);
            const int nk = (groups[g].K + Cfg::kKB - 1) / Cfg::kKB;
            for (int kb = 0; kb < nk; ++kb) {
                bool w = mbar_wait(full_bar(stage), phase, abort_flag, status);
                if (!__all_sync(0xffffffffu, w)) { ok = false; break; }
                float4* src = reinterpret_cast<float4*>(base_ptr + stage * Cfg::kStageBytes);
                float4* dst = reinterpret_cast<float4*>(base_ptr + (lo0 - base) + stage * Cfg::kStageBytes);
#pragma unroll 4
                for (int i = tid; i < Cfg::kStageBytes / 16; i += 128) {
                    const float4 v = src[i];
                    float4 l;
                    l.x = tf32_round_rne(v.x - tf32_trunc(v.x));
                    l.y = tf32_round_rne(v.y - tf32_trunc(v.y));
                    l.z = tf32_round_rne(v.z - tf32_trunc(v.z));
                    l.w = tf32_round_rne(v.w - tf32_trunc(v.w));
                    dst[i] = l;
                }
                fence_proxy_async_smem();
                mbar_arrive(ready_bar(stage));
                if (++stage == Cfg::kStages) { stage = 0; phase ^= 1u; }
            }
        }
    }

    __syncthreads();
    if (warp == 2) {
        tc_fence_after();
        tmem_dealloc(tmem_base, Cfg::kTmemCols);
    }
}

// ---------------------------------------------------------------------------------------------
// Pair-of-SMs variant (cta_group::2) for the pre-split modes and TF32.  A cluster of two
// CTAs computes one 256 x 256 output tile: CTA r (cluster rank) loads rows
// [128 r, 128 r + 128) of the A tile and of the B^T tile into its own shared
// memory; CTA 0 issues M = 256 tcgen05.mma instructions that read both CTAs'
// halves, and each CTA's tensor memory holds its 128 rows of the accumulator.
// Per SM this halves the B-operand shared-memory traffic of the single-CTA
// kernel (operand reads + TMA writes 80 KB instead of 120 KB per K step).
//   both CTAs  warp 0: TMA producer into local stages; the copies of both CTAs
//                      complete on CTA 0's full barrier (the cta_group::2 form of
//                      the tensor copy), which CTA 0 arms with the bytes of both
//              warp 2: TMEM allocation, collective over the pair
//              warps 4-7: epilogue of the local 128 rows; each warp then
//                         arrives once on CTA 0's accumulator-free barrier
//   CTA 0      warp 1: MMA issuer; commits are multicast to both CTAs, so each
//              CTA's producer waits on its own empty barrier
//
// FUSED: the last Winograd level inside the leaf launch.  A schedule unit is one
// 256 x 256 tile position of one last-level node; the pair computes the node's
// seven products at that position back to back, in the order P1, P2, P6, P7,
// P5, P3, P4 (each into the next of the two accumulators), and the epilogue
// folds each product into the node's four output quadrants as it lands:
//   P1: X = P1            P2: C11 = X + P2      P6: X = X + P6 (U2)
//   P7: Y = X + P7 (U3)   P5: X = X + P5 (U4), C22 = Y + P5 (U7)
//   P3: C12 = X + P3 (U5) P4: C21 = Y - P4 (U6)
// X and Y are per-CTA running tiles in a global scratch area (read back by the
// same thread that wrote them; stored and loaded with an L2 evict-last policy so
// that they stay on chip while the operand stream passes through L2).  These
// are the fp32 additions of the U-chain in its own order, so the node outputs
// equal those of storing the seven products and running the post-addition pass
// over them, bit for bit; the products themselves never reach memory.
// Leaf index of a unit's pp-th product: node * 7 + kFusedOrder[pp].
__device__ __constant__ int kFusedOrder[7] = {0, 1, 5, 6, 4, 2, 3};

__device__ __forceinline__ uint64_t l2_evict_last_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ void st_keep(float4* a, float4 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(a), "f"(v.x), "f"(v.y),
                 "f"(v.z), "f"(v.w), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ float4 ld_keep(const float4* a, uint64_t pol) {
    float4 v;
    asm volatile("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(a), "l"(pol)
                 : "memory");
    return v;
}

// One 32-column chunk of a node-output quadrant (rows and columns of the leaf
// tile; `o` already points at the quadrant's row) from 32 values in v.
__device__ __forceinline__ void store_quadrant_chunk(float* o, const float (&v)[32], bool row_ok, int col0, int ncols,
                                                     int vec_ok) {
    if (!row_ok || col0 >= ncols) return;
    if (vec_ok && col0 + 32 <= ncols) {
#pragma unroll
        for (int j = 0; j < 32; j += 4)
            __stcs(reinterpret_cast<float4*>(o + j), make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]));
    } else {
        const int lim = min(32, ncols - col0);
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if (j < lim) o[j] = v[j];
    }
}

template <int MODE>
struct PairCfg {
    static constexpr bool kPlain = MODE == kLeafTF32;          // fp32 A | B tiles, one product
    static constexpr int kRows = 128;                          // rows per CTA of A and of B^T
    // 128-byte rows (128-byte swizzle): split planes A hi | B hi | A lo | B lo,
    // 64 KB per stage; TF32: A | B, 32 KB per stage
    static constexpr int kStageBytes = (kPlain ? 2 : 4) * kRows * 128;
    static constexpr int kStages = kPlain ? 6 : 3;
    static constexpr int kKB = (MODE == kLeaf3xTF32P || kPlain) ? 32 : 64;   // K elements per stage (one row)
    static constexpr int kTmemCols = 512;                      // 2 x 256-column accumulators
    static constexpr int kBarBytes = 256;
    static constexpr int kThreads = 256;
    static constexpr size_t kSmem = 1024 + (size_t)kStages * kStageBytes + kBarBytes;
    static_assert((2 * kStages + 4) * 8 + 16 <= kBarBytes, "barrier area");
    static_assert(kSmem <= 227 * 1024, "shared memory");
};

template <int MODE, bool FUSED>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(256, 1)
    leaf_gemm_pair_kernel(const __grid_constant__ GemmArgs args) {
    using Cfg = PairCfg<MODE>;
    constexpr int kProducts = FUSED ? 7 : 1;   // products per schedule unit
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw_addr = smem_u32(smem_raw);
    const uint32_t base = (raw_addr + 1023u) & ~1023u;
    uint8_t* base_ptr = smem_raw + (base - raw_addr);
    const uint32_t stage0 = base;
    const uint32_t bar0 = base + Cfg::kStages * Cfg::kStageBytes;
    uint8_t* bar_ptr = base_ptr + (bar0 - base);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar_ptr + 8 * (2 * Cfg::kStages + 4));
    volatile int* abort_flag = reinterpret_cast<volatile int*>(bar_ptr + 8 * (2 * Cfg::kStages + 4) + 8);
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (Cfg::kStages + s); };
    auto tfull_bar = [&](int a) { return bar0 + 8u * (2 * Cfg::kStages + a); };
    auto tempty_bar = [&](int a) { return bar0 + 8u * (2 * Cfg::kStages + 2 + a); };

    const uint32_t rank = cluster_ctarank();
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const CUtensorMap* maps = args.ext_maps ? args.ext_maps : args.maps;
    const GemmGroup* groups = args.ext_groups ? args.ext_groups : args.groups;
    const int ng = args.num_groups;
    const long long total = args.total_tiles;   // 256 x 256 pair tiles
    const long long pair = blockIdx.x >> 1, npairs = gridDim.x >> 1;
    unsigned* status = args.status;
    const bool dyn = args.tile_counter != nullptr;   // dynamic tile order (the pair's ring)
    unsigned long long* seq = dyn ? args.tile_seq + pair * kPairSeqSlots : nullptr;

    if (threadIdx.x == 0) {
        for (int s = 0; s < Cfg::kStages; ++s) {
            mbar_init(full_bar(s), 1);     // CTA 0's arming arrival (used in CTA 0)
            mbar_init(empty_bar(s), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(tfull_bar(a), 1);
            mbar_init(tempty_bar(a), 8);   // every epilogue warp of both CTAs (used in CTA 0)
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 2) {
        tmem_alloc_pair(smem_u32(tmem_slot), Cfg::kTmemCols);
        tmem_relinquish_pair();
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync();   // the peer's barriers are initialised before any remote arrival
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer (both CTAs)
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true;
            long long issued = 0;
            long long t_next = (dyn && rank == 0) ? (long long)atomicAdd(args.tile_counter, 1) : 0;
            for (unsigned i = 0; ok; ++i) {
                long long t;
                if (!dyn) {
                    t = pair + (long long)i * npairs;
                } else if (rank == 0) {   // take the next tile (one ahead) and publish it
                    t = t_next;
                    seq_publish(seq + (i % kPairSeqSlots), i, t < total ? t : total);
                    if (t < total) t_next = atomicAdd(args.tile_counter, 1);
                } else {
                    t = seq_read(seq + (i % kPairSeqSlots), i, abort_flag, status);
                    if (t < 0) { ok = false; break; }
                }
                if (t >= total) break;
                int g, b, tm, tn;
                decode_tile(groups, ng, args.raster_m, t, g, b, tm, tn);
                const GemmGroup& G = groups[g];
                const int nk = (G.K + Cfg::kKB - 1) / Cfg::kKB;
                // the pair's MMA reads B rows [0, ncols / 2) of the tile from CTA 0
                // and [ncols / 2, ncols) from CTA 1 (ncols < 256 in the last tile
                // column under the dynamic tile order, as in the MMA issuer)
                const int ncols = dyn ? (int)tile_cols(G.N, tn, 256) : 256;
                const int a0 = tm * 256 + (int)rank * Cfg::kRows, b0 = tn * 256 + (int)rank * (ncols / 2);
                for (int pp = 0; pp < kProducts && ok; ++pp) {
                const int leaf = FUSED ? b * 7 + kFusedOrder[pp] : b;
                const int ab = leaf + G.a_batch_off, bb = leaf + G.b_batch_off;
                for (int kb = 0; kb < nk; ++kb) {
                    // the stage is free in this CTA once the MMAs that read it
                    // completed (their commit is multicast to both CTAs)
                    if (!mbar_wait(empty_bar(stage), phase ^ 1u, abort_flag, status)) { ok = false; break; }
                    // CTA 0 arms its full barrier with the bytes of both CTAs; a
                    // peer copy that lands first only drives the tx-count below
                    // zero, which the arming arrival brings back
                    if (rank == 0) mbar_arrive_expect_tx(full_bar(stage), 2 * Cfg::kStageBytes);
                    const uint32_t ah = stage0 + stage * Cfg::kStageBytes;
                    const int x = kb * Cfg::kKB;
                    if constexpr (Cfg::kPlain) {
                        tma_load_3d_pair(ah, maps + G.map_a, full_bar(stage), x, a0, ab);
                        tma_load_3d_pair(ah + Cfg::kRows * 128, maps + G.map_b, full_bar(stage), x, b0, bb);
                    } else {
                        const uint32_t bh = ah + Cfg::kRows * 128, al = bh + Cfg::kRows * 128, bl = al + Cfg::kRows * 128;
                        tma_load_3d_pair(ah, maps + G.map_a, full_bar(stage), x, a0, ab);
                        tma_load_3d_pair(bh, maps + G.map_b, full_bar(stage), x, b0, bb);
                        tma_load_3d_pair(al, maps + G.map_a_lo, full_bar(stage), x, a0, ab);
                        tma_load_3d_pair(bl, maps + G.map_b_lo, full_bar(stage), x, b0, bb);
                    }
                    ++issued;
                    if (++stage == Cfg::kStages) { stage = 0; phase ^= 1u; }
                }
                }
            }
            // the copies of both CTAs complete on CTA 0's full barriers, and the
            // closing cluster barrier holds CTA 1 until CTA 0 has drained them
            if (rank == 0 && (!ok || *abort_flag)) drain_fills(full_bar(0), stage, phase, issued, Cfg::kStages);
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer (CTA 0)
        if (lane == 0 && rank == 0) {
            constexpr uint32_t fmt = (MODE == kLeaf3xTF32P || MODE == kLeafTF32) ? 2u : (MODE == kLeafBF16x3P ? 1u : 0u);
            constexpr uint32_t idesc_full = make_idesc(fmt, 256, 256);
            int stage = 0;
            uint32_t phase = 0;
            int acc = 0;
            uint32_t acc_phase = 0;
            bool ok = true;
            for (unsigned i = 0; ok; ++i) {
                const long long t = dyn ? seq_read(seq + (i % kPairSeqSlots), i, abort_flag, status)
                                        : pair + (long long)i * npairs;
                if (t < 0 || t >= total) break;
                int g, b, tm, tn;
                decode_tile(groups, ng, args.raster_m, t, g, b, tm, tn);
                const int nk = (groups[g].K + Cfg::kKB - 1) / Cfg::kKB;
                const uint32_t idesc = idesc_with_n(idesc_full, dyn ? tile_cols(groups[g].N, tn, 256) : 256u);
                for (int pp = 0; pp < kProducts && ok; ++pp) {
                if (!mbar_wait_cluster(tempty_bar(acc), acc_phase ^ 1u, abort_flag, status)) { ok = false; break; }
                tc_fence_after();
                const uint32_t d = tmem_base + (uint32_t)(acc * 256);
                for (int kb = 0; kb < nk; ++kb) {
                    // both CTAs' copies complete on this CTA's barrier (complete_tx of
                    // the async proxy, read by the async proxy): a CTA-scope acquire
                    // suffices, and avoids a cluster-scope fence per stage
                    if (!mbar_wait(full_bar(stage), phase, abort_flag, status)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t ah = stage0 + stage * Cfg::kStageBytes;
                    if constexpr (Cfg::kPlain) {
                        // fp32 tiles with 128-byte rows (32 elements of K): 4 MMAs of K = 8
                        const uint32_t bh = ah + Cfg::kRows * 128;
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)
                            mma_tf32_pair(d, sdesc_kmajor_sw128(ah + kk * 32), sdesc_kmajor_sw128(bh + kk * 32), idesc,
                                          (kb == 0 && kk == 0) ? 0u : 1u);
                    } else {
                        // hi / lo tiles with 128-byte rows: 4 MMAs of 32 bytes of K per product
                        const uint32_t bh = ah + Cfg::kRows * 128, al = bh + Cfg::kRows * 128, bl = al + Cfg::kRows * 128;
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint32_t first = (kb == 0 && kk == 0) ? 0u : 1u;
                            const uint64_t ahd = sdesc_kmajor_sw128(ah + kk * 32);
                            const uint64_t bhd = sdesc_kmajor_sw128(bh + kk * 32);
                            const uint64_t ald = sdesc_kmajor_sw128(al + kk * 32);
                            const uint64_t bld = sdesc_kmajor_sw128(bl + kk * 32);
                            if constexpr (MODE == kLeaf3xTF32P) {
                                mma_tf32_pair(d, ald, bhd, idesc, first);  // lo_a * hi_b
                                mma_tf32_pair(d, ahd, bld, idesc, 1u);     // hi_a * lo_b
                                mma_tf32_pair(d, ahd, bhd, idesc, 1u);     // hi_a * hi_b
                            } else {
                                mma_f16_pair(d, ald, bhd, idesc, first);
                                mma_f16_pair(d, ahd, bld, idesc, 1u);
                                mma_f16_pair(d, ahd, bhd, idesc, 1u);
                            }
                        }
                    }
                    mma_commit_pair(empty_bar(stage), (uint16_t)0x3);
                    if (++stage == Cfg::kStages) { stage = 0; phase ^= 1u; }
                }
                if (!ok) break;
                mma_commit_pair(tfull_bar(acc), (uint16_t)0x3);
                acc ^= 1;
                if (acc == 0) acc_phase ^= 1u;
                }
            }
        }
    } else if (warp >= 4) {
        // ------------------------------------------------ epilogue (both CTAs)
        const int q = warp & 3;
        int acc = 0;
        uint32_t acc_phase = 0;
        // FUSED: this CTA's running tiles X, Y (128 rows x 256 columns each),
        // float4 (row r, columns c*32 + 4jj .. +3) at index (c * 8 + jj) * 128 + r,
        // so a warp's accesses are 512 contiguous bytes
        float4* X4 = nullptr;
        uint64_t keep = 0;
        if constexpr (FUSED) {
            X4 = reinterpret_cast<float4*>(args.fuse_scratch) + (size_t)blockIdx.x * (2 * 128 * 256 / 4) + q * 32 + lane;
            keep = l2_evict_last_policy();
        }
        bool stop = false;
        for (unsigned i = 0; !stop; ++i) {
            long long t = pair + (long long)i * npairs;
            if (dyn) {
                if (lane == 0) t = seq_read(seq + (i % kPairSeqSlots), i, abort_flag, status);
                t = __shfl_sync(0xffffffffu, t, 0);
            }
            if (t < 0 || t >= total) break;
            int g, b, tm, tn;
            decode_tile(groups, ng, args.raster_m, t, g, b, tm, tn);
            const GemmGroup& G = groups[g];
            const int row = tm * 256 + (int)rank * Cfg::kRows + q * 32 + lane;
            const bool row_ok = row < G.M;
            float alpha = G.alpha;
            const float beta = G.beta;
            if (MODE == kLeafFP16x3P && G.scale) alpha = alpha / (G.scale[0] * G.scale[1]);
            for (int pp = 0; pp < kProducts; ++pp) {
            bool ok = mbar_wait(tfull_bar(acc), acc_phase, abort_flag, status);
            if (!__all_sync(0xffffffffu, ok)) { stop = true; break; }
            tc_fence_after();
            if constexpr (!FUSED) {
            float* crow = G.C + (long long)b * G.c_batch_stride + (long long)(row_ok ? row : 0) * G.ldc;
#pragma unroll 1
            for (int c = 0; c < 256 / 32; ++c) {
                uint32_t r[32];
                tmem_ld_32x32b_x32(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * 256 + c * 32), r);
                tmem_ld_wait();
                const int col0 = tn * 256 + c * 32;
                if (row_ok && col0 < G.N) {
                    float* cp = crow + col0;
                    if (G.vec_ok && col0 + 32 <= G.N) {
#pragma unroll
                        for (int j = 0; j < 32; j += 4) {
                            float4 v;
                            v.x = alpha * __uint_as_float(r[j + 0]);
                            v.y = alpha * __uint_as_float(r[j + 1]);
                            v.z = alpha * __uint_as_float(r[j + 2]);
                            v.w = alpha * __uint_as_float(r[j + 3]);
                            if (beta != 0.0f) {
                                const float4 o = *reinterpret_cast<const float4*>(cp + j);
                                v.x += beta * o.x; v.y += beta * o.y; v.z += beta * o.z; v.w += beta * o.w;
                            }
                            // evict-first: the products are read only after the
                            // whole launch, and must not push operand lines out of L2
                            __stcs(reinterpret_cast<float4*>(cp + j), v);
                        }
                    } else {
                        const int lim = min(32, G.N - col0);
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            if (j < lim) {
                                float v = alpha * __uint_as_float(r[j]);
                                if (beta != 0.0f) v += beta * cp[j];
                                cp[j] = v;
                            }
                        }
                    }
                }
            }
            } else {
            // node output: quadrant (qi, qj) at rows qi * M + row, columns qj * N + col
            float* node = G.C + (long long)b * G.c_batch_stride + (long long)(row_ok ? row : 0) * G.ldc;
            const long long qrow = (long long)G.M * G.ldc;
#pragma unroll 1
            for (int c = 0; c < 256 / 32; ++c) {
                uint32_t r[32];
                tmem_ld_32x32b_x32(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * 256 + c * 32), r);
                tmem_ld_wait();
                const int col0 = tn * 256 + c * 32;
                float4* xs = X4 + c * 8 * 128;
                float4* ys = xs + 128 * 256 / 4;
                float v[32], o[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = alpha * __uint_as_float(r[j]);
                if (pp == 0) {                                      // P1: X = P1
#pragma unroll
                    for (int jj = 0; jj < 8; ++jj)
                        st_keep(xs + jj * 128, make_float4(v[4 * jj], v[4 * jj + 1], v[4 * jj + 2], v[4 * jj + 3]), keep);
                } else if (pp == 2 || pp == 3) {                    // P6: X = X + P6;  P7: Y = X + P7
                    float4 x[8];
#pragma unroll
                    for (int jj = 0; jj < 8; ++jj) x[jj] = ld_keep(xs + jj * 128, keep);
                    float4* dst = pp == 2 ? xs : ys;
#pragma unroll
                    for (int jj = 0; jj < 8; ++jj)
                        st_keep(dst + jj * 128, make_float4(x[jj].x + v[4 * jj], x[jj].y + v[4 * jj + 1],
                                                            x[jj].z + v[4 * jj + 2], x[jj].w + v[4 * jj + 3]), keep);
                } else if (pp == 4) {                               // P5: X = X + P5 (U4), C22 = Y + P5 (U7)
                    float4 x[8], y[8];
#pragma unroll
                    for (int jj = 0; jj < 8; ++jj) { x[jj] = ld_keep(xs + jj * 128, keep); y[jj] = ld_keep(ys + jj * 128, keep); }
#pragma unroll
                    for (int jj = 0; jj < 8; ++jj) {
                        st_keep(xs + jj * 128, make_float4(x[jj].x + v[4 * jj], x[jj].y + v[4 * jj + 1],
                                                           x[jj].z + v[4 * jj + 2], x[jj].w + v[4 * jj + 3]), keep);
                        o[4 * jj] = y[jj].x + v[4 * jj];
                        o[4 * jj + 1] = y[jj].y + v[4 * jj + 1];
                        o[4 * jj + 2] = y[jj].z + v[4 * jj + 2];
                        o[4 * jj + 3] = y[jj].w + v[4 * jj + 3];
                    }
                    store_quadrant_chunk(node + qrow + G.N + col0, o, row_ok, col0, G.N, G.vec_ok);
                } else {                                            // P2 -> C11, P3 -> C12 (from X); P4 -> C21 (from Y)
                    const float4* src = pp == 6 ? ys : xs;
                    float4 x[8];
#pragma unroll
                    for (int jj = 0; jj < 8; ++jj) x[jj] = ld_keep(src + jj * 128, keep);
                    if (pp == 6) {
#pragma unroll
                        for (int jj = 0; jj < 8; ++jj) {
                            o[4 * jj] = x[jj].x - v[4 * jj];
                            o[4 * jj + 1] = x[jj].y - v[4 * jj + 1];
                            o[4 * jj + 2] = x[jj].z - v[4 * jj + 2];
                            o[4 * jj + 3] = x[jj].w - v[4 * jj + 3];
                        }
                    } else {
#pragma unroll
                        for (int jj = 0; jj < 8; ++jj) {
                            o[4 * jj] = x[jj].x + v[4 * jj];
                            o[4 * jj + 1] = x[jj].y + v[4 * jj + 1];
                            o[4 * jj + 2] = x[jj].z + v[4 * jj + 2];
                            o[4 * jj + 3] = x[jj].w + v[4 * jj + 3];
                        }
                    }
                    float* dst = pp == 1 ? node : pp == 5 ? node + G.N : node + qrow;
                    store_quadrant_chunk(dst + col0, o, row_ok, col0, G.N, G.vec_ok);
                }
            }
            }
            // every lane's tensor-memory reads are complete (wait::ld above);
            // one arrival per warp releases the accumulator to CTA 0's MMAs
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                if (rank == 0) mbar_arrive(tempty_bar(acc));
                else mbar_arrive_cluster(tempty_bar(acc), 0);
            }
            acc ^= 1;
            if (acc == 0) acc_phase ^= 1u;
            }
        }
    }

    __syncthreads();
    cluster_sync();   // every pair MMA and remote arrival of both CTAs is done
    if (warp == 2) {
        tc_fence_after();
        tmem_dealloc_pair(tmem_base, Cfg::kTmemCols);
    }
}

template <int MODE, bool FUSED>
static cudaError_t launch_pair_impl(const GemmArgs& args, int num_sms, cudaStream_t stream) {
    using Cfg = PairCfg<MODE>;
    auto kern = leaf_gemm_pair_kernel<MODE, FUSED>;
    static bool attr_done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !attr_done[dev]) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::kSmem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_done[dev] = true;
    }
    // persistent pairs: only as many clusters as can be resident at once (a
    // cluster's two CTAs must share a GPC, so this can be below num_sms / 2)
    static int max_clusters[64] = {};
    if (dev >= 0 && dev < 64 && max_clusters[dev] == 0) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr;
        attr.id = cudaLaunchAttributeClusterDimension;
        attr.val.clusterDim.x = 2;
        attr.val.clusterDim.y = 1;
        attr.val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)(num_sms & ~1));
        cfg.blockDim = dim3(Cfg::kThreads);
        cfg.dynamicSmemBytes = Cfg::kSmem;
        cfg.attrs = &attr;
        cfg.numAttrs = 1;
        int n = 0;
        e = cudaOccupancyMaxActiveClusters(&n, (void*)kern, &cfg);
        if (e != cudaSuccess || n <= 0) {
            cudaGetLastError();
            n = num_sms / 2;
        }
        max_clusters[dev] = n < num_sms / 2 ? n : num_sms / 2;
    }
    long long cap = (dev >= 0 && dev < 64) ? max_clusters[dev] : num_sms / 2;
    if (args.tile_counter && cap > kMaxSeqRings) cap = kMaxSeqRings;   // one ring per pair
    if (FUSED && cap > kFuseMaxPairs) cap = kFuseMaxPairs;           // one pair of running tiles per pair
    if (args.total_tiles <= 0) return cudaSuccess;
    const long long pairs = args.total_tiles < cap ? args.total_tiles : cap;
    kern<<<(unsigned)(2 * pairs), Cfg::kThreads, Cfg::kSmem, stream>>>(args);
    return cudaGetLastError();
}

cudaError_t launch_leaf_gemm_pair(const GemmArgs& args, int mode, int num_sms, cudaStream_t stream) {
    if (args.fuse_scratch) {
        // the fused last level reads every group as Winograd nodes of seven leaves
        if (args.ext_groups || args.num_groups != 1 || args.groups[0].beta != 0.0f) return cudaErrorInvalidValue;
        switch (mode) {
            case kLeaf3xTF32P: return launch_pair_impl<kLeaf3xTF32P, true>(args, num_sms, stream);
            case kLeafBF16x3P: return launch_pair_impl<kLeafBF16x3P, true>(args, num_sms, stream);
            case kLeafFP16x3P: return launch_pair_impl<kLeafFP16x3P, true>(args, num_sms, stream);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (mode) {
        case kLeafTF32: return launch_pair_impl<kLeafTF32, false>(args, num_sms, stream);
        case kLeaf3xTF32P: return launch_pair_impl<kLeaf3xTF32P, false>(args, num_sms, stream);
        case kLeafBF16x3P: return launch_pair_impl<kLeafBF16x3P, false>(args, num_sms, stream);
        case kLeafFP16x3P: return launch_pair_impl<kLeafFP16x3P, false>(args, num_sms, stream);
        default: return cudaErrorInvalidValue;
    }
}

template <int BN, int MODE>
static cudaError_t launch_impl(const GemmArgs& args, int num_sms, cudaStream_t stream) {
    using Cfg = LeafCfg<BN, MODE>;
    auto kern = leaf_gemm_kernel<BN, MODE>;
    // once per device and instantiation (keeps later launches free of other API
    // calls, e.g. while a stream is being captured into a CUDA graph)
    static bool attr_done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !attr_done[dev]) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::kSmem);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_done[dev] = true;
    }
    if (args.total_tiles <= 0) return cudaSuccess;
    long long grid = args.total_tiles < num_sms ? args.total_tiles : num_sms;
    if (args.tile_counter && grid > kMaxSeqRings) grid = kMaxSeqRings;   // one ring per CTA
    kern<<<(unsigned)grid, Cfg::kThreads, Cfg::kSmem, stream>>>(args);
    return cudaGetLastError();
}

size_t leaf_smem_bytes(int mode, int bn) {
    if (mode == kLeafTF32) return bn == 256 ? LeafCfg<256, kLeafTF32>::kSmem : LeafCfg<128, kLeafTF32>::kSmem;
    return bn == 256 ? LeafCfg<256, kLeaf3xTF32>::kSmem : LeafCfg<128, kLeaf3xTF32>::kSmem;
}

cudaError_t launch_leaf_gemm(const GemmArgs& args, int mode, int bn, int num_sms, cudaStream_t stream) {
#define FMM_LEAF(MODE_)                                                                 \
    return bn == 256 ? launch_impl<256, MODE_>(args, num_sms, stream)                  \
                     : launch_impl<128, MODE_>(args, num_sms, stream)
    switch (mode) {
        case kLeafTF32: FMM_LEAF(kLeafTF32);
        case kLeafBF16x3: FMM_LEAF(kLeafBF16x3);
        case kLeafFP16x3: FMM_LEAF(kLeafFP16x3);
        case kLeafBF16x3P: FMM_LEAF(kLeafBF16x3P);
        case kLeafFP16x3P: FMM_LEAF(kLeafFP16x3P);
        case kLeaf3xTF32P: FMM_LEAF(kLeaf3xTF32P);
        default: FMM_LEAF(kLeaf3xTF32);
    }
#undef FMM_LEAF
}

}  // namespace fmm
