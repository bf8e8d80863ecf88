// fmm.cu -- C ABI, plans and the recursion scheduler.
//
// Schedule of one Winograd call of depth d (breadth-first: every node of a
// level is processed by one launch per step):
//   level 0           root pre-additions read the caller's A (row-major,
//                     virtually zero-padded to M0 x K0) and B (transposed on
//                     the fly) and write all 7 child operands of each side;
//   levels 1..d-2     pre-additions write all 7 child operands per node;
//   level d-1         pre-additions write only S1..S4 / T1..T4; the leaves read
//                     the three plain quadrants (P1, P2, P4 / P1, P2, P3) as
//                     strided views of the parent operands;
//   leaves            one persistent tcgen05 launch over all 7^d products;
//   levels d-1..0     post-additions U1..U7; the root applies alpha/beta into C.
// The padded sizes M0, K0, N0 are multiples of 4 * 2^d so that every level
// splits exactly (Eq. 1's ceil/floor split then has equal halves) and every
// operand row starts on a 16-byte boundary, as the TMA tile loads require.
// Zero padding changes no value of the product: padded rows/columns only ever
// add exact zeros.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <cmath>
#include <mutex>
#include <new>
#include <vector>

#include <cudaTypedefs.h>

#include "../../include/fmm.h"
#include "fmm_internal.h"

using namespace fmm;

namespace {

thread_local char g_last_error[512] = "";

fmm_status_t cuda_fail(cudaError_t e, const char* where) {
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%d)", where, cudaGetErrorString(e), (int)e);
    return FMM_ERR_CUDA;
}
#define FMM_CUDA(call)                                          \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);     \
    } while (0)

struct DeviceInfo {
    int ok = 0;
    int num_sms = 0;
    int major = 0, minor = 0;
};

std::mutex g_mu;
DeviceInfo g_dev[64];
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

fmm_status_t device_info(DeviceInfo* out) {
    int dev = 0;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) {
        cudaGetLastError();
        snprintf(g_last_error, sizeof(g_last_error), "no CUDA device");
        return FMM_ERR_NO_DEVICE;
    }
    FMM_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_mu);
    if (dev < 0 || dev >= 64) return FMM_ERR_NO_DEVICE;
    DeviceInfo& d = g_dev[dev];
    if (!d.ok) {
        FMM_CUDA(cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, dev));
        FMM_CUDA(cudaDeviceGetAttribute(&d.major, cudaDevAttrComputeCapabilityMajor, dev));
        FMM_CUDA(cudaDeviceGetAttribute(&d.minor, cudaDevAttrComputeCapabilityMinor, dev));
        d.ok = 1;
    }
    if (!(d.major == 10 && d.minor == 3)) {
        snprintf(g_last_error, sizeof(g_last_error), "device is sm_%d%d; this library is built for sm_103a",
                 d.major, d.minor);
        return FMM_ERR_NO_DEVICE;
    }
    if (!g_encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cuda_fail(e, "cuTensorMapEncodeTiled");
        g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    *out = d;
    return FMM_OK;
}

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
inline long long rup(long long x, long long a) { return (x + a - 1) / a * a; }
inline long long ipow7(int l) { long long r = 1; while (l-- > 0) r *= 7; return r; }

// 3-D K-major fp32 tile map: dims {cols, rows, batch}, box {32, box_rows, 1},
// 128-byte swizzle, zero fill outside the dims.
fmm_status_t encode_map(CUtensorMap* map, const float* base, long long cols, long long rows, long long batch,
                        long long ld, long long batch_stride, int box_rows) {
    if (cols <= 0 || rows <= 0 || batch <= 0) {
        snprintf(g_last_error, sizeof(g_last_error), "empty tensor map");
        return FMM_ERR_INVALID_ARG;
    }
    if ((reinterpret_cast<uintptr_t>(base) & 15) || (ld * 4) % 16 || (batch_stride * 4) % 16)
        return FMM_ERR_ALIGNMENT;
    cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)batch};
    cuuint64_t strides[2] = {(cuuint64_t)(ld * 4), (cuuint64_t)(batch_stride * 4)};
    cuuint32_t box[3] = {32u, (cuuint32_t)box_rows, 1u};
    cuuint32_t estr[3] = {1u, 1u, 1u};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        snprintf(g_last_error, sizeof(g_last_error), "cuTensorMapEncodeTiled failed (%d)", (int)r);
        return FMM_ERR_CUDA;
    }
    return FMM_OK;
}

// 3-D K-major tile map of a split plane: 64-byte rows (32 16-bit or 16 fp32
// elements of K), box {row, box_rows, 1}, 64-byte swizzle.
// Tensor map over split planes: wide = the CTA-pair kernel's 128-byte box rows
// with 128-byte swizzle, else the single-CTA kernel's 64-byte rows with 64-byte
// swizzle.
fmm_status_t encode_map16(CUtensorMap* map, const void* base, int kind, long long cols, long long rows,
                          long long batch, long long ld, long long batch_stride, int box_rows, bool wide = false) {
    if (cols <= 0 || rows <= 0 || batch <= 0) return FMM_ERR_INVALID_ARG;
    const long long es = kind == kSplitTF32 ? 4 : 2;
    if ((reinterpret_cast<uintptr_t>(base) & 15) || (ld * es) % 16 || (batch_stride * es) % 16) return FMM_ERR_ALIGNMENT;
    cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)batch};
    cuuint64_t strides[2] = {(cuuint64_t)(ld * es), (cuuint64_t)(batch_stride * es)};
    cuuint32_t box[3] = {(cuuint32_t)((wide ? 128 : 64) / es), (cuuint32_t)box_rows, 1u};
    cuuint32_t estr[3] = {1u, 1u, 1u};
    const CUtensorMapDataType dt = kind == kSplitTF32   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : kind == kSplitBF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                        : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    CUresult r = g_encode(map, dt, 3, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          wide ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        snprintf(g_last_error, sizeof(g_last_error), "cuTensorMapEncodeTiled (16-bit) failed (%d)", (int)r);
        return FMM_ERR_CUDA;
    }
    return FMM_OK;
}

struct Level {
    long long m, k, n;        // node operand sizes at this level
    long long nodes;          // 7^l
    float* achild = nullptr;  // full: 7^(l+1) child A operands; sums-only: 4 S per node
    float* bchild = nullptr;  // same, transposed B side
    int full = 1;
    float* cnode = nullptr;   // node outputs (levels >= 1)
};

}  // namespace

struct fmm_plan_s {
    long long M, N, K, lda, ldb, ldc;
    fmm_options_t opt;
    int depth;
    int bn;
    int mode;                 // LeafMode
    long long M0, K0, N0;     // padded root sizes (Winograd)
    long long Mw, Kw, Nw;     // sizes the recursion covers (all of M, K, N; the even core when peeling)
    int peel = 0;
    fmm_odd_t odd = FMM_ODD_PAD;   // odd-size mode after resolving FMM_ODD_AUTO
    // peel granule of M and N (K: 4 * 2^d): 4 * 2^d, or a whole leaf tile
    // times 2^d for FMM_ODD_TILE
    long long peel_gm = 0, peel_gn = 0;
    float border_beta = 0.f;
    // pre-split plans: the leaf operands are written as hi / lo planes (SplitKind)
    int pre16 = 0;
    int split_kind = 0;
    int pair = 0;        // leaves on CTA pairs (cta_group::2), 256 x 256 tiles
    int tile_req = 256;  // leaf tile the plan was made for (512: CTA pairs where the precision allows)
    int rmul = 0;        // classical recursion (Table 1) depth; the Winograd depth is then 0
    // the last Winograd level inside the leaf launch (CTA pairs, split planes,
    // depth 2 to 4): the launch writes the level-(d-1) node outputs, not the
    // 7^d products, through per-pair running tiles (fuse_scratch)
    int fused = 0;
    float* fuse_scratch = nullptr;
    char* tile_sched = nullptr;   // dynamic tile order of the leaf launches (counter + rings)
    int sched = 1;                // 0: static tile order, no scheduling area (the allocation-free entry)
    void* a16[2] = {};   // hi, lo planes of the leaf A operands (stack or the whole A)
    void* b16[2] = {};   // hi, lo planes of the leaf B^T operands
    long long ld16 = 0;
    size_t es16() const { return split_kind == kSplitTF32 ? 4 : 2; }
    // depth >= 4: the last three levels of pre-additions (split-plane plans) and
    // of post-additions run as one pass each; the middle levels are never stored
    bool fuse_pre() const { return pre16 && depth >= 4; }
    bool fuse_post() const { return depth >= 4; }
    // depth 2: both levels at once from / into the caller's matrices
    bool fuse_root_pre() const { return pre16 && depth == 2; }
    bool fuse_root_post() const { return depth == 2; }
    // depth 3: all three levels at once from / into the caller's matrices
    bool fuse_root_pre3() const { return pre16 && depth == 3; }
    bool fuse_root_post3() const { return depth == 3; }
    // algorithmic bytes (reads + writes the passes need) of the last call's
    // addition phases: [0] before the leaf launch, [1] after it
    double acct[2] = {0.0, 0.0};
    // host-resident operands: root level depth-first over the 7 products with
    // quadrant transfers on two copy streams; children run on device buffers
    int host = 0;
    fmm_plan_s* child = nullptr;
    float* hq[27] = {};               // A quads 0-3, B quads 4-7, S 8-11, T 12-15, P 16-22, C quads 23-26
    long long hm = 0, hk = 0, hn = 0; // quadrant sizes
    char* child_ws = nullptr;
    size_t child_ws_bytes = 0;
    cudaStream_t s_h2d = nullptr, s_d2h = nullptr;
    cudaEvent_t hev[8] = {};
    // library-default host copies: the input transfers of recent calls that
    // used the copy engines, each bracketed by a pair of timing events in a
    // ring, judged at a later call once complete (callers run ahead of the GPU)
    static constexpr int kJudgeRing = 16;
    cudaEvent_t hx[kJudgeRing][2] = {};
    double hx_bytes[kJudgeRing] = {};   // bytes a slot's transfers moved (0: free)
    int hx_next = 0;
    long long host_calls = 0;
    int host_sm_latched = 0;    // the copy engines stalled: SM copies from now on
    // FP16x3: device operand scales {s_a, s_b} and reduction scratch, inside the status block
    float* fp16_scale() const { return scale_override ? scale_override : reinterpret_cast<float*>(status + 16); }
    float* scale_override = nullptr;   // batched sub-plans: the problem's own {s_a, s_b}
    unsigned* fp16_scratch() const { return status + 24; }
    char* ws = nullptr;
    size_t ws_bytes = 0;
    unsigned* status = nullptr;
    Level lv[8];
    float* P = nullptr;       // leaf products
    float* Bt = nullptr;      // classical: transposed B
    float* Acopy = nullptr;   // classical: aligned copy of A when A is not TMA-aligned
    long long ld_bt = 0, ld_acopy = 0;
    int num_sms = 0;
    cudaStream_t last_stream = nullptr;
    // phase profiling: events around pre-additions / leaves / post-additions
    struct EvSet { cudaEvent_t e[4]; };
    int profile = 0;
    EvSet* cur = nullptr;
    std::vector<EvSet> ev_pending, ev_free;
    double prof_ms[3] = {0.0, 0.0, 0.0};
    long long launches = 0, calls = 0;
};

namespace {

// Workspace carve-out.  `base` may be null (size query).
struct Carver {
    char* base;
    size_t off = 0;
    explicit Carver(char* b) : base(b) {}
    template <class T>
    T* take(size_t count) {
        off = align_up(off, 256);
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

void make_child(const fmm_plan_s* p, fmm_plan_s& c);

void layout(fmm_plan_s* p, char* ws, size_t* needed) {
    Carver cv(ws);
    p->status = cv.take<unsigned>(64);
    if (p->sched && !p->host) p->tile_sched = cv.take<char>(kTileSchedBytes);
    const int d = p->depth;
    if (p->host) {
        // device copies of the root quadrants; the children run on these
        const long long g = d > 0 ? (4LL << d) : 4;
        p->M0 = rup(p->M, g); p->K0 = rup(p->K, g); p->N0 = rup(p->N, g);
        p->Mw = p->M; p->Kw = p->K; p->Nw = p->N;
        const int parts = d > 0 ? 2 : 1;   // depth 0: one "quadrant" = the whole matrix
        p->hm = p->M0 / parts; p->hk = p->K0 / parts; p->hn = p->N0 / parts;
        const size_t qa = (size_t)(p->hm * p->hk), qb = (size_t)(p->hk * p->hn), qc = (size_t)(p->hm * p->hn);
        const int nq = d > 0 ? 4 : 1;
        for (int i = 0; i < nq; ++i) p->hq[i] = cv.take<float>(qa);
        for (int i = 0; i < nq; ++i) p->hq[4 + i] = cv.take<float>(qb);
        for (int i = 0; i < nq; ++i) p->hq[23 + i] = cv.take<float>(qc);
        if (d > 0) {
            for (int i = 0; i < 4; ++i) p->hq[8 + i] = cv.take<float>(qa);
            for (int i = 0; i < 4; ++i) p->hq[12 + i] = cv.take<float>(qb);
            for (int i = 0; i < 7; ++i) p->hq[16 + i] = cv.take<float>(qc);
        }
        fmm_plan_s c;
        make_child(p, c);
        size_t cneed = 0;
        layout(&c, nullptr, &cneed);
        p->child_ws_bytes = cneed;
        p->child_ws = cv.take<char>(cneed);
        if (needed) *needed = align_up(cv.off, 256);
        return;
    }
    if (d == 0 && p->pre16) {
        p->ld16 = rup(p->K, 128 / (long long)p->es16());   // 128-byte row pitch
        for (int i = 0; i < 2; ++i) p->a16[i] = cv.take<char>((size_t)p->M * p->ld16 * p->es16());
        for (int i = 0; i < 2; ++i) p->b16[i] = cv.take<char>((size_t)p->N * p->ld16 * p->es16());
    } else if (d == 0) {
        p->ld_bt = rup(p->K, 4);
        p->Bt = cv.take<float>((size_t)p->N * p->ld_bt);
        p->ld_acopy = rup(p->K, 4);
        const bool a_ok = (p->lda % 4) == 0;  // base alignment checked per call
        (void)a_ok;
        p->Acopy = cv.take<float>((size_t)p->M * p->ld_acopy);
    } else {
        const long long g = 4LL << d;
        if (p->peel) {
            const long long gm = p->peel_gm ? p->peel_gm : g, gn = p->peel_gn ? p->peel_gn : g;
            p->Mw = p->M / gm * gm;
            p->Kw = p->K / g * g;
            p->Nw = p->N / gn * gn;
            p->M0 = p->Mw;
            p->K0 = p->Kw;
            p->N0 = p->Nw;
        } else {
            p->Mw = p->M;
            p->Kw = p->K;
            p->Nw = p->N;
            p->M0 = rup(p->M, g);
            p->K0 = rup(p->K, g);
            p->N0 = rup(p->N, g);
        }
        for (int l = 0; l <= d; ++l) {
            p->lv[l].m = p->M0 >> l;
            p->lv[l].k = p->K0 >> l;
            p->lv[l].n = p->N0 >> l;
            p->lv[l].nodes = ipow7(l);
        }
        for (int l = 0; l < d; ++l) {
            Level& L = p->lv[l];
            const Level& C = p->lv[l + 1];
            L.full = (l < d - 1 || l == 0 || p->pre16) ? 1 : 0;
            const long long per = L.full ? 7 : 4;
            if (p->fuse_pre() && (l == d - 3 || l == d - 2)) continue;   // written by no pass: fused away
            if (p->fuse_root_pre() && l == 0) continue;   // fused away (both sides read the caller's operands)
            if (p->fuse_root_pre3() && l < d - 1) continue;   // fused away (both sides read the caller's operands)
            if (p->pre16 && l == d - 1) {   // the leaves' operands, as split planes
                p->ld16 = rup(C.k, 128 / (long long)p->es16());   // 128-byte row pitch
                for (int i = 0; i < 2; ++i) p->a16[i] = cv.take<char>((size_t)(L.nodes * 7 * C.m * p->ld16) * p->es16());
                for (int i = 0; i < 2; ++i) p->b16[i] = cv.take<char>((size_t)(L.nodes * 7 * C.n * p->ld16) * p->es16());
                continue;
            }
            L.achild = cv.take<float>((size_t)(L.nodes * per * C.m * C.k));
            L.bchild = cv.take<float>((size_t)(L.nodes * per * C.n * C.k));
        }
        const Level& Lf = p->lv[d];
        if (!p->fused) p->P = cv.take<float>((size_t)(Lf.nodes * Lf.m * Lf.n));
        for (int l = 1; l < d; ++l) {
            if (p->fused && l == d - 1) {   // written by the leaf launch itself
                Level& L = p->lv[l];
                L.cnode = cv.take<float>((size_t)(L.nodes * L.m * L.n));
                continue;
            }
            if (p->fused) continue;   // the remaining levels fold straight into C
            if (p->fuse_post() && (l == d - 1 || l == d - 2)) continue;   // fused away
            if (p->fuse_root_post() && l == d - 1) continue;
            if (p->fuse_root_post3()) continue;
            Level& L = p->lv[l];
            L.cnode = cv.take<float>((size_t)(L.nodes * L.m * L.n));
        }
        if (p->fused) p->fuse_scratch = cv.take<float>(kFuseMaxPairs * kFuseBytesPerPair / sizeof(float));
        if (p->peel && (p->Mw < p->M || p->Kw < p->K || p->Nw < p->N)) {
            // border products (classical leaves) read B transposed and A TMA-aligned
            p->ld_bt = rup(p->K, 4);
            p->Bt = cv.take<float>((size_t)p->N * p->ld_bt);
            p->ld_acopy = rup(p->K, 4);
            p->Acopy = cv.take<float>((size_t)p->M * p->ld_acopy);
        }
    }
    if (needed) *needed = align_up(cv.off, 256);
}

inline void mark(fmm_plan_s* p, int i, cudaStream_t s) {
    if (p->cur) cudaEventRecord(p->cur->e[i], s);
}

fmm_status_t drain_profile(fmm_plan_s* p) {
    for (auto& es : p->ev_pending) {
        FMM_CUDA(cudaEventSynchronize(es.e[3]));
        for (int i = 0; i < 3; ++i) {
            float ms = 0.f;
            FMM_CUDA(cudaEventElapsedTime(&ms, es.e[i], es.e[i + 1]));
            p->prof_ms[i] += ms;
        }
        p->ev_free.push_back(es);
    }
    p->ev_pending.clear();
    return FMM_OK;
}

fmm_status_t check_opts(const fmm_options_t* o) {
    if (o->depth < -1 || o->depth > 6) return FMM_ERR_INVALID_ARG;
    if (o->leaf_tile != 0 && o->leaf_tile != 128 && o->leaf_tile != 256 && o->leaf_tile != 512)
        return FMM_ERR_INVALID_ARG;
    if (o->precision < FMM_PREC_FP32 || o->precision > FMM_PREC_FP16X3) return FMM_ERR_INVALID_ARG;
    if (o->odd < FMM_ODD_PAD || o->odd > FMM_ODD_AUTO) return FMM_ERR_INVALID_ARG;
    if (o->planner < FMM_PLANNER_FIXED || o->planner > FMM_PLANNER_MLP) return FMM_ERR_INVALID_ARG;
    if (o->algo != FMM_ALGO_WINOGRAD && o->algo != FMM_ALGO_CLASSICAL) return FMM_ERR_INVALID_ARG;
    if (o->algo == FMM_ALGO_CLASSICAL && o->host_operands) return FMM_ERR_UNSUPPORTED;
    if (o->host_operands && o->odd != FMM_ODD_PAD && o->odd != FMM_ODD_AUTO) return FMM_ERR_UNSUPPORTED;
    if (o->fuse_last < -1 || o->fuse_last > 1) return FMM_ERR_INVALID_ARG;
    if (o->host_copy < 0 || o->host_copy > 2) return FMM_ERR_INVALID_ARG;
    return FMM_OK;
}

int leaf_mode(fmm_precision_t p) {
    switch (p) {
        case FMM_PREC_TF32: return kLeafTF32;
        case FMM_PREC_BF16X3: return kLeafBF16x3;
        case FMM_PREC_FP16X3: return kLeafFP16x3;
        default: return kLeaf3xTF32;
    }
}

// Whether plans that can fuse the last Winograd level into the leaf launch do
// so when the caller leaves fmm_options_t.fuse_last at 0.
constexpr bool kFuseLastDefault = true;

// Host-resident plans whose caller leaves fmm_options_t.host_copy at 0 use the
// copy engines (the faster path on a healthy link: duplex, and no SMs taken from
// the compute) until the input transfers of one call arrive at under half of
// the link's rate, then SM copies for the rest of the plan's life.  On these
// GPUs' virtual machines the copy engines can stall for 40-175 ms every few
// hundred ms after other processes pinned and freed host memory, while SM
// loads and stores over the same link do not.  Calls moving less than
// kHostJudgeBytes, and a plan's first call, are not judged.
constexpr double kHostStallGBs = 100.0;
constexpr double kHostJudgeBytes = 64.0 * (1 << 20);

// Fixed-threshold planner: one more level while every dimension of the next
// level's leaves stays at or above the cut-off (the recursion point of Sec. 3.1).
int fixed_depth(long long M, long long N, long long K, int cutoff) {
    if (cutoff <= 0) cutoff = 1024;
    int d = 0;
    long long mn = M < N ? M : N;
    if (K < mn) mn = K;
    while (d < 4 && (mn >> (d + 1)) >= cutoff) ++d;
    return d;
}

// Leaf tile when the caller leaves it open: the CTA-pair 256 x 256 tile once
// both output sides of every leaf reach 1024 (from there on it is at least as
// fast as the single-CTA tile and cuts the per-SM operand traffic by a third),
// the single-CTA 128 x 256 tile otherwise.
int auto_tile(long long M, long long N, int depth, const fmm_options_t& o) {
    (void)o;
    const long long mn = M < N ? M : N;
    return (mn >> depth) >= 1024 ? 512 : 256;
}

// Whether a leaf launch takes its tiles in dynamic order: launches over several
// leaves of K >= 1024, where the CTAs drift apart over many long waves (n =
// 16384, depth 3: 4-7 % faster, DRAM reads 44 -> 28 GB).  A single product
// keeps the static round robin (1 % faster there: the CTAs stay in step), and
// so do short tiles, whose work the slot read at each tile start would dent
// (the batched set: 2.5 % slower in dynamic order).
bool dynamic_order(const fmm_plan_s* p, const GemmArgs& args) {
    if (!p->tile_sched || args.num_groups < 1) return false;
    long long leaves = 0;
    for (int g = 0; g < args.num_groups; ++g) {
        if (args.groups[g].K < 1024) return false;
        leaves += args.groups[g].batch;
    }
    return leaves > 1;
}

// Leaf launch over `groups` (already filled except tile bookkeeping).
fmm_status_t run_leaves(fmm_plan_s* p, GemmArgs& args, cudaStream_t stream, int mode = -1) {
    const bool pair = p->pair && mode < 0;   // the peel border (explicit mode) stays single-CTA
    if (mode < 0) mode = p->mode;
    if (pair) {
        long long t = 0;
        for (int g = 0; g < args.num_groups; ++g) {
            GemmGroup& G = args.groups[g];
            G.tiles_m = (G.M + 255) / 256;
            G.tiles_n = (G.N + 255) / 256;
            G.tile_begin = t;
            t += (long long)G.tiles_m * G.tiles_n * G.batch;
            if (mode == kLeafFP16x3P) G.scale = p->fp16_scale();
        }
        args.total_tiles = t;
        args.raster_m = 16;
        args.ext_maps = nullptr;
        args.ext_groups = nullptr;
        args.status = p->status;
        if (dynamic_order(p, args)) {   // dynamic tile order: counter and rings start from zero
            FMM_CUDA(cudaMemsetAsync(p->tile_sched, 0, kTileSchedBytes, stream));
            args.tile_counter = reinterpret_cast<int*>(p->tile_sched);
            args.tile_seq = reinterpret_cast<unsigned long long*>(p->tile_sched + 256);
        }
        args.fuse_scratch = p->fused ? p->fuse_scratch : nullptr;
        FMM_CUDA(launch_leaf_gemm_pair(args, mode, p->num_sms, stream));
        p->launches += args.total_tiles > 0 ? 1 : 0;
        return FMM_OK;
    }
    long long t = 0;
    for (int g = 0; g < args.num_groups; ++g) {
        GemmGroup& G = args.groups[g];
        G.tiles_m = (G.M + kBM - 1) / kBM;
        G.tiles_n = (G.N + p->bn - 1) / p->bn;
        G.tile_begin = t;
        t += (long long)G.tiles_m * G.tiles_n * G.batch;
    }
    args.total_tiles = t;
    args.raster_m = 16;
    args.ext_maps = nullptr;
    args.ext_groups = nullptr;
    if (dynamic_order(p, args)) {   // dynamic tile order: counter and rings start from zero
        FMM_CUDA(cudaMemsetAsync(p->tile_sched, 0, kTileSchedBytes, stream));
        args.tile_counter = reinterpret_cast<int*>(p->tile_sched);
        args.tile_seq = reinterpret_cast<unsigned long long*>(p->tile_sched + 256);
    }
    if (mode == kLeafFP16x3 || mode == kLeafFP16x3P)
        for (int g = 0; g < args.num_groups; ++g) args.groups[g].scale = p->fp16_scale();
    args.status = p->status;
    FMM_CUDA(launch_leaf_gemm(args, mode, p->bn, p->num_sms, stream));
    p->launches += args.total_tiles > 0 ? 1 : 0;
    return FMM_OK;
}

// K chunks of the classical recursion of Table 1 (RMUL) at depth d: every level
// halves each chunk with Eq. 1's split (the first half takes the ceiling),
// rounded up to a multiple of 8 elements so that each chunk's tile copies start
// on 16 bytes.  The chunks are the k-blocks of C_ij = sum_k A_ik B_kj in the
// recursion's order; depth 0 is one chunk.
std::vector<std::pair<long long, long long>> rmul_chunks(long long K, int d) {
    std::vector<std::pair<long long, long long>> c{{0, K}};
    for (int l = 0; l < d; ++l) {
        std::vector<std::pair<long long, long long>> n;
        for (auto& [k0, len] : c) {
            const long long h = std::min(len, rup((len + 1) / 2, 8));
            n.push_back({k0, h});
            n.push_back({k0 + h, len - h});
        }
        c.swap(n);
    }
    return c;
}

// Classical product: the operands are prepared once (split into hi / lo planes,
// or B transposed for TF32), then one leaf launch per K chunk of the plan's
// classical recursion: the first writes C = alpha A_0 B_0 + beta C, every later
// one accumulates C += alpha A_s B_s (Table 1's C = AB, then C += AB leaves).
// Depth 0 is the single-launch tensor-core GEMM.
fmm_status_t run_classical(fmm_plan_s* p, float alpha, const float* A, const float* B, float beta, float* C,
                           cudaStream_t stream) {
    const int bf = p->split_kind;
    const long long ld = p->ld16;
    const float* Aop = A;
    long long lda = p->lda;
    // FP32 (3xTF32): the hi plane is the raw value, so an aligned A is read in
    // place and only its lo plane is written
    const bool a_raw = p->pre16 && bf == kSplitTF32 && (reinterpret_cast<uintptr_t>(A) & 15) == 0 && p->lda % 4 == 0;
    if (p->pre16) {
        const float* scale = p->mode == kLeafFP16x3P ? p->fp16_scale() : nullptr;
        Stack16 sa{a_raw ? nullptr : p->a16[0], p->a16[1], ld, 0, 1};
        Stack16 sb{p->b16[0], p->b16[1], ld, 0, 1};
        FMM_CUDA(launch_split16(A, p->lda, p->M, p->K, sa, 0, bf, scale, 0, stream));
        FMM_CUDA(launch_split16(B, p->ldb, p->K, p->N, sb, 1, bf, scale, 1, stream));
        p->launches += 2;
        p->acct[0] += (double)(p->M * p->K + p->K * p->N) * (4.0 + 2.0 * p->es16()) - (a_raw ? 4.0 * (double)(p->M * p->K) : 0.0);
    } else {
        FMM_CUDA(launch_transpose(B, p->ldb, p->K, p->N, p->Bt, p->ld_bt, stream));
        p->launches += 1;
        p->acct[0] += 8.0 * (double)(p->K * p->N);
        if ((reinterpret_cast<uintptr_t>(A) & 15) || (p->lda % 4)) {
            FMM_CUDA(launch_copy2d(A, p->lda, p->M, p->K, p->Acopy, p->ld_acopy, stream));
            p->launches += 1;
            p->acct[0] += 8.0 * (double)(p->M * p->K);
            Aop = p->Acopy;
            lda = p->ld_acopy;
        }
    }
    mark(p, 1, stream);
    bool first = true;
    for (const auto& [k0, kc] : rmul_chunks(p->K, p->rmul)) {
        if (kc <= 0) continue;
        GemmArgs args;
        memset(&args, 0, sizeof(args));
        fmm_status_t s;
        GemmGroup& G = args.groups[0];
        if (p->pre16) {
            const size_t off = (size_t)k0 * p->es16();   // bytes; k0 is a multiple of 8
            for (int i = 0; i < 2; ++i) {
                if (i == 0 && a_raw) {
                    if ((s = encode_map16(&args.maps[0], A + k0, bf, kc, p->M, 1, p->lda, p->M * p->lda, kBM,
                                          p->pair)) != FMM_OK)
                        return s;
                } else if ((s = encode_map16(&args.maps[i], static_cast<char*>(p->a16[i]) + off, bf, kc, p->M, 1, ld,
                                             p->M * ld, kBM, p->pair)) != FMM_OK) {
                    return s;
                }
                if ((s = encode_map16(&args.maps[2 + i], static_cast<char*>(p->b16[i]) + off, bf, kc, p->N, 1, ld,
                                      p->N * ld, p->pair ? 128 : p->bn, p->pair)) != FMM_OK)
                    return s;
            }
            G.map_a = 0; G.map_a_lo = 1; G.map_b = 2; G.map_b_lo = 3;
        } else {
            if ((s = encode_map(&args.maps[0], Aop + k0, kc, p->M, 1, lda, p->M * lda, kBM)) != FMM_OK) return s;
            if ((s = encode_map(&args.maps[1], p->Bt + k0, kc, p->N, 1, p->ld_bt, p->N * p->ld_bt,
                                p->pair ? 128 : p->bn)) != FMM_OK)
                return s;
            G.map_a = 0; G.map_b = 1;
        }
        G.M = (int)p->M; G.N = (int)p->N; G.K = (int)kc; G.batch = 1;
        G.C = C; G.ldc = p->ldc; G.c_batch_stride = 0;
        G.alpha = alpha; G.beta = first ? beta : 1.0f;
        G.vec_ok = ((reinterpret_cast<uintptr_t>(C) & 15) == 0 && p->ldc % 4 == 0) ? 1 : 0;
        args.num_groups = 1;
        if ((s = run_leaves(p, args, stream)) != FMM_OK) return s;
        if (!first) p->acct[1] += 8.0 * (double)(p->M * p->N);   // the accumulating launch reads and writes C
        first = false;
    }
    mark(p, 2, stream);
    return FMM_OK;
}

// Peeled border of a Winograd call on the even core (Mw x Kw x Nw), as classical
// tensor-core leaves in one launch (dynamic peeling, generalised from one row /
// column to the remainder modulo the level granule):
//   K > Kw:  C[:Mw, :Nw] += alpha * A[:Mw, Kw:] B[Kw:, :Nw]   (after the core)
//   M > Mw:  C[Mw:, :]    = alpha * A[Mw:, :] B + beta * C[Mw:, :]
//   N > Nw:  C[:Mw, Nw:]  = alpha * A[:Mw, :] B[:, Nw:] + beta * C[:Mw, Nw:]
fmm_status_t run_border(fmm_plan_s* p, float alpha, const float* A, const float* B, float* C, cudaStream_t stream) {
    FMM_CUDA(launch_transpose(B, p->ldb, p->K, p->N, p->Bt, p->ld_bt, stream));
    p->launches += 1;
    p->acct[1] += 8.0 * (double)(p->K * p->N);
    const float* Aop = A;
    long long lda = p->lda;
    if ((reinterpret_cast<uintptr_t>(A) & 15) || (p->lda % 4)) {
        FMM_CUDA(launch_copy2d(A, p->lda, p->M, p->K, p->Acopy, p->ld_acopy, stream));
        p->launches += 1;
        p->acct[1] += 8.0 * (double)(p->M * p->K);
        Aop = p->Acopy;
        lda = p->ld_acopy;
    }
    const long long ldt = p->ld_bt;
    const bool cvec = (reinterpret_cast<uintptr_t>(C) & 15) == 0 && p->ldc % 4 == 0;
    GemmArgs args;
    memset(&args, 0, sizeof(args));
    int ng = 0, nm = 0;
    fmm_status_t s;
    auto add = [&](const float* a, long long a_cols, long long a_rows, const float* b, long long b_rows, float* c,
                   long long M, long long N, long long K, float al, float be) -> fmm_status_t {
        if (M <= 0 || N <= 0 || K <= 0) return FMM_OK;
        fmm_status_t st;
        if ((st = encode_map(&args.maps[nm], a, a_cols, a_rows, 1, lda, a_rows * lda, kBM)) != FMM_OK) return st;
        if ((st = encode_map(&args.maps[nm + 1], b, a_cols, b_rows, 1, ldt, b_rows * ldt, p->bn)) != FMM_OK) return st;
        GemmGroup& G = args.groups[ng++];
        G.M = (int)M; G.N = (int)N; G.K = (int)K; G.batch = 1;
        G.C = c; G.ldc = p->ldc; G.c_batch_stride = 0; G.alpha = al; G.beta = be;
        G.map_a = nm; G.map_b = nm + 1; G.vec_ok = cvec ? 1 : 0;
        nm += 2;
        return FMM_OK;
    };
    const long long Mw = p->Mw, Kw = p->Kw, Nw = p->Nw, M = p->M, N = p->N, K = p->K;
    if ((s = add(Aop + Kw, K - Kw, Mw, p->Bt + Kw, Nw, C, Mw, Nw, K - Kw, alpha, 1.0f)) != FMM_OK) return s;
    if ((s = add(Aop + Mw * lda, K, M - Mw, p->Bt, N, C + Mw * p->ldc, M - Mw, N, K, alpha, p->border_beta)) != FMM_OK)
        return s;
    if ((s = add(Aop, K, Mw, p->Bt + Nw * ldt, N - Nw, C + Nw, Mw, N - Nw, K, alpha, p->border_beta)) != FMM_OK)
        return s;
    args.num_groups = ng;
    if (ng == 0) return FMM_OK;
    // the border reads fp32 operands: split-precision plans split them in shared memory
    const int mode = p->mode == kLeafBF16x3P   ? kLeafBF16x3
                     : p->mode == kLeafFP16x3P ? kLeafFP16x3
                     : p->mode == kLeaf3xTF32P ? kLeaf3xTF32
                                               : p->mode;
    return run_leaves(p, args, stream, mode);
}

// Pre-additions of every level (breadth-first), reading the caller's A and B at the root.
fmm_status_t winograd_pre(fmm_plan_s* p, const float* A, const float* B, cudaStream_t stream) {
    const int d = p->depth;
    Level* lv = p->lv;
    const int kind = p->split_kind;
    const float* scale = p->mode == kLeafFP16x3P ? p->fp16_scale() : nullptr;
    const double pl = 2.0 * (double)p->es16();   // bytes per element of a hi + lo plane pair
    const double root_in = 4.0 * (double)(p->Mw * p->Kw + p->Kw * p->Nw);
    if (p->fuse_root_pre3()) {
        // all three levels at once: root -> the 343 leaf operands of each side
        const Level& Lf = lv[3];
        View va{A, p->lda, 0, p->M0, p->K0, p->Mw, p->Kw};
        Stack16 sa{p->a16[0], p->a16[1], p->ld16, Lf.m * p->ld16, 343};
        Stack16 sb{p->b16[0], p->b16[1], p->ld16, Lf.n * p->ld16, 343};
        FMM_CUDA(launch_pre_add3(va, 1, sa, 0, kind, scale, stream));
        // B: the caller's row-major B straight into the K-major leaf planes,
        // transposed through shared memory
        FMM_CUDA(launch_pre_add3_bt(B, p->ldb, p->Kw, p->Nw, Lf.n, Lf.k, sb, kind, scale, stream));
        p->launches += 2;
        p->acct[0] += root_in + 343.0 * (double)(Lf.m * Lf.k + Lf.n * Lf.k) * pl;
        return FMM_OK;
    }
    if (p->fuse_root_pre()) {
        // both levels at once: root -> the 49 leaf operands; the B side reads the
        // caller's row-major B and writes the K-major (transposed) leaf planes
        const Level& Lf = lv[2];
        View va{A, p->lda, 0, p->M0, p->K0, p->Mw, p->Kw};
        Stack16 sa{p->a16[0], p->a16[1], p->ld16, Lf.m * p->ld16, 49};
        Stack16 sb{p->b16[0], p->b16[1], p->ld16, Lf.n * p->ld16, 49};
        FMM_CUDA(launch_pre_add2(va, 1, sa, 0, kind, scale, stream));
        FMM_CUDA(launch_pre_add2_b_root(B, p->ldb, p->Kw, p->Nw, Lf.n, Lf.k, sb, kind, scale, stream));
        p->launches += 2;
        p->acct[0] += root_in + 49.0 * (double)(Lf.m * Lf.k + Lf.n * Lf.k) * pl;
        return FMM_OK;
    }
    {
        const Level& C1 = lv[1];
        View va{A, p->lda, 0, lv[0].m, lv[0].k, p->Mw, p->Kw};
        if (p->pre16 && d == 1) {
            Stack16 sa{p->a16[0], p->a16[1], p->ld16, C1.m * p->ld16, 7};
            Stack16 sb{p->b16[0], p->b16[1], p->ld16, C1.n * p->ld16, 7};
            FMM_CUDA(launch_pre_add16(va, 1, sa, 0, kind, scale, stream));
            FMM_CUDA(launch_pre_add16_b_root(B, p->ldb, p->Kw, p->Nw, C1.k, C1.n, sb, kind, scale, stream));
            p->acct[0] += root_in + 7.0 * (double)(C1.m * C1.k + C1.n * C1.k) * pl;
        } else {
            Stack sa{lv[0].achild, C1.k, C1.m * C1.k, 7};
            FMM_CUDA(launch_pre_add(va, 1, sa, 0, 1, stream));
            Stack sb{lv[0].bchild, C1.k, C1.n * C1.k, 7};
            FMM_CUDA(launch_pre_add_b_root(B, p->ldb, p->Kw, p->Nw, C1.k, C1.n, sb, 1, stream));
            p->acct[0] += root_in + 7.0 * (double)(C1.m * C1.k + C1.n * C1.k) * 4.0;
        }
        p->launches += 2;
    }
    for (int l = 1; l < d; ++l) {
        const Level& L = lv[l];
        const Level& Ch = lv[l + 1];
        const Level& Pa = lv[l - 1];
        View va{Pa.achild, L.k, L.m * L.k, L.m, L.k, L.m, L.k};
        View vb{Pa.bchild, L.k, L.n * L.k, L.n, L.k, L.n, L.k};
        const double in = 4.0 * (double)L.nodes * (double)(L.m * L.k + L.n * L.k);
        if (p->fuse_pre() && l == d - 3) {
            // levels d-3 .. d-1 at once: level-(d-3) node operands -> the leaf operands
            const Level& Lf = lv[d];
            Stack16 sa{p->a16[0], p->a16[1], p->ld16, Lf.m * p->ld16, 343};
            Stack16 sb{p->b16[0], p->b16[1], p->ld16, Lf.n * p->ld16, 343};
            FMM_CUDA(launch_pre_add3(va, L.nodes, sa, 0, kind, scale, stream));
            FMM_CUDA(launch_pre_add3(vb, L.nodes, sb, 1, kind, scale, stream));
            p->launches += 2;
            p->acct[0] += in + 343.0 * (double)L.nodes * (double)(Lf.m * Lf.k + Lf.n * Lf.k) * pl;
            break;
        }
        if (p->pre16 && l == d - 1) {
            Stack16 sa{p->a16[0], p->a16[1], p->ld16, Ch.m * p->ld16, 7};
            Stack16 sb{p->b16[0], p->b16[1], p->ld16, Ch.n * p->ld16, 7};
            FMM_CUDA(launch_pre_add16(va, L.nodes, sa, 0, kind, scale, stream));
            FMM_CUDA(launch_pre_add16(vb, L.nodes, sb, 1, kind, scale, stream));
            p->launches += 2;
            p->acct[0] += in + 7.0 * (double)L.nodes * (double)(Ch.m * Ch.k + Ch.n * Ch.k) * pl;
            continue;
        }
        const int per = L.full ? 7 : 4;
        Stack sa{L.achild, Ch.k, Ch.m * Ch.k, per};
        Stack sb{L.bchild, Ch.k, Ch.n * Ch.k, per};
        FMM_CUDA(launch_pre_add(va, L.nodes, sa, 0, L.full, stream));
        FMM_CUDA(launch_pre_add(vb, L.nodes, sb, 1, L.full, stream));
        p->launches += 2;
        p->acct[0] += in + (double)per * (double)L.nodes * (double)(Ch.m * Ch.k + Ch.n * Ch.k) * 4.0;
    }
    return FMM_OK;
}

// Append the leaf groups of the plan's last level (and their tensor maps) to
// the given arrays; map indices are absolute in `maps`.
fmm_status_t winograd_leaf_groups(fmm_plan_s* p, CUtensorMap* maps, int& nm, GemmGroup* groups, int& ng) {
    const int d = p->depth;
    Level* lv = p->lv;
    const Level& Lf = lv[d];      // leaf sizes
    const Level& Ll = lv[d - 1];  // last recursion level
    fmm_status_t s;
    const long long mm = Lf.m, kk = Lf.k, nn = Lf.n;
    if (p->pre16) {
        const long long batch = Lf.nodes, ld = p->ld16;
        const int bf = p->split_kind;
        for (int i = 0; i < 2; ++i) {
            if ((s = encode_map16(&maps[nm + i], p->a16[i], bf, kk, mm, batch, ld, mm * ld, kBM, p->pair)) != FMM_OK)
                return s;
            if ((s = encode_map16(&maps[nm + 2 + i], p->b16[i], bf, kk, nn, batch, ld, nn * ld, p->pair ? 128 : p->bn,
                                  p->pair)) !=
                FMM_OK)
                return s;
        }
        GemmGroup& G = groups[ng++];
        memset(&G, 0, sizeof(G));
        G.M = (int)mm; G.N = (int)nn; G.K = (int)kk; G.batch = (int)batch;
        G.C = p->P; G.ldc = nn; G.c_batch_stride = mm * nn;
        if (p->fused) {
            // schedule units are (last-level node, tile); the launch writes the
            // node outputs (2 mm x 2 nn each, quadrants of the U-chain)
            G.batch = (int)Ll.nodes;
            G.C = Ll.cnode; G.ldc = Ll.n; G.c_batch_stride = Ll.m * Ll.n;
        }
        G.alpha = 1.f; G.beta = 0.f; G.map_a = nm; G.map_a_lo = nm + 1; G.map_b = nm + 2; G.map_b_lo = nm + 3;
        G.vec_ok = 1;
        nm += 4;
        return FMM_OK;
    }
    if (Ll.full) {
        const long long batch = Lf.nodes;
        if ((s = encode_map(&maps[nm], Ll.achild, kk, mm, batch, kk, mm * kk, kBM)) != FMM_OK) return s;
        if ((s = encode_map(&maps[nm + 1], Ll.bchild, kk, nn, batch, kk, nn * kk, p->pair ? 128 : p->bn)) != FMM_OK)
            return s;
        GemmGroup& G = groups[ng++];
        memset(&G, 0, sizeof(G));
        G.M = (int)mm; G.N = (int)nn; G.K = (int)kk; G.batch = (int)batch;
        G.C = p->P; G.ldc = nn; G.c_batch_stride = mm * nn;
        G.alpha = 1.f; G.beta = 0.f; G.map_a = nm; G.map_b = nm + 1; G.vec_ok = 1;
        nm += 2;
        return FMM_OK;
    }
    // parent operands of the last level: stacks of Ll.nodes matrices (Ll.m x Ll.k, Ll.n x Ll.k)
    const Level& Pa = lv[d - 2];
    const float* pa = Pa.achild;
    const float* pb = Pa.bchild;
    const long long nodes = Ll.nodes;
    const long long ka = Ll.k;  // parent row length
    auto qa = [&](int qi, int qj) { return pa + qi * mm * ka + qj * kk; };
    auto qb = [&](int qi, int qj) { return pb + qi * nn * ka + qj * kk; };
    const int b0 = nm;
    // A side: b0+0..2 quadrant views Q0, Q1, Q3; b0+3..6 sums S1..S4
    if ((s = encode_map(&maps[b0 + 0], qa(0, 0), kk, mm, nodes, ka, Ll.m * ka, kBM)) != FMM_OK) return s;
    if ((s = encode_map(&maps[b0 + 1], qa(0, 1), kk, mm, nodes, ka, Ll.m * ka, kBM)) != FMM_OK) return s;
    if ((s = encode_map(&maps[b0 + 2], qa(1, 1), kk, mm, nodes, ka, Ll.m * ka, kBM)) != FMM_OK) return s;
    for (int j = 0; j < 4; ++j)
        if ((s = encode_map(&maps[b0 + 3 + j], Ll.achild + j * mm * kk, kk, mm, nodes, kk, 4 * mm * kk, kBM)) != FMM_OK)
            return s;
    // B side (transposed): b0+7..9 views Y0, Y1, Y3; b0+10..13 sums T1..T4
    const int bbox = p->pair ? 128 : p->bn;
    if ((s = encode_map(&maps[b0 + 7], qb(0, 0), kk, nn, nodes, ka, Ll.n * ka, bbox)) != FMM_OK) return s;
    if ((s = encode_map(&maps[b0 + 8], qb(0, 1), kk, nn, nodes, ka, Ll.n * ka, bbox)) != FMM_OK) return s;
    if ((s = encode_map(&maps[b0 + 9], qb(1, 1), kk, nn, nodes, ka, Ll.n * ka, bbox)) != FMM_OK) return s;
    for (int j = 0; j < 4; ++j)
        if ((s = encode_map(&maps[b0 + 10 + j], Ll.bchild + j * nn * kk, kk, nn, nodes, kk, 4 * nn * kk, bbox)) !=
            FMM_OK)
            return s;
    //                       P1  P2  P3  P4  P5  P6  P7
    const int amap[7] = {0, 1, 6, 2, 3, 4, 5};       // Q0, Q1, S4, Q3, S1, S2, S3
    const int bmap[7] = {7, 8, 9, 13, 10, 11, 12};   // Y0, Y1, Y3, T4, T1, T2, T3
    for (int i = 0; i < 7; ++i) {
        GemmGroup& G = groups[ng++];
        memset(&G, 0, sizeof(G));
        G.M = (int)mm; G.N = (int)nn; G.K = (int)kk; G.batch = (int)nodes;
        G.C = p->P + i * mm * nn; G.ldc = nn; G.c_batch_stride = 7 * mm * nn;
        G.alpha = 1.f; G.beta = 0.f; G.map_a = b0 + amap[i]; G.map_b = b0 + bmap[i]; G.vec_ok = 1;
    }
    nm += 14;
    return FMM_OK;
}

// Post-additions bottom-up; the root applies alpha/beta into the caller's C.
fmm_status_t winograd_post(fmm_plan_s* p, float alpha, float beta, float* C, cudaStream_t stream) {
    const int d = p->depth;
    Level* lv = p->lv;
    int top = d - 1;
    const double root_out = 4.0 * (double)(p->Mw * p->Nw) * (beta != 0.0f ? 2.0 : 1.0);
    if (p->fused) {
        // the leaf launch left the level-(d-1) node outputs: the remaining levels
        // straight into the caller's C
        const Level& L = lv[d - 1];
        if (d == 4)
            FMM_CUDA(launch_post_add3(L.cnode, L.n, L.m * L.n, 1, L.m, L.n, C, p->ldc, 0, p->Mw, p->Nw, alpha, beta,
                                      stream));
        else if (d == 3)
            FMM_CUDA(launch_post_add2(L.cnode, L.n, L.m * L.n, 1, L.m, L.n, C, p->ldc, 0, p->Mw, p->Nw, alpha, beta,
                                      stream));
        else
            FMM_CUDA(launch_post_add(L.cnode, L.n, L.m * L.n, 1, L.m, L.n, C, p->ldc, 0, p->Mw, p->Nw, alpha, beta,
                                     stream));
        p->launches += 1;
        p->acct[1] += (double)L.nodes * 4.0 * (double)(L.m * L.n) + root_out;
        return FMM_OK;
    }
    if (p->fuse_root_post3()) {
        // all three levels at once: leaf products -> the caller's C
        const Level& Lf = lv[3];
        FMM_CUDA(launch_post_add3(p->P, Lf.n, Lf.m * Lf.n, 1, Lf.m, Lf.n, C, p->ldc, 0, p->Mw, p->Nw, alpha, beta,
                                  stream));
        p->launches += 1;
        p->acct[1] += 343.0 * 4.0 * (double)(Lf.m * Lf.n) + root_out;
        return FMM_OK;
    }
    if (p->fuse_root_post()) {
        // both levels at once: leaf products -> the caller's C (alpha, beta, valid window)
        const Level& Lf = lv[2];
        FMM_CUDA(launch_post_add2(p->P, Lf.n, Lf.m * Lf.n, 1, Lf.m, Lf.n, C, p->ldc, 0, p->Mw, p->Nw, alpha, beta,
                                  stream));
        p->launches += 1;
        p->acct[1] += 49.0 * 4.0 * (double)(Lf.m * Lf.n) + root_out;
        return FMM_OK;
    }
    if (p->fuse_post()) {
        // levels d-1 .. d-3 at once: leaf products -> level-(d-3) node outputs
        const Level& L = lv[d - 3];
        const Level& Lf = lv[d];
        FMM_CUDA(launch_post_add3(p->P, Lf.n, Lf.m * Lf.n, L.nodes, Lf.m, Lf.n, L.cnode, L.n, L.m * L.n, -1, -1, 1.f,
                                  0.f, stream));
        p->launches += 1;
        p->acct[1] += 4.0 * (double)L.nodes * (343.0 * (double)(Lf.m * Lf.n) + (double)(L.m * L.n));
        top = d - 4;
    }
    for (int l = top; l >= 0; --l) {
        const Level& L = lv[l];
        const Level& Ch = lv[l + 1];
        const float* in = (l == d - 1) ? p->P : lv[l + 1].cnode;
        if (l > 0) {
            FMM_CUDA(launch_post_add(in, Ch.n, Ch.m * Ch.n, L.nodes, Ch.m, Ch.n, L.cnode, L.n, L.m * L.n, -1, -1, 1.f,
                                     0.f, stream));
            p->acct[1] += 4.0 * (double)L.nodes * (7.0 * (double)(Ch.m * Ch.n) + (double)(L.m * L.n));
        } else {
            FMM_CUDA(launch_post_add(in, Ch.n, Ch.m * Ch.n, 1, Ch.m, Ch.n, C, p->ldc, 0, p->Mw, p->Nw, alpha, beta,
                                     stream));
            p->acct[1] += 4.0 * 7.0 * (double)(Ch.m * Ch.n) + root_out;
        }
        p->launches += 1;
    }
    return FMM_OK;
}

fmm_status_t run_winograd(fmm_plan_s* p, float alpha, const float* A, const float* B, float beta, float* C,
                          cudaStream_t stream) {
    p->border_beta = beta;
    fmm_status_t s;
    if ((s = winograd_pre(p, A, B, stream)) != FMM_OK) return s;
    mark(p, 1, stream);
    {
        GemmArgs args;
        memset(&args, 0, sizeof(args));
        int nm = 0, ng = 0;
        if ((s = winograd_leaf_groups(p, args.maps, nm, args.groups, ng)) != FMM_OK) return s;
        args.num_groups = ng;
        if ((s = run_leaves(p, args, stream)) != FMM_OK) return s;
    }
    mark(p, 2, stream);
    if ((s = winograd_post(p, alpha, beta, C, stream)) != FMM_OK) return s;
    if (p->peel && (p->Mw < p->M || p->Kw < p->K || p->Nw < p->N)) return run_border(p, alpha, A, B, C, stream);
    return FMM_OK;
}

// One multiply with the plan's schedule (FP16x3 first derives its operand scales).
fmm_status_t execute(fmm_plan_s* p, float alpha, const float* A, const float* B, float beta, float* C,
                     cudaStream_t stream) {
    p->acct[0] = p->acct[1] = 0.0;
    if (p->mode == kLeafFP16x3 || p->mode == kLeafFP16x3P) {
        // operand magnitudes of the leaves are bounded by 4^depth times the root's
        const float bound = (float)(1LL << (2 * p->depth));
        FMM_CUDA(launch_fp16_scales(A, p->lda, p->M, p->K, B, p->ldb, p->N, bound, p->fp16_scale(),
                                    p->fp16_scratch(), stream));
        p->launches += 3;
        p->acct[0] += 4.0 * (double)(p->M * p->K + p->K * p->N);
    }
    return (p->depth == 0) ? run_classical(p, alpha, A, B, beta, C, stream)
                           : run_winograd(p, alpha, A, B, beta, C, stream);
}

}  // namespace

// ----------------------------------------------------------------------------------------- batched
struct fmm_batched_s {
    int count = 0;
    int bn = 256, mode = kLeaf3xTF32, num_sms = 0;
    int pair = 0;                      // leaf tiles of 256 x 256 on CTA pairs (pre-split precisions)
    // FP16x3: per-problem operand maxima, bounds (4^depth) and scales {s_a, s_b}
    int fp16 = 0;
    AbsJob* d_ajobs = nullptr;
    int najobs = 0;
    long long ajob_tiles = 0;
    unsigned* d_absmax = nullptr;
    float* d_bound = nullptr;
    float* d_scales = nullptr;
    unsigned* status = nullptr;
    CUtensorMap* d_maps = nullptr;
    GemmGroup* d_groups = nullptr;
    int num_groups = 0;
    long long total_tiles = 0;
    CopyJob* d_jobs = nullptr;
    int njobs = 0;
    long long job_tiles = 0;
    // pre-split leaves: split jobs instead of copy jobs
    int pre = 0, split_kind = 0;
    SplitJob* d_sjobs = nullptr;
    std::vector<fmm_plan_s*> subs;     // Winograd sub-plans (problems with depth >= 1)
    std::vector<int> sub_problem;
    std::vector<int> depth;            // per problem
    std::vector<int> scale_only;       // problems with K == 0 or alpha == 0: C <- beta C
    std::vector<const float*> A, B;
    std::vector<float*> C;
    std::vector<long long> M, N, ldc;
    std::vector<float> alpha, beta;
    std::vector<int> cls;              // size class of each problem (-1: no product)
    int nclasses = 0;
    int tile = 512;                    // leaf tile of the launch (512: CTA pairs)
    long long launches = 0;
    ~fmm_batched_s() {
        for (auto* q : subs) delete q;
    }
};

namespace {

// Deepest level a batched problem may take: at most 4, leaves at least 64 wide.
int batched_max_depth(long long M, long long N, long long K) {
    const long long mn = std::min(std::min(M, N), K);
    int d = 4;
    while (d > 0 && (mn >> d) < 64) --d;
    return d;
}

// Depth of problem i under the fixed rule (or the caller's depth), kept to leaves
// at least 64 wide; -1 for problems with no product to compute.
int batched_fixed_depth(long long M, long long N, long long K, float alpha, const fmm_options_t& o) {
    if (M == 0 || N == 0 || K == 0 || alpha == 0.0f) return -1;
    int d = o.depth >= 0 ? o.depth : fixed_depth(M, N, K, o.cutoff);
    return std::min(d, batched_max_depth(M, N, K));
}

// depth_in: per-problem depths chosen by a planner (nullptr: the fixed rule);
// tile_req: the launch's leaf tile (0: from the options).
fmm_status_t batched_build(fmm_batched_s* b, int count, const int64_t* M, const int64_t* N, const int64_t* K,
                           const float* const* A, const int64_t* lda, const float* const* B, const int64_t* ldb,
                           float* const* C, const int64_t* ldc, const float* alpha, const float* beta,
                           const fmm_options_t& o, char* ws, size_t* needed, const int* depth_in = nullptr,
                           int tile_req = 0) {
    Carver cv(ws);
    b->status = cv.take<unsigned>(64);
    b->count = count;
    b->mode = leaf_mode(o.precision);
    b->fp16 = o.precision == FMM_PREC_FP16X3 ? 1 : 0;
    b->pre = o.precision == FMM_PREC_FP32 || o.precision == FMM_PREC_BF16X3 || b->fp16;
    // leaf tile 512 (and the default 0): 256 x 256 tiles on CTA pairs for the
    // pre-split precisions (512 uneven products: 8.70 ms per replay against 9.10
    // on single CTAs); TF32 batched launches stay on single CTAs (128 x 256)
    const int lt = tile_req ? tile_req : o.leaf_tile;
    b->pair = ((lt == 512 || lt == 0) && b->pre) ? 1 : 0;
    b->bn = (lt && lt != 512) ? lt : 256;
    b->tile = b->pair ? 512 : b->bn;
    if (b->pre) {
        b->split_kind = o.precision == FMM_PREC_BF16X3 ? kSplitBF16 : b->fp16 ? kSplitFP16 : kSplitTF32;
        b->mode = o.precision == FMM_PREC_BF16X3 ? kLeafBF16x3P : b->fp16 ? kLeafFP16x3P : kLeaf3xTF32P;
    }
    const size_t es = b->split_kind == kSplitTF32 ? 4 : 2;
    // per-problem depth and resource counts
    int total_maps = 0, total_groups = 0, total_jobs = 0;
    b->depth.assign(count, 0);
    b->scale_only.assign(count, 0);
    for (int i = 0; i < count; ++i) {
        if (M[i] == 0 || N[i] == 0) { b->depth[i] = -1; continue; }
        if (K[i] == 0 || alpha[i] == 0.0f) { b->depth[i] = -1; b->scale_only[i] = 1; continue; }
        int d = depth_in ? std::min(std::max(depth_in[i], 0), batched_max_depth(M[i], N[i], K[i]))
                         : batched_fixed_depth(M[i], N[i], K[i], alpha[i], o);
        b->depth[i] = d;
        if (b->pre) { total_maps += 4; total_groups += 1; total_jobs += d == 0 ? 2 : 0; }
        else if (d == 0) { total_maps += 2; total_groups += 1; total_jobs += 2; }
        else { total_maps += 14; total_groups += 7; }
    }
    b->d_maps = cv.take<CUtensorMap>(total_maps > 0 ? total_maps : 1);
    b->d_groups = cv.take<GemmGroup>(total_groups > 0 ? total_groups : 1);
    b->d_jobs = cv.take<CopyJob>(total_jobs > 0 ? total_jobs : 1);
    b->d_sjobs = cv.take<SplitJob>(total_jobs > 0 ? total_jobs : 1);
    std::vector<AbsJob> ajobs;
    std::vector<float> bound;
    if (b->fp16) {
        b->d_ajobs = cv.take<AbsJob>(2 * (size_t)(count > 0 ? count : 1));
        b->d_absmax = cv.take<unsigned>(2 * (size_t)(count > 0 ? count : 1));
        b->d_bound = cv.take<float>((size_t)(count > 0 ? count : 1));
        b->d_scales = cv.take<float>(2 * (size_t)(count > 0 ? count : 1));
        bound.assign(count > 0 ? count : 1, 1.0f);
    }
    // the problem's scales (FP16x3), or null
    auto scale_of = [&](int i) -> float* { return b->fp16 && b->d_scales ? b->d_scales + 2 * i : nullptr; };
    std::vector<SplitJob> sjobs;
    std::vector<CUtensorMap> maps(total_maps > 0 ? total_maps : 1);
    std::vector<GemmGroup> groups(total_groups > 0 ? total_groups : 1);
    std::vector<CopyJob> jobs;
    int nm = 0, ng = 0;
    for (int i = 0; i < count; ++i) {
        const int d = b->depth[i];
        if (d < 0) continue;
        if (b->fp16 && ws) {
            // operand magnitudes of the leaves are bounded by 4^depth times the problem's
            bound[i] = (float)(1LL << (2 * d));
            ajobs.push_back(AbsJob{A[i], lda[i], M[i], K[i], b->d_absmax + 2 * i, 0, (int)((K[i] + 127) / 128)});
            ajobs.push_back(AbsJob{B[i], ldb[i], K[i], N[i], b->d_absmax + 2 * i + 1, 0, (int)((N[i] + 127) / 128)});
        }
        if (d == 0 && b->pre) {
            const long long ld = rup(K[i], 128 / (long long)es);   // 128-byte row pitch
            void* ah = cv.take<char>((size_t)M[i] * ld * es);
            void* al = cv.take<char>((size_t)M[i] * ld * es);
            void* bh = cv.take<char>((size_t)N[i] * ld * es);
            void* bl = cv.take<char>((size_t)N[i] * ld * es);
            if (!ws) continue;
            // FP32 (3xTF32) planes hold the raw value as hi: an aligned A is read in place
            // and only its lo plane is written
            const bool a_raw = b->split_kind == kSplitTF32 && (reinterpret_cast<uintptr_t>(A[i]) & 15) == 0 &&
                               lda[i] % 4 == 0;
            sjobs.push_back(SplitJob{A[i], lda[i], M[i], K[i], a_raw ? nullptr : ah, al, ld, 0,
                                     (int)((K[i] + 127) / 128), 0, scale_of(i)});
            sjobs.push_back(SplitJob{B[i], ldb[i], K[i], N[i], bh, bl, ld, 0, (int)((N[i] + 127) / 128), 1, scale_of(i)});
            fmm_status_t s;
            const int kd = b->split_kind;
            const bool wide = b->pair != 0;              // pair: 128-byte rows, 128 rows of B per CTA
            const int bbox = wide ? 128 : b->bn;
            if (a_raw) {
                if ((s = encode_map16(&maps[nm], A[i], kd, K[i], M[i], 1, lda[i], M[i] * lda[i], kBM, wide)) != FMM_OK)
                    return s;
            } else if ((s = encode_map16(&maps[nm], ah, kd, K[i], M[i], 1, ld, M[i] * ld, kBM, wide)) != FMM_OK) {
                return s;
            }
            if ((s = encode_map16(&maps[nm + 1], al, kd, K[i], M[i], 1, ld, M[i] * ld, kBM, wide)) != FMM_OK) return s;
            if ((s = encode_map16(&maps[nm + 2], bh, kd, K[i], N[i], 1, ld, N[i] * ld, bbox, wide)) != FMM_OK) return s;
            if ((s = encode_map16(&maps[nm + 3], bl, kd, K[i], N[i], 1, ld, N[i] * ld, bbox, wide)) != FMM_OK) return s;
            GemmGroup& G = groups[ng++];
            memset(&G, 0, sizeof(G));
            G.M = (int)M[i]; G.N = (int)N[i]; G.K = (int)K[i]; G.batch = 1;
            G.C = C[i]; G.ldc = ldc[i]; G.alpha = alpha[i]; G.beta = beta[i];
            G.map_a = nm; G.map_a_lo = nm + 1; G.map_b = nm + 2; G.map_b_lo = nm + 3;
            G.vec_ok = ((reinterpret_cast<uintptr_t>(C[i]) & 15) == 0 && ldc[i] % 4 == 0) ? 1 : 0;
            G.scale = scale_of(i);
            nm += 4;
        } else if (d == 0) {
            const long long ldt = rup(K[i], 4);
            float* Bt = cv.take<float>((size_t)N[i] * ldt);
            const float* Aop = A ? A[i] : nullptr;   // A is null in a size query
            long long la = lda[i];
            float* Acopy = nullptr;
            if (!A || (reinterpret_cast<uintptr_t>(A[i]) & 15) || (lda[i] % 4)) {  // size query: assume a copy
                la = rup(K[i], 4);
                Acopy = cv.take<float>((size_t)M[i] * la);
                Aop = Acopy;
            }
            if (!ws) continue;
            jobs.push_back(CopyJob{B[i], ldb[i], K[i], N[i], Bt, ldt, 0, (int)((N[i] + 31) / 32), 1});
            if (Acopy) jobs.push_back(CopyJob{A[i], lda[i], M[i], K[i], Acopy, la, 0, (int)((K[i] + 31) / 32), 0});
            fmm_status_t s;
            if ((s = encode_map(&maps[nm], Aop, K[i], M[i], 1, la, M[i] * la, kBM)) != FMM_OK) return s;
            if ((s = encode_map(&maps[nm + 1], Bt, K[i], N[i], 1, ldt, N[i] * ldt, b->bn)) != FMM_OK) return s;
            GemmGroup& G = groups[ng++];
            memset(&G, 0, sizeof(G));
            G.M = (int)M[i]; G.N = (int)N[i]; G.K = (int)K[i]; G.batch = 1;
            G.C = C[i]; G.ldc = ldc[i]; G.alpha = alpha[i]; G.beta = beta[i];
            G.map_a = nm; G.map_b = nm + 1;
            G.vec_ok = ((reinterpret_cast<uintptr_t>(C[i]) & 15) == 0 && ldc[i] % 4 == 0) ? 1 : 0;
            nm += 2;
        } else {
            fmm_plan_s tmp;
            tmp.M = M[i]; tmp.N = N[i]; tmp.K = K[i]; tmp.lda = lda[i]; tmp.ldb = ldb[i]; tmp.ldc = ldc[i];
            tmp.opt = o;
            tmp.depth = d;
            tmp.bn = b->bn;
            tmp.pair = b->pair;
            tmp.mode = b->mode;
            tmp.peel = 0;
            tmp.pre16 = b->pre;
            tmp.split_kind = b->split_kind;
            tmp.sched = 0;   // its leaves run in the batched launch
            size_t need = 0;
            layout(&tmp, nullptr, &need);
            char* sub_ws = cv.take<char>(need);
            if (!ws) continue;
            fmm_plan_s* q = new (std::nothrow) fmm_plan_s(tmp);
            if (!q) return FMM_ERR_OOM;
            layout(q, sub_ws, nullptr);
            q->status = b->status;
            q->scale_override = scale_of(i);
            b->subs.push_back(q);
            b->sub_problem.push_back(i);
            fmm_status_t s;
            const int ng0 = ng;
            if ((s = winograd_leaf_groups(q, maps.data(), nm, groups.data(), ng)) != FMM_OK) return s;
            for (int g = ng0; g < ng; ++g) groups[g].scale = scale_of(i);
        }
    }
    if (needed) *needed = align_up(cv.off, 256);
    if (!ws) return FMM_OK;
    // longest tiles (largest K) first: round-robin tile assignment then balances like LPT
    std::stable_sort(groups.begin(), groups.begin() + ng,
                     [](const GemmGroup& x, const GemmGroup& y) { return x.K > y.K; });
    long long t = 0;
    for (int g = 0; g < ng; ++g) {
        GemmGroup& G = groups[g];
        const int tile_rows = b->pair ? 256 : kBM;
        G.tiles_m = (G.M + tile_rows - 1) / tile_rows;
        G.tiles_n = (G.N + b->bn - 1) / b->bn;
        G.tile_begin = t;
        t += (long long)G.tiles_m * G.tiles_n * G.batch;
    }
    b->num_groups = ng;
    b->total_tiles = t;
    long long jt = 0;
    for (auto& J : jobs) {
        J.tile_begin = jt;
        jt += ((J.rows + 31) / 32) * (long long)J.tiles_c;
    }
    for (auto& J : sjobs) {
        J.tile_begin = jt;
        jt += ((J.rows + 31) / 32) * (long long)J.tiles_c;
    }
    b->njobs = (int)(b->pre ? sjobs.size() : jobs.size());
    b->job_tiles = jt;
    if (b->fp16) {
        long long at = 0;
        for (auto& J : ajobs) {
            J.tile_begin = at;
            at += ((J.rows + 31) / 32) * (long long)J.tiles_c;
        }
        b->najobs = (int)ajobs.size();
        b->ajob_tiles = at;
        if (!ajobs.empty())
            FMM_CUDA(cudaMemcpy(b->d_ajobs, ajobs.data(), sizeof(AbsJob) * ajobs.size(), cudaMemcpyHostToDevice));
        FMM_CUDA(cudaMemcpy(b->d_bound, bound.data(), sizeof(float) * bound.size(), cudaMemcpyHostToDevice));
    }
    if (!sjobs.empty())
        FMM_CUDA(cudaMemcpy(b->d_sjobs, sjobs.data(), sizeof(SplitJob) * sjobs.size(), cudaMemcpyHostToDevice));
    FMM_CUDA(cudaMemcpy(b->d_maps, maps.data(), sizeof(CUtensorMap) * (nm > 0 ? nm : 1), cudaMemcpyHostToDevice));
    FMM_CUDA(cudaMemcpy(b->d_groups, groups.data(), sizeof(GemmGroup) * (ng > 0 ? ng : 1), cudaMemcpyHostToDevice));
    if (!jobs.empty())
        FMM_CUDA(cudaMemcpy(b->d_jobs, jobs.data(), sizeof(CopyJob) * jobs.size(), cudaMemcpyHostToDevice));
    FMM_CUDA(cudaMemset(b->status, 0, 64 * sizeof(unsigned)));
    for (int i = 0; i < count; ++i) {
        b->A.push_back(A[i]); b->B.push_back(B[i]); b->C.push_back(C[i]);
        b->M.push_back(M[i]); b->N.push_back(N[i]); b->ldc.push_back(ldc[i]);
        b->alpha.push_back(alpha[i]); b->beta.push_back(beta[i]);
    }
    return FMM_OK;
}

fmm_status_t batched_check(int count, const int64_t* M, const int64_t* N, const int64_t* K, const float* const* A,
                           const int64_t* lda, const float* const* B, const int64_t* ldb, float* const* C,
                           const int64_t* ldc, const float* alpha, const float* beta, const fmm_options_t* opt) {
    if (count < 0 || (count > 0 && (!M || !N || !K || !lda || !ldb || !ldc || !alpha || !beta))) return FMM_ERR_INVALID_ARG;
    for (int i = 0; i < count; ++i) {
        if (M[i] < 0 || N[i] < 0 || K[i] < 0 || M[i] > INT32_MAX || N[i] > INT32_MAX || K[i] > INT32_MAX)
            return FMM_ERR_INVALID_ARG;
        if (lda[i] < (K[i] > 0 ? K[i] : 1) || ldb[i] < (N[i] > 0 ? N[i] : 1) || ldc[i] < (N[i] > 0 ? N[i] : 1))
            return FMM_ERR_INVALID_ARG;
    }
    if (opt) {
        fmm_status_t s = check_opts(opt);
        if (s != FMM_OK) return s;
        if ((opt->odd != FMM_ODD_PAD && opt->odd != FMM_ODD_AUTO) || opt->algo == FMM_ALGO_CLASSICAL)
            return FMM_ERR_UNSUPPORTED;
    }
    (void)A; (void)B; (void)C;
    return FMM_OK;
}

}  // namespace

namespace {

// ----------------------------------------------------------------------------------------- planner
void make_tmp(fmm_plan_s& t, long long M, long long N, long long K, long long lda, long long ldb, long long ldc,
              const fmm_options_t& o, int depth, int bn) {
    t.M = M; t.N = N; t.K = K; t.lda = lda; t.ldb = ldb; t.ldc = ldc;
    t.opt = o;
    t.host = o.host_operands ? 1 : 0;
    t.depth = (M == 0 || N == 0 || K == 0) ? 0 : depth;
    t.rmul = 0;
    if (o.algo == FMM_ALGO_CLASSICAL) {   // classical recursion: depth-0 operands, K chunks
        t.rmul = t.depth;
        t.depth = 0;
    }
    // odd sizes: AUTO peels to whole leaf tiles when every peeled dimension's
    // remainder is at most an eighth of its granule (the last tile row or
    // column of every leaf would be mostly padding) and pads otherwise.  Same-GPU
    // sweeps over n = 4352 .. 19712 against padded plans (the last level unfused
    // on their ragged leaves): every eighth-granule case gained (+0.8 to +12.5 %
    // at depth 3), quarter-granule ones were mixed (-5.2 to +3.3 %).  Host-resident
    // plans always pad
    fmm_odd_t odd = o.odd;
    const long long tm = (bn == 512) ? 256 : kBM, tn = (bn == 512) ? 256 : bn;
    if (odd == FMM_ODD_AUTO) {
        odd = FMM_ODD_PAD;
        if (!t.host && t.depth > 0 && o.algo == FMM_ALGO_WINOGRAD) {
            const long long gm = tm << t.depth, gn = tn << t.depth;
            const long long rm = M % gm, rn = N % gn;
            if (M >= gm && N >= gn && (rm > 0 || rn > 0) && 8 * rm <= gm && 8 * rn <= gn) odd = FMM_ODD_TILE;
        }
    }
    t.odd = odd;
    t.peel = (odd == FMM_ODD_PEEL || odd == FMM_ODD_TILE) ? 1 : 0;
    t.peel_gm = t.peel_gn = 0;
    if (t.peel && t.depth > 0) {
        const long long g = 4LL << t.depth;
        if (M / g == 0 || N / g == 0 || K / g == 0) t.depth = 0;  // no even core: classical leaf
    }
    if (odd == FMM_ODD_TILE && t.depth > 0) {
        // leaves of whole tiles in M and N (pair tiles: 256 x 256; one CTA:
        // 128 rows x leaf-tile columns); a dimension with no whole-tile core
        // keeps the 4 * 2^d granule
        const long long gm = tm << t.depth, gn = tn << t.depth;
        t.peel_gm = M / gm > 0 ? gm : 0;
        t.peel_gn = N / gn > 0 ? gn : 0;
    }
    t.bn = bn;
    t.tile_req = bn;
    t.mode = leaf_mode(o.precision);
    t.pre16 = 0;
    t.pair = 0;
    if (t.bn == 512) t.bn = 256;   // the pair tile is 256 wide: set below when the plan can use it
    if (!t.host) t.pair = bn == 512 ? 1 : 0;
    if (!t.host && o.precision != FMM_PREC_TF32) {
        t.pre16 = 1;
        t.split_kind = o.precision == FMM_PREC_BF16X3   ? kSplitBF16
                       : o.precision == FMM_PREC_FP16X3 ? kSplitFP16
                                                        : kSplitTF32;
        t.mode = o.precision == FMM_PREC_BF16X3   ? kLeafBF16x3P
                 : o.precision == FMM_PREC_FP16X3 ? kLeafFP16x3P
                                                  : kLeaf3xTF32P;
    }
    // the fused last level needs the CTA-pair kernel on split planes and a
    // Winograd depth of 2 to 4 (the node outputs then fold into C in one pass)
    const bool fusable = t.pair && t.pre16 && !t.host && t.rmul == 0 && t.depth >= 2 && t.depth <= 4;
    // by default at depths 2 and 3 where every leaf is whole 256 x 256 pair tiles
    // in M and N (n = 16384, depth 3: 0.4-0.6 ms faster per call); with ragged
    // leaves a unit's seven products run as one, so its edge tiles and the
    // launch's last partial wave of units cost more than the post pass saves
    // (n = 19000, leaves 2376 wide: 0.3-1.9 ms slower at depth 3, 0.2-0.9 ms at
    // depth 2); at depth 4 on request (n = 32768: post-additions 8.8 -> 4.8 ms
    // but the call measured slower, 172-182 against 163-165 ms)
    bool whole = false;
    if (t.depth > 0) {
        const long long g = 4LL << t.depth;
        auto leaf_side = [&](long long X, long long gx) {
            const long long gg = gx ? gx : g;
            return (t.peel ? X / gg * gg : (X + g - 1) / g * g) >> t.depth;
        };
        whole = leaf_side(M, t.peel_gm) % 256 == 0 && leaf_side(N, t.peel_gn) % 256 == 0;
    }
    t.fused = fusable && (o.fuse_last > 0 || (o.fuse_last == 0 && kFuseLastDefault && t.depth <= 3 && whole))
                  ? 1
                  : 0;
}

size_t plan_bytes(long long M, long long N, long long K, long long lda, long long ldb, long long ldc,
                  const fmm_options_t& o, int depth, int bn) {
    fmm_plan_s t;
    make_tmp(t, M, N, K, lda, ldb, ldc, o, depth, bn);
    size_t need = 0;
    layout(&t, nullptr, &need);
    return need;
}

struct Cand { int depth, bn; };

int candidates(long long M, long long N, long long K, const fmm_options_t& o, Cand* out) {
    long long mn = std::min(std::min(M, N), K);
    int n = 0;
    for (int d = 0; d <= 4; ++d) {
        if (d > 0 && (mn >> d) < 128) break;
        if (o.depth >= 0 && d != o.depth) continue;
        for (int bn : {128, 256, 512}) {
            if (o.leaf_tile && bn != o.leaf_tile) continue;
            // CTA-pair tiles: leaves of at least one pair tile
            if (bn == 512 && (std::min(M, N) >> d) < 256) continue;
            out[n++] = Cand{d, bn};
        }
    }
    if (n == 0) out[n++] = Cand{o.depth >= 0 ? o.depth : 0, o.leaf_tile ? o.leaf_tile : 256};
    return n;
}

struct CostModel {
    bool set = false;
    float params[FMM_MLP_NPARAM];
    float mean[6], stdv[6];
    float* dev_params[64] = {};
    float* dev_io[64] = {};   // 16 x 6 features + 16 outputs
    int version = 0;
    int dev_version[64] = {};
};
CostModel g_model;

void raw_features(long long M, long long N, long long K, int depth, int bn, int prec, float* f) {
    f[0] = (float)std::log2((double)std::max(M, 1LL));
    f[1] = (float)std::log2((double)std::max(K, 1LL));
    f[2] = (float)std::log2((double)std::max(N, 1LL));
    f[3] = (float)depth;
    f[4] = (float)bn / 128.0f;
    f[5] = (float)prec;
}

// Child problem of a host-resident plan: one root quadrant product on device
// buffers (depth - 1 levels), or the whole product at depth 0.
void make_child(const fmm_plan_s* p, fmm_plan_s& c) {
    fmm_options_t o = p->opt;
    o.host_operands = 0;
    o.odd = FMM_ODD_PAD;   // the quadrant buffers are padded to the level granule already
    make_tmp(c, p->hm, p->hn, p->hk, p->hk, p->hn, p->hn, o, p->depth > 0 ? p->depth - 1 : 0, p->tile_req);
}

// Host-resident multiply.  The root level runs depth-first over the seven
// products so that transfers overlap compute: A11, B11 are copied first (P1
// starts on them), then A12, B21 (P2), then the rest; C11 = P1 + P2 is copied
// back while P3..P7 run.  Copies run on the plan's two copy streams, ordered
// after `stream` by events; `stream` waits for the last device-to-host copy.
fmm_status_t run_host(fmm_plan_s* p, float alpha, const float* A, const float* B, float beta, float* C,
                      cudaStream_t stream) {
    // device-side addresses of the three operands (the device mapping of pinned
    // host memory, or the pointer itself for device memory); null where a
    // block has none, and then the copy engines move it
    void* mapped[3] = {nullptr, nullptr, nullptr};
    {
        const void* ptrs[3] = {A, B, C};
        for (int i = 0; i < 3; ++i) {
            cudaPointerAttributes at;
            if (cudaPointerGetAttributes(&at, ptrs[i]) != cudaSuccess) {
                cudaGetLastError();
                return FMM_ERR_INVALID_ARG;
            }
            if (at.type == cudaMemoryTypeUnregistered) {
                snprintf(g_last_error, sizeof(g_last_error), "host operands must be page-locked (pinned) memory");
                return FMM_ERR_INVALID_ARG;
            }
            mapped[i] = at.devicePointer;
        }
    }
    const bool mapped_all = mapped[0] && mapped[1] && mapped[2];
    if (p->opt.host_copy == 0) {
        // judge the earlier calls' input transfers that have completed
        for (int i = 0; i < fmm_plan_s::kJudgeRing; ++i) {
            if (p->hx_bytes[i] <= 0.0) continue;
            const cudaError_t q = cudaEventQuery(p->hx[i][1]);
            if (q == cudaErrorNotReady) {
                cudaGetLastError();   // a status, not an error of this call
                continue;
            }
            float ms = 0.f;
            if (q == cudaSuccess && cudaEventElapsedTime(&ms, p->hx[i][0], p->hx[i][1]) == cudaSuccess && ms > 0.f &&
                p->hx_bytes[i] / ((double)ms * 1e6) < kHostStallGBs)
                p->host_sm_latched = 1;
            cudaGetLastError();
            p->hx_bytes[i] = 0.0;
        }
    }
    const bool sm_copy = mapped_all && (p->opt.host_copy == 2 || (p->opt.host_copy == 0 && p->host_sm_latched));
    // the library default times this call's input transfers on the copy engines
    // (in the next ring slot, unless that slot still waits for its call)
    const int slot = p->hx_next;
    const bool judge = p->opt.host_copy == 0 && !sm_copy && p->host_calls > 0 && mapped_all &&
                       p->hx_bytes[slot] <= 0.0;
    p->host_calls += 1;
    double in_bytes = 0.0;
    fmm_plan_s* c = p->child;
    cudaEvent_t* ev = p->hev;
    float** q = p->hq;
    const long long hm = p->hm, hk = p->hk, hn = p->hn;
    FMM_CUDA(cudaEventRecord(ev[0], stream));
    FMM_CUDA(cudaStreamWaitEvent(p->s_h2d, ev[0], 0));
    FMM_CUDA(cudaStreamWaitEvent(p->s_d2h, ev[0], 0));
    if (judge) FMM_CUDA(cudaEventRecord(p->hx[slot][0], p->s_h2d));
    // valid part of quadrant (qi, qj) of an R x W host matrix split at (h, w)
    // host_c / host: the caller's pointer; host_m: its device mapping (SM copies)
    auto copy = [&](bool to_dev, float* dev, long long ldd, const float* host_c, float* host, const void* host_m,
                    long long ldh, long long R, long long W, long long h, long long w, int qi, int qj) -> fmm_status_t {
        const long long r0 = qi * h, c0 = qj * w;
        const long long rows = std::min(h, R - r0), cols = std::min(w, W - c0);
        if (rows <= 0 || cols <= 0) return FMM_OK;
        if (to_dev) in_bytes += 4.0 * (double)(rows * cols);
        if (sm_copy) {
            float* hm_ = const_cast<float*>(static_cast<const float*>(host_m)) + r0 * ldh + c0;
            if (to_dev) FMM_CUDA(launch_host_copy2d(hm_, ldh, dev, ldd, rows, cols, p->s_h2d));
            else FMM_CUDA(launch_host_copy2d(dev, ldd, hm_, ldh, rows, cols, p->s_d2h));
            p->launches += 1;
            return FMM_OK;
        }
        if (to_dev)
            FMM_CUDA(cudaMemcpy2DAsync(dev, ldd * 4, host_c + r0 * ldh + c0, ldh * 4, cols * 4, rows,
                                       cudaMemcpyHostToDevice, p->s_h2d));
        else
            FMM_CUDA(cudaMemcpy2DAsync(host + r0 * ldh + c0, ldh * 4, dev, ldd * 4, cols * 4, rows,
                                       cudaMemcpyDeviceToHost, p->s_d2h));
        return FMM_OK;
    };
    auto inA = [&](int i) {
        return copy(true, q[i], hk, A, nullptr, mapped[0], p->lda, p->M, p->K, hm, hk, i / 2, i % 2);
    };
    auto inB = [&](int i) {
        return copy(true, q[4 + i], hn, B, nullptr, mapped[1], p->ldb, p->K, p->N, hk, hn, i / 2, i % 2);
    };
    auto inC = [&](int i) {
        return copy(true, q[23 + i], hn, C, nullptr, mapped[2], p->ldc, p->M, p->N, hm, hn, i / 2, i % 2);
    };
    auto outC = [&](int i) {
        return copy(false, q[23 + i], hn, nullptr, C, mapped[2], p->ldc, p->M, p->N, hm, hn, i / 2, i % 2);
    };
    fmm_status_t s;
#define FMM_TRY(x) do { if ((s = (x)) != FMM_OK) return s; } while (0)
    if (p->depth == 0) {
        FMM_TRY(inA(0));
        FMM_TRY(inB(0));
        if (beta != 0.0f) FMM_TRY(inC(0));
        FMM_CUDA(cudaEventRecord(ev[1], p->s_h2d));
        if (judge) FMM_CUDA(cudaEventRecord(p->hx[slot][1], p->s_h2d));
        FMM_CUDA(cudaStreamWaitEvent(stream, ev[1], 0));
        FMM_TRY(execute(c, alpha, q[0], q[4], beta, q[23], stream));
        FMM_CUDA(cudaEventRecord(ev[4], stream));
        FMM_CUDA(cudaStreamWaitEvent(p->s_d2h, ev[4], 0));
        FMM_TRY(outC(0));
    } else {
        // Transfers in order of first use, products in an order that lets each
        // C quadrant leave as soon as its U-chain is complete:
        //   P1, P2 -> C11;  T sums (all of B) -> P4;  S sums (A21 last) -> P6, P7
        //   -> C21;  P5 -> C22;  P3 -> C12.
        // Only the last quadrant's device-to-host copy is not hidden.
        FMM_TRY(inA(0)); FMM_TRY(inB(0));                        // A11, B11 -> P1
        FMM_CUDA(cudaEventRecord(ev[1], p->s_h2d));
        FMM_TRY(inA(1)); FMM_TRY(inB(2));                        // A12, B21 -> P2
        FMM_CUDA(cudaEventRecord(ev[2], p->s_h2d));
        if (beta != 0.0f) FMM_TRY(inC(0));
        FMM_CUDA(cudaEventRecord(ev[6], p->s_h2d));              // C11 (beta != 0)
        FMM_TRY(inA(3)); FMM_TRY(inB(1)); FMM_TRY(inB(3));       // A22, B12, B22 -> T sums, P4
        FMM_CUDA(cudaEventRecord(ev[3], p->s_h2d));
        FMM_TRY(inA(2));                                         // A21 -> S sums
        FMM_CUDA(cudaEventRecord(ev[5], p->s_h2d));
        if (beta != 0.0f) for (int i = 1; i < 4; ++i) FMM_TRY(inC(i));
        FMM_CUDA(cudaEventRecord(ev[7], p->s_h2d));              // C12, C21, C22 (beta != 0)
        if (judge) FMM_CUDA(cudaEventRecord(p->hx[slot][1], p->s_h2d));
        float* P[7];
        for (int i = 0; i < 7; ++i) P[i] = q[16 + i];
        QuadPost qp{};
        for (int i = 0; i < 7; ++i) qp.p[i] = P[i];
        for (int i = 0; i < 4; ++i) qp.c[i] = q[23 + i];
        qp.ld = hn; qp.h = hm; qp.w = hn; qp.alpha = alpha; qp.beta = beta;
        // C quadrant i is formed on `stream`, then copied out on the d2h stream
        auto post_out = [&](int i) -> fmm_status_t {
            FMM_CUDA(launch_quad_post(qp, i, stream));
            FMM_CUDA(cudaEventRecord(ev[4], stream));
            FMM_CUDA(cudaStreamWaitEvent(p->s_d2h, ev[4], 0));
            return outC(i);
        };
        QuadPre pa{{q[0], q[1], q[2], q[3]}, {q[8], q[9], q[10], q[11]}, hk, hm, hk};
        QuadPre pb{{q[4], q[5], q[6], q[7]}, {q[12], q[13], q[14], q[15]}, hn, hk, hn};
        FMM_CUDA(cudaStreamWaitEvent(stream, ev[1], 0));
        FMM_TRY(execute(c, 1.f, q[0], q[4], 0.f, P[0], stream));   // P1 = A11 B11
        FMM_CUDA(cudaStreamWaitEvent(stream, ev[2], 0));
        FMM_TRY(execute(c, 1.f, q[1], q[6], 0.f, P[1], stream));   // P2 = A12 B21
        FMM_CUDA(cudaStreamWaitEvent(stream, ev[6], 0));
        FMM_TRY(post_out(0));                                      // C11 = alpha U1 + beta C11
        FMM_CUDA(cudaStreamWaitEvent(stream, ev[3], 0));
        FMM_CUDA(launch_quad_pre(pb, 1, stream));                 // T1..T4
        FMM_TRY(execute(c, 1.f, q[3], q[15], 0.f, P[3], stream));  // P4 = A22 T4
        FMM_CUDA(cudaStreamWaitEvent(stream, ev[5], 0));
        FMM_CUDA(launch_quad_pre(pa, 0, stream));                 // S1..S4
        FMM_TRY(execute(c, 1.f, q[9], q[13], 0.f, P[5], stream));  // P6 = S2 T2
        FMM_TRY(execute(c, 1.f, q[10], q[14], 0.f, P[6], stream)); // P7 = S3 T3
        FMM_CUDA(cudaStreamWaitEvent(stream, ev[7], 0));
        FMM_TRY(post_out(2));                                      // C21 = alpha U6 + beta C21
        FMM_TRY(execute(c, 1.f, q[8], q[12], 0.f, P[4], stream));  // P5 = S1 T1
        FMM_TRY(post_out(3));                                      // C22 = alpha U7 + beta C22
        FMM_TRY(execute(c, 1.f, q[11], q[7], 0.f, P[2], stream));  // P3 = S4 B22
        FMM_TRY(post_out(1));                                      // C12 = alpha U5 + beta C12
        p->launches += 6;
    }
#undef FMM_TRY
    if (judge && in_bytes >= kHostJudgeBytes) {
        p->hx_bytes[slot] = in_bytes;
        p->hx_next = (slot + 1) % fmm_plan_s::kJudgeRing;
    }
    FMM_CUDA(cudaEventRecord(ev[0], p->s_d2h));
    FMM_CUDA(cudaStreamWaitEvent(stream, ev[0], 0));
    p->launches += c->launches;
    c->launches = 0;
    return FMM_OK;
}

// Score the candidates with the registered network (one inference launch) and
// return the index of the smallest predicted time (ties: smaller depth, then
// the larger tile).
fmm_status_t choose_mlp(long long M, long long N, long long K, const fmm_options_t& o, const Cand* c, int n,
                        int* best, cudaStream_t stream) {
    int dev = 0;
    FMM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return FMM_ERR_NO_DEVICE;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_model.dev_params[dev]) {
        FMM_CUDA(cudaMalloc(&g_model.dev_params[dev], sizeof(float) * FMM_MLP_NPARAM));
        FMM_CUDA(cudaMalloc(&g_model.dev_io[dev], sizeof(float) * (16 * 6 + 16)));
    }
    if (g_model.dev_version[dev] != g_model.version) {
        FMM_CUDA(cudaMemcpy(g_model.dev_params[dev], g_model.params, sizeof(float) * FMM_MLP_NPARAM,
                            cudaMemcpyHostToDevice));
        g_model.dev_version[dev] = g_model.version;
    }
    float X[16 * 6], Y[16];
    for (int i = 0; i < n; ++i) {
        raw_features(M, N, K, c[i].depth, c[i].bn, (int)o.precision, X + 6 * i);
        for (int j = 0; j < 6; ++j) X[6 * i + j] = (X[6 * i + j] - g_model.mean[j]) / g_model.stdv[j];
    }
    float* dX = g_model.dev_io[dev];
    float* dY = dX + 16 * 6;
    FMM_CUDA(cudaMemcpyAsync(dX, X, sizeof(float) * 6 * n, cudaMemcpyHostToDevice, stream));
    FMM_CUDA(mlp_forward(g_model.dev_params[dev], dX, dY, n, stream));
    FMM_CUDA(cudaMemcpyAsync(Y, dY, sizeof(float) * n, cudaMemcpyDeviceToHost, stream));
    FMM_CUDA(cudaStreamSynchronize(stream));
    int b = 0;
    for (int i = 1; i < n; ++i) {
        const float d = Y[i] - Y[b];
        if (d < -1e-6f) b = i;
        else if (d <= 1e-6f && (c[i].depth < c[b].depth || (c[i].depth == c[b].depth && c[i].bn > c[b].bn))) b = i;
    }
    *best = b;
    return FMM_OK;
}

// Time each candidate on A, B, C (dense row-major) with the workspace `ws`.
fmm_status_t autotune_core(long long M, long long N, long long K, const fmm_options_t& o, const float* A,
                           const float* B, float* C, char* ws, size_t ws_bytes, const Cand* c, int n, int reps,
                           float* times, cudaStream_t stream) {
    DeviceInfo di;
    fmm_status_t s;
    if ((s = device_info(&di)) != FMM_OK) return s;
    cudaEvent_t e0, e1;
    FMM_CUDA(cudaEventCreate(&e0));
    FMM_CUDA(cudaEventCreate(&e1));
    s = FMM_OK;
    for (int i = 0; i < n && s == FMM_OK; ++i) {
        fmm_plan_s t;
        fmm_options_t od = o;
        od.host_operands = 0;   // candidates are timed on device operands
        make_tmp(t, M, N, K, K, N, N, od, c[i].depth, c[i].bn);
        size_t need = 0;
        layout(&t, nullptr, &need);
        if (need > ws_bytes) { s = FMM_ERR_WORKSPACE; break; }
        layout(&t, ws, nullptr);
        t.ws = ws;
        t.ws_bytes = ws_bytes;
        t.num_sms = di.num_sms;
        std::vector<float> ms;
        for (int r = 0; r <= reps && s == FMM_OK; ++r) {
            cudaEventRecord(e0, stream);
            s = execute(&t, 1.f, A, B, 0.f, C, stream);
            cudaEventRecord(e1, stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) { s = cuda_fail(cudaGetLastError(), "autotune"); break; }
            float x = 0.f;
            cudaEventElapsedTime(&x, e0, e1);
            if (r > 0) ms.push_back(x);
        }
        if (s != FMM_OK) break;
        std::sort(ms.begin(), ms.end());
        times[i] = ms.empty() ? 0.f : ms[ms.size() / 2];
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return s;
}

size_t scratch_bytes(long long M, long long N, long long K) {
    return align_up((size_t)M * K * 4, 256) + align_up((size_t)K * N * 4, 256) + align_up((size_t)M * N * 4, 256);
}

// Choose (depth, leaf tile) for a plan and the workspace bytes it needs.
fmm_status_t plan_choose(long long M, long long N, long long K, long long lda, long long ldb, long long ldc,
                         const fmm_options_t& o, void* ws, size_t ws_bytes, size_t* need, int& depth, int& bn,
                         cudaStream_t stream, bool query) {
    if (o.planner == FMM_PLANNER_FIXED || o.algo == FMM_ALGO_CLASSICAL || M == 0 || N == 0 || K == 0) {
        depth = o.depth >= 0 ? o.depth : fixed_depth(M, N, K, o.cutoff);
        if (o.algo == FMM_ALGO_CLASSICAL) {   // one launch spans all of C: tile by M, N
            bn = o.leaf_tile ? o.leaf_tile : auto_tile(M, N, 0, o);
            *need = plan_bytes(M, N, K, lda, ldb, ldc, o, depth, bn);
            return FMM_OK;
        }
        bn = o.leaf_tile ? o.leaf_tile : auto_tile(M, N, depth, o);
        *need = plan_bytes(M, N, K, lda, ldb, ldc, o, depth, bn);
        return FMM_OK;
    }
    Cand c[16];
    const int n = candidates(M, N, K, o, c);
    if (o.planner == FMM_PLANNER_MLP && g_model.set) {
        int b = 0;
        fmm_status_t s = choose_mlp(M, N, K, o, c, n, &b, stream);
        if (s != FMM_OK) return s;
        depth = c[b].depth;
        bn = c[b].bn;
        *need = plan_bytes(M, N, K, lda, ldb, ldc, o, depth, bn);
        return FMM_OK;
    }
    // exhaustive (also the fallback of the learned planner): the largest
    // candidate plus scratch operands for the timing runs
    size_t mx = 0;
    fmm_options_t od = o;
    od.host_operands = 0;
    for (int i = 0; i < n; ++i) {
        fmm_plan_s t;
        make_tmp(t, M, N, K, K, N, N, od, c[i].depth, c[i].bn);
        size_t q = 0;
        layout(&t, nullptr, &q);
        mx = std::max(mx, q);
        mx = std::max(mx, plan_bytes(M, N, K, lda, ldb, ldc, o, c[i].depth, c[i].bn));
    }
    *need = align_up(mx, 256) + scratch_bytes(M, N, K);
    depth = c[0].depth;
    bn = c[0].bn;
    if (query) return FMM_OK;
    if (!ws || ws_bytes < *need) return FMM_ERR_WORKSPACE;
    char* base = static_cast<char*>(ws);
    float* sA = reinterpret_cast<float*>(base + align_up(mx, 256));
    float* sB = reinterpret_cast<float*>(reinterpret_cast<char*>(sA) + align_up((size_t)M * K * 4, 256));
    float* sC = reinterpret_cast<float*>(reinterpret_cast<char*>(sB) + align_up((size_t)K * N * 4, 256));
    FMM_CUDA(launch_fill(sA, (size_t)M * K, 12345u, stream));
    FMM_CUDA(launch_fill(sB, (size_t)K * N, 54321u, stream));
    float times[16];
    fmm_status_t s = autotune_core(M, N, K, o, sA, sB, sC, base, align_up(mx, 256), c, n, 1, times, stream);
    if (s != FMM_OK) return s;
    int b = 0;
    for (int i = 1; i < n; ++i)
        if (times[i] < times[b]) b = i;
    depth = c[b].depth;
    bn = c[b].bn;
    return FMM_OK;
}

}  // namespace

extern "C" {

fmm_status_t fmm_plan_features(int64_t M, int64_t N, int64_t K, int depth, int leaf_tile, int precision,
                               float* out6) {
    if (!out6 || M < 0 || N < 0 || K < 0) return FMM_ERR_INVALID_ARG;
    raw_features(M, N, K, depth, leaf_tile, precision, out6);
    return FMM_OK;
}

fmm_status_t fmm_set_cost_model(const float* params, const float* mean6, const float* std6) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!params) {
        g_model.set = false;
        return FMM_OK;
    }
    if (!mean6 || !std6) return FMM_ERR_INVALID_ARG;
    for (int j = 0; j < 6; ++j)
        if (!(std6[j] > 0.f)) return FMM_ERR_INVALID_ARG;
    memcpy(g_model.params, params, sizeof(g_model.params));
    memcpy(g_model.mean, mean6, sizeof(g_model.mean));
    memcpy(g_model.stdv, std6, sizeof(g_model.stdv));
    g_model.set = true;
    g_model.version += 1;
    return FMM_OK;
}

fmm_status_t fmm_autotune(int64_t M, int64_t N, int64_t K, const fmm_options_t* opt, const float* A, const float* B,
                          float* C, void* workspace, size_t workspace_bytes, size_t* workspace_needed, int* depths,
                          int* tiles, float* times_ms, int* count, int reps, fmm_stream_t stream) {
    if (M <= 0 || N <= 0 || K <= 0 || reps < 1) return FMM_ERR_INVALID_ARG;
    fmm_options_t o;
    if (opt) o = *opt; else fmm_options_default(&o);
    fmm_status_t s = check_opts(&o);
    if (s != FMM_OK) return s;
    if (o.algo == FMM_ALGO_CLASSICAL) return FMM_ERR_UNSUPPORTED;   // candidates are Winograd plans
    Cand c[16];
    const int n = candidates(M, N, K, o, c);
    size_t mx = 0;
    for (int i = 0; i < n; ++i) mx = std::max(mx, plan_bytes(M, N, K, K, N, N, o, c[i].depth, c[i].bn));
    if (workspace_needed) *workspace_needed = mx;
    if (count) *count = n;
    for (int i = 0; i < n; ++i) {
        if (depths) depths[i] = c[i].depth;
        if (tiles) tiles[i] = c[i].bn;
    }
    if (!workspace) return FMM_OK;
    if (!A || !B || !C) return FMM_ERR_INVALID_ARG;
    if (workspace_bytes < mx) return FMM_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(workspace) & 255) return FMM_ERR_ALIGNMENT;
    float t[16];
    s = autotune_core(M, N, K, o, A, B, C, static_cast<char*>(workspace), workspace_bytes, c, n, reps, t,
                      (cudaStream_t)stream);
    if (s != FMM_OK) return s;
    if (times_ms)
        for (int i = 0; i < n; ++i) times_ms[i] = t[i];
    return FMM_OK;
}

}  // extern "C"

namespace {

fmm_status_t batched_run(fmm_batched_s* b, cudaStream_t stream) {
    fmm_status_t s;
    if (b->fp16 && b->count > 0) {   // per-problem operand scales first: the splits and sub-plans apply them
        FMM_CUDA(cudaMemsetAsync(b->d_absmax, 0, 2 * sizeof(unsigned) * (size_t)b->count, stream));
        FMM_CUDA(launch_batched_absmax(b->d_ajobs, b->najobs, b->ajob_tiles, stream));
        FMM_CUDA(launch_batched_fp16_scales(b->d_absmax, b->d_bound, b->d_scales, b->count, stream));
        b->launches += 2;
    }
    if (b->njobs > 0) {
        if (b->pre) FMM_CUDA(launch_batched_split(b->d_sjobs, b->njobs, b->job_tiles, b->split_kind, stream));
        else FMM_CUDA(launch_batched_copy(b->d_jobs, b->njobs, b->job_tiles, stream));
        b->launches += 1;
    }
    for (size_t j = 0; j < b->subs.size(); ++j) {
        const int i = b->sub_problem[j];
        if ((s = winograd_pre(b->subs[j], b->A[i], b->B[i], stream)) != FMM_OK) return s;
    }
    if (b->total_tiles > 0) {
        GemmArgs args;
        memset(&args, 0, sizeof(args));
        args.ext_maps = b->d_maps;
        args.ext_groups = b->d_groups;
        args.num_groups = b->num_groups;
        args.total_tiles = b->total_tiles;
        args.raster_m = 16;
        args.status = b->status;
        // static round robin over tiles sorted by K (longest first) balances the
        // uneven tiles like LPT; dynamic order measured 2.5 % slower here
        if (b->pair) FMM_CUDA(launch_leaf_gemm_pair(args, b->mode, b->num_sms, stream));
        else FMM_CUDA(launch_leaf_gemm(args, b->mode, b->bn, b->num_sms, stream));
        b->launches += 1;
    }
    for (size_t j = 0; j < b->subs.size(); ++j) {
        const int i = b->sub_problem[j];
        if ((s = winograd_post(b->subs[j], b->alpha[i], b->beta[i], b->C[i], stream)) != FMM_OK) return s;
    }
    for (int i = 0; i < b->count; ++i)
        if (b->scale_only[i] && b->M[i] > 0 && b->N[i] > 0) {
            FMM_CUDA(launch_scale(b->C[i], b->ldc[i], b->M[i], b->N[i], b->beta[i], stream));
            b->launches += 1;
        }
    for (auto* q : b->subs) { b->launches += q->launches; q->launches = 0; }
    return FMM_OK;
}


// Size class of a batched problem: its smallest and largest dimension, each
// rounded to the nearest power of two (the smallest sets how deep the
// recursion can go; the largest, how much work a level saves).
int size_class(long long M, long long N, long long K) {
    const long long mn = std::min(std::min(M, N), K), mx = std::max(std::max(M, N), K);
    const int a = (int)std::lround(std::log2((double)std::max(mn, 1LL)));
    const int c = (int)std::lround(std::log2((double)std::max(mx, 1LL)));
    return a * 64 + c;
}

// Leaf tiles a batched planner chooses among (one per launch).
std::vector<int> batched_tiles(const fmm_options_t& o) {
    if (o.leaf_tile) return {o.leaf_tile};
    if (o.precision == FMM_PREC_TF32) return {256, 128};
    return {512, 256};
}

struct BatchedTuner {
    int count;
    const int64_t *M, *N, *K, *lda, *ldb;
    const float* const* A;
    const float* const* B;
    const float* alpha;
    fmm_options_t o;
    char* region;                 // where trial plans are built
    std::vector<float*> Cs;       // scratch outputs (M_i x N_i)
    std::vector<int64_t> ldc;
    std::vector<float> zeros;
    int num_sms;
    cudaStream_t stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;

    // Whole-batch time of one configuration: built in `region`, one untimed
    // run, then the best of two timed runs.
    fmm_status_t time(const std::vector<int>& depth, int tile, float* ms) {
        fmm_batched_s t;
        t.num_sms = num_sms;
        fmm_status_t s = batched_build(&t, count, M, N, K, A, lda, B, ldb, Cs.data(), ldc.data(), alpha,
                                       zeros.data(), o, region, nullptr, depth.data(), tile);
        if (s != FMM_OK) return s;
        for (auto* q : t.subs) q->num_sms = num_sms;
        if ((s = batched_run(&t, stream)) != FMM_OK) return s;
        float best = 1e30f;
        for (int r = 0; r < 2; ++r) {
            FMM_CUDA(cudaEventRecord(e0, stream));
            if ((s = batched_run(&t, stream)) != FMM_OK) return s;
            FMM_CUDA(cudaEventRecord(e1, stream));
            FMM_CUDA(cudaEventSynchronize(e1));
            float x = 0.f;
            FMM_CUDA(cudaEventElapsedTime(&x, e0, e1));
            best = std::min(best, x);
        }
        unsigned w = 0;
        FMM_CUDA(cudaMemcpy(&w, t.status, sizeof(w), cudaMemcpyDeviceToHost));
        if (w & FMM_DEV_TIMEOUT_BIT) return FMM_ERR_TIMEOUT;
        *ms = best;
        return FMM_OK;
    }
};

// Per-size-class plan of a batched launch.  depth[i] receives every problem's
// depth (-1: no product) and *tile the launch's leaf tile.
//   FIXED       the fixed rule per problem (or the caller's depth).
//   EXHAUSTIVE  for each leaf tile candidate, one pass of coordinate descent
//               over the size classes (largest work first): every candidate
//               depth of the class is timed as a whole-batch launch on scratch
//               outputs, the others held; a change is kept when it saves >= 1 %.
//   MLP         the registered cost model predicts log(ms) of every problem at
//               every candidate (depth, tile) in one inference launch; each
//               class takes the depth of least predicted sum, the launch the
//               tile of least predicted total (no model: EXHAUSTIVE).
// Scratch (EXHAUSTIVE / MLP) follows `region_bytes` in the workspace.
fmm_status_t batched_choose(int count, const int64_t* M, const int64_t* N, const int64_t* K, const float* const* A,
                            const int64_t* lda, const float* const* B, const int64_t* ldb, const float* alpha,
                            const fmm_options_t& o, char* ws, size_t region_bytes, int num_sms, cudaStream_t stream,
                            std::vector<int>& depth, std::vector<int>& cls, int& nclasses, int& tile) {
    depth.assign(count, -1);
    cls.assign(count, -1);
    std::vector<int> ids;
    for (int i = 0; i < count; ++i) {
        depth[i] = batched_fixed_depth(M[i], N[i], K[i], alpha[i], o);
        if (depth[i] < 0) continue;
        const int c = size_class(M[i], N[i], K[i]);
        auto it = std::find(ids.begin(), ids.end(), c);
        cls[i] = (int)(it - ids.begin());
        if (it == ids.end()) ids.push_back(c);
    }
    nclasses = (int)ids.size();
    const std::vector<int> tiles = batched_tiles(o);
    tile = o.leaf_tile ? o.leaf_tile : tiles[0];
    if (o.planner == FMM_PLANNER_FIXED || o.depth >= 0 || nclasses == 0) return FMM_OK;
    // classes, largest work first; a class's candidate depths reach its deepest member's limit
    std::vector<double> work(nclasses, 0.0);
    std::vector<int> cmax(nclasses, 0);
    for (int i = 0; i < count; ++i)
        if (cls[i] >= 0) {
            work[cls[i]] += 2.0 * (double)M[i] * (double)N[i] * (double)K[i];
            cmax[cls[i]] = std::max(cmax[cls[i]], batched_max_depth(M[i], N[i], K[i]));
        }
    std::vector<int> order(nclasses);
    for (int c = 0; c < nclasses; ++c) order[c] = c;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work[x] > work[y]; });
    auto with_class_depth = [&](const std::vector<int>& base, int c, int d) {
        std::vector<int> r = base;
        for (int i = 0; i < count; ++i)
            if (cls[i] == c) r[i] = std::min(d, batched_max_depth(M[i], N[i], K[i]));
        return r;
    };
    char* scratch = ws + align_up(region_bytes, 256);
    // whole-batch timings on scratch outputs (the exhaustive search, and the
    // check on the cost model's proposal)
    BatchedTuner T;
    T.count = count; T.M = M; T.N = N; T.K = K; T.lda = lda; T.ldb = ldb; T.A = A; T.B = B; T.alpha = alpha;
    T.o = o; T.region = ws; T.num_sms = num_sms; T.stream = stream;
    T.Cs.assign(count, nullptr);
    T.ldc.assign(count, 1);
    T.zeros.assign(count, 0.0f);
    auto carve_outputs = [&]() {
        Carver cv(scratch);
        for (int i = 0; i < count; ++i) {
            T.ldc[i] = std::max<int64_t>(N[i], 1);
            T.Cs[i] = cv.take<float>((size_t)M[i] * (size_t)T.ldc[i]);
        }
    };
    struct Events {
        BatchedTuner& t;
        ~Events() {
            if (t.e0) cudaEventDestroy(t.e0);
            if (t.e1) cudaEventDestroy(t.e1);
        }
    } events{T};
    if (o.planner == FMM_PLANNER_MLP && g_model.set) {
        // rows: (problem, tile, depth) for every depth up to the problem's limit
        std::vector<float> X;
        std::vector<int> row_i, row_t, row_d;
        for (int i = 0; i < count; ++i) {
            if (cls[i] < 0) continue;
            for (int t = 0; t < (int)tiles.size(); ++t)
                for (int d = 0; d <= batched_max_depth(M[i], N[i], K[i]); ++d) {
                    float f[6];
                    raw_features(M[i], N[i], K[i], d, tiles[t], (int)o.precision, f);
                    for (int j = 0; j < 6; ++j) X.push_back((f[j] - g_model.mean[j]) / g_model.stdv[j]);
                    row_i.push_back(i); row_t.push_back(t); row_d.push_back(d);
                }
        }
        const int rows = (int)row_i.size();
        float* dX = reinterpret_cast<float*>(scratch);
        float* dY = dX + align_up((size_t)rows * 6, 64);
        float* dP = dY + align_up((size_t)rows, 64);
        {
            std::lock_guard<std::mutex> lk(g_mu);
            FMM_CUDA(cudaMemcpyAsync(dP, g_model.params, sizeof(float) * FMM_MLP_NPARAM, cudaMemcpyHostToDevice, stream));
        }
        FMM_CUDA(cudaMemcpyAsync(dX, X.data(), sizeof(float) * X.size(), cudaMemcpyHostToDevice, stream));
        FMM_CUDA(mlp_forward(dP, dX, dY, rows, stream));
        std::vector<float> Y(rows);
        FMM_CUDA(cudaMemcpyAsync(Y.data(), dY, sizeof(float) * rows, cudaMemcpyDeviceToHost, stream));
        FMM_CUDA(cudaStreamSynchronize(stream));
        // predicted ms of problem i at (tile t, depth d); ties: smaller depth, larger tile
        const int nd = 5, nt = (int)tiles.size();
        std::vector<double> pms((size_t)count * nt * nd, 0.0);
        for (int r = 0; r < rows; ++r) pms[((size_t)row_i[r] * nt + row_t[r]) * nd + row_d[r]] = std::exp((double)Y[r]);
        double best_total = 1e300;
        std::vector<int> best_cd(nclasses, 0);
        for (int t = 0; t < (int)tiles.size(); ++t) {
            double total = 0.0;
            std::vector<int> cd(nclasses, 0);
            for (int c = 0; c < nclasses; ++c) {
                double bd = 1e300;
                for (int d = 0; d <= cmax[c]; ++d) {
                    // a depth the deepest member can take but a shallower one cannot
                    // is predicted at the member's own limit, as it would run
                    double v = 0.0;
                    for (int i = 0; i < count; ++i)
                        if (cls[i] == c)
                            v += pms[((size_t)i * nt + t) * nd + std::min(d, batched_max_depth(M[i], N[i], K[i]))];
                    if (v < bd * (1.0 - 1e-6)) { bd = v; cd[c] = d; }
                }
                total += bd;
            }
            if (total < best_total * (1.0 - 1e-6)) { best_total = total; best_cd = cd; tile = tiles[t]; }
        }
        std::vector<int> proposed(depth);
        for (int i = 0; i < count; ++i)
            if (cls[i] >= 0) proposed[i] = std::min(best_cd[cls[i]], batched_max_depth(M[i], N[i], K[i]));
        // the model predicts each problem alone; inside one shared launch a level
        // also costs its own addition launches, so the proposal is timed against
        // the fixed rule's plan as a whole batch and kept only if faster (the
        // inference buffers are done with: the outputs reuse that scratch)
        carve_outputs();
        FMM_CUDA(cudaEventCreate(&T.e0));
        FMM_CUDA(cudaEventCreate(&T.e1));
        const int fixed_tile = o.leaf_tile ? o.leaf_tile : tiles[0];
        float t_model = 0.f, t_fixed = 0.f;
        fmm_status_t s;
        if ((s = T.time(proposed, tile, &t_model)) != FMM_OK) return s;
        if ((s = T.time(depth, fixed_tile, &t_fixed)) != FMM_OK) return s;
        if (t_model < t_fixed) depth = proposed;
        else tile = fixed_tile;
        return FMM_OK;
    }
    // exhaustive: whole-batch timings on scratch outputs
    carve_outputs();
    FMM_CUDA(cudaEventCreate(&T.e0));
    FMM_CUDA(cudaEventCreate(&T.e1));
    fmm_status_t s = FMM_OK;
    float best_total = 1e30f;
    std::vector<int> best_depth = depth;
    for (int t = 0; t < (int)tiles.size() && s == FMM_OK; ++t) {
        std::vector<int> cur = depth;   // start from the fixed rule
        float cur_ms = 0.f;
        if ((s = T.time(cur, tiles[t], &cur_ms)) != FMM_OK) break;
        for (int c : order) {
            int at = -1;
            for (int i = 0; i < count; ++i)
                if (cls[i] == c) { at = cur[i]; break; }
            for (int d = 0; d <= cmax[c] && s == FMM_OK; ++d) {
                if (d == at) continue;
                std::vector<int> trial = with_class_depth(cur, c, d);
                float ms = 0.f;
                if ((s = T.time(trial, tiles[t], &ms)) != FMM_OK) break;
                if (ms < 0.99f * cur_ms) { cur = trial; cur_ms = ms; at = d; }
            }
            if (s != FMM_OK) break;
        }
        if (s == FMM_OK && cur_ms < best_total) { best_total = cur_ms; best_depth = cur; tile = tiles[t]; }
    }
    if (s != FMM_OK) return s;
    depth = best_depth;
    return FMM_OK;
}

// Workspace of a batched plan: the largest plan any candidate configuration
// builds (each problem at its most demanding depth, the larger tile's tables),
// then, for EXHAUSTIVE / MLP, scratch outputs and inference buffers.
fmm_status_t batched_need(int count, const int64_t* M, const int64_t* N, const int64_t* K, const int64_t* lda,
                          const int64_t* ldb, const int64_t* ldc, const float* alpha, const float* beta,
                          const fmm_options_t& o, size_t* region, size_t* total) {
    fmm_status_t s;
    std::vector<int> dfix(count);
    for (int i = 0; i < count; ++i) dfix[i] = batched_fixed_depth(M[i], N[i], K[i], alpha[i], o);
    const bool tune = o.planner != FMM_PLANNER_FIXED && o.depth < 0;
    size_t r = 0;
    const std::vector<int> tiles = tune ? batched_tiles(o) : std::vector<int>{o.leaf_tile};
    for (int tile : tiles) {
        size_t need = 0;
        fmm_batched_s tmp;
        if ((s = batched_build(&tmp, count, M, N, K, nullptr, lda, nullptr, ldb, nullptr, ldc, alpha, beta, o, nullptr,
                               &need, dfix.data(), tile)) != FMM_OK)
            return s;
        r = std::max(r, need);
        if (!tune) continue;
        // every problem at its most demanding candidate depth, priced one problem at a time
        size_t sum = 0;
        for (int i = 0; i < count; ++i) {
            size_t best = 0;
            for (int d = 0; d <= batched_max_depth(M[i], N[i], K[i]); ++d) {
                size_t ni = 0;
                fmm_batched_s one;
                if ((s = batched_build(&one, 1, M + i, N + i, K + i, nullptr, lda + i, nullptr, ldb + i, nullptr,
                                       ldc + i, alpha + i, beta + i, o, nullptr, &ni, &d, tile)) != FMM_OK)
                    return s;
                best = std::max(best, ni);
            }
            sum += best;
        }
        r = std::max(r, sum + (size_t)count * 4096 + (1u << 20));
    }
    *region = align_up(r, 256);
    size_t t = *region;
    if (tune) {
        size_t c = 0;
        for (int i = 0; i < count; ++i) c += align_up((size_t)M[i] * (size_t)std::max<int64_t>(N[i], 1) * 4, 256);
        size_t rows = 0;
        for (int i = 0; i < count; ++i) rows += (size_t)(batched_max_depth(M[i], N[i], K[i]) + 1) * 2;
        const size_t io = (align_up(rows * 6, 64) + align_up(rows, 64) + FMM_MLP_NPARAM) * 4 + 1024;
        t += std::max(c, io);
    }
    *total = align_up(t, 256);
    return FMM_OK;
}

}  // namespace

extern "C" {

fmm_status_t fmm_batched_plan(fmm_batched_t* out, int count, const int64_t* M, const int64_t* N, const int64_t* K,
                              const float* const* A, const int64_t* lda, const float* const* B, const int64_t* ldb,
                              float* const* C, const int64_t* ldc, const float* alpha, const float* beta,
                              const fmm_options_t* opt, void* workspace, size_t workspace_bytes,
                              size_t* workspace_needed, fmm_stream_t stream) {
    if (out) *out = nullptr;
    fmm_status_t s = batched_check(count, M, N, K, A, lda, B, ldb, C, ldc, alpha, beta, opt);
    if (s != FMM_OK) return s;
    fmm_options_t o;
    if (opt) o = *opt; else fmm_options_default(&o);
    size_t region = 0, need = 0;
    if ((s = batched_need(count, M, N, K, lda, ldb, ldc, alpha, beta, o, &region, &need)) != FMM_OK) return s;
    if (workspace_needed) *workspace_needed = need;
    if (!out) return FMM_OK;
    DeviceInfo di;
    if ((s = device_info(&di)) != FMM_OK) return s;
    if (count > 0 && (!A || !B || !C)) return FMM_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < need) return FMM_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(workspace) & 255) return FMM_ERR_ALIGNMENT;
    std::vector<int> depth, cls;
    int nclasses = 0, tile = 0;
    if ((s = batched_choose(count, M, N, K, A, lda, B, ldb, alpha, o, static_cast<char*>(workspace), region,
                            di.num_sms, (cudaStream_t)stream, depth, cls, nclasses, tile)) != FMM_OK)
        return s;
    fmm_batched_s* b = new (std::nothrow) fmm_batched_s();
    if (!b) return FMM_ERR_OOM;
    b->num_sms = di.num_sms;
    if ((s = batched_build(b, count, M, N, K, A, lda, B, ldb, C, ldc, alpha, beta, o, static_cast<char*>(workspace),
                           nullptr, depth.data(), tile)) != FMM_OK) {
        delete b;
        return s;
    }
    b->cls = cls;
    b->nclasses = nclasses;
    for (auto* q : b->subs) q->num_sms = di.num_sms;
    *out = b;
    return FMM_OK;
}

fmm_status_t fmm_batched_run(fmm_batched_t b, fmm_stream_t stream_) {
    if (!b) return FMM_ERR_INVALID_ARG;
    return batched_run(b, (cudaStream_t)stream_);
}

void fmm_batched_free(fmm_batched_t b) { delete b; }

fmm_status_t fmm_batched_classes(fmm_batched_t b, int* classes, int* nclasses, int* leaf_tile) {
    if (!b) return FMM_ERR_INVALID_ARG;
    if (classes) for (int i = 0; i < b->count; ++i) classes[i] = b->cls.empty() ? -1 : b->cls[i];
    if (nclasses) *nclasses = b->nclasses;
    if (leaf_tile) *leaf_tile = b->tile;
    return FMM_OK;
}

fmm_status_t fmm_batched_info(fmm_batched_t b, int* depths, int64_t* total_tiles, int64_t* launches) {
    if (!b) return FMM_ERR_INVALID_ARG;
    if (depths) for (int i = 0; i < b->count; ++i) depths[i] = b->depth[i];
    if (total_tiles) *total_tiles = b->total_tiles;
    if (launches) *launches = b->launches;
    return FMM_OK;
}

fmm_status_t fmm_options_default(fmm_options_t* o) {
    if (!o) return FMM_ERR_INVALID_ARG;
    memset(o, 0, sizeof(*o));
    o->depth = -1;
    o->cutoff = 2048;
    o->leaf_tile = 0;
    o->precision = FMM_PREC_FP32;
    o->odd = FMM_ODD_AUTO;
    o->planner = FMM_PLANNER_FIXED;
    o->algo = FMM_ALGO_WINOGRAD;
    o->host_operands = 0;
    o->refine_fp64 = 0;
    o->fuse_last = 0;
    o->host_copy = 0;
    return FMM_OK;
}

const char* fmm_status_string(fmm_status_t s) {
    switch (s) {
        case FMM_OK: return "FMM_OK";
        case FMM_ERR_INVALID_ARG: return "FMM_ERR_INVALID_ARG";
        case FMM_ERR_ALIGNMENT: return "FMM_ERR_ALIGNMENT";
        case FMM_ERR_SHAPE_MISMATCH: return "FMM_ERR_SHAPE_MISMATCH";
        case FMM_ERR_OOM: return "FMM_ERR_OOM";
        case FMM_ERR_CUDA: return "FMM_ERR_CUDA";
        case FMM_ERR_UNSUPPORTED: return "FMM_ERR_UNSUPPORTED";
        case FMM_ERR_TIMEOUT: return "FMM_ERR_TIMEOUT";
        case FMM_ERR_NO_DEVICE: return "FMM_ERR_NO_DEVICE";
        case FMM_ERR_WORKSPACE: return "FMM_ERR_WORKSPACE";
    }
    return "FMM_ERR_UNKNOWN";
}

const char* fmm_last_error(void) { return g_last_error; }

fmm_status_t fmm_plan(fmm_plan_t* out, int64_t M, int64_t N, int64_t K, int64_t lda, int64_t ldb, int64_t ldc,
                      const fmm_options_t* opt, void* workspace, size_t workspace_bytes, size_t* workspace_needed,
                      fmm_stream_t stream) {
    if (out) *out = nullptr;
    if (M < 0 || N < 0 || K < 0) return FMM_ERR_INVALID_ARG;
    if (M > INT32_MAX || N > INT32_MAX || K > INT32_MAX) return FMM_ERR_INVALID_ARG;
    if (lda < (K > 0 ? K : 1) || ldb < (N > 0 ? N : 1) || ldc < (N > 0 ? N : 1)) return FMM_ERR_INVALID_ARG;
    fmm_options_t o;
    if (opt) o = *opt; else fmm_options_default(&o);
    fmm_status_t s = check_opts(&o);
    if (s != FMM_OK) return s;
    int depth = 0, bn = 256;
    size_t need = 0;
    // the planner may time candidates on scratch operands carved from the workspace
    const bool ws_ok = workspace && !(reinterpret_cast<uintptr_t>(workspace) & 255);
    if ((s = plan_choose(M, N, K, lda, ldb, ldc, o, ws_ok ? workspace : nullptr, workspace_bytes, &need, depth, bn,
                         (cudaStream_t)stream, out == nullptr)) != FMM_OK)
        return s;
    fmm_plan_s tmp;
    make_tmp(tmp, M, N, K, lda, ldb, ldc, o, depth, bn);
    if (workspace_needed) *workspace_needed = need;
    if (!out) return FMM_OK;
    DeviceInfo di;
    if ((s = device_info(&di)) != FMM_OK) return s;
    if (!workspace || workspace_bytes < need) return FMM_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(workspace) & 255) return FMM_ERR_ALIGNMENT;
    fmm_plan_s* p = new (std::nothrow) fmm_plan_s(tmp);
    if (!p) return FMM_ERR_OOM;
    p->ws = static_cast<char*>(workspace);
    p->ws_bytes = workspace_bytes;
    p->num_sms = di.num_sms;
    layout(p, p->ws, nullptr);
    cudaError_t e = cudaMemsetAsync(p->status, 0, 64 * sizeof(unsigned), (cudaStream_t)stream);
    if (e != cudaSuccess) { delete p; return cuda_fail(e, "cudaMemsetAsync(status)"); }

    if (p->host) {
        fmm_plan_s c;
        make_child(p, c);
        p->child = new (std::nothrow) fmm_plan_s(c);
        if (!p->child) { fmm_free(p); return FMM_ERR_OOM; }
        layout(p->child, p->child_ws, nullptr);
        p->child->ws = p->child_ws;
        p->child->ws_bytes = p->child_ws_bytes;
        p->child->num_sms = di.num_sms;
        e = cudaMemsetAsync(p->child->status, 0, 64 * sizeof(unsigned), (cudaStream_t)stream);
        // the child's kernels report into the host plan's status word, which
        // fmm_get_device_status reads
        p->child->status = p->status;
        // zero the quadrant buffers once: each call rewrites only the valid parts,
        // so the padding rows/columns stay zero
        const size_t qa = (size_t)(p->hm * p->hk), qb = (size_t)(p->hk * p->hn), qc = (size_t)(p->hm * p->hn);
        for (int i = 0; i < 4 && e == cudaSuccess; ++i) {
            if (p->hq[i]) e = cudaMemsetAsync(p->hq[i], 0, qa * 4, (cudaStream_t)stream);
            if (e == cudaSuccess && p->hq[4 + i]) e = cudaMemsetAsync(p->hq[4 + i], 0, qb * 4, (cudaStream_t)stream);
            if (e == cudaSuccess && p->hq[23 + i]) e = cudaMemsetAsync(p->hq[23 + i], 0, qc * 4, (cudaStream_t)stream);
        }
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->s_h2d, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->s_d2h, cudaStreamNonBlocking);
        for (int i = 0; i < 8 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&p->hev[i], cudaEventDisableTiming);
        for (int i = 0; i < fmm_plan_s::kJudgeRing * 2 && e == cudaSuccess; ++i)
            e = cudaEventCreate(&p->hx[i / 2][i % 2]);
        if (e != cudaSuccess) { fmm_free(p); return cuda_fail(e, "host-resident plan setup"); }
    }
    p->last_stream = (cudaStream_t)stream;
    *out = p;
    return FMM_OK;
}

fmm_status_t fmm_gemm(fmm_plan_t p, float alpha, const float* A, const float* B, float beta, float* C,
                      fmm_stream_t stream_) {
    if (!p) return FMM_ERR_INVALID_ARG;
    cudaStream_t stream = (cudaStream_t)stream_;
    p->last_stream = stream;
    if (p->M == 0 || p->N == 0) return FMM_OK;
    if (!C) return FMM_ERR_INVALID_ARG;
    if (alpha == 0.0f || p->K == 0) {
        FMM_CUDA(launch_scale(C, p->ldc, p->M, p->N, beta, stream));
        return FMM_OK;
    }
    if (!A || !B) return FMM_ERR_INVALID_ARG;
    fmm_plan_s::EvSet es;
    if (p->profile) {
        if (!p->ev_free.empty()) {
            es = p->ev_free.back();
            p->ev_free.pop_back();
        } else {
            for (int i = 0; i < 4; ++i) FMM_CUDA(cudaEventCreate(&es.e[i]));
        }
        p->cur = &es;
        mark(p, 0, stream);
    }
    fmm_status_t st = p->host ? run_host(p, alpha, A, B, beta, C, stream) : execute(p, alpha, A, B, beta, C, stream);
    p->calls += 1;
    if (p->cur) {
        mark(p, 3, stream);
        p->cur = nullptr;
        p->ev_pending.push_back(es);
    }
    return st;
}

fmm_status_t fmm_plan_profile(fmm_plan_t p, int enable) {
    if (!p) return FMM_ERR_INVALID_ARG;
    fmm_status_t s = drain_profile(p);
    p->profile = enable ? 1 : 0;
    p->prof_ms[0] = p->prof_ms[1] = p->prof_ms[2] = 0.0;
    p->launches = 0;
    p->calls = 0;
    return s;
}

fmm_status_t fmm_plan_phase_bytes(fmm_plan_t p, double* pre_bytes, double* post_bytes) {
    if (!p) return FMM_ERR_INVALID_ARG;
    // host-resident plans stream quadrants through a child plan: not reported
    if (pre_bytes) *pre_bytes = p->host ? 0.0 : p->acct[0];
    if (post_bytes) *post_bytes = p->host ? 0.0 : p->acct[1];
    return FMM_OK;
}

fmm_status_t fmm_plan_profile_read(fmm_plan_t p, double* pre_ms, double* leaf_ms, double* post_ms,
                                   int64_t* launches, int64_t* calls) {
    if (!p) return FMM_ERR_INVALID_ARG;
    fmm_status_t s = drain_profile(p);
    if (pre_ms) *pre_ms = p->prof_ms[0];
    if (leaf_ms) *leaf_ms = p->prof_ms[1];
    if (post_ms) *post_ms = p->prof_ms[2];
    if (launches) *launches = p->launches;
    if (calls) *calls = p->calls;
    return s;
}

fmm_status_t fmm_gemm_batched(int count, const int64_t* M, const int64_t* N, const int64_t* K, const float* const* A,
                              const int64_t* lda, const float* const* B, const int64_t* ldb, float* const* C,
                              const int64_t* ldc, const float* alpha, const float* beta, const fmm_options_t* opt,
                              void* workspace, size_t workspace_bytes, size_t* workspace_needed, fmm_stream_t stream) {
    if (!workspace) return fmm_batched_plan(nullptr, count, M, N, K, A, lda, B, ldb, C, ldc, alpha, beta, opt, nullptr,
                                            0, workspace_needed, stream);
    fmm_batched_t b = nullptr;
    fmm_status_t s = fmm_batched_plan(&b, count, M, N, K, A, lda, B, ldb, C, ldc, alpha, beta, opt, workspace,
                                      workspace_bytes, workspace_needed, stream);
    if (s != FMM_OK) return s;
    s = fmm_batched_run(b, stream);
    fmm_batched_free(b);  // device tables live in the caller's workspace; host state is not needed after launch
    return s;
}

void fmm_free(fmm_plan_t p) {
    if (!p) return;
    drain_profile(p);
    if (p->s_h2d) cudaStreamSynchronize(p->s_h2d);
    if (p->s_d2h) cudaStreamSynchronize(p->s_d2h);
    if (p->s_h2d) cudaStreamDestroy(p->s_h2d);
    if (p->s_d2h) cudaStreamDestroy(p->s_d2h);
    for (auto& e : p->hev)
        if (e) cudaEventDestroy(e);
    for (auto& pair : p->hx)
        for (auto& e : pair)
            if (e) cudaEventDestroy(e);
    delete p->child;
    for (auto& es : p->ev_free)
        for (int i = 0; i < 4; ++i) cudaEventDestroy(es.e[i]);
    delete p;
}

fmm_status_t fmm_get_device_status(fmm_plan_t p) {
    if (!p) return FMM_ERR_INVALID_ARG;
    FMM_CUDA(cudaStreamSynchronize(p->last_stream));
    unsigned w = 0;
    FMM_CUDA(cudaMemcpy(&w, p->status, sizeof(w), cudaMemcpyDeviceToHost));
    if (w) FMM_CUDA(cudaMemset(p->status, 0, sizeof(unsigned)));
    if (w & FMM_DEV_TIMEOUT_BIT) return FMM_ERR_TIMEOUT;
    return w ? FMM_ERR_CUDA : FMM_OK;
}

fmm_status_t fmm_wait_selftest(fmm_plan_t p, int64_t limit_ns, fmm_stream_t stream_) {
    if (!p || limit_ns < 1000000 || limit_ns > 10000000000LL) return FMM_ERR_INVALID_ARG;
    cudaStream_t stream = (cudaStream_t)stream_;
    p->last_stream = stream;
    FMM_CUDA(launch_wait_selftest(p->status, (unsigned long long)limit_ns, stream));
    return FMM_OK;
}

fmm_status_t fmm_plan_host_copy(fmm_plan_t p, int* mode) {
    if (!p || !mode) return FMM_ERR_INVALID_ARG;
    if (!p->host) *mode = 0;
    else if (p->opt.host_copy) *mode = p->opt.host_copy;
    else *mode = p->host_sm_latched ? 2 : 1;
    return FMM_OK;
}

fmm_status_t fmm_plan_fuse_last(fmm_plan_t p, int* fused) {
    if (!p || !fused) return FMM_ERR_INVALID_ARG;
    *fused = p->fused || (p->child && p->child->fused) ? 1 : 0;
    return FMM_OK;
}

fmm_status_t fmm_plan_info(fmm_plan_t p, int* depth, int* leaf_tile, int* precision, int* odd, int* algo) {
    if (!p) return FMM_ERR_INVALID_ARG;
    if (depth) *depth = p->rmul ? p->rmul : p->depth;
    if (leaf_tile) *leaf_tile = (p->pair || (p->host && p->tile_req == 512)) ? 512 : p->bn;
    if (precision) *precision = (int)p->opt.precision;
    if (odd) *odd = (int)p->odd;
    if (algo) *algo = (int)p->opt.algo;
    return FMM_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------
// Allocation-free entry point.  Its temporaries (child operands of one Winograd
// level and the seven products) live in a fixed device array compiled into the
// library, so the call needs no workspace from the caller and makes no device
// or host allocation.  The array is shared by every call on a device: calls
// that overlap on the GPU race on it.
namespace {
constexpr long long kStaticMaxDim = 1024;
// status block + 7 child operands per side + 7 products, each (1024/2)^2 floats
constexpr size_t kStaticBytes = 256 + 3 * (size_t)7 * (kStaticMaxDim / 2) * (kStaticMaxDim / 2) * sizeof(float);
__device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];
// device address of the array, per device; filled on a device's first call and
// read under g_mu, so host threads making first calls at once do not race
void* g_static_scratch_addr[64] = {};

// The array's device address on the current device (looked up once per device,
// with that device current: the host-side name of the array is not a device
// address).
fmm_status_t static_scratch(void** out) {
    int dev = 0;
    FMM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return FMM_ERR_NO_DEVICE;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_static_scratch_addr[dev]) {
        void* ptr = nullptr;
        FMM_CUDA(cudaGetSymbolAddress(&ptr, g_static_scratch));
        g_static_scratch_addr[dev] = ptr;
    }
    *out = g_static_scratch_addr[dev];
    return FMM_OK;
}
}  // namespace

extern "C" fmm_status_t fmm_gemm_static(int64_t M, int64_t N, int64_t K, float alpha, const float* A, int64_t lda,
                                        const float* B, int64_t ldb, float beta, float* C, int64_t ldc,
                                        fmm_stream_t stream_) {
    cudaStream_t stream = (cudaStream_t)stream_;
    if (M < 0 || N < 0 || K < 0) return FMM_ERR_INVALID_ARG;
    if (M > kStaticMaxDim || N > kStaticMaxDim || K > kStaticMaxDim) {
        snprintf(g_last_error, sizeof(g_last_error),
                 "fmm_gemm_static: M, N, K must each be <= %lld (static scratch of %zu bytes)", kStaticMaxDim,
                 kStaticBytes);
        return FMM_ERR_INVALID_ARG;
    }
    if (lda < (K > 0 ? K : 1) || ldb < (N > 0 ? N : 1) || ldc < (N > 0 ? N : 1)) return FMM_ERR_INVALID_ARG;
    if (M == 0 || N == 0) return FMM_OK;
    if (!C) return FMM_ERR_INVALID_ARG;
    DeviceInfo di;
    fmm_status_t s = device_info(&di);
    if (s != FMM_OK) return s;
    void* scratch = nullptr;
    if ((s = static_scratch(&scratch)) != FMM_OK) return s;
    if (alpha == 0.0f || K == 0) {
        // no kernel of this call can report into the status word: clear it so
        // that fmm_gemm_static_status describes this call
        FMM_CUDA(cudaMemsetAsync(scratch, 0, 64 * sizeof(unsigned), stream));
        FMM_CUDA(launch_scale(C, ldc, M, N, beta, stream));
        return FMM_OK;
    }
    if (!A || !B) return FMM_ERR_INVALID_ARG;
    fmm_options_t o;
    fmm_options_default(&o);
    o.depth = 1;
    fmm_plan_s p;
    make_tmp(p, M, N, K, lda, ldb, ldc, o, 1, 256);
    // leaves split their fp32 tiles in shared memory: the temporaries are then
    // the 7 child operands per side and the 7 products, which the array holds
    p.pre16 = 0;
    p.mode = kLeaf3xTF32;
    p.sched = 0;   // static tile order: no scheduling area in the fixed scratch
    size_t need = 0;
    layout(&p, nullptr, &need);
    if (need > kStaticBytes) return FMM_ERR_WORKSPACE;
    p.ws = static_cast<char*>(scratch);
    p.ws_bytes = kStaticBytes;
    p.num_sms = di.num_sms;
    layout(&p, p.ws, nullptr);
    // the array keeps the previous call's contents: the status word must start at zero
    FMM_CUDA(cudaMemsetAsync(p.status, 0, 64 * sizeof(unsigned), stream));
    return execute(&p, alpha, A, B, beta, C, stream);
}

extern "C" fmm_status_t fmm_gemm_static_status(fmm_stream_t stream) {
    DeviceInfo di;
    fmm_status_t s = device_info(&di);
    if (s != FMM_OK) return s;
    void* scratch = nullptr;
    if ((s = static_scratch(&scratch)) != FMM_OK) return s;
    FMM_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    unsigned w = 0;
    // the status word is the first word of the array (the layout's first carve-out)
    FMM_CUDA(cudaMemcpy(&w, scratch, sizeof(w), cudaMemcpyDeviceToHost));
    if (w) FMM_CUDA(cudaMemset(scratch, 0, sizeof(unsigned)));
    if (w & FMM_DEV_TIMEOUT_BIT) return FMM_ERR_TIMEOUT;
    return w ? FMM_ERR_CUDA : FMM_OK;
}
