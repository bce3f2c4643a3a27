// MBBP-LD decode kernels for sm_103a: the generic single-code BP kernel (any
// code within the library's limits; per-item device code in bp_generic.cuh),
// Frequency-Weighted Scoring of each shot's converged candidates (Section
// III-B), the fixed scratch behind mbbp_decode_noalloc, and the cached launch
// preparation shared by every kernel.
#include <map>
#include <mutex>
#include <tuple>

#include "bp_generic.cuh"

// Fixed scratch for mbbp_decode_noalloc: the workspace (candidates + work
// counter) of callers that cannot allocate device memory.  Every GPU that
// loads this library holds it until the process exits.
static __device__ __align__(256) unsigned char g_static_scratch[mbbp::kStaticScratchBytes];

namespace mbbp {
namespace {

constexpr unsigned kFull = 0xffffffffu;

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Block-size classes of the generic kernel: up to 8 warps (the usual case)
// and up to 16 warps for big codes, where a block holds H's columns once plus
// one message area per warp and one large block fits more warps per SM than
// several small ones.  Each class is compiled for its own block size.
constexpr int kGenericWideWarps = 16;

// G warps decode each item together (G = 1: one warp per item; G = 2 or 4
// for codes whose per-item shared memory, not registers, limits the resident
// warps: the same shared memory then holds G times the warps).  Group g of
// the block uses named barrier 1 + g (at most 8 groups: ids 1..8).
template <int DC, int DV, int RULE, int MAXW, bool TRACE = false, int G = 1>
__global__ void __launch_bounds__(MAXW * 32)
decode_kernel(const DecodeArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long group_item[MAXW];
    const DevBases& B = a.B;
    const int lane = threadIdx.x & 31;
    const int grp = (int)(threadIdx.x >> 5) / G;
    const int gt = (int)(threadIdx.x % (32 * G));
    const int bar = 1 + grp;
    const generic_bp::WarpLayout L = generic_bp::warp_layout(DC, B.MP, B.mpad, B.n);
    uint16_t* hcol_s = reinterpret_cast<uint16_t*>(smem);
    unsigned char* area = smem + L.hcol_bytes + grp * L.per_warp;
    for (int i = threadIdx.x; i < DC * B.mpad; i += blockDim.x) hcol_s[i] = __ldg(B.hcol + i);
    __syncthreads();
    // Work items are taken representation-major (item = b * batch + shot):
    // the warps resident at one time mostly decode the same representation,
    // so its descriptor tables stay in L1 instead of one table per warp.
    const unsigned long long batch = (unsigned long long)a.io.batch;
    for (;;) {
        unsigned long long item = 0;
        if constexpr (G == 1) {
            if (lane == 0) item = atomicAdd(a.counter, 1ull);
            item = __shfl_sync(kFull, item, 0);
        } else {
            // the group's first thread takes the item; the slot is rewritten
            // only after the item's last barrier, which every reader passed
            if (gt == 0) group_item[grp] = atomicAdd(a.counter, 1ull);
            generic_bp::gsync<G>(bar);
            item = group_item[grp];
        }
        if (item >= a.total_items) break;
        const int b = (int)(item / batch);
        const int shot = (int)(item - (unsigned long long)b * batch);
        generic_bp::run_item<DC, DV, RULE, TRACE, G>(B, a.io, shot, b, area, hcol_s, bar);
    }
}

// The serial-schedule kernel: same work list as decode_kernel, one warp per
// (shot, representation) item, run_item_serial per item.
template <int DC, int DV, int RULE>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
decode_serial_kernel(const DecodeArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const DevBases& B = a.B;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int R = B.R;
    const generic_bp::WarpLayout L = generic_bp::warp_layout(DC, B.MP, B.mpad, B.n);
    const int per_warp = generic_bp::serial_warp_bytes(DC, B.MP, B.mpad, B.n);
    uint16_t* hcol_s = reinterpret_cast<uint16_t*>(smem);
    unsigned char* area = smem + L.hcol_bytes + warp * per_warp;
    for (int i = threadIdx.x; i < DC * B.mpad; i += blockDim.x) hcol_s[i] = __ldg(B.hcol + i);
    __syncthreads();
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(a.counter, 1ull);
        item = __shfl_sync(kFull, item, 0);
        if (item >= a.total_items) break;
        const int shot = (int)(item / (unsigned long long)R);
        const int b = (int)(item - (unsigned long long)shot * R);
        generic_bp::run_item_serial<DC, DV, RULE>(B, a.io, shot, b, area, hcol_s);
    }
}

struct FwsBest {
    long long cnt, w;
    int idx, valid;
};

__device__ __forceinline__ bool fws_better(const FwsBest& x, const FwsBest& y) {
    if (!x.valid) return false;
    if (!y.valid) return true;
    const long long lhs = x.cnt * (y.w + 1), rhs = y.cnt * (x.w + 1);
    if (lhs != rhs) return lhs > rhs;
    return x.idx < y.idx;
}

// One warp per shot: FWS over the R candidates (R <= 64).
__global__ void __launch_bounds__(kWarpsPerBlock * 32) fws_kernel(const FwsArgs a) {
    extern __shared__ __align__(16) uint32_t fsm[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int shot = blockIdx.x * (blockDim.x >> 5) + warp;
    if (shot >= a.batch) return;  // uniform per warp
    const int R = a.R, W = a.W, n = a.n;
    uint32_t* cw = fsm + (size_t)warp * R * W;
    const uint32_t* src = a.cand + (size_t)shot * R * W;
    for (int i = lane; i < R * W; i += 32) cw[i] = __ldg(src + i);
    const uint8_t* cv = a.conv + (size_t)shot * R;
    const uint32_t c_lo = __ballot_sync(kFull, lane < R && __ldg(cv + lane));
    const uint32_t c_hi = __ballot_sync(kFull, lane + 32 < R && __ldg(cv + lane + 32));
    __syncwarp();
    FwsBest best{0, 0, 0, 0};
    for (int h = 0; h < 2; ++h) {
        const int ai = lane + 32 * h;
        FwsBest c{0, 0, ai, 0};
        if (ai < R && (((h ? c_hi : c_lo) >> lane) & 1u)) {
            c.valid = 1;
            const uint32_t* ca = cw + (size_t)ai * W;
            for (int k = 0; k < W; ++k) c.w += __popc(ca[k]);
            for (int bi = 0; bi < R; ++bi) {
                const uint32_t cb = (bi < 32) ? (c_lo >> bi) & 1u : (c_hi >> (bi - 32)) & 1u;
                if (!cb) continue;
                const uint32_t* pb = cw + (size_t)bi * W;
                bool eq = true;
                for (int k = 0; k < W && eq; ++k) eq = (ca[k] == pb[k]);
                c.cnt += eq ? 1 : 0;
            }
        }
        if (fws_better(c, best)) best = c;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        FwsBest o;
        o.cnt = __shfl_xor_sync(kFull, best.cnt, off);
        o.w = __shfl_xor_sync(kFull, best.w, off);
        o.idx = __shfl_xor_sync(kFull, best.idx, off);
        o.valid = __shfl_xor_sync(kFull, best.valid, off);
        if (fws_better(o, best)) best = o;
    }
    const int sel = best.valid ? best.idx : -1;
    uint8_t* out = a.e_hat + (size_t)shot * n;
    for (int v = lane; v < n; v += 32)
        out[v] = (sel >= 0) ? (uint8_t)((cw[(size_t)sel * W + (v >> 5)] >> (v & 31)) & 1u) : 0;
    if (lane == 0) {
        a.success[shot] = sel >= 0 ? 1 : 0;
        if (a.selected) a.selected[shot] = (int16_t)sel;
    }
}

// One warp per shot: the least-metric selector over the R candidates
// (R <= 64).  The metric of candidate a is the float sum, in ascending
// variable order, of the shot's LLRs over the set bits of a; the smallest
// metric wins, ties to the lowest index.
__global__ void __launch_bounds__(kWarpsPerBlock * 32) lms_kernel(const FwsArgs a) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int shot = blockIdx.x * (blockDim.x >> 5) + warp;
    if (shot >= a.batch) return;  // uniform per warp
    const int R = a.R, W = a.W, n = a.n;
    const uint32_t* src = a.cand + (size_t)shot * R * W;
    const uint8_t* cv = a.conv + (size_t)shot * R;
    const float* mu = a.llr + (size_t)shot * a.llr_stride;
    float best_m = 0.0f;
    int best = -1;  // lowest index among this lane's minima
    for (int h = 0; h < 2; ++h) {
        const int ai = lane + 32 * h;
        if (ai < R && __ldg(cv + ai)) {
            const uint32_t* ca = src + (size_t)ai * W;
            float mt = 0.0f;
            for (int k = 0; k < W; ++k) {
                uint32_t word = __ldg(ca + k);
                while (word) {
                    const int bit = __ffs(word) - 1;
                    mt = __fadd_rn(mt, __ldg(mu + 32 * k + bit));
                    word &= word - 1u;
                }
            }
            if (best < 0 || mt < best_m) {
                best = ai;
                best_m = mt;
            }
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float om = __shfl_xor_sync(kFull, best_m, off);
        const int ob = __shfl_xor_sync(kFull, best, off);
        if (ob >= 0 && (best < 0 || om < best_m || (om == best_m && ob < best))) {
            best = ob;
            best_m = om;
        }
    }
    uint8_t* out = a.e_hat + (size_t)shot * n;
    for (int v = lane; v < n; v += 32)
        out[v] = (best >= 0) ? (uint8_t)((__ldg(src + (size_t)best * W + (v >> 5)) >> (v & 31)) & 1u) : 0;
    if (lane == 0) {
        a.success[shot] = best >= 0 ? 1 : 0;
        if (a.selected) a.selected[shot] = (int16_t)best;
    }
}

template <int K, int RULE>
cudaError_t launch_serial_t(const DecodeArgs& a, cudaStream_t s, int sm_count) {
    auto kern = decode_serial_kernel<K, K, RULE>;
    const generic_bp::WarpLayout L = generic_bp::warp_layout(K, a.B.MP, a.B.mpad, a.B.n);
    const int per_warp = generic_bp::serial_warp_bytes(K, a.B.MP, a.B.mpad, a.B.n);
    int warps = kWarpsPerBlock;
    while (warps > 1 && (size_t)L.hcol_bytes + (size_t)warps * per_warp > 200 * 1024) --warps;
    const size_t smem = (size_t)L.hcol_bytes + (size_t)warps * per_warp;
    int per_sm = 0;
    cudaError_t e = prepare_kernel(reinterpret_cast<const void*>(kern), warps * 32, smem, &per_sm);
    if (e != cudaSuccess) return e;
    unsigned long long want = (a.total_items + warps - 1) / warps;
    unsigned long long grid = (unsigned long long)per_sm * (unsigned long long)sm_count;
    if (want < grid) grid = want;
    kern<<<(unsigned)grid, warps * 32, smem, s>>>(a);
    return cudaGetLastError();
}

template <int K, int RULE, bool TRACE, int G>
cudaError_t launch_decode_g(const DecodeArgs& a, int cls, int warps, int per_sm, size_t smem, cudaStream_t s,
                            int sm_count) {
    const unsigned long long groups = (unsigned long long)(warps / G);
    unsigned long long want = (a.total_items + groups - 1) / groups;
    unsigned long long grid = (unsigned long long)per_sm * (unsigned long long)sm_count;
    if (want < grid) grid = want;
    const dim3 gd((unsigned)grid), bd((unsigned)(warps * 32));
    if (cls == 0)
        decode_kernel<K, K, RULE, kWarpsPerBlock, TRACE, G><<<gd, bd, smem, s>>>(a);
    else
        decode_kernel<K, K, RULE, kGenericWideWarps, TRACE, G><<<gd, bd, smem, s>>>(a);
    return cudaGetLastError();
}

template <int K, int RULE, bool TRACE>
cudaError_t launch_decode_t(const DecodeArgs& a, cudaStream_t s, int sm_count) {
    // Launch shapes: (block class, warps per item G in {1, 2, 4}).  The narrow
    // class runs blocks of up to 8 warps, the wide class up to 16 (compiled
    // for 512-thread blocks, it takes more registers).  For each shape, the
    // block size with the most resident warps per SM (ties: the smaller
    // block) within 200 KB of shared memory per block; a block holds H's
    // columns once plus one message area per item.  Among G = 1 shapes the
    // wide class only when it holds at least a quarter more warps; a larger G
    // only when it holds at least half again as many warps as the best
    // smaller one (codes whose message areas, not registers, limit the
    // resident warps).
    const void* kerns[3][2] = {
        {reinterpret_cast<const void*>(decode_kernel<K, K, RULE, kWarpsPerBlock, TRACE, 1>),
         reinterpret_cast<const void*>(decode_kernel<K, K, RULE, kGenericWideWarps, TRACE, 1>)},
        {reinterpret_cast<const void*>(decode_kernel<K, K, RULE, kWarpsPerBlock, TRACE, 2>),
         reinterpret_cast<const void*>(decode_kernel<K, K, RULE, kGenericWideWarps, TRACE, 2>)},
        {reinterpret_cast<const void*>(decode_kernel<K, K, RULE, kWarpsPerBlock, TRACE, 4>),
         reinterpret_cast<const void*>(decode_kernel<K, K, RULE, kGenericWideWarps, TRACE, 4>)}};
    const generic_bp::WarpLayout L = generic_bp::warp_layout(K, a.B.MP, a.B.mpad, a.B.n);
    int choice[3][2][2] = {};  // [log2 G][class] = {warps per block, blocks per SM}
    for (int gi = 0; gi < 3; ++gi) {
        const int G = 1 << gi;
        for (int w = G; w <= kGenericWideWarps; w += G) {
            const size_t sm_w = (size_t)L.hcol_bytes + (size_t)(w / G) * L.per_warp;
            if (sm_w > 200 * 1024) break;
            const int cls = w <= kWarpsPerBlock ? 0 : 1;
            int b = 0;
            cudaError_t e = prepare_kernel(kerns[gi][cls], w * 32, sm_w, &b);
            if (e != cudaSuccess) return e;
            if (b * w > choice[gi][cls][0] * choice[gi][cls][1]) {
                choice[gi][cls][0] = w;
                choice[gi][cls][1] = b;
            }
        }
    }
    auto resident = [&](int gi, int cls) { return choice[gi][cls][0] * choice[gi][cls][1]; };
    int gi_best = 0, cls_best = resident(0, 1) * 4 >= resident(0, 0) * 5 ? 1 : 0;
    for (int gi = 1; gi < 3; ++gi) {
        const int cls = resident(gi, 1) > resident(gi, 0) ? 1 : 0;
        if (2 * resident(gi, cls) >= 3 * resident(gi_best, cls_best)) {
            gi_best = gi;
            cls_best = cls;
        }
    }
    const int warps = choice[gi_best][cls_best][0], per_sm = choice[gi_best][cls_best][1];
    if (warps == 0) return cudaErrorInvalidConfiguration;
    const size_t smem = (size_t)L.hcol_bytes + (size_t)(warps >> gi_best) * L.per_warp;
    if (gi_best == 0) return launch_decode_g<K, RULE, TRACE, 1>(a, cls_best, warps, per_sm, smem, s, sm_count);
    if (gi_best == 1) return launch_decode_g<K, RULE, TRACE, 2>(a, cls_best, warps, per_sm, smem, s, sm_count);
    return launch_decode_g<K, RULE, TRACE, 4>(a, cls_best, warps, per_sm, smem, s, sm_count);
}

template <int K, int RULE>
cudaError_t launch_decode_k(const DecodeArgs& a, cudaStream_t s, int sm_count) {
    return a.io.c2v ? launch_decode_t<K, RULE, true>(a, s, sm_count) : launch_decode_t<K, RULE, false>(a, s, sm_count);
}

}  // namespace

cudaError_t static_scratch(void** ptr) {
    // The array's name is a host-side stand-in in host code; the device
    // address comes from cudaGetSymbolAddress, looked up once per device with
    // that device current.
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *ptr = g_scratch_addr[dev];
    return cudaSuccess;
}

cudaError_t prepare_kernel(const void* func, int threads, size_t smem, int* blocks_per_sm) {
    // The dynamic shared-memory limit of a kernel only ever grows (a launch
    // with less shared memory than the limit is valid), and the occupancy of
    // every (kernel, block size, shared memory, device) is queried once; later
    // launches only read these caches, so a launch enqueues nothing but the
    // kernel (stream-capture friendly).
    static std::mutex mu;
    static std::map<std::tuple<const void*, int, size_t, int>, int> occupancy;
    static std::map<std::pair<const void*, int>, size_t> smem_limit;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    size_t& limit = smem_limit[std::make_pair(func, dev)];
    if (smem > limit) {
        e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        limit = smem;
    }
    const auto key = std::make_tuple(func, threads, smem, dev);
    auto it = occupancy.find(key);
    if (it != occupancy.end()) {
        *blocks_per_sm = it->second;
        return cudaSuccess;
    }
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, func, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    occupancy[key] = per_sm;
    *blocks_per_sm = per_sm;
    return cudaSuccess;
}

cudaError_t launch_decode(const DecodeArgs& a, cudaStream_t s, int sm_count) {
    if (a.B.shape != 0) return launch_decode_small(a, s, sm_count);
    const int K = a.B.DC;
    if (a.rule == MBBP_RULE_NMS) {
        if (K == 6) return launch_decode_k<6, MBBP_RULE_NMS>(a, s, sm_count);
        if (K == 8) return launch_decode_k<8, MBBP_RULE_NMS>(a, s, sm_count);
        if (K == 12) return launch_decode_k<12, MBBP_RULE_NMS>(a, s, sm_count);
    } else {
        if (K == 6) return launch_decode_k<6, MBBP_RULE_SP>(a, s, sm_count);
        if (K == 8) return launch_decode_k<8, MBBP_RULE_SP>(a, s, sm_count);
        if (K == 12) return launch_decode_k<12, MBBP_RULE_SP>(a, s, sm_count);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_decode_serial_generic(const DecodeArgs& a, cudaStream_t s, int sm_count) {
    const int K = a.B.DC;
    if (a.rule == MBBP_RULE_NMS) {
        if (K == 6) return launch_serial_t<6, MBBP_RULE_NMS>(a, s, sm_count);
        if (K == 8) return launch_serial_t<8, MBBP_RULE_NMS>(a, s, sm_count);
        if (K == 12) return launch_serial_t<12, MBBP_RULE_NMS>(a, s, sm_count);
    } else {
        if (K == 6) return launch_serial_t<6, MBBP_RULE_SP>(a, s, sm_count);
        if (K == 8) return launch_serial_t<8, MBBP_RULE_SP>(a, s, sm_count);
        if (K == 12) return launch_serial_t<12, MBBP_RULE_SP>(a, s, sm_count);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_fws(const FwsArgs& a, cudaStream_t s) {
    if (a.decision == MBBP_DECISION_LMS) {
        if (!a.llr) return cudaErrorInvalidValue;
        const int warps = kWarpsPerBlock;
        const unsigned grid = (unsigned)((a.batch + warps - 1) / warps);
        lms_kernel<<<grid, warps * 32, 0, s>>>(a);
        return cudaGetLastError();
    }
    const size_t per_warp = (size_t)a.R * a.W * 4;
    int warps = kWarpsPerBlock;
    while (warps > 1 && warps * per_warp > 96 * 1024) --warps;
    const size_t smem = warps * per_warp;
    int per_sm = 0;
    cudaError_t e = prepare_kernel(reinterpret_cast<const void*>(fws_kernel), warps * 32, smem, &per_sm);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)((a.batch + warps - 1) / warps);
    fws_kernel<<<grid, warps * 32, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace mbbp
