// Persistent mixed-batch BP kernels: one launch decodes the shots of several
// codes (each with its own R representations and sizes) that the plan
// assigned to one kernel body — the generic path (bp_generic.cuh), or the
// small-code path (bp_small.cuh) for one of its shapes; a plan issues one
// launch per body and shape present, on the stream.  Each launch gets its own
// register budget: the small path at 96 registers in one-warp blocks (the
// single-code kernel's budget) and the generic path at about 64; one kernel
// holding every small shape needed 128 registers, and one holding both paths
// would hold the generic items to the small path's occupancy.  Warps pull
// work items (code, chunk of shots, representation) from the launch's
// counter, in the order the plan chose (heaviest codes first by default).
// Every per-code argument travels in the kernel parameters, so a captured
// CUDA graph holds them by value.  Within a code, items are taken
// representation-major.
#include "bp_generic.cuh"
#include "bp_small.cuh"

namespace mbbp {
namespace {

// The next work item of this warp: code c, representation b, shots
// [s0, s1).  Warp-uniform; false once the launch's items are exhausted.
struct MixedItem {
    int c, b, s0, s1;
};

__device__ __forceinline__ bool next_item(const MixedArgs& a, MixedItem& it) {
    unsigned long long g = 0;
    if ((threadIdx.x & 31) == 0) g = atomicAdd(a.counter, 1ull);
    g = __shfl_sync(0xffffffffu, g, 0);
    if (g >= a.total) return false;
    int c = 0;
    while (c + 1 < a.n_codes && g >= a.codes[c + 1].first) ++c;
    const MixedCode& mc = a.codes[c];
    const unsigned long long l = g - mc.first;
    // representation-major within a code: the warps resident at one time
    // mostly work on one representation, whose tables then stay in L1
    const unsigned long long nchunks = ((unsigned long long)mc.io.batch + mc.chunk - 1) / mc.chunk;
    const int b = (int)(l / nchunks);
    const int sblock = (int)(l - (unsigned long long)b * nchunks);
    it.c = c;
    it.b = b;
    it.s0 = sblock * mc.chunk;
    it.s1 = min(mc.io.batch, it.s0 + mc.chunk);
    return true;
}

// Small-code path of one shape, regular rows only (the plan sends irregular
// codes to the generic path).
template <int RULE, int VS, int RS, int ORS>
__global__ void __launch_bounds__(32, small_min_blocks(RS, RULE)) mixed_small_kernel(const MixedArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    char* smc = reinterpret_cast<char*>(smem);
    const uint32_t wbase = (uint32_t)(threadIdx.x >> 5) * a.warp_bytes;
    MixedItem it;
    while (next_item(a, it)) {
        const MixedCode& mc = a.codes[it.c];
        small_bp::run_chunk<VS, RS, ORS, RULE, true>(mc.B, mc.io, it.b, it.s0, it.s1, smc, wbase);
    }
}

template <int RULE>
__global__ void __launch_bounds__(kMixedMaxWarps * 32) mixed_generic_kernel(const MixedArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t wbase = (uint32_t)(threadIdx.x >> 5) * a.warp_bytes;
    MixedItem it;
    while (next_item(a, it)) {
        const MixedCode& mc = a.codes[it.c];
        for (int s = it.s0; s < it.s1; ++s)
            generic_bp::run_item_any<RULE>(mc.B, mc.io, s, it.b, smem + wbase, mc.B.hcol);
    }
}

// One persistent launch: as many blocks as fit on the GPU, at most one warp
// per work item.
cudaError_t launch_persistent(void (*kern)(const MixedArgs), const MixedArgs& a, int warps, cudaStream_t s,
                              int sm_count) {
    const size_t smem = (size_t)warps * a.warp_bytes;
    int per_sm = 0;
    cudaError_t e = prepare_kernel(reinterpret_cast<const void*>(kern), warps * 32, smem, &per_sm);
    if (e != cudaSuccess) return e;
    unsigned long long want = (a.total + warps - 1) / warps;
    unsigned long long grid = (unsigned long long)per_sm * (unsigned long long)sm_count;
    if (want < grid) grid = want;
    if (grid == 0) return cudaSuccess;
    kern<<<(unsigned)grid, warps * 32, smem, s>>>(a);
    return cudaGetLastError();
}

template <int RULE>
cudaError_t launch_group(const MixedArgs& a, int group, int warps, cudaStream_t s, int sm_count) {
    constexpr SmallShape s1 = kSmallShapes[0], s2 = kSmallShapes[1], s3 = kSmallShapes[2];
    switch (group) {
        case 0: return launch_persistent(mixed_generic_kernel<RULE>, a, warps, s, sm_count);
        case 1: return launch_persistent(mixed_small_kernel<RULE, s1.VS, s1.RS, s1.ORS>, a, 1, s, sm_count);
        case 2: return launch_persistent(mixed_small_kernel<RULE, s2.VS, s2.RS, s2.ORS>, a, 1, s, sm_count);
        case 3: return launch_persistent(mixed_small_kernel<RULE, s3.VS, s3.RS, s3.ORS>, a, 1, s, sm_count);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

size_t mixed_warp_bytes(const DevBases& B, int kind) {
    if (kind == kKindSmall) {
        const SmallShape& sh = kSmallShapes[B.shape - 1];
        return (size_t)small_bp::warp_floats(B.MP, sh.VS, sh.ORS) * 4;
    }
    return (size_t)generic_bp::warp_layout(B.DC, B.MP, B.mpad, B.n).per_warp;
}

cudaError_t launch_mixed(const MixedArgs& a, int group, int warps, int rule, cudaStream_t s, int sm_count) {
    return rule == MBBP_RULE_NMS ? launch_group<MBBP_RULE_NMS>(a, group, warps, s, sm_count)
                                 : launch_group<MBBP_RULE_SP>(a, group, warps, s, sm_count);
}

}  // namespace mbbp
