// Persistent mixed-batch BP kernels: one launch decodes the shots of several
// codes (each with its own R representations and sizes) that the plan
// assigned to one kernel body — the small-code path (bp_small.cuh) or the
// generic path (bp_generic.cuh); a plan with both kinds issues one launch of
// each on the stream.  Each body gets its own register budget: the small
// path needs about 128 registers per thread, the generic path about 40, and
// sharing one kernel would hold the generic items to the small path's
// occupancy.  Warps pull work items (code, chunk of shots, representation)
// from the launch's counter, in the order the plan chose (heaviest codes
// first by default).  Every per-code argument travels in the kernel
// parameters, so a captured CUDA graph holds them by value.
#include "bp_generic.cuh"
#include "bp_small.cuh"

namespace mbbp {
namespace {

template <int RULE, int KIND>
__device__ __forceinline__ void mixed_body(const MixedArgs& a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const uint32_t wbase = (uint32_t)warp * a.warp_bytes;
    for (;;) {
        unsigned long long g = 0;
        if (lane == 0) g = atomicAdd(a.counter, 1ull);
        g = __shfl_sync(0xffffffffu, g, 0);
        if (g >= a.total) break;
        int c = 0;
        while (c + 1 < a.n_codes && g >= a.codes[c + 1].first) ++c;
        const MixedCode& mc = a.codes[c];
        const unsigned long long l = g - mc.first;
        const int R = mc.B.R;
        const int sblock = (int)(l / (unsigned long long)R);
        const int b = (int)(l - (unsigned long long)sblock * R);
        const int s0 = sblock * mc.chunk;
        const int s1 = min(mc.io.batch, s0 + mc.chunk);
        if (KIND == kKindSmall) {
            // small-code path, regular rows only (keeps the kernel within its
            // register budget; the plan sends irregular codes to the generic path)
            char* smc = reinterpret_cast<char*>(smem);
            switch (mc.B.shape) {
                case 1: small_bp::run_chunk<3, 2, 2, RULE, true>(mc.B, mc.io, b, s0, s1, smc, wbase); break;
                case 2: small_bp::run_chunk<5, 3, 3, RULE, true>(mc.B, mc.io, b, s0, s1, smc, wbase); break;
                default: small_bp::run_chunk<5, 4, 3, RULE, true>(mc.B, mc.io, b, s0, s1, smc, wbase); break;
            }
        } else {
            for (int s = s0; s < s1; ++s)
                generic_bp::run_item_any<RULE>(mc.B, mc.io, s, b, smem + wbase, mc.B.hcol);
        }
    }
}

template <int RULE>
__global__ void __launch_bounds__(kMixedMaxWarps * 32, 2) mixed_small_kernel(const MixedArgs a) {
    mixed_body<RULE, kKindSmall>(a);
}

template <int RULE>
__global__ void __launch_bounds__(kMixedMaxWarps * 32) mixed_generic_kernel(const MixedArgs a) {
    mixed_body<RULE, kKindGeneric>(a);
}

}  // namespace

size_t mixed_warp_bytes(const DevBases& B, int kind) {
    if (kind == kKindSmall) {
        const SmallShape& sh = kSmallShapes[B.shape - 1];
        return (size_t)small_bp::warp_floats(B.MP, sh.VS, sh.ORS) * 4;
    }
    return (size_t)generic_bp::warp_layout(B.DC, B.MP, B.mpad, B.n).per_warp;
}

cudaError_t launch_mixed(const MixedArgs& a, int kind, int warps, int rule, cudaStream_t s, int sm_count) {
    const bool nms = rule == MBBP_RULE_NMS;
    const void* kern =
        kind == kKindSmall
            ? (nms ? reinterpret_cast<const void*>(mixed_small_kernel<MBBP_RULE_NMS>)
                   : reinterpret_cast<const void*>(mixed_small_kernel<MBBP_RULE_SP>))
            : (nms ? reinterpret_cast<const void*>(mixed_generic_kernel<MBBP_RULE_NMS>)
                   : reinterpret_cast<const void*>(mixed_generic_kernel<MBBP_RULE_SP>));
    const size_t smem = (size_t)warps * a.warp_bytes;
    int per_sm = 0;
    cudaError_t e = prepare_kernel(kern, warps * 32, smem, &per_sm);
    if (e != cudaSuccess) return e;
    unsigned long long want = (a.total + warps - 1) / warps;
    unsigned long long grid = (unsigned long long)per_sm * (unsigned long long)sm_count;
    if (want < grid) grid = want;
    if (grid == 0) return cudaSuccess;
    if (kind == kKindSmall) {
        if (nms) mixed_small_kernel<MBBP_RULE_NMS><<<(unsigned)grid, warps * 32, smem, s>>>(a);
        else mixed_small_kernel<MBBP_RULE_SP><<<(unsigned)grid, warps * 32, smem, s>>>(a);
    } else {
        if (nms) mixed_generic_kernel<MBBP_RULE_NMS><<<(unsigned)grid, warps * 32, smem, s>>>(a);
        else mixed_generic_kernel<MBBP_RULE_SP><<<(unsigned)grid, warps * 32, smem, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace mbbp
