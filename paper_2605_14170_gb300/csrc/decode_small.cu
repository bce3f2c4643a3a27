// Single-code launch of the register-resident BP path for small codes (the
// [[72,12,6]] and [[144,12,12]] bivariate bicycle codes of Section IV); the
// per-chunk device code is in bp_small.cuh.  Warps pull
// (chunk of kChunk shots, representation) work items from a global counter.
#include "bp_small.cuh"

namespace mbbp {
namespace {

constexpr int kSmallWarps = 1;  // warps per block: each warp works alone
constexpr int kChunk = 8;       // shots per work item of a warp (same representation)

template <int VS, int RS, int ORS, int RULE, bool REG, bool OUT>
__global__ void __launch_bounds__(kSmallWarps * 32, small_min_blocks(RS, RULE))
decode_small_kernel(const DecodeArgs a) {
    extern __shared__ __align__(16) float smsg[];
    const DevBases& B = a.B;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int R = B.R;
    char* smc = reinterpret_cast<char*>(smsg);
    const uint32_t wbase = (uint32_t)(warp * small_bp::warp_floats(B.MP, VS, ORS) * 4);
    const unsigned long long chunks_per_rep = ((unsigned long long)a.io.batch + kChunk - 1) / kChunk;
    const unsigned long long total_chunks = chunks_per_rep * (unsigned long long)R;
    for (;;) {
        unsigned long long chunk = 0;
        if (lane == 0) chunk = atomicAdd(a.counter, 1ull);
        chunk = __shfl_sync(small_bp::kFull, chunk, 0);
        if (chunk >= total_chunks) break;
        const int sblock = (int)(chunk / (unsigned long long)R);
        const int b = (int)(chunk - (unsigned long long)sblock * R);
        const int s0 = sblock * kChunk;
        const int s1 = min(a.io.batch, s0 + kChunk);
        small_bp::run_chunk<VS, RS, ORS, RULE, REG, OUT>(B, a.io, b, s0, s1, smc, wbase);
    }
}

template <int VS, int RS, int ORS, int RULE, bool REG>
cudaError_t launch_small_t(const DecodeArgs& a, cudaStream_t s, int sm_count) {
    // calls that ask for posteriors or the message trace take the kernel
    // that writes them; the plain decode has no test for them in its loops
    auto kern = (a.io.c2v || a.io.post) ? decode_small_kernel<VS, RS, ORS, RULE, REG, true>
                                        : decode_small_kernel<VS, RS, ORS, RULE, REG, false>;
    const int warps = kSmallWarps;
    const size_t smem = (size_t)warps * small_bp::warp_floats(a.B.MP, VS, ORS) * sizeof(float);
    int per_sm = 0;
    cudaError_t e = prepare_kernel(reinterpret_cast<const void*>(kern), warps * 32, smem, &per_sm);
    if (e != cudaSuccess) return e;
    const unsigned long long chunks =
        ((unsigned long long)a.io.batch + kChunk - 1) / kChunk * (unsigned long long)a.B.R;
    unsigned long long want = (chunks + warps - 1) / warps;
    unsigned long long grid = (unsigned long long)per_sm * (unsigned long long)sm_count;
    if (want < grid) grid = want;
    kern<<<(unsigned)grid, warps * 32, smem, s>>>(a);
    return cudaGetLastError();
}

template <int VS, int RS, int ORS>
cudaError_t launch_shape(const DecodeArgs& a, cudaStream_t s, int sm_count) {
    const bool reg = a.B.regular != 0;
    if (a.rule == MBBP_RULE_NMS)
        return reg ? launch_small_t<VS, RS, ORS, MBBP_RULE_NMS, true>(a, s, sm_count)
                   : launch_small_t<VS, RS, ORS, MBBP_RULE_NMS, false>(a, s, sm_count);
    return reg ? launch_small_t<VS, RS, ORS, MBBP_RULE_SP, true>(a, s, sm_count)
               : launch_small_t<VS, RS, ORS, MBBP_RULE_SP, false>(a, s, sm_count);
}

}  // namespace

cudaError_t launch_decode_small(const DecodeArgs& a, cudaStream_t s, int sm_count) {
    if (a.B.shape == 1) return launch_shape<3, 2, 2>(a, s, sm_count);
    if (a.B.shape == 2) return launch_shape<5, 3, 3>(a, s, sm_count);
    if (a.B.shape == 3) return launch_shape<5, 4, 3>(a, s, sm_count);
    return cudaErrorInvalidValue;
}

}  // namespace mbbp
