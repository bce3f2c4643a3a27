// Serial-schedule launches (Section II-B).  Kernel widths 6 and 8 use the
// slot path of bp_serial.cuh: a persistent grid whose warps pull shots of
// one representation at a time from per-representation counters and decode
// CS of them at once (CS = 4, 2 or 1, the largest that leaves about half of
// the SM's shared memory to L1 with two 8-warp blocks per SM).  Width 12 uses the
// one-item-per-warp generic serial kernel.
#include "bp_serial.cuh"

namespace mbbp {
namespace {

constexpr int kSerialWarps = serial_bp::kWarps;
// Blocks per SM the register budget is sized for (80 registers; measured
// against 2 blocks at 119 registers and 4 at 64: 2-4% and 10-12% slower).
constexpr int kSerialMinBlocks = 3;

template <int DC, int NO, int NV, int RULE, bool REG, int CS>
__global__ void __launch_bounds__(kSerialWarps * 32, kSerialMinBlocks)
decode_serial_chunk_kernel(const DecodeArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const DevBases& B = a.B;
    const int warp = threadIdx.x >> 5;
    const int R = B.R;
    const int hcol_bytes = generic_bp::align16(DC * B.mpad * 2);
    const serial_bp::Layout L = serial_bp::layout(DC, B.MP, B.n, CS);
    uint16_t* hcol_s = reinterpret_cast<uint16_t*>(smem);
    unsigned char* area = smem + hcol_bytes + warp * L.bytes;
    for (int i = threadIdx.x; i < DC * B.mpad; i += blockDim.x) hcol_s[i] = __ldg(B.hcol + i);
    __syncthreads();
    // the warps of a block work on the same representation (its edge
    // descriptors stay in L1); blocks start spread over the representations
    // and move on to the next one when the shots of theirs run out
    for (int k = 0; k < R; ++k) {
        const int b = (int)((blockIdx.x + k) % (unsigned)R);
        serial_bp::run_rep<DC, NO, NV, RULE, REG, CS>(B, a.io, b, a.rep_counter + b, area, hcol_s);
    }
}

template <int DC, int NO, int NV, int RULE, bool REG, int CS>
cudaError_t launch_t(const DecodeArgs& a, cudaStream_t s, int sm_count, int warps) {
    auto kern = decode_serial_chunk_kernel<DC, NO, NV, RULE, REG, CS>;
    const serial_bp::Layout L = serial_bp::layout(DC, a.B.MP, a.B.n, CS);
    const size_t smem = (size_t)generic_bp::align16(DC * a.B.mpad * 2) + (size_t)warps * L.bytes;
    int per_sm = 0;
    cudaError_t e = prepare_kernel(reinterpret_cast<const void*>(kern), warps * 32, smem, &per_sm);
    if (e != cudaSuccess) return e;
    const unsigned long long items = ((unsigned long long)a.io.batch + CS - 1) / CS * (unsigned long long)a.B.R;
    unsigned long long want = (items + warps - 1) / warps;
    unsigned long long grid = (unsigned long long)per_sm * (unsigned long long)sm_count;
    if (want < grid) grid = want;
    kern<<<(unsigned)grid, warps * 32, smem, s>>>(a);
    return cudaGetLastError();
}

template <int DC, int NO, int NV, int RULE, bool REG>
cudaError_t launch_cs(const DecodeArgs& a, cudaStream_t s, int sm_count) {
    // the largest CS whose 8-warp block fits twice in about half of the
    // SM's shared memory (the rest stays L1, which holds the edge
    // descriptors of the blocks' representations), else the largest warp
    // count at CS = 1 that fits once
    const size_t hb = (size_t)generic_bp::align16(DC * a.B.mpad * 2);
    const size_t budget1 = 200 * 1024;
    const int cs = serial_bp::shots_per_warp(DC, a.B.MP, a.B.mpad, a.B.n);
    if (cs == 4) return launch_t<DC, NO, NV, RULE, REG, 4>(a, s, sm_count, kSerialWarps);
    if (cs == 2) return launch_t<DC, NO, NV, RULE, REG, 2>(a, s, sm_count, kSerialWarps);
    if (hb + kSerialWarps * (size_t)serial_bp::layout(DC, a.B.MP, a.B.n, 1).bytes <= serial_bp::kBudget2)
        return launch_t<DC, NO, NV, RULE, REG, 1>(a, s, sm_count, kSerialWarps);
    int warps = kSerialWarps;
    const size_t per = (size_t)serial_bp::layout(DC, a.B.MP, a.B.n, 1).bytes;
    while (warps > 1 && hb + warps * per > budget1) --warps;
    return launch_t<DC, NO, NV, RULE, REG, 1>(a, s, sm_count, warps);
}

template <int RULE, bool REG>
cudaError_t launch_width(const DecodeArgs& a, cudaStream_t s, int sm_count) {
    if (a.B.DC == 6) {
        if (a.B.DV <= 4) return launch_cs<6, 3, 4, RULE, REG>(a, s, sm_count);
        return launch_cs<6, 5, 6, RULE, REG>(a, s, sm_count);
    }
    return launch_cs<8, 7, 8, RULE, REG>(a, s, sm_count);
}

}  // namespace

cudaError_t launch_decode_serial(const DecodeArgs& a, cudaStream_t s, int sm_count) {
    if (!a.B.edesc || (a.B.DC != 6 && a.B.DC != 8)) return launch_decode_serial_generic(a, s, sm_count);
    const bool reg = a.B.regular != 0;
    if (a.rule == MBBP_RULE_NMS)
        return reg ? launch_width<MBBP_RULE_NMS, true>(a, s, sm_count)
                   : launch_width<MBBP_RULE_NMS, false>(a, s, sm_count);
    return reg ? launch_width<MBBP_RULE_SP, true>(a, s, sm_count)
               : launch_width<MBBP_RULE_SP, false>(a, s, sm_count);
}

}  // namespace mbbp
