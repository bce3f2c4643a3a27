// Internal layout shared by the host library (host.cpp) and the kernels.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/mbbp.h"

namespace mbbp {

constexpr int kWarpsPerBlock = 8;
// Size of the fixed scratch array behind mbbp_decode_noalloc.
constexpr size_t kStaticScratchBytes = MBBP_NOALLOC_SCRATCH_BYTES;

inline int words_for(int n) { return (n + 31) / 32; }
inline int round_up(int x, int a) { return (x + a - 1) / a * a; }

// Device copy of the R representations of one code.  Rows of H^(t) are laid
// out ELL-style: the j-th edge of row r of representation t is "slot"
// j * MP + r of that representation's message array, so lane r of a warp
// reads the j-th message of its row with unit stride across the warp.
struct DevBases {
    const uint32_t* rowinfo;  // [R][MP] src row (bits 0-15) | degree (16-23) | valid (bit 31)
    const uint2* vdesc;       // [R][n]  x = first slot-list entry, y = variable | degree << 16;
                              //         variables sorted by degree (stable)
    const uint16_t* vslot;    // slot ids of every variable, ascending row of H^(t)
    const uint4* vdesc6;      // width 6 only: [R][n] in vdesc order, x = vdesc.y, y/z/w = byte
                              //         offsets (4 * slot id) of the variable's slots, 2 per word
    const int32_t* rows;      // [R] rows of H^(t)
    const int32_t* rowptr;    // [R][MP] first edge of each row (edges numbered row by row)
    const uint16_t* hcol;     // [DC][mpad] columns of the rows of H (n = padding)
    const uint32_t* hmask;    // [m][W] rows of H as bit masks
    int m, n, R, DC, DV, MP, mpad, W;
    int regular;              // every row of H has weight DC

    // Small-code layout (shape != 0; K = 6 and n <= 32 VS): rows placed at
    // ELL index sigma(r), edge j of the row at slot
    // j*MP + (sigma(r) & ~31) + ((sigma(r) + rot(j)) & 31), chosen by the host
    // to spread the variable pass over the shared-memory banks.
    const uint4* vdesc2;      // [R][VS*32] x = variable | degree << 16, y/z/w = 6 slot ids (u16)
    const uint32_t* rinfo2;   // [R][MP] ELL index -> src row | degree << 16
    const uint32_t* hmask2;   // [R][VS][ORS*32] rows of H as bit masks over positions
    const int32_t* sedge;     // [R][6*MP] edge id of every message slot (-1: none), for message traces
    int shape, VS, RS, ORS;

    // Serial schedule: rows of H^(t) in layer order, layer boundaries and,
    // per edge slot, the variable's slot list (x = first vslot entry,
    // y = variable | degree << 16).
    const uint16_t* lrows;    // [R][MP]
    const uint16_t* lptr;     // [R][MP+1]
    const int32_t* nlayers;   // [R]
    const uint2* evar;        // [R][DC*MP]
    // Serial schedule, widths 6 and 8 (null otherwise): per edge slot,
    // x = variable | first other edge << 16 and y/z/w = further other edges of
    // the variable (byte offsets of their slots, ascending row, padded with
    // the offset 4 * DC * MP of a -0.0f slot); per variable, its 8 slot byte
    // offsets (ascending row, padded the same way).
    const uint4* edesc;       // [R][DC*MP], by row position
    const uint4* vdesc3;      // [R][n]
    // chunk-kernel row positions (a permutation of the rows of H^(t) placed
    // to spread the kernel's shared-memory accesses over the banks): the
    // positions in layer order, and per position src row | degree << 16
    const uint16_t* lpos;     // [R][MP]
    const uint32_t* rinfo_s;  // [R][MP]
};

// Shared memory of one warp of the serial chunk kernel (bp_serial.cuh) for
// CS shots, and the CS the launch uses (the host places rows for it).
namespace serial_bp {
struct Layout {
    int SH;     // floats per shot message area (DC * MP messages, the -0 slot, padding)
    int NP;     // floats of mu per shot
    int EP;     // bytes of hard decisions per shot (n + 1 rounded to 16)
    int RW;     // syndrome words per shot (MP / 32), twice: by row position, by row of H
    int bytes;  // per warp (a multiple of 16)
};

__host__ __device__ inline Layout layout(int DC, int MP, int n, int CS) {
    Layout L;
    L.SH = DC * MP + 4;
    L.NP = (n + 3) & ~3;
    L.EP = (n + 16) & ~15;
    L.RW = MP >> 5;
    L.bytes = CS * (L.SH * 4 + L.NP * 4 + L.EP) + ((2 * CS * L.RW * 4 + 15) & ~15);
    return L;
}

constexpr int kWarps = 8;              // warps per block
constexpr int kBudget2 = 56 * 1024;    // shared memory per block that leaves about half of an SM to L1

// The largest CS in {4, 2, 1} whose 8-warp block fits kBudget2 (1 when none
// does; the launch then takes fewer warps at CS = 1).
inline int shots_per_warp(int DC, int MP, int mpad, int n) {
    const int hb = (DC * mpad * 2 + 15) & ~15;
    for (int cs : {4, 2})
        if (hb + kWarps * layout(DC, MP, n, cs).bytes <= kBudget2) return cs;
    return 1;
}
}  // namespace serial_bp

// Bank rotation of edge position j in the small-code layout.
__host__ __device__ constexpr int slot_rot(int j) { return (j * 11) & 31; }

struct SmallShape {
    int VS, RS, ORS;  // variable steps, row steps of H^(t), row steps of H (32 lanes each)
};
constexpr SmallShape kSmallShapes[] = {{3, 2, 2}, {5, 3, 3}, {5, 4, 3}};
constexpr int kNumSmallShapes = 3;

// Resident one-warp blocks per SM that the register budget of a small-code
// kernel (decode_small.cu, decode_mixed.cu) is sized for.  Measured on
// [[144]], R = 16: with 18, ptxas settles at 96 registers (20 resident warps
// per SM) and the kernel runs 9% faster than with 8-warp blocks at 116
// registers (16 warps per SM); tighter budgets (20 or 21 blocks), or 2-warp
// blocks at 10, were slower.  Four row steps and the sum-product rule need
// more registers: 16 keeps them unspilled.
__host__ __device__ constexpr int small_min_blocks(int RS, int rule) {
    return (RS <= 3 && rule == MBBP_RULE_NMS) ? 18 : 16;
}

// Inputs and per-representation outputs of one code's batch of shots.
struct ShotIO {
    const uint8_t* synd;      // [batch][m]
    const float* llr;         // [n] or [batch][llr_stride]
    int llr_stride;
    int batch, iters;
    float alpha;
    uint32_t* cand;           // [batch][R][W]
    uint8_t* conv;            // [batch][R]
    uint16_t* iters_run;      // [batch][R] or null
    float* post;              // [batch][R][n] or null
    float* c2v;               // [batch][R][c2v_stride] message trace (flooding kernels) or null
    int c2v_stride;           // the largest edge count of the representations
};

struct DecodeArgs {
    DevBases B;
    ShotIO io;
    int rule;
    unsigned long long* counter;
    unsigned long long total_items;
    unsigned int* rep_counter;  // [R] next shot of each representation (serial slot path)
};

struct FwsArgs {
    const uint32_t* cand;
    const uint8_t* conv;
    int batch, R, n, W;
    uint8_t* e_hat;
    uint8_t* success;
    int16_t* selected;
    int decision;             // MBBP_DECISION_FWS or MBBP_DECISION_LMS
    const float* llr;         // LMS metric weights: [n] or [batch][llr_stride]
    int llr_stride;
};

struct DevLogicals {
    const uint16_t* hcol;     // [DC][mpad]
    const uint32_t* lmask;    // [k][W]
    int m, n, k, DC, mpad, W;
};

// One code of a mixed batch (decode_mixed.cu).
constexpr int kMixedMaxCodes = 8;
constexpr int kMixedMaxWarps = 8;
constexpr int kKindSmall = 0;    // register-resident small-code path
constexpr int kKindGeneric = 1;  // generic path
struct MixedCode {
    DevBases B;
    ShotIO io;
    int kind;                   // kKindSmall / kKindGeneric
    int chunk;                  // shots per work item
    unsigned long long first;   // first global work index of this code
};
struct MixedArgs {
    MixedCode codes[kMixedMaxCodes];
    int n_codes;
    uint32_t warp_bytes;        // shared memory per warp (largest over codes)
    unsigned long long total;   // work items
    unsigned long long* counter;
};
size_t mixed_warp_bytes(const DevBases& B, int kind);
// Launch groups of a mixed batch: 0 = the generic path (blocks of `warps`
// warps), 1..kNumSmallShapes = the small-code path of that shape (one-warp
// blocks).
constexpr int kMixedGroups = 1 + kNumSmallShapes;
cudaError_t launch_mixed(const MixedArgs& a, int group, int warps, int rule, cudaStream_t s, int sm_count);

// Weighted min-sum forward / backward / decode (wms.cu).
struct WmsArgs {
    DevBases B;
    const uint8_t* synd;
    const float* llr;
    int llr_stride;
    int T, ckpt, nckpt, E;      // iterations, checkpoint interval, stored checkpoints, edges per row of w/g
    const float* w;             // [R][T][E]
    const float* g;             // [R][T][E]
    const uint32_t* etrue;      // [batch][W] bit-packed true errors, or null
    float scale;
    int all_iters;              // loss: mean BCE over all iterations instead of the last
    float* post;                // [batch][R][n]
    float* loss;                // [batch][R] or null
    float* ckpt_buf;            // [batch][R][nckpt][DC*MP]
    float* seg_buf;             // backward: [kWmsMaxWarps][ckpt][DC*MP], one segment per warp
    float* gw;                  // [R][T][E]
    float* gg;
    int decode, iters;          // decode mode: halting rule, candidates
    const float2* wg;           // decode mode: (w, g) in the message layout [R][T][DC][MP], or null
    uint32_t* cand;
    uint8_t* conv;
    uint16_t* iters_run;
    unsigned long long* counter;
    unsigned long long total_items;
};
constexpr int kWmsMaxWarps = 152 * 16;  // warps of the backward grid (segment buffers)
// Whether the WMS backward pass keeps its segment states in shared memory
// (then it needs no per-warp segment buffers in the workspace).
bool wms_states_in_smem(const DevBases& B, int ckpt);
cudaError_t launch_wms(const WmsArgs& a, bool backward, cudaStream_t s, int sm_count);
// Fills a.wg-style packed parameters from a.w / a.g (a.T iterations).
cudaError_t launch_wms_pack(const WmsArgs& a, float2* wg, cudaStream_t s, int sm_count);
cudaError_t launch_adam(float* p, const float* g, float* m1, float* m2, size_t count, float lr, float b1,
                        float b2, float eps, int step, float lo, float hi, cudaStream_t s);

// Launchers (decode.cu, decode_small.cu, aux.cu).  They return cudaGetLastError().
cudaError_t launch_decode(const DecodeArgs& a, cudaStream_t s, int sm_count);
cudaError_t launch_decode_serial(const DecodeArgs& a, cudaStream_t s, int sm_count);
cudaError_t launch_decode_serial_generic(const DecodeArgs& a, cudaStream_t s, int sm_count);
cudaError_t launch_decode_small(const DecodeArgs& a, cudaStream_t s, int sm_count);
cudaError_t launch_fws(const FwsArgs& a, cudaStream_t s);
// Device address of the fixed scratch array on the current device (looked up
// on the first call per device).
cudaError_t static_scratch(void** ptr);
// Sets the dynamic shared-memory limit of a kernel and returns its blocks per
// SM, once per (kernel, block size, shared memory, device); cached afterwards.
cudaError_t prepare_kernel(const void* func, int threads, size_t smem, int* blocks_per_sm);
// Throughput probe (probe.cu): one launch of probe `kind` (MBBP_PROBE_*);
// *work = its lane operations or shared-memory bytes.
cudaError_t launch_probe(int kind, int rounds, float* sink, cudaStream_t s, double* work);
cudaError_t launch_sample(int n, int batch, uint64_t first_shot, uint64_t seed, uint64_t T,
                          int noise, uint32_t* ex, uint32_t* ez, cudaStream_t s);
cudaError_t launch_syndrome(const DevBases& B, int batch, const uint32_t* e, uint8_t* synd,
                            cudaStream_t s);
cudaError_t launch_judge(const DevLogicals& L, int batch, const uint32_t* e,
                         const uint8_t* e_hat, uint8_t* fail, unsigned long long* counts,
                         cudaStream_t s);

}  // namespace mbbp
