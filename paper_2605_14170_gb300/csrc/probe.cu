// Throughput probes: the per-SM issue rates that the BP kernels' roofline
// divides by, measured on the GPU at hand rather than taken from a data
// sheet.  Each probe keeps every SM full (1024-thread blocks, as many as
// fit) with one kind of operation:
//   FP32 add, FP32 min/max and 3-input logic — 8 dependency chains per
//   thread that feed each other (a chain's next operand is a neighbour's
//   value), so no two operations can be merged and every one executes;
//   shared-memory loads — 16-byte loads at conflict-free addresses that move
//   with the round, folded into one word by 3-input XORs.
// The caller times one launch with CUDA events and divides the work the
// launch reports by the time, the SM count and the SM clock.
#include "mbbp_internal.h"

namespace mbbp {
namespace {

constexpr int kProbeThreads = 1024;
constexpr int kProbeChains = 8;
constexpr int kProbeSteps = 8;       // unrolled steps per round: 64 operations per thread
constexpr int kProbeTile = 2048;     // float4 elements of the shared-memory probe (32 KB)

template <int KIND>
__global__ void __launch_bounds__(kProbeThreads, 2) probe_kernel(int rounds, float key, float* sink) {
    extern __shared__ float4 tile[];
    const int t = threadIdx.x;
    if (KIND == MBBP_PROBE_SMEM) {
        for (int i = t; i < kProbeTile; i += blockDim.x)
            tile[i] = make_float4(key * i, key + i, key - i, key * (i + 1));
        __syncthreads();
        uint32_t acc = 0;
        for (int r = 0; r < rounds; ++r) {
            // warp w reads 32 consecutive float4 (four conflict-free wavefronts)
            const float4* base = tile + ((t + 32 * r) & 255);
#pragma unroll
            for (int s = 0; s < kProbeSteps; ++s) {
                const float4 v = base[256 * s];
                acc ^= __float_as_uint(v.x) ^ __float_as_uint(v.y) ^ __float_as_uint(v.z) ^ __float_as_uint(v.w);
            }
        }
        if (__uint_as_float(acc) == key) sink[0] = __uint_as_float(acc);
        return;
    }
    if (KIND == MBBP_PROBE_LOP3) {
        uint32_t u[kProbeChains];
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) u[k] = __float_as_uint(key) * (uint32_t)(t + 7 * k + 1);
        for (int r = 0; r < rounds; ++r) {
#pragma unroll
            for (int s = 0; s < kProbeSteps; ++s)
#pragma unroll
                for (int k = 0; k < kProbeChains; ++k)
                    asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;"
                                 : "+r"(u[k])
                                 : "r"(u[(k + 1) % kProbeChains]), "r"(u[(k + 3) % kProbeChains]));
        }
        uint32_t acc = 0;
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) acc += u[k];
        if (__uint_as_float(acc) == key) sink[0] = __uint_as_float(acc);
        return;
    }
    float a[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = key * (float)(t + 7 * k + 1);
    for (int r = 0; r < rounds; ++r) {
#pragma unroll
        for (int s = 0; s < kProbeSteps; ++s)
#pragma unroll
            for (int k = 0; k < kProbeChains; ++k) {
                const float b = a[(k + 1) % kProbeChains];
                if (KIND == MBBP_PROBE_FADD) {
                    asm volatile("add.rn.f32 %0, %0, %1;" : "+f"(a[k]) : "f"(b));
                } else if (s & 1) {
                    asm volatile("max.f32 %0, %0, %1;" : "+f"(a[k]) : "f"(b));
                } else {
                    asm volatile("min.f32 %0, %0, %1;" : "+f"(a[k]) : "f"(b));
                }
            }
    }
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) acc += a[k];
    if (acc == key) sink[0] = acc;
}

template <int KIND>
cudaError_t launch_probe_t(int rounds, float* sink, cudaStream_t s, double* work) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const size_t smem = KIND == MBBP_PROBE_SMEM ? kProbeTile * sizeof(float4) : 0;
    int per_sm = 0;
    e = prepare_kernel(reinterpret_cast<const void*>(probe_kernel<KIND>), kProbeThreads, smem, &per_sm);
    if (e != cudaSuccess) return e;
    const double threads = (double)per_sm * sms * kProbeThreads;
    const double per_round = KIND == MBBP_PROBE_SMEM ? kProbeSteps * sizeof(float4)
                                                     : (double)kProbeSteps * kProbeChains;
    *work = threads * rounds * per_round;
    // key 1e-30: no chain can end equal to it, so the sink is never written
    probe_kernel<KIND><<<per_sm * sms, kProbeThreads, smem, s>>>(rounds, 1e-30f, sink);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_probe(int kind, int rounds, float* sink, cudaStream_t s, double* work) {
    switch (kind) {
        case MBBP_PROBE_FADD: return launch_probe_t<MBBP_PROBE_FADD>(rounds, sink, s, work);
        case MBBP_PROBE_FMNMX: return launch_probe_t<MBBP_PROBE_FMNMX>(rounds, sink, s, work);
        case MBBP_PROBE_LOP3: return launch_probe_t<MBBP_PROBE_LOP3>(rounds, sink, s, work);
        case MBBP_PROBE_SMEM: return launch_probe_t<MBBP_PROBE_SMEM>(rounds, sink, s, work);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mbbp
