// Monte-Carlo producer and logical judge around the decoder (Section IV):
// counter-based error sampling (splitmix64), syndromes s = H e over GF(2),
// and the residual test r = e XOR e_hat against H and the logical operators.
#include "mbbp_internal.h"

namespace mbbp {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ULL;

// splitmix64 output function (Steele, Lea & Flood, OOPSLA 2014).
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// One thread per (shot, 32-qubit word).
__global__ void sample_kernel(int n, int batch, uint64_t first_shot, uint64_t seed, uint64_t T,
                              int noise, uint32_t* __restrict__ ex, uint32_t* __restrict__ ez) {
    const int W = (n + 31) >> 5;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (long long)batch * W) return;
    const int b = (int)(tid / W);
    const int w = (int)(tid - (long long)b * W);
    const uint64_t shot = first_shot + (uint64_t)b;
    const uint64_t t1 = T / 3;
    const uint64_t base = seed + (shot * (uint64_t)n + (uint64_t)(32 * w) + 1ull) * kGolden;
    uint32_t x = 0, z = 0;
    const int cnt = min(32, n - 32 * w);
    for (int i = 0; i < cnt; ++i) {
        const uint64_t u = mix64(base + (uint64_t)i * kGolden);
        if (noise == MBBP_NOISE_BSC) {
            x |= (u < T ? 1u : 0u) << i;
        } else if (u < T) {
            if (u < t1) {
                x |= 1u << i;
            } else if (u < 2 * t1) {
                x |= 1u << i;
                z |= 1u << i;
            } else {
                z |= 1u << i;
            }
        }
    }
    ex[tid] = x;
    if (ez) ez[tid] = z;
}

// One warp per shot; lane r computes check r (and r + 32, ...).
__global__ void syndrome_kernel(const DevBases B, int batch, const uint32_t* __restrict__ e,
                                uint8_t* __restrict__ s) {
    const int lane = threadIdx.x & 31;
    const int shot = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (shot >= batch) return;
    const uint32_t* es = e + (size_t)shot * B.W;
    for (int r = lane; r < B.m; r += 32) {
        uint32_t par = 0;
        for (int j = 0; j < B.DC; ++j) {
            const int c = __ldg(B.hcol + j * B.mpad + r);
            if (c < B.n) par ^= (__ldg(es + (c >> 5)) >> (c & 31)) & 1u;
        }
        s[(size_t)shot * B.m + r] = (uint8_t)par;
    }
}

// One warp per shot: r = e ^ e_hat, then H r and the logical overlaps.
__global__ void judge_kernel(const DevLogicals L, int batch, const uint32_t* __restrict__ e,
                             const uint8_t* __restrict__ e_hat, uint8_t* __restrict__ fail,
                             unsigned long long* __restrict__ counts) {
    extern __shared__ uint32_t jsm[];
    __shared__ unsigned int block_counts[3];
    if (threadIdx.x < 3) block_counts[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int shot = blockIdx.x * (blockDim.x >> 5) + warp;
    const int W = L.W, n = L.n;
    if (shot < batch) {
        uint32_t* rw = jsm + (size_t)warp * W;
        for (int w = 0; w < W; ++w) {
            const int v = 32 * w + lane;
            const uint32_t bit = (v < n) ? (uint32_t)(e_hat[(size_t)shot * n + v] & 1u) : 0u;
            const uint32_t word = __ballot_sync(kFull, bit);
            if (lane == 0) rw[w] = word ^ __ldg(e + (size_t)shot * W + w);
        }
        __syncwarp();
        bool bad = false;
        for (int r = lane; r < L.m; r += 32) {
            uint32_t par = 0;
            for (int j = 0; j < L.DC; ++j) {
                const int c = __ldg(L.hcol + j * L.mpad + r);
                if (c < n) par ^= (rw[c >> 5] >> (c & 31)) & 1u;
            }
            bad = bad || par;
        }
        int code = 0;
        if (__any_sync(kFull, bad)) {
            code = 1;
        } else {
            bool odd = false;
            for (int i = lane; i < L.k; i += 32) {
                uint32_t acc = 0;
                for (int w = 0; w < W; ++w) acc ^= __ldg(L.lmask + (size_t)i * W + w) & rw[w];
                odd = odd || (__popc(acc) & 1);
            }
            if (__any_sync(kFull, odd)) code = 2;
        }
        if (lane == 0) {
            if (fail) fail[shot] = (uint8_t)code;
            if (counts) atomicAdd(&block_counts[code], 1u);
        }
    }
    __syncthreads();
    if (counts && threadIdx.x < 3 && block_counts[threadIdx.x])
        atomicAdd(counts + threadIdx.x, (unsigned long long)block_counts[threadIdx.x]);
}

}  // namespace

cudaError_t launch_sample(int n, int batch, uint64_t first_shot, uint64_t seed, uint64_t T,
                          int noise, uint32_t* ex, uint32_t* ez, cudaStream_t s) {
    const long long threads = (long long)batch * words_for(n);
    const int block = 256;
    const unsigned grid = (unsigned)((threads + block - 1) / block);
    sample_kernel<<<grid, block, 0, s>>>(n, batch, first_shot, seed, T, noise, ex, ez);
    return cudaGetLastError();
}

cudaError_t launch_syndrome(const DevBases& B, int batch, const uint32_t* e, uint8_t* synd,
                            cudaStream_t s) {
    const int warps = 8;
    const unsigned grid = (unsigned)((batch + warps - 1) / warps);
    syndrome_kernel<<<grid, warps * 32, 0, s>>>(B, batch, e, synd);
    return cudaGetLastError();
}

cudaError_t launch_judge(const DevLogicals& L, int batch, const uint32_t* e,
                         const uint8_t* e_hat, uint8_t* fail, unsigned long long* counts,
                         cudaStream_t s) {
    const int warps = 8;
    const unsigned grid = (unsigned)((batch + warps - 1) / warps);
    const size_t smem = (size_t)warps * L.W * 4;
    judge_kernel<<<grid, warps * 32, smem, s>>>(L, batch, e, e_hat, fail, counts);
    return cudaGetLastError();
}

}  // namespace mbbp
