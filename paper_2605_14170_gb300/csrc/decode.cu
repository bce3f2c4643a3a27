// MBBP-LD decode kernels for sm_103a: flooding BP on every (shot,
// representation) pair (Section II-B), then Frequency-Weighted Scoring of
// each shot's converged candidates (Section III-B); Algorithm 1 as a whole.
//
// Mapping.  One warp decodes one (shot, representation) item and keeps all
// of its edge messages in shared memory: a single float per edge, which
// holds q_{v->c} after the variable pass and m_{c->v} after the check pass
// (each pass reads every message of a node before it overwrites them, and
// every edge belongs to exactly one check and one variable, so no other lane
// touches it).  Lanes own checks r = lane + 32k; edge j of check r lives at
// slot j * MP + r, so the check pass reads and writes with unit stride across
// the warp.  Variables are visited in degree-sorted order so that the lanes
// of one step mostly share a degree.  Items come from a global work counter,
// which balances the early exits of the halting rule.
//
// Arithmetic.  Every float operation is a correctly rounded intrinsic
// (__fadd_rn / __fmul_rn) in the order the oracle uses: variable sums in
// ascending row order of H^(t) excluding the own edge, sum-product phi sums
// in ascending column order excluding the own edge.  Min-sum takes its min
// over the other edges and MBBP_LMAX with a min1/min2 pair, which gives the
// same value as the direct min.  Hence normalized min-sum reproduces the FP32
// oracle bit for bit; sum-product differs only through expm1f/log1pf.
#include <mutex>

#include "mbbp_internal.h"

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

__host__ __device__ __forceinline__ int align16(int x) { return (x + 15) & ~15; }

struct WarpLayout {
    int S, npad, ehpad, per_warp, hcol_bytes;
};

__host__ __device__ __forceinline__ WarpLayout warp_layout(int DC, int MP, int mpad, int n) {
    WarpLayout L;
    L.S = DC * MP;
    L.npad = (n + 4) & ~3;
    L.ehpad = align16(n + 1);
    L.per_warp = L.S * 4 + L.npad * 4 + L.ehpad;
    L.hcol_bytes = align16(DC * mpad * 2);
    return L;
}

// Gallager's phi(x) = log((e^x + 1) / (e^x - 1)) = log1p(2 / expm1(x)), with
// phi(0) = inf and phi(inf) = 0; phi is its own inverse on (0, inf).
__device__ __forceinline__ float phi(float x) {
    return log1pf(__fdiv_rn(2.0f, expm1f(x)));
}

// Check-node update of row r (Eq. (2) with the syndrome sign, or the
// sum-product rule).  deg <= DC edges at slots j * MP + r.
template <int DC, int RULE>
__device__ __forceinline__ void check_row(float* msg, int r, int MP, int deg, uint32_t sbit,
                                          float alpha) {
    float q[DC];
#pragma unroll
    for (int j = 0; j < DC; ++j) q[j] = (j < deg) ? msg[j * MP + r] : MBBP_LMAX;
    if (RULE == MBBP_RULE_NMS) {
        float min1 = MBBP_LMAX, min2 = MBBP_LMAX;
        uint32_t par = sbit;
#pragma unroll
        for (int j = 0; j < DC; ++j) {
            const float x = fabsf(q[j]);
            min2 = fminf(min2, fmaxf(min1, x));
            min1 = fminf(min1, x);
            par ^= (q[j] < 0.f) ? 1u : 0u;
        }
        const float am1 = __fmul_rn(alpha, min1);
        const float am2 = __fmul_rn(alpha, min2);
#pragma unroll
        for (int j = 0; j < DC; ++j) {
            if (j < deg) {
                const float mag = (fabsf(q[j]) == min1) ? am2 : am1;
                const uint32_t neg = par ^ ((q[j] < 0.f) ? 1u : 0u);
                msg[j * MP + r] = neg ? -mag : mag;
            }
        }
    } else {
        // sum-product with Gallager's phi: |m| = phi(sum_{k != j} phi(|q_k|))
        float f[DC];
        uint32_t par = sbit;
#pragma unroll
        for (int j = 0; j < DC; ++j) {
            f[j] = (j < deg) ? phi(fabsf(q[j])) : 0.0f;
            par ^= (q[j] < 0.f) ? 1u : 0u;
        }
        float pre = 0.0f;  // f_0 + ... + f_{j-1}, left to right
#pragma unroll
        for (int j = 0; j < DC; ++j) {
            if (j < deg) {
                float sum = pre;
#pragma unroll
                for (int k = j + 1; k < DC; ++k)
                    if (k < deg) sum = __fadd_rn(sum, f[k]);
                const float mag = fminf(phi(sum), MBBP_SP_MAX);
                const uint32_t neg = par ^ ((q[j] < 0.f) ? 1u : 0u);
                msg[j * MP + r] = neg ? -mag : mag;
            }
            pre = __fadd_rn(pre, f[j]);
        }
    }
}

// Variable-node update of a degree-D variable (Eq. (3)): q_i = mu + sum of
// the other messages in ascending row order, clamped; returns the posterior.
template <int D>
__device__ __forceinline__ float var_update(float* msg, const uint16_t* __restrict__ sl,
                                            float mu) {
    int s[D];
    float m[D];
#pragma unroll
    for (int i = 0; i < D; ++i) s[i] = __ldg(sl + i);
#pragma unroll
    for (int i = 0; i < D; ++i) m[i] = msg[s[i]];
    float P[D + 1];
    P[0] = mu;
#pragma unroll
    for (int i = 0; i < D; ++i) P[i + 1] = __fadd_rn(P[i], m[i]);
#pragma unroll
    for (int i = 0; i < D; ++i) {
        float q = P[i];
#pragma unroll
        for (int k = i + 1; k < D; ++k) q = __fadd_rn(q, m[k]);
        msg[s[i]] = fminf(fmaxf(q, -MBBP_LMAX), MBBP_LMAX);
    }
    return P[D];
}

template <int D, int DV>
__device__ __forceinline__ float var_dispatch(int deg, float* msg, const uint16_t* sl, float mu) {
    if constexpr (D > DV) {
        return mu;
    } else {
        if (deg == D) return var_update<D>(msg, sl, mu);
        return var_dispatch<D + 1, DV>(deg, msg, sl, mu);
    }
}

template <int DC, int DV, int RULE>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
decode_kernel(const DecodeArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const DevBases& B = a.B;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int MP = B.MP, n = B.n, m = B.m, R = B.R, W = B.W, mpad = B.mpad;
    const WarpLayout L = warp_layout(DC, MP, mpad, n);
    uint16_t* hcol_s = reinterpret_cast<uint16_t*>(smem);
    float* msg = reinterpret_cast<float*>(smem + L.hcol_bytes + warp * L.per_warp);
    float* mu_s = msg + L.S;
    uint8_t* eh = reinterpret_cast<uint8_t*>(mu_s + L.npad);

    for (int i = threadIdx.x; i < DC * mpad; i += blockDim.x) hcol_s[i] = __ldg(B.hcol + i);
    __syncthreads();

    const int row_steps = MP >> 5;
    const int orow_steps = mpad >> 5;
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(a.counter, 1ull);
        item = __shfl_sync(kFull, item, 0);
        if (item >= a.total_items) break;
        const int shot = (int)(item / (unsigned long long)R);
        const int b = (int)(item - (unsigned long long)shot * R);
        const uint32_t* rinfo = B.rowinfo + (size_t)b * MP;
        const uint2* vd = B.vdesc + (size_t)b * n;
        const int Mb = __ldg(B.rows + b);
        const float* llr = a.llr + (size_t)shot * a.llr_stride;
        const uint8_t* sy = a.synd + (size_t)shot * m;

        // channel LLRs, hard decision of the LLRs, syndrome bits of my rows
        for (int v = lane; v < n; v += 32) {
            const float x = __ldg(llr + v);
            mu_s[v] = x;
            eh[v] = (x < 0.f) ? 1 : 0;
        }
        if (lane == 0) eh[n] = 0;  // padding column of hcol
        uint32_t sb = 0;
        for (int k = 0; k < row_steps; ++k) {
            const int r = lane + 32 * k;
            if (r < Mb) sb |= (uint32_t)(__ldg(sy + (__ldg(rinfo + r) & 0xffffu)) & 1u) << k;
        }
        __syncwarp();
        // q^(0)_{v->c} = mu_v
        for (int p = lane; p < n; p += 32) {
            const uint2 d = __ldg(vd + p);
            const int v = d.y & 0xffff, deg = (int)(d.y >> 16);
            const float x = mu_s[v];
            for (int i = 0; i < deg; ++i) msg[__ldg(B.vslot + d.x + i)] = x;
            if (a.post) a.post[item * n + v] = x;
        }
        __syncwarp();

        int K = 0;
        bool conv = false;
        for (int it = 0;; ++it) {
            // halting rule: H e = s on the rows of H (the extra rows are copies)
            bool ok = true;
            for (int k = 0; k < orow_steps; ++k) {
                const int r = lane + 32 * k;
                if (r < m) {
                    uint32_t par = (sb >> k) & 1u;
#pragma unroll
                    for (int j = 0; j < DC; ++j) par ^= eh[hcol_s[j * mpad + r]];
                    ok = ok && (par == 0u);
                }
            }
            if (__all_sync(kFull, ok)) {
                conv = true;
                K = it;
                break;
            }
            if (it == a.iters) {
                K = it;
                break;
            }
            // check pass
            for (int k = 0; k < row_steps; ++k) {
                const int r = lane + 32 * k;
                if (r < Mb) {
                    const int deg = B.regular ? DC : (int)((__ldg(rinfo + r) >> 16) & 0xffu);
                    check_row<DC, RULE>(msg, r, MP, deg, (sb >> k) & 1u, a.alpha);
                }
            }
            __syncwarp();
            // variable pass, posterior, hard decision
            for (int p = lane; p < n; p += 32) {
                const uint2 d = __ldg(vd + p);
                const int v = d.y & 0xffff, deg = (int)(d.y >> 16);
                const float post = var_dispatch<1, DV>(deg, msg, B.vslot + d.x, mu_s[v]);
                eh[v] = (post < 0.f) ? 1 : 0;
                if (a.post) a.post[item * n + v] = post;
            }
            __syncwarp();
        }
        // candidate e_t (bit-packed), convergence flag, iterations
        uint32_t myword = 0;
        for (int w = 0; w < W; ++w) {
            const int v = 32 * w + lane;
            const uint32_t bit = (v < n) ? (uint32_t)eh[v] : 0u;
            const uint32_t word = __ballot_sync(kFull, bit);
            if ((w & 31) == lane) myword = word;
            if ((w & 31) == 31 || w == W - 1) {
                const int base = w & ~31;
                if (base + lane <= w) a.cand[item * W + base + lane] = myword;
            }
        }
        if (lane == 0) {
            a.conv[item] = conv ? 1 : 0;
            if (a.iters_run) a.iters_run[item] = (uint16_t)K;
        }
        __syncwarp();
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

template <int K, int RULE>
cudaError_t launch_decode_t(const DecodeArgs& a, cudaStream_t s, int sm_count) {
    auto kern = decode_kernel<K, K, RULE>;
    const WarpLayout L = warp_layout(K, a.B.MP, a.B.mpad, a.B.n);
    int warps = kWarpsPerBlock;
    while (warps > 1 && (size_t)L.hcol_bytes + (size_t)warps * L.per_warp > 200 * 1024) --warps;
    const size_t smem = (size_t)L.hcol_bytes + (size_t)warps * L.per_warp;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    unsigned long long want = (a.total_items + warps - 1) / warps;
    unsigned long long grid = (unsigned long long)per_sm * (unsigned long long)sm_count;
    if (want < grid) grid = want;
    kern<<<(unsigned)grid, warps * 32, smem, s>>>(a);
    return cudaGetLastError();
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

size_t decode_smem_bytes(const DevBases& B, int warps) {
    const WarpLayout L = warp_layout(B.DC, B.MP, B.mpad, B.n);
    return (size_t)L.hcol_bytes + (size_t)warps * L.per_warp;
}

cudaError_t launch_decode(const DecodeArgs& a, cudaStream_t s, int sm_count) {
    if (a.B.shape != 0) return launch_decode_small(a, s, sm_count);
    const int K = a.B.DC;
    if (a.rule == MBBP_RULE_NMS) {
        if (K == 6) return launch_decode_t<6, MBBP_RULE_NMS>(a, s, sm_count);
        if (K == 8) return launch_decode_t<8, MBBP_RULE_NMS>(a, s, sm_count);
        if (K == 12) return launch_decode_t<12, MBBP_RULE_NMS>(a, s, sm_count);
    } else {
        if (K == 6) return launch_decode_t<6, MBBP_RULE_SP>(a, s, sm_count);
        if (K == 8) return launch_decode_t<8, MBBP_RULE_SP>(a, s, sm_count);
        if (K == 12) return launch_decode_t<12, MBBP_RULE_SP>(a, s, sm_count);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_fws(const FwsArgs& a, cudaStream_t s) {
    const size_t per_warp = (size_t)a.R * a.W * 4;
    int warps = kWarpsPerBlock;
    while (warps > 1 && warps * per_warp > 96 * 1024) --warps;
    const size_t smem = warps * per_warp;
    cudaError_t e = cudaFuncSetAttribute(fws_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)((a.batch + warps - 1) / warps);
    fws_kernel<<<grid, warps * 32, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace mbbp
