// Register-resident BP kernel for small codes (n <= 160, rows of H^(t) <= 128,
// check weight <= 6): the [[72,12,6]] and [[144,12,12]] bivariate bicycle
// codes of Section IV.  Same item mapping and arithmetic as decode_kernel
// (one warp per (shot, representation), flooding BP of Section II-B, halting
// rule, messages in shared memory, FP32 oracle order), organised to issue as
// few instructions per edge as possible:
//   - a warp takes a chunk of kChunk consecutive shots of one representation,
//     so everything fixed for the representation is loaded once per chunk:
//     the shared-memory byte addresses of every variable's edges in ascending
//     row order of H^(t) and the variable degrees stay in registers, the rows
//     of H as bit masks over positions go to the warp's shared memory;
//   - variables are visited in degree-sorted order, so the lanes of a step
//     mostly take the same case of the degree switch;
//   - check messages leave the check pass pre-signed: one select and one
//     LOP3 per edge;
//   - the halting test H e = s uses the ballot-packed hard decisions, W
//     AND-XORs and a popcount per row, with no shared-memory traffic.
// The host places rows and variables (row index sigma(r), bank rotation of
// edge position j) to spread the variable pass over the shared-memory banks.
#include "mbbp_internal.h"

namespace mbbp {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kSmallWarps = 8;
constexpr int kChunk = 4;  // shots per work item of a warp (same representation)

__device__ __forceinline__ float phi_s(float x) {
    return log1pf(__fdiv_rn(2.0f, expm1f(x)));
}

// Byte address (shared window) of edge i of a variable descriptor.
__device__ __forceinline__ uint32_t addr_of(const uint4& d, int i) {
    const uint32_t w = (i < 2) ? d.y : (i < 4 ? d.z : d.w);
    return (i & 1) ? (w >> 16) : (w & 0xffffu);
}

// Shared-memory accesses by byte offset from the start of the dynamic
// shared array (the compiler keeps them in the shared state space).
__device__ __forceinline__ float lds(const char* smc, uint32_t off) {
    return *reinterpret_cast<const float*>(smc + off);
}
__device__ __forceinline__ void sts(char* smc, uint32_t off, float v) {
    *reinterpret_cast<float*>(smc + off) = v;
}

// Check update of one row (one row per lane) whose messages q[] were loaded
// from byte offsets cb[j] + 128 k.
template <int K, int RULE, bool REG>
__device__ __forceinline__ void check_row(char* smc, const float (&q)[K], const uint32_t (&cb)[K],
                                           int k, int deg, bool valid, uint32_t sbit, float alpha) {
    uint32_t sx = sbit << 31;
#pragma unroll
    for (int j = 0; j < K; ++j) sx ^= __float_as_uint(q[j]);
    sx &= 0x80000000u;
    if (RULE == MBBP_RULE_NMS) {
        // min over the other edges and LMAX, from prefix and suffix minima
        float pre[K], suf[K];
        pre[0] = MBBP_LMAX;
#pragma unroll
        for (int j = 1; j < K; ++j) pre[j] = fminf(pre[j - 1], fabsf(q[j - 1]));
        suf[K - 1] = MBBP_LMAX;
#pragma unroll
        for (int j = K - 2; j >= 0; --j)
            suf[j] = (j == K - 2) ? fabsf(q[K - 1]) : fminf(suf[j + 1], fabsf(q[j + 1]));
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const float excl = (j == K - 1) ? pre[j] : (j == 0 ? fminf(MBBP_LMAX, suf[0]) : fminf(pre[j], suf[j]));
            const uint32_t mag = __float_as_uint(__fmul_rn(alpha, excl));
            const uint32_t out = mag ^ ((sx ^ __float_as_uint(q[j])) & 0x80000000u);
            if (valid && (REG || j < deg)) sts(smc, cb[j] + 128 * k, __uint_as_float(out));
        }
    } else {
        float f[K];
#pragma unroll
        for (int j = 0; j < K; ++j) f[j] = (REG || j < deg) ? phi_s(fabsf(q[j])) : 0.0f;
        float pre = 0.0f;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            float sum = pre;
#pragma unroll
            for (int t = j + 1; t < K; ++t)
                if (REG || t < deg) sum = __fadd_rn(sum, f[t]);
            const float mag = fminf(phi_s(sum), MBBP_SP_MAX);
            const uint32_t out = (__float_as_uint(mag) ^ sx) ^ (__float_as_uint(q[j]) & 0x80000000u);
            if (valid && (REG || j < deg)) sts(smc, cb[j] + 128 * k, __uint_as_float(out));
            pre = __fadd_rn(pre, f[j]);
        }
    }
}

// Variable update of a degree-D variable (Eq. (3), ascending row order of
// H^(t)); returns the posterior.  The clamp of q to [-LMAX, LMAX] is not
// applied here because nothing observable depends on it: q only feeds the
// check rule, whose min also runs over LMAX (so |q| >= LMAX and LMAX give the
// same message and sign), and phi(|q|) underflows to 0 for |q| >= 104 under
// either value; q stays finite (|q| <= |mu| + 6 LMAX).
template <int D>
__device__ __forceinline__ float var_upd(char* smc, const uint4& d, float mu) {
    uint32_t a[D];
    float m[D];
#pragma unroll
    for (int i = 0; i < D; ++i) a[i] = addr_of(d, i);
#pragma unroll
    for (int i = 0; i < D; ++i) m[i] = lds(smc, a[i]);
    float P[D + 1];
    P[0] = mu;
#pragma unroll
    for (int i = 0; i < D; ++i) P[i + 1] = __fadd_rn(P[i], m[i]);
#pragma unroll
    for (int i = 0; i < D; ++i) {
        float q = P[i];
#pragma unroll
        for (int t = i + 1; t < D; ++t) q = __fadd_rn(q, m[t]);
        sts(smc, a[i], q);
    }
    return P[D];
}

__device__ __forceinline__ float var_step(char* smc, int deg, const uint4& d, float mu) {
    switch (deg) {
        case 1: return var_upd<1>(smc, d, mu);
        case 2: return var_upd<2>(smc, d, mu);
        case 3: return var_upd<3>(smc, d, mu);
        case 4: return var_upd<4>(smc, d, mu);
        case 5: return var_upd<5>(smc, d, mu);
        case 6: return var_upd<6>(smc, d, mu);
        default: return mu;
    }
}

// Shared memory of one warp: K*MP messages, a zero slot (padded to 16 B),
// then the halting-test masks of its representation (ORS*32 rows x VS words).
__host__ __device__ constexpr int small_warp_floats(int MP, int VS, int ORS) {
    return 6 * MP + 4 + VS * ORS * 32;
}

// Blocks per SM the register budget is sized for (measured: 3 blocks at 80
// registers issue more instructions than they gain in occupancy).
template <int RS, int RULE, bool REG>
constexpr int small_min_blocks() { return 2; }

template <int VS, int RS, int ORS, int RULE, bool REG>
__global__ void __launch_bounds__(kSmallWarps * 32, (small_min_blocks<RS, RULE, REG>()))
decode_small_kernel(const DecodeArgs a) {
    constexpr int K = 6;
    extern __shared__ __align__(16) float smsg[];
    const DevBases& B = a.B;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int MP = B.MP, n = B.n, m = B.m, R = B.R;
    const int warp_floats = small_warp_floats(MP, VS, ORS);
    char* smc = reinterpret_cast<char*>(smsg);
    float* msg = smsg + (size_t)warp * warp_floats;
    uint32_t* hms = reinterpret_cast<uint32_t*>(msg + K * MP + 4);  // [VS][ORS*32]
    const uint32_t wbase = (uint32_t)(warp * warp_floats * 4);  // byte offset of this warp's area
    if (lane == 0) msg[K * MP] = 0.0f;
    uint32_t cb[K];
#pragma unroll
    for (int j = 0; j < K; ++j) cb[j] = wbase + 4u * (uint32_t)(j * MP + ((lane + slot_rot(j)) & 31));
    __syncwarp();
    const unsigned long long chunks_per_rep = ((unsigned long long)a.batch + kChunk - 1) / kChunk;
    const unsigned long long total_chunks = chunks_per_rep * (unsigned long long)R;
    const uint32_t wshift = wbase | (wbase << 16);

    for (;;) {
        unsigned long long chunk = 0;
        if (lane == 0) chunk = atomicAdd(a.counter, 1ull);
        chunk = __shfl_sync(kFull, chunk, 0);
        if (chunk >= total_chunks) break;
        const int sblock = (int)(chunk / (unsigned long long)R);
        const int b = (int)(chunk - (unsigned long long)sblock * R);
        const int Mb = __ldg(B.rows + b);
        const uint4* vd = B.vdesc2 + (size_t)b * (VS * 32);
        const uint32_t* ri = B.rinfo2 + (size_t)b * MP;
        const uint32_t* hm = B.hmask2 + (size_t)b * VS * (ORS * 32);

        // fixed for the representation: descriptors, step degrees, masks, rows
        // edge addresses of every variable (y/z/w of the descriptors) and the
        // degrees, 4 bits per variable step; variable ids are re-read from L1
        // when a shot starts and ends
        uint4 desc[VS];
        uint32_t degs = 0;
#pragma unroll
        for (int k = 0; k < VS; ++k) {
            desc[k] = __ldg(vd + 32 * k + lane);
            desc[k].y += wshift;
            desc[k].z += wshift;
            desc[k].w += wshift;
            degs |= (desc[k].x >> 16) << (4 * k);
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < ORS; ++k)
#pragma unroll
            for (int w = 0; w < VS; ++w)
                hms[w * (ORS * 32) + lane + 32 * k] = __ldg(hm + w * (ORS * 32) + lane + 32 * k);
        uint32_t rowdeg = 0;  // degree of every row of this lane, 4 bits each (irregular H)
        if (!REG) {
#pragma unroll
            for (int k = 0; k < RS; ++k) {
                const int idx = lane + 32 * k;
                if (idx < Mb) rowdeg |= ((__ldg(ri + idx) >> 16) & 0xfu) << (4 * k);
            }
        }

        const int shot_end = min(a.batch, (sblock + 1) * kChunk);
        for (int shot = sblock * kChunk; shot < shot_end; ++shot) {
            const unsigned long long item = (unsigned long long)shot * R + b;
            const float* llr = a.llr + (size_t)shot * a.llr_stride;
            const uint8_t* sy = a.synd + (size_t)shot * m;
            float mu[VS];
            uint32_t ew[VS];
#pragma unroll
            for (int k = 0; k < VS; ++k) {
                const bool live = (32 * k + lane) < n;
                const uint32_t v = __ldg(&vd[32 * k + lane].x) & 0xffffu;
                // + 0.0f turns -0 into +0: decision-neutral, keeps -0 out of every sum
                mu[k] = live ? __fadd_rn(__ldg(llr + v), 0.0f) : 0.0f;
                ew[k] = __ballot_sync(kFull, mu[k] < 0.f);
            }
            uint32_t sb = 0, sbo = 0;
#pragma unroll
            for (int k = 0; k < RS; ++k)
                if (lane + 32 * k < Mb) sb |= (uint32_t)(__ldg(sy + (__ldg(ri + lane + 32 * k) & 0xffffu)) & 1u) << k;
#pragma unroll
            for (int k = 0; k < ORS; ++k)
                if (lane + 32 * k < m) sbo |= (uint32_t)(__ldg(sy + lane + 32 * k) & 1u) << k;
            // q^(0) = mu on every edge
#pragma unroll
            for (int k = 0; k < VS; ++k) {
                const int deg = (int)((degs >> (4 * k)) & 0xfu);
#pragma unroll
                for (int i = 0; i < K; ++i)
                    if (i < deg) sts(smc, addr_of(desc[k], i), mu[k]);
            }
            if (a.post) {
#pragma unroll
                for (int k = 0; k < VS; ++k)
                    if (32 * k + lane < n) a.post[item * n + (__ldg(&vd[32 * k + lane].x) & 0xffffu)] = mu[k];
            }
            __syncwarp();

            int K_run = 0;
            bool conv = false;
            for (int it = 0;; ++it) {
                // halting rule: the first row group of every lane decides most
                // unconverged iterations; the rest is tested only if it passed
                bool ok;
                {
                    uint32_t acc = 0;
#pragma unroll
                    for (int w = 0; w < VS; ++w) acc ^= hms[w * (ORS * 32) + lane] & ew[w];
                    ok = ((__popc(acc) ^ sbo) & 1u) == 0u;
                }
                bool conv_now = __all_sync(kFull, ok);
                if (ORS > 1 && conv_now) {
#pragma unroll
                    for (int k = 1; k < ORS; ++k) {
                        uint32_t acc = 0;
#pragma unroll
                        for (int w = 0; w < VS; ++w) acc ^= hms[w * (ORS * 32) + lane + 32 * k] & ew[w];
                        ok = ok && (((__popc(acc) ^ (sbo >> k)) & 1u) == 0u);
                    }
                    conv_now = __all_sync(kFull, ok);
                }
                if (conv_now) {
                    conv = true;
                    K_run = it;
                    break;
                }
                if (it == a.iters) {
                    K_run = it;
                    break;
                }
                // check pass: all rows' messages are loaded first, then updated
                float q[RS][K];
#pragma unroll
                for (int k = 0; k < RS; ++k) {
                    if (32 * k < Mb) {
                        const int deg = REG ? K : (int)((rowdeg >> (4 * k)) & 0xfu);
#pragma unroll
                        for (int j = 0; j < K; ++j)
                            q[k][j] = (REG || j < deg) ? lds(smc, cb[j] + 128 * k) : MBBP_LMAX;
                    }
                }
#pragma unroll
                for (int k = 0; k < RS; ++k) {
                    if (32 * k < Mb) {
                        const bool valid = lane + 32 * k < Mb;
                        const int deg = REG ? K : (int)((rowdeg >> (4 * k)) & 0xfu);
                        check_row<K, RULE, REG>(smc, q[k], cb, k, deg, valid, (sb >> k) & 1u, a.alpha);
                    }
                }
                __syncwarp();
                // variable pass
#pragma unroll
                for (int k = 0; k < VS; ++k) {
                    if (32 * k < n) {
                        const int deg = (int)((degs >> (4 * k)) & 0xfu);
                        const float post = var_step(smc, deg, desc[k], mu[k]);
                        ew[k] = __ballot_sync(kFull, post < 0.f);
                        if (a.post && 32 * k + lane < n)
                            a.post[item * n + (__ldg(&vd[32 * k + lane].x) & 0xffffu)] = post;
                    }
                }
                __syncwarp();
            }
            // Candidate in variable order (bit v = variable v), through a byte
            // per variable in the message area, then one ballot per word.
            __syncwarp();
            uint8_t* ebytes = reinterpret_cast<uint8_t*>(msg);
#pragma unroll
            for (int k = 0; k < VS; ++k)
                if (32 * k + lane < n)
                    ebytes[__ldg(&vd[32 * k + lane].x) & 0xffffu] = (uint8_t)((ew[k] >> lane) & 1u);
            __syncwarp();
            uint32_t myword = 0;
#pragma unroll
            for (int w = 0; w < VS; ++w) {
                const int v = 32 * w + lane;
                const uint32_t word = __ballot_sync(kFull, v < n && ebytes[v]);
                if (lane == w) myword = word;
            }
            const int W = (n + 31) >> 5;
            if (lane < W) a.cand[item * W + lane] = myword;
            if (lane == 0) {
                a.conv[item] = conv ? 1 : 0;
                if (a.iters_run) a.iters_run[item] = (uint16_t)K_run;
            }
            __syncwarp();
        }
    }
}

template <int VS, int RS, int ORS, int RULE, bool REG>
cudaError_t launch_small_t(const DecodeArgs& a, cudaStream_t s, int sm_count) {
    auto kern = decode_small_kernel<VS, RS, ORS, RULE, REG>;
    const int warps = kSmallWarps;
    const size_t smem = (size_t)warps * small_warp_floats(a.B.MP, VS, ORS) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const unsigned long long chunks =
        ((unsigned long long)a.batch + kChunk - 1) / kChunk * (unsigned long long)a.B.R;
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
