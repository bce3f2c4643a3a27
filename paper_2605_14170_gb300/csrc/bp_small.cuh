// Device code of the register-resident BP path for small codes (n <= 160,
// rows of H^(t) <= 128, check weight <= 6), shared by the single-code kernel
// (decode_small.cu) and the persistent mixed-batch kernel (decode_mixed.cu).
//
// One warp decodes one (shot, representation) pair at a time: flooding BP of
// Section II-B with the halting rule, messages in shared memory, arithmetic in
// the FP32 oracle's order.  A warp takes a chunk of consecutive shots of one
// representation, so everything fixed for the representation is loaded once:
// the shared-memory byte addresses of every variable's edges in ascending row
// order of H^(t) and the variable degrees stay in registers, the rows of H as
// bit masks over positions go to the warp's shared memory.  Variables are
// visited in degree-sorted order, 32 per step, and each step runs at the
// largest degree among its lanes (no divergence); check messages leave the
// check pass pre-signed;
// the halting test H e = s runs on ballot-packed hard decisions, a row group
// at a time.  The host places rows and variables (row index sigma(r), bank
// rotation of edge position j) to spread the variable pass over the banks.
#pragma once

#include "mbbp_internal.h"

namespace mbbp {
namespace small_bp {

constexpr unsigned kFull = 0xffffffffu;

// Shared memory of one warp (floats): K*MP messages, a zero slot (padded to
// 16 B), then the halting-test masks of its representation (VS*ORS*32 words).
__host__ __device__ constexpr int warp_floats(int MP, int VS, int ORS) {
    return 6 * MP + 4 + VS * ORS * 32;
}

__device__ __forceinline__ float phi(float x) {
    return log1pf(__fdiv_rn(2.0f, expm1f(x)));
}

// Byte address (within the dynamic shared array) of edge i of a descriptor.
__device__ __forceinline__ uint32_t addr_of(const uint4& d, int i) {
    const uint32_t w = (i < 2) ? d.y : (i < 4 ? d.z : d.w);
    return (i & 1) ? (w >> 16) : (w & 0xffffu);
}

__device__ __forceinline__ float lds(const char* smc, uint32_t off) {
    return *reinterpret_cast<const float*>(smc + off);
}
__device__ __forceinline__ void sts(char* smc, uint32_t off, float v) {
    *reinterpret_cast<float*>(smc + off) = v;
}

// Check update of one row (one row per lane) whose messages q[] were loaded
// from byte offsets cb[j] + 128 k: Eq. (2) with the syndrome sign, or the
// sum-product rule through Gallager's phi.  With TRACE and a trace pointer
// tr, every message also goes to tr[edge id], the edge id of slot
// j * MP + ((lane + rot(j)) & 31) + 32 k coming from se (the
// representation's slot-to-edge table).
template <int K, int RULE, bool REG, bool TRACE>
__device__ __forceinline__ void check_row(char* smc, const float (&q)[K], const uint32_t (&cb)[K],
                                          int k, int deg, bool valid, uint32_t sbit, float alpha,
                                          float* tr, const int32_t* se, int MP) {
    const int lane = threadIdx.x & 31;
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
            if (valid && (REG || j < deg)) {
                sts(smc, cb[j] + 128 * k, __uint_as_float(out));
                if (TRACE && tr) tr[__ldg(se + j * MP + ((lane + slot_rot(j)) & 31) + 32 * k)] = __uint_as_float(out);
            }
        }
    } else {
        float f[K];
#pragma unroll
        for (int j = 0; j < K; ++j) f[j] = (REG || j < deg) ? phi(fabsf(q[j])) : 0.0f;
        float pre = 0.0f;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            float sum = pre;
#pragma unroll
            for (int t = j + 1; t < K; ++t)
                if (REG || t < deg) sum = __fadd_rn(sum, f[t]);
            const float mag = fminf(phi(sum), MBBP_SP_MAX);
            const uint32_t out = (__float_as_uint(mag) ^ sx) ^ (__float_as_uint(q[j]) & 0x80000000u);
            if (valid && (REG || j < deg)) {
                sts(smc, cb[j] + 128 * k, __uint_as_float(out));
                if (TRACE && tr) tr[__ldg(se + j * MP + ((lane + slot_rot(j)) & 31) + 32 * k)] = __uint_as_float(out);
            }
            pre = __fadd_rn(pre, f[j]);
        }
    }
}

// Variable update (Eq. (3)): q_i = mu + the other messages of the variable in
// ascending row order of H^(t), posterior = mu + all of them.  The clamp of q
// to [-LMAX, LMAX] is not applied here because nothing observable depends on
// it: q only feeds the check rule, whose min also runs over LMAX (so
// |q| >= LMAX and LMAX give the same message and sign), and phi(|q|)
// underflows to 0 for |q| >= 104 under either value; q stays finite
// (|q| <= |mu| + 6 LMAX).
//
// The update runs for the 32 lanes of a variable step at once: DM is the largest
// degree among the step's lanes (warp-uniform).  The descriptor of a lane of
// degree deg < DM points its edges i >= deg at the warp's zero slot, so the
// lane loads +0.0 for them, which leaves every sum unchanged (x + 0 = x
// exactly for every x but -0, and no sum here is -0: they start from mu + 0
// and a sum that cancels rounds to +0); it stores only its own deg messages,
// so the zero slot stays zero.  Each lane's sums are therefore those of its
// own degree (same terms, same order, exact), while the step issues one load
// and one store instruction per edge position instead of one per degree
// case present among its lanes.
template <int DM>
__device__ __forceinline__ float var_upd_step(char* smc, const uint4& d, float mu, int deg) {
    uint32_t a[DM];
    float m[DM];
#pragma unroll
    for (int i = 0; i < DM; ++i) a[i] = addr_of(d, i);
#pragma unroll
    for (int i = 0; i < DM; ++i) m[i] = lds(smc, a[i]);
    float P[DM + 1];
    P[0] = mu;
#pragma unroll
    for (int i = 0; i < DM; ++i) P[i + 1] = __fadd_rn(P[i], m[i]);
#pragma unroll
    for (int i = 0; i < DM; ++i) {
        float q = P[i];
#pragma unroll
        for (int t = i + 1; t < DM; ++t) q = __fadd_rn(q, m[t]);
        if (i < deg) sts(smc, a[i], q);
    }
    return P[DM];
}

// The step's body by its largest degree: a chain of uniform tests, the
// common case first (measured: a six-way switch compiled to slower branches,
// 7.56 vs 8.63 M shots/s on the [[144,12,12]] workload).  Steps whose lanes
// have at most 3 edges run the degree-3 body (the missing edges read the zero
// slot, exactly as above).
__device__ __forceinline__ float var_step(char* smc, int dmax, int deg, const uint4& d, float mu) {
    if (dmax <= 3) return var_upd_step<3>(smc, d, mu, deg);
    if (dmax == 4) return var_upd_step<4>(smc, d, mu, deg);
    if (dmax == 5) return var_upd_step<5>(smc, d, mu, deg);
    return var_upd_step<6>(smc, d, mu, deg);
}

// Decode shots [shot_begin, shot_end) on representation b.  smc is the
// dynamic shared array, wbase the byte offset of this warp's area in it.
// OUT: the call asks for per-representation outputs beyond the candidates:
// io.post (posteriors) and / or io.c2v (the check messages of every
// iteration; the last one run remains); without OUT neither is written and
// the loops carry no test for them.
template <int VS, int RS, int ORS, int RULE, bool REG, bool OUT = false>
__device__ __forceinline__ void run_chunk(const DevBases& B, const ShotIO& io, int b, int shot_begin,
                                          int shot_end, char* smc, uint32_t wbase) {
    constexpr int K = 6;
    const int lane = threadIdx.x & 31;
    const int MP = B.MP, n = B.n, m = B.m, R = B.R;
    float* msg = reinterpret_cast<float*>(smc + wbase);
    uint32_t* hms = reinterpret_cast<uint32_t*>(msg + K * MP + 4);  // [VS][ORS*32]
    uint32_t cb[K];
#pragma unroll
    for (int j = 0; j < K; ++j) cb[j] = wbase + 4u * (uint32_t)(j * MP + ((lane + slot_rot(j)) & 31));
    const uint32_t wshift = wbase | (wbase << 16);
    const int Mb = __ldg(B.rows + b);
    const uint4* vd = B.vdesc2 + (size_t)b * (VS * 32);
    const uint32_t* ri = B.rinfo2 + (size_t)b * MP;
    const uint32_t* hm = B.hmask2 + (size_t)b * VS * (ORS * 32);

    __syncwarp();
    if (lane == 0) msg[K * MP] = 0.0f;
    // edge addresses of every variable (y/z/w of the descriptors) and the
    // degrees, 4 bits per variable step; variable ids are re-read from L1
    // when a shot starts and ends
    uint4 desc[VS];
    static_assert(VS <= 5 && RS <= 8, "degrees are packed 3 bits per step, twice, in 32 bits");
    // this lane's degree (bits 3k..3k+2) and the step's largest degree
    // (bits 16+3k..) of every variable step k; degrees are at most 6
    uint32_t degs = 0;
#pragma unroll
    for (int k = 0; k < VS; ++k) {
        desc[k] = __ldg(vd + 32 * k + lane);
        desc[k].y += wshift;
        desc[k].z += wshift;
        desc[k].w += wshift;
        const uint32_t dk = desc[k].x >> 16;
        degs |= (dk << (3 * k)) | (__reduce_max_sync(kFull, dk) << (16 + 3 * k));
    }
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

    // channel LLRs of this lane's variables: once per chunk when every shot
    // shares one LLR vector (llr_stride 0), else per shot
    float mu[VS];
    auto load_mu = [&](const float* llr) {
#pragma unroll
        for (int k = 0; k < VS; ++k) {
            const bool live = (32 * k + lane) < n;
            const uint32_t v = __ldg(&vd[32 * k + lane].x) & 0xffffu;
            // + 0.0f turns -0 into +0: decision-neutral, keeps -0 out of every sum
            mu[k] = live ? __fadd_rn(__ldg(llr + v), 0.0f) : 0.0f;
        }
    };
    if (io.llr_stride == 0) load_mu(io.llr);

    for (int shot = shot_begin; shot < shot_end; ++shot) {
        const unsigned long long item = (unsigned long long)shot * R + b;
        const uint8_t* sy = io.synd + (size_t)shot * m;
        float* tr = (OUT && io.c2v) ? io.c2v + item * (unsigned long long)io.c2v_stride : nullptr;
        if (io.llr_stride != 0) load_mu(io.llr + (size_t)shot * io.llr_stride);
        uint32_t ew[VS];
#pragma unroll
        for (int k = 0; k < VS; ++k) ew[k] = __ballot_sync(kFull, mu[k] < 0.f);
        uint32_t sb = 0, sbo = 0;
#pragma unroll
        for (int k = 0; k < RS; ++k)
            if (lane + 32 * k < Mb) sb |= (uint32_t)(__ldg(sy + (__ldg(ri + lane + 32 * k) & 0xffffu)) & 1u) << k;
#pragma unroll
        for (int k = 0; k < ORS; ++k)
            if (lane + 32 * k < m) sbo |= (uint32_t)(__ldg(sy + lane + 32 * k) & 1u) << k;
        __syncwarp();
        // q^(0) = mu on every edge
#pragma unroll
        for (int k = 0; k < VS; ++k) {
            const int deg = (int)((degs >> (3 * k)) & 7u);
#pragma unroll
            for (int i = 0; i < K; ++i)
                if (i < deg) sts(smc, addr_of(desc[k], i), mu[k]);
        }
        if (OUT && io.post) {
#pragma unroll
            for (int k = 0; k < VS; ++k)
                if (32 * k + lane < n) io.post[item * n + (__ldg(&vd[32 * k + lane].x) & 0xffffu)] = mu[k];
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
            if (it == io.iters) {
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
                    check_row<K, RULE, REG, OUT>(smc, q[k], cb, k, deg, valid, (sb >> k) & 1u, io.alpha, tr,
                                                   B.sedge + (size_t)b * K * MP, MP);
                }
            }
            __syncwarp();
            // variable pass
#pragma unroll
            for (int k = 0; k < VS; ++k) {
                if (32 * k < n) {
                    const int deg = (int)((degs >> (3 * k)) & 7u);
                    const float post = var_step(smc, (int)((degs >> (16 + 3 * k)) & 7u), deg, desc[k], mu[k]);
                    ew[k] = __ballot_sync(kFull, post < 0.f);
                    if (OUT && io.post && 32 * k + lane < n)
                        io.post[item * n + (__ldg(&vd[32 * k + lane].x) & 0xffffu)] = post;
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
        if (lane < W) io.cand[item * W + lane] = myword;
        if (lane == 0) {
            io.conv[item] = conv ? 1 : 0;
            if (io.iters_run) io.iters_run[item] = (uint16_t)K_run;
        }
        __syncwarp();
    }
}

}  // namespace small_bp
}  // namespace mbbp
