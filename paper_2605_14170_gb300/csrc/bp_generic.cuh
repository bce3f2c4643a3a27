// Device code of the generic BP path (any code within the library's limits),
// shared by the single-code kernel (decode.cu) and the persistent mixed-batch
// kernel (decode_mixed.cu).
//
// One warp decodes one (shot, representation) item and keeps all of its edge
// messages in shared memory: a single float per edge, which holds q_{v->c}
// after the variable pass and m_{c->v} after the check pass (each pass reads
// every message of a node before it overwrites them, and every edge belongs
// to exactly one check and one variable, so no other lane touches it).  Lanes
// own checks r = lane + 32k; edge j of check r lives at slot j * MP + r, so
// the check pass reads and writes with unit stride across the warp.
// Variables are visited in degree-sorted order so that the lanes of one step
// mostly share a degree.
//
// Arithmetic.  Every float operation is a correctly rounded intrinsic
// (__fadd_rn / __fmul_rn) in the order the oracle uses: variable sums in
// ascending row order of H^(t) excluding the own edge, sum-product phi sums
// in ascending column order excluding the own edge.  Min-sum takes its min
// over the other edges and MBBP_LMAX from prefix and suffix minima (exact),
// then one correctly rounded alpha product per edge.  Signs come from the
// sign bits: the LLRs enter as mu + 0 (turning -0 into +0) and every q is a
// sum that starts from mu, so no q is -0 and its sign bit is set exactly
// when q < 0, the oracle's sign rule.  Hence normalized min-sum reproduces
// the FP32 oracle bit for bit; sum-product differs only through
// expm1f/log1pf.
#pragma once

#include "mbbp_internal.h"

namespace mbbp {
namespace generic_bp {

constexpr unsigned kFull = 0xffffffffu;

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
// sum-product rule) from its incoming messages q[0..deg) (q[j] = MBBP_LMAX
// for j >= deg); writes the deg outgoing messages to slots j * MP + r.
template <int DC, int RULE>
__device__ __forceinline__ void check_out(const float (&q)[DC], float* msg, int r, int MP, int deg,
                                          uint32_t sbit, float alpha) {
    if (RULE == MBBP_RULE_NMS) {
        // sign parity of the row (syndrome bit included) from the sign bits
        uint32_t sx = sbit << 31;
#pragma unroll
        for (int j = 0; j < DC; ++j) sx ^= __float_as_uint(q[j]);
        sx &= 0x80000000u;
        // min over the other edges and LMAX: prefix and suffix minima
        float pre[DC], suf[DC];
        pre[0] = MBBP_LMAX;
#pragma unroll
        for (int j = 1; j < DC; ++j) pre[j] = fminf(pre[j - 1], fabsf(q[j - 1]));
        suf[DC - 1] = MBBP_LMAX;
#pragma unroll
        for (int j = DC - 2; j >= 0; --j)
            suf[j] = (j == DC - 2) ? fabsf(q[DC - 1]) : fminf(suf[j + 1], fabsf(q[j + 1]));
#pragma unroll
        for (int j = 0; j < DC; ++j) {
            if (j < deg) {
                const float excl = (j == DC - 1) ? pre[j] : (j == 0 ? fminf(MBBP_LMAX, suf[0]) : fminf(pre[j], suf[j]));
                const uint32_t mag = __float_as_uint(__fmul_rn(alpha, excl));
                msg[j * MP + r] = __uint_as_float(mag ^ ((sx ^ __float_as_uint(q[j])) & 0x80000000u));
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

// Flooding check pass of row r: its q messages are in its own slots.  With
// a trace pointer tr, the row's new messages also go to tr[0..deg) (edge j of
// the row is its j-th column in ascending order).
template <int DC, int RULE>
__device__ __forceinline__ void check_row(float* msg, int r, int MP, int deg, uint32_t sbit,
                                          float alpha, float* tr = nullptr) {
    float q[DC];
#pragma unroll
    for (int j = 0; j < DC; ++j) q[j] = (j < deg) ? msg[j * MP + r] : MBBP_LMAX;
    check_out<DC, RULE>(q, msg, r, MP, deg, sbit, alpha);
    if (tr) {
#pragma unroll
        for (int j = 0; j < DC; ++j)
            if (j < deg) tr[j] = msg[j * MP + r];
    }
}

// Variable-node update of a degree-D variable (Eq. (3)): q_i = mu + sum of
// the other messages in ascending row order; returns the posterior.  The
// clamp of q to [-LMAX, LMAX] is not applied because nothing observable
// depends on it: q only feeds the check rule, whose min also runs over LMAX
// (so |q| >= LMAX and LMAX give the same message and sign), and phi(|q|)
// underflows to 0 for |q| >= 104 under either value; q stays finite
// (|q| <= |mu| + 12 LMAX).
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
        msg[s[i]] = q;
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

// Byte offset of slot i (0..5) of a packed width-6 descriptor (vdesc6).
__device__ __forceinline__ uint32_t packed_off(const uint4& d, int i) {
    const uint32_t w = (i < 2) ? d.y : (i < 4 ? d.z : d.w);
    return (i & 1) ? (w >> 16) : (w & 0xffffu);
}

__device__ __forceinline__ float& msg_at(float* msg, uint32_t byte_off) {
    return *reinterpret_cast<float*>(reinterpret_cast<char*>(msg) + byte_off);
}

// var_update with the slots taken from a packed descriptor: the same sums in
// the same order, without the slot-list load.
template <int D>
__device__ __forceinline__ float var_update_packed(float* msg, const uint4& d, float mu) {
    uint32_t a[D];
    float m[D];
#pragma unroll
    for (int i = 0; i < D; ++i) a[i] = packed_off(d, i);
#pragma unroll
    for (int i = 0; i < D; ++i) m[i] = msg_at(msg, a[i]);
    float P[D + 1];
    P[0] = mu;
#pragma unroll
    for (int i = 0; i < D; ++i) P[i + 1] = __fadd_rn(P[i], m[i]);
#pragma unroll
    for (int i = 0; i < D; ++i) {
        float q = P[i];
#pragma unroll
        for (int k = i + 1; k < D; ++k) q = __fadd_rn(q, m[k]);
        msg_at(msg, a[i]) = q;
    }
    return P[D];
}

__device__ __forceinline__ float var_dispatch_packed(int deg, float* msg, const uint4& d, float mu) {
    switch (deg) {
        case 1: return var_update_packed<1>(msg, d, mu);
        case 2: return var_update_packed<2>(msg, d, mu);
        case 3: return var_update_packed<3>(msg, d, mu);
        case 4: return var_update_packed<4>(msg, d, mu);
        case 5: return var_update_packed<5>(msg, d, mu);
        case 6: return var_update_packed<6>(msg, d, mu);
        default: return mu;
    }
}


// A "group" of G warps decodes one item together (G = 1: one warp).  Its
// threads synchronise on named barrier `bar` (bar.sync / bar.red with the
// group's thread count), which only its own 32 G threads use.
template <int G>
__device__ __forceinline__ void gsync(int bar) {
    if constexpr (G == 1) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(32 * G) : "memory");
    }
}

// AND of p over the group's threads (all of them must call it).
template <int G>
__device__ __forceinline__ bool gall(bool p, int bar) {
    if constexpr (G == 1) {
        return __all_sync(kFull, p);
    } else {
        uint32_t r;
        asm volatile(
            "{\n\t.reg .pred pi, po;\n\t"
            "setp.ne.u32 pi, %1, 0;\n\t"
            "bar.red.and.pred po, %2, %3, pi;\n\t"
            "selp.u32 %0, 1, 0, po;\n\t}"
            : "=r"(r)
            : "r"((uint32_t)p), "r"(bar), "r"(32 * G)
            : "memory");
        return r != 0;
    }
}

// Bit-pack the hard decision eh[0..n) into the candidate words of `item`,
// and store the convergence flag and iteration count.
__device__ __forceinline__ void store_item(const ShotIO& io, unsigned long long item, int n, int W,
                                           const uint8_t* eh, bool conv, int K) {
    const int lane = threadIdx.x & 31;
    uint32_t myword = 0;
    for (int w = 0; w < W; ++w) {
        const int v = 32 * w + lane;
        const uint32_t bit = (v < n) ? (uint32_t)eh[v] : 0u;
        const uint32_t word = __ballot_sync(kFull, bit);
        if ((w & 31) == lane) myword = word;
        if ((w & 31) == 31 || w == W - 1) {
            const int base = w & ~31;
            if (base + lane <= w) io.cand[item * W + base + lane] = myword;
        }
    }
    if (lane == 0) {
        io.conv[item] = conv ? 1 : 0;
        if (io.iters_run) io.iters_run[item] = (uint16_t)K;
    }
}

// store_item for a group of G > 1 warps: warp wig of the group packs the
// words wig, wig + G, ...
template <int G>
__device__ __forceinline__ void store_item_group(const ShotIO& io, unsigned long long item, int n, int W,
                                                 const uint8_t* eh, bool conv, int K, int wig) {
    const int lane = threadIdx.x & 31;
    for (int w = wig; w < W; w += G) {
        const int v = 32 * w + lane;
        const uint32_t word = __ballot_sync(kFull, v < n && eh[v]);
        if (lane == 0) io.cand[item * W + w] = word;
    }
    if (wig == 0 && lane == 0) {
        io.conv[item] = conv ? 1 : 0;
        if (io.iters_run) io.iters_run[item] = (uint16_t)K;
    }
}

// Decode one (shot, representation) item.  area: the shared-memory area of
// the warp (G = 1) or group of G warps that decodes it (warp_layout(DC,
// ...).per_warp bytes); hcol: columns of the rows of H ([DC][mpad], shared
// or global memory).  A group's threads own rows gt, gt + 32 G, ... and
// variable positions likewise (gt: the thread's index in the group) and meet
// on named barrier `bar` between passes; the arithmetic of every row and
// variable is the same whatever G.  TRACE: io.c2v receives the check
// messages of every iteration (the last one run remains).
template <int DC, int DV, int RULE, bool TRACE = false, int G = 1>
__device__ __forceinline__ void run_item(const DevBases& B, const ShotIO& io, int shot, int b,
                                         unsigned char* area, const uint16_t* hcol, int bar = 0) {
    constexpr int GT = 32 * G;
    const int lane = (int)(threadIdx.x % GT);  // the thread's index in its group
    const int MP = B.MP, n = B.n, m = B.m, R = B.R, W = B.W, mpad = B.mpad;
    const WarpLayout L = warp_layout(DC, MP, mpad, n);
    float* msg = reinterpret_cast<float*>(area);
    float* mu_s = msg + L.S;
    uint8_t* eh = reinterpret_cast<uint8_t*>(mu_s + L.npad);
    const int row_steps = (MP + GT - 1) / GT;
    const int orow_steps = (mpad + GT - 1) / GT;
    const unsigned long long item = (unsigned long long)shot * R + b;
    const uint32_t* rinfo = B.rowinfo + (size_t)b * MP;
    const uint2* vd = B.vdesc + (size_t)b * n;
    const int Mb = __ldg(B.rows + b);
    const float* llr = io.llr + (size_t)shot * io.llr_stride;
    const uint8_t* sy = io.synd + (size_t)shot * m;

    gsync<G>(bar);
    // channel LLRs, hard decision of the LLRs, syndrome bits of my rows
    for (int v = lane; v < n; v += GT) {
        const float x = __ldg(llr + v);
        mu_s[v] = __fadd_rn(x, 0.0f);  // -0 -> +0 (sign bits decide the check rule)
        eh[v] = (x < 0.f) ? 1 : 0;
    }
    if (lane == 0) eh[n] = 0;  // padding column of hcol
    uint32_t sb = 0;
    for (int k = 0; k < row_steps; ++k) {
        const int r = lane + GT * k;
        if (r < Mb) sb |= (uint32_t)(__ldg(sy + (__ldg(rinfo + r) & 0xffffu)) & 1u) << k;
    }
    gsync<G>(bar);
    // q^(0)_{v->c} = mu_v
    if constexpr (DC == 6) {
        const uint4* vd6 = B.vdesc6 + (size_t)b * n;
        for (int p = lane; p < n; p += GT) {
            const uint4 d = __ldg(vd6 + p);
            const int v = d.x & 0xffff, deg = (int)(d.x >> 16);
            const float x = mu_s[v];
#pragma unroll
            for (int i = 0; i < 6; ++i)
                if (i < deg) msg_at(msg, packed_off(d, i)) = x;
            if (io.post) io.post[item * n + v] = x;
        }
    } else {
        for (int p = lane; p < n; p += GT) {
            const uint2 d = __ldg(vd + p);
            const int v = d.y & 0xffff, deg = (int)(d.y >> 16);
            const float x = mu_s[v];
            for (int i = 0; i < deg; ++i) msg[__ldg(B.vslot + d.x + i)] = x;
            if (io.post) io.post[item * n + v] = x;
        }
    }
    gsync<G>(bar);

    int K = 0;
    bool conv = false;
    int kf = 0;  // the row group whose test failed last (group-uniform)
    for (int it = 0;; ++it) {
        // halting rule: H e = s on the rows of H (the extra rows are copies).
        // One row group at a time until one fails, starting with the group
        // that failed at the previous test: near convergence the same few
        // checks stay unsatisfied, so one group usually decides
        bool ok = true;
        for (int s = 0; s < orow_steps; ++s) {
            const int k = (kf + s < orow_steps) ? kf + s : kf + s - orow_steps;
            const int r = lane + GT * k;
            bool gok = true;
            if (r < m) {
                uint32_t par = (sb >> k) & 1u;
#pragma unroll
                for (int j = 0; j < DC; ++j) par ^= eh[hcol[j * mpad + r]];
                gok = (par == 0u);
            }
            if (!gall<G>(gok, bar)) {  // group-uniform
                ok = false;
                kf = k;
                break;
            }
        }
        if (ok) {
            conv = true;
            K = it;
            break;
        }
        if (it == io.iters) {
            K = it;
            break;
        }
        // check pass
        for (int k = 0; k < row_steps; ++k) {
            const int r = lane + GT * k;
            if (r < Mb) {
                const int deg = B.regular ? DC : (int)((__ldg(rinfo + r) >> 16) & 0xffu);
                float* tr = TRACE ? io.c2v + item * (unsigned long long)io.c2v_stride +
                                        __ldg(B.rowptr + (size_t)b * MP + r)
                                  : nullptr;
                check_row<DC, RULE>(msg, r, MP, deg, (sb >> k) & 1u, io.alpha, tr);
            }
        }
        gsync<G>(bar);
        // variable pass, posterior, hard decision; each step's descriptor is
        // loaded one step ahead (width 6: with the slots packed in, so no load
        // of the pass waits on L1; other widths: the slot list still does)
        if constexpr (DC == 6) {
            const uint4* vd6 = B.vdesc6 + (size_t)b * n;
            uint4 dn = (lane < n) ? __ldg(vd6 + lane) : make_uint4(0u, 0u, 0u, 0u);
            for (int p = lane; p < n; p += GT) {
                const uint4 d = dn;
                if (p + GT < n) dn = __ldg(vd6 + p + GT);
                const int v = d.x & 0xffff, deg = (int)(d.x >> 16);
                const float post = var_dispatch_packed(deg, msg, d, mu_s[v]);
                eh[v] = (post < 0.f) ? 1 : 0;
                if (io.post) io.post[item * n + v] = post;
            }
        } else {
            uint2 dn = (lane < n) ? __ldg(vd + lane) : make_uint2(0u, 0u);
            for (int p = lane; p < n; p += GT) {
                const uint2 d = dn;
                if (p + GT < n) dn = __ldg(vd + p + GT);
                const int v = d.y & 0xffff, deg = (int)(d.y >> 16);
                const float post = var_dispatch<1, DV>(deg, msg, B.vslot + d.x, mu_s[v]);
                eh[v] = (post < 0.f) ? 1 : 0;
                if (io.post) io.post[item * n + v] = post;
            }
        }
        gsync<G>(bar);
    }
    // candidate e_t (bit-packed), convergence flag, iterations
    if constexpr (G == 1)
        store_item(io, item, n, W, eh, conv, K);
    else
        store_item_group<G>(io, item, n, W, eh, conv, K, lane >> 5);
    gsync<G>(bar);
}

// Per-warp shared memory of the serial schedule: the flooding layout plus
// the syndrome bits of the rows of H^(t) (MP / 32 words).
__host__ __device__ __forceinline__ int serial_warp_bytes(int DC, int MP, int mpad, int n) {
    return warp_layout(DC, MP, mpad, n).per_warp + align16(MP / 8);
}

// Decode one (shot, representation) item with the serial schedule.  The
// edge slots hold m_{c->v} for the whole decode.  Within a layer the rows
// share no variable: lane-parallel rows read only messages of other layers'
// rows (through their variables) and write only their own slots, so the
// layer's result is that of visiting its rows one by one.  q_{v->c} is
// mu_v plus v's other messages in ascending row order (the slot list of v
// is sorted that way), clamped, exactly as the oracle forms it.
template <int DC, int DV, int RULE>
__device__ __forceinline__ void run_item_serial(const DevBases& B, const ShotIO& io, int shot, int b,
                                                unsigned char* area, const uint16_t* hcol) {
    const int lane = threadIdx.x & 31;
    const int MP = B.MP, n = B.n, m = B.m, R = B.R, W = B.W, mpad = B.mpad;
    const WarpLayout L = warp_layout(DC, MP, mpad, n);
    float* msg = reinterpret_cast<float*>(area);
    float* mu_s = msg + L.S;
    uint8_t* eh = reinterpret_cast<uint8_t*>(mu_s + L.npad);
    uint32_t* sbits = reinterpret_cast<uint32_t*>(area + L.per_warp);
    const int row_steps = MP >> 5;
    const int orow_steps = mpad >> 5;
    const unsigned long long item = (unsigned long long)shot * R + b;
    const uint32_t* rinfo = B.rowinfo + (size_t)b * MP;
    const uint2* vd = B.vdesc + (size_t)b * n;
    const uint16_t* lrows = B.lrows + (size_t)b * MP;
    const uint16_t* lptr = B.lptr + (size_t)b * (MP + 1);
    const uint2* ev = B.evar + (size_t)b * DC * MP;
    const int nl = __ldg(B.nlayers + b);
    const int Mb = __ldg(B.rows + b);
    const float* llr = io.llr + (size_t)shot * io.llr_stride;
    const uint8_t* sy = io.synd + (size_t)shot * m;

    __syncwarp();
    for (int v = lane; v < n; v += 32) {
        const float x = __ldg(llr + v);
        mu_s[v] = __fadd_rn(x, 0.0f);  // -0 -> +0 (sign bits decide the check rule)
        eh[v] = (x < 0.f) ? 1 : 0;
        if (io.post) io.post[item * n + v] = x;
    }
    if (lane == 0) eh[n] = 0;
    for (int i = lane; i < L.S; i += 32) msg[i] = 0.0f;  // m^(0)_{c->v} = 0
    uint32_t sb = 0;  // syndrome bits of the rows lane + 32k (halting test)
    for (int k = 0; k < row_steps; ++k) {
        const int r = lane + 32 * k;
        const uint32_t bit = (r < Mb) ? (uint32_t)(__ldg(sy + (__ldg(rinfo + r) & 0xffffu)) & 1u) : 0u;
        sb |= bit << k;
        const uint32_t word = __ballot_sync(kFull, bit);
        if (lane == 0) sbits[k] = word;
    }
    __syncwarp();

    int K = 0;
    bool conv = false;
    for (int it = 0;; ++it) {
        bool ok = true;  // halting rule, first row group first (as in run_item)
        for (int k = 0; k < orow_steps; ++k) {
            const int r = lane + 32 * k;
            if (r < m) {
                uint32_t par = (sb >> k) & 1u;
#pragma unroll
                for (int j = 0; j < DC; ++j) par ^= eh[hcol[j * mpad + r]];
                ok = ok && (par == 0u);
            }
            if (k == 0 && orow_steps > 1) {  // warp-uniform condition
                const bool first_ok = __all_sync(kFull, ok);
                if (!first_ok) break;
            }
        }
        if (__all_sync(kFull, ok)) {
            conv = true;
            K = it;
            break;
        }
        if (it == io.iters) {
            K = it;
            break;
        }
        for (int l = 0; l < nl; ++l) {
            const int i1 = __ldg(lptr + l + 1);
            for (int idx = __ldg(lptr + l) + lane; idx < i1; idx += 32) {
                const int r = __ldg(lrows + idx);
                const int deg = B.regular ? DC : (int)((__ldg(rinfo + r) >> 16) & 0xffu);
                float q[DC];
#pragma unroll
                for (int j = 0; j < DC; ++j) {
                    q[j] = MBBP_LMAX;
                    if (j < deg) {
                        const int slot = j * MP + r;
                        const uint2 e = __ldg(ev + slot);
                        const int dv = (int)(e.y >> 16);
                        float x = mu_s[e.y & 0xffffu];
#pragma unroll
                        for (int i = 0; i < DV; ++i) {
                            if (i < dv) {
                                const int sl = __ldg(B.vslot + e.x + i);
                                if (sl != slot) x = __fadd_rn(x, msg[sl]);
                            }
                        }
                        q[j] = x;  // unclamped, as in var_update
                    }
                }
                check_out<DC, RULE>(q, msg, r, MP, deg, (sbits[r >> 5] >> (r & 31)) & 1u, io.alpha);
            }
            __syncwarp();
        }
        // posterior mu_v + all messages of v (ascending row), hard decision
        for (int p = lane; p < n; p += 32) {
            const uint2 d = __ldg(vd + p);
            const int v = d.y & 0xffff, deg = (int)(d.y >> 16);
            float P = mu_s[v];
            for (int i = 0; i < deg; ++i) P = __fadd_rn(P, msg[__ldg(B.vslot + d.x + i)]);
            eh[v] = (P < 0.f) ? 1 : 0;
            if (io.post) io.post[item * n + v] = P;
        }
        __syncwarp();
    }
    store_item(io, item, n, W, eh, conv, K);
    __syncwarp();
}

// Dispatch on the kernel width of a representation set.
template <int RULE>
__device__ __forceinline__ void run_item_any(const DevBases& B, const ShotIO& io, int shot, int b,
                                             unsigned char* area, const uint16_t* hcol) {
    if (B.DC == 6) run_item<6, 6, RULE>(B, io, shot, b, area, hcol);
    else if (B.DC == 8) run_item<8, 8, RULE>(B, io, shot, b, area, hcol);
    else run_item<12, 12, RULE>(B, io, shot, b, area, hcol);
}

}  // namespace generic_bp
}  // namespace mbbp
