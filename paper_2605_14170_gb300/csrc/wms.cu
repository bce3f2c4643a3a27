// Differentiable weighted min-sum (WMS): the normalized min-sum of Section
// II-B (Eq. (2)-(3)) with a weight w and a damping factor g per edge and per
// iteration of every representation H^(t), unrolled for T flooding
// iterations; w == alpha, g == 0 is normalized min-sum:
//   m^(t)_e = g^(t)_e m^(t-1)_e + (1 - g^(t)_e) w^(t)_e S_e mn_e,
//   S_e = (-1)^{s_c} prod_{other e' of c} sign(q^(t-1)_e'),
//   mn_e = min(LMAX, min_{other e' of c} |q^(t-1)_e'|),
//   q^(t)_e = mu_v + sum_{other e' of v} m^(t)_e',  m^(0) = 0, q^(0) = mu.
// Loss of an item: scale * sum_v BCE(sigmoid(-post_v), e_v), post = mu + sum m^(T),
// or (all_iters) the mean of that over the posteriors of iterations 1..T.
//
// Kernels (generic slot layout; the backward pass one warp per (shot,
// representation), the forward pass G warps per item, G in {1, 2, 4}):
//   wms_forward   T iterations, posterior, loss, a checkpoint of m every
//                 `ckpt` iterations; or, in decode mode, the halting rule
//                 after every iteration and the candidate for FWS
//                 (iterations past T reuse the weights of iteration T),
//                 with w and g rearranged by wms_pack beforehand into the
//                 message layout;
//   wms_backward  segment by segment from the last checkpoint: recompute the
//                 segment's forward states, then the adjoint through it
//                 (the min's derivative goes to the arg-min edge, lowest index
//                 on ties; the sign's derivative is 0); parameter gradients are
//                 added to gw / gg with atomics;
//   adam_step     Adam update of the parameters, clamped to [lo, hi].
#include "bp_generic.cuh"

namespace mbbp {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWmsWarps = 8;       // largest block (warps); the launch picks the block size
constexpr int kWmsStateWarps = 4;  // warps whose segment states must fit for the shared-memory path

struct WmsLayout {
    int S, npad;
    size_t fwd_bytes, bwd_bytes;
};

__host__ __device__ inline WmsLayout wms_layout(int DC, int MP, int n, int ckpt) {
    WmsLayout L;
    L.S = DC * MP;
    L.npad = (n + 4) & ~3;
    // forward: m, q (S each), mu, post (npad each: n, a padding column)
    L.fwd_bytes = (size_t)(2 * L.S + 2 * L.npad) * 4;
    // backward: q, gm (updated in place from dL/dm^(t) to dL/dm^(t-1)), gq
    // (S each), mu (npad); the segment's states follow in shared memory or
    // live in a per-warp global buffer of ckpt * S floats
    L.bwd_bytes = (size_t)(3 * L.S + L.npad) * 4;
    return L;
}

// One variable of degree D from a packed width-6 descriptor: q_i = mu + the
// other messages in ascending row order, as prefix sums P_i = mu + m_0 + ...
// + m_{i-1} and q_i = P_i + m_{i+1} + ... (term for term the same sums);
// returns the posterior P_D.  m and q share the slot layout.
template <int D>
__device__ __forceinline__ float wms_var_packed(const float* m, float* q, const uint4& d, float mu) {
    uint32_t s[D];
    float mv[D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
        s[i] = generic_bp::packed_off(d, i);
        mv[i] = generic_bp::msg_at(const_cast<float*>(m), s[i]);
    }
    float P[D + 1];
    P[0] = mu;
#pragma unroll
    for (int i = 0; i < D; ++i) P[i + 1] = __fadd_rn(P[i], mv[i]);
#pragma unroll
    for (int i = 0; i < D; ++i) {
        float x = P[i];
#pragma unroll
        for (int k = i + 1; k < D; ++k) x = __fadd_rn(x, mv[k]);
        generic_bp::msg_at(q, s[i]) = x;
    }
    return P[D];
}

__device__ __forceinline__ float wms_var_dispatch(int deg, const float* m, float* q, const uint4& d, float mu) {
    switch (deg) {
        case 1: return wms_var_packed<1>(m, q, d, mu);
        case 2: return wms_var_packed<2>(m, q, d, mu);
        case 3: return wms_var_packed<3>(m, q, d, mu);
        case 4: return wms_var_packed<4>(m, q, d, mu);
        case 5: return wms_var_packed<5>(m, q, d, mu);
        case 6: return wms_var_packed<6>(m, q, d, mu);
        default: return mu;
    }
}

// q^(t)_e and the posterior from m (variable pass, ascending row order).
// Each step's descriptor is loaded one step ahead; a variable's slots and
// messages are read once into registers (at most DV of them).  G warps
// share the item: the thread with group index gt takes positions gt,
// gt + 32 G, ...
template <int DV, int G = 1>
__device__ __forceinline__ void wms_var_pass(const DevBases& B, int b, const uint2* vd, const float* m,
                                             float* q, const float* mu, float* post) {
    constexpr int GT = 32 * G;
    const int lane = (int)(threadIdx.x % GT);
    const int n = B.n;
    if constexpr (DV == 6) {
        // width 6: the slots come packed in the descriptor (vdesc6), no
        // slot-list load; the body is chosen by the variable's degree (the
        // degree-sorted order keeps a warp's lanes on one case)
        const uint4* vd6 = B.vdesc6 + (size_t)b * n;
        uint4 dn = (lane < n) ? __ldg(vd6 + lane) : make_uint4(0u, 0u, 0u, 0u);
        for (int p = lane; p < n; p += GT) {
            const uint4 d = dn;
            if (p + GT < n) dn = __ldg(vd6 + p + GT);
            const int v = d.x & 0xffff, deg = (int)(d.x >> 16);
            const float pv = wms_var_dispatch(deg, m, q, d, mu[v]);
            if (post) post[v] = pv;
        }
        return;
    }
    uint2 dn = (lane < n) ? __ldg(vd + lane) : make_uint2(0u, 0u);
    for (int p = lane; p < n; p += GT) {
        const uint2 d = dn;
        if (p + GT < n) dn = __ldg(vd + p + GT);
        const int v = d.y & 0xffff, deg = (int)(d.y >> 16);
        const uint16_t* sl = B.vslot + d.x;
        int s[DV];
        float mv[DV];
#pragma unroll
        for (int i = 0; i < DV; ++i) {
            s[i] = (i < deg) ? (int)__ldg(sl + i) : 0;
            mv[i] = (i < deg) ? m[s[i]] : 0.0f;
        }
        float P[DV + 1];  // prefix sums, as in the packed branch
        P[0] = mu[v];
#pragma unroll
        for (int i = 0; i < DV; ++i) P[i + 1] = (i < deg) ? __fadd_rn(P[i], mv[i]) : P[i];
        if (post) post[v] = P[DV];
#pragma unroll
        for (int i = 0; i < DV; ++i) {
            if (i < deg) {
                float x = P[i];
#pragma unroll
                for (int k = i + 1; k < DV; ++k)
                    if (k < deg) x = __fadd_rn(x, mv[k]);
                q[s[i]] = x;
            }
        }
    }
}

// One WMS check pass: m <- g m + (1 - g) w S mn(q).  wt, gt: parameters of
// this iteration for representation b ([E] in row-major edge order); or,
// with SLOT, wt points at the iteration's (w, g) pairs in the message layout
// (pair of edge j of row r at float2 index j * MP + r: one coalesced load
// per edge).  With G warps per item the thread with group index gt takes
// rows gt, gt + 32 G, ...; bit k of sb is the syndrome bit of its k-th row.
template <int DC, int G = 1, bool SLOT = false>
__device__ __forceinline__ void wms_check_pass(const DevBases& B, int b, const uint32_t* rinfo,
                                               int Mb, uint32_t sb, const float* q, float* m,
                                               const float* wt, const float* gt) {
    constexpr int GT = 32 * G;
    const int lane = (int)(threadIdx.x % GT);
    const int MP = B.MP;
    const int32_t* rp = B.rowptr + (size_t)b * MP;
    for (int k = 0; k < (MP + GT - 1) / GT; ++k) {
        const int r = lane + GT * k;
        if (r >= Mb) continue;
        const int deg = B.regular ? DC : (int)((__ldg(rinfo + r) >> 16) & 0xffu);
        const int e0 = SLOT ? 0 : __ldg(rp + r);
        float qq[DC];
#pragma unroll
        for (int j = 0; j < DC; ++j) qq[j] = (j < deg) ? q[j * MP + r] : MBBP_LMAX;
        // the min over the other edges (and LMAX) from prefix and suffix
        // minima, the sign parity from the sign bits (no q is -0: the LLRs
        // enter as mu + 0), both exact
        uint32_t sx = ((sb >> k) & 1u) << 31;
#pragma unroll
        for (int j = 0; j < DC; ++j) sx ^= __float_as_uint(qq[j]);
        sx &= 0x80000000u;
        float pre[DC], suf[DC];
        pre[0] = MBBP_LMAX;
#pragma unroll
        for (int j = 1; j < DC; ++j) pre[j] = fminf(pre[j - 1], fabsf(qq[j - 1]));
        suf[DC - 1] = MBBP_LMAX;
#pragma unroll
        for (int j = DC - 2; j >= 0; --j)
            suf[j] = (j == DC - 2) ? fabsf(qq[DC - 1]) : fminf(suf[j + 1], fabsf(qq[j + 1]));
#pragma unroll
        for (int j = 0; j < DC; ++j) {
            if (j >= deg) continue;
            const float mn = (j == DC - 1) ? pre[j] : (j == 0 ? fminf(MBBP_LMAX, suf[0]) : fminf(pre[j], suf[j]));
            const float smn = __uint_as_float(__float_as_uint(mn) ^ ((sx ^ __float_as_uint(qq[j])) & 0x80000000u));
            float wj, gg;
            if constexpr (SLOT) {
                const float2 p = __ldg(reinterpret_cast<const float2*>(wt) + j * MP + r);
                wj = p.x;
                gg = p.y;
            } else {
                wj = __ldg(wt + e0 + j);
                gg = __ldg(gt + e0 + j);
            }
            const float c = __fmul_rn(wj, smn);
            const float mo = m[j * MP + r];
            m[j * MP + r] = __fadd_rn(__fmul_rn(gg, mo), __fmul_rn(__fsub_rn(1.0f, gg), c));
        }
    }
}

__device__ __forceinline__ float bce_neg_sigmoid(float post, int e) {
    const float x = e ? post : -post;
    return x > 0.f ? x + log1pf(expf(-x)) : log1pf(expf(x));
}

// G warps decode each item together (G = 1: one warp per item; G > 1 for
// codes whose two message arrays per item, not registers, limit the resident
// warps).  Group g of the block uses named barrier 1 + g; the arithmetic of
// every row and variable is the same whatever G.  The hard decisions are the
// posteriors' sign bits (no posterior is -0: it is a sum that starts from
// mu, and mu enters as llr + 0).  The arguments come by value (taken by
// reference from the kernel's parameter, the decode on a length-882 code
// measured 5% slower).
template <int DC, int DV, int G>
__device__ __forceinline__ void wms_forward_items(const WmsArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long group_item[kWmsWarps];
    __shared__ float group_part[kWmsWarps];
    constexpr int GT = 32 * G;
    const DevBases& B = a.B;
    const int lane = (int)(threadIdx.x % GT);  // the thread's index in its group
    const int wig = lane >> 5;                  // the warp's index in its group
    const int grp = (int)(threadIdx.x >> 5) / G;
    const int bar = 1 + grp;
    const int MP = B.MP, n = B.n, m_rows = B.m, R = B.R, W = B.W;
    const WmsLayout L = wms_layout(DC, MP, n, a.ckpt);
    float* m = reinterpret_cast<float*>(smem + grp * L.fwd_bytes);
    float* q = m + L.S;
    float* mu = q + L.S;
    float* post = mu + L.npad;  // post[n] = +0: the padding column of hcol
    const int orow_steps = (B.mpad + GT - 1) / GT;
    const int row_steps = (MP + GT - 1) / GT;
    // H's columns for the halting test, once per block
    uint16_t* hcol_s = reinterpret_cast<uint16_t*>(smem + (blockDim.x / GT) * L.fwd_bytes);
    if (a.decode) {
        for (int i = threadIdx.x; i < DC * B.mpad; i += blockDim.x) hcol_s[i] = __ldg(B.hcol + i);
        __syncthreads();
    }
    // work items representation-major (g = b * batch + shot): the warps
    // resident at one time share a representation's tables in L1; outputs
    // stay indexed by item = shot * R + b
    const unsigned long long batch = a.total_items / (unsigned long long)R;
    for (;;) {
        unsigned long long g = 0;
        if constexpr (G == 1) {
            if (lane == 0) g = atomicAdd(a.counter, 1ull);
            g = __shfl_sync(kFull, g, 0);
        } else {
            // rewritten only after the item's last barrier, which every reader passed
            if (lane == 0) group_item[grp] = atomicAdd(a.counter, 1ull);
            generic_bp::gsync<G>(bar);
            g = group_item[grp];
        }
        if (g >= a.total_items) break;
        const int b = (int)(g / batch);
        const int shot = (int)(g - (unsigned long long)b * batch);
        const unsigned long long item = (unsigned long long)shot * R + b;
        const uint32_t* rinfo = B.rowinfo + (size_t)b * MP;
        const uint2* vd = B.vdesc + (size_t)b * n;
        const int Mb = __ldg(B.rows + b);
        const float* llr = a.llr + (size_t)shot * a.llr_stride;
        const uint8_t* sy = a.synd + (size_t)shot * m_rows;
        for (int v = lane; v < n; v += GT) {
            const float x = __fadd_rn(__ldg(llr + v), 0.0f);  // -0 -> +0 (sign bits decide the check rule)
            mu[v] = x;
            post[v] = x;
        }
        if (lane == 0) post[n] = 0.0f;
        for (int i = lane; i < L.S; i += GT) m[i] = 0.0f;
        uint32_t sb = 0;
        for (int k = 0; k < row_steps; ++k) {
            const int r = lane + GT * k;
            if (r < Mb) sb |= (uint32_t)(__ldg(sy + (__ldg(rinfo + r) & 0xffffu)) & 1u) << k;
        }
        generic_bp::gsync<G>(bar);
        for (int p = lane; p < n; p += GT) {  // q^(0) = mu
            const uint2 d = __ldg(vd + p);
            const int v = d.y & 0xffff, deg = (int)(d.y >> 16);
            for (int i = 0; i < deg; ++i) q[__ldg(B.vslot + d.x + i)] = mu[v];
        }
        generic_bp::gsync<G>(bar);
        int K = 0;
        bool conv = false;
        float lacc = 0.f;  // this lane's BCE of the posteriors of iterations 1..T-1 (all_iters)
        const int iters = a.decode ? a.iters : a.T;
        for (int it = 0;; ++it) {
            if (a.decode) {
                // the first row group decides most unconverged iterations,
                // so the other groups are tested only if it passed
                bool ok = true;
                for (int k = 0; k < orow_steps; ++k) {
                    const int r = lane + GT * k;
                    if (r < m_rows) {
                        uint32_t par = (sb >> k) & 1u;
#pragma unroll
                        for (int j = 0; j < DC; ++j) par ^= __float_as_uint(post[hcol_s[j * B.mpad + r]]) >> 31;
                        ok = ok && (par == 0u);
                    }
                    if (k == 0 && orow_steps > 1 && !generic_bp::gall<G>(ok, bar)) break;  // group-uniform
                }
                if (generic_bp::gall<G>(ok, bar)) {
                    conv = true;
                    K = it;
                    break;
                }
            }
            if (it == iters) {
                K = it;
                break;
            }
            const int tp = min(it, a.T - 1);  // iterations past T reuse the last weights
            if (a.wg) {
                const float2* wgt = a.wg + ((size_t)b * a.T + tp) * DC * MP;
                wms_check_pass<DC, G, true>(B, b, rinfo, Mb, sb, q, m, reinterpret_cast<const float*>(wgt),
                                            nullptr);
            } else {
                const float* wt = a.w + ((size_t)b * a.T + tp) * a.E;
                const float* gt = a.g + ((size_t)b * a.T + tp) * a.E;
                wms_check_pass<DC, G>(B, b, rinfo, Mb, sb, q, m, wt, gt);
            }
            generic_bp::gsync<G>(bar);
            wms_var_pass<DV, G>(B, b, vd, m, q, mu, post);
            generic_bp::gsync<G>(bar);
            if (!a.decode) {
                if (a.ckpt_buf && (it + 1) % a.ckpt == 0 && it + 1 < a.T) {
                    float* dst = a.ckpt_buf + ((size_t)item * a.nckpt + ((it + 1) / a.ckpt - 1)) * L.S;
                    for (int i = lane; i < L.S; i += GT) dst[i] = m[i];
                }
                if (a.all_iters && a.etrue && a.loss && it + 1 < a.T) {
                    for (int v = lane; v < n; v += GT)
                        lacc += bce_neg_sigmoid(post[v], (int)((__ldg(a.etrue + (size_t)shot * W + (v >> 5)) >> (v & 31)) & 1u));
                }
            }
        }
        if (a.post)
            for (int v = lane; v < n; v += GT) a.post[item * n + v] = post[v];
        if (a.decode) {
            // warp wig packs the candidate words wig, wig + G, ...
            const int wl = lane & 31;
            for (int w = wig; w < W; w += G) {
                const int v = 32 * w + wl;
                const uint32_t word = __ballot_sync(kFull, v < n && post[v] < 0.f);
                if (wl == 0) a.cand[item * W + w] = word;
            }
            if (lane == 0) {
                a.conv[item] = conv ? 1 : 0;
                if (a.iters_run) a.iters_run[item] = (uint16_t)K;
            }
        } else if (a.etrue && a.loss) {
            float acc = 0.f;
            for (int v = lane; v < n; v += GT)
                acc += bce_neg_sigmoid(post[v], (int)((__ldg(a.etrue + (size_t)shot * W + (v >> 5)) >> (v & 31)) & 1u));
            acc += lacc;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(kFull, acc, off);
            if constexpr (G > 1) {
                // the group's warps' sums, added in warp order
                if ((lane & 31) == 0) group_part[grp * G + wig] = acc;
                generic_bp::gsync<G>(bar);
                if (lane == 0)
                    for (int w = 1; w < G; ++w) acc += group_part[grp * G + w];
            }
            if (lane == 0) a.loss[item] = a.scale * acc * (a.all_iters ? 1.0f / a.T : 1.0f);
        }
        generic_bp::gsync<G>(bar);
    }
}

// One warp per item: the compiler's own register choice.
template <int DC, int DV>
__global__ void __launch_bounds__(kWmsWarps * 32) wms_forward_warp_kernel(const WmsArgs a) {
    wms_forward_items<DC, DV, 1>(a);
}

// G > 1 warps per item: registers for three 8-warp blocks per SM, the
// residency that the message areas allow for the codes that take G > 1
// (without the bound the compiler stops at 64 registers and spills).
template <int DC, int DV, int G>
__global__ void __launch_bounds__(kWmsWarps * 32, 3) wms_forward_kernel(const WmsArgs a) {
    wms_forward_items<DC, DV, G>(a);
}

// SMEM_ST: the segment's recomputed states sit in shared memory after the
// warp's other arrays (small codes); otherwise in the warp's global buffer.
// Register bound: with the states in shared memory, shared memory limits
// the resident warps (12 per SM on [[144]]), so the kernel may take up to
// 128 registers (measured 4.76 -> 4.69 ms on [[144]] R = 8); the global-state
// path keeps 64 (its residency is set by registers).
template <int DC, int DV, bool SMEM_ST>
__global__ void __launch_bounds__(kWmsWarps * 32, SMEM_ST ? 2 : 4)
wms_backward_kernel(const WmsArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const DevBases& B = a.B;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int MP = B.MP, n = B.n, m_rows = B.m, R = B.R;
    const WmsLayout L = wms_layout(DC, MP, n, a.ckpt);
    const size_t gwarp = (size_t)blockIdx.x * (blockDim.x >> 5) + warp;
    const size_t st_bytes = SMEM_ST ? (size_t)a.ckpt * L.S * 4 : 0;
    unsigned char* wbase = smem + warp * (L.bwd_bytes + st_bytes);
    float* states = SMEM_ST ? reinterpret_cast<float*>(wbase + L.bwd_bytes)
                            : a.seg_buf + gwarp * (size_t)a.ckpt * L.S;  // [ckpt][S], this warp's
    float* q = reinterpret_cast<float*>(wbase);
    float* gm = q + L.S;
    float* gq = gm + L.S;
    float* mu = gq + L.S;
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(a.counter, 1ull);
        item = __shfl_sync(kFull, item, 0);
        if (item >= a.total_items) break;
        const int shot = (int)(item / (unsigned long long)R);
        const int b = (int)(item - (unsigned long long)shot * R);
        const uint32_t* rinfo = B.rowinfo + (size_t)b * MP;
        const uint2* vd = B.vdesc + (size_t)b * n;
        const int32_t* rp = B.rowptr + (size_t)b * MP;
        const int Mb = __ldg(B.rows + b);
        const float* llr = a.llr + (size_t)shot * a.llr_stride;
        const uint8_t* sy = a.synd + (size_t)shot * m_rows;
        for (int v = lane; v < n; v += 32) mu[v] = __fadd_rn(__ldg(llr + v), 0.0f);  // as the forward pass
        uint32_t sb = 0;
        for (int k = 0; k < (MP >> 5); ++k) {
            const int r = lane + 32 * k;
            if (r < Mb) sb |= (uint32_t)(__ldg(sy + (__ldg(rinfo + r) & 0xffffu)) & 1u) << k;
        }
        for (int i = lane; i < L.S; i += 32) gm[i] = 0.0f;
        const float lw = a.scale * (a.all_iters ? 1.0f / a.T : 1.0f);  // weight of one iteration's BCE
        __syncwarp();
        // dL/dm^(T)_e = lw (e_v - sigmoid(-post_v)) on every edge of v
        for (int p = lane; p < n; p += 32) {
            const uint2 d = __ldg(vd + p);
            const int v = d.y & 0xffff, deg = (int)(d.y >> 16);
            const float pv = __ldg(a.post + item * n + v);
            const float sig = 1.0f / (1.0f + expf(pv));
            const uint32_t ev = (__ldg(a.etrue + (size_t)shot * B.W + (v >> 5)) >> (v & 31)) & 1u;
            const float gp = lw * ((float)ev - sig);
            for (int i = 0; i < deg; ++i) gm[__ldg(B.vslot + d.x + i)] = gp;
        }
        __syncwarp();
        const int nseg = (a.T + a.ckpt - 1) / a.ckpt;
        for (int seg = nseg - 1; seg >= 0; --seg) {
            const int t0 = seg * a.ckpt;
            const int t1 = min(a.T, t0 + a.ckpt);
            // states[0] = m^(t0): zero or a checkpoint
            if (t0 == 0) {
                for (int i = lane; i < L.S; i += 32) states[i] = 0.0f;
            } else {
                const float* src = a.ckpt_buf + ((size_t)item * a.nckpt + (t0 / a.ckpt - 1)) * L.S;
                for (int i = lane; i < L.S; i += 32) states[i] = src[i];
            }
            __syncwarp();
            // recompute m^(t0+1 .. t1 - 1) (the adjoint needs m^(t-1) and q^(t-1))
            for (int t = t0 + 1; t < t1; ++t) {
                float* mprev = states + (size_t)(t - 1 - t0) * L.S;
                float* mcur = states + (size_t)(t - t0) * L.S;
                if (t - 1 == 0) {
                    for (int p = lane; p < n; p += 32) {
                        const uint2 d = __ldg(vd + p);
                        const int v = d.y & 0xffff, deg = (int)(d.y >> 16);
                        for (int i = 0; i < deg; ++i) q[__ldg(B.vslot + d.x + i)] = mu[v];
                    }
                } else {
                    wms_var_pass<DV>(B, b, vd, mprev, q, mu, nullptr);
                }
                for (int i = lane; i < L.S; i += 32) mcur[i] = mprev[i];
                __syncwarp();
                const float* wt = a.w + ((size_t)b * a.T + (t - 1)) * a.E;
                const float* gt = a.g + ((size_t)b * a.T + (t - 1)) * a.E;
                wms_check_pass<DC>(B, b, rinfo, Mb, sb, q, mcur, wt, gt);
                __syncwarp();
            }
            // adjoint of iterations t1 .. t0 + 1
            for (int t = t1; t > t0; --t) {
                const float* mprev = states + (size_t)(t - 1 - t0) * L.S;
                if (t - 1 == 0) {
                    for (int p = lane; p < n; p += 32) {
                        const uint2 d = __ldg(vd + p);
                        const int v = d.y & 0xffff, deg = (int)(d.y >> 16);
                        for (int i = 0; i < deg; ++i) q[__ldg(B.vslot + d.x + i)] = mu[v];
                    }
                } else {
                    wms_var_pass<DV>(B, b, vd, mprev, q, mu, nullptr);
                }
                for (int i = lane; i < L.S; i += 32) gq[i] = 0.0f;
                __syncwarp();
                const float* wt = a.w + ((size_t)b * a.T + (t - 1)) * a.E;
                const float* gt = a.g + ((size_t)b * a.T + (t - 1)) * a.E;
                float* gwt = a.gw + ((size_t)b * a.T + (t - 1)) * a.E;
                float* ggt = a.gg + ((size_t)b * a.T + (t - 1)) * a.E;
                for (int k = 0; k < (MP >> 5); ++k) {
                    const int r = lane + 32 * k;
                    if (r >= Mb) continue;
                    const int deg = B.regular ? DC : (int)((__ldg(rinfo + r) >> 16) & 0xffu);
                    const int e0 = __ldg(rp + r);
                    // the row's parameters first: L2 loads (the shared memory
                    // leaves little L1) that then overlap the arithmetic below
                    float wv[DC], gv[DC];
#pragma unroll
                    for (int j = 0; j < DC; ++j) {
                        wv[j] = (j < deg) ? __ldg(wt + e0 + j) : 0.0f;
                        gv[j] = (j < deg) ? __ldg(gt + e0 + j) : 0.0f;
                    }
                    float qq[DC];
#pragma unroll
                    for (int j = 0; j < DC; ++j) qq[j] = (j < deg) ? q[j * MP + r] : MBBP_LMAX;
                    // the smallest and second smallest |q| below LMAX with
                    // their lowest-index positions, and the sign parity: the
                    // min over the edges other than j is (min1, a1) unless
                    // j == a1, then (min2, a2)
                    float min1 = MBBP_LMAX, min2 = MBBP_LMAX;
                    int a1 = -1, a2 = -1;
                    uint32_t par = (sb >> k) & 1u;
#pragma unroll
                    for (int u = 0; u < DC; ++u) {
                        if (u >= deg) continue;
                        const float x = fabsf(qq[u]);
                        if (x < min1) {
                            min2 = min1; a2 = a1;
                            min1 = x; a1 = u;
                        } else if (x < min2) {
                            min2 = x; a2 = u;
                        }
                        par ^= (qq[u] < 0.f) ? 1u : 0u;
                    }
                    float G1 = 0.0f, G2 = 0.0f;  // dL/d|min| routed to a1 / a2
#pragma unroll
                    for (int j = 0; j < DC; ++j) {
                        if (j >= deg) continue;
                        const bool own = (j == a1);
                        const float mn = own ? min2 : min1;
                        const uint32_t neg = par ^ ((qq[j] < 0.f) ? 1u : 0u);
                        const float sgn = neg ? -1.0f : 1.0f;
                        const float ww = wv[j], gg = gv[j];
                        const float gmj = gm[j * MP + r];
                        const float c = ww * sgn * mn;
                        atomicAdd(ggt + e0 + j, gmj * (mprev[j * MP + r] - c));
                        atomicAdd(gwt + e0 + j, gmj * (1.0f - gg) * sgn * mn);
                        gm[j * MP + r] = gmj * gg;  // becomes dL/dm^(t-1): only this lane owns the slot
                        const float gmn = gmj * (1.0f - gg) * ww * sgn;
                        if (own) G2 += gmn;
                        else G1 += gmn;
                    }
#pragma unroll
                    for (int j = 0; j < DC; ++j) {
                        if (j >= deg) continue;
                        const float sq = (qq[j] < 0.f) ? -1.0f : 1.0f;
                        float gj = 0.0f;
                        if (j == a1) gj = G1 * sq;
                        if (j == a2) gj = G2 * sq;
                        gq[j * MP + r] = gj;
                    }
                }
                __syncwarp();
                if (t >= 2 && DV == 6) {
                    // width 6: the same pass with the slots from the packed
                    // descriptors, each step's descriptor loaded one step ahead
                    const uint4* vd6 = B.vdesc6 + (size_t)b * n;
                    uint4 dn = (lane < n) ? __ldg(vd6 + lane) : make_uint4(0u, 0u, 0u, 0u);
                    for (int p = lane; p < n; p += 32) {
                        const uint4 d = dn;
                        if (p + 32 < n) dn = __ldg(vd6 + p + 32);
                        const int v = d.x & 0xffff, deg = (int)(d.x >> 16);
                        uint32_t o[6];
#pragma unroll
                        for (int i = 0; i < 6; ++i) o[i] = generic_bp::packed_off(d, i);
                        float G = 0.0f;
#pragma unroll
                        for (int i = 0; i < 6; ++i)
                            if (i < deg) G += generic_bp::msg_at(gq, o[i]);
                        float gp = 0.0f;
                        if (a.all_iters) {
                            float acc = mu[v];
#pragma unroll
                            for (int i = 0; i < 6; ++i)
                                if (i < deg) acc = __fadd_rn(acc, generic_bp::msg_at(const_cast<float*>(mprev), o[i]));
                            const uint32_t ev = (__ldg(a.etrue + (size_t)shot * B.W + (v >> 5)) >> (v & 31)) & 1u;
                            gp = lw * ((float)ev - 1.0f / (1.0f + expf(acc)));
                        }
#pragma unroll
                        for (int i = 0; i < 6; ++i)
                            if (i < deg) generic_bp::msg_at(gm, o[i]) += G - generic_bp::msg_at(gq, o[i]) + gp;
                    }
                } else if (t >= 2) {
                    for (int p = lane; p < n; p += 32) {
                        const uint2 d = __ldg(vd + p);
                        const int v = d.y & 0xffff, deg = (int)(d.y >> 16);
                        const uint16_t* sl = B.vslot + d.x;
                        float G = 0.0f;
                        for (int i = 0; i < deg; ++i) G += gq[__ldg(sl + i)];
                        // all_iters: the BCE of post^(t-1) joins dL/dm^(t-1)
                        float gp = 0.0f;
                        if (a.all_iters) {
                            float acc = mu[v];
                            for (int i = 0; i < deg; ++i) acc = __fadd_rn(acc, mprev[__ldg(sl + i)]);
                            const uint32_t ev = (__ldg(a.etrue + (size_t)shot * B.W + (v >> 5)) >> (v & 31)) & 1u;
                            gp = lw * ((float)ev - 1.0f / (1.0f + expf(acc)));
                        }
                        for (int i = 0; i < deg; ++i) {
                            const int e = __ldg(sl + i);
                            gm[e] += G - gq[e] + gp;
                        }
                    }
                }
                __syncwarp();
            }
        }
    }
}

// Decode mode: the parameters of every (representation, iteration) in the
// message layout, w and g side by side: wg[((b T + t) DC + j) MP + r] is the
// (w, g) of edge j of row r of H^(b) at iteration t, zeros where the row has
// no edge j, so that the check pass reads one coalesced float2 per edge.
template <int DC>
__global__ void wms_pack_kernel(const WmsArgs a, float2* __restrict__ wg) {
    const DevBases& B = a.B;
    const int MP = B.MP;
    const size_t total = (size_t)B.R * a.T * MP;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(i % MP);
        const size_t bt = i / MP;  // b T + t
        const int b = (int)(bt / a.T);
        int deg = 0, e0 = 0;
        if (r < __ldg(B.rows + b)) {
            deg = B.regular ? DC : (int)((__ldg(B.rowinfo + (size_t)b * MP + r) >> 16) & 0xffu);
            e0 = __ldg(B.rowptr + (size_t)b * MP + r);
        }
        const float* wt = a.w + bt * a.E + e0;
        const float* gt = a.g + bt * a.E + e0;
#pragma unroll
        for (int j = 0; j < DC; ++j)
            wg[(bt * DC + j) * MP + r] = (j < deg) ? make_float2(__ldg(wt + j), __ldg(gt + j)) : make_float2(0.f, 0.f);
    }
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ grad, float* __restrict__ m1,
                            float* __restrict__ m2, size_t count, float lr, float b1, float b2, float eps,
                            float c1, float c2, float lo, float hi) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float gi = grad[i];
    const float a = b1 * m1[i] + (1.0f - b1) * gi;
    const float v = b2 * m2[i] + (1.0f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = v;
    const float x = p[i] - lr * (a / c1) / (sqrtf(v / c2) + eps);
    p[i] = fminf(fmaxf(x, lo), hi);
}

template <int K, int G>
cudaError_t launch_forward_g(const WmsArgs& a, size_t fixed, size_t per_item, int warps, int per_sm,
                             cudaStream_t s, int sm_count) {
    const unsigned long long groups = (unsigned long long)(warps / G);
    const size_t smem = fixed + groups * per_item;
    unsigned long long want = (a.total_items + groups - 1) / groups;
    unsigned long long grid = (unsigned long long)per_sm * sm_count;
    if (want < grid) grid = want;
    if constexpr (G == 1)
        wms_forward_warp_kernel<K, K><<<(unsigned)grid, warps * 32, smem, s>>>(a);
    else
        wms_forward_kernel<K, K, G><<<(unsigned)grid, warps * 32, smem, s>>>(a);
    return cudaGetLastError();
}

template <int K>
cudaError_t launch_wms_t(const WmsArgs& a, bool backward, cudaStream_t s, int sm_count) {
    const WmsLayout L = wms_layout(K, a.B.MP, a.B.n, a.ckpt);
    if (!backward) {
        // forward / decode: G warps per item, G in {1, 2, 4}; per G the block
        // size (a multiple of G, up to 8 warps) with the most resident warps
        // per SM within 200 KB of shared memory per block (H's columns once,
        // then one area per item); a larger G only when it holds at least
        // half again as many warps as the best smaller one
        if (L.fwd_bytes > 200 * 1024) return cudaErrorInvalidConfiguration;
        const size_t fixed = (size_t)((K * a.B.mpad * 2 + 15) & ~15);
        const void* kerns[3] = {reinterpret_cast<const void*>(wms_forward_warp_kernel<K, K>),
                                reinterpret_cast<const void*>(wms_forward_kernel<K, K, 2>),
                                reinterpret_cast<const void*>(wms_forward_kernel<K, K, 4>)};
        int best_g = -1, best_w = 0, best_b = 0;
        for (int gi = 0; gi < 3; ++gi) {
            const int G = 1 << gi;
            int warps = 0, per_sm = 0;
            for (int w = G; w <= kWmsWarps && fixed + (size_t)(w / G) * L.fwd_bytes <= 200 * 1024; w += G) {
                int b = 0;
                cudaError_t e = prepare_kernel(kerns[gi], w * 32, fixed + (size_t)(w / G) * L.fwd_bytes, &b);
                if (e != cudaSuccess) return e;
                if (b * w > per_sm * warps) {
                    warps = w;
                    per_sm = b;
                }
            }
            if (warps > 0 && (best_g < 0 || 2 * warps * per_sm >= 3 * best_w * best_b)) {
                best_g = gi;
                best_w = warps;
                best_b = per_sm;
            }
        }
        if (best_g < 0) return cudaErrorInvalidConfiguration;
        if (best_g == 0) return launch_forward_g<K, 1>(a, fixed, L.fwd_bytes, best_w, best_b, s, sm_count);
        if (best_g == 1) return launch_forward_g<K, 2>(a, fixed, L.fwd_bytes, best_w, best_b, s, sm_count);
        return launch_forward_g<K, 4>(a, fixed, L.fwd_bytes, best_w, best_b, s, sm_count);
    }
    const size_t st_bytes = (size_t)a.ckpt * L.S * 4;
    const bool smem_st = wms_states_in_smem(a.B, a.ckpt);
    const size_t per_warp = L.bwd_bytes + (smem_st ? st_bytes : 0);
    if (per_warp > 200 * 1024) return cudaErrorInvalidConfiguration;
    const void* kern = smem_st ? reinterpret_cast<const void*>(wms_backward_kernel<K, K, true>)
                               : reinterpret_cast<const void*>(wms_backward_kernel<K, K, false>);
    // the block size with the most resident warps per SM (ties: the smaller
    // block), within 200 KB of shared memory per block
    int warps = 0, per_sm = 0;
    for (int w = 1; w <= kWmsWarps && (size_t)w * per_warp <= 200 * 1024; ++w) {
        int b = 0;
        cudaError_t e = prepare_kernel(kern, w * 32, (size_t)w * per_warp, &b);
        if (e != cudaSuccess) return e;
        if (b * w > per_sm * warps) {
            warps = w;
            per_sm = b;
        }
    }
    if (warps == 0) return cudaErrorInvalidConfiguration;
    const size_t smem = warps * per_warp;
    unsigned long long want = (a.total_items + warps - 1) / warps;
    unsigned long long grid = (unsigned long long)per_sm * sm_count;
    if (want < grid) grid = want;
    // one segment buffer per warp: at most kWmsMaxWarps warps
    const unsigned long long cap = kWmsMaxWarps / warps;
    if (grid > cap) grid = cap;
    if (smem_st)
        wms_backward_kernel<K, K, true><<<(unsigned)grid, warps * 32, smem, s>>>(a);
    else
        wms_backward_kernel<K, K, false><<<(unsigned)grid, warps * 32, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

bool wms_states_in_smem(const DevBases& B, int ckpt) {
    // the backward pass keeps a segment's states in shared memory when four
    // warps' worth fits in about half of an SM's shared memory
    const WmsLayout L = wms_layout(B.DC, B.MP, B.n, ckpt);
    return (size_t)kWmsStateWarps * (L.bwd_bytes + (size_t)ckpt * L.S * 4) <= 110 * 1024;
}

cudaError_t launch_wms(const WmsArgs& a, bool backward, cudaStream_t s, int sm_count) {
    if (a.B.DC == 6) return launch_wms_t<6>(a, backward, s, sm_count);
    if (a.B.DC == 8) return launch_wms_t<8>(a, backward, s, sm_count);
    if (a.B.DC == 12) return launch_wms_t<12>(a, backward, s, sm_count);
    return cudaErrorInvalidValue;
}

cudaError_t launch_wms_pack(const WmsArgs& a, float2* wg, cudaStream_t s, int sm_count) {
    const size_t total = (size_t)a.B.R * a.T * a.B.MP;
    if (total == 0) return cudaSuccess;
    size_t grid = (total + 255) / 256;
    if (grid > (size_t)sm_count * 8) grid = (size_t)sm_count * 8;
    if (a.B.DC == 6) wms_pack_kernel<6><<<(unsigned)grid, 256, 0, s>>>(a, wg);
    else if (a.B.DC == 8) wms_pack_kernel<8><<<(unsigned)grid, 256, 0, s>>>(a, wg);
    else if (a.B.DC == 12) wms_pack_kernel<12><<<(unsigned)grid, 256, 0, s>>>(a, wg);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_adam(float* p, const float* g, float* m1, float* m2, size_t count, float lr, float b1,
                        float b2, float eps, int step, float lo, float hi, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    const float c1 = 1.0f - powf(b1, (float)step);
    const float c2 = 1.0f - powf(b2, (float)step);
    const unsigned grid = (unsigned)((count + 255) / 256);
    adam_kernel<<<grid, 256, 0, s>>>(p, g, m1, m2, count, lr, b1, b2, eps, c1, c2, lo, hi);
    return cudaGetLastError();
}

}  // namespace mbbp
