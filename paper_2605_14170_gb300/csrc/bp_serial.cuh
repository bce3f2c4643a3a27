// Device code of the serial-schedule path for kernel widths 6 and 8.
//
// A warp decodes shots of one representation, CS at a time, pulling them
// from a per-representation counter.  Each shot keeps its check-to-variable
// messages m_{c->v} in shared memory (edge j of the row at position p at
// slot j * MP + p, followed by one slot holding -0.0f, the exact additive
// identity of IEEE addition); the host places the rows (a permutation of
// the positions) so that the lanes of one access hit different banks.  A serial iteration visits the layers
// of the representation in order; within a layer the (row, shot) pairs are
// spread over the lanes.  Rows of a layer share no variable, so the pairs of
// one layer read only messages of other layers' rows and write only their
// own slots: the result is that of visiting the rows one at a time.
//
// Per edge, a 16-byte descriptor gives the variable and the byte offsets of
// its other edges in ascending row order (padded with the -0.0f slot), so
// q_{v->c} = mu_v + m_1 + m_2 + ... is one load, a fixed chain of shared
// loads and correctly rounded adds, in the oracle's order; the padding adds
// leave every value, -0.0f included, unchanged.  The check rule is the
// flooding path's (check_out).  After the last layer, the posteriors
// mu_v + all messages (ascending row, from a per-variable descriptor of the
// same form), the hard decisions and the halting test H e = s per shot.
#pragma once

#include "bp_generic.cuh"

namespace mbbp {
namespace serial_bp {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float lds_b(const float* base, uint32_t byte_off) {
    return *reinterpret_cast<const float*>(reinterpret_cast<const char*>(base) + byte_off);
}

// The q_{v->c} of one edge: mu_v plus NO other messages of v (byte offsets
// in the descriptor; unused ones point at the -0.0f slot).  Unclamped: q only
// feeds check_out, whose min runs over LMAX and whose sum-product phi
// underflows to 0 beyond |q| = 104, so a clamp changes no message.
template <int NO>
__device__ __forceinline__ float edge_q(const float* msg, const float* mu, uint4 d) {
    const uint32_t o[7] = {d.x >> 16, d.y & 0xffffu, d.y >> 16, d.z & 0xffffu, d.z >> 16,
                           d.w & 0xffffu, d.w >> 16};
    float x = mu[d.x & 0xffffu];
#pragma unroll
    for (int i = 0; i < NO; ++i) x = __fadd_rn(x, lds_b(msg, o[i]));
    return x;
}

// Posterior of one variable: mu_v plus its NV message slots (padded).
template <int NV>
__device__ __forceinline__ float var_post(const float* msg, float mu, uint4 d) {
    const uint32_t o[8] = {d.x & 0xffffu, d.x >> 16, d.y & 0xffffu, d.y >> 16,
                           d.z & 0xffffu, d.z >> 16, d.w & 0xffffu, d.w >> 16};
    float P = mu;
#pragma unroll
    for (int i = 0; i < NV; ++i) P = __fadd_rn(P, lds_b(msg, o[i]));
    return P;
}

// Load shot `shot` into slot sh: zero messages, the -0.0f slot, LLRs, the
// hard decision of the LLRs and the syndrome bits of the rows of H^(t) (by
// row position) and of the rows of H (by row).
template <int DC, int CS>
__device__ __forceinline__ void load_shot(const DevBases& B, const ShotIO& io, int b, int shot, int sh,
                                          const Layout& L, float* msg, float* mu, uint8_t* eh,
                                          uint32_t* sbits) {
    const int lane = threadIdx.x & 31;
    const int MP = B.MP, n = B.n, m = B.m;
    const int Mb = __ldg(B.rows + b);
    const uint32_t* rinfo = B.rinfo_s + (size_t)b * MP;
    const unsigned long long item = (unsigned long long)shot * B.R + b;
    const float* llr = io.llr + (size_t)shot * io.llr_stride;
    const uint8_t* sy = io.synd + (size_t)shot * m;
    float* ms = msg + sh * L.SH;
    __syncwarp();
    for (int i = lane; i < DC * MP; i += 32) ms[i] = 0.0f;  // m^(0)_{c->v} = 0
    if (lane == 0) ms[DC * MP] = -0.0f;
    for (int v = lane; v < n; v += 32) {
        const float x = __ldg(llr + v);
        mu[sh * L.NP + v] = __fadd_rn(x, 0.0f);  // -0 -> +0 (sign bits decide the check rule)
        eh[sh * L.EP + v] = (x < 0.f) ? 1 : 0;
        if (io.post) io.post[item * n + v] = x;
    }
    if (lane == 0) eh[sh * L.EP + n] = 0;  // padding column of hcol
    // syndrome bits by row position (check rule) and by row of H (halting)
    uint32_t* sbh = sbits + CS * L.RW;
    for (int k = 0; k < L.RW; ++k) {
        const int r = lane + 32 * k;
        const uint32_t bit = (r < Mb) ? (uint32_t)(__ldg(sy + (__ldg(rinfo + r) & 0xffffu)) & 1u) : 0u;
        const uint32_t word = __ballot_sync(kFull, bit);
        const uint32_t hbit = (r < m) ? (uint32_t)(__ldg(sy + r) & 1u) : 0u;
        const uint32_t hword = __ballot_sync(kFull, hbit);
        if (lane == 0) {
            sbits[sh * L.RW + k] = word;
            sbh[sh * L.RW + k] = hword;
        }
    }
    __syncwarp();
}

// Halting rule of the shot in slot sh: H e = s on the rows of H (the extra
// rows of H^(t) are copies), one row group at a time until one fails,
// starting with kf, the group that failed at the slot's previous test (kf is
// updated).  Warp-uniform result.
template <int DC>
__device__ __forceinline__ bool halted(int m, int mpad, const uint16_t* hcol, const uint8_t* e,
                                       const uint32_t* sb, int& kf) {
    const int lane = threadIdx.x & 31;
    const int groups = (m + 31) >> 5;
    for (int s = 0; s < groups; ++s) {
        const int g = (kf + s < groups) ? kf + s : kf + s - groups;
        const int r = 32 * g + lane;
        bool ok = true;
        if (r < m) {
            uint32_t par = (sb[g] >> lane) & 1u;
#pragma unroll
            for (int j = 0; j < DC; ++j) par ^= e[hcol[j * mpad + r]];
            ok = (par == 0u);
        }
        if (!__all_sync(kFull, ok)) {  // warp-uniform
            kf = g;
            return false;
        }
    }
    return true;
}

// Next shot of representation b from its shared counter (warp-uniform; -1
// when every shot of b has been taken).
__device__ __forceinline__ int pull_shot(unsigned int* ctr, int batch) {
    unsigned int k = 0;
    if ((threadIdx.x & 31) == 0) k = atomicAdd(ctr, 1u);
    k = __shfl_sync(kFull, k, 0);
    return k < (unsigned int)batch ? (int)k : -1;
}

// Decode shots of representation b with CS slots until its shot counter is
// exhausted: every slot runs its own shot; a slot whose shot halts (or
// reaches the iteration limit) stores it and pulls the next shot of b, so a
// slow shot does not hold the lanes of the others.  area: this warp's
// layout(DC, MP, n, CS).bytes of shared memory; hcol: columns of the rows
// of H ([DC][mpad], shared memory).
template <int DC, int NO, int NV, int RULE, bool REG, int CS>
__device__ __forceinline__ void run_rep(const DevBases& B, const ShotIO& io, int b, unsigned int* ctr,
                                        unsigned char* area, const uint16_t* hcol) {
    constexpr int CSH = (CS == 4) ? 2 : (CS == 2) ? 1 : 0;
    const int lane = threadIdx.x & 31;
    const int MP = B.MP, n = B.n, m = B.m, R = B.R, W = B.W, mpad = B.mpad;
    const Layout L = layout(DC, MP, n, CS);
    float* msg = reinterpret_cast<float*>(area);
    float* mu = msg + CS * L.SH;
    uint8_t* eh = reinterpret_cast<uint8_t*>(mu + CS * L.NP);
    uint32_t* sbits = reinterpret_cast<uint32_t*>(eh + CS * L.EP);
    const int nl = __ldg(B.nlayers + b);
    const uint32_t* rinfo = B.rinfo_s + (size_t)b * MP;
    const uint16_t* lrows = B.lpos + (size_t)b * MP;
    const uint16_t* lptr = B.lptr + (size_t)b * (MP + 1);
    const uint4* ed = B.edesc + (size_t)b * DC * MP;
    const uint4* vd = B.vdesc3 + (size_t)b * n;

    // warp-uniform slot state
    int shot[CS], iter[CS], kf[CS];
    uint32_t active = 0;
#pragma unroll
    for (int sh = 0; sh < CS; ++sh) {
        iter[sh] = 0;
        kf[sh] = 0;
        shot[sh] = pull_shot(ctr, io.batch);
        if (shot[sh] >= 0) {
            active |= 1u << sh;
            load_shot<DC, CS>(B, io, b, shot[sh], sh, L, msg, mu, eh, sbits);
        }
    }
    while (active) {
        // halting test, output and refill of every slot
#pragma unroll
        for (int sh = 0; sh < CS; ++sh) {
            while ((active >> sh) & 1u) {
                const bool ok = halted<DC>(m, mpad, hcol, eh + sh * L.EP, sbits + CS * L.RW + sh * L.RW, kf[sh]);
                if (!ok && iter[sh] < io.iters) break;
                const unsigned long long item = (unsigned long long)shot[sh] * R + b;
                generic_bp::store_item(io, item, n, W, eh + sh * L.EP, ok, iter[sh]);
                shot[sh] = pull_shot(ctr, io.batch);
                if (shot[sh] >= 0) {
                    iter[sh] = 0;
                    kf[sh] = 0;
                    load_shot<DC, CS>(B, io, b, shot[sh], sh, L, msg, mu, eh, sbits);
                } else {
                    active &= ~(1u << sh);
                }
            }
        }
        if (!active) break;
        // one serial iteration of every active slot: layers in order
        for (int l = 0; l < nl; ++l) {
            const int i0 = __ldg(lptr + l);
            const int cnt = (__ldg(lptr + l + 1) - i0) << CSH;
            for (int idx = lane; idx < cnt; idx += 32) {
                const int sh = idx & (CS - 1);
                if (!((active >> sh) & 1u)) continue;
                const int r = __ldg(lrows + i0 + (idx >> CSH));
                const int deg = REG ? DC : (int)((__ldg(rinfo + r) >> 16) & 0xffu);
                float* ms = msg + sh * L.SH;
                const float* mus = mu + sh * L.NP;
                float q[DC];
#pragma unroll
                for (int j = 0; j < DC; ++j) {
                    if (REG || j < deg) q[j] = edge_q<NO>(ms, mus, __ldg(ed + j * MP + r));
                    else q[j] = MBBP_LMAX;
                }
                const uint32_t sbit = (sbits[sh * L.RW + (r >> 5)] >> (r & 31)) & 1u;
                generic_bp::check_out<DC, RULE>(q, ms, r, MP, deg, sbit, io.alpha);
            }
            __syncwarp();
        }
        // posteriors and hard decisions
        const int cnt = n << CSH;
        for (int idx = lane; idx < cnt; idx += 32) {
            const int sh = idx & (CS - 1);
            if (!((active >> sh) & 1u)) continue;
            const int v = idx >> CSH;
            const float P = var_post<NV>(msg + sh * L.SH, mu[sh * L.NP + v], __ldg(vd + v));
            eh[sh * L.EP + v] = (P < 0.f) ? 1 : 0;
            if (io.post) {
                int s_of = shot[0];
#pragma unroll
                for (int k = 1; k < CS; ++k) s_of = (sh == k) ? shot[k] : s_of;
                io.post[((unsigned long long)s_of * R + b) * n + v] = P;
            }
        }
        __syncwarp();
#pragma unroll
        for (int sh = 0; sh < CS; ++sh) iter[sh] += (int)((active >> sh) & 1u);
    }
    __syncwarp();
}

}  // namespace serial_bp
}  // namespace mbbp
