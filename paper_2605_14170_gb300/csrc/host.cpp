// Host side of the C ABI in include/mbbp.h: Algorithm 2 and the collection of
// representations (Section III-A), packing of every H^(t) = [H; H_t]
// (Eq. (4)) into the kernels' layout, the logical basis for the judge, and
// argument checking for the launches.
#include <algorithm>
#include <array>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <set>
#include <string>
#include <thread>
#include <vector>

#include "mbbp_internal.h"

using namespace mbbp;

struct mbbp_bases {
    int m = 0, n = 0, R = 0, K = 0, DV = 0, MP = 0, mpad = 0, W = 0, regular = 0;
    int device = 0, sm_count = 0;
    std::vector<uint8_t> H;
    std::vector<int32_t> set_ptr, set_rows, rows, edges;
    std::vector<int32_t> lorder, lptr, nlayers;  // serial schedule, [R][MP], [R][MP+1], [R]
    void* dmem = nullptr;
    DevBases dev{};
};

struct mbbp_plan {
    std::vector<const mbbp_bases*> codes;
    int device = 0, sm_count = 0;
    int warps = 8;               // warps per block of the persistent kernel
    std::vector<int> chunk;      // shots per work item, per code
    std::vector<int> kind;       // kKindSmall / kKindGeneric, per code
    std::vector<int> order;      // codes in work-list order
};

struct mbbp_logicals {
    int m = 0, n = 0, k = 0, K = 0, mpad = 0, W = 0, device = 0;
    std::vector<uint8_t> ops;  // k x n
    void* dmem = nullptr;
    DevLogicals dev{};
};

namespace {

thread_local std::string g_err;

mbbp_status fail(mbbp_status st, const std::string& msg) {
    g_err = msg;
    return st;
}

mbbp_status cuda_fail(cudaError_t e, const char* what) {
    return fail(MBBP_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// splitmix64 (Steele, Lea & Flood, OOPSLA 2014): output number i >= 1 of the
// generator whose state starts at `state`.
uint64_t sm64_at(uint64_t state, uint64_t i) {
    uint64_t z = state + i * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

struct Tanner {
    int m = 0, n = 0;
    std::vector<std::vector<int>> rcols;  // columns of each row, ascending
    std::vector<std::vector<int>> crows;  // rows of each column, ascending
};

mbbp_status make_tanner(const uint8_t* H, int m, int n, Tanner& g) {
    if (!H) return fail(MBBP_E_INVALID, "H is NULL");
    if (m < 1 || n < 1) return fail(MBBP_E_INVALID, "m and n must be >= 1");
    if (m > 65535 || n > MBBP_MAX_N) return fail(MBBP_E_TOO_LARGE, "H is larger than the limits");
    g.m = m;
    g.n = n;
    g.rcols.assign(m, {});
    g.crows.assign(n, {});
    for (int r = 0; r < m; ++r)
        for (int v = 0; v < n; ++v) {
            const uint8_t x = H[(size_t)r * n + v];
            if (x > 1) return fail(MBBP_E_INVALID, "H entries must be 0 or 1");
            if (x) {
                g.rcols[r].push_back(v);
                g.crows[v].push_back(r);
            }
        }
    return MBBP_OK;
}

// Algorithm 2 on an adjacency-list Tanner graph.  Per-subtree "visited" and
// "tested" marks are stamps equal to the current subtree index.
int subtrees_impl(const Tanner& g, const int32_t* perm, int32_t* cs, int32_t* order) {
    std::vector<int> vmark(g.n, 0), tmark(g.m, 0);
    std::vector<int> queue;
    std::fill(cs, cs + g.m, 0);
    int s = 0, nord = 0;
    for (int idx = 0; idx < g.m; ++idx) {
        const int root = perm[idx];
        if (cs[root] != 0) continue;
        ++s;
        queue.clear();
        queue.push_back(root);
        for (size_t head = 0; head < queue.size(); ++head) {
            const int u = queue[head];
            if (tmark[u] == s) continue;
            tmark[u] = s;
            int eta = 0;
            for (int v : g.rcols[u]) eta += (vmark[v] == s) ? 1 : 0;
            if (eta > 1) continue;
            cs[u] = s;
            if (order) order[nord++] = u;
            for (int v : g.rcols[u]) {
                vmark[v] = s;
                for (int c : g.crows[v])
                    if (tmark[c] != s && cs[c] == 0) queue.push_back(c);
            }
        }
    }
    return s;
}

void permutation_impl(uint64_t seed, int j, int m, int32_t* perm) {
    for (int i = 0; i < m; ++i) perm[i] = i;
    if (j == 0) return;
    const uint64_t state = seed ^ (uint64_t)j;
    uint64_t draw = 0;
    for (int i = m - 1; i >= 1; --i) {
        const uint64_t x = sm64_at(state, ++draw);
        std::swap(perm[i], perm[(int)(x % (uint64_t)(i + 1))]);
    }
}

constexpr int kMaxPerms = 1024;

mbbp_status collect_impl(const Tanner& g, int R, uint64_t seed, std::vector<int32_t>& set_ptr,
                         std::vector<int32_t>& set_rows) {
    std::vector<int32_t> perm(g.m), cs(g.m), order(g.m);
    std::set<std::vector<int32_t>> seen;
    set_ptr.assign(1, 0);
    set_rows.clear();
    int found = 0;
    for (int j = 0; j < kMaxPerms && found < R; ++j) {
        permutation_impl(seed, j, g.m, perm.data());
        subtrees_impl(g, perm.data(), cs.data(), order.data());
        int pos = 0;
        while (pos < g.m && found < R) {
            const int start = pos, t = cs[order[pos]];
            while (pos < g.m && cs[order[pos]] == t) ++pos;
            std::vector<int32_t> key(order.begin() + start, order.begin() + pos);
            std::sort(key.begin(), key.end());
            if (!seen.insert(key).second) continue;
            set_rows.insert(set_rows.end(), order.begin() + start, order.begin() + pos);
            set_ptr.push_back((int32_t)set_rows.size());
            ++found;
        }
    }
    if (found < R)
        return fail(MBBP_E_NOT_FOUND, "only " + std::to_string(found) +
                                          " distinct subtrees exist among the first " +
                                          std::to_string(kMaxPerms) + " root orders");
    return MBBP_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Small-code layout: ELL index sigma[r] of every row r of H^(t), the slot
// s = slot[r][j] < deg(r) that holds the j-th edge of row r (j in H's column
// order), and the variable at every position (32 positions = one warp step of
// the variable pass).  Slot s of row r lives in shared-memory bank
// (sigma[r] + rot(s)) & 31.  In the variable pass the 32 lanes of a step read
// the i-th edge of their variables together; the cost of that access is the
// largest number of lanes that hit one bank.  Simulated annealing over row
// swaps, swaps of two edge slots within a row and swaps of equal-degree
// variables between steps lowers the summed cost.  The normalized min-sum
// check rule is symmetric in a row's edges (minima and sign parity are
// exact), so any layout gives the same results; the sum-product rule adds
// its terms in slot order, which moves its rounding by a few ulps.
struct SmallLayout {
    std::vector<int> sigma;               // ELL index of row r
    std::vector<std::array<int, 6>> slot;  // slot of the j-th edge of row r
    std::vector<int> order;               // variable at position p
};

SmallLayout small_layout(const Tanner& g, const std::vector<int>& src, int n, int MP, uint64_t seed) {
    const int M = (int)src.size();
    constexpr int DVX = 8;
    std::vector<std::vector<std::pair<int, int>>> ve(n);  // (row, j), ascending row
    std::vector<std::array<int, 6>> ei(M);                 // edge index i of (r, j) in ve[v]
    for (int r = 0; r < M; ++r) {
        const auto& cols = g.rcols[src[r]];
        for (int j = 0; j < (int)cols.size(); ++j) {
            ei[r][j] = (int)ve[cols[j]].size();
            ve[cols[j]].push_back({r, j});
        }
    }
    std::vector<std::vector<std::pair<int, int>>> re(M);  // (variable, edge index i)
    for (int v = 0; v < n; ++v)
        for (int i = 0; i < (int)ve[v].size(); ++i) re[ve[v][i].first].push_back({v, i});
    SmallLayout L;
    L.sigma.resize(M);
    L.slot.resize(M);
    for (int r = 0; r < M; ++r) {
        L.sigma[r] = r;
        for (int j = 0; j < 6; ++j) L.slot[r][j] = j;
    }
    // variables by descending degree: the last step, the one that n leaves
    // partly empty, then holds the smallest degrees (every step costs its
    // largest degree for all 32 lanes)
    L.order.resize(n);
    for (int v = 0; v < n; ++v) L.order[v] = v;
    std::stable_sort(L.order.begin(), L.order.end(),
                     [&](int a, int b) { return ve[a].size() > ve[b].size(); });
    std::vector<int> posof(n);
    for (int p = 0; p < n; ++p) posof[L.order[p]] = p;
    const int steps = (n + 31) / 32;
    std::vector<int> cnt((size_t)steps * DVX * 32, 0), mx((size_t)steps * DVX, 0);
    // per cell, kept up to date on every count change: the number of banks
    // holding each count, the largest count and the colliding lane pairs, so
    // that a cell's cost is read in O(1) (the same values as counting its 32
    // banks)
    constexpr int kMaxCount = 40;
    std::vector<int> hist((size_t)steps * DVX * (kMaxCount + 1), 0), top((size_t)steps * DVX, 0),
        pairs((size_t)steps * DVX, 0);
    for (int c = 0; c < steps * DVX; ++c) hist[(size_t)c * (kMaxCount + 1)] = 32;
    auto inc = [&](size_t idx) {
        const size_t c = idx >> 5;
        const int q = cnt[idx]++;
        int* h = &hist[c * (kMaxCount + 1)];
        --h[q];
        ++h[q + 1];
        pairs[c] += q;
        if (q + 1 > top[c]) top[c] = q + 1;
    };
    auto dec = [&](size_t idx) {
        const size_t c = idx >> 5;
        const int q = cnt[idx]--;
        int* h = &hist[c * (kMaxCount + 1)];
        --h[q];
        ++h[q - 1];
        pairs[c] -= q - 1;
        if (q == top[c] && h[q] == 0) top[c] = q - 1;
    };
    auto bank = [&](int r, int j) { return (L.sigma[r] + slot_rot(L.slot[r][j])) & 31; };
    auto cell = [&](int v, int i) { return (posof[v] >> 5) * DVX + i; };
    for (int v = 0; v < n; ++v)
        for (int i = 0; i < (int)ve[v].size(); ++i) inc((size_t)cell(v, i) * 32 + bank(ve[v][i].first, ve[v][i].second));
    // The kernel runs every edge position i of a step up to the step's
    // largest degree; lanes with fewer edges (and the padding positions past
    // n) read the warp's zero slot there, all at one address (a broadcast):
    // one more access in the zero slot's bank, fixed because moves only swap
    // variables of equal degree between steps.
    {
        const int zero_bank = (6 * MP) & 31;
        for (int st = 0; st < steps; ++st) {
            int dmin = 1 << 30, dmax = 0;
            for (int l = 0; l < 32; ++l) {
                const int pp = 32 * st + l;
                const int d = pp < n ? (int)ve[L.order[pp]].size() : 0;
                dmin = std::min(dmin, d);
                dmax = std::max(dmax, d);
            }
            for (int i = dmin; i < dmax && i < DVX; ++i) inc(((size_t)st * DVX + i) * 32 + zero_bank);
        }
    }
    // cost of a cell: its largest bank count (the wavefronts of the access)
    // first, then its colliding lane pairs, so that a move removing one
    // collision of several is rewarded before the largest count drops
    auto remax = [&](int c) { mx[c] = top[c] * 1024 + pairs[c]; };
    long total = 0;
    for (int c = 0; c < steps * DVX; ++c) { remax(c); total += mx[c]; }
    std::vector<int> best_sigma = L.sigma, best_order = L.order;
    std::vector<std::array<int, 6>> best_slot = L.slot;
    long best = LONG_MAX;  // none yet
    uint64_t rs = seed;
    auto rnd = [&]() { rs += 0x9E3779B97F4A7C15ULL; uint64_t z = rs;
                       z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
                       z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL; return z ^ (z >> 31); };
    std::vector<int> cells;
    const int iters = 1000000;
    for (int it = 0; it < iters; ++it) {
        const double T = 0.6 * (1.0 - (double)it / iters) + 0.02;
        cells.clear();
        long before = 0, after = 0;
        const int kind = (int)(rnd() % 3);  // 0: two rows, 1: two edge slots of a row, 2: two variables
        const bool row_move = kind == 0 || (kind == 2 && steps == 1);
        int a = 0, b = 0;
        if (kind == 1) {
            const int r = (int)(rnd() % M);
            const auto& cols = g.rcols[src[r]];
            const int d = (int)cols.size();
            const int ja = (int)(rnd() % d), jb = (int)(rnd() % d);
            if (ja == jb) continue;
            const int ca = cell(cols[ja], ei[r][ja]), cb = cell(cols[jb], ei[r][jb]);
            cells.push_back(ca);
            if (cb != ca) cells.push_back(cb);
            for (int c : cells) before += mx[c];
            auto swap_slots = [&]() {
                dec((size_t)ca * 32 + bank(r, ja));
                dec((size_t)cb * 32 + bank(r, jb));
                std::swap(L.slot[r][ja], L.slot[r][jb]);
                inc((size_t)ca * 32 + bank(r, ja));
                inc((size_t)cb * 32 + bank(r, jb));
            };
            swap_slots();
            for (int c : cells) { remax(c); after += mx[c]; }
            const long dd = after - before;
            const double u = (double)(rnd() >> 11) * (1.0 / 9007199254740992.0);
            if (dd <= 0 || u < std::exp(-(double)dd / T)) {
                total += dd;
            } else {
                swap_slots();
                for (int c : cells) remax(c);
            }
        } else if (row_move) {
            a = (int)(rnd() % M);
            b = (int)(rnd() % M);
            if (a == b) continue;
            for (int rr : {a, b})
                for (auto& e : re[rr]) cells.push_back(cell(e.first, e.second));
            std::sort(cells.begin(), cells.end());
            cells.erase(std::unique(cells.begin(), cells.end()), cells.end());
            for (int c : cells) before += mx[c];
            const std::vector<int>& keep = cells;  // not changed below
            for (int rr : {a, b})
                for (auto& e : re[rr]) dec((size_t)cell(e.first, e.second) * 32 + bank(rr, ve[e.first][e.second].second));
            std::swap(L.sigma[a], L.sigma[b]);
            for (int rr : {a, b})
                for (auto& e : re[rr]) inc((size_t)cell(e.first, e.second) * 32 + bank(rr, ve[e.first][e.second].second));
            for (int c : keep) { remax(c); after += mx[c]; }
            const long d = after - before;
            const double u = (double)(rnd() >> 11) * (1.0 / 9007199254740992.0);
            if (d <= 0 || u < std::exp(-(double)d / T)) {
                total += d;
            } else {
                for (int rr : {a, b})
                    for (auto& e : re[rr]) dec((size_t)cell(e.first, e.second) * 32 + bank(rr, ve[e.first][e.second].second));
                std::swap(L.sigma[a], L.sigma[b]);
                for (int rr : {a, b})
                    for (auto& e : re[rr]) inc((size_t)cell(e.first, e.second) * 32 + bank(rr, ve[e.first][e.second].second));
                for (int c : keep) remax(c);
            }
        } else {
            const int pa = (int)(rnd() % n), pb = (int)(rnd() % n);
            const int va = L.order[pa], vb = L.order[pb];
            if ((pa >> 5) == (pb >> 5) || ve[va].size() != ve[vb].size()) continue;
            for (int v : {va, vb})
                for (int i = 0; i < (int)ve[v].size(); ++i) cells.push_back(cell(v, i));
            for (int i = 0; i < (int)ve[va].size(); ++i) {
                cells.push_back((pb >> 5) * DVX + i);
                cells.push_back((pa >> 5) * DVX + i);
            }
            std::sort(cells.begin(), cells.end());
            cells.erase(std::unique(cells.begin(), cells.end()), cells.end());
            for (int c : cells) before += mx[c];
            const std::vector<int>& keep = cells;  // not changed below
            auto swap_vars = [&]() {
                for (int v : {va, vb})
                    for (int i = 0; i < (int)ve[v].size(); ++i)
                        dec((size_t)cell(v, i) * 32 + bank(ve[v][i].first, ve[v][i].second));
                std::swap(L.order[posof[va]], L.order[posof[vb]]);
                std::swap(posof[va], posof[vb]);
                for (int v : {va, vb})
                    for (int i = 0; i < (int)ve[v].size(); ++i)
                        inc((size_t)cell(v, i) * 32 + bank(ve[v][i].first, ve[v][i].second));
            };
            swap_vars();
            for (int c : keep) { remax(c); after += mx[c]; }
            const long d = after - before;
            const double u = (double)(rnd() >> 11) * (1.0 / 9007199254740992.0);
            if (d <= 0 || u < std::exp(-(double)d / T)) {
                total += d;
            } else {
                swap_vars();
                for (int c : keep) remax(c);
            }
        }
        // the best state of the cold half of the schedule (the hot half
        // only wanders; snapshotting it would copy the layout thousands of
        // times)
        if (2 * it >= iters && total < best) {
            best = total;
            best_sigma = L.sigma;
            best_slot = L.slot;
            best_order = L.order;
        }
    }
    if (best < total) {  // else the final state is the best one seen
        L.sigma = best_sigma;
        L.slot = best_slot;
        L.order = best_order;
    }
    return L;
}

// Row positions for the serial chunk kernel.  In a layer the kernel spreads
// (row, shot) pairs over the lanes, 32 / CS rows per lane step; for edge j of
// its row a lane stores to slot j * MP + pos(row) and gathers the messages of
// the edge's variable from the slots j' * MP + pos(row') of its other rows.
// With MP a multiple of 32, slot s of shot sh sits in bank
// (pos + 4 sh) mod 32, so the accesses of one instruction conflict when the
// positions they touch collide mod 32.  Simulated annealing over a
// permutation of the positions 0..M-1 minimizes the summed worst bank load
// of every (layer, lane step, j, access) group; the arithmetic is unchanged
// (the gathers keep ascending row order), only bank conflicts change.
std::vector<int> serial_positions(const std::vector<std::vector<int>>& rcols, const std::vector<int>& layer_of,
                                  const std::vector<int>& idx_in_layer, int CS, int DC, int n, uint64_t seed) {
    const int M = (int)rcols.size();
    std::vector<int> pos(M);
    for (int r = 0; r < M; ++r) pos[r] = r;
    if (M < 2) return pos;
    std::vector<std::vector<int>> vrows(n);  // rows of each variable, ascending
    for (int r = 0; r < M; ++r)
        for (int v : rcols[r]) vrows[v].push_back(r);
    int maxdv = 1;
    for (int v = 0; v < n; ++v) maxdv = std::max(maxdv, (int)vrows[v].size());
    const int A = maxdv;  // accesses per edge: the store and up to maxdv - 1 gathers
    const int rpg = std::max(1, 32 / CS);
    // cell of (layer, lane step, j, access)
    int nl = 0, maxg = 0;
    for (int r = 0; r < M; ++r) {
        nl = std::max(nl, layer_of[r] + 1);
        maxg = std::max(maxg, idx_in_layer[r] / rpg + 1);
    }
    auto cell = [&](int L, int gidx, int j, int a) { return ((L * maxg + gidx) * DC + j) * A + a; };
    const int ncell = nl * maxg * DC * A;
    std::vector<std::vector<int>> target_cells(M);  // cells each row's position appears in
    for (int r = 0; r < M; ++r) {
        const int L = layer_of[r], gidx = idx_in_layer[r] / rpg;
        for (int j = 0; j < (int)rcols[r].size() && j < DC; ++j) {
            target_cells[r].push_back(cell(L, gidx, j, 0));
            int a = 1;
            for (int r2 : vrows[rcols[r][j]])
                if (r2 != r && a < A) target_cells[r2].push_back(cell(L, gidx, j, a++));
        }
    }
    std::vector<int> cnt((size_t)ncell * 32, 0), mx(ncell, 0);
    auto add = [&](int r, int d) {
        for (int c : target_cells[r])
            for (int sh = 0; sh < CS; ++sh) cnt[(size_t)c * 32 + ((pos[r] + 4 * sh) & 31)] += d;
    };
    // cost of a cell: its largest bank count first, then its colliding access
    // pairs (as in the small-code layout)
    auto remax = [&](int c) {
        int x = 0, pairs = 0;
        for (int k = 0; k < 32; ++k) {
            const int q = cnt[(size_t)c * 32 + k];
            x = std::max(x, q);
            pairs += q * (q - 1) / 2;
        }
        mx[c] = x * 1024 + pairs;
    };
    for (int r = 0; r < M; ++r) add(r, 1);
    for (int c = 0; c < ncell; ++c) remax(c);
    uint64_t rs = seed;
    auto rnd = [&]() {
        rs += 0x9E3779B97F4A7C15ULL;
        uint64_t z = rs;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        return z ^ (z >> 31);
    };
    std::vector<int> cells;
    const int iters = 12000;
    for (int it = 0; it < iters; ++it) {
        const double T = 0.6 * (1.0 - (double)it / iters) + 0.02;
        const int a = (int)(rnd() % M), b = (int)(rnd() % M);
        if (a == b || ((pos[a] ^ pos[b]) & 31) == 0) continue;
        cells.clear();
        for (int r : {a, b}) cells.insert(cells.end(), target_cells[r].begin(), target_cells[r].end());
        std::sort(cells.begin(), cells.end());
        cells.erase(std::unique(cells.begin(), cells.end()), cells.end());
        long before = 0, after = 0;
        for (int c : cells) before += mx[c];
        add(a, -1);
        add(b, -1);
        std::swap(pos[a], pos[b]);
        add(a, 1);
        add(b, 1);
        for (int c : cells) { remax(c); after += mx[c]; }
        const long d = after - before;
        const double u = (double)(rnd() >> 11) * (1.0 / 9007199254740992.0);
        if (!(d <= 0 || u < std::exp(-(double)d / T))) {
            add(a, -1);
            add(b, -1);
            std::swap(pos[a], pos[b]);
            add(a, 1);
            add(b, 1);
            for (int c : cells) remax(c);
        }
    }
    return pos;
}

mbbp_status build_impl(const uint8_t* H, int m, int n, int R, const int32_t* set_ptr,
                       const int32_t* set_rows, mbbp_bases** out) {
    if (!out) return fail(MBBP_E_INVALID, "out is NULL");
    *out = nullptr;
    if (R < 1 || R > MBBP_MAX_R) return fail(MBBP_E_INVALID, "R must be in [1, 64]");
    if (!set_ptr || (set_ptr[R] > 0 && !set_rows)) return fail(MBBP_E_INVALID, "sets are NULL");
    Tanner g;
    if (mbbp_status st = make_tanner(H, m, n, g)) return st;
    int dc = 0;
    bool regular = true;
    for (int r = 0; r < m; ++r) dc = std::max(dc, (int)g.rcols[r].size());
    for (int r = 0; r < m; ++r) regular = regular && ((int)g.rcols[r].size() == dc);
    if (dc < 1) return fail(MBBP_E_INVALID, "H has no nonzero entry");
    if (set_ptr[0] != 0) return fail(MBBP_E_INVALID, "set_ptr[0] must be 0");
    int maxM = 0;
    for (int t = 0; t < R; ++t) {
        if (set_ptr[t + 1] < set_ptr[t]) return fail(MBBP_E_INVALID, "set_ptr must be non-decreasing");
        for (int i = set_ptr[t]; i < set_ptr[t + 1]; ++i)
            if (set_rows[i] < 0 || set_rows[i] >= m) return fail(MBBP_E_INVALID, "set row out of range");
        maxM = std::max(maxM, m + set_ptr[t + 1] - set_ptr[t]);
    }
    if (maxM > MBBP_MAX_ROWS) return fail(MBBP_E_TOO_LARGE, "a representation has more than 1024 rows");
    // Variable degrees in every H^(t).
    int dv = 0;
    for (int t = 0; t < R; ++t) {
        std::vector<int> deg(n, 0);
        for (int r = 0; r < m; ++r)
            for (int v : g.rcols[r]) ++deg[v];
        for (int i = set_ptr[t]; i < set_ptr[t + 1]; ++i)
            for (int v : g.rcols[set_rows[i]]) ++deg[v];
        for (int v = 0; v < n; ++v) dv = std::max(dv, deg[v]);
    }
    const int need = std::max(dc, dv);
    int K = 0;
    for (int cand : {6, 8, 12})
        if (need <= cand) { K = cand; break; }
    if (K == 0) return fail(MBBP_E_TOO_LARGE, "row or column weight above 12");
    const int MP = round_up(maxM, 32);
    if ((long long)K * MP > MBBP_MAX_SLOTS) return fail(MBBP_E_TOO_LARGE, "too many edge slots");
    const int mpad = round_up(m, 32), W = words_for(n);

    mbbp_bases* B = new (std::nothrow) mbbp_bases();
    if (!B) return fail(MBBP_E_NOMEM, "host allocation failed");
    B->m = m; B->n = n; B->R = R; B->K = K; B->DV = dv; B->MP = MP; B->mpad = mpad;
    B->W = W; B->regular = (regular && dc == K) ? 1 : 0;  // every row fills the kernel width
    B->H.assign(H, H + (size_t)m * n);
    B->set_ptr.assign(set_ptr, set_ptr + R + 1);
    B->set_rows.assign(set_rows ? set_rows : set_ptr, set_rows ? set_rows + set_ptr[R] : set_ptr);

    std::vector<uint32_t> rowinfo((size_t)R * MP, 0);
    std::vector<int32_t> rowptr((size_t)R * MP, 0);
    std::vector<uint2> vdesc((size_t)R * n);
    std::vector<uint16_t> vslot;
    // width 6: the slot list packed into the descriptor itself (byte offsets
    // of up to 6 slots, ascending row), so the variable pass needs no second
    // dependent load
    std::vector<uint4> vdesc6(K == 6 ? (size_t)R * n : 0, make_uint4(0, 0, 0, 0));
    std::vector<int32_t> rows(R), edges(R);
    std::vector<uint2> evar((size_t)R * K * MP, make_uint2(0, 0));
    // chunked serial path (widths 6 and 8): per-edge and per-variable slot
    // descriptors with byte offsets, padded with the -0.0f slot
    const bool chunked = (K == 6 || K == 8);
    const uint32_t negz = 4u * (uint32_t)(K * MP);
    std::vector<uint4> edesc(chunked ? (size_t)R * K * MP : 0, make_uint4(0, 0, 0, 0));
    std::vector<uint4> vdesc3(chunked ? (size_t)R * n : 0, make_uint4(0, 0, 0, 0));
    std::vector<uint16_t> lpos(chunked ? (size_t)R * MP : 0, 0);
    std::vector<uint32_t> rinfo_s(chunked ? (size_t)R * MP : 0, 0);
    B->lorder.assign((size_t)R * MP, 0);
    B->lptr.assign((size_t)R * (MP + 1), 0);
    B->nlayers.assign(R, 0);
    for (int t = 0; t < R; ++t) {
        const int extra = set_ptr[t + 1] - set_ptr[t];
        const int M = m + extra;
        rows[t] = M;
        std::vector<std::vector<uint16_t>> vl(n);
        int E = 0;
        for (int r = 0; r < M; ++r) {
            const int src = r < m ? r : set_rows[set_ptr[t] + (r - m)];
            const auto& cols = g.rcols[src];
            rowinfo[(size_t)t * MP + r] = (uint32_t)src | ((uint32_t)cols.size() << 16) | (1u << 31);
            rowptr[(size_t)t * MP + r] = E;
            for (int j = 0; j < (int)cols.size(); ++j) vl[cols[j]].push_back((uint16_t)(j * MP + r));
            E += (int)cols.size();
        }
        edges[t] = E;
        std::vector<int> ord(n);
        for (int v = 0; v < n; ++v) ord[v] = v;
        std::stable_sort(ord.begin(), ord.end(),
                         [&](int a, int b) { return vl[a].size() < vl[b].size(); });
        std::vector<uint2> vstart(n);
        for (int p = 0; p < n; ++p) {
            const int v = ord[p];
            uint2 d;
            d.x = (uint32_t)vslot.size();
            d.y = (uint32_t)v | ((uint32_t)vl[v].size() << 16);
            vdesc[(size_t)t * n + p] = d;
            vstart[v] = d;
            vslot.insert(vslot.end(), vl[v].begin(), vl[v].end());
            if (K == 6) {
                uint32_t o[6] = {0, 0, 0, 0, 0, 0};
                for (int i = 0; i < (int)vl[v].size() && i < 6; ++i) o[i] = 4u * vl[v][i];
                vdesc6[(size_t)t * n + p] = make_uint4(d.y, o[0] | (o[1] << 16), o[2] | (o[3] << 16), o[4] | (o[5] << 16));
            }
        }
        // Serial schedule: every edge slot points at its variable's slot list;
        // rows go, in row order, into the first layer holding none of their
        // variables.
        std::vector<std::vector<uint8_t>> layer_vars;
        std::vector<int> layer_of(M);
        for (int r = 0; r < M; ++r) {
            const int src = r < m ? r : set_rows[set_ptr[t] + (r - m)];
            const auto& cols = g.rcols[src];
            for (int j = 0; j < (int)cols.size(); ++j) evar[(size_t)t * K * MP + (size_t)j * MP + r] = vstart[cols[j]];
            size_t L = 0;
            for (; L < layer_vars.size(); ++L) {
                bool clash = false;
                for (int v : cols) clash = clash || layer_vars[L][v];
                if (!clash) break;
            }
            if (L == layer_vars.size()) layer_vars.emplace_back(n, 0);
            for (int v : cols) layer_vars[L][v] = 1;
            layer_of[r] = (int)L;
        }
        const int nl = (int)layer_vars.size();
        int32_t* lo = B->lorder.data() + (size_t)t * MP;
        int32_t* lp = B->lptr.data() + (size_t)t * (MP + 1);
        int pos = 0;
        for (int L = 0; L < nl; ++L) {
            lp[L] = pos;
            for (int r = 0; r < M; ++r)
                if (layer_of[r] == L) lo[pos++] = r;
        }
        lp[nl] = pos;
        B->nlayers[t] = nl;
        if (chunked) {
            // chunk kernel: rows at bank-aware positions, descriptors by position
            std::vector<std::vector<int>> rc(M);
            std::vector<int> idx_in(M);
            for (int r = 0; r < M; ++r) {
                const int src = r < m ? r : set_rows[set_ptr[t] + (r - m)];
                rc[r] = g.rcols[src];
            }
            for (int L = 0; L < nl; ++L)
                for (int i = lp[L]; i < lp[L + 1]; ++i) idx_in[lo[i]] = i - lp[L];
            const int CS = serial_bp::shots_per_warp(K, MP, mpad, n);
            const std::vector<int> sp = serial_positions(rc, layer_of, idx_in, CS, K, n, 0xBA4Cull + (uint64_t)t);
            for (int i = 0; i < M; ++i) lpos[(size_t)t * MP + i] = (uint16_t)sp[lo[i]];
            for (int r = 0; r < M; ++r) {
                const int src = r < m ? r : set_rows[set_ptr[t] + (r - m)];
                rinfo_s[(size_t)t * MP + sp[r]] = (uint32_t)src | ((uint32_t)rc[r].size() << 16);
            }
            auto pack = [](const uint32_t* o) {
                return make_uint4(o[0] | (o[1] << 16), o[2] | (o[3] << 16), o[4] | (o[5] << 16),
                                  o[6] | (o[7] << 16));
            };
            // slot j * MP + r of the logical layout -> byte offset of j * MP + pos(r)
            auto off = [&](uint32_t slot) { return 4u * (uint32_t)((slot / MP) * MP + sp[slot % MP]); };
            for (int v = 0; v < n; ++v) {
                uint32_t o[8];
                for (int i = 0; i < 8; ++i) o[i] = i < (int)vl[v].size() ? off(vl[v][i]) : negz;
                vdesc3[(size_t)t * n + v] = pack(o);
                for (int k = 0; k < (int)vl[v].size(); ++k) {
                    uint32_t e[8];
                    e[0] = (uint32_t)v;
                    int c = 1;
                    for (int i = 0; i < (int)vl[v].size(); ++i)
                        if (i != k) e[c++] = off(vl[v][i]);
                    while (c < 8) e[c++] = negz;
                    edesc[(size_t)t * K * MP + off(vl[v][k]) / 4] = pack(e);
                }
            }
        }
    }
    std::vector<uint16_t> lrows16(B->lorder.begin(), B->lorder.end());
    std::vector<uint16_t> lptr16(B->lptr.begin(), B->lptr.end());
    // Small-code tables (register-resident kernel), when a shape fits.
    int shape = 0;
    if (K == 6)
        for (int i = 0; i < kNumSmallShapes && !shape; ++i)
            if (n <= 32 * kSmallShapes[i].VS && MP <= 32 * kSmallShapes[i].RS &&
                m <= 32 * kSmallShapes[i].ORS)
                shape = i + 1;
    std::vector<uint4> vdesc2;
    std::vector<uint32_t> rinfo2, hmask2;
    std::vector<int32_t> sedge;  // [R][6*MP] edge id (row by row, columns ascending) of every slot, or -1
    int VS = 0, RS = 0, ORS = 0;
    if (shape) {
        VS = kSmallShapes[shape - 1].VS;
        RS = kSmallShapes[shape - 1].RS;
        ORS = kSmallShapes[shape - 1].ORS;
        vdesc2.assign((size_t)R * VS * 32, make_uint4(0, 0, 0, 0));
        rinfo2.assign((size_t)R * MP, 0);
        hmask2.assign((size_t)R * VS * ORS * 32, 0);
        sedge.assign((size_t)R * 6 * MP, -1);
        // the bank placements of the R representations are independent:
        // anneal them on the host's cores
        std::vector<SmallLayout> layouts(R);
        {
            const int nth = std::max(1, std::min(R, (int)std::thread::hardware_concurrency()));
            std::atomic<int> next{0};
            auto worker = [&]() {
                for (int t = next++; t < R; t = next++) {
                    const int extra = set_ptr[t + 1] - set_ptr[t];
                    std::vector<int> src(m + extra);
                    for (int r = 0; r < m + extra; ++r) src[r] = r < m ? r : set_rows[set_ptr[t] + (r - m)];
                    layouts[t] = small_layout(g, src, n, MP, 0x5EEDull + (uint64_t)t);
                }
            };
            std::vector<std::thread> pool;
            for (int i = 1; i < nth; ++i) pool.emplace_back(worker);
            worker();
            for (auto& th : pool) th.join();
        }
        for (int t = 0; t < R; ++t) {
            const int extra = set_ptr[t + 1] - set_ptr[t];
            std::vector<int> src(m + extra);
            for (int r = 0; r < m + extra; ++r) src[r] = r < m ? r : set_rows[set_ptr[t] + (r - m)];
            const SmallLayout& L = layouts[t];
            std::vector<int> posof(n);
            for (int p = 0; p < n; ++p) posof[L.order[p]] = p;
            std::vector<std::vector<uint16_t>> vs(n);
            for (int r = 0; r < (int)src.size(); ++r) {
                const auto& cols = g.rcols[src[r]];
                const int sg = L.sigma[r];
                rinfo2[(size_t)t * MP + sg] = (uint32_t)src[r] | ((uint32_t)cols.size() << 16);
                for (int j = 0; j < (int)cols.size(); ++j) {
                    const int sj = L.slot[r][j];
                    const int sl = sj * MP + (sg & ~31) + ((sg + slot_rot(sj)) & 31);
                    vs[cols[j]].push_back((uint16_t)sl);
                    sedge[(size_t)t * 6 * MP + sl] = rowptr[(size_t)t * MP + r] + j;
                }
            }
            // byte offsets within a warp's message area; a missing edge (and
            // every edge of a padding position) points at the zero slot
            const uint16_t zero_slot = (uint16_t)(4 * 6 * MP);
            for (int p = n; p < VS * 32; ++p) {
                const uint32_t z = zero_slot | ((uint32_t)zero_slot << 16);
                vdesc2[(size_t)t * VS * 32 + p] = make_uint4(0, z, z, z);
            }
            for (int p = 0; p < n; ++p) {
                const int v = L.order[p];
                uint16_t sl[6] = {zero_slot, zero_slot, zero_slot, zero_slot, zero_slot, zero_slot};
                for (int i = 0; i < (int)vs[v].size(); ++i) sl[i] = (uint16_t)(4 * vs[v][i]);
                uint4 d;
                d.x = (uint32_t)v | ((uint32_t)vs[v].size() << 16);
                d.y = sl[0] | ((uint32_t)sl[1] << 16);
                d.z = sl[2] | ((uint32_t)sl[3] << 16);
                d.w = sl[4] | ((uint32_t)sl[5] << 16);
                vdesc2[(size_t)t * VS * 32 + p] = d;
            }
            for (int r = 0; r < m; ++r)
                for (int c : g.rcols[r]) {
                    const int pp = posof[c];
                    hmask2[((size_t)t * VS + (pp >> 5)) * (ORS * 32) + r] |= 1u << (pp & 31);
                }
        }
    }

    std::vector<uint16_t> hcol((size_t)K * mpad, (uint16_t)n);
    std::vector<uint32_t> hmask((size_t)m * W, 0);
    for (int r = 0; r < m; ++r)
        for (int j = 0; j < (int)g.rcols[r].size(); ++j) {
            const int v = g.rcols[r][j];
            hcol[(size_t)j * mpad + r] = (uint16_t)v;
            hmask[(size_t)r * W + (v >> 5)] |= 1u << (v & 31);
        }
    B->rows = rows;
    B->edges = edges;

    // One device allocation for all tables.
    const size_t o_rowinfo = 0;
    const size_t o_vdesc = o_rowinfo + align256(rowinfo.size() * 4);
    const size_t o_vslot = o_vdesc + align256(vdesc.size() * sizeof(uint2));
    const size_t o_rows = o_vslot + align256(std::max<size_t>(vslot.size(), 1) * 2);
    const size_t o_hcol = o_rows + align256(rows.size() * 4);
    const size_t o_hmask = o_hcol + align256(hcol.size() * 2);
    const size_t o_rowptr = o_hmask + align256(hmask.size() * 4);
    const size_t o_vdesc2 = o_rowptr + align256(rowptr.size() * 4);
    const size_t o_rinfo2 = o_vdesc2 + align256(vdesc2.size() * sizeof(uint4));
    const size_t o_hmask2 = o_rinfo2 + align256(rinfo2.size() * 4);
    const size_t o_lrows = o_hmask2 + align256(hmask2.size() * 4);
    const size_t o_lptr = o_lrows + align256(lrows16.size() * 2);
    const size_t o_nlayers = o_lptr + align256(lptr16.size() * 2);
    const size_t o_evar = o_nlayers + align256((size_t)R * 4);
    const size_t o_edesc = o_evar + align256(evar.size() * sizeof(uint2));
    const size_t o_vdesc3 = o_edesc + align256(edesc.size() * sizeof(uint4));
    const size_t o_lpos = o_vdesc3 + align256(vdesc3.size() * sizeof(uint4));
    const size_t o_rinfo_s = o_lpos + align256(lpos.size() * 2);
    const size_t o_sedge = o_rinfo_s + align256(rinfo_s.size() * 4);
    const size_t o_vdesc6 = o_sedge + align256(sedge.size() * 4);
    const size_t total = o_vdesc6 + align256(vdesc6.size() * sizeof(uint4));
    cudaError_t e = cudaGetDevice(&B->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&B->sm_count, cudaDevAttrMultiProcessorCount, B->device);
    if (e == cudaSuccess) e = cudaMalloc(&B->dmem, total);
    if (e != cudaSuccess) {
        delete B;
        return cuda_fail(e, "mbbp_build_bases");
    }
    char* base = static_cast<char*>(B->dmem);
    struct Copy { size_t off; const void* src; size_t bytes; } copies[] = {
        {o_rowinfo, rowinfo.data(), rowinfo.size() * 4},
        {o_vdesc, vdesc.data(), vdesc.size() * sizeof(uint2)},
        {o_vslot, vslot.data(), vslot.size() * 2},
        {o_rows, rows.data(), rows.size() * 4},
        {o_hcol, hcol.data(), hcol.size() * 2},
        {o_hmask, hmask.data(), hmask.size() * 4},
        {o_rowptr, rowptr.data(), rowptr.size() * 4},
        {o_vdesc2, vdesc2.data(), vdesc2.size() * sizeof(uint4)},
        {o_rinfo2, rinfo2.data(), rinfo2.size() * 4},
        {o_hmask2, hmask2.data(), hmask2.size() * 4},
        {o_lrows, lrows16.data(), lrows16.size() * 2},
        {o_lptr, lptr16.data(), lptr16.size() * 2},
        {o_nlayers, B->nlayers.data(), (size_t)R * 4},
        {o_evar, evar.data(), evar.size() * sizeof(uint2)},
        {o_edesc, edesc.data(), edesc.size() * sizeof(uint4)},
        {o_vdesc3, vdesc3.data(), vdesc3.size() * sizeof(uint4)},
        {o_lpos, lpos.data(), lpos.size() * 2},
        {o_rinfo_s, rinfo_s.data(), rinfo_s.size() * 4},
        {o_sedge, sedge.data(), sedge.size() * 4},
        {o_vdesc6, vdesc6.data(), vdesc6.size() * sizeof(uint4)},
    };
    for (const Copy& c : copies) {
        if (c.bytes == 0) continue;
        e = cudaMemcpy(base + c.off, c.src, c.bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(B->dmem);
            delete B;
            return cuda_fail(e, "mbbp_build_bases copy");
        }
    }
    DevBases& d = B->dev;
    d.rowinfo = reinterpret_cast<const uint32_t*>(base + o_rowinfo);
    d.vdesc = reinterpret_cast<const uint2*>(base + o_vdesc);
    d.vslot = reinterpret_cast<const uint16_t*>(base + o_vslot);
    d.rows = reinterpret_cast<const int32_t*>(base + o_rows);
    d.hcol = reinterpret_cast<const uint16_t*>(base + o_hcol);
    d.hmask = reinterpret_cast<const uint32_t*>(base + o_hmask);
    d.rowptr = reinterpret_cast<const int32_t*>(base + o_rowptr);
    d.m = m; d.n = n; d.R = R; d.DC = K; d.DV = dv; d.MP = MP; d.mpad = mpad; d.W = W;
    d.regular = B->regular;
    d.shape = shape;
    d.VS = VS;
    d.RS = RS;
    d.ORS = ORS;
    d.vdesc2 = shape ? reinterpret_cast<const uint4*>(base + o_vdesc2) : nullptr;
    d.rinfo2 = shape ? reinterpret_cast<const uint32_t*>(base + o_rinfo2) : nullptr;
    d.hmask2 = shape ? reinterpret_cast<const uint32_t*>(base + o_hmask2) : nullptr;
    d.sedge = shape ? reinterpret_cast<const int32_t*>(base + o_sedge) : nullptr;
    d.vdesc6 = K == 6 ? reinterpret_cast<const uint4*>(base + o_vdesc6) : nullptr;
    d.lrows = reinterpret_cast<const uint16_t*>(base + o_lrows);
    d.lptr = reinterpret_cast<const uint16_t*>(base + o_lptr);
    d.nlayers = reinterpret_cast<const int32_t*>(base + o_nlayers);
    d.evar = reinterpret_cast<const uint2*>(base + o_evar);
    d.edesc = chunked ? reinterpret_cast<const uint4*>(base + o_edesc) : nullptr;
    d.vdesc3 = chunked ? reinterpret_cast<const uint4*>(base + o_vdesc3) : nullptr;
    d.lpos = chunked ? reinterpret_cast<const uint16_t*>(base + o_lpos) : nullptr;
    d.rinfo_s = chunked ? reinterpret_cast<const uint32_t*>(base + o_rinfo_s) : nullptr;
    *out = B;
    return MBBP_OK;
}

mbbp_status check_device(int device) {
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (cur != device) return fail(MBBP_E_INVALID, "handle belongs to another device");
    return MBBP_OK;
}

// GF(2) row reduction on bit-packed rows (uint64 words).
struct Gf2Rows {
    int n = 0, words = 0;
    std::vector<std::vector<uint64_t>> rows;  // reduced rows
    std::vector<int> pivots;                  // pivot column of each row
    explicit Gf2Rows(int n_) : n(n_), words((n_ + 63) / 64) {}
    static bool get(const std::vector<uint64_t>& x, int c) { return (x[c >> 6] >> (c & 63)) & 1ull; }
    void reduce(std::vector<uint64_t>& x) const {
        for (size_t i = 0; i < rows.size(); ++i)
            if (get(x, pivots[i]))
                for (int w = 0; w < words; ++w) x[w] ^= rows[i][w];
    }
    // Adds x if it is independent; returns whether it was.
    bool insert(std::vector<uint64_t> x) {
        reduce(x);
        int piv = -1;
        for (int c = 0; c < n && piv < 0; ++c)
            if (get(x, c)) piv = c;
        if (piv < 0) return false;
        for (size_t i = 0; i < rows.size(); ++i)
            if (get(rows[i], piv))
                for (int w = 0; w < words; ++w) rows[i][w] ^= x[w];
        rows.push_back(std::move(x));
        pivots.push_back(piv);
        return true;
    }
};

std::vector<uint64_t> pack_row(const uint8_t* row, int n) {
    std::vector<uint64_t> x((n + 63) / 64, 0);
    for (int c = 0; c < n; ++c)
        if (row[c]) x[c >> 6] |= 1ull << (c & 63);
    return x;
}

}  // namespace

extern "C" {

const char* mbbp_last_error(void) { return g_err.c_str(); }

const char* mbbp_version(void) { return "mbbp-gb300 0.1 (sm_103a)"; }

mbbp_status mbbp_permutation(uint64_t seed, int j, int m, int32_t* perm) {
    if (!perm || m < 1 || j < 0) return fail(MBBP_E_INVALID, "mbbp_permutation: bad arguments");
    permutation_impl(seed, j, m, perm);
    return MBBP_OK;
}

mbbp_status mbbp_subtrees(const uint8_t* H, int m, int n, const int32_t* perm,
                          int32_t* check_sets, int32_t* order, int32_t* n_subtrees) {
    if (!perm || !check_sets) return fail(MBBP_E_INVALID, "mbbp_subtrees: NULL argument");
    Tanner g;
    if (mbbp_status st = make_tanner(H, m, n, g)) return st;
    std::vector<char> seen(m, 0);
    for (int i = 0; i < m; ++i) {
        if (perm[i] < 0 || perm[i] >= m || seen[perm[i]])
            return fail(MBBP_E_INVALID, "perm is not a permutation of 0..m-1");
        seen[perm[i]] = 1;
    }
    const int s = subtrees_impl(g, perm, check_sets, order);
    if (n_subtrees) *n_subtrees = s;
    return MBBP_OK;
}

mbbp_status mbbp_collect_subtrees(const uint8_t* H, int m, int n, int R, uint64_t seed,
                                  int32_t* set_ptr, int32_t* set_rows) {
    if (!set_ptr || !set_rows) return fail(MBBP_E_INVALID, "mbbp_collect_subtrees: NULL output");
    if (R < 1 || R > MBBP_MAX_R) return fail(MBBP_E_INVALID, "R must be in [1, 64]");
    Tanner g;
    if (mbbp_status st = make_tanner(H, m, n, g)) return st;
    std::vector<int32_t> ptr, rows;
    if (mbbp_status st = collect_impl(g, R, seed, ptr, rows)) return st;
    std::copy(ptr.begin(), ptr.end(), set_ptr);
    std::copy(rows.begin(), rows.end(), set_rows);
    return MBBP_OK;
}

mbbp_status mbbp_build_bases(const uint8_t* H, int m, int n, int R, uint64_t seed,
                             mbbp_bases** out) {
    if (out) *out = nullptr;
    if (R < 1 || R > MBBP_MAX_R) return fail(MBBP_E_INVALID, "R must be in [1, 64]");
    Tanner g;
    if (mbbp_status st = make_tanner(H, m, n, g)) return st;
    std::vector<int32_t> ptr, rows;
    if (mbbp_status st = collect_impl(g, R, seed, ptr, rows)) return st;
    return build_impl(H, m, n, R, ptr.data(), rows.data(), out);
}

mbbp_status mbbp_build_bases_from_sets(const uint8_t* H, int m, int n, int R,
                                       const int32_t* set_ptr, const int32_t* set_rows,
                                       mbbp_bases** out) {
    return build_impl(H, m, n, R, set_ptr, set_rows, out);
}

mbbp_status mbbp_bases_info(const mbbp_bases* B, int32_t* m, int32_t* n, int32_t* R,
                            int32_t* rows, int32_t* edges, int32_t* set_ptr, int32_t* set_rows) {
    if (!B) return fail(MBBP_E_INVALID, "mbbp_bases_info: NULL handle");
    if (m) *m = B->m;
    if (n) *n = B->n;
    if (R) *R = B->R;
    if (rows) std::copy(B->rows.begin(), B->rows.end(), rows);
    if (edges) std::copy(B->edges.begin(), B->edges.end(), edges);
    if (set_ptr) std::copy(B->set_ptr.begin(), B->set_ptr.end(), set_ptr);
    if (set_rows) std::copy(B->set_rows.begin(), B->set_rows.end(), set_rows);
    return MBBP_OK;
}

mbbp_status mbbp_bases_layers(const mbbp_bases* B, int t, int32_t* order, int32_t* layer_ptr,
                              int32_t* n_layers) {
    if (!B) return fail(MBBP_E_INVALID, "mbbp_bases_layers: NULL handle");
    if (t < 0 || t >= B->R) return fail(MBBP_E_INVALID, "mbbp_bases_layers: t out of range");
    const int M = B->rows[t], nl = B->nlayers[t];
    if (order) std::copy_n(B->lorder.begin() + (size_t)t * B->MP, M, order);
    if (layer_ptr) std::copy_n(B->lptr.begin() + (size_t)t * (B->MP + 1), nl + 1, layer_ptr);
    if (n_layers) *n_layers = nl;
    return MBBP_OK;
}

mbbp_status mbbp_random_sets(int m, int R, const int32_t* sizes, uint64_t seed, int32_t* set_ptr,
                             int32_t* set_rows) {
    if (m < 1 || R < 0) return fail(MBBP_E_INVALID, "mbbp_random_sets: bad sizes");
    if (R > 0 && (!sizes || !set_ptr)) return fail(MBBP_E_INVALID, "mbbp_random_sets: NULL buffer");
    if (R == 0) {
        if (set_ptr) set_ptr[0] = 0;
        return MBBP_OK;
    }
    for (int t = 0; t < R; ++t)
        if (sizes[t] < 0) return fail(MBBP_E_INVALID, "mbbp_random_sets: negative size");
    std::vector<int32_t> perm(m);
    set_ptr[0] = 0;
    for (int t = 0; t < R; ++t) {
        permutation_impl(seed, t + 1, m, perm.data());
        const int k = std::min(sizes[t], m);
        if (k > 0 && !set_rows) return fail(MBBP_E_INVALID, "mbbp_random_sets: set_rows is NULL");
        std::copy_n(perm.begin(), k, set_rows + set_ptr[t]);
        set_ptr[t + 1] = set_ptr[t] + k;
    }
    return MBBP_OK;
}

void mbbp_bases_free(mbbp_bases* B) {
    if (!B) return;
    if (B->dmem) cudaFree(B->dmem);
    delete B;
}

mbbp_status mbbp_sample_errors(int n, int batch, uint64_t first_shot, uint64_t seed, double p,
                               int noise, uint32_t* ex, uint32_t* ez, void* stream) {
    if (n < 1 || n > MBBP_MAX_N || batch < 0) return fail(MBBP_E_INVALID, "mbbp_sample_errors: bad sizes");
    if (!(p >= 0.0 && p < 1.0)) return fail(MBBP_E_INVALID, "p must be in [0, 1)");
    if (noise != MBBP_NOISE_BSC && noise != MBBP_NOISE_DEPOLARIZING)
        return fail(MBBP_E_INVALID, "unknown noise model");
    if (!ex) return fail(MBBP_E_INVALID, "ex is NULL");
    if (batch == 0) return MBBP_OK;
    const uint64_t T = (uint64_t)std::ldexp(p, 64);
    cudaError_t e = launch_sample(n, batch, first_shot, seed, T, noise, ex, ez, (cudaStream_t)stream);
    return e == cudaSuccess ? MBBP_OK : cuda_fail(e, "mbbp_sample_errors");
}

mbbp_status mbbp_syndrome(const mbbp_bases* B, int batch, const uint32_t* e, uint8_t* s,
                          void* stream) {
    if (!B || batch < 0) return fail(MBBP_E_INVALID, "mbbp_syndrome: bad arguments");
    if (batch == 0) return MBBP_OK;
    if (!e || !s) return fail(MBBP_E_INVALID, "mbbp_syndrome: NULL buffer");
    if (mbbp_status st = check_device(B->device)) return st;
    cudaError_t err = launch_syndrome(B->dev, batch, e, s, (cudaStream_t)stream);
    return err == cudaSuccess ? MBBP_OK : cuda_fail(err, "mbbp_syndrome");
}

size_t mbbp_decode_workspace_size(const mbbp_bases* B, int batch) {
    if (!B || batch < 0) return 0;
    // candidates, then the work counter (8 bytes) and one shot counter per
    // representation (4 bytes each)
    return align256((size_t)batch * B->R * B->W * 4) + 512;
}

mbbp_status mbbp_decode(const mbbp_bases* B, int batch, const uint8_t* syndromes,
                        const float* llr, int llr_stride, int iters, float alpha, int rule,
                        uint8_t* e_hat, uint8_t* conv, uint16_t* iters_run, uint8_t* success,
                        int16_t* selected, float* posterior, void* workspace,
                        size_t workspace_bytes, void* stream) {
    mbbp_options o{};
    o.rule = rule;
    o.alpha = alpha;
    o.schedule = MBBP_SCHEDULE_FLOODING;
    o.decision = MBBP_DECISION_FWS;
    return mbbp_decode_ex(B, batch, syndromes, llr, llr_stride, iters, &o, e_hat, conv, iters_run,
                          success, selected, posterior, workspace, workspace_bytes, stream);
}

namespace {

// Argument checks of mbbp_decode_ex, before any CUDA call (the workspace
// only when `need_ws`).  *launch = false when there is nothing to enqueue.
mbbp_status decode_validate(const mbbp_bases* B, int batch, const uint8_t* syndromes, const float* llr,
                            int llr_stride, int iters, const mbbp_options* opt, const uint8_t* e_hat,
                            const uint8_t* conv, const uint8_t* success, bool need_ws, const void* workspace,
                            size_t workspace_bytes, bool* launch) {
    *launch = false;
    if (!B) return fail(MBBP_E_INVALID, "mbbp_decode: NULL handle");
    if (!opt) return fail(MBBP_E_INVALID, "mbbp_decode_ex: NULL options");
    const int rule = opt->rule;
    const float alpha = opt->alpha;
    if (opt->schedule != MBBP_SCHEDULE_FLOODING && opt->schedule != MBBP_SCHEDULE_SERIAL)
        return fail(MBBP_E_INVALID, "unknown schedule");
    if (opt->decision != MBBP_DECISION_FWS && opt->decision != MBBP_DECISION_LMS)
        return fail(MBBP_E_INVALID, "unknown decision rule");
    if (batch < 0) return fail(MBBP_E_INVALID, "batch must be >= 0");
    if (iters < 0 || iters > MBBP_MAX_ITERS) return fail(MBBP_E_INVALID, "iters out of range");
    if (rule != MBBP_RULE_NMS && rule != MBBP_RULE_SP) return fail(MBBP_E_INVALID, "unknown rule");
    if (rule == MBBP_RULE_NMS && !(alpha > 0.f && alpha <= 1.f))
        return fail(MBBP_E_INVALID, "alpha must be in (0, 1]");
    if (llr_stride != 0 && llr_stride < B->n) return fail(MBBP_E_INVALID, "llr_stride must be 0 or >= n");
    if (batch == 0) return MBBP_OK;
    if (!syndromes || !llr || !e_hat || !conv || !success)
        return fail(MBBP_E_INVALID, "mbbp_decode: NULL buffer");
    if (need_ws) {
        if (!workspace) return fail(MBBP_E_INVALID, "mbbp_decode: NULL buffer");
        if (workspace_bytes < mbbp_decode_workspace_size(B, batch))
            return fail(MBBP_E_INVALID, "workspace too small");
        if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0)
            return fail(MBBP_E_INVALID, "workspace must be 256-byte aligned");
    }
    if (mbbp_status st = check_device(B->device)) return st;
    *launch = true;
    return MBBP_OK;
}

}  // namespace

namespace {

mbbp_status decode_impl(const mbbp_bases* B, int batch, const uint8_t* syndromes, const float* llr,
                        int llr_stride, int iters, const mbbp_options* opt, uint8_t* e_hat, uint8_t* conv,
                        uint16_t* iters_run, uint8_t* success, int16_t* selected, float* posterior,
                        void* workspace, size_t workspace_bytes, float* c2v, void* stream) {
    bool launch = false;
    if (mbbp_status st = decode_validate(B, batch, syndromes, llr, llr_stride, iters, opt, e_hat, conv, success,
                                         true, workspace, workspace_bytes, &launch))
        return st;
    if (!launch) return MBBP_OK;
    const int rule = opt->rule;
    const float alpha = opt->alpha;
    cudaStream_t s = (cudaStream_t)stream;
    DecodeArgs a{};
    a.B = B->dev;
    a.io.synd = syndromes;
    a.io.llr = llr;
    a.io.llr_stride = llr_stride;
    a.io.batch = batch;
    a.io.iters = iters;
    a.io.alpha = alpha;
    a.rule = rule;
    const size_t cand_bytes = align256((size_t)batch * B->R * B->W * 4);
    a.io.cand = static_cast<uint32_t*>(workspace);
    a.counter = reinterpret_cast<unsigned long long*>(static_cast<char*>(workspace) + cand_bytes);
    a.io.conv = conv;
    a.io.iters_run = iters_run;
    a.io.post = posterior;
    a.io.c2v = c2v;
    a.io.c2v_stride = *std::max_element(B->edges.begin(), B->edges.end());
    a.total_items = (unsigned long long)batch * B->R;
    a.rep_counter = reinterpret_cast<unsigned int*>(a.counter + 1);
    const size_t counter_bytes = sizeof(unsigned long long) + sizeof(unsigned int) * (size_t)B->R;
    cudaError_t e = cudaMemsetAsync(a.counter, 0, counter_bytes, s);
    if (e == cudaSuccess)
        e = opt->schedule == MBBP_SCHEDULE_SERIAL ? launch_decode_serial(a, s, B->sm_count)
                                                  : launch_decode(a, s, B->sm_count);
    if (e != cudaSuccess) return cuda_fail(e, "mbbp_decode (BP)");
    FwsArgs f{};
    f.cand = a.io.cand;
    f.conv = conv;
    f.batch = batch;
    f.R = B->R;
    f.n = B->n;
    f.W = B->W;
    f.e_hat = e_hat;
    f.success = success;
    f.selected = selected;
    f.decision = opt->decision;
    f.llr = llr;
    f.llr_stride = llr_stride;
    e = launch_fws(f, s);
    return e == cudaSuccess ? MBBP_OK : cuda_fail(e, "mbbp_decode (selection)");
}

}  // namespace

mbbp_status mbbp_decode_ex(const mbbp_bases* B, int batch, const uint8_t* syndromes,
                           const float* llr, int llr_stride, int iters, const mbbp_options* opt,
                           uint8_t* e_hat, uint8_t* conv, uint16_t* iters_run, uint8_t* success,
                           int16_t* selected, float* posterior, void* workspace,
                           size_t workspace_bytes, void* stream) {
    return decode_impl(B, batch, syndromes, llr, llr_stride, iters, opt, e_hat, conv, iters_run, success,
                       selected, posterior, workspace, workspace_bytes, nullptr, stream);
}

mbbp_status mbbp_decode_trace(const mbbp_bases* B, int batch, const uint8_t* syndromes,
                              const float* llr, int llr_stride, int iters, const mbbp_options* opt,
                              uint8_t* e_hat, uint8_t* conv, uint16_t* iters_run, uint8_t* success,
                              int16_t* selected, float* posterior, float* c2v, void* workspace,
                              size_t workspace_bytes, void* stream) {
    if (opt && opt->schedule != MBBP_SCHEDULE_FLOODING)
        return fail(MBBP_E_INVALID, "mbbp_decode_trace: flooding schedule only");
    if (!c2v && batch > 0) return fail(MBBP_E_INVALID, "mbbp_decode_trace: NULL c2v");
    return decode_impl(B, batch, syndromes, llr, llr_stride, iters, opt, e_hat, conv, iters_run, success,
                       selected, posterior, workspace, workspace_bytes, c2v, stream);
}

mbbp_status mbbp_decode_noalloc(const mbbp_bases* B, int batch, const uint8_t* syndromes,
                                const float* llr, int llr_stride, int iters, float alpha, int rule,
                                uint8_t* e_hat, uint8_t* conv, uint16_t* iters_run,
                                uint8_t* success, int16_t* selected, float* posterior,
                                void* stream) {
    if (!B) return fail(MBBP_E_INVALID, "mbbp_decode_noalloc: NULL handle");
    mbbp_options o{};
    o.rule = rule;
    o.alpha = alpha;
    o.schedule = MBBP_SCHEDULE_FLOODING;
    o.decision = MBBP_DECISION_FWS;
    // every argument is checked (and batch 0 returns) before the scratch
    // address is looked up, so a call that launches nothing makes no CUDA call
    bool launch = false;
    if (mbbp_status st = decode_validate(B, batch, syndromes, llr, llr_stride, iters, &o, e_hat, conv, success,
                                         false, nullptr, 0, &launch))
        return st;
    if (!launch) return MBBP_OK;
    const size_t need = mbbp_decode_workspace_size(B, batch);
    if (need > kStaticScratchBytes) {
        const size_t per_shot = (size_t)B->R * B->W * 4;
        const size_t max_batch = (kStaticScratchBytes - 512) / per_shot;
        return fail(MBBP_E_TOO_LARGE, "mbbp_decode_noalloc: batch " + std::to_string(batch) +
                                          " needs " + std::to_string(need) +
                                          " bytes of scratch; the fixed scratch holds " +
                                          std::to_string(kStaticScratchBytes) +
                                          " bytes (at most " + std::to_string(max_batch) +
                                          " shots for this handle)");
    }
    void* scratch = nullptr;
    cudaError_t e = static_scratch(&scratch);
    if (e != cudaSuccess) return cuda_fail(e, "mbbp_decode_noalloc (cudaGetSymbolAddress)");
    return mbbp_decode(B, batch, syndromes, llr, llr_stride, iters, alpha, rule, e_hat, conv,
                       iters_run, success, selected, posterior, scratch, kStaticScratchBytes,
                       stream);
}

// ------------------------------------------------------------ mixed batches

mbbp_status mbbp_plan_create(const mbbp_bases* const* codes, int n_codes, mbbp_plan** out) {
    if (!out) return fail(MBBP_E_INVALID, "out is NULL");
    *out = nullptr;
    if (!codes || n_codes < 1 || n_codes > kMixedMaxCodes)
        return fail(MBBP_E_INVALID, "n_codes must be in [1, 8]");
    int dev = -1;
    for (int c = 0; c < n_codes; ++c) {
        if (!codes[c]) return fail(MBBP_E_INVALID, "NULL code handle");
        if (c > 0 && codes[c]->device != dev) return fail(MBBP_E_INVALID, "codes on different devices");
        dev = codes[c]->device;
    }
    mbbp_plan* P = new (std::nothrow) mbbp_plan();
    if (!P) return fail(MBBP_E_NOMEM, "host allocation failed");
    P->codes.assign(codes, codes + n_codes);
    P->device = dev;
    P->sm_count = codes[0]->sm_count;
    P->chunk.assign(n_codes, 4);
    P->kind.resize(n_codes);
    for (int c = 0; c < n_codes; ++c)
        P->kind[c] = (codes[c]->dev.shape != 0 && codes[c]->regular) ? kKindSmall : kKindGeneric;
    // heaviest codes first: work = R * edges per representation
    std::vector<double> cost(n_codes);
    for (int c = 0; c < n_codes; ++c) {
        double e = 0;
        for (int t = 0; t < codes[c]->R; ++t) e += codes[c]->edges[t];
        cost[c] = e;
    }
    P->order.resize(n_codes);
    for (int c = 0; c < n_codes; ++c) P->order[c] = c;
    std::stable_sort(P->order.begin(), P->order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    *out = P;
    return MBBP_OK;
}

void mbbp_plan_free(mbbp_plan* P) { delete P; }

size_t mbbp_plan_workspace_size(const mbbp_plan* P, const int32_t* batches) {
    if (!P || !batches) return 0;
    static_assert(kMixedGroups * sizeof(unsigned long long) <= 256, "work counters");
    size_t total = 256;  // work counters
    for (size_t c = 0; c < P->codes.size(); ++c) {
        if (batches[c] < 0) return 0;
        total += align256((size_t)batches[c] * P->codes[c]->R * P->codes[c]->W * 4);
    }
    return total;
}

mbbp_status mbbp_plan_info(const mbbp_plan* P, int32_t* warps, int32_t* chunk, int32_t* kind,
                           int32_t* order) {
    if (!P) return fail(MBBP_E_INVALID, "mbbp_plan_info: NULL plan");
    if (warps) *warps = P->warps;
    for (size_t c = 0; c < P->codes.size(); ++c) {
        if (chunk) chunk[c] = P->chunk[c];
        if (kind) kind[c] = P->kind[c];
        if (order) order[c] = P->order[c];
    }
    return MBBP_OK;
}

namespace {

mbbp_status mixed_impl(const mbbp_plan* P, const mbbp_code_io* io, int iters, float alpha, int rule,
                       void* workspace, size_t workspace_bytes, cudaStream_t s) {
    const int nc = (int)P->codes.size();
    if (!io) return fail(MBBP_E_INVALID, "io is NULL");
    if (iters < 0 || iters > MBBP_MAX_ITERS) return fail(MBBP_E_INVALID, "iters out of range");
    if (rule != MBBP_RULE_NMS && rule != MBBP_RULE_SP) return fail(MBBP_E_INVALID, "unknown rule");
    if (rule == MBBP_RULE_NMS && !(alpha > 0.f && alpha <= 1.f))
        return fail(MBBP_E_INVALID, "alpha must be in (0, 1]");
    std::vector<int32_t> batches(nc);
    for (int c = 0; c < nc; ++c) {
        const mbbp_code_io& x = io[c];
        const mbbp_bases* B = P->codes[c];
        if (x.batch < 0) return fail(MBBP_E_INVALID, "batch must be >= 0");
        if (x.batch > 0 && (!x.syndromes || !x.llr || !x.e_hat || !x.conv || !x.success))
            return fail(MBBP_E_INVALID, "mbbp_decode_mixed: NULL buffer");
        if (x.llr_stride != 0 && x.llr_stride < B->n) return fail(MBBP_E_INVALID, "llr_stride must be 0 or >= n");
        batches[c] = x.batch;
    }
    if (!workspace || workspace_bytes < mbbp_plan_workspace_size(P, batches.data()))
        return fail(MBBP_E_INVALID, "workspace too small");
    if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0)
        return fail(MBBP_E_INVALID, "workspace must be 256-byte aligned");
    if (mbbp_status st = check_device(P->device)) return st;
    // one launch per kernel body and small-code shape (group), each with its
    // own work list and counter; the groups launch in the order their first
    // codes have in the plan
    MixedArgs args[kMixedGroups] = {};
    char* ws = static_cast<char*>(workspace);
    std::vector<uint32_t*> cand(nc);
    for (int c = 0; c < nc; ++c) {
        cand[c] = reinterpret_cast<uint32_t*>(ws);
        ws += align256((size_t)batches[c] * P->codes[c]->R * P->codes[c]->W * 4);
    }
    unsigned long long* counters = reinterpret_cast<unsigned long long*>(ws);
    unsigned long long firsts[kMixedGroups] = {};
    size_t wbytes[kMixedGroups];
    int slots[kMixedGroups] = {};
    std::vector<int> launch_order;
    for (int g = 0; g < kMixedGroups; ++g) wbytes[g] = 16;
    for (int oi = 0; oi < nc; ++oi) {
        const int c = P->order[oi];
        const mbbp_bases* B = P->codes[c];
        const mbbp_code_io& x = io[c];
        if (x.batch == 0) continue;
        const bool small = P->kind[c] == kKindSmall && B->dev.shape >= 1 && B->dev.shape <= kNumSmallShapes;
        const int g = small ? B->dev.shape : 0;
        if (std::find(launch_order.begin(), launch_order.end(), g) == launch_order.end())
            launch_order.push_back(g);
        MixedArgs& a = args[g];
        unsigned long long& first = firsts[g];
        MixedCode& mc = a.codes[slots[g]++];
        mc.B = B->dev;
        mc.kind = small ? kKindSmall : kKindGeneric;
        mc.chunk = P->chunk[c];
        mc.io.synd = x.syndromes;
        mc.io.llr = x.llr;
        mc.io.llr_stride = x.llr_stride;
        mc.io.batch = x.batch;
        mc.io.iters = iters;
        mc.io.alpha = alpha;
        mc.io.cand = cand[c];
        mc.io.conv = x.conv;
        mc.io.iters_run = x.iters_run;
        mc.io.post = nullptr;
        mc.first = first;
        first += (unsigned long long)((x.batch + mc.chunk - 1) / mc.chunk) * B->R;
        wbytes[g] = std::max(wbytes[g], mixed_warp_bytes(B->dev, mc.kind));
    }
    for (int g = 0; g < kMixedGroups; ++g) {
        args[g].n_codes = slots[g];
        args[g].total = firsts[g];
        args[g].warp_bytes = (uint32_t)((wbytes[g] + 15) & ~(size_t)15);
        args[g].counter = counters + g;
        const int warps = g == 0 ? P->warps : 1;
        if ((size_t)warps * args[g].warp_bytes > 200 * 1024)
            return fail(MBBP_E_TOO_LARGE, "shared memory per block");
    }
    cudaError_t e = cudaMemsetAsync(counters, 0, kMixedGroups * sizeof(unsigned long long), s);
    for (size_t i = 0; i < launch_order.size() && e == cudaSuccess; ++i) {
        const int g = launch_order[i];
        if (args[g].total > 0) e = launch_mixed(args[g], g, P->warps, rule, s, P->sm_count);
    }
    if (e != cudaSuccess) return cuda_fail(e, "mbbp_decode_mixed (BP)");
    for (int c = 0; c < nc; ++c) {
        const mbbp_code_io& x = io[c];
        if (x.batch == 0) continue;
        FwsArgs f{};
        f.cand = cand[c];
        f.conv = x.conv;
        f.batch = x.batch;
        f.R = P->codes[c]->R;
        f.n = P->codes[c]->n;
        f.W = P->codes[c]->W;
        f.e_hat = x.e_hat;
        f.success = x.success;
        f.selected = x.selected;
        e = launch_fws(f, s);
        if (e != cudaSuccess) return cuda_fail(e, "mbbp_decode_mixed (FWS)");
    }
    return MBBP_OK;
}

}  // namespace

mbbp_status mbbp_decode_mixed(const mbbp_plan* P, const mbbp_code_io* io, int iters, float alpha,
                              int rule, void* workspace, size_t workspace_bytes, void* stream) {
    if (!P) return fail(MBBP_E_INVALID, "mbbp_decode_mixed: NULL plan");
    return mixed_impl(P, io, iters, alpha, rule, workspace, workspace_bytes, (cudaStream_t)stream);
}

mbbp_status mbbp_plan_autotune(mbbp_plan* P, const mbbp_code_io* io, int iters, float alpha, int rule,
                               void* workspace, size_t workspace_bytes, void* stream, float* best_ms) {
    if (!P) return fail(MBBP_E_INVALID, "mbbp_plan_autotune: NULL plan");
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    if (err != cudaSuccess) return cuda_fail(err, "mbbp_plan_autotune");
    // time one configuration: one untimed run, then the best of two
    auto measure = [&](float* ms) -> mbbp_status {
        if (mbbp_status st = mixed_impl(P, io, iters, alpha, rule, workspace, workspace_bytes, s)) return st;
        float best = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
            cudaEventRecord(e0, s);
            if (mbbp_status st = mixed_impl(P, io, iters, alpha, rule, workspace, workspace_bytes, s)) return st;
            cudaEventRecord(e1, s);
            cudaError_t e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) return cuda_fail(e, "mbbp_plan_autotune");
            float t = 0;
            cudaEventElapsedTime(&t, e0, e1);
            best = std::min(best, t);
        }
        *ms = best;
        return MBBP_OK;
    };
    float best = 0;
    mbbp_status st = measure(&best);
    const int nc = (int)P->codes.size();
    // coordinate descent over: block size, per-code chunk, per-code path, order
    auto try_value = [&](int* knob, int value) -> mbbp_status {
        const int old = *knob;
        if (old == value) return MBBP_OK;
        *knob = value;
        float t = 0;
        mbbp_status r = measure(&t);
        if (r != MBBP_OK) { *knob = old; return r; }
        if (t < best) best = t;
        else *knob = old;
        return MBBP_OK;
    };
    for (int w : {4, 6, 7, 8}) if (st == MBBP_OK) st = try_value(&P->warps, w);
    for (int c = 0; c < nc && st == MBBP_OK; ++c) {
        for (int ch : {1, 2, 4, 8, 16}) if (st == MBBP_OK) st = try_value(&P->chunk[c], ch);
        if (st == MBBP_OK && P->codes[c]->dev.shape != 0 && P->codes[c]->regular)
            st = try_value(&P->kind[c], P->kind[c] == kKindSmall ? kKindGeneric : kKindSmall);
    }
    if (st == MBBP_OK && nc > 1) {
        std::vector<int> old = P->order;
        std::reverse(P->order.begin(), P->order.end());
        float t = 0;
        st = measure(&t);
        if (st == MBBP_OK && t < best) best = t;
        else P->order = old;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != MBBP_OK) return st;
    if (best_ms) *best_ms = best;
    return MBBP_OK;
}

// -------------------------------------------------- weighted min-sum (WMS)

namespace {

int max_edges(const mbbp_bases* B) {
    return *std::max_element(B->edges.begin(), B->edges.end());
}

mbbp_status wms_check(const mbbp_bases* B, int batch, int T, int ckpt) {
    if (!B) return fail(MBBP_E_INVALID, "NULL handle");
    if (batch < 0) return fail(MBBP_E_INVALID, "batch must be >= 0");
    if (T < 1 || T > MBBP_MAX_ITERS) return fail(MBBP_E_INVALID, "T out of range");
    if (ckpt < 1) return fail(MBBP_E_INVALID, "ckpt must be >= 1");
    return check_device(B->device);
}

}  // namespace

size_t mbbp_wms_decode_workspace_size(const mbbp_bases* B, int batch, int T) {
    if (!B || batch < 0 || T < 1) return 0;
    // mbbp_decode's workspace, then (w, g) of every representation and
    // iteration in the message layout
    return mbbp_decode_workspace_size(B, batch) + align256((size_t)B->R * T * B->dev.DC * B->MP * 8);
}

size_t mbbp_wms_workspace_size(const mbbp_bases* B, int batch, int T, int ckpt) {
    if (!B || batch < 0 || T < 1 || ckpt < 1) return 0;
    const size_t nckpt = (size_t)((T - 1) / ckpt);
    const size_t S = (size_t)B->dev.DC * B->MP;
    // per-warp segment buffers only when the backward pass cannot keep the
    // segment states in shared memory
    const size_t seg = wms_states_in_smem(B->dev, ckpt) ? 0 : align256((size_t)kWmsMaxWarps * ckpt * S * 4);
    return 256 + align256((size_t)batch * B->R * nckpt * S * 4) + seg;
}

namespace {
// The per-warp segment buffers (null when the backward pass keeps the
// segment states in shared memory and the workspace has no such region).
float* wms_seg_buf(const mbbp_bases* B, int batch, int T, int ckpt, void* workspace) {
    if (wms_states_in_smem(B->dev, ckpt)) return nullptr;
    const size_t nckpt = (size_t)((T - 1) / ckpt);
    const size_t S = (size_t)B->dev.DC * B->MP;
    return reinterpret_cast<float*>(static_cast<char*>(workspace) + 256 +
                                    align256((size_t)batch * B->R * nckpt * S * 4));
}
}  // namespace

mbbp_status mbbp_wms_forward(const mbbp_bases* B, int batch, const uint8_t* syndromes, const float* llr,
                             int llr_stride, int T, const float* w, const float* g, int ckpt,
                             const uint32_t* etrue, float scale, int all_iters, float* posterior,
                             float* loss,
                             void* workspace, size_t workspace_bytes, void* stream) {
    if (mbbp_status st = wms_check(B, batch, T, ckpt)) return st;
    if (batch == 0) return MBBP_OK;
    if (!syndromes || !llr || !w || !g || !posterior || !workspace)
        return fail(MBBP_E_INVALID, "mbbp_wms_forward: NULL buffer");
    if (loss && !etrue) return fail(MBBP_E_INVALID, "loss needs etrue");
    if (llr_stride != 0 && llr_stride < B->n) return fail(MBBP_E_INVALID, "llr_stride must be 0 or >= n");
    if (workspace_bytes < mbbp_wms_workspace_size(B, batch, T, ckpt)) return fail(MBBP_E_INVALID, "workspace too small");
    WmsArgs a{};
    a.B = B->dev;
    a.synd = syndromes;
    a.llr = llr;
    a.llr_stride = llr_stride;
    a.T = T;
    a.ckpt = ckpt;
    a.nckpt = (T - 1) / ckpt;
    a.E = max_edges(B);
    a.w = w;
    a.g = g;
    a.etrue = etrue;
    a.scale = scale;
    a.all_iters = all_iters ? 1 : 0;
    a.post = posterior;
    a.loss = loss;
    a.counter = static_cast<unsigned long long*>(workspace);
    a.ckpt_buf = a.nckpt ? reinterpret_cast<float*>(static_cast<char*>(workspace) + 256) : nullptr;
    a.total_items = (unsigned long long)batch * B->R;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(a.counter, 0, 8, s);
    if (e == cudaSuccess) e = launch_wms(a, false, s, B->sm_count);
    return e == cudaSuccess ? MBBP_OK : cuda_fail(e, "mbbp_wms_forward");
}

mbbp_status mbbp_wms_backward(const mbbp_bases* B, int batch, const uint8_t* syndromes, const float* llr,
                              int llr_stride, int T, const float* w, const float* g, int ckpt,
                              const uint32_t* etrue, float scale, int all_iters, const float* posterior,
                              float* gw,
                              float* gg, void* workspace, size_t workspace_bytes, void* stream) {
    if (mbbp_status st = wms_check(B, batch, T, ckpt)) return st;
    if (batch == 0) return MBBP_OK;
    if (!syndromes || !llr || !w || !g || !etrue || !posterior || !gw || !gg || !workspace)
        return fail(MBBP_E_INVALID, "mbbp_wms_backward: NULL buffer");
    if (llr_stride != 0 && llr_stride < B->n) return fail(MBBP_E_INVALID, "llr_stride must be 0 or >= n");
    if (workspace_bytes < mbbp_wms_workspace_size(B, batch, T, ckpt)) return fail(MBBP_E_INVALID, "workspace too small");
    WmsArgs a{};
    a.B = B->dev;
    a.synd = syndromes;
    a.llr = llr;
    a.llr_stride = llr_stride;
    a.T = T;
    a.ckpt = ckpt;
    a.nckpt = (T - 1) / ckpt;
    a.E = max_edges(B);
    a.w = w;
    a.g = g;
    a.etrue = etrue;
    a.scale = scale;
    a.all_iters = all_iters ? 1 : 0;
    a.post = const_cast<float*>(posterior);
    a.gw = gw;
    a.gg = gg;
    a.seg_buf = wms_seg_buf(B, batch, T, ckpt, workspace);
    a.counter = static_cast<unsigned long long*>(workspace);
    a.ckpt_buf = a.nckpt ? reinterpret_cast<float*>(static_cast<char*>(workspace) + 256) : nullptr;
    a.total_items = (unsigned long long)batch * B->R;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(a.counter, 0, 8, s);
    if (e == cudaSuccess) e = launch_wms(a, true, s, B->sm_count);
    return e == cudaSuccess ? MBBP_OK : cuda_fail(e, "mbbp_wms_backward");
}

mbbp_status mbbp_wms_decode(const mbbp_bases* B, int batch, const uint8_t* syndromes, const float* llr,
                            int llr_stride, int iters, int T, const float* w, const float* g,
                            uint8_t* e_hat, uint8_t* conv, uint16_t* iters_run, uint8_t* success,
                            int16_t* selected, void* workspace, size_t workspace_bytes, void* stream) {
    if (mbbp_status st = wms_check(B, batch, T, 1)) return st;
    if (iters < 0 || iters > MBBP_MAX_ITERS) return fail(MBBP_E_INVALID, "iters out of range");
    if (batch == 0) return MBBP_OK;
    if (!syndromes || !llr || !w || !g || !e_hat || !conv || !success || !workspace)
        return fail(MBBP_E_INVALID, "mbbp_wms_decode: NULL buffer");
    if (llr_stride != 0 && llr_stride < B->n) return fail(MBBP_E_INVALID, "llr_stride must be 0 or >= n");
    if (workspace_bytes < mbbp_wms_decode_workspace_size(B, batch, T))
        return fail(MBBP_E_INVALID, "workspace too small");
    WmsArgs a{};
    a.B = B->dev;
    a.synd = syndromes;
    a.llr = llr;
    a.llr_stride = llr_stride;
    a.T = T;
    a.ckpt = 1;
    a.E = max_edges(B);
    a.w = w;
    a.g = g;
    a.decode = 1;
    a.iters = iters;
    const size_t cand_bytes = align256((size_t)batch * B->R * B->W * 4);
    a.cand = static_cast<uint32_t*>(workspace);
    a.counter = reinterpret_cast<unsigned long long*>(static_cast<char*>(workspace) + cand_bytes);
    a.conv = conv;
    a.iters_run = iters_run;
    a.total_items = (unsigned long long)batch * B->R;
    // the parameters in the message layout follow the decode workspace
    float2* wg = reinterpret_cast<float2*>(static_cast<char*>(workspace) + mbbp_decode_workspace_size(B, batch));
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(a.counter, 0, 8, s);
    if (e == cudaSuccess) e = launch_wms_pack(a, wg, s, B->sm_count);
    a.wg = wg;
    if (e == cudaSuccess) e = launch_wms(a, false, s, B->sm_count);
    if (e != cudaSuccess) return cuda_fail(e, "mbbp_wms_decode");
    FwsArgs f{};
    f.cand = a.cand;
    f.conv = conv;
    f.batch = batch;
    f.R = B->R;
    f.n = B->n;
    f.W = B->W;
    f.e_hat = e_hat;
    f.success = success;
    f.selected = selected;
    e = launch_fws(f, s);
    return e == cudaSuccess ? MBBP_OK : cuda_fail(e, "mbbp_wms_decode (FWS)");
}

mbbp_status mbbp_adam_step(float* params, const float* grad, float* m, float* v, size_t count, float lr,
                           float beta1, float beta2, float eps, int step, float lo, float hi, void* stream) {
    if (count == 0) return MBBP_OK;
    if (!params || !grad || !m || !v) return fail(MBBP_E_INVALID, "mbbp_adam_step: NULL buffer");
    if (step < 1 || !(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f))
        return fail(MBBP_E_INVALID, "mbbp_adam_step: bad hyper-parameters");
    cudaError_t e = launch_adam(params, grad, m, v, count, lr, beta1, beta2, eps, step, lo, hi,
                                (cudaStream_t)stream);
    return e == cudaSuccess ? MBBP_OK : cuda_fail(e, "mbbp_adam_step");
}

mbbp_status mbbp_logicals_build(const uint8_t* H, int m, const uint8_t* H_other, int m_other,
                                int n, mbbp_logicals** out) {
    if (!out) return fail(MBBP_E_INVALID, "out is NULL");
    *out = nullptr;
    if (!H_other || m_other < 1) return fail(MBBP_E_INVALID, "H_other is empty");
    Tanner g, go;
    if (mbbp_status st = make_tanner(H, m, n, g)) return st;
    if (mbbp_status st = make_tanner(H_other, m_other, n, go)) return st;
    int dc = 0;
    for (int r = 0; r < m; ++r) dc = std::max(dc, (int)g.rcols[r].size());
    if (dc > MBBP_MAX_ROW_WEIGHT) return fail(MBBP_E_TOO_LARGE, "row weight above 12");
    // ker(H_other): reduced row echelon form of H_other, one vector per free column.
    Gf2Rows ech(n);
    for (int r = 0; r < m_other; ++r) ech.insert(pack_row(H_other + (size_t)r * n, n));
    std::vector<int> is_pivot(n, -1);
    for (size_t i = 0; i < ech.rows.size(); ++i) is_pivot[ech.pivots[i]] = (int)i;
    // rowspace(H), then add kernel vectors that are independent of it.
    Gf2Rows span(n);
    for (int r = 0; r < m; ++r) span.insert(pack_row(H + (size_t)r * n, n));
    const int rank_h = (int)span.rows.size();
    std::vector<std::vector<uint64_t>> logicals;
    for (int f = 0; f < n; ++f) {
        if (is_pivot[f] >= 0) continue;
        std::vector<uint64_t> x((n + 63) / 64, 0);
        x[f >> 6] |= 1ull << (f & 63);
        for (size_t i = 0; i < ech.rows.size(); ++i)
            if (Gf2Rows::get(ech.rows[i], f)) {
                const int c = ech.pivots[i];
                x[c >> 6] |= 1ull << (c & 63);
            }
        if (span.insert(x)) logicals.push_back(x);
    }
    const int k = (int)logicals.size();
    if (k != n - rank_h - (int)ech.rows.size())
        return fail(MBBP_E_INVALID, "H H_other^T != 0: not a CSS pair");
    mbbp_logicals* L = new (std::nothrow) mbbp_logicals();
    if (!L) return fail(MBBP_E_NOMEM, "host allocation failed");
    const int K = dc <= 6 ? 6 : (dc <= 8 ? 8 : 12);
    L->m = m; L->n = n; L->k = k; L->K = K; L->mpad = round_up(m, 32); L->W = words_for(n);
    L->ops.assign((size_t)k * n, 0);
    std::vector<uint32_t> lmask((size_t)std::max(k, 1) * L->W, 0);
    for (int i = 0; i < k; ++i)
        for (int c = 0; c < n; ++c)
            if (Gf2Rows::get(logicals[i], c)) {
                L->ops[(size_t)i * n + c] = 1;
                lmask[(size_t)i * L->W + (c >> 5)] |= 1u << (c & 31);
            }
    std::vector<uint16_t> hcol((size_t)K * L->mpad, (uint16_t)n);
    for (int r = 0; r < m; ++r)
        for (int j = 0; j < (int)g.rcols[r].size(); ++j) hcol[(size_t)j * L->mpad + r] = (uint16_t)g.rcols[r][j];
    const size_t o_l = align256(hcol.size() * 2);
    const size_t total = o_l + align256(lmask.size() * 4);
    cudaError_t e = cudaGetDevice(&L->device);
    if (e == cudaSuccess) e = cudaMalloc(&L->dmem, total);
    if (e == cudaSuccess) e = cudaMemcpy(L->dmem, hcol.data(), hcol.size() * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(static_cast<char*>(L->dmem) + o_l, lmask.data(), lmask.size() * 4,
                       cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        if (L->dmem) cudaFree(L->dmem);
        delete L;
        return cuda_fail(e, "mbbp_logicals_build");
    }
    L->dev.hcol = static_cast<const uint16_t*>(L->dmem);
    L->dev.lmask = reinterpret_cast<const uint32_t*>(static_cast<char*>(L->dmem) + o_l);
    L->dev.m = m; L->dev.n = n; L->dev.k = k; L->dev.DC = K; L->dev.mpad = L->mpad; L->dev.W = L->W;
    *out = L;
    return MBBP_OK;
}

mbbp_status mbbp_logicals_info(const mbbp_logicals* L, int32_t* k, uint8_t* ops) {
    if (!L) return fail(MBBP_E_INVALID, "mbbp_logicals_info: NULL handle");
    if (k) *k = L->k;
    if (ops) std::copy(L->ops.begin(), L->ops.end(), ops);
    return MBBP_OK;
}

mbbp_status mbbp_probe(int kind, int rounds, float* sink, double* work, void* stream) {
    if (kind < MBBP_PROBE_FADD || kind > MBBP_PROBE_SMEM) return fail(MBBP_E_INVALID, "mbbp_probe: unknown kind");
    if (rounds < 1 || !sink || !work) return fail(MBBP_E_INVALID, "mbbp_probe: bad arguments");
    const cudaError_t e = launch_probe(kind, rounds, sink, (cudaStream_t)stream, work);
    return e == cudaSuccess ? MBBP_OK : cuda_fail(e, "mbbp_probe");
}

mbbp_status mbbp_judge(const mbbp_logicals* L, int batch, const uint32_t* e, const uint8_t* e_hat,
                       uint8_t* fail_out, unsigned long long* counts, void* stream) {
    if (!L || batch < 0) return fail(MBBP_E_INVALID, "mbbp_judge: bad arguments");
    if (batch == 0) return MBBP_OK;
    if (!e || !e_hat) return fail(MBBP_E_INVALID, "mbbp_judge: NULL buffer");
    if (mbbp_status st = check_device(L->device)) return st;
    cudaError_t err = launch_judge(L->dev, batch, e, e_hat, fail_out, counts, (cudaStream_t)stream);
    return err == cudaSuccess ? MBBP_OK : cuda_fail(err, "mbbp_judge");
}

void mbbp_logicals_free(mbbp_logicals* L) {
    if (!L) return;
    if (L->dmem) cudaFree(L->dmem);
    delete L;
}

}  // extern "C"
