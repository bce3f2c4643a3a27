/* CPU oracle for Multiple-Bases BP List Decoding (MBBP-LD).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, step-by-step CPU
 * restatement of the paper's method, written to check the CUDA path.  Only
 * tests/, the package's smoke() check and bench.py's CPU-baseline leg may
 * load it.  It shares no code with the CUDA library and includes none of its
 * headers.  Build: gcc -O2 -ffp-contract=off -fPIC -shared (no FMA
 * contraction, so FP32 results are the IEEE results of the written
 * operations in the written order).
 *
 * Contents, each with the passage it follows:
 *   or_splitmix64_at, or_sample   counter-based error sampler (splitmix64 of
 *                                 Steele, Lea & Flood, 2014) for the BSC and
 *                                 depolarizing channels of Section IV
 *   or_gf2_rank, or_syndrome      GF(2) rank and s = H e (Section II-A)
 *   or_subtrees                   Algorithm 2 (maximal subtrees)
 *   or_permutation,
 *   or_collect_subtrees           root orders pi and the collection T of
 *                                 subtrees over several orders (Section III-A)
 *   or_bp_f64 / or_bp_f32         syndrome BP on one representation
 *                                 (Section II-B, Eqs. (2)-(3)), see bp_body.inc
 *   or_bp_serial_f64 / _f32       the serial schedule of Section II-B
 *   or_fws                        Frequency-Weighted Scoring (Section III-B)
 *   or_lms                        least-metric selector (Section III-A)
 *   or_random_sets                random augmentation of Table II
 *   or_mbbp_decode_f64 / _f32     Algorithm 1 over a batch of syndromes
 *   or_judge                      logical-error test by GF(2) rank (Section IV)
 *   or_wms_forward / _backward    weighted min-sum and its adjoint (FP64;
 *                                 not in the paper, reduces to Eq. (2)-(3))
 *   or_clamp_reset, or_clamp_stats  how often BP's message clamp acts (a
 *                                 diagnostic of the clamp reading)
 *
 * Parity of normalized min-sum with alpha < 1 on loopy graphs is unpinned by
 * the paper (no printed values); the tests pin BP through trees, where it is
 * exact, and through closed forms.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_RULE_NMS 0
#define OR_RULE_SP 1
/* Message clamp (not stated in the paper; see bp_body.inc). */
#define OR_LMAX 1.0e4

/* How often the clamp acts: v->c messages computed and messages clamped, by
 * the BP calls of the calling thread since its last or_clamp_reset (a
 * diagnostic; the counts do not enter any result). */
static _Thread_local long long or_q_total, or_q_clamped;
void or_clamp_reset(void) { or_q_total = 0; or_q_clamped = 0; }
void or_clamp_stats(long long* total, long long* clamped) {
    *total = or_q_total;
    *clamped = or_q_clamped;
}
/* Sum-product magnitude clamp: 2 atanh(1 - 2^-23) = ln(2^24 - 1). */
#define OR_SPMAX 16.635532333438686

/* Gallager's phi(x) = log((e^x + 1) / (e^x - 1)) = log1p(2 / expm1(x)). */
static double or_phi64(double x) { return log1p(2.0 / expm1(x)); }
static float or_phi32(float x) { return log1pf(2.0f / expm1f(x)); }

/* ------------------------------------------------------------------ RNG -- */

static uint64_t or_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* i-th output (i >= 1) of the splitmix64 generator started at `state`:
 * the state advances by the golden-ratio increment before each output. */
uint64_t or_splitmix64_at(uint64_t state, uint64_t i)
{
    return or_mix64(state + i * 0x9E3779B97F4A7C15ULL);
}

/* Error sampler.  Qubit q of shot `shot` draws u = output number
 * (shot * n + q + 1) of the stream seeded with `seed`; T = floor(p * 2^64).
 * noise 0 (BSC, X errors only, Section IV): X iff u < T.
 * noise 1 (depolarizing): with t1 = floor(T / 3): X iff u < t1,
 *   Y iff t1 <= u < 2 t1, Z iff 2 t1 <= u < T.
 * ex = X part (X or Y), decoded with H_Z; ez = Z part (Z or Y), decoded with
 * H_X (Section II-A).  Outputs are (batch, n) bytes. */
void or_sample(uint64_t seed, uint64_t first_shot, int batch, int n, double p,
               int noise, uint8_t* ex, uint8_t* ez)
{
    uint64_t T = (uint64_t)ldexp(p, 64);
    uint64_t t1 = T / 3;
    for (int b = 0; b < batch; b++) {
        uint64_t shot = first_shot + (uint64_t)b;
        for (int q = 0; q < n; q++) {
            uint64_t u = or_splitmix64_at(seed, shot * (uint64_t)n + (uint64_t)q + 1);
            uint8_t x = 0, z = 0;
            if (noise == 0) {
                x = (uint8_t)(u < T);
            } else if (u < T) {
                if (u < t1) x = 1;
                else if (u < 2 * t1) { x = 1; z = 1; }
                else z = 1;
            }
            ex[(size_t)b * n + q] = x;
            if (ez) ez[(size_t)b * n + q] = z;
        }
    }
}

/* ---------------------------------------------------------------- GF(2) -- */

int or_gf2_rank(const uint8_t* A, int rows, int cols)
{
    uint8_t* W = (uint8_t*)malloc((size_t)rows * cols + 1);
    for (size_t z = 0; z < (size_t)rows * cols; z++) W[z] = A[z] & 1;
    int rank = 0;
    for (int c = 0; c < cols && rank < rows; c++) {
        int piv = -1;
        for (int r = rank; r < rows; r++)
            if (W[(size_t)r * cols + c]) { piv = r; break; }
        if (piv < 0) continue;
        if (piv != rank)
            for (int k = 0; k < cols; k++) {
                uint8_t tmp = W[(size_t)piv * cols + k];
                W[(size_t)piv * cols + k] = W[(size_t)rank * cols + k];
                W[(size_t)rank * cols + k] = tmp;
            }
        for (int r = 0; r < rows; r++)
            if (r != rank && W[(size_t)r * cols + c])
                for (int k = 0; k < cols; k++)
                    W[(size_t)r * cols + k] ^= W[(size_t)rank * cols + k];
        rank++;
    }
    free(W);
    return rank;
}

/* s = H e over GF(2) for a batch of error vectors (Section II-A). */
void or_syndrome(const uint8_t* H, int m, int n, int batch, const uint8_t* e,
                 uint8_t* s)
{
    for (int b = 0; b < batch; b++)
        for (int r = 0; r < m; r++) {
            int par = 0;
            for (int v = 0; v < n; v++)
                if (H[(size_t)r * n + v] && e[(size_t)b * n + v]) par ^= 1;
            s[(size_t)b * m + r] = (uint8_t)par;
        }
}

/* 1 iff every row of H satisfies its syndrome bit (halting rule, II-B). */
static int or_syndrome_ok(const uint8_t* H, int M, int n, const uint8_t* s,
                          const uint8_t* e)
{
    for (int r = 0; r < M; r++) {
        int par = 0;
        for (int v = 0; v < n; v++)
            if (H[(size_t)r * n + v] && e[v]) par ^= 1;
        if (par != (s[r] & 1)) return 0;
    }
    return 1;
}

/* ---------------------------------------------------------- Algorithm 2 -- */

/* Maximal subtrees (Algorithm 2).  Roots are taken in the order perm[0..m-1];
 * check_sets[c] receives the 1-based index of the subtree holding check c;
 * order[] receives the checks in the order they were accepted (subtree by
 * subtree, BFS order inside a subtree), which is the row order of H_t
 * (Fig. 2).  N(u) is taken in ascending column order and N(v) in ascending
 * row order; a check already tested is not tested again when it is
 * dequeued a second time (eta can only have grown since).  Returns the
 * number of subtrees. */
int or_subtrees(const uint8_t* H, int m, int n, const int32_t* perm,
                int32_t* check_sets, int32_t* order)
{
    int E = 0, maxcol = 0;
    for (int v = 0; v < n; v++) {
        int d = 0;
        for (int r = 0; r < m; r++) d += H[(size_t)r * n + v] ? 1 : 0;
        E += d;
        if (d > maxcol) maxcol = d;
    }
    size_t qcap = (size_t)E * (size_t)(maxcol > 0 ? maxcol : 1) + (size_t)m + 1;
    int* Q = (int*)malloc(sizeof(int) * qcap);
    uint8_t* visited = (uint8_t*)malloc((size_t)n + 1);
    uint8_t* tested = (uint8_t*)malloc((size_t)m + 1);
    for (int c = 0; c < m; c++) check_sets[c] = 0;
    int s = 0, nord = 0;
    for (int idx = 0; idx < m; idx++) {
        int c = perm[idx];
        if (check_sets[c] != 0) continue;
        s++;
        size_t head = 0, tail = 0;
        Q[tail++] = c;
        memset(visited, 0, (size_t)n);
        memset(tested, 0, (size_t)m);
        while (head < tail) {
            int u = Q[head++];
            if (tested[u]) continue;
            tested[u] = 1;
            int eta = 0;
            for (int v = 0; v < n; v++)
                if (H[(size_t)u * n + v] && visited[v]) eta++;
            if (eta <= 1) {
                check_sets[u] = s;
                order[nord++] = u;
                for (int v = 0; v < n; v++) {
                    if (!H[(size_t)u * n + v]) continue;
                    visited[v] = 1;
                    for (int c2 = 0; c2 < m; c2++)
                        if (H[(size_t)c2 * n + v] && !tested[c2] && check_sets[c2] == 0)
                            Q[tail++] = c2;
                }
            }
        }
    }
    free(Q); free(visited); free(tested);
    return s;
}

/* Root order pi_j.  pi_0 is the identity.  For j >= 1: Fisher-Yates
 * (Durstenfeld) shuffle of the identity, i = m-1 down to 1, swapping entry i
 * with entry x mod (i+1), x the successive outputs of splitmix64 seeded with
 * seed XOR j. */
void or_permutation(uint64_t seed, int j, int m, int32_t* perm)
{
    for (int i = 0; i < m; i++) perm[i] = i;
    if (j == 0) return;
    uint64_t state = seed ^ (uint64_t)j;
    uint64_t draw = 1;
    for (int i = m - 1; i >= 1; i--) {
        uint64_t x = or_splitmix64_at(state, draw++);
        int k = (int)(x % (uint64_t)(i + 1));
        int32_t tmp = perm[i];
        perm[i] = perm[k];
        perm[k] = tmp;
    }
}

/* The collection of R subtrees: the subtrees of pi_0, pi_1, ... in creation
 * order, skipping any whose set of checks equals an earlier one, until R are
 * found or max_perms orders have been tried.  set_ptr[R+1] / set_rows hold
 * the rows of each H_t in acceptance order.  Returns the number found. */
int or_collect_subtrees(const uint8_t* H, int m, int n, int R, uint64_t seed,
                        int max_perms, int32_t* set_ptr, int32_t* set_rows)
{
    int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m + 1));
    int32_t* cs = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m + 1));
    int32_t* ord = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m + 1));
    uint8_t* mine = (uint8_t*)malloc((size_t)m + 1);
    uint8_t* other = (uint8_t*)malloc((size_t)m + 1);
    int found = 0, used = 0;
    set_ptr[0] = 0;
    for (int j = 0; j < max_perms && found < R; j++) {
        or_permutation(seed, j, m, perm);
        int ns = or_subtrees(H, m, n, perm, cs, ord);
        int pos = 0;
        for (int t = 1; t <= ns && found < R; t++) {
            int start = pos;
            while (pos < m && cs[ord[pos]] == t) pos++;
            int len = pos - start;
            memset(mine, 0, (size_t)m);
            for (int i = start; i < pos; i++) mine[ord[i]] = 1;
            int dup = 0;
            for (int f = 0; f < found && !dup; f++) {
                int flen = set_ptr[f + 1] - set_ptr[f];
                if (flen != len) continue;
                memset(other, 0, (size_t)m);
                for (int i = set_ptr[f]; i < set_ptr[f + 1]; i++) other[set_rows[i]] = 1;
                if (memcmp(mine, other, (size_t)m) == 0) dup = 1;
            }
            if (dup) continue;
            for (int i = start; i < pos; i++) set_rows[used++] = ord[i];
            found++;
            set_ptr[found] = used;
        }
    }
    free(perm); free(cs); free(ord); free(mine); free(other);
    return found;
}

/* ------------------------------------------------------------------ FWS -- */

/* Frequency-Weighted Scoring (Section III-B): among the converged candidates
 * pick argmax count(e) / (w_H(e) + 1); ratios are compared exactly as
 * count_a (w_b + 1) vs count_b (w_a + 1).  Ties go to the candidate seen
 * first (lowest representation index).  An empty list is a decoding failure
 * and gives the all-zero vector.  Returns 1 on success, 0 on failure. */
int or_fws(const uint8_t* cand, const uint8_t* conv, int R, int n,
           uint8_t* ehat, int* selected)
{
    int best = -1;
    long long best_cnt = 0, best_w = 0;
    for (int a = 0; a < R; a++) {
        if (!conv[a]) continue;
        long long cnt = 0, w = 0;
        for (int b = 0; b < R; b++) {
            if (!conv[b]) continue;
            if (memcmp(cand + (size_t)a * n, cand + (size_t)b * n, (size_t)n) == 0) cnt++;
        }
        for (int v = 0; v < n; v++) w += cand[(size_t)a * n + v] ? 1 : 0;
        if (best < 0 || cnt * (best_w + 1) > best_cnt * (w + 1)) {
            best = a;
            best_cnt = cnt;
            best_w = w;
        }
    }
    if (selected) *selected = best;
    if (best < 0) {
        memset(ehat, 0, (size_t)n);
        return 0;
    }
    memcpy(ehat, cand + (size_t)best * n, (size_t)n);
    return 1;
}

/* ---------------------------------------------------- LMS, random sets -- */

/* Least-metric selector of classical MBBP (Section III-A): among the
 * converged candidates the most likely one under the channel, i.e. the
 * smallest sum_i mu_i e_i (for an i.i.d. channel the smallest weight).  The
 * metric is a float sum in ascending i (the precision of the GPU path, which
 * takes the same decision); ties go to the first candidate.  Returns 1 on
 * success, 0 (and e = 0) when no candidate converged. */
int or_lms(const uint8_t* cand, const uint8_t* conv, int R, int n, const float* mu,
           uint8_t* ehat, int* selected)
{
    int best = -1;
    float best_m = 0.0f;
    for (int a = 0; a < R; a++) {
        if (!conv[a]) continue;
        float mt = 0.0f;
        for (int v = 0; v < n; v++)
            if (cand[(size_t)a * n + v]) mt = mt + mu[v];
        if (best < 0 || mt < best_m) { best = a; best_m = mt; }
    }
    if (selected) *selected = best;
    if (best < 0) { memset(ehat, 0, (size_t)n); return 0; }
    memcpy(ehat, cand + (size_t)best * n, (size_t)n);
    return 1;
}

/* ------------------------------------------------------------------- BP -- */

#define REAL double
#define BP_FN or_bp_f64
#define BPS_FN or_bp_serial_f64
#define DECODE_FN or_mbbp_decode_f64
#define FABS fabs
#define PHI or_phi64
#include "bp_body.inc"
#undef REAL
#undef BP_FN
#undef BPS_FN
#undef DECODE_FN
#undef FABS
#undef PHI

#define REAL float
#define BP_FN or_bp_f32
#define BPS_FN or_bp_serial_f32
#define DECODE_FN or_mbbp_decode_f32
#define FABS fabsf
#define PHI or_phi32
#include "bp_body.inc"
#undef REAL
#undef BP_FN
#undef BPS_FN
#undef DECODE_FN
#undef FABS
#undef PHI

/* Exported single-instance entry points (BP on one representation). */
void or_bp_one_f64(const uint8_t* Ht, int M, int n, const uint8_t* st,
                   const double* mu, int iters, double alpha, int rule,
                   int early_stop, uint8_t* ehat, int* conv, int* K,
                   double* post, double* c2v)
{
    or_bp_f64(Ht, M, n, st, mu, iters, alpha, rule, early_stop, ehat, conv, K, post, c2v);
}

void or_bp_one_f32(const uint8_t* Ht, int M, int n, const uint8_t* st,
                   const float* mu, int iters, float alpha, int rule,
                   int early_stop, uint8_t* ehat, int* conv, int* K,
                   float* post, float* c2v)
{
    or_bp_f32(Ht, M, n, st, mu, iters, alpha, rule, early_stop, ehat, conv, K, post, c2v);
}

void or_bp_serial_one_f64(const uint8_t* Ht, int M, int n, const uint8_t* st,
                          const double* mu, int iters, double alpha, int rule, int early_stop,
                          uint8_t* ehat, int* conv, int* K, double* post)
{
    or_bp_serial_f64(Ht, M, n, st, mu, iters, alpha, rule, early_stop, ehat, conv, K, post);
}

void or_bp_serial_one_f32(const uint8_t* Ht, int M, int n, const uint8_t* st,
                          const float* mu, int iters, float alpha, int rule, int early_stop,
                          uint8_t* ehat, int* conv, int* K, float* post)
{
    or_bp_serial_f32(Ht, M, n, st, mu, iters, alpha, rule, early_stop, ehat, conv, K, post);
}

/* ---------------------------------------------------------------- judge -- */

/* Logical-error test (Section IV reports logical error rates).  For a batch
 * of (error e, estimate ehat) pairs, r = e XOR ehat:
 *   fail = 1  if Hc r != 0 (the estimate does not reproduce the syndrome),
 *   fail = 2  if Hc r == 0 but r is not in the row space of Ho (the
 *             stabilizers of the other type), i.e. rank([Ho; r]) > rank(Ho),
 *   fail = 0  otherwise. */
void or_judge(const uint8_t* Hc, int mc, const uint8_t* Ho, int mo, int n,
              int batch, const uint8_t* e, const uint8_t* ehat, uint8_t* fail)
{
    uint8_t* A = (uint8_t*)malloc((size_t)(mo + 1) * n + 1);
    memcpy(A, Ho, (size_t)mo * n);
    int base = or_gf2_rank(Ho, mo, n);
    uint8_t* r = A + (size_t)mo * n;
    for (int b = 0; b < batch; b++) {
        for (int v = 0; v < n; v++)
            r[v] = (uint8_t)((e[(size_t)b * n + v] ^ ehat[(size_t)b * n + v]) & 1);
        int synd = 0;
        for (int i = 0; i < mc && !synd; i++) {
            int par = 0;
            for (int v = 0; v < n; v++)
                if (Hc[(size_t)i * n + v] && r[v]) par ^= 1;
            if (par) synd = 1;
        }
        if (synd) { fail[b] = 1; continue; }
        fail[b] = (uint8_t)(or_gf2_rank(A, mo + 1, n) > base ? 2 : 0);
    }
    free(A);
}

/* ------------------------------------------------- weighted min-sum (WMS) -- */

/* Differentiable weighted min-sum on one representation (FP64), a reading of
 * the paper's normalized min-sum (Section II-B, Eq. (2)-(3)) with a weight
 * and a damping factor per edge and per iteration; w == alpha and g == 0
 * gives normalized min-sum (flooding, no early stop):
 *   m^(t)_e = g^(t)_e m^(t-1)_e + (1 - g^(t)_e) w^(t)_e S_e mn_e,
 *   S_e = (-1)^{s_c} prod_{other e' of c} sign(q^(t-1)_e'),
 *   mn_e = min(LMAX, min_{other e' of c} |q^(t-1)_e'|),
 *   q^(t)_e = mu_v + sum_{other e' of v} m^(t)_e' (ascending row order),
 * with m^(0) = 0, q^(0) = mu, for t = 1..T.  Edges are numbered row by row,
 * columns ascending; w and g are [T][E].  Loss of the item:
 *   L = scale * sum_v BCE(sigmoid(-post_v), e_v),  post = mu + sum_c m^(T),
 * or, with all_iters, the mean of that over the posteriors of t = 1..T.
 * Outputs post[n] (of iteration T) and returns L. */
static int or_wms_graph(const uint8_t* Ht, int M, int n, int** row_start, int** edge_col,
                        int** col_start, int** col_edges)
{
    int E = 0;
    for (int r = 0; r < M; r++)
        for (int v = 0; v < n; v++) E += Ht[(size_t)r * n + v] ? 1 : 0;
    *row_start = (int*)calloc((size_t)M + 1, sizeof(int));
    *edge_col = (int*)malloc(sizeof(int) * (size_t)(E + 1));
    *col_start = (int*)calloc((size_t)n + 1, sizeof(int));
    *col_edges = (int*)malloc(sizeof(int) * (size_t)(E + 1));
    int* fill = (int*)calloc((size_t)n + 1, sizeof(int));
    int e = 0;
    for (int r = 0; r < M; r++) {
        (*row_start)[r] = e;
        for (int v = 0; v < n; v++)
            if (Ht[(size_t)r * n + v]) { (*edge_col)[e++] = v; (*col_start)[v + 1]++; }
    }
    (*row_start)[M] = e;
    for (int v = 0; v < n; v++) (*col_start)[v + 1] += (*col_start)[v];
    for (int k = 0; k < E; k++) {
        int v = (*edge_col)[k];
        (*col_edges)[(*col_start)[v] + fill[v]++] = k;
    }
    free(fill);
    return E;
}

/* one WMS iteration: m_new from (m_prev, q_prev); then q_new and post */
static void or_wms_step(int M, int n, const int* row_start, const int* col_start,
                        const int* col_edges, const int* edge_col, const uint8_t* st,
                        const double* mu, const double* w, const double* g,
                        const double* m_prev, const double* q_prev, double* m_new,
                        double* q_new, double* post)
{
    for (int r = 0; r < M; r++) {
        int a = row_start[r], b = row_start[r + 1];
        for (int j = a; j < b; j++) {
            double mn = OR_LMAX;
            int neg = st[r] & 1;
            for (int k = a; k < b; k++) {
                if (k == j) continue;
                double x = fabs(q_prev[k]);
                if (x < mn) mn = x;
                if (q_prev[k] < 0) neg ^= 1;
            }
            double sgn = neg ? -1.0 : 1.0;
            m_new[j] = g[j] * m_prev[j] + (1.0 - g[j]) * w[j] * sgn * mn;
        }
    }
    for (int v = 0; v < n; v++) {
        int a = col_start[v], b = col_start[v + 1];
        double acc = mu[v];
        for (int i = a; i < b; i++) acc = acc + m_new[col_edges[i]];
        if (post) post[v] = acc;
        for (int i = a; i < b; i++) {
            double q = mu[v];
            for (int k = a; k < b; k++) {
                if (k == i) continue;
                q = q + m_new[col_edges[k]];
            }
            q_new[col_edges[i]] = q;
        }
    }
    (void)edge_col;
}

static double or_bce_sigmoid_neg(double post, int e)
{
    /* BCE(p, e) with p = sigmoid(-post) = P(e = 1), written stably:
     * -log p = log(1 + exp(post)), -log(1 - p) = log(1 + exp(-post)) */
    double x = e ? post : -post;
    return x > 0 ? x + log1p(exp(-x)) : log1p(exp(x));
}

double or_wms_forward(const uint8_t* Ht, int M, int n, const uint8_t* st, const double* mu,
                      int T, const double* w, const double* g, const uint8_t* etrue,
                      double scale, int all_iters, double* post_out)
{
    int *row_start, *edge_col, *col_start, *col_edges;
    int E = or_wms_graph(Ht, M, n, &row_start, &edge_col, &col_start, &col_edges);
    double* m_prev = (double*)calloc((size_t)E + 1, sizeof(double));
    double* m_new = (double*)calloc((size_t)E + 1, sizeof(double));
    double* q = (double*)calloc((size_t)E + 1, sizeof(double));
    double* q_new = (double*)calloc((size_t)E + 1, sizeof(double));
    double* post = (double*)calloc((size_t)n + 1, sizeof(double));
    for (int k = 0; k < E; k++) q[k] = mu[edge_col[k]];
    for (int v = 0; v < n; v++) post[v] = mu[v];
    double L = 0;
    for (int t = 0; t < T; t++) {
        or_wms_step(M, n, row_start, col_start, col_edges, edge_col, st, mu,
                    w + (size_t)t * E, g + (size_t)t * E, m_prev, q, m_new, q_new, post);
        double* tmp = m_prev; m_prev = m_new; m_new = tmp;
        tmp = q; q = q_new; q_new = tmp;
        /* all_iters: the loss is the mean over t = 1..T of the BCE of post^(t) */
        if (etrue && all_iters && t < T - 1)
            for (int v = 0; v < n; v++) L += or_bce_sigmoid_neg(post[v], etrue[v] & 1) / T;
    }
    for (int v = 0; v < n; v++) {
        if (post_out) post_out[v] = post[v];
        if (etrue) L += or_bce_sigmoid_neg(post[v], etrue[v] & 1) / (all_iters ? T : 1);
    }
    free(row_start); free(edge_col); free(col_start); free(col_edges);
    free(m_prev); free(m_new); free(q); free(q_new); free(post);
    return scale * L;
}

/* Adjoint of or_wms_forward: adds dL/dw and dL/dg ([T][E]) to gw, gg.  The
 * derivative of the min goes to the other edge of the row with the smallest
 * |q| (the lowest-numbered one on ties), times sign(q) (+1 at 0), when that
 * |q| is below LMAX; the derivative of the sign is 0.  Returns L. */
double or_wms_backward(const uint8_t* Ht, int M, int n, const uint8_t* st, const double* mu,
                       int T, const double* w, const double* g, const uint8_t* etrue,
                       double scale, int all_iters, double* gw, double* gg)
{
    int *row_start, *edge_col, *col_start, *col_edges;
    int E = or_wms_graph(Ht, M, n, &row_start, &edge_col, &col_start, &col_edges);
    /* forward, keeping every m^(t) and q^(t) */
    double* ms = (double*)calloc((size_t)(T + 1) * E + 1, sizeof(double));
    double* qs = (double*)calloc((size_t)(T + 1) * E + 1, sizeof(double));
    double* post = (double*)calloc((size_t)n + 1, sizeof(double));
    for (int k = 0; k < E; k++) qs[k] = mu[edge_col[k]];
    for (int v = 0; v < n; v++) post[v] = mu[v];
    for (int t = 0; t < T; t++)
        or_wms_step(M, n, row_start, col_start, col_edges, edge_col, st, mu,
                    w + (size_t)t * E, g + (size_t)t * E, ms + (size_t)t * E,
                    qs + (size_t)t * E, ms + (size_t)(t + 1) * E, qs + (size_t)(t + 1) * E, post);
    double L = 0;
    const double wt_loss = all_iters ? 1.0 / T : 1.0;  /* weight of one iteration's BCE */
    double* gm = (double*)calloc((size_t)E + 1, sizeof(double));   /* dL/dm^(t) */
    double* gm_prev = (double*)calloc((size_t)E + 1, sizeof(double));
    double* gq = (double*)calloc((size_t)E + 1, sizeof(double));   /* dL/dq^(t-1) */
    double* pst = (double*)calloc((size_t)n + 1, sizeof(double));
    for (int v = 0; v < n; v++) {
        int e = etrue[v] & 1;
        L += or_bce_sigmoid_neg(post[v], e) * wt_loss;
        /* dBCE/dpost = e - sigmoid(-post) */
        double p = 1.0 / (1.0 + exp(post[v]));
        double gp = scale * wt_loss * ((double)e - p);
        for (int i = col_start[v]; i < col_start[v + 1]; i++) gm[col_edges[i]] = gp;
    }
    for (int t = T; t >= 1; t--) {
        const double* m_prev = ms + (size_t)(t - 1) * E;
        const double* q_prev = qs + (size_t)(t - 1) * E;
        const double* wt = w + (size_t)(t - 1) * E;
        const double* gt = g + (size_t)(t - 1) * E;
        for (int k = 0; k < E; k++) gq[k] = 0;
        for (int r = 0; r < M; r++) {
            int a = row_start[r], b = row_start[r + 1];
            for (int j = a; j < b; j++) {
                double mn = OR_LMAX;
                int neg = st[r] & 1, arg = -1;
                for (int k = a; k < b; k++) {
                    if (k == j) continue;
                    double x = fabs(q_prev[k]);
                    if (x < mn) { mn = x; arg = k; }
                    if (q_prev[k] < 0) neg ^= 1;
                }
                double sgn = neg ? -1.0 : 1.0;
                double c = wt[j] * sgn * mn;
                gg[(size_t)(t - 1) * E + j] += gm[j] * (m_prev[j] - c);
                gw[(size_t)(t - 1) * E + j] += gm[j] * (1.0 - gt[j]) * sgn * mn;
                gm_prev[j] = gm[j] * gt[j];
                if (arg >= 0) {
                    double gmn = gm[j] * (1.0 - gt[j]) * wt[j] * sgn;
                    gq[arg] += gmn * (q_prev[arg] < 0 ? -1.0 : 1.0);
                }
            }
        }
        /* q^(t-1)_e = mu + sum_{other e'} m^(t-1)_e'  (q^(0) = mu has no m) */
        if (t >= 2) {
            for (int v = 0; v < n; v++) {
                double G = 0;
                for (int i = col_start[v]; i < col_start[v + 1]; i++) G += gq[col_edges[i]];
                for (int i = col_start[v]; i < col_start[v + 1]; i++) {
                    int e = col_edges[i];
                    gm_prev[e] += G - gq[e];
                }
            }
        }
        /* all_iters: the BCE of post^(t-1) (t - 1 >= 1) joins dL/dm^(t-1) */
        if (all_iters && t >= 2) {
            for (int v = 0; v < n; v++) {
                double acc = mu[v];
                for (int i = col_start[v]; i < col_start[v + 1]; i++) acc = acc + m_prev[col_edges[i]];
                pst[v] = acc;
                int e = etrue[v] & 1;
                L += or_bce_sigmoid_neg(acc, e) * wt_loss;
                double p = 1.0 / (1.0 + exp(acc));
                double gp = scale * wt_loss * ((double)e - p);
                for (int i = col_start[v]; i < col_start[v + 1]; i++) gm_prev[col_edges[i]] += gp;
            }
        }
        double* tmp = gm; gm = gm_prev; gm_prev = tmp;
    }
    free(row_start); free(edge_col); free(col_start); free(col_edges);
    free(ms); free(qs); free(post); free(gm); free(gm_prev); free(gq); free(pst);
    return scale * L;
}

/* Random augmentation, the comparison of Table II: representation t keeps
 * the number of extra rows of subtree t, sizes[t], but draws them as
 * distinct uniformly random rows of H.  Draw for representation t: a
 * Fisher-Yates shuffle (i = m-1 down to 1, swap with x mod (i+1), x the
 * outputs of splitmix64 seeded with seed XOR (t + 1)) of 0..m-1, first
 * sizes[t] entries.  set_ptr[R+1] / set_rows as or_collect_subtrees. */
void or_random_sets(int m, int R, const int32_t* sizes, uint64_t seed, int32_t* set_ptr,
                    int32_t* set_rows)
{
    int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m + 1));
    set_ptr[0] = 0;
    for (int t = 0; t < R; t++) {
        for (int i = 0; i < m; i++) perm[i] = i;
        uint64_t state = seed ^ (uint64_t)(t + 1);
        uint64_t draw = 1;
        for (int i = m - 1; i >= 1; i--) {
            uint64_t x = or_splitmix64_at(state, draw++);
            int k = (int)(x % (uint64_t)(i + 1));
            int32_t tmp = perm[i]; perm[i] = perm[k]; perm[k] = tmp;
        }
        int len = sizes[t] < m ? sizes[t] : m;
        for (int i = 0; i < len; i++) set_rows[set_ptr[t] + i] = perm[i];
        set_ptr[t + 1] = set_ptr[t] + len;
    }
    free(perm);
}
