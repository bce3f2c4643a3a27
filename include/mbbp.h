/* mbbp.h — C ABI of the GB300 (sm_103a) Multiple-Bases BP List Decoder.
 *
 * The decoder of "Multiple-Bases Belief Propagation List Decoding for
 * Quantum LDPC Codes" (Rabeti & Mahdavifar): syndrome-based belief
 * propagation run in parallel over R redundant parity-check representations
 * H^(t) = [H; H_t] (Section III-A, Eq. (4)) built from the maximal subtrees of
 * Algorithm 2, followed by Frequency-Weighted Scoring of the converged
 * candidates (Section III-B).  Algorithm 1 states the whole decoder.
 *
 * Conventions for every entry point:
 *  - Matrices are row-major.  A "host" pointer is ordinary CPU memory, a
 *    "device" pointer is CUDA global memory of the current device.
 *  - Bit vectors are packed little-endian into uint32_t words: bit i of word
 *    w is entry 32*w + i; W(n) = ceil(n / 32) words per vector; bits past n
 *    are zero on output and ignored on input.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Entry points that take a stream only enqueue work on it and
 *    return before it runs; they allocate no memory.
 *  - Errors are status codes; nothing throws across the ABI and no kernel
 *    traps.  mbbp_last_error() gives a message for the last non-OK status of
 *    the calling thread.
 *  - Handles (mbbp_bases, mbbp_logicals) are owned by the library and freed
 *    with their *_free function; they hold host and device copies of their
 *    tables and belong to the device that was current when they were built.
 */
#ifndef MBBP_H
#define MBBP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MBBP_OK = 0,
    MBBP_E_INVALID = 1,   /* an argument is out of range or inconsistent      */
    MBBP_E_TOO_LARGE = 2, /* sizes beyond the limits below                    */
    MBBP_E_CUDA = 3,      /* a CUDA runtime call failed                       */
    MBBP_E_TIMEOUT = 4,   /* reserved for a bounded device-side wait; no entry
                             point of this build waits on the device (work is
                             pulled with atomic counters), so none returns it */
    MBBP_E_NOMEM = 5,     /* host or device allocation failed                 */
    MBBP_E_NOT_FOUND = 6  /* fewer distinct subtrees than requested exist     */
} mbbp_status;

/* Check-node rules (Section II-B). */
enum { MBBP_RULE_NMS = 0, /* normalized min-sum, Eq. (2)                       */
       MBBP_RULE_SP = 1   /* sum-product: 2 atanh(prod tanh(q/2)), used by the
                             BPGD baselines of Section IV                      */ };

/* Noise models of the error sampler. */
enum { MBBP_NOISE_BSC = 0,          /* independent X errors (Section IV)     */
       MBBP_NOISE_DEPOLARIZING = 1  /* X, Y, Z each with probability p/3     */ };

/* Limits. */
#define MBBP_MAX_R 64          /* representations per handle                   */
#define MBBP_MAX_N 16384       /* variables (qubits)                           */
#define MBBP_MAX_ROW_WEIGHT 12 /* check degree d_c of H                        */
#define MBBP_MAX_COL_WEIGHT 12 /* variable degree in any H^(t)                 */
#define MBBP_MAX_ROWS 1024     /* rows of any H^(t) = m + |t|                   */
#define MBBP_MAX_SLOTS 65536   /* d_c * (rows of the largest H^(t), padded to 32) */
#define MBBP_MAX_ITERS 65535

/* Readings of the paper that the kernels fix (the paper states none):
 * v->c messages are clamped to [-MBBP_LMAX, MBBP_LMAX]; the min of Eq. (2)
 * also runs over MBBP_LMAX (a degree-1 row sends alpha*LMAX); sum-product
 * check messages are evaluated as phi(sum phi(|q|)) with Gallager's
 * phi(x) = log((e^x+1)/(e^x-1)) and clamped to MBBP_SP_MAX = 2 atanh(1 - 2^-23)
 * in magnitude. */
#define MBBP_LMAX 1.0e4f
#define MBBP_SP_MAX 16.635532f

typedef struct mbbp_bases mbbp_bases;
typedef struct mbbp_logicals mbbp_logicals;

/* Message for the last non-OK status returned on this thread ("" if none). */
const char* mbbp_last_error(void);
/* Library version string. */
const char* mbbp_version(void);

/* ------------------------------------------------------------------------
 * Representation construction (host only, Section III-A).
 * ---------------------------------------------------------------------- */

/* Root order pi_j for Algorithm 2 (Section III-A: "different permutations
 * lead to different collections").  pi_0 is the identity; for j >= 1 the
 * identity is shuffled by Fisher-Yates (i = m-1 down to 1, swap i with
 * x mod (i+1)) with x the successive outputs of splitmix64 seeded with
 * seed XOR j.  perm: host int32[m], written. */
mbbp_status mbbp_permutation(uint64_t seed, int j, int m, int32_t* perm);

/* Algorithm 2: partition the checks of H into maximal subtrees.
 * H: host uint8[m*n] 0/1; perm: host int32[m], a permutation of 0..m-1 (root
 * order).  check_sets: host int32[m], receives the 1-based subtree index of
 * each check.  order: host int32[m] or NULL, receives the checks in the order
 * they were accepted (subtree by subtree; BFS order inside each), which is
 * the row order of H_t (Fig. 2).  n_subtrees: host int32, or NULL.
 * Neighbours are visited in ascending index order; a check is tested at most
 * once per subtree. */
mbbp_status mbbp_subtrees(const uint8_t* H, int m, int n, const int32_t* perm,
                          int32_t* check_sets, int32_t* order, int32_t* n_subtrees);

/* The R subtrees used as representations: the subtrees of pi_0, pi_1, ... in
 * creation order, skipping any whose check set equals an earlier one, until R
 * are found (at most 1024 orders are tried; fewer found -> MBBP_E_NOT_FOUND).
 * set_ptr: host int32[R+1]; set_rows: host int32[R*m]; subtree t has rows
 * set_rows[set_ptr[t] .. set_ptr[t+1]) in acceptance order. */
mbbp_status mbbp_collect_subtrees(const uint8_t* H, int m, int n, int R, uint64_t seed,
                                  int32_t* set_ptr, int32_t* set_rows);

/* Build the R representations H^(t) = [H; H_t] (Eq. (4)) from the subtrees
 * that mbbp_collect_subtrees(H, m, n, R, seed) returns, pack their Tanner
 * graphs into the kernels' layout and copy them to the current device (a
 * synchronous copy; call once per code).  H: host uint8[m*n] 0/1.  *out
 * receives a handle owned by the library. */
mbbp_status mbbp_build_bases(const uint8_t* H, int m, int n, int R, uint64_t seed,
                             mbbp_bases** out);

/* Same, with the extra rows of every representation given explicitly:
 * representation t appends rows set_rows[set_ptr[t] .. set_ptr[t+1]) of H, in
 * that order (an empty set gives plain BP on H; any rows of H are allowed,
 * e.g. the random augmentations the paper compares against in Table II). */
mbbp_status mbbp_build_bases_from_sets(const uint8_t* H, int m, int n, int R,
                                       const int32_t* set_ptr, const int32_t* set_rows,
                                       mbbp_bases** out);

/* Random augmentation, the comparison of Table II: representation t gets
 * sizes[t] distinct rows of H (at most m), the first entries of the
 * Fisher-Yates shuffle of 0..m-1 that mbbp_permutation(seed, t + 1, m)
 * defines.  sizes: host int32[R]; set_ptr: host int32[R+1]; set_rows: host
 * int32[sum of min(sizes[t], m)].  Pass the result to
 * mbbp_build_bases_from_sets (e.g. with the sizes of the subtrees it
 * replaces, which keeps the number of duplicated rows). */
mbbp_status mbbp_random_sets(int m, int R, const int32_t* sizes, uint64_t seed,
                             int32_t* set_ptr, int32_t* set_rows);

/* Shape of a handle.  Each output is host memory or NULL: m, n, R (int32);
 * rows, edges (int32[R]: rows and edges of each H^(t)); set_ptr (int32[R+1])
 * and set_rows (int32[set_ptr[R]]): the extra rows. */
mbbp_status mbbp_bases_info(const mbbp_bases* B, int32_t* m, int32_t* n, int32_t* R,
                            int32_t* rows, int32_t* edges, int32_t* set_ptr,
                            int32_t* set_rows);

/* Check order of the serial schedule of representation t (see
 * mbbp_decode_ex): the rows of H^(t) split greedily, in row order, into
 * layers of rows that share no variable (each row joins the first layer it
 * does not clash with).  order: host int32[rows of H^(t)] or NULL, the rows
 * layer by layer (ascending inside a layer); layer_ptr: host
 * int32[rows + 1] or NULL, layer L holds order[layer_ptr[L] ..
 * layer_ptr[L+1]); n_layers: host int32 or NULL. */
mbbp_status mbbp_bases_layers(const mbbp_bases* B, int t, int32_t* order, int32_t* layer_ptr,
                              int32_t* n_layers);

/* Free a handle and its device tables (NULL is a no-op).  Not stream-ordered:
 * no work that uses B may still be pending. */
void mbbp_bases_free(mbbp_bases* B);

/* ------------------------------------------------------------------------
 * Monte-Carlo producer (Section IV: independent X errors; code-capacity
 * depolarizing noise for the other workloads).
 * ---------------------------------------------------------------------- */

/* Sample errors for shots first_shot .. first_shot+batch-1 on n qubits.
 * Qubit q of shot k draws u = output number k*n + q + 1 of splitmix64 seeded
 * with `seed` (so any split of the shots gives the same errors);
 * T = floor(p * 2^64), 0 <= p < 1.  BSC: X iff u < T.  Depolarizing, with
 * t1 = floor(T/3): X iff u < t1, Y iff t1 <= u < 2 t1, Z iff 2 t1 <= u < T.
 * ex: device uint32[batch*W(n)], X part (X or Y; decoded with H_Z).
 * ez: device uint32[batch*W(n)] or NULL, Z part (Z or Y; decoded with H_X). */
mbbp_status mbbp_sample_errors(int n, int batch, uint64_t first_shot, uint64_t seed,
                               double p, int noise, uint32_t* ex, uint32_t* ez,
                               void* stream);

/* Syndromes s = H e over GF(2) for the H of a handle.  e: device
 * uint32[batch*W(n)]; s: device uint8[batch*m], 0/1. */
mbbp_status mbbp_syndrome(const mbbp_bases* B, int batch, const uint32_t* e, uint8_t* s,
                          void* stream);

/* ------------------------------------------------------------------------
 * Decoder (Algorithm 1 with BP of Section II-B and FWS of Section III-B).
 * ---------------------------------------------------------------------- */

/* Bytes of device workspace mbbp_decode needs for `batch` shots. */
size_t mbbp_decode_workspace_size(const mbbp_bases* B, int batch);

/* Decode `batch` syndromes on all R representations of B, then select.
 *
 * syndromes: device uint8[batch*m], 0/1 (bit r = check r of H).
 * llr: device float[n] when llr_stride == 0 (one channel for every shot), or
 *      float[batch*llr_stride] with llr_stride >= n (per-shot LLRs; the LLR
 *      mu_i = log((1-p)/p) of Section II-B for an i.i.d. channel).
 * iters: maximum BP iterations (0..MBBP_MAX_ITERS); alpha: normalization of
 *      Eq. (2), 0 < alpha <= 1 (ignored by MBBP_RULE_SP); rule: MBBP_RULE_*.
 * Every representation runs flooding BP: each iteration computes all check
 * messages from the previous variable messages, then all variable messages,
 * posteriors and hard decisions e_i = [m_i < 0].  It stops at the first
 * iteration K (K = 0 is the hard decision of the LLRs themselves) whose hard
 * decision satisfies H e = s, else after `iters`.  FWS picks, among the
 * converged representations, the estimate maximising count / (weight + 1)
 * (ties: lowest representation index); none converged -> e_hat = 0.
 *
 * Outputs (device): e_hat uint8[batch*n] 0/1; conv uint8[batch*R] (1 iff
 * representation t converged); success uint8[batch] (1 iff any converged).
 * Optional (device, or NULL): iters_run uint16[batch*R] (K of each
 * representation); selected int16[batch] (chosen representation or -1);
 * posterior float[batch*R*n] (last posterior LLRs of each representation).
 * workspace: device memory of workspace_bytes >= mbbp_decode_workspace_size;
 * on return (once the stream has run) its first batch*R*W(n) uint32 words
 * hold the final hard decision of every (shot, representation), bit-packed,
 * shot-major.  The call allocates nothing; concurrent calls need distinct
 * workspaces. */
mbbp_status mbbp_decode(const mbbp_bases* B, int batch, const uint8_t* syndromes,
                        const float* llr, int llr_stride, int iters, float alpha, int rule,
                        uint8_t* e_hat, uint8_t* conv, uint16_t* iters_run,
                        uint8_t* success, int16_t* selected, float* posterior,
                        void* workspace, size_t workspace_bytes, void* stream);

/* Decoder options: the BP schedule and the decision rule. */
#define MBBP_SCHEDULE_FLOODING 0
#define MBBP_SCHEDULE_SERIAL 1
#define MBBP_DECISION_FWS 0
#define MBBP_DECISION_LMS 1

typedef struct {
    int rule;      /* MBBP_RULE_NMS or MBBP_RULE_SP                        */
    float alpha;   /* normalization of Eq. (2), 0 < alpha <= 1 (NMS only)   */
    int schedule;  /* MBBP_SCHEDULE_*                                      */
    int decision;  /* MBBP_DECISION_*                                      */
} mbbp_options;

/* mbbp_decode with a choice of schedule and decision rule; every argument
 * other than opt (host pointer, not kept) is that of mbbp_decode, and
 * {rule, alpha, FLOODING, FWS} gives mbbp_decode's result.
 *
 * MBBP_SCHEDULE_SERIAL (Section II-B: checks are updated one after the other
 * and the newest messages are used within the iteration; the numerical
 * results run MBBP-LD this way): check messages start at 0; an iteration
 * visits the checks of H^(t) in the layer order of mbbp_bases_layers, and a
 * visited check first forms q_{v->c} = mu_v + the current messages of v's
 * other checks (ascending row order, clamped to +-MBBP_LMAX), then replaces
 * its messages by the check rule.  After the last layer come the
 * posteriors, hard decisions and the halting test of mbbp_decode.  Rows of a
 * layer share no variable, so the kernel updates a layer's rows at once and
 * the result equals the one-check-at-a-time order.
 *
 * MBBP_DECISION_LMS (the least-metric selector of classical MBBP, Section
 * III-A): among the converged candidates, the one with the smallest
 * sum_i mu_i e_i, with mu the shot's LLRs and the sum a float sum in
 * ascending i; ties go to the lowest representation index; none converged
 * -> e_hat = 0, selected = -1. */
mbbp_status mbbp_decode_ex(const mbbp_bases* B, int batch, const uint8_t* syndromes,
                           const float* llr, int llr_stride, int iters, const mbbp_options* opt,
                           uint8_t* e_hat, uint8_t* conv, uint16_t* iters_run,
                           uint8_t* success, int16_t* selected, float* posterior,
                           void* workspace, size_t workspace_bytes, void* stream);

/* mbbp_decode_ex (flooding schedule only) that also records the messages
 * behind the posteriors: for every (shot, representation), the check-to-
 * variable messages m_{c->v} of Eq. (2) of the last iteration it ran.
 * c2v: device float[batch*R*E], E = the largest edge count of the
 * representations (mbbp_bases_info); entry e of (shot, t) is edge e of H^(t)
 * with edges numbered row by row, columns ascending (the numbering of the
 * WMS weights).  Entries past the representation's own edge count, and all
 * entries of an item that stopped at K = 0, are left as they were.  For
 * tests and debugging (comparison with a reference decoder); the trace
 * costs one extra global store per message and iteration.  MBBP_E_INVALID
 * for the serial schedule or a NULL c2v. */
mbbp_status mbbp_decode_trace(const mbbp_bases* B, int batch, const uint8_t* syndromes,
                              const float* llr, int llr_stride, int iters, const mbbp_options* opt,
                              uint8_t* e_hat, uint8_t* conv, uint16_t* iters_run,
                              uint8_t* success, int16_t* selected, float* posterior, float* c2v,
                              void* workspace, size_t workspace_bytes, void* stream);

/* ------------------------------------------------------------------------
 * Mixed batches: several codes decoded by persistent launches.
 * ---------------------------------------------------------------------- */

/* A plan for decoding the shots of up to 8 codes together (Algorithm 1 for
 * each code's shots, as mbbp_decode).  The plan keeps the code handles
 * (which must outlive it) and its launch configuration: warps per block of
 * the generic-path launch, shots per work item and kernel path per code, and
 * the order of the codes in the work list (heaviest first by default). */
typedef struct mbbp_plan mbbp_plan;

/* Inputs and outputs of one code in a mixed batch; the meaning, layout and
 * optionality of every field are those of the mbbp_decode argument of the
 * same name (device pointers; llr_stride 0 = one LLR vector for all shots). */
typedef struct {
    int batch;
    const uint8_t* syndromes;
    const float* llr;
    int llr_stride;
    uint8_t* e_hat;
    uint8_t* conv;
    uint16_t* iters_run;
    uint8_t* success;
    int16_t* selected;
} mbbp_code_io;

mbbp_status mbbp_plan_create(const mbbp_bases* const* codes, int n_codes, mbbp_plan** out);
void mbbp_plan_free(mbbp_plan* P);

/* Workspace bytes for the given per-code batches (host int32[n_codes]). */
size_t mbbp_plan_workspace_size(const mbbp_plan* P, const int32_t* batches);

/* Decode io[c] (host array of n_codes entries) with code c of the plan: one
 * persistent BP launch per kernel body the plan uses (the generic path in
 * blocks of the plan's warps, the small-code path once per shape in use, in
 * one-warp blocks; each with its own register budget) over every (code, shot
 * chunk, representation) work item of that launch, then FWS per code.
 * Outputs are identical to one mbbp_decode per
 * code.  Only kernel launches and a memset are enqueued, so the call can be
 * captured into a CUDA graph (after the first call with the same plan, shapes
 * and block size, which sets kernel attributes).  Workspace: as mbbp_decode,
 * its first region holds each code's candidates in code order. */
mbbp_status mbbp_decode_mixed(const mbbp_plan* P, const mbbp_code_io* io, int iters, float alpha,
                              int rule, void* workspace, size_t workspace_bytes, void* stream);

/* Choose the plan's launch configuration by timing mbbp_decode_mixed on the
 * given inputs (coordinate descent over the generic launch's warps per block
 * in {4, 6, 7, 8}, shots per work item in {1, 2, 4, 8, 16} and the kernel
 * path per code, then the code order).  Synchronises the stream, overwrites the outputs; not capturable.
 * best_ms: host float or NULL, the time of the chosen configuration. */
mbbp_status mbbp_plan_autotune(mbbp_plan* P, const mbbp_code_io* io, int iters, float alpha,
                               int rule, void* workspace, size_t workspace_bytes, void* stream,
                               float* best_ms);

/* The plan's configuration: warps per block (generic path); per code (host int32[n_codes]
 * each, or NULL) shots per work item, path (0 small-code, 1 generic) and the
 * work-list order. */
mbbp_status mbbp_plan_info(const mbbp_plan* P, int32_t* warps, int32_t* chunk, int32_t* kind,
                           int32_t* order);

/* ------------------------------------------------------------------------
 * Differentiable weighted min-sum (WMS) and learned weights.
 * ---------------------------------------------------------------------- */

/* WMS is normalized min-sum (Section II-B, Eq. (2)-(3)) with a weight w and a
 * damping factor g per edge and per iteration of every representation; the
 * paper defines no such variant, w == alpha and g == 0 reproduces Eq. (2):
 *   m^(t)_e = g^(t)_e m^(t-1)_e + (1 - g^(t)_e) w^(t)_e S_e mn_e,
 *   S_e = (-1)^{s_c} prod_{other e' of c} sign(q^(t-1)_e'),
 *   mn_e = min(LMAX, min_{other e' of c} |q^(t-1)_e'|),
 *   q^(t)_e = mu_v + sum_{other e' of v} m^(t)_e', m^(0) = 0, q^(0) = mu,
 * for t = 1..T (flooding, no early stop); loss of a (shot, representation):
 *   scale * sum_v BCE(sigmoid(-post_v), e_v), post = mu + sum_c m^(T),
 * or, with all_iters != 0, the mean of that over the posteriors of t = 1..T.
 * w and g are device float[R][T][E], E = the largest edge count of the
 * representations (mbbp_bases_info), edges numbered row by row of H^(t),
 * columns ascending. */

/* Workspace of mbbp_wms_forward / mbbp_wms_backward: the checkpoints of m,
 * one every `ckpt` iterations ((T-1)/ckpt of them per (shot, representation)),
 * and, for codes whose segment states do not fit in shared memory, the
 * recomputed states of one segment per warp of the backward grid. */
size_t mbbp_wms_workspace_size(const mbbp_bases* B, int batch, int T, int ckpt);

/* Forward pass.  syndromes, llr, llr_stride: as mbbp_decode.  etrue: device
 * uint32[batch*W(n)] bit-packed true errors (as mbbp_sample_errors writes
 * them) or NULL; posterior: device float[batch*R*n]
 * (needed by the backward pass); loss: device float[batch*R] or NULL (needs
 * etrue).  The workspace keeps the checkpoints for mbbp_wms_backward. */
mbbp_status mbbp_wms_forward(const mbbp_bases* B, int batch, const uint8_t* syndromes, const float* llr,
                             int llr_stride, int T, const float* w, const float* g, int ckpt,
                             const uint32_t* etrue, float scale, int all_iters, float* posterior,
                             float* loss,
                             void* workspace, size_t workspace_bytes, void* stream);

/* Backward pass (hand-written adjoint): adds dL/dw and dL/dg (device
 * float[R][T][E]) of the summed loss of every (shot, representation).  The
 * inputs, posterior and workspace must be those of the forward call.  The
 * min's derivative goes to the other edge of the check with the smallest
 * |q| (lowest index on ties) when it is below LMAX, times sign(q) (+1 at 0);
 * the sign's derivative is 0.  Segments of `ckpt` iterations are recomputed
 * from their checkpoint.  Accumulation order varies (atomics). */
mbbp_status mbbp_wms_backward(const mbbp_bases* B, int batch, const uint8_t* syndromes, const float* llr,
                              int llr_stride, int T, const float* w, const float* g, int ckpt,
                              const uint32_t* etrue, float scale, int all_iters, const float* posterior,
                              float* gw,
                              float* gg, void* workspace, size_t workspace_bytes, void* stream);

/* Workspace of mbbp_wms_decode: mbbp_decode's, then a copy of w and g
 * rearranged into the kernel's message layout, 8 bytes per slot and
 * R * T * K * MP slots: K the smallest of 6, 8, 12 not below any row or
 * column weight of the H^(t), MP the rows of the largest H^(t) rounded up to
 * a multiple of 32.  Returns 0 for a NULL handle, batch < 0 or T < 1. */
size_t mbbp_wms_decode_workspace_size(const mbbp_bases* B, int batch, int T);

/* Algorithm 1 with WMS as the BP of every representation: the halting rule
 * after every iteration (up to `iters`; iterations past T use the weights of
 * iteration T), then FWS.  Outputs as mbbp_decode; the workspace holds at
 * least mbbp_wms_decode_workspace_size(B, batch, T) bytes. */
mbbp_status mbbp_wms_decode(const mbbp_bases* B, int batch, const uint8_t* syndromes, const float* llr,
                            int llr_stride, int iters, int T, const float* w, const float* g,
                            uint8_t* e_hat, uint8_t* conv, uint16_t* iters_run, uint8_t* success,
                            int16_t* selected, void* workspace, size_t workspace_bytes, void* stream);

/* One Adam step on `count` device floats (params, grad, first and second
 * moments m and v), bias-corrected with the 1-based step number; the updated
 * parameters are clamped to [lo, hi]. */
mbbp_status mbbp_adam_step(float* params, const float* grad, float* m, float* v, size_t count, float lr,
                           float beta1, float beta2, float eps, int step, float lo, float hi, void* stream);

/* Size of the fixed device scratch behind mbbp_decode_noalloc (8 MiB). */
#define MBBP_NOALLOC_SCRATCH_BYTES ((size_t)8 << 20)

/* mbbp_decode for callers that cannot allocate device memory — for example a
 * decoder embedded in a real-time control loop, where a cudaMalloc could block
 * or fail mid-run, or a host program that links only this library and has no
 * device allocator of its own.  The paper has no counterpart: this is a
 * library convenience.  Arguments and outputs are those of mbbp_decode minus
 * the workspace: the scratch lives in a fixed array of
 * MBBP_NOALLOC_SCRATCH_BYTES inside the library, which every GPU that loads the
 * library holds until the process exits.  A batch whose
 * mbbp_decode_workspace_size exceeds it is rejected with MBBP_E_TOO_LARGE
 * (about 26,000 shots for [[144,12,12]] with R = 16).  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.  The call
 * allocates nothing and clears the part of the scratch that must start at
 * zero.  Every call shares the one array, which keeps the last call's
 * contents: calls whose work overlaps on the GPU (other streams, other host
 * threads) race on it and must be ordered by the caller. */
mbbp_status mbbp_decode_noalloc(const mbbp_bases* B, int batch, const uint8_t* syndromes,
                                const float* llr, int llr_stride, int iters, float alpha,
                                int rule, uint8_t* e_hat, uint8_t* conv, uint16_t* iters_run,
                                uint8_t* success, int16_t* selected, float* posterior,
                                void* stream);

/* ------------------------------------------------------------------------
 * Logical-error judge (the logical error rate of Section IV).
 * ---------------------------------------------------------------------- */

/* Logical operators for judging errors decoded with H (m x n): a basis of
 * ker(H_other) modulo rowspace(H), k = n - rank(H) - rank(H_other) vectors
 * (for X errors: H = H_Z, H_other = H_X).  Host inputs; the handle keeps
 * device copies. */
mbbp_status mbbp_logicals_build(const uint8_t* H, int m, const uint8_t* H_other, int m_other,
                                int n, mbbp_logicals** out);

/* k and, if ops != NULL, the operators as host uint8[k*n]. */
mbbp_status mbbp_logicals_info(const mbbp_logicals* L, int32_t* k, uint8_t* ops);

/* Judge shots: r = e XOR e_hat; fail = 1 if H r != 0, 2 if H r = 0 but some
 * logical operator has odd overlap with r, else 0.  e: device
 * uint32[batch*W(n)]; e_hat: device uint8[batch*n]; fail: device uint8[batch]
 * or NULL; counts: device uint64[3] or NULL, incremented by the number of
 * shots with fail = 0, 1, 2 (zero it first to count one batch). */
mbbp_status mbbp_judge(const mbbp_logicals* L, int batch, const uint32_t* e,
                       const uint8_t* e_hat, uint8_t* fail, unsigned long long* counts,
                       void* stream);

/* Free a logicals handle (NULL is a no-op). */
void mbbp_logicals_free(mbbp_logicals* L);

/* ------------------------------------------------------------------------
 * Throughput probes (measurement; no counterpart in the paper).
 * ---------------------------------------------------------------------- */

/* Probe kinds: FP32 add, FP32 min/max, 3-input logic (the operation classes
 * of the BP update rules, Eq. (2)-(3)), and 16-byte shared-memory loads. */
enum { MBBP_PROBE_FADD = 0, MBBP_PROBE_FMNMX = 1, MBBP_PROBE_LOP3 = 2, MBBP_PROBE_SMEM = 3 };

/* Enqueue one launch of probe `kind` on `stream`: every SM full of
 * 1024-thread blocks, each thread running `rounds` rounds of 64 operations
 * (8 interdependent chains, so none can be merged away) or of eight 16-byte
 * shared-memory loads at conflict-free addresses.  *work (host, written
 * before the launch runs) = the lane operations, or the shared-memory bytes,
 * that the launch performs; the caller times the launch (CUDA events on
 * `stream`) to get the per-SM rate behind the BP kernels' roofline.  sink:
 * device float[1], written only if a chain ends equal to 1e-30, which does
 * not happen (it keeps the work alive).  MBBP_E_INVALID for an unknown kind,
 * rounds < 1 or a NULL pointer. */
mbbp_status mbbp_probe(int kind, int rounds, float* sink, double* work, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MBBP_H */
