/*
 * jabba.h -- C ABI of the GB300 (sm_103a) JABBA symbolization library.
 *
 * JABBA (joint adaptive Brownian-bridge-based aggregation, arXiv 2401.00109)
 * turns many time series into symbols over ONE shared dictionary:
 *   1. domains      series are cut into domains with shared endpoints
 *                   (Alg. 1 Phase I; Sec. 4.1.1)
 *   2. compress     each domain becomes (len, inc) pieces under tol
 *                   (Sec. 3.1 Eq. 1; Alg. 1 Phase II; Sec. 4.1.2)
 *   3. digitize     pieces are normalised by their standard deviations
 *      (local)      (Sec. 3.2 Eq. 4) and greedily aggregated within alpha,
 *                   separately in each domain (Sec. 5 Stage I)
 *   4. merge        the local groups, taken at their centres, are aggregated
 *                   once more into the shared dictionary (Sec. 5 Stage II)
 *   5. symbolize    labels are composed through the local->global map
 *                   (Sec. 5 label propagation; no reassignment pass)
 *   6. reconstruct  symbols -> quantized chain -> series (Sec. 3.3)
 *
 * Conventions for every call below.
 *  - Pointers are DEVICE pointers (caller-owned, e.g. torch tensor storage)
 *    unless the name ends in _host.  The library never frees them.
 *  - Calls are asynchronous and ordered on `stream`.  Argument errors are
 *    returned synchronously.  Errors found on the device (non-finite input,
 *    values out of range, capacity overflow, a bounded wait that timed out)
 *    set the context's device status word; jabba_sync_status() synchronizes
 *    `stream` and returns (and clears) it.
 *  - Counts that depend on the data (pieces, groups, dictionary size) are
 *    written to device scalars so that a whole step can be captured in a
 *    CUDA graph; the context owns only scratch space, allocated by
 *    jabba_reserve() (or grown by a call made outside graph capture).
 *  - Floating point is IEEE binary64.  Every decision the paper's method
 *    takes (breakpoints, orderings, memberships) equals the decision of the
 *    FP64 definition stated at each call.
 *  - Layout: a collection of S series is CSR: x[n_points] (float64) and
 *    series_off[S+1] (int64); series s is x[series_off[s] .. series_off[s+1]).
 *    Contract: every x is finite with |x| < 2^31; a series has < 2^31 points.
 *  - Pieces and per-piece labels are SLOTTED: the pieces of domain d occupy
 *    slots [dom_slot_off[d], dom_slot_off[d] + dom_piece_cnt[d]) of arrays
 *    sized n_slots = total number of intervals (an upper bound on pieces).
 *    dom_piece_off[d] (exclusive scan of dom_piece_cnt) is the compact
 *    concatenation P = P^(1) + ... + P^(M) of Sec. 4.1.3, used by the symbols.
 *  - One context per stream at a time; contexts are not thread-safe.
 */
#ifndef JABBA_H
#define JABBA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* jabba_stream; /* same type as cudaStream_t; NULL = legacy default stream */

typedef enum {
  JABBA_OK = 0,
  JABBA_ERR_INVALID_ARG = 1, /* bad argument (returned synchronously)                          */
  JABBA_ERR_CAPACITY = 2,    /* an output or scratch capacity is too small                      */
  JABBA_ERR_NONFINITE = 3,   /* NaN or infinity in the input series                             */
  JABBA_ERR_CUDA = 4,        /* a CUDA runtime call failed                                      */
  JABBA_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up                              */
  JABBA_ERR_STATE = 6,       /* call out of order (e.g. missing reservation during capture)     */
  JABBA_ERR_RANGE = 7        /* an input value is outside the documented range (|x| >= 2^31)    */
} jabba_status;

typedef struct jabba_ctx jabba_ctx;

typedef struct {
  double tol;           /* compression tolerance, >= 0 (Eq. 1)                                 */
  double alpha;         /* aggregation radius in normalised units, >= 0 (Sec. 3.2)              */
  double scl;           /* length weight, >= 0 (Eq. 4); 0 ignores lengths                      */
  int32_t domain_mode;  /* 0 = EQUAL_COUNT: min(value, n_s-1) domains per series,
                           boundaries floor(k (n_s-1) / M_s);
                           1 = FIXED_LEN: domains of `value` intervals (last one shorter)      */
  int32_t round_mode;   /* quantization rounding (Sec. 3.3): 0 = half away from zero, 1 = half to even */
  int64_t domain_value; /* M (EQUAL_COUNT) or interval count (FIXED_LEN), >= 1                  */
  int32_t key_mode;     /* sort key of the greedy aggregation (Sec. 5 "norm or PCA projection"):
                           0 = X*X + Y*Y (orders as the norm); 1 = vx X + vy Y, the projection on
                           the first principal axis of the normalised pieces (see
                           jabba_digitize_local); the block form accepts 0 only                 */
  int32_t reserved;     /* 0                                                                     */
} jabba_params;

/* Local group record (Sec. 5 Stage I output), 48 bytes.  Exact sums make every
 * centre independent of summation order. */
typedef struct {
  uint64_t inc[3];  /* sum of member increments, signed 192-bit two's complement in units of 2^-64
                       (each increment truncated toward zero at 2^-64)                          */
  int64_t lensum;   /* sum of member lengths                                                     */
  int32_t count;    /* member count                                                              */
  int32_t local_id; /* id within its domain (creation order of the greedy)                       */
  int32_t domain;   /* domain index                                                              */
  int32_t pad;
} jabba_group;

#define JABBA_PIECE_STATS_BYTES 256 /* opaque exact-sum accumulators of jabba_compress */

/* ---------------------------------------------------------------- context */
jabba_status jabba_create(jabba_ctx** ctx, int device);
void jabba_destroy(jabba_ctx* ctx);
const char* jabba_status_string(jabba_status s);
const char* jabba_version(void);

/* Synchronize `stream`, return the device status word (first error wins) and
 * clear it. */
jabba_status jabba_sync_status(jabba_ctx* ctx, jabba_stream stream);

/* Poll limit of the context's bounded device-side waits (no counterpart in
 * the paper): the compression's waits for its staged series chunks, the
 * merge sort's look-back and the merge rounds' grid barrier each give up
 * after `polls` unsuccessful polls, set JABBA_ERR_TIMEOUT and leave their
 * kernel (the compression still lets its copies in flight land first).
 * 0 restores the default (2^26 polls, far beyond any wait that can end).
 * Synchronizes the device; kernels read the limit when they start.  Meant
 * for tests of the timeout path: a small limit makes waits that would have
 * ended give up (below 1024 the compression polls without suspending, so
 * each poll returns at once). */
jabba_status jabba_set_spin_limit(jabba_ctx* ctx, uint32_t polls);

/* Host-side planning (Alg. 1 Phase I): number of domains, of slots (total
 * intervals) and the largest domain (in intervals) for
 * series_off_host[n_series+1].  max_dom_intervals may be NULL. */
jabba_status jabba_plan(const int64_t* series_off_host, int64_t n_series, const jabba_params* p,
                        int64_t* n_domains, int64_t* n_slots, int64_t* max_dom_intervals);

/* Pre-allocate the context's scratch for collections up to these sizes, so
 * that later calls allocate nothing (required before CUDA-graph capture).
 * max_dom_intervals (from jabba_plan) sizes the scratch of domains with more
 * pieces than the on-chip tile (4096); a domain above the reservation makes
 * jabba_digitize_local report JABBA_ERR_CAPACITY. */
jabba_status jabba_reserve(jabba_ctx* ctx, int64_t n_points, int64_t n_series, int64_t n_domains,
                           int64_t n_slots, int64_t group_capacity, int64_t max_dom_intervals);

/* ---------------------------------------------------------------- 1+2. compress
 * Builds the domain table (Alg. 1 Phase I, Sec. 4.1.1: consecutive domains of
 * one series share an endpoint, s_{k+1} = e_k) and compresses every domain
 * independently (Sec. 3.1 Eq. 1, greedy extension): from start s the end e
 * grows while the next end is admissible and stops at the first inadmissible
 * end.  Admissibility is Eq. 1 multiplied through by L^2 (the same criterion
 * in exact arithmetic, with no division):
 *     sum_{k=1}^{L-1} n_k^2 <= ((L - 1) * (tol * tol)) * (L * L),
 *     n_k = ((x_s * L) + (inc * k)) - (x_{s+k} * L),
 * L = e - s, inc = x_e - x_s; every n_k and n_k * n_k is a binary64 operation
 * in that order (no fused multiply-add), the squares are summed EXACTLY
 * (each truncated to a multiple of 2^-96, summed as an integer, the total
 * rounded once to nearest-even), so the sum has no summation order.  Eq. 1
 * read literally (residuals (x_s + (inc * k) / L) - x_{s+k} summed in
 * ascending k, compared with (L - 1) * (tol * tol)) agrees with this except
 * where the error lies within rounding of the bound.  A piece is
 * (len = L, inc).
 * Outputs (device):
 *   dom_begin, dom_end [n_domains]  inclusive global indices into x
 *   dom_series [n_domains]          series of each domain
 *   series_dom_off [n_series+1]     first domain of each series
 *   dom_slot_off [n_domains+1]      first slot of each domain (exclusive scan of intervals)
 *   piece_len, piece_inc [n_slots]  slotted pieces
 *   dom_piece_cnt [n_domains]       pieces per domain
 *   dom_piece_off [n_domains+1]     compact offsets (exclusive scan of counts)
 *   piece_stats [JABBA_PIECE_STATS_BYTES]  exact sums for the normalisation
 * n_domains, n_slots must equal jabba_plan()'s values for this series_off. */
jabba_status jabba_compress(jabba_ctx* ctx, const double* x, int64_t n_points, const int64_t* series_off,
                            int64_t n_series, const jabba_params* p, int64_t n_domains, int64_t n_slots,
                            int64_t* dom_begin, int64_t* dom_end, int32_t* dom_series, int64_t* series_dom_off,
                            int64_t* dom_slot_off, int32_t* piece_len, double* piece_inc, int32_t* dom_piece_cnt,
                            int64_t* dom_piece_off, void* piece_stats, jabba_stream stream);

/* ---------------------------------------------------------------- 3. local digitization
 * Normalisation (Sec. 3.2 Eq. 4): sigma_len, sigma_inc = population standard
 * deviations over ALL pieces (from exact sums: m = S1/N, v = S2/N - m*m,
 * sigma = sqrt(v), or 1 when v <= 0), X = (scl * len) / sigma_len,
 * Y = inc / sigma_inc.  Greedy aggregation per domain (Sec. 3.2, Sec. 5
 * Stage I with one block per domain): pieces in order of X*X + Y*Y (ties by
 * position); each unassigned piece starts a group and every later unassigned
 * piece q with (X_q - X_p)^2 + (Y_q - Y_p)^2 <= alpha^2 joins it.
 * Sort key (key_mode): X*X + Y*Y, or with key_mode = 1 the projection
 * vx * X + vy * Y on the first principal axis (vx, vy) of the normalised
 * pieces.  The axis: normalising by the standard deviations makes the
 * covariance of (X, Y) [[scl^2, scl r], [scl r, 1]] in exact arithmetic (a
 * zero variance stays zero), r = (S_li / N - m_l * m_i) / (sigma_len *
 * sigma_inc) with S_li the exact sum of the products len * inc (each
 * truncated toward zero at 2^-64) and m_l, m_i the means; with a = scl * scl,
 * d = 1, b = scl * r (0 for a zero variance), the leading eigenvector is
 * (1, 0) or (0, 1) when b = 0 (a >= d picks the first), else, with
 * h = (a - d) / 2 and lam = (a + d) / 2 + sqrt(h * h + b * b), the vector
 * (lam - d, b) if a >= d, else (b, lam - a), divided by its norm and signed
 * so that vx > 0 (or vx = 0 and vy > 0); binary64 in this order.  The
 * greedy's key gap bound becomes |key_q - key_p| > alpha (a projection on a
 * unit axis changes by at most the distance).
 * Outputs: sigma[2] = {sigma_len, sigma_inc} (sigma[4] with key_mode = 1:
 * then sigma[2], sigma[3] = vx, vy); local_label [n_slots] (slotted,
 * group id within the domain); dom_group_cnt [n_domains]; dom_group_off
 * [n_domains+1] (exclusive scan); groups[group_capacity] (one record per
 * local group, in no particular order; record identity = (domain, local_id));
 * n_groups (device scalar).  Overflow of group_capacity -> JABBA_ERR_CAPACITY. */
jabba_status jabba_digitize_local(jabba_ctx* ctx, const int32_t* piece_len, const double* piece_inc,
                                  const int64_t* dom_slot_off, const int32_t* dom_piece_cnt, int64_t n_domains,
                                  const void* piece_stats, const jabba_params* p, double* sigma,
                                  int32_t* local_label, int32_t* dom_group_cnt, int64_t* dom_group_off,
                                  jabba_group* groups, int64_t group_capacity, int64_t* n_groups,
                                  jabba_stream stream);

/* ---------------------------------------------------------------- 4. global merge
 * Sec. 5 Stage II: the same greedy over all local groups, each taken as the
 * point (X, Y) of its centre (c_len = lensum / count, c_inc = round(inc) / count,
 * X = (scl * c_len) / sigma_len, Y = c_inc / sigma_inc), ordered by X*X + Y*Y
 * (key_mode = 1: by vx * X + vy * Y with the axis sigma[2..3] that
 * jabba_digitize_local wrote) with ties broken by compact group index
 * dom_group_off[domain] + local_id.
 * Global ids follow creation order.  Outputs: l2g [G] indexed by compact
 * group index; dictionary entry c = exact mean of its member pieces:
 * dict_len[c] = lensum / count, dict_inc[c] = round(sum inc) / count,
 * dict_count[c] = count; k (device scalar).  k > dict_capacity ->
 * JABBA_ERR_CAPACITY. */
jabba_status jabba_merge_global(jabba_ctx* ctx, const jabba_group* groups, const int64_t* n_groups,
                                int64_t group_capacity, const int64_t* dom_group_off, const double* sigma,
                                const jabba_params* p, int32_t* l2g, double* dict_len, double* dict_inc,
                                int64_t* dict_count, int64_t dict_capacity, int64_t* k, jabba_stream stream);

/* Stage II over given points (the block form below merges the local groups'
 * starting points, as Sec. 5 states Stage II): as jabba_merge_global, but
 * group record r is taken as the binary64 point (item_X[r], item_Y[r])
 * (indexed like `groups`) instead of its centre; the dictionary entries are
 * still the exact means of the member pieces. */
jabba_status jabba_merge_global_points(jabba_ctx* ctx, const jabba_group* groups, const double* item_X,
                                       const double* item_Y, const int64_t* n_groups, int64_t group_capacity,
                                       const int64_t* dom_group_off, const double* sigma, const jabba_params* p,
                                       int32_t* l2g, double* dict_len, double* dict_inc, int64_t* dict_count,
                                       int64_t dict_capacity, int64_t* k, jabba_stream stream);

/* ---------------------------------------------------------------- 4b. block form of Sec. 5
 * The two-stage digitization as Sec. 5 states it, for comparison with the
 * per-domain form above: (1) jabba_block_order sorts ALL pieces once by
 * rho = X*X + Y*Y (binary64, Eq. 4 coordinates; equal keys in compact-piece
 * order) and cuts the sorted order into n_blocks contiguous blocks of
 * ceil(N / n_blocks) pieces (the last ones shorter or empty); it writes sigma
 * (as jabba_digitize_local), order[i] = compact index of the piece at sorted
 * position i, the pieces in sorted order (blk_len, blk_inc [N]) and the
 * blocks as domains: blk_slot_off [n_blocks+1], blk_piece_cnt [n_blocks].
 * (2) jabba_digitize_local on those arrays is Stage I (each block aggregated
 * in its sorted order).  (3) jabba_block_items writes, for every group record
 * r, the normalised point of the group's starting piece (its first piece in
 * key order) into item_X/item_Y [group_capacity].  (4)
 * jabba_merge_global_points merges those points (Stage II).  (5)
 * jabba_symbolize with the block arrays (dom_piece_off = blk_slot_off) gives
 * the symbols in sorted order; jabba_block_scatter(order, ...) puts them in
 * compact-piece order.  Scratch for n_pieces items (about 36 B each) is
 * allocated on the first call that needs more (not during graph capture:
 * JABBA_ERR_STATE); jabba_block_items before any jabba_block_order ->
 * JABBA_ERR_STATE.  n_pieces (host) = the compact piece count. */
jabba_status jabba_block_order(jabba_ctx* ctx, const int32_t* piece_len, const double* piece_inc,
                               const int64_t* dom_slot_off, const int32_t* dom_piece_cnt, const int64_t* dom_piece_off,
                               int64_t n_domains, int64_t n_pieces, const void* piece_stats, const jabba_params* p,
                               int64_t n_blocks, double* sigma, int32_t* order, int32_t* blk_len, double* blk_inc,
                               int64_t* blk_slot_off, int32_t* blk_piece_cnt, jabba_stream stream);
jabba_status jabba_block_items(jabba_ctx* ctx, const int32_t* local_label, const int64_t* blk_slot_off,
                               const int32_t* blk_piece_cnt, const int64_t* blk_group_off, int64_t n_blocks,
                               const int32_t* blk_len, const double* blk_inc, const jabba_group* groups,
                               const int64_t* n_groups, int64_t group_capacity, const double* sigma,
                               const jabba_params* p, double* item_X, double* item_Y, jabba_stream stream);
/* dst[order[i]] = src[i] for i < n. */
jabba_status jabba_block_scatter(jabba_ctx* ctx, const int32_t* order, const int32_t* src, int64_t n, int32_t* dst,
                                 jabba_stream stream);

/* ---------------------------------------------------------------- 5. symbolize
 * Sec. 5 label propagation: symbol[dom_piece_off[d] + j] =
 * l2g[dom_group_off[d] + local_label[dom_slot_off[d] + j]], j < dom_piece_cnt[d].
 * symbol is compact (length = total pieces). */
jabba_status jabba_symbolize(jabba_ctx* ctx, const int32_t* local_label, const int64_t* dom_slot_off,
                             const int32_t* dom_piece_cnt, const int64_t* dom_piece_off,
                             const int64_t* dom_group_off, int64_t n_domains, const int32_t* l2g,
                             int32_t* symbol, jabba_stream stream);

/* ---------------------------------------------------------------- full reassignment (variant)
 * Alg. 1's Digitize(P^(m), D) with the argmin of Sec. 3.2: every piece is
 * assigned the dictionary entry nearest to it in normalised coordinates,
 *     c* = argmin_c d2,  d2 = dx*dx + dy*dy,  dx = X_p - X_c,  dy = Y_p - Y_c,
 * X = (scl * len) / sigma_len and Y = inc / sigma_inc for pieces and entries
 * (binary64 in that order, no fused operations); a tie goes to the smaller
 * entry index.  This is the O(N k) pass that Sec. 5's label propagation
 * (jabba_symbolize) replaces; it exists for comparing the two.  Pieces and
 * domains as for jabba_symbolize; the dictionary is dict_len/dict_inc[*k]
 * (k a device scalar, k <= dict_capacity).  Output: symbol (compact, one per
 * piece, like jabba_symbolize's).  The first call allocates the call's
 * scratch for dict_capacity entries (not during graph capture:
 * JABBA_ERR_STATE). */
jabba_status jabba_reassign(jabba_ctx* ctx, const int32_t* piece_len, const double* piece_inc,
                            const int64_t* dom_slot_off, const int32_t* dom_piece_cnt, const int64_t* dom_piece_off,
                            int64_t n_domains, const double* sigma, const double* dict_len, const double* dict_inc,
                            const int64_t* k, int64_t dict_capacity, const jabba_params* p, int32_t* symbol,
                            jabba_stream stream);

/* Sum of squared errors of an assignment (Sec. 3.2; the quantity whose ratio
 * Table 2 reports): sse (device scalar) = sum over pieces of d2(piece, entry
 * symbol[piece]) with d2 as in jabba_reassign, each term truncated to 2^-64
 * fixed point and the sum rounded once (independent of summation order). */
jabba_status jabba_sse(jabba_ctx* ctx, const int32_t* piece_len, const double* piece_inc, const int64_t* dom_slot_off,
                       const int32_t* dom_piece_cnt, const int64_t* dom_piece_off, int64_t n_domains,
                       const double* sigma, const double* dict_len, const double* dict_inc, const int32_t* symbol,
                       const jabba_params* p, double* sse, jabba_stream stream);

/* ---------------------------------------------------------------- 6. reconstruct
 * Sec. 3.3, per series: inverse digitization (l~, i~) = dictionary entry of
 * each symbol; quantization v = l~ + e, l^ = round(v) (round_mode), e = v - l^,
 * e_0 = 0; inverse compression from t_0 = x[series_off[s]]:
 * xhat[pos + q] = level + (i~ * q) / l^ for q = 1..l^, then level += i~ and
 * pos += l^; points past the series end are dropped, a short chain leaves the
 * tail at the final level.  The pieces of series s are compact symbols
 * [dom_piece_off[series_dom_off[s]], dom_piece_off[series_dom_off[s+1]]).
 * Outputs: qlen (compact, l^ per piece), xhat [n_points]. */
jabba_status jabba_reconstruct(jabba_ctx* ctx, const double* x, int64_t n_points, const int64_t* series_off,
                               int64_t n_series, const int64_t* series_dom_off, const int64_t* dom_piece_off,
                               const int32_t* symbol, const double* dict_len, const double* dict_inc,
                               const jabba_params* p, int32_t* qlen, double* xhat, jabba_stream stream);

/* Adjoint of the reconstruction MSE = (1/n) sum (xhat - x)^2 with respect to
 * dict_inc, lengths l^ (qlen from jabba_reconstruct) held fixed: xhat is then
 * affine in dict_inc and d xhat_{pos_j+q} / d i~_{a_j} = q / l^_j (q <= l^_j),
 * = 1 for every later point of the series.  Recomputes xhat on the fly (no
 * per-point activations are stored).  grad_dict_inc [k] is overwritten. */
jabba_status jabba_reconstruct_backward(jabba_ctx* ctx, const double* x, int64_t n_points,
                                        const int64_t* series_off, int64_t n_series,
                                        const int64_t* series_dom_off, const int64_t* dom_piece_off,
                                        const int32_t* symbol, const int32_t* qlen, const double* dict_inc,
                                        int64_t k, double* grad_dict_inc, jabba_stream stream);

/* Timing hooks for benchmarks (no counterpart in the paper).  While
 * `slot` >= 0 (0..255), every call of a step records a pair of CUDA events
 * around its main kernel on the call's stream, into that slot; the records
 * use cudaEventRecordExternal, so a graph captured meanwhile keeps them.
 * slot = -1 stops recording.  jabba_profile_elapsed synchronizes the events
 * of (slot, stage) and returns the milliseconds between them.  Stages:
 * 0 = compression kernel (with the domain packing), 1 = increments + exact
 * sums, 2 = local aggregation, 3 = global merge (whole call), 4 = label
 * propagation, 5 = the merge-rounds kernel alone. */
jabba_status jabba_profile_slot(jabba_ctx* ctx, int slot);
jabba_status jabba_profile_elapsed(jabba_ctx* ctx, int slot, int stage, float* ms);

/* Diagnostic counters of the last calls (no counterpart in the paper);
 * synchronizes the device.  out[0] = admissibility decisions that needed the
 * exact FP64 evaluation in the last jabba_compress; out[1] = rounds of the
 * last global merge.  n = entries wanted. */
jabba_status jabba_diagnostics(jabba_ctx* ctx, int64_t* out, int n);

/* Self-check of the binary64 division that jabba_merge_global evaluates on
 * the integer units for the exact centres of Eq. 4 (no counterpart in the
 * paper): for i < n, a[i] / b[i] by that path is compared bit for bit with
 * the correctly rounded binary64 quotient.  a, b: device arrays of n
 * doubles; counts: device int64[2], set to (quotients the path handled,
 * quotients that differ); elements outside the path (non-normal operands or
 * quotient, b <= 0) are skipped.  mode 0: b is any divisor; mode 1: b holds
 * member counts 1..4096, divided through their tabulated reciprocals (other
 * values are skipped).  Asynchronous on `stream`. */
jabba_status jabba_check_division(jabba_ctx* ctx, const double* a, const double* b, int64_t n, int mode,
                                  int64_t* counts, jabba_stream stream);

/* Reconstruction error (Sec. 3.3): *out (device scalar) = (1/n) sum (x - xhat)^2,
 * summed in a fixed order (the same result on every call on a device). */
jabba_status jabba_mse(jabba_ctx* ctx, const double* x, const double* xhat, int64_t n_points, double* out,
                       jabba_stream stream);

/* ---------------------------------------------------------------- launch tuning
 * (No counterpart in the paper.)  Launch configuration of the batched
 * kernels.  Every configuration computes the same results (bit for bit); only
 * the speed differs.  Domains of up to 512 pieces are aggregated by one warp
 * each; larger domains by the number of warps chosen here.
 * Defaults: {2, 1, 4, 4, 4, 0, 1, 0, 1, 8}. */
typedef struct {
  int32_t compress_ctas_per_sm; /* CTAs (of 4 warps) per SM of the persistent compression kernel: 1..3; two
                                   are resident at once (shared memory), a third waits for a slot         */
  int32_t compress_pack;        /* 1 = domains handed to warps longest first (length packing), 0 = in order    */
  int32_t local_mid_warps;      /* warps that aggregate one domain of 1025..2048 pieces together: 1, 2, 4, 8   */
  int32_t local_big_warps;      /* warps that aggregate one domain of 2049..4096 pieces together: 4 or 8       */
  int32_t merge_ctas_per_sm;    /* CTAs per SM of the cooperative merge-rounds kernel: 1, 2 or 4 (capped by the
                                   kernel's occupancy so that the grid stays co-resident)                     */
  int32_t per_domain_launch;    /* 1 = the plain (unbatched) form: jabba_compress and jabba_digitize_local
                                   issue one kernel launch per domain, eagerly (they read the piece counts
                                   back to the host); refused during graph capture and autotuning
                                   (JABBA_ERR_STATE).  0 = the batched persistent launches (default)         */
  int32_t local_k_warps;        /* warps that aggregate one domain of 513..1024 pieces together: 1 or 4        */
  int32_t local_ctas_cap;       /* resident CTAs per SM of each local-aggregation kernel: 0 = as many as fit,
                                   1..16 = at most that many (leaves room for a concurrent kernel)            */
  int32_t merge_form;           /* merge rounds: 1 = one grid barrier per round, coverage by the decided
                                   starts tested on the fly (default); 0 = two barriers per round, coverage
                                   marked between them                                                       */
  int32_t merge_warps;          /* warps per CTA of the one-barrier rounds kernel: 8 (default) or 4           */
} jabba_tuning;

/* Autotuning mode.  While enabled (enable = 1), each call of jabba_compress,
 * jabba_digitize_local and jabba_merge_global runs its kernels once per
 * candidate configuration on the call's own inputs, times them with CUDA
 * events, keeps the fastest in the context and returns after synchronizing
 * `stream` (the outputs are those of the call, as without tuning).  Candidates:
 * compression {1, 2, 3} CTAs per SM x {packed, in order}; local aggregation
 * {1, 4} warps per domain of 513..1024 pieces, {1, 2, 4, 8} of 1025..2048 and
 * {4, 8} of 2049..4096; merge {1, 2, 4} CTAs per SM (x {8, 4} warps per CTA in the
 * one-barrier form).  Tuning calls must not be captured in a CUDA graph
 * (JABBA_ERR_STATE).  enable = 0 ends the mode; the choice stays in effect. */
jabba_status jabba_autotune(jabba_ctx* ctx, int enable);
/* Current configuration of the context. */
jabba_status jabba_get_tuning(jabba_ctx* ctx, jabba_tuning* out);
/* Set a configuration (e.g. one cached from an earlier autotuning run);
 * out-of-range fields -> JABBA_ERR_INVALID_ARG and nothing changes. */
jabba_status jabba_set_tuning(jabba_ctx* ctx, const jabba_tuning* in);

/* ---------------------------------------------------------------- allocation-free reconstruction
 * (No counterpart in the paper.)  The same result as jabba_reconstruct, for
 * callers that cannot allocate device memory -- code that runs where
 * cudaMalloc is not allowed or must not be called (inside a stream capture
 * someone else owns, under an allocation-free memory budget, in a callback)
 * and therefore cannot create a context, whose scratch comes from cudaMalloc.
 * No context: the scratch is a fixed array in the library's own device
 * memory (JABBA_NOALLOC_MAX_PIECES pieces and JABBA_NOALLOC_MAX_SERIES series,
 * about 4.5 MB, held by every GPU that loads the library until the process
 * exits).  Larger inputs return JABBA_ERR_CAPACITY; nothing is allocated or
 * freed.  The first call on a device looks up the array's device address
 * (set-up, once per device): make that first call before any stream capture.
 * Every call shares the one array, which keeps the last call's contents:
 * calls that overlap on the GPU (different streams, concurrent host threads)
 * race and must be serialized by the caller.  Arguments as for
 * jabba_reconstruct, plus n_pieces (host value, the number of compact
 * symbols) and round_mode.  The kernels also check on the device that every
 * series' first piece dom_piece_off[series_dom_off[s]] lies in [0, n_pieces]
 * (so an understated n_pieces cannot make them write past the scratch or
 * qlen); when it does not, the call writes nothing and records
 * JABBA_ERR_CAPACITY in a status word that jabba_reconstruct_noalloc_status
 * returns. */
#define JABBA_NOALLOC_MAX_PIECES (1 << 18)
#define JABBA_NOALLOC_MAX_SERIES (1 << 14)
jabba_status jabba_reconstruct_noalloc(const double* x, int64_t n_points, const int64_t* series_off,
                                       int64_t n_series, const int64_t* series_dom_off,
                                       const int64_t* dom_piece_off, int64_t n_pieces, const int32_t* symbol,
                                       const double* dict_len, const double* dict_inc, int32_t round_mode,
                                       int32_t* qlen, double* xhat, jabba_stream stream);
/* Synchronize `stream` and return (and clear) the status word of the
 * allocation-free reconstruction on the current device: JABBA_OK, or
 * JABBA_ERR_CAPACITY when a call since the last query failed its device-side
 * bounds check (that call wrote no output). */
jabba_status jabba_reconstruct_noalloc_status(jabba_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* JABBA_H */
