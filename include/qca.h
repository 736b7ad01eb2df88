/*
 * qca.h -- C ABI of libqca, a GB300 (sm_103a) implementation of the local
 * message-passing automaton decoder of arXiv 2506.03266 ("Fast offline
 * decoding with local message-passing automata") for the 2D toric code.
 *
 * The decoder (Sec. 3.2, Def. "D-dimensional message passing automaton", D = 2,
 * run as a synchronous automaton decoder, Def. "synchronous automaton decoder"):
 * every site of an L x L torus holds four message fields m^{+x}, m^{-x}, m^{+y},
 * m^{-y}.  One time step applies the automaton rule v times with the syndrome
 * held fixed (messages are emitted by anyons, propagate one site per sub-step
 * along their direction over an infinity-norm light cone, and carry the
 * distance travelled; smaller values overwrite larger), then moves every anyon
 * one link toward the smallest message it holds (feedback, Eq. ddfeedback);
 * anyons that meet annihilate.  Steps repeat until no anyon is left or the
 * step budget is spent; the logical failure check follows (Def. plogandtdec,
 * Sec. 7.2).
 *
 * Conventions shared by every entry point:
 *   - site r = (x, y), 0 <= x, y < L, row-major index y*L + x; periodic.
 *   - edge (qubit) arrays: uint8 [shots][2][L][L], values 0 / 1.  Plane 0 is
 *     e_x(r) = <r, r + x^>, plane 1 is e_y(r) = <r, r + y^>.
 *   - all array pointers are caller-owned DEVICE memory unless the entry point
 *     name ends in _host; the library never frees them.
 *   - a typed array (int32, int64, float ...) must start on a multiple of its
 *     element size, else QCA_ERR_ARG.  uint8 arrays may start anywhere: where
 *     an input or correction array (or a packed shot block) is not 4-byte
 *     aligned, the decoder uses its byte-access kernel instead of the faster
 *     word-access ones, with the same results.
 *   - "stream" arguments are cudaStream_t handles passed as void*; NULL means
 *     the legacy default stream.  *_async calls return after enqueueing; the
 *     others synchronise before returning.
 *   - return value: 0 on success, or a negative QCA_ERR_* code; on error
 *     qca_last_error() describes the cause.  No entry point aborts, traps or
 *     prints.  Every device loop is bounded by max_steps.
 */
#ifndef QCA_H
#define QCA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QCA_OK 0
#define QCA_ERR_ARG (-1)         /* bad argument: L < 3, negative count, NULL pointer ... */
#define QCA_ERR_UNSUPPORTED (-2) /* size or option outside what the kernels support      */
#define QCA_ERR_CUDA (-3)        /* a CUDA runtime call or kernel launch failed           */
#define QCA_ERR_WATCHDOG (-4)    /* a bounded device wait gave up                          */

#define QCA_MAX_L 1024       /* largest lattice any kernel accepts                  */
#define QCA_MAX_STEPS (1 << 20)
#define QCA_MAX_L_1D 16384   /* longest ring of the 1D decoder                      */

/* Decoder options.  Defaults (qca_default_config) are the paper's numerics
 * (Sec. 7: v = 3, deterministic rule) with an 8-bit message register.
 * tie_order and balance_rule select between readings of Eqs. blahdef /
 * degbreak; the 2D torus entry points (uniform, uneven, syndrome, host, no
 * allocation, net + automaton) take every value, the 1D, open-boundary and
 * desynchronised decoders only the defaults (QCA_ERR_UNSUPPORTED otherwise). */
typedef struct qca_config {
  int32_t v;             /* message sub-steps per time step (A^(v,D) = (A^(D))^v, Def.
                            Dd_msg_passing); supported: 1..8; default 3                     */
  int32_t m_max;         /* message cap (Eq. mvals); values above it disappear; 1..255;
                            default 255                                                     */
  double p_move;         /* probability that an anyon moves in a uniformly random direction
                            instead of following its messages (the random motion of the
                            limited-memory corollary of Sec. 5.1); default 0                 */
  int64_t shot_offset;   /* index of this batch's first shot in the random-move stream;
                            default 0                                                       */
  int32_t tie_order;     /* argmin' of Eq. degbreak among equal-valued fields:
                            QCA_TIE_LEX (default): smallest m, then the smallest s*a, i.e.
                              (-,y) before (-,x) before (+,x) before (+,y);
                            QCA_TIE_LITERAL: the printed offset s*a/(D+1) taken as is, i.e.
                              the smallest integer key 3m + s*a, and where two keys are
                              equal (m^{-y} = k+1 against m^{+x} = k, or m^{-x} = k+1
                              against m^{+y} = k) the larger m                              */
  int32_t balance_rule;  /* anyon whose chosen axis a is balanced (m^{+a} = m^{-a} > 0):
                            QCA_BALANCE_STAY (default): no move (the deterministic rule of
                              the paper's footnote on steady states, Sec. 5.3);
                            QCA_BALANCE_RANDOM: one link along +a or -a, +a when the top bit
                              of splitmix64(splitmix64(splitmix64(splitmix64(rng_seed ^
                              0x42414C414E4345) ^ (shot_offset + shot)) ^ t) ^ (y L + x))
                              is 0 (t = step index from 0)                                   */
} qca_config;

#define QCA_TIE_LEX 0
#define QCA_TIE_LITERAL 1
#define QCA_BALANCE_STAY 0
#define QCA_BALANCE_RANDOM 1

/* Fill *cfg with the defaults above.  Returns QCA_ERR_ARG if cfg is NULL. */
int qca_default_config(qca_config* cfg);

/* i.i.d. bit-flip noise of strength p on every link (Sec. 7 numerics, the
 * i.i.d. case of Eq. final_channel).  Writes out_errors, device uint8
 * [shots][2][L][L].  Link e of shot s (e = 2*(y*L+x) + plane, s counted from
 * shot0) flips iff splitmix64(splitmix64(splitmix64(seed ^ 0x4E4F495345) ^ s) ^ e)
 * < floor(p * 2^64), so the same (seed, shot, link) gives the same draw at any
 * batch split, and a lower p flips a subset of a higher p's links.
 * Errors: QCA_ERR_ARG for L < 3, L > QCA_MAX_L, shots < 0, NULL with shots > 0,
 * p outside [0, 1]. */
int qca_sample_errors(int L, int shots, double p, uint64_t seed, uint8_t* out_errors);
int qca_sample_errors_async(int L, int64_t shot0, int64_t shots, double p, uint64_t seed,
                            uint8_t* out_errors, void* stream);

/* Decode a batch of noise realisations (the decoding problem of
 * Def. plogandtdec; Sec. 7 Monte Carlo).
 *   syndrome          device uint8 [shots][2][L][L]: the per-shot noise realisation N
 *                     (link bits); the syndrome sigma is measured from it on the device
 *                     (Def. synch_ccqs).  N is needed because the failure flag is a
 *                     property of N xor C, not of sigma alone.
 *   L                 lattice size, 3 <= L <= QCA_MAX_L
 *   shots             number of independent shots, >= 0
 *   max_steps         step budget per shot, 0 <= max_steps <= QCA_MAX_STEPS
 *   rng_seed          seed of the optional random-move rule; unused with p_move = 0
 *   out_correction    device uint8 [shots][2][L][L]: the applied correction C
 *   out_steps         device int32 [shots]: feedback steps until no anyon is left
 *                     (T_dec of the shot, Eq. tdecrhodef), or max_steps
 *   out_logical_fail  device uint8 [shots]: 0 success; 1 N xor C wraps a torus cycle
 *                     (either cycle, Sec. 7.2); 2 the budget ran out with anyons left
 * Uses the default qca_config; synchronises.  Outputs are bit-identical to the
 * library's CPU oracle for every input.  Errors: QCA_ERR_ARG (sizes, NULL with
 * shots > 0), QCA_ERR_UNSUPPORTED, QCA_ERR_CUDA. */
int qca_decode_batch(const uint8_t* syndrome, int L, int shots, int max_steps,
                     uint64_t rng_seed, uint8_t* out_correction, int32_t* out_steps,
                     uint8_t* out_logical_fail);
/* As qca_decode_batch with options (cfg may be NULL for the defaults), enqueued
 * on `stream` without synchronising. */
int qca_decode_batch_async(const uint8_t* syndrome, int L, int64_t shots, int max_steps,
                           uint64_t rng_seed, uint8_t* out_correction, int32_t* out_steps,
                           uint8_t* out_logical_fail, const qca_config* cfg, void* stream);

/* Decode pure syndromes: sigma is device uint8 [shots][L][L] with 1 marking an
 * anyon (sigma_r = -1).  Writes the correction C, the steps, out_cut_parity
 * device uint8 [shots][2] = (w_x, w_y) of C alone (w_x = XOR over y of
 * C.e_x((0,y)), w_y = XOR over x of C.e_y((x,0))), and out_exhausted device
 * uint8 [shots] (1 if the budget ran out; may be NULL).  Because N xor C is a
 * cycle on success, the caller's failure flag is cut(N) xor cut(C).  An odd
 * number of anyons cannot empty and runs to the budget. */
int qca_decode_syndrome_batch_async(const uint8_t* sigma, int L, int64_t shots, int max_steps,
                                    uint64_t rng_seed, uint8_t* out_correction,
                                    int32_t* out_steps, uint8_t* out_cut_parity,
                                    uint8_t* out_exhausted, const qca_config* cfg,
                                    void* stream);

/* Synchronous companion of qca_decode_batch for pure syndromes (footnote of
 * Def. plogandtdec: the decoder sees sigma only): the arguments of
 * qca_decode_syndrome_batch_async without out_exhausted, options and stream;
 * default options, legacy default stream, synchronises before returning.  An
 * exhausted budget shows as out_steps[s] == max_steps with the syndrome left
 * non-empty (use the async form's out_exhausted to tell it apart).  Errors
 * as for the async form. */
int qca_decode_syndrome_batch(const uint8_t* sigma, int L, int shots, int max_steps,
                              uint64_t rng_seed, uint8_t* out_correction, int32_t* out_steps,
                              uint8_t* out_cut_parity);

/* End-to-end form of qca_decode_batch on HOST buffers (same layouts): copies
 * the noise to the device in chunks, decodes, and copies the correction, steps
 * and flags back, overlapping transfers with decoding.  Host buffers should be
 * page-locked for full speed.  out_correction may be NULL (not copied back).
 * Uses a device staging workspace cached by the library (qca_free_workspace
 * releases it).  Synchronises; on an error it still waits for the copies it
 * had enqueued, so none touches the caller's buffers after it returns. */
int qca_decode_batch_host(const uint8_t* syndrome, int L, int64_t shots, int max_steps,
                          uint64_t rng_seed, uint8_t* out_correction, int32_t* out_steps,
                          uint8_t* out_logical_fail, const qca_config* cfg);

/* Size of the fixed device array behind qca_decode_batch_noalloc: 16 MiB. */
#define QCA_NOALLOC_SCRATCH_BYTES (16 << 20)

/* qca_decode_batch_async for callers that must not allocate device memory.
 * (The paper has no counterpart; this is a property of the library.)
 *
 * Who needs it: code that may not call cudaMalloc or any routine that
 * allocates -- for instance a control loop that has reserved all device memory
 * up front and must keep its latency free of allocator calls, a host that hands
 * the whole device to its own memory pool, or a caller in the middle of work
 * where allocation is not permitted.  This entry point allocates nothing: the
 * caller passes the inputs and outputs (same meaning and layout as
 * qca_decode_batch), and the decoder state lives in a fixed array of
 * QCA_NOALLOC_SCRATCH_BYTES that the library places in device memory when it is
 * loaded (every GPU that loads the library keeps it until the process exits).
 * It always runs the generic sweep, so results are bit-identical to
 * qca_decode_batch.
 *
 *  - The first call on a device (with that device current) looks up the
 *    array's device address, which loads the array and the kernel onto the
 *    device; a call with shots = 0 does this and nothing else.  Make that
 *    first call while setting up, before reserving the device's memory for
 *    other uses and before any stream capture.
 *  - Each shot needs 14 * L * L bytes (rounded up to 256) of the array; an L
 *    whose single shot does not fit is rejected with QCA_ERR_UNSUPPORTED.
 *    min(4 * SMs, floor(QCA_NOALLOC_SCRATCH_BYTES / that)) shots are decoded
 *    at once, one CTA each, and larger batches take turns: 608 at once on a
 *    152-SM GPU up to L = 44, 18 at L = 256, 8 at L = 384, and one at
 *    L = 1024 (a single CTA then decodes the whole batch, shot after shot,
 *    which is correct but slow).
 *  - Every call shares the one array, which keeps the last call's contents:
 *    calls that overlap on the GPU (for instance on two streams without an
 *    ordering between them) race and give wrong results.  Issue them on one
 *    stream, or order them.
 * Errors as for qca_decode_batch_async. */
int qca_decode_batch_noalloc(const uint8_t* syndrome, int L, int64_t shots, int max_steps,
                             uint64_t rng_seed, uint8_t* out_correction, int32_t* out_steps,
                             uint8_t* out_logical_fail, const qca_config* cfg, void* stream);

/* ---- Uneven batches: shots of different lattice sizes in one decode ------
 * The Monte-Carlo sweeps of Sec. 7 cover several L; these entry points decode a
 * mix of sizes together.  Shots are packed back to back: shot s occupies the
 * uint8 [2][L_s][L_s] block at byte offset off_s = sum_{t<s} 2 L_t^2 of the
 * input (and of the correction output); steps and flags are indexed by s. */

/* Per-shot L and noise threshold of the mixed synthetic workload (host only):
 * L_s in {24, 48, 64, 96, 128, 192} with probabilities 30/25/20/12/8/5 %,
 * drawn as splitmix64(splitmix64(seed ^ 0x4C53495A45) ^ s) against cumulative
 * cut points floor(c/100 * 2^64); the flip threshold is
 * floor(0.01 * 2^64) + ((v * floor(0.06 * 2^64)) >> 64) with
 * v = splitmix64(splitmix64(seed ^ 0x5052415445) ^ s), i.e. p ~ U[0.01, 0.07).
 * Writes out_L[shots] and out_thr[shots] (host arrays). */
int qca_uneven_draw(int64_t shots, uint64_t seed, int32_t* out_L, uint64_t* out_thr);

typedef struct qca_uneven_plan_s* qca_uneven_plan_t;

/* Group the shots (host array L_host[shots]) by size and place the shot lists,
 * the block offsets and the work counters in device memory owned by the plan.
 * offsets_host (may be NULL) receives off_s; total_bytes (may be NULL) the size
 * of the packed input.  Not for use under stream capture (it allocates). */
int qca_uneven_plan_create(const int32_t* L_host, int64_t shots, int64_t* offsets_host,
                           int64_t* total_bytes, qca_uneven_plan_t* out_plan);
int qca_uneven_plan_destroy(qca_uneven_plan_t plan);
/* Launch form of qca_decode_uneven_async for this plan: 0 (default) one
 * mixed-size persistent launch, 1 one persistent launch per size. */
int qca_uneven_plan_set_mode(qca_uneven_plan_t plan, int mode);
/* Device array of the plan's block offsets (int64 [shots]), owned by the plan. */
int qca_uneven_plan_offsets_device(qca_uneven_plan_t plan, const int64_t** offsets_device);

/* i.i.d. noise for a packed uneven batch: shot s gets the L_s x L_s torus at
 * offsets_dev[s] with flip threshold thr_dev[s] (all device arrays); the link
 * draws are those of qca_sample_errors for shot index s. */
int qca_sample_errors_uneven_async(const int32_t* L_dev, const int64_t* offsets_dev,
                                   const uint64_t* thr_dev, int64_t shots, uint64_t seed,
                                   uint8_t* out_errors, void* stream);

/* Decode a packed uneven batch.  Default (mode 0 of qca_uneven_plan_set_mode):
 * one persistent launch for the shots of every size the on-chip sweep takes
 * (multiples of 4 up to 128 and of 8 up to 256, blocks on a 4-byte boundary;
 * the 8 largest such sizes), queued pairs first, then by group size, then
 * largest L first.
 * Clusters of two CTAs take the shots with L > 192; every other size is
 * decoded by a group of 512, 256 or 128 threads (the smallest that fits), a
 * 512-thread CTA halving into up to four groups as the queue reaches smaller
 * sizes; each takes its next shot when the last one is done (work stealing
 * across sizes; every shot retires after its own number of steps); shots of
 * other sizes go to per-size launches on streams forked from `stream` before
 * it, which run beside it.  Mode 1: one persistent launch per
 * size, each on a stream forked from and joined to `stream`, so that the sizes
 * run side by side.  Only kernel launches, memset and
 * event operations are enqueued, so the call can be captured in a CUDA graph
 * once one uncaptured call has sized the library's workspaces.  Outputs are
 * bit-identical to decoding each shot with qca_decode_batch in either mode. */
int qca_decode_uneven_async(qca_uneven_plan_t plan, const uint8_t* errors, int max_steps,
                            uint64_t rng_seed, uint8_t* out_correction, int32_t* out_steps,
                            uint8_t* out_logical_fail, const qca_config* cfg, void* stream);

/* ---- Tuning of the on-chip sweep (per lattice size, process-wide) --------
 * band_height: rows of one plane a warp segment sweeps (4, 8, 16 or 32; it sets
 * the threads per CTA and so the CTAs per SM); 0 = built-in heuristic (the band
 * whose warp count is nearest 4 up to L = 64, L / 8 above, at most 16; where
 * none of the four heights fits a size, another divisor of the CTA's rows of
 * at least 4, by the same rule).
 * sparse_divisor: steps with at most L^2 / sparse_divisor anyons write the
 * anyon terms per anyon, busier steps compute them densely; 0 = the default,
 * 64 for the one-CTA kernel (L <= 128) and 256 for the two-CTA cluster.
 * An override that does not fit a size is ignored. */
int qca_set_tuning(int L, int band_height, int sparse_divisor);
/* CTAs per cluster of the on-chip sweep for 128 < L <= 256 (L % 8 == 0): 2 (each
 * CTA holds half the rows of every plane, one CTA per SM; the default) or 4 (a
 * quarter of the rows, 256 threads; two clusters' CTAs share an SM, so one
 * shot's latency-bound phases overlap another's message update; measured
 * slower on GB300 at L = 192 and 256).  Same results either way.
 * Process-wide; QCA_ERR_ARG outside that range. */
int qca_set_cluster_ctas(int L, int ctas);
/* Current effective values and the resulting threads per CTA (QCA_ERR_UNSUPPORTED
 * if L has no on-chip kernel). */
int qca_get_tuning(int L, int* band_height, int* sparse_divisor, int* threads_per_cta);
/* Time every valid (band_height, sparse_divisor) on `shots` shots of i.i.d.
 * noise p (seed) and keep the fastest as the setting for L.  Allocates
 * temporary device memory; synchronises. */
int qca_autotune(int L, int64_t shots, double p, uint64_t seed, int max_steps,
                 int* best_band_height, int* best_sparse_divisor, float* best_ms);

/* ---------------------------------------------------------------------------
 * 1D message-passing automaton decoder for the repetition code (Sec. 3.1,
 * Def. "message passing automaton, 1D"; Sec. 7.1 numerics).  A ring of L sites
 * (3 <= L <= QCA_MAX_L_1D); the qubit of link <r, r+1> is byte r of the noise
 * and correction arrays, device uint8 [shots][L]; anyons sit on sites.  Each
 * step applies A^(1) v times (fields m^+ from the left, m^- from the right,
 * value = distance travelled, a value above m_max vanishes), then moves every
 * anyon one link toward the smaller field (an empty field counts as +infinity;
 * no move on a tie), a link crossed from both ends flipping once.  With
 * cfg->p_move > 0 an anyon moves in a uniformly random direction with that
 * probability instead (Sec. 7.1 uses 10 %); the draw per (shot, step, site)
 * is splitmix64 of the same key chain as the 2D option.
 * ------------------------------------------------------------------------- */

/* Noise: link r of shot s (counted from shot0) flips iff
 * splitmix64(splitmix64(splitmix64(seed ^ 0x4E4F49534531) ^ s) ^ r) < floor(p * 2^64). */
int qca_sample_errors_1d_async(int L, int64_t shot0, int64_t shots, double p, uint64_t seed,
                               uint8_t* out_errors, void* stream);

/* Decode: out_correction [shots][L]; out_steps int32 [shots]; out_flag uint8
 * [shots] = 0 when N xor C is all zeros (the encoded value), 1 when it is all
 * ones (a logical error), 2 when the budget ran out with anyons left;
 * out_majority_flag (may be NULL) = 1 when the decoded value differs from the
 * majority vote of the input bits (more than L/2 set), the success criterion
 * of the paper's 1D numerics, 2 on an exhausted budget.  cfg may be NULL
 * (v = 3, m_max = 255, no random moves); v 1..8, m_max 1..255. */
int qca_decode_1d_batch_async(const uint8_t* noise, int L, int64_t shots, int max_steps,
                              uint64_t rng_seed, const qca_config* cfg, uint8_t* out_correction,
                              int32_t* out_steps, uint8_t* out_flag, uint8_t* out_majority_flag,
                              void* stream);

/* ---------------------------------------------------------------------------
 * Two variants of the 2D decoder (literal per-site sweep, state in a cached
 * device workspace of 14 L^2 bytes per resident shot; noise, correction,
 * steps and flag arrays as in qca_decode_batch).
 * ------------------------------------------------------------------------- */

/* Open boundaries (Appendix "Open boundary conditions", Def. "message passing
 * automaton with open boundaries"): an L x L grid without wrap whose columns
 * x = 0 and x = L-1 are rough boundaries.  Qubits: e_x(x, y) for x <= L-2 and
 * e_y(x, y) for 1 <= x <= L-2, y <= L-2; the other entries of the noise array
 * are ignored and stay 0 in the correction.  The boundary holds no messages,
 * sources x messages into the bulk (m^{+x} from x = 0, m^{-x} from x = L-1)
 * and absorbs anyons; sets C^(a) lose their members outside the grid.
 * out_logical_fail: 0 success, 1 N xor C crosses the cut between columns 0
 * and 1 an odd number of times (it joins the two boundaries), 2 budget.  cfg:
 * v and m_max as for the torus; p_move must be 0. */
int qca_decode_open_batch_async(const uint8_t* noise, int L, int64_t shots, int max_steps,
                                const qca_config* cfg, uint8_t* out_correction,
                                int32_t* out_steps, uint8_t* out_logical_fail, void* stream);

/* Uncoordinated desynchronisation (Sec. 7.3) on the torus: time advances in
 * ticks of length q (0 <= q <= 1); per tick each site fires its message
 * update with probability min(1, v q) and, holding an anyon, its move with
 * probability q, from the draws
 *   splitmix64(splitmix64(splitmix64(splitmix64(rng_seed ^ 0x444553594E43)
 *              ^ (shot_offset + shot)) ^ tick) ^ (2 r + c)) < floor(prob * 2^64),
 * c = 0 (messages) or 1 (move), r = y L + x.  The firing message updates of a
 * tick are one application of A^(D) at those sites, from the fields before
 * the tick; the firing anyons then move by the forces of the updated fields
 * (OR feedback); sigma is updated last.  out_ticks: ticks until no anyon is
 * left (or max_ticks); out_logical_fail as for qca_decode_batch.  q = 1 with
 * v = 1 is exactly the synchronous decoder with v = 1. */
int qca_decode_desync_batch_async(const uint8_t* noise, int L, int64_t shots, int max_ticks,
                                  double q, uint64_t rng_seed, const qca_config* cfg,
                                  uint8_t* out_correction, int32_t* out_ticks,
                                  uint8_t* out_logical_fail, void* stream);

/* ---------------------------------------------------------------------------
 * Learned pre-decoder in front of the automaton.  The paper has no learned
 * component; this stage is an addition whose only job is to pair off nearby
 * anyons before the automaton (the paper's decoder, unchanged) finishes every
 * shot: every anyon the net leaves is decoded exactly as without it, and the
 * shot's outcome is the automaton's.
 *
 * The net: four 3x3 convolutions with circular (periodic) padding,
 * 2 -> 32 -> 32 -> 32 -> 4 channels, ReLU between layers.  Input channel 0 is
 * the anyon indicator (sigma_r = -1), channel 1 is constant 1.  Output channel
 * k is the logit of a move in direction k: 0 = +x, 1 = -x, 2 = +y, 3 = -y
 * (the fifth class "no move" has logit 0).  Parameters: fp32, flat, per layer
 * W[c_out][c_in][3][3] (tap (ky, kx) reads site (x + kx - 1, y + ky - 1))
 * followed by b[c_out]; qca_net_param_count() floats in all.
 *
 * Inference rounds the weights and each layer's input to bfloat16 (round to
 * nearest even) and accumulates in fp32 (tensor cores for layers 2-4); logits
 * are fp32.  Pairing: an anyon proposes direction argmax_k z_k if that logit
 * is > 0 (first index on ties), else nothing; the link <r, r + a^> joins the
 * pre-decoder correction C0 iff r proposes +a and r + a^ proposes -a.
 *
 * Labels (training targets) come from the automaton's own first step: with all
 * fields empty, v = 3 sub-steps and the forces of Eqs. blahdef / degbreak give
 * each anyon a move direction (or none); an anyon is labelled with its
 * direction when the anyon next to it in that direction moves back toward it
 * (the pair annihilates in that step), else 4 ("no move"); non-anyon sites
 * are 255 (ignored).
 *
 * A qca_net_t handle belongs to the device that was current when it was
 * created; calls on one handle must not overlap (no internal locking).
 * ------------------------------------------------------------------------- */
typedef struct qca_net_s* qca_net_t;

/* Number of fp32 parameters of the net. */
int64_t qca_net_param_count(void);

/* Create a net with He-normal weights drawn from splitmix64(seed ...) and zero
 * biases; *out receives the handle.  Allocates a few hundred KB of device
 * memory on the current device. */
int qca_net_create(uint64_t seed, qca_net_t* out);

/* Free the handle and its device memory (NULL is accepted). */
int qca_net_destroy(qca_net_t net);

/* Copy the fp32 parameters to / from HOST memory; count must equal
 * qca_net_param_count().  Synchronous. */
int qca_net_get_params(qca_net_t net, float* host_params, int64_t count);
int qca_net_set_params(qca_net_t net, const float* host_params, int64_t count);

/* Train on freshly drawn syndromes: `iterations` Adam steps (betas 0.9 /
 * 0.999, epsilon 1e-8, learning rate lr), each on `batch` L x L tori whose
 * links flip i.i.d. with a per-torus probability drawn uniformly from
 * [p_lo, p_hi) (splitmix64 counter stream of `seed`; the stream position
 * advances across calls on the same handle).  Loss: mean softmax
 * cross-entropy over the anyon sites against the first-step labels above,
 * smoothed by 0.1 (that mass spread evenly over the five classes).
 * Forward, input gradients and weight gradients run as bf16 tensor-core
 * implicit GEMMs with fp32 accumulation and fp32 master weights.  out_losses (HOST, may be
 * NULL) receives one loss per iteration.  4 <= L <= 128, batch * L * L <=
 * 2^24.  Allocates its buffers for the duration of the call; synchronous. */
int qca_net_train(qca_net_t net, int L, int64_t iterations, int batch, double p_lo, double p_hi,
                  uint64_t seed, float lr, float* out_losses);

/* One forward and backward pass of the training loss on given noise
 * realisations (device uint8 [batch][2][L][L], labels from the automaton's
 * first step as for qca_net_train) without updating the weights: host_grads
 * (HOST, count = qca_net_param_count() floats) receives the gradient in the
 * parameter layout, *host_loss (may be NULL) the loss.  Same arithmetic as a
 * training step.  4 <= L <= 128; synchronous. */
int qca_net_gradients(qca_net_t net, const uint8_t* noise, int L, int batch, float* host_grads,
                      int64_t count, float* host_loss);

/* First-step labels of noise realisations: noise uint8 [shots][2][L][L],
 * out_labels uint8 [shots][L][L] (values as above), scratch >= 2 * shots * L^2
 * bytes of device memory.  4 <= L <= QCA_MAX_L. */
int qca_net_labels_async(const uint8_t* noise, int L, int64_t shots, uint8_t* out_labels,
                         uint8_t* scratch, void* stream);

/* Shots per inference chunk at size L (the net runs chunk by chunk: six
 * kernel launches per chunk), or QCA_ERR_ARG for L outside [4, QCA_MAX_L]. */
int64_t qca_net_chunk_shots(int L);

/* Logits of the net: out_logits fp32 [shots][4][L][L].  The handle keeps an
 * inference workspace (about 130 bytes per site of up to 4 GiB worth of
 * shots) that grows on demand; growth synchronises the device, so make one
 * call of the largest size before capturing a stream. */
int qca_net_logits_async(qca_net_t net, const uint8_t* noise, int L, int64_t shots,
                         float* out_logits, void* stream);

/* Checking aid: run the net's forward (the active precision and tensor path)
 * on noise device uint8 [shots][2][L][L] and write the activations of layer
 * `layer` (1..3) as the next layer reads them into out (device fp32
 * [shots][32][L][L]): the bf16 values, or in the FP8 form the e4m3 values,
 * which the next layer multiplies by the scale s_layer.  Lets a test feed the kernels' own layer-k output into an
 * FP64 layer k+1.  1 <= shots <= qca_net_chunk_shots(L).  Allocates a
 * temporary buffer; runs on the legacy default stream and synchronises. */
int qca_net_activations(qca_net_t net, const uint8_t* noise, int L, int64_t shots, int layer,
                        float* out);

/* Pre-decode: out_residual uint8 [shots][2][L][L] = N xor C0 and, if out_c0
 * is not NULL, out_c0 = C0 (same layout). */
int qca_net_predecode_async(qca_net_t net, const uint8_t* noise, int L, int64_t shots,
                            uint8_t* out_residual, uint8_t* out_c0, void* stream);

/* FP8 (E4M3) form of the net.  Layers 2-4 run on e4m3 tensor-core MMAs with
 * fp32 accumulation: weights quantised per output channel as e4m3(W / s_co),
 * s_co = max|W_co| / 448 (fp32; 1 for an all-zero channel), each layer's input
 * quantised as e4m3(x / s_l) with per-layer activation scales s_1..s_3
 * (round to nearest even, saturating at 448); layer 1 is the bf16 form's.
 * qca_net_calibrate_fp8 sets s_l = max(activation) / 448 from the bf16 form's
 * activations on the given noise (device uint8 [shots][2][L][L]; at most one
 * inference chunk of it is used); synchronous.  qca_net_set_fp8_scales sets
 * them directly (three positive floats, HOST), qca_net_get_fp8_scales reads
 * them.  qca_net_set_precision(net, 1) makes every inference entry point
 * (logits, pre-decode, net + automaton decode) use the FP8 form, 0 the bf16
 * form; FP8 needs scales first (QCA_ERR_ARG otherwise). */
int qca_net_calibrate_fp8(qca_net_t net, const uint8_t* noise, int L, int64_t shots, void* stream);
int qca_net_set_fp8_scales(qca_net_t net, const float* scales);
int qca_net_get_fp8_scales(qca_net_t net, float* scales);
int qca_net_set_precision(qca_net_t net, int precision);

/* Tensor path of layers 2-4 where L is a multiple of 128 (mma.sync elsewhere):
 * 2 (default) = tcgen05 MMAs with the accumulator in tensor memory,
 * warp-specialised (producer warps stage rows into a ring, one thread issues
 * the MMAs, epilogue warps drain two accumulators, all handed over through
 * mbarriers), kind::f16 for the bf16 form and kind::f8f6f4 for the FP8 form;
 * 1 = the bf16 form's MMAs with the roles in lock-step (block barriers per
 * row), the FP8 form on mma.sync; 0 = mma.sync everywhere.  The bf16 form
 * gives the same bits on every path; the FP8 form's tcgen05 and mma.sync
 * instructions add the 32 products of a K step in different orders (last-bit
 * fp32 differences).  QCA_ERR_ARG for any other value. */
int qca_net_set_tensor_path(qca_net_t net, int path);

/* Synchronise and report the device watchdog of the tensor-core kernels:
 * QCA_ERR_WATCHDOG if a wait for an MMA timed out since the last call (the
 * flag is then cleared), else QCA_OK. */
int qca_net_status(qca_net_t net);

/* Self-test of the device watchdog (no fault is involved): one thread of a
 * one-CTA kernel waits on an mbarrier that nothing completes, with the bounded
 * polling the tensor-core kernels use (about 2 s of SM clock), gives up and
 * raises the CTA's stop flag; a second warp waiting on another such barrier
 * must then give up at once.  Outputs (host pointers, each may be NULL): 1 if
 * the first / second wait gave up, the first wait's duration and the second
 * waiter's return after the first gave up, in seconds at the device's nominal
 * clock.  Synchronises the device; QCA_OK unless a CUDA call fails.  The
 * context stays usable afterwards. */
int qca_watchdog_selftest(int* first_gave_up, int* second_gave_up, double* first_wait_s,
                          double* second_lag_s);

/* Net + automaton: pre-decode, run qca_decode_batch_async on the residual
 * N xor C0 (arguments as there), then out_correction = C0 xor C_automaton.
 * out_steps counts the automaton's steps; out_logical_fail is the failure
 * flag of N xor C (the automaton's flag on the residual).  residual_scratch
 * is caller-owned device memory of 2 * shots * L^2 bytes. */
int qca_net_decode_batch_async(qca_net_t net, const uint8_t* noise, int L, int64_t shots,
                               int max_steps, uint64_t rng_seed, uint8_t* out_correction,
                               int32_t* out_steps, uint8_t* out_logical_fail,
                               const qca_config* cfg, uint8_t* residual_scratch, void* stream);

/* Kernel path chosen for a lattice size: 1 = on-chip fast sweep, 2 = on-chip
 * sweep on a 2-CTA cluster, 3 = large-lattice sweep (8-CTA cluster per shot,
 * state in global memory, bulk-copy staged bands; L a multiple of 128, chosen
 * automatically above 256), 0 = generic sweep with HBM-resident state.
 * Returns a negative code for an unsupported L. */
int qca_kernel_path(int L, const qca_config* cfg);

/* Override the kernel path for one lattice size: path -1 = automatic (the
 * default), 0 = generic sweep, 3 = large-lattice sweep (L a multiple of 128,
 * 128 <= L <= QCA_MAX_L).  Every path gives bit-identical results; the
 * override exists to compare them and to run the large-lattice kernel on
 * sizes the oracle checks quickly.  Not thread-safe against concurrent
 * decodes of the same L.  With the large-lattice path, out_logical_fail = 3
 * marks a shot whose decode a device watchdog stopped (a staged copy did not
 * complete within about two seconds); the rest of that call's outputs are
 * then unreliable. */
int qca_set_kernel_path(int L, int path);

/* Release the device workspaces the library caches (generic-kernel state and
 * host-path staging buffers) on the current device. */
int qca_free_workspace(void);

/* Microbenchmarks of the sweep's roofline denominators on the current device
 * (no counterpart in the paper: measurement only).  Four kernels, each one
 * wave of resident 512-thread CTAs on every SM for a few tens of
 * milliseconds, time one instruction written as inline PTX: min.u16x2 (the
 * sweep's byte-pair minimum), lop3.b32, min.u32, and conflict-free 16-byte
 * shared-memory loads.  Thread 0 of every CTA reads the SM clock (clock64) and
 * the global timer around its loop; the per-clock rates divide the work of
 * the CTAs resident on an SM by the median CTA's cycles, the per-second rates
 * use the launch's CUDA-event time.  Synchronises the device.  Errors:
 * QCA_ERR_ARG for NULL, QCA_ERR_CUDA. */
typedef struct qca_peaks {
  int sms;                        /* multiprocessors */
  int ctas_per_sm;                /* resident probe CTAs per SM (one wave) */
  double sm_clock_mhz;            /* median SM clock during the min.u16x2 probe */
  double min16x2_per_clk_sm;      /* min.u16x2 instructions per clock per SM (2 lanes each) */
  double lop3_per_clk_sm;         /* lop3.b32 instructions per clock per SM */
  double min_u32_per_clk_sm;      /* min.u32 instructions per clock per SM */
  double smem_bytes_per_clk_sm;   /* shared-memory load bytes per clock per SM */
  double min16x2_lane_ops_per_s;  /* 2 x min.u16x2 instructions per second, whole device */
  double smem_bytes_per_s;        /* shared-memory load bytes per second, whole device */
} qca_peaks;
int qca_probe_peaks(qca_peaks* out);

/* Static, thread-local description of the last error (never NULL). */
const char* qca_last_error(void);

/* ABI version: 100 * major + minor. */
int qca_version(void);

#ifdef __cplusplus
}
#endif
#endif /* QCA_H */
