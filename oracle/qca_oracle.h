/*
 * qca_oracle.h -- plain, slow, single-threaded CPU oracle of the synchronous
 * message-passing automaton decoder for the 2D toric code (arXiv 2506.03266).
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA library.  Only
 * the test-suite, the smoke entry point and the CPU-baseline leg of the bench
 * may load it; the product path never does.  It shares no code, header, table
 * or constant generator with the CUDA path.
 *
 * Conventions (all arrays row-major, periodic L x L torus, L >= 3):
 *   site r = (x, y), index y*L + x.
 *   edge bits: uint8 [2][L][L]; plane 0 holds e_x(r) = <r, r + x^>, plane 1
 *   holds e_y(r) = <r, r + y^>.  (Qubits live on links, Sec. 2.)
 *   sigma: int8 [L][L] with values +1 / -1 (the vertex-stabiliser eigenvalue;
 *   -1 marks an anyon, Def. "synchronous automaton decoder", Eq. adef).
 *   message fields m^{s a}: int32 [4][L][L], field order
 *     k = 0: (+,x)   k = 1: (-,x)   k = 2: (+,y)   k = 3: (-,y)
 *   with values in {0, 1, ..., m_max}; 0 means "no message" (Eq. mvals).
 *   forces f^a: int8 [2][L][L] (a = x, y), values in {-1, 0, +1}.
 */
#ifndef QCA_ORACLE_H
#define QCA_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* SplitMix64 output function (Steele, Lea & Flood, OOPSLA 2014). */
uint64_t qo_splitmix64(uint64_t z);
/* floor(p * 2^64) clamped to [0, 2^64 - 1]; an edge flips iff u < threshold. */
uint64_t qo_prob_threshold(double p);
/* i.i.d. bit-flip noise of strength p (Sec. 7): shots [shot0, shot0+shots). */
void qo_sample_errors(int L, int64_t shot0, int64_t shots, uint64_t thr, uint64_t seed,
                      uint8_t* out_edges);
/* Per-shot L and flip threshold of the mixed-size workload (see the .c file). */
void qo_uneven_draw(int64_t shots, uint64_t seed, int32_t* out_L, uint64_t* out_thr);
/* sigma_r from the parity of the four links incident to r (Def. synch_ccqs). */
void qo_syndrome(int L, const uint8_t* edges, int8_t* sigma);
/* One application of the automaton rule A^(D), D = 2 (Def. Dd_msg_passing). */
void qo_message_substep(int L, int m_max, const int8_t* sigma, const int32_t* m_in,
                        int32_t* m_out);
/* Tie orders of argmin' (Eq. degbreak) and rules for a balanced axis (see
 * readings R3 and R4 in the .c file). */
#define QO_TIE_LEX 0
#define QO_TIE_LITERAL 1
#define QO_BALANCE_STAY 0
#define QO_BALANCE_RANDOM 1
/* Forces f^a_r of Eqs. blahdef / degbreak for every anyon site (0 elsewhere),
 * default tie order. */
void qo_forces(int L, const int8_t* sigma, const int32_t* m, int8_t* f);
/* Same with a tie order; balanced (may be NULL) receives the chosen axis (1 x,
 * 2 y) at anyons whose chosen axis is balanced, else 0. */
void qo_forces_rule(int L, int tie_order, const int8_t* sigma, const int32_t* m, int8_t* f,
                    uint8_t* balanced);
/* Links flipped by the feedback operator of Eq. ddfeedback: uint8 [2][L][L]. */
void qo_feedback_links(int L, const int8_t* sigma, const int8_t* f, uint8_t* flips);
/* One decoder time step in place: v message sub-steps, forces, feedback,
 * correction update C ^= F and syndrome update sigma <- sigma * sigma_F.
 * tie_order / balance_rule select the readings of Eq. degbreak and of a
 * balanced axis (QO_TIE_*, QO_BALANCE_*; 0 / 0 are the defaults).
 * move_thr > 0 enables the optional random-move rule (Sec. 5, corollary on
 * limited memory): an anyon whose draw is below move_thr moves in a random
 * direction instead.  flips_out (may be NULL) receives the flipped links.
 * Returns the number of anyons after the step. */
int qo_step(int L, int v, int m_max, int tie_order, int balance_rule, uint64_t move_thr,
            uint64_t seed, int64_t shot, int32_t t, int8_t* sigma, int32_t* m, uint8_t* C,
            uint8_t* flips_out);
/* Cut parities of a link set R: wx = XOR_y R.e_x((0,y)), wy = XOR_x R.e_y((x,0)). */
void qo_cut_parity(int L, const uint8_t* R, int* wx, int* wy);
/* Decode one shot whose noise realisation is N (Sec. 7; Def. plogandtdec).
 * Writes the correction C, the number of feedback steps, and the failure flag
 * (0 success, 1 nontrivial homology of N xor C, 2 step budget exhausted).
 * anyon_trace (may be NULL) receives the anyon count after each step, at most
 * trace_cap entries.  Returns the flag. */
int qo_decode_shot(const uint8_t* N, int L, int v, int m_max, int tie_order, int balance_rule,
                   int max_steps, uint64_t move_thr, uint64_t seed, int64_t shot,
                   uint8_t* C, int32_t* steps, int32_t* anyon_trace, int trace_cap);
/* Same, from a pure syndrome (anyon indicator uint8 [L][L], 1 = anyon).
 * Writes C, steps, and the cut parities of C alone in cut[0] (wx) / cut[1]
 * (wy).  Returns 0 if the syndrome emptied, 2 if the budget ran out. */
int qo_decode_syndrome_shot(const uint8_t* anyon, int L, int v, int m_max, int tie_order,
                            int balance_rule, int max_steps, uint64_t move_thr, uint64_t seed,
                            int64_t shot, uint8_t* C, int32_t* steps, uint8_t* cut);
/* Loop of qo_decode_shot over shots [shot0, shot0+shots); arrays are per shot. */
void qo_decode_batch(const uint8_t* N, int L, int64_t shot0, int64_t shots, int v, int m_max,
                     int tie_order, int balance_rule, int max_steps, uint64_t move_thr,
                     uint64_t seed, uint8_t* C, int32_t* steps, uint8_t* flags);

/* ---- 1D repetition code (qca_oracle_1d.c; Sec. 3.1, Def. "message passing
 * automaton, 1D"; Sec. 7.1).  Ring of L sites, link <r, r+1> = bit r. */
void qo1_sample_errors(int L, int64_t shot0, int64_t shots, uint64_t thr, uint64_t seed,
                       uint8_t* out);
void qo1_syndrome(int L, const uint8_t* links, int8_t* sigma);
/* One application of A^(1); m is int32 [2][L] (m^+, m^-). */
void qo1_substep(int L, int m_max, const int8_t* sigma, const int32_t* m_in, int32_t* m_out);
void qo1_forces(int L, const int8_t* sigma, const int32_t* m, int8_t* f);
void qo1_feedback(int L, const int8_t* sigma, const int8_t* f, uint8_t* flips);
int qo1_step(int L, int v, int m_max, uint64_t move_thr, uint64_t seed, int64_t shot, int32_t t,
             int8_t* sigma, int32_t* m, uint8_t* C);
/* Returns the flag: 0 success (N xor C = 0), 1 N xor C = all ones, 2 budget.
 * maj_fail (may be NULL): 1 if the output value differs from majority(N). */
int qo1_decode_shot(const uint8_t* N, int L, int v, int m_max, int max_steps, uint64_t move_thr,
                    uint64_t seed, int64_t shot, uint8_t* C, int32_t* steps, uint8_t* maj_fail);

/* ---- 2D variants (qca_oracle_variants.c): open boundaries (Appendix "Open
 * boundary conditions"; readings R17 in the .c file) and uncoordinated
 * desynchronisation (Sec. 7.3; reading R16). */
int qo_open_link_exists(int L, int plane, int x, int y);
void qo_open_syndrome(int L, const uint8_t* E, int8_t* sigma);
void qo_open_substep(int L, int m_max, const int8_t* sigma, const int32_t* m_in, int32_t* m_out);
/* Returns 0 success, 1 logical error (odd crossing of the cut x = 0|1), 2 budget. */
int qo_open_decode_shot(const uint8_t* N, int L, int v, int m_max, int max_steps, uint8_t* C,
                        int32_t* steps);
/* Returns the flag as qo_decode_shot; ticks receives the ticks taken. */
int qo_desync_decode_shot(const uint8_t* N, int L, int v, int m_max, int max_ticks,
                          uint64_t thr_msg, uint64_t thr_move, uint64_t seed, int64_t shot,
                          uint8_t* C, int32_t* ticks);

#ifdef __cplusplus
}
#endif
#endif
