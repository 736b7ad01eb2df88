/*
 * qca_oracle_1d.c -- plain, slow, single-threaded CPU oracle of the 1D
 * message-passing automaton decoder for the repetition code (arXiv 2506.03266,
 * Sec. 3.1, Def. "message passing automaton, 1D"; numerics of Sec. 7.1).
 *
 * TEST INFRASTRUCTURE ONLY (see qca_oracle.h).  Shares nothing with the CUDA
 * path.
 *
 * Conventions: a ring of L >= 3 sites r = 0 .. L-1 (periodic); the qubit of
 * link <r, r+1> is bit r of the noise / correction arrays (uint8 [L]); sigma
 * int8 [L] in {+1, -1}, -1 an anyon; fields m^+ and m^- int32 [2][L] (row 0
 * m^+, row 1 m^-), values 0 .. m_max with 0 meaning "no message".
 *
 * Readings (shared with the 2D oracle where they apply):
 *   R1  in f_r = sgn(-m^+_r + m^-_r) an empty field counts as +infinity, and
 *       the feedback operator decides the direction: X on <r, r+1> when
 *       sigma_r f_r = 1 (an anyon at r with f_r = -1 moves right) or
 *       sigma_{r+1} (-f_{r+1}) = 1 (an anyon at r+1 with f = +1 moves left).
 *       This is the prose's rule: toward the only message heard, or toward
 *       the smaller of two; no move when they are equal.
 *   R2  only anyon sites move.
 *   R5  a value above m_max vanishes (becomes 0).
 *   R10 a budget of steps; flag 2 when it runs out with anyons left.
 *   R14 optional random moves (Sec. 7.1 uses 10 %): per step an anyon whose
 *       draw u = sm(sm(sm(sm(seed ^ "MOVE") ^ shot) ^ t) ^ r) is below
 *       move_thr moves right if sm(u) >> 63 is 0, else left, ignoring its
 *       messages.
 *   R15 success (Sec. 7.1): after decoding, N xor C is all zeros or all ones;
 *       the output's logical value is that bit.  The paper counts a shot as
 *       decoded when that value equals the majority vote of the input bits N;
 *       flag 1 marks output value != 0 (the encoded state) and the majority
 *       flag marks output value != majority(N), majority(N) = 1 iff more than
 *       L/2 bits of N are set.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "qca_oracle.h"

#define QO1_TAG_NOISE 0x4E4F49534531ULL /* "NOISE1" */
#define QO1_TAG_MOVE 0x4D4F5645ULL      /* "MOVE", as in 2D */

static int w1(int i, int L) {
  int r = i % L;
  return r < 0 ? r + L : r;
}

/* Noise: link r of shot s flips iff sm(sm(sm(seed ^ "NOISE1") ^ s) ^ r) < thr. */
void qo1_sample_errors(int L, int64_t shot0, int64_t shots, uint64_t thr, uint64_t seed,
                       uint8_t* out) {
  const uint64_t k = qo_splitmix64(seed ^ QO1_TAG_NOISE);
  for (int64_t s = 0; s < shots; ++s) {
    const uint64_t ks = qo_splitmix64(k ^ (uint64_t)(shot0 + s));
    for (int r = 0; r < L; ++r) out[s * L + r] = qo_splitmix64(ks ^ (uint64_t)r) < thr ? 1 : 0;
  }
}

/* sigma_r = parity of the links <r-1, r> and <r, r+1>. */
void qo1_syndrome(int L, const uint8_t* links, int8_t* sigma) {
  for (int r = 0; r < L; ++r) sigma[r] = (links[w1(r - 1, L)] ^ links[r]) ? -1 : 1;
}

/* One application of A^(1):
 *   m^+_r <- 1 if an anyon sits at r-1, else 0 if m^+_{r-1} = 0, else m^+_{r-1} + 1;
 *   m^-_r likewise from r+1; then a value above m_max vanishes. */
void qo1_substep(int L, int m_max, const int8_t* sigma, const int32_t* m_in, int32_t* m_out) {
  for (int k = 0; k < 2; ++k) {
    const int s = k == 0 ? 1 : -1; /* m^+ reads r - 1, m^- reads r + 1 */
    for (int r = 0; r < L; ++r) {
      const int u = w1(r - s, L);
      int32_t nv;
      if (sigma[u] == -1)
        nv = 1;
      else if (m_in[k * L + u] == 0)
        nv = 0;
      else
        nv = m_in[k * L + u] + 1;
      if (nv > m_max) nv = 0;
      m_out[k * L + r] = nv;
    }
  }
}

/* f_r = sgn(-m^+_r + m^-_r) at anyon sites, 0 read as +infinity (R1); 0 elsewhere. */
void qo1_forces(int L, const int8_t* sigma, const int32_t* m, int8_t* f) {
  for (int r = 0; r < L; ++r) {
    f[r] = 0;
    if (sigma[r] != -1) continue;
    const int32_t mp = m[r], mm = m[L + r];
    if (mp == 0 && mm == 0) continue;
    if (mp == 0) {
      f[r] = -1; /* sgn(-inf + m^-) */
      continue;
    }
    if (mm == 0) {
      f[r] = 1; /* sgn(-m^+ + inf) */
      continue;
    }
    const int d = -mp + mm;
    f[r] = (int8_t)((d > 0) - (d < 0));
  }
}

/* Links flipped by F^(1): <r, r+1> iff sigma_r f_r = 1 or sigma_{r+1}(-f_{r+1}) = 1,
 * with only anyon sites contributing (R2). */
void qo1_feedback(int L, const int8_t* sigma, const int8_t* f, uint8_t* flips) {
  for (int r = 0; r < L; ++r) {
    const int rn = w1(r + 1, L);
    const int t1 = sigma[r] == -1 ? sigma[r] * f[r] : 0;
    const int t2 = sigma[rn] == -1 ? sigma[rn] * (-f[rn]) : 0;
    flips[r] = (t1 == 1 || t2 == 1) ? 1 : 0;
  }
}

int qo1_step(int L, int v, int m_max, uint64_t move_thr, uint64_t seed, int64_t shot, int32_t t,
             int8_t* sigma, int32_t* m, uint8_t* C) {
  int32_t* tmp = (int32_t*)malloc(2 * (size_t)L * sizeof(int32_t));
  int8_t* f = (int8_t*)malloc((size_t)L);
  uint8_t* F = (uint8_t*)malloc((size_t)L);
  for (int i = 0; i < v; ++i) {
    qo1_substep(L, m_max, sigma, m, tmp);
    memcpy(m, tmp, 2 * (size_t)L * sizeof(int32_t));
  }
  qo1_forces(L, sigma, m, f);
  if (move_thr) {
    const uint64_t k1 = qo_splitmix64(qo_splitmix64(seed ^ QO1_TAG_MOVE) ^ (uint64_t)shot);
    const uint64_t k2 = qo_splitmix64(k1 ^ (uint64_t)(uint32_t)t);
    for (int r = 0; r < L; ++r) {
      if (sigma[r] != -1) continue;
      const uint64_t u = qo_splitmix64(k2 ^ (uint64_t)r);
      if (u >= move_thr) continue;
      /* an anyon moves right when f = -1, left when f = +1 (R1) */
      f[r] = (qo_splitmix64(u) >> 63) == 0 ? -1 : 1;
    }
  }
  qo1_feedback(L, sigma, f, F);
  int anyons = 0;
  for (int r = 0; r < L; ++r) C[r] ^= F[r];
  for (int r = 0; r < L; ++r) {
    if (F[w1(r - 1, L)] ^ F[r]) sigma[r] = (int8_t)-sigma[r];
    anyons += sigma[r] == -1;
  }
  free(F);
  free(f);
  free(tmp);
  return anyons;
}

int qo1_decode_shot(const uint8_t* N, int L, int v, int m_max, int max_steps, uint64_t move_thr,
                    uint64_t seed, int64_t shot, uint8_t* C, int32_t* steps, uint8_t* maj_fail) {
  int8_t* sigma = (int8_t*)malloc((size_t)L);
  int32_t* m = (int32_t*)calloc(2 * (size_t)L, sizeof(int32_t));
  qo1_syndrome(L, N, sigma);
  memset(C, 0, (size_t)L);
  int anyons = 0, weight = 0;
  for (int r = 0; r < L; ++r) {
    anyons += sigma[r] == -1;
    weight += N[r];
  }
  int t = 0, flag = 0;
  while (anyons > 0) {
    if (t >= max_steps) {
      flag = 2;
      break;
    }
    anyons = qo1_step(L, v, m_max, move_thr, seed, shot, t, sigma, m, C);
    ++t;
  }
  const int value = N[0] ^ C[0]; /* N xor C is constant when no anyon is left */
  const int majority = 2 * weight > L ? 1 : 0;
  if (flag == 0) flag = value;
  if (maj_fail) *maj_fail = (uint8_t)(flag == 2 ? 2 : (value != majority));
  *steps = t;
  free(m);
  free(sigma);
  return flag;
}
