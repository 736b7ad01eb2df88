/*
 * qca_oracle.c -- plain CPU oracle of the message-passing automaton decoder of
 * arXiv 2506.03266 ("Fast offline decoding with local message-passing
 * automata"), 2D toric code, i.i.d. bit-flip noise, synchronous dynamics.
 *
 * TEST INFRASTRUCTURE ONLY (see qca_oracle.h).  Single-threaded, no blocking,
 * no fusion, no bit tricks: every function follows one definition of the paper
 * in the paper's order and notation so that it can be checked by eye.
 *
 * Readings of points where the paper is silent, ambiguous or garbled (each is
 * also listed with its justification in the design notes of the repository):
 *   R1  In the force f = sgn(-m^{+a} + m^{-a}) a field value 0 ("no message")
 *       is read as +infinity, so that an anyon that hears only m^{+a} moves
 *       along -a (Sec. 3.1 prose; Def. 1d_msg_passing operator).
 *   R2  Only anyon sites (sigma_r = -1) move; the feedback exponent is
 *       evaluated for anyon sites only (Sec. 3.1: "Consider an anyon at r").
 *   R3  argmin' of Eq. degbreak is read lexicographically: smallest m first,
 *       then the smallest s*a, i.e. the preference (-,y) > (-,x) > (+,x) > (+,y)
 *       (tie order QO_TIE_LEX, the default).  The printed offset s*a/(D+1) is
 *       kept as the option QO_TIE_LITERAL: smallest integer key 3m + s*a, and
 *       where two keys are equal (m^{-y} = k+1 against m^{+x} = k, m^{-x} = k+1
 *       against m^{+y} = k) the larger m.
 *   R4  Balanced messages on the chosen axis give f = 0 (no move), the
 *       deterministic rule (balance rule QO_BALANCE_STAY, the default).  The
 *       option QO_BALANCE_RANDOM moves such an anyon one link along +a or -a,
 *       chosen by a counter draw (footnote of Sec. 5.3 contrasts the two).
 *   R5  A message whose value would exceed m_max disappears (becomes 0).
 *   R6  C^(a)_r = the three sites r + j b^, j in {-1,0,1}, b != a.
 *   R7  "min + 1" in A^(D) runs over the nonzero neighbour values only.
 *   R8  One time step = v applications of A^(D) with sigma fixed, then the
 *       feedback, then the syndrome update.
 *   R9  A shot with no anyons takes 0 steps.
 *   R10 A shot still holding anyons after max_steps steps gets flag 2.
 *   R11 Logical failure = N xor C wraps either torus cycle (Sec. 7.2).
 */
#include "qca_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- RNG ---- */

/* Stream tags: the noise draw and the optional random-move draw use disjoint
 * key derivations.  (ASCII "NOISE" and "MOVE".) */
#define QO_TAG_NOISE 0x4E4F495345ULL
#define QO_TAG_MOVE 0x4D4F5645ULL
/* ASCII "BALANCE": draws of the balanced-axis random rule (R4 option). */
#define QO_TAG_BALANCE 0x42414C414E4345ULL

uint64_t qo_splitmix64(uint64_t z) {
  /* Steele, Lea & Flood (2014), SplitMix64: golden-gamma increment followed by
   * the variant-13 mixing function. */
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t qo_prob_threshold(double p) {
  if (!(p > 0.0)) return 0;
  if (p >= 1.0) return UINT64_MAX;
  double t = floor(ldexp(p, 64));
  if (t >= 18446744073709551615.0) return UINT64_MAX;
  return (uint64_t)t;
}

/* Edge index used for the noise key: 2 * (y*L + x) + dir. */
void qo_sample_errors(int L, int64_t shot0, int64_t shots, uint64_t thr, uint64_t seed,
                      uint8_t* out_edges) {
  const uint64_t kseed = qo_splitmix64(seed ^ QO_TAG_NOISE);
  for (int64_t s = 0; s < shots; ++s) {
    const uint64_t kshot = qo_splitmix64(kseed ^ (uint64_t)(shot0 + s));
    uint8_t* E = out_edges + (size_t)s * 2 * L * L;
    for (int y = 0; y < L; ++y)
      for (int x = 0; x < L; ++x)
        for (int dir = 0; dir < 2; ++dir) {
          uint64_t e = 2 * ((uint64_t)y * L + x) + dir;
          uint64_t u = qo_splitmix64(kshot ^ e);
          E[(size_t)dir * L * L + (size_t)y * L + x] = (u < thr) ? 1 : 0;
        }
  }
}

/* Mixed-size workload of the Monte Carlo sweeps: per-shot L in
 * {24, 48, 64, 96, 128, 192} with probabilities 30/25/20/12/8/5 per cent and
 * a flip probability uniform in [0.01, 0.07), both from counter draws. */
#define QO_TAG_SIZE 0x4C53495A45ULL
#define QO_TAG_RATE 0x5052415445ULL

void qo_uneven_draw(int64_t shots, uint64_t seed, int32_t* out_L, uint64_t* out_thr) {
  static const int sizes[6] = {24, 48, 64, 96, 128, 192};
  static const int percent_upto[6] = {30, 55, 75, 87, 95, 100};
  const uint64_t klsize = qo_splitmix64(seed ^ QO_TAG_SIZE);
  const uint64_t krate = qo_splitmix64(seed ^ QO_TAG_RATE);
  const uint64_t t_lo = qo_prob_threshold(0.01), t_span = qo_prob_threshold(0.06);
  for (int64_t s = 0; s < shots; ++s) {
    uint64_t u = qo_splitmix64(klsize ^ (uint64_t)s);
    /* class k is chosen when u < floor(percent_upto[k] / 100 * 2^64) */
    int k;
    for (k = 0; k < 5; ++k) {
      unsigned __int128 cut = ((unsigned __int128)percent_upto[k] << 64) / 100;
      if ((unsigned __int128)u < cut) break;
    }
    out_L[s] = sizes[k];
    uint64_t v = qo_splitmix64(krate ^ (uint64_t)s);
    unsigned __int128 scaled = (unsigned __int128)v * t_span;
    out_thr[s] = t_lo + (uint64_t)(scaled >> 64);
  }
}

/* ------------------------------------------------------------ lattice ---- */

static int wrap(int i, int L) {
  int r = i % L;
  return r < 0 ? r + L : r;
}
static size_t site(int x, int y, int L) { return (size_t)wrap(y, L) * L + wrap(x, L); }

/* Field k <-> (s, a): k = 0 (+,x), 1 (-,x), 2 (+,y), 3 (-,y). */
static int field_s(int k) { return (k % 2 == 0) ? +1 : -1; }
static int field_a(int k) { return (k < 2) ? 1 : 2; } /* a = 1 is x, a = 2 is y */
static int field_index(int s, int a) { return (a == 1 ? 0 : 2) + (s > 0 ? 0 : 1); }

/* Def. synch_ccqs: sigma_r is the eigenvalue of the vertex stabiliser g_r,
 * i.e. (-1)^(number of flipped links incident to r).  The links incident to
 * r = (x, y) are e_x(r), e_x(r - x^), e_y(r), e_y(r - y^). */
void qo_syndrome(int L, const uint8_t* edges, int8_t* sigma) {
  const uint8_t* ex = edges;
  const uint8_t* ey = edges + (size_t)L * L;
  for (int y = 0; y < L; ++y)
    for (int x = 0; x < L; ++x) {
      int parity = ex[site(x, y, L)] ^ ex[site(x - 1, y, L)] ^ ey[site(x, y, L)] ^
                   ey[site(x, y - 1, L)];
      sigma[site(x, y, L)] = parity ? -1 : +1;
    }
}

/* ------------------------------------------------------ automaton rule ---- */

/* The set C^(a)_{r'} (Def. Dd_msg_passing): the unit infinity-norm ball in the
 * direction normal to a, centred on r' (reading R6).  Fills 3 site indices. */
static void normal_ball(int x, int y, int a, int L, size_t out[3]) {
  for (int j = -1; j <= 1; ++j) {
    if (a == 1)
      out[j + 1] = site(x, y + j, L); /* normal to x^: vary y */
    else
      out[j + 1] = site(x + j, y, L); /* normal to y^: vary x */
  }
}

/* Def. Dd_msg_passing, rule A^(D):
 *   m^{s a}_r <- 1                        if an anyon lies in C^(a)_{r - s a^}
 *             <- 0                        if every m^{s a} in that set is 0
 *             <- min{m^{s a}} + 1         otherwise (min over nonzero, R7),
 * and a value above m_max disappears (R5).  All sites update simultaneously
 * from m_in (the previous configuration) into m_out. */
void qo_message_substep(int L, int m_max, const int8_t* sigma, const int32_t* m_in,
                        int32_t* m_out) {
  const size_t LL = (size_t)L * L;
  for (int k = 0; k < 4; ++k) {
    const int s = field_s(k), a = field_a(k);
    const int32_t* mk = m_in + k * LL;
    for (int y = 0; y < L; ++y)
      for (int x = 0; x < L; ++x) {
        /* r - s a^ */
        int ux = x - (a == 1 ? s : 0);
        int uy = y - (a == 2 ? s : 0);
        size_t C[3];
        normal_ball(ux, uy, a, L, C);
        int anyon = 0;
        int32_t best = 0; /* 0 = no nonzero value seen */
        for (int i = 0; i < 3; ++i) {
          if (sigma[C[i]] == -1) anyon = 1;
          int32_t val = mk[C[i]];
          if (val > 0 && (best == 0 || val < best)) best = val;
        }
        int32_t nv;
        if (anyon)
          nv = 1;
        else if (best == 0)
          nv = 0;
        else
          nv = best + 1;
        if (nv > m_max) nv = 0;
        m_out[k * LL + site(x, y, L)] = nv;
      }
  }
}

/* sgn(-m^{+a} + m^{-a}) with 0 read as +infinity (R1). */
static int force_sign(int32_t mplus, int32_t mminus) {
  if (mplus == 0 && mminus == 0) return 0;
  if (mplus == 0) return -1;  /* only m^{-a}: -inf + finite -> sgn < 0 */
  if (mminus == 0) return +1; /* only m^{+a}: sgn(+inf) */
  int d = -mplus + mminus;
  return (d > 0) - (d < 0);
}

/* Eqs. blahdef / degbreak:
 *   M_r = {(s, a) : m^{s a}_r > 0},
 *   (s_r, a_r) = argmin' over M_r of m^{s a}_r (tie order R3),
 *   f^a_r = delta_{a, a_r} sgn(-m^{+a}_r + m^{-a}_r).
 * Evaluated at anyon sites only (R2); f = 0 elsewhere.  balanced (may be
 * NULL) receives a_r (1 or 2) where the chosen axis is balanced (both fields
 * nonzero and equal, so f = 0 by R4), else 0. */
void qo_forces_rule(int L, int tie_order, const int8_t* sigma, const int32_t* m, int8_t* f,
                    uint8_t* balanced) {
  const size_t LL = (size_t)L * L;
  memset(f, 0, 2 * LL);
  if (balanced) memset(balanced, 0, LL);
  for (size_t r = 0; r < LL; ++r) {
    if (sigma[r] != -1) continue;
    int best_k = -1;
    for (int k = 0; k < 4; ++k) {
      int32_t val = m[k * LL + r];
      if (val <= 0) continue; /* not in M_r */
      if (best_k < 0) {
        best_k = k;
        continue;
      }
      int32_t bv = m[best_k * LL + r];
      int sa = field_s(k) * field_a(k), bsa = field_s(best_k) * field_a(best_k);
      if (tie_order == QO_TIE_LITERAL) {
        /* argmin of m + s a / (D + 1), D = 2, as the integer 3 m + s a */
        int64_t key = 3 * (int64_t)val + sa, bkey = 3 * (int64_t)bv + bsa;
        if (key < bkey || (key == bkey && val > bv)) best_k = k;
      } else {
        if (val < bv || (val == bv && sa < bsa)) best_k = k;
      }
    }
    if (best_k < 0) continue; /* M_r empty: (s_r, a_r) = (0, 0) */
    int a = field_a(best_k);
    int32_t mp = m[field_index(+1, a) * LL + r];
    int32_t mm = m[field_index(-1, a) * LL + r];
    f[(size_t)(a - 1) * LL + r] = (int8_t)force_sign(mp, mm);
    if (balanced && mp > 0 && mp == mm) balanced[r] = (uint8_t)a;
  }
}

void qo_forces(int L, const int8_t* sigma, const int32_t* m, int8_t* f) {
  qo_forces_rule(L, QO_TIE_LEX, sigma, m, f, NULL);
}

/* The OR of Def. 1d_msg_passing: 1 iff x = 1 or y = 1. */
static int or_pm(int xv, int yv) { return (xv == 1 || yv == 1) ? 1 : 0; }

/* Eq. ddfeedback: link <r, r + a^> is flipped iff
 *   sigma_r f^a_r  OR  sigma_{r+a^} (-f^a_{r+a^})  equals 1,
 * with only anyon sites contributing (R2). */
void qo_feedback_links(int L, const int8_t* sigma, const int8_t* f, uint8_t* flips) {
  const size_t LL = (size_t)L * L;
  for (int a = 1; a <= 2; ++a) {
    const int8_t* fa = f + (size_t)(a - 1) * LL;
    for (int y = 0; y < L; ++y)
      for (int x = 0; x < L; ++x) {
        size_t r = site(x, y, L);
        size_t rn = (a == 1) ? site(x + 1, y, L) : site(x, y + 1, L);
        int t1 = (sigma[r] == -1) ? sigma[r] * fa[r] : 0;
        int t2 = (sigma[rn] == -1) ? sigma[rn] * (-fa[rn]) : 0;
        flips[(size_t)(a - 1) * LL + r] = (uint8_t)or_pm(t1, t2);
      }
  }
}

/* Balance rule QO_BALANCE_RANDOM (R4 option): an anyon whose chosen axis a
 * is balanced moves one link along +a if the top bit of its draw
 * u = sm(sm(sm(sm(seed ^ BALANCE) ^ shot) ^ t) ^ r) is 0, along -a if it is 1. */
static void balanced_moves(int L, uint64_t seed, int64_t shot, int32_t t, const uint8_t* balanced,
                           int8_t* f) {
  const size_t LL = (size_t)L * L;
  const uint64_t k1 = qo_splitmix64(qo_splitmix64(seed ^ QO_TAG_BALANCE) ^ (uint64_t)shot);
  const uint64_t k2 = qo_splitmix64(k1 ^ (uint64_t)(uint32_t)t);
  for (size_t r = 0; r < LL; ++r) {
    if (!balanced[r]) continue;
    uint64_t u = qo_splitmix64(k2 ^ (uint64_t)r);
    /* an anyon moves +a^ when f^a = -1 and -a^ when f^a = +1 */
    f[(size_t)(balanced[r] - 1) * LL + r] = (int8_t)((u >> 63) ? +1 : -1);
  }
}

/* Optional random-move rule: an anyon whose key falls below move_thr is given
 * a force that moves it one link in a uniformly drawn direction. */
static void random_moves(int L, uint64_t move_thr, uint64_t seed, int64_t shot, int32_t t,
                         const int8_t* sigma, int8_t* f) {
  if (move_thr == 0) return;
  const size_t LL = (size_t)L * L;
  const uint64_t k1 = qo_splitmix64(qo_splitmix64(seed ^ QO_TAG_MOVE) ^ (uint64_t)shot);
  const uint64_t k2 = qo_splitmix64(k1 ^ (uint64_t)(uint32_t)t);
  for (size_t r = 0; r < LL; ++r) {
    if (sigma[r] != -1) continue;
    uint64_t u = qo_splitmix64(k2 ^ (uint64_t)r);
    if (u >= move_thr) continue;
    int dir = (int)(qo_splitmix64(u) >> 62); /* 0:+x 1:-x 2:+y 3:-y */
    f[r] = 0;
    f[LL + r] = 0;
    /* an anyon (sigma = -1) moves +a^ when f^a = -1 and -a^ when f^a = +1 */
    int8_t val = (dir % 2 == 0) ? -1 : +1;
    f[(size_t)(dir / 2) * LL + r] = val;
  }
}

int qo_step(int L, int v, int m_max, int tie_order, int balance_rule, uint64_t move_thr,
            uint64_t seed, int64_t shot, int32_t t, int8_t* sigma, int32_t* m, uint8_t* C,
            uint8_t* flips_out) {
  const size_t LL = (size_t)L * L;
  int32_t* tmp = (int32_t*)malloc(4 * LL * sizeof(int32_t));
  int8_t* f = (int8_t*)malloc(2 * LL);
  uint8_t* F = (uint8_t*)malloc(2 * LL);
  uint8_t* bal = (uint8_t*)malloc(LL);
  /* 1. A^(v,D) = (A^(D))^v with sigma held fixed. */
  for (int i = 0; i < v; ++i) {
    qo_message_substep(L, m_max, sigma, m, tmp);
    memcpy(m, tmp, 4 * LL * sizeof(int32_t));
  }
  /* 2. feedback F(m, sigma) */
  qo_forces_rule(L, tie_order, sigma, m, f, bal);
  if (balance_rule == QO_BALANCE_RANDOM) balanced_moves(L, seed, shot, t, bal, f);
  random_moves(L, move_thr, seed, shot, t, sigma, f);
  qo_feedback_links(L, sigma, f, F);
  /* 3. apply: C <- C xor F, sigma <- sigma * sigma_F */
  for (size_t i = 0; i < 2 * LL; ++i) C[i] ^= F[i];
  int8_t* sigF = (int8_t*)malloc(LL);
  qo_syndrome(L, F, sigF);
  int anyons = 0;
  for (size_t r = 0; r < LL; ++r) {
    sigma[r] = (int8_t)(sigma[r] * sigF[r]);
    anyons += (sigma[r] == -1);
  }
  if (flips_out) memcpy(flips_out, F, 2 * LL);
  free(sigF);
  free(bal);
  free(F);
  free(f);
  free(tmp);
  return anyons;
}

void qo_cut_parity(int L, const uint8_t* R, int* wx, int* wy) {
  const size_t LL = (size_t)L * L;
  int px = 0, py = 0;
  for (int y = 0; y < L; ++y) px ^= R[site(0, y, L)];      /* e_x((0, y)) */
  for (int x = 0; x < L; ++x) py ^= R[LL + site(x, 0, L)]; /* e_y((x, 0)) */
  *wx = px;
  *wy = py;
}

static int run_decoder(int8_t* sigma, int L, int v, int m_max, int tie_order, int balance_rule,
                       int max_steps, uint64_t move_thr, uint64_t seed, int64_t shot, uint8_t* C,
                       int32_t* steps, int32_t* anyon_trace, int trace_cap) {
  const size_t LL = (size_t)L * L;
  int32_t* m = (int32_t*)calloc(4 * LL, sizeof(int32_t)); /* m_0 = 0 everywhere */
  memset(C, 0, 2 * LL);
  int anyons = 0;
  for (size_t r = 0; r < LL; ++r) anyons += (sigma[r] == -1);
  int t = 0;
  int flag = 0;
  while (anyons > 0) {
    if (t >= max_steps) {
      flag = 2;
      break;
    }
    anyons = qo_step(L, v, m_max, tie_order, balance_rule, move_thr, seed, shot, t, sigma, m, C,
                     NULL);
    if (anyon_trace && t < trace_cap) anyon_trace[t] = anyons;
    ++t;
  }
  *steps = t;
  free(m);
  return flag;
}

int qo_decode_shot(const uint8_t* N, int L, int v, int m_max, int tie_order, int balance_rule,
                   int max_steps, uint64_t move_thr, uint64_t seed, int64_t shot, uint8_t* C,
                   int32_t* steps, int32_t* anyon_trace, int trace_cap) {
  const size_t LL = (size_t)L * L;
  int8_t* sigma = (int8_t*)malloc(LL);
  qo_syndrome(L, N, sigma);
  int flag = run_decoder(sigma, L, v, m_max, tie_order, balance_rule, max_steps, move_thr, seed,
                         shot, C, steps, anyon_trace, trace_cap);
  free(sigma);
  if (flag == 2) return 2;
  /* Def. plogandtdec / Sec. 7.2: failure iff N xor C wraps a torus cycle. */
  uint8_t* R = (uint8_t*)malloc(2 * LL);
  for (size_t i = 0; i < 2 * LL; ++i) R[i] = N[i] ^ C[i];
  int wx, wy;
  qo_cut_parity(L, R, &wx, &wy);
  free(R);
  return (wx || wy) ? 1 : 0;
}

int qo_decode_syndrome_shot(const uint8_t* anyon, int L, int v, int m_max, int tie_order,
                            int balance_rule, int max_steps, uint64_t move_thr, uint64_t seed,
                            int64_t shot, uint8_t* C, int32_t* steps, uint8_t* cut) {
  const size_t LL = (size_t)L * L;
  int8_t* sigma = (int8_t*)malloc(LL);
  for (size_t r = 0; r < LL; ++r) sigma[r] = anyon[r] ? -1 : +1;
  int flag = run_decoder(sigma, L, v, m_max, tie_order, balance_rule, max_steps, move_thr, seed,
                         shot, C, steps, NULL, 0);
  free(sigma);
  int wx, wy;
  qo_cut_parity(L, C, &wx, &wy);
  cut[0] = (uint8_t)wx;
  cut[1] = (uint8_t)wy;
  return flag;
}

void qo_decode_batch(const uint8_t* N, int L, int64_t shot0, int64_t shots, int v, int m_max,
                     int tie_order, int balance_rule, int max_steps, uint64_t move_thr,
                     uint64_t seed, uint8_t* C, int32_t* steps, uint8_t* flags) {
  const size_t E = 2 * (size_t)L * L;
  for (int64_t s = 0; s < shots; ++s) {
    int fl = qo_decode_shot(N + s * E, L, v, m_max, tie_order, balance_rule, max_steps, move_thr,
                            seed, shot0 + s, C + s * E, steps + s, NULL, 0);
    flags[s] = (uint8_t)fl;
  }
}
