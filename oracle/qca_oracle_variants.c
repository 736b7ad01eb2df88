/*
 * qca_oracle_variants.c -- plain CPU oracle of two variants of the 2D decoder
 * (arXiv 2506.03266):
 *   - open boundaries (Appendix "Open boundary conditions", Def. "message
 *     passing automaton with open boundaries");
 *   - uncoordinated desynchronisation (Sec. 7.3).
 *
 * TEST INFRASTRUCTURE ONLY (see qca_oracle.h).  Shares nothing with the CUDA
 * path; arrays and field order as in qca_oracle.c (edges uint8 [2][L][L],
 * sigma int8 +1/-1, fields int32 [4][L][L] in the order (+,x) (-,x) (+,y) (-,y)).
 *
 * Readings for the open lattice (R17):
 *   - sites r = (x, y), 0 <= x, y < L, not periodic; the rough boundary is
 *     B = {x = 0} u {x = L-1};
 *   - qubits: e_x(x, y) = <(x,y), (x+1,y)> for 0 <= x <= L-2 (every y) and
 *     e_y(x, y) = <(x,y), (x,y+1)> for 1 <= x <= L-2, 0 <= y <= L-2; entries of
 *     the [2][L][L] arrays for other links are ignored in the input and zero in
 *     the correction;
 *   - sigma lives on the interior sites (1 <= x <= L-2), the parity of their
 *     existing links; boundary sites are never anyons;
 *   - A_open: a boundary site holds no message; an interior site takes 1 when
 *     an anyon lies on C^(a)_{r - s a^} (members outside the lattice dropped)
 *     or when r - s a^ is a boundary site; 0 when r - s a^ is outside the
 *     lattice or the set holds no anyon and no message; else 1 + the smallest
 *     nonzero message of the set; values above m_max vanish;
 *   - forces and feedback as on the torus (R1-R4);
 *   - failure: after the syndrome empties, N xor C joins the two boundaries an
 *     odd number of times, read as the parity of the links e_x(0, y) over y.
 *
 * Readings for uncoordinated desynchronisation (R16): each site carries two
 * Poisson clocks, one for its message registers (rate v) and one for anyon
 * motion (rate 1), discretised into ticks of length q: per tick a site fires
 * its message update with probability min(1, v q) and, if it holds an anyon,
 * its move with probability q, from draws
 *   u = sm(sm(sm(sm(seed ^ "DESYNC") ^ shot) ^ tick) ^ (2 r + c)),
 * c = 0 for the messages and 1 for the move, fired iff u < floor(prob 2^64).
 * Within a tick the firing message updates apply together (one application
 * of A^(D) at those sites, from the fields before the tick), then the firing
 * anyons move by the forces of the updated fields (the OR feedback among
 * them), then sigma is updated.  With q = 1 and v = 1 every site fires every
 * tick and the dynamics is the synchronous decoder with v = 1.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "qca_oracle.h"

#define QOV_TAG_DESYNC 0x444553594E43ULL /* "DESYNC" */

/* ------------------------------------------------------------ open lattice */

static int in_lat(int x, int y, int L) { return x >= 0 && x < L && y >= 0 && y < L; }
static int is_bdry(int x, int L) { return x == 0 || x == L - 1; }

/* Existence of the qubits of the open lattice (R17). */
int qo_open_link_exists(int L, int plane, int x, int y) {
  if (!in_lat(x, y, L)) return 0;
  if (plane == 0) return x <= L - 2;
  return x >= 1 && x <= L - 2 && y <= L - 2;
}

void qo_open_syndrome(int L, const uint8_t* E, int8_t* sigma) {
  const size_t LL = (size_t)L * L;
  for (int y = 0; y < L; ++y)
    for (int x = 0; x < L; ++x) {
      int par = 0;
      if (!is_bdry(x, L)) {
        if (qo_open_link_exists(L, 0, x, y)) par ^= E[(size_t)y * L + x];
        if (qo_open_link_exists(L, 0, x - 1, y)) par ^= E[(size_t)y * L + x - 1];
        if (qo_open_link_exists(L, 1, x, y)) par ^= E[LL + (size_t)y * L + x];
        if (qo_open_link_exists(L, 1, x, y - 1)) par ^= E[LL + (size_t)(y - 1) * L + x];
      }
      sigma[(size_t)y * L + x] = par ? -1 : 1;
    }
}

void qo_open_substep(int L, int m_max, const int8_t* sigma, const int32_t* m_in, int32_t* m_out) {
  const size_t LL = (size_t)L * L;
  for (int k = 0; k < 4; ++k) {
    const int s = (k % 2 == 0) ? 1 : -1;
    const int ax = k < 2;
    for (int y = 0; y < L; ++y)
      for (int x = 0; x < L; ++x) {
        const size_t i = (size_t)y * L + x;
        if (is_bdry(x, L)) {
          m_out[k * LL + i] = 0;
          continue;
        }
        const int ux = ax ? x - s : x, uy = ax ? y : y - s;
        int32_t nv;
        if (!in_lat(ux, uy, L)) {
          nv = 0;
        } else if (is_bdry(ux, L) && ax) {
          nv = 1; /* the rough boundary sources messages into the bulk */
        } else {
          int anyon = 0;
          int32_t best = 0;
          for (int j = -1; j <= 1; ++j) {
            const int xx = ax ? ux : ux + j, yy = ax ? uy + j : uy;
            if (!in_lat(xx, yy, L)) continue;
            const size_t c = (size_t)yy * L + xx;
            if (sigma[c] == -1) anyon = 1;
            const int32_t val = m_in[k * LL + c];
            if (val > 0 && (best == 0 || val < best)) best = val;
          }
          nv = anyon ? 1 : (best == 0 ? 0 : best + 1);
        }
        if (nv > m_max) nv = 0;
        m_out[k * LL + i] = nv;
      }
  }
}

int qo_open_decode_shot(const uint8_t* N, int L, int v, int m_max, int max_steps, uint8_t* C,
                        int32_t* steps) {
  const size_t LL = (size_t)L * L;
  int8_t* sigma = (int8_t*)malloc(LL);
  int32_t* m = (int32_t*)calloc(4 * LL, sizeof(int32_t));
  int32_t* tmp = (int32_t*)malloc(4 * LL * sizeof(int32_t));
  int8_t* f = (int8_t*)malloc(2 * LL);
  uint8_t* F = (uint8_t*)malloc(2 * LL);
  qo_open_syndrome(L, N, sigma);
  memset(C, 0, 2 * LL);
  int anyons = 0;
  for (size_t i = 0; i < LL; ++i) anyons += sigma[i] == -1;
  int t = 0, flag = 0;
  while (anyons > 0) {
    if (t >= max_steps) {
      flag = 2;
      break;
    }
    for (int i = 0; i < v; ++i) {
      qo_open_substep(L, m_max, sigma, m, tmp);
      memcpy(m, tmp, 4 * LL * sizeof(int32_t));
    }
    qo_forces(L, sigma, m, f); /* same selection rule as the torus (R1-R4) */
    /* feedback on existing links only; a force never points off the lattice
     * (the field from outside is always empty) */
    memset(F, 0, 2 * LL);
    for (int y = 0; y < L; ++y)
      for (int x = 0; x < L; ++x)
        for (int a = 0; a < 2; ++a) {
          if (!qo_open_link_exists(L, a, x, y)) continue;
          const int xn = a == 0 ? x + 1 : x, yn = a == 0 ? y : y + 1;
          const size_t r = (size_t)y * L + x, rn = (size_t)yn * L + xn;
          const int t1 = sigma[r] == -1 ? sigma[r] * f[a * LL + r] : 0;
          const int t2 = sigma[rn] == -1 ? sigma[rn] * (-f[a * LL + rn]) : 0;
          F[a * LL + r] = (t1 == 1 || t2 == 1) ? 1 : 0;
        }
    for (size_t i = 0; i < 2 * LL; ++i) C[i] ^= F[i];
    int8_t* sF = (int8_t*)malloc(LL);
    qo_open_syndrome(L, F, sF);
    anyons = 0;
    for (size_t i = 0; i < LL; ++i) {
      sigma[i] = (int8_t)(sigma[i] * sF[i]);
      anyons += sigma[i] == -1;
    }
    free(sF);
    ++t;
  }
  if (flag == 0) {
    int par = 0;
    for (int y = 0; y < L; ++y) par ^= N[(size_t)y * L] ^ C[(size_t)y * L];  /* e_x(0, y) */
    flag = par;
  }
  *steps = t;
  free(F);
  free(f);
  free(tmp);
  free(m);
  free(sigma);
  return flag;
}

/* ------------------------------------------------------- desynchronisation */

int qo_desync_decode_shot(const uint8_t* N, int L, int v, int m_max, int max_ticks,
                          uint64_t thr_msg, uint64_t thr_move, uint64_t seed, int64_t shot,
                          uint8_t* C, int32_t* ticks) {
  (void)v; /* the message rate v enters through thr_msg = floor(min(1, v q) 2^64) */
  const size_t LL = (size_t)L * L;
  int8_t* sigma = (int8_t*)malloc(LL);
  int32_t* m = (int32_t*)calloc(4 * LL, sizeof(int32_t));
  int32_t* tmp = (int32_t*)malloc(4 * LL * sizeof(int32_t));
  int8_t* f = (int8_t*)malloc(2 * LL);
  uint8_t* F = (uint8_t*)malloc(2 * LL);
  int8_t* sF = (int8_t*)malloc(LL);
  qo_syndrome(L, N, sigma);
  memset(C, 0, 2 * LL);
  int anyons = 0;
  for (size_t i = 0; i < LL; ++i) anyons += sigma[i] == -1;
  const uint64_t k1 = qo_splitmix64(qo_splitmix64(seed ^ QOV_TAG_DESYNC) ^ (uint64_t)shot);
  int t = 0, flag = 0;
  while (anyons > 0) {
    if (t >= max_ticks) {
      flag = 2;
      break;
    }
    const uint64_t k2 = qo_splitmix64(k1 ^ (uint64_t)(uint32_t)t);
    /* message jumps: one application of A^(D) at the firing sites */
    qo_message_substep(L, m_max, sigma, m, tmp);
    for (size_t i = 0; i < LL; ++i) {
      const int fire = qo_splitmix64(k2 ^ (uint64_t)(2 * i)) < thr_msg;
      if (!fire)
        for (int k = 0; k < 4; ++k) tmp[k * LL + i] = m[k * LL + i];
    }
    memcpy(m, tmp, 4 * LL * sizeof(int32_t));
    /* move jumps of the firing anyons */
    qo_forces(L, sigma, m, f);
    for (size_t i = 0; i < LL; ++i) {
      const int fire = qo_splitmix64(k2 ^ (uint64_t)(2 * i + 1)) < thr_move;
      if (!fire) f[i] = f[LL + i] = 0;
    }
    qo_feedback_links(L, sigma, f, F);
    for (size_t i = 0; i < 2 * LL; ++i) C[i] ^= F[i];
    qo_syndrome(L, F, sF);
    anyons = 0;
    for (size_t i = 0; i < LL; ++i) {
      sigma[i] = (int8_t)(sigma[i] * sF[i]);
      anyons += sigma[i] == -1;
    }
    ++t;
  }
  if (flag == 0) {
    /* either torus cycle (R11), as in qo_decode_shot */
    uint8_t* R = (uint8_t*)malloc(2 * LL);
    for (size_t i = 0; i < 2 * LL; ++i) R[i] = N[i] ^ C[i];
    int wx, wy;
    qo_cut_parity(L, R, &wx, &wy);
    flag = (wx | wy) ? 1 : 0;
    free(R);
  }
  *ticks = t;
  free(sF);
  free(F);
  free(f);
  free(tmp);
  free(m);
  free(sigma);
  return flag;
}
