// On-chip synchronous sweep for v = 3 and L a multiple of 4 (L <= 128, one CTA
// per shot) or of 8 (128 < L <= 256, a two-CTA cluster per shot).
//
// State per shot, resident in shared memory for the whole decode:
//   * four message planes of bytes, one per field (+x, -x, +y, -y).  Each plane
//     is stored in its own frame so that its messages always travel along the
//     byte (column) axis: the x fields as [y][x], the y fields as [x][y].
//     Values use an offset encoding w = m - 1 + (255 - m_max), with 0xFF for
//     "no message" (m = 0).  Then "min over nonzero neighbours", "+1" and
//     "a value above m_max disappears" become a plain unsigned min and an add
//     that saturates at 0xFF.
//   * site bitmaps with rows padded to a power-of-two number of 32-bit words:
//     sigma (the whole lattice in every CTA), two flipped-link maps (x and y
//     links; the pair alternates with the step parity so the next step can
//     clear one while the other is read), the correction (own rows); and a
//     compacted list of the current anyons ((y << 8) | x).
//
// One decoder step (Def. "synchronous automaton decoder"):
//   1. message update, the v = 3 applications of A^(D) (Def. Dd_msg_passing)
//      fused exactly into one pass: with sigma fixed, three sub-steps give
//        w3(r) = min( [anyon on the cone section at distance d] ? off + d - 1
//                     for d = 1, 2, 3,
//                     satadd( min_{|j| <= 3} w0(r - 3 a^ + j b^), 3 ) ),
//      i.e. a width-7 transverse window at longitudinal distance 3 (dense,
//      in place with a rolling register window), then the anyon terms: dense
//      from dilated sigma rows on the first step and whenever anyons are
//      many, else per anyon (each anyon writes its light-cone sections,
//      largest value first).  The unsigned byte min runs on the native 16x2
//      integer min, each site in the high byte of a 16-bit lane.
//   2. forces and feedback (Eqs. blahdef, degbreak, ddfeedback) for the listed
//      anyons: each ORs the bit of the link it crosses into the flipped-link
//      map of every CTA of the cluster, so a link crossed from both ends flips
//      once (the OR of the feedback rule).
//   3. a dense pass over the own rows: sigma <- sigma xor (syndrome of the
//      flipped links), correction ^= flipped links, the next anyon list, and
//      the early exit when sigma is empty; budget check.
// The homology check and the byte outputs follow the last step.
//
// Two-CTA clusters (L > 128) split every plane by rows; each CTA keeps the full
// sigma, writes the cone sections that fall in its rows, moves the anyons of its
// rows, and reaches the partner's planes and bitmaps through distributed shared
// memory.  Two cluster barriers per step.  With a work counter (uneven
// batches) the clusters take shots from it until it runs past the batch; rank
// 0 fetches, the cluster reads the value over DSMEM between two barriers, and a
// final barrier keeps every CTA's shared memory alive until its partner's last
// remote access is done.
#include <cooperative_groups.h>

#include <algorithm>
#include <mutex>
#include <type_traits>
#include <vector>

#include "qca_internal.cuh"

namespace cg = cooperative_groups;

namespace qca {

namespace {

constexpr int kListCap = 16384;  // anyon-list entries (at most)

// Periodic-orbit fast-forward.  With the deterministic rules (no random moves,
// a balanced axis stays) the step is a function of sigma and the planes, and
// the planes after a step's message update are a function of the last
// kOrbitWindow syndromes alone: a message grows by 3 per step from at most
// off + 2 and is gone (0xFF) after ceil(255 / 3) = 85 steps.  So if the anyon
// set of the last kOrbitWindow + 1 steps repeats that of the steps P earlier,
// the whole state repeats with period P, the shot never ends, and the budget's
// outcome is known: sigma and the planes at max_steps equal those P-periodic
// images, and the correction, which gains the same flips every period, repeats
// with period 2P.  A shot in such an orbit stops at the first step congruent
// to max_steps modulo 2P and reports max_steps and flag 2 with that
// correction, as if it had run to the budget.  The anyon sets of the steps of
// the current run of steps with at most kOrbitAnyons anyons are kept as sorted
// 16-bit sites in a ring of 64-bit entries; steps with more anyons cost nothing.
constexpr int kOrbitWindow = 88;
constexpr int kOrbitAnyons = 4;
// ring entries: periods up to kOrbitRing - 1 - kOrbitWindow = 935 steps are
// found (the orbits seen at L = 24 to 192 repeat after 1 step, or L to 15 L
// steps for pairs chasing around the torus)
constexpr int kOrbitRing = 1024;

struct FastGeom {
  int L;
  int rows_local;       // plane rows held by one CTA (L / CL)
  int G;                // lanes per row segment (L / 4 / KW)
  int spw;              // row segments per warp
  int H;                // band height (rows per segment)
  int bands;            // bands per plane per CTA
  int segments;         // 4 * bands
  int lws;              // log2 of the 32-bit words per bitmap row
  int nws;              // words of one site bitmap (L << lws)
  int off;              // 255 - m_max
  int cap;              // anyon-list capacity
  int sparse_max;       // most anyons for which the per-anyon scatter beats the dense pass
  int ls;               // plane row stride in bytes (L + 4 or L + 8), so that a column
                        // of a plane does not fall into one shared-memory bank
  size_t plane_bytes;   // 4 * rows_local * ls
};

template <int CL>
struct Cluster {
  template <class T>
  __device__ static __forceinline__ T* at(T* p, int r) {
    if constexpr (CL == 1) {
      return p;
    } else {
      return cg::this_cluster().map_shared_rank(p, (unsigned)r);
    }
  }
  __device__ static __forceinline__ void sync() {
    if constexpr (CL == 1) {
      __syncthreads();
    } else {
      cg::this_cluster().sync();
    }
  }
  __device__ static __forceinline__ int rank() {
    if constexpr (CL == 1) {
      return 0;
    } else {
      return (int)cg::this_cluster().block_rank();
    }
  }
};

// The threads that decode one shot: the whole CTA (barrier 0, the plain block
// barrier) or a slice of it (threads [base, base + nt) with named barrier
// `bar`), so that one CTA can decode several small lattices at once.
struct Grp {
  int tid;  // thread index within the group
  int nt;   // threads in the group (a multiple of 32)
  int bar;  // 0: the whole CTA; else a named barrier id (1..15)
  __device__ __forceinline__ void sync() const {
    if (bar == 0) {
      __syncthreads();
    } else {
      asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nt) : "memory");
    }
  }
  // barrier with the OR of p over the group
  __device__ __forceinline__ int sync_or(int p) const {
    if (bar == 0) return __syncthreads_or(p);
    int r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.s32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n"
        " selp.s32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"(p), "r"(bar), "r"(nt)
        : "memory");
    return r;
  }
};

__device__ __forceinline__ uint32_t vmin2(uint32_t a, uint32_t b) { return __vminu2(a, b); }

// Rolling width-7 window over rows for one 16-bit-lane chain:
//   p2(i) = min(a(i), a(i+1)), p4(i) = min(p2(i), p2(i+2)),
//   t7(i) = min(p4(i-3), p4(i)) = min of a(i-3 .. i+3).
struct Chain {
  uint32_t a2;                  // a(i+2)
  uint32_t q0, q1, q2;          // p2(i), p2(i+1), p2(i+2) (q2 set by step)
  uint32_t r0, r1, r2;          // p4(i-3), p4(i-2), p4(i-1)
  __device__ __forceinline__ void init(const uint32_t a[6]) {
    // a[k] = a(k - 3), k = 0..5
    const uint32_t pm3 = vmin2(a[0], a[1]), pm2 = vmin2(a[1], a[2]), pm1 = vmin2(a[2], a[3]);
    const uint32_t p0 = vmin2(a[3], a[4]), p1 = vmin2(a[4], a[5]);
    r0 = vmin2(pm3, pm1);
    r1 = vmin2(pm2, p0);
    r2 = vmin2(pm1, p1);
    q0 = p0;
    q1 = p1;
    a2 = a[5];
  }
  // consume a(i+3); return t7(i)
  __device__ __forceinline__ uint32_t step(uint32_t a3) {
    q2 = vmin2(a2, a3);
    const uint32_t p4 = vmin2(q0, q2);
    const uint32_t t7 = vmin2(r0, p4);
    a2 = a3;
    q0 = q1;
    q1 = q2;
    r0 = r1;
    r1 = r2;
    r2 = p4;
    return t7;
  }
};

// High bytes of the 16-bit lanes carry the sites: the H chain holds bytes 1
// and 3 of a natural word, the L chain (word << 8) holds bytes 0 and 2.
__device__ __forceinline__ uint32_t finish_word(uint32_t tL, uint32_t tH) {
  // satadd(.,3) on the high bytes: clamp at 0xFC, then +3 (no carry leaves a lane)
  tL = vmin2(tL, 0xFCFFFCFFu) + 0x03000300u;
  tH = vmin2(tH, 0xFCFFFCFFu) + 0x03000300u;
  return __byte_perm(tL, tH, 0x7351);  // [L.b1, H.b1, L.b3, H.b3] = sites 0..3
}

__device__ __forceinline__ int wrapi(int i, int L) { return i < 0 ? i + L : (i >= L ? i - L : i); }

template <int CL>
__device__ __forceinline__ uint8_t* plane_ptr(uint8_t* planes, const FastGeom& g, int p, int R,
                                              int c) {
  const int owner = (CL == 1) ? 0 : (CL == 2 ? (R >= g.rows_local ? 1 : 0) : R / g.rows_local);
  const int lr = R - owner * g.rows_local;
  return Cluster<CL>::at(planes, owner) + ((size_t)(p * g.rows_local + lr)) * g.ls + c;
}

// 4 bytes that are each 0 or 1 -> 4 bits (byte k -> bit k).
__device__ __forceinline__ uint32_t nibble_of(uint32_t w) { return (w * 0x01020408u) >> 24; }
// 4 bytes -> 4 bits "byte is nonzero".
__device__ __forceinline__ uint32_t nonzero_nibble(uint32_t w) {
  const uint32_t nz = (((w & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | w) & 0x80808080u;
  return nibble_of(nz >> 7);
}

// Rebuild the anyon list from sigma; returns "any anyon" (block-uniform).
__device__ __forceinline__ int build_list(const uint32_t* sig, const FastGeom& g, uint16_t* list,
                                          int* count, const Grp& G) {
  // thread t owns words t, t + nt, ... (a warp's accesses hit distinct banks):
  // one scan and one atomic per warp
  const int tid = G.tid, nt = G.nt, lane = tid & 31;
  const int wsm = (1 << g.lws) - 1;
  int n = 0;
  for (int w = tid; w < g.nws; w += nt) n += __popc(sig[w]);
  int incl = n;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  int wbase = 0;
  if (lane == 31 && total) wbase = atomicAdd(count, total);
  wbase = __shfl_sync(0xffffffffu, wbase, 31);
  int pos = wbase + incl - n;
  for (int w = tid; w < g.nws; w += nt) {
    uint32_t b = sig[w];
    const int y = w >> g.lws, xb = (w & wsm) << 5;
    while (b) {
      const int k = __ffs(b) - 1;
      b &= b - 1;
      if (pos < g.cap) list[pos] = (uint16_t)((y << 8) | (xb + k));
      ++pos;
    }
  }
  return G.sync_or(n);
}

// Feedback applied densely, 32 sites per word: sigma <- sigma * sigma_F with
// F the flipped links (bit of e_x(r) / e_y(r) at site r); a site's parity
// toggles once per flipped incident link e_x(r), e_x(r - x^), e_y(r),
// e_y(r - y^).  The CTA's rows of the correction take F as well.  Every CTA
// holds the whole flipped-link map.  Then the anyon list is rebuilt from the
// new sigma; returns "any anyon" (block-uniform).
template <int kMaxPer>
__device__ __forceinline__ int apply_flips(uint32_t* sig, const uint32_t* flip, uint32_t* Cb,
                                           const FastGeom& g, uint16_t* list, int* count,
                                           int row_lo, int row_hi, const Grp& G) {
  const int tid = G.tid, nt = G.nt, lane = tid & 31, L = g.L;
  const int wsm = (1 << g.lws) - 1;
  const int last_w = (L - 1) >> 5, last_b = (L - 1) & 31;
  // thread t owns words t, t + nt, ... (a warp's accesses hit distinct banks),
  // handled as independent chains (unrolled for up to kMaxPer words, the most
  // the configuration gives a thread)
  uint32_t snew[kMaxPer];
  int n = 0;
#pragma unroll
  for (int k = 0; k < kMaxPer; ++k) {
    const int w = tid + k * nt;
    snew[k] = 0;
    if (w >= g.nws) continue;
    const int y = w >> g.lws, j = w & wsm, x0 = j << 5;
    if (x0 >= L) continue;  // padding word
    const int ym = (y == 0) ? L - 1 : y - 1;
    const uint32_t fx = flip[w], fy = flip[g.nws + w];
    const uint32_t fyu = flip[g.nws + (ym << g.lws) + j];
    // e_x(r - x^) for bit x: bit x - 1 of this row (wrapping to x = L - 1)
    const uint32_t carry = (j > 0) ? (flip[w - 1] >> 31)
                                   : ((flip[(y << g.lws) + last_w] >> last_b) & 1u);
    const uint32_t fxl = (fx << 1) | carry;
    const uint32_t valid = (L - x0 >= 32) ? 0xFFFFFFFFu : ((1u << (L - x0)) - 1u);
    const uint32_t s = sig[w] ^ ((fx ^ fxl ^ fy ^ fyu) & valid);
    sig[w] = s;
    snew[k] = s;
    n += __popc(s);
    if (y >= row_lo && y < row_hi) {
      // the correction of this CTA's rows: [x-links, y-links][local row][word]
      const int lw = ((y - row_lo) << g.lws) + j;
      Cb[lw] ^= fx;
      Cb[(g.rows_local << g.lws) + lw] ^= fy;
    }
  }
  // new anyon list (same layout as build_list)
  int incl = n;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  int wbase = 0;
  if (lane == 31 && total) wbase = atomicAdd(count, total);
  wbase = __shfl_sync(0xffffffffu, wbase, 31);
  int pos = wbase + incl - n;
#pragma unroll
  for (int k = 0; k < kMaxPer; ++k) {
    const int w = tid + k * nt;
    uint32_t b = snew[k];
    const int y = w >> g.lws, xb = (w & wsm) << 5;
    while (b) {
      const int q = __ffs(b) - 1;
      b &= b - 1;
      if (pos < g.cap) list[pos] = (uint16_t)((y << 8) | (xb + q));
      ++pos;
    }
  }
  return G.sync_or(n);
}

// Calls f(x, y) for every anyon of the current sigma, from the list when it
// held them all, else straight from the bitmap.
template <class F>
__device__ __forceinline__ void for_each_anyon(const uint16_t* list, int count, const uint32_t* sig,
                                               const FastGeom& g, const Grp& G, F&& f) {
  const int tid = G.tid, nt = G.nt;
  if (count <= g.cap) {
    // The list is sorted by site; give the 32 lanes of a warp entries far apart
    // (list index = lane-major transpose) so that their accesses spread over banks.
    const int stride = (count + 31) >> 5;
    for (int i = tid; i < 32 * stride; i += nt) {
      const int idx = (i & 31) * stride + (i >> 5);
      if (idx >= count) continue;
      const int e = list[idx];
      f(e & 0xFF, e >> 8);
    }
  } else {
    const int wsm = (1 << g.lws) - 1;
    for (int w = tid; w < g.nws; w += nt) {
      uint32_t b = sig[w];
      const int y = w >> g.lws, xb = (w & wsm) << 5;
      while (b) {
        const int k = __ffs(b) - 1;
        b &= b - 1;
        f(xb + k, y);
      }
    }
  }
}

// n (<= 32) bits of bitmap row r starting at column c (c + n <= L).
__device__ __forceinline__ uint32_t row_bits(const uint32_t* bm, const FastGeom& g, int r, int c,
                                             int n) {
  const uint32_t* row = bm + (r << g.lws);
  const int w = c >> 5, s = c & 31;
  const uint32_t lo = row[w];
  const uint32_t hi = (w + 1 < (1 << g.lws)) ? row[w + 1] : 0u;
  const uint32_t v = __funnelshift_r(lo, hi, s);
  return n >= 32 ? v : (v & ((1u << n) - 1u));
}

// Bits of columns start, start+1, ..., start+n-1 (mod L) of bitmap row r, n <= 32.
__device__ __forceinline__ uint32_t row_window(const uint32_t* bm, const FastGeom& g, int r,
                                               int start, int n) {
  const int L = g.L;
  const int s = start < 0 ? start + L : start;
  const int n1 = min(n, L - s);
  uint32_t v = row_bits(bm, g, r, s, n1);
  if (n1 < n) v |= row_bits(bm, g, r, 0, n - n1) << n1;
  return v;
}

// KW consecutive 32-bit words of a plane row: one 32- or 64-bit access (the
// 64-bit form keeps a warp's row access free of bank conflicts).
template <int KW>
__device__ __forceinline__ void load_words(const uint8_t* p, uint32_t (&w)[KW]) {
  if constexpr (KW == 2) {
    const uint2 v = *reinterpret_cast<const uint2*>(p);
    w[0] = v.x;
    w[1] = v.y;
  } else {
    w[0] = *reinterpret_cast<const uint32_t*>(p);
  }
}
template <int KW>
__device__ __forceinline__ void store_words(uint8_t* p, const uint32_t (&w)[KW]) {
  if constexpr (KW == 2) {
    *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]);
  } else {
    *reinterpret_cast<uint32_t*>(p) = w[0];
  }
}

// Anyon terms of the fused message update computed densely for every site of
// this thread's band: w(r) = off + d - 1 for the smallest d in {1, 2, 3} with an
// anyon on the cone section at distance d.  The section at distance d of a site
// at longitudinal position l is the transverse run of 2d + 1 sites at l -+ d, so
// with V_d = OR of the sigma rows t-d .. t+d (in the plane's frame) the term is
// bit l -+ d of V_d; 32 sites per bitmap operation.
// MERGE = false: the planes were empty (first step), the result is stored as is.
// MERGE = true: the planes hold the propagated values of this step, which are
// all above any anyon term, so the term replaces the value where it exists.
// sT (nws words) receives the transposed sigma.  Ends with a block barrier.
template <int KW, bool MERGE>
__device__ void dense_terms(const uint32_t* sig, const uint16_t* list, int count, uint32_t* sT,
                            const FastGeom& g, uint8_t* planes, int pl, int lrow0, int R0,
                            bool plus, int cword, bool lane_on, const Grp& G, bool yframe,
                            bool build_sT) {
  const int tid = G.tid, nt = G.nt, L = g.L;
  if (build_sT) {
    // transposed sigma: bit (row x, column y), the frame of the y planes
    for (int i = tid; i < g.nws; i += nt) sT[i] = 0;
    G.sync();
    for_each_anyon(list, count, sig, g, G, [&](int x, int y) {
      atomicOr(&sT[(x << g.lws) + (y >> 5)], 1u << (y & 31));
    });
    G.sync();
  }
  if (lane_on) {
    const uint32_t* bm = yframe ? sT : sig;
    const uint32_t off2 = (uint32_t)(g.off + 2) * 0x01010101u;
    // the lane's KW plane words cover sites 4c .. 4c + 4KW - 1 of a row; window
    // bit i <-> column 4c - 3 + i, i in [0, 4KW + 6)
    const int c = cword;
    constexpr int NB = 4 * KW + 6;
    auto ext = [&](int i) -> uint32_t {
      int R = R0 + i;
      R = R < 0 ? R + L : (R >= L ? R - L : R);
      return row_window(bm, g, R, 4 * c - 3, NB);
    };
    uint32_t e0 = ext(-3), e1 = ext(-2), e2 = ext(-1), e3 = ext(0), e4 = ext(1), e5 = ext(2);
    uint8_t* dst = planes + ((size_t)(pl * g.rows_local + lrow0)) * g.ls + 4 * c;
    for (int i = 0; i < g.H; ++i) {
      const uint32_t e6 = ext(i + 3);  // window rows i-3 .. i+3 = e0 .. e6
      const uint32_t v1 = e2 | e3 | e4;
      const uint32_t v2 = v1 | e1 | e5;
      const uint32_t v3 = v2 | e0 | e6;
      uint32_t val[KW], old[KW];
      if (MERGE) load_words<KW>(dst + (size_t)i * g.ls, old);
#pragma unroll
      for (int q = 0; q < KW; ++q) {
        uint32_t a1, a2, a3;
        if (plus) {  // term at site l comes from column l - d
          a1 = (v1 >> (2 + 4 * q)) & 0xFu;
          a2 = (v2 >> (1 + 4 * q)) & 0xFu;
          a3 = (v3 >> (4 * q)) & 0xFu;
        } else {     // from column l + d
          a1 = (v1 >> (4 + 4 * q)) & 0xFu;
          a2 = (v2 >> (5 + 4 * q)) & 0xFu;
          a3 = (v3 >> (6 + 4 * q)) & 0xFu;
        }
        // bit k -> byte k (0 / 1)
        const uint32_t b1 = (a1 * 0x00204081u) & 0x01010101u;
        const uint32_t b12 = ((a1 | a2) * 0x00204081u) & 0x01010101u;
        const uint32_t m = (((a1 | a2 | a3) * 0x00204081u) & 0x01010101u) * 0xFFu;
        // off + d - 1 = (off + 2) - [d = 1] - [d <= 2]
        val[q] = off2 - b1 - b12;
        val[q] = MERGE ? ((val[q] & m) | (old[q] & ~m)) : (val[q] | ~m);
      }
      store_words<KW>(dst + (size_t)i * g.ls, val);
      e0 = e1;
      e1 = e2;
      e2 = e3;
      e3 = e4;
      e4 = e5;
      e5 = e6;
    }
  }
  G.sync();
}

// Most bitmap words a thread handles in the dense feedback pass: geometries
// are accepted only within it (make_geom).
template <int CL, int KW>
constexpr int kWordsPerThread = CL == 1 ? (KW == 2 ? 4 : 2) : (CL == 2 ? 4 : 8);

// One step of the orbit watch, run by the 32 lanes of one warp at the start of
// a step t with at most kOrbitAnyons anyons (sigma and the list are those of
// step t; every step since `from` had that few): records the step's anyon set
// in the ring and looks for the smallest period P whose last kOrbitWindow + 1
// anyon sets, all since `from`, repeat.  Returns the step at which the shot can
// stop with the budget's outcome, or -1.
__device__ __forceinline__ int orbit_watch(uint64_t* ring, const uint16_t* list, int count, int t,
                                           int from, int max_steps, int lane) {
  constexpr int ring_mask = kOrbitRing - 1;
  uint64_t e;
  {
    uint32_t q[kOrbitAnyons];
#pragma unroll
    for (int k = 0; k < kOrbitAnyons; ++k) q[k] = k < count ? list[k] : 0xFFFFu;
    // sorting network for four keys
    auto cs = [](uint32_t& u, uint32_t& v) {
      const uint32_t lo = min(u, v), hi = max(u, v);
      u = lo;
      v = hi;
    };
    cs(q[0], q[1]);
    cs(q[2], q[3]);
    cs(q[0], q[2]);
    cs(q[1], q[3]);
    cs(q[1], q[2]);
    e = (uint64_t)q[0] | ((uint64_t)q[1] << 16) | ((uint64_t)q[2] << 32) | ((uint64_t)q[3] << 48);
  }
  if (lane == 0) ring[t & ring_mask] = e;
  // P <= t - kOrbitWindow - from keeps every compared step in the run;
  // P + kOrbitWindow <= ring_mask keeps them in the ring and off this step's
  // entry
  const int pmax = min(t - kOrbitWindow - from, ring_mask - kOrbitWindow);
  if (pmax < 1) return -1;
  int best = 0x7fffffff;
  for (int P = 1 + lane; P <= pmax; P += 32) {
    if (ring[(t - P) & ring_mask] != e) continue;
    bool ok = true;
    for (int j = 1; j <= kOrbitWindow && ok; ++j)
      ok = ring[(t - j) & ring_mask] == ring[(t - P - j) & ring_mask];
    if (ok) {
      best = P;
      break;  // this lane's candidates increase
    }
  }
  best = __reduce_min_sync(0xffffffffu, best);
  if (best == 0x7fffffff) return -1;
  // the remaining R = max_steps - t steps are n whole periods and r steps;
  // the correction repeats with period 2P
  const int R = max_steps - t, n = R / best, r = R - n * best;
  int stop = t + r + ((n & 1) ? best : 0);
  if (stop == t) stop = t + 2 * best;  // R = n P with n even and >= 2
  return stop;
}

// Decodes one shot with the group G (the whole CTA or a slice of it, CL = 1;
// or the CTAs of a 2-CTA cluster, each with its whole block, CL = 2) on the
// shared-memory state at `smem` laid out for geometry g.  Every thread of the
// group (and of the cluster) calls it with the same shot.
template <int CL, int KW>
__device__ __forceinline__ void decode_shot(const DecodeArgs& a, const FastGeom& g, uint8_t* smem,
                                            int64_t shot, const Grp& G) {
  const int L = g.L;
  const int LL = L * L;
  const int rank = Cluster<CL>::rank();
  uint8_t* planes = smem;
  uint32_t* const bits_base = reinterpret_cast<uint32_t*>(smem + g.plane_bytes);
  uint32_t* const sig_cur = bits_base;            // sigma (the full lattice in every CTA)
  uint32_t* const flipb = bits_base + g.nws;      // [step parity][x-links, y-links][nws]
  uint32_t* const Cb = flipb + 4 * g.nws;         // [2][rows_local][words]: this CTA's rows
  const int cbk = g.rows_local << g.lws;          // words of one link kind of Cb
  uint16_t* list = reinterpret_cast<uint16_t*>(Cb + 2 * cbk);
  int* misc = reinterpret_cast<int*>(list + ((g.cap + 7) & ~7));
  uint64_t* const ring = reinterpret_cast<uint64_t*>(misc + 16);  // orbit watch

  const int tid = G.tid, nt = G.nt;
  const int warp = tid >> 5, lane = tid & 31;
  // ---- dense-sweep role of this thread
  const int seg = warp * g.spw + lane / g.G;
  const int lis = lane % g.G;
  const bool warp_on = warp * g.spw < g.segments;
  const bool lane_on = (lane < g.spw * g.G) && (seg < g.segments);
  const int segc = lane_on ? seg : 0;
  const int pl = segc / g.bands;                 // plane
  const int lrow0 = (segc % g.bands) * g.H;      // first local row of the band
  const int R0 = rank * g.rows_local + lrow0;    // first global row
  const bool plus = (pl % 2) == 0;
  const int seg_base = lane - lis;
  const int left_lane = lane_on ? seg_base + (lis + g.G - 1) % g.G : lane;
  const int right_lane = lane_on ? seg_base + (lis + 1) % g.G : lane;
  const int cword = lis * KW;                    // first 32-bit word of the column strip
  const int LS = g.ls;
  uint8_t* my_rows = planes + ((size_t)(pl * g.rows_local + lrow0)) * LS + cword * 4;
  const int row_lo = rank * g.rows_local, row_hi = row_lo + g.rows_local;

  const int wpr = 1 << g.lws;  // bitmap words per row
  // barrier of the whole decoder: the group's, or the cluster's
  auto csync = [&]() {
    if constexpr (CL == 1) {
      G.sync();
    } else {
      Cluster<CL>::sync();
    }
  };

  uint32_t halo[6][KW];
  auto snapshot = [&]() {
    if (warp_on) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        load_words<KW>(plane_ptr<CL>(planes, g, pl, wrapi(R0 - 3 + k, L), cword * 4), halo[k]);
        int Rb = R0 + g.H + k;
        if (Rb >= L) Rb -= L;
        load_words<KW>(plane_ptr<CL>(planes, g, pl, Rb, cword * 4), halo[3 + k]);
      }
    }
  };

  const int64_t base = shot_offset_of(a, shot);
  const uint8_t* N = a.in + base;
  // ---- init: bitmaps cleared, sigma measured (every CTA of the cluster holds
  //      the full sigma); the planes are written whole by the first step
  {
    for (int i = tid; i < 4 * g.nws + 2 * cbk; i += nt) flipb[i] = 0;  // flip maps and Cb
    if (tid == 0) {
      misc[0] = 0;
      misc[5] = -1;  // orbit stop step
      misc[6] = 0;   // start of the run of steps with few anyons
    }
  }
  // sigma, 32 sites per thread and word; Def. synch_ccqs: parity of the four
  // links incident to r (or the given anyon indicator)
  for (int w = tid; w < g.nws; w += nt) {
    const int y = w >> g.lws, x0 = (w & (wpr - 1)) << 5;
    uint32_t bits = 0;
    if (x0 < L) {
      const int n = min(32, L - x0);
      if (a.from_sigma) {
        const uint8_t* row = N + (size_t)y * L + x0;
        for (int k = 0; k < n; k += 4)
          bits |= nonzero_nibble(*reinterpret_cast<const uint32_t*>(row + k)) << k;
      } else {
        const uint8_t* ex = N + (size_t)y * L + x0;
        const uint8_t* ey = N + LL + (size_t)y * L + x0;
        const uint8_t* eyd = N + LL + (size_t)wrapi(y - 1, L) * L + x0;
        uint32_t bx = 0, by = 0, byd = 0;
        for (int k = 0; k < n; k += 4) {
          bx |= nibble_of(*reinterpret_cast<const uint32_t*>(ex + k)) << k;
          by |= nibble_of(*reinterpret_cast<const uint32_t*>(ey + k)) << k;
          byd |= nibble_of(*reinterpret_cast<const uint32_t*>(eyd + k)) << k;
        }
        const uint32_t left = N[(size_t)y * L + wrapi(x0 - 1, L)] & 1u;  // e_x(r - x^) at x0
        bits = bx ^ ((bx << 1) | left) ^ by ^ byd;
        if (n < 32) bits &= (1u << n) - 1u;
      }
    }
    sig_cur[w] = bits;
  }
  G.sync();
  int any = build_list(sig_cur, g, list, &misc[0], G);
  int count = misc[0];

  int t = 0, flag = 0;
  // orbit watch: t_stop is -1 while watching, -2 when the rules draw random
  // numbers (the step is then not a function of the state alone), else the
  // step at which the shot stops
  int t_stop = (a.move_thr == 0 && a.balance_rule == QCA_BALANCE_STAY) ? -1 : -2;
  while (any) {
    if (t >= a.max_steps || t == t_stop) {
      // the budget ran out, or the shot is in a periodic orbit and its state
      // is that of the budget's last step
      flag = 2;
      t = a.max_steps;
      break;
    }
    if (t_stop == -1 && warp == 0) {
      // misc[6]: first step of the current run of steps with few anyons
      if (count > kOrbitAnyons) {
        if (lane == 0) misc[6] = t + 1;
      } else {
        const int stop = orbit_watch(ring, list, count, t, misc[6], a.max_steps, lane);
        if (stop >= 0 && lane == 0) misc[5] = stop;  // read by all after the step's barriers
      }
    }
    // flipped-link maps alternate by step parity: a partner CTA may still read
    // the previous step's map while this step writes the other one
    uint32_t* const flip = flipb + (t & 1) * 2 * g.nws;
    if (t == 0) {
      // ================= 1. first step: the planes start empty, so the
      // message update reduces to the anyon terms; compute them densely
      // for every site (32 sites per bitmap operation) instead of
      // scattering the cone sections of the many initial anyons.
      dense_terms<KW, false>(sig_cur, list, count, flip, g, planes, pl, lrow0, R0, plus, cword,
                             lane_on, G, pl >= 2, true);
    } else if (warp_on) {
      // ================= 1a. dense message update of this thread's band
      Chain cH[KW], cL[KW];
      uint32_t first[3][KW];
#pragma unroll
      for (int k = 0; k < 3; ++k) load_words<KW>(my_rows + (size_t)k * LS, first[k]);
#pragma unroll
      for (int q = 0; q < KW; ++q) {
        uint32_t ah[6], al[6];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          ah[k] = halo[k][q];
          ah[3 + k] = first[k][q];
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) al[k] = ah[k] << 8;
        cH[q].init(ah);
        cL[q].init(al);
      }
      auto row = [&](int i, const uint32_t (&in)[KW]) {
        uint32_t m[KW];
#pragma unroll
        for (int q = 0; q < KW; ++q) {
          const uint32_t tH = cH[q].step(in[q]);
          const uint32_t tL = cL[q].step(in[q] << 8);
          m[q] = finish_word(tL, tH);
        }
        uint32_t out[KW];
        if (KW == 1) {
          if (plus) {
            const uint32_t nb = __shfl_sync(0xffffffffu, m[0], left_lane);
            out[0] = __funnelshift_r(nb, m[0], 8);
          } else {
            const uint32_t nb = __shfl_sync(0xffffffffu, m[0], right_lane);
            out[0] = __funnelshift_r(m[0], nb, 24);
          }
        } else {
          const uint32_t sendv = plus ? m[KW - 1] : m[0];
          const uint32_t nb = __shfl_sync(0xffffffffu, sendv, plus ? left_lane : right_lane);
          if (plus) {
            out[0] = __funnelshift_r(nb, m[0], 8);
#pragma unroll
            for (int q = 1; q < KW; ++q) out[q] = __funnelshift_r(m[q - 1], m[q], 8);
          } else {
#pragma unroll
            for (int q = 0; q + 1 < KW; ++q) out[q] = __funnelshift_r(m[q], m[q + 1], 24);
            out[KW - 1] = __funnelshift_r(m[KW - 1], nb, 24);
          }
        }
        if (lane_on) store_words<KW>(my_rows + (size_t)i * LS, out);
      };
#pragma unroll 4
      for (int i = 0; i < g.H - 3; ++i) {
        uint32_t in[KW];
        load_words<KW>(my_rows + (size_t)(i + 3) * LS, in);
        row(i, in);
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        uint32_t in[KW];
#pragma unroll
        for (int q = 0; q < KW; ++q) in[q] = halo[3 + k][q];
        row(g.H - 3 + k, in);
      }
    }
    // ================= 1b. anyon terms of steps after the first
    if (t > 0) {
      if (count <= g.cap && count <= g.sparse_max) {
        // light-cone sections written per anyon, d = 3, 2, 1 (largest value
        // first); a warp takes one anyon, lane = (plane, transverse offset), so
        // the lanes of a store hit consecutive rows (distinct banks).  Each CTA
        // writes the sections that fall in its rows.
        G.sync();
        auto pass = [&](auto dconst) {
          constexpr int d = decltype(dconst)::value;
          const uint8_t val = (uint8_t)(g.off + d - 1);
          const int p = lane >> 3, jj = lane & 7;
          const bool act = jj < 2 * d + 1;
          const int nw = nt >> 5;
          // four anyons per warp and iteration (independent loads, then stores)
          for (int i0 = warp; i0 < count; i0 += 4 * nw) {
            int e[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const int i = i0 + k * nw;
              e[k] = (i < count) ? (int)list[i] : -1;
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const int x0 = e[k] & 0xFF, y0 = e[k] >> 8;
              if (act && e[k] >= 0) {
                const int row0 = (p < 2) ? y0 : x0;
                const int col0 = (p < 2) ? x0 : y0;
                const int col = wrapi((p % 2 == 0) ? col0 + d : col0 - d, L);
                const int R = wrapi(row0 + jj - d, L);
                if (CL == 1 || (R >= row_lo && R < row_hi))
                  planes[(size_t)(p * g.rows_local + R - row_lo) * LS + col] = val;
              }
            }
          }
          G.sync();
        };
        pass(std::integral_constant<int, 3>{});
        pass(std::integral_constant<int, 2>{});
        pass(std::integral_constant<int, 1>{});
      } else {
        G.sync();  // the dense update above is complete
        dense_terms<KW, true>(sig_cur, list, count, flip, g, planes, pl, lrow0, R0, plus, cword,
                              lane_on, G, pl >= 2, true);
      }
    }
    // clear this step's flipped-link map (also the scratch of the dense terms)
    G.sync();
    for (int i = tid; i < 2 * g.nws; i += nt) flip[i] = 0;
    // every plane of the cluster final; flip maps ready
    csync();
    snapshot();  // halo rows for the next step
    // ================= 2. forces and feedback for the anyons of this CTA's rows
    uint64_t kstep = 0, kbal = 0;
    if (a.move_thr) kstep = move_step_key(a.move_key, a.shot_offset + shot, t);
    if (a.balance_rule) kbal = move_step_key(a.balance_key, a.shot_offset + shot, t);
    auto decide = [&](int x, int y) -> int {
      // Eqs. blahdef / degbreak on the offset-encoded fields (0xFF = none)
      int dir = force_code(*plane_ptr<CL>(planes, g, 0, y, x), *plane_ptr<CL>(planes, g, 1, y, x),
                           *plane_ptr<CL>(planes, g, 2, x, y), *plane_ptr<CL>(planes, g, 3, x, y),
                           a.tie_order);
      if (dir >= 5) dir = a.balance_rule ? balance_resolve(dir, kbal, y * L + x) : 0;
      if (a.move_thr) {
        const uint64_t u = splitmix64(kstep ^ (uint64_t)(y * L + x));
        if (u < a.move_thr) dir = 1 + (int)(splitmix64(u) >> 62);
      }
      return dir;
    };
    auto apply = [&](int x, int y, int dir) {
      // mark link <lo, lo + a^>; a link crossed from both ends is marked
      // twice and flips once (the OR of Eq. ddfeedback)
      const int ax = (dir <= 2) ? 0 : 1;
      const int lx = (dir == 2) ? wrapi(x - 1, L) : x;
      const int ly = (dir == 4) ? wrapi(y - 1, L) : y;
      const int wlo = (ly << g.lws) + (lx >> 5);
      // every CTA keeps the whole map (fire-and-forget ORs, the remote one
      // through distributed shared memory)
#pragma unroll
      for (int r = 0; r < CL; ++r)
        atomicOr(Cluster<CL>::at(flip, r) + ax * g.nws + wlo, 1u << (lx & 31));
    };
    if (count <= g.cap) {
      // four anyons per thread and iteration: all field loads are issued before
      // the first atomic (latency hiding with few warps per SM)
      const int stride = (count + 31) >> 5, span = 32 * stride;
      for (int i0 = tid; i0 < span; i0 += 4 * nt) {
        int ex[4], ey[4], dir[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int i = i0 + k * nt;
          const int idx = (i & 31) * stride + (i >> 5);
          const bool ok = i < span && idx < count;
          const int e = ok ? list[idx] : 0;
          ex[k] = e & 0xFF;
          ey[k] = e >> 8;
          const bool mine = ok && (CL == 1 || (ey[k] >= row_lo && ey[k] < row_hi));
          dir[k] = mine ? decide(ex[k], ey[k]) : 0;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (dir[k]) apply(ex[k], ey[k], dir[k]);
      }
    } else {
      for_each_anyon(list, count, sig_cur, g, G, [&](int x, int y) {
        if (CL > 1 && (y < row_lo || y >= row_hi)) return;
        const int dir = decide(x, y);
        if (dir) apply(x, y, dir);
      });
    }
    if (tid == 0) misc[0] = 0;  // list counter (count already read by every thread)
    csync();
    // ================= 3. sigma and correction from the flipped links, new
    //                   anyon list, early exit
    any = apply_flips<kWordsPerThread<CL, KW>>(sig_cur, flip, Cb, g, list, &misc[0], row_lo, row_hi,
                                            G);
    count = misc[0];
    if (t_stop == -1) t_stop = misc[5];
    ++t;
  }
  // ================= outputs: correction bytes, homology, steps, flag
  // (each CTA holds the correction of its own rows)
  uint8_t* outC = a.out_C + correction_offset_of(a, shot);
  const int gpr = L / 4;  // 4-site groups per row
  for (int ax = 0; ax < 2; ++ax) {
    for (int i = tid; i < g.rows_local * gpr; i += nt) {
      const int yl = i / gpr, y = row_lo + yl, x = (i - yl * gpr) * 4;
      const uint32_t bits = Cb[ax * cbk + (yl << g.lws) + (x >> 5)];
      const uint32_t nib = (bits >> (x & 31)) & 0xFu;
      *reinterpret_cast<uint32_t*>(outC + (size_t)ax * LL + (size_t)y * L + x) =
          (nib * 0x00204081u) & 0x01010101u;
    }
  }
  if (tid == 0) misc[1] = misc[2] = 0;
  // every CTA's last correction update is done before rank 0 reads the
  // partners' shares below
  csync();
  if (rank == 0) {
    int wx = 0, wy = 0;
    for (int i = tid; i < L; i += nt) {
      // e_x((0, i)): row i, held by CTA i / rows_local; e_y((i, 0)): row 0, CTA 0
      const int owner = (CL == 1) ? 0 : i / g.rows_local;
      const uint32_t bx = Cluster<CL>::at(Cb, owner)[(i - owner * g.rows_local) << g.lws];
      const uint32_t by = Cb[cbk + (i >> 5)] >> (i & 31);
      wx ^= (int)(bx & 1);
      wy ^= (int)(by & 1);
      if (!a.from_sigma) {
        wx ^= N[(size_t)i * L];
        wy ^= N[LL + i];
      }
    }
    if (wx) atomicXor(&misc[1], 1);
    if (wy) atomicXor(&misc[2], 1);
    G.sync();
    if (tid == 0) {
      a.out_steps[shot] = t;
      if (a.from_sigma) {
        a.out_cut[2 * shot] = (uint8_t)misc[1];
        a.out_cut[2 * shot + 1] = (uint8_t)misc[2];
        if (a.out_exhausted) a.out_exhausted[shot] = (uint8_t)(flag == 2);
      } else {
        a.out_flag[shot] = (uint8_t)(flag == 2 ? 2 : ((misc[1] | misc[2]) ? 1 : 0));
      }
    }
  }
  // partners may still read this CTA's correction share
  csync();
}

template <int CL, int KW>
__global__ void __launch_bounds__(CL == 1 ? 1024 : (CL == 2 ? 512 : 256), CL == 4 ? 2 : 1)
    fast_kernel(DecodeArgs a, FastGeom g) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int rank = Cluster<CL>::rank();
  const int tid = threadIdx.x;
  const Grp G{tid, (int)blockDim.x, 0};
  int* misc = reinterpret_cast<int*>(smem + g.plane_bytes +
                                     (size_t)(5 * g.nws + 2 * (g.rows_local << g.lws)) * 4 +
                                     (size_t)((g.cap + 7) & ~7) * 2);
  const int nclusters = gridDim.x / CL;
  const int cid = blockIdx.x / CL;
  // Work: static (cluster c takes c, c + nclusters, ...) or, with a queue,
  // dynamic (rank 0 of the cluster takes the next index and shares it).
  auto next_work = [&](int64_t prev) -> int64_t {
    if (!a.queue) return prev < 0 ? (int64_t)cid : prev + nclusters;
    if (rank == 0 && tid == 0) misc[4] = (int)atomicAdd(a.queue, 1u);
    Cluster<CL>::sync();
    const int64_t k = (int64_t)*Cluster<CL>::at(&misc[4], 0);
    // rank 0 must neither overwrite the index nor exit (its shared memory goes
    // away) before every CTA of the cluster has read it
    if (CL > 1) Cluster<CL>::sync();
    return k;
  };
  for (int64_t k = next_work(-1); k < a.shots; k = next_work(k)) {
    const int64_t shot = a.shot_list ? (int64_t)a.shot_list[k] : k;
    decode_shot<CL, KW>(a, g, smem, shot, G);
  }
  // no CTA of a cluster leaves while a partner could still reach its shared memory
  if (CL > 1) Cluster<CL>::sync();
}

// ---------------------------------------------------------------- host ----

// Tuning overrides per lattice size, set by qca_set_tuning / qca_autotune:
// band height (0 = heuristic) and the anyon count below which the anyon terms
// are scattered per anyon, as a divisor of L^2 (0 = 64).
int g_tune_H[QCA_MAX_L + 1];
int g_tune_div[QCA_MAX_L + 1];
// Sizes above 128 decoded by a cluster of four CTAs (64 rows each, two clusters
// sharing each SM pair) instead of two.
int g_cluster4[QCA_MAX_L + 1];

// Anyon count (as a divisor of L^2) below which a step writes the anyon terms
// per anyon: measured best 64 for the one-CTA kernel and 256 for the two-CTA
// cluster, where the dense pass is split between the CTAs while every CTA
// scatters every anyon.
int sparse_divisor_for(int L, int CL) {
  if (g_tune_div[L] > 0) return g_tune_div[L];
  return CL >= 2 ? 256 : 64;
}

// Geometry of the on-chip sweep for L: CL (1 or 2 CTAs per shot), KW (words per
// lane), bands and shared-memory layout.  warp_cap > 0 asks for a one-CTA
// geometry with at most that many warps (the groups of the mixed-size kernel),
// also above L = 128, where the list is capped so that a lattice up to L = 192
// fits one CTA; the caller checks the shared memory.
bool make_geom(int L, int m_max, int& CL, int& KW, FastGeom& g, int& threads, size_t& smem,
               int warp_cap = 0) {
  if (L % 4 != 0 || L < 8 || L > 256) return false;
  if (m_max < 3) return false;  // the first-step fill assumes the d <= 3 terms fit below 0xFF
  if (L > 128 && L % 8 != 0) return false;
  // a group of the mixed-size kernel decodes its shot alone, up to L = 192
  CL = (L > 128 && warp_cap == 0) ? (g_cluster4[L] ? 4 : 2) : 1;
  KW = (L / 4 > 32) ? 2 : 1;
  g.L = L;
  g.rows_local = L / CL;
  g.G = L / 4 / KW;
  if (g.G > 32) return false;
  g.spw = 32 / g.G;
  // band height: 32, 16, 8 or 4 rows, dividing the CTA's rows, within the
  // thread limit; the one whose warp count is nearest a target (4 warps up to
  // L = 64, L / 8 above, at most 16; measured over band heights at L = 24 to
  // 128), the taller band on a tie.  The sweep takes any height of at least 4
  // that divides the CTA's rows; other heights are used only where none of
  // these four fits.
  const int max_warps = warp_cap > 0 ? std::min(32, warp_cap) : (CL == 1 ? 32 : (CL == 2 ? 16 : 8));
  const int target = std::min(max_warps, L <= 64 ? 4 : std::min(16, L / 8));
  int best_H = 0, best_d = 1 << 30;
  for (int H : {4, 8, 16, 32}) {
    if (g.rows_local % H) continue;
    const int segments = 4 * (g.rows_local / H);
    const int warps = (segments + g.spw - 1) / g.spw;
    if (warps > max_warps) continue;
    const int d = warps > target ? warps - target : target - warps;
    if (d <= best_d) {
      best_d = d;
      best_H = H;
    }
  }
  if (!best_H) {
    // no power-of-two band fits (for example L = 100 or 160): any other
    // divisor of the CTA's rows of at least 4 whose warp count is nearest the
    // target, the shorter band on a tie (heights are tried in increasing
    // order and only a strictly nearer count replaces the choice)
    for (int H = 5; H <= g.rows_local; ++H) {
      if (g.rows_local % H) continue;
      const int warps = (4 * (g.rows_local / H) + g.spw - 1) / g.spw;
      if (warps > max_warps) continue;
      const int d = warps > target ? warps - target : target - warps;
      if (d < best_d) {
        best_d = d;
        best_H = H;
      }
    }
  }
  for (int H : {4, 8, 16, 32}) {  // a valid override wins
    if (g_tune_H[L] != H || g.rows_local % H) continue;
    const int warps = (4 * (g.rows_local / H) + g.spw - 1) / g.spw;
    if (warps <= max_warps) best_H = H;
  }
  if (!best_H) return false;
  g.H = best_H;
  g.bands = g.rows_local / g.H;
  g.segments = 4 * g.bands;
  const int warps = (g.segments + g.spw - 1) / g.spw;
  threads = warps * 32;
  int wpr = (L + 31) / 32, lws = 0;
  while ((1 << lws) < wpr) ++lws;
  g.lws = lws;
  g.nws = L << lws;
  // the dense feedback pass handles at most this many words per thread
  const int max_per = CL == 1 ? (KW == 2 ? kWordsPerThread<1, 2> : kWordsPerThread<1, 1>)
                               : (CL == 2 ? kWordsPerThread<2, 2> : kWordsPerThread<4, 2>);
  if ((g.nws + threads - 1) / threads > max_per) return false;
  g.off = 255 - m_max;
  // up to half the lattice in the list (more anyons than that are iterated
  // from the bitmap; a noise rate below 0.5 rarely comes near it)
  g.cap = std::min(L * L / 2, kListCap);
  if (CL == 4) g.cap = std::min(g.cap, 1024);  // two CTAs of a cluster of four share an SM
  if (CL == 1 && L > 128) g.cap = std::min(g.cap, 8192);  // a whole L <= 192 lattice in one CTA
  g.sparse_max = L * L / sparse_divisor_for(L, CL);
  // row pitch: L + 4 bytes (one extra bank per row); L + 8 keeps the 8-byte
  // alignment of the 64-bit accesses used with two words per lane
  g.ls = L + (KW == 2 ? 8 : 4);
  g.plane_bytes = (size_t)4 * g.rows_local * g.ls;
  // sigma, two flipped-link maps (x and y each), the correction of the CTA's
  // rows (x and y), list, 64 bytes of counters, orbit ring
  smem = g.plane_bytes + (size_t)(5 * g.nws + 2 * (g.rows_local << lws)) * 4 +
         (size_t)((g.cap + 7) & ~7) * 2 + 64 + (size_t)kOrbitRing * 8;
  return true;
}

// Launch shape of one kernel variant for one (threads, shared memory) pair on
// one device: found once with the occupancy calculator and cached, so that a
// later call (for instance under CUDA-graph capture) only enqueues the launch.
struct LaunchShape {
  int dev, cl, kw, threads;
  size_t smem;
  int units;  // resident CTAs (CL = 1) or clusters (CL = 2) on the whole GPU
};
std::mutex g_shape_mu;
std::vector<LaunchShape> g_shapes;

// ------------------------------------------------ mixed lattice sizes ----
//
// One persistent launch for a batch of shots of different sizes.  The items
// (shots) are queued by group size, then largest L first, so that the long
// shots start early and the short ones fill the tail, and every group takes
// the next item from one counter when it has finished its last (work stealing
// across sizes; every shot retires after its own number of steps).
//   * pair items, sizes that no CTA holds alone (above L = 192), are decoded
//     by the two CTAs of a cluster;
//   * every other size has a group size of 512, 256 or 128 threads (the
//     smallest whose band geometry and shared memory fit; 512 with two plane
//     words per lane for 128 < L <= 192): a CTA of 512
//     threads starts as one group and halves whenever the item it holds needs
//     a smaller group, the first half keeping the item and the second fetching
//     its own, so that up to four small lattices are decoded at once per CTA.
// Each group has its own named barrier and its own slice of shared memory: the
// 64-thread slice s (threads 64s .. 64s + 63) owns bytes [s, s + 1) * S / 8 of
// the S-byte block, a group the slices of its threads.
// Rank 0 of a cluster fetches pair items and shares the index over DSMEM; the
// first other index it sees ends the pair phase for both CTAs (rank 0 keeps
// that item).
constexpr int kMixThreads = 512;
constexpr int kMixMaxClasses = 8;

struct MixArgs {
  DecodeArgs a;                   // outputs, offsets, rules; shot_list = item -> shot
  const uint8_t* item_class;      // item -> class
  int64_t n_pair, n_items;
  size_t slice_bytes;             // shared memory of a 64-thread slice (S / 8)
  int group_threads[kMixMaxClasses];  // 0 for pair classes
  FastGeom geom[kMixMaxClasses];
};

// named barrier of the group of `gsz` threads starting at thread `gofs`:
// 0 for the whole CTA, then 1-2 (256), 3-6 (128), 7-14 (64)
__device__ __forceinline__ int mix_barrier(int gsz, int gofs) {
  if (gsz >= kMixThreads) return 0;
  if (gsz == 256) return 1 + gofs / 256;
  if (gsz == 128) return 3 + gofs / 128;
  return 7 + gofs / 64;
}

__global__ void __launch_bounds__(kMixThreads, 1) mixed_kernel(MixArgs m) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ long long s_item[16];
  const int tid = threadIdx.x;
  cg::cluster_group cluster = cg::this_cluster();
  const int csize = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  long long k = -1;
  // ---- pair items: both CTAs of the cluster on one shot
  if (m.n_pair > 0 && csize == 2) {
    const Grp whole{tid, kMixThreads, 0};
    for (;;) {
      if (rank == 0 && tid == 0) s_item[15] = (long long)atomicAdd(m.a.queue, 1u);
      cluster.sync();
      const long long kk = *cluster.map_shared_rank(&s_item[15], 0);
      // rank 0 must not overwrite the index before its partner has read it
      cluster.sync();
      if (kk >= m.n_pair) {
        k = (rank == 0) ? kk : -1;
        break;
      }
      decode_shot<2, 2>(m.a, m.geom[m.item_class[kk]], smem, m.a.shot_list[kk], whole);
    }
  }
  // ---- every other item: groups of 512, 256, 128 or 64 threads
  int gsz = kMixThreads, gofs = 0;
  for (;;) {
    const int bar = mix_barrier(gsz, gofs);
    const Grp G{tid - gofs, gsz, bar};
    if (k < 0) {
      if (G.tid == 0) s_item[bar] = (long long)atomicAdd(m.a.queue, 1u);
      G.sync();
      k = s_item[bar];
      G.sync();
    }
    if (k >= m.n_items) break;
    const int c = m.item_class[k];
    if (m.group_threads[c] < gsz) {
      // the item needs a smaller group: halve; the first half keeps it
      gsz >>= 1;
      if (tid - gofs >= gsz) {
        gofs += gsz;
        k = -1;
      }
      continue;
    }
    if (m.geom[c].L > 128)  // two plane words per lane
      decode_shot<1, 2>(m.a, m.geom[c], smem + (size_t)(gofs / 64) * m.slice_bytes,
                        m.a.shot_list[k], G);
    else
      decode_shot<1, 1>(m.a, m.geom[c], smem + (size_t)(gofs / 64) * m.slice_bytes,
                        m.a.shot_list[k], G);
    k = -1;
  }
  __syncthreads();
  // a partner's pair-phase accesses to this CTA's shared memory are over, but
  // keep the exit ordered as in the one-size kernel
  if (csize == 2) cluster.sync();
}

template <int CL, int KW>
int launch_t(const DecodeArgs& a, const FastGeom& g, int threads, size_t smem,
             cudaStream_t stream) {
  auto kern = fast_kernel<CL, KW>;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  if (CL > 1) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  int units = -1;
  {
    std::lock_guard<std::mutex> lk(g_shape_mu);
    for (const LaunchShape& s : g_shapes)
      if (s.dev == dev && s.cl == CL && s.kw == KW && s.threads == threads && s.smem == smem)
        units = s.units;
  }
  if (units < 0) {
    // first use of this shape: allow the largest dynamic shared memory any
    // configuration asks for, then ask the occupancy calculator
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "fast sweep smem attribute");
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (CL == 1) {
      int resident = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, kern, threads, smem);
      if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
      units = resident * sms;
    } else {
      cfg.gridDim = dim3((unsigned)(CL * sms));
      e = cudaOccupancyMaxActiveClusters(&units, kern, &cfg);
      if (e != cudaSuccess) return cuda_fail(e, "cluster occupancy query");
    }
    if (units < 1) {
      set_error("fast sweep does not fit on an SM (L=%d)", a.L);
      return QCA_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_shape_mu);
    g_shapes.push_back({dev, CL, KW, threads, smem, units});
  } else {
    // the attribute is per function; a shape with less shared memory than a
    // previous one still launches within the larger allowance
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "fast sweep smem attribute");
  }
  int64_t grid = units;
  if (grid > a.shots) grid = a.shots;
  cfg.gridDim = dim3((unsigned)(grid * CL));
  e = cudaLaunchKernelEx(&cfg, kern, a, g);
  return cuda_fail(e, "fast sweep launch");
}

}  // namespace

int fast_path_for(int L, int v, int m_max) {
  if (v != 3) return 0;
  int CL, KW, threads;
  FastGeom g;
  size_t smem;
  if (!make_geom(L, m_max, CL, KW, g, threads, smem)) return 0;
  return CL > 2 ? 2 : CL;
}

int launch_fast(const DecodeArgs& a, cudaStream_t stream) {
  int CL, KW, threads;
  FastGeom g;
  size_t smem;
  if (a.v != 3 || !make_geom(a.L, a.m_max, CL, KW, g, threads, smem)) {
    set_error("no on-chip kernel for L=%d v=%d", a.L, a.v);
    return QCA_ERR_UNSUPPORTED;
  }
  if (CL == 1 && KW == 1) return launch_t<1, 1>(a, g, threads, smem, stream);
  if (CL == 2 && KW == 2) return launch_t<2, 2>(a, g, threads, smem, stream);
  if (CL == 4 && KW == 2) return launch_t<4, 2>(a, g, threads, smem, stream);
  set_error("no on-chip kernel variant for L=%d", a.L);
  return QCA_ERR_UNSUPPORTED;
}

// Host side of the mixed-size kernel.  Dynamic shared memory available to one
// CTA (227 KB less room for the kernel's static shared memory).
constexpr size_t kMixSmemLimit = 227 * 1024 - 1024;

// Group size of each size in the mixed kernel: 512, 256 or 128 threads, the
// smallest whose one-CTA band geometry fits its warps and whose shared memory
// times the groups of a CTA fits the limit; else 0 for a pair item (two-CTA
// cluster; sizes above 192); -1 if the on-chip sweep does not take the size.
// (One CTA per L = 192 shot instead of a pair took the C3 batch from 67.7 to
// 58.8 ms; groups of 64 threads, eight small lattices per CTA, measured
// slower: 109 against 99 ms.)
int mixed_group_threads(int L, int m_max) {
  int CL, KW, th;
  FastGeom g;
  size_t sm;
  if (!make_geom(L, m_max, CL, KW, g, th, sm)) return -1;
  const bool pair_ok = CL == 2 && sm <= kMixSmemLimit;
  for (int gs = 128; gs <= kMixThreads; gs *= 2) {
    int cl, kw, t2;
    size_t s2;
    if (!make_geom(L, m_max, cl, kw, g, t2, s2, gs / 32)) continue;
    const size_t per = (s2 + 127) & ~(size_t)127;
    if (per * (kMixThreads / gs) <= kMixSmemLimit) return gs;
  }
  return pair_ok ? 0 : -1;
}

int launch_mixed(const DecodeArgs& a, const uint8_t* item_class, const int* sizes,
                 const int* group_threads, int nclass, int64_t n_pair, int64_t n_items,
                 cudaStream_t stream) {
  if (nclass > kMixMaxClasses) {
    set_error("mixed-size decode: more than %d sizes", kMixMaxClasses);
    return QCA_ERR_UNSUPPORTED;
  }
  MixArgs m;
  memset(&m, 0, sizeof(m));
  m.a = a;
  m.item_class = item_class;
  m.n_pair = n_pair;
  m.n_items = n_items;
  // S: the largest of the pair classes' shared memory and, per other class,
  // its shared memory times the groups of its size in a CTA
  size_t S = 0;
  size_t cls_smem[kMixMaxClasses] = {};
  for (int c = 0; c < nclass; ++c) {
    int CL, KW, th;
    const int gs = group_threads[c];
    m.group_threads[c] = gs;
    if (gs < 0) continue;
    const bool ok = make_geom(sizes[c], a.m_max, CL, KW, m.geom[c], th, cls_smem[c],
                              gs > 0 ? gs / 32 : 0) &&
                    (gs == 0) == (CL == 2);
    if (!ok) {
      set_error("mixed-size decode: no geometry for L = %d", sizes[c]);
      return QCA_ERR_UNSUPPORTED;
    }
    cls_smem[c] = (cls_smem[c] + 127) & ~(size_t)127;
    S = std::max(S, gs == 0 ? cls_smem[c] : cls_smem[c] * (kMixThreads / gs));
  }
  S = (S + 1023) & ~(size_t)1023;  // eight slices, each a multiple of 128 bytes
  if (S > kMixSmemLimit) {
    set_error("mixed-size decode: %zu bytes of shared memory needed", S);
    return QCA_ERR_UNSUPPORTED;
  }
  m.slice_bytes = S / 8;
  const int CL = n_pair > 0 ? 2 : 1;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cfg.blockDim = dim3(kMixThreads);
  cfg.dynamicSmemBytes = S;
  cfg.stream = stream;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int units = -1;
  {
    std::lock_guard<std::mutex> lk(g_shape_mu);
    for (const LaunchShape& sh : g_shapes)
      if (sh.dev == dev && sh.cl == CL && sh.kw == -1 && sh.threads == kMixThreads && sh.smem == S)
        units = sh.units;
  }
  e = cudaFuncSetAttribute(mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S);
  if (e != cudaSuccess) return cuda_fail(e, "mixed kernel smem attribute");
  if (units < 0) {
    cfg.gridDim = dim3((unsigned)(CL * sms));
    e = cudaOccupancyMaxActiveClusters(&units, mixed_kernel, &cfg);
    if (e != cudaSuccess) return cuda_fail(e, "mixed kernel occupancy query");
    if (units < 1) {
      set_error("mixed-size kernel does not fit on an SM");
      return QCA_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_shape_mu);
    g_shapes.push_back({dev, CL, -1, kMixThreads, S, units});
  }
  int64_t grid = units;
  // no more clusters than items (each takes at least one)
  const int64_t need = (n_items + CL - 1) / CL;
  if (grid > need) grid = need > 0 ? need : 1;
  cfg.gridDim = dim3((unsigned)(grid * CL));
  e = cudaLaunchKernelEx(&cfg, mixed_kernel, m);
  return cuda_fail(e, "mixed kernel launch");
}

}  // namespace qca

using namespace qca;

extern "C" {

int qca_set_tuning(int L, int band_height, int sparse_divisor) {
  if (L < 3 || L > QCA_MAX_L || band_height < 0 || sparse_divisor < 0) {
    set_error("qca_set_tuning: bad arguments");
    return QCA_ERR_ARG;
  }
  g_tune_H[L] = band_height;
  g_tune_div[L] = sparse_divisor;
  return QCA_OK;
}

int qca_set_cluster_ctas(int L, int ctas) {
  if (L <= 128 || L > 256 || L % 8 != 0 || (ctas != 2 && ctas != 4)) {
    set_error("qca_set_cluster_ctas: L must be a multiple of 8 in (128, 256], ctas 2 or 4");
    return QCA_ERR_ARG;
  }
  g_cluster4[L] = ctas == 4 ? 1 : 0;
  return QCA_OK;
}

int qca_get_tuning(int L, int* band_height, int* sparse_divisor, int* threads_per_cta) {
  if (L < 3 || L > QCA_MAX_L) {
    set_error("qca_get_tuning: bad L");
    return QCA_ERR_ARG;
  }
  int CL, KW, threads = 0;
  FastGeom g;
  size_t smem;
  const bool fast = make_geom(L, 255, CL, KW, g, threads, smem);
  if (band_height) *band_height = fast ? g.H : 0;
  if (sparse_divisor) *sparse_divisor = sparse_divisor_for(L, fast ? CL : 1);
  if (threads_per_cta) *threads_per_cta = fast ? threads : 0;
  return fast ? QCA_OK : QCA_ERR_UNSUPPORTED;
}

int qca_autotune(int L, int64_t shots, double p, uint64_t seed, int max_steps,
                 int* best_band_height, int* best_sparse_divisor, float* best_ms) {
  if (L < 3 || L > QCA_MAX_L || shots <= 0 || !(p >= 0.0 && p <= 1.0)) {
    set_error("qca_autotune: bad arguments");
    return QCA_ERR_ARG;
  }
  int CL, KW, threads;
  FastGeom g;
  size_t smem;
  if (!make_geom(L, 255, CL, KW, g, threads, smem)) {
    set_error("qca_autotune: L = %d has no on-chip kernel to tune", L);
    return QCA_ERR_UNSUPPORTED;
  }
  const size_t E = 2 * (size_t)L * L;
  uint8_t *N = nullptr, *C = nullptr, *F = nullptr;
  int32_t* S = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&N, E * shots);
  if (e == cudaSuccess) e = cudaMalloc(&C, E * shots);
  if (e == cudaSuccess) e = cudaMalloc(&F, shots);
  if (e == cudaSuccess) e = cudaMalloc(&S, 4 * shots);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  int rc = cuda_fail(e, "qca_autotune setup");
  if (rc == QCA_OK) rc = qca_sample_errors_async(L, 0, shots, p, seed, N, st);
  const int saved_H = g_tune_H[L], saved_div = g_tune_div[L];
  int bH = 0, bD = 0;
  float bms = 1e30f;
  for (int H : {4, 8, 16, 32}) {
    if (rc != QCA_OK) break;
    g_tune_H[L] = H;
    int CL2, KW2, th2;
    FastGeom g2;
    size_t sm2;
    if (!make_geom(L, 255, CL2, KW2, g2, th2, sm2) || g2.H != H) continue;  // invalid here
    for (int div : {256, 128, 64, 32}) {
      g_tune_div[L] = div;
      // one untimed run, then the median of three timed runs
      rc = qca_decode_batch_async(N, L, shots, max_steps, 0, C, S, F, nullptr, st);
      float t[3];
      for (int r = 0; r < 3 && rc == QCA_OK; ++r) {
        cudaEventRecord(e0, st);
        rc = qca_decode_batch_async(N, L, shots, max_steps, 0, C, S, F, nullptr, st);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) rc = cuda_fail(e, "qca_autotune timing");
        if (rc == QCA_OK) cudaEventElapsedTime(&t[r], e0, e1);
      }
      if (rc != QCA_OK) break;
      std::sort(t, t + 3);
      if (t[1] < bms) {
        bms = t[1];
        bH = H;
        bD = div;
      }
    }
  }
  if (rc == QCA_OK && bH) {
    g_tune_H[L] = bH;
    g_tune_div[L] = bD;
  } else {
    g_tune_H[L] = saved_H;
    g_tune_div[L] = saved_div;
  }
  if (best_band_height) *best_band_height = bH;
  if (best_sparse_divisor) *best_sparse_divisor = bD;
  if (best_ms) *best_ms = bms;
  if (st) cudaStreamSynchronize(st);
  cudaFree(N);
  cudaFree(C);
  cudaFree(F);
  cudaFree(S);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  return rc;
}

}  // extern "C"
