// Large-lattice synchronous sweep: L a multiple of 128 up to 1024, v = 3.
//
// A 1024^2 lattice needs 4 MB of message fields, more than one SM holds, so the
// state of a shot lives in a per-cluster slot of global memory (mostly L2
// resident) and a cluster of 8 CTAs decodes one shot, each CTA owning L/8 rows
// of every plane.  Each step:
//   1. messages (the v = 3 applications of A^(D), Def. Dd_msg_passing, fused
//      exactly as in the on-chip kernel): every CTA streams bands of 16 rows of
//      each plane plus 3 halo rows on either side, and the matching rows of the
//      syndrome bitmap, from the previous step's buffer into shared memory with
//      bulk asynchronous copies (completion on an mbarrier, the next band
//      prefetched while this one is computed); computes
//        w3(r) = min( off + d - 1 for the smallest d <= 3 with an anyon on
//                     {r - s d a^ + j b^, |j| <= d},
//                     satadd( min_{|j| <= 3} w0(r - 3 s a^ + j b^), 3 ) )
//      and writes the band to the other buffer;
//   2. forces and feedback (Eqs. blahdef, degbreak, ddfeedback) for the anyons
//      of the CTA's rows: each ORs the bit of the link it crosses into the
//      flipped-link maps (a link crossed from both ends flips once);
//   3. sigma <- sigma xor (syndrome of the flipped links), correction ^= flips,
//      anyon count; the cluster agrees on the early exit.
// Cluster barriers separate the phases (three per step).  Planes are stored as
// in the on-chip kernel, each in the frame where its messages travel along the
// byte axis (x fields [y][x], y fields [x][y]), with the offset encoding
// w = m - 1 + (255 - m_max), 0xFF = no message.  The syndrome and the flipped
// links are kept as bitmaps in both frames, so the terms of either plane family
// and the sigma update read rows only.
#include <cooperative_groups.h>

#include <mutex>
#include <vector>

#include "qca_internal.cuh"

namespace cg = cooperative_groups;

namespace qca {

namespace {

constexpr int kTCL = 8;        // CTAs per cluster: one shot
constexpr int kTThreads = 256;
// Plane rows per staged band, staged with 3 halo rows on either side.  16-row
// bands keep a CTA at 51 KB of shared memory and 64 registers, four CTAs per
// SM; 32-row bands (two CTAs per SM) measured slower.
constexpr int kTB = 16;
constexpr int kTRows = kTB + 6;
constexpr int kTCtasPerSm = 4;
constexpr long long kWaitCycles = 4000000000LL;  // watchdog on a copy (about 2 s)
// bitmap rows whose global loads are issued together (move phase, sigma update)
constexpr int kMoveBatch = 2;
constexpr int kSigBatch = 2;

struct TiledGeom {
  int L;
  int W;      // 32-bit words per bitmap row (L / 32)
  int RL;     // rows per CTA in either frame (L / 8)
  int cols;   // 32-bit words per plane row (L / 4)
  int off;    // 255 - m_max
  size_t LL;
  // slot layout (byte offsets)
  size_t o_sig, o_flip, o_C, slot;
  // shared memory layout (byte offsets)
  size_t s_band, s_sband, s_bar, s_misc, smem;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bulk copy global -> this CTA's shared memory, completion counted on bar.
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Generic-proxy global writes <-> bulk-copy (async proxy) reads.
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Wait for phase `parity` of bar, at most kWaitCycles; false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > kWaitCycles) return false;
  }
  return true;
}

__device__ __forceinline__ int twrap(int i, int L) { return i < 0 ? i + L : (i >= L ? i - L : i); }

// 4 bits -> 4 bytes of 0xFF / 0x00 (bit k -> byte k).
__device__ __forceinline__ uint32_t nib_mask(uint32_t nib) {
  return ((nib * 0x00204081u) & 0x01010101u) * 0xFFu;
}
__device__ __forceinline__ uint32_t nibble_of_bytes(uint32_t w) { return (w * 0x01020408u) >> 24; }

// n words (a multiple of 4, 16-byte aligned: every row range of the slot's
// planes and bitmaps is) set to v by the threads of the CTA, 16 bytes a store.
__device__ __forceinline__ void fill_words(uint32_t* p, int n, uint32_t v, int tid, int nt) {
  uint4* q = reinterpret_cast<uint4*>(p);
  const uint4 vv = make_uint4(v, v, v, v);
  for (int i = tid; i < (n >> 2); i += nt) q[i] = vv;
}

template <class T>
__device__ __forceinline__ T* rank_ptr(T* p, int r) {
  return cg::this_cluster().map_shared_rank(p, (unsigned)r);
}

__global__ void __launch_bounds__(kTThreads, kTCtasPerSm) tiled_kernel(DecodeArgs a, TiledGeom g,
                                                             uint8_t* ws) {
  extern __shared__ __align__(128) uint8_t smem[];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int L = g.L, W = g.W, RL = g.RL, cols = g.cols;
  const size_t LL = g.LL;
  const int r0 = rank * RL;  // first own row in either frame
  const int nclusters = gridDim.x / kTCL;
  const int cid = blockIdx.x / kTCL;

  uint8_t* band = smem + g.s_band;                                         // [2][kTRows][L]
  uint32_t* sband = reinterpret_cast<uint32_t*>(smem + g.s_sband);         // [2][kTRows][W]
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + g.s_bar);             // [2]
  int* misc = reinterpret_cast<int*>(smem + g.s_misc);
  // misc: [0..1] anyon counts by step parity (rank 0), [2] wx, [3] wy (rank 0),
  //       [4] next shot (rank 0), [5] abort (rank 0), [6] block scratch

  uint8_t* slot = ws + (size_t)cid * g.slot;
  auto plane = [&](int buf, int p) -> uint8_t* { return slot + ((size_t)(buf * 4 + p)) * LL; };
  uint32_t* sig = reinterpret_cast<uint32_t*>(slot + g.o_sig);  // [frame][L][W]
  auto sigf = [&](int frame) -> uint32_t* { return sig + (size_t)frame * L * W; };
  uint32_t* flipb = reinterpret_cast<uint32_t*>(slot + g.o_flip);  // [par][frame][kind][L][W]
  auto flip = [&](int par, int frame, int kind) -> uint32_t* {
    return flipb + ((size_t)((par * 2 + frame) * 2 + kind)) * L * W;
  };
  uint32_t* Cb = reinterpret_cast<uint32_t*>(slot + g.o_C);  // [kind][L][W], x frame

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  if (tid < 8) misc[tid] = 0;
  __syncthreads();
  uint32_t phase[2] = {0u, 0u};
  bool inflight[2] = {false, false};  // copies issued and not yet waited for (thread 0)

  const int nbands = RL / kTB;
  const int ntasks = 4 * nbands;
  const uint32_t task_bytes = (uint32_t)(kTRows * L + kTRows * W * 4);

  // issue the copies of task i (plane p, band b) of a step reading buffer `src`
  // called by the 32 lanes of warp 0: lane 0 posts the expected bytes, then
  // every lane issues the copies of its rows
  auto issue = [&](int i, int src) {
    const int p = i / nbands, b = i - p * nbands;
    const int buf = i & 1;
    const int R0 = r0 + b * kTB;
    const uint8_t* P = plane(src, p);
    const uint32_t* S = sigf(p < 2 ? 0 : 1);
    fence_proxy_async_global();
    if (lane == 0) {
      inflight[buf] = true;
      mbar_expect_tx(&bar[buf], task_bytes);
    }
    __syncwarp();
    for (int j = lane; j < kTRows; j += 32) {
      const int R = twrap(R0 - 3 + j, L);
      bulk_g2s(band + ((size_t)buf * kTRows + j) * L, P + (size_t)R * L, (uint32_t)L, &bar[buf]);
      bulk_g2s(sband + ((size_t)buf * kTRows + j) * W, S + (size_t)R * W, (uint32_t)(W * 4),
               &bar[buf]);
    }
  };

  auto next_work = [&](int64_t prev) -> int64_t {
    if (!a.queue) return prev < 0 ? (int64_t)cid : prev + nclusters;
    if (rank == 0 && tid == 0) misc[4] = (int)atomicAdd(a.queue, 1u);
    cluster.sync();
    const int64_t k = (int64_t)*rank_ptr(&misc[4], 0);
    cluster.sync();
    return k;
  };

  bool aborted = false;
  for (int64_t k = next_work(-1); k < a.shots && !aborted; k = next_work(k)) {
    const int64_t shot = a.shot_list ? (int64_t)a.shot_list[k] : k;
    const uint8_t* N = a.in + shot_offset_of(a, shot);

    // ---- init (own rows): empty planes, cleared maps, sigma in the x frame
    {
      for (int p = 0; p < 4; ++p) {
        uint32_t* P = reinterpret_cast<uint32_t*>(plane(0, p)) + (size_t)r0 * cols;
        fill_words(P, RL * cols, 0xFFFFFFFFu, tid, nt);
      }
      for (int par = 0; par < 2; ++par)
        for (int fr = 0; fr < 2; ++fr)
          for (int kd = 0; kd < 2; ++kd) {
            uint32_t* F = flip(par, fr, kd) + (size_t)r0 * W;
            fill_words(F, RL * W, 0u, tid, nt);
          }
      for (int kd = 0; kd < 2; ++kd) {
        uint32_t* C = Cb + (size_t)kd * L * W + (size_t)r0 * W;
        fill_words(C, RL * W, 0u, tid, nt);
      }
      // sigma (Def. synch_ccqs: parity of the four links incident to r)
      uint32_t* Sx = sigf(0);
      int cnt = 0;
      // a warp per row, a lane per word (W <= 32)
      for (int rr = warp; rr < RL; rr += nw) {
        if (lane >= W) continue;
        const int y = r0 + rr, x0 = lane * 32;
        uint32_t bits = 0;
        if (a.from_sigma) {
          const uint8_t* row = N + (size_t)y * L + x0;
          for (int q = 0; q < 32; q += 4) {
            const uint32_t w = *reinterpret_cast<const uint32_t*>(row + q);
            const uint32_t nz = (((w & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | w) & 0x80808080u;
            bits |= nibble_of_bytes(nz >> 7) << q;
          }
        } else {
          const uint8_t* ex = N + (size_t)y * L + x0;
          const uint8_t* ey = N + LL + (size_t)y * L + x0;
          const uint8_t* eyd = N + LL + (size_t)twrap(y - 1, L) * L + x0;
          uint32_t bx = 0, by = 0, byd = 0;
          for (int q = 0; q < 32; q += 4) {
            bx |= nibble_of_bytes(*reinterpret_cast<const uint32_t*>(ex + q)) << q;
            by |= nibble_of_bytes(*reinterpret_cast<const uint32_t*>(ey + q)) << q;
            byd |= nibble_of_bytes(*reinterpret_cast<const uint32_t*>(eyd + q)) << q;
          }
          const uint32_t left = N[(size_t)y * L + twrap(x0 - 1, L)] & 1u;  // e_x(r - x^)
          bits = bx ^ ((bx << 1) | left) ^ by ^ byd;
        }
        Sx[(size_t)y * W + lane] = bits;
        cnt += __popc(bits);
      }
      fence_proxy_async_global();
      cluster.sync();  // the x-frame sigma of every row is written
      // y-frame sigma of the own rows (x = r0 .. r0 + RL - 1) by 32 x 32 bit
      // transposes: lane i loads row y = 32 wy + i, ballot j gives column x
      uint32_t* Sy = sigf(1);
      const int qlo = r0 >> 5, nq = ((r0 + RL - 1) >> 5) - qlo + 1;
      for (int blk = warp; blk < W * nq; blk += nw) {
        const int wy = blk / nq, qx = qlo + blk % nq;
        const uint32_t v = Sx[(size_t)(32 * wy + lane) * W + qx];
        uint32_t mine = 0;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const uint32_t col = __ballot_sync(0xFFFFFFFFu, (v >> j) & 1u);
          if (lane == j) mine = col;
        }
        const int x = 32 * qx + lane;
        if (x >= r0 && x < r0 + RL) Sy[(size_t)x * W + wy] = mine;
      }
      // anyon count of the own x-frame rows, summed on rank 0
      for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
      if (lane == 0 && cnt) atomicAdd(rank_ptr(&misc[1], 0), cnt);
      fence_proxy_async_global();
      cluster.sync();
    }
    int any = *rank_ptr(&misc[1], 0);

    int t = 0, flag = 0;
    while (any) {
      if (t >= a.max_steps) {
        flag = 2;
        break;
      }
      const int src = t & 1, dst = src ^ 1;
      // ================= 1. messages: bands staged by bulk copies
      if (warp == 0) issue(0, src);
      for (int i = 0; i < ntasks; ++i) {
        if (warp == 0 && i + 1 < ntasks && !aborted) issue(i + 1, src);
        const int buf = i & 1;
        const bool ok = mbar_wait_bounded(&bar[buf], phase[buf]);
        // every thread waited on the copies itself; a wait that gave up is
        // agreed on at the band's closing barrier (the band is then garbage,
        // read and written at the same data-independent places, and the shot
        // ends with flag 3)
        if (ok) {
          phase[buf] ^= 1u;
          inflight[buf] = false;
        }
        const int p = i / nbands, b = i - p * nbands;
        const int R0 = r0 + b * kTB;
        const uint8_t* Bk = band + (size_t)buf * kTRows * L;
        const uint32_t* Sb = sband + (size_t)buf * kTRows * W;
        // fused message update of the band, one 4-site column word per thread:
        // every staged row is shifted by 3 sites along the byte axis as it is
        // loaded (funnel shift with the neighbouring column word, wrapping at
        // the row end).  The shift commutes with the bytewise min over rows and
        // with the saturating add, so the transverse min over 7 rows (rolling
        // down the band, 3 mins per half-word and row), the +3 and the anyon
        // terms then give the output word directly.
        const bool plus = (p % 2) == 0;  // m^{+a} reads from r - 3 a^
        uint32_t* out = reinterpret_cast<uint32_t*>(plane(dst, p)) + (size_t)R0 * cols;
        const uint32_t v1 = (uint32_t)(g.off) * 0x01010101u;
        for (int kc = tid; kc < cols; kc += nt) {
          const uint32_t* col = reinterpret_cast<const uint32_t*>(Bk) + kc;
          const int kn = plus ? (kc == 0 ? cols - 1 : kc - 1) : (kc + 1 == cols ? 0 : kc + 1);
          const uint32_t* nbc = reinterpret_cast<const uint32_t*>(Bk) + kn;
          auto shifted = [&](int j) -> uint32_t {
            const uint32_t w = col[(size_t)j * cols], nb = nbc[(size_t)j * cols];
            return plus ? __funnelshift_r(nb, w, 8) : __funnelshift_r(w, nb, 24);
          };
          // the d <= 3 cones of the word's four sites read positions
          // 4 kc - 3 .. 4 kc + 2 (m^+) or 4 kc + 1 .. 4 kc + 6 (m^-) of the
          // dilated syndrome rows
          const int pos6 = twrap(4 * kc + (plus ? -3 : 1), L);
          const int q6 = pos6 >> 5, sh6 = pos6 & 31, q6n = (q6 + 1 == W) ? 0 : q6 + 1;
          // six syndrome bits pos6 .. pos6 + 5 of staged row j
          auto sig6 = [&](int j) -> uint32_t {
            const uint32_t* row = Sb + (size_t)j * W;
            return __funnelshift_r(row[q6], row[q6n], sh6) & 0x3Fu;
          };
          // dilated rows D_d of band row r = OR of staged syndrome rows
          // r + 3 - d .. r + 3 + d, rolled down the band with the planes; the
          // four bits of D_d for the word sit at offset 3 - d (m^+) or d - 1 (m^-)
          uint32_t sg[7];
#pragma unroll
          for (int j = 0; j < 6; ++j) sg[j] = sig6(j);
          // rolling window over staged rows a(j): pair mins q, quad mins u,
          // out(r) = min(u(r), u(r + 3)) = min of staged rows r .. r + 6
          uint32_t ah[7], al[7];
#pragma unroll
          for (int j = 0; j < 6; ++j) {
            const uint32_t w = shifted(j);
            ah[j] = w & 0xFF00FF00u;
            al[j] = w & 0x00FF00FFu;
          }
          uint32_t qh[6], ql[6], uh[3], ul[3];
#pragma unroll
          for (int j = 0; j < 5; ++j) {
            qh[j] = __vminu2(ah[j], ah[j + 1]);
            ql[j] = __vminu2(al[j], al[j + 1]);
          }
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            uh[j] = __vminu2(qh[j], qh[j + 2]);
            ul[j] = __vminu2(ql[j], ql[j + 2]);
          }
          uint32_t lasth = ah[5], lastl = al[5];
#pragma unroll
          for (int r = 0; r < kTB; ++r) {
            // consume staged row r + 6: q(r + 5), u(r + 3), out(r)
            const uint32_t w = shifted(r + 6);
            const uint32_t h6 = w & 0xFF00FF00u, l6 = w & 0x00FF00FFu;
            const uint32_t q5h = __vminu2(lasth, h6), q5l = __vminu2(lastl, l6);
            const uint32_t u3h = __vminu2(qh[3], q5h), u3l = __vminu2(ql[3], q5l);
            const uint32_t mh = __vminu2(uh[0], u3h), ml = __vminu2(ul[0], u3l);
            // +3 saturating at 0xFF while each byte sits alone in a 16-bit lane:
            // clamp at 0xFC, then add (no carry leaves the lane)
            uint32_t v = (__vminu2(mh, 0xFC00FC00u) + 0x03000300u) |
                         (__vminu2(ml, 0x00FC00FCu) + 0x00030003u);
            // roll: q(r + 1 ..) and u(r + 1 ..)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              qh[j] = qh[j + 1];
              ql[j] = ql[j + 1];
            }
            qh[4] = q5h;
            ql[4] = q5l;
            uh[0] = uh[1];
            ul[0] = ul[1];
            uh[1] = uh[2];
            ul[1] = ul[2];
            uh[2] = u3h;
            ul[2] = u3l;
            lasth = h6;
            lastl = l6;
            // terms: the smallest d wins (d = 3 first, overwritten by smaller
            // d), and every term lies below every propagated value, so it
            // replaces it; D_3 contains D_2 and D_1, so if the six bits of D_3
            // are clear there is no term
            sg[6] = sig6(r + 6);
            const uint32_t d1 = sg[2] | sg[3] | sg[4];
            const uint32_t d2 = d1 | sg[1] | sg[5];
            const uint32_t d3 = d2 | sg[0] | sg[6];
#pragma unroll
            for (int j = 0; j < 6; ++j) sg[j] = sg[j + 1];
            if (d3) {
              const uint32_t dd[3] = {d1, d2, d3};
              uint32_t T = 0u, any = 0u;
#pragma unroll
              for (int d = 3; d >= 1; --d) {
                const int off = plus ? 3 - d : d - 1;
                const uint32_t m = nib_mask((dd[d - 1] >> off) & 0xFu);
                T = (T & ~m) | ((v1 + (uint32_t)(d - 1) * 0x01010101u) & m);
                any |= m;
              }
              v = (v & ~any) | (T & any);
            }
            out[(size_t)r * cols + kc] = v;
          }
        }
        // the band buffer is free again
        if (__syncthreads_or(!ok)) {
          aborted = true;
          break;
        }
      }
      fence_proxy_async_global();
      if (aborted && tid == 0) atomicOr(rank_ptr(&misc[5], 0), 1);
      cluster.sync();  // every plane of the new buffer is complete
      // ================= 2. forces and feedback for the anyons of own x-frame rows
      const int par = t & 1;
      if (!*rank_ptr(&misc[5], 0)) {
        const uint8_t* Ppx = plane(dst, 0);
        const uint8_t* Pmx = plane(dst, 1);
        const uint8_t* Ppy = plane(dst, 2);
        const uint8_t* Pmy = plane(dst, 3);
        const uint32_t* Sx = sigf(0);
        uint64_t kstep = 0, kbal = 0;
        if (a.move_thr) kstep = move_step_key(a.move_key, a.shot_offset + shot, t);
        if (a.balance_rule) kbal = move_step_key(a.balance_key, a.shot_offset + shot, t);
        // the sigma words of kMoveBatch rows are loaded before the first is
        // used (one global latency per batch instead of one per row)
        for (int rb = warp; rb < RL; rb += nw * kMoveBatch) {
          uint32_t words[kMoveBatch];
#pragma unroll
          for (int u = 0; u < kMoveBatch; ++u) {
            const int rr = rb + u * nw;
            words[u] = (rr < RL && lane < W) ? Sx[(size_t)(r0 + rr) * W + lane] : 0u;
          }
#pragma unroll
          for (int u = 0; u < kMoveBatch; ++u) {
          const int y = r0 + rb + u * nw, wq = lane;
          uint32_t bits = words[u];
          while (bits) {
            // up to four anyons of the word at a time: all sixteen field loads
            // are issued before the first one is used
            int xs[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              xs[k] = -1;
              if (bits) {
                xs[k] = wq * 32 + __ffs(bits) - 1;
                bits &= bits - 1;
              }
            }
            uint32_t f[4][4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const int x = xs[k] < 0 ? 0 : xs[k];
              f[k][0] = Ppx[(size_t)y * L + x];
              f[k][1] = Pmx[(size_t)y * L + x];
              f[k][2] = Ppy[(size_t)x * L + y];
              f[k][3] = Pmy[(size_t)x * L + y];
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              if (xs[k] < 0) continue;
              const int x = xs[k];
              // Eqs. blahdef / degbreak on the offset-encoded fields (0xFF = none)
              int dir = force_code(f[k][0], f[k][1], f[k][2], f[k][3], a.tie_order);
              if (dir >= 5)
                dir = a.balance_rule ? balance_resolve(dir, kbal, (int64_t)y * L + x) : 0;
              if (a.move_thr) {
                const uint64_t u = splitmix64(kstep ^ (uint64_t)((int64_t)y * L + x));
                if (u < a.move_thr) dir = 1 + (int)(splitmix64(u) >> 62);
              }
              if (!dir) continue;
              const int kind = (dir <= 2) ? 0 : 1;
              const int lx = (dir == 2) ? twrap(x - 1, L) : x;
              const int ly = (dir == 4) ? twrap(y - 1, L) : y;
              atomicOr(flip(par, 0, kind) + (size_t)ly * W + (lx >> 5), 1u << (lx & 31));
              atomicOr(flip(par, 1, kind) + (size_t)lx * W + (ly >> 5), 1u << (ly & 31));
            }
          }
          }
        }
      }
      cluster.sync();  // flipped-link maps complete
      // ================= 3. sigma and correction from the flipped links
      int cnt = 0;
      if (!*rank_ptr(&misc[5], 0)) {
        for (int fr = 0; fr < 2; ++fr) {
          // frame 0: rows y, kind 0 (x links) along the row, kind 1 (y links) across rows;
          // frame 1: rows x, kind 1 along the row, kind 0 across rows
          const uint32_t* Fa = flip(par, fr, fr == 0 ? 0 : 1);  // links along the row
          const uint32_t* Fc = flip(par, fr, fr == 0 ? 1 : 0);  // links across rows
          uint32_t* S = sigf(fr);
          // kSigBatch rows at a time: every load of the batch is issued
          // before the first store
          for (int rb = warp; rb < RL; rb += nw * kSigBatch) {
            uint32_t fa[kSigBatch], fc[kSigBatch], fcu[kSigBatch], sv[kSigBatch];
            uint32_t cx[kSigBatch], cy[kSigBatch];
#pragma unroll
            for (int u = 0; u < kSigBatch; ++u) {
              const int rr = rb + u * nw;
              const bool on = rr < RL && lane < W;
              const int R = r0 + (rr < RL ? rr : 0), Rm = twrap(R - 1, L);
              fa[u] = on ? Fa[(size_t)R * W + lane] : 0u;
              fc[u] = on ? Fc[(size_t)R * W + lane] : 0u;
              fcu[u] = on ? Fc[(size_t)Rm * W + lane] : 0u;
              sv[u] = on ? S[(size_t)R * W + lane] : 0u;
              cx[u] = (on && fr == 0) ? Cb[(size_t)R * W + lane] : 0u;
              cy[u] = (on && fr == 0) ? Cb[(size_t)L * W + (size_t)R * W + lane] : 0u;
            }
#pragma unroll
            for (int u = 0; u < kSigBatch; ++u) {
              const int rr = rb + u * nw;
              const bool on = rr < RL && lane < W;
              const int R = r0 + (rr < RL ? rr : 0);
              // e_a of the previous word of the row (wrapping at the row end)
              const uint32_t fa_prev = __shfl_sync(0xFFFFFFFFu, fa[u], lane == 0 ? W - 1 : lane - 1);
              const uint32_t along = fa[u] ^ ((fa[u] << 1) | (fa_prev >> 31));
              const uint32_t across = fc[u] ^ fcu[u];
              const uint32_t sn = sv[u] ^ along ^ across;
              if (on) {
                S[(size_t)R * W + lane] = sn;
                if (fr == 0) {
                  cnt += __popc(sn);
                  Cb[(size_t)R * W + lane] = cx[u] ^ fa[u];                 // x links
                  Cb[(size_t)L * W + (size_t)R * W + lane] = cy[u] ^ fc[u];  // y links
                }
              }
            }
          }
        }
        // the other parity's maps (read last step, written next step): clear own rows
        for (int fr = 0; fr < 2; ++fr)
          for (int kd = 0; kd < 2; ++kd) {
            uint32_t* F = flip(par ^ 1, fr, kd) + (size_t)r0 * W;
            fill_words(F, RL * W, 0u, tid, nt);
          }
      }
      for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
      if (lane == 0 && cnt) atomicAdd(rank_ptr(&misc[par], 0), cnt);
      fence_proxy_async_global();
      cluster.sync();
      ++t;
      any = *rank_ptr(&misc[par], 0);
      if (*rank_ptr(&misc[5], 0)) {
        aborted = true;
        flag = 3;
        break;
      }
      // rank 0 clears the counter of the next step (last read a step ago)
      if (rank == 0 && tid == 0) misc[par ^ 1] = 0;
    }
    if (aborted) {
      // copies may still be in flight: wait for them (bounded) before leaving
      if (tid == 0)
        for (int b2 = 0; b2 < 2; ++b2)
          if (inflight[b2]) (void)mbar_wait_bounded(&bar[b2], phase[b2]);
      __syncthreads();
      flag = 3;
    }
    // ================= outputs: correction bytes, homology, steps, flag
    uint8_t* outC = a.out_C + correction_offset_of(a, shot);
    for (int kd = 0; kd < 2; ++kd) {
      const uint32_t* C = Cb + (size_t)kd * L * W;
      for (int i = tid; i < RL * (L / 4); i += nt) {
        const int q = i / cols, y = r0 + q, x = (i - q * cols) * 4;
        const uint32_t nib = (C[(size_t)y * W + (x >> 5)] >> (x & 31)) & 0xFu;
        *reinterpret_cast<uint32_t*>(outC + (size_t)kd * LL + (size_t)y * L + x) =
            (nib * 0x00204081u) & 0x01010101u;
      }
    }
    int wx = 0, wy = 0;
    for (int y = r0 + tid; y < r0 + RL; y += nt) {  // e_x((0, y))
      wx ^= (int)(Cb[(size_t)y * W] & 1u);
      if (!a.from_sigma) wx ^= N[(size_t)y * L];
    }
    if (rank == 0) {
      for (int x = tid; x < L; x += nt) {  // e_y((x, 0))
        wy ^= (int)((Cb[(size_t)L * W + (x >> 5)] >> (x & 31)) & 1u);
        if (!a.from_sigma) wy ^= N[LL + x];
      }
    }
    wx = __reduce_xor_sync(0xFFFFFFFFu, wx);
    wy = __reduce_xor_sync(0xFFFFFFFFu, wy);
    if (lane == 0) {
      if (wx) atomicXor(rank_ptr(&misc[2], 0), 1);
      if (wy) atomicXor(rank_ptr(&misc[3], 0), 1);
    }
    cluster.sync();
    if (rank == 0 && tid == 0) {
      a.out_steps[shot] = t;
      if (a.from_sigma) {
        a.out_cut[2 * shot] = (uint8_t)misc[2];
        a.out_cut[2 * shot + 1] = (uint8_t)misc[3];
        if (a.out_exhausted) a.out_exhausted[shot] = (uint8_t)(flag == 2);
      } else {
        a.out_flag[shot] = (uint8_t)(flag >= 2 ? flag : ((misc[2] | misc[3]) ? 1 : 0));
      }
      misc[0] = misc[1] = misc[2] = misc[3] = 0;
    }
    cluster.sync();  // counters reset before the next shot's init
  }
  // no CTA leaves while a partner could still reach its shared memory
  cluster.sync();
}

}  // namespace

// ---------------------------------------------------------------- host ----

namespace {

// Kernel-path overrides per L (qca_set_kernel_path): -1 automatic.
int g_path_override[QCA_MAX_L + 1];
std::once_flag g_override_once;

void init_overrides() {
  for (int i = 0; i <= QCA_MAX_L; ++i) g_path_override[i] = -1;
}

bool tiled_geom(int L, int m_max, TiledGeom& g) {
  if (L % 128 != 0 || L < 128 || L > QCA_MAX_L || m_max < 3 || m_max > 255) return false;
  g.L = L;
  g.W = L / 32;
  g.RL = L / kTCL;
  g.cols = L / 4;
  g.off = 255 - m_max;
  const int TR = kTRows;
  g.LL = (size_t)L * L;
  const size_t bm = (size_t)L * g.W * 4;  // one bitmap, bytes
  g.o_sig = 8 * g.LL;
  g.o_flip = g.o_sig + 2 * bm;
  g.o_C = g.o_flip + 8 * bm;
  g.slot = ((g.o_C + 2 * bm) + 255) & ~(size_t)255;
  size_t o = 0;
  g.s_band = o;
  o += 2 * (size_t)TR * L;
  g.s_sband = o;
  o += 2 * (size_t)TR * g.W * 4;
  o = (o + 15) & ~(size_t)15;
  g.s_bar = o;
  o += 16;
  g.s_misc = o;
  o += 64;
  g.smem = o;
  return true;
}

struct TiledWorkspace {
  uint8_t* ptr = nullptr;
  size_t bytes = 0;
  cudaEvent_t done = nullptr;
};
std::mutex g_tws_mu;
TiledWorkspace g_tws[64];

struct TiledShape {
  int dev;
  size_t smem;
  int clusters;
};
std::mutex g_tshape_mu;
std::vector<TiledShape> g_tshapes;

}  // namespace

int tiled_path_for(int L, int v, int m_max) {
  std::call_once(g_override_once, init_overrides);
  if (v != 3) return 0;
  TiledGeom g;
  if (!tiled_geom(L, m_max, g)) return 0;
  const int ov = g_path_override[L];
  if (ov == 3) return 1;
  if (ov == 0) return 0;
  return L > 256 ? 1 : 0;
}

int generic_forced(int L) {
  std::call_once(g_override_once, init_overrides);
  return (L >= 3 && L <= QCA_MAX_L && g_path_override[L] == 0) ? 1 : 0;
}

int launch_tiled(const DecodeArgs& a, cudaStream_t stream) {
  if (a.shots == 0) return QCA_OK;
  TiledGeom g;
  if (a.v != 3 || !tiled_geom(a.L, a.m_max, g)) {
    set_error("no tiled kernel for L=%d v=%d m_max=%d", a.L, a.v, a.m_max);
    return QCA_ERR_UNSUPPORTED;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) {
    set_error("device index %d out of range", dev);
    return QCA_ERR_UNSUPPORTED;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kTCL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.blockDim = dim3(kTThreads);
  cfg.dynamicSmemBytes = g.smem;
  cfg.stream = stream;
  auto kern = tiled_kernel;
  int clusters = -1;
  {
    std::lock_guard<std::mutex> lk(g_tshape_mu);
    for (const TiledShape& s : g_tshapes)
      if (s.dev == dev && s.smem == g.smem) clusters = s.clusters;
  }
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)g.smem);
  if (e != cudaSuccess) return cuda_fail(e, "tiled sweep smem attribute");
  if (clusters < 0) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cfg.gridDim = dim3((unsigned)(kTCL * sms));
    e = cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg);
    if (e != cudaSuccess) return cuda_fail(e, "tiled cluster occupancy query");
    if (clusters < 1) {
      set_error("tiled sweep cluster does not fit (L=%d)", a.L);
      return QCA_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_tshape_mu);
    g_tshapes.push_back({dev, g.smem, clusters});
  }
  int64_t grid = clusters;
  if (grid > a.shots) grid = a.shots;
  const size_t need = g.slot * (size_t)grid;
  std::lock_guard<std::mutex> lk(g_tws_mu);
  TiledWorkspace& w = g_tws[dev];
  if (w.bytes < need) {
    // the previous workspace may still be in use by queued work on any stream
    if (w.ptr) {
      e = cudaDeviceSynchronize();
      if (e != cudaSuccess) return cuda_fail(e, "synchronise before workspace growth");
      cudaFree(w.ptr);
      w.ptr = nullptr;
      w.bytes = 0;
    }
    e = cudaMalloc(&w.ptr, need);
    if (e != cudaSuccess) return cuda_fail(e, "tiled workspace allocation");
    w.bytes = need;
  }
  if (!w.done) {
    e = cudaEventCreateWithFlags(&w.done, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "event creation");
  }
  // launches on different streams share the workspace: order them
  e = cudaStreamWaitEvent(stream, w.done, 0);
  if (e != cudaSuccess) return cuda_fail(e, "stream wait");
  cfg.gridDim = dim3((unsigned)(grid * kTCL));
  e = cudaLaunchKernelEx(&cfg, kern, a, g, w.ptr);
  if (e != cudaSuccess) return cuda_fail(e, "tiled sweep launch");
  return cuda_fail(cudaEventRecord(w.done, stream), "event record");
}

int tiled_workspace_release() {
  std::lock_guard<std::mutex> lk(g_tws_mu);
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !g_tws[dev].ptr) return QCA_OK;
  cudaError_t e = cudaFree(g_tws[dev].ptr);
  g_tws[dev].ptr = nullptr;
  g_tws[dev].bytes = 0;
  return cuda_fail(e, "tiled workspace free");
}

}  // namespace qca

using namespace qca;

extern "C" int qca_set_kernel_path(int L, int path) {
  std::call_once(g_override_once, init_overrides);
  if (L < 3 || L > QCA_MAX_L || (path != -1 && path != 0 && path != 3)) {
    set_error("qca_set_kernel_path: L=%d path=%d (allowed: -1 automatic, 0 generic, 3 tiled)", L,
              path);
    return QCA_ERR_ARG;
  }
  TiledGeom g;
  if (path == 3 && !tiled_geom(L, 255, g)) {
    set_error("qca_set_kernel_path: the tiled kernel needs L a multiple of 128 (L=%d)", L);
    return QCA_ERR_UNSUPPORTED;
  }
  g_path_override[L] = path;
  return QCA_OK;
}
