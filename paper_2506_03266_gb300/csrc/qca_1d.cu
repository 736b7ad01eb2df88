// 1D message-passing automaton decoder for the repetition code on a ring
// (Sec. 3.1, Def. "message passing automaton, 1D"; Sec. 7.1 numerics).
//
// One CTA decodes one shot at a time with the whole state in shared memory:
// the fields m^+ and m^- as bytes in the offset encoding w = m - 1 + (255 -
// m_max) (0xFF = no message; double-buffered), sigma, the correction and the
// per-site move.  One step:
//   1. v applications of A^(1), fused exactly: with sigma fixed,
//        w_v(r) = nearest anyon at r - s d, d <= v ?  (d <= m_max ? off + d - 1 : 0xFF)
//                                             :  satadd(w_0(r - s v), v)
//      (s = +1 for m^+, -1 for m^-; the anyon nearest upstream overwrites
//      every older message, and an unbroken chain of v increments carries the
//      old value, vanishing above m_max);
//   2. forces f_r = sgn(-m^+ + m^-) with an empty field as +infinity (an
//      anyon moves toward the smaller field; none on a tie), or a random
//      direction with probability p_move;
//   3. feedback: link <r, r+1> flips iff the anyon at r moves right or the
//      anyon at r+1 moves left (the OR); C ^= F, sigma updated.
// A thread decides the moves of its own sites right after their fields, so a
// step takes three block barriers.
// After the last step N xor C is constant on the ring; its value is the
// decoded logical value.
#include "qca_internal.cuh"

namespace qca {

namespace {

constexpr uint64_t kTagNoise1D = 0x4E4F49534531ULL;  // "NOISE1"
constexpr int k1DThreads = 128;

__global__ void sample_1d_kernel(int L, int64_t shot0, int64_t shots, uint64_t thr, uint64_t seed,
                                 uint8_t* __restrict__ out) {
  const uint64_t k = splitmix64(seed ^ kTagNoise1D);
  const int64_t n = shots * (int64_t)L;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = i / L;
    const int r = (int)(i - s * L);
    const uint64_t ks = splitmix64(k ^ (uint64_t)(shot0 + s));
    out[i] = splitmix64(ks ^ (uint64_t)r) < thr ? 1 : 0;
  }
}

struct Args1D {
  const uint8_t* in;
  int L;
  int64_t shots;
  int max_steps;
  int v;
  int m_max;
  uint64_t move_thr;
  uint64_t move_key;
  int64_t shot_offset;
  uint8_t* out_C;
  int32_t* out_steps;
  uint8_t* out_flag;
  uint8_t* out_maj;
};

// i mod L: one correction covers every offset of a ring of at least 8 sites
// (offsets are at most v = 8); shorter rings take the remainder
__device__ __forceinline__ int rwrap(int i, int L) {
  if (i < 0) {
    i += L;
  } else if (i >= L) {
    i -= L;
  }
  if (i < 0 || i >= L) {
    i %= L;
    if (i < 0) i += L;
  }
  return i;
}

__global__ void __launch_bounds__(k1DThreads) decode_1d_kernel(Args1D a) {
  extern __shared__ __align__(16) uint8_t sm[];
  const int L = a.L, tid = threadIdx.x, nt = blockDim.x;
  uint8_t* wbuf = sm;            // [2 buffers][2 fields][L]
  uint8_t* sig = sm + 4 * L;     // 1 = anyon
  uint8_t* C = sig + L;
  uint8_t* mv = C + L;           // per-site move: 0 none, 1 right, 2 left
  uint8_t* F = mv + L;           // link <r, r + 1> flipped this step
  const int off = 255 - a.m_max, v = a.v;
  const int reach = v < a.m_max ? v : a.m_max;  // terms d <= reach are representable
  for (int64_t shot = blockIdx.x; shot < a.shots; shot += gridDim.x) {
    const uint8_t* N = a.in + shot * L;
    int cnt = 0, weight = 0;
    for (int r = tid; r < L; r += nt) {
      const uint8_t s = N[rwrap(r - 1, L)] ^ N[r];
      sig[r] = s;
      C[r] = 0;
      wbuf[r] = 0xFF;
      wbuf[L + r] = 0xFF;
      cnt += s;
      weight += N[r];
    }
    int any = __syncthreads_count(cnt > 0);
    int t = 0, flag = 0, cur = 0;
    while (any) {
      if (t >= a.max_steps) {
        flag = 2;
        break;
      }
      // 1. fused v sub-steps of A^(1) for both fields of the thread's sites,
      // 2. and at once the move of an anyon there (it reads only its own site)
      const uint8_t* w0 = wbuf + cur * 2 * L;
      uint8_t* w1 = wbuf + (cur ^ 1) * 2 * L;
      uint64_t kstep = 0;
      if (a.move_thr) kstep = move_step_key(a.move_key, a.shot_offset + shot, t);
      for (int r = tid; r < L; r += nt) {
        uint32_t wk[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const int s = k == 0 ? 1 : -1;
          int d = 1;
          for (; d <= v; ++d)
            if (sig[rwrap(r - s * d, L)]) break;
          uint32_t out;
          if (d <= v) {
            out = d <= reach ? (uint32_t)(off + d - 1) : 0xFFu;
          } else {
            const uint32_t old = w0[k * L + rwrap(r - s * v, L)];
            out = old + (uint32_t)v > 0xFEu ? 0xFFu : old + (uint32_t)v;
          }
          w1[k * L + r] = (uint8_t)out;
          wk[k] = out;
        }
        uint8_t m = 0;
        if (sig[r]) {
          const uint32_t wp = wk[0], wm = wk[1];
          m = wm < wp ? 1 : (wp < wm ? 2 : 0);  // toward the smaller field; 0xFF = none
          if (a.move_thr) {
            const uint64_t u = splitmix64(kstep ^ (uint64_t)r);
            if (u < a.move_thr) m = (splitmix64(u) >> 63) == 0 ? 1 : 2;
          }
        }
        mv[r] = m;
      }
      cur ^= 1;
      __syncthreads();
      // 3. feedback (OR) and correction
      for (int r = tid; r < L; r += nt) {
        const uint8_t f = (mv[r] == 1 || mv[rwrap(r + 1, L)] == 2) ? 1 : 0;
        F[r] = f;
        C[r] ^= f;
      }
      __syncthreads();
      cnt = 0;
      for (int r = tid; r < L; r += nt) {
        const uint8_t s = sig[r] ^ F[rwrap(r - 1, L)] ^ F[r];
        sig[r] = s;
        cnt += s;
      }
      any = __syncthreads_count(cnt > 0);
      ++t;
    }
    // outputs
    uint8_t* outC = a.out_C + shot * L;
    for (int r = tid; r < L; r += nt) outC[r] = C[r];
    // weight of N (block sum) for the majority vote
    __shared__ int wsum;
    if (tid == 0) wsum = 0;
    __syncthreads();
    atomicAdd(&wsum, weight);
    __syncthreads();
    if (tid == 0) {
      const int value = (N[0] ^ C[0]) & 1;
      const int majority = 2 * wsum > L ? 1 : 0;
      a.out_steps[shot] = t;
      a.out_flag[shot] = (uint8_t)(flag == 2 ? 2 : value);
      if (a.out_maj) a.out_maj[shot] = (uint8_t)(flag == 2 ? 2 : (value != majority));
    }
    __syncthreads();
  }
}

uint64_t thr_1d(double p) {
  if (!(p > 0.0)) return 0;
  if (p >= 1.0) return UINT64_MAX;
  const double t = floor(ldexp(p, 64));
  return t >= 18446744073709551615.0 ? UINT64_MAX : (uint64_t)t;
}

}  // namespace

}  // namespace qca

using namespace qca;

extern "C" {

int qca_sample_errors_1d_async(int L, int64_t shot0, int64_t shots, double p, uint64_t seed,
                               uint8_t* out_errors, void* stream) {
  if (L < 3 || L > QCA_MAX_L_1D || shots < 0 || shot0 < 0 || !(p >= 0.0 && p <= 1.0) ||
      (shots > 0 && !out_errors)) {
    set_error("qca_sample_errors_1d_async: bad arguments");
    return QCA_ERR_ARG;
  }
  if (shots == 0) return QCA_OK;
  const int64_t n = shots * (int64_t)L;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  sample_1d_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(L, shot0, shots, thr_1d(p),
                                                                       seed, out_errors);
  return cuda_fail(cudaGetLastError(), "1D sampler launch");
}

int qca_decode_1d_batch_async(const uint8_t* noise, int L, int64_t shots, int max_steps,
                              uint64_t rng_seed, const qca_config* cfg, uint8_t* out_correction,
                              int32_t* out_steps, uint8_t* out_flag, uint8_t* out_majority_flag,
                              void* stream) {
  qca_config c;
  qca_default_config(&c);
  if (cfg) c = *cfg;
  if (L < 3 || L > QCA_MAX_L_1D || shots < 0 || max_steps < 0 || max_steps > QCA_MAX_STEPS) {
    set_error("qca_decode_1d_batch_async: L=%d (3..%d), shots, max_steps out of range", L,
              QCA_MAX_L_1D);
    return QCA_ERR_ARG;
  }
  if (c.v < 1 || c.v > 8 || c.m_max < 1 || c.m_max > 255 || !(c.p_move >= 0.0 && c.p_move <= 1.0)) {
    set_error("qca_decode_1d_batch_async: v must be 1..8, m_max 1..255, p_move in [0, 1]");
    return QCA_ERR_UNSUPPORTED;
  }
  if (c.tie_order != QCA_TIE_LEX || c.balance_rule != QCA_BALANCE_STAY) {
    set_error("qca_decode_1d_batch_async: only the default tie order and balance rule");
    return QCA_ERR_UNSUPPORTED;
  }
  if (shots > 0 && (!noise || !out_correction || !out_steps || !out_flag)) {
    set_error("qca_decode_1d_batch_async: NULL array pointer");
    return QCA_ERR_ARG;
  }
  if (int rc = check_aligned(out_steps, 4, "qca_decode_1d_batch_async: out_steps")) return rc;
  if (shots == 0) return QCA_OK;
  Args1D a;
  a.in = noise;
  a.L = L;
  a.shots = shots;
  a.max_steps = max_steps;
  a.v = c.v;
  a.m_max = c.m_max;
  a.move_thr = thr_1d(c.p_move);
  a.move_key = splitmix64(rng_seed ^ kTagMove);
  a.shot_offset = c.shot_offset;
  a.out_C = out_correction;
  a.out_steps = out_steps;
  a.out_flag = out_flag;
  a.out_maj = out_majority_flag;
  const size_t smem = 8 * (size_t)L;
  cudaError_t e = cudaFuncSetAttribute(decode_1d_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "1D decode smem attribute");
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, decode_1d_kernel, k1DThreads, smem);
  if (e != cudaSuccess) return cuda_fail(e, "1D decode occupancy");
  int64_t grid = (int64_t)(per_sm > 0 ? per_sm : 1) * sms;
  if (grid > shots) grid = shots;
  decode_1d_kernel<<<(unsigned)grid, k1DThreads, smem, (cudaStream_t)stream>>>(a);
  return cuda_fail(cudaGetLastError(), "1D decode launch");
}

}  // extern "C"
