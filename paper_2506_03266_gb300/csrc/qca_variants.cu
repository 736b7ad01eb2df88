// Two variants of the 2D decoder, on a literal per-site sweep with the state in
// a per-CTA slot (one CTA per shot, grid-stride over shots): shared memory
// where the 14 L^2 bytes of a shot fit (L <= 85), else global memory:
//
//   OPEN   open boundaries (Appendix "Open boundary conditions", Def. "message
//          passing automaton with open boundaries"): an L x L grid without
//          wrap; the rough boundary B is the columns x = 0 and x = L-1.  The
//          qubits are e_x(x, y) for x <= L-2 and e_y(x, y) for 1 <= x <= L-2,
//          y <= L-2 (other entries of the arrays are ignored / left zero).
//          B holds no messages, sources m^{+x} (from x = 0) and m^{-x} (from
//          x = L-1) into the bulk, and absorbs anyons; cone members outside
//          the grid are dropped.  Failure: N xor C crosses the column cut
//          x = 0 | 1 an odd number of times.
//   DESYNC uncoordinated desynchronisation (Sec. 7.3) on the torus: per tick,
//          site r fires its message update with probability min(1, v q) and,
//          holding an anyon, its move with probability q, from counter draws
//          sm(sm(sm(sm(seed ^ "DESYNC") ^ shot) ^ tick) ^ (2 r + c)); the
//          firing updates of a tick apply together from the fields before the
//          tick, then the firing anyons move on the updated fields (OR
//          feedback), then sigma is updated.
//
// Forces follow readings R1-R4 as everywhere else (smallest field, ties
// (-,y) < (-,x) < (+,x) < (+,y), toward the smaller of the chosen axis' two
// fields, no move on a tie).
#include <mutex>

#include "qca_internal.cuh"

namespace qca {

namespace {

constexpr int kVThreads = 512;
constexpr size_t kVSmemSlot = 100 * 1024;  // largest per-shot state kept in shared memory
constexpr uint64_t kTagDesync = 0x444553594E43ULL;  // "DESYNC"

enum VariantMode { kOpen = 0, kDesync = 1 };

struct VariantArgs {
  const uint8_t* in;  // noise [shots][2][L][L]
  int L;
  int64_t shots;
  int max_steps;      // steps (OPEN) or ticks (DESYNC)
  int v;
  int m_max;
  uint64_t thr_msg, thr_move;  // DESYNC firing thresholds
  uint64_t key;                // DESYNC: splitmix64(seed ^ "DESYNC")
  int64_t shot_offset;
  uint8_t* out_C;
  int32_t* out_steps;
  uint8_t* out_flag;
};

__device__ __forceinline__ int vwrap(int i, int L) { return i < 0 ? i + L : (i >= L ? i - L : i); }

__device__ __forceinline__ int variant_dir(int mpx, int mmx, int mpy, int mmy) {
  const int val[4] = {mmy, mmx, mpx, mpy};  // preference order on equal values
  int best = -1, bv = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (val[i] > 0 && (best < 0 || val[i] < bv)) {
      best = i;
      bv = val[i];
    }
  if (best < 0) return 0;
  const bool yaxis = (best == 0 || best == 3);
  const int mp = yaxis ? mpy : mpx, mm = yaxis ? mmy : mmx;
  const unsigned up = mp ? (unsigned)mp : 0x7fffffffu, um = mm ? (unsigned)mm : 0x7fffffffu;
  if (up == um) return 0;
  if (up < um) return yaxis ? 4 : 2;
  return yaxis ? 3 : 1;
}

// qubit existence on the open lattice
__device__ __forceinline__ bool open_link(int L, int plane, int x, int y) {
  if (x < 0 || y < 0 || x >= L || y >= L) return false;
  return plane == 0 ? x <= L - 2 : (x >= 1 && x <= L - 2 && y <= L - 2);
}

// (x, y) of site i = threadIdx.x + k blockDim.x, stepped with one carry per
// iteration instead of a division (blockDim.x % L < L)
struct SitePos {
  int x, y, dx, dy, L;
  __device__ explicit SitePos(int L_) : L(L_) {
    x = (int)threadIdx.x % L;
    y = (int)threadIdx.x / L;
    dx = (int)blockDim.x % L;
    dy = (int)blockDim.x / L;
  }
  __device__ void next() {
    x += dx;
    y += dy;
    if (x >= L) {
      x -= L;
      ++y;
    }
  }
};

// ws == nullptr: the slot is this CTA's dynamic shared memory (small L)
template <int MODE>
__global__ void __launch_bounds__(kVThreads) variant_kernel(VariantArgs a, uint8_t* ws,
                                                           size_t slot_bytes) {
  extern __shared__ __align__(16) uint8_t vsm[];
  const int L = a.L;
  const int LL = L * L;
  uint8_t* slot = ws ? ws + (size_t)blockIdx.x * slot_bytes : vsm;
  uint8_t* mcur = slot;             // [4][L][L]
  uint8_t* mnxt = mcur + 4 * LL;    // [4][L][L]
  uint8_t* sig = mnxt + 4 * LL;     // [L][L] 1 = anyon
  uint8_t* Cc = sig + LL;           // [2][L][L]
  uint8_t* dir = Cc + 2 * LL;       // [L][L]
  uint8_t* fl = dir + LL;           // [L][L] bit0 e_x flipped, bit1 e_y flipped
  __shared__ int s_red;
  for (int64_t shot = blockIdx.x; shot < a.shots; shot += gridDim.x) {
    const uint8_t* N = a.in + shot * 2 * (int64_t)LL;
    int any = 0;
    SitePos pi(L);
    for (int i = threadIdx.x; i < LL; i += blockDim.x, pi.next()) {
      const int x = pi.x, y = pi.y;
      int s;
      if (MODE == kOpen) {
        s = 0;
        if (x != 0 && x != L - 1) {
          if (open_link(L, 0, x, y)) s ^= N[i];
          if (open_link(L, 0, x - 1, y)) s ^= N[i - 1];
          if (open_link(L, 1, x, y)) s ^= N[LL + i];
          if (open_link(L, 1, x, y - 1)) s ^= N[LL + i - L];
        }
      } else {
        s = N[i] ^ N[y * L + vwrap(x - 1, L)] ^ N[LL + i] ^ N[LL + vwrap(y - 1, L) * L + x];
      }
      sig[i] = (uint8_t)s;
      any |= s;
      mcur[i] = mcur[LL + i] = mcur[2 * LL + i] = mcur[3 * LL + i] = 0;
      Cc[i] = Cc[LL + i] = 0;
    }
    any = __syncthreads_or(any);
    const uint64_t k1 = MODE == kDesync ? splitmix64(a.key ^ (uint64_t)(a.shot_offset + shot)) : 0;
    int t = 0, flag = 0;
    while (any) {
      if (t >= a.max_steps) {
        flag = 2;
        break;
      }
      const uint64_t k2 = MODE == kDesync ? splitmix64(k1 ^ (uint64_t)(uint32_t)t) : 0;
      // ---- message sub-steps: v per step (OPEN), one at the firing sites (DESYNC)
      const int subs = MODE == kOpen ? a.v : 1;
      for (int k = 0; k < subs; ++k) {
        SitePos pm(L);
        for (int i = threadIdx.x; i < LL; i += blockDim.x, pm.next()) {
          const int x = pm.x, y = pm.y;
          bool fire = true;
          if (MODE == kDesync) fire = splitmix64(k2 ^ (uint64_t)(2 * (int64_t)i)) < a.thr_msg;
#pragma unroll
          for (int f = 0; f < 4; ++f) {
            if (!fire) {
              mnxt[f * LL + i] = mcur[f * LL + i];
              continue;
            }
            const int s = (f % 2 == 0) ? 1 : -1;
            const bool ax = f < 2;
            int nv = 0;
            if (MODE == kOpen) {
              if (x == 0 || x == L - 1) {
                nv = 0;  // the rough boundary holds no messages
              } else {
                const int ux = ax ? x - s : x, uy = ax ? y : y - s;
                if (ux < 0 || ux >= L || uy < 0 || uy >= L) {
                  nv = 0;
                } else if (ax && (ux == 0 || ux == L - 1)) {
                  nv = 1;  // the boundary sources messages into the bulk
                } else {
                  int anyon = 0, best = 0;
#pragma unroll
                  for (int j = -1; j <= 1; ++j) {
                    const int xx = ax ? ux : ux + j, yy = ax ? uy + j : uy;
                    if (xx < 0 || xx >= L || yy < 0 || yy >= L) continue;
                    const int idx = yy * L + xx;
                    anyon |= sig[idx];
                    const int val = mcur[f * LL + idx];
                    if (val > 0 && (best == 0 || val < best)) best = val;
                  }
                  nv = anyon ? 1 : (best ? best + 1 : 0);
                }
              }
            } else {
              const int ux = ax ? vwrap(x - s, L) : x, uy = ax ? y : vwrap(y - s, L);
              int anyon = 0, best = 0;
#pragma unroll
              for (int j = -1; j <= 1; ++j) {
                const int xx = ax ? ux : vwrap(ux + j, L), yy = ax ? vwrap(uy + j, L) : uy;
                const int idx = yy * L + xx;
                anyon |= sig[idx];
                const int val = mcur[f * LL + idx];
                if (val > 0 && (best == 0 || val < best)) best = val;
              }
              nv = anyon ? 1 : (best ? best + 1 : 0);
            }
            if (nv > a.m_max) nv = 0;
            mnxt[f * LL + i] = (uint8_t)nv;
          }
        }
        __syncthreads();
        uint8_t* tmp = mcur;
        mcur = mnxt;
        mnxt = tmp;
      }
      // ---- forces at the (firing) anyons
      for (int i = threadIdx.x; i < LL; i += blockDim.x) {
        int d = 0;
        if (sig[i]) {
          bool fire = true;
          if (MODE == kDesync) fire = splitmix64(k2 ^ (uint64_t)(2 * (int64_t)i + 1)) < a.thr_move;
          if (fire) d = variant_dir(mcur[i], mcur[LL + i], mcur[2 * LL + i], mcur[3 * LL + i]);
        }
        dir[i] = (uint8_t)d;
      }
      __syncthreads();
      // ---- feedback (OR) on the existing links
      SitePos pf(L);
      for (int i = threadIdx.x; i < LL; i += blockDim.x, pf.next()) {
        const int x = pf.x, y = pf.y;
        int fx, fy;
        if (MODE == kOpen) {
          fx = open_link(L, 0, x, y) ? ((dir[i] == 1) | (dir[i + 1] == 2)) : 0;
          fy = open_link(L, 1, x, y) ? ((dir[i] == 3) | (dir[i + L] == 4)) : 0;
        } else {
          fx = (dir[i] == 1) | (dir[y * L + vwrap(x + 1, L)] == 2);
          fy = (dir[i] == 3) | (dir[vwrap(y + 1, L) * L + x] == 4);
        }
        fl[i] = (uint8_t)(fx | (fy << 1));
        Cc[i] ^= (uint8_t)fx;
        Cc[LL + i] ^= (uint8_t)fy;
      }
      __syncthreads();
      // ---- syndrome update
      any = 0;
      SitePos ps(L);
      for (int i = threadIdx.x; i < LL; i += blockDim.x, ps.next()) {
        const int x = ps.x, y = ps.y;
        int s;
        if (MODE == kOpen) {
          if (x == 0 || x == L - 1) {
            s = 0;  // the boundary absorbs anyons
          } else {
            s = sig[i] ^ (fl[i] & 1) ^ (fl[i - 1] & 1) ^ (fl[i] >> 1) ^ (y > 0 ? fl[i - L] >> 1 : 0);
          }
        } else {
          s = sig[i] ^ (fl[i] & 1) ^ (fl[y * L + vwrap(x - 1, L)] & 1) ^ (fl[i] >> 1) ^
              (fl[vwrap(y - 1, L) * L + x] >> 1);
        }
        sig[i] = (uint8_t)s;
        any |= s;
      }
      any = __syncthreads_or(any);
      ++t;
    }
    // ---- outputs and failure flag
    uint8_t* outC = a.out_C + shot * 2 * (int64_t)LL;
    for (int i = threadIdx.x; i < 2 * LL; i += blockDim.x) outC[i] = Cc[i];
    if (threadIdx.x == 0) s_red = 0;
    __syncthreads();
    int w = 0;
    if (MODE == kOpen) {
      for (int y = threadIdx.x; y < L; y += blockDim.x) w ^= N[y * L] ^ Cc[y * L];  // e_x(0, y)
      if (w) atomicXor(&s_red, 1);
    } else {
      int wx = 0, wy = 0;
      for (int i = threadIdx.x; i < L; i += blockDim.x) {
        wx ^= N[i * L] ^ Cc[i * L];        // e_x((0, i))
        wy ^= N[LL + i] ^ Cc[LL + i];      // e_y((i, 0))
      }
      if (wx) atomicXor(&s_red, 1);
      if (wy) atomicXor(&s_red, 2);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      a.out_steps[shot] = t;
      a.out_flag[shot] = (uint8_t)(flag == 2 ? 2 : (s_red ? 1 : 0));
    }
    __syncthreads();
  }
}

struct VariantWorkspace {
  uint8_t* ptr = nullptr;
  size_t bytes = 0;
  cudaEvent_t done = nullptr;
};
std::mutex g_vws_mu;
VariantWorkspace g_vws[64];

uint64_t vthr(double p) {
  if (!(p > 0.0)) return 0;
  if (p >= 1.0) return UINT64_MAX;
  const double t = floor(ldexp(p, 64));
  return t >= 18446744073709551615.0 ? UINT64_MAX : (uint64_t)t;
}

int launch_variant(int mode, const VariantArgs& a, cudaStream_t stream) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (dev < 0 || dev >= 64) {
    set_error("device index %d out of range", dev);
    return QCA_ERR_UNSUPPORTED;
  }
  const size_t LL = (size_t)a.L * a.L;
  const size_t slot = ((14 * LL) + 255) & ~(size_t)255;
  if (slot <= kVSmemSlot) {
    // the whole state of a shot in shared memory: as many CTAs as fit
    auto kern = mode == kOpen ? variant_kernel<kOpen> : variant_kernel<kDesync>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kVSmemSlot);
    if (e != cudaSuccess) return cuda_fail(e, "variant smem attribute");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kVThreads, slot);
    if (e != cudaSuccess) return cuda_fail(e, "variant occupancy");
    int64_t grid = (int64_t)(per_sm > 0 ? per_sm : 1) * sms;
    if (grid > a.shots) grid = a.shots;
    kern<<<(unsigned)grid, kVThreads, slot, stream>>>(a, nullptr, slot);
    return cuda_fail(cudaGetLastError(), "variant sweep launch");
  }
  int64_t slots = (int64_t)sms * 4;
  const int64_t cap = (int64_t)((size_t(2) << 30) / slot);
  if (slots > cap) slots = cap;
  if (slots < 1) slots = 1;
  if (slots > a.shots) slots = a.shots;
  const size_t need = slot * (size_t)slots;
  std::lock_guard<std::mutex> lk(g_vws_mu);
  VariantWorkspace& w = g_vws[dev];
  cudaError_t e;
  if (w.bytes < need) {
    if (w.ptr) {
      e = cudaDeviceSynchronize();
      if (e != cudaSuccess) return cuda_fail(e, "synchronise before workspace growth");
      cudaFree(w.ptr);
      w.ptr = nullptr;
      w.bytes = 0;
    }
    e = cudaMalloc(&w.ptr, need);
    if (e != cudaSuccess) return cuda_fail(e, "variant workspace allocation");
    w.bytes = need;
  }
  if (!w.done) {
    e = cudaEventCreateWithFlags(&w.done, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "event creation");
  }
  e = cudaStreamWaitEvent(stream, w.done, 0);
  if (e != cudaSuccess) return cuda_fail(e, "stream wait");
  if (mode == kOpen)
    variant_kernel<kOpen><<<(unsigned)slots, kVThreads, 0, stream>>>(a, w.ptr, slot);
  else
    variant_kernel<kDesync><<<(unsigned)slots, kVThreads, 0, stream>>>(a, w.ptr, slot);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "variant sweep launch");
  return cuda_fail(cudaEventRecord(w.done, stream), "event record");
}

int variant_args(VariantArgs& a, const uint8_t* noise, int L, int64_t shots, int max_steps,
                 const qca_config* cfg, uint8_t* out_C, int32_t* out_steps, uint8_t* out_flag,
                 const char* who) {
  qca_config c;
  qca_default_config(&c);
  if (cfg) c = *cfg;
  if (L < 3 || L > QCA_MAX_L || shots < 0 || max_steps < 0 || max_steps > QCA_MAX_STEPS) {
    set_error("%s: L=%d, shots or max_steps out of range", who, L);
    return L > QCA_MAX_L ? QCA_ERR_UNSUPPORTED : QCA_ERR_ARG;
  }
  if (c.v < 1 || c.v > 8 || c.m_max < 1 || c.m_max > 255) {
    set_error("%s: v must be 1..8 and m_max 1..255", who);
    return QCA_ERR_UNSUPPORTED;
  }
  if (c.tie_order != QCA_TIE_LEX || c.balance_rule != QCA_BALANCE_STAY) {
    set_error("%s: only the default tie order and balance rule", who);
    return QCA_ERR_UNSUPPORTED;
  }
  if (shots > 0 && (!noise || !out_C || !out_steps || !out_flag)) {
    set_error("%s: NULL array pointer", who);
    return QCA_ERR_ARG;
  }
  if (int rc = check_aligned(out_steps, 4, "out_steps (or out_ticks)")) return rc;
  a.in = noise;
  a.L = L;
  a.shots = shots;
  a.max_steps = max_steps;
  a.v = c.v;
  a.m_max = c.m_max;
  a.thr_msg = a.thr_move = 0;
  a.key = 0;
  a.shot_offset = c.shot_offset;
  a.out_C = out_C;
  a.out_steps = out_steps;
  a.out_flag = out_flag;
  return QCA_OK;
}

}  // namespace

}  // namespace qca

using namespace qca;

extern "C" {

int qca_decode_open_batch_async(const uint8_t* noise, int L, int64_t shots, int max_steps,
                                const qca_config* cfg, uint8_t* out_correction,
                                int32_t* out_steps, uint8_t* out_logical_fail, void* stream) {
  VariantArgs a;
  int rc = variant_args(a, noise, L, shots, max_steps, cfg, out_correction, out_steps,
                        out_logical_fail, "qca_decode_open_batch_async");
  if (rc) return rc;
  if (cfg && cfg->p_move != 0.0) {
    set_error("qca_decode_open_batch_async: random moves are not defined on the open lattice");
    return QCA_ERR_UNSUPPORTED;
  }
  if (shots == 0) return QCA_OK;
  return launch_variant(kOpen, a, (cudaStream_t)stream);
}

int qca_decode_desync_batch_async(const uint8_t* noise, int L, int64_t shots, int max_ticks,
                                  double q, uint64_t rng_seed, const qca_config* cfg,
                                  uint8_t* out_correction, int32_t* out_ticks,
                                  uint8_t* out_logical_fail, void* stream) {
  VariantArgs a;
  int rc = variant_args(a, noise, L, shots, max_ticks, cfg, out_correction, out_ticks,
                        out_logical_fail, "qca_decode_desync_batch_async");
  if (rc) return rc;
  if (!(q >= 0.0 && q <= 1.0)) {
    set_error("qca_decode_desync_batch_async: q must lie in [0, 1]");
    return QCA_ERR_ARG;
  }
  if (cfg && cfg->p_move != 0.0) {
    set_error("qca_decode_desync_batch_async: random moves are not combined with desynchronisation");
    return QCA_ERR_UNSUPPORTED;
  }
  const double qm = a.v * q < 1.0 ? a.v * q : 1.0;
  a.thr_msg = vthr(qm);
  a.thr_move = vthr(q);
  a.key = splitmix64(rng_seed ^ kTagDesync);
  if (shots == 0) return QCA_OK;
  return launch_variant(kDesync, a, (cudaStream_t)stream);
}

}  // extern "C"
