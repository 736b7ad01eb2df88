// Generic synchronous sweep: any L in [3, QCA_MAX_L], any v and m_max.
//
// One CTA decodes one shot at a time (grid-stride over shots).  The automaton
// state lives in a per-CTA slot of a device workspace (HBM, mostly L2 hits):
// message fields double-buffered as bytes in plain encoding (0 = no message),
// the anyon indicator, the correction, the per-site move and the per-site
// flipped-link bits.  Each phase is a plain parallel loop over sites separated
// by __syncthreads, in the order of Def. "synchronous automaton decoder":
// v sub-steps of A^(D) (Def. Dd_msg_passing), forces (Eqs. blahdef, degbreak),
// feedback (Eq. ddfeedback), syndrome update; then the homology check.
//
// This kernel is the path for lattice sizes the on-chip kernels do not take
// (L not a multiple of 4, L > 256) and for options they do not implement.
#include <mutex>

#include "qca_internal.cuh"

namespace qca {

namespace {

constexpr int kThreads = 512;

__device__ __forceinline__ int wrapi(int i, int L) { return i < 0 ? i + L : (i >= L ? i - L : i); }

// Plain field value (0 = no message) in the encoding force_code takes.
__device__ __forceinline__ uint32_t enc(int m) { return (uint32_t)(m - 1) & 0xFFu; }

__global__ void __launch_bounds__(kThreads) sweep_generic_kernel(DecodeArgs a, uint8_t* ws,
                                                                 size_t slot_bytes) {
  const int L = a.L;
  const int LL = L * L;
  uint8_t* base = ws + (size_t)blockIdx.x * slot_bytes;
  uint8_t* mcur = base;              // [4][L][L]
  uint8_t* mnxt = mcur + 4 * LL;     // [4][L][L]
  uint8_t* sig = mnxt + 4 * LL;      // [L][L] 1 = anyon
  uint8_t* Cc = sig + LL;            // [2][L][L]
  uint8_t* dir = Cc + 2 * LL;        // [L][L]
  uint8_t* fl = dir + LL;            // [L][L] bit0: e_x flipped, bit1: e_y flipped
  __shared__ int s_red[2];

  __shared__ int64_t s_next;
  // static work (CTA b takes b, b + gridDim.x, ...) or a dynamic queue
  auto next_work = [&](int64_t prev) -> int64_t {
    if (!a.queue) return prev < 0 ? (int64_t)blockIdx.x : prev + gridDim.x;
    __syncthreads();
    if (threadIdx.x == 0) s_next = (int64_t)atomicAdd(a.queue, 1u);
    __syncthreads();
    return s_next;
  };
  for (int64_t k = next_work(-1); k < a.shots; k = next_work(k)) {
    const int64_t shot = a.shot_list ? (int64_t)a.shot_list[k] : k;
    const int64_t base = shot_offset_of(a, shot);
    const uint8_t* in = a.in + base;
    int any = 0;
    for (int i = threadIdx.x; i < LL; i += blockDim.x) {
      const int x = i % L, y = i / L;
      uint8_t s;
      if (a.from_sigma) {
        s = in[i] ? 1 : 0;
      } else {
        // Def. synch_ccqs: parity of the four links incident to r.
        s = in[i] ^ in[y * L + wrapi(x - 1, L)] ^ in[LL + i] ^ in[LL + wrapi(y - 1, L) * L + x];
      }
      sig[i] = s;
      any |= s;
      mcur[i] = mcur[LL + i] = mcur[2 * LL + i] = mcur[3 * LL + i] = 0;
      Cc[i] = Cc[LL + i] = 0;
    }
    any = __syncthreads_or(any);
    int t = 0, flag = 0;
    while (any) {
      if (t >= a.max_steps) {
        flag = 2;
        break;
      }
      // ---- v sub-steps of A^(D), sigma fixed
      for (int k = 0; k < a.v; ++k) {
        for (int i = threadIdx.x; i < LL; i += blockDim.x) {
          const int x = i % L, y = i / L;
#pragma unroll
          for (int f = 0; f < 4; ++f) {
            // f: 0 (+,x) 1 (-,x) 2 (+,y) 3 (-,y); upstream centre r - s a^
            const int s = (f % 2 == 0) ? 1 : -1;
            const bool ax = f < 2;
            const int ux = ax ? wrapi(x - s, L) : x;
            const int uy = ax ? y : wrapi(y - s, L);
            int anyon = 0, best = 0;
#pragma unroll
            for (int j = -1; j <= 1; ++j) {
              const int xx = ax ? ux : wrapi(ux + j, L);
              const int yy = ax ? wrapi(uy + j, L) : uy;
              const int idx = yy * L + xx;
              anyon |= sig[idx];
              const int val = mcur[f * LL + idx];
              if (val > 0 && (best == 0 || val < best)) best = val;
            }
            int nv = anyon ? 1 : (best ? best + 1 : 0);
            if (nv > a.m_max) nv = 0;
            mnxt[f * LL + i] = (uint8_t)nv;
          }
        }
        __syncthreads();
        uint8_t* tmp = mcur;
        mcur = mnxt;
        mnxt = tmp;
      }
      // ---- forces at anyon sites
      uint64_t kstep = 0, kbal = 0;
      if (a.move_thr) kstep = move_step_key(a.move_key, a.shot_offset + shot, t);
      if (a.balance_rule) kbal = move_step_key(a.balance_key, a.shot_offset + shot, t);
      for (int i = threadIdx.x; i < LL; i += blockDim.x) {
        int d = 0;
        if (sig[i]) {
          // Eqs. blahdef / degbreak; codes 1 +x, 2 -x, 3 +y, 4 -y, 5 / 6 balanced
          d = force_code(enc(mcur[i]), enc(mcur[LL + i]), enc(mcur[2 * LL + i]),
                         enc(mcur[3 * LL + i]), a.tie_order);
          if (d >= 5) d = a.balance_rule ? balance_resolve(d, kbal, i) : 0;
          if (a.move_thr) {
            const uint64_t u = splitmix64(kstep ^ (uint64_t)i);
            if (u < a.move_thr) d = 1 + (int)(splitmix64(u) >> 62);
          }
        }
        dir[i] = (uint8_t)d;
      }
      __syncthreads();
      // ---- feedback: link <r, r+a^> flips iff r moves +a or r+a^ moves -a (OR)
      for (int i = threadIdx.x; i < LL; i += blockDim.x) {
        const int x = i % L, y = i / L;
        const int fx = (dir[i] == 1) | (dir[y * L + wrapi(x + 1, L)] == 2);
        const int fy = (dir[i] == 3) | (dir[wrapi(y + 1, L) * L + x] == 4);
        fl[i] = (uint8_t)(fx | (fy << 1));
        Cc[i] ^= (uint8_t)fx;
        Cc[LL + i] ^= (uint8_t)fy;
      }
      __syncthreads();
      // ---- syndrome update sigma <- sigma * sigma_F
      any = 0;
      for (int i = threadIdx.x; i < LL; i += blockDim.x) {
        const int x = i % L, y = i / L;
        const int s = sig[i] ^ (fl[i] & 1) ^ (fl[y * L + wrapi(x - 1, L)] & 1) ^ (fl[i] >> 1) ^
                      (fl[wrapi(y - 1, L) * L + x] >> 1);
        sig[i] = (uint8_t)s;
        any |= s;
      }
      any = __syncthreads_or(any);
      ++t;
    }
    // ---- outputs and homology (cut parities of N xor C, or of C alone)
    uint8_t* outC = a.out_C + correction_offset_of(a, shot);
    int wx = 0, wy = 0;
    for (int i = threadIdx.x; i < 2 * LL; i += blockDim.x) outC[i] = Cc[i];
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
      wx ^= Cc[i * L];       // e_x((0, i))
      wy ^= Cc[LL + i];      // e_y((i, 0))
      if (!a.from_sigma) {
        wx ^= in[i * L];
        wy ^= in[LL + i];
      }
    }
    if (threadIdx.x == 0) s_red[0] = s_red[1] = 0;
    __syncthreads();
    if (wx) atomicXor(&s_red[0], 1);
    if (wy) atomicXor(&s_red[1], 1);
    __syncthreads();
    if (threadIdx.x == 0) {
      a.out_steps[shot] = t;
      if (a.from_sigma) {
        a.out_cut[2 * shot] = (uint8_t)s_red[0];
        a.out_cut[2 * shot + 1] = (uint8_t)s_red[1];
        if (a.out_exhausted) a.out_exhausted[shot] = (uint8_t)(flag == 2);
      } else {
        a.out_flag[shot] = (uint8_t)(flag == 2 ? 2 : ((s_red[0] | s_red[1]) ? 1 : 0));
      }
    }
    __syncthreads();
  }
}

// Workspace cache: one per device, grown on demand.
struct Workspace {
  uint8_t* ptr = nullptr;
  size_t bytes = 0;
  cudaEvent_t done = nullptr;  // recorded after the last launch that used ptr
};
std::mutex g_ws_mu;
Workspace g_ws[64];

}  // namespace

int generic_workspace_release() {
  std::lock_guard<std::mutex> lk(g_ws_mu);
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return QCA_OK;
  if (g_ws[dev].ptr) {
    cudaError_t e = cudaFree(g_ws[dev].ptr);
    g_ws[dev].ptr = nullptr;
    g_ws[dev].bytes = 0;
    return cuda_fail(e, "workspace free");
  }
  return QCA_OK;
}

int launch_generic(const DecodeArgs& a, cudaStream_t stream) {
  if (a.shots == 0) return QCA_OK;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (dev < 0 || dev >= 64) {
    set_error("device index %d out of range", dev);
    return QCA_ERR_UNSUPPORTED;
  }
  const size_t LL = (size_t)a.L * a.L;
  const size_t slot = ((14 * LL) + 255) & ~(size_t)255;
  // Slots: enough CTAs to fill the GPU, capped so the workspace stays <= 2 GiB.
  int64_t slots = (int64_t)sms * 4;
  const int64_t cap = (int64_t)((size_t(2) << 30) / slot);
  if (slots > cap) slots = cap;
  if (slots < 1) slots = 1;
  if (slots > a.shots) slots = a.shots;
  const size_t need = slot * (size_t)slots;
  uint8_t* ws = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_ws_mu);
    if (g_ws[dev].bytes < need) {
      // The previous workspace may still be in use by queued work on any
      // stream: wait for the device before releasing it.
      if (g_ws[dev].ptr) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(e, "synchronise before workspace growth");
        cudaFree(g_ws[dev].ptr);
        g_ws[dev].ptr = nullptr;
        g_ws[dev].bytes = 0;
      }
      cudaError_t e = cudaMalloc(&g_ws[dev].ptr, need);
      if (e != cudaSuccess) return cuda_fail(e, "workspace allocation");
      g_ws[dev].bytes = need;
    }
    ws = g_ws[dev].ptr;
    if (!g_ws[dev].done) {
      cudaError_t e = cudaEventCreateWithFlags(&g_ws[dev].done, cudaEventDisableTiming);
      if (e != cudaSuccess) return cuda_fail(e, "event creation");
    }
    // Launches on different streams share the workspace: order them.
    cudaError_t e = cudaStreamWaitEvent(stream, g_ws[dev].done, 0);
    if (e != cudaSuccess) return cuda_fail(e, "stream wait");
    sweep_generic_kernel<<<(unsigned)slots, kThreads, 0, stream>>>(a, ws, slot);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "generic sweep launch");
    return cuda_fail(cudaEventRecord(g_ws[dev].done, stream), "event record");
  }
}

// ---------------------------------------------------------------------------
// Decoding without any allocation.  The per-shot state of the generic sweep
// lives in this fixed array instead of the cached workspace.  Every GPU that
// loads the library holds the array until the process exits.  The sweep
// writes all state it reads (fields, syndrome, correction, move and flip
// bytes) at the start of each shot, so the array needs no clearing between
// calls; it keeps whatever the last call left in it.
static __device__ __align__(256) uint8_t g_noalloc_scratch[QCA_NOALLOC_SCRATCH_BYTES];

namespace {
// Device address of g_noalloc_scratch, looked up once per device.
std::mutex g_noalloc_mu;
uint8_t* g_noalloc_ptr[64] = {};
}  // namespace

size_t noalloc_slot_bytes(int L) {
  const size_t LL = (size_t)L * L;
  return ((14 * LL) + 255) & ~(size_t)255;
}

int launch_generic_noalloc(const DecodeArgs& a, cudaStream_t stream) {
  const size_t slot = noalloc_slot_bytes(a.L);
  if (slot > (size_t)QCA_NOALLOC_SCRATCH_BYTES) {
    set_error("L = %d needs %zu bytes of decoder state per shot, more than the %d-byte "
              "fixed scratch of the no-allocation entry point",
              a.L, slot, QCA_NOALLOC_SCRATCH_BYTES);
    return QCA_ERR_UNSUPPORTED;
  }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) {
    set_error("device index %d out of range", dev);
    return QCA_ERR_UNSUPPORTED;
  }
  uint8_t* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      // In host code the array's name only stands in for it; the kernel needs
      // the device address, valid on the current device.  The lookup loads the
      // module that holds the array; querying the kernel's attributes loads
      // the kernel too, so that a later call only launches.
      uint8_t* ptr = nullptr;
      e = cudaGetSymbolAddress(reinterpret_cast<void**>(&ptr), g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the no-allocation scratch");
      cudaFuncAttributes fa;
      e = cudaFuncGetAttributes(&fa, sweep_generic_kernel);
      if (e != cudaSuccess) return cuda_fail(e, "loading the no-allocation sweep kernel");
      g_noalloc_ptr[dev] = ptr;
    }
    scratch = g_noalloc_ptr[dev];
  }
  if (a.shots == 0) return QCA_OK;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(e, "SM count query");
  int64_t slots = (int64_t)(QCA_NOALLOC_SCRATCH_BYTES / slot);
  if (slots > (int64_t)sms * 4) slots = (int64_t)sms * 4;
  if (slots > a.shots) slots = a.shots;
  sweep_generic_kernel<<<(unsigned)slots, kThreads, 0, stream>>>(a, scratch, slot);
  return cuda_fail(cudaGetLastError(), "no-allocation sweep launch");
}

}  // namespace qca
