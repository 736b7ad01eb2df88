// Microbenchmarks of the two denominators of the sweep's roofline on the
// current device: the issue rate of the integer instructions the sweep is
// built from (16 x 2 unsigned min, three-input logic, 32-bit min) and the
// shared-memory load bandwidth.  Each kernel keeps every SM busy for tens of
// milliseconds with one instruction written as inline PTX: eight chains per
// thread, each chain's next operand being its neighbour's current value, so
// that no chain is constant or idempotent and none can be folded.  The grid
// is exactly one wave of resident CTAs; thread 0 of every CTA reads the SM
// clock and the global timer around the timed loop, which gives the rates per
// SM and clock as well as the SM clock itself.
#include <algorithm>
#include <vector>

#include "qca_internal.cuh"

namespace qca {

namespace {

constexpr int kProbeThreads = 512;
constexpr int kChains = 8;
constexpr int kSmemProbeBytes = 32768;

enum ProbeOp { kOpMin16x2 = 0, kOpLop3 = 1, kOpMinU32 = 2 };

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// times[2 * cta] = SM cycles of the timed loop, times[2 * cta + 1] = its ns.
template <int OP>
__global__ void __launch_bounds__(kProbeThreads, 4) probe_alu_kernel(int iters, uint32_t seed,
                                                                  uint32_t* sink,
                                                                  unsigned long long* times) {
  uint32_t x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c)
    x[c] = (seed + 0x9E3779B9u * (uint32_t)(c + 1)) ^ (threadIdx.x * 0x85EBCA6Bu) ^ blockIdx.x;
  __syncthreads();
  const long long c0 = clock64();
  const uint64_t t0 = global_ns();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) {
        const uint32_t a = x[(c + 1) % kChains], b = x[(c + 2) % kChains];
        if constexpr (OP == kOpMin16x2)
          asm volatile("min.u16x2 %0, %0, %1;" : "+r"(x[c]) : "r"(a));
        else if constexpr (OP == kOpLop3)
          asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(x[c]) : "r"(a), "r"(b));
        else
          asm volatile("min.u32 %0, %0, %1;" : "+r"(x[c]) : "r"(a));
      }
    }
  }
  __syncthreads();
  const long long c1 = clock64();
  const uint64_t t1 = global_ns();
  uint32_t r = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) r ^= x[c];
  if (r == (seed ^ 0x5BD1E995u)) sink[blockIdx.x] = r;  // keeps the chains live
  if (threadIdx.x == 0) {
    times[2 * blockIdx.x] = (unsigned long long)(c1 - c0);
    times[2 * blockIdx.x + 1] = (unsigned long long)(t1 - t0);
  }
}

// Every warp instruction loads 512 contiguous bytes (16 per lane): four
// 128-byte wavefronts, free of bank conflicts.  The loads are volatile: the
// buffer does not change inside the loop, so plain loads would be hoisted.
__global__ void __launch_bounds__(kProbeThreads, 2) probe_smem_kernel(int iters, uint32_t seed,
                                                                   uint32_t* sink,
                                                                   unsigned long long* times) {
  __shared__ __align__(16) uint32_t buf[kSmemProbeBytes / 4];
  for (int i = threadIdx.x; i < kSmemProbeBytes / 4; i += blockDim.x)
    buf[i] = seed ^ ((uint32_t)i * 0x9E3779B9u);
  __syncthreads();
  // lane address within the first 8 KB; the eight loads of an iteration add
  // immediate offsets 0, 2 KB, ..., 14 KB, all inside the 32 KB buffer
  const uint32_t addr = (uint32_t)__cvta_generic_to_shared(buf) +
                        (uint32_t)((threadIdx.x >> 5) * 512 + (threadIdx.x & 31) * 16);
  uint32_t acc0 = 0, acc1 = 0, acc2 = 0, acc3 = 0;
#define QCA_PROBE_LD(OFF)                                                        \
  {                                                                              \
    uint32_t a, b, c, d;                                                         \
    asm volatile("ld.volatile.shared.v4.u32 {%0, %1, %2, %3}, [%4+" #OFF "];"   \
                 : "=r"(a), "=r"(b), "=r"(c), "=r"(d)                            \
                 : "r"(addr));                                                   \
    acc0 ^= a;                                                                   \
    acc1 ^= b;                                                                   \
    acc2 ^= c;                                                                   \
    acc3 ^= d;                                                                   \
  }
  const long long c0 = clock64();
  const uint64_t t0 = global_ns();
  for (int i = 0; i < iters; ++i) {
    QCA_PROBE_LD(0) QCA_PROBE_LD(2048) QCA_PROBE_LD(4096) QCA_PROBE_LD(6144)
    QCA_PROBE_LD(8192) QCA_PROBE_LD(10240) QCA_PROBE_LD(12288) QCA_PROBE_LD(14336)
  }
#undef QCA_PROBE_LD
  __syncthreads();
  const long long c1 = clock64();
  const uint64_t t1 = global_ns();
  const uint32_t r = acc0 ^ acc1 ^ acc2 ^ acc3;
  if (r == (seed ^ 0x5BD1E995u)) sink[blockIdx.x] = r;
  if (threadIdx.x == 0) {
    times[2 * blockIdx.x] = (unsigned long long)(c1 - c0);
    times[2 * blockIdx.x + 1] = (unsigned long long)(t1 - t0);
  }
}

struct ProbeRun {
  double ms = 0;          // CUDA-event duration of the launch
  double cycles = 0;      // median SM cycles of a CTA's timed loop
  double ns = 0;          // median nanoseconds of the same loop
};

double median(std::vector<double> v) {
  std::sort(v.begin(), v.end());
  return v.empty() ? 0.0 : v[v.size() / 2];
}

template <typename K>
int run_probe(K kern, int grid, int iters, uint32_t* sink, unsigned long long* dtimes,
              ProbeRun& out) {
  kern<<<grid, kProbeThreads>>>(iters / 16, 1u, sink, dtimes);  // warm-up
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0);
  if (e == cudaSuccess) {
    kern<<<grid, kProbeThreads>>>(iters, 2u, sink, dtimes);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  std::vector<unsigned long long> h(2 * (size_t)grid);
  if (e == cudaSuccess)
    e = cudaMemcpy(h.data(), dtimes, h.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(e, "qca_probe_peaks");
  std::vector<double> cyc(grid), ns(grid);
  for (int i = 0; i < grid; ++i) {
    cyc[i] = (double)h[2 * i];
    ns[i] = (double)h[2 * i + 1];
  }
  out.ms = ms;
  out.cycles = median(cyc);
  out.ns = median(ns);
  return QCA_OK;
}

}  // namespace

}  // namespace qca

extern "C" int qca_probe_peaks(qca_peaks* out) {
  using namespace qca;
  if (!out) {
    set_error("qca_probe_peaks: NULL output");
    return QCA_ERR_ARG;
  }
  int dev = 0, sms = 0, per_alu = 0, per_smem = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_alu, probe_alu_kernel<kOpMin16x2>,
                                                      kProbeThreads, 0);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_smem, probe_smem_kernel, kProbeThreads, 0);
  if (e != cudaSuccess) return cuda_fail(e, "qca_probe_peaks");
  if (sms <= 0 || per_alu <= 0 || per_smem <= 0) {
    set_error("qca_probe_peaks: the probe kernels do not fit on this device");
    return QCA_ERR_CUDA;
  }
  const int grid = sms * (per_alu < per_smem ? per_alu : per_smem);
  uint32_t* sink = nullptr;
  unsigned long long* dtimes = nullptr;
  e = cudaMalloc(&sink, sizeof(uint32_t) * grid);
  if (e == cudaSuccess) e = cudaMalloc(&dtimes, sizeof(unsigned long long) * 2 * grid);
  if (e != cudaSuccess) {
    cudaFree(sink);
    return cuda_fail(e, "qca_probe_peaks");
  }
  constexpr int kAluIters = 16384, kSmemIters = 16384;
  ProbeRun r[4];
  int rc = run_probe(probe_alu_kernel<kOpMin16x2>, grid, kAluIters, sink, dtimes, r[0]);
  if (!rc) rc = run_probe(probe_alu_kernel<kOpLop3>, grid, kAluIters, sink, dtimes, r[1]);
  if (!rc) rc = run_probe(probe_alu_kernel<kOpMinU32>, grid, kAluIters, sink, dtimes, r[2]);
  if (!rc) rc = run_probe(probe_smem_kernel, grid, kSmemIters, sink, dtimes, r[3]);
  cudaFree(sink);
  cudaFree(dtimes);
  if (rc) return rc;
  const double ctas = (double)grid / sms;  // resident CTAs per SM, all in one wave
  const double alu_per_thread = (double)kAluIters * 8 * kChains;
  const double smem_per_thread = (double)kSmemIters * 8 * 16;
  auto per_clk_sm = [&](const ProbeRun& p, double per_thread) {
    return p.cycles > 0 ? per_thread * kProbeThreads * ctas / p.cycles : 0.0;
  };
  out->sms = sms;
  out->ctas_per_sm = (int)ctas;
  out->sm_clock_mhz = r[0].ns > 0 ? 1e3 * r[0].cycles / r[0].ns : 0.0;
  out->min16x2_per_clk_sm = per_clk_sm(r[0], alu_per_thread);
  out->lop3_per_clk_sm = per_clk_sm(r[1], alu_per_thread);
  out->min_u32_per_clk_sm = per_clk_sm(r[2], alu_per_thread);
  out->smem_bytes_per_clk_sm = per_clk_sm(r[3], smem_per_thread);
  const double threads = (double)grid * kProbeThreads;
  out->min16x2_lane_ops_per_s = r[0].ms > 0 ? 2.0 * alu_per_thread * threads / (r[0].ms * 1e-3) : 0.0;
  out->smem_bytes_per_s = r[3].ms > 0 ? smem_per_thread * threads / (r[3].ms * 1e-3) : 0.0;
  return QCA_OK;
}
