// Host side of the libqca C ABI: argument checks, option handling, kernel
// dispatch, error reporting and the host-buffer (end-to-end) entry point.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "qca_internal.cuh"

namespace qca {

namespace {
thread_local char g_err[512] = "no error";

uint64_t prob_threshold(double p) {
  if (!(p > 0.0)) return 0;
  if (p >= 1.0) return UINT64_MAX;
  const double t = floor(ldexp(p, 64));
  if (t >= 18446744073709551615.0) return UINT64_MAX;
  return (uint64_t)t;
}

// Staging buffers of the host-buffer entry point, one set per device.
struct Staging {
  uint8_t* buf = nullptr;
  size_t bytes = 0;
  cudaStream_t streams[2] = {nullptr, nullptr};
};
std::mutex g_stage_mu;
Staging g_stage[64];
}  // namespace

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int cuda_fail(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return QCA_OK;
  set_error("%s: %s", what, cudaGetErrorString(e));
  return QCA_ERR_CUDA;
}

int check_aligned(const void* p, size_t align, const char* what) {
  if (reinterpret_cast<uintptr_t>(p) & (align - 1)) {
    set_error("%s is not %zu-byte aligned", what, align);
    return QCA_ERR_ARG;
  }
  return QCA_OK;
}

static int check_config(const qca_config* cfg, qca_config* out) {
  qca_default_config(out);
  if (cfg) *out = *cfg;
  if (out->v < 1 || out->v > 8) {
    set_error("v = %d outside the supported range 1..8", out->v);
    return QCA_ERR_UNSUPPORTED;
  }
  if (out->m_max < 1 || out->m_max > 255) {
    set_error("m_max = %d outside the supported range 1..255", out->m_max);
    return QCA_ERR_UNSUPPORTED;
  }
  if (!(out->p_move >= 0.0 && out->p_move <= 1.0)) {
    set_error("p_move must lie in [0, 1]");
    return QCA_ERR_ARG;
  }
  if (out->tie_order != QCA_TIE_LEX && out->tie_order != QCA_TIE_LITERAL) {
    set_error("tie_order = %d is neither QCA_TIE_LEX nor QCA_TIE_LITERAL", out->tie_order);
    return QCA_ERR_ARG;
  }
  if (out->balance_rule != QCA_BALANCE_STAY && out->balance_rule != QCA_BALANCE_RANDOM) {
    set_error("balance_rule = %d is neither QCA_BALANCE_STAY nor QCA_BALANCE_RANDOM",
              out->balance_rule);
    return QCA_ERR_ARG;
  }
  return QCA_OK;
}

static int check_sizes(int L, int64_t shots, int max_steps) {
  if (L < 3 || L > QCA_MAX_L) {
    set_error("L = %d outside [3, %d]", L, QCA_MAX_L);
    return L < 3 ? QCA_ERR_ARG : QCA_ERR_UNSUPPORTED;
  }
  if (shots < 0) {
    set_error("shots = %lld is negative", (long long)shots);
    return QCA_ERR_ARG;
  }
  if (max_steps < 0 || max_steps > QCA_MAX_STEPS) {
    set_error("max_steps = %d outside [0, %d]", max_steps, QCA_MAX_STEPS);
    return QCA_ERR_ARG;
  }
  return QCA_OK;
}

int decode_path(int L, int v, int m_max) {
  if (generic_forced(L)) return 0;
  if (tiled_path_for(L, v, m_max) > 0) return 3;
  return fast_path_for(L, v, m_max);
}

int launch_decode(const DecodeArgs& a, cudaStream_t stream) {
  if (a.shots == 0) return QCA_OK;
  if (int rc = check_aligned(a.out_steps, 4, "out_steps")) return rc;
  int path = decode_path(a.L, a.v, a.m_max);
  // The on-chip and large-lattice kernels read the input and write the
  // correction as 32-bit words.  A caller array or shot block off a 4-byte
  // boundary goes to the generic sweep, which accesses bytes (same results).
  const uintptr_t wide = reinterpret_cast<uintptr_t>(a.in) | reinterpret_cast<uintptr_t>(a.out_C);
  if (path > 0 && (a.bytewise || (wide & 3))) path = 0;
  if (path == 3) return launch_tiled(a, stream);
  if (path > 0) return launch_fast(a, stream);
  return launch_generic(a, stream);
}

static int dispatch(DecodeArgs& a, cudaStream_t stream) { return launch_decode(a, stream); }

static int fill_args(DecodeArgs& a, const uint8_t* in, int L, int64_t shots, int max_steps,
                     uint64_t seed, const qca_config& c) {
  memset(&a, 0, sizeof(a));
  a.in = in;
  a.L = L;
  a.shots = shots;
  a.max_steps = max_steps;
  a.v = c.v;
  a.m_max = c.m_max;
  a.move_thr = prob_threshold(c.p_move);
  a.move_key = splitmix64(seed ^ kTagMove);
  a.shot_offset = c.shot_offset;
  a.tie_order = c.tie_order;
  a.balance_rule = c.balance_rule;
  a.balance_key = splitmix64(seed ^ kTagBalance);
  return QCA_OK;
}

int fill_decode_args(DecodeArgs& a, const uint8_t* in, int L, int64_t shots, int max_steps,
                     uint64_t seed, const qca_config* cfg) {
  int rc = check_sizes(L, shots, max_steps);
  if (rc) return rc;
  qca_config c;
  if ((rc = check_config(cfg, &c))) return rc;
  return fill_args(a, in, L, shots, max_steps, seed, c);
}

}  // namespace qca

using namespace qca;

extern "C" {

int qca_version(void) { return 101; }

const char* qca_last_error(void) { return g_err; }

int qca_default_config(qca_config* cfg) {
  if (!cfg) {
    set_error("cfg is NULL");
    return QCA_ERR_ARG;
  }
  cfg->v = 3;
  cfg->m_max = 255;
  cfg->p_move = 0.0;
  cfg->shot_offset = 0;
  cfg->tie_order = QCA_TIE_LEX;
  cfg->balance_rule = QCA_BALANCE_STAY;
  return QCA_OK;
}

int qca_sample_errors_async(int L, int64_t shot0, int64_t shots, double p, uint64_t seed,
                            uint8_t* out_errors, void* stream) {
  int rc = check_sizes(L, shots, 0);
  if (rc) return rc;
  if (!(p >= 0.0 && p <= 1.0)) {
    set_error("p = %g outside [0, 1]", p);
    return QCA_ERR_ARG;
  }
  if (shots > 0 && !out_errors) {
    set_error("out_errors is NULL");
    return QCA_ERR_ARG;
  }
  return launch_sample_errors(L, shot0, shots, prob_threshold(p), seed, out_errors,
                              (cudaStream_t)stream);
}

int qca_sample_errors(int L, int shots, double p, uint64_t seed, uint8_t* out_errors) {
  int rc = qca_sample_errors_async(L, 0, shots, p, seed, out_errors, nullptr);
  if (rc) return rc;
  return cuda_fail(cudaStreamSynchronize(nullptr), "qca_sample_errors");
}

int qca_decode_batch_async(const uint8_t* syndrome, int L, int64_t shots, int max_steps,
                           uint64_t rng_seed, uint8_t* out_correction, int32_t* out_steps,
                           uint8_t* out_logical_fail, const qca_config* cfg, void* stream) {
  int rc = check_sizes(L, shots, max_steps);
  if (rc) return rc;
  qca_config c;
  if ((rc = check_config(cfg, &c))) return rc;
  if (shots > 0 && (!syndrome || !out_correction || !out_steps || !out_logical_fail)) {
    set_error("NULL array pointer");
    return QCA_ERR_ARG;
  }
  DecodeArgs a;
  fill_args(a, syndrome, L, shots, max_steps, rng_seed, c);
  a.out_C = out_correction;
  a.out_steps = out_steps;
  a.out_flag = out_logical_fail;
  return dispatch(a, (cudaStream_t)stream);
}

int qca_decode_batch(const uint8_t* syndrome, int L, int shots, int max_steps, uint64_t rng_seed,
                     uint8_t* out_correction, int32_t* out_steps, uint8_t* out_logical_fail) {
  int rc = qca_decode_batch_async(syndrome, L, shots, max_steps, rng_seed, out_correction,
                                  out_steps, out_logical_fail, nullptr, nullptr);
  if (rc) return rc;
  return cuda_fail(cudaStreamSynchronize(nullptr), "qca_decode_batch");
}

int qca_decode_syndrome_batch_async(const uint8_t* sigma, int L, int64_t shots, int max_steps,
                                    uint64_t rng_seed, uint8_t* out_correction,
                                    int32_t* out_steps, uint8_t* out_cut_parity,
                                    uint8_t* out_exhausted, const qca_config* cfg,
                                    void* stream) {
  int rc = check_sizes(L, shots, max_steps);
  if (rc) return rc;
  qca_config c;
  if ((rc = check_config(cfg, &c))) return rc;
  if (shots > 0 && (!sigma || !out_correction || !out_steps || !out_cut_parity)) {
    set_error("NULL array pointer");
    return QCA_ERR_ARG;
  }
  DecodeArgs a;
  fill_args(a, sigma, L, shots, max_steps, rng_seed, c);
  a.from_sigma = 1;
  a.out_C = out_correction;
  a.out_steps = out_steps;
  a.out_cut = out_cut_parity;
  a.out_exhausted = out_exhausted;
  return dispatch(a, (cudaStream_t)stream);
}

int qca_decode_syndrome_batch(const uint8_t* sigma, int L, int shots, int max_steps,
                              uint64_t rng_seed, uint8_t* out_correction, int32_t* out_steps,
                              uint8_t* out_cut_parity) {
  int rc = qca_decode_syndrome_batch_async(sigma, L, shots, max_steps, rng_seed, out_correction,
                                           out_steps, out_cut_parity, nullptr, nullptr,
                                           nullptr);
  if (rc) return rc;
  return cuda_fail(cudaStreamSynchronize(nullptr), "qca_decode_syndrome_batch");
}

int qca_decode_batch_noalloc(const uint8_t* syndrome, int L, int64_t shots, int max_steps,
                             uint64_t rng_seed, uint8_t* out_correction, int32_t* out_steps,
                             uint8_t* out_logical_fail, const qca_config* cfg, void* stream) {
  int rc = check_sizes(L, shots, max_steps);
  if (rc) return rc;
  qca_config c;
  if ((rc = check_config(cfg, &c))) return rc;
  if (shots > 0 && (!syndrome || !out_correction || !out_steps || !out_logical_fail)) {
    set_error("NULL array pointer");
    return QCA_ERR_ARG;
  }
  if ((rc = check_aligned(out_steps, 4, "out_steps"))) return rc;
  DecodeArgs a;
  fill_args(a, syndrome, L, shots, max_steps, rng_seed, c);
  a.out_C = out_correction;
  a.out_steps = out_steps;
  a.out_flag = out_logical_fail;
  // a call with no shots still runs the one-time set-up of the device (the
  // scratch address and the kernel's module), so it can serve as the warm-up
  return launch_generic_noalloc(a, (cudaStream_t)stream);
}

int qca_kernel_path(int L, const qca_config* cfg) {
  int rc = check_sizes(L, 0, 0);
  if (rc) return rc;
  qca_config c;
  if ((rc = check_config(cfg, &c))) return rc;
  return decode_path(L, c.v, c.m_max);
}

int qca_decode_batch_host(const uint8_t* syndrome, int L, int64_t shots, int max_steps,
                          uint64_t rng_seed, uint8_t* out_correction, int32_t* out_steps,
                          uint8_t* out_logical_fail, const qca_config* cfg) {
  int rc = check_sizes(L, shots, max_steps);
  if (rc) return rc;
  qca_config c;
  if ((rc = check_config(cfg, &c))) return rc;
  if (shots == 0) return QCA_OK;
  if (!syndrome || !out_steps || !out_logical_fail) {
    set_error("NULL array pointer");
    return QCA_ERR_ARG;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) {
    set_error("device index %d out of range", dev);
    return QCA_ERR_UNSUPPORTED;
  }
  const size_t E = 2 * (size_t)L * L;
  // ~64 MiB of noise per chunk; at least one shot.
  int64_t chunk = (int64_t)((size_t(64) << 20) / E);
  if (chunk < 1) chunk = 1;
  if (chunk > shots) chunk = shots;
  const size_t per_set = ((chunk * E + 255) & ~(size_t)255) * 2 + ((chunk * 5 + 255) & ~(size_t)255) + 512;
  // the generic and tiled paths share one workspace per device: no concurrent chunks
  const int path = decode_path(L, c.v, c.m_max);
  const bool concurrent = path == 1 || path == 2;
  std::lock_guard<std::mutex> lk(g_stage_mu);
  Staging& st = g_stage[dev];
  if (st.bytes < 2 * per_set) {
    if (st.buf) {
      cudaError_t e = cudaDeviceSynchronize();
      if (e != cudaSuccess) return cuda_fail(e, "synchronise before staging growth");
      cudaFree(st.buf);
      st.buf = nullptr;
      st.bytes = 0;
    }
    cudaError_t e = cudaMalloc(&st.buf, 2 * per_set);
    if (e != cudaSuccess) return cuda_fail(e, "staging allocation");
    st.bytes = 2 * per_set;
  }
  for (int i = 0; i < 2; ++i)
    if (!st.streams[i]) {
      cudaError_t e = cudaStreamCreateWithFlags(&st.streams[i], cudaStreamNonBlocking);
      if (e != cudaSuccess) return cuda_fail(e, "stream creation");
    }
  // Chunk k uses buffer set k % 2 on stream k % 2.  The input copy of chunk
  // k + 1 is enqueued before the output copies of chunk k: where the driver
  // serves both directions from one copy queue, an input copy queued behind an
  // output copy would wait for that chunk's decode, and the next decode with it.
  const int64_t nchunks = (shots + chunk - 1) / chunk;
  auto set_of = [&](int64_t k) { return concurrent ? (int)(k & 1) : 0; };
  auto dN_of = [&](int64_t k) { return st.buf + set_of(k) * per_set; };
  auto input_copy = [&](int64_t k) -> int {
    const int64_t s0 = k * chunk, n = (shots - s0 < chunk) ? shots - s0 : chunk;
    cudaError_t e = cudaMemcpyAsync(dN_of(k), syndrome + s0 * E, n * E, cudaMemcpyHostToDevice,
                                    st.streams[set_of(k)]);
    return e == cudaSuccess ? QCA_OK : cuda_fail(e, "host-to-device copy");
  };
  // on an error, wait for what was already enqueued before returning, so that
  // no copy touches the caller's buffers afterwards
  auto drain = [&](int err) {
    for (int i = 0; i < 2; ++i) cudaStreamSynchronize(st.streams[i]);
    return err;
  };
  if ((rc = input_copy(0))) return drain(rc);
  for (int64_t k = 0; k < nchunks; ++k) {
    const int64_t s0 = k * chunk, n = (shots - s0 < chunk) ? shots - s0 : chunk;
    cudaStream_t sm = st.streams[set_of(k)];
    uint8_t* dN = dN_of(k);
    uint8_t* dC = dN + ((chunk * E + 255) & ~(size_t)255);
    uint8_t* dF = dC + ((chunk * E + 255) & ~(size_t)255);
    int32_t* dS = (int32_t*)(dF + ((chunk + 15) & ~(int64_t)15));
    qca_config cc = c;
    cc.shot_offset = c.shot_offset + s0;
    rc = qca_decode_batch_async(dN, L, n, max_steps, rng_seed, dC, dS, dF, &cc, sm);
    if (rc) return drain(rc);
    // one buffer set without concurrency: the next input waits for this chunk
    if (concurrent && k + 1 < nchunks && (rc = input_copy(k + 1))) return drain(rc);
    cudaError_t e = cudaSuccess;
    if (out_correction)
      e = cudaMemcpyAsync(out_correction + s0 * E, dC, n * E, cudaMemcpyDeviceToHost, sm);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(out_steps + s0, dS, n * sizeof(int32_t), cudaMemcpyDeviceToHost, sm);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(out_logical_fail + s0, dF, n, cudaMemcpyDeviceToHost, sm);
    if (e != cudaSuccess) return drain(cuda_fail(e, "device-to-host copy"));
    if (!concurrent && k + 1 < nchunks && (rc = input_copy(k + 1))) return drain(rc);
  }
  for (int i = 0; i < 2; ++i) {
    cudaError_t e = cudaStreamSynchronize(st.streams[i]);
    if (e != cudaSuccess) return drain(cuda_fail(e, "qca_decode_batch_host"));
  }
  return QCA_OK;
}

int qca_free_workspace(void) {
  int rc = generic_workspace_release();
  const int rc2 = tiled_workspace_release();
  if (rc == QCA_OK) rc = rc2;
  std::lock_guard<std::mutex> lk(g_stage_mu);
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && g_stage[dev].buf) {
    cudaError_t e = cudaFree(g_stage[dev].buf);
    g_stage[dev].buf = nullptr;
    g_stage[dev].bytes = 0;
    if (e != cudaSuccess && rc == QCA_OK) rc = cuda_fail(e, "staging free");
  }
  return rc;
}

}  // extern "C"
