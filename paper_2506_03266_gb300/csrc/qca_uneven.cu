// Uneven batches: shots of different lattice sizes decoded together.
//
// A plan groups the shots by L once (host side) and keeps on the device the
// shot lists, the byte offsets of every shot's [2][L][L] block in the packed
// input, and the work counters.  A decode makes one persistent launch of the
// mixed-size on-chip kernel over every shot whose size it takes (a single
// queue, largest L first, work stealing across sizes, each shot retiring on
// its own step count).  Shots of other sizes (or packed off a 4-byte boundary)
// go to per-size persistent launches of their own kernel on side streams
// forked from and joined back to the caller's stream (beside the mixed-size
// launch, which has no dependence on them), and that per-size form
// can also be chosen for every size (qca_uneven_plan_set_mode).  Either way
// the decode can be captured in one CUDA graph.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <utility>
#include <mutex>
#include <vector>

#include "qca_internal.cuh"

namespace qca {

namespace {

constexpr uint64_t kTagSize = 0x4C53495A45ULL;  // "LSIZE"
constexpr uint64_t kTagRate = 0x5052415445ULL;  // "PRATE"

uint64_t threshold_of(double p) {
  if (!(p > 0.0)) return 0;
  if (p >= 1.0) return UINT64_MAX;
  const double t = floor(ldexp(p, 64));
  return t >= 18446744073709551615.0 ? UINT64_MAX : (uint64_t)t;
}

// One CTA per shot (grid-stride); threads over rows x groups of 8 columns.
__global__ void __launch_bounds__(256) sample_uneven_kernel(const int32_t* Ls, const int64_t* offs,
                                                            const uint64_t* thr, int64_t shots,
                                                            uint64_t seed_key, uint8_t* out) {
  for (int64_t s = blockIdx.x; s < shots; s += gridDim.x) {
    const int L = Ls[s];
    const uint64_t t = thr[s];
    const uint64_t kshot = splitmix64(seed_key ^ (uint64_t)s);
    uint8_t* ex = out + offs[s];
    uint8_t* ey = ex + (int64_t)L * L;
    const int groups = (L + 7) / 8;
    for (int it = threadIdx.x; it < L * groups; it += blockDim.x) {
      const int y = it / groups, x0 = (it - y * groups) * 8;
      for (int x = x0; x < x0 + 8 && x < L; ++x) {
        const uint64_t e = 2 * ((uint64_t)y * L + x);
        ex[(int64_t)y * L + x] = splitmix64(kshot ^ e) < t ? 1 : 0;
        ey[(int64_t)y * L + x] = splitmix64(kshot ^ (e + 1)) < t ? 1 : 0;
      }
    }
  }
}

}  // namespace

}  // namespace qca

using namespace qca;

struct qca_uneven_plan_s {
  int mode = 0;                  // 0 (default): one mixed-size launch; 1: one launch per size
  // mixed-size queue: the shots of the sizes the on-chip sweep takes (and whose
  // blocks are 4-byte aligned), pairs first, then by group size, then largest
  // L first
  std::vector<int> msizes;       // its sizes in queue order
  std::vector<int> mgroup;       // group size of each (0 = pair), as planned
  std::vector<int64_t> mcount;   // shots of each
  std::vector<int> in_mixed;     // per size of `sizes`: 1 if it is in the queue
  int64_t m_items = 0;
  int32_t* d_mitems = nullptr;   // item -> shot
  uint8_t* d_mclass = nullptr;   // item -> index into msizes
  int64_t shots = 0;
  int64_t total_bytes = 0;
  int device = 0;
  std::vector<int> sizes;        // distinct L
  std::vector<int64_t> start;    // first list index of each size
  std::vector<int64_t> count;    // shots of each size
  std::vector<int> bytewise;     // per size: some block of it starts off a 4-byte boundary
  int32_t* d_list = nullptr;     // shot indices grouped by size
  int64_t* d_offsets = nullptr;  // byte offset of each shot's block
  unsigned int* d_counters = nullptr;
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
};

extern "C" {

int qca_uneven_draw(int64_t shots, uint64_t seed, int32_t* out_L, uint64_t* out_thr) {
  if (shots < 0 || (shots > 0 && (!out_L || !out_thr))) {
    set_error("qca_uneven_draw: bad arguments");
    return QCA_ERR_ARG;
  }
  // sizes and weights (per cent) of the mixed workload
  static const int kL[6] = {24, 48, 64, 96, 128, 192};
  static const int kCum[6] = {30, 55, 75, 87, 95, 100};
  unsigned __int128 cut[6];
  for (int i = 0; i < 6; ++i) cut[i] = ((unsigned __int128)kCum[i] << 64) / 100;
  const uint64_t lo = threshold_of(0.01), span = threshold_of(0.06);
  const uint64_t kL0 = splitmix64(seed ^ kTagSize), kP0 = splitmix64(seed ^ kTagRate);
  for (int64_t s = 0; s < shots; ++s) {
    const uint64_t u = splitmix64(kL0 ^ (uint64_t)s);
    int c = 0;
    while (c < 5 && (unsigned __int128)u >= cut[c]) ++c;
    out_L[s] = kL[c];
    const uint64_t v = splitmix64(kP0 ^ (uint64_t)s);
    out_thr[s] = lo + (uint64_t)(((unsigned __int128)v * span) >> 64);  // p ~ U[0.01, 0.07)
  }
  return QCA_OK;
}

int qca_uneven_plan_create(const int32_t* L_host, int64_t shots, int64_t* offsets_host,
                           int64_t* total_bytes, qca_uneven_plan_t* out_plan) {
  if (!out_plan || shots < 0 || (shots > 0 && !L_host)) {
    set_error("qca_uneven_plan_create: bad arguments");
    return QCA_ERR_ARG;
  }
  *out_plan = nullptr;
  std::vector<int64_t> offs(shots);
  int64_t acc = 0;
  for (int64_t s = 0; s < shots; ++s) {
    const int L = L_host[s];
    if (L < 3 || L > QCA_MAX_L) {
      set_error("shot %lld: L = %d outside [3, %d]", (long long)s, L, QCA_MAX_L);
      return L < 3 ? QCA_ERR_ARG : QCA_ERR_UNSUPPORTED;
    }
    offs[s] = acc;
    acc += 2 * (int64_t)L * L;
  }
  qca_uneven_plan_s* p = new qca_uneven_plan_s();
  p->shots = shots;
  p->total_bytes = acc;
  cudaGetDevice(&p->device);
  // group by size (counting sort, stable in shot order)
  std::vector<int> distinct(L_host, L_host + shots);
  std::sort(distinct.begin(), distinct.end());
  distinct.erase(std::unique(distinct.begin(), distinct.end()), distinct.end());
  p->sizes = distinct;
  std::vector<int64_t> cnt(distinct.size(), 0);
  auto cls = [&](int L) {
    return (int)(std::lower_bound(distinct.begin(), distinct.end(), L) - distinct.begin());
  };
  for (int64_t s = 0; s < shots; ++s) ++cnt[cls(L_host[s])];
  p->count = cnt;
  // an odd L before a shot moves its block off a 4-byte boundary
  p->bytewise.assign(distinct.size(), 0);
  for (int64_t s = 0; s < shots; ++s)
    if (offs[s] & 3) p->bytewise[cls(L_host[s])] = 1;
  p->start.assign(distinct.size(), 0);
  for (size_t i = 1; i < distinct.size(); ++i) p->start[i] = p->start[i - 1] + cnt[i - 1];
  std::vector<int32_t> list(shots);
  std::vector<int64_t> fill = p->start;
  for (int64_t s = 0; s < shots; ++s) list[fill[cls(L_host[s])]++] = (int32_t)s;
  // the mixed-size queue: sizes the on-chip sweep takes with the default
  // options, aligned blocks only, at most kMixClasses sizes (the largest),
  // ordered by group size (pairs first, then 512 .. 64 threads) and then by
  // decreasing L
  constexpr int kMixClasses = 8;
  p->in_mixed.assign(distinct.size(), 0);
  std::vector<std::pair<int, int>> order;  // (group rank, size index)
  for (int i = (int)distinct.size() - 1; i >= 0; --i) {
    if (p->bytewise[i] || (int)order.size() >= kMixClasses) continue;
    const int gs = qca::mixed_group_threads(distinct[i], 255);
    if (gs < 0) continue;
    order.push_back({gs == 0 ? 1 << 20 : gs, i});
  }
  std::stable_sort(order.begin(), order.end(),
                   [](const std::pair<int, int>& a, const std::pair<int, int>& b) {
                     return a.first > b.first;
                   });
  std::vector<int32_t> mitems;
  std::vector<uint8_t> mclass;
  for (const auto& o : order) {
    const int i = o.second;
    p->in_mixed[i] = 1;
    const uint8_t c = (uint8_t)p->msizes.size();
    p->msizes.push_back(distinct[i]);
    p->mgroup.push_back(o.first == (1 << 20) ? 0 : o.first);
    p->mcount.push_back(cnt[i]);
    for (int64_t j = 0; j < cnt[i]; ++j) {
      mitems.push_back(list[p->start[i] + j]);
      mclass.push_back(c);
    }
  }
  p->m_items = (int64_t)mitems.size();
  cudaError_t e = cudaSuccess;
  const size_t nc = distinct.size();
  if (shots > 0) {
    e = cudaMalloc(&p->d_list, sizeof(int32_t) * shots);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_offsets, sizeof(int64_t) * shots);
    // one counter per size, and the mixed queue's after them
    if (e == cudaSuccess) e = cudaMalloc(&p->d_counters, sizeof(unsigned) * (nc + 1));
    if (e == cudaSuccess)
      e = cudaMemcpy(p->d_list, list.data(), sizeof(int32_t) * shots, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(p->d_offsets, offs.data(), sizeof(int64_t) * shots, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess && p->m_items > 0) {
    e = cudaMalloc(&p->d_mitems, sizeof(int32_t) * p->m_items);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_mclass, p->m_items);
    if (e == cudaSuccess)
      e = cudaMemcpy(p->d_mitems, mitems.data(), sizeof(int32_t) * p->m_items,
                     cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(p->d_mclass, mclass.data(), p->m_items, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming);
  for (size_t i = 0; i < nc && e == cudaSuccess; ++i) {
    cudaStream_t st;
    cudaEvent_t ev;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) p->side.push_back(st);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) p->join.push_back(ev);
  }
  if (e != cudaSuccess) {
    qca_uneven_plan_destroy(p);
    return cuda_fail(e, "qca_uneven_plan_create");
  }
  if (offsets_host) memcpy(offsets_host, offs.data(), sizeof(int64_t) * shots);
  if (total_bytes) *total_bytes = acc;
  *out_plan = p;
  return QCA_OK;
}

int qca_uneven_plan_destroy(qca_uneven_plan_t p) {
  if (!p) return QCA_OK;
  cudaFree(p->d_list);
  cudaFree(p->d_mitems);
  cudaFree(p->d_mclass);
  cudaFree(p->d_offsets);
  cudaFree(p->d_counters);
  for (auto s : p->side) cudaStreamDestroy(s);
  for (auto e : p->join) cudaEventDestroy(e);
  if (p->fork) cudaEventDestroy(p->fork);
  delete p;
  return QCA_OK;
}

int qca_uneven_plan_set_mode(qca_uneven_plan_t p, int mode) {
  if (!p || (mode != 0 && mode != 1)) {
    set_error("qca_uneven_plan_set_mode: bad arguments");
    return QCA_ERR_ARG;
  }
  p->mode = mode;
  return QCA_OK;
}

int qca_uneven_plan_offsets_device(qca_uneven_plan_t p, const int64_t** offsets_device) {
  if (!p || !offsets_device) {
    set_error("qca_uneven_plan_offsets_device: bad arguments");
    return QCA_ERR_ARG;
  }
  *offsets_device = p->d_offsets;
  return QCA_OK;
}

int qca_sample_errors_uneven_async(const int32_t* L_dev, const int64_t* offsets_dev,
                                   const uint64_t* thr_dev, int64_t shots, uint64_t seed,
                                   uint8_t* out_errors, void* stream) {
  if (shots < 0 || (shots > 0 && (!L_dev || !offsets_dev || !thr_dev || !out_errors))) {
    set_error("qca_sample_errors_uneven_async: bad arguments");
    return QCA_ERR_ARG;
  }
  if (int rc = check_aligned(L_dev, 4, "L_dev")) return rc;
  if (int rc = check_aligned(offsets_dev, 8, "offsets_dev")) return rc;
  if (int rc = check_aligned(thr_dev, 8, "thr_dev")) return rc;
  if (shots == 0) return QCA_OK;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t blocks = shots < (int64_t)sms * 16 ? shots : (int64_t)sms * 16;
  sample_uneven_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(
      L_dev, offsets_dev, thr_dev, shots, splitmix64(seed ^ kTagNoise), out_errors);
  return cuda_fail(cudaGetLastError(), "uneven sampler launch");
}

int qca_decode_uneven_async(qca_uneven_plan_t p, const uint8_t* errors, int max_steps,
                            uint64_t rng_seed, uint8_t* out_correction, int32_t* out_steps,
                            uint8_t* out_logical_fail, const qca_config* cfg, void* stream) {
  if (!p) {
    set_error("qca_decode_uneven_async: NULL plan");
    return QCA_ERR_ARG;
  }
  if (max_steps < 0 || max_steps > QCA_MAX_STEPS) {
    set_error("max_steps = %d outside [0, %d]", max_steps, QCA_MAX_STEPS);
    return QCA_ERR_ARG;
  }
  if (p->shots == 0) return QCA_OK;
  if (!errors || !out_correction || !out_steps || !out_logical_fail) {
    set_error("NULL array pointer");
    return QCA_ERR_ARG;
  }
  qca_config c;
  qca_default_config(&c);
  if (cfg) c = *cfg;
  cudaStream_t st = (cudaStream_t)stream;
  // the mixed-size launch takes the queued sizes unless the per-size form is
  // chosen, or the options leave the on-chip sweep (v != 3, m_max < 3) or
  // change a planned group size (tuning overrides)
  bool mixed = p->mode == 0 && p->m_items > 0 && c.v == 3;
  for (size_t i = 0; mixed && i < p->msizes.size(); ++i)
    mixed = mixed_group_threads(p->msizes[i], c.m_max) == p->mgroup[i];
  cudaError_t e = cudaMemsetAsync(p->d_counters, 0, sizeof(unsigned) * (p->sizes.size() + 1), st);
  if (e != cudaSuccess) return cuda_fail(e, "uneven decode counters");
  // the side streams fork before the mixed-size launch, so that the sizes
  // outside its queue take SMs as its CTAs retire
  e = cudaEventRecord(p->fork, st);
  if (e != cudaSuccess) return cuda_fail(e, "uneven decode fork");
  if (mixed) {
    DecodeArgs a;
    int rc = fill_decode_args(a, errors, p->msizes[0], p->m_items, max_steps, rng_seed, &c);
    if (rc) return rc;
    a.out_C = out_correction;
    a.out_steps = out_steps;
    a.out_flag = out_logical_fail;
    a.shot_list = p->d_mitems;
    a.offsets = p->d_offsets;
    a.queue = p->d_counters + p->sizes.size();
    int64_t n_pair = 0;
    for (size_t i = 0; i < p->mgroup.size(); ++i)
      if (p->mgroup[i] == 0) n_pair += p->mcount[i];
    rc = launch_mixed(a, p->d_mclass, p->msizes.data(), p->mgroup.data(), (int)p->msizes.size(),
                      n_pair, p->m_items, st);
    if (rc) return rc;
  }
  for (size_t i = 0; i < p->sizes.size(); ++i) {
    if (mixed && p->in_mixed[i]) continue;
    e = cudaStreamWaitEvent(p->side[i], p->fork, 0);
    if (e != cudaSuccess) return cuda_fail(e, "uneven decode fork wait");
    DecodeArgs a;
    int rc = fill_decode_args(a, errors, p->sizes[i], p->count[i], max_steps, rng_seed, &c);
    if (rc) return rc;
    a.out_C = out_correction;
    a.out_steps = out_steps;
    a.out_flag = out_logical_fail;
    a.shot_list = p->d_list + p->start[i];
    a.offsets = p->d_offsets;
    a.queue = p->d_counters + i;
    a.bytewise = p->bytewise[i];
    rc = launch_decode(a, p->side[i]);
    if (rc) return rc;
    e = cudaEventRecord(p->join[i], p->side[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, p->join[i], 0);
    if (e != cudaSuccess) return cuda_fail(e, "uneven decode join");
  }
  return QCA_OK;
}

}  // extern "C"
