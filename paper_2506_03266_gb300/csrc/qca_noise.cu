// i.i.d. bit-flip noise sampler (Sec. 7 numerics): every link of every shot
// flips independently with probability p, decided by a counter-based
// SplitMix64 draw keyed by (seed, shot, link) so that any batch split, any
// kernel shape and the CPU side give the same realisation.
#include "qca_internal.cuh"

namespace qca {

namespace {

// One thread per (shot, row y, group of 8 columns); writes both link planes.
__global__ void __launch_bounds__(256) sample_kernel(int L, int64_t shot0, int64_t shots,
                                                     uint64_t thr, uint64_t seed_key,
                                                     uint8_t* __restrict__ out) {
  const int groups = (L + 7) / 8;
  const int64_t items = shots * (int64_t)L * groups;
  for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < items;
       it += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = it / ((int64_t)L * groups);
    const int rem = (int)(it - s * (int64_t)L * groups);
    const int y = rem / groups;
    const int x0 = (rem - y * groups) * 8;
    const uint64_t kshot = splitmix64(seed_key ^ (uint64_t)(shot0 + s));
    uint8_t* ex = out + s * 2 * (int64_t)L * L + (int64_t)y * L;
    uint8_t* ey = ex + (int64_t)L * L;
    for (int x = x0; x < x0 + 8 && x < L; ++x) {
      const uint64_t e = 2 * ((uint64_t)y * L + x);
      ex[x] = splitmix64(kshot ^ e) < thr ? 1 : 0;
      ey[x] = splitmix64(kshot ^ (e + 1)) < thr ? 1 : 0;
    }
  }
}

}  // namespace

int launch_sample_errors(int L, int64_t shot0, int64_t shots, uint64_t thr, uint64_t seed,
                         uint8_t* out, cudaStream_t stream) {
  if (shots == 0) return QCA_OK;
  const int groups = (L + 7) / 8;
  const int64_t items = shots * (int64_t)L * groups;
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t blocks = (items + 255) / 256;
  const int64_t cap = (int64_t)(sms > 0 ? sms : 1) * 16;
  if (blocks > cap) blocks = cap;
  sample_kernel<<<(unsigned)blocks, 256, 0, stream>>>(L, shot0, shots, thr,
                                                      splitmix64(seed ^ kTagNoise), out);
  return cuda_fail(cudaGetLastError(), "noise sampler launch");
}

}  // namespace qca
