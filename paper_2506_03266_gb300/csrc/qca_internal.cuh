// Internal declarations shared by the libqca CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "qca.h"

namespace qca {

// Stream tags of the counter-based generator (ASCII "NOISE" and "MOVE").
constexpr uint64_t kTagNoise = 0x4E4F495345ULL;
constexpr uint64_t kTagMove = 0x4D4F5645ULL;
// Stream tag of the balanced-axis random rule (ASCII "BALANCE").
constexpr uint64_t kTagBalance = 0x42414C414E4345ULL;

// SplitMix64 output function (Steele, Lea & Flood, OOPSLA 2014): golden-gamma
// increment, then the variant-13 mix.  Device copy of the published definition.
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// Everything a sweep kernel needs for one batch.
struct DecodeArgs {
  const uint8_t* in;       // noise N [shots][2][L][L], or sigma [shots][L][L] if from_sigma
  int L;
  int64_t shots;
  int max_steps;
  int v;                   // message sub-steps per step
  int m_max;               // message cap (1..255)
  uint64_t move_thr;       // random-move threshold (0 = deterministic rule)
  uint64_t move_key;       // splitmix64(seed ^ kTagMove)
  int64_t shot_offset;     // global index of shot 0 of this batch
  int tie_order;           // QCA_TIE_LEX or QCA_TIE_LITERAL (Eq. degbreak)
  int balance_rule;        // QCA_BALANCE_STAY or QCA_BALANCE_RANDOM
  uint64_t balance_key;    // splitmix64(seed ^ kTagBalance)
  int from_sigma;          // input is a syndrome, not a noise realisation
  uint8_t* out_C;          // [shots][2][L][L]
  int32_t* out_steps;      // [shots]
  uint8_t* out_flag;       // [shots]   (noise input)
  uint8_t* out_cut;        // [shots][2] (syndrome input)
  uint8_t* out_exhausted;  // [shots] or null (syndrome input)
  // Uneven batches (optional): this launch decodes the shots shot_list[0 ..
  // shots); a shot's input and correction blocks start at byte offsets[shot];
  // CTAs take work from the counter *queue (work stealing) when it is set.
  const int32_t* shot_list;
  const int64_t* offsets;
  unsigned int* queue;
  // Some shot block starts off a 4-byte boundary (packed uneven batches with
  // odd L): only the byte-access generic sweep may read it.
  int bytewise;
};

// Byte offset of shot `shot`'s input block: [2][L][L] noise, or [L][L] sigma.
__host__ __device__ __forceinline__ int64_t shot_offset_of(const DecodeArgs& a, int64_t shot) {
  if (a.offsets) return a.offsets[shot];
  const int64_t LL = (int64_t)a.L * a.L;
  return shot * (a.from_sigma ? LL : 2 * LL);
}
// Byte offset of shot `shot`'s correction block ([2][L][L] for either input).
__host__ __device__ __forceinline__ int64_t correction_offset_of(const DecodeArgs& a,
                                                                 int64_t shot) {
  if (a.offsets) return a.offsets[shot];
  return shot * 2 * (int64_t)a.L * a.L;
}

// Per-thread error text (set by the host layer).
void set_error(const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
// A typed device array must start on a multiple of its element size (the
// kernels would fault on it otherwise): QCA_ERR_ARG with the array's name if
// it does not, else QCA_OK.  NULL passes (the NULL checks are separate).
int check_aligned(const void* p, size_t align, const char* what);

// Random-move key chain shared by the kernels: key for (shot, step).
__device__ __forceinline__ uint64_t move_step_key(uint64_t move_key, int64_t shot, int t) {
  uint64_t k1 = splitmix64(move_key ^ (uint64_t)shot);
  return splitmix64(k1 ^ (uint64_t)(uint32_t)t);
}

// Forces of Eqs. blahdef / degbreak at an anyon site from its four fields,
// given in any encoding that is monotone in m and maps "no message" to 0xFF
// (the on-chip kernels' offset encoding; (m - 1) & 0xFF for plain values).
// The argmin' over the nonzero fields is lexicographic (smallest m, then the
// smallest s*a: (-,y), (-,x), (+,x), (+,y)) or, with QCA_TIE_LITERAL, the
// smallest integer key 3m + s*a with equal keys going to the larger m; the
// key difference of two fields does not depend on the encoding's offset.  The
// anyon then moves toward the smaller field of the chosen axis (m^{+a} comes
// from the -a side, so it moves -a).
// Returns 0 (no message), 1 +x, 2 -x, 3 +y, 4 -y, or 5 / 6 for a balanced
// x / y axis (both fields set and equal), which the caller resolves with its
// balance rule (no move, or balance_resolve).
__host__ __device__ __forceinline__ int force_code(uint32_t wpx, uint32_t wmx, uint32_t wpy,
                                                   uint32_t wmy, int tie_order) {
  int ay;
  if (tie_order == QCA_TIE_LITERAL) {
    // composite key: (3w + s*a + 2) * 256 + (255 - w); equal keys cannot come
    // from two fields, so the minimum is unique
    int best = 0x7fffffff;
    ay = -1;
    const uint32_t w4[4] = {wpx, wmx, wpy, wmy};
    const int sa4[4] = {1, -1, 2, -2};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (w4[k] == 0xFFu) continue;
      const int key = ((3 * (int)w4[k] + sa4[k] + 2) << 8) + (255 - (int)w4[k]);
      if (key < best) {
        best = key;
        ay = k >> 1;
      }
    }
    if (ay < 0) return 0;
  } else {
    uint32_t best = wmy;
    ay = 1;
    if (wmx < best) { best = wmx; ay = 0; }
    if (wpx < best) { best = wpx; ay = 0; }
    if (wpy < best) { best = wpy; ay = 1; }
    if (best == 0xFFu) return 0;
  }
  const uint32_t up = ay ? wpy : wpx, um = ay ? wmy : wmx;
  if (up == um) return 5 + ay;
  if (up < um) return ay ? 4 : 2;
  return ay ? 3 : 1;
}

// Draw of the balanced-axis random rule for site r at step t of a shot:
// splitmix64(splitmix64(splitmix64(balance_key ^ shot) ^ t) ^ r); its top bit
// picks +a (0) or -a (1).
__device__ __forceinline__ int balance_resolve(int code, uint64_t key_step, int64_t r) {
  const uint64_t u = splitmix64(key_step ^ (uint64_t)r);
  return (code == 5 ? 1 : 3) + (int)(u >> 63);
}

// Validate sizes and options and fill the common fields of a DecodeArgs.
int fill_decode_args(DecodeArgs& a, const uint8_t* in, int L, int64_t shots, int max_steps,
                     uint64_t seed, const qca_config* cfg);

// Launchers (return QCA_OK or an error code; errors already recorded).
int launch_sample_errors(int L, int64_t shot0, int64_t shots, uint64_t thr, uint64_t seed,
                         uint8_t* out, cudaStream_t stream);
int launch_generic(const DecodeArgs& a, cudaStream_t stream);
int generic_workspace_release();
int fast_path_for(int L, int v, int m_max);  // 0 generic, 1 single-CTA, 2 two-CTA cluster
int launch_fast(const DecodeArgs& a, cudaStream_t stream);
// Large-lattice kernel (cluster of 8 CTAs per shot, state in global memory).
int tiled_path_for(int L, int v, int m_max);  // 1 if it takes (L, v, m_max)
int launch_tiled(const DecodeArgs& a, cudaStream_t stream);
int tiled_workspace_release();
int generic_forced(int L);  // qca_set_kernel_path(L, 0) is in effect
// Kernel path for (L, v, m_max) with the overrides applied: 0 generic,
// 1 / 2 on-chip (one CTA / two-CTA cluster), 3 tiled; and the launch.
int decode_path(int L, int v, int m_max);
int launch_decode(const DecodeArgs& a, cudaStream_t stream);
// Mixed lattice sizes in one persistent launch (on-chip sweep): the group
// size of a lattice size in it (0 two-CTA pair, else 512, 256, 128 or 64
// threads; -1 not on the on-chip sweep), and the launch over items queued by
// group size (pairs first), then by decreasing L.
int mixed_group_threads(int L, int m_max);
int launch_mixed(const DecodeArgs& a, const uint8_t* item_class, const int* sizes,
                 const int* group_threads, int nclass, int64_t n_pair, int64_t n_items,
                 cudaStream_t stream);
// Generic sweep on the library's fixed device array (no allocation).
int launch_generic_noalloc(const DecodeArgs& a, cudaStream_t stream);
size_t noalloc_slot_bytes(int L);

}  // namespace qca
