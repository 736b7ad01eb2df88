// Learned local pre-decoder (not part of the paper) in front of the exact
// automaton.  A 4-layer 3x3 convolutional net with circular padding
// (2 -> 32 -> 32 -> 32 -> 4 channels, ReLU between layers) reads the anyon
// indicator and a constant channel and gives every site four logits, one per
// move direction (+x, -x, +y, -y).  An anyon proposes the direction of its
// largest logit when that logit is positive; a link whose two end anyons
// propose each other is flipped (the pair annihilates).  The automaton then
// decodes the residual N xor C0; the final correction is C0 xor C_automaton and
// the failure flag is the automaton's on the residual (N xor C0 xor C_automaton
// = N xor C).
//
// Training labels come from the automaton itself: the direction an anyon moves
// in the automaton's first step (all fields empty before it, so the fields are
// the cone distances <= 3), kept when its neighbour in that direction moves
// back (the pair annihilates in that step); other anyons get label 4 (none).
//
// Inference: layers 2-4 as implicit-GEMM convolutions on the tensor cores,
// bf16 operands and fp32 accumulation: tcgen05 with the accumulator in tensor
// memory where L is a multiple of 128 (layer 1 then a table of the 512 3 x 3
// anyon patterns), mma.sync elsewhere (layer 1 on the CUDA cores);
// activations bf16 in NHWC layout.
// Training: bf16 tensor-core implicit GEMMs with fp32 accumulation and fp32
// master weights (forward, input gradients, weight gradients), Adam.
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "qca_internal.cuh"

namespace qca {

namespace {

// ---- parameter layout: per layer W[co][ci][3][3] then b[co], fp32
constexpr int kLayers = 4;
constexpr int kCo[kLayers] = {32, 32, 32, 4};
constexpr int kCi[kLayers] = {2, 32, 32, 32};
constexpr int kW0 = 0, kB0 = kW0 + 32 * 2 * 9;
constexpr int kW1 = kB0 + 32, kB1 = kW1 + 32 * 32 * 9;
constexpr int kW2 = kB1 + 32, kB2 = kW2 + 32 * 32 * 9;
constexpr int kW3 = kB2 + 32, kB3 = kW3 + 4 * 32 * 9;
constexpr int kParams = kB3 + 4;
constexpr int kWoff[kLayers] = {kW0, kW1, kW2, kW3};

constexpr uint64_t kTagTrain = 0x545241494EULL;  // "TRAIN"

__device__ __forceinline__ int wrapL(int i, int L) { return i < 0 ? i + L : (i >= L ? i - L : i); }

// ---------------------------------------------------------------- labels --

// sigma (1 = anyon) from noise [2][L][L] for every shot, byte per site
__global__ void syndrome_kernel(const uint8_t* __restrict__ N, int L, int64_t shots,
                                uint8_t* __restrict__ sig) {
  const int64_t LL = (int64_t)L * L;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < shots * LL;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = i / LL;
    const int r = (int)(i - s * LL), x = r % L, y = r / L;
    const uint8_t* n = N + s * 2 * LL;
    sig[i] = n[r] ^ n[y * L + wrapL(x - 1, L)] ^ n[LL + r] ^ n[LL + wrapL(y - 1, L) * L + x];
  }
}

// First-step direction of every anyon (0 +x, 1 -x, 2 +y, 3 -y, 4 none; 255 no
// anyon).  With empty fields, three applications of A^(D) leave in m^{s a}_r
// the smallest d <= 3 with an anyon on {r - s d a^ + j b^, |j| <= d}; the
// forces follow readings R1-R4 (smallest field, ties (-,y) < (-,x) < (+,x) <
// (+,y), no move on a balanced axis).
__global__ void first_dir_kernel(const uint8_t* __restrict__ sig, int L, int64_t shots,
                                 uint8_t* __restrict__ dir) {
  const int64_t LL = (int64_t)L * L;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < shots * LL;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = i / LL;
    const int r = (int)(i - s * LL), x = r % L, y = r / L;
    const uint8_t* g = sig + s * LL;
    if (!g[r]) {
      dir[i] = 255;
      continue;
    }
    int m[4];  // (+,x) (-,x) (+,y) (-,y); 0 = none
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const int sgn = (f % 2 == 0) ? 1 : -1;
      const bool ax = f < 2;
      int best = 0;
      for (int d = 1; d <= 3 && !best; ++d) {
        for (int j = -d; j <= d; ++j) {
          const int xx = ax ? wrapL(x - sgn * d, L) : wrapL(x + j, L);
          const int yy = ax ? wrapL(y + j, L) : wrapL(y - sgn * d, L);
          if (g[yy * L + xx]) {
            best = d;
            break;
          }
        }
      }
      m[f] = best;
    }
    const int val[4] = {m[3], m[1], m[0], m[2]};  // preference order (-,y) (-,x) (+,x) (+,y)
    int bi = -1, bv = 0;
    for (int k = 0; k < 4; ++k)
      if (val[k] > 0 && (bi < 0 || val[k] < bv)) {
        bi = k;
        bv = val[k];
      }
    int code = 4;
    if (bi >= 0) {
      const bool yaxis = (bi == 0 || bi == 3);
      const int mp = yaxis ? m[2] : m[0], mm = yaxis ? m[3] : m[1];
      const unsigned up = mp ? (unsigned)mp : 0xFFu, um = mm ? (unsigned)mm : 0xFFu;
      if (up != um) code = (up < um) ? (yaxis ? 3 : 1) : (yaxis ? 2 : 0);
    }
    dir[i] = (uint8_t)code;
  }
}

// label = direction if the neighbour in that direction moves back, else 4
__global__ void mutual_label_kernel(const uint8_t* __restrict__ dir, int L, int64_t shots,
                                    uint8_t* __restrict__ lab) {
  const int64_t LL = (int64_t)L * L;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < shots * LL;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = i / LL;
    const int r = (int)(i - s * LL), x = r % L, y = r / L;
    const int d = dir[i];
    if (d == 255) {
      lab[i] = 255;
      continue;
    }
    int out = 4;
    if (d < 4) {
      const int dx = (d == 0) ? 1 : (d == 1 ? -1 : 0), dy = (d == 2) ? 1 : (d == 3 ? -1 : 0);
      const int nb = wrapL(y + dy, L) * L + wrapL(x + dx, L);
      const int back = d ^ 1;
      if (dir[s * LL + nb] == back) out = d;
    }
    lab[i] = (uint8_t)out;
  }
}

// ------------------------------------------------------- training (fp32) --

// Random training syndromes: shot b of batch `it` uses global index
// it * B + b; p ~ U[p_lo, p_hi) per shot; links drawn like qca_sample_errors.
__global__ void train_sample_kernel(int L, int B, int64_t it, uint64_t seed, uint64_t t_lo,
                                    uint64_t t_span, uint8_t* __restrict__ sig) {
  const int LL = L * L;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B * LL; i += gridDim.x * blockDim.x) {
    const int b = i / LL, r = i - b * LL, x = r % L, y = r / L;
    const uint64_t shot = (uint64_t)it * B + b;
    const uint64_t ks = splitmix64(splitmix64(seed ^ kTagTrain) ^ shot);
    const uint64_t thr = t_lo + (uint64_t)(((unsigned __int128)splitmix64(ks ^ 0x5052ULL) * t_span) >> 64);
    auto link = [&](int xx, int yy, int dirb) -> uint8_t {
      const uint64_t e = 2 * ((uint64_t)yy * L + xx) + dirb;
      return splitmix64(ks ^ e) < thr ? 1 : 0;
    };
    sig[i] = link(x, y, 0) ^ link(wrapL(x - 1, L), y, 0) ^ link(x, y, 1) ^ link(x, wrapL(y - 1, L), 1);
  }
}

__global__ void count_labelled_kernel(const uint8_t* __restrict__ lab, int n,
                                      unsigned int* __restrict__ count) {
  unsigned int c = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    c += lab[i] != 255;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

// Label smoothing of the training target: eps spread evenly over the five
// classes.  It bounds the logits the loss drives toward (target margin
// log((1 - eps + eps/5) / (eps/5)), about 3.8 at eps = 0.1), which keeps the
// activations, and so the size of one bf16 rounding step in them, small.
constexpr float kLabelSmoothing = 0.1f;

// Adam (Kingma & Ba, ICLR 2015) with bias corrections c1 = 1 / (1 - b1^t),
// c2 = 1 / (1 - b2^t) computed on the host; epsilon 1e-8.
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g,
                            float* __restrict__ m1, float* __restrict__ m2, int n, float lr,
                            float b1, float b2, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    p[i] -= lr * (a * c1) / (sqrtf(b * c2) + 1e-8f);
  }
}

// ---------------------------------------------------- inference (bf16) ----

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// bf16 weights of layers 2..4 as [tap][co][ci] (co padded to 8 for layer 4),
// layer 1 fp32 [co][ci][tap], biases fp32; built from the fp32 parameters.
__global__ void prepare_weights_kernel(const float* __restrict__ P, __nv_bfloat16* __restrict__ Wb,
                                       float* __restrict__ W1) {
  const int n23 = 9 * 32 * 32, n4 = 9 * 8 * 32;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 2 * n23 + n4 + 32 * 2 * 9;
       i += gridDim.x * blockDim.x) {
    if (i < 2 * n23) {
      const int l = i / n23, j = i - l * n23;  // layers 2, 3
      const int tap = j / (32 * 32), co = (j / 32) % 32, ci = j % 32;
      const int off = (l == 0) ? kW1 : kW2;
      Wb[i] = __float2bfloat16_rn(P[off + (co * 32 + ci) * 9 + tap]);
    } else if (i < 2 * n23 + n4) {
      const int j = i - 2 * n23, tap = j / (8 * 32), co = (j / 32) % 8, ci = j % 32;
      Wb[i] = __float2bfloat16_rn(co < 4 ? P[kW3 + (co * 32 + ci) * 9 + tap] : 0.f);
    } else {
      const int j = i - 2 * n23 - n4;  // layer 1, rounded to bf16 like the others
      W1[j] = __bfloat162float(__float2bfloat16_rn(P[kW0 + j]));
    }
  }
}

// layer 1 (2 -> 32, CUDA cores).  The inputs (anyon, 1) are exact in bf16;
// the constant channel's nine taps are folded into the bias once per CTA, and
// each anyon tap adds its weight column.
__global__ void layer1_kernel(const uint8_t* __restrict__ sig, int L, int64_t shots,
                              const float* __restrict__ W1, const float* __restrict__ P,
                              __nv_bfloat16* __restrict__ out) {
  __shared__ float sW[9][32];  // anyon-channel weights by tap
  __shared__ float sb[32];     // bias + constant-channel taps
  for (int i = threadIdx.x; i < 32 * 9; i += blockDim.x) sW[i % 9][i / 9] = W1[(i / 9) * 18 + i % 9];
  for (int co = threadIdx.x; co < 32; co += blockDim.x) {
    float b = P[kB0 + co];
    for (int tap = 0; tap < 9; ++tap) b += W1[co * 18 + 9 + tap];
    sb[co] = b;
  }
  __syncthreads();
  const int64_t LL = (int64_t)L * L;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < shots * LL;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = i / LL;
    const int r = (int)(i - s * LL), x = r % L, y = r / L;
    const uint8_t* g = sig + s * LL;
    float acc[32];
#pragma unroll
    for (int co = 0; co < 32; ++co) acc[co] = sb[co];
#pragma unroll 1
    for (int tap = 0; tap < 9; ++tap) {
      const int nb = wrapL(y + tap / 3 - 1, L) * L + wrapL(x + tap % 3 - 1, L);
      if (g[nb]) {
#pragma unroll
        for (int co = 0; co < 32; ++co) acc[co] += sW[tap][co];
      }
    }
    uint4* o = reinterpret_cast<uint4*>(out + i * 32);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      uint4 w;
      w.x = pack_bf16(fmaxf(acc[8 * c + 0], 0.f), fmaxf(acc[8 * c + 1], 0.f));
      w.y = pack_bf16(fmaxf(acc[8 * c + 2], 0.f), fmaxf(acc[8 * c + 3], 0.f));
      w.z = pack_bf16(fmaxf(acc[8 * c + 4], 0.f), fmaxf(acc[8 * c + 5], 0.f));
      w.w = pack_bf16(fmaxf(acc[8 * c + 6], 0.f), fmaxf(acc[8 * c + 7], 0.f));
      o[c] = w;
    }
  }
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Implicit-GEMM 3x3 circular convolution, 32 input channels (bf16 NHWC, 64
// bytes per site), NT n-tiles of 8 output channels.  A warp computes 16
// consecutive sites (GEMM rows, possibly spanning shots) x 8*NT channels;
// K = 9 taps x 32 channels in k-steps of 16.  Weights sit in shared memory as
// [tap][co][ci pair] words with a row pitch of 20 words (conflict-free B
// fragment reads).  Epilogue by MODE:
//   kActs:      bias + ReLU, bf16 NHWC activations to `out`;
//   kLogits:    fp32 logits [shot][4][L][L] (channels < 4) to `logits`;
//   kProposals: per anyon (sig != 0) the channel of the largest logit if it is
//               positive, else 4; non-anyons 4; one byte per site to `prop`;
//   kGradMasked (training, backward data): no bias; the sum times the ReLU
//               mask (act > 0) of the layer input `act`, bf16 NHWC to `out`.
enum ConvMode { kActs = 0, kLogits = 1, kProposals = 2, kGradMasked = 3 };
constexpr int kWPitch = 20;

template <int NT, int MODE>
__global__ void __launch_bounds__(128) conv_mma_kernel(
    const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ Wg,
    const float* __restrict__ bias, int L, int64_t shots, __nv_bfloat16* __restrict__ out,
    float* __restrict__ logits, const uint8_t* __restrict__ sig, uint8_t* __restrict__ prop,
    const __nv_bfloat16* __restrict__ act) {
  constexpr int CO = 8 * NT;
  __shared__ uint32_t sW[9 * CO * kWPitch];
  __shared__ float sb[CO];
  for (int i = threadIdx.x; i < 9 * CO * 16; i += blockDim.x)
    sW[(i / 16) * kWPitch + (i % 16)] = reinterpret_cast<const uint32_t*>(Wg)[i];
  for (int i = threadIdx.x; i < CO; i += blockDim.x)
    sb[i] = MODE == kGradMasked ? 0.f : ((MODE == kActs || i < 4) ? bias[i] : 0.f);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int64_t LL = (int64_t)L * L, S = shots * LL;
  const int64_t tiles = (S + 15) / 16;
  const uint32_t* inw = reinterpret_cast<const uint32_t*>(in);  // 16 words per site
  for (int64_t tile = blockIdx.x * 4 + warp; tile < tiles; tile += (int64_t)gridDim.x * 4) {
    const int64_t s0 = tile * 16;
    // the two sites this lane feeds (rows g and g + 8 of the tile)
    int64_t site[2], shot[2];
    int xs[2], ys[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      site[h] = s0 + g + 8 * h;
      const int64_t sc = site[h] < S ? site[h] : S - 1;
      shot[h] = sc / LL;
      const int r = (int)(sc - shot[h] * LL);
      xs[h] = r % L;
      ys[h] = r / L;
    }
    float acc[NT][4];
#pragma unroll
    for (int n = 0; n < NT; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int dy = tap / 3 - 1, dx = tap % 3 - 1;
      int64_t nbw[2];
#pragma unroll
      for (int h = 0; h < 2; ++h)
        nbw[h] = (shot[h] * LL + wrapL(ys[h] + dy, L) * L + wrapL(xs[h] + dx, L)) * 16;
#pragma unroll
      for (int kh = 0; kh < 2; ++kh) {  // input channels 16 kh .. 16 kh + 15
        uint32_t a[4];
        a[0] = __ldg(inw + nbw[0] + kh * 8 + t);      // row g,     k = 2t, 2t+1
        a[1] = __ldg(inw + nbw[1] + kh * 8 + t);      // row g + 8
        a[2] = __ldg(inw + nbw[0] + kh * 8 + 4 + t);  // row g,     k = 2t+8, 2t+9
        a[3] = __ldg(inw + nbw[1] + kh * 8 + 4 + t);  // row g + 8
#pragma unroll
        for (int n = 0; n < NT; ++n) {
          const uint32_t* wr = sW + (tap * CO + n * 8 + g) * kWPitch + kh * 8 + t;
          mma_bf16(acc[n], a, wr[0], wr[4]);
        }
      }
    }
    // epilogue: rows g and g + 8, columns 2t and 2t + 1 of every n-tile
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const bool valid = site[h] < S;
      const int r = ys[h] * L + xs[h];
      if (MODE == kProposals) {
        // channels 0,1 sit in lane t = 0, channels 2,3 in lane t = 1 of the group
        const float v0 = acc[0][2 * h] + sb[2 * t], v1 = acc[0][2 * h + 1] + sb[2 * t + 1];
        const float w0 = __shfl_down_sync(0xFFFFFFFFu, v0, 1);
        const float w1 = __shfl_down_sync(0xFFFFFFFFu, v1, 1);
        if (t == 0 && valid) {
          const float z[4] = {v0, v1, w0, w1};
          float best = z[0];
          int bk = 0;
#pragma unroll
          for (int q = 1; q < 4; ++q)
            if (z[q] > best) {
              best = z[q];
              bk = q;
            }
          prop[site[h]] = (sig[site[h]] && best > 0.f) ? (uint8_t)bk : (uint8_t)4;
        }
        continue;
      }
      if (!valid) continue;
#pragma unroll
      for (int n = 0; n < NT; ++n) {
        const int c0 = n * 8 + 2 * t;
        const float v0 = acc[n][2 * h] + sb[c0], v1 = acc[n][2 * h + 1] + sb[c0 + 1];
        if (MODE == kLogits) {
          float* lb = logits + shot[h] * 4 * LL + r;
          if (c0 < 4) lb[(int64_t)c0 * LL] = v0;
          if (c0 + 1 < 4) lb[(int64_t)(c0 + 1) * LL] = v1;
        } else if (MODE == kGradMasked) {
          const __nv_bfloat162 m = reinterpret_cast<const __nv_bfloat162*>(act)[site[h] * 16 + c0 / 2];
          reinterpret_cast<uint32_t*>(out)[site[h] * 16 + c0 / 2] =
              pack_bf16(__bfloat162float(m.x) > 0.f ? v0 : 0.f, __bfloat162float(m.y) > 0.f ? v1 : 0.f);
        } else {
          reinterpret_cast<uint32_t*>(out)[site[h] * 16 + c0 / 2] =
              pack_bf16(fmaxf(v0, 0.f), fmaxf(v1, 0.f));
        }
      }
    }
  }
}

// Layer 1 as a table: its output at a site depends only on the 3 x 3 anyon
// pattern around it (bit tap = ky * 3 + kx).  Entry p holds the 32 bf16
// outputs for pattern p, summed in the order layer1_kernel uses (bias, the
// constant channel's taps, then the anyon taps), so both give the same bits.
__global__ void layer1_lut_kernel(const float* __restrict__ W1, const float* __restrict__ P,
                                  __nv_bfloat16* __restrict__ lut) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 512 * 32; i += gridDim.x * blockDim.x) {
    const int pat = i / 32, co = i % 32;
    float b = P[kB0 + co];
    for (int tap = 0; tap < 9; ++tap) b += W1[co * 18 + 9 + tap];
    for (int tap = 0; tap < 9; ++tap)
      if ((pat >> tap) & 1) b += W1[co * 18 + tap];
    lut[i] = __float2bfloat16_rn(fmaxf(b, 0.f));
  }
}

// ------------------------------------------------ inference (tcgen05) -----
//
// Layers 2-4 of the bf16 form on the fifth-generation tensor cores, for L a
// multiple of 128: a CTA takes tiles of 128 consecutive sites of one row and
// issues, for each of the 9 taps and both 16-channel halves, one tcgen05.mma
// (M = 128 sites, N = 32 output channels (16 for layer 4, 4 real), K = 16,
// bf16 operands, fp32 accumulator in tensor memory).  Both operands sit in
// shared memory in the no-swizzle K-major layout built from 8 x 16-byte core
// matrices: activations as [row y-1, y, y+1][channel octet][site x0-1 ..
// x0+128][8 bf16], so the operand of tap (dy, dx) is the same layout started
// dx sites (16 bytes) later and the periodic wrap lives in the halo sites;
// weights as [tap][channel octet][co][8 bf16].  The epilogue reads the
// accumulator with tcgen05.ld (one site per thread, one column per channel).

constexpr int kTcM = 128;            // sites per tile
constexpr int kTcRow = kTcM + 2;     // staged sites per row (one halo site each side)
constexpr int kTcThreads = 256;   // two warpgroups: each reads half the accumulator columns
constexpr long long kTcWaitCycles = 4000000000LL;

__device__ __forceinline__ uint32_t tc_smem(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start address, leading-dimension (K)
// and stride-dimension (M/N) byte offsets in 16-byte units, descriptor
// version 1 (bits 46-48), base offset 0, no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: D f32 (bits 4-5 = 1), A and B bf16
// (bits 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bit 17,
// M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t tc_idesc(int N, int M) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t adesc, uint64_t bdesc,
                                       uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   tc_smem(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_proxy_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tc_bar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ bool tc_bar_wait(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(tc_smem(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > kTcWaitCycles) return false;
  }
}

// cp.async 16-byte copy global -> shared, and its group fences
__device__ __forceinline__ void tc_cp16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc_smem(dst)), "l"(src) : "memory");
}
// the same through L1 (for small tables that stay cached)
__device__ __forceinline__ void tc_cp16_ca(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(tc_smem(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void tc_cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void tc_cp_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

constexpr int kTcStrip = 64;  // rows per work unit (a vertical strip of one 128-site column block)

// 16 consecutive accumulator columns of this thread's lane
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// NOUT = 32 (layers 2, 3; weights [tap][32][32]) or 16 (layer 4; weights
// [tap][8][32], channels 8..15 zero).  A work unit is a strip of kTcStrip
// rows of one 128-site column block of one shot: the staged rows live in a
// ring of four [octet][site][16 B] buffers; while tile y's accumulator is read
// out, the MMAs of tile y + 1 (rows y .. y + 2) run into the other of two
// accumulators and row y + 3 streams into the buffer tile y no longer needs.
// err: device word, set to 1 when a wait for the tensor core times out (the
// CTA then stops).
// FROM_SIG: the layer's input is layer 1 of the net, looked up while staging
// from the anyon bytes `sig` in the table `lut` of layer-1 outputs per 3 x 3
// anyon pattern, so the layer-1 activations never reach global memory.
template <int NOUT, int MODE, bool FROM_SIG>
__global__ void __launch_bounds__(kTcThreads) conv_tc_kernel(
    const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ Wg,
    const float* __restrict__ bias, int L, int64_t shots, __nv_bfloat16* __restrict__ out,
    float* __restrict__ logits, const uint8_t* __restrict__ sig, uint8_t* __restrict__ prop,
    unsigned int* __restrict__ err, const __nv_bfloat16* __restrict__ lut) {
  constexpr int CO_SRC = NOUT == 32 ? 32 : 8;
  constexpr uint32_t kRowBytes = 4 * kTcRow * 16;  // one staged row
  constexpr uint32_t kA = 4 * kRowBytes;           // ring of four rows
  constexpr uint32_t kB = 9 * 4 * NOUT * 16;       // weights
  extern __shared__ __align__(128) uint8_t sm[];
  uint8_t* sA = sm;
  uint8_t* sB = sm + kA;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kA + kB);  // [2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + kA + kB + 16);
  float* sbias = reinterpret_cast<float*>(sm + kA + kB + 32);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  for (int i = tid; i < 9 * NOUT * 4; i += kTcThreads) {
    const int tap = i / (NOUT * 4), rem = i % (NOUT * 4), co = rem / 4, oct = rem % 4;
    uint4 w = make_uint4(0, 0, 0, 0);
    if (co < CO_SRC)
      w = *reinterpret_cast<const uint4*>(Wg + ((size_t)(tap * CO_SRC + co) * 32 + oct * 8));
    *reinterpret_cast<uint4*>(sB + ((size_t)(tap * 4 + oct) * NOUT + co) * 16) = w;
  }
  for (int i = tid; i < NOUT; i += kTcThreads) sbias[i] = (MODE == kActs || i < 4) ? bias[i] : 0.f;
  if (tid == 0) {
    tc_bar_init(&bar[0]);
    tc_bar_init(&bar[1]);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     tc_smem(tslot)),
                 "r"(64)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;  // two accumulators: columns 0-31 and 32-63
  const uint32_t idesc = tc_idesc(NOUT, kTcM);
  const int64_t LL = (int64_t)L * L;
  const int xblocks = L / kTcM, strips = L / kTcStrip;
  const int64_t units = shots * xblocks * strips;
  uint32_t phase[2] = {0u, 0u};
  bool stop = false;

  // stage row yy of (shot, x0) into ring slot `slot` (asynchronous copies)
  auto stage = [&](int64_t shot, int yy, int x0, int slot) {
    yy = yy < 0 ? yy + L : (yy >= L ? yy - L : yy);
    uint8_t* dst = sA + (size_t)slot * kRowBytes;
    if (FROM_SIG) {
      // layer 1 (2 -> 32, ReLU, bf16) of every staged site: its 3 x 3 anyon
      // pattern indexes the 512-entry table `lut` (64 bytes per pattern)
      const uint8_t* g = sig + shot * LL;
      const int ym = yy == 0 ? L - 1 : yy - 1, yp = yy == L - 1 ? 0 : yy + 1;
      for (int j = tid; j < kTcRow; j += kTcThreads) {
        int xx = x0 + j - 1;
        xx = xx < 0 ? xx + L : (xx >= L ? xx - L : xx);
        const int xm = xx == 0 ? L - 1 : xx - 1, xp = xx == L - 1 ? 0 : xx + 1;
        const int rows[3] = {ym, yy, yp}, cols[3] = {xm, xx, xp};
        uint32_t idx = 0;
#pragma unroll
        for (int tap = 0; tap < 9; ++tap)
          idx |= (g[(int64_t)rows[tap / 3] * L + cols[tap % 3]] ? 1u : 0u) << tap;
        const __nv_bfloat16* src = lut + (size_t)idx * 32;
#pragma unroll
        for (int oct = 0; oct < 4; ++oct)
          tc_cp16_ca(dst + ((size_t)oct * kTcRow + j) * 16, src + oct * 8);
      }
      return;
    }
    const __nv_bfloat16* row = in + (shot * LL + (int64_t)yy * L) * 32;
    for (int i = tid; i < kTcRow * 4; i += kTcThreads) {
      const int j = i / 4, oct = i % 4;
      int xx = x0 + j - 1;
      xx = xx < 0 ? xx + L : (xx >= L ? xx - L : xx);
      tc_cp16(dst + ((size_t)oct * kTcRow + j) * 16, row + (int64_t)xx * 32 + oct * 8);
    }
  };
  // MMAs of tile y (rows y-1, y, y+1 in ring slots) into accumulator `acc`
  auto issue = [&](int y, int acc) {
    const uint32_t a0 = tc_smem(sA), b0 = tc_smem(sB);
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int dy = tap / 3, dx = tap % 3 - 1;
      const int slot = (y - 1 + dy + 4 * L) & 3;  // ring slot of row y - 1 + dy
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint32_t aaddr =
            a0 + (uint32_t)slot * kRowBytes + ((uint32_t)((2 * h) * kTcRow + 1 + dx)) * 16;
        const uint32_t baddr = b0 + ((uint32_t)((tap * 4 + 2 * h) * NOUT)) * 16;
        tc_mma(tmem + (uint32_t)(acc * 32), tc_desc(aaddr, kTcRow * 16, 128),
               tc_desc(baddr, NOUT * 16, 128), idesc, (tap | h) != 0);
      }
    }
    tc_commit(&bar[acc]);
  };

  for (int64_t u = blockIdx.x; u < units && !stop; u += gridDim.x) {
    const int64_t shot = u / ((int64_t)xblocks * strips);
    const int rem = (int)(u - shot * (int64_t)xblocks * strips);
    const int x0 = (rem % xblocks) * kTcM, y0 = (rem / xblocks) * kTcStrip;
    // prologue: rows y0-1 .. y0+1, then tile y0's MMAs; row y0+2 in flight
    for (int r = -1; r <= 1; ++r) stage(shot, y0 + r, x0, (y0 + r + 4 * L) & 3);
    tc_cp_commit();
    tc_cp_wait_all();
    tc_fence_proxy_shared();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      issue(y0, 0);
    }
    stage(shot, y0 + 2, x0, (y0 + 2 + 4 * L) & 3);
    tc_cp_commit();
    for (int i = 0; i < kTcStrip; ++i) {
      const int y = y0 + i, acc = i & 1;
      // row y + 2 has landed: tile y + 1 can start while tile y is read out
      tc_cp_wait_all();
      tc_fence_proxy_shared();
      tc_fence_before();
      __syncthreads();
      if (tid == 0 && i + 1 < kTcStrip) {
        tc_fence_after();
        issue(y + 1, acc ^ 1);
      }
      const bool ok = tc_bar_wait(&bar[acc], phase[acc]);
      if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicOr(err, 1u);
        (void)tc_bar_wait(&bar[acc], phase[acc]);
        (void)tc_bar_wait(&bar[acc ^ 1], phase[acc ^ 1]);
        stop = true;
        break;
      }
      phase[acc] ^= 1u;
      // tile y no longer needs row y - 1: its slot takes row y + 3
      if (i + 2 < kTcStrip) stage(shot, y + 3, x0, (y + 3 + 4 * L) & 3);
      tc_cp_commit();
      tc_fence_after();
      // epilogue: thread (warp w, lane l) holds site x0 + 32 (w % 4) + l; the
      // warpgroup w / 4 reads accumulator columns 16 (w / 4) .. + 15
      const int x = x0 + 32 * (warp & 3) + lane, half = warp >> 2;
      const int64_t site = shot * LL + (int64_t)y * L + x;
      float v[16];
      tc_ld16(tmem + (uint32_t)(acc * 32 + 16 * half) + ((uint32_t)(32 * (warp & 3)) << 16), v);
      if (MODE == kActs) {
        uint32_t w[8];
#pragma unroll
        for (int c = 0; c < 8; ++c)
          w[c] = pack_bf16(fmaxf(v[2 * c] + sbias[16 * half + 2 * c], 0.f),
                           fmaxf(v[2 * c + 1] + sbias[16 * half + 2 * c + 1], 0.f));
        uint4* o = reinterpret_cast<uint4*>(out + site * 32 + 16 * half);
        o[0] = make_uint4(w[0], w[1], w[2], w[3]);
        o[1] = make_uint4(w[4], w[5], w[6], w[7]);
      } else if (half == 0) {
        const float z[4] = {v[0] + sbias[0], v[1] + sbias[1], v[2] + sbias[2], v[3] + sbias[3]};
        if (MODE == kLogits) {
          float* lb = logits + shot * 4 * LL + (int64_t)y * L + x;
#pragma unroll
          for (int k = 0; k < 4; ++k) lb[(int64_t)k * LL] = z[k];
        } else {
          float best = z[0];
          int bk = 0;
#pragma unroll
          for (int q = 1; q < 4; ++q)
            if (z[q] > best) {
              best = z[q];
              bk = q;
            }
          prop[site] = (sig[site] && best > 0.f) ? (uint8_t)bk : (uint8_t)4;
        }
      }
    }
    tc_cp_wait_all();
    __syncthreads();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(64)
                 : "memory");
}

template <int NOUT>
constexpr size_t tc_smem_bytes() {
  return 4 * 4 * kTcRow * 16 + 9 * 4 * NOUT * 16 + 32 + 4 * NOUT;
}

// Warp-specialised form of the same convolution (the same MMAs in the same
// order, so the same bits): the roles hand rows and accumulators to one
// another through mbarriers instead of block barriers, so that the staging of
// later rows, the MMAs of the next tile and the read-out of the last one
// overlap.  Its activations use a planar layout of their own,
// [shot][y][channel octet][x][8 bf16], so that a staged row is four
// contiguous 2 KB runs (plus one halo site at either end) and the epilogue's
// stores are contiguous across a warp.
//   * producers stage the rows of the CTA's work units, in order, into a ring
//     of row buffers (WsShape).  From planar activations one thread issues bulk
//     copies (cp.async.bulk, completion by transaction count on full[slot]);
//     for layer 2 the kWsProd producer warps gather layer 1 from the table
//     with cp.async, each thread publishing a row kWsLag rows after issuing
//     it, once its copies have landed (wait_group, proxy fence, arrive).  A
//     slot is refilled only after the MMAs that read it are complete
//     (empty[slot], tcgen05.commit);
//   * one MMA thread issues the 18 MMAs of each tile into one of two TMEM
//     accumulators (once its epilogue is drained: acc_empty) and commits them
//     to acc_full and to the release of the ring slot the tile reads last;
//   * eight epilogue warps (two per TMEM lane quarter, one per column half)
//     read each accumulator, free it, and apply bias and ReLU / write logits
//     or proposals.
// Every wait is bounded; a timeout sets err and a stop flag that every role
// polls, and the CTA drains its MMAs before freeing the TMEM.
// Ring of staged rows and resident CTAs per SM, per form: the layer that
// gathers layer 1 from the table (FROM_SIG) keeps more of the SM's L1 for the
// table with two CTAs and a ring of 8; the bulk-copied layers run three CTAs
// with a ring of 6 (registers, shared and tensor memory all fit)
template <bool FROM_SIG>
struct WsShape {
  static constexpr int R = FROM_SIG ? 8 : 6;
  static constexpr int ctas = FROM_SIG ? 2 : 3;
};
constexpr int kWsLag = 4;        // rows a producer thread keeps in flight (<= ring - 3)
constexpr int kWsEpi = 8;        // epilogue warps
constexpr int kWsProd = 4;       // producer warps
constexpr int kWsThreads = 32 * (kWsEpi + kWsProd + 1);
constexpr int kWsMmaWarp = kWsEpi + kWsProd;
static_assert(kWsLag <= WsShape<true>::R - 3,
              "a producer must be able to publish the rows the MMA waits for");

__device__ __forceinline__ void ws_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc_smem(bar)) : "memory");
}
__device__ __forceinline__ void ws_bar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_smem(bar)), "r"(count)
               : "memory");
}
// bounded wait on phase `parity`; on timeout, or when another role has already
// stopped, returns false
__device__ __forceinline__ bool ws_wait(uint64_t* bar, uint32_t parity, volatile int* stop) {
  const long long t0 = clock64();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(tc_smem(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if (*stop) return false;
    if (clock64() - t0 > kTcWaitCycles) {
      *stop = 1;
      return false;
    }
  }
}

__device__ __forceinline__ void mbar_expect_tx_ws(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc_smem(bar)),
               "r"(bytes)
               : "memory");
}
// Bulk copy global -> this CTA's shared memory, completion counted on bar.
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s_ws(void* dst, const void* src, uint32_t bytes,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          tc_smem(dst)),
      "l"(src), "r"(bytes), "r"(tc_smem(bar))
      : "memory");
}

template <int NOUT, int MODE, bool FROM_SIG>
__global__ void __launch_bounds__(kWsThreads, WsShape<FROM_SIG>::ctas) conv_ws_kernel(
    const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ Wg,
    const float* __restrict__ bias, int L, int64_t shots, __nv_bfloat16* __restrict__ out,
    float* __restrict__ logits, const uint8_t* __restrict__ sig, uint8_t* __restrict__ prop,
    unsigned int* __restrict__ err, const __nv_bfloat16* __restrict__ lut) {
  constexpr int CO_SRC = NOUT == 32 ? 32 : 8;
  constexpr int kR = WsShape<FROM_SIG>::R;         // staged rows in the ring
  constexpr uint32_t kRowBytes = 4 * kTcRow * 16;  // one staged row
  constexpr uint32_t kA = kR * kRowBytes;          // the ring
  constexpr uint32_t kB = 9 * 4 * NOUT * 16;       // weights
  extern __shared__ __align__(128) uint8_t sm[];
  uint8_t* sA = sm;
  uint8_t* sB = sm + kA;
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + kA + kB);  // [kR]
  uint64_t* empty = full + kR;                               // [kR]
  uint64_t* acc_full = empty + kR;                           // [2]
  uint64_t* acc_empty = acc_full + 2;                          // [2]
  uint64_t* drained = acc_empty + 2;                           // [1]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(drained + 1);
  volatile int* stop = reinterpret_cast<volatile int*>(tslot + 1);
  float* sbias = reinterpret_cast<float*>(tslot + 4);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  for (int i = tid; i < 9 * NOUT * 4; i += kWsThreads) {
    const int tap = i / (NOUT * 4), rem = i % (NOUT * 4), co = rem / 4, oct = rem % 4;
    uint4 w = make_uint4(0, 0, 0, 0);
    if (co < CO_SRC)
      w = *reinterpret_cast<const uint4*>(Wg + ((size_t)(tap * CO_SRC + co) * 32 + oct * 8));
    *reinterpret_cast<uint4*>(sB + ((size_t)(tap * 4 + oct) * NOUT + co) * 16) = w;
  }
  for (int i = tid; i < NOUT; i += kWsThreads) sbias[i] = (MODE == kActs || i < 4) ? bias[i] : 0.f;
  if (tid == 0) {
    for (int k = 0; k < kR; ++k) {
      ws_bar_init(&full[k], FROM_SIG ? 32 * kWsProd : 1);
      ws_bar_init(&empty[k], 1);
    }
    for (int k = 0; k < 2; ++k) {
      ws_bar_init(&acc_full[k], 1);
      ws_bar_init(&acc_empty[k], kWsEpi);
    }
    ws_bar_init(drained, 1);
    *stop = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     tc_smem(tslot)),
                 "r"(64)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // the weights are read by the tensor core (async proxy)
  tc_fence_proxy_shared();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;  // two accumulators: columns 0-31 and 32-63
  const int64_t LL = (int64_t)L * L;
  const int xblocks = L / kTcM, strips = L / kTcStrip;
  const int64_t units = shots * xblocks * strips;
  auto unit_of = [&](int64_t u, int64_t& shot, int& x0, int& y0) {
    shot = u / ((int64_t)xblocks * strips);
    const int rem = (int)(u - shot * (int64_t)xblocks * strips);
    x0 = (rem % xblocks) * kTcM;
    y0 = (rem / xblocks) * kTcStrip;
  };

  if (!FROM_SIG && warp >= kWsEpi && warp < kWsMmaWarp) {
    // ================= producer (one thread): bulk copies of planar rows; the
    // other producer warps have no work in this form
    if (warp == kWsEpi && lane == 0) {
      int64_t e = 0;
      for (int64_t u = blockIdx.x; u < units && !*stop; u += gridDim.x) {
        int64_t shot;
        int x0, y0;
        unit_of(u, shot, x0, y0);
        const int xl = x0 == 0 ? L - 1 : x0 - 1, xr = x0 + kTcM == L ? 0 : x0 + kTcM;
        int r = -1;
        for (; r <= kTcStrip; ++r, ++e) {
          const int slot = (int)(e % kR);
          if (e >= kR && !ws_wait(&empty[slot], (uint32_t)((e / kR - 1) & 1), stop)) break;
          int yy = y0 + r;
          yy = yy < 0 ? yy + L : (yy >= L ? yy - L : yy);
          uint8_t* dst = sA + (size_t)slot * kRowBytes;
          mbar_expect_tx_ws(&full[slot], kRowBytes);
#pragma unroll
          for (int oct = 0; oct < 4; ++oct) {
            const __nv_bfloat16* src = in + (((shot * L + yy) * 4 + oct) * (int64_t)L) * 8;
            uint8_t* d = dst + (size_t)oct * kTcRow * 16;
            bulk_g2s_ws(d + 16, src + (int64_t)x0 * 8, kTcM * 16, &full[slot]);
            bulk_g2s_ws(d, src + (int64_t)xl * 8, 16, &full[slot]);
            bulk_g2s_ws(d + (kTcRow - 1) * 16, src + (int64_t)xr * 8, 16, &full[slot]);
          }
        }
        if (r <= kTcStrip) break;  // stopped
      }
      // no copy may still be landing when the CTA exits: wait (bounded) for the
      // last entry of every slot (a no-op unless the CTA stopped early)
      for (int64_t f = e > kR ? e - kR : 0; f < e; ++f)
        (void)tc_bar_wait(&full[f % kR], (uint32_t)((f / kR) & 1));
    }
    __syncwarp();
  } else if (FROM_SIG && warp >= kWsEpi && warp < kWsMmaWarp) {
    // ================= producers: rows y0 - 1 .. y0 + kTcStrip of every unit,
    // layer 1 gathered from the table
    const int pt = tid - 32 * kWsEpi;  // 0 .. 32 * kWsProd - 1
    int64_t e = 0;                     // entries issued by this CTA
    for (int64_t u = blockIdx.x; u < units && !*stop; u += gridDim.x) {
      int64_t shot;
      int x0, y0;
      unit_of(u, shot, x0, y0);
      for (int r = -1; r <= kTcStrip && !*stop; ++r, ++e) {
        const int slot = (int)(e % kR);
        if (e >= kR && !ws_wait(&empty[slot], (uint32_t)((e / kR - 1) & 1), stop)) break;
        int yy = y0 + r;
        yy = yy < 0 ? yy + L : (yy >= L ? yy - L : yy);
        uint8_t* dst = sA + (size_t)slot * kRowBytes;
        {
          const uint8_t* g = sig + shot * LL;
          const int ym = yy == 0 ? L - 1 : yy - 1, yp = yy == L - 1 ? 0 : yy + 1;
          for (int j = pt; j < kTcRow; j += 32 * kWsProd) {
            int xx = x0 + j - 1;
            xx = xx < 0 ? xx + L : (xx >= L ? xx - L : xx);
            const int xm = xx == 0 ? L - 1 : xx - 1, xp = xx == L - 1 ? 0 : xx + 1;
            const int rows[3] = {ym, yy, yp}, cols[3] = {xm, xx, xp};
            uint32_t idx = 0;
#pragma unroll
            for (int tap = 0; tap < 9; ++tap)
              idx |= (g[(int64_t)rows[tap / 3] * L + cols[tap % 3]] ? 1u : 0u) << tap;
            const __nv_bfloat16* src = lut + (size_t)idx * 32;
#pragma unroll
            for (int oct = 0; oct < 4; ++oct)
              tc_cp16_ca(dst + ((size_t)oct * kTcRow + j) * 16, src + oct * 8);
          }
        }
        tc_cp_commit();
        if (e >= kWsLag) {
          // the copies of entry e - kWsLag have landed: publish it
          asm volatile("cp.async.wait_group %0;" ::"n"(kWsLag) : "memory");
          tc_fence_proxy_shared();
          ws_arrive(&full[(e - kWsLag) % kR]);
        }
      }
    }
    // publish the entries still in flight
    tc_cp_wait_all();
    tc_fence_proxy_shared();
    for (int64_t f = e > kWsLag ? e - kWsLag : 0; f < e; ++f) ws_arrive(&full[f % kR]);
  } else if (warp == kWsMmaWarp) {
    // ================= MMA issue (one thread)
    if (lane == 0) {
      const uint32_t idesc = tc_idesc(NOUT, kTcM);
      const uint32_t a0 = tc_smem(sA), b0 = tc_smem(sB);
      int64_t e = 0, T = 0;  // first entry of the current unit, tiles issued
      bool ok = true;
      for (int64_t u = blockIdx.x; u < units && ok; u += gridDim.x) {
        for (int j = 0; j < kTcStrip && ok; ++j, ++T) {
          const int64_t eb = e + j;  // entries eb .. eb + 2: rows y - 1 .. y + 1
#pragma unroll
          for (int dy = 0; dy < 3; ++dy)
            ok = ok && ws_wait(&full[(eb + dy) % kR], (uint32_t)(((eb + dy) / kR) & 1), stop);
          const int acc = (int)(T & 1);
          if (ok && T >= 2) ok = ws_wait(&acc_empty[acc], (uint32_t)(((T >> 1) - 1) & 1), stop);
          if (!ok) break;
          tc_fence_after();
#pragma unroll
          for (int tap = 0; tap < 9; ++tap) {
            const int dy = tap / 3, dx = tap % 3 - 1;
            const uint32_t slot = (uint32_t)((eb + dy) % kR);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const uint32_t aaddr =
                  a0 + slot * kRowBytes + ((uint32_t)((2 * h) * kTcRow + 1 + dx)) * 16;
              const uint32_t baddr = b0 + ((uint32_t)((tap * 4 + 2 * h) * NOUT)) * 16;
              tc_mma(tmem + (uint32_t)(acc * 32), tc_desc(aaddr, kTcRow * 16, 128),
                     tc_desc(baddr, NOUT * 16, 128), idesc, (tap | h) != 0);
            }
          }
          tc_commit(&acc_full[acc]);
          tc_commit(&empty[eb % kR]);  // no later tile reads entry eb
          if (j == kTcStrip - 1) {       // nor the unit's last two rows
            tc_commit(&empty[(eb + 1) % kR]);
            tc_commit(&empty[(eb + 2) % kR]);
          }
        }
        e += kTcStrip + 2;
      }
      // every MMA issued so far has completed before the TMEM is freed
      tc_commit(drained);
      if (!tc_bar_wait(drained, 0)) *stop = 1;
    }
    __syncwarp();
  } else {
    // ================= epilogue: warp w reads TMEM lanes 32 (w % 4) .., columns
    // 16 (w / 4) .. + 15 of the tile's accumulator
    const int half = warp >> 2;
    int64_t T = 0;
    for (int64_t u = blockIdx.x; u < units && !*stop; u += gridDim.x) {
      int64_t shot;
      int x0, y0;
      unit_of(u, shot, x0, y0);
      bool ok = true;
      for (int j = 0; j < kTcStrip; ++j, ++T) {
        const int acc = (int)(T & 1);
        ok = ws_wait(&acc_full[acc], (uint32_t)((T >> 1) & 1), stop);
        if (!__all_sync(0xffffffffu, ok)) {
          ok = false;
          break;
        }
        tc_fence_after();
        float v[16];
        tc_ld16(tmem + (uint32_t)(acc * 32 + 16 * half) + ((uint32_t)(32 * (warp & 3)) << 16), v);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) ws_arrive(&acc_empty[acc]);
        const int y = y0 + j, x = x0 + 32 * (warp & 3) + lane;
        const int64_t site = shot * LL + (int64_t)y * L + x;
        if (MODE == kActs) {
          uint32_t w[8];
#pragma unroll
          for (int c = 0; c < 8; ++c)
            w[c] = pack_bf16(fmaxf(v[2 * c] + sbias[16 * half + 2 * c], 0.f),
                             fmaxf(v[2 * c + 1] + sbias[16 * half + 2 * c + 1], 0.f));
          // planar: octets 2 half and 2 half + 1 of site x
          const int64_t rowo = (shot * L + y) * 4 + 2 * half;
          *reinterpret_cast<uint4*>(out + (rowo * L + x) * 8) = make_uint4(w[0], w[1], w[2], w[3]);
          *reinterpret_cast<uint4*>(out + ((rowo + 1) * L + x) * 8) =
              make_uint4(w[4], w[5], w[6], w[7]);
        } else if (half == 0) {
          const float z[4] = {v[0] + sbias[0], v[1] + sbias[1], v[2] + sbias[2], v[3] + sbias[3]};
          if (MODE == kLogits) {
            float* lb = logits + shot * 4 * LL + (int64_t)y * L + x;
#pragma unroll
            for (int k = 0; k < 4; ++k) lb[(int64_t)k * LL] = z[k];
          } else {
            float best = z[0];
            int bk = 0;
#pragma unroll
            for (int q = 1; q < 4; ++q)
              if (z[q] > best) {
                best = z[q];
                bk = q;
              }
            prop[site] = (sig[site] && best > 0.f) ? (uint8_t)bk : (uint8_t)4;
          }
        }
      }
      if (!ok) break;
    }
  }
  __syncthreads();
  if (tid == 0 && *stop) atomicOr(err, 1u);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(64)
                 : "memory");
}

template <int NOUT, bool FROM_SIG>
constexpr size_t ws_smem_bytes() {
  constexpr int R = WsShape<FROM_SIG>::R;
  return (size_t)R * 4 * kTcRow * 16 + 9 * 4 * NOUT * 16 + (2 * R + 5) * 8 + 16 + 4 * NOUT;
}

// two floats -> two E4M3 bytes (lo in the low byte), saturating
__device__ __forceinline__ uint16_t pack_e4m3x2(float lo, float hi) {
  return (uint16_t)__nv_cvt_float2_to_fp8x2(make_float2(lo, hi), __NV_SATFINITE, __NV_E4M3);
}

// FP8 (E4M3) form of the warp-specialised convolution (tcgen05.mma
// kind::f8f6f4).  K = 32 e4m3 values per MMA are two 16-byte planes, the same
// byte geometry as K = 16 bf16, so the descriptors are those of the bf16 form
// and a tap is one MMA.  Activations are planar as [shot][y][16-channel group]
// [x][16 bytes]; the epilogue dequantises with s_in * s_co (the weight
// scale of its output channel), adds the bias, and requantises to e4m3 with the
// next layer's scale, as the mma.sync FP8 kernel does.
__host__ __device__ constexpr uint32_t tc_idesc_e4m3(int N, int M) {
  // D f32 (bits 4-5 = 1), A and B E4M3 (bits 7-9 and 10-12 = 0), K-major, N >> 3, M >> 4
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma_e4m3(uint32_t tmem, uint64_t adesc, uint64_t bdesc,
                                            uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// layer 1 of the FP8 form for every 3 x 3 anyon pattern: e4m3(relu(.) / s_out),
// summed in the order of layer1_fp8_kernel; 32 bytes per pattern
__global__ void layer1_lut8_kernel(const float* __restrict__ W1, const float* __restrict__ P,
                                   float inv_s_out, uint8_t* __restrict__ lut8) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 512 * 16; i += gridDim.x * blockDim.x) {
    const int pat = i / 16, co = 2 * (i % 16);
    float b[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      b[k] = P[kB0 + co + k];
      for (int tap = 0; tap < 9; ++tap) b[k] += W1[(co + k) * 18 + 9 + tap];
      for (int tap = 0; tap < 9; ++tap)
        if ((pat >> tap) & 1) b[k] += W1[(co + k) * 18 + tap];
    }
    reinterpret_cast<uint16_t*>(lut8)[i] =
        pack_e4m3x2(fmaxf(b[0], 0.f) * inv_s_out, fmaxf(b[1], 0.f) * inv_s_out);
  }
}

template <int NOUT, int MODE, bool FROM_SIG>
__global__ void __launch_bounds__(kWsThreads, WsShape<FROM_SIG>::ctas) conv_ws8_kernel(
    const uint8_t* __restrict__ in, const uint8_t* __restrict__ Wq,
    const float* __restrict__ wscale, const float* __restrict__ bias, float s_in,
    float inv_s_out, int L, int64_t shots, uint8_t* __restrict__ out,
    float* __restrict__ logits, const uint8_t* __restrict__ sig, uint8_t* __restrict__ prop,
    unsigned int* __restrict__ err, const uint8_t* __restrict__ lut8) {
  constexpr int CO_SRC = NOUT == 32 ? 32 : 8;
  constexpr int kR = WsShape<FROM_SIG>::R;         // staged rows in the ring
  constexpr uint32_t kRowBytes = 2 * kTcRow * 16;  // one staged row: two 16-channel planes
  constexpr uint32_t kA = kR * kRowBytes;          // the ring
  constexpr uint32_t kB = 9 * 2 * NOUT * 16;       // weights
  extern __shared__ __align__(128) uint8_t sm[];
  uint8_t* sA = sm;
  uint8_t* sB = sm + kA;
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + kA + kB);  // [kR]
  uint64_t* empty = full + kR;                               // [kR]
  uint64_t* acc_full = empty + kR;                           // [2]
  uint64_t* acc_empty = acc_full + 2;                          // [2]
  uint64_t* drained = acc_empty + 2;                           // [1]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(drained + 1);
  volatile int* stop = reinterpret_cast<volatile int*>(tslot + 1);
  float* sbias = reinterpret_cast<float*>(tslot + 4);
  float* sscale = sbias + NOUT;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // weights [tap][co][32 ci] bytes -> [tap][group][co][16 bytes]
  for (int i = tid; i < 9 * NOUT * 2; i += kWsThreads) {
    const int tap = i / (NOUT * 2), rem = i % (NOUT * 2), co = rem / 2, grp = rem % 2;
    uint4 w = make_uint4(0, 0, 0, 0);
    if (co < CO_SRC)
      w = *reinterpret_cast<const uint4*>(Wq + ((size_t)(tap * CO_SRC + co) * 32 + grp * 16));
    *reinterpret_cast<uint4*>(sB + ((size_t)(tap * 2 + grp) * NOUT + co) * 16) = w;
  }
  for (int i = tid; i < NOUT; i += kWsThreads) {
    const bool real = MODE == kActs || i < 4;
    sbias[i] = real ? bias[i] : 0.f;
    sscale[i] = real ? s_in * wscale[i] : 0.f;
  }
  if (tid == 0) {
    for (int k = 0; k < kR; ++k) {
      ws_bar_init(&full[k], FROM_SIG ? 32 * kWsProd : 1);
      ws_bar_init(&empty[k], 1);
    }
    for (int k = 0; k < 2; ++k) {
      ws_bar_init(&acc_full[k], 1);
      ws_bar_init(&acc_empty[k], kWsEpi);
    }
    ws_bar_init(drained, 1);
    *stop = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     tc_smem(tslot)),
                 "r"(64)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_proxy_shared();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;  // two accumulators: columns 0-31 and 32-63
  const int64_t LL = (int64_t)L * L;
  const int xblocks = L / kTcM, strips = L / kTcStrip;
  const int64_t units = shots * xblocks * strips;
  auto unit_of = [&](int64_t u, int64_t& shot, int& x0, int& y0) {
    shot = u / ((int64_t)xblocks * strips);
    const int rem = (int)(u - shot * (int64_t)xblocks * strips);
    x0 = (rem % xblocks) * kTcM;
    y0 = (rem / xblocks) * kTcStrip;
  };

  if (!FROM_SIG && warp >= kWsEpi && warp < kWsMmaWarp) {
    // ================= producer (one thread): bulk copies of planar rows
    if (warp == kWsEpi && lane == 0) {
      int64_t e = 0;
      for (int64_t u = blockIdx.x; u < units && !*stop; u += gridDim.x) {
        int64_t shot;
        int x0, y0;
        unit_of(u, shot, x0, y0);
        const int xl = x0 == 0 ? L - 1 : x0 - 1, xr = x0 + kTcM == L ? 0 : x0 + kTcM;
        int r = -1;
        for (; r <= kTcStrip; ++r, ++e) {
          const int slot = (int)(e % kR);
          if (e >= kR && !ws_wait(&empty[slot], (uint32_t)((e / kR - 1) & 1), stop)) break;
          int yy = y0 + r;
          yy = yy < 0 ? yy + L : (yy >= L ? yy - L : yy);
          uint8_t* dst = sA + (size_t)slot * kRowBytes;
          mbar_expect_tx_ws(&full[slot], kRowBytes);
#pragma unroll
          for (int grp = 0; grp < 2; ++grp) {
            const uint8_t* src = in + (((shot * L + yy) * 2 + grp) * (int64_t)L) * 16;
            uint8_t* d = dst + (size_t)grp * kTcRow * 16;
            bulk_g2s_ws(d + 16, src + (int64_t)x0 * 16, kTcM * 16, &full[slot]);
            bulk_g2s_ws(d, src + (int64_t)xl * 16, 16, &full[slot]);
            bulk_g2s_ws(d + (kTcRow - 1) * 16, src + (int64_t)xr * 16, 16, &full[slot]);
          }
        }
        if (r <= kTcStrip) break;  // stopped
      }
      // no copy may still be landing when the CTA exits
      for (int64_t f = e > kR ? e - kR : 0; f < e; ++f)
        (void)tc_bar_wait(&full[f % kR], (uint32_t)((f / kR) & 1));
    }
    __syncwarp();
  } else if (FROM_SIG && warp >= kWsEpi && warp < kWsMmaWarp) {
    // ================= producers: layer 1 gathered from the e4m3 table
    const int pt = tid - 32 * kWsEpi;
    int64_t e = 0;
    for (int64_t u = blockIdx.x; u < units && !*stop; u += gridDim.x) {
      int64_t shot;
      int x0, y0;
      unit_of(u, shot, x0, y0);
      for (int r = -1; r <= kTcStrip && !*stop; ++r, ++e) {
        const int slot = (int)(e % kR);
        if (e >= kR && !ws_wait(&empty[slot], (uint32_t)((e / kR - 1) & 1), stop)) break;
        int yy = y0 + r;
        yy = yy < 0 ? yy + L : (yy >= L ? yy - L : yy);
        uint8_t* dst = sA + (size_t)slot * kRowBytes;
        const uint8_t* g = sig + shot * LL;
        const int ym = yy == 0 ? L - 1 : yy - 1, yp = yy == L - 1 ? 0 : yy + 1;
        for (int j = pt; j < kTcRow; j += 32 * kWsProd) {
          int xx = x0 + j - 1;
          xx = xx < 0 ? xx + L : (xx >= L ? xx - L : xx);
          const int xm = xx == 0 ? L - 1 : xx - 1, xp = xx == L - 1 ? 0 : xx + 1;
          const int rows[3] = {ym, yy, yp}, cols[3] = {xm, xx, xp};
          uint32_t idx = 0;
#pragma unroll
          for (int tap = 0; tap < 9; ++tap)
            idx |= (g[(int64_t)rows[tap / 3] * L + cols[tap % 3]] ? 1u : 0u) << tap;
          const uint8_t* src = lut8 + (size_t)idx * 32;
          tc_cp16_ca(dst + (size_t)j * 16, src);
          tc_cp16_ca(dst + ((size_t)kTcRow + j) * 16, src + 16);
        }
        tc_cp_commit();
        if (e >= kWsLag) {
          asm volatile("cp.async.wait_group %0;" ::"n"(kWsLag) : "memory");
          tc_fence_proxy_shared();
          ws_arrive(&full[(e - kWsLag) % kR]);
        }
      }
    }
    tc_cp_wait_all();
    tc_fence_proxy_shared();
    for (int64_t f = e > kWsLag ? e - kWsLag : 0; f < e; ++f) ws_arrive(&full[f % kR]);
  } else if (warp == kWsMmaWarp) {
    // ================= MMA issue (one thread): one K = 32 MMA per tap
    if (lane == 0) {
      const uint32_t idesc = tc_idesc_e4m3(NOUT, kTcM);
      const uint32_t a0 = tc_smem(sA), b0 = tc_smem(sB);
      int64_t e = 0, T = 0;
      bool ok = true;
      for (int64_t u = blockIdx.x; u < units && ok; u += gridDim.x) {
        for (int j = 0; j < kTcStrip && ok; ++j, ++T) {
          const int64_t eb = e + j;
#pragma unroll
          for (int dy = 0; dy < 3; ++dy)
            ok = ok && ws_wait(&full[(eb + dy) % kR], (uint32_t)(((eb + dy) / kR) & 1), stop);
          const int acc = (int)(T & 1);
          if (ok && T >= 2) ok = ws_wait(&acc_empty[acc], (uint32_t)(((T >> 1) - 1) & 1), stop);
          if (!ok) break;
          tc_fence_after();
#pragma unroll
          for (int tap = 0; tap < 9; ++tap) {
            const int dy = tap / 3, dx = tap % 3 - 1;
            const uint32_t slot = (uint32_t)((eb + dy) % kR);
            const uint32_t aaddr = a0 + slot * kRowBytes + (uint32_t)(1 + dx) * 16;
            const uint32_t baddr = b0 + (uint32_t)(tap * 2 * NOUT) * 16;
            tc_mma_e4m3(tmem + (uint32_t)(acc * 32), tc_desc(aaddr, kTcRow * 16, 128),
                        tc_desc(baddr, NOUT * 16, 128), idesc, tap != 0);
          }
          tc_commit(&acc_full[acc]);
          tc_commit(&empty[eb % kR]);
          if (j == kTcStrip - 1) {
            tc_commit(&empty[(eb + 1) % kR]);
            tc_commit(&empty[(eb + 2) % kR]);
          }
        }
        e += kTcStrip + 2;
      }
      tc_commit(drained);
      if (!tc_bar_wait(drained, 0)) *stop = 1;
    }
    __syncwarp();
  } else {
    // ================= epilogue: warp w reads TMEM lanes 32 (w % 4) .., columns
    // 16 (w / 4) .. + 15 (output channels of one 16-channel group)
    const int half = warp >> 2;
    int64_t T = 0;
    for (int64_t u = blockIdx.x; u < units && !*stop; u += gridDim.x) {
      int64_t shot;
      int x0, y0;
      unit_of(u, shot, x0, y0);
      bool ok = true;
      for (int j = 0; j < kTcStrip; ++j, ++T) {
        const int acc = (int)(T & 1);
        ok = ws_wait(&acc_full[acc], (uint32_t)((T >> 1) & 1), stop);
        if (!__all_sync(0xffffffffu, ok)) {
          ok = false;
          break;
        }
        tc_fence_after();
        float v[16];
        tc_ld16(tmem + (uint32_t)(acc * 32 + 16 * half) + ((uint32_t)(32 * (warp & 3)) << 16), v);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) ws_arrive(&acc_empty[acc]);
        const int y = y0 + j, x = x0 + 32 * (warp & 3) + lane;
        const int64_t site = shot * LL + (int64_t)y * L + x;
        if (MODE == kActs) {
          uint32_t w[4];
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int co = 16 * half + 4 * c;
            const uint32_t lo =
                pack_e4m3x2(fmaxf(v[4 * c] * sscale[co] + sbias[co], 0.f) * inv_s_out,
                            fmaxf(v[4 * c + 1] * sscale[co + 1] + sbias[co + 1], 0.f) * inv_s_out);
            const uint32_t hi =
                pack_e4m3x2(fmaxf(v[4 * c + 2] * sscale[co + 2] + sbias[co + 2], 0.f) * inv_s_out,
                            fmaxf(v[4 * c + 3] * sscale[co + 3] + sbias[co + 3], 0.f) * inv_s_out);
            w[c] = lo | (hi << 16);
          }
          *reinterpret_cast<uint4*>(out + (((shot * L + y) * 2 + half) * (int64_t)L + x) * 16) =
              make_uint4(w[0], w[1], w[2], w[3]);
        } else if (half == 0) {
          float z[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) z[k] = v[k] * sscale[k] + sbias[k];
          if (MODE == kLogits) {
            float* lb = logits + shot * 4 * LL + (int64_t)y * L + x;
#pragma unroll
            for (int k = 0; k < 4; ++k) lb[(int64_t)k * LL] = z[k];
          } else {
            float best = z[0];
            int bk = 0;
#pragma unroll
            for (int q = 1; q < 4; ++q)
              if (z[q] > best) {
                best = z[q];
                bk = q;
              }
            prop[site] = (sig[site] && best > 0.f) ? (uint8_t)bk : (uint8_t)4;
          }
        }
      }
      if (!ok) break;
    }
  }
  __syncthreads();
  if (tid == 0 && *stop) atomicOr(err, 1u);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(64)
                 : "memory");
}

template <int NOUT, bool FROM_SIG>
constexpr size_t ws8_smem_bytes() {
  constexpr int R = WsShape<FROM_SIG>::R;
  return (size_t)R * 2 * kTcRow * 16 + 9 * 2 * NOUT * 16 + (2 * R + 5) * 8 + 16 + 8 * NOUT;
}

// Self-test of the bounded waits the tensor-core kernels use: thread 0 waits
// (ws_wait) on an mbarrier that nothing completes, gives up after its bound
// and raises the stop flag; warp 1 waits on another such barrier and must give
// up as soon as the flag is raised.  out[0] / out[1]: 1 if the first / second
// wait gave up; out[2]: the first wait in units of 2^20 SM cycles; out[3]: the
// second waiter's return after the first gave up, in units of 2^10 cycles.
__global__ void watchdog_selftest_kernel(unsigned int* out) {
  __shared__ uint64_t bars[2];
  __shared__ int stop_s;
  __shared__ long long t_stop;
  volatile int* stop = &stop_s;
  if (threadIdx.x == 0) {
    ws_bar_init(&bars[0], 1);
    ws_bar_init(&bars[1], 1);
    *stop = 0;
    t_stop = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const long long t0 = clock64();
    const bool ok = ws_wait(&bars[0], 0, stop);  // raises *stop when it gives up
    const long long t1 = clock64();
    t_stop = t1;
    out[0] = ok ? 0u : 1u;
    out[2] = (unsigned int)((t1 - t0) >> 20);
  } else if (threadIdx.x == 32) {
    out[1] = ws_wait(&bars[1], 0, stop) ? 0u : 1u;
    const long long t1 = clock64();
    // t_stop is written just after the flag; wait (bounded) until it is visible
    volatile long long* ts = &t_stop;
    for (int k = 0; k < (1 << 20) && *ts == 0; ++k) {
    }
    const long long d = t1 - *ts;
    out[3] = (unsigned int)((d > 0 ? d : 0) >> 10);
  }
  // the barriers leave the CTA with their phases incomplete; nothing else
  // refers to them
}

// ------------------------------------------------------ inference (FP8) ----
//
// FP8 (E4M3) form of layers 2-4: weights quantised per output channel,
// e4m3(W / s_co) with s_co = amax_co / 448; each layer's input quantised per
// layer, e4m3(x / s_in), with calibrated scales; products accumulate in fp32,
// and the epilogue dequantises with s_in * s_co.  This section holds the
// mma.sync m16n8k32 (e4m3 x e4m3) kernels used where L is not a multiple of
// 128, with layer 1 on the CUDA cores; conv_ws8_kernel above is the tcgen05
// form for the other sizes.

// One CTA per (layer, output channel): 32 + 32 + 8 CTAs (layer 4 padded to 8
// channels with zeros).  Wq layout per layer: [tap][co][ci] bytes.
__global__ void prepare_fp8_kernel(const float* __restrict__ P, uint8_t* __restrict__ Wq,
                                   float* __restrict__ wscale) {
  const int b = blockIdx.x;
  const int l = b < 32 ? 0 : (b < 64 ? 1 : 2);
  const int co = b - 32 * l;
  const int CO = l < 2 ? 32 : 8;
  const bool real = l < 2 || co < 4;
  const float* W = P + (l == 0 ? kW1 : (l == 1 ? kW2 : kW3)) + (size_t)co * 32 * 9;
  __shared__ float red[32];
  float amax = 0.f;
  for (int i = threadIdx.x; i < 32 * 9; i += blockDim.x) amax = fmaxf(amax, real ? fabsf(W[i]) : 0.f);
  for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xFFFFFFFFu, amax, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = amax;
  __syncthreads();
  if (threadIdx.x < 32) {
    amax = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xFFFFFFFFu, amax, o));
    if (threadIdx.x == 0) red[0] = amax;
  }
  __syncthreads();
  amax = red[0];
  const float s = amax > 0.f ? amax / 448.f : 1.f;
  uint8_t* out = Wq + (size_t)l * 9 * 32 * 32;
  for (int i = threadIdx.x; i < 32 * 9; i += blockDim.x) {
    const int ci = i / 9, tap = i % 9;
    const float q = real ? W[i] / s : 0.f;
    out[((size_t)tap * CO + co) * 32 + ci] =
        (uint8_t)__nv_cvt_float_to_fp8(q, __NV_SATFINITE, __NV_E4M3);
  }
  if (threadIdx.x == 0) wscale[l * 32 + co] = s;
}

// layer 1 (CUDA cores) writing e4m3(relu(.) / s_out), 32 bytes per site
__global__ void layer1_fp8_kernel(const uint8_t* __restrict__ sig, int L, int64_t shots,
                                  const float* __restrict__ W1, const float* __restrict__ P,
                                  float inv_s_out, uint8_t* __restrict__ out) {
  __shared__ float sW[9][32];
  __shared__ float sb[32];
  for (int i = threadIdx.x; i < 32 * 9; i += blockDim.x) sW[i % 9][i / 9] = W1[(i / 9) * 18 + i % 9];
  for (int co = threadIdx.x; co < 32; co += blockDim.x) {
    float b = P[kB0 + co];
    for (int tap = 0; tap < 9; ++tap) b += W1[co * 18 + 9 + tap];
    sb[co] = b;
  }
  __syncthreads();
  const int64_t LL = (int64_t)L * L;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < shots * LL;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = i / LL;
    const int r = (int)(i - s * LL), x = r % L, y = r / L;
    const uint8_t* g = sig + s * LL;
    float acc[32];
#pragma unroll
    for (int co = 0; co < 32; ++co) acc[co] = sb[co];
#pragma unroll 1
    for (int tap = 0; tap < 9; ++tap) {
      const int nb = wrapL(y + tap / 3 - 1, L) * L + wrapL(x + tap % 3 - 1, L);
      if (g[nb]) {
#pragma unroll
        for (int co = 0; co < 32; ++co) acc[co] += sW[tap][co];
      }
    }
    uint32_t w[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const uint32_t lo = pack_e4m3x2(fmaxf(acc[4 * c], 0.f) * inv_s_out,
                                      fmaxf(acc[4 * c + 1], 0.f) * inv_s_out);
      const uint32_t hi = pack_e4m3x2(fmaxf(acc[4 * c + 2], 0.f) * inv_s_out,
                                      fmaxf(acc[4 * c + 3], 0.f) * inv_s_out);
      w[c] = lo | (hi << 16);
    }
    uint4* o = reinterpret_cast<uint4*>(out + i * 32);
    o[0] = make_uint4(w[0], w[1], w[2], w[3]);
    o[1] = make_uint4(w[4], w[5], w[6], w[7]);
  }
}

__device__ __forceinline__ void mma_e4m3(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k32.row.col.f32.e4m3.e4m3.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

constexpr int kW8Pitch = 12;  // words per [tap][co] row of 32 e4m3 weights (conflict-free)

// FP8 implicit-GEMM conv: as conv_mma_kernel with 32 input channels of e4m3
// (32 bytes per site) and one k32 step per tap.  acc * (s_in * s_co) + bias;
// kActs writes e4m3(relu(.) * inv_s_out).
template <int NT, int MODE>
__global__ void __launch_bounds__(128) conv_fp8_kernel(
    const uint8_t* __restrict__ in, const uint8_t* __restrict__ Wq,
    const float* __restrict__ wscale, const float* __restrict__ bias, float s_in,
    float inv_s_out, int L, int64_t shots, uint8_t* __restrict__ out,
    float* __restrict__ logits, const uint8_t* __restrict__ sig, uint8_t* __restrict__ prop) {
  constexpr int CO = 8 * NT;
  __shared__ uint32_t sW[9 * CO * kW8Pitch];
  __shared__ float sb[CO], sc[CO];
  for (int i = threadIdx.x; i < 9 * CO * 8; i += blockDim.x)
    sW[(i / 8) * kW8Pitch + (i % 8)] = reinterpret_cast<const uint32_t*>(Wq)[i];
  for (int i = threadIdx.x; i < CO; i += blockDim.x) {
    const bool real = MODE == kActs || i < 4;
    sb[i] = real ? bias[i] : 0.f;
    sc[i] = real ? s_in * wscale[i] : 0.f;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int64_t LL = (int64_t)L * L, S = shots * LL;
  const int64_t tiles = (S + 15) / 16;
  const uint32_t* inw = reinterpret_cast<const uint32_t*>(in);  // 8 words per site
  for (int64_t tile = blockIdx.x * 4 + warp; tile < tiles; tile += (int64_t)gridDim.x * 4) {
    const int64_t s0 = tile * 16;
    int64_t site[2], shot[2];
    int xs[2], ys[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      site[h] = s0 + g + 8 * h;
      const int64_t scl = site[h] < S ? site[h] : S - 1;
      shot[h] = scl / LL;
      const int r = (int)(scl - shot[h] * LL);
      xs[h] = r % L;
      ys[h] = r / L;
    }
    float acc[NT][4];
#pragma unroll
    for (int n = 0; n < NT; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int dy = tap / 3 - 1, dx = tap % 3 - 1;
      int64_t nbw[2];
#pragma unroll
      for (int h = 0; h < 2; ++h)
        nbw[h] = (shot[h] * LL + wrapL(ys[h] + dy, L) * L + wrapL(xs[h] + dx, L)) * 8;
      uint32_t a[4];
      a[0] = __ldg(inw + nbw[0] + t);      // row g,     k = 4t .. 4t+3
      a[1] = __ldg(inw + nbw[1] + t);      // row g + 8
      a[2] = __ldg(inw + nbw[0] + 4 + t);  // row g,     k = 16+4t ..
      a[3] = __ldg(inw + nbw[1] + 4 + t);  // row g + 8
#pragma unroll
      for (int n = 0; n < NT; ++n) {
        const uint32_t* wr = sW + (tap * CO + n * 8 + g) * kW8Pitch + t;
        mma_e4m3(acc[n], a, wr[0], wr[4]);
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const bool valid = site[h] < S;
      const int r = ys[h] * L + xs[h];
      if (MODE == kProposals) {
        const float v0 = acc[0][2 * h] * sc[2 * t] + sb[2 * t];
        const float v1 = acc[0][2 * h + 1] * sc[2 * t + 1] + sb[2 * t + 1];
        const float w0 = __shfl_down_sync(0xFFFFFFFFu, v0, 1);
        const float w1 = __shfl_down_sync(0xFFFFFFFFu, v1, 1);
        if (t == 0 && valid) {
          const float z[4] = {v0, v1, w0, w1};
          float best = z[0];
          int bk = 0;
#pragma unroll
          for (int q = 1; q < 4; ++q)
            if (z[q] > best) {
              best = z[q];
              bk = q;
            }
          prop[site[h]] = (sig[site[h]] && best > 0.f) ? (uint8_t)bk : (uint8_t)4;
        }
        continue;
      }
      if (!valid) continue;
#pragma unroll
      for (int n = 0; n < NT; ++n) {
        const int c0 = n * 8 + 2 * t;
        const float v0 = acc[n][2 * h] * sc[c0] + sb[c0];
        const float v1 = acc[n][2 * h + 1] * sc[c0 + 1] + sb[c0 + 1];
        if (MODE == kLogits) {
          float* lb = logits + shot[h] * 4 * LL + r;
          if (c0 < 4) lb[(int64_t)c0 * LL] = v0;
          if (c0 + 1 < 4) lb[(int64_t)(c0 + 1) * LL] = v1;
        } else {
          reinterpret_cast<uint16_t*>(out)[site[h] * 16 + c0 / 2] =
              pack_e4m3x2(fmaxf(v0, 0.f) * inv_s_out, fmaxf(v1, 0.f) * inv_s_out);
        }
      }
    }
  }
}

// max over a bf16 activation buffer (values >= 0 after ReLU): float bits
// compare as integers
__global__ void amax_bf16_kernel(const __nv_bfloat16* __restrict__ a, int64_t n,
                                 unsigned int* __restrict__ out) {
  float m = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, __bfloat162float(a[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// Links whose two end anyons propose each other: e_x(r) iff prop(r) = +x and
// prop(r + x^) = -x; e_y likewise.  residual = N xor C0; C0 written if given.
__global__ void pairing_kernel(const uint8_t* __restrict__ N, const uint8_t* __restrict__ prop,
                               int L, int64_t shots, uint8_t* __restrict__ resid,
                               uint8_t* __restrict__ c0) {
  const int64_t LL = (int64_t)L * L;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < shots * LL;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = i / LL;
    const int r = (int)(i - s * LL), x = r % L, y = r / L;
    const uint8_t* ps = prop + s * LL;
    const uint8_t fx = (ps[r] == 0 && ps[y * L + wrapL(x + 1, L)] == 1) ? 1 : 0;
    const uint8_t fy = (ps[r] == 2 && ps[wrapL(y + 1, L) * L + x] == 3) ? 1 : 0;
    const int64_t e = s * 2 * LL + r;
    if (c0) {
      c0[e] = fx;
      c0[e + LL] = fy;
    }
    resid[e] = N[e] ^ fx;
    resid[e + LL] = N[e + LL] ^ fy;
  }
}

// C ^= N ^ R (C0 = N xor R recovered from the noise and the residual)
__global__ void combine_kernel(uint8_t* __restrict__ C, const uint8_t* __restrict__ N,
                               const uint8_t* __restrict__ R, int64_t n) {
  const int64_t n16 = n / 16;
  const uint4* N4 = reinterpret_cast<const uint4*>(N);
  const uint4* R4 = reinterpret_cast<const uint4*>(R);
  uint4* C4 = reinterpret_cast<uint4*>(C);
  const bool vec = ((reinterpret_cast<uintptr_t>(C) | reinterpret_cast<uintptr_t>(N) |
                     reinterpret_cast<uintptr_t>(R)) & 15) == 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (vec) {
    for (int64_t i = i0; i < n16; i += stride) {
      uint4 c = C4[i];
      const uint4 a = N4[i], b = R4[i];
      c.x ^= a.x ^ b.x;
      c.y ^= a.y ^ b.y;
      c.z ^= a.z ^ b.z;
      c.w ^= a.w ^ b.w;
      C4[i] = c;
    }
    i0 += n16 * 16;
  }
  for (int64_t i = i0; i < n; i += stride) C[i] ^= N[i] ^ R[i];
}

// ------------------------------------------------ training (tensor cores) --
//
// One training step in bf16 with fp32 accumulation and fp32 master weights:
// forward through layer1_kernel and conv_mma_kernel (the inference kernels),
// the loss gradient as bf16 NHWC, then per layer the weight gradient
// (wgrad_mma_kernel: dW[co][ci][tap] = sum_s dout[s][co] in[s + tap][ci] as a
// GEMM with M = output channels, N = (tap, input channel), K = sites, on
// mma.sync m16n8k16), the bias gradient, and the input gradient
// (conv_mma_kernel in kGradMasked mode: the same 3x3 convolution with the
// weights transposed in channels and mirrored in taps, times the ReLU mask).

// Backward-data weights: Wt[l][tap][ci][co] = W_l[co][ci][8 - tap] for the
// layers 2, 3, 4 (layer 4's co >= 4 zero), bf16.
__global__ void prepare_bwd_weights_kernel(const float* __restrict__ P,
                                           __nv_bfloat16* __restrict__ Wt) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 3 * 9 * 32 * 32;
       i += gridDim.x * blockDim.x) {
    const int l = i / (9 * 32 * 32), j = i % (9 * 32 * 32);
    const int tap = j / (32 * 32), ci = (j / 32) % 32, co = j % 32;
    const int CO = l < 2 ? 32 : 4;
    const int off = l == 0 ? kW1 : (l == 1 ? kW2 : kW3);
    const float w = co < CO ? P[off + (co * 32 + ci) * 9 + (8 - tap)] : 0.f;
    Wt[i] = __float2bfloat16_rn(w);
  }
}

// network input as bf16 NHWC with 32 channels: (anyon, 1, 0, ..., 0)
__global__ void x0_nhwc_kernel(const uint8_t* __restrict__ sig, int64_t S,
                               __nv_bfloat16* __restrict__ x0) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < S;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint4* o = reinterpret_cast<uint4*>(x0 + i * 32);
    o[0] = make_uint4(pack_bf16(sig[i] ? 1.f : 0.f, 1.f), 0, 0, 0);
    o[1] = o[2] = o[3] = make_uint4(0, 0, 0, 0);
  }
}

// Softmax over (z0..z3, 0) at labelled sites, the fifth class ("no move")
// with its logit fixed at 0; target q = smoothed one-hot of the label;
// dz = (p - q) / n_labelled as bf16 NHWC with 32 channels (4 used), loss =
// mean cross-entropy -sum q log p.
__global__ void loss_grad_nhwc_kernel(const float* __restrict__ z, const uint8_t* __restrict__ lab,
                                      int L, int B, const unsigned int* __restrict__ count,
                                      __nv_bfloat16* __restrict__ dz, float* __restrict__ loss) {
  const int LL = L * L;
  const float inv_n = 1.f / (float)(*count > 0 ? *count : 1u);
  const float q_off = kLabelSmoothing / 5.f, q_on = 1.f - kLabelSmoothing + q_off;
  float local = 0.f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B * LL; i += gridDim.x * blockDim.x) {
    const int b = i / LL, r = i - b * LL;
    const float* zb = z + (size_t)b * 4 * LL;
    uint4* o = reinterpret_cast<uint4*>(dz + (size_t)i * 32);
    const int t = lab[i];
    float g[4] = {0.f, 0.f, 0.f, 0.f};
    if (t != 255) {
      float v[5] = {zb[r], zb[LL + r], zb[2 * LL + r], zb[3 * LL + r], 0.f};
      float mx = v[0];
      for (int k = 1; k < 5; ++k) mx = fmaxf(mx, v[k]);
      float sum = 0.f;
      for (int k = 0; k < 5; ++k) sum += expf(v[k] - mx);
      const float lse = mx + logf(sum);
      for (int k = 0; k < 5; ++k) {
        const float q = (t == k) ? q_on : q_off;
        if (k < 4) g[k] = (expf(v[k] - lse) - q) * inv_n;
        local += q * (lse - v[k]);
      }
    }
    o[0] = make_uint4(pack_bf16(g[0], g[1]), pack_bf16(g[2], g[3]), 0, 0);
    o[1] = o[2] = o[3] = make_uint4(0, 0, 0, 0);
  }
  for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xFFFFFFFFu, local, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, local * inv_n);
}

// per-channel sum of a bf16 NHWC [S][32] gradient into db[0 .. CO)
template <int CO>
__global__ void bias_grad_kernel(const __nv_bfloat16* __restrict__ d, int64_t S,
                                 float* __restrict__ part) {
  __shared__ float red[8][32];
  const int c = threadIdx.x & 31, row = threadIdx.x >> 5;
  float acc = 0.f;
  for (int64_t s = blockIdx.x * 8 + row; s < S; s += (int64_t)gridDim.x * 8)
    acc += __bfloat162float(d[s * 32 + c]);
  red[row][c] = acc;
  __syncthreads();
  if (row == 0) {
    float v = 0.f;
    for (int r = 0; r < 8; ++r) v += red[r][c];
    part[(size_t)blockIdx.x * 32 + c] = v;  // this CTA's partial sums, [CTA][32]
  }
}

// out[i] = sum over p = 0 .. nparts - 1, in that order, of part[p * stride + i]:
// the per-CTA partial sums of a gradient added in a fixed order, so that a
// training run repeats bit for bit.
__global__ void reduce_parts_kernel(const float* __restrict__ part, int nparts, int stride, int n,
                                    float* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float v = 0.f;
    for (int q = 0; q < nparts; ++q) v += part[(size_t)q * stride + i];
    out[i] = v;
  }
}

constexpr int kWgChunk = 64;   // sites staged per round
constexpr int kWgPitch = 36;   // words per staged row (64 sites = 32 words, padded)

// dW[co][ci][tap] += sum over the CTA's sites s of dout[s][co] in[nb(s, tap)][ci]
// (nb: the circular neighbour of s at tap offset (ky - 1, kx - 1)); dout and in
// bf16 NHWC [S][32]; only co < CO_REAL, ci < CI_REAL are written (param layout
// [co][CI_REAL][9]).  256 threads: warp w owns output channels 16 (w / 4) ..
// +15 and the n-tiles 9 (w % 4) .. +8 of the 36 (tap, 8-channel block) tiles.
template <int CO_REAL, int CI_REAL>
__global__ void __launch_bounds__(256) wgrad_mma_kernel(const __nv_bfloat16* __restrict__ dout,
                                                        const __nv_bfloat16* __restrict__ in,
                                                        int L, int64_t S, int64_t chunk,
                                                        float* __restrict__ part) {
  __shared__ uint32_t sD[32 * kWgPitch];       // [co][site pair]
  __shared__ uint32_t sI[9 * 32 * kWgPitch];   // [tap][ci][site pair]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int mt = warp >> 2, nt0 = (warp & 3) * 9;
  const int64_t LL = (int64_t)L * L;
  const int64_t s_begin = blockIdx.x * chunk, s_end = min(S, s_begin + chunk);
  float acc[9][4];
#pragma unroll
  for (int k = 0; k < 9; ++k) acc[k][0] = acc[k][1] = acc[k][2] = acc[k][3] = 0.f;
  __nv_bfloat16* sDh = reinterpret_cast<__nv_bfloat16*>(sD);
  __nv_bfloat16* sIh = reinterpret_cast<__nv_bfloat16*>(sI);
  for (int64_t base = s_begin; base < s_end; base += kWgChunk) {
    __syncthreads();
    // stage: thread (site j, octet o) transposes 8 channels of dout and of the
    // nine neighbours of site base + j
    {
      const int j = tid >> 2, o = tid & 3;
      const int64_t s = base + j;
      const bool ok = s < s_end;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (ok) v = *reinterpret_cast<const uint4*>(dout + s * 32 + o * 8);
      const __nv_bfloat16* vh = reinterpret_cast<const __nv_bfloat16*>(&v);
#pragma unroll
      for (int k = 0; k < 8; ++k) sDh[(o * 8 + k) * (2 * kWgPitch) + j] = vh[k];
      int64_t shot = 0;
      int x = 0, y = 0;
      if (ok) {
        shot = s / LL;
        const int r = (int)(s - shot * LL);
        x = r % L;
        y = r / L;
      }
#pragma unroll
      for (int tap = 0; tap < 9; ++tap) {
        uint4 u = make_uint4(0, 0, 0, 0);
        if (ok) {
          const int xx = wrapL(x + tap % 3 - 1, L), yy = wrapL(y + tap / 3 - 1, L);
          u = *reinterpret_cast<const uint4*>(in + (shot * LL + (int64_t)yy * L + xx) * 32 + o * 8);
        }
        const __nv_bfloat16* uh = reinterpret_cast<const __nv_bfloat16*>(&u);
#pragma unroll
        for (int k = 0; k < 8; ++k) sIh[((tap * 32) + o * 8 + k) * (2 * kWgPitch) + j] = uh[k];
      }
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < kWgChunk / 16; ++ks) {
      uint32_t a[4];
      const uint32_t* ar = sD + (mt * 16 + g) * kWgPitch + ks * 8 + t;
      a[0] = ar[0];
      a[1] = ar[8 * kWgPitch];
      a[2] = ar[4];
      a[3] = ar[8 * kWgPitch + 4];
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const int ntile = nt0 + k, tap = ntile >> 2, ci = (ntile & 3) * 8 + g;
        const uint32_t* br = sI + (tap * 32 + ci) * kWgPitch + ks * 8 + t;
        mma_bf16(acc[k], a, br[0], br[4]);
      }
    }
  }
  // rows g, g + 8 (output channels), columns 2t, 2t + 1 (input channels) of each tile
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int ntile = nt0 + k, tap = ntile >> 2, cb = (ntile & 3) * 8 + 2 * t;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int co = mt * 16 + g + 8 * h;
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int ci = cb + e;
        if (co < CO_REAL && ci < CI_REAL)  // this CTA's partial sums, [CTA][param]
          part[(size_t)blockIdx.x * (CO_REAL * CI_REAL * 9) + (co * CI_REAL + ci) * 9 + tap] =
              acc[k][2 * h + e];
      }
    }
  }
}

// Read-out of one layer's activations as the next layer consumes them, as
// fp32 [shot][32][L][L] (a checking aid, not part of inference).  form: 0 bf16
// [site][32], 1 bf16 planar [shot][y][octet][x][8], 2 e4m3 [site][32], 3 e4m3
// planar [shot][y][16-channel group][x][16], 4 / 5 the bf16 / e4m3 layer-1
// table [512][32] indexed by the 3 x 3 anyon pattern of sig (bit ky * 3 + kx).
// e4m3 codes are written as their e4m3 values (exact in fp32), not rescaled.
__global__ void capture_kernel(const void* __restrict__ src, int form,
                               const uint8_t* __restrict__ sig, int L, int64_t shots,
                               float* __restrict__ out) {
  const int64_t LL = (int64_t)L * L;
  const int64_t n = shots * 32 * LL;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t shot = i / (32 * LL);
    const int64_t r = i - shot * 32 * LL;
    const int c = (int)(r / LL);
    const int site = (int)(r - (int64_t)c * LL);
    const int y = site / L, x = site - (site / L) * L;
    const int64_t gs = shot * LL + site;
    const __nv_bfloat16* b = reinterpret_cast<const __nv_bfloat16*>(src);
    const uint8_t* q = reinterpret_cast<const uint8_t*>(src);
    float v = 0.f;
    int code = -1;
    if (form == 0) {
      v = __bfloat162float(b[gs * 32 + c]);
    } else if (form == 1) {
      v = __bfloat162float(b[(((shot * L + y) * 4 + c / 8) * (int64_t)L + x) * 8 + c % 8]);
    } else if (form == 2) {
      code = q[gs * 32 + c];
    } else if (form == 3) {
      code = q[(((shot * L + y) * 2 + c / 16) * (int64_t)L + x) * 16 + c % 16];
    } else {
      int pat = 0;
      for (int tap = 0; tap < 9; ++tap) {
        const int yy = wrapL(y + tap / 3 - 1, L), xx = wrapL(x + tap % 3 - 1, L);
        if (sig[shot * LL + (int64_t)yy * L + xx]) pat |= 1 << tap;
      }
      if (form == 4)
        v = __bfloat162float(b[pat * 32 + c]);
      else
        code = q[pat * 32 + c];
    }
    if (code >= 0) {
      const __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)code, __NV_E4M3);
      v = __half2float(__half(h));
    }
    out[i] = v;
  }
}

int grid_for(int64_t items, int threads) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t b = (items + threads - 1) / threads;
  const int64_t cap = (int64_t)(sms > 0 ? sms : 1) * 32;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

}  // namespace qca

using namespace qca;

struct qca_net_s {
  int device = 0;
  float* params = nullptr;         // fp32 [kParams]
  float* grads = nullptr;          // fp32 [kParams]
  float* m1 = nullptr;             // Adam first moments [kParams]
  float* m2 = nullptr;             // Adam second moments [kParams]
  int64_t adam_t = 0;              // optimiser steps taken
  int64_t train_shots = 0;         // training syndromes drawn so far
  __nv_bfloat16* wb = nullptr;     // bf16 weights of layers 2-4, [tap][co][ci]
  float* w1 = nullptr;             // layer 1 fp32 (bf16-rounded) [co][ci][tap]
  bool prepared = false;
  // FP8 form: per-channel e4m3 weights of layers 2-4 ([tap][co][ci] bytes), their
  // scales, the per-layer input scales (host), and the active precision
  uint8_t* wq = nullptr;
  float* wscale = nullptr;
  float act_scale[3] = {0.f, 0.f, 0.f};
  int precision = 0;  // 0 bf16, 1 fp8
  bool prepared8 = false;
  int use_tc = 2;                // bf16 layers 2-4: 0 mma.sync, 1 tcgen05 row-synchronous,
                                 // 2 tcgen05 warp-specialised (tcgen05 where L % 128 == 0)
  unsigned int* err = nullptr;   // device word: a tensor-core wait timed out
  __nv_bfloat16* lut = nullptr;  // layer-1 outputs per 3 x 3 anyon pattern [512][32]
  uint8_t* lut8 = nullptr;        // the same in e4m3 at the layer-1 activation scale
  // inference workspace
  uint8_t* ws = nullptr;
  size_t ws_bytes = 0;
};

extern "C" {

int64_t qca_net_param_count(void) { return kParams; }

int qca_net_create(uint64_t seed, qca_net_t* out) {
  if (!out) {
    set_error("qca_net_create: NULL output");
    return QCA_ERR_ARG;
  }
  *out = nullptr;
  // He-normal-like init from the counter generator (Box-Muller), biases 0
  std::vector<float> h(kParams, 0.f);
  uint64_t k = splitmix64(seed ^ 0x494E4954ULL);  // "INIT"
  for (int l = 0; l < kLayers; ++l) {
    const float sd = sqrtf(2.f / (kCi[l] * 9.f));
    for (int i = 0; i < kCo[l] * kCi[l] * 9; ++i) {
      const double u1 = ((splitmix64(k ^ (2 * (uint64_t)i)) >> 11) + 1) * (1.0 / 9007199254740993.0);
      const double u2 = (splitmix64(k ^ (2 * (uint64_t)i + 1)) >> 11) * (1.0 / 9007199254740992.0);
      h[kWoff[l] + i] = (float)(sd * sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2));
    }
    k = splitmix64(k);
  }
  qca_net_s* n = new qca_net_s();
  cudaGetDevice(&n->device);
  cudaError_t e = cudaMalloc(&n->params, sizeof(float) * kParams);
  if (e == cudaSuccess) e = cudaMalloc(&n->grads, sizeof(float) * kParams);
  if (e == cudaSuccess) e = cudaMalloc(&n->m1, sizeof(float) * kParams);
  if (e == cudaSuccess) e = cudaMalloc(&n->m2, sizeof(float) * kParams);
  if (e == cudaSuccess) e = cudaMalloc(&n->wb, sizeof(__nv_bfloat16) * (2 * 9 * 32 * 32 + 9 * 8 * 32));
  if (e == cudaSuccess) e = cudaMalloc(&n->w1, sizeof(float) * 32 * 2 * 9);
  if (e == cudaSuccess) e = cudaMalloc(&n->wq, 2 * 9 * 32 * 32 + 9 * 8 * 32);
  if (e == cudaSuccess) e = cudaMalloc(&n->wscale, sizeof(float) * 96);
  if (e == cudaSuccess) e = cudaMalloc(&n->err, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMalloc(&n->lut, sizeof(__nv_bfloat16) * 512 * 32);
  if (e == cudaSuccess) e = cudaMalloc(&n->lut8, 512 * 32);
  if (e == cudaSuccess) e = cudaMemset(n->err, 0, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemcpy(n->params, h.data(), sizeof(float) * kParams, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(n->m1, 0, sizeof(float) * kParams);
  if (e == cudaSuccess) e = cudaMemset(n->m2, 0, sizeof(float) * kParams);
  if (e != cudaSuccess) {
    qca_net_destroy(n);
    return cuda_fail(e, "qca_net_create");
  }
  *out = n;
  return QCA_OK;
}

int qca_net_destroy(qca_net_t n) {
  if (!n) return QCA_OK;
  cudaFree(n->params);
  cudaFree(n->grads);
  cudaFree(n->m1);
  cudaFree(n->m2);
  cudaFree(n->wb);
  cudaFree(n->w1);
  cudaFree(n->wq);
  cudaFree(n->wscale);
  cudaFree(n->err);
  cudaFree(n->lut);
  cudaFree(n->lut8);
  cudaFree(n->ws);
  delete n;
  return QCA_OK;
}

int qca_net_get_params(qca_net_t n, float* host, int64_t count) {
  if (!n || !host || count != kParams) {
    set_error("qca_net_get_params: bad arguments (count must be %d)", kParams);
    return QCA_ERR_ARG;
  }
  return cuda_fail(cudaMemcpy(host, n->params, sizeof(float) * kParams, cudaMemcpyDeviceToHost),
                   "qca_net_get_params");
}

int qca_net_set_params(qca_net_t n, const float* host, int64_t count) {
  if (!n || !host || count != kParams) {
    set_error("qca_net_set_params: bad arguments (count must be %d)", kParams);
    return QCA_ERR_ARG;
  }
  n->prepared = false;
  n->prepared8 = false;
  return cuda_fail(cudaMemcpy(n->params, host, sizeof(float) * kParams, cudaMemcpyHostToDevice),
                   "qca_net_set_params");
}

}  // extern "C"

namespace {

// Device buffers of one training batch of S sites.
// Gradient reductions split the sites into at most kGradParts CTAs, a number
// fixed by the batch size alone (not by the device), and add the CTAs' partial
// sums in order.
constexpr int kGradParts = 256;

struct TrainBufs {
  int64_t S = 0;
  uint8_t* bytes = nullptr;        // sig, dir, lab
  __nv_bfloat16* h = nullptr;      // x0, a1, a2, a3, dz, g1, g2: bf16 NHWC [S][32] each
  float* z = nullptr;              // logits fp32 [B][4][L][L]
  __nv_bfloat16* wt = nullptr;     // backward-data weights [3][9][32][32]
  float* part = nullptr;           // per-CTA gradient partial sums [kGradParts][9216]
  uint8_t* sig() const { return bytes; }
  uint8_t* dir() const { return bytes + S; }
  uint8_t* lab() const { return bytes + 2 * S; }
  __nv_bfloat16* act(int k) const { return h + (size_t)k * S * 32; }
  int alloc(int64_t sites) {
    S = sites;
    cudaError_t e = cudaMalloc(&bytes, 3 * S);
    if (e == cudaSuccess) e = cudaMalloc(&h, sizeof(__nv_bfloat16) * 7 * 32 * S);
    if (e == cudaSuccess) e = cudaMalloc(&z, sizeof(float) * 4 * S);
    if (e == cudaSuccess) e = cudaMalloc(&wt, sizeof(__nv_bfloat16) * 3 * 9 * 32 * 32);
    if (e == cudaSuccess) e = cudaMalloc(&part, sizeof(float) * kGradParts * 9 * 32 * 32);
    return cuda_fail(e, "training buffers");
  }
  ~TrainBufs() {
    cudaFree(bytes);
    cudaFree(h);
    cudaFree(z);
    cudaFree(wt);
    cudaFree(part);
  }
};

// Forward and backward of one batch whose syndromes (bufs.sig) and labels
// (bufs.lab) are in place: n->grads receives the gradient of the mean
// smoothed cross-entropy over the labelled sites, *loss that loss.
int train_forward_backward(qca_net_s* n, const TrainBufs& b, int L, int batch,
                           const unsigned int* count, float* loss) {
  const int64_t S = b.S;
  const int gS = grid_for(S, 256);
  const int gm = grid_for((S + 15) / 16 * 32, 128);
  // weight gradients: CTAs of `chunk` sites (a multiple of the staging chunk);
  // bias gradients: gB CTAs; both counts depend on S only
  int64_t chunk = (S + kGradParts - 1) / kGradParts;
  chunk = ((chunk + kWgChunk - 1) / kWgChunk) * kWgChunk;
  const int gW = (int)((S + chunk - 1) / chunk);
  const int gB = (int)std::min<int64_t>(kGradParts, (S + 255) / 256);
  auto reduce = [&](int nparts, int stride, int n, float* out) {
    reduce_parts_kernel<<<(n + 255) / 256, 256>>>(b.part, nparts, stride, n, out);
  };
  __nv_bfloat16 *x0 = b.act(0), *a1 = b.act(1), *a2 = b.act(2), *a3 = b.act(3), *dz = b.act(4),
                *g1 = b.act(5), *g2 = b.act(6);
  // weights of this step: bf16 forward copies, mirrored backward copies
  prepare_weights_kernel<<<64, 256>>>(n->params, n->wb, n->w1);
  prepare_bwd_weights_kernel<<<64, 256>>>(n->params, b.wt);
  n->prepared = false;  // the inference table follows the weights on the next inference call
  // forward
  x0_nhwc_kernel<<<gS, 256>>>(b.sig(), S, x0);
  layer1_kernel<<<gS, 256>>>(b.sig(), L, batch, n->w1, n->params, a1);
  conv_mma_kernel<4, kActs><<<gm, 128>>>(a1, n->wb, n->params + kB1, L, batch, a2, nullptr, nullptr,
                                         nullptr, nullptr);
  conv_mma_kernel<4, kActs><<<gm, 128>>>(a2, n->wb + 9 * 32 * 32, n->params + kB2, L, batch, a3,
                                         nullptr, nullptr, nullptr, nullptr);
  conv_mma_kernel<1, kLogits><<<gm, 128>>>(a3, n->wb + 2 * 9 * 32 * 32, n->params + kB3, L, batch,
                                           nullptr, b.z, nullptr, nullptr, nullptr);
  loss_grad_nhwc_kernel<<<gS, 256>>>(b.z, b.lab(), L, batch, count, dz, loss);
  // backward: layer 4, 3, 2 (weights, bias, masked input gradient), layer 1
  float* G = n->grads;
  wgrad_mma_kernel<4, 32><<<gW, 256>>>(dz, a3, L, S, chunk, b.part);
  reduce(gW, 4 * 32 * 9, 4 * 32 * 9, G + kW3);
  bias_grad_kernel<4><<<gB, 256>>>(dz, S, b.part);
  reduce(gB, 32, 4, G + kB3);
  conv_mma_kernel<4, kGradMasked><<<gm, 128>>>(dz, b.wt + 2 * 9 * 32 * 32, nullptr, L, batch, g1,
                                               nullptr, nullptr, nullptr, a3);
  wgrad_mma_kernel<32, 32><<<gW, 256>>>(g1, a2, L, S, chunk, b.part);
  reduce(gW, 32 * 32 * 9, 32 * 32 * 9, G + kW2);
  bias_grad_kernel<32><<<gB, 256>>>(g1, S, b.part);
  reduce(gB, 32, 32, G + kB2);
  conv_mma_kernel<4, kGradMasked><<<gm, 128>>>(g1, b.wt + 9 * 32 * 32, nullptr, L, batch, g2,
                                               nullptr, nullptr, nullptr, a2);
  wgrad_mma_kernel<32, 32><<<gW, 256>>>(g2, a1, L, S, chunk, b.part);
  reduce(gW, 32 * 32 * 9, 32 * 32 * 9, G + kW1);
  bias_grad_kernel<32><<<gB, 256>>>(g2, S, b.part);
  reduce(gB, 32, 32, G + kB1);
  conv_mma_kernel<4, kGradMasked><<<gm, 128>>>(g2, b.wt, nullptr, L, batch, g1, nullptr, nullptr,
                                               nullptr, a1);
  wgrad_mma_kernel<32, 2><<<gW, 256>>>(g1, x0, L, S, chunk, b.part);
  reduce(gW, 32 * 2 * 9, 32 * 2 * 9, G + kW0);
  bias_grad_kernel<32><<<gB, 256>>>(g1, S, b.part);
  reduce(gB, 32, 32, G + kB0);
  return cuda_fail(cudaGetLastError(), "training kernels");
}

uint64_t train_thr(double p) {
  const double v = ldexp(p, 64);
  return v >= 18446744073709549568.0 ? ~0ull : (uint64_t)v;
}

}  // namespace

extern "C" {

int qca_net_train(qca_net_t n, int L, int64_t iterations, int batch, double p_lo, double p_hi,
                  uint64_t seed, float lr, float* out_losses) {
  if (!n || L < 4 || L > 128 || iterations < 0 || iterations > (1 << 24) || batch < 1 ||
      (int64_t)batch * L * L > (1 << 24) || !(p_lo >= 0 && p_hi <= 1 && p_lo <= p_hi) ||
      !(lr > 0.f)) {
    set_error("qca_net_train: bad arguments");
    return QCA_ERR_ARG;
  }
  if (iterations == 0) return QCA_OK;
  const int64_t S = (int64_t)batch * L * L;
  TrainBufs b;
  int rc = b.alloc(S);
  if (rc) return rc;
  float* losses = nullptr;
  unsigned int* counts = nullptr;
  cudaError_t e = cudaMalloc(&losses, sizeof(float) * iterations);
  if (e == cudaSuccess) e = cudaMalloc(&counts, sizeof(unsigned int) * iterations);
  if (e == cudaSuccess) e = cudaMemset(losses, 0, sizeof(float) * iterations);
  if (e == cudaSuccess) e = cudaMemset(counts, 0, sizeof(unsigned int) * iterations);
  if (e != cudaSuccess) {
    cudaFree(losses);
    cudaFree(counts);
    return cuda_fail(e, "qca_net_train allocation");
  }
  const uint64_t t_lo = train_thr(p_lo), t_span = train_thr(p_hi - p_lo);
  const int gS = grid_for(S, 256);
  const float b1 = 0.9f, b2 = 0.999f;
  for (int64_t it = 0; it < iterations && rc == QCA_OK; ++it) {
    train_sample_kernel<<<gS, 256>>>(L, batch, n->train_shots, seed, t_lo, t_span, b.sig());
    first_dir_kernel<<<gS, 256>>>(b.sig(), L, batch, b.dir());
    mutual_label_kernel<<<gS, 256>>>(b.dir(), L, batch, b.lab());
    count_labelled_kernel<<<gS, 256>>>(b.lab(), (int)S, counts + it);
    rc = train_forward_backward(n, b, L, batch, counts + it, losses + it);
    if (rc) break;
    n->adam_t += 1;
    const float c1 = 1.f / (1.f - powf(b1, (float)n->adam_t));
    const float c2 = 1.f / (1.f - powf(b2, (float)n->adam_t));
    adam_kernel<<<grid_for(kParams, 256), 256>>>(n->params, n->grads, n->m1, n->m2, kParams, lr, b1,
                                                b2, c1, c2);
    n->train_shots += batch;
    e = cudaGetLastError();
    if (e != cudaSuccess) rc = cuda_fail(e, "training kernels");
  }
  if (rc == QCA_OK) rc = cuda_fail(cudaDeviceSynchronize(), "qca_net_train");
  if (rc == QCA_OK && out_losses)
    rc = cuda_fail(cudaMemcpy(out_losses, losses, sizeof(float) * iterations, cudaMemcpyDeviceToHost),
                   "training loss copy");
  cudaFree(losses);
  cudaFree(counts);
  n->prepared = false;
  n->prepared8 = false;
  return rc;
}

int qca_net_gradients(qca_net_t n, const uint8_t* noise, int L, int batch, float* host_grads,
                      int64_t count, float* host_loss) {
  if (!n || !noise || !host_grads || count != kParams || L < 4 || L > 128 || batch < 1 ||
      (int64_t)batch * L * L > (1 << 24)) {
    set_error("qca_net_gradients: bad arguments (count must be %d, 4 <= L <= 128)", kParams);
    return QCA_ERR_ARG;
  }
  const int64_t S = (int64_t)batch * L * L;
  TrainBufs b;
  int rc = b.alloc(S);
  if (rc) return rc;
  float* dl = nullptr;
  unsigned int* cnt = nullptr;
  cudaError_t e = cudaMalloc(&dl, sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&cnt, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemset(dl, 0, sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(cnt, 0, sizeof(unsigned int));
  if (e != cudaSuccess) {
    cudaFree(dl);
    cudaFree(cnt);
    return cuda_fail(e, "qca_net_gradients allocation");
  }
  const int gS = grid_for(S, 256);
  syndrome_kernel<<<gS, 256>>>(noise, L, batch, b.sig());
  first_dir_kernel<<<gS, 256>>>(b.sig(), L, batch, b.dir());
  mutual_label_kernel<<<gS, 256>>>(b.dir(), L, batch, b.lab());
  count_labelled_kernel<<<gS, 256>>>(b.lab(), (int)S, cnt);
  rc = train_forward_backward(n, b, L, batch, cnt, dl);
  if (rc == QCA_OK) rc = cuda_fail(cudaDeviceSynchronize(), "qca_net_gradients");
  if (rc == QCA_OK)
    rc = cuda_fail(cudaMemcpy(host_grads, n->grads, sizeof(float) * kParams, cudaMemcpyDeviceToHost),
                   "gradient copy");
  if (rc == QCA_OK && host_loss)
    rc = cuda_fail(cudaMemcpy(host_loss, dl, sizeof(float), cudaMemcpyDeviceToHost), "loss copy");
  cudaFree(dl);
  cudaFree(cnt);
  return rc;
}

int qca_net_labels_async(const uint8_t* noise, int L, int64_t shots, uint8_t* out_labels,
                         uint8_t* scratch, void* stream) {
  if (L < 4 || L > QCA_MAX_L || shots < 0 || (shots > 0 && (!noise || !out_labels || !scratch))) {
    set_error("qca_net_labels_async: bad arguments");
    return QCA_ERR_ARG;
  }
  if (shots == 0) return QCA_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = shots * (int64_t)L * L;
  uint8_t* sig = scratch;
  uint8_t* dir = scratch + n;
  syndrome_kernel<<<grid_for(n, 256), 256, 0, st>>>(noise, L, shots, sig);
  first_dir_kernel<<<grid_for(n, 256), 256, 0, st>>>(sig, L, shots, dir);
  mutual_label_kernel<<<grid_for(n, 256), 256, 0, st>>>(dir, L, shots, out_labels);
  return cuda_fail(cudaGetLastError(), "label kernels");
}

}  // extern "C"

namespace {

// Bytes of inference workspace per site: sig, prop, two bf16 activation maps
constexpr int64_t kWsPerSite = 2 + 2 * 64;

int64_t net_chunk(int L) {
  const int64_t per = (int64_t)L * L * kWsPerSite;
  const int64_t c = ((int64_t)4 << 30) / per;  // about 4 GiB of workspace
  return c < 1 ? 1 : c;
}

int net_workspace(qca_net_s* n, int64_t sites) {
  const size_t need = (size_t)sites * kWsPerSite + 512;
  if (n->ws_bytes >= need) return QCA_OK;
  if (n->ws) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "net workspace sync");
    cudaFree(n->ws);
    n->ws = nullptr;
    n->ws_bytes = 0;
  }
  cudaError_t e = cudaMalloc(&n->ws, need);
  if (e != cudaSuccess) return cuda_fail(e, "net workspace");
  n->ws_bytes = need;
  return QCA_OK;
}

// Net inference over `shots` noise realisations in chunks: logits (fp32
// [shots][4][L][L]) when `logits` is set, else proposals and the pairing
// (residual, optional C0).
int net_run(qca_net_s* n, const uint8_t* noise, int L, int64_t shots, float* logits,
            uint8_t* resid, uint8_t* c0, cudaStream_t st) {
  if (!n->prepared) {
    prepare_weights_kernel<<<64, 256, 0, st>>>(n->params, n->wb, n->w1);
    layer1_lut_kernel<<<64, 256, 0, st>>>(n->w1, n->params, n->lut);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "prepare weights");
    n->prepared = true;
  }
  if (n->precision == 1 && !n->prepared8) {
    prepare_fp8_kernel<<<72, 288, 0, st>>>(n->params, n->wq, n->wscale);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "prepare fp8 weights");
    n->prepared8 = true;
  }
  const int64_t LL = (int64_t)L * L;
  const int64_t chunk = net_chunk(L);
  int rc = net_workspace(n, (shots < chunk ? shots : chunk) * LL);
  if (rc) return rc;
  for (int64_t c0s = 0; c0s < shots; c0s += chunk) {
    const int64_t m = (shots - c0s < chunk) ? shots - c0s : chunk;
    const int64_t S = m * LL;
    uint8_t* sig = n->ws;
    uint8_t* prop = sig + S;
    __nv_bfloat16* actA =
        reinterpret_cast<__nv_bfloat16*>(n->ws + ((2 * S + 255) & ~(int64_t)255));
    __nv_bfloat16* actB = actA + S * 32;
    const uint8_t* Nc = noise + c0s * 2 * LL;
    syndrome_kernel<<<grid_for(S, 256), 256, 0, st>>>(Nc, L, m, sig);
    const int64_t tiles = (S + 15) / 16;
    const int gm = grid_for(tiles * 32, 128);
    if (n->precision == 1 && n->use_tc == 2 && L % kTcM == 0 && L % kTcStrip == 0) {
      // FP8 form on tcgen05 (kind::f8f6f4), warp-specialised; planar e4m3
      // activations, 32 bytes per site, in the bf16 buffers
      uint8_t* a8A = reinterpret_cast<uint8_t*>(actA);
      uint8_t* a8B = a8A + S * 32;
      const float* sa = n->act_scale;
      int dev = 0, sms = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      const int64_t units = S / ((int64_t)kTcM * kTcStrip);
      auto grid_of = [&](int ctas) {
        return (int)(units < (int64_t)sms * ctas ? units : (int64_t)sms * ctas);
      };
      const int gs = grid_of(WsShape<true>::ctas), gt = grid_of(WsShape<false>::ctas);
      if (c0s == 0) layer1_lut8_kernel<<<32, 256, 0, st>>>(n->w1, n->params, 1.f / sa[0], n->lut8);
      cudaFuncSetAttribute(conv_ws8_kernel<32, kActs, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)ws8_smem_bytes<32, true>());
      cudaFuncSetAttribute(conv_ws8_kernel<32, kActs, false>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)ws8_smem_bytes<32, false>());
      cudaFuncSetAttribute(conv_ws8_kernel<16, kLogits, false>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)ws8_smem_bytes<16, false>());
      cudaFuncSetAttribute(conv_ws8_kernel<16, kProposals, false>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)ws8_smem_bytes<16, false>());
      // layers 1 + 2 (layer 1 looked up while staging), 3, 4
      conv_ws8_kernel<32, kActs, true><<<gs, kWsThreads, ws8_smem_bytes<32, true>(), st>>>(
          nullptr, n->wq, n->wscale, n->params + kB1, sa[0], 1.f / sa[1], L, m, a8B, nullptr, sig,
          nullptr, n->err, n->lut8);
      conv_ws8_kernel<32, kActs, false><<<gt, kWsThreads, ws8_smem_bytes<32, false>(), st>>>(
          a8B, n->wq + 9 * 32 * 32, n->wscale + 32, n->params + kB2, sa[1], 1.f / sa[2], L, m,
          a8A, nullptr, nullptr, nullptr, n->err, nullptr);
      if (logits) {
        conv_ws8_kernel<16, kLogits, false><<<gt, kWsThreads, ws8_smem_bytes<16, false>(), st>>>(
            a8A, n->wq + 2 * 9 * 32 * 32, n->wscale + 64, n->params + kB3, sa[2], 0.f, L, m,
            nullptr, logits + c0s * 4 * LL, nullptr, nullptr, n->err, nullptr);
      } else {
        conv_ws8_kernel<16, kProposals, false><<<gt, kWsThreads, ws8_smem_bytes<16, false>(), st>>>(
            a8A, n->wq + 2 * 9 * 32 * 32, n->wscale + 64, n->params + kB3, sa[2], 0.f, L, m,
            nullptr, nullptr, sig, prop, n->err, nullptr);
        pairing_kernel<<<grid_for(S, 256), 256, 0, st>>>(Nc, prop, L, m, resid + c0s * 2 * LL,
                                                         c0 ? c0 + c0s * 2 * LL : nullptr);
      }
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_fail(e, "net fp8 tcgen05 inference kernels");
      continue;
    }
    if (n->precision == 1) {
      // FP8 form: e4m3 activations, 32 bytes per site, in the bf16 buffers
      uint8_t* a8A = reinterpret_cast<uint8_t*>(actA);
      uint8_t* a8B = a8A + S * 32;
      const float* sa = n->act_scale;
      layer1_fp8_kernel<<<grid_for(S, 256), 256, 0, st>>>(sig, L, m, n->w1, n->params,
                                                          1.f / sa[0], a8A);
      conv_fp8_kernel<4, kActs><<<gm, 128, 0, st>>>(a8A, n->wq, n->wscale, n->params + kB1,
                                                    sa[0], 1.f / sa[1], L, m, a8B, nullptr,
                                                    nullptr, nullptr);
      conv_fp8_kernel<4, kActs><<<gm, 128, 0, st>>>(a8B, n->wq + 9 * 32 * 32, n->wscale + 32,
                                                    n->params + kB2, sa[1], 1.f / sa[2], L, m,
                                                    a8A, nullptr, nullptr, nullptr);
      if (logits) {
        conv_fp8_kernel<1, kLogits><<<gm, 128, 0, st>>>(
            a8A, n->wq + 2 * 9 * 32 * 32, n->wscale + 64, n->params + kB3, sa[2], 0.f, L, m,
            nullptr, logits + c0s * 4 * LL, nullptr, nullptr);
      } else {
        conv_fp8_kernel<1, kProposals><<<gm, 128, 0, st>>>(
            a8A, n->wq + 2 * 9 * 32 * 32, n->wscale + 64, n->params + kB3, sa[2], 0.f, L, m,
            nullptr, nullptr, sig, prop);
        pairing_kernel<<<grid_for(S, 256), 256, 0, st>>>(Nc, prop, L, m, resid + c0s * 2 * LL,
                                                         c0 ? c0 + c0s * 2 * LL : nullptr);
      }
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_fail(e, "net fp8 inference kernels");
      continue;
    }
    if (n->use_tc == 2 && L % kTcM == 0 && L % kTcStrip == 0) {
      int dev = 0, sms = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      const int64_t units = S / ((int64_t)kTcM * kTcStrip);
      auto grid_of = [&](int ctas) {
        return (int)(units < (int64_t)sms * ctas ? units : (int64_t)sms * ctas);
      };
      const int gs = grid_of(WsShape<true>::ctas), gt = grid_of(WsShape<false>::ctas);
      cudaFuncSetAttribute(conv_ws_kernel<32, kActs, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)ws_smem_bytes<32, true>());
      cudaFuncSetAttribute(conv_ws_kernel<32, kActs, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)ws_smem_bytes<32, false>());
      cudaFuncSetAttribute(conv_ws_kernel<16, kLogits, false>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)ws_smem_bytes<16, false>());
      cudaFuncSetAttribute(conv_ws_kernel<16, kProposals, false>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)ws_smem_bytes<16, false>());
      // layers 1 + 2 (layer 1 looked up while staging), 3, 4
      conv_ws_kernel<32, kActs, true><<<gs, kWsThreads, ws_smem_bytes<32, true>(), st>>>(
          nullptr, n->wb, n->params + kB1, L, m, actB, nullptr, sig, nullptr, n->err, n->lut);
      conv_ws_kernel<32, kActs, false><<<gt, kWsThreads, ws_smem_bytes<32, false>(), st>>>(
          actB, n->wb + 9 * 32 * 32, n->params + kB2, L, m, actA, nullptr, nullptr, nullptr,
          n->err, nullptr);
      if (logits) {
        conv_ws_kernel<16, kLogits, false><<<gt, kWsThreads, ws_smem_bytes<16, false>(), st>>>(
            actA, n->wb + 2 * 9 * 32 * 32, n->params + kB3, L, m, nullptr, logits + c0s * 4 * LL,
            nullptr, nullptr, n->err, nullptr);
      } else {
        conv_ws_kernel<16, kProposals, false><<<gt, kWsThreads, ws_smem_bytes<16, false>(), st>>>(
            actA, n->wb + 2 * 9 * 32 * 32, n->params + kB3, L, m, nullptr, nullptr, sig, prop,
            n->err, nullptr);
        pairing_kernel<<<grid_for(S, 256), 256, 0, st>>>(Nc, prop, L, m, resid + c0s * 2 * LL,
                                                         c0 ? c0 + c0s * 2 * LL : nullptr);
      }
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_fail(e, "net warp-specialised tcgen05 kernels");
      continue;
    }
    if (n->use_tc && L % kTcM == 0 && L % kTcStrip == 0) {
      int dev = 0, sms = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      const int64_t units = S / ((int64_t)kTcM * kTcStrip);
      const int gt = (int)(units < (int64_t)sms * 4 ? units : (int64_t)sms * 4);
      cudaFuncSetAttribute(conv_tc_kernel<32, kActs, true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem_bytes<32>());
      cudaFuncSetAttribute(conv_tc_kernel<32, kActs, false>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem_bytes<32>());
      cudaFuncSetAttribute(conv_tc_kernel<16, kLogits, false>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem_bytes<16>());
      cudaFuncSetAttribute(conv_tc_kernel<16, kProposals, false>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem_bytes<16>());
      // layers 1 + 2 (layer 1 computed while staging), 3, 4
      conv_tc_kernel<32, kActs, true><<<gt, kTcThreads, tc_smem_bytes<32>(), st>>>(
          nullptr, n->wb, n->params + kB1, L, m, actB, nullptr, sig, nullptr, n->err, n->lut);
      conv_tc_kernel<32, kActs, false><<<gt, kTcThreads, tc_smem_bytes<32>(), st>>>(
          actB, n->wb + 9 * 32 * 32, n->params + kB2, L, m, actA, nullptr, nullptr, nullptr,
          n->err, nullptr);
      if (logits) {
        conv_tc_kernel<16, kLogits, false><<<gt, kTcThreads, tc_smem_bytes<16>(), st>>>(
            actA, n->wb + 2 * 9 * 32 * 32, n->params + kB3, L, m, nullptr, logits + c0s * 4 * LL,
            nullptr, nullptr, n->err, nullptr);
      } else {
        conv_tc_kernel<16, kProposals, false><<<gt, kTcThreads, tc_smem_bytes<16>(), st>>>(
            actA, n->wb + 2 * 9 * 32 * 32, n->params + kB3, L, m, nullptr, nullptr, sig, prop,
            n->err, nullptr);
        pairing_kernel<<<grid_for(S, 256), 256, 0, st>>>(Nc, prop, L, m, resid + c0s * 2 * LL,
                                                         c0 ? c0 + c0s * 2 * LL : nullptr);
      }
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_fail(e, "net tcgen05 inference kernels");
      continue;
    }
    layer1_kernel<<<grid_for(S, 256), 256, 0, st>>>(sig, L, m, n->w1, n->params, actA);
    conv_mma_kernel<4, kActs><<<gm, 128, 0, st>>>(actA, n->wb, n->params + kB1, L, m, actB,
                                                  nullptr, nullptr, nullptr, nullptr);
    conv_mma_kernel<4, kActs><<<gm, 128, 0, st>>>(actB, n->wb + 9 * 32 * 32, n->params + kB2, L, m,
                                                  actA, nullptr, nullptr, nullptr, nullptr);
    if (logits) {
      conv_mma_kernel<1, kLogits><<<gm, 128, 0, st>>>(actA, n->wb + 2 * 9 * 32 * 32,
                                                      n->params + kB3, L, m, nullptr,
                                                      logits + c0s * 4 * LL, nullptr, nullptr, nullptr);
    } else {
      conv_mma_kernel<1, kProposals><<<gm, 128, 0, st>>>(actA, n->wb + 2 * 9 * 32 * 32,
                                                         n->params + kB3, L, m, nullptr, nullptr,
                                                         sig, prop, nullptr);
      pairing_kernel<<<grid_for(S, 256), 256, 0, st>>>(Nc, prop, L, m, resid + c0s * 2 * LL,
                                                       c0 ? c0 + c0s * 2 * LL : nullptr);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "net inference kernels");
  }
  return QCA_OK;
}

}  // namespace

extern "C" {

int64_t qca_net_chunk_shots(int L) {
  if (L < 4 || L > QCA_MAX_L) {
    set_error("qca_net_chunk_shots: L = %d outside [4, %d]", L, QCA_MAX_L);
    return QCA_ERR_ARG;
  }
  return net_chunk(L);
}

int qca_net_logits_async(qca_net_t n, const uint8_t* noise, int L, int64_t shots,
                         float* out_logits, void* stream) {
  if (!n || L < 4 || L > QCA_MAX_L || shots < 0 || (shots > 0 && (!noise || !out_logits))) {
    set_error("qca_net_logits_async: bad arguments");
    return QCA_ERR_ARG;
  }
  if (int rc = check_aligned(out_logits, 4, "out_logits")) return rc;
  if (shots == 0) return QCA_OK;
  return net_run(n, noise, L, shots, out_logits, nullptr, nullptr, (cudaStream_t)stream);
}

int qca_net_activations(qca_net_t n, const uint8_t* noise, int L, int64_t shots, int layer,
                        float* out) {
  if (!n || L < 4 || L > QCA_MAX_L || shots < 1 || !noise || !out || layer < 1 || layer > 3) {
    set_error("qca_net_activations: bad arguments");
    return QCA_ERR_ARG;
  }
  if (shots > net_chunk(L)) {
    set_error("qca_net_activations: at most %lld shots at L = %d (one inference chunk)",
              (long long)net_chunk(L), L);
    return QCA_ERR_ARG;
  }
  if (int rc = check_aligned(out, 4, "out")) return rc;
  const int64_t LL = (int64_t)L * L, S = shots * LL;
  float* logits = nullptr;
  cudaError_t e = cudaMalloc(&logits, sizeof(float) * 4 * S);
  if (e != cudaSuccess) return cuda_fail(e, "qca_net_activations buffer");
  int rc = net_run(n, noise, L, shots, logits, nullptr, nullptr, nullptr);
  const bool tc_tile = L % kTcM == 0 && L % kTcStrip == 0;
  const bool fp8 = n->precision == 1;
  const bool planar = n->use_tc == 2 && tc_tile;
  uint8_t* sig = n->ws;
  __nv_bfloat16* actA = reinterpret_cast<__nv_bfloat16*>(n->ws + ((2 * S + 255) & ~(int64_t)255));
  __nv_bfloat16* actB = actA + S * 32;
  const void* src = nullptr;
  int form = 0;
  if (rc == QCA_OK) {
    if (layer == 1) {
      if (fp8) {
        layer1_lut8_kernel<<<32, 256>>>(n->w1, n->params, 1.f / n->act_scale[0], n->lut8);
        src = n->lut8;
        form = 5;
      } else {
        src = n->lut;
        form = 4;
      }
    } else {
      // the FP8 form keeps its e4m3 maps (32 bytes per site) in the same
      // workspace: layer 2 at byte S * 32, layer 3 at the start
      const uint8_t* a8A = reinterpret_cast<const uint8_t*>(actA);
      src = fp8 ? ((layer == 2) ? (const void*)(a8A + S * 32) : (const void*)a8A)
                : ((layer == 2) ? (const void*)actB : (const void*)actA);
      form = fp8 ? (planar ? 3 : 2) : (planar ? 1 : 0);
    }
    capture_kernel<<<grid_for(S * 32, 256), 256>>>(src, form, sig, L, shots, out);
    rc = cuda_fail(cudaGetLastError(), "activation read-out");
  }
  if (rc == QCA_OK) rc = cuda_fail(cudaDeviceSynchronize(), "qca_net_activations");
  cudaFree(logits);
  return rc;
}

int qca_net_predecode_async(qca_net_t n, const uint8_t* noise, int L, int64_t shots,
                            uint8_t* out_residual, uint8_t* out_c0, void* stream) {
  if (!n || L < 4 || L > QCA_MAX_L || shots < 0 || (shots > 0 && (!noise || !out_residual))) {
    set_error("qca_net_predecode_async: bad arguments");
    return QCA_ERR_ARG;
  }
  if (shots == 0) return QCA_OK;
  return net_run(n, noise, L, shots, nullptr, out_residual, out_c0, (cudaStream_t)stream);
}

int qca_net_set_fp8_scales(qca_net_t n, const float* scales) {
  if (!n || !scales || !(scales[0] > 0.f && scales[1] > 0.f && scales[2] > 0.f)) {
    set_error("qca_net_set_fp8_scales: NULL or non-positive scale");
    return QCA_ERR_ARG;
  }
  for (int i = 0; i < 3; ++i) n->act_scale[i] = scales[i];
  return QCA_OK;
}

int qca_net_get_fp8_scales(qca_net_t n, float* scales) {
  if (!n || !scales) {
    set_error("qca_net_get_fp8_scales: NULL argument");
    return QCA_ERR_ARG;
  }
  for (int i = 0; i < 3; ++i) scales[i] = n->act_scale[i];
  return QCA_OK;
}

int qca_net_set_tensor_path(qca_net_t n, int path) {
  if (!n || path < 0 || path > 2) {
    set_error("qca_net_set_tensor_path: 0 (mma.sync), 1 (tcgen05, row-synchronous) or 2 "
              "(tcgen05, warp-specialised), the tcgen05 forms where L %% 128 == 0");
    return QCA_ERR_ARG;
  }
  n->use_tc = path;
  return QCA_OK;
}

int qca_net_status(qca_net_t n) {
  if (!n) {
    set_error("qca_net_status: NULL net");
    return QCA_ERR_ARG;
  }
  unsigned int h = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&h, n->err, sizeof(h), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "qca_net_status");
  if (h) {
    cudaMemset(n->err, 0, sizeof(h));
    set_error("qca_net_status: a tensor-core wait timed out; the outputs since the last check are unreliable");
    return QCA_ERR_WATCHDOG;
  }
  return QCA_OK;
}

int qca_watchdog_selftest(int* first_gave_up, int* second_gave_up, double* first_wait_s,
                          double* second_lag_s) {
  unsigned int* d = nullptr;
  unsigned int h[4] = {0, 0, 0, 0};
  cudaError_t e = cudaMalloc(&d, sizeof(h));
  if (e == cudaSuccess) e = cudaMemset(d, 0, sizeof(h));
  if (e == cudaSuccess) {
    watchdog_selftest_kernel<<<1, 64>>>(d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(e, "qca_watchdog_selftest");
  int clk_khz = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
  const double hz = clk_khz > 0 ? clk_khz * 1e3 : 0.0;
  if (first_gave_up) *first_gave_up = (int)h[0];
  if (second_gave_up) *second_gave_up = (int)h[1];
  if (first_wait_s) *first_wait_s = hz > 0 ? (double)h[2] * 1048576.0 / hz : -1.0;
  if (second_lag_s) *second_lag_s = hz > 0 ? (double)h[3] * 1024.0 / hz : -1.0;
  return QCA_OK;
}

int qca_net_set_precision(qca_net_t n, int precision) {
  if (!n || (precision != 0 && precision != 1)) {
    set_error("qca_net_set_precision: precision must be 0 (bf16) or 1 (fp8)");
    return QCA_ERR_ARG;
  }
  if (precision == 1 && !(n->act_scale[0] > 0.f && n->act_scale[1] > 0.f && n->act_scale[2] > 0.f)) {
    set_error("qca_net_set_precision: fp8 needs activation scales (calibrate or set them)");
    return QCA_ERR_ARG;
  }
  n->precision = precision;
  return QCA_OK;
}

int qca_net_calibrate_fp8(qca_net_t n, const uint8_t* noise, int L, int64_t shots, void* stream) {
  if (!n || L < 4 || L > QCA_MAX_L || shots < 1 || !noise) {
    set_error("qca_net_calibrate_fp8: bad arguments");
    return QCA_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (!n->prepared) {
    prepare_weights_kernel<<<64, 256, 0, st>>>(n->params, n->wb, n->w1);
    layer1_lut_kernel<<<64, 256, 0, st>>>(n->w1, n->params, n->lut);
    n->prepared = true;
  }
  const int64_t LL = (int64_t)L * L;
  const int64_t m = shots < net_chunk(L) ? shots : net_chunk(L);
  int rc = net_workspace(n, m * LL);
  if (rc) return rc;
  unsigned int* amax = nullptr;
  cudaError_t e = cudaMalloc(&amax, 3 * sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemsetAsync(amax, 0, 3 * sizeof(unsigned int), st);
  if (e != cudaSuccess) {
    cudaFree(amax);
    return cuda_fail(e, "calibration buffer");
  }
  const int64_t S = m * LL;
  uint8_t* sig = n->ws;
  __nv_bfloat16* actA = reinterpret_cast<__nv_bfloat16*>(n->ws + ((2 * S + 255) & ~(int64_t)255));
  __nv_bfloat16* actB = actA + S * 32;
  const int gm = grid_for((S + 15) / 16 * 32, 128);
  const int ga = grid_for(S * 32, 256);
  syndrome_kernel<<<grid_for(S, 256), 256, 0, st>>>(noise, L, m, sig);
  layer1_kernel<<<grid_for(S, 256), 256, 0, st>>>(sig, L, m, n->w1, n->params, actA);
  amax_bf16_kernel<<<ga, 256, 0, st>>>(actA, S * 32, amax + 0);
  conv_mma_kernel<4, kActs><<<gm, 128, 0, st>>>(actA, n->wb, n->params + kB1, L, m, actB, nullptr,
                                                nullptr, nullptr, nullptr);
  amax_bf16_kernel<<<ga, 256, 0, st>>>(actB, S * 32, amax + 1);
  conv_mma_kernel<4, kActs><<<gm, 128, 0, st>>>(actB, n->wb + 9 * 32 * 32, n->params + kB2, L, m,
                                                actA, nullptr, nullptr, nullptr, nullptr);
  amax_bf16_kernel<<<ga, 256, 0, st>>>(actA, S * 32, amax + 2);
  unsigned int h[3] = {0, 0, 0};
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, amax, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(amax);
  if (e != cudaSuccess) return cuda_fail(e, "qca_net_calibrate_fp8");
  for (int i = 0; i < 3; ++i) {
    float a;
    memcpy(&a, &h[i], sizeof(a));
    n->act_scale[i] = a > 0.f ? a / 448.f : 1.f;
  }
  return QCA_OK;
}

int qca_net_decode_batch_async(qca_net_t n, const uint8_t* noise, int L, int64_t shots,
                               int max_steps, uint64_t rng_seed, uint8_t* out_correction,
                               int32_t* out_steps, uint8_t* out_logical_fail,
                               const qca_config* cfg, uint8_t* residual_scratch, void* stream) {
  if (!n || (shots > 0 && !residual_scratch)) {
    set_error("qca_net_decode_batch_async: NULL net or residual scratch");
    return QCA_ERR_ARG;
  }
  int rc = qca_net_predecode_async(n, noise, L, shots, residual_scratch, nullptr, stream);
  if (rc) return rc;
  rc = qca_decode_batch_async(residual_scratch, L, shots, max_steps, rng_seed, out_correction,
                              out_steps, out_logical_fail, cfg, stream);
  if (rc || shots == 0) return rc;
  const int64_t E = shots * 2 * (int64_t)L * L;
  combine_kernel<<<grid_for(E / 16 + 1, 256), 256, 0, (cudaStream_t)stream>>>(
      out_correction, noise, residual_scratch, E);
  return cuda_fail(cudaGetLastError(), "combine kernel");
}

}  // extern "C"
