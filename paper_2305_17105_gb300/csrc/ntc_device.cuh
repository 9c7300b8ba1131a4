// Device-side building blocks of the NTC hot path: query -> texel, feature
// level selection, bilinear taps, dequantisation, positional encoding,
// counter-based random numbers and the training-texel sampler.
//
// Paper: "Random-Access Neural Compression of Material Textures" (2023).
#pragma once

#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include "ntc.h"

namespace ntc {

constexpr int kTile = 128;       // queries per CTA tile (one per thread)
constexpr int kHidden = NTC_HIDDEN;
constexpr int kMaxC = NTC_MAX_CHANNELS;
constexpr int kMaxGridCh = 20;   // features per cell of one grid (Sec. 6: profile 0.5's G1)
constexpr int kGridPad = 24;     // kMaxGridCh rounded up to whole groups of 8 features
constexpr int kFastGridCh = 16;  // widest grid of the 16-byte-vector gather paths

// ---------------------------------------------------------------------------
// Counter-based random numbers: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014),
// golden-gamma increment followed by the variant-13 output mix.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
// Per-(seed, stream) key; a draw is splitmix64(key ^ counter).
__host__ __device__ __forceinline__ uint64_t rng_key(uint64_t seed, uint64_t stream) {
  return splitmix64(seed ^ splitmix64(stream));
}
// Streams of training step s: the texel sampler uses 2s, the noise 2s+1.
__host__ __device__ __forceinline__ uint64_t sampler_stream(int64_t step) {
  return (uint64_t)step << 1;
}
__host__ __device__ __forceinline__ uint64_t noise_stream(int64_t step) {
  return ((uint64_t)step << 1) | 1u;
}

// ---------------------------------------------------------------------------
// Pyramid rules (Sec. 4.1, Table 1)
// ---------------------------------------------------------------------------
// Feature level of mip m: level 0 serves mips 0..3, later levels two mips
// each, the last level every remaining mip.
__host__ __device__ __forceinline__ int level_of_mip(int m, int levels) {
  int j = m < 4 ? 0 : (m - 2) >> 1;
  return j < levels - 1 ? j : levels - 1;
}
__host__ __device__ __forceinline__ int mip_dim(int side, int m) {
  int s = side >> m;
  return s > 0 ? s : 1;
}

// Nearest texel of a (u, v, lod) query: m = floor(lod) in [0, M-1],
// x = floor(u * w_m) in [0, w_m - 1]; NaN counts as 0.  u * w_m is exact
// (w_m is a power of two), so x matches a double-precision evaluation.
__device__ __forceinline__ void query_texel(const ntc_material& M, float u, float v, float lod,
                                            int& x, int& y, int& m) {
  int mm;
  if (!(lod >= 0.f)) mm = 0;
  else if (lod >= (float)(M.mips - 1)) mm = M.mips - 1;
  else mm = (int)floorf(lod);
  const int wm = mip_dim(M.width, mm), hm = mip_dim(M.height, mm);
  const float tu = u * (float)wm, tv = v * (float)hm;
  x = !(tu >= 0.f) ? 0 : (tu >= (float)wm ? wm - 1 : (int)floorf(tu));
  y = !(tv >= 0.f) ? 0 : (tv >= (float)hm ? hm - 1 : (int)floorf(tv));
  m = mm;
}

// Stochastic filtering (Sec. 5.3).  Query q of frame `step` takes one
// SplitMix64 draw h = splitmix64(jitter_key ^ q): xi_x = h[40,64) 2^-24,
// xi_y = h[16,40) 2^-24, xi_l = h[0,16) 2^-16.  The texel is the nearest one
// of the jittered position u w_m - 1/2 + xi_x (x0 or x0 + 1 with the
// bilinear weights; taps wrap like the trilinear filter's), the mip
// floor(lod + xi_l) (floor(lod) or floor(lod) + 1 with the linear weights).
// Every step is an FP32 operation without contraction, so the texel choice
// is reproducible bit for bit; u is taken as 0 when NaN and clamped to
// +-16384 (textures repeat).
__host__ __device__ __forceinline__ uint64_t jitter_key(uint64_t seed, int64_t step) {
  return rng_key(seed, ((uint64_t)step << 2) | 2u);
}
__device__ __forceinline__ int stochastic_mip(float lod, int mips, uint64_t h) {
  const float xl = (float)(uint32_t)(h & 0xFFFFu) * (1.f / 65536.f);
  const float l = !(lod >= 0.f) ? 0.f : fminf(lod, (float)(mips - 1));
  return min((int)floorf(__fadd_rn(l, xl)), mips - 1);
}
__device__ __forceinline__ int stochastic_coord(float u, int w, uint32_t b24) {
  const float xi = (float)b24 * (1.f / 16777216.f);
  const float uc = fminf(fmaxf(u == u ? u : 0.f, -16384.f), 16384.f);
  const float p = __fadd_rn(__fadd_rn(__fmul_rn(uc, (float)w), -0.5f), xi);
  const int i = (int)floorf(p);
  return (i % w + w) % w;
}

// Bilinear taps of a gw x gh grid for texel (x, y) of a wm x hm mip
// (Sec. 4.3.1): texel centre (x + 1/2)/wm maps to p = centre * gw - 1/2 in
// cell-centre coordinates; taps clamp to the grid edge.  With power-of-two
// sizes every step is exact in FP32, so the weights equal the double ones.
struct Taps {
  int cell[4];
  float w[4];
};
__device__ __forceinline__ Taps bilinear_taps(int x, int y, int wm, int hm, int gw, int gh) {
  const float px = ((float)x + 0.5f) / (float)wm * (float)gw - 0.5f;
  const float py = ((float)y + 0.5f) / (float)hm * (float)gh - 0.5f;
  const float fx0 = floorf(px), fy0 = floorf(py);
  const float fx = px - fx0, fy = py - fy0;
  int ix0 = (int)fx0, iy0 = (int)fy0;
  int ix1 = min(max(ix0 + 1, 0), gw - 1), iy1 = min(max(iy0 + 1, 0), gh - 1);
  ix0 = min(max(ix0, 0), gw - 1);
  iy0 = min(max(iy0, 0), gh - 1);
  Taps t;
  t.cell[0] = iy0 * gw + ix0; t.w[0] = (1.f - fx) * (1.f - fy);
  t.cell[1] = iy0 * gw + ix1; t.w[1] = fx * (1.f - fy);
  t.cell[2] = iy1 * gw + ix0; t.w[2] = (1.f - fx) * fy;
  t.cell[3] = iy1 * gw + ix1; t.w[3] = fx * fy;
  return t;
}

// Triangle wave with period 1: +1 at t = 0, -1 at t = 1/2.
__device__ __forceinline__ float tri(float t) { return 4.f * fabsf(t - 0.5f) - 1.f; }

// Tiled positional encoding (Sec. 4.3.2): per axis, octaves of period 8, 4
// and 2 texels, a sine-like then a cosine-like triangle wave each; x first.
// All values are dyadic and exact.
template <class Sink>
__device__ __forceinline__ void positional_encoding(int x, int y, int base, Sink& sink) {
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const int c = a ? y : x;
#pragma unroll
    for (int h = 0; h < 3; ++h) {
      const float period = (float)(8 >> h);
      float t = ((float)c + 0.5f) / period;
      t -= floorf(t);
      float ts = t - 0.25f;
      ts -= floorf(ts);
      sink(base + 6 * a + 2 * h + 0, tri(ts));
      sink(base + 6 * a + 2 * h + 1, tri(t));
    }
  }
}

// One uniform draw of the simulated-quantisation noise (Sec. 4.2): a 64-bit
// draw per (level, grid, cell, channel pair); even channels use bits 40..63,
// odd channels bits 16..39, noise = (u - 1/2) * Q.
__device__ __forceinline__ float noise_of(uint64_t key, int level, int grid, int cell, int ch,
                                          int c, float q) {
  const uint64_t pairs = (uint64_t)((c + 1) >> 1);
  const uint64_t counter = ((uint64_t)(2 * level + grid) << 40) |
                           ((uint64_t)cell * pairs + (uint64_t)(ch >> 1));
  const uint64_t h = splitmix64(key ^ counter);
  const uint32_t b24 = (ch & 1) ? (uint32_t)((h >> 16) & 0xFFFFFFu) : (uint32_t)(h >> 40);
  return ((float)b24 * (1.0f / 16777216.0f) - 0.5f) * q;
}

// Packed cell of up to 16 bytes.
struct Cell {
  uint64_t lo, hi;
};
__device__ __forceinline__ Cell load_cell(const uint8_t* base, int cell, int cb) {
  Cell c{0, 0};
  const uint8_t* p = base + (size_t)cell * cb;
  switch (cb) {
    case 1: c.lo = __ldg(p); break;
    case 2: c.lo = __ldg(reinterpret_cast<const uint16_t*>(p)); break;
    case 4: c.lo = __ldg(reinterpret_cast<const uint32_t*>(p)); break;
    case 8: c.lo = __ldg(reinterpret_cast<const unsigned long long*>(p)); break;
    default: {
      const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
      c.lo = ((uint64_t)v.y << 32) | v.x;
      c.hi = ((uint64_t)v.w << 32) | v.z;
    }
  }
  return c;
}
__device__ __forceinline__ uint32_t cell_index(const Cell& c, int ch, int bits) {
  const int bit = ch * bits;
  const uint64_t w = bit < 64 ? c.lo : c.hi;
  return (uint32_t)(w >> (bit & 63)) & ((1u << bits) - 1u);
}

__host__ __device__ __forceinline__ int cell_bytes(int c, int bits) {
  int need = (c * bits + 7) / 8, b = 1;
  while (b < need) b <<= 1;
  return b;
}

// ---------------------------------------------------------------------------
// Features of one grid at texel (x, y) of mip m: acc[ch] = sum_t w_t g_t[ch].
// ---------------------------------------------------------------------------
struct GridSample {
  float acc[kGridPad];  // channels >= c are zero
};

// Vector-quantised G0 (vq_books > 0): the c0 features of cell `cell` of
// level j, the sum of the codebook entries its indices select.
__device__ __forceinline__ void vq_cell(const ntc_material& M, int j, int cell,
                                        float (&v)[kMaxGridCh]) {
  const uint8_t* ib = static_cast<const uint8_t*>(M.lv[j].grid0) + (size_t)cell * M.vq_books;
#pragma unroll
  for (int ch = 0; ch < kMaxGridCh; ++ch) v[ch] = 0.f;
  for (int b = 0; b < M.vq_books; ++b) {
    const float* e = M.codebook0 + ((size_t)b * 256 + ib[b]) * M.c0;
    if ((M.c0 & 3) == 0) {  // rows of 4k values: float4 reads
#pragma unroll
      for (int q4 = 0; q4 < kMaxGridCh / 4; ++q4)
        if (4 * q4 < M.c0) {
          const float4 f = __ldg(reinterpret_cast<const float4*>(e) + q4);
          v[4 * q4] += f.x; v[4 * q4 + 1] += f.y; v[4 * q4 + 2] += f.z; v[4 * q4 + 3] += f.w;
        }
    } else {
#pragma unroll
      for (int ch = 0; ch < kMaxGridCh; ++ch)
        if (ch < M.c0) v[ch] += __ldg(e + ch);
    }
  }
}

__device__ __forceinline__ void sample_grid(const ntc_material& M, int j, int k, int x, int y,
                                            int wm, int hm, bool noise, uint64_t nkey,
                                            GridSample& gs, Taps* taps_out = nullptr) {
  const ntc_level& L = M.lv[j];
  const int gw = k ? L.g1_w : L.g0_w, gh = k ? L.g1_h : L.g0_h;
  const int c = k ? M.c1 : M.c0;
  const float q = k ? M.q1 : M.q0;
  const Taps t = bilinear_taps(x, y, wm, hm, gw, gh);
  if (taps_out) *taps_out = t;
#pragma unroll
  for (int ch = 0; ch < kGridPad; ++ch) gs.acc[ch] = 0.f;
  if (k == 0 && M.vq_books > 0) {
#pragma unroll
    for (int tp = 0; tp < 4; ++tp) {
      float v[kMaxGridCh];
      vq_cell(M, j, t.cell[tp], v);
#pragma unroll
      for (int ch = 0; ch < kMaxGridCh; ++ch)
        if (ch < c) gs.acc[ch] = fmaf(t.w[tp], v[ch], gs.acc[ch]);
    }
    return;
  }
  if (M.encoding == NTC_GRID_PACKED) {
    const int bits = k ? M.bits1 : M.bits0;
    const int off = (1 << (bits - 1)) - 1;
    const int cb = cell_bytes(c, bits);
    const uint8_t* base = static_cast<const uint8_t*>(k ? L.grid1 : L.grid0);
#pragma unroll
    for (int tp = 0; tp < 4; ++tp) {
      const Cell cl = load_cell(base, t.cell[tp], cb);
#pragma unroll
      for (int ch = 0; ch < kMaxGridCh; ++ch)
        if (ch < c) {
          const float v = (float)((int)cell_index(cl, ch, bits) - off) * q;
          gs.acc[ch] = fmaf(t.w[tp], v, gs.acc[ch]);
        }
    }
  } else {
    const float* base = static_cast<const float*>(k ? L.grid1 : L.grid0);
#pragma unroll
    for (int tp = 0; tp < 4; ++tp) {
      const float* g = base + (size_t)t.cell[tp] * c;
      if ((c & 3) == 0) {
#pragma unroll
        for (int c4 = 0; c4 < kMaxGridCh / 4; ++c4)
          if (4 * c4 < c) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(g) + c4);
            float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              float val = e[i];
              if (noise) val += noise_of(nkey, j, k, t.cell[tp], 4 * c4 + i, c, q);
              gs.acc[4 * c4 + i] = fmaf(t.w[tp], val, gs.acc[4 * c4 + i]);
            }
          }
      } else {
#pragma unroll
        for (int ch = 0; ch < kMaxGridCh; ++ch)
          if (ch < c) {
            float val = __ldg(g + ch);
            if (noise) val += noise_of(nkey, j, k, t.cell[tp], ch, c, q);
            gs.acc[ch] = fmaf(t.w[tp], val, gs.acc[ch]);
          }
      }
    }
  }
}

// One latent value of grid k at a cell: dequantised index (packed) or the
// FP32 value plus this step's noise.
__device__ __forceinline__ float grid_value(const ntc_material& M, int j, int k, int cell, int ch,
                                            bool noise, uint64_t nkey) {
  const ntc_level& L = M.lv[j];
  if (k == 0 && M.vq_books > 0) {
    const uint8_t* ib = static_cast<const uint8_t*>(L.grid0) + (size_t)cell * M.vq_books;
    float v = 0.f;
    for (int b = 0; b < M.vq_books; ++b)
      v += __ldg(M.codebook0 + ((size_t)b * 256 + ib[b]) * M.c0 + ch);
    return v;
  }
  const int c = k ? M.c1 : M.c0;
  const float q = k ? M.q1 : M.q0;
  if (M.encoding == NTC_GRID_PACKED) {
    const int bits = k ? M.bits1 : M.bits0;
    const Cell cl = load_cell(static_cast<const uint8_t*>(k ? L.grid1 : L.grid0), cell,
                              cell_bytes(c, bits));
    return (float)((int)cell_index(cl, ch, bits) - ((1 << (bits - 1)) - 1)) * q;
  }
  float val = __ldg(static_cast<const float*>(k ? L.grid1 : L.grid0) + (size_t)cell * c + ch);
  if (noise) val += noise_of(nkey, j, k, cell, ch, c, q);
  return val;
}

// The MLP input row of texel (x, y, m) (Sec. 4.3, 4.4):
// [G0 features | G1 features | 12 PE values | m/(M-1) | 0 ...], written
// through sink(index, value) for indices 0 .. k_in-1.
template <class Sink>
__device__ __forceinline__ void featurize(const ntc_material& M, int x, int y, int m, bool noise,
                                          uint64_t nkey, Sink& sink) {
  const int j = level_of_mip(m, M.levels);
  const int wm = mip_dim(M.width, m), hm = mip_dim(M.height, m);
  GridSample gs;
  int w0 = M.c0;
  if (M.interp0 == NTC_INTERP_LEARNED) {
    // learned interpolation (Sec. 4.3.1): the four G0 taps concatenated
    const ntc_level& L = M.lv[j];
    const Taps t = bilinear_taps(x, y, wm, hm, L.g0_w, L.g0_h);
#pragma unroll 1
    for (int tp = 0; tp < 4; ++tp)
      for (int ch = 0; ch < M.c0; ++ch) sink(tp * M.c0 + ch, grid_value(M, j, 0, t.cell[tp], ch, noise, nkey));
    w0 = 4 * M.c0;
  } else {
    sample_grid(M, j, 0, x, y, wm, hm, noise, nkey, gs);
#pragma unroll
    for (int ch = 0; ch < kMaxGridCh; ++ch)
      if (ch < M.c0) sink(ch, gs.acc[ch]);
  }
  sample_grid(M, j, 1, x, y, wm, hm, noise, nkey, gs);
#pragma unroll
  for (int ch = 0; ch < kMaxGridCh; ++ch)
    if (ch < M.c1) sink(w0 + ch, gs.acc[ch]);
  const int pe = w0 + M.c1;
  positional_encoding(x, y, pe, sink);
  sink(pe + 12, M.mips > 1 ? (float)m / (float)(M.mips - 1) : 0.f);
  for (int i = pe + 13; i < M.k_in; ++i) sink(i, 0.f);
}

// Level of detail of a training draw (Sec. 5.1) from the hashes of counters
// c0, c1: with probability 0.05 a mip uniform over the chain, else LOD =
// floor(-log4 X), X = k/2^24, k = (draw>>40)+1, i.e. the largest m with
// k <= 2^(24-2m), clamped to the last mip.  Integer-only, identical on every
// platform.
__device__ __forceinline__ int sampled_lod(uint64_t skey, uint64_t c0, uint64_t c1, int mips) {
  const uint64_t h0 = splitmix64(skey ^ c0);
  if ((h0 >> 40) < 838861ull) return (int)(((h0 & 0xFFFFFFFFull) * (uint64_t)mips) >> 32);
  const uint64_t kk = (splitmix64(skey ^ c1) >> 40) + 1;
  int mm = 0;
#pragma unroll
  for (int t = 1; t <= 12; ++t)
    if (kk <= (1ull << (24 - 2 * t))) mm = t;
  return mm > mips - 1 ? mips - 1 : mm;
}

// Training texel i of a step, independent texels: its own LOD (counters
// 4i, 4i+1), then a uniform texel of that mip (counter 4i+2).
__device__ __forceinline__ void sample_texel(uint64_t skey, int64_t i, int width, int height,
                                             int mips, int& x, int& y, int& m) {
  const int mm = sampled_lod(skey, 4ull * (uint64_t)i + 0, 4ull * (uint64_t)i + 1, mips);
  const uint64_t h2 = splitmix64(skey ^ (4ull * (uint64_t)i + 2));
  const uint64_t wm = (uint64_t)mip_dim(width, mm), hm = (uint64_t)mip_dim(height, mm);
  x = (int)(((h2 & 0xFFFFFFFFull) * wm) >> 32);
  y = (int)(((h2 >> 32) * hm) >> 32);
  m = mm;
}

// Training texel i of a step cut into crops (Sec. 5.1): one LOD for the
// whole batch (counters 0, 1); crop k = i / S^2 (S = kCropSide) has its
// origin uniform over the mip (counter 4k+2) and wraps around the mip's
// edges (the material tiles); texel i sits at (i mod S, (i / S) mod S)
// inside its crop.
constexpr int kCropSide = 256;
__device__ __forceinline__ void sample_crop_texel(uint64_t skey, int64_t i, int width, int height,
                                                  int mips, int& x, int& y, int& m) {
  const int mm = sampled_lod(skey, 0, 1, mips);
  const uint64_t k = (uint64_t)i / (uint64_t)(kCropSide * kCropSide);
  const uint64_t h2 = splitmix64(skey ^ (4ull * k + 2));
  const uint64_t wm = (uint64_t)mip_dim(width, mm), hm = (uint64_t)mip_dim(height, mm);
  const uint64_t x0 = ((h2 & 0xFFFFFFFFull) * wm) >> 32, y0 = ((h2 >> 32) * hm) >> 32;
  x = (int)((x0 + (uint64_t)i % kCropSide) % wm);
  y = (int)((y0 + (uint64_t)i / kCropSide % kCropSide) % hm);
  m = mm;
}

// The sampler of a training step: crops or independent texels.
__device__ __forceinline__ void sample_train_texel(bool crops, uint64_t skey, int64_t i, int width,
                                                   int height, int mips, int& x, int& y, int& m) {
  if (crops) sample_crop_texel(skey, i, width, height, mips, x, y, m);
  else sample_texel(skey, i, width, height, mips, x, y, m);
}

// Activations (Sec. 4.4).
__device__ __forceinline__ float act_fwd(int act, float z) {
  if (act == NTC_ACT_HARDGELU) {
    if (z < -1.5f) return 0.f;
    if (z > 1.5f) return z;
    return z * (1.f / 3.f) * (z + 1.5f);
  }
  return fmaxf(z, 0.f);
}
__device__ __forceinline__ float act_grad(int act, float z) {
  if (act == NTC_ACT_HARDGELU) {
    if (z < -1.5f) return 0.f;
    if (z > 1.5f) return 1.f;
    return (2.f * z + 1.5f) * (1.f / 3.f);
  }
  return z > 0.f ? 1.f : 0.f;
}
__device__ __forceinline__ float out_fwd(int out_act, float z) {
  return out_act == NTC_OUT_IDENTITY ? z : 1.f / (1.f + __expf(-z));
}

// Element idx of the third hidden layer's weights (hidden_layers == 3) as
// float: FP32 or FP16.
__device__ __forceinline__ float load_weight_h3(const ntc_material& M, int idx) {
  if (M.precision == NTC_PREC_F16) return __half2float(static_cast<const __half*>(M.w_h3)[idx]);
  return static_cast<const float*>(M.w_h3)[idx];
}

// Weight element l (0..2) at [o][i] as float, from the material's precision.
__device__ __forceinline__ float load_weight(const ntc_material& M, int l, int idx) {
  switch (M.precision) {
    case NTC_PREC_F16: return __half2float(static_cast<const __half*>(M.w[l])[idx]);
    case NTC_PREC_F8: {
      const __nv_fp8_e4m3 v = static_cast<const __nv_fp8_e4m3*>(M.w[l])[idx];
      return (float)v * M.scale[l];
    }
    default: return static_cast<const float*>(M.w[l])[idx];
  }
}

}  // namespace ntc
