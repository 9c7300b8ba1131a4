// Device building blocks shared by the tensor-core decode kernels
// (tc_decode.cu: warpgroup pipelines, FP8, many materials; tc_decode_ws.cu:
// the warp-specialised form): the input-row plan and its shared-memory
// staging, the query -> texel -> cells front end, the 4-bit fast-layout and
// generic feature builders, the epilogues and the output store.
#pragma once

#include <cuda_fp16.h>

#include <cmath>

#include "ntc_device.cuh"
#include "ntc_internal.h"
#include "tc_ptx.cuh"

namespace ntc {
namespace {


constexpr int kRows = 128;
constexpr int kN3 = 16;
// TMEM columns of a warpgroup (128): the FP32 accumulator D, the hidden
// rows H (A operand of layers 2 and 3), the input rows X (A operand of layer
// 1; separate from H so the next tile's X is built while layer 2 runs) and the
// constant-one block of the FP16 bias steps.
constexpr int kColH = 64;              // FP16: 32 columns (64 halves); FP8: 16
constexpr int kColX = 96;              // FP16: up to 24 columns (48 halves); FP8: 16
constexpr int kColCst = 120;           // FP16: 8 columns
constexpr uint32_t kWaitLimit = 1u << 18;  // suspended tries: ms to seconds
// Shared-memory B descriptor table: W1 K-steps [0, 8) (K <= 128), W2 [8, 12),
// its bias block 12, W3 [13, 17), its bias block 17, and with a third hidden
// layer (FP16) Wh [18, 22), its bias block 22.
constexpr int kDescW2 = 8, kDescW3 = 13, kDescWh = 18, kDescs = 23;

template <bool F8>
struct Cfg {
  static constexpr int EB = F8 ? 1 : 2;       // operand bytes
  static constexpr int KSTEP = F8 ? 32 : 16;  // K per MMA instruction (= 8 TMEM columns)
};

// Per-mip constants (structure of arrays: lanes that look up different mips
// read different banks).
struct MipTab {
  // fast layout: per grid {8 G_x / w_m, 8 G_y / h_m, G_x, G_y}: the texel
  // centre 2x+1 times the first entry, minus 8, is the tap position in 1/16
  // cell units
  int4 tk0[NTC_MAX_MIPS], tk1[NTC_MAX_MIPS];
  uint32_t lodh[NTC_MAX_MIPS];  // half2 (LOD input, 0)
  const uint8_t* grid0[NTC_MAX_MIPS];
  const uint8_t* grid1[NTC_MAX_MIPS];
  int wm[NTC_MAX_MIPS], hm[NTC_MAX_MIPS];
  int g0w[NTC_MAX_MIPS], g0h[NTC_MAX_MIPS], g1w[NTC_MAX_MIPS], g1h[NTC_MAX_MIPS];
  float sx0[NTC_MAX_MIPS], sy0[NTC_MAX_MIPS], sx1[NTC_MAX_MIPS], sy1[NTC_MAX_MIPS];
  float lodn[NTC_MAX_MIPS];
};

// Input-row layout and shared memory plan (byte offsets).
struct Plan {
  int fast, learned, vq, eo0, eo1, t0, t1, f0, f1, gpe, k_int, cb0, cb1, h3;
  uint32_t w1, w2, w3, wb2, wb3, wh, wbh, cbk, bias, tab, pe, desc, total;
  // `taps_ok`: every grid/mip size ratio puts the taps on the 1/16 lattice and
  // the bin widths are powers of two (fast_layout_ok).
  __host__ __device__ Plan(const ntc_material& M, bool f8, bool taps_ok) {
    const int c0 = M.c0, c1 = M.c1, bits0 = M.bits0, bits1 = M.bits1;
    const bool packed = M.encoding == NTC_GRID_PACKED;
    // learned interpolation of G0 (Sec. 4.3.1): the generic layout with one
    // group range per tap
    learned = M.interp0 != 0;
    const int eb = f8 ? 1 : 2, kstep = f8 ? 32 : 16;
    cb0 = cb1 = 0;
    if (packed) {
      cb0 = cell_bytes(c0, bits0);
      cb1 = cell_bytes(c1, bits1);
    }
    // the fast layout reads whole 32-bit cell words: 4-bit cells of 4 or 8
    // bytes; a vector-quantised G0 (FP16, bilinear, two books of 8 or 16
    // values) joins it with 2-byte index cells and the codebooks in shared
    // memory
    vq = M.vq_books > 0;
    const bool g1_ok = packed && bits1 == 4 && (cb1 == 4 || cb1 == 8);
    if (vq) {
      fast = taps_ok && g1_ok && !f8 && !learned && M.vq_books == 2 && (c0 == 8 || c0 == 16);
    } else {
      fast = taps_ok && g1_ok && bits0 == 4 && (cb0 == 4 || cb0 == 8) && !(f8 && learned);
    }
    eo0 = eo1 = t0 = t1 = 0;
    if (fast) {
      // word 0 holds 5-8 channels; word 1 (8-byte cells) the other c - 8;
      // vector-quantised G0: c0 / 8 groups of channels in order
      eo0 = vq ? c0 / 8 : ((cb0 == 8 && c0 > 12) ? 2 : 1);
      eo1 = (cb1 == 8 && c1 > 12) ? 2 : 1;
      t0 = (!vq && cb0 == 8 && c0 <= 12) ? 1 : 0;
      t1 = (cb1 == 8 && c1 <= 12) ? 1 : 0;
      f0 = f1 = 0;
      // learned interpolation: each G0 tap's words, the tail halves of taps
      // (0,1) and (2,3) sharing a group, G1's tail half alone
      gpe = learned ? 4 * eo0 + 2 * t0 + eo1 + t1 : eo0 + eo1 + ((t0 | t1) ? 1 : 0);
    } else {
      f0 = (learned ? 4 : 1) * ((c0 + 7) / 8);
      f1 = (c1 + 7) / 8;
      gpe = f0 + f1;
    }
    k_int = (8 * (gpe + 2) + kstep - 1) / kstep * kstep;
    uint32_t o = 0;
    w1 = o;   o += kHidden * k_int * eb;          // B: W1 (internal slot order)
    w2 = o;   o += kHidden * kHidden * eb;        // B: W2
    w3 = o;   o += kN3 * kHidden * eb;            // B: W3 (rows >= C zero)
    wb2 = o;  o += f8 ? 0 : kHidden * 16 * 2;     // B: bias block of layer 2 (FP16)
    wb3 = o;  o += f8 ? 0 : kN3 * 16 * 2;         // B: bias block of layer 3 (FP16)
    h3 = !f8 && M.hidden_layers == 3;             // third hidden layer (FP16 forms)
    wh = o;   o += h3 ? kHidden * kHidden * 2 : 0;  // B: Wh
    wbh = o;  o += h3 ? kHidden * 16 * 2 : 0;       // B: its bias block
    cbk = o;  o += (vq && !f8) ? M.vq_books * 256 * c0 * 2 : 0;  // FP16 codebooks
    bias = o; o += (2 * kHidden + kN3) * 4;       // FP32 biases (FP8 epilogues)
    o = (o + 15) / 16 * 16;
    tab = o;  o += sizeof(MipTab);
    pe = o;   o += 8 * 16;                        // per x & 7: half2 (sin, cos) of 3 octaves, 0
    desc = o; o += kDescs * 8;                    // B descriptors: W1 0-7, W2 8-11, b2 12, W3 13-16, b3 17
    total = o;
  }
};

__device__ __forceinline__ uint32_t h2u(__half2 h) {
  union { __half2 h; uint32_t u; } c;
  c.h = h;
  return c.u;
}
__device__ __forceinline__ __half2 u2h(uint32_t u) {
  union { __half2 h; uint32_t u; } c;
  c.u = u;
  return c.h;
}

// User column of internal input slot s: >= 0 a W1 column, -1 zero padding,
// -2 / -3 the constant-one slots carrying the FP16 bias head / tail.
__device__ __forceinline__ int w1_column(const ntc_material& M, const Plan& P, int s, bool f8) {
  int g = s >> 3;
  const int e = s & 7;
  const int j = e >> 1, l = e & 1;  // half2 j of the group, lane l
  if (P.fast && P.learned) {
    const int eo = 2 * (j & 1) + (j >> 1) + 4 * l;
    if (g < 4 * P.eo0) {  // tap g / eo0, word g % eo0
      const int tap = g / P.eo0, ch = 8 * (g - tap * P.eo0) + eo;
      return ch < M.c0 ? tap * M.c0 + ch : -1;
    }
    g -= 4 * P.eo0;
    if (P.t0) {
      if (g < 2) {  // tail halves (lo T, hi T) = channels (8,9) (10,11) of taps 2g, 2g+1
        const int tap = 2 * g + (j >> 1), ch = 8 + 2 * (j & 1) + l;
        return ch < M.c0 ? tap * M.c0 + ch : -1;
      }
      g -= 2;
    }
    const int w0 = 4 * M.c0;
    if (g < P.eo1) return 8 * g + eo < M.c1 ? w0 + 8 * g + eo : -1;
    g -= P.eo1;
    if (P.t1) {
      if (g == 0) {
        const int ch = 8 + 2 * (j & 1) + l;
        return j < 2 && ch < M.c1 ? w0 + ch : -1;
      }
      g -= 1;
    }
  } else if (P.fast) {
    // 5-8 channel word: half2 (lo E, hi E, lo O, hi O) = channels (0,4) (2,6) (1,5) (3,7)
    const int eo = 2 * (j & 1) + (j >> 1) + 4 * l;
    if (g < P.eo0) {  // vector-quantised G0: channels in order
      const int ch = P.vq ? 8 * g + e : 8 * g + eo;
      return ch < M.c0 ? ch : -1;
    }
    g -= P.eo0;
    if (g < P.eo1) return 8 * g + eo < M.c1 ? M.c0 + 8 * g + eo : -1;
    g -= P.eo1;
    if (P.t0 | P.t1) {
      if (g == 0) {
        // tail words: half2 (lo T, hi T) = channels (8,9) (10,11) of G0, then of G1
        const bool both = P.t0 && P.t1;
        if (!both && j >= 2) return -1;
        const int k = both ? (j >> 1) : (P.t0 ? 0 : 1);
        const int ch = 8 + 2 * (j & 1) + l;
        if (k == 0) return ch < M.c0 ? ch : -1;
        return ch < M.c1 ? M.c0 + ch : -1;
      }
      g -= 1;
    }
  } else {
    if (g < P.f0) {
      if (P.learned) {
        // tap t's c0 values in groups [t f0t, (t+1) f0t); user columns t c0 + ch
        const int f0t = (M.c0 + 7) / 8, tap = g / f0t, ch = 8 * (g - tap * f0t) + e;
        return ch < M.c0 ? tap * M.c0 + ch : -1;
      }
      return 8 * g + e < M.c0 ? 8 * g + e : -1;
    }
    g -= P.f0;
    const int w0 = P.learned ? 4 * M.c0 : M.c0;
    if (g < P.f1) return 8 * g + e < M.c1 ? w0 + 8 * g + e : -1;
    g -= P.f1;
  }
  const int pe = (P.learned ? 4 * M.c0 : M.c0) + M.c1;
  if (g == 0) return pe + e;
  if (g == 1) {
    if (e < 4) return pe + 8 + e;
    if (e == 4) return pe + 12;
    if (!f8 && e == 6) return -2;
    if (!f8 && e == 7) return -3;
  }
  return -1;
}

// Split an FP32 bias into an FP16 head and tail: b ~ head + tail.
__device__ __forceinline__ void split_bias(float b, __half& hd, __half& tl) {
  hd = __float2half_rn(b);
  tl = __float2half_rn(b - __half2float(hd));
}

template <bool F8>
__device__ void stage_shared(const ntc_material& M, const Plan& P, uint8_t* sm, int tid, int nt) {
  constexpr int EB = Cfg<F8>::EB;
  for (int i = tid; i < kHidden * P.k_int; i += nt) {
    const int n = i / P.k_int, s = i - n * P.k_int;
    const int col = w1_column(M, P, s, F8);
    const uint32_t off = P.w1 + tc::canon_offset(n, s, kHidden, EB);
    if (F8) {
      sm[off] = col < 0 ? 0 : static_cast<const uint8_t*>(M.w[0])[n * M.k_in + col];
    } else {
      __half hv = __float2half_rn(0.f);
      if (col >= 0) {
        hv = static_cast<const __half*>(M.w[0])[n * M.k_in + col];
      } else if (col < -1) {
        __half hd, tl;
        split_bias(M.b[0][n], hd, tl);
        hv = col == -2 ? hd : tl;
      }
      *reinterpret_cast<__half*>(sm + off) = hv;
    }
  }
  for (int i = tid; i < kHidden * kHidden; i += nt) {
    const int n = i / kHidden, k = i - n * kHidden;
    const uint32_t off = P.w2 + tc::canon_offset(n, k, kHidden, EB);
    if (F8) sm[off] = static_cast<const uint8_t*>(M.w[1])[i];
    else *reinterpret_cast<__half*>(sm + off) = static_cast<const __half*>(M.w[1])[i];
  }
  // sigmoid(z) = (1 + tanh(z / 2)) / 2: layer 3 is staged pre-halved (exact
  // but for FP16 subnormals) so the output epilogue is one tanh and one FMA
  const float h3 = M.out_act == NTC_OUT_IDENTITY ? 1.f : 0.5f;
  for (int i = tid; i < kN3 * kHidden; i += nt) {
    const int n = i / kHidden, k = i - n * kHidden;
    const uint32_t off = P.w3 + tc::canon_offset(n, k, kN3, EB);
    const bool live = n < M.channels;
    if (F8) sm[off] = live ? static_cast<const uint8_t*>(M.w[2])[i] : 0;
    else *reinterpret_cast<__half*>(sm + off) = __float2half_rn(
        live ? h3 * __half2float(static_cast<const __half*>(M.w[2])[i]) : 0.f);
  }
  if (!F8 && P.vq) {  // FP16 codebooks [books][256][c0]
    __half* cb = reinterpret_cast<__half*>(sm + P.cbk);
    for (int i = tid; i < M.vq_books * 256 * M.c0; i += nt) cb[i] = __float2half_rn(M.codebook0[i]);
  }
  if (!F8 && P.h3) {
    for (int i = tid; i < kHidden * kHidden; i += nt) {
      const int n = i / kHidden, k = i - n * kHidden;
      *reinterpret_cast<__half*>(sm + P.wh + tc::canon_offset(n, k, kHidden, 2)) =
          static_cast<const __half*>(M.w_h3)[i];
    }
    for (int i = tid; i < kHidden * 16; i += nt) {
      const int n = i / 16, k = i - n * 16;
      __half hd, tl;
      split_bias(M.b_h3[n], hd, tl);
      *reinterpret_cast<__half*>(sm + P.wbh + tc::canon_offset(n, k, kHidden, 2)) =
          k == 0 ? hd : (k == 1 ? tl : __float2half_rn(0.f));
    }
  }
  float* bias = reinterpret_cast<float*>(sm + P.bias);
  for (int i = tid; i < kHidden; i += nt) {
    bias[i] = M.b[0][i];
    bias[kHidden + i] = M.b[1][i];
  }
  for (int i = tid; i < kN3; i += nt) bias[2 * kHidden + i] = i < M.channels ? h3 * M.b[2][i] : 0.f;
  if (!F8) {
    for (int i = tid; i < kHidden * 16; i += nt) {
      const int n = i / 16, k = i - n * 16;
      __half hd, tl;
      split_bias(M.b[1][n], hd, tl);
      *reinterpret_cast<__half*>(sm + P.wb2 + tc::canon_offset(n, k, kHidden, 2)) =
          k == 0 ? hd : (k == 1 ? tl : __float2half_rn(0.f));
    }
    for (int i = tid; i < kN3 * 16; i += nt) {
      const int n = i / 16, k = i - n * 16;
      __half hd = __float2half_rn(0.f), tl = __float2half_rn(0.f);
      if (n < M.channels) split_bias(h3 * M.b[2][n], hd, tl);
      *reinterpret_cast<__half*>(sm + P.wb3 + tc::canon_offset(n, k, kN3, 2)) =
          k == 0 ? hd : (k == 1 ? tl : __float2half_rn(0.f));
    }
  }
  MipTab* tb = reinterpret_cast<MipTab*>(sm + P.tab);
  for (int m = tid; m < M.mips; m += nt) {
    const int wm = mip_dim(M.width, m), hm = mip_dim(M.height, m);
    const ntc_level& L = M.lv[level_of_mip(m, M.levels)];
    tb->grid0[m] = static_cast<const uint8_t*>(L.grid0);
    tb->grid1[m] = static_cast<const uint8_t*>(L.grid1);
    tb->wm[m] = wm;
    tb->hm[m] = hm;
    tb->g0w[m] = L.g0_w; tb->g0h[m] = L.g0_h; tb->g1w[m] = L.g1_w; tb->g1h[m] = L.g1_h;
    tb->sx0[m] = (float)L.g0_w / (float)wm;
    tb->sy0[m] = (float)L.g0_h / (float)hm;
    tb->sx1[m] = (float)L.g1_w / (float)wm;
    tb->sy1[m] = (float)L.g1_h / (float)hm;
    tb->lodn[m] = M.mips > 1 ? (float)m / (float)(M.mips - 1) : 0.f;
    tb->lodh[m] = tc::pack_f16x2(tb->lodn[m], 0.f);
    tb->tk0[m] = make_int4(8 * L.g0_w / wm, 8 * L.g0_h / hm, L.g0_w, L.g0_h);
    tb->tk1[m] = make_int4(8 * L.g1_w / wm, 8 * L.g1_h / hm, L.g1_w, L.g1_h);
  }
  // positional encoding: per octave h and coordinate c & 7 the (sin, cos)
  // pair, exact in FP16
  struct Pe {
    float v[16];
    __device__ void operator()(int i, float x) { v[i] = x; }
  };
  for (int c = tid; c < 8; c += nt) {
    Pe pe;
    positional_encoding(c, 0, 0, pe);
    reinterpret_cast<uint4*>(sm + P.pe)[c] =
        make_uint4(tc::pack_f16x2(pe.v[0], pe.v[1]), tc::pack_f16x2(pe.v[2], pe.v[3]),
                   tc::pack_f16x2(pe.v[4], pe.v[5]), 0u);
  }
  // shared-memory descriptors of every B operand K-step (K-major, no swizzle:
  // LBO = K-direction core-matrix stride, SBO = 128 between 8-row groups)
  if (tid == 0) {
    constexpr int KS = Cfg<F8>::KSTEP;
    constexpr uint32_t lbo = (kHidden / 8) * 128, lbo3 = (kN3 / 8) * 128;
    uint64_t* d = reinterpret_cast<uint64_t*>(sm + P.desc);
    const uint32_t sb = tc::smem_u32(sm);
    for (int k = 0; k < P.k_int / KS; ++k) d[k] = tc::smem_desc(sb + P.w1 + 2 * k * lbo, lbo, 128);
    for (int k = 0; k < kHidden / KS; ++k) {
      d[kDescW2 + k] = tc::smem_desc(sb + P.w2 + 2 * k * lbo, lbo, 128);
      d[kDescW3 + k] = tc::smem_desc(sb + P.w3 + 2 * k * lbo3, lbo3, 128);
    }
    d[kDescW2 + 4] = tc::smem_desc(sb + P.wb2, lbo, 128);
    d[kDescW3 + 4] = tc::smem_desc(sb + P.wb3, lbo3, 128);
    if (P.h3) {
      for (int k = 0; k < kHidden / KS; ++k) d[kDescWh + k] = tc::smem_desc(sb + P.wh + 2 * k * lbo, lbo, 128);
      d[kDescWh + 4] = tc::smem_desc(sb + P.wbh, lbo, 128);
    }
  }
}

// Where a thread's input row goes: its TMEM lane (A operand read from TMEM;
// an 8-slot group is 4 FP16 / 2 FP8 columns) or its 16-byte chunks of a
// 128-row canonical K-major tile in shared memory (A read through a
// descriptor; chunk stride 16 row groups x 128 bytes along K).
struct TmemRow {
  uint32_t ta;
  __device__ __forceinline__ void put4(int g, uint4 w) const { tc::tmem_st4(ta + 4 * g, w); }
  __device__ __forceinline__ void put2(int g, uint32_t a, uint32_t b) const {
    tc::tmem_st2(ta + 2 * g, a, b);
  }
};
struct SmemRow {
  uint8_t* p;  // this row's chunk of K group 0
  __device__ __forceinline__ void put4(int g, uint4 w) const {
    *reinterpret_cast<uint4*>(p + g * 2048) = w;
  }
  __device__ __forceinline__ void put2(int g, uint32_t a, uint32_t b) const {
    *reinterpret_cast<uint2*>(p + (g >> 1) * 2048 + (g & 1) * 8) = make_uint2(a, b);
  }
};
__device__ __forceinline__ uint8_t* smem_row(uint8_t* tile, int row) {
  return tile + (row >> 3) * 128 + (row & 7) * 16;
}

// One 8-slot group of this thread's row: FP16, or FP8 (scaled by
// `inv_scale` first).
template <bool F8, class S>
__device__ __forceinline__ void put_group(const S& dst, int g, const float (&v)[8], float inv_scale) {
  if (F8) {
    const uint32_t a = tc::pack_e4m3x2(v[0] * inv_scale, v[1] * inv_scale) |
                       (tc::pack_e4m3x2(v[2] * inv_scale, v[3] * inv_scale) << 16);
    const uint32_t b = tc::pack_e4m3x2(v[4] * inv_scale, v[5] * inv_scale) |
                       (tc::pack_e4m3x2(v[6] * inv_scale, v[7] * inv_scale) << 16);
    dst.put2(g, a, b);
  } else {
    uint4 w;
    w.x = tc::pack_f16x2(v[0], v[1]);
    w.y = tc::pack_f16x2(v[2], v[3]);
    w.z = tc::pack_f16x2(v[4], v[5]);
    w.w = tc::pack_f16x2(v[6], v[7]);
    dst.put4(g, w);
  }
}

__device__ __forceinline__ void taps_of(int x, int y, float sx, float sy, int gw, int gh, Taps& t) {
  const float px = ((float)x + 0.5f) * sx - 0.5f;
  const float py = ((float)y + 0.5f) * sy - 0.5f;
  const float fx0 = floorf(px), fy0 = floorf(py);
  const float fx = px - fx0, fy = py - fy0;
  int ix0 = (int)fx0, iy0 = (int)fy0;
  const int ix1 = min(max(ix0 + 1, 0), gw - 1), iy1 = min(max(iy0 + 1, 0), gh - 1);
  ix0 = min(max(ix0, 0), gw - 1);
  iy0 = min(max(iy0, 0), gh - 1);
  t.cell[0] = iy0 * gw + ix0; t.w[0] = (1.f - fx) * (1.f - fy);
  t.cell[1] = iy0 * gw + ix1; t.w[1] = fx * (1.f - fy);
  t.cell[2] = iy1 * gw + ix0; t.w[2] = (1.f - fx) * fy;
  t.cell[3] = iy1 * gw + ix1; t.w[3] = fx * fy;
}

// One row's texel, its tap weights and (fast layout) its gathered cells.
// Filled one tile ahead so the gathers overlap the previous tile's MMAs.
struct Row {
  uint2 c0[4], c1[4];  // cells of the 4 taps of G0 / G1 (at most 8 bytes each)
  int frac;            // tap fractions in 1/16: fx0 | fy0 << 4 | fx1 << 8 | fy1 << 12
  float wtap;          // trilinear blend weight of this row
  int x, y, m;
  int valid;
};

// A query's (u, v, lod), loaded ahead of use.
struct Query {
  float u, v, l;
  int valid;
};
__device__ __forceinline__ Query load_query(const float* __restrict__ uvl, int64_t q, bool valid) {
  Query r{0.f, 0.f, 0.f, valid};
  if (valid) {
    r.u = __ldg(uvl + 3 * q);
    r.v = __ldg(uvl + 3 * q + 1);
    r.l = __ldg(uvl + 3 * q + 2);
  }
  return r;
}

// Query -> texel of this row (nearest and stochastic: one per query;
// trilinear: tap `row & 7` of query `row / 8`).  q: the query's index (the
// stochastic filter's counter), jkey: jitter_key of the frame.
// MM: anything with the material's `mips` (ntc_material, or MipCount for a
// kernel that keeps it in a register).
struct MipCount {
  int mips;
};
template <class MM>
__device__ __forceinline__ void locate(const MM& M, const MipTab* tb, const Query& qu,
                                       int filter, int row, Row& r, int64_t q = 0,
                                       uint64_t jkey = 0) {
  r.valid = qu.valid;
  r.wtap = 0.f;
  r.x = r.y = r.m = 0;
  if (!qu.valid) return;
  const float u = qu.u, v = qu.v, l = qu.l;
  if (filter == NTC_FILTER_NEAREST) {
    const int m = !(l >= 0.f) ? 0 : (l >= (float)(M.mips - 1) ? M.mips - 1 : (int)floorf(l));
    const int wm = tb->wm[m], hm = tb->hm[m];
    const float tu = u * (float)wm, tv = v * (float)hm;
    r.x = !(tu >= 0.f) ? 0 : (tu >= (float)wm ? wm - 1 : (int)floorf(tu));
    r.y = !(tv >= 0.f) ? 0 : (tv >= (float)hm ? hm - 1 : (int)floorf(tv));
    r.m = m;
  } else if (filter == NTC_FILTER_TRILINEAR) {
    const int tap = row & 7, s = tap >> 2, dx = tap & 1, dy = (tap >> 1) & 1;
    const float lam = !(l >= 0.f) ? 0.f : fminf(l, (float)(M.mips - 1));
    const int m0 = min((int)floorf(lam), M.mips - 1);
    const int m1 = min(m0 + 1, M.mips - 1);
    const float t = lam - (float)m0;
    const int m = s ? m1 : m0;
    const float wl = s ? t : 1.f - t;
    const int wm = tb->wm[m], hm = tb->hm[m];
    const float px = u * (float)wm - 0.5f, py = v * (float)hm - 0.5f;
    const float fx0 = floorf(px), fy0 = floorf(py);
    const float fx = px - fx0, fy = py - fy0;
    r.x = (((int)fx0 + dx) % wm + wm) % wm;
    r.y = (((int)fy0 + dy) % hm + hm) % hm;
    r.m = m;
    r.wtap = wl * (dx ? fx : 1.f - fx) * (dy ? fy : 1.f - fy);
  } else {
    const uint64_t h = splitmix64(jkey ^ (uint64_t)q);
    const int m = stochastic_mip(l, M.mips, h);
    r.x = stochastic_coord(u, tb->wm[m], (uint32_t)(h >> 40));
    r.y = stochastic_coord(v, tb->hm[m], (uint32_t)(h >> 16) & 0xFFFFFFu);
    r.m = m;
  }
}

// Fast-layout taps of one grid: with the grid/mip ratio r = G / w_m a
// multiple of 1/8, the tap position p = (x + 1/2) r - 1/2 is exactly
// ((2x+1) 8r - 8) / 16, so its integer part and its fraction (in 1/16) come
// from a shift and a mask.  p lies in [-1/2, G - 1/2): only the lower tap can
// fall below 0 and only the upper one beyond G - 1.
__device__ __forceinline__ void taps16(int x2, int y2, int4 k, int (&cell)[4], int& frac) {
  const int px = x2 * k.x - 8, py = y2 * k.y - 8;
  const int ix = px >> 4, iy = py >> 4;
  frac = (px & 15) | ((py & 15) << 4);
  const int ix0 = max(ix, 0), ix1 = min(ix + 1, k.z - 1);
  const int r0 = max(iy, 0) * k.z, r1 = min(iy + 1, k.w - 1) * k.z;
  cell[0] = r0 + ix0;
  cell[1] = r0 + ix1;
  cell[2] = r1 + ix0;
  cell[3] = r1 + ix1;
}

// Fast-layout class of a material known at compile time: CLS = 1 + 3 k0 + k1
// with grid class k = 0 (one 5-8 channel cell word), 1 (a 5-8 channel word
// and a 1-4 channel tail word) or 2 (two 5-8 channel words).  Kernels that
// take the class at run time pass the Plan, which has the same fields.
// Classes 11..19 are the same grid classes with learned interpolation of G0.
template <int CLS>
struct FastLayout {
  static constexpr int vq = 0;  // vector-quantised G0 runs on the Plan (run-time class)
  static constexpr int base = CLS > 10 ? CLS - 10 : CLS;
  static constexpr int k0 = (base - 1) / 3, k1 = (base - 1) % 3;
  static constexpr int eo0 = k0 == 2 ? 2 : 1, t0 = k0 == 1 ? 1 : 0, cb0 = k0 == 0 ? 4 : 8;
  static constexpr int eo1 = k1 == 2 ? 2 : 1, t1 = k1 == 1 ? 1 : 0, cb1 = k1 == 0 ? 4 : 8;
  static constexpr int learned = CLS > 10 ? 1 : 0;
};

// Issue the eight cell loads of a fast-layout row (invalid rows load nothing).
// VQ: the vector-quantised G0 branch is compiled in.
template <class L, bool VQ = true>
__device__ __forceinline__ void gather_fast(const L& lay, const MipTab* tb, Row& r) {
#pragma unroll
  for (int t = 0; t < 4; ++t) r.c0[t] = r.c1[t] = make_uint2(0, 0);
  r.frac = 0;
  if (!r.valid) return;
  const int m = r.m;
  const int x2 = 2 * r.x + 1, y2 = 2 * r.y + 1;
  int cell0[4], cell1[4], f0, f1;
  taps16(x2, y2, tb->tk0[m], cell0, f0);
  taps16(x2, y2, tb->tk1[m], cell1, f1);
  r.frac = f0 | (f1 << 8);
  const uint8_t* g0 = tb->grid0[m];
  const uint8_t* g1 = tb->grid1[m];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    if (VQ && lay.vq) r.c0[t].x = __ldg(reinterpret_cast<const unsigned short*>(g0) + cell0[t]);
    else if (lay.cb0 == 8) r.c0[t] = __ldg(reinterpret_cast<const uint2*>(g0) + cell0[t]);
    else r.c0[t].x = __ldg(reinterpret_cast<const uint32_t*>(g0) + cell0[t]);
    if (lay.cb1 == 8) r.c1[t] = __ldg(reinterpret_cast<const uint2*>(g1) + cell1[t]);
    else r.c1[t].x = __ldg(reinterpret_cast<const uint32_t*>(g1) + cell1[t]);
  }
}

__device__ __forceinline__ uint32_t word_of(const uint2& c, int f) { return f ? c.y : c.x; }

// y-interpolation constants of one grid: with wy0 = 16 - fy, wy1 = fy and
// s = Q / 256, c0 = wy0 s, c1 = wy1 s and o = -7 Q - 1024 c0 (all exact in
// FP16 for power-of-two Q in [2^-6, 2^6]).
struct YLerp {
  __half2 c0, c1, o;
};
__device__ __forceinline__ YLerp ylerp_of(int fy, __half2 s, __half2 s16, __half2 m7q) {
  YLerp y;
  const __half2 k = u2h((uint32_t)(16 - fy) * 0x10001u + 0x64006400u);  // 1024 + wy0
  y.c0 = __hfma2(k, s, __hmul2(s, __float2half2_rn(-1024.f)));
  y.c1 = __hsub2(s16, y.c0);
  y.o = __hfma2(y.c0, __float2half2_rn(-1024.f), m7q);
  return y;
}

// Lanes (0, 2) / (1, 3) of the x-interpolated rows A0, A1 (16 x the
// x-lerp of q, <= 240) -> dequantised bilinear value (lerp/16 - 7) Q.  The
// byte goes into the mantissa of 1024 + lane; the first FMA cancels the 1024
// exactly, so each output is rounded twice.
__device__ __forceinline__ uint32_t ylerp(uint32_t A0, uint32_t A1, uint32_t sel, const YLerp& y) {
  const uint32_t k = 0x64646464u;
  const __half2 a0 = u2h(__byte_perm(A0, k, sel));
  const __half2 a1 = __hsub2(u2h(__byte_perm(A1, k, sel)), __float2half2_rn(1024.f));
  return h2u(__hfma2(a1, y.c1, __hfma2(a0, y.c0, y.o)));
}

// A 5-8 channel word of the four taps -> one group (channels 0,4,2,6,1,5,3,7).
__device__ __forceinline__ uint4 eo_group(const uint32_t (&w)[4], uint32_t wx0, uint32_t wx1,
                                          const YLerp& y) {
  uint32_t e[4], o[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    e[t] = w[t] & 0x0F0F0F0Fu;
    o[t] = (w[t] >> 4) & 0x0F0F0F0Fu;
  }
  const uint32_t e0 = e[0] * wx0 + e[1] * wx1, e1 = e[2] * wx0 + e[3] * wx1;
  const uint32_t o0 = o[0] * wx0 + o[1] * wx1, o1 = o[2] * wx0 + o[3] * wx1;
  return make_uint4(ylerp(e0, e1, 0x4240u, y), ylerp(e0, e1, 0x4341u, y), ylerp(o0, o1, 0x4240u, y),
                    ylerp(o0, o1, 0x4341u, y));
}

// A 1-4 channel word (low 16 bits) of the four taps -> half a group
// (channels 0,1 and 2,3).
__device__ __forceinline__ uint2 t_half(const uint32_t (&w)[4], uint32_t wx0, uint32_t wx1,
                                        const YLerp& y) {
  uint32_t t4[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) t4[t] = __byte_perm(w[t], w[t] << 12, 0x7610u) & 0x0F0F0F0Fu;
  const uint32_t a0 = t4[0] * wx0 + t4[1] * wx1, a1 = t4[2] * wx0 + t4[3] * wx1;
  return make_uint2(ylerp(a0, a1, 0x4240u, y), ylerp(a0, a1, 0x4341u, y));
}

// The two PE groups (FP16): (sin, cos) pairs of the 3 octaves of x, then of
// y, then (LOD, 0) and the constant-one bias slots.
template <class S>
__device__ __forceinline__ void pe_groups(const Plan& P, const uint8_t* sm, uint32_t lodh, int x,
                                          int y, const S& dst) {
  const uint4* pe = reinterpret_cast<const uint4*>(sm + P.pe);
  const uint4 px = pe[x & 7], py = pe[y & 7];
  dst.put4(P.gpe, make_uint4(px.x, px.y, px.z, py.x));
  dst.put4(P.gpe + 1, make_uint4(py.y, py.z, lodh, tc::pack_f16x2(1.f, 1.f)));
}

// Per-grid FP16 constants of the fast layout.
struct FastK {
  __half2 s[2], s16[2], m7q[2], q[2], o1031[2];
  __device__ FastK(const ntc_material& M) {
    const float qq[2] = {M.q0, M.q1};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      s[k] = __float2half2_rn(qq[k] * (1.f / 256.f));
      s16[k] = __float2half2_rn(qq[k] * (16.f / 256.f));
      m7q[k] = __float2half2_rn(-7.f * qq[k]);
      q[k] = __float2half2_rn(qq[k]);
      o1031[k] = __float2half2_rn(-1031.f * qq[k]);
    }
  }
};

// Fast layout: every group of the row from the prefetched cells.
template <class L, class S, bool VQ = true>
__device__ __forceinline__ void build_fast(const L& lay, const Plan& P, const FastK& K,
                                           const uint8_t* sm, const Row& r, const S& dst) {
  const uint32_t fx0 = r.frac & 15, fx1 = (r.frac >> 8) & 15;
  const YLerp y1 = ylerp_of((r.frac >> 12) & 15, K.s[1], K.s16[1], K.m7q[1]);
  int kg = 0;
  if (lay.learned) {
    // learned interpolation of G0: every tap's channels, dequantised as
    // (1024 + q) Q - 1031 Q = (q - 7) Q in one FMA (exact for power-of-two Q)
    const __half2 q2 = K.q[0], o2 = K.o1031[0];
    const uint32_t kk = 0x64646464u;
    auto dq = [&](uint32_t a, uint32_t sel) { return h2u(__hfma2(u2h(__byte_perm(a, kk, sel)), q2, o2)); };
    uint32_t tl[4][2];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
#pragma unroll
      for (int f = 0; f < 2; ++f)
        if (f < lay.eo0) {
          const uint32_t w = word_of(r.c0[t], f);
          const uint32_t e = w & 0x0F0F0F0Fu, o = (w >> 4) & 0x0F0F0F0Fu;
          dst.put4(kg++, make_uint4(dq(e, 0x4240u), dq(e, 0x4341u), dq(o, 0x4240u), dq(o, 0x4341u)));
        }
      if (lay.t0) {
        const uint32_t tw = __byte_perm(r.c0[t].y, r.c0[t].y << 12, 0x7610u) & 0x0F0F0F0Fu;
        tl[t][0] = dq(tw, 0x4240u);
        tl[t][1] = dq(tw, 0x4341u);
      }
    }
    if (lay.t0) {
      dst.put4(kg++, make_uint4(tl[0][0], tl[0][1], tl[1][0], tl[1][1]));
      dst.put4(kg++, make_uint4(tl[2][0], tl[2][1], tl[3][0], tl[3][1]));
    }
#pragma unroll
    for (int f = 0; f < 2; ++f)
      if (f < lay.eo1) {
        const uint32_t w[4] = {word_of(r.c1[0], f), word_of(r.c1[1], f), word_of(r.c1[2], f),
                               word_of(r.c1[3], f)};
        dst.put4(kg++, eo_group(w, 16 - fx1, fx1, y1));
      }
    if (lay.t1) {
      const uint32_t w[4] = {r.c1[0].y, r.c1[1].y, r.c1[2].y, r.c1[3].y};
      const uint2 b = t_half(w, 16 - fx1, fx1, y1);
      dst.put4(kg++, make_uint4(b.x, b.y, 0u, 0u));
    }
    const MipTab* tb = reinterpret_cast<const MipTab*>(sm + P.tab);
    pe_groups(P, sm, tb->lodh[r.m], r.x, r.y, dst);
    return;
  }
  const YLerp y0 = ylerp_of((r.frac >> 4) & 15, K.s[0], K.s16[0], K.m7q[0]);
  if (VQ && lay.vq) {
    // vector-quantised G0: per tap the sum of its two FP16 codebook entries,
    // blended with the bilinear weights (multiples of 1/256: exact in FP16)
    const uint32_t fy0 = (r.frac >> 4) & 15;
    const __half2 wt[4] = {
        __float2half2_rn((float)((16 - fx0) * (16 - fy0)) * (1.f / 256.f)),
        __float2half2_rn((float)(fx0 * (16 - fy0)) * (1.f / 256.f)),
        __float2half2_rn((float)((16 - fx0) * fy0) * (1.f / 256.f)),
        __float2half2_rn((float)(fx0 * fy0) * (1.f / 256.f))};
    const int c0 = 8 * lay.eo0;
    const uint8_t* cbk = sm + P.cbk;
#pragma unroll
    for (int f = 0; f < 2; ++f)
      if (f < lay.eo0) {
        __half2 acc[4] = {u2h(0u), u2h(0u), u2h(0u), u2h(0u)};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const uint32_t i0 = r.c0[t].x & 0xFFu, i1 = (r.c0[t].x >> 8) & 0xFFu;
          const uint4 a = *reinterpret_cast<const uint4*>(cbk + ((i0 * c0) + 8 * f) * 2);
          const uint4 b = *reinterpret_cast<const uint4*>(cbk + (((256 + i1) * c0) + 8 * f) * 2);
          const uint32_t av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[j] = __hfma2(wt[t], __hadd2(u2h(av[j]), u2h(bv[j])), acc[j]);
        }
        dst.put4(kg++, make_uint4(h2u(acc[0]), h2u(acc[1]), h2u(acc[2]), h2u(acc[3])));
      }
  } else {
#pragma unroll
    for (int f = 0; f < 2; ++f)
      if (f < lay.eo0) {
        const uint32_t w[4] = {word_of(r.c0[0], f), word_of(r.c0[1], f), word_of(r.c0[2], f),
                               word_of(r.c0[3], f)};
        dst.put4(kg++, eo_group(w, 16 - fx0, fx0, y0));
      }
  }
#pragma unroll
  for (int f = 0; f < 2; ++f)
    if (f < lay.eo1) {
      const uint32_t w[4] = {word_of(r.c1[0], f), word_of(r.c1[1], f), word_of(r.c1[2], f),
                             word_of(r.c1[3], f)};
      dst.put4(kg++, eo_group(w, 16 - fx1, fx1, y1));
    }
  if (lay.t0 | lay.t1) {
    uint2 a = make_uint2(0, 0), b = make_uint2(0, 0);
    if (lay.t0) {
      const uint32_t w[4] = {r.c0[0].y, r.c0[1].y, r.c0[2].y, r.c0[3].y};
      a = t_half(w, 16 - fx0, fx0, y0);
    }
    if (lay.t1) {
      const uint32_t w[4] = {r.c1[0].y, r.c1[1].y, r.c1[2].y, r.c1[3].y};
      b = t_half(w, 16 - fx1, fx1, y1);
    }
    if (!lay.t0) { a = b; b = make_uint2(0, 0); }
    dst.put4(kg++, make_uint4(a.x, a.y, b.x, b.y));
  }
  const MipTab* tb = reinterpret_cast<const MipTab*>(sm + P.tab);
  pe_groups(P, sm, tb->lodh[r.m], r.x, r.y, dst);
}

// Zero groups between the PE groups and K (written once per material: the
// per-tile builds never touch them).
template <bool F8, class S>
__device__ __forceinline__ void zero_tail_groups(const Plan& P, const S& dst) {
  const float z[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int g = P.gpe + 2; g < P.k_int / 8; ++g) put_group<F8>(dst, g, z, 1.f);
}

// Generic layout (other bit widths, F32 grids, FP8 operands): float
// dequantisation and interpolation, channels in order.
// VQ: the vector-quantised G0 branch is compiled in (kernels that decode
// such materials).
template <bool F8, class S, bool VQ = true>
__device__ __forceinline__ void generic_grid(const ntc_material& M, const MipTab* tb, int k,
                                             const Plan& P, const Row& r, const S& dst, int kg0,
                                             float inv_sa) {
  const int c = k ? M.c1 : M.c0;
  const float q = k ? M.q1 : M.q0;
  const int m = r.m;
  if (k == 0 && P.learned) {
    // learned interpolation: each tap's dequantised values, unweighted
    const int f0t = (c + 7) / 8;
    Taps t;
    taps_of(r.x, r.y, tb->sx0[m], tb->sy0[m], tb->g0w[m], tb->g0h[m], t);
    const uint8_t* base = tb->grid0[m];
#pragma unroll 1
    for (int tp = 0; tp < 4; ++tp) {
      float acc[kGridPad];
      if (VQ && M.vq_books > 0) {
        const int cell = r.valid ? t.cell[tp] : 0;
#pragma unroll
        for (int ch = 0; ch < kGridPad; ++ch) acc[ch] = 0.f;
        for (int b = 0; b < M.vq_books; ++b) {
          const float* e = M.codebook0 + ((size_t)b * 256 + base[(size_t)cell * M.vq_books + b]) * c;
#pragma unroll
          for (int ch = 0; ch < kMaxGridCh; ++ch)
            if (ch < c) acc[ch] += __ldg(e + ch);
        }
      } else if (M.encoding == NTC_GRID_PACKED) {
        const int off = (1 << (M.bits0 - 1)) - 1;
        const Cell cl = load_cell(base, r.valid ? t.cell[tp] : 0, P.cb0);
#pragma unroll
        for (int ch = 0; ch < kGridPad; ++ch)
          acc[ch] = ch < c ? (float)((int)cell_index(cl, ch, M.bits0) - off) * q : 0.f;
      } else {
        const float* g = reinterpret_cast<const float*>(base) + (size_t)(r.valid ? t.cell[tp] : 0) * c;
#pragma unroll
        for (int ch = 0; ch < kGridPad; ++ch) acc[ch] = ch < c ? __ldg(g + ch) : 0.f;
      }
#pragma unroll
      for (int g2 = 0; g2 < kGridPad / 8; ++g2)
        if (g2 < f0t) {
          float v[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) v[e] = r.valid ? acc[8 * g2 + e] : 0.f;
          put_group<F8>(dst, kg0 + tp * f0t + g2, v, inv_sa);
        }
    }
    return;
  }
  float acc[kGridPad];
#pragma unroll
  for (int ch = 0; ch < kGridPad; ++ch) acc[ch] = 0.f;
  if (r.valid) {
    Taps t;
    if (k) taps_of(r.x, r.y, tb->sx1[m], tb->sy1[m], tb->g1w[m], tb->g1h[m], t);
    else taps_of(r.x, r.y, tb->sx0[m], tb->sy0[m], tb->g0w[m], tb->g0h[m], t);
    const uint8_t* base = k ? tb->grid1[m] : tb->grid0[m];
    if (VQ && k == 0 && M.vq_books > 0) {
      // vector-quantised G0: each tap's cell is the sum of its codebook
      // entries (rows of 4k values read as float4)
#pragma unroll
      for (int tp = 0; tp < 4; ++tp) {
        float v[kMaxGridCh];
#pragma unroll
        for (int ch = 0; ch < kMaxGridCh; ++ch) v[ch] = 0.f;
        for (int b = 0; b < M.vq_books; ++b) {
          const float* e =
              M.codebook0 + ((size_t)b * 256 + base[(size_t)t.cell[tp] * M.vq_books + b]) * c;
          if ((c & 3) == 0) {
#pragma unroll
            for (int q4 = 0; q4 < kMaxGridCh / 4; ++q4)
              if (4 * q4 < c) {
                const float4 f = __ldg(reinterpret_cast<const float4*>(e) + q4);
                v[4 * q4] += f.x; v[4 * q4 + 1] += f.y; v[4 * q4 + 2] += f.z; v[4 * q4 + 3] += f.w;
              }
          } else {
#pragma unroll
            for (int ch = 0; ch < kMaxGridCh; ++ch)
              if (ch < c) v[ch] += __ldg(e + ch);
          }
        }
#pragma unroll
        for (int ch = 0; ch < kMaxGridCh; ++ch)
          if (ch < c) acc[ch] = fmaf(t.w[tp], v[ch], acc[ch]);
      }
    } else if (M.encoding == NTC_GRID_PACKED) {
      const int bits = k ? M.bits1 : M.bits0;
      const int off = (1 << (bits - 1)) - 1;
      const int cb = k ? P.cb1 : P.cb0;
      Cell cl[4];
#pragma unroll
      for (int tp = 0; tp < 4; ++tp) cl[tp] = load_cell(base, t.cell[tp], cb);
#pragma unroll
      for (int tp = 0; tp < 4; ++tp)
#pragma unroll
        for (int ch = 0; ch < kMaxGridCh; ++ch)
          if (ch < c)
            acc[ch] = fmaf(t.w[tp], (float)((int)cell_index(cl[tp], ch, bits) - off) * q, acc[ch]);
    } else {
      const float* fb = reinterpret_cast<const float*>(base);
#pragma unroll
      for (int tp = 0; tp < 4; ++tp) {
        const float* g = fb + (size_t)t.cell[tp] * c;
#pragma unroll
        for (int ch = 0; ch < kMaxGridCh; ++ch)
          if (ch < c) acc[ch] = fmaf(t.w[tp], __ldg(g + ch), acc[ch]);
      }
    }
  }
  const int ng = k ? P.f1 : P.f0;
#pragma unroll
  for (int g = 0; g < kGridPad / 8; ++g)
    if (g < ng) {
      float v[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = acc[8 * g + e];
      put_group<F8>(dst, kg0 + g, v, inv_sa);
    }
}

template <bool F8, class S, bool VQ = true>
__device__ __forceinline__ void build_generic(const ntc_material& M, const Plan& P,
                                              const uint8_t* sm, const Row& r, const S& dst,
                                              float inv_sa) {
  const MipTab* tb = reinterpret_cast<const MipTab*>(sm + P.tab);
  generic_grid<F8, S, VQ>(M, tb, 0, P, r, dst, 0, inv_sa);
  generic_grid<F8, S, VQ>(M, tb, 1, P, r, dst, P.f0, inv_sa);
  if (!F8) {
    pe_groups(P, sm, tb->lodh[r.m], r.x, r.y, dst);
  } else {
    struct Pe {
      float v[16];
      __device__ void operator()(int i, float x) { v[i] = x; }
    } pe;
    positional_encoding(r.x, r.y, 0, pe);
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = pe.v[e];
    put_group<F8>(dst, P.gpe, v, inv_sa);
#pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = pe.v[8 + e];
    v[4] = tb->lodn[r.m];
    v[5] = v[6] = v[7] = 0.f;
    put_group<F8>(dst, P.gpe + 1, v, inv_sa);
  }
}

// Output activation of a texel's 16 accumulators of the pre-halved layer 3:
// sigmoid as (1 + tanh)/2 with paired FP32 FMAs, or identity.
__device__ __forceinline__ void out_activate(float (&yv)[16], int out_act) {
  if (out_act == NTC_OUT_IDENTITY) return;
#pragma unroll
  for (int c = 0; c < 16; c += 2) {
    const float2 t = __ffma2_rn(make_float2(tc::tanh_fast(yv[c]), tc::tanh_fast(yv[c + 1])),
                                make_float2(0.5f, 0.5f), make_float2(0.5f, 0.5f));
    yv[c] = t.x;
    yv[c + 1] = t.y;
  }
}

// 8-bit UNORM of four outputs, packed low byte first: rn(sat(y) 255).
__device__ __forceinline__ uint32_t unorm8x4(float a, float b, float c, float d) {
  return __float2uint_rn(__saturatef(a) * 255.f) | (__float2uint_rn(__saturatef(b) * 255.f) << 8) |
         (__float2uint_rn(__saturatef(c) * 255.f) << 16) |
         (__float2uint_rn(__saturatef(d) * 255.f) << 24);
}

// One texel's C outputs (FP16, FP32 or 8-bit UNORM) at output row q.
__device__ __forceinline__ void store_texel(void* out, int out_dtype, int64_t q, int C,
                                            const float (&yv)[16]) {
  if (out_dtype == NTC_DTYPE_U8) {
    uint8_t* o = static_cast<uint8_t*>(out) + q * C;
    uint32_t w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) w[j] = unorm8x4(yv[4 * j], yv[4 * j + 1], yv[4 * j + 2], yv[4 * j + 3]);
    if (C == 16) {
      *reinterpret_cast<uint4*>(o) = make_uint4(w[0], w[1], w[2], w[3]);
    } else if ((C & 3) == 0) {
#pragma unroll
      for (int c = 0; c < 16; c += 4)
        if (c < C) *reinterpret_cast<uint32_t*>(o + c) = w[c >> 2];
    } else {
#pragma unroll
      for (int c = 0; c < 16; ++c)
        if (c < C) o[c] = (uint8_t)(w[c >> 2] >> (8 * (c & 3)));
    }
  } else if (out_dtype == NTC_DTYPE_F16) {
    __half* o = static_cast<__half*>(out) + q * C;
    if (C == 16) {
      uint4 a, b;
      a.x = tc::pack_f16x2(yv[0], yv[1]); a.y = tc::pack_f16x2(yv[2], yv[3]);
      a.z = tc::pack_f16x2(yv[4], yv[5]); a.w = tc::pack_f16x2(yv[6], yv[7]);
      b.x = tc::pack_f16x2(yv[8], yv[9]); b.y = tc::pack_f16x2(yv[10], yv[11]);
      b.z = tc::pack_f16x2(yv[12], yv[13]); b.w = tc::pack_f16x2(yv[14], yv[15]);
      reinterpret_cast<uint4*>(o)[0] = a;
      reinterpret_cast<uint4*>(o)[1] = b;
    } else if ((C & 3) == 0) {
#pragma unroll
      for (int c = 0; c < 16; c += 4)
        if (c < C)
          *reinterpret_cast<uint2*>(o + c) =
              make_uint2(tc::pack_f16x2(yv[c], yv[c + 1]), tc::pack_f16x2(yv[c + 2], yv[c + 3]));
    } else {
#pragma unroll
      for (int c = 0; c < 16; ++c)
        if (c < C) o[c] = __float2half_rn(yv[c]);
    }
  } else {
    float* o = static_cast<float*>(out) + q * C;
    if ((C & 3) == 0) {
#pragma unroll
      for (int c = 0; c < 16; c += 4)
        if (c < C) *reinterpret_cast<float4*>(o + c) = make_float4(yv[c], yv[c + 1], yv[c + 2], yv[c + 3]);
    } else {
#pragma unroll
      for (int c = 0; c < 16; ++c)
        if (c < C) o[c] = yv[c];
    }
  }
}

// hardGELU (Sec. 4.4) as z * clamp(z/3 + 1/2, 0, 1): one saturating FMA and
// one multiply, the same function as its three-piece definition.
__device__ __forceinline__ float hardgelu_sat(float z) {
  return z * __saturatef(fmaf(z, 1.f / 3.f, 0.5f));
}

// FP16 hidden-layer epilogue in quarters of 16 accumulators (a smaller
// register footprint, for the warp-specialised kernel's compute warps).
__device__ __forceinline__ void hidden_epilogue_q(uint32_t td, uint32_t ta, int act) {
#pragma unroll
  for (int qtr = 0; qtr < 4; ++qtr) {
    float a[16];
    tc::tmem_ld16(td + 16 * qtr, a);
    tc::tmem_ld_wait();
    uint32_t w[8];
    if (act == NTC_ACT_RELU) {
#pragma unroll
      for (int i = 0; i < 8; ++i) w[i] = tc::pack_f16x2_relu(a[2 * i], a[2 * i + 1]);
    } else {
#pragma unroll
      for (int i = 0; i < 8; ++i) w[i] = tc::pack_f16x2(hardgelu_sat(a[2 * i]), hardgelu_sat(a[2 * i + 1]));
    }
    tc::tmem_st8(ta + 8 * qtr, w);
  }
}

// Hidden-layer epilogue: D row (TMEM) -> activation -> A row (TMEM).
// FP8: (s_w s_a) acc + b, activation, scale by 1/s_a(next), E4M3.
template <bool F8>
__device__ __forceinline__ void hidden_epilogue(uint32_t td, uint32_t ta, int act,
                                                const float* bias, float scale, float inv_next) {
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    float a[16], b[16];
    tc::tmem_ld16(td + 32 * half, a);
    tc::tmem_ld16(td + 32 * half + 16, b);
    tc::tmem_ld_wait();
    float v[32];
#pragma unroll
    for (int i = 0; i < 16; ++i) { v[i] = a[i]; v[16 + i] = b[i]; }
    if (F8) {
      uint32_t w[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        float e[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
          e[j] = act_fwd(act, fmaf(v[4 * i + j], scale, bias[32 * half + 4 * i + j])) * inv_next;
        w[i] = tc::pack_e4m3x2(e[0], e[1]) | (tc::pack_e4m3x2(e[2], e[3]) << 16);
      }
      tc::tmem_st4(ta + 8 * half, make_uint4(w[0], w[1], w[2], w[3]));
      tc::tmem_st4(ta + 8 * half + 4, make_uint4(w[4], w[5], w[6], w[7]));
    } else {
      uint32_t w[16];
      if (act == NTC_ACT_RELU) {
#pragma unroll
        for (int i = 0; i < 16; ++i) w[i] = tc::pack_f16x2_relu(v[2 * i], v[2 * i + 1]);
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i)
          w[i] = tc::pack_f16x2(hardgelu_sat(v[2 * i]), hardgelu_sat(v[2 * i + 1]));
      }
      tc::tmem_st16(ta + 16 * half, w);
    }
  }
}

// Issue one layer: D (+)= A[tmem] B[smem]^T over `ksteps` K-steps of W
// (descriptors desc[0..ksteps)), then (FP16, `bias`) the bias step desc[ksteps]
// against the constant-one A block, then commit.  Layers are issued by lane 0
// of warps 0, 1, 2 of the warpgroup, spreading the issue work.
template <bool F8>
__device__ __forceinline__ void issue_layer(uint32_t tmem_d, uint32_t tmem_a, const uint64_t* desc,
                                            int ksteps, uint32_t id, bool bias, uint32_t tmem_cst,
                                            uint64_t* bar) {
  tc::fence_after_sync();
  for (int s = 0; s < ksteps; ++s) {
    if (F8) tc::mma_f8_ta(tmem_d, tmem_a + 8 * s, desc[s], id, s > 0);
    else tc::mma_f16_ta(tmem_d, tmem_a + 8 * s, desc[s], id, s > 0);
  }
  if (!F8 && bias) tc::mma_f16_ta(tmem_d, tmem_cst, desc[ksteps], id, 1);
  tc::mma_commit(bar);
}

}  // namespace
}  // namespace ntc
