// Tensor-core (tcgen05) random-access decode, FP16 or FP8-E4M3 operands with
// FP32 accumulation (Sec. 4.3-4.4, 5.2-5.3).
//
// One persistent CTA per SM runs 2-4 independent warpgroup pipelines that
// share one copy of the weights (the B operands, in shared memory).  A
// warpgroup owns a stream of tiles of 128 MLP rows (one query per row, or
// for trilinear filtering 16 queries x 8 texel taps), one mbarrier and 128
// TMEM columns: 64 for the FP32 accumulator D and the rest for the A operand.
// Activations never touch shared memory: thread r owns row r = TMEM lane r,
// writes its input row and its hidden rows into the A columns with
// tcgen05.st, and tcgen05.mma reads A from TMEM.  Per tile:
//   1. every thread gathers the 8 cells of its texel (4 bilinear taps x 2
//      grids; fetched one tile ahead), dequantises, interpolates, appends the
//      positional encoding and the LOD and stores the row into A;
//   2. one thread issues layer 1 (M=128, N=64) and commits to the mbarrier;
//      the warpgroup fetches the next tile's cells, waits, loads D with
//      tcgen05.ld, applies the activation and stores the hidden row into A;
//   3. likewise layer 2 (N=64) and layer 3 (N=16), whose epilogue applies the
//      output activation and stores the texel to global memory.
//
// Input-slot order (W1's columns permuted to match when staged), 8 slots per
// group.  Fast layout (4-bit packed grids, FP16, tap fractions on a 1/16
// lattice): a cell word of 5-8 channels is split into its even and odd
// nibbles (4 byte lanes each), both rows of taps are interpolated along x in
// integer byte-lane arithmetic (16 q_0 + f (q_1 - q_0) <= 240, exact), and
// each pair of lanes is put into the mantissa of the half 1024 + lane and
// interpolated along y with two half FMAs: slots hold channels
// 0,4,2,6,1,5,3,7.  Words of 1-4 channels (the tail of a 9-12 channel cell)
// hold channels 0,1,2,3 in half a group; the tails of G0 and G1 share one
// group.  Generic layout: channels in order.
// Then [PE0..7][PE8..11, LOD, 0, 1, 1].  For FP16 the biases ride on the
// tensor core: layer 1 through the two constant-one slots (bias split into
// an FP16 head and tail), layers 2 and 3 through one extra K=16 step against
// a constant-one A block kept in TMEM.  FP8: each epilogue applies
// (s_w * s_a) * acc + b in FP32.
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
  int fast, eo0, eo1, t0, t1, f0, f1, gpe, k_int, cb0, cb1;
  uint32_t w1, w2, w3, wb2, wb3, bias, tab, pe, desc, total;
  // `taps_ok`: every grid/mip size ratio puts the taps on the 1/16 lattice and
  // the bin widths are powers of two (fast_layout_ok).
  __host__ __device__ Plan(int c0, int c1, int bits0, int bits1, bool packed, bool f8,
                           bool taps_ok) {
    const int eb = f8 ? 1 : 2, kstep = f8 ? 32 : 16;
    cb0 = cb1 = 0;
    if (packed) {
      cb0 = cell_bytes(c0, bits0);
      cb1 = cell_bytes(c1, bits1);
    }
    // the fast layout reads whole 32-bit cell words: 4-bit cells of 4 or 8 bytes
    fast = taps_ok && !f8 && packed && bits0 == 4 && bits1 == 4 && (cb0 == 4 || cb0 == 8) &&
           (cb1 == 4 || cb1 == 8);
    eo0 = eo1 = t0 = t1 = 0;
    if (fast) {
      // word 0 holds 5-8 channels; word 1 (8-byte cells) the other c - 8
      eo0 = (cb0 == 8 && c0 > 12) ? 2 : 1;
      eo1 = (cb1 == 8 && c1 > 12) ? 2 : 1;
      t0 = (cb0 == 8 && c0 <= 12) ? 1 : 0;
      t1 = (cb1 == 8 && c1 <= 12) ? 1 : 0;
      f0 = f1 = 0;
      gpe = eo0 + eo1 + ((t0 | t1) ? 1 : 0);
    } else {
      f0 = (c0 + 7) / 8;
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
    bias = o; o += (2 * kHidden + kN3) * 4;       // FP32 biases (FP8 epilogues)
    o = (o + 15) / 16 * 16;
    tab = o;  o += sizeof(MipTab);
    pe = o;   o += 8 * 16;                        // per x & 7: half2 (sin, cos) of 3 octaves, 0
    desc = o; o += 16 * 8;                        // B descriptors: W1 0-3, W2 4-7, b2 8, W3 9-12, b3 13
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
  if (P.fast) {
    // 5-8 channel word: half2 (lo E, hi E, lo O, hi O) = channels (0,4) (2,6) (1,5) (3,7)
    const int eo = 2 * (j & 1) + (j >> 1) + 4 * l;
    if (g < P.eo0) return 8 * g + eo < M.c0 ? 8 * g + eo : -1;
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
    if (g < P.f0) return 8 * g + e < M.c0 ? 8 * g + e : -1;
    g -= P.f0;
    if (g < P.f1) return 8 * g + e < M.c1 ? M.c0 + 8 * g + e : -1;
    g -= P.f1;
  }
  const int pe = M.c0 + M.c1;
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
      d[4 + k] = tc::smem_desc(sb + P.w2 + 2 * k * lbo, lbo, 128);
      d[9 + k] = tc::smem_desc(sb + P.w3 + 2 * k * lbo3, lbo3, 128);
    }
    d[8] = tc::smem_desc(sb + P.wb2, lbo, 128);
    d[13] = tc::smem_desc(sb + P.wb3, lbo3, 128);
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

// Query -> texel of this row (nearest: one per query; trilinear: tap `row & 7`
// of query `row / 8`).
__device__ __forceinline__ void locate(const ntc_material& M, const MipTab* tb, const Query& qu,
                                       bool tri, int row, Row& r) {
  r.valid = qu.valid;
  r.wtap = 0.f;
  r.x = r.y = r.m = 0;
  if (!qu.valid) return;
  const float u = qu.u, v = qu.v, l = qu.l;
  if (!tri) {
    const int m = !(l >= 0.f) ? 0 : (l >= (float)(M.mips - 1) ? M.mips - 1 : (int)floorf(l));
    const int wm = tb->wm[m], hm = tb->hm[m];
    const float tu = u * (float)wm, tv = v * (float)hm;
    r.x = !(tu >= 0.f) ? 0 : (tu >= (float)wm ? wm - 1 : (int)floorf(tu));
    r.y = !(tv >= 0.f) ? 0 : (tv >= (float)hm ? hm - 1 : (int)floorf(tv));
    r.m = m;
  } else {
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

// Issue the eight cell loads of a fast-layout row (invalid rows load nothing).
__device__ __forceinline__ void gather_fast(const MipTab* tb, const Plan& P, Row& r) {
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
    if (P.cb0 == 8) r.c0[t] = __ldg(reinterpret_cast<const uint2*>(g0) + cell0[t]);
    else r.c0[t].x = __ldg(reinterpret_cast<const uint32_t*>(g0) + cell0[t]);
    if (P.cb1 == 8) r.c1[t] = __ldg(reinterpret_cast<const uint2*>(g1) + cell1[t]);
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
  __half2 s[2], s16[2], m7q[2];
  __device__ FastK(const ntc_material& M) {
    const float q[2] = {M.q0, M.q1};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      s[k] = __float2half2_rn(q[k] * (1.f / 256.f));
      s16[k] = __float2half2_rn(q[k] * (16.f / 256.f));
      m7q[k] = __float2half2_rn(-7.f * q[k]);
    }
  }
};

// Fast layout: every group of the row from the prefetched cells.
template <class S>
__device__ __forceinline__ void build_fast(const Plan& P, const FastK& K, const uint8_t* sm,
                                           const Row& r, const S& dst) {
  const uint32_t fx0 = r.frac & 15, fx1 = (r.frac >> 8) & 15;
  const YLerp y0 = ylerp_of((r.frac >> 4) & 15, K.s[0], K.s16[0], K.m7q[0]);
  const YLerp y1 = ylerp_of((r.frac >> 12) & 15, K.s[1], K.s16[1], K.m7q[1]);
  int kg = 0;
#pragma unroll
  for (int f = 0; f < 2; ++f)
    if (f < P.eo0) {
      const uint32_t w[4] = {word_of(r.c0[0], f), word_of(r.c0[1], f), word_of(r.c0[2], f),
                             word_of(r.c0[3], f)};
      dst.put4(kg++, eo_group(w, 16 - fx0, fx0, y0));
    }
#pragma unroll
  for (int f = 0; f < 2; ++f)
    if (f < P.eo1) {
      const uint32_t w[4] = {word_of(r.c1[0], f), word_of(r.c1[1], f), word_of(r.c1[2], f),
                             word_of(r.c1[3], f)};
      dst.put4(kg++, eo_group(w, 16 - fx1, fx1, y1));
    }
  if (P.t0 | P.t1) {
    uint2 a = make_uint2(0, 0), b = make_uint2(0, 0);
    if (P.t0) {
      const uint32_t w[4] = {r.c0[0].y, r.c0[1].y, r.c0[2].y, r.c0[3].y};
      a = t_half(w, 16 - fx0, fx0, y0);
    }
    if (P.t1) {
      const uint32_t w[4] = {r.c1[0].y, r.c1[1].y, r.c1[2].y, r.c1[3].y};
      b = t_half(w, 16 - fx1, fx1, y1);
    }
    if (!P.t0) { a = b; b = make_uint2(0, 0); }
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
template <bool F8, class S>
__device__ __forceinline__ void generic_grid(const ntc_material& M, const MipTab* tb, int k,
                                             const Plan& P, const Row& r, const S& dst, int kg0,
                                             float inv_sa) {
  const int c = k ? M.c1 : M.c0;
  const float q = k ? M.q1 : M.q0;
  const int m = r.m;
  float acc[kMaxGridCh];
#pragma unroll
  for (int ch = 0; ch < kMaxGridCh; ++ch) acc[ch] = 0.f;
  if (r.valid) {
    Taps t;
    if (k) taps_of(r.x, r.y, tb->sx1[m], tb->sy1[m], tb->g1w[m], tb->g1h[m], t);
    else taps_of(r.x, r.y, tb->sx0[m], tb->sy0[m], tb->g0w[m], tb->g0h[m], t);
    const uint8_t* base = k ? tb->grid1[m] : tb->grid0[m];
    if (M.encoding == NTC_GRID_PACKED) {
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
  for (int g = 0; g < 2; ++g)
    if (g < ng) {
      float v[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = acc[8 * g + e];
      put_group<F8>(dst, kg0 + g, v, inv_sa);
    }
}

template <bool F8, class S>
__device__ __forceinline__ void build_generic(const ntc_material& M, const Plan& P,
                                              const uint8_t* sm, const Row& r, const S& dst,
                                              float inv_sa) {
  const MipTab* tb = reinterpret_cast<const MipTab*>(sm + P.tab);
  generic_grid<F8>(M, tb, 0, P, r, dst, 0, inv_sa);
  generic_grid<F8>(M, tb, 1, P, r, dst, P.f0, inv_sa);
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

// One texel's C outputs (FP16 or FP32) at output row q.
__device__ __forceinline__ void store_texel(void* out, int out_dtype, int64_t q, int C,
                                            const float (&yv)[16]) {
  if (out_dtype == NTC_DTYPE_F16) {
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
      for (int i = 0; i < 8; ++i) w[i] = tc::pack_f16x2(act_fwd(act, a[2 * i]), act_fwd(act, a[2 * i + 1]));
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
          w[i] = tc::pack_f16x2(act_fwd(act, v[2 * i]), act_fwd(act, v[2 * i + 1]));
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

template <bool F8, bool FAST, int kNWG>
__global__ void __launch_bounds__(kRows* kNWG, 1) decode_tc_kernel(
    const ntc_material M, const float* __restrict__ uvl, int64_t n, void* __restrict__ out,
    int out_dtype, int filter, int* status) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ uint64_t mbar[kNWG];
  __shared__ uint32_t tmem_base;
  __shared__ int wg_abort[kNWG];
  constexpr int KSTEP = Cfg<F8>::KSTEP;
  constexpr uint32_t kCols = kNWG <= 2 ? 256 : 512;  // 128 columns per warpgroup
  const Plan P(M.c0, M.c1, M.bits0, M.bits1, M.encoding == NTC_GRID_PACKED, F8, FAST);
  uint8_t* sm = smem_raw;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int wg = tid / kRows, row = tid % kRows;
  const int bar_id = 1 + wg;

  stage_shared<F8>(M, P, sm, threadIdx.x, blockDim.x);
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, kCols);
    tc::tmem_relinquish();
  }
  if (tid < kNWG) {
    tc::mbar_init(&mbar[tid], 1);
    wg_abort[tid] = 0;
  }
  tc::fence_mbar_init();
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  // this warpgroup's 128 columns; per-thread addresses carry the warp's lane quarter
  const uint32_t tw = tmem_base + 128u * wg;
  const uint32_t lane = (uint32_t)((warp & 3) * 32) << 16;
  const uint32_t td = tw + lane, th = tw + kColH + lane, tx = tw + kColX + lane;
  uint64_t* bar = &mbar[wg];
  volatile int* abort_flag = &wg_abort[wg];
  if (!F8) {
    // constant-one A block (bias steps of layers 2 and 3): k = 0, 1 are one
    tc::tmem_st4(tw + kColCst + lane, make_uint4(tc::pack_f16x2(1.f, 1.f), 0, 0, 0));
    tc::tmem_st4(tw + kColCst + 4 + lane, make_uint4(0, 0, 0, 0));
  }
  zero_tail_groups<F8>(P, TmemRow{tx});

  float sc[3] = {1.f, 1.f, 1.f}, inv_sa[3] = {1.f, 1.f, 1.f};
  if (F8) {
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      sc[l] = M.scale[l] * M.scale[3 + l];
      inv_sa[l] = 1.f / M.scale[3 + l];
    }
    if (M.out_act != NTC_OUT_IDENTITY) sc[2] *= 0.5f;  // layer 3 pre-halved (tanh form)
  }
  const FastK K(M);
  const float* bias = reinterpret_cast<const float*>(sm + P.bias);
  const MipTab* tb = reinterpret_cast<const MipTab*>(sm + P.tab);
  const uint64_t* dsc = reinterpret_cast<const uint64_t*>(sm + P.desc);
  constexpr uint32_t id64 = tc::idesc(kRows, kHidden), id16 = tc::idesc(kRows, kN3);

  const bool tri = filter == NTC_FILTER_TRILINEAR;
  const int per_tile = tri ? kRows / 8 : kRows;
  const int64_t ntiles = (n + per_tile - 1) / per_tile;
  const int64_t stride = (int64_t)gridDim.x * kNWG;
  auto qindex = [&](int64_t t) { return tri ? t * per_tile + (row >> 3) : t * per_tile + row; };
  uint32_t phase = 0;
  const int C = M.channels;
  bool aborted = false;

  // Prologue: the first tile's input rows, and the next tile's query.
  int64_t tl = (int64_t)blockIdx.x * kNWG + wg;
  int cur_valid;
  float cur_wtap;
  Query nq;
  {
    const int64_t q0 = qindex(tl);
    Row r;
    locate(M, tb, load_query(uvl, q0, tl < ntiles && q0 < n), tri, row, r);
    if (FAST) {
      gather_fast(tb, P, r);
      build_fast(P, K, sm, r, TmemRow{tx});
    } else {
      build_generic<F8>(M, P, sm, r, TmemRow{tx}, inv_sa[0]);
    }
    cur_valid = r.valid;
    cur_wtap = r.wtap;
    const int64_t q1 = qindex(tl + stride);
    nq = load_query(uvl, q1, tl + stride < ntiles && q1 < n);
    tc::tmem_st_wait();
    tc::fence_before_sync();
    tc::bar_sync(bar_id, kRows);
  }

  for (; tl < ntiles; tl += stride) {
    const int64_t q = qindex(tl);
    const bool valid = cur_valid != 0;
    const float wtap = cur_wtap;

    // ---- layer 1 (X of this tile is in TMEM) ---------------------------------
    if (row == 0) issue_layer<F8>(tw, tw + kColX, dsc, P.k_int / KSTEP, id64, false, 0, bar);
    // next tile: texel and cell gathers now, its query two tiles ahead
    Row nxt;
    locate(M, tb, nq, tri, row, nxt);
    if (FAST) gather_fast(tb, P, nxt);
    {
      const int64_t t2 = tl + 2 * stride;
      const int64_t q2 = qindex(t2);
      nq = load_query(uvl, q2, t2 < ntiles && q2 < n);
    }
    if (!tc::mbar_wait(bar, phase, kWaitLimit)) *abort_flag = 1;
    phase ^= 1;
    tc::fence_after_sync();
    hidden_epilogue<F8>(td, th, M.act, bias, sc[0], inv_sa[1]);
    tc::tmem_st_wait();
    tc::fence_before_sync();
    tc::bar_sync(bar_id, kRows);

    // ---- layer 2; meanwhile the next tile's X (layer 1 is done with X) -------
    if (row == 32) issue_layer<F8>(tw, tw + kColH, dsc + 4, kHidden / KSTEP, id64, !F8, tw + kColCst, bar);
    if (FAST) build_fast(P, K, sm, nxt, TmemRow{tx});
    else build_generic<F8>(M, P, sm, nxt, TmemRow{tx}, inv_sa[0]);
    cur_valid = nxt.valid;
    cur_wtap = nxt.wtap;
    if (!tc::mbar_wait(bar, phase, kWaitLimit)) *abort_flag = 1;
    phase ^= 1;
    tc::fence_after_sync();
    hidden_epilogue<F8>(td, th, M.act, bias + kHidden, sc[1], inv_sa[2]);
    tc::tmem_st_wait();
    tc::fence_before_sync();
    tc::bar_sync(bar_id, kRows);
    if (*abort_flag) { aborted = true; break; }

    // ---- layer 3 + output ----------------------------------------------
    if (row == 64) issue_layer<F8>(tw, tw + kColH, dsc + 9, kHidden / KSTEP, id16, !F8, tw + kColCst, bar);
    if (!tc::mbar_wait(bar, phase, kWaitLimit)) *abort_flag = 1;
    phase ^= 1;
    tc::fence_after_sync();
    float yv[16];
    tc::tmem_ld16(td, yv);
    tc::tmem_ld_wait();
    tc::fence_before_sync();
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      float z = yv[c];
      if (F8) z = fmaf(z, sc[2], bias[2 * kHidden + c]);
      yv[c] = M.out_act == NTC_OUT_IDENTITY ? z : fmaf(0.5f, tc::tanh_fast(z), 0.5f);
    }
    if (tri) {
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        float s = yv[c] * wtap;
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        s += __shfl_xor_sync(0xffffffffu, s, 2);
        s += __shfl_xor_sync(0xffffffffu, s, 4);
        yv[c] = s;
      }
    }
    if (valid && (!tri || (row & 7) == 0)) store_texel(out, out_dtype, q, C, yv);
    // the next tile's layer 1 overwrites D: every row must have read it
    tc::bar_sync(bar_id, kRows);
    if (*abort_flag) { aborted = true; break; }
  }

  tc::fence_before_sync();
  __syncthreads();
  if (tid == 0) {
    int any = 0;
    for (int w = 0; w < kNWG; ++w) any |= wg_abort[w];
    if (any || aborted) atomicExch(status, NTC_ERR_TIMEOUT);
  }
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem_base, kCols);
  }
}

// ---------------------------------------------------------------------------
// Warp-specialised form (FP16): four compute warpgroups, each running its own
// stream of tiles, and one issuer warpgroup whose warp w issues every
// tcgen05.mma chain of compute warpgroup w.  A chain of dependent MMAs holds
// its issuing thread until it drains, so issuing from the compute warps
// stalls them; here they only hand over through mbarriers and keep working:
//   X(i) in shared memory --x--> L1 --d--> epilogue 1 -> H --h--> L2 --d-->
//   epilogue 2 -> H --h--> L3 (own accumulator D3) --o--> output,
// and while L2(i) runs the compute warps build X(i+1), while L3(i) runs they
// gather the cells of tile i+2, while L1(i+1) runs they write tile i.  L1
// reads its A operand from shared memory, the bias steps a constant-one A
// block in shared memory; L2 and L3 read H from TMEM.
// TMEM per compute warpgroup (128 columns): D [0, 64), H [64, 96),
// D3 [96, 112).
// ---------------------------------------------------------------------------
constexpr int kWsCompute = 4;
constexpr int kWsThreads = kRows * (kWsCompute + 1);
constexpr int kColD3 = 96;

struct WsPlan {
  uint32_t cst, x, xbytes, total;
  __host__ __device__ explicit WsPlan(const Plan& P) {
    uint32_t o = (P.total + 1023) / 1024 * 1024;
    cst = o;  o += kRows * 16 * 2;                 // constant-one A block (K = 16)
    xbytes = kRows * P.k_int * 2;
    x = o;    o += kWsCompute * xbytes;            // one X tile per compute warpgroup
    total = o;
  }
};

template <bool FAST>
__global__ void __launch_bounds__(kWsThreads, 1) decode_ws_kernel(
    const ntc_material M, const float* __restrict__ uvl, int64_t n, void* __restrict__ out,
    int out_dtype, int filter, int* status) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ uint64_t bar_x[kWsCompute], bar_h[kWsCompute], bar_d[kWsCompute],
      bar_o[kWsCompute], bar_fin[kWsCompute];
  __shared__ uint32_t tmem_base;
  __shared__ int wg_abort[kWsCompute];
  const Plan P(M.c0, M.c1, M.bits0, M.bits1, M.encoding == NTC_GRID_PACKED, false, FAST);
  const WsPlan W(P);
  uint8_t* sm = smem_raw;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wg = warp >> 2, row = tid & (kRows - 1);

  stage_shared<false>(M, P, sm, tid, blockDim.x);
  // constant-one A block: every row (1, 1, 0, ..., 0)
  for (int i = tid; i < kRows * 16 / 2; i += blockDim.x) {
    const int chunk = i >> 2, e = i & 3;
    reinterpret_cast<uint32_t*>(sm + W.cst)[i] =
        (chunk < kRows && e == 0) ? tc::pack_f16x2(1.f, 1.f) : 0u;
  }
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, 512);
    tc::tmem_relinquish();
  }
  if (tid < kWsCompute) {
    tc::mbar_init(&bar_x[tid], 4);
    tc::mbar_init(&bar_h[tid], 4);
    tc::mbar_init(&bar_d[tid], 1);
    tc::mbar_init(&bar_o[tid], 1);
    tc::mbar_init(&bar_fin[tid], 1);
    wg_abort[tid] = 0;
  }
  if (wg < kWsCompute) zero_tail_groups<false>(P, SmemRow{smem_row(sm + W.x + wg * W.xbytes, row)});
  tc::fence_mbar_init();
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();

  const bool tri = filter == NTC_FILTER_TRILINEAR;
  const int per_tile = tri ? kRows / 8 : kRows;
  const int64_t ntiles = (n + per_tile - 1) / per_tile;
  const int64_t stride = (int64_t)gridDim.x * kWsCompute;
  constexpr uint32_t id64 = tc::idesc(kRows, kHidden), id16 = tc::idesc(kRows, kN3);
  const int w = wg < kWsCompute ? wg : (warp & 3);  // the compute warpgroup served
  const int64_t first = (int64_t)blockIdx.x * kWsCompute + w;
  const uint32_t tw = tmem_base + 128u * w;

  if (wg == kWsCompute) {
    // ---- issuer warp w ------------------------------------------------------
    if (lane == 0) {
      const uint64_t* d = reinterpret_cast<const uint64_t*>(sm + P.desc);
      const uint32_t xa = tc::smem_u32(sm + W.x + w * W.xbytes);
      const uint64_t cst = tc::smem_desc(tc::smem_u32(sm + W.cst), 2048, 128);
      const int k1 = P.k_int / 16;
      uint32_t px = 0, ph = 0;
      bool ok = true;
      for (int64_t tl = first; tl < ntiles; tl += stride) {
        if (!(ok = tc::mbar_wait(&bar_x[w], px, kWaitLimit))) break;
        px ^= 1;
        tc::fence_after_sync();
        for (int s = 0; s < k1; ++s)
          tc::mma_f16(tw, tc::smem_desc(xa + s * 4096, 2048, 128), d[s], id64, s > 0);
        tc::mma_commit(&bar_d[w]);
        if (!(ok = tc::mbar_wait(&bar_h[w], ph, kWaitLimit))) break;
        ph ^= 1;
        tc::fence_after_sync();
        for (int s = 0; s < kHidden / 16; ++s)
          tc::mma_f16_ta(tw, tw + kColH + 8 * s, d[4 + s], id64, s > 0);
        tc::mma_f16(tw, cst, d[8], id64, 1);
        tc::mma_commit(&bar_d[w]);
        if (!(ok = tc::mbar_wait(&bar_h[w], ph, kWaitLimit))) break;
        ph ^= 1;
        tc::fence_after_sync();
        for (int s = 0; s < kHidden / 16; ++s)
          tc::mma_f16_ta(tw + kColD3, tw + kColH + 8 * s, d[9 + s], id16, s > 0);
        tc::mma_f16(tw + kColD3, cst, d[13], id16, 1);
        tc::mma_commit(&bar_o[w]);
      }
      if (!ok) *reinterpret_cast<volatile int*>(&wg_abort[w]) = 1;
      // every MMA of this thread completes before TMEM is released
      tc::mma_commit(&bar_fin[w]);
      if (!tc::mbar_wait(&bar_fin[w], 0, kWaitLimit)) *reinterpret_cast<volatile int*>(&wg_abort[w]) = 1;
    }
  } else {
    // ---- compute warpgroup w -------------------------------------------------
    const uint32_t lq = (uint32_t)((warp & 3) * 32) << 16;
    const uint32_t td = tw + lq, th = tw + kColH + lq, td3 = tw + kColD3 + lq;
    const SmemRow xs{smem_row(sm + W.x + w * W.xbytes, row)};
    const MipTab* tb = reinterpret_cast<const MipTab*>(sm + P.tab);
    const FastK K(M);
    volatile int* abort_flag = &wg_abort[w];
    auto qindex = [&](int64_t t) { return tri ? t * per_tile + (row >> 3) : t * per_tile + row; };
    auto build = [&](const Row& r) {
      if (FAST) build_fast(P, K, sm, r, xs);
      else build_generic<false>(M, P, sm, r, xs, 1.f);
      tc::fence_proxy_async();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&bar_x[w]);
    };
    const int C = M.channels;
    uint32_t pd = 0, po = 0;
    int64_t tl = first;
    int cur_valid = 0;
    float cur_wtap = 0.f;
    Row nxt;
    Query nq;
    if (tl < ntiles) {
      Row r;
      const int64_t q0 = qindex(tl);
      locate(M, tb, load_query(uvl, q0, q0 < n), tri, row, r);
      if (FAST) gather_fast(tb, P, r);
      build(r);
      cur_valid = r.valid;
      cur_wtap = r.wtap;
      const int64_t q1 = qindex(tl + stride);
      locate(M, tb, load_query(uvl, q1, tl + stride < ntiles && q1 < n), tri, row, nxt);
      if (FAST) gather_fast(tb, P, nxt);
      const int64_t q2 = qindex(tl + 2 * stride);
      nq = load_query(uvl, q2, tl + 2 * stride < ntiles && q2 < n);
    }
    for (; tl < ntiles; tl += stride) {
      const int64_t q = qindex(tl);
      const bool valid = cur_valid != 0;
      const float wtap = cur_wtap;
      // layer 1 -> H1
      if (!tc::mbar_wait(&bar_d[w], pd, kWaitLimit)) *abort_flag = 1;
      pd ^= 1;
      tc::fence_after_sync();
      hidden_epilogue_q(td, th, M.act);
      tc::tmem_st_wait();
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&bar_h[w]);
      // the next tile's input rows (layer 1 is done with X)
      if (tl + stride < ntiles) {
        build(nxt);
        cur_valid = nxt.valid;
        cur_wtap = nxt.wtap;
      }
      // layer 2 -> H2
      if (!tc::mbar_wait(&bar_d[w], pd, kWaitLimit)) *abort_flag = 1;
      pd ^= 1;
      tc::fence_after_sync();
      hidden_epilogue_q(td, th, M.act);
      tc::tmem_st_wait();
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&bar_h[w]);
      if (*abort_flag) break;
      // the tile after next: texel and cells; its successor's query
      locate(M, tb, nq, tri, row, nxt);
      if (FAST) gather_fast(tb, P, nxt);
      {
        const int64_t t3 = tl + 3 * stride;
        const int64_t q3 = qindex(t3);
        nq = load_query(uvl, q3, t3 < ntiles && q3 < n);
      }
      // layer 3 -> output
      if (!tc::mbar_wait(&bar_o[w], po, kWaitLimit)) *abort_flag = 1;
      po ^= 1;
      tc::fence_after_sync();
      float yv[16];
      tc::tmem_ld16(td3, yv);
      tc::tmem_ld_wait();
      tc::fence_before_sync();
#pragma unroll
      for (int c = 0; c < 16; ++c)
        yv[c] = M.out_act == NTC_OUT_IDENTITY ? yv[c] : fmaf(0.5f, tc::tanh_fast(yv[c]), 0.5f);
      if (tri) {
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          float s = yv[c] * wtap;
          s += __shfl_xor_sync(0xffffffffu, s, 1);
          s += __shfl_xor_sync(0xffffffffu, s, 2);
          s += __shfl_xor_sync(0xffffffffu, s, 4);
          yv[c] = s;
        }
      }
      if (valid && (!tri || (row & 7) == 0)) store_texel(out, out_dtype, q, C, yv);
      if (*abort_flag) break;
    }
  }

  tc::fence_before_sync();
  __syncthreads();
  if (tid == 0) {
    int any = 0;
    for (int i = 0; i < kWsCompute; ++i) any |= wg_abort[i];
    if (any) atomicExch(status, NTC_ERR_TIMEOUT);
  }
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem_base, 512);
  }
}

template <bool FAST>
cudaError_t launch_ws(const ntc_material& m, const float* uvl, int64_t n, void* out, int out_dtype,
                      int filter, cudaStream_t s) {
  const Plan P(m.c0, m.c1, m.bits0, m.bits1, m.encoding == NTC_GRID_PACKED, false, FAST);
  const WsPlan W(P);
  cudaError_t e = cudaFuncSetAttribute(decode_ws_kernel<FAST>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)W.total);
  if (e != cudaSuccess) return e;
  const int per_tile = filter == NTC_FILTER_TRILINEAR ? kRows / 8 : kRows;
  const int64_t tiles = (n + per_tile - 1) / per_tile;
  const int64_t ctas = (tiles + kWsCompute - 1) / kWsCompute;
  const int64_t cap = sm_count();
  const int grid = (int)(ctas < cap ? ctas : cap);
  decode_ws_kernel<FAST><<<grid, kWsThreads, W.total, s>>>(m, uvl, n, out, out_dtype, filter,
                                                           status_word());
  return cudaGetLastError();
}

template <bool F8, bool FAST, int kNWG>
cudaError_t launch_k(const ntc_material& m, const float* uvl, int64_t n, void* out, int out_dtype,
                     int filter, cudaStream_t s) {
  const Plan P(m.c0, m.c1, m.bits0, m.bits1, m.encoding == NTC_GRID_PACKED, F8, FAST);
  const size_t smem = P.total;
  cudaError_t e = cudaFuncSetAttribute(decode_tc_kernel<F8, FAST, kNWG>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int per_tile = filter == NTC_FILTER_TRILINEAR ? kRows / 8 : kRows;
  const int64_t tiles = (n + per_tile - 1) / per_tile;
  const int64_t ctas = (tiles + kNWG - 1) / kNWG;
  const int64_t cap = sm_count();
  const int grid = (int)(ctas < cap ? ctas : cap);
  decode_tc_kernel<F8, FAST, kNWG><<<grid, kRows * kNWG, smem, s>>>(m, uvl, n, out, out_dtype,
                                                                    filter, status_word());
  return cudaGetLastError();
}

template <bool F8, bool FAST>
cudaError_t launch_shape(const ntc_material& m, const float* uvl, int64_t n, void* out,
                         int out_dtype, int filter, cudaStream_t s, int nwg) {
  switch (nwg) {
    case 2: return launch_k<F8, FAST, 2>(m, uvl, n, out, out_dtype, filter, s);
    case 3: return launch_k<F8, FAST, 3>(m, uvl, n, out, out_dtype, filter, s);
    default: return launch_k<F8, FAST, 4>(m, uvl, n, out, out_dtype, filter, s);
  }
}

// ---------------------------------------------------------------------------
// Many materials in one persistent launch (FP16).  The batch descriptor in
// device memory lists the materials, the prefix sums of their tiles and the
// offsets of their queries and outputs; tiles are ordered by material.  Each
// warpgroup takes a contiguous range of tiles and keeps a private copy of the
// current material's weights and tables in shared memory, restaged when its
// range crosses into the next material.
// ---------------------------------------------------------------------------
template <bool FAST>
__global__ void __launch_bounds__(kRows * 4, 1) decode_batched_kernel(
    const BatchHeader* __restrict__ B, const float* __restrict__ uvl, void* __restrict__ out,
    int out_dtype, int filter, uint32_t wg_smem, int* status) {
  constexpr int kNWG = 4;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ uint64_t mbar[kNWG];
  __shared__ uint32_t tmem_base;
  __shared__ int wg_abort[kNWG];
  __shared__ ntc_material mat_s[kNWG];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int wg = tid / kRows, row = tid % kRows;
  const int bar_id = 1 + wg;
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, 512);
    tc::tmem_relinquish();
  }
  if (tid < kNWG) {
    tc::mbar_init(&mbar[tid], 1);
    wg_abort[tid] = 0;
  }
  tc::fence_mbar_init();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tw = tmem_base + 128u * wg;
  const uint32_t lane = (uint32_t)((warp & 3) * 32) << 16;
  const uint32_t td = tw + lane, th = tw + kColH + lane, tx = tw + kColX + lane;
  uint64_t* bar = &mbar[wg];
  volatile int* abort_flag = &wg_abort[wg];
  tc::tmem_st4(tw + kColCst + lane, make_uint4(tc::pack_f16x2(1.f, 1.f), 0, 0, 0));
  tc::tmem_st4(tw + kColCst + 4 + lane, make_uint4(0, 0, 0, 0));
  uint8_t* sm = smem_raw + (size_t)wg * wg_smem;
  constexpr uint32_t id64 = tc::idesc(kRows, kHidden), id16 = tc::idesc(kRows, kN3);
  const bool tri = filter == NTC_FILTER_TRILINEAR;
  const int per_tile = tri ? kRows / 8 : kRows;
  const int nm = B->n_materials;
  const int64_t total = B->total_tiles;
  const int64_t nwgs = (int64_t)gridDim.x * kNWG, gwg = (int64_t)blockIdx.x * kNWG + wg;
  const int64_t t_begin = total * gwg / nwgs, t_end = total * (gwg + 1) / nwgs;
  uint32_t phase = 0;
  int cur = -1;
  bool aborted = false;
  const float dummy_scale[3] = {1.f, 1.f, 1.f};
  (void)dummy_scale;

  for (int64_t tl = t_begin; tl < t_end; ++tl) {
    // material of this tile (tiles are ordered by material)
    int mid = cur < 0 ? 0 : cur;
    while (mid + 1 < nm && tl >= B->tile_start[mid + 1]) ++mid;
    if (mid != cur) {
      tc::bar_sync(bar_id, kRows);  // every row is done with the previous material
      if (row == 0) mat_s[wg] = B->mats[mid];
      tc::bar_sync(bar_id, kRows);
      const ntc_material& Mn = mat_s[wg];
      const Plan Pn(Mn.c0, Mn.c1, Mn.bits0, Mn.bits1, Mn.encoding == NTC_GRID_PACKED, false, FAST);
      stage_shared<false>(Mn, Pn, sm, row, kRows);
      zero_tail_groups<false>(Pn, TmemRow{tx});
      tc::tmem_st_wait();
      tc::fence_proxy_async();
      tc::bar_sync(bar_id, kRows);
      cur = mid;
    }
    const ntc_material& M = mat_s[wg];
    const Plan P(M.c0, M.c1, M.bits0, M.bits1, M.encoding == NTC_GRID_PACKED, false, FAST);
    const MipTab* tb = reinterpret_cast<const MipTab*>(sm + P.tab);
    const uint64_t* dsc = reinterpret_cast<const uint64_t*>(sm + P.desc);
    const int64_t local = tl - B->tile_start[mid];
    const int64_t nq = B->q_off[mid + 1] - B->q_off[mid];
    const int64_t ql = tri ? local * per_tile + (row >> 3) : local * per_tile + row;
    const bool valid = ql < nq;
    const int64_t qg = B->q_off[mid] + ql;
    Row r;
    locate(M, tb, load_query(uvl, qg, valid), tri, row, r);
    if (FAST) {
      gather_fast(tb, P, r);
      build_fast(P, FastK(M), sm, r, TmemRow{tx});
    } else {
      build_generic<false>(M, P, sm, r, TmemRow{tx}, 1.f);
    }
    tc::tmem_st_wait();
    tc::fence_before_sync();
    tc::bar_sync(bar_id, kRows);

    if (row == 0)
      issue_layer<false>(tw, tw + kColX, dsc, P.k_int / 16, id64, false, 0, bar);
    if (!tc::mbar_wait(bar, phase, kWaitLimit)) *abort_flag = 1;
    phase ^= 1;
    tc::fence_after_sync();
    hidden_epilogue<false>(td, th, M.act, nullptr, 1.f, 1.f);
    tc::tmem_st_wait();
    tc::fence_before_sync();
    tc::bar_sync(bar_id, kRows);
    if (row == 32)
      issue_layer<false>(tw, tw + kColH, dsc + 4, 4, id64, true, tw + kColCst, bar);
    if (!tc::mbar_wait(bar, phase, kWaitLimit)) *abort_flag = 1;
    phase ^= 1;
    tc::fence_after_sync();
    hidden_epilogue<false>(td, th, M.act, nullptr, 1.f, 1.f);
    tc::tmem_st_wait();
    tc::fence_before_sync();
    tc::bar_sync(bar_id, kRows);
    if (*abort_flag) { aborted = true; break; }
    if (row == 64)
      issue_layer<false>(tw, tw + kColH, dsc + 9, 4, id16, true, tw + kColCst, bar);
    if (!tc::mbar_wait(bar, phase, kWaitLimit)) *abort_flag = 1;
    phase ^= 1;
    tc::fence_after_sync();
    float yv[16];
    tc::tmem_ld16(td, yv);
    tc::tmem_ld_wait();
    tc::fence_before_sync();
#pragma unroll
    for (int c = 0; c < 16; ++c)
      yv[c] = M.out_act == NTC_OUT_IDENTITY ? yv[c] : fmaf(0.5f, tc::tanh_fast(yv[c]), 0.5f);
    if (tri) {
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        float s = yv[c] * r.wtap;
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        s += __shfl_xor_sync(0xffffffffu, s, 2);
        s += __shfl_xor_sync(0xffffffffu, s, 4);
        yv[c] = s;
      }
    }
    const int C = M.channels;
    if (valid && (!tri || (row & 7) == 0)) {
      const int64_t o = B->o_off[mid] + ql * C;
      if (out_dtype == NTC_DTYPE_F16) {
        __half* op = static_cast<__half*>(out) + o;
#pragma unroll
        for (int c = 0; c < 16; ++c)
          if (c < C) op[c] = __float2half_rn(yv[c]);
      } else {
        float* op = static_cast<float*>(out) + o;
#pragma unroll
        for (int c = 0; c < 16; ++c)
          if (c < C) op[c] = yv[c];
      }
    }
    tc::bar_sync(bar_id, kRows);
    if (*abort_flag) { aborted = true; break; }
  }

  tc::fence_before_sync();
  __syncthreads();
  if (tid == 0) {
    int any = aborted ? 1 : 0;
    for (int w = 0; w < kNWG; ++w) any |= wg_abort[w];
    if (any) atomicExch(status, NTC_ERR_TIMEOUT);
  }
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem_base, 512);
  }
}

}  // namespace

// The fast layout's exactness conditions: every grid/mip size ratio of every
// mip is a multiple of 1/8 (taps on the 1/16 lattice) and the bin widths are
// powers of two in [2^-6, 2^6] (the half constants of ylerp_of exact).
bool fast_layout_ok(const ntc_material& m) {
  for (int mi = 0; mi < m.mips; ++mi) {
    const int wm = mip_dim(m.width, mi), hm = mip_dim(m.height, mi);
    const ntc_level& L = m.lv[level_of_mip(mi, m.levels)];
    if ((8 * L.g0_w) % wm || (8 * L.g0_h) % hm || (8 * L.g1_w) % wm || (8 * L.g1_h) % hm)
      return false;
  }
  for (float q : {m.q0, m.q1}) {
    int e = 0;
    if (!(q > 0.f) || std::frexp(q, &e) != 0.5f || e < -5 || e > 7) return false;
  }
  return true;
}

// Launch shape: one CTA per SM with `nwg` warpgroup pipelines (2, 3 or 4),
// each holding 128 of the SM's 512 TMEM columns, or (5, the default for 0)
// the warp-specialised form: 4 compute warpgroups plus their MMA issuers
// (FP16; FP8 runs 4 pipelines).
cudaError_t launch_decode_tc(const ntc_material& m, const float* uvl, int64_t n, void* out,
                             int out_dtype, int filter, cudaStream_t s, int nwg) {
  if (n == 0) return cudaSuccess;
  if (nwg == 0) nwg = 5;
  if (nwg < 2 || nwg > 5) return cudaErrorInvalidValue;
  if (m.precision == NTC_PREC_F8)
    return launch_shape<true, false>(m, uvl, n, out, out_dtype, filter, s, nwg == 5 ? 4 : nwg);
  if (m.precision != NTC_PREC_F16) return cudaErrorInvalidValue;
  const Plan P(m.c0, m.c1, m.bits0, m.bits1, m.encoding == NTC_GRID_PACKED, false,
               fast_layout_ok(m));
  if (nwg == 5)
    return P.fast ? launch_ws<true>(m, uvl, n, out, out_dtype, filter, s)
                  : launch_ws<false>(m, uvl, n, out, out_dtype, filter, s);
  if (P.fast) return launch_shape<false, true>(m, uvl, n, out, out_dtype, filter, s, nwg);
  return launch_shape<false, false>(m, uvl, n, out, out_dtype, filter, s, nwg);
}

uint32_t batched_wg_smem(const ntc_material& m, bool fast) {
  const Plan P(m.c0, m.c1, m.bits0, m.bits1, m.encoding == NTC_GRID_PACKED, false, fast);
  return (P.total + 127) / 128 * 128;
}
bool batched_fast(const ntc_material& m) {
  return Plan(m.c0, m.c1, m.bits0, m.bits1, m.encoding == NTC_GRID_PACKED, false,
              fast_layout_ok(m)).fast != 0;
}

cudaError_t launch_decode_batched(const BatchHeader* dev, int64_t total_tiles, uint32_t wg_smem,
                                  bool fast, const float* uvl, void* out, int out_dtype, int filter,
                                  cudaStream_t s) {
  if (total_tiles == 0) return cudaSuccess;
  const size_t smem = (size_t)wg_smem * 4;
  const void* fn = fast ? (const void*)decode_batched_kernel<true> : (const void*)decode_batched_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t cap = sm_count();
  const int64_t ctas = (total_tiles + 3) / 4;
  const int grid = (int)(ctas < cap ? ctas : cap);
  if (fast)
    decode_batched_kernel<true><<<grid, kRows * 4, smem, s>>>(dev, uvl, out, out_dtype, filter, wg_smem,
                                                              status_word());
  else
    decode_batched_kernel<false><<<grid, kRows * 4, smem, s>>>(dev, uvl, out, out_dtype, filter, wg_smem,
                                                               status_word());
  return cudaGetLastError();
}

}  // namespace ntc
