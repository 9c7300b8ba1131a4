// Tensor-core (tcgen05) fused forward + L2 loss + backward of the NTC
// optimisation step (Sec. 4.2, 4.5, 5.1), FP16 operands, FP32 accumulation.
//
// One persistent CTA per SM runs NWG warpgroup pipelines (3, 2 or 1: the most
// whose tiles fit in shared memory); a warpgroup owns a stream of tiles of 128
// training texels (one per thread = one row = one TMEM lane).  Per tile, with
// every activation kept on chip:
//   forward   X -> Z1 = X W1^T (+b1) -> H1 = act(Z1) -> Z2 (+b2) -> H2 -> Z3 (+b3)
//             -> y = out(Z3), loss, dZ3 = 2 (y - t) out'(Z3); with a third
//             hidden layer H2 -> Zh (+bh) -> H3 feeds the output layer, and
//             the backward passes through it the same way (dWh += dZh^T
//             [H2 | 1], dZ2 over H2 from dH2 = dZh Wh)
//   backward  dH2 = dZ3 W3 and [dW3^T; db3] += [H2^T; 1] dZ3;
//             dZ2 = dH2 * act'(Z2) (over H2); dH1 = dZ2 W2 and
//             [dW2 db2] += dZ2^T [H1 | 1]; dZ1 = dH1 * act'(Z1) (over H1);
//             dX = dZ1 W1 and [dW1 db1] += dZ1^T X; dX -> scatter-add into
//             the grid gradients through the taps (FP32 atomics): bilinear
//             weights for a bilinear grid, weight 1 per tap slot for learned
//             interpolation of G0 (Sec. 4.3.1).
// The weight-gradient accumulators live in TMEM once per CTA, shared by its
// pipelines (zeroed at the start; every pipeline's MMAs add into them, the
// tensor pipe applies them in order) and leave it once at the end.  Each
// weight gradient is issued as soon as its operands exist, so dZ2 and dZ1
// overwrite H2 and H1 in place.  X, H1, H2, dZ3 are FP16 tiles in shared
// memory, one row per texel in the canonical K-major layout (8 x 16-byte core
// matrices, row group fastest): K-major A operands of the layers and, read
// with the MN-major descriptor mode (K = the 128 texels), operands of the
// weight-gradient MMAs; those take M = 128 rows from 16 consecutive groups,
// of which the first 8 (or 9) are meaningful.  The backward layers read the
// forward weight tiles as MN-major B operands (no transposed copies).  The
// biases of layer 1 ride in X's two constant-one slots, so X's columns of
// the dW1 accumulator give db1.  The forward products whose result passes a
// ReLU (or hardGELU) kink take their A operand as an FP16 head plus an FP16
// tail (v = head + tail to ~2^-22): X for layer 1, H1 for layer 2 and, with
// a third hidden layer, H2 for it.  With FP16 heads alone the sign of a Z
// near zero follows the rounding of its inputs, and the few units whose
// activation mask then differs from the exact one move a tensor's gradient
// by about 1% of its norm; the tails make the masks those of the exact
// forward.  A tail tile is needed only by the one MMA that reads it, so it
// lives in a tile of the region that is still free at that point: X's tail
// in the H1 tile (and the H2 tile beyond 64 inputs), H1's tail in the H2
// tile, H2's tail in the H3 tile.  ReLU's derivative is read back from the sign
// of H; hardGELU's act'(Z) is written in FP16 into a G tile by the forward
// epilogue.  dZ3 carries the loss scale B*C (2 (y - t) instead of
// 2 (y - t) / (B C)) so it stays well inside FP16's range; every gradient is
// multiplied by 1 / (B C) in FP32 when it leaves the chip.
#pragma once

#include <cuda_fp16.h>

#include "ntc_device.cuh"
#include "ntc_internal.h"
#include "tc_ptx.cuh"

namespace ntc {

namespace {

constexpr int kRows = 128;
constexpr int kN3 = 16;
constexpr int kMaxNWG = 3;              // warpgroup pipelines per CTA (at most)
constexpr uint32_t kCols = 512;         // TMEM columns of the CTA
constexpr uint32_t kGroup = 2048;       // bytes per 8-unit group of a 128-row tile
constexpr uint32_t kWaitLimit = 1u << 18;  // suspended tries: ms to seconds
constexpr int kDxStride = 84;           // floats per row of the dX staging rows
// Coalesced grid scatter: per warp, 32 dX rows of 36 floats (conflict-free
// 16-byte stores) and 32 rows of 112 bytes holding the 8 (grid, tap) cell
// addresses and weights of a texel; 8 KB per warp, 32 KB per pipeline.
constexpr int kScatDx = 36, kScatMeta = 112, kScatWarp = 32 * kScatDx * 4 + 32 * kScatMeta;
constexpr uint32_t kSmemMax = 232448u - 2048u;  // dynamic shared memory (static reserve)

// Shared-memory and TMEM plan.  Input slots: G0 groups (c0 values, or the
// four taps' 4 c0 values with learned interpolation), G1 groups,
// [PE0..7][PE8..11, LOD, 0, 1, 1], zero groups up to k_int.
struct TPlan {
  int w0, f0, f1, gpe, k_int, dx_n, nwg, h3, f8, k8;
  uint32_t w1, w2, w3, wb2, wb3, wh, wbh, tab, wg0, wg_bytes, total;
  // FP8-E4M3 forward (R24): E4M3 weight tiles, FP32 biases, and per
  // pipeline S8, the E4M3 tile of H2 (X's E4M3 tile lives in the H1 tile
  // and H1's in the H2 tile until the MMA that reads each has completed)
  uint32_t w1_8, w2_8, w3_8, bf, S8;
  uint32_t dmax, colW1, colW2, colWh, colW3, cols;  // TMEM: D of pipeline p at p dmax, then
                                                    // the shared weight-gradient accumulators
  // offsets inside one pipeline's region, in this order (the MN-major reads
  // of 16 groups from H1, H2 or H3 stay inside it): H1 (= dZ1), ONEa (2
  // groups: the K = 16 bias steps and the ones column of dW2), H2 (= dZ2),
  // with a third hidden layer ONEc (2 groups: the ones column of dWh) and H3
  // (= dZh), then ONEb (1 group: the db3 row of dW3), DZ3, X, and for
  // hardGELU G1, G2 (, G3): act'(Z) of each hidden layer.  HL is the last
  // hidden tile (H2 or H3).
  uint32_t H1, ONEa, H2, ONEc, H3, HL, ONEb, DZ3, X, G1, G2, G3;
  // k_lay, dx_lay: a batch's largest k_int and dx_n; the offsets and TMEM
  // columns follow the larger of them and this material's own, so that
  // every material of a batch shares one layout (0: this material alone).
  __host__ __device__ TPlan(int c0, int c1, bool learned, bool gelu, int n_wg, bool third,
                            int k_lay = 0, int dx_lay = 0, bool fp8 = false) {
    w0 = learned ? 4 * c0 : c0;
    f0 = (w0 + 7) / 8;
    f1 = (c1 + 7) / 8;
    gpe = f0 + f1;
    k_int = (8 * (gpe + 2) + 15) / 16 * 16;
    dx_n = (8 * gpe + 15) / 16 * 16;     // dX columns: the grid slots
    nwg = n_wg;
    h3 = third;
    f8 = fp8;
    k8 = (k_int + 31) / 32 * 32;  // E4M3 K-steps take 32 inputs
    const int kl = k_int > k_lay ? k_int : k_lay, dl = dx_n > dx_lay ? dx_n : dx_lay;
    uint32_t o = 0;
    w1 = o;  o += kHidden * kl * 2;      // W1 [64][k_int]: B of layer 1, MN-major B of dX
    w2 = o;  o += kHidden * kHidden * 2; // W2: B of layer 2, MN-major B of dH1
    w3 = o;  o += kN3 * kHidden * 2;     // W3 [16][64]: B of layer 3, MN-major B of dH2
    wb2 = o; o += kHidden * 16 * 2;      // bias blocks (head, tail)
    wb3 = o; o += kN3 * 16 * 2;
    wh = o;  o += h3 ? kHidden * kHidden * 2 : 0;  // Wh: B of the third layer, MN-major B of dH2
    wbh = o; o += h3 ? kHidden * 16 * 2 : 0;
    o = (o + 15) / 16 * 16;
    tab = o; o += 16 * 16 * 4;           // per-mip table (MipTabT)
    w1_8 = o; o += fp8 ? kHidden * k8 : 0;
    w2_8 = o; o += fp8 ? kHidden * kHidden : 0;
    w3_8 = o; o += fp8 ? kN3 * kHidden : 0;
    bf = o;   o += fp8 ? (2 * kHidden + kN3) * 4 : 0;
    o = (o + 1023) / 1024 * 1024;
    wg0 = o;
    H1 = 0;
    ONEa = H1 + 8 * kGroup;
    H2 = ONEa + 2 * kGroup;
    ONEc = H2 + 8 * kGroup;
    H3 = ONEc + (h3 ? 2 * kGroup : 0);
    HL = h3 ? H3 : H2;
    ONEb = HL + 8 * kGroup;
    DZ3 = ONEb + 1 * kGroup;
    X = DZ3 + 2 * kGroup;
    G1 = X + (kl / 8) * kGroup;
    G2 = G1 + (gelu ? 8 * kGroup : 0);
    G3 = G2 + (gelu ? 8 * kGroup : 0);
    wg_bytes = G3 + (gelu && h3 ? 8 * kGroup : 0);
    if (wg_bytes < HL + 16 * kGroup) wg_bytes = HL + 16 * kGroup;
    S8 = wg_bytes;
    if (fp8) wg_bytes += kRows * kHidden;
    total = wg0 + nwg * wg_bytes;
    dmax = dl > kHidden ? dl : kHidden;
    colW1 = nwg * dmax;
    colW2 = colW1 + kl;
    colWh = colW2 + kHidden + 16;
    colW3 = colWh + (h3 ? kHidden + 16 : 0);
    cols = colW3 + kN3;
  }
  // fits one CTA: shared memory, TMEM, the dX staging rows
  __host__ __device__ bool fits() const {
    return total <= kSmemMax && cols <= kCols && (uint32_t)kRows * kDxStride * 4 <= wg_bytes &&
           dmax <= kDxStride && colW2 - colW1 <= 2 * kHidden && (!f8 || (!h3 && k8 <= 2 * kHidden));
  }
};

struct MipTabT {
  int wm[16], hm[16], level[16];
  float lodn[16];
};

// User column of internal input slot s: >= 0 a W1 column, -1 zero padding,
// -2 / -3 the constant-one slots (bias head / tail).
__device__ __forceinline__ int slot_column(const ntc_material& M, const TPlan& P, int s) {
  int g = s >> 3;
  const int e = s & 7;
  if (g < P.f0) return 8 * g + e < P.w0 ? 8 * g + e : -1;
  g -= P.f0;
  if (g < P.f1) return 8 * g + e < M.c1 ? P.w0 + 8 * g + e : -1;
  g -= P.f1;
  const int pe = P.w0 + M.c1;
  if (g == 0) return pe + e;
  if (g == 1) {
    if (e < 4) return pe + 8 + e;
    if (e == 4) return pe + 12;
    if (e == 6) return -2;
    if (e == 7) return -3;
  }
  return -1;
}

__device__ __forceinline__ void split_bias(float b, __half& hd, __half& tl) {
  hd = __float2half_rn(b);
  tl = __float2half_rn(b - __half2float(hd));
}

__device__ __forceinline__ __half w_at(const ntc_material& M, int l, int idx) {
  return static_cast<const __half*>(M.w[l])[idx];
}

// Packed E4M3x2 (byte 0 -> low half) -> packed f16x2; exact (every E4M3
// value is an FP16 value).
__device__ __forceinline__ uint32_t e4m3x2_to_f16x2(uint32_t b) {
  uint32_t d;
  const uint16_t h = (uint16_t)b;
  asm("cvt.rn.f16x2.e4m3x2 %0, %1;\n" : "=r"(d) : "h"(h));
  return d;
}

// E4M3 byte -> FP16 (exact).
__device__ __forceinline__ __half e4m3_to_half(uint8_t b) {
  union { uint32_t u; __half2 h; } c;
  c.u = e4m3x2_to_f16x2(b);
  return __low2half(c.h);
}

// FP8 form (R24): the material's weights are E4M3 bytes (the step's pre-pass
// quantised them from the FP32 masters with power-of-two scales).  The
// forward reads them as E4M3 tiles; the backward reads FP16 tiles holding
// the same E4M3 values (unscaled: the scales enter the FP32 epilogues); the
// biases go to FP32 arrays for the epilogues.
__device__ void stage_train_f8(const ntc_material& M, const TPlan& P, uint8_t* sm) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const uint8_t* w1 = static_cast<const uint8_t*>(M.w[0]);
  const uint8_t* w2 = static_cast<const uint8_t*>(M.w[1]);
  const uint8_t* w3 = static_cast<const uint8_t*>(M.w[2]);
  for (int i = tid; i < kHidden * P.k8; i += nt) {
    const int o = i / P.k8, s = i - o * P.k8;
    const int col = s < P.k_int ? slot_column(M, P, s) : -1;
    const uint8_t b = col >= 0 ? w1[o * M.k_in + col] : (uint8_t)0;
    sm[P.w1_8 + tc::canon_offset(o, s, kHidden, 1)] = b;
    if (s < P.k_int)
      *reinterpret_cast<__half*>(sm + P.w1 + tc::canon_offset(o, s, kHidden, 2)) = e4m3_to_half(b);
  }
  for (int i = tid; i < kHidden * kHidden; i += nt) {
    const int o = i / kHidden, k = i - o * kHidden;
    const uint8_t b = w2[i];
    sm[P.w2_8 + tc::canon_offset(o, k, kHidden, 1)] = b;
    *reinterpret_cast<__half*>(sm + P.w2 + tc::canon_offset(o, k, kHidden, 2)) = e4m3_to_half(b);
  }
  for (int i = tid; i < kN3 * kHidden; i += nt) {
    const int c = i / kHidden, k = i - c * kHidden;
    const uint8_t b = c < M.channels ? w3[i] : (uint8_t)0;
    sm[P.w3_8 + tc::canon_offset(c, k, kN3, 1)] = b;
    *reinterpret_cast<__half*>(sm + P.w3 + tc::canon_offset(c, k, kN3, 2)) = e4m3_to_half(b);
  }
  float* bf = reinterpret_cast<float*>(sm + P.bf);
  for (int i = tid; i < 2 * kHidden + kN3; i += nt)
    bf[i] = i < kHidden ? M.b[0][i]
                        : (i < 2 * kHidden ? M.b[1][i - kHidden]
                                           : (i - 2 * kHidden < M.channels ? M.b[2][i - 2 * kHidden] : 0.f));
}

// Eight consecutive FP16 values of row `row` of a [rows][ld] weight matrix,
// columns k0 .. k0 + 7 (one 16-byte chunk of the canonical K-major layout).
__device__ __forceinline__ uint4 w_chunk(const __half* w, int ld, int row, int k0) {
  const __half* p = w + (size_t)row * ld + k0;
  if ((reinterpret_cast<uintptr_t>(p) & 15) == 0) return __ldg(reinterpret_cast<const uint4*>(p));
  uint32_t h[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) h[e] = __ldg(reinterpret_cast<const unsigned short*>(p) + e);
  return make_uint4(h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16), h[6] | (h[7] << 16));
}

// A bias block chunk: (head, tail, 0, ..., 0) of an FP32 bias in group 0,
// zeros in group 1.
__device__ __forceinline__ uint4 bias_chunk(float b, int g) {
  if (g) return make_uint4(0u, 0u, 0u, 0u);
  __half hd, tl;
  split_bias(b, hd, tl);
  return make_uint4((uint32_t)__half_as_ushort(hd) | ((uint32_t)__half_as_ushort(tl) << 16), 0u, 0u, 0u);
}

// One staging job of the FP16 weight tiles: a 16-byte chunk (8 consecutive
// K values of one output row) of W1 (internal slot order, the bias head and
// tail in the constant-one slots), W2, W3 (rows >= C zero), the bias blocks
// of layers 2 and 3, and with a third hidden layer Wh and its bias block.
// Returns the chunk's byte offset in shared memory.
__device__ __forceinline__ uint32_t stage_job(const ntc_material& M, const TPlan& P, int j, uint4& v) {
  const int n1 = kHidden * (P.k_int / 8);
  if (j < n1) {
    const int o = j / (P.k_int / 8), g = j - o * (P.k_int / 8);
    uint32_t h[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int col = slot_column(M, P, 8 * g + e);
      __half x = __float2half_rn(0.f);
      if (col >= 0) {
        x = __ldg(static_cast<const __half*>(M.w[0]) + o * M.k_in + col);
      } else if (col < -1) {
        __half hd, tl;
        split_bias(__ldg(M.b[0] + o), hd, tl);
        x = col == -2 ? hd : tl;
      }
      h[e] = __half_as_ushort(x);
    }
    v = make_uint4(h[0] | (h[1] << 16), h[2] | (h[3] << 16), h[4] | (h[5] << 16), h[6] | (h[7] << 16));
    return P.w1 + tc::canon_chunk(o, g, kHidden);
  }
  j -= n1;
  if (j < kHidden * 8) {  // W2 [64][64]
    const int o = j >> 3, g = j & 7;
    v = w_chunk(static_cast<const __half*>(M.w[1]), kHidden, o, 8 * g);
    return P.w2 + tc::canon_chunk(o, g, kHidden);
  }
  j -= kHidden * 8;
  if (j < kN3 * 8) {  // W3 [C][64], rows >= C zero
    const int c = j >> 3, g = j & 7;
    v = c < M.channels ? w_chunk(static_cast<const __half*>(M.w[2]), kHidden, c, 8 * g)
                       : make_uint4(0u, 0u, 0u, 0u);
    return P.w3 + tc::canon_chunk(c, g, kN3);
  }
  j -= kN3 * 8;
  if (j < kHidden * 2) {  // bias block of layer 2
    const int o = j >> 1, g = j & 1;
    v = bias_chunk(g ? 0.f : __ldg(M.b[1] + o), g);
    return P.wb2 + tc::canon_chunk(o, g, kHidden);
  }
  j -= kHidden * 2;
  if (j < kN3 * 2) {  // bias block of layer 3, rows >= C zero
    const int c = j >> 1, g = j & 1;
    v = c < M.channels ? bias_chunk(g ? 0.f : __ldg(M.b[2] + c), g) : make_uint4(0u, 0u, 0u, 0u);
    return P.wb3 + tc::canon_chunk(c, g, kN3);
  }
  j -= kN3 * 2;
  if (j < kHidden * 8) {  // Wh [64][64] (third hidden layer)
    const int o = j >> 3, g = j & 7;
    v = w_chunk(static_cast<const __half*>(M.w_h3), kHidden, o, 8 * g);
    return P.wh + tc::canon_chunk(o, g, kHidden);
  }
  j -= kHidden * 8;
  const int o = j >> 1, g = j & 1;  // its bias block
  v = bias_chunk(g ? 0.f : __ldg(M.b_h3 + o), g);
  return P.wbh + tc::canon_chunk(o, g, kHidden);
}

__device__ void stage_train(const ntc_material& M, const TPlan& P, uint8_t* sm) {
  const int tid = threadIdx.x, nt = blockDim.x;
  if (P.f8) {
    stage_train_f8(M, P, sm);
  } else {
    // every thread issues the loads of up to four chunks before it stores
    // any of them, so the staging costs about one global round trip per
    // four chunks instead of one per element
    const int jobs = kHidden * (P.k_int / 8) + kHidden * 8 + kN3 * 8 + kHidden * 2 + kN3 * 2 +
                     (P.h3 ? kHidden * 8 + kHidden * 2 : 0);
    for (int j0 = tid; j0 < jobs; j0 += 4 * nt) {
      uint4 v[4];
      uint32_t off[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (j0 + u * nt < jobs) off[u] = stage_job(M, P, j0 + u * nt, v[u]);
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (j0 + u * nt < jobs) *reinterpret_cast<uint4*>(sm + off[u]) = v[u];
    }
  }
  MipTabT* tb = reinterpret_cast<MipTabT*>(sm + P.tab);
  for (int m = tid; m < M.mips; m += nt) {
    tb->wm[m] = mip_dim(M.width, m);
    tb->hm[m] = mip_dim(M.height, m);
    tb->level[m] = level_of_mip(m, M.levels);
    tb->lodn[m] = M.mips > 1 ? (float)m / (float)(M.mips - 1) : 0.f;
  }
  // the constant-one tiles of every pipeline: columns 0 and 1 are one
  // (ONEa, ONEc: groups 0 and 1; ONEb: group 0)
  for (int i = tid; i < P.nwg * 5 * kRows; i += nt) {
    const int w = i / (5 * kRows), t = (i / kRows) % 5, r = i % kRows;
    if (t >= 3 && !P.h3) continue;
    const uint32_t tile = t == 2 ? P.ONEb : (t < 2 ? P.ONEa : P.ONEc);
    const int g = (t == 1 || t == 4) ? 1 : 0;
    const uint4 one = make_uint4(tc::pack_f16x2(1.f, 1.f), 0u, 0u, 0u);
    *reinterpret_cast<uint4*>(sm + P.wg0 + w * P.wg_bytes + tile + tc::canon_chunk(r, g, kRows)) =
        g ? make_uint4(0, 0, 0, 0) : one;
  }
}

__device__ __forceinline__ void put_chunk(uint8_t* tile, int row, int g, const float (&v)[8]) {
  uint4 w;
  w.x = tc::pack_f16x2(v[0], v[1]);
  w.y = tc::pack_f16x2(v[2], v[3]);
  w.z = tc::pack_f16x2(v[4], v[5]);
  w.w = tc::pack_f16x2(v[6], v[7]);
  *reinterpret_cast<uint4*>(tile + tc::canon_chunk(row, g, kRows)) = w;
}

// Eight FP32 values -> their FP16 heads into the chunk at `hi` and the FP16
// tails v - head into the chunk at `lo`.
__device__ __forceinline__ void put_chunk_split(uint8_t* hi, uint8_t* lo, const float (&v)[8]) {
  uint32_t h[4], t[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    h[j] = tc::pack_f16x2(v[2 * j], v[2 * j + 1]);
    union { uint32_t u; __half2 h; } c;
    c.u = h[j];
    const float2 f = __half22float2(c.h);
    t[j] = tc::pack_f16x2(v[2 * j] - f.x, v[2 * j + 1] - f.y);
  }
  *reinterpret_cast<uint4*>(hi) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(lo) = make_uint4(t[0], t[1], t[2], t[3]);
}

// Region offset of group g of X's tail: the H1 tile's 8 groups, then the H2
// tile's (k_int <= 128).
__device__ __forceinline__ uint32_t xlo_group(const TPlan& P, int g) {
  return g < 8 ? P.H1 + (uint32_t)g * kGroup : P.H2 + (uint32_t)(g - 8) * kGroup;
}

// 64 values of a TMEM row (starting at column `col`) -> f(v) -> 8 FP16
// chunks of a tile.
template <class F>
__device__ __forceinline__ void row64_to_tile(uint32_t taddr, uint8_t* tile, int row, F f) {
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    float a[16], b[16];
    tc::tmem_ld16(taddr + 32 * half, a);
    tc::tmem_ld16(taddr + 32 * half + 16, b);
    tc::tmem_ld_wait();
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      float v[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int i = 8 * g + e;
        v[e] = f(32 * half + i, i < 16 ? a[i] : b[i - 16]);
      }
      put_chunk(tile, row, 4 * half + g, v);
    }
  }
}

// One tile's own row of an FP16 tile, unpacked (8 groups = 64 values).
__device__ __forceinline__ void tile_row64(const uint8_t* tile, int row, __half2 (&h)[32]) {
#pragma unroll
  for (int g = 0; g < 8; ++g) {
    const uint4 w = *reinterpret_cast<const uint4*>(tile + tc::canon_chunk(row, g, kRows));
    const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      union { uint32_t u; __half2 h; } c;
      c.u = u[j];
      h[4 * g + j] = c.h;
    }
  }
}

__device__ __forceinline__ float half_of(const __half2 (&h)[32], int i) {
  return (i & 1) ? __high2float(h[i >> 1]) : __low2float(h[i >> 1]);
}

__device__ __forceinline__ void issue_kmajor(uint32_t d, uint32_t a, uint32_t a_lbo, uint32_t b,
                                             uint32_t b_lbo, int ksteps, uint32_t id,
                                             uint32_t acc0) {
  for (int s = 0; s < ksteps; ++s)
    tc::mma_f16(d, tc::smem_desc(a + 2 * s * a_lbo, a_lbo, 128),
                tc::smem_desc(b + 2 * s * b_lbo, b_lbo, 128), id, (s > 0) | acc0);
}

// MN-major operands with K = the 128 texels of the tile: 8 K-steps of 16
// texels (2 row groups = 256 bytes).  Without swizzling the descriptor's
// stride-dimension offset steps between core matrices along M/N (the 8-unit
// groups, 2048 bytes apart) and the leading-dimension offset along K (the
// 8-texel groups, 128 bytes apart), as in the K-major case.
__device__ __forceinline__ void issue_mnmajor(uint32_t d, uint32_t a, uint32_t b, uint32_t id,
                                              uint32_t acc0) {
  for (int s = 0; s < kRows / 16; ++s)
    tc::mma_f16(d, tc::smem_desc(a + 256 * s, 128, kGroup), tc::smem_desc(b + 256 * s, 128, kGroup),
                id, (s > 0) | acc0);
}

// 32-byte read-only global load (sm_100+), 32-byte aligned address.
__device__ __forceinline__ void ld_nc_v8(const float* p, float4& a, float4& b) {
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
      : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
      : "l"(p));
}

// Bilinear sample of one FP32 grid of 4k <= 16 channels with 16-byte loads,
// all taps' loads issued before the interpolation (same FMA order as
// sample_grid, so the same values).
// `base` (nullable) replaces the level's grid pointer (the trainer's noisy
// copy of the same layout).
__device__ __forceinline__ void sample_grid_f32x4(const ntc_material& M, int j, int k, int x, int y,
                                                  int wm, int hm, GridSample& gs,
                                                  const float* base = nullptr) {
  const ntc_level& L = M.lv[j];
  const int gw = k ? L.g1_w : L.g0_w, gh = k ? L.g1_h : L.g0_h;
  const int c4 = (k ? M.c1 : M.c0) >> 2;
  const Taps t = bilinear_taps(x, y, wm, hm, gw, gh);
  const float4* g = static_cast<const float4*>(base ? static_cast<const void*>(base) : (k ? L.grid1 : L.grid0));
  float4 v[4][kFastGridCh / 4];
  if ((c4 == 2 || c4 == 4) && (reinterpret_cast<uintptr_t>(g) & 31) == 0) {
    // 32-byte loads: one L1 wavefront brings 8 channels
#pragma unroll
    for (int tp = 0; tp < 4; ++tp)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (2 * h < c4) ld_nc_v8(reinterpret_cast<const float*>(g + (size_t)t.cell[tp] * c4 + 2 * h),
                                 v[tp][2 * h], v[tp][2 * h + 1]);
        else v[tp][2 * h] = v[tp][2 * h + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
  } else {
#pragma unroll
    for (int tp = 0; tp < 4; ++tp)
#pragma unroll
      for (int q = 0; q < kFastGridCh / 4; ++q)
        v[tp][q] = q < c4 ? __ldg(g + (size_t)t.cell[tp] * c4 + q) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
#pragma unroll
  for (int ch = 0; ch < kGridPad; ++ch) gs.acc[ch] = 0.f;
#pragma unroll
  for (int tp = 0; tp < 4; ++tp)
#pragma unroll
    for (int q = 0; q < kFastGridCh / 4; ++q) {
      gs.acc[4 * q] = fmaf(t.w[tp], v[tp][q].x, gs.acc[4 * q]);
      gs.acc[4 * q + 1] = fmaf(t.w[tp], v[tp][q].y, gs.acc[4 * q + 1]);
      gs.acc[4 * q + 2] = fmaf(t.w[tp], v[tp][q].z, gs.acc[4 * q + 2]);
      gs.acc[4 * q + 3] = fmaf(t.w[tp], v[tp][q].w, gs.acc[4 * q + 3]);
    }
}

// K-major A, MN-major B: a forward weight tile [out][in] (K-major, `R` rows
// of outputs) read as B[n = in][k = out]; its core matrices step 128 bytes
// along K (8 outputs) and (R / 8) * 128 bytes along N.
__device__ __forceinline__ void issue_kmn(uint32_t d, uint32_t a, uint32_t a_lbo, uint32_t b,
                                          uint32_t b_sbo, int ksteps, uint32_t id) {
  for (int s = 0; s < ksteps; ++s)
    tc::mma_f16(d, tc::smem_desc(a + 2 * s * a_lbo, a_lbo, 128),
                tc::smem_desc(b + 256 * s, 128, b_sbo), id, s > 0);
}

// Forward epilogue of a hidden layer: H = act(Z) into `htile` (FP16 heads;
// with `ltile` the FP16 tails go there); hardGELU also writes act'(Z) into
// `gtile`.
template <int ACT>
__device__ __forceinline__ void hidden_forward(uint32_t taddr, uint8_t* htile, uint8_t* gtile,
                                               uint8_t* ltile, int row) {
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    float a[16], b[16];
    tc::tmem_ld16(taddr + 32 * half, a);
    tc::tmem_ld16(taddr + 32 * half + 16, b);
    tc::tmem_ld_wait();
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      float v[8], dv[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int i = 8 * g + e;
        const float z = i < 16 ? a[i] : b[i - 16];
        v[e] = act_fwd(ACT, z);
        dv[e] = act_grad(ACT, z);
      }
      const uint32_t ch = tc::canon_chunk(row, 4 * half + g, kRows);
      if (ltile) put_chunk_split(htile + ch, ltile + ch, v);
      else put_chunk(htile, row, 4 * half + g, v);
      if (ACT == NTC_ACT_HARDGELU) put_chunk(gtile, row, 4 * half + g, dv);
    }
  }
}

// FP8 form: eight features of a row rounded to E4M3 in units of the layer-1
// activation scale (x_hat = s_a e4m3(x / s_a)): the E4M3 bytes go to the A
// tile of layer 1 (laid over the H1 tile), the same values in FP16 (unscaled)
// to X for the weight-gradient MMA.  `ones`: the group holding the two
// constant-one slots (elements 6, 7), which stay 1 in X and 0 in the E4M3
// tile (the biases enter the epilogue).  amax: the largest |x| seen.
__device__ __forceinline__ void put_x8(uint8_t* W, const TPlan& P, int row, int g,
                                       const float (&v)[8], float inv, bool ones, float& amax) {
  uint32_t h[4], b[2] = {0u, 0u};
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const bool one = ones && j == 3;
    if (!one) amax = fmaxf(amax, fmaxf(fabsf(v[2 * j]), fabsf(v[2 * j + 1])));
    const uint32_t e = one ? 0u : tc::pack_e4m3x2(v[2 * j] * inv, v[2 * j + 1] * inv);
    h[j] = one ? tc::pack_f16x2(1.f, 1.f) : e4m3x2_to_f16x2(e);
    b[j >> 1] |= e << (16 * (j & 1));
  }
  *reinterpret_cast<uint4*>(W + P.X + (uint32_t)g * kGroup + tc::canon_chunk(row, 0, kRows)) =
      make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint2*>(W + P.H1 + tc::canon_chunk(row, g >> 1, kRows) + (g & 1) * 8) =
      make_uint2(b[0], b[1]);
}

// FP8 forward epilogue of a hidden layer: z = s_in acc + b (s_in = s_a s_w of
// the layer), H = act(z) rounded to E4M3 in units of the next layer's
// activation scale (inv = 1 / s_a'): bytes into `h8` (the next layer's A
// tile), the same values in FP16 into `h16` (for the backward); a ReLU unit
// with z > 0 whose value rounds to zero is stored as -0 so that the backward
// still reads its mask.  hardGELU writes act'(z) into `gtile`.
template <int ACT>
__device__ __forceinline__ void hidden_forward_f8(uint32_t taddr, float s_in, const float* bias,
                                                  float inv, uint8_t* h16, uint8_t* h8,
                                                  uint8_t* gtile, int row, float& amax) {
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    float a[16], b[16];
    tc::tmem_ld16(taddr + 32 * half, a);
    tc::tmem_ld16(taddr + 32 * half + 16, b);
    tc::tmem_ld_wait();
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      float z[8], dv[8];
      uint32_t hw[4], bw[2] = {0u, 0u};
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int i = 8 * g + e;
        z[e] = fmaf(i < 16 ? a[i] : b[i - 16], s_in, bias[32 * half + i]);
        dv[e] = act_grad(ACT, z[e]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float h0 = act_fwd(ACT, z[2 * j]), h1 = act_fwd(ACT, z[2 * j + 1]);
        amax = fmaxf(amax, fmaxf(fabsf(h0), fabsf(h1)));
        const uint32_t e = tc::pack_e4m3x2(h0 * inv, h1 * inv);
        uint32_t f = e4m3x2_to_f16x2(e);
        if (ACT == NTC_ACT_RELU) {
          if (z[2 * j] > 0.f && (f & 0xFFFFu) == 0u) f |= 0x8000u;
          if (z[2 * j + 1] > 0.f && (f >> 16) == 0u) f |= 0x80000000u;
        }
        hw[j] = f;
        bw[j >> 1] |= e << (16 * (j & 1));
      }
      const int gg = 4 * half + g;
      *reinterpret_cast<uint4*>(h16 + tc::canon_chunk(row, gg, kRows)) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
      *reinterpret_cast<uint2*>(h8 + tc::canon_chunk(row, gg >> 1, kRows) + (gg & 1) * 8) =
          make_uint2(bw[0], bw[1]);
      if (ACT == NTC_ACT_HARDGELU) put_chunk(gtile, row, gg, dv);
    }
  }
}

__device__ __forceinline__ void issue_kmajor_f8(uint32_t d, uint32_t a, uint32_t a_lbo, uint32_t b,
                                                uint32_t b_lbo, int ksteps, uint32_t id) {
  for (int s = 0; s < ksteps; ++s)
    tc::mma_f8(d, tc::smem_desc(a + 2 * s * a_lbo, a_lbo, 128),
               tc::smem_desc(b + 2 * s * b_lbo, b_lbo, 128), id, s > 0);
}

// Backward epilogue: dZ = dH * act'(Z) over the layer's H tile (this row is
// read before it is overwritten): ReLU takes act' from the sign of H,
// hardGELU from the forward's G tile.
// FP8 form: the accumulator is dZ_next W8 (E4M3 weight values), scaled by
// the layer's weight scale `sc`; a ReLU unit's mask is any nonzero bit
// pattern of H (its -0 marks a positive Z whose value rounded to zero).
template <int ACT, bool F8>
__device__ __forceinline__ void hidden_backward(uint32_t taddr, const uint8_t* gtile,
                                                uint8_t* htile, int row, float sc = 1.f) {
  __half2 h[32];
  tile_row64(ACT == NTC_ACT_HARDGELU ? gtile : htile, row, h);
  row64_to_tile(taddr, htile, row, [&](int q, float g) {
    if (F8) g *= sc;
    if (ACT == NTC_ACT_HARDGELU) return g * half_of(h, q);
    if (F8) {
      const __half hv = (q & 1) ? __high2half(h[q >> 1]) : __low2half(h[q >> 1]);
      return __half_as_ushort(hv) != 0 ? g : 0.f;
    }
    return half_of(h, q) > 0.f ? g : 0.f;
  });
}

// X slot s of a row: FP16 head into X, FP16 tail into X's tail groups.
__device__ __forceinline__ void put_half(uint8_t* W, const TPlan& P, int row, int s, float v) {
  const __half h = __float2half_rn(v);
  const uint32_t o = tc::canon_chunk(row, 0, kRows) + (s & 7) * 2;
  *reinterpret_cast<__half*>(W + P.X + (uint32_t)(s >> 3) * kGroup + o) = h;
  *reinterpret_cast<__half*>(W + xlo_group(P, s >> 3) + o) = __float2half_rn(v - __half2float(h));
}
// four values at slots s .. s+3, s a multiple of 4
__device__ __forceinline__ void put_half4(uint8_t* W, const TPlan& P, int row, int s, float4 v) {
  const uint32_t h0 = tc::pack_f16x2(v.x, v.y), h1 = tc::pack_f16x2(v.z, v.w);
  union { uint32_t u; __half2 h; } c0, c1;
  c0.u = h0;
  c1.u = h1;
  const float2 f0 = __half22float2(c0.h), f1 = __half22float2(c1.h);
  const uint32_t o = tc::canon_chunk(row, 0, kRows) + (s & 7) * 2;
  *reinterpret_cast<uint2*>(W + P.X + (uint32_t)(s >> 3) * kGroup + o) = make_uint2(h0, h1);
  *reinterpret_cast<uint2*>(W + xlo_group(P, s >> 3) + o) =
      make_uint2(tc::pack_f16x2(v.x - f0.x, v.y - f0.y), tc::pack_f16x2(v.z - f1.x, v.w - f1.y));
}
// Chunk g of a row of X: heads into X, tails into X's tail groups.
__device__ __forceinline__ void put_x(uint8_t* W, const TPlan& P, int row, int g,
                                      const float (&v)[8]) {
  const uint32_t o = tc::canon_chunk(row, 0, kRows);
  put_chunk_split(W + P.X + (uint32_t)g * kGroup + o, W + xlo_group(P, g) + o, v);
}

// Learned interpolation of G0 (Sec. 4.3.1): the c0 values of the four
// bilinear-footprint cells at slots tap * c0 + ch, zeros up to the group
// boundary.  FP32 grid values (plus this step's noise when asked).
__device__ __forceinline__ void learned_g0(const ntc_material& M, const TPlan& P, int j, int x,
                                           int y, int wm, int hm, bool valid, bool noise,
                                           uint64_t nkey, uint8_t* W, int row) {
  const ntc_level& L = M.lv[j];
  const Taps t = bilinear_taps(x, y, wm, hm, L.g0_w, L.g0_h);
  const int c = M.c0;
  if ((c & 3) == 0 && c <= kFastGridCh && !noise) {
    const float* g = static_cast<const float*>(L.grid0);
    float4 v[4][kFastGridCh / 4];
#pragma unroll
    for (int tp = 0; tp < 4; ++tp)
#pragma unroll
      for (int q = 0; q < kFastGridCh / 4; ++q)
        v[tp][q] = (valid && 4 * q < c)
                       ? __ldg(reinterpret_cast<const float4*>(g + (size_t)t.cell[tp] * c) + q)
                       : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int tp = 0; tp < 4; ++tp)
#pragma unroll
      for (int q = 0; q < kFastGridCh / 4; ++q)
        if (4 * q < c) put_half4(W, P, row, tp * c + 4 * q, v[tp][q]);
  } else {
#pragma unroll
    for (int tp = 0; tp < 4; ++tp)
      for (int ch = 0; ch < c; ++ch)
        put_half(W, P, row, tp * c + ch,
                 valid ? grid_value(M, j, 0, t.cell[tp], ch, noise, nkey) : 0.f);
  }
  for (int s = P.w0; s < 8 * P.f0; ++s) put_half(W, P, row, s, 0.f);
}

// Scatter-add of `d` (c values) into grid cell rows through four taps,
// weight w[tp] * gs each.
__device__ __forceinline__ void scatter_taps(float* g, int c, const Taps& t, const float* d,
                                             int tap_stride, bool bilinear, float gs) {
#pragma unroll
  for (int tp = 0; tp < 4; ++tp) {
    const float wgt = (bilinear ? t.w[tp] : 1.f) * gs;
    float* gp = g + (size_t)t.cell[tp] * c;
    const float* dt = d + tp * tap_stride;
    if ((c & 3) == 0) {
#pragma unroll
      for (int q = 0; q < kMaxGridCh / 4; ++q)
        if (4 * q < c) {
          const float4 v = *reinterpret_cast<const float4*>(dt + 4 * q);
          atomicAdd(reinterpret_cast<float4*>(gp) + q,
                    make_float4(v.x * wgt, v.y * wgt, v.z * wgt, v.w * wgt));
        }
    } else {
      for (int ch = 0; ch < c; ++ch) atomicAdd(gp + ch, dt[ch] * wgt);
    }
  }
}

// One lane's part of the coalesced grid scatter: slot `slot` (grid, tap) and
// channels 4q .. 4q+3 of each of the warp's 32 texels, whose cell addresses
// and weights sit at meta + t * kScatMeta and whose dX values at
// dx + t * dx_stride.  MERGE: consecutive texels that share the cell are
// summed in registers and reduced once per run (coherent texels: crops or
// given queries); otherwise one reduction per texel.
template <bool MERGE>
__device__ __forceinline__ void scatter_lane(const uint8_t* meta, const float* dx, int dx_stride,
                                             int slot, int q) {
  float* run = nullptr;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
  for (int t = 0; t < 32; ++t) {
    float* const ga = *reinterpret_cast<float* const*>(meta + t * kScatMeta + 8 * slot);
    if (MERGE) {
      if (ga != run) {
        if (run) atomicAdd(reinterpret_cast<float4*>(run) + q, acc);
        run = ga;
        acc = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    if (ga) {
      const float w = *reinterpret_cast<const float*>(meta + t * kScatMeta + 64 + 4 * slot);
      const float4 d = *reinterpret_cast<const float4*>(dx + t * dx_stride);
      if (MERGE) {
        acc.x = fmaf(d.x, w, acc.x);
        acc.y = fmaf(d.y, w, acc.y);
        acc.z = fmaf(d.z, w, acc.z);
        acc.w = fmaf(d.w, w, acc.w);
      } else {
        atomicAdd(reinterpret_cast<float4*>(ga) + q, make_float4(d.x * w, d.y * w, d.z * w, d.w * w));
      }
    }
  }
  if (MERGE && run) atomicAdd(reinterpret_cast<float4*>(run) + q, acc);
}

__device__ __forceinline__ bool wait_phase(uint64_t* bar, uint32_t& phase, int bar_id) {
  const bool ok = tc::mbar_wait(bar, phase, kWaitLimit);
  phase ^= 1;
  return !tc::bar_or(bar_id, kRows, !ok);
}

// BATCHED: the CTA takes an even share of the batch's tile list (ordered by
// material) and runs it material by material: for each material it stages
// the weights and tables, zeroes the shared weight-gradient accumulators,
// runs its tiles on the NWG pipelines, waits for their MMAs and flushes the
// accumulators into that material's gradient.  Otherwise one material (M0,
// A0) whose tiles the CTAs take in turn, NWG at a time.
template <int ACT, bool LEARNED, int NWG, bool BATCHED, bool F8>
__global__ void __launch_bounds__(kRows* NWG, 1) train_tc_kernel(const ntc_material M0,
                                                                  const BwdArgs A0,
                                                                  const TrainBatchDev* hb,
                                                                  int k_lay, int dx_lay,
                                                                  int* status) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ uint64_t mbar[NWG], fin[NWG];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_any;
  __shared__ float red[NWG * 4];
  __shared__ uint32_t dout_max;  // bits of the CTA's largest |dout| (dout mode)
  // the current material and step arguments of a batched launch
  __shared__ __align__(16) uint8_t seg_buf[BATCHED ? sizeof(ntc_material) + sizeof(BwdArgs) : 16];
  uint8_t* sm = smem_raw;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int wg = tid / kRows, row = tid % kRows;
  const int bar_id = 1 + wg;
  const uint32_t lane = (uint32_t)((warp & 3) * 32) << 16;
  const ntc_material& M = BATCHED ? *reinterpret_cast<const ntc_material*>(seg_buf) : M0;
  const BwdArgs& A =
      BATCHED ? *reinterpret_cast<const BwdArgs*>(seg_buf + sizeof(ntc_material)) : A0;

  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, kCols);
    tc::tmem_relinquish();
  }
  if (tid < NWG) {
    tc::mbar_init(&mbar[tid], 1);
    tc::mbar_init(&fin[tid], 1);
  }
  if (tid == 0) abort_any = 0;
  tc::fence_mbar_init();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();

  int64_t c_begin = 0, c_end = 0;
  int seg = 0;
  if (BATCHED) {
    const int64_t T = hb->total_tiles;
    c_begin = T * blockIdx.x / gridDim.x;
    c_end = T * (blockIdx.x + 1) / gridDim.x;
    while (seg < hb->n && hb->tile_start[seg + 1] <= c_begin) ++seg;
  }
  uint32_t phase = 0, fin_phase = 0;

  for (;;) {
  int64_t t_lo, t_hi, t_step;
  if (BATCHED) {
    if (seg >= hb->n || hb->tile_start[seg] >= c_end) break;
    const int64_t t0 = hb->tile_start[seg], t1 = hb->tile_start[seg + 1];
    if (t1 == t0) { ++seg; continue; }  // a material that sits out the step
    {
      const uint32_t* src_m = reinterpret_cast<const uint32_t*>(&hb->mats[seg]);
      const uint32_t* src_a = reinterpret_cast<const uint32_t*>(&hb->args[seg]);
      uint32_t* dst = reinterpret_cast<uint32_t*>(seg_buf);
      constexpr int nm = sizeof(ntc_material) / 4, na = sizeof(BwdArgs) / 4;
      for (int i = tid; i < nm + na; i += kRows * NWG) dst[i] = i < nm ? src_m[i] : src_a[i - nm];
    }
    __syncthreads();
    t_lo = (c_begin > t0 ? c_begin : t0) - t0 + wg;
    t_hi = (c_end < t1 ? c_end : t1) - t0;
    t_step = NWG;
  } else {
    t_lo = (int64_t)blockIdx.x * NWG + wg;
    t_hi = (A.n + kRows - 1) / kRows;
    t_step = (int64_t)gridDim.x * NWG;
  }
  const TPlan P(M.c0, M.c1, LEARNED, ACT == NTC_ACT_HARDGELU, NWG, M.hidden_layers == 3, k_lay,
                dx_lay, F8);
  const int C = M.channels;
  stage_train(M, P, sm);
  // FP8 form: this step's scales (weights s_w, layer inputs s_a; powers of
  // two written by the step's pre-pass) and the largest |input| of each
  // layer seen by this thread (delayed scaling of the next step)
  float sw[3] = {1.f, 1.f, 1.f}, sa[3] = {1.f, 1.f, 1.f}, am[3] = {0.f, 0.f, 0.f};
  if (F8)
    for (int l = 0; l < 3; ++l) {
      sw[l] = M.scale[l];
      sa[l] = M.scale[3 + l];
    }
  if (tid == 0) dout_max = 0u;
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  // the shared weight-gradient accumulators start at zero (warpgroup 0 holds
  // every lane; every MMA into them accumulates)
  if (wg == 0) {
    const uint32_t z[16] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (uint32_t c = P.colW1; c < P.cols; c += 16) tc::tmem_st16(tmem_base + c + lane, z);
    tc::tmem_st_wait();
  }
  // dout mode: the largest |dout| over the rows of this CTA's tiles
  if (A.dout) {
    float mx = 0.f;
    for (int64_t tl = t_lo; tl < t_hi; tl += t_step) {
      const int64_t i = tl * kRows + row;
      if (i < A.n)
        for (int c = 0; c < C; ++c) mx = fmaxf(mx, fabsf(A.dout[i * C + c]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((tid & 31) == 0) atomicMax(&dout_max, __float_as_uint(mx));
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  // An upstream gradient of any magnitude enters the FP16 dZ3 tile scaled by
  // a power of two that brings this CTA's largest |dout| into [1, 2) (the
  // loss mode's 2 (y - t) lies in the same range); every gradient leaving the
  // CTA is divided by it again in FP32.  One scale per CTA keeps its shared
  // weight-gradient accumulators consistent.
  float dscale = 1.f;
  if (A.dout) {
    const float mx = __uint_as_float(dout_max);
    if (mx > 0.f && mx < __int_as_float(0x7f800000)) {
      int e = 0;
      frexpf(mx, &e);  // mx = f 2^e, f in [0.5, 1)
      int k = 1 - e;
      k = k < -120 ? -120 : (k > 120 ? 120 : k);
      dscale = __int_as_float((127 + k) << 23);
    }
  }
  const float gscale = A.grad_scale / dscale;

  const uint32_t tD = tmem_base + P.dmax * wg;
  uint64_t* bar = &mbar[wg];
  uint8_t* W = sm + P.wg0 + wg * P.wg_bytes;
  const uint32_t sW = tc::smem_u32(W), sbase = tc::smem_u32(sm);
  const MipTabT* tb = reinterpret_cast<const MipTabT*>(sm + P.tab);
  constexpr uint32_t lbo_a = (kRows / 8) * 128, lbo64 = (kHidden / 8) * 128, lbo16 = (kN3 / 8) * 128;
  constexpr uint32_t id64 = tc::idesc(kRows, kHidden), id16 = tc::idesc(kRows, kN3);
  constexpr uint32_t idb = 1u << 16, ida = 1u << 15;  // B / A read MN-major
  const uint32_t id_dx = tc::idesc(kRows, P.dx_n) | idb;
  const uint32_t id_w1 = tc::idesc(kRows, P.k_int) | ida | idb;
  constexpr uint32_t id_w2 = tc::idesc(kRows, kHidden + 16) | ida | idb;
  constexpr uint32_t id_w3 = tc::idesc(kRows, kN3) | ida | idb;
  const uint32_t tW1 = tmem_base + P.colW1, tW2 = tmem_base + P.colW2, tW3 = tmem_base + P.colW3;
  const uint32_t tWh = tmem_base + P.colWh;

  const int64_t step = A.step_dev ? *A.step_dev : A.noise_step;
  const uint64_t nkey = rng_key(A.noise_seed, noise_stream(step));
  // folded noise check: the noisy copy is current when its tag is {seed, step}
  const bool use_copy = A.noisy_tag && A.noisy_tag[0] == (int64_t)A.noise_seed && A.noisy_tag[1] == step;
  const bool noise_on = A.noise != 0 && !use_copy;
  const uint64_t skey = rng_key(A.sample_seed, sampler_stream(step));
  float loss_acc = 0.f;
  bool aborted = false;

  for (int64_t tl = t_lo; tl < t_hi; tl += t_step) {
    const int64_t i = tl * kRows + row;
    const bool valid = i < A.n;
    // ---- texel, target, features -> X -----------------------------------
    int x = 0, y = 0, m = 0;
    if (valid) {
      if (A.uvl) query_texel(M, A.uvl[3 * i], A.uvl[3 * i + 1], A.uvl[3 * i + 2], x, y, m);
      else sample_train_texel(A.crops != 0, skey, i, M.width, M.height, M.mips, x, y, m);
    }
    // loss mode: the texel's C <= 16 target bytes, loaded here and parked in
    // the (free) DZ3 tile once the features are built, so their latency
    // hides behind the gathers; the loss reads them back
    uint32_t tw[4] = {0u, 0u, 0u, 0u};
    if (A.target && valid) {
      const uint8_t* trow = A.target + A.tgt_off[m] + ((int64_t)y * tb->wm[m] + x) * C;
      if ((C & 3) == 0) {
        // whole 4-byte words of the u8 row (row offsets are multiples of 4)
#pragma unroll
        for (int c4 = 0; c4 < kN3 / 4; ++c4)
          if (4 * c4 < C) tw[c4] = __ldg(reinterpret_cast<const uint32_t*>(trow) + c4);
      } else {
#pragma unroll
        for (int c = 0; c < kN3; ++c)
          if (c < C) tw[c >> 2] |= (uint32_t)trow[c] << (8 * (c & 3));
      }
    }
    {
      const int j = tb->level[m];
      const int wm = tb->wm[m], hm = tb->hm[m];
      GridSample gs;
      if (LEARNED) learned_g0(M, P, j, x, y, wm, hm, valid, noise_on, nkey, W, row);
#pragma unroll
      for (int k = LEARNED ? 1 : 0; k < 2; ++k) {
        const int ck = k ? M.c1 : M.c0;
        if (!noise_on && (ck & 3) == 0 && ck <= kFastGridCh)
          sample_grid_f32x4(M, j, k, x, y, wm, hm, gs, use_copy ? (k ? A.noisy1[j] : A.noisy0[j]) : nullptr);
        else
          sample_grid(M, j, k, x, y, wm, hm, noise_on && valid, nkey, gs);
        const int g0 = k ? P.f0 : 0, ng = k ? P.f1 : P.f0;
#pragma unroll
        for (int g = 0; g < kGridPad / 8; ++g)
          if (g < ng) {
            float v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = valid ? gs.acc[8 * g + e] : 0.f;
            if (F8) put_x8(W, P, row, g0 + g, v, 1.f / sa[0], false, am[0]);
            else put_x(W, P, row, g0 + g, v);
          }
      }
      struct Pe {
        float v[16];
        __device__ void operator()(int q, float t) { v[q] = t; }
      } pe;
      positional_encoding(x, y, 0, pe);
      float v[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = pe.v[e];
      if (F8) put_x8(W, P, row, P.gpe, v, 1.f / sa[0], false, am[0]);
      else put_x(W, P, row, P.gpe, v);
#pragma unroll
      for (int e = 0; e < 4; ++e) v[e] = pe.v[8 + e];
      v[4] = tb->lodn[m];
      v[5] = 0.f;
      v[6] = v[7] = 1.f;
      if (F8) put_x8(W, P, row, P.gpe + 1, v, 1.f / sa[0], true, am[0]);
      else put_x(W, P, row, P.gpe + 1, v);
      const float zz[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      for (int g = P.gpe + 2; g < P.k_int / 8; ++g) {
        if (F8) put_x8(W, P, row, g, zz, 1.f, false, am[0]);
        else put_x(W, P, row, g, zz);
      }
      // the E4M3 tile's K padding up to a multiple of 32 inputs
      if (F8)
        for (int g = P.k_int / 8; g < P.k8 / 8; ++g)
          *reinterpret_cast<uint2*>(W + P.H1 + tc::canon_chunk(row, g >> 1, kRows) + (g & 1) * 8) =
              make_uint2(0u, 0u);
    }
    if (A.target)
      *reinterpret_cast<uint4*>(W + P.DZ3 + tc::canon_chunk(row, 1, kRows)) =
          make_uint4(tw[0], tw[1], tw[2], tw[3]);
    tc::fence_proxy_async();
    tc::bar_sync(bar_id, kRows);

    // ---- layer 1 -----------------------------------------------------------------
    if (row == 0) {
      tc::fence_after_sync();
      if (F8) {
        issue_kmajor_f8(tD, sW + P.H1, lbo_a, sbase + P.w1_8, lbo64, P.k8 / 32, id64);
      } else {
        issue_kmajor(tD, sW + P.X, lbo_a, sbase + P.w1, lbo64, P.k_int / 16, id64, 0);
        for (int s = 0; s < P.k_int / 16; ++s)
          tc::mma_f16(tD, tc::smem_desc(sW + xlo_group(P, 2 * s), lbo_a, 128),
                      tc::smem_desc(sbase + P.w1 + 2 * s * lbo64, lbo64, 128), id64, 1);
      }
      tc::mma_commit(bar);
    }
    if (!wait_phase(bar, phase, bar_id)) { aborted = true; break; }
    tc::fence_after_sync();
    if (F8)
      hidden_forward_f8<ACT>(tD + lane, sa[0] * sw[0], reinterpret_cast<const float*>(sm + P.bf),
                             1.f / sa[1], W + P.H1, W + P.H2, W + P.G1, row, am[1]);
    else
      hidden_forward<ACT>(tD + lane, W + P.H1, W + P.G1, W + P.H2, row);
    tc::fence_before_sync();
    tc::fence_proxy_async();
    tc::bar_sync(bar_id, kRows);

    // ---- layer 2 -----------------------------------------------------------------
    if (row == 0) {
      tc::fence_after_sync();
      if (F8) {
        issue_kmajor_f8(tD, sW + P.H2, lbo_a, sbase + P.w2_8, lbo64, 2, id64);
      } else {
        issue_kmajor(tD, sW + P.H1, lbo_a, sbase + P.w2, lbo64, 4, id64, 0);
        issue_kmajor(tD, sW + P.H2, lbo_a, sbase + P.w2, lbo64, 4, id64, 1);
        issue_kmajor(tD, sW + P.ONEa, lbo_a, sbase + P.wb2, lbo64, 1, id64, 1);
      }
      tc::mma_commit(bar);
    }
    if (!wait_phase(bar, phase, bar_id)) { aborted = true; break; }
    tc::fence_after_sync();
    if (F8)
      hidden_forward_f8<ACT>(tD + lane, sa[1] * sw[1],
                             reinterpret_cast<const float*>(sm + P.bf) + kHidden, 1.f / sa[2],
                             W + P.H2, W + P.S8, W + P.G2, row, am[2]);
    else
      hidden_forward<ACT>(tD + lane, W + P.H2, W + P.G2, P.h3 ? W + P.H3 : nullptr, row);
    tc::fence_before_sync();
    tc::fence_proxy_async();
    tc::bar_sync(bar_id, kRows);

    // ---- third hidden layer (Sec. 4.4) -------------------------------------------
    if (P.h3) {
      if (row == 0) {
        tc::fence_after_sync();
        issue_kmajor(tD, sW + P.H2, lbo_a, sbase + P.wh, lbo64, 4, id64, 0);
        issue_kmajor(tD, sW + P.H3, lbo_a, sbase + P.wh, lbo64, 4, id64, 1);
        issue_kmajor(tD, sW + P.ONEa, lbo_a, sbase + P.wbh, lbo64, 1, id64, 1);
        tc::mma_commit(bar);
      }
      if (!wait_phase(bar, phase, bar_id)) { aborted = true; break; }
      tc::fence_after_sync();
      hidden_forward<ACT>(tD + lane, W + P.H3, W + P.G3, nullptr, row);
      tc::fence_before_sync();
      tc::fence_proxy_async();
      tc::bar_sync(bar_id, kRows);
    }

    // ---- layer 3, loss, dZ3 ----------------------------------------------------
    if (row == 0) {
      tc::fence_after_sync();
      if (F8) {
        issue_kmajor_f8(tD, sW + P.S8, lbo_a, sbase + P.w3_8, lbo16, 2, id16);
      } else {
        issue_kmajor(tD, sW + P.HL, lbo_a, sbase + P.w3, lbo16, 4, id16, 0);
        issue_kmajor(tD, sW + P.ONEa, lbo_a, sbase + P.wb3, lbo16, 1, id16, 1);
      }
      tc::mma_commit(bar);
    }
    if (!wait_phase(bar, phase, bar_id)) { aborted = true; break; }
    tc::fence_after_sync();
    {
      float zv[16];
      tc::tmem_ld16(tD + lane, zv);
      tc::tmem_ld_wait();
      if (F8) {
        const float* b3 = reinterpret_cast<const float*>(sm + P.bf) + 2 * kHidden;
#pragma unroll
        for (int c = 0; c < kN3; ++c) zv[c] = fmaf(zv[c], sa[2] * sw[2], b3[c]);
      }
      // the target texel (loss mode) or the upstream gradient row (dout mode)
      float tgt[kN3];
      if (A.target) {
        const uint4 t4 = *reinterpret_cast<const uint4*>(W + P.DZ3 + tc::canon_chunk(row, 1, kRows));
        const uint32_t tv[4] = {t4.x, t4.y, t4.z, t4.w};
#pragma unroll
        for (int c = 0; c < kN3; ++c) tgt[c] = (float)((tv[c >> 2] >> (8 * (c & 3))) & 0xFFu) * (1.f / 255.f);
      } else {
#pragma unroll
        for (int c = 0; c < kN3; ++c) tgt[c] = (valid && c < C) ? A.dout[i * C + c] : 0.f;
      }
      float d[16];
#pragma unroll
      for (int c = 0; c < kN3; ++c) {
        float g = 0.f;
        if (valid && c < C) {
          // sigmoid; the fast division is within 2 ulp
          const float yc = M.out_act == NTC_OUT_IDENTITY ? zv[c] : __fdividef(1.f, 1.f + __expf(-zv[c]));
          if (A.target) {
            const float e = yc - tgt[c];
            loss_acc = fmaf(e, e, loss_acc);
            g = M.out_act == NTC_OUT_IDENTITY ? 2.f * e : 2.f * e * yc * (1.f - yc);
          } else {
            const float d = tgt[c] * dscale;
            g = M.out_act == NTC_OUT_IDENTITY ? d : d * yc * (1.f - yc);
          }
        }
        d[c] = g;
      }
      float v0[8], v1[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) { v0[e] = d[e]; v1[e] = d[8 + e]; }
      put_chunk(W + P.DZ3, row, 0, v0);
      put_chunk(W + P.DZ3, row, 1, v1);
    }
    tc::fence_before_sync();
    tc::fence_proxy_async();
    tc::bar_sync(bar_id, kRows);

    // ---- dHL = dZ3 W3; [dW3^T; db3] += [HL^T; 1] dZ3; then dZL over HL -------
    if (row == 0) {
      tc::fence_after_sync();
      issue_kmn(tD, sW + P.DZ3, lbo_a, sbase + P.w3, (kN3 / 8) * 128, 1, id64 | idb);
      issue_mnmajor(tW3, sW + P.HL, sW + P.DZ3, id_w3, 1);
      tc::mma_commit(bar);
    }
    if (!wait_phase(bar, phase, bar_id)) { aborted = true; break; }
    tc::fence_after_sync();
    hidden_backward<ACT, F8>(tD + lane, W + (P.h3 ? P.G3 : P.G2), W + P.HL, row, sw[2]);
    tc::fence_before_sync();
    tc::fence_proxy_async();
    tc::bar_sync(bar_id, kRows);

    // ---- third layer: dH2 = dZh Wh; [dWh dbh] += dZh^T [H2 | 1]; dZ2 over H2 --
    if (P.h3) {
      if (row == 0) {
        tc::fence_after_sync();
        issue_kmn(tD, sW + P.H3, lbo_a, sbase + P.wh, lbo64, 4, id64 | idb);
        issue_mnmajor(tWh, sW + P.H3, sW + P.H2, id_w2, 1);
        tc::mma_commit(bar);
      }
      if (!wait_phase(bar, phase, bar_id)) { aborted = true; break; }
      tc::fence_after_sync();
      hidden_backward<ACT, F8>(tD + lane, W + P.G2, W + P.H2, row);
      tc::fence_before_sync();
      tc::fence_proxy_async();
      tc::bar_sync(bar_id, kRows);
    }

    // ---- dH1 = dZ2 W2; [dW2 db2] += dZ2^T [H1 | 1]; then dZ1 over H1 ----------
    if (row == 0) {
      tc::fence_after_sync();
      issue_kmn(tD, sW + P.H2, lbo_a, sbase + P.w2, lbo64, 4, id64 | idb);
      issue_mnmajor(tW2, sW + P.H2, sW + P.H1, id_w2, 1);
      tc::mma_commit(bar);
    }
    if (!wait_phase(bar, phase, bar_id)) { aborted = true; break; }
    tc::fence_after_sync();
    hidden_backward<ACT, F8>(tD + lane, W + P.G1, W + P.H1, row, sw[1]);
    tc::fence_before_sync();
    tc::fence_proxy_async();
    tc::bar_sync(bar_id, kRows);

    // ---- dX = dZ1 W1; [dW1 db1] += dZ1^T X ------------------------------------
    if (row == 0) {
      tc::fence_after_sync();
      issue_kmn(tD, sW + P.H1, lbo_a, sbase + P.w1, lbo64, 4, id_dx);
      issue_mnmajor(tW1, sW + P.H1, sW + P.X, id_w1, 1);
      tc::mma_commit(bar);
    }
    if (!wait_phase(bar, phase, bar_id)) { aborted = true; break; }
    tc::fence_after_sync();
    const bool staged = LEARNED || M.c0 > kFastGridCh || M.c1 > kFastGridCh;
    const bool vec_scatter = A.grids && !staged && (M.c0 & 3) == 0 && (M.c1 & 3) == 0;
    // coherent texels (crop batches, given queries): merge runs of equal cells
    const bool merge = A.crops || A.uvl;
    // the staged form of the coalesced scatter: grids of 4k <= 16 channels
    // (learned G0) and room for the per-warp tap tables past the 128 rows
    const bool vec_staged = A.grids && staged && (M.c0 & 3) == 0 && M.c0 <= kFastGridCh &&
                            (M.c1 & 3) == 0 && M.c1 <= kFastGridCh &&
                            P.wg_bytes >= (uint32_t)(kRows * kDxStride * 4 + 4 * 32 * kScatMeta);
    if (A.grids && staged) {
      // dX row -> this thread's staging row (the operand tiles are free now),
      // then G0 per tap slot (weight 1; learned interpolation) or through
      // the bilinear taps, and G1 through the bilinear taps
      float* dxs = reinterpret_cast<float*>(W) + row * kDxStride;
      for (int cb = 0; cb < P.dx_n; cb += 16) {
        float v[16];
        tc::tmem_ld16(tD + lane + cb, v);
        tc::tmem_ld_wait();
#pragma unroll
        for (int q = 0; q < 4; ++q)
          *reinterpret_cast<float4*>(dxs + cb + 4 * q) =
              make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      }
      if (vec_staged) {
        // the coalesced scatter below over the staging rows: each warp puts
        // its texels' 8 (grid, tap) cell addresses and weights past the
        // 128 rows, lane j then adds grid j / 16, tap (j / 4) % 4, channels
        // 4 (j % 4) .. +3 texel by texel, once per run of equal cells
        const int ln = tid & 31, wq = warp & 3;
        uint8_t* mbase = W + kRows * kDxStride * 4 + wq * 32 * kScatMeta;
        {
          float* ga[8];
          float wt[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) { ga[e] = nullptr; wt[e] = 0.f; }
          if (valid) {
            const int j = tb->level[m];
            const int wm = tb->wm[m], hm = tb->hm[m];
            const ntc_level& L = M.lv[j];
            const float gsc = F8 ? gscale * sw[0] : gscale;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
              float* g = k ? A.g.grid1[j] : A.g.grid0[j];
              if (!g) continue;
              const int c = k ? M.c1 : M.c0;
              const Taps t = bilinear_taps(x, y, wm, hm, k ? L.g1_w : L.g0_w, k ? L.g1_h : L.g0_h);
#pragma unroll
              for (int tp = 0; tp < 4; ++tp) {
                ga[4 * k + tp] = g + (size_t)t.cell[tp] * c;
                wt[4 * k + tp] = (LEARNED && k == 0 ? 1.f : t.w[tp]) * gsc;
              }
            }
          }
          uint4* mq = reinterpret_cast<uint4*>(mbase + ln * kScatMeta);
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const uint64_t a0 = reinterpret_cast<uint64_t>(ga[2 * e]), a1 = reinterpret_cast<uint64_t>(ga[2 * e + 1]);
            mq[e] = make_uint4((uint32_t)a0, (uint32_t)(a0 >> 32), (uint32_t)a1, (uint32_t)(a1 >> 32));
          }
          mq[4] = make_uint4(__float_as_uint(wt[0]), __float_as_uint(wt[1]), __float_as_uint(wt[2]), __float_as_uint(wt[3]));
          mq[5] = make_uint4(__float_as_uint(wt[4]), __float_as_uint(wt[5]), __float_as_uint(wt[6]), __float_as_uint(wt[7]));
        }
        __syncwarp();
        const int k = ln >> 4, slot = ln >> 2, q = ln & 3;
        if (4 * q < (k ? M.c1 : M.c0)) {
          const int col = (k ? 8 * P.f0 : (LEARNED ? ((ln >> 2) & 3) * M.c0 : 0)) + 4 * q;
          const float* dx0 = reinterpret_cast<const float*>(W) + (32 * wq) * kDxStride + col;
          if (merge) scatter_lane<true>(mbase, dx0, kDxStride, slot, q);
          else scatter_lane<false>(mbase, dx0, kDxStride, slot, q);
        }
      } else if (valid) {
        const int j = tb->level[m];
        const int wm = tb->wm[m], hm = tb->hm[m];
        const ntc_level& L = M.lv[j];
        if (float* g = A.g.grid0[j])
          scatter_taps(g, M.c0, bilinear_taps(x, y, wm, hm, L.g0_w, L.g0_h), dxs,
                       LEARNED ? M.c0 : 0, !LEARNED, F8 ? gscale * sw[0] : gscale);
        if (float* g = A.g.grid1[j])
          scatter_taps(g, M.c1, bilinear_taps(x, y, wm, hm, L.g1_w, L.g1_h), dxs + 8 * P.f0, 0,
                       true, F8 ? gscale * sw[0] : gscale);
      }
      // the staging rows ran over the constant-one tiles: once every row has
      // been read, each thread writes its row's chunks back
      tc::bar_sync(bar_id, kRows);
      const uint4 one = make_uint4(tc::pack_f16x2(1.f, 1.f), 0u, 0u, 0u);
      *reinterpret_cast<uint4*>(W + P.ONEa + tc::canon_chunk(row, 0, kRows)) = one;
      *reinterpret_cast<uint4*>(W + P.ONEa + tc::canon_chunk(row, 1, kRows)) = make_uint4(0, 0, 0, 0);
      *reinterpret_cast<uint4*>(W + P.ONEb + tc::canon_chunk(row, 0, kRows)) = one;
      if (P.h3) {
        *reinterpret_cast<uint4*>(W + P.ONEc + tc::canon_chunk(row, 0, kRows)) = one;
        *reinterpret_cast<uint4*>(W + P.ONEc + tc::canon_chunk(row, 1, kRows)) = make_uint4(0, 0, 0, 0);
      }
    } else if (vec_scatter) {
      // Coalesced scatter (grids of 4k <= 16 channels): each warp stages
      // its 32 texels' dX rows, cell addresses and tap weights in its 8 KB
      // of the freed operand tiles, then adds them texel by texel with lane
      // j taking grid j / 16, tap (j / 4) % 4 and channels 4 (j % 4) .. +3.
      // The four lanes of a tap write 16 consecutive channels of one cell,
      // so one warp instruction touches 8 cell rows instead of 32, and a
      // lane whose consecutive texels share the cell reduces once per run.
      const int ln = tid & 31;
      uint8_t* ws = W + (warp & 3) * kScatWarp;
      float* dxr = reinterpret_cast<float*>(ws) + ln * kScatDx;
      uint8_t* mr = ws + 32 * kScatDx * 4 + ln * kScatMeta;
#pragma unroll
      for (int cb = 0; cb < 32; cb += 16) {
        float v[16];
        tc::tmem_ld16(tD + lane + cb, v);
        tc::tmem_ld_wait();
#pragma unroll
        for (int q = 0; q < 4; ++q)
          *reinterpret_cast<float4*>(dxr + cb + 4 * q) =
              make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      }
      {
        float* ga[8];
        float wt[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) { ga[e] = nullptr; wt[e] = 0.f; }
        if (valid) {
          const int j = tb->level[m];
          const int wm = tb->wm[m], hm = tb->hm[m];
          const ntc_level& L = M.lv[j];
          const float gsc = F8 ? gscale * sw[0] : gscale;
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            float* g = k ? A.g.grid1[j] : A.g.grid0[j];
            if (!g) continue;
            const int c = k ? M.c1 : M.c0;
            const Taps t = bilinear_taps(x, y, wm, hm, k ? L.g1_w : L.g0_w, k ? L.g1_h : L.g0_h);
#pragma unroll
            for (int tp = 0; tp < 4; ++tp) {
              ga[4 * k + tp] = g + (size_t)t.cell[tp] * c;
              wt[4 * k + tp] = t.w[tp] * gsc;
            }
          }
        }
        uint4* mq = reinterpret_cast<uint4*>(mr);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const uint64_t a0 = reinterpret_cast<uint64_t>(ga[2 * e]), a1 = reinterpret_cast<uint64_t>(ga[2 * e + 1]);
          mq[e] = make_uint4((uint32_t)a0, (uint32_t)(a0 >> 32), (uint32_t)a1, (uint32_t)(a1 >> 32));
        }
        mq[4] = make_uint4(__float_as_uint(wt[0]), __float_as_uint(wt[1]), __float_as_uint(wt[2]), __float_as_uint(wt[3]));
        mq[5] = make_uint4(__float_as_uint(wt[4]), __float_as_uint(wt[5]), __float_as_uint(wt[6]), __float_as_uint(wt[7]));
      }
      __syncwarp();
      {
        const int k = ln >> 4, slot = ln >> 2, q = ln & 3;
        const int col = (k ? 8 * P.f0 : 0) + 4 * q;
        if (4 * q < (k ? M.c1 : M.c0)) {
          const float* dx0 = reinterpret_cast<const float*>(ws) + col;
          const uint8_t* m0 = ws + 32 * kScatDx * 4;
          if (merge) scatter_lane<true>(m0, dx0, kScatDx, slot, q);
          else scatter_lane<false>(m0, dx0, kScatDx, slot, q);
        }
      }
      // the staging ran over ONEa: once every warp of the pipeline is done
      // with its rows, each thread writes its row's chunks back
      tc::bar_sync(bar_id, kRows);
      const uint4 one = make_uint4(tc::pack_f16x2(1.f, 1.f), 0u, 0u, 0u);
      *reinterpret_cast<uint4*>(W + P.ONEa + tc::canon_chunk(row, 0, kRows)) = one;
      *reinterpret_cast<uint4*>(W + P.ONEa + tc::canon_chunk(row, 1, kRows)) = make_uint4(0, 0, 0, 0);
    } else if (A.grids) {
      // dX slots: G0 at columns 0.., G1 at 8 * f0.. (f0 is 1 or 2)
      float d[32], dg0[16], dg1[16];
      {
        float lo[16], hi[16];
        tc::tmem_ld16(tD + lane, lo);
        tc::tmem_ld16(tD + lane + 16, hi);
        tc::tmem_ld_wait();
#pragma unroll
        for (int e = 0; e < 16; ++e) { d[e] = lo[e]; d[16 + e] = hi[e]; }
      }
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        dg0[e] = d[e];
        dg1[e] = P.f0 == 1 ? d[8 + e] : d[16 + e];
      }
      if (valid) {
        const int j = tb->level[m];
        const int wm = tb->wm[m], hm = tb->hm[m];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const ntc_level& L = M.lv[j];
          float* g = k ? A.g.grid1[j] : A.g.grid0[j];
          if (!g) continue;
          const int c = k ? M.c1 : M.c0;
          const Taps t = bilinear_taps(x, y, wm, hm, k ? L.g1_w : L.g0_w, k ? L.g1_h : L.g0_h);
#pragma unroll
          for (int tp = 0; tp < 4; ++tp) {
            const float wgt = t.w[tp] * (F8 ? gscale * sw[0] : gscale);
            float* gp = g + (size_t)t.cell[tp] * c;
            if ((c & 3) == 0) {
#pragma unroll
              for (int c4 = 0; c4 < 4; ++c4)
                if (4 * c4 < c) {
                  const float* d = k ? dg1 : dg0;
                  atomicAdd(reinterpret_cast<float4*>(gp) + c4,
                            make_float4(d[4 * c4] * wgt, d[4 * c4 + 1] * wgt, d[4 * c4 + 2] * wgt,
                                        d[4 * c4 + 3] * wgt));
                }
            } else {
#pragma unroll
              for (int ch = 0; ch < kFastGridCh; ++ch)
                if (ch < c) atomicAdd(gp + ch, (k ? dg1[ch] : dg0[ch]) * wgt);
            }
          }
        }
      }
    }
    tc::fence_before_sync();
    if (staged || vec_scatter) tc::fence_proxy_async();  // restored constants, read by the next tile's MMAs
    tc::bar_sync(bar_id, kRows);  // the next tile's features overwrite the operand tiles
  }

  // ---- every MMA of this pipeline has completed (bounded) ---------------------
  if (row == 0) {
    tc::fence_after_sync();
    tc::mma_commit(&fin[wg]);
    if (!tc::mbar_wait(&fin[wg], fin_phase, kWaitLimit)) aborted = true;
    if (aborted) abort_any = 1;
  }
  fin_phase ^= 1;
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();

  // ---- flush the CTA's weight gradients ----------------------------------------
  const float gs = gscale;
  const int wq = warp & 3;  // lane quarter of this warp: rows 32 wq .. 32 wq + 31
  const int r = 32 * wq + (tid & 31);
  if (!abort_any && (BATCHED || (int64_t)blockIdx.x * NWG < t_hi)) {
    // flush jobs 0 dW1, 1 dW2, 2 dW3, 3 dWh, one warpgroup each (round robin)
    for (int job = wg; job < (P.h3 ? 4 : 3); job += NWG) {
      if (job == 0 && wq < 2) {
        // [dW1 db1]: row r, X columns (the head constant-one slot gives db1
        // r); four slots that map to four consecutive, 16-byte aligned user
        // columns leave as one vector reduction
        float* gw = A.g.w[0];
#pragma unroll 1
        for (int cb = 0; cb < P.k_int; cb += 16) {
          float v[16];
          tc::tmem_ld16(tW1 + lane + cb, v);
          tc::tmem_ld_wait();
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            int uc[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) uc[e] = slot_column(M, P, cb + 4 * q + e);
            const int64_t o = (int64_t)r * M.k_in + uc[0];
            if (gw && uc[0] >= 0 && uc[1] == uc[0] + 1 && uc[2] == uc[0] + 2 && uc[3] == uc[0] + 3 &&
                (reinterpret_cast<uintptr_t>(gw + o) & 15) == 0) {
              const float f = gs * sa[0];
              atomicAdd(reinterpret_cast<float4*>(gw + o),
                        make_float4(v[4 * q] * f, v[4 * q + 1] * f, v[4 * q + 2] * f, v[4 * q + 3] * f));
            } else {
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                if (uc[e] >= 0 && gw) atomicAdd(gw + r * M.k_in + uc[e], v[4 * q + e] * gs * sa[0]);
                else if (uc[e] == -2 && A.g.b[0]) atomicAdd(A.g.b[0] + r, v[4 * q + e] * gs);
              }
            }
          }
        }
      } else if ((job == 1 || job == 3) && wq < 2) {
        // [dW2 db2] / [dWh dbh]: row r, input columns 0..63 (vector
        // reductions where the row is 16-byte aligned), the ones column 64
        // gives the bias
        const uint32_t ta = job == 1 ? tW2 : tWh;
        float* gw = job == 1 ? A.g.w[1] : A.g.w_h3;
        float* gb = job == 1 ? A.g.b[1] : A.g.b_h3;
        const float gsw = gs * (job == 1 ? sa[1] : 1.f);  // FP8: H1 was held in units of s_a1
        const bool vec = gw && (reinterpret_cast<uintptr_t>(gw + r * kHidden) & 15) == 0;
#pragma unroll 1
        for (int cb = 0; cb < kHidden + 16; cb += 16) {
          float v[16];
          tc::tmem_ld16(ta + lane + cb, v);
          tc::tmem_ld_wait();
          if (cb < kHidden && vec) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
              atomicAdd(reinterpret_cast<float4*>(gw + r * kHidden + cb) + q,
                        make_float4(v[4 * q] * gsw, v[4 * q + 1] * gsw, v[4 * q + 2] * gsw,
                                    v[4 * q + 3] * gsw));
          } else {
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              const int col = cb + e;
              if (col < kHidden && gw) atomicAdd(gw + r * kHidden + col, v[e] * gsw);
              else if (col == kHidden && gb) atomicAdd(gb + r, v[e] * gs);
            }
          }
        }
      } else if (job == 2 && wq < 3) {
        // [dW3^T; db3]: row r < 64 -> dW3[:, r]; row 64 -> db3
        float v[16];
        tc::tmem_ld16(tW3 + lane, v);
        tc::tmem_ld_wait();
#pragma unroll
        for (int c = 0; c < kN3; ++c) {
          if (c >= C) continue;
          if (r < kHidden && A.g.w[2]) atomicAdd(A.g.w[2] + c * kHidden + r, v[c] * gs * sa[2]);
          if (r == kHidden && A.g.b[2]) atomicAdd(A.g.b[2] + c, v[c] * gs);
        }
      }
    }
  }
  // FP8: the largest |input| of each layer, for the next step's scales
  if (F8) {
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      float v = am[l];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
      if ((tid & 31) == 0 && v > 0.f)
        atomicMax(reinterpret_cast<unsigned int*>(const_cast<float*>(M.scale)) + 6 + l,
                  __float_as_uint(v));
    }
  }
  // loss
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) loss_acc += __shfl_xor_sync(0xffffffffu, loss_acc, o);
  if ((tid & 31) == 0) red[warp] = loss_acc;
  tc::fence_before_sync();
  __syncthreads();
  if (tid == 0) {
    float s = 0.f;
    for (int w = 0; w < NWG * 4; ++w) s += red[w];
    if (A.loss) atomicAdd(A.loss, s * A.loss_scale);
    if (abort_any) atomicExch(status, NTC_ERR_TIMEOUT);
  }
  // the next material's staging overwrites the shared memory read above
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (!BATCHED || abort_any) break;
  ++seg;
  }  // materials

  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem_base, kCols);
  }
}

template <int ACT, bool LEARNED, int NWG, bool BATCHED, bool F8>
cudaError_t launch_t(const ntc_material& m, const BwdArgs& a, const TrainBatchDev* hb,
                     int64_t tiles, int k_lay, int dx_lay, cudaStream_t s) {
  const TPlan P(m.c0, m.c1, LEARNED, ACT == NTC_ACT_HARDGELU, NWG, m.hidden_layers == 3, k_lay,
                dx_lay, F8);
  const size_t smem = P.total;
  cudaError_t e = cudaFuncSetAttribute(train_tc_kernel<ACT, LEARNED, NWG, BATCHED, F8>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t ctas = (tiles + NWG - 1) / NWG;
  const int64_t cap = sm_count();
  const int grid = (int)(ctas < cap ? ctas : cap);
  train_tc_kernel<ACT, LEARNED, NWG, BATCHED, F8>
      <<<grid, kRows * NWG, smem, s>>>(m, a, hb, k_lay, dx_lay, status_word());
  return cudaGetLastError();
}

// Pipelines per CTA: the most (3, 2 or 1) whose tiles fit (0: none fits).
int pipelines_for(const ntc_material& m, int k_lay, int dx_lay) {
  const bool learned = m.interp0 == NTC_INTERP_LEARNED, gelu = m.act == NTC_ACT_HARDGELU;
  const bool f8 = m.precision == NTC_PREC_F8;
  for (int n = kMaxNWG; n >= 1; --n)
    if (TPlan(m.c0, m.c1, learned, gelu, n, m.hidden_layers == 3, k_lay, dx_lay, f8).fits())
      return n;
  return 0;
}
int train_pipelines(const ntc_material& m) { return pipelines_for(m, 0, 0); }

template <int ACT, bool LEARNED, bool BATCHED, bool F8>
cudaError_t launch_n(const ntc_material& m, const BwdArgs& a, const TrainBatchDev* hb,
                     int64_t tiles, int k_lay, int dx_lay, cudaStream_t s) {
  int np = pipelines_for(m, k_lay, dx_lay);
  if (a.pipelines > 0 && a.pipelines < np) np = a.pipelines;  // the autotuner's choice
  switch (np) {
    case 3: return launch_t<ACT, LEARNED, 3, BATCHED, F8>(m, a, hb, tiles, k_lay, dx_lay, s);
    case 2: return launch_t<ACT, LEARNED, 2, BATCHED, F8>(m, a, hb, tiles, k_lay, dx_lay, s);
    default: return launch_t<ACT, LEARNED, 1, BATCHED, F8>(m, a, hb, tiles, k_lay, dx_lay, s);
  }
}

template <bool BATCHED>
cudaError_t launch_class(const ntc_material& m, const BwdArgs& a, const TrainBatchDev* hb,
                         int64_t tiles, int k_lay, int dx_lay, cudaStream_t s) {
  const bool learned = m.interp0 == NTC_INTERP_LEARNED;
  if (m.act == NTC_ACT_HARDGELU)
    return learned ? launch_n<NTC_ACT_HARDGELU, true, BATCHED, false>(m, a, hb, tiles, k_lay, dx_lay, s)
                   : launch_n<NTC_ACT_HARDGELU, false, BATCHED, false>(m, a, hb, tiles, k_lay, dx_lay, s);
  return learned ? launch_n<NTC_ACT_RELU, true, BATCHED, false>(m, a, hb, tiles, k_lay, dx_lay, s)
                 : launch_n<NTC_ACT_RELU, false, BATCHED, false>(m, a, hb, tiles, k_lay, dx_lay, s);
}

// The FP8-E4M3 form (single material, bilinear G0).
inline cudaError_t launch_class_f8(const ntc_material& m, const BwdArgs& a, int64_t tiles,
                                   cudaStream_t s) {
  if (m.act == NTC_ACT_HARDGELU)
    return launch_n<NTC_ACT_HARDGELU, false, false, true>(m, a, nullptr, tiles, 0, 0, s);
  return launch_n<NTC_ACT_RELU, false, false, true>(m, a, nullptr, tiles, 0, 0, s);
}

}  // namespace
}  // namespace ntc
