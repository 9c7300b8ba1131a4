// Tensor-core (tcgen05) random-access decode, FP16 or FP8-E4M3 operands with
// FP32 accumulation in TMEM (Sec. 4.3-4.4, 5.2-5.3).
//
// Persistent CTAs of 128 threads; a tile is 128 MLP rows (one query per row,
// or for trilinear filtering 16 queries x 8 texel taps).  Per tile:
//   1. every thread gathers and dequantises its row's latent features, adds
//      the positional encoding and LOD, and writes the row into the A tile
//      (canonical K-major layout in shared memory);
//   2. one thread issues layer 1 (M=128, N=64) into TMEM and commits to an
//      mbarrier; every thread waits, loads its accumulator row with
//      tcgen05.ld, applies the activation and writes the hidden row back as
//      the next A tile;
//   3. likewise layer 2 (N=64) and layer 3 (N=16), whose epilogue applies the
//      output activation and stores the texel.
// Several CTAs per SM overlap one CTA's gathers with another's MMAs.
//
// The MLP input row is stored in an internal slot order that keeps every
// 8-slot group register-resident: [G0 | pad][G1 | pad][12 PE, LOD, 0, 1, 1]
// [0 ...]; W1's columns are permuted to match when staged.  For FP16 the
// biases ride on the tensor core: layer 1 through two constant-one slots
// (bias split into an FP16 head and tail), layers 2 and 3 through one extra
// K=16 block of a constant tile.  For FP8 each layer's epilogue applies
// (s_w * s_a) * acc + b in FP32.
#include "ntc_device.cuh"
#include "ntc_internal.h"
#include "tc_ptx.cuh"

namespace ntc {

namespace {

constexpr int kRows = 128;
constexpr int kN3 = 16;
constexpr uint32_t kWaitLimit = 1u << 22;

template <bool F8>
struct Cfg {
  static constexpr int EB = F8 ? 1 : 2;       // operand bytes
  static constexpr int KSTEP = F8 ? 32 : 16;  // K per MMA instruction
};

// Shared memory plan (bytes from a 1024-aligned base).
struct Plan {
  int k_int;                     // internal MLP input width
  int ng0, ng1;                  // 8-slot groups of G0 / G1
  uint32_t x, h, cst, w1, w2, w3, wb2, wb3, bias, total;
  __host__ __device__ Plan(int c0, int c1, bool f8) {
    const int eb = f8 ? 1 : 2, kstep = f8 ? 32 : 16;
    ng0 = (c0 + 7) / 8;
    ng1 = (c1 + 7) / 8;
    const int slots = 8 * (ng0 + ng1 + 2);
    k_int = (slots + kstep - 1) / kstep * kstep;
    uint32_t o = 0;
    x = o;   o += kRows * k_int * eb;      // A: input rows
    h = o;   o += kRows * kHidden * eb;    // A: hidden rows
    cst = o; o += f8 ? 0 : kRows * 16 * 2; // A: constant-one block (FP16)
    w1 = o;  o += kHidden * k_int * eb;    // B: W1 (internal slot order)
    w2 = o;  o += kHidden * kHidden * eb;  // B: W2
    w3 = o;  o += kN3 * kHidden * eb;      // B: W3 (rows >= C zero)
    wb2 = o; o += f8 ? 0 : kHidden * 16 * 2;  // B: bias block of layer 2 (FP16)
    wb3 = o; o += f8 ? 0 : kN3 * 16 * 2;      // B: bias block of layer 3 (FP16)
    bias = o; o += (2 * kHidden + kN3) * 4;   // FP32 biases (FP8 epilogues)
    total = o;
  }
};

struct Smem {
  uint64_t mbar;
  uint32_t tmem;
  int abort;
};

// User column of internal input slot s: >= 0 a W1 column, -1 zero padding,
// -2 / -3 the constant-one slots carrying the FP16 bias head / tail.
__device__ __forceinline__ int w1_column(const ntc_material& M, const Plan& P, int s, bool f8) {
  const int g0 = 8 * P.ng0, g1 = 8 * P.ng1;
  if (s < g0) return s < M.c0 ? s : -1;
  if (s < g0 + g1) return (s - g0) < M.c1 ? M.c0 + (s - g0) : -1;
  const int e = s - g0 - g1;
  if (e < 13) return M.c0 + M.c1 + e;
  if (!f8 && e == 14) return -2;
  if (!f8 && e == 15) return -3;
  return -1;
}

// Split an FP32 bias into an FP16 head and tail: b ~ head + tail.
__device__ __forceinline__ void split_bias(float b, __half& hd, __half& tl) {
  hd = __float2half_rn(b);
  tl = __float2half_rn(b - __half2float(hd));
}

template <bool F8>
__device__ void stage_weights_tc(const ntc_material& M, const Plan& P, uint8_t* sm) {
  const int tid = threadIdx.x, nt = blockDim.x;
  constexpr int EB = Cfg<F8>::EB;
  // W1 [64][k_int] in internal slot order
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
  // W2 [64][64], W3 [16][64]
  for (int i = tid; i < kHidden * kHidden; i += nt) {
    const int n = i / kHidden, k = i - n * kHidden;
    const uint32_t off = P.w2 + tc::canon_offset(n, k, kHidden, EB);
    if (F8) sm[off] = static_cast<const uint8_t*>(M.w[1])[i];
    else *reinterpret_cast<__half*>(sm + off) = static_cast<const __half*>(M.w[1])[i];
  }
  for (int i = tid; i < kN3 * kHidden; i += nt) {
    const int n = i / kHidden, k = i - n * kHidden;
    const uint32_t off = P.w3 + tc::canon_offset(n, k, kN3, EB);
    const bool live = n < M.channels;
    if (F8) sm[off] = live ? static_cast<const uint8_t*>(M.w[2])[i] : 0;
    else *reinterpret_cast<__half*>(sm + off) =
        live ? static_cast<const __half*>(M.w[2])[i] : __float2half_rn(0.f);
  }
  float* bias = reinterpret_cast<float*>(sm + P.bias);
  for (int i = tid; i < kHidden; i += nt) {
    bias[i] = M.b[0][i];
    bias[kHidden + i] = M.b[1][i];
  }
  for (int i = tid; i < kN3; i += nt) bias[2 * kHidden + i] = i < M.channels ? M.b[2][i] : 0.f;
  if (!F8) {
    // constant-one A block [128][16]: columns 0 and 1 = 1; bias B blocks
    for (int i = tid; i < kRows * 16; i += nt) {
      const int r = i / 16, k = i - r * 16;
      *reinterpret_cast<__half*>(sm + P.cst + tc::canon_offset(r, k, kRows, 2)) =
          __float2half_rn(k < 2 ? 1.f : 0.f);
    }
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
      if (n < M.channels) split_bias(M.b[2][n], hd, tl);
      *reinterpret_cast<__half*>(sm + P.wb3 + tc::canon_offset(n, k, kN3, 2)) =
          k == 0 ? hd : (k == 1 ? tl : __float2half_rn(0.f));
    }
  }
}

// Write one 8-slot group of a row: FP16 -> one 16-byte chunk; FP8 -> 8 bytes
// (scaled by `inv_scale` before rounding to E4M3).
template <bool F8>
__device__ __forceinline__ void put_group(uint8_t* tile, int row, int g, const float (&v)[8],
                                          float inv_scale) {
  if (F8) {
    uint2 w;
    w.x = tc::pack_e4m3x2(v[0] * inv_scale, v[1] * inv_scale) |
          (tc::pack_e4m3x2(v[2] * inv_scale, v[3] * inv_scale) << 16);
    w.y = tc::pack_e4m3x2(v[4] * inv_scale, v[5] * inv_scale) |
          (tc::pack_e4m3x2(v[6] * inv_scale, v[7] * inv_scale) << 16);
    *reinterpret_cast<uint2*>(tile + tc::canon_offset(row, 8 * g, kRows, 1)) = w;
  } else {
    uint4 w;
    w.x = tc::pack_f16x2(v[0], v[1]);
    w.y = tc::pack_f16x2(v[2], v[3]);
    w.z = tc::pack_f16x2(v[4], v[5]);
    w.w = tc::pack_f16x2(v[6], v[7]);
    *reinterpret_cast<uint4*>(tile + tc::canon_chunk(row, g, kRows)) = w;
  }
}

struct PeSink {
  float v[16];
  __device__ __forceinline__ void operator()(int i, float x) { v[i] = x; }
};

// Gather, dequantise and encode one texel into the A tile (internal order).
template <bool F8>
__device__ __forceinline__ void feature_row(const ntc_material& M, const Plan& P, uint8_t* tile,
                                            int row, int x, int y, int m, bool valid,
                                            float inv_sa) {
  const int groups = P.k_int / 8;
  if (!valid) {
    const float z[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int g = 0; g < groups; ++g) put_group<F8>(tile, row, g, z, 1.f);
    return;
  }
  const int j = level_of_mip(m, M.levels);
  const int wm = mip_dim(M.width, m), hm = mip_dim(M.height, m);
  GridSample gs;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    sample_grid(M, j, k, x, y, wm, hm, false, 0, gs);
    const int base = k ? P.ng0 : 0, ng = k ? P.ng1 : P.ng0;
#pragma unroll
    for (int g = 0; g < 2; ++g)
      if (g < ng) {
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = gs.acc[8 * g + e];
        put_group<F8>(tile, row, base + g, v, inv_sa);
      }
  }
  PeSink pe;
  positional_encoding(x, y, 0, pe);
  pe.v[12] = M.mips > 1 ? (float)m / (float)(M.mips - 1) : 0.f;
  pe.v[13] = 0.f;
  pe.v[14] = F8 ? 0.f : 1.f;
  pe.v[15] = F8 ? 0.f : 1.f;
  const int gp = P.ng0 + P.ng1;
  float v[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) v[e] = pe.v[e];
  put_group<F8>(tile, row, gp, v, inv_sa);
#pragma unroll
  for (int e = 0; e < 8; ++e) v[e] = pe.v[8 + e];
  if (F8) {
    // the constant-one slots are FP16-only; scale the LOD group like the rest
    put_group<F8>(tile, row, gp + 1, v, inv_sa);
  } else {
    put_group<F8>(tile, row, gp + 1, v, 1.f);
  }
  const float z[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int g = gp + 2; g < groups; ++g) put_group<F8>(tile, row, g, z, 1.f);
}

// Layer epilogue for a 64-wide hidden layer: TMEM row -> activation -> next
// A tile.  FP8: (s_w s_a) acc + b, activation, scale by 1/s_a(next), E4M3.
template <bool F8>
__device__ __forceinline__ void hidden_epilogue(uint32_t tmem_row, uint8_t* htile, int row, int act,
                                                const float* bias, float scale, float inv_next) {
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    float a[16], b[16];
    tc::tmem_ld16(tmem_row + 32 * half, a);
    tc::tmem_ld16(tmem_row + 32 * half + 16, b);
    tc::tmem_ld_wait();
    float v[32];
#pragma unroll
    for (int i = 0; i < 16; ++i) { v[i] = a[i]; v[16 + i] = b[i]; }
    if (F8) {
#pragma unroll
      for (int i = 0; i < 32; ++i) v[i] = fmaf(v[i], scale, bias[32 * half + i]);
    }
    if (!F8 && act == NTC_ACT_RELU) {
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        uint4 w;
        w.x = tc::pack_f16x2_relu(v[8 * g + 0], v[8 * g + 1]);
        w.y = tc::pack_f16x2_relu(v[8 * g + 2], v[8 * g + 3]);
        w.z = tc::pack_f16x2_relu(v[8 * g + 4], v[8 * g + 5]);
        w.w = tc::pack_f16x2_relu(v[8 * g + 6], v[8 * g + 7]);
        *reinterpret_cast<uint4*>(htile + tc::canon_chunk(row, 4 * half + g, kRows)) = w;
      }
    } else {
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        float e[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) e[i] = act_fwd(act, v[8 * g + i]);
        put_group<F8>(htile, row, 4 * half + g, e, inv_next);
      }
    }
  }
}

template <bool F8>
__global__ void __launch_bounds__(kRows) decode_tc_kernel(const ntc_material M,
                                                          const float* __restrict__ uvl, int64_t n,
                                                          void* __restrict__ out, int out_dtype,
                                                          int filter, int* status) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ Smem ctl;
  const Plan P(M.c0, M.c1, F8);
  uint8_t* sm = smem_raw;
  const int tid = threadIdx.x, warp = tid >> 5;
  constexpr int KSTEP = Cfg<F8>::KSTEP;

  stage_weights_tc<F8>(M, P, sm);
  if (warp == 0) {
    tc::tmem_alloc(&ctl.tmem, 64);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&ctl.mbar, 1);
    tc::fence_mbar_init();
    ctl.abort = 0;
  }
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = ctl.tmem;
  const uint32_t tmem_row = tmem + ((uint32_t)(warp * 32) << 16);

  // per-layer scales (FP8): acc * s_w * s_a + b; inputs scaled by 1 / s_a
  float sc[3] = {1.f, 1.f, 1.f}, inv_sa[3] = {1.f, 1.f, 1.f};
  if (F8) {
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      sc[l] = M.scale[l] * M.scale[3 + l];
      inv_sa[l] = 1.f / M.scale[3 + l];
    }
  }
  const float* bias = reinterpret_cast<const float*>(sm + P.bias);
  const uint32_t sbase = tc::smem_u32(sm);
  const uint32_t lbo_a = (kRows / 8) * 128, lbo_w = (kHidden / 8) * 128, lbo_w3 = (kN3 / 8) * 128;
  constexpr uint32_t id64 = tc::idesc(kRows, kHidden), id16 = tc::idesc(kRows, kN3);

  const bool tri = filter == NTC_FILTER_TRILINEAR;
  const int per_tile = tri ? kRows / 8 : kRows;
  const int64_t ntiles = (n + per_tile - 1) / per_tile;
  uint32_t phase = 0;
  const int C = M.channels;

  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    // ---- 1. features ---------------------------------------------------------
    const int64_t q = tri ? tile * per_tile + (tid >> 3) : tile * per_tile + tid;
    const bool valid = q < n;
    float wtap = 0.f;
    int x = 0, yy = 0, m = 0;
    if (valid) {
      const float u = uvl[3 * q], v = uvl[3 * q + 1], l = uvl[3 * q + 2];
      if (!tri) {
        query_texel(M, u, v, l, x, yy, m);
      } else {
        const int tap = tid & 7, s = tap >> 2, dx = tap & 1, dy = (tap >> 1) & 1;
        const float lam = !(l >= 0.f) ? 0.f : fminf(l, (float)(M.mips - 1));
        const int m0 = min((int)floorf(lam), M.mips - 1);
        const int m1 = min(m0 + 1, M.mips - 1);
        const float t = lam - (float)m0;
        m = s ? m1 : m0;
        const float wl = s ? t : 1.f - t;
        const int wm = mip_dim(M.width, m), hm = mip_dim(M.height, m);
        const float px = u * (float)wm - 0.5f, py = v * (float)hm - 0.5f;
        const float fx0 = floorf(px), fy0 = floorf(py);
        const float fx = px - fx0, fy = py - fy0;
        x = (((int)fx0 + dx) % wm + wm) % wm;
        yy = (((int)fy0 + dy) % hm + hm) % hm;
        wtap = wl * (dx ? fx : 1.f - fx) * (dy ? fy : 1.f - fy);
      }
    }
    feature_row<F8>(M, P, sm + P.x, tid, x, yy, m, valid, inv_sa[0]);
    tc::fence_proxy_async();
    __syncthreads();

    // ---- 2. layer 1 ----------------------------------------------------------
    if (tid == 0) {
      tc::fence_after_sync();
      const int ksteps = P.k_int / KSTEP;
      for (int s = 0; s < ksteps; ++s) {
        const uint64_t a = tc::smem_desc(sbase + P.x + 2 * s * lbo_a, lbo_a, 128);
        const uint64_t b = tc::smem_desc(sbase + P.w1 + 2 * s * lbo_w, lbo_w, 128);
        if (F8) tc::mma_f8(tmem, a, b, id64, s > 0);
        else tc::mma_f16(tmem, a, b, id64, s > 0);
      }
      tc::mma_commit(&ctl.mbar);
    }
    bool ok = tc::mbar_wait(&ctl.mbar, phase, kWaitLimit);
    phase ^= 1;
    if (__syncthreads_or(!ok)) { ctl.abort = 1; break; }
    tc::fence_after_sync();
    hidden_epilogue<F8>(tmem_row, sm + P.h, tid, M.act, bias, sc[0], inv_sa[1]);
    tc::fence_before_sync();
    tc::fence_proxy_async();
    __syncthreads();

    // ---- 3. layer 2 ----------------------------------------------------------
    if (tid == 0) {
      tc::fence_after_sync();
      for (int s = 0; s < kHidden / KSTEP; ++s) {
        const uint64_t a = tc::smem_desc(sbase + P.h + 2 * s * lbo_a, lbo_a, 128);
        const uint64_t b = tc::smem_desc(sbase + P.w2 + 2 * s * lbo_w, lbo_w, 128);
        if (F8) tc::mma_f8(tmem, a, b, id64, s > 0);
        else tc::mma_f16(tmem, a, b, id64, s > 0);
      }
      if (!F8) {
        const uint64_t a = tc::smem_desc(sbase + P.cst, lbo_a, 128);
        const uint64_t b = tc::smem_desc(sbase + P.wb2, lbo_w, 128);
        tc::mma_f16(tmem, a, b, id64, 1);
      }
      tc::mma_commit(&ctl.mbar);
    }
    ok = tc::mbar_wait(&ctl.mbar, phase, kWaitLimit);
    phase ^= 1;
    if (__syncthreads_or(!ok)) { ctl.abort = 1; break; }
    tc::fence_after_sync();
    hidden_epilogue<F8>(tmem_row, sm + P.h, tid, M.act, bias + kHidden, sc[1], inv_sa[2]);
    tc::fence_before_sync();
    tc::fence_proxy_async();
    __syncthreads();

    // ---- 4. layer 3 + output ----------------------------------------------
    if (tid == 0) {
      tc::fence_after_sync();
      for (int s = 0; s < kHidden / KSTEP; ++s) {
        const uint64_t a = tc::smem_desc(sbase + P.h + 2 * s * lbo_a, lbo_a, 128);
        const uint64_t b = tc::smem_desc(sbase + P.w3 + 2 * s * lbo_w3, lbo_w3, 128);
        if (F8) tc::mma_f8(tmem, a, b, id16, s > 0);
        else tc::mma_f16(tmem, a, b, id16, s > 0);
      }
      if (!F8) {
        const uint64_t a = tc::smem_desc(sbase + P.cst, lbo_a, 128);
        const uint64_t b = tc::smem_desc(sbase + P.wb3, lbo_w3, 128);
        tc::mma_f16(tmem, a, b, id16, 1);
      }
      tc::mma_commit(&ctl.mbar);
    }
    ok = tc::mbar_wait(&ctl.mbar, phase, kWaitLimit);
    phase ^= 1;
    if (__syncthreads_or(!ok)) { ctl.abort = 1; break; }
    tc::fence_after_sync();
    float yv[16];
    tc::tmem_ld16(tmem_row, yv);
    tc::tmem_ld_wait();
    tc::fence_before_sync();
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      float z = yv[c];
      if (F8) z = fmaf(z, sc[2], bias[2 * kHidden + c]);
      yv[c] = out_fwd(M.out_act, z);
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
    const bool writer = valid && (!tri || (tid & 7) == 0);
    if (writer) {
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
  }

  tc::fence_before_sync();
  __syncthreads();
  if (tid == 0 && ctl.abort) atomicExch(status, NTC_ERR_TIMEOUT);
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, 64);
  }
}

template <bool F8>
cudaError_t launch_k(const ntc_material& m, const float* uvl, int64_t n, void* out, int out_dtype,
                     int filter, cudaStream_t s, int ctas_per_sm) {
  const Plan P(m.c0, m.c1, F8);
  const size_t smem = P.total;
  cudaError_t e = cudaFuncSetAttribute(decode_tc_kernel<F8>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, decode_tc_kernel<F8>, kRows, smem);
  if (e != cudaSuccess) return e;
  // TMEM: 64 columns per CTA, 512 per SM
  per_sm = per_sm > 8 ? 8 : per_sm;
  if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
  if (per_sm < 1) per_sm = 1;
  const int per_tile = filter == NTC_FILTER_TRILINEAR ? kRows / 8 : kRows;
  const int64_t tiles = (n + per_tile - 1) / per_tile;
  const int64_t cap = (int64_t)sm_count() * per_sm;
  const int grid = (int)(tiles < cap ? tiles : cap);
  decode_tc_kernel<F8><<<grid, kRows, smem, s>>>(m, uvl, n, out, out_dtype, filter, status_word());
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_decode_tc(const ntc_material& m, const float* uvl, int64_t n, void* out,
                             int out_dtype, int filter, cudaStream_t s, int ctas_per_sm) {
  if (n == 0) return cudaSuccess;
  if (m.precision == NTC_PREC_F16)
    return launch_k<false>(m, uvl, n, out, out_dtype, filter, s, ctas_per_sm);
  if (m.precision == NTC_PREC_F8)
    return launch_k<true>(m, uvl, n, out, out_dtype, filter, s, ctas_per_sm);
  return cudaErrorInvalidValue;
}

cudaError_t launch_backward_tc(const ntc_material&, const BwdArgs&, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace ntc
