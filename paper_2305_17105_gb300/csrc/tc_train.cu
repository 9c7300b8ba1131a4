// Tensor-core (tcgen05) fused forward + L2 loss + backward of the NTC
// optimisation step (Sec. 4.2, 4.5, 5.1), FP16 operands, FP32 accumulation.
//
// One persistent CTA per SM runs two warpgroup pipelines; a warpgroup owns a
// stream of tiles of 128 training texels (one per thread = one row = one
// TMEM lane).  Per tile, with every activation kept on chip:
//   forward   X -> Z1 = X W1^T (+b1) -> H1 = relu -> Z2 (+b2) -> H2 -> Z3 (+b3)
//             -> y = sigmoid, loss, dZ3 = 2 (y - t) y (1 - y)
//   backward  dH2 = dZ3 W3, dZ2 = dH2 * [H2 > 0], dH1 = dZ2 W2,
//             dZ1 = dH1 * [H1 > 0], dX = dZ1 W1 -> scatter-add into the grid
//             gradients through the bilinear taps (FP32 atomics)
//   weights   [dW1 db1; dW2 db2] += [dZ1^T; dZ2^T] [X | H1 | 1] and
//             [dW3^T; db3] += [H2^T; 1] dZ3, accumulated in TMEM over all of
//             the CTA's tiles and added to global memory once at the end.
// X, H1, H2, dZ1, dZ2, dZ3 are FP16 tiles in shared memory, stored one row
// per texel in the canonical K-major layout (8 x 16-byte core matrices, row
// group fastest).  The same bytes serve as K-major A operands of the forward
// and backward layers and, read with the MN-major descriptor mode (K = the
// 128 texels), as the operands of the weight-gradient MMAs.  dZ3 carries the
// loss scale B*C (2 (y - t) instead of 2 (y - t) / (B C)) so it stays well
// inside FP16's range; every gradient is multiplied by 1 / (B C) in FP32 when
// it leaves the chip.
#include <cuda_fp16.h>

#include "ntc_device.cuh"
#include "ntc_internal.h"
#include "tc_ptx.cuh"

namespace ntc {

namespace {

constexpr int kRows = 128;
constexpr int kN3 = 16;
constexpr int kNWG = 2;                 // warpgroup pipelines per CTA
constexpr uint32_t kCols = 512;         // 2 x 256 TMEM columns
constexpr int kColD = 0;                // per warpgroup: layer accumulator (64)
constexpr int kColW12 = 64;             // [dW1 db1; dW2 db2] accumulator (128)
constexpr int kColW3 = 192;             // [dW3^T; db3] accumulator (16)
constexpr uint32_t kGroup = 2048;       // bytes per 8-unit group of a 128-row tile
constexpr uint32_t kWaitLimit = 1u << 18;  // suspended tries: ms to seconds

// Shared-memory plan.  Input slots (generic layout): G0 groups, G1 groups,
// [PE0..7][PE8..11, LOD, 0, 1, 1], zero groups up to k_int.
struct TPlan {
  int f0, f1, gpe, k_int;
  uint32_t w1, w2, w3, w1t, w2t, w3t, wb2, wb3, tab, wg0, wg_bytes, total;
  // offsets inside one warpgroup's region
  uint32_t P, X, H1, ONE, R, H2, ONE2, Q, DZ1, DZ2, DZ3;
  __host__ __device__ TPlan(int c0, int c1) {
    f0 = (c0 + 7) / 8;
    f1 = (c1 + 7) / 8;
    gpe = f0 + f1;
    k_int = (8 * (gpe + 2) + 15) / 16 * 16;
    uint32_t o = 0;
    w1 = o;  o += kHidden * k_int * 2;   // B of layer 1: W1 [64][k_int]
    w2 = o;  o += kHidden * kHidden * 2; // B of layer 2
    w3 = o;  o += kN3 * kHidden * 2;     // B of layer 3: W3 [16][64]
    w1t = o; o += k_int * kHidden * 2;   // B of dX: W1^T [k_int][64]
    w2t = o; o += kHidden * kHidden * 2; // B of dH1: W2^T
    w3t = o; o += kHidden * kN3 * 2;     // B of dH2: W3^T [64][16]
    wb2 = o; o += kHidden * 16 * 2;      // bias blocks (head, tail)
    wb3 = o; o += kN3 * 16 * 2;
    o = (o + 15) / 16 * 16;
    tab = o; o += 16 * 16 * 4;           // per-mip table (MipTabT)
    o = (o + 1023) / 1024 * 1024;
    wg0 = o;
    // per warpgroup: P = [X | H1 | ONE], R = [H2 | ONE2], Q = [dZ1 | dZ2], DZ3;
    // R must be followed by Q: the dW3 operand reads 16 groups from R's start
    P = 0;
    X = P;
    H1 = X + (k_int / 8) * kGroup;
    ONE = H1 + 8 * kGroup;
    R = ONE + 2 * kGroup;
    H2 = R;
    ONE2 = H2 + 8 * kGroup;
    Q = ONE2 + 2 * kGroup;
    DZ1 = Q;
    DZ2 = DZ1 + 8 * kGroup;
    DZ3 = DZ2 + 8 * kGroup;
    wg_bytes = DZ3 + 2 * kGroup;
    total = wg0 + kNWG * wg_bytes;
  }
};

struct MipTabT {
  int wm[16], hm[16], level[16];
  float lodn[16];
};

// User column of internal input slot s (generic layout): >= 0 a W1 column,
// -1 zero padding, -2 / -3 the constant-one slots (bias head / tail).
__device__ __forceinline__ int slot_column(const ntc_material& M, const TPlan& P, int s) {
  int g = s >> 3;
  const int e = s & 7;
  if (g < P.f0) return 8 * g + e < M.c0 ? 8 * g + e : -1;
  g -= P.f0;
  if (g < P.f1) return 8 * g + e < M.c1 ? M.c0 + 8 * g + e : -1;
  g -= P.f1;
  const int pe = M.c0 + M.c1;
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

__device__ void stage_train(const ntc_material& M, const TPlan& P, uint8_t* sm) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const __half z = __float2half_rn(0.f);
  for (int i = tid; i < kHidden * P.k_int; i += nt) {
    const int o = i / P.k_int, s = i - o * P.k_int;
    const int col = slot_column(M, P, s);
    __half v = z;
    if (col >= 0) {
      v = w_at(M, 0, o * M.k_in + col);
    } else if (col < -1) {
      __half hd, tl;
      split_bias(M.b[0][o], hd, tl);
      v = col == -2 ? hd : tl;
    }
    *reinterpret_cast<__half*>(sm + P.w1 + tc::canon_offset(o, s, kHidden, 2)) = v;
    // the bias slots carry no gradient path back into the grids
    *reinterpret_cast<__half*>(sm + P.w1t + tc::canon_offset(s, o, P.k_int, 2)) = col >= 0 ? v : z;
  }
  for (int i = tid; i < kHidden * kHidden; i += nt) {
    const int o = i / kHidden, k = i - o * kHidden;
    const __half v = w_at(M, 1, i);
    *reinterpret_cast<__half*>(sm + P.w2 + tc::canon_offset(o, k, kHidden, 2)) = v;
    *reinterpret_cast<__half*>(sm + P.w2t + tc::canon_offset(k, o, kHidden, 2)) = v;
  }
  for (int i = tid; i < kN3 * kHidden; i += nt) {
    const int c = i / kHidden, k = i - c * kHidden;
    const __half v = c < M.channels ? w_at(M, 2, i) : z;
    *reinterpret_cast<__half*>(sm + P.w3 + tc::canon_offset(c, k, kN3, 2)) = v;
    *reinterpret_cast<__half*>(sm + P.w3t + tc::canon_offset(k, c, kHidden, 2)) = v;
  }
  for (int i = tid; i < kHidden * 16; i += nt) {
    const int n = i / 16, k = i - n * 16;
    __half hd, tl;
    split_bias(M.b[1][n], hd, tl);
    *reinterpret_cast<__half*>(sm + P.wb2 + tc::canon_offset(n, k, kHidden, 2)) =
        k == 0 ? hd : (k == 1 ? tl : z);
  }
  for (int i = tid; i < kN3 * 16; i += nt) {
    const int n = i / 16, k = i - n * 16;
    __half hd = z, tl = z;
    if (n < M.channels) split_bias(M.b[2][n], hd, tl);
    *reinterpret_cast<__half*>(sm + P.wb3 + tc::canon_offset(n, k, kN3, 2)) =
        k == 0 ? hd : (k == 1 ? tl : z);
  }
  MipTabT* tb = reinterpret_cast<MipTabT*>(sm + P.tab);
  for (int m = tid; m < M.mips; m += nt) {
    tb->wm[m] = mip_dim(M.width, m);
    tb->hm[m] = mip_dim(M.height, m);
    tb->level[m] = level_of_mip(m, M.levels);
    tb->lodn[m] = M.mips > 1 ? (float)m / (float)(M.mips - 1) : 0.f;
  }
  // constant-one groups of every warpgroup (columns 0 and 1 of ONE and ONE2)
  for (int i = tid; i < kNWG * kRows * 2; i += nt) {
    const int w = i / (kRows * 2), r = (i / 2) % kRows, which = i & 1;
    uint8_t* base = sm + P.wg0 + w * P.wg_bytes + (which ? P.ONE2 : P.ONE);
    const uint4 one = make_uint4(tc::pack_f16x2(1.f, 1.f), 0u, 0u, 0u);
    *reinterpret_cast<uint4*>(base + tc::canon_chunk(r, 0, kRows)) = one;
    *reinterpret_cast<uint4*>(base + tc::canon_chunk(r, 1, kRows)) = make_uint4(0, 0, 0, 0);
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

// Bilinear sample of one FP32 grid of 4k channels with 16-byte loads, all
// taps' loads issued before the interpolation (same FMA order as
// sample_grid, so the same values).
__device__ __forceinline__ void sample_grid_f32x4(const ntc_material& M, int j, int k, int x, int y,
                                                  int wm, int hm, GridSample& gs) {
  const ntc_level& L = M.lv[j];
  const int gw = k ? L.g1_w : L.g0_w, gh = k ? L.g1_h : L.g0_h;
  const int c4 = (k ? M.c1 : M.c0) >> 2;
  const Taps t = bilinear_taps(x, y, wm, hm, gw, gh);
  const float4* g = static_cast<const float4*>(k ? L.grid1 : L.grid0);
  float4 v[4][kMaxGridCh / 4];
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
      for (int q = 0; q < kMaxGridCh / 4; ++q)
        v[tp][q] = q < c4 ? __ldg(g + (size_t)t.cell[tp] * c4 + q) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
#pragma unroll
  for (int ch = 0; ch < kMaxGridCh; ++ch) gs.acc[ch] = 0.f;
#pragma unroll
  for (int tp = 0; tp < 4; ++tp)
#pragma unroll
    for (int q = 0; q < kMaxGridCh / 4; ++q) {
      gs.acc[4 * q] = fmaf(t.w[tp], v[tp][q].x, gs.acc[4 * q]);
      gs.acc[4 * q + 1] = fmaf(t.w[tp], v[tp][q].y, gs.acc[4 * q + 1]);
      gs.acc[4 * q + 2] = fmaf(t.w[tp], v[tp][q].z, gs.acc[4 * q + 2]);
      gs.acc[4 * q + 3] = fmaf(t.w[tp], v[tp][q].w, gs.acc[4 * q + 3]);
    }
}

__device__ __forceinline__ bool wait_phase(uint64_t* bar, uint32_t& phase, int bar_id) {
  const bool ok = tc::mbar_wait(bar, phase, kWaitLimit);
  phase ^= 1;
  return !tc::bar_or(bar_id, kRows, !ok);
}

__global__ void __launch_bounds__(kRows* kNWG, 1) train_tc_kernel(const ntc_material M,
                                                                   const BwdArgs A, int* status) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ uint64_t mbar[kNWG];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_any;
  __shared__ float red[kNWG * 4];
  const TPlan P(M.c0, M.c1);
  uint8_t* sm = smem_raw;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int wg = tid / kRows, row = tid % kRows;
  const int bar_id = 1 + wg;
  const int C = M.channels;

  stage_train(M, P, sm);
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, kCols);
    tc::tmem_relinquish();
  }
  if (tid < kNWG) tc::mbar_init(&mbar[tid], 1);
  if (tid == 0) abort_any = 0;
  tc::fence_mbar_init();
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();

  const uint32_t tw = tmem_base + 256u * wg;
  const uint32_t lane = (uint32_t)((warp & 3) * 32) << 16;
  uint64_t* bar = &mbar[wg];
  uint8_t* W = sm + P.wg0 + wg * P.wg_bytes;
  const uint32_t sW = tc::smem_u32(W), sbase = tc::smem_u32(sm);
  const MipTabT* tb = reinterpret_cast<const MipTabT*>(sm + P.tab);
  constexpr uint32_t lbo_a = (kRows / 8) * 128, lbo64 = (kHidden / 8) * 128, lbo16 = (kN3 / 8) * 128;
  const uint32_t lbo_k = (uint32_t)(P.k_int / 8) * 128;
  constexpr uint32_t id64 = tc::idesc(kRows, kHidden), id16 = tc::idesc(kRows, kN3);
  const uint32_t idk = tc::idesc(kRows, P.k_int);
  const uint32_t id_w12 = tc::idesc(kRows, P.k_int + 80) | (1u << 15) | (1u << 16);
  const uint32_t id_w3 = tc::idesc(kRows, kN3) | (1u << 15) | (1u << 16);

  const int64_t step = A.step_dev ? *A.step_dev : A.noise_step;
  const uint64_t nkey = rng_key(A.noise_seed, noise_stream(step));
  const uint64_t skey = rng_key(A.sample_seed, sampler_stream(step));
  const int64_t ntiles = (A.n + kRows - 1) / kRows;
  uint32_t phase = 0;
  uint32_t acc = 0;  // weight-gradient accumulators start empty
  float loss_acc = 0.f;
  bool aborted = false;

  for (int64_t tl = (int64_t)blockIdx.x * kNWG + wg; tl < ntiles; tl += (int64_t)gridDim.x * kNWG) {
    const int64_t i = tl * kRows + row;
    const bool valid = i < A.n;
    // ---- texel, target, features -> X -----------------------------------
    int x = 0, y = 0, m = 0;
    if (valid) {
      if (A.uvl) query_texel(M, A.uvl[3 * i], A.uvl[3 * i + 1], A.uvl[3 * i + 2], x, y, m);
      else sample_texel(skey, i, M.width, M.height, M.mips, x, y, m);
    }
    float tgt[kN3];
    {
      const uint8_t* trow = A.target + A.tgt_off[m] + ((int64_t)y * tb->wm[m] + x) * C;
      if ((C & 3) == 0) {
        // whole 4-byte words of the u8 row (row offsets are multiples of 4)
#pragma unroll
        for (int c4 = 0; c4 < kN3 / 4; ++c4) {
          const uint32_t wv = (valid && 4 * c4 < C) ? __ldg(reinterpret_cast<const uint32_t*>(trow) + c4) : 0u;
#pragma unroll
          for (int b = 0; b < 4; ++b) tgt[4 * c4 + b] = (float)((wv >> (8 * b)) & 0xFFu) * (1.f / 255.f);
        }
      } else {
#pragma unroll
        for (int c = 0; c < kN3; ++c) tgt[c] = (valid && c < C) ? (float)trow[c] * (1.f / 255.f) : 0.f;
      }
    }
    uint8_t* X = W + P.X;
    {
      const int j = tb->level[m];
      const int wm = tb->wm[m], hm = tb->hm[m];
      GridSample gs;
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int ck = k ? M.c1 : M.c0;
        if (!A.noise && (ck & 3) == 0) sample_grid_f32x4(M, j, k, x, y, wm, hm, gs);
        else sample_grid(M, j, k, x, y, wm, hm, A.noise != 0 && valid, nkey, gs);
        const int g0 = k ? P.f0 : 0, ng = k ? P.f1 : P.f0;
#pragma unroll
        for (int g = 0; g < 2; ++g)
          if (g < ng) {
            float v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = valid ? gs.acc[8 * g + e] : 0.f;
            put_chunk(X, row, g0 + g, v);
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
      put_chunk(X, row, P.gpe, v);
#pragma unroll
      for (int e = 0; e < 4; ++e) v[e] = pe.v[8 + e];
      v[4] = tb->lodn[m];
      v[5] = 0.f;
      v[6] = v[7] = 1.f;
      put_chunk(X, row, P.gpe + 1, v);
      const float zz[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      for (int g = P.gpe + 2; g < P.k_int / 8; ++g) put_chunk(X, row, g, zz);
    }
    tc::fence_proxy_async();
    tc::bar_sync(bar_id, kRows);

    // ---- layer 1 -----------------------------------------------------------------
    if (row == 0) {
      tc::fence_after_sync();
      issue_kmajor(tw + kColD, sW + P.X, lbo_a, sbase + P.w1, lbo64, P.k_int / 16, id64, 0);
      tc::mma_commit(bar);
    }
    if (!wait_phase(bar, phase, bar_id)) { aborted = true; break; }
    tc::fence_after_sync();
    row64_to_tile(tw + kColD + lane, W + P.H1, row, [](int, float z) { return fmaxf(z, 0.f); });
    tc::fence_before_sync();
    tc::fence_proxy_async();
    tc::bar_sync(bar_id, kRows);

    // ---- layer 2 -----------------------------------------------------------------
    if (row == 0) {
      tc::fence_after_sync();
      issue_kmajor(tw + kColD, sW + P.H1, lbo_a, sbase + P.w2, lbo64, 4, id64, 0);
      issue_kmajor(tw + kColD, sW + P.ONE, lbo_a, sbase + P.wb2, lbo64, 1, id64, 1);
      tc::mma_commit(bar);
    }
    if (!wait_phase(bar, phase, bar_id)) { aborted = true; break; }
    tc::fence_after_sync();
    row64_to_tile(tw + kColD + lane, W + P.H2, row, [](int, float z) { return fmaxf(z, 0.f); });
    tc::fence_before_sync();
    tc::fence_proxy_async();
    tc::bar_sync(bar_id, kRows);

    // ---- layer 3, loss, dZ3 ----------------------------------------------------
    if (row == 0) {
      tc::fence_after_sync();
      issue_kmajor(tw + kColD, sW + P.H2, lbo_a, sbase + P.w3, lbo16, 4, id16, 0);
      issue_kmajor(tw + kColD, sW + P.ONE, lbo_a, sbase + P.wb3, lbo16, 1, id16, 1);
      tc::mma_commit(bar);
    }
    if (!wait_phase(bar, phase, bar_id)) { aborted = true; break; }
    tc::fence_after_sync();
    {
      float zv[16];
      tc::tmem_ld16(tw + kColD + lane, zv);
      tc::tmem_ld_wait();
      float d[16];
#pragma unroll
      for (int c = 0; c < kN3; ++c) {
        float g = 0.f;
        if (valid && c < C) {
          const float yc = M.out_act == NTC_OUT_IDENTITY ? zv[c] : 1.f / (1.f + __expf(-zv[c]));
          const float e = yc - tgt[c];
          loss_acc = fmaf(e, e, loss_acc);
          g = M.out_act == NTC_OUT_IDENTITY ? 2.f * e : 2.f * e * yc * (1.f - yc);
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

    // ---- dH2 = dZ3 W3 -> dZ2 ------------------------------------------------------
    if (row == 0) {
      tc::fence_after_sync();
      issue_kmajor(tw + kColD, sW + P.DZ3, lbo_a, sbase + P.w3t, lbo64, 1, id64, 0);
      tc::mma_commit(bar);
    }
    if (!wait_phase(bar, phase, bar_id)) { aborted = true; break; }
    tc::fence_after_sync();
    {
      __half2 h[32];
      tile_row64(W + P.H2, row, h);
      row64_to_tile(tw + kColD + lane, W + P.DZ2, row,
                    [&](int q, float g) { return half_of(h, q) > 0.f ? g : 0.f; });
    }
    tc::fence_before_sync();
    tc::fence_proxy_async();
    tc::bar_sync(bar_id, kRows);

    // ---- dH1 = dZ2 W2 -> dZ1 ------------------------------------------------------
    if (row == 0) {
      tc::fence_after_sync();
      issue_kmajor(tw + kColD, sW + P.DZ2, lbo_a, sbase + P.w2t, lbo64, 4, id64, 0);
      tc::mma_commit(bar);
    }
    if (!wait_phase(bar, phase, bar_id)) { aborted = true; break; }
    tc::fence_after_sync();
    {
      __half2 h[32];
      tile_row64(W + P.H1, row, h);
      row64_to_tile(tw + kColD + lane, W + P.DZ1, row,
                    [&](int q, float g) { return half_of(h, q) > 0.f ? g : 0.f; });
    }
    tc::fence_before_sync();
    tc::fence_proxy_async();
    tc::bar_sync(bar_id, kRows);

    // ---- dX = dZ1 W1, and the weight gradients of this tile ---------------------
    if (row == 0) {
      tc::fence_after_sync();
      issue_kmajor(tw + kColD, sW + P.DZ1, lbo_a, sbase + P.w1t, lbo_k, 4, idk, 0);
      issue_mnmajor(tw + kColW12, sW + P.Q, sW + P.P, id_w12, acc);
      issue_mnmajor(tw + kColW3, sW + P.R, sW + P.DZ3, id_w3, acc);
      tc::mma_commit(bar);
    }
    acc = 1;
    if (!wait_phase(bar, phase, bar_id)) { aborted = true; break; }
    tc::fence_after_sync();
    if (A.grids) {
      // dX slots: G0 at columns 0.., G1 at 8 * f0.. (f0 is 1 or 2)
      float d[32], dg0[16], dg1[16];
      {
        float lo[16], hi[16];
        tc::tmem_ld16(tw + kColD + lane, lo);
        tc::tmem_ld16(tw + kColD + lane + 16, hi);
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
            const float wgt = t.w[tp] * A.grad_scale;
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
              for (int ch = 0; ch < kMaxGridCh; ++ch)
                if (ch < c) atomicAdd(gp + ch, (k ? dg1[ch] : dg0[ch]) * wgt);
            }
          }
        }
      }
    }
    tc::fence_before_sync();
    tc::bar_sync(bar_id, kRows);  // the next tile's features overwrite the operand tiles
  }

  // ---- flush the weight gradients of this warpgroup ----------------------------
  if (aborted && row == 0) abort_any = 1;
  tc::fence_after_sync();
  const float gs = A.grad_scale;
  if (!aborted && acc) {
    // [dW1 db1; dW2 db2]: row r < 64 -> (dW1 row r, db1 r), else (dW2 row r-64, db2 r-64)
    const int kin = P.k_int;
#pragma unroll 1
    for (int cb = 0; cb < 128; cb += 16) {
      float v[16];
      tc::tmem_ld16(tw + kColW12 + lane + cb, v);
      tc::tmem_ld_wait();
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int col = cb + e;
        if (row < kHidden) {
          if (col < kin) {
            const int uc = slot_column(M, P, col);
            if (uc >= 0 && A.g.w[0]) atomicAdd(A.g.w[0] + row * M.k_in + uc, v[e] * gs);
          } else if (col == kin + 64 && A.g.b[0]) {
            atomicAdd(A.g.b[0] + row, v[e] * gs);
          }
        } else {
          const int o = row - kHidden;
          if (col >= kin && col < kin + 64 && A.g.w[1])
            atomicAdd(A.g.w[1] + o * kHidden + (col - kin), v[e] * gs);
          else if (col == kin + 64 && A.g.b[1])
            atomicAdd(A.g.b[1] + o, v[e] * gs);
        }
      }
    }
    // [dW3^T; db3]: row r < 64 -> dW3[:, r]; row 64 -> db3
    float v[16];
    tc::tmem_ld16(tw + kColW3 + lane, v);
    tc::tmem_ld_wait();
#pragma unroll
    for (int c = 0; c < kN3; ++c) {
      if (c >= C) continue;
      if (row < kHidden && A.g.w[2]) atomicAdd(A.g.w[2] + c * kHidden + row, v[c] * gs);
      if (row == kHidden && A.g.b[2]) atomicAdd(A.g.b[2] + c, v[c] * gs);
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
    for (int w = 0; w < kNWG * 4; ++w) s += red[w];
    if (A.loss) atomicAdd(A.loss, s * A.loss_scale);
    if (abort_any) atomicExch(status, NTC_ERR_TIMEOUT);
  }
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem_base, kCols);
  }
}

}  // namespace

cudaError_t launch_train_tc(const ntc_material& m, const BwdArgs& a, cudaStream_t s) {
  if (a.n == 0) return cudaSuccess;
  if (m.precision != NTC_PREC_F16 || m.act != NTC_ACT_RELU || m.interp0 != NTC_INTERP_BILINEAR ||
      !a.train)
    return cudaErrorNotSupported;
  const TPlan P(m.c0, m.c1);
  const size_t smem = P.total;
  cudaError_t e = cudaFuncSetAttribute(train_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t tiles = (a.n + kRows - 1) / kRows;
  const int64_t ctas = (tiles + kNWG - 1) / kNWG;
  const int64_t cap = sm_count();
  const int grid = (int)(ctas < cap ? ctas : cap);
  train_tc_kernel<<<grid, kRows * kNWG, smem, s>>>(m, a, status_word());
  return cudaGetLastError();
}

}  // namespace ntc
