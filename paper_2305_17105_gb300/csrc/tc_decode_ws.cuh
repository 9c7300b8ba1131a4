// Warp-specialised tensor-core decode kernel (FP16 and FP8-E4M3), shared by
// the translation units that instantiate it: every fast-layout class of the
// FP16 form in tc_decode_ws.cu, the FP8 form in tc_decode_ws_f8.cu.
#pragma once
#include "tc_decode_common.cuh"

namespace ntc {

namespace {

// ---------------------------------------------------------------------------
// Warp-specialised form (FP16 or FP8-E4M3): four compute warpgroups, each running its own
// stream of tiles, and one issuer warpgroup whose warp w issues every
// tcgen05.mma chain of compute warpgroup w.  A chain of dependent MMAs holds
// its issuing thread until it drains, so issuing from the compute warps
// stalls them; here they only hand over through mbarriers and keep working:
//   X(i) in shared memory --x--> L1 --d--> epilogue 1 -> H --h--> L2 --d-->
//   epilogue 2 -> H --h--> L3 (own accumulator D3) --o--> output,
// and while L2(i) runs the compute warps build X(i+1), while L3(i) runs they
// gather the cells of tile i+2, while L1(i+1) runs they write tile i.  L1
// reads its A operand from shared memory, the bias steps a constant-one A
// block in shared memory; L2 and L3 read H from TMEM.  FP8 (kind::f8f6f4):
// X and H hold E4M3 values of the layer inputs divided by their activation
// scales s_a; the epilogues apply s_w s_a and add the FP32 biases.
// TMEM per compute warpgroup (128 columns): D [0, 64), H [64, 96),
// D3 [96, 112).
// ---------------------------------------------------------------------------
constexpr int kWsCompute = 4;
constexpr int kWsThreads = kRows * (kWsCompute + 1);
constexpr int kColD3 = 96;

struct WsPlan {
  uint32_t cst, x, xbytes, total;
  __host__ __device__ WsPlan(const Plan& P, bool f8) {
    uint32_t o = (P.total + 1023) / 1024 * 1024;
    cst = o;  o += kRows * 16 * 2;                 // constant-one A block (K = 16, FP16)
    xbytes = kRows * P.k_int * (f8 ? 1 : 2);
    x = o;    o += kWsCompute * xbytes;            // one X tile per compute warpgroup
    total = o;
  }
};

// FP8 input rows: the FP16 groups the builders produce, divided by the
// layer-1 activation scale and rounded to E4M3 (saturating), 8 bytes a group.
struct F8Row {
  SmemRow dst;
  __half2 inv;
  __device__ __forceinline__ uint32_t cv(uint32_t a, uint32_t b) const {
    return tc::h2_to_e4m3x2(h2u(__hmul2(u2h(a), inv))) |
           (tc::h2_to_e4m3x2(h2u(__hmul2(u2h(b), inv))) << 16);
  }
  __device__ __forceinline__ void put4(int g, uint4 w) const { dst.put2(g, cv(w.x, w.y), cv(w.z, w.w)); }
  __device__ __forceinline__ void put2(int g, uint32_t a, uint32_t b) const { dst.put2(g, a, b); }
};

// FP8 hidden-layer epilogue in quarters, in the next layer's input units:
// z' = (s_w s_a / s_a') acc + b / s_a' (paired FMAs; `bias` holds b / s_a'),
// then act(z) / s_a' = max(z', 0) (folded into the E4M3 conversion) or, for
// hardGELU, z' sat(z' s_a' / 3 + 1/2); E4M3 into the A row (TMEM, four
// values per column).
__device__ __forceinline__ void hidden_epilogue_q8(uint32_t td, uint32_t ta, int act,
                                                   const float* bias, float scale, float hk) {
  const float2 sc2 = make_float2(scale, scale);
#pragma unroll
  for (int qtr = 0; qtr < 4; ++qtr) {
    float a[16];
    tc::tmem_ld16(td + 16 * qtr, a);
    tc::tmem_ld_wait();
    const float2* b2 = reinterpret_cast<const float2*>(bias + 16 * qtr);
    uint32_t e[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float2 z = __ffma2_rn(make_float2(a[2 * i], a[2 * i + 1]), sc2, b2[i]);
      e[i] = act == NTC_ACT_RELU
                 ? tc::pack_e4m3x2_relu(z.x, z.y)
                 : tc::pack_e4m3x2(z.x * __saturatef(fmaf(z.x, hk, 0.5f)),
                                   z.y * __saturatef(fmaf(z.y, hk, 0.5f)));
    }
    tc::tmem_st4(ta + 4 * qtr, make_uint4(e[0] | (e[1] << 16), e[2] | (e[3] << 16),
                                          e[4] | (e[5] << 16), e[6] | (e[7] << 16)));
  }
}

// H3: a third hidden layer (FP16; the runtime-class and generic layouts).
template <int CLS, bool F8, bool H3>
__global__ void __launch_bounds__(kWsThreads, 1) decode_ws_kernel(
    const ntc_material M, const float* __restrict__ uvl, int64_t n, void* __restrict__ out,
    int out_dtype, int filter, uint64_t jkey, int* status) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ uint64_t bar_x[kWsCompute], bar_h[kWsCompute], bar_d[kWsCompute],
      bar_o[kWsCompute], bar_fin[kWsCompute];
  __shared__ uint32_t tmem_base;
  __shared__ int wg_abort[kWsCompute];
  // CLS > 0: compile-time fast class; -1: fast layout with the class read
  // from the plan (learned interpolation); 0: generic layout
  constexpr bool FAST = CLS != 0;
  const Plan P(M, F8, FAST);
  const WsPlan W(P, F8);
  uint8_t* sm = smem_raw;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wg = warp >> 2, row = tid & (kRows - 1);

  stage_shared<F8>(M, P, sm, tid, blockDim.x);
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
  if (wg < kWsCompute) zero_tail_groups<F8>(P, SmemRow{smem_row(sm + W.x + wg * W.xbytes, row)});
  tc::fence_mbar_init();
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (F8) {
    // hidden biases in the next layer's input units: b / s_a'
    float* b = reinterpret_cast<float*>(sm + P.bias);
    const float i1 = 1.f / M.scale[4], i2 = 1.f / M.scale[5];
    for (int i = tid; i < kHidden; i += blockDim.x) {
      b[i] *= i1;
      b[kHidden + i] *= i2;
    }
    __syncthreads();
  }

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
      constexpr int KSTEP = Cfg<F8>::KSTEP;
      const int k1 = P.k_int / KSTEP;
      uint32_t px = 0, ph = 0;
      bool ok = true;
      for (int64_t tl = first; tl < ntiles; tl += stride) {
        if (!(ok = tc::mbar_wait(&bar_x[w], px, kWaitLimit))) break;
        px ^= 1;
        tc::fence_after_sync();
        // one K-step = 32 bytes of every row = two 16-byte chunk columns
        for (int s = 0; s < k1; ++s) {
          if (F8) tc::mma_f8(tw, tc::smem_desc(xa + s * 4096, 2048, 128), d[s], id64, s > 0);
          else tc::mma_f16(tw, tc::smem_desc(xa + s * 4096, 2048, 128), d[s], id64, s > 0);
        }
        tc::mma_commit(&bar_d[w]);
        if (!(ok = tc::mbar_wait(&bar_h[w], ph, kWaitLimit))) break;
        ph ^= 1;
        tc::fence_after_sync();
        for (int s = 0; s < kHidden / KSTEP; ++s) {
          if (F8) tc::mma_f8_ta(tw, tw + kColH + 8 * s, d[kDescW2 + s], id64, s > 0);
          else tc::mma_f16_ta(tw, tw + kColH + 8 * s, d[kDescW2 + s], id64, s > 0);
        }
        if (!F8) tc::mma_f16(tw, cst, d[kDescW2 + 4], id64, 1);
        tc::mma_commit(&bar_d[w]);
        if (H3) {
          // third hidden layer: H -> D, like layer 2
          if (!(ok = tc::mbar_wait(&bar_h[w], ph, kWaitLimit))) break;
          ph ^= 1;
          tc::fence_after_sync();
          for (int s = 0; s < kHidden / 16; ++s)
            tc::mma_f16_ta(tw, tw + kColH + 8 * s, d[kDescWh + s], id64, s > 0);
          tc::mma_f16(tw, cst, d[kDescWh + 4], id64, 1);
          tc::mma_commit(&bar_d[w]);
        }
        if (!(ok = tc::mbar_wait(&bar_h[w], ph, kWaitLimit))) break;
        ph ^= 1;
        tc::fence_after_sync();
        for (int s = 0; s < kHidden / KSTEP; ++s) {
          if (F8) tc::mma_f8_ta(tw + kColD3, tw + kColH + 8 * s, d[kDescW3 + s], id16, s > 0);
          else tc::mma_f16_ta(tw + kColD3, tw + kColH + 8 * s, d[kDescW3 + s], id16, s > 0);
        }
        if (!F8) tc::mma_f16(tw + kColD3, cst, d[kDescW3 + 4], id16, 1);
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
    // FP8: per-layer accumulator scales s_w s_a (layer 3 pre-halved for the
    // tanh form of the sigmoid) and inverse activation scales
    float sc[3] = {1.f, 1.f, 1.f}, inv_sa[3] = {1.f, 1.f, 1.f};
    if (F8) {
#pragma unroll
      for (int l = 0; l < 3; ++l) {
        sc[l] = M.scale[l] * M.scale[3 + l];
        inv_sa[l] = 1.f / M.scale[3 + l];
      }
      if (M.out_act != NTC_OUT_IDENTITY) sc[2] *= 0.5f;
    }
    const float* bias = reinterpret_cast<const float*>(sm + P.bias);
    const F8Row x8{xs, __float2half2_rn(inv_sa[0])};
    auto qindex = [&](int64_t t) { return tri ? t * per_tile + (row >> 3) : t * per_tile + row; };
    auto build = [&](const Row& r) {
      if (F8) {
        if (CLS > 0) build_fast(FastLayout<(CLS > 0 ? CLS : 1)>(), P, K, sm, r, x8);
        else build_generic<true>(M, P, sm, r, xs, inv_sa[0]);
      } else {
        if (CLS > 0) build_fast(FastLayout<(CLS > 0 ? CLS : 1)>(), P, K, sm, r, xs);
        else if (CLS < 0) build_fast(P, P, K, sm, r, xs);
        else build_generic<false>(M, P, sm, r, xs, 1.f);
      }
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
      locate(M, tb, load_query(uvl, q0, q0 < n), filter, row, r, q0, jkey);
      if (CLS > 0) gather_fast(FastLayout<(CLS > 0 ? CLS : 1)>(), tb, r);
      else if (CLS < 0) gather_fast(P, tb, r);
      build(r);
      cur_valid = r.valid;
      cur_wtap = r.wtap;
      const int64_t q1 = qindex(tl + stride);
      locate(M, tb, load_query(uvl, q1, tl + stride < ntiles && q1 < n), filter, row, nxt, q1, jkey);
      if (CLS > 0) gather_fast(FastLayout<(CLS > 0 ? CLS : 1)>(), tb, nxt);
      else if (CLS < 0) gather_fast(P, tb, nxt);
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
      if (F8) hidden_epilogue_q8(td, th, M.act, bias, sc[0] * inv_sa[1], M.scale[4] * (1.f / 3.f));
      else hidden_epilogue_q(td, th, M.act);
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
      if (F8) hidden_epilogue_q8(td, th, M.act, bias + kHidden, sc[1] * inv_sa[2], M.scale[5] * (1.f / 3.f));
      else hidden_epilogue_q(td, th, M.act);
      tc::tmem_st_wait();
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&bar_h[w]);
      if (H3) {
        // third hidden layer -> H
        if (!tc::mbar_wait(&bar_d[w], pd, kWaitLimit)) *abort_flag = 1;
        pd ^= 1;
        tc::fence_after_sync();
        hidden_epilogue_q(td, th, M.act);
        tc::tmem_st_wait();
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&bar_h[w]);
      }
      if (*abort_flag) break;
      // the tile after next: texel and cells; its successor's query
      locate(M, tb, nq, filter, row, nxt, qindex(tl + 2 * stride), jkey);
      if (CLS > 0) gather_fast(FastLayout<(CLS > 0 ? CLS : 1)>(), tb, nxt);
      else if (CLS < 0) gather_fast(P, tb, nxt);
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
      if (F8) {
        const float2* b3 = reinterpret_cast<const float2*>(bias + 2 * kHidden);
#pragma unroll
        for (int c = 0; c < 16; c += 2) {
          const float2 z = __ffma2_rn(make_float2(yv[c], yv[c + 1]), make_float2(sc[2], sc[2]), b3[c / 2]);
          yv[c] = z.x;
          yv[c + 1] = z.y;
        }
      }
      out_activate(yv, M.out_act);
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

template <int CLS, bool F8, bool H3 = false>
cudaError_t launch_ws(const ntc_material& m, const float* uvl, int64_t n, void* out, int out_dtype,
                      int filter, uint64_t jkey, cudaStream_t s) {
  static_assert(!(F8 && H3), "three hidden layers run in FP16");
  const Plan P(m, F8, CLS != 0);
  if (P.h3 != H3) return cudaErrorInvalidValue;
  const WsPlan W(P, F8);
  cudaError_t e = cudaFuncSetAttribute(decode_ws_kernel<CLS, F8, H3>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)W.total);
  if (e != cudaSuccess) return e;
  const int per_tile = filter == NTC_FILTER_TRILINEAR ? kRows / 8 : kRows;
  const int64_t tiles = (n + per_tile - 1) / per_tile;
  const int64_t ctas = (tiles + kWsCompute - 1) / kWsCompute;
  const int64_t cap = sm_count();
  const int grid = (int)(ctas < cap ? ctas : cap);
  decode_ws_kernel<CLS, F8, H3><<<grid, kWsThreads, W.total, s>>>(m, uvl, n, out, out_dtype,
                                                                  filter, jkey, status_word());
  return cudaGetLastError();
}

// Compile-time class of a fast-layout grid: 0 (cell of 4 bytes), 1 (9-12
// channels in 8 bytes), 2 (13-16 channels).
inline int grid_class(int c, int cb) { return cb == 4 ? 0 : (c > 12 ? 2 : 1); }

}  // namespace

}  // namespace ntc
