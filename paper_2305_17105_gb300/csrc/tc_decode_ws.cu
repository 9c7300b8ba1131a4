// Warp-specialised tensor-core decode (FP16), instantiated per fast-layout
// class so that the per-row feature code has no runtime layout branches, and
// its many-material form.
#include "tc_decode_ws.cuh"

namespace ntc {

namespace {

// ---------------------------------------------------------------------------
// Many materials in one launch, warp-specialised.  The batch descriptor
// (device) lists the materials and the prefix sums of their tiles; compute
// warpgroup w of CTA b takes a contiguous range of the tile list and keeps
// its current material (weights, tables, B descriptors) in its own region
// of shared memory.  At a material boundary it lets its pipeline drain (the
// last tile's L3 done means every MMA that read the old weights is done),
// restages the region, then carries on; its issuer reads the descriptors
// and K from the region on every tile, after the X hand-over.
//   CLS: -1 fast layout with the class read from each material's Plan,
//   0 generic layout, 1..9 one compile-time fast class for the whole batch.
// ---------------------------------------------------------------------------
struct WsBatchSmem {
  uint32_t region, cst, x, xbytes, total;  // per-warpgroup region size; offsets
  // packed: plan bytes of the largest material | largest internal K << 24
  __host__ __device__ explicit WsBatchSmem(uint32_t packed) {
    const uint32_t plan_bytes = packed & 0xFFFFFFu, kmax = packed >> 24;
    region = (plan_bytes + 1023) / 1024 * 1024;
    cst = kWsCompute * region;
    x = cst + kRows * 16 * 2;
    xbytes = kRows * kmax * 2;
    total = x + kWsCompute * xbytes;
  }
};

template <int CLS>
__global__ void __launch_bounds__(kWsThreads, 1) decode_ws_batched_kernel(
    const BatchHeader* __restrict__ B, const float* __restrict__ uvl, void* __restrict__ out,
    int out_dtype, int filter, uint32_t plan_bytes, int* status) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ uint64_t bar_x[kWsCompute], bar_h[kWsCompute], bar_d[kWsCompute],
      bar_o[kWsCompute], bar_fin[kWsCompute];
  __shared__ uint32_t tmem_base;
  __shared__ int wg_abort[kWsCompute];
  __shared__ int kint_s[kWsCompute];
  __shared__ uint32_t desc_s[kWsCompute];
  __shared__ ntc_material mat_s[kWsCompute];
  constexpr bool FAST = CLS != 0;
  using Lay = FastLayout<(CLS > 0 ? CLS : 1)>;
  const WsBatchSmem S(plan_bytes);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wg = warp >> 2, row = tid & (kRows - 1);
  for (int i = tid; i < kRows * 16 / 2; i += blockDim.x) {
    const int chunk = i >> 2, e = i & 3;
    reinterpret_cast<uint32_t*>(smem_raw + S.cst)[i] =
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
  tc::fence_mbar_init();
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();

  const bool tri = filter == NTC_FILTER_TRILINEAR;
  const int per_tile = tri ? kRows / 8 : kRows;
  const int nm = B->n_materials;
  const int64_t total = B->total_tiles;
  const int w = wg < kWsCompute ? wg : (warp & 3);
  const int64_t nwgs = (int64_t)gridDim.x * kWsCompute, gw = (int64_t)blockIdx.x * kWsCompute + w;
  // tile indices fit 32 bits (ntc_batch_prepare refuses larger batches)
  const int t_begin = (int)(total * gw / nwgs), t_end = (int)(total * (gw + 1) / nwgs);
  constexpr uint32_t id64 = tc::idesc(kRows, kHidden), id16 = tc::idesc(kRows, kN3);
  const uint32_t tw = tmem_base + 128u * w;
  uint8_t* region = smem_raw + (size_t)w * S.region;
  uint8_t* xtile = smem_raw + S.x + (size_t)w * S.xbytes;

  if (wg == kWsCompute) {
    // ---- issuer warp w ------------------------------------------------------
    if (lane == 0) {
      const uint32_t xa = tc::smem_u32(xtile);
      const uint64_t cst = tc::smem_desc(tc::smem_u32(smem_raw + S.cst), 2048, 128);
      uint32_t px = 0, ph = 0;
      bool ok = true;
      for (int tl = t_begin; tl < t_end; ++tl) {
        if (!(ok = tc::mbar_wait(&bar_x[w], px, kWaitLimit))) break;
        px ^= 1;
        tc::fence_after_sync();
        const uint64_t* d = reinterpret_cast<const uint64_t*>(
            region + *reinterpret_cast<volatile uint32_t*>(&desc_s[w]));
        const int k1 = *reinterpret_cast<volatile int*>(&kint_s[w]) / 16;
        for (int s = 0; s < k1; ++s)
          tc::mma_f16(tw, tc::smem_desc(xa + s * 4096, 2048, 128), d[s], id64, s > 0);
        tc::mma_commit(&bar_d[w]);
        if (!(ok = tc::mbar_wait(&bar_h[w], ph, kWaitLimit))) break;
        ph ^= 1;
        tc::fence_after_sync();
        for (int s = 0; s < kHidden / 16; ++s)
          tc::mma_f16_ta(tw, tw + kColH + 8 * s, d[kDescW2 + s], id64, s > 0);
        tc::mma_f16(tw, cst, d[kDescW2 + 4], id64, 1);
        tc::mma_commit(&bar_d[w]);
        if (!(ok = tc::mbar_wait(&bar_h[w], ph, kWaitLimit))) break;
        ph ^= 1;
        tc::fence_after_sync();
        for (int s = 0; s < kHidden / 16; ++s)
          tc::mma_f16_ta(tw + kColD3, tw + kColH + 8 * s, d[kDescW3 + s], id16, s > 0);
        tc::mma_f16(tw + kColD3, cst, d[kDescW3 + 4], id16, 1);
        tc::mma_commit(&bar_o[w]);
      }
      if (!ok) *reinterpret_cast<volatile int*>(&wg_abort[w]) = 1;
      tc::mma_commit(&bar_fin[w]);
      if (!tc::mbar_wait(&bar_fin[w], 0, kWaitLimit)) *reinterpret_cast<volatile int*>(&wg_abort[w]) = 1;
    }
  } else {
    // ---- compute warpgroup w -------------------------------------------------
    const uint32_t lq = (uint32_t)((warp & 3) * 32) << 16;
    const uint32_t td = tw + lq, th = tw + kColH + lq, td3 = tw + kColD3 + lq;
    const SmemRow xs{smem_row(xtile, row)};
    volatile int* abort_flag = &wg_abort[w];
    const int bar_id = 1 + w;
    const ntc_material& M = mat_s[w];
    // the current material: its plan, its tile range and query/output bases
    int mid = 0;
    Plan P(mat_s[w], false, false);
    // the current material's tiles [m_t0, m_t1), its first query and output
    // element in the batch, its query count (< 2^31)
    int m_t0 = 0, m_t1 = 0, m_nq = 0;
    int64_t m_q0 = 0, m_o0 = 0;
    // the fields the tile loop reads, held in registers (the fences and
    // waits of the loop clobber memory, so fields read from mat_s would be
    // loaded again every tile)
    int m_mips = 1, m_act = 0, m_oact = 0, m_C = 0;
    // stage material `mid` (no MMA of this warpgroup in flight, no thread
    // still reading the region)
    auto stage = [&](int id) {
      mid = id;
      tc::bar_sync(bar_id, kRows);
      if (row == 0) mat_s[w] = B->mats[id];
      tc::bar_sync(bar_id, kRows);
      P = Plan(M, false, FAST);
      m_mips = M.mips;
      m_act = M.act;
      m_oact = M.out_act;
      m_C = M.channels;
      stage_shared<false>(M, P, region, row, kRows);
      zero_tail_groups<false>(P, xs);
      if (row == 0) {
        kint_s[w] = P.k_int;
        desc_s[w] = P.desc;
      }
      m_t0 = (int)B->tile_start[id];
      m_t1 = (int)B->tile_start[id + 1];
      m_q0 = B->q_off[id];
      m_nq = (int)(B->q_off[id + 1] - m_q0);
      m_o0 = B->o_off[id];
      tc::fence_proxy_async();
      tc::bar_sync(bar_id, kRows);
    };
    auto next_material = [&](int t) {
      int m = mid;
      while (m + 1 < nm && t >= B->tile_start[m + 1]) ++m;
      return m;
    };
    const MipTab* tb = nullptr;
    // tile t's query of this row (tile t of the current material)
    auto query_of = [&](int t) {
      const int ql = tri ? (t - m_t0) * per_tile + (row >> 3) : (t - m_t0) * per_tile + row;
      return load_query(uvl, m_q0 + ql, ql < m_nq);
    };
    auto locate_from = [&](const Query& qu, Row& r) {
      locate(MipCount{m_mips}, tb, qu, filter, row, r);
      if (CLS > 0) gather_fast(Lay(), tb, r);
      else if (CLS < 0) gather_fast<Plan, false>(P, tb, r);  // batches: no VQ
    };
    auto build = [&](const Row& r) {
      if (CLS > 0) build_fast(Lay(), P, FastK(M), region, r, xs);
      else if (CLS < 0) build_fast<Plan, SmemRow, false>(P, P, FastK(M), region, r, xs);
      else build_generic<false, SmemRow, false>(M, P, region, r, xs, 1.f);  // batches: no VQ
      tc::fence_proxy_async();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&bar_x[w]);
    };
    uint32_t pd = 0, po = 0;
    int cur_valid = 0;
    float cur_wtap = 0.f;
    Row nxt;
    bool have_nxt = false;  // nxt holds tile tl+1, of the current material, gathered
    Query nq;               // with have_nq: the query of tile tl+2, loaded a tile ahead
    bool have_nq = false;
    // first tile of a material run (after staging): build it, gather its successor
    auto begin_run = [&](int t) {
      tb = reinterpret_cast<const MipTab*>(region + P.tab);
      Row r;
      locate_from(query_of(t), r);
      build(r);
      cur_valid = r.valid;
      cur_wtap = r.wtap;
      have_nxt = t + 1 < t_end && t + 1 < m_t1;
      if (have_nxt) locate_from(query_of(t + 1), nxt);
      have_nq = t + 2 < t_end && t + 2 < m_t1;
      if (have_nq) nq = query_of(t + 2);
    };
    if (t_begin < t_end) {
      stage(next_material(t_begin));
      begin_run(t_begin);
    }
    for (int tl = t_begin; tl < t_end; ++tl) {
      const int ql = tri ? (tl - m_t0) * per_tile + (row >> 3) : (tl - m_t0) * per_tile + row;
      const bool valid = cur_valid != 0;
      const float wtap = cur_wtap;
      const int64_t obase = m_o0;
      // layer 1 -> H1
      if (!tc::mbar_wait(&bar_d[w], pd, kWaitLimit)) *abort_flag = 1;
      pd ^= 1;
      tc::fence_after_sync();
      hidden_epilogue_q(td, th, m_act);
      tc::tmem_st_wait();
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&bar_h[w]);
      // the next tile's input rows, when it is of the same material
      const bool next_same = have_nxt;
      if (next_same) {
        build(nxt);
        cur_valid = nxt.valid;
        cur_wtap = nxt.wtap;
        have_nxt = false;
      }
      // layer 2 -> H2
      if (!tc::mbar_wait(&bar_d[w], pd, kWaitLimit)) *abort_flag = 1;
      pd ^= 1;
      tc::fence_after_sync();
      hidden_epilogue_q(td, th, m_act);
      tc::tmem_st_wait();
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&bar_h[w]);
      if (*abort_flag) break;
      // the tile after next, when it is of the current material (its query
      // was loaded a tile ago), then the query of its successor
      if (next_same && have_nq) {
        locate_from(nq, nxt);
        have_nxt = true;
        have_nq = tl + 3 < t_end && tl + 3 < m_t1;
        if (have_nq) nq = query_of(tl + 3);
      }
      // layer 3 -> output
      if (!tc::mbar_wait(&bar_o[w], po, kWaitLimit)) *abort_flag = 1;
      po ^= 1;
      tc::fence_after_sync();
      float yv[16];
      tc::tmem_ld16(td3, yv);
      tc::tmem_ld_wait();
      tc::fence_before_sync();
      out_activate(yv, m_oact);
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
      const int C = m_C;
      if (valid && (!tri || (row & 7) == 0)) {
        // vector stores need the material's output block 16-byte aligned
        const int eb = out_dtype == NTC_DTYPE_U8 ? 1 : (out_dtype == NTC_DTYPE_F16 ? 2 : 4);
        if (((obase * eb) & 15) == 0) {
          store_texel(static_cast<uint8_t*>(out) + obase * eb, out_dtype, ql, C, yv);
        } else if (out_dtype == NTC_DTYPE_U8) {
          uint8_t* o = static_cast<uint8_t*>(out) + obase + (int64_t)ql * C;
#pragma unroll
          for (int c = 0; c < 16; ++c)
            if (c < C) o[c] = (uint8_t)__float2uint_rn(__saturatef(yv[c]) * 255.f);
        } else if (out_dtype == NTC_DTYPE_F16) {
          __half* o = static_cast<__half*>(out) + obase + (int64_t)ql * C;
#pragma unroll
          for (int c = 0; c < 16; ++c)
            if (c < C) o[c] = __float2half_rn(yv[c]);
        } else {
          float* o = static_cast<float*>(out) + obase + (int64_t)ql * C;
#pragma unroll
          for (int c = 0; c < 16; ++c)
            if (c < C) o[c] = yv[c];
        }
      }
      if (*abort_flag) break;
      // a material boundary: every MMA of this warpgroup is done; restage,
      // then the next tile's input rows and its successor's cells
      if (!next_same && tl + 1 < t_end) {
        stage(next_material(tl + 1));
        begin_run(tl + 1);
      }
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

template <int CLS>
cudaError_t launch_ws_batched(const BatchHeader* dev, int64_t total_tiles, uint32_t plan_bytes,
                              const float* uvl, void* out, int out_dtype, int filter,
                              cudaStream_t s) {
  const WsBatchSmem S(plan_bytes);
  cudaError_t e = cudaFuncSetAttribute(decode_ws_batched_kernel<CLS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S.total);
  if (e != cudaSuccess) return e;
  const int64_t cap = sm_count();
  const int64_t ctas = (total_tiles + kWsCompute - 1) / kWsCompute;
  const int grid = (int)(ctas < cap ? ctas : cap);
  decode_ws_batched_kernel<CLS><<<grid, kWsThreads, S.total, s>>>(dev, uvl, out, out_dtype, filter,
                                                                  plan_bytes, status_word());
  return cudaGetLastError();
}

}  // namespace

int fast_class(const ntc_material& m) {
  const Plan P(m, false, fast_layout_ok(m));
  if (!P.fast) return 0;
  if (P.learned) return -1;
  return 1 + 3 * grid_class(m.c0, P.cb0) + grid_class(m.c1, P.cb1);
}

uint32_t ws_plan_bytes(const ntc_material& m, bool fast) {
  const Plan P(m, false, fast);
  return P.total | ((uint32_t)P.k_int << 24);
}
uint32_t ws_batched_smem(uint32_t packed) { return WsBatchSmem(packed).total; }

cudaError_t launch_decode_ws_batched(const BatchHeader* dev, int64_t total_tiles,
                                     uint32_t plan_bytes, int cls, const float* uvl, void* out,
                                     int out_dtype, int filter, cudaStream_t s) {
  if (total_tiles == 0) return cudaSuccess;
  switch (cls) {
    case 0: return launch_ws_batched<0>(dev, total_tiles, plan_bytes, uvl, out, out_dtype, filter, s);
    case 5: return launch_ws_batched<5>(dev, total_tiles, plan_bytes, uvl, out, out_dtype, filter, s);
    default: return launch_ws_batched<-1>(dev, total_tiles, plan_bytes, uvl, out, out_dtype, filter, s);
  }
}

cudaError_t launch_decode_ws(const ntc_material& m, const float* uvl, int64_t n, void* out,
                             int out_dtype, int filter, uint64_t jkey, cudaStream_t s, bool fast) {
  if (m.hidden_layers == 3) {  // a third hidden layer: the paper's profiles, else run time
    if (!fast) return launch_ws<0, false, true>(m, uvl, n, out, out_dtype, filter, jkey, s);
    const Plan P(m, false, true);
    const int cls = P.vq ? -1 : (P.learned ? 11 : 1) + 3 * grid_class(m.c0, P.cb0) +
                                    grid_class(m.c1, P.cb1);
    if (cls == 16) return launch_ws<16, false, true>(m, uvl, n, out, out_dtype, filter, jkey, s);
    if (cls == 18) return launch_ws<18, false, true>(m, uvl, n, out, out_dtype, filter, jkey, s);
    return launch_ws<-1, false, true>(m, uvl, n, out, out_dtype, filter, jkey, s);
  }
  if (!fast) return launch_ws<0, false>(m, uvl, n, out, out_dtype, filter, jkey, s);
  const Plan P(m, false, true);
  if (P.vq) return launch_ws<-1, false>(m, uvl, n, out, out_dtype, filter, jkey, s);
  if (P.learned) {
    // the paper's profiles 0.5 and 2.25 (4-bit G0 of 12 / 16 channels, G1 of
    // 16 / 12) as compile-time classes, other learned layouts at run time
    switch (11 + 3 * grid_class(m.c0, P.cb0) + grid_class(m.c1, P.cb1)) {
      case 16: return launch_ws<16, false>(m, uvl, n, out, out_dtype, filter, jkey, s);
      case 18: return launch_ws<18, false>(m, uvl, n, out, out_dtype, filter, jkey, s);
      default: return launch_ws<-1, false>(m, uvl, n, out, out_dtype, filter, jkey, s);
    }
  }
  switch (1 + 3 * grid_class(m.c0, P.cb0) + grid_class(m.c1, P.cb1)) {
    case 1: return launch_ws<1, false>(m, uvl, n, out, out_dtype, filter, jkey, s);
    case 2: return launch_ws<2, false>(m, uvl, n, out, out_dtype, filter, jkey, s);
    case 3: return launch_ws<3, false>(m, uvl, n, out, out_dtype, filter, jkey, s);
    case 4: return launch_ws<4, false>(m, uvl, n, out, out_dtype, filter, jkey, s);
    case 5: return launch_ws<5, false>(m, uvl, n, out, out_dtype, filter, jkey, s);
    case 6: return launch_ws<6, false>(m, uvl, n, out, out_dtype, filter, jkey, s);
    case 7: return launch_ws<7, false>(m, uvl, n, out, out_dtype, filter, jkey, s);
    case 8: return launch_ws<8, false>(m, uvl, n, out, out_dtype, filter, jkey, s);
    default: return launch_ws<9, false>(m, uvl, n, out, out_dtype, filter, jkey, s);
  }
}

}  // namespace ntc
