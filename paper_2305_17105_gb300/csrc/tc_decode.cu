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
#include "tc_decode_common.cuh"

namespace ntc {

namespace {

template <bool F8, bool FAST, int kNWG>
__global__ void __launch_bounds__(kRows* kNWG, 1) decode_tc_kernel(
    const ntc_material M, const float* __restrict__ uvl, int64_t n, void* __restrict__ out,
    int out_dtype, int filter, uint64_t jkey, int* status) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ uint64_t mbar[kNWG];
  __shared__ uint32_t tmem_base;
  __shared__ int wg_abort[kNWG];
  constexpr int KSTEP = Cfg<F8>::KSTEP;
  constexpr uint32_t kCols = kNWG <= 2 ? 256 : 512;  // 128 columns per warpgroup
  const Plan P(M, F8, FAST);
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
    locate(M, tb, load_query(uvl, q0, tl < ntiles && q0 < n), filter, row, r, q0, jkey);
    if (FAST) {
      gather_fast(P, tb, r);
      build_fast(P, P, K, sm, r, TmemRow{tx});
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
    locate(M, tb, nq, filter, row, nxt, qindex(tl + stride), jkey);
    if (FAST) gather_fast(P, tb, nxt);
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
    if (row == 32) issue_layer<F8>(tw, tw + kColH, dsc + kDescW2, kHidden / KSTEP, id64, !F8, tw + kColCst, bar);
    if (FAST) build_fast(P, P, K, sm, nxt, TmemRow{tx});
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
    if (row == 64) issue_layer<F8>(tw, tw + kColH, dsc + kDescW3, kHidden / KSTEP, id16, !F8, tw + kColCst, bar);
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

template <bool F8, bool FAST, int kNWG>
cudaError_t launch_k(const ntc_material& m, const float* uvl, int64_t n, void* out, int out_dtype,
                     int filter, uint64_t jkey, cudaStream_t s) {
  const Plan P(m, F8, FAST);
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
                                                                    filter, jkey, status_word());
  return cudaGetLastError();
}

template <bool F8, bool FAST>
cudaError_t launch_shape(const ntc_material& m, const float* uvl, int64_t n, void* out,
                         int out_dtype, int filter, uint64_t jkey, cudaStream_t s, int nwg) {
  switch (nwg) {
    case 2: return launch_k<F8, FAST, 2>(m, uvl, n, out, out_dtype, filter, jkey, s);
    case 3: return launch_k<F8, FAST, 3>(m, uvl, n, out, out_dtype, filter, jkey, s);
    default: return launch_k<F8, FAST, 4>(m, uvl, n, out, out_dtype, filter, jkey, s);
  }
}

}  // namespace

// Failure-detection self-test: one thread waits, with the tensor-core
// kernels' bounded wait, on an mbarrier that nothing arrives at; when the
// limit runs out it records NTC_ERR_TIMEOUT in the status word and returns.
__global__ void selftest_wait_kernel(uint32_t limit, int* status) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_mbar_init();
    if (!tc::mbar_wait(&bar, 0, limit)) atomicExch(status, NTC_ERR_TIMEOUT);
  }
}

cudaError_t launch_selftest_wait(uint32_t limit, cudaStream_t s) {
  selftest_wait_kernel<<<1, 32, 0, s>>>(limit, status_word());
  return cudaGetLastError();
}

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
// (FP16 and FP8).
cudaError_t launch_decode_tc(const ntc_material& m, const float* uvl, int64_t n, void* out,
                             int out_dtype, int filter, uint64_t jkey, cudaStream_t s, int nwg) {
  if (n == 0) return cudaSuccess;
  if (nwg == 0) nwg = 5;
  if (nwg < 2 || nwg > 5) return cudaErrorInvalidValue;
  if (m.precision == NTC_PREC_F8) {
    if (nwg == 5) return launch_decode_ws_f8(m, uvl, n, out, out_dtype, filter, jkey, s);
    return launch_shape<true, false>(m, uvl, n, out, out_dtype, filter, jkey, s, nwg);
  }
  if (m.precision != NTC_PREC_F16) return cudaErrorInvalidValue;
  const Plan P(m, false, fast_layout_ok(m));
  // the warpgroup-pipeline kernel keeps X in 24 TMEM columns (K <= 48) and
  // runs two hidden layers
  if (nwg == 5 || P.k_int > 48 || m.hidden_layers == 3)
    return launch_decode_ws(m, uvl, n, out, out_dtype, filter, jkey, s, P.fast != 0);
  if (P.fast) return launch_shape<false, true>(m, uvl, n, out, out_dtype, filter, jkey, s, nwg);
  return launch_shape<false, false>(m, uvl, n, out, out_dtype, filter, jkey, s, nwg);
}

}  // namespace ntc
