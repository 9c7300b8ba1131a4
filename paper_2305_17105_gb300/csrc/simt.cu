// FP32 CUDA-core form of the NTC hot path: random-access decode (nearest and
// trilinear) and the fused forward + loss + backward of the optimisation
// (Sec. 4.3-4.5, 5.1, 5.3).  One query / training texel per thread, the
// material's weights staged once per CTA in shared memory, every activation
// recomputed on chip (nothing but the per-tile operands of the weight-gradient
// reduction touches memory).
#include "ntc_device.cuh"
#include "ntc_internal.h"

namespace ntc {

namespace {

constexpr int kThreads = kTile;  // 128

// Shared-memory weights in float: W1^T [K][64] (input-major, for the
// forward), W2 [64][64] and W3 [16][64] ([out][in]; W3 rows >= C are zero),
// b1, b2, b3 (16), and with a third hidden layer Wh [64][64], bh.  Offsets in
// floats, all multiples of 4.
struct SW {
  int w1t, w2, w3, b1, b2, b3, wh, bh, size;
  bool h3;
  __host__ __device__ SW(int K, bool third) {
    w1t = 0;
    w2 = w1t + K * kHidden;
    w3 = w2 + kHidden * kHidden;
    b1 = w3 + kMaxC * kHidden;
    b2 = b1 + kHidden;
    b3 = b2 + kHidden;
    wh = b3 + kMaxC;
    bh = wh + (third ? kHidden * kHidden : 0);
    size = bh + (third ? kHidden : 0);
    h3 = third;
  }
};

__device__ void stage_weights(const ntc_material& M, const SW& L, float* s) {
  const int C = M.channels, K = M.k_in;
  for (int i = threadIdx.x; i < kHidden * K; i += blockDim.x) {
    const int o = i / K, k = i - o * K;
    s[L.w1t + k * kHidden + o] = load_weight(M, 0, i);
  }
  for (int i = threadIdx.x; i < kHidden * kHidden; i += blockDim.x) s[L.w2 + i] = load_weight(M, 1, i);
  for (int i = threadIdx.x; i < kMaxC * kHidden; i += blockDim.x)
    s[L.w3 + i] = (i / kHidden) < C ? load_weight(M, 2, i) : 0.f;
  for (int i = threadIdx.x; i < kHidden; i += blockDim.x) {
    s[L.b1 + i] = M.b[0][i];
    s[L.b2 + i] = M.b[1][i];
  }
  for (int i = threadIdx.x; i < kMaxC; i += blockDim.x) s[L.b3 + i] = i < C ? M.b[2][i] : 0.f;
  if (L.h3) {
    for (int i = threadIdx.x; i < kHidden * kHidden; i += blockDim.x) s[L.wh + i] = load_weight_h3(M, i);
    for (int i = threadIdx.x; i < kHidden; i += blockDim.x) s[L.bh + i] = M.b_h3[i];
  }
}

// Layer 1: z = W1 x + b1 with x a K-float row in shared memory (16-byte
// aligned) and W1^T input-major: 64 independent accumulators per thread,
// one broadcast float4 of weights per four FMAs.
__device__ __forceinline__ void layer1(const float* __restrict__ w1t, const float* __restrict__ b1,
                                       const float* __restrict__ xrow, int K, float (&z)[kHidden]) {
#pragma unroll
  for (int o = 0; o < kHidden; ++o) z[o] = b1[o];
#pragma unroll 1
  for (int i = 0; i < K; i += 4) {
    const float4 xv = *reinterpret_cast<const float4*>(xrow + i);
    const float xs[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float* wr = w1t + (i + j) * kHidden;
#pragma unroll
      for (int o = 0; o < kHidden; o += 4) {
        const float4 w = *reinterpret_cast<const float4*>(wr + o);
        z[o] = fmaf(w.x, xs[j], z[o]);
        z[o + 1] = fmaf(w.y, xs[j], z[o + 1]);
        z[o + 2] = fmaf(w.z, xs[j], z[o + 2]);
        z[o + 3] = fmaf(w.w, xs[j], z[o + 3]);
      }
    }
  }
}

// y = W x + b for W [OUT][64] in shared memory, x in registers; four outputs
// at a time so each thread carries four independent FMA chains.
template <int OUT>
__device__ __forceinline__ void dense64(const float* __restrict__ W, const float* __restrict__ b,
                                        const float (&x)[kHidden], float (&y)[OUT]) {
#pragma unroll
  for (int o = 0; o < OUT; o += 4) {
    float a0 = b[o], a1 = b[o + 1], a2 = b[o + 2], a3 = b[o + 3];
#pragma unroll
    for (int i = 0; i < kHidden; i += 4) {
      const float4 w0 = *reinterpret_cast<const float4*>(W + (o + 0) * kHidden + i);
      const float4 w1 = *reinterpret_cast<const float4*>(W + (o + 1) * kHidden + i);
      const float4 w2 = *reinterpret_cast<const float4*>(W + (o + 2) * kHidden + i);
      const float4 w3 = *reinterpret_cast<const float4*>(W + (o + 3) * kHidden + i);
      a0 = fmaf(w0.x, x[i], a0); a0 = fmaf(w0.y, x[i + 1], a0);
      a0 = fmaf(w0.z, x[i + 2], a0); a0 = fmaf(w0.w, x[i + 3], a0);
      a1 = fmaf(w1.x, x[i], a1); a1 = fmaf(w1.y, x[i + 1], a1);
      a1 = fmaf(w1.z, x[i + 2], a1); a1 = fmaf(w1.w, x[i + 3], a1);
      a2 = fmaf(w2.x, x[i], a2); a2 = fmaf(w2.y, x[i + 1], a2);
      a2 = fmaf(w2.z, x[i + 2], a2); a2 = fmaf(w2.w, x[i + 3], a2);
      a3 = fmaf(w3.x, x[i], a3); a3 = fmaf(w3.y, x[i + 1], a3);
      a3 = fmaf(w3.z, x[i + 2], a3); a3 = fmaf(w3.w, x[i + 3], a3);
    }
    y[o] = a0; y[o + 1] = a1; y[o + 2] = a2; y[o + 3] = a3;
  }
}

// din = W^T d for W [OUT][64]: outer-product order over the outputs so that
// every weight row is one broadcast read.
template <int OUT>
__device__ __forceinline__ void dense64_t(const float* __restrict__ W, const float (&d)[OUT],
                                          float (&din)[kHidden]) {
#pragma unroll
  for (int i = 0; i < kHidden; ++i) din[i] = 0.f;
#pragma unroll
  for (int o = 0; o < OUT; ++o) {
#pragma unroll
    for (int i = 0; i < kHidden; i += 4) {
      const float4 w = *reinterpret_cast<const float4*>(W + o * kHidden + i);
      din[i] = fmaf(w.x, d[o], din[i]);
      din[i + 1] = fmaf(w.y, d[o], din[i + 1]);
      din[i + 2] = fmaf(w.z, d[o], din[i + 2]);
      din[i + 3] = fmaf(w.w, d[o], din[i + 3]);
    }
  }
}

// Full decoder MLP on one input row held in shared memory.
__device__ __forceinline__ void mlp_forward(const float* sw, const SW& L, const float* xrow, int K,
                                            int act, int out_act, float (&y)[kMaxC]) {
  float h1[kHidden];
  layer1(sw + L.w1t, sw + L.b1, xrow, K, h1);
#pragma unroll
  for (int i = 0; i < kHidden; ++i) h1[i] = act_fwd(act, h1[i]);
  float h2[kHidden];
  dense64<kHidden>(sw + L.w2, sw + L.b2, h1, h2);
#pragma unroll
  for (int i = 0; i < kHidden; ++i) h2[i] = act_fwd(act, h2[i]);
  if (L.h3) {
    // third hidden layer (Sec. 4.4: activations on three layers)
    dense64<kHidden>(sw + L.wh, sw + L.bh, h2, h1);
#pragma unroll
    for (int i = 0; i < kHidden; ++i) h2[i] = act_fwd(act, h1[i]);
  }
  dense64<kMaxC>(sw + L.w3, sw + L.b3, h2, y);
#pragma unroll
  for (int c = 0; c < kMaxC; ++c) y[c] = out_fwd(out_act, y[c]);
}

struct RowSink {
  float* row;
  __device__ __forceinline__ void operator()(int i, float v) const { row[i] = v; }
};

// Row stride of the per-thread input rows: K + 4 keeps rows 16-byte aligned
// and makes a quarter-warp's float4 reads hit eight disjoint bank groups.
__host__ __device__ __forceinline__ int row_stride(int K) { return K + 4; }

__global__ void __launch_bounds__(kThreads) decode_simt_kernel(
    const ntc_material M, const float* __restrict__ uvl, int64_t n, void* __restrict__ out,
    int out_dtype, int filter, int noise, uint64_t nkey, uint64_t jkey) {
  extern __shared__ __align__(16) float smem[];
  const int K = M.k_in, C = M.channels;
  const SW L(K, M.hidden_layers == 3);
  float* sw = smem;
  stage_weights(M, L, sw);
  __syncthreads();
  RowSink sink{smem + L.size + threadIdx.x * row_stride(K)};
  for (int64_t q = (int64_t)blockIdx.x * kThreads + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * kThreads) {
    const float u = uvl[3 * q], v = uvl[3 * q + 1], l = uvl[3 * q + 2];
    float y[kMaxC];
    if (filter == NTC_FILTER_NEAREST) {
      int x, yy, m;
      query_texel(M, u, v, l, x, yy, m);
      featurize(M, x, yy, m, noise != 0, nkey, sink);
      mlp_forward(sw, L, sink.row, K, M.act, M.out_act, y);
    } else if (filter == NTC_FILTER_STOCHASTIC) {
      const uint64_t h = splitmix64(jkey ^ (uint64_t)q);
      const int m = stochastic_mip(l, M.mips, h);
      const int x = stochastic_coord(u, mip_dim(M.width, m), (uint32_t)(h >> 40));
      const int yy = stochastic_coord(v, mip_dim(M.height, m), (uint32_t)(h >> 16) & 0xFFFFFFu);
      featurize(M, x, yy, m, false, 0, sink);
      mlp_forward(sw, L, sink.row, K, M.act, M.out_act, y);
    } else {
      // software trilinear filtering (Sec. 5.3): 2x2 texels on two mips
      const float lam = !(l >= 0.f) ? 0.f : fminf(l, (float)(M.mips - 1));
      const int m0 = min((int)floorf(lam), M.mips - 1);
      const int m1 = min(m0 + 1, M.mips - 1);
      const float t = lam - (float)m0;
#pragma unroll
      for (int c = 0; c < kMaxC; ++c) y[c] = 0.f;
#pragma unroll 1
      for (int tap = 0; tap < 8; ++tap) {
        const int s = tap >> 2, dx = tap & 1, dy = (tap >> 1) & 1;
        const int m = s ? m1 : m0;
        const float wl = s ? t : 1.f - t;
        const int wm = mip_dim(M.width, m), hm = mip_dim(M.height, m);
        const float px = u * (float)wm - 0.5f, py = v * (float)hm - 0.5f;
        const float fx0 = floorf(px), fy0 = floorf(py);
        const float fx = px - fx0, fy = py - fy0;
        const int xx = (((int)fx0 + dx) % wm + wm) % wm, yv = (((int)fy0 + dy) % hm + hm) % hm;
        const float w = wl * (dx ? fx : 1.f - fx) * (dy ? fy : 1.f - fy);
        featurize(M, xx, yv, m, false, 0, sink);
        float yt[kMaxC];
        mlp_forward(sw, L, sink.row, K, M.act, M.out_act, yt);
#pragma unroll
        for (int c = 0; c < kMaxC; ++c) y[c] = fmaf(w, yt[c], y[c]);
      }
    }
    if (out_dtype == NTC_DTYPE_F32) {
      float* o = static_cast<float*>(out) + q * C;
#pragma unroll
      for (int c = 0; c < kMaxC; ++c)
        if (c < C) o[c] = y[c];
    } else if (out_dtype == NTC_DTYPE_U8) {
      uint8_t* o = static_cast<uint8_t*>(out) + q * C;
#pragma unroll
      for (int c = 0; c < kMaxC; ++c)
        if (c < C) o[c] = (uint8_t)__float2uint_rn(__saturatef(y[c]) * 255.f);
    } else {
      __half* o = static_cast<__half*>(out) + q * C;
#pragma unroll
      for (int c = 0; c < kMaxC; ++c)
        if (c < C) o[c] = __float2half_rn(y[c]);
    }
  }
}

// Calibration of the FP8-E4M3 form: the largest magnitude of each layer's
// input (the feature row, act(Z1), act(Z2)) over the nearest decodes of the
// queries, in FP32, reduced per warp and merged into amax[3] (float bits;
// every value is non-negative, so the unsigned order is the float order).
__global__ void __launch_bounds__(kThreads) f8_calib_kernel(const ntc_material M,
                                                            const float* __restrict__ uvl,
                                                            int64_t n, uint32_t* amax) {
  extern __shared__ __align__(16) float smem[];
  const int K = M.k_in;
  const SW L(K, false);
  float* sw = smem;
  stage_weights(M, L, sw);
  __syncthreads();
  RowSink sink{smem + L.size + threadIdx.x * row_stride(K)};
  float mx[3] = {0.f, 0.f, 0.f};
  for (int64_t q = (int64_t)blockIdx.x * kThreads + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * kThreads) {
    int x, yy, m;
    query_texel(M, uvl[3 * q], uvl[3 * q + 1], uvl[3 * q + 2], x, yy, m);
    featurize(M, x, yy, m, false, 0, sink);
    for (int k = 0; k < K; ++k) mx[0] = fmaxf(mx[0], fabsf(sink.row[k]));
    float h1[kHidden], h2[kHidden];
    layer1(sw + L.w1t, sw + L.b1, sink.row, K, h1);
#pragma unroll
    for (int i = 0; i < kHidden; ++i) {
      h1[i] = act_fwd(M.act, h1[i]);
      mx[1] = fmaxf(mx[1], fabsf(h1[i]));
    }
    dense64<kHidden>(sw + L.w2, sw + L.b2, h1, h2);
#pragma unroll
    for (int i = 0; i < kHidden; ++i) mx[2] = fmaxf(mx[2], fabsf(act_fwd(M.act, h2[i])));
  }
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    float v = mx[l];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&amax[l], __float_as_uint(v));
  }
}

// amax[3] (float bits) -> the activation scales s_a[l]: the smallest power
// of two with amax / s_a <= 448 (the largest finite E4M3 value); 1 for an
// all-zero input.
__global__ void f8_scales_kernel(const uint32_t* amax, float* sa) {
  const int l = threadIdx.x;
  if (l >= 3) return;
  const float a = __uint_as_float(amax[l]);
  float s = 1.f;
  if (a > 0.f && a < __int_as_float(0x7f800000)) {
    int e = 0;
    const float f = frexpf(a / 448.f, &e);  // a / 448 = f 2^e, f in [0.5, 1)
    if (f == 0.5f) e -= 1;                    // an exact power of two needs no headroom
    e = e < -126 ? -126 : (e > 127 ? 127 : e);
    s = __int_as_float((127 + e) << 23);
  }
  sa[l] = s;
}

// ---------------------------------------------------------------------------
// Fused forward + loss + backward (Sec. 5.1): per 128-texel tile,
//  A) per thread: texel, features (+noise), forward; the pre-activations Z1,
//     Z2 and the output gradient D3 go to shared memory;
//  C3) CTA: dW3 += D3^T act(Z2), db3;
//  B1) per thread: D2 over Z2's row, D1 in registers, grid-gradient
//      scatter-add of dX through the bilinear taps;
//  C2) CTA: dW2 += D2^T act(Z1), db2;
//  B2) per thread: D1 over Z1's row;
//  C1) CTA: dW1 += D1^T X, db1.
// Weight gradients accumulate in shared memory over all tiles of the CTA and
// are flushed once with atomics.
// ---------------------------------------------------------------------------
struct SB {
  SW w;
  int g, x, z1, z2, d3, dx, red, size;
  __host__ __device__ explicit SB(int K) : w(K, false) {
    g = w.size;                                  // gradient accumulators, layout of w
    x = g + w.size;                              // [128][K+4]
    z1 = x + kTile * row_stride(K);              // [128][65]
    z2 = z1 + kTile * (kHidden + 1);             // [128][65]
    d3 = z2 + kTile * (kHidden + 1);             // [128][17]
    dx = d3 + kTile * (kMaxC + 1);               // [128][K+1]: dX over the feature slots
    red = dx + kTile * (K + 1);                  // [4]
    size = red + 4;
  }
};

__global__ void __launch_bounds__(kThreads, 1) backward_simt_kernel(const ntc_material M,
                                                                    const BwdArgs A) {
  extern __shared__ __align__(16) float smem[];
  const int K = M.k_in, C = M.channels;
  const int W0 = M.interp0 == NTC_INTERP_LEARNED ? 4 * M.c0 : M.c0;  // width of the G0 slots
  const int F = W0 + M.c1;
  const SB S(K);
  float* sw = smem;
  float* sg = smem + S.g;
  stage_weights(M, S.w, sw);
  for (int i = threadIdx.x; i < S.w.size; i += blockDim.x) sg[i] = 0.f;
  const int tid = threadIdx.x;
  const int64_t step = A.step_dev ? *A.step_dev : A.noise_step;
  const uint64_t nkey = rng_key(A.noise_seed, noise_stream(step));
  const uint64_t skey = rng_key(A.sample_seed, sampler_stream(step));
  float* xrow = smem + S.x + tid * row_stride(K);
  float* z1row = smem + S.z1 + tid * (kHidden + 1);
  float* z2row = smem + S.z2 + tid * (kHidden + 1);
  float* d3row = smem + S.d3 + tid * (kMaxC + 1);
  float* dxrow = smem + S.dx + tid * (K + 1);
  RowSink sink{xrow};
  float loss_acc = 0.f;
  __syncthreads();

  for (int64_t base = (int64_t)blockIdx.x * kTile; base < A.n; base += (int64_t)gridDim.x * kTile) {
    const int64_t i = base + tid;
    const bool valid = i < A.n;
    // ---- A: forward --------------------------------------------------------
    int x = 0, y = 0, m = 0;
    if (valid) {
      if (A.uvl) query_texel(M, A.uvl[3 * i], A.uvl[3 * i + 1], A.uvl[3 * i + 2], x, y, m);
      else sample_train_texel(A.crops != 0, skey, i, M.width, M.height, M.mips, x, y, m);
    }
    featurize(M, x, y, m, A.noise != 0, nkey, sink);
    float d1[kHidden];  // h1 during the forward, dZ1 during the backward
    layer1(sw + S.w.w1t, sw + S.w.b1, xrow, K, d1);
#pragma unroll
    for (int k = 0; k < kHidden; ++k) { z1row[k] = d1[k]; d1[k] = act_fwd(M.act, d1[k]); }
    float z2[kHidden];
    dense64<kHidden>(sw + S.w.w2, sw + S.w.b2, d1, z2);
#pragma unroll
    for (int k = 0; k < kHidden; ++k) { z2row[k] = z2[k]; z2[k] = act_fwd(M.act, z2[k]); }
    float d3[kMaxC];
    dense64<kMaxC>(sw + S.w.w3, sw + S.w.b3, z2, d3);
    {
      const int wm = mip_dim(M.width, m);
      const uint8_t* trow = A.train ? A.target + A.tgt_off[m] + ((int64_t)y * wm + x) * C : nullptr;
#pragma unroll
      for (int c = 0; c < kMaxC; ++c) {
        float g = 0.f;
        if (valid && c < C) {
          const float yc = out_fwd(M.out_act, d3[c]);
          float dy;
          if (A.train) {
            const float e = yc - (float)trow[c] * (1.f / 255.f);
            loss_acc = fmaf(e, e, loss_acc);
            dy = 2.f * e;
          } else {
            dy = A.dout[i * C + c];
          }
          g = M.out_act == NTC_OUT_IDENTITY ? dy : dy * yc * (1.f - yc);
        }
        d3[c] = g;
        d3row[c] = g;
      }
    }
    __syncthreads();
    // ---- C3: dW3 += D3^T act(Z2), db3 -----------------------------------
    {
      const int c0 = 4 * (tid & 3), i0 = 2 * (tid >> 2);
      float acc[4][2] = {};
      float accb = 0.f;
#pragma unroll 4
      for (int b = 0; b < kTile; ++b) {
        const float* zr = smem + S.z2 + b * (kHidden + 1);
        const float* dr = smem + S.d3 + b * (kMaxC + 1);
        const float h0 = act_fwd(M.act, zr[i0]), h1 = act_fwd(M.act, zr[i0 + 1]);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          acc[r][0] = fmaf(dr[c0 + r], h0, acc[r][0]);
          acc[r][1] = fmaf(dr[c0 + r], h1, acc[r][1]);
        }
        if (tid < kMaxC) accb += dr[tid];
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        sg[S.w.w3 + (c0 + r) * kHidden + i0] += acc[r][0];
        sg[S.w.w3 + (c0 + r) * kHidden + i0 + 1] += acc[r][1];
      }
      if (tid < kMaxC) sg[S.w.b3 + tid] += accb;
    }
    // ---- B1: D2 over Z2's row, D1 in registers, grid scatter ------------
    {
      float dh[kHidden];
      dense64_t<kMaxC>(sw + S.w.w3, d3, dh);
#pragma unroll
      for (int k = 0; k < kHidden; ++k) dh[k] *= act_grad(M.act, z2row[k]);
      __syncthreads();  // every thread is done reading Z2 (C3)
#pragma unroll
      for (int k = 0; k < kHidden; ++k) z2row[k] = dh[k];
      dense64_t<kHidden>(sw + S.w.w2, dh, d1);
#pragma unroll
      for (int k = 0; k < kHidden; ++k) d1[k] *= act_grad(M.act, z1row[k]);
    }
    if (A.grids && valid) {
      // dX = W1^T D1 over the feature slots (through shared memory, so the
      // runtime offsets of the G0 / G1 slots need no register indexing)
      const float* w1t = sw + S.w.w1t;
#pragma unroll 1
      for (int s = 0; s < F; ++s) {
        float a = 0.f;
#pragma unroll
        for (int o = 0; o < kHidden; o += 4) {
          const float4 w = *reinterpret_cast<const float4*>(w1t + s * kHidden + o);
          a = fmaf(w.x, d1[o], a);
          a = fmaf(w.y, d1[o + 1], a);
          a = fmaf(w.z, d1[o + 2], a);
          a = fmaf(w.w, d1[o + 3], a);
        }
        dxrow[s] = a;
      }
      const int j = level_of_mip(m, M.levels);
      const int wm = mip_dim(M.width, m), hm = mip_dim(M.height, m);
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const ntc_level& Lv = M.lv[j];
        float* g = k ? A.g.grid1[j] : A.g.grid0[j];
        if (!g) continue;
        const int c = k ? M.c1 : M.c0;
        const bool learned = k == 0 && W0 != M.c0;
        const Taps t = bilinear_taps(x, y, wm, hm, k ? Lv.g1_w : Lv.g0_w, k ? Lv.g1_h : Lv.g0_h);
#pragma unroll
        for (int tp = 0; tp < 4; ++tp) {
          // bilinear: the tap's weight on the shared slots; learned
          // interpolation: the tap's own slots with weight 1
          const float* dk = dxrow + (k ? W0 : (learned ? tp * c : 0));
          const float wgt = (learned ? 1.f : t.w[tp]) * A.grad_scale;
          float* gp = g + (size_t)t.cell[tp] * c;
          if ((c & 3) == 0) {
            for (int c4 = 0; 4 * c4 < c; ++c4)
              atomicAdd(reinterpret_cast<float4*>(gp) + c4,
                        make_float4(dk[4 * c4] * wgt, dk[4 * c4 + 1] * wgt, dk[4 * c4 + 2] * wgt,
                                    dk[4 * c4 + 3] * wgt));
          } else {
            for (int ch = 0; ch < c; ++ch) atomicAdd(gp + ch, dk[ch] * wgt);
          }
        }
      }
    }
    __syncthreads();  // D2 complete in Z2's rows
    // ---- C2: dW2 += D2^T act(Z1), db2 -----------------------------------
    {
      const int o0 = 4 * (tid & 15), i0 = 8 * (tid >> 4);
      float acc[4][8] = {};
      float accb = 0.f;
#pragma unroll 2
      for (int b = 0; b < kTile; ++b) {
        const float* zr = smem + S.z1 + b * (kHidden + 1);
        const float* dr = smem + S.z2 + b * (kHidden + 1);
        float h[8];
#pragma unroll
        for (int s = 0; s < 8; ++s) h[s] = act_fwd(M.act, zr[i0 + s]);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const float d = dr[o0 + r];
#pragma unroll
          for (int s = 0; s < 8; ++s) acc[r][s] = fmaf(d, h[s], acc[r][s]);
        }
        if (tid < kHidden) accb += dr[tid];
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int s = 0; s < 8; ++s) sg[S.w.w2 + (o0 + r) * kHidden + i0 + s] += acc[r][s];
      if (tid < kHidden) sg[S.w.b2 + tid] += accb;
    }
    __syncthreads();  // Z1 no longer read
    // ---- B2: D1 over Z1's row ----------------------------------------------
#pragma unroll
    for (int k = 0; k < kHidden; ++k) z1row[k] = d1[k];
    __syncthreads();
    // ---- C1: dW1 += D1^T X (4x8 output blocks), db1 ------------------------
    {
      const int nblk = (kHidden / 4) * (K / 8);
      for (int blk = tid; blk < nblk; blk += kThreads) {
        const int o0 = 4 * (blk & 15), i0 = 8 * (blk >> 4);
        float acc[4][8] = {};
#pragma unroll 2
        for (int b = 0; b < kTile; ++b) {
          const float* xr = smem + S.x + b * row_stride(K);
          const float* dr = smem + S.z1 + b * (kHidden + 1);
          const float4 xa = *reinterpret_cast<const float4*>(xr + i0);
          const float4 xb = *reinterpret_cast<const float4*>(xr + i0 + 4);
          const float xv[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const float d = dr[o0 + r];
#pragma unroll
            for (int s = 0; s < 8; ++s) acc[r][s] = fmaf(d, xv[s], acc[r][s]);
          }
        }
        // dW1 is [64][K] row-major in the accumulator (the flush layout)
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int s = 0; s < 8; ++s) sg[S.w.w1t + (o0 + r) * K + i0 + s] += acc[r][s];
      }
      if (tid < kHidden) {
        float accb = 0.f;
        for (int b = 0; b < kTile; ++b) accb += smem[S.z1 + b * (kHidden + 1) + tid];
        sg[S.w.b1 + tid] += accb;
      }
    }
    __syncthreads();  // tile buffers free
  }

  // ---- flush the CTA's weight gradients and loss ---------------------------
  const float gs = A.grad_scale;
  if (A.g.w[0])
    for (int i = tid; i < kHidden * K; i += blockDim.x) atomicAdd(A.g.w[0] + i, sg[S.w.w1t + i] * gs);
  if (A.g.w[1])
    for (int i = tid; i < kHidden * kHidden; i += blockDim.x)
      atomicAdd(A.g.w[1] + i, sg[S.w.w2 + i] * gs);
  if (A.g.w[2])
    for (int i = tid; i < C * kHidden; i += blockDim.x) atomicAdd(A.g.w[2] + i, sg[S.w.w3 + i] * gs);
  if (A.g.b[0])
    for (int i = tid; i < kHidden; i += blockDim.x) atomicAdd(A.g.b[0] + i, sg[S.w.b1 + i] * gs);
  if (A.g.b[1])
    for (int i = tid; i < kHidden; i += blockDim.x) atomicAdd(A.g.b[1] + i, sg[S.w.b2 + i] * gs);
  if (A.g.b[2])
    for (int i = tid; i < C; i += blockDim.x) atomicAdd(A.g.b[2] + i, sg[S.w.b3 + i] * gs);
  if (A.train && A.loss) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) loss_acc += __shfl_xor_sync(0xffffffffu, loss_acc, o);
    float* red = smem + S.red;
    if ((tid & 31) == 0) red[tid >> 5] = loss_acc;
    __syncthreads();
    if (tid == 0) atomicAdd(A.loss, (red[0] + red[1] + red[2] + red[3]) * A.loss_scale);
  }
}

}  // namespace

cudaError_t launch_decode_simt(const ntc_material& m, const float* uvl, int64_t n, void* out,
                               int out_dtype, int filter, int noise, uint64_t noise_seed,
                               int64_t noise_step, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const uint64_t nkey = rng_key(noise_seed, noise_stream(noise_step));
  const uint64_t jkey = jitter_key(noise_seed, noise_step);
  const SW L(m.k_in, m.hidden_layers == 3);
  const size_t smem = (size_t)(L.size + kThreads * row_stride(m.k_in)) * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(decode_simt_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, decode_simt_kernel, kThreads, smem);
  if (e != cudaSuccess) return e;
  const int64_t tiles = (n + kThreads - 1) / kThreads;
  const int64_t cap = (int64_t)sm_count() * (per_sm > 0 ? per_sm : 1);
  const int grid = (int)(tiles < cap ? tiles : cap);
  decode_simt_kernel<<<grid, kThreads, smem, s>>>(m, uvl, n, out, out_dtype, filter, noise, nkey,
                                                  jkey);
  return cudaGetLastError();
}

cudaError_t launch_f8_calibrate(const ntc_material& m, const float* uvl, int64_t n,
                               uint32_t* amax, float* sa, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(amax, 0, 3 * sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  if (n > 0) {
    const SW L(m.k_in, false);
    const size_t smem = (size_t)(L.size + kThreads * row_stride(m.k_in)) * sizeof(float);
    e = cudaFuncSetAttribute(f8_calib_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (n + kThreads - 1) / kThreads;
    const int64_t cap = (int64_t)sm_count() * 4;
    f8_calib_kernel<<<(int)(tiles < cap ? tiles : cap), kThreads, smem, s>>>(m, uvl, n, amax);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  f8_scales_kernel<<<1, 32, 0, s>>>(amax, sa);
  return cudaGetLastError();
}

cudaError_t launch_backward_simt(const ntc_material& m, const BwdArgs& a, cudaStream_t s) {
  if (a.n == 0) return cudaSuccess;
  const SB S(m.k_in);
  const size_t smem = (size_t)S.size * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(backward_simt_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t tiles = (a.n + kTile - 1) / kTile;
  const int64_t cap = sm_count();
  const int grid = (int)(tiles < cap ? tiles : cap);
  backward_simt_kernel<<<grid, kThreads, smem, s>>>(m, a);
  return cudaGetLastError();
}

}  // namespace ntc
