// Element-wise kernels around the fused passes: Adam with cosine-annealed
// learning rates and quantisation-range clamping (Sec. 4.2, 5.1), the final
// quantisation and packing of the grids (Sec. 4.2), and test entry points for
// the sampler and the MLP input rows.
#include <math.h>

#include "ntc_device.cuh"
#include "ntc_internal.h"
#include "tc_ptx.cuh"

namespace ntc {

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  return n > 0 ? n : 1;
}

namespace {
__device__ int g_status_word;
}  // namespace

int* status_word() {
  static int* ptr[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  if (!ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_status_word) != cudaSuccess) return nullptr;
    ptr[dev] = static_cast<int*>(p);
  }
  return ptr[dev];
}

int read_status_word(int reset) {
  int* p = status_word();
  if (!p) return -1;
  int v = 0;
  if (cudaDeviceSynchronize() != cudaSuccess) return -1;
  if (cudaMemcpy(&v, p, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
  if (reset && v != 0) {
    const int z = 0;
    if (cudaMemcpy(p, &z, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) return -1;
  }
  return v;
}

namespace {

// The noise of channels ch and ch + 1 (ch even) of a cell: both come from
// the same 64-bit draw (the values noise_of gives for each).
__device__ __forceinline__ float2 noise_pair_of(uint64_t key, int level, int grid, int cell,
                                                int ch, int c, float q) {
  const uint64_t pairs = (uint64_t)((c + 1) >> 1);
  const uint64_t counter = ((uint64_t)(2 * level + grid) << 40) |
                           ((uint64_t)cell * pairs + (uint64_t)(ch >> 1));
  const uint64_t h = splitmix64(key ^ counter);
  const uint32_t e = (uint32_t)(h >> 40), o = (uint32_t)((h >> 16) & 0xFFFFFFu);
  return make_float2(((float)e * (1.0f / 16777216.0f) - 0.5f) * q,
                     ((float)o * (1.0f / 16777216.0f) - 0.5f) * q);
}

// One Adam step (Kingma & Ba, bias-corrected) at the device step counter t,
// learning rate lr0 (1 + cos(pi t / T)) / 2 per group, then the grid clamp
// to [-(N-1)/2 Q, N/2 Q] (Sec. 4.2: clamp after the update).  The gradient is
// zeroed for the next step; half-precision weight copies are refreshed.  Each
// thread owns kAdamPerThread consecutive elements (float4 accesses); the
// schedule factors are computed once per block in FP32.
// Block b of one material's Adam pass (A: its segments, block prefix sums).
// The step's schedule factors (cosine-annealed learning rate of both groups,
// bias corrections) and the next step's noise key, from the device counter.
struct AdamSched {
  float lr[2], ic1, ic2;
  uint64_t key;
};
__device__ __forceinline__ AdamSched adam_sched(const AdamArgs& A) {
  AdamSched c;
  const int64_t t = *A.step;
  c.key = rng_key(A.noise_seed, noise_stream(t + 1));
  const float x = (float)((double)t / (double)A.total);
  const float cosf_ = 0.5f * (1.f + cospif(x));
  c.lr[0] = A.lr[0] * cosf_;
  c.lr[1] = A.lr[1] * cosf_;
  c.ic1 = 1.f / (1.f - powf(A.beta1, (float)(t + 1)));
  c.ic2 = 1.f / (1.f - powf(A.beta2, (float)(t + 1)));
  return c;
}

// The elements of block `lb` of segment S (no barrier inside).
__device__ __forceinline__ void adam_seg_block(const AdamArgs& A, const AdamSeg& S, int64_t lb,
                                               const AdamSched& sc) {
  const float lr = sc.lr[S.group], inv_c1 = sc.ic1, inv_c2 = sc.ic2;
  const float b1 = A.beta1, b2 = A.beta2, eps = A.eps;
  const int64_t first = (lb * (int64_t)kAdamBlock + threadIdx.x) * kAdamPerThread;
  if (first >= S.len) return;
  const int64_t e0 = S.off + first;
  auto upd = [&](float p, float m, float v, float g, float& po, float& mo, float& vo) {
    mo = fmaf(b1, m, (1.f - b1) * g);
    vo = fmaf(b2, v, (1.f - b2) * g * g);
    po = p - lr * (mo * inv_c1) / (sqrtf(vo * inv_c2) + eps);
    if (S.clamp) po = fminf(fmaxf(po, S.lo), S.hi);
  };
  // the next step's noisy value of segment element k (the same FP32 sum as
  // the dense noise pass)
  const bool fold = A.fold && S.noise_c > 0;
  const uint64_t nkey = sc.key;
  auto noisy = [&](int64_t k, float po) {
    const int c = S.noise_c;
    const int64_t cell = k / c;
    const int ch = (int)(k - cell * c);
    return po + noise_of(nkey, S.noise_level, S.noise_grid, (int)cell, ch, c, S.noise_q);
  };
  if (first + kAdamPerThread <= S.len) {
    // segments start 16-byte aligned: whole float4 groups
    const float4 p = *reinterpret_cast<const float4*>(A.p + e0);
    const float4 m = *reinterpret_cast<const float4*>(A.m + e0);
    const float4 v = *reinterpret_cast<const float4*>(A.v + e0);
    const float4 g = *reinterpret_cast<const float4*>(A.g + e0);
    float4 po, mo, vo;
    upd(p.x, m.x, v.x, g.x, po.x, mo.x, vo.x);
    upd(p.y, m.y, v.y, g.y, po.y, mo.y, vo.y);
    upd(p.z, m.z, v.z, g.z, po.z, mo.z, vo.z);
    upd(p.w, m.w, v.w, g.w, po.w, mo.w, vo.w);
    *reinterpret_cast<float4*>(A.p + e0) = po;
    *reinterpret_cast<float4*>(A.m + e0) = mo;
    *reinterpret_cast<float4*>(A.v + e0) = vo;
    *reinterpret_cast<float4*>(A.g + e0) = make_float4(0.f, 0.f, 0.f, 0.f);
    if (fold) {
      float4 nv;
      const int c = S.noise_c;
      if ((c & 1) == 0) {
        // even channel counts: elements (first, first+1) and (first+2,
        // first+3) are channel pairs of one cell, one draw each
        const int64_t cell0 = first / c, cell1 = (first + 2) / c;
        const float2 n0 = noise_pair_of(nkey, S.noise_level, S.noise_grid, (int)cell0,
                                        (int)(first - cell0 * c), c, S.noise_q);
        const float2 n1 = noise_pair_of(nkey, S.noise_level, S.noise_grid, (int)cell1,
                                        (int)(first + 2 - cell1 * c), c, S.noise_q);
        nv = make_float4(po.x + n0.x, po.y + n0.y, po.z + n1.x, po.w + n1.y);
      } else {
        nv = make_float4(noisy(first, po.x), noisy(first + 1, po.y), noisy(first + 2, po.z),
                         noisy(first + 3, po.w));
      }
      *reinterpret_cast<float4*>(A.noisy + e0) = nv;
    }
    if (S.half_copy) {
      __half2* h = reinterpret_cast<__half2*>(S.half_copy + first);
      h[0] = __floats2half2_rn(po.x, po.y);
      h[1] = __floats2half2_rn(po.z, po.w);
    }
  } else {
    for (int64_t k = first; k < S.len; ++k) {
      const int64_t e = S.off + k;
      float po, mo, vo;
      upd(A.p[e], A.m[e], A.v[e], A.g[e], po, mo, vo);
      A.p[e] = po;
      A.m[e] = mo;
      A.v[e] = vo;
      A.g[e] = 0.f;
      if (fold) A.noisy[e] = noisy(k, po);
      if (S.half_copy) S.half_copy[k] = __float2half_rn(po);
    }
  }
}

// Block b of one material's Adam pass (A: its segments, block prefix sums).
__device__ __forceinline__ void adam_block(const AdamArgs& A, int64_t b) {
  __shared__ AdamSched s_sc;
  int s = 0;
  while (s + 1 < A.nseg && b >= A.block_start[s + 1]) ++s;
  const AdamSeg& S = A.seg[s];
  if (threadIdx.x == 0) s_sc = adam_sched(A);
  __syncthreads();
  if (A.freeze_grids && S.group == 0) return;
  adam_seg_block(A, S, b - A.block_start[s], s_sc);
}

__global__ void __launch_bounds__(kAdamBlock) adam_kernel(const AdamArgs A) {
  adam_block(A, blockIdx.x);
}

// Index i of the prefix-sum interval start[i] <= b < start[i + 1] (start
// non-decreasing, start[0] = 0 <= b < start[n]).
__device__ __forceinline__ int find_interval(const int64_t* start, int n, int64_t b) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (start[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Adam over every material of a batch.  Persistent: CTA j walks the
// contiguous range [T j / G, T (j+1) / G) of the batch's blocks, looking its
// material and segment up once and advancing them as its range crosses into
// the next (the descriptors live in global memory; a lookup per block would
// put chains of dependent loads before every block's work).  The last CTA
// to finish advances the step counter of every material that took part
// (each CTA has read its materials' counters before it counts itself done)
// and tags their folded noisy copies.
__global__ void __launch_bounds__(kAdamBlock) adam_batched_kernel(TrainBatchDev* D) {
  __shared__ AdamSched sc;
  const int64_t total = D->adam_blocks;
  const int64_t b0 = total * blockIdx.x / gridDim.x, b1 = total * (blockIdx.x + 1) / gridDim.x;
  int i = -1, s = 0;
  for (int64_t b = b0; b < b1; ++b) {
    if (i < 0 || b >= D->adam_start[i + 1]) {
      i = i < 0 ? find_interval(D->adam_start, D->n, b) : i + 1;
      while (b >= D->adam_start[i + 1]) ++i;  // materials without blocks
      s = 0;
      __syncthreads();  // every thread is done with the previous schedule
      if (threadIdx.x == 0) sc = adam_sched(D->adam[i]);
      __syncthreads();
    }
    const AdamArgs& A = D->adam[i];
    const int64_t lb = b - D->adam_start[i];
    while (s + 1 < A.nseg && lb >= A.block_start[s + 1]) ++s;
    const AdamSeg& S = A.seg[s];
    if (!(A.freeze_grids && S.group == 0)) adam_seg_block(A, S, lb - A.block_start[s], sc);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const uint32_t done = atomicAdd(&D->adam_done, 1u) + 1u;
    if (done == gridDim.x) {
      __threadfence();
      for (int k = 0; k < D->n; ++k)
        if (D->adam_start[k + 1] > D->adam_start[k]) {
          int64_t* st = const_cast<int64_t*>(D->adam[k].step);
          *st += 1;
          if (D->adam[k].fold && D->adam[k].noisy_tag) {
            D->adam[k].noisy_tag[0] = (int64_t)D->adam[k].noise_seed;
            D->adam[k].noisy_tag[1] = *st;
          }
        }
      D->adam_done = 0u;
      __threadfence();
    }
  }
}

__global__ void advance_step_kernel(int64_t* step, int64_t* tag, uint64_t seed) {
  *step += 1;
  if (tag) {
    tag[0] = (int64_t)seed;
    tag[1] = *step;
  }
}

// One thread per channel pair of a grid cell: both channels' noise comes
// from the same 64-bit draw (noise_of), added in FP32 exactly as the fused
// step adds it per tap.
// The previous step's Adam already wrote this step's noisy grids.
__device__ __forceinline__ bool noisy_current(const NoiseArgs& a) {
  return a.tag && a.tag[0] == (int64_t)a.seed && a.tag[1] == *a.step;
}

__device__ __forceinline__ void noise_block(const NoiseArgs& a, int64_t blk) {
  int s = 0;
  while (s + 1 < a.nseg && blk >= a.block_start[s + 1]) ++s;
  const NoiseSeg& g = a.seg[s];
  const int64_t p = (blk - a.block_start[s]) * kNoiseBlock + threadIdx.x;
  if (p >= g.pairs) return;
  const int pc = (g.c + 1) >> 1;
  const int64_t cell = p / pc;
  const int ch = 2 * (int)(p - cell * pc);
  const uint64_t key = rng_key(a.seed, noise_stream(*a.step));
  const int64_t i = g.off + cell * g.c + ch;
  float v = a.src[i];
  v += noise_of(key, g.level, g.grid, (int)cell, ch, g.c, g.q);
  a.dst[i] = v;
  if (ch + 1 < g.c) {
    float w = a.src[i + 1];
    w += noise_of(key, g.level, g.grid, (int)cell, ch + 1, g.c, g.q);
    a.dst[i + 1] = w;
  }
}

// A few CTAs per SM walk the blocks of the pass, so that a pass whose copy
// is already current costs one check per CTA.
__global__ void __launch_bounds__(kNoiseBlock) noise_grids_kernel(const NoiseArgs a) {
  if (noisy_current(a)) return;
  const int64_t blocks = a.block_start[a.nseg];
  for (int64_t b = blockIdx.x; b < blocks; b += gridDim.x) noise_block(a, b);
}

// The noise pass of every material of a batch in one launch.
// Persistent like adam_batched_kernel: a contiguous range of blocks per CTA,
// one lookup and one currency check per material it reaches; a material
// whose noisy copy is current is jumped over.
__global__ void __launch_bounds__(kNoiseBlock) noise_batched_kernel(const TrainBatchDev* D) {
  const int64_t total = D->noise_blocks;
  const int64_t b0 = total * blockIdx.x / gridDim.x, b1 = total * (blockIdx.x + 1) / gridDim.x;
  int i = -1;
  for (int64_t b = b0; b < b1; ++b) {
    if (i < 0 || b >= D->noise_start[i + 1]) {
      i = i < 0 ? find_interval(D->noise_start, D->n, b) : i + 1;
      while (b >= D->noise_start[i + 1]) ++i;
      if (noisy_current(D->noise[i])) {
        b = D->noise_start[i + 1] - 1;  // the whole material
        continue;
      }
    }
    noise_block(D->noise[i], b - D->noise_start[i]);
  }
}

// q = clamp(rint(x / Q) + N/2 - 1, 0, N - 1), ties to even, evaluated in
// double so that the index never depends on the rounding of x / Q.
__global__ void quantize_pack_kernel(const float* __restrict__ x, int64_t cells, int c, int bits,
                                     float q, uint8_t* __restrict__ packed,
                                     float* __restrict__ snapped) {
  const int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= cells) return;
  const int n = 1 << bits, off = n / 2 - 1;
  uint64_t lo = 0, hi = 0;
  for (int ch = 0; ch < c; ++ch) {
    const float v = x[cell * c + ch];
    double k = rint((double)v / (double)q) + (double)off;
    k = fmin(fmax(k, 0.0), (double)(n - 1));
    const uint64_t qi = (uint64_t)k;
    const int bit = ch * bits;
    if (bit < 64) lo |= qi << bit;
    else hi |= qi << (bit - 64);
    if (snapped) snapped[cell * c + ch] = (float)((int)qi - off) * q;
  }
  if (!packed) return;
  const int cb = cell_bytes(c, bits);
  uint8_t* p = packed + cell * cb;
  switch (cb) {
    case 1: *p = (uint8_t)lo; break;
    case 2: *reinterpret_cast<uint16_t*>(p) = (uint16_t)lo; break;
    case 4: *reinterpret_cast<uint32_t*>(p) = (uint32_t)lo; break;
    case 8: *reinterpret_cast<unsigned long long*>(p) = lo; break;
    default:
      *reinterpret_cast<uint4*>(p) =
          make_uint4((uint32_t)lo, (uint32_t)(lo >> 32), (uint32_t)hi, (uint32_t)(hi >> 32));
  }
}

__global__ void unpack_kernel(const uint8_t* __restrict__ packed, int64_t cells, int c, int bits,
                              float q, int32_t* __restrict__ idx, float* __restrict__ values) {
  const int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= cells) return;
  const int off = (1 << (bits - 1)) - 1;
  const int cb = cell_bytes(c, bits);
  const Cell cc = load_cell(packed + cell * cb, 0, cb);
  for (int ch = 0; ch < c; ++ch) {
    const int v = (int)cell_index(cc, ch, bits);
    if (idx) idx[cell * c + ch] = v;
    if (values) values[cell * c + ch] = (float)(v - off) * q;
  }
}

__global__ void sample_batch_kernel(uint64_t skey, int64_t batch, int w, int h, int mips, int crops,
                                    int32_t* __restrict__ xym) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= batch) return;
  int x, y, m;
  sample_train_texel(crops != 0, skey, i, w, h, mips, x, y, m);
  xym[3 * i] = x;
  xym[3 * i + 1] = y;
  xym[3 * i + 2] = m;
}

struct GlobalRowSink {
  float* row;
  __device__ __forceinline__ void operator()(int i, float v) const { row[i] = v; }
};

__global__ void sample_features_kernel(const ntc_material M, const float* __restrict__ uvl,
                                       int64_t n, float* __restrict__ rows, int noise,
                                       uint64_t nkey) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int x, y, m;
  query_texel(M, uvl[3 * i], uvl[3 * i + 1], uvl[3 * i + 2], x, y, m);
  GlobalRowSink sink{rows + i * M.k_in};
  featurize(M, x, y, m, noise != 0, nkey, sink);
}

inline int blocks_for(int64_t n, int per) { return (int)((n + per - 1) / per); }

}  // namespace

cudaError_t launch_adam(const AdamArgs& a, int64_t blocks, cudaStream_t s) {
  if (blocks == 0) return cudaSuccess;
  adam_kernel<<<(unsigned)blocks, kAdamBlock, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_noise_grids(const NoiseArgs& a, cudaStream_t s) {
  const int64_t blocks = a.block_start[a.nseg];
  if (blocks == 0) return cudaSuccess;
  const int64_t cap = (int64_t)sm_count() * 8;
  noise_grids_kernel<<<(unsigned)(blocks < cap ? blocks : cap), kNoiseBlock, 0, s>>>(a);
  return cudaGetLastError();
}

namespace {
// One weight matrix [rows][cols] (FP32) -> E4M3 with one scale: s = max|W| /
// 448 (the largest finite E4M3 value; 1 for an all-zero matrix), W8 = rn(W /
// s) saturating, rows padded with zero bytes to cols_out.  One block.
__global__ void __launch_bounds__(256) f8_weights_kernel(const float* __restrict__ w, int rows,
                                                         int cols, int cols_out,
                                                         uint8_t* __restrict__ w8, float* scale) {
  __shared__ float red[8];
  float mx = 0.f;
  for (int i = threadIdx.x; i < rows * cols; i += blockDim.x) mx = fmaxf(mx, fabsf(w[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  float m = 0.f;
  for (int k = 0; k < 8; ++k) m = fmaxf(m, red[k]);
  const float sc = m > 0.f ? m / 448.f : 1.f;
  if (threadIdx.x == 0) *scale = sc;
  for (int i = threadIdx.x; i < rows * cols_out; i += blockDim.x) {
    const int r = i / cols_out, c = i - r * cols_out;
    const float v = c < cols ? w[r * cols + c] / sc : 0.f;
    w8[i] = (uint8_t)(tc::pack_e4m3x2(v, 0.f) & 0xFFu);
  }
}
}  // namespace

namespace {
// The smallest power of two p with a / p <= 448 (1 for a = 0 or not finite).
__device__ __forceinline__ float pow2_scale(float a) {
  if (!(a > 0.f) || !(a < __int_as_float(0x7f800000))) return 1.f;
  int e = 0;
  const float f = frexpf(a / 448.f, &e);  // a / 448 = f 2^e, f in [0.5, 1)
  if (f == 0.5f) e -= 1;
  e = e < -126 ? -126 : (e > 127 ? 127 : e);
  return __int_as_float((127 + e) << 23);
}

struct F8Prep {
  const float* w[3];
  uint8_t* w8[3];
  int rows[3], cols[3];
};

// Block l: layer l's weight scale and E4M3 weights; block 0 also turns the
// recorded layer-input maxima (scale9[6..8], float bits) into the
// activation scales scale9[3..5] and clears them.
__global__ void __launch_bounds__(256) f8_train_prep_kernel(const F8Prep a, float* scale9) {
  __shared__ float red[8];
  const int l = blockIdx.x;
  const float* w = a.w[l];
  const int n = a.rows[l] * a.cols[l];
  float mx = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) mx = fmaxf(mx, fabsf(w[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  float m = 0.f;
  for (int k = 0; k < 8; ++k) m = fmaxf(m, red[k]);
  const float sw = pow2_scale(m), inv = 1.f / sw;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    a.w8[l][i] = (uint8_t)(tc::pack_e4m3x2(w[i] * inv, 0.f) & 0xFFu);
  if (threadIdx.x == 0) scale9[l] = sw;
  if (l == 0 && threadIdx.x < 3) {
    uint32_t* amax = reinterpret_cast<uint32_t*>(scale9 + 6);
    const float v = __uint_as_float(amax[threadIdx.x]);
    if (v > 0.f) scale9[3 + threadIdx.x] = pow2_scale(v);
    amax[threadIdx.x] = 0u;
  }
}
}  // namespace

cudaError_t launch_f8_train_prep(const float* const* w_master, uint8_t* const* w8, int k_in,
                                 int channels, float* scale9, cudaStream_t s) {
  F8Prep a;
  for (int l = 0; l < 3; ++l) {
    a.w[l] = w_master[l];
    a.w8[l] = w8[l];
  }
  a.rows[0] = kHidden; a.cols[0] = k_in;
  a.rows[1] = kHidden; a.cols[1] = kHidden;
  a.rows[2] = channels; a.cols[2] = kHidden;
  f8_train_prep_kernel<<<3, 256, 0, s>>>(a, scale9);
  return cudaGetLastError();
}

cudaError_t launch_f8_weights(const float* w, int rows, int cols, int cols_out, uint8_t* w8,
                              float* scale, cudaStream_t s) {
  f8_weights_kernel<<<1, 256, 0, s>>>(w, rows, cols, cols_out, w8, scale);
  return cudaGetLastError();
}

cudaError_t launch_adam_batched(TrainBatchDev* dev, int64_t blocks, cudaStream_t s) {
  if (blocks == 0) return cudaSuccess;
  const int64_t cap = (int64_t)sm_count() * 8;
  adam_batched_kernel<<<(unsigned)(blocks < cap ? blocks : cap), kAdamBlock, 0, s>>>(dev);
  return cudaGetLastError();
}

cudaError_t launch_noise_batched(const TrainBatchDev* dev, int64_t blocks, cudaStream_t s) {
  if (blocks == 0) return cudaSuccess;
  const int64_t cap = (int64_t)sm_count() * 8;
  noise_batched_kernel<<<(unsigned)(blocks < cap ? blocks : cap), kNoiseBlock, 0, s>>>(dev);
  return cudaGetLastError();
}

cudaError_t launch_advance_step(int64_t* step, cudaStream_t s, int64_t* tag, uint64_t seed) {
  advance_step_kernel<<<1, 1, 0, s>>>(step, tag, seed);
  return cudaGetLastError();
}

cudaError_t launch_quantize_pack(const float* values, int64_t cells, int c, int bits, float q,
                                 uint8_t* packed, float* snapped, cudaStream_t s) {
  if (cells == 0) return cudaSuccess;
  quantize_pack_kernel<<<blocks_for(cells, 256), 256, 0, s>>>(values, cells, c, bits, q, packed,
                                                               snapped);
  return cudaGetLastError();
}

cudaError_t launch_unpack(const uint8_t* packed, int64_t cells, int c, int bits, float q,
                          int32_t* idx, float* values, cudaStream_t s) {
  if (cells == 0) return cudaSuccess;
  unpack_kernel<<<blocks_for(cells, 256), 256, 0, s>>>(packed, cells, c, bits, q, idx, values);
  return cudaGetLastError();
}

// Index of the entry of one codebook (256 x c0 floats in shared memory)
// nearest to r: squared distance in FP32, the channels summed in order
// without fused multiply-add, ties to the lowest index.  Rows of 4k values
// are read as float4 (same arithmetic).
__device__ __forceinline__ int vq_nearest(const float* book, const float (&r)[kMaxGridCh], int c0) {
  float best = __int_as_float(0x7f800000);  // +inf
  int kb = 0;
  if ((c0 & 3) == 0) {
#pragma unroll 1
    for (int k = 0; k < 256; ++k) {
      const float4* e4 = reinterpret_cast<const float4*>(book + k * c0);
      float d = 0.f;
#pragma unroll
      for (int q4 = 0; q4 < kMaxGridCh / 4; ++q4)
        if (4 * q4 < c0) {
          const float4 e = e4[q4];
          const float ev[4] = {e.x, e.y, e.z, e.w};
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float df = __fsub_rn(r[4 * q4 + i], ev[i]);
            d = __fadd_rn(d, __fmul_rn(df, df));
          }
        }
      if (d < best) {
        best = d;
        kb = k;
      }
    }
  } else {
#pragma unroll 1
    for (int k = 0; k < 256; ++k) {
      const float* e = book + k * c0;
      float d = 0.f;
#pragma unroll
      for (int ch = 0; ch < kMaxGridCh; ++ch)
        if (ch < c0) {
          const float df = __fsub_rn(r[ch], e[ch]);
          d = __fadd_rn(d, __fmul_rn(df, df));
        }
      if (d < best) {
        best = d;
        kb = k;
      }
    }
  }
  return kb;
}

// Greedy residual vector quantisation of one row per thread against the
// codebooks staged in shared memory: FP32 squared distances with the channels
// summed in order and no fused multiply-add, ties to the lowest index.
__global__ void __launch_bounds__(256) vq_assign_kernel(const float* __restrict__ values,
                                                        int64_t cells, int c0,
                                                        const float* __restrict__ books, int nb,
                                                        uint8_t* __restrict__ idx) {
  extern __shared__ float cb[];  // [nb][256][c0]
  for (int i = threadIdx.x; i < nb * 256 * c0; i += blockDim.x) cb[i] = books[i];
  __syncthreads();
  for (int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; cell < cells;
       cell += (int64_t)gridDim.x * blockDim.x) {
    float r[kMaxGridCh];
#pragma unroll
    for (int ch = 0; ch < kMaxGridCh; ++ch) r[ch] = ch < c0 ? values[cell * c0 + ch] : 0.f;
    for (int b = 0; b < nb; ++b) {
      const int kb = vq_nearest(cb + b * 256 * c0, r, c0);
      idx[cell * nb + b] = (uint8_t)kb;
      const float* e = cb + (b * 256 + kb) * c0;
#pragma unroll
      for (int ch = 0; ch < kMaxGridCh; ++ch)
        if (ch < c0) r[ch] = __fsub_rn(r[ch], e[ch]);
    }
  }
}

// One training step's vector quantisation of a G0 level (VQ-VAE terms): per
// latent row z, greedy residual assignment (as vq_assign_kernel); q, the sum
// of the selected entries, goes to the scratch grid the fused step reads;
// the codebook loss (1/N) sum ||sg(r_b) - e_b||^2 gives dE_b[k] += scale
// (e_b[k] - r_b) and the commitment loss beta (1/N) sum ||z - sg(q)||^2
// gives dz += scale beta (z - q), scale = 2 / N.  dE is summed per CTA in
// shared memory and added to global memory once.
__global__ void __launch_bounds__(256) vq_step_kernel(const float* __restrict__ z, int64_t cells,
                                                      int c0, const float* __restrict__ books,
                                                      int nb, uint8_t* __restrict__ idx,
                                                      float* __restrict__ q_out,
                                                      float* __restrict__ dz,
                                                      float* __restrict__ dE, float scale,
                                                      float beta) {
  extern __shared__ float sm[];
  float* cb = sm;                    // [nb][256][c0]
  float* acc = sm + nb * 256 * c0;   // [nb][256][c0] codebook-gradient partial sums
  for (int i = threadIdx.x; i < nb * 256 * c0; i += blockDim.x) {
    cb[i] = books[i];
    acc[i] = 0.f;
  }
  __syncthreads();
  for (int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; cell < cells;
       cell += (int64_t)gridDim.x * blockDim.x) {
    float zr[kMaxGridCh], r[kMaxGridCh], q[kMaxGridCh];
#pragma unroll
    for (int ch = 0; ch < kMaxGridCh; ++ch) {
      zr[ch] = r[ch] = ch < c0 ? z[cell * c0 + ch] : 0.f;
      q[ch] = 0.f;
    }
    for (int b = 0; b < nb; ++b) {
      const int kb = vq_nearest(cb + b * 256 * c0, r, c0);
      idx[cell * nb + b] = (uint8_t)kb;
      const float* e = cb + (b * 256 + kb) * c0;
      float* a = acc + (b * 256 + kb) * c0;
#pragma unroll
      for (int ch = 0; ch < kMaxGridCh; ++ch)
        if (ch < c0) {
          if (dE) atomicAdd(a + ch, scale * (e[ch] - r[ch]));
          r[ch] = __fsub_rn(r[ch], e[ch]);
          q[ch] += e[ch];
        }
    }
    // the decoder trains on q (the value the exported indices decode to)
#pragma unroll
    for (int ch = 0; ch < kMaxGridCh; ++ch)
      if (ch < c0) {
        q_out[cell * c0 + ch] = q[ch];
        if (dz) dz[cell * c0 + ch] += scale * beta * (zr[ch] - q[ch]);
      }
  }
  __syncthreads();
  if (dE)
    for (int i = threadIdx.x; i < nb * 256 * c0; i += blockDim.x)
      if (acc[i] != 0.f) atomicAdd(dE + i, acc[i]);
}

cudaError_t launch_vq_step(const float* z, int64_t cells, int c0, const float* books, int nb,
                           uint8_t* idx, float* q_out, float* dz, float* dE, float scale,
                           float beta, cudaStream_t s) {
  if (cells == 0) return cudaSuccess;
  const size_t smem = 2 * (size_t)nb * 256 * c0 * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(vq_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, vq_step_kernel, 256, smem);
  if (e != cudaSuccess) return e;
  const int64_t blocks = (cells + 255) / 256;
  const int64_t cap = (int64_t)sm_count() * (per_sm > 0 ? per_sm : 1);
  vq_step_kernel<<<(int)(blocks < cap ? blocks : cap), 256, smem, s>>>(z, cells, c0, books, nb, idx,
                                                                     q_out, dz, dE, scale, beta);
  return cudaGetLastError();
}

cudaError_t launch_vq_assign(const float* values, int64_t cells, int c0, const float* books, int nb,
                             uint8_t* idx, cudaStream_t s) {
  if (cells == 0) return cudaSuccess;
  const size_t smem = (size_t)nb * 256 * c0 * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(vq_assign_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, vq_assign_kernel, 256, smem);
  if (e != cudaSuccess) return e;
  const int64_t blocks = (cells + 255) / 256;
  const int64_t cap = (int64_t)sm_count() * (per_sm > 0 ? per_sm : 1);
  vq_assign_kernel<<<(int)(blocks < cap ? blocks : cap), 256, smem, s>>>(values, cells, c0, books,
                                                                       nb, idx);
  return cudaGetLastError();
}

cudaError_t launch_sample_batch(uint64_t seed, int64_t step, int64_t batch, int w, int h, int mips,
                                int crops, int32_t* xym, cudaStream_t s) {
  if (batch == 0) return cudaSuccess;
  sample_batch_kernel<<<blocks_for(batch, 256), 256, 0, s>>>(rng_key(seed, sampler_stream(step)),
                                                             batch, w, h, mips, crops, xym);
  return cudaGetLastError();
}

cudaError_t launch_sample_features(const ntc_material& m, const float* uvl, int64_t n, float* rows,
                                   int noise, uint64_t seed, int64_t step, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  sample_features_kernel<<<blocks_for(n, 128), 128, 0, s>>>(m, uvl, n, rows, noise,
                                                            rng_key(seed, noise_stream(step)));
  return cudaGetLastError();
}

}  // namespace ntc
