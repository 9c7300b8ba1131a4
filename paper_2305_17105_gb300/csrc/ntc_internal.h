// Internal launch interface between the C-ABI layer (ntc_api.cu) and the
// kernel translation units.  Every launcher returns a cudaError_t from the
// launch; arguments are validated by the caller.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ntc.h"

namespace ntc {

// What the fused forward+backward kernel differentiates.
struct BwdArgs {
  const float* uvl;        // queries (nullable in training mode: sampler instead)
  const float* dout;       // [n][C] upstream gradient (backward mode) or nullptr
  const uint8_t* target;   // training mode: u8 mip chain
  int64_t tgt_off[NTC_MAX_MIPS];
  int64_t n;
  ntc_grads g;             // gradient destinations (accumulated)
  float grad_scale;        // multiplies every accumulated gradient
  float* loss;             // training mode: += mean squared error
  float loss_scale;        // 1 / (n * C)
  int noise;               // simulated-quantisation noise on
  uint64_t noise_seed;
  int64_t noise_step;      // used when step_dev == nullptr
  uint64_t sample_seed;
  const int64_t* step_dev; // training mode: device step counter (noise + sampler)
  int train;               // 1: loss mode (dout = 2 (y - t)), 0: dout given
  int grids;               // 0: skip grid gradients (frozen grids)
  int crops;               // training sampler: 256 x 256 crops of one mip (Sec. 5.1)
  int pipelines;           // tensor-core step: warpgroup pipelines per CTA (0: the most that fit)
  // Noise check folded into the tensor-core step (single material, bilinear
  // G0, grids of 4k <= 16 channels): with noisy_tag set, a CTA that finds it
  // current ({noise_seed, step}) gathers from the trainer's noisy copy
  // (noisy0/1, level pointers) without noise; otherwise from the material's
  // grids with the noise added per tap (the same values).
  const int64_t* noisy_tag;
  const float* noisy0[NTC_MAX_LEVELS];
  const float* noisy1[NTC_MAX_LEVELS];
};

cudaError_t launch_decode_simt(const ntc_material& m, const float* uvl, int64_t n, void* out,
                               int out_dtype, int filter, int noise, uint64_t noise_seed,
                               int64_t noise_step, cudaStream_t s);
cudaError_t launch_backward_simt(const ntc_material& m, const BwdArgs& a, cudaStream_t s);

// jkey: jitter_key(seed, frame) of the stochastic filter (unused otherwise).
cudaError_t launch_decode_tc(const ntc_material& m, const float* uvl, int64_t n, void* out,
                             int out_dtype, int filter, uint64_t jkey, cudaStream_t s, int nwg);
// FP16 fused training step: ReLU or hardGELU, bilinear or learned G0, while
// the operand tiles of two pipelines fit one CTA (k_int <= 96).
bool train_tc_supported(const ntc_material& m);
cudaError_t launch_train_tc(const ntc_material& m, const BwdArgs& a, cudaStream_t s);
// The FP8-E4M3 form of the fused step (R24: E4M3 forward on kind::f8f6f4,
// FP16 backward on the same values, straight-through); m.w[] hold E4M3
// bytes and m.scale 9 floats (s_w[3], s_a[3], layer-input maxima[3]).
cudaError_t launch_train_tc_f8(const ntc_material& m, const BwdArgs& a, cudaStream_t s);
// The FP8 step's pre-pass: s_w[l] = the smallest power of two with
// max|W_l| / s_w <= 448 from the FP32 masters, W8_l = e4m3(W_l / s_w[l])
// into the material's weight bytes, and s_a[l] from the layer-input maxima
// the previous step recorded (kept where none was recorded), which it clears.
cudaError_t launch_f8_train_prep(const float* const* w_master, uint8_t* const* w8, int k_in,
                                 int channels, float* scale9, cudaStream_t s);

// Adam over the segments of the trainer's parameter array.
// grids (2 per level), W1..W3 and biases (6), the third hidden layer (2), codebooks (1)
constexpr int kMaxSegs = 2 * NTC_MAX_LEVELS + 9;
struct AdamSeg {
  int64_t off, len;   // float offset into params and element count
  float lo, hi;       // clamp range (grids)
  int group;          // 0 grids, 1 MLP
  int clamp;
  __half* half_copy;  // refresh target (F16 weights) or nullptr
  // grid segments: the next step's noisy copy (AdamArgs::fold); c = 0: none
  int noise_c, noise_level, noise_grid;
  float noise_q;
};
struct AdamArgs {
  AdamSeg seg[kMaxSegs];
  int64_t block_start[kMaxSegs + 1];  // prefix sums of blocks per segment
  int nseg;
  float* p;
  float* m;
  float* v;
  float* g;
  const int64_t* step;
  int64_t total;
  float lr[2];
  float beta1, beta2, eps;
  int freeze_grids;
  // With fold, the update also writes the next step's noisy grids
  // (params + the noise of (noise_seed, step + 1)) into `noisy`, and the
  // step counter's advance tags them (noisy_tag = {seed, step + 1}), so that
  // the next step's dense noise pass finds them current and skips.
  int fold;
  float* noisy;
  uint64_t noise_seed;
  int64_t* noisy_tag;
};
constexpr int kAdamBlock = 256;
constexpr int kAdamPerThread = 4;  // one float4 per thread
cudaError_t launch_adam(const AdamArgs& a, int64_t blocks, cudaStream_t s);

// Dense quantisation-noise pass of one step: dst = src + noise for every
// value of every grid segment (offsets into params / the noisy scratch).
struct NoiseSeg {
  int64_t off, pairs;  // first value; channel pairs (cells * ceil(c / 2))
  int c, level, grid;
  float q;
};
struct NoiseArgs {
  const float* src;
  float* dst;
  const int64_t* tag;  // nullable: skip when {seed, *step} (the copy is current)
  NoiseSeg seg[2 * NTC_MAX_LEVELS];
  int64_t block_start[2 * NTC_MAX_LEVELS + 1];
  int nseg;
  uint64_t seed;
  const int64_t* step;
};
constexpr int kNoiseBlock = 256;
cudaError_t launch_noise_grids(const NoiseArgs& a, cudaStream_t s);
// FP8-E4M3 form: one weight matrix quantised with its scale max|W| / 448, and
// the power-of-two activation scales from the per-layer input maxima of an
// FP32 decode of calibration queries (amax: 3 words of scratch, may alias sa).
cudaError_t launch_f8_weights(const float* w, int rows, int cols, int cols_out, uint8_t* w8,
                              float* scale, cudaStream_t s);
cudaError_t launch_f8_calibrate(const ntc_material& m, const float* uvl, int64_t n,
                                uint32_t* amax, float* sa, cudaStream_t s);

// *step += 1; with tag (nullable): tag = {seed, new step}.
cudaError_t launch_advance_step(int64_t* step, cudaStream_t s, int64_t* tag = nullptr,
                                uint64_t seed = 0);

cudaError_t launch_quantize_pack(const float* values, int64_t cells, int c, int bits, float q,
                                 uint8_t* packed, float* snapped, cudaStream_t s);
cudaError_t launch_unpack(const uint8_t* packed, int64_t cells, int c, int bits, float q,
                          int32_t* idx, float* values, cudaStream_t s);
cudaError_t launch_vq_step(const float* z, int64_t cells, int c0, const float* books, int nb,
                           uint8_t* idx, float* q_out, float* dz, float* dE, float scale,
                           float beta, cudaStream_t s);
cudaError_t launch_vq_assign(const float* values, int64_t cells, int c0, const float* books, int nb,
                             uint8_t* idx, cudaStream_t s);
cudaError_t launch_sample_batch(uint64_t seed, int64_t step, int64_t batch, int w, int h, int mips,
                                int crops, int32_t* xym, cudaStream_t s);
cudaError_t launch_sample_features(const ntc_material& m, const float* uvl, int64_t n, float* rows,
                                   int noise, uint64_t seed, int64_t step, cudaStream_t s);

// Device-side descriptor of a batch of materials (ntc_batch_prepare).
constexpr int kMaxBatch = 1024;
struct BatchHeader {
  int32_t n_materials;
  int32_t pad;
  int64_t total_tiles;
  int64_t tile_start[kMaxBatch + 1];  // prefix sums of tiles, ordered by material
  int64_t q_off[kMaxBatch + 1];       // query row offsets
  int64_t o_off[kMaxBatch + 1];       // output element offsets
  ntc_material mats[kMaxBatch];
};
// Device-side descriptor of a batch of optimisation steps
// (ntc_train_batch_prepare): per material the material as the fused step
// reads it, the step's arguments, its Adam segments and its noise segments;
// the 128-texel tiles of all materials in one list ordered by material.
constexpr int kMaxTrainBatch = 256;
struct TrainBatchDev {
  int32_t n;                              // materials
  uint32_t adam_done;                     // Adam blocks finished in this step (reset by the last)
  int64_t total_tiles, adam_blocks, noise_blocks;
  int64_t tile_start[kMaxTrainBatch + 1]; // prefix sums of tiles
  int64_t adam_start[kMaxTrainBatch + 1]; // prefix sums of Adam blocks (0 for a skipped material)
  int64_t noise_start[kMaxTrainBatch + 1];
  ntc_material mats[kMaxTrainBatch];
  BwdArgs args[kMaxTrainBatch];
  AdamArgs adam[kMaxTrainBatch];
  NoiseArgs noise[kMaxTrainBatch];
};
// The fused step over a batch: one persistent launch; every material shares
// act, interp0 and hidden_layers (the kernel class) and the layout of the
// largest k_int / dX width.
cudaError_t launch_train_tc_batched(const TrainBatchDev* dev, const ntc_material& first,
                                    int64_t total_tiles, int k_lay, int dx_lay, cudaStream_t s);
// Pipelines per CTA of the batched step for that class and layout (0: none fits).
int train_pipelines_layout(const ntc_material& first, int k_lay, int dx_lay);
// Internal widths of a material's training rows: k_int and the dX columns.
void train_widths(const ntc_material& m, int* k_int, int* dx_n);
// Adam over every material of the batch in one launch; its last block
// advances the step counter of every material that took part.
cudaError_t launch_adam_batched(TrainBatchDev* dev, int64_t blocks, cudaStream_t s);
cudaError_t launch_noise_batched(const TrainBatchDev* dev, int64_t blocks, cudaStream_t s);

// Input-layout class of a material for the warp-specialised kernels: 0
// generic, 1..9 fast 4-bit layout (1 + 3 k0 + k1 by grid class).
int fast_class(const ntc_material& m);
// Shared-memory plan bytes of one material | its internal K << 24, and the
// batched kernel's total for the batch's maxima of both.
uint32_t ws_plan_bytes(const ntc_material& m, bool fast);
uint32_t ws_batched_smem(uint32_t plan_bytes);
// Many materials in one warp-specialised launch; cls: 0 generic, 1..9 one
// fast class for every material, -1 fast with per-material classes.
cudaError_t launch_decode_ws_batched(const BatchHeader* dev, int64_t total_tiles,
                                     uint32_t plan_bytes, int cls, const float* uvl, void* out,
                                     int out_dtype, int filter, cudaStream_t s);
bool fast_layout_ok(const ntc_material& m);
cudaError_t launch_selftest_wait(uint32_t limit, cudaStream_t s);
// Warp-specialised tensor-core decode (FP16), fast 4-bit layout or generic.
cudaError_t launch_decode_ws(const ntc_material& m, const float* uvl, int64_t n, void* out,
                             int out_dtype, int filter, uint64_t jkey, cudaStream_t s, bool fast);
// The same kernel in FP8-E4M3 (kind::f8f6f4): fast 4-bit layout when
// fast_layout_ok, generic layout otherwise.
cudaError_t launch_decode_ws_f8(const ntc_material& m, const float* uvl, int64_t n, void* out,
                                int out_dtype, int filter, uint64_t jkey, cudaStream_t s);


int sm_count();
// FP32 FMA throughput of the current device (TFLOP/s, best of 5 timed
// launches of an FMA-chain kernel); synchronises `s`.
cudaError_t probe_fma_tflops(float* tflops, cudaStream_t s);

// Record a thread-local error message (ntc_last_error) and return `code`.
int report_error(int code, const char* fmt, ...);

// Device status word of the current device (bounded waits write
// NTC_ERR_TIMEOUT there); read and cleared by ntc_device_status.
int* status_word();
int read_status_word(int reset);  // synchronises the device; -1 on CUDA error

}  // namespace ntc

// ntc_train_step's argument checks alone (no stream operation; the same
// status and message as ntc_train_step would give).  Library-internal.
extern "C" __attribute__((visibility("hidden"))) int ntc_train_step_check(
    const ntc_material* m, const ntc_trainer* tr, const ntc_target* t, int64_t batch,
    uint64_t seed, const float* uvl_or_null, float* loss_out, int32_t flags);
