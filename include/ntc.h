/*
 * ntc.h -- C ABI of the GB300 neural-texture-compression library (libntc.so).
 *
 * The library implements the data-parallel hot path of "Random-Access Neural
 * Compression of Material Textures" (Vaidyanathan et al., 2023): the
 * per-texel random-access decode (Sec. 4.3-4.4, Sec. 5.2) and the per-material
 * fused forward+backward optimisation that compresses a material (Sec. 4.2,
 * 4.5, 5.1), as hand-written CUDA for sm_103a.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every array argument is a DEVICE pointer owned by the caller unless the
 *    parameter says "host".  The library never allocates or frees device
 *    memory and never synchronises the device (ntc_device_status and the
 *    autotuner excepted); all work is enqueued on the caller's `stream` (a
 *    cudaStream_t passed as void*; NULL = legacy default stream) in launch
 *    order.  ntc_decode_host also uses two helper streams and a few events
 *    that it creates once per device, joined back into `stream`.
 *  - Structs (ntc_material, ntc_grads, ntc_trainer, ntc_target) are passed by
 *    HOST pointer; their fields point to device memory.  They are read during
 *    the call only; the call does not keep them.
 *  - Every call returns an ntc_status.  On failure nothing was enqueued
 *    (argument errors) or the CUDA launch error is reported (NTC_ERR_CUDA);
 *    ntc_last_error() returns a thread-local human-readable message.  No C++
 *    exception crosses this boundary.
 *  - Device arrays must be 16-byte aligned (NTC_ERR_ALIGN otherwise).
 *  - Calls on one stream are ordered; calls that write the same memory from
 *    different streams race.
 */
#ifndef NTC_H
#define NTC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NTC_MAX_LEVELS 8    /* feature levels F^j (Sec. 4.1) */
#define NTC_MAX_MIPS 16     /* mip levels: textures up to 32768^2 */
#define NTC_MAX_CHANNELS 16 /* texture-set channels c (Sec. 4) */
#define NTC_MAX_FEATURES 32 /* c0 + c1 latent features per query */
#define NTC_MAX_K 128       /* padded MLP input width */
#define NTC_HIDDEN 64       /* hidden width of the decoder MLP (Sec. 4.4) */

typedef enum {
  NTC_OK = 0,
  NTC_ERR_ARG = 1,         /* null pointer, negative size, bad enum value */
  NTC_ERR_SHAPE = 2,       /* sizes violate the pyramid / MLP shape rules */
  NTC_ERR_ALIGN = 3,       /* a device pointer is not 16-byte aligned */
  NTC_ERR_UNSUPPORTED = 4, /* a valid combination the library does not implement */
  NTC_ERR_CUDA = 5,        /* a CUDA launch or API call failed */
  NTC_ERR_TIMEOUT = 6      /* a bounded device-side wait gave up (status word) */
} ntc_status;

/* Latent grid storage. */
enum {
  NTC_GRID_PACKED = 0, /* B-bit quantisation indices, one power-of-two-sized cell
                          per grid position (see ntc_cell_bytes) */
  NTC_GRID_F32 = 1     /* float32 values [g_h][g_w][c] (training form) */
};
/* Arithmetic of the decoder MLP. */
enum {
  NTC_PREC_F32 = 0, /* FP32 CUDA-core form: weights float32 */
  NTC_PREC_F16 = 1, /* tcgen05 tensor-core form: weights float16, FP32 accumulation */
  NTC_PREC_F8 = 2   /* tcgen05 tensor-core form: weights FP8-E4M3 with per-layer scales */
};
enum { NTC_ACT_RELU = 0, NTC_ACT_HARDGELU = 1 };   /* hidden activation (Sec. 4.4) */
enum { NTC_OUT_SIGMOID = 0, NTC_OUT_IDENTITY = 1 }; /* output activation */
/* Sec. 5.3: nearest texel of (u, v) at mip floor(lod); trilinear (8 texels
 * decoded and blended); stochastic: one decode at the nearest texel of the
 * jittered position u w_m - 1/2 + xi_x (same for v) on mip floor(lod + xi_l),
 * xi uniform in [0, 1) from a counter hash of (noise_seed, noise_step, query
 * index), which equals trilinear filtering in expectation. */
enum { NTC_FILTER_NEAREST = 0, NTC_FILTER_TRILINEAR = 1, NTC_FILTER_STOCHASTIC = 2 };
/* Output element type.  U8: 8-bit UNORM, each output y stored as
 * round-half-to-even(clamp(y, 0, 1) * 255) computed in float32 (NaN -> 0),
 * the 8-bit encoding of the evaluation textures (appendix "Evaluation
 * Texture Set Details"). */
enum { NTC_DTYPE_F32 = 0, NTC_DTYPE_F16 = 1, NTC_DTYPE_U8 = 2 };
/* Resampling of G0 (Sec. 4.3.1): bilinear like G1, or learned interpolation:
 * the four neighbouring G0 feature vectors of the bilinear footprint (taps
 * (x0,y0), (x1,y0), (x0,y1), (x1,y1)) concatenated in the MLP input, which
 * then holds 4 c0 + c1 + 13 used values.  Learned interpolation runs on the
 * FP32 and FP16 decode forms and both training forms. */
enum { NTC_INTERP_BILINEAR = 0, NTC_INTERP_LEARNED = 1 };

/* Flags of ntc_decode / ntc_backward / ntc_train_step. */
#define NTC_FLAG_NOISE 0x1        /* add simulated-quantisation noise (Sec. 4.2); F32 grids */
#define NTC_FLAG_FREEZE_GRIDS 0x2 /* train_step: grids fixed (Sec. 4.2 final phase) */
#define NTC_FLAG_NO_NOISE 0x4     /* train_step: no noise while grids still train */
#define NTC_FLAG_SIMT 0x8         /* force the FP32 CUDA-core kernels (any precision
                                     is converted to FP32 on load) */
#define NTC_FLAG_GRAD_ONLY 0x10   /* train_step: accumulate the batch's gradient into
                                     tr->grad and stop (no Adam update, step counter
                                     unchanged); the next regular step applies the sum */
#define NTC_FLAG_CROPS 0x20       /* train_step: sample the batch as 256 x 256 texel
                                     crops of one mip (Sec. 5.1, ntc_sample_crops)
                                     instead of independent texels (ntc_sample_batch) */

/* One feature level F^j = (G^j_0, G^j_1) (Sec. 4.1, Table 1). */
typedef struct {
  int32_t g0_w, g0_h; /* G0 resolution */
  int32_t g1_w, g1_h; /* G1 resolution */
  const void* grid0;  /* PACKED: [g0_h][g0_w] cells of ntc_cell_bytes(c0,bits0) bytes;
                         F32: float [g0_h][g0_w][c0] */
  const void* grid1;  /* likewise with c1, bits1 */
} ntc_level;

/* A compressed material: feature pyramid + decoder (Sec. 4). */
typedef struct {
  int32_t width, height; /* mip-0 texture-set resolution w x h, powers of two */
  int32_t channels;      /* c, decoder outputs, 1..NTC_MAX_CHANNELS */
  int32_t mips;          /* M = log2(max(w, h)) + 1 */
  int32_t levels;        /* feature levels L, 1..NTC_MAX_LEVELS */
  int32_t c0, c1;        /* features per cell of G0 / G1; c0 + c1 <= NTC_MAX_FEATURES */
  int32_t bits0, bits1;  /* quantisation bits B_k in {1,2,4,8}: N_k = 2^B_k levels */
  float q0, q1;          /* bin width Q_k: level values (k - (N/2-1)) * Q (Sec. 4.2) */
  int32_t encoding;      /* NTC_GRID_PACKED | NTC_GRID_F32 */
  int32_t k_in;          /* MLP input width: >= c0 + c1 + 13 (4 c0 + c1 + 13 with
                            learned interpolation), multiple of 16
                            (of 32 for NTC_PREC_F8), <= NTC_MAX_K */
  int32_t hidden;        /* must be NTC_HIDDEN */
  int32_t act;           /* NTC_ACT_* */
  int32_t out_act;       /* NTC_OUT_* */
  int32_t precision;     /* NTC_PREC_* */
  int32_t interp0;       /* NTC_INTERP_*: resampling of G0 (Sec. 4.3.1) */
  ntc_level lv[NTC_MAX_LEVELS];
  const void* w[3];      /* layer weights [out][in]: W1 [hidden][k_in], W2 [hidden][hidden],
                            W3 [channels][hidden]; float / half / e4m3 by precision */
  const float* b[3];     /* biases, float32 [out] */
  const float* scale;    /* NTC_PREC_F8 only: 6 device floats, weight scales s_w[3]
                            then input-activation scales s_a[3]; layer l computes
                            (s_w[l]*s_a[l]) * (W8 . q8(x / s_a[l])) + b.  NULL otherwise */
  int32_t hidden_layers; /* hidden layers with activations (Sec. 4.4): 2 (0 reads as 2),
                            or 3 -- a third [hidden][hidden] layer w_h3, b_h3 between
                            W2 and the output layer W3.  Three hidden layers run on
                            the FP32 decode, the FP16 warp-specialised decode and the
                            FP16 training step */
  const void* w_h3;      /* [hidden][hidden], the precision's type (hidden_layers == 3) */
  const float* b_h3;     /* [hidden] float32 */
  int32_t vq_books;      /* 0: G0 scalar-quantised like G1.  1..4: vector-quantised G0
                            (the paper's comparison with vector quantisation): grid0 of
                            every level holds uint8 [g0_h][g0_w][vq_books] indices, index
                            b into codebook b of 256 entries of c0 values, and a cell's
                            features are the sum of its vq_books entries (bits0 is
                            unused).  Decode: FP32 and FP16 forms, no noise.
                            Training form (encoding NTC_GRID_F32, ntc_train_step
                            only): grid0 holds the continuous latents, quantised by
                            every step (see ntc_train_step) */
  const float* codebook0; /* [vq_books][256][c0] float32, device (vq_books > 0) */
} ntc_material;

/* Gradient outputs of ntc_backward, ACCUMULATED (+=) in float32, same
 * layouts as the F32 grids and the weights. */
typedef struct {
  float* grid0[NTC_MAX_LEVELS];
  float* grid1[NTC_MAX_LEVELS];
  float* w[3];
  float* b[3];
  float* w_h3;           /* third hidden layer (hidden_layers == 3), nullable */
  float* b_h3;
} ntc_grads;

/* Optimiser state of ntc_train_step (Sec. 5.1: Adam, two learning rates,
 * cosine annealing).  `params` is one float32 array holding every trainable
 * tensor; the material passed to ntc_train_step must point its F32 grids and
 * its biases into it, and w_master[l] gives the FP32 master of W_l inside it
 * (for NTC_PREC_F32 the material's w[l] must equal w_master[l]; for F16 the
 * step rewrites the material's half copies from the masters after each
 * update).  adam_m, adam_v and grad have params' length; grad is scratch that
 * every step leaves zeroed (initialise it to zero once).  `noisy` (nullable)
 * is scratch of params' length: with it a noisy step first writes the grids
 * plus this step's quantisation noise (Sec. 4.2) into it in one dense pass
 * and the fused step gathers from there (each grid value is hashed once per
 * step instead of once per tap that reads it); without it the fused step
 * adds the noise per tap.  Both give the same noisy values. */
typedef struct {
  float* params;
  float* adam_m;
  float* adam_v;
  float* grad;
  int64_t n_params;
  float* w_master[3];
  int64_t* step;        /* device int64: 0-based index of the next step; the step
                           reads it and increments it on the device */
  int64_t total_steps;  /* T of the cosine schedule lr_t = lr0 (1 + cos(pi t / T)) / 2 */
  float lr_grid;        /* 0.01 in the paper */
  float lr_mlp;         /* 0.005 in the paper */
  float beta1, beta2, eps;
  float* noisy;         /* optional scratch, params' length (see above) */
  float* w_master_h3;   /* FP32 master of the third hidden layer (hidden_layers == 3),
                           inside params like w_master[]; its bias is the material's
                           b_h3, also inside params */
  uint8_t* vq_idx;      /* vector-quantised G0 (material vq_books > 0): scratch of
                           sum over levels of g0_w g0_h vq_books bytes (the step's
                           indices); needs `noisy`.  NULL otherwise */
  float vq_beta;        /* commitment weight of the vector-quantised G0 */
  int64_t* noisy_tag;   /* nullable, device int64[2] (initialise to {-1, -1}): with `noisy`,
                           each step's Adam also writes the next step's noisy grids and
                           tags them {seed, step}; the next step's noise pass skips when
                           the tag matches its own seed and step.  When the previous
                           step on this trainer folded with the same seed (bilinear G0,
                           grids of 4k <= 16 channels, tensor-core step) the fused step
                           checks the tag itself and launches no noise pass; a stale
                           tag then makes it add the noise per tap (the same values).
                           Reset it to {-1, -1} after changing params outside the
                           library */
} ntc_trainer;

/* Reference texture set: the 8-bit mip chain, texel values q/255. */
typedef struct {
  const uint8_t* texels;           /* device */
  int64_t offset[NTC_MAX_MIPS];    /* byte offset of mip m: [h_m][w_m][channels] u8 */
} ntc_target;

/* Library version string (static storage). */
const char* ntc_version(void);

/* Message of the last failing call on this thread (static, thread-local). */
const char* ntc_last_error(void);

/* Synchronises the current device, then returns NTC_OK or the error that a
 * kernel recorded in the library's device status word since the last reset:
 * NTC_ERR_TIMEOUT when a bounded wait of a tensor-core kernel (TMEM
 * allocation, MMA completion) gave up -- that launch's outputs are then
 * incomplete.  reset != 0 clears the word.  The only call that synchronises. */
int ntc_device_status(int32_t reset);

/* Failure-detection self-test (no counterpart in the paper): enqueues a kernel
 * whose bounded wait cannot complete (an mbarrier nothing arrives at, with
 * the wait the tensor-core kernels use); after `limit` suspended tries of up
 * to ~10 us each it records NTC_ERR_TIMEOUT in the device status word --
 * as a kernel whose MMA completion never arrived would -- and returns, the
 * context intact.  limit in 1..2^20; read the result with ntc_device_status. */
int ntc_selftest_wait(int32_t limit, void* stream);

/* Bytes of one packed grid cell for c features of `bits` bits: c*bits bits
 * rounded up to a power-of-two number of bytes.  Channel ch occupies bits
 * [ch*bits, (ch+1)*bits) counting from bit 0 of byte 0.  0 on bad input. */
int32_t ntc_cell_bytes(int32_t c, int32_t bits);

/* Feature pyramid of a w x h texture set (Sec. 4.1, Table 1): G0 of level j
 * is (w >> (2j+2), h >> (2j+2)) (each at least 1), G1 half of G0; levels
 * continue while G0's longer side is at least 4.  Writes up to
 * NTC_MAX_LEVELS entries into the HOST arrays and returns the level count
 * (0 on bad input).  Mip m is served by level min(L-1, m < 4 ? 0 : (m-2)/2). */
int32_t ntc_pyramid(int32_t width, int32_t height, int32_t* g0_w, int32_t* g0_h,
                    int32_t* g1_w, int32_t* g1_h);

/* Random-access decode (Sec. 4.3-4.4; filtering Sec. 5.3).
 *  uvl  [n][3] float: u, v in [0,1) and the level of detail.  NEAREST: mip
 *       m = floor(lod) clamped to [0, M-1], texel x = floor(u w_m) clamped to
 *       [0, w_m - 1] (NaN -> 0).  TRILINEAR: lod is continuous; 2x2 texels
 *       around (u, v) on mips floor(lod) and floor(lod)+1 (clamped), texel
 *       taps wrap around, 8 decodes blended.
 *  out  [n][channels] float32, float16 or 8-bit UNORM (out_dtype), row-major.
 *  flags NTC_FLAG_NOISE (F32 grids only: decode the noisy training grids of
 *       (noise_seed, noise_step)), NTC_FLAG_SIMT.
 * Decodes each query from the level of its mip: bilinear G0 and G1 features,
 * 12 positional-encoding values, normalised LOD m/(M-1), zero padding, then
 * the 3-layer MLP.  n == 0 is a no-op. */
int ntc_decode(const ntc_material* m, const float* uvl, int64_t n, void* out,
               int32_t out_dtype, int32_t filter, int32_t flags, uint64_t noise_seed,
               int64_t noise_step, void* stream);

/* Decode with HOST query and output buffers (pinned host memory for the
 * copies to overlap): the queries stream through `workspace` (device,
 * caller-owned, 16-byte aligned) in chunks; the copy of chunk i+1 to the
 * device, the decode of chunk i (on `stream`) and the copy of chunk i-1 back
 * run concurrently on two helper streams that the library creates once per
 * device.  Outputs equal ntc_decode's.  The call returns once the work is
 * enqueued: `out_host` is complete when `stream` reaches the call's end
 * (fork and join through events, so the call can be captured in a CUDA
 * graph).  The chunk is workspace_bytes / (2 (12 + channels * element bytes))
 * queries rounded down to a multiple of 128 (NTC_ERR_ARG below 128);
 * ntc_decode_host_workspace_bytes gives the size for a chosen chunk.
 * Nearest and trilinear filtering (stochastic filtering hashes the query
 * index: NTC_ERR_UNSUPPORTED); flags as ntc_decode. */
int ntc_decode_host(const ntc_material* m, const float* uvl_host, int64_t n, void* out_host,
                    int32_t out_dtype, int32_t filter, int32_t flags, uint64_t noise_seed,
                    int64_t noise_step, void* workspace, size_t workspace_bytes, void* stream);

/* Workspace bytes of ntc_decode_host for chunks of `chunk` queries (0 for
 * invalid arguments). */
size_t ntc_decode_host_workspace_bytes(int32_t channels, int32_t out_dtype, int64_t chunk);

/* Launch shape of the tensor-core decode: warpgroup tile pipelines per CTA
 * (one CTA per SM, 128 TMEM columns per pipeline), 2, 3 or 4, or 5 for the
 * warp-specialised form (4 compute warpgroups whose MMA chains a fifth
 * warpgroup issues; FP16 and FP8); 0 restores the default (5).
 * Process-wide; takes effect for later ntc_decode calls. */
int ntc_set_decode_warpgroups(int32_t nwg);

/* Autotuner of the tensor-core decode: times every launch shape (1 warm-up
 * + 3 timed launches each, CUDA events on `stream`) on the caller's queries
 * (writing `out`) and records the fastest in the library's tuning cache
 * under this call's key -- the material's shape, channel counts, bit widths,
 * K, activations, precision and layout, the filter, the output type, the
 * device's SM count and the query count's power-of-two bucket -- and in
 * *best (host).  Later decodes with the same key use it unless
 * ntc_set_decode_warpgroups chose a shape.  ms_out (host, nullable, 4 floats)
 * receives the mean time per launch of the shapes 2, 3, 4, 5.  out_dtype and
 * filter as ntc_decode (NTC_ERR_ARG otherwise).  Synchronises the stream. */
int ntc_autotune_decode(const ntc_material* m, const float* uvl, int64_t n, void* out,
                        int32_t out_dtype, int32_t filter, int32_t* best, float* ms_out,
                        void* stream);

/* FP8-E4M3 form (the precision step below the paper's half-precision
 * tensor cores, Sec. 5.1, 7): one layer's weights w [rows][cols] (device
 * float32) quantised to E4M3 bytes w8_out [rows][cols_out] (columns cols ..
 * cols_out-1 zero; the FP8 form takes k_in in steps of 32) with the layer's
 * weight scale s_w = max|w| / 448 (448: the largest finite E4M3 value; 1
 * for an all-zero matrix) written to *scale_out (device float): the layer
 * computes (s_w s_a) (W8 . e4m3(x / s_a)) + b.  E4M3 rounding to nearest
 * even, saturating.  rows, cols_out <= NTC_MAX_K.  Only launches a kernel. */
int ntc_f8_quantize_weights(const float* w, int32_t rows, int32_t cols, int32_t cols_out,
                            uint8_t* w8_out, float* scale_out, void* stream);

/* Activation scales of the FP8-E4M3 form from calibration queries: decodes
 * the n queries uvl (nearest texels, FP32 arithmetic) with material m (FP32
 * or FP16 weights, two hidden layers) and writes to act_scale_out (device,
 * 3 floats) for each layer l the smallest power of two s_a[l] with
 * max|x_l| / s_a[l] <= 448 over the queries, x_l the layer's input (the
 * feature row, act(Z1), act(Z2)); 1 where the input is all zero.  Powers of
 * two keep the FP8 training form's FP16 operand copies exact.  With
 * ntc_f8_quantize_weights this fills the 6 scales of an NTC_PREC_F8
 * material (s_w[0..2], then s_a[0..2]).  Only launches kernels. */
int ntc_f8_activation_scales(const ntc_material* m, const float* uvl, int64_t n,
                             float* act_scale_out, void* stream);

/* Measurement helper (no counterpart in the paper): the FP32 FMA throughput
 * of the current device in TFLOP/s (*tflops_out, host), the best of five
 * timed launches of a kernel in which every thread advances 16 independent
 * fused multiply-add chains -- the ALU roof of the FP32 CUDA-core forms.
 * Synchronises `stream`. */
int ntc_probe_fma_tflops(float* tflops_out, void* stream);

/* Autotuner of the tensor-core training step: times the fused
 * forward+backward with 1, 2 and 3 warpgroup pipelines per CTA (those whose
 * tiles fit; 1 warm-up + 3 timed gradient-only steps each, CUDA events on
 * `stream`) on the arguments of ntc_train_step (no NTC_FLAG_SIMT or
 * GRAD_ONLY), records the fastest in the tuning cache (key: the material's
 * shape and precision, crops or not, the SM count and the batch's
 * power-of-two bucket) and in *best (host); ntc_train_step and
 * ntc_train_step_noalloc with that key use it.  ms_out (host, nullable, 3
 * floats): mean time per step for 1, 2, 3 pipelines (0 where they do not
 * fit).  Leaves params, Adam state, the step counter and (FP8 form) the
 * scales as they were and tr->grad zeroed; *loss_out is scratch.
 * Synchronises the stream. */
int ntc_autotune_train(const ntc_material* m, const ntc_trainer* tr, const ntc_target* t,
                       int64_t batch, uint64_t seed, int32_t flags, float* loss_out,
                       int32_t* best, float* ms_out, void* stream);

/* The tuning cache as text, one "<key> <value>" line per entry, for a caller
 * to keep between processes: ntc_tuning_export writes it NUL-terminated
 * into buf (host; NULL: only the size) and its size including the NUL into
 * *len_out (host, nullable); NTC_ERR_ARG if cap is too small.
 * ntc_tuning_import adds the entries of such text (values 1..5) to the
 * cache, replacing equal keys; ntc_tuning_clear empties it.  Host only. */
int ntc_tuning_export(char* buf, size_t cap, size_t* len_out);
int ntc_tuning_import(const char* text);
int ntc_tuning_clear(void);

/* Gradient of sum_i sum_c dout[i][c] * y[i][c] for nearest decodes y of the
 * queries uvl (Sec. 4.5, reverse mode of ntc_decode), ACCUMULATED into g.
 * Requires NTC_GRID_F32 grids.  With NTC_FLAG_NOISE the forward uses the
 * noisy grids of (noise_seed, noise_step), whose noise passes gradients
 * unchanged.  Activations are recomputed, never stored.  g fields may be
 * NULL to skip that tensor (grid entries: per level).
 * NTC_PREC_F16 materials run the tensor-core adjoint (the fused kernel of
 * ntc_train_step fed dout instead of the loss: FP16 operands with the
 * forward's head + tail inputs, FP32 accumulation; any k_in, two or three
 * hidden layers, bilinear or learned G0).  dout may have any magnitude: each
 * CTA scales the rows of its tiles by a power of two that brings their
 * largest |dout| into [1, 2) before the FP16 products and divides the
 * gradients by it in FP32.  FP32 and FP8 materials, and NTC_FLAG_SIMT, run
 * the FP32 CUDA-core adjoint (k_in <= 64, two hidden layers). */
int ntc_backward(const ntc_material* m, const float* uvl, int64_t n, const float* dout,
                 const ntc_grads* g, int32_t flags, uint64_t noise_seed, int64_t noise_step,
                 void* stream);

/* One optimisation step of a material (Sec. 4.2, 4.5, 5.1), fully on the
 * device: draw `batch` training texels (or use uvl_or_null [batch][3] texel
 * queries), decode them with simulated-quantisation noise, L2 loss against the
 * 8-bit reference t (mean over batch*channels, written to *loss_out, a device
 * float), backward into tr->grad, then Adam with cosine-annealed learning
 * rates lr_grid / lr_mlp, clamping of every grid to its quantisation range
 * [-(N-1)/2 Q, N/2 Q], refresh of half-precision weight copies, and
 * *tr->step += 1.  Sampling and noise are counter-based from (seed, *step),
 * so the call is CUDA-graph capturable and replays identically.
 * flags: NTC_FLAG_FREEZE_GRIDS (no noise, grids neither differentiated nor
 * updated), NTC_FLAG_NO_NOISE, NTC_FLAG_SIMT, NTC_FLAG_GRAD_ONLY,
 * NTC_FLAG_CROPS (crop sampler; ignored when uvl_or_null gives the texels).
 * Vector-quantised G0 (vq_books > 0, training form): each step assigns every
 * G0 latent row z to codebook entries by greedy residual search (as
 * ntc_vq_assign), trains the decoder on the quantised rows q (sum of the
 * entries; G1 keeps its noise), passes q's gradient straight through to z,
 * and adds the codebook loss (1/N) sum ||sg(r_b) - e_b||^2 and the
 * commitment loss vq_beta (1/N) sum ||z - sg(q)||^2 (r_b: what books
 * 0..b-1 leave of z; N: every G0 latent value) to the gradients of the
 * codebooks (inside params, Adam with lr_grid, unclamped) and of z
 * (unclamped); loss_out stays the L2 loss.  FP16
 * weights train on the tensor cores (tcgen05; ReLU or hardGELU, sigmoid or
 * identity output, bilinear or learned G0); FP32 weights or NTC_FLAG_SIMT on
 * the FP32 CUDA cores (k_in <= 64); FP8 weights: NTC_ERR_UNSUPPORTED. */
int ntc_train_step(const ntc_material* m, const ntc_trainer* tr, const ntc_target* t,
                   int64_t batch, uint64_t seed, const float* uvl_or_null, float* loss_out,
                   int32_t flags, void* stream);

/* ---- many materials in one launch -------------------------------------- */

/* A prepared batch of materials (filled by ntc_batch_prepare, host memory). */
typedef struct {
  const void* workspace;   /* device descriptor block, ntc_batch_workspace_bytes() bytes */
  int32_t n_materials;
  int32_t filter;          /* NTC_FILTER_* the batch was prepared for */
  int64_t total_queries;   /* rows of the concatenated uvl array */
  int64_t total_outputs;   /* elements of the concatenated output: sum of n_i * channels_i */
  int64_t total_tiles;
  int32_t wg_smem;         /* internal: shared-memory bytes of one material's plan */
  int32_t fast;            /* internal: input-layout class of the batch */
} ntc_batch;

#define NTC_MAX_BATCH 1024

/* Bytes of the device workspace a batch descriptor needs (about 0.4 MB). */
size_t ntc_batch_workspace_bytes(void);

/* Prepare a batch decode of n_materials materials (HOST array `mats`, all
 * NTC_PREC_F16) with n_queries[i] (HOST) queries
 * each: validates every material, lays the materials' queries out back to
 * back (material i's rows start at sum_{j<i} n_queries[j] of the uvl array
 * and its outputs at sum_{j<i} n_queries[j] * channels_j of the output
 * array), splits them into tiles ordered by material and copies the
 * descriptor into `workspace` (device, caller-owned) on `stream` with a
 * host-to-device copy from pageable memory: call it outside graph capture.
 * The workspace must stay untouched while batch decodes that use it run.
 * A material takes at most 2^31 - 1 queries and a batch at most 2^31 - 1
 * tiles (128 queries each, 16 with trilinear filtering): NTC_ERR_SHAPE
 * beyond. */
int ntc_batch_prepare(const ntc_material* mats, const int64_t* n_queries, int32_t n_materials,
                      int32_t filter, void* workspace, size_t workspace_bytes, ntc_batch* batch_out,
                      void* stream);

/* Decode every material of a prepared batch in one persistent launch (the
 * multi-material case of Sec. 5.2 / App. A, done by sorting work by material
 * instead of per-SIMD-group loops): uvl [total_queries][3], out (f32, f16 or u8)
 * [total_outputs].  Only launches a kernel: capturable in a CUDA graph. */
int ntc_decode_batched(const ntc_batch* batch, const float* uvl, void* out, int32_t out_dtype,
                       void* stream);

/* A batch of optimisation steps: many materials compressed side by side, one
 * step of each per call (the paper compresses every material of a scene with
 * the same fused trainer, Sec. 5.1, and runs many materials in one launch for
 * decoding, Sec. 5.2 / App. A; here training does the same). */
typedef struct {
  void* workspace;         /* device descriptor written by ntc_train_batch_prepare */
  float* loss_out;         /* device [n_materials]: each step's L2 loss per material */
  int32_t n_materials;
  int32_t flags;           /* the NTC_FLAG_* the batch was prepared with */
  int64_t total_tiles;     /* 128-texel tiles of all materials */
  int64_t adam_blocks;     /* internal: blocks of the batched Adam pass */
  int64_t noise_blocks;    /* internal: blocks of the batched noise pass */
  int32_t act, interp0, hidden_layers;  /* the kernel class every material shares */
  int32_t k_layout, dx_layout;          /* internal: shared layout of the batch */
} ntc_train_batch;

#define NTC_MAX_TRAIN_BATCH 256

/* Bytes of the device workspace of a training batch (about 1 MB). */
size_t ntc_train_batch_workspace_bytes(void);

/* Prepare one optimisation step for each of n_materials materials (HOST
 * arrays mats, trainers, targets, batches; each entry as for ntc_train_step;
 * n_materials in 1..NTC_MAX_TRAIN_BATCH).  Every material is NTC_PREC_F16 on
 * the tensor-core trainer and shares act, interp0 and hidden_layers with the
 * others; sides, channel counts, c0, c1 and k_in may differ.  batches[i] >= 0
 * sampled texels of material i per step; 0 leaves material i out (no update,
 * its step counter unchanged, its loss 0).  Material i samples and draws its
 * noise with seed + i at its own device step counter, as
 * ntc_train_step(.., seed + i, ..) would.  flags: NTC_FLAG_FREEZE_GRIDS,
 * NO_NOISE, CROPS, GRAD_ONLY (NTC_FLAG_SIMT is refused).  loss_out: device
 * [n_materials] floats.  Validates everything, then copies the descriptor into
 * `workspace` (device, caller-owned, ntc_train_batch_workspace_bytes()) on
 * `stream` from pageable memory: call it outside graph capture.  The trainers
 * must be distinct, and the workspace, trainers and targets must stay alive
 * and unmoved while steps of the batch run. */
int ntc_train_batch_prepare(const ntc_material* mats, const ntc_trainer* trainers,
                            const ntc_target* targets, const int64_t* batches,
                            int32_t n_materials, uint64_t seed, int32_t flags, float* loss_out,
                            void* workspace, size_t workspace_bytes, ntc_train_batch* batch_out,
                            void* stream);

/* One optimisation step of every material of a prepared batch: the dense
 * noise pass of every material with a noisy scratch (one launch), the fused
 * forward + loss + backward of all materials' texels in one persistent
 * launch (tiles ordered by material; a CTA restages the weights and flushes
 * its weight-gradient accumulators where its share of tiles crosses from one
 * material to the next), and Adam over every material's parameters (one
 * launch, whose last block advances the step counters).  Each material's
 * result equals that of ntc_train_step with the same arguments, up to the
 * order of floating-point atomic sums.  Only launches kernels and a memset:
 * capturable in a CUDA graph. */
int ntc_train_step_batched(const ntc_train_batch* batch, void* stream);

/* ntc_train_step for callers that cannot allocate device memory: code that
 * runs inside an engine's frame loop or a real-time thread (cudaMalloc may
 * synchronise the device and stall it), code that enqueues into a stream that
 * is being captured into a CUDA graph (allocation is not a capturable
 * operation), and plugins that only receive device buffers from their host.
 * The paper has no counterpart: this is a deployment variant of the same step.
 *
 * Identical to ntc_train_step except that tr->grad is ignored (may be NULL)
 * and NTC_FLAG_GRAD_ONLY is refused with NTC_ERR_ARG (that flag's only
 * result, the gradient, would stay in the library's private array).  Every
 * argument check runs before the call puts anything on `stream`.  Otherwise:
 * the scratch gradient is a fixed array of NTC_NOALLOC_MAX_PARAMS floats
 * (8 MiB) compiled into the library, which every GPU that loads the library
 * holds until the process exits.  tr->n_params above NTC_NOALLOC_MAX_PARAMS
 * is rejected with NTC_ERR_SHAPE.  Each call clears the first n_params floats
 * of the array on `stream` before using it; nothing else is allocated.  The
 * first call on a device looks up the array's device address (with that
 * device current); make that first call before capturing a stream.  All
 * calls on a device share the one array: calls that overlap on the GPU
 * (different streams, or different materials in flight) race and corrupt
 * each other's gradients. */
#define NTC_NOALLOC_MAX_PARAMS (1 << 21)
int ntc_train_step_noalloc(const ntc_material* m, const ntc_trainer* tr, const ntc_target* t,
                           int64_t batch, uint64_t seed, const float* uvl_or_null,
                           float* loss_out, int32_t flags, void* stream);

/* Final quantisation (Sec. 4.2): for `cells` cells of c float32 values,
 * index q = clamp(rint(x / Q) + N/2 - 1, 0, N-1) (ties to even), packed into
 * packed_out ([cells][ntc_cell_bytes(c, bits)], may be NULL) and, if
 * snapped_out is not NULL, the level value (q - (N/2-1)) Q written back as
 * float32 (may alias `values`). */
int ntc_quantize_pack(const float* values, int64_t cells, int32_t c, int32_t bits, float q,
                      uint8_t* packed_out, float* snapped_out, void* stream);

/* Inverse of the packing: indices (int32 [cells][c], may be NULL) and/or
 * level values (float32 [cells][c], may be NULL). */
int ntc_unpack(const uint8_t* packed, int64_t cells, int32_t c, int32_t bits, float q,
               int32_t* idx_out, float* values_out, void* stream);

/* The training-texel sampler of ntc_train_step (Sec. 5.1), exposed for
 * testing: [batch][3] int32 rows (x, y, m) of step `step`, device memory.
 * Every texel draws its own level of detail (with probability 0.05 a mip
 * uniform over the chain, else floor(-log4 X), X uniform in (0, 1], clamped
 * to the last mip) and a uniform texel of that mip. */
int ntc_sample_batch(uint64_t seed, int64_t step, int64_t batch, int32_t width,
                     int32_t height, int32_t mips, int32_t* xym_out, void* stream);

/* The crop sampler of ntc_train_step with NTC_FLAG_CROPS (Sec. 5.1), same
 * output: one level of detail for the whole batch (the rule above), the
 * batch cut into crops of 256 x 256 texels; crop k = i / 65536 has its
 * origin (x0, y0) uniform over the mip and texel i of the batch is
 * ((x0 + i mod 256) mod w_m, (y0 + (i / 256) mod 256) mod h_m), i.e. a crop
 * wraps around the mip's edges (the material tiles).  A mip smaller than
 * the crop repeats inside it. */
int ntc_sample_crops(uint64_t seed, int64_t step, int64_t batch, int32_t width,
                     int32_t height, int32_t mips, int32_t* xym_out, void* stream);

/* Vector quantisation of `cells` rows of c0 float32 values (device) against
 * `books` codebooks [books][256][c0] (device float32), greedy residual
 * search: index b is the entry nearest (squared distance, FP32, channels
 * summed in order without fused multiply-add, ties to the lowest index) to
 * what the entries of books 0..b-1 leave of the row.  idx_out [cells][books]
 * uint8, device.  Produces the indices of a vector-quantised G0. */
int ntc_vq_assign(const float* values, int64_t cells, int32_t c0, const float* codebooks,
                  int32_t books, uint8_t* idx_out, void* stream);

/* The MLP input rows of nearest decodes (Sec. 4.3), exposed for testing:
 * float32 [n][k_in]. */
int ntc_sample_features(const ntc_material* m, const float* uvl, int64_t n, float* rows_out,
                        int32_t flags, uint64_t noise_seed, int64_t noise_step, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* NTC_H */
