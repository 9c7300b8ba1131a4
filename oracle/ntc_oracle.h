/*
 * Neural texture compression -- plain CPU FP64 oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the bench may load this library.  It shares no code, header
 * or constant with the CUDA library; it restates the method of
 * "Random-Access Neural Compression of Material Textures" (Vaidyanathan et
 * al., SIGGRAPH 2023) step by step in double precision, slowly and plainly.
 *
 * Every function names the paper passage it follows.  Readings of points the
 * paper leaves open are stated at the function that takes them.
 */
#ifndef NTC_ORACLE_H
#define NTC_ORACLE_H
#include <stdint.h>

#define OR_MAX_LEVELS 8

/* A material's compressed representation plus its decoder (Sec. 4). */
typedef struct {
  int width, height;        /* mip-0 texture-set resolution w x h (Sec. 4) */
  int channels;             /* c: decoder outputs */
  int mips;                 /* M: mip levels, log2(max(w,h)) + 1 */
  int levels;               /* feature levels F^j (Sec. 4.1, Table 1) */
  int c0, c1;               /* features per cell in G_0 and G_1 */
  int n0, n1;               /* quantisation levels N_k = 2^B_k (Sec. 4.2) */
  double q0, q1;            /* bin width Q_k (Sec. 4.2) */
  int g0w[OR_MAX_LEVELS], g0h[OR_MAX_LEVELS];
  int g1w[OR_MAX_LEVELS], g1h[OR_MAX_LEVELS];
  const double* grid0[OR_MAX_LEVELS]; /* [g0h][g0w][c0] latent values */
  const double* grid1[OR_MAX_LEVELS]; /* [g1h][g1w][c1] */
  int k_in, hidden;         /* MLP input width (zero padded) and hidden width */
  int act;                  /* 0 ReLU, 1 hardGELU (Sec. 4.4) */
  int out_act;              /* 0 sigmoid, 1 identity */
  const double *w1, *b1;    /* [hidden][k_in], [hidden] */
  const double *w2, *b2;    /* [hidden][hidden], [hidden] */
  const double *w3, *b3;    /* [channels][hidden], [channels] */
  int interp0;              /* G0 resampling (Sec. 4.3.1): 0 bilinear, 1 learned
                               interpolation (the four taps concatenated) */
  int hidden_layers;        /* hidden layers with activations: 2, or 3 (Sec. 4.4
                               gives activations to three layers after the
                               first): a third hidden layer wm, bm between w2
                               and the output layer w3 */
  const double *wm, *bm;    /* [hidden][hidden], [hidden] (hidden_layers == 3) */
  int vq_g0;                /* G0 holds vector-quantised values: the training noise
                               applies to G1 only */
  const double* f8_sa;      /* FP8-E4M3 form (NULL: off; the paper trains with
                               half-precision tensor cores, Sec. 5.1, and leaves
                               lower precision to future work, Sec. 7): per-layer activation
                               scales s_a[3]; every layer input v is used as
                               s_a[l] e4m3(v / s_a[l]) (two hidden layers; the
                               weights are given already quantised).  Reverse
                               mode treats each rounding as the identity
                               (straight-through), so the weight gradients see
                               the rounded inputs and the input gradients pass
                               through the roundings unchanged. */
} or_model;

/* Simulated-quantisation noise switch (Sec. 4.2). */
typedef struct {
  int enabled;
  uint64_t seed;
  int64_t step;
} or_noise;

/* Gradient outputs, accumulated (+=) into caller-zeroed arrays. */
typedef struct {
  double* grid0[OR_MAX_LEVELS];
  double* grid1[OR_MAX_LEVELS];
  double *w1, *b1, *w2, *b2, *w3, *b3;
  double *wm, *bm;          /* third hidden layer (hidden_layers == 3) */
  double* rows;             /* nullable: [n][k_in] gradient of each texel's MLP
                               input row (written, not accumulated) */
} or_grads;

/* --- pyramid (Sec. 4.1, Table 1) --- */
int or_mips(int width, int height);
int or_pyramid(int width, int height, int* g0w, int* g0h, int* g1w, int* g1h);
int or_level_of_mip(int mip, int levels);

/* --- quantisation (Sec. 4.2) --- */
void or_quantize(const double* x, int64_t n, int n_levels, double q, int32_t* idx);
void or_dequantize(const int32_t* idx, int64_t n, int n_levels, double q, double* x);
int or_cell_bytes(int c, int bits);
void or_pack(const int32_t* idx, int64_t cells, int c, int bits, uint8_t* out);
void or_unpack(const uint8_t* in, int64_t cells, int c, int bits, int32_t* idx);

/* --- counter-based random numbers (SplitMix64 output function) --- */
uint64_t or_splitmix64(uint64_t x);
uint64_t or_rng(uint64_t seed, uint64_t stream, uint64_t counter);
double or_noise_value(uint64_t seed, int64_t step, int level, int grid, int64_t cell,
                      int ch, int c, double q);
void or_sample_batch(uint64_t seed, int64_t step, int64_t batch, int width, int height,
                     int mips, int32_t* xym);
void or_sample_batch_crops(uint64_t seed, int64_t step, int64_t batch, int width, int height,
                           int mips, int32_t* xym);

/* --- sampling + decoder (Sec. 4.3, 4.4) --- */
void or_positional_encoding(int x, int y, double* pe12);
double or_activation(int act, double z);
double or_activation_grad(int act, double z);
void or_features(const or_model* md, int x, int y, int m, const or_noise* nz, double* row);
void or_features_uvl(const or_model* md, int64_t n, const float* uvl, double* rows);
void or_decode_xym(const or_model* md, int64_t n, const int32_t* xym, const or_noise* nz,
                   double* out, int nthreads);
void or_decode_uvl(const or_model* md, int64_t n, const float* uvl, const or_noise* nz,
                   double* out, int nthreads);
void or_decode_trilinear(const or_model* md, int64_t n, const float* uvl, double* out,
                         int nthreads);
/* Stochastic filtering (Sec. 5.3): one nearest decode per query at the
 * jittered texel and mip of frame `step` (see ntc_oracle.c). */
void or_decode_stochastic(const or_model* md, int64_t n, const float* uvl, uint64_t seed,
                          int64_t step, double* out, int nthreads);

/* --- FP8-E4M3 (OCP 8-bit floating point: bias 7, 3 mantissa bits, ties to
 * even, saturating at 448, no infinities) --- */
double or_round_e4m3(double v);

/* --- backward and loss (Sec. 4.5, 5.1) --- */
void or_backward_xym(const or_model* md, int64_t n, const int32_t* xym, const double* dout,
                     const or_noise* nz, const or_grads* g, int nthreads);
double or_loss_grad_xym(const or_model* md, int64_t n, const int32_t* xym,
                        const double* target, const or_noise* nz, const or_grads* g,
                        int nthreads);

/* --- optimiser (Sec. 5.1) --- */
double or_cosine_lr(double lr0, int64_t t, int64_t total);
void or_adam(double* p, double* m, double* v, const double* g, int64_t n, double lr,
             int64_t t, double beta1, double beta2, double eps, int clamp, double lo,
             double hi);

#endif
