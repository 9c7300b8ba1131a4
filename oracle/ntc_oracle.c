/*
 * Neural texture compression -- plain CPU FP64 oracle (implementation).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * bench's CPU-baseline leg, never by the product path.  Plain loops in double
 * precision; no blocking, fusion or reordering beyond what the method states.
 * Shares no code with the CUDA library.
 *
 * Paper: "Random-Access Neural Compression of Material Textures",
 * Vaidyanathan et al., 2023.  Section numbers below are the paper's.
 */
#include "ntc_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

static int imax(int a, int b) { return a > b ? a : b; }
static int imin(int a, int b) { return a < b ? a : b; }

/* ------------------------------------------------------------------------ */
/* Feature pyramid (Sec. 4.1, Table 1)                                       */
/* ------------------------------------------------------------------------ */

/* Number of mip levels of a w x h texture set: down to 1x1. */
int or_mips(int width, int height) {
  int s = imax(width, height), m = 1;
  while (s > 1) { s >>= 1; ++m; }
  return m;
}

/* Grid resolutions of every feature level.  Table 1 (1024^2 set): G0 is a
 * quarter of the texture side at level 0 and shrinks by 4 per level; G1 is
 * half of G0.  Levels continue while G0 is at least 4 cells on its longer
 * side (1024^2 -> 256, 64, 16, 4), i.e. until the grids "cannot be further
 * downsampled"; at least one level always exists.  Returns the level count. */
int or_pyramid(int width, int height, int* g0w, int* g0h, int* g1w, int* g1h) {
  int levels = 0;
  for (int j = 0; j < OR_MAX_LEVELS; ++j) {
    int sh = 2 * j + 2;
    int w0 = imax(1, width >> sh), h0 = imax(1, height >> sh);
    if (j > 0 && imax(w0, h0) < 4) break;
    g0w[j] = w0; g0h[j] = h0;
    g1w[j] = imax(1, w0 >> 1); g1h[j] = imax(1, h0 >> 1);
    ++levels;
  }
  return levels;
}

/* Feature level that predicts mip m (Table 1): level 0 serves mips 0..3,
 * every further level two mips (4,5 -> 1; 6,7 -> 2; ...), and the last level
 * also serves every mip below it. */
int or_level_of_mip(int mip, int levels) {
  int j = (mip < 4) ? 0 : (mip - 2) / 2;
  return imin(j, levels - 1);
}

/* ------------------------------------------------------------------------ */
/* Quantisation (Sec. 4.2)                                                   */
/* ------------------------------------------------------------------------ */

/* The N quantisation levels are k*Q for integers k in [-(N/2-1), N/2]: the
 * asymmetric range of Sec. 4.2 puts zero exactly on a level.  Index
 * q = k + (N/2 - 1) in [0, N-1].  Rounding is to nearest, ties to even. */
void or_quantize(const double* x, int64_t n, int n_levels, double q, int32_t* idx) {
  int off = n_levels / 2 - 1;
  for (int64_t i = 0; i < n; ++i) {
    double k = rint(x[i] / q) + off;
    if (k < 0) k = 0;
    if (k > n_levels - 1) k = n_levels - 1;
    idx[i] = (int32_t)k;
  }
}

void or_dequantize(const int32_t* idx, int64_t n, int n_levels, double q, double* x) {
  int off = n_levels / 2 - 1;
  for (int64_t i = 0; i < n; ++i) x[i] = (double)(idx[i] - off) * q;
}

/* Bytes per packed cell: c*bits bits rounded up to a power-of-two number of
 * bytes, so that one aligned load fetches a whole cell. */
int or_cell_bytes(int c, int bits) {
  int need = (c * bits + 7) / 8, b = 1;
  while (b < need) b <<= 1;
  return b;
}

/* Channel ch of a cell occupies bits [ch*bits, ch*bits + bits) of the cell,
 * counting from bit 0 of byte 0 (little endian, lowest bits first). */
void or_pack(const int32_t* idx, int64_t cells, int c, int bits, uint8_t* out) {
  int cb = or_cell_bytes(c, bits);
  memset(out, 0, (size_t)(cells * cb));
  for (int64_t i = 0; i < cells; ++i)
    for (int ch = 0; ch < c; ++ch) {
      int bit = ch * bits;
      out[i * cb + bit / 8] |= (uint8_t)((idx[i * c + ch] & ((1 << bits) - 1)) << (bit % 8));
    }
}

void or_unpack(const uint8_t* in, int64_t cells, int c, int bits, int32_t* idx) {
  int cb = or_cell_bytes(c, bits);
  for (int64_t i = 0; i < cells; ++i)
    for (int ch = 0; ch < c; ++ch) {
      int bit = ch * bits;
      idx[i * c + ch] = (in[i * cb + bit / 8] >> (bit % 8)) & ((1 << bits) - 1);
    }
}

/* ------------------------------------------------------------------------ */
/* Counter-based random numbers                                              */
/* ------------------------------------------------------------------------ */

/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): add the golden gamma, then
 * the variant-13 output mix.  Written from the published definition. */
static uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t or_splitmix64(uint64_t x) { return splitmix64(x); }

/* One 64-bit draw for (seed, stream, counter). */
uint64_t or_rng(uint64_t seed, uint64_t stream, uint64_t counter) {
  uint64_t key = splitmix64(seed ^ splitmix64(stream));
  return splitmix64(key ^ counter);
}

/* Uniform noise in [-Q/2, Q/2) for one latent value (Sec. 4.2).  Reading:
 * one value per (step, feature level, grid, cell, channel).  One 64-bit draw
 * serves a channel pair: counter = (2*level + grid) << 40 | (cell *
 * ceil(c/2) + ch/2) on stream 2*step + 1; even channels take draw bits
 * 40..63, odd channels bits 16..39, as a 24-bit fraction u; noise (u-1/2) Q. */
double or_noise_value(uint64_t seed, int64_t step, int level, int grid, int64_t cell,
                      int ch, int c, double q) {
  uint64_t stream = ((uint64_t)step << 1) | 1u;
  uint64_t pairs = (uint64_t)((c + 1) / 2);
  uint64_t counter = ((uint64_t)(2 * level + grid) << 40) | ((uint64_t)cell * pairs + (uint64_t)(ch / 2));
  uint64_t h = or_rng(seed, stream, counter);
  uint64_t bits24 = (ch & 1) ? ((h >> 16) & 0xFFFFFFULL) : (h >> 40);
  double u = (double)bits24 * (1.0 / 16777216.0);
  return (u - 0.5) * q;
}

/* Level of detail of one training draw (Sec. 5.1): LOD = floor(-log4 X),
 * X ~ U(0,1], and with probability 0.05 a LOD uniform over the mip chain
 * instead.  Reading: X = k / 2^24 with k = (draw >> 40) + 1, so
 * floor(-log4 X) is the largest m with k <= 2^(24-2m), clamped to the last
 * mip; counters c_mode (the 5% choice and the uniform mip) and c_exp. */
static int or_train_lod(uint64_t seed, uint64_t stream, uint64_t c_mode, uint64_t c_exp,
                        int mips) {
  uint64_t h0 = or_rng(seed, stream, c_mode);
  if ((h0 >> 40) < 838861ULL) /* 0.05 * 2^24, rounded up */
    return (int)(((h0 & 0xFFFFFFFFULL) * (uint64_t)mips) >> 32);
  uint64_t k = (or_rng(seed, stream, c_exp) >> 40) + 1;
  int m = 0;
  while (m + 1 <= 12 && k <= (1ULL << (24 - 2 * (m + 1)))) ++m;
  return m > mips - 1 ? mips - 1 : m;
}

/* A uniform integer in [0, n) from 32 random bits (fixed-point product). */
static uint64_t or_uniform_below(uint64_t bits32, uint64_t n) { return (bits32 * n) >> 32; }

/* Training-batch texels (Sec. 5.1), independent texels: each texel i draws
 * its LOD (counters 4i, 4i+1) and a uniform texel of that mip (counter
 * 4i+2).  Output rows (x, y, m). */
void or_sample_batch(uint64_t seed, int64_t step, int64_t batch, int width, int height,
                     int mips, int32_t* xym) {
  uint64_t stream = ((uint64_t)step << 1);
  for (int64_t i = 0; i < batch; ++i) {
    int m = or_train_lod(seed, stream, 4 * (uint64_t)i + 0, 4 * (uint64_t)i + 1, mips);
    uint64_t h2 = or_rng(seed, stream, 4 * (uint64_t)i + 2);
    uint64_t wm = (uint64_t)imax(1, width >> m), hm = (uint64_t)imax(1, height >> m);
    xym[3 * i + 0] = (int32_t)or_uniform_below(h2 & 0xFFFFFFFFULL, wm);
    xym[3 * i + 1] = (int32_t)or_uniform_below(h2 >> 32, hm);
    xym[3 * i + 2] = m;
  }
}

/* Training-batch texels (Sec. 5.1), crops: the batch is a sequence of
 * square crops of side S = 256 taken from one level of detail, drawn once
 * for the batch (counters 0, 1).  Crop k starts at a uniform texel (x0, y0)
 * of that mip (counter 4k+2); reading: a crop that runs past the mip's edge
 * wraps around (the material tiles), so a mip smaller than S repeats inside
 * the crop.  The crop is walked row by row: its texel (cx, cy) is batch
 * entry k S^2 + cy S + cx. */
void or_sample_batch_crops(uint64_t seed, int64_t step, int64_t batch, int width, int height,
                           int mips, int32_t* xym) {
  const int64_t S = 256;
  uint64_t stream = ((uint64_t)step << 1);
  int m = or_train_lod(seed, stream, 0, 1, mips);
  int64_t wm = imax(1, width >> m), hm = imax(1, height >> m);
  int64_t n_crops = (batch + S * S - 1) / (S * S);
  for (int64_t k = 0; k < n_crops; ++k) {
    uint64_t h = or_rng(seed, stream, 4 * (uint64_t)k + 2);
    int64_t x0 = (int64_t)or_uniform_below(h & 0xFFFFFFFFULL, (uint64_t)wm);
    int64_t y0 = (int64_t)or_uniform_below(h >> 32, (uint64_t)hm);
    for (int64_t cy = 0; cy < S; ++cy)
      for (int64_t cx = 0; cx < S; ++cx) {
        int64_t i = k * S * S + cy * S + cx;
        if (i >= batch) return;
        xym[3 * i + 0] = (int32_t)((x0 + cx) % wm);
        xym[3 * i + 1] = (int32_t)((y0 + cy) % hm);
        xym[3 * i + 2] = m;
      }
  }
}

/* ------------------------------------------------------------------------ */
/* Sampling and concatenation (Sec. 4.3)                                     */
/* ------------------------------------------------------------------------ */

/* Triangle wave with period 1: +1 at t = 0, -1 at t = 1/2. */
static double tri(double t) { return 4.0 * fabs(t - 0.5) - 1.0; }
static double fracd(double t) { return t - floor(t); }

/* Tiled positional encoding (Sec. 4.3.2, Fig. 5): log2(8) = 3 octaves of
 * triangle waves over the texel position inside an 8x8 tile, a sine-like and
 * a cosine-like wave per octave, 6 values for x then 6 for y.  Periods are
 * 8, 4 and 2 texels, sampled at texel centres; the period-2 cosine-like wave
 * is 0 at every texel centre -- the constant last value of each axis. */
void or_positional_encoding(int x, int y, double* pe) {
  int coord[2] = {x, y};
  for (int a = 0; a < 2; ++a)
    for (int h = 0; h < 3; ++h) {
      double period = 8.0 / (double)(1 << h);
      double t = fracd(((double)coord[a] + 0.5) / period);
      pe[6 * a + 2 * h + 0] = tri(fracd(t - 0.25));
      pe[6 * a + 2 * h + 1] = tri(t);
    }
}

static int mip_w(const or_model* md, int m) { return imax(1, md->width >> m); }
static int mip_h(const or_model* md, int m) { return imax(1, md->height >> m); }

/* Bilinear taps of a gw x gh grid at the centre of texel (x, y) of mip m
 * (Sec. 4.3.1).  Reading: texel centre (x+1/2)/w_m maps onto the grid with
 * cell centres at (i+1/2)/gw; taps are clamped to the grid edge. */
static void bilinear_taps(int x, int y, int wm, int hm, int gw, int gh, int64_t cell[4],
                          double wt[4]) {
  double px = ((x + 0.5) / wm) * gw - 0.5;
  double py = ((y + 0.5) / hm) * gh - 0.5;
  double fx0 = floor(px), fy0 = floor(py);
  double fx = px - fx0, fy = py - fy0;
  int ix0 = (int)fx0, iy0 = (int)fy0;
  int ix1 = ix0 + 1, iy1 = iy0 + 1;
  ix0 = imin(imax(ix0, 0), gw - 1); ix1 = imin(imax(ix1, 0), gw - 1);
  iy0 = imin(imax(iy0, 0), gh - 1); iy1 = imin(imax(iy1, 0), gh - 1);
  cell[0] = (int64_t)iy0 * gw + ix0; wt[0] = (1 - fx) * (1 - fy);
  cell[1] = (int64_t)iy0 * gw + ix1; wt[1] = fx * (1 - fy);
  cell[2] = (int64_t)iy1 * gw + ix0; wt[2] = (1 - fx) * fy;
  cell[3] = (int64_t)iy1 * gw + ix1; wt[3] = fx * fy;
}

/* Latent value at (level j, grid k, cell, ch), plus training noise. */
static double grid_value(const or_model* md, int j, int k, int64_t cell, int ch,
                         const or_noise* nz) {
  const double* g = k ? md->grid1[j] : md->grid0[j];
  int c = k ? md->c1 : md->c0;
  double v = g[cell * c + ch];
  /* a vector-quantised G0 is trained through its quantised values: no noise */
  if (nz && nz->enabled && !(k == 0 && md->vq_g0))
    v += or_noise_value(nz->seed, nz->step, j, k, cell, ch, c, k ? md->q1 : md->q0);
  return v;
}

/* The decoder's input row (Sec. 4.3, 4.4): bilinear G0 features, bilinear G1
 * features, 12 positional-encoding values, the normalised LOD m/(M-1), then
 * zeros up to k_in. */
/* Width of the G0 part of the input row: c0 (bilinear) or 4 c0 (learned
 * interpolation, Sec. 4.3.1: the four neighbouring feature vectors of the
 * bilinear footprint concatenated, taps in the order (x0,y0), (x1,y0),
 * (x0,y1), (x1,y1), so that the MLP weighs them by the texel's phase). */
static int g0_width(const or_model* md) { return md->interp0 ? 4 * md->c0 : md->c0; }

void or_features(const or_model* md, int x, int y, int m, const or_noise* nz, double* row) {
  int j = or_level_of_mip(m, md->levels);
  int wm = mip_w(md, m), hm = mip_h(md, m);
  for (int i = 0; i < md->k_in; ++i) row[i] = 0.0;
  for (int k = 0; k < 2; ++k) {
    int gw = k ? md->g1w[j] : md->g0w[j], gh = k ? md->g1h[j] : md->g0h[j];
    int c = k ? md->c1 : md->c0, base = k ? g0_width(md) : 0;
    int64_t cell[4]; double wt[4];
    bilinear_taps(x, y, wm, hm, gw, gh, cell, wt);
    if (k == 0 && md->interp0) {
      for (int t = 0; t < 4; ++t)
        for (int ch = 0; ch < c; ++ch) row[t * c + ch] = grid_value(md, j, 0, cell[t], ch, nz);
      continue;
    }
    for (int ch = 0; ch < c; ++ch) {
      double s = 0.0;
      for (int t = 0; t < 4; ++t) s += wt[t] * grid_value(md, j, k, cell[t], ch, nz);
      row[base + ch] = s;
    }
  }
  double* pe = row + g0_width(md) + md->c1;
  or_positional_encoding(x, y, pe);
  pe[12] = md->mips > 1 ? (double)m / (double)(md->mips - 1) : 0.0;
}

/* ------------------------------------------------------------------------ */
/* Decoder MLP (Sec. 4.4)                                                    */
/* ------------------------------------------------------------------------ */

/* hardGELU (Sec. 4.4) or ReLU. */
static double act_f(int act, double z) {
  if (act == 1) {
    if (z < -1.5) return 0.0;
    if (z > 1.5) return z;
    return z / 3.0 * (z + 1.5);
  }
  return z > 0.0 ? z : 0.0;
}
static double act_df(int act, double z) {
  if (act == 1) {
    if (z < -1.5) return 0.0;
    if (z > 1.5) return 1.0;
    return (2.0 * z + 1.5) / 3.0;
  }
  return z > 0.0 ? 1.0 : 0.0;
}

double or_activation(int act, double z) { return act_f(act, z); }
double or_activation_grad(int act, double z) { return act_df(act, z); }

typedef struct {
  double *x, *z1, *h1, *z2, *h2, *zm, *hm, *z3, *y;
} mlp_buf;

static void mlp_alloc(const or_model* md, mlp_buf* b) {
  b->x = calloc((size_t)md->k_in, sizeof(double));
  b->z1 = calloc((size_t)md->hidden, sizeof(double));
  b->h1 = calloc((size_t)md->hidden, sizeof(double));
  b->z2 = calloc((size_t)md->hidden, sizeof(double));
  b->h2 = calloc((size_t)md->hidden, sizeof(double));
  b->zm = calloc((size_t)md->hidden, sizeof(double));
  b->hm = calloc((size_t)md->hidden, sizeof(double));
  b->z3 = calloc((size_t)md->channels, sizeof(double));
  b->y = calloc((size_t)md->channels, sizeof(double));
}
static void mlp_free(mlp_buf* b) {
  free(b->x); free(b->z1); free(b->h1); free(b->z2); free(b->h2); free(b->zm); free(b->hm);
  free(b->z3); free(b->y);
}

/* z = W v + b for W stored [out][in]. */
static void linear(const double* w, const double* bias, const double* v, int in, int out,
                   double* z) {
  for (int o = 0; o < out; ++o) {
    double s = bias[o];
    for (int i = 0; i < in; ++i) s += w[(int64_t)o * in + i] * v[i];
    z[o] = s;
  }
}

/* The last hidden activation: h2, or hm with a third hidden layer. */
static const double* last_hidden(const or_model* md, const mlp_buf* b) {
  return md->hidden_layers == 3 ? b->hm : b->h2;
}

/* Nearest FP8-E4M3 value: in the binade [2^e, 2^(e+1)) the values are the
 * multiples of 2^(e-3) for e >= -6; below 2^-6 the subnormals are multiples
 * of 2^-9; rint rounds half to even; magnitudes above 448 saturate. */
double or_round_e4m3(double v) {
  double a = fabs(v);
  int e = 0;
  frexp(a, &e); /* a = f 2^e, f in [0.5, 1) */
  int ex = e - 1 < -6 ? -6 : e - 1;
  double quantum = ldexp(1.0, ex - 3);
  double r = rint(a / quantum) * quantum;
  if (r > 448.0) r = 448.0;
  return copysign(r, v);
}

/* FP8 form: a layer input used in units of its activation scale, rounded. */
static void round_input(const or_model* md, int layer, double* v, int n) {
  if (!md->f8_sa) return;
  double s = md->f8_sa[layer];
  for (int i = 0; i < n; ++i) v[i] = s * or_round_e4m3(v[i] / s);
}

/* Linear layers with hidden activations, then the output layer and its
 * activation (Sec. 4.4): two hidden layers, or three.  In the FP8 form the
 * buffers x, h1, h2 end up holding the rounded layer inputs. */
static void mlp_forward(const or_model* md, mlp_buf* b) {
  int H = md->hidden, C = md->channels;
  round_input(md, 0, b->x, md->k_in);
  linear(md->w1, md->b1, b->x, md->k_in, H, b->z1);
  for (int i = 0; i < H; ++i) b->h1[i] = act_f(md->act, b->z1[i]);
  round_input(md, 1, b->h1, H);
  linear(md->w2, md->b2, b->h1, H, H, b->z2);
  for (int i = 0; i < H; ++i) b->h2[i] = act_f(md->act, b->z2[i]);
  round_input(md, 2, b->h2, H);
  if (md->hidden_layers == 3) {
    linear(md->wm, md->bm, b->h2, H, H, b->zm);
    for (int i = 0; i < H; ++i) b->hm[i] = act_f(md->act, b->zm[i]);
  }
  linear(md->w3, md->b3, last_hidden(md, b), H, C, b->z3);
  for (int i = 0; i < C; ++i)
    b->y[i] = md->out_act == 1 ? b->z3[i] : 1.0 / (1.0 + exp(-b->z3[i]));
}

/* Nearest-texel query -> (x, y, m) (Sec. 5.3: decode at a texel; filtering is
 * built on top).  m = floor(lod) clamped to [0, M-1]; x = floor(u * w_m)
 * clamped to [0, w_m - 1]; a NaN coordinate counts as 0. */
static void query_to_xym(const or_model* md, float u, float v, float lod, int* x, int* y,
                         int* m) {
  int mm;
  if (!(lod >= 0.0f)) mm = 0;
  else if (lod >= (float)(md->mips - 1)) mm = md->mips - 1;
  else mm = (int)floor((double)lod);
  int wm = mip_w(md, mm), hm = mip_h(md, mm);
  double tu = (double)u * wm, tv = (double)v * hm;
  int xx = !(tu >= 0.0) ? 0 : (tu >= wm ? wm - 1 : (int)floor(tu));
  int yy = !(tv >= 0.0) ? 0 : (tv >= hm ? hm - 1 : (int)floor(tv));
  *x = xx; *y = yy; *m = mm;
}

/* ------------------------------------------------------------------------ */
/* Threading helper: contiguous chunks of [0, n), one per thread.            */
/* ------------------------------------------------------------------------ */
typedef struct job_s {
  void (*fn)(struct job_s*, int64_t, int64_t);
  const or_model* md;
  const int32_t* xym;
  const float* uvl;
  const double* dout;
  const double* target;
  const or_noise* nz;
  double* out;
  or_grads g;       /* this thread's private accumulators */
  double* rows;     /* the caller's per-texel input-row gradients, or NULL */
  double loss;
  uint64_t seed;    /* stochastic filtering: seed and frame of the jitter */
  int64_t step;
  int64_t lo, hi;
} job;

static void* job_entry(void* p) {
  job* jb = (job*)p;
  jb->fn(jb, jb->lo, jb->hi);
  return NULL;
}

static void run_jobs(job* jobs, int nthreads, int64_t n) {
  pthread_t* th = calloc((size_t)nthreads, sizeof(pthread_t));
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].lo = n * t / nthreads;
    jobs[t].hi = n * (t + 1) / nthreads;
  }
  for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, job_entry, &jobs[t]);
  job_entry(&jobs[0]);
  for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
  free(th);
}

static int clamp_threads(int nthreads, int64_t n) {
  if (nthreads < 1) nthreads = 1;
  if (n < nthreads) nthreads = (int)(n > 0 ? n : 1);
  return nthreads;
}

/* ------------------------------------------------------------------------ */
/* Decode                                                                    */
/* ------------------------------------------------------------------------ */
static void decode_xym_job(job* jb, int64_t lo, int64_t hi) {
  mlp_buf b;
  mlp_alloc(jb->md, &b);
  int C = jb->md->channels;
  for (int64_t i = lo; i < hi; ++i) {
    or_features(jb->md, jb->xym[3 * i], jb->xym[3 * i + 1], jb->xym[3 * i + 2], jb->nz, b.x);
    mlp_forward(jb->md, &b);
    for (int c = 0; c < C; ++c) jb->out[i * C + c] = b.y[c];
  }
  mlp_free(&b);
}

void or_decode_xym(const or_model* md, int64_t n, const int32_t* xym, const or_noise* nz,
                   double* out, int nthreads) {
  nthreads = clamp_threads(nthreads, n);
  job* jobs = calloc((size_t)nthreads, sizeof(job));
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].fn = decode_xym_job; jobs[t].md = md; jobs[t].xym = xym; jobs[t].nz = nz;
    jobs[t].out = out;
  }
  run_jobs(jobs, nthreads, n);
  free(jobs);
}

static void decode_uvl_job(job* jb, int64_t lo, int64_t hi) {
  mlp_buf b;
  mlp_alloc(jb->md, &b);
  int C = jb->md->channels;
  for (int64_t i = lo; i < hi; ++i) {
    int x, y, m;
    query_to_xym(jb->md, jb->uvl[3 * i], jb->uvl[3 * i + 1], jb->uvl[3 * i + 2], &x, &y, &m);
    or_features(jb->md, x, y, m, jb->nz, b.x);
    mlp_forward(jb->md, &b);
    for (int c = 0; c < C; ++c) jb->out[i * C + c] = b.y[c];
  }
  mlp_free(&b);
}

/* The MLP input rows of the nearest texels of n queries (no noise). */
void or_features_uvl(const or_model* md, int64_t n, const float* uvl, double* rows) {
  for (int64_t i = 0; i < n; ++i) {
    int x, y, m;
    query_to_xym(md, uvl[3 * i], uvl[3 * i + 1], uvl[3 * i + 2], &x, &y, &m);
    or_features(md, x, y, m, NULL, rows + i * (int64_t)md->k_in);
  }
}

void or_decode_uvl(const or_model* md, int64_t n, const float* uvl, const or_noise* nz,
                   double* out, int nthreads) {
  nthreads = clamp_threads(nthreads, n);
  job* jobs = calloc((size_t)nthreads, sizeof(job));
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].fn = decode_uvl_job; jobs[t].md = md; jobs[t].uvl = uvl; jobs[t].nz = nz;
    jobs[t].out = out;
  }
  run_jobs(jobs, nthreads, n);
  free(jobs);
}

/* Software trilinear filtering (Sec. 5.3): decode the 2x2 texels around
 * (u, v) on mips floor(lambda) and floor(lambda)+1 (8 decodes) and blend them
 * with bilinear weights inside each mip and linear weights across the two.
 * Readings: lambda is clamped to [0, M-1] (NaN -> 0); the upper mip is
 * clamped to M-1; texel taps wrap around (a material repeats on a surface). */
static void decode_tri_job(job* jb, int64_t lo, int64_t hi) {
  const or_model* md = jb->md;
  mlp_buf b;
  mlp_alloc(md, &b);
  int C = md->channels;
  double* acc = calloc((size_t)C, sizeof(double));
  for (int64_t i = lo; i < hi; ++i) {
    float u = jb->uvl[3 * i], v = jb->uvl[3 * i + 1], lam = jb->uvl[3 * i + 2];
    double l = !(lam >= 0.0f) ? 0.0 : ((double)lam > md->mips - 1 ? md->mips - 1 : (double)lam);
    int m0 = (int)floor(l);
    if (m0 > md->mips - 1) m0 = md->mips - 1;
    int m1 = imin(m0 + 1, md->mips - 1);
    double t = l - m0;
    for (int c = 0; c < C; ++c) acc[c] = 0.0;
    for (int s = 0; s < 2; ++s) {
      int m = s ? m1 : m0;
      double wl = s ? t : 1.0 - t;
      int wm = mip_w(md, m), hm = mip_h(md, m);
      double px = (double)u * wm - 0.5, py = (double)v * hm - 0.5;
      double fx0 = floor(px), fy0 = floor(py);
      double fx = px - fx0, fy = py - fy0;
      int x0 = (int)fx0, y0 = (int)fy0;
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          int xx = ((x0 + dx) % wm + wm) % wm, yy = ((y0 + dy) % hm + hm) % hm;
          double w = wl * (dx ? fx : 1.0 - fx) * (dy ? fy : 1.0 - fy);
          or_features(md, xx, yy, m, NULL, b.x);
          mlp_forward(md, &b);
          for (int c = 0; c < C; ++c) acc[c] += w * b.y[c];
        }
    }
    for (int c = 0; c < C; ++c) jb->out[i * C + c] = acc[c];
  }
  free(acc);
  mlp_free(&b);
}

void or_decode_trilinear(const or_model* md, int64_t n, const float* uvl, double* out,
                         int nthreads) {
  nthreads = clamp_threads(nthreads, n);
  job* jobs = calloc((size_t)nthreads, sizeof(job));
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].fn = decode_tri_job; jobs[t].md = md; jobs[t].uvl = uvl; jobs[t].out = out;
  }
  run_jobs(jobs, nthreads, n);
  free(jobs);
}


/* Stochastic filtering (Sec. 5.3): add noise to the texel position and the
 * LOD, then take the nearest texel -- one decode per query, equal to the
 * trilinear filter above in expectation.  Reading of the noise: per query q
 * of frame `step` one 64-bit draw h on stream 4*step + 2 (counter q); xi_x
 * = h bits 40..63, xi_y = bits 16..39 as 24-bit fractions, xi_l = bits 0..15
 * as a 16-bit fraction, all uniform in [0, 1).  The texel is the nearest one
 * of the jittered position u*w_m - 1/2 + xi_x (x0 with probability 1 - f,
 * x0 + 1 with probability f: the bilinear weights), wrapped like the
 * trilinear taps; the mip floor(lod + xi_l) (the linear weights across
 * mips).  The texel choice is an integer decided in FP32, the kernels'
 * precision: each step below is one FP32 operation (this file is compiled
 * without FMA contraction); u is taken as 0 when NaN and clamped to
 * [-16384, 16384]. */
static int stoch_mip(float lod, int mips, uint64_t h) {
  float xl = (float)(uint32_t)(h & 0xFFFFu) * (1.0f / 65536.0f);
  float l = !(lod >= 0.0f) ? 0.0f : (lod > (float)(mips - 1) ? (float)(mips - 1) : lod);
  float s = l + xl;
  int m = (int)floorf(s);
  return m < mips - 1 ? m : mips - 1;
}

static int stoch_coord(float u, int w, uint32_t b24) {
  float xi = (float)b24 * (1.0f / 16777216.0f);
  float uc = (u == u) ? u : 0.0f;
  if (uc < -16384.0f) uc = -16384.0f;
  if (uc > 16384.0f) uc = 16384.0f;
  float p = uc * (float)w;
  p = p - 0.5f;
  p = p + xi;
  int i = (int)floorf(p);
  return ((i % w) + w) % w;
}

static void decode_stoch_job(job* jb, int64_t lo, int64_t hi) {
  const or_model* md = jb->md;
  mlp_buf b;
  mlp_alloc(md, &b);
  int C = md->channels;
  for (int64_t i = lo; i < hi; ++i) {
    float u = jb->uvl[3 * i], v = jb->uvl[3 * i + 1], lod = jb->uvl[3 * i + 2];
    uint64_t h = or_rng(jb->seed, ((uint64_t)jb->step << 2) | 2u, (uint64_t)i);
    int m = stoch_mip(lod, md->mips, h);
    int x = stoch_coord(u, mip_w(md, m), (uint32_t)(h >> 40));
    int y = stoch_coord(v, mip_h(md, m), (uint32_t)((h >> 16) & 0xFFFFFFu));
    or_features(md, x, y, m, NULL, b.x);
    mlp_forward(md, &b);
    for (int c = 0; c < C; ++c) jb->out[i * C + c] = b.y[c];
  }
  mlp_free(&b);
}

void or_decode_stochastic(const or_model* md, int64_t n, const float* uvl, uint64_t seed,
                          int64_t step, double* out, int nthreads) {
  nthreads = clamp_threads(nthreads, n);
  job* jobs = calloc((size_t)nthreads, sizeof(job));
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].fn = decode_stoch_job; jobs[t].md = md; jobs[t].uvl = uvl; jobs[t].out = out;
    jobs[t].seed = seed; jobs[t].step = step;
  }
  run_jobs(jobs, nthreads, n);
  free(jobs);
}

/* ------------------------------------------------------------------------ */
/* Backward (Sec. 4.5, 5.1): exact reverse mode of the decode above.         */
/* ------------------------------------------------------------------------ */

/* Gradient of sum_i sum_c dout[i][c] * y[i][c] with respect to every latent
 * value and every weight, for one texel, accumulated into g.  The noise adds
 * a constant, so it passes gradients unchanged; clamping to the quantisation
 * range happens after the update (Sec. 4.2) and is not differentiated. */
static void backward_one(const or_model* md, int x, int y, int m, const double* dy,
                         const or_noise* nz, mlp_buf* b, const or_grads* g, double* drow) {
  int K = md->k_in, H = md->hidden, C = md->channels;
  or_features(md, x, y, m, nz, b->x);
  mlp_forward(md, b);
  double dz3[64], dh2[256], dz2[256], dh1[256], dz1[256], dx[256], dhm[256], dzm[256];
  const double* hl = last_hidden(md, b);
  for (int c = 0; c < C; ++c) {
    double d = md->out_act == 1 ? 1.0 : b->y[c] * (1.0 - b->y[c]);
    dz3[c] = dy[c] * d;
  }
  for (int c = 0; c < C; ++c) {
    g->b3[c] += dz3[c];
    for (int i = 0; i < H; ++i) g->w3[(int64_t)c * H + i] += dz3[c] * hl[i];
  }
  if (md->hidden_layers == 3) {
    /* through the third hidden layer: dhm = W3^T dz3, dzm = dhm act'(zm),
     * dWm = dzm h2^T, then dh2 = Wm^T dzm */
    for (int i = 0; i < H; ++i) {
      double s = 0.0;
      for (int c = 0; c < C; ++c) s += md->w3[(int64_t)c * H + i] * dz3[c];
      dhm[i] = s;
      dzm[i] = dhm[i] * act_df(md->act, b->zm[i]);
    }
    for (int o = 0; o < H; ++o) {
      g->bm[o] += dzm[o];
      for (int i = 0; i < H; ++i) g->wm[(int64_t)o * H + i] += dzm[o] * b->h2[i];
    }
    for (int i = 0; i < H; ++i) {
      double s = 0.0;
      for (int o = 0; o < H; ++o) s += md->wm[(int64_t)o * H + i] * dzm[o];
      dh2[i] = s;
      dz2[i] = dh2[i] * act_df(md->act, b->z2[i]);
    }
  } else {
    for (int i = 0; i < H; ++i) {
      double s = 0.0;
      for (int c = 0; c < C; ++c) s += md->w3[(int64_t)c * H + i] * dz3[c];
      dh2[i] = s;
      dz2[i] = dh2[i] * act_df(md->act, b->z2[i]);
    }
  }
  for (int o = 0; o < H; ++o) {
    g->b2[o] += dz2[o];
    for (int i = 0; i < H; ++i) g->w2[(int64_t)o * H + i] += dz2[o] * b->h1[i];
  }
  for (int i = 0; i < H; ++i) {
    double s = 0.0;
    for (int o = 0; o < H; ++o) s += md->w2[(int64_t)o * H + i] * dz2[o];
    dh1[i] = s;
    dz1[i] = dh1[i] * act_df(md->act, b->z1[i]);
  }
  for (int o = 0; o < H; ++o) {
    g->b1[o] += dz1[o];
    for (int i = 0; i < K; ++i) g->w1[(int64_t)o * K + i] += dz1[o] * b->x[i];
  }
  for (int i = 0; i < K; ++i) {
    double s = 0.0;
    for (int o = 0; o < H; ++o) s += md->w1[(int64_t)o * K + i] * dz1[o];
    dx[i] = s;
  }
  if (drow)
    for (int i = 0; i < K; ++i) drow[i] = dx[i];
  /* scatter the feature part of dx back through the taps: bilinear weights,
   * or (learned interpolation of G0) each tap's own slots with weight 1 */
  int j = or_level_of_mip(m, md->levels);
  int wm = mip_w(md, m), hm = mip_h(md, m);
  for (int k = 0; k < 2; ++k) {
    int gw = k ? md->g1w[j] : md->g0w[j], gh = k ? md->g1h[j] : md->g0h[j];
    int c = k ? md->c1 : md->c0, base = k ? g0_width(md) : 0;
    double* gg = k ? g->grid1[j] : g->grid0[j];
    int64_t cell[4]; double wt[4];
    bilinear_taps(x, y, wm, hm, gw, gh, cell, wt);
    if (k == 0 && md->interp0) {
      for (int t = 0; t < 4; ++t)
        for (int ch = 0; ch < c; ++ch) gg[cell[t] * c + ch] += dx[t * c + ch];
      continue;
    }
    for (int t = 0; t < 4; ++t)
      for (int ch = 0; ch < c; ++ch) gg[cell[t] * c + ch] += wt[t] * dx[base + ch];
  }
}

static int64_t grid_len(const or_model* md, int j, int k) {
  return k ? (int64_t)md->g1w[j] * md->g1h[j] * md->c1 : (int64_t)md->g0w[j] * md->g0h[j] * md->c0;
}

/* Private gradient buffers for one worker thread. */
static void grads_alloc(const or_model* md, or_grads* g) {
  int K = md->k_in, H = md->hidden, C = md->channels;
  memset(g, 0, sizeof(*g));
  for (int j = 0; j < md->levels; ++j) {
    g->grid0[j] = calloc((size_t)grid_len(md, j, 0), sizeof(double));
    g->grid1[j] = calloc((size_t)grid_len(md, j, 1), sizeof(double));
  }
  g->w1 = calloc((size_t)H * K, sizeof(double)); g->b1 = calloc((size_t)H, sizeof(double));
  g->w2 = calloc((size_t)H * H, sizeof(double)); g->b2 = calloc((size_t)H, sizeof(double));
  g->w3 = calloc((size_t)C * H, sizeof(double)); g->b3 = calloc((size_t)C, sizeof(double));
  g->wm = calloc((size_t)H * H, sizeof(double)); g->bm = calloc((size_t)H, sizeof(double));
}
static void grads_free(const or_model* md, or_grads* g) {
  for (int j = 0; j < md->levels; ++j) { free(g->grid0[j]); free(g->grid1[j]); }
  free(g->w1); free(g->b1); free(g->w2); free(g->b2); free(g->w3); free(g->b3);
  free(g->wm); free(g->bm);
}
static void add_into(double* dst, const double* src, int64_t n) {
  if (!dst) return;
  for (int64_t i = 0; i < n; ++i) dst[i] += src[i];
}
static void grads_reduce(const or_model* md, const or_grads* dst, const or_grads* src) {
  int K = md->k_in, H = md->hidden, C = md->channels;
  for (int j = 0; j < md->levels; ++j) {
    add_into(dst->grid0[j], src->grid0[j], grid_len(md, j, 0));
    add_into(dst->grid1[j], src->grid1[j], grid_len(md, j, 1));
  }
  add_into(dst->w1, src->w1, (int64_t)H * K); add_into(dst->b1, src->b1, H);
  add_into(dst->w2, src->w2, (int64_t)H * H); add_into(dst->b2, src->b2, H);
  add_into(dst->w3, src->w3, (int64_t)C * H); add_into(dst->b3, src->b3, C);
  add_into(dst->wm, src->wm, (int64_t)H * H); add_into(dst->bm, src->bm, H);
}

static void backward_job(job* jb, int64_t lo, int64_t hi) {
  mlp_buf b;
  mlp_alloc(jb->md, &b);
  int C = jb->md->channels;
  for (int64_t i = lo; i < hi; ++i)
    backward_one(jb->md, jb->xym[3 * i], jb->xym[3 * i + 1], jb->xym[3 * i + 2],
                 jb->dout + i * C, jb->nz, &b, &jb->g,
                 jb->rows ? jb->rows + i * jb->md->k_in : NULL);
  mlp_free(&b);
}

void or_backward_xym(const or_model* md, int64_t n, const int32_t* xym, const double* dout,
                     const or_noise* nz, const or_grads* g, int nthreads) {
  nthreads = clamp_threads(nthreads, n);
  job* jobs = calloc((size_t)nthreads, sizeof(job));
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].fn = backward_job; jobs[t].md = md; jobs[t].xym = xym; jobs[t].dout = dout;
    jobs[t].nz = nz; jobs[t].rows = g->rows;
    grads_alloc(md, &jobs[t].g);
  }
  run_jobs(jobs, nthreads, n);
  for (int t = 0; t < nthreads; ++t) { grads_reduce(md, g, &jobs[t].g); grads_free(md, &jobs[t].g); }
  free(jobs);
}

/* L2 loss (Sec. 4.5) over a batch: L = 1/(n*c) * sum (y - t)^2 (reading:
 * the mean over every decoded value), and its gradient through the decode:
 * dL/dy = 2 (y - t) / (n*c), then the reverse mode above.  Returns L. */
double or_loss_grad_xym(const or_model* md, int64_t n, const int32_t* xym,
                        const double* target, const or_noise* nz, const or_grads* g,
                        int nthreads) {
  int C = md->channels;
  double* y = calloc((size_t)(n * C), sizeof(double));
  double* dy = calloc((size_t)(n * C), sizeof(double));
  or_decode_xym(md, n, xym, nz, y, nthreads);
  double sum = 0.0, inv = 1.0 / ((double)n * (double)C);
  for (int64_t i = 0; i < n * C; ++i) {
    double e = y[i] - target[i];
    sum += e * e;
    dy[i] = 2.0 * e * inv;
  }
  or_backward_xym(md, n, xym, dy, nz, g, nthreads);
  free(y);
  free(dy);
  return sum * inv;
}

/* ------------------------------------------------------------------------ */
/* Optimiser (Sec. 5.1)                                                      */
/* ------------------------------------------------------------------------ */

/* Cosine annealing from lr0 at step 0 to 0 at step `total` (Sec. 5.1). */
double or_cosine_lr(double lr0, int64_t t, int64_t total) {
  const double pi = 3.14159265358979323846;
  return lr0 * 0.5 * (1.0 + cos(pi * (double)t / (double)total));
}

/* One Adam step (Kingma & Ba, with bias correction) at 0-based step t with
 * learning rate lr; then, for latent grids, clamp to the quantisation range
 * [lo, hi] after the update (Sec. 4.2). */
void or_adam(double* p, double* m, double* v, const double* g, int64_t n, double lr,
             int64_t t, double beta1, double beta2, double eps, int clamp, double lo,
             double hi) {
  double c1 = 1.0 - pow(beta1, (double)(t + 1));
  double c2 = 1.0 - pow(beta2, (double)(t + 1));
  for (int64_t i = 0; i < n; ++i) {
    m[i] = beta1 * m[i] + (1.0 - beta1) * g[i];
    v[i] = beta2 * v[i] + (1.0 - beta2) * g[i] * g[i];
    double mh = m[i] / c1, vh = v[i] / c2;
    p[i] -= lr * mh / (sqrt(vh) + eps);
    if (clamp) {
      if (p[i] < lo) p[i] = lo;
      if (p[i] > hi) p[i] = hi;
    }
  }
}
