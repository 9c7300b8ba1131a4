// C-ABI entry points of libntc.so (declared in include/ntc.h): argument
// validation, error reporting and dispatch to the kernels.
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <memory>
#include <vector>
#include <stdarg.h>
#include <stdlib.h>
#include <stdio.h>
#include <string.h>

#include "ntc_device.cuh"
#include "ntc_internal.h"

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

int cuda_status(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return NTC_OK;
  if (e == cudaErrorNotSupported) return fail(NTC_ERR_UNSUPPORTED, "%s: not supported", what);
  return fail(NTC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
bool aligned(const void* p) { return ((uintptr_t)p & 15u) == 0; }
int log2i(int v) {
  int r = 0;
  while ((1 << r) < v) ++r;
  return r;
}

#define CHECK_PTR(p, name)                                                        \
  do {                                                                            \
    if (!(p)) return fail(NTC_ERR_ARG, "%s is NULL", name);                       \
    if (!aligned(p)) return fail(NTC_ERR_ALIGN, "%s is not 16-byte aligned", name); \
  } while (0)

// Shape and pointer rules shared by every call that takes a material.
int check_material(const ntc_material* m, bool need_f32_grids, bool vq_training = false) {
  if (!m) return fail(NTC_ERR_ARG, "material is NULL");
  if (!pow2(m->width) || !pow2(m->height) || m->width > 32768 || m->height > 32768)
    return fail(NTC_ERR_SHAPE, "texture %dx%d: sides must be powers of two <= 32768", m->width,
                m->height);
  const int mips = log2i(m->width > m->height ? m->width : m->height) + 1;
  if (m->mips != mips) return fail(NTC_ERR_SHAPE, "mips = %d, expected %d", m->mips, mips);
  if (m->channels < 1 || m->channels > NTC_MAX_CHANNELS)
    return fail(NTC_ERR_SHAPE, "channels = %d outside 1..%d", m->channels, NTC_MAX_CHANNELS);
  if (m->levels < 1 || m->levels > NTC_MAX_LEVELS)
    return fail(NTC_ERR_SHAPE, "levels = %d outside 1..%d", m->levels, NTC_MAX_LEVELS);
  if (m->c0 < 1 || m->c1 < 1 || m->c0 > ntc::kMaxGridCh || m->c1 > ntc::kMaxGridCh)
    return fail(NTC_ERR_SHAPE, "c0 = %d, c1 = %d outside 1..%d", m->c0, m->c1, ntc::kMaxGridCh);
  for (int b : {m->bits0, m->bits1})
    if (b != 1 && b != 2 && b != 4 && b != 8) return fail(NTC_ERR_ARG, "bits %d not in {1,2,4,8}", b);
  if (m->encoding == NTC_GRID_PACKED &&
      (m->c1 * m->bits1 > 128 || (m->vq_books == 0 && m->c0 * m->bits0 > 128)))
    return fail(NTC_ERR_SHAPE, "packed cells hold at most 128 bits (c0 x bits0 = %d, c1 x bits1 = %d)",
                m->c0 * m->bits0, m->c1 * m->bits1);
  if (!(m->q0 > 0.f) || !(m->q1 > 0.f)) return fail(NTC_ERR_ARG, "bin widths must be positive");
  if (m->encoding != NTC_GRID_PACKED && m->encoding != NTC_GRID_F32)
    return fail(NTC_ERR_ARG, "encoding %d", m->encoding);
  if (need_f32_grids && m->encoding != NTC_GRID_F32)
    return fail(NTC_ERR_ARG, "this call needs NTC_GRID_F32 grids");
  if (m->hidden != NTC_HIDDEN) return fail(NTC_ERR_UNSUPPORTED, "hidden = %d (only %d)", m->hidden, NTC_HIDDEN);
  if (m->precision < NTC_PREC_F32 || m->precision > NTC_PREC_F8)
    return fail(NTC_ERR_ARG, "precision %d", m->precision);
  const int kmul = m->precision == NTC_PREC_F8 ? 32 : 16;
  if (m->interp0 != NTC_INTERP_BILINEAR && m->interp0 != NTC_INTERP_LEARNED)
    return fail(NTC_ERR_ARG, "interp0 %d", m->interp0);
  if (m->interp0 == NTC_INTERP_LEARNED && m->precision == NTC_PREC_F8)
    return fail(NTC_ERR_UNSUPPORTED, "learned interpolation: FP32 or FP16 weights");
  const int used = (m->interp0 == NTC_INTERP_LEARNED ? 4 * m->c0 : m->c0) + m->c1 + 13;
  if (m->k_in % kmul != 0 || m->k_in < used || m->k_in > NTC_MAX_K)
    return fail(NTC_ERR_SHAPE, "k_in = %d: need a multiple of %d in [%d, %d]", m->k_in, kmul, used,
                NTC_MAX_K);
  if (m->act != NTC_ACT_RELU && m->act != NTC_ACT_HARDGELU) return fail(NTC_ERR_ARG, "act %d", m->act);
  if (m->out_act != NTC_OUT_SIGMOID && m->out_act != NTC_OUT_IDENTITY)
    return fail(NTC_ERR_ARG, "out_act %d", m->out_act);
  for (int j = 0; j < m->levels; ++j) {
    const ntc_level& L = m->lv[j];
    if (L.g0_w < 1 || L.g0_h < 1 || L.g1_w < 1 || L.g1_h < 1 || L.g0_w > 32768 || L.g0_h > 32768 ||
        L.g1_w > 32768 || L.g1_h > 32768)
      return fail(NTC_ERR_SHAPE, "level %d grid sizes must be in 1..32768", j);
    if ((int64_t)L.g0_w * L.g0_h * (m->encoding == NTC_GRID_F32 ? m->c0 : 1) >= (1LL << 31) ||
        (int64_t)L.g1_w * L.g1_h * (m->encoding == NTC_GRID_F32 ? m->c1 : 1) >= (1LL << 31))
      return fail(NTC_ERR_SHAPE, "level %d grid too large", j);
    CHECK_PTR(L.grid0, "grid0");
    CHECK_PTR(L.grid1, "grid1");
  }
  for (int l = 0; l < 3; ++l) {
    CHECK_PTR(m->w[l], "weight");
    CHECK_PTR(m->b[l], "bias");
  }
  if (m->precision == NTC_PREC_F8) CHECK_PTR(m->scale, "scale");
  if (m->hidden_layers != 0 && m->hidden_layers != 2 && m->hidden_layers != 3)
    return fail(NTC_ERR_ARG, "hidden_layers = %d (2 or 3)", m->hidden_layers);
  if (m->hidden_layers == 3) {
    CHECK_PTR(m->w_h3, "w_h3");
    CHECK_PTR(m->b_h3, "b_h3");
    if (m->precision == NTC_PREC_F8)
      return fail(NTC_ERR_UNSUPPORTED, "three hidden layers: FP32 or FP16 weights");
  }
  if (m->vq_books < 0 || m->vq_books > 4)
    return fail(NTC_ERR_ARG, "vq_books = %d outside 0..4", m->vq_books);
  if (m->vq_books > 0) {
    CHECK_PTR(m->codebook0, "codebook0");
    if (m->precision == NTC_PREC_F8)
      return fail(NTC_ERR_UNSUPPORTED, "vector-quantised G0: FP32 or FP16 weights");
    if (vq_training) {
      if (m->encoding != NTC_GRID_F32)
        return fail(NTC_ERR_ARG, "vector-quantised G0 training: F32 latents");
    } else if (need_f32_grids || m->encoding != NTC_GRID_PACKED) {
      return fail(NTC_ERR_UNSUPPORTED,
                  "vector-quantised G0: decode packed indices without noise (export a trainer's "
                  "material first)");
    }
  }
  return NTC_OK;
}

std::atomic<int> g_decode_nwg{0};  // tensor-core decode warpgroups per CTA (0 = default)

// Tuning cache: the autotuners' choices keyed by what decides them -- the
// kind of launch, the material's shape and precision, the filter, the SM
// count and the size of the call (log2 bucket).  One line of text per
// entry, "<key> <value>", for export and import.
std::mutex g_tune_mu;
std::map<std::string, int> g_tune;

int log2_bucket(int64_t n) {
  int b = 0;
  while (b < 62 && ((int64_t)1 << (b + 1)) <= n) ++b;
  return b;
}

std::string tune_key(const char* kind, const ntc_material& m, int filter, int out_dtype,
                     int64_t n) {
  char buf[320];
  snprintf(buf, sizeof(buf),
           "%s:prec=%d:c=%d:c0=%d:c1=%d:b0=%d:b1=%d:k=%d:act=%d:out=%d:interp=%d:hl=%d:vq=%d:"
           "taps=%d:filter=%d:dtype=%d:sms=%d:n=2^%d",
           kind, m.precision, m.channels, m.c0, m.c1, m.bits0, m.bits1, m.k_in, m.act, m.out_act,
           m.interp0, m.hidden_layers == 3 ? 3 : 2, m.vq_books, ntc::fast_layout_ok(m) ? 1 : 0,
           filter, out_dtype, ntc::sm_count(), log2_bucket(n));
  return std::string(buf);
}

int tune_lookup(const std::string& key) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tune.find(key);
  return it == g_tune.end() ? 0 : it->second;
}

void tune_store(const std::string& key, int value) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune[key] = value;
}

// Helper streams and events of ntc_decode_host, created once per device and
// used under g_pipe_mu (one enqueue sequence at a time).
struct HostPipe {
  bool ready = false;
  cudaStream_t up = nullptr, down = nullptr;
  cudaEvent_t fork, join_up, join_down, uploaded[2], decoded[2], downloaded[2];
};
std::mutex g_pipe_mu;
HostPipe g_pipes[64];

bool out_dtype_ok(int32_t d) {
  return d == NTC_DTYPE_F32 || d == NTC_DTYPE_F16 || d == NTC_DTYPE_U8;
}
size_t out_elem_bytes(int32_t d) { return d == NTC_DTYPE_U8 ? 1 : (d == NTC_DTYPE_F16 ? 2 : 4); }

bool use_simt(const ntc_material* m, int flags) {
  return (flags & NTC_FLAG_SIMT) || m->precision == NTC_PREC_F32;
}

// The decode of a validated call.
int decode_impl(const ntc_material* m, const float* uvl, int64_t n, void* out, int32_t out_dtype,
                int32_t filter, int32_t flags, uint64_t noise_seed, int64_t noise_step,
                cudaStream_t s) {
  if (use_simt(m, flags) || (flags & NTC_FLAG_NOISE))
    return cuda_status(ntc::launch_decode_simt(*m, uvl, n, out, out_dtype, filter,
                                               (flags & NTC_FLAG_NOISE) != 0, noise_seed,
                                               noise_step, s),
                       "decode (FP32 CUDA cores)");
  int nwg = g_decode_nwg.load();  // ntc_set_decode_warpgroups, else the autotuner's choice
  if (nwg == 0) nwg = tune_lookup(tune_key("decode", *m, filter, out_dtype, n));
  return cuda_status(ntc::launch_decode_tc(*m, uvl, n, out, out_dtype, filter,
                                           ntc::jitter_key(noise_seed, noise_step), s, nwg),
                     "decode (tcgen05)");
}

// This device's helper streams and events (created on first use; caller
// holds g_pipe_mu).
int host_pipe(HostPipe** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
    return cuda_status(cudaErrorInvalidDevice, "decode_host device");
  HostPipe& P = g_pipes[dev];
  if (!P.ready) {
    cudaError_t e = cudaStreamCreateWithFlags(&P.up, cudaStreamNonBlocking);
    if (!e) e = cudaStreamCreateWithFlags(&P.down, cudaStreamNonBlocking);
    cudaEvent_t* evs[9] = {&P.fork, &P.join_up, &P.join_down, &P.uploaded[0], &P.uploaded[1],
                           &P.decoded[0], &P.decoded[1], &P.downloaded[0], &P.downloaded[1]};
    for (cudaEvent_t* ev : evs)
      if (!e) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e) return cuda_status(e, "decode_host streams");
    P.ready = true;
  }
  *out = &P;
  return NTC_OK;
}

}  // namespace

namespace ntc {
int report_error(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}
}  // namespace ntc

extern "C" {

const char* ntc_version(void) { return "ntc-gb300 0.1 (sm_103a)"; }

const char* ntc_last_error(void) { return g_err; }

int ntc_device_status(int32_t reset) {
  const int v = ntc::read_status_word(reset);
  if (v < 0) return fail(NTC_ERR_CUDA, "device status: %s", cudaGetErrorString(cudaGetLastError()));
  if (v == NTC_ERR_TIMEOUT) return fail(NTC_ERR_TIMEOUT, "a device-side wait timed out");
  return v == 0 ? NTC_OK : fail(v, "device status %d", v);
}

int ntc_selftest_wait(int32_t limit, void* stream) {
  if (limit < 1 || limit > (1 << 20)) return fail(NTC_ERR_ARG, "limit %d outside 1..2^20", limit);
  return cuda_status(ntc::launch_selftest_wait((uint32_t)limit, static_cast<cudaStream_t>(stream)),
                     "selftest_wait");
}

int32_t ntc_cell_bytes(int32_t c, int32_t bits) {
  if (c < 1 || c > 64 || (bits != 1 && bits != 2 && bits != 4 && bits != 8) || c * bits > 128)
    return 0;
  return ntc::cell_bytes(c, bits);
}

int32_t ntc_pyramid(int32_t width, int32_t height, int32_t* g0_w, int32_t* g0_h, int32_t* g1_w,
                    int32_t* g1_h) {
  if (!pow2(width) || !pow2(height) || !g0_w || !g0_h || !g1_w || !g1_h) return 0;
  int levels = 0;
  for (int j = 0; j < NTC_MAX_LEVELS; ++j) {
    const int sh = 2 * j + 2;
    const int w0 = (width >> sh) > 0 ? (width >> sh) : 1;
    const int h0 = (height >> sh) > 0 ? (height >> sh) : 1;
    if (j > 0 && (w0 > h0 ? w0 : h0) < 4) break;
    g0_w[j] = w0;
    g0_h[j] = h0;
    g1_w[j] = (w0 >> 1) > 0 ? (w0 >> 1) : 1;
    g1_h[j] = (h0 >> 1) > 0 ? (h0 >> 1) : 1;
    ++levels;
  }
  return levels;
}

int ntc_decode(const ntc_material* m, const float* uvl, int64_t n, void* out, int32_t out_dtype,
               int32_t filter, int32_t flags, uint64_t noise_seed, int64_t noise_step,
               void* stream) {
  int st = check_material(m, (flags & NTC_FLAG_NOISE) != 0);
  if (st) return st;
  if (n < 0) return fail(NTC_ERR_ARG, "n < 0");
  if (!out_dtype_ok(out_dtype)) return fail(NTC_ERR_ARG, "out_dtype %d", out_dtype);
  if (filter != NTC_FILTER_NEAREST && filter != NTC_FILTER_TRILINEAR &&
      filter != NTC_FILTER_STOCHASTIC)
    return fail(NTC_ERR_ARG, "filter");
  if ((flags & NTC_FLAG_NOISE) && filter != NTC_FILTER_NEAREST)
    return fail(NTC_ERR_ARG, "noise needs nearest filtering");
  if (n == 0) return NTC_OK;
  CHECK_PTR(uvl, "uvl");
  CHECK_PTR(out, "out");
  return decode_impl(m, uvl, n, out, out_dtype, filter, flags, noise_seed, noise_step,
                     static_cast<cudaStream_t>(stream));
}

size_t ntc_decode_host_workspace_bytes(int32_t channels, int32_t out_dtype, int64_t chunk) {
  if (channels < 1 || channels > NTC_MAX_CHANNELS || chunk < 0 || !out_dtype_ok(out_dtype)) return 0;
  const size_t eb = out_elem_bytes(out_dtype);
  return 2 * (size_t)chunk * (12 + (size_t)channels * eb);
}

int ntc_decode_host(const ntc_material* m, const float* uvl_host, int64_t n, void* out_host,
                    int32_t out_dtype, int32_t filter, int32_t flags, uint64_t noise_seed,
                    int64_t noise_step, void* workspace, size_t workspace_bytes, void* stream) {
  int st = check_material(m, (flags & NTC_FLAG_NOISE) != 0);
  if (st) return st;
  if (n < 0) return fail(NTC_ERR_ARG, "n < 0");
  if (!out_dtype_ok(out_dtype)) return fail(NTC_ERR_ARG, "out_dtype %d", out_dtype);
  if (filter == NTC_FILTER_STOCHASTIC)
    return fail(NTC_ERR_UNSUPPORTED, "decode_host: nearest or trilinear filtering");
  if (filter != NTC_FILTER_NEAREST && filter != NTC_FILTER_TRILINEAR)
    return fail(NTC_ERR_ARG, "filter");
  if ((flags & NTC_FLAG_NOISE) && filter != NTC_FILTER_NEAREST)
    return fail(NTC_ERR_ARG, "noise needs nearest filtering");
  if (n == 0) return NTC_OK;
  if (!uvl_host || !out_host) return fail(NTC_ERR_ARG, "host buffer is NULL");
  CHECK_PTR(workspace, "workspace");
  const size_t eb = out_elem_bytes(out_dtype), C = (size_t)m->channels;
  const size_t per = 12 + C * eb;
  const int64_t chunk = (int64_t)(workspace_bytes / (2 * per)) / 128 * 128;
  if (chunk < 128) return fail(NTC_ERR_ARG, "decode_host: workspace below two 128-query chunks");
  uint8_t* ws = static_cast<uint8_t*>(workspace);
  // slots: inputs [2][chunk][3] floats, then outputs [2][chunk][C] (16-byte aligned:
  // chunk is a multiple of 128)
  float* in_slot[2] = {reinterpret_cast<float*>(ws), reinterpret_cast<float*>(ws + chunk * 12)};
  uint8_t* out_slot[2] = {ws + 2 * chunk * 12, ws + 2 * chunk * 12 + chunk * C * eb};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lock(g_pipe_mu);
  HostPipe* P = nullptr;
  if (int e = host_pipe(&P)) return e;
  // fork: the helper streams start after the work already on `stream`
  {
    cudaError_t e = cudaEventRecord(P->fork, s);
    if (!e) e = cudaStreamWaitEvent(P->up, P->fork, 0);
    if (!e) e = cudaStreamWaitEvent(P->down, P->fork, 0);
    if (e) return cuda_status(e, "decode_host fork");
  }
  for (int64_t i = 0; i * chunk < n; ++i) {
    const int sl = (int)(i & 1);
    const int64_t off = i * chunk, cnt = n - off < chunk ? n - off : chunk;
    cudaError_t e = cudaSuccess;
    // chunk i up: its slot is free once the decode of chunk i-2 has read it
    if (i >= 2) e = cudaStreamWaitEvent(P->up, P->decoded[sl], 0);
    if (!e) e = cudaMemcpyAsync(in_slot[sl], uvl_host + 3 * off, (size_t)cnt * 12,
                                cudaMemcpyHostToDevice, P->up);
    if (!e) e = cudaEventRecord(P->uploaded[sl], P->up);
    // decode on the caller's stream once the inputs are there and the output
    // slot has been copied back (chunk i-2)
    if (!e) e = cudaStreamWaitEvent(s, P->uploaded[sl], 0);
    if (!e && i >= 2) e = cudaStreamWaitEvent(s, P->downloaded[sl], 0);
    if (e) return cuda_status(e, "decode_host enqueue");
    st = decode_impl(m, in_slot[sl], cnt, out_slot[sl], out_dtype, filter, flags, noise_seed,
                     noise_step, s);
    if (st) return st;
    e = cudaEventRecord(P->decoded[sl], s);
    // chunk i down
    if (!e) e = cudaStreamWaitEvent(P->down, P->decoded[sl], 0);
    if (!e) e = cudaMemcpyAsync(static_cast<uint8_t*>(out_host) + (size_t)off * C * eb,
                                out_slot[sl], (size_t)cnt * C * eb, cudaMemcpyDeviceToHost, P->down);
    if (!e) e = cudaEventRecord(P->downloaded[sl], P->down);
    if (e) return cuda_status(e, "decode_host enqueue");
  }
  // join: `stream` continues after the last copies of both helpers
  cudaError_t e = cudaEventRecord(P->join_up, P->up);
  if (!e) e = cudaEventRecord(P->join_down, P->down);
  if (!e) e = cudaStreamWaitEvent(s, P->join_up, 0);
  if (!e) e = cudaStreamWaitEvent(s, P->join_down, 0);
  return cuda_status(e, "decode_host join");
}

int ntc_set_decode_warpgroups(int32_t nwg) {
  if (nwg != 0 && (nwg < 2 || nwg > 5)) return fail(NTC_ERR_ARG, "warpgroups %d", nwg);
  g_decode_nwg.store(nwg);
  return NTC_OK;
}

int ntc_f8_quantize_weights(const float* w, int32_t rows, int32_t cols, int32_t cols_out,
                            uint8_t* w8_out, float* scale_out, void* stream) {
  if (rows < 1 || cols < 1 || cols_out < cols || cols_out > NTC_MAX_K || rows > NTC_MAX_K)
    return fail(NTC_ERR_ARG, "f8 weights: rows %d, cols %d, cols_out %d", rows, cols, cols_out);
  if (!w || !w8_out || !scale_out) return fail(NTC_ERR_ARG, "f8 weights: NULL pointer");
  if (((uintptr_t)w & 3u) || ((uintptr_t)scale_out & 3u))
    return fail(NTC_ERR_ALIGN, "f8 weights: float arrays must be 4-byte aligned");
  return cuda_status(ntc::launch_f8_weights(w, rows, cols, cols_out, w8_out, scale_out,
                                            static_cast<cudaStream_t>(stream)),
                     "f8 weights");
}

int ntc_f8_activation_scales(const ntc_material* m, const float* uvl, int64_t n,
                             float* act_scale_out, void* stream) {
  int st = check_material(m, false);
  if (st) return st;
  if (m->precision == NTC_PREC_F8)
    return fail(NTC_ERR_ARG, "f8 activation scales: calibrate the FP32 or FP16 model");
  if (m->hidden_layers == 3)
    return fail(NTC_ERR_UNSUPPORTED, "f8 activation scales: the FP8 form has two hidden layers");
  if (m->vq_books > 0) return fail(NTC_ERR_UNSUPPORTED, "f8 activation scales: scalar grids");
  if (n < 0) return fail(NTC_ERR_ARG, "n < 0");
  if (n > 0) CHECK_PTR(uvl, "uvl");
  if (!act_scale_out || ((uintptr_t)act_scale_out & 3u))
    return fail(NTC_ERR_ARG, "act_scale_out is NULL or not 4-byte aligned");
  return cuda_status(ntc::launch_f8_calibrate(*m, uvl, n, reinterpret_cast<uint32_t*>(act_scale_out),
                                              act_scale_out, static_cast<cudaStream_t>(stream)),
                     "f8 activation scales");
}

int ntc_probe_fma_tflops(float* tflops_out, void* stream) {
  if (!tflops_out) return fail(NTC_ERR_ARG, "tflops_out is NULL");
  return cuda_status(ntc::probe_fma_tflops(tflops_out, static_cast<cudaStream_t>(stream)),
                     "FMA probe");
}

int ntc_autotune_decode(const ntc_material* m, const float* uvl, int64_t n, void* out,
                        int32_t out_dtype, int32_t filter, int32_t* best, float* ms_out,
                        void* stream) {
  if (!best) return fail(NTC_ERR_ARG, "best is NULL");
  int st = check_material(m, false);
  if (st) return st;
  if (m->precision == NTC_PREC_F32) return fail(NTC_ERR_ARG, "the FP32 form has no launch shapes");
  if (n <= 0) return fail(NTC_ERR_ARG, "n must be positive");
  if (!out_dtype_ok(out_dtype)) return fail(NTC_ERR_ARG, "out_dtype %d", out_dtype);
  if (filter != NTC_FILTER_NEAREST && filter != NTC_FILTER_TRILINEAR &&
      filter != NTC_FILTER_STOCHASTIC)
    return fail(NTC_ERR_ARG, "filter");
  CHECK_PTR(uvl, "uvl");
  CHECK_PTR(out, "out");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int shapes[4] = {2, 3, 4, 5};
  const uint64_t jk = ntc::jitter_key(0, 0);  // stochastic filtering: frame 0 of seed 0
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return cuda_status(cudaGetLastError(), "autotune events");
  float best_ms = 1e30f;
  int best_nwg = 0, rc = NTC_OK;
  for (int i = 0; i < 4 && rc == NTC_OK; ++i) {
    cudaError_t e = ntc::launch_decode_tc(*m, uvl, n, out, out_dtype, filter, jk, s, shapes[i]);
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    for (int r = 0; r < 3 && e == cudaSuccess; ++r)
      e = ntc::launch_decode_tc(*m, uvl, n, out, out_dtype, filter, jk, s, shapes[i]);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) rc = cuda_status(e, "autotune");
    if (ms_out) ms_out[i] = ms / 3.f;
    if (ms < best_ms) { best_ms = ms; best_nwg = shapes[i]; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != NTC_OK) return rc;
  tune_store(tune_key("decode", *m, filter, out_dtype, n), best_nwg);
  *best = best_nwg;
  return NTC_OK;
}



int ntc_backward(const ntc_material* m, const float* uvl, int64_t n, const float* dout,
                 const ntc_grads* g, int32_t flags, uint64_t noise_seed, int64_t noise_step,
                 void* stream) {
  int st = check_material(m, true);
  if (st) return st;
  // FP16 weights: the tensor-core adjoint (the fused training kernel fed dout
  // instead of the loss); otherwise the FP32 CUDA-core adjoint
  const bool tc = m->precision == NTC_PREC_F16 && !(flags & NTC_FLAG_SIMT) &&
                  m->vq_books == 0 && ntc::train_tc_supported(*m);
  if (!tc && m->hidden_layers == 3)
    return fail(NTC_ERR_UNSUPPORTED, "ntc_backward: two hidden layers on the FP32 adjoint "
                                     "(three run on the FP16 tensor-core adjoint)");
  if (n < 0) return fail(NTC_ERR_ARG, "n < 0");
  if (!g) return fail(NTC_ERR_ARG, "grads is NULL");
  if (n == 0) return NTC_OK;
  CHECK_PTR(uvl, "uvl");
  CHECK_PTR(dout, "dout");
  ntc::BwdArgs a{};
  a.uvl = uvl;
  a.dout = dout;
  a.n = n;
  a.g = *g;
  for (int j = 0; j < m->levels; ++j) {
    if (a.g.grid0[j] && !aligned(a.g.grid0[j])) return fail(NTC_ERR_ALIGN, "grad grid0");
    if (a.g.grid1[j] && !aligned(a.g.grid1[j])) return fail(NTC_ERR_ALIGN, "grad grid1");
  }
  for (int j = m->levels; j < NTC_MAX_LEVELS; ++j) a.g.grid0[j] = a.g.grid1[j] = nullptr;
  a.grad_scale = 1.f;
  a.noise = (flags & NTC_FLAG_NOISE) != 0;
  a.noise_seed = noise_seed;
  a.noise_step = noise_step;
  a.train = 0;
  a.grids = 1;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (tc) return cuda_status(ntc::launch_train_tc(*m, a, s), "backward (FP16 tensor cores)");
  // FP32 / FP8 weights (widened on load) or NTC_FLAG_SIMT
  if (m->k_in > 64) return fail(NTC_ERR_UNSUPPORTED, "FP32 backward supports k_in <= 64");
  return cuda_status(ntc::launch_backward_simt(*m, a, s), "backward (FP32 CUDA cores)");
}

// Everything one optimisation step launches, validated and built on the
// host without any CUDA call.
struct StepPlan {
  ntc::AdamArgs a;
  ntc::BwdArgs b;
  ntc::NoiseArgs na;
  ntc_material mt;   // the material as the fused step reads it
  bool noise_pass;   // dense noise pass into the trainer's noisy scratch
  bool vq, simt;
  int cb_seg;        // Adam segment of the codebooks (vector-quantised G0)
};

static int plan_train_step(const ntc_material* m, const ntc_trainer* tr, const ntc_target* t,
                           int64_t batch, uint64_t seed, const float* uvl_or_null,
                           float* loss_out, int32_t flags, StepPlan* plan) {
  StepPlan& sp = *plan;
  ntc::AdamArgs& a = sp.a;
  ntc::BwdArgs& b = sp.b;
  a = ntc::AdamArgs{};
  b = ntc::BwdArgs{};
  const bool vq = m && m->vq_books > 0;
  int st = check_material(m, true, vq);
  if (st) return st;
  if (!tr || !t) return fail(NTC_ERR_ARG, "trainer / target is NULL");
  if (vq) {
    CHECK_PTR(tr->noisy, "trainer noisy scratch (vector-quantised G0)");
    if (!tr->vq_idx) return fail(NTC_ERR_ARG, "trainer vq_idx is NULL");
    if (!(tr->vq_beta >= 0.f)) return fail(NTC_ERR_ARG, "vq_beta must be >= 0");
  }
  if (batch <= 0) return fail(NTC_ERR_ARG, "batch must be positive");
  if (m->precision == NTC_PREC_F8 && use_simt(m, flags))
    return fail(NTC_ERR_UNSUPPORTED, "FP8 training runs on the tensor cores (no NTC_FLAG_SIMT)");
  if (m->precision == NTC_PREC_F8 && !ntc::train_tc_supported(*m))
    return fail(NTC_ERR_UNSUPPORTED, "FP8 training: bilinear G0, two hidden layers, k_in a "
                                     "multiple of 32, scalar grids");
  if (use_simt(m, flags)) {
    if (m->k_in > 64) return fail(NTC_ERR_UNSUPPORTED, "FP32 training supports k_in <= 64");
    if (m->hidden_layers == 3)
      return fail(NTC_ERR_UNSUPPORTED, "FP32 training: two hidden layers (three train on FP16)");
  } else if (!ntc::train_tc_supported(*m)) {
    return fail(NTC_ERR_UNSUPPORTED,
                "tensor-core training: activation or feature layout not supported "
                "(use NTC_FLAG_SIMT)");
  }
  CHECK_PTR(tr->params, "params");
  CHECK_PTR(tr->adam_m, "adam_m");
  CHECK_PTR(tr->adam_v, "adam_v");
  CHECK_PTR(tr->grad, "grad");
  CHECK_PTR(tr->step, "step");
  CHECK_PTR(t->texels, "target texels");
  CHECK_PTR(loss_out, "loss_out");
  if (uvl_or_null && !aligned(uvl_or_null)) return fail(NTC_ERR_ALIGN, "uvl");
  if (tr->total_steps <= 0) return fail(NTC_ERR_ARG, "total_steps must be positive");
  for (int l = 0; l < 3; ++l) CHECK_PTR(tr->w_master[l], "w_master");
  if (m->precision == NTC_PREC_F32)
    for (int l = 0; l < 3; ++l)
      if (m->w[l] != tr->w_master[l]) return fail(NTC_ERR_ARG, "F32 weights must be the masters");

  // Segments of the parameter array: grids (group 0, clamped), MLP (group 1).
  const float* P = tr->params;
  auto offset_of = [&](const void* ptr, int64_t len, int64_t* off) -> bool {
    const float* f = static_cast<const float*>(ptr);
    if (f < P || f + len > P + tr->n_params) return false;
    *off = f - P;
    return true;
  };
  auto add_seg = [&](const void* ptr, int64_t len, int group, bool clamp, float lo, float hi,
                     __half* half_copy) -> bool {
    if (a.nseg >= ntc::kMaxSegs) return false;
    ntc::AdamSeg& sg = a.seg[a.nseg++];
    if (!offset_of(ptr, len, &sg.off)) return false;
    sg.len = len;
    sg.group = group;
    sg.clamp = clamp;
    sg.lo = lo;
    sg.hi = hi;
    sg.half_copy = half_copy;
    return true;
  };
  const int n0 = 1 << m->bits0, n1 = 1 << m->bits1;
  const float lo0 = -(float)(n0 - 1) / 2.f * m->q0, hi0 = (float)n0 / 2.f * m->q0;
  const float lo1 = -(float)(n1 - 1) / 2.f * m->q1, hi1 = (float)n1 / 2.f * m->q1;
  for (int j = 0; j < m->levels; ++j) {
    const ntc_level& L = m->lv[j];
    if (!add_seg(L.grid0, (int64_t)L.g0_w * L.g0_h * m->c0, 0, !vq, lo0, hi0, nullptr) ||
        !add_seg(L.grid1, (int64_t)L.g1_w * L.g1_h * m->c1, 0, true, lo1, hi1, nullptr))
      return fail(NTC_ERR_ARG, "grid %d is not inside params", j);
  }
  const int64_t wlen[3] = {(int64_t)NTC_HIDDEN * m->k_in, (int64_t)NTC_HIDDEN * NTC_HIDDEN,
                           (int64_t)m->channels * NTC_HIDDEN};
  const int64_t blen[3] = {NTC_HIDDEN, NTC_HIDDEN, m->channels};
  for (int l = 0; l < 3; ++l) {
    __half* hc = m->precision == NTC_PREC_F16 ? (__half*)m->w[l] : nullptr;
    if (!add_seg(tr->w_master[l], wlen[l], 1, false, 0, 0, hc) ||
        !add_seg(m->b[l], blen[l], 1, false, 0, 0, nullptr))
      return fail(NTC_ERR_ARG, "MLP tensor %d is not inside params", l);
  }
  const bool h3 = m->hidden_layers == 3;
  if (h3) {
    CHECK_PTR(tr->w_master_h3, "w_master_h3");
    if (m->precision == NTC_PREC_F32 && m->w_h3 != tr->w_master_h3)
      return fail(NTC_ERR_ARG, "F32 weights must be the masters");
    __half* hc = m->precision == NTC_PREC_F16 ? (__half*)m->w_h3 : nullptr;
    if (!add_seg(tr->w_master_h3, (int64_t)NTC_HIDDEN * NTC_HIDDEN, 1, false, 0, 0, hc) ||
        !add_seg(m->b_h3, NTC_HIDDEN, 1, false, 0, 0, nullptr))
      return fail(NTC_ERR_ARG, "third hidden layer is not inside params");
  }
  const int cb_seg = a.nseg;  // the codebooks of a vector-quantised G0 (lr_grid, unclamped)
  if (vq && !add_seg(m->codebook0, (int64_t)m->vq_books * 256 * m->c0, 0, false, 0, 0, nullptr))
    return fail(NTC_ERR_ARG, "codebooks are not inside params");
  const int64_t per_block = ntc::kAdamBlock * ntc::kAdamPerThread;
  a.block_start[0] = 0;
  for (int i = 0; i < a.nseg; ++i)
    a.block_start[i + 1] = a.block_start[i] + (a.seg[i].len + per_block - 1) / per_block;
  a.p = tr->params;
  a.m = tr->adam_m;
  a.v = tr->adam_v;
  a.g = tr->grad;
  a.step = tr->step;
  a.total = tr->total_steps;
  a.lr[0] = tr->lr_grid;
  a.lr[1] = tr->lr_mlp;
  a.beta1 = tr->beta1;
  a.beta2 = tr->beta2;
  a.eps = tr->eps;
  const bool freeze = (flags & NTC_FLAG_FREEZE_GRIDS) != 0;
  a.freeze_grids = freeze;

  // Fused forward + loss + backward into tr->grad.
  b.uvl = uvl_or_null;
  b.target = t->texels;
  for (int i = 0; i < NTC_MAX_MIPS; ++i) b.tgt_off[i] = t->offset[i];
  b.n = batch;
  float* G = tr->grad;
  for (int j = 0; j < m->levels; ++j) {
    b.g.grid0[j] = freeze ? nullptr : G + a.seg[2 * j].off;
    b.g.grid1[j] = freeze ? nullptr : G + a.seg[2 * j + 1].off;
  }
  for (int l = 0; l < 3; ++l) {
    b.g.w[l] = G + a.seg[2 * m->levels + 2 * l].off;
    b.g.b[l] = G + a.seg[2 * m->levels + 2 * l + 1].off;
  }
  if (h3) {
    b.g.w_h3 = G + a.seg[2 * m->levels + 6].off;
    b.g.b_h3 = G + a.seg[2 * m->levels + 7].off;
  }
  b.grad_scale = (float)(1.0 / ((double)batch * (double)m->channels));
  b.loss = loss_out;
  b.loss_scale = b.grad_scale;
  b.noise = !(freeze || (flags & NTC_FLAG_NO_NOISE));
  b.noise_seed = seed;
  b.sample_seed = seed;
  b.step_dev = tr->step;
  b.train = 1;
  b.grids = !freeze;
  b.crops = (flags & NTC_FLAG_CROPS) != 0;
  sp.vq = vq;
  sp.simt = use_simt(m, flags);
  b.pipelines = sp.simt ? 0 : tune_lookup(tune_key("train", *m, b.crops ? 1 : 0, 0, batch));
  sp.cb_seg = cb_seg;
  // With the noisy scratch: one dense noise pass, and the fused step reads
  // the noisy grids at the same offsets of the scratch.
  ntc_material& mt = sp.mt;
  mt = *m;
  sp.na = ntc::NoiseArgs{};
  sp.noise_pass = false;
  if (b.noise && tr->noisy) {
    CHECK_PTR(tr->noisy, "trainer noisy scratch");
    ntc::NoiseArgs& na = sp.na;
    na.src = tr->params;
    na.dst = tr->noisy;
    na.seed = seed;
    na.step = tr->step;
    na.block_start[0] = 0;
    for (int j = 0; j < m->levels; ++j)
      for (int k = 0; k < 2; ++k) {
        if (k == 0 && vq) continue;  // a vector-quantised G0 trains through q, noise-free
        const ntc::AdamSeg& sg = a.seg[2 * j + k];
        const int c = k ? m->c1 : m->c0;
        ntc::NoiseSeg& g = na.seg[na.nseg];
        g.off = sg.off;
        g.c = c;
        g.pairs = sg.len / c * ((c + 1) / 2);
        g.level = j;
        g.grid = k;
        g.q = k ? m->q1 : m->q0;
        na.block_start[na.nseg + 1] =
            na.block_start[na.nseg] + (g.pairs + ntc::kNoiseBlock - 1) / ntc::kNoiseBlock;
        ++na.nseg;
        (k ? mt.lv[j].grid1 : mt.lv[j].grid0) = tr->noisy + sg.off;
      }
    sp.noise_pass = true;
    b.noise = 0;
    // fold the next step's noise into this step's Adam (no VQ: its G0
    // scratch holds the quantised rows)
    if (tr->noisy_tag && !vq) {
      if (((uintptr_t)tr->noisy_tag & 7u) != 0) return fail(NTC_ERR_ALIGN, "noisy_tag");
      na.tag = tr->noisy_tag;
      a.fold = 1;
      a.noisy = tr->noisy;
      a.noise_seed = seed;
      a.noisy_tag = tr->noisy_tag;
      for (int j = 0; j < m->levels; ++j)
        for (int k = 0; k < 2; ++k) {
          ntc::AdamSeg& sg = a.seg[2 * j + k];
          sg.noise_c = k ? m->c1 : m->c0;
          sg.noise_level = j;
          sg.noise_grid = k;
          sg.noise_q = k ? m->q1 : m->q0;
        }
    }
  }
  return NTC_OK;
}

// Seed of the last step that folded the next step's noise into its Adam,
// per noisy tag (host-side guess of whether the copy will be current).
static std::mutex g_fold_mu;
static std::map<const int64_t*, uint64_t> g_fold_seed;
static bool fold_expected(const int64_t* tag, uint64_t seed) {
  std::lock_guard<std::mutex> lock(g_fold_mu);
  const auto it = g_fold_seed.find(tag);
  return it != g_fold_seed.end() && it->second == seed;
}
static void note_fold(const int64_t* tag, bool folded, uint64_t seed) {
  if (!tag) return;
  std::lock_guard<std::mutex> lock(g_fold_mu);
  if (folded) g_fold_seed[tag] = seed;
  else g_fold_seed.erase(tag);
}

// Launches a planned step on `s`.
static int launch_train_plan(const ntc_material* m, const ntc_trainer* tr, StepPlan& sp,
                             float* loss_out, int32_t flags, cudaStream_t s) {
  ntc::AdamArgs& a = sp.a;
  ntc::BwdArgs& b = sp.b;
  ntc_material& mt = sp.mt;
  const bool vq = sp.vq, freeze = (flags & NTC_FLAG_FREEZE_GRIDS) != 0;
  const int cb_seg = sp.cb_seg;
  float* G = tr->grad;
  cudaError_t e = cudaMemsetAsync(loss_out, 0, sizeof(float), s);
  if (e != cudaSuccess) return cuda_status(e, "train_step memset");
  if (m->precision == NTC_PREC_F8) {
    // this step's E4M3 weights and scales from the masters and the previous
    // step's layer-input maxima (R24)
    const float* wm[3] = {tr->w_master[0], tr->w_master[1], tr->w_master[2]};
    uint8_t* w8[3];
    for (int l = 0; l < 3; ++l) w8[l] = static_cast<uint8_t*>(const_cast<void*>(m->w[l]));
    e = ntc::launch_f8_train_prep(wm, w8, m->k_in, m->channels, const_cast<float*>(m->scale), s);
    if (e != cudaSuccess) return cuda_status(e, "train_step FP8 weights");
  }
  // With the noise folded into the previous step's Adam, the fused
  // tensor-core step checks the noisy copy's tag itself (bilinear G0, grids
  // of 4k <= 16 channels): no launch for the usual case of a current copy,
  // the noise per tap otherwise.
  // The check only pays when the copy is expected to be current: the
  // previous step on this trainer folded with the same seed (a process-wide
  // note per tag; the kernel still checks the tag, so a wrong guess costs
  // time, not correctness).  Otherwise the dense pass runs.
  const bool kernel_fold = sp.noise_pass && sp.na.tag && !sp.simt && !vq &&
                           m->interp0 == NTC_INTERP_BILINEAR && (m->c0 & 3) == 0 &&
                           m->c0 <= 16 && (m->c1 & 3) == 0 && m->c1 <= 16 &&
                           fold_expected(sp.na.tag, sp.na.seed);
  ntc::BwdArgs bk = sp.b;
  ntc_material mk = sp.mt;
  if (kernel_fold) {
    bk.noise = 1;
    bk.noisy_tag = sp.na.tag;
    for (int j = 0; j < m->levels; ++j) {
      bk.noisy0[j] = static_cast<const float*>(sp.mt.lv[j].grid0);
      bk.noisy1[j] = static_cast<const float*>(sp.mt.lv[j].grid1);
      mk.lv[j].grid0 = m->lv[j].grid0;
      mk.lv[j].grid1 = m->lv[j].grid1;
    }
  } else if (sp.noise_pass) {
    e = ntc::launch_noise_grids(sp.na, s);
    if (e != cudaSuccess) return cuda_status(e, "train_step noise pass");
  }
  if (vq) {
    // quantise every G0 level into the scratch (the fused step reads q), with
    // the codebook and commitment gradients of the step
    int64_t n_lat = 0;
    for (int j = 0; j < m->levels; ++j) n_lat += a.seg[2 * j].len;
    const float scale = (float)(2.0 / (double)n_lat);
    uint8_t* ip = tr->vq_idx;
    for (int j = 0; j < m->levels; ++j) {
      const ntc::AdamSeg& sg = a.seg[2 * j];
      const int64_t cells = sg.len / m->c0;
      e = ntc::launch_vq_step(tr->params + sg.off, cells, m->c0, m->codebook0, m->vq_books, ip,
                              tr->noisy + sg.off, freeze ? nullptr : G + sg.off,
                              freeze ? nullptr : G + a.seg[cb_seg].off, scale, tr->vq_beta, s);
      if (e != cudaSuccess) return cuda_status(e, "train_step vector quantisation");
      mt.lv[j].grid0 = tr->noisy + sg.off;
      ip += cells * m->vq_books;
    }
    mt.vq_books = 0;  // the fused step sees q as a plain FP32 grid
    mt.codebook0 = nullptr;
  }
  e = sp.simt ? ntc::launch_backward_simt(mt, b, s)
              : (kernel_fold ? ntc::launch_train_tc(mk, bk, s) : ntc::launch_train_tc(mt, b, s));
  if (e != cudaSuccess) return cuda_status(e, "train_step forward/backward");
  if (flags & NTC_FLAG_GRAD_ONLY) return NTC_OK;
  e = ntc::launch_adam(a, a.block_start[a.nseg], s);
  if (e != cudaSuccess) return cuda_status(e, "train_step adam");
  note_fold(tr->noisy_tag, a.fold != 0, a.noise_seed);
  return cuda_status(ntc::launch_advance_step(tr->step, s, a.fold ? a.noisy_tag : nullptr,
                                              a.noise_seed),
                     "train_step step counter");
}

int ntc_autotune_train(const ntc_material* m, const ntc_trainer* tr, const ntc_target* t,
                       int64_t batch, uint64_t seed, int32_t flags, float* loss_out,
                       int32_t* best, float* ms_out, void* stream) {
  if (!best) return fail(NTC_ERR_ARG, "best is NULL");
  if (flags & (NTC_FLAG_SIMT | NTC_FLAG_GRAD_ONLY))
    return fail(NTC_ERR_ARG, "the autotuner times the tensor-core step (no SIMT or GRAD_ONLY flag)");
  const int32_t f = flags | NTC_FLAG_GRAD_ONLY;  // timed steps leave params and step unchanged
  StepPlan sp;
  int st = plan_train_step(m, tr, t, batch, seed, nullptr, loss_out, f, &sp);
  if (st) return st;
  if (sp.simt) return fail(NTC_ERR_ARG, "the FP32 form has no pipeline choice");
  if (m->vq_books > 0) return fail(NTC_ERR_UNSUPPORTED, "autotune: scalar-quantised grids");
  const int np_max = ntc::train_pipelines_layout(*m, 0, 0);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the FP8 form's scales (and recorded maxima) are restored afterwards
  float saved[9];
  const bool f8 = m->precision == NTC_PREC_F8;
  if (f8) {
    cudaError_t e = cudaMemcpyAsync(saved, m->scale, sizeof(saved), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return cuda_status(e, "autotune: save FP8 scales");
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return cuda_status(cudaGetLastError(), "autotune events");
  float best_ms = 1e30f;
  int best_np = 0, rc = NTC_OK;
  for (int np = 1; np <= np_max && rc == NTC_OK; ++np) {
    sp.b.pipelines = np;
    rc = launch_train_plan(m, tr, sp, loss_out, f, s);  // warm-up
    cudaError_t e = rc == NTC_OK ? cudaEventRecord(e0, s) : cudaErrorUnknown;
    for (int r = 0; r < 3 && rc == NTC_OK && e == cudaSuccess; ++r)
      rc = launch_train_plan(m, tr, sp, loss_out, f, s);
    if (rc != NTC_OK) break;
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) rc = cuda_status(e, "autotune");
    if (ms_out) ms_out[np - 1] = ms / 3.f;
    if (ms < best_ms) { best_ms = ms; best_np = np; }
  }
  for (int np = np_max + 1; np <= 3 && ms_out; ++np) ms_out[np - 1] = 0.f;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // the timed gradient-only steps accumulated into the scratch gradient
  cudaError_t e = cudaMemsetAsync(tr->grad, 0, (size_t)tr->n_params * sizeof(float), s);
  if (!e && f8) e = cudaMemcpyAsync(const_cast<float*>(m->scale), saved, sizeof(saved),
                                    cudaMemcpyHostToDevice, s);
  if (!e) e = cudaStreamSynchronize(s);
  if (rc == NTC_OK && e) rc = cuda_status(e, "autotune: restore");
  if (rc != NTC_OK) return rc;
  tune_store(tune_key("train", *m, (flags & NTC_FLAG_CROPS) ? 1 : 0, 0, batch), best_np);
  *best = best_np;
  return NTC_OK;
}

int ntc_tuning_export(char* buf, size_t cap, size_t* len_out) {
  std::string text;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (const auto& kv : g_tune) text += kv.first + " " + std::to_string(kv.second) + "\n";
  }
  if (len_out) *len_out = text.size() + 1;
  if (!buf) return NTC_OK;
  if (cap < text.size() + 1) return fail(NTC_ERR_ARG, "tuning export: %zu bytes needed", text.size() + 1);
  memcpy(buf, text.c_str(), text.size() + 1);
  return NTC_OK;
}

int ntc_tuning_import(const char* text) {
  if (!text) return fail(NTC_ERR_ARG, "text is NULL");
  std::map<std::string, int> add;
  const char* p = text;
  while (*p) {
    const char* e = strchr(p, '\n');
    const std::string line = e ? std::string(p, e) : std::string(p);
    p = e ? e + 1 : p + line.size();
    if (line.empty()) continue;
    const size_t sp = line.rfind(' ');
    if (sp == std::string::npos || sp == 0)
      return fail(NTC_ERR_ARG, "tuning import: malformed line '%.60s'", line.c_str());
    char* end = nullptr;
    const long v = strtol(line.c_str() + sp + 1, &end, 10);
    if (*end != '\0' || v < 1 || v > 5)
      return fail(NTC_ERR_ARG, "tuning import: bad value in '%.60s'", line.c_str());
    add[line.substr(0, sp)] = (int)v;
  }
  std::lock_guard<std::mutex> lock(g_tune_mu);
  for (const auto& kv : add) g_tune[kv.first] = kv.second;
  return NTC_OK;
}

int ntc_tuning_clear(void) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune.clear();
  return NTC_OK;
}

// The optimisation step.  With `check_only` the call validates its
// arguments and returns before its first stream operation.
static int train_step_impl(const ntc_material* m, const ntc_trainer* tr, const ntc_target* t,
                           int64_t batch, uint64_t seed, const float* uvl_or_null,
                           float* loss_out, int32_t flags, void* stream, bool check_only) {
  StepPlan sp;
  const int st = plan_train_step(m, tr, t, batch, seed, uvl_or_null, loss_out, flags, &sp);
  if (st != NTC_OK || check_only) return st;
  return launch_train_plan(m, tr, sp, loss_out, flags, static_cast<cudaStream_t>(stream));
}

int ntc_train_step(const ntc_material* m, const ntc_trainer* tr, const ntc_target* t,
                   int64_t batch, uint64_t seed, const float* uvl_or_null, float* loss_out,
                   int32_t flags, void* stream) {
  return train_step_impl(m, tr, t, batch, seed, uvl_or_null, loss_out, flags, stream, false);
}

int ntc_train_step_check(const ntc_material* m, const ntc_trainer* tr, const ntc_target* t,
                         int64_t batch, uint64_t seed, const float* uvl_or_null, float* loss_out,
                         int32_t flags) {
  return train_step_impl(m, tr, t, batch, seed, uvl_or_null, loss_out, flags, nullptr, true);
}

size_t ntc_train_batch_workspace_bytes(void) { return sizeof(ntc::TrainBatchDev); }

int ntc_train_batch_prepare(const ntc_material* mats, const ntc_trainer* trainers,
                            const ntc_target* targets, const int64_t* batches,
                            int32_t n_materials, uint64_t seed, int32_t flags, float* loss_out,
                            void* workspace, size_t workspace_bytes, ntc_train_batch* out,
                            void* stream) {
  if (!mats || !trainers || !targets || !batches || !out)
    return fail(NTC_ERR_ARG, "train batch: NULL argument");
  if (n_materials < 1 || n_materials > ntc::kMaxTrainBatch)
    return fail(NTC_ERR_ARG, "train batch: n_materials = %d outside 1..%d", n_materials,
                ntc::kMaxTrainBatch);
  const int32_t allowed =
      NTC_FLAG_FREEZE_GRIDS | NTC_FLAG_NO_NOISE | NTC_FLAG_CROPS | NTC_FLAG_GRAD_ONLY;
  if (flags & ~allowed)
    return fail(NTC_ERR_ARG, "train batch: flags 0x%x (batches train on the tensor cores; "
                             "FREEZE_GRIDS, NO_NOISE, CROPS, GRAD_ONLY)", (unsigned)flags);
  CHECK_PTR(workspace, "workspace");
  CHECK_PTR(loss_out, "loss_out");
  if (workspace_bytes < sizeof(ntc::TrainBatchDev))
    return fail(NTC_ERR_ARG, "train batch: workspace of %zu bytes, need %zu", workspace_bytes,
                sizeof(ntc::TrainBatchDev));
  std::unique_ptr<ntc::TrainBatchDev> H(new ntc::TrainBatchDev());
  memset(H.get(), 0, sizeof(ntc::TrainBatchDev));
  const int hl0 = mats[0].hidden_layers == 0 ? 2 : mats[0].hidden_layers;
  int k_lay = 0, dx_lay = 0;
  for (int i = 0; i < n_materials; ++i) {
    const ntc_material* m = &mats[i];
    if (batches[i] < 0) return fail(NTC_ERR_ARG, "train batch material %d: negative batch", i);
    if (m->precision != NTC_PREC_F16)
      return fail(NTC_ERR_UNSUPPORTED,
                  "train batch material %d: batches train FP16 materials on the tensor cores", i);
    if (m->vq_books > 0)
      return fail(NTC_ERR_UNSUPPORTED, "train batch material %d: scalar-quantised grids only", i);
    const int hl = m->hidden_layers == 0 ? 2 : m->hidden_layers;
    if (m->act != mats[0].act || m->interp0 != mats[0].interp0 || hl != hl0)
      return fail(NTC_ERR_UNSUPPORTED,
                  "train batch material %d: every material shares act, interp0 and "
                  "hidden_layers with material 0", i);
    for (int j = 0; j < i; ++j)
      if (trainers[j].params == trainers[i].params || trainers[j].step == trainers[i].step)
        return fail(NTC_ERR_ARG, "train batch: materials %d and %d share a trainer", j, i);
  }
  for (int i = 0; i < n_materials; ++i) {
    const ntc_material* m = &mats[i];
    StepPlan sp;
    const int64_t nb = batches[i] > 0 ? batches[i] : 1;
    // (the loss array was checked as a whole; each material adds into its element)
    int st = plan_train_step(m, &trainers[i], &targets[i], nb, seed + (uint64_t)i, nullptr,
                             loss_out, flags, &sp);
    if (st) {
      char why[sizeof(g_err)];
      memcpy(why, g_err, sizeof(why));
      return fail(st, "train batch material %d: %s", i, why);
    }
    if (sp.simt || sp.vq)
      return fail(NTC_ERR_UNSUPPORTED, "train batch material %d: tensor-core trainer only", i);
    const bool active = batches[i] > 0;
    sp.b.loss = loss_out + i;
    H->mats[i] = sp.mt;
    H->args[i] = sp.b;
    H->tile_start[i + 1] = H->tile_start[i] + (active ? (batches[i] + 127) / 128 : 0);
    const bool adam = active && !(flags & NTC_FLAG_GRAD_ONLY);
    if (adam) H->adam[i] = sp.a;
    H->adam_start[i + 1] = H->adam_start[i] + (adam ? sp.a.block_start[sp.a.nseg] : 0);
    const bool noise = active && sp.noise_pass;
    if (noise) H->noise[i] = sp.na;
    H->noise_start[i + 1] = H->noise_start[i] + (noise ? sp.na.block_start[sp.na.nseg] : 0);
    int k = 0, dx = 0;
    ntc::train_widths(*m, &k, &dx);
    k_lay = k > k_lay ? k : k_lay;
    dx_lay = dx > dx_lay ? dx : dx_lay;
  }
  if (ntc::train_pipelines_layout(mats[0], k_lay, dx_lay) == 0)
    return fail(NTC_ERR_UNSUPPORTED, "train batch: the shared layout does not fit one CTA");
  H->n = n_materials;
  H->adam_done = 0;
  H->total_tiles = H->tile_start[n_materials];
  H->adam_blocks = H->adam_start[n_materials];
  H->noise_blocks = H->noise_start[n_materials];
  if (H->adam_blocks > 0x7fffffff || H->noise_blocks > 0x7fffffff)
    return fail(NTC_ERR_SHAPE, "train batch: too many parameters for one launch");
  cudaError_t e = cudaMemcpyAsync(workspace, H.get(), sizeof(ntc::TrainBatchDev),
                                  cudaMemcpyHostToDevice, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_status(e, "train batch: descriptor upload");
  out->workspace = workspace;
  out->loss_out = loss_out;
  out->n_materials = n_materials;
  out->flags = flags;
  out->total_tiles = H->total_tiles;
  out->adam_blocks = H->adam_blocks;
  out->noise_blocks = H->noise_blocks;
  out->act = mats[0].act;
  out->interp0 = mats[0].interp0;
  out->hidden_layers = hl0;
  out->k_layout = k_lay;
  out->dx_layout = dx_lay;
  return NTC_OK;
}

int ntc_train_step_batched(const ntc_train_batch* batch, void* stream) {
  if (!batch || !batch->workspace || !batch->loss_out)
    return fail(NTC_ERR_ARG, "train batch is not prepared");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  auto* dev = static_cast<ntc::TrainBatchDev*>(batch->workspace);
  cudaError_t e = cudaMemsetAsync(batch->loss_out, 0, sizeof(float) * batch->n_materials, s);
  if (e != cudaSuccess) return cuda_status(e, "train batch: loss reset");
  e = ntc::launch_noise_batched(dev, batch->noise_blocks, s);
  if (e != cudaSuccess) return cuda_status(e, "train batch: noise pass");
  // the kernel class of the batch (its layout comes from k_layout, dx_layout)
  ntc_material cls{};
  cls.c0 = cls.c1 = 1;
  cls.act = batch->act;
  cls.interp0 = batch->interp0;
  cls.hidden_layers = batch->hidden_layers;
  cls.precision = NTC_PREC_F16;
  e = ntc::launch_train_tc_batched(dev, cls, batch->total_tiles, batch->k_layout,
                                   batch->dx_layout, s);
  if (e != cudaSuccess) return cuda_status(e, "train batch: forward/backward");
  if (batch->flags & NTC_FLAG_GRAD_ONLY) return NTC_OK;
  return cuda_status(ntc::launch_adam_batched(dev, batch->adam_blocks, s), "train batch: adam");
}

size_t ntc_batch_workspace_bytes(void) { return sizeof(ntc::BatchHeader); }

int ntc_batch_prepare(const ntc_material* mats, const int64_t* n_queries, int32_t n_materials,
                      int32_t filter, void* workspace, size_t workspace_bytes, ntc_batch* batch_out,
                      void* stream) {
  if (!mats || !n_queries || !batch_out) return fail(NTC_ERR_ARG, "batch: NULL argument");
  if (n_materials < 1 || n_materials > NTC_MAX_BATCH)
    return fail(NTC_ERR_ARG, "batch: n_materials = %d outside 1..%d", n_materials, NTC_MAX_BATCH);
  if (filter != NTC_FILTER_NEAREST && filter != NTC_FILTER_TRILINEAR) return fail(NTC_ERR_ARG, "filter");
  CHECK_PTR(workspace, "workspace");
  if (workspace_bytes < sizeof(ntc::BatchHeader))
    return fail(NTC_ERR_ARG, "batch: workspace of %zu bytes, need %zu", workspace_bytes,
                sizeof(ntc::BatchHeader));
  std::vector<ntc::BatchHeader> host(1);
  ntc::BatchHeader& B = host[0];
  memset(&B, 0, sizeof(B));
  const int per_tile = filter == NTC_FILTER_TRILINEAR ? 16 : 128;
  uint32_t plan_bytes = 0;
  // input-layout class: one fast class for all, -1 fast with mixed classes, 0 generic
  int cls = -2;
  for (int i = 0; i < n_materials; ++i) {
    const ntc_material* m = &mats[i];
    int st = check_material(m, false);
    if (st) {
      char why[sizeof(g_err)];
      memcpy(why, g_err, sizeof(why));
      return fail(st, "batch material %d: %s", i, why);
    }
    if (m->precision != NTC_PREC_F16)
      return fail(NTC_ERR_UNSUPPORTED, "batch material %d: batches decode FP16 materials", i);
    if (m->hidden_layers == 3)
      return fail(NTC_ERR_UNSUPPORTED, "batch material %d: batches decode two hidden layers", i);
    if (m->vq_books > 0)
      return fail(NTC_ERR_UNSUPPORTED, "batch material %d: batches decode scalar grids", i);
    if (n_queries[i] < 0) return fail(NTC_ERR_ARG, "batch material %d: negative query count", i);
    if (n_queries[i] > INT32_MAX)
      return fail(NTC_ERR_SHAPE, "batch material %d: more than 2^31 - 1 queries", i);
    const int c = ntc::fast_class(*m);
    cls = cls == -2 ? c : (cls == c ? cls : (cls != 0 && c != 0 ? -1 : 0));
    B.mats[i] = *m;
    B.tile_start[i + 1] = B.tile_start[i] + (n_queries[i] + per_tile - 1) / per_tile;
    B.q_off[i + 1] = B.q_off[i] + n_queries[i];
    B.o_off[i + 1] = B.o_off[i] + n_queries[i] * m->channels;
  }
  if (B.tile_start[n_materials] > INT32_MAX)
    return fail(NTC_ERR_SHAPE, "batch: more than 2^31 - 1 tiles");
  uint32_t kmax = 0;
  for (int i = 0; i < n_materials; ++i) {
    const uint32_t need = ntc::ws_plan_bytes(mats[i], cls != 0);
    plan_bytes = (need & 0xFFFFFFu) > plan_bytes ? (need & 0xFFFFFFu) : plan_bytes;
    kmax = (need >> 24) > kmax ? (need >> 24) : kmax;
  }
  plan_bytes |= kmax << 24;  // internal: plan bytes | largest K << 24
  if (ntc::ws_batched_smem(plan_bytes) > 227 * 1024)
    return fail(NTC_ERR_UNSUPPORTED, "batch: shared memory");
  B.n_materials = n_materials;
  B.total_tiles = B.tile_start[n_materials];
  cudaError_t e = cudaMemcpyAsync(workspace, &B, sizeof(B), cudaMemcpyHostToDevice,
                                  static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_status(e, "batch: descriptor upload");
  batch_out->workspace = workspace;
  batch_out->n_materials = n_materials;
  batch_out->filter = filter;
  batch_out->total_queries = B.q_off[n_materials];
  batch_out->total_outputs = B.o_off[n_materials];
  batch_out->total_tiles = B.total_tiles;
  batch_out->wg_smem = (int32_t)plan_bytes;
  batch_out->fast = cls;
  return NTC_OK;
}

int ntc_decode_batched(const ntc_batch* batch, const float* uvl, void* out, int32_t out_dtype,
                       void* stream) {
  if (!batch || !batch->workspace) return fail(NTC_ERR_ARG, "batch is not prepared");
  if (!out_dtype_ok(out_dtype)) return fail(NTC_ERR_ARG, "out_dtype %d", out_dtype);
  if (batch->total_queries == 0) return NTC_OK;
  CHECK_PTR(uvl, "uvl");
  CHECK_PTR(out, "out");
  return cuda_status(
      ntc::launch_decode_ws_batched(static_cast<const ntc::BatchHeader*>(batch->workspace),
                                    batch->total_tiles, (uint32_t)batch->wg_smem, batch->fast, uvl,
                                    out, out_dtype, batch->filter, static_cast<cudaStream_t>(stream)),
      "decode_batched");
}

int ntc_quantize_pack(const float* values, int64_t cells, int32_t c, int32_t bits, float q,
                      uint8_t* packed_out, float* snapped_out, void* stream) {
  if (cells < 0 || ntc_cell_bytes(c, bits) == 0 || !(q > 0.f)) return fail(NTC_ERR_ARG, "quantize args");
  if (cells == 0) return NTC_OK;
  CHECK_PTR(values, "values");
  if (packed_out && !aligned(packed_out)) return fail(NTC_ERR_ALIGN, "packed_out");
  if (snapped_out && !aligned(snapped_out)) return fail(NTC_ERR_ALIGN, "snapped_out");
  return cuda_status(ntc::launch_quantize_pack(values, cells, c, bits, q, packed_out, snapped_out,
                                               static_cast<cudaStream_t>(stream)),
                     "quantize_pack");
}

int ntc_unpack(const uint8_t* packed, int64_t cells, int32_t c, int32_t bits, float q,
               int32_t* idx_out, float* values_out, void* stream) {
  if (cells < 0 || ntc_cell_bytes(c, bits) == 0 || !(q > 0.f)) return fail(NTC_ERR_ARG, "unpack args");
  if (cells == 0) return NTC_OK;
  CHECK_PTR(packed, "packed");
  if (idx_out && !aligned(idx_out)) return fail(NTC_ERR_ALIGN, "idx_out");
  if (values_out && !aligned(values_out)) return fail(NTC_ERR_ALIGN, "values_out");
  return cuda_status(ntc::launch_unpack(packed, cells, c, bits, q, idx_out, values_out,
                                        static_cast<cudaStream_t>(stream)),
                     "unpack");
}

static int sample_batch(uint64_t seed, int64_t step, int64_t batch, int32_t width,
                        int32_t height, int32_t mips, int crops, int32_t* xym_out, void* stream) {
  if (batch < 0 || step < 0 || !pow2(width) || !pow2(height) || mips < 1 || mips > NTC_MAX_MIPS)
    return fail(NTC_ERR_ARG, "sample_batch args");
  if (batch == 0) return NTC_OK;
  CHECK_PTR(xym_out, "xym_out");
  return cuda_status(ntc::launch_sample_batch(seed, step, batch, width, height, mips, crops,
                                              xym_out, static_cast<cudaStream_t>(stream)),
                     "sample_batch");
}

int ntc_sample_batch(uint64_t seed, int64_t step, int64_t batch, int32_t width, int32_t height,
                     int32_t mips, int32_t* xym_out, void* stream) {
  return sample_batch(seed, step, batch, width, height, mips, 0, xym_out, stream);
}

int ntc_vq_assign(const float* values, int64_t cells, int32_t c0, const float* codebooks,
                  int32_t books, uint8_t* idx_out, void* stream) {
  if (cells < 0 || c0 < 1 || c0 > ntc::kMaxGridCh || books < 1 || books > 4)
    return fail(NTC_ERR_ARG, "vq_assign args");
  if (cells == 0) return NTC_OK;
  CHECK_PTR(values, "values");
  CHECK_PTR(codebooks, "codebooks");
  if (!idx_out) return fail(NTC_ERR_ARG, "idx_out is NULL");
  return cuda_status(ntc::launch_vq_assign(values, cells, c0, codebooks, books, idx_out,
                                           static_cast<cudaStream_t>(stream)),
                     "vq_assign");
}

int ntc_sample_crops(uint64_t seed, int64_t step, int64_t batch, int32_t width, int32_t height,
                     int32_t mips, int32_t* xym_out, void* stream) {
  return sample_batch(seed, step, batch, width, height, mips, 1, xym_out, stream);
}

int ntc_sample_features(const ntc_material* m, const float* uvl, int64_t n, float* rows_out,
                        int32_t flags, uint64_t noise_seed, int64_t noise_step, void* stream) {
  int st = check_material(m, (flags & NTC_FLAG_NOISE) != 0);
  if (st) return st;
  if (n < 0) return fail(NTC_ERR_ARG, "n < 0");
  if (n == 0) return NTC_OK;
  CHECK_PTR(uvl, "uvl");
  CHECK_PTR(rows_out, "rows_out");
  return cuda_status(ntc::launch_sample_features(*m, uvl, n, rows_out, (flags & NTC_FLAG_NOISE) != 0,
                                                 noise_seed, noise_step,
                                                 static_cast<cudaStream_t>(stream)),
                     "sample_features");
}

}  // extern "C"
