// C-ABI entry points (include/crom.h): argument checks, context and weight
// management, dispatch to the FP32 CUDA-core and the tcgen05 kernels.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <thread>
#include <cstdio>
#include <string>
#include <vector>

#include <cuda_fp16.h>

#include "crom_internal.h"

namespace crom {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

namespace {

int fail(int code, const std::string& msg) {
  set_error(msg);
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  return fail(CROM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

size_t param_count(const crom_decoder_desc& d) {
  size_t in = (size_t)d.m + d.r, w = d.width;
  size_t n = w * in + w;
  n += (size_t)(d.hidden - 1) * (w * w + w);
  n += w + 1;
  return n;
}

// f16 bits of f rounded to nearest even (the conversion of cuda_fp16.h, usable
// on the host), and back.
uint16_t f32_to_f16(float f) {
  const __half h = __float2half_rn(f);
  uint16_t u;
  memcpy(&u, &h, 2);
  return u;
}
float f16_to_f32(uint16_t u) {
  __half h;
  memcpy(&h, &u, 2);
  return __half2float(h);
}
// Largest power of two 2^e with v * 2^e < 2 (v > 0), so that v * 2^e lies in [1, 2).
float pow2_scale(float v) {
  if (!(v > 0.f) || !isfinite(v)) return 1.f;
  return ldexpf(1.f, -ilogbf(v));
}

// Byte offset of element (row, k) of a [rows][128] bf16 operand stored K-major
// with the 128-byte swizzle: two k-blocks of 64 columns, each rows x 128 bytes,
// 16-byte chunk c of row `row` stored at chunk position c ^ (row % 8).
size_t kmajor_sw128(int row, int k, int rows) {
  const int region = k >> 6, kk = k & 63;
  return (size_t)region * rows * 128 + (size_t)row * 128 + (size_t)(((kk >> 3) ^ (row & 7)) << 4) +
         (size_t)(kk & 7) * 2;
}

void free_weights(crom_ctx* ctx) {
  ++ctx->scratch_gen;  // a recorded rollout refers to these buffers
  auto& w = ctx->w;
  cudaFree(w.w1);
  cudaFree(w.b1);
  cudaFree(w.wt);
  cudaFree(w.bh);
  cudaFree(w.wout);
  cudaFree(w.tc_img);
  cudaFree(w.tc_lo);
  w = DeviceWeights{};
  ctx->has_weights = false;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// Device allocations freed together when the holder goes out of scope; the first
// failure is kept in err and later requests return nullptr.
struct DeviceAllocs {
  std::vector<void*> ptrs;
  cudaError_t err = cudaSuccess;
  template <class T>
  T* get(size_t n) {
    void* p = nullptr;
    if (err == cudaSuccess) err = cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T));
    if (p) ptrs.push_back(p);
    return static_cast<T*>(p);
  }
  ~DeviceAllocs() {
    for (void* p : ptrs) cudaFree(p);
  }
};

bool tc_shape_ok(const crom_decoder_desc& d) {
  return d.width == kTcWidth && d.hidden >= 2 && d.hidden <= 5 && d.m >= 1 && d.m <= 2 &&
         d.r >= 1 && d.r <= kTcProjRows - 1 && d.activation == CROM_ACT_ELU;
}

}  // namespace
}  // namespace crom

using namespace crom;

extern "C" {

int crom_version(void) { return 10000; }

const char* crom_last_error(void) { return g_last_error.c_str(); }

int crom_create(crom_ctx** out, const crom_decoder_desc* desc, int device) {
  if (!out || !desc) return fail(CROM_ERR_INVALID_ARG, "crom_create: null argument");
  *out = nullptr;
  crom_decoder_desc d = *desc;
  if (d.m < 1 || d.m > 3 || d.r < 1 || d.r > 32 || d.width < 32 || d.width > 256 ||
      d.width % 32 != 0 || d.hidden < 1 || d.hidden > 8)
    return fail(CROM_ERR_INVALID_ARG,
                "crom_create: need 1<=m<=3, 1<=r<=32, width%32==0 in [32,256], 1<=hidden<=8");
  if (d.activation != CROM_ACT_ELU && d.activation != CROM_ACT_SIREN)
    return fail(CROM_ERR_INVALID_ARG, "crom_create: unknown activation");
  if (!(d.omega0 >= 0.f) || !isfinite(d.omega0)) return fail(CROM_ERR_INVALID_ARG, "crom_create: bad omega0");
  if (d.activation == CROM_ACT_SIREN && d.omega0 == 0.f) d.omega0 = 30.f;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n == 0) return fail(CROM_ERR_CUDA, "crom_create: no CUDA device");
  if (device < 0 || device >= n) return fail(CROM_ERR_INVALID_ARG, "crom_create: bad device index");
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, device);
  if (e != cudaSuccess) return cuda_fail(e, "crom_create");
  if (prop.major != 10 || prop.minor != 3)
    return fail(CROM_ERR_CUDA, "crom_create: the library is built for sm_103a only (found sm_" +
                                   std::to_string(prop.major) + std::to_string(prop.minor) + ")");
  crom_ctx* ctx = new crom_ctx();
  ctx->device = device;
  ctx->desc = d;
  ctx->num_sms = prop.multiProcessorCount;
  {
    DeviceGuard g(device);
    e = cudaMalloc(&ctx->queue, sizeof(int) * 4);
    if (e == cudaSuccess) e = cudaMemset(ctx->queue, 0, sizeof(int) * 4);
  }
  if (e != cudaSuccess) {
    delete ctx;
    return cuda_fail(e, "crom_create");
  }
  *out = ctx;
  return CROM_OK;
}

int crom_destroy(crom_ctx* ctx) {
  if (!ctx) return CROM_OK;
  {
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    free_weights(ctx);
    cudaFree(ctx->partials);
    cudaFree(ctx->counters);
    cudaFree(ctx->targets);
    cudaFree(ctx->qbase);
    cudaFree(ctx->tangent);
    cudaFree(ctx->host_stage);
    cudaFree(ctx->order);
    cudaFree(ctx->queue);
    if (ctx->rollout_exec) cudaGraphExecDestroy(ctx->rollout_exec);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  }
  delete ctx;
  return CROM_OK;
}

int crom_set_weights(crom_ctx* ctx, const float* params, size_t n, int params_on_device,
                     crom_stream stream) {
  if (!ctx || !params) return fail(CROM_ERR_INVALID_ARG, "crom_set_weights: null argument");
  const crom_decoder_desc d = ctx->desc;
  const size_t need = param_count(d);
  if (n != need)
    return fail(CROM_ERR_INVALID_ARG, "crom_set_weights: expected " + std::to_string(need) +
                                          " floats, got " + std::to_string(n));
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<float> h(n);
  cudaError_t e;
  if (params_on_device) {
    e = cudaMemcpyAsync(h.data(), params, n * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "crom_set_weights (read params)");
  } else {
    memcpy(h.data(), params, n * sizeof(float));
  }
  for (size_t i = 0; i < n; ++i)
    if (!isfinite(h[i])) return fail(CROM_ERR_NONFINITE, "crom_set_weights: non-finite parameter");

  const int m = d.m, r = d.r, w = d.width, L = d.hidden;
  const size_t in = (size_t)m + r;
  const float* W1 = h.data();
  const float* B1 = W1 + w * in;
  const float* cur = B1 + w;
  std::vector<float> wt((size_t)(L - 1) * w * w), bh((size_t)(L - 1) * w);
  std::vector<const float*> hidden_w(L - 1);
  for (int l = 0; l < L - 1; ++l) {
    const float* Wl = cur;
    const float* bl = Wl + (size_t)w * w;
    hidden_w[l] = Wl;
    for (int o = 0; o < w; ++o)
      for (int k = 0; k < w; ++k) wt[(size_t)l * w * w + (size_t)k * w + o] = Wl[(size_t)o * w + k];
    for (int o = 0; o < w; ++o) bh[(size_t)l * w + o] = bl[o];
    cur = bl + w;
  }
  const float* Wout = cur;
  const float bout = Wout[w];

  free_weights(ctx);
  DeviceWeights& dw = ctx->w;
  auto up = [&](float** dst, const float* src, size_t count) -> cudaError_t {
    cudaError_t err = cudaMalloc(dst, std::max<size_t>(count, 1) * sizeof(float));
    if (err != cudaSuccess) return err;
    if (count == 0) return cudaSuccess;
    return cudaMemcpy(*dst, src, count * sizeof(float), cudaMemcpyHostToDevice);
  };
  if ((e = up(&dw.w1, W1, w * in)) != cudaSuccess || (e = up(&dw.b1, B1, w)) != cudaSuccess ||
      (e = up(&dw.wt, wt.data(), wt.size())) != cudaSuccess ||
      (e = up(&dw.bh, bh.data(), bh.size())) != cudaSuccess ||
      (e = up(&dw.wout, Wout, w)) != cudaSuccess) {
    free_weights(ctx);
    return cuda_fail(e, "crom_set_weights (upload)");
  }
  dw.bout = bout;

  // f16 images of the tensor-core kernels; left out (those precisions then return
  // CROM_ERR_UNSUPPORTED) when a weight lies outside the f16 range.
  bool f16_range = true;
  for (int l = 0; l < L - 1 && f16_range; ++l)
    for (size_t i = 0; i < (size_t)w * w; ++i)
      if (fabsf(hidden_w[l][i]) > 65000.f) { f16_range = false; break; }
  for (size_t i = 0; i < bh.size() && f16_range; ++i)
    if (fabsf(bh[i]) > 45000.f) f16_range = false;  // log2 e * b in f16
  for (int k = 0; k < w && f16_range; ++k) {
    if (fabsf(Wout[k]) > 65000.f) f16_range = false;
    for (int j = 0; j < r; ++j)
      if (fabsf(W1[(size_t)k * in + m + j]) > 65000.f) f16_range = false;
  }
  if (tc_shape_ok(d) && f16_range) {
    // hidden matrices (K-major SW128), the projection matrix P, then the
    // reconstruction's output operand (row 0 = f16(w_out), row 1 = its low part)
    const size_t layers_bytes = (size_t)(L - 1) * kTcLayerBytes;
    std::vector<uint8_t> img(layers_bytes + 2 * kTcProjBytes + kTcBiasBytes, 0);
    std::vector<uint16_t> lo((size_t)(L - 1) * w * w);
    for (int l = 0; l < L - 1; ++l)
      for (int o = 0; o < w; ++o)
        for (int k = 0; k < w; ++k) {
          const float x = hidden_w[l][(size_t)o * w + k];
          const uint16_t v = f32_to_f16(x);
          memcpy(&img[(size_t)l * kTcLayerBytes + kmajor_sw128(o, k, w)], &v, 2);
          lo[((size_t)l * w + o) * w + k] = f32_to_f16(x - f16_to_f32(v));  // exact difference, rounded once
        }
    for (int row = 0; row < kTcProjRows; ++row)
      for (int k = 0; k < w; ++k) {
        float val = 0.f;
        if (row == 0) val = Wout[k];
        else if (row <= r) val = W1[(size_t)k * in + m + (row - 1)];
        const uint16_t v = f32_to_f16(val);
        memcpy(&img[layers_bytes + kmajor_sw128(row, k, kTcProjRows)], &v, 2);
      }
    // the f16 reconstruction's output and bias operands: high and low f16 parts of
    // ln 2 * w_out and of log2 e * b_l (its activations are carried times log2 e)
    auto split16 = [](double v, uint16_t& hi, uint16_t& lo) {
      hi = f32_to_f16((float)v);
      lo = f32_to_f16((float)(v - (double)f16_to_f32(hi)));
    };
    const double kLn2 = 0.6931471805599453, kLog2e = 1.4426950408889634;
    for (int k = 0; k < w; ++k) {
      uint16_t hi, lo;
      split16(kLn2 * Wout[k], hi, lo);
      memcpy(&img[layers_bytes + kTcProjBytes + kmajor_sw128(0, k, kTcProjRows)], &hi, 2);
      memcpy(&img[layers_bytes + kTcProjBytes + kmajor_sw128(1, k, kTcProjRows)], &lo, 2);
    }
    for (int l = 0; l < L - 1; ++l)
      for (int u = 0; u < w; ++u) {
        uint16_t hi, lo;
        split16(kLog2e * bh[(size_t)l * w + u], hi, lo);
        memcpy(&img[layers_bytes + 2 * kTcProjBytes + kmajor_sw128(u, 16 * l, w)], &hi, 2);
        memcpy(&img[layers_bytes + 2 * kTcProjBytes + kmajor_sw128(u, 16 * l + 1, w)], &lo, 2);
      }
    e = cudaMalloc(&dw.tc_img, img.size());
    if (e == cudaSuccess) e = cudaMemcpy(dw.tc_img, img.data(), img.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&dw.tc_lo, lo.size() * 2);
    if (e == cudaSuccess) e = cudaMemcpy(dw.tc_lo, lo.data(), lo.size() * 2, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      free_weights(ctx);
      return cuda_fail(e, "crom_set_weights (tensor-core image)");
    }
    dw.tc_img_bytes = layers_bytes + kTcProjBytes;  // what the step loads; the output operand follows
    dw.tc_lo_bytes = lo.size() * 2;
    float mx = 0.f, mo = 0.f;
    for (int u = 0; u < w; ++u) {
      for (int k = 0; k < m; ++k) mx = fmaxf(mx, fabsf(W1[(size_t)u * in + k]));
      mo = fmaxf(mo, fabsf(Wout[u]));
    }
    dw.tc_sx = pow2_scale(mx);
    dw.tc_sr = pow2_scale(mo);
  }
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    free_weights(ctx);
    return cuda_fail(e, "crom_set_weights");
  }
  ctx->has_weights = true;
  return CROM_OK;
}

int crom_decode(crom_ctx* ctx, int n_inst, const double* q, const int* pt_off, const float* x,
                int n_pts, unsigned want, float* out, crom_stream stream) {
  if (!ctx) return fail(CROM_ERR_INVALID_ARG, "crom_decode: null context");
  if (!ctx->has_weights) return fail(CROM_ERR_INVALID_ARG, "crom_decode: weights not set");
  if (n_inst < 0 || n_pts < 0) return fail(CROM_ERR_INVALID_ARG, "crom_decode: negative size");
  if ((want & ~31u) != 0 || want == 0) return fail(CROM_ERR_INVALID_ARG, "crom_decode: bad channel mask");
  if (n_pts == 0) return CROM_OK;
  if (n_inst == 0 || !q || !pt_off || !x || !out)
    return fail(CROM_ERR_INVALID_ARG, "crom_decode: null array or no instance for the points");
  DeviceGuard g(ctx->device);
  cudaError_t e = launch_decode_fp32(ctx, n_inst, q, pt_off, x, n_pts, want, out, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "crom_decode");
  return CROM_OK;
}

int crom_decode_tc(crom_ctx* ctx, int precision, int n_inst, const double* q, const int* pt_off, const float* x,
                   int n_pts, unsigned want, float* out, crom_stream stream) {
  const char* fn = "crom_decode_tc";
  if (!ctx) return fail(CROM_ERR_INVALID_ARG, std::string(fn) + ": null context");
  if (!ctx->has_weights) return fail(CROM_ERR_INVALID_ARG, std::string(fn) + ": weights not set");
  if (n_inst < 0 || n_pts < 0) return fail(CROM_ERR_INVALID_ARG, std::string(fn) + ": negative size");
  if ((want & ~31u) != 0 || want == 0) return fail(CROM_ERR_INVALID_ARG, std::string(fn) + ": bad channel mask");
  if (want & CROM_WANT_DXX)
    return fail(CROM_ERR_UNSUPPORTED, std::string(fn) + ": the per-coordinate second derivatives (CROM_WANT_DXX) "
                                                        "are FP32-only (crom_decode); the Laplacian is available");
  if (precision != CROM_PREC_F16X2 && precision != CROM_PREC_F16)
    return fail(CROM_ERR_UNSUPPORTED, std::string(fn) + ": precision F16X2 or F16");
  if (!tc_shape_ok(ctx->desc) || !ctx->w.tc_img)
    return fail(CROM_ERR_UNSUPPORTED, std::string(fn) + ": needs width 128, 2<=hidden<=5, m<=2, r<=15, ELU");
  if (n_pts == 0) return CROM_OK;
  if (n_inst == 0 || !q || !pt_off || !x || !out)
    return fail(CROM_ERR_INVALID_ARG, std::string(fn) + ": null array or no instance for the points");
  DeviceGuard g(ctx->device);
  cudaError_t e = launch_decode_tc(ctx, precision == CROM_PREC_F16X2, n_inst, q, pt_off, x, n_pts, want, out,
                                   (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, fn);
  return CROM_OK;
}

int crom_device_flags(crom_ctx* ctx, int* flags, crom_stream stream) {
  if (!ctx || !flags) return fail(CROM_ERR_INVALID_ARG, "crom_device_flags: null argument");
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  int q[4] = {0, 0, 0, 0};
  cudaError_t e = cudaMemcpyAsync(q, ctx->queue, sizeof(q), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->queue + 2, 0, sizeof(int), s);  // the reconstruction's flag is sticky
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "crom_device_flags");
  *flags = (q[1] ? 1 : 0) | (q[2] ? 2 : 0);
  return CROM_OK;
}

int crom_tangent_velocity(crom_ctx* ctx, int n_inst, const double* q, const double* q_prev, double dt,
                          const int* pt_off, const float* x, int n_pts, float* out, crom_stream stream) {
  const char* fn = "crom_tangent_velocity";
  if (!ctx) return fail(CROM_ERR_INVALID_ARG, std::string(fn) + ": null context");
  if (!ctx->has_weights) return fail(CROM_ERR_INVALID_ARG, std::string(fn) + ": weights not set");
  if (n_inst < 0 || n_pts < 0) return fail(CROM_ERR_INVALID_ARG, std::string(fn) + ": negative size");
  if (!(dt > 0.0) || !isfinite(dt)) return fail(CROM_ERR_INVALID_ARG, std::string(fn) + ": dt must be finite and > 0");
  if (n_pts == 0) return CROM_OK;
  if (n_inst == 0 || !q || !q_prev || !pt_off || !x || !out)
    return fail(CROM_ERR_INVALID_ARG, std::string(fn) + ": null array or no instance for the points");
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t need = (size_t)n_inst * ctx->desc.width;  // layer-1 seeds W_1q qdot_i
  if (need > ctx->tangent_cap) {
    cudaFree(ctx->tangent);
    ctx->tangent = nullptr;
    ctx->tangent_cap = 0;
    cudaError_t e = cudaMalloc(&ctx->tangent, need * sizeof(float));
    if (e != cudaSuccess) return cuda_fail(e, fn);
    ctx->tangent_cap = need;
  }
  cudaError_t e = launch_tangent_fp32(ctx, n_inst, q, q_prev, dt, pt_off, x, n_pts, ctx->tangent, out, s);
  if (e != cudaSuccess) return cuda_fail(e, fn);
  return CROM_OK;
}

int crom_step(crom_ctx* ctx, const crom_step_desc* step, int precision, int n_inst, double* q,
              const float* alpha, const float* vel, const int* s_off, const float* samples,
              int n_samples, int max_samples, int* status, crom_stream stream) {
  if (!ctx || !step) return fail(CROM_ERR_INVALID_ARG, "crom_step: null argument");
  if (!ctx->has_weights) return fail(CROM_ERR_INVALID_ARG, "crom_step: weights not set");
  if (n_inst < 0 || n_samples < 0) return fail(CROM_ERR_INVALID_ARG, "crom_step: negative size");
  if (!(step->dt > 0.0) || !isfinite(step->dt)) return fail(CROM_ERR_INVALID_ARG, "crom_step: dt must be finite and > 0");
  if (step->gn_iters < 1 || step->gn_iters > 16) return fail(CROM_ERR_INVALID_ARG, "crom_step: gn_iters must be in 1..16");
  if (step->pde != CROM_PDE_HEAT && step->pde != CROM_PDE_ADVDIFF) return fail(CROM_ERR_INVALID_ARG, "crom_step: unknown pde");
  if (step->coef_per_sample != 0 && step->coef_per_sample != 1)
    return fail(CROM_ERR_INVALID_ARG, "crom_step: coef_per_sample must be 0 or 1");
  if (step->line_search < 0 || step->line_search > 16)
    return fail(CROM_ERR_INVALID_ARG, "crom_step: line_search must be in 0..16");
  if (step->line_search > 0 && precision != CROM_PREC_F16X2 && precision != CROM_PREC_F16)
    return fail(CROM_ERR_UNSUPPORTED, "crom_step: the line search is available with CROM_PREC_F16X2 and CROM_PREC_F16");
  if (n_inst == 0) return CROM_OK;
  if (!q || !alpha || !s_off || !status || (n_samples > 0 && !samples))
    return fail(CROM_ERR_INVALID_ARG, "crom_step: null array");
  if (step->pde == CROM_PDE_ADVDIFF && !vel) return fail(CROM_ERR_INVALID_ARG, "crom_step: advection needs vel");
  if (max_samples < 1) return fail(CROM_ERR_INVALID_ARG, "crom_step: max_samples must be >= 1");
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (precision == CROM_PREC_FP32) {
    if (step_fp32_max_tiles(ctx, n_inst, max_samples) > 65535)
      return fail(CROM_ERR_INVALID_ARG, "crom_step: max_samples too large for the FP32 step's grid (at most 65535 "
                                        "CTAs per instance); use CROM_PREC_F16X2 or split the instance");
    e = launch_step_fp32(ctx, step, n_inst, q, alpha, vel, s_off, samples, n_samples, max_samples, status, s);
  } else if (precision == CROM_PREC_F16X2 || precision == CROM_PREC_F16) {
    if (!tc_shape_ok(ctx->desc) || !ctx->w.tc_img)
      return fail(CROM_ERR_UNSUPPORTED, "crom_step: F16X2 and F16 need width 128, 2<=hidden<=5, m<=2, r<=15, ELU");
    e = launch_step_tc(ctx, step, precision == CROM_PREC_F16X2, n_inst, q, alpha, vel, s_off, samples, n_samples,
                       max_samples, status, s);
  } else {
    return fail(CROM_ERR_UNSUPPORTED, "crom_step: precision not available for the step");
  }
  if (e != cudaSuccess) return cuda_fail(e, "crom_step");
  return CROM_OK;
}

int crom_step_host(crom_ctx* ctx, const crom_step_desc* step, int precision, int n_inst, double* q,
                   const float* alpha, const float* vel, const int* s_off, const float* samples, int n_samples,
                   int max_samples, int* status, crom_stream stream) {
  const char* fn = "crom_step_host";
  if (!ctx || !step) return fail(CROM_ERR_INVALID_ARG, std::string(fn) + ": null argument");
  if (n_inst < 0 || n_samples < 0) return fail(CROM_ERR_INVALID_ARG, std::string(fn) + ": negative size");
  if (n_inst == 0) return CROM_OK;
  if (!q || !alpha || !s_off || !status || (n_samples > 0 && !samples))
    return fail(CROM_ERR_INVALID_ARG, std::string(fn) + ": null array");
  if (step->pde == CROM_PDE_ADVDIFF && !vel)
    return fail(CROM_ERR_INVALID_ARG, std::string(fn) + ": advection needs vel");
  // the offsets are on the host here, so they can be checked before anything runs
  if (s_off[0] != 0 || s_off[n_inst] != n_samples)
    return fail(CROM_ERR_INVALID_ARG, std::string(fn) + ": s_off must start at 0 and end at n_samples");
  for (int i = 0; i < n_inst; ++i)
    if (s_off[i + 1] < s_off[i]) return fail(CROM_ERR_INVALID_ARG, std::string(fn) + ": s_off must not decrease");
  const int m = ctx->desc.m, r = ctx->desc.r;
  const size_t n_alpha = step->coef_per_sample ? (size_t)n_samples : (size_t)n_inst;
  // packed staging: q, status, alpha, offsets, samples, velocities at 256-byte offsets
  const size_t sizes[6] = {(size_t)n_inst * r * sizeof(double), (size_t)n_inst * sizeof(int), n_alpha * sizeof(float),
                           (size_t)(n_inst + 1) * sizeof(int), (size_t)n_samples * m * sizeof(float),
                           step->pde == CROM_PDE_ADVDIFF ? (size_t)n_samples * m * sizeof(float) : 0};
  size_t off[6], total = 0;
  for (int k = 0; k < 6; ++k) {
    off[k] = total;
    total += (sizes[k] + 255) / 256 * 256;
  }
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (total > ctx->host_stage_cap) {
    e = cudaStreamSynchronize(s);  // the previous staging buffer may still be in use on this stream
    if (e == cudaSuccess) {
      cudaFree(ctx->host_stage);
      ctx->host_stage = nullptr;
      ctx->host_stage_cap = 0;
      e = cudaMalloc(&ctx->host_stage, total);
    }
    if (e != cudaSuccess) return cuda_fail(e, fn);
    ctx->host_stage_cap = total;
  }
  uint8_t* d = ctx->host_stage;
  const void* src[6] = {q, nullptr, alpha, s_off, samples, vel};
  for (int k = 0; k < 6 && e == cudaSuccess; ++k)
    if (src[k] && sizes[k]) e = cudaMemcpyAsync(d + off[k], src[k], sizes[k], cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e, fn);
  const int rc = crom_step(ctx, step, precision, n_inst, reinterpret_cast<double*>(d + off[0]),
                           reinterpret_cast<const float*>(d + off[2]),
                           sizes[5] ? reinterpret_cast<const float*>(d + off[5]) : nullptr,
                           reinterpret_cast<const int*>(d + off[3]), reinterpret_cast<const float*>(d + off[4]),
                           n_samples, max_samples, reinterpret_cast<int*>(d + off[1]), stream);
  if (rc != CROM_OK) {
    cudaStreamSynchronize(s);  // the input copies read the caller's arrays: finish them before returning
    return rc;
  }
  e = cudaMemcpyAsync(q, d + off[0], sizes[0], cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(status, d + off[1], sizes[1], cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, fn);
  return CROM_OK;
}

int crom_rollout(crom_ctx* ctx, const crom_step_desc* step, int precision, int n_steps, int n_inst, double* q,
                 const float* alpha, const float* vel, const int* s_off, const float* samples, int n_samples,
                 int max_samples, int* status, crom_stream stream) {
  if (!ctx || !step) return fail(CROM_ERR_INVALID_ARG, "crom_rollout: null argument");
  if (n_steps < 0) return fail(CROM_ERR_INVALID_ARG, "crom_rollout: n_steps must be >= 0");
  if (n_steps == 0 || n_inst == 0) return CROM_OK;
  // Validate exactly as crom_step does (nothing is launched on failure).
  if (!ctx->has_weights) return fail(CROM_ERR_INVALID_ARG, "crom_rollout: weights not set");
  if (n_inst < 0 || n_samples < 0) return fail(CROM_ERR_INVALID_ARG, "crom_rollout: negative size");
  if (!(step->dt > 0.0) || !isfinite(step->dt)) return fail(CROM_ERR_INVALID_ARG, "crom_rollout: dt must be finite and > 0");
  if (step->gn_iters < 1 || step->gn_iters > 16) return fail(CROM_ERR_INVALID_ARG, "crom_rollout: gn_iters must be in 1..16");
  if (step->pde != CROM_PDE_HEAT && step->pde != CROM_PDE_ADVDIFF) return fail(CROM_ERR_INVALID_ARG, "crom_rollout: unknown pde");
  if (step->coef_per_sample != 0 && step->coef_per_sample != 1)
    return fail(CROM_ERR_INVALID_ARG, "crom_rollout: coef_per_sample must be 0 or 1");
  if (step->line_search < 0 || step->line_search > 16)
    return fail(CROM_ERR_INVALID_ARG, "crom_rollout: line_search must be in 0..16");
  if (step->line_search > 0 && precision != CROM_PREC_F16X2 && precision != CROM_PREC_F16)
    return fail(CROM_ERR_UNSUPPORTED, "crom_rollout: the line search is available with CROM_PREC_F16X2 and CROM_PREC_F16");
  if (!q || !alpha || !s_off || !status || (n_samples > 0 && !samples))
    return fail(CROM_ERR_INVALID_ARG, "crom_rollout: null array");
  if (step->pde == CROM_PDE_ADVDIFF && !vel) return fail(CROM_ERR_INVALID_ARG, "crom_rollout: advection needs vel");
  if (max_samples < 1) return fail(CROM_ERR_INVALID_ARG, "crom_rollout: max_samples must be >= 1");
  if (precision == CROM_PREC_F16X2 || precision == CROM_PREC_F16) {
    if (!tc_shape_ok(ctx->desc) || !ctx->w.tc_img)
      return fail(CROM_ERR_UNSUPPORTED, "crom_rollout: F16X2 and F16 need width 128, 2<=hidden<=5, m<=2, r<=15, ELU");
  } else if (precision != CROM_PREC_FP32) {
    return fail(CROM_ERR_UNSUPPORTED, "crom_rollout: precision not available for the step");
  } else if (step_fp32_max_tiles(ctx, n_inst, max_samples) > 65535) {
    return fail(CROM_ERR_INVALID_ARG, "crom_rollout: max_samples too large for the FP32 step's grid (at most 65535 "
                                      "CTAs per instance)");
  }
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  // The key: every argument that the recorded launches depend on.
  // The key: every argument that the recorded launches depend on, and the
  // generation of the context's weights and scratch (a reallocation by a later
  // crom_step, crom_autotune, crom_robust_samples or crom_set_weights on this
  // context frees the buffers an older recording refers to).
  struct Key {
    int precision, n_steps, n_inst, n_samples, max_samples, pde, gn_iters, coef_per_sample, line_search, tiles;
    double dt;
    const void *q, *alpha, *vel, *s_off, *samples, *status;
    unsigned long long gen;
  };
  auto make_key = [&]() {
    Key key{};
    memset(&key, 0, sizeof(Key));  // padding bytes take part in the comparison
    key.precision = precision;
    key.n_steps = n_steps;
    key.n_inst = n_inst;
    key.n_samples = n_samples;
    key.max_samples = max_samples;
    key.pde = step->pde;
    key.gn_iters = step->gn_iters;
    key.coef_per_sample = step->coef_per_sample;
    key.line_search = step->line_search;
    key.tiles = ctx->tc_tile_s1;
    key.dt = step->dt;
    key.q = q;
    key.alpha = alpha;
    key.vel = vel;
    key.s_off = s_off;
    key.samples = samples;
    key.status = status;
    key.gen = ctx->scratch_gen;
    std::vector<unsigned char> kb(sizeof(Key));
    memcpy(kb.data(), &key, sizeof(Key));
    return kb;
  };
  const std::vector<unsigned char> kb = make_key();
  cudaError_t e;
  if (!ctx->rollout_exec || kb != ctx->rollout_key) {
    if (!ctx->cap_stream) {
      e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking);
      if (e != cudaSuccess) return cuda_fail(e, "crom_rollout (stream)");
    }
    // Make the captured stream wait for the caller's stream is not needed: the
    // recording does not execute anything; relaxed mode lets the first-use
    // scratch growth inside the launch helpers allocate while recording.
    e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return cuda_fail(e, "crom_rollout (begin capture)");
    cudaError_t le = cudaSuccess;
    for (int k = 0; k < n_steps && le == cudaSuccess; ++k) {
      le = (precision == CROM_PREC_FP32)
               ? launch_step_fp32(ctx, step, n_inst, q, alpha, vel, s_off, samples, n_samples, max_samples, status,
                                  ctx->cap_stream)
               : launch_step_tc(ctx, step, precision == CROM_PREC_F16X2, n_inst, q, alpha, vel, s_off, samples,
                                n_samples, max_samples, status, ctx->cap_stream);
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(ctx->cap_stream, &graph);
    if (le != cudaSuccess || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return cuda_fail(le != cudaSuccess ? le : e, "crom_rollout (record)");
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "crom_rollout (instantiate)");
    if (ctx->rollout_exec) cudaGraphExecDestroy(ctx->rollout_exec);
    ctx->rollout_exec = exec;
    // taken after recording: a first use that grew the scratch while recording has
    // bumped the generation, and the recording refers to the new buffers
    ctx->rollout_key = make_key();
  }
  e = cudaGraphLaunch(ctx->rollout_exec, s);
  if (e != cudaSuccess) return cuda_fail(e, "crom_rollout (launch)");
  return CROM_OK;
}

int crom_set_step_tiles(crom_ctx* ctx, int s0, int s1) {
  if (!ctx) return fail(CROM_ERR_INVALID_ARG, "crom_set_step_tiles: null context");
  if (s0 != crom::kTcTileS0 || (s1 != crom::kTcTileS1Large && s1 != crom::kTcTileS1Small))
    return fail(CROM_ERR_UNSUPPORTED, "crom_set_step_tiles: tiles (" + std::to_string(crom::kTcTileS0) + ", " +
                                          std::to_string(crom::kTcTileS1Large) + ") or (" + std::to_string(crom::kTcTileS0) +
                                          ", " + std::to_string(crom::kTcTileS1Small) + ")");
  ctx->tc_tile_s1 = s1;
  return CROM_OK;
}

int crom_get_step_tiles(const crom_ctx* ctx, int* s0, int* s1, float* ms) {
  if (!ctx || !s0 || !s1) return fail(CROM_ERR_INVALID_ARG, "crom_get_step_tiles: null argument");
  *s0 = crom::kTcTileS0;
  *s1 = ctx->tc_tile_s1;
  if (ms) {
    ms[0] = ctx->tune_ms[0];
    ms[1] = ctx->tune_ms[1];
  }
  return CROM_OK;
}

int crom_autotune(crom_ctx* ctx, const crom_step_desc* step, int n_inst, const double* q, const float* alpha,
                  const float* vel, const int* s_off, const float* samples, int n_samples, int max_samples,
                  int* status, crom_stream stream) {
  const char* fn = "crom_autotune";
  if (!ctx || !step || !q) return fail(CROM_ERR_INVALID_ARG, std::string(fn) + ": null argument");
  if (!tc_shape_ok(ctx->desc) || !ctx->w.tc_img)
    return fail(CROM_ERR_UNSUPPORTED, std::string(fn) + ": the tensor-core step needs width 128, 2<=hidden<=5, "
                                                        "m<=2, r<=15, ELU");
  if (n_inst <= 0) return fail(CROM_ERR_INVALID_ARG, std::string(fn) + ": empty batch");
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  DeviceAllocs buf;
  double* qs = buf.get<double>((size_t)n_inst * ctx->desc.r);  // the caller's q is left untouched
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = buf.err;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int variants[2] = {crom::kTcTileS1Large, crom::kTcTileS1Small};
  const int saved = ctx->tc_tile_s1;
  float best_ms = 0.f;
  int best = saved;
  for (int v = 0; v < 2 && e == cudaSuccess; ++v) {
    ctx->tc_tile_s1 = variants[v];
    const size_t qb = (size_t)n_inst * ctx->desc.r * sizeof(double);
    e = cudaMemcpyAsync(qs, q, qb, cudaMemcpyDeviceToDevice, s);
    int rc = CROM_OK;
    if (e == cudaSuccess)  // warm-up (first launch of this variant, shared-memory attribute)
      rc = crom_step(ctx, step, CROM_PREC_F16X2, n_inst, qs, alpha, vel, s_off, samples, n_samples, max_samples,
                     status, stream);
    if (rc != CROM_OK) {
      ctx->tc_tile_s1 = saved;
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return rc;
    }
    const int reps = 5;
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    for (int k = 0; k < reps && e == cudaSuccess; ++k) {
      e = cudaMemcpyAsync(qs, q, qb, cudaMemcpyDeviceToDevice, s);
      if (e == cudaSuccess &&
          crom_step(ctx, step, CROM_PREC_F16X2, n_inst, qs, alpha, vel, s_off, samples, n_samples, max_samples,
                    status, stream) != CROM_OK)
        e = cudaErrorUnknown;
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) {
      ctx->tune_ms[v] = ms / reps;
      if (v == 0 || ms < best_ms) {
        best_ms = ms;
        best = variants[v];
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  ctx->tc_tile_s1 = e == cudaSuccess ? best : saved;
  if (e != cudaSuccess) return cuda_fail(e, fn);
  return CROM_OK;
}

int crom_step_noalloc(crom_ctx* ctx, const crom_step_desc* step, int n_inst, double* q, const float* alpha,
                      const float* vel, const int* s_off, const float* samples, int n_samples, int max_samples,
                      int* status, crom_stream stream) {
  if (!ctx || !step) return fail(CROM_ERR_INVALID_ARG, "crom_step_noalloc: null argument");
  if (!ctx->has_weights) return fail(CROM_ERR_INVALID_ARG, "crom_step_noalloc: weights not set");
  if (n_inst < 0 || n_samples < 0) return fail(CROM_ERR_INVALID_ARG, "crom_step_noalloc: negative size");
  if (!(step->dt > 0.0) || !isfinite(step->dt))
    return fail(CROM_ERR_INVALID_ARG, "crom_step_noalloc: dt must be finite and > 0");
  if (step->gn_iters < 1 || step->gn_iters > 16)
    return fail(CROM_ERR_INVALID_ARG, "crom_step_noalloc: gn_iters must be in 1..16");
  if (step->pde != CROM_PDE_HEAT && step->pde != CROM_PDE_ADVDIFF)
    return fail(CROM_ERR_INVALID_ARG, "crom_step_noalloc: unknown pde");
  if (step->coef_per_sample != 0 && step->coef_per_sample != 1)
    return fail(CROM_ERR_INVALID_ARG, "crom_step_noalloc: coef_per_sample must be 0 or 1");
  if (step->line_search < 0 || step->line_search > 16)
    return fail(CROM_ERR_INVALID_ARG, "crom_step_noalloc: line_search must be in 0..16");
  if (step->line_search > 0)
    return fail(CROM_ERR_UNSUPPORTED, "crom_step_noalloc: the line search is available with CROM_PREC_F16X2");
  if (n_inst == 0) return CROM_OK;
  if (!q || !alpha || !s_off || !status || (n_samples > 0 && !samples))
    return fail(CROM_ERR_INVALID_ARG, "crom_step_noalloc: null array");
  if (step->pde == CROM_PDE_ADVDIFF && !vel)
    return fail(CROM_ERR_INVALID_ARG, "crom_step_noalloc: advection needs vel");
  if (max_samples < 1) return fail(CROM_ERR_INVALID_ARG, "crom_step_noalloc: max_samples must be >= 1");
  if (step_fp32_max_tiles(ctx, n_inst, max_samples) > 65535)
    return fail(CROM_ERR_INVALID_ARG, "crom_step_noalloc: max_samples too large for the FP32 step's grid (at most "
                                      "65535 CTAs per instance)");
  DeviceGuard g(ctx->device);
  size_t need = 0;
  cudaError_t e = launch_step_fp32_noalloc(ctx, step, n_inst, q, alpha, vel, s_off, samples, n_samples,
                                           max_samples, status, (cudaStream_t)stream, &need);
  if (need > noalloc_scratch_capacity())
    return fail(CROM_ERR_INVALID_ARG, "crom_step_noalloc: this batch needs " + std::to_string(need) +
                                          " bytes of scratch, more than the fixed " +
                                          std::to_string(noalloc_scratch_capacity()) +
                                          " bytes; use crom_step or a smaller batch");
  if (e != cudaSuccess) return cuda_fail(e, "crom_step_noalloc");
  return CROM_OK;
}

int crom_fom_step(int kind, int n_batch, int nx, int ny, const float* coef, const float* ax, const float* ay,
                  double dt, int n_steps, float* u, float* tmp, crom_stream stream) {
  if (kind < CROM_FOM_HEAT1D_DIRICHLET || kind > CROM_FOM_ADVDIFF2D_PERIODIC_CENTRAL)
    return fail(CROM_ERR_INVALID_ARG, "crom_fom_step: unknown kind");
  if (n_batch < 0 || n_batch > 65535 || n_steps < 0) return fail(CROM_ERR_INVALID_ARG, "crom_fom_step: bad batch or step count");
  if (nx < 3) return fail(CROM_ERR_INVALID_ARG, "crom_fom_step: nx must be >= 3");
  if ((kind == CROM_FOM_HEAT1D_DIRICHLET || kind == CROM_FOM_HEAT1D_DIRICHLET_FIELD) ? ny != 1 : ny != nx)
    return fail(CROM_ERR_INVALID_ARG, "crom_fom_step: ny must be 1 (1D) or nx (2D)");
  if (!(dt > 0.0) || !isfinite(dt)) return fail(CROM_ERR_INVALID_ARG, "crom_fom_step: dt must be finite and > 0");
  if (n_batch == 0 || n_steps == 0) return CROM_OK;
  if (!coef || !u || !tmp || u == tmp) return fail(CROM_ERR_INVALID_ARG, "crom_fom_step: null or aliased array");
  if ((kind == CROM_FOM_ADVDIFF2D_PERIODIC || kind == CROM_FOM_ADVDIFF2D_PERIODIC_CENTRAL) && (!ax || !ay))
    return fail(CROM_ERR_INVALID_ARG, "crom_fom_step: advection needs ax and ay");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return fail(CROM_ERR_CUDA, "crom_fom_step: no CUDA device");
  cudaError_t e = launch_fom(kind, n_batch, nx, ny, coef, ax, ay, dt, n_steps, u, tmp, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "crom_fom_step");
  return CROM_OK;
}

int crom_trainer_create(crom_trainer** out, const crom_decoder_desc* dec, int P, int B, int S, int device) {
  if (!out || !dec) return fail(CROM_ERR_INVALID_ARG, "crom_trainer_create: null argument");
  *out = nullptr;
  const crom_decoder_desc d = *dec;
  if (d.m < 1 || d.m > 3 || d.r < 1 || d.r > 32 || d.width < 1 || d.width > 1024 || d.hidden < 1 || d.hidden > 8)
    return fail(CROM_ERR_INVALID_ARG, "crom_trainer_create: bad decoder shape");
  if (d.activation != CROM_ACT_ELU)
    return fail(CROM_ERR_UNSUPPORTED, "crom_trainer_create: the training step is built for ELU decoders");
  if (P < 38 || B < 1 || S < 1 || (long long)B * S > (1LL << 26))
    return fail(CROM_ERR_INVALID_ARG, "crom_trainer_create: need P >= 38 (one convolution of length >= 32), "
                                      "B, S >= 1, B*S <= 2^26");
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) return fail(CROM_ERR_CUDA, "crom_trainer_create: no CUDA device");
  if (device < 0 || device >= n) return fail(CROM_ERR_INVALID_ARG, "crom_trainer_create: bad device index");
  crom_trainer* t = new crom_trainer();
  t->device = device;
  t->dec = d;
  t->P = P;
  t->B = B;
  t->S = S;
  t->lens.push_back(P);
  while ((t->lens.back() - 6) / 4 + 1 >= 32) t->lens.push_back((t->lens.back() - 6) / 4 + 1);
  DeviceGuard g(device);
  cudaError_t e = cudaDeviceGetAttribute(&t->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = trainer_alloc(t);
  if (e != cudaSuccess) {
    trainer_free(t);
    delete t;
    return cuda_fail(e, "crom_trainer_create");
  }
  *out = t;
  return CROM_OK;
}

int crom_trainer_destroy(crom_trainer* tr) {
  if (!tr) return CROM_OK;
  {
    DeviceGuard g(tr->device);
    cudaDeviceSynchronize();
    trainer_free(tr);
  }
  delete tr;
  return CROM_OK;
}

// ---- checkpoint / resume of a trainer, and a host-side deadline on a stream

unsigned crom_crc32(const void* data, size_t n) {
  // CRC-32 (IEEE 802.3): reflected polynomial 0xEDB88320, initial value and final
  // xor 0xFFFFFFFF, one bit at a time
  const unsigned char* b = static_cast<const unsigned char*>(data);
  uint32_t c = 0xFFFFFFFFu;
  for (size_t i = 0; i < n; ++i) {
    c ^= b[i];
    for (int k = 0; k < 8; ++k) c = (c >> 1) ^ (0xEDB88320u & (0u - (c & 1u)));
  }
  return c ^ 0xFFFFFFFFu;
}

namespace {
struct CkptHeader {
  char magic[8];  // "CROMCKPT"
  uint32_t version;
  int32_t m, r, width, hidden, activation, P;
  uint64_t n_params;
  int64_t step;
  uint32_t crc;  // of params, first and second Adam moments, in that order
  uint32_t pad;
};
constexpr uint32_t kCkptVersion = 1;

// The trainer's parameters and Adam moments on the host, in file order.
int trainer_state_to_host(crom_trainer* tr, std::vector<float>& buf, const char* fn) {
  const size_t n = trainer_param_count(tr);
  buf.resize(3 * n);
  DeviceGuard g(tr->device);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(buf.data(), tr->params, n * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(buf.data() + n, tr->am, n * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(buf.data() + 2 * n, tr->av, n * 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, fn);
  return CROM_OK;
}
}  // namespace

int crom_trainer_save(crom_trainer* tr, const char* path) {
  const char* fn = "crom_trainer_save";
  if (!tr || !path) return fail(CROM_ERR_INVALID_ARG, std::string(fn) + ": null argument");
  std::vector<float> buf;
  int st = trainer_state_to_host(tr, buf, fn);
  if (st != CROM_OK) return st;
  CkptHeader h{};
  memcpy(h.magic, "CROMCKPT", 8);
  h.version = kCkptVersion;
  h.m = tr->dec.m;
  h.r = tr->dec.r;
  h.width = tr->dec.width;
  h.hidden = tr->dec.hidden;
  h.activation = tr->dec.activation;
  h.P = tr->P;
  h.n_params = trainer_param_count(tr);
  h.step = tr->step;
  h.crc = crom_crc32(buf.data(), buf.size() * 4);
  FILE* f = fopen(path, "wb");
  if (!f) return fail(CROM_ERR_INVALID_ARG, std::string(fn) + ": cannot open " + path);
  const bool ok = fwrite(&h, sizeof(h), 1, f) == 1 && fwrite(buf.data(), 4, buf.size(), f) == buf.size();
  const bool closed = fclose(f) == 0;
  if (!ok || !closed) return fail(CROM_ERR_INVALID_ARG, std::string(fn) + ": write failed for " + path);
  return CROM_OK;
}

int crom_trainer_load(crom_trainer* tr, const char* path) {
  const char* fn = "crom_trainer_load";
  if (!tr || !path) return fail(CROM_ERR_INVALID_ARG, std::string(fn) + ": null argument");
  FILE* f = fopen(path, "rb");
  if (!f) return fail(CROM_ERR_INVALID_ARG, std::string(fn) + ": cannot open " + path);
  CkptHeader h{};
  const size_t n = trainer_param_count(tr);
  std::vector<float> buf;
  bool ok = fread(&h, sizeof(h), 1, f) == 1;
  if (ok && (memcmp(h.magic, "CROMCKPT", 8) != 0 || h.version != kCkptVersion)) {
    fclose(f);
    return fail(CROM_ERR_INVALID_ARG, std::string(fn) + ": not a trainer checkpoint of this version");
  }
  if (ok && (h.m != tr->dec.m || h.r != tr->dec.r || h.width != tr->dec.width || h.hidden != tr->dec.hidden ||
             h.activation != tr->dec.activation || h.P != tr->P || h.n_params != n)) {
    fclose(f);
    return fail(CROM_ERR_INVALID_ARG, std::string(fn) + ": the checkpoint's shapes differ from the trainer's");
  }
  if (ok) {
    buf.resize(3 * n);
    ok = fread(buf.data(), 4, buf.size(), f) == buf.size();
  }
  fclose(f);
  if (!ok) return fail(CROM_ERR_INVALID_ARG, std::string(fn) + ": truncated file " + path);
  if (crom_crc32(buf.data(), buf.size() * 4) != h.crc)
    return fail(CROM_ERR_INVALID_ARG, std::string(fn) + ": checksum mismatch in " + path);
  DeviceGuard g(tr->device);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(tr->params, buf.data(), n * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(tr->am, buf.data() + n, n * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(tr->av, buf.data() + 2 * n, n * 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, fn);
  tr->step = h.step;
  return CROM_OK;
}

int crom_stream_wait(crom_stream stream, double timeout_ms) {
  if (!(timeout_ms >= 0.0)) return fail(CROM_ERR_INVALID_ARG, "crom_stream_wait: timeout must be >= 0");
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t e = cudaStreamQuery((cudaStream_t)stream);
    if (e == cudaSuccess) return CROM_OK;
    if (e != cudaErrorNotReady) return cuda_fail(e, "crom_stream_wait");
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (ms >= timeout_ms) return fail(CROM_ERR_TIMEOUT, "crom_stream_wait: the stream's work did not finish in time");
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

int crom_trainer_set_precision(crom_trainer* tr, int precision) {
  if (!tr) return fail(CROM_ERR_INVALID_ARG, "crom_trainer_set_precision: null trainer");
  if (precision != CROM_PREC_FP32 && precision != CROM_PREC_BF16_MIXED)
    return fail(CROM_ERR_UNSUPPORTED, "crom_trainer_set_precision: FP32 or BF16_MIXED");
  if (precision == CROM_PREC_BF16_MIXED && !trainer_tc_supported(tr))
    return fail(CROM_ERR_UNSUPPORTED, "crom_trainer_set_precision: BF16_MIXED needs width 64, 128 or 256, "
                                      "hidden >= 2 and m + r <= 32");
  DeviceGuard g(tr->device);
  const int rc = trainer_set_precision(tr, precision);
  if (rc != CROM_OK) return fail(rc, "crom_trainer_set_precision: allocation of the tensor-core buffers failed");
  return CROM_OK;
}

int crom_trainer_param_count(const crom_trainer* tr, size_t* n) {
  if (!tr || !n) return fail(CROM_ERR_INVALID_ARG, "crom_trainer_param_count: null argument");
  *n = trainer_param_count(tr);
  return CROM_OK;
}

static int trainer_copy(crom_trainer* tr, float* dev_buf, float* other, size_t n, int on_device, bool to_dev,
                        crom_stream stream, const char* who) {
  if (!tr || !other) return fail(CROM_ERR_INVALID_ARG, std::string(who) + ": null argument");
  if (n != trainer_param_count(tr))
    return fail(CROM_ERR_INVALID_ARG, std::string(who) + ": expected " + std::to_string(trainer_param_count(tr)) +
                                          " floats");
  DeviceGuard g(tr->device);
  cudaStream_t s = (cudaStream_t)stream;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice
                                        : (to_dev ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost);
  cudaError_t e = to_dev ? cudaMemcpyAsync(dev_buf, other, n * 4, kind, s) : cudaMemcpyAsync(other, dev_buf, n * 4, kind, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, who);
  return CROM_OK;
}

int crom_trainer_set_params(crom_trainer* tr, const float* params, size_t n, int on_device, crom_stream stream) {
  int st = trainer_copy(tr, tr ? tr->params : nullptr, const_cast<float*>(params), n, on_device, true, stream,
                        "crom_trainer_set_params");
  if (st != CROM_OK) return st;
  DeviceGuard g(tr->device);
  cudaError_t e = cudaMemset(tr->am, 0, n * 4);
  if (e == cudaSuccess) e = cudaMemset(tr->av, 0, n * 4);
  if (e != cudaSuccess) return cuda_fail(e, "crom_trainer_set_params");
  tr->step = 0;
  return CROM_OK;
}

int crom_trainer_get_params(crom_trainer* tr, float* params, size_t n, int on_device, crom_stream stream) {
  return trainer_copy(tr, tr ? tr->params : nullptr, params, n, on_device, false, stream, "crom_trainer_get_params");
}

int crom_trainer_get_grads(crom_trainer* tr, float* grads, size_t n, int on_device, crom_stream stream) {
  return trainer_copy(tr, tr ? tr->grads : nullptr, grads, n, on_device, false, stream, "crom_trainer_get_grads");
}

int crom_train_step(crom_trainer* tr, const float* snaps, const int* pt_idx, const float* coords, float lr,
                    double* loss_out, crom_stream stream) {
  if (!tr || !snaps || !pt_idx || !coords) return fail(CROM_ERR_INVALID_ARG, "crom_train_step: null argument");
  if (!(lr >= 0.f) || !isfinite(lr)) return fail(CROM_ERR_INVALID_ARG, "crom_train_step: lr must be finite and >= 0");
  DeviceGuard g(tr->device);
  cudaError_t e = trainer_step(tr, snaps, pt_idx, coords, lr, loss_out, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "crom_train_step");
  return CROM_OK;
}

int crom_encode(crom_trainer* tr, int n, const float* snaps, float* q, crom_stream stream) {
  if (!tr || !snaps || !q) return fail(CROM_ERR_INVALID_ARG, "crom_encode: null argument");
  if (n < 0 || n > tr->B) return fail(CROM_ERR_INVALID_ARG, "crom_encode: n must be in 0..B");
  if (n == 0) return CROM_OK;
  DeviceGuard g(tr->device);
  cudaError_t e = trainer_encode(tr, n, snaps, q, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "crom_encode");
  return CROM_OK;
}

int crom_reconstruct(crom_ctx* ctx, int precision, int n_codes, const double* q, int n_pts,
                     const float* x, float* out, crom_stream stream) {
  if (!ctx) return fail(CROM_ERR_INVALID_ARG, "crom_reconstruct: null context");
  if (!ctx->has_weights) return fail(CROM_ERR_INVALID_ARG, "crom_reconstruct: weights not set");
  if (n_codes < 0 || n_pts < 0) return fail(CROM_ERR_INVALID_ARG, "crom_reconstruct: negative size");
  if (n_codes == 0 || n_pts == 0) return CROM_OK;
  if (!q || !x || !out) return fail(CROM_ERR_INVALID_ARG, "crom_reconstruct: null array");
  if (n_codes > 65535) return fail(CROM_ERR_INVALID_ARG, "crom_reconstruct: at most 65535 codes per call");
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (precision == CROM_PREC_FP32) {
    e = launch_recon_fp32(ctx, n_codes, q, n_pts, x, out, s);
  } else if (precision == CROM_PREC_F16X2 || precision == CROM_PREC_F16) {
    if (!tc_shape_ok(ctx->desc) || !ctx->w.tc_img)
      return fail(CROM_ERR_UNSUPPORTED, "crom_reconstruct: tensor-core path needs width 128, 2<=hidden<=5, m<=2, ELU");
    e = launch_recon_tc(ctx, precision == CROM_PREC_F16X2 ? 1 : 0, n_codes, q, n_pts, x, out, s);
  } else {
    return fail(CROM_ERR_UNSUPPORTED, "crom_reconstruct: unknown precision");
  }
  if (e != cudaSuccess) return cuda_fail(e, "crom_reconstruct");
  return CROM_OK;
}

int crom_robust_samples(crom_ctx* ctx, const crom_step_desc* step, int precision, int n_params, const double* q0,
                        const float* coef, int n_steps, int n_nodes, const float* nodes, const float* fom_final,
                        int n_init, const int* init_idx, int n_try, double target, int max_samples, int* idx_out,
                        int* count_out, double* metric_out, crom_stream stream) {
  const char* fn = "crom_robust_samples";
  if (!ctx || !step || !init_idx || !idx_out || !count_out || !metric_out)
    return fail(CROM_ERR_INVALID_ARG, std::string(fn) + ": null argument");
  if (!ctx->has_weights) return fail(CROM_ERR_INVALID_ARG, std::string(fn) + ": weights not set");
  if (!q0 || !coef || !nodes || !fom_final) return fail(CROM_ERR_INVALID_ARG, std::string(fn) + ": null array");
  if (n_params < 1 || n_steps < 0 || n_nodes < 1 || n_init < 0 || n_try < 1 || n_try > 64 || max_samples < n_init ||
      max_samples > 4096 || max_samples > n_nodes || (size_t)n_try * n_params > 65535 || !(target >= 0.0))
    return fail(CROM_ERR_INVALID_ARG, std::string(fn) + ": bad sizes (n_params, n_nodes >= 1; 1 <= n_try <= 64; "
                                                        "n_init <= max_samples <= min(n_nodes, 4096); target >= 0)");
  if (step->pde != CROM_PDE_HEAT || step->line_search < 0 || step->line_search > 16 || step->gn_iters < 1 ||
      step->gn_iters > 16 || !(step->dt > 0.0) || !isfinite(step->dt) ||
      (step->coef_per_sample != 0 && step->coef_per_sample != 1))
    return fail(CROM_ERR_INVALID_ARG, std::string(fn) + ": needs a heat step with valid gn_iters, dt, coefficient mode");
  if (precision == CROM_PREC_F16X2) {
    if (!tc_shape_ok(ctx->desc) || !ctx->w.tc_img)
      return fail(CROM_ERR_UNSUPPORTED, std::string(fn) + ": F16X2 needs width 128, 2<=hidden<=5, m<=2, r<=15");
  } else if (precision != CROM_PREC_FP32 || step->line_search > 0) {
    return fail(CROM_ERR_UNSUPPORTED, std::string(fn) + ": precision FP32 (no line search) or F16X2");
  }
  std::vector<int> M(init_idx, init_idx + n_init);
  {
    std::vector<char> seen(n_nodes, 0);
    for (int i : M) {
      if (i < 0 || i >= n_nodes || seen[i]) return fail(CROM_ERR_INVALID_ARG, std::string(fn) + ": bad initial index");
      seen[i] = 1;
    }
  }
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int m = ctx->desc.m, r = ctx->desc.r;
  const int max_inst = n_try * n_params;
  const size_t max_samp = (size_t)max_inst * max_samples;
  // Work buffers for one batch of candidate sets (freed on every exit path).
  DeviceAllocs buf;
  int* d_idx = buf.get<int>(max_samp);
  int* d_param = buf.get<int>(max_samp);
  float* d_samples = buf.get<float>(max_samp * m);
  float* d_alpha_s = buf.get<float>(max_samp);
  int* d_off = buf.get<int>(max_inst + 1);
  double* d_q = buf.get<double>((size_t)max_inst * r);
  float* d_alpha = buf.get<float>(max_inst);
  int* d_status = buf.get<int>(max_inst);
  float* d_out = buf.get<float>((size_t)max_inst * n_nodes);
  double* d_res = buf.get<double>((size_t)(n_try + 1) * n_nodes);
  double* d_metric = buf.get<double>(n_try);
  int* d_taken = buf.get<int>(n_nodes);
  int* d_cand = buf.get<int>(n_try);
  if (buf.err != cudaSuccess) return cuda_fail(buf.err, fn);
  crom_step_desc sd = *step;

  // Metric of each candidate set (sets[c] = M plus extra[c], extra -1 = none);
  // their residual rows land in d_res rows 0..C-1.
  auto evaluate = [&](const std::vector<int>& extra, std::vector<double>& metrics) -> cudaError_t {
    const int C = (int)extra.size(), n_inst = C * n_params;
    std::vector<int> h_idx, h_param, h_off(1, 0);
    int max_s = 1;
    for (int c = 0; c < C; ++c)
      for (int mu = 0; mu < n_params; ++mu) {
        for (int i : M) { h_idx.push_back(i); h_param.push_back(mu); }
        if (extra[c] >= 0) { h_idx.push_back(extra[c]); h_param.push_back(mu); }
        h_off.push_back((int)h_idx.size());
        max_s = std::max(max_s, h_off.back() - h_off[h_off.size() - 2]);
      }
    const int n_s = (int)h_idx.size();
    cudaError_t e = cudaMemcpyAsync(d_idx, h_idx.data(), (size_t)n_s * sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_param, h_param.data(), (size_t)n_s * sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_off, h_off.data(), h_off.size() * sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = launch_sampling_gather(nodes, d_idx, d_param, n_s, m, n_nodes, sd.coef_per_sample ? coef : nullptr,
                                 d_samples, d_alpha_s, s);
    if (e == cudaSuccess)
      e = launch_sampling_replicate(q0, sd.coef_per_sample ? nullptr : coef, n_params, n_inst, r, d_q, d_alpha, s);
    const float* a = sd.coef_per_sample ? d_alpha_s : d_alpha;
    if (e == cudaSuccess && n_steps == 0) e = cudaMemsetAsync(d_status, 0, (size_t)n_inst * sizeof(int), s);
    for (int t = 0; t < n_steps && e == cudaSuccess; ++t)
      e = precision != CROM_PREC_FP32
              ? launch_step_tc(ctx, &sd, precision == CROM_PREC_F16X2, n_inst, d_q, a, nullptr, d_off, d_samples, n_s,
                               max_s, d_status, s)
              : launch_step_fp32(ctx, &sd, n_inst, d_q, a, nullptr, d_off, d_samples, n_s, max_s, d_status, s);
    if (e == cudaSuccess) e = launch_recon_fp32(ctx, n_inst, d_q, n_nodes, nodes, d_out, s);
    if (e == cudaSuccess) e = launch_sampling_metric(d_out, fom_final, d_status, C, n_params, n_nodes, d_res, d_metric, s);
    metrics.assign(C, 0.0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(metrics.data(), d_metric, C * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
  };

  std::vector<double> met;
  cudaError_t e = evaluate(std::vector<int>{-1}, met);
  if (e != cudaSuccess) return cuda_fail(e, fn);
  double cur = met[0];
  // d_res row 0 holds the residual of M; the candidates' rows go after it.
  while (!(cur < target) && (int)M.size() < max_samples) {
    std::vector<char> taken(n_nodes, 0);
    for (int i : M) taken[i] = 1;
    std::vector<int> h_taken(taken.begin(), taken.end());
    e = cudaMemcpyAsync(d_taken, h_taken.data(), (size_t)n_nodes * sizeof(int), cudaMemcpyHostToDevice, s);
    const int k = std::min(n_try, n_nodes - (int)M.size());
    if (e == cudaSuccess) e = launch_sampling_topk(d_res, d_taken, n_nodes, k, d_cand, s);
    std::vector<int> cand(k, -1);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cand.data(), d_cand, k * sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, fn);
    cand.erase(std::remove(cand.begin(), cand.end(), -1), cand.end());
    if (cand.empty()) break;
    // candidates' residual rows 1..k: shift the batch by one row
    double* base_res = d_res;
    d_res = base_res + n_nodes;
    e = evaluate(cand, met);
    d_res = base_res;
    if (e != cudaSuccess) return cuda_fail(e, fn);
    int best = 0;
    for (int c = 1; c < (int)cand.size(); ++c)
      if (met[c] < met[best]) best = c;
    M.push_back(cand[best]);
    cur = met[best];
    e = cudaMemcpyAsync(d_res, d_res + (size_t)(1 + best) * n_nodes, (size_t)n_nodes * sizeof(double),
                        cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, fn);
  }
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, fn);
  std::copy(M.begin(), M.end(), idx_out);
  *count_out = (int)M.size();
  *metric_out = cur;
  return CROM_OK;
}

}  // extern "C"
