// C-ABI entry points (include/crom.h): argument checks, context and weight
// management, dispatch to the FP32 CUDA-core and the tcgen05 kernels.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cstdio>
#include <string>
#include <vector>

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

uint16_t f32_to_bf16(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7fffffffu) > 0x7f800000u) return 0x7fc0;  // NaN stays NaN
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
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
  auto& w = ctx->w;
  cudaFree(w.w1);
  cudaFree(w.b1);
  cudaFree(w.wt);
  cudaFree(w.bh);
  cudaFree(w.wout);
  cudaFree(w.tc_img);
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

bool tc_shape_ok(const crom_decoder_desc& d) {
  return d.width == kTcWidth && d.hidden >= 2 && d.hidden <= 5 && d.m >= 1 && d.m <= 2 &&
         d.r >= 1 && d.r <= kTcProjRows - 1;
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
  const crom_decoder_desc d = *desc;
  if (d.m < 1 || d.m > 3 || d.r < 1 || d.r > 32 || d.width < 32 || d.width > 256 ||
      d.width % 32 != 0 || d.hidden < 1 || d.hidden > 8)
    return fail(CROM_ERR_INVALID_ARG,
                "crom_create: need 1<=m<=3, 1<=r<=32, width%32==0 in [32,256], 1<=hidden<=8");
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
    cudaFree(ctx->order);
    cudaFree(ctx->queue);
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

  if (tc_shape_ok(d)) {
    // bf16 image: hidden matrices (K-major SW128), then the projection matrix P.
    const size_t layers_bytes = (size_t)(L - 1) * kTcLayerBytes;
    std::vector<uint8_t> img(layers_bytes + kTcProjBytes, 0);
    for (int l = 0; l < L - 1; ++l)
      for (int o = 0; o < w; ++o)
        for (int k = 0; k < w; ++k) {
          uint16_t v = f32_to_bf16(hidden_w[l][(size_t)o * w + k]);
          memcpy(&img[(size_t)l * kTcLayerBytes + kmajor_sw128(o, k, w)], &v, 2);
        }
    for (int row = 0; row < kTcProjRows; ++row)
      for (int k = 0; k < w; ++k) {
        float val = 0.f;
        if (row == 0) val = Wout[k];
        else if (row <= r) val = W1[(size_t)k * in + m + (row - 1)];
        uint16_t v = f32_to_bf16(val);
        memcpy(&img[layers_bytes + kmajor_sw128(row, k, kTcProjRows)], &v, 2);
      }
    e = cudaMalloc(&dw.tc_img, img.size());
    if (e == cudaSuccess) e = cudaMemcpy(dw.tc_img, img.data(), img.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      free_weights(ctx);
      return cuda_fail(e, "crom_set_weights (tensor-core image)");
    }
    dw.tc_img_bytes = img.size();
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

int crom_step(crom_ctx* ctx, const crom_step_desc* step, int precision, int n_inst, double* q,
              const float* alpha, const float* vel, const int* s_off, const float* samples,
              int n_samples, int max_samples, int* status, crom_stream stream) {
  if (!ctx || !step) return fail(CROM_ERR_INVALID_ARG, "crom_step: null argument");
  if (!ctx->has_weights) return fail(CROM_ERR_INVALID_ARG, "crom_step: weights not set");
  if (n_inst < 0 || n_samples < 0) return fail(CROM_ERR_INVALID_ARG, "crom_step: negative size");
  if (!(step->dt > 0.0) || !isfinite(step->dt)) return fail(CROM_ERR_INVALID_ARG, "crom_step: dt must be finite and > 0");
  if (step->gn_iters < 1 || step->gn_iters > 16) return fail(CROM_ERR_INVALID_ARG, "crom_step: gn_iters must be in 1..16");
  if (step->pde != CROM_PDE_HEAT && step->pde != CROM_PDE_ADVDIFF) return fail(CROM_ERR_INVALID_ARG, "crom_step: unknown pde");
  if (n_inst == 0) return CROM_OK;
  if (!q || !alpha || !s_off || !status || (n_samples > 0 && !samples))
    return fail(CROM_ERR_INVALID_ARG, "crom_step: null array");
  if (step->pde == CROM_PDE_ADVDIFF && !vel) return fail(CROM_ERR_INVALID_ARG, "crom_step: advection needs vel");
  if (max_samples < 1) return fail(CROM_ERR_INVALID_ARG, "crom_step: max_samples must be >= 1");
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (precision == CROM_PREC_FP32) {
    e = launch_step_fp32(ctx, step, n_inst, q, alpha, vel, s_off, samples, n_samples, max_samples, status, s);
  } else if (precision == CROM_PREC_BF16X2) {
    if (!tc_shape_ok(ctx->desc) || !ctx->w.tc_img)
      return fail(CROM_ERR_UNSUPPORTED, "crom_step: BF16X2 needs width 128, 2<=hidden<=5, m<=2, r<=15");
    e = launch_step_tc(ctx, step, n_inst, q, alpha, vel, s_off, samples, n_samples, max_samples, status, s);
  } else {
    return fail(CROM_ERR_UNSUPPORTED, "crom_step: precision not available for the step");
  }
  if (e != cudaSuccess) return cuda_fail(e, "crom_step");
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
  if (n_inst == 0) return CROM_OK;
  if (!q || !alpha || !s_off || !status || (n_samples > 0 && !samples))
    return fail(CROM_ERR_INVALID_ARG, "crom_step_noalloc: null array");
  if (step->pde == CROM_PDE_ADVDIFF && !vel)
    return fail(CROM_ERR_INVALID_ARG, "crom_step_noalloc: advection needs vel");
  if (max_samples < 1) return fail(CROM_ERR_INVALID_ARG, "crom_step_noalloc: max_samples must be >= 1");
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
  } else if (precision == CROM_PREC_BF16X2 || precision == CROM_PREC_BF16) {
    if (!tc_shape_ok(ctx->desc) || !ctx->w.tc_img)
      return fail(CROM_ERR_UNSUPPORTED, "crom_reconstruct: tensor-core path needs width 128, 2<=hidden<=5, m<=2");
    e = launch_recon_tc(ctx, precision == CROM_PREC_BF16X2 ? 1 : 0, n_codes, q, n_pts, x, out, s);
  } else {
    return fail(CROM_ERR_UNSUPPORTED, "crom_reconstruct: unknown precision");
  }
  if (e != cudaSuccess) return cuda_fail(e, "crom_reconstruct");
  return CROM_OK;
}

}  // extern "C"
