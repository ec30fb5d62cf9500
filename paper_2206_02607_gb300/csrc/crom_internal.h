// Internal declarations shared by the C-ABI layer and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/crom.h"

namespace crom {

// Tensor-core decoder image (f16), one per context.  Layout in bytes, every
// part 1024-byte aligned so that it can be bulk-copied into shared memory and
// used there directly as 128B-swizzled UMMA operands:
//   [0, L*32768)           hidden matrices W_2..W_{hidden}, each 128x128 f16,
//                          K-major, 128B swizzle, two 64-column k-blocks
//   [L*32768, +4096)       projection matrix P (16 x 128 f16, K-major, SW128):
//                          row 0 = w_out, rows 1..r = W_1[:, m+j] (dg/dq projection)
//   [L*32768+4096, +4096)  output operand O of the f16 reconstruction (same
//                          layout): row 0 = f16(v), row 1 = f16(v - f16(v)) for
//                          v = ln 2 * w_out (its activations carry a log2 e factor)
//   [L*32768+8192, +16384) bias operand of the f16 reconstruction: 128 x 64 f16,
//                          K-major, SW128; columns 16 l and 16 l + 1 hold the high
//                          and low f16 parts of log2 e * b_l for hidden matrix l
// (tc_img_bytes counts the first two parts, which the step loads), and a second image of the hidden matrices' low parts W - f16(W), rounded to f16,
// row-major [L][128][128] (loaded into tensor memory by the reconstruction kernel,
// where it is the A operand of a third product per layer).
constexpr int kTcWidth = 128;
constexpr int kTcLayerBytes = kTcWidth * kTcWidth * 2;
// Sample tiles of the tensor-core step: kTcTileS0 samples per forward tile at GN
// iteration 0 (two of them share one reverse pass); kTcTileS1Large or
// kTcTileS1Small samples per tile at later iterations.
constexpr int kTcTileS0 = 8;
constexpr int kTcTileS1Large = 16;
constexpr int kTcTileS1Small = 8;
constexpr int kTcProjRows = 16;
constexpr int kTcProjBytes = kTcProjRows * kTcWidth * 2;
constexpr int kTcBiasBytes = kTcWidth * 64 * 2;

struct DeviceWeights {
  // FP32 copies for the CUDA-core path.
  float* w1 = nullptr;    // [width][m+r] row-major
  float* b1 = nullptr;    // [width]
  float* wt = nullptr;    // (hidden-1) x [width(in)][width(out)]: transposed hidden matrices
  float* bh = nullptr;    // (hidden-1) x [width]
  float* wout = nullptr;  // [width]
  float bout = 0.f;
  // f16 tensor-core images (see above); nullptr when the shape is not supported
  // by the tensor-core kernels or a weight lies outside the f16 range.
  uint8_t* tc_img = nullptr;
  size_t tc_img_bytes = 0;
  uint8_t* tc_lo = nullptr;
  size_t tc_lo_bytes = 0;
  // Power-of-two scales of the step's f16 channels: max_u |W_1x[u][k]| * tc_sx and
  // max_u |w_out[u]| * tc_sr lie in [1, 2).
  float tc_sx = 1.f, tc_sr = 1.f;
};

}  // namespace crom

struct crom_ctx {
  int device = 0;
  int num_sms = 0;
  crom_decoder_desc desc{};
  bool has_weights = false;
  crom::DeviceWeights w;
  // Scratch of the FP32 multi-CTA step (grown on demand, never shrunk).
  double* partials = nullptr;  // [n_inst][max_tiles][n_entries]
  size_t partials_cap = 0;     // in doubles
  int* counters = nullptr;     // [n_inst], zero between launches
  size_t counters_cap = 0;
  double* targets = nullptr;   // [n_samples]: Delta f_j (FP64) from GN iteration 0
  size_t targets_cap = 0;
  double* qbase = nullptr;     // [n_inst][r]: q_n kept for the difference channel
  size_t qbase_cap = 0;
  float* tangent = nullptr;    // [n_inst][width]: layer-1 seeds W_1q qdot_i of the tangent velocity
  size_t tangent_cap = 0;
  uint8_t* host_stage = nullptr;  // crom_step_host: device copies of the caller's host arrays
  size_t host_stage_cap = 0;
  // Scratch of the tensor-core step: instance order (largest |M_i| first) and the
  // queue counter / timeout flag.
  int* order = nullptr;
  size_t order_cap = 0;
  int* queue = nullptr;
  // Sample-tile shape of the tensor-core step for GN iterations >= 1
  // (kTcTileS1Large or kTcTileS1Small), set by crom_set_step_tiles or measured by
  // crom_autotune; the timings of the last crom_autotune per variant (ms, < 0 = not
  // measured).
  int tc_tile_s1 = crom::kTcTileS1Large;
  float tune_ms[2] = {-1.f, -1.f};
  // Bumped whenever a device buffer that a recorded launch refers to (weights or
  // step scratch) is freed and reallocated: part of the rollout graph's key, so a
  // graph recorded before the change is never replayed against freed memory.
  unsigned long long scratch_gen = 0;
  // Cached rollout graph and the arguments it was recorded with.
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t rollout_exec = nullptr;
  std::vector<unsigned char> rollout_key;
};

namespace crom {
struct TrainerLayout {
  std::vector<long> dec_w, dec_b;  // offsets of W_l, b_l (l = 0..hidden) in the parameter vector
  std::vector<long> conv;          // offsets of convolution l (w[6], b)
  long d1w = 0, d1b = 0, d2w = 0, d2b = 0;
  long total = 0;
};
}  // namespace crom

namespace crom {
// Buffers of the tensor-core decoder pass of training (CROM_PREC_BF16_MIXED),
// allocated when that precision is first selected.
struct TrainerTc {
  bool ready = false;
  uint16_t* wh = nullptr;   // bf16 hidden matrices W_1..W_{L-1}, [w][w] each
  std::vector<uint16_t*> H; // bf16 activations of the hidden layers, [B*S][w] each
  uint16_t *d0 = nullptr, *d1 = nullptr;  // bf16 deltas [B*S][w]
  float *colpart = nullptr, *colpart2 = nullptr, *rowpart = nullptr;  // per-32-row partial sums
  float* resid = nullptr;   // [B*S]: g - f per point (FP32)
  float* colmid = nullptr;  // first level of the column-sum reduction
  float* split = nullptr;   // split-K partials of the weight gradients
  float* xin = nullptr;     // [B*S][m]: the sampled points' coordinates
  float* c0 = nullptr;      // [B][w]: b_0 + W_0q q_b, the latent part of layer 0 per snapshot
  float* part0 = nullptr;   // [B][chunks][w][1 + m]: row-chunk moments of delta_0
  float* snap0 = nullptr;   // [B][w][1 + m]: per-snapshot moments of delta_0
  long* off_w = nullptr;    // device copy of the decoder weight offsets
  int* flag = nullptr;      // set by a GEMM whose bounded wait ran out
};
}  // namespace crom

// Training state: FP32 master parameters, gradients, Adam moments, activations.
struct crom_trainer {
  int device = 0;
  crom_decoder_desc dec{};
  int P = 0, B = 0, S = 0;
  std::vector<int> lens;  // convolution lengths: P, ..., L_last
  crom::TrainerLayout lay;
  float *params = nullptr, *grads = nullptr, *am = nullptr, *av = nullptr;
  long step = 0;
  std::vector<float*> conv_z, conv_h;  // per convolution: [B][L_l]
  float *d1z = nullptr, *d1h = nullptr, *q = nullptr;
  float *in0 = nullptr, *target = nullptr, *g = nullptr, *dg = nullptr;
  std::vector<float*> Z, H;  // per hidden layer: [B*S][width]
  float *delta = nullptr, *delta2 = nullptr, *din = nullptr, *dq = nullptr;
  float* split = nullptr;  // split-K partial sums of weight gradients
  float *edh = nullptr, *edx = nullptr, *ed1 = nullptr;
  double* partial = nullptr;
  double* loss_dev = nullptr;
  double* red = nullptr;  // partial sums of the deterministic column / convolution reductions
  double* colpart = nullptr;  // per-block column partial sums fused into the TF32 epilogues
  std::vector<void*> owned;
  int precision = CROM_PREC_FP32;  // of the decoder pass (FP32 or BF16_MIXED)
  int num_sms = 0;
  crom::TrainerTc tc;
};

namespace crom {

void set_error(const std::string& msg);

// Training (train.cu).
size_t trainer_param_count(const crom_trainer* t);
cudaError_t trainer_alloc(crom_trainer* t);
void trainer_free(crom_trainer* t);
int trainer_set_precision(crom_trainer* t, int precision);
cudaError_t trainer_encode(crom_trainer* t, int nb, const float* snaps, float* q_out, cudaStream_t s);
cudaError_t trainer_step(crom_trainer* t, const float* snaps, const int* pt_idx, const float* coords, float lr,
                         double* loss_out, cudaStream_t s);
// tensor-core decoder pass (train_tc.cu): loss, decoder gradients and the latent
// codes' gradient t->dq ([B][r]) from t->tc.xin, t->q and t->target
bool trainer_tc_supported(const crom_trainer* t);
cudaError_t trainer_tc_alloc(crom_trainer* t);
cudaError_t trainer_decoder_tc(crom_trainer* t, double* loss_out, int num_sms, cudaStream_t s);

// Channel configuration of the FP32 forward-mode evaluation.
enum SecondOrder { kSecondNone = 0, kSecondPerK = 1, kSecondLap = 2 };

struct ChannelSet {
  int nx;      // number of dg/dx_k channels carried (0 or m)
  int second;  // SecondOrder
  int nq;      // number of dg/dq_j channels carried (0 or r)
  int count(int m) const { return 1 + nx + (second == kSecondPerK ? m : (second == kSecondLap ? 1 : 0)) + nq; }
};

// FP32 CUDA-core launches (simt_fp32.cu).
cudaError_t launch_decode_fp32(const crom_ctx* ctx, int n_inst, const double* q, const int* pt_off,
                               const float* x, int n_pts, unsigned want, float* out, cudaStream_t s);
cudaError_t launch_recon_fp32(const crom_ctx* ctx, int n_codes, const double* q, int n_pts,
                              const float* x, float* out, cudaStream_t s);
cudaError_t launch_step_fp32(crom_ctx* ctx, const crom_step_desc* step, int n_inst, double* q,
                             const float* alpha, const float* vel, const int* s_off,
                             const float* samples, int n_samples, int max_samples, int* status,
                             cudaStream_t s);
// Second grid dimension (CTAs per instance) of the FP32 step for a batch; the
// launch needs it <= 65535.
int step_fp32_max_tiles(const crom_ctx* ctx, int n_inst, int max_samples);

// v_p = (dg/dq)(x_p, q_i) . (q_i - q_prev_i) / dt from dq [r][n_pts] (decode output).
cudaError_t launch_tangent_fp32(const crom_ctx* ctx, int n_inst, const double* q, const double* q_prev, double dt,
                                const int* pt_off, const float* x, int n_pts, float* seed, float* out,
                                cudaStream_t s);

// FP32 step with its scratch in a fixed-size device array (no allocation).
size_t noalloc_scratch_capacity();
cudaError_t launch_step_fp32_noalloc(const crom_ctx* ctx, const crom_step_desc* step, int n_inst, double* q,
                                     const float* alpha, const float* vel, const int* s_off,
                                     const float* samples, int n_samples, int max_samples, int* status,
                                     cudaStream_t s, size_t* need_bytes);

// Full-order model stencils (fom.cu).
cudaError_t launch_fom(int kind, int n_batch, int nx, int ny, const float* coef, const float* ax, const float* ay,
                       double dt, int n_steps, float* u, float* tmp, cudaStream_t s);

// Tensor-core launches (tc_step.cu, tc_recon.cu).
// lo_parts: 1 for F16X2 (activations as f16 hi + lo parts), 0 for F16 (hi parts only)
cudaError_t launch_step_tc(crom_ctx* ctx, const crom_step_desc* step, int lo_parts, int n_inst, double* q,
                           const float* alpha, const float* vel, const int* s_off,
                           const float* samples, int n_samples, int max_samples, int* status,
                           cudaStream_t s);
// Step 1 alone on the tensor cores (tc_step.cu, the step kernel's decode mode):
// want ⊆ VAL | DX | LAP | DQ, out as crom_decode without the DXX rows.
cudaError_t launch_decode_tc(crom_ctx* ctx, int lo_parts, int n_inst, const double* q, const int* pt_off,
                             const float* x, int n_pts, unsigned want, float* out, cudaStream_t s);
cudaError_t launch_recon_tc(const crom_ctx* ctx, int split, int n_codes, const double* q, int n_pts,
                            const float* x, float* out, cudaStream_t s);

// bf16 GEMM on the tcgen05 tensor cores with fused training epilogues (tc_gemm.cu):
// D[m][n] = sum_k A(m, k) B(n, k), FP32 accumulation.  A(m, k) = A[m * lda + k]
// (a_mn = 0) or A[k * lda + m] (a_mn = 1); B(n, k) = B[n * ldb + k] (b_mn = 0) or
// B[k * ldb + n] (b_mn = 1); bf16 operands, 16-byte aligned, row strides multiples of
// 8 elements; N in {64, 128, 256} (one tile spans all N columns), M and K any.
enum GemmEpi {
  kGemmEpiF32 = 0,        // out_f32[split][m][n] = D (K split into `splits` ranges)
  kGemmEpiBiasElu = 1,    // out_bf16[m][n] = ELU(D + bias[n])
  kGemmEpiTimesEluD = 2,  // out_bf16[m][n] = D * s'(z), s' from hprev[m][n] = h = ELU(z); colpart = column sums
  kGemmEpiOut = 3         // last hidden layer: out_bf16 = h_L = ELU(D + bias); per row the residual
                          // resid[m] = wout . h_L + *bout - target[m] (FP32 from the FP32 h_L)
};
struct TcGemm {
  int M = 0, N = 0, K = 0;
  const void* A = nullptr;
  long lda = 0;
  int a_mn = 0;
  const void* B = nullptr;
  long ldb = 0;
  int b_mn = 0;
  int splits = 1;
  int epi = kGemmEpiF32;
  float* out_f32 = nullptr;
  long ldo = 0;
  uint16_t* out_bf16 = nullptr;
  const float* bias = nullptr;
  const uint16_t* hprev = nullptr;
  float* colpart = nullptr;  // [ceil(M / 128) * 4][N]: per-warp column sums (32 rows each)
  const float* wout = nullptr;
  const float* bout = nullptr;  // device scalar
  const float* target = nullptr;
  float* resid = nullptr;  // [M]
};
bool tc_gemm_supported(int n);
cudaError_t tc_gemm(const TcGemm& g, int num_sms, int* flag, cudaStream_t s);
int tc_gemm_splits_used(int K, int splits);

// Robust-sample selection kernels (sampling.cu).
cudaError_t launch_sampling_gather(const float* nodes, const int* idx, const int* param_of, int n, int m,
                                   int n_nodes, const float* coef_nodes, float* samples, float* alpha_s,
                                   cudaStream_t s);
cudaError_t launch_sampling_replicate(const double* q0, const float* coef, int n_params, int n_inst, int r,
                                      double* q, float* alpha, cudaStream_t s);
cudaError_t launch_sampling_metric(const float* out, const float* fom, const int* status, int n_cand, int n_params,
                                   int n_nodes, double* res, double* metric, cudaStream_t s);
cudaError_t launch_sampling_topk(const double* res, int* taken, int n_nodes, int k, int* out, cudaStream_t s);

}  // namespace crom
