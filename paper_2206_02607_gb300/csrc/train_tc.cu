// Decoder part of the training step on the tcgen05 tensor cores (paper §3, Eq. loss;
// App. D), precision CROM_PREC_BF16_MIXED: bf16 weights, activations and deltas
// in HBM, FP32 accumulation in tensor memory, FP32 master weights (the parameter
// vector) and Adam.
//
// With hidden layers h = 0..L-1 (H[h] = ELU(z_h), z_0 = W_0 [x; q] + b_0,
// z_h = W_h H[h-1] + b_h), output g = w_out . H[L-1] + b_out and
// loss = mean (g - f)^2 over the B*S sampled points:
//   forward:  H[0] on the CUDA cores (K = m + r is too short for the tensor cores);
//             H[h] = ELU(H[h-1] W_h^T + b_h) by the GEMM's bias + ELU epilogue;
//             the last layer's epilogue also forms g, the residual, dL/dg and
//             delta[L-1] = dL/dg w_out s'(z_{L-1}), with the column sums that give
//             the gradients of w_out, b_out and b_{L-1};
//   backward: for h = L-1 .. 1: dW_h = delta[h]^T H[h-1] (K = B*S, split over CTAs,
//             the splits added in a fixed order) and delta[h-1] = (delta[h] W_h) s'(z_{h-1})
//             with its column sums (db_{h-1}); then dW_0 = delta[0]^T [x; q] on the
//             CUDA cores and din = delta[0] W_0 (GEMM, N padded to 64) for the encoder.
// s'(z) is taken from h = ELU(z): 1 where h > 0, else h + 1 = e^z.  Every reduction
// runs in a fixed order, so a step is deterministic.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>

#include "crom_internal.h"

namespace crom {
namespace {

constexpr int kSplitsW = 64;      // K splits of the weight-gradient GEMMs
constexpr int kGw0Chunks = 512;   // row chunks of the input-layer weight gradient
constexpr int kDinCols = 64;      // din = delta[0] W_0 padded to 64 columns

inline unsigned nblk(long n, int t) { return (unsigned)((n + t - 1) / t); }

__device__ __forceinline__ uint16_t bf16_bits(float f) {
  __nv_bfloat16 h = __float2bfloat16_rn(f);
  return *reinterpret_cast<uint16_t*>(&h);
}
__device__ __forceinline__ float bf16_val(uint16_t u) { return __uint_as_float((uint32_t)u << 16); }

// bf16 copies of the hidden matrices W_1..W_{L-1} ([w][w] each) and of W_0 transposed
// into a [w][64] block (row u holds W_0[u][0..m+r), zeros after).
__global__ void weights_bf16_kernel(const float* params, const long* off_w, int L, int w, int kin, uint16_t* wh,
                                    uint16_t* w0p) {
  const long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  const long per = (long)w * w;
  if (e < (long)(L - 1) * per) {
    const int h = 1 + (int)(e / per);
    wh[e] = bf16_bits(params[off_w[h] + e % per]);
  }
  if (e < (long)w * kDinCols) {
    const int u = (int)(e / kDinCols), j = (int)(e % kDinCols);
    w0p[e] = bf16_bits(j < kin ? params[off_w[0] + (long)u * kin + j] : 0.f);
  }
}

// H[0][n][u] = ELU(W_0[u] . in[n] + b_0[u]) in bf16: one thread per unit, 32 rows per
// block (the rows' inputs staged in shared memory); the K = m + r <= 32 loops are
// unrolled to their bound and predicated, so W_0's row stays in registers.
constexpr int kRows0 = 32;
__global__ void layer0_fwd_kernel(const float* in, long N, int kin, const float* W0, const float* b0, int w,
                                  uint16_t* H) {
  __shared__ float xs[kRows0][33];
  const int u = threadIdx.x;
  const long n0 = (long)blockIdx.x * kRows0;
  for (int i = threadIdx.x; i < kRows0 * 32; i += blockDim.x) {
    const long n = n0 + i / 32;
    const int j = i % 32;
    xs[i / 32][j] = (n < N && j < kin) ? in[n * kin + j] : 0.f;   // zeros beyond kin
  }
  __syncthreads();
  if (u >= w) return;
  float wr[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) wr[j] = j < kin ? W0[(long)u * kin + j] : 0.f;
  const float b = b0[u];
  for (int i = 0; i < kRows0; ++i) {
    const long n = n0 + i;
    if (n >= N) break;
    float z = b;
#pragma unroll
    for (int j = 0; j < 32; ++j) z = fmaf(wr[j], xs[i][j], z);
    H[n * w + u] = bf16_bits(z > 0.f ? z : expm1f(z));
  }
}

// dW_0 partials: part[c][u][j] = sum over the rows of chunk c of delta[n][u] in[n][j]
// (loops over j unrolled to 32 and predicated: the accumulators stay in registers).
__global__ void gw0_part_kernel(const uint16_t* delta, const float* in, long N, int kin, int w, float* part) {
  __shared__ float xs[64][33];
  const int u = threadIdx.x;
  const long per = (N + gridDim.x - 1) / gridDim.x;
  const long r0 = (long)blockIdx.x * per, r1 = (r0 + per < N ? r0 + per : N);
  float acc[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) acc[j] = 0.f;
  for (long b = r0; b < r1; b += 64) {
    const int nr = (int)(r1 - b < 64 ? r1 - b : 64);
    __syncthreads();
    for (int i = threadIdx.x; i < 64 * 32; i += blockDim.x) {
      const int row = i / 32, j = i % 32;
      xs[row][j] = (row < nr && j < kin) ? in[(b + row) * kin + j] : 0.f;
    }
    __syncthreads();
    if (u < w)
      for (int i = 0; i < nr; ++i) {
        const float d = bf16_val(delta[(b + i) * w + u]);
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j] = fmaf(d, xs[i][j], acc[j]);
      }
  }
  if (u < w)
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (j < kin) part[((long)blockIdx.x * w + u) * kin + j] = acc[j];
}

// out[e] = sum_p part[p * stride + e], in order of p (FP64 accumulation).
__global__ void sum_parts_kernel(const float* part, int nparts, long stride, long n, float* out) {
  const long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (e >= n) return;
  double s = 0.0;
  for (int p = 0; p < nparts; ++p) s += part[(long)p * stride + e];
  out[e] = (float)s;
}

// Column sums of part [nparts][cols] in a fixed order, first level: block (x, y)
// adds parts y * kColPer .. of columns 32 x .. (32 columns x 8 part lanes, the lanes
// combined in order) into mid[y][col].  The second level adds mid's rows in order
// (sum_parts_kernel).
constexpr int kColPer = 128;
__global__ void colsum_level1_kernel(const float* part, int nparts, int cols, float* mid) {
  __shared__ double red[8][32];
  const int col = blockIdx.x * 32 + threadIdx.x;
  const int p0 = blockIdx.y * kColPer, p1 = min(nparts, p0 + kColPer);
  double acc = 0.0;
  if (col < cols)
    for (int p = p0 + threadIdx.y; p < p1; p += 8) acc += part[(long)p * cols + col];
  red[threadIdx.y][threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.y == 0 && col < cols) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += red[k][threadIdx.x];
    mid[(long)blockIdx.y * cols + col] = (float)t;
  }
}

// loss = sum_p rowpart[p][0] * inv_count; gb_out = sum_p rowpart[p][1] (in order).
__global__ void loss_parts_kernel(const float* rowpart, int nparts, double inv_count, double* loss, float* gbout) {
  __shared__ double red[2][256];
  double a = 0.0, b = 0.0;
  const int per = (nparts + 255) / 256;
  for (int p = threadIdx.x * per; p < min(nparts, (int)(threadIdx.x + 1) * per); ++p) {
    a += rowpart[2 * p];
    b += rowpart[2 * p + 1];
  }
  red[0][threadIdx.x] = a;
  red[1][threadIdx.x] = b;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      red[0][threadIdx.x] += red[0][threadIdx.x + o];
      red[1][threadIdx.x] += red[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *loss = red[0][0] * inv_count;
    *gbout = (float)red[1][0];
  }
}

// out[c] = sum over the parts of part[p][c] (deterministic two-level sum through mid)
void colsum_parts(const float* part, int nparts, int cols, float* mid, float* out, cudaStream_t s) {
  const int chunks = (nparts + kColPer - 1) / kColPer;
  colsum_level1_kernel<<<dim3((cols + 31) / 32, chunks), dim3(32, 8), 0, s>>>(part, nparts, cols, mid);
  sum_parts_kernel<<<nblk(cols, 256), 256, 0, s>>>(mid, chunks, cols, cols, out);
}

}  // namespace

bool trainer_tc_supported(const crom_trainer* t) {
  return tc_gemm_supported(t->dec.width) && t->dec.hidden >= 2 && t->dec.m + t->dec.r <= 32;
}

cudaError_t trainer_tc_alloc(crom_trainer* t) {
  if (t->tc.ready) return cudaSuccess;
  const int w = t->dec.width, L = t->dec.hidden, kin = t->dec.m + t->dec.r;
  const long N = (long)t->B * t->S;
  const long tiles_m = (N + 127) / 128;
  auto A = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes > 0 ? bytes : 16) != cudaSuccess) p = nullptr;
    t->owned.push_back(p);
    return p;
  };
  auto& c = t->tc;
  c.wh = (uint16_t*)A((size_t)(L - 1) * w * w * 2);
  c.w0p = (uint16_t*)A((size_t)w * kDinCols * 2);
  for (int h = 0; h < L; ++h) c.H.push_back((uint16_t*)A((size_t)N * w * 2));
  c.d0 = (uint16_t*)A((size_t)N * w * 2);
  c.d1 = (uint16_t*)A((size_t)N * w * 2);
  c.colpart = (float*)A((size_t)tiles_m * 4 * w * 4);
  c.colpart2 = (float*)A((size_t)tiles_m * 4 * w * 4);
  c.rowpart = (float*)A((size_t)tiles_m * 4 * 2 * 4);
  c.colmid = (float*)A((size_t)std::max<long>((tiles_m * 4 + kColPer - 1) / kColPer * w,
                                              (long)(kGw0Chunks + kColPer - 1) / kColPer * w * kin) * 4);
  c.split = (float*)A((size_t)kSplitsW * w * w * 4);
  c.din = (float*)A((size_t)N * kDinCols * 4);
  c.gw0part = (float*)A((size_t)kGw0Chunks * w * kin * 4);
  c.off_w = (long*)A((size_t)(L + 1) * sizeof(long));
  c.flag = (int*)A(sizeof(int));
  for (void* p : t->owned)
    if (!p) return cudaErrorMemoryAllocation;
  cudaError_t e = cudaMemcpy(c.off_w, t->lay.dec_w.data(), (size_t)(L + 1) * sizeof(long), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(c.flag, 0, sizeof(int));
  if (e == cudaSuccess) c.ready = true;
  return e;
}

cudaError_t trainer_decoder_tc(crom_trainer* t, double* loss_out, int num_sms, cudaStream_t s) {
  const int w = t->dec.width, L = t->dec.hidden, kin = t->dec.m + t->dec.r;
  const long N = (long)t->B * t->S;
  const int tiles_m = (int)((N + 127) / 128);
  const int parts = tiles_m * 4;
  auto& c = t->tc;
  const TrainerLayout& lay = t->lay;
  const float* p = t->params;
  float* gr = t->grads;
  cudaError_t e;
  weights_bf16_kernel<<<nblk(std::max<long>((long)(L - 1) * w * w, (long)w * kDinCols), 256), 256, 0, s>>>(
      p, c.off_w, L, w, kin, c.wh, c.w0p);
  // ---- forward
  layer0_fwd_kernel<<<nblk(N, kRows0), std::max(w, 64), 0, s>>>(t->in0, N, kin, p + lay.dec_w[0], p + lay.dec_b[0], w,
                                                          c.H[0]);
  for (int h = 1; h < L; ++h) {
    TcGemm g;
    g.M = (int)N;
    g.N = w;
    g.K = w;
    g.A = c.H[h - 1];
    g.lda = w;
    g.B = c.wh + (size_t)(h - 1) * w * w;  // B(n, k) = W_h[n][k]
    g.ldb = w;
    g.ldo = w;
    g.out_bf16 = c.H[h];
    g.bias = p + lay.dec_b[h];
    if (h < L - 1) {
      g.epi = kGemmEpiBiasElu;
    } else {
      g.epi = kGemmEpiOut;
      g.wout = p + lay.dec_w[L];
      g.bout = p + lay.dec_b[L];
      g.target = t->target;
      g.delta_out = c.d0;
      g.colpart = c.colpart;
      g.colpart2 = c.colpart2;
      g.rowpart = c.rowpart;
      g.inv_count = (float)(1.0 / (double)N);
    }
    if ((e = tc_gemm(g, num_sms, c.flag, s)) != cudaSuccess) return e;
  }
  loss_parts_kernel<<<1, 256, 0, s>>>(c.rowpart, parts, 1.0 / (double)N, loss_out ? loss_out : t->loss_dev,
                                      gr + lay.dec_b[L]);
  colsum_parts(c.colpart2, parts, w, c.colmid, gr + lay.dec_w[L], s);   // dL/dw_out
  colsum_parts(c.colpart, parts, w, c.colmid, gr + lay.dec_b[L - 1], s);
  // ---- backward
  uint16_t* dcur = c.d0;
  uint16_t* dnext = c.d1;
  for (int h = L - 1; h >= 1; --h) {
    {  // dW_h = delta[h]^T H[h-1]: A(u, n) = delta[n][u], B(k, n) = H[h-1][n][k]
      TcGemm g;
      g.M = w;
      g.N = w;
      g.K = (int)N;
      g.A = dcur;
      g.lda = w;
      g.a_mn = 1;
      g.B = c.H[h - 1];
      g.ldb = w;
      g.b_mn = 1;
      g.splits = kSplitsW;
      g.epi = kGemmEpiF32;
      g.out_f32 = c.split;
      g.ldo = w;
      if ((e = tc_gemm(g, num_sms, c.flag, s)) != cudaSuccess) return e;
      const int sp = tc_gemm_splits_used((int)N, kSplitsW);
      sum_parts_kernel<<<nblk((long)w * w, 256), 256, 0, s>>>(c.split, sp, (long)w * w, (long)w * w,
                                                             gr + lay.dec_w[h]);
    }
    {  // delta[h-1] = (delta[h] W_h) s'(z_{h-1}): A(n, u) = delta[n][u], B(k, u) = W_h[u][k]
      TcGemm g;
      g.M = (int)N;
      g.N = w;
      g.K = w;
      g.A = dcur;
      g.lda = w;
      g.B = c.wh + (size_t)(h - 1) * w * w;
      g.ldb = w;
      g.b_mn = 1;
      g.epi = kGemmEpiTimesEluD;
      g.out_bf16 = dnext;
      g.ldo = w;
      g.hprev = c.H[h - 1];
      g.colpart = c.colpart;
      if ((e = tc_gemm(g, num_sms, c.flag, s)) != cudaSuccess) return e;
      colsum_parts(c.colpart, parts, w, c.colmid, gr + lay.dec_b[h - 1], s);
    }
    std::swap(dcur, dnext);
  }
  // ---- input layer: dW_0 on the CUDA cores, din = delta[0] W_0 on the tensor cores
  gw0_part_kernel<<<kGw0Chunks, std::max(w, 64), 0, s>>>(dcur, t->in0, N, kin, w, c.gw0part);
  colsum_parts(c.gw0part, kGw0Chunks, w * kin, c.colmid, gr + lay.dec_w[0], s);
  TcGemm g;
  g.M = (int)N;
  g.N = kDinCols;
  g.K = w;
  g.A = dcur;
  g.lda = w;
  g.B = c.w0p;  // B(j, u) = W_0[u][j] stored [u][64]
  g.ldb = kDinCols;
  g.b_mn = 1;
  g.epi = kGemmEpiF32;
  g.out_f32 = c.din;
  g.ldo = kDinCols;
  if ((e = tc_gemm(g, num_sms, c.flag, s)) != cudaSuccess) return e;
  return cudaGetLastError();
}

int trainer_tc_din_ld() { return kDinCols; }

}  // namespace crom
