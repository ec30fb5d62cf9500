// One training step of the CROM manifold (paper §3, Eq. loss; App. D): strided
// 1D-convolution encoder + MLP decoder, MSE over sampled points, hand-written
// reverse pass and Adam with FP32 master weights.
//
// Encoder (App. D): convolutions of kernel 6, stride 4, one channel, no padding,
// ELU after each, repeated while the output length stays >= 32; then a dense
// layer to 32 (ELU) and a linear layer to r.  Decoder: g(x, q) with the layer
// sizes of the crom_decoder_desc.  Loss: mean over the B x S sampled points of
// (g(x_j, e(f_b)) - f_b(x_j))^2.  Adam with beta1 = 0.9, beta2 = 0.999, eps = 1e-8.
//
// Parameter vector (FP32, also the layout of crom_trainer_get/set_params):
// decoder layers as in crom_set_weights (W row-major, then b), then for each
// convolution w[6], b, then the dense layers (W [32][L_last], b[32]),
// (W [r][32], b[r]).
//
// The decoder pass runs either here in FP32 (one tiled FP32 GEMM with strided
// operands and fused epilogues, bias + ELU and multiply by s'(z); weight gradients
// reduce over the B*S points with a fixed split along K and a second pass that adds
// the splits in order, so a step is deterministic) or, with CROM_PREC_BF16_MIXED, on
// the tensor cores (train_tc.cu).  The encoder, the latent gradient and Adam are
// shared.
#include <math.h>

#include <vector>

#include "crom_internal.h"

namespace crom {
namespace {

constexpr int kTile = 64;
constexpr int kTK = 16;
constexpr int kSplitK = 32;

__device__ __forceinline__ float elu_f(float z) { return z > 0.f ? z : expm1f(z); }
__device__ __forceinline__ float elu_d(float z) { return z > 0.f ? 1.f : expf(z); }

// Compensated (Kahan) FP32 accumulation: the running sum s - c stays within a few
// ulps of the exact sum whatever the number of terms, in FP32 instructions (FP64 is
// a slow pipe on this GPU: per-element FP64 adds made these reductions FP64-bound).
struct CompSum {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float y = __fsub_rn(v, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

enum Epi { kEpiStore = 0, kEpiBiasElu = 1, kEpiTimesEluD = 2 };

// C[i][j] = sum_k A(i, k) B(k, j), A(i, k) = A[i*sai + k*sak], B(k, j) = B[k*sbk + j*sbj].
// Epilogues: kEpiStore (C row-major, ldc); kEpiBiasElu (Z = C + bias[j] stored in C,
// ELU(Z) stored in H); kEpiTimesEluD (C *= s'(Zp[i][j])).  blockIdx.z splits K into
// gridDim.z contiguous ranges writing to C + z * split_stride (kEpiStore only).
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, const float* __restrict__ A, long sai,
                                                   long sak, const float* __restrict__ B, long sbk, long sbj,
                                                   float* __restrict__ C, long ldc, long split_stride, int epi,
                                                   const float* __restrict__ bias, float* __restrict__ H,
                                                   const float* __restrict__ Zp) {
  __shared__ float As[kTK][kTile + 4];
  __shared__ float Bs[kTK][kTile + 4];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int i0 = blockIdx.y * kTile, j0 = blockIdx.x * kTile;
  const int splits = gridDim.z;
  const int kchunk = ((K + splits - 1) / splits + kTK - 1) / kTK * kTK;
  const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
  float acc[4][4] = {};
  for (int k0 = kbeg; k0 < kend; k0 += kTK) {
    for (int e = threadIdx.x; e < kTK * kTile; e += 256) {
      const int kk = e / kTile, ii = e % kTile;
      const int k = k0 + kk;
      As[kk][ii] = (i0 + ii < M && k < kend) ? A[(long)(i0 + ii) * sai + (long)k * sak] : 0.f;
      Bs[kk][ii] = (j0 + ii < N && k < kend) ? B[(long)k * sbk + (long)(j0 + ii) * sbj] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kTK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        a[t] = As[kk][ty + 16 * t];
        b[t] = Bs[kk][tx + 16 * t];
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(a[p], b[q], acc[p][q]);
    }
    __syncthreads();
  }
  float* Cz = C + (long)blockIdx.z * split_stride;
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int i = i0 + ty + 16 * p;
    if (i >= M) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = j0 + tx + 16 * q;
      if (j >= N) continue;
      float v = acc[p][q];
      const long o = (long)i * ldc + j;
      if (epi == kEpiBiasElu) {
        v += bias[j];
        Cz[o] = v;
        H[o] = elu_f(v);
      } else if (epi == kEpiTimesEluD) {
        Cz[o] = v * elu_d(Zp[o]);
      } else {
        Cz[o] = v;
      }
    }
  }
}

// out[e] = sum_s parts[s * stride + e] (in split order), then optionally out[e] = val.
__global__ void sum_splits_kernel(const float* parts, int splits, long stride, long n, float* out) {
  const long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (e >= n) return;
  float s = 0.f;
  for (int k = 0; k < splits; ++k) s += parts[k * stride + e];
  out[e] = s;
}

// Column sums of X [rows][cols] in fixed order: out[c] = sum_r X[r][c] (one block per column).
// Column sums of X [rows][cols] in two fixed-order passes (deterministic):

// colsum_part_kernel: block (32 columns x 8 row lanes) per (column group, row chunk),
// coalesced across columns; colsum_final_kernel adds the chunk partials in order.
constexpr int kColChunks = 128;
__global__ void colsum_part_kernel(const float* X, long rows, int cols, double* part) {
  const int c = blockIdx.x * 32 + threadIdx.x;
  const long per = (rows + gridDim.y - 1) / gridDim.y;
  const long r0 = (long)blockIdx.y * per, r1 = min(rows, r0 + per);
  CompSum s;
  if (c < cols)
    for (long r = r0 + threadIdx.y; r < r1; r += 8) s.add(X[r * cols + c]);
  __shared__ double red[8][33];
  red[threadIdx.y][threadIdx.x] = s.value();
  __syncthreads();
  if (threadIdx.y == 0 && c < cols) {
    double t = 0.0;
    for (int y = 0; y < 8; ++y) t += red[y][threadIdx.x];
    part[(long)blockIdx.y * cols + c] = t;
  }
}
// Column sums four columns at a time (cols % 4 == 0): block (64 column quads x 4
// row lanes) per (column-quad group, row chunk).
__global__ void colsum_part4_kernel(const float* X, long rows, int cols, double* part) {
  const int q = blockIdx.x * 64 + threadIdx.x, cols4 = cols / 4;
  const long per = (rows + gridDim.y - 1) / gridDim.y;
  const long r0 = (long)blockIdx.y * per, r1 = min(rows, r0 + per);
  CompSum s0, s1, s2, s3;
  if (q < cols4)
    for (long r = r0 + threadIdx.y; r < r1; r += 4) {
      const float4 v = reinterpret_cast<const float4*>(X + r * cols)[q];
      s0.add(v.x);
      s1.add(v.y);
      s2.add(v.z);
      s3.add(v.w);
    }
  __shared__ double red[4][64][4];
  red[threadIdx.y][threadIdx.x][0] = s0.value();
  red[threadIdx.y][threadIdx.x][1] = s1.value();
  red[threadIdx.y][threadIdx.x][2] = s2.value();
  red[threadIdx.y][threadIdx.x][3] = s3.value();
  __syncthreads();
  if (threadIdx.y == 0 && q < cols4)
    for (int e = 0; e < 4; ++e)
      part[(long)blockIdx.y * cols + 4 * q + e] =
          (red[0][threadIdx.x][e] + red[1][threadIdx.x][e]) + (red[2][threadIdx.x][e] + red[3][threadIdx.x][e]);
}
// Sum over the 32 lanes by a fixed butterfly (every lane ends with the same value).
__device__ __forceinline__ double warp_sum_fixed(double t) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double u = __shfl_xor_sync(0xffffffffu, t, o);
    t = (threadIdx.x & o) ? u + t : t + u;  // the lower lane's value first on both lanes
  }
  return t;
}
// out[c] = sum of the chunks' partials of column c: one warp per column, lanes take
// every 32nd chunk, then a fixed butterfly.
__global__ void colsum_final_kernel(const double* part, int chunks, int cols, float* out) {
  const int c = (int)((blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= cols) return;  // whole warps leave together
  double t = 0.0;
  for (int k = lane; k < chunks; k += 32) t += part[(long)k * cols + c];
  t = warp_sum_fixed(t);
  if (lane == 0) out[c] = (float)t;
}

__global__ void conv_fwd_kernel(const float* x, int Lin, int Lout, int B, const float* w, float* z, float* h) {
  const long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (e >= (long)B * Lout) return;
  const int b = (int)(e / Lout), i = (int)(e % Lout);
  const float* xb = x + (long)b * Lin + 4 * i;
  float s = w[6];
  for (int k = 0; k < 6; ++k) s = fmaf(w[k], xb[k], s);
  z[e] = s;
  h[e] = elu_f(s);
}

// Backward of one convolution: dz = dh * s'(z) (in place into dz), input gradient
// dx[b][j] = sum over i with 0 <= j - 4i < 6 of w[j - 4i] dz[b][i].
__global__ void conv_dz_kernel(const float* dh, const float* z, long n, float* dz) {
  const long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (e < n) dz[e] = dh[e] * elu_d(z[e]);
}
__global__ void conv_dx_kernel(const float* dz, int Lin, int Lout, int B, const float* w, float* dx) {
  const long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (e >= (long)B * Lin) return;
  const int b = (int)(e / Lin), j = (int)(e % Lin);
  float s = 0.f;
  int ihi = j / 4;
  if (ihi > Lout - 1) ihi = Lout - 1;
  for (int i = ihi; i >= 0 && j - 4 * i < 6; --i) s = fmaf(w[j - 4 * i], dz[(long)b * Lout + i], s);
  dx[e] = s;
}
// Parameter gradients of one convolution: gw[k] = sum_{b,i} dz[b][i] x[b][4i+k], gb = sum dz.
// Gradient of one convolution's 6 weights and bias: sums over B * Lout outputs,
// split into gridDim.y fixed chunks (partials part[chunk][7]) and added in order.
__global__ void conv_grad_part_kernel(const float* dz, const float* x, int Lin, int Lout, int B, double* part) {
  const int k = blockIdx.x;  // 0..6 (6 = bias)
  const long n = (long)B * Lout;
  const long per = (n + gridDim.y - 1) / gridDim.y;
  const long e0 = (long)blockIdx.y * per, e1 = min(n, e0 + per);
  // products split exactly into p + err (one FMA), the p summed with compensation
  CompSum s;
  float err = 0.f;
  for (long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const int b = (int)(e / Lout), i = (int)(e % Lout);
    const float a = dz[e], xv = k < 6 ? x[(long)b * Lin + 4 * i + k] : 1.f;
    const float p = __fmul_rn(a, xv);
    err += fmaf(a, xv, -p);
    s.add(p);
  }
  __shared__ double red[256];
  red[threadIdx.x] = s.value() + (double)err;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(long)blockIdx.y * 7 + k] = red[0];
}
// gw[k] = sum over the chunks of part[chunk][k]: warp k, lanes take every 32nd chunk.
__global__ void conv_grad_final_kernel(const double* part, int chunks, float* gw) {
  const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (k >= 7) return;
  double t = 0.0;
  for (int c = lane; c < chunks; c += 32) t += part[(long)c * 7 + k];
  t = warp_sum_fixed(t);
  if (lane == 0) gw[k] = (float)t;
}

__global__ void gather_kernel(const float* snaps, const int* pt_idx, const float* coords, const float* q, int B,
                              int S, int P, int m, int r, float* in, float* target) {
  const long n = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (n >= (long)B * S) return;
  const int b = (int)(n / S);
  const int node = pt_idx[n];
  const int ld = m + r;
  for (int k = 0; k < m; ++k) in[n * ld + k] = coords[(long)node * m + k];
  for (int j = 0; j < r; ++j) in[n * ld + m + j] = q[(long)b * r + j];
  target[n] = snaps[(long)b * P + node];
}
// The tensor-core pass's inputs: the points' coordinates x [B*S][m] (the latent part
// of the input layer is formed per snapshot) and the targets.
__global__ void gather_x_kernel(const float* snaps, const int* pt_idx, const float* coords, int B, int S, int P,
                                int m, float* x, float* target) {
  const long n = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (n >= (long)B * S) return;
  const int b = (int)(n / S);
  const int node = pt_idx[n];
  for (int k = 0; k < m; ++k) x[n * m + k] = coords[(long)node * m + k];
  target[n] = snaps[(long)b * P + node];
}

// Output layer g = w_out . h + b_out, residual and dL/dg = 2 (g - t) / N; per-block
// partial sums of the squared residual (FP64).
__global__ void output_loss_kernel(const float* H, int w, long N, const float* wout, const float* bout,
                                   const float* target, float* dg, double* partial) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const long n = blockIdx.x * 8L + warp;
  double sq = 0.0;
  if (n < N) {
    float s = 0.f;
    for (int u = lane; u < w; u += 32) s = fmaf(wout[u], H[n * w + u], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const float res = s + bout[0] - target[n];
    if (lane == 0) {
      dg[n] = 2.f * res / (float)N;
      sq = (double)res * (double)res;
    }
  }
  __shared__ double red[8];
  if (lane == 0) red[warp] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < 8; ++i) s += red[i];
    partial[blockIdx.x] = s;
  }
}
// loss = sum(partial) / N: 1024 threads, strided partial sums, fixed tree.
__global__ void loss_final_kernel(const double* partial, int n, long N, double* loss) {
  __shared__ double red[1024];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = red[0] / (double)N;
}
// delta_L[n][u] = dL/dg_n w_out[u] s'(z_L[n][u]).
__global__ void out_delta_kernel(const float* dg, const float* wout, const float* Z, int w, long N, float* delta) {
  const long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (e >= N * w) return;
  const long n = e / w;
  const int u = (int)(e % w);
  delta[e] = dg[n] * wout[u] * elu_d(Z[e]);
}
// The same, four units per thread (w % 4 == 0, N * w / 4 < 2^31, 16-byte aligned):
// quad e covers row e / (w / 4), units 4 (e % (w / 4)) ..
__global__ void out_delta4_kernel(const float* dg, const float* wout, const float* Z, int w, unsigned n_quads,
                                  float* delta) {
  const unsigned e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_quads) return;
  const unsigned q = (unsigned)w / 4;
  const long n = e / q;
  const int u = 4 * (int)(e % q);
  const float d = dg[n];
  const float4 z = *reinterpret_cast<const float4*>(Z + n * w + u);
  const float4 wo = *reinterpret_cast<const float4*>(wout + u);
  *reinterpret_cast<float4*>(delta + n * w + u) =
      make_float4(d * wo.x * elu_d(z.x), d * wo.y * elu_d(z.y), d * wo.z * elu_d(z.z), d * wo.w * elu_d(z.w));
}

// dq[b][j] = sum_s din[b S + s][m + j] (din rows ld floats apart): one block per
// (snapshot, latent component), 256 row lanes with compensated sums, fixed-order tree.
__global__ void dq_kernel(const float* din, int ld, int B, int S, int m, int r, float* dq) {
  const int b = blockIdx.x, j = blockIdx.y;
  __shared__ double red[256];
  CompSum s;
  for (int i = threadIdx.x; i < S; i += blockDim.x) s.add(din[((long)b * S + i) * ld + m + j]);
  red[threadIdx.x] = s.value();
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) dq[(long)b * r + j] = (float)red[0];
}
__global__ void adam_kernel(float* p, const float* g, float* m, float* v, long n, float lr, float c1, float c2) {
  const long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (e >= n) return;
  const float gi = g[e];
  const float mi = 0.9f * m[e] + 0.1f * gi;
  const float vi = 0.999f * v[e] + 0.001f * gi * gi;
  m[e] = mi;
  v[e] = vi;
  p[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

inline unsigned blocks(long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

size_t trainer_param_count(const crom_trainer* t) { return (size_t)t->lay.total; }

cudaError_t trainer_alloc(crom_trainer* t) {
  auto A = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes > 0 ? bytes : 16) != cudaSuccess) p = nullptr;
    t->owned.push_back(p);  // a failed allocation leaves a nullptr here for the check below
    return p;
  };
  const int m = t->dec.m, r = t->dec.r, w = t->dec.width, L = t->dec.hidden;
  const long N = (long)t->B * t->S;
  // parameter layout
  TrainerLayout& lay = t->lay;
  long o = 0;
  std::vector<int> dims = {m + r};
  for (int l = 0; l < L; ++l) dims.push_back(w);
  dims.push_back(1);
  for (int l = 0; l + 1 < (int)dims.size(); ++l) {
    lay.dec_w.push_back(o);
    o += (long)dims[l + 1] * dims[l];
    lay.dec_b.push_back(o);
    o += dims[l + 1];
  }
  for (size_t c = 1; c < t->lens.size(); ++c) {
    lay.conv.push_back(o);
    o += 7;
  }
  const int Llast = t->lens.back();
  lay.d1w = o; o += 32L * Llast;
  lay.d1b = o; o += 32;
  lay.d2w = o; o += (long)r * 32;
  lay.d2b = o; o += r;
  lay.total = o;
  t->params = (float*)A(o * 4);
  t->grads = (float*)A(o * 4);
  t->am = (float*)A(o * 4);
  t->av = (float*)A(o * 4);
  for (size_t c = 1; c < t->lens.size(); ++c) {
    t->conv_z.push_back((float*)A((size_t)t->B * t->lens[c] * 4));
    t->conv_h.push_back((float*)A((size_t)t->B * t->lens[c] * 4));
  }
  t->d1z = (float*)A((size_t)t->B * 32 * 4);
  t->d1h = (float*)A((size_t)t->B * 32 * 4);
  t->q = (float*)A((size_t)t->B * r * 4);
  t->in0 = (float*)A((size_t)N * (m + r) * 4);
  t->target = (float*)A((size_t)N * 4);
  t->g = (float*)A((size_t)N * 4);
  t->dg = (float*)A((size_t)N * 4);
  for (int l = 0; l < L; ++l) {
    t->Z.push_back((float*)A((size_t)N * w * 4));
    t->H.push_back((float*)A((size_t)N * w * 4));
  }
  t->delta = (float*)A((size_t)N * w * 4);
  t->delta2 = (float*)A((size_t)N * w * 4);
  t->din = (float*)A((size_t)N * (m + r) * 4);
  t->dq = (float*)A((size_t)t->B * r * 4);
  t->split = (float*)A((size_t)kSplitK * w * std::max(w, m + r) * 4);
  t->edh = (float*)A((size_t)t->B * t->lens[0] * 4);
  t->edx = (float*)A((size_t)t->B * t->lens[0] * 4);
  t->ed1 = (float*)A((size_t)t->B * 32 * 4);
  t->partial = (double*)A((size_t)blocks(N, 8) * 8);
  t->loss_dev = (double*)A(8);
  t->red = (double*)A((size_t)kColChunks * std::max(std::max(w, 32), std::max(r, 7)) * 8);
  for (void* p : t->owned)
    if (!p) return cudaErrorMemoryAllocation;
  cudaError_t e = cudaMemset(t->am, 0, o * 4);
  if (e == cudaSuccess) e = cudaMemset(t->av, 0, o * 4);
  return e;
}

void trainer_free(crom_trainer* t) {
  for (void* p : t->owned) cudaFree(p);
  t->owned.clear();
  t->tc = TrainerTc{};
}

// C = A * B (strided operands) with an epilogue; K split over kSplitK partials when requested.
// A[i][k] = A[i * sai + k * sak], B[k][j] = B[k * sbk + j * sbj]; one of each pair of
// strides is 1 (row-major or transposed storage).
static cudaError_t gemm(crom_trainer* t, cudaStream_t s, int M, int N, int K, const float* A, long sai, long sak,
                        const float* B, long sbk, long sbj, float* C, long ldc, int epi, const float* bias,
                        float* H, const float* Zp, float* split = nullptr) {
  (void)t;
  dim3 grid(blocks(N, kTile), blocks(M, kTile), split ? kSplitK : 1);
  if (split) {
    gemm_kernel<<<grid, 256, 0, s>>>(M, N, K, A, sai, sak, B, sbk, sbj, split, ldc, (long)M * ldc, kEpiStore,
                                     nullptr, nullptr, nullptr);
    sum_splits_kernel<<<blocks((long)M * ldc, 256), 256, 0, s>>>(split, kSplitK, (long)M * ldc, (long)M * ldc, C);
  } else {
    gemm_kernel<<<grid, 256, 0, s>>>(M, N, K, A, sai, sak, B, sbk, sbj, C, ldc, 0, epi, bias, H, Zp);
  }
  return cudaGetLastError();
}

// Deterministic column sums (two passes through t->red).
static void colsum(crom_trainer* t, cudaStream_t s, const float* X, long rows, int cols, float* out) {
  const int chunks = (int)std::min<long>(kColChunks, std::max<long>(rows, 1));
  if (cols % 4 == 0 && ((uintptr_t)X & 15) == 0)
    colsum_part4_kernel<<<dim3(blocks(cols / 4, 64), chunks), dim3(64, 4), 0, s>>>(X, rows, cols, t->red);
  else
    colsum_part_kernel<<<dim3(blocks(cols, 32), chunks), dim3(32, 8), 0, s>>>(X, rows, cols, t->red);
  colsum_final_kernel<<<blocks(32L * cols, 128), 128, 0, s>>>(t->red, chunks, cols, out);
}

int trainer_set_precision(crom_trainer* t, int precision) {
  if (precision == CROM_PREC_BF16_MIXED && trainer_tc_alloc(t) != cudaSuccess) return CROM_ERR_CUDA;
  t->precision = precision;
  return CROM_OK;
}

cudaError_t trainer_encode(crom_trainer* t, int nb, const float* snaps, float* q_out, cudaStream_t s) {
  // nb <= B; forward through the encoder only
  const int r = t->dec.r;
  const float* x = snaps;
  for (size_t c = 1; c < t->lens.size(); ++c) {
    const int Lin = t->lens[c - 1], Lout = t->lens[c];
    conv_fwd_kernel<<<blocks((long)nb * Lout, 256), 256, 0, s>>>(x, Lin, Lout, nb, t->params + t->lay.conv[c - 1],
                                                                t->conv_z[c - 1], t->conv_h[c - 1]);
    x = t->conv_h[c - 1];
  }
  const int Ll = t->lens.back();
  cudaError_t e = gemm(t, s, nb, 32, Ll, x, Ll, 1, t->params + t->lay.d1w, 1, Ll, t->d1z, 32, kEpiBiasElu,
                       t->params + t->lay.d1b, t->d1h, nullptr);
  if (e != cudaSuccess) return e;
  // q = W2 h1 + b2: the bias + ELU epilogue leaves Z = q in C (its ELU is discarded
  // into the ed1 scratch)
  return gemm(t, s, nb, r, 32, t->d1h, 32, 1, t->params + t->lay.d2w, 1, 32, q_out, r, kEpiBiasElu,
              t->params + t->lay.d2b, t->ed1, nullptr);
}

cudaError_t trainer_step(crom_trainer* t, const float* snaps, const int* pt_idx, const float* coords, float lr,
                         double* loss_out, cudaStream_t s) {
  const int m = t->dec.m, r = t->dec.r, w = t->dec.width, L = t->dec.hidden;
  const int B = t->B, S = t->S, P = t->P;
  const long N = (long)B * S;
  const TrainerLayout& lay = t->lay;
  float* p = t->params;
  float* gr = t->grads;
  cudaError_t e;
  // ---- encoder forward: q_b
  if ((e = trainer_encode(t, B, snaps, t->q, s)) != cudaSuccess) return e;
  // ---- decoder forward and reverse pass on the sampled points
  const bool tc = t->precision == CROM_PREC_BF16_MIXED;
  if (tc) {
    gather_x_kernel<<<blocks(N, 256), 256, 0, s>>>(snaps, pt_idx, coords, B, S, P, m, t->tc.xin, t->target);
    // the decoder pass also leaves dL/dq_b in t->dq
    if ((e = trainer_decoder_tc(t, loss_out, t->num_sms, s)) != cudaSuccess) return e;
  } else {
    gather_kernel<<<blocks(N, 256), 256, 0, s>>>(snaps, pt_idx, coords, t->q, B, S, P, m, r, t->in0, t->target);
    const float* hin = t->in0;
    int kin = m + r;
    for (int l = 0; l < L; ++l) {
      e = gemm(t, s, (int)N, w, kin, hin, kin, 1, p + lay.dec_w[l], 1, kin, t->Z[l], w, kEpiBiasElu, p + lay.dec_b[l],
               t->H[l], nullptr);
      if (e != cudaSuccess) return e;
      hin = t->H[l];
      kin = w;
    }
    output_loss_kernel<<<blocks(N, 8), 256, 0, s>>>(t->H[L - 1], w, N, p + lay.dec_w[L], p + lay.dec_b[L], t->target,
                                                     t->dg, t->partial);
    loss_final_kernel<<<1, 1024, 0, s>>>(t->partial, (int)blocks(N, 8), N, loss_out ? loss_out : t->loss_dev);
    // output layer: gW_out[u] = sum_n dg[n] H_L[n][u], gb_out = sum dg
    e = gemm(t, s, 1, w, (int)N, t->dg, 0, 1, t->H[L - 1], w, 1, gr + lay.dec_w[L], w, kEpiStore, nullptr, nullptr,
             nullptr, t->split);
    if (e != cudaSuccess) return e;
    colsum(t, s, t->dg, N, 1, gr + lay.dec_b[L]);
    const float* wout = p + lay.dec_w[L];
    const float* zl = t->Z[L - 1];
    if (w % 4 == 0 && ((uintptr_t)wout & 15) == 0 && ((uintptr_t)zl & 15) == 0 && ((uintptr_t)t->delta & 15) == 0 &&
        N * (w / 4) < (1L << 31)) {
      const unsigned nq = (unsigned)(N * (w / 4));
      out_delta4_kernel<<<blocks(N * (w / 4), 256), 256, 0, s>>>(t->dg, wout, zl, w, nq, t->delta);
    } else {
      out_delta_kernel<<<blocks(N * w, 256), 256, 0, s>>>(t->dg, wout, zl, w, N, t->delta);
    }
    float* dcur = t->delta;
    float* dnext = t->delta2;
    for (int l = L - 1; l >= 0; --l) {
      const float* hprev = (l == 0) ? t->in0 : t->H[l - 1];
      const int kprev = (l == 0) ? m + r : w;
      // gW_l [w][kprev] = delta^T hprev (K = N, split), gb_l = column sums of delta
      e = gemm(t, s, w, kprev, (int)N, dcur, 1, w, hprev, kprev, 1, gr + lay.dec_w[l], kprev, kEpiStore, nullptr,
               nullptr, nullptr, t->split);
      if (e != cudaSuccess) return e;
      colsum(t, s, dcur, N, w, gr + lay.dec_b[l]);
      if (l > 0) {
        // delta_{l-1} = (delta_l W_l) * s'(Z_{l-1})
        e = gemm(t, s, (int)N, w, w, dcur, w, 1, p + lay.dec_w[l], w, 1, dnext, w, kEpiTimesEluD, nullptr, nullptr,
                 t->Z[l - 1]);
      } else {
        // input gradient din = delta_1 W_1  [N][m + r]
        e = gemm(t, s, (int)N, m + r, w, dcur, w, 1, p + lay.dec_w[0], m + r, 1, t->din, m + r, kEpiStore, nullptr,
                 nullptr, nullptr);
      }
      if (e != cudaSuccess) return e;
      float* tmp = dcur;
      dcur = dnext;
      dnext = tmp;
    }
  }
  if (!tc) dq_kernel<<<dim3(B, r), 256, 0, s>>>(t->din, m + r, B, S, m, r, t->dq);
  // ---- encoder reverse pass
  // dense 2: gW2 = dq^T h1, gb2 = sum dq, dz1 = (dq W2) * s'(z1)
  const int Ll = t->lens.back();
  if ((e = gemm(t, s, r, 32, B, t->dq, 1, r, t->d1h, 32, 1, gr + lay.d2w, 32, kEpiStore, nullptr, nullptr, nullptr)) !=
      cudaSuccess)
    return e;
  colsum(t, s, t->dq, B, r, gr + lay.d2b);
  if ((e = gemm(t, s, B, 32, r, t->dq, r, 1, p + lay.d2w, 32, 1, t->ed1, 32, kEpiTimesEluD, nullptr, nullptr,
                t->d1z)) != cudaSuccess)
    return e;
  // dense 1: gW1 = dz1^T h_conv, gb1 = sum dz1, dh_conv = dz1 W1
  const float* hconv = t->conv_h.back();
  if ((e = gemm(t, s, 32, Ll, B, t->ed1, 1, 32, hconv, Ll, 1, gr + lay.d1w, Ll, kEpiStore, nullptr, nullptr,
                nullptr)) != cudaSuccess)
    return e;
  colsum(t, s, t->ed1, B, 32, gr + lay.d1b);
  if ((e = gemm(t, s, B, Ll, 32, t->ed1, 32, 1, p + lay.d1w, Ll, 1, t->edh, Ll, kEpiStore, nullptr, nullptr,
                nullptr)) != cudaSuccess)
    return e;
  // convolutions, last to first
  for (int c = (int)t->lens.size() - 1; c >= 1; --c) {
    const int Lin = t->lens[c - 1], Lout = t->lens[c];
    const long n = (long)B * Lout;
    conv_dz_kernel<<<blocks(n, 256), 256, 0, s>>>(t->edh, t->conv_z[c - 1], n, t->edx);  // dz in edx
    const float* xin = (c == 1) ? snaps : t->conv_h[c - 2];
    {
      const int chunks = (int)std::min<long>(kColChunks, std::max<long>((long)B * Lout / 1024, 1));
      conv_grad_part_kernel<<<dim3(7, chunks), 256, 0, s>>>(t->edx, xin, Lin, Lout, B, t->red);
      conv_grad_final_kernel<<<1, 7 * 32, 0, s>>>(t->red, chunks, gr + lay.conv[c - 1]);
    }
    if (c > 1) conv_dx_kernel<<<blocks((long)B * Lin, 256), 256, 0, s>>>(t->edx, Lin, Lout, B,
                                                                         p + lay.conv[c - 1], t->edh);
  }
  // ---- Adam
  t->step += 1;
  const float c1 = (float)(1.0 - pow(0.9, (double)t->step));
  const float c2 = (float)(1.0 - pow(0.999, (double)t->step));
  adam_kernel<<<blocks(lay.total, 256), 256, 0, s>>>(p, gr, t->am, t->av, lay.total, lr, c1, c2);
  return cudaGetLastError();
}

}  // namespace crom
