// Decoder part of the training step on the tcgen05 tensor cores (paper §3, Eq. loss;
// App. D), precision CROM_PREC_BF16_MIXED: bf16 weights, activations and deltas
// in HBM, FP32 accumulation in tensor memory, FP32 master weights (the parameter
// vector) and Adam.
//
// With hidden layers h = 0..L-1 (H[h] = ELU(z_h), z_0 = W_0 [x; q] + b_0,
// z_h = W_h H[h-1] + b_h), output g = w_out . H[L-1] + b_out and
// loss = mean (g - f)^2 over the B*S sampled points:
//   forward:  H[0] on the CUDA cores: the latent part W_0q q_b + b_0 is one vector per
//             snapshot, so a point costs m FMAs per unit;
//             H[h] = ELU(H[h-1] W_h^T + b_h) by the GEMM's bias + ELU epilogue;
//             the last layer's epilogue also forms g (FP32, from the FP32 h) and the
//             residual g - f; a row kernel then forms dL/dg, delta[L-1] =
//             dL/dg w_out s'(z_{L-1}) and the column sums that give the gradients of
//             w_out, b_out and b_{L-1};
//   backward: for h = L-1 .. 1: dW_h = delta[h]^T H[h-1] (K = B*S, split over CTAs,
//             the splits added in a fixed order) and delta[h-1] = (delta[h] W_h) s'(z_{h-1})
//             with its column sums (db_{h-1}); then one pass over delta[0] forms, per
//             snapshot, D_b = sum of its rows and their x-weighted sums, from which
//             dW_0, db_0 and the encoder's dL/dq_b = W_0q^T D_b follow (the latent
//             inputs are constant over a snapshot).
// s'(z) is taken from h = ELU(z): 1 where h > 0, else h + 1 = e^z.  Every reduction
// runs in a fixed order, so a step is deterministic.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "crom_internal.h"

namespace crom {
namespace {

constexpr int kSplitsW = 64;      // K splits of the weight-gradient GEMMs

inline unsigned nblk(long n, int t) { return (unsigned)((n + t - 1) / t); }

__device__ __forceinline__ uint16_t bf16_bits(float f) {
  __nv_bfloat16 h = __float2bfloat16_rn(f);
  return *reinterpret_cast<uint16_t*>(&h);
}
__device__ __forceinline__ float bf16_val(uint16_t u) { return __uint_as_float((uint32_t)u << 16); }
// ELU with e^z - 1 from the hardware 2^x, as the GEMM epilogues form it (relative
// error ~2^-22, far below the bf16 rounding of the stored activations).
__device__ __forceinline__ float elu_fast(float z) {
  if (z > 0.f) return z;
  float e;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(z * 1.4426950408889634f));
  return e - 1.f;
}

// bf16 copies of the hidden matrices W_1..W_{L-1} ([w][w] each).
__global__ void weights_bf16_kernel(const float* params, const long* off_w, int L, int w, uint16_t* wh) {
  const long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  const long per = (long)w * w;
  if (e < (long)(L - 1) * per) {
    const int h = 1 + (int)(e / per);
    wh[e] = bf16_bits(params[off_w[h] + e % per]);
  }
}

// The latent part of the input layer is the same for every point of a snapshot:
// c0[b][u] = b_0[u] + sum_j W_0[u][m + j] q_b[j] (FP32, in order of j).
__global__ void layer0_const_kernel(const float* W0, const float* b0, const float* q, int m, int r, int w,
                                    float* c0) {
  const int b = blockIdx.x, u = threadIdx.x;
  if (u >= w) return;
  const float* wr = W0 + (long)u * (m + r) + m;
  float z = b0[u];
  for (int j = 0; j < r; ++j) z = fmaf(wr[j], q[(long)b * r + j], z);
  c0[(long)b * w + u] = z;
}

// H[0][n][u] = ELU(c0[b(n)][u] + sum_k W_0[u][k] x_n[k]) in bf16, x [N][m] the
// points' coordinates: a thread per four units, kRows0 rows per block (their
// coordinates staged in shared memory).
constexpr int kRows0 = 64;
__global__ void layer0_fwd_kernel(const float* x_in, long N, int kin, int m, int S, const float* W0, const float* c0,
                                  int w, uint16_t* H) {
  __shared__ float xs[kRows0][3];
  const long n0 = (long)blockIdx.x * kRows0;
  for (int i = threadIdx.x; i < kRows0 * 3; i += blockDim.x) {  // zeros beyond m and N
    const long n = n0 + i / 3;
    xs[i / 3][i % 3] = (n < N && i % 3 < m) ? x_in[n * m + i % 3] : 0.f;
  }
  __syncthreads();
  const int u = 4 * threadIdx.x;  // four units per thread: 8-byte stores
  if (u >= w) return;
  float wu[4][3];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int k = 0; k < 3; ++k) wu[j][k] = k < m ? W0[(long)(u + j) * kin + k] : 0.f;
  const long n1 = n0 + kRows0 < N ? n0 + kRows0 : N;
  long b = n0 / S, nb = (b + 1) * S;  // snapshot of row n and the first row of the next
  float4 cb = *reinterpret_cast<const float4*>(c0 + b * w + u);
#pragma unroll 4
  for (long n = n0; n < n1; ++n) {
    if (n == nb) {
      ++b;
      nb += S;
      cb = *reinterpret_cast<const float4*>(c0 + b * w + u);
    }
    float z[4] = {cb.x, cb.y, cb.z, cb.w};
    const float* x = xs[n - n0];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int k = 0; k < 3; ++k) z[j] = fmaf(wu[j][k], x[k], z[j]);
    *reinterpret_cast<uint2*>(H + n * w + u) =
        make_uint2((uint32_t)bf16_bits(elu_fast(z[0])) | ((uint32_t)bf16_bits(elu_fast(z[1])) << 16),
                   (uint32_t)bf16_bits(elu_fast(z[2])) | ((uint32_t)bf16_bits(elu_fast(z[3])) << 16));
  }
}

// Input-layer moments of delta_0 per chunk of a snapshot's rows: part[b][c][u][0] =
// sum_n delta_0[n][u], part[b][c][u][1 + k] = sum_n delta_0[n][u] x_n[k] over rows
// b S + c R .. (R = kRowsB), FP32 in row order.  A thread per pair of units, one block
// per (chunk, snapshot).  With D[b][u] = sum over snapshot b of delta_0[n][u] the
// input layer's gradients need nothing else: dW_0[u][k] (k < m) is the sum of the
// x-moments, dW_0[u][m + j] = sum_b D[b][u] q_b[j], db_0[u] = sum_b D[b][u] and the
// encoder's dL/dq_b[j] = sum_u W_0[u][m + j] D[b][u].
constexpr int kRowsB = 256;
__global__ void layer0_bwd_part_kernel(const uint16_t* delta, const float* x_in, int m, int S, int w,
                                       float* part) {
  __shared__ float xs[kRowsB][3];
  const int b = blockIdx.y, cidx = blockIdx.x;
  const long r0 = (long)b * S + (long)cidx * kRowsB;
  const int nr = min(kRowsB, S - cidx * kRowsB);
  for (int i = threadIdx.x; i < nr * 3; i += blockDim.x)  // zeros beyond m
    xs[i / 3][i % 3] = i % 3 < m ? x_in[(r0 + i / 3) * m + i % 3] : 0.f;
  __syncthreads();
  const int u = 2 * threadIdx.x;
  if (u >= w) return;
  float sa = 0.f, sb = 0.f, xa[3] = {0.f, 0.f, 0.f}, xb[3] = {0.f, 0.f, 0.f};
  const uint32_t* dp = reinterpret_cast<const uint32_t*>(delta + r0 * w + u);
  const int ldw = w / 2;
  int i = 0;
  for (; i + 4 <= nr; i += 4) {
    uint32_t d4[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) d4[k] = __ldg(dp + (long)(i + k) * ldw);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float da = bf16_val((uint16_t)(d4[k] & 0xffffu)), db = bf16_val((uint16_t)(d4[k] >> 16));
      sa += da;
      sb += db;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        xa[j] = fmaf(da, xs[i + k][j], xa[j]);
        xb[j] = fmaf(db, xs[i + k][j], xb[j]);
      }
    }
  }
  for (; i < nr; ++i) {
    const uint32_t d = __ldg(dp + (long)i * ldw);
    const float da = bf16_val((uint16_t)(d & 0xffffu)), db = bf16_val((uint16_t)(d >> 16));
    sa += da;
    sb += db;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      xa[j] = fmaf(da, xs[i][j], xa[j]);
      xb[j] = fmaf(db, xs[i][j], xb[j]);
    }
  }
  float* o = part + (((long)b * gridDim.x + cidx) * w + u) * (1 + m);
  o[0] = sa;
  o[1 + m] = sb;
  for (int k = 0; k < m; ++k) {
    o[1 + k] = xa[k];
    o[1 + m + 1 + k] = xb[k];
  }
}

// Compensated FP32 sum (Knuth's two-sum per term): ~2^-48 relative for the term
// counts here, deterministic in a fixed order, and without the FP64 pipe, which is
// narrow on this GPU.
struct CSum {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = __fadd_rn(s, x);
    const float bp = __fsub_rn(t, s);
    c += __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
    s = t;
  }
  __device__ __forceinline__ void add(const CSum& o) {
    add(o.s);
    c += o.c;
  }
  __device__ __forceinline__ float value() const { return s + c; }
};
// The 32 lanes' sums combined by a fixed butterfly (every lane ends with the same value).
__device__ __forceinline__ float warp_csum(CSum v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    CSum w;
    w.s = __shfl_xor_sync(0xffffffffu, v.s, o);
    w.c = __shfl_xor_sync(0xffffffffu, v.c, o);
    // the lower lane's sum first, so that both lanes of a pair add in the same order
    CSum lo = (threadIdx.x & o) ? w : v, hi = (threadIdx.x & o) ? v : w;
    lo.add(hi);
    v = lo;
  }
  return v.value();
}

// snap[b][u][k] = sum over the chunks of snapshot b of part[b][c][u][k] (in order).
__global__ void layer0_bwd_snap_kernel(const float* part, int chunks, int w, int m, float* snap) {
  const int b = blockIdx.x;
  const int e = threadIdx.x + blockIdx.y * blockDim.x;  // (u, k)
  const int per = w * (1 + m);
  if (e >= per) return;
  CSum s;
  for (int c = 0; c < chunks; ++c) s.add(part[((long)b * chunks + c) * per + e]);
  snap[(long)b * per + e] = s.value();
}

// The input layer's gradients from the per-snapshot moments, one warp per output
// entry (lanes take every 32nd term, then a fixed butterfly): entries e < w kin are
// dW_0[u][j] (u = e / kin), the next w are db_0, the last B r are the encoder's
// dL/dq_b[j].  Products are formed exactly (two-product) and added compensated.
__global__ void layer0_grad_kernel(const float* snap, const float* q, const float* W0, int B, int m, int r, int w,
                                   float* gW0, float* gb0, float* dq) {
  const int kin = m + r;
  const long e = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const long nw = (long)w * kin;
  const int per = w * (1 + m);
  if (e >= nw + w + (long)B * r) return;  // whole warps leave together
  CSum s;
  auto add_prod = [&](float a, float b) {
    const float p = __fmul_rn(a, b);
    s.add(p);
    s.c += fmaf(a, b, -p);
  };
  if (e < nw) {
    const int u = (int)(e / kin), j = (int)(e % kin);
    if (j < m) {
      for (int b = lane; b < B; b += 32) s.add(snap[(long)b * per + u * (1 + m) + 1 + j]);
    } else {
      for (int b = lane; b < B; b += 32) add_prod(snap[(long)b * per + u * (1 + m)], q[(long)b * r + j - m]);
    }
  } else if (e < nw + w) {
    const int u = (int)(e - nw);
    for (int b = lane; b < B; b += 32) s.add(snap[(long)b * per + u * (1 + m)]);
  } else {
    const int b = (int)((e - nw - w) / r), j = (int)((e - nw - w) % r);
    for (int u = lane; u < w; u += 32) add_prod(W0[(long)u * kin + m + j], snap[(long)b * per + u * (1 + m)]);
  }
  const float t = warp_csum(s);
  if (lane == 0) {
    if (e < nw) gW0[e] = t;
    else if (e < nw + w) gb0[e - nw] = t;
    else dq[e - nw - w] = t;
  }
}

// The output layer's backward from h_L (bf16 rows of kW) and the residuals r = g - f
// (FP32, from the GEMM epilogue that formed g from the FP32 h_L): per row
// dL/dg = 2 r / N and delta_L[n][u] = dL/dg w_out[u] s'(z_u), s'(z) = 1 where h > 0,
// else h + 1.  Warp p handles rows 32 p .. 32 p + 31 (one part), lane l columns
// l kPer .. (kPer = kW / 32), four rows' loads in flight; per part the column sums of
// delta (db_L) and of dL/dg h (dw_out) and the row sums of r^2 and dL/dg, each in
// row order.
constexpr int kOutWarps = 8;
template <int kW>
__global__ void out_delta_kernel(const uint16_t* H, const float* resid, const float* wout, long N, long nparts,
                                 float inv_count, uint16_t* delta, float* colpart, float* colpart2, float* rowpart) {
  constexpr int kPer = kW / 32;  // 2, 4 or 8 bf16 per lane
  typedef typename std::conditional<kPer == 8, uint4, typename std::conditional<kPer == 4, uint2, uint32_t>::type>::type
      Vec;
  const long part = (long)blockIdx.x * kOutWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  const long r0 = part * 32;
  if (part >= nparts) return;  // whole warps; parts past N write zero sums
  float wo[kPer], cs[kPer], cs2[kPer];
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    wo[k] = wout[lane * kPer + k];
    cs[k] = 0.f;
    cs2[k] = 0.f;
  }
  float rr = 0.f, dgs = 0.f;
  for (int i0 = 0; i0 < 32; i0 += 4) {
    Vec hv[4];
    float res[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const long n = r0 + i0 + j;
      const bool in = n < N;
      hv[j] = in ? *reinterpret_cast<const Vec*>(H + n * kW + lane * kPer) : Vec{};
      res[j] = in ? resid[n] : 0.f;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const long n = r0 + i0 + j;
      const uint32_t* hw = reinterpret_cast<const uint32_t*>(&hv[j]);
      const float dg = 2.f * res[j] * inv_count;
      uint32_t dw[kPer / 2];
#pragma unroll
      for (int k = 0; k < kPer / 2; ++k) {
        const float h0 = bf16_val((uint16_t)(hw[k] & 0xffffu)), h1 = bf16_val((uint16_t)(hw[k] >> 16));
        const float d0 = dg * wo[2 * k] * (h0 > 0.f ? 1.f : h0 + 1.f);
        const float d1 = dg * wo[2 * k + 1] * (h1 > 0.f ? 1.f : h1 + 1.f);
        cs[2 * k] += d0;
        cs[2 * k + 1] += d1;
        cs2[2 * k] = fmaf(dg, h0, cs2[2 * k]);
        cs2[2 * k + 1] = fmaf(dg, h1, cs2[2 * k + 1]);
        dw[k] = (uint32_t)bf16_bits(d0) | ((uint32_t)bf16_bits(d1) << 16);
      }
      if (n < N) *reinterpret_cast<Vec*>(delta + n * kW + lane * kPer) = *reinterpret_cast<const Vec*>(dw);
      rr = fmaf(res[j], res[j], rr);
      dgs += dg;
    }
  }
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    colpart[part * kW + lane * kPer + k] = cs[k];
    colpart2[part * kW + lane * kPer + k] = cs2[k];
  }
  if (lane == 0) {
    rowpart[2 * part] = rr;
    rowpart[2 * part + 1] = dgs;
  }
}

// out[e] = sum_p part[p * stride + e], in order of p (compensated).  Eight loads are
// issued before their additions, so that their latencies overlap.
__global__ void sum_parts_kernel(const float* part, int nparts, long stride, long n, float* out) {
  const long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (e >= n) return;
  CSum s;
  int p = 0;
  for (; p + 8 <= nparts; p += 8) {
    float v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = __ldg(part + (long)(p + k) * stride + e);
#pragma unroll
    for (int k = 0; k < 8; ++k) s.add(v[k]);
  }
  for (; p < nparts; ++p) s.add(part[(long)p * stride + e]);
  out[e] = s.value();
}

// Column sums of part [nparts][cols] in a fixed order, first level: block (x, y)
// adds parts y * kColPer .. of columns 32 x .. (32 columns x 8 part lanes, the lanes
// combined in order) into mid[y][col].  The second level adds mid's rows in order
// (sum_parts_kernel).
constexpr int kColPer = 128;
__global__ void colsum_level1_kernel(const float* part, int nparts, int cols, float* mid) {
  __shared__ float red_s[8][32], red_c[8][32];
  const int col = blockIdx.x * 32 + threadIdx.x;
  const int p0 = blockIdx.y * kColPer, p1 = min(nparts, p0 + kColPer);
  CSum acc;
  if (col < cols) {
    constexpr int kPer = kColPer / 8;  // parts per thread, loaded before they are added in order
    float v[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int p = p0 + threadIdx.y + 8 * k;
      v[k] = p < p1 ? __ldg(part + (long)p * cols + col) : 0.f;
    }
#pragma unroll
    for (int k = 0; k < kPer; ++k) acc.add(v[k]);
  }
  red_s[threadIdx.y][threadIdx.x] = acc.s;
  red_c[threadIdx.y][threadIdx.x] = acc.c;
  __syncthreads();
  if (threadIdx.y == 0 && col < cols) {
    CSum t;
    for (int k = 0; k < 8; ++k) {
      CSum o;
      o.s = red_s[k][threadIdx.x];
      o.c = red_c[k][threadIdx.x];
      t.add(o);
    }
    mid[(long)blockIdx.y * cols + col] = t.value();
  }
}

// loss = sum_p rowpart[p][0] * inv_count; gb_out = sum_p rowpart[p][1]: each thread
// a contiguous range of parts (compensated), then a fixed tree in FP64.
__global__ void loss_parts_kernel(const float* rowpart, int nparts, double inv_count, double* loss, float* gbout) {
  constexpr int kT = 1024;
  __shared__ double red[2][kT];
  CSum a, b;
  const int per = (nparts + kT - 1) / kT;
  for (int p = threadIdx.x * per; p < min(nparts, (int)(threadIdx.x + 1) * per); ++p) {
    a.add(rowpart[2 * p]);
    b.add(rowpart[2 * p + 1]);
  }
  red[0][threadIdx.x] = (double)a.s + (double)a.c;
  red[1][threadIdx.x] = (double)b.s + (double)b.c;
  __syncthreads();
  for (int o = kT / 2; o > 0; o >>= 1) {
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
  for (int h = 0; h < L; ++h) c.H.push_back((uint16_t*)A((size_t)N * w * 2));
  c.d0 = (uint16_t*)A((size_t)N * w * 2);
  c.d1 = (uint16_t*)A((size_t)N * w * 2);
  c.colpart = (float*)A((size_t)tiles_m * 4 * w * 4);
  c.colpart2 = (float*)A((size_t)tiles_m * 4 * w * 4);
  c.rowpart = (float*)A((size_t)tiles_m * 4 * 2 * 4);
  c.resid = (float*)A((size_t)N * 4);
  c.colmid = (float*)A((size_t)(tiles_m * 4 + kColPer - 1) / kColPer * w * 4);
  c.split = (float*)A((size_t)kSplitsW * w * w * 4);
  const int m = t->dec.m;
  c.xin = (float*)A((size_t)N * m * 4);
  c.c0 = (float*)A((size_t)t->B * w * 4);
  c.part0 = (float*)A((size_t)t->B * ((t->S + kRowsB - 1) / kRowsB) * w * (1 + m) * 4);
  c.snap0 = (float*)A((size_t)t->B * w * (1 + m) * 4);
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
  const int m = t->dec.m, r = t->dec.r, B = t->B, S = t->S;
  weights_bf16_kernel<<<nblk((long)(L - 1) * w * w, 256), 256, 0, s>>>(p, c.off_w, L, w, c.wh);
  // ---- forward
  layer0_const_kernel<<<B, w, 0, s>>>(p + lay.dec_w[0], p + lay.dec_b[0], t->q, m, r, w, c.c0);
  layer0_fwd_kernel<<<nblk(N, kRows0), w / 4, 0, s>>>(c.xin, N, kin, m, S, p + lay.dec_w[0], c.c0, w, c.H[0]);
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
      g.resid = c.resid;
    }
    if ((e = tc_gemm(g, num_sms, c.flag, s)) != cudaSuccess) return e;
  }
  // delta_L, the loss terms and the output layer's column sums from h_L and the residuals
  {
    const unsigned blocks = (unsigned)(((long)parts + kOutWarps - 1) / kOutWarps);
    const float inv = (float)(1.0 / (double)N);
    if (w == 256)
      out_delta_kernel<256><<<blocks, 32 * kOutWarps, 0, s>>>(c.H[L - 1], c.resid, p + lay.dec_w[L], N, parts, inv, c.d0,
                                                               c.colpart, c.colpart2, c.rowpart);
    else if (w == 128)
      out_delta_kernel<128><<<blocks, 32 * kOutWarps, 0, s>>>(c.H[L - 1], c.resid, p + lay.dec_w[L], N, parts, inv, c.d0,
                                                               c.colpart, c.colpart2, c.rowpart);
    else
      out_delta_kernel<64><<<blocks, 32 * kOutWarps, 0, s>>>(c.H[L - 1], c.resid, p + lay.dec_w[L], N, parts, inv, c.d0,
                                                              c.colpart, c.colpart2, c.rowpart);
  }
  loss_parts_kernel<<<1, 1024, 0, s>>>(c.rowpart, parts, 1.0 / (double)N, loss_out ? loss_out : t->loss_dev,
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
      if (h > 1) colsum_parts(c.colpart, parts, w, c.colmid, gr + lay.dec_b[h - 1], s);  // db_0 below
    }
    std::swap(dcur, dnext);
  }
  // ---- input layer: per-snapshot moments of delta[0], then dW_0, db_0 and dL/dq
  const int chunks = (S + kRowsB - 1) / kRowsB;
  layer0_bwd_part_kernel<<<dim3(chunks, B), w / 2, 0, s>>>(dcur, c.xin, m, S, w, c.part0);
  layer0_bwd_snap_kernel<<<dim3(B, nblk((long)w * (1 + m), 256)), 256, 0, s>>>(c.part0, chunks, w, m, c.snap0);
  layer0_grad_kernel<<<nblk(32 * ((long)w * kin + w + (long)B * r), 256), 256, 0, s>>>(
      c.snap0, t->q, p + lay.dec_w[0], B, m, r, w, gr + lay.dec_w[0], gr + lay.dec_b[0], t->dq);
  return cudaGetLastError();
}

}  // namespace crom
