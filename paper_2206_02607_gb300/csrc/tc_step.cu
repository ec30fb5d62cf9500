// Batched latent step on the tcgen05 tensor cores (crom_step, CROM_PREC_BF16X2).
//
// One persistent launch per step; one CTA per SM (128 threads, thread u = hidden
// unit u = TMEM lane u) takes whole instances from a queue ordered by |M_i|,
// largest first.  Per instance, per Gauss-Newton iteration k, per tile of 32
// samples (paper §4, Algorithm 3):
//
//  Step 1 (network inference) as a forward pass whose UMMA columns are
//  (channel, sample) pairs.  Iteration 0 carries the value, dg/dx_k and a single
//  Laplacian channel: the Laplacian obeys d2z = W d2h with
//  d2h = s''(z) * sum_k (dz/dx_k)^2 + s'(z) d2z, so the m second-derivative
//  channels of Algorithm 2 collapse into one.  Iteration k >= 1 carries the value
//  at q^(k) and the difference channel h(q^(k)) - h(q_n).
//    D[u][n] = sum_k W_l[u][k] H[k][n]    (M = 128 units, N = channels x 32, K = 128)
//  The epilogue (bias, ELU chain, s'(z) kept in TMEM for the backward pass) runs in
//  FP32 registers; the result is written back as bf16 hi/lo operand pairs.
//
//  Step 2 (PDE update): Delta f_j = dt * alpha_i * Lap g(y_j) (or the
//  advection-diffusion form), kept per sample in shared memory.
//
//  Step 3 (network inversion): the Jacobian rows dg/dq(y_j) come from one
//  reverse-mode pass, delta_L = w_out * s'(z_L), delta_{l-1} = (W_l^T delta_l) *
//  s'(z_{l-1}) on the tensor cores (A = W_l read MN-major from the same shared
//  image), then J = W_1q^T delta_1 by a projection UMMA.  J^T J and J^T rho are
//  accumulated in FP64 from the FP32 rows (exact products); the r x r system is
//  solved by FP64 Cholesky and q is updated in FP64.
//
// The output layer w_out . h_L and the projection W_1q^T delta_1 share one
// 16-row bf16 matrix P (row 0 = w_out, rows 1..r = W_1q columns).
#include <math.h>

#include <algorithm>

#include "crom_internal.h"
#include "tc_common.cuh"

namespace crom {
namespace {

using namespace tc;

constexpr int kThreads = 128;
constexpr int kS = 32;            // samples per tile
constexpr int kMaxSamples = 2048; // |M_i| limit (per-sample Delta f kept in shared memory)
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kAcc = 0;      // accumulator, up to 128 columns
constexpr uint32_t kSig = 128;    // s'(z_l), l = 1..L: 32 columns each
constexpr uint32_t kPrj = 288;    // projection output, 16 columns
constexpr uint32_t kWaitLimit = 1u << 25;
constexpr size_t kH = (size_t)kTcWidth * 128 * 2;  // one bf16 operand buffer, 32 KB

struct StepParams {
  const uint8_t* img;
  int img_bytes;
  int L;  // hidden layers
  int m, r;
  const float* w1;
  const float* b1;
  const float* bh;
  const float* wout;
  float bout;
  int pde;
  int gn_iters;
  double dt;
  int n_inst;
  double* q;
  const float* alpha;
  const float* vel;
  const int* off;
  const float* x;
  int max_samples;
  int* status;
  const int* order;
  int* queue;  // [0] work counter, [1] timeout flag
};

struct __align__(16) Tail {
  uint64_t bar_w;
  uint64_t bar_mma;
  uint32_t tmem_base;
  int s_idx;
  int s_status;
  int pad;
  double qn[16];
  double qcur[16];
  double amat[15 * 16];
  float c1[kTcWidth];
  float dz1[kTcWidth];
  float w1x[2][kTcWidth];
  float w1q[16][kTcWidth];
  float bh[4][kTcWidth];
  float wout[kTcWidth];
  float xs[2][kS];
  float gout[4][kS];
  float rho[kS];
  float jt[kS][16];
  float df[kMaxSamples];
};

__device__ __forceinline__ void split_store16(uint8_t* Hhi, uint8_t* Hlo, int k, int n0, const float* v) {
  uint32_t hi[8], lo[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    hi[j] = pack_bf16(v[2 * j], v[2 * j + 1]);
    lo[j] = pack_bf16(v[2 * j] - bf16_lo_f(hi[j]), v[2 * j + 1] - bf16_hi_f(hi[j]));
  }
  *reinterpret_cast<uint4*>(Hhi + mn_offset(k, n0)) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
  *reinterpret_cast<uint4*>(Hhi + mn_offset(k, n0 + 8)) = make_uint4(hi[4], hi[5], hi[6], hi[7]);
  *reinterpret_cast<uint4*>(Hlo + mn_offset(k, n0)) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
  *reinterpret_cast<uint4*>(Hlo + mn_offset(k, n0 + 8)) = make_uint4(lo[4], lo[5], lo[6], lo[7]);
}

// s(a) - s(a - d) without cancellation (see the FP32 path).
__device__ __forceinline__ float elu_diff(float a, float d) {
  const float b = a - d;
  if (a > 0.f && b > 0.f) return d;
  if (a <= 0.f && b <= 0.f) return -__expf(a) * expm1f(-d);
  const float sa = a > 0.f ? a : expm1f(a);
  const float sb = b > 0.f ? b : expm1f(b);
  return sa - sb;
}

// Issue the UMMAs of one stage and wait for them.  Every thread returns the same value.
struct Pipe {
  uint64_t* bar;
  uint32_t phase;
};

__device__ __forceinline__ bool sync_and_wait(Pipe& pp) {
  bool ok = __syncthreads_and(mbar_wait(pp.bar, pp.phase, kWaitLimit));
  pp.phase ^= 1;
  tc_fence_after();
  return ok;
}

__device__ __forceinline__ void before_issue() {
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
}

// D(+)= A * B^T over K = 128 with hi/lo B (or A) operands.
__device__ __forceinline__ void issue_layer(uint32_t d, uint32_t a_base, bool a_mn, uint32_t hhi, uint32_t hlo,
                                           uint32_t idesc) {
  for (int kk = 0; kk < 8; ++kk) {
    const uint64_t a = a_mn ? desc_mnmajor(a_base, kk) : desc_kmajor(a_base, 128, kk);
    umma_f16(d, a, desc_mnmajor(hhi, kk), idesc, kk > 0);
  }
  for (int kk = 0; kk < 8; ++kk) {
    const uint64_t a = a_mn ? desc_mnmajor(a_base, kk) : desc_kmajor(a_base, 128, kk);
    umma_f16(d, a, desc_mnmajor(hlo, kk), idesc, 1);
  }
}
__device__ __forceinline__ void issue_proj(uint32_t d, uint32_t hhi, uint32_t hlo, uint32_t proj) {
  constexpr uint32_t id = idesc_f16(128, 16, true, false, true);
  for (int kk = 0; kk < 8; ++kk) umma_f16(d, desc_mnmajor(hhi, kk), desc_kmajor(proj, 16, kk), id, kk > 0);
  for (int kk = 0; kk < 8; ++kk) umma_f16(d, desc_mnmajor(hlo, kk), desc_kmajor(proj, 16, kk), id, 1);
}

__global__ void __launch_bounds__(kThreads, 1) step_tc_kernel(StepParams p) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* Wimg = sm;
  uint8_t* Hhi = sm + ((p.img_bytes + 1023) & ~1023);
  uint8_t* Hlo = Hhi + kH;
  Tail* T = reinterpret_cast<Tail*>(Hlo + kH);
  const int tid = threadIdx.x, warp = tid >> 5, u = tid;
  const int m = p.m, r = p.r, L = p.L;
  const uint32_t lane_base = (uint32_t)warp * 32;

  if (tid == 0) {
    mbar_init(&T->bar_w, 1);
    mbar_init(&T->bar_mma, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(&T->tmem_base, kTmemCols);
    tmem_relinquish();
  }
  for (int l = 0; l < L - 1; ++l) T->bh[l][u] = p.bh[l * kTcWidth + u];
  for (int k = 0; k < m; ++k) T->w1x[k][u] = p.w1[u * (m + r) + k];
  for (int j = 0; j < r; ++j) T->w1q[j][u] = p.w1[u * (m + r) + m + j];
  T->wout[u] = p.wout[u];
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tb = T->tmem_base;
  if (tid == 0) {
    mbar_arrive_expect_tx(&T->bar_w, (uint32_t)p.img_bytes);
    for (int o = 0; o < p.img_bytes; o += 16384)
      bulk_g2s(Wimg + o, p.img + o, (uint32_t)min(16384, p.img_bytes - o), &T->bar_w);
  }
  bool ok = __syncthreads_and(mbar_wait(&T->bar_w, 0, kWaitLimit));
  Pipe pp{&T->bar_mma, 0};
  const uint32_t wbase = smem_u32(Wimg);
  const uint32_t proj = wbase + (uint32_t)(L - 1) * kTcLayerBytes;
  const uint32_t hhi = smem_u32(Hhi), hlo = smem_u32(Hlo);
  const int ntri = r * (r + 1) / 2;
  const int n_entries = ntri + r;
  // entries handled by this thread: e0 = tid, e1 = tid + 128
  int ea[2], eb[2];
  for (int h = 0; h < 2; ++h) {
    const int e = tid + h * kThreads;
    ea[h] = -1; eb[h] = -1;
    if (e < ntri) {
      int a = 0, rem = e;
      while (rem >= r - a) { rem -= r - a; ++a; }
      ea[h] = a; eb[h] = a + rem;
    } else if (e < n_entries) {
      ea[h] = e - ntri; eb[h] = -2;  // -2: right-hand side entry J^T rho
    }
  }

  while (ok) {
    __syncthreads();  // everyone has finished with the previous instance's shared state
    if (tid == 0) T->s_idx = atomicAdd(&p.queue[0], 1);
    __syncthreads();
    const int idx = T->s_idx;
    if (idx >= p.n_inst) break;
    const int inst = p.order[idx];
    const int o0 = p.off[inst];
    const int M = p.off[inst + 1] - o0;
    if (M < r || M > p.max_samples || M > kMaxSamples) {
      if (tid == 0) p.status[inst] = CROM_ERR_INVALID_ARG;
      continue;
    }
    if (tid < r) {
      const double v = p.q[(size_t)inst * r + tid];
      T->qn[tid] = v;
      T->qcur[tid] = v;
    }
    if (tid == 0) T->s_status = CROM_OK;
    const float alpha = p.alpha[inst];
    __syncthreads();
    const int ntiles = (M + kS - 1) / kS;

    for (int it = 0; it < p.gn_iters && ok; ++it) {
      const bool first = (it == 0);
      const int nch = first ? 2 + m : 2;  // iteration 0: v, dx_1..dx_m, Lap; later: v(q^(k)), diff
      const int N = nch * kS;
      {
        double c = (double)p.b1[u], dz = 0.0;
        for (int j = 0; j < r; ++j) {
          c += (double)T->w1q[j][u] * T->qcur[j];
          dz += (double)T->w1q[j][u] * (T->qcur[j] - T->qn[j]);
        }
        T->c1[u] = (float)c;
        T->dz1[u] = (float)dz;
      }
      double acc[2] = {0.0, 0.0};
      for (int t = 0; t < ntiles && ok; ++t) {
        const int ns = min(kS, M - t * kS);
        if (tid < kS) {
          const int s = tid < ns ? tid : 0;
          for (int k = 0; k < m; ++k) T->xs[k][tid] = p.x[(size_t)(o0 + t * kS + s) * m + k];
        }
        __syncthreads();
        // ---------------- layer 1 (CUDA cores)
        {
          const float c = T->c1[u], dz = T->dz1[u];
          const float wx0 = T->w1x[0][u], wx1 = (m > 1) ? T->w1x[1][u] : 0.f;
          const float wsq = wx0 * wx0 + wx1 * wx1;
#pragma unroll 1
          for (int s0 = 0; s0 < kS; s0 += 16) {
            float v[4][16], sg[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              float z = fmaf(wx0, T->xs[0][s0 + i], c);
              if (m > 1) z = fmaf(wx1, T->xs[1][s0 + i], z);
              const float e = __expf(fminf(z, 0.f));
              const bool pos = z > 0.f;
              const float s1 = pos ? 1.f : e, s2 = pos ? 0.f : e;
              sg[i] = s1;
              v[0][i] = pos ? z : e - 1.f;
              if (first) {
                v[1][i] = s1 * wx0;
                if (m > 1) { v[2][i] = s1 * wx1; v[3][i] = s2 * wsq; }
                else v[2][i] = s2 * wsq;
              } else {
                v[1][i] = elu_diff(z, dz);
              }
            }
            tmem_st16(taddr(tb, lane_base, kSig + s0), sg);
#pragma unroll
            for (int ch = 0; ch < 4; ++ch)
              if (ch < nch) split_store16(Hhi, Hlo, u, ch * kS + s0, v[ch]);
          }
          tmem_st_wait();
        }
        // ---------------- hidden layers 2..L (tensor cores)
        const uint32_t id_fwd = idesc_f16(128, N, false, true, true);
        for (int l = 0; l < L - 1 && ok; ++l) {
          before_issue();
          if (tid == 0) {
            tc_fence_after();
            issue_layer(tb + kAcc, wbase + (uint32_t)l * kTcLayerBytes, false, hhi, hlo, id_fwd);
            umma_commit(pp.bar);
          }
          ok = sync_and_wait(pp);
          if (!ok) break;
          const float bias = T->bh[l][u];
#pragma unroll 1
          for (int s0 = 0; s0 < kS; s0 += 16) {
            float v[4][16], sg[16];
#pragma unroll
            for (int ch = 0; ch < 4; ++ch)
              if (ch < nch) tmem_ld16(taddr(tb, lane_base, kAcc + ch * kS + s0), v[ch]);
            tmem_ld_wait();
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const float z = v[0][i] + bias;
              const float e = __expf(fminf(z, 0.f));
              const bool pos = z > 0.f;
              const float s1 = pos ? 1.f : e, s2 = pos ? 0.f : e;
              sg[i] = s1;
              v[0][i] = pos ? z : e - 1.f;
              if (first) {
                if (m > 1) {
                  const float a = v[1][i], b = v[2][i];
                  v[1][i] = s1 * a;
                  v[2][i] = s1 * b;
                  v[3][i] = fmaf(s2, a * a + b * b, s1 * v[3][i]);
                } else {
                  const float a = v[1][i];
                  v[1][i] = s1 * a;
                  v[2][i] = fmaf(s2, a * a, s1 * v[2][i]);
                }
              } else {
                v[1][i] = elu_diff(z, v[1][i]);
              }
            }
            tmem_st16(taddr(tb, lane_base, kSig + (l + 1) * kS + s0), sg);
#pragma unroll
            for (int ch = 0; ch < 4; ++ch)
              if (ch < nch) split_store16(Hhi, Hlo, u, ch * kS + s0, v[ch]);
          }
          tmem_st_wait();
        }
        if (!ok) break;
        // ---------------- output layer: PRJ[n][0] = w_out . h_L[:, n]
        before_issue();
        if (tid == 0) {
          tc_fence_after();
          issue_proj(tb + kPrj, hhi, hlo, proj);
          umma_commit(pp.bar);
        }
        ok = sync_and_wait(pp);
        if (!ok) break;
        {
          float v[16];
          tmem_ld16(taddr(tb, lane_base, kPrj), v);
          tmem_ld_wait();
          if (tid < N) T->gout[tid / kS][tid % kS] = v[0] + ((tid < kS && first) ? p.bout : 0.f);
        }
        __syncthreads();
        // ---------------- Step 2 and the residual rho_j
        if (tid < kS) {
          float rho = 0.f;
          if (tid < ns) {
            const int j = t * kS + tid;
            if (first) {
              const float lap = T->gout[m + 1][tid];
              double df;
              if (p.pde == CROM_PDE_HEAT) {
                df = p.dt * (double)alpha * (double)lap;
              } else {
                double adv = 0.0;
                for (int k = 0; k < m; ++k)
                  adv += (double)p.vel[(size_t)(o0 + j) * m + k] * (double)T->gout[1 + k][tid];
                df = p.dt * (-adv + (double)alpha * (double)lap);
              }
              T->df[j] = (float)df;
              rho = -(float)df;
            } else {
              rho = T->gout[1][tid] - T->df[j];
            }
          }
          T->rho[tid] = rho;
        }
        // ---------------- reverse pass for dg/dq at q^(k)
        {
          // delta_L = w_out * s'(z_L) (N = 32 sample columns)
          float sg[2][16];
          tmem_ld16(taddr(tb, lane_base, kSig + (L - 1) * kS), sg[0]);
          tmem_ld16(taddr(tb, lane_base, kSig + (L - 1) * kS + 16), sg[1]);
          tmem_ld_wait();
          const float w = T->wout[u];
          for (int h = 0; h < 2; ++h) {
            float v[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = w * sg[h][i];
            split_store16(Hhi, Hlo, u, h * 16, v);
          }
        }
        constexpr uint32_t id_bwd = idesc_f16(128, kS, true, true, true);
        for (int l = L - 2; l >= 0 && ok; --l) {
          // accumulator = W_{l+2}^T delta_{l+2}; times s'(z_{l+1}) gives delta_{l+1}
          before_issue();
          if (tid == 0) {
            tc_fence_after();
            issue_layer(tb + kAcc, wbase + (uint32_t)l * kTcLayerBytes, true, hhi, hlo, id_bwd);
            umma_commit(pp.bar);
          }
          ok = sync_and_wait(pp);
          if (!ok) break;
          for (int h = 0; h < 2; ++h) {
            float v[16], sg[16];
            tmem_ld16(taddr(tb, lane_base, kAcc + h * 16), v);
            tmem_ld16(taddr(tb, lane_base, kSig + l * kS + h * 16), sg);
            tmem_ld_wait();
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] *= sg[i];
            split_store16(Hhi, Hlo, u, h * 16, v);
          }
        }
        if (!ok) break;
        // J[s][j] = sum_u W_1q[u][j] delta_1[u][s]
        before_issue();
        if (tid == 0) {
          tc_fence_after();
          issue_proj(tb + kPrj, hhi, hlo, proj);
          umma_commit(pp.bar);
        }
        ok = sync_and_wait(pp);
        if (!ok) break;
        if (warp == 0) {
          float v[16];
          tmem_ld16(taddr(tb, 0, kPrj), v);
          tmem_ld_wait();
#pragma unroll
          for (int j = 0; j < 15; ++j) T->jt[tid][j] = v[j + 1];
        }
        __syncthreads();
        // ---------------- normal equations in FP64 (exact products of FP32 rows)
        for (int h = 0; h < 2; ++h) {
          if (ea[h] < 0) continue;
          double s = 0.0;
          if (eb[h] >= 0) {
            for (int i = 0; i < ns; ++i) s = fma((double)T->jt[i][ea[h]], (double)T->jt[i][eb[h]], s);
          } else {
            for (int i = 0; i < ns; ++i) s = fma((double)T->jt[i][ea[h]], (double)T->rho[i], s);
          }
          acc[h] += s;
        }
      }  // tiles
      if (!ok) break;
      for (int h = 0; h < 2; ++h) {
        if (ea[h] < 0) continue;
        if (eb[h] >= 0) {
          T->amat[ea[h] * (r + 1) + eb[h]] = acc[h];
          T->amat[eb[h] * (r + 1) + ea[h]] = acc[h];
        } else {
          T->amat[ea[h] * (r + 1) + r] = -acc[h];
        }
      }
      __syncthreads();
      if (tid == 0) {
        double* A = T->amat;
        const int R = r + 1;
        int st = CROM_OK;
        double dmax = 0.0;
        for (int a = 0; a < r; ++a)
          for (int b = 0; b <= r; ++b)
            if (!isfinite(A[a * R + b])) st = CROM_ERR_NONFINITE;
        for (int a = 0; a < r; ++a) dmax = fmax(dmax, A[a * R + a]);
        const double tol = 1e-14 * dmax;
        for (int j = 0; j < r && st == CROM_OK; ++j) {
          double d = A[j * R + j];
          for (int k = 0; k < j; ++k) d -= A[j * R + k] * A[j * R + k];
          if (!(d > tol)) { st = CROM_ERR_SINGULAR; break; }
          const double ljj = sqrt(d);
          A[j * R + j] = ljj;
          for (int i = j + 1; i < r; ++i) {
            double v = A[i * R + j];
            for (int k = 0; k < j; ++k) v -= A[i * R + k] * A[j * R + k];
            A[i * R + j] = v / ljj;
          }
        }
        if (st == CROM_OK) {
          double y[16], xs[16];
          for (int i = 0; i < r; ++i) {
            double v = A[i * R + r];
            for (int k = 0; k < i; ++k) v -= A[i * R + k] * y[k];
            y[i] = v / A[i * R + i];
          }
          for (int i = r - 1; i >= 0; --i) {
            double v = y[i];
            for (int k = i + 1; k < r; ++k) v -= A[k * R + i] * xs[k];
            xs[i] = v / A[i * R + i];
          }
          for (int i = 0; i < r; ++i) T->qcur[i] += xs[i];
        }
        T->s_status = st;
      }
      __syncthreads();
      if (T->s_status != CROM_OK) break;
    }  // GN iterations
    if (!ok) break;
    if (tid < r) p.q[(size_t)inst * r + tid] = T->qcur[tid];
    if (tid == 0) p.status[inst] = T->s_status;
  }
  if (!ok && tid == 0) atomicExch(&p.queue[1], 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tb, kTmemCols);
}

// Instances in order of decreasing |M_i| (counting sort), status preset to
// TIMEOUT (overwritten by the step for every instance it finishes), queue reset.
__global__ void order_kernel(const int* off, int n_inst, int max_samples, int* order, int* status, int* queue) {
  extern __shared__ int hist[];  // max_samples + 2 buckets, bucket b holds size (max_samples + 1 - b)
  const int nb = max_samples + 2;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < n_inst; i += blockDim.x) {
    const int sz = min(max(off[i + 1] - off[i], 0), max_samples + 1);
    atomicAdd(&hist[max_samples + 1 - sz], 1);
    status[i] = CROM_ERR_TIMEOUT;
  }
  __syncthreads();
  // exclusive scan: each thread owns a contiguous chunk, then a block scan of chunk sums
  __shared__ int part[1024];
  const int per = (nb + blockDim.x - 1) / blockDim.x;
  const int lo = threadIdx.x * per, hi = min(lo + per, nb);
  int sum = 0;
  for (int i = lo; i < hi; ++i) sum += hist[i];
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int d = 1; d < (int)blockDim.x; d <<= 1) {
    const int v = threadIdx.x >= (unsigned)d ? part[threadIdx.x - d] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int run = part[threadIdx.x] - sum;
  for (int i = lo; i < hi; ++i) {
    const int c = hist[i];
    hist[i] = run;
    run += c;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n_inst; i += blockDim.x) {
    const int sz = min(max(off[i + 1] - off[i], 0), max_samples + 1);
    order[atomicAdd(&hist[max_samples + 1 - sz], 1)] = i;
  }
  if (threadIdx.x == 0) {
    queue[0] = 0;
    queue[1] = 0;
  }
}

}  // namespace

int tc_step_max_samples() { return kMaxSamples; }

cudaError_t launch_step_tc(crom_ctx* ctx, const crom_step_desc* step, int n_inst, double* q,
                           const float* alpha, const float* vel, const int* s_off, const float* samples,
                           int max_samples, int* status, cudaStream_t s) {
  if ((size_t)n_inst > ctx->order_cap) {
    if (ctx->order) cudaFree(ctx->order);
    ctx->order = nullptr;
    ctx->order_cap = 0;
    cudaError_t e = cudaMalloc(&ctx->order, (size_t)n_inst * sizeof(int));
    if (e != cudaSuccess) return e;
    ctx->order_cap = n_inst;
  }
  order_kernel<<<1, 1024, (size_t)(max_samples + 2) * sizeof(int), s>>>(s_off, n_inst, max_samples, ctx->order,
                                                                       status, ctx->queue);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  StepParams p{};
  p.img = ctx->w.tc_img;
  p.img_bytes = (int)ctx->w.tc_img_bytes;
  p.L = ctx->desc.hidden;
  p.m = ctx->desc.m;
  p.r = ctx->desc.r;
  p.w1 = ctx->w.w1;
  p.b1 = ctx->w.b1;
  p.bh = ctx->w.bh;
  p.wout = ctx->w.wout;
  p.bout = ctx->w.bout;
  p.pde = step->pde;
  p.gn_iters = step->gn_iters;
  p.dt = step->dt;
  p.n_inst = n_inst;
  p.q = q;
  p.alpha = alpha;
  p.vel = vel;
  p.off = s_off;
  p.x = samples;
  p.max_samples = max_samples;
  p.status = status;
  p.order = ctx->order;
  p.queue = ctx->queue;
  const size_t smem = 1024 + (((size_t)p.img_bytes + 1023) & ~(size_t)1023) + 2 * kH + sizeof(Tail);
  e = cudaFuncSetAttribute(step_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = std::min(n_inst, ctx->num_sms);
  step_tc_kernel<<<grid, kThreads, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace crom
