// Batched latent step on the tcgen05 tensor cores (crom_step, CROM_PREC_BF16X2).
//
// One persistent launch per step, one CTA per SM holding the decoder's bf16
// hidden matrices in shared memory.  The CTA runs two independent groups of 256
// threads; each group takes whole instances from a queue ordered by |M_i|
// (largest first) and has its own operand buffers, TMEM columns, mbarrier and
// named barrier, so the UMMAs of one group overlap the CUDA-core epilogue of the
// other.  Inside a group, hidden unit u is TMEM lane u and is served by two
// threads (warps w and w + 4 of the group share a lane quadrant), each taking
// half of the 16 samples of a tile.
//
// Per instance, per Gauss-Newton iteration k, per tile of 16 samples
// (paper §4, Algorithm 3):
//
//  Step 1 (network inference): a forward pass whose UMMA columns are
//  (channel, sample) pairs, D[u][n] = sum_k W_l[u][k] H[k][n] (M = 128 units,
//  K = 128).  Iteration 0 carries the value, dg/dx_k and a single Laplacian
//  channel (d2z = W d2h with d2h = s''(z) sum_k (dz/dx_k)^2 + s'(z) d2z, the
//  m diagonal second-derivative channels of Algorithm 2 summed); iteration
//  k >= 1 carries the value at q^(k) and the difference channel
//  h(q^(k)) - h(q_n).  The epilogue (bias, ELU chain; s'(z) kept in TMEM for the
//  reverse pass) runs in FP32 registers and writes bf16 hi/lo operand pairs.
//
//  Step 2 (PDE update): Delta f_j = dt * alpha_i * Lap g(y_j) (or the
//  advection-diffusion form), kept per sample in global scratch (FP64).
//
//  Step 3 (network inversion): Jacobian rows dg/dq(y_j) from one reverse-mode
//  pass, delta_L = w_out * s'(z_L), delta_{l-1} = (W_l^T delta_l) * s'(z_{l-1}) on
//  the tensor cores (A = W_l read MN-major from the same shared image), then
//  J = W_1q^T delta_1 by a projection UMMA.  J^T J and J^T rho are accumulated
//  in FP64 from the FP32 rows (exact products); the r x r system is solved by
//  FP64 Cholesky and q is updated in FP64.
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

constexpr int kGroups = 2;
constexpr int kGT = 256;                 // threads per group
constexpr int kThreads = kGroups * kGT;
constexpr int kS = 16;                   // samples per tile
constexpr int kHalf = kS / 2;            // samples per thread
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kGroupCols = 256;     // TMEM columns per group
constexpr uint32_t kAcc = 0;             // accumulator, up to 64 columns
constexpr uint32_t kSig = 64;            // s'(z_l), l = 1..L (<= 5): 16 columns each
constexpr uint32_t kPrj = 144;           // projection output, 16 columns
constexpr uint32_t kWaitLimit = 1u << 25;
constexpr size_t kHBuf = (size_t)kTcWidth * 64 * 2;  // one bf16 operand buffer (<= 64 columns), 16 KB

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
  int* queue;   // [0] work counter, [1] timeout flag
  double* df;   // [n_samples] Delta f_j
};

struct __align__(16) Shared {
  uint64_t bar_w;
  uint32_t tmem_base;
  int pad;
  float w1x[2][kTcWidth];
  float w1q[16][kTcWidth];
  float bh[4][kTcWidth];
  float wout[kTcWidth];
};

struct __align__(16) Group {
  uint64_t bar_mma;
  int s_idx;
  int s_status;
  double qn[16];
  double qcur[16];
  double amat[15 * 16];
  float c1[kTcWidth];
  float dz1[kTcWidth];
  float xs[2][kS];
  float gout[4][kS];
  float rho[kS];
  float jt[kS][16];
};

// The projection UMMA reads 128 rows (two 64-column blocks) of a 64-column
// operand buffer; the rows past the buffer are never used, but the reads must stay
// inside the CTA's shared memory: at least 16 KB follow the last buffer.
static_assert(sizeof(Shared) + kGroups * sizeof(Group) >= 16384, "projection over-read must stay in smem");

__device__ __forceinline__ void group_sync(int g) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(kGT) : "memory");
}
__device__ __forceinline__ bool group_sync_and(int g, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)pred), "r"(1 + g), "r"(kGT)
      : "memory");
  return r != 0;
}

// Eight consecutive columns n0..n0+7 of row k as a bf16 hi/lo pair (one 16-byte
// chunk in each buffer).
__device__ __forceinline__ void split_store8(uint8_t* Hhi, uint8_t* Hlo, int k, int n0, const float (&v)[8]) {
  uint32_t hi[4], lo[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    hi[j] = pack_bf16(v[2 * j], v[2 * j + 1]);
    lo[j] = pack_bf16(v[2 * j] - bf16_lo_f(hi[j]), v[2 * j + 1] - bf16_hi_f(hi[j]));
  }
  const uint32_t off = mn_offset(k, n0);
  *reinterpret_cast<uint4*>(Hhi + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
  *reinterpret_cast<uint4*>(Hlo + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
}

// e^x - 1: degree-5 Taylor polynomial for |x| < 1/16 (truncation < 1.3e-9
// relative), the library function otherwise.
__device__ __forceinline__ float expm1_small(float x) {
  if (fabsf(x) < 0.0625f)
    return x * fmaf(x, fmaf(x, fmaf(x, fmaf(x, 1.f / 120.f, 1.f / 24.f), 1.f / 6.f), 0.5f), 1.f);
  return expm1f(x);
}

// s(a) - s(a - d) without cancellation, given e = exp(min(a, 0)): the difference
// channel carries h(q^(k)) - h(q_n), so the residual g(y, q^(k)) - g(y, q_n) - Delta f
// keeps its relative accuracy although the two evaluations agree to many digits.
__device__ __forceinline__ float elu_diff(float a, float d, float e) {
  const float b = a - d;
  if (a > 0.f && b > 0.f) return d;
  if (a <= 0.f && b <= 0.f) return -e * expm1_small(-d);
  const float sa = a > 0.f ? a : expm1f(a);
  const float sb = b > 0.f ? b : expm1f(b);
  return sa - sb;
}

// D(+)= A * B^T over K = 128 with the B operand as hi + lo parts.  a0: descriptor
// of A's first K slice; A is K-major (forward, W_l) or MN-major (reverse pass,
// W_l^T read from the same image); B descriptors are MN-major.
template <bool kAMN>
__device__ __forceinline__ void issue_layer(uint32_t d, uint64_t a0, uint64_t bhi, uint64_t blo, uint32_t idesc) {
#pragma unroll
  for (int kk = 0; kk < 8; ++kk)
    umma_f16(d, desc_add(a0, kAMN ? mnmajor_kslice(kk) : kmajor_kslice(128, kk)), desc_add(bhi, mnmajor_kslice(kk)),
             idesc, kk > 0);
#pragma unroll
  for (int kk = 0; kk < 8; ++kk)
    umma_f16(d, desc_add(a0, kAMN ? mnmajor_kslice(kk) : kmajor_kslice(128, kk)), desc_add(blo, mnmajor_kslice(kk)),
             idesc, 1);
}
// PRJ[n][j] = sum_u H[u][n] P[j][u] with H (MN-major A) as the hi + lo parts.
__device__ __forceinline__ void issue_proj(uint32_t d, uint64_t ahi, uint64_t alo, uint64_t p0) {
  constexpr uint32_t id = idesc_f16(128, 16, true, false, true);
#pragma unroll
  for (int kk = 0; kk < 8; ++kk)
    umma_f16(d, desc_add(ahi, mnmajor_kslice(kk)), desc_add(p0, kmajor_kslice(16, kk)), id, kk > 0);
#pragma unroll
  for (int kk = 0; kk < 8; ++kk)
    umma_f16(d, desc_add(alo, mnmajor_kslice(kk)), desc_add(p0, kmajor_kslice(16, kk)), id, 1);
}

__global__ void __launch_bounds__(kThreads, 1) step_tc_kernel(StepParams p) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x;
  const int g = tid / kGT, gt = tid % kGT;
  const int gw = gt >> 5;                 // warp within the group
  const int lq = gw & 3;                  // TMEM lane quadrant of this warp
  const int half = gw >> 2;               // which 8 samples of a tile
  const int u = lq * 32 + (gt & 31);      // hidden unit = TMEM lane
  const int s0 = half * kHalf;
  const uint32_t lane_base = (uint32_t)lq * 32;
  const int m = p.m, r = p.r, L = p.L;

  uint8_t* Wimg = sm;
  uint8_t* Hbase = sm + ((p.img_bytes + 1023) & ~1023);
  uint8_t* Hhi = Hbase + (size_t)g * 2 * kHBuf;
  uint8_t* Hlo = Hhi + kHBuf;
  Shared* S = reinterpret_cast<Shared*>(Hbase + (size_t)kGroups * 2 * kHBuf);
  Group* G = reinterpret_cast<Group*>(S + 1) + g;

  if (tid == 0) {
    mbar_init(&S->bar_w, 1);
    fence_mbar_init();
  }
  if (gt == 0) {
    mbar_init(&G->bar_mma, 1);
    fence_mbar_init();
  }
  if (tid < 32) {
    tmem_alloc(&S->tmem_base, kTmemCols);
    tmem_relinquish();
  }
  if (tid < kTcWidth) {
    for (int l = 0; l < L - 1; ++l) S->bh[l][tid] = p.bh[l * kTcWidth + tid];
    for (int k = 0; k < m; ++k) S->w1x[k][tid] = p.w1[tid * (m + r) + k];
    for (int j = 0; j < r; ++j) S->w1q[j][tid] = p.w1[tid * (m + r) + m + j];
    S->wout[tid] = p.wout[tid];
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tb = S->tmem_base + (uint32_t)g * kGroupCols;
  if (tid == 0) {
    mbar_arrive_expect_tx(&S->bar_w, (uint32_t)p.img_bytes);
    for (int o = 0; o < p.img_bytes; o += 16384)
      bulk_g2s(Wimg + o, p.img + o, (uint32_t)min(16384, p.img_bytes - o), &S->bar_w);
  }
  bool ok = __syncthreads_and(mbar_wait(&S->bar_w, 0, kWaitLimit));
  uint32_t phase = 0;
  const uint32_t wbase = smem_u32(Wimg);
  // Base UMMA descriptors; every operand slice is base + a compile-time offset.
  const uint64_t dW_k = smem_desc_sw128(wbase, 16, 1024);       // W_l as K-major A
  const uint64_t dW_mn = smem_desc_sw128(wbase, 16384, 1024);   // W_l^T as MN-major A
  const uint64_t dP = smem_desc_sw128(wbase + (uint32_t)(L - 1) * kTcLayerBytes, 16, 1024);
  const uint64_t dHhi = smem_desc_sw128(smem_u32(Hhi), 16384, 1024);
  const uint64_t dHlo = smem_desc_sw128(smem_u32(Hlo), 16384, 1024);
  const int ntri = r * (r + 1) / 2;
  const int n_entries = ntri + r;  // <= 135 < kGT
  // FP64 normal-equation entry owned by this thread
  int ea = -1, eb = -1;
  if (gt < ntri) {
    int a = 0, rem = gt;
    while (rem >= r - a) { rem -= r - a; ++a; }
    ea = a; eb = a + rem;
  } else if (gt < n_entries) {
    ea = gt - ntri; eb = -2;
  }
  const float wx0 = S->w1x[0][u], wx1 = (m > 1) ? S->w1x[1][u] : 0.f;
  const float wsq = wx0 * wx0 + wx1 * wx1;
  const float wo = S->wout[u];

  // Issue + wait of one UMMA stage of this group: one thread issues, the first
  // warp waits on the mbarrier, the rest wait at the group barrier; every thread
  // returns the same value.
  auto stage = [&](auto issue) -> bool {
    fence_proxy_async_smem();
    tc_fence_before();
    group_sync(g);
    bool done = true;
    if (gw == 0) {
      if (gt == 0) {
        tc_fence_after();
        issue();
        umma_commit(&G->bar_mma);
      }
      __syncwarp();
      done = mbar_wait(&G->bar_mma, phase, kWaitLimit);
    }
    done = group_sync_and(g, done);
    phase ^= 1;
    tc_fence_after();
    return done;
  };

  while (ok) {
    group_sync(g);  // everyone is done with the previous instance's group state
    if (gt == 0) G->s_idx = atomicAdd(&p.queue[0], 1);
    group_sync(g);
    const int idx = G->s_idx;
    if (idx >= p.n_inst) break;
    const int inst = p.order[idx];
    const int o0 = p.off[inst];
    const int M = p.off[inst + 1] - o0;
    if (M < r || M > p.max_samples) {
      if (gt == 0) p.status[inst] = CROM_ERR_INVALID_ARG;
      continue;
    }
    if (gt < r) {
      const double v = p.q[(size_t)inst * r + gt];
      G->qn[gt] = v;
      G->qcur[gt] = v;
    }
    if (gt == 0) G->s_status = CROM_OK;
    const float alpha = p.alpha[inst];
    group_sync(g);
    const int ntiles = (M + kS - 1) / kS;

    for (int it = 0; it < p.gn_iters && ok; ++it) {
      const bool first = (it == 0);
      const int nch = first ? 2 + m : 2;  // iteration 0: v, dx_1..dx_m, Lap; later: v(q^(k)), diff
      const int N = nch * kS;
      if (half == 0) {
        double c = (double)p.b1[u], dz = 0.0;
        for (int j = 0; j < r; ++j) {
          c += (double)S->w1q[j][u] * G->qcur[j];
          dz += (double)S->w1q[j][u] * (G->qcur[j] - G->qn[j]);
        }
        G->c1[u] = (float)c;
        G->dz1[u] = (float)dz;
      }
      double acc = 0.0;
      for (int t = 0; t < ntiles && ok; ++t) {
        const int ns = min(kS, M - t * kS);
        if (gt < kS) {
          const int s = gt < ns ? gt : 0;
          for (int k = 0; k < m; ++k) G->xs[k][gt] = p.x[(size_t)(o0 + t * kS + s) * m + k];
        }
        group_sync(g);
        // ---------------- layer 1 (CUDA cores)
        {
          const float c = G->c1[u], dz = G->dz1[u];
          float v[4][kHalf], sg[kHalf];
#pragma unroll
          for (int i = 0; i < kHalf; ++i) {
            float z = fmaf(wx0, G->xs[0][s0 + i], c);
            if (m > 1) z = fmaf(wx1, G->xs[1][s0 + i], z);
            const float e = __expf(fminf(z, 0.f));
            const bool pos = z > 0.f;
            const float s1 = pos ? 1.f : e, s2 = pos ? 0.f : e;
            sg[i] = s1;
            v[0][i] = pos ? z : e - 1.f;
            if (first) {
              v[1][i] = s1 * wx0;
              if (m > 1) {
                v[2][i] = s1 * wx1;
                v[3][i] = s2 * wsq;
              } else {
                v[2][i] = s2 * wsq;
              }
            } else {
              v[1][i] = elu_diff(z, dz, e);
            }
          }
          tmem_st8(taddr(tb, lane_base, kSig + s0), sg);
#pragma unroll
          for (int ch = 0; ch < 4; ++ch)
            if (ch < nch) split_store8(Hhi, Hlo, u, ch * kS + s0, v[ch]);
          tmem_st_wait();
        }
        // ---------------- hidden layers 2..L (tensor cores)
        const uint32_t id_fwd = idesc_f16(128, N, false, true, true);
        for (int l = 0; l < L - 1 && ok; ++l) {
          ok = stage([&] {
            issue_layer<false>(tb + kAcc, desc_add(dW_k, (uint32_t)l * kTcLayerBytes), dHhi, dHlo, id_fwd);
          });
          if (!ok) break;
          const float bias = S->bh[l][u];
          float v[4][kHalf], sg[kHalf];
#pragma unroll
          for (int ch = 0; ch < 4; ++ch)
            if (ch < nch) tmem_ld8(taddr(tb, lane_base, kAcc + ch * kS + s0), v[ch]);
          tmem_ld_wait();
#pragma unroll
          for (int i = 0; i < kHalf; ++i) {
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
                v[3][i] = fmaf(s2, fmaf(a, a, b * b), s1 * v[3][i]);
              } else {
                const float a = v[1][i];
                v[1][i] = s1 * a;
                v[2][i] = fmaf(s2, a * a, s1 * v[2][i]);
              }
            } else {
              v[1][i] = elu_diff(z, v[1][i], e);
            }
          }
          tmem_st8(taddr(tb, lane_base, kSig + (l + 1) * kS + s0), sg);
#pragma unroll
          for (int ch = 0; ch < 4; ++ch)
            if (ch < nch) split_store8(Hhi, Hlo, u, ch * kS + s0, v[ch]);
          tmem_st_wait();
        }
        if (!ok) break;
        // ---------------- output layer: PRJ[n][0] = w_out . h_L[:, n]
        ok = stage([&] { issue_proj(tb + kPrj, dHhi, dHlo, dP); });
        if (!ok) break;
        if (half == 0) {
          float v[8];
          tmem_ld8(taddr(tb, lane_base, kPrj), v);
          tmem_ld_wait();
          if (u < N) G->gout[u / kS][u % kS] = v[0];
        }
        group_sync(g);
        // ---------------- Step 2 and the residual rho_j
        if (gt < kS) {
          float rho = 0.f;
          if (gt < ns) {
            const int j = o0 + t * kS + gt;
            if (first) {
              const float lap = G->gout[m + 1][gt];
              double df;
              if (p.pde == CROM_PDE_HEAT) {
                df = p.dt * (double)alpha * (double)lap;
              } else {
                double adv = 0.0;
                for (int k = 0; k < m; ++k) adv += (double)p.vel[(size_t)j * m + k] * (double)G->gout[1 + k][gt];
                df = p.dt * (-adv + (double)alpha * (double)lap);
              }
              p.df[j] = df;
              rho = (float)(-df);
            } else {
              rho = (float)((double)G->gout[1][gt] - p.df[j]);
            }
          }
          G->rho[gt] = rho;
        }
        // ---------------- reverse pass for dg/dq at q^(k)
        {
          float sg[kHalf];
          tmem_ld8(taddr(tb, lane_base, kSig + (L - 1) * kS + s0), sg);
          tmem_ld_wait();
#pragma unroll
          for (int i = 0; i < kHalf; ++i) sg[i] *= wo;
          split_store8(Hhi, Hlo, u, s0, sg);  // delta_L
        }
        constexpr uint32_t id_bwd = idesc_f16(128, kS, true, true, true);
        for (int l = L - 2; l >= 0 && ok; --l) {
          // accumulator = W_{l+2}^T delta_{l+2}; times s'(z_{l+1}) gives delta_{l+1}
          ok = stage([&] {
            issue_layer<true>(tb + kAcc, desc_add(dW_mn, (uint32_t)l * kTcLayerBytes), dHhi, dHlo, id_bwd);
          });
          if (!ok) break;
          float v[kHalf], sg[kHalf];
          tmem_ld8(taddr(tb, lane_base, kAcc + s0), v);
          tmem_ld8(taddr(tb, lane_base, kSig + l * kS + s0), sg);
          tmem_ld_wait();
#pragma unroll
          for (int i = 0; i < kHalf; ++i) v[i] *= sg[i];
          split_store8(Hhi, Hlo, u, s0, v);
        }
        if (!ok) break;
        // J[s][j] = sum_u W_1q[u][j] delta_1[u][s]
        ok = stage([&] { issue_proj(tb + kPrj, dHhi, dHlo, dP); });
        if (!ok) break;
        if (gw == 0) {
          float v[16];
          tmem_ld16(taddr(tb, 0, kPrj), v);
          tmem_ld_wait();
          if (gt < kS) {
#pragma unroll
            for (int j = 0; j < 15; ++j) G->jt[gt][j] = v[j + 1];
          }
        }
        group_sync(g);
        // ---------------- normal equations in FP64 (exact products of FP32 rows)
        if (ea >= 0) {
          double s = 0.0;
          if (eb >= 0) {
            for (int i = 0; i < ns; ++i) s = fma((double)G->jt[i][ea], (double)G->jt[i][eb], s);
          } else {
            for (int i = 0; i < ns; ++i) s = fma((double)G->jt[i][ea], (double)G->rho[i], s);
          }
          acc += s;
        }
      }  // tiles
      if (!ok) break;
      const int R = r + 1;
      if (ea >= 0) {
        if (eb >= 0) {
          G->amat[ea * R + eb] = acc;
          G->amat[eb * R + ea] = acc;
        } else {
          G->amat[ea * R + r] = -acc;
        }
      }
      group_sync(g);
      if (gt == 0) {
        double* A = G->amat;
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
          for (int i = 0; i < r; ++i) G->qcur[i] += xs[i];
        }
        G->s_status = st;
      }
      group_sync(g);
      if (G->s_status != CROM_OK) break;
    }  // GN iterations
    if (!ok) break;
    if (gt < r) p.q[(size_t)inst * r + gt] = G->qcur[gt];
    if (gt == 0) p.status[inst] = G->s_status;
  }
  if (!ok && gt == 0) atomicExch(&p.queue[1], 1);
  tc_fence_before();
  __syncthreads();
  if (tid < 32) tmem_dealloc(S->tmem_base, kTmemCols);
}

// Instances in order of decreasing |M_i| (counting sort over sizes clamped to
// kBuckets - 1), status preset to TIMEOUT (overwritten by the step for every
// instance it finishes), queue reset.
constexpr int kBuckets = 4096;

__global__ void order_kernel(const int* off, int n_inst, int* order, int* status, int* queue) {
  __shared__ int hist[kBuckets];
  __shared__ int part[1024];
  for (int i = threadIdx.x; i < kBuckets; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < n_inst; i += blockDim.x) {
    const int sz = min(max(off[i + 1] - off[i], 0), kBuckets - 1);
    atomicAdd(&hist[kBuckets - 1 - sz], 1);
    status[i] = CROM_ERR_TIMEOUT;
  }
  __syncthreads();
  const int per = kBuckets / 1024;
  const int lo = threadIdx.x * per;
  int sum = 0;
  for (int i = lo; i < lo + per; ++i) sum += hist[i];
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int d = 1; d < 1024; d <<= 1) {
    const int v = threadIdx.x >= (unsigned)d ? part[threadIdx.x - d] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int run = part[threadIdx.x] - sum;
  for (int i = lo; i < lo + per; ++i) {
    const int c = hist[i];
    hist[i] = run;
    run += c;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n_inst; i += blockDim.x) {
    const int sz = min(max(off[i + 1] - off[i], 0), kBuckets - 1);
    order[atomicAdd(&hist[kBuckets - 1 - sz], 1)] = i;
  }
  if (threadIdx.x == 0) {
    queue[0] = 0;
    queue[1] = 0;
  }
}

}  // namespace

size_t tc_step_smem_bytes(int img_bytes) {
  return 1024 + (((size_t)img_bytes + 1023) & ~(size_t)1023) + (size_t)kGroups * 2 * kHBuf + sizeof(Shared) +
         kGroups * sizeof(Group);
}

cudaError_t launch_step_tc(crom_ctx* ctx, const crom_step_desc* step, int n_inst, double* q,
                           const float* alpha, const float* vel, const int* s_off, const float* samples,
                           int n_samples, int max_samples, int* status, cudaStream_t s) {
  if ((size_t)n_inst > ctx->order_cap) {
    if (ctx->order) cudaFree(ctx->order);
    ctx->order = nullptr;
    ctx->order_cap = 0;
    cudaError_t e = cudaMalloc(&ctx->order, (size_t)n_inst * sizeof(int));
    if (e != cudaSuccess) return e;
    ctx->order_cap = n_inst;
  }
  if ((size_t)n_samples > ctx->targets_cap) {
    if (ctx->targets) cudaFree(ctx->targets);
    ctx->targets = nullptr;
    ctx->targets_cap = 0;
    cudaError_t e = cudaMalloc(&ctx->targets, (size_t)std::max(n_samples, 1) * sizeof(double));
    if (e != cudaSuccess) return e;
    ctx->targets_cap = n_samples;
  }
  order_kernel<<<1, 1024, 0, s>>>(s_off, n_inst, ctx->order, status, ctx->queue);
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
  p.df = ctx->targets;
  const size_t smem = tc_step_smem_bytes(p.img_bytes);
  e = cudaFuncSetAttribute(step_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = std::min((n_inst + kGroups - 1) / kGroups, ctx->num_sms);
  step_tc_kernel<<<grid, kThreads, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace crom
