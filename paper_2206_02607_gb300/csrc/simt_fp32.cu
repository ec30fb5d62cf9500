// FP32 CUDA-core path: forward-mode decoder evaluation with derivative channels
// (paper Algorithm 2, App. E.1.1, extended to second order), used by
// crom_decode, FP32 crom_reconstruct and the plain FP32 crom_step.
//
// One CTA = KS threads per hidden unit (blockDim = KS * width) and a tile of S
// samples.  All channels of a (unit, sample) pair live in one thread, so the
// ELU chain rule needs no communication:
//   z = W h + b;  dz = W dh;  d2z = W d2h
//   h = s(z);     dh = s'(z) dz;  d2h = s''(z) dz^2 + s'(z) d2z
// The activations of the whole tile (width x S*C floats) sit in shared memory;
// the transposed hidden matrices are read through L1 (coalesced in the unit index).
// Each contraction over the width is split in KS slices (one per thread of a unit)
// whose partial sums are added through shared memory, which shortens the serial
// dependency chain of the small single-instance problems this path serves.
//
// The FP32 step spreads one instance over ceil(|M_i| / S) CTAs.  Each CTA forms
// its partial normal equations sum_j J_j J_j^T and sum_j J_j rho_j in FP64 from
// the FP32 Jacobian rows (exact products), writes them to scratch and takes a
// ticket; the CTA holding the last ticket adds the partials in tile order
// (deterministic), solves by FP64 Cholesky and updates q (paper §4.3, App. C).
// Nothing ever waits on another CTA.
#include <math.h>

#include <mutex>

#include "crom_internal.h"
#include "linalg.cuh"

namespace crom {
namespace {

constexpr int kMaxM = 3;
constexpr int kMaxR = 32;
constexpr int kKSplit = 4;  // threads per hidden unit (width <= 256 -> <= 1024 threads)

enum Mode { kModeDecode = 0, kModeRecon = 1, kModeStep = 2 };

struct FwdParams {
  int mode;
  // decoder
  int m, r, width, hidden;
  const float* w1;
  const float* b1;
  const float* wt;
  const float* bh;
  const float* wout;
  float bout;
  // channels carried: [value, (difference), dg/dx_k..., second order..., dg/dq_j...]
  int diff, nx, second, nq, C;
  int S;   // samples per CTA
  int LD;  // row stride (floats) of the activation buffers
  // inputs
  const double* q;  // [n][r]
  const int* off;   // decode: pt_off, step: s_off
  const float* x;   // [n][m]
  int n_pts;
  int n_inst;
  int act;        // CROM_ACT_ELU or CROM_ACT_SIREN
  float omega0;   // SIREN frequency
  // decode / recon
  float* out;
  unsigned want;
  // decode of a directional derivative (nq == 1): the one latent channel is seeded
  // with jvp_seed[instance][unit] = (W_1q u_i)[unit] instead of a W_1q column
  const float* jvp_seed;
  // step
  int iter;
  int pde;
  int coef_per_sample;  // alpha indexed by sample (1) or by instance (0)
  double dt;
  const float* alpha;
  const float* vel;
  int max_samples;
  double* qio;
  int* status;
  int n_samples;  // length of the sample arrays: every instance's range must lie inside
  double* partials;
  int max_tiles;
  int n_entries;
  int* counters;
  double* targets;  // Delta f_j per sample (FP64), written at GN iteration 0
  double* qbase;    // q_n per instance, written at GN iteration 0
};

__device__ __forceinline__ void elu3(float z, float& s0, float& s1, float& s2) {
  if (z > 0.f) {
    s0 = z;
    s1 = 1.f;
    s2 = 0.f;
  } else {
    float e = expf(z);
    s0 = expm1f(z);
    s1 = e;
    s2 = e;
  }
}

// s(a) - s(a - d) without cancellation: the difference channel carries
// h(q^(k)) - h(q_n) through the network, so that the Gauss-Newton residual
// g(y, q^(k)) - g(y, q_n) - Delta f keeps its relative accuracy when the two
// evaluations agree to many digits.
__device__ __forceinline__ float elu_diff(float a, float d) {
  const float b = a - d;
  if (a > 0.f && b > 0.f) return d;
  if (a <= 0.f && b <= 0.f) return -expf(a) * expm1f(-d);
  const float sa = a > 0.f ? a : expm1f(a);
  const float sb = b > 0.f ? b : expm1f(b);
  return sa - sb;
}

// SIREN, s(z) = sin(w z): s' = w cos(w z), s'' = -w^2 sin(w z).
__device__ __forceinline__ void siren3(float z, float w, float& s0, float& s1, float& s2) {
  float sn, cs;
  sincosf(w * z, &sn, &cs);
  s0 = sn;
  s1 = w * cs;
  s2 = -w * w * sn;
}

// sin(w a) - sin(w (a - d)) = 2 cos(w (a - d/2)) sin(w d / 2), without the
// cancellation of the direct difference.
__device__ __forceinline__ float siren_diff(float a, float d, float w) {
  return 2.f * cosf(w * (a - 0.5f * d)) * sinf(0.5f * w * d);
}

// Apply the activation chain in place to row `row` (pre-activation channels of
// one hidden unit) for the samples s0, s0 + ds, ... < S.
__device__ __forceinline__ void activate_row(float* row, const FwdParams& p, int sbeg, int ds) {
  const int C = p.C;
  for (int s = sbeg; s < p.S; s += ds) {
    float* c = row + s * C;
    float s0, s1, s2;
    const float za = c[0];
    if (p.act == CROM_ACT_SIREN) {
      siren3(za, p.omega0, s0, s1, s2);
      if (p.diff) c[1] = siren_diff(za, c[1], p.omega0);
    } else {
      elu3(za, s0, s1, s2);
      if (p.diff) c[1] = elu_diff(za, c[1]);
    }
    c[0] = s0;
    const int ox = 1 + p.diff;
    float zx[kMaxM];
    float sq = 0.f;
    for (int k = 0; k < p.nx; ++k) {
      zx[k] = c[ox + k];
      c[ox + k] = s1 * zx[k];
      sq += zx[k] * zx[k];
    }
    int o = ox + p.nx;
    if (p.second == kSecondPerK) {
      for (int k = 0; k < p.m; ++k) c[o + k] = s2 * zx[k] * zx[k] + s1 * c[o + k];
      o += p.m;
    } else if (p.second == kSecondLap) {
      c[o] = s2 * sq + s1 * c[o];
      o += 1;
    }
    for (int j = 0; j < p.nq; ++j) c[o + j] *= s1;
  }
}

__device__ int find_instance(const int* off, int n_inst, int point) {
  int lo = 0, hi = n_inst - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(&off[mid]) <= point) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// kJvp: the tangent-velocity decode, whose directional channel is seeded per
// instance (kept out of the other instantiation, whose register budget it would
// change).
template <bool kJvp>
__device__ __forceinline__ void fwd_fp32_body(const FwdParams& p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int W = p.width, S = p.S, C = p.C, LD = p.LD, m = p.m, r = p.r;
  // KS threads per hidden unit: thread (u, ks) owns unit u and the ks-th slice of
  // the K range of every contraction (and the samples s = ks mod KS elsewhere).
  const int tid = threadIdx.x, NT = blockDim.x;
  const int u = tid % W, ks = tid / W, KS = NT / W;
  const int NP = S * C;
  const int NPP = (NP + 15) & ~15;

  float* Hin = reinterpret_cast<float*>(smem_raw);
  float* Hout = Hin + W * LD;
  double* qs = reinterpret_cast<double*>(Hout + W * LD);  // [S][r]
  double* rho = qs + S * r;                               // [S]
  double* Amat = rho + S;                                 // [r][r + 1]
  double* dqs = Amat + r * (r + 1);                       // [r]: q^(k) - q_n
  float* xs = reinterpret_cast<float*>(dqs + r);          // [S][m]
  float* outv = xs + S * m;                               // [NPP]
  // [KS][W][16] split-K partial sums (16-byte aligned: also reused as doubles)
  float* red = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(outv + NPP) + 15) & ~uintptr_t(15));
  __shared__ int s_flag;

  // ---- which samples does this CTA own?
  int inst = 0, first = 0, ns = 0, ntiles = 0, msz = 0;
  if (p.mode == kModeStep) {
    inst = blockIdx.x;
    const int t = blockIdx.y;
    const int o0 = __ldg(&p.off[inst]);
    msz = __ldg(&p.off[inst + 1]) - o0;
    if (p.iter == 0) {
      if (msz < r || msz > p.max_samples || o0 < 0 || o0 + msz > p.n_samples) {
        if (t == 0 && tid == 0) p.status[inst] = CROM_ERR_INVALID_ARG;
        return;
      }
    } else if (p.status[inst] != CROM_OK) {
      return;
    }
    ntiles = (msz + S - 1) / S;
    if (t >= ntiles) return;
    first = o0 + t * S;
    ns = min(S, msz - t * S);
  } else {
    first = blockIdx.x * S;
    ns = min(S, p.n_pts - first);
    if (ns <= 0) return;
  }

  // ---- stage coordinates and latent codes (padding samples repeat the first one)
  for (int i = tid; i < S * m; i += NT) {
    const int s = i / m, k = i % m;
    xs[i] = p.x[(size_t)(first + (s < ns ? s : 0)) * m + k];
  }
  for (int i = tid; i < S * r; i += NT) {
    const int s = i / r, j = i % r;
    int code;
    if (p.mode == kModeStep) code = inst;
    else if (p.mode == kModeRecon) code = blockIdx.y;
    else code = find_instance(p.off, p.n_inst, first + (s < ns ? s : 0));
    qs[i] = (p.mode == kModeStep) ? p.qio[(size_t)code * r + j] : p.q[(size_t)code * r + j];
  }
  if (p.diff)
    for (int j = tid; j < r; j += NT) dqs[j] = p.qio[(size_t)inst * r + j] - p.qbase[(size_t)inst * r + j];
  for (int i = tid; i < 2 * W * LD; i += NT) Hin[i] = 0.f;  // zero both buffers incl. padding
  __syncthreads();

  // ---- layer 1: pre-activation channels of unit u, then the activation chain
  {
    float* row = Hin + u * LD;
    const float* w1 = p.w1 + (size_t)u * (m + r);
    const double b1 = (double)p.b1[u];
    double cshared = b1;
    const bool shared_q = (p.mode != kModeDecode);
    if (shared_q) {
      for (int j = 0; j < r; ++j) cshared += (double)w1[m + j] * qs[j];
    }
    double zd = 0.0;
    if (p.diff) {
      for (int j = 0; j < r; ++j) zd += (double)w1[m + j] * dqs[j];
    }
    for (int s = ks; s < S; s += KS) {
      double c = cshared;
      if (!shared_q) {
        c = b1;
        for (int j = 0; j < r; ++j) c += (double)w1[m + j] * qs[s * r + j];
      }
      float z = (float)c;
      for (int k = 0; k < m; ++k) z = fmaf(w1[k], xs[s * m + k], z);
      float* ch = row + s * C;
      ch[0] = z;
      if (p.diff) ch[1] = (float)zd;
      const int ox = 1 + p.diff;
      for (int k = 0; k < p.nx; ++k) ch[ox + k] = w1[k];
      int o = ox + p.nx;
      const int n2 = (p.second == kSecondPerK) ? m : (p.second == kSecondLap ? 1 : 0);
      for (int k = 0; k < n2; ++k) ch[o + k] = 0.f;
      o += n2;
      if (kJvp) {
        const int code = find_instance(p.off, p.n_inst, first + (s < ns ? s : 0));
        ch[o] = __ldg(&p.jvp_seed[(size_t)code * W + u]);
      } else {
        for (int j = 0; j < p.nq; ++j) ch[o + j] = w1[m + j];
      }
    }
    activate_row(row, p, ks, KS);
  }
  __syncthreads();

  // ---- hidden layers 2..hidden
  for (int l = 0; l < p.hidden - 1; ++l) {
    const float* Wt = p.wt + (size_t)l * W * W;
    float* orow = Hout + u * LD;
    const int kper = W / KS;
    for (int j0 = 0; j0 < NPP; j0 += 16) {
      float acc[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) acc[i] = 0.f;
      const float* hcol = Hin + j0;
#pragma unroll 4
      for (int k = ks * kper; k < (ks + 1) * kper; ++k) {
        const float wk = __ldg(&Wt[(size_t)k * W + u]);
        const float4* h4 = reinterpret_cast<const float4*>(hcol + k * LD);
        const float4 a = h4[0], b = h4[1], c = h4[2], d = h4[3];
        acc[0] = fmaf(wk, a.x, acc[0]);  acc[1] = fmaf(wk, a.y, acc[1]);
        acc[2] = fmaf(wk, a.z, acc[2]);  acc[3] = fmaf(wk, a.w, acc[3]);
        acc[4] = fmaf(wk, b.x, acc[4]);  acc[5] = fmaf(wk, b.y, acc[5]);
        acc[6] = fmaf(wk, b.z, acc[6]);  acc[7] = fmaf(wk, b.w, acc[7]);
        acc[8] = fmaf(wk, c.x, acc[8]);  acc[9] = fmaf(wk, c.y, acc[9]);
        acc[10] = fmaf(wk, c.z, acc[10]); acc[11] = fmaf(wk, c.w, acc[11]);
        acc[12] = fmaf(wk, d.x, acc[12]); acc[13] = fmaf(wk, d.y, acc[13]);
        acc[14] = fmaf(wk, d.z, acc[14]); acc[15] = fmaf(wk, d.w, acc[15]);
      }
      // add the KS partial sums of unit u: thread (u, ks) finishes 16 / KS of the columns
      float* mine = red + ((size_t)ks * W + u) * 16;
#pragma unroll
      for (int i = 0; i < 16; ++i) mine[i] = acc[i];
      __syncthreads();
      for (int i = ks * (16 / KS); i < (ks + 1) * (16 / KS); ++i) {
        float v = 0.f;
        for (int kk = 0; kk < KS; ++kk) v += red[((size_t)kk * W + u) * 16 + i];
        orow[j0 + i] = v;
      }
      __syncthreads();
    }
    const float bias = p.bh[(size_t)l * W + u];
    for (int s = ks; s < S; s += KS) orow[s * C] += bias;
    activate_row(orow, p, ks, KS);
    __syncthreads();
    float* tmp = Hin; Hin = Hout; Hout = tmp;
  }

  // ---- linear output layer: one thread per (sample, channel) column
  for (int t = tid; t < NP; t += NT) {
    float acc = 0.f;
    for (int k = 0; k < W; ++k) acc = fmaf(__ldg(&p.wout[k]), Hin[k * LD + t], acc);
    if (t % C == 0) acc += p.bout;
    outv[t] = acc;
  }
  __syncthreads();

  if (p.mode == kModeRecon) {
    if (tid < ns) p.out[(size_t)blockIdx.y * p.n_pts + first + tid] = outv[tid * C];
    return;
  }
  const int n2 = (p.second == kSecondPerK) ? m : (p.second == kSecondLap ? 1 : 0);
  const int ox = 1 + p.diff, o2 = ox + p.nx, oq = o2 + n2;
  if (p.mode == kModeDecode) {
    for (int s = tid; s < ns; s += NT) {
      const float* c = outv + s * C;
      const size_t N = (size_t)p.n_pts, pt = (size_t)(first + s);
      int row = 0;
      if (p.want & CROM_WANT_VAL) p.out[(row++) * N + pt] = c[0];
      if (p.want & CROM_WANT_DX)
        for (int k = 0; k < m; ++k) p.out[(row++) * N + pt] = c[ox + k];
      if (p.want & CROM_WANT_DXX)
        for (int k = 0; k < m; ++k) p.out[(row++) * N + pt] = c[o2 + k];
      if (p.want & CROM_WANT_LAP) {
        float lap = 0.f;
        for (int k = 0; k < n2; ++k) lap += c[o2 + k];
        p.out[(row++) * N + pt] = lap;
      }
      if (p.want & CROM_WANT_DQ)  // r rows, or the one directional row of a tangent decode
        for (int j = 0; j < p.nq; ++j) p.out[(row++) * N + pt] = c[oq + j];
    }
    return;
  }

  // ---- step: residual per sample (Step 2 at iteration 0), partial normal equations
  const int t = blockIdx.y;
  for (int s = tid; s < S; s += NT) {
    double res = 0.0;
    if (s < ns) {
      const float* c = outv + s * C;
      const size_t j = (size_t)(first + s);
      if (p.iter == 0) {
        double df;
        const double a = (double)p.alpha[p.coef_per_sample ? j : (size_t)inst];
        if (p.pde == CROM_PDE_HEAT) {
          df = p.dt * a * (double)c[o2];
        } else {
          double adv = 0.0;
          for (int k = 0; k < m; ++k) adv += (double)p.vel[j * m + k] * (double)c[ox + k];
          df = p.dt * (-adv + a * (double)c[o2]);
        }
        p.targets[j] = df;
        res = -df;  // g(y_j, q^(0)) - f_{n+1}(y_j) with f_{n+1} = g(y_j, q_n) + Delta f_j
      } else {
        // g(y_j, q^(k)) - f_{n+1}(y_j) = [g(y_j, q^(k)) - g(y_j, q_n)] - Delta f_j,
        // the bracket being the difference channel.
        res = (double)c[1] - p.targets[j];
      }
    }
    rho[s] = res;
  }
  __syncthreads();
  double* part = p.partials + ((size_t)inst * p.max_tiles + t) * p.n_entries;
  for (int e = tid; e < p.n_entries; e += NT) {
    const int ntri = r * (r + 1) / 2;
    double acc = 0.0;
    if (e < ntri) {
      int a = 0, rem = e;
      while (rem >= r - a) { rem -= r - a; ++a; }
      const int b = a + rem;
      for (int s = 0; s < ns; ++s)
        acc += (double)outv[s * C + oq + a] * (double)outv[s * C + oq + b];
    } else {
      const int a = e - ntri;
      for (int s = 0; s < ns; ++s) acc += (double)outv[s * C + oq + a] * rho[s];
    }
    part[e] = acc;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    const int ticket = atomicAdd(&p.counters[inst], 1);
    s_flag = (ticket == ntiles - 1);
  }
  __syncthreads();
  if (!s_flag) return;
  __threadfence();

  // ---- last CTA of the instance: reduce partials in a fixed order, solve, update q
  // (thread (j, e) adds the tiles j, j + per, ... of entry e; then the per partial
  // sums of each entry are added in order).
  const double* base = p.partials + (size_t)inst * p.max_tiles * p.n_entries;
  const int ne = p.n_entries;
  const int per = NT >= ne ? NT / ne : 1;
  double* red2 = reinterpret_cast<double*>(red);  // [per][ne]
  for (int idx = tid; idx < per * ne; idx += NT) {
    const int e = idx % ne, j = idx / ne;
    double acc = 0.0;
    for (int tt = j; tt < ntiles; tt += per) acc += __ldcg(&base[(size_t)tt * ne + e]);
    red2[(size_t)j * ne + e] = acc;
  }
  __syncthreads();
  for (int e = tid; e < ne; e += NT) {
    double acc = 0.0;
    for (int j = 0; j < per; ++j) acc += red2[(size_t)j * ne + e];
    const int ntri = r * (r + 1) / 2;
    if (e < ntri) {
      int a = 0, rem = e;
      while (rem >= r - a) { rem -= r - a; ++a; }
      const int b = a + rem;
      Amat[a * (r + 1) + b] = acc;
      Amat[b * (r + 1) + a] = acc;
    } else {
      Amat[(e - ntri) * (r + 1) + r] = -acc;  // right-hand side -J^T rho
    }
  }
  __syncthreads();
  if (tid < 32) {
    // Cholesky A = L L^T and the two triangular solves, spread over one warp
    __shared__ double s_invd[kMaxR];
    const int st = chol_solve_warp(Amat, s_invd, r, tid);
    if (st == CROM_OK && tid < r) {
      if (p.iter == 0) p.qbase[(size_t)inst * r + tid] = p.qio[(size_t)inst * r + tid];
      p.qio[(size_t)inst * r + tid] += Amat[tid * (r + 1) + r];
    }
    if (tid == 0) {
      p.status[inst] = st;
      p.counters[inst] = 0;
    }
  }
}

__global__ void fwd_fp32_kernel(FwdParams p) { fwd_fp32_body<false>(p); }
// up to 1024 threads per CTA: the bound keeps it within 64 registers
__global__ void __launch_bounds__(1024) fwd_fp32_jvp_kernel(FwdParams p) { fwd_fp32_body<true>(p); }

size_t fwd_smem_bytes(int W, int S, int C, int m, int r, int* LD_out) {
  const int NP = S * C;
  const int NPP = (NP + 15) & ~15;
  int LD = NPP + 4;
  *LD_out = LD;
  size_t b = (size_t)2 * W * LD * sizeof(float);
  b += (size_t)S * r * sizeof(double) + (size_t)S * sizeof(double) + (size_t)r * (r + 1) * sizeof(double) +
       (size_t)r * sizeof(double);
  b += (size_t)S * m * sizeof(float) + (size_t)NPP * sizeof(float);
  b += (size_t)kKSplit * W * 16 * sizeof(float);  // split-K partial sums
  return b + 64;
}

cudaError_t launch_fwd(FwdParams& p, dim3 grid, cudaStream_t s) {
  size_t smem = fwd_smem_bytes(p.width, p.S, p.C, p.m, p.r, &p.LD);
  auto kernel = p.jvp_seed ? fwd_fp32_jvp_kernel : fwd_fp32_kernel;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  kernel<<<grid, p.width * kKSplit, smem, s>>>(p);
  return cudaGetLastError();
}

void fill_decoder(FwdParams& p, const crom_ctx* ctx) {
  p.m = ctx->desc.m;
  p.r = ctx->desc.r;
  p.width = ctx->desc.width;
  p.hidden = ctx->desc.hidden;
  p.w1 = ctx->w.w1;
  p.b1 = ctx->w.b1;
  p.wt = ctx->w.wt;
  p.bh = ctx->w.bh;
  p.wout = ctx->w.wout;
  p.bout = ctx->w.bout;
  p.act = ctx->desc.activation;
  p.omega0 = ctx->desc.omega0;
}

// Largest tile that keeps the two activation buffers within 200 KB.
int pick_samples(int W, int C, int m, int r, int want) {
  int S = want;
  int LD;
  while (S > 1 && fwd_smem_bytes(W, S, C, m, r, &LD) > 200 * 1024) S >>= 1;
  return S;
}

}  // namespace

namespace {
// Layer-1 seed of the directional derivative along qdot_i = (q_i - q_prev_i) / dt:
// seed[i][u] = sum_j W_1[u][m + j] qdot_i[j], an FP64 sum rounded once.
__global__ void jvp_seed_kernel(const float* __restrict__ w1, int m, int r, int W, const double* __restrict__ q,
                                const double* __restrict__ q_prev, double inv_dt, int n_inst, float* seed) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_inst * W) return;
  const int i = e / W, u = e % W;
  double v = 0.0;
  for (int j = 0; j < r; ++j)
    v += (double)w1[(size_t)u * (m + r) + m + j] * ((q[(size_t)i * r + j] - q_prev[(size_t)i * r + j]) * inv_dt);
  seed[e] = (float)v;
}
}  // namespace

// Tangent velocity v = dg/dq . qdot as one forward-mode directional channel (the
// DQ channel machinery with the seed W_1q qdot instead of r columns of W_1q).
cudaError_t launch_tangent_fp32(const crom_ctx* ctx, int n_inst, const double* q, const double* q_prev, double dt,
                                const int* pt_off, const float* x, int n_pts, float* seed, float* out,
                                cudaStream_t s) {
  FwdParams p{};
  p.mode = kModeDecode;
  fill_decoder(p, ctx);
  const int W = p.width;
  jvp_seed_kernel<<<(n_inst * W + 255) / 256, 256, 0, s>>>(p.w1, p.m, p.r, W, q, q_prev, 1.0 / dt, n_inst, seed);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  p.nx = 0;
  p.second = kSecondNone;
  p.nq = 1;
  p.C = ChannelSet{p.nx, p.second, p.nq}.count(p.m);
  p.S = pick_samples(p.width, p.C, p.m, p.r, 8);
  p.q = q;
  p.off = pt_off;
  p.x = x;
  p.n_pts = n_pts;
  p.n_inst = n_inst;
  p.out = out;
  p.want = CROM_WANT_DQ;
  p.jvp_seed = seed;
  dim3 grid((n_pts + p.S - 1) / p.S, 1);
  return launch_fwd(p, grid, s);
}

cudaError_t launch_decode_fp32(const crom_ctx* ctx, int n_inst, const double* q, const int* pt_off,
                               const float* x, int n_pts, unsigned want, float* out, cudaStream_t s) {
  FwdParams p{};
  p.mode = kModeDecode;
  fill_decoder(p, ctx);
  const int m = p.m;
  p.nx = (want & (CROM_WANT_DX | CROM_WANT_DXX | CROM_WANT_LAP)) ? m : 0;
  p.second = (want & CROM_WANT_DXX) ? kSecondPerK : ((want & CROM_WANT_LAP) ? kSecondLap : kSecondNone);
  p.nq = (want & CROM_WANT_DQ) ? p.r : 0;
  p.C = ChannelSet{p.nx, p.second, p.nq}.count(m);
  p.S = pick_samples(p.width, p.C, m, p.r, 8);
  p.q = q;
  p.off = pt_off;
  p.x = x;
  p.n_pts = n_pts;
  p.n_inst = n_inst;
  p.out = out;
  p.want = want;
  dim3 grid((n_pts + p.S - 1) / p.S, 1);
  return launch_fwd(p, grid, s);
}

cudaError_t launch_recon_fp32(const crom_ctx* ctx, int n_codes, const double* q, int n_pts,
                              const float* x, float* out, cudaStream_t s) {
  FwdParams p{};
  p.mode = kModeRecon;
  fill_decoder(p, ctx);
  p.nx = 0;
  p.second = kSecondNone;
  p.nq = 0;
  p.C = 1;
  p.S = 32;
  p.q = q;
  p.x = x;
  p.n_pts = n_pts;
  p.n_inst = n_codes;
  p.out = out;
  dim3 grid((n_pts + p.S - 1) / p.S, n_codes);
  return launch_fwd(p, grid, s);
}

// Samples per CTA of the FP32 step: enough CTAs to cover the GPU at least twice
// when possible, within the shared-memory budget of the first iteration's channels.
int step_samples_per_cta(const crom_ctx* ctx, int n_inst, int max_samples) {
  const int m = ctx->desc.m, r = ctx->desc.r;
  const int C0 = ChannelSet{m, kSecondLap, r}.count(m);
  int S = 4;
  while (S > 1 && (long long)n_inst * ((max_samples + S - 1) / S) < 2LL * ctx->num_sms) S >>= 1;
  return pick_samples(ctx->desc.width, C0, m, r, S);
}

int step_fp32_max_tiles(const crom_ctx* ctx, int n_inst, int max_samples) {
  const int S = step_samples_per_cta(ctx, n_inst, max_samples);
  const long long t = ((long long)max_samples + S - 1) / S;
  return t > (1LL << 30) ? (1 << 30) : (int)t;
}

cudaError_t launch_step_fp32(crom_ctx* ctx, const crom_step_desc* step, int n_inst, double* q,
                             const float* alpha, const float* vel, const int* s_off,
                             const float* samples, int n_samples, int max_samples, int* status,
                             cudaStream_t s) {
  FwdParams p{};
  p.mode = kModeStep;
  fill_decoder(p, ctx);
  const int m = p.m, r = p.r;
  const int S = step_samples_per_cta(ctx, n_inst, max_samples);
  const int max_tiles = (max_samples + S - 1) / S;
  const int n_entries = r * (r + 1) / 2 + r;

  // Scratch: partial normal equations, per-instance tickets, per-sample targets.
  const size_t need_part = (size_t)n_inst * max_tiles * n_entries;
  if (need_part > ctx->partials_cap) {
    if (ctx->partials) cudaFree(ctx->partials);
    ++ctx->scratch_gen;
    ctx->partials = nullptr;
    ctx->partials_cap = 0;
    cudaError_t e = cudaMalloc(&ctx->partials, need_part * sizeof(double));
    if (e != cudaSuccess) return e;
    ctx->partials_cap = need_part;
  }
  if ((size_t)n_inst > ctx->counters_cap) {
    if (ctx->counters) cudaFree(ctx->counters);
    ++ctx->scratch_gen;
    ctx->counters = nullptr;
    ctx->counters_cap = 0;
    cudaError_t e = cudaMalloc(&ctx->counters, (size_t)n_inst * sizeof(int));
    if (e != cudaSuccess) return e;
    e = cudaMemset(ctx->counters, 0, (size_t)n_inst * sizeof(int));
    if (e != cudaSuccess) return e;
    ctx->counters_cap = n_inst;
  }
  if ((size_t)n_samples > ctx->targets_cap) {
    if (ctx->targets) cudaFree(ctx->targets);
    ++ctx->scratch_gen;
    ctx->targets = nullptr;
    ctx->targets_cap = 0;
    cudaError_t e = cudaMalloc(&ctx->targets, (size_t)n_samples * sizeof(double));
    if (e != cudaSuccess) return e;
    ctx->targets_cap = n_samples;
  }
  if ((size_t)n_inst * r > ctx->qbase_cap) {
    if (ctx->qbase) cudaFree(ctx->qbase);
    ++ctx->scratch_gen;
    ctx->qbase = nullptr;
    ctx->qbase_cap = 0;
    cudaError_t e = cudaMalloc(&ctx->qbase, (size_t)n_inst * r * sizeof(double));
    if (e != cudaSuccess) return e;
    ctx->qbase_cap = (size_t)n_inst * r;
  }

  p.S = S;
  p.off = s_off;
  p.x = samples;
  p.n_inst = n_inst;
  p.pde = step->pde;
  p.coef_per_sample = step->coef_per_sample;
  p.dt = step->dt;
  p.alpha = alpha;
  p.vel = vel;
  p.max_samples = max_samples;
  p.qio = q;
  p.status = status;
  p.n_samples = n_samples;
  p.partials = ctx->partials;
  p.max_tiles = max_tiles;
  p.n_entries = n_entries;
  p.counters = ctx->counters;
  p.targets = ctx->targets;
  p.qbase = ctx->qbase;
  if (max_tiles > 65535) return cudaErrorInvalidValue;
  dim3 grid(n_inst, max_tiles);
  for (int it = 0; it < step->gn_iters; ++it) {
    // Iteration 0: value, dg/dx_k, Laplacian, dg/dq at q_n.  Later iterations:
    // value and dg/dq at q^(k) plus the difference channel h(q^(k)) - h(q_n).
    p.iter = it;
    p.diff = (it == 0) ? 0 : 1;
    p.nx = (it == 0) ? m : 0;
    p.second = (it == 0) ? kSecondLap : kSecondNone;
    p.nq = r;
    p.C = 1 + p.diff + ChannelSet{p.nx, p.second, p.nq}.count(m) - 1;
    cudaError_t e = launch_fwd(p, grid, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace crom

// ---------------------------------------------------------------------------
// FP32 step without any device allocation (crom_step_noalloc).
//
// Some callers cannot allocate device memory at the time they step: a host
// application or framework that owns the device's memory through its own pool
// and forbids direct cudaMalloc/cudaFree by libraries it loads, and
// latency-critical loops where an allocation may synchronise the device.  For them this variant of the FP32 step
// takes its scratch (per-CTA partial normal equations, per-instance tickets,
// per-sample Delta f and per-instance q_n) from one file-scope device array of
// fixed size instead of the context's growable buffers.
//
// The array exists once per device for the life of the process (every GPU that
// loads the library holds its 8 MiB).  All calls on a device share it and it
// keeps the last call's contents: the tickets are cleared with a memset at every
// call; two calls whose kernels overlap on the GPU (different streams, no
// ordering between them) race on it and must not be issued.
namespace crom {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
void* g_noalloc_ptr[kMaxDevices] = {};
int g_noalloc_ready[kMaxDevices] = {};

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

size_t noalloc_scratch_capacity() { return kNoAllocScratchBytes; }

// Set-up, once per device and with that device current: the host-side name of
// the array is only a stand-in, the kernel needs its device address.
cudaError_t noalloc_scratch_address(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  if (!g_noalloc_ready[device]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[device] = ptr;
    g_noalloc_ready[device] = 1;
  }
  *out = g_noalloc_ptr[device];
  return cudaSuccess;
}

cudaError_t launch_step_fp32_noalloc(const crom_ctx* ctx, const crom_step_desc* step, int n_inst, double* q,
                                     const float* alpha, const float* vel, const int* s_off,
                                     const float* samples, int n_samples, int max_samples, int* status,
                                     cudaStream_t s, size_t* need_bytes) {
  FwdParams p{};
  p.mode = kModeStep;
  fill_decoder(p, ctx);
  const int m = p.m, r = p.r;
  const int S = step_samples_per_cta(ctx, n_inst, max_samples);
  const int max_tiles = (max_samples + S - 1) / S;
  const int n_entries = r * (r + 1) / 2 + r;
  // layout inside the static array
  const size_t off_cnt = 0;
  const size_t off_part = off_cnt + align256((size_t)n_inst * sizeof(int));
  const size_t off_tgt = off_part + align256((size_t)n_inst * max_tiles * n_entries * sizeof(double));
  const size_t off_qb = off_tgt + align256((size_t)n_samples * sizeof(double));
  const size_t total = off_qb + align256((size_t)n_inst * r * sizeof(double));
  *need_bytes = total;
  if (total > kNoAllocScratchBytes || max_tiles > 65535) return cudaErrorInvalidValue;
  void* base = nullptr;
  cudaError_t e = noalloc_scratch_address(ctx->device, &base);
  if (e != cudaSuccess) return e;
  unsigned char* b = static_cast<unsigned char*>(base);
  e = cudaMemsetAsync(b + off_cnt, 0, (size_t)n_inst * sizeof(int), s);
  if (e != cudaSuccess) return e;
  p.S = S;
  p.off = s_off;
  p.x = samples;
  p.n_inst = n_inst;
  p.pde = step->pde;
  p.coef_per_sample = step->coef_per_sample;
  p.dt = step->dt;
  p.alpha = alpha;
  p.vel = vel;
  p.max_samples = max_samples;
  p.qio = q;
  p.status = status;
  p.n_samples = n_samples;
  p.partials = reinterpret_cast<double*>(b + off_part);
  p.max_tiles = max_tiles;
  p.n_entries = n_entries;
  p.counters = reinterpret_cast<int*>(b + off_cnt);
  p.targets = reinterpret_cast<double*>(b + off_tgt);
  p.qbase = reinterpret_cast<double*>(b + off_qb);
  dim3 grid(n_inst, max_tiles);
  for (int it = 0; it < step->gn_iters; ++it) {
    p.iter = it;
    p.diff = (it == 0) ? 0 : 1;
    p.nx = (it == 0) ? m : 0;
    p.second = (it == 0) ? kSecondLap : kSecondNone;
    p.nq = r;
    p.C = 1 + p.diff + ChannelSet{p.nx, p.second, p.nq}.count(m) - 1;
    e = launch_fwd(p, grid, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace crom
