// Batched latent step on the tcgen05 tensor cores (crom_step, CROM_PREC_F16X2).
//
// One persistent launch per step, one CTA per SM holding the decoder's bf16
// hidden matrices in shared memory.  The CTA runs four independent groups of 128
// threads; each group takes whole instances from a queue ordered by |M_i|
// (largest first) and has its own 64-column operand block, 128 TMEM columns,
// mbarrier and named barrier, so the UMMAs of one group overlap the CUDA-core
// epilogues of the others.  Inside a group, hidden unit u is TMEM lane u and
// thread u of the group.
//
// Per instance, per Gauss-Newton iteration k, per tile of samples (paper §4,
// Algorithm 3; at iteration 0 forward tiles of 8 samples, taken in pairs by one
// reverse pass over 16; later 16-sample tiles, or 8 as the autotuner picks):
//
//  Step 1 (network inference): a forward pass whose UMMA columns are
//  (channel, sample) pairs, D[u][n] = sum_k W_l[u][k] H[k][n] (M = 128 units,
//  K = 128, 32 columns of bf16 hi parts followed by 32 columns of lo parts, one
//  N = 64 UMMA per K slice).  Iteration 0 carries the value, dg/dx_k and a single
//  Laplacian channel (d2z = W d2h with d2h = s''(z) sum_k (dz/dx_k)^2 + s'(z) d2z,
//  the m diagonal second-derivative channels of Algorithm 2 summed); iteration
//  k >= 1 carries the value at q^(k) and the difference channel
//  h(q^(k)) - h(q_n).  The epilogue (bias, ELU chain; s'(z) of layers 2..L kept in
//  TMEM for the reverse pass) runs in FP32 registers and writes bf16 hi/lo pairs.
//
//  Step 2 (PDE update): Delta f_j = dt * alpha_i * Lap g(y_j) (or the
//  advection-diffusion form), kept per sample in global scratch (FP64).
//
//  Step 3 (network inversion): Jacobian rows dg/dq(y_j) from one reverse-mode
//  pass, delta_L = w_out * s'(z_L), delta_{l-1} = (W_l^T delta_l) * s'(z_{l-1}) on
//  the tensor cores (A = W_l read MN-major from the same shared image, B = the hi
//  and lo parts of delta side by side); s'(z_1) is recomputed from the samples.
//  J = W_1q^T delta_1 by a projection UMMA.  J^T J and J^T rho are formed from
//  exact FP32 products (two-product) with compensated sums per tile and added in
//  FP64; the r x r system is solved by an FP64 Cholesky factorisation spread
//  over a warp; q is updated in FP64.
//
// The output layer w_out . h_L is formed on the CUDA cores in the last forward
// epilogue, in FP32 from h_L itself, for the channels the residual needs (a warp
// butterfly over the 32 units of each warp, then the four lane quadrants' partial
// sums).  The projection J = W_1q^T delta_1 is a UMMA against the 16-row bf16
// matrix P (rows 1..r = W_1q columns) that reads the activation buffer as the
// M = 128 operand, delta's hi parts in rows 0..kS-1 and lo parts in rows
// kS..2kS-1 (rows from 64 on read the next 16 KB of shared memory and are not
// used); the epilogue adds the two rows.
#include <math.h>

#include <algorithm>

#include "crom_internal.h"
#include "linalg.cuh"
#include "tc_common.cuh"

namespace crom {
namespace {

using namespace tc;

constexpr int kGroups = 4;
constexpr int kTPU = 1;                  // threads per hidden unit
constexpr int kGT = 128 * kTPU;          // threads per group
constexpr int kThreads = kGroups * kGT;
// Samples per forward tile at GN iteration 0 (4 channels): kTcTileS0 when the
// operands carry hi and lo parts (2 x 4 x kTcTileS0 columns fill one N = 64 UMMA),
// twice that with hi parts only (CROM_PREC_F16).
template <bool kLoP>
__host__ __device__ constexpr int tile_s0() {
  return kLoP ? kTcTileS0 : 2 * kTcTileS0;
}
// Samples per tile at later iterations (2 channels): kTcTileS1Large or
// kTcTileS1Small (doubled with hi parts only), a template parameter of the kernel
// chosen per context (crom_autotune measures both).
constexpr int kSMax = 4 * kTcTileS0;  // sample slots of a group
static_assert(2 * kTcTileS1Large <= kSMax && 2 * tile_s0<false>() <= kSMax, "sample slots");
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kGroupCols = 128;     // TMEM columns per group
// Accumulator in columns 0..63 (forward: W h_hi in 0..31, W h_lo in 32..63, or
// W h_hi in 0..63 with hi parts only; reverse: hi part in 0..kS-1, lo part in
// kS..2kS-1; projections: 16 columns); s'(z_l) of hidden layers l = 2..L (<= 5)
// from column 64, kS FP32 columns each, or kS / 2 columns of f16 pairs with hi
// parts only (whose tiles hold twice the samples).
constexpr uint32_t kAcc = 0;
constexpr uint32_t kSig = 64;
// Forward operand block of a group: 64 columns, the bf16 hi parts of the (channel,
// sample) pairs in columns 0..kLo-1 and their lo parts in kLo..2 kLo-1.
constexpr int kLo = 32;
constexpr uint32_t kWaitLimit = 1u << 25;
constexpr double kArmijoC1 = 1e-4;      // sufficient-decrease constant of the line search
constexpr size_t kHBuf = (size_t)kTcWidth * 64 * 2;  // one 64-column bf16 MN-major block (16 KB) per group

struct StepParams {
  const uint8_t* img;
  int img_bytes;
  // power-of-two channel scales (f16 operand range): sx for dg/dx_k (sxi = 1/sx,
  // sx2i = 1/sx^2 for the Laplacian), sr for the reverse pass (sri = 1/sr)
  float sx, sxi, sx2i, sr, sri;
  int L;  // hidden layers
  int r;
  const float* w1;
  const float* b1;
  const float* bh;
  const float* wout;
  float bout;
  int pde;
  int coef_per_sample;  // alpha indexed by sample (1) or by instance (0)
  int gn_iters;
  int line_search;  // backtracking halvings per GN iteration (0: full steps)
  double dt;
  int n_inst;
  double* q;
  const float* alpha;
  const float* vel;
  const int* off;
  const float* x;
  int max_samples;
  int n_samples;  // length of the sample arrays: every instance's range must lie inside
  int* status;
  const int* order;
  int* queue;   // [0] work counter, [1] timeout flag
  double* df;   // [n_samples] Delta f_j
  // decode mode (crom_decode_tc, the kernel's kDec instantiations): Step 1 alone at the points
  // x[0 .. n_samples) of the instances off[], written channel-major to dec_out
  // [rows][n_samples]; the output row of each channel, -1 where not wanted
  float* dec_out;
  int row_val, row_dx, row_lap, row_dq;
};
// Points per work item of the decode mode (a chunk may span several instances).
constexpr int kDecChunk = 256;

struct __align__(16) Shared {
  uint64_t bar_w;
  uint32_t tmem_base;
  int pad;
  float w1x[2][kTcWidth];
  float bh[4][kTcWidth];
  float wout[kTcWidth];
};

struct __align__(16) Group {
  uint64_t bar_mma;
  int s_idx;
  int s_status;
  double qn[16];
  double qcur[16];
  double qtry[16];    // line search: trial point q + a delta
  double delta[16];   // line search: the GN direction
  double phi0, phi, slope;
  double amat[15 * 16];
  double invd[16];
  float c1[kTcWidth];
  float dz1[kTcWidth];
  float dmax[4];
  float xs[2][kSMax];
  float rho[kSMax];
  float zero[kSMax];
  // Jacobian rows from the hi (rows 0..15) and the lo (rows 16..31) parts of delta_1,
  // or rows 0..31 of up to 32 samples with hi parts only (jrow)
  float jt[2][16][16];
};
// Row s of the Jacobian rows from part `part` (0 = hi, 1 = lo) of delta_1.
__device__ __forceinline__ float* jrow(Group* G, int part, int s) { return &G->jt[0][0][0] + (part * 16 + s) * 16; }

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

// kC (4 or 8) consecutive columns of row k as an f16 hi/lo pair: the hi parts go
// to columns n_hi.., the lo parts to n_lo.. of the MN-major operand H (columns
// >= 64 lie in the next 64-column block); one 2 kC-byte chunk each.  Without lo
// parts (kLoP false) only the hi chunk is written.
template <int kC, bool kLoP>
__device__ __forceinline__ void split_store(uint8_t* H, int k, int n_hi, int n_lo, const float* v) {
  uint32_t hi[kC / 2], lo[kC / 2];
#pragma unroll
  for (int j = 0; j < kC / 2; ++j) {
    hi[j] = pack_f16(v[2 * j], v[2 * j + 1]);
    if (kLoP) lo[j] = pack_f16_lo(hi[j], v[2 * j], v[2 * j + 1]);
  }
  if constexpr (kC == 8) {
    *reinterpret_cast<uint4*>(H + mn_offset(k, n_hi)) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
    if (kLoP) *reinterpret_cast<uint4*>(H + mn_offset(k, n_lo)) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
  } else {
    static_assert(kC == 4, "chunks of 4 or 8 columns");
    *reinterpret_cast<uint2*>(H + mn_offset(k, n_hi)) = make_uint2(hi[0], hi[1]);
    if (kLoP) *reinterpret_cast<uint2*>(H + mn_offset(k, n_lo)) = make_uint2(lo[0], lo[1]);
  }
}

// s'(z) of kC = 8 samples of hidden layer l + 2 in tensor memory (region of kSS
// samples per layer from column kSig): FP32 columns with hi/lo operands; with hi
// parts only (tiles of twice the samples) f16 pairs, sample 2i in the low half of
// column i, rounded like the f16 deltas they multiply.
template <bool kLoP>
__device__ __forceinline__ void store_sig(uint32_t tb, uint32_t lb, int kSS, int l, int slot, const float (&sg)[8]) {
  if constexpr (kLoP) {
    tmem_st8(taddr(tb, lb, kSig + l * kSS + slot), sg);
  } else {
    const float pk[4] = {__uint_as_float(pack_f16(sg[0], sg[1])), __uint_as_float(pack_f16(sg[2], sg[3])),
                         __uint_as_float(pack_f16(sg[4], sg[5])), __uint_as_float(pack_f16(sg[6], sg[7]))};
    tmem_st4(taddr(tb, lb, kSig + l * (kSS / 2) + slot / 2), pk);
  }
}
// Issues the load of store_sig's columns; unpack_sig (after tmem_ld_wait) gives the values.
template <bool kLoP>
__device__ __forceinline__ void load_sig(uint32_t tb, uint32_t lb, int kSS, int l, int slot, float (&sg)[8]) {
  if constexpr (kLoP) {
    tmem_ld8(taddr(tb, lb, kSig + l * kSS + slot), sg);
  } else {
    float pk[4];
    tmem_ld4(taddr(tb, lb, kSig + l * (kSS / 2) + slot / 2), pk);
#pragma unroll
    for (int i = 0; i < 4; ++i) sg[i] = pk[i];
  }
}
__device__ __forceinline__ void f16x2_to_f32(uint32_t v, float& a, float& b) {
  asm("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %2;\n\tcvt.f32.f16 %0, l;\n\tcvt.f32.f16 %1, h;\n\t}"
      : "=f"(a), "=f"(b)
      : "r"(v));
}
template <bool kLoP>
__device__ __forceinline__ void unpack_sig(float (&sg)[8]) {
  if constexpr (!kLoP) {
#pragma unroll
    for (int i = 3; i >= 0; --i) f16x2_to_f32(__float_as_uint(sg[i]), sg[2 * i], sg[2 * i + 1]);
  }
}

// (e^x - 1) / x for |x| < 1/16 by the degree-4 polynomial of the Taylor series of
// e^x - 1 divided by x (truncation < 1.3e-9 relative).
__device__ __forceinline__ float expm1_over_x(float x) {
  return fmaf(x, fmaf(x, fmaf(x, fmaf(x, 1.f / 120.f, 1.f / 24.f), 1.f / 6.f), 0.5f), 1.f);
}
// s(a) - s(a - d) for the cases the inline path leaves: mixed signs of a and
// a - d, or both non-positive with |d| >= 1/16.  Kept out of line: these cases are
// rare, and inlining them at every activation multiplies the kernel's code size.
__device__ __noinline__ float elu_diff_slow(float a, float d, float e) {
  const float b = a - d;
  if (a <= 0.f && b <= 0.f) return -e * expm1f(-d);
  const float sa = a > 0.f ? a : expm1f(a);
  const float sb = b > 0.f ? b : expm1f(b);
  return sa - sb;
}
// s(a) - s(a - d) without cancellation, given e = exp(min(a, 0)): the difference
// channel carries h(q^(k)) - h(q_n), so the residual g(y, q^(k)) - g(y, q_n) - Delta f
// keeps its relative accuracy although the two evaluations agree to many digits.
// Both positive: d; both non-positive: e^a - e^(a-d) = -e^a (e^(-d) - 1).
// The channel is carried scaled by a power of two, ds = d * sc (sci = 1 / sc), so
// that its f16 operands stay in range; the result is returned with the same scale.
__device__ __forceinline__ float elu_diff(float a, float ds, float e, float sc, float sci) {
  const float d = ds * sci;
  const float b = a - d;
  if (a > 0.f && b > 0.f) return ds;
  if (a <= 0.f && b <= 0.f && fabsf(d) < 0.0625f) return e * ds * expm1_over_x(-d);
  return elu_diff_slow(a, d, e) * sc;
}

// Forward activation chain of kC samples of one hidden unit, in place, on packed
// pairs.  v[0] holds the value channel's pre-activation z (bias included); at
// iteration 0 v[1..m] the gradient channels dz/dx_k and v[kCh-1] the Laplacian
// channel; later v[1] the difference channel.  sg receives s'(z).
//   h = s(z); dh/dx_k = s'(z) dz/dx_k; Lap h = s''(z) sum_k (dz/dx_k)^2 + s'(z) Lap z.
template <int kM, bool kFirst, int kCh, int kC>
__device__ __forceinline__ void act(float (&v)[kCh][kC], float (&sg)[kC], float dsc, float dsci) {
#pragma unroll
  for (int j = 0; j < kC / 2; ++j) {
    const int i0 = 2 * j, i1 = 2 * j + 1;
    const float z0 = v[0][i0], z1 = v[0][i1];
    float e0, e1;
    const f32x2 h = elu2(pk2(z0, z1), e0, e1);
    const float s10 = z0 > 0.f ? 1.f : e0, s11 = z1 > 0.f ? 1.f : e1;
    sg[i0] = s10;
    sg[i1] = s11;
    unpk2(h, v[0][i0], v[0][i1]);
    if (kFirst) {
      const f32x2 s1 = pk2(s10, s11);
      const f32x2 s2 = pk2(z0 > 0.f ? 0.f : e0, z1 > 0.f ? 0.f : e1);
      const f32x2 a = pk2(v[1][i0], v[1][i1]);
      f32x2 sq = mul2(a, a);
      unpk2(mul2(s1, a), v[1][i0], v[1][i1]);
      if (kM > 1) {
        const f32x2 b = pk2(v[2][i0], v[2][i1]);
        sq = fma2(b, b, sq);
        unpk2(mul2(s1, b), v[2][i0], v[2][i1]);
      }
      const f32x2 lz = pk2(v[kCh - 1][i0], v[kCh - 1][i1]);
      unpk2(fma2(s2, sq, mul2(s1, lz)), v[kCh - 1][i0], v[kCh - 1][i1]);
    } else {
      v[1][i0] = elu_diff(z0, v[1][i0], e0, dsc, dsci);
      v[1][i1] = elu_diff(z1, v[1][i1], e1, dsc, dsci);
    }
  }
}

// D = A * B^T over K = 128, one UMMA per K slice, issued by warp-converged code
// (all lanes run it, an elected lane issues).  A is K-major (forward, W_l) or
// MN-major (reverse pass, W_l^T read from the same image); B is the MN-major
// activation buffer holding the hi and lo parts side by side along N, so each
// UMMA yields W h_hi and W h_lo in separate accumulator columns.
template <bool kAMN>
__device__ __forceinline__ void issue_layer(uint32_t d, uint64_t a0, uint64_t b0, uint32_t idesc) {
#pragma unroll
  for (int kk = 0; kk < 8; ++kk)
    umma_f16_warp(d, desc_add(a0, kAMN ? mnmajor_kslice(kk) : kmajor_kslice(128, kk)),
                  desc_add(b0, mnmajor_kslice(kk)), idesc, kk > 0);
}
// PRJ[n][j] = sum_u H[u][n] P[j][u]: the activation buffer (both 64-column blocks)
// is the MN-major A operand, so row n < 64 projects a hi part and row 64 + n the
// matching lo part.
__device__ __forceinline__ void issue_proj(uint32_t d, uint64_t a0, uint64_t p0) {
  constexpr uint32_t id = idesc_f16(128, 16, true, false, false);
#pragma unroll
  for (int kk = 0; kk < 8; ++kk)
    umma_f16_warp(d, desc_add(a0, mnmajor_kslice(kk)), desc_add(p0, kmajor_kslice(16, kk)), id, kk > 0);
}

// Per-thread view of the group it belongs to.
struct Lane {
  int g, gt, gw, u, part;
  uint32_t lane_base, tb;
  uint8_t* H;
  Shared* S;
  Group* G;
  uint64_t dW_k, dW_mn, dP, dH;
  float wx0, wx1, wsq, wo;
  // Power-of-two scales of the channels carried in f16: gx0/gx1 = W_1x[:, k] * sx
  // (dg/dx_k channels, scale sx; the Laplacian channel then carries sx^2), wos =
  // w_out * sr (reverse pass), dsc = difference-channel scale of the current GN
  // iteration (dsci = 1 / dsc)
  float gx0, gx1, wos, dsc, dsci;
  uint32_t phase;
};

// Normal-equation entries owned by a thread (up to two: r = 15 has 135 of them and
// a group 128 threads): (ea, eb) of J^T J, (ea, -2) of J^T rho, ea = -3 for rho^T rho
// (the line search's objective), ea = -1 for none; acc holds the running sums.
struct Own {
  int ea[2], eb[2];
  double acc[2];
};

// One UMMA stage of the group: fence the epilogue's shared-memory writes, meet,
// the first warp issues and commits (one elected lane) and waits on the mbarrier,
// the rest wait at the group barrier.  Returns the group-uniform completion flag.
enum StageKind { kStageFwd = 0, kStageBwd = 1, kStageProj = 2 };
template <StageKind kKind>
__device__ __forceinline__ bool stage(Lane& c, int layer, uint32_t idesc) {
  fence_proxy_async_smem();
  tc_fence_before();
  group_sync(c.g);
  bool done = true;
  if (c.gw == 0) {
    tc_fence_after();
    if (kKind == kStageFwd)
      issue_layer<false>(c.tb + kAcc, desc_add(c.dW_k, (uint32_t)layer * kTcLayerBytes), c.dH, idesc);
    else if (kKind == kStageBwd)
      issue_layer<true>(c.tb + kAcc, desc_add(c.dW_mn, (uint32_t)layer * kTcLayerBytes), c.dH, idesc);
    else
      issue_proj(c.tb + kAcc, c.dH, c.dP);
    umma_commit_warp(&c.G->bar_mma);
    done = mbar_wait(&c.G->bar_mma, c.phase, kWaitLimit);
  }
  done = group_sync_and(c.g, done);
  c.phase ^= 1;
  tc_fence_after();
  return done;
}

// s + p = t + err exactly (Knuth's two-sum); t replaces s, err is added to comp.
__device__ __forceinline__ void two_sum_into(float& s, float& comp, float p) {
  const float t = __fadd_rn(s, p);
  const float bp = __fsub_rn(t, s);
  comp += __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
  s = t;
}

// Exact product-sum of up to kSMax FP32 pairs: two-product (a*b = p + e exactly by
// one FMA) and a compensated (two-sum) accumulation of the p, in FP32; returned in
// FP64.  Relative error ~2^-46, well below the FP32 inputs' own rounding.  A factor
// is the FP32 sum of two parts (a0 + a1) where kTA (kTB) is set, else a0 (b0).
// Four interleaved accumulators (element i goes to i mod 4) shorten the dependent
// chain; they are merged by two-sums in a fixed order.
template <bool kTA, bool kTB>
__device__ __forceinline__ double dot_exact(const float* a0, const float* a1, int sa, const float* b0,
                                            const float* b1, int sb, int n) {
  float s[4] = {0.f, 0.f, 0.f, 0.f}, comp[4] = {0.f, 0.f, 0.f, 0.f};
  for (int i0 = 0; i0 < n; i0 += 4) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int i = i0 + k;
      if (i < n) {
        const float x = kTA ? __fadd_rn(a0[i * sa], a1[i * sa]) : a0[i * sa];
        const float y = kTB ? __fadd_rn(b0[i * sb], b1[i * sb]) : b0[i * sb];
        const float p = __fmul_rn(x, y);  // rounded product (kept out of FMA contraction)
        const float e = fmaf(x, y, -p);   // its exact rounding error
        two_sum_into(s[k], comp[k], p);
        comp[k] += e;
      }
    }
  }
  two_sum_into(s[0], comp[0], s[1]);
  two_sum_into(s[2], comp[2], s[3]);
  two_sum_into(s[0], comp[0], s[2]);
  comp[0] += comp[1] + (comp[2] + comp[3]);
  return (double)s[0] + (double)comp[0];
}

// Sum over the 32 lanes of a warp (32 hidden units) of 8 per-lane values v[s]: three
// exchange rounds halve the set each time (offsets 16, 8, 4), two more add across the
// remaining lanes (offsets 2, 1).  Lane l ends with the total of sample (l >> 2) & 7.
__device__ __forceinline__ float warp_sum8(const float (&v)[8], int lane) {
  float a[4], b[2];
  const bool u16 = lane & 16, u8 = lane & 8, u4 = lane & 4;
#pragma unroll
  for (int s = 0; s < 4; ++s)
    a[s] = (u16 ? v[s + 4] : v[s]) + __shfl_xor_sync(0xffffffffu, u16 ? v[s] : v[s + 4], 16);
#pragma unroll
  for (int s = 0; s < 2; ++s)
    b[s] = (u8 ? a[s + 2] : a[s]) + __shfl_xor_sync(0xffffffffu, u8 ? a[s] : a[s + 2], 8);
  float t = (u4 ? b[1] : b[0]) + __shfl_xor_sync(0xffffffffu, u4 ? b[0] : b[1], 4);
  t += __shfl_xor_sync(0xffffffffu, t, 2);
  t += __shfl_xor_sync(0xffffffffu, t, 1);
  return t;
}

// s'(z_1) of kC samples of this thread's unit, recomputed exactly as the
// forward pass formed it (same FP32 operations), for the last reverse step.
template <int kM, int kC>
__device__ __forceinline__ void sig1(const Lane& c, const Group* G, float cc, int s, float (&sg)[kC]) {
#pragma unroll
  for (int i = 0; i < kC; i += 2) {
    float z0 = fmaf(c.wx0, G->xs[0][s + i], cc), z1 = fmaf(c.wx0, G->xs[0][s + i + 1], cc);
    if (kM > 1) {
      z0 = fmaf(c.wx1, G->xs[1][s + i], z0);
      z1 = fmaf(c.wx1, G->xs[1][s + i + 1], z1);
    }
    float e0, e1;
    (void)elu2(pk2(z0, z1), e0, e1);
    sg[i] = z0 > 0.f ? 1.f : e0;
    sg[i + 1] = z1 > 0.f ? 1.f : e1;
  }
}

// Steps after the residual of kSm samples (the group's sample slots 0..kSm-1): the
// reverse pass for dg/dq at q^(k) (delta hi parts in columns 0..kSm-1, lo parts in
// kSm..2kSm-1), the Jacobian projection and these samples' share of J^T J, J^T rho
// (and rho^T rho for the line search).  s'(z_l) of hidden layer l + 2 is read from
// TMEM column kSig + l * kSS + slot.
template <int kM, int kSm, int kSS, bool kLoP, bool kDec = false>
__device__ __forceinline__ bool reverse_tile(Lane& c, const StepParams& p, int j0, int ns, Own& o) {
  constexpr int kPer = kSm / kTPU;
  constexpr int kC = kPer < 8 ? kPer : 8;
  Group* G = c.G;
  const int u = c.u, s0 = c.part * kPer;
  const uint32_t lb = c.lane_base, tb = c.tb;
  // ---------------- reverse pass
#pragma unroll 1
  for (int h8 = 0; h8 < kPer; h8 += kC) {
    static_assert(kC == 8, "s'(z) is kept in chunks of 8 samples");
    float sg[kC];
    load_sig<kLoP>(tb, lb, kSS, p.L - 2, s0 + h8, sg);
    tmem_ld_wait();
    unpack_sig<kLoP>(sg);
#pragma unroll
    for (int i = 0; i < kC; ++i) sg[i] *= c.wos;
    split_store<kC, kLoP>(c.H, u, s0 + h8, kSm + s0 + h8, sg);  // delta_L
  }
  constexpr uint32_t id_bwd = idesc_f16(128, kLoP ? 2 * kSm : kSm, true, true, false);
  for (int l = p.L - 2; l >= 0; --l) {
    // accumulator = W_{l+2}^T delta_{l+2}; times s'(z_{l+1}) gives delta_{l+1}
    if (!stage<kStageBwd>(c, l, id_bwd)) return false;
    const float cc = G->c1[u];
#pragma unroll 1
    for (int h8 = 0; h8 < kPer; h8 += kC) {
      float v[kC], w[kC], sg[kC];
      tmem_ldc(taddr(tb, lb, kAcc + s0 + h8), v);
      if (kLoP) tmem_ldc(taddr(tb, lb, kAcc + kSm + s0 + h8), w);
      if (l > 0) load_sig<kLoP>(tb, lb, kSS, l - 1, s0 + h8, sg);
      else sig1<kM, kC>(c, G, cc, s0 + h8, sg);
      tmem_ld_wait();
      if (l > 0) unpack_sig<kLoP>(sg);
      if (kLoP) {
#pragma unroll
        for (int i = 0; i < kC; i += 2)
          unpk2(mul2(add2(pk2(v[i], v[i + 1]), pk2(w[i], w[i + 1])), pk2(sg[i], sg[i + 1])), v[i], v[i + 1]);
      } else {
#pragma unroll
        for (int i = 0; i < kC; i += 2) unpk2(mul2(pk2(v[i], v[i + 1]), pk2(sg[i], sg[i + 1])), v[i], v[i + 1]);
      }
      split_store<kC, kLoP>(c.H, u, s0 + h8, kSm + s0 + h8, v);
    }
  }
  // J[s][j] = sum_u W_1q[u][j] delta_1[u][s]: rows s (hi) and kSm + s (lo)
  constexpr int kRows = kLoP ? 2 * kSm : kSm;
  if (!stage<kStageProj>(c, 0, 0)) return false;
  if (c.gw < (kRows + 31) / 32) {
    float v[16];
    tmem_ld16(taddr(tb, lb, kAcc), v);
    tmem_ld_wait();
    const int part = u / kSm, s = u % kSm;
    if (u < kRows) {
      float* jr = jrow(G, part, s);
#pragma unroll
      for (int j = 0; j < 15; ++j) jr[j] = v[j + 1] * p.sri;
    }
  }
  group_sync(c.g);
  if constexpr (kDec) {  // decode mode: dg/dq rows of the tile's samples (hi + lo parts)
    const int n = ns * p.r;
    for (int e = c.gt; e < n; e += kGT) {
      const int jq = e / ns, sq = e % ns;
      float v = jrow(G, 0, sq)[jq];
      if (kLoP) v = __fadd_rn(v, jrow(G, 1, sq)[jq]);
      p.dec_out[(size_t)(p.row_dq + jq) * p.n_samples + j0 + sq] = v;
    }
    return true;
  }
  // ---------------- this tile's normal-equation terms
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int ea = o.ea[e], eb = o.eb[e];
    if (ea >= 0) {
      const float* a0 = jrow(G, 0, 0) + ea;
      const float* a1 = jrow(G, 1, 0) + ea;
      if (eb >= 0) o.acc[e] += dot_exact<kLoP, kLoP>(a0, a1, 16, jrow(G, 0, 0) + eb, jrow(G, 1, 0) + eb, 16, ns);
      else o.acc[e] += dot_exact<kLoP, false>(a0, a1, 16, G->rho, G->zero, 1, ns);
    } else if (ea == -3) {
      o.acc[e] += dot_exact<false, false>(G->rho, G->zero, 1, G->rho, G->zero, 1, ns);  // rho^T rho for the line search
    }
  }
  return true;
}

// Forward pass of one tile of kSm samples (global sample indices j0 .. j0 + ns - 1,
// ns >= 1; the tile's padding repeats its first sample), then Step 2 and the
// residual rho_j.  The tile occupies the group's sample slots so .. so + kSm - 1
// (coordinates xs, residual rho, and the TMEM columns kSig + l * kSS + slot that keep
// s'(z) of hidden layer l + 2 for the reverse pass), so that two tiles of iteration
// 0 can share one reverse pass.
template <int kM, int kSm, bool kFirst, int kSS, bool kLoP, bool kDec = false>
__device__ __forceinline__ bool forward_tile(Lane& c, const StepParams& p, int j0, int so, int ns, float alpha) {
  constexpr int kCh = kFirst ? 2 + kM : 2;  // iteration 0: v, dx_1..dx_m, Lap; later: v(q^(k)), diff
  constexpr int kN = kCh * kSm;             // hi columns 0..kN-1, lo columns kLo..kLo+kN-1
  constexpr int kPer = kSm / kTPU;          // samples of this thread
  constexpr int kC = kPer < 8 ? kPer : 8;    // samples per chunk
  static_assert(kN <= (kLoP ? kLo : 64) && kPer % kC == 0 && kC == 8 && kSS >= kSm &&
                    kSig + 4 * (kLoP ? kSS : kSS / 2) <= kGroupCols,
                "tile shape");
  Group* G = c.G;
  const Shared* S = c.S;
  const int u = c.u, s0 = c.part * kPer;
  const uint32_t lb = c.lane_base, tb = c.tb;
  // Step 2's per-sample inputs are loaded here, so that their latency overlaps the
  // forward pass: Delta f_j of iteration 0 (later iterations), alpha_j (per-sample
  // coefficient)
  double df_j = 0.0;
  if (c.gt < kSm) {
    const int s = c.gt < ns ? c.gt : 0;
    for (int k = 0; k < kM; ++k) G->xs[k][so + c.gt] = p.x[(size_t)(j0 + s) * kM + k];
    if (!kFirst) df_j = p.df[j0 + s];
    else if (p.coef_per_sample) alpha = p.alpha[j0 + s];
  }
  group_sync(c.g);
  // ---------------- layer 1 (CUDA cores)
  {
    const float cc = G->c1[u], dz = G->dz1[u];
#pragma unroll 1
    for (int h8 = 0; h8 < kPer; h8 += kC) {
      // layer-1 pre-activation channels: z = W_1x x + W_1q q + b_1, dz/dx_k = W_1[:, k],
      // Laplacian 0; later iterations: the difference channel's W_1q (q^(k) - q_n)
      float v[kCh][kC], sg[kC];
#pragma unroll
      for (int i = 0; i < kC; ++i) {
        float z = fmaf(c.wx0, G->xs[0][so + s0 + h8 + i], cc);
        if (kM > 1) z = fmaf(c.wx1, G->xs[1][so + s0 + h8 + i], z);
        v[0][i] = z;
        if (kFirst) {
          v[1][i] = c.gx0;
          if (kM > 1) v[2][i] = c.gx1;
          v[kCh - 1][i] = 0.f;
        } else {
          v[1][i] = dz;
        }
      }
      act<kM, kFirst, kCh, kC>(v, sg, c.dsc, c.dsci);
#pragma unroll
      for (int ch = 0; ch < kCh; ++ch) {
        const int n = ch * kSm + s0 + h8;
        split_store<kC, kLoP>(c.H, u, n, kLo + n, v[ch]);
      }
    }
  }
  // ---------------- hidden layers 2..L (tensor cores): one UMMA per K slice whose N
  // spans the hi columns (0..kLo-1) and the used lo columns (kLo..kLo+kN-1), or the
  // kN hi columns alone, rounded up to a multiple of 16
  constexpr uint32_t id_fwd = idesc_f16(128, (kLoP ? kLo : 0) + ((kN + 15) & ~15), false, true, false);
  for (int l = 0; l < p.L - 1; ++l) {
    if (!stage<kStageFwd>(c, l, id_fwd)) return false;
    const float bias = S->bh[l][u];
#pragma unroll 1
    for (int h8 = 0; h8 < kPer; h8 += kC) {
      float v[kCh][kC], w[kCh][kC], sg[kC];
#pragma unroll
      for (int ch = 0; ch < kCh; ++ch) {
        tmem_ldc(taddr(tb, lb, kAcc + ch * kSm + s0 + h8), v[ch]);
        if (kLoP) tmem_ldc(taddr(tb, lb, kAcc + kLo + ch * kSm + s0 + h8), w[ch]);
      }
      tmem_ld_wait();
      if (kLoP) {
#pragma unroll
        for (int ch = 0; ch < kCh; ++ch)
#pragma unroll
          for (int i = 0; i < kC; i += 2)
            unpk2(add2(pk2(v[ch][i], v[ch][i + 1]), pk2(w[ch][i], w[ch][i + 1])), v[ch][i], v[ch][i + 1]);
      }
#pragma unroll
      for (int i = 0; i < kC; i += 2) unpk2(add2(pk2(v[0][i], v[0][i + 1]), pk2(bias, bias)), v[0][i], v[0][i + 1]);
      act<kM, kFirst, kCh, kC>(v, sg, c.dsc, c.dsci);
      store_sig<kLoP>(tb, lb, kSS, l, so + s0 + h8, sg);
      if (l < p.L - 2) {
#pragma unroll
        for (int ch = 0; ch < kCh; ++ch) {
          const int n = ch * kSm + s0 + h8;
          split_store<kC, kLoP>(c.H, u, n, kLo + n, v[ch]);
        }
      } else {
        // output layer on the CUDA cores, in FP32 from h_L itself: this warp's share
        // (32 units) of w_out . h_L for the channels the residual needs; the four
        // lane quadrants' shares meet in shared memory (the Jacobian buffer is free
        // until the projection of this tile)
        static_assert(kC == 8, "the output-layer reduction works on chunks of 8 samples");
        const int lane = c.gt & 31, lq = c.gw & 3, sl = s0 + h8 + ((lane >> 2) & 7);
        float* pr = &G->jt[0][0][0];
#pragma unroll
        for (int ch = 0; ch < kCh; ++ch) {
          // step, iteration 0: the gradient channels only for advection, the Laplacian
          // always; later: the difference channel; decode: the requested channels
          const bool need = kDec ? (ch == 0 ? p.row_val >= 0 : ch == kCh - 1 ? p.row_lap >= 0 : p.row_dx >= 0)
                                 : ch >= 1 && (!kFirst || ch == kCh - 1 || p.pde != CROM_PDE_HEAT);
          if (need) {
            float wv[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) wv[i] = c.wo * v[ch][i];
            const float t = warp_sum8(wv, lane);
            if ((lane & 3) == 0) pr[(ch * 4 + lq) * kSm + sl] = t;
          }
        }
      }
    }
    // the s'(z) stores complete in the background: nothing reads those columns
    // before the reverse pass, which waits for them
  }
  group_sync(c.g);
  // output channel ch of tile sample s: the four quadrants' partial sums
  auto gout = [&](int ch, int s) {
    const float* pr = &G->jt[0][0][0];
    const int b = ch * 4 * kSm + s;
    return (pr[b] + pr[b + kSm]) + (pr[b + 2 * kSm] + pr[b + 3 * kSm]);
  };
  if constexpr (kDec) {  // decode mode: the requested channels of the tile's samples
    if (c.gt < ns) {
      const size_t n = (size_t)p.n_samples, j = (size_t)(j0 + c.gt);
      if (p.row_val >= 0) p.dec_out[(size_t)p.row_val * n + j] = gout(0, c.gt) + p.bout;
      if (p.row_dx >= 0)
        for (int k = 0; k < kM; ++k) p.dec_out[(size_t)(p.row_dx + k) * n + j] = gout(1 + k, c.gt) * p.sxi;
      if (p.row_lap >= 0) p.dec_out[(size_t)p.row_lap * n + j] = gout(kCh - 1, c.gt) * p.sx2i;
    }
    tmem_st_wait();
    return true;
  }
  // ---------------- Step 2 and the residual rho_j
  if (c.gt < kSm) {
    float rho = 0.f;
    if (c.gt < ns) {
      const int j = j0 + c.gt;
      if (kFirst) {
        const float lap = gout(kCh - 1, c.gt) * p.sx2i;
        double df;
        if (p.pde == CROM_PDE_HEAT) {
          df = p.dt * (double)alpha * (double)lap;
        } else {
          double adv = 0.0;
          for (int k = 0; k < kM; ++k)
            adv += (double)p.vel[(size_t)j * kM + k] * (double)(gout(1 + k, c.gt) * p.sxi);
          df = p.dt * (-adv + (double)alpha * (double)lap);
        }
        p.df[j] = df;
        rho = (float)(-df);
      } else {
        rho = (float)((double)(gout(1, c.gt) * c.dsci) - df_j);
      }
    }
    G->rho[so + c.gt] = rho;
  }
  tmem_st_wait();  // s'(z) of the forward pass is in TMEM
  return true;
}

// One tile of kSm samples of one GN iteration k >= 1: forward pass, PDE update /
// residual, reverse pass, Jacobian projection and this tile's share of J^T J and
// J^T rho; or, for a line-search trial (kValueOnly), the forward pass and rho^T rho.
template <int kM, int kSm, bool kLoP, bool kValueOnly = false>
__device__ __forceinline__ bool run_tile(Lane& c, const StepParams& p, int o0, int t, int ns, float alpha, Own& o) {
  if (!forward_tile<kM, kSm, false, kSm, kLoP>(c, p, o0 + t * kSm, 0, ns, alpha)) return false;
  if constexpr (kValueOnly) {  // line-search trial: only sum_j rho_j^2 is needed
    group_sync(c.g);
#pragma unroll
    for (int e = 0; e < 2; ++e)
      if (o.ea[e] == -3) o.acc[e] += dot_exact<false, false>(c.G->rho, c.G->zero, 1, c.G->rho, c.G->zero, 1, ns);
    return true;
  } else {
    return reverse_tile<kM, kSm, kSm, kLoP>(c, p, o0 + t * kSm, ns, o);
  }
}

// Samples 2 kS0 * t .. of GN iteration 0 (ns >= 1 of them, at most 2 kS0): two
// forward tiles of kS0 samples (the second only if ns > kS0) into sample slots
// 0..kS0-1 and kS0..2kS0-1, then one reverse pass and projection over all of them:
// the four-channel forward pass needs narrow tiles to fit the 32 hi columns of one
// N = 64 UMMA, the
// reverse pass does not.
template <int kM, bool kLoP, bool kDec = false>
__device__ __forceinline__ bool run_pair(Lane& c, const StepParams& p, int o0, int t, int ns, float alpha, Own& o) {
  constexpr int kS0 = tile_s0<kLoP>();
  constexpr int kSS = 2 * kS0;
  const int j0 = o0 + t * kSS;
  if (!forward_tile<kM, kS0, true, kSS, kLoP, kDec>(c, p, j0, 0, min(ns, kS0), alpha)) return false;
  const bool rev = !kDec || p.row_dq >= 0;  // decode mode: the reverse pass only for dg/dq
  if (ns <= kS0) return rev ? reverse_tile<kM, kS0, kSS, kLoP, kDec>(c, p, j0, ns, o) : true;
  if (!forward_tile<kM, kS0, true, kSS, kLoP, kDec>(c, p, j0 + kS0, kS0, ns - kS0, alpha)) return false;
  return rev ? reverse_tile<kM, kSS, kSS, kLoP, kDec>(c, p, j0, ns, o) : true;
}


// Layer-1 constants of the tile passes at the point q: c1 = b_1 + W_1q q (value
// channel) and dz1 = W_1q (q - q_n) (difference channel), FP64 sums rounded once;
// W_1q is read from global memory (L1-cached: once per GN iteration).  The
// difference channel is carried scaled by dsc = 2^e with max_u |dz1_u| * dsc in
// [1, 2) (its f16 operands would otherwise be subnormal); every thread of the group
// takes part (a group barrier inside).
template <int kM>
__device__ __forceinline__ void set_layer1(Lane& c, const StepParams& p, Group* G, const double* q) {
  const float* w = p.w1 + (size_t)c.u * (kM + p.r) + kM;
  double cc = (double)p.b1[c.u];
  for (int j = 0; j < p.r; ++j) cc = fma((double)w[j], q[j], cc);
  G->c1[c.u] = (float)cc;
  double dz = 0.0;
  for (int j = 0; j < p.r; ++j) dz = fma((double)w[j], q[j] - G->qn[j], dz);
  const float dzf = (float)dz;
  float mx = fabsf(dzf);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((c.gt & 31) == 0) G->dmax[c.gw & 3] = mx;
  group_sync(c.g);
  mx = fmaxf(fmaxf(G->dmax[0], G->dmax[1]), fmaxf(G->dmax[2], G->dmax[3]));
  int ex = 0;
  if (mx > 0.f && mx < 3.0e38f) ex = min(max(-ilogbf(mx), -100), 100);
  c.dsc = ldexpf(1.f, ex);
  c.dsci = ldexpf(1.f, -ex);
  G->dz1[c.u] = dzf * c.dsc;
}

// Decode mode: the points a .. b-1 of one work item, instance by instance (the
// instance of point a found by bisection of off; off non-decreasing from off[0] = 0).
// Points beyond off[n_inst] are left untouched.
template <int kM, bool kLoP>
__device__ __forceinline__ bool decode_chunk(Lane& c, const StepParams& p, int a, int b, Own& o) {
  constexpr int kS0 = tile_s0<kLoP>();
  Group* G = c.G;
  int lo = 0, hi = p.n_inst;  // largest inst with off[inst] <= a, in [0, n_inst)
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (p.off[mid] <= a) lo = mid;
    else hi = mid;
  }
  bool ok = true;
  for (int inst = lo; inst < p.n_inst && a < b && ok; ++inst) {
    const int e = min(b, p.off[inst + 1]);
    if (e <= a) continue;
    group_sync(c.g);  // the previous range's layer-1 constants are no longer read
    if (c.gt < p.r) {
      const double v = p.q[(size_t)inst * p.r + c.gt];
      G->qn[c.gt] = v;
      G->qcur[c.gt] = v;
    }
    group_sync(c.g);
    set_layer1<kM>(c, p, G, G->qcur);
    const int M = e - a, nt = (M + 2 * kS0 - 1) / (2 * kS0);
    for (int t = 0; t < nt && ok; ++t)
      ok = run_pair<kM, kLoP, true>(c, p, a, t, min(2 * kS0, M - t * 2 * kS0), 0.f, o);
    a = e;
  }
  return ok;
}

template <int kM, int kS1, bool kLoP, bool kDec = false>
__global__ void __launch_bounds__(kThreads, 1) step_tc_kernel(StepParams p) {
  constexpr int kS0 = tile_s0<kLoP>();
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x;
  const int r = p.r, L = p.L;
  Lane c;
  c.g = tid / kGT;
  c.gt = tid % kGT;
  c.gw = c.gt >> 5;
  const int lq = c.gw & 3;        // TMEM lane quadrant of this warp
  c.part = c.gw >> 2;              // which part of a tile's samples
  c.u = lq * 32 + (c.gt & 31);     // hidden unit = TMEM lane
  c.lane_base = (uint32_t)lq * 32;

  uint8_t* Wimg = sm;
  uint8_t* Hbase = sm + ((p.img_bytes + 1023) & ~1023);
  c.H = Hbase + (size_t)c.g * kHBuf;  // this group's 64-column operand block
  c.S = reinterpret_cast<Shared*>(Hbase + (size_t)kGroups * kHBuf);
  c.G = reinterpret_cast<Group*>(c.S + 1) + c.g;
  Shared* S = c.S;
  Group* G = c.G;

  if (tid == 0) {
    mbar_init(&S->bar_w, 1);
    fence_mbar_init();
  }
  if (c.gt == 0) {
    mbar_init(&G->bar_mma, 1);
    fence_mbar_init();
  }
  if (c.gt < kSMax) G->zero[c.gt] = 0.f;
  if (tid < 32) {
    tmem_alloc(&S->tmem_base, kTmemCols);
    tmem_relinquish();
  }
  if (tid < kTcWidth) {
    for (int l = 0; l < L - 1; ++l) S->bh[l][tid] = p.bh[l * kTcWidth + tid];
    for (int k = 0; k < kM; ++k) S->w1x[k][tid] = p.w1[tid * (kM + r) + k];
    S->wout[tid] = p.wout[tid];
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  c.tb = S->tmem_base + (uint32_t)c.g * kGroupCols;
  if (tid == 0) {
    mbar_arrive_expect_tx(&S->bar_w, (uint32_t)p.img_bytes);
    for (int o = 0; o < p.img_bytes; o += 16384)
      bulk_g2s(Wimg + o, p.img + o, (uint32_t)min(16384, p.img_bytes - o), &S->bar_w);
  }
  bool ok = __syncthreads_and(mbar_wait(&S->bar_w, 0, kWaitLimit));
  c.phase = 0;
  const uint32_t wbase = smem_u32(Wimg);
  // Base UMMA descriptors; every operand slice is base + a compile-time offset.
  c.dW_k = smem_desc_sw128(wbase, 16, 1024);       // W_l as K-major A
  c.dW_mn = smem_desc_sw128(wbase, 16384, 1024);   // W_l^T as MN-major A
  c.dP = smem_desc_sw128(wbase + (uint32_t)(L - 1) * kTcLayerBytes, 16, 1024);
  c.dH = smem_desc_sw128(smem_u32(c.H), 16384, 1024);
  c.wx0 = S->w1x[0][c.u];
  c.wx1 = (kM > 1) ? S->w1x[1][c.u] : 0.f;
  c.wsq = c.wx0 * c.wx0 + c.wx1 * c.wx1;
  c.wo = S->wout[c.u];
  c.gx0 = c.wx0 * p.sx;
  c.gx1 = c.wx1 * p.sx;
  c.wos = c.wo * p.sr;
  c.dsc = c.dsci = 1.f;
  const int ntri = r * (r + 1) / 2;
  const int n_entries = ntri + r;  // <= 135; with the line search's rho^T rho <= 136 <= 2 kGT
  // normal-equation entries k = c.gt and c.gt + kGT owned by this thread
  Own own;
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int k = c.gt + e * kGT;
    int ea = -1, eb = -1;
    if (k < ntri) {
      int a = 0, rem = k;
      while (rem >= r - a) { rem -= r - a; ++a; }
      ea = a; eb = a + rem;
    } else if (k < n_entries) {
      ea = k - ntri; eb = -2;
    } else if (k == n_entries && p.line_search > 0) {
      ea = -3;  // rho^T rho, the line search's objective
    }
    own.ea[e] = ea;
    own.eb[e] = eb;
  }

  while (ok) {
    group_sync(c.g);  // everyone is done with the previous instance's group state
    if (c.gt == 0) G->s_idx = atomicAdd(&p.queue[0], 1);
    group_sync(c.g);
    const int idx = G->s_idx;
    if constexpr (kDec) {  // decode mode: work item idx is a chunk of kDecChunk points
      const long a0 = (long)idx * kDecChunk;
      if (a0 >= p.n_samples) break;
      ok = decode_chunk<kM, kLoP>(c, p, (int)a0, (int)min(a0 + kDecChunk, (long)p.n_samples), own);
      continue;
    }
    if (idx >= p.n_inst) break;
    const int inst = p.order[idx];
    const int o0 = p.off[inst];
    const int M = p.off[inst + 1] - o0;
    if (M < r || M > p.max_samples || o0 < 0 || o0 + M > p.n_samples) {
      if (c.gt == 0) p.status[inst] = CROM_ERR_INVALID_ARG;
      continue;
    }
    if (c.gt < r) {
      const double v = p.q[(size_t)inst * r + c.gt];
      G->qn[c.gt] = v;
      G->qcur[c.gt] = v;
    }
    if (c.gt == 0) G->s_status = CROM_OK;
    const float alpha = p.coef_per_sample ? 0.f : p.alpha[inst];  // per-sample values are read in the tile
    group_sync(c.g);

    for (int it = 0; it < p.gn_iters && ok; ++it) {
      set_layer1<kM>(c, p, G, G->qcur);
      own.acc[0] = own.acc[1] = 0.0;
      if (it == 0) {
        const int nt = (M + 2 * kS0 - 1) / (2 * kS0);
        for (int t = 0; t < nt && ok; ++t)
          ok = run_pair<kM, kLoP>(c, p, o0, t, min(2 * kS0, M - t * 2 * kS0), alpha, own);
      } else {
        const int nt = (M + kS1 - 1) / kS1;
        for (int t = 0; t < nt && ok; ++t)
          ok = run_tile<kM, kS1, kLoP>(c, p, o0, t, min(kS1, M - t * kS1), alpha, own);
      }
      if (!ok) break;
      const int R = r + 1;
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int ea = own.ea[e], eb = own.eb[e];
        if (ea >= 0) {
          if (eb >= 0) {
            G->amat[ea * R + eb] = own.acc[e];
            G->amat[eb * R + ea] = own.acc[e];
          } else {
            G->amat[ea * R + r] = -own.acc[e];
          }
        } else if (ea == -3) {
          G->phi0 = 0.5 * own.acc[e];
        }
      }
      group_sync(c.g);
      if (c.gw == 0) {
        const double minus_v = c.gt < r ? G->amat[c.gt * R + r] : 0.0;  // -(J^T rho)_k
        const int st = chol_solve_warp(G->amat, G->invd, r, c.gt);
        if (st == CROM_OK && c.gt < r) {
          const double d = G->amat[c.gt * R + r];
          if (p.line_search > 0) G->delta[c.gt] = d;
          else G->qcur[c.gt] += d;
        }
        if (p.line_search > 0) {  // slope = (J^T rho) . delta
          double sl = st == CROM_OK && c.gt < r ? -minus_v * G->amat[c.gt * R + r] : 0.0;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) sl += __shfl_xor_sync(0xffffffffu, sl, o);
          if (c.gt == 0) G->slope = sl;
        }
        if (c.gt == 0) G->s_status = st;
      }
      group_sync(c.g);
      if (G->s_status != CROM_OK) break;
      if (p.line_search > 0) {
        // Backtracking (Armijo) along delta: a = 1, 1/2, ..., 2^-line_search.
        bool accepted = false;
        double a = 1.0;
        for (int trial = 0; trial <= p.line_search && ok; ++trial, a *= 0.5) {
          if (c.gt < r) G->qtry[c.gt] = G->qcur[c.gt] + a * G->delta[c.gt];
          group_sync(c.g);
          set_layer1<kM>(c, p, G, G->qtry);
          own.acc[0] = own.acc[1] = 0.0;
          const int nt = (M + kS1 - 1) / kS1;
          for (int t = 0; t < nt && ok; ++t)
            ok = run_tile<kM, kS1, kLoP, true>(c, p, o0, t, min(kS1, M - t * kS1), alpha, own);
          if (!ok) break;
#pragma unroll
          for (int e = 0; e < 2; ++e)
            if (own.ea[e] == -3) G->phi = 0.5 * own.acc[e];
          group_sync(c.g);
          if (G->phi <= G->phi0 + kArmijoC1 * a * G->slope) {
            if (c.gt < r) G->qcur[c.gt] = G->qtry[c.gt];
            accepted = true;
            break;
          }
        }
        group_sync(c.g);
        if (!ok || !accepted) break;  // no acceptable length: keep q and stop iterating
      }
    }  // GN iterations
    if (!ok) break;
    if (c.gt < r) p.q[(size_t)inst * r + c.gt] = G->qcur[c.gt];
    if (c.gt == 0) p.status[inst] = G->s_status;
  }
  if (!ok && c.gt == 0) atomicExch(&p.queue[1], 1);
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
  return 1024 + (((size_t)img_bytes + 1023) & ~(size_t)1023) + (size_t)kGroups * kHBuf + sizeof(Shared) +
         kGroups * sizeof(Group);
}

cudaError_t launch_step_tc(crom_ctx* ctx, const crom_step_desc* step, int lo_parts, int n_inst, double* q,
                           const float* alpha, const float* vel, const int* s_off, const float* samples,
                           int n_samples, int max_samples, int* status, cudaStream_t s) {
  if ((size_t)n_inst > ctx->order_cap) {
    if (ctx->order) cudaFree(ctx->order);
    ++ctx->scratch_gen;
    ctx->order = nullptr;
    ctx->order_cap = 0;
    cudaError_t e = cudaMalloc(&ctx->order, (size_t)n_inst * sizeof(int));
    if (e != cudaSuccess) return e;
    ctx->order_cap = n_inst;
  }
  if ((size_t)n_samples > ctx->targets_cap) {
    if (ctx->targets) cudaFree(ctx->targets);
    ++ctx->scratch_gen;
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
  p.sx = ctx->w.tc_sx;
  p.sxi = 1.f / ctx->w.tc_sx;
  p.sx2i = p.sxi * p.sxi;
  p.sr = ctx->w.tc_sr;
  p.sri = 1.f / ctx->w.tc_sr;
  p.L = ctx->desc.hidden;
  p.r = ctx->desc.r;
  p.w1 = ctx->w.w1;
  p.b1 = ctx->w.b1;
  p.bh = ctx->w.bh;
  p.wout = ctx->w.wout;
  p.bout = ctx->w.bout;
  p.pde = step->pde;
  p.coef_per_sample = step->coef_per_sample;
  p.gn_iters = step->gn_iters;
  p.line_search = step->line_search;
  p.dt = step->dt;
  p.n_inst = n_inst;
  p.q = q;
  p.alpha = alpha;
  p.vel = vel;
  p.off = s_off;
  p.x = samples;
  p.max_samples = max_samples;
  p.n_samples = n_samples;
  p.status = status;
  p.order = ctx->order;
  p.queue = ctx->queue;
  p.df = ctx->targets;
  const size_t smem = tc_step_smem_bytes(p.img_bytes);
  const int grid = std::min((n_inst + kGroups - 1) / kGroups, ctx->num_sms);
  auto launch = [&](auto kernel) -> cudaError_t {
    cudaError_t err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    kernel<<<grid, kThreads, smem, s>>>(p);
    return cudaGetLastError();
  };
  constexpr int kLarge = kTcTileS1Large, kSmall = kTcTileS1Small;
  const bool small_tiles = ctx->tc_tile_s1 == kSmall;
  if (lo_parts) {
    if (ctx->desc.m == 2)
      return small_tiles ? launch(step_tc_kernel<2, kSmall, true>) : launch(step_tc_kernel<2, kLarge, true>);
    return small_tiles ? launch(step_tc_kernel<1, kSmall, true>) : launch(step_tc_kernel<1, kLarge, true>);
  }
  // hi parts only: tiles of twice the samples for the same UMMA width
  if (ctx->desc.m == 2)
    return small_tiles ? launch(step_tc_kernel<2, 2 * kSmall, false>) : launch(step_tc_kernel<2, 2 * kLarge, false>);
  return small_tiles ? launch(step_tc_kernel<1, 2 * kSmall, false>) : launch(step_tc_kernel<1, 2 * kLarge, false>);
}

cudaError_t launch_decode_tc(crom_ctx* ctx, int lo_parts, int n_inst, const double* q, const int* pt_off,
                             const float* x, int n_pts, unsigned want, float* out, cudaStream_t s) {
  StepParams p{};
  p.img = ctx->w.tc_img;
  p.img_bytes = (int)ctx->w.tc_img_bytes;
  p.sx = ctx->w.tc_sx;
  p.sxi = 1.f / ctx->w.tc_sx;
  p.sx2i = p.sxi * p.sxi;
  p.sr = ctx->w.tc_sr;
  p.sri = 1.f / ctx->w.tc_sr;
  p.L = ctx->desc.hidden;
  p.r = ctx->desc.r;
  p.w1 = ctx->w.w1;
  p.b1 = ctx->w.b1;
  p.bh = ctx->w.bh;
  p.wout = ctx->w.wout;
  p.bout = ctx->w.bout;
  p.pde = CROM_PDE_HEAT;
  p.gn_iters = 1;
  p.dt = 1.0;
  p.n_inst = n_inst;
  p.q = const_cast<double*>(q);  // read only in decode mode
  p.off = pt_off;
  p.x = x;
  p.max_samples = n_pts;
  p.n_samples = n_pts;
  p.queue = ctx->queue;
  p.dec_out = out;
  const int m = ctx->desc.m;
  int row = 0;
  p.row_val = (want & CROM_WANT_VAL) ? row++ : -1;
  p.row_dx = (want & CROM_WANT_DX) ? row : -1;
  if (want & CROM_WANT_DX) row += m;
  p.row_lap = (want & CROM_WANT_LAP) ? row++ : -1;
  p.row_dq = (want & CROM_WANT_DQ) ? row : -1;
  cudaError_t e = cudaMemsetAsync(ctx->queue, 0, 2 * sizeof(int), s);  // work counter, timeout flag
  if (e != cudaSuccess) return e;
  const size_t smem = tc_step_smem_bytes(p.img_bytes);
  const long chunks = ((long)n_pts + kDecChunk - 1) / kDecChunk;
  const int grid = (int)std::min<long>((chunks + kGroups - 1) / kGroups, ctx->num_sms);
  auto launch = [&](auto kernel) -> cudaError_t {
    cudaError_t err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    kernel<<<grid, kThreads, smem, s>>>(p);
    return cudaGetLastError();
  };
  // the later-iteration tile size is not used in decode mode: the default instantiations
  constexpr int kLarge = kTcTileS1Large;
  if (lo_parts)
    return m == 2 ? launch(step_tc_kernel<2, kLarge, true, true>) : launch(step_tc_kernel<1, kLarge, true, true>);
  return m == 2 ? launch(step_tc_kernel<2, 2 * kLarge, false, true>)
                : launch(step_tc_kernel<1, 2 * kLarge, false, true>);
}

}  // namespace crom
