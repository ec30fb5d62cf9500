// Dense reconstruction g(x_p, q_c) on the tcgen05 tensor cores (value channel only).
//
// Persistent kernel, one CTA per SM with the decoder's bf16 hidden matrices in
// shared memory, four independent groups of 128 threads (one tile each, own
// 64-column operand block / 128 TMEM columns / mbarrier / named barrier) so that
// one group's UMMAs overlap the others' epilogues.  Hidden unit u is TMEM lane u
// and thread u of its group.  A tile is 32 points of one code with hi/lo operand
// parts, 64 points with hi parts only:
//   layer 1 (K = m + r, too small for UMMA) on CUDA cores: the q part of
//     W_1 [x; q] + b_1 is hoisted per code; h = ELU(W_1x x + c);
//   layers 2..L: D[u][n] = sum_k W_l[u][k] H[k][n] by UMMA (M = 128 units,
//     N = 64, K = 128), A = W_l (K-major, resident), B = H (MN-major, written by
//     the previous epilogue: the hi and lo parts of 32 points side by side, added
//     in the epilogue, or the hi parts of 64 points); epilogue: bias, ELU, bf16
//     split, store;
//   output layer: w_out . h_L on the CUDA cores in the last hidden layer's
//     epilogue, in FP32 from h_L itself (a warp butterfly over the 32 units of
//     each warp, then the four lane quadrants' partial sums), written coalesced.
// Precision: each activation operand h is stored as hi = bf16(h) and
// lo = bf16(h - hi) and both are multiplied into the same FP32 accumulator
// (kSplit = 1); kSplit = 0 keeps the high part only.
#include <math.h>

#include <algorithm>

#include "crom_internal.h"
#include "tc_common.cuh"

namespace crom {
namespace {

using namespace tc;

constexpr int kGroups = 4;
constexpr int kGT = 128;  // one thread per TMEM lane (hidden unit), all of the tile's points
constexpr int kThreads = kGroups * kGT;
// Points per tile: 32 with hi/lo operand parts (N = 64 = 32 hi + 32 lo columns),
// 64 with hi parts only (N = 64 points); one 64-column operand block and 64
// accumulator columns per group either way.
constexpr int kTileSplit = 32, kTileHi = 64;
constexpr int kTileN = kTileHi;  // sizes of the per-tile arrays
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kGroupCols = 128;
constexpr uint32_t kAccCol = 0;    // W h_hi in columns 0..31, W h_lo in 32..63 (hi only: 64 points)
constexpr uint32_t kWaitLimit = 1u << 25;
constexpr size_t kHBuf = (size_t)kTcWidth * 64 * 2;  // one 64-column bf16 operand block, 16 KB

struct ReconParams {
  const uint8_t* img;
  int img_bytes;
  int n_hidden_mats;  // hidden - 1
  int m, r;
  const float* w1;  // [128][m+r]
  const float* b1;
  const float* bh;  // [(hidden-1)][128]
  const float* wout;  // [128]
  float bout;
  const double* q;  // [n_codes][r]
  const float* x;   // [n_pts][m]
  float* out;       // [n_codes][n_pts]
  int n_pts, n_codes;
  int tiles_per_code;
  int* flag;  // set to 1 on a device-side wait timeout
};

struct __align__(16) Shared {
  uint64_t bar_w;
  uint32_t tmem_base;
  int pad;
  float bh[4][kTcWidth];
  float w1x[2][kTcWidth];
  float wout[kTcWidth];
};

struct __align__(16) Group {
  uint64_t bar_mma;
  int pad[2];
  float c1[kTcWidth];
  float xs[2][kTileN];
  float outp[4][kTileN];  // output layer: partial sums of the four lane quadrants
};

constexpr size_t kTailBytes = sizeof(Shared) + kGroups * sizeof(Group);

// Sum over the 32 lanes of a warp (32 hidden units) of 16 per-lane values v[s]:
// four exchange rounds halve the set (offsets 16, 8, 4, 2), one more adds across
// the lane pair (offset 1).  Lane l ends with the total of point (l >> 1) & 15.
__device__ __forceinline__ float warp_sum16(const float (&v)[16], int lane) {
  float a[8], b[4], c[2];
  const bool u16 = lane & 16, u8 = lane & 8, u4 = lane & 4, u2 = lane & 2;
#pragma unroll
  for (int s = 0; s < 8; ++s)
    a[s] = (u16 ? v[s + 8] : v[s]) + __shfl_xor_sync(0xffffffffu, u16 ? v[s] : v[s + 8], 16);
#pragma unroll
  for (int s = 0; s < 4; ++s)
    b[s] = (u8 ? a[s + 4] : a[s]) + __shfl_xor_sync(0xffffffffu, u8 ? a[s] : a[s + 4], 8);
#pragma unroll
  for (int s = 0; s < 2; ++s)
    c[s] = (u4 ? b[s + 2] : b[s]) + __shfl_xor_sync(0xffffffffu, u4 ? b[s] : b[s + 2], 4);
  float t = (u2 ? c[1] : c[0]) + __shfl_xor_sync(0xffffffffu, u2 ? c[0] : c[1], 2);
  t += __shfl_xor_sync(0xffffffffu, t, 1);
  return t;
}

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

// Sixteen consecutive columns of row k, given as 8 packed pairs, stored as bf16 hi
// parts at columns n0..n0+15 (and lo = bf16(h - hi) parts at nl..nl+15 when kSplit)
// of the MN-major operand H.
template <int kSplit>
__device__ __forceinline__ void store_split16(uint8_t* H, int k, int n0, int nl, const f32x2 (&h)[8]) {
  uint32_t hi[8], lo[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    float a, b;
    unpk2(h[j], a, b);
    hi[j] = pack_bf16(a, b);
    if (kSplit) lo[j] = pack_bf16_lo(hi[j], a, b);
  }
  *reinterpret_cast<uint4*>(H + mn_offset(k, n0)) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
  *reinterpret_cast<uint4*>(H + mn_offset(k, n0 + 8)) = make_uint4(hi[4], hi[5], hi[6], hi[7]);
  if (kSplit) {
    *reinterpret_cast<uint4*>(H + mn_offset(k, nl)) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    *reinterpret_cast<uint4*>(H + mn_offset(k, nl + 8)) = make_uint4(lo[4], lo[5], lo[6], lo[7]);
  }
}

template <int kSplit>
__global__ void __launch_bounds__(kThreads, 1) recon_tc_kernel(ReconParams p) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x;
  const int g = tid / kGT, gt = tid % kGT;
  const int lq = (gt >> 5) & 3;
  const int u = lq * 32 + (gt & 31);           // hidden unit = TMEM lane
  constexpr int kTile = kSplit ? kTileSplit : kTileHi;
  const uint32_t lane_base = (uint32_t)lq * 32;
  const int m = p.m, r = p.r;
  uint8_t* Wimg = sm;
  uint8_t* Hbase = sm + ((p.img_bytes + 1023) & ~1023);
  uint8_t* H = Hbase + (size_t)g * kHBuf;  // this group's 64-column operand block
  Shared* S = reinterpret_cast<Shared*>(Hbase + (size_t)kGroups * kHBuf);
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
    for (int l = 0; l < p.n_hidden_mats; ++l) S->bh[l][tid] = p.bh[l * kTcWidth + tid];
    for (int k = 0; k < m; ++k) S->w1x[k][tid] = p.w1[tid * (m + r) + k];
    S->wout[tid] = p.wout[tid];
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tb = S->tmem_base + (uint32_t)g * kGroupCols;
  if (tid == 0) {
    mbar_arrive_expect_tx(&S->bar_w, (uint32_t)p.img_bytes);
    for (int off = 0; off < p.img_bytes; off += 16384)
      bulk_g2s(Wimg + off, p.img + off, (uint32_t)min(16384, p.img_bytes - off), &S->bar_w);
  }
  // Every wait is bounded; the outcome is made uniform across the CTA (or group)
  // before anyone acts on it, so no thread leaves while others wait at a barrier.
  bool ok = __syncthreads_and(mbar_wait(&S->bar_w, 0, kWaitLimit));
  uint32_t phase = 0;
  const uint32_t wbase = smem_u32(Wimg);
  // Base UMMA descriptors; every operand slice is base + a compile-time offset.
  const uint64_t dW = smem_desc_sw128(wbase, 16, 1024);
  const uint64_t dH = smem_desc_sw128(smem_u32(H), 16384, 1024);
  constexpr uint32_t id_layer = idesc_f16(128, 64, false, true, true);
  int cur_code = -1;
  float c = 0.f;
  const float wx0 = S->w1x[0][u], wx1 = (m > 1) ? S->w1x[1][u] : 0.f;
  const float wo = S->wout[u];
  const int lane = gt & 31;
  const int n_tiles = p.n_codes * p.tiles_per_code;

  for (int tile = blockIdx.x * kGroups + g; tile < n_tiles && ok; tile += gridDim.x * kGroups) {
    const int code = tile / p.tiles_per_code;
    const int p0 = (tile % p.tiles_per_code) * kTile;
    if (code != cur_code) {
      double cc = (double)p.b1[u];
      for (int j = 0; j < r; ++j) cc += (double)p.w1[u * (m + r) + m + j] * p.q[(size_t)code * r + j];
      c = (float)cc;
      cur_code = code;
    }
    if (gt < kTile) {
      const int n = p0 + gt;
      for (int k = 0; k < m; ++k) G->xs[k][gt] = (n < p.n_pts) ? p.x[(size_t)n * m + k] : 0.f;
    }
    group_sync(g);
    // ---- layer 1 on CUDA cores
#pragma unroll 1
    for (int n0 = 0; n0 < kTile; n0 += 16) {
      f32x2 h[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        f32x2 z = fma2(pk2(wx0, wx0), pk2(G->xs[0][n0 + 2 * j], G->xs[0][n0 + 2 * j + 1]), pk2(c, c));
        if (m > 1) z = fma2(pk2(wx1, wx1), pk2(G->xs[1][n0 + 2 * j], G->xs[1][n0 + 2 * j + 1]), z);
        float e0, e1;
        h[j] = elu2(z, e0, e1);
      }
      store_split16<kSplit>(H, u, n0, kTileSplit + n0, h);
    }
    // ---- hidden layers on the tensor cores; the output layer in the last epilogue
    for (int l = 0; l < p.n_hidden_mats; ++l) {
      const bool last = (l == p.n_hidden_mats - 1);
      fence_proxy_async_smem();
      tc_fence_before();
      group_sync(g);
      bool done = true;
      if ((gt >> 5) == 0) {  // the first warp issues (one elected lane) and waits, the rest wait at the barrier
        tc_fence_after();
        // The lo parts follow the hi parts in the same 64-column block, so one UMMA
        // with N = 64 multiplies both at once: accumulator columns 0..31 get W h_hi,
        // columns 32..63 W h_lo (hi only: 64 points).
        const uint64_t a0 = desc_add(dW, (uint32_t)l * kTcLayerBytes);
#pragma unroll
        for (int kk = 0; kk < 8; ++kk)
          umma_f16_warp(tb + kAccCol, desc_add(a0, kmajor_kslice(128, kk)), desc_add(dH, mnmajor_kslice(kk)),
                        id_layer, kk != 0);
        umma_commit_warp(&G->bar_mma);
        done = mbar_wait(&G->bar_mma, phase, kWaitLimit);
      }
      ok = group_sync_and(g, done);
      phase ^= 1;
      tc_fence_after();
      if (!ok) break;
      const float bias = S->bh[l][u];
#pragma unroll 1
      for (int n0 = 0; n0 < kTile; n0 += 16) {
        float v[16], w[16];
        tmem_ld16(taddr(tb, lane_base, kAccCol + n0), v);
        if (kSplit) tmem_ld16(taddr(tb, lane_base, kAccCol + kTileSplit + n0), w);
        tmem_ld_wait();
        f32x2 h[8];
        const f32x2 b2 = pk2(bias, bias);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          float e0, e1;
          f32x2 z = add2(pk2(v[2 * j], v[2 * j + 1]), b2);
          if (kSplit) z = add2(z, pk2(w[2 * j], w[2 * j + 1]));
          h[j] = elu2(z, e0, e1);
        }
        if (!last) {
          store_split16<kSplit>(H, u, n0, kTileSplit + n0, h);
        } else {
          float wv[16];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            unpk2(h[j], wv[2 * j], wv[2 * j + 1]);
            wv[2 * j] *= wo;
            wv[2 * j + 1] *= wo;
          }
          const float t = warp_sum16(wv, lane);
          if ((lane & 1) == 0) G->outp[lq][n0 + ((lane >> 1) & 15)] = t;
        }
      }
    }
    if (!ok) break;
    group_sync(g);
    if (gt < kTile) {
      const int n = p0 + gt;
      const float o = (G->outp[0][gt] + G->outp[1][gt]) + (G->outp[2][gt] + G->outp[3][gt]);
      if (n < p.n_pts) p.out[(size_t)code * p.n_pts + n] = o + p.bout;
    }
  }
  if (!ok && gt == 0) atomicExch(p.flag, 1);
  tc_fence_before();
  __syncthreads();
  if (tid < 32) tmem_dealloc(S->tmem_base, kTmemCols);
}

}  // namespace

cudaError_t launch_recon_tc(const crom_ctx* ctx, int split, int n_codes, const double* q, int n_pts,
                            const float* x, float* out, cudaStream_t s) {
  ReconParams p{};
  p.img = ctx->w.tc_img;
  p.img_bytes = (int)ctx->w.tc_img_bytes;
  p.n_hidden_mats = ctx->desc.hidden - 1;
  p.m = ctx->desc.m;
  p.r = ctx->desc.r;
  p.w1 = ctx->w.w1;
  p.b1 = ctx->w.b1;
  p.bh = ctx->w.bh;
  p.wout = ctx->w.wout;
  p.bout = ctx->w.bout;
  p.q = q;
  p.x = x;
  p.out = out;
  p.n_pts = n_pts;
  p.n_codes = n_codes;
  const int tile_pts = split ? kTileSplit : kTileHi;
  p.tiles_per_code = (n_pts + tile_pts - 1) / tile_pts;
  p.flag = ctx->queue + 2;
  const size_t smem = 1024 + (((size_t)p.img_bytes + 1023) & ~(size_t)1023) + (size_t)kGroups * kHBuf +
                      kTailBytes;
  const long long tiles = (long long)n_codes * p.tiles_per_code;
  if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  const int grid = (int)std::min<long long>((tiles + kGroups - 1) / kGroups, ctx->num_sms);
  cudaError_t e;
  if (split) {
    e = cudaFuncSetAttribute(recon_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    recon_tc_kernel<1><<<grid, kThreads, smem, s>>>(p);
  } else {
    e = cudaFuncSetAttribute(recon_tc_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    recon_tc_kernel<0><<<grid, kThreads, smem, s>>>(p);
  }
  return cudaGetLastError();
}

}  // namespace crom
