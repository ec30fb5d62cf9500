// Dense reconstruction g(x_p, q_c) on the tcgen05 tensor cores (value channel only).
//
// Persistent kernel, one CTA per SM, warp-specialised: one MMA warp issues every
// UMMA of the CTA, and two tile slots of eight epilogue warps each (two threads
// per hidden unit, each on half of the tile's points) run the CUDA-core work.
// The slots alternate on the tensor cores: while the MMA warp multiplies one
// slot's tile through a layer, the other slot's warps run their epilogue.  Hand-
// offs are mbarriers, per slot: `full` (the slot's operand block is written: one
// arrival per epilogue warp) and `acc` (the slot's accumulator is complete: the
// UMMA commit).  Hidden unit u is TMEM lane u.
//
// Per tile (64 points of one code with hi/lo operand parts, or 128 points with
// high parts only):
//   layer 1 (K = m + r, too small for UMMA) on CUDA cores: the q part of
//     W_1 [x; q] + b_1 is hoisted per code; h = ELU(W_1x x + c);
//   layers 2..L: D[u][n] = sum_k W_l[u][k] H[k][n] by UMMA (M = 128 units,
//     K = 128), A = W_l (f16, K-major, resident in shared memory), B = H
//     (MN-major, written by the previous epilogue).  With hi/lo parts, B holds
//     hi = f16(h) in columns 0..63 and lo = f16(h - hi) in 64..127: one N = 128
//     UMMA per K slice gives W hi and W lo in separate accumulator columns; a
//     third product W_lo hi (N = 64) adds the weights' own low parts
//     W_lo = f16(W - f16(W)), read from tensor memory (the A operand of the
//     TMEM form), into the first 64 columns.  The epilogue adds the two halves,
//     the bias, applies ELU and writes the next operand.  With high parts only
//     (kSplit = 0), where the epilogue's instruction issue is the limit, the
//     activations are carried times log2 e (so that 2^x needs no scaling) and
//     the bias enters the accumulator as one more UMMA, log2 e (b_hi + b_lo)
//     times a ones operand (K = 16), leaving the epilogue ELU and the f16 store;
//   output layer, kSplit = 0: one more UMMA stage, O[n][j] = sum_k H[k][n] Wo[j][k]
//     with the last hidden layer's operand block H (the tile's 128 points) as the
//     MN-major A operand against the 16-row output operand Wo (row 0 =
//     f16(ln 2 w_out), row 1 = its low part); the epilogue adds a point's two
//     products and the bias, one thread per point, written coalesced;
//   output layer, kSplit = 1: w_out . h_L on the CUDA cores in the last hidden
//     layer's epilogue, in FP32 from h_L itself (a warp butterfly over the 32
//     units of each warp, then the four lane quadrants' partial sums).  The
//     tensor-core stage measured slower here: the 64-point tiles make its fixed
//     cost per point twice as large, on a tensor pipe that the third product
//     already keeps busier.
// Precision (kSplit = 1): activations carry ~2^-22 relative (hi + lo), weights
// W + W_lo ~2^-22 (the W_lo lo product is below that and left out), FP32
// accumulation.  kSplit = 0: f16 activations and hidden weights (2^-11 relative
// each), biases and w_out ~2^-22.
// TMEM: slot s accumulator in columns 128 s .. 128 s + 127 (the output stage's
// 16 columns at its start); W_lo of hidden matrix l in columns 256 + 64 l .. + 63.
#include <math.h>

#include <algorithm>

#include "crom_internal.h"
#include "tc_common.cuh"

namespace crom {
namespace {

using namespace tc;

constexpr int kSlots = 2;
constexpr int kEpiWarps = 8;                       // per slot
constexpr int kSlotThreads = kEpiWarps * 32;       // 256
constexpr int kMmaWarp = kSlots * kEpiWarps;       // warp 16
constexpr int kThreads = (kMmaWarp + 1) * 32;      // 544
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kSlotCols = 128;
constexpr uint32_t kLoCol = 256;                   // W_lo of hidden matrix l at kLoCol + 64 l
constexpr uint32_t kWaitLimit = 1u << 25;
constexpr size_t kHBuf = (size_t)kTcWidth * 128 * 2;  // one slot's operand block: 128 columns, 32 KB
constexpr int kMaxPts = 128;
constexpr int kOnesBytes = 4096;  // ones operand of the bias product: 16 k-rows x 128 n, f16

struct ReconParams {
  const uint8_t* img;  // hidden matrices, f16 K-major SW128
  int hidden_bytes;    // (hidden - 1) * 32 KB
  const uint8_t* oimg;  // kSplit = 0: output operand Wo, 16 x 128 f16 K-major SW128 (4 KB),
                        // then the bias operand, 128 x 64 f16 K-major SW128 (16 KB)
  const uint16_t* lo;  // W_lo, f16 row-major [hidden - 1][128][128]
  int n_hidden_mats;   // hidden - 1
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
  int n_tiles;
  int* flag;  // set to 1 on a device-side wait timeout
};

struct __align__(16) Shared {
  uint64_t bar_w;           // the weight image arrived
  uint64_t full[kSlots];    // the slot's operand block is written (kEpiWarps arrivals)
  uint64_t acc[kSlots];     // the slot's accumulator is complete (UMMA commit)
  uint64_t drain;           // the MMA warp's last UMMAs completed
  uint32_t tmem_base;
  int abort;                // a bounded wait ran out: every wait and UMMA is skipped from then on
  float bh[4][kTcWidth];
  float w1x[2][kTcWidth];
  float wout[kTcWidth];
  float xs[kSlots][2][kMaxPts];
  float outp[kSlots][4][kMaxPts];  // CUDA-core output layer: the four lane quadrants' partial sums
};

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

// tcgen05.wait::ld that also names the registers of the loads it waits for, so that
// the compiler keeps their uses after it (a load's destination registers are valid
// only once the wait returns).
__device__ __forceinline__ void tmem_wait_regs(float (&v)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+f"(v[0]), "+f"(v[1]), "+f"(v[2]), "+f"(v[3]), "+f"(v[4]), "+f"(v[5]), "+f"(v[6]), "+f"(v[7]),
                 "+f"(v[8]), "+f"(v[9]), "+f"(v[10]), "+f"(v[11]), "+f"(v[12]), "+f"(v[13]), "+f"(v[14]),
                 "+f"(v[15])
               :
               : "memory");
}
// Marks registers as written by a preceding wait (after tmem_wait_regs of other
// registers has waited for all loads).
__device__ __forceinline__ void tmem_bind_regs(float (&v)[16]) {
  asm volatile(""
               : "+f"(v[0]), "+f"(v[1]), "+f"(v[2]), "+f"(v[3]), "+f"(v[4]), "+f"(v[5]), "+f"(v[6]), "+f"(v[7]),
                 "+f"(v[8]), "+f"(v[9]), "+f"(v[10]), "+f"(v[11]), "+f"(v[12]), "+f"(v[13]), "+f"(v[14]),
                 "+f"(v[15])
               :
               : "memory");
}

__device__ __forceinline__ void slot_sync(int s) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + s), "r"(kSlotThreads) : "memory");
}

__device__ __forceinline__ bool aborted(Shared* S) { return *reinterpret_cast<volatile int*>(&S->abort) != 0; }
// Bounded wait unless the kernel already gave up; a wait that runs out raises abort.
__device__ __forceinline__ void wait_or_abort(Shared* S, uint64_t* bar, uint32_t parity) {
  if (aborted(S)) return;
  if (!mbar_wait(bar, parity, kWaitLimit)) *reinterpret_cast<volatile int*>(&S->abort) = 1;
}

// ELU in units of log2 e: for t = log2 e * z returns log2 e * ELU(z) =
// max(t, log2 e (2^-|t| - 1)) (the maximum as in elu2_val); one multiply less a pair
// than elu2_val on unscaled values.
__device__ __forceinline__ f32x2 elu2_log2(f32x2 t) {
  constexpr float kLog2e = 1.4426950408889634f;
  float t0, t1, d0, d1;
  unpk2(t, t0, t1);
  unpk2(fma2(pk2(ex2_approx(-fabsf(t0)), ex2_approx(-fabsf(t1))), pk2(kLog2e, kLog2e), pk2(-kLog2e, -kLog2e)), d0,
        d1);
  return pk2(fmaxf(t0, d0), fmaxf(t1, d1));
}

// shared memory of the largest decoder (four hidden matrices) within the 227 KB per block
static_assert(1024 + 4 * kTcLayerBytes + kTcProjBytes + kTcBiasBytes + kOnesBytes + kSlots * kHBuf + sizeof(Shared) <=
                  232448,
              "reconstruction shared memory");

// Sixteen consecutive columns of row k, given as 8 packed pairs, stored as f16 hi
// parts at columns n0..n0+15 (and lo = f16(h - hi) parts at 64 + n0.. when kSplit)
// of the MN-major operand H.
template <int kSplit>
__device__ __forceinline__ void store_split16(uint8_t* H, int k, int n0, const f32x2 (&h)[8]) {
  uint32_t hi[8], lo[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    float a, b;
    unpk2(h[j], a, b);
    hi[j] = pack_f16(a, b);
    if (kSplit) lo[j] = pack_f16_lo(hi[j], a, b);
  }
  *reinterpret_cast<uint4*>(H + mn_offset(k, n0)) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
  *reinterpret_cast<uint4*>(H + mn_offset(k, n0 + 8)) = make_uint4(hi[4], hi[5], hi[6], hi[7]);
  if (kSplit) {
    *reinterpret_cast<uint4*>(H + mn_offset(k, 64 + n0)) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    *reinterpret_cast<uint4*>(H + mn_offset(k, 64 + n0 + 8)) = make_uint4(lo[4], lo[5], lo[6], lo[7]);
  }
}

template <int kSplit>
__global__ void __launch_bounds__(kThreads, 1) recon_tc_kernel(ReconParams p) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr int kPts = kSplit ? 64 : 128;   // points per tile
  constexpr bool kOutTc = !kSplit;          // output layer on the tensor cores
  constexpr int kPer = kPts / 2;            // points per epilogue thread
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m = p.m, r = p.r, L1 = p.n_hidden_mats;
  uint8_t* Wimg = sm;
  uint8_t* Oimg = sm + p.hidden_bytes;     // kSplit = 0: output operand,
  uint8_t* Bimg = Oimg + kTcProjBytes;     // bias operand,
  uint8_t* Ones = Bimg + kTcBiasBytes;     // and the ones operand of the bias product
  uint8_t* Hbase = Ones + kOnesBytes;
  Shared* S = reinterpret_cast<Shared*>(Hbase + (size_t)kSlots * kHBuf);

  if (tid == 0) {
    mbar_init(&S->bar_w, 1);
    for (int s = 0; s < kSlots; ++s) {
      mbar_init(&S->full[s], kEpiWarps);
      mbar_init(&S->acc[s], 1);
    }
    mbar_init(&S->drain, 1);
    S->abort = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(&S->tmem_base, kTmemCols);
    tmem_relinquish();
  }
  if (!kSplit) {
    // ones operand (MN-major, 16 k-rows x 128 n, two 64-column blocks of 2 KB):
    // k-rows 0 and 1 are ones, the rest zero (a whole row is one value, so the
    // swizzle leaves it in place)
    for (int i = tid; i < kOnesBytes / 4; i += kThreads)
      reinterpret_cast<uint32_t*>(Ones)[i] = ((i * 4) % 2048) / 128 < 2 ? 0x3C003C00u : 0u;
    fence_proxy_async_smem();
  }
  if (tid < kTcWidth) {
    for (int l = 0; l < L1; ++l) S->bh[l][tid] = p.bh[l * kTcWidth + tid];
    for (int k = 0; k < m; ++k) S->w1x[k][tid] = p.w1[tid * (m + r) + k];
    S->wout[tid] = p.wout[tid];
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tb = S->tmem_base;
  if (tid == 0) {
    mbar_arrive_expect_tx(&S->bar_w, (uint32_t)(p.hidden_bytes + (kSplit ? 0 : kTcProjBytes + kTcBiasBytes)));
    for (int off = 0; off < p.hidden_bytes; off += 16384)
      bulk_g2s(Wimg + off, p.img + off, (uint32_t)min(16384, p.hidden_bytes - off), &S->bar_w);
    if (!kSplit) {
      bulk_g2s(Oimg, p.oimg, (uint32_t)kTcProjBytes, &S->bar_w);
      bulk_g2s(Bimg, p.oimg + kTcProjBytes, (uint32_t)kTcBiasBytes, &S->bar_w);
    }
  }
  if (kSplit && warp < 4) {
    // W_lo into tensor memory: lane u = row u, column c = (k = 2c, 2c + 1)
    const int row = warp * 32 + lane;
    for (int l = 0; l < L1; ++l) {
      const uint4* src = reinterpret_cast<const uint4*>(p.lo + ((size_t)l * kTcWidth + row) * kTcWidth);
#pragma unroll 1
      for (int c0 = 0; c0 < 64; c0 += 16) {
        float v[16];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const uint4 w = __ldg(src + c0 / 4 + j);
          v[4 * j] = __uint_as_float(w.x);
          v[4 * j + 1] = __uint_as_float(w.y);
          v[4 * j + 2] = __uint_as_float(w.z);
          v[4 * j + 3] = __uint_as_float(w.w);
        }
        tmem_st16(taddr(tb, (uint32_t)warp * 32, kLoCol + (uint32_t)l * 64 + c0), v);
      }
    }
    tmem_st_wait();
  }
  wait_or_abort(S, &S->bar_w, 0);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  const int stride = gridDim.x * kSlots;
  if (warp == kMmaWarp) {
    // ------------------------------------------------------------ MMA warp
    const uint32_t wbase = smem_u32(Wimg);
    const uint64_t dW = smem_desc_sw128(wbase, 16, 1024);
    constexpr uint32_t id_main = idesc_f16(128, 128, false, true, false);
    constexpr uint32_t id_lo = idesc_f16(128, 64, false, true, false);
    constexpr uint32_t id_out = idesc_f16(128, 16, true, false, false);
    const uint64_t dO = smem_desc_sw128(smem_u32(Oimg), 16, 1024);
    const uint64_t dB = smem_desc_sw128(smem_u32(Bimg), 16, 1024);
    const uint64_t dOnes = smem_desc_sw128(smem_u32(Ones), 2048, 1024);
    uint32_t pf[kSlots] = {0, 0};
    bool issued = false;
    for (int t0 = blockIdx.x * kSlots; t0 < p.n_tiles; t0 += stride) {
      const int nslot = min(kSlots, p.n_tiles - t0);
      for (int l = 0; l < L1 + (kOutTc ? 1 : 0); ++l) {
        for (int s = 0; s < nslot; ++s) {
          wait_or_abort(S, &S->full[s], pf[s]);
          pf[s] ^= 1;
          if (aborted(S)) continue;
          tc_fence_after();
          const uint32_t d = tb + (uint32_t)s * kSlotCols;
          const uint64_t b0 = smem_desc_sw128(smem_u32(Hbase + (size_t)s * kHBuf), 16384, 1024);
          if (kOutTc && l == L1) {
            // output stage: the operand block as the MN-major A operand
#pragma unroll
            for (int kk = 0; kk < 8; ++kk)
              umma_f16_warp(d, desc_add(b0, mnmajor_kslice(kk)), desc_add(dO, kmajor_kslice(16, kk)), id_out,
                            kk != 0);
            umma_commit_warp(&S->acc[s]);
            issued = true;
            continue;
          }
          const uint64_t a0 = desc_add(dW, (uint32_t)l * kTcLayerBytes);
          // kSplit = 0: the bias enters as a 17th product, (b_hi + b_lo) x ones
          if (!kSplit) umma_f16_warp(d, desc_add(dB, kmajor_kslice(128, l)), dOnes, id_main, false);
#pragma unroll
          for (int kk = 0; kk < 8; ++kk)
            umma_f16_warp(d, desc_add(a0, kmajor_kslice(128, kk)), desc_add(b0, mnmajor_kslice(kk)), id_main,
                          !kSplit || kk != 0);
          if (kSplit) {
#pragma unroll
            for (int kk = 0; kk < 8; ++kk)
              umma_ts_warp(d, tb + kLoCol + (uint32_t)l * 64 + kk * 8, desc_add(b0, mnmajor_kslice(kk)), id_lo, 1);
          }
          umma_commit_warp(&S->acc[s]);
          issued = true;
        }
      }
    }
    if (issued && !aborted(S)) {
      umma_commit_warp(&S->drain);  // arrives when every UMMA issued above has completed
      wait_or_abort(S, &S->drain, 0);
    }
  } else {
    // ------------------------------------------------------------ epilogue warps
    const int s = warp / kEpiWarps, j = warp % kEpiWarps;
    const int lq = j & 3, hf = j >> 2;
    const int u = lq * 32 + lane;             // hidden unit = TMEM lane
    const int et = j * 32 + lane;             // thread index within the slot
    const uint32_t lane_base = (uint32_t)lq * 32;
    const uint32_t acc = tb + (uint32_t)s * kSlotCols;
    uint8_t* H = Hbase + (size_t)s * kHBuf;
    // kSplit = 0 carries every activation times log2 e (layer 1 scaled here, the
    // hidden biases and w_out in their operands)
    constexpr float kAs = kSplit ? 1.f : 1.4426950408889634f;
    const float wx0 = kAs * S->w1x[0][u], wx1 = (m > 1) ? kAs * S->w1x[1][u] : 0.f;
    const float wo = S->wout[u];
    uint32_t pa = 0;
    int cur_code = -1;
    float c = 0.f;
    // coordinates of this thread's point of a tile (thread et < kPts), loaded one
    // tile ahead so that their latency hides behind the current tile
    auto load_x = [&](int tt, float& x0, float& x1) {
      const int n = (tt % p.tiles_per_code) * kPts + et;
      const bool ok = tt >= 0 && tt < p.n_tiles && et < kPts && n >= 0 && n < p.n_pts;
      x0 = ok ? __ldg(p.x + (size_t)n * m) : 0.f;
      x1 = (ok && m > 1) ? __ldg(p.x + (size_t)n * m + 1) : 0.f;
    };
    float xn0, xn1;
    load_x(blockIdx.x * kSlots + s, xn0, xn1);
    for (int t = blockIdx.x * kSlots + s; t < p.n_tiles; t += stride) {
      const int code = t / p.tiles_per_code;
      const int p0 = (t % p.tiles_per_code) * kPts;
      if (code != cur_code) {
        double cc = (double)p.b1[u];
        for (int jj = 0; jj < r; ++jj) cc += (double)p.w1[u * (m + r) + m + jj] * p.q[(size_t)code * r + jj];
        c = (float)(kSplit ? cc : cc * 1.4426950408889634);
        cur_code = code;
      }
      slot_sync(s);  // the previous tile's coordinates and outputs are used
      if (et < kPts) {
        S->xs[s][0][et] = xn0;
        S->xs[s][1][et] = xn1;
      }
      load_x(t + stride, xn0, xn1);
      slot_sync(s);
      // ---- layer 1 on CUDA cores
#pragma unroll 1
      for (int n0 = hf * kPer; n0 < hf * kPer + kPer; n0 += 16) {
        f32x2 h[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          f32x2 z = fma2(pk2(wx0, wx0), pk2(S->xs[s][0][n0 + 2 * i], S->xs[s][0][n0 + 2 * i + 1]), pk2(c, c));
          if (m > 1) z = fma2(pk2(wx1, wx1), pk2(S->xs[s][1][n0 + 2 * i], S->xs[s][1][n0 + 2 * i + 1]), z);
          h[i] = kSplit ? elu2_val(z) : elu2_log2(z);
        }
        store_split16<kSplit>(H, u, n0, h);
      }
      fence_proxy_async_smem();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&S->full[s]);
      // ---- hidden layers: the accumulator, then the next operand (or the output)
      for (int l = 0; l < L1; ++l) {
        const bool last_cc = !kOutTc && (l == L1 - 1);  // the output on the CUDA cores
        wait_or_abort(S, &S->acc[s], pa);
        pa ^= 1;
        tc_fence_after();
        const float bias = S->bh[l][u];
        const f32x2 b2 = pk2(bias, bias);
        // The accumulator chunks (16 points each) of this thread's half: the next
        // chunk's TMEM load is in flight while this one is computed.
        constexpr int kChunks = kPer / 16;
        float va[16], vb[16], wa[16], wb[16];
        tmem_ld16(taddr(acc, lane_base, hf * kPer), va);
        if (kSplit) tmem_ld16(taddr(acc, lane_base, 64 + hf * kPer), wa);
        if (kSplit) {
          tmem_wait_regs(va);
          tmem_bind_regs(wa);
        } else {
          tmem_wait_regs(va);
        }
#pragma unroll
        for (int ci = 0; ci < kChunks; ++ci) {
          const int n0 = hf * kPer + 16 * ci;
          float(&v)[16] = (ci & 1) ? vb : va;
          float(&w)[16] = (ci & 1) ? wb : wa;
          float(&vn)[16] = (ci & 1) ? va : vb;
          float(&wn)[16] = (ci & 1) ? wa : wb;
          if (ci + 1 < kChunks) {
            tmem_ld16(taddr(acc, lane_base, n0 + 16), vn);
            if (kSplit) tmem_ld16(taddr(acc, lane_base, 64 + n0 + 16), wn);
          }
          f32x2 h[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            if (kSplit) {
              const f32x2 z = add2(add2(pk2(v[2 * i], v[2 * i + 1]), b2), pk2(w[2 * i], w[2 * i + 1]));
              h[i] = elu2_val(z);
            } else {
              h[i] = elu2_log2(pk2(v[2 * i], v[2 * i + 1]));  // the bias is in the accumulator
            }
          }
          if (!last_cc) {
            store_split16<kSplit>(H, u, n0, h);
          } else {
            float wv[16];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              unpk2(h[i], wv[2 * i], wv[2 * i + 1]);
              wv[2 * i] *= wo;
              wv[2 * i + 1] *= wo;
            }
            const float tsum = warp_sum16(wv, lane);
            if ((lane & 1) == 0) S->outp[s][lq][n0 + ((lane >> 1) & 15)] = tsum;
          }
          if (ci + 1 < kChunks) {
            tmem_wait_regs(vn);
            if (kSplit) tmem_bind_regs(wn);
          }
        }
        tc_fence_before();
        if (!last_cc) {
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) mbar_arrive(&S->full[s]);
        }
      }
      if constexpr (kOutTc) {
        // ---- output stage: row u = 32 lq + lane of O (point u) in the first four warps
        wait_or_abort(S, &S->acc[s], pa);
        pa ^= 1;
        tc_fence_after();
        if (hf == 0) {
          float ov[4];
          tmem_ld4(taddr(acc, lane_base, 0), ov);
          asm volatile("tcgen05.wait::ld.sync.aligned;"
                       : "+f"(ov[0]), "+f"(ov[1]), "+f"(ov[2]), "+f"(ov[3])::"memory");
          const int n = p0 + u;
          // (log2 e h) . f16(ln 2 w_out) + (log2 e h) . (its low part)
          if (n < p.n_pts) p.out[(size_t)code * p.n_pts + n] = (ov[0] + ov[1]) + p.bout;
        }
        tc_fence_before();
      } else {
        slot_sync(s);
        if (et < kPts) {
          const int n = p0 + et;
          const float o = (S->outp[s][0][et] + S->outp[s][1][et]) + (S->outp[s][2][et] + S->outp[s][3][et]);
          if (n < p.n_pts) p.out[(size_t)code * p.n_pts + n] = o + p.bout;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && aborted(S)) atomicExch(p.flag, 1);
  if (warp == 0) tmem_dealloc(tb, kTmemCols);
}

}  // namespace

cudaError_t launch_recon_tc(const crom_ctx* ctx, int split, int n_codes, const double* q, int n_pts,
                            const float* x, float* out, cudaStream_t s) {
  ReconParams p{};
  p.img = ctx->w.tc_img;
  p.n_hidden_mats = ctx->desc.hidden - 1;
  p.hidden_bytes = p.n_hidden_mats * kTcLayerBytes;
  p.lo = reinterpret_cast<const uint16_t*>(ctx->w.tc_lo);
  p.m = ctx->desc.m;
  p.r = ctx->desc.r;
  p.w1 = ctx->w.w1;
  p.b1 = ctx->w.b1;
  p.bh = ctx->w.bh;
  p.oimg = ctx->w.tc_img + ctx->w.tc_img_bytes;  // output operand, then the bias operand
  p.wout = ctx->w.wout;
  p.bout = ctx->w.bout;
  p.q = q;
  p.x = x;
  p.out = out;
  p.n_pts = n_pts;
  p.n_codes = n_codes;
  const int tile_pts = split ? 64 : 128;
  p.tiles_per_code = (n_pts + tile_pts - 1) / tile_pts;
  p.flag = ctx->queue + 2;
  const long long tiles = (long long)n_codes * p.tiles_per_code;
  if (tiles > 0x7fffffffLL - 4096) return cudaErrorInvalidValue;  // t + stride stays an int
  p.n_tiles = (int)tiles;
  const size_t smem =
      1024 + (size_t)p.hidden_bytes + kTcProjBytes + kTcBiasBytes + kOnesBytes + (size_t)kSlots * kHBuf + sizeof(Shared);
  const int grid = (int)std::min<long long>((tiles + kSlots - 1) / kSlots, ctx->num_sms);
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
