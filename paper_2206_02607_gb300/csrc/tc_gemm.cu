// bf16 GEMM on the tcgen05 tensor cores for the training step (paper §3, Eq. loss;
// App. D): D[m][n] = sum_k A(m, k) B(n, k) with FP32 accumulation in tensor memory
// and the training pass's elementwise work fused into the epilogue.
//
// Persistent, one CTA per SM, 320 threads in warp roles:
//   warp 0   TMA producer: one elected lane loads the A and B boxes of each 64-wide
//            K block (cp.async.bulk.tensor, 128-byte swizzle) into a 3-stage ring;
//   warp 1   MMA issuer: four UMMAs (M = 128, N = BN, K = 16) per K block into one of
//            two tensor-memory accumulators, commits free the ring stage and, after
//            the tile's last block, hand the accumulator to the epilogue;
//   warps 2-9 epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (one tile row per
//            thread) and one half of the BN columns (warps 2-5 the first, 6-9 the
//            second), applies the fused operation, frees the accumulator; bf16 rows
//            go through a per-warp shared-memory staging area so that global loads
//            and stores move whole half rows (coalesced).  Two warps per SM
//            sub-partition hide each other's load, shuffle and exp latencies.
// With two accumulators the epilogue of one tile overlaps the MMAs of the next.
// Operands: A(m, k) K-major (A[m * lda + k]) or MN-major (A[k * lda + m]); B(n, k)
// likewise; both are read through tensor maps whose boxes land in shared memory in
// the layouts the UMMA descriptors describe (K-major: rows of 64 K elements, 8-row
// groups 1024 B apart; MN-major: 64-element MN blocks of 64 K rows, 8 KB apart).
// Every wait is bounded: a wait that runs out sets the error flag and the CTA stops
// issuing work, frees its tensor memory and returns.
#include <cuda.h>
#include <math.h>

#include <algorithm>
#include <mutex>

#include "crom_internal.h"
#include "tc_common.cuh"

namespace crom {
namespace {

using namespace tc;

constexpr int kBM = 128, kBK = 64, kStages = 3;
constexpr int kEpiWarps = 8;
constexpr int kGemmThreads = 64 + 32 * kEpiWarps;
constexpr uint32_t kWait = 1u << 26;

struct Args {
  int M, N, K;
  int a_mn, b_mn;
  int tiles_m, splits, kb_per_split;  // K blocks of 64 per split
  int epi;
  float* out_f32;
  long ldo;
  uint16_t* out_bf16;
  const float* bias;
  const uint16_t* hprev;
  float* colpart;   // [tiles_m * 4][N]
  const float* wout;
  const float* bout;
  const float* target;
  float* resid;     // [M]: g - target per row (output-layer epilogue)
  int* flag;
};

struct __align__(8) Bars {
  uint64_t full[kStages], empty[kStages], tfull[2], tempty[2];
  uint32_t tmem_base;
  int abort;
  float gpart[2][2][4][32];  // output layer: [tile parity][column half][lane quadrant][row] partial sums
  float bias[256];           // the epilogue's per-column vectors, staged once
  float wout[256];
};

// tcgen05.wait::ld that names the destination registers of the loads it waits for,
// so that their uses stay after it.
__device__ __forceinline__ void tmem_wait32(float (&v)[32]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+f"(v[0]), "+f"(v[1]), "+f"(v[2]), "+f"(v[3]), "+f"(v[4]), "+f"(v[5]), "+f"(v[6]), "+f"(v[7]),
                 "+f"(v[8]), "+f"(v[9]), "+f"(v[10]), "+f"(v[11]), "+f"(v[12]), "+f"(v[13]), "+f"(v[14]),
                 "+f"(v[15]), "+f"(v[16]), "+f"(v[17]), "+f"(v[18]), "+f"(v[19]), "+f"(v[20]), "+f"(v[21]),
                 "+f"(v[22]), "+f"(v[23]), "+f"(v[24]), "+f"(v[25]), "+f"(v[26]), "+f"(v[27]), "+f"(v[28]),
                 "+f"(v[29]), "+f"(v[30]), "+f"(v[31])
               :
               : "memory");
}
// f(c, v) on the kChunks consecutive 32-column chunks of a warp's accumulator rows
// (TMEM address ta).  kPipe: the next chunk's load is in flight while f works on
// this one (32 more registers); otherwise each chunk is loaded and waited for.
template <int kChunks, bool kPipe, class F>
__device__ __forceinline__ void acc_chunks(uint32_t ta, F&& f) {
  if constexpr (kPipe) {
    float va[32], vb[32];
    tmem_ld32(ta, va);
    tmem_wait32(va);
#pragma unroll
    for (int ci = 0; ci < kChunks; ++ci) {
      float(&v)[32] = (ci & 1) ? vb : va;
      float(&vn)[32] = (ci & 1) ? va : vb;
      if (ci + 1 < kChunks) tmem_ld32(ta + 32 * (ci + 1), vn);
      f(32 * ci, v);
      if (ci + 1 < kChunks) tmem_wait32(vn);
    }
  } else {
#pragma unroll 1
    for (int ci = 0; ci < kChunks; ++ci) {
      float v[32];
      tmem_ld32(ta + 32 * ci, v);
      tmem_wait32(v);
      f(32 * ci, v);
    }
  }
}

__device__ __forceinline__ bool g_aborted(Bars* b) { return *reinterpret_cast<volatile int*>(&b->abort) != 0; }
// the abort flag as lane 0 of the warp read it (a warp-uniform decision)
__device__ __forceinline__ bool g_aborted_warp(Bars* b, int lane) {
  const int v = lane == 0 ? *reinterpret_cast<volatile int*>(&b->abort) : 0;
  return __shfl_sync(0xffffffffu, v, 0) != 0;
}
__device__ __forceinline__ void g_wait(Bars* b, uint64_t* bar, uint32_t parity) {
  if (g_aborted(b)) return;
  if (!mbar_wait(bar, parity, kWait)) *reinterpret_cast<volatile int*>(&b->abort) = 1;
}

// ELU with e^z - 1 from the hardware 2^x (relative error ~2^-22; near z = 0 the
// subtraction leaves ~1e-7 absolute, far below the bf16 rounding of the outputs).
__device__ __forceinline__ float elu_g(float z) {
  return z > 0.f ? z : ex2_approx(z * 1.4426950408889634f) - 1.f;
}
__device__ __forceinline__ float elud_from_h(float h) { return h > 0.f ? 1.f : h + 1.f; }
__device__ __forceinline__ uint16_t to_bf16(float f) {
  __nv_bfloat16 h = __float2bfloat16_rn(f);
  return *reinterpret_cast<uint16_t*>(&h);
}

// Column sums over the 32 lanes of a warp of 32 per-lane values: five exchange
// rounds halve the set each time; lane l ends with the sum of column l.
__device__ __forceinline__ float warp_colsum32(float (&v)[32], int lane) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    const bool up = lane & off;
#pragma unroll
    for (int j = 0; j < off; ++j) {
      const float send = up ? v[j] : v[j + off];
      const float keep = up ? v[j + off] : v[j];
      v[j] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  return v[0];
}

// Per-warp staging of 32 bf16 rows of kW columns in shared memory, rows padded by
// 16 bytes so that one lane per row writing 16 bytes is conflict-free.
template <int kW>
struct Staging {
  static constexpr int kSt = kW + 8;  // row stride in elements
  uint16_t* base;                     // this warp's 32 rows
  __device__ __forceinline__ void put32(int lane, int c0, const float (&v)[32]) const {
    uint32_t w[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) w[j] = (uint32_t)to_bf16(v[2 * j]) | ((uint32_t)to_bf16(v[2 * j + 1]) << 16);
    uint4* d = reinterpret_cast<uint4*>(base + lane * kSt + c0);
#pragma unroll
    for (int j = 0; j < 4; ++j) d[j] = make_uint4(w[4 * j], w[4 * j + 1], w[4 * j + 2], w[4 * j + 3]);
  }
  __device__ __forceinline__ void get32(int lane, int c0, float (&v)[32]) const {
    const uint4* sp = reinterpret_cast<const uint4*>(base + lane * kSt + c0);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint4 q = sp[j];
      const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        v[8 * j + 2 * i] = __uint_as_float(w[i] << 16);
        v[8 * j + 2 * i + 1] = __uint_as_float(w[i] & 0xFFFF0000u);
      }
    }
  }
  // columns col0 .. col0 + kW - 1 of rows row0 .. row0 + 31 (those < M) of the [M][ld]
  // global array, whole staged rows per instruction (kW / 8 lanes per row)
  __device__ __forceinline__ void store_rows(uint16_t* dst, long ld, int row0, int col0, int M, int lane) const {
    __syncwarp();
    constexpr int kLpr = kW / 8, kRpi = 32 / kLpr;
#pragma unroll
    for (int r0 = 0; r0 < 32; r0 += kRpi) {
      const int r = r0 + lane / kLpr, c = (lane % kLpr) * 8;
      if (row0 + r < M)
        *reinterpret_cast<uint4*>(dst + (long)(row0 + r) * ld + col0 + c) =
            *reinterpret_cast<const uint4*>(base + r * kSt + c);
    }
    __syncwarp();
  }
  __device__ __forceinline__ void load_rows(const uint16_t* src, long ld, int row0, int col0, int M, int lane) const {
    __syncwarp();
    constexpr int kLpr = kW / 8, kRpi = 32 / kLpr;
#pragma unroll
    for (int r0 = 0; r0 < 32; r0 += kRpi) {
      const int r = r0 + lane / kLpr, c = (lane % kLpr) * 8;
      uint4 q = make_uint4(0u, 0u, 0u, 0u);
      if (row0 + r < M) q = __ldg(reinterpret_cast<const uint4*>(src + (long)(row0 + r) * ld + col0 + c));
      *reinterpret_cast<uint4*>(base + r * kSt + c) = q;
    }
    __syncwarp();
  }
  // load_rows in two halves: fetch_rows issues the global loads into registers (the
  // loads stay in flight while the caller does other work), put_rows writes them to
  // the staging rows
  static constexpr int kFetch = 32 / (32 / (kW / 8));  // 16-byte loads per lane
  __device__ __forceinline__ void fetch_rows(const uint16_t* src, long ld, int row0, int col0, int M, int lane,
                                             uint4 (&R)[kFetch]) const {
    constexpr int kLpr = kW / 8, kRpi = 32 / kLpr;
#pragma unroll
    for (int i = 0; i < kFetch; ++i) {
      const int r = i * kRpi + lane / kLpr, c = (lane % kLpr) * 8;
      R[i] = make_uint4(0u, 0u, 0u, 0u);
      if (row0 + r < M) R[i] = __ldg(reinterpret_cast<const uint4*>(src + (long)(row0 + r) * ld + col0 + c));
    }
  }
  __device__ __forceinline__ void put_rows(int lane, const uint4 (&R)[kFetch]) const {
    constexpr int kLpr = kW / 8, kRpi = 32 / kLpr;
    __syncwarp();
#pragma unroll
    for (int i = 0; i < kFetch; ++i) {
      const int r = i * kRpi + lane / kLpr, c = (lane % kLpr) * 8;
      *reinterpret_cast<uint4*>(base + r * kSt + c) = R[i];
    }
    __syncwarp();
  }
};

template <int kBN, int kEpi>
__global__ void __launch_bounds__(kGemmThreads, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, Args g) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr uint32_t kABytes = kBM * kBK * 2, kBBytes = kBN * kBK * 2, kStageBytes = kABytes + kBBytes;
  constexpr int kHalf = kBN / 2;  // columns per epilogue warp
  constexpr size_t kStgBytes = (size_t)kEpiWarps * 32 * Staging<kHalf>::kSt * 2;
  Bars* bars = reinterpret_cast<Bars*>(sm + kStages * kStageBytes + kStgBytes);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&bars->full[s], 1);
      mbar_init(&bars->empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&bars->tfull[a], 1);
      mbar_init(&bars->tempty[a], kEpiWarps);
    }
    bars->abort = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(&bars->tmem_base, 2 * kBN);
    tmem_relinquish();
  }
  for (int i = tid; i < g.N; i += blockDim.x) {
    bars->bias[i] = g.bias ? g.bias[i] : 0.f;
    bars->wout[i] = g.wout ? g.wout[i] : 0.f;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tb = bars->tmem_base;
  const int tiles = g.tiles_m * g.splits;
  const int kblocks_total = (g.K + kBK - 1) / kBK;

  if (warp == 0) {
    // ------------------------------------------------ TMA producer (one thread)
    uint32_t stage = 0, phase = 0;
    for (int t = blockIdx.x; t < tiles && lane == 0; t += gridDim.x) {
      const int mt = t % g.tiles_m, sp = t / g.tiles_m;
      const int kb0 = sp * g.kb_per_split, kb1 = min(kblocks_total, kb0 + g.kb_per_split);
      for (int kb = kb0; kb < kb1; ++kb) {
        g_wait(bars, &bars->empty[stage], phase ^ 1);
        if (!g_aborted(bars)) {
          uint8_t* As = sm + stage * kStageBytes;
          uint8_t* Bs = As + kABytes;
          mbar_arrive_expect_tx(&bars->full[stage], kStageBytes);
          const int k0 = kb * kBK, m0 = mt * kBM;
          if (!g.a_mn) {
            tma_load_2d(As, &tmA, k0, m0, &bars->full[stage]);
          } else {
            tma_load_2d(As, &tmA, m0, k0, &bars->full[stage]);
            tma_load_2d(As + 8192, &tmA, m0 + 64, k0, &bars->full[stage]);
          }
          if (!g.b_mn) {
            tma_load_2d(Bs, &tmB, k0, 0, &bars->full[stage]);
          } else {
#pragma unroll
            for (int j = 0; j < kBN / 64; ++j) tma_load_2d(Bs + j * 8192, &tmB, j * 64, k0, &bars->full[stage]);
          }
        }
        if (++stage == kStages) {
          stage = 0;
          phase ^= 1;
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------ MMA issuer
    uint32_t stage = 0, phase = 0;
    uint32_t tphase[2] = {0, 0};
    const uint32_t idesc = idesc_f16(kBM, kBN, g.a_mn != 0, g.b_mn != 0, true);
    int local = 0;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++local) {
      const int acc = local & 1;
      const int sp = t / g.tiles_m;
      const int kb0 = sp * g.kb_per_split, kb1 = min(kblocks_total, kb0 + g.kb_per_split);
      g_wait(bars, &bars->tempty[acc], tphase[acc] ^ 1);
      tphase[acc] ^= 1;
      tc_fence_after();
      const uint32_t d = tb + (uint32_t)acc * kBN;
      for (int kb = kb0; kb < kb1; ++kb) {
        g_wait(bars, &bars->full[stage], phase);
        tc_fence_after();
        if (!g_aborted_warp(bars, lane)) {
          const uint32_t a_addr = smem_u32(sm + stage * kStageBytes), b_addr = a_addr + kABytes;
#pragma unroll
          for (int kk = 0; kk < kBK / 16; ++kk) {
            const uint64_t ad = g.a_mn ? smem_desc_sw128(a_addr + kk * 2048, 8192, 1024)
                                       : smem_desc_sw128(a_addr + kk * 32, 16, 1024);
            const uint64_t bd = g.b_mn ? smem_desc_sw128(b_addr + kk * 2048, 8192, 1024)
                                       : smem_desc_sw128(b_addr + kk * 32, 16, 1024);
            umma_f16_warp(d, ad, bd, idesc, (kb > kb0 || kk > 0) ? 1u : 0u);
          }
          umma_commit_warp(&bars->empty[stage]);
        }
        if (++stage == kStages) {
          stage = 0;
          phase ^= 1;
        }
      }
      if (!g_aborted_warp(bars, lane)) umma_commit_warp(&bars->tfull[acc]);
    }
  } else {
    // ------------------------------------------------ epilogue
    const int ew = warp - 2;
    const int q = warp & 3;                 // TMEM lane quadrant of this warp
    const int half = ew >> 2, cb = half * kHalf;  // its column half
    const Staging<kHalf> stg{reinterpret_cast<uint16_t*>(sm + kStages * kStageBytes) + ew * 32 * Staging<kHalf>::kSt};
    uint32_t tphase[2] = {0, 0};
    int local = 0;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++local) {
      const int acc = local & 1;
      const int mt = t % g.tiles_m, sp = t / g.tiles_m;
      const int row0 = mt * kBM + q * 32;
      const int row = row0 + lane;
      const bool in = row < g.M;
      // h_{l-1} of the tile's rows does not depend on the accumulator: the first tile
      // reads it here, later ones were fetched during the previous tile's stores
      if (kEpi == kGemmEpiTimesEluD && local == 0) stg.load_rows(g.hprev, g.ldo, row0, cb, g.M, lane);
      g_wait(bars, &bars->tfull[acc], tphase[acc]);
      tphase[acc] ^= 1;
      tc_fence_after();
      const uint32_t ta = tb + (uint32_t)acc * kBN + (uint32_t)cb + ((uint32_t)(q * 32) << 16);
      float gval = 0.f;
      constexpr int kCh = kHalf / 32;
      const float* sbias = bars->bias + cb;
      const float* swout = bars->wout + cb;
      if (kEpi == kGemmEpiOut) {
        // h_L = ELU(z + b) and this half's share of the output layer w_out . h_L (FP32)
        acc_chunks<kCh, true>(ta, [&](int c0, float(&v)[32]) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const float h = elu_g(v[j] + sbias[c0 + j]);
            v[j] = h;
            gval = fmaf(swout[c0 + j], h, gval);
          }
          stg.put32(lane, c0, v);
        });
      } else {
      // pipelined where the epilogue holds one 32-value row (bias + ELU, FP32 partials)
      acc_chunks<kCh, kEpi == kGemmEpiBiasElu || kEpi == kGemmEpiF32>(ta, [&](int c0, float(&v)[32]) {
        const int col = cb + c0;
        if (kEpi == kGemmEpiF32) {
          if (in) {
            float4* o = reinterpret_cast<float4*>(g.out_f32 + (long)sp * g.M * g.ldo + (long)row * g.ldo + col);
#pragma unroll
            for (int j = 0; j < 8; ++j) o[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
          }
        } else if (kEpi == kGemmEpiBiasElu) {
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] = elu_g(v[j] + sbias[c0 + j]);
          stg.put32(lane, c0, v);
        } else if (kEpi == kGemmEpiTimesEluD) {
          float hp[32];
          stg.get32(lane, c0, hp);
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] = in ? v[j] * elud_from_h(hp[j]) : 0.f;
          stg.put32(lane, c0, v);                    // in place of the h values just read
          const float cs = warp_colsum32(v, lane);  // column sums of delta over this warp's rows
          g.colpart[(long)(mt * 4 + q) * g.N + col + lane] = cs;
        }
      });
      }
      // the accumulator is read: hand it back before the stores
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars->tempty[acc]);
      if (kEpi == kGemmEpiBiasElu) stg.store_rows(g.out_bf16, g.ldo, row0, cb, g.M, lane);
      if (kEpi == kGemmEpiTimesEluD) {
        // the next tile's h_{l-1} rows are loaded while this tile's delta rows are stored
        const int tn = t + gridDim.x;
        uint4 R[Staging<kHalf>::kFetch];
        if (tn < tiles) stg.fetch_rows(g.hprev, g.ldo, (tn % g.tiles_m) * kBM + q * 32, cb, g.M, lane, R);
        stg.store_rows(g.out_bf16, g.ldo, row0, cb, g.M, lane);
        if (tn < tiles) stg.put_rows(lane, R);
      }
      if (kEpi == kGemmEpiOut) {
        stg.store_rows(g.out_bf16, g.ldo, row0, cb, g.M, lane);
        // the two column halves' partial sums meet in shared memory, added in a fixed
        // order; the residual g - target of each row
        bars->gpart[local & 1][half][q][lane] = gval;
        asm volatile("bar.sync %0, 64;" ::"r"(1 + q) : "memory");  // the two warps of quadrant q
        gval = bars->gpart[local & 1][0][q][lane] + bars->gpart[local & 1][1][q][lane];
        if (half == 0 && in) g.resid[row] = gval + __ldg(g.bout) - __ldg(g.target + row);
      }
    }
  }
  // drain: the producer's last loads and the issuer's last UMMAs have been waited
  // for by the epilogue (tile completions); a CTA that gave up waits no further
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && g_aborted(bars)) atomicExch(g.flag, 1);
  if (warp == 1) tmem_dealloc(tb, 2 * kBN);
}

// ---- tensor maps (driver entry point fetched through the runtime once)
typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
  static EncodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  });
  return fn;
}

// 2D bf16 map over a matrix with `inner` contiguous elements per row (row stride
// `ld` elements) and `outer` rows; box (64, box_outer), 128-byte swizzle, zero fill
// outside the matrix.
bool make_map(CUtensorMap* m, const void* base, long inner, long outer, long ld, int box_outer) {
  EncodeTiled fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {64, (cuuint32_t)box_outer};
  const cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int kBN, int kEpi>
cudaError_t launch_bn(const CUtensorMap& ta, const CUtensorMap& tbm, const Args& a, int grid, cudaStream_t s) {
  const size_t smem = 1024 + (size_t)kStages * (kBM * kBK * 2 + kBN * kBK * 2) +
                      (size_t)kEpiWarps * 32 * Staging<kBN / 2>::kSt * 2 + sizeof(Bars);
  auto k = gemm_tc_kernel<kBN, kEpi>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<grid, kGemmThreads, smem, s>>>(ta, tbm, a);
  return cudaGetLastError();
}

template <int kEpi>
cudaError_t launch_epi(int bn, const CUtensorMap& ta, const CUtensorMap& tbm, const Args& a, int grid,
                       cudaStream_t s) {
  if (bn == 64) return launch_bn<64, kEpi>(ta, tbm, a, grid, s);
  if (bn == 128) return launch_bn<128, kEpi>(ta, tbm, a, grid, s);
  return launch_bn<256, kEpi>(ta, tbm, a, grid, s);
}

}  // namespace

bool tc_gemm_supported(int n) { return n == 64 || n == 128 || n == 256; }

cudaError_t tc_gemm(const TcGemm& p, int num_sms, int* flag, cudaStream_t s) {
  if (!tc_gemm_supported(p.N) || p.M <= 0 || p.K <= 0 || p.splits < 1) return cudaErrorInvalidValue;
  // TMA row strides are multiples of 16 bytes, boxes start on 64-element columns
  if ((p.lda * 2) % 16 || (p.ldb * 2) % 16 || ((uintptr_t)p.A & 15) || ((uintptr_t)p.B & 15))
    return cudaErrorInvalidValue;
  CUtensorMap ta, tbm;
  bool ok = p.a_mn ? make_map(&ta, p.A, p.M, p.K, p.lda, 64) : make_map(&ta, p.A, p.K, p.M, p.lda, kBM);
  ok = ok && (p.b_mn ? make_map(&tbm, p.B, p.N, p.K, p.ldb, 64) : make_map(&tbm, p.B, p.K, p.N, p.ldb, p.N));
  if (!ok) return cudaErrorInvalidValue;
  Args a{};
  a.M = p.M;
  a.N = p.N;
  a.K = p.K;
  a.a_mn = p.a_mn;
  a.b_mn = p.b_mn;
  a.tiles_m = (p.M + kBM - 1) / kBM;
  const int kblocks = (p.K + kBK - 1) / kBK;
  a.splits = std::min(p.splits, kblocks);
  a.kb_per_split = (kblocks + a.splits - 1) / a.splits;
  a.splits = (kblocks + a.kb_per_split - 1) / a.kb_per_split;
  a.epi = p.epi;
  a.out_f32 = p.out_f32;
  a.ldo = p.ldo;
  a.out_bf16 = p.out_bf16;
  a.bias = p.bias;
  a.hprev = p.hprev;
  a.colpart = p.colpart;
  a.wout = p.wout;
  a.bout = p.bout;
  a.target = p.target;
  a.resid = p.resid;
  a.flag = flag;
  const long tiles = (long)a.tiles_m * a.splits;
  const int grid = (int)std::min<long>(tiles, num_sms);
  switch (p.epi) {
    case kGemmEpiF32: return launch_epi<kGemmEpiF32>(p.N, ta, tbm, a, grid, s);
    case kGemmEpiBiasElu: return launch_epi<kGemmEpiBiasElu>(p.N, ta, tbm, a, grid, s);
    case kGemmEpiTimesEluD: return launch_epi<kGemmEpiTimesEluD>(p.N, ta, tbm, a, grid, s);
    case kGemmEpiOut: return launch_epi<kGemmEpiOut>(p.N, ta, tbm, a, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

int tc_gemm_splits_used(int K, int splits) {
  const int kblocks = (K + kBK - 1) / kBK;
  const int sp = std::min(splits, kblocks);
  const int per = (kblocks + sp - 1) / sp;
  return (kblocks + per - 1) / per;
}

}  // namespace crom
