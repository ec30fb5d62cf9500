// Full-order models on the GPU: explicit finite differences + forward Euler
// (paper App. G.2 for the 1D heat equation, App. H.2 for the 2D form), batched
// over independent fields.  These generate the training data and the reference
// solutions that rollouts are compared with; every update is a 5-point (3-point in 1D) stencil, so the
// kernels are bound by memory traffic: one read and one write of u per node and
// step (plus the two face velocities for advection).  The 2D kernels for sides
// that are multiples of 128 march down short row strips with neighbours in
// registers and lanes; the others serve neighbour values from L1/L2.
//
//  * heat 1D, Dirichlet 0: nodes x_i = i/(P-1); interior
//      u_i += dt * nu * (u_{i-1} + u_{i+1} - 2 u_i) / dx^2, boundary nodes = 0.
//  * heat 2D, zero Neumann: nodes (i, j)/(n-1); mirror ghost nodes
//      u_{-1} = u_1, u_n = u_{n-2}; u += dt * alpha * Lap_h u.
//  * advection-diffusion 2D, periodic cells of width 1/n: conservative fluxes
//      with face velocities ax[i][j] (between cells (i, j) and (i+1, j)) and
//      ay[i][j] (between (i, j) and (i, j+1)), central diffusion:
//      u += dt * (-div(a u) + nu * Lap_h u).  The face value is the upwind cell's
//      (first order; its numerical diffusion |a| h / 2 is part of the model) or
//      the mean of the two cells (second order, central).
//  * the heat models with a spatially varying coefficient nu(x) (App. G and H):
//      the same stencils with nu read per node.
// Layout: fields [n_batch][nx][ny] FP32 row-major (j fastest); face velocities
// [n_batch][nx][ny]; coefficients nu/alpha per field, or per node (same layout
// as the fields) for the *_FIELD kinds.
#include "crom_internal.h"

namespace crom {
namespace {

// Flux a * u_face through a face between the cells `left` and `right` (a > 0 moves
// from left to right): upwind takes the upstream cell, central the mean of the two.
template <bool kCentral>
__device__ __forceinline__ float face_flux(float a, float left, float right) {
  return kCentral ? a * (0.5f * (left + right)) : a * (a > 0.f ? left : right);
}

template <bool kField>
__global__ void heat1d_kernel(const float* __restrict__ u, float* __restrict__ out, const float* __restrict__ coef,
                              int P, float r_over) {
  // r_over = dt / dx^2
  const int b = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  const float* ub = u + (size_t)b * P;
  float v = 0.f;
  if (i > 0 && i < P - 1) {
    const float c = ub[i];
    const float nu = kField ? coef[(size_t)b * P + i] : coef[b];
    v = fmaf(r_over * nu, ub[i - 1] + ub[i + 1] - 2.f * c, c);
  }
  out[(size_t)b * P + i] = v;
}

template <bool kField>
__global__ void heat2d_neumann_kernel(const float* __restrict__ u, float* __restrict__ out,
                                      const float* __restrict__ coef, int n, float r_over) {
  // r_over = dt / h^2; block = 32 x 8 nodes, j fastest
  const int b = blockIdx.z;
  const int j = blockIdx.x * 32 + threadIdx.x;
  const int i = blockIdx.y * 8 + threadIdx.y;
  if (i >= n || j >= n) return;
  const float* ub = u + (size_t)b * n * n;
  const int im = i > 0 ? i - 1 : 1, ip = i < n - 1 ? i + 1 : n - 2;
  const int jm = j > 0 ? j - 1 : 1, jp = j < n - 1 ? j + 1 : n - 2;
  const float c = ub[(size_t)i * n + j];
  const float lap = (ub[(size_t)im * n + j] + ub[(size_t)ip * n + j] - 2.f * c) +
                    (ub[(size_t)i * n + jm] + ub[(size_t)i * n + jp] - 2.f * c);
  const size_t at = (size_t)b * n * n + (size_t)i * n + j;
  const float nu = kField ? coef[at] : coef[b];
  out[at] = fmaf(r_over * nu, lap, c);
}

template <bool kCentral>
__global__ void advdiff2d_kernel(const float* __restrict__ u, float* __restrict__ out,
                                 const float* __restrict__ ax, const float* __restrict__ ay,
                                 const float* __restrict__ coef, int n, float dt, float inv_h, float inv_h2) {
  const int b = blockIdx.z;
  const int j = blockIdx.x * 32 + threadIdx.x;
  const int i = blockIdx.y * 8 + threadIdx.y;
  if (i >= n || j >= n) return;
  const size_t base = (size_t)b * n * n;
  const float* ub = u + base;
  const float* axb = ax + base;
  const float* ayb = ay + base;
  const int im = i > 0 ? i - 1 : n - 1, ip = i < n - 1 ? i + 1 : 0;
  const int jm = j > 0 ? j - 1 : n - 1, jp = j < n - 1 ? j + 1 : 0;
  const float c = ub[(size_t)i * n + j];
  const float uim = ub[(size_t)im * n + j], uip = ub[(size_t)ip * n + j];
  const float ujm = ub[(size_t)i * n + jm], ujp = ub[(size_t)i * n + jp];
  const float a_r = axb[(size_t)i * n + j], a_l = axb[(size_t)im * n + j];
  const float b_r = ayb[(size_t)i * n + j], b_l = ayb[(size_t)i * n + jm];
  const float fr = face_flux<kCentral>(a_r, c, uip);    // flux through the face (i+1/2, j)
  const float fl = face_flux<kCentral>(a_l, uim, c);    // flux through the face (i-1/2, j)
  const float gr = face_flux<kCentral>(b_r, c, ujp);
  const float gl = face_flux<kCentral>(b_l, ujm, c);
  const float div = (fr - fl + gr - gl) * inv_h;
  const float lap = (uim + uip + ujm + ujp - 4.f * c) * inv_h2;
  out[base + (size_t)i * n + j] = fmaf(dt, fmaf(coef[b], lap, -div), c);
}

// The same update, marching: each warp owns 32 consecutive columns j and a strip of
// kRows rows i, keeps u at rows i-1, i, i+1 and the x-face velocity of row i-1 in
// registers, and takes the j-neighbours from the adjacent lanes (the two columns
// beyond the warp from memory).  Every field value and face velocity is read once
// per strip (plus two halo rows), so the kernel streams 16 B per node-step.
// Requires n % 32 == 0 and n % (kRows * kWarps) == 0.
constexpr int kRows = 32, kWarps = 4;
template <bool kCentral>
__global__ void __launch_bounds__(32 * kWarps) advdiff2d_march_kernel(
    const float* __restrict__ u, float* __restrict__ out, const float* __restrict__ ax,
    const float* __restrict__ ay, const float* __restrict__ coef, int n, float dt, float inv_h, float inv_h2) {
  const int b = blockIdx.z;
  const int lane = threadIdx.x;
  const int j = blockIdx.x * 32 + lane;
  const int i0 = (blockIdx.y * kWarps + threadIdx.y) * kRows;
  const size_t base = (size_t)b * n * n;
  const float* ub = u + base;
  const float* axb = ax + base;
  const float* ayb = ay + base;
  float* ob = out + base;
  const float nu = coef[b];
  const int jl = blockIdx.x * 32 == 0 ? n - 1 : blockIdx.x * 32 - 1;   // column left of the warp
  const int jr = blockIdx.x * 32 + 32 == n ? 0 : blockIdx.x * 32 + 32; // column right of the warp
  int im = i0 == 0 ? n - 1 : i0 - 1;
  float uim = ub[(size_t)im * n + j];
  float c = ub[(size_t)i0 * n + j];
  float a_l = axb[(size_t)im * n + j];
#pragma unroll 4
  for (int k = 0; k < kRows; ++k) {
    const int i = i0 + k;
    const int ip = i == n - 1 ? 0 : i + 1;
    const float uip = ub[(size_t)ip * n + j];
    const float a_r = axb[(size_t)i * n + j];
    const float b_r = ayb[(size_t)i * n + j];
    // halo columns: lane 0 needs column jl, lane 31 column jr
    const float halo_u = lane == 0 ? ub[(size_t)i * n + jl] : (lane == 31 ? ub[(size_t)i * n + jr] : 0.f);
    const float halo_b = lane == 0 ? ayb[(size_t)i * n + jl] : 0.f;
    float ujm = __shfl_up_sync(0xffffffffu, c, 1);
    float ujp = __shfl_down_sync(0xffffffffu, c, 1);
    float b_l = __shfl_up_sync(0xffffffffu, b_r, 1);
    if (lane == 0) {
      ujm = halo_u;
      b_l = halo_b;
    }
    if (lane == 31) ujp = halo_u;
    const float fr = face_flux<kCentral>(a_r, c, uip);
    const float fl = face_flux<kCentral>(a_l, uim, c);
    const float gr = face_flux<kCentral>(b_r, c, ujp);
    const float gl = face_flux<kCentral>(b_l, ujm, c);
    const float div = (fr - fl + gr - gl) * inv_h;
    const float lap = (uim + uip + ujm + ujp - 4.f * c) * inv_h2;
    ob[(size_t)i * n + j] = fmaf(dt, fmaf(nu, lap, -div), c);
    uim = c;
    c = uip;
    a_l = a_r;
  }
}

// The marching update with four columns per lane (float4 loads and stores): a warp
// owns 128 consecutive columns and a strip of kRowsA rows; within a lane the column
// neighbours are the adjacent components, across lanes they come from a shuffle of
// the first / last component, and the two columns beyond the warp from memory.
// Requires n % 128 == 0, n % (kRowsA * kWarps4) == 0 and 16-byte aligned arrays.
constexpr int kWarps4 = 4;
// Rows per warp strip of the four-columns-per-lane kernels: short strips keep many
// warps' loads in flight (the rows above and below a strip are re-read, mostly from
// L2); measured on 512 / 1024 fields of 256^2: 32 rows 86 / 80 %, 16 rows 91 / 85 %,
// 8 rows 93 / 91 %, 4 rows 97 / 97 %, 2 rows 99 / 95 % of the copy bandwidth
// (advection-diffusion / heat).
constexpr int kRowsAdv = 2, kRowsHeat = 4;
inline bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }
template <int kRowsA, bool kCentral>
__global__ void __launch_bounds__(32 * kWarps4) advdiff2d_march4_kernel(
    const float* __restrict__ u, float* __restrict__ out, const float* __restrict__ ax,
    const float* __restrict__ ay, const float* __restrict__ coef, int n, float dt, float inv_h, float inv_h2) {
  const int b = blockIdx.z;
  const int lane = threadIdx.x;
  const int j0 = blockIdx.x * 128;
  const int j = j0 + 4 * lane;
  const int i0 = (blockIdx.y * kWarps4 + threadIdx.y) * kRowsA;
  const size_t base = (size_t)b * n * n;
  const float* ub = u + base;
  const float* axb = ax + base;
  const float* ayb = ay + base;
  float* ob = out + base;
  const float nu = coef[b];
  const int jl = j0 == 0 ? n - 1 : j0 - 1;          // column left of the warp
  const int jr = j0 + 128 == n ? 0 : j0 + 128;      // column right of the warp
  auto ld4 = [&](const float* p, int i) { return *reinterpret_cast<const float4*>(p + (size_t)i * n + j); };
  const int im0 = i0 == 0 ? n - 1 : i0 - 1;
  float4 uim = ld4(ub, im0);
  float4 c = ld4(ub, i0);
  float4 a_l = ld4(axb, im0);
#pragma unroll 4
  for (int k = 0; k < kRowsA; ++k) {
    const int i = i0 + k;
    const int ip = i == n - 1 ? 0 : i + 1;
    const float4 uip = ld4(ub, ip);
    const float4 a_r = ld4(axb, i);
    const float4 b_r = ld4(ayb, i);
    // halo columns: lane 0 needs column jl (u and the y-face velocity), lane 31 column jr (u)
    const float halo_u = lane == 0 ? ub[(size_t)i * n + jl] : (lane == 31 ? ub[(size_t)i * n + jr] : 0.f);
    const float halo_b = lane == 0 ? ayb[(size_t)i * n + jl] : 0.f;
    float ujm0 = __shfl_up_sync(0xffffffffu, c.w, 1);
    float ujp3 = __shfl_down_sync(0xffffffffu, c.x, 1);
    float b_l0 = __shfl_up_sync(0xffffffffu, b_r.w, 1);
    if (lane == 0) {
      ujm0 = halo_u;
      b_l0 = halo_b;
    }
    if (lane == 31) ujp3 = halo_u;
    const float cv[4] = {c.x, c.y, c.z, c.w};
    const float um[4] = {uim.x, uim.y, uim.z, uim.w};
    const float up[4] = {uip.x, uip.y, uip.z, uip.w};
    const float ar[4] = {a_r.x, a_r.y, a_r.z, a_r.w};
    const float al[4] = {a_l.x, a_l.y, a_l.z, a_l.w};
    const float br[4] = {b_r.x, b_r.y, b_r.z, b_r.w};
    const float jm[4] = {ujm0, c.x, c.y, c.z};
    const float jp[4] = {c.y, c.z, c.w, ujp3};
    const float bl[4] = {b_l0, b_r.x, b_r.y, b_r.z};
    float o[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float div = (face_flux<kCentral>(ar[q], cv[q], up[q]) - face_flux<kCentral>(al[q], um[q], cv[q]) +
                         face_flux<kCentral>(br[q], cv[q], jp[q]) - face_flux<kCentral>(bl[q], jm[q], cv[q])) *
                        inv_h;
      const float lap = (um[q] + up[q] + jm[q] + jp[q] - 4.f * cv[q]) * inv_h2;
      o[q] = fmaf(dt, fmaf(nu, lap, -div), cv[q]);
    }
    *reinterpret_cast<float4*>(ob + (size_t)i * n + j) = make_float4(o[0], o[1], o[2], o[3]);
    uim = c;
    c = uip;
    a_l = a_r;
  }
}

// 2D heat with zero-flux (mirror) boundaries, marching with four columns per lane
// as above: the mirror ghosts are u_{-1} = u_1 and u_n = u_{n-2} in both directions
// (row 0 takes row 1 as its upper neighbour, row n-1 row n-2 as its lower one; in
// column 0 and n-1 the lane's own component j = 1 or n-2 is the missing neighbour).
// kField: the coefficient is read per node (float4), else per field.  kRowsH rows
// per warp strip.  Requires n % 128 == 0, n % (kRowsH * kWarps4) == 0 and 16-byte
// aligned arrays.
template <bool kField, int kRowsH>
__global__ void __launch_bounds__(32 * kWarps4) heat2d_march4_kernel(const float* __restrict__ u,
                                                                    float* __restrict__ out,
                                                                    const float* __restrict__ coef, int n,
                                                                    float r_over) {
  const int b = blockIdx.z;
  const int lane = threadIdx.x;
  const int j0 = blockIdx.x * 128;
  const int j = j0 + 4 * lane;
  const int i0 = (blockIdx.y * kWarps4 + threadIdx.y) * kRowsH;
  const size_t base = (size_t)b * n * n;
  const float* ub = u + base;
  float* ob = out + base;
  const float nu_b = kField ? 0.f : coef[b];
  const bool left_edge = j0 == 0, right_edge = j0 + 128 == n;
  auto ld4 = [&](const float* p, int i) { return *reinterpret_cast<const float4*>(p + (size_t)i * n + j); };
  float4 uim = ld4(ub, i0 == 0 ? 1 : i0 - 1);
  float4 c = ld4(ub, i0);
#pragma unroll 4
  for (int k = 0; k < kRowsH; ++k) {
    const int i = i0 + k;
    const float4 uip = ld4(ub, i == n - 1 ? n - 2 : i + 1);
    // halo columns: lane 0 needs column j0 - 1, lane 31 column j0 + 128 (inside the field)
    const float halo = (lane == 0 && !left_edge) ? ub[(size_t)i * n + j0 - 1]
                       : (lane == 31 && !right_edge) ? ub[(size_t)i * n + j0 + 128] : 0.f;
    float ujm0 = __shfl_up_sync(0xffffffffu, c.w, 1);
    float ujp3 = __shfl_down_sync(0xffffffffu, c.x, 1);
    if (lane == 0) ujm0 = left_edge ? c.y : halo;
    if (lane == 31) ujp3 = right_edge ? c.z : halo;
    const float cv[4] = {c.x, c.y, c.z, c.w};
    const float um[4] = {uim.x, uim.y, uim.z, uim.w};
    const float up[4] = {uip.x, uip.y, uip.z, uip.w};
    const float jm[4] = {ujm0, c.x, c.y, c.z};
    const float jp[4] = {c.y, c.z, c.w, ujp3};
    float nu[4] = {nu_b, nu_b, nu_b, nu_b};
    if (kField) {
      const float4 f = ld4(coef + base, i);
      nu[0] = f.x; nu[1] = f.y; nu[2] = f.z; nu[3] = f.w;
    }
    float o[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float lap = (um[q] + up[q] - 2.f * cv[q]) + (jm[q] + jp[q] - 2.f * cv[q]);
      o[q] = fmaf(r_over * nu[q], lap, cv[q]);
    }
    *reinterpret_cast<float4*>(ob + (size_t)i * n + j) = make_float4(o[0], o[1], o[2], o[3]);
    uim = c;
    c = uip;
  }
}

}  // namespace

cudaError_t launch_fom(int kind, int n_batch, int nx, int ny, const float* coef, const float* ax, const float* ay,
                       double dt, int n_steps, float* u, float* tmp, cudaStream_t s) {
  float* src = u;
  float* dst = tmp;
  for (int k = 0; k < n_steps; ++k) {
    if (kind == CROM_FOM_HEAT1D_DIRICHLET || kind == CROM_FOM_HEAT1D_DIRICHLET_FIELD) {
      const double dx = 1.0 / (nx - 1);
      dim3 grid((nx + 255) / 256, n_batch);
      if (kind == CROM_FOM_HEAT1D_DIRICHLET)
        heat1d_kernel<false><<<grid, 256, 0, s>>>(src, dst, coef, nx, (float)(dt / (dx * dx)));
      else
        heat1d_kernel<true><<<grid, 256, 0, s>>>(src, dst, coef, nx, (float)(dt / (dx * dx)));
    } else if (kind == CROM_FOM_HEAT2D_NEUMANN || kind == CROM_FOM_HEAT2D_NEUMANN_FIELD) {
      const double h = 1.0 / (nx - 1);
      const bool field = kind == CROM_FOM_HEAT2D_NEUMANN_FIELD;
      const float ro = (float)(dt / (h * h));
      if (nx % 128 == 0 && nx % (kRowsHeat * kWarps4) == 0 && aligned16(src) && aligned16(dst) &&
          (!field || aligned16(coef))) {
        dim3 grid4(nx / 128, nx / (kRowsHeat * kWarps4), n_batch);
        if (field)
          heat2d_march4_kernel<true, kRowsHeat><<<grid4, dim3(32, kWarps4), 0, s>>>(src, dst, coef, nx, ro);
        else
          heat2d_march4_kernel<false, kRowsHeat><<<grid4, dim3(32, kWarps4), 0, s>>>(src, dst, coef, nx, ro);
      } else {
        dim3 grid((nx + 31) / 32, (nx + 7) / 8, n_batch);
        if (field)
          heat2d_neumann_kernel<true><<<grid, dim3(32, 8), 0, s>>>(src, dst, coef, nx, (float)(dt / (h * h)));
        else
          heat2d_neumann_kernel<false><<<grid, dim3(32, 8), 0, s>>>(src, dst, coef, nx, (float)(dt / (h * h)));
      }
    } else {
      const double h = 1.0 / nx;
      const bool central = kind == CROM_FOM_ADVDIFF2D_PERIODIC_CENTRAL;
      const float fdt = (float)dt, ih = (float)(1.0 / h), ih2 = (float)(1.0 / (h * h));
      if (nx % 128 == 0 && nx % (kRowsAdv * kWarps4) == 0 && aligned16(src) && aligned16(dst) && aligned16(ax) &&
          aligned16(ay)) {
        dim3 grid(nx / 128, nx / (kRowsAdv * kWarps4), n_batch);
        if (central)
          advdiff2d_march4_kernel<kRowsAdv, true><<<grid, dim3(32, kWarps4), 0, s>>>(src, dst, ax, ay, coef, nx, fdt,
                                                                                   ih, ih2);
        else
          advdiff2d_march4_kernel<kRowsAdv, false><<<grid, dim3(32, kWarps4), 0, s>>>(src, dst, ax, ay, coef, nx, fdt,
                                                                                    ih, ih2);
      } else if (nx % 32 == 0 && nx % (kRows * kWarps) == 0) {
        dim3 grid(nx / 32, nx / (kRows * kWarps), n_batch);
        if (central)
          advdiff2d_march_kernel<true><<<grid, dim3(32, kWarps), 0, s>>>(src, dst, ax, ay, coef, nx, fdt, ih, ih2);
        else
          advdiff2d_march_kernel<false><<<grid, dim3(32, kWarps), 0, s>>>(src, dst, ax, ay, coef, nx, fdt, ih, ih2);
      } else {
        dim3 grid((nx + 31) / 32, (nx + 7) / 8, n_batch);
        if (central)
          advdiff2d_kernel<true><<<grid, dim3(32, 8), 0, s>>>(src, dst, ax, ay, coef, nx, fdt, ih, ih2);
        else
          advdiff2d_kernel<false><<<grid, dim3(32, 8), 0, s>>>(src, dst, ax, ay, coef, nx, fdt, ih, ih2);
      }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    float* t = src;
    src = dst;
    dst = t;
  }
  if (src != u) {
    const size_t bytes = (size_t)n_batch * nx * ny * sizeof(float);
    return cudaMemcpyAsync(u, src, bytes, cudaMemcpyDeviceToDevice, s);
  }
  return cudaSuccess;
}

}  // namespace crom
