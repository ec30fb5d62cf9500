// Kernels of the robust integration-sample selection (paper App. B, Algorithm 1):
// batch assembly (one rollout instance per candidate sample set and training
// parameter), the per-node residual res[c][i] = sum_mu |g(x_i, q_T) - f_FOM(x_i)|,
// Metric = mean + max per candidate, and the n_try largest residuals.  The
// greedy loop itself runs on the host (crom_robust_samples in crom_api.cu).
#include <math.h>

#include "crom_internal.h"

namespace crom {
namespace {

// samples[j] = nodes[idx[j]] (m coordinates); per-sample coefficient (if coef_nodes)
// alpha_s[j] = coef_nodes[param_of_j * n_nodes + idx[j]].
__global__ void gather_kernel(const float* __restrict__ nodes, const int* __restrict__ idx,
                              const int* __restrict__ param_of, int n, int m, int n_nodes,
                              const float* __restrict__ coef_nodes, float* __restrict__ samples,
                              float* __restrict__ alpha_s) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int i = idx[j];
  for (int k = 0; k < m; ++k) samples[(size_t)j * m + k] = nodes[(size_t)i * m + k];
  if (coef_nodes) alpha_s[j] = coef_nodes[(size_t)param_of[j] * n_nodes + i];
}

// Instance (c, mu) starts from q0[mu] with coefficient coef[mu].
__global__ void replicate_kernel(const double* __restrict__ q0, const float* __restrict__ coef, int n_params,
                                 int n_inst, int r, double* __restrict__ q, float* __restrict__ alpha) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_inst * r) return;
  const int inst = t / r, k = t % r, mu = inst % n_params;
  q[t] = q0[(size_t)mu * r + k];
  if (k == 0 && coef) alpha[inst] = coef[mu];
}

// res[c][i] = sum_mu |out[(c n_params + mu)][i] - fom[mu][i]| in FP64; NaN -> +inf.
__global__ void residual_kernel(const float* __restrict__ out, const float* __restrict__ fom, int n_params,
                                int n_nodes, double* __restrict__ res) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (i >= n_nodes) return;
  double s = 0.0;
  for (int mu = 0; mu < n_params; ++mu) {
    const double d = fabs((double)out[((size_t)c * n_params + mu) * n_nodes + i] - (double)fom[(size_t)mu * n_nodes + i]);
    s += isnan(d) ? INFINITY : d;
  }
  res[(size_t)c * n_nodes + i] = s;
}

// metric[c] = mean_i res[c][i] + max_i res[c][i]; +inf when a rollout of c failed.
// The sum is taken in a fixed order (per-thread strided partial sums, then a
// fixed-shape tree), so repeated calls give identical metrics.
__global__ void metric_kernel(const double* __restrict__ res, const int* __restrict__ status, int n_params,
                              int n_nodes, double* __restrict__ metric) {
  __shared__ double ssum[256], smax[256];
  __shared__ int sbad;
  const int c = blockIdx.x;
  if (threadIdx.x == 0) sbad = 0;
  __syncthreads();
  for (int mu = threadIdx.x; mu < n_params; mu += blockDim.x)
    if (status[(size_t)c * n_params + mu] != CROM_OK) atomicOr(&sbad, 1);
  double sum = 0.0, mx = 0.0;
  for (int i = threadIdx.x; i < n_nodes; i += blockDim.x) {
    const double v = res[(size_t)c * n_nodes + i];
    sum += v;
    mx = fmax(mx, v);
  }
  ssum[threadIdx.x] = sum;
  smax[threadIdx.x] = mx;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      ssum[threadIdx.x] += ssum[threadIdx.x + w];
      smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) metric[c] = sbad ? INFINITY : ssum[0] / n_nodes + smax[0];
}

// The k nodes with the largest res (ties: lower index), skipping nodes with
// taken[i] != 0; taken is updated.  One CTA of 1024 threads, k rounds of a block
// argmax.  Writes -1 when fewer than k nodes are free.
__global__ void topk_kernel(const double* __restrict__ res, int* __restrict__ taken, int n_nodes, int k,
                            int* __restrict__ out) {
  __shared__ double sv[32];
  __shared__ int si[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int round = 0; round < k; ++round) {
    double best = -1.0;
    int bi = -1;
    for (int i = threadIdx.x; i < n_nodes; i += blockDim.x) {
      if (taken[i]) continue;
      const double v = res[i];
      if (bi < 0 || v > best || (v == best && i < bi)) {
        best = v;
        bi = i;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (oi >= 0 && (bi < 0 || ov > best || (ov == best && oi < bi))) {
        best = ov;
        bi = oi;
      }
    }
    if (lane == 0) {
      sv[warp] = best;
      si[warp] = bi;
    }
    __syncthreads();
    if (warp == 0) {
      best = lane < (int)(blockDim.x >> 5) ? sv[lane] : -1.0;
      bi = lane < (int)(blockDim.x >> 5) ? si[lane] : -1;
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (oi >= 0 && (bi < 0 || ov > best || (ov == best && oi < bi))) {
          best = ov;
          bi = oi;
        }
      }
      if (lane == 0) {
        out[round] = bi;
        if (bi >= 0) taken[bi] = 1;
      }
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_sampling_gather(const float* nodes, const int* idx, const int* param_of, int n, int m,
                                   int n_nodes, const float* coef_nodes, float* samples, float* alpha_s,
                                   cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  gather_kernel<<<(n + 255) / 256, 256, 0, s>>>(nodes, idx, param_of, n, m, n_nodes, coef_nodes, samples, alpha_s);
  return cudaGetLastError();
}

cudaError_t launch_sampling_replicate(const double* q0, const float* coef, int n_params, int n_inst, int r,
                                      double* q, float* alpha, cudaStream_t s) {
  const int n = n_inst * r;
  replicate_kernel<<<(n + 255) / 256, 256, 0, s>>>(q0, coef, n_params, n_inst, r, q, alpha);
  return cudaGetLastError();
}

cudaError_t launch_sampling_metric(const float* out, const float* fom, const int* status, int n_cand, int n_params,
                                   int n_nodes, double* res, double* metric, cudaStream_t s) {
  residual_kernel<<<dim3((n_nodes + 255) / 256, n_cand), 256, 0, s>>>(out, fom, n_params, n_nodes, res);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  metric_kernel<<<n_cand, 256, 0, s>>>(res, status, n_params, n_nodes, metric);
  return cudaGetLastError();
}

cudaError_t launch_sampling_topk(const double* res, int* taken, int n_nodes, int k, int* out, cudaStream_t s) {
  topk_kernel<<<1, 1024, 0, s>>>(res, taken, n_nodes, k, out);
  return cudaGetLastError();
}

}  // namespace crom
