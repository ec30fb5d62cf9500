/*
 * crom.h — C ABI of the GB300 (sm_103a) implementation of CROM's online
 * latent-space time step (Continuous Reduced-Order Modeling, arXiv 2206.02607).
 *
 * The decoder g(x, q): R^{m+r} -> R is an MLP with `hidden` ELU layers of width
 * `width` and a linear output layer (paper App. D).  One latent step
 * q_n -> q_{n+1} (paper Algorithm 3) is:
 *   1. network inference at the integration samples y_j in M: g, dg/dx, the
 *      network Laplacian and dg/dq (paper §4.1, Algorithm 4, Algorithm 2);
 *   2. explicit PDE update Delta f_j at every sample (paper §4.2, Eqs.
 *      discrete-time / time-integration; App. G and H for the heat equation);
 *   3. network inversion by Gauss-Newton on
 *      min_q sum_j (g(y_j, q) - g(y_j, q_n) - Delta f_j)^2 from q^(0) = q_n
 *      (paper §4.3, Eq. invert; App. C), each iteration solving the r x r normal
 *      equations by an FP64 Cholesky factorisation.
 *
 * Conventions for every entry point:
 *   - Array arguments are DEVICE pointers owned by the caller (e.g. from
 *     torch.empty(...).data_ptr()), unless an argument says otherwise.  The
 *     context owns only its weight images and its scratch.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy default
 *     stream).  Nothing is synchronised unless stated.
 *   - The return value is a crom_status.  Host-side argument checks return
 *     CROM_ERR_INVALID_ARG before anything is launched; CUDA launch errors return
 *     CROM_ERR_CUDA.  crom_last_error() gives a message for the calling thread.
 *   - Per-instance numerical failures of crom_step are written to status[i]
 *     (the call itself still returns CROM_OK); q[i] then keeps its last good
 *     iterate.
 *   - There is no CPU fallback: without a usable sm_103a device every compute
 *     entry point returns CROM_ERR_CUDA.
 */
#ifndef CROM_H
#define CROM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct crom_ctx crom_ctx;
typedef void* crom_stream; /* cudaStream_t */

typedef enum {
  CROM_OK = 0,
  CROM_ERR_INVALID_ARG = 1, /* also: r > |M_i| (well-posedness r <= d|M|, paper §4.4) */
  CROM_ERR_CUDA = 2,
  CROM_ERR_SINGULAR = 3,    /* Cholesky pivot <= 1e-14 * max diag(J^T J) */
  CROM_ERR_NONFINITE = 4,   /* NaN/Inf in J^T J or J^T rho */
  CROM_ERR_TIMEOUT = 5,     /* a bounded device-side wait ran out */
  CROM_ERR_UNSUPPORTED = 6  /* shape or precision not built for this entry point */
} crom_status;

/* Arithmetic of the decoder evaluation.
 *  FP32   : CUDA-core FP32 forward-mode channels (paper Algorithm 2), FP64 normal
 *           equations.  Any shape with width % 32 == 0, width <= 256.
 *  F16X2  : tcgen05 tensor cores, f16 operands with FP32 accumulation.  Every
 *           activation operand is split into an f16 high part and an f16 low part
 *           (multiplied by the same MMAs into separate FP32 accumulator columns,
 *           added in the epilogue), so it carries ~2^-22 relative.  The step
 *           rounds the hidden weights once to f16 (2^-12 relative); the dense
 *           reconstruction also multiplies their f16 low parts W - f16(W) (held in
 *           tensor memory) into the accumulator, ~2^-22.  The step carries the
 *           derivative channels scaled by powers of two chosen from the weights
 *           (and per Gauss-Newton iteration for the difference channel), so that
 *           their f16 operands stay in range.  FP32 activation/derivative chains,
 *           FP64 normal equations.  width == 128, 2 <= hidden <= 5, m <= 2, r <= 15,
 *           ELU, every hidden weight, w_out and W_1q entry of magnitude <= 65000
 *           and every hidden bias of magnitude <= 45000.
 *           f16 rather than bf16 operands: both run at the same tensor rate, and
 *           bf16 weights (2^-9) move dense outputs by ~5e-3 and latent increments by
 *           several per cent against FP32 weights.
 *  F16    : as F16X2 with the high parts of the activations only (single f16
 *           operands, 2^-12 relative) and f16 weights (the dense reconstruction
 *           adds the hidden biases and w_out as f16 high and low parts, ~2^-22, on
 *           the tensor cores, and scales its activations by log2 e inside; the
 *           outputs are unscaled): dense error ~1e-3 against FP64 (F16X2 ~1e-6).
 *           Dense reconstruction and
 *           the step: the step's sample tiles hold twice the samples for the same
 *           UMMA widths (about 1.5x the F16X2 step's speed); its per-step errors
 *           are up to ~10x F16X2's on ill-conditioned decoders (kappa(J) ~ 1e5).
 *  BF16_MIXED : training step only: the decoder's dense products on the tcgen05
 *           tensor cores (the library's TMA-fed GEMM) with bf16 weights,
 *           activations and deltas and FP32 accumulation, the elementwise work
 *           fused into the GEMM epilogues; FP32 master weights, FP32 Adam, FP32
 *           encoder and input layer.  width in {64, 128, 256}, hidden >= 2,
 *           m + r <= 32.
 *  BF16X2, BF16: earlier names of F16X2 and F16 (the same values).  The value 3
 *           (a TF32 training mode of an earlier version) is no longer accepted. */
typedef enum {
  CROM_PREC_FP32 = 0,
  CROM_PREC_F16X2 = 1,
  CROM_PREC_F16 = 2,
  CROM_PREC_BF16_MIXED = 4,
  CROM_PREC_BF16X2 = 1,
  CROM_PREC_BF16 = 2
} crom_precision;

typedef enum { CROM_PDE_HEAT = 0, CROM_PDE_ADVDIFF = 1 } crom_pde;

/* Channels requested from crom_decode.  Output rows appear in this order:
 * VAL (1 row), DX (m rows, dg/dx_k), DXX (m rows, d2g/dx_k^2), LAP (1 row,
 * sum_k d2g/dx_k^2), DQ (r rows, dg/dq_j). */
enum {
  CROM_WANT_VAL = 1u,
  CROM_WANT_DX = 2u,
  CROM_WANT_DXX = 4u,
  CROM_WANT_LAP = 8u,
  CROM_WANT_DQ = 16u
};

/* Hidden-layer activation (paper App. D: ELU or SIREN, both continuously
 * differentiable).  ELU: s(z) = z (z > 0), e^z - 1 otherwise.  SIREN:
 * s(z) = sin(omega0 z) with omega0 = 30 by default (Sitzmann et al.). */
typedef enum { CROM_ACT_ELU = 0, CROM_ACT_SIREN = 1 } crom_activation;

/* Decoder shape: m spatial dims (1..3), r latent dims (1..32), width of the
 * hidden layers, hidden = number of hidden layers (1..8), their activation, and
 * omega0 for SIREN (0 selects 30; ignored for ELU).  Output dim d = 1; the
 * output layer is linear.  Derivatives are taken with respect to the decoder's
 * input coordinates x (for SIREN the paper feeds x scaled to [-1, 1]; the
 * caller states the PDE in the coordinates it feeds). */
typedef struct {
  int m;
  int r;
  int width;
  int hidden;
  int activation;
  float omega0;
} crom_decoder_desc;

/* Tangent-space velocity of the field (paper App. L, "Solid Mechanics": the second-order-in-time
 * elastodynamics ROM): v(x_p) = (dg/dq)(x_p, q_i) . qdot_i with
 * qdot_i = (q_i - q_prev_i) / dt (q_prev = q gives qdot = 0, the start of a
 * rollout).  Points as in crom_decode (instance i owns points
 * pt_off[i] .. pt_off[i+1]-1); q, q_prev [n_inst][r] FP64; out [n_pts] FP32.
 * One forward-mode directional channel in FP32 (the layer-1 seed W_1q qdot_i
 * formed in FP64 and rounded once), i.e. the Jacobian-vector product without the
 * r Jacobian columns.  The context keeps an n_inst x width scratch for the seeds
 * (grown on demand: do not call during stream capture with more instances than
 * before). */
int crom_tangent_velocity(crom_ctx* ctx, int n_inst, const double* q, const double* q_prev, double dt,
                          const int* pt_off, const float* x, int n_pts, float* out, crom_stream stream);

/* One latent step.
 *  pde      : CROM_PDE_HEAT     Delta f_j = dt * alpha * Lap g(y_j, q_n)
 *             CROM_PDE_ADVDIFF  Delta f_j = dt * (-vel_j . grad g + alpha * Lap g)
 *             (alpha plays the role of nu for advection-diffusion)
 *  gn_iters : Gauss-Newton iterations per step, 1..16 (1 = the linearised least
 *             squares of paper App. C.2)
 *  dt       : time step (finite, > 0)
 *  coef_per_sample : 0 — alpha holds one coefficient per instance, alpha[i];
 *             1 — alpha holds one per integration sample, alpha[j] = nu(y_j), for
 *             spatially varying coefficients u_t = nu(x) Lap u (paper App. G, the 1D
 *             thermodynamics example, and App. H, the image-diffusion example, with
 *             nu piecewise constant over regions); the caller evaluates nu at the
 *             fixed sample set once.
 *  line_search : 0 — full Gauss-Newton steps; L in 1..16 — each iteration takes
 *             the first step length a = 1, 1/2, ..., 2^-L along the GN direction
 *             delta that satisfies the sufficient-decrease (Armijo) condition
 *             phi(q + a delta) <= phi(q) + 1e-4 a (J^T rho).delta, phi = 1/2 sum_j rho_j^2
 *             (the paper's backtracking line search, §4.3); if none does, q is
 *             kept and the instance's remaining iterations are skipped.  Each
 *             trial costs one value-only pass over the instance's samples.
 *             Available with CROM_PREC_F16X2 and CROM_PREC_F16 (the FP32
 *             path returns CROM_ERR_UNSUPPORTED). */
typedef struct {
  int pde;
  int gn_iters;
  double dt;
  int coef_per_sample;
  int line_search;
} crom_step_desc;

/* Library version (major*10000 + minor*100 + patch). */
int crom_version(void);

/* Message describing the last failed call on this thread ("" if none). */
const char* crom_last_error(void);

/* Create a context for one decoder shape on CUDA device `device` (made current
 * for the duration of the call).  *out receives the context; release it with
 * crom_destroy.  Returns CROM_ERR_CUDA if no sm_103a-capable device is usable. */
int crom_create(crom_ctx** out, const crom_decoder_desc* desc, int device);

/* Free every device buffer the context owns.  Synchronises the device. */
int crom_destroy(crom_ctx* ctx);

/* Load decoder weights.  `params` is a packed FP32 image of n floats: for each
 * layer l = 1..hidden+1, W_l row-major [out][in] then b_l [out]; layer 1 takes
 * (x_1..x_m, q_1..q_r).  n must equal the parameter count.  params_on_device
 * selects whether `params` is a device (1) or host (0) pointer.  The call builds
 * the FP32 copies and the f16 tensor-core images and synchronises `stream`. */
int crom_set_weights(crom_ctx* ctx, const float* params, size_t n, int params_on_device,
                     crom_stream stream);

/* Step 1 alone (paper §4.1, Algorithm 4; Algorithm 2 for the derivatives), FP32.
 * n_inst latent codes q [n_inst][r] (FP64); point set of instance i is
 * x[pt_off[i] .. pt_off[i+1]) with x [n_pts][m] FP32 and pt_off [n_inst+1]
 * int32 (pt_off[0] = 0, pt_off[n_inst] = n_pts, non-decreasing).  `want` is a
 * mask of CROM_WANT_*; out is channel-major [C][n_pts] FP32 with C rows in the
 * order given above.  n_pts may be 0. */
int crom_decode(crom_ctx* ctx, int n_inst, const double* q, const int* pt_off, const float* x,
                int n_pts, unsigned want, float* out, crom_stream stream);

/* Step 1 alone on the tcgen05 tensor cores (paper §4.1, Algorithm 4: the batched
 * network inference of the latent step, as the tensor-core step computes it):
 * the same arguments, point layout and channel-major output as crom_decode, with
 * precision CROM_PREC_F16X2 or CROM_PREC_F16 and want ⊆ VAL | DX | LAP | DQ
 * (CROM_WANT_DXX returns CROM_ERR_UNSUPPORTED: the tensor-core path carries the
 * m second-derivative channels summed into one Laplacian channel).  DQ comes from
 * one reverse-mode pass.  The points are processed in chunks of 256 spread over
 * the GPU whatever the instances' sizes; pt_off must be non-decreasing from 0 to
 * n_pts (points outside [pt_off[0], pt_off[n_inst]) are not written).  Same shape
 * limits as the F16X2 step; precision as the step's (f16 weights; F16X2 hi/lo
 * activations, F16 single).  Asynchronous on `stream`; a device-side wait that ran
 * out is reported by crom_device_flags. */
int crom_decode_tc(crom_ctx* ctx, int precision, int n_inst, const double* q, const int* pt_off, const float* x,
                   int n_pts, unsigned want, float* out, crom_stream stream);

/* Device-side failure flags of the context's tensor-core kernels: synchronises
 * `stream` and sets *flags to bit 0 = the last tensor-core step or decode launch
 * gave up on a bounded wait (its unfinished instances carry CROM_ERR_TIMEOUT),
 * bit 1 = a tensor-core reconstruction gave up since the last call (its output is
 * incomplete); bit 1 is cleared by the call.  0 after every normal run. */
int crom_device_flags(crom_ctx* ctx, int* flags, crom_stream stream);

/* One latent step for n_inst independent instances sharing the decoder
 * (paper Algorithm 3).  Instance i has latent state q[i] (FP64 [n_inst][r],
 * updated in place), coefficient alpha[i] (FP32), and integration samples
 * samples[s_off[i] .. s_off[i+1]) (FP32 [n_samples][m]; s_off int32
 * [n_inst+1], s_off[0] = 0, s_off[n_inst] = n_samples).  vel (FP32
 * [n_samples][m]) is the advection velocity at each sample, required for
 * CROM_PDE_ADVDIFF and ignored (may be NULL) otherwise.  max_samples must bound
 * every |M_i|; an instance with |M_i| > max_samples or |M_i| < r gets
 * status CROM_ERR_INVALID_ARG and is left unchanged.  status [n_inst] int32
 * receives CROM_OK / CROM_ERR_SINGULAR / CROM_ERR_NONFINITE /
 * CROM_ERR_INVALID_ARG per instance.
 * precision CROM_PREC_FP32: each GN iteration is one launch spreading an
 *   instance over several CTAs (the last CTA to finish reduces and solves); the
 *   context grows its scratch on first use, so the first call for a given size
 *   must not be made during stream capture.
 * precision CROM_PREC_F16X2 or CROM_PREC_F16: one persistent launch per step
 *   (plus a small ordering kernel); each of a CTA's four 128-thread groups takes
 *   whole instances, largest |M_i| first, from a queue. */
int crom_step(crom_ctx* ctx, const crom_step_desc* step, int precision, int n_inst, double* q,
              const float* alpha, const float* vel, const int* s_off, const float* samples,
              int n_samples, int max_samples, int* status, crom_stream stream);

/* A rollout: n_steps consecutive crom_step calls (same arguments, q advanced in
 * place) recorded once into a CUDA graph and replayed with one launch.  The graph
 * is built on the first call for a given argument set (pointers, sizes, step
 * description, precision, n_steps) and cached in the context; a call with the
 * same arguments relaunches the cached graph, a call with different arguments
 * rebuilds it.  status receives the per-instance status of the last step.  The
 * first call for an argument set allocates and records: do not make it during
 * stream capture. */
int crom_rollout(crom_ctx* ctx, const crom_step_desc* step, int precision, int n_steps, int n_inst, double* q,
                 const float* alpha, const float* vel, const int* s_off, const float* samples, int n_samples,
                 int max_samples, int* status, crom_stream stream);

/* Sample-tile shape of the tensor-core step (CROM_PREC_F16X2): s0 samples per
 * forward tile in the first Gauss-Newton iteration (4 channels: 8, fixed by the
 * 32 hi-part operand columns of a tile; two such tiles share one reverse pass),
 * s1 in later ones (2 channels: 16 or 8).  CROM_PREC_F16 (hi parts only) runs
 * tiles of twice these sizes under the same setting.  Larger tiles issue half as many UMMA
 * stages; smaller ones waste less on the ragged last tile of each instance.
 * crom_set_step_tiles fixes the shape (default (8, 16)); crom_get_step_tiles reads
 * it and, into ms[2] (may be NULL), the per-step times that the last crom_autotune
 * measured for s1 = 16 and 8 (-1 when not measured). */
int crom_set_step_tiles(crom_ctx* ctx, int s0, int s1);
int crom_get_step_tiles(const crom_ctx* ctx, int* s0, int* s1, float* ms);

/* Autotuner of the tile shape: times the F16X2 step on the given batch (same
 * arguments as crom_step; q is read, not updated: the trials run on a copy; status
 * is overwritten) for every tile shape, five steps each after one warm-up, and
 * keeps the fastest in the context.  Blocks until the timing completes; allocates
 * a copy of q (not during stream capture).  The rollout graph cache is keyed on the
 * tile shape, so a re-tuned context records a new graph. */
int crom_autotune(crom_ctx* ctx, const crom_step_desc* step, int n_inst, const double* q, const float* alpha,
                  const float* vel, const int* s_off, const float* samples, int n_samples, int max_samples,
                  int* status, crom_stream stream);

/* crom_step on host arrays (the same step, paper §4, Algorithm 3): q, alpha, vel,
 * s_off, samples and status are host pointers with the layouts of crom_step.  The
 * call checks s_off on the host (starts at 0, never decreases, ends at n_samples),
 * copies the inputs into a device staging buffer owned by the context (allocated
 * or grown on first use, freed by crom_destroy), runs crom_step on `stream`,
 * copies q and status back and waits for the stream before returning, so q and
 * status are valid when it returns.  Pinned host memory (cudaHostAlloc,
 * torch.Tensor.pin_memory) makes the copies asynchronous DMA; pageable memory
 * works too.  The staging buffer is shared by the context's calls: calls on one
 * context must not run concurrently from several host threads.  The call synchronises the stream: it cannot be recorded into a CUDA
 * graph.  Status codes as crom_step. */
int crom_step_host(crom_ctx* ctx, const crom_step_desc* step, int precision, int n_inst, double* q,
                   const float* alpha, const float* vel, const int* s_off, const float* samples, int n_samples,
                   int max_samples, int* status, crom_stream stream);

/* crom_step with precision CROM_PREC_FP32, for callers that cannot allocate
 * device memory when they step: host applications or frameworks that own the
 * device's memory through their own pool and forbid direct cudaMalloc/cudaFree by
 * the libraries they load, and latency-critical loops that must not risk an
 * allocation that synchronises the device.  The paper has no
 * counterpart; this is an operational variant of the same step.
 * Arguments, results and status codes are those of crom_step.  The scratch lives
 * in one fixed 8 MiB device array per GPU, held from library load until process
 * exit; a batch that needs more (about n_inst * ceil(max_samples / S) *
 * (r(r+1)/2 + r) * 8 bytes of partial sums, S <= 4 samples per CTA, plus
 * 8 * (n_samples + n_inst * r) bytes) is rejected with CROM_ERR_INVALID_ARG and
 * nothing is launched.  The call allocates and frees nothing.  Its first call on
 * a device looks up the array's device address (cudaGetSymbolAddress); make that
 * first call before any stream capture.  Every call shares the array and finds
 * the previous call's contents in it: the call clears the parts that must start
 * at zero, but two calls whose work may overlap on the GPU (different streams
 * without ordering) race on the array and must not be issued. */
int crom_step_noalloc(crom_ctx* ctx, const crom_step_desc* step, int n_inst, double* q,
                      const float* alpha, const float* vel, const int* s_off, const float* samples,
                      int n_samples, int max_samples, int* status, crom_stream stream);

/* Full-order model: n_steps explicit finite-difference steps with forward Euler
 * (paper App. G.2 and H.2) for n_batch independent FP32 fields, in place on the
 * current CUDA device.  Fields u [n_batch][nx][ny] row-major (ny fastest);
 * tmp is caller-owned scratch of the same size (distinct from u); coef
 * [n_batch] is nu (heat 1D), alpha (heat 2D) or nu (advection-diffusion).
 *  CROM_FOM_HEAT1D_DIRICHLET   ny == 1, nodes x_i = i/(nx-1), boundary nodes 0.
 *  CROM_FOM_HEAT2D_NEUMANN     ny == nx, nodes (i, j)/(nx-1), zero-flux boundary
 *                              by mirror ghost nodes (u_{-1} = u_1).
 *  CROM_FOM_ADVDIFF2D_PERIODIC ny == nx, periodic cells of width 1/nx,
 *                              conservative first-order upwind advection with face
 *                              velocities ax (between cells (i,j),(i+1,j)) and ay
 *                              (between (i,j),(i,j+1)), [n_batch][nx][ny] each,
 *                              plus central diffusion.
 *  CROM_FOM_HEAT1D_DIRICHLET_FIELD, CROM_FOM_HEAT2D_NEUMANN_FIELD
 *                              the two heat models with a spatially varying
 *                              coefficient, u_t = nu(x) Lap u (paper App. G,
 *                              thermodynamics, and App. H, image diffusion): coef
 *                              holds nu at every node, [n_batch][nx][ny].
 *  CROM_FOM_ADVDIFF2D_PERIODIC_CENTRAL
 *                              as CROM_FOM_ADVDIFF2D_PERIODIC with the face value
 *                              the mean of the two cells (second order, no
 *                              numerical diffusion; forward Euler is then stable
 *                              for (a dt / h)^2 <= 2 nu dt / h^2 and
 *                              nu dt / h^2 <= 1/4).
 * nx >= 3, n_batch <= 65535.  The result is in u when the call's work completes. */
typedef enum {
  CROM_FOM_HEAT1D_DIRICHLET = 0,
  CROM_FOM_HEAT2D_NEUMANN = 1,
  CROM_FOM_ADVDIFF2D_PERIODIC = 2,
  CROM_FOM_HEAT1D_DIRICHLET_FIELD = 3,
  CROM_FOM_HEAT2D_NEUMANN_FIELD = 4,
  CROM_FOM_ADVDIFF2D_PERIODIC_CENTRAL = 5
} crom_fom_kind;

int crom_fom_step(int kind, int n_batch, int nx, int ny, const float* coef, const float* ax, const float* ay,
                  double dt, int n_steps, float* u, float* tmp, crom_stream stream);

/* ---- Manifold construction: one training step (paper §3, Eq. loss; App. D) ----
 * Encoder e(f): 1D convolutions (kernel 6, stride 4, one channel, no padding,
 * ELU after each) on the flattened snapshot of P nodes, repeated while the output
 * stays >= 32 long; a dense layer to 32 (ELU); a linear layer to r.  Decoder:
 * g(x, q) of the given crom_decoder_desc.  Loss: mean over B snapshots x S
 * sampled nodes of (g(x_j, e(f_b)) - f_b(x_j))^2.  Adam (beta1 0.9, beta2 0.999,
 * eps 1e-8) on FP32 master parameters; the decoder pass in FP32 on CUDA cores or
 * in bf16 on the tensor cores (crom_trainer_set_precision).
 * Parameter vector (FP32): the decoder exactly as crom_set_weights packs it, then
 * per convolution w[6], b, then the dense layers W[32][L_last], b[32], W[r][32],
 * b[r].  The trainer owns all its device memory. */
typedef struct crom_trainer crom_trainer;

/* P snapshot nodes, B snapshots and S sampled nodes per step (fixed per trainer).
 * Parameters start at zero: load them with crom_trainer_set_params. */
int crom_trainer_create(crom_trainer** out, const crom_decoder_desc* dec, int P, int B, int S, int device);
int crom_trainer_destroy(crom_trainer* tr);
/* Number of floats in the parameter vector. */
int crom_trainer_param_count(const crom_trainer* tr, size_t* n);
/* Copy the parameter vector in (set) or out (get); on_device selects device (1)
 * or host (0) memory for `params`.  set also resets the Adam moments and step. */
int crom_trainer_set_params(crom_trainer* tr, const float* params, size_t n, int on_device, crom_stream stream);
int crom_trainer_get_params(crom_trainer* tr, float* params, size_t n, int on_device, crom_stream stream);
/* Gradient of the last crom_train_step (same layout as the parameters). */
int crom_trainer_get_grads(crom_trainer* tr, float* grads, size_t n, int on_device, crom_stream stream);
/* One step: snaps [B][P] FP32, pt_idx [B][S] int32 node indices in [0, P),
 * coords [P][m] FP32 node coordinates, learning rate lr; loss_out (device, one
 * double, may be NULL) receives the loss before the update. */
int crom_train_step(crom_trainer* tr, const float* snaps, const int* pt_idx, const float* coords, float lr,
                    double* loss_out, crom_stream stream);
/* Arithmetic of the trainer's decoder pass: CROM_PREC_FP32 (default; the
 * library's FP32 CUDA-core GEMM, split-K weight gradients reduced in a fixed
 * order) or CROM_PREC_BF16_MIXED (the library's tcgen05 GEMMs with fused
 * epilogues, bf16 operands and activations, FP32 accumulation and master
 * weights; see crom_precision).  Selecting BF16_MIXED the first time allocates its
 * buffers (about (hidden + 2) * B * S * width * 2 bytes): not during stream
 * capture.  Returns CROM_ERR_UNSUPPORTED for other values or shapes. */
int crom_trainer_set_precision(crom_trainer* tr, int precision);
/* Encoder only: q [n][r] FP32 for n <= B snapshots [n][P] (initial latent codes). */
int crom_encode(crom_trainer* tr, int n, const float* snaps, float* q, crom_stream stream);

/* Checkpoint / resume of a trainer (the paper trains in stages; this lets a run stop
 * and continue).  crom_trainer_save writes, after synchronising the device, a
 * binary file: a 64-byte header (magic "CROMCKPT", version 1, m, r, width, hidden,
 * activation, P, the parameter count, the Adam step count, the CRC-32 of the
 * payload) and the payload: FP32 parameters, first and second Adam moments, host
 * byte order.  crom_trainer_load checks magic, version, shapes (the decoder's and
 * P; B and S may differ) and the checksum (CROM_ERR_INVALID_ARG on any mismatch,
 * the trainer then unchanged) and restores parameters, moments and step count, so
 * that the following steps are bit-identical to an uninterrupted run. */
int crom_trainer_save(crom_trainer* tr, const char* path);
int crom_trainer_load(crom_trainer* tr, const char* path);

/* CRC-32 (IEEE 802.3, reflected polynomial 0xEDB88320) of n bytes: the checksum
 * of the checkpoint files. */
unsigned crom_crc32(const void* data, size_t n);

/* Host-side watchdog: polls the stream until its work has finished (CROM_OK) or
 * timeout_ms have passed (CROM_ERR_TIMEOUT; the work keeps running and the call
 * may be repeated); a CUDA error on the stream gives CROM_ERR_CUDA.  Never blocks
 * in the driver. */
int crom_stream_wait(crom_stream stream, double timeout_ms);

/* Dense reconstruction g(x_p, q_c) for n_codes latent codes q [n_codes][r]
 * (FP64) at n_pts points x [n_pts][m] (FP32); out [n_codes][n_pts] FP32.
 * precision FP32 (any shape), F16X2 or F16 (tensor cores; width 128). */
int crom_reconstruct(crom_ctx* ctx, int precision, int n_codes, const double* q, int n_pts,
                     const float* x, float* out, crom_stream stream);

/* Robust integration-sample selection (paper App. B, Algorithm 1): greedy
 * growth of the sample set M from n_init starting nodes.  Each round computes,
 * for the current M, res[i] = sum over training parameters mu of
 * |g(x_i, q_T(mu)) - f_FOM(x_i, T; mu)| at every FOM node, where q_T(mu) is the
 * latent state after n_steps steps (`step`, `precision`) from q0[mu] with
 * samples M; Metric = mean(res) + max(res).  While Metric >= target and
 * |M| < max_samples, the n_try nodes with the largest res (not in M; ties to the
 * lower index) are tried, each as M + {x_i}, and the one with the smallest Metric
 * (ties to the earlier) is added.  A set whose rollout reports a non-OK step
 * status has Metric = +inf.  All candidate sets x parameters of a round run as one
 * batched rollout (one instance each), then one dense reconstruction.
 *  q0        [n_params][r] FP64, device
 *  coef      [n_params] FP32 (coef_per_sample = 0) or [n_params][n_nodes]
 *            (coef_per_sample = 1: nu at every node), device
 *  nodes     [n_nodes][m] FP32 node coordinates, device
 *  fom_final [n_params][n_nodes] FP32 FOM fields at the final step, device
 *  init_idx  [n_init] distinct node indices, host
 *  idx_out   [max_samples] host: the selected node indices in order of addition
 *            (the initial ones first); count_out, metric_out host scalars.
 * step->pde must be CROM_PDE_HEAT; precision FP32 (no line search) or F16X2.
 * Limits: 1 <= n_try <= 64, n_init <= max_samples <= min(n_nodes, 4096),
 * n_try * n_params <= 65535.  The call allocates its work buffers and returns
 * after the work on `stream` completed (not usable during stream capture). */
int crom_robust_samples(crom_ctx* ctx, const crom_step_desc* step, int precision, int n_params, const double* q0,
                        const float* coef, int n_steps, int n_nodes, const float* nodes, const float* fom_final,
                        int n_init, const int* init_idx, int n_try, double target, int max_samples, int* idx_out,
                        int* count_out, double* metric_out, crom_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* CROM_H */
