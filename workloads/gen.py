"""Seeded input generators for the CROM latent-space step workloads.

Everything here is input preparation: random draws (numpy PCG64 via
``np.random.default_rng``, identical on x86-64 and aarch64), uniform grids,
sample-set selection and array packing.  Nothing here evaluates the decoder,
a PDE update or the Gauss-Newton projection; both the FP64 oracle and the CUDA
library consume the exact same arrays produced here.

Workload recipes (paper: §5 and App. G/H for the PDEs, App. D for the network):

* ``heat1d_small``   1D heat u_t = u_xx on [0,1], Dirichlet 0, P=256 nodes,
  u0 = sum_{k=1..4} a_k sin(k pi x), a_k ~ U(-1,1); decoder R^{1+3} -> R,
  4 ELU layers of width 64, Xavier-normal (seed 0); |M| = 16 distinct interior
  nodes; dt = 1e-5; 100 steps; 1 Gauss-Newton iteration.
* ``heat2d_single``  2D heat u_t = alpha Lap u on a 128x128 grid, zero Neumann,
  alpha = 1; u0 = 8 Gaussian bumps; decoder R^{2+8} -> R, 5 ELU layers of
  width 128; |M| = 200 interior nodes; dt = 1e-5; 1000 steps; 2 GN iterations.
* ``recon_dense``    the same 2D decoder; dense reconstruction at 1024^2 points x
  64 codes q ~ N(0,1); plus a 2048-sample step.
* ``heat2d_batched`` 1024 instances of the 2D heat problem, alpha ~ U(0.5, 2),
  |M_i| ~ U{32..512}, per-instance seeds 1000+i.
* ``advdiff_learned`` the learned-model workload: periodic 2D advection-diffusion
  on 256^2 cells, one velocity field from a random Fourier stream function
  (max |face velocity| = 1), one initial field of 8 periodic Gaussian bumps, 64
  trajectories with nu ~ U(1e-3, 1e-2), dt = 2.5e-4, 2000 steps, a snapshot every
  10 (56 trajectories for training, 8 held out).

Weights are FP32 values (Xavier-normal draws rounded to float32 once), the form a
trained decoder has; both sides read the same packed float32 image.

Initial latent codes: an untrained, randomly initialised decoder cannot represent
the Gaussian-bump initial fields, so q0 ~ N(0,1) is drawn per instance (the bumps
are still generated for the full-order solver).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "DecoderSpec", "xavier_decoder", "siren_decoder", "pack_params", "param_count",
    "interior_nodes_1d", "interior_nodes_2d", "gaussian_bumps_2d", "sine_modes_1d",
    "StepWorkload", "heat1d_small", "heat2d_single", "heat2d_batched", "recon_dense",
    "grid_points_2d", "ragged_offsets", "piecewise_nu",
    "cell_centers_2d", "periodic_bumps_2d", "stream_function_faces", "cell_velocity", "AdvDiffWorkload",
    "advdiff_learned",
]


@dataclass(frozen=True)
class DecoderSpec:
    """Shape of the implicit-neural-representation decoder g: R^{m+r} -> R.

    m: spatial dimension, r: latent dimension, width: hidden width (beta*d in
    App. D), hidden: number of ELU hidden layers (the output layer is linear).
    """
    m: int
    r: int
    width: int
    hidden: int

    @property
    def dims(self):
        return [self.m + self.r] + [self.width] * self.hidden + [1]


def xavier_decoder(spec: DecoderSpec, seed: int, bias_std: float = 0.0):
    """Xavier-normal weights (std = sqrt(2/(fan_in+fan_out))), zero biases (App. D.1).

    Returns a list of (W [out][in], b [out]) float64 pairs, layer 1 first.  Layer 1
    takes the input vector ordered (x_1..x_m, q_1..q_r).  ``bias_std`` > 0 draws
    N(0, bias_std^2) biases instead of zeros (used by tests to exercise bias paths).
    """
    rng = np.random.default_rng(seed)
    dims = spec.dims
    params = []
    for l in range(len(dims) - 1):
        fan_in, fan_out = dims[l], dims[l + 1]
        std = np.sqrt(2.0 / (fan_in + fan_out))
        W = rng.standard_normal((fan_out, fan_in)) * std
        b = rng.standard_normal(fan_out) * bias_std if bias_std > 0 else np.zeros(fan_out)
        W, b = W.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64)
        params.append((W, b))
    return params


def siren_decoder(spec: DecoderSpec, seed: int, omega0: float = 30.0):
    """SIREN initialisation (Sitzmann et al., the paper's "default initialization
    (omega0 = 30)"): layer 1 W ~ U(-1/fan_in, 1/fan_in); later layers
    W ~ U(-sqrt(6/fan_in)/omega0, +sqrt(6/fan_in)/omega0); biases
    U(-1/sqrt(fan_in), 1/sqrt(fan_in)).  Same layout as xavier_decoder."""
    rng = np.random.default_rng(seed)
    dims = spec.dims
    params = []
    for l in range(len(dims) - 1):
        fan_in, fan_out = dims[l], dims[l + 1]
        lim = 1.0 / fan_in if l == 0 else np.sqrt(6.0 / fan_in) / omega0
        W = rng.uniform(-lim, lim, size=(fan_out, fan_in))
        b = rng.uniform(-1.0 / np.sqrt(fan_in), 1.0 / np.sqrt(fan_in), size=fan_out)
        W, b = W.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64)
        params.append((W, b))
    return params


def param_count(spec: DecoderSpec) -> int:
    d = spec.dims
    return sum(d[l + 1] * d[l] + d[l + 1] for l in range(len(d) - 1))


def pack_params(params) -> np.ndarray:
    """Packed float32 image: for each layer, W row-major [out][in], then b [out]."""
    parts = []
    for W, b in params:
        parts.append(np.asarray(W, dtype=np.float32).ravel())
        parts.append(np.asarray(b, dtype=np.float32).ravel())
    return np.ascontiguousarray(np.concatenate(parts))


def interior_nodes_1d(P: int, count: int, rng) -> np.ndarray:
    """Distinct interior nodes i/(P-1), i in 1..P-2, drawn without replacement."""
    idx = rng.choice(np.arange(1, P - 1), size=count, replace=False)
    return (idx / (P - 1)).astype(np.float32).reshape(-1, 1)


def interior_nodes_2d(n: int, count: int, rng) -> np.ndarray:
    """Distinct interior nodes (i/(n-1), j/(n-1)), 1 <= i, j <= n-2, without replacement."""
    inner = n - 2
    flat = rng.choice(inner * inner, size=count, replace=False)
    i = flat // inner + 1
    j = flat % inner + 1
    return np.stack([i / (n - 1), j / (n - 1)], axis=1).astype(np.float32)


def grid_points_2d(n: int) -> np.ndarray:
    """All n*n nodes of the uniform grid on [0,1]^2, row-major (x1 slow, x2 fast)."""
    t = np.arange(n) / (n - 1)
    X1, X2 = np.meshgrid(t, t, indexing="ij")
    return np.stack([X1.ravel(), X2.ravel()], axis=1).astype(np.float32)


def sine_modes_1d(P: int, rng, modes: int = 4):
    """u0(x) = sum_k a_k sin(k pi x) on x_i = i/(P-1), a_k ~ U(-1,1)."""
    a = rng.uniform(-1.0, 1.0, size=modes)
    x = np.arange(P) / (P - 1)
    u0 = sum(a[k] * np.sin((k + 1) * np.pi * x) for k in range(modes))
    return a, u0


def gaussian_bumps_2d(n: int, rng, count: int = 8, sigma=(0.03, 0.1)):
    """Sum of Gaussian bumps on the n x n grid: centres U[0,1]^2, sigma ~ U(sigma),
    amplitude ~ U(0.5, 1)."""
    c = rng.uniform(0.0, 1.0, size=(count, 2))
    s = rng.uniform(sigma[0], sigma[1], size=count)
    a = rng.uniform(0.5, 1.0, size=count)
    t = np.arange(n) / (n - 1)
    X1, X2 = np.meshgrid(t, t, indexing="ij")
    u = np.zeros((n, n))
    for k in range(count):
        u += a[k] * np.exp(-((X1 - c[k, 0]) ** 2 + (X2 - c[k, 1]) ** 2) / (2 * s[k] ** 2))
    return u


def piecewise_nu(x, values) -> np.ndarray:
    """nu at points x [N][m] for a coefficient that is piecewise constant over
    len(values) equal-width regions of [0, 1] along x_1 (region k holds
    k/R <= x_1 < (k+1)/R, the last one closed).  Returns float32 [N]."""
    values = np.asarray(values, np.float32)
    R = values.shape[0]
    k = np.clip(np.floor(np.asarray(x, np.float64)[:, 0] * R).astype(np.int64), 0, R - 1)
    return values[k]


def ragged_offsets(sizes) -> np.ndarray:
    off = np.zeros(len(sizes) + 1, dtype=np.int32)
    off[1:] = np.cumsum(sizes)
    return off


@dataclass
class StepWorkload:
    """Inputs of one batched latent step (all instances share one decoder)."""
    name: str
    spec: DecoderSpec
    params: list
    q0: np.ndarray          # [n_inst][r] float64
    alpha: np.ndarray       # [n_inst] float32 (diffusivity per instance)
    s_off: np.ndarray       # [n_inst+1] int32
    samples: np.ndarray     # [S_total][m] float32
    dt: float
    gn_iters: int
    steps: int
    extra: dict = field(default_factory=dict)

    @property
    def n_inst(self) -> int:
        return int(self.q0.shape[0])

    @property
    def sizes(self) -> np.ndarray:
        return np.diff(self.s_off)


def heat1d_small(bias_std: float = 0.0) -> StepWorkload:
    spec = DecoderSpec(m=1, r=3, width=64, hidden=4)
    params = xavier_decoder(spec, seed=0, bias_std=bias_std)
    a, u0 = sine_modes_1d(256, np.random.default_rng(1))
    samples = interior_nodes_1d(256, 16, np.random.default_rng(2))
    q0 = np.random.default_rng(5).standard_normal((1, spec.r))
    return StepWorkload("heat1d_P256_M16_r3_w64", spec, params, q0,
                        np.ones(1, np.float32), ragged_offsets([16]), samples,
                        dt=1e-5, gn_iters=1, steps=100, extra={"a": a, "u0": u0, "P": 256})


def heat2d_single(bias_std: float = 0.0) -> StepWorkload:
    spec = DecoderSpec(m=2, r=8, width=128, hidden=5)
    params = xavier_decoder(spec, seed=0, bias_std=bias_std)
    u0 = gaussian_bumps_2d(128, np.random.default_rng(3))
    samples = interior_nodes_2d(128, 200, np.random.default_rng(6))
    q0 = np.random.default_rng(5).standard_normal((1, spec.r))
    return StepWorkload("heat2d_128sq_M200_r8_w128", spec, params, q0,
                        np.ones(1, np.float32), ragged_offsets([200]), samples,
                        dt=1e-5, gn_iters=2, steps=1000, extra={"u0": u0, "n": 128})


def heat2d_batched(n_inst: int = 1024, m_lo: int = 32, m_hi: int = 512,
                   bias_std: float = 0.0,
                   with_bumps: bool = False, first: int = 0) -> StepWorkload:
    """Instances first .. first+n_inst-1 of the batched 2D heat workload (instance i
    draws from seed 1000+i, so disjoint ranges give disjoint instances)."""
    spec = DecoderSpec(m=2, r=8, width=128, hidden=5)
    params = xavier_decoder(spec, seed=0, bias_std=bias_std)
    sizes, alphas, qs, samp, bumps = [], [], [], [], []
    for i in range(first, first + n_inst):
        rng = np.random.default_rng(1000 + i)
        alphas.append(rng.uniform(0.5, 2.0))
        M = int(rng.integers(m_lo, m_hi + 1))
        sizes.append(M)
        samp.append(interior_nodes_2d(128, M, rng))
        qs.append(rng.standard_normal(spec.r))
        if with_bumps:
            bumps.append(gaussian_bumps_2d(128, rng))
    return StepWorkload(f"heat2d_batched_{n_inst}x_M{m_lo}-{m_hi}_r8_w128", spec, params,
                        np.array(qs), np.array(alphas, dtype=np.float32),
                        ragged_offsets(sizes), np.concatenate(samp, axis=0),
                        dt=1e-5, gn_iters=2, steps=1000,
                        extra={"u0": bumps} if with_bumps else {})


def recon_dense(n_side: int = 1024, n_codes: int = 64):
    """Dense reconstruction workload: grid points, latent codes and the 2D decoder."""
    spec = DecoderSpec(m=2, r=8, width=128, hidden=5)
    params = xavier_decoder(spec, seed=0)
    codes = np.random.default_rng(4).standard_normal((n_codes, spec.r))
    return spec, params, codes, grid_points_2d(n_side)


def cell_centers_2d(n: int) -> np.ndarray:
    """Centres ((i + 1/2)/n, (j + 1/2)/n) of the n x n periodic cells of [0,1)^2,
    row-major (i slow, j fast), float32 [n*n][2]."""
    t = (np.arange(n) + 0.5) / n
    X1, X2 = np.meshgrid(t, t, indexing="ij")
    return np.stack([X1.ravel(), X2.ravel()], axis=1).astype(np.float32)


def periodic_bumps_2d(n: int, rng, count: int = 8, sigma=(0.03, 0.1)):
    """Sum of Gaussian bumps on the periodic unit square at the cell centres: centres
    U[0,1)^2, sigma ~ U(sigma), amplitude ~ U(0.5, 1), distances to the nearest
    periodic image of each centre."""
    c = rng.uniform(0.0, 1.0, size=(count, 2))
    s = rng.uniform(sigma[0], sigma[1], size=count)
    a = rng.uniform(0.5, 1.0, size=count)
    t = (np.arange(n) + 0.5) / n
    X1, X2 = np.meshgrid(t, t, indexing="ij")
    u = np.zeros((n, n))
    for k in range(count):
        d1 = (X1 - c[k, 0] + 0.5) % 1.0 - 0.5
        d2 = (X2 - c[k, 1] + 0.5) % 1.0 - 0.5
        u += a[k] * np.exp(-(d1 ** 2 + d2 ** 2) / (2 * s[k] ** 2))
    return u


def stream_function_faces(n: int, rng, modes: int = 4):
    """Face velocities of a random periodic stream function
    psi(x, y) = sum_{k,l=1..modes} c_kl sin(2 pi (k x + l y) + phi_kl) / (k^2 + l^2),
    c_kl ~ N(0,1), phi_kl ~ U(0, 2 pi), sampled at the cell corners
    C[i][j] = psi((i+1)/n, (j+1)/n).  The face between cells (i,j) and (i+1,j) gets
    ax[i][j] = n (C[i][j] - C[i][j-1]) (the mean of u = dpsi/dy over it), the face
    between (i,j) and (i,j+1) gets ay[i][j] = -n (C[i][j] - C[i-1][j]) (v = -dpsi/dx),
    so every cell's net outflow cancels exactly; both are scaled so that the largest
    face speed is 1.  Returns (ax, ay) as float32 [n][n]."""
    k = np.arange(1, modes + 1)
    c = rng.standard_normal((modes, modes))
    phi = rng.uniform(0.0, 2 * np.pi, size=(modes, modes))
    t = (np.arange(n) + 1.0) / n
    X, Y = np.meshgrid(t, t, indexing="ij")
    C = np.zeros((n, n))
    for a in range(modes):
        for b in range(modes):
            C += c[a, b] * np.sin(2 * np.pi * (k[a] * X + k[b] * Y) + phi[a, b]) / (k[a] ** 2 + k[b] ** 2)
    ax = n * (C - np.roll(C, 1, axis=1))
    ay = -n * (C - np.roll(C, 1, axis=0))
    scale = 1.0 / max(np.abs(ax).max(), np.abs(ay).max())
    return (ax * scale).astype(np.float32), (ay * scale).astype(np.float32)


def cell_velocity(ax, ay) -> np.ndarray:
    """Velocity at the cell centres, the mean of each cell's two faces per direction:
    a_x[i][j] = (ax[i][j] + ax[i-1][j]) / 2, a_y[i][j] = (ay[i][j] + ay[i][j-1]) / 2;
    float32 [n*n][2] row-major like cell_centers_2d."""
    vx = 0.5 * (ax + np.roll(ax, 1, axis=0))
    vy = 0.5 * (ay + np.roll(ay, 1, axis=1))
    return np.stack([vx.ravel(), vy.ravel()], axis=1).astype(np.float32)


@dataclass
class AdvDiffWorkload:
    """Inputs of the learned-model workload (trajectories differ only in nu)."""
    n: int
    ax: np.ndarray      # [n][n] float32 face velocities
    ay: np.ndarray
    u0: np.ndarray      # [n][n] float32 initial field
    nu: np.ndarray      # [n_traj] float32
    dt: float
    steps: int
    every: int
    n_train: int


def advdiff_learned(n: int = 256, n_traj: int = 64, n_train: int = 56, seed: int = 40) -> AdvDiffWorkload:
    rng = np.random.default_rng(seed)
    ax, ay = stream_function_faces(n, rng)
    u0 = periodic_bumps_2d(n, rng).astype(np.float32)
    nu = rng.uniform(1e-3, 1e-2, size=n_traj).astype(np.float32)
    return AdvDiffWorkload(n, ax, ay, u0, nu, dt=2.5e-4, steps=2000, every=10, n_train=n_train)
