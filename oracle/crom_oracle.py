"""Plain FP64 oracle of CROM's online latent-space time step.  TEST INFRASTRUCTURE ONLY.

This module is the parity reference for the CUDA library.  It is deliberately slow
and literal: numpy FP64 arrays, one line per equation, no blocking, no fusion and
no reordering beyond what the paper's definitions state.  Library primitives used
as single steps: ``@`` (matrix product), ``np.linalg.qr`` (only in ``lls_qr``, the
independent solver used by the pins).

What it follows (section / equation / algorithm of arXiv 2206.02607):

* Decoder g(x, q): an MLP R^{m+r} -> R with ELU or SIREN hidden layers and a
  linear output layer (App. D).  ELU with alpha = 1 (Clevert et al.):
  s(z) = z (z > 0) else expm1(z); s'(z) = 1 (z > 0) else e^z; s''(z) = 0 (z > 0) else e^z.
  The tie z = 0 takes the negative branch.  SIREN (Sitzmann et al., omega0 = 30):
  s(z) = sin(omega0 z); s'(z) = omega0 cos(omega0 z); s''(z) = -omega0^2 sin(omega0 z).
* Step 1, network inference (§4.1, Algorithm 4): value, spatial gradient and the
  latent Jacobian dg/dq at every integration sample.  Derivatives are carried
  layer by layer with the value in one forward pass, which is Algorithm 2
  (network gradient, App. E.1.1) written per channel and extended to second
  order: z = W h + b; dz = W dh; d2z = W d2h; h = s(z); dh = s'(z) dz;
  d2h = s''(z) dz^2 + s'(z) d2z.  At layer 1, dz/dx_k = W[:, k], d2z = 0 and
  dz/dq_j = W[:, m+j].
* Step 2, PDE time stepping (§4.2, Eqs. discrete-time / time-integration):
  explicit forward Euler with the network Laplacian (App. G.3 and App. H.3):
  Delta f_j = dt * alpha * sum_k d2g/dx_k^2 (heat);
  Delta f_j = dt * (-a(y_j) . grad g + nu * Lap g) (advection-diffusion).
* Step 3, network inversion (§4.3, Eq. invert; App. C): Gauss-Newton on
  min_q sum_j (g(y_j, q) - f_{n+1}(y_j))^2 with f_{n+1}(y_j) = g(y_j, q_n) + Delta f_j,
  starting from q^(0) = q_n (App. C.1).  Each iteration solves the normal
  equations (J^T J) delta = -J^T rho by an unpivoted FP64 Cholesky factorisation.
  One iteration equals the linearised least squares of App. C.2.
  A Cholesky pivot <= 1e-14 * max(diag) stops the iteration with status SINGULAR
  and keeps the last iterate (a reading: the paper does not say what to do).
* Full-order models (App. G.2, App. H.2): second-order central finite differences
  and forward Euler.  1D Dirichlet 0; 2D zero Neumann via mirror ghost nodes;
  2D periodic advection-diffusion in conservative upwind flux form.
* Dense reconstruction: g(x_i, q_c) at arbitrary points (§3, continuous field).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

STATUS_OK = 0
STATUS_BAD_ARG = 1
STATUS_SINGULAR = 3
STATUS_NONFINITE = 4

__all__ = [
    "elu", "elu_d1", "elu_d2", "siren", "siren_d1", "siren_d2", "Evaluation", "MLPDecoder", "cholesky_solve", "lls_qr",
    "heat_delta_f", "advdiff_delta_f", "crom_step", "crom_rollout", "crom_step_batched",
    "reconstruct", "tangent_velocity", "fom_heat1d_step", "fom_heat2d_neumann_step", "fom_advdiff2d_step",
    "STATUS_OK", "STATUS_BAD_ARG", "STATUS_SINGULAR", "STATUS_NONFINITE",
]


# --------------------------------------------------------------------------- ELU

def elu(z):
    """ELU activation, alpha = 1 (App. D)."""
    return np.where(z > 0, z, np.expm1(np.minimum(z, 0.0)))


def elu_d1(z):
    """First derivative of ELU."""
    return np.where(z > 0, 1.0, np.exp(np.minimum(z, 0.0)))


def elu_d2(z):
    """Second derivative of ELU."""
    return np.where(z > 0, 0.0, np.exp(np.minimum(z, 0.0)))


def siren(z, w0=30.0):
    """SIREN activation sin(omega0 z) (App. D)."""
    return np.sin(w0 * z)


def siren_d1(z, w0=30.0):
    return w0 * np.cos(w0 * z)


def siren_d2(z, w0=30.0):
    return -w0 * w0 * np.sin(w0 * z)


# ---------------------------------------------------------------- decoder (Step 1)

@dataclass
class Evaluation:
    """Decoder outputs at N points.

    g: [N] value; gx: [N, m] dg/dx_k; gxx: [N, m] d2g/dx_k^2 (diagonal of the
    spatial Hessian); gq: [N, r] dg/dq_j (rows of the Jacobian J)."""
    g: np.ndarray
    gx: np.ndarray
    gxx: np.ndarray
    gq: np.ndarray

    @property
    def lap(self):
        return self.gxx.sum(axis=1)


class MLPDecoder:
    """g(x, q) = W_L s(... s(W_1 [x; q] + b_1) ...) + b_L, FP64 (App. D).

    params: list of (W [out][in], b [out]); layer 1 input is (x_1..x_m, q_1..q_r).
    """

    def __init__(self, params, m: int, activation: str = "elu", omega0: float = 30.0):
        self.params = [(np.asarray(W, np.float64), np.asarray(b, np.float64)) for W, b in params]
        self.m = m
        self.r = self.params[0][0].shape[1] - m
        self.width = self.params[0][0].shape[0]
        if activation == "elu":
            self.acts = (elu, elu_d1, elu_d2)
        elif activation == "siren":
            w0 = float(omega0)
            self.acts = (lambda z: siren(z, w0), lambda z: siren_d1(z, w0), lambda z: siren_d2(z, w0))
        else:
            raise ValueError(activation)

    def __call__(self, X, Q) -> Evaluation:
        return self.evaluate(X, Q)

    def evaluate(self, X, Q) -> Evaluation:
        """Forward pass carrying value and derivative channels (Algorithm 2, App. E.1.1).

        X: [N, m] points; Q: [N, r] latent code per point (or [r], broadcast)."""
        X = np.asarray(X, np.float64).reshape(-1, self.m)
        N = X.shape[0]
        Q = np.broadcast_to(np.asarray(Q, np.float64), (N, self.r))
        m, r = self.m, self.r
        W1, b1 = self.params[0]
        # Layer 1 pre-activation and its derivatives with respect to the inputs.
        z = X @ W1[:, :m].T + Q @ W1[:, m:].T + b1
        dz_x = [np.broadcast_to(W1[:, k], z.shape) for k in range(m)]
        d2z_x = [np.zeros_like(z) for _ in range(m)]
        dz_q = [np.broadcast_to(W1[:, m + j], z.shape) for j in range(r)]
        for W, b in self.params[1:]:
            s0, s1, s2 = self.acts[0](z), self.acts[1](z), self.acts[2](z)
            h = s0
            dh_x = [s1 * dz_x[k] for k in range(m)]
            d2h_x = [s2 * dz_x[k] ** 2 + s1 * d2z_x[k] for k in range(m)]
            dh_q = [s1 * dz_q[j] for j in range(r)]
            z = h @ W.T + b
            dz_x = [d @ W.T for d in dh_x]
            d2z_x = [d @ W.T for d in d2h_x]
            dz_q = [d @ W.T for d in dh_q]
        # The output layer is linear: z now holds g and its channels, shape [N, 1].
        g = z[:, 0]
        gx = np.stack([d[:, 0] for d in dz_x], axis=1)
        gxx = np.stack([d[:, 0] for d in d2z_x], axis=1)
        gq = np.stack([d[:, 0] for d in dz_q], axis=1) if r else np.zeros((N, 0))
        return Evaluation(g, gx, gxx, gq)

    def value(self, X, Q):
        """Value channel only: plain forward pass."""
        X = np.asarray(X, np.float64).reshape(-1, self.m)
        Q = np.broadcast_to(np.asarray(Q, np.float64), (X.shape[0], self.r))
        h = np.concatenate([X, Q], axis=1)
        for li, (W, b) in enumerate(self.params):
            z = h @ W.T + b
            h = self.acts[0](z) if li + 1 < len(self.params) else z
        return h[:, 0]


# ------------------------------------------------------------ linear algebra

def cholesky_solve(A, rhs, pivot_rel: float = 1e-14):
    """Solve A x = rhs for symmetric positive definite A by an unpivoted Cholesky
    factorisation A = L L^T and two triangular solves (FP64).

    Returns (x, status).  status = SINGULAR when a pivot is <= pivot_rel * max(diag A)
    (or not positive), NONFINITE when A or rhs holds a NaN/Inf."""
    A = np.asarray(A, np.float64)
    rhs = np.asarray(rhs, np.float64)
    n = A.shape[0]
    if not (np.all(np.isfinite(A)) and np.all(np.isfinite(rhs))):
        return np.zeros(n), STATUS_NONFINITE
    tol = pivot_rel * max(np.max(np.diag(A)), 0.0)
    L = np.zeros((n, n))
    for j in range(n):
        d = A[j, j] - np.dot(L[j, :j], L[j, :j])
        if not d > tol:
            return np.zeros(n), STATUS_SINGULAR
        L[j, j] = np.sqrt(d)
        for i in range(j + 1, n):
            L[i, j] = (A[i, j] - np.dot(L[i, :j], L[j, :j])) / L[j, j]
    y = np.zeros(n)
    for i in range(n):
        y[i] = (rhs[i] - np.dot(L[i, :i], y[:i])) / L[i, i]
    x = np.zeros(n)
    for i in reversed(range(n)):
        x[i] = (y[i] - np.dot(L[i + 1:, i], x[i + 1:])) / L[i, i]
    return x, STATUS_OK


def lls_qr(J, b):
    """Linear least squares min_d ||J d - b||_2 by Householder QR (independent of
    the normal equations; used only by the pins)."""
    Qm, R = np.linalg.qr(np.asarray(J, np.float64))
    return np.linalg.solve(R, Qm.T @ np.asarray(b, np.float64))


# ------------------------------------------------------------ Step 2: PDE update

def heat_delta_f(ev: Evaluation, alpha, dt: float):
    """Forward Euler increment of u_t = alpha * Lap u with the network Laplacian
    (App. G.2/G.3 and App. H.2/H.3): Delta f_j = dt * alpha * sum_k d2g/dx_k^2.
    alpha is a scalar or one value per sample (nu(y_j) for u_t = nu(x) Lap u)."""
    return dt * alpha * ev.lap


def advdiff_delta_f(ev: Evaluation, vel, nu: float, dt: float):
    """Forward Euler increment of u_t + a . grad u = nu Lap u at the samples:
    Delta f_j = dt * (-a(y_j) . grad g(y_j) + nu * Lap g(y_j))."""
    return dt * (-(np.asarray(vel, np.float64) * ev.gx).sum(axis=1) + nu * ev.lap)


# ------------------------------------------------------- one latent step (Alg. 3)

ARMIJO_C1 = 1e-4   # sufficient-decrease constant of the backtracking line search


def crom_step(decoder, q_n, Y, dt: float, gn_iters: int, alpha: float = 1.0,
              pde: str = "heat", vel=None, nu: float = 0.0, return_info: bool = False,
              line_search: int = 0):
    """One latent-space step q_n -> q_{n+1} (Algorithm 3 = Algorithms 4, then the PDE
    update, then Algorithm 5).

    decoder: callable (X, q) -> Evaluation (an MLPDecoder, or any test decoder).
    Y: [M, m] integration samples.  Returns (q_{n+1}, status[, info]).

    line_search = L > 0 equips each Gauss-Newton iteration with a standard
    backtracking line search (§4.3 / App. C; Nocedal & Wright, Alg. 3.1): with
    phi(q) = 1/2 sum_j (g(y_j, q) - target_j)^2, v = J^T rho and the GN direction
    delta, the step length a = 1, 1/2, ..., 2^-L is the first that satisfies
    phi(q + a delta) <= phi(q) + c1 a v.delta (c1 = 1e-4).  If none does, q is kept
    and the remaining iterations are skipped (the direction no longer decreases phi
    at any tried length)."""
    q_n = np.asarray(q_n, np.float64)
    Y = np.asarray(Y, np.float64)
    r = q_n.shape[0]
    if Y.shape[0] < r:                           # well-posedness r <= d|M| (§4.4)
        return q_n.copy(), STATUS_BAD_ARG
    # Step 1: network inference at q_n.
    ev = decoder(Y, q_n)
    # Step 2: explicit PDE update at the samples; target f_{n+1}(y_j).
    if pde == "heat":
        df = heat_delta_f(ev, alpha, dt)
    else:
        df = advdiff_delta_f(ev, vel, nu, dt)
    target = ev.g + df
    # Step 3: Gauss-Newton on sum_j (g(y_j, q) - target_j)^2 from q^(0) = q_n.
    q = q_n.copy()
    status = STATUS_OK
    deltas, trials = [], []
    for k in range(gn_iters):
        if k > 0:
            ev = decoder(Y, q)
        rho = ev.g - target
        J = ev.gq
        A = J.T @ J
        v = J.T @ rho
        delta, status = cholesky_solve(A, -v)
        if status != STATUS_OK:
            break
        if line_search <= 0:
            q = q + delta
            deltas.append(delta)
            continue
        phi0 = 0.5 * float(rho @ rho)
        slope = float(v @ delta)
        a, accepted, tried = 1.0, False, []
        for _ in range(line_search + 1):
            q_try = q + a * delta
            r_try = decoder(Y, q_try).g - target
            phi = 0.5 * float(r_try @ r_try)
            bound = phi0 + ARMIJO_C1 * a * slope
            tried.append((a, phi, bound))
            if phi <= bound:
                accepted = True
                break
            a *= 0.5
        trials.append(tried)
        if not accepted:
            break
        deltas.append(q_try - q)
        q = q_try
    if return_info:
        return q, status, {"delta_f": df, "deltas": deltas, "line_search_trials": trials}
    return q, status


def crom_step_batched(decoder, q, s_off, samples, alpha, dt, gn_iters, alpha_per_sample: bool = False,
                      line_search: int = 0):
    """Independent heat steps for a batch of instances sharing one decoder.

    alpha: one diffusion coefficient per instance, or (alpha_per_sample) one per
    integration sample, nu(y_j), for the spatially varying coefficient of
    u_t = nu(x) Lap u (App. G thermodynamics, App. H image diffusion)."""
    q = np.asarray(q, np.float64)
    out = np.empty_like(q)
    status = np.zeros(q.shape[0], np.int32)
    for i in range(q.shape[0]):
        Y = samples[s_off[i]:s_off[i + 1]]
        a = np.asarray(alpha[s_off[i]:s_off[i + 1]], np.float64) if alpha_per_sample else float(alpha[i])
        out[i], status[i] = crom_step(decoder, q[i], Y, dt, gn_iters, alpha=a, line_search=line_search)
    return out, status


def crom_rollout(decoder, q0, Y, dt, gn_iters, steps, alpha=1.0):
    """Repeat crom_step; returns the trajectory [steps+1, r]."""
    traj = [np.asarray(q0, np.float64)]
    q = traj[0]
    for _ in range(steps):
        q, st = crom_step(decoder, q, Y, dt, gn_iters, alpha=alpha)
        if st != STATUS_OK:
            raise RuntimeError(f"oracle step failed with status {st}")
        traj.append(q)
    return np.stack(traj)


def tangent_velocity(decoder, X, q, q_prev, dt: float):
    """Velocity of the field on the manifold's tangent space (App. L, Solid
    Mechanics): v(x) = dg/dq(x, q_n) . qdot with qdot = (q_n - q_{n-1}) / dt."""
    qdot = (np.asarray(q, np.float64) - np.asarray(q_prev, np.float64)) / dt
    return decoder(X, q).gq @ qdot


# ------------------------------------------------------------ reconstruction

def reconstruct(decoder: MLPDecoder, codes, X):
    """Dense field g(x_i, q_c): returns [n_codes][n_pts]."""
    return np.stack([decoder.value(X, c) for c in np.asarray(codes, np.float64)])


# ------------------------------------------------------------ full-order models

def fom_heat1d_step(u, dt: float, nu=1.0):
    """1D heat, Dirichlet 0 (App. G.2): u_i += dt * nu_i * (u_{i-1} + u_{i+1} - 2u_i) / dx^2
    on interior nodes of x_i = i/(P-1); the two boundary nodes stay 0."""
    u = np.asarray(u, np.float64)
    dx = 1.0 / (u.shape[0] - 1)
    nu = np.broadcast_to(np.asarray(nu, np.float64), u.shape)
    out = np.zeros_like(u)
    out[1:-1] = u[1:-1] + dt * nu[1:-1] * (u[:-2] + u[2:] - 2.0 * u[1:-1]) / dx ** 2
    return out


def fom_heat2d_neumann_step(u, dt: float, alpha=1.0):
    """2D heat on the n x n grid of [0,1]^2 (App. H.2), zero Neumann boundary by
    mirror ghost nodes u_{-1} = u_1 and u_n = u_{n-2} in each direction."""
    u = np.asarray(u, np.float64)
    n = u.shape[0]
    h = 1.0 / (n - 1)
    p = np.pad(u, 1, mode="reflect")   # reflect: ghost value equals the node one step inside
    lap = (p[:-2, 1:-1] + p[2:, 1:-1] - 2.0 * u) / h ** 2 + (p[1:-1, :-2] + p[1:-1, 2:] - 2.0 * u) / h ** 2
    return u + dt * np.asarray(alpha, np.float64) * lap


def fom_advdiff2d_step(u, ax_face, ay_face, nu: float, dt: float, scheme: str = "upwind"):
    """2D periodic advection-diffusion u_t + div(a u) = nu Lap u on n x n cells of
    width h = 1/n, forward Euler.  Advection in conservative flux form with face
    velocities: ax_face[i, j] lives on the face between cells (i, j) and (i+1, j);
    ay_face[i, j] between (i, j) and (i, j+1); the face value of u is the upwind
    cell's (scheme "upwind", first order) or the mean of the two cells ("central",
    second order).  Diffusion by the central 5-point stencil.  For a discretely
    divergence-free face field this equals the advective form a . grad u."""
    u = np.asarray(u, np.float64)
    n = u.shape[0]
    h = 1.0 / n
    up_x = np.roll(u, -1, axis=0)
    up_y = np.roll(u, -1, axis=1)
    if scheme == "central":
        Fx = ax_face * 0.5 * (u + up_x)
        Fy = ay_face * 0.5 * (u + up_y)
    else:
        Fx = np.where(ax_face > 0, ax_face * u, ax_face * up_x)
        Fy = np.where(ay_face > 0, ay_face * u, ay_face * up_y)
    div = (Fx - np.roll(Fx, 1, axis=0) + Fy - np.roll(Fy, 1, axis=1)) / h
    lap = (np.roll(u, 1, 0) + np.roll(u, -1, 0) + np.roll(u, 1, 1) + np.roll(u, -1, 1) - 4.0 * u) / h ** 2
    return u + dt * (-div + nu * lap)
