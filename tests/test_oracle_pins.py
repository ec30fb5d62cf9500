"""Pins of the FP64 oracle against facts fixed outside it (CPU only).

Each test checks the oracle against something other than itself: closed forms,
a hand-worked example, finite differences, an independent autodiff evaluation,
an independent least-squares solver or brute-force minimisation.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import crom_oracle as O
from workloads import gen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# ------------------------------------------------------------------ O8 hand example

def test_hand_worked_mlp():
    """A 1-hidden-layer decoder evaluated by hand (golden fixture, App. D + Alg. 2)."""
    with open(os.path.join(GOLDEN, "hand_mlp.json")) as f:
        fx = json.load(f)
    net = fx["network"]
    dec = O.MLPDecoder([(net["W1"], net["b1"]), (net["W2"], net["b2"])], m=1)
    for c in fx["cases"]:
        ev = dec(np.array([[c["x"]]]), np.array([c["q"]]))
        assert ev.g[0] == pytest.approx(c["g"], rel=1e-14)
        assert ev.gx[0, 0] == pytest.approx(c["gx"], rel=1e-14)
        assert ev.gxx[0, 0] == pytest.approx(c["gxx"], rel=1e-14)
        assert ev.gq[0, 0] == pytest.approx(c["gq"], rel=1e-14)
        assert dec.value(np.array([[c["x"]]]), np.array([c["q"]]))[0] == pytest.approx(c["g"], rel=1e-14)


def test_elu_closed_forms():
    z = np.array([-3.0, -1e-9, 0.0, 1e-9, 2.5])
    np.testing.assert_allclose(O.elu(z), [math.exp(-3) - 1, math.expm1(-1e-9), 0.0, 1e-9, 2.5], rtol=1e-15)
    np.testing.assert_allclose(O.elu_d1(z), [math.exp(-3), math.exp(-1e-9), 1.0, 1.0, 1.0], rtol=1e-15)
    np.testing.assert_allclose(O.elu_d2(z), [math.exp(-3), math.exp(-1e-9), 1.0, 0.0, 0.0], rtol=1e-15)


# ------------------------------------------------------------ O2 decoder derivatives

def _kink_margin(params, X, Q, m):
    """Smallest |pre-activation| over all hidden units (plain forward, test-side)."""
    h = np.concatenate([X, np.broadcast_to(Q, (X.shape[0], Q.shape[-1]))], axis=1)
    margin = np.full(X.shape[0], np.inf)
    for W, b in params[:-1]:
        z = h @ W.T + b
        margin = np.minimum(margin, np.abs(z).min(axis=1))
        h = np.where(z > 0, z, np.expm1(np.minimum(z, 0)))
    return margin


@pytest.mark.parametrize("m,r,width,hidden", [(1, 3, 32, 3), (2, 4, 32, 3), (2, 8, 48, 4)])
def test_decoder_derivatives_vs_central_fd(m, r, width, hidden):
    """dg/dx, d2g/dx2, dg/dq against central differences of the value (rel err <= 1e-6)."""
    spec = gen.DecoderSpec(m, r, width, hidden)
    params = gen.xavier_decoder(spec, seed=11, bias_std=0.3)
    dec = O.MLPDecoder(params, m)
    rng = np.random.default_rng(12)
    X = rng.uniform(0, 1, size=(2048, m))
    q = rng.standard_normal(r)
    keep = _kink_margin(dec.params, X, q[None, :], m) > 1e-2
    X = X[keep]
    assert X.shape[0] >= 16
    ev = dec(X, q)
    h1, h2 = 1e-5, 1e-3
    for k in range(m):
        e = np.zeros(m); e[k] = 1
        fd1 = (dec.value(X + h1 * e, q) - dec.value(X - h1 * e, q)) / (2 * h1)
        # fourth-order five-point stencil for the second derivative
        v = [dec.value(X + s * h2 * e, q) for s in (-2, -1, 0, 1, 2)]
        fd2 = (-v[0] + 16 * v[1] - 30 * v[2] + 16 * v[3] - v[4]) / (12 * h2 ** 2)
        assert rel(ev.gx[:, k], fd1) < 1e-6
        assert rel(ev.gxx[:, k], fd2) < 1e-6
    for j in range(r):
        e = np.zeros(r); e[j] = 1
        fd = (dec.value(X, q + h1 * e) - dec.value(X, q - h1 * e)) / (2 * h1)
        assert rel(ev.gq[:, j], fd) < 1e-6
    np.testing.assert_allclose(ev.g, dec.value(X, q), rtol=1e-13, atol=1e-15)


def test_decoder_derivatives_vs_autodiff():
    """Exact check of every channel against reverse-mode autodiff of an independently
    written torch FP64 forward pass (no truncation error: 1e-12)."""
    torch = pytest.importorskip("torch")
    spec = gen.DecoderSpec(2, 5, 24, 3)
    params = gen.xavier_decoder(spec, seed=3, bias_std=0.5)
    dec = O.MLPDecoder(params, 2)
    rng = np.random.default_rng(4)
    X = rng.uniform(0, 1, size=(10, 2))
    q = rng.standard_normal(5)
    ev = dec(X, q)
    Wt = [(torch.tensor(W), torch.tensor(b)) for W, b in params]

    def f(xq):
        h = xq
        for li, (W, b) in enumerate(Wt):
            z = W @ h + b
            h = torch.nn.functional.elu(z) if li + 1 < len(Wt) else z
        return h[0]

    for i in range(X.shape[0]):
        xq = torch.tensor(np.concatenate([X[i], q]), requires_grad=True)
        grad = torch.autograd.functional.jacobian(f, xq).numpy()
        hess = torch.autograd.functional.hessian(f, xq).numpy()
        np.testing.assert_allclose(ev.gx[i], grad[:2], rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(ev.gq[i], grad[2:], rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(ev.gxx[i], np.diag(hess)[:2], rtol=1e-12, atol=1e-14)


# ------------------------------------------------------------------ linear algebra

def test_cholesky_solve_against_closed_form_and_singular():
    rng = np.random.default_rng(0)
    B = rng.standard_normal((12, 8))
    A = B.T @ B + 0.1 * np.eye(8)
    x_true = rng.standard_normal(8)
    x, st = O.cholesky_solve(A, A @ x_true)
    assert st == O.STATUS_OK and rel(x, x_true) < 1e-12
    # rank-deficient normal matrix (duplicate columns) must be flagged, not solved
    Bs = np.concatenate([B[:, :4], B[:, :4]], axis=1)
    _, st = O.cholesky_solve(Bs.T @ Bs, np.ones(8))
    assert st == O.STATUS_SINGULAR
    _, st = O.cholesky_solve(A, np.array([np.nan] + [0.0] * 7))
    assert st == O.STATUS_NONFINITE


# ---------------------------------------------------------- test decoders (callables)

class FourierDecoder1D:
    """g(x, q) = sum_k q_k sin(k pi x) + c(x): linear in q, Lap g known exactly."""

    def __init__(self, r, offset=False):
        self.r, self.offset = r, offset

    def __call__(self, X, q):
        x = np.asarray(X, np.float64)[:, 0]
        k = np.arange(1, self.r + 1)
        S = np.sin(np.pi * np.outer(x, k))
        C = np.pi * k * np.cos(np.pi * np.outer(x, k))
        g = S @ q + (x ** 2 if self.offset else 0.0)
        gx = C @ q + (2 * x if self.offset else 0.0)
        gxx = -(np.pi * k) ** 2 * S @ q + (2.0 if self.offset else 0.0)
        return O.Evaluation(g, gx[:, None], gxx[:, None] if np.ndim(gxx) else np.full((x.size, 1), gxx), S)


class CosineDecoder2D:
    """g(x, q) = sum_{(k,l)} q_(k,l) cos(k pi x1) cos(l pi x2); Lap = -pi^2 (k^2 + l^2) g_kl."""

    def __init__(self, modes):
        self.modes = modes

    def __call__(self, X, q):
        X = np.asarray(X, np.float64)
        cols, lap, gx1, gx2, gxx1, gxx2 = [], [], [], [], [], []
        for (k, l) in self.modes:
            ck, cl = np.cos(k * np.pi * X[:, 0]), np.cos(l * np.pi * X[:, 1])
            sk, sl = np.sin(k * np.pi * X[:, 0]), np.sin(l * np.pi * X[:, 1])
            cols.append(ck * cl)
            gx1.append(-k * np.pi * sk * cl); gx2.append(-l * np.pi * ck * sl)
            gxx1.append(-(k * np.pi) ** 2 * ck * cl); gxx2.append(-(l * np.pi) ** 2 * ck * cl)
        J = np.stack(cols, 1)
        return O.Evaluation(J @ q, np.stack([np.stack(gx1, 1) @ q, np.stack(gx2, 1) @ q], 1),
                            np.stack([np.stack(gxx1, 1) @ q, np.stack(gxx2, 1) @ q], 1), J)


# ------------------------------------------------------------- O3, O4, O5, O6: GN

def test_gn_linear_in_q_equals_qr_lls_and_is_stationary():
    """O3: g linear in q -> one GN iteration is the exact LLS; a second one is a no-op."""
    dec = FourierDecoder1D(4, offset=True)
    rng = np.random.default_rng(1)
    Y = rng.uniform(0.05, 0.95, size=(11, 1))
    q0 = rng.standard_normal(4)
    dt, alpha = 3e-3, 0.7
    q1, st = O.crom_step(dec, q0, Y, dt, 1, alpha=alpha)
    ev = dec(Y, q0)
    target = ev.g + dt * alpha * ev.lap
    # LLS of min ||J q - (target - c)|| solved by Householder QR, independent of the normal eqs.
    c = Y[:, 0] ** 2
    q_lls = O.lls_qr(ev.gq, target - c)
    assert st == O.STATUS_OK and rel(q1, q_lls) < 1e-12
    q2, _ = O.crom_step(dec, q0, Y, dt, 2, alpha=alpha)
    assert rel(q2, q1) < 1e-12


def test_gn_one_iteration_equals_linearised_lls():
    """O4: with one GN iteration the step equals q_n + argmin ||J(q_n) d - Delta f|| (App. C.2)."""
    spec = gen.DecoderSpec(2, 6, 32, 3)
    dec = O.MLPDecoder(gen.xavier_decoder(spec, seed=5, bias_std=0.2), 2)
    rng = np.random.default_rng(2)
    Y = rng.uniform(0, 1, size=(40, 2))
    q0 = rng.standard_normal(6)
    dt = 1e-2
    q1, st = O.crom_step(dec, q0, Y, dt, 1, alpha=1.3)
    ev = dec(Y, q0)
    d_lls = O.lls_qr(ev.gq, dt * 1.3 * ev.lap)
    assert st == O.STATUS_OK and rel(q1 - q0, d_lls) < 1e-10


def test_fourier_decoder_step_closed_form_1d():
    """O5: sine decoder, heat equation -> q_k(n) = q_k(0) (1 - dt alpha k^2 pi^2)^n exactly."""
    r = 5
    dec = FourierDecoder1D(r)
    Y = (np.arange(1, 13) / 13.0)[:, None]
    q0 = np.random.default_rng(3).standard_normal(r)
    dt, alpha, n = 1e-4, 0.9, 25
    traj = O.crom_rollout(dec, q0, Y, dt, gn_iters=2, steps=n, alpha=alpha)
    k = np.arange(1, r + 1)
    expect = q0 * (1 - dt * alpha * (k * np.pi) ** 2) ** n
    assert rel(traj[-1], expect) < 1e-12


def test_cosine_decoder_step_closed_form_2d():
    """O5 (2D): cosine-product decoder -> multiplier 1 - dt alpha pi^2 (k^2 + l^2) per mode."""
    modes = [(0, 1), (1, 0), (1, 1), (2, 1), (1, 3)]
    dec = CosineDecoder2D(modes)
    rng = np.random.default_rng(4)
    Y = rng.uniform(0, 1, size=(30, 2))
    q0 = rng.standard_normal(len(modes))
    dt, alpha = 2e-4, 1.7
    q1, st = O.crom_step(dec, q0, Y, dt, 2, alpha=alpha)
    lam = np.array([k * k + l * l for k, l in modes]) * np.pi ** 2
    assert st == O.STATUS_OK and rel(q1, q0 * (1 - dt * alpha * lam)) < 1e-12


class PlaneWaveDecoder2D:
    """g(x, q) = q_1 sin(theta) + q_2 cos(theta), theta = 2 pi (k x1 + l x2): linear in q;
    grad g = 2 pi (k, l) (q_1 cos - q_2 sin), d2g/dx_i^2 = -(2 pi k_i)^2 g."""

    def __init__(self, k, l):
        self.k, self.l = k, l

    def __call__(self, X, q):
        X = np.asarray(X, np.float64)
        th = 2 * np.pi * (self.k * X[:, 0] + self.l * X[:, 1])
        J = np.stack([np.sin(th), np.cos(th)], 1)
        g = J @ q
        dth = q[0] * np.cos(th) - q[1] * np.sin(th)
        kk = 2 * np.pi * np.array([self.k, self.l], np.float64)
        return O.Evaluation(g, dth[:, None] * kk[None, :], -(kk[None, :] ** 2) * g[:, None], J)


def test_advection_diffusion_step_closed_form_and_continuous_limit():
    """O5 (advection-diffusion): for u_t + a . grad u = nu Lap u with a uniform velocity,
    a plane wave travels along a and decays: with z = q_1 + i q_2,
    z(t) = exp(-(nu lam + i w) t) z(0), lam = 4 pi^2 (k^2 + l^2), w = 2 pi (a_1 k + a_2 l).
    The decoder is linear in q, so each latent step is the forward Euler factor
    1 - dt (nu lam + i w) exactly, and n steps converge to z(t) at first order.
    k != l and a_1 != a_2, so swapped velocity components, a wrong sign on the
    advection term or a dropped diffusion term each fail."""
    k, l = 1, 2
    a, nu = np.array([0.7, -0.3]), 0.02
    dec = PlaneWaveDecoder2D(k, l)
    rng = np.random.default_rng(41)
    Y = rng.uniform(0, 1, size=(23, 2))
    vel = np.tile(a, (Y.shape[0], 1))           # one velocity per sample, here uniform
    q0 = np.array([0.8, -0.45])
    lam = 4 * np.pi ** 2 * (k * k + l * l)
    w = 2 * np.pi * (a[0] * k + a[1] * l)
    z0 = complex(q0[0], q0[1])
    dt = 1e-3
    q1, st, info = O.crom_step(dec, q0, Y, dt, 2, pde="advdiff", vel=vel, nu=nu, return_info=True)
    z1 = (1 - dt * (nu * lam + 1j * w)) * z0
    assert st == O.STATUS_OK and rel(q1, [z1.real, z1.imag]) < 1e-12
    assert np.abs(info["deltas"][1]).max() < 1e-14     # the second GN iteration is a no-op
    # n steps: the discrete closed form, and first-order convergence to the continuous wave
    T = 0.05
    errs = []
    for n in (50, 100, 200):
        q = q0.copy()
        for _ in range(n):
            q, st = O.crom_step(dec, q, Y, T / n, 1, pde="advdiff", vel=vel, nu=nu)
            assert st == O.STATUS_OK
        zn = (1 - T / n * (nu * lam + 1j * w)) ** n * z0
        assert rel(q, [zn.real, zn.imag]) < 1e-11
        zt = np.exp(-(nu * lam + 1j * w) * T) * z0
        errs.append(abs(complex(q[0], q[1]) - zt))
    assert 1.8 < errs[0] / errs[1] < 2.2 and 1.8 < errs[1] / errs[2] < 2.2
    assert errs[-1] < 5e-3 * abs(z0)


@pytest.mark.parametrize("r", [1, 2])
def test_gn_converges_to_brute_force_minimiser(r):
    """O6: converged GN (20 iterations) equals the brute-force minimiser of the NLS
    objective sum_j (g(y_j, q) - target_j)^2 on a tiny decoder."""
    spec = gen.DecoderSpec(1, r, 16, 2)
    dec = O.MLPDecoder(gen.xavier_decoder(spec, seed=7 + r, bias_std=0.3), 1)
    Y = (np.arange(1, 10) / 10.0)[:, None]
    q0 = np.random.default_rng(8).standard_normal(r) * 0.5
    dt = 0.02
    ev = dec(Y, q0)
    target = ev.g + dt * ev.lap

    def F(q):
        return float(np.sum((dec.value(Y, q) - target) ** 2))

    q_gn, st = O.crom_step(dec, q0, Y, dt, 20)
    assert st == O.STATUS_OK
    # brute force: dense grid around q0, then golden-section refinement per coordinate
    if r == 1:
        grid = q0[0] + np.linspace(-1, 1, 4001)
        vals = [F(np.array([g])) for g in grid]
        best = grid[int(np.argmin(vals))]
        lo, hi = best - 1e-3, best + 1e-3
        phi = (math.sqrt(5) - 1) / 2
        for _ in range(80):
            a, b = hi - phi * (hi - lo), lo + phi * (hi - lo)
            if F(np.array([a])) < F(np.array([b])):
                hi = b
            else:
                lo = a
        q_bf = np.array([(lo + hi) / 2])
    else:
        g1 = q0[0] + np.linspace(-0.5, 0.5, 201)
        g2 = q0[1] + np.linspace(-0.5, 0.5, 201)
        vals = np.array([[F(np.array([a, b])) for b in g2] for a in g1])
        i, j = np.unravel_index(np.argmin(vals), vals.shape)
        q_bf = np.array([g1[i], g2[j]])
        # derivative-free refinement (Nelder-Mead) from the grid minimiser
        from scipy.optimize import minimize
        res = minimize(F, q_bf, method="Nelder-Mead",
                       options={"xatol": 1e-12, "fatol": 1e-30, "maxiter": 20000, "maxfev": 40000})
        q_bf = res.x
    assert np.max(np.abs(q_gn - q_bf)) < 1e-7


def test_too_few_samples_is_bad_arg():
    """Well-posedness r <= d|M| (§4.4)."""
    dec = FourierDecoder1D(4)
    q, st = O.crom_step(dec, np.ones(4), np.array([[0.2], [0.4], [0.6]]), 1e-4, 1)
    assert st == O.STATUS_BAD_ARG


def test_duplicate_samples_singular():
    """rank(J) < r (all samples at one point) is reported as SINGULAR; q is kept."""
    spec = gen.DecoderSpec(2, 3, 16, 2)
    dec = O.MLPDecoder(gen.xavier_decoder(spec, seed=1), 2)
    Y = np.tile([[0.3, 0.6]], (8, 1))
    q0 = np.array([0.1, -0.2, 0.3])
    q, st = O.crom_step(dec, q0, Y, 1e-3, 2)
    assert st == O.STATUS_SINGULAR and np.array_equal(q, q0)


# ------------------------------------------------------------------ O1: FOMs

def test_fom_heat1d_discrete_eigenmodes_and_continuous_decay():
    P = 256
    dx = 1 / (P - 1)
    a, u0 = gen.sine_modes_1d(P, np.random.default_rng(1))
    dt = dx ** 2 / 4
    n = 400
    u = u0.copy()
    for _ in range(n):
        u = O.fom_heat1d_step(u, dt)
    x = np.arange(P) * dx
    k = np.arange(1, 5)
    lam = 1 - 4 * dt / dx ** 2 * np.sin(k * np.pi * dx / 2) ** 2
    exact_discrete = sum(a[i] * lam[i] ** n * np.sin(k[i] * np.pi * x) for i in range(4))
    assert rel(u, exact_discrete) < 1e-12
    t = n * dt
    exact_cont = sum(a[i] * np.exp(-(k[i] * np.pi) ** 2 * t) * np.sin(k[i] * np.pi * x) for i in range(4))
    assert rel(u, exact_cont) < 1e-3


def test_fom_heat2d_neumann_cosine_modes_and_mass():
    n = 64
    h = 1 / (n - 1)
    t = np.arange(n) * h
    X1, X2 = np.meshgrid(t, t, indexing="ij")
    k, l = 2, 3
    u0 = np.cos(k * np.pi * X1) * np.cos(l * np.pi * X2)
    dt, alpha, steps = h ** 2 / 8, 1.0, 50
    u = u0.copy()
    for _ in range(steps):
        u = O.fom_heat2d_neumann_step(u, dt, alpha)
    mult = 1 - 4 * alpha * dt / h ** 2 * (np.sin(k * np.pi * h / 2) ** 2 + np.sin(l * np.pi * h / 2) ** 2)
    assert rel(u, u0 * mult ** steps) < 1e-12
    # trapezoid-weighted mass is conserved by the mirror-ghost Neumann scheme
    w = np.ones(n); w[0] = w[-1] = 0.5
    W = np.outer(w, w)
    v = gen.gaussian_bumps_2d(n, np.random.default_rng(3))
    m0 = np.sum(W * v)
    for _ in range(50):
        v = O.fom_heat2d_neumann_step(v, dt, alpha)
    assert abs(np.sum(W * v) - m0) < 1e-12 * abs(m0)


def _stream_faces(n, rng):
    """Face velocities from a nodal stream function (discretely divergence-free)."""
    psi = rng.standard_normal((n, n))
    h = 1 / n
    ax = (psi - np.roll(psi, 1, axis=1)) / h      # on x-faces
    ay = -(psi - np.roll(psi, 1, axis=0)) / h     # on y-faces
    return ax, ay


def test_fom_advdiff_conservation_and_constants():
    n = 32
    rng = np.random.default_rng(9)
    ax, ay = _stream_faces(n, rng)
    h = 1 / n
    dt = 0.2 * h / np.max(np.abs(np.concatenate([ax.ravel(), ay.ravel()])))
    u = rng.uniform(0, 1, size=(n, n))
    m0 = u.sum()
    for _ in range(20):
        u = O.fom_advdiff2d_step(u, ax, ay, 1e-3, dt)
    assert abs(u.sum() - m0) < 1e-12 * m0
    c = np.full((n, n), 0.7)
    c1 = O.fom_advdiff2d_step(c, ax, ay, 1e-3, dt)
    assert np.max(np.abs(c1 - 0.7)) < 1e-12


def test_fom_advdiff_translation_and_diffusion_modes():
    n = 16
    h = 1 / n
    rng = np.random.default_rng(2)
    u = rng.uniform(size=(n, n))
    a = 3.0
    ax, ay = np.full((n, n), a), np.zeros((n, n))
    u1 = O.fom_advdiff2d_step(u, ax, ay, 0.0, h / a)       # Courant number 1: exact shift
    np.testing.assert_allclose(u1, np.roll(u, 1, axis=0), rtol=0, atol=1e-14)
    ax, ay = -np.full((n, n), a), np.zeros((n, n))
    u1 = O.fom_advdiff2d_step(u, ax, ay, 0.0, h / a)
    np.testing.assert_allclose(u1, np.roll(u, -1, axis=0), rtol=0, atol=1e-14)
    # pure diffusion: periodic Fourier modes are exact eigenvectors
    t = np.arange(n) * h
    X1, X2 = np.meshgrid(t, t, indexing="ij")
    v = np.sin(2 * np.pi * 2 * X1) * np.cos(2 * np.pi * 3 * X2)
    nu, dt = 0.01, 0.1 * h * h / 0.01
    v1 = O.fom_advdiff2d_step(v, np.zeros((n, n)), np.zeros((n, n)), nu, dt)
    mult = 1 - 4 * nu * dt / h ** 2 * (np.sin(2 * np.pi * h) ** 2 + np.sin(3 * np.pi * h) ** 2)
    assert rel(v1, mult * v) < 1e-12


# ------------------------------------------------------------------ reconstruction

def test_reconstruct_matches_value_channel():
    spec = gen.DecoderSpec(2, 3, 16, 2)
    dec = O.MLPDecoder(gen.xavier_decoder(spec, seed=2, bias_std=0.1), 2)
    X = gen.grid_points_2d(9)
    codes = np.random.default_rng(1).standard_normal((3, 3))
    R = O.reconstruct(dec, codes, X)
    for c in range(3):
        np.testing.assert_allclose(R[c], dec(X, codes[c]).g, rtol=1e-13, atol=1e-15)


# ------------------------------------------------------------------ f3: spatially varying nu(x)

def test_fom_heat1d_field_energy_balance():
    """u_t = nu(x) u_xx (App. G) with nu piecewise constant over 3 regions: the
    discrete heat content sum_i u_i / nu_i changes by exactly dt/dx^2 times the
    boundary fluxes -(u_1 + u_{P-2}) per step (interior telescoping sum with
    Dirichlet-0 ends): stored energy + escaped energy = total, step by step."""
    P = 201
    dx = 1 / (P - 1)
    x = np.arange(P) * dx
    nu = gen.piecewise_nu(x[:, None], [0.2, 1.0, 0.6]).astype(np.float64)
    _, u = gen.sine_modes_1d(P, np.random.default_rng(5))
    dt = dx ** 2 / 4
    for _ in range(60):
        v = O.fom_heat1d_step(u, dt, nu)
        stored = np.sum((v[1:-1] - u[1:-1]) / nu[1:-1])
        escaped = -dt / dx ** 2 * (u[1] + u[-2])
        assert abs(stored - escaped) < 1e-11 * (abs(escaped) + np.sum(np.abs(u)))
        u = v


def test_fom_heat_field_domain_of_dependence():
    """A bump inside one region evolves exactly as with that region's constant nu
    while its support (one node per step) stays inside the region."""
    P = 301
    dx = 1 / (P - 1)
    x = np.arange(P) * dx
    nu = gen.piecewise_nu(x[:, None], [0.3, 0.9, 0.5]).astype(np.float64)
    u0 = np.where(np.abs(x - 0.5) < 0.05, np.cos((x - 0.5) / 0.05 * np.pi / 2) ** 2, 0.0)
    dt = dx ** 2 / 4
    a, b = u0.copy(), u0.copy()
    for _ in range(20):   # support grows from |x - 0.5| < 0.05 by 20 dx = 0.067 < 1/6 - 0.05
        a = O.fom_heat1d_step(a, dt, nu)
        b = O.fom_heat1d_step(b, dt, nu[P // 2])   # the middle region's value
    assert np.array_equal(a, b)
    # 2D Neumann with a 4-region field: trapezoid-weighted sum of u / nu is conserved
    n = 48
    h = 1 / (n - 1)
    t = np.arange(n) * h
    X1, X2 = np.meshgrid(t, t, indexing="ij")
    nu2 = gen.piecewise_nu(np.stack([X1.ravel(), X2.ravel()], 1), [0.2, 0.0, 0.2, 0.1]).reshape(n, n).astype(np.float64)
    nu2 = np.where(nu2 == 0, 1.0, nu2)   # a zero region has no heat capacity weight; use 1 there (u unchanged)
    w = np.ones(n); w[0] = w[-1] = 0.5
    W = np.outer(w, w)
    v = gen.gaussian_bumps_2d(n, np.random.default_rng(6))
    m0 = np.sum(W * v / nu2)
    for _ in range(30):
        v = O.fom_heat2d_neumann_step(v, h ** 2 / 8, nu2)
    assert abs(np.sum(W * v / nu2) - m0) < 1e-12 * abs(m0)


def test_step_per_sample_coefficient_sine_decoder():
    """Per-sample nu(y_j) in the latent step: for the sine decoder (linear in q) the
    step is q_n + argmin ||S d - dt nu .* Lap g||, with S and Lap g written from the
    sine formulas here (one GN iteration is exact; a second leaves q unchanged)."""
    r = 4
    dec = FourierDecoder1D(r)
    Y = (np.arange(1, 16) / 16.0)[:, None]
    nu = gen.piecewise_nu(Y, [0.2, 1.0, 0.5]).astype(np.float64)
    q0 = np.random.default_rng(8).standard_normal(r)
    dt = 1e-4
    k = np.arange(1, r + 1)
    S = np.sin(np.pi * np.outer(Y[:, 0], k))
    lap = -(S * (np.pi * k) ** 2) @ q0
    d_ref = np.linalg.lstsq(S, dt * nu * lap, rcond=None)[0]
    for gn in (1, 2):
        q1, st = O.crom_step(dec, q0, Y, dt, gn, alpha=nu)
        assert st == O.STATUS_OK and rel(q1 - q0, d_ref) < 1e-10
    # the region values matter: constant nu = 1 gives a different step
    q_const, _ = O.crom_step(dec, q0, Y, dt, 1, alpha=1.0)
    assert rel(q_const - q0, d_ref) > 0.1




def test_fom_advdiff_central_fourier_multiplier():
    """Central fluxes under a uniform velocity: the real Fourier mode
    cos(th_x i + th_y j + phi) is an eigenvector of one step with the complex
    multiplier mu = 1 - dt [i (a_x sin th_x + a_y sin th_y) / h
    + 4 nu (sin^2(th_x / 2) + sin^2(th_y / 2)) / h^2]; after s steps the mode is
    |mu|^s cos(. + s arg mu).  Upwinding, a dropped term or a sign flip fails it."""
    n, ax, ay, nu, dt, steps = 32, 0.7, -0.4, 2e-3, 2e-3, 25
    h = 1.0 / n
    kx, ky, phi = 3, 5, 0.3
    tx, ty = 2 * np.pi * kx / n, 2 * np.pi * ky / n
    I, J = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    u = np.cos(tx * I + ty * J + phi)
    axf, ayf = np.full((n, n), ax), np.full((n, n), ay)
    for _ in range(steps):
        u = O.fom_advdiff2d_step(u, axf, ayf, nu, dt, scheme="central")
    mu = 1 - dt * (1j * (ax * np.sin(tx) + ay * np.sin(ty)) / h
                   + 4 * nu * (np.sin(tx / 2) ** 2 + np.sin(ty / 2) ** 2) / h ** 2)
    ref = np.abs(mu) ** steps * np.cos(tx * I + ty * J + phi + steps * np.angle(mu))
    assert np.max(np.abs(u - ref)) < 1e-12
    # the upwind scheme damps the same mode more (its numerical diffusion)
    v = np.cos(tx * I + ty * J + phi)
    for _ in range(steps):
        v = O.fom_advdiff2d_step(v, axf, ayf, nu, dt)
    assert np.linalg.norm(v) < np.linalg.norm(u) * 0.99


@pytest.mark.parametrize("per_sample", [False, True])
def test_step_batched_closed_form_per_instance(per_sample):
    """crom_step_batched against the sine decoder's least-squares closed form, one
    instance at a time: uneven sizes in no particular order (a larger instance after
    a smaller one, one at |M| = r, one below r), each instance with its own samples,
    q_n and coefficient.  With per-sample coefficients every sample has a different
    nu(y_j), so handing an instance its neighbour's samples or coefficients, or
    indexing the coefficient by instance, changes the step."""
    r = 4
    dec = FourierDecoder1D(r)
    rng = np.random.default_rng(21)
    sizes = [9, 15, r, 2, 11]
    Ys = [np.sort(rng.uniform(0.02, 0.98, size=n))[:, None] for n in sizes]
    samples = np.concatenate(Ys)
    off = gen.ragged_offsets(sizes)
    q = rng.standard_normal((len(sizes), r))
    dt = 1e-4
    alpha = rng.uniform(0.2, 1.0, size=samples.shape[0] if per_sample else len(sizes))
    got, st = O.crom_step_batched(dec, q, off, samples, alpha, dt, 1, alpha_per_sample=per_sample)
    k = np.arange(1, r + 1)
    for i, Y in enumerate(Ys):
        if sizes[i] < r:
            assert st[i] == O.STATUS_BAD_ARG and np.array_equal(got[i], q[i])
            continue
        nu = alpha[off[i]:off[i + 1]] if per_sample else alpha[i]
        S = np.sin(np.pi * np.outer(Y[:, 0], k))
        lap = -(S * (np.pi * k) ** 2) @ q[i]
        d_ref = np.linalg.lstsq(S, dt * nu * lap, rcond=None)[0]
        assert st[i] == O.STATUS_OK
        assert rel(got[i] - q[i], d_ref) < 1e-10, i


# ------------------------------------------------------------------ f1: backtracking line search

class CubicDecoder:
    """g(x, q) = q^3 + c x^2 (r = 1, m = 1): Lap g = 2c, dg/dq = 3 q^2 - a toy
    nonlinearity whose Gauss-Newton steps can be followed by hand."""

    def __init__(self, c):
        self.c = c

    def __call__(self, X, q):
        x = np.asarray(X, np.float64)[:, 0]
        q0 = float(np.asarray(q)[0])
        g = q0 ** 3 + self.c * x ** 2
        return O.Evaluation(g, (2 * self.c * x)[:, None], np.full((x.size, 1), 2 * self.c),
                            np.full((x.size, 1), 3 * q0 ** 2))


def test_line_search_by_hand_on_cubic():
    """q_n = 1, Delta f = 2 dt alpha c = 9: the residual is rho(q) = q^3 - 10 at every
    sample.  GN: delta = 3; a = 1 gives q = 4, rho = 54 (phi grows): rejected;
    a = 1/2 gives q = 2.5, rho = 5.625: accepted.  Next: delta = -5.625/18.75 = -0.3,
    accepted at a = 1, q = 2.2.  Without the line search: q = 4, then 4 - 54/48."""
    dec = CubicDecoder(4.5)
    Y = np.linspace(0.1, 0.9, 7)[:, None]
    q, st, info = O.crom_step(dec, [1.0], Y, 1.0, 1, alpha=1.0, line_search=3, return_info=True)
    assert st == O.STATUS_OK and q[0] == 2.5
    assert [t[0] for t in info["line_search_trials"][0]] == [1.0, 0.5]
    q, st = O.crom_step(dec, [1.0], Y, 1.0, 2, alpha=1.0, line_search=3)
    assert abs(q[0] - 2.2) < 1e-14
    q, st = O.crom_step(dec, [1.0], Y, 1.0, 2, alpha=1.0, line_search=0)
    assert q[0] == 4.0 - 54.0 / 48.0
    # no acceptable length among a = 1, 1/2 (target 1000): q stays, iterations stop
    dec2 = CubicDecoder(499.5)
    q, st, info = O.crom_step(dec2, [1.0], Y, 1.0, 3, alpha=1.0, line_search=1, return_info=True)
    assert st == O.STATUS_OK and q[0] == 1.0 and len(info["line_search_trials"]) == 1


def test_line_search_accepts_full_step_for_linear_decoders():
    """For a decoder linear in q the objective is quadratic and the GN step is its
    exact minimiser, phi(q + delta) = phi(q) + v.delta / 2 <= phi(q) + c1 v.delta:
    the line search takes a = 1 in the first iteration.  Later iterations start at
    the minimiser, where delta and the decrease are rounding noise: they may stop
    the search, which leaves q at the minimiser."""
    dec = FourierDecoder1D(5, offset=True)
    Y = (np.arange(1, 14) / 14.0)[:, None]
    q0 = np.random.default_rng(11).standard_normal(5)
    a, sa = O.crom_step(dec, q0, Y, 1e-3, 3, alpha=0.7, line_search=0)
    b, sb, info = O.crom_step(dec, q0, Y, 1e-3, 3, alpha=0.7, line_search=4, return_info=True)
    assert sa == sb == O.STATUS_OK and rel(b - q0, a - q0) < 1e-12
    first = info["line_search_trials"][0]
    assert len(first) == 1 and first[0][0] == 1.0


# ------------------------------------------------------------------ f4: SIREN decoders

def test_siren_decoder_derivatives_vs_autodiff_and_closed_form():
    """SIREN (sin(30 z)) hidden layers: every channel against reverse-mode autodiff
    of an independently written torch FP64 forward pass; a one-hidden-layer decoder
    against its closed form Lap g = -w0^2 sum_u w_u |a_u|^2 sin(w0 z_u)."""
    torch = pytest.importorskip("torch")
    spec = gen.DecoderSpec(2, 4, 32, 3)
    params = gen.siren_decoder(spec, seed=5)
    dec = O.MLPDecoder(params, 2, activation="siren")
    rng = np.random.default_rng(6)
    X = rng.uniform(-1, 1, size=(8, 2))
    q = rng.standard_normal(4)
    ev = dec(X, q)
    Wt = [(torch.tensor(W), torch.tensor(b)) for W, b in params]

    def f(xq):
        h = xq
        for li, (W, b) in enumerate(Wt):
            z = W @ h + b
            h = torch.sin(30.0 * z) if li + 1 < len(Wt) else z
        return h[0]

    for i in range(X.shape[0]):
        xq = torch.tensor(np.concatenate([X[i], q]), requires_grad=True)
        grad = torch.autograd.functional.jacobian(f, xq).numpy()
        hess = torch.autograd.functional.hessian(f, xq).numpy()
        np.testing.assert_allclose(ev.g[i], f(xq).item(), rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(ev.gx[i], grad[:2], rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(ev.gq[i], grad[2:], rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(ev.gxx[i], np.diag(hess)[:2], rtol=1e-10, atol=1e-10)
    # one hidden layer: closed forms
    spec1 = gen.DecoderSpec(2, 3, 16, 1)
    (W1, b1), (Wo, bo) = gen.siren_decoder(spec1, seed=7)
    dec1 = O.MLPDecoder([(W1, b1), (Wo, bo)], 2, activation="siren")
    ev1 = dec1(X, q[:3])
    z = X @ W1[:, :2].T + q[:3] @ W1[:, 2:].T + b1
    w = Wo[0]
    np.testing.assert_allclose(ev1.g, np.sin(30 * z) @ w + bo[0], rtol=1e-13, atol=1e-14)
    lap = -900.0 * (np.sin(30 * z) * (W1[:, 0] ** 2 + W1[:, 1] ** 2)) @ w
    np.testing.assert_allclose(ev1.lap, lap, rtol=1e-12, atol=1e-12)
    gq = 30.0 * (np.cos(30 * z) * w) @ W1[:, 2:]
    np.testing.assert_allclose(ev1.gq, gq, rtol=1e-12, atol=1e-12)


def test_tangent_velocity_closed_form_and_difference_quotient():
    """v = dg/dq . (q_n - q_{n-1}) / dt: exact for a decoder linear in q (the sine
    decoder: v = sum_k qdot_k sin(k pi x)); for an MLP it is the limit of the
    difference quotient (g(x, q_n) - g(x, q_n - eps qdot dt)) / (eps dt)."""
    dec = FourierDecoder1D(4)
    X = np.linspace(0.05, 0.95, 11)[:, None]
    rng = np.random.default_rng(13)
    q, qp = rng.standard_normal(4), rng.standard_normal(4)
    v = O.tangent_velocity(dec, X, q, qp, 0.01)
    S = np.sin(np.pi * np.outer(X[:, 0], np.arange(1, 5)))
    assert rel(v, S @ ((q - qp) / 0.01)) < 1e-14
    spec = gen.DecoderSpec(2, 3, 32, 3)
    mlp = O.MLPDecoder(gen.xavier_decoder(spec, seed=2, bias_std=0.2), 2)
    X2 = rng.uniform(0, 1, size=(40, 2))
    q, qp = rng.standard_normal(3), rng.standard_normal(3)
    dt, eps = 0.1, 1e-6
    v = O.tangent_velocity(mlp, X2, q, qp, dt)
    qdot = (q - qp) / dt
    fd = (mlp.value(X2, q + eps * qdot) - mlp.value(X2, q - eps * qdot)) / (2 * eps)
    keep = _kink_margin(mlp.params, X2, q[None, :], 2) > 1e-4   # ELU is C^1: stay off kinks
    assert rel(v[keep], fd[keep]) < 1e-7
