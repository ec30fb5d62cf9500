"""GPU full-order models (crom_fom_step) against the FP64 oracle's FOMs and the
closed forms that pin them (discrete sine / cosine eigenmodes, conservation,
Courant-1 translation).  FP32 arithmetic over <= 200 steps: relative L2 <= 1e-5
against the oracle, invariants to FP32 round-off."""
import numpy as np
import pytest

from oracle import crom_oracle as O
from workloads import gen

from helpers import dev, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c():
    from paper_2206_02607_gb300 import build
    build()
    from paper_2206_02607_gb300 import crom
    return crom


def run(c, kind, u0, coef, dt, n, ax=None, ay=None):
    import torch
    u = dev(u0, torch.float32)
    tmp = torch.empty_like(u)
    c.crom_fom_step(kind, u, tmp, dev(coef, torch.float32), dt=dt, n_steps=n,
                    ax=None if ax is None else dev(ax, torch.float32), ay=None if ay is None else dev(ay, torch.float32))
    torch.cuda.synchronize()
    return u.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("steps", [1, 7, 100])
def test_heat1d_matches_oracle_and_eigenmodes(c, steps):
    P = 256
    dx = 1 / (P - 1)
    rng = np.random.default_rng(1)
    batch = []
    for b in range(5):
        a, u0 = gen.sine_modes_1d(P, rng)
        batch.append(u0)
    u0 = np.stack(batch)
    nu = np.array([1.0, 0.5, 0.2, 0.8, 1.0])
    dt = dx ** 2 / 4
    got = run(c, c.CROM_FOM_HEAT1D_DIRICHLET, u0, nu, dt, steps)
    for b in range(5):
        ref = u0[b].astype(np.float32).astype(np.float64)
        for _ in range(steps):
            ref = O.fom_heat1d_step(ref, dt, nu[b])
        assert rel_l2(got[b], ref) < 1e-5
        assert got[b, 0] == 0.0 and got[b, -1] == 0.0


def test_heat2d_neumann_matches_oracle_and_conserves_mass(c):
    n = 128
    h = 1 / (n - 1)
    rng = np.random.default_rng(3)
    u0 = np.stack([gen.gaussian_bumps_2d(n, rng) for _ in range(3)])
    alpha = np.array([1.0, 0.5, 2.0])
    dt = h * h / 8 / 2.0
    got = run(c, c.CROM_FOM_HEAT2D_NEUMANN, u0, alpha, dt, 50)
    w = np.ones(n); w[0] = w[-1] = 0.5
    W = np.outer(w, w)
    for b in range(3):
        ref = u0[b].astype(np.float32).astype(np.float64)
        for _ in range(50):
            ref = O.fom_heat2d_neumann_step(ref, dt, alpha[b])
        assert rel_l2(got[b], ref) < 1e-5
        m0 = np.sum(W * u0[b].astype(np.float32))
        assert abs(np.sum(W * got[b]) - m0) < 2e-5 * abs(m0)


@pytest.mark.parametrize("n", [64, 256])   # 256: the four-columns-per-lane marching kernel
def test_heat2d_neumann_cosine_mode_closed_form(c, n):
    h = 1 / (n - 1)
    t = np.arange(n) * h
    X1, X2 = np.meshgrid(t, t, indexing="ij")
    k, l = 2, 3
    u0 = (np.cos(k * np.pi * X1) * np.cos(l * np.pi * X2))[None]
    dt, steps = h * h / 8, 40
    got = run(c, c.CROM_FOM_HEAT2D_NEUMANN, u0, np.array([1.0]), dt, steps)
    mult = 1 - 4 * dt / h ** 2 * (np.sin(k * np.pi * h / 2) ** 2 + np.sin(l * np.pi * h / 2) ** 2)
    assert rel_l2(got[0], u0[0] * mult ** steps) < 1e-5


def _faces(n, rng, nb):
    ax, ay = [], []
    h = 1 / n
    for _ in range(nb):
        psi = rng.standard_normal((n, n)) * 0.05
        ax.append((psi - np.roll(psi, 1, axis=1)) / h)
        ay.append(-(psi - np.roll(psi, 1, axis=0)) / h)
    return np.stack(ax), np.stack(ay)


@pytest.mark.parametrize("n", [96, 128, 256])   # 128 and 256: the marching kernel (n % 128 == 0)
def test_advdiff_matches_oracle_conserves_mass_and_translates(c, n):
    h = 1 / n
    rng = np.random.default_rng(9)
    ax, ay = _faces(n, rng, 2)
    ax, ay = ax.astype(np.float32), ay.astype(np.float32)
    u0 = rng.uniform(0, 1, size=(2, n, n))
    nu = np.array([1e-3, 5e-3])
    amax = max(np.abs(ax).max(), np.abs(ay).max())
    dt = 0.2 * min(h / amax, h * h / (4 * nu.max()))
    got = run(c, c.CROM_FOM_ADVDIFF2D_PERIODIC, u0, nu, dt, 30, ax, ay)
    for b in range(2):
        ref = u0[b].astype(np.float32).astype(np.float64)
        for _ in range(30):
            ref = O.fom_advdiff2d_step(ref, ax[b].astype(np.float64), ay[b].astype(np.float64), nu[b], dt)
        assert rel_l2(got[b], ref) < 1e-5
        m0 = u0[b].astype(np.float32).astype(np.float64).sum()
        assert abs(got[b].sum() - m0) < 1e-5 * m0
    # Courant number 1 with a uniform velocity is an exact one-cell shift
    a = 2.0
    u1 = rng.uniform(size=(1, 16, 16)).astype(np.float32)
    got = run(c, c.CROM_FOM_ADVDIFF2D_PERIODIC, u1, np.array([0.0]), (1 / 16) / a, 1,
              np.full((1, 16, 16), a, np.float32), np.zeros((1, 16, 16), np.float32))
    np.testing.assert_allclose(got[0], np.roll(u1[0], 1, axis=0), rtol=0, atol=1e-6)
    # ... in both directions on the marching kernel's grid (lane-to-lane and halo neighbours)
    u2 = rng.uniform(size=(2, 128, 128)).astype(np.float32)
    vx = np.stack([np.full((128, 128), a, np.float32), np.zeros((128, 128), np.float32)])
    vy = np.stack([np.zeros((128, 128), np.float32), np.full((128, 128), -a, np.float32)])
    got = run(c, c.CROM_FOM_ADVDIFF2D_PERIODIC, u2, np.array([0.0, 0.0]), (1 / 128) / a, 1, vx, vy)
    np.testing.assert_allclose(got[0], np.roll(u2[0], 1, axis=0), rtol=0, atol=1e-6)
    np.testing.assert_allclose(got[1], np.roll(u2[1], -1, axis=1), rtol=0, atol=1e-6)



@pytest.mark.parametrize("n", [96, 128, 256])
def test_advdiff_central_matches_oracle_and_conserves_mass(c, n):
    """The second-order (central-flux) advection-diffusion model against the oracle's
    central scheme; dt within both forward-Euler limits, (a dt/h)^2 <= 2 nu dt/h^2
    and nu dt/h^2 <= 1/4, so FP32 and FP64 stay together over the steps."""
    h = 1 / n
    rng = np.random.default_rng(19)
    ax, ay = _faces(n, rng, 2)
    ax, ay = ax.astype(np.float32), ay.astype(np.float32)
    u0 = rng.uniform(0, 1, size=(2, n, n))
    nu = np.array([2e-3, 5e-3])
    amax = max(np.abs(ax).max(), np.abs(ay).max())
    dt = 0.5 * min(2 * nu.min() / amax ** 2, h * h / (4 * nu.max()))
    got = run(c, c.CROM_FOM_ADVDIFF2D_PERIODIC_CENTRAL, u0, nu, dt, 30, ax, ay)
    for b in range(2):
        ref = u0[b].astype(np.float32).astype(np.float64)
        for _ in range(30):
            ref = O.fom_advdiff2d_step(ref, ax[b].astype(np.float64), ay[b].astype(np.float64), nu[b], dt,
                                       scheme="central")
        assert rel_l2(got[b], ref) < 1e-5
        m0 = u0[b].astype(np.float32).astype(np.float64).sum()
        assert abs(got[b].sum() - m0) < 1e-5 * m0


def test_fom_rejects_bad_arguments(c):
    import torch
    u = torch.zeros((1, 8, 8), device="cuda")
    for kw in [dict(dt=0.0, n_steps=1), dict(dt=1e-3, n_steps=-1)]:
        with pytest.raises(c.CromError):
            c.crom_fom_step(c.CROM_FOM_HEAT2D_NEUMANN, u, torch.zeros_like(u), torch.ones(1, device="cuda"), **kw)
    with pytest.raises(c.CromError):   # advection without velocities
        c.crom_fom_step(c.CROM_FOM_ADVDIFF2D_PERIODIC, u, torch.zeros_like(u), torch.ones(1, device="cuda"),
                        dt=1e-3, n_steps=1)
    with pytest.raises(c.CromError):   # 1D kind with a 2D field
        c.crom_fom_step(c.CROM_FOM_HEAT1D_DIRICHLET, u, torch.zeros_like(u), torch.ones(1, device="cuda"),
                        dt=1e-3, n_steps=1)


@pytest.mark.parametrize("kind", ["heat", "heat_field", "advdiff", "advdiff_central"])
def test_marching_kernels_match_unaligned_fallback(c, kind):
    """Sides that are multiples of 128 with 16-byte aligned arrays take the
    four-columns-per-lane marching kernels; the same fields placed one float off
    alignment take the scalar kernels.  Both evaluate the same stencil expression, so
    the results agree to FP32 rounding (and every value of both is finite)."""
    import torch
    n, nb, steps = 256, 3, 5
    rng = np.random.default_rng(12)
    u0 = rng.uniform(size=(nb, n, n)).astype(np.float32)
    h = 1 / (n - 1)
    if kind.startswith("advdiff"):
        ax, ay = _faces(n, rng, nb)
        ax, ay = ax.astype(np.float32), ay.astype(np.float32)
        coef = np.array([1e-3, 5e-3, 2e-3], np.float32)
        dt = 0.2 * min((1 / n) / max(np.abs(ax).max(), np.abs(ay).max()), (1 / n) ** 2 / (4 * 5e-3))
        k = c.CROM_FOM_ADVDIFF2D_PERIODIC if kind == "advdiff" else c.CROM_FOM_ADVDIFF2D_PERIODIC_CENTRAL
    else:
        ax = ay = None
        coef = (rng.uniform(0.2, 1.0, size=(nb, n, n)) if kind == "heat_field" else np.array([1.0, 0.5, 2.0]))
        coef = coef.astype(np.float32)
        dt = h * h / 8 / 2.0
        k = c.CROM_FOM_HEAT2D_NEUMANN_FIELD if kind == "heat_field" else c.CROM_FOM_HEAT2D_NEUMANN

    def place(a, off):
        buf = torch.zeros(a.size + off, dtype=torch.float32, device="cuda")
        v = buf[off:].view(a.shape)
        v.copy_(torch.from_numpy(np.ascontiguousarray(a)).cuda())
        return v

    def go(off):
        u = place(u0, off)
        tmp = place(np.zeros_like(u0), off)
        cf = place(coef, off) if kind == "heat_field" else dev(coef, torch.float32)
        c.crom_fom_step(k, u, tmp, cf, dt=dt, n_steps=steps,
                        ax=None if ax is None else place(ax, off), ay=None if ay is None else place(ay, off))
        torch.cuda.synchronize()
        return u.cpu().numpy().astype(np.float64)

    fast, slow = go(0), go(1)
    assert np.all(np.isfinite(fast)) and np.all(np.isfinite(slow))
    assert rel_l2(fast, slow) < 1e-6


@pytest.mark.parametrize("kind", ["advdiff", "heat"])
def test_bench_size_fields_sampled(c, kind):
    """The bench's full-order launches (512 periodic 256^2 fields with face velocities,
    1024 zero-flux 256^2 fields), two steps; four fields (first, last, two inside) are
    recomputed by the oracle and every value of every field must be finite."""
    import torch
    n = 256
    nb = 512 if kind == "advdiff" else 1024
    rng = np.random.default_rng(0)
    u0 = rng.uniform(0, 1, size=(nb, n, n)).astype(np.float32)
    u = dev(u0, torch.float32)
    tmp = torch.empty_like(u)
    if kind == "advdiff":
        ax = rng.uniform(-0.5, 0.5, size=(nb, n, n)).astype(np.float32)
        ay = rng.uniform(-0.5, 0.5, size=(nb, n, n)).astype(np.float32)
        nu, dt = 5e-3, 2.5e-5
        c.crom_fom_step(c.CROM_FOM_ADVDIFF2D_PERIODIC, u, tmp, torch.full((nb,), nu, device="cuda"), dt=dt, n_steps=2,
                        ax=dev(ax, torch.float32), ay=dev(ay, torch.float32))
    else:
        nu, dt = 1.0, (1 / (n - 1)) ** 2 / 8
        c.crom_fom_step(c.CROM_FOM_HEAT2D_NEUMANN, u, tmp, torch.full((nb,), nu, device="cuda"), dt=dt, n_steps=2)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(u).all().item())
    for b in (0, 1, nb // 2 + 3, nb - 1):
        ref = u0[b].astype(np.float64)
        for _ in range(2):
            if kind == "advdiff":
                ref = O.fom_advdiff2d_step(ref, ax[b].astype(np.float64), ay[b].astype(np.float64), nu, dt)
            else:
                ref = O.fom_heat2d_neumann_step(ref, dt, nu)
        assert rel_l2(u[b].cpu().numpy().astype(np.float64), ref) < 1e-6, b
