"""Spatially varying coefficient nu(x) (u_t = nu(x) Lap u, paper App. G and H):
the latent step with one coefficient per integration sample (FP32 and BF16X2
paths) and the full-order heat models with a per-node coefficient field, against
the FP64 oracle."""
import numpy as np
import pytest

from oracle import crom_oracle as O
from workloads import gen

from helpers import StepInputs, dev, increment_errors, make_ctx, rel_l2

pytestmark = pytest.mark.gpu

NU_REGIONS = [0.2, 1.0, 0.5, 0.0]   # four equal-width regions along x_1, one without diffusion


@pytest.fixture(scope="module")
def c():
    from paper_2206_02607_gb300 import build
    build()
    from paper_2206_02607_gb300 import crom
    return crom


def _step(c, w, alpha, per_sample, prec):
    import torch
    d = StepInputs(w)
    c.crom_step(make_ctx(w.spec, w.params), d.q, dev(alpha, torch.float32), d.s_off, d.samples, d.status,
                dt=w.dt, gn_iters=w.gn_iters, max_samples=d.max_samples, precision=prec,
                coef_per_sample=per_sample)
    torch.cuda.synchronize()
    return d.q.cpu().numpy(), d.status.cpu().numpy()


# res: ||J (d_gpu - d_ref)|| / ||Delta f||; F16X2 rounds the hidden weights to f16, which moves the
# network Laplacian (two digits of cancellation in the output layer) and so the fit by up to ~10 %
@pytest.mark.parametrize("prec_name,res_tol", [("CROM_PREC_FP32", 2e-4), ("CROM_PREC_F16X2", 0.15)])
def test_step_per_sample_coefficient_matches_oracle(c, prec_name, res_tol):
    w = gen.heat2d_batched(n_inst=10, m_lo=16, m_hi=300, bias_std=0.1)
    nu = gen.piecewise_nu(w.samples, NU_REGIONS)
    q1, st = _step(c, w, nu, True, getattr(c, prec_name))
    ref, rst = O.crom_step_batched(O.MLPDecoder(w.params, 2), w.q0, w.s_off, w.samples, nu, w.dt, w.gn_iters,
                                   alpha_per_sample=True)
    assert np.array_equal(st, rst)
    for i in range(w.n_inst):
        Y = w.samples[w.s_off[i]:w.s_off[i + 1]]
        nu_i = nu[w.s_off[i]:w.s_off[i + 1]]
        assert rel_l2(q1[i], ref[i]) < (1e-5 if prec_name == "CROM_PREC_FP32" else 5e-5)
        if np.all(nu_i == 0):
            assert np.array_equal(q1[i], w.q0[i])
            continue
        inc, res, kappa, margin = increment_errors(w.params, 2, w.q0[i], Y, q1[i], ref[i], w.dt, nu_i)
        assert res < (res_tol if margin > 1e-4 else max(res_tol, 5e-2)), (i, inc, res, kappa, margin)


@pytest.mark.parametrize("prec_name", ["CROM_PREC_FP32", "CROM_PREC_F16X2", "CROM_PREC_F16"])
def test_per_sample_coefficient_equal_to_instance_value_is_the_same_step(c, prec_name):
    """nu(y_j) = alpha_i at every sample of instance i reproduces the per-instance
    step bit for bit (same arithmetic, coefficient read from another index)."""
    w = gen.heat2d_batched(n_inst=7, m_lo=20, m_hi=200)
    prec = getattr(c, prec_name)
    per_sample = np.repeat(w.alpha, w.sizes).astype(np.float32)
    qa, sa = _step(c, w, w.alpha, False, prec)
    qb, sb = _step(c, w, per_sample, True, prec)
    assert np.array_equal(sa, sb) and np.array_equal(qa, qb)


def test_step_rejects_bad_coefficient_mode(c):
    import ctypes
    w = gen.heat2d_batched(n_inst=2, m_lo=20, m_hi=30)
    ctx = make_ctx(w.spec, w.params)
    d = StepInputs(w)
    desc = c.crom_step_desc(c.CROM_PDE_HEAT, 1, 1e-5, 2, 0)   # coef_per_sample = 2 is invalid
    rc = c.raw_call("crom_step", ctx.handle, ctypes.byref(desc), c.CROM_PREC_FP32, w.n_inst, d.q.data_ptr(),
                    d.alpha.data_ptr(), None, d.s_off.data_ptr(), d.samples.data_ptr(), int(w.sizes.sum()),
                    d.max_samples, d.status.data_ptr(), None)
    assert rc == c.CROM_ERR_INVALID_ARG and "coef_per_sample" in c.last_error()


def test_fom_heat_field_kinds_match_oracle(c):
    import torch
    # 1D thermodynamics: 3 regions of nu in [0.2, 1], 501 nodes (App. G)
    P = 501
    dx = 1 / (P - 1)
    x = (np.arange(P) * dx)[:, None]
    rng = np.random.default_rng(2)
    values = rng.uniform(0.2, 1.0, size=(4, 3))
    u0 = np.stack([gen.sine_modes_1d(P, rng)[1] for _ in range(4)])
    nu = np.stack([gen.piecewise_nu(x, v) for v in values])
    dt = dx ** 2 / 4
    u = dev(u0, torch.float32)
    c.crom_fom_step(c.CROM_FOM_HEAT1D_DIRICHLET_FIELD, u, torch.empty_like(u), dev(nu, torch.float32), dt=dt,
                    n_steps=50)
    got = u.cpu().numpy()
    for b in range(4):
        ref = u0[b].astype(np.float32).astype(np.float64)
        for _ in range(50):
            ref = O.fom_heat1d_step(ref, dt, nu[b].astype(np.float64))
        assert rel_l2(got[b], ref) < 1e-5
    # 2D image diffusion: 4 regions, nu in {0, 0.2} (App. H)
    n = 128
    h = 1 / (n - 1)
    t = np.arange(n) * h
    X1, X2 = np.meshgrid(t, t, indexing="ij")
    pts = np.stack([X1.ravel(), X2.ravel()], 1)
    vals = [[0.2, 0.0, 0.2, 0.2], [0.0, 0.2, 0.0, 0.2]]
    nu2 = np.stack([gen.piecewise_nu(pts, v).reshape(n, n) for v in vals])
    u0 = np.stack([gen.gaussian_bumps_2d(n, rng) for _ in range(2)])
    dt = h ** 2 / 8
    u = dev(u0, torch.float32)
    c.crom_fom_step(c.CROM_FOM_HEAT2D_NEUMANN_FIELD, u, torch.empty_like(u), dev(nu2, torch.float32), dt=dt,
                    n_steps=20)
    got = u.cpu().numpy()
    for b in range(2):
        ref = u0[b].astype(np.float32).astype(np.float64)
        for _ in range(20):
            ref = O.fom_heat2d_neumann_step(ref, dt, nu2[b].astype(np.float64))
        assert rel_l2(got[b], ref) < 1e-5
        frozen = (nu2[b] == 0)
        # nodes of a region without diffusion keep their values exactly
        assert np.array_equal(got[b][frozen], u0[b].astype(np.float32)[frozen])
