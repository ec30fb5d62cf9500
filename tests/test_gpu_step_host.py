"""crom_step_host: the latent step (paper §4, Algorithm 3) on host arrays.  It must
equal crom_step on device copies of the same arrays bit for bit (the same kernels
run on the same values), for both step precisions, from pinned and from pageable
host memory, on consecutive calls whose batch grows (the staging buffer is reused,
then enlarged); bad offsets are rejected on the host before anything runs."""
import numpy as np
import pytest

from workloads import gen

from helpers import StepInputs, make_ctx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c():
    from paper_2206_02607_gb300 import build
    build()
    from paper_2206_02607_gb300 import crom
    return crom


def _host(a, dtype, pinned):
    import torch
    t = torch.tensor(np.ascontiguousarray(a), dtype=dtype)
    return t.pin_memory() if pinned else t


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("prec_name", ["CROM_PREC_FP32", "CROM_PREC_F16X2"])
def test_step_host_equals_device_step(c, prec_name, pinned):
    import torch
    prec = getattr(c, prec_name)
    w0 = gen.heat2d_batched(n_inst=64, m_lo=16, m_hi=300)
    ctx = make_ctx(w0.spec, w0.params)
    for n in (24, 64):  # the second batch is larger: the staging buffer grows
        idx = np.arange(n)
        sizes = w0.sizes[idx]
        samples = np.concatenate([w0.samples[w0.s_off[i]:w0.s_off[i + 1]] for i in idx])
        w = gen.StepWorkload("host", w0.spec, w0.params, w0.q0[idx], w0.alpha[idx], gen.ragged_offsets(sizes),
                             samples, w0.dt, w0.gn_iters, 1)
        d = StepInputs(w)
        c.crom_step(ctx, d.q, d.alpha, d.s_off, d.samples, d.status, dt=w.dt, gn_iters=w.gn_iters,
                    max_samples=d.max_samples, precision=prec)
        torch.cuda.synchronize()
        hq = _host(w.q0, torch.float64, pinned)
        hst = _host(np.full(n, -1, np.int32), torch.int32, pinned)
        c.crom_step_host(ctx, hq, _host(w.alpha, torch.float32, pinned), _host(w.s_off, torch.int32, pinned),
                         _host(w.samples, torch.float32, pinned), hst, dt=w.dt, gn_iters=w.gn_iters,
                         max_samples=d.max_samples, precision=prec)
        assert np.array_equal(hst.numpy(), d.status.cpu().numpy())
        assert np.array_equal(hq.numpy(), d.q.cpu().numpy())
        assert np.all(hst.numpy() == c.CROM_OK)


def test_step_host_rejects_bad_offsets(c):
    import torch
    w = gen.heat2d_batched(n_inst=3, m_lo=20, m_hi=40)
    ctx = make_ctx(w.spec, w.params)
    good = w.s_off.astype(np.int32)
    swapped = good.copy()
    swapped[[1, 2]] = swapped[[2, 1]]  # decreasing in the middle, correct ends
    bad = [good + 1, swapped, np.concatenate([good[:-1], [good[-1] - 1]]).astype(np.int32)]
    for off in bad:
        hq = torch.tensor(w.q0)
        with pytest.raises(c.CromError) as e:
            c.crom_step_host(ctx, hq, torch.tensor(w.alpha), torch.tensor(off), torch.tensor(w.samples),
                             torch.zeros(3, dtype=torch.int32), dt=w.dt, gn_iters=2, max_samples=64)
        assert e.value.code == c.CROM_ERR_INVALID_ARG
        assert np.array_equal(hq.numpy(), w.q0)
    with pytest.raises(ValueError):   # device tensors belong to crom_step
        c.crom_step_host(ctx, torch.tensor(w.q0, device="cuda"), torch.tensor(w.alpha), torch.tensor(good),
                         torch.tensor(w.samples), torch.zeros(3, dtype=torch.int32), dt=w.dt, gn_iters=2,
                         max_samples=64)


def test_step_host_advection_and_per_sample_coefficient(c):
    """The optional arrays travel too: advection velocities (one per sample and
    dimension) and a per-sample coefficient; equal to crom_step bit for bit."""
    import torch
    w = gen.heat2d_batched(n_inst=12, m_lo=20, m_hi=200)
    ctx = make_ctx(w.spec, w.params)
    rng = np.random.default_rng(4)
    vel = rng.standard_normal((w.samples.shape[0], 2)).astype(np.float32)
    nu = rng.uniform(0.005, 0.02, w.samples.shape[0]).astype(np.float32)
    kw = dict(dt=1e-4, gn_iters=2, max_samples=int(w.sizes.max()), pde=c.CROM_PDE_ADVDIFF,
              coef_per_sample=True, precision=c.CROM_PREC_F16X2)
    d = StepInputs(w)
    c.crom_step(ctx, d.q, torch.tensor(nu, device="cuda"), d.s_off, d.samples, d.status,
                vel=torch.tensor(vel, device="cuda"), **kw)
    torch.cuda.synchronize()
    hq = torch.tensor(w.q0)
    hst = torch.full((w.n_inst,), -1, dtype=torch.int32)
    c.crom_step_host(ctx, hq, torch.tensor(nu), torch.tensor(w.s_off), torch.tensor(w.samples), hst,
                     vel=torch.tensor(vel), **kw)
    assert np.array_equal(hst.numpy(), d.status.cpu().numpy()) and np.all(hst.numpy() == c.CROM_OK)
    assert np.array_equal(hq.numpy(), d.q.cpu().numpy())
