"""Guards of the device-pointer entry points, through the C ABI:

* a cached rollout graph is recorded again when the context's scratch or weights
  were reallocated after it was recorded (the old recording refers to freed memory);
* an instance whose sample range s_off[i] .. s_off[i+1] reaches past n_samples is
  rejected on the device with INVALID_ARG and left unchanged (the input buffers here
  are larger than n_samples, so every access stays inside them);
* an FP32 step whose grid would exceed 65535 CTAs per instance is rejected on the
  host before anything is launched.
"""
import numpy as np
import pytest

from workloads import gen

from helpers import StepInputs, dev, make_ctx, run_steps

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2206_02607_gb300 import build
    build()


def crom():
    from paper_2206_02607_gb300 import crom as c
    return c


@pytest.mark.parametrize("prec_name", ["CROM_PREC_FP32", "CROM_PREC_F16X2"])
def test_rollout_rerecorded_after_scratch_grows(prec_name):
    """rollout(A), then crom_step on a larger batch B (which reallocates the step's
    scratch), then rollout(A) with the very same arguments: the result equals the same
    number of crom_step calls on A."""
    import torch
    c = crom()
    prec = getattr(c, prec_name)
    wa = gen.heat2d_batched(n_inst=8, m_lo=20, m_hi=60)
    wb = gen.heat2d_batched(n_inst=200, m_lo=100, m_hi=400, first=500)
    ctx = make_ctx(wa.spec, wa.params)
    q = dev(wa.q0, torch.float64)
    a, o, s = dev(wa.alpha, torch.float32), dev(wa.s_off, torch.int32), dev(wa.samples, torch.float32)
    st = torch.full((wa.n_inst,), -1, dtype=torch.int32, device="cuda")

    def roll():
        c.crom_rollout(ctx, q, a, o, s, st, n_steps=5, dt=wa.dt, gn_iters=wa.gn_iters,
                       max_samples=int(wa.sizes.max()), precision=prec)

    roll()
    run_steps(ctx, wb, 1, prec)          # larger batch: the context's scratch is reallocated
    roll()
    torch.cuda.synchronize()
    q_ref, st_ref = run_steps(ctx, wa, 10, prec)
    assert np.array_equal(q.cpu().numpy(), q_ref)
    assert np.array_equal(st.cpu().numpy(), st_ref)
    # new weights (same shape) also invalidate the recording
    spec = wa.spec
    params2 = gen.xavier_decoder(spec, seed=5)
    c.crom_set_weights(ctx, gen.pack_params(params2))
    q.copy_(dev(wa.q0, torch.float64))
    roll()
    torch.cuda.synchronize()
    w2 = gen.StepWorkload("w2", spec, params2, wa.q0, wa.alpha, wa.s_off, wa.samples, wa.dt, wa.gn_iters, 5)
    q_ref2, _ = run_steps(ctx, w2, 5, prec)
    assert np.array_equal(q.cpu().numpy(), q_ref2)
    ctx.close()


@pytest.mark.parametrize("entry", ["fp32", "bf16x2", "noalloc"])
def test_step_rejects_ranges_past_n_samples(entry):
    """s_off ends past n_samples: the offending instance gets INVALID_ARG and keeps q;
    the instance inside the range is stepped as usual."""
    import torch
    c = crom()
    w = gen.heat2d_batched(n_inst=2, m_lo=30, m_hi=30)
    ctx = make_ctx(w.spec, w.params)
    rng = np.random.default_rng(3)
    big = np.concatenate([w.samples, gen.interior_nodes_2d(128, 40, rng)])   # 100 rows in the buffer
    samples = dev(big, torch.float32)[:60]                                  # n_samples = 60
    s_off = dev(np.array([0, 30, 80], np.int32), torch.int32)                # instance 1 ends at 80 > 60
    q = dev(w.q0, torch.float64)
    alpha = dev(w.alpha, torch.float32)
    st = torch.full((2,), -1, dtype=torch.int32, device="cuda")
    kw = dict(dt=w.dt, gn_iters=w.gn_iters, max_samples=64)
    if entry == "noalloc":
        c.crom_step_noalloc(ctx, q, alpha, s_off, samples, st, **kw)
    else:
        prec = c.CROM_PREC_FP32 if entry == "fp32" else c.CROM_PREC_F16X2
        c.crom_step(ctx, q, alpha, s_off, samples, st, precision=prec, **kw)
    torch.cuda.synchronize()
    qg, sg = q.cpu().numpy(), st.cpu().numpy()
    assert list(sg) == [c.CROM_OK, c.CROM_ERR_INVALID_ARG]
    assert np.array_equal(qg[1], w.q0[1])
    assert not np.array_equal(qg[0], w.q0[0])
    ctx.close()


def test_fp32_step_grid_limit_is_an_argument_error():
    import torch
    c = crom()
    w = gen.heat2d_single()
    ctx = make_ctx(w.spec, w.params)
    q, a, o, s = dev(w.q0, torch.float64), dev(w.alpha, torch.float32), dev(w.s_off, torch.int32), \
        dev(w.samples, torch.float32)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    for fn in (lambda: c.crom_step(ctx, q, a, o, s, st, dt=w.dt, gn_iters=2, max_samples=2_000_000,
                                   precision=c.CROM_PREC_FP32),
               lambda: c.crom_step_noalloc(ctx, q, a, o, s, st, dt=w.dt, gn_iters=2, max_samples=2_000_000),
               lambda: c.crom_rollout(ctx, q, a, o, s, st, n_steps=2, dt=w.dt, gn_iters=2, max_samples=2_000_000,
                                      precision=c.CROM_PREC_FP32)):
        with pytest.raises(c.CromError) as e:
            fn()
        assert e.value.code == c.CROM_ERR_INVALID_ARG and "65535" in str(e.value)
    assert np.array_equal(q.cpu().numpy(), w.q0)
    ctx.close()


def test_stream_wait_deadline():
    """The host watchdog: a 1000-step rollout of the 1024-instance batch (about a
    second of GPU work) is not finished after 1 ms, so crom_stream_wait reports
    TIMEOUT without blocking; waiting again with a long deadline returns OK, and the
    kernels' own bounded-wait flags stayed clear."""
    import time
    import torch
    c = crom()
    w = gen.heat2d_batched(n_inst=1024)
    ctx = make_ctx(w.spec, w.params)
    d = StepInputs(w)
    stream = torch.cuda.current_stream()
    c.crom_rollout(ctx, d.q, d.alpha, d.s_off, d.samples, d.status, n_steps=1000, dt=w.dt, gn_iters=w.gn_iters,
                   max_samples=d.max_samples, precision=c.CROM_PREC_F16X2)   # records the graph
    torch.cuda.synchronize()
    c.crom_rollout(ctx, d.q, d.alpha, d.s_off, d.samples, d.status, n_steps=1000, dt=w.dt, gn_iters=w.gn_iters,
                   max_samples=d.max_samples, precision=c.CROM_PREC_F16X2)
    t0 = time.perf_counter()
    with pytest.raises(c.CromError) as e:
        c.crom_stream_wait(1.0, stream)
    assert e.value.code == c.CROM_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 0.5
    c.crom_stream_wait(60000.0, stream)
    assert np.all(d.status.cpu().numpy() == 0)
    assert c.crom_device_flags(ctx) == 0
    ctx.close()
