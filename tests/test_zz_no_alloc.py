"""crom_step_noalloc: the FP32 step for callers that cannot allocate device memory
while stepping (hosts that own the device memory, allocation-free loops), with its
scratch in a fixed device array.  Its results must equal crom_step's (same kernel, same
reduction order), on consecutive calls that reuse the shared scratch with
different batch shapes.  Collected last on purpose."""
import numpy as np
import pytest

from workloads import gen

from helpers import dev, make_ctx, rel_l2

pytestmark = pytest.mark.gpu


def _state(w):
    import torch
    return (dev(w.q0, torch.float64), dev(w.alpha, torch.float32), dev(w.s_off, torch.int32),
            dev(w.samples, torch.float32), torch.full((w.n_inst,), -1, dtype=torch.int32, device="cuda"))


def _two_calls(ctx, w, fn, crom):
    import torch
    q, a, o, s, st = _state(w)
    out = []
    for _ in range(2):
        fn(ctx, q, a, o, s, st, dt=w.dt, gn_iters=w.gn_iters, max_samples=int(w.sizes.max()))
        torch.cuda.synchronize()
        out.append((q.cpu().numpy().copy(), st.cpu().numpy().copy()))
    return out


def test_noalloc_step_matches_crom_step_on_consecutive_calls():
    from paper_2206_02607_gb300 import build
    build()
    from paper_2206_02607_gb300 import crom
    w1 = gen.heat2d_single()
    w2 = gen.heat2d_batched(n_inst=6, m_lo=8, m_hi=120, bias_std=0.1)
    for w in (w1, w2, w1):          # the second shape re-lays out the shared array, then back
        ctx = make_ctx(w.spec, w.params)

        def ref_step(*args, **kw):
            crom.crom_step(*args, precision=crom.CROM_PREC_FP32, **kw)

        ref = _two_calls(ctx, w, ref_step, crom)
        got = _two_calls(ctx, w, crom.crom_step_noalloc, crom)
        for (qr, sr), (qg, sg) in zip(ref, got):
            assert np.array_equal(sr, sg) and np.all(sg == 0)
            assert rel_l2(qg, qr) < 1e-12
            assert rel_l2(qg - w.q0, qr - w.q0) < 1e-9
        ctx.close()


def test_noalloc_step_rejects_batches_beyond_its_fixed_scratch():
    import torch
    from paper_2206_02607_gb300 import crom
    w = gen.heat2d_single()
    ctx = make_ctx(w.spec, w.params)
    n = 4096                         # 4096 instances x up to 4096 samples: far beyond 8 MiB of partial sums
    q = torch.zeros((n, 8), dtype=torch.float64, device="cuda")
    a = torch.ones(n, dtype=torch.float32, device="cuda")
    o = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    s = torch.zeros((1, 2), dtype=torch.float32, device="cuda")
    st = torch.zeros(n, dtype=torch.int32, device="cuda")
    with pytest.raises(crom.CromError) as e:
        crom.crom_step_noalloc(ctx, q, a, o, s, st, dt=1e-5, gn_iters=2, max_samples=4096)
    assert e.value.code == crom.CROM_ERR_INVALID_ARG
    assert "scratch" in str(e.value)
    ctx.close()
