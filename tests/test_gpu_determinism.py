"""Run-to-run determinism of every GPU kernel family (the race-detection plan without
compute-sanitizer): the same inputs twice give bit-identical outputs.  Every
reduction in the library has a fixed order and no kernel uses floating-point
atomics, so any difference would point at a race or an uninitialised read."""
import numpy as np
import pytest

from workloads import gen

from helpers import StepInputs, dev, make_ctx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c():
    from paper_2206_02607_gb300 import build
    build()
    from paper_2206_02607_gb300 import crom
    return crom


@pytest.mark.parametrize("prec_name", ["CROM_PREC_FP32", "CROM_PREC_F16X2", "CROM_PREC_F16"])
def test_step_twice_identical(c, prec_name):
    import torch
    w = gen.heat2d_batched(n_inst=200, m_lo=8, m_hi=400, bias_std=0.1)
    ctx = make_ctx(w.spec, w.params)
    out = []
    for _ in range(2):
        d = StepInputs(w)
        c.crom_step(ctx, d.q, d.alpha, d.s_off, d.samples, d.status, dt=w.dt, gn_iters=3,
                    max_samples=d.max_samples, precision=getattr(c, prec_name))
        torch.cuda.synchronize()
        out.append((d.q.cpu().numpy(), d.status.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    ctx.close()


@pytest.mark.parametrize("prec_name", ["CROM_PREC_FP32", "CROM_PREC_F16X2", "CROM_PREC_F16"])
def test_reconstruct_and_decode_twice_identical(c, prec_name):
    import torch
    spec = gen.DecoderSpec(2, 8, 128, 5)
    params = gen.xavier_decoder(spec, seed=5, bias_std=0.1)
    ctx = make_ctx(spec, params)
    rng = np.random.default_rng(1)
    X = dev(rng.uniform(0, 1, size=(20000, 2)).astype(np.float32), torch.float32)
    q = dev(rng.standard_normal((3, 8)), torch.float64)
    prec = getattr(c, prec_name)
    recon = []
    for _ in range(2):
        out = torch.full((3, 20000), np.nan, dtype=torch.float32, device="cuda")
        c.crom_reconstruct(ctx, q, X, out, precision=prec)
        torch.cuda.synchronize()
        recon.append(out.cpu().numpy())
    assert np.array_equal(recon[0], recon[1])
    off = dev(np.array([0, 5000, 12000, 20000], np.int32), torch.int32)
    dec = []
    for _ in range(2):
        if prec_name == "CROM_PREC_FP32":
            out = torch.full((1 + 2 + 2 + 1 + 8, 20000), np.nan, dtype=torch.float32, device="cuda")
            c.crom_decode(ctx, q, off, X, 31, out)
        else:
            out = torch.full((1 + 2 + 1 + 8, 20000), np.nan, dtype=torch.float32, device="cuda")
            want = c.CROM_WANT_VAL | c.CROM_WANT_DX | c.CROM_WANT_LAP | c.CROM_WANT_DQ
            c.crom_decode_tc(ctx, q, off, X, want, out, precision=prec)
        torch.cuda.synchronize()
        dec.append(out.cpu().numpy())
    assert np.all(np.isfinite(dec[0])) and np.array_equal(dec[0], dec[1])
    ctx.close()


@pytest.mark.parametrize("prec_name", ["CROM_PREC_FP32", "CROM_PREC_BF16_MIXED"])
def test_training_steps_twice_identical(c, prec_name):
    import torch
    from oracle import train_oracle as T
    n, r, width, hidden, B, S = 64, 8, 128, 4, 8, 512
    rng = np.random.default_rng(2)
    P = n * n
    lens = T.conv_lengths(P)
    enc = {"conv": [(rng.standard_normal(6) * 0.4, 0.05) for _ in lens[1:]],
           "dense": [(rng.standard_normal((32, lens[-1])) * 0.2, np.zeros(32)),
                     (rng.standard_normal((r, 32)) * 0.3, np.zeros(r))]}
    dec = gen.xavier_decoder(gen.DecoderSpec(2, r, width, hidden), seed=4, bias_std=0.1)
    p0 = T.flatten(enc, dec).astype(np.float32)
    snaps = dev(rng.standard_normal((B, P)).astype(np.float32), torch.float32)
    pts = dev(np.stack([rng.choice(P, size=S, replace=False) for _ in range(B)]).astype(np.int32), torch.int32)
    coords = dev(gen.grid_points_2d(n), torch.float32)
    res = []
    for _ in range(2):
        tr = c.CromTrainer(2, r, width, hidden, P, B, S)
        tr.set_precision(getattr(c, prec_name))
        tr.set_params(p0)
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        for _ in range(5):
            c.crom_train_step(tr, snaps, pts, coords, 1e-3, loss)
        torch.cuda.synchronize()
        res.append((tr.get_params(), loss.item()))
        tr.close()
    assert np.array_equal(res[0][0], res[1][0]) and res[0][1] == res[1][1]


def test_fom_twice_identical(c):
    import torch
    w = gen.advdiff_learned(n=64, n_traj=4, n_train=2)
    out = []
    for _ in range(2):
        u = dev(np.repeat(w.u0[None], 4, axis=0), torch.float32)
        tmp = torch.empty_like(u)
        ax = dev(np.repeat(w.ax[None], 4, axis=0), torch.float32)
        ay = dev(np.repeat(w.ay[None], 4, axis=0), torch.float32)
        c.crom_fom_step(c.CROM_FOM_ADVDIFF2D_PERIODIC_CENTRAL, u, tmp, dev(w.nu, torch.float32), dt=w.dt,
                        n_steps=50, ax=ax, ay=ay)
        torch.cuda.synchronize()
        out.append(u.cpu().numpy())
    assert np.array_equal(out[0], out[1])
