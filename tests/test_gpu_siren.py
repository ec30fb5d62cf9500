"""SIREN decoders (sin(omega0 z), omega0 = 30; paper App. D) on the FP32 CUDA-core
path, and the tangent-space velocity dg/dq . qdot (App. L), against the FP64
oracle.

SIREN's derivatives grow with omega0 (the Laplacian channel carries omega0^2 per
layer), and the FP32 argument omega0 * z carries ~1e-6 relative rounding into
sin and cos: tolerances are 1e-4 on values and first derivatives and 1e-3 on the
Laplacian channel (relative L2 over the points)."""
import numpy as np
import pytest

from oracle import crom_oracle as O
from workloads import gen

from helpers import StepInputs, dev, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c():
    from paper_2206_02607_gb300 import build
    build()
    from paper_2206_02607_gb300 import crom
    return crom


def _siren_ctx(c, spec, params):
    ctx = c.crom_create(spec.m, spec.r, spec.width, spec.hidden, 0, activation=c.CROM_ACT_SIREN, omega0=30.0)
    c.crom_set_weights(ctx, gen.pack_params(params))
    return ctx


def test_siren_decode_all_channels(c):
    import torch
    spec = gen.DecoderSpec(2, 4, 64, 3)
    params = gen.siren_decoder(spec, seed=3)
    ctx = _siren_ctx(c, spec, params)
    rng = np.random.default_rng(4)
    X = rng.uniform(-1, 1, size=(777, 2)).astype(np.float32)
    q = rng.standard_normal((3, 4)) * 0.5
    off = np.array([0, 300, 301, 777], np.int32)
    want = c.CROM_WANT_VAL | c.CROM_WANT_DX | c.CROM_WANT_LAP | c.CROM_WANT_DQ
    C = 1 + 2 + 1 + 4
    out = torch.empty((C, 777), dtype=torch.float32, device="cuda")
    c.crom_decode(ctx, dev(q, torch.float64), dev(off, torch.int32), dev(X, torch.float32), want, out)
    got = out.cpu().numpy().astype(np.float64)
    dec = O.MLPDecoder(params, 2, activation="siren")
    ref_g, ref_gx, ref_lap, ref_gq = [], [], [], []
    for i in range(3):
        ev = dec(X[off[i]:off[i + 1]], q[i])
        ref_g.append(ev.g); ref_gx.append(ev.gx); ref_lap.append(ev.lap); ref_gq.append(ev.gq)
    assert rel_l2(got[0], np.concatenate(ref_g)) < 1e-4
    assert rel_l2(got[1:3].T, np.concatenate(ref_gx)) < 1e-4
    assert rel_l2(got[3], np.concatenate(ref_lap)) < 1e-3
    assert rel_l2(got[4:8].T, np.concatenate(ref_gq)) < 1e-4


def test_siren_step_and_reconstruction_fp32(c):
    import torch
    spec = gen.DecoderSpec(2, 6, 64, 3)
    params = gen.siren_decoder(spec, seed=8)
    ctx = _siren_ctx(c, spec, params)
    w = gen.heat2d_batched(n_inst=6, m_lo=40, m_hi=200)
    w.samples = (2.0 * w.samples - 1.0).astype(np.float32)     # SIREN inputs in [-1, 1]
    w.q0 = w.q0[:, :6] * 0.5
    w.spec, w.params = spec, params
    d = StepInputs(w)
    c.crom_step(ctx, d.q, d.alpha, d.s_off, d.samples, d.status, dt=1e-6, gn_iters=2, max_samples=d.max_samples,
                precision=c.CROM_PREC_FP32)
    torch.cuda.synchronize()
    q1, st = d.q.cpu().numpy(), d.status.cpu().numpy()
    dec = O.MLPDecoder(params, 2, activation="siren")
    for i in range(w.n_inst):
        Y = w.samples[w.s_off[i]:w.s_off[i + 1]]
        ref, rst = O.crom_step(dec, w.q0[i], Y, 1e-6, 2, alpha=float(w.alpha[i]))
        assert st[i] == rst == 0
        ev = dec(Y, w.q0[i])
        df = 1e-6 * float(w.alpha[i]) * ev.lap
        res = np.linalg.norm(ev.gq @ ((q1[i] - ref))) / np.linalg.norm(df)
        assert res < 1e-3, (i, res)
    # reconstruction
    X = np.random.default_rng(2).uniform(-1, 1, size=(5000, 2)).astype(np.float32)
    out = torch.empty((2, 5000), dtype=torch.float32, device="cuda")
    c.crom_reconstruct(ctx, dev(w.q0[:2], torch.float64), dev(X, torch.float32), out, precision=c.CROM_PREC_FP32)
    assert rel_l2(out.cpu().numpy(), O.reconstruct(dec, w.q0[:2], X)) < 1e-4


def test_siren_unsupported_paths(c):
    import torch
    spec = gen.DecoderSpec(2, 6, 128, 3)
    params = gen.siren_decoder(spec, seed=8)
    ctx = _siren_ctx(c, spec, params)
    X = dev(np.zeros((10, 2), np.float32), torch.float32)
    out = torch.empty((1, 10), dtype=torch.float32, device="cuda")
    with pytest.raises(c.CromError):
        c.crom_reconstruct(ctx, dev(np.zeros((1, 6)), torch.float64), X, out, precision=c.CROM_PREC_F16X2)
    with pytest.raises(c.CromError):   # the training step is built for ELU decoders
        _siren_trainer(c)


def _siren_trainer(c):
    import ctypes
    h = ctypes.c_void_p()
    d = c.crom_decoder_desc(2, 6, 128, 3, c.CROM_ACT_SIREN, 30.0)
    c._check(c.raw_call("crom_trainer_create", ctypes.byref(h), ctypes.byref(d), 4096, 4, 64, 0))


@pytest.mark.parametrize("activation", ["elu", "siren"])
def test_tangent_velocity(c, activation):
    import torch
    spec = gen.DecoderSpec(2, 5, 64, 3)
    if activation == "elu":
        params = gen.xavier_decoder(spec, seed=4, bias_std=0.1)
        ctx = c.crom_create(2, 5, 64, 3)
        c.crom_set_weights(ctx, gen.pack_params(params))
        X = np.random.default_rng(5).uniform(0, 1, size=(900, 2)).astype(np.float32)
    else:
        params = gen.siren_decoder(spec, seed=4)
        ctx = _siren_ctx(c, spec, params)
        X = np.random.default_rng(5).uniform(-1, 1, size=(900, 2)).astype(np.float32)
    rng = np.random.default_rng(6)
    q = rng.standard_normal((4, 5)) * 0.5
    qp = q + 1e-3 * rng.standard_normal((4, 5))
    qp[2] = q[2]                                      # first step of a rollout: qdot = 0
    off = np.array([0, 250, 251, 600, 900], np.int32)
    out = torch.full((900,), float("nan"), dtype=torch.float32, device="cuda")
    c.crom_tangent_velocity(ctx, dev(q, torch.float64), dev(qp, torch.float64), dev(off, torch.int32),
                            dev(X, torch.float32), out, dt=1e-2)
    got = out.cpu().numpy()
    dec = O.MLPDecoder(params, 2, activation=activation)
    ref = np.concatenate([O.tangent_velocity(dec, X[off[i]:off[i + 1]], q[i], qp[i], 1e-2) for i in range(4)])
    assert np.all(got[251:600] == 0.0)
    assert rel_l2(got, ref) < 1e-4
