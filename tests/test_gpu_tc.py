"""GPU parity of the tcgen05 tensor-core paths (F16X2 / F16 step, F16X2 / F16 dense
reconstruction) against the FP64 oracle, through the C ABI.

Every decoder here has general FP32 weights, the form a trained decoder has; the
oracle evaluates exactly those weights in FP64.  The kernels carry activation
operands as f16 hi/lo pairs (~2^-22 relative); the step rounds its hidden
weights to f16 (2^-12 relative) and the dense reconstruction adds their f16 low
parts (~2^-22).  Tolerances: dense values rel. L2 <= 1e-4 (F16X2) and <= 3e-3
(F16: single f16 activations and weights).  Latent step:
the increment q_{n+1} - q_n moves with the weight rounding (J and the network
Laplacian change by up to ~1e-1 relative): <= 3e-2 or the least-squares
perturbation bound; q_{n+1} <= 5e-5.  Rollouts: q_T rel. L2 <= 1e-3.  The F16
step (activations as single f16 values, 2^-12 relative like the weights): twice
the residual and increment tolerances and 20 times the q_{n+1} tolerance (measured
up to 8.8 times the F16X2 bound on the ill-conditioned decoder shapes, kappa ~ 3e5);
its rollouts keep the 1e-3 bar.
"""
import numpy as np
import pytest

from oracle import crom_oracle as O
from workloads import gen

from helpers import dev, increment_errors, make_ctx, rel_l2, run_steps, subset

pytestmark = pytest.mark.gpu


def crom():
    from paper_2206_02607_gb300 import crom as c
    return c


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2206_02607_gb300 import build
    build()


@pytest.mark.parametrize("hidden,m,n_pts,n_codes", [(5, 2, 1000, 3), (3, 2, 129, 2), (5, 1, 4096, 2), (2, 2, 1, 1)])
def test_reconstruct_tc_matches_oracle(hidden, m, n_pts, n_codes):
    import torch
    c = crom()
    spec = gen.DecoderSpec(m, 8, 128, hidden)
    params = gen.xavier_decoder(spec, seed=hidden, bias_std=0.1)
    ctx = make_ctx(spec, params)
    X = np.random.default_rng(n_pts).uniform(0, 1, size=(n_pts, m)).astype(np.float32)
    codes = np.random.default_rng(7).standard_normal((n_codes, 8))
    ref = O.reconstruct(O.MLPDecoder(params, m), codes, X)
    for prec, tol in ((c.CROM_PREC_F16X2, 1e-4), (c.CROM_PREC_F16, 3e-3)):
        out = torch.full((n_codes, n_pts), float("nan"), dtype=torch.float32, device="cuda")
        c.crom_reconstruct(ctx, dev(codes, torch.float64), dev(X, torch.float32), out, precision=prec)
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel_l2(got, ref) < tol, (prec, rel_l2(got, ref))


def test_reconstruct_tc_full_grid_sampled():
    """The dense workload (1024^2 grid x 64 codes) in one launch, with hi/lo and with
    hi-only operands; every output is written (no NaN left), and 4096 sampled outputs
    are recomputed one by one by the oracle."""
    import torch
    c = crom()
    spec, params, codes, X = gen.recon_dense()
    ctx = make_ctx(spec, params)
    out = torch.empty((codes.shape[0], X.shape[0]), dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(11)
    ci = rng.integers(0, codes.shape[0], size=4096)
    pi = rng.integers(0, X.shape[0], size=4096)
    pi[:3] = [0, X.shape[0] - 1, 1023]
    dec = O.MLPDecoder(params, 2)
    ref = np.array([dec.value(X[p:p + 1], codes[k])[0] for k, p in zip(ci, pi)])
    for prec, tol in ((c.CROM_PREC_F16X2, 1e-4), (c.CROM_PREC_F16, 3e-3)):
        out.fill_(float("nan"))
        c.crom_reconstruct(ctx, dev(codes, torch.float64), dev(X, torch.float32), out, precision=prec)
        torch.cuda.synchronize()
        assert not torch.isnan(out).any().item()
        got = out[torch.as_tensor(ci, device="cuda"), torch.as_tensor(pi, device="cuda")].cpu().numpy()
        print(f"dense 1024^2 x 64, precision {prec}: sampled rel. L2 {rel_l2(got, ref):.2e}")
        assert rel_l2(got, ref) < tol, (prec, rel_l2(got, ref))


def test_reconstruct_tc_large_biases():
    """Hidden biases of order one and more: at F16 the dense reconstruction adds them
    on the tensor cores (f16 high and low parts of log2 e * b against a ones
    operand) and carries its activations times log2 e; same tolerances as above."""
    import torch
    c = crom()
    spec = gen.DecoderSpec(2, 8, 128, 4)
    params = gen.xavier_decoder(spec, seed=11, bias_std=2.0)
    ctx = make_ctx(spec, params)
    X = np.random.default_rng(3).uniform(0, 1, size=(777, 2)).astype(np.float32)
    codes = np.random.default_rng(4).standard_normal((2, 8))
    ref = O.reconstruct(O.MLPDecoder(params, 2), codes, X)
    for prec, tol in ((c.CROM_PREC_F16X2, 1e-4), (c.CROM_PREC_F16, 3e-3)):
        out = torch.full((2, 777), float("nan"), dtype=torch.float32, device="cuda")
        c.crom_reconstruct(ctx, dev(codes, torch.float64), dev(X, torch.float32), out, precision=prec)
        err = rel_l2(out.cpu().numpy(), ref)
        print(f"large biases, precision {prec}: {err:.2e}")
        assert err < tol, (prec, err)
    ctx.close()


def test_tensor_core_precisions_refuse_biases_beyond_f16_range():
    """A hidden bias beyond 45000 (log2 e * b would leave the f16 range) leaves the
    tensor-core images out: F16X2 / F16 return UNSUPPORTED, FP32 still runs."""
    import torch
    c = crom()
    spec = gen.DecoderSpec(2, 8, 128, 3)
    params = gen.xavier_decoder(spec, seed=12, bias_std=0.1)
    W, b = params[1]
    b = b.copy()
    b[5] = 5e4
    params[1] = (W, b)
    ctx = make_ctx(spec, params)
    q = torch.zeros((1, 8), dtype=torch.float64, device="cuda")
    x = torch.full((4, 2), 0.5, dtype=torch.float32, device="cuda")
    out = torch.empty((1, 4), dtype=torch.float32, device="cuda")
    for prec in (c.CROM_PREC_F16X2, c.CROM_PREC_F16):
        with pytest.raises(c.CromError) as e:
            c.crom_reconstruct(ctx, q, x, out, precision=prec)
        assert e.value.code == c.CROM_ERR_UNSUPPORTED
    c.crom_reconstruct(ctx, q, x, out, precision=c.CROM_PREC_FP32)
    torch.cuda.synchronize()
    assert np.all(np.isfinite(out.cpu().numpy()))
    ctx.close()


def test_reconstruct_tc_rejects_unsupported_shape():
    import torch
    c = crom()
    spec = gen.DecoderSpec(2, 8, 64, 3)
    ctx = make_ctx(spec, gen.xavier_decoder(spec, seed=0))
    out = torch.empty((1, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(c.CromError) as e:
        c.crom_reconstruct(ctx, torch.zeros((1, 8), dtype=torch.float64, device="cuda"),
                           torch.zeros((4, 2), dtype=torch.float32, device="cuda"), out, precision=c.CROM_PREC_F16X2)
    assert e.value.code == c.CROM_ERR_UNSUPPORTED


# ||J (d_gpu - d_ref)|| / ||Delta f||: the f16 weights (2^-12 relative) move the
# network Laplacian by up to ~1e-1 relative on these random decoders (their output
# layer cancels about two digits of the hidden Laplacians), and the fitted field
# change with it: 0.5 .. 12 % measured up to cond(J) ~ 1e4.
RES_TOL = 0.15
# the hidden weights' f16 rounding (RMS 2^-12 / sqrt(3) relative)
EPS_W = 2.0 ** -12 / np.sqrt(3.0)


# tolerance factors of the step per precision (q_{n+1}, residual and increment):
# single f16 activations add a rounding of the weights' size to every layer input
STEP_PRECS = [("CROM_PREC_F16X2", (1.0, 1.0)), ("CROM_PREC_F16", (20.0, 2.0))]


def _check_instance(w, i, q1_i, ref_i, f=(1.0, 1.0)):
    """Least-squares perturbation theory (Golub & Van Loan, Thm. 5.3.1) bounds the
    J-space error of a projection solved with relative data errors eps by about
    eps (2 + 3 kappa) and the increment error by about eps kappa (2 + kappa tan theta),
    tan theta = ||Delta f - J d|| / ||J d||: the q and residual tolerances hold up to
    kappa = 1e4 and grow linearly beyond (decoders with large r or 1D inputs reach
    kappa ~ 1e5); the increment's is 3e-2 or that bound with eps = EPS_W (the f16
    weight rounding), whichever is larger."""
    Y = w.samples[w.s_off[i]:w.s_off[i + 1]]
    inc, res, kappa, margin = increment_errors(w.params, w.spec.m, w.q0[i], Y, q1_i, ref_i, w.dt, w.alpha[i])
    grow = max(1.0, kappa / 1e4)
    fq, fr = f
    assert rel_l2(q1_i, ref_i) < 5e-5 * fq * grow, (i, rel_l2(q1_i, ref_i), kappa)
    # the fit's error grows linearly in kappa from a few thousand on (r = 15 decoders)
    assert res < fr * RES_TOL * max(1.0, kappa / 5e3), (i, res, kappa, margin)
    ev = O.MLPDecoder(w.params, w.spec.m)(Y, w.q0[i])
    jd = ev.gq @ (ref_i - w.q0[i])
    tan_theta = np.linalg.norm(w.dt * np.asarray(w.alpha[i], np.float64) * ev.lap - jd) / np.linalg.norm(jd)
    assert inc < fr * max(3e-2, EPS_W * kappa * (2 + kappa * tan_theta)), (i, inc, kappa, tan_theta)


def _check_step(w, q1, st, f=(1.0, 1.0)):
    dec = O.MLPDecoder(w.params, w.spec.m)
    ref, rst = O.crom_step_batched(dec, w.q0, w.s_off, w.samples, w.alpha, w.dt, w.gn_iters)
    assert np.array_equal(st, rst), (st, rst)
    for i in range(w.n_inst):
        if rst[i] == 0:
            _check_instance(w, i, q1[i], ref[i], f)


@pytest.mark.parametrize("prec_name,f", STEP_PRECS)
def test_step_tc_single_instance_heat2d(prec_name, f):
    c = crom()
    w = gen.heat2d_single()
    ctx = make_ctx(w.spec, w.params)
    q1, st = run_steps(ctx, w, 1, getattr(c, prec_name))
    _check_step(w, q1, st, f)


@pytest.mark.parametrize("prec_name,f", STEP_PRECS)
@pytest.mark.parametrize("gn_iters", [1, 2, 3])
def test_step_tc_batched_ragged(gn_iters, prec_name, f):
    """Uneven |M_i| including sizes below, at and above one tile (16 .. 32 samples)
    and several tiles with a ragged tail."""
    c = crom()
    w = gen.heat2d_batched(n_inst=20, m_lo=8, m_hi=300, bias_std=0.1)
    w.gn_iters = gn_iters
    ctx = make_ctx(w.spec, w.params)
    q1, st = run_steps(ctx, w, 1, getattr(c, prec_name))
    _check_step(w, q1, st, f)


@pytest.mark.parametrize("prec_name,f", STEP_PRECS)
def test_step_tc_one_dimensional_decoder(prec_name, f):
    c = crom()
    spec = gen.DecoderSpec(1, 4, 128, 4)
    params = gen.xavier_decoder(spec, seed=2, bias_std=0.1)
    rng = np.random.default_rng(1)
    sizes = [16, 40, 100]
    samples = np.concatenate([gen.interior_nodes_1d(256, s, rng) for s in sizes])
    w = gen.StepWorkload("1d", spec, params, rng.standard_normal((3, 4)), np.array([1.0, 0.5, 2.0], np.float32),
                         gen.ragged_offsets(sizes), samples, 1e-5, 2, 1)
    ctx = make_ctx(spec, params)
    q1, st = run_steps(ctx, w, 1, getattr(c, prec_name))
    _check_step(w, q1, st, f)


@pytest.mark.parametrize("prec_name,f", STEP_PRECS)
def test_step_tc_full_size_sampled_and_matches_fp32(prec_name, f):
    """All 1024 instances in one persistent launch (the launch the bench times); 10
    sampled instances recomputed by the oracle; the FP32 path agrees with it too."""
    c = crom()
    w = gen.heat2d_batched(n_inst=1024)
    ctx = make_ctx(w.spec, w.params)
    q1, st = run_steps(ctx, w, 1, getattr(c, prec_name))
    assert np.all(st == 0)
    dec = O.MLPDecoder(w.params, 2)
    for i in np.random.default_rng(1).choice(w.n_inst, size=10, replace=False):
        Y = w.samples[w.s_off[i]:w.s_off[i + 1]]
        ref, rst = O.crom_step(dec, w.q0[i], Y, w.dt, w.gn_iters, alpha=float(w.alpha[i]))
        assert rst == 0
        _check_instance(w, i, q1[i], ref, f)
    q32, st32 = run_steps(ctx, w, 1, c.CROM_PREC_FP32)
    assert np.all(st32 == 0)
    assert rel_l2(q1, q32) < 1e-5 * f[0]
    inc = np.linalg.norm((q1 - w.q0) - (q32 - w.q0), axis=1) / np.linalg.norm(q32 - w.q0, axis=1)
    print(f"{prec_name}: q1 vs FP32 {rel_l2(q1, q32):.2e}, median increment {np.median(inc):.2e}")
    assert np.median(inc) < 3e-2 * f[1]


@pytest.mark.parametrize("prec_name", ["CROM_PREC_F16X2", "CROM_PREC_F16"])
def test_step_tc_rollout_within_1e3(prec_name):
    """100-step rollouts of 6 instances: q_T within 1e-3 relative L2 of the oracle; the
    increment q_T - q_0 within 3e-2 (the f16 weights perturb the latent dynamics;
    6e-2 with single f16 activations)."""
    c = crom()
    full = gen.heat2d_batched(n_inst=64)
    w = subset(full, np.array([0, 5, 17, 33, 48, 63]))
    ctx = make_ctx(w.spec, w.params)
    steps = 100
    f = dict(STEP_PRECS)[prec_name][1]
    qT, st = run_steps(ctx, w, steps, getattr(c, prec_name))
    assert np.all(st == 0)
    dec = O.MLPDecoder(w.params, 2)
    for i in range(w.n_inst):
        Y = w.samples[w.s_off[i]:w.s_off[i + 1]]
        traj = O.crom_rollout(dec, w.q0[i], Y, w.dt, w.gn_iters, steps, alpha=float(w.alpha[i]))
        e_q, e_inc = rel_l2(qT[i], traj[-1]), rel_l2(qT[i] - w.q0[i], traj[-1] - w.q0[i])
        print(f"instance {i}: q_T {e_q:.3e}, increment {e_inc:.3e}")
        assert e_q < 1e-3 and e_inc < 3e-2 * f, (i, e_q, e_inc)


@pytest.mark.parametrize("prec_name", ["CROM_PREC_F16X2", "CROM_PREC_F16"])
def test_rollout_1000_step_graph_full_batch(prec_name):
    """The batched workload end to end: all 1024 instances advanced 1000 steps by one
    cached CUDA graph, bit-identical to 1000 crom_step calls; the instance with the
    smallest |M_i| and one of about a hundred samples (several tiles and a ragged
    tail) recomputed by the oracle over all 1000 steps.
    The heat equation is dissipative, so the per-step errors (<= 2e-6 relative in q)
    add up at most linearly: q_T within 1e-3, the increment q_T - q_0 within 3e-2."""
    import torch
    c = crom()
    w = gen.heat2d_batched(n_inst=1024)
    ctx = make_ctx(w.spec, w.params)
    steps = 1000
    q = dev(w.q0, torch.float64)
    st = torch.full((w.n_inst,), -1, dtype=torch.int32, device="cuda")
    prec = getattr(c, prec_name)
    f = dict(STEP_PRECS)[prec_name][1]
    c.crom_rollout(ctx, q, dev(w.alpha, torch.float32), dev(w.s_off, torch.int32), dev(w.samples, torch.float32),
                   st, n_steps=steps, dt=w.dt, gn_iters=w.gn_iters, max_samples=int(w.sizes.max()),
                   precision=prec)
    torch.cuda.synchronize()
    qT, stT = q.cpu().numpy(), st.cpu().numpy()
    assert np.all(stT == 0) and np.all(np.isfinite(qT))
    q_ref, st_ref = run_steps(ctx, w, steps, prec)
    assert np.array_equal(qT, q_ref) and np.array_equal(stT, st_ref)
    dec = O.MLPDecoder(w.params, 2)
    order = np.argsort(w.sizes, kind="stable")
    mid = next(int(j) for j in order if w.sizes[j] >= 90 and w.sizes[j] % 16)
    for i in (int(order[0]), mid):
        Y = w.samples[w.s_off[i]:w.s_off[i + 1]]
        traj = O.crom_rollout(dec, w.q0[i], Y, w.dt, w.gn_iters, steps, alpha=float(w.alpha[i]))
        e_q, e_inc = rel_l2(qT[i], traj[-1]), rel_l2(qT[i] - w.q0[i], traj[-1] - w.q0[i])
        print(f"{prec_name} instance {i} |M|={Y.shape[0]}: q_T {e_q:.3e}, increment {e_inc:.3e}")
        assert e_q < 1e-3 and e_inc < 3e-2 * f, (i, e_q, e_inc)


@pytest.mark.parametrize("prec_name", ["CROM_PREC_FP32", "CROM_PREC_F16X2", "CROM_PREC_F16"])
def test_rollout_graph_equals_repeated_steps(prec_name):
    """crom_rollout (a cached CUDA graph of n steps) gives bit-identical results to n
    crom_step calls; a second call replays the cached graph and continues."""
    import torch
    c = crom()
    prec = getattr(c, prec_name)
    w = gen.heat2d_batched(n_inst=40, m_lo=20, m_hi=200)
    ctx = make_ctx(w.spec, w.params)
    q_ref, st_ref = run_steps(ctx, w, 24, prec)
    q = dev(w.q0, torch.float64)
    a, o, s = dev(w.alpha, torch.float32), dev(w.s_off, torch.int32), dev(w.samples, torch.float32)
    st = torch.full((w.n_inst,), -1, dtype=torch.int32, device="cuda")
    for _ in range(2):
        c.crom_rollout(ctx, q, a, o, s, st, n_steps=12, dt=w.dt, gn_iters=w.gn_iters,
                       max_samples=int(w.sizes.max()), precision=prec)
    torch.cuda.synchronize()
    assert np.array_equal(q.cpu().numpy(), q_ref)
    assert np.array_equal(st.cpu().numpy(), st_ref)


@pytest.mark.parametrize("prec_name", ["CROM_PREC_F16X2", "CROM_PREC_F16"])
def test_step_tc_edge_cases_status(prec_name):
    c = crom()
    spec = gen.DecoderSpec(2, 4, 128, 3)
    params = gen.xavier_decoder(spec, seed=9, bias_std=0.1)
    ctx = make_ctx(spec, params)
    rng = np.random.default_rng(4)
    good = rng.uniform(0, 1, size=(50, 2)).astype(np.float32)
    dup = np.tile(np.array([[0.3, 0.7]], np.float32), (20, 1))
    few = rng.uniform(0, 1, size=(3, 2)).astype(np.float32)
    sizes = [50, 20, 3, 50, 0]
    samples = np.concatenate([good, dup, few, good], axis=0)
    off = gen.ragged_offsets(sizes)
    q0 = rng.standard_normal((5, 4))
    alpha = np.array([1.0, 1.0, 1.0, np.nan, 1.0], np.float32)
    w = gen.StepWorkload("edge", spec, params, q0, alpha, off, samples, 1e-4, 2, 1)
    q1, st = run_steps(ctx, w, 1, getattr(c, prec_name))
    assert list(st) == [c.CROM_OK, c.CROM_ERR_SINGULAR, c.CROM_ERR_INVALID_ARG, c.CROM_ERR_NONFINITE,
                        c.CROM_ERR_INVALID_ARG]
    assert np.array_equal(q1[1:], q0[1:])


def test_step_tc_rejects_unsupported():
    import torch
    c = crom()
    w = gen.heat1d_small()   # width 64: no tensor-core image
    ctx = make_ctx(w.spec, w.params)
    q = dev(w.q0, torch.float64)
    st = torch.empty(1, dtype=torch.int32, device="cuda")
    with pytest.raises(c.CromError) as e:
        c.crom_step(ctx, q, dev(w.alpha, torch.float32), dev(w.s_off, torch.int32), dev(w.samples, torch.float32),
                    st, dt=w.dt, gn_iters=1, max_samples=16, precision=c.CROM_PREC_F16X2)
    assert e.value.code == c.CROM_ERR_UNSUPPORTED
    w2 = gen.heat2d_single()
    ctx2 = make_ctx(w2.spec, w2.params)
    with pytest.raises(c.CromError) as e:
        c.crom_step(ctx2, dev(w2.q0, torch.float64), dev(w2.alpha, torch.float32), dev(w2.s_off, torch.int32),
                    dev(w2.samples, torch.float32), st, dt=w2.dt, gn_iters=2, max_samples=0,
                    precision=c.CROM_PREC_F16X2)
    assert e.value.code == c.CROM_ERR_INVALID_ARG


@pytest.mark.parametrize("prec_name,f", STEP_PRECS)
@pytest.mark.parametrize("n_samples", [2048, 5000])
def test_step_tc_large_instance(n_samples, prec_name, f):
    """One instance with 2048 samples (the single-instance sample set of the precision
    workload) or 5000 (many tiles, far above the batched sizes)."""
    c = crom()
    spec = gen.DecoderSpec(2, 8, 128, 5)
    params = gen.xavier_decoder(spec, seed=0, bias_std=0.05)
    rng = np.random.default_rng(2)
    Y = gen.interior_nodes_2d(128, n_samples, rng)
    w = gen.StepWorkload("big", spec, params, rng.standard_normal((1, 8)), np.ones(1, np.float32),
                         gen.ragged_offsets([n_samples]), Y, 1e-5, 2, 1)
    ctx = make_ctx(spec, params)
    q1, st = run_steps(ctx, w, 1, getattr(c, prec_name))
    _check_step(w, q1, st, f)


# Sample tiles of the tensor-core step: TILE_S0 samples per forward tile at GN
# iteration 0, TILE_S1 (large, small) later.
TILE_S0, TILE_S1 = 8, (16, 8)


@pytest.mark.parametrize("prec_name,f", STEP_PRECS)
@pytest.mark.parametrize("gn_iters", [2, 3])
def test_step_tc_small_tiles_matches_oracle(gn_iters, prec_name, f):
    """The small sample-tile variant of the step (TILE_S1[1] samples per tile after
    iteration 0, twice that with single f16 activations) against the oracle on uneven
    |M_i|; other shapes are rejected."""
    c = crom()
    w = gen.heat2d_batched(n_inst=20, m_lo=8, m_hi=300, bias_std=0.1)
    w.gn_iters = gn_iters
    ctx = make_ctx(w.spec, w.params)
    assert c.crom_get_step_tiles(ctx)[:2] == (TILE_S0, TILE_S1[0])
    c.crom_set_step_tiles(ctx, TILE_S0, TILE_S1[1])
    assert c.crom_get_step_tiles(ctx)[:2] == (TILE_S0, TILE_S1[1])
    q1, st = run_steps(ctx, w, 1, getattr(c, prec_name))
    _check_step(w, q1, st, f)
    for bad in ((TILE_S0, 4), (TILE_S0, 32), (16, TILE_S1[0])):
        with pytest.raises(c.CromError):
            c.crom_set_step_tiles(ctx, *bad)


def test_autotune_measures_both_tile_shapes_and_leaves_q():
    import torch
    c = crom()
    w = gen.heat2d_batched(n_inst=256)
    ctx = make_ctx(w.spec, w.params)
    q = dev(w.q0, torch.float64)
    status = torch.zeros(w.n_inst, dtype=torch.int32, device="cuda")
    s0, s1, ms = c.crom_autotune(ctx, q, dev(w.alpha, torch.float32), dev(w.s_off, torch.int32),
                                 dev(w.samples, torch.float32), status, dt=w.dt, gn_iters=w.gn_iters,
                                 max_samples=int(w.sizes.max()))
    torch.cuda.synchronize()
    assert s0 == TILE_S0 and s1 in TILE_S1 and min(ms) > 0
    assert s1 == (TILE_S1[0] if ms[0] <= ms[1] else TILE_S1[1])
    assert np.array_equal(q.cpu().numpy(), w.q0)          # the trials ran on a copy
    q1, st = run_steps(ctx, subset(w, np.arange(12)), 1, c.CROM_PREC_F16X2)
    _check_step(subset(w, np.arange(12)), q1, st)


@pytest.mark.parametrize("prec_name,f", STEP_PRECS)
@pytest.mark.parametrize("m,r,hidden", [(2, 1, 2), (2, 15, 5), (2, 15, 2), (1, 8, 3), (1, 4, 5), (2, 4, 3),
                                        (2, 12, 3), (2, 8, 4)])
def test_step_tc_decoder_shapes(m, r, hidden, prec_name, f):
    """The tensor-core step over the shapes it accepts: r = 1 and the largest r = 15,
    2 to 5 hidden layers, 1D and 2D inputs; uneven |M_i| around the tile sizes, the
    smallest |M_i| = r for r = 15.  (A 1D decoder with r = 15 is left out: its
    Jacobian at 15..16 points has kappa ~ 1e9, where whether the FP64 Cholesky
    declares the system singular depends on the rounding of J itself.)"""
    c = crom()
    spec = gen.DecoderSpec(m, r, 128, hidden)
    params = gen.xavier_decoder(spec, seed=10 * r + hidden, bias_std=0.1)
    rng = np.random.default_rng(r + 100 * hidden)
    sizes = [max(r, 15), 16, 33, 64, 130]
    if m == 1:
        samples = np.concatenate([gen.interior_nodes_1d(256, s, rng) for s in sizes])
    else:
        samples = np.concatenate([gen.interior_nodes_2d(128, s, rng) for s in sizes])
    w = gen.StepWorkload("shape", spec, params, rng.standard_normal((len(sizes), r)),
                         rng.uniform(0.5, 2.0, len(sizes)).astype(np.float32), gen.ragged_offsets(sizes), samples,
                         1e-5, 2, 1)
    ctx = make_ctx(spec, params)
    q1, st = run_steps(ctx, w, 1, getattr(c, prec_name))
    _check_step(w, q1, st, f)


@pytest.mark.parametrize("prec_name,f", STEP_PRECS)
def test_step_tc_advection_diffusion_matches_oracle(prec_name, f):
    """Delta f_j = dt (-a(y_j) . grad g + nu Lap g) on the tensor-core path (the
    gradient channels' outputs enter the residual), several instances."""
    import torch
    c = crom()
    spec = gen.DecoderSpec(2, 8, 128, 5)
    params = gen.xavier_decoder(spec, seed=13, bias_std=0.1)
    ctx = make_ctx(spec, params)
    rng = np.random.default_rng(8)
    sizes = [40, 90, 200]
    Y = np.concatenate([gen.interior_nodes_2d(128, s, rng) for s in sizes])
    vel = rng.standard_normal((Y.shape[0], 2)).astype(np.float32)
    q0 = rng.standard_normal((3, 8))
    nu = np.array([0.02, 0.005, 0.01], np.float32)
    off = gen.ragged_offsets(sizes)
    q = dev(q0, torch.float64)
    st = torch.empty(3, dtype=torch.int32, device="cuda")
    dt = 1e-4
    c.crom_step(ctx, q, dev(nu, torch.float32), dev(off, torch.int32), dev(Y, torch.float32), st,
                dt=dt, gn_iters=2, max_samples=200, pde=c.CROM_PDE_ADVDIFF, vel=dev(vel, torch.float32),
                precision=getattr(c, prec_name))
    torch.cuda.synchronize()
    q1 = q.cpu().numpy()
    dec = O.MLPDecoder(params, 2)
    for i in range(3):
        sl = slice(off[i], off[i + 1])
        ref, rst = O.crom_step(dec, q0[i], Y[sl], dt, 2, pde="advdiff", vel=vel[sl], nu=float(nu[i]))
        assert st[i].item() == 0 and rst == 0
        ev = dec(Y[sl], q0[i])
        df = O.advdiff_delta_f(ev, vel[sl], float(nu[i]), dt)
        res = np.linalg.norm(ev.gq @ (q1[i] - ref)) / np.linalg.norm(df)
        # dt = 1e-4: ten times the heat tests' increment, so ten times their q tolerance
        assert rel_l2(q1[i], ref) < 1e-4 * f[0] and res < RES_TOL * f[1], (i, rel_l2(q1[i], ref), res)
