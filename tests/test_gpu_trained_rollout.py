"""End to end on the GPU: the full-order solver generates snapshots, the encoder
and decoder are trained on them (crom_train_step), and the latent dynamics of a
held-out parameter, started from the encoder's code of the initial condition, is
rolled out (crom_rollout) and reconstructed at every node (crom_reconstruct);
the result is compared with the full-order solution (paper §3 manifold
construction, §4 latent dynamics; App. H.2 for the 2D heat FOM).

Workload: 2D heat u_t = alpha Lap u on 48 x 48 nodes, zero Neumann, u0 = the same
8 Gaussian bumps (sigma in [0.06, 0.12], resolved by the 48-node grid) for every
trajectory; training alpha in {0.5, 0.75, ..., 2.0},
test alpha = 1.3; 96 FOM steps of dt = h^2 / 16, snapshots every 4 steps.
Decoder R^{2+8} -> R, 5 ELU layers of width 128; 80000 Adam steps (the library's
bf16 tensor-core decoder pass) of 32 snapshots x 1024 nodes, learning rate 1e-3
for a quarter of them, then decayed to 2e-5 (with 40000 steps the final-field
error sat at the 1e-2 bar, 7.6e-3 .. 1.2e-2 depending on rounding details);
200 integration samples.

Bar: relative L2 of the final reconstructed field against the FOM <= 1e-2 for
the FP32 step and for the F16X2 step, and of the decoded initial field <= 2e-2
(the paper quotes 0.43 % for a 1D heat model trained for 180k epochs; this model
trains for under a minute)."""
import numpy as np
import pytest

from workloads import gen

from helpers import dev, rel_l2

pytestmark = pytest.mark.gpu

N_SIDE, STEPS, EVERY = 48, 96, 4
TRAIN_ALPHAS = np.linspace(0.5, 2.0, 7)
TEST_ALPHA = 1.3


@pytest.fixture(scope="module")
def c():
    from paper_2206_02607_gb300 import build
    build()
    from paper_2206_02607_gb300 import crom
    return crom


def _fom(c, alphas, u0, dt):
    """Snapshots [len(alphas)][STEPS / EVERY + 1][P] of the GPU full-order solver."""
    import torch
    nb = len(alphas)
    u = dev(np.repeat(u0[None], nb, axis=0), torch.float32)
    tmp = torch.empty_like(u)
    coef = dev(np.asarray(alphas, np.float32), torch.float32)
    snaps = [u.reshape(nb, -1).clone()]
    for _ in range(STEPS // EVERY):
        c.crom_fom_step(c.CROM_FOM_HEAT2D_NEUMANN, u, tmp, coef, dt=dt, n_steps=EVERY)
        snaps.append(u.reshape(nb, -1).clone())
    return torch.stack(snaps, dim=1)


COORD_SCALE = float(np.std(np.arange(N_SIDE) / (N_SIDE - 1)))


@pytest.fixture(scope="module")
def trained(c):
    """Fields and coordinates are standardised as in the paper (App. D: zero mean,
    unit variance; coordinates centred and scaled): v = (u - mu) / sigma solves the
    same heat equation, and in the scaled coordinates x' = (x - 1/2) / s the
    diffusivity becomes alpha / s^2."""
    import torch
    from oracle import train_oracle as T
    n = N_SIDE
    P = n * n
    h = 1.0 / (n - 1)
    dt = h * h / 16
    u0 = gen.gaussian_bumps_2d(n, np.random.default_rng(3), sigma=(0.06, 0.12)).astype(np.float32)
    train = _fom(c, TRAIN_ALPHAS, u0, dt).reshape(-1, P)          # [n_snap][P]
    mu, sigma = float(train.mean()), float(train.std())
    train = (train - mu) / sigma
    r, width, hidden, B, S = 8, 128, 5, 32, 1024
    spec = gen.DecoderSpec(2, r, width, hidden)
    tr = c.CromTrainer(2, r, width, hidden, P, B, S)
    tr.set_precision(c.CROM_PREC_BF16_MIXED)
    rng = np.random.default_rng(7)
    lens = T.conv_lengths(P)
    enc = {"conv": [(rng.standard_normal(6) * np.sqrt(2.0 / 6), 0.0) for _ in lens[1:]],
           "dense": [(rng.standard_normal((32, lens[-1])) * np.sqrt(2.0 / (lens[-1] + 32)), np.zeros(32)),
                     (rng.standard_normal((r, 32)) * np.sqrt(2.0 / (32 + r)), np.zeros(r))]}
    dec = gen.xavier_decoder(spec, seed=11)
    p0 = T.flatten(enc, dec).astype(np.float32)
    assert p0.size == tr.n_params
    tr.set_params(p0)
    X = ((gen.grid_points_2d(n) - 0.5) / COORD_SCALE).astype(np.float32)
    coords = dev(X, torch.float32)
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    n_steps, losses = 80000, []
    for k in range(n_steps):
        lr = 1e-3 if k < 20000 else 1e-3 * (2e-5 / 1e-3) ** ((k - 20000) / (n_steps - 20001))
        pick = torch.randint(0, train.shape[0], (B,), device="cuda", generator=g)
        pts = torch.randint(0, P, (B, S), device="cuda", generator=g, dtype=torch.int32)
        c.crom_train_step(tr, train[pick].contiguous(), pts, coords, lr, loss)
        if k % 16000 == 0 or k == n_steps - 1:
            losses.append(loss.item())
    torch.cuda.synchronize()
    params = tr.get_params()
    q0 = torch.empty((1, r), dtype=torch.float32, device="cuda")
    c.crom_encode(tr, dev(((u0.reshape(1, -1) - mu) / sigma).astype(np.float32), torch.float32), q0)
    torch.cuda.synchronize()
    test = _fom(c, [TEST_ALPHA], u0, dt)[0]                         # [n_snap][P]
    print(f"training losses (standardised fields): {['%.2e' % v for v in losses]}")
    return dict(spec=spec, params=params[:gen.param_count(spec)], q0=q0.cpu().numpy().astype(np.float64), dt=dt,
                test=test.cpu().numpy().astype(np.float64), mu=mu, sigma=sigma, X=X, tr=tr)


@pytest.mark.parametrize("prec_name", ["CROM_PREC_FP32", "CROM_PREC_F16X2"])
def test_trained_rollout_matches_full_order_solver(c, trained, prec_name):
    import torch
    spec, n = trained["spec"], N_SIDE
    mu, sigma = trained["mu"], trained["sigma"]
    ctx = c.crom_create(spec.m, spec.r, spec.width, spec.hidden)
    c.crom_set_weights(ctx, trained["params"])
    Xd = dev(trained["X"], torch.float32)
    out = torch.empty((1, n * n), dtype=torch.float32, device="cuda")

    def field(q):
        c.crom_reconstruct(ctx, q, Xd, out)
        torch.cuda.synchronize()
        return out.cpu().numpy()[0].astype(np.float64) * sigma + mu

    q = dev(trained["q0"], torch.float64)
    fit0 = rel_l2(field(q), trained["test"][0])          # the decoder reproduces u0 from the encoder's code
    # latent rollout of the held-out alpha with 200 interior integration samples
    samples = ((gen.interior_nodes_2d(n, 200, np.random.default_rng(9)) - 0.5) / COORD_SCALE).astype(np.float32)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    alpha_eff = TEST_ALPHA / COORD_SCALE ** 2
    c.crom_rollout(ctx, q, dev(np.array([alpha_eff], np.float32), torch.float32),
                   dev(np.array([0, 200], np.int32), torch.int32), dev(samples, torch.float32), status,
                   n_steps=STEPS, dt=trained["dt"], gn_iters=2, max_samples=200,
                   precision=getattr(c, prec_name))
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    err = rel_l2(field(q), trained["test"][-1])
    moved = rel_l2(trained["test"][-1], trained["test"][0])
    print(f"trained rollout ({prec_name}): fit of u0 {fit0:.3e}, final-field error {err:.3e} "
          f"(the field itself changes by {moved:.3e})")
    assert fit0 < 2e-2 and err < 1e-2, (fit0, err)
