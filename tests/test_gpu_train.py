"""GPU training step (crom_train_step, crom_encode) against the FP64 training
oracle: loss, every gradient and the Adam update, through the C ABI.

FP32 arithmetic: the loss and gradients are sums over B*S points, so they are
held to relative L2 <= 1e-4 per parameter group against FP64; the Adam update is
compared where the gradient is not negligible (a gradient within FP32 noise of 0
may legitimately flip the sign of a first Adam step)."""
import numpy as np
import pytest

from oracle import train_oracle as T
from workloads import gen

from helpers import dev, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c():
    from paper_2206_02607_gb300 import build
    build()
    from paper_2206_02607_gb300 import crom
    return crom


def make_problem(seed, n, r, width, hidden, B, S):
    rng = np.random.default_rng(seed)
    P = n * n
    lens = T.conv_lengths(P)
    enc = {"conv": [(rng.standard_normal(6) * 0.4, rng.standard_normal() * 0.1) for _ in lens[1:]],
           "dense": [(rng.standard_normal((32, lens[-1])) * 0.2, rng.standard_normal(32) * 0.1),
                     (rng.standard_normal((r, 32)) * 0.3, rng.standard_normal(r) * 0.1)]}
    dec = gen.xavier_decoder(gen.DecoderSpec(2, r, width, hidden), seed=seed + 1, bias_std=0.2)
    enc = {"conv": [(np.float32(w).astype(np.float64), float(np.float32(b))) for w, b in enc["conv"]],
           "dense": [(np.float32(W).astype(np.float64), np.float32(b).astype(np.float64)) for W, b in enc["dense"]]}
    snaps = rng.standard_normal((B, P)).astype(np.float32)
    pt_idx = np.stack([rng.choice(P, size=S, replace=False) for _ in range(B)]).astype(np.int32)
    coords = gen.grid_points_2d(n)
    return enc, dec, snaps, pt_idx, coords


def groups(enc, dec):
    """Slices of the flat parameter vector: one per weight/bias array."""
    sizes = []
    for W, b in dec:
        sizes += [np.size(W), np.size(b)]
    for w, b in enc["conv"]:
        sizes += [6, 1]
    for W, b in enc["dense"]:
        sizes += [np.size(W), np.size(b)]
    o, out = 0, []
    for s in sizes:
        out.append(slice(o, o + s))
        o += s
    return out


@pytest.mark.parametrize("cfg", [dict(seed=0, n=16, r=3, width=32, hidden=3, B=3, S=37),
                                 dict(seed=1, n=64, r=8, width=64, hidden=4, B=5, S=300)])
def test_train_step_loss_gradients_and_adam(c, cfg):
    import torch
    enc, dec, snaps, pt_idx, coords = make_problem(**cfg)
    n, B, S = cfg["n"], cfg["B"], cfg["S"]
    tr = c.CromTrainer(2, cfg["r"], cfg["width"], cfg["hidden"], n * n, B, S)
    p0 = T.flatten(enc, dec)
    assert tr.n_params == p0.size
    tr.set_params(p0.astype(np.float32))
    loss_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    lr = 1e-3
    c.crom_train_step(tr, dev(snaps, torch.float32), dev(pt_idx, torch.int32), dev(coords, torch.float32), lr,
                      loss_dev)
    torch.cuda.synchronize()
    loss, eg, dg = T.loss_and_grads(enc, dec, snaps.astype(np.float64), pt_idx, coords.astype(np.float64), 2)
    assert abs(loss_dev.item() - loss) < 1e-5 * loss
    g_ref = T.flatten(eg, dg)
    g_gpu = tr.get_grads().astype(np.float64)
    for sl in groups(enc, dec):
        assert rel_l2(g_gpu[sl], g_ref[sl]) < 1e-4, sl
    p1_ref, _, _ = T.adam_step(p0, g_ref, np.zeros_like(p0), np.zeros_like(p0), 1, lr)
    p1 = tr.get_params().astype(np.float64)
    big = np.abs(g_ref) > 1e-3 * np.abs(g_ref).max()
    np.testing.assert_allclose(p1[big] - p0[big], p1_ref[big] - p0[big], rtol=1e-3, atol=1e-7)
    tr.close()


def test_encode_matches_oracle(c):
    import torch
    enc, dec, snaps, pt_idx, coords = make_problem(3, 64, 8, 32, 2, 4, 10)
    tr = c.CromTrainer(2, 8, 32, 2, 64 * 64, 4, 10)
    tr.set_params(T.flatten(enc, dec).astype(np.float32))
    q = torch.empty((3, 8), dtype=torch.float32, device="cuda")
    c.crom_encode(tr, dev(snaps[:3], torch.float32), q)
    torch.cuda.synchronize()
    q_ref, _ = T.encoder_forward(enc, snaps[:3].astype(np.float64))
    assert rel_l2(q.cpu().numpy(), q_ref) < 1e-5
    tr.close()


def test_training_reduces_the_loss(c):
    """20 Adam steps on snapshots of smooth fields lower the loss."""
    import torch
    n, r, B, S = 32, 4, 4, 256
    enc, dec, _, _, coords = make_problem(5, n, r, 32, 3, B, S)
    rng = np.random.default_rng(6)
    snaps = np.stack([gen.gaussian_bumps_2d(n, rng, count=3).ravel() for _ in range(B)]).astype(np.float32)
    tr = c.CromTrainer(2, r, 32, 3, n * n, B, S)
    tr.set_params(T.flatten(enc, dec).astype(np.float32))
    s_d, c_d = dev(snaps, torch.float32), dev(coords, torch.float32)
    losses = []
    for k in range(20):
        pt = dev(np.stack([rng.choice(n * n, size=S, replace=False) for _ in range(B)]).astype(np.int32), torch.int32)
        l = torch.zeros(1, dtype=torch.float64, device="cuda")
        c.crom_train_step(tr, s_d, pt, c_d, 3e-3, l)
        losses.append(l.item())
    assert np.mean(losses[-5:]) < 0.7 * np.mean(losses[:5]), losses
    tr.close()


def _step_and_check(c, cfg, precision, loss_tol, grad_tol, adam_big, adam_rtol):
    import torch
    enc, dec, snaps, pt_idx, coords = make_problem(**cfg)
    n, B, S = cfg["n"], cfg["B"], cfg["S"]
    tr = c.CromTrainer(2, cfg["r"], cfg["width"], cfg["hidden"], n * n, B, S)
    tr.set_precision(precision)
    p0 = T.flatten(enc, dec)
    tr.set_params(p0.astype(np.float32))
    loss_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    lr = 1e-3
    c.crom_train_step(tr, dev(snaps, torch.float32), dev(pt_idx, torch.int32), dev(coords, torch.float32), lr,
                      loss_dev)
    torch.cuda.synchronize()
    loss, eg, dg = T.loss_and_grads(enc, dec, snaps.astype(np.float64), pt_idx, coords.astype(np.float64), 2)
    errs = {}
    assert abs(loss_dev.item() - loss) < loss_tol * loss, (loss_dev.item(), loss)
    g_ref = T.flatten(eg, dg)
    g_gpu = tr.get_grads().astype(np.float64)
    for k, sl in enumerate(groups(enc, dec)):
        errs[k] = rel_l2(g_gpu[sl], g_ref[sl])
        assert errs[k] < grad_tol, (k, sl, errs[k])
    p1_ref, _, _ = T.adam_step(p0, g_ref, np.zeros_like(p0), np.zeros_like(p0), 1, lr)
    p1 = tr.get_params().astype(np.float64)
    big = np.abs(g_ref) > adam_big * np.abs(g_ref).max()
    np.testing.assert_allclose(p1[big] - p0[big], p1_ref[big] - p0[big], rtol=adam_rtol, atol=1e-7)
    tr.close()
    return errs


def test_train_step_bf16_tensor_cores(c):
    """The same step with the decoder's dense products on the library's tcgen05 GEMMs
    (bf16 weights, activations and deltas, FP32 accumulation): bf16 rounds each
    operand to 8 significant bits (2^-9 relative), so loss and gradients are held to
    relative L2 <= 1e-2 and 3e-2 per group; the first Adam step (-lr sign(g)) matches
    where |g| > 1e-2 max |g|."""
    _step_and_check(c, dict(seed=1, n=64, r=8, width=64, hidden=4, B=5, S=300), c.CROM_PREC_BF16_MIXED,
                    1e-2, 3e-2, 1e-2, 1e-2)


def test_train_step_precision_checks(c):
    tr = c.CromTrainer(2, 8, 32, 3, 64 * 64, 2, 10)
    with pytest.raises(c.CromError):
        tr.set_precision(c.CROM_PREC_BF16_MIXED)      # width 32: not a tensor-core tile width
    with pytest.raises(c.CromError):
        tr.set_precision(c.CROM_PREC_F16X2)
    with pytest.raises(c.CromError):
        tr.set_precision(3)                            # the former TF32 mode
    tr.close()


@pytest.mark.parametrize("prec_name,loss_tol,grad_tol", [("CROM_PREC_FP32", 1e-5, 1e-4),
                                                          ("CROM_PREC_BF16_MIXED", 1e-2, 3e-2)])
def test_train_step_learned_model_shapes(c, prec_name, loss_tol, grad_tol):
    """The training step at the learned-model shapes the bench times: 256 x 256
    snapshots (five convolutions 65536 -> 63), decoder R^{2+16} -> R with five ELU
    layers of width 256, 64 snapshots x 4096 sampled points (262,144 decoder rows):
    loss, every gradient group and the Adam update against the FP64 oracle, with the
    split-K weight gradients and fixed-order reductions at full depth."""
    errs = _step_and_check(c, dict(seed=4, n=256, r=16, width=256, hidden=5, B=64, S=4096),
                           getattr(c, prec_name), loss_tol, grad_tol, 1e-2, 1e-2)
    print(prec_name, "max gradient-group rel. L2", max(errs.values()),
          "largest:", sorted(errs.items(), key=lambda kv: -kv[1])[:4])


@pytest.mark.parametrize("prec_name", ["CROM_PREC_FP32", "CROM_PREC_BF16_MIXED"])
def test_checkpoint_resume_is_bit_identical(c, prec_name, tmp_path):
    """Train 4 steps, save, train 3 more; a fresh trainer that loads the checkpoint
    and takes the same 3 steps ends with bit-identical parameters and loss (Adam
    moments and step count restored; every reduction has a fixed order).  A
    checkpoint of other shapes and a corrupted one are refused and leave the
    trainer unchanged."""
    import torch
    n, r, width, hidden, B, S = 64, 8, 64, 4, 4, 256
    enc, dec, snaps, pt_idx, coords = make_problem(3, n, r, width, hidden, B, S)
    p0 = T.flatten(enc, dec).astype(np.float32)
    sn, pi, co = dev(snaps, torch.float32), dev(pt_idx, torch.int32), dev(coords, torch.float32)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")

    def trainer():
        tr = c.CromTrainer(2, r, width, hidden, n * n, B, S)
        tr.set_precision(getattr(c, prec_name))
        return tr

    a = trainer()
    a.set_params(p0)
    for _ in range(4):
        c.crom_train_step(a, sn, pi, co, 1e-3, loss)
    path = tmp_path / "trainer.ckpt"
    c.crom_trainer_save(a, path)
    for _ in range(3):
        c.crom_train_step(a, sn, pi, co, 1e-3, loss)
    torch.cuda.synchronize()
    pa, la = a.get_params(), loss.item()
    b = trainer()
    c.crom_trainer_load(b, path)
    for _ in range(3):
        c.crom_train_step(b, sn, pi, co, 1e-3, loss)
    torch.cuda.synchronize()
    assert np.array_equal(b.get_params(), pa) and loss.item() == la
    # refused: other shapes, a flipped payload byte
    other = c.CromTrainer(2, r, width, hidden + 1, n * n, B, S)
    with pytest.raises(c.CromError) as e:
        c.crom_trainer_load(other, path)
    assert e.value.code == c.CROM_ERR_INVALID_ARG
    raw = bytearray(path.read_bytes())
    raw[100] ^= 0x01
    bad = tmp_path / "bad.ckpt"
    bad.write_bytes(bytes(raw))
    before = b.get_params()
    with pytest.raises(c.CromError) as e:
        c.crom_trainer_load(b, bad)
    assert e.value.code == c.CROM_ERR_INVALID_ARG and "checksum" in c.last_error()
    assert np.array_equal(b.get_params(), before)
    for t in (a, b, other):
        t.close()
