"""Pins of the training-step oracle (encoder + decoder loss, hand-written backward,
Adam) against finite differences, an independent torch autodiff evaluation and
closed forms (CPU only)."""
import numpy as np
import pytest

from oracle import train_oracle as T
from workloads import gen


def tiny_problem(seed=0, n=16, r=3, width=16, hidden=2, B=3, S=7):
    rng = np.random.default_rng(seed)
    P = n * n
    lens = T.conv_lengths(P)
    enc = {"conv": [(rng.standard_normal(6) * 0.4, rng.standard_normal() * 0.1) for _ in lens[1:]],
           "dense": [(rng.standard_normal((32, lens[-1])) * 0.2, rng.standard_normal(32) * 0.1),
                     (rng.standard_normal((r, 32)) * 0.3, rng.standard_normal(r) * 0.1)]}
    dec = gen.xavier_decoder(gen.DecoderSpec(2, r, width, hidden), seed=seed + 1, bias_std=0.2)
    snaps = rng.standard_normal((B, P))
    pt_idx = np.stack([rng.choice(P, size=S, replace=False) for _ in range(B)])
    coords = gen.grid_points_2d(n).astype(np.float64)
    return enc, dec, snaps, pt_idx, coords


def test_conv_lengths_follow_the_paper_rule():
    assert T.conv_lengths(65536) == [65536, 16383, 4095, 1023, 255, 63]
    assert T.conv_lengths(256) == [256, 63]


def test_gradients_vs_central_differences():
    enc, dec, snaps, pt_idx, coords = tiny_problem()
    loss, eg, dg = T.loss_and_grads(enc, dec, snaps, pt_idx, coords, 2)
    p0 = T.flatten(enc, dec)
    gvec = T.flatten(eg, dg)
    rng = np.random.default_rng(5)
    h = 1e-6
    for i in rng.choice(p0.size, size=25, replace=False):
        pp, pm = p0.copy(), p0.copy()
        pp[i] += h
        pm[i] -= h
        e1, d1 = T.unflatten(pp, enc, dec)
        e2, d2 = T.unflatten(pm, enc, dec)
        lp = T.loss_and_grads(e1, d1, snaps, pt_idx, coords, 2)[0]
        lm = T.loss_and_grads(e2, d2, snaps, pt_idx, coords, 2)[0]
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gvec[i]) <= 1e-6 * max(1e-3, abs(gvec[i])) + 1e-9, (i, fd, gvec[i])


def test_gradients_vs_torch_autodiff():
    torch = pytest.importorskip("torch")
    enc, dec, snaps, pt_idx, coords = tiny_problem(seed=3)
    loss, eg, dg = T.loss_and_grads(enc, dec, snaps, pt_idx, coords, 2)
    p = torch.tensor(T.flatten(enc, dec), requires_grad=True)
    e_t, d_t = T.unflatten(np.zeros(p.numel()), enc, dec)

    def unpack(vec):
        o = 0
        out_dec, out_conv, out_dense = [], [], []
        for W, b in dec:
            nW, nb = np.size(W), np.size(b)
            out_dec.append((vec[o:o + nW].reshape(np.shape(W)), vec[o + nW:o + nW + nb]))
            o += nW + nb
        for w, b in enc["conv"]:
            out_conv.append((vec[o:o + 6], vec[o + 6]))
            o += 7
        for W, b in enc["dense"]:
            nW, nb = np.size(W), np.size(b)
            out_dense.append((vec[o:o + nW].reshape(np.shape(W)), vec[o + nW:o + nW + nb]))
            o += nW + nb
        return out_dec, out_conv, out_dense

    tdec, tconv, tdense = unpack(p)
    F = torch.nn.functional
    h = torch.tensor(snaps)[:, None, :]
    for w, b in tconv:
        h = F.elu(F.conv1d(h, w.view(1, 1, 6), b.view(1), stride=4))
    h = h[:, 0, :]
    h = F.elu(h @ tdense[0][0].T + tdense[0][1])
    q = h @ tdense[1][0].T + tdense[1][1]
    S = pt_idx.shape[1]
    X = torch.tensor(coords[pt_idx.ravel()])
    z = torch.cat([X, q.repeat_interleave(S, 0)], 1)
    for li, (W, b) in enumerate(tdec):
        z = z @ W.T + b
        if li + 1 < len(tdec):
            z = F.elu(z)
    target = torch.tensor(np.take_along_axis(snaps, pt_idx, 1).ravel())
    L = torch.mean((z[:, 0] - target) ** 2)
    L.backward()
    assert abs(L.item() - loss) < 1e-12 * max(1.0, abs(loss))
    np.testing.assert_allclose(T.flatten(eg, dg), p.grad.numpy(), rtol=1e-9, atol=1e-12)


def test_adam_first_step_closed_form_and_second_step():
    rng = np.random.default_rng(0)
    p = rng.standard_normal(50)
    g = rng.standard_normal(50)
    lr = 1e-3
    p1, m, v = T.adam_step(p, g, np.zeros(50), np.zeros(50), 1, lr)
    # first step: m_hat = g, v_hat = g^2  ->  p - lr * g / (|g| + eps)
    np.testing.assert_allclose(p1, p - lr * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    g2 = rng.standard_normal(50)
    p2, m2, v2 = T.adam_step(p1, g2, m, v, 2, lr)
    m_ref = 0.9 * 0.1 * g + 0.1 * g2
    v_ref = 0.999 * 0.001 * g * g + 0.001 * g2 * g2
    np.testing.assert_allclose(m2, m_ref, rtol=1e-13)
    np.testing.assert_allclose(v2, v_ref, rtol=1e-13)
    np.testing.assert_allclose(p2, p1 - lr * (m_ref / (1 - 0.81)) / (np.sqrt(v_ref / (1 - 0.999 ** 2)) + 1e-8),
                               rtol=1e-14)
