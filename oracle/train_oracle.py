"""FP64 oracle of one CROM training step (manifold construction, paper §3 and App. D).
TEST INFRASTRUCTURE ONLY.

* Encoder e(f) (App. D): 1D convolutions of kernel 6, stride 4, one channel, no
  padding, on the flattened snapshot, repeated while the output stays >= 32
  (65536 -> 16383 -> 4095 -> 1023 -> 255 -> 63 for a 256 x 256 field), ELU after
  each; then a dense layer to 32 with ELU and a linear layer to r.
* Decoder g(x, q): the MLP of crom_oracle.MLPDecoder (value channel only).
* Loss (Eq. loss, encoder + decoder): mean over the batch of snapshots b and the
  sampled points j of (g(x_j, e(f_b)) - f_b(x_j))^2.
* Gradients by hand (chain rule written out layer by layer, reverse order).
* Adam (Kingma and Ba) with beta1 = 0.9, beta2 = 0.999, eps = 1e-8 (the paper
  names Adam and the learning rate only; these are the defaults of its framework).
"""
from __future__ import annotations

import numpy as np

from .crom_oracle import elu, elu_d1

__all__ = ["conv_lengths", "encoder_forward", "encoder_backward", "decoder_forward_value",
           "decoder_backward", "loss_and_grads", "adam_step", "flatten", "unflatten"]


def conv_lengths(P: int, kernel: int = 6, stride: int = 4, stop: int = 32):
    """Output lengths of the strided convolutions: keep convolving while the next
    length would still be >= stop (App. D: closest to 32 but no smaller)."""
    lens = [P]
    while True:
        nxt = (lens[-1] - kernel) // stride + 1
        if nxt < stop:
            break
        lens.append(nxt)
    return lens


def _conv1d(x, w, b, stride):
    """y_i = b + sum_k w_k x_{stride * i + k}, x: [B, L]."""
    K = w.shape[0]
    Lout = (x.shape[1] - K) // stride + 1
    y = np.full((x.shape[0], Lout), b, dtype=np.float64)
    for k in range(K):
        y += w[k] * x[:, k: k + stride * (Lout - 1) + 1: stride]
    return y


def encoder_forward(enc, f):
    """enc: dict with 'conv' = [(w[6], b)], 'dense' = [(W1 [32][L], b1), (W2 [r][32], b2)].
    f: [B, P] snapshots.  Returns (q [B, r], cache)."""
    h = np.asarray(f, np.float64)
    cache = {"conv_in": [], "conv_z": [], "dense_in": [], "dense_z": []}
    for w, b in enc["conv"]:
        cache["conv_in"].append(h)
        z = _conv1d(h, np.asarray(w, np.float64), float(b), 4)
        cache["conv_z"].append(z)
        h = elu(z)
    (W1, b1), (W2, b2) = enc["dense"]
    cache["dense_in"].append(h)
    z1 = h @ np.asarray(W1).T + b1
    cache["dense_z"].append(z1)
    h1 = elu(z1)
    cache["dense_in"].append(h1)
    q = h1 @ np.asarray(W2).T + b2
    return q, cache


def encoder_backward(enc, cache, dq):
    """Gradients of the loss with respect to the encoder parameters, given dL/dq."""
    (W1, b1), (W2, b2) = enc["dense"]
    h0, h1 = cache["dense_in"]
    gW2 = dq.T @ h1
    gb2 = dq.sum(0)
    dz1 = (dq @ np.asarray(W2)) * elu_d1(cache["dense_z"][0])
    gW1 = dz1.T @ h0
    gb1 = dz1.sum(0)
    dh = dz1 @ np.asarray(W1)
    g_conv = [None] * len(enc["conv"])
    for li in reversed(range(len(enc["conv"]))):
        w, b = enc["conv"][li]
        dz = dh * elu_d1(cache["conv_z"][li])
        x = cache["conv_in"][li]
        K, Lout = len(w), dz.shape[1]
        gw = np.array([np.sum(dz * x[:, k: k + 4 * (Lout - 1) + 1: 4]) for k in range(K)])
        gb = dz.sum()
        dx = np.zeros_like(x)
        for k in range(K):
            dx[:, k: k + 4 * (Lout - 1) + 1: 4] += w[k] * dz
        g_conv[li] = (gw, gb)
        dh = dx
    return {"conv": g_conv, "dense": [(gW1, gb1), (gW2, gb2)]}


def decoder_forward_value(dec, X, Q):
    """dec: list of (W, b); X [N, m], Q [N, r].  Returns (g [N], cache)."""
    h = np.concatenate([np.asarray(X, np.float64), np.asarray(Q, np.float64)], axis=1)
    ins, zs = [], []
    for li, (W, b) in enumerate(dec):
        ins.append(h)
        z = h @ np.asarray(W, np.float64).T + np.asarray(b, np.float64)
        zs.append(z)
        h = elu(z) if li + 1 < len(dec) else z
    return h[:, 0], {"ins": ins, "zs": zs}


def decoder_backward(dec, cache, dg):
    """Gradients with respect to the decoder parameters and to its inputs, given dL/dg."""
    grads = [None] * len(dec)
    delta = dg[:, None]
    for li in reversed(range(len(dec))):
        W, _ = dec[li]
        if li + 1 < len(dec):
            delta = delta * elu_d1(cache["zs"][li])
        grads[li] = (delta.T @ cache["ins"][li], delta.sum(0))
        delta = delta @ np.asarray(W, np.float64)
    return grads, delta   # delta = dL/d[x; q] per point


def loss_and_grads(enc, dec, snaps, pt_idx, coords, m):
    """One training step's loss (Eq. loss) and gradients.
    snaps [B, P]; pt_idx [B, S] sampled node indices; coords [P, m]."""
    B, S = pt_idx.shape
    q, ecache = encoder_forward(enc, snaps)
    X = coords[pt_idx.ravel()]
    Q = np.repeat(q, S, axis=0)
    target = np.take_along_axis(np.asarray(snaps, np.float64), pt_idx, axis=1).ravel()
    g, dcache = decoder_forward_value(dec, X, Q)
    resid = g - target
    loss = float(np.mean(resid ** 2))
    dg = 2.0 * resid / resid.size
    dgrads, dinp = decoder_backward(dec, dcache, dg)
    dq = dinp[:, m:].reshape(B, S, -1).sum(axis=1)
    egrads = encoder_backward(enc, ecache, dq)
    return loss, egrads, dgrads


def flatten(enc, dec):
    """All parameters in one vector, in the order of the library's packed image:
    decoder layers (W row-major, b), then encoder convs (w[6], b), then the two
    encoder dense layers (W row-major, b)."""
    parts = []
    for W, b in dec:
        parts += [np.ravel(W), np.ravel(b)]
    for w, b in enc["conv"]:
        parts += [np.ravel(w), np.atleast_1d(b)]
    for W, b in enc["dense"]:
        parts += [np.ravel(W), np.ravel(b)]
    return np.concatenate([np.asarray(p, np.float64) for p in parts])


def unflatten(vec, enc_like, dec_like):
    vec = np.asarray(vec, np.float64)
    o = 0

    def take(shape):
        nonlocal o
        n = int(np.prod(shape)) if shape else 1
        out = vec[o:o + n].reshape(shape) if shape else float(vec[o])
        o += n
        return out

    dec = [(take(np.shape(W)), take(np.shape(b))) for W, b in dec_like]
    conv = [(take(np.shape(w)), take(())) for w, b in enc_like["conv"]]
    dense = [(take(np.shape(W)), take(np.shape(b))) for W, b in enc_like["dense"]]
    return {"conv": conv, "dense": dense}, dec


def adam_step(p, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update of the parameter vector p (t = 1 for the first step).
    Returns (p, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mhat = m / (1 - b1 ** t)
    vhat = v / (1 - b2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v
