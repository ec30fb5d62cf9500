"""Pins of the robust-sampling oracle (paper App. B, Algorithm 1) on the CPU.

Calculate_Residual is checked against closed forms of a decoder linear in q (the
sine decoder: no dynamics, and one exact least-squares step); Max_Indices against
a brute-force sort; the greedy loop against its own definition recomputed from
independent calls (each added node is a top-n_try residual node, has the smallest
metric among the tried candidates, and the loop stops at the target)."""
import numpy as np

from oracle import crom_oracle as O
from oracle import sampling_oracle as SO
from workloads import gen


class SineDecoder:
    """g(x, q) = sum_k q_k sin(k pi x): linear in q, Lap g = -sum_k (k pi)^2 q_k sin(k pi x)."""

    def __init__(self, r):
        self.r = r

    def __call__(self, X, q):
        x = np.asarray(X, np.float64)[:, 0]
        k = np.arange(1, self.r + 1)
        S = np.sin(np.pi * np.outer(x, k))
        C = np.pi * k * np.cos(np.pi * np.outer(x, k))
        q = np.asarray(q, np.float64)
        return O.Evaluation(S @ q, (C @ q)[:, None], (-(S * (np.pi * k) ** 2) @ q)[:, None], S)


def _problem(r=3, P=33, n_params=2, seed=0):
    rng = np.random.default_rng(seed)
    nodes = (np.arange(P) / (P - 1))[:, None]
    q0s = rng.standard_normal((n_params, r))
    alphas = rng.uniform(0.5, 1.5, size=n_params)
    fom = rng.standard_normal((n_params, P)) * 0.1 + np.stack(
        [SineDecoder(r)(nodes, q).g for q in q0s])
    return nodes, q0s, alphas, fom


def test_residual_without_dynamics_is_the_pointwise_misfit():
    nodes, q0s, alphas, fom = _problem()
    dec = SineDecoder(3)
    res, ok = SO.calculate_residual(dec, [3, 9, 20], nodes, q0s, alphas, 1e-3, 1, 0, fom)
    x = nodes[:, 0]
    k = np.arange(1, 4)
    expect = sum(np.abs(np.sin(np.pi * np.outer(x, k)) @ q0s[m] - fom[m]) for m in range(2))
    assert ok and np.allclose(res, expect, rtol=1e-14, atol=1e-15)
    assert SO.metric(res) == float(np.mean(res) + np.max(res))


def test_residual_after_one_step_matches_the_least_squares_closed_form():
    nodes, q0s, alphas, fom = _problem()
    dec = SineDecoder(3)
    M = [2, 7, 11, 19, 25]
    dt = 1e-3
    res, ok = SO.calculate_residual(dec, M, nodes, q0s, alphas, dt, 1, 1, fom)
    x = nodes[:, 0]
    k = np.arange(1, 4)
    S_all = np.sin(np.pi * np.outer(x, k))
    S = S_all[M]
    expect = np.zeros(len(x))
    for m in range(2):
        lap = -(S * (np.pi * k) ** 2) @ q0s[m]
        q1 = q0s[m] + np.linalg.lstsq(S, dt * alphas[m] * lap, rcond=None)[0]
        expect += np.abs(S_all @ q1 - fom[m])
    assert ok and np.allclose(res, expect, rtol=1e-12, atol=1e-14)


def test_residual_of_an_ill_posed_set_is_infinite():
    nodes, q0s, alphas, fom = _problem()
    res, ok = SO.calculate_residual(SineDecoder(3), [4, 9], nodes, q0s, alphas, 1e-3, 1, 1, fom)  # |M| < r
    assert not ok and np.all(np.isinf(res))


def test_max_indices_against_sorting():
    rng = np.random.default_rng(3)
    res = np.round(rng.uniform(0, 1, 200), 2)   # many ties
    got = SO.max_indices(res, 12, exclude=[5, 17, 40])
    allowed = [i for i in range(200) if i not in (5, 17, 40)]
    expect = sorted(allowed, key=lambda i: (-res[i], i))[:12]
    assert got == expect


def test_greedy_loop_follows_its_definition():
    """A 1D heat problem with an MLP decoder: every step of the returned
    history is recomputed by independent calls."""
    spec = gen.DecoderSpec(1, 3, 16, 2)
    params = gen.xavier_decoder(spec, seed=4, bias_std=0.2)
    dec = O.MLPDecoder(params, 1)
    P = 25
    nodes = (np.arange(P) / (P - 1))[:, None]
    rng = np.random.default_rng(5)
    q0s = rng.standard_normal((2, 3))
    alphas = np.array([0.8, 1.2])
    fom = np.stack([dec.value(nodes, q) for q in q0s]) + 0.05 * rng.standard_normal((2, P))
    args = dict(dt=1e-3, gn_iters=1, n_steps=3)
    M, m_final, hist = SO.robust_sampling(dec, nodes, [3, 12, 20], q0s, alphas, args["dt"], args["gn_iters"],
                                          args["n_steps"], fom, n_try=4, target=0.0, max_samples=6)
    assert len(M) == 6 and M[:3] == [3, 12, 20] and len(set(M)) == 6
    cur = [3, 12, 20]
    for h in hist[:-1]:
        res, _ = SO.calculate_residual(dec, cur, nodes, q0s, alphas, args["dt"], args["gn_iters"], args["n_steps"], fom)
        assert abs(h["metric"] - SO.metric(res)) <= 1e-12 * h["metric"]
        assert h["candidates"] == SO.max_indices(res, 4, cur)
        cms = [SO.metric(SO.calculate_residual(dec, cur + [i], nodes, q0s, alphas, args["dt"], args["gn_iters"],
                                               args["n_steps"], fom)[0]) for i in h["candidates"]]
        assert h["chosen"] == h["candidates"][int(np.argmin(cms))]
        cur = cur + [h["chosen"]]
    assert cur == M
    # a reachable target stops the loop as soon as the metric falls below it
    M2, m2, hist2 = SO.robust_sampling(dec, nodes, [3, 12, 20], q0s, alphas, args["dt"], args["gn_iters"],
                                       args["n_steps"], fom, n_try=4, target=hist[1]["metric"] * 1.0000001,
                                       max_samples=10)
    assert len(M2) == 4 and m2 < hist[1]["metric"] * 1.0000001
