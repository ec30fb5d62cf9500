"""FP64 oracle of the robust (greedy) integration-sample selection, paper App. B
(Algorithm 1, "Robust sampling").

TEST INFRASTRUCTURE ONLY: imported by tests/ and nothing on the product path.

The algorithm, in the paper's order:
  * Calculate_Residual(M): for every training parameter mu, run the latent
    dynamics with integration samples M to the final step, q_T(mu); add
    |g(x_i, q_T(mu)) - f_FOM(x_i, T; mu)| into res[i] for every FOM node x_i.
  * Metric(res) = mean(res) + max(res).
  * Start from an initial M; while Metric(Calculate_Residual(M)) >= target: take
    the n_try nodes with the largest individual residuals, evaluate
    Metric(Calculate_Residual(M + {x_i})) for each, add the one with the smallest.

Readings where the paper is silent (kept identical on the GPU side):
  * candidates exclude nodes already in M (adding a member leaves the set
    unchanged);
  * ties: larger residual first, equal residuals by lower node index; equal
    metrics keep the earlier candidate;
  * a rollout whose step reports a non-OK status makes that set's metric +inf;
  * the loop also stops when |M| reaches max_samples.
"""
from __future__ import annotations

import numpy as np

from .crom_oracle import STATUS_OK, crom_step

__all__ = ["calculate_residual", "metric", "max_indices", "robust_sampling"]


def calculate_residual(decoder, M, nodes, q0s, alphas, dt, gn_iters, n_steps, fom_final):
    """res[i] = sum_mu |g(x_i, q_T(mu)) - f_FOM(x_i, T; mu)| (Algorithm 1's
    Calculate_Residual).  Returns (res, ok): ok is False when a step failed."""
    nodes = np.asarray(nodes, np.float64)
    Y = nodes[np.asarray(M, np.int64)]
    res = np.zeros(nodes.shape[0])
    for mu in range(len(q0s)):
        q = np.asarray(q0s[mu], np.float64)
        for _ in range(n_steps):
            q, st = crom_step(decoder, q, Y, dt, gn_iters, alpha=float(alphas[mu]))
            if st != STATUS_OK:
                return np.full(nodes.shape[0], np.inf), False
        g = decoder.value(nodes, q) if hasattr(decoder, "value") else decoder(nodes, q).g
        res += np.abs(g - np.asarray(fom_final[mu], np.float64))
    return res, True


def metric(res):
    """Algorithm 1's Metric: mean plus max of the per-node residuals."""
    res = np.asarray(res, np.float64)
    return float(np.mean(res) + np.max(res))


def max_indices(res, k, exclude):
    """The k nodes with the largest residuals, not in `exclude` (ties: lower index)."""
    res = np.asarray(res, np.float64)
    excl = set(int(e) for e in exclude)
    order = sorted((i for i in range(res.shape[0]) if i not in excl), key=lambda i: (-res[i], i))
    return order[:k]


def robust_sampling(decoder, nodes, init, q0s, alphas, dt, gn_iters, n_steps, fom_final, n_try, target,
                    max_samples):
    """Greedy robust sampling.  Returns (M, final metric, history), history being a
    list of dicts {metric, candidates, candidate_metrics, chosen} per iteration."""
    M = [int(i) for i in init]
    res, _ = calculate_residual(decoder, M, nodes, q0s, alphas, dt, gn_iters, n_steps, fom_final)
    history = []
    while True:
        m = metric(res)
        if m < target or len(M) >= max_samples:
            history.append({"metric": m, "candidates": [], "candidate_metrics": [], "chosen": None})
            return M, m, history
        cand = max_indices(res, n_try, M)
        best, best_m, best_res, cms = None, np.inf, None, []
        for i in cand:
            r_i, _ = calculate_residual(decoder, M + [i], nodes, q0s, alphas, dt, gn_iters, n_steps, fom_final)
            m_i = metric(r_i)
            cms.append(m_i)
            if best is None or m_i < best_m:
                best, best_m, best_res = i, m_i, r_i
        history.append({"metric": m, "candidates": cand, "candidate_metrics": cms, "chosen": best})
        if best is None:
            return M, m, history
        M.append(best)
        res = best_res
