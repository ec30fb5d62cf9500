"""Shared helpers of the GPU parity tests: device upload and error norms."""
import numpy as np


def rel_l2(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def make_ctx(spec, params, device=0):
    from workloads import gen
    from paper_2206_02607_gb300 import crom
    ctx = crom.crom_create(spec.m, spec.r, spec.width, spec.hidden, device)
    crom.crom_set_weights(ctx, gen.pack_params(params))
    return ctx


def dev(a, dtype):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


class StepInputs:
    """Device copies of a StepWorkload's arrays."""

    def __init__(self, w):
        import torch
        self.q = dev(w.q0, torch.float64)
        self.alpha = dev(w.alpha, torch.float32)
        self.s_off = dev(w.s_off, torch.int32)
        self.samples = dev(w.samples, torch.float32)
        self.status = torch.full((w.n_inst,), -1, dtype=torch.int32, device="cuda")
        self.max_samples = int(np.max(w.sizes)) if w.n_inst else 1


def run_steps(ctx, w, steps, precision, gn_iters=None, dt=None):
    import torch
    from paper_2206_02607_gb300 import crom
    d = StepInputs(w)
    for _ in range(steps):
        crom.crom_step(ctx, d.q, d.alpha, d.s_off, d.samples, d.status, dt=dt or w.dt,
                       gn_iters=gn_iters or w.gn_iters, max_samples=d.max_samples, precision=precision)
    torch.cuda.synchronize()
    return d.q.cpu().numpy(), d.status.cpu().numpy()


def kink_margin(params, Y, q):
    """Smallest |pre-activation| over all hidden units at any of the samples
    (plain test-side forward pass).  ELU is C^1 but not C^2: its s'' jumps from
    e^0 = 1 to 0 at z = 0, so the network Laplacian is discontinuous there and two
    correct evaluations in different precisions may take opposite branches at a
    sample that lies within rounding distance of a kink."""
    Y = np.asarray(Y, np.float64)
    h = np.concatenate([Y, np.broadcast_to(np.asarray(q, np.float64), (Y.shape[0], len(q)))], axis=1)
    margin = np.inf
    for W, b in params[:-1]:
        z = h @ np.asarray(W).T + np.asarray(b)
        margin = min(margin, float(np.abs(z).min()))
        h = np.where(z > 0, z, np.expm1(np.minimum(z, 0)))
    return margin


def increment_errors(params, m, q0, Y, q_gpu, q_ref, dt, alpha):
    """Errors of a GPU step against the oracle's, for one instance.

    Returns (inc, res, kappa, margin):
      inc    = ||d_gpu - d_ref|| / ||d_ref||, d = q_{n+1} - q_n (the latent increment);
      res    = ||J (d_gpu - d_ref)|| / ||Delta f|| with the FP64 Jacobian J = dg/dq(Y, q_n)
               and the oracle's PDE update Delta f at the samples: the error of the
               fitted field change, relative to the update being fitted (a backward-
               error measure of the least-squares projection);
      kappa  = condition number of J;
      margin = kink_margin at q_n.
    Least-squares perturbation theory bounds inc by about kappa times the relative
    errors of J and Delta f, so ill-conditioned instances legitimately show a larger
    `inc` while `res` stays at the level of the arithmetic."""
    from oracle import crom_oracle as O
    dec = O.MLPDecoder(params, m)
    ev = dec(Y, q0)
    J = ev.gq
    df = dt * np.asarray(alpha, np.float64) * ev.lap   # alpha: scalar or one value per sample
    d_gpu, d_ref = q_gpu - q0, q_ref - q0
    inc = float(np.linalg.norm(d_gpu - d_ref) / np.linalg.norm(d_ref))
    res = float(np.linalg.norm(J @ (d_gpu - d_ref)) / np.linalg.norm(df))
    return inc, res, float(np.linalg.cond(J)), kink_margin(params, Y, q0)


def subset(w, idx):
    """A StepWorkload restricted to the instances in idx (oracle-sized sample)."""
    from workloads import gen
    sizes = w.sizes[idx]
    samp = np.concatenate([w.samples[w.s_off[i]:w.s_off[i + 1]] for i in idx], axis=0)
    return gen.StepWorkload(w.name + "_subset", w.spec, w.params, w.q0[idx], w.alpha[idx],
                            gen.ragged_offsets(sizes), samp, w.dt, w.gn_iters, w.steps)
