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


def subset(w, idx):
    """A StepWorkload restricted to the instances in idx (oracle-sized sample)."""
    from workloads import gen
    sizes = w.sizes[idx]
    samp = np.concatenate([w.samples[w.s_off[i]:w.s_off[i + 1]] for i in idx], axis=0)
    return gen.StepWorkload(w.name + "_subset", w.spec, w.params, w.q0[idx], w.alpha[idx],
                            gen.ragged_offsets(sizes), samp, w.dt, w.gn_iters, w.steps)
