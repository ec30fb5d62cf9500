"""Benchmark of the CROM latent-space step on GB300.

Workload: 1024 independent 2D heat instances sharing one decoder R^{2+8} -> R
(5 ELU layers of width 128), alpha ~ U(0.5, 2), |M_i| ~ U{32..512} integration
samples, 2 Gauss-Newton iterations, dt = 1e-5 (seeded synthetic inputs from
workloads.gen.heat2d_batched).  One bench step = one crom_step call advancing
every instance by one latent step (decode with derivatives, PDE update,
Gauss-Newton projection) on the tensor-core path (f16 hi/lo activation operands,
f16 weights, FP32 accumulation, FP64 normal equations).

Printed (one JSON line on rank 0): instance-steps/s of that step with inputs
resident in HBM (L2 flushed before every timed step), the same metric end to
end through the C ABI with host buffers, the plain FP32 single-instance path
on the 200-sample 2D heat problem (the reference point of the batched speed-up),
dense reconstruction throughput, the roofline of the step kernel, clocks, and the
FP64 oracle timed on a bounded sample on the host cores.

--impl reference times the FP64 oracle (the only reference available: the paper
ships no code) on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "instance-steps/s, batched BF16 vs plain FP32 same GB300, rel-L2<=1e-3 vs FP64"
WORKLOAD = "heat2d_batched_1024inst_M32-512_r8_w128_L5_gn2"


# dram__bytes_read.sum + dram__bytes_write.sum of one step_tc_kernel launch on the
# 1024-instance workload, from an ncu capture of the current kernel; None until it has
# been taken for the current kernel.
STEP_KERNEL_DRAM_BYTES = 2596096 + 0   # ncu dram__bytes_read.sum + write.sum of one launch (1024 instances)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--n-inst", type=int, default=1024)
    ap.add_argument("--n-codes", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fom-fields", type=int, default=512)
    ap.add_argument("--tiles", default="auto",
                    help="sample tiles of the tensor-core step: auto (measured by crom_autotune) or s0,s1 "
                         "(fixed; profilers distort the autotuner's timings)")
    ap.add_argument("--prec", default="f16x2", choices=["f16x2", "f16"],
                    help="tensor-core precision of --only step / recon")
    ap.add_argument("--only", default=None, choices=["step", "recon", "plain", "fom", "heat", "train", "decode"],
                    help="run only one part (warmup + steps launches) for profiling; prints a short JSON line")
    return ap.parse_args()


def run_only(args):
    """Profiling driver: the named part alone, on the bench's workloads."""
    import torch
    from paper_2206_02607_gb300 import build
    build()
    from paper_2206_02607_gb300 import crom
    from workloads import gen
    torch.cuda.set_device(0)
    n = args.warmup + args.steps
    if args.only in ("step", "plain"):
        w = gen.heat2d_batched(n_inst=args.n_inst) if args.only == "step" else gen.heat2d_single()
        tc_prec = crom.CROM_PREC_F16X2 if args.prec == "f16x2" else crom.CROM_PREC_F16
        prec = tc_prec if args.only == "step" else crom.CROM_PREC_FP32
        ctx = crom.crom_create(w.spec.m, w.spec.r, w.spec.width, w.spec.hidden, 0)
        crom.crom_set_weights(ctx, gen.pack_params(w.params))
        q = torch.tensor(w.q0, device="cuda")
        a, o = torch.tensor(w.alpha, device="cuda"), torch.tensor(w.s_off, device="cuda")
        s, st = torch.tensor(w.samples, device="cuda"), torch.zeros(w.n_inst, dtype=torch.int32, device="cuda")
        for _ in range(n):
            crom.crom_step(ctx, q, a, o, s, st, dt=w.dt, gn_iters=w.gn_iters, max_samples=int(w.sizes.max()),
                           precision=prec)
        torch.cuda.synchronize()
        print(json.dumps({"only": args.only, "instances": w.n_inst, "calls": n,
                          "status_all_ok": bool((st.cpu().numpy() == 0).all())}))
    elif args.only == "decode":
        # crom_decode_tc (value, dg/dx, Laplacian, dg/dq) at the batch's integration samples
        w = gen.heat2d_batched(n_inst=args.n_inst)
        ctx = crom.crom_create(w.spec.m, w.spec.r, w.spec.width, w.spec.hidden, 0)
        crom.crom_set_weights(ctx, gen.pack_params(w.params))
        prec = crom.CROM_PREC_F16X2 if args.prec == "f16x2" else crom.CROM_PREC_F16
        q, o = torch.tensor(w.q0, device="cuda"), torch.tensor(w.s_off, device="cuda")
        x = torch.tensor(w.samples, device="cuda")
        out = torch.empty((4 + w.spec.r, x.shape[0]), dtype=torch.float32, device="cuda")
        want = crom.CROM_WANT_VAL | crom.CROM_WANT_DX | crom.CROM_WANT_LAP | crom.CROM_WANT_DQ
        for _ in range(n):
            crom.crom_decode_tc(ctx, q, o, x, want, out, precision=prec)
        torch.cuda.synchronize()
        print(json.dumps({"only": "decode", "instances": w.n_inst, "points": x.shape[0], "calls": n}))
    elif args.only == "train":
        # the learned-model training step (64 snapshots x 4096 points, width 256), bf16 tensor-core pass
        Bt, St, nt_side, rt, wt, Lt = 64, 4096, 256, 16, 256, 5
        rng = np.random.default_rng(0)
        tr = crom.CromTrainer(2, rt, wt, Lt, nt_side * nt_side, Bt, St, 0)
        tr.set_precision(crom.CROM_PREC_BF16_MIXED)
        tr.set_params((rng.standard_normal(tr.n_params) * 0.05).astype(np.float32))
        snaps_t = torch.tensor(rng.standard_normal((Bt, nt_side * nt_side)).astype(np.float32), device="cuda")
        idx_t = torch.tensor(rng.integers(0, nt_side * nt_side, size=(Bt, St)).astype(np.int32), device="cuda")
        coords_t = torch.tensor(gen.grid_points_2d(nt_side), device="cuda")
        loss_t = torch.zeros(1, dtype=torch.float64, device="cuda")
        for _ in range(n):
            crom.crom_train_step(tr, snaps_t, idx_t, coords_t, 1e-4, loss_t)
        torch.cuda.synchronize()
        print(json.dumps({"only": "train", "steps": n, "loss": float(loss_t.item())}))
        tr.close()
        return
    elif args.only == "fom":
        nb, nn = args.fom_fields, 256
        rng = np.random.default_rng(0)
        u = torch.tensor(rng.uniform(0, 1, size=(nb, nn, nn)).astype(np.float32), device="cuda")
        ax = torch.tensor(rng.uniform(-0.5, 0.5, size=(nb, nn, nn)).astype(np.float32), device="cuda")
        ay = torch.tensor(rng.uniform(-0.5, 0.5, size=(nb, nn, nn)).astype(np.float32), device="cuda")
        nu = torch.full((nb,), 5e-3, dtype=torch.float32, device="cuda")
        tmp = torch.empty_like(u)
        crom.crom_fom_step(crom.CROM_FOM_ADVDIFF2D_PERIODIC, u, tmp, nu, dt=2.5e-5, n_steps=n, ax=ax, ay=ay)
        torch.cuda.synchronize()
        print(json.dumps({"only": "fom", "fields": nb, "nodes": nn * nn, "steps": n}))
        return
    elif args.only == "heat":
        nb, nn = args.fom_fields, 256
        rng = np.random.default_rng(0)
        u = torch.tensor(rng.uniform(0, 1, size=(nb, nn, nn)).astype(np.float32), device="cuda")
        tmp = torch.empty_like(u)
        al = torch.full((nb,), 1.0, dtype=torch.float32, device="cuda")
        crom.crom_fom_step(crom.CROM_FOM_HEAT2D_NEUMANN, u, tmp, al, dt=(1.0 / (nn - 1)) ** 2 / 8, n_steps=n)
        torch.cuda.synchronize()
        print(json.dumps({"only": "heat", "fields": nb, "nodes": nn * nn, "steps": n}))
        return
    else:
        spec, params, codes, X = gen.recon_dense(n_codes=args.n_codes)
        ctx = crom.crom_create(spec.m, spec.r, spec.width, spec.hidden, 0)
        crom.crom_set_weights(ctx, gen.pack_params(params))
        c, x = torch.tensor(codes, device="cuda"), torch.tensor(X, device="cuda")
        out = torch.empty((codes.shape[0], X.shape[0]), device="cuda")
        for _ in range(n):
            crom.crom_reconstruct(ctx, c, x, out,
                                  precision=crom.CROM_PREC_F16X2 if args.prec == "f16x2" else crom.CROM_PREC_F16)
        torch.cuda.synchronize()
        print(json.dumps({"only": "recon", "codes": codes.shape[0], "points": X.shape[0], "calls": n}))
    ctx.close()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def step_flops_per_sample(w=128, L=5, m=2, r=8, gn_iters=2):
    """Algorithmic FLOPs of one sample for the tensor-core step as implemented:
    forward channels (value, m gradients, 1 Laplacian) at iteration 0, (value,
    difference) later, one reverse pass per iteration, output and Jacobian
    projections.  Each w x w contraction costs 2 w^2 per column."""
    ww = 2 * w * w * (L - 1)
    f = 0
    for it in range(gn_iters):
        nch = 2 + m if it == 0 else 2
        f += nch * ww + ww                    # forward channels + reverse pass
        f += 2 * w * nch + 2 * w * r          # output projection + Jacobian projection
        f += 2 * (m + r) * w                  # layer 1 (CUDA cores)
    return f


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return pk["bf16_tflops"], pk["hbm_gbs"], "measured"
    except Exception:
        return 1900.0, 6800.0, "fallback"


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "25"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(1.0)   # nvidia-smi needs a moment before its first sample
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0])); mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_rate(w, budget_s=12.0, max_inst=512):
    """FP64 oracle (single process) on the first instances of the workload until
    the time budget is used; returns (instance-steps/s, instances done)."""
    from oracle import crom_oracle as O
    dec = O.MLPDecoder(w.params, w.spec.m)
    t0 = time.perf_counter()
    done = 0
    samples = 0
    for i in range(min(w.n_inst, max_inst)):
        Y = w.samples[w.s_off[i]:w.s_off[i + 1]]
        O.crom_step(dec, w.q0[i], Y, w.dt, w.gn_iters, alpha=float(w.alpha[i]))
        done += 1
        samples += Y.shape[0]
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    # normalise to the workload's mean |M_i| so the unit matches instance-steps/s of the full batch
    mean_all = float(np.mean(w.sizes))
    rate_samples = samples / el
    return rate_samples / mean_all, done, samples, el


# ---- the FP64 oracle on every host core: a process pool (spawn start method: a
# forked child of a process that has used CUDA can hang), one numpy thread per
# worker, each worker stepping whole instances of the workload
_POOL_W = None


def _pool_init(params, m, q0, s_off, samples, alpha, dt, gn_iters):
    global _POOL_W
    _POOL_W = (params, m, q0, s_off, samples, alpha, dt, gn_iters)


def _pool_steps(idx):
    from oracle import crom_oracle as O
    params, m, q0, s_off, samples, alpha, dt, gn_iters = _POOL_W
    dec = O.MLPDecoder(params, m)
    n = 0
    for i in idx:
        Y = samples[s_off[i]:s_off[i + 1]]
        O.crom_step(dec, q0[i], Y, dt, gn_iters, alpha=float(alpha[i]))
        n += Y.shape[0]
    return n


class OraclePool:
    """The oracle as it stands, run on all host cores (one instance per task)."""

    def __init__(self, w, cores=None):
        import multiprocessing as mp
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[k] = "1"      # inherited by the workers: one thread each
        self.cores = cores or os.cpu_count() or 1
        self.w = w
        self.pool = mp.get_context("spawn").Pool(
            self.cores, initializer=_pool_init,
            initargs=(w.params, w.spec.m, w.q0, w.s_off, w.samples, w.alpha, w.dt, w.gn_iters))
        # start-up outside any timing; every wait on the pool is bounded (a worker that
        # dies leaves a plain map() waiting forever)
        self.pool.map_async(_pool_steps, [[] for _ in range(self.cores)]).get(timeout=300)

    def rate(self, n_inst):
        """Steps the first n_inst instances once; returns (instance-steps/s normalised by
        the workload's mean |M_i|, samples, seconds)."""
        idx = [[i] for i in range(min(n_inst, self.w.n_inst))]
        t0 = time.perf_counter()
        samples = sum(self.pool.map_async(_pool_steps, idx, chunksize=1).get(timeout=600))
        el = time.perf_counter() - t0
        return samples / el / float(np.mean(self.w.sizes)), samples, el

    def close(self):
        self.pool.terminate()
        self.pool.join()


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def bench_config(n_inst, world, samples_per_step):
    """The workload's config, shared by both arms of the bench."""
    return {"workload": WORKLOAD, "global_batch": world * n_inst, "samples_per_step": samples_per_step,
            "parallelism": f"instances sharded, {n_inst} per GPU" if world > 1 else "single GPU",
            "l2": "flushed (256 MB write) before every timed step (GPU arm)"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from workloads import gen
    w = gen.heat2d_batched(n_inst=args.n_inst)
    pool = OraclePool(w)
    n_sample = 4 * pool.cores        # instances per reference step: a bounded sample of the batch
    times = []
    for k in range(args.warmup + args.steps):
        rate, samples, el = pool.rate(n_sample)
        if k >= args.warmup:
            times.append(rate)
    pool.close()
    value = float(np.mean(times))
    line = {"metric": METRIC, "value": value, "unit": "instance-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * args.n_inst / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": bench_config(args.n_inst, 1, int(w.sizes.sum())),
            "cpu_baseline": {"value": value, "unit": "instance-steps/s", "cores": pool.cores, "kind": "oracle",
                             "cpu": cpu_model(),
                             "sample": f"each step: the FP64 numpy oracle on the first {n_sample} instances of "
                                       f"the workload, one instance per task on {pool.cores} worker processes; "
                                       f"rate normalised by the workload's mean |M_i| (ms_per_step is the full "
                                       f"{args.n_inst}-instance batch at that rate)"},
            "e2e": {"value": value, "unit": "instance-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def measure_next_rows(crom, gen, ctx, w, q0, alpha, s_off, samples, status, stream, flush, local):
    """The paper's further rows on the bench's GPU, each on a workload of its own
    (CUDA events; L2 flushed before each timed step on the 1024-instance batch):
    f1 the backtracking line search, f3 a per-sample coefficient, f4 a SIREN decoder
    (FP32 path) and the tangent velocity, f2 greedy robust sample selection."""
    import torch
    out = {}
    max_s = int(w.sizes.max())
    q = torch.empty_like(q0)

    def timed(fn, reps, flush_l2=True):
        fn()
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(reps):
            if flush_l2:
                flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        return tot / reps

    # f1: line search (value-only trial passes).  At the bench's dt the first GN
    # iteration accepts its full step; in the second the trial objective equals the
    # Armijo bound up to rounding, so the decisions there can go either way.  At
    # dt = 0.1 most full steps overshoot and backtrack.
    for name, dt in (("line_search_bench_dt", w.dt), ("line_search_dt_0.1", 0.1)):
        def f1():
            q.copy_(q0)
            crom.crom_step(ctx, q, alpha, s_off, samples, status, dt=dt, gn_iters=w.gn_iters, max_samples=max_s,
                           precision=crom.CROM_PREC_F16X2, line_search=4)
        ms = timed(f1, 5)
        out[name] = {"ms_per_step": ms, "instance_steps_per_s": w.n_inst / (ms * 1e-3), "halvings_max": 4,
                     "workload": f"1024 instances of the step's workload, dt = {dt:g}, 2 GN iterations, "
                                 "up to 4 halvings"}
    # f3: per-sample coefficient nu(y_j) (the instance's alpha repeated at its samples)
    alpha_s = torch.repeat_interleave(alpha, torch.tensor(w.sizes, device="cuda"))

    def f3():
        q.copy_(q0)
        crom.crom_step(ctx, q, alpha_s, s_off, samples, status, dt=w.dt, gn_iters=w.gn_iters, max_samples=max_s,
                       precision=crom.CROM_PREC_F16X2, coef_per_sample=True)
    ms = timed(f3, 5)
    out["coef_per_sample"] = {"ms_per_step": ms, "instance_steps_per_s": w.n_inst / (ms * 1e-3),
                              "workload": "1024 instances, alpha per sample"}
    # f4: SIREN decoder (omega0 = 30) on the FP32 CUDA-core path, 64 instances
    spec = gen.DecoderSpec(2, 8, 128, 5)
    ctx_s = crom.crom_create(2, 8, 128, 5, local, activation=crom.CROM_ACT_SIREN, omega0=30.0)
    crom.crom_set_weights(ctx_s, gen.pack_params(gen.siren_decoder(spec, seed=3)))
    n64 = 64
    s64 = torch.tensor((2.0 * w.samples[:w.s_off[n64]] - 1.0).astype(np.float32), device="cuda")
    q64 = (q0[:n64] * 0.5).contiguous()
    qs = torch.empty_like(q64)

    def f4():
        qs.copy_(q64)
        crom.crom_step(ctx_s, qs, alpha[:n64].contiguous(), s_off[:n64 + 1].contiguous(), s64, status[:n64],
                       dt=1e-6, gn_iters=w.gn_iters, max_samples=max_s, precision=crom.CROM_PREC_FP32)
    ms = timed(f4, 5, flush_l2=False)
    out["siren_fp32_step"] = {"ms_per_step": ms, "instance_steps_per_s": n64 / (ms * 1e-3),
                              "workload": "64 instances of the step's workload on [-1, 1]^2, SIREN width 128 x 5"}
    ctx_s.close()
    # f4: tangent velocity dg/dq . qdot at the integration samples of the 1024 instances
    # (one FP32 forward-mode directional channel seeded with W_1q qdot)
    n_pts = int(w.s_off[-1])
    vout = torch.empty(n_pts, device="cuda")
    qprev = q0 * 0.999

    def f4t():
        crom.crom_tangent_velocity(ctx, q0, qprev, s_off, samples, vout, dt=1e-3)
    ms = timed(f4t, 5)
    out["tangent_velocity"] = {"ms": ms, "points_per_s": n_pts / (ms * 1e-3),
                               "workload": f"the {n_pts} integration samples of the 1024 instances, r = 8"}
    # f2: greedy robust sampling (Algorithm 1) on a 1D heat problem: 257 nodes, 4
    # training parameters, 8 initial samples grown to 24, 8 candidates per round,
    # 20-step candidate rollouts; the "full-order" fields are synthetic sines
    spec1 = gen.DecoderSpec(1, 4, 128, 3)
    ctx1 = crom.crom_create(1, 4, 128, 3, local)
    crom.crom_set_weights(ctx1, gen.pack_params(gen.xavier_decoder(spec1, seed=9, bias_std=0.1)))
    P = 257
    xs = np.arange(P) / (P - 1)
    nodes = torch.tensor(xs.astype(np.float32)[:, None], device="cuda")
    rng = np.random.default_rng(21)
    q0r = torch.tensor(rng.standard_normal((4, 4)) * 0.5, device="cuda")
    coef = torch.tensor(rng.uniform(0.5, 1.5, 4).astype(np.float32), device="cuda")
    fom = torch.tensor(np.stack([np.sin((k + 1) * np.pi * xs) * 0.1 for k in range(4)]).astype(np.float32),
                       device="cuda")
    init = list(np.linspace(8, P - 9, 8).astype(int))
    for prec_name in ("CROM_PREC_FP32", "CROM_PREC_F16X2"):
        t0 = time.perf_counter()
        idx, met = crom.crom_robust_samples(ctx1, q0r, coef, nodes, fom, init, dt=3e-4, gn_iters=1, n_steps=20,
                                            n_try=8, target=0.0, max_samples=24,
                                            precision=getattr(crom, prec_name))
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        rounds = len(idx) - len(init)
        out["robust_sampling_" + prec_name[10:].lower()] = {
            "s": sec, "rounds": rounds, "candidate_rollouts_per_s": rounds * 8 * 4 / sec,
            "workload": "1D heat, 257 nodes, 4 parameters, |M| 8 -> 24, 8 candidates per round, 20-step rollouts"}
    ctx1.close()
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.only:
        run_only(args)
        return
    import torch
    from paper_2206_02607_gb300 import build
    build()
    from paper_2206_02607_gb300 import crom
    from workloads import gen

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist

    def barrier():
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()

    w = gen.heat2d_batched(n_inst=args.n_inst, first=rank * args.n_inst)   # each rank: its own instances
    ctx = crom.crom_create(w.spec.m, w.spec.r, w.spec.width, w.spec.hidden, local)
    crom.crom_set_weights(ctx, gen.pack_params(w.params))
    q0 = torch.tensor(w.q0, dtype=torch.float64, device="cuda")
    q = q0.clone()
    alpha = torch.tensor(w.alpha, device="cuda")
    s_off = torch.tensor(w.s_off, device="cuda")
    samples = torch.tensor(w.samples, device="cuda")
    status = torch.zeros(w.n_inst, dtype=torch.int32, device="cuda")
    max_s = int(w.sizes.max())
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")   # > 129 MB L2

    def step(prec=crom.CROM_PREC_F16X2, qq=None):
        crom.crom_step(ctx, q if qq is None else qq, alpha, s_off, samples, status, dt=w.dt,
                       gn_iters=w.gn_iters, max_samples=max_s, precision=prec)

    # ---- tile shape of the tensor-core step: measured on this batch (outside the timed region)
    if args.tiles == "auto":
        tile_s0, tile_s1, tile_ms = crom.crom_autotune(ctx, q, alpha, s_off, samples, status, dt=w.dt,
                                                       gn_iters=w.gn_iters, max_samples=max_s)
    else:
        crom.crom_set_step_tiles(ctx, *[int(v) for v in args.tiles.split(",")])
        tile_s0, tile_s1, tile_ms = crom.crom_get_step_tiles(ctx)

    # ---- device-resident timing, L2 flushed before each timed step
    for _ in range(args.warmup):
        step()
    barrier()
    sampler = ClockSampler(local)
    evs = []
    for _ in range(args.steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        evs.append((e0, e1))
    barrier()
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    ms = float(np.mean(step_ms))
    if pg is not None:
        t = torch.tensor([ms], device="cuda")
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        ms = float(t.item())
    st = status.cpu().numpy()
    value = world * w.n_inst / (ms * 1e-3)

    # ---- accuracy of the timed configuration: sampled instances vs the FP64 oracle (rank 0)
    acc_ids = np.random.default_rng(0).choice(w.n_inst, size=6, replace=False)
    acc_ref = {}

    def accuracy(prec):
        from oracle import crom_oracle as O
        qa = q0.clone()
        step(prec, qq=qa)
        torch.cuda.synchronize()
        qg = qa.cpu().numpy()
        dec = O.MLPDecoder(w.params, 2)
        errs, incs = [], []
        for i in acc_ids:
            if i not in acc_ref:
                Y = w.samples[w.s_off[i]:w.s_off[i + 1]]
                acc_ref[i] = O.crom_step(dec, w.q0[i], Y, w.dt, w.gn_iters, alpha=float(w.alpha[i]))[0]
            ref = acc_ref[i]
            errs.append(np.linalg.norm(qg[i] - ref) / np.linalg.norm(ref))
            incs.append(np.linalg.norm((qg[i] - w.q0[i]) - (ref - w.q0[i])) / np.linalg.norm(ref - w.q0[i]))
        return {"q_rel_l2_max": float(max(errs)), "increment_rel_l2_max": float(max(incs)), "instances": 6}

    acc = accuracy(crom.CROM_PREC_F16X2) if rank == 0 else None

    # ---- the same step with single f16 activations (CROM_PREC_F16): time and accuracy
    def time_step(prec, n):
        for _ in range(3):
            step(prec)
        torch.cuda.synchronize()
        evs_p = []
        for _ in range(n):
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step(prec)
            b.record(stream)
            evs_p.append((a, b))
        torch.cuda.synchronize()
        return float(np.mean([a.elapsed_time(b) for a, b in evs_p]))

    f16_ms = time_step(crom.CROM_PREC_F16, min(args.steps, 100))
    f16_acc = accuracy(crom.CROM_PREC_F16) if rank == 0 else None

    # ---- Step 1 alone on the tensor cores (crom_decode_tc): value, dg/dx, Laplacian and
    # dg/dq at the batch's 273,723 integration samples
    want_all = crom.CROM_WANT_VAL | crom.CROM_WANT_DX | crom.CROM_WANT_LAP | crom.CROM_WANT_DQ
    dec_out = torch.empty((1 + 2 + 1 + w.spec.r, samples.shape[0]), dtype=torch.float32, device="cuda")

    def time_decode(prec, n=20):
        for _ in range(3):
            crom.crom_decode_tc(ctx, q0, s_off, samples, want_all, dec_out, precision=prec)
        torch.cuda.synchronize()
        evs_d = []
        for _ in range(n):
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            crom.crom_decode_tc(ctx, q0, s_off, samples, want_all, dec_out, precision=prec)
            b.record(stream)
            evs_d.append((a, b))
        torch.cuda.synchronize()
        return float(np.mean([a.elapsed_time(b) for a, b in evs_d]))

    dec_ms = time_decode(crom.CROM_PREC_F16X2)
    dec_ms_f16 = time_decode(crom.CROM_PREC_F16)
    # forward channels (value, dg/dx_1, dg/dx_2, Laplacian) and one reverse pass over the
    # 4 hidden matrices, 2 w^2 FLOP each
    dec_flops = int(w.sizes.sum()) * 5 * 4 * 2 * 128 * 128

    # ---- end to end through the C ABI on host arrays (crom_step_host: the library
    # copies the pinned inputs in, steps, copies q and status out and synchronises)
    hq0 = torch.tensor(w.q0, dtype=torch.float64)
    hq = hq0.clone().pin_memory()
    ha = torch.tensor(w.alpha).pin_memory()
    ho = torch.tensor(w.s_off).pin_memory()
    hs = torch.tensor(w.samples).pin_memory()
    hst = torch.empty(w.n_inst, dtype=torch.int32).pin_memory()
    h2d = hq.numel() * 8 + ha.numel() * 4 + ho.numel() * 4 + hs.numel() * 4
    d2h = hq.numel() * 8 + hst.numel() * 4

    def e2e_step():
        hq.copy_(hq0)  # every step starts from the same state
        crom.crom_step_host(ctx, hq, ha, ho, hs, hst, dt=w.dt, gn_iters=w.gn_iters, max_samples=max_s,
                            precision=crom.CROM_PREC_F16X2)

    # wall-clock timing of host-synchronised steps: at least 100 of them, so that a
    # host-side hiccup of a few ms does not dominate a short run
    n_e2e = max(args.steps, 100)
    for _ in range(5):
        e2e_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        e2e_step()
    barrier()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / n_e2e
    e2e_ok = bool((hst.numpy() == 0).all())
    e2e_value = world * w.n_inst / (e2e_ms * 1e-3)

    # ---- kernel-only duration of the step kernel for the roofline (same stream)
    # (two launches per call: the ordering kernel and the persistent step kernel)
    flops = step_flops_per_sample() * int(w.sizes.sum())
    peak_tf, hbm, peak_kind = load_peaks()
    achieved_tf = flops / (ms * 1e-3) / 1e12

    # ---- plain FP32 single-instance path (200-sample 2D heat problem)
    ws = gen.heat2d_single()
    ctx32 = crom.crom_create(2, 8, 128, 5, local)
    crom.crom_set_weights(ctx32, gen.pack_params(ws.params))
    q32 = torch.tensor(ws.q0, dtype=torch.float64, device="cuda")
    a32 = torch.tensor(ws.alpha, device="cuda")
    o32 = torch.tensor(ws.s_off, device="cuda")
    s32 = torch.tensor(ws.samples, device="cuda")
    st32 = torch.zeros(1, dtype=torch.int32, device="cuda")

    def step32():
        crom.crom_step(ctx32, q32, a32, o32, s32, st32, dt=ws.dt, gn_iters=ws.gn_iters, max_samples=200,
                       precision=crom.CROM_PREC_FP32)

    for _ in range(5):
        step32()
    torch.cuda.synchronize()
    n32 = 200
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n32):
        step32()
    e1.record(stream)
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1) / n32
    plain_value = 1.0 / (plain_ms * 1e-3)

    # ---- dense reconstruction 1024^2 points x 64 codes
    spec, params, codes, X = gen.recon_dense()
    ctxr = crom.crom_create(spec.m, spec.r, spec.width, spec.hidden, local)
    crom.crom_set_weights(ctxr, gen.pack_params(params))
    dcodes = torch.tensor(codes, device="cuda")
    dX = torch.tensor(X, device="cuda")
    out = torch.empty((codes.shape[0], X.shape[0]), dtype=torch.float32, device="cuda")

    def time_recon(prec):
        crom.crom_reconstruct(ctxr, dcodes, dX, out, precision=prec)
        torch.cuda.synchronize()
        rt = []
        for _ in range(3):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            crom.crom_reconstruct(ctxr, dcodes, dX, out, precision=prec)
            e1.record(stream)
            torch.cuda.synchronize()
            rt.append(e0.elapsed_time(e1))
        return float(np.median(rt))

    recon_ms_f16 = time_recon(crom.CROM_PREC_F16)
    recon_ms = time_recon(crom.CROM_PREC_F16X2)
    recon_pts = codes.shape[0] * X.shape[0]
    recon_flops = recon_pts * 2 * (2 * 128 + 4 * 128 * 128 + 128)

    # ---- rollout: 1000 steps of the same batch replayed from one cached CUDA graph
    qr = q0.clone()
    n_roll = 1000
    crom.crom_rollout(ctx, qr, alpha, s_off, samples, status, n_steps=n_roll, dt=w.dt, gn_iters=w.gn_iters,
                      max_samples=max_s, precision=crom.CROM_PREC_F16X2)   # records the graph
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    crom.crom_rollout(ctx, qr, alpha, s_off, samples, status, n_steps=n_roll, dt=w.dt, gn_iters=w.gn_iters,
                      max_samples=max_s, precision=crom.CROM_PREC_F16X2)
    e1.record(stream)
    torch.cuda.synchronize()
    roll_ms = e0.elapsed_time(e1) / n_roll

    # ---- GPU full-order model: 2D advection-diffusion, 512 fields of 256^2 (> L2)
    nb, nn = 512, 256
    rng = np.random.default_rng(0)
    u_f = torch.tensor(rng.uniform(0, 1, size=(nb, nn, nn)).astype(np.float32), device="cuda")
    tmp_f = torch.empty_like(u_f)
    ax_f = torch.tensor(rng.uniform(-0.5, 0.5, size=(nb, nn, nn)).astype(np.float32), device="cuda")
    ay_f = torch.tensor(rng.uniform(-0.5, 0.5, size=(nb, nn, nn)).astype(np.float32), device="cuda")
    nu_f = torch.full((nb,), 5e-3, dtype=torch.float32, device="cuda")
    fom_steps = 20
    crom.crom_fom_step(crom.CROM_FOM_ADVDIFF2D_PERIODIC, u_f, tmp_f, nu_f, dt=2.5e-5, n_steps=2, ax=ax_f, ay=ay_f)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    crom.crom_fom_step(crom.CROM_FOM_ADVDIFF2D_PERIODIC, u_f, tmp_f, nu_f, dt=2.5e-5, n_steps=fom_steps, ax=ax_f, ay=ay_f)
    e1.record(stream)
    torch.cuda.synchronize()
    fom_ms = e0.elapsed_time(e1) / fom_steps
    fom_nodes = nb * nn * nn
    fom_gbs = fom_nodes * 16 / (fom_ms * 1e-3) / 1e9
    del u_f, tmp_f, ax_f, ay_f
    # ---- GPU full-order model: 2D heat, zero-flux boundaries, 1024 fields of 256^2 (268 MB > L2)
    nbh = 1024
    u_h = torch.tensor(rng.uniform(0, 1, size=(nbh, nn, nn)).astype(np.float32), device="cuda")
    tmp_h = torch.empty_like(u_h)
    al_h = torch.full((nbh,), 1.0, dtype=torch.float32, device="cuda")
    dt_h = (1.0 / (nn - 1)) ** 2 / 8
    crom.crom_fom_step(crom.CROM_FOM_HEAT2D_NEUMANN, u_h, tmp_h, al_h, dt=dt_h, n_steps=2)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    crom.crom_fom_step(crom.CROM_FOM_HEAT2D_NEUMANN, u_h, tmp_h, al_h, dt=dt_h, n_steps=fom_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    heat_ms = e0.elapsed_time(e1) / fom_steps
    heat_nodes = nbh * nn * nn
    heat_gbs = heat_nodes * 8 / (heat_ms * 1e-3) / 1e9
    del u_h, tmp_h

    # ---- training step at the learned-model shapes (64 snapshots x 4096 points, width 256, r = 16)
    Bt, St, nt_side, rt, wt, Lt = 64, 4096, 256, 16, 256, 5
    tr = crom.CromTrainer(2, rt, wt, Lt, nt_side * nt_side, Bt, St, local)
    tr.set_params((rng.standard_normal(tr.n_params) * 0.05).astype(np.float32))
    snaps_t = torch.tensor(rng.standard_normal((Bt, nt_side * nt_side)).astype(np.float32), device="cuda")
    idx_t = torch.tensor(np.stack([rng.choice(nt_side * nt_side, size=St, replace=False) for _ in range(Bt)])
                         .astype(np.int32), device="cuda")
    coords_t = torch.tensor(gen.grid_points_2d(nt_side), device="cuda")
    loss_t = torch.zeros(1, dtype=torch.float64, device="cuda")
    def time_train(prec, reps):
        tr.set_precision(prec)
        crom.crom_train_step(tr, snaps_t, idx_t, coords_t, 1e-4, loss_t)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            crom.crom_train_step(tr, snaps_t, idx_t, coords_t, 1e-4, loss_t)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    train_ms_fp32 = time_train(crom.CROM_PREC_FP32, 3)
    train_ms = time_train(crom.CROM_PREC_BF16_MIXED, 10)
    pts = Bt * St
    train_flops = pts * 6 * (2 * (2 + rt) * wt + 2 * (Lt - 1) * wt * wt + 2 * wt) / 2
    train_bytes = (7 * Lt - 3) * pts * wt * 2
    tr.close()

    next_rows = measure_next_rows(crom, gen, ctx, w, q0, alpha, s_off, samples, status, stream, flush, local)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rate1, done, ns, el = cpu_oracle_rate(w, budget_s=8.0)
        pool = OraclePool(w)
        n_all = min(w.n_inst, 16 * pool.cores)
        rate_all, ns_all, el_all = pool.rate(n_all)
        pool.close()
        cpu = {"value": rate_all, "unit": "instance-steps/s", "cores": pool.cores, "kind": "oracle",
               "cpu": cpu_model(),
               "sample": f"FP64 numpy oracle, one step of the first {n_all} instances ({ns_all} samples, "
                         f"{el_all:.1f} s) on {pool.cores} worker processes (one numpy thread each), normalised "
                         f"by the workload's mean |M_i|",
               "single_thread": {"value": rate1, "cores": 1,
                                 "sample": f"one step of the first {done} instances ({ns} samples, {el:.1f} s)"}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "instance-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f16x2 (f16 hi/lo activation operands, f16 weights, f32 accum, f64 solve)",
            "data": "synthetic",
            "config": bench_config(w.n_inst, world, int(w.sizes.sum())),
            "tiles": {"s0": tile_s0, "s1": tile_s1, "autotuned": args.tiles == "auto",
                      "ms_per_step_large_small_s1": [round(tile_ms[0], 4), round(tile_ms[1], 4)]},
            "status_all_ok": bool(np.all(st == 0)),
            "accuracy_vs_fp64_oracle": acc,
            "decode_tc": {"points_per_s": int(w.sizes.sum()) / (dec_ms * 1e-3), "ms": dec_ms,
                          "tflops_algorithmic": dec_flops / (dec_ms * 1e-3) / 1e12,
                          "frac_of_measured_bf16": dec_flops / (dec_ms * 1e-3) / 1e12 / peak_tf,
                          "f16_single_ms": dec_ms_f16,
                          "workload": "crom_decode_tc F16X2: g, dg/dx, Laplacian, dg/dq (r = 8) at the batch's "
                                      "273,723 samples of 1024 instances"},
            "f16_single_step": {"ms_per_step": f16_ms, "value": world * w.n_inst / (f16_ms * 1e-3),
                                "unit": "instance-steps/s",
                                "tflops_algorithmic": flops / (f16_ms * 1e-3) / 1e12,
                                "frac_of_measured_bf16": flops / (f16_ms * 1e-3) / 1e12 / peak_tf,
                                "accuracy_vs_fp64_oracle": f16_acc,
                                "note": "CROM_PREC_F16: activations as single f16 values (tiles of twice the "
                                        "samples per UMMA); per-step errors up to ~10x F16X2's on "
                                        "ill-conditioned decoders, so F16X2 is the headline"},
            "plain_fp32_single": {"value": plain_value, "unit": "instance-steps/s", "us_per_step": plain_ms * 1e3,
                                  "workload": "heat2d_single_M200_r8_w128_L5_gn2 (FP32 CUDA cores)"},
            "speedup_vs_plain_fp32": value / world / plain_value,
            "dense_reconstruction": {"points_per_s": recon_pts / (recon_ms * 1e-3), "ms": recon_ms,
                                     "tflops_algorithmic": recon_flops / (recon_ms * 1e-3) / 1e12,
                                     "frac_of_measured_bf16": recon_flops / (recon_ms * 1e-3) / 1e12 / peak_tf,
                                     "workload": "1024^2 points x 64 codes, F16X2 (f16 hi/lo activations, "
                                                 "f16 hi+lo weights)",
                                     "f16_single_ms": recon_ms_f16,
                                     "f16_single_frac_of_measured_bf16":
                                         recon_flops / (recon_ms_f16 * 1e-3) / 1e12 / peak_tf},
            "graph_rollout": {"value": w.n_inst / (roll_ms * 1e-3), "unit": "instance-steps/s",
                              "ms_per_step": roll_ms, "steps_per_graph": n_roll,
                              "note": "crom_rollout: 1000 steps replayed from a cached CUDA graph, no L2 flush"},
            "fom_advdiff2d": {"node_steps_per_s": fom_nodes / (fom_ms * 1e-3), "ms_per_step": fom_ms,
                              "gbs_algorithmic": fom_gbs, "frac_of_measured_hbm": fom_gbs / hbm,
                              "workload": "512 periodic 256^2 fields, 16 B per node-step (u, ax, ay read, u written)"},
            "next_rows": next_rows,
            "fom_heat2d": {"node_steps_per_s": heat_nodes / (heat_ms * 1e-3), "ms_per_step": heat_ms,
                           "gbs_algorithmic": heat_gbs, "frac_of_measured_hbm": heat_gbs / hbm,
                           "workload": "1024 zero-flux 256^2 fields, 8 B per node-step (u read and written)"},
            "training": {"point_samples_per_s": pts / (train_ms * 1e-3), "ms_per_step": train_ms,
                         "tflops_algorithmic": train_flops / (train_ms * 1e-3) / 1e12,
                         "frac_of_measured_bf16": train_flops / (train_ms * 1e-3) / 1e12 / peak_tf,
                         "hbm_gbs_algorithmic": train_bytes / (train_ms * 1e-3) / 1e9,
                         "frac_of_measured_hbm": train_bytes / (train_ms * 1e-3) / 1e9 / hbm,
                         "bytes_note": "decoder pass: 7 L - 3 reads or writes of a [B*S][w] bf16 array "
                                       "per step (activations, deltas), the roofline that binds here",
                         "precision": "library tcgen05 GEMMs with fused epilogues, bf16 operands, FP32 "
                                      "accumulation and master weights",
                         "fp32_ms_per_step": train_ms_fp32,
                         "workload": "64 snapshots x 4096 points, decoder R^{2+16}->R width 256 x 5 ELU, "
                                     "strided-conv encoder, Adam"},
            "roofline": {"bound": "tensor", "achieved": achieved_tf, "peak": peak_tf, "unit": "TFLOP/s",
                         "frac": achieved_tf / peak_tf,
                         "traffic": STEP_KERNEL_DRAM_BYTES if args.n_inst == 1024 and world == 1 else None,
                         "note": f"step kernel, algorithmic FLOPs {step_flops_per_sample()} per sample x "
                                 f"{int(w.sizes.sum())} samples; peak = {peak_kind} bf16 burst; traffic = "
                                 "dram read+write bytes per launch from one ncu capture of this kernel at this "
                                 "workload"},
            "e2e": {"value": e2e_value, "unit": "instance-steps/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "steps": n_e2e, "status_all_ok": e2e_ok,
                    "call": "crom_step_host (pinned host arrays; copies, step and synchronisation inside the call)"},
            "gpu_launches": 2 * args.steps,
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    ctx.close(); ctx32.close(); ctxr.close()
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
